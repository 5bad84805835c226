// CUDA kernels for sm_103a: the stencil walk of the multipole and monopole
// interaction passes (with the coarse-fine boundary rules on both sides), its
// transposed (adjoint) walk, cell moments with their M2M shift, the L2L
// down-pass and its adjoint, the same passes about explicit (centre-of-mass)
// expansion centres, double-float variants of the forward contractions, and
// the FP64 FMA probe.
//
// Design (B300): the interaction passes are bound by the FP64 FMA pipe, which
// on this part runs at a small fraction of the FP32 rate; memory traffic per
// pair is a few bytes.  So every FP64 operation that is not a contraction FMA
// is moved out of the pair loop:
//   * derivative tensors come from a table of integer offsets (geometric cell
//     centres make D depend on the offset only; the level enters as powers of
//     h applied once per cell);
//   * source moments are pre-scaled once per cell by (-1)^m/m!, the index
//     multiplicity and h^-m, and reduced to 16 traceless combinations;
//   * only the 16 independent Taylor coefficients are accumulated.
// A warp owns 32 target cells of one parity class of one sub-grid, so the
// stencil offset, its table row and the neighbour lookup are warp-uniform;
// integer address arithmetic runs on the integer pipes.
#include <atomic>

#include "ot_internal.h"

namespace otk {

// ---------------------------------------------------------------------------
// double-float arithmetic: a value is an unevaluated sum hi + lo of two FP32
// numbers (|lo| <= ulp(hi)/2, 48 significant bits).  The _rn intrinsics are
// never contracted into FMAs, which the error-free transformations need.
// ---------------------------------------------------------------------------

// s + e = a + b exactly (Knuth's two-sum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (ah, al) += (xh, xl) * (yh, yl), accurate double-word accumulation: the
// high product is split exactly with an FMA, the cross terms and the split's
// error go to the low part (xl * yl is dropped), the high parts are summed by
// two-sum, and (ah, al) is renormalized by a second two-sum, so that
// |al| <= ulp(ah) / 2 after every call.  With u = 2^-24, k calls on one
// accumulator err by at most about (3k + 6) u^2 times the sum of |products|
// (the low-part roundings are u times quantities of order u * |partial sum|).
__device__ __forceinline__ void df_fma(float& ah, float& al, float xh, float xl, float yh, float yl) {
    const float ph = __fmul_rn(xh, yh);
    const float pe = __fmaf_rn(xh, yh, -ph);
    const float pl = __fmaf_rn(xh, yl, __fmaf_rn(xl, yh, pe));
    float sh, se;
    two_sum(ah, ph, sh, se);
    const float t = __fadd_rn(__fadd_rn(al, pl), se);
    two_sum(sh, t, ah, al);
}

// (sh, sl) = (ah, al) + (bh, bl), renormalized
__device__ __forceinline__ void df_add(float ah, float al, float bh, float bl, float& sh, float& sl) {
    float s, e;
    two_sum(ah, bh, s, e);
    e = __fadd_rn(e, __fadd_rn(al, bl));
    sh = __fadd_rn(s, e);
    sl = __fsub_rn(e, __fsub_rn(sh, s));
}

#include "ot_contract.inc"

__device__ __forceinline__ void report(int* status, int code, int item) {
    if (atomicCAS(status, 0, code) == 0) atomicExch(status + 1, item);
}

// 2^e built from its bit pattern (exact; |e| < 1000)
__device__ __forceinline__ double pow2i(int e) {
    return __longlong_as_double(static_cast<long long>(1023 + e) << 52);
}

__device__ __forceinline__ void load_row16(double (&d)[36], const double* __restrict__ Dt, int row) {
    const double2* p = reinterpret_cast<const double2*>(Dt + static_cast<size_t>(row) * DROW);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const double2 v = __ldg(p + i);
        d[2 * i] = v.x;
        d[2 * i + 1] = v.y;
    }
}

__device__ __forceinline__ void load_row(double (&d)[36], const double* __restrict__ Dt, int row) {
    const double2* p = reinterpret_cast<const double2*>(Dt + static_cast<size_t>(row) * DROW);
#pragma unroll
    for (int i = 0; i < 18; ++i) {
        const double2 v = __ldg(p + i);
        d[2 * i] = v.x;
        d[2 * i + 1] = v.y;
    }
}

__device__ __forceinline__ void load_row32f(float (&r)[32], const float* __restrict__ Dt32, int row) {
    const float4* p = reinterpret_cast<const float4*>(Dt32 + static_cast<size_t>(row) * 32);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float4 v = __ldg(p + i);
        r[4 * i] = v.x;
        r[4 * i + 1] = v.y;
        r[4 * i + 2] = v.z;
        r[4 * i + 3] = v.w;
    }
}

__device__ __forceinline__ int offset_row(int ox, int oy, int oz) {
    return (ox + 7) + 15 * (oy + 7) + 225 * (oz + 7);
}

// lane -> local cell of the warp's 32 cells of parity `par`, half `half`
__device__ __forceinline__ void lane_cell(int lane, int par, int half, int& x, int& y, int& z) {
    x = (par & 1) + 2 * (lane & 3);
    y = ((par >> 1) & 1) + 2 * ((lane >> 2) & 3);
    z = ((par >> 2) & 1) + 2 * (2 * half + (lane >> 4));
}

// the same with the item's two halves split along axis `slab` (0 z, 1 x,
// 2 y): the warp's 32 cells are 2 layers of that axis times 4 x 4 of the
// others, all of one parity
__device__ __forceinline__ void lane_cell_slab(int lane, int par, int half, int slab, int& x, int& y, int& z) {
    const int u = lane & 3, v = (lane >> 2) & 3, w = 2 * half + (lane >> 4);
    const int cx = slab == 1 ? w : u, cy = slab == 2 ? w : (slab == 1 ? u : v), cz = slab == 0 ? w : v;
    x = (par & 1) + 2 * cx;
    y = ((par >> 1) & 1) + 2 * cy;
    z = ((par >> 2) & 1) + 2 * cz;
}

// ---------------------------------------------------------------------------
// forward stencil walk
// ---------------------------------------------------------------------------

// point mass of the source at local position s (in [-7, 14]^3) seen through
// neighbour entry e; 0 unless it is a leaf cell or a virtual descendant
__device__ __forceinline__ double source_mass(const FwdParams& p, int2 e, int kind, int sx, int sy, int sz) {
    if (kind == K_LEAF) return __ldg(p.m + static_cast<size_t>(e.x) * NCELL + (sx & 7) + 8 * (sy & 7) + 64 * (sz & 7));
    if (kind == K_VIRT) {
        const unsigned meta = static_cast<unsigned>(e.y);
        const int d = (meta >> 2) & 7;
        const int vx = static_cast<int>(((meta >> 8) & 0xffu) + (sx & 7)) >> d;
        const int vy = static_cast<int>(((meta >> 16) & 0xffu) + (sy & 7)) >> d;
        const int vz = static_cast<int>((meta >> 24) + (sz & 7)) >> d;
        return __ldg(p.m + static_cast<size_t>(e.x) * NCELL + vx + 8 * vy + 64 * vz) * pow2i(-3 * d);
    }
    return 0.0;
}

// the same point mass as a double-float pair (hi, lo) from the split masses
__device__ __forceinline__ void source_mass_df(const FwdParams& p, int2 e, int kind, int sx, int sy, int sz,
                                               float& mh, float& ml) {
    mh = 0.0f;
    ml = 0.0f;
    if (kind == K_LEAF) {
        const float2 v = __ldg(p.mf + static_cast<size_t>(e.x) * NCELL + (sx & 7) + 8 * (sy & 7) + 64 * (sz & 7));
        mh = v.x;
        ml = v.y;
    } else if (kind == K_VIRT) {
        const unsigned meta = static_cast<unsigned>(e.y);
        const int d = (meta >> 2) & 7;
        const int vx = static_cast<int>(((meta >> 8) & 0xffu) + (sx & 7)) >> d;
        const int vy = static_cast<int>(((meta >> 16) & 0xffu) + (sy & 7)) >> d;
        const int vz = static_cast<int>((meta >> 24) + (sz & 7)) >> d;
        const float2 v = __ldg(p.mf + static_cast<size_t>(e.x) * NCELL + vx + 8 * vy + 64 * vz);
        const float sc = __int_as_float((127 - 3 * d) << 23);      // 8^-d exactly
        mh = __fmul_rn(v.x, sc);
        ml = __fmul_rn(v.y, sc);
    }
}

__device__ __forceinline__ void source_moments(const FwdParams& p, int2 e, bool multi, int sx, int sy, int sz,
                                               double (&r)[16]) {
    if (multi) {
        const double* src = p.Mhat + static_cast<size_t>(e.x) * NRED * NCELL + (sx & 7) + 8 * (sy & 7) + 64 * (sz & 7);
#pragma unroll
        for (int q = 0; q < 16; ++q) r[q] = __ldg(src + q * NCELL);
    } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) r[q] = 0.0;
    }
}

__device__ __forceinline__ int checked_kind(const FwdParams& p, int2 e, int item) {
    int kind = e.y & 3;
    if (kind != K_NONE && static_cast<unsigned>(e.x) >= static_cast<unsigned>(p.n_nodes)) {
        report(p.status, 1, item);
        kind = K_NONE;
    }
    return kind;
}

__device__ __forceinline__ int nb_index(int sx, int sy, int sz) {
    return ((sx + 8) >> 3) + 3 * ((sy + 8) >> 3) + 9 * ((sz + 8) >> 3);
}

// ---------------------------------------------------------------------------
// coarse leaf targets next to refined sub-grids
//
// A leaf target cell a whose near source b (offset o) is a cell of a refined
// sub-grid is refined virtually: its 8 children (an eighth of the cell each)
// meet b's 8 children s (offset cs in {0,1}^3; leaf cells one level down) as
// point masses, and a takes the mean of its children's coefficients.  In
// units of the target level's h the child pair (cv, cs) has the table row of
// q - cv, q = 2o + cs, and the child level's h^-(n+1) is 2^(n+1) times the
// target level's, so the mean over the target's children is one row per q:
//   Dv[q][j] = 2^(n_j+1) / 8 * sum_cv row(q - cv)[j],
// and b contributes sum_cs m_s Dv[2o + cs].  The partner source at -o uses
// the same rows with its child 7 - cs and odd orders negated.
// ---------------------------------------------------------------------------

__device__ __forceinline__ int vrow_index(int ox, int oy, int oz, int cs) {
    return (2 * ox + (cs & 1) + 6) + 14 * (2 * oy + ((cs >> 1) & 1) + 6) + 196 * (2 * oz + (cs >> 2) + 6);
}

__device__ __forceinline__ void load_vrow16(double (&d)[36], const double* __restrict__ Dv, int r) {
    const double2* src = reinterpret_cast<const double2*>(Dv + static_cast<size_t>(r) * 16);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const double2 v = __ldg(src + q);
        d[2 * q] = v.x;
        d[2 * q + 1] = v.y;
    }
}

// child cs of the cell at local position (sx, sy, sz) of the refined node
// `node`: returns the child node (or -1 after reporting a bad table entry)
// and its cell
template <class P>
__device__ __forceinline__ int child_cell(const P& p, int node, int sx, int sy, int sz, int cs, int& cell, int item) {
    const int fx = 2 * (sx & 7) + (cs & 1), fy = 2 * (sy & 7) + ((cs >> 1) & 1), fz = 2 * (sz & 7) + (cs >> 2);
    const int c = __ldg(p.child_of + 8 * node + (fx >> 3) + 2 * (fy >> 3) + 4 * (fz >> 3));
    cell = (fx & 7) + 8 * (fy & 7) + 64 * (fz & 7);
    if (static_cast<unsigned>(c) >= static_cast<unsigned>(p.n_nodes)) {
        report(p.status, 5, item);
        return -1;
    }
    return c;
}

// forward: refined near sources at t + o (vp) and t - o (vm) of one entry
__device__ __forceinline__ void refined_near_fwd(const FwdParams& p, int ox, int oy, int oz, int2 ep, bool vp, int px,
                                                 int py, int pz, int2 em, bool vm, int mx, int my, int mz,
                                                 double (&a)[16], int item) {
    const int bx = 2 * (px & 7), by = 2 * (py & 7), bz = 2 * (pz & 7);
    const int cx = 2 * (mx & 7), cy = 2 * (my & 7), cz = 2 * (mz & 7);
    const int* chp = p.child_of + 8 * (vp ? ep.x : 0);
    const int* chm = p.child_of + 8 * (vm ? em.x : 0);
#pragma unroll 1
    for (int cs = 0; cs < 8; ++cs) {
        double mp = 0.0, mm = 0.0;
        if (vp) {
            const int fx = bx + (cs & 1), fy = by + ((cs >> 1) & 1), fz = bz + (cs >> 2);
            const int c = __ldg(chp + (fx >> 3) + 2 * (fy >> 3) + 4 * (fz >> 3));
            if (static_cast<unsigned>(c) < static_cast<unsigned>(p.n_nodes))
                mp = __ldg(p.m + static_cast<size_t>(c) * NCELL + (fx & 7) + 8 * (fy & 7) + 64 * (fz & 7));
            else report(p.status, 5, item);
        }
        if (vm) {
            const int k = 7 - cs;
            const int fx = cx + (k & 1), fy = cy + ((k >> 1) & 1), fz = cz + (k >> 2);
            const int c = __ldg(chm + (fx >> 3) + 2 * (fy >> 3) + 4 * (fz >> 3));
            if (static_cast<unsigned>(c) < static_cast<unsigned>(p.n_nodes))
                mm = __ldg(p.m + static_cast<size_t>(c) * NCELL + (fx & 7) + 8 * (fy & 7) + 64 * (fz & 7));
            else report(p.status, 5, item);
        }
        // even orders take the sum, odd orders the difference (the partner's
        // rows are the same with odd orders negated)
        const double* row = p.Dv + static_cast<size_t>(vrow_index(ox, oy, oz, cs)) * 16;
        const double sm = mp + mm, df = mp - mm;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int n = j == 0 ? 0 : j < 4 ? 1 : j < 9 ? 2 : 3;
            a[j] = fma((n & 1) ? df : sm, __ldg(row + j), a[j]);
        }
    }
}

// the transpose, by target: the children of the refined sources receive
// their share of the target's adjoint by atomic adds
template <class P>
__device__ __forceinline__ void refined_near_scatter(const P& p, int ox, int oy, int oz, int2 ep, bool vp, int px,
                                                     int py, int pz, int2 em, bool vm, int mx, int my, int mz,
                                                     const double (&lb)[16], int item) {
#pragma unroll 1
    for (int cs = 0; cs < 8; ++cs) {
        double d[36];
        load_vrow16(d, p.Dv, vrow_index(ox, oy, oz, cs));
        double e, q;
        ot_mono_adj_split(e, q, lb, d);
        int cell;
        if (vp) {
            const int c = child_cell(p, ep.x, px, py, pz, cs, cell, item);
            if (c >= 0) atomicAdd(p.mbar + static_cast<size_t>(c) * NCELL + cell, e + q);
        }
        if (vm) {
            const int c = child_cell(p, em.x, mx, my, mz, 7 - cs, cell, item);
            if (c >= 0) atomicAdd(p.mbar + static_cast<size_t>(c) * NCELL + cell, e - q);
        }
    }
}

// the order scale 2^(n+1)/8 of the reduced components, for the adjoint
// gather from a coarse leaf's virtual children
__device__ __forceinline__ double vchild_scale(int j) { return j == 0 ? 0.25 : j < 4 ? 0.5 : j < 9 ? 1.0 : 2.0; }

// Double-float accumulators of one lane: the 16 coefficients and, when the
// multipole contractions run in double-float too, the angular term's source
// and target parts.  They move into the FP64 accumulators by groups -- the
// coefficients of orders 0, 1, 2, 3, the angular source part, the angular
// target part -- each as soon as its next entry would take it past DF_MAX
// products since its last move (the error bound of df_fma then stays below
// (3 * 64 + 6) 2^-48 ~ 7e-13 of the sum of |products|).  Per entry a
// multipole source adds 16, 9, 4, 1 products to the four coefficient groups
// (and 7 and 1 to the angular ones), a point mass 1 to each coefficient group.
constexpr int DF_MAX = 64;

struct DFAcc {
    float ah[16], al[16];
    float ch[3], cl[3];
    float th[9], tl[9];
    int cnt[6];
};

__device__ __forceinline__ void df_zero(DFAcc& f) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        f.ah[j] = 0.0f;
        f.al[j] = 0.0f;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        f.ch[i] = 0.0f;
        f.cl[i] = 0.0f;
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        f.th[q] = 0.0f;
        f.tl[q] = 0.0f;
    }
#pragma unroll
    for (int g = 0; g < 6; ++g) f.cnt[g] = 0;
}

template <int LO, int HI>
__device__ __forceinline__ void df_move(double* a, float* h, float* l) {
#pragma unroll
    for (int j = LO; j < HI; ++j) {
        a[j] += static_cast<double>(h[j]) + static_cast<double>(l[j]);
        h[j] = 0.0f;
        l[j] = 0.0f;
    }
}

// make room for an entry adding inc[g] products to group g.  The counts are
// warp-uniform; the __syncwarp() keeps each move a real (rarely taken) branch:
// if-converted into predicated code, the moves' FP64 conversions and adds
// would issue on the FP64 pipe at every entry.
__device__ __forceinline__ void df_reserve(double (&a)[16], double (&c)[3], double (&t4)[9], DFAcc& f, int i0, int i1,
                                           int i2, int i3, int i4, int i5) {
    if (f.cnt[0] + i0 > DF_MAX) { __syncwarp(); df_move<0, 1>(a, f.ah, f.al); f.cnt[0] = 0; }
    if (f.cnt[1] + i1 > DF_MAX) { __syncwarp(); df_move<1, 4>(a, f.ah, f.al); f.cnt[1] = 0; }
    if (f.cnt[2] + i2 > DF_MAX) { __syncwarp(); df_move<4, 9>(a, f.ah, f.al); f.cnt[2] = 0; }
    if (f.cnt[3] + i3 > DF_MAX) { __syncwarp(); df_move<9, 16>(a, f.ah, f.al); f.cnt[3] = 0; }
    if (f.cnt[4] + i4 > DF_MAX) { __syncwarp(); df_move<0, 3>(c, f.ch, f.cl); f.cnt[4] = 0; }
    if (f.cnt[5] + i5 > DF_MAX) { __syncwarp(); df_move<0, 9>(t4, f.th, f.tl); f.cnt[5] = 0; }
    f.cnt[0] += i0;
    f.cnt[1] += i1;
    f.cnt[2] += i2;
    f.cnt[3] += i3;
    f.cnt[4] += i4;
    f.cnt[5] += i5;
}

template <bool ANG>
__device__ __forceinline__ void df_flush_all(double (&a)[16], double (&c)[3], double (&t4)[9], DFAcc& f) {
    df_move<0, 16>(a, f.ah, f.al);
    if (ANG) {
        df_move<0, 3>(c, f.ch, f.cl);
        df_move<0, 9>(t4, f.th, f.tl);
    }
#pragma unroll
    for (int g = 0; g < 6; ++g) f.cnt[g] = 0;
}

// reduced moments of a multipole source as double-float pairs
__device__ __forceinline__ void source_moments_df(const FwdParams& p, int2 e, bool multi, int sx, int sy, int sz,
                                                  float (&rh)[16], float (&rl)[16]) {
    if (multi) {
        const float2* src = p.Mf + static_cast<size_t>(e.x) * NRED * NCELL + (sx & 7) + 8 * (sy & 7) + 64 * (sz & 7);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const float2 v = __ldg(src + q * NCELL);
            rh[q] = v.x;
            rl[q] = v.y;
        }
    } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            rh[q] = 0.0f;
            rl[q] = 0.0f;
        }
    }
}

// PAIRED: each entry o stands for the offsets o and -o (sources at t + o and
// t - o share the table row of o, with odd-order derivatives negated for -o).
// EMU bits: 1 point-mass contractions in double-float (the partial sums in
// DFAcc), 2 multipole ones too
// ---------------------------------------------------------------------------
// point masses by reflection class (leaf targets)
//
// The sources at t + s*o (s in {+1, -1}^3 per axis, o = (a, b, c) >= 0) share
// one table row up to signs: D^(kx,ky,kz) at -s*o is sx^kx sy^ky sz^kz times
// its value at -o, since G is even in every coordinate.  So a target adds
// row_q * W[pi(q)] to reduced coefficient q, W the Walsh-Hadamard transform
// of the members' masses over the sign axes, W[pi] = sum_i (-1)^|i & pi| m_i
// (member i negated on the axes set in i), pi(q) the parity pattern of q.
// Eight point-mass pairs then cost 24 adds + 16 FMAs instead of four +-o
// entries of 2 adds + 16 FMAs each.  An axis with o = 0 holds one member and
// no odd orders on it (their table entries are exactly zero): class Z skips
// those axes and components.  The adjoint by target is the transpose: the
// partial dot products of L-bar and the row by parity pattern, transformed
// the same way (the transform is symmetric), give each member's share.
// ---------------------------------------------------------------------------

template <int Z>
__device__ __forceinline__ void class_transform(double (&w)[8]) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        if ((Z >> b) & 1) continue;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (((i >> b) & 1) || (i & Z)) continue;
            const double u = w[i], v = w[i | (1 << b)];
            w[i] = u + v;
            w[i | (1 << b)] = u - v;
        }
    }
}

// local position of member i of class (a, b, c) seen from target t
__device__ __forceinline__ void class_member(int i, int a, int b, int c, int tx, int ty, int tz, int& sx, int& sy,
                                             int& sz) {
    sx = (i & 1) ? tx - a : tx + a;
    sy = (i & 2) ? ty - b : ty + b;
    sz = (i & 4) ? tz - c : tz + c;
}

template <int Z>
__device__ __forceinline__ void walk_classes_fwd(const int* __restrict__ list, int len, int tx, int ty, int tz,
                                                 const int2* __restrict__ s_nb, const FwdParams& p,
                                                 double (&acc)[16], int item) {
    for (int k = 0; k < len; ++k) {
        const int e = __ldg(list + k);
        const int a = e & 0xff, b = (e >> 8) & 0xff, c = (e >> 16) & 0xff;
        const unsigned members = static_cast<unsigned>(e) >> 24;
        double w[8];
        bool any = false;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            w[i] = 0.0;
            if (i & Z) continue;
            if ((members >> i) & 1u) {
                int sx, sy, sz;
                class_member(i, a, b, c, tx, ty, tz, sx, sy, sz);
                const int2 es = s_nb[nb_index(sx, sy, sz)];
                const int ks = checked_kind(p, es, item);
                any |= ks >= K_LEAF;
                w[i] = source_mass(p, es, ks, sx, sy, sz);
            }
        }
        if (!__any_sync(0xffffffffu, any)) continue;
        double d[36];
        load_row16(d, p.Dt, offset_row(a, b, c));
        class_transform<Z>(w);
#pragma unroll
        for (int q = 0; q < 16; ++q)
            if (!(comp_parity(q) & Z)) acc[q] = fma(w[comp_parity(q)], d[q], acc[q]);
    }
}

// the transform stages after the x stage (y and z axes not in Z)
template <int Z>
__device__ __forceinline__ void class_transform_yz(double (&w)[8]) {
#pragma unroll
    for (int b = 1; b < 3; ++b) {
        if ((Z >> b) & 1) continue;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (((i >> b) & 1) || (i & Z)) continue;
            const double u = w[i], v = w[i | (1 << b)];
            w[i] = u + v;
            w[i | (1 << b)] = u - v;
        }
    }
}

// x-complete point-mass classes of a node whose neighbours are all leaf or
// empty: the first transform stage comes from the prebuilt x butterflies of
// the masses at the positions t + (0, +-b, +-c)
template <int Z>
__device__ __forceinline__ void walk_classes_fwd_x(const int* __restrict__ list, int len, int tx, int ty, int tz,
                                                   const int2* __restrict__ s_nb, const int* __restrict__ s_sl, const FwdParams& p,
                                                   double (&acc)[16], int item) {
    static_assert((Z & 1) == 0, "the x stage needs a > 0");
    for (int k = 0; k < len; ++k) {
        const int e = __ldg(list + k);
        const int a = e & 0xff, b = (e >> 8) & 0xff, c = (e >> 16) & 0xff;
        const unsigned members = static_cast<unsigned>(e) >> 24;
        double w[8];
        bool any = false;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            w[2 * q] = 0.0;
            w[2 * q + 1] = 0.0;
            if ((2 * q) & Z) continue;
            if ((members >> (2 * q)) & 1u) {
                const int sy = (q & 1) ? ty - b : ty + b, sz = (q & 2) ? tz - c : tz + c;
                const int nbi = nb_index(tx, sy, sz);
                const int ks = checked_kind(p, s_nb[nbi], item);
                const int slot = s_sl[nbi];
                if (slot >= 0) {
                    const double* src = p.Sm + static_cast<size_t>(slot * 7 + a - 1) * 2 * NCELL +
                                        (tx & 7) + 8 * (sy & 7) + 64 * (sz & 7);
                    w[2 * q] = __ldg(src);
                    w[2 * q + 1] = __ldg(src + NCELL);
                    any = true;
                } else if (ks != K_NONE) {
                    report(p.status, 7, item);    // the node's flag promised a table slot for every region
                }
            }
        }
        if (!__any_sync(0xffffffffu, any)) continue;
        double d[36];
        load_row16(d, p.Dt, offset_row(a, b, c));
        class_transform_yz<Z>(w);
#pragma unroll
        for (int q = 0; q < 16; ++q)
            if (!(comp_parity(q) & Z)) acc[q] = fma(w[comp_parity(q)], d[q], acc[q]);
    }
}

// Double-float point-mass classes (EMU bit 1): the members' masses as
// (hi, lo) pairs, the transform by df_add, one df_fma per component into the
// double-float accumulators.  The transform of up to eight masses errs by at
// most 3 * 2^-48 of the sum of their magnitudes, so a product's error stays
// within a few 2^-48 of the |terms| its members stand for, inside the grouped
// accumulation's bound.
template <int Z, int B0>
__device__ __forceinline__ void class_transform_df(float (&wh)[8], float (&wl)[8]) {
#pragma unroll
    for (int b = B0; b < 3; ++b) {
        if ((Z >> b) & 1) continue;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (((i >> b) & 1) || (i & Z)) continue;
            const int j = i | (1 << b);
            float sh, sl, dh, dl;
            df_add(wh[i], wl[i], wh[j], wl[j], sh, sl);
            df_add(wh[i], wl[i], -wh[j], -wl[j], dh, dl);
            wh[i] = sh;
            wl[i] = sl;
            wh[j] = dh;
            wl[j] = dl;
        }
    }
}

template <int Z>
__device__ __forceinline__ void class_fma_df(DFAcc& f, const float (&wh)[8], const float (&wl)[8],
                                             const float (&r)[32]) {
#pragma unroll
    for (int q = 0; q < 16; ++q)
        if (!(comp_parity(q) & Z)) df_fma(f.ah[q], f.al[q], wh[comp_parity(q)], wl[comp_parity(q)], r[q], r[16 + q]);
}

template <int Z>
__device__ __forceinline__ void walk_classes_fwd_df(const int* __restrict__ list, int len, int tx, int ty, int tz,
                                                    const int2* __restrict__ s_nb, const FwdParams& p,
                                                    double (&acc)[16], double (&c)[3], double (&t4)[9], DFAcc& f,
                                                    int item) {
    for (int k = 0; k < len; ++k) {
        const int e = __ldg(list + k);
        const int a = e & 0xff, b = (e >> 8) & 0xff, cc = (e >> 16) & 0xff;
        const unsigned members = static_cast<unsigned>(e) >> 24;
        float wh[8], wl[8];
        bool any = false;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            wh[i] = 0.0f;
            wl[i] = 0.0f;
            if (i & Z) continue;
            if ((members >> i) & 1u) {
                int sx, sy, sz;
                class_member(i, a, b, cc, tx, ty, tz, sx, sy, sz);
                const int2 es = s_nb[nb_index(sx, sy, sz)];
                const int ks = checked_kind(p, es, item);
                any |= ks >= K_LEAF;
                source_mass_df(p, es, ks, sx, sy, sz, wh[i], wl[i]);
            }
        }
        if (!__any_sync(0xffffffffu, any)) continue;
        df_reserve(acc, c, t4, f, 1, 1, 1, 1, 0, 0);
        float r[32];
        load_row32f(r, p.Dt32, offset_row(a, b, cc));
        class_transform_df<Z, 0>(wh, wl);
        class_fma_df<Z>(f, wh, wl, r);
    }
}

// the same with the x stage from the prebuilt x butterflies of the masses,
// split into (hi, lo) pairs
template <int Z>
__device__ __forceinline__ void walk_classes_fwd_df_x(const int* __restrict__ list, int len, int tx, int ty, int tz,
                                                      const int2* __restrict__ s_nb, const int* __restrict__ s_sl, const FwdParams& p,
                                                      double (&acc)[16], double (&c)[3], double (&t4)[9], DFAcc& f,
                                                      int item) {
    static_assert((Z & 1) == 0, "the x stage needs a > 0");
    for (int k = 0; k < len; ++k) {
        const int e = __ldg(list + k);
        const int a = e & 0xff, b = (e >> 8) & 0xff, cc = (e >> 16) & 0xff;
        const unsigned members = static_cast<unsigned>(e) >> 24;
        float wh[8], wl[8];
        bool any = false;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            wh[2 * q] = wl[2 * q] = wh[2 * q + 1] = wl[2 * q + 1] = 0.0f;
            if ((2 * q) & Z) continue;
            if ((members >> (2 * q)) & 1u) {
                const int sy = (q & 1) ? ty - b : ty + b, sz = (q & 2) ? tz - cc : tz + cc;
                const int nbi = nb_index(tx, sy, sz);
                const int ks = checked_kind(p, s_nb[nbi], item);
                const int slot = s_sl[nbi];
                if (slot >= 0) {
                    const float2* src = p.Smf + static_cast<size_t>(slot * 7 + a - 1) * 2 * NCELL +
                                        (tx & 7) + 8 * (sy & 7) + 64 * (sz & 7);
                    const float2 vp = __ldg(src), vm = __ldg(src + NCELL);
                    wh[2 * q] = vp.x;
                    wl[2 * q] = vp.y;
                    wh[2 * q + 1] = vm.x;
                    wl[2 * q + 1] = vm.y;
                    any = true;
                } else if (ks != K_NONE) {
                    report(p.status, 7, item);
                }
            }
        }
        if (!__any_sync(0xffffffffu, any)) continue;
        df_reserve(acc, c, t4, f, 1, 1, 1, 1, 0, 0);
        float r[32];
        load_row32f(r, p.Dt32, offset_row(a, b, cc));
        class_transform_df<Z, 1>(wh, wl);
        class_fma_df<Z>(f, wh, wl, r);
    }
}

template <int Z = 0, class CH>
__device__ __forceinline__ void walk_classes_fwd_df_all(const int* __restrict__ list, const int* zoff, const int* xc,
                                                        bool xpath, const CH& ch, int tx, int ty, int tz,
                                                        const int2* __restrict__ s_nb, const int* __restrict__ s_sl, const FwdParams& p,
                                                        double (&acc)[16], double (&c)[3], double (&t4)[9], DFAcc& f,
                                                        int item) {
    const int len = zoff[Z + 1] - zoff[Z];
    int nx = 0;
    if constexpr ((Z & 1) == 0) {
        if (xpath) {
            nx = xc[Z];
            walk_classes_fwd_df_x<Z>(list + zoff[Z] + ch.lo(nx), ch.n(nx), tx, ty, tz, s_nb, s_sl, p, acc, c, t4, f, item);
        }
    }
    // targets without x tables run their classes by the FP64 walk: in
    // double-float their transform and loads cost more issue slots and
    // instruction-cache room than the FP64 pipe time they save
    if (xpath)
        walk_classes_fwd_df<Z>(list + zoff[Z] + nx + ch.lo(len - nx), ch.n(len - nx), tx, ty, tz, s_nb, p, acc, c, t4,
                               f, item);
    else
        walk_classes_fwd<Z>(list + zoff[Z] + nx + ch.lo(len - nx), ch.n(len - nx), tx, ty, tz, s_nb, p, acc, item);
    if constexpr (Z < 6)
        walk_classes_fwd_df_all<Z + 1>(list, zoff, xc, xpath, ch, tx, ty, tz, s_nb, s_sl, p, acc, c, t4, f, item);
}

// xy-complete point-mass classes (a, b > 0) of a leaf target with leaf or
// empty neighbours: the first two transform stages come from the (x, y)
// table at the positions t + (0, 0, +-c).  The walk is software-pipelined:
// the next entry's table values are requested before this entry's
// transform and FMAs, so their latency (the table streams from DRAM)
// overlaps the FP64 work.
template <int Z>
__device__ __forceinline__ bool xy_fetch(int e, int tx, int ty, int tz, const int2* __restrict__ s_nb,
                                         const int* __restrict__ s_sl, const FwdParams& p, double (&w)[8],
                                         int item) {
    const int a = e & 0xff, b = (e >> 8) & 0xff, c = (e >> 16) & 0xff;
    const unsigned members = static_cast<unsigned>(e) >> 24;
    bool any = false;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
#pragma unroll
        for (int q = 0; q < 4; ++q) w[4 * r + q] = 0.0;
        if ((4 * r) & Z) continue;
        if ((members >> (4 * r)) & 1u) {
            const int sz = r ? tz - c : tz + c;
            const int nbi = nb_index(tx, ty, sz);
            const int ks = checked_kind(p, s_nb[nbi], item);
            const int slot = s_sl[nbi];
            if (slot >= 0) {
                const double* src = p.Sxy + static_cast<size_t>(slot * 49 + (a - 1) * 7 + b - 1) * 4 * NCELL +
                                    (tx & 7) + 8 * (ty & 7) + 64 * (sz & 7);
#pragma unroll
                for (int q = 0; q < 4; ++q) w[4 * r + q] = __ldg(src + q * NCELL);
                any = true;
            } else if (ks != K_NONE) {
                report(p.status, 7, item);
            }
        }
    }
    return any;
}

template <int Z>
__device__ __forceinline__ void walk_classes_fwd_xy(const int* __restrict__ list, int len, int tx, int ty, int tz,
                                                    const int2* __restrict__ s_nb, const int* __restrict__ s_sl,
                                                    const FwdParams& p, double (&acc)[16], int item) {
    static_assert((Z & 3) == 0, "the x and y stages need a, b > 0");
    if (len <= 0) return;
    int en = __ldg(list);
    double wn[8];
    bool anyn = xy_fetch<Z>(en, tx, ty, tz, s_nb, s_sl, p, wn, item);
    for (int k = 0; k < len; ++k) {
        const int e = en;
        double w[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) w[q] = wn[q];
        const bool any = anyn;
        if (k + 1 < len) {
            en = __ldg(list + k + 1);
            anyn = xy_fetch<Z>(en, tx, ty, tz, s_nb, s_sl, p, wn, item);
        }
        if (!__any_sync(0xffffffffu, any)) continue;
        const int a = e & 0xff, b = (e >> 8) & 0xff, c = (e >> 16) & 0xff;
        double d[36];
        load_row16(d, p.Dt, offset_row(a, b, c));
        if constexpr (!(Z & 4)) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const double u = w[i], v = w[i | 4];
                w[i] = u + v;
                w[i | 4] = u - v;
            }
        }
#pragma unroll
        for (int q = 0; q < 16; ++q)
            if (!(comp_parity(q) & Z)) acc[q] = fma(w[comp_parity(q)], d[q], acc[q]);
    }
}

// the seven zero patterns of a class list (Z = 7 would be the self pair);
// with xpath, each group's x-complete head (xc[Z] entries, Z without bit 0)
// takes the prebuilt x butterflies
template <int Z = 0, class CH>
__device__ __forceinline__ void walk_classes_fwd_all(const int* __restrict__ list, const int* zoff, const int* xc,
                                                     const int* xyc, bool xpath, const CH& ch, int tx, int ty, int tz,
                                                     const int2* __restrict__ s_nb, const int* __restrict__ s_sl, const FwdParams& p,
                                                     double (&acc)[16], int item) {
    const int len = zoff[Z + 1] - zoff[Z];
    int nx = 0;
    if constexpr ((Z & 1) == 0) {
        if (xpath) {
            int nxy = 0;
            if constexpr ((Z & 2) == 0) {
                if (p.Sxy != nullptr) {
                    nxy = xyc[Z];
                    walk_classes_fwd_xy<Z>(list + zoff[Z] + ch.lo(nxy), ch.n(nxy), tx, ty, tz, s_nb, s_sl, p, acc, item);
                }
            }
            nx = xc[Z];
            walk_classes_fwd_x<Z>(list + zoff[Z] + nxy + ch.lo(nx - nxy), ch.n(nx - nxy), tx, ty, tz, s_nb, s_sl, p,
                                  acc, item);
        }
    }
    walk_classes_fwd<Z>(list + zoff[Z] + nx + ch.lo(len - nx), ch.n(len - nx), tx, ty, tz, s_nb, p, acc, item);
    if constexpr (Z < 6) walk_classes_fwd_all<Z + 1>(list, zoff, xc, xyc, xpath, ch, tx, ty, tz, s_nb, s_sl, p, acc, item);
}

// multipole sources by reflection class (non-leaf targets): the members'
// reduced moments feed the class contraction (see gen_contract.py), which
// transforms them over the sign axes component by component
template <int Z, bool ANG>
__device__ __forceinline__ void walk_mclasses_fwd(const int* __restrict__ list, int len, int tx, int ty, int tz,
                                                  const int2* __restrict__ s_nb, const FwdParams& p,
                                                  double (&acc)[16], double (&c)[3], double (&t4)[9], int item) {
    for (int k = 0; k < len; ++k) {
        const int e = __ldg(list + k);
        const int ox = e & 0xff, oy = (e >> 8) & 0xff, oz = (e >> 16) & 0xff;
        const unsigned members = static_cast<unsigned>(e) >> 24;
        const double* src[8];
        bool any = false;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            src[i] = nullptr;
            if (i & Z) continue;
            if ((members >> i) & 1u) {
                int sx, sy, sz;
                class_member(i, ox, oy, oz, tx, ty, tz, sx, sy, sz);
                const int2 es = s_nb[nb_index(sx, sy, sz)];
                if (checked_kind(p, es, item) == K_MULTI) {
                    src[i] = p.Mhat + static_cast<size_t>(es.x) * NRED * NCELL + (sx & 7) + 8 * (sy & 7) + 64 * (sz & 7);
                    any = true;
                }
            }
        }
        if (!__any_sync(0xffffffffu, any)) continue;
        ot_mclass_fwd<Z, ANG>(acc, c, t4, src, p.Dt + static_cast<size_t>(offset_row(ox, oy, oz)) * DROW);
    }
}

// x-complete multipole classes of a node whose neighbours are all multipole
// or empty: the first transform stage of every source component comes from
// the prebuilt x butterflies at the positions t + (0, +-b, +-c)
template <int Z, bool ANG>
__device__ __forceinline__ void walk_mclasses_fwd_x(const int* __restrict__ list, int len, int tx, int ty, int tz,
                                                    const int2* __restrict__ s_nb, const int* __restrict__ s_sl, const FwdParams& p,
                                                    double (&acc)[16], double (&c)[3], double (&t4)[9], int item) {
    static_assert((Z & 1) == 0, "the x stage needs a > 0");
    for (int k = 0; k < len; ++k) {
        const int e = __ldg(list + k);
        const int ox = e & 0xff, oy = (e >> 8) & 0xff, oz = (e >> 16) & 0xff;
        const unsigned members = static_cast<unsigned>(e) >> 24;
        const double* pos[4];
        bool any = false;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            pos[q] = nullptr;
            if ((2 * q) & Z) continue;
            if ((members >> (2 * q)) & 1u) {
                const int sy = (q & 1) ? ty - oy : ty + oy, sz = (q & 2) ? tz - oz : tz + oz;
                const int nbi = nb_index(tx, sy, sz);
                const int ks = checked_kind(p, s_nb[nbi], item);
                const int slot = s_sl[nbi];
                if (slot >= 0) {
                    pos[q] = p.Sx + static_cast<size_t>(slot * 7 + ox - 1) * 32 * NCELL + (tx & 7) +
                             8 * (sy & 7) + 64 * (sz & 7);
                    any = true;
                } else if (ks != K_NONE) {
                    report(p.status, 7, item);    // the node's flag promised a table slot for every region
                }
            }
        }
        if (!__any_sync(0xffffffffu, any)) continue;
        ot_mclass_fwd_x<Z, ANG>(acc, c, t4, pos, p.Dt + static_cast<size_t>(offset_row(ox, oy, oz)) * DROW);
    }
}

// xy-complete multipole classes (a, b > 0) of a node whose neighbours are
// all multipole or empty: the first two transform stages of every source
// component come from the moments' (x, y) table at the positions
// t + (0, 0, +-c)
template <int Z, bool ANG>
__device__ __forceinline__ void walk_mclasses_fwd_xy(const int* __restrict__ list, int len, int tx, int ty, int tz,
                                                     const int2* __restrict__ s_nb, const int* __restrict__ s_sl,
                                                     const FwdParams& p, double (&acc)[16], double (&c)[3],
                                                     double (&t4)[9], int item) {
    static_assert((Z & 3) == 0, "the x and y stages need a, b > 0");
    for (int k = 0; k < len; ++k) {
        const int e = __ldg(list + k);
        const int ox = e & 0xff, oy = (e >> 8) & 0xff, oz = (e >> 16) & 0xff;
        const unsigned members = static_cast<unsigned>(e) >> 24;
        const double* pos[2];
        bool any = false;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            pos[r] = nullptr;
            if ((4 * r) & Z) continue;
            if ((members >> (4 * r)) & 1u) {
                const int sz = r ? tz - oz : tz + oz;
                const int nbi = nb_index(tx, ty, sz);
                const int ks = checked_kind(p, s_nb[nbi], item);
                const int slot = s_sl[nbi];
                if (slot >= 0) {
                    pos[r] = p.Sxym + (static_cast<size_t>((slot * 49 + (ox - 1) * 7 + oy - 1) * 16) * NCELL +
                                       (tx & 7) + 8 * (ty & 7) + 64 * (sz & 7)) * 4;
                    any = true;
                } else if (ks != K_NONE) {
                    report(p.status, 7, item);    // the node's flag promised a table slot for every region
                }
            }
        }
        if (!__any_sync(0xffffffffu, any)) continue;
        ot_mclass_fwd_xy<Z, ANG>(acc, c, t4, pos, p.Dt + static_cast<size_t>(offset_row(ox, oy, oz)) * DROW);
    }
}

template <bool ANG, int Z = 0, class CH>
__device__ __forceinline__ void walk_mclasses_fwd_all(const int* __restrict__ list, const int (&zoff)[8],
                                                      const int (&xc)[8], const int (&xyc)[8], bool xpath,
                                                      const CH& ch, int tx, int ty, int tz,
                                                      const int2* __restrict__ s_nb, const int* __restrict__ s_sl,
                                                      const FwdParams& p, double (&acc)[16], double (&c)[3],
                                                      double (&t4)[9], int item) {
    const int len = zoff[Z + 1] - zoff[Z];
    int nx = 0;
    if constexpr ((Z & 1) == 0) {
        if (xpath) {
            int nxy = 0;
            if constexpr ((Z & 2) == 0) {
                if (p.Sxym != nullptr) {
                    nxy = xyc[Z];
                    walk_mclasses_fwd_xy<Z, ANG>(list + zoff[Z] + ch.lo(nxy), ch.n(nxy), tx, ty, tz, s_nb, s_sl, p,
                                                 acc, c, t4, item);
                }
            }
            nx = xc[Z];
            walk_mclasses_fwd_x<Z, ANG>(list + zoff[Z] + nxy + ch.lo(nx - nxy), ch.n(nx - nxy), tx, ty, tz, s_nb,
                                        s_sl, p, acc, c, t4, item);
        }
    }
    walk_mclasses_fwd<Z, ANG>(list + zoff[Z] + nx + ch.lo(len - nx), ch.n(len - nx), tx, ty, tz, s_nb, p, acc, c, t4,
                              item);
    if constexpr (Z < 6)
        walk_mclasses_fwd_all<ANG, Z + 1>(list, zoff, xc, xyc, xpath, ch, tx, ty, tz, s_nb, s_sl, p, acc, c, t4,
                                          item);
}

template <int MODE, bool PAIRED, int EMU, bool NEAR = false, bool PM = true, bool NEG = false>
__device__ __forceinline__ void walk_forward(const int* __restrict__ list, int len, bool angular,
                                             int tx, int ty, int tz, const int2* __restrict__ s_nb,
                                             const FwdParams& p, double (&a)[16], double (&c)[3],
                                             double (&t4)[9], DFAcc& f, int item) {
    for (int k = 0; k < len; ++k) {
        const int po = __ldg(list + k);
        // NEG (single walks only): the list's offsets negated, the other
        // members of its +-o pairs
        const int sg = NEG ? -1 : 1;
        const int ox = sg * ((po & 0xff) - 8), oy = sg * (((po >> 8) & 0xff) - 8), oz = sg * (((po >> 16) & 0xff) - 8);
        const int px = tx + ox, py = ty + oy, pz = tz + oz;   // in [-7, 14]
        const int mx = tx - ox, my = ty - oy, mz = tz - oz;
        const int2 ep = s_nb[nb_index(px, py, pz)];
        const int kp = checked_kind(p, ep, item);
        int2 em = make_int2(-1, 0);
        int km = K_NONE;
        if (PAIRED) {
            em = s_nb[nb_index(mx, my, mz)];
            km = checked_kind(p, em, item);
        }
        const int row = offset_row(ox, oy, oz);
        if ((MODE & 2) && PM) {
            const bool mono = kp >= K_LEAF || km >= K_LEAF;
            if (__any_sync(0xffffffffu, mono)) {
                if (EMU & 1) {
                    df_reserve(a, c, t4, f, 1, 1, 1, 1, 0, 0);
                    float mh, ml;
                    source_mass_df(p, ep, kp, px, py, pz, mh, ml);
                    float r[32];
                    load_row32f(r, p.Dt32, row);
                    if (PAIRED) {
                        float nh, nl, sh, sl, dh, dl;
                        source_mass_df(p, em, km, mx, my, mz, nh, nl);
                        df_add(mh, ml, nh, nl, sh, sl);
                        df_add(mh, ml, -nh, -nl, dh, dl);
                        ot_mono_fwd_pair_df(f.ah, f.al, sh, sl, dh, dl, r);
                    } else {
                        ot_mono_fwd_df(f.ah, f.al, mh, ml, r);
                    }
                } else {
                    const double mp = source_mass(p, ep, kp, px, py, pz);
                    double d[36];
                    load_row16(d, p.Dt, row);
                    if (PAIRED) {
                        const double mm = source_mass(p, em, km, mx, my, mz);
                        ot_mono_fwd_pair(a, mp + mm, mp - mm, d);
                    } else {
                        ot_mono_fwd(a, mp, d);
                    }
                }
            }
        }
        if ((MODE & 2) && NEAR) {
            // near sources in refined sub-grids: the target refined virtually
            const bool rp = kp == K_MULTI, rm = km == K_MULTI;
            if (__any_sync(0xffffffffu, rp || rm))
                refined_near_fwd(p, ox, oy, oz, ep, rp, px, py, pz, em, rm, mx, my, mz, a, item);
        }
        if ((MODE & 1) && !NEAR && (EMU & 2)) {
            const bool multi = kp == K_MULTI || km == K_MULTI;
            if (__any_sync(0xffffffffu, multi)) {
                df_reserve(a, c, t4, f, 16, 9, 4, 1, angular ? 7 : 0, angular ? 1 : 0);
                float rh[16], rl[16];
                source_moments_df(p, ep, kp == K_MULTI, px, py, pz, rh, rl);
                const float2* drow = p.Dt2 + static_cast<size_t>(row) * DROW;
                if (PAIRED) {
                    float mh[16], ml[16];
                    source_moments_df(p, em, km == K_MULTI, mx, my, mz, mh, ml);
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        float sh, sl, dh, dl;
                        df_add(rh[q], rl[q], mh[q], ml[q], sh, sl);       // sum
                        df_add(rh[q], rl[q], -mh[q], -ml[q], dh, dl);     // difference
                        rh[q] = sh;
                        rl[q] = sl;
                        mh[q] = dh;
                        ml[q] = dl;
                    }
                    ot_multi_fwd_pair_df(f.ah, f.al, rh, rl, mh, ml, drow);
                } else {
                    ot_multi_fwd_df(f.ah, f.al, rh, rl, drow);
                }
                if (angular) ot_angular_fwd_df(f.ch, f.cl, f.th, f.tl, rh, rl, drow);
            }
        }
        if ((MODE & 1) && !NEAR && !(EMU & 2)) {
            const bool multi = kp == K_MULTI || km == K_MULTI;
            if (__any_sync(0xffffffffu, multi)) {
                double r[16];
                source_moments(p, ep, kp == K_MULTI, px, py, pz, r);
                double d[36];
                load_row(d, p.Dt, row);
                if (PAIRED) {
                    double rm[16];
                    source_moments(p, em, km == K_MULTI, mx, my, mz, rm);
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const double t = r[q];
                        r[q] = t + rm[q];     // sum
                        rm[q] = t - rm[q];    // difference
                    }
                    ot_multi_fwd_pair(a, r, rm, d);
                } else {
                    ot_multi_fwd(a, r, d);
                }
                if (angular) ot_angular_fwd(c, t4, r, r[0], d);
            }
        }
    }
}

// a leaf target's multipole sources (cells of refined neighbours) by its
// axis-pair list: an entry o pairs with o reflected along axis A.  Where
// some lane has a multipole source at both members the two share the row of
// o through the sum and the difference of their moments (d^K G at the
// reflection is (-1)^{K_A} d^K G(o)); where only one member has one in some
// lane it runs alone with its own row; otherwise the entry is skipped
template <int A>
__device__ __forceinline__ void walk_multi_apairs(const int* __restrict__ list, int len, bool paired, int tx,
                                                  int ty, int tz, const int2* __restrict__ s_nb,
                                                  const FwdParams& p, double (&a)[16], int item) {
    for (int k = 0; k < len; ++k) {
        const int po = __ldg(list + k);
        const int ox = (po & 0xff) - 8, oy = ((po >> 8) & 0xff) - 8, oz = ((po >> 16) & 0xff) - 8;
        const int rx = A == 0 ? -ox : ox, ry = A == 1 ? -oy : oy, rz = A == 2 ? -oz : oz;
        const int px = tx + ox, py = ty + oy, pz = tz + oz;
        const int qx = tx + rx, qy = ty + ry, qz = tz + rz;
        const int2 e1 = s_nb[nb_index(px, py, pz)];
        const bool v1 = checked_kind(p, e1, item) == K_MULTI;
        int2 e2 = make_int2(-1, 0);
        bool v2 = false;
        if (paired) {
            e2 = s_nb[nb_index(qx, qy, qz)];
            v2 = checked_kind(p, e2, item) == K_MULTI;
        }
        const bool a1 = __any_sync(0xffffffffu, v1), a2 = __any_sync(0xffffffffu, v2);
        if (!a1 && !a2) continue;
        double r[16];
        double d[36];
        if (a1 && a2) {
            double rm[16];
            source_moments(p, e1, v1, px, py, pz, r);
            source_moments(p, e2, v2, qx, qy, qz, rm);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const double t = r[q];
                r[q] = t + rm[q];     // sum
                rm[q] = t - rm[q];    // difference
            }
            load_row(d, p.Dt, offset_row(ox, oy, oz));
            if constexpr (A == 0) ot_multi_fwd_xpair(a, r, rm, d);
            else if constexpr (A == 1) ot_multi_fwd_ypair(a, r, rm, d);
            else ot_multi_fwd_zpair(a, r, rm, d);
        } else if (a1) {
            source_moments(p, e1, v1, px, py, pz, r);
            load_row(d, p.Dt, offset_row(ox, oy, oz));
            ot_multi_fwd(a, r, d);
        } else {
            source_moments(p, e2, v2, qx, qy, qz, r);
            load_row(d, p.Dt, offset_row(rx, ry, rz));
            ot_multi_fwd(a, r, d);
        }
    }
}

template <int A, class CH>
__device__ __forceinline__ void walk_multi_apair_list(const CH& ch, int par, int tx, int ty, int tz,
                                                      const int2* __restrict__ s_nb, const FwdParams& p,
                                                      double (&a)[16], int item) {
    const int* al = p.L.lists + p.L.ap_off[A] + par * p.L.ap_len[A];
    const int np = p.L.ap_pairs[A], ns = p.L.ap_len[A] - np;
    walk_multi_apairs<A>(al + ch.lo(np), ch.n(np), true, tx, ty, tz, s_nb, p, a, item);
    walk_multi_apairs<A>(al + np + ch.lo(ns), ch.n(ns), false, tx, ty, tz, s_nb, p, a, item);
}

// a non-leaf target's point-mass sources (leaf cells and virtual
// descendants in its neighbours) by its axis-pair list: an entry o and its
// reflection along axis A share the row of o through the sum and the
// difference of their masses (a member without a point mass counts 0, and
// a lone member's sum and difference are its mass, exactly); the entry is
// skipped where no lane has a point mass at either member
template <int A>
__device__ __forceinline__ void walk_mono_apairs(const int* __restrict__ list, int len, bool paired, int tx,
                                                 int ty, int tz, const int2* __restrict__ s_nb,
                                                 const FwdParams& p, double (&a)[16], int item) {
    for (int k = 0; k < len; ++k) {
        const int po = __ldg(list + k);
        const int ox = (po & 0xff) - 8, oy = ((po >> 8) & 0xff) - 8, oz = ((po >> 16) & 0xff) - 8;
        const int px = tx + ox, py = ty + oy, pz = tz + oz;
        const int qx = A == 0 ? tx - ox : px, qy = A == 1 ? ty - oy : py, qz = A == 2 ? tz - oz : pz;
        const int2 e1 = s_nb[nb_index(px, py, pz)];
        const int k1 = checked_kind(p, e1, item);
        int2 e2 = make_int2(-1, 0);
        int k2 = K_NONE;
        if (paired) {
            e2 = s_nb[nb_index(qx, qy, qz)];
            k2 = checked_kind(p, e2, item);
        }
        if (!__any_sync(0xffffffffu, k1 >= K_LEAF || k2 >= K_LEAF)) continue;
        const double m1 = source_mass(p, e1, k1, px, py, pz);
        const double m2 = paired ? source_mass(p, e2, k2, qx, qy, qz) : 0.0;
        double d[36];
        load_row16(d, p.Dt, offset_row(ox, oy, oz));
        if constexpr (A == 0) ot_mono_fwd_xpair(a, m1 + m2, m1 - m2, d);
        else if constexpr (A == 1) ot_mono_fwd_ypair(a, m1 + m2, m1 - m2, d);
        else ot_mono_fwd_zpair(a, m1 + m2, m1 - m2, d);
    }
}

template <int A, class CH>
__device__ __forceinline__ void walk_mono_apair_list(const CH& ch, int par, int tx, int ty, int tz,
                                                     const int2* __restrict__ s_nb, const FwdParams& p,
                                                     double (&a)[16], int item) {
    const int* al = p.L.lists + p.L.ap_off[A] + par * p.L.ap_len[A];
    const int np = p.L.ap_pairs[A], ns = p.L.ap_len[A] - np;
    walk_mono_apairs<A>(al + ch.lo(np), ch.n(np), true, tx, ty, tz, s_nb, p, a, item);
    walk_mono_apairs<A>(al + np + ch.lo(ns), ch.n(ns), false, tx, ty, tz, s_nb, p, a, item);
}

template <int MODE>
__device__ __forceinline__ void store_forward(const FwdParams& p, int node, int level, bool leafT, int tcell,
                                              const double (&a)[16], const double (&c)[3],
                                              const double (&t4)[9]) {
    const double h1 = p.hinv[level], h2 = h1 * h1, h3 = h2 * h1, h4 = h2 * h2;
    double L[20];
    L[0] = a[0] * h1;
    L[1] = a[1] * h2;
    L[2] = a[2] * h2;
    L[3] = a[3] * h2;
    L[4] = a[4] * h3;
    L[5] = a[5] * h3;
    L[6] = a[6] * h3;
    L[7] = a[7] * h3;
    L[8] = a[8] * h3;
    L[9] = -(a[4] + a[7]) * h3;
    L[10] = a[9] * h4;
    L[11] = a[10] * h4;
    L[12] = a[11] * h4;
    L[13] = a[12] * h4;
    L[14] = a[13] * h4;
    L[15] = -(a[9] + a[12]) * h4;
    L[16] = a[14] * h4;
    L[17] = a[15] * h4;
    L[18] = -(a[10] + a[14]) * h4;
    L[19] = -(a[11] + a[15]) * h4;
    double* out = p.Lout + static_cast<size_t>(node) * NCOMP * NCELL + tcell;
    if (p.accumulate) {
#pragma unroll
        for (int q = 0; q < 20; ++q) out[q * NCELL] += L[q];
    } else {
#pragma unroll
        for (int q = 0; q < 20; ++q) out[q * NCELL] = L[q];
    }
    if ((MODE & 1) && p.Lc != nullptr) {
        double lc[3] = {0.0, 0.0, 0.0};
        if (!leafT) {
            const double* mh = p.Mhat + static_cast<size_t>(node) * NRED * NCELL + tcell;
            const double mA = mh[0];
            if (mA != 0.0) {
                double rA[16];
#pragma unroll
                for (int q = 0; q < 9; ++q) rA[q] = 0.0;
#pragma unroll
                for (int q = 9; q < 16; ++q) rA[q] = mh[q * NCELL];
                double o[3];
                ot_angular_target(o, t4, rA);
#pragma unroll
                for (int i = 0; i < 3; ++i) lc[i] = h2 * (c[i] - o[i] / mA);
            }
        }
        double* lo = p.Lc + static_cast<size_t>(node) * 3 * NCELL + tcell;
        lo[0] = lc[0];
        lo[NCELL] = lc[1];
        lo[2 * NCELL] = lc[2];
    }
}

// chunk c of k of a work item walks entries [len c / k, len (c + 1) / k) of
// every list
struct Chunk {
    int c, k;
    __device__ __forceinline__ int lo(int len) const { return len * c / k; }
    __device__ __forceinline__ int n(int len) const { return len * (c + 1) / k - len * c / k; }
};

// the chunk's NV accumulators into its partial slot; true for the last chunk
// of the (node, parity, half) to finish, which then holds the sum of all
// chunks in chunk order (the same bits whichever chunk finishes last).  Each
// lane's stores are fenced before lane 0 counts the chunk; the last chunk
// fences again before it reads the slots (L1 bypassed).  Nothing waits.
template <int NV>
__device__ __forceinline__ bool chunk_combine(double* part, int* ctr, int2 ci, int ph, Chunk ch, int lane,
                                              double (&v)[NV]) {
    double* slot = part + static_cast<size_t>(ci.x + ph * ch.k + ch.c) * NV * 32 + lane;
#pragma unroll
    for (int q = 0; q < NV; ++q) __stcg(slot + q * 32, v[q]);
    __threadfence();
    __syncwarp();
    int last = 0;
    if (lane == 0) last = atomicAdd(ctr + (ci.y >> 4) + ph, 1) == ch.k - 1;
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last) return false;
    __threadfence();
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = 0.0;
    for (int j = 0; j < ch.k; ++j) {
        const double* src = part + static_cast<size_t>(ci.x + ph * ch.k + j) * NV * 32 + lane;
#pragma unroll
        for (int q = 0; q < NV; ++q) v[q] += __ldcg(src + q * 32);
    }
    return true;
}

// the forward's accumulators: the 16 coefficients, the angular term's source
// and target parts
__device__ __forceinline__ bool chunk_combine_fwd(const FwdParams& p, int2 ci, int ph, Chunk ch, int lane,
                                                  double (&a)[16], double (&c)[3], double (&t4)[9]) {
    double v[PART_VALS];
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = a[q];
#pragma unroll
    for (int q = 0; q < 3; ++q) v[16 + q] = c[q];
#pragma unroll
    for (int q = 0; q < 9; ++q) v[19 + q] = t4[q];
    if (!chunk_combine(p.part, p.chunk_ctr, ci, ph, ch, lane, v)) return false;
#pragma unroll
    for (int q = 0; q < 16; ++q) a[q] = v[q];
#pragma unroll
    for (int q = 0; q < 3; ++q) c[q] = v[16 + q];
#pragma unroll
    for (int q = 0; q < 9; ++q) t4[q] = v[19 + q];
    return true;
}

// MINB: resident blocks of 256 threads per SM the register allocation must
// allow (2 caps a thread at 128 registers, 1 at 255)
template <int MODE, int EMU, int MINB = (EMU ? 1 : 2)>
__global__ void __launch_bounds__(256, MINB) forward_kernel(const FwdParams p, int persistent) {
    __shared__ int2 s_nb[8][27];
    __shared__ int s_sl[8][27];   // x-table slots of the neighbours (leaf or multipole)
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    int it = blockIdx.x * wpb + warp;
    for (;;) {
        if (persistent) {
            int v = 0;
            if (lane == 0) v = atomicAdd(p.counter, 1);
            it = __shfl_sync(0xffffffffu, v, 0);
        }
        if (it >= p.n_items) break;
        const int item = __ldg(p.items + it);
        const int node = (item >> 4) & 0x3fffff, par = (item >> 1) & 7, half = item & 1;
        Chunk ch{(item >> 26) & 15, 1};
        int2 ci = make_int2(-1, 0);
        if (p.cinfo != nullptr) {
            ci = __ldg(p.cinfo + node);
            if (ci.x >= 0) ch.k = (ci.y & 15) + 1;
        }
        if (ch.c >= ch.k) {        // a chunk index the node does not have
            report(p.status, 6, it);
            if (!persistent) break;
            continue;
        }
        if (lane < 27) {
            const int2 e = __ldg(p.nbr + static_cast<size_t>(node) * 27 + lane);
            s_nb[warp][lane] = e;
            const int k = e.y & 3;
            s_sl[warp][lane] = (p.nslot != nullptr && k != K_NONE) ? __ldg(p.nslot + static_cast<size_t>(node) * 27 + lane)
                                                                    : -1;
        }
        __syncwarp();
        const int info = __ldg(p.ninfo + node);
        const int level = info & 0xff;
        const bool leafT = (info >> 8) & 1;
        int tx, ty, tz;
        lane_cell_slab(lane, par, half, (info >> NI_SLAB_SHIFT) & 3, tx, ty, tz);
        double a[16], c[3], t4[9];
        DFAcc f;
        df_zero(f);
#pragma unroll
        for (int q = 0; q < 16; ++q) a[q] = 0.0;
#pragma unroll
        for (int q = 0; q < 3; ++q) c[q] = 0.0;
#pragma unroll
        for (int q = 0; q < 9; ++q) t4[q] = 0.0;
        if ((MODE & 2) && level > 0 && leafT) {
            // leaf target, point masses: by reflection class over the far
            // and near offsets (FP64, or double-float with EMU bit 1);
            // multipole sources (refined neighbours) over the full far list,
            // refined near sources over the near list
            const int2* nb = s_nb[warp];
            const bool xpath = (EMU & 1) ? p.Smf != nullptr && (info & NI_XMASS) : p.Sm != nullptr && (info & NI_XMASS);
            const int* cf = p.L.lists + p.L.cf_off + par * p.L.cf_stride;
            const int* cn = p.L.lists + p.L.cn_off;
            if constexpr ((EMU & 1) != 0) {
                // one inlined copy of the double-float class walk serves the
                // far and the near class lists: with a copy for each, the code
                // of all its paths overflowed the instruction cache on trees
                // whose leaves take every path
#pragma unroll 1
                for (int sgm = 0; sgm < 2; ++sgm) {
                    int zo[8], xo[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        zo[k] = sgm ? p.L.cn_z[k] : p.L.cf_z[k];
                        xo[k] = sgm ? p.L.cn_x[k] : p.L.cf_x[k];
                    }
                    walk_classes_fwd_df_all(sgm ? cn : cf, zo, xo, xpath, ch, tx, ty, tz, nb, s_sl[warp], p, a, c, t4, f,
                                            it);
                }
            } else {
                walk_classes_fwd_all(cf, p.L.cf_z, p.L.cf_x, p.L.cf_xy, xpath, ch, tx, ty, tz, nb, s_sl[warp], p, a, it);
            }
            cf += p.L.cf_z[7];
            cn += p.L.cn_z[7];
            if constexpr ((EMU & 1) != 0) {
                // the classes' leftover +-o pairs of both lists through one
                // inlined copy as well
#pragma unroll 1
                for (int sgm = 0; sgm < 2; ++sgm) {
                    const int np = sgm ? p.L.cn_pairs : p.L.cf_pairs;
                    walk_forward<2, true, EMU>((sgm ? cn : cf) + ch.lo(np), ch.n(np), false, tx, ty, tz, nb, p, a, c,
                                               t4, f, it);
                }
            } else {
                walk_forward<2, true, EMU>(cf + ch.lo(p.L.cf_pairs), ch.n(p.L.cf_pairs), false, tx, ty, tz, nb, p, a,
                                           c, t4, f, it);
            }
            cf += p.L.cf_pairs;
            walk_forward<2, false, EMU>(cf + ch.lo(p.L.cf_singles), ch.n(p.L.cf_singles), false, tx, ty, tz, nb, p, a,
                                        c, t4, f, it);
            if constexpr ((EMU & 1) == 0) {
                walk_classes_fwd_all(cn - p.L.cn_z[7], p.L.cn_z, p.L.cn_x, p.L.cn_xy, xpath, ch, tx, ty, tz, nb,
                                     s_sl[warp], p, a, it);
                walk_forward<2, true, EMU>(cn + ch.lo(p.L.cn_pairs), ch.n(p.L.cn_pairs), false, tx, ty, tz, nb, p, a,
                                           c, t4, f, it);
            }
            if (__any_sync(0xffffffffu, lane < 27 && (nb[lane < 27 ? lane : 0].y & 3) == K_MULTI)) {
                if (MODE & 1) {
                    const int* lf = p.L.lists + par * p.L.far_len;
                    const int ns = p.L.far_len - p.L.far_pairs;
                    walk_forward<1, true, EMU>(lf + ch.lo(p.L.far_pairs), ch.n(p.L.far_pairs), false, tx, ty, tz, nb,
                                               p, a, c, t4, f, it);
                    walk_forward<1, false, EMU>(lf + p.L.far_pairs + ch.lo(ns), ch.n(ns), false, tx, ty, tz, nb, p, a,
                                                c, t4, f, it);
                }
                walk_forward<2, true, EMU, true, false>(p.L.lists + p.L.near_off + ch.lo(p.L.near_len),
                                                        ch.n(p.L.near_len), false, tx, ty, tz, nb, p, a, c, t4, f, it);
            }
        } else if (!leafT && !(EMU & 2)) {
            // non-leaf target, FP64 multipole contractions: multipole sources
            // by reflection class (root or far list), the classes' leftover
            // pairs and singles; point masses (leaf neighbours of an adaptive
            // tree) over the far list
            const int2* nb = s_nb[warp];
            if (MODE & 1) {
                const bool root = level == 0;
                int zo[8], xc[8], xyc[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    zo[q] = root ? p.L.mr_z[q] : p.L.mf_z[q];
                    xc[q] = root ? p.L.mr_x[q] : p.L.mf_x[q];
                    xyc[q] = root ? p.L.mr_xy[q] : p.L.mf_xy[q];
                }
                const bool xpath = p.Sx != nullptr && (info & NI_XMULTI);
                const int* ml = p.L.lists + (root ? p.L.mr_off : p.L.mf_off + par * p.L.mf_stride);
                walk_mclasses_fwd_all<true>(ml, zo, xc, xyc, xpath, ch, tx, ty, tz, nb, s_sl[warp], p, a, c, t4, it);
                ml += zo[7];
                const int np = root ? p.L.mr_pairs : p.L.mf_pairs, ns = root ? 0 : p.L.mf_singles;
                walk_forward<1, true, EMU>(ml + ch.lo(np), ch.n(np), true, tx, ty, tz, nb, p, a, c, t4, f, it);
                walk_forward<1, false, EMU>(ml + np + ch.lo(ns), ch.n(ns), true, tx, ty, tz, nb, p, a, c, t4, f, it);
            }
            if ((MODE & 2) && level > 0 &&
                __any_sync(0xffffffffu, lane < 27 && (nb[lane < 27 ? lane : 0].y & 3) >= K_LEAF)) {
                if constexpr ((EMU & 1) == 0) {
                    // point masses (leaf neighbours) paired along the node's axis
                    const int A = (info >> NI_APAIR_SHIFT) & 3;
                    if (A == 0)
                        walk_mono_apair_list<0>(ch, par, tx, ty, tz, nb, p, a, it);
                    else if (A == 1)
                        walk_mono_apair_list<1>(ch, par, tx, ty, tz, nb, p, a, it);
                    else
                        walk_mono_apair_list<2>(ch, par, tx, ty, tz, nb, p, a, it);
                } else {
                    const int* lf = p.L.lists + par * p.L.far_len;
                    const int ns = p.L.far_len - p.L.far_pairs;
                    walk_forward<2, true, EMU>(lf + ch.lo(p.L.far_pairs), ch.n(p.L.far_pairs), true, tx, ty, tz, nb,
                                               p, a, c, t4, f, it);
                    walk_forward<2, false, EMU>(lf + p.L.far_pairs + ch.lo(ns), ch.n(ns), true, tx, ty, tz, nb, p, a,
                                                c, t4, f, it);
                }
            }
        } else {
            if (level == 0) {
                walk_forward<MODE, true, EMU>(p.L.lists + p.L.root_off + ch.lo(p.L.root_len), ch.n(p.L.root_len),
                                              !leafT, tx, ty, tz, s_nb[warp], p, a, c, t4, f, it);
            } else if (MODE == 1 && leafT && !(EMU & 2)) {
                // a leaf target's multipole sources lie in refined neighbours,
                // mostly on one side: paired with their reflections along the
                // node's axis, each pair or member only where some lane has a
                // source
                const int A = (info >> NI_APAIR_SHIFT) & 3;
                if (A == 0)
                    walk_multi_apair_list<0>(ch, par, tx, ty, tz, s_nb[warp], p, a, it);
                else if (A == 1)
                    walk_multi_apair_list<1>(ch, par, tx, ty, tz, s_nb[warp], p, a, it);
                else
                    walk_multi_apair_list<2>(ch, par, tx, ty, tz, s_nb[warp], p, a, it);
            } else {
                const int* lf = p.L.lists + par * p.L.far_len;
                const int ns = p.L.far_len - p.L.far_pairs;
                walk_forward<MODE, true, EMU>(lf + ch.lo(p.L.far_pairs), ch.n(p.L.far_pairs), !leafT, tx, ty, tz,
                                              s_nb[warp], p, a, c, t4, f, it);
                walk_forward<MODE, false, EMU>(lf + p.L.far_pairs + ch.lo(ns), ch.n(ns), !leafT, tx, ty, tz,
                                               s_nb[warp], p, a, c, t4, f, it);
            }
            if (leafT && (MODE & 2))
                walk_forward<MODE, true, EMU, true>(p.L.lists + p.L.near_off + ch.lo(p.L.near_len), ch.n(p.L.near_len),
                                                    false, tx, ty, tz, s_nb[warp], p, a, c, t4, f, it);
        }
        if (EMU) df_flush_all<(EMU & 2) != 0>(a, c, t4, f);
        if (ch.k == 1 || chunk_combine_fwd(p, ci, item & 15, ch, lane, a, c, t4))
            store_forward<MODE>(p, node, level, leafT, tx + 8 * ty + 64 * tz, a, c, t4);
        __syncwarp();
        if (!persistent) break;
    }
}

// ---------------------------------------------------------------------------
// adjoint (transposed) stencil walk: a gather over source cells
// ---------------------------------------------------------------------------

// lb of one adjoint target: a real cell's reduced L-bar, or for a virtual
// child of a coarse leaf (depth 1; the coarse leaf refined as a target) the
// covering cell's, times 2^(n+1)/8 (the mean over the children, in the
// finer level's h units)
__device__ __forceinline__ void adjoint_target_lb(const AdjParams& p, int2 e, bool real, bool vchild, int tx, int ty,
                                                  int tz, double (&lb)[16]) {
    if (real) {
        const double* src = p.Lrbar + static_cast<size_t>(e.x) * NRED * NCELL + (tx & 7) + 8 * (ty & 7) + 64 * (tz & 7);
#pragma unroll
        for (int q = 0; q < 16; ++q) lb[q] = __ldg(src + q * NCELL);
    } else if (vchild) {
        const unsigned meta = static_cast<unsigned>(e.y);
        const int vx = static_cast<int>(((meta >> 8) & 0xffu) + (tx & 7)) >> 1;
        const int vy = static_cast<int>(((meta >> 16) & 0xffu) + (ty & 7)) >> 1;
        const int vz = static_cast<int>((meta >> 24) + (tz & 7)) >> 1;
        const double* src = p.Lrbar + static_cast<size_t>(e.x) * NRED * NCELL + vx + 8 * vy + 64 * vz;
#pragma unroll
        for (int q = 0; q < 16; ++q) lb[q] = vchild_scale(q) * __ldg(src + q * NCELL);
    } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) lb[q] = 0.0;
    }
}

// the reduced L-bar of a real target cell as double-float pairs (or zeros)
__device__ __forceinline__ void adjoint_target_lb_df(const AdjParams& p, int2 e, bool real, int tx, int ty, int tz,
                                                     float (&lh)[16], float (&ll)[16]) {
    if (real) {
        const float2* src = p.Lf + static_cast<size_t>(e.x) * NRED * NCELL + (tx & 7) + 8 * (ty & 7) + 64 * (tz & 7);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const float2 v = __ldg(src + q * NCELL);
            lh[q] = v.x;
            ll[q] = v.y;
        }
    } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            lh[q] = 0.0f;
            ll[q] = 0.0f;
        }
    }
}

// a depth-1 virtual descendant (the child of a coarse leaf cell) as a target
// of a real point-mass source
__device__ __forceinline__ bool virtual_child_target(int2 e, bool virt_t) {
    return virt_t && (e.y & 3) == K_VIRT && ((static_cast<unsigned>(e.y) >> 2) & 7u) == 1u;
}

// Source B of parity p gathers from targets A = B + o' for o' in the forward
// list of parity p (far pairs are symmetric under o -> -o with the parities
// swapped), with the table row of the forward offset o = -o'.  A paired
// entry o' also gathers from A = B - o' (row of o', odd orders negated).
// virt_t: a real leaf source also gathers from depth-1 virtual children of
// coarse leaves (the transpose of the coarse-target refinement).
// EMU (multipole sources only): the contraction in double-float into f,
// moved into g by coefficient-order groups (at most 64 products each)
template <bool MULTI, bool PAIRED, bool EMU = false>
__device__ __forceinline__ void walk_adjoint(const int* __restrict__ list, int len, bool near_seg, bool virt_t,
                                             int sx0, int sy0, int sz0, const int2* __restrict__ s_nb,
                                             const AdjParams& p, double (&g)[16], double (&g4)[4],
                                             DFAcc& f, int item) {
    for (int k = 0; k < len; ++k) {
        const int po = __ldg(list + k);
        const int ox = (po & 0xff) - 8, oy = ((po >> 8) & 0xff) - 8, oz = ((po >> 16) & 0xff) - 8;
        const int px = sx0 + ox, py = sy0 + oy, pz = sz0 + oz;
        const int mx = sx0 - ox, my = sy0 - oy, mz = sz0 - oz;
        const int2 ep = s_nb[nb_index(px, py, pz)];
        int kp = ep.y & 3;
        bool vp = (kp == K_MULTI || kp == K_LEAF) && (!near_seg || kp == K_LEAF);
        bool wp = !MULTI && virtual_child_target(ep, virt_t);
        if ((vp || wp) && static_cast<unsigned>(ep.x) >= static_cast<unsigned>(p.n_nodes)) {
            report(p.status, 2, item);
            vp = wp = false;
        }
        int2 em = make_int2(-1, 0);
        bool vm = false, wm = false;
        if (PAIRED) {
            em = s_nb[nb_index(mx, my, mz)];
            const int km = em.y & 3;
            vm = (km == K_MULTI || km == K_LEAF) && (!near_seg || km == K_LEAF);
            wm = !MULTI && virtual_child_target(em, virt_t);
            if ((vm || wm) && static_cast<unsigned>(em.x) >= static_cast<unsigned>(p.n_nodes)) {
                report(p.status, 2, item);
                vm = wm = false;
            }
        }
        if (!__any_sync(0xffffffffu, vp || vm || wp || wm)) continue;
        const int row = NOFF - 1 - offset_row(ox, oy, oz);
        if constexpr (MULTI && EMU) {
            double dc[3], dt[9];     // the angular groups are not used here
            df_reserve(g, dc, dt, f, 16, 9, 4, 1, 0, 0);
            float lh[16], ll[16];
            adjoint_target_lb_df(p, ep, vp, px, py, pz, lh, ll);
            const float2* drow = p.Dt2 + static_cast<size_t>(row) * DROW;
            if (PAIRED) {
                float mh[16], ml[16];
                adjoint_target_lb_df(p, em, vm, mx, my, mz, mh, ml);
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    float sh, sl, dh, dl;
                    df_add(lh[q], ll[q], mh[q], ml[q], sh, sl);
                    df_add(lh[q], ll[q], -mh[q], -ml[q], dh, dl);
                    lh[q] = sh;
                    ll[q] = sl;
                    mh[q] = dh;
                    ml[q] = dl;
                }
                ot_multi_adj_pair_df(f.ah, f.al, lh, ll, mh, ml, drow);
            } else {
                ot_multi_adj_df(f.ah, f.al, lh, ll, drow);
            }
            continue;
        }
        double lb[16];
        adjoint_target_lb(p, ep, vp, wp, px, py, pz, lb);
        double d[36];
        if (MULTI) {
            load_row(d, p.Dt, row);
            if (PAIRED) {
                double lm[16];
                if (vm) {
                    const double* src = p.Lrbar + static_cast<size_t>(em.x) * NRED * NCELL + (mx & 7) +
                                        8 * (my & 7) + 64 * (mz & 7);
#pragma unroll
                    for (int q = 0; q < 16; ++q) lm[q] = __ldg(src + q * NCELL);
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q) lm[q] = 0.0;
                }
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const double t = lb[q];
                    lb[q] = t + lm[q];
                    lm[q] = t - lm[q];
                }
                ot_multi_adj_pair(g, lb, lm, d);
            } else {
                ot_multi_adj(g, lb, d);
            }
        } else {
            load_row16(d, p.Dt, row);
            ot_mono_adj(g4, lb, d);
            if (PAIRED) {
                double lm[16];
                adjoint_target_lb(p, em, vm, wm, mx, my, mz, lm);
                ot_mono_adj_neg(g4, lm, d);
            }
        }
    }
}

// the multipole gather by reflection class: the members are the targets
// B + s*o of source B (multipole or leaf cells of B's level, as in
// walk_adjoint), whose reduced L-bar feed the transposed class contraction
// (see gen_contract.py) with the table row of -o
template <int Z>
__device__ __forceinline__ void walk_mclasses_adj(const int* __restrict__ list, int len, int sx0, int sy0, int sz0,
                                                  const int2* __restrict__ s_nb, const AdjParams& p,
                                                  double (&g)[16], int item) {
    for (int k = 0; k < len; ++k) {
        const int e = __ldg(list + k);
        const int ox = e & 0xff, oy = (e >> 8) & 0xff, oz = (e >> 16) & 0xff;
        const unsigned members = static_cast<unsigned>(e) >> 24;
        const double* src[8];
        bool any = false;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            src[i] = nullptr;
            if (i & Z) continue;
            if ((members >> i) & 1u) {
                int tx, ty, tz;
                class_member(i, ox, oy, oz, sx0, sy0, sz0, tx, ty, tz);
                const int2 et = s_nb[nb_index(tx, ty, tz)];
                const int kt = et.y & 3;
                if (kt == K_MULTI || kt == K_LEAF) {
                    if (static_cast<unsigned>(et.x) >= static_cast<unsigned>(p.n_nodes)) {
                        report(p.status, 2, item);
                    } else {
                        src[i] = p.Lrbar + static_cast<size_t>(et.x) * NRED * NCELL + (tx & 7) + 8 * (ty & 7) +
                                 64 * (tz & 7);
                        any = true;
                    }
                }
            }
        }
        if (!__any_sync(0xffffffffu, any)) continue;
        ot_mclass_adj<Z>(g, src, p.Dt + static_cast<size_t>(NOFF - 1 - offset_row(ox, oy, oz)) * DROW);
    }
}

// x-complete classes of a source whose neighbours are real or empty: the
// first transform stage of every target component comes from the prebuilt
// L-bar x butterflies at the positions B + (0, +-b, +-c)
template <int Z>
__device__ __forceinline__ void walk_mclasses_adj_x(const int* __restrict__ list, int len, int sx0, int sy0, int sz0,
                                                    const int2* __restrict__ s_nb, const int* __restrict__ s_sl, const AdjParams& p,
                                                    double (&g)[16], int item) {
    static_assert((Z & 1) == 0, "the x stage needs a > 0");
    for (int k = 0; k < len; ++k) {
        const int e = __ldg(list + k);
        const int ox = e & 0xff, oy = (e >> 8) & 0xff, oz = (e >> 16) & 0xff;
        const unsigned members = static_cast<unsigned>(e) >> 24;
        const double* pos[4];
        bool any = false;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            pos[q] = nullptr;
            if ((2 * q) & Z) continue;
            if ((members >> (2 * q)) & 1u) {
                const int ty = (q & 1) ? sy0 - oy : sy0 + oy, tz = (q & 2) ? sz0 - oz : sz0 + oz;
                const int nbi = nb_index(sx0, ty, tz);
                const int kt = s_nb[nbi].y & 3;
                const int slot = s_sl[nbi];
                if (slot >= 0) {
                    pos[q] = p.Tx + static_cast<size_t>(slot * 7 + ox - 1) * 32 * NCELL + (sx0 & 7) +
                             8 * (ty & 7) + 64 * (tz & 7);
                    any = true;
                } else if (kt != K_NONE) {
                    report(p.status, 7, item);    // the source's flag promised a table slot for every region
                }
            }
        }
        if (!__any_sync(0xffffffffu, any)) continue;
        ot_mclass_adj_x<Z>(g, pos, p.Dt + static_cast<size_t>(NOFF - 1 - offset_row(ox, oy, oz)) * DROW);
    }
}

template <int Z = 0, class CH>
__device__ __forceinline__ void walk_mclasses_adj_all(const int* __restrict__ list, const int (&zoff)[8],
                                                      const int (&xc)[8], bool xpath, const CH& ch, int sx0, int sy0,
                                                      int sz0, const int2* __restrict__ s_nb, const int* __restrict__ s_sl, const AdjParams& p,
                                                      double (&g)[16], int item) {
    const int len = zoff[Z + 1] - zoff[Z];
    int nx = 0;
    if constexpr ((Z & 1) == 0) {
        if (xpath) {
            nx = xc[Z];
            walk_mclasses_adj_x<Z>(list + zoff[Z] + ch.lo(nx), ch.n(nx), sx0, sy0, sz0, s_nb, s_sl, p, g, item);
        }
    }
    walk_mclasses_adj<Z>(list + zoff[Z] + nx + ch.lo(len - nx), ch.n(len - nx), sx0, sy0, sz0, s_nb, p, g, item);
    if constexpr (Z < 6) walk_mclasses_adj_all<Z + 1>(list, zoff, xc, xpath, ch, sx0, sy0, sz0, s_nb, s_sl, p, g, item);
}

// M-bar of one source cell from the gathered g (reduced, h-scaled): expand
// the traceless reduction and apply (-1)^m/m! * multiplicity * h^-m
__device__ __forceinline__ void store_mbar(double* __restrict__ Mbar, int src, int scell, double h1,
                                           const double (&g)[16]) {
    const double h2 = h1 * h1, h3 = h2 * h1;
    double Mb[20];
    Mb[0] = g[0];
    Mb[1] = -h1 * g[1];
    Mb[2] = -h1 * g[2];
    Mb[3] = -h1 * g[3];
    Mb[4] = 0.5 * h2 * g[4];
    Mb[5] = h2 * g[5];
    Mb[6] = h2 * g[6];
    Mb[7] = 0.5 * h2 * g[7];
    Mb[8] = h2 * g[8];
    Mb[9] = -0.5 * h2 * (g[4] + g[7]);
    const double s6 = -h3 / 6.0, s2 = -0.5 * h3;
    Mb[10] = s6 * g[9];
    Mb[11] = s2 * g[10];
    Mb[12] = s2 * g[11];
    Mb[13] = s2 * g[12];
    Mb[14] = -h3 * g[13];
    Mb[15] = -s2 * (g[9] + g[12]);
    Mb[16] = s6 * g[14];
    Mb[17] = s2 * g[15];
    Mb[18] = -s2 * (g[10] + g[14]);
    Mb[19] = -s6 * (g[11] + g[15]);
    double* out = Mbar + static_cast<size_t>(src) * NCOMP * NCELL + scell;
#pragma unroll
    for (int q = 0; q < 20; ++q) out[q * NCELL] = Mb[q];
}

template <bool EMU = false, class P>
__device__ __forceinline__ void scatter_item(const P& p, const int2* __restrict__ nbr, const int* __restrict__ ninfo, int2* s_nb,
                             int* s_sl, int node, int par, int half, int lane, int it);

// MODE 1: multipole gather items; 2, 3: the point masses gathered too (the
// deterministic adjoint); 4: point-mass items by target (atomic adds).
// EMU: double-float multipole gather and point-mass scatter (MODE 1, 4)
template <int MODE, bool EMU = false>
__global__ void __launch_bounds__(256, 1) adjoint_kernel(const AdjParams p, int persistent) {
    __shared__ int2 s_nb[8][27];
    __shared__ int s_sl[8][27];   // x-table slots of the neighbours
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    int it = blockIdx.x * wpb + warp;
    for (;;) {
        if (persistent) {
            int v = 0;
            if (lane == 0) v = atomicAdd(p.counter, 1);
            it = __shfl_sync(0xffffffffu, v, 0);
        }
        if (it >= p.n_items) break;
        const int item = __ldg(p.items + it);
        if ((MODE & 4) && ((item >> 30) & 1)) {       // point-mass adjoint by target (atomic adds)
            const int tgt = item & 0x3fffffff;
            scatter_item<EMU>(p, p.nbr, p.ninfo, s_nb[warp], s_sl[warp], tgt >> 4, (tgt >> 1) & 7, tgt & 1, lane, it);
            __syncwarp();
            if (!persistent) break;
            continue;
        }
        Chunk ch{0, 1};
        int2 ci = make_int2(-1, 0);
        int src = item >> 4;
        if (item < 0) {            // a chunk of a multipole gather item
            src = (item >> 4) & 0x3fffff;
            ch.c = (item >> 26) & 15;
            if (p.cinfo != nullptr && src < p.n_nodes) {
                ci = __ldg(p.cinfo + src);
                if (ci.x >= 0) ch.k = (ci.y & 15) + 1;
            }
            if (ch.c >= ch.k) {
                report(p.status, 6, it);
                if (!persistent) break;
                continue;
            }
        }
        const int par = (item >> 1) & 7, half = item & 1;
        const bool virt = src >= p.n_nodes;
        const int2* nbt = virt ? p.vnbr + static_cast<size_t>(src - p.n_nodes) * 27
                               : p.nbr + static_cast<size_t>(src) * 27;
        if (lane < 27) {
            const int2 e = __ldg(nbt + lane);
            s_nb[warp][lane] = e;
            const int k = e.y & 3;
            s_sl[warp][lane] = (p.nslot != nullptr && !virt && k != K_NONE)
                                   ? __ldg(p.nslot + static_cast<size_t>(src) * 27 + lane) : -1;
        }
        __syncwarp();
        int level, skind;
        if (virt) {
            level = __ldg(p.vinfo + (src - p.n_nodes));
            skind = K_VIRT;
        } else {
            const int info = __ldg(p.ninfo + src);
            level = info & 0xff;
            skind = ((info >> 8) & 1) ? K_LEAF : K_MULTI;
        }
        int sx, sy, sz;
        lane_cell(lane, par, half, sx, sy, sz);
        const int scell = sx + 8 * sy + 64 * sz;
        const int* l1 = (level == 0) ? p.L.lists + p.L.root_off : p.L.lists + par * p.L.far_len;
        const int n1 = (level == 0) ? p.L.root_len : p.L.far_len;
        const int* l2 = p.L.lists + p.L.near_off;
        const double h1 = p.hinv[level];
        double g[16], g4[4];
        DFAcc f;
        if (EMU) df_zero(f);
#pragma unroll
        for (int q = 0; q < 16; ++q) g[q] = 0.0;
#pragma unroll
        for (int q = 0; q < 4; ++q) g4[q] = 0.0;
        if (skind == K_MULTI) {
            // targets of the transposed far (root) stencil; near leaf targets
            // of a refined cell see its children instead
            if ((MODE & 1) && p.Mbar != nullptr) {
                if (!EMU) {
                    // by reflection class (root or far list of the source's
                    // parity), then the classes' leftover pairs and singles
                    const bool root = level == 0;
                    int zo[8], xc[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        zo[q] = root ? p.L.mr_z[q] : p.L.mf_z[q];
                        xc[q] = root ? p.L.mr_x[q] : p.L.mf_x[q];
                    }
                    const bool xpath = p.Tx != nullptr && (__ldg(p.ninfo + src) & NI_XGATHER);
                    const int* ml = p.L.lists + (root ? p.L.mr_off : p.L.mf_off + par * p.L.mf_stride);
                    walk_mclasses_adj_all(ml, zo, xc, xpath, ch, sx, sy, sz, s_nb[warp], s_sl[warp], p, g, it);
                    ml += zo[7];
                    const int np = root ? p.L.mr_pairs : p.L.mf_pairs, ns = root ? 0 : p.L.mf_singles;
                    walk_adjoint<true, true>(ml + ch.lo(np), ch.n(np), false, false, sx, sy, sz, s_nb[warp], p, g, g4,
                                             f, it);
                    walk_adjoint<true, false>(ml + np + ch.lo(ns), ch.n(ns), false, false, sx, sy, sz, s_nb[warp], p,
                                              g, g4, f, it);
                } else if (level == 0) {
                    walk_adjoint<true, true, EMU>(l1 + ch.lo(n1), ch.n(n1), false, false, sx, sy, sz, s_nb[warp], p, g,
                                                  g4, f, it);
                } else {
                    const int ns = n1 - p.L.far_pairs;
                    walk_adjoint<true, true, EMU>(l1 + ch.lo(p.L.far_pairs), ch.n(p.L.far_pairs), false, false, sx,
                                                  sy, sz, s_nb[warp], p, g, g4, f, it);
                    walk_adjoint<true, false, EMU>(l1 + p.L.far_pairs + ch.lo(ns), ch.n(ns), false, false, sx, sy, sz,
                                                   s_nb[warp], p, g, g4, f, it);
                }
                if (EMU) {
                    double dc[3], dt[9];
                    df_flush_all<false>(g, dc, dt, f);
                }
                if (ch.k == 1 || chunk_combine(p.part, p.chunk_ctr, ci, item & 15, ch, lane, g))
                    store_mbar(p.Mbar, src, scell, h1, g);
            }
        } else if ((MODE & 2) && p.mbar != nullptr) {
            const bool vt = skind == K_LEAF;   // real leaf cells also feed coarse leaves' virtual children
            if (level == 0) {
                walk_adjoint<false, true>(l1, n1, false, vt, sx, sy, sz, s_nb[warp], p, g, g4, f, it);
            } else {
                walk_adjoint<false, true>(l1, p.L.far_pairs, false, vt, sx, sy, sz, s_nb[warp], p, g, g4, f, it);
                walk_adjoint<false, false>(l1 + p.L.far_pairs, n1 - p.L.far_pairs, false, vt, sx, sy, sz, s_nb[warp],
                                           p, g, g4, f, it);
            }
            walk_adjoint<false, true>(l2, p.L.near_len, true, vt, sx, sy, sz, s_nb[warp], p, g, g4, f, it);
            const double v = (g4[0] + g4[1]) + (g4[2] + g4[3]);
            if (virt) p.vbar[static_cast<size_t>(src - p.n_nodes) * NCELL + scell] = v;
            else p.mbar[static_cast<size_t>(src) * NCELL + scell] = v;
        }
        __syncwarp();
        if (!persistent) break;
    }
}

// ---------------------------------------------------------------------------
// point-mass adjoint by target: mbar[B] += <Lrbar(A), d G(X_A - X_B)>
// ---------------------------------------------------------------------------

template <class P>
__device__ __forceinline__ void scatter_mass(const P& p, int2 e, int kind, int sx, int sy, int sz, double v) {
    if (kind == K_LEAF) {
        atomicAdd(p.mbar + static_cast<size_t>(e.x) * NCELL + (sx & 7) + 8 * (sy & 7) + 64 * (sz & 7), v);
    } else if (kind == K_VIRT) {
        const unsigned meta = static_cast<unsigned>(e.y);
        const int d = (meta >> 2) & 7;
        const int vx = static_cast<int>(((meta >> 8) & 0xffu) + (sx & 7)) >> d;
        const int vy = static_cast<int>(((meta >> 16) & 0xffu) + (sy & 7)) >> d;
        const int vz = static_cast<int>((meta >> 24) + (sz & 7)) >> d;
        atomicAdd(p.mbar + static_cast<size_t>(e.x) * NCELL + vx + 8 * vy + 64 * vz, v * pow2i(-3 * d));
    }
}

// A paired entry o: with e, q the even- and odd-order parts of <lb, row(o)>,
// the source at t+o (pair offset R = -o) receives e + q and the source at
// t-o (R = +o, odd orders change sign) receives e - q.
// EMU: the target's L-bar as double-float pairs (lbh, lbl; lb unused), each
// entry's dot product in fresh double-float accumulators (at most 8 products
// each, error below 30 * 2^-48 of its |terms|), added in FP64.  The pairs are
// loaded, not split here: a split the compiler may recompute inside the loop
// would put FP64 work back on the slow pipe.
// the point-mass adjoint by target over a class list (see walk_classes_fwd):
// member i of a class receives sum_pi (-1)^|i & pi| P[pi], P[pi] the partial
// dot product of the target's L-bar and the row over the components of
// parity pattern pi
// a class's eight member shares of a target's L-bar: the partial dot
// products by parity pattern, transformed over the sign axes from B0 on (B0 =
// 1: the x stage left to the deferred pass).  EMU: the partials and the
// transform in double-float (at most 3 products per partial), each share
// converted to FP64 once.
template <int Z, int B0, bool EMU, class P>
__device__ __forceinline__ void class_scatter_values(const P& p, int row, const double (&lb)[16],
                                                     const float (&lbh)[16], const float (&lbl)[16], double (&w)[8]) {
    if constexpr (EMU) {
        float r[32];
        load_row32f(r, p.Dt32, row);
        float wh[8], wl[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) wh[i] = wl[i] = 0.0f;
#pragma unroll
        for (int q = 0; q < 16; ++q)
            if (!(comp_parity(q) & Z)) df_fma(wh[comp_parity(q)], wl[comp_parity(q)], lbh[q], lbl[q], r[q], r[16 + q]);
        class_transform_df<Z, B0>(wh, wl);
#pragma unroll
        for (int i = 0; i < 8; ++i)
            w[i] = (i & Z) ? 0.0 : static_cast<double>(wh[i]) + static_cast<double>(wl[i]);
    } else {
        double d[36];
        load_row16(d, p.Dt, row);
#pragma unroll
        for (int i = 0; i < 8; ++i) w[i] = 0.0;
#pragma unroll
        for (int q = 0; q < 16; ++q)
            if (!(comp_parity(q) & Z)) w[comp_parity(q)] = fma(lb[q], d[q], w[comp_parity(q)]);
        if constexpr (B0 == 0) class_transform<Z>(w);
        else class_transform_yz<Z>(w);
    }
}

template <int Z, bool EMU, class P>
__device__ __forceinline__ void walk_classes_scatter(const int* __restrict__ list, int len, int tx, int ty, int tz,
                                                     const int2* __restrict__ s_nb, const P& p,
                                                     const double (&lb)[16], const float (&lbh)[16],
                                                     const float (&lbl)[16], int item) {
    for (int k = 0; k < len; ++k) {
        const int e = __ldg(list + k);
        const int a = e & 0xff, b = (e >> 8) & 0xff, c = (e >> 16) & 0xff;
        const unsigned members = static_cast<unsigned>(e) >> 24;
        int2 es[8];
        int ks[8];
        bool any = false;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            ks[i] = K_NONE;
            es[i] = make_int2(-1, 0);
            if (i & Z) continue;
            if ((members >> i) & 1u) {
                int sx, sy, sz;
                class_member(i, a, b, c, tx, ty, tz, sx, sy, sz);
                es[i] = s_nb[nb_index(sx, sy, sz)];
                int kind = es[i].y & 3;
                if (kind != K_NONE && static_cast<unsigned>(es[i].x) >= static_cast<unsigned>(p.n_nodes)) {
                    report(p.status, 3, item);
                    kind = K_NONE;
                }
                ks[i] = kind;
                any |= kind >= K_LEAF;
            }
        }
        if (!__any_sync(0xffffffffu, any)) continue;
        double w[8];
        class_scatter_values<Z, 0, EMU>(p, offset_row(a, b, c), lb, lbh, lbl, w);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (i & Z) continue;
            if (ks[i] >= K_LEAF) {
                int sx, sy, sz;
                class_member(i, a, b, c, tx, ty, tz, sx, sy, sz);
                scatter_mass(p, es[i], ks[i], sx, sy, sz, w[i]);
            }
        }
    }
}

// x-complete classes of a leaf target with leaf or empty neighbours: the
// partial dot products transformed over y and z only; for each (y, z) sign
// the two x channels go to the deferred butterfly accumulators of the
// position t + (0, +-b, +-c) (the members at +-a receive their sum and
// difference in xbutterfly_masses_adjoint_kernel)
template <int Z, bool EMU, class P>
__device__ __forceinline__ void walk_classes_scatter_x(const int* __restrict__ list, int len, int tx, int ty, int tz,
                                                       const int2* __restrict__ s_nb, const int* __restrict__ s_sl, const P& p,
                                                       const double (&lb)[16], const float (&lbh)[16],
                                                       const float (&lbl)[16], int item) {
    static_assert((Z & 1) == 0, "the x stage needs a > 0");
    for (int k = 0; k < len; ++k) {
        const int e = __ldg(list + k);
        const int a = e & 0xff, b = (e >> 8) & 0xff, c = (e >> 16) & 0xff;
        const unsigned members = static_cast<unsigned>(e) >> 24;
        double* dst[4];
        bool any = false;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            dst[q] = nullptr;
            if ((2 * q) & Z) continue;
            if ((members >> (2 * q)) & 1u) {
                const int sy = (q & 1) ? ty - b : ty + b, sz = (q & 2) ? tz - c : tz + c;
                const int nbi = nb_index(tx, sy, sz);
                const int ks = s_nb[nbi].y & 3;
                const int slot = s_sl[nbi];
                if (slot >= 0) {
                    dst[q] = p.Sbar + static_cast<size_t>(slot * 7 + a - 1) * 2 * NCELL + (tx & 7) +
                             8 * (sy & 7) + 64 * (sz & 7);
                    any = true;
                } else if (ks != K_NONE) {
                    report(p.status, 7, item);    // the target's flag promised a table slot for every region
                }
            }
        }
        if (!__any_sync(0xffffffffu, any)) continue;
        double w[8];
        class_scatter_values<Z, 1, EMU>(p, offset_row(a, b, c), lb, lbh, lbl, w);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if ((2 * q) & Z) continue;
            if (dst[q] != nullptr) {
                atomicAdd(dst[q], w[2 * q]);
                atomicAdd(dst[q] + NCELL, w[2 * q + 1]);
            }
        }
    }
}

template <bool EMU, int Z = 0, class P>
__device__ __forceinline__ void walk_classes_scatter_all(const int* __restrict__ list, const int* zoff, const int* xc,
                                                         bool xpath, int tx, int ty, int tz,
                                                         const int2* __restrict__ s_nb, const int* __restrict__ s_sl, const P& p,
                                                         const double (&lb)[16], const float (&lbh)[16],
                                                         const float (&lbl)[16], int item) {
    const int len = zoff[Z + 1] - zoff[Z];
    int nx = 0;
    if constexpr ((Z & 1) == 0) {
        if (xpath) {
            nx = xc[Z];
            walk_classes_scatter_x<Z, EMU>(list + zoff[Z], nx, tx, ty, tz, s_nb, s_sl, p, lb, lbh, lbl, item);
        }
    }
    walk_classes_scatter<Z, EMU>(list + zoff[Z] + nx, len - nx, tx, ty, tz, s_nb, p, lb, lbh, lbl, item);
    if constexpr (Z < 6)
        walk_classes_scatter_all<EMU, Z + 1>(list, zoff, xc, xpath, tx, ty, tz, s_nb, s_sl, p, lb, lbh, lbl, item);
}

template <bool PAIRED, bool NEAR, bool EMU = false, bool PM = true, class P>
__device__ __forceinline__ void walk_scatter(const int* __restrict__ list, int len, int tx, int ty,
                                             int tz, const int2* __restrict__ s_nb, const P& p,
                                             const double (&lb)[16], const float (&lbh)[16], const float (&lbl)[16],
                                             int item) {
    for (int k = 0; k < len; ++k) {
        const int po = __ldg(list + k);
        const int ox = (po & 0xff) - 8, oy = ((po >> 8) & 0xff) - 8, oz = ((po >> 16) & 0xff) - 8;
        const int px = tx + ox, py = ty + oy, pz = tz + oz;
        const int mx = tx - ox, my = ty - oy, mz = tz - oz;
        const int2 ep = s_nb[nb_index(px, py, pz)];
        int kp = ep.y & 3;
        if (kp != K_NONE && static_cast<unsigned>(ep.x) >= static_cast<unsigned>(p.n_nodes)) {
            report(p.status, 3, item);
            kp = K_NONE;
        }
        int2 em = make_int2(-1, 0);
        int km = K_NONE;
        if (PAIRED) {
            em = s_nb[nb_index(mx, my, mz)];
            km = em.y & 3;
            if (km != K_NONE && static_cast<unsigned>(em.x) >= static_cast<unsigned>(p.n_nodes)) {
                report(p.status, 3, item);
                km = K_NONE;
            }
        }
        if (NEAR) {
            // near sources in refined sub-grids: their children, through the
            // target's virtual children
            const bool rp = kp == K_MULTI, rm = km == K_MULTI;
            if (__any_sync(0xffffffffu, rp || rm)) {
                if constexpr (EMU) {
                    double lbd[16];
#pragma unroll
                    for (int q = 0; q < 16; ++q) lbd[q] = static_cast<double>(lbh[q]) + static_cast<double>(lbl[q]);
                    refined_near_scatter(p, ox, oy, oz, ep, rp, px, py, pz, em, rm, mx, my, mz, lbd, item);
                } else {
                    refined_near_scatter(p, ox, oy, oz, ep, rp, px, py, pz, em, rm, mx, my, mz, lb, item);
                }
            }
        }
        if (!PM || !__any_sync(0xffffffffu, kp >= K_LEAF || km >= K_LEAF)) continue;
        if constexpr (EMU) {
            float r[32];
            load_row32f(r, p.Dt32, offset_row(ox, oy, oz));
            float eh, el, qh, ql, sh, sl, dh, dl;
            ot_mono_adj_split_df(eh, el, qh, ql, lbh, lbl, r);
            df_add(eh, el, qh, ql, sh, sl);
            df_add(eh, el, -qh, -ql, dh, dl);
            scatter_mass(p, ep, kp, px, py, pz, static_cast<double>(sh) + static_cast<double>(sl));
            if (PAIRED) scatter_mass(p, em, km, mx, my, mz, static_cast<double>(dh) + static_cast<double>(dl));
        } else {
            double d[36];
            load_row16(d, p.Dt, offset_row(ox, oy, oz));
            double e, q;
            ot_mono_adj_split(e, q, lb, d);
            scatter_mass(p, ep, kp, px, py, pz, e + q);
            if (PAIRED) scatter_mass(p, em, km, mx, my, mz, e - q);
        }
    }
}

// the point-mass adjoint of a non-leaf target by its axis-pair list: with
// e, q the parts of <lb, row(o)> with an even and an odd A order, the source
// at t+o receives e + q and the one at o reflected along A receives e - q
template <int A, class P>
__device__ __forceinline__ void walk_scatter_apairs(const int* __restrict__ list, int len, bool paired, int tx,
                                                    int ty, int tz, const int2* __restrict__ s_nb, const P& p,
                                                    const double (&lb)[16], int item) {
    for (int k = 0; k < len; ++k) {
        const int po = __ldg(list + k);
        const int ox = (po & 0xff) - 8, oy = ((po >> 8) & 0xff) - 8, oz = ((po >> 16) & 0xff) - 8;
        const int px = tx + ox, py = ty + oy, pz = tz + oz;
        const int qx = A == 0 ? tx - ox : px, qy = A == 1 ? ty - oy : py, qz = A == 2 ? tz - oz : pz;
        const int2 e1 = s_nb[nb_index(px, py, pz)];
        int k1 = e1.y & 3;
        if (k1 != K_NONE && static_cast<unsigned>(e1.x) >= static_cast<unsigned>(p.n_nodes)) {
            report(p.status, 3, item);
            k1 = K_NONE;
        }
        int2 e2 = make_int2(-1, 0);
        int k2 = K_NONE;
        if (paired) {
            e2 = s_nb[nb_index(qx, qy, qz)];
            k2 = e2.y & 3;
            if (k2 != K_NONE && static_cast<unsigned>(e2.x) >= static_cast<unsigned>(p.n_nodes)) {
                report(p.status, 3, item);
                k2 = K_NONE;
            }
        }
        if (!__any_sync(0xffffffffu, k1 >= K_LEAF || k2 >= K_LEAF)) continue;
        double d[36];
        load_row16(d, p.Dt, offset_row(ox, oy, oz));
        double e, q;
        if constexpr (A == 0) ot_mono_adj_split_x(e, q, lb, d);
        else if constexpr (A == 1) ot_mono_adj_split_y(e, q, lb, d);
        else ot_mono_adj_split_z(e, q, lb, d);
        scatter_mass(p, e1, k1, px, py, pz, e + q);
        if (paired) scatter_mass(p, e2, k2, qx, qy, qz, e - q);
    }
}

template <int A, class P>
__device__ __forceinline__ void walk_scatter_apair_list(int par, int tx, int ty, int tz,
                                                        const int2* __restrict__ s_nb, const P& p,
                                                        const double (&lb)[16], int item) {
    const int* al = p.L.lists + p.L.ap_off[A] + par * p.L.ap_len[A];
    const int np = p.L.ap_pairs[A];
    walk_scatter_apairs<A>(al, np, true, tx, ty, tz, s_nb, p, lb, item);
    walk_scatter_apairs<A>(al + np, p.L.ap_len[A] - np, false, tx, ty, tz, s_nb, p, lb, item);
}

// one scatter work item: the warp's 32 target cells of `node` push their
// point-mass adjoint contributions into mbar
template <bool EMU, class P>
__device__ __forceinline__ void scatter_item(const P& p, const int2* __restrict__ nbr, const int* __restrict__ ninfo, int2* s_nb,
                             int* s_sl, int node, int par, int half, int lane, int it) {
    int tx, ty, tz;
    lane_cell_slab(lane, par, half, (__ldg(ninfo + node) >> NI_SLAB_SHIFT) & 3, tx, ty, tz);
    double lb[16];
    float lbh[16], lbl[16];
    bool nz = false;
    if constexpr (EMU) {
        const float2* src = p.Lf + static_cast<size_t>(node) * NRED * NCELL + tx + 8 * ty + 64 * tz;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const float2 v = __ldg(src + q * NCELL);
            lbh[q] = v.x;
            lbl[q] = v.y;
            nz |= v.x != 0.0f;
        }
    } else {
        const double* src = p.Lrbar + static_cast<size_t>(node) * NRED * NCELL + tx + 8 * ty + 64 * tz;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            lb[q] = __ldg(src + q * NCELL);
            nz |= lb[q] != 0.0;
        }
    }
    if (!__any_sync(0xffffffffu, nz)) return;     // targets without an adjoint contribute nothing
    if (lane < 27) {
        const int2 e = __ldg(nbr + static_cast<size_t>(node) * 27 + lane);
        s_nb[lane] = e;
        s_sl[lane] = (p.nslot != nullptr && (e.y & 3) != K_NONE) ? __ldg(p.nslot + static_cast<size_t>(node) * 27 + lane)
                                                                 : -1;
    }
    __syncwarp();
    const int info = __ldg(ninfo + node);
    const int level = info & 0xff;
    const bool leafT = (info >> 8) & 1;
    if (level > 0 && leafT) {
        // by reflection class (see the forward); refined near sources over the near list
        const bool xpath = p.Sbar != nullptr && (info & NI_XMASS);
        const int* cf = p.L.lists + p.L.cf_off + par * p.L.cf_stride;
        const int* cn = p.L.lists + p.L.cn_off;
        if constexpr (EMU) {
            // one inlined copy of the double-float class scatter for the far
            // and the near class lists (as in the forward)
#pragma unroll 1
            for (int sgm = 0; sgm < 2; ++sgm) {
                int zo[8], xo[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    zo[k] = sgm ? p.L.cn_z[k] : p.L.cf_z[k];
                    xo[k] = sgm ? p.L.cn_x[k] : p.L.cf_x[k];
                }
                walk_classes_scatter_all<EMU>(sgm ? cn : cf, zo, xo, xpath, tx, ty, tz, s_nb, s_sl, p, lb, lbh, lbl, it);
            }
        } else {
            walk_classes_scatter_all<EMU>(cf, p.L.cf_z, p.L.cf_x, xpath, tx, ty, tz, s_nb, s_sl, p, lb, lbh, lbl, it);
        }
        cf += p.L.cf_z[7];
        if constexpr (EMU) {
#pragma unroll 1
            for (int sgm = 0; sgm < 2; ++sgm)
                walk_scatter<true, false, EMU>(sgm ? cn + p.L.cn_z[7] : cf, sgm ? p.L.cn_pairs : p.L.cf_pairs, tx, ty, tz,
                                               s_nb, p, lb, lbh, lbl, it);
            walk_scatter<false, false, EMU>(cf + p.L.cf_pairs, p.L.cf_singles, tx, ty, tz, s_nb, p, lb, lbh, lbl, it);
        } else {
            walk_scatter<true, false, EMU>(cf, p.L.cf_pairs, tx, ty, tz, s_nb, p, lb, lbh, lbl, it);
            walk_scatter<false, false, EMU>(cf + p.L.cf_pairs, p.L.cf_singles, tx, ty, tz, s_nb, p, lb, lbh, lbl, it);
            walk_classes_scatter_all<EMU>(cn, p.L.cn_z, p.L.cn_x, xpath, tx, ty, tz, s_nb, s_sl, p, lb, lbh, lbl, it);
            walk_scatter<true, false, EMU>(cn + p.L.cn_z[7], p.L.cn_pairs, tx, ty, tz, s_nb, p, lb, lbh, lbl, it);
        }
        if (__any_sync(0xffffffffu, lane < 27 && (s_nb[lane < 27 ? lane : 0].y & 3) == K_MULTI))
            walk_scatter<true, true, EMU, false>(p.L.lists + p.L.near_off, p.L.near_len, tx, ty, tz, s_nb, p, lb, lbh,
                                                 lbl, it);
        return;
    }
    if (level == 0) {
        walk_scatter<true, false, EMU>(p.L.lists + p.L.root_off, p.L.root_len, tx, ty, tz, s_nb, p, lb, lbh, lbl, it);
    } else if (!EMU && !leafT) {
        // a non-leaf target: its point-mass sources paired along its axis
        const int A = (info >> NI_APAIR_SHIFT) & 3;
        if (A == 0)
            walk_scatter_apair_list<0>(par, tx, ty, tz, s_nb, p, lb, it);
        else if (A == 1)
            walk_scatter_apair_list<1>(par, tx, ty, tz, s_nb, p, lb, it);
        else
            walk_scatter_apair_list<2>(par, tx, ty, tz, s_nb, p, lb, it);
    } else {
        const int* lf = p.L.lists + par * p.L.far_len;
        walk_scatter<true, false, EMU>(lf, p.L.far_pairs, tx, ty, tz, s_nb, p, lb, lbh, lbl, it);
        walk_scatter<false, false, EMU>(lf + p.L.far_pairs, p.L.far_len - p.L.far_pairs, tx, ty, tz, s_nb, p, lb, lbh,
                                        lbl, it);
    }
    if (leafT) walk_scatter<true, true, EMU>(p.L.lists + p.L.near_off, p.L.near_len, tx, ty, tz, s_nb, p, lb, lbh,
                                            lbl, it);
}

__global__ void __launch_bounds__(256) scatter_adjoint_kernel(const ScatParams p, int persistent) {
    __shared__ int2 s_nb[8][27];
    __shared__ int s_sl[8][27];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    int it = blockIdx.x * wpb + warp;
    for (;;) {
        if (persistent) {
            int v = 0;
            if (lane == 0) v = atomicAdd(p.counter, 1);
            it = __shfl_sync(0xffffffffu, v, 0);
        }
        if (it >= p.n_items) break;
        const int item = __ldg(p.items + it);
        scatter_item(p, p.nbr, p.ninfo, s_nb[warp], s_sl[warp], item >> 4, (item >> 1) & 7, item & 1, lane, it);
        __syncwarp();
        if (!persistent) break;
    }
}

// ---------------------------------------------------------------------------
// prescaling (once per cell)
// ---------------------------------------------------------------------------

// Mhat (reduced): (-1)^m/m! * multiplicity * h^-m * M, zz-traces folded.
__global__ void prescale_moments_kernel(const PrepParams p) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p.n_list * NCELL) return;
    const int node = __ldg(p.nodes + t / NCELL), cell = t % NCELL;
    const double h1 = p.hinv[__ldg(p.ninfo + node) & 0xff], h2 = h1 * h1, h3 = h2 * h1;
    const double* M = p.src + static_cast<size_t>(node) * NCOMP * NCELL + cell;
    double v[20];
#pragma unroll
    for (int q = 0; q < 20; ++q) v[q] = M[q * NCELL];
    const double Mxx = 0.5 * h2 * v[4], Myy = 0.5 * h2 * v[7], Mzz = 0.5 * h2 * v[9];
    const double a6 = -h3 / 6.0, a2 = -0.5 * h3;
    const double Mxzz = a2 * v[15], Myzz = a2 * v[18], Mzzz = a6 * v[19];
    double r[16];
    r[0] = v[0];
    r[1] = -h1 * v[1];
    r[2] = -h1 * v[2];
    r[3] = -h1 * v[3];
    r[4] = Mxx - Mzz;
    r[5] = h2 * v[5];
    r[6] = h2 * v[6];
    r[7] = Myy - Mzz;
    r[8] = h2 * v[8];
    r[9] = a6 * v[10] - Mxzz;
    r[10] = a2 * v[11] - Myzz;
    r[11] = a2 * v[12] - Mzzz;
    r[12] = a2 * v[13] - Mxzz;
    r[13] = -h3 * v[14];
    r[14] = a6 * v[16] - Myzz;
    r[15] = a2 * v[17] - Mzzz;
    double* o = p.dst + static_cast<size_t>(node) * NRED * NCELL + cell;
#pragma unroll
    for (int q = 0; q < 16; ++q) o[q * NCELL] = r[q];
}

// Lrbar (reduced): h^-(n+1) * Lbar, with the adjoint of the derived
// components zz, xzz, yzz, zzz folded in.
__global__ void prescale_adjoint_kernel(const PrepParams p) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p.n_list * NCELL) return;
    const int node = __ldg(p.nodes + t / NCELL), cell = t % NCELL;
    const double h1 = p.hinv[__ldg(p.ninfo + node) & 0xff], h2 = h1 * h1, h3 = h2 * h1, h4 = h2 * h2;
    const double* Lb = p.src + static_cast<size_t>(node) * NCOMP * NCELL + cell;
    double v[20];
#pragma unroll
    for (int q = 0; q < 20; ++q) v[q] = Lb[q * NCELL];
    double r[16];
    r[0] = h1 * v[0];
    r[1] = h2 * v[1];
    r[2] = h2 * v[2];
    r[3] = h2 * v[3];
    r[4] = h3 * (v[4] - v[9]);
    r[5] = h3 * v[5];
    r[6] = h3 * v[6];
    r[7] = h3 * (v[7] - v[9]);
    r[8] = h3 * v[8];
    r[9] = h4 * (v[10] - v[15]);
    r[10] = h4 * (v[11] - v[18]);
    r[11] = h4 * (v[12] - v[19]);
    r[12] = h4 * (v[13] - v[15]);
    r[13] = h4 * v[14];
    r[14] = h4 * (v[16] - v[18]);
    r[15] = h4 * (v[17] - v[19]);
    double* o = p.dst + static_cast<size_t>(node) * NRED * NCELL + cell;
#pragma unroll
    for (int q = 0; q < 16; ++q) o[q * NCELL] = r[q];
}

// mbar[P][c] += sum over its virtual descendant cells of 8^-d vbar
__global__ void restrict_virtual_kernel(const double* __restrict__ vbar, const int* __restrict__ vmap,
                                        int n_rows, double* __restrict__ mbar) {
    // vmap: [n_rows] row headers (target P*512+c), then [n_rows+1] offsets,
    // then entries (v*512 + s) | d << 28
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_rows) return;
    const int* ptr = vmap + n_rows;
    const int* ent = vmap + 2 * n_rows + 1;
    double acc = 0.0;
    for (int k = ptr[t]; k < ptr[t + 1]; ++k) {
        const int e = ent[k];
        acc += vbar[e & 0x0fffffff] * pow2i(-3 * (e >> 28));
    }
    mbar[vmap[t]] += acc;
}

// ---------------------------------------------------------------------------
// moments
// ---------------------------------------------------------------------------

// Moments in a dense [4][4][4] exponent array (entries with a+b+c <= 3 used);
// every loop bound below is a compile-time constant, so after unrolling all
// indices are static and the arrays live in registers.
#define OT_STORAGE_EXPONENTS                                                                       \
    {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 2, 0}, {0, 1, 1}, \
     {0, 0, 2}, {3, 0, 0}, {2, 1, 0}, {2, 0, 1}, {1, 2, 0}, {1, 1, 1}, {1, 0, 2}, {0, 3, 0}, {0, 2, 1}, \
     {0, 1, 2}, {0, 0, 3}}

struct Dense4 {
    double v[4][4][4];
};

__device__ __forceinline__ void to_dense(const double* __restrict__ src, Dense4& D) {
    constexpr int E[20][3] = OT_STORAGE_EXPONENTS;
#pragma unroll
    for (int q = 0; q < 20; ++q) D.v[E[q][0]][E[q][1]][E[q][2]] = src[q * NCELL];
}

__device__ __forceinline__ void from_dense(const Dense4& D, double* __restrict__ out, bool add) {
    constexpr int E[20][3] = OT_STORAGE_EXPONENTS;
#pragma unroll
    for (int q = 0; q < 20; ++q) {
        const double x = D.v[E[q][0]][E[q][1]][E[q][2]];
        out[q * NCELL] = add ? out[q * NCELL] + x : x;
    }
}

// binomial shift of raw moments along one axis by d:
//   out[..a..] = sum_{j <= a} C(a, j) d^(a-j) in[..j..]
template <int AXIS>
__device__ __forceinline__ void shift1(Dense4& D, double d) {
    const double d2 = d * d, d3 = d2 * d;
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; p + q < 4; ++q) {
            double m[4];
#pragma unroll
            for (int a = 0; a + p + q < 4; ++a)
                m[a] = (AXIS == 0) ? D.v[a][p][q] : (AXIS == 1) ? D.v[p][a][q] : D.v[p][q][a];
            const int top = 3 - p - q;
            double o[4];
            o[0] = m[0];
            if (top >= 1) o[1] = m[1] + d * m[0];
            if (top >= 2) o[2] = m[2] + 2.0 * d * m[1] + d2 * m[0];
            if (top >= 3) o[3] = m[3] + 3.0 * d * m[2] + 3.0 * d2 * m[1] + d3 * m[0];
#pragma unroll
            for (int a = 0; a + p + q < 4; ++a) {
                if (AXIS == 0) D.v[a][p][q] = o[a];
                else if (AXIS == 1) D.v[p][a][q] = o[a];
                else D.v[p][q][a] = o[a];
            }
        }
}

// transpose of shift1
template <int AXIS>
__device__ __forceinline__ void shift1_t(Dense4& D, double d) {
    const double d2 = d * d, d3 = d2 * d;
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; p + q < 4; ++q) {
            double g[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
            for (int a = 0; a + p + q < 4; ++a)
                g[a] = (AXIS == 0) ? D.v[a][p][q] : (AXIS == 1) ? D.v[p][a][q] : D.v[p][q][a];
            const int top = 3 - p - q;
            double o[4];
            o[0] = g[0] + (top >= 1 ? d * g[1] : 0.0) + (top >= 2 ? d2 * g[2] : 0.0) + (top >= 3 ? d3 * g[3] : 0.0);
            o[1] = (top >= 1 ? g[1] : 0.0) + (top >= 2 ? 2.0 * d * g[2] : 0.0) + (top >= 3 ? 3.0 * d2 * g[3] : 0.0);
            o[2] = (top >= 2 ? g[2] : 0.0) + (top >= 3 ? 3.0 * d * g[3] : 0.0);
            o[3] = (top >= 3 ? g[3] : 0.0);
#pragma unroll
            for (int a = 0; a + p + q < 4; ++a) {
                if (AXIS == 0) D.v[a][p][q] = o[a];
                else if (AXIS == 1) D.v[p][a][q] = o[a];
                else D.v[p][q][a] = o[a];
            }
        }
}

// One-dimensional Taylor shift of a degree-3 local expansion (coefficients
// are derivatives): out[..a..] = sum_{k <= 3 - |rest| - a} in[..a+k..] d^k / k!
template <int AXIS>
__device__ __forceinline__ void lshift1(Dense4& D, double d) {
    const double d2h = 0.5 * d * d, d3s = d * d * d / 6.0;
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; p + q < 4; ++q) {
            double m[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
            for (int a = 0; a + p + q < 4; ++a)
                m[a] = (AXIS == 0) ? D.v[a][p][q] : (AXIS == 1) ? D.v[p][a][q] : D.v[p][q][a];
            const int top = 3 - p - q;
            double o[4];
            o[0] = m[0] + (top >= 1 ? d * m[1] : 0.0) + (top >= 2 ? d2h * m[2] : 0.0) + (top >= 3 ? d3s * m[3] : 0.0);
            o[1] = m[1] + (top >= 2 ? d * m[2] : 0.0) + (top >= 3 ? d2h * m[3] : 0.0);
            o[2] = m[2] + (top >= 3 ? d * m[3] : 0.0);
            o[3] = m[3];
#pragma unroll
            for (int a = 0; a + p + q < 4; ++a) {
                if (AXIS == 0) D.v[a][p][q] = o[a];
                else if (AXIS == 1) D.v[p][a][q] = o[a];
                else D.v[p][q][a] = o[a];
            }
        }
}

// transpose of lshift1
template <int AXIS>
__device__ __forceinline__ void lshift1_t(Dense4& D, double d) {
    const double d2h = 0.5 * d * d, d3s = d * d * d / 6.0;
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; p + q < 4; ++q) {
            double g[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
            for (int a = 0; a + p + q < 4; ++a)
                g[a] = (AXIS == 0) ? D.v[a][p][q] : (AXIS == 1) ? D.v[p][a][q] : D.v[p][q][a];
            const int top = 3 - p - q;
            double o[4];
            o[0] = g[0];
            o[1] = (top >= 1) ? g[1] + d * g[0] : 0.0;
            o[2] = (top >= 2) ? g[2] + d * g[1] + d2h * g[0] : 0.0;
            o[3] = (top >= 3) ? g[3] + d * g[2] + d2h * g[1] + d3s * g[0] : 0.0;
#pragma unroll
            for (int a = 0; a + p + q < 4; ++a) {
                if (AXIS == 0) D.v[a][p][q] = o[a];
                else if (AXIS == 1) D.v[p][a][q] = o[a];
                else D.v[p][q][a] = o[a];
            }
        }
}

// L2L down-pass of one level: every child cell of the listed parents adds
// the parent cell's local expansion shifted to its own centre
__global__ void l2l_kernel(double* __restrict__ L, const int* __restrict__ parents, int n_list,
                           const int* __restrict__ children, const int* __restrict__ ninfo,
                           const double* __restrict__ hinv) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_list * 8 * NCELL) return;
    const int k = t / (8 * NCELL);
    const int oct = (t / NCELL) % 8, ccell = t % NCELL;
    const int P = parents[k];
    const int C = children[8 * k + oct];
    const int cx = (oct & 1) * 8 + (ccell & 7), cy = ((oct >> 1) & 1) * 8 + ((ccell >> 3) & 7),
              cz = (oct >> 2) * 8 + (ccell >> 6);
    const int pcell = (cx >> 1) + 8 * (cy >> 1) + 64 * (cz >> 1);
    const double hc = 0.5 / hinv[ninfo[P] & 0xff];
    Dense4 v;
    to_dense(L + static_cast<size_t>(P) * NCOMP * NCELL + pcell, v);
    lshift1<0>(v, ((cx & 1) - 0.5) * hc);
    lshift1<1>(v, ((cy & 1) - 0.5) * hc);
    lshift1<2>(v, ((cz & 1) - 0.5) * hc);
    from_dense(v, L + static_cast<size_t>(C) * NCOMP * NCELL + ccell, true);
}

// transpose of one level of the down-pass: every parent cell adds the
// transposed shifts of its 8 child cells' adjoints
__global__ void l2l_adjoint_kernel(double* __restrict__ Lb, const int* __restrict__ parents, int n_list,
                                   const int* __restrict__ children, const int* __restrict__ ninfo,
                                   const double* __restrict__ hinv) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_list * NCELL) return;
    const int k = t / NCELL, cell = t % NCELL;
    const int P = parents[k];
    const int gx = cell & 7, gy = (cell >> 3) & 7, gz = cell >> 6;
    const double hc = 0.5 / hinv[ninfo[P] & 0xff];
    Dense4 acc;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc.v[a][b][c] = 0.0;
#pragma unroll 1
    for (int b = 0; b < 8; ++b) {
        const int bx = b & 1, by = (b >> 1) & 1, bz = b >> 2;
        const int cx = 2 * gx + bx, cy = 2 * gy + by, cz = 2 * gz + bz;
        const int C = children[8 * k + (cx >> 3) + 2 * (cy >> 3) + 4 * (cz >> 3)];
        Dense4 v;
        to_dense(Lb + static_cast<size_t>(C) * NCOMP * NCELL + (cx & 7) + 8 * (cy & 7) + 64 * (cz & 7), v);
        lshift1_t<2>(v, (bz - 0.5) * hc);
        lshift1_t<1>(v, (by - 0.5) * hc);
        lshift1_t<0>(v, (bx - 0.5) * hc);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int bb = 0; a + bb < 4; ++bb)
#pragma unroll
                for (int c = 0; a + bb + c < 4; ++c) acc.v[a][bb][c] += v.v[a][bb][c];
    }
    from_dense(acc, Lb + static_cast<size_t>(P) * NCOMP * NCELL + cell, true);
}

__global__ void cube_moments_kernel(const double* __restrict__ rho, double* __restrict__ M, double* __restrict__ m,
                                    const int* __restrict__ nodes, int n_list, const int* __restrict__ ninfo,
                                    const double* __restrict__ hinv) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_list * NCELL) return;
    const int node = nodes[t / NCELL], cell = t % NCELL;
    const double h = 1.0 / hinv[ninfo[node] & 0xff];
    const double r = rho[static_cast<size_t>(node) * NCELL + cell];
    const double m0 = r * h * h * h;
    const double q2 = m0 * h * h / 12.0;
    double* o = M + static_cast<size_t>(node) * NCOMP * NCELL + cell;
    for (int q = 0; q < 20; ++q) o[q * NCELL] = 0.0;
    o[0] = m0;
    o[4 * NCELL] = q2;
    o[7 * NCELL] = q2;
    o[9 * NCELL] = q2;
    m[static_cast<size_t>(node) * NCELL + cell] = m0;
}

// parents[k]: node index; children[8k + b]: child node of octant b (x fastest)
__global__ void m2m_kernel(double* __restrict__ M, double* __restrict__ m, const int* __restrict__ parents,
                           int n_list, const int* __restrict__ children, const int* __restrict__ ninfo,
                           const double* __restrict__ hinv) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_list * NCELL) return;
    const int k = t / NCELL, cell = t % NCELL;
    const int P = parents[k];
    const int gx = cell & 7, gy = (cell >> 3) & 7, gz = cell >> 6;
    const double hc = 0.5 / hinv[ninfo[P] & 0xff];
    Dense4 acc;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc.v[a][b][c] = 0.0;
#pragma unroll 1
    for (int b = 0; b < 8; ++b) {
        const int bx = b & 1, by = (b >> 1) & 1, bz = b >> 2;
        const int cx = 2 * gx + bx, cy = 2 * gy + by, cz = 2 * gz + bz;   // in [0, 16)
        const int oct = (cx >> 3) + 2 * (cy >> 3) + 4 * (cz >> 3);
        const int C = children[8 * k + oct];
        const int ccell = (cx & 7) + 8 * (cy & 7) + 64 * (cz & 7);
        Dense4 v;
        to_dense(M + static_cast<size_t>(C) * NCOMP * NCELL + ccell, v);
        shift1<0>(v, (bx - 0.5) * hc);
        shift1<1>(v, (by - 0.5) * hc);
        shift1<2>(v, (bz - 0.5) * hc);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int bb = 0; a + bb < 4; ++bb)
#pragma unroll
                for (int c = 0; a + bb + c < 4; ++c) acc.v[a][bb][c] += v.v[a][bb][c];
    }
    from_dense(acc, M + static_cast<size_t>(P) * NCOMP * NCELL + cell, false);
    m[static_cast<size_t>(P) * NCELL + cell] = acc.v[0][0][0];
}

__global__ void moments_adjoint_init_kernel(const double* __restrict__ Mbar, const double* __restrict__ mbar,
                                            double* __restrict__ Mb, int n) {
    const size_t t = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const size_t total = static_cast<size_t>(n) * NCOMP * NCELL;
    if (t >= total) return;
    double v = Mbar ? Mbar[t] : 0.0;
    const size_t comp = (t / NCELL) % NCOMP;
    if (comp == 0 && mbar) v += mbar[(t / (NCOMP * NCELL)) * NCELL + t % NCELL];
    Mb[t] = v;
}

// children's Mb += transpose of the parent's M2M applied to the parent's Mb
__global__ void m2m_adjoint_kernel(double* __restrict__ Mb, const int* __restrict__ parents, int n_list,
                                   const int* __restrict__ children, const int* __restrict__ ninfo,
                                   const double* __restrict__ hinv) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_list * 8 * NCELL) return;
    const int k = t / (8 * NCELL);
    const int oct = (t / NCELL) % 8, ccell = t % NCELL;
    const int P = parents[k];
    const int C = children[8 * k + oct];
    const int cx = (oct & 1) * 8 + (ccell & 7), cy = ((oct >> 1) & 1) * 8 + ((ccell >> 3) & 7),
              cz = (oct >> 2) * 8 + (ccell >> 6);
    const int pcell = (cx >> 1) + 8 * (cy >> 1) + 64 * (cz >> 1);
    const double hc = 0.5 / hinv[ninfo[P] & 0xff];
    Dense4 v;
    to_dense(Mb + static_cast<size_t>(P) * NCOMP * NCELL + pcell, v);
    shift1_t<2>(v, ((cz & 1) - 0.5) * hc);
    shift1_t<1>(v, ((cy & 1) - 0.5) * hc);
    shift1_t<0>(v, ((cx & 1) - 0.5) * hc);
    from_dense(v, Mb + static_cast<size_t>(C) * NCOMP * NCELL + ccell, true);
}

__global__ void cube_adjoint_kernel(const double* __restrict__ Mb, double* __restrict__ rhobar,
                                    const int* __restrict__ nodes, int n_list, const int* __restrict__ ninfo,
                                    const double* __restrict__ hinv) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_list * NCELL) return;
    const int node = nodes[t / NCELL], cell = t % NCELL;
    const double h = 1.0 / hinv[ninfo[node] & 0xff];
    const double* b = Mb + static_cast<size_t>(node) * NCOMP * NCELL + cell;
    const double h3 = h * h * h;
    rhobar[static_cast<size_t>(node) * NCELL + cell] =
        b[0] * h3 + (b[4 * NCELL] + b[7 * NCELL] + b[9 * NCELL]) * (h3 * h * h / 12.0);
}

// ---------------------------------------------------------------------------
// explicit (centre-of-mass) expansion centres
//
// Cells of non-leaf sub-grids are expanded about the centres C; cells of leaf
// sub-grids and virtual descendants are uniform cubes about their geometric
// centres (C is never read for them).  The passes work in the units of the
// target level's h exactly as the table path does (same prescaling, same
// epilogue): a pair whose two centres are geometric is at an integer offset
// and reads the derivative table; any other pair evaluates the derivatives
// at its own R/h.
// ---------------------------------------------------------------------------

// geometric centre coordinate of local cell s (in [-8, 16)) of a sub-grid
// whose first cell is at integer position org: (org + s + 1/2) h
__device__ __forceinline__ double geo_centre(int org, int s, double h) { return (org + s + 0.5) * h; }

__global__ void geometric_centres_kernel(double* __restrict__ C, const int* __restrict__ nodes, int n_list,
                                         const int* __restrict__ ninfo, const int* __restrict__ ncoord, double h0) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_list * NCELL) return;
    const int node = nodes[t / NCELL], cell = t % NCELL;
    const double h = ldexp(h0, -(ninfo[node] & 0xff));
    const int loc[3] = {cell & 7, (cell >> 3) & 7, cell >> 6};
    for (int a = 0; a < 3; ++a)
        C[(static_cast<size_t>(node) * 3 + a) * NCELL + cell] = geo_centre(8 * ncoord[3 * node + a], loc[a], h);
}

// parent cell: centre = mass-weighted mean of the 8 children's centres
// (geometric if the mass is exactly zero), moments = the children's moments
// shifted binomially to it
__global__ void m2m_com_kernel(double* __restrict__ M, double* __restrict__ m, double* __restrict__ C,
                               const int* __restrict__ parents, int n_list, const int* __restrict__ children,
                               const int* __restrict__ ninfo, const int* __restrict__ ncoord, double h0) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_list * NCELL) return;
    const int k = t / NCELL, cell = t % NCELL;
    const int P = parents[k];
    const int g[3] = {cell & 7, (cell >> 3) & 7, cell >> 6};
    double mass = 0.0, w[3] = {0.0, 0.0, 0.0};
#pragma unroll 1
    for (int b = 0; b < 8; ++b) {
        const int cx = 2 * g[0] + (b & 1), cy = 2 * g[1] + ((b >> 1) & 1), cz = 2 * g[2] + (b >> 2);
        const int cn = children[8 * k + (cx >> 3) + 2 * (cy >> 3) + 4 * (cz >> 3)];
        const int cc = (cx & 7) + 8 * (cy & 7) + 64 * (cz & 7);
        const double mc = M[static_cast<size_t>(cn) * NCOMP * NCELL + cc];
        mass += mc;
        for (int a = 0; a < 3; ++a) w[a] += mc * C[(static_cast<size_t>(cn) * 3 + a) * NCELL + cc];
    }
    double X[3];
    const double h = ldexp(h0, -(ninfo[P] & 0xff));
    for (int a = 0; a < 3; ++a) X[a] = (mass != 0.0) ? w[a] / mass : geo_centre(8 * ncoord[3 * P + a], g[a], h);
    Dense4 acc;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc.v[a][b][c] = 0.0;
#pragma unroll 1
    for (int b = 0; b < 8; ++b) {
        const int cx = 2 * g[0] + (b & 1), cy = 2 * g[1] + ((b >> 1) & 1), cz = 2 * g[2] + (b >> 2);
        const int cn = children[8 * k + (cx >> 3) + 2 * (cy >> 3) + 4 * (cz >> 3)];
        const int cc = (cx & 7) + 8 * (cy & 7) + 64 * (cz & 7);
        Dense4 v;
        to_dense(M + static_cast<size_t>(cn) * NCOMP * NCELL + cc, v);
        const double* Cc = C + static_cast<size_t>(cn) * 3 * NCELL + cc;
        shift1<0>(v, Cc[0] - X[0]);
        shift1<1>(v, Cc[NCELL] - X[1]);
        shift1<2>(v, Cc[2 * NCELL] - X[2]);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int bb = 0; a + bb < 4; ++bb)
#pragma unroll
                for (int c = 0; a + bb + c < 4; ++c) acc.v[a][bb][c] += v.v[a][bb][c];
    }
    from_dense(acc, M + static_cast<size_t>(P) * NCOMP * NCELL + cell, false);
    m[static_cast<size_t>(P) * NCELL + cell] = acc.v[0][0][0];
    for (int a = 0; a < 3; ++a) C[(static_cast<size_t>(P) * 3 + a) * NCELL + cell] = X[a];
}

// centre of one cell of `node`: C for non-leaf sub-grids, geometric otherwise
__device__ __forceinline__ void cell_centre(const double* __restrict__ C, const int* __restrict__ ninfo,
                                            const int* __restrict__ ncoord, double h0, int node, int cell,
                                            double (&X)[3]) {
    const int info = ninfo[node];
    if ((info >> 8) & 1) {
        const double h = ldexp(h0, -(info & 0xff));
        X[0] = geo_centre(8 * ncoord[3 * node], cell & 7, h);
        X[1] = geo_centre(8 * ncoord[3 * node + 1], (cell >> 3) & 7, h);
        X[2] = geo_centre(8 * ncoord[3 * node + 2], cell >> 6, h);
    } else {
        const double* c = C + static_cast<size_t>(node) * 3 * NCELL + cell;
        X[0] = c[0];
        X[1] = c[NCELL];
        X[2] = c[2 * NCELL];
    }
}

__global__ void l2l_com_kernel(double* __restrict__ L, const double* __restrict__ C, const int* __restrict__ parents,
                               int n_list, const int* __restrict__ children, const int* __restrict__ ninfo,
                               const int* __restrict__ ncoord, double h0) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_list * 8 * NCELL) return;
    const int k = t / (8 * NCELL);
    const int oct = (t / NCELL) % 8, ccell = t % NCELL;
    const int P = parents[k];
    const int Cn = children[8 * k + oct];
    const int cx = (oct & 1) * 8 + (ccell & 7), cy = ((oct >> 1) & 1) * 8 + ((ccell >> 3) & 7),
              cz = (oct >> 2) * 8 + (ccell >> 6);
    const int pcell = (cx >> 1) + 8 * (cy >> 1) + 64 * (cz >> 1);
    double Xc[3], Xp[3];
    cell_centre(C, ninfo, ncoord, h0, Cn, ccell, Xc);
    cell_centre(C, ninfo, ncoord, h0, P, pcell, Xp);
    Dense4 v;
    to_dense(L + static_cast<size_t>(P) * NCOMP * NCELL + pcell, v);
    lshift1<0>(v, Xc[0] - Xp[0]);
    lshift1<1>(v, Xc[1] - Xp[1]);
    lshift1<2>(v, Xc[2] - Xp[2]);
    from_dense(v, L + static_cast<size_t>(Cn) * NCOMP * NCELL + ccell, true);
}

// transpose of l2l_com_kernel (centres held fixed)
__global__ void l2l_com_adjoint_kernel(double* __restrict__ Lb, const double* __restrict__ C,
                                       const int* __restrict__ parents, int n_list,
                                       const int* __restrict__ children, const int* __restrict__ ninfo,
                                       const int* __restrict__ ncoord, double h0) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_list * NCELL) return;
    const int k = t / NCELL, cell = t % NCELL;
    const int P = parents[k];
    const int gx = cell & 7, gy = (cell >> 3) & 7, gz = cell >> 6;
    double Xp[3];
    cell_centre(C, ninfo, ncoord, h0, P, cell, Xp);
    Dense4 acc;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc.v[a][b][c] = 0.0;
#pragma unroll 1
    for (int b = 0; b < 8; ++b) {
        const int cx = 2 * gx + (b & 1), cy = 2 * gy + ((b >> 1) & 1), cz = 2 * gz + (b >> 2);
        const int Cn = children[8 * k + (cx >> 3) + 2 * (cy >> 3) + 4 * (cz >> 3)];
        const int ccell = (cx & 7) + 8 * (cy & 7) + 64 * (cz & 7);
        double Xc[3];
        cell_centre(C, ninfo, ncoord, h0, Cn, ccell, Xc);
        Dense4 v;
        to_dense(Lb + static_cast<size_t>(Cn) * NCOMP * NCELL + ccell, v);
        lshift1_t<2>(v, Xc[2] - Xp[2]);
        lshift1_t<1>(v, Xc[1] - Xp[1]);
        lshift1_t<0>(v, Xc[0] - Xp[0]);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int bb = 0; a + bb < 4; ++bb)
#pragma unroll
                for (int c = 0; a + bb + c < 4; ++c) acc.v[a][bb][c] += v.v[a][bb][c];
    }
    from_dense(acc, Lb + static_cast<size_t>(P) * NCOMP * NCELL + cell, true);
}

// R/h for a pair whose source sits at X: lanes without a source of the class
// being contracted get a unit separation (their terms are zero)
__device__ __forceinline__ void scaled_sep(bool has, const double (&XA)[3], const double (&X)[3], double hinv,
                                           double& rx, double& ry, double& rz) {
    if (has) {
        rx = (XA[0] - X[0]) * hinv;
        ry = (XA[1] - X[1]) * hinv;
        rz = (XA[2] - X[2]) * hinv;
    } else {
        rx = 0.0;
        ry = 0.0;
        rz = 1.0;
    }
}

// One stencil segment of a target with explicit centres.  PAIRED: each entry
// o stands for the sources at t + o and t - o.
template <int MODE, bool PAIRED, bool NEAR = false, bool PM = true>
__device__ __forceinline__ void walk_forward_com(const int* __restrict__ list, int len, bool angular, bool leafT,
                                                 int tx, int ty, int tz, const int2* __restrict__ s_nb,
                                                 const FwdParams& p, const int (&org)[3], double h, double hinv,
                                                 const double (&XA)[3], double (&a)[16], double (&c)[3],
                                                 double (&t4)[9], int item) {
    constexpr int NS = PAIRED ? 2 : 1;
    for (int k = 0; k < len; ++k) {
        const int po = __ldg(list + k);
        const int ox = (po & 0xff) - 8, oy = ((po >> 8) & 0xff) - 8, oz = ((po >> 16) & 0xff) - 8;
        int sx[NS], sy[NS], sz[NS], kd[NS];
        int2 e[NS];
#pragma unroll
        for (int sd = 0; sd < NS; ++sd) {
            const int sg = sd ? -1 : 1;
            sx[sd] = tx + sg * ox;
            sy[sd] = ty + sg * oy;
            sz[sd] = tz + sg * oz;
            e[sd] = s_nb[nb_index(sx[sd], sy[sd], sz[sd])];
            kd[sd] = checked_kind(p, e[sd], item);
        }
        if (MODE & 2) {
            if (leafT) {
                // both centres geometric: R/h = -o, the table row (paired as on the table path)
                bool mono = kd[0] >= K_LEAF;
                if (PAIRED) mono = mono || kd[NS - 1] >= K_LEAF;
                if (PM && __any_sync(0xffffffffu, mono)) {
                    const double mp = source_mass(p, e[0], kd[0], sx[0], sy[0], sz[0]);
                    double d[36];
                    load_row16(d, p.Dt, offset_row(ox, oy, oz));
                    if (PAIRED) {
                        const double mm = source_mass(p, e[NS - 1], kd[NS - 1], sx[NS - 1], sy[NS - 1], sz[NS - 1]);
                        ot_mono_fwd_pair(a, mp + mm, mp - mm, d);
                    } else {
                        ot_mono_fwd(a, mp, d);
                    }
                }
                if (PAIRED && NEAR) {
                    // near sources in refined sub-grids (all centres geometric)
                    const bool rp = kd[0] == K_MULTI, rm = kd[NS - 1] == K_MULTI;
                    if (__any_sync(0xffffffffu, rp || rm))
                        refined_near_fwd(p, ox, oy, oz, e[0], rp, sx[0], sy[0], sz[0], e[NS - 1], rm, sx[NS - 1],
                                         sy[NS - 1], sz[NS - 1], a, item);
                }
            } else {
#pragma unroll
                for (int sd = 0; sd < NS; ++sd) {
                    const bool mono = kd[sd] >= K_LEAF;
                    if (!__any_sync(0xffffffffu, mono)) continue;
                    const double X[3] = {geo_centre(org[0], sx[sd], h), geo_centre(org[1], sy[sd], h),
                                         geo_centre(org[2], sz[sd], h)};
                    double rx, ry, rz, d[36];
                    scaled_sep(mono, XA, X, hinv, rx, ry, rz);
                    ot_deriv16_at(rx, ry, rz, d);
                    ot_mono_fwd(a, source_mass(p, e[sd], kd[sd], sx[sd], sy[sd], sz[sd]), d);
                }
            }
        }
        if ((MODE & 1) && !NEAR) {
#pragma unroll
            for (int sd = 0; sd < NS; ++sd) {
                const bool multi = kd[sd] == K_MULTI;
                if (!__any_sync(0xffffffffu, multi)) continue;
                double X[3] = {0.0, 0.0, 0.0};
                if (multi) {
                    const double* cb = p.C + static_cast<size_t>(e[sd].x) * 3 * NCELL + (sx[sd] & 7) +
                                       8 * (sy[sd] & 7) + 64 * (sz[sd] & 7);
                    X[0] = cb[0];
                    X[1] = cb[NCELL];
                    X[2] = cb[2 * NCELL];
                }
                double rx, ry, rz, d[36];
                scaled_sep(multi, XA, X, hinv, rx, ry, rz);
                if (angular) ot_deriv31_at(rx, ry, rz, d);
                else ot_deriv19_at(rx, ry, rz, d);
                double r[16];
                source_moments(p, e[sd], multi, sx[sd], sy[sd], sz[sd], r);
                ot_multi_fwd(a, r, d);
                if (angular) ot_angular_fwd(c, t4, r, r[0], d);
            }
        }
    }
}

template <int MODE>
__global__ void __launch_bounds__(256) forward_com_kernel(const FwdParams p) {
    __shared__ int2 s_nb[8][27];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    for (;;) {
        int v = 0;
        if (lane == 0) v = atomicAdd(p.counter, 1);
        const int it = __shfl_sync(0xffffffffu, v, 0);
        if (it >= p.n_items) break;
        const int item = __ldg(p.items + it);
        const int node = (item >> 4) & 0x3fffff, par = (item >> 1) & 7, half = item & 1;
        Chunk ch{(item >> 26) & 15, 1};
        int2 ci = make_int2(-1, 0);
        if (p.cinfo != nullptr) {
            ci = __ldg(p.cinfo + node);
            if (ci.x >= 0) ch.k = (ci.y & 15) + 1;
        }
        if (ch.c >= ch.k) {
            report(p.status, 6, it);
            continue;
        }
        if (lane < 27) s_nb[warp][lane] = __ldg(p.nbr + static_cast<size_t>(node) * 27 + lane);
        __syncwarp();
        const int info = __ldg(p.ninfo + node);
        const int level = info & 0xff;
        const bool leafT = (info >> 8) & 1;
        const double h = p.hreal[level], hinv = p.hinv[level];
        const int org[3] = {8 * __ldg(p.ncoord + 3 * node), 8 * __ldg(p.ncoord + 3 * node + 1),
                            8 * __ldg(p.ncoord + 3 * node + 2)};
        int tx, ty, tz;
        lane_cell(lane, par, half, tx, ty, tz);
        const int tcell = tx + 8 * ty + 64 * tz;
        double XA[3];
        if (leafT) {
            XA[0] = geo_centre(org[0], tx, h);
            XA[1] = geo_centre(org[1], ty, h);
            XA[2] = geo_centre(org[2], tz, h);
        } else {
            const double* ca = p.C + static_cast<size_t>(node) * 3 * NCELL + tcell;
            XA[0] = ca[0];
            XA[1] = ca[NCELL];
            XA[2] = ca[2 * NCELL];
        }
        double a[16], c[3], t4[9];
#pragma unroll
        for (int q = 0; q < 16; ++q) a[q] = 0.0;
#pragma unroll
        for (int q = 0; q < 3; ++q) c[q] = 0.0;
#pragma unroll
        for (int q = 0; q < 9; ++q) t4[q] = 0.0;
        if ((MODE & 2) && leafT && level > 0) {
            // leaf target: its point masses have geometric centres, so they run
            // the table path's class walk; multipole sources (refined
            // neighbours) and refined near sources keep the explicit-centre walk
            const int2* nb = s_nb[warp];
            DFAcc f;
            df_zero(f);
            const int* cf = p.L.lists + p.L.cf_off + par * p.L.cf_stride;
            walk_classes_fwd_all(cf, p.L.cf_z, p.L.cf_x, p.L.cf_xy, false, ch, tx, ty, tz, nb, nullptr, p, a, it);
            cf += p.L.cf_z[7];
            walk_forward<2, true, 0>(cf + ch.lo(p.L.cf_pairs), ch.n(p.L.cf_pairs), false, tx, ty, tz, nb, p, a, c,
                                     t4, f, it);
            cf += p.L.cf_pairs;
            walk_forward<2, false, 0>(cf + ch.lo(p.L.cf_singles), ch.n(p.L.cf_singles), false, tx, ty, tz, nb, p, a,
                                      c, t4, f, it);
            const int* cn = p.L.lists + p.L.cn_off;
            walk_classes_fwd_all(cn, p.L.cn_z, p.L.cn_x, p.L.cn_xy, false, ch, tx, ty, tz, nb, nullptr, p, a, it);
            cn += p.L.cn_z[7];
            walk_forward<2, true, 0>(cn + ch.lo(p.L.cn_pairs), ch.n(p.L.cn_pairs), false, tx, ty, tz, nb, p, a, c,
                                     t4, f, it);
            if (__any_sync(0xffffffffu, lane < 27 && (nb[lane < 27 ? lane : 0].y & 3) == K_MULTI)) {
                if constexpr ((MODE & 1) != 0) {
                    const int* lf = p.L.lists + par * p.L.far_len;
                    const int ns = p.L.far_len - p.L.far_pairs;
                    walk_forward_com<1, true>(lf + ch.lo(p.L.far_pairs), ch.n(p.L.far_pairs), false, true, tx, ty,
                                              tz, nb, p, org, h, hinv, XA, a, c, t4, it);
                    walk_forward_com<1, false>(lf + p.L.far_pairs + ch.lo(ns), ch.n(ns), false, true, tx, ty, tz,
                                               nb, p, org, h, hinv, XA, a, c, t4, it);
                }
                walk_forward_com<2, true, true, false>(p.L.lists + p.L.near_off + ch.lo(p.L.near_len),
                                                       ch.n(p.L.near_len), false, true, tx, ty, tz, nb, p, org, h,
                                                       hinv, XA, a, c, t4, it);
            }
        } else if (level == 0) {
            walk_forward_com<MODE, true>(p.L.lists + p.L.root_off + ch.lo(p.L.root_len), ch.n(p.L.root_len), !leafT,
                                         leafT, tx, ty, tz, s_nb[warp], p, org, h, hinv, XA, a, c, t4, it);
        } else {
            const int* lf = p.L.lists + par * p.L.far_len;
            const int ns = p.L.far_len - p.L.far_pairs;
            walk_forward_com<MODE, true>(lf + ch.lo(p.L.far_pairs), ch.n(p.L.far_pairs), !leafT, leafT, tx, ty, tz,
                                         s_nb[warp], p, org, h, hinv, XA, a, c, t4, it);
            walk_forward_com<MODE, false>(lf + p.L.far_pairs + ch.lo(ns), ch.n(ns), !leafT, leafT, tx, ty, tz,
                                          s_nb[warp], p, org, h, hinv, XA, a, c, t4, it);
        }
        if (leafT && !((MODE & 2) && level > 0))
            walk_forward_com<MODE, true, true>(p.L.lists + p.L.near_off + ch.lo(p.L.near_len), ch.n(p.L.near_len),
                                               false, true, tx, ty, tz, s_nb[warp], p, org, h, hinv, XA, a, c, t4, it);
        if (ch.k == 1 || chunk_combine_fwd(p, ci, item & 15, ch, lane, a, c, t4))
            store_forward<MODE>(p, node, level, leafT, tcell, a, c, t4);
        __syncwarp();
    }
}

// Adjoint gather with fixed centres: source cell B collects from the targets
// of its transposed stencil (target = source + sg * o, sg = +1, and -1 too
// when PAIRED).  MULTI: multipole source, derivatives per pair.  Otherwise a
// point-mass source: a leaf target is at an integer offset (the table row of
// R/h = sg * o), a non-leaf target uses its own centre.
template <bool MULTI, bool PAIRED>
__device__ __forceinline__ void walk_adjoint_com(const int* __restrict__ list, int len, bool near_seg, bool virt_t,
                                                 int sx0, int sy0, int sz0, const int2* __restrict__ s_nb,
                                                 const AdjParams& p,
                                                 const int (&org)[3], double h, double hinv, const double (&XB)[3],
                                                 double (&g)[16], double (&g4)[4], int item) {
    for (int k = 0; k < len; ++k) {
        const int po = __ldg(list + k);
        const int ox = (po & 0xff) - 8, oy = ((po >> 8) & 0xff) - 8, oz = ((po >> 16) & 0xff) - 8;
#pragma unroll
        for (int sd = 0; sd < (PAIRED ? 2 : 1); ++sd) {
            const int sg = sd ? -1 : 1;
            const int tx = sx0 + sg * ox, ty = sy0 + sg * oy, tz = sz0 + sg * oz;
            const int2 e = s_nb[nb_index(tx, ty, tz)];
            const int kind = e.y & 3;
            bool valid = (kind == K_MULTI || kind == K_LEAF) && (!near_seg || kind == K_LEAF);
            bool vchild = !MULTI && virtual_child_target(e, virt_t);
            if ((valid || vchild) && static_cast<unsigned>(e.x) >= static_cast<unsigned>(p.n_nodes)) {
                report(p.status, 4, item);
                valid = vchild = false;
            }
            if (!__any_sync(0xffffffffu, valid || vchild)) continue;
            const int tcell = (tx & 7) + 8 * (ty & 7) + 64 * (tz & 7);
            double lb[16];
            adjoint_target_lb(p, e, valid, vchild, tx, ty, tz, lb);
            double d[36];
            if (MULTI) {
                double XA[3] = {0.0, 0.0, 0.0};
                if (valid) {
                    if (kind == K_MULTI) {
                        const double* ca = p.C + static_cast<size_t>(e.x) * 3 * NCELL + tcell;
                        XA[0] = ca[0];
                        XA[1] = ca[NCELL];
                        XA[2] = ca[2 * NCELL];
                    } else {
                        XA[0] = geo_centre(org[0], tx, h);
                        XA[1] = geo_centre(org[1], ty, h);
                        XA[2] = geo_centre(org[2], tz, h);
                    }
                }
                double rx, ry, rz;
                scaled_sep(valid, XA, XB, hinv, rx, ry, rz);
                ot_deriv19_at(rx, ry, rz, d);
                ot_multi_adj(g, lb, d);
            } else {
                // the table row of R/h = sg * o is that of the offset -sg * o
                const int row = sd ? offset_row(ox, oy, oz) : NOFF - 1 - offset_row(ox, oy, oz);
                load_row16(d, p.Dt, row);
                const bool own = valid && kind == K_MULTI;
                if (__any_sync(0xffffffffu, own) && own) {
                    const double* ca = p.C + static_cast<size_t>(e.x) * 3 * NCELL + tcell;
                    const double XA[3] = {ca[0], ca[NCELL], ca[2 * NCELL]};
                    double rx, ry, rz;
                    scaled_sep(true, XA, XB, hinv, rx, ry, rz);
                    ot_deriv16_at(rx, ry, rz, d);
                }
                ot_mono_adj(g4, lb, d);
            }
        }
    }
}

// point-mass adjoint by a non-leaf target (centre from C): every point-mass
// source of its stencil receives <lb, dG(R/h)> by atomic add
template <bool PAIRED>
__device__ __forceinline__ void walk_scatter_com(const int* __restrict__ list, int len, int tx, int ty, int tz,
                                                 const int2* __restrict__ s_nb, const AdjParams& p,
                                                 const int (&org)[3], double h, double hinv, const double (&XA)[3],
                                                 const double (&lb)[16], int item) {
    for (int k = 0; k < len; ++k) {
        const int po = __ldg(list + k);
        const int ox = (po & 0xff) - 8, oy = ((po >> 8) & 0xff) - 8, oz = ((po >> 16) & 0xff) - 8;
#pragma unroll
        for (int sd = 0; sd < (PAIRED ? 2 : 1); ++sd) {
            const int sg = sd ? -1 : 1;
            const int sx = tx + sg * ox, sy = ty + sg * oy, sz = tz + sg * oz;
            const int2 e = s_nb[nb_index(sx, sy, sz)];
            int kind = e.y & 3;
            if (kind != K_NONE && static_cast<unsigned>(e.x) >= static_cast<unsigned>(p.n_nodes)) {
                report(p.status, 3, item);
                kind = K_NONE;
            }
            const bool mono = kind >= K_LEAF;
            if (!__any_sync(0xffffffffu, mono)) continue;
            const double X[3] = {geo_centre(org[0], sx, h), geo_centre(org[1], sy, h), geo_centre(org[2], sz, h)};
            double rx, ry, rz, d[36];
            scaled_sep(mono, XA, X, hinv, rx, ry, rz);
            ot_deriv16_at(rx, ry, rz, d);
            double ev, od;
            ot_mono_adj_split(ev, od, lb, d);
            scatter_mass(p, e, kind, sx, sy, sz, ev + od);
        }
    }
}

__device__ void scatter_item_com(const AdjParams& p, int2* s_nb, int node, int par, int half, int lane, int it) {
    int tx, ty, tz;
    lane_cell(lane, par, half, tx, ty, tz);
    const int tcell = tx + 8 * ty + 64 * tz;
    double lb[16];
    const double* src = p.Lrbar + static_cast<size_t>(node) * NRED * NCELL + tcell;
    bool nz = false;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        lb[q] = __ldg(src + q * NCELL);
        nz |= lb[q] != 0.0;
    }
    if (!__any_sync(0xffffffffu, nz)) return;
    if (lane < 27) s_nb[lane] = __ldg(p.nbr + static_cast<size_t>(node) * 27 + lane);
    __syncwarp();
    const int level = __ldg(p.ninfo + node) & 0xff;
    const double h = p.hreal[level], hinv = p.hinv[level];
    const int org[3] = {8 * __ldg(p.ncoord + 3 * node), 8 * __ldg(p.ncoord + 3 * node + 1),
                        8 * __ldg(p.ncoord + 3 * node + 2)};
    const double* ca = p.C + static_cast<size_t>(node) * 3 * NCELL + tcell;
    const double XA[3] = {ca[0], ca[NCELL], ca[2 * NCELL]};
    if (level == 0) {
        walk_scatter_com<true>(p.L.lists + p.L.root_off, p.L.root_len, tx, ty, tz, s_nb, p, org, h, hinv, XA, lb, it);
    } else {
        const int* lf = p.L.lists + par * p.L.far_len;
        walk_scatter_com<true>(lf, p.L.far_pairs, tx, ty, tz, s_nb, p, org, h, hinv, XA, lb, it);
        walk_scatter_com<false>(lf + p.L.far_pairs, p.L.far_len - p.L.far_pairs, tx, ty, tz, s_nb, p, org, h, hinv,
                                XA, lb, it);
    }
}

// MODE bits: 1 multipole sources (gather), 2 point-mass sources (gather),
// 4 point-mass adjoint by target (items with bit 30 set, atomic adds)
template <int MODE>
__global__ void __launch_bounds__(256) adjoint_com_kernel(const AdjParams p) {
    __shared__ int2 s_nb[8][27];
    __shared__ int s_sl[8][27];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    for (;;) {
        int v = 0;
        if (lane == 0) v = atomicAdd(p.counter, 1);
        const int it = __shfl_sync(0xffffffffu, v, 0);
        if (it >= p.n_items) break;
        const int item = __ldg(p.items + it);
        if ((MODE & 4) && ((item >> 30) & 1)) {
            const int tgt = item & 0x3fffffff;
            const int node = tgt >> 4;
            // a leaf target has a geometric centre: the table path's scatter
            if ((__ldg(p.ninfo + node) >> 8) & 1)
                scatter_item(p, p.nbr, p.ninfo, s_nb[warp], s_sl[warp], node, (tgt >> 1) & 7, tgt & 1, lane, it);
            else
                scatter_item_com(p, s_nb[warp], node, (tgt >> 1) & 7, tgt & 1, lane, it);
            __syncwarp();
            continue;
        }
        Chunk ch{0, 1};
        int2 ci = make_int2(-1, 0);
        int src = item >> 4;
        if (item < 0) {            // a chunk of a multipole gather item (as on the table path)
            src = (item >> 4) & 0x3fffff;
            ch.c = (item >> 26) & 15;
            if (p.cinfo != nullptr && src < p.n_nodes) {
                ci = __ldg(p.cinfo + src);
                if (ci.x >= 0) ch.k = (ci.y & 15) + 1;
            }
            if (ch.c >= ch.k) {
                report(p.status, 6, it);
                continue;
            }
        }
        const int par = (item >> 1) & 7, half = item & 1;
        const bool virt = src >= p.n_nodes;
        const int2* nbt = virt ? p.vnbr + static_cast<size_t>(src - p.n_nodes) * 27
                               : p.nbr + static_cast<size_t>(src) * 27;
        if (lane < 27) s_nb[warp][lane] = __ldg(nbt + lane);
        __syncwarp();
        int level, skind;
        const int* crd;
        if (virt) {
            level = __ldg(p.vinfo + (src - p.n_nodes));
            skind = K_VIRT;
            crd = p.vcoord + 3 * (src - p.n_nodes);
        } else {
            const int info = __ldg(p.ninfo + src);
            level = info & 0xff;
            skind = ((info >> 8) & 1) ? K_LEAF : K_MULTI;
            crd = p.ncoord + 3 * src;
        }
        const double h = p.hreal[level], hinv = p.hinv[level];
        const int org[3] = {8 * __ldg(crd), 8 * __ldg(crd + 1), 8 * __ldg(crd + 2)};
        int sx, sy, sz;
        lane_cell(lane, par, half, sx, sy, sz);
        const int scell = sx + 8 * sy + 64 * sz;
        double XB[3];
        if (skind == K_MULTI) {
            const double* cb = p.C + static_cast<size_t>(src) * 3 * NCELL + scell;
            XB[0] = cb[0];
            XB[1] = cb[NCELL];
            XB[2] = cb[2 * NCELL];
        } else {
            XB[0] = geo_centre(org[0], sx, h);
            XB[1] = geo_centre(org[1], sy, h);
            XB[2] = geo_centre(org[2], sz, h);
        }
        const int* l1 = (level == 0) ? p.L.lists + p.L.root_off : p.L.lists + par * p.L.far_len;
        const int* l2 = p.L.lists + p.L.near_off;
        const int np = (level == 0) ? p.L.root_len : p.L.far_pairs;
        const int ns = (level == 0) ? 0 : p.L.far_len - p.L.far_pairs;
        double g[16], g4[4];
#pragma unroll
        for (int q = 0; q < 16; ++q) g[q] = 0.0;
#pragma unroll
        for (int q = 0; q < 4; ++q) g4[q] = 0.0;
        if (skind == K_MULTI) {
            // targets of the transposed far (root) stencil; near leaf targets
            // of a refined cell see its children instead
            if ((MODE & 1) && p.Mbar != nullptr) {
                walk_adjoint_com<true, true>(l1 + ch.lo(np), ch.n(np), false, false, sx, sy, sz, s_nb[warp], p, org,
                                             h, hinv, XB, g, g4, it);
                walk_adjoint_com<true, false>(l1 + np + ch.lo(ns), ch.n(ns), false, false, sx, sy, sz, s_nb[warp], p,
                                              org, h, hinv, XB, g, g4, it);
                if (ch.k == 1 || chunk_combine(p.part, p.chunk_ctr, ci, item & 15, ch, lane, g))
                    store_mbar(p.Mbar, src, scell, hinv, g);
            }
        } else if ((MODE & 2) && p.mbar != nullptr) {
            const bool vt = skind == K_LEAF;
            walk_adjoint_com<false, true>(l1, np, false, vt, sx, sy, sz, s_nb[warp], p, org, h, hinv, XB, g, g4, it);
            walk_adjoint_com<false, false>(l1 + np, ns, false, vt, sx, sy, sz, s_nb[warp], p, org, h, hinv, XB, g, g4,
                                           it);
            walk_adjoint_com<false, true>(l2, p.L.near_len, true, vt, sx, sy, sz, s_nb[warp], p, org, h, hinv, XB, g,
                                          g4, it);
            const double val = (g4[0] + g4[1]) + (g4[2] + g4[3]);
            if (virt) p.vbar[static_cast<size_t>(src - p.n_nodes) * NCELL + scell] = val;
            else p.mbar[static_cast<size_t>(src) * NCELL + scell] = val;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// FP64 FMA throughput probe
// ---------------------------------------------------------------------------

// variant 0: 16 chains a = a * b + c; variant 1: 16 accumulators a += s * x[j]
// (shared scalar, distinct multiplier per chain).  Streams of FP64 operations
// on register operands alone keep the FP64 pipe about 84 % busy.
template <int VARIANT>
__global__ void __launch_bounds__(256) fp64_probe_kernel(double* out, int iters) {
    constexpr int K = 16;
    double a[K], x[K];
    const double b = 0.999999, c = 1e-6 * (1.0 + threadIdx.x * 1e-9), sc = 1e-9 * (1.0 + threadIdx.x * 1e-9);
#pragma unroll
    for (int j = 0; j < K; ++j) {
        a[j] = 0.5 + 0.01 * j;
        x[j] = 1.0 + 0.03 * j;
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < K; ++j) a[j] = (VARIANT == 0) ? fma(a[j], b, c) : fma(sc, x[j], a[j]);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < K; ++j) s += a[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// variant 2, the point-mass contraction's pattern: 64 rows of 16 derivative
// values staged in shared memory (128-bit loads), each row's 16 values times
// one of 4 per-thread source values accumulated into 16 sums -- 1024 DFMAs
// per iteration with operands arriving from shared memory, which keeps the
// FP64 pipe busy at its full issue rate.
__global__ void __launch_bounds__(256) fp64_probe_contraction_kernel(double* out, int iters) {
    __shared__ double2 rows[64][8];
    for (int t = threadIdx.x; t < 64 * 8; t += blockDim.x) {
        const int r = t >> 3, c = t & 7;
        const double v = 1e-3 * (1.0 + 0.01 * r + 0.001 * c);
        rows[r][c] = make_double2(v, 0.5 * v);
    }
    __syncthreads();
    double acc[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[c] = 0.0;
    double src[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const double lo = 1.0 + 1e-3 * (threadIdx.x + q), hi = 1.0 + 1e-3 * (threadIdx.x + q + 4);
        src[q] = (q & 1) ? hi - lo : lo + hi;
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll 1
        for (int o = 0; o < 64; o += 4) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const double2 d = rows[o + q][c];
                    acc[2 * c] = fma(src[q], d.x, acc[2 * c]);
                    acc[2 * c + 1] = fma(src[q], d.y, acc[2 * c + 1]);
                }
            }
        }
    }
    double z = 0.0;
#pragma unroll
    for (int c = 0; c < 16; ++c) z += acc[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = z;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

namespace {
std::atomic<long long> g_launches{0};
thread_local long long t_launches = 0;

inline cudaError_t counted(cudaError_t e) {
    if (e == cudaSuccess) {
        g_launches.fetch_add(1, std::memory_order_relaxed);
        ++t_launches;
    }
    return e;
}
}  // namespace

long long launch_count_total() { return g_launches.load(std::memory_order_relaxed); }
long long launch_count_thread() { return t_launches; }
void launch_count_adjust(long long delta) {
    g_launches.fetch_add(delta, std::memory_order_relaxed);
    t_launches += delta;
}

cudaError_t launch_forward(const FwdParams& p, int mode, bool persistent, int wpb, int grid, cudaStream_t s,
                           bool one_block_per_sm) {
    if (p.n_items == 0) return cudaSuccess;
    const dim3 block(32 * wpb);
    const int per = persistent ? 1 : 0;
    // double-float point masses when split masses are given, multipole
    // contractions too when split moments are given
    const int emu = (p.mf != nullptr && (mode & 2) ? 1 : 0) | (p.Mf != nullptr && (mode & 1) ? 2 : 0);
    switch (mode * 4 + emu) {
        case 4:
            // at 128 registers the multipole pass spills; with one block per
            // SM it keeps its working set in registers
            if (one_block_per_sm)
                forward_kernel<1, 0, 1><<<grid, block, 0, s>>>(p, per);
            else
                forward_kernel<1, 0><<<grid, block, 0, s>>>(p, per);
            break;
        case 6: forward_kernel<1, 2><<<grid, block, 0, s>>>(p, per); break;
        case 8: forward_kernel<2, 0><<<grid, block, 0, s>>>(p, per); break;
        case 9: forward_kernel<2, 1><<<grid, block, 0, s>>>(p, per); break;
        case 12: forward_kernel<3, 0><<<grid, block, 0, s>>>(p, per); break;
        case 13: forward_kernel<3, 1><<<grid, block, 0, s>>>(p, per); break;
        case 15: forward_kernel<3, 3><<<grid, block, 0, s>>>(p, per); break;
        default: return cudaErrorInvalidValue;
    }
    return counted(cudaGetLastError());
}

// reduced moments of the listed nodes as double-float pairs (hi, lo)
__global__ void split_moments_kernel(const double* __restrict__ Mhat, float2* __restrict__ Mf,
                                     const int* __restrict__ nodes, int n_list) {
    const size_t t = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= static_cast<size_t>(n_list) * NRED * NCELL) return;
    const size_t off = static_cast<size_t>(nodes[t / (NRED * NCELL)]) * NRED * NCELL + t % (NRED * NCELL);
    const double v = Mhat[off];
    const float hi = __double2float_rn(v);
    Mf[off] = make_float2(hi, __double2float_rn(v - static_cast<double>(hi)));
}

cudaError_t launch_split_moments(const double* Mhat, float2* Mf, const int* nodes, int n_list, cudaStream_t s) {
    if (n_list == 0) return cudaSuccess;
    const long long n = 1LL * n_list * NRED * NCELL;
    split_moments_kernel<<<static_cast<int>((n + 255) / 256), 256, 0, s>>>(Mhat, Mf, nodes, n_list);
    return counted(cudaGetLastError());
}

__global__ void split_masses_kernel(const double* __restrict__ m, float2* __restrict__ mf, size_t n) {
    const size_t t = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const double v = m[t];
    const float hi = __double2float_rn(v);
    mf[t] = make_float2(hi, __double2float_rn(v - static_cast<double>(hi)));
}

cudaError_t launch_split_masses(const double* m, float2* mf, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    split_masses_kernel<<<static_cast<int>((n + 255) / 256), 256, 0, s>>>(m, mf, n);
    return counted(cudaGetLastError());
}

cudaError_t launch_adjoint(const AdjParams& p, int mode, bool persistent, int wpb, int grid, cudaStream_t s) {
    if (p.n_items == 0) return cudaSuccess;
    const dim3 block(32 * wpb);
    const int per = persistent ? 1 : 0;
    if (p.Dt32 != nullptr) {           // double-float (split L-bar and tables given)
        switch (mode) {
            case 1: adjoint_kernel<1, true><<<grid, block, 0, s>>>(p, per); break;
            case 4: adjoint_kernel<4, true><<<grid, block, 0, s>>>(p, per); break;
            default: return cudaErrorInvalidValue;
        }
        return counted(cudaGetLastError());
    }
    switch (mode) {
        case 1: adjoint_kernel<1><<<grid, block, 0, s>>>(p, per); break;
        case 2: adjoint_kernel<2><<<grid, block, 0, s>>>(p, per); break;
        case 4: adjoint_kernel<4><<<grid, block, 0, s>>>(p, per); break;
        default: adjoint_kernel<3><<<grid, block, 0, s>>>(p, per); break;
    }
    return counted(cudaGetLastError());
}

cudaError_t launch_scatter_adjoint(const ScatParams& p, bool persistent, int wpb, int grid, cudaStream_t s) {
    if (p.n_items == 0) return cudaSuccess;
    scatter_adjoint_kernel<<<grid, 32 * wpb, 0, s>>>(p, persistent ? 1 : 0);
    return counted(cudaGetLastError());
}

int scatter_max_blocks_per_sm(int wpb) {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, (const void*)scatter_adjoint_kernel, 32 * wpb, 0);
    return n;
}

// mode 1-3 FP64; 6, 7 double-float point masses (modes 2, 3); 5, 8 double-float
// multipole contractions too (modes 1, 3)
int forward_max_blocks_per_sm(int mode, int wpb) {
    int n = 0;
    const void* f = (mode == 1)   ? (const void*)forward_kernel<1, 0>
                    : (mode == 2) ? (const void*)forward_kernel<2, 0>
                    : (mode == 3) ? (const void*)forward_kernel<3, 0>
                    : (mode == 5) ? (const void*)forward_kernel<1, 2>
                    : (mode == 6) ? (const void*)forward_kernel<2, 1>
                    : (mode == 7) ? (const void*)forward_kernel<3, 1>
                                  : (const void*)forward_kernel<3, 3>;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, 32 * wpb, 0);
    return n;
}

// mode 1-4 FP64; 9, 12: the double-float variants of modes 1, 4
int adjoint_max_blocks_per_sm(int mode, int wpb) {
    int n = 0;
    const void* f = (mode == 1)    ? (const void*)adjoint_kernel<1>
                    : (mode == 2)  ? (const void*)adjoint_kernel<2>
                    : (mode == 4)  ? (const void*)adjoint_kernel<4>
                    : (mode == 9)  ? (const void*)adjoint_kernel<1, true>
                    : (mode == 12) ? (const void*)adjoint_kernel<4, true>
                                   : (const void*)adjoint_kernel<3>;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, 32 * wpb, 0);
    return n;
}

static inline int blocks_for(long long n, int per) { return static_cast<int>((n + per - 1) / per); }

// x butterflies for the first transform stage of x-complete classes: for
// every cell c of the listed nodes (slot = list index) and a = 1..7,
// v(c + a x) + v(c - a x) and v(c + a x) - v(c - a x), v the value the pass
// reads at that position (reduced moments of multipole cells; point masses
// of leaf and virtual cells), 0 elsewhere
__global__ void xbutterfly_moments_kernel(const int2* __restrict__ snb, int n_slots, const double* __restrict__ Mhat,
                                          int n_nodes, double* __restrict__ Sx) {
    const long long gid = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (gid >= 7LL * NCELL * n_slots) return;
    const int cell = static_cast<int>(gid % NCELL);
    const int a = static_cast<int>((gid / NCELL) % 7) + 1;
    const int slot = static_cast<int>(gid / (7 * NCELL));
    const int x = cell & 7, y = (cell >> 3) & 7, z = cell >> 6;
    const int2* nb = snb + static_cast<size_t>(slot) * 27;
    const double* src[2] = {nullptr, nullptr};
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
        const int sx = sd ? x - a : x + a;
        const int2 e = __ldg(nb + nb_index(sx, y, z));
        if ((e.y & 3) == K_MULTI && static_cast<unsigned>(e.x) < static_cast<unsigned>(n_nodes))
            src[sd] = Mhat + static_cast<size_t>(e.x) * NRED * NCELL + (sx & 7) + 8 * y + 64 * z;
    }
    double* out = Sx + static_cast<size_t>(slot * 7 + a - 1) * 32 * NCELL + cell;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const double vp = src[0] ? __ldg(src[0] + k * NCELL) : 0.0;
        const double vm = src[1] ? __ldg(src[1] + k * NCELL) : 0.0;
        out[(2 * k) * NCELL] = vp + vm;
        out[(2 * k + 1) * NCELL] = vp - vm;
    }
}

// the same over the targets' reduced L-bar: multipole and leaf cells of the
// node's level (the multipole gather's targets)
__global__ void xbutterfly_lbar_kernel(const int2* __restrict__ snb, int n_slots, const double* __restrict__ Lrbar,
                                       int n_nodes, double* __restrict__ Tx) {
    const long long gid = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (gid >= 7LL * NCELL * n_slots) return;
    const int cell = static_cast<int>(gid % NCELL);
    const int a = static_cast<int>((gid / NCELL) % 7) + 1;
    const int slot = static_cast<int>(gid / (7 * NCELL));
    const int x = cell & 7, y = (cell >> 3) & 7, z = cell >> 6;
    const int2* nb = snb + static_cast<size_t>(slot) * 27;
    const double* src[2] = {nullptr, nullptr};
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
        const int sx = sd ? x - a : x + a;
        const int2 e = __ldg(nb + nb_index(sx, y, z));
        const int k = e.y & 3;
        if ((k == K_MULTI || k == K_LEAF) && static_cast<unsigned>(e.x) < static_cast<unsigned>(n_nodes))
            src[sd] = Lrbar + static_cast<size_t>(e.x) * NRED * NCELL + (sx & 7) + 8 * y + 64 * z;
    }
    double* out = Tx + static_cast<size_t>(slot * 7 + a - 1) * 32 * NCELL + cell;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const double vp = src[0] ? __ldg(src[0] + k * NCELL) : 0.0;
        const double vm = src[1] ? __ldg(src[1] + k * NCELL) : 0.0;
        out[(2 * k) * NCELL] = vp + vm;
        out[(2 * k + 1) * NCELL] = vp - vm;
    }
}

__device__ __forceinline__ double mass_at(const double* __restrict__ m, int2 e, int n_nodes, int sx, int sy, int sz) {
    const int kind = e.y & 3;
    if (static_cast<unsigned>(e.x) >= static_cast<unsigned>(n_nodes)) return 0.0;
    if (kind == K_LEAF) return __ldg(m + static_cast<size_t>(e.x) * NCELL + (sx & 7) + 8 * (sy & 7) + 64 * (sz & 7));
    if (kind == K_VIRT) {
        const unsigned meta = static_cast<unsigned>(e.y);
        const int d = (meta >> 2) & 7;
        const int vx = static_cast<int>(((meta >> 8) & 0xffu) + (sx & 7)) >> d;
        const int vy = static_cast<int>(((meta >> 16) & 0xffu) + (sy & 7)) >> d;
        const int vz = static_cast<int>((meta >> 24) + (sz & 7)) >> d;
        return __ldg(m + static_cast<size_t>(e.x) * NCELL + vx + 8 * vy + 64 * vz) * pow2i(-3 * d);
    }
    return 0.0;
}

// the transpose of xbutterfly_masses_kernel: each cell c of a point-mass
// region (a leaf node or a virtual block) collects, for a = 1..7, the
// deferred x channels (A, B) of the positions c - a x (c is their +a member:
// A + B) and c + a x (their -a member: A - B), and adds the sum to its mass
// adjoint (a virtual cell's, times 8^-d, to the cell of its coarse leaf)
__global__ void xbutterfly_masses_adjoint_kernel(const int2* __restrict__ ent, const int* __restrict__ xs,
                                                 int n_members, const double* __restrict__ Sbar, int n_nodes,
                                                 double* __restrict__ mbar) {
    const long long gid = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (gid >= 1LL * NCELL * n_members) return;
    const int cell = static_cast<int>(gid % NCELL);
    const int k = static_cast<int>(gid / NCELL);
    const int x = cell & 7, y = (cell >> 3) & 7, z = cell >> 6;
    int cs[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) cs[r] = __ldg(xs + 3 * k + r);
    double acc = 0.0;
    for (int a = 1; a <= 7; ++a) {
#pragma unroll
        for (int sd = 0; sd < 2; ++sd) {
            const int qx = sd ? x + a : x - a;         // the position whose member c is
            const int slot = cs[(qx >> 3) + 1];
            if (slot < 0) continue;
            const double* src = Sbar + static_cast<size_t>(slot * 7 + a - 1) * 2 * NCELL + (qx & 7) + 8 * y + 64 * z;
            const double A = __ldg(src), B = __ldg(src + NCELL);
            acc += sd ? A - B : A + B;
        }
    }
    if (acc == 0.0) return;
    const int2 e = __ldg(ent + k);
    if (static_cast<unsigned>(e.x) >= static_cast<unsigned>(n_nodes)) return;
    if ((e.y & 3) == K_LEAF) {
        atomicAdd(mbar + static_cast<size_t>(e.x) * NCELL + cell, acc);
    } else if ((e.y & 3) == K_VIRT) {
        const unsigned meta = static_cast<unsigned>(e.y);
        const int d = (meta >> 2) & 7;
        const int vx = static_cast<int>(((meta >> 8) & 0xffu) + x) >> d;
        const int vy = static_cast<int>(((meta >> 16) & 0xffu) + y) >> d;
        const int vz = static_cast<int>((meta >> 24) + z) >> d;
        atomicAdd(mbar + static_cast<size_t>(e.x) * NCELL + vx + 8 * vy + 64 * vz, acc * pow2i(-3 * d));
    }
}

__global__ void xbutterfly_masses_kernel(const int2* __restrict__ snb, int n_slots, const double* __restrict__ m,
                                         int n_nodes, double* __restrict__ Sm) {
    const long long gid = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (gid >= 7LL * NCELL * n_slots) return;
    const int cell = static_cast<int>(gid % NCELL);
    const int a = static_cast<int>((gid / NCELL) % 7) + 1;
    const int slot = static_cast<int>(gid / (7 * NCELL));
    const int x = cell & 7, y = (cell >> 3) & 7, z = cell >> 6;
    const int2* nb = snb + static_cast<size_t>(slot) * 27;
    const double vp = mass_at(m, __ldg(nb + nb_index(x + a, y, z)), n_nodes, x + a, y, z);
    const double vm = mass_at(m, __ldg(nb + nb_index(x - a, y, z)), n_nodes, x - a, y, z);
    double* out = Sm + static_cast<size_t>(slot * 7 + a - 1) * 2 * NCELL + cell;
    out[0] = vp + vm;
    out[NCELL] = vp - vm;
}

cudaError_t launch_prescale_moments(const PrepParams& p, cudaStream_t s) {
    if (p.n_list == 0) return cudaSuccess;
    prescale_moments_kernel<<<blocks_for(1LL * p.n_list * NCELL, 256), 256, 0, s>>>(p);
    return counted(cudaGetLastError());
}

cudaError_t launch_xbutterfly_moments(const int2* snb, int n_slots, const double* Mhat, int n_nodes, double* Sx,
                                      cudaStream_t s) {
    if (n_slots == 0) return cudaSuccess;
    xbutterfly_moments_kernel<<<blocks_for(7LL * NCELL * n_slots, 256), 256, 0, s>>>(snb, n_slots, Mhat, n_nodes, Sx);
    return counted(cudaGetLastError());
}

// (x, y) butterflies of the masses: for every cell c of a slot's region and
// a, b = 1..7, the four transforms over x and y of the masses at
// c + (+-a, +-b, 0), out[pi] = sum_i (-1)^|i & pi| v_i (i, pi: bit 0 x
// negated / x odd, bit 1 y).  A block of 256 threads covers four z layers
// of one slot's region: it stages the masses of those layers in the 3 x 3
// regions around it in shared memory once; per a it then forms the x stage
// (the sum and the difference of the masses a cells to either side in x)
// at the rows y - 7 .. y + 14 once, shared by the seven b of every cell, and
// each thread runs the y stage of its cell, every store of a warp covering
// 32 consecutive cells.  The operations per output are those of the
// transform written out, so the table is the same to the bit.
__global__ void xybutterfly_masses_kernel(const int2* __restrict__ snb, int n_slots, const double* __restrict__ m,
                                          int n_nodes, double* __restrict__ Sxy) {
    constexpr int ROWS = 22;                  // y' = -7 .. 14
    __shared__ double sm[9][256];
    __shared__ double sx[2][4][ROWS][8];      // [sum, difference][z layer][y' + 7][x]
    const long long first = static_cast<long long>(blockIdx.x) * blockDim.x;
    const int slot = static_cast<int>(first / NCELL);
    if (slot >= n_slots) return;              // whole blocks: a slot is two blocks of 256 cells
    const int z0 = static_cast<int>(first % NCELL) >> 6;          // 0 or 4
    const int2* nb = snb + static_cast<size_t>(slot) * 27 + 9;    // the z = 0 layer of the regions
    for (int t = threadIdx.x; t < 9 * 256; t += blockDim.x) {
        const int r = t >> 8, c = t & 255;
        sm[r][c] = mass_at(m, __ldg(nb + r), n_nodes, c & 7, (c >> 3) & 7, z0 + (c >> 6));
    }
    __syncthreads();
    const int cell = static_cast<int>((first + threadIdx.x) % NCELL);
    const int x = cell & 7, y = (cell >> 3) & 7, zl = (cell >> 6) - z0;
    double* out = Sxy + static_cast<size_t>(slot) * 49 * 4 * NCELL + cell;
#pragma unroll 1
    for (int a = 1; a <= 7; ++a) {
        for (int t = threadIdx.x; t < 4 * ROWS * 8; t += blockDim.x) {
            const int px = t & 7, row = (t >> 3) % ROWS, pz = t / (ROWS * 8);
            const int py = row - 7, xp = px + a, xm = px - a;
            const double vp = sm[((xp + 8) >> 3) + 3 * ((py + 8) >> 3)][(xp & 7) + 8 * (py & 7) + 64 * pz];
            const double vm = sm[((xm + 8) >> 3) + 3 * ((py + 8) >> 3)][(xm & 7) + 8 * (py & 7) + 64 * pz];
            sx[0][pz][row][px] = vp + vm;
            sx[1][pz][row][px] = vp - vm;
        }
        __syncthreads();
#pragma unroll
        for (int b = 1; b <= 7; ++b) {
            const double u0 = sx[0][zl][y + b + 7][x], u1 = sx[1][zl][y + b + 7][x];
            const double u2 = sx[0][zl][y - b + 7][x], u3 = sx[1][zl][y - b + 7][x];
            double* o = out + static_cast<size_t>((a - 1) * 7 + b - 1) * 4 * NCELL;
            o[0] = u0 + u2;
            o[NCELL] = u1 + u3;
            o[2 * NCELL] = u0 - u2;
            o[3 * NCELL] = u1 - u3;
        }
        __syncthreads();
    }
}

cudaError_t launch_xybutterfly_masses(const int2* snb, int n_slots, const double* m, int n_nodes, double* Sxy,
                                      cudaStream_t s) {
    if (n_slots == 0) return cudaSuccess;
    xybutterfly_masses_kernel<<<blocks_for(1LL * NCELL * n_slots, 256), 256, 0, s>>>(snb, n_slots, m, n_nodes, Sxy);
    return counted(cudaGetLastError());
}

// (x, y) butterflies of the reduced moments, component by component: for
// every cell c of a slot's region, a, b = 1..7 and component k, the four
// transforms over x and y of Mhat_k at c + (+-a, +-b, 0) (multipole cells;
// 0 elsewhere), in the masses' table's channel order, a cell's four channels
// adjacent.  Built from the x table (the y stage only: its sums and
// differences at c + (0, +-b, 0) read from the slots of the regions at y-1,
// y, y+1, so the same bits as a transform from the moments); a thread owns
// one cell, and a block's cells share the x-table rows they read through L1.
__global__ void xybutterfly_moments_kernel(const int* __restrict__ ys, int n_slots, const double* __restrict__ Sx,
                                           double* __restrict__ Sxym) {
    const long long gid = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (gid >= 1LL * NCELL * n_slots) return;
    const int slot = static_cast<int>(gid / NCELL);
    const int cell = static_cast<int>(gid % NCELL);
    const int x = cell & 7, y = (cell >> 3) & 7, z = cell >> 6;
    const int s_lo = __ldg(ys + 3 * slot), s_mid = __ldg(ys + 3 * slot + 1), s_hi = __ldg(ys + 3 * slot + 2);
    // layout [slot][(a - 1) 7 + b - 1][k][cell][channel]
    double* out = Sxym + (static_cast<size_t>(slot) * 49 * 16 * NCELL + cell) * 4;
#pragma unroll 1
    for (int a = 1; a <= 7; ++a) {
#pragma unroll 1
        for (int k = 0; k < 16; ++k) {
#pragma unroll
            for (int b = 1; b <= 7; ++b) {
                const int yp = y + b, ym = y - b;
                const int sp = yp >= 8 ? s_hi : s_mid, sm = ym < 0 ? s_lo : s_mid;
                double u0 = 0.0, u1 = 0.0, u2 = 0.0, u3 = 0.0;
                if (sp >= 0) {
                    const double* q = Sx + (static_cast<size_t>(sp * 7 + a - 1) * 32 + 2 * k) * NCELL + x +
                                      8 * (yp & 7) + 64 * z;
                    u0 = __ldg(q);
                    u1 = __ldg(q + NCELL);
                }
                if (sm >= 0) {
                    const double* q = Sx + (static_cast<size_t>(sm * 7 + a - 1) * 32 + 2 * k) * NCELL + x +
                                      8 * (ym & 7) + 64 * z;
                    u2 = __ldg(q);
                    u3 = __ldg(q + NCELL);
                }
                double2* o = reinterpret_cast<double2*>(
                    out + (static_cast<size_t>((a - 1) * 7 + b - 1) * 16 + k) * NCELL * 4);
                o[0] = make_double2(u0 + u2, u1 + u3);
                o[1] = make_double2(u0 - u2, u1 - u3);
            }
        }
    }
}

cudaError_t launch_xybutterfly_moments(const int* ys, int n_slots, const double* Sx, double* Sxym, cudaStream_t s) {
    if (n_slots == 0) return cudaSuccess;
    xybutterfly_moments_kernel<<<blocks_for(1LL * NCELL * n_slots, 256), 256, 0, s>>>(ys, n_slots, Sx, Sxym);
    return counted(cudaGetLastError());
}

cudaError_t launch_xbutterfly_masses_adjoint(const int2* ent, const int* xs, int n_members, const double* Sbar,
                                             int n_nodes, double* mbar, cudaStream_t s) {
    if (n_members == 0) return cudaSuccess;
    xbutterfly_masses_adjoint_kernel<<<blocks_for(1LL * NCELL * n_members, 256), 256, 0, s>>>(ent, xs, n_members, Sbar,
                                                                                                n_nodes, mbar);
    return counted(cudaGetLastError());
}

cudaError_t launch_xbutterfly_lbar(const int2* snb, int n_slots, const double* Lrbar, int n_nodes, double* Tx,
                                   cudaStream_t s) {
    if (n_slots == 0) return cudaSuccess;
    xbutterfly_lbar_kernel<<<blocks_for(7LL * NCELL * n_slots, 256), 256, 0, s>>>(snb, n_slots, Lrbar, n_nodes, Tx);
    return counted(cudaGetLastError());
}

cudaError_t launch_xbutterfly_masses(const int2* snb, int n_slots, const double* m, int n_nodes, double* Sm,
                                     cudaStream_t s) {
    if (n_slots == 0) return cudaSuccess;
    xbutterfly_masses_kernel<<<blocks_for(7LL * NCELL * n_slots, 256), 256, 0, s>>>(snb, n_slots, m, n_nodes, Sm);
    return counted(cudaGetLastError());
}

cudaError_t launch_prescale_adjoint(const PrepParams& p, cudaStream_t s) {
    if (p.n_list == 0) return cudaSuccess;
    prescale_adjoint_kernel<<<blocks_for(1LL * p.n_list * NCELL, 256), 256, 0, s>>>(p);
    return counted(cudaGetLastError());
}

cudaError_t launch_restrict_virtual(const double* vbar, const int* vmap, int n_rows, double* mbar, cudaStream_t s) {
    if (n_rows == 0) return cudaSuccess;
    restrict_virtual_kernel<<<blocks_for(n_rows, 256), 256, 0, s>>>(vbar, vmap, n_rows, mbar);
    return counted(cudaGetLastError());
}

cudaError_t launch_cube_moments(const double* rho, double* M, double* m, const int* nodes, int n_list,
                                const int* ninfo, const double* hinv, cudaStream_t s) {
    if (n_list == 0) return cudaSuccess;
    cube_moments_kernel<<<blocks_for(1LL * n_list * NCELL, 256), 256, 0, s>>>(rho, M, m, nodes, n_list, ninfo, hinv);
    return counted(cudaGetLastError());
}

cudaError_t launch_m2m(double* M, double* m, const int* parents, int n_list, const int* children,
                       const int* ninfo, const double* hinv, cudaStream_t s) {
    if (n_list == 0) return cudaSuccess;
    m2m_kernel<<<blocks_for(1LL * n_list * NCELL, 128), 128, 0, s>>>(M, m, parents, n_list, children, ninfo, hinv);
    return counted(cudaGetLastError());
}

cudaError_t launch_moments_adjoint_init(const double* Mbar, const double* mbar, double* Mb, int n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    moments_adjoint_init_kernel<<<blocks_for(1LL * n * NCOMP * NCELL, 256), 256, 0, s>>>(Mbar, mbar, Mb, n);
    return counted(cudaGetLastError());
}

cudaError_t launch_m2m_adjoint(double* Mb, const int* parents, int n_list, const int* children, const int* ninfo,
                               const double* hinv, cudaStream_t s) {
    if (n_list == 0) return cudaSuccess;
    m2m_adjoint_kernel<<<blocks_for(1LL * n_list * 8 * NCELL, 128), 128, 0, s>>>(Mb, parents, n_list, children,
                                                                                  ninfo, hinv);
    return counted(cudaGetLastError());
}

cudaError_t launch_cube_adjoint(const double* Mb, double* rhobar, const int* nodes, int n_list, const int* ninfo,
                                const double* hinv, cudaStream_t s) {
    if (n_list == 0) return cudaSuccess;
    cube_adjoint_kernel<<<blocks_for(1LL * n_list * NCELL, 256), 256, 0, s>>>(Mb, rhobar, nodes, n_list, ninfo, hinv);
    return counted(cudaGetLastError());
}

cudaError_t launch_geometric_centres(double* C, const int* nodes, int n_list, const int* ninfo, const int* ncoord,
                                     double h0, cudaStream_t s) {
    if (n_list == 0) return cudaSuccess;
    geometric_centres_kernel<<<blocks_for(1LL * n_list * NCELL, 256), 256, 0, s>>>(C, nodes, n_list, ninfo, ncoord,
                                                                                    h0);
    return counted(cudaGetLastError());
}

cudaError_t launch_m2m_com(double* M, double* m, double* C, const int* parents, int n_list, const int* children,
                           const int* ninfo, const int* ncoord, double h0, cudaStream_t s) {
    if (n_list == 0) return cudaSuccess;
    m2m_com_kernel<<<blocks_for(1LL * n_list * NCELL, 128), 128, 0, s>>>(M, m, C, parents, n_list, children, ninfo,
                                                                          ncoord, h0);
    return counted(cudaGetLastError());
}

cudaError_t launch_l2l_com(double* L, const double* C, const int* parents, int n_list, const int* children,
                           const int* ninfo, const int* ncoord, double h0, cudaStream_t s) {
    if (n_list == 0) return cudaSuccess;
    l2l_com_kernel<<<blocks_for(1LL * n_list * 8 * NCELL, 128), 128, 0, s>>>(L, C, parents, n_list, children, ninfo,
                                                                              ncoord, h0);
    return counted(cudaGetLastError());
}

cudaError_t launch_l2l_com_adjoint(double* Lb, const double* C, const int* parents, int n_list, const int* children,
                                   const int* ninfo, const int* ncoord, double h0, cudaStream_t s) {
    if (n_list == 0) return cudaSuccess;
    l2l_com_adjoint_kernel<<<blocks_for(1LL * n_list * NCELL, 128), 128, 0, s>>>(Lb, C, parents, n_list, children,
                                                                                  ninfo, ncoord, h0);
    return counted(cudaGetLastError());
}

cudaError_t launch_forward_com(const FwdParams& p, int mode, int wpb, int grid, cudaStream_t s) {
    if (p.n_items == 0) return cudaSuccess;
    switch (mode) {
        case 1: forward_com_kernel<1><<<grid, 32 * wpb, 0, s>>>(p); break;
        case 2: forward_com_kernel<2><<<grid, 32 * wpb, 0, s>>>(p); break;
        default: forward_com_kernel<3><<<grid, 32 * wpb, 0, s>>>(p); break;
    }
    return counted(cudaGetLastError());
}

cudaError_t launch_adjoint_com(const AdjParams& p, int mode, int wpb, int grid, cudaStream_t s) {
    if (p.n_items == 0) return cudaSuccess;
    switch (mode) {
        case 1: adjoint_com_kernel<1><<<grid, 32 * wpb, 0, s>>>(p); break;
        case 2: adjoint_com_kernel<2><<<grid, 32 * wpb, 0, s>>>(p); break;
        case 3: adjoint_com_kernel<3><<<grid, 32 * wpb, 0, s>>>(p); break;
        case 4: adjoint_com_kernel<4><<<grid, 32 * wpb, 0, s>>>(p); break;
        default: adjoint_com_kernel<5><<<grid, 32 * wpb, 0, s>>>(p); break;
    }
    return counted(cudaGetLastError());
}

int deriv_flops(int ncomp) {
    return ncomp == 31 ? OT_DERIV31_FLOPS : ncomp == 19 ? OT_DERIV19_FLOPS : OT_DERIV16_FLOPS;
}

int forward_com_max_blocks_per_sm(int mode, int wpb) {
    int n = 0;
    const void* f = (mode == 1) ? (const void*)forward_com_kernel<1>
                  : (mode == 2) ? (const void*)forward_com_kernel<2> : (const void*)forward_com_kernel<3>;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, 32 * wpb, 0);
    return n;
}

int adjoint_com_max_blocks_per_sm(int mode, int wpb) {
    int n = 0;
    const void* f = (mode == 1)   ? (const void*)adjoint_com_kernel<1>
                    : (mode == 2) ? (const void*)adjoint_com_kernel<2>
                    : (mode == 3) ? (const void*)adjoint_com_kernel<3>
                    : (mode == 4) ? (const void*)adjoint_com_kernel<4>
                                  : (const void*)adjoint_com_kernel<5>;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, 32 * wpb, 0);
    return n;
}

cudaError_t launch_l2l(double* L, const int* parents, int n_list, const int* children, const int* ninfo,
                       const double* hinv, cudaStream_t s) {
    if (n_list == 0) return cudaSuccess;
    l2l_kernel<<<blocks_for(1LL * n_list * 8 * NCELL, 128), 128, 0, s>>>(L, parents, n_list, children, ninfo, hinv);
    return counted(cudaGetLastError());
}

cudaError_t launch_l2l_adjoint(double* Lb, const int* parents, int n_list, const int* children, const int* ninfo,
                               const double* hinv, cudaStream_t s) {
    if (n_list == 0) return cudaSuccess;
    l2l_adjoint_kernel<<<blocks_for(1LL * n_list * NCELL, 128), 128, 0, s>>>(Lb, parents, n_list, children, ninfo,
                                                                             hinv);
    return counted(cudaGetLastError());
}

cudaError_t launch_fp64_probe(double* out, int blocks, int iters, int variant, cudaStream_t s) {
    if (variant == 0) fp64_probe_kernel<0><<<blocks, 256, 0, s>>>(out, iters);
    else if (variant == 1) fp64_probe_kernel<1><<<blocks, 256, 0, s>>>(out, iters);
    else fp64_probe_contraction_kernel<<<blocks, 256, 0, s>>>(out, iters);
    return counted(cudaGetLastError());
}

}  // namespace otk
