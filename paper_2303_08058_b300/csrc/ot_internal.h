// Library-internal declarations shared by the host code (ot_lib.cu) and the
// kernels (ot_kernels.cu).  Not part of the public ABI (include/ot.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ot_contract_counts.h"

namespace otk {

constexpr int NCELL = 512;        // cells per 8^3 sub-grid
constexpr int NCOMP = 20;         // moments / Taylor coefficients of orders 0..3
constexpr int NRED = 16;          // traceless-reduced components
constexpr int DROW = 36;          // doubles per derivative-table row
constexpr int NOFF = 15 * 15 * 15;  // integer offsets in [-7, 7]^3
constexpr int NVROW = 14 * 14 * 14; // rows of the virtual-child table: q = 2o + c in [-6, 7]^3
constexpr int MAXLEV = 21;        // levels 0..20
constexpr int PART_VALS = 28;     // accumulators of a chunk: 16 coefficients, 3 + 9 angular

// Parity pattern of reduced component q (bit 0: x, bit 1: y, bit 2: z order
// odd).  Reduced order: 0; x y z; xx xy xz yy yz; xxx xxy xxz xyy xyz yyy yyz.
__host__ __device__ constexpr int comp_parity(int q) {
    return static_cast<int>((0x4271421605304210ULL >> (4 * q)) & 0xfULL);
}
// FP64 instructions per lane of a reflection class with zero pattern Z: the
// Walsh-Hadamard transform over the d = 3 - |Z| sign axes (d 2^d adds) and one
// FMA per component whose parity avoids Z (the others are exactly zero).
__host__ __device__ constexpr int class_fmas(int Z) {
    int n = 0;
    for (int q = 0; q < NRED; ++q) n += (comp_parity(q) & Z) == 0;
    return n;
}
__host__ __device__ constexpr int class_adds(int Z) {
    return (3 - ((Z & 1) + ((Z >> 1) & 1) + ((Z >> 2) & 1))) << (3 - ((Z & 1) + ((Z >> 1) & 1) + ((Z >> 2) & 1)));
}

// Neighbour-table entry (one per 3x3x3 neighbour of a sub-grid at its own level).
//   x: node index (real node, or the coarse leaf of a virtual descendant)
//   y: kind (bits 0-1) | d (bits 2-4, virtual depth) | ov.x << 8 | ov.y << 16 | ov.z << 24
// kind: 0 empty, 1 multipole cells (non-leaf node), 2 point masses (leaf node),
// 3 virtual descendant of a coarser leaf: level-l local cell s maps to the
// leaf's cell ((ov + s) >> d) per axis and holds 8^-d of its mass.
enum Kind : int { K_NONE = 0, K_MULTI = 1, K_LEAF = 2, K_VIRT = 3 };

// Stencil lists are packed offsets (ox + 8) | (oy + 8) << 8 | (oz + 8) << 16.
// Table row of offset o: (ox + 7) + 15 (oy + 7) + 225 (oz + 7); the row holds
// the derivatives of G at R = -o (unit spacing), i.e. for the pair
// target -> source at offset o.  The row of -o is NOFF - 1 - row(o).

// Each far list holds far_pairs entries standing for an offset o and its
// negation -o (both in the list), then far_len - far_pairs single offsets.
// The near and root lists are closed under negation: every entry is paired.
//
// Point masses at leaf targets (and multipole sources at non-leaf targets)
// walk the same far, near and root offsets grouped by reflection class: the
// offsets (±a, ±b, ±c) of one list, a, b, c >= 0.  A
// class entry is a | b << 8 | c << 16 | members << 24, member bit i standing
// for the offset with x negated if i & 1, y if i & 2, z if i & 4 (for a zero
// component only the bit-clear member).  Entries are grouped by the zero
// pattern Z (bit 0: a == 0, bit 1: b == 0, bit 2: c == 0): group Z spans
// [zoff[Z], zoff[Z + 1]).  Offsets of classes that would cost more than their
// +-o pairs and singles follow as pairs, then singles.  The far class list of
// parity p is the far list of parity 0 reflected on the axes set in p, so
// every parity has the same class counts.  The point-mass and multipole
// class lists differ only in which classes stay pairs and singles (their
// costs differ).
struct Lists {
    const int* lists;      // far[8][far_len] | near | root | cfar[8][cf_stride] | cnear | mfar[8][mf_stride] | mroot
    int far_len, far_pairs, near_len, root_len;
    int near_off, root_off;
    int cf_off, cf_stride, cf_pairs, cf_singles;   // far classes; leftover pairs and singles follow zoff[7]
    int cn_off, cn_pairs;                          // near classes, then leftover pairs
    int cf_z[8], cn_z[8];                          // class group bounds by zero pattern
    // multipole sources by class: far lists per parity and the root list
    int mf_off, mf_stride, mf_pairs, mf_singles, mf_z[8];
    int mr_off, mr_pairs, mr_z[8];
    // per group Z with a > 0: the number of x-complete entries at its start
    // (both or neither x member at every (y, z) sign), which may read their
    // first transform stage from the prebuilt x butterflies
    int cf_x[8], cn_x[8], mf_x[8], mr_x[8];
    // per point-mass group Z with a, b > 0: the number of xy-complete entries
    // at the start of the x-complete head (all four or none of the (x, y)
    // members at every z sign), which may read their first two stages from
    // the (x, y) table
    int cf_xy[8], cn_xy[8];
    // the same for the multipole lists (far per parity, root): xy-complete
    // entries at the start of the x-complete head, which may read their first
    // two stages from the reduced moments' (x, y) table
    int mf_xy[8], mr_xy[8];
    // a leaf target's multipole sources (refined neighbours) and a non-leaf
    // target's point masses (leaf neighbours) paired along one axis A: per
    // A, the far list of each parity (stride ap_len[A]) as
    // ap_pairs[A] entries o with o_A > 0 whose reflection along A is also in
    // the list, then the remaining offsets as singles
    int ap_off[3], ap_len[3], ap_pairs[3];
};

struct FwdParams {
    const int* items;      // packed (node << 4) | (parity << 1) | half
    int n_items;
    int* counter;          // persistent queue head (zeroed before the launch)
    const int2* nbr;       // [n][27]
    const int* ninfo;      // [n]: level | is_leaf << 8
    const double* Dt;      // [NOFF][DROW]
    Lists L;
    const double* Mhat;    // [n][16][512] reduced scaled moments (non-leaf nodes)
    const double* m;       // [n][512]
    const float2* mf;      // [n][512] masses as double-float (hi, lo), or null for FP64
    const float* Dt32;     // [NOFF][32] hi then lo parts of the 16 point-mass derivatives
    const float2* Mf;      // [n][16][512] reduced moments as (hi, lo) pairs, or null (FP64 multipole pass)
    const float2* Dt2;     // [NOFF][DROW] the derivative table as (hi, lo) pairs
    double* Lout;          // [n][20][512]
    double* Lc;            // [n][3][512] or null
    int accumulate;
    int n_nodes;
    int* status;           // [2]: first error code, its item
    double hinv[MAXLEV];   // 1 / h_l
    // explicit expansion centres (centre-of-mass mode)
    const double* C;       // [n][3][512] or null
    const int* ncoord;     // [n][3] node positions
    double hreal[MAXLEV];  // h_l
    // coarse leaf targets refined virtually next to refined sub-grids
    const int* child_of;   // [n][8] child node per octant (x fastest), -1 for leaves
    const double* Dv;      // [NVROW][16] virtual-child mean rows (built by build_grid)
    // chunked items (item bits 26-29: chunk index); null: every item is whole
    const int2* cinfo;     // [n]: partial slot base, counter base << 4 | (chunks - 1); x < 0: whole
    double* part;          // [slots][PART_VALS][32] chunk accumulators
    int* chunk_ctr;        // [counters] chunks finished per (node, parity, half), zeroed per launch
    // prebuilt x butterflies (null: not built for this launch), per slot of a
    // space of regions (nodes and virtual blocks): X around non-leaf nodes, M
    // around leaf nodes; nslot[node][j] is the slot of the node's neighbour
    // region j in its own kind's space (-1: outside the domain)
    const double* Sx;      // [X slot][7][16][2][512]: Mhat(c + a x) +- Mhat(c - a x), multipole cells
    const double* Sm;      // [M slot][7][2][512]: the same for the point masses
    const float2* Smf;     // the masses' table as double-float (hi, lo) pairs (double-float point masses)
    const double* Sxy;     // [M slot][49: (a - 1) 7 + b - 1][4][512]: the masses at c + (+-a, +-b, 0)
                           // transformed over x and y (null: not built)
    const double* Sxym;    // [X slot][49][16][512][4]: the same for the reduced moments, component by
                           // component, a cell's four channels adjacent (null: not built)
    const int* nslot;      // [n][27]
};

struct AdjParams {
    const int* items;      // packed (src << 4) | (parity << 1) | half; src >= n_nodes: virtual
    int n_items;
    int* counter;
    const int2* nbr;       // [n][27] real nodes
    const int2* vnbr;      // [nvirt][27] virtual nodes
    const int* ninfo;      // [n]
    const int* vinfo;      // [nvirt]: level
    const double* Dt;
    Lists L;
    const double* Lrbar;   // [n][16][512] reduced scaled adjoint of L
    double* Mbar;          // [n][20][512] or null
    double* mbar;          // [n][512] or null
    double* vbar;          // [nvirt][512]
    int n_nodes;
    int* status;
    double hinv[MAXLEV];
    const double* C;       // [n][3][512] or null (centre-of-mass mode)
    const int* ncoord;     // [n][3]
    const int* vcoord;     // [nvirt][3] positions of virtual sub-grids at their level
    double hreal[MAXLEV];
    const int* child_of;   // as in FwdParams
    const double* Dv;
    // double-float adjoint
    const float2* Lf;      // [n][16][512] reduced L-bar as (hi, lo) pairs
    const float2* Dt2;     // [NOFF][DROW] the derivative table as (hi, lo) pairs
    const float* Dt32;     // [NOFF][32] hi then lo parts of the 16 point-mass derivatives
    // prebuilt x butterflies of the targets' reduced L-bar (null: not built)
    const double* Tx;      // [X slot][7][16][2][512]: Lrbar(c + a x) +- Lrbar(c - a x) over real cells
    // the point-mass scatter's x stage deferred (null: scatter to mbar directly):
    // a leaf target with leaf or empty neighbours adds its x-complete classes'
    // two x channels at the positions t + (0, +-b, +-c), and a later pass
    // (xbutterfly_masses_adjoint) forms the members' sums and differences
    double* Sbar;          // [M slot][7][2][512], zeroed before the launch
    const int* nslot;      // [n][27]: neighbour regions' slots (M for leaf nodes, X for non-leaf)
    // chunked multipole gather items (bit 31 set: source in bits 4-25, chunk
    // index in bits 26-29); null: every item is whole
    const int2* cinfo;     // [n]: partial slot base, counter base << 4 | (chunks - 1); x < 0: whole
    double* part;          // [slots][NRED][32] chunk accumulators
    int* chunk_ctr;        // [counters] chunks finished per (source, parity, half), zeroed per launch
};

// point-mass adjoint organised by target cells (the forward's walk) with the
// contributions scattered into mbar by atomic adds
struct ScatParams {
    const int* items;      // forward work items (node << 4 | parity << 1 | half)
    int n_items;
    int* counter;
    const int2* nbr;
    const int* ninfo;
    const double* Dt;
    Lists L;
    const double* Lrbar;   // [n][16][512]
    double* mbar;          // [n][512], zeroed before the launch
    int n_nodes;
    int* status;
    const int* child_of;   // as in FwdParams
    const double* Dv;
    double* Sbar;          // as in AdjParams (null here: the plain schedule scatters directly)
    const int* nslot;
};

struct PrepParams {
    const double* src;     // M [n][20][512] (forward) or Lbar (adjoint)
    double* dst;           // [n][16][512]
    const int* nodes;      // node list
    int n_list;
    const int* ninfo;
    double hinv[MAXLEV];
};

// node info bits (ninfo): level (0-7), leaf (8), and whether the node's
// classes may read the prebuilt x butterflies: bit 9 multipole sources (a
// non-leaf node whose 26 neighbours are all multipole or empty), bit 10
// point masses (a leaf node whose neighbours are all leaf or empty)
constexpr int NI_XMULTI = 1 << 9;
constexpr int NI_XMASS = 1 << 10;
// bit 11: a non-leaf source whose multipole gather may read the targets'
// prebuilt L-bar x butterflies (no virtual neighbour)
constexpr int NI_XGATHER = 1 << 11;
// bits 13-14: the axis along which a node's target items split their two
// halves (0 z, 1 x, 2 y): the axis of the node's faces whose neighbours hold
// no source of its passes, so that a warp's lanes reach such a face together
constexpr int NI_SLAB_SHIFT = 13;
// bits 15-16: the axis (0 x, 1 y, 2 z) along which a node's sources of the
// other kind pair with their reflections (a leaf node's multipole sources, a
// non-leaf node's point masses): the axis with the fewest faces on
// neighbours holding such sources, so that both members of a pair tend to
// lie in the same neighbour
constexpr int NI_APAIR_SHIFT = 15;

// launchers (ot_kernels.cu)
// one_block_per_sm: the grid holds one block per SM, so the FP64 multipole
// pass may take the register budget of a single resident block
cudaError_t launch_forward(const FwdParams& p, int mode, bool persistent, int wpb, int grid,
                           cudaStream_t s, bool one_block_per_sm = false);
cudaError_t launch_adjoint(const AdjParams& p, int mode, bool persistent, int wpb, int grid,
                           cudaStream_t s);
cudaError_t launch_prescale_moments(const PrepParams& p, cudaStream_t s);
// x-butterfly builders over the slots of a region space: snb [slots][27]
// holds each slot's region's neighbour entries
cudaError_t launch_xbutterfly_moments(const int2* snb, int n_slots, const double* Mhat, int n_nodes, double* Sx,
                                      cudaStream_t s);
cudaError_t launch_xbutterfly_lbar(const int2* snb, int n_slots, const double* Lrbar, int n_nodes, double* Tx,
                                   cudaStream_t s);
// the scatter's deferred x stage: per point-mass region of space M (own
// entry ent, M slots of its regions at x-1, x, x+1 in xs)
cudaError_t launch_xbutterfly_masses_adjoint(const int2* ent, const int* xs, int n_members, const double* Sbar,
                                             int n_nodes, double* mbar, cudaStream_t s);
cudaError_t launch_xybutterfly_masses(const int2* snb, int n_slots, const double* m, int n_nodes, double* Sxy,
                                      cudaStream_t s);
cudaError_t launch_xybutterfly_moments(const int* ys, int n_slots, const double* Sx, double* Sxym, cudaStream_t s);
cudaError_t launch_xbutterfly_masses(const int2* snb, int n_slots, const double* m, int n_nodes, double* Sm,
                                     cudaStream_t s);
cudaError_t launch_prescale_adjoint(const PrepParams& p, cudaStream_t s);
cudaError_t launch_restrict_virtual(const double* vbar, const int* vmap, int n_pairs_map,
                                    double* mbar, cudaStream_t s);
cudaError_t launch_cube_moments(const double* rho, double* M, double* m, const int* nodes, int n_list,
                                const int* ninfo, const double* hinv, cudaStream_t s);
cudaError_t launch_geometric_centres(double* C, const int* nodes, int n_list, const int* ninfo, const int* ncoord,
                                     double h0, cudaStream_t s);
cudaError_t launch_m2m_com(double* M, double* m, double* C, const int* parents, int n_list, const int* children,
                           const int* ninfo, const int* ncoord, double h0, cudaStream_t s);
cudaError_t launch_l2l_com(double* L, const double* C, const int* parents, int n_list, const int* children,
                           const int* ninfo, const int* ncoord, double h0, cudaStream_t s);
cudaError_t launch_l2l_com_adjoint(double* Lb, const double* C, const int* parents, int n_list, const int* children,
                                   const int* ninfo, const int* ncoord, double h0, cudaStream_t s);
cudaError_t launch_forward_com(const FwdParams& p, int mode, int wpb, int grid, cudaStream_t s);
cudaError_t launch_adjoint_com(const AdjParams& p, int mode, int wpb, int grid, cudaStream_t s);
int forward_com_max_blocks_per_sm(int mode, int wpb);
int adjoint_com_max_blocks_per_sm(int mode, int wpb);
int deriv_flops(int ncomp);   // algorithmic FLOPs of one per-pair derivative evaluation (16, 19 or 31 components)
int adjoint_com_max_blocks_per_sm(int mode, int wpb);
cudaError_t launch_m2m(double* M, double* m, const int* parents, int n_list, const int* children,
                       const int* ninfo, const double* hinv, cudaStream_t s);
cudaError_t launch_moments_adjoint_init(const double* Mbar, const double* mbar, double* Mb, int n,
                                        cudaStream_t s);
cudaError_t launch_m2m_adjoint(double* Mb, const int* parents, int n_list, const int* children,
                               const int* ninfo, const double* hinv, cudaStream_t s);
cudaError_t launch_cube_adjoint(const double* Mb, double* rhobar, const int* nodes, int n_list,
                                const int* ninfo, const double* hinv, cudaStream_t s);
cudaError_t launch_l2l(double* L, const int* parents, int n_list, const int* children, const int* ninfo,
                       const double* hinv, cudaStream_t s);
cudaError_t launch_l2l_adjoint(double* Lb, const int* parents, int n_list, const int* children,
                               const int* ninfo, const double* hinv, cudaStream_t s);
cudaError_t launch_fp64_probe(double* out, int blocks, int iters, int variant, cudaStream_t s);
cudaError_t launch_scatter_adjoint(const ScatParams& p, bool persistent, int wpb, int grid, cudaStream_t s);
int scatter_max_blocks_per_sm(int wpb);
int forward_max_blocks_per_sm(int mode, int wpb);   // mode 6/7: double-float point masses
cudaError_t launch_split_moments(const double* Mhat, float2* Mf, const int* nodes, int n_list, cudaStream_t s);
cudaError_t launch_split_masses(const double* m, float2* mf, size_t n, cudaStream_t s);
int adjoint_max_blocks_per_sm(int mode, int wpb);

// Kernel launches issued by the launchers above: a process-wide total and
// the calling thread's own count.  A launcher counts its kernel when the
// launch succeeds; a graph capture takes its kernels back out
// (launch_count_adjust with minus the thread's count over the capture) and
// every replay of the graph adds them again.
long long launch_count_total();
long long launch_count_thread();
void launch_count_adjust(long long delta);

}  // namespace otk
