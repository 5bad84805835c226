// Host side of libotfmm: grid geometry (neighbour tables, stencils, the
// derivative table, virtual descendants), work lists and their ordering,
// CUDA-graph capture and replay, the tile-shape autotuner, and the C ABI.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <array>
#include <atomic>
#include <chrono>
#include <deque>
#include <map>
#include <mutex>
#include <set>
#include <new>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "ot.h"
#include "ot_internal.h"

using namespace otk;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------

static thread_local std::string g_last_error;

static ot_status fail(ot_status code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

#define OT_CUDA(call)                                                                        \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(OT_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),    \
                        __FILE__, __LINE__);                                                 \
    } while (0)

// ---------------------------------------------------------------------------
// derivative table: d^K G for G = -1/|R| at integer R, by composing truncated
// multivariate Taylor series:  |R + e|^2 = r^2 (1 + w),  w = (2 R.e + e.e) / r^2,
// (1 + w)^(-1/2) = sum_k binom(-1/2, k) w^k, truncated at total degree 4;
// d^K G = K! * (coefficient of e^K).
// ---------------------------------------------------------------------------

namespace {

struct Poly4 {
    double c[5][5][5];   // c[a][b][d] for a + b + d <= 4
    Poly4() { std::memset(c, 0, sizeof(c)); }
};

Poly4 pmul(const Poly4& x, const Poly4& y) {
    Poly4 z;
    for (int a = 0; a <= 4; ++a)
        for (int b = 0; a + b <= 4; ++b)
            for (int d = 0; a + b + d <= 4; ++d) {
                if (x.c[a][b][d] == 0.0) continue;
                for (int e = 0; a + e <= 4; ++e)
                    for (int f = 0; a + b + e + f <= 4; ++f)
                        for (int g = 0; a + b + d + e + f + g <= 4; ++g)
                            z.c[a + e][b + f][d + g] += x.c[a][b][d] * y.c[e][f][g];
            }
    return z;
}

double fact(int k) {
    double r = 1.0;
    for (int i = 2; i <= k; ++i) r *= i;
    return r;
}

// row layout: IND16 (ranks 0..3 with at most one z), zz xzz yzz zzz, rank 4 in storage order
const int ROW_EXP[35][3] = {
    {0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 2, 0}, {0, 1, 1},
    {3, 0, 0}, {2, 1, 0}, {2, 0, 1}, {1, 2, 0}, {1, 1, 1}, {0, 3, 0}, {0, 2, 1},
    {0, 0, 2}, {1, 0, 2}, {0, 1, 2}, {0, 0, 3},
    {4, 0, 0}, {3, 1, 0}, {3, 0, 1}, {2, 2, 0}, {2, 1, 1}, {2, 0, 2}, {1, 3, 0}, {1, 2, 1}, {1, 1, 2},
    {1, 0, 3}, {0, 4, 0}, {0, 3, 1}, {0, 2, 2}, {0, 1, 3}, {0, 0, 4}};

void derivative_row(const double R[3], double* row) {
    const double r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
    Poly4 w;
    w.c[1][0][0] = 2.0 * R[0] / r2;
    w.c[0][1][0] = 2.0 * R[1] / r2;
    w.c[0][0][1] = 2.0 * R[2] / r2;
    w.c[2][0][0] = 1.0 / r2;
    w.c[0][2][0] = 1.0 / r2;
    w.c[0][0][2] = 1.0 / r2;
    // binom(-1/2, k): 1, -1/2, 3/8, -5/16, 35/128 ; Horner in w
    const double bk[5] = {1.0, -0.5, 0.375, -0.3125, 0.2734375};
    Poly4 s;
    s.c[0][0][0] = bk[4];
    for (int k = 3; k >= 0; --k) {
        s = pmul(s, w);
        s.c[0][0][0] += bk[k];
    }
    const double scale = -1.0 / std::sqrt(r2);
    for (int q = 0; q < 35; ++q) {
        const int a = ROW_EXP[q][0], b = ROW_EXP[q][1], d = ROW_EXP[q][2];
        row[q] = scale * s.c[a][b][d] * fact(a) * fact(b) * fact(d);
    }
    row[35] = 0.0;
}

inline int pack_offset(int ox, int oy, int oz) { return (ox + 8) | ((oy + 8) << 8) | ((oz + 8) << 16); }
inline int fdiv2(int a) { return (a >= 0) ? a / 2 : -((1 - a) / 2); }   // floor(a / 2)
// a class entry whose members come in x pairs: at every (y, z) sign both or
// neither of the members with x = +a, -a
inline bool x_complete(int e) {
    const unsigned m = static_cast<unsigned>(e) >> 24;
    for (int q = 0; q < 4; ++q)
        if (((m >> (2 * q)) & 1u) != ((m >> (2 * q + 1)) & 1u)) return false;
    return true;
}

// a class entry whose members come in (x, y) quadruples: at every z sign
// all four or none of the members with x = +-a, y = +-b
inline bool xy_complete(int e) {
    const unsigned m = static_cast<unsigned>(e) >> 24;
    for (int r = 0; r < 2; ++r) {
        const unsigned q = (m >> (4 * r)) & 15u;
        if (q != 0u && q != 15u) return false;
    }
    return true;
}

// Locational code of node (l, x, y, z), 0 <= x, y, z < 2^l: a leading 1 at
// bit 3l marks the level, so the codes of a level lie in [2^3l, 2^(3l+1))
// and never meet another level's; levels 0..21 fit in 64 bits.
inline uint64_t node_key(int l, int x, int y, int z) {
    return (uint64_t{1} << (3 * l)) | (static_cast<uint64_t>(x) << (2 * l)) | (static_cast<uint64_t>(y) << l) |
           static_cast<uint64_t>(z);
}

// the cell a lane of a target item holds (the kernels' lane_cell_slab)
inline void lane_cell_host(int lane, int par, int half, int slab, int& x, int& y, int& z) {
    const int u = lane & 3, v = (lane >> 2) & 3, w = 2 * half + (lane >> 4);
    const int cx = slab == 1 ? w : u, cy = slab == 2 ? w : (slab == 1 ? u : v), cz = slab == 0 ? w : v;
    x = (par & 1) + 2 * cx;
    y = ((par >> 1) & 1) + 2 * cy;
    z = ((par >> 2) & 1) + 2 * cz;
}

// The axis along which a node's target items split their halves (0 z, 1 x,
// 2 y): the one with the most faces whose neighbour holds no source of the
// node's main pass (refined or outside the domain for a leaf; leaf, virtual
// or outside for a non-leaf node), z on ties.  Lanes then reach such a face
// together, and entries that only reach it are skipped by whole warps.
inline int slab_axis(const int2* nb27, bool leaf) {
    static const int face[6] = {12, 14, 10, 16, 4, 22};   // -x +x -y +y -z +z
    int bad[3] = {0, 0, 0};                               // x, y, z
    for (int f = 0; f < 6; ++f) {
        const int k = nb27[face[f]].y & 3;
        const bool none = leaf ? (k == K_MULTI || k == K_NONE) : (k != K_MULTI);
        if (none) bad[f / 2]++;
    }
    if (bad[0] > bad[2] && bad[0] >= bad[1]) return 1;
    if (bad[1] > bad[2] && bad[1] > bad[0]) return 2;
    return 0;
}

// the axis (0 x, 1 y, 2 z) along which a node's sources of the other kind
// pair with their reflections (a leaf node's multipole sources, a non-leaf
// node's point masses): the one with the fewest faces on neighbours holding
// such sources; ties go to the axis its items split their halves along
// (slab 0 z, 1 x, 2 y), then to the lower axis
inline int pair_axis(const int2* nb27, int slab, bool leaf) {
    static const int face[6] = {12, 14, 10, 16, 4, 22};   // -x +x -y +y -z +z
    int refined[3] = {0, 0, 0};
    for (int f = 0; f < 6; ++f) {
        const int k = nb27[face[f]].y & 3;
        if (leaf ? k == K_MULTI : (k == K_LEAF || k == K_VIRT)) refined[f / 2]++;
    }
    const int split = slab == 0 ? 2 : slab == 1 ? 0 : 1;
    int best = split;
    for (int a = 0; a < 3; ++a)
        if (refined[a] < refined[best] || (refined[a] == refined[best] && a != split && best != split && a < best))
            best = a;
    return best;
}


}  // namespace

// ---------------------------------------------------------------------------
// the grid handle
// ---------------------------------------------------------------------------

struct GraphKey {
    int op;
    const void* a;
    const void* b;
    const void* c;
    const void* d;
    int w, bps;
    const void* e;
    bool operator<(const GraphKey& o) const {
        return std::tie(op, a, b, c, d, w, bps, e) < std::tie(o.op, o.a, o.b, o.c, o.d, o.w, o.bps, o.e);
    }
};

struct M2MLevel {
    int level;
    std::vector<int> parents;
    std::vector<int> children;   // 8 per parent, octant x fastest
    int* d_parents = nullptr;
    int* d_children = nullptr;
};

struct ot_grid {
    int n = 0, nvirt = 0, max_level = 0, device = 0, num_sms = 0;
    double h0 = 1.0;
    std::vector<int> level, is_leaf;
    std::vector<int2> nbr, vnbr;
    std::vector<int> ninfo, vinfo;
    std::vector<int> lists;
    int far_len = 0, far_pairs = 0, near_len = 0, root_len = 0, far_offsets = 0;
    Lists Lh = {};                      // list layout; Lh.lists is set to d_lists after the upload
    double hinv[MAXLEV];

    // device buffers
    std::vector<void*> allocs;
    int2* d_nbr = nullptr;
    int2* d_vnbr = nullptr;
    int* d_ninfo = nullptr;
    int* d_vinfo = nullptr;
    int* d_ncoord = nullptr;            // [n][3] sub-grid positions (explicit-centre kernels)
    int* d_vcoord = nullptr;            // [nvirt][3]
    int* d_child_of = nullptr;          // [n][8] children (coarse leaves refined virtually as targets)
    double* d_Dv = nullptr;             // [NVROW][16] virtual-child mean rows
    double* d_Dt = nullptr;
    float* d_Dt32 = nullptr;            // double-float split of the point-mass derivatives
    float2* d_mf = nullptr;             // masses as double-float pairs (scratch)
    int precision = 0;                  // OT_PREC_*: 0 FP64; 1 double-float point masses; 2 both passes
    float2* d_Mf = nullptr;             // reduced moments as double-float pairs (scratch)
    float2* d_Dt2 = nullptr;            // the derivative table as double-float pairs
    int maxb_emu2[4][9] = {};           // forward with double-float multipole contractions, modes 1 and 3
    int maxb_adj_emu[13][9] = {};       // double-float adjoint, modes 9, 12 (= 1, 4 + 8)
    int* d_lists = nullptr;
    double* d_hinv = nullptr;
    int* d_items_fwd[4] = {nullptr, nullptr, nullptr, nullptr};     // LPT order, by mode
    int n_items_fwd[4] = {0, 0, 0, 0};
    int* d_items_fwd_node = nullptr;                                 // node order (plain path)
    // chunked items of the multipole and fused passes (table path)
    std::vector<int> itemsc_fwd[4], itemsc_node, itemc_node_start;
    std::vector<int2> cinfo;            // [n]: partial slot base, counter base << 4 | (chunks - 1); x < 0: whole
    int n_part_slots = 0, n_chunk_ctrs = 0;
    int* d_itemsc_fwd[4] = {nullptr, nullptr, nullptr, nullptr};
    int n_itemsc_fwd[4] = {0, 0, 0, 0};
    int* d_itemsc_node = nullptr;
    int2* d_cinfo = nullptr;
    double* d_part = nullptr;           // [slots][28][32] chunk accumulators
    int* d_chunk_ctr = nullptr;         // [counters] chunks finished per (node, parity, half)
    // prebuilt x butterflies of the classes' first transform stage, per slot
    // of two spaces of regions (nodes and virtual blocks): M around leaf
    // nodes, X around non-leaf nodes
    std::vector<int> nslot;             // [n][27]: slot of each neighbour region in the node's space, -1: none
    std::vector<int2> snbM, snbX;       // [slot][27]: each slot's region's neighbour entries
    int n_slotM = 0, n_slotX = 0;
    int n_slotXY = 0;                   // M slots [0, n_slotXY): the leaves' z columns, the (x, y) table's
    int n_slotXyz = 0;                  // X slots [0, n_slotXyz): the yz planes of the non-leaf nodes, the
                                        // x tables' (read only at t + (0, +-b, +-c))
    int n_slotXz = 0;                   // X slots [0, n_slotXz): their z columns, the moments' (x, y) table's
    int* d_nslot = nullptr;
    int2* d_snbM = nullptr;
    int2* d_snbX = nullptr;
    std::vector<int2> mem_ent;          // point-mass regions of M: own entry (leaf node or virtual block)
    std::vector<int> mem_xs;            // [member][3]: M slots of the regions at x-1, x, x+1 (-1: none)
    std::vector<int> xym_ys;            // [X slot < n_slotXz][3]: X slots of the regions at y-1, y, y+1
    int* d_xym_ys = nullptr;
    int2* d_mem_ent = nullptr;
    int* d_mem_xs = nullptr;
    int* d_leaf = nullptr;              // childless nodes (cube moments)
    double* d_Sx = nullptr;             // [X slot][7][16][2][512]: reduced moments
    double* d_Sm = nullptr;             // [M slot][7][2][512]: masses
    double* d_Sxy = nullptr;            // [M slot][49][4][512]: the masses' (x, y) butterflies
    double* d_Sxym = nullptr;           // [X slot][49][16][512][4]: the reduced moments' (x, y) butterflies
    bool use_xym = false;               // the moments' (x, y) table fits (its size is capped)
    bool use_xy = false;                // the (x, y) table fits (its size is capped)
    float2* d_Smf = nullptr;            // the masses' table as double-float pairs
    double* d_Tx = nullptr;             // [X slot][7][16][2][512]: reduced L-bar of real cells
    double* d_Sbar = nullptr;           // [M slot][7][2][512]: the point-mass scatter's deferred x stage
    // chunked multipole gather items of the adjoint (modes 1 and 3, and the
    // default adjoint's merged list); they share d_part and d_chunk_ctr
    std::vector<int> itemsc_adj[4], itemsc_adj_node[4], itemc_adj_start[4], itemsc_adj_fast1;
    std::vector<int2> cinfo_adj;
    int n_part_slots_adj = 0, n_chunk_ctrs_adj = 0;
    int* d_itemsc_adj[4] = {nullptr, nullptr, nullptr, nullptr};
    int n_itemsc_adj[4] = {0, 0, 0, 0};
    int* d_itemsc_adj_node[4] = {nullptr, nullptr, nullptr, nullptr};
    int* d_itemsc_adj_fast1 = nullptr;
    int n_itemsc_adj_fast1 = 0;
    int2* d_cinfo_adj = nullptr;
    std::vector<int> node_item_start;                                // [n + 1] into d_items_fwd_node
    int* d_items_adj[4] = {nullptr, nullptr, nullptr, nullptr};
    int n_items_adj[4] = {0, 0, 0, 0};
    int* d_items_adj_node[4] = {nullptr, nullptr, nullptr, nullptr};   // source order (plain path)
    int* d_items_adj_fast[2] = {nullptr, nullptr};    // [0]: point-mass scatter items only, [1]: + multipole gather
    int n_items_adj_fast[2] = {0, 0};
    std::vector<int> adj_item_start[4];                                // [n + nvirt + 1]
    int maxb_fwd[4][9] = {};
    int maxb_adj[4][9] = {};
    int maxb_scat[9] = {};
    int maxb_emu[4][9] = {};            // forward with double-float point masses, modes 2 and 3
    int maxb_com_fwd[4][9] = {};        // explicit expansion centres
    int maxb_com_adj[6][9] = {};        // modes 1-3 gather, 4-5 with point-mass items by target
    int deterministic = 0;              // 1: point-mass adjoint as a gather (fixed summation order)
    long long flops_adj_det = 0, ops_adj_det = 0, flops_adj_fast = 0, ops_adj_fast = 0;
    long long fp64_ops_adj_det = 0, fp64_ops_adj_fast = 0;
    int* d_nonleaf = nullptr;
    int n_nonleaf = 0;
    int* d_all = nullptr;
    int* d_cube = nullptr;
    int n_cube = 0;
    std::vector<M2MLevel> m2m;       // deepest parents first
    int* d_vmap = nullptr;
    int vmap_rows = 0;
    double* d_Mhat = nullptr;
    double* d_Lrbar = nullptr;
    double* d_vbar = nullptr;
    double* d_Mb = nullptr;
    int* d_counters = nullptr;       // [0] forward, [1] adjoint gather, [2] adjoint scatter
    int* d_status = nullptr;         // [2]
    cudaStream_t cap_stream = nullptr;

    int schedule = OT_SCHED_PERSISTENT;
    int wpb = 4, bps = 0, use_graph = 1;
    std::map<GraphKey, cudaGraphExec_t> graphs;
    std::map<GraphKey, long long> graph_kernels;   // kernels recorded in each graph

    ot_grid_info_t info{};

    template <class T>
    ot_status alloc(T** out, size_t count) {
        void* p = nullptr;
        const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(OT_ENOMEM, "cudaMalloc of %zu bytes failed", bytes);
        }
        allocs.push_back(p);
        *out = static_cast<T*>(p);
        return OT_OK;
    }

    template <class T>
    ot_status upload(T** out, const std::vector<T>& v, cudaStream_t s) {
        ot_status st = alloc(out, v.size());
        if (st != OT_OK) return st;
        if (!v.empty()) OT_CUDA(cudaMemcpyAsync(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
        return OT_OK;
    }

    ~ot_grid() {
        for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
        for (void* p : allocs) cudaFree(p);
        if (cap_stream) cudaStreamDestroy(cap_stream);
    }
};

// Live handles: every entry point checks its handle against this set, so a
// destroyed or foreign pointer is refused (OT_EINVAL) instead of used.
static std::mutex g_handles_mu;
static std::set<const ot_grid*> g_handles;

static bool grid_live(const ot_grid* g) {
    std::lock_guard<std::mutex> lk(g_handles_mu);
    return g_handles.count(g) != 0;
}

// ---------------------------------------------------------------------------
// geometry
// ---------------------------------------------------------------------------

namespace {

struct Builder {
    const ot_grid_desc* desc;
    std::unordered_map<uint64_t, int> index;

    int find(int l, long x, long y, long z) const {
        if (l < 0 || x < 0 || y < 0 || z < 0) return -1;
        const long s = 1L << l;
        if (x >= s || y >= s || z >= s) return -1;
        auto it = index.find(node_key(l, (int)x, (int)y, (int)z));
        return it == index.end() ? -1 : it->second;
    }

    // neighbour entry for same-level node position q at level l
    ot_status entry(int l, const long q[3], bool for_adjoint, int2* out, int* vdepth, long* vq) const {
        out->x = -1;
        out->y = K_NONE;
        *vdepth = 0;
        const long s = 1L << l;
        for (int a = 0; a < 3; ++a)
            if (q[a] < 0 || q[a] >= s) return OT_OK;
        int j = find(l, q[0], q[1], q[2]);
        if (j >= 0) {
            out->x = j;
            out->y = desc->is_leaf[j] ? K_LEAF : K_MULTI;
            return OT_OK;
        }
        if (for_adjoint) return OT_OK;     // targets are real nodes only
        for (int d = 1; d <= l; ++d) {
            j = find(l - d, q[0] >> d, q[1] >> d, q[2] >> d);
            if (j < 0) continue;
            if (!desc->is_leaf[j]) return OT_OK;   // covered by a non-leaf without finer data
            if (d > 5) return fail(OT_EINVAL, "virtual descendant %d levels below its leaf (max 5)", d);
            unsigned ov[3];
            for (int a = 0; a < 3; ++a) ov[a] = static_cast<unsigned>(8 * (q[a] - ((q[a] >> d) << d)));
            out->x = j;
            out->y = static_cast<int>(K_VIRT | (d << 2) | (ov[0] << 8) | (ov[1] << 16) | (ov[2] << 24));
            *vdepth = d;
            for (int a = 0; a < 3; ++a) vq[a] = q[a];
            return OT_OK;
        }
        return OT_OK;
    }
};

}  // namespace

static ot_status build_grid(ot_grid* g, const ot_grid_desc* desc, cudaStream_t s) {
    const int n = desc->n_subgrids;
    g->n = n;
    g->h0 = desc->h0;
    g->level.assign(desc->level, desc->level + n);
    g->is_leaf.resize(n);
    Builder B;
    B.desc = desc;
    B.index.reserve(static_cast<size_t>(n) * 2);
    g->max_level = 0;
    for (int i = 0; i < n; ++i) {
        const int l = desc->level[i];
        if (l < 0 || l >= MAXLEV) return fail(OT_EINVAL, "node %d: level %d outside [0, %d]", i, l, MAXLEV - 1);
        const long s = 1L << l;
        for (int a = 0; a < 3; ++a) {
            const int c = desc->coord[3 * i + a];
            if (c < 0 || c >= s) return fail(OT_EINVAL, "node %d: coord %d outside [0, 2^%d)", i, c, l);
        }
        if (desc->is_leaf[i] > 1) return fail(OT_EINVAL, "node %d: is_leaf must be 0 or 1", i);
        g->is_leaf[i] = desc->is_leaf[i];
        auto ins = B.index.emplace(node_key(l, desc->coord[3 * i], desc->coord[3 * i + 1], desc->coord[3 * i + 2]), i);
        if (!ins.second) return fail(OT_EINVAL, "node %d duplicates node %d", i, ins.first->second);
        g->max_level = std::max(g->max_level, l);
    }
    for (int l = 0; l < MAXLEV; ++l) g->hinv[l] = std::ldexp(1.0, l) / desc->h0;

    // --- stencils -------------------------------------------------------------
    // far[p]: well separated at this level, parents not; near: not well
    // separated; root: well separated.  Each list is stored as entries o
    // standing for the pair {o, -o} when both are in it (flag bit 24; the
    // representative has the larger packed key), then the single offsets.
    const int c = 12;
    auto key = [](int ox, int oy, int oz) { return ((oz + 8) << 16) | ((oy + 8) << 8) | (ox + 8); };
    auto split = [&](const std::vector<std::array<int, 3>>& offs, std::vector<int>& pairs, std::vector<int>& singles) {
        std::set<int> in;
        for (auto& o : offs) in.insert(key(o[0], o[1], o[2]));
        for (auto& o : offs) {
            const int k = key(o[0], o[1], o[2]), kn = key(-o[0], -o[1], -o[2]);
            if (in.count(kn)) {
                if (k > kn) pairs.push_back(pack_offset(o[0], o[1], o[2]) | (1 << 24));
            } else {
                singles.push_back(pack_offset(o[0], o[1], o[2]));
            }
        }
    };
    std::vector<int> far_pair[8], far_single[8], near_pair, near_single, root_pair, root_single;
    std::vector<std::array<int, 3>> far_offs[8], near_offs, root_offs;
    for (int p = 0; p < 8; ++p) {
        const int px = p & 1, py = (p >> 1) & 1, pz = (p >> 2) & 1;
        std::vector<std::array<int, 3>>& offs = far_offs[p];
        for (int oz = -7; oz <= 7; ++oz)
            for (int oy = -7; oy <= 7; ++oy)
                for (int ox = -7; ox <= 7; ++ox) {
                    const int n2 = ox * ox + oy * oy + oz * oz;
                    const int qx = fdiv2(px + ox), qy = fdiv2(py + oy), qz = fdiv2(pz + oz);
                    if (n2 > c && qx * qx + qy * qy + qz * qz <= c) offs.push_back({ox, oy, oz});
                }
        split(offs, far_pair[p], far_single[p]);
    }
    {
        std::vector<std::array<int, 3>> nr, rt;
        for (int oz = -7; oz <= 7; ++oz)
            for (int oy = -7; oy <= 7; ++oy)
                for (int ox = -7; ox <= 7; ++ox) {
                    const int n2 = ox * ox + oy * oy + oz * oz;
                    if (n2 > 0 && n2 <= c) nr.push_back({ox, oy, oz});
                    if (n2 > c) rt.push_back({ox, oy, oz});
                }
        split(nr, near_pair, near_single);
        split(rt, root_pair, root_single);
        near_offs = nr;
        root_offs = rt;
    }
    for (int p = 1; p < 8; ++p)
        if (far_pair[p].size() != far_pair[0].size() || far_single[p].size() != far_single[0].size())
            return fail(OT_EINVAL, "internal: parity stencils differ in shape");
    if (!near_single.empty() || !root_single.empty())
        return fail(OT_EINVAL, "internal: near/root stencils not closed under negation");
    g->far_pairs = static_cast<int>(far_pair[0].size());
    g->far_len = g->far_pairs + static_cast<int>(far_single[0].size());
    g->near_len = static_cast<int>(near_pair.size());
    g->root_len = static_cast<int>(root_pair.size());
    g->lists.clear();
    for (int p = 0; p < 8; ++p) {
        g->lists.insert(g->lists.end(), far_pair[p].begin(), far_pair[p].end());
        g->lists.insert(g->lists.end(), far_single[p].begin(), far_single[p].end());
    }
    g->lists.insert(g->lists.end(), near_pair.begin(), near_pair.end());
    g->lists.insert(g->lists.end(), root_pair.begin(), root_pair.end());
    g->far_offsets = static_cast<int>(2 * far_pair[0].size() + far_single[0].size());

    // reflection classes of the far (per parity) and near offsets, for point
    // masses at leaf targets: a class is kept where its FP64 instructions per
    // lane (class_adds + class_fmas) are fewer than those of its +-o pairs
    // (18) and singles (16); its offsets are walked as pairs and singles
    // otherwise
    auto class_split = [&](const std::vector<std::array<int, 3>>& offs, std::vector<int> (&cls)[8],
                           std::vector<int>& pairs, std::vector<int>& singles, bool multipole) {
        std::map<int, std::vector<std::array<int, 3>>> byrep;
        for (auto& o : offs) byrep[std::abs(o[0]) | (std::abs(o[1]) << 8) | (std::abs(o[2]) << 16)].push_back(o);
        for (auto& kv : byrep) {
            const int a = kv.first & 0xff, b = (kv.first >> 8) & 0xff, cc = kv.first >> 16;
            const int Z = (a == 0 ? 1 : 0) | (b == 0 ? 2 : 0) | (cc == 0 ? 4 : 0);
            int members = 0;
            for (auto& o : kv.second) members |= 1 << ((o[0] < 0 ? 1 : 0) | (o[1] < 0 ? 2 : 0) | (o[2] < 0 ? 4 : 0));
            std::vector<int> pp, ss;
            split(kv.second, pp, ss);
            // FP64 instructions per lane: point masses 18 per pair, 16 per
            // single; multipole sources with the angular term 132 and 100
            const int ccost = multipole ? OT_MCLASS_ADDS[1][Z] + OT_MCLASS_FMAS[1][Z] : class_adds(Z) + class_fmas(Z);
            const int pcost = multipole ? 132 : 18, scost = multipole ? 100 : 16;
            if (ccost < static_cast<int>(pcost * pp.size() + scost * ss.size())) {
                cls[Z].push_back(kv.first | (members << 24));
            } else {
                pairs.insert(pairs.end(), pp.begin(), pp.end());
                singles.insert(singles.end(), ss.begin(), ss.end());
            }
        }
        // within a group with a > 0, the x-complete classes first (both or
        // neither of the x members at every (y, z) sign): their first
        // transform stage can come from the prebuilt x butterflies
        for (int z = 0; z < 8; z += 2) {
            auto xe = std::stable_partition(cls[z].begin(), cls[z].end(), [](int e) { return x_complete(e); });
            // and within that head, for a, b > 0, the xy-complete classes
            // first: their first two stages can come from the (x, y) table
            if (!(z & 2)) std::stable_partition(cls[z].begin(), xe, [](int e) { return xy_complete(e); });
        }
    };
    std::vector<int> cfar[8][8], cfar_pair[8], cfar_single[8], cnear[8], cnear_pair, cnear_single;
    for (int p = 0; p < 8; ++p) class_split(far_offs[p], cfar[p], cfar_pair[p], cfar_single[p], false);
    class_split(near_offs, cnear, cnear_pair, cnear_single, false);
    // the same for multipole sources: far lists and the root list
    std::vector<int> mfar[8][8], mfar_pair[8], mfar_single[8], mroot[8], mroot_pair, mroot_single;
    for (int p = 0; p < 8; ++p) class_split(far_offs[p], mfar[p], mfar_pair[p], mfar_single[p], true);
    class_split(root_offs, mroot, mroot_pair, mroot_single, true);
    for (int p = 1; p < 8; ++p) {
        bool same = mfar_pair[p].size() == mfar_pair[0].size() && mfar_single[p].size() == mfar_single[0].size();
        for (int z = 0; z < 8; ++z) same = same && mfar[p][z].size() == mfar[0][z].size();
        if (!same) return fail(OT_EINVAL, "internal: parity class stencils differ in shape");
    }
    if (!mroot_single.empty()) return fail(OT_EINVAL, "internal: root class stencil not closed under negation");
    for (int p = 1; p < 8; ++p) {
        bool same = cfar_pair[p].size() == cfar_pair[0].size() && cfar_single[p].size() == cfar_single[0].size();
        for (int z = 0; z < 8; ++z) same = same && cfar[p][z].size() == cfar[0][z].size();
        if (!same) return fail(OT_EINVAL, "internal: parity class stencils differ in shape");
    }
    if (!cnear_single.empty()) return fail(OT_EINVAL, "internal: near class stencil not closed under negation");
    Lists& Lh = g->Lh;
    std::memset(&Lh, 0, sizeof(Lh));
    Lh.far_len = g->far_len;
    Lh.far_pairs = g->far_pairs;
    Lh.near_len = g->near_len;
    Lh.root_len = g->root_len;
    Lh.near_off = 8 * g->far_len;
    Lh.root_off = 8 * g->far_len + g->near_len;
    // x-complete entries at the start of each group (the same count for every parity)
    auto xcount = [](const std::vector<int>& v) {
        int c = 0;
        while (c < static_cast<int>(v.size()) && x_complete(v[c])) ++c;
        return c;
    };
    auto xycount = [](const std::vector<int>& v) {
        int c = 0;
        while (c < static_cast<int>(v.size()) && xy_complete(v[c])) ++c;
        return c;
    };
    for (int z = 0; z < 8; ++z) {
        Lh.cf_xy[z] = (z & 3) ? 0 : xycount(cfar[0][z]);
        Lh.cn_xy[z] = (z & 3) ? 0 : xycount(cnear[z]);
        for (int p = 1; p < 8; ++p)
            if (!(z & 3) && xycount(cfar[p][z]) != Lh.cf_xy[z])
                return fail(OT_EINVAL, "internal: parity class stencils differ in shape");
        Lh.cf_x[z] = (z & 1) ? 0 : xcount(cfar[0][z]);
        Lh.cn_x[z] = (z & 1) ? 0 : xcount(cnear[z]);
        Lh.mf_x[z] = (z & 1) ? 0 : xcount(mfar[0][z]);
        Lh.mf_xy[z] = (z & 3) ? 0 : xycount(mfar[0][z]);
        Lh.mr_xy[z] = (z & 3) ? 0 : xycount(mroot[z]);
        for (int p = 1; p < 8; ++p)
            if (!(z & 3) && xycount(mfar[p][z]) != Lh.mf_xy[z])
                return fail(OT_EINVAL, "internal: parity class stencils differ in shape");
        Lh.mr_x[z] = (z & 1) ? 0 : xcount(mroot[z]);
        for (int p = 1; p < 8; ++p)
            if (((z & 1) == 0) && (xcount(cfar[p][z]) != Lh.cf_x[z] || xcount(mfar[p][z]) != Lh.mf_x[z]))
                return fail(OT_EINVAL, "internal: parity class stencils differ in shape");
    }
    Lh.cf_z[0] = 0;
    for (int z = 0; z < 7; ++z) Lh.cf_z[z + 1] = Lh.cf_z[z] + static_cast<int>(cfar[0][z].size());
    Lh.cf_pairs = static_cast<int>(cfar_pair[0].size());
    Lh.cf_singles = static_cast<int>(cfar_single[0].size());
    Lh.cf_stride = Lh.cf_z[7] + Lh.cf_pairs + Lh.cf_singles;
    Lh.cf_off = static_cast<int>(g->lists.size());
    for (int p = 0; p < 8; ++p) {
        for (int z = 0; z < 7; ++z) g->lists.insert(g->lists.end(), cfar[p][z].begin(), cfar[p][z].end());
        g->lists.insert(g->lists.end(), cfar_pair[p].begin(), cfar_pair[p].end());
        g->lists.insert(g->lists.end(), cfar_single[p].begin(), cfar_single[p].end());
    }
    Lh.cn_z[0] = 0;
    for (int z = 0; z < 7; ++z) Lh.cn_z[z + 1] = Lh.cn_z[z] + static_cast<int>(cnear[z].size());
    Lh.cn_pairs = static_cast<int>(cnear_pair.size());
    Lh.cn_off = static_cast<int>(g->lists.size());
    for (int z = 0; z < 7; ++z) g->lists.insert(g->lists.end(), cnear[z].begin(), cnear[z].end());
    g->lists.insert(g->lists.end(), cnear_pair.begin(), cnear_pair.end());
    Lh.mf_z[0] = 0;
    for (int z = 0; z < 7; ++z) Lh.mf_z[z + 1] = Lh.mf_z[z] + static_cast<int>(mfar[0][z].size());
    Lh.mf_pairs = static_cast<int>(mfar_pair[0].size());
    Lh.mf_singles = static_cast<int>(mfar_single[0].size());
    Lh.mf_stride = Lh.mf_z[7] + Lh.mf_pairs + Lh.mf_singles;
    Lh.mf_off = static_cast<int>(g->lists.size());
    for (int p = 0; p < 8; ++p) {
        for (int z = 0; z < 7; ++z) g->lists.insert(g->lists.end(), mfar[p][z].begin(), mfar[p][z].end());
        g->lists.insert(g->lists.end(), mfar_pair[p].begin(), mfar_pair[p].end());
        g->lists.insert(g->lists.end(), mfar_single[p].begin(), mfar_single[p].end());
    }
    Lh.mr_z[0] = 0;
    for (int z = 0; z < 7; ++z) Lh.mr_z[z + 1] = Lh.mr_z[z] + static_cast<int>(mroot[z].size());
    Lh.mr_pairs = static_cast<int>(mroot_pair.size());
    Lh.mr_off = static_cast<int>(g->lists.size());
    for (int z = 0; z < 7; ++z) g->lists.insert(g->lists.end(), mroot[z].begin(), mroot[z].end());
    g->lists.insert(g->lists.end(), mroot_pair.begin(), mroot_pair.end());
    // a leaf target's multipole sources paired along one axis A: per A and
    // parity, the offsets o with o_A > 0 whose reflection along A is in the
    // same far list, then every other offset as a single
    for (int A = 0; A < 3; ++A) {
        Lh.ap_off[A] = static_cast<int>(g->lists.size());
        for (int p = 0; p < 8; ++p) {
            std::set<int> in;
            for (auto& o : far_offs[p]) in.insert(key(o[0], o[1], o[2]));
            std::vector<int> pp, ss;
            for (auto& o : far_offs[p]) {
                std::array<int, 3> r = o;
                r[A] = -r[A];
                if (o[A] != 0 && in.count(key(r[0], r[1], r[2]))) {
                    if (o[A] > 0) pp.push_back(pack_offset(o[0], o[1], o[2]));
                } else {
                    ss.push_back(pack_offset(o[0], o[1], o[2]));
                }
            }
            if (2 * pp.size() + ss.size() != far_offs[p].size())
                return fail(OT_EINVAL, "internal: axis-pair stencils do not cover the offsets");
            if (p == 0) {
                Lh.ap_pairs[A] = static_cast<int>(pp.size());
                Lh.ap_len[A] = static_cast<int>(pp.size() + ss.size());
            } else if (Lh.ap_pairs[A] != static_cast<int>(pp.size()) ||
                       Lh.ap_len[A] != static_cast<int>(pp.size() + ss.size())) {
                return fail(OT_EINVAL, "internal: parity axis-pair stencils differ in shape");
            }
            g->lists.insert(g->lists.end(), pp.begin(), pp.end());
            g->lists.insert(g->lists.end(), ss.begin(), ss.end());
        }
    }
    {
        // every far and near offset exactly once
        long long nf = 2LL * Lh.cf_pairs + Lh.cf_singles, nn = 2LL * Lh.cn_pairs;
        for (int k = 0; k < Lh.cf_z[7]; ++k) nf += __builtin_popcount(static_cast<unsigned>(g->lists[Lh.cf_off + k]) >> 24);
        for (int k = 0; k < Lh.cn_z[7]; ++k) nn += __builtin_popcount(static_cast<unsigned>(g->lists[Lh.cn_off + k]) >> 24);
        long long mf = 2LL * Lh.mf_pairs + Lh.mf_singles, mr = 2LL * Lh.mr_pairs;
        for (int k = 0; k < Lh.mf_z[7]; ++k) mf += __builtin_popcount(static_cast<unsigned>(g->lists[Lh.mf_off + k]) >> 24);
        for (int k = 0; k < Lh.mr_z[7]; ++k) mr += __builtin_popcount(static_cast<unsigned>(g->lists[Lh.mr_off + k]) >> 24);
        if (nf != g->far_offsets || nn != 2LL * g->near_len || mf != g->far_offsets || mr != 2LL * g->root_len)
            return fail(OT_EINVAL, "internal: class stencils do not cover the offsets");
    }

    // --- derivative table ----------------------------------------------------
    std::vector<double> Dt(static_cast<size_t>(NOFF) * DROW, 0.0);
    for (int oz = -7; oz <= 7; ++oz)
        for (int oy = -7; oy <= 7; ++oy)
            for (int ox = -7; ox <= 7; ++ox) {
                if (ox == 0 && oy == 0 && oz == 0) continue;
                const double R[3] = {-1.0 * ox, -1.0 * oy, -1.0 * oz};
                derivative_row(R, &Dt[static_cast<size_t>((ox + 7) + 15 * (oy + 7) + 225 * (oz + 7)) * DROW]);
            }

    // --- neighbour tables, virtual descendants --------------------------------
    g->nbr.assign(static_cast<size_t>(n) * 27, int2{-1, K_NONE});
    g->ninfo.resize(n);
    std::map<std::tuple<int, long, long, long>, int> vindex;   // (level, q) -> virtual id
    struct VNode { int level; long q[3]; int leaf; int d; int2 e; };
    std::vector<VNode> vnodes;
    // region of each neighbour position: a node (its index) or a virtual
    // block (n + its virtual id); -1 outside the domain / without data
    std::vector<int> nreg(static_cast<size_t>(n) * 27, -1);
    for (int i = 0; i < n; ++i) {
        const int l = desc->level[i];
        g->ninfo[i] = l | (g->is_leaf[i] << 8);
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const long q[3] = {desc->coord[3 * i] + dx, desc->coord[3 * i + 1] + dy,
                                       desc->coord[3 * i + 2] + dz};
                    int2 e;
                    int vd;
                    long vq[3];
                    ot_status st = B.entry(l, q, false, &e, &vd, vq);
                    if (st != OT_OK) return st;
                    const size_t jj = static_cast<size_t>(i) * 27 + (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
                    g->nbr[jj] = e;
                    if ((e.y & 3) == K_VIRT) {
                        auto key = std::make_tuple(l, q[0], q[1], q[2]);
                        if (!vindex.count(key)) {
                            vindex[key] = static_cast<int>(vnodes.size());
                            vnodes.push_back(VNode{l, {q[0], q[1], q[2]}, e.x, vd, e});
                        }
                        nreg[jj] = n + vindex[key];
                    } else if ((e.y & 3) != K_NONE) {
                        nreg[jj] = e.x;
                    }
                }
    }
    g->nvirt = static_cast<int>(vnodes.size());
    g->vnbr.assign(static_cast<size_t>(std::max(g->nvirt, 1)) * 27, int2{-1, K_NONE});
    g->vinfo.assign(std::max(g->nvirt, 1), 0);
    std::vector<int> vcoord(static_cast<size_t>(std::max(g->nvirt, 1)) * 3, 0);
    for (int v = 0; v < g->nvirt; ++v)
        for (int a = 0; a < 3; ++a) vcoord[3 * v + a] = static_cast<int>(vnodes[v].q[a]);
    std::vector<std::pair<int, int>> vrows;   // (P*512 + pcell, entry)
    for (int v = 0; v < g->nvirt; ++v) {
        const VNode& V = vnodes[v];
        g->vinfo[v] = V.level;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const long q[3] = {V.q[0] + dx, V.q[1] + dy, V.q[2] + dz};
                    int2 e;
                    int vd;
                    long vq[3];
                    ot_status st = B.entry(V.level, q, true, &e, &vd, vq);
                    if (st != OT_OK) return st;
                    g->vnbr[static_cast<size_t>(v) * 27 + (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)] = e;
                }
        for (int sc = 0; sc < NCELL; ++sc) {
            const int s3[3] = {sc & 7, (sc >> 3) & 7, sc >> 6};
            int pc[3];
            for (int a = 0; a < 3; ++a) {
                const long ov = 8 * (V.q[a] - ((V.q[a] >> V.d) << V.d));
                pc[a] = static_cast<int>((ov + s3[a]) >> V.d);
            }
            const int row = V.leaf * NCELL + pc[0] + 8 * pc[1] + 64 * pc[2];
            vrows.emplace_back(row, (v * NCELL + sc) | (V.d << 28));
        }
    }
    if (static_cast<long long>(g->nvirt) * NCELL >= (1LL << 28))
        return fail(OT_EINVAL, "too many virtual descendant sub-grids (%d)", g->nvirt);
    std::stable_sort(vrows.begin(), vrows.end(),
                     [](const std::pair<int, int>& a, const std::pair<int, int>& b) { return a.first < b.first; });
    std::vector<int> vmap;
    {
        std::vector<int> heads, ptr, ent;
        for (size_t k = 0; k < vrows.size(); ++k) {
            if (k == 0 || vrows[k].first != vrows[k - 1].first) {
                heads.push_back(vrows[k].first);
                ptr.push_back(static_cast<int>(k));
            }
            ent.push_back(vrows[k].second);
        }
        ptr.push_back(static_cast<int>(vrows.size()));
        g->vmap_rows = static_cast<int>(heads.size());
        vmap = heads;
        vmap.insert(vmap.end(), ptr.begin(), ptr.end());
        vmap.insert(vmap.end(), ent.begin(), ent.end());
    }

    // --- prebuilt x butterflies ----------------------------------------------
    // A class's first transform stage along x at a position q -- the sum and
    // the difference of the values a cells to either side, a = 1..7 -- is
    // built per call for every cell of every region that can hold such a q:
    // the same-level blocks of the 27-neighbourhoods of the nodes that read
    // it.  A region is a node or a virtual block (a same-level block covered
    // by a coarser leaf).  Two slot spaces:
    //   M: the regions around leaf nodes -- the point masses of the leaf
    //      targets' classes (leaf cells and virtual descendants; 0 in
    //      refined blocks) and the point-mass scatter's deferred x stage;
    //   X: the regions around non-leaf nodes -- the reduced moments of
    //      non-leaf cells (0 elsewhere) for the non-leaf targets' classes,
    //      and the reduced L-bar of real cells for the multipole gather.
    // nslot[i][j] is the slot of node i's neighbour region j in the space of
    // node i's kind (M for a leaf, X otherwise); every slot carries its
    // region's 27 neighbour entries (snb) for the builder kernels.
    {
        const int nregions = n + g->nvirt;
        std::vector<int> slotM(nregions, -1), slotX(nregions, -1), regM, regX;
        // space M numbers first the regions in the z columns of the leaves
        // (neighbours j = 4, 13, 22: dx = dy = 0): the (x, y) table is read
        // only at centres t + (0, 0, +-c), so it covers slots [0, n_slotXY)
        for (int i = 0; i < n; ++i) {
            if (!g->is_leaf[i]) continue;
            for (int j = 4; j < 27; j += 9) {
                const int r = nreg[static_cast<size_t>(i) * 27 + j];
                if (r >= 0 && slotM[r] < 0) {
                    slotM[r] = static_cast<int>(regM.size());
                    regM.push_back(r);
                }
            }
        }
        g->n_slotXY = static_cast<int>(regM.size());
        // space X likewise numbers first the regions in the z columns of the
        // non-leaf nodes (the moments' (x, y) table, read at t + (0, 0, +-c)),
        // then the rest of their yz planes (neighbours with dx = 0): the x
        // tables of reduced moments and L-bar are read only at t + (0, +-b, +-c)
        for (int i = 0; i < n; ++i) {
            if (g->is_leaf[i]) continue;
            for (int j = 4; j < 27; j += 9) {
                const int r = nreg[static_cast<size_t>(i) * 27 + j];
                if (r >= 0 && slotX[r] < 0) {
                    slotX[r] = static_cast<int>(regX.size());
                    regX.push_back(r);
                }
            }
        }
        g->n_slotXz = static_cast<int>(regX.size());
        for (int i = 0; i < n; ++i) {
            if (g->is_leaf[i]) continue;
            for (int j = 1; j < 27; j += 3) {
                const int r = nreg[static_cast<size_t>(i) * 27 + j];
                if (r >= 0 && slotX[r] < 0) {
                    slotX[r] = static_cast<int>(regX.size());
                    regX.push_back(r);
                }
            }
        }
        g->n_slotXyz = static_cast<int>(regX.size());
        for (int i = 0; i < n; ++i) {
            std::vector<int>& slot = g->is_leaf[i] ? slotM : slotX;
            std::vector<int>& reg = g->is_leaf[i] ? regM : regX;
            for (int j = 0; j < 27; ++j) {
                const int r = nreg[static_cast<size_t>(i) * 27 + j];
                if (r >= 0 && slot[r] < 0) {
                    slot[r] = static_cast<int>(reg.size());
                    reg.push_back(r);
                }
            }
        }
        // the 27 neighbour entries of a region (a node's own; a virtual
        // block's as the forward sees them); false if a position needs a
        // virtual descendant deeper than the limit
        auto region_row = [&](int r, int2* row) -> bool {
            if (r < n) {
                std::memcpy(row, &g->nbr[static_cast<size_t>(r) * 27], 27 * sizeof(int2));
                return true;
            }
            const VNode& V = vnodes[r - n];
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const long q[3] = {V.q[0] + dx, V.q[1] + dy, V.q[2] + dz};
                        int vd;
                        long vq[3];
                        int2 e;
                        if (B.entry(V.level, q, false, &e, &vd, vq) != OT_OK) {
                            g_last_error.clear();
                            return false;
                        }
                        row[(dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)] = e;
                    }
            return true;
        };
        std::vector<char> okM(regM.size(), 1), okX(regX.size(), 1);
        g->snbM.assign(regM.size() * 27, int2{-1, K_NONE});
        g->snbX.assign(regX.size() * 27, int2{-1, K_NONE});
        for (size_t k = 0; k < regM.size(); ++k) okM[k] = region_row(regM[k], &g->snbM[k * 27]);
        for (size_t k = 0; k < regX.size(); ++k) okX[k] = region_row(regX[k], &g->snbX[k * 27]);
        g->n_slotM = static_cast<int>(regM.size());
        g->n_slotX = static_cast<int>(regX.size());
        g->nslot.assign(static_cast<size_t>(n) * 27, -1);
        for (int i = 0; i < n; ++i) {
            const bool leaf = g->is_leaf[i];
            bool ok = true;
            for (int j = 0; j < 27; ++j) {
                const int r = nreg[static_cast<size_t>(i) * 27 + j];
                if (r < 0) continue;
                const int sl = leaf ? slotM[r] : slotX[r];
                g->nslot[static_cast<size_t>(i) * 27 + j] = sl;
                ok = ok && (leaf ? okM[sl] : okX[sl]);
            }
            // every class of the node may read its first stage from the
            // tables (multipole gather included for non-leaf sources)
            if (ok) g->ninfo[i] |= leaf ? NI_XMASS : (NI_XMULTI | NI_XGATHER);
        }
        // the scatter's deferred x stage: each point-mass region of space M
        // (leaf node or virtual block) collects, per cell, from the centres
        // a cells to either side in x -- in the regions at x-1, x, x+1
        g->mem_ent.clear();
        g->mem_xs.clear();
        for (size_t k = 0; k < regM.size(); ++k) {
            const int r = regM[k];
            int2 self;
            long q[3];
            int lvl;
            if (r < n) {
                if (!g->is_leaf[r]) continue;
                self = int2{r, K_LEAF};
                lvl = desc->level[r];
                for (int a = 0; a < 3; ++a) q[a] = desc->coord[3 * r + a];
            } else {
                self = vnodes[r - n].e;
                lvl = vnodes[r - n].level;
                for (int a = 0; a < 3; ++a) q[a] = vnodes[r - n].q[a];
            }
            int xs[3] = {-1, -1, -1};
            for (int dx = -1; dx <= 1; ++dx) {
                const long qq[3] = {q[0] + dx, q[1], q[2]};
                int rr = B.find(lvl, qq[0], qq[1], qq[2]);
                if (rr < 0) {
                    auto it = vindex.find(std::make_tuple(lvl, qq[0], qq[1], qq[2]));
                    if (it != vindex.end()) rr = n + it->second;
                }
                if (rr >= 0 && slotM[rr] >= 0 && okM[slotM[rr]]) xs[dx + 1] = slotM[rr];
            }
            g->mem_ent.push_back(self);
            g->mem_xs.insert(g->mem_xs.end(), xs, xs + 3);
        }
        // the moments' (x, y) table is built from the x table: for each of
        // its slots (the z columns of the non-leaf nodes) the X slots of the
        // regions at y-1, y, y+1, all in the yz planes the x table covers
        g->xym_ys.assign(static_cast<size_t>(std::max(g->n_slotXz, 1)) * 3, -1);
        for (int k = 0; k < g->n_slotXz; ++k) {
            const int r = regX[k];
            long q[3];
            int lvl;
            if (r < n) {
                lvl = desc->level[r];
                for (int a = 0; a < 3; ++a) q[a] = desc->coord[3 * r + a];
            } else {
                lvl = vnodes[r - n].level;
                for (int a = 0; a < 3; ++a) q[a] = vnodes[r - n].q[a];
            }
            for (int dy = -1; dy <= 1; ++dy) {
                int rr = B.find(lvl, q[0], q[1] + dy, q[2]);
                if (rr < 0) {
                    auto it = vindex.find(std::make_tuple(lvl, q[0], q[1] + dy, q[2]));
                    if (it != vindex.end()) rr = n + it->second;
                }
                if (rr >= 0 && slotX[rr] >= 0 && slotX[rr] < g->n_slotXyz)
                    g->xym_ys[static_cast<size_t>(k) * 3 + dy + 1] = slotX[rr];
            }
            if (g->xym_ys[static_cast<size_t>(k) * 3 + 1] != k)
                return fail(OT_EINVAL, "internal: a z-column slot is not its own y neighbour");
        }
    }
    for (int i = 0; i < n; ++i) {
        const int2* nb27 = &g->nbr[static_cast<size_t>(i) * 27];
        const int sl = slab_axis(nb27, g->is_leaf[i]);
        g->ninfo[i] |= sl << NI_SLAB_SHIFT;
        g->ninfo[i] |= pair_axis(nb27, sl, g->is_leaf[i]) << NI_APAIR_SHIFT;
    }
    // the (x, y) table of the masses takes 0.8 MB per slot: built up to 16 GiB
    g->use_xy = static_cast<double>(g->n_slotXY) * 49 * 4 * NCELL * sizeof(double) <= 16.0 * (1u << 30);
    // the moments' (x, y) table takes 12.8 MB per slot: built up to 48 GiB
    g->use_xym = static_cast<double>(g->n_slotXz) * 49 * 64 * NCELL * sizeof(double) <= 48.0 * (1u << 30);

    // --- exact pair counts, FLOPs and per-item costs ------------------------
    // For each (parity, half) warp pattern and list entry: which of the 27
    // neighbours the warp's 32 cells reach (both sides of a paired entry), and
    // per neighbour how many (cell, source) pairs land there, split by
    // paired / single entries.  Segments: 0 far, 1 near, 2 root.
    const int seg_len[3] = {g->far_len, g->near_len, g->root_len};
    // [slab][pattern][segment]: the masks for each of the three lane layouts
    std::vector<uint32_t> mask[3][16][3];
    std::vector<uint32_t> maskside[3][16][3][2];   // the neighbours each member of an entry reaches
    std::vector<uint8_t> pflag[16][3];
    long long cnt[3][2][27];   // [segment][paired][neighbour]: pairs over all 512 cells
    std::memset(cnt, 0, sizeof(cnt));
    for (int ph = 0; ph < 16; ++ph) {
        const int par = ph >> 1, half = ph & 1;
        for (int sg = 0; sg < 3; ++sg) {
            const int* lst = (sg == 0) ? &g->lists[par * g->far_len]
                           : (sg == 1) ? &g->lists[8 * g->far_len] : &g->lists[8 * g->far_len + g->near_len];
            for (int sl = 0; sl < 3; ++sl) {
                mask[sl][ph][sg].resize(seg_len[sg]);
                maskside[sl][ph][sg][0].resize(seg_len[sg]);
                maskside[sl][ph][sg][1].resize(seg_len[sg]);
            }
            pflag[ph][sg].resize(seg_len[sg]);
            for (int k = 0; k < seg_len[sg]; ++k) {
                const int po = lst[k];
                const int paired = (po >> 24) & 1;
                const int ox = (po & 0xff) - 8, oy = ((po >> 8) & 0xff) - 8, oz = ((po >> 16) & 0xff) - 8;
                for (int sl = 0; sl < 3; ++sl) {
                    uint32_t m = 0, ms[2] = {0, 0};
                    for (int lane = 0; lane < 32; ++lane) {
                        int tx, ty, tz;
                        lane_cell_host(lane, par, half, sl, tx, ty, tz);
                        for (int side = 0; side <= paired; ++side) {
                            const int sgn = side ? -1 : 1;
                            const int nb = ((tx + sgn * ox + 8) >> 3) + 3 * ((ty + sgn * oy + 8) >> 3) +
                                           9 * ((tz + sgn * oz + 8) >> 3);
                            m |= 1u << nb;
                            ms[side] |= 1u << nb;
                            if (sl == 0) cnt[sg][paired][nb]++;
                        }
                    }
                    mask[sl][ph][sg][k] = m;
                    maskside[sl][ph][sg][0][k] = ms[0];
                    maskside[sl][ph][sg][1][k] = ms[1];
                }
                pflag[ph][sg][k] = static_cast<uint8_t>(paired);
            }
        }
    }
    // The axis-pair lists of a leaf target's multipole sources: per axis A,
    // lane layout and warp pattern, the neighbours each member of an entry
    // reaches; per A the pairs landing in each neighbour over all 512 cells,
    // by paired / single entries.
    std::vector<uint32_t> amask[3][3][16][2];   // [A][slab][pattern][member]
    long long acnt[3][2][27];                   // [A][paired][neighbour]
    std::memset(acnt, 0, sizeof(acnt));
    for (int A = 0; A < 3; ++A)
        for (int ph = 0; ph < 16; ++ph) {
            const int par = ph >> 1, half = ph & 1;
            const int* lst = &g->lists[g->Lh.ap_off[A] + par * g->Lh.ap_len[A]];
            for (int sl = 0; sl < 3; ++sl)
                for (int side = 0; side < 2; ++side) amask[A][sl][ph][side].assign(g->Lh.ap_len[A], 0u);
            for (int k = 0; k < g->Lh.ap_len[A]; ++k) {
                const int po = lst[k];
                const int paired = k < g->Lh.ap_pairs[A] ? 1 : 0;
                int o[3] = {(po & 0xff) - 8, ((po >> 8) & 0xff) - 8, ((po >> 16) & 0xff) - 8};
                for (int sl = 0; sl < 3; ++sl)
                    for (int lane = 0; lane < 32; ++lane) {
                        int t[3];
                        lane_cell_host(lane, par, half, sl, t[0], t[1], t[2]);
                        for (int side = 0; side <= paired; ++side) {
                            int q[3] = {t[0] + o[0], t[1] + o[1], t[2] + o[2]};
                            if (side) q[A] = t[A] - o[A];
                            const int nb = ((q[0] + 8) >> 3) + 3 * ((q[1] + 8) >> 3) + 9 * ((q[2] + 8) >> 3);
                            amask[A][sl][ph][side][k] |= 1u << nb;
                            if (sl == 0) acnt[A][paired][nb]++;
                        }
                    }
            }
        }
    // The class lists of leaf targets (point masses): per warp pattern and
    // entry the neighbours its members reach; per entry its FP64 instructions
    // per lane (forward, scatter adjoint), members and FLOPs; per neighbour
    // the FLOPs of the pairs landing there over all 512 cells, an entry's
    // FLOPs shared equally by its members.
    // Class segments: 0 point masses, far (per parity); 1 point masses,
    // near; 2 multipole sources with the angular term, far (per parity);
    // 3 the same, root.
    const int cseg_len[4] = {g->Lh.cf_stride, g->Lh.cn_z[7] + g->Lh.cn_pairs, g->Lh.mf_stride,
                             g->Lh.mr_z[7] + g->Lh.mr_pairs};
    std::vector<uint32_t> cmask[3][16][4];
    std::vector<int> ccost_f[4], ccost_s[4], cmem[4];
    double cfl_f[4][27], cfl_s[4][27], cop_f[4][27], cop_s[4][27];   // FLOPs; FP64 instructions
    // the forward's figures for a node whose x-complete classes read the
    // prebuilt x butterflies (the x stage's adds gone)
    double cfl_fx[4][27], cop_fx[4][27], cfl_sx[4][27], cop_sx[4][27];
    std::vector<int> ccost_fx[4], ccost_sx[4];
    std::memset(cfl_f, 0, sizeof(cfl_f));
    std::memset(cfl_s, 0, sizeof(cfl_s));
    std::memset(cop_f, 0, sizeof(cop_f));
    std::memset(cop_s, 0, sizeof(cop_s));
    std::memset(cfl_fx, 0, sizeof(cfl_fx));
    std::memset(cop_fx, 0, sizeof(cop_fx));
    std::memset(cfl_sx, 0, sizeof(cfl_sx));
    std::memset(cop_sx, 0, sizeof(cop_sx));
    for (int cg = 0; cg < 4; ++cg) {
        const int nz = cg == 0 ? g->Lh.cf_z[7] : cg == 1 ? g->Lh.cn_z[7] : cg == 2 ? g->Lh.mf_z[7] : g->Lh.mr_z[7];
        const int npair = cg == 0 ? g->Lh.cf_pairs : cg == 1 ? g->Lh.cn_pairs : cg == 2 ? g->Lh.mf_pairs : g->Lh.mr_pairs;
        const bool multi = cg >= 2;
        ccost_f[cg].resize(cseg_len[cg]);
        ccost_fx[cg].resize(cseg_len[cg]);
        ccost_sx[cg].resize(cseg_len[cg]);
        ccost_s[cg].resize(cseg_len[cg]);
        cmem[cg].resize(cseg_len[cg]);
        const int* zx = cg == 0 ? g->Lh.cf_x : cg == 1 ? g->Lh.cn_x : cg == 2 ? g->Lh.mf_x : g->Lh.mr_x;
        const int* zz = cg == 0 ? g->Lh.cf_z : cg == 1 ? g->Lh.cn_z : cg == 2 ? g->Lh.mf_z : g->Lh.mr_z;
        const int* zxy = cg == 0 ? g->Lh.cf_xy : cg == 1 ? g->Lh.cn_xy : cg == 2 ? g->Lh.mf_xy : g->Lh.mr_xy;
        for (int ph = 0; ph < 16; ++ph) {
            const int par = ph >> 1, half = ph & 1;
            const int off = cg == 0 ? g->Lh.cf_off + par * g->Lh.cf_stride : cg == 1 ? g->Lh.cn_off
                          : cg == 2 ? g->Lh.mf_off + par * g->Lh.mf_stride : g->Lh.mr_off;
            const int* lst = &g->lists[off];
            for (int sl = 0; sl < 3; ++sl) cmask[sl][ph][cg].resize(cseg_len[cg]);
            for (int k = 0; k < cseg_len[cg]; ++k) {
                const int e = lst[k];
                std::vector<std::array<int, 3>> mem;
                int cf, cs, fl_f, fl_s, cfx, fl_fx, csx, fl_sx;
                if (k < nz) {
                    const int a = e & 0xff, b = (e >> 8) & 0xff, cc = (e >> 16) & 0xff;
                    const int Z = (a == 0 ? 1 : 0) | (b == 0 ? 2 : 0) | (cc == 0 ? 4 : 0);
                    for (int t = 0; t < 8; ++t)
                        if ((static_cast<unsigned>(e) >> 24 >> t) & 1u)
                            mem.push_back({t & 1 ? -a : a, t & 2 ? -b : b, t & 4 ? -cc : cc});
                    const bool xe = !(Z & 1) && k - zz[Z] < zx[Z];     // x-complete head of its group
                    if (multi) {   // forward with the angular term; the adjoint's gather
                        cf = OT_MCLASS_ADDS[1][Z] + OT_MCLASS_FMAS[1][Z];
                        cs = OT_MCLASS_ADJ_ADDS[Z] + OT_MCLASS_ADJ_FMAS[Z];
                        fl_f = OT_MCLASS_ADDS[1][Z] + 2 * OT_MCLASS_FMAS[1][Z];
                        fl_s = OT_MCLASS_ADJ_ADDS[Z] + 2 * OT_MCLASS_ADJ_FMAS[Z];
                        // the x stage prebuilt (x-complete head); the x and y
                        // stages (its xy-complete head, a and b > 0)
                        const bool xye = xe && !(Z & 2) && k - zz[Z] < zxy[Z] && g->use_xym;
                        const int madds = xye ? OT_MCLASS_XY_ADDS[1][Z] : xe ? OT_MCLASS_X_ADDS[1][Z]
                                                                              : OT_MCLASS_ADDS[1][Z];
                        cfx = madds + OT_MCLASS_FMAS[1][Z];
                        fl_fx = madds + 2 * OT_MCLASS_FMAS[1][Z];
                        csx = xe ? OT_MCLASS_ADJ_X_ADDS[Z] + OT_MCLASS_ADJ_FMAS[Z] : cs;
                        fl_sx = xe ? OT_MCLASS_ADJ_X_ADDS[Z] + 2 * OT_MCLASS_ADJ_FMAS[Z] : fl_s;
                    } else {
                        cf = cs = class_adds(Z) + class_fmas(Z);
                        fl_f = fl_s = class_adds(Z) + 2 * class_fmas(Z);
                        // without the x stage: (d - 1) 2^d adds; without the x
                        // and y stages (xy-complete head, a and b > 0): (d - 2) 2^d
                        const int d = 3 - __builtin_popcount(Z);
                        const bool xye = xe && !(Z & 2) && k - zz[Z] < zxy[Z] && g->use_xy;
                        const int xadds = xye ? class_adds(Z) - 2 * (1 << d) : xe ? class_adds(Z) - (1 << d)
                                                                                  : class_adds(Z);
                        cfx = xadds + class_fmas(Z);
                        fl_fx = xadds + 2 * class_fmas(Z);
                        // the scatter defers its x stage only
                        const int sadds = xe ? class_adds(Z) - (1 << d) : class_adds(Z);
                        csx = sadds + class_fmas(Z);
                        fl_sx = sadds + 2 * class_fmas(Z);
                    }
                } else {
                    const int ox = (e & 0xff) - 8, oy = ((e >> 8) & 0xff) - 8, oz = ((e >> 16) & 0xff) - 8;
                    mem.push_back({ox, oy, oz});
                    if (k < nz + npair) {
                        mem.push_back({-ox, -oy, -oz});
                        cf = multi ? 132 : 18;
                        cs = multi ? 102 : 18;
                        fl_f = multi ? 232 : 34;
                        fl_s = multi ? 172 : 34;
                    } else {
                        cf = multi ? 100 : 16;
                        cs = multi ? 70 : 17;
                        fl_f = multi ? 200 : 32;
                        fl_s = multi ? 140 : 32;
                    }
                    cfx = cf;
                    fl_fx = fl_f;
                    csx = cs;
                    fl_sx = fl_s;
                }
                ccost_f[cg][k] = cf;
                ccost_fx[cg][k] = cfx;
                ccost_sx[cg][k] = csx;
                ccost_s[cg][k] = cs;
                cmem[cg][k] = static_cast<int>(mem.size());
                for (int sl = 1; sl < 3; ++sl) {
                    uint32_t ml = 0;
                    for (int lane = 0; lane < 32; ++lane) {
                        int tx, ty, tz;
                        lane_cell_host(lane, par, half, sl, tx, ty, tz);
                        for (auto& o : mem)
                            ml |= 1u << (((tx + o[0] + 8) >> 3) + 3 * ((ty + o[1] + 8) >> 3) + 9 * ((tz + o[2] + 8) >> 3));
                    }
                    cmask[sl][ph][cg][k] = ml;
                }
                uint32_t m = 0;
                for (int lane = 0; lane < 32; ++lane) {
                    int tx, ty, tz;
                    lane_cell_host(lane, par, half, 0, tx, ty, tz);
                    for (auto& o : mem) {
                        const int nb = ((tx + o[0] + 8) >> 3) + 3 * ((ty + o[1] + 8) >> 3) + 9 * ((tz + o[2] + 8) >> 3);
                        m |= 1u << nb;
                        cfl_f[cg][nb] += static_cast<double>(fl_f) / mem.size();
                        cfl_s[cg][nb] += static_cast<double>(fl_s) / mem.size();
                        cop_f[cg][nb] += static_cast<double>(cf) / mem.size();
                        cop_s[cg][nb] += static_cast<double>(cs) / mem.size();
                        cfl_fx[cg][nb] += static_cast<double>(fl_fx) / mem.size();
                        cop_fx[cg][nb] += static_cast<double>(cfx) / mem.size();
                        cfl_sx[cg][nb] += static_cast<double>(fl_sx) / mem.size();
                        cop_sx[cg][nb] += static_cast<double>(csx) / mem.size();
                    }
                }
                cmask[0][ph][cg][k] = m;
            }
        }
    }
    // algorithmic FLOPs per in-domain pair (2 per FMA, 1 per add):
    //   point mass 32, or 17 in a paired entry (16 FMA + 2 adds per two pairs);
    //   point masses at leaf targets (level > 0) by class: class_adds +
    //   2 class_fmas per class entry, shared by its members;
    //   multipole 140 (200 with the angular term), or 86 (116) paired;
    //   multipole sources at non-leaf targets by class: OT_MCLASS_ADDS +
    //   2 OT_MCLASS_FMAS (angular) per class entry, shared by its members;
    //   the adjoint's multipole gather by class likewise (OT_MCLASS_ADJ_*);
    //   adjoint: point mass 32, multipole 140, or 86 paired.
    // FP64 instructions per lane and active entry (empty lanes included):
    //   forward point mass 16 | 18 paired; multipole 70 (+30) | 102 (+30);
    //   adjoint point mass 16 | 32 paired; multipole 70 | 102 paired.
    //   refined near entries (a leaf target's near source in a refined
    //   sub-grid): 8 point-mass contractions from the virtual-child table,
    //   counted as one interaction (one stencil pair).
    long long pairs_multi = 0, pairs_mono = 0, pairs_virt = 0, pairs_ang = 0, pairs_ref = 0, lanes = 0;
    long long padded = 0;   // pairs the lanes run, out-of-domain sources included
    long long flops_fwd = 0, flops_adj = 0, ops_fwd = 0, ops_adj = 0;
    long long flops_adj_scat = 0, ops_adj_scat = 0, count_single_mono = 0;
    long long flops_adj_multi = 0, ops_adj_multi = 0;
    long long flops_fwd_com = 0, flops_adj_com = 0;   // explicit centres (see ot_interactions_com)
    // algorithmic FP64 instructions (one per FMA or add) of the in-domain
    // pairs, shared per entry like the FLOPs: the FP64 pipe's work
    double alg_fwd = 0.0, alg_adj_scat = 0.0, alg_adj_multi = 0.0, alg_adj_det = 0.0;
    double alg_fwd_multi = 0.0;        // the multipole pass alone (pass 1)
    long long ops_fwd_multi = 0;
    std::vector<std::pair<long long, int>> fwd[4];
    std::vector<int> node_order_items;
    std::vector<long long> node_cost(n, 0);   // largest item of the node (both passes)
    long long total_cost = 0;
    g->node_item_start.assign(n + 1, 0);
    for (int i = 0; i < n; ++i) {
        uint32_t mm = 0, mo = 0, mv = 0;
        for (int j = 0; j < 27; ++j) {
            const int k = g->nbr[static_cast<size_t>(i) * 27 + j].y & 3;
            if (k == K_MULTI) mm |= 1u << j;
            if (k == K_LEAF || k == K_VIRT) mo |= 1u << j;
            if (k == K_VIRT) mv |= 1u << j;
        }
        const bool leaf = g->is_leaf[i];
        const int s1 = (desc->level[i] == 0) ? 2 : 0;
        const bool by_class = leaf && desc->level[i] > 0;   // point masses by reflection class
        // the node's classes read the prebuilt x butterflies
        const bool xnode = (g->ninfo[i] & (leaf ? NI_XMASS : NI_XMULTI)) != 0;
        const auto& CFL = xnode ? cfl_fx : cfl_f;
        const auto& COP = xnode ? cop_fx : cop_f;
        const std::vector<int>* CCF = xnode ? ccost_fx : ccost_f;
        for (int j = 0; j < 27; ++j) {
            const long long cpf = cnt[s1][1][j], csf = cnt[s1][0][j];                 // far / root
            const long long cpn = leaf ? cnt[1][1][j] : 0, csn = leaf ? cnt[1][0][j] : 0;   // near
            const long long cp = cpf + cpn, cs = csf + csn;
            if (mm >> j & 1u) {
                pairs_multi += cpf + csf;
                if (!leaf) {
                    pairs_ang += cpf + csf;
                    flops_fwd += std::llround(CFL[desc->level[i] == 0 ? 3 : 2][j]);
                    alg_fwd += COP[desc->level[i] == 0 ? 3 : 2][j];
                    alg_fwd_multi += COP[desc->level[i] == 0 ? 3 : 2][j];
                } else if (desc->level[i] > 0) {
                    // a leaf target's multipole sources by the node's axis-pair
                    // list: 70 FMAs + 32 adds per two pairs, 70 FMAs single
                    const int A = (g->ninfo[i] >> NI_APAIR_SHIFT) & 3;
                    const long long ap = acnt[A][1][j], as = acnt[A][0][j];
                    if (ap + as != cpf + csf) return fail(OT_EINVAL, "internal: axis-pair counts differ");
                    flops_fwd += 86 * ap + 140 * as;
                    alg_fwd += 51.0 * ap + 70.0 * as;
                    alg_fwd_multi += 51.0 * ap + 70.0 * as;
                } else {
                    flops_fwd += 86 * cpf + 140 * csf;
                    alg_fwd += 51.0 * cpf + 70.0 * csf;
                    alg_fwd_multi += 51.0 * cpf + 70.0 * csf;
                }
                // explicit centres: every multipole pair evaluates its derivatives
                flops_fwd_com += (cpf + csf) * (leaf ? deriv_flops(19) + 140 : deriv_flops(31) + 200);
                flops_adj_com += (cpf + csf) * (deriv_flops(19) + 140);
                // near sources in the refined sub-grid: its cells' children
                pairs_ref += cpn + csn;
                pairs_mono += cpn + csn;
                flops_fwd += 8 * (17 * cpn + 32 * csn);
                alg_fwd += 8 * (9.0 * cpn + 16.0 * csn);
                flops_fwd_com += 8 * (17 * cpn + 32 * csn);
                flops_adj_scat += 8 * (16 * cpn + 32 * csn);
                alg_adj_scat += 8 * (9.0 * cpn + 16.0 * csn);
                flops_adj_com += 8 * (16 * cpn + 32 * csn);
            }
            if (mo >> j & 1u) {
                pairs_mono += cp + cs;
                if (by_class) {
                    flops_fwd += std::llround(CFL[0][j] + CFL[1][j]);
                    alg_fwd += COP[0][j] + COP[1][j];
                    if (xnode) {
                        flops_adj_scat += std::llround(cfl_sx[0][j] + cfl_sx[1][j]);
                        alg_adj_scat += cop_sx[0][j] + cop_sx[1][j];
                    } else {
                        flops_adj_scat += std::llround(cfl_s[0][j] + cfl_s[1][j]);
                        alg_adj_scat += cop_s[0][j] + cop_s[1][j];
                    }
                } else if (!leaf && desc->level[i] > 0) {
                    // a non-leaf target's point masses by its axis-pair list
                    const int A = (g->ninfo[i] >> NI_APAIR_SHIFT) & 3;
                    const long long ap = acnt[A][1][j], as = acnt[A][0][j];
                    if (ap + as != cp + cs) return fail(OT_EINVAL, "internal: axis-pair counts differ");
                    flops_fwd += 17 * ap + 32 * as;
                    flops_adj_scat += 16 * ap + 32 * as;
                    alg_fwd += 9.0 * ap + 16.0 * as;
                    alg_adj_scat += 9.0 * ap + 17.0 * as;
                } else {
                    flops_fwd += 17 * cp + 32 * cs;
                    flops_adj_scat += 16 * cp + 32 * cs;
                    alg_fwd += 9.0 * cp + 16.0 * cs;
                    alg_adj_scat += 9.0 * cp + 17.0 * cs;
                }
                // explicit centres: a leaf target reads the table, a non-leaf one evaluates
                flops_fwd_com += leaf ? 17 * cp + 32 * cs : (cp + cs) * (deriv_flops(16) + 32);
                flops_adj_com += leaf ? 16 * cp + 32 * cs : (cp + cs) * (deriv_flops(16) + 32);
            }
            if (mv >> j & 1u) pairs_virt += cp + cs;
        }
        g->node_item_start[i] = static_cast<int>(node_order_items.size());
        const int sl = (g->ninfo[i] >> NI_SLAB_SHIFT) & 3;   // the node's item lane layout
        for (int ph = 0; ph < 16; ++ph) {
            long long cost[3] = {0, 0, 0};   // [1] multipole class, [2] point-mass class
            auto scan = [&](int sg) {
                const std::vector<uint32_t>& mk = mask[sl][ph][sg];
                const std::vector<uint8_t>& pf = pflag[ph][sg];
                for (size_t k = 0; k < mk.size(); ++k) {
                    if (mk[k] & mm) {
                        if (sg == 1) {
                            cost[2] += 8 * 18;     // refined near source: 8 paired contractions
                        } else if (leaf && desc->level[i] > 0) {
                            // not reached: a leaf target's multipole sources run
                            // by the axis-pair lists (below)
                        } else {
                            cost[1] += (pf[k] ? 102 : 70) + (leaf ? 0 : 30);
                        }
                    }
                    if (mk[k] & mo) {
                        cost[2] += pf[k] ? 18 : 16;
                        if (!pf[k]) count_single_mono -= 1;    // 17 ops single in the scatter
                    }
                    if (mk[k] & (mm | mo)) {
                        lanes += 32;
                        padded += 32 * (pf[k] ? 2 : 1);
                    }
                }
            };
            if (by_class) {
                // multipole sources (refined neighbours) by the node's axis-pair
                // list: an entry runs as a pair where both members reach a
                // refined neighbour in some lane, as a single where one does;
                // refined near sources by the near list; point masses by class
                if (mm != 0) {
                    const int A = (g->ninfo[i] >> NI_APAIR_SHIFT) & 3;
                    const std::vector<uint32_t>& m0 = amask[A][sl][ph][0];
                    const std::vector<uint32_t>& m1 = amask[A][sl][ph][1];
                    for (size_t k = 0; k < m0.size(); ++k) {
                        const bool a0 = (m0[k] & mm) != 0, a1 = (m1[k] & mm) != 0;
                        if (a0 && a1) {
                            cost[1] += 102;
                            lanes += 32;
                            padded += 64;
                        } else if (a0 || a1) {
                            cost[1] += 70;
                            lanes += 32;
                            padded += 32;
                        }
                    }
                }
                const uint32_t mo_keep = mo;
                mo = 0;
                scan(1);
                mo = mo_keep;
                long long cost_s = cost[2];    // refined near sources
                for (int cg = 0; cg < 2; ++cg)
                    for (size_t k = 0; k < cmask[sl][ph][cg].size(); ++k)
                        if (cmask[sl][ph][cg][k] & mo) {
                            cost[2] += CCF[cg][k];
                            cost_s += xnode ? ccost_sx[cg][k] : ccost_s[cg][k];
                            lanes += 32;
                            padded += 32 * cmem[cg][k];
                        }
                ops_adj_scat += 32 * cost_s;
            } else if (!leaf) {
                // multipole sources by class, point masses (leaf neighbours)
                // over the far list
                const int cgm = desc->level[i] == 0 ? 3 : 2;
                for (size_t k = 0; k < cmask[sl][ph][cgm].size(); ++k)
                    if (cmask[sl][ph][cgm][k] & mm) {
                        cost[1] += CCF[cgm][k];
                        lanes += 32;
                        padded += 32 * cmem[cgm][k];
                    }
                if (desc->level[i] > 0) {
                    // point masses (leaf neighbours) by the node's axis-pair
                    // list: an entry runs where some lane has a point mass at
                    // either member, 16 FMAs + 2 adds forward and adjoint
                    if (mo != 0) {
                        const int A = (g->ninfo[i] >> NI_APAIR_SHIFT) & 3;
                        const std::vector<uint32_t>& m0 = amask[A][sl][ph][0];
                        const std::vector<uint32_t>& m1 = amask[A][sl][ph][1];
                        for (size_t k = 0; k < m0.size(); ++k) {
                            const bool a0 = (m0[k] & mo) != 0, a1 = (m1[k] & mo) != 0;
                            if (a0 || a1) {
                                cost[2] += 18;
                                lanes += 32;
                                padded += (a0 && a1) ? 64 : 32;
                            }
                        }
                    }
                    ops_adj_scat += 32 * cost[2];
                } else {
                    const uint32_t mm_keep = mm;
                    mm = 0;
                    scan(s1);
                    mm = mm_keep;
                    ops_adj_scat += 32 * (cost[2] - count_single_mono);
                }
            } else {
                scan(s1);
                scan(1);
                // the point-mass adjoint organised by target walks the same active
                // entries: 16 products + 2 adds per paired entry, 16 + 1 single
                ops_adj_scat += 32 * (cost[2] - count_single_mono);
            }
            ops_fwd += 32 * (cost[1] + cost[2]);
            ops_fwd_multi += 32 * cost[1];
            count_single_mono = 0;
            const int item = (i << 4) | ph;
            node_order_items.push_back(item);
            for (int mode = 1; mode <= 3; ++mode) {
                long long cst = ((mode & 1) ? cost[1] : 0) + ((mode & 2) ? cost[2] : 0);
                if (cst > 0) fwd[mode].emplace_back(cst, item);
            }
            node_cost[i] = std::max(node_cost[i], cost[1] + cost[2]);
            total_cost += cost[1] + cost[2];
        }
    }
    g->node_item_start[n] = static_cast<int>(node_order_items.size());
    for (int mode = 1; mode <= 3; ++mode)
        std::stable_sort(fwd[mode].begin(), fwd[mode].end(),
                         [](const std::pair<long long, int>& a, const std::pair<long long, int>& b) {
                             return a.first > b.first;
                         });
    // Long items split into list chunks.  A warp shares its scheduler's FP64
    // unit with the other resident warps for the whole launch, so an item
    // whose work is a large share of one SM's (the root's walk of its 3196
    // offsets, the coarse levels' far lists) would finish last by a wide
    // margin.  Items of a node whose largest item exceeds
    // cap = total / (SMs * 32) run as K = ceil(largest / cap) <= 16 chunks
    // (every walked list cut into K equal ranges); each chunk leaves its
    // accumulators in a partial slot and the node's last chunk to finish sums
    // the K slots in chunk order and stores (the same bits whatever the
    // schedule).  The multipole and fused passes use the chunked lists; the
    // point-mass pass and its adjoint keep whole items.
    {
        const long long cap = std::max<long long>(1024, total_cost / (32LL * std::max(g->num_sms, 1)));
        std::vector<int> nchunk(n, 1);
        g->cinfo.assign(n, int2{-1, 0});
        int slots = 0, ctrs = 0;
        for (int i = 0; i < n; ++i) {
            const long long k = (node_cost[i] + cap - 1) / cap;
            nchunk[i] = static_cast<int>(std::min<long long>(16, std::max<long long>(1, k)));
            if (nchunk[i] > 1) {
                g->cinfo[i] = int2{slots, (ctrs << 4) | (nchunk[i] - 1)};
                slots += 16 * nchunk[i];
                ctrs += 16;
            }
        }
        g->n_part_slots = slots;
        g->n_chunk_ctrs = ctrs;
        for (int mode = 1; mode <= 3; mode += 2) {
            std::vector<std::pair<long long, int>> v;
            for (auto& pr : fwd[mode]) {
                const int k = nchunk[pr.second >> 4];
                for (int c = 0; c < k; ++c) v.emplace_back(pr.first / k, pr.second | (c << 26));
            }
            std::stable_sort(v.begin(), v.end(), [](const std::pair<long long, int>& a,
                                                    const std::pair<long long, int>& b) { return a.first > b.first; });
            g->itemsc_fwd[mode].clear();
            for (auto& pr : v) g->itemsc_fwd[mode].push_back(pr.second);
        }
        g->itemc_node_start.assign(n + 1, 0);
        g->itemsc_node.clear();
        for (int i = 0; i < n; ++i) {
            g->itemc_node_start[i] = static_cast<int>(g->itemsc_node.size());
            for (int ph = 0; ph < 16; ++ph)
                for (int c = 0; c < nchunk[i]; ++c) g->itemsc_node.push_back((i << 4) | ph | (c << 26));
        }
        g->itemc_node_start[n] = static_cast<int>(g->itemsc_node.size());
    }
    // adjoint items: real sources by class, virtual sources (point masses)
    std::vector<std::pair<long long, int>> adj[4];
    std::vector<int> adj_node[4];
    std::vector<long long> adj_node_cost(n, 0);   // largest multipole gather item of a real non-leaf source
    long long total_adj_cost = 0;
    for (int mode = 1; mode <= 3; ++mode) g->adj_item_start[mode].assign(n + g->nvirt + 1, 0);
    for (int i = 0; i < n + g->nvirt; ++i) {
        const bool virt = i >= n;
        const bool leaf = virt || g->is_leaf[i];
        const int2* tbl = virt ? &g->vnbr[static_cast<size_t>(i - n) * 27] : &g->nbr[static_cast<size_t>(i) * 27];
        const int lvl = virt ? g->vinfo[i - n] : desc->level[i];
        const int s1 = (lvl == 0) ? 2 : 0;
        // targets: multipole or leaf cells (far / root), leaf cells (near, for
        // point-mass sources only), and for real leaf sources the virtual
        // children of coarse leaves (depth 1), far and near
        uint32_t tv = 0, tl = 0, tw = 0;
        for (int j = 0; j < 27; ++j) {
            const int k = tbl[j].y & 3;
            if (k == K_MULTI || k == K_LEAF) tv |= 1u << j;
            if (k == K_LEAF) tl |= 1u << j;
            if (!virt && leaf && k == K_VIRT && ((static_cast<unsigned>(tbl[j].y) >> 2) & 7u) == 1u) tw |= 1u << j;
        }
        for (int j = 0; j < 27; ++j) {
            long long cp = ((tv | tw) >> j & 1u) ? cnt[s1][1][j] : 0, cs = ((tv | tw) >> j & 1u) ? cnt[s1][0][j] : 0;
            if (leaf && ((tl | tw) >> j & 1u)) {
                cp += cnt[1][1][j];
                cs += cnt[1][0][j];
            }
            if (leaf) {
                flops_adj += 32 * (cp + cs);
                alg_adj_det += 16.0 * (cp + cs);
            } else if (((tv | tw) >> j) & 1u) {
                // multipole gather by class (segment 2 far, 3 root), with the
                // targets' prebuilt x butterflies when the source is flagged
                const bool xs = !virt && (g->ninfo[i] & NI_XGATHER);
                const int sg = lvl == 0 ? 3 : 2;
                const long long fl = std::llround(xs ? cfl_sx[sg][j] : cfl_s[sg][j]);
                flops_adj += fl;
                flops_adj_multi += fl;
                alg_adj_det += xs ? cop_sx[sg][j] : cop_s[sg][j];
                alg_adj_multi += xs ? cop_sx[sg][j] : cop_s[sg][j];
            }
        }
        const int bit = leaf ? 2 : 1;
        for (int mode = 1; mode <= 3; ++mode) g->adj_item_start[mode][i] = static_cast<int>(adj_node[mode].size());
        for (int ph = 0; ph < 16; ++ph) {
            long long cst = 0;
            if (leaf) {
                for (size_t k = 0; k < mask[0][ph][s1].size(); ++k)
                    if (mask[0][ph][s1][k] & (tv | tw)) cst += pflag[ph][s1][k] ? 32 : 16;
            } else {
                const int cgm = lvl == 0 ? 3 : 2;
                const bool xs = !virt && (g->ninfo[i] & NI_XGATHER);
                for (size_t k = 0; k < cmask[0][ph][cgm].size(); ++k)
                    if (cmask[0][ph][cgm][k] & tv) cst += xs ? ccost_sx[cgm][k] : ccost_s[cgm][k];
            }
            if (leaf)
                for (size_t k = 0; k < mask[0][ph][1].size(); ++k)
                    if (mask[0][ph][1][k] & (tl | tw)) cst += 32;
            if (cst == 0) continue;
            ops_adj += 32 * cst;
            if (!leaf) {
                ops_adj_multi += 32 * cst;
                adj_node_cost[i] = std::max(adj_node_cost[i], cst);
                total_adj_cost += cst;
            }
            const int item = (i << 4) | ph;
            for (int mode = 1; mode <= 3; ++mode)
                if (mode & bit) {
                    adj[mode].emplace_back(cst, item);
                    adj_node[mode].push_back(item);
                }
        }
    }
    for (int mode = 1; mode <= 3; ++mode) g->adj_item_start[mode][n + g->nvirt] = static_cast<int>(adj_node[mode].size());
    for (int mode = 1; mode <= 3; ++mode)
        std::stable_sort(adj[mode].begin(), adj[mode].end(),
                         [](const std::pair<long long, int>& a, const std::pair<long long, int>& b) {
                             return a.first > b.first;
                         });
    // forward items hold the node in bits 4-25 (chunk index in 26-29), adjoint
    // items the source in bits 4-29
    if (n >= (1 << 22) || static_cast<long long>(n + g->nvirt) >= (1LL << 26))
        return fail(OT_EINVAL, "too many sub-grids");
    // the default adjoint: point-mass scatter items (forward items of the
    // point-mass class, flagged with bit 30) merged with the multipole gather
    // items, longest first, in one persistent launch
    std::vector<std::pair<long long, int>> fast[2];
    for (auto& pr : fwd[2]) {
        fast[0].emplace_back(pr.first, pr.second | (1 << 30));
        fast[1].emplace_back(pr.first, pr.second | (1 << 30));
    }
    for (auto& pr : adj[1]) fast[1].push_back(pr);
    for (int k = 0; k < 2; ++k)
        std::stable_sort(fast[k].begin(), fast[k].end(),
                         [](const std::pair<long long, int>& a, const std::pair<long long, int>& b) {
                             return a.first > b.first;
                         });
    // Multipole gather items split into list chunks as the forward's are
    // (a source's gather walks the transposed stencil: the same long lists
    // at the root and the coarse levels).  A chunked item sets bit 31 and
    // holds the source in bits 4-25, the chunk index in bits 26-29.
    {
        const long long cap = std::max<long long>(1024, total_adj_cost / (32LL * std::max(g->num_sms, 1)));
        std::vector<int> nchunk(n, 1);
        g->cinfo_adj.assign(n, int2{-1, 0});
        int slots = 0, ctrs = 0;
        for (int i = 0; i < n; ++i) {
            const long long k = (adj_node_cost[i] + cap - 1) / cap;
            nchunk[i] = static_cast<int>(std::min<long long>(16, std::max<long long>(1, k)));
            if (nchunk[i] > 1) {
                g->cinfo_adj[i] = int2{slots, (ctrs << 4) | (nchunk[i] - 1)};
                slots += 16 * nchunk[i];
                ctrs += 16;
            }
        }
        g->n_part_slots_adj = slots;
        g->n_chunk_ctrs_adj = ctrs;
        auto chunk_list = [&](const std::vector<std::pair<long long, int>>& in, std::vector<int>& out) {
            std::vector<std::pair<long long, int>> v;
            for (auto& pr : in) {
                const int src = (pr.second >> 4) & 0x3ffffff;
                const bool gather = !((pr.second >> 30) & 1) && src < n;
                const int k = gather ? nchunk[src] : 1;
                if (k == 1) {
                    v.push_back(pr);
                } else {
                    for (int c = 0; c < k; ++c)
                        v.emplace_back(pr.first / k, static_cast<int>(0x80000000u | static_cast<unsigned>(
                                                                         (src << 4) | (pr.second & 15) | (c << 26))));
                }
            }
            std::stable_sort(v.begin(), v.end(), [](const std::pair<long long, int>& a,
                                                    const std::pair<long long, int>& b) { return a.first > b.first; });
            out.clear();
            for (auto& pr : v) out.push_back(pr.second);
        };
        for (int mode = 1; mode <= 3; mode += 2) {
            chunk_list(adj[mode], g->itemsc_adj[mode]);
            // source order (plain path)
            g->itemc_adj_start[mode].assign(n + g->nvirt + 1, 0);
            g->itemsc_adj_node[mode].clear();
            for (int i = 0; i < n + g->nvirt; ++i) {
                g->itemc_adj_start[mode][i] = static_cast<int>(g->itemsc_adj_node[mode].size());
                for (int t = g->adj_item_start[mode][i]; t < g->adj_item_start[mode][i + 1]; ++t) {
                    const int item = adj_node[mode][t];
                    const int k = i < n ? nchunk[i] : 1;
                    for (int c = 0; c < k; ++c)
                        g->itemsc_adj_node[mode].push_back(
                            k == 1 ? item : static_cast<int>(0x80000000u | static_cast<unsigned>(item | (c << 26))));
                }
            }
            g->itemc_adj_start[mode][n + g->nvirt] = static_cast<int>(g->itemsc_adj_node[mode].size());
        }
        chunk_list(fast[1], g->itemsc_adj_fast1);
    }

    // --- coarse leaf targets next to refined sub-grids ------------------------
    // A leaf's near sources in a refined neighbour are replaced by that
    // cell's children one level down (seen from the leaf's virtual
    // children); they must be leaf cells, which 2:1 balance guarantees: every
    // child of a refined neighbour that touches the leaf must be a leaf.
    std::vector<int> child_of(static_cast<size_t>(n) * 8, -1);
    for (int i = 0; i < n; ++i)
        for (int b = 0; b < 8; ++b)
            child_of[static_cast<size_t>(i) * 8 + b] =
                B.find(desc->level[i] + 1, 2L * desc->coord[3 * i] + (b & 1),
                       2L * desc->coord[3 * i + 1] + ((b >> 1) & 1), 2L * desc->coord[3 * i + 2] + (b >> 2));
    for (int i = 0; i < n; ++i) {
        if (!g->is_leaf[i]) continue;
        for (int j = 0; j < 27; ++j) {
            const int2 e = g->nbr[static_cast<size_t>(i) * 27 + j];
            if ((e.y & 3) != K_MULTI) continue;
            for (int b = 0; b < 8; ++b) {
                const int c = child_of[static_cast<size_t>(e.x) * 8 + b];
                if (c < 0 || g->is_leaf[c]) continue;
                bool touch = true;
                for (int a = 0; a < 3; ++a) {
                    const long cc = 2L * desc->coord[3 * e.x + a] + ((b >> a) & 1);
                    const long lo = 2L * desc->coord[3 * i + a];
                    touch = touch && cc >= lo - 1 && cc <= lo + 2;
                }
                if (touch)
                    return fail(OT_EINVAL,
                                "tree is not 2:1 balanced: leaf sub-grid %d (level %d) touches refined sub-grid %d "
                                "of its neighbour's children",
                                i, desc->level[i], c);
            }
        }
    }
    // virtual-child mean rows: Dv[q][j] = 2^(n_j+1)/8 * sum_cv Dt[row(q - cv)][j],
    // q = 2o + cs in [-6, 7]^3 (row(o) holds the derivatives at -o)
    std::vector<double> Dv(static_cast<size_t>(NVROW) * 16, 0.0);
    {
        const double fo[4] = {0.25, 0.5, 1.0, 2.0};
        const int ord[16] = {0, 1, 1, 1, 2, 2, 2, 2, 2, 3, 3, 3, 3, 3, 3, 3};
        for (int qz = -6; qz <= 7; ++qz)
            for (int qy = -6; qy <= 7; ++qy)
                for (int qx = -6; qx <= 7; ++qx) {
                    double* out = &Dv[static_cast<size_t>((qx + 6) + 14 * (qy + 6) + 196 * (qz + 6)) * 16];
                    for (int cv = 0; cv < 8; ++cv) {
                        const int rx = qx - (cv & 1), ry = qy - ((cv >> 1) & 1), rz = qz - (cv >> 2);
                        const double* row = &Dt[static_cast<size_t>((rx + 7) + 15 * (ry + 7) + 225 * (rz + 7)) * DROW];
                        for (int j = 0; j < 16; ++j) out[j] += row[j];
                    }
                    for (int j = 0; j < 16; ++j) out[j] *= fo[ord[j]];
                }
    }

    // --- M2M schedule ---------------------------------------------------------
    std::vector<int> nonleaf, all(n), cube;
    for (int i = 0; i < n; ++i) {
        all[i] = i;
        if (!g->is_leaf[i]) nonleaf.push_back(i);
    }
    std::map<int, M2MLevel> lv;
    for (int i = 0; i < n; ++i) {
        const int l = desc->level[i];
        int ch[8];
        int nch = 0;
        for (int b = 0; b < 8; ++b) {
            ch[b] = B.find(l + 1, 2L * desc->coord[3 * i] + (b & 1), 2L * desc->coord[3 * i + 1] + ((b >> 1) & 1),
                           2L * desc->coord[3 * i + 2] + (b >> 2));
            if (ch[b] >= 0) nch++;
        }
        if (nch == 8) {
            M2MLevel& L = lv[l];
            L.level = l;
            L.parents.push_back(i);
            L.children.insert(L.children.end(), ch, ch + 8);
        } else {
            cube.push_back(i);
        }
    }
    g->m2m.clear();
    for (auto it = lv.rbegin(); it != lv.rend(); ++it) g->m2m.push_back(it->second);

    // --- info -----------------------------------------------------------------
    ot_grid_info_t& I = g->info;
    std::memset(&I, 0, sizeof(I));
    I.n_subgrids = n;
    I.n_virtual = g->nvirt;
    I.max_level = g->max_level;
    I.far_offsets = g->far_offsets;
    I.near_offsets = 2 * g->near_len;
    I.root_offsets = 2 * g->root_len;
    I.pairs_multipole = pairs_multi;
    I.pairs_monopole = pairs_mono;
    I.pairs_virtual = pairs_virt;
    I.pairs_refined = pairs_ref;
    I.pairs_angular = pairs_ang;
    I.lanes_fwd = lanes;
    I.pairs_padded_fwd = padded;
    I.chunked_subgrids = g->n_chunk_ctrs / 16;
    I.flops_fwd = flops_fwd;
    I.fp64_ops_fwd = std::llround(alg_fwd);
    I.fp64_ops_fwd_multi = std::llround(alg_fwd_multi);
    I.ops_fwd_multi = ops_fwd_multi;
    g->fp64_ops_adj_det = std::llround(alg_adj_det);
    g->fp64_ops_adj_fast = std::llround(alg_adj_multi + alg_adj_scat);
    I.fp64_ops_adj = g->fp64_ops_adj_fast;
    I.fp64_ops_adj_multi = std::llround(alg_adj_multi);
    I.ops_adj_multi = ops_adj_multi;
    g->flops_adj_det = flops_adj;
    g->ops_adj_det = ops_adj;
    g->flops_adj_fast = flops_adj_multi + flops_adj_scat;
    g->ops_adj_fast = ops_adj_multi + ops_adj_scat;
    I.flops_adj = g->flops_adj_fast;
    I.ops_fwd = ops_fwd;
    I.ops_adj = g->ops_adj_fast;
    I.flops_fwd_com = flops_fwd_com;
    I.flops_adj_com = flops_adj_com;
    for (int w = 2; w <= 8; w *= 2) {
        g->maxb_emu[2][w] = forward_max_blocks_per_sm(6, w);
        g->maxb_emu[3][w] = forward_max_blocks_per_sm(7, w);
        g->maxb_emu2[1][w] = forward_max_blocks_per_sm(5, w);
        g->maxb_emu2[3][w] = forward_max_blocks_per_sm(8, w);
        for (int m : {9, 12}) g->maxb_adj_emu[m][w] = adjoint_max_blocks_per_sm(m, w);
        g->maxb_scat[w] = scatter_max_blocks_per_sm(w);
        g->maxb_adj[4 - 4][w] = adjoint_max_blocks_per_sm(4, w);   // slot 0: fused, point masses only
    }
    for (int mode = 1; mode <= 3; ++mode)
        for (int w = 2; w <= 8; w *= 2) {
            g->maxb_fwd[mode][w] = forward_max_blocks_per_sm(mode, w);
            g->maxb_adj[mode][w] = adjoint_max_blocks_per_sm(mode, w);
            g->maxb_com_fwd[mode][w] = forward_com_max_blocks_per_sm(mode, w);
            g->maxb_com_adj[mode][w] = adjoint_com_max_blocks_per_sm(mode, w);
            if (mode <= 2) g->maxb_com_adj[3 + mode][w] = adjoint_com_max_blocks_per_sm(3 + mode, w);
        }

    // --- uploads ----------------------------------------------------------------
    ot_status st;
#define UP(ptr, vec) \
    if ((st = g->upload(&(ptr), vec, s)) != OT_OK) return st;
    UP(g->d_nbr, g->nbr);
    UP(g->d_vnbr, g->vnbr);
    UP(g->d_ninfo, g->ninfo);
    UP(g->d_vinfo, g->vinfo);
    UP(g->d_vcoord, vcoord);
    UP(g->d_child_of, child_of);
    UP(g->d_Dv, Dv);
    {
        std::vector<int> nc(desc->coord, desc->coord + 3 * static_cast<size_t>(n));
        UP(g->d_ncoord, nc);
    }
    UP(g->d_Dt, Dt);
    {
        std::vector<float> Dt32(static_cast<size_t>(NOFF) * 32, 0.0f);
        for (int r = 0; r < NOFF; ++r)
            for (int j = 0; j < 16; ++j) {
                const double v = Dt[static_cast<size_t>(r) * DROW + j];
                const float hi = static_cast<float>(v);
                Dt32[static_cast<size_t>(r) * 32 + j] = hi;
                Dt32[static_cast<size_t>(r) * 32 + 16 + j] = static_cast<float>(v - static_cast<double>(hi));
            }
        UP(g->d_Dt32, Dt32);
        std::vector<float2> Dt2(static_cast<size_t>(NOFF) * DROW);
        for (size_t i = 0; i < Dt2.size(); ++i) {
            const float hi = static_cast<float>(Dt[i]);
            Dt2[i] = make_float2(hi, static_cast<float>(Dt[i] - static_cast<double>(hi)));
        }
        UP(g->d_Dt2, Dt2);
    }
    UP(g->d_lists, g->lists);
    g->Lh.lists = g->d_lists;
    std::vector<double> hv(g->hinv, g->hinv + MAXLEV);
    UP(g->d_hinv, hv);
    for (int mode = 1; mode <= 3; ++mode) {
        std::vector<int> items;
        for (auto& pr : fwd[mode]) items.push_back(pr.second);
        g->n_items_fwd[mode] = static_cast<int>(items.size());
        UP(g->d_items_fwd[mode], items);
        std::vector<int> aitems;
        for (auto& pr : adj[mode]) aitems.push_back(pr.second);
        g->n_items_adj[mode] = static_cast<int>(aitems.size());
        UP(g->d_items_adj[mode], aitems);
        UP(g->d_items_adj_node[mode], adj_node[mode]);
    }
    UP(g->d_items_fwd_node, node_order_items);
    for (int mode = 1; mode <= 3; mode += 2) {
        g->n_itemsc_fwd[mode] = static_cast<int>(g->itemsc_fwd[mode].size());
        UP(g->d_itemsc_fwd[mode], g->itemsc_fwd[mode]);
    }
    UP(g->d_itemsc_node, g->itemsc_node);
    UP(g->d_cinfo, g->cinfo);
    for (int mode = 1; mode <= 3; mode += 2) {
        g->n_itemsc_adj[mode] = static_cast<int>(g->itemsc_adj[mode].size());
        UP(g->d_itemsc_adj[mode], g->itemsc_adj[mode]);
        UP(g->d_itemsc_adj_node[mode], g->itemsc_adj_node[mode]);
    }
    g->n_itemsc_adj_fast1 = static_cast<int>(g->itemsc_adj_fast1.size());
    UP(g->d_itemsc_adj_fast1, g->itemsc_adj_fast1);
    UP(g->d_cinfo_adj, g->cinfo_adj);
    for (int k = 0; k < 2; ++k) {
        std::vector<int> items;
        for (auto& pr : fast[k]) items.push_back(pr.second);
        g->n_items_adj_fast[k] = static_cast<int>(items.size());
        UP(g->d_items_adj_fast[k], items);
    }
    g->n_nonleaf = static_cast<int>(nonleaf.size());
    UP(g->d_nonleaf, nonleaf);
    UP(g->d_all, all);
    g->n_cube = static_cast<int>(cube.size());
    UP(g->d_cube, cube);
    UP(g->d_leaf, cube);
    UP(g->d_nslot, g->nslot);
    UP(g->d_snbM, g->snbM);
    UP(g->d_snbX, g->snbX);
    UP(g->d_mem_ent, g->mem_ent);
    UP(g->d_mem_xs, g->mem_xs);
    UP(g->d_xym_ys, g->xym_ys);
    for (auto& L : g->m2m) {
        UP(L.d_parents, L.parents);
        UP(L.d_children, L.children);
    }
    UP(g->d_vmap, vmap);
#undef UP
    if ((st = g->alloc(&g->d_Mhat, static_cast<size_t>(n) * NRED * NCELL)) != OT_OK) return st;
    if ((st = g->alloc(&g->d_Sx, static_cast<size_t>(std::max(g->n_slotXyz, 1)) * 7 * 32 * NCELL)) != OT_OK)
        return st;
    if ((st = g->alloc(&g->d_Sm, static_cast<size_t>(std::max(g->n_slotM, 1)) * 7 * 2 * NCELL)) != OT_OK) return st;
    if ((st = g->alloc(&g->d_Tx, static_cast<size_t>(std::max(g->n_slotXyz, 1)) * 7 * 32 * NCELL)) != OT_OK)
        return st;
    if ((st = g->alloc(&g->d_Sbar, static_cast<size_t>(std::max(g->n_slotM, 1)) * 7 * 2 * NCELL)) != OT_OK) return st;
    if ((st = g->alloc(&g->d_Smf, static_cast<size_t>(std::max(g->n_slotM, 1)) * 7 * 2 * NCELL)) != OT_OK) return st;
    if (g->use_xy &&
        (st = g->alloc(&g->d_Sxy, static_cast<size_t>(std::max(g->n_slotXY, 1)) * 49 * 4 * NCELL)) != OT_OK)
        return st;
    if (g->use_xym &&
        (st = g->alloc(&g->d_Sxym, static_cast<size_t>(std::max(g->n_slotXz, 1)) * 49 * 64 * NCELL)) != OT_OK)
        return st;
    if ((st = g->alloc(&g->d_Lrbar, static_cast<size_t>(n) * NRED * NCELL)) != OT_OK) return st;
    if ((st = g->alloc(&g->d_vbar, static_cast<size_t>(std::max(g->nvirt, 1)) * NCELL)) != OT_OK) return st;
    if ((st = g->alloc(&g->d_Mb, static_cast<size_t>(n) * NCOMP * NCELL)) != OT_OK) return st;
    if ((st = g->alloc(&g->d_mf, static_cast<size_t>(n) * NCELL)) != OT_OK) return st;
    if ((st = g->alloc(&g->d_Mf, static_cast<size_t>(n) * NRED * NCELL)) != OT_OK) return st;
    if ((st = g->alloc(&g->d_counters, 4)) != OT_OK) return st;
    {
        const size_t part = std::max<size_t>({static_cast<size_t>(g->n_part_slots) * PART_VALS,
                                              static_cast<size_t>(g->n_part_slots_adj) * NRED, 1});
        const size_t ctrs = std::max({g->n_chunk_ctrs, g->n_chunk_ctrs_adj, 1});
        if ((st = g->alloc(&g->d_part, part * 32)) != OT_OK) return st;
        if ((st = g->alloc(&g->d_chunk_ctr, ctrs)) != OT_OK) return st;
    }
    if ((st = g->alloc(&g->d_status, 2)) != OT_OK) return st;
    OT_CUDA(cudaMemsetAsync(g->d_status, 0, 2 * sizeof(int), s));
    OT_CUDA(cudaMemsetAsync(g->d_counters, 0, 4 * sizeof(int), s));
    return OT_OK;
}

// ---------------------------------------------------------------------------
// launches
// ---------------------------------------------------------------------------

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

static int grid_blocks(ot_grid* g, int bps_max) {
    int bps = g->bps > 0 ? std::min(g->bps, bps_max) : bps_max;
    if (bps < 1) bps = 1;
    return g->num_sms * bps;
}

static FwdParams fwd_params(ot_grid* g, const double* m, double* L, double* Lc, int accumulate) {
    FwdParams p;
    std::memset(&p, 0, sizeof(p));
    p.counter = g->d_counters;
    p.nbr = g->d_nbr;
    p.ninfo = g->d_ninfo;
    p.Dt = g->d_Dt;
    p.L = g->Lh;
    p.Mhat = g->d_Mhat;
    p.m = m;
    p.Lout = L;
    p.Lc = Lc;
    p.accumulate = accumulate;
    p.n_nodes = g->n;
    p.status = g->d_status;
    p.child_of = g->d_child_of;
    p.Dv = g->d_Dv;
    p.nslot = g->d_nslot;
    for (int l = 0; l < MAXLEV; ++l) p.hinv[l] = g->hinv[l];
    return p;
}

// enqueue one forward pass (mode 1, 2 or 3) on stream s
static ot_status enqueue_forward(ot_grid* g, int mode, const double* M, const double* m, double* L, double* Lc,
                                 int accumulate, cudaStream_t s) {
    if (mode == 3 && (g->precision != 0 || g->use_xy)) {
        // Both passes as two launches.  With double-float contractions the
        // one kernel holds the multipole code and the double-float point-mass
        // code at once, and the mix of the two item kinds on an SM ran
        // 1.5-1.7x slower than the two launches.  In FP64 with the masses'
        // (x, y) table the point-mass items stream that table (0.8 MB per
        // leaf sub-grid) through L2 while the multipole items reread theirs:
        // fused, the two passes took 8.35 ms against 4.40 + 3.51 ms apart.
        // The per-sub-grid schedule splits alike, so that both schedules sum
        // in the same order.
        ot_status st = enqueue_forward(g, 1, M, m, L, Lc, accumulate, s);
        if (st != OT_OK) return st;
        return enqueue_forward(g, 2, M, m, L, nullptr, 1, s);
    }
    const size_t nL = static_cast<size_t>(g->n) * NCOMP * NCELL;
    if (mode & 1) {
        PrepParams pp;
        std::memset(&pp, 0, sizeof(pp));
        pp.src = M;
        pp.dst = g->d_Mhat;
        pp.nodes = g->d_nonleaf;
        pp.n_list = g->n_nonleaf;
        pp.ninfo = g->d_ninfo;
        for (int l = 0; l < MAXLEV; ++l) pp.hinv[l] = g->hinv[l];
        OT_CUDA(launch_prescale_moments(pp, s));
    }
    if (!accumulate) OT_CUDA(cudaMemsetAsync(L, 0, nL * sizeof(double), s));
    if ((mode & 1) && Lc) OT_CUDA(cudaMemsetAsync(Lc, 0, static_cast<size_t>(g->n) * 3 * NCELL * sizeof(double), s));
    FwdParams p = fwd_params(g, m, L, (mode & 1) ? Lc : nullptr, 1);
    // prebuilt x butterflies of the class transforms (FP64 contractions only)
    if ((mode & 1) && g->precision != 2 && g->n_slotX > 0) {
        OT_CUDA(launch_xbutterfly_moments(g->d_snbX, g->n_slotXyz, g->d_Mhat, g->n, g->d_Sx, s));
        p.Sx = g->d_Sx;
        if (g->use_xym) {
            OT_CUDA(launch_xybutterfly_moments(g->d_xym_ys, g->n_slotXz, g->d_Sx, g->d_Sxym, s));
            p.Sxym = g->d_Sxym;
        }
    }
    if ((mode & 2) && g->n_slotM > 0) {
        OT_CUDA(launch_xbutterfly_masses(g->d_snbM, g->n_slotM, m, g->n, g->d_Sm, s));
        if (g->precision == 0) {
            p.Sm = g->d_Sm;
            if (g->use_xy) {
                OT_CUDA(launch_xybutterfly_masses(g->d_snbM, g->n_slotXY, m, g->n, g->d_Sxy, s));
                p.Sxy = g->d_Sxy;
            }
        } else {
            // double-float point masses read the table as (hi, lo) pairs
            OT_CUDA(launch_split_masses(g->d_Sm, g->d_Smf, static_cast<size_t>(g->n_slotM) * 7 * 2 * NCELL, s));
            p.Smf = g->d_Smf;
        }
    }
    const bool emu = g->precision >= 1 && (mode & 2);       // double-float point masses
    const bool emu2 = g->precision == 2 && (mode & 1);      // double-float multipole contractions
    if (emu) {
        OT_CUDA(launch_split_masses(m, g->d_mf, static_cast<size_t>(g->n) * NCELL, s));
        p.mf = g->d_mf;
        p.Dt32 = g->d_Dt32;
    }
    if (emu2) {
        OT_CUDA(launch_split_moments(g->d_Mhat, g->d_Mf, g->d_nonleaf, g->n_nonleaf, s));
        p.Mf = g->d_Mf;
        p.Dt2 = g->d_Dt2;
    }
    // zeroed above, so the kernel always accumulates
    const bool chunked = (mode & 1) != 0;     // the multipole and fused passes run chunked items
    if (chunked) {
        p.cinfo = g->d_cinfo;
        p.part = g->d_part;
        p.chunk_ctr = g->d_chunk_ctr;
        if (g->n_chunk_ctrs > 0)
            OT_CUDA(cudaMemsetAsync(g->d_chunk_ctr, 0, static_cast<size_t>(g->n_chunk_ctrs) * sizeof(int), s));
    }
    if (g->schedule == OT_SCHED_PER_SUBGRID) {
        const int* base = chunked ? g->d_itemsc_node : g->d_items_fwd_node;
        const std::vector<int>& start = chunked ? g->itemc_node_start : g->node_item_start;
        for (int i = 0; i < g->n; ++i) {
            FwdParams q = p;
            q.items = base + start[i];
            q.n_items = start[i + 1] - start[i];
            const int blocks = (q.n_items + g->wpb - 1) / g->wpb;
            OT_CUDA(launch_forward(q, mode, false, g->wpb, blocks, s));
        }
    } else {
        p.items = chunked ? g->d_itemsc_fwd[mode] : g->d_items_fwd[mode];
        p.n_items = chunked ? g->n_itemsc_fwd[mode] : g->n_items_fwd[mode];
        OT_CUDA(cudaMemsetAsync(g->d_counters, 0, sizeof(int), s));
        const int maxb = emu2 ? g->maxb_emu2[mode][g->wpb]
                         : emu ? g->maxb_emu[mode][g->wpb] : g->maxb_fwd[mode][g->wpb];
        const int blocks = grid_blocks(g, maxb);
        OT_CUDA(launch_forward(p, mode, true, g->wpb, blocks, s, blocks == g->num_sms));
    }
    return OT_OK;
}

static ot_status enqueue_scatter(ot_grid* g, double* mbar, cudaStream_t s) {
    ScatParams p;
    std::memset(&p, 0, sizeof(p));
    p.counter = g->d_counters + 2;
    p.nbr = g->d_nbr;
    p.ninfo = g->d_ninfo;
    p.Dt = g->d_Dt;
    p.L = g->Lh;
    p.Lrbar = g->d_Lrbar;
    p.mbar = mbar;
    p.n_nodes = g->n;
    p.status = g->d_status;
    p.child_of = g->d_child_of;
    p.Dv = g->d_Dv;
    if (g->schedule == OT_SCHED_PER_SUBGRID) {
        for (int i = 0; i < g->n; ++i) {
            ScatParams q = p;
            q.items = g->d_items_fwd_node + g->node_item_start[i];
            q.n_items = g->node_item_start[i + 1] - g->node_item_start[i];
            OT_CUDA(launch_scatter_adjoint(q, false, g->wpb, (q.n_items + g->wpb - 1) / g->wpb, s));
        }
    } else {
        p.items = g->d_items_fwd[2];
        p.n_items = g->n_items_fwd[2];
        OT_CUDA(cudaMemsetAsync(g->d_counters + 2, 0, sizeof(int), s));
        OT_CUDA(launch_scatter_adjoint(p, true, g->wpb, grid_blocks(g, g->maxb_scat[g->wpb]), s));
    }
    return OT_OK;
}

// lbar_ready: d_Lrbar already holds this call's prescaled L-bar
static ot_status enqueue_backward(ot_grid* g, const double* Lbar, double* Mbar, double* mbar, cudaStream_t s,
                                  bool lbar_ready = false) {
    int mode = (Mbar ? 1 : 0) | (mbar ? 2 : 0);
    if (mode == 0) return OT_OK;
    const bool scatter = !g->deterministic && mbar != nullptr;
    if (mode == 3 && scatter && g->schedule == OT_SCHED_PERSISTENT) {
        // the multipole gather and the point-mass scatter as two launches:
        // the gather's kernel holds 254 registers (8 warps per SM), the
        // scatter's 128 (16 warps per SM); on the 64^3 polytrope the two
        // launches take 7.19 ms against 7.47 ms for one kernel holding both
        // walks (double-float: 1.35x)
        ot_status st = enqueue_backward(g, Lbar, Mbar, nullptr, s, lbar_ready);
        if (st != OT_OK) return st;
        return enqueue_backward(g, Lbar, nullptr, mbar, s, true);
    }
    if (!lbar_ready) {
        PrepParams pp;
        std::memset(&pp, 0, sizeof(pp));
        pp.src = Lbar;
        pp.dst = g->d_Lrbar;
        pp.nodes = g->d_all;
        pp.n_list = g->n;
        pp.ninfo = g->d_ninfo;
        for (int l = 0; l < MAXLEV; ++l) pp.hinv[l] = g->hinv[l];
        OT_CUDA(launch_prescale_adjoint(pp, s));
    }
    if (Mbar) OT_CUDA(cudaMemsetAsync(Mbar, 0, static_cast<size_t>(g->n) * NCOMP * NCELL * sizeof(double), s));
    if (mbar) OT_CUDA(cudaMemsetAsync(mbar, 0, static_cast<size_t>(g->n) * NCELL * sizeof(double), s));
    if (scatter && g->schedule == OT_SCHED_PER_SUBGRID) {
        ot_status st = enqueue_scatter(g, mbar, s);
        if (st != OT_OK) return st;
        mode &= 1;               // multipole sources still gather
        if (mode == 0) return OT_OK;
    }
    AdjParams p;
    std::memset(&p, 0, sizeof(p));
    // multipole gathers (modes 1 and 3, and the merged default list) run the
    // chunked items
    const bool chunked = (mode & 1) != 0;
    p.items = chunked ? g->d_itemsc_adj[mode] : g->d_items_adj[mode];
    p.n_items = chunked ? g->n_itemsc_adj[mode] : g->n_items_adj[mode];
    if (chunked) {
        p.cinfo = g->d_cinfo_adj;
        p.part = g->d_part;
        p.chunk_ctr = g->d_chunk_ctr;
        if (g->n_chunk_ctrs_adj > 0)
            OT_CUDA(cudaMemsetAsync(g->d_chunk_ctr, 0, static_cast<size_t>(g->n_chunk_ctrs_adj) * sizeof(int), s));
        // the targets' L-bar x butterflies for the FP64 multipole gather
        if (g->precision != 2 && g->n_slotX > 0) {
            OT_CUDA(launch_xbutterfly_lbar(g->d_snbX, g->n_slotXyz, g->d_Lrbar, g->n, g->d_Tx, s));
            p.Tx = g->d_Tx;
        }
    }
    p.nslot = g->d_nslot;
    p.counter = g->d_counters + 1;
    p.nbr = g->d_nbr;
    p.vnbr = g->d_vnbr;
    p.ninfo = g->d_ninfo;
    p.vinfo = g->d_vinfo;
    p.Dt = g->d_Dt;
    p.L = g->Lh;
    p.Lrbar = g->d_Lrbar;
    p.Mbar = Mbar;
    p.mbar = mbar;
    p.vbar = g->d_vbar;
    p.n_nodes = g->n;
    p.status = g->d_status;
    p.child_of = g->d_child_of;
    p.Dv = g->d_Dv;
    for (int l = 0; l < MAXLEV; ++l) p.hinv[l] = g->hinv[l];
    if (g->schedule == OT_SCHED_PER_SUBGRID) {
        // one launch per source sub-grid (real and virtual)
        const std::vector<int>& st = chunked ? g->itemc_adj_start[mode] : g->adj_item_start[mode];
        const int* base = chunked ? g->d_itemsc_adj_node[mode] : g->d_items_adj_node[mode];
        for (int i = 0; i + 1 < static_cast<int>(st.size()); ++i) {
            AdjParams q = p;
            q.items = base + st[i];
            q.n_items = st[i + 1] - st[i];
            if (q.n_items == 0) continue;
            OT_CUDA(launch_adjoint(q, mode, false, g->wpb, (q.n_items + g->wpb - 1) / g->wpb, s));
        }
    } else if (scatter) {
        // the point-mass adjoint by target as one persistent launch, longest
        // items first (mode 2 only here: a call that wants M-bar too ran the
        // gather before it as its own launch)
        p.items = g->d_items_adj_fast[0];
        p.n_items = g->n_items_adj_fast[0];
        int maxb = g->maxb_adj[0][g->wpb];
        if (g->precision == OT_PREC_DF64) {
            // double-float: L-bar split into (hi, lo) pairs in the moments'
            // scratch (calls on one grid are serialized)
            OT_CUDA(launch_split_moments(g->d_Lrbar, g->d_Mf, g->d_all, g->n, s));
            p.Lf = g->d_Mf;
            p.Dt2 = g->d_Dt2;
            p.Dt32 = g->d_Dt32;
            maxb = g->maxb_adj_emu[12][g->wpb];
        }
        // FP64 scatter: the x stage of x-complete classes deferred to a pass
        // over the leaf cells
        const bool defer = !g->mem_ent.empty();
        if (defer) {
            OT_CUDA(cudaMemsetAsync(g->d_Sbar, 0, static_cast<size_t>(g->n_slotM) * 7 * 2 * NCELL * sizeof(double), s));
            p.Sbar = g->d_Sbar;
        }
        OT_CUDA(cudaMemsetAsync(g->d_counters + 1, 0, sizeof(int), s));
        OT_CUDA(launch_adjoint(p, 4, true, g->wpb, grid_blocks(g, maxb), s));
        if (defer)
            OT_CUDA(launch_xbutterfly_masses_adjoint(g->d_mem_ent, g->d_mem_xs, static_cast<int>(g->mem_ent.size()),
                                                     g->d_Sbar, g->n, mbar, s));
    } else {
        int maxb = g->maxb_adj[mode][g->wpb];
        if (g->precision == OT_PREC_DF64 && mode == 1) {
            OT_CUDA(launch_split_moments(g->d_Lrbar, g->d_Mf, g->d_all, g->n, s));
            p.Lf = g->d_Mf;
            p.Dt2 = g->d_Dt2;
            p.Dt32 = g->d_Dt32;
            maxb = g->maxb_adj_emu[9][g->wpb];
        }
        OT_CUDA(cudaMemsetAsync(g->d_counters + 1, 0, sizeof(int), s));
        OT_CUDA(launch_adjoint(p, mode, true, g->wpb, grid_blocks(g, maxb), s));
    }
    if (!scatter && mbar && g->vmap_rows > 0)
        OT_CUDA(launch_restrict_virtual(g->d_vbar, g->d_vmap, g->vmap_rows, mbar, s));
    return OT_OK;
}

// --- explicit expansion centres ---------------------------------------------
// The same units as the table path (sources prescaled by h^-m, coefficients
// by h^-(n+1)); pairs involving a centre from C evaluate their derivatives at
// R/h.  Always the persistent schedule (LPT-ordered items, one launch).

static void com_scales(ot_grid* g, double* hinv, double* hreal) {
    for (int l = 0; l < MAXLEV; ++l) {
        hinv[l] = g->hinv[l];
        hreal[l] = std::ldexp(g->h0, -l);
    }
}

static ot_status enqueue_forward_com(ot_grid* g, int mode, const double* M, const double* m, const double* C,
                                     double* L, double* Lc, cudaStream_t s) {
    if (mode & 1) {
        PrepParams pp;
        std::memset(&pp, 0, sizeof(pp));
        pp.src = M;
        pp.dst = g->d_Mhat;
        pp.nodes = g->d_nonleaf;
        pp.n_list = g->n_nonleaf;
        pp.ninfo = g->d_ninfo;
        for (int l = 0; l < MAXLEV; ++l) pp.hinv[l] = g->hinv[l];
        OT_CUDA(launch_prescale_moments(pp, s));
    }
    OT_CUDA(cudaMemsetAsync(L, 0, static_cast<size_t>(g->n) * NCOMP * NCELL * sizeof(double), s));
    if ((mode & 1) && Lc) OT_CUDA(cudaMemsetAsync(Lc, 0, static_cast<size_t>(g->n) * 3 * NCELL * sizeof(double), s));
    FwdParams p = fwd_params(g, m, L, (mode & 1) ? Lc : nullptr, 1);
    com_scales(g, p.hinv, p.hreal);
    p.C = C;
    p.ncoord = g->d_ncoord;
    // the multipole and fused passes run the table path's chunked items
    const bool chunked = (mode & 1) != 0;
    if (chunked) {
        p.cinfo = g->d_cinfo;
        p.part = g->d_part;
        p.chunk_ctr = g->d_chunk_ctr;
        if (g->n_chunk_ctrs > 0)
            OT_CUDA(cudaMemsetAsync(g->d_chunk_ctr, 0, static_cast<size_t>(g->n_chunk_ctrs) * sizeof(int), s));
    }
    p.items = chunked ? g->d_itemsc_fwd[mode] : g->d_items_fwd[mode];
    p.n_items = chunked ? g->n_itemsc_fwd[mode] : g->n_items_fwd[mode];
    OT_CUDA(cudaMemsetAsync(g->d_counters, 0, sizeof(int), s));
    OT_CUDA(launch_forward_com(p, mode, g->wpb, grid_blocks(g, g->maxb_com_fwd[mode][g->wpb]), s));
    return OT_OK;
}

static ot_status enqueue_backward_com(ot_grid* g, const double* Lbar, const double* C, double* Mbar, double* mbar,
                                      cudaStream_t s) {
    const int mode = (Mbar ? 1 : 0) | (mbar ? 2 : 0);
    if (mode == 0) return OT_OK;
    const bool scatter = !g->deterministic && mbar != nullptr;
    PrepParams pp;
    std::memset(&pp, 0, sizeof(pp));
    pp.src = Lbar;
    pp.dst = g->d_Lrbar;
    pp.nodes = g->d_all;
    pp.n_list = g->n;
    pp.ninfo = g->d_ninfo;
    for (int l = 0; l < MAXLEV; ++l) pp.hinv[l] = g->hinv[l];
    OT_CUDA(launch_prescale_adjoint(pp, s));
    if (Mbar) OT_CUDA(cudaMemsetAsync(Mbar, 0, static_cast<size_t>(g->n) * NCOMP * NCELL * sizeof(double), s));
    if (mbar) OT_CUDA(cudaMemsetAsync(mbar, 0, static_cast<size_t>(g->n) * NCELL * sizeof(double), s));
    AdjParams p;
    std::memset(&p, 0, sizeof(p));
    p.counter = g->d_counters + 1;
    p.nbr = g->d_nbr;
    p.vnbr = g->d_vnbr;
    p.ninfo = g->d_ninfo;
    p.vinfo = g->d_vinfo;
    p.Dt = g->d_Dt;
    p.L = g->Lh;
    p.Lrbar = g->d_Lrbar;
    p.Mbar = Mbar;
    p.mbar = mbar;
    p.vbar = g->d_vbar;
    p.n_nodes = g->n;
    p.status = g->d_status;
    p.child_of = g->d_child_of;
    p.Dv = g->d_Dv;
    com_scales(g, p.hinv, p.hreal);
    p.C = C;
    p.ncoord = g->d_ncoord;
    p.vcoord = g->d_vcoord;
    int kmode = mode;
    // the multipole gathers run the table path's chunked items (long sources
    // as list chunks, combined in chunk order)
    if (mode & 1) {
        p.cinfo = g->d_cinfo_adj;
        p.part = g->d_part;
        p.chunk_ctr = g->d_chunk_ctr;
        if (g->n_chunk_ctrs_adj > 0)
            OT_CUDA(cudaMemsetAsync(g->d_chunk_ctr, 0, static_cast<size_t>(g->n_chunk_ctrs_adj) * sizeof(int), s));
    }
    if (scatter) {
        // one launch: multipole gather items (if Mbar) and point-mass items by target
        const int k = (mode & 1) ? 1 : 0;
        p.items = k ? g->d_itemsc_adj_fast1 : g->d_items_adj_fast[0];
        p.n_items = k ? g->n_itemsc_adj_fast1 : g->n_items_adj_fast[0];
        kmode = k ? 5 : 4;
    } else {
        p.items = (mode & 1) ? g->d_itemsc_adj[mode] : g->d_items_adj[mode];
        p.n_items = (mode & 1) ? g->n_itemsc_adj[mode] : g->n_items_adj[mode];
    }
    OT_CUDA(cudaMemsetAsync(g->d_counters + 1, 0, sizeof(int), s));
    OT_CUDA(launch_adjoint_com(p, kmode, g->wpb, grid_blocks(g, g->maxb_com_adj[kmode][g->wpb]), s));
    if (!scatter && mbar && g->vmap_rows > 0)
        OT_CUDA(launch_restrict_virtual(g->d_vbar, g->d_vmap, g->vmap_rows, mbar, s));
    return OT_OK;
}

// Multipole pass with the reduced-moment scratch supplied by the caller
// (the allocation-free entry point passes its static device array here).
// The scratch covers the node-index span of the non-leaf sub-grids only;
// nothing on this path allocates memory.
ot_status otk_set_error(ot_status code, const char* msg) { return fail(code, "%s", msg); }
bool otk_grid_live(const ot_grid* g) { return grid_live(g); }

ot_status otk_multipole_with_scratch(ot_grid* g, const double* M, double* L, double* Lc, double* scratch,
                                     size_t scratch_doubles, cudaStream_t s) {
    if (!g) return fail(OT_EINVAL, "grid is NULL");
    if (!grid_live(g)) return fail(OT_EINVAL, "grid handle is not live (destroyed or never created)");
    if (!M || !aligned16(M)) return fail(OT_EINVAL, "M is NULL or not 16-byte aligned");
    if (!L || !aligned16(L)) return fail(OT_EINVAL, "L is NULL or not 16-byte aligned");
    if (Lc && !aligned16(Lc)) return fail(OT_EINVAL, "Lc is not 16-byte aligned");
    int dev = -1;
    OT_CUDA(cudaGetDevice(&dev));
    if (dev != g->device) return fail(OT_EINVAL, "grid lives on device %d, current device is %d", g->device, dev);
    int lo = -1, hi = -1;
    for (int i = 0; i < g->n; ++i)
        if (!g->is_leaf[i]) {
            if (lo < 0) lo = i;
            hi = i;
        }
    const size_t per = static_cast<size_t>(NRED) * NCELL;
    const size_t span = (lo < 0) ? 0 : static_cast<size_t>(hi - lo + 1);
    if (span * per > scratch_doubles)
        return fail(OT_EINVAL,
                    "multipole sources span %zu sub-grids (node indices %d..%d); the static scratch holds %zu",
                    span, lo, hi, scratch_doubles / per);
    // Mhat of node i lives at scratch + (i - lo) * per; form the base address
    // as an integer so no out-of-range pointer is created on the host.
    const uintptr_t base = reinterpret_cast<uintptr_t>(scratch) - static_cast<uintptr_t>(lo < 0 ? 0 : lo) * per *
                                                                       sizeof(double);
    double* mhat = reinterpret_cast<double*>(base);
    PrepParams pp;
    std::memset(&pp, 0, sizeof(pp));
    pp.src = M;
    pp.dst = mhat;
    pp.nodes = g->d_nonleaf;
    pp.n_list = g->n_nonleaf;
    pp.ninfo = g->d_ninfo;
    for (int l = 0; l < MAXLEV; ++l) pp.hinv[l] = g->hinv[l];
    OT_CUDA(launch_prescale_moments(pp, s));
    OT_CUDA(cudaMemsetAsync(L, 0, static_cast<size_t>(g->n) * NCOMP * NCELL * sizeof(double), s));
    if (Lc) OT_CUDA(cudaMemsetAsync(Lc, 0, static_cast<size_t>(g->n) * 3 * NCELL * sizeof(double), s));
    FwdParams p = fwd_params(g, nullptr, L, Lc, 1);
    p.Mhat = mhat;
    p.items = g->d_items_fwd[1];
    p.n_items = g->n_items_fwd[1];
    OT_CUDA(cudaMemsetAsync(g->d_counters, 0, sizeof(int), s));
    OT_CUDA(launch_forward(p, 1, true, g->wpb, grid_blocks(g, g->maxb_fwd[1][g->wpb]), s));
    return OT_OK;
}

// run `body` directly, or capture it once into a graph keyed by `key` and replay
template <class F>
static ot_status run_graphed(ot_grid* g, const GraphKey& key, cudaStream_t s, F body) {
    if (!g->use_graph || g->schedule != OT_SCHED_PERSISTENT) return body(s);
    auto it = g->graphs.find(key);
    if (it == g->graphs.end()) {
        if (g->graphs.size() >= 16) {
            cudaGraphExecDestroy(g->graphs.begin()->second);
            g->graph_kernels.erase(g->graphs.begin()->first);
            g->graphs.erase(g->graphs.begin());
        }
        OT_CUDA(cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal));
        const long long before = launch_count_thread();
        ot_status st = body(g->cap_stream);
        // the captured kernels are not launches yet: each replay counts them
        const long long recorded = launch_count_thread() - before;
        launch_count_adjust(-recorded);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(g->cap_stream, &graph);
        if (st != OT_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) return fail(OT_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return fail(OT_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
        it = g->graphs.emplace(key, exec).first;
        g->graph_kernels[key] = recorded;
    }
    OT_CUDA(cudaGraphLaunch(it->second, s));
    launch_count_adjust(g->graph_kernels[key]);
    return OT_OK;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

#define GUARD_BEGIN try {
#define GUARD_END                                                           \
    }                                                                       \
    catch (const std::bad_alloc&) {                                         \
        return fail(OT_ENOMEM, "host allocation failed");                   \
    }                                                                       \
    catch (...) {                                                           \
        return fail(OT_EINVAL, "unexpected host exception");                \
    }

#define CHECK_PTR(p, name)                                                          \
    do {                                                                            \
        if ((p) == nullptr) return fail(OT_EINVAL, "%s is NULL", name);             \
        if (!aligned16(p)) return fail(OT_EINVAL, "%s is not 16-byte aligned", name); \
    } while (0)

extern "C" {

const char* ot_last_error(void) { return g_last_error.c_str(); }

ot_status ot_grid_create(const ot_grid_desc* desc, void* stream, ot_grid** out) {
    GUARD_BEGIN
    if (!out) return fail(OT_EINVAL, "out is NULL");
    *out = nullptr;
    if (!desc) return fail(OT_EINVAL, "desc is NULL");
    if (desc->n_subgrids <= 0) return fail(OT_EINVAL, "n_subgrids must be positive");
    if (!desc->level || !desc->coord || !desc->is_leaf) return fail(OT_EINVAL, "desc arrays must not be NULL");
    if (!(desc->h0 > 0.0) || !std::isfinite(desc->h0)) return fail(OT_EINVAL, "h0 must be positive and finite");
    if (desc->stencil_c != 0 && desc->stencil_c != 12)
        return fail(OT_ENOTSUP, "stencil_c %d not supported (only 12, theta = 0.5)", desc->stencil_c);
    if (desc->flags != OT_GEOMETRIC_CENTRES) return fail(OT_ENOTSUP, "only geometric expansion centres are built");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ot_grid* g = new ot_grid();
    cudaError_t e = cudaGetDevice(&g->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete g;
        return fail(OT_ECUDA, "device query failed: %s", cudaGetErrorString(e));
    }
    ot_status st = build_grid(g, desc, s);
    if (st == OT_OK) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = fail(OT_ECUDA, "upload failed: %s", cudaGetErrorString(e));
    }
    if (st != OT_OK) {
        delete g;
        return st;
    }
    g->info.schedule = g->schedule;
    g->info.warps_per_block = g->wpb;
    g->info.blocks_per_sm = g->bps;
    g->info.graphs_enabled = g->use_graph;
    {
        std::lock_guard<std::mutex> lk(g_handles_mu);
        g_handles.insert(g);
    }
    *out = g;
    return OT_OK;
    GUARD_END
}

ot_status ot_grid_destroy(ot_grid* grid) {
    GUARD_BEGIN
    if (!grid) return OT_OK;
    {
        std::lock_guard<std::mutex> lk(g_handles_mu);
        if (!g_handles.erase(grid)) return fail(OT_EINVAL, "grid handle is not live (destroyed or never created)");
    }
    cudaDeviceSynchronize();
    delete grid;
    return OT_OK;
    GUARD_END
}

ot_status ot_grid_info(const ot_grid* grid, ot_grid_info_t* info) {
    if (!grid || !info) return fail(OT_EINVAL, "grid and info must not be NULL");
    if (!grid_live(grid)) return fail(OT_EINVAL, "grid handle is not live (destroyed or never created)");
    *info = grid->info;
    return OT_OK;
}

ot_status ot_set_schedule(ot_grid* g, int32_t schedule, int32_t warps_per_block, int32_t blocks_per_sm,
                          int32_t use_graph) {
    GUARD_BEGIN
    if (!g) return fail(OT_EINVAL, "grid is NULL");
    if (!grid_live(g)) return fail(OT_EINVAL, "grid handle is not live (destroyed or never created)");
    if (schedule != OT_SCHED_PERSISTENT && schedule != OT_SCHED_PER_SUBGRID)
        return fail(OT_EINVAL, "unknown schedule %d", schedule);
    if (warps_per_block != 2 && warps_per_block != 4 && warps_per_block != 8)
        return fail(OT_EINVAL, "warps_per_block must be 2, 4 or 8");
    if (blocks_per_sm < 0 || blocks_per_sm > 16) return fail(OT_EINVAL, "blocks_per_sm must be in [0, 16]");
    if (use_graph != 0 && use_graph != 1) return fail(OT_EINVAL, "use_graph must be 0 or 1");
    if (g->wpb != warps_per_block || g->bps != blocks_per_sm || g->schedule != schedule) {
        for (auto& kv : g->graphs) cudaGraphExecDestroy(kv.second);
        g->graphs.clear();
        g->graph_kernels.clear();
    }
    g->schedule = schedule;
    g->wpb = warps_per_block;
    g->bps = blocks_per_sm;
    g->use_graph = use_graph;
    g->info.schedule = schedule;
    g->info.warps_per_block = warps_per_block;
    g->info.blocks_per_sm = blocks_per_sm;
    g->info.graphs_enabled = use_graph;
    return OT_OK;
    GUARD_END
}

// ---------------------------------------------------------------------------
// completion-notification study: many small per-sub-grid launches whose
// completions reach the host by different mechanisms
// ---------------------------------------------------------------------------

namespace {

using Clock = std::chrono::steady_clock;

struct CompletionSlot {
    Clock::time_point submitted;
    Clock::time_point done;
    std::atomic<int> flag{0};
    std::atomic<int>* counter = nullptr;
};

void CUDART_CB host_completion(void* arg) {    // runs on a CUDA runtime thread: no CUDA calls
    CompletionSlot* s = static_cast<CompletionSlot*>(arg);
    s->done = Clock::now();
    s->flag.store(1, std::memory_order_release);
    s->counter->fetch_add(1, std::memory_order_acq_rel);
}

}  // namespace

ot_status ot_completion_study(ot_grid* g, const double* M, const double* m, double* L, double* Lc, int32_t mechanism,
                              int32_t n_streams, double timeout_s, ot_completion_stats* out) {
    GUARD_BEGIN
    if (!g || !out) return fail(OT_EINVAL, "grid and out must not be NULL");
    CHECK_PTR(M, "M");
    CHECK_PTR(m, "m");
    CHECK_PTR(L, "L");
    if (mechanism < 0 || mechanism > 4) return fail(OT_EINVAL, "mechanism must be 0..4");
    if (n_streams < 1 || n_streams > 128) return fail(OT_EINVAL, "n_streams must be in [1, 128]");
    if (!(timeout_s > 0.0)) return fail(OT_EINVAL, "timeout_s must be positive");
    std::memset(out, 0, sizeof(*out));
    // set-up (untimed): pre-scaled moments, zeroed outputs.  The study runs on
    // streams of its own that do not order after the caller's: work already
    // queued on this grid (its scratch, queue and chunk counters) finishes first.
    OT_CUDA(cudaDeviceSynchronize());
    std::vector<cudaStream_t> streams(n_streams, nullptr);
    for (auto& st : streams) OT_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    struct StreamGuard {
        std::vector<cudaStream_t>& v;
        ~StreamGuard() {
            for (auto st : v)
                if (st) cudaStreamDestroy(st);
        }
    } guard{streams};
    const int save_sched = g->schedule;
    g->schedule = OT_SCHED_PERSISTENT;
    ot_status st0 = enqueue_forward(g, 3, M, m, L, Lc, 0, streams[0]);    // warm-up, fills Mhat
    g->schedule = save_sched;
    if (st0 != OT_OK) return st0;
    OT_CUDA(cudaMemsetAsync(L, 0, static_cast<size_t>(g->n) * NCOMP * NCELL * sizeof(double), streams[0]));
    OT_CUDA(cudaDeviceSynchronize());
    FwdParams p = fwd_params(g, m, L, Lc, 1);
    // the per-sub-grid launches run the batched launch's chunked items (the
    // same summation order); chunk counters zeroed once, each node owns its own
    p.cinfo = g->d_cinfo;
    p.part = g->d_part;
    p.chunk_ctr = g->d_chunk_ctr;
    // and the x butterflies the warm-up built from the same M and m
    if (g->precision != 2 && g->n_slotX > 0) p.Sx = g->d_Sx;
    if (g->precision != 2 && g->use_xym && g->n_slotXz > 0) p.Sxym = g->d_Sxym;
    if (g->precision == 0 && g->n_slotM > 0) p.Sm = g->d_Sm;
    if (g->precision == 0 && g->n_slotM > 0 && g->use_xy) p.Sxy = g->d_Sxy;
    if (g->precision != 0 && g->n_slotM > 0) p.Smf = g->d_Smf;
    if (g->n_chunk_ctrs > 0) {
        OT_CUDA(cudaMemsetAsync(g->d_chunk_ctr, 0, static_cast<size_t>(g->n_chunk_ctrs) * sizeof(int), streams[0]));
        OT_CUDA(cudaStreamSynchronize(streams[0]));
    }
    const int n = g->n;
    std::vector<CompletionSlot> slots(n);
    std::atomic<int> done_count{0};
    std::vector<cudaEvent_t> events;
    if (mechanism == 2 || mechanism == 4) {
        events.resize(n, nullptr);
        for (auto& e : events) OT_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    struct EventGuard {
        std::vector<cudaEvent_t>& v;
        ~EventGuard() {
            for (auto e : v)
                if (e) cudaEventDestroy(e);
        }
    } eguard{events};
    const Clock::time_point t0 = Clock::now();
    const auto deadline = t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
    bool timed_out = false;
    long long launches = 0;
    if (mechanism == 4) {
        // a pool of host threads drains a shared queue of pending events with
        // cudaEventQuery while the launching thread keeps submitting: the
        // analogue of event polling by the task scheduler's worker threads
        const int n_workers = 4;
        std::mutex qm;
        std::deque<int> queue;
        std::atomic<bool> stop{false};
        std::atomic<int> first_error{0};
        const int dev = g->device;
        auto worker = [&]() {
            cudaSetDevice(dev);
            std::vector<int> mine, again;
            while (!stop.load(std::memory_order_acquire)) {
                {
                    std::lock_guard<std::mutex> lock(qm);
                    while (!queue.empty() && mine.size() < 64) {
                        mine.push_back(queue.front());
                        queue.pop_front();
                    }
                }
                if (mine.empty()) {
                    std::this_thread::yield();
                    continue;
                }
                for (int i : mine) {
                    const cudaError_t q = cudaEventQuery(events[i]);
                    if (q == cudaSuccess) {
                        slots[i].done = Clock::now();
                        done_count.fetch_add(1, std::memory_order_acq_rel);
                    } else if (q == cudaErrorNotReady) {
                        again.push_back(i);
                    } else {
                        int zero = 0;
                        first_error.compare_exchange_strong(zero, static_cast<int>(q));
                        slots[i].done = Clock::now();
                        done_count.fetch_add(1, std::memory_order_acq_rel);
                    }
                }
                mine.clear();
                if (!again.empty()) {
                    std::lock_guard<std::mutex> lock(qm);
                    for (int i : again) queue.push_back(i);
                    again.clear();
                }
            }
        };
        std::vector<std::thread> pool;
        for (int w = 0; w < n_workers; ++w) pool.emplace_back(worker);
        struct PoolGuard {
            std::vector<std::thread>& pool;
            std::atomic<bool>& stop;
            ~PoolGuard() {
                stop.store(true, std::memory_order_release);
                for (auto& t : pool)
                    if (t.joinable()) t.join();
            }
        } pguard{pool, stop};
        ot_status submit = OT_OK;
        for (int i = 0; i < n && submit == OT_OK; ++i) {
            cudaStream_t s = streams[i % n_streams];
            FwdParams q = p;
            q.items = g->d_itemsc_node + g->itemc_node_start[i];
            q.n_items = g->itemc_node_start[i + 1] - g->itemc_node_start[i];
            slots[i].submitted = Clock::now();
            cudaError_t e = launch_forward(q, 3, false, g->wpb, (q.n_items + g->wpb - 1) / g->wpb, s);
            if (e == cudaSuccess) e = cudaEventRecord(events[i], s);
            if (e != cudaSuccess) {
                submit = fail(OT_ECUDA, "%s", cudaGetErrorString(e));
                break;
            }
            ++launches;
            std::lock_guard<std::mutex> lock(qm);
            queue.push_back(i);
        }
        while (submit == OT_OK && done_count.load(std::memory_order_acquire) < n) {
            if (Clock::now() > deadline) {
                timed_out = true;
                break;
            }
            std::this_thread::yield();
        }
        stop.store(true, std::memory_order_release);
        for (auto& t : pool) t.join();
        if (submit != OT_OK) {
            cudaDeviceSynchronize();
            return submit;
        }
        if (first_error.load() != 0)
            return fail(OT_ECUDA, "event query: %s", cudaGetErrorString(static_cast<cudaError_t>(first_error.load())));
    } else if (mechanism == 3) {
        // one batched persistent launch over every sub-grid, one completion
        g->schedule = OT_SCHED_PERSISTENT;
        for (auto& sl : slots) sl.submitted = Clock::now();
        ot_status st = enqueue_forward(g, 3, M, m, L, Lc, 0, streams[0]);   // zeroes L itself
        g->schedule = save_sched;
        if (st != OT_OK) return st;
        launches = 1;
        cudaEvent_t ev;
        OT_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        OT_CUDA(cudaEventRecord(ev, streams[0]));
        cudaError_t q;
        while ((q = cudaEventQuery(ev)) == cudaErrorNotReady) {
            if (Clock::now() > deadline) {
                timed_out = true;
                break;
            }
        }
        const Clock::time_point t = Clock::now();
        cudaEventDestroy(ev);
        if (!timed_out && q != cudaSuccess) return fail(OT_ECUDA, "event query: %s", cudaGetErrorString(q));
        for (auto& sl : slots) sl.done = t;
    } else {
        std::vector<int> pending;
        pending.reserve(n);
        auto poll = [&]() {
            size_t w = 0;
            for (size_t k = 0; k < pending.size(); ++k) {
                const int i = pending[k];
                const cudaError_t q = cudaEventQuery(events[i]);
                if (q == cudaSuccess) {
                    slots[i].done = Clock::now();
                } else {
                    pending[w++] = i;
                }
            }
            pending.resize(w);
        };
        for (int i = 0; i < n; ++i) {
            cudaStream_t s = streams[i % n_streams];
            FwdParams q = p;
            q.items = g->d_itemsc_node + g->itemc_node_start[i];
            q.n_items = g->itemc_node_start[i + 1] - g->itemc_node_start[i];
            slots[i].counter = &done_count;
            slots[i].submitted = Clock::now();
            OT_CUDA(launch_forward(q, 3, false, g->wpb, (q.n_items + g->wpb - 1) / g->wpb, s));
            ++launches;
            if (mechanism == 0) {
                OT_CUDA(cudaStreamSynchronize(s));
                slots[i].done = Clock::now();
            } else if (mechanism == 1) {
                OT_CUDA(cudaLaunchHostFunc(s, host_completion, &slots[i]));
            } else {
                OT_CUDA(cudaEventRecord(events[i], s));
                pending.push_back(i);
                poll();                      // between submissions, like a scheduler between tasks
            }
        }
        if (mechanism == 1) {
            while (done_count.load(std::memory_order_acquire) < n) {
                if (Clock::now() > deadline) {
                    timed_out = true;
                    break;
                }
            }
        } else if (mechanism == 2) {
            while (!pending.empty()) {
                poll();
                if (Clock::now() > deadline) {
                    timed_out = true;
                    break;
                }
            }
        }
    }
    const Clock::time_point t1 = Clock::now();
    if (timed_out) {
        cudaDeviceSynchronize();             // let the queued work finish before the slots go away
        return fail(OT_ETIMEOUT, "completions did not all arrive within %.1f s", timeout_s);
    }
    double sum = 0.0, mx = 0.0;
    for (auto& sl : slots) {
        const double us = std::chrono::duration<double, std::micro>(sl.done - sl.submitted).count();
        sum += us;
        mx = std::max(mx, us);
    }
    out->wall_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    out->mean_latency_us = sum / n;
    out->max_latency_us = mx;
    out->launches = launches;
    OT_CUDA(cudaDeviceSynchronize());
    return OT_OK;
    GUARD_END
}

ot_status ot_set_precision(ot_grid* g, int32_t mode) {
    GUARD_BEGIN
    if (!g) return fail(OT_EINVAL, "grid is NULL");
    if (!grid_live(g)) return fail(OT_EINVAL, "grid handle is not live (destroyed or never created)");
    if (mode != OT_PREC_FP64 && mode != OT_PREC_DF64_POINT_MASS && mode != OT_PREC_DF64)
        return fail(OT_EINVAL, "unknown precision mode %d", mode);
    g->precision = mode;
    return OT_OK;
    GUARD_END
}

ot_status ot_set_deterministic(ot_grid* g, int32_t on) {
    GUARD_BEGIN
    if (!g) return fail(OT_EINVAL, "grid is NULL");
    if (!grid_live(g)) return fail(OT_EINVAL, "grid handle is not live (destroyed or never created)");
    if (on != 0 && on != 1) return fail(OT_EINVAL, "on must be 0 or 1");
    g->deterministic = on;
    g->info.flops_adj = on ? g->flops_adj_det : g->flops_adj_fast;
    g->info.fp64_ops_adj = on ? g->fp64_ops_adj_det : g->fp64_ops_adj_fast;
    g->info.ops_adj = on ? g->ops_adj_det : g->ops_adj_fast;
    return OT_OK;
    GUARD_END
}

ot_status ot_moments(ot_grid* g, const double* rho, double* M, double* m, void* stream) {
    GUARD_BEGIN
    if (!g) return fail(OT_EINVAL, "grid is NULL");
    if (!grid_live(g)) return fail(OT_EINVAL, "grid handle is not live (destroyed or never created)");
    CHECK_PTR(rho, "rho");
    CHECK_PTR(M, "M");
    CHECK_PTR(m, "m");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    OT_CUDA(launch_cube_moments(rho, M, m, g->d_cube, g->n_cube, g->d_ninfo, g->d_hinv, s));
    for (auto& L : g->m2m)
        OT_CUDA(launch_m2m(M, m, L.d_parents, static_cast<int>(L.parents.size()), L.d_children, g->d_ninfo,
                           g->d_hinv, s));
    return OT_OK;
    GUARD_END
}

ot_status ot_moments_backward(ot_grid* g, const double* Mbar, const double* mbar, double* rhobar, void* stream) {
    GUARD_BEGIN
    if (!g) return fail(OT_EINVAL, "grid is NULL");
    if (!grid_live(g)) return fail(OT_EINVAL, "grid handle is not live (destroyed or never created)");
    CHECK_PTR(rhobar, "rhobar");
    if (Mbar && !aligned16(Mbar)) return fail(OT_EINVAL, "Mbar is not 16-byte aligned");
    if (mbar && !aligned16(mbar)) return fail(OT_EINVAL, "mbar is not 16-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    OT_CUDA(launch_moments_adjoint_init(Mbar, mbar, g->d_Mb, g->n, s));
    for (auto it = g->m2m.rbegin(); it != g->m2m.rend(); ++it)
        OT_CUDA(launch_m2m_adjoint(g->d_Mb, it->d_parents, static_cast<int>(it->parents.size()), it->d_children,
                                   g->d_ninfo, g->d_hinv, s));
    OT_CUDA(cudaMemsetAsync(rhobar, 0, static_cast<size_t>(g->n) * NCELL * sizeof(double), s));
    OT_CUDA(launch_cube_adjoint(g->d_Mb, rhobar, g->d_cube, g->n_cube, g->d_ninfo, g->d_hinv, s));
    return OT_OK;
    GUARD_END
}

ot_status ot_l2l(ot_grid* g, double* L, void* stream) {
    GUARD_BEGIN
    if (!g) return fail(OT_EINVAL, "grid is NULL");
    if (!grid_live(g)) return fail(OT_EINVAL, "grid handle is not live (destroyed or never created)");
    CHECK_PTR(L, "L");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // m2m holds the parents deepest level first: walk it from the root down
    for (auto it = g->m2m.rbegin(); it != g->m2m.rend(); ++it)
        OT_CUDA(launch_l2l(L, it->d_parents, static_cast<int>(it->parents.size()), it->d_children, g->d_ninfo,
                           g->d_hinv, s));
    return OT_OK;
    GUARD_END
}

ot_status ot_l2l_backward(ot_grid* g, double* Lbar, void* stream) {
    GUARD_BEGIN
    if (!g) return fail(OT_EINVAL, "grid is NULL");
    if (!grid_live(g)) return fail(OT_EINVAL, "grid handle is not live (destroyed or never created)");
    CHECK_PTR(Lbar, "Lbar");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (auto& L : g->m2m)
        OT_CUDA(launch_l2l_adjoint(Lbar, L.d_parents, static_cast<int>(L.parents.size()), L.d_children, g->d_ninfo,
                                   g->d_hinv, s));
    return OT_OK;
    GUARD_END
}

ot_status ot_multipole_interactions(ot_grid* g, const double* M, const double* centres, double* L, double* Lc,
                                    void* stream) {
    GUARD_BEGIN
    if (!g) return fail(OT_EINVAL, "grid is NULL");
    if (!grid_live(g)) return fail(OT_EINVAL, "grid handle is not live (destroyed or never created)");
    if (centres) return ot_interactions_com(g, M, nullptr, centres, L, Lc, stream);
    CHECK_PTR(M, "M");
    CHECK_PTR(L, "L");
    if (Lc && !aligned16(Lc)) return fail(OT_EINVAL, "Lc is not 16-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    GraphKey key{1 + 16 * g->precision, M, nullptr, L, Lc, g->wpb, g->bps};
    return run_graphed(g, key, s, [&](cudaStream_t st) { return enqueue_forward(g, 1, M, nullptr, L, Lc, 0, st); });
    GUARD_END
}

ot_status ot_monopole_interactions(ot_grid* g, const double* m, double* L, void* stream) {
    GUARD_BEGIN
    if (!g) return fail(OT_EINVAL, "grid is NULL");
    if (!grid_live(g)) return fail(OT_EINVAL, "grid handle is not live (destroyed or never created)");
    CHECK_PTR(m, "m");
    CHECK_PTR(L, "L");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    GraphKey key{2 + 16 * g->precision, nullptr, m, L, nullptr, g->wpb, g->bps};
    return run_graphed(g, key, s, [&](cudaStream_t st) { return enqueue_forward(g, 2, nullptr, m, L, nullptr, 1, st); });
    GUARD_END
}

ot_status ot_interactions(ot_grid* g, const double* M, const double* m, double* L, double* Lc, void* stream) {
    GUARD_BEGIN
    if (!g) return fail(OT_EINVAL, "grid is NULL");
    if (!grid_live(g)) return fail(OT_EINVAL, "grid handle is not live (destroyed or never created)");
    CHECK_PTR(M, "M");
    CHECK_PTR(m, "m");
    CHECK_PTR(L, "L");
    if (Lc && !aligned16(Lc)) return fail(OT_EINVAL, "Lc is not 16-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    GraphKey key{3 + 16 * g->precision, M, m, L, Lc, g->wpb, g->bps};
    return run_graphed(g, key, s, [&](cudaStream_t st) { return enqueue_forward(g, 3, M, m, L, Lc, 0, st); });
    GUARD_END
}

ot_status ot_interactions_backward(ot_grid* g, const double* Lbar, double* Mbar, double* mbar, void* stream) {
    GUARD_BEGIN
    if (!g) return fail(OT_EINVAL, "grid is NULL");
    if (!grid_live(g)) return fail(OT_EINVAL, "grid handle is not live (destroyed or never created)");
    CHECK_PTR(Lbar, "Lbar");
    if (Mbar && !aligned16(Mbar)) return fail(OT_EINVAL, "Mbar is not 16-byte aligned");
    if (mbar && !aligned16(mbar)) return fail(OT_EINVAL, "mbar is not 16-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    GraphKey key{4 + 8 * g->deterministic + 16 * g->precision, Lbar, Mbar, mbar, nullptr, g->wpb, g->bps};
    return run_graphed(g, key, s, [&](cudaStream_t st) { return enqueue_backward(g, Lbar, Mbar, mbar, st); });
    GUARD_END
}

ot_status ot_moments_com(ot_grid* g, const double* rho, double* M, double* m, double* C, void* stream) {
    GUARD_BEGIN
    if (!g) return fail(OT_EINVAL, "grid is NULL");
    if (!grid_live(g)) return fail(OT_EINVAL, "grid handle is not live (destroyed or never created)");
    CHECK_PTR(rho, "rho");
    CHECK_PTR(M, "M");
    CHECK_PTR(m, "m");
    CHECK_PTR(C, "C");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    OT_CUDA(launch_cube_moments(rho, M, m, g->d_cube, g->n_cube, g->d_ninfo, g->d_hinv, s));
    OT_CUDA(launch_geometric_centres(C, g->d_cube, g->n_cube, g->d_ninfo, g->d_ncoord, g->h0, s));
    for (auto& L : g->m2m)
        OT_CUDA(launch_m2m_com(M, m, C, L.d_parents, static_cast<int>(L.parents.size()), L.d_children, g->d_ninfo,
                               g->d_ncoord, g->h0, s));
    return OT_OK;
    GUARD_END
}

ot_status ot_interactions_com(ot_grid* g, const double* M, const double* m, const double* C, double* L, double* Lc,
                              void* stream) {
    GUARD_BEGIN
    if (!g) return fail(OT_EINVAL, "grid is NULL");
    if (!grid_live(g)) return fail(OT_EINVAL, "grid handle is not live (destroyed or never created)");
    if (!M && !m) return fail(OT_EINVAL, "M and m are both NULL");
    if (M && !aligned16(M)) return fail(OT_EINVAL, "M is not 16-byte aligned");
    if (m && !aligned16(m)) return fail(OT_EINVAL, "m is not 16-byte aligned");
    CHECK_PTR(C, "C");
    CHECK_PTR(L, "L");
    if (Lc && !aligned16(Lc)) return fail(OT_EINVAL, "Lc is not 16-byte aligned");
    const int mode = (M ? 1 : 0) | (m ? 2 : 0);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    GraphKey key{100 + mode, M, m, L, Lc, g->wpb, g->bps, C};
    return run_graphed(g, key, s, [&](cudaStream_t st) { return enqueue_forward_com(g, mode, M, m, C, L, Lc, st); });
    GUARD_END
}

ot_status ot_interactions_backward_com(ot_grid* g, const double* Lbar, const double* C, double* Mbar, double* mbar,
                                       void* stream) {
    GUARD_BEGIN
    if (!g) return fail(OT_EINVAL, "grid is NULL");
    if (!grid_live(g)) return fail(OT_EINVAL, "grid handle is not live (destroyed or never created)");
    CHECK_PTR(Lbar, "Lbar");
    CHECK_PTR(C, "C");
    if (Mbar && !aligned16(Mbar)) return fail(OT_EINVAL, "Mbar is not 16-byte aligned");
    if (mbar && !aligned16(mbar)) return fail(OT_EINVAL, "mbar is not 16-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    GraphKey key{110 + g->deterministic, Lbar, Mbar, mbar, nullptr, g->wpb, g->bps, C};
    return run_graphed(g, key, s, [&](cudaStream_t st) { return enqueue_backward_com(g, Lbar, C, Mbar, mbar, st); });
    GUARD_END
}

ot_status ot_l2l_com(ot_grid* g, const double* C, double* L, void* stream) {
    GUARD_BEGIN
    if (!g) return fail(OT_EINVAL, "grid is NULL");
    if (!grid_live(g)) return fail(OT_EINVAL, "grid handle is not live (destroyed or never created)");
    CHECK_PTR(C, "C");
    CHECK_PTR(L, "L");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (auto it = g->m2m.rbegin(); it != g->m2m.rend(); ++it)
        OT_CUDA(launch_l2l_com(L, C, it->d_parents, static_cast<int>(it->parents.size()), it->d_children,
                               g->d_ninfo, g->d_ncoord, g->h0, s));
    return OT_OK;
    GUARD_END
}

ot_status ot_l2l_com_backward(ot_grid* g, const double* C, double* Lbar, void* stream) {
    GUARD_BEGIN
    if (!g) return fail(OT_EINVAL, "grid is NULL");
    if (!grid_live(g)) return fail(OT_EINVAL, "grid handle is not live (destroyed or never created)");
    CHECK_PTR(C, "C");
    CHECK_PTR(Lbar, "Lbar");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (auto& L : g->m2m)
        OT_CUDA(launch_l2l_com_adjoint(Lbar, C, L.d_parents, static_cast<int>(L.parents.size()), L.d_children,
                                       g->d_ninfo, g->d_ncoord, g->h0, s));
    return OT_OK;
    GUARD_END
}

ot_status ot_autotune(ot_grid* g, const double* M, const double* m, double* L, double* Lc, void* stream,
                      int32_t* best_warps, int32_t* best_blocks, double* best_ms) {
    GUARD_BEGIN
    if (!g) return fail(OT_EINVAL, "grid is NULL");
    if (!grid_live(g)) return fail(OT_EINVAL, "grid handle is not live (destroyed or never created)");
    CHECK_PTR(M, "M");
    CHECK_PTR(m, "m");
    CHECK_PTR(L, "L");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int save_sched = g->schedule, save_w = g->wpb, save_b = g->bps, save_g = g->use_graph;
    g->schedule = OT_SCHED_PERSISTENT;
    g->use_graph = 0;
    cudaEvent_t e0, e1;
    OT_CUDA(cudaEventCreate(&e0));
    OT_CUDA(cudaEventCreate(&e1));
    double best = 1e30;
    int bw = save_w, bb = save_b;
    const int ws[3] = {2, 4, 8};
    // the adjoint's m-bar output (its M-bar goes to the grid's scratch)
    double* mbar = nullptr;
    OT_CUDA(cudaMalloc(&mbar, static_cast<size_t>(g->n) * NCELL * sizeof(double)));
    struct Free {
        double* q;
        ~Free() { cudaFree(q); }
    } free_mbar{mbar};
    for (int wi = 0; wi < 3; ++wi) {
        const int w = ws[wi];
        const int maxb = std::max({g->maxb_fwd[1][w], g->maxb_fwd[2][w], g->maxb_fwd[3][w], g->maxb_adj[0][w],
                                   g->maxb_adj[1][w]});
        for (int b = 1; b <= std::min(maxb, 16); ++b) {
            g->wpb = w;
            g->bps = b;
            auto step = [&]() -> ot_status {
                ot_status st = enqueue_forward(g, 3, M, m, L, Lc, 0, s);
                if (st != OT_OK) return st;
                return enqueue_backward(g, L, g->d_Mb, mbar, s);
            };
            ot_status st = step();   // warm-up
            if (st != OT_OK) return st;
            float best_run = 1e30f;
            for (int r = 0; r < 2; ++r) {
                OT_CUDA(cudaEventRecord(e0, s));
                st = step();
                if (st != OT_OK) return st;
                OT_CUDA(cudaEventRecord(e1, s));
                OT_CUDA(cudaEventSynchronize(e1));
                float ms = 0.f;
                OT_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                best_run = std::min(best_run, ms);
            }
            if (best_run < best) {
                best = best_run;
                bw = w;
                bb = b;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    g->schedule = save_sched;
    g->use_graph = save_g;
    g->wpb = save_w;
    g->bps = save_b;
    ot_status st = ot_set_schedule(g, save_sched, bw, bb, save_g);
    if (st != OT_OK) return st;
    if (best_warps) *best_warps = bw;
    if (best_blocks) *best_blocks = bb;
    if (best_ms) *best_ms = best;
    return OT_OK;
    GUARD_END
}

ot_status ot_grid_check(ot_grid* g, void* stream) {
    GUARD_BEGIN
    if (!g) return fail(OT_EINVAL, "grid is NULL");
    if (!grid_live(g)) return fail(OT_EINVAL, "grid handle is not live (destroyed or never created)");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int h[2] = {0, 0};
    OT_CUDA(cudaMemcpyAsync(h, g->d_status, sizeof(h), cudaMemcpyDeviceToHost, s));
    OT_CUDA(cudaStreamSynchronize(s));
    if (h[0] != 0) {
        OT_CUDA(cudaMemsetAsync(g->d_status, 0, sizeof(h), s));
        OT_CUDA(cudaStreamSynchronize(s));
        return fail(OT_EDEVICE, "device bounds check %d fired at work item %d", h[0], h[1]);
    }
    return OT_OK;
    GUARD_END
}

ot_status ot_fp64_fma_probe(double* out, int32_t blocks, int32_t iters, int32_t variant, void* stream) {
    GUARD_BEGIN
    CHECK_PTR(out, "out");
    if (blocks <= 0 || iters <= 0) return fail(OT_EINVAL, "blocks and iters must be positive");
    if (variant < 0 || variant > 2) return fail(OT_EINVAL, "variant must be 0, 1 or 2");
    OT_CUDA(launch_fp64_probe(out, blocks, iters, variant, static_cast<cudaStream_t>(stream)));
    return OT_OK;
    GUARD_END
}

ot_status ot_launch_count(int64_t* out) {
    if (!out) return fail(OT_EINVAL, "out is NULL");
    *out = launch_count_total();
    return OT_OK;
}

}  // extern "C"
