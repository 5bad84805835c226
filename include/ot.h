/*
 * ot.h -- C ABI of the B300 FMM cell-interaction library (libotfmm.so).
 *
 * The operations are the stencil-based cell-to-cell interactions of a fast
 * multipole gravity solver on an adaptive octree whose nodes each carry an
 * 8x8x8 sub-grid of cells, every kernel working on one sub-grid plus the
 * ghost cells of its neighbours (the paper, Sec. 2.1 and Sec. 2.2.1: FMM
 * gravity solver on an octree of 8^3 sub-grids; kernels per sub-grid with
 * ghost layers).  The paper fixes FP64 (Sec. 4.1.1); it gives no formulas, so
 * the definitions below are the project's reading of the method:
 *
 *   Units G = 1, Green's function G(R) = -1/|R|.
 *   Cell moments (raw, about the geometric cell centre), 20 per cell:
 *     M[K] = int rho(y) (y - X)^K dy, |K| <= 3.
 *   Taylor coefficients of the potential at a cell centre, 20 per cell:
 *     L[J] = d^J Phi(X), |J| <= 3.
 *   Component order (both): 0; x y z; xx xy xz yy yz zz;
 *     xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz.
 *   Contraction with the symmetric n + m <= 3 truncation:
 *     L_A[J] += sum_{m <= 3-|J|} ((-1)^m/m!) sum_{i in {x,y,z}^m} M_B[i] d^{J u i} G(X_A - X_B).
 *   Opening rule theta = 0.5: cells at integer offset o are well separated iff
 *     |o|^2 > 12.  A pair is "far" at level l >= 1 when its parents are not well
 *     separated, at level 0 whenever it is well separated; "near" pairs
 *     (0 < |o|^2 <= 12) are evaluated for leaf targets only.  Per target parity
 *     there are 1253 far offsets; there are 178 near offsets.
 *   Source classes: cells of non-leaf nodes are multipole sources; cells of
 *     leaf nodes are point masses; a same-level position with no node but
 *     covered by a coarser leaf is a virtual descendant holding 8^-d of that
 *     leaf's cell mass (coarse-fine boundary); anything else is empty.
 *   Coarse leaf targets (the other side of that boundary): a leaf target's
 *     near source that is a cell of a refined node is not contracted as a
 *     multipole.  The target cell is refined virtually instead -- its 8
 *     children, an eighth of the cell each, meet the source cell's 8 children
 *     (leaf cells one level down) as point masses -- and takes the mean of
 *     its children's coefficients.  This is part of the monopole pass.
 *
 * Memory and ownership.  Every array argument is a DEVICE pointer owned by
 * the caller, 16-byte aligned, densely packed in the layout given, and must
 * stay valid until the work queued on `stream` has finished.  The library
 * owns the grid metadata, its work lists, its scratch arena and its CUDA
 * graphs; all of them live inside the ot_grid handle.
 *
 * Errors.  Every call returns OT_OK or an error code and never throws.  A
 * call returns after queueing its work on `stream` (a cudaStream_t; NULL is
 * the legacy default stream); its status covers argument checks and launch
 * errors.  Faults detected by the kernels' own bounds checks are latched in
 * a device status word that ot_grid_check() reads (it synchronizes).
 * ot_last_error() gives a message for the calling thread's last failure.
 */
#ifndef OT_H
#define OT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ot_grid ot_grid;

typedef enum {
    OT_OK = 0,
    OT_EINVAL = 1,     /* bad argument: null, misaligned, out of range, bad tree */
    OT_ENOMEM = 2,     /* device or host allocation failed                      */
    OT_ECUDA = 3,      /* a CUDA runtime call failed                            */
    OT_ETIMEOUT = 4,   /* a bounded device-side wait ran out                    */
    OT_ESTATE = 5,     /* handle in a bad state (e.g. a latched device fault)   */
    OT_ENOTSUP = 6,    /* valid request this library does not implement         */
    OT_EDEVICE = 7     /* a kernel's own bounds check fired                      */
} ot_status;

/* Grid description.  Node i sits at `level[i]` with integer position
 * `coord[3i..3i+2]` in [0, 2^level); its cell (a,b,c) has flat index
 * a + 8b + 64c and centre (8*coord + (a,b,c) + 0.5) * h0 / 2^level.
 * `is_leaf[i]` selects the source class of its cells (see above).
 * (level, coord) pairs must be unique; level <= 20.  Host pointers, read
 * during ot_grid_create only. */
typedef struct {
    int32_t n_subgrids;
    const int32_t* level;      /* [n]    */
    const int32_t* coord;      /* [n][3] */
    const uint8_t* is_leaf;    /* [n]    */
    double h0;                 /* cell size at level 0, > 0 */
    int32_t stencil_c;         /* opening rule |o|^2 > c; 0 or 12 (theta = 0.5) */
    uint32_t flags;            /* OT_GEOMETRIC_CENTRES (the only mode built)  */
} ot_grid_desc;

#define OT_GEOMETRIC_CENTRES 0u

/* Execution schedule of the interaction kernels. */
typedef enum {
    OT_SCHED_PERSISTENT = 0,   /* one persistent launch over a device work list */
    OT_SCHED_PER_SUBGRID = 1   /* one launch per target sub-grid (the plain path) */
} ot_schedule;

/* Summary of a grid (host struct filled by ot_grid_info). */
typedef struct {
    int32_t n_subgrids;
    int32_t n_virtual;             /* virtual descendant sub-grids seen by the adjoint */
    int32_t max_level;
    int32_t far_offsets;           /* per parity (1253 at theta = 0.5) */
    int32_t near_offsets;          /* 178 */
    int32_t root_offsets;          /* 3196 */
    int64_t pairs_multipole;       /* in-domain (target, source) pairs of each pass */
    int64_t pairs_monopole;
    int64_t pairs_virtual;         /* part of pairs_monopole with a virtual source */
    int64_t pairs_angular;         /* part of pairs_multipole with a non-leaf target */
    int64_t lanes_fwd;             /* warp lanes run by the forward pair loops of both
                                      passes, lanes with an empty source included */
    int64_t flops_fwd;             /* algorithmic FP64 flops of one forward launch over
                                      the in-domain pairs (2 per FMA, 1 per add) */
    int64_t flops_adj;             /* the same for the adjoint */
    int64_t ops_fwd;               /* FP64 instructions x lanes one forward launch
                                      executes, lanes with an empty source included */
    int64_t ops_adj;               /* the same for the adjoint */
    int32_t schedule;              /* ot_schedule in use */
    int32_t warps_per_block;       /* tile shape in use */
    int32_t blocks_per_sm;
    int32_t graphs_enabled;
    int64_t flops_fwd_com;         /* algorithmic FLOPs of ot_interactions_com (both passes, with Lc):
                                      per pair the derivative evaluation plus the contraction */
    int64_t flops_adj_com;         /* the same for ot_interactions_backward_com */
    int64_t pairs_refined;         /* near pairs of a leaf target and a cell of a refined
                                      sub-grid, evaluated through the leaf's virtual children
                                      (each counted once in pairs_monopole) */
    int64_t pairs_padded_fwd;      /* pairs the forward's lanes run, sources outside the domain
                                      included (a paired entry runs two per lane) */
    int32_t chunked_subgrids;      /* sub-grids whose multipole work items run as several
                                      list chunks (summed in chunk order by the last one) */
    int32_t reserved0;
    int64_t fp64_ops_fwd;          /* algorithmic FP64 instructions (one per FMA or add) of one
                                      forward launch over the in-domain pairs: the FP64 pipe's
                                      work (a class or +-o entry's shared by its members) */
    int64_t fp64_ops_adj;          /* the same for the adjoint in use */
    int64_t fp64_ops_fwd_multi;    /* the part of fp64_ops_fwd in the multipole pass (the
                                      launch of ot_multipole_interactions) */
    int64_t ops_fwd_multi;         /* the part of ops_fwd in the multipole pass */
    int64_t fp64_ops_adj_multi;    /* the part of fp64_ops_adj in the multipole gather (the
                                      adjoint's first launch; the rest is the point masses) */
    int64_t ops_adj_multi;         /* the part of ops_adj in the multipole gather */
} ot_grid_info_t;

/* Builds neighbour tables, stencils, the derivative table, work lists and the
 * scratch arena on the current device.  `stream` orders the uploads.  The
 * arena holds, besides per-sub-grid scratch, the tables the passes rebuild
 * each call: x butterflies of the reduced moments, L-bar and the masses
 * (0.9 MB, 0.9 MB and 57 KB per region slot), the masses' (x, y) table
 * (0.8 MB per slot in the leaves' z columns, used up to 16 GiB) and the
 * reduced moments' (x, y) table (12.8 MB per slot in the non-leaf nodes' z
 * columns, used up to 48 GiB; about 21 GB on a 9,500-sub-grid octree);
 * a table over its cap is not allocated and its classes take the
 * x-butterfly walk instead.
 * Errors: OT_EINVAL (bad description; also a tree that is not 2:1 balanced
 * in the sense the coarse-leaf rule needs: a child of a refined neighbour of
 * a leaf sub-grid that touches the leaf must itself be a leaf; also a
 * sub-grid whose halo would hold virtual descendants more than 5 levels
 * below their covering leaf; 2^22 or more sub-grids, or 2^26 or more with
 * the virtual ones the adjoint adds), OT_ENOMEM,
 * OT_ECUDA, OT_ENOTSUP (stencil_c other than 12, flags other than geometric
 * centres). */
ot_status ot_grid_create(const ot_grid_desc* desc, void* stream, ot_grid** out);

/* Frees everything the handle owns (synchronizes the device first). NULL is OK. */
ot_status ot_grid_destroy(ot_grid* grid);

ot_status ot_grid_info(const ot_grid* grid, ot_grid_info_t* info);

/* Cell moments from densities (the input preparation): rho [n][512] (cell
 * densities sampled at cell centres) -> M [n][20][512], m [n][512] (= M[:,0]).
 * Nodes with all 8 children present get the exact binomial (M2M) shift of
 * their children's moments to their own cell centres; other nodes get the
 * moments of uniform cubes (M0 = rho h^3, Mii = rho h^5/12).  M and m are
 * overwritten. */
ot_status ot_moments(ot_grid* grid, const double* rho, double* M, double* m, void* stream);

/* Adjoint of ot_moments: rhobar [n][512] (overwritten) from Mbar [n][20][512]
 * and mbar [n][512] (either may be NULL = zero). */
ot_status ot_moments_backward(ot_grid* grid, const double* Mbar, const double* mbar,
                              double* rhobar, void* stream);

/* Multipole pass: every target cell of every node gathers the multipole
 * sources of its stencil.  M [n][20][512] in; L [n][20][512] OVERWRITTEN;
 * Lc [n][3][512] (angular-momentum correction, non-leaf targets with
 * non-zero mass, multipole sources only; may be NULL) overwritten:
 *   Lc_A[i] = -(1/6) sum_B sum_{jkl} (M3_B - (m_B/m_A) M3_A)[jkl] d^{ijkl} G.
 * `centres` NULL: geometric cell centres.  Non-NULL: explicit expansion
 * centres [n][3][512], the same as ot_interactions_com(grid, M, NULL,
 * centres, L, Lc, stream). */
ot_status ot_multipole_interactions(ot_grid* grid, const double* M, const double* centres,
                                    double* L, double* Lc, void* stream);

/* Monopole pass: every target cell gathers the point-mass sources of its
 * stencil (leaf cells, virtual descendants of coarser leaves).  m [n][512] in;
 * L [n][20][512] is ACCUMULATED into (call after the multipole pass, or zero it). */
ot_status ot_monopole_interactions(ot_grid* grid, const double* m, double* L, void* stream);

/* Both passes as batched launches (the schedule set by ot_set_schedule;
 * replayed from a CUDA graph when graphs are enabled): one launch holding
 * both passes' work items, or the multipole pass then the monopole pass as
 * two launches when the point masses read the per-call (x, y) table or the
 * contractions run in double-float (the same sums either way, up to the
 * order of the two passes' additions into L).  L overwritten with the sum
 * of both passes; Lc as above (may be NULL). */
ot_status ot_interactions(ot_grid* grid, const double* M, const double* m,
                          double* L, double* Lc, void* stream);

/* Adjoint of both passes with respect to their sources (Lc not included):
 *   Mbar = (d L / d M)^T Lbar  for the multipole pass  [n][20][512] overwritten,
 *   mbar = (d L / d m)^T Lbar  for the monopole pass   [n][512]     overwritten,
 * with virtual descendants' gradients restricted onto their coarse leaf.
 * Mbar comes from the transposed stencil (a gather over sources).  mbar comes
 * by default from the target-ordered walk with atomic adds into mbar (fewer
 * FP64 operations; summation order, hence the last bits, vary from run to
 * run); after ot_set_deterministic(grid, 1) it also comes from the gather
 * (fixed order, bit-reproducible).  Under the persistent schedule the gather
 * and the target-ordered walk are two launches.  Stores nothing from the
 * forward pass.  Mbar / mbar may be NULL to skip that half. */
ot_status ot_interactions_backward(ot_grid* grid, const double* Lbar, double* Mbar,
                                   double* mbar, void* stream);

/* Local-expansion down-pass (L2L) completing the multilevel solve, in place
 * on L [n][20][512]: level by level from the root, every cell of a sub-grid
 * whose parent is present adds its parent cell's expansion shifted to its own
 * centre (degree-3 Taylor shift, d = +-h/2 per axis):
 *   L_child[J] += sum_{|J|+|I| <= 3} L_parent[J+I] d^I / I!.
 * After moments, both passes and this call, L[:,0] of a leaf cell is the
 * potential at its centre (without the cell's self-potential) and -L[:,1:4]
 * the gravitational field. */
ot_status ot_l2l(ot_grid* grid, double* L, void* stream);

/* Adjoint of ot_l2l, in place on Lbar [n][20][512]: from the deepest level
 * up, every parent cell adds the transposed shifts of its children's Lbar. */
ot_status ot_l2l_backward(ot_grid* grid, double* Lbar, void* stream);

/* Centre-of-mass expansion centres (the octree FMM of Sec. 2.1 expands
 * every cell about its centre of mass).  Cells of non-leaf sub-grids are
 * expanded about per-cell centres C [n][3][512] (x, y, z planes; positions in
 * the units of h0); cells of leaf sub-grids are uniform cubes and stay at
 * their geometric centres, as do virtual descendants -- C is never read for
 * leaf sub-grids.  The pair set of both passes is unchanged.  A pair whose
 * two centres are geometric (a leaf target and a point-mass source) sits at
 * an integer offset and uses the derivative table; every other pair
 * evaluates the derivatives of G at its own R = C_A - C_B (one sqrt and one
 * division, the order 0..4 polynomials it needs).
 *
 * ot_moments_com: rho [n][512] -> M [n][20][512], m [n][512], C [n][3][512]
 * (all overwritten).  A node without all 8 children: C = geometric centre,
 * M = uniform-cube moments (as ot_moments).  A node with 8 children, from the
 * deepest level up: C = mass-weighted mean of the 8 child cells' centres
 * (the geometric centre where that mass is exactly 0), M = the children's
 * moments shifted binomially to C. */
ot_status ot_moments_com(ot_grid* grid, const double* rho, double* M, double* m, double* C,
                         void* stream);

/* Both passes (or one: M or m NULL, not both) with explicit centres C, in one
 * persistent launch (graph-replayed when graphs are enabled).  L [n][20][512]
 * OVERWRITTEN with the sum of the passes run; Lc [n][3][512] (may be NULL;
 * multipole pass only) overwritten, as in ot_multipole_interactions.  Always
 * the persistent schedule; FP64 throughout (ot_set_precision does not apply).
 * Every pair must keep |C_A - C_B| > 0, which holds for centres inside their
 * cells (any centre of mass of non-negative densities). */
ot_status ot_interactions_com(ot_grid* grid, const double* M, const double* m, const double* C,
                              double* L, double* Lc, void* stream);

/* Adjoint of ot_interactions_com with the centres held fixed (a partial
 * gradient: the dependence of C on the densities is not differentiated).
 * Mbar [n][20][512], mbar [n][512] overwritten (either may be NULL to skip).
 * As ot_interactions_backward: mbar by atomic adds from the targets by
 * default, by the fixed-order gather after ot_set_deterministic(grid, 1). */
ot_status ot_interactions_backward_com(ot_grid* grid, const double* Lbar, const double* C,
                                       double* Mbar, double* mbar, void* stream);

/* Down-pass with explicit centres, in place on L: d = X_child - X_parent per
 * child cell, X the centre as above (C for non-leaf sub-grids, geometric for
 * leaf sub-grids); otherwise as ot_l2l.  And its adjoint with C fixed. */
ot_status ot_l2l_com(ot_grid* grid, const double* C, double* L, void* stream);
ot_status ot_l2l_com_backward(ot_grid* grid, const double* C, double* Lbar, void* stream);

/* Arithmetic of the contractions of the table path (ot_interactions_com
 * stays FP64).
 * OT_PREC_FP64 (default): FP64 FMAs throughout.
 * OT_PREC_DF64_POINT_MASS: point-mass pairs are contracted in double-float
 *   arithmetic on the FP32 pipe -- every value an unevaluated sum hi + lo of
 *   two FP32 numbers (48-bit significand), products split exactly with FMAs,
 *   accumulated by two-sums with renormalization -- and the partial sums move
 *   into FP64 accumulators before any of them holds more than 64 products, so
 *   each coefficient stays within ~7e-13 of the sum of |terms| of its FP64
 *   value.  Leaf targets without prebuilt x tables (leaves bordering a
 *   coarser leaf or a refined sub-grid) keep the FP64 class walk for their
 *   point-mass classes, which costs less there.
 *   Requires point masses m with |m| in [2^-100, 2^100] or m = 0 and
 *   derivative-table values in the same range (true for cell sizes within
 *   2^-10 .. 2^10 of level 0's).
 * OT_PREC_DF64: the multipole contractions too (the 70-product contraction
 *   and the angular term, with the reduced moments split into double-float
 *   pairs once per call), under the same 64-product rule and bound, and the
 *   default adjoint (persistent schedule, not deterministic): the multipole
 *   gather under the same rule, each point-mass contribution as a fresh
 *   double-float dot product added to mbar in FP64.  The same range
 *   requirement holds for the reduced moments and L-bar (scaled by h, so of
 *   the order of the mass and L-bar).  With ot_set_deterministic or the
 *   per-sub-grid schedule the adjoint stays FP64. */
#define OT_PREC_FP64 0
#define OT_PREC_DF64_POINT_MASS 1
#define OT_PREC_DF64 2
ot_status ot_set_precision(ot_grid* grid, int32_t mode);

/* 1: every adjoint result in a fixed summation order (bit-reproducible);
 * 0 (default): the point-mass adjoint uses atomic adds (faster). */
ot_status ot_set_deterministic(ot_grid* grid, int32_t on);

/* Schedule and tile shape of later calls (forward and adjoint; the plain
 * schedule launches once per target sub-grid forward and once per source
 * sub-grid in the adjoint).  warps_per_block in {2,4,8},
 * blocks_per_sm in {0 (max resident), 1..16}; use_graph 0/1. */
ot_status ot_set_schedule(ot_grid* grid, int32_t schedule, int32_t warps_per_block,
                          int32_t blocks_per_sm, int32_t use_graph);

/* Times every tile shape of the persistent schedule with CUDA events and
 * keeps the fastest: one step of the forward (both passes, on the given
 * buffers, which it overwrites) and the adjoint (reading L as L-bar, writing
 * library scratch).  A shape's blocks_per_sm is capped per kernel by its
 * resident limit, so a shape can give the adjoint more warps than the
 * forward.  Writes the chosen (warps_per_block, blocks_per_sm) and its step
 * time in ms to the outputs.  Synchronizes `stream`. */
ot_status ot_autotune(ot_grid* grid, const double* M, const double* m, double* L, double* Lc,
                      void* stream, int32_t* best_warps, int32_t* best_blocks, double* best_ms);

/* Allocation-free multipole pass.  The paper has no counterpart: this entry
 * point exists for callers that must not allocate device memory when they
 * call the kernels -- code recording a CUDA graph by stream capture (an
 * allocation is not a stream operation and breaks the capture), real-time
 * loops that forbid allocator calls after set-up, hosts whose device memory
 * is owned by another allocator.  It computes the multipole pass of
 * ot_multipole_interactions (M, L, Lc as there, centres implied NULL) with
 * the same pair set, derivative table and contractions, but not the same
 * instruction path: it runs in FP64 whatever ot_set_precision chose, on the
 * persistent schedule, without the prebuilt x-butterfly tables and without
 * splitting long work items into chunks, so its result equals
 * ot_multipole_interactions' within the parity bar (1e-12 of each
 * coefficient's sum of |terms|), not bit for bit.  Its scratch (the
 * pre-scaled, reduced source moments, 64 KiB per sub-grid) lives in one
 * static device array of OT_NOALLOC_SCRATCH_BYTES instead of the grid's
 * arena, and it calls no cudaMalloc, cudaFree or allocating library routine.
 *   - Limit: the non-leaf sub-grids' node indices must span at most
 *     OT_NOALLOC_SCRATCH_BYTES / 64 KiB = 256 consecutive indices; larger
 *     grids are rejected with OT_EINVAL and a message.
 *   - The array's device address is looked up (cudaGetSymbolAddress, with
 *     the device current) on the first call on each device, and again only
 *     if that device's context was replaced; make that first call before any
 *     stream capture.  Every device that loads the library holds the array
 *     until the process exits.
 *   - All calls share the one array, which keeps the last call's contents;
 *     each call writes every scratch entry it reads before reading it, so
 *     nothing needs clearing.  Calls whose GPU work overlaps (other streams,
 *     other grids on the same device) race on the array: serialize them.
 *   - No CUDA graph is recorded or replayed by this call. */
#define OT_NOALLOC_SCRATCH_BYTES (16u << 20)
ot_status ot_multipole_interactions_noalloc(ot_grid* grid, const double* M, double* L, double* Lc,
                                            void* stream);

/* Completion-notification study.  The paper's integration question: when a
 * task runtime launches many small per-sub-grid kernels, how does each
 * kernel's completion reach the host tasks waiting on it (Sec. 3.2: SYCL
 * host tasks versus event polling inside the scheduler)?  This runs the
 * forward interactions of every sub-grid as its own launch, round-robin over
 * `n_streams` streams, and signals each completion by
 *   0: cudaStreamSynchronize after the launch (no integration: synchronous),
 *   1: a cudaLaunchHostFunc callback (the host-task analogue),
 *   2: an event polled by the launching thread between submissions and
 *      afterwards (the event-polling analogue),
 *   3: one batched persistent launch over all sub-grids, one event,
 *   4: an event per launch, polled with cudaEventQuery by a pool of 4 host
 *      threads draining a shared queue while the launching thread keeps
 *      submitting (event polling by the scheduler's worker threads).
 * L, Lc are overwritten with the forward result.  Outputs: wall time from
 * the first submission to the last completion, mean and max latency from a
 * sub-grid's submission to its completion being seen on the host.  Host
 * waits give up after `timeout_s` with OT_ETIMEOUT.  Synchronizes the device. */
typedef struct {
    double wall_ms;
    double mean_latency_us;
    double max_latency_us;
    int64_t launches;
} ot_completion_stats;
ot_status ot_completion_study(ot_grid* grid, const double* M, const double* m, double* L, double* Lc,
                              int32_t mechanism, int32_t n_streams, double timeout_s,
                              ot_completion_stats* out);

/* Reads and clears the device status word (synchronizes `stream`): OT_OK, or
 * OT_EDEVICE with the failing work item in ot_last_error(). */
ot_status ot_grid_check(ot_grid* grid, void* stream);

/* FP64 FMA throughput probe: `blocks` x 256 threads each run `iters` rounds
 * of independent FMAs -- variant 0: 16 chains a = a*b + c; variant 1: 16
 * accumulators a_j += s * x_j; variant 2: the point-mass contraction's
 * pattern, 64 rows of 16 values staged in shared memory, each row times one
 * of 4 per-thread values accumulated into 16 sums (1024 FMAs per round; the
 * only variant whose operands arrive from shared memory, as the
 * interaction kernels' do).  FMAs per round: 16, 16, 1024.  out
 * [blocks*256] receives the results (keeps them live).  Time it with events. */
ot_status ot_fp64_fma_probe(double* out, int32_t blocks, int32_t iters, int32_t variant, void* stream);

/* Kernels this library has launched in this process so far, across all
 * grids and threads: each kernel launched directly counts once, each kernel
 * inside a replayed CUDA graph once per replay (recording a graph counts
 * nothing).  Reads a counter, no device work.  OT_EINVAL if out is NULL. */
ot_status ot_launch_count(int64_t* out);

/* Message for the calling thread's last non-OK status ("" if none). */
const char* ot_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* OT_H */
