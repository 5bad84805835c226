/*
 * ot_oracle.c -- plain, slow CPU FP64 oracle of the FMM cell-interaction passes.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path links,
 * loads or calls this file; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg do.  It shares no code, table or constant with
 * the CUDA library.
 *
 * The paper (Sec. 2.1) states that the gravity solver is a fast multipole
 * method on an adaptive octree whose nodes carry 8x8x8 sub-grids, and (Sec. 2.2.1)
 * that every kernel works on one sub-grid plus its ghost layers; all runs are
 * FP64 (Sec. 4.1.1).  It gives no formulas for the interactions, so every
 * formula below follows the reading fixed once for this project:
 *
 *   G(R) = -1/|R| (G = 1).  Moments M_B[K] = int rho (y - X_B)^K dy (raw,
 *   K an exponent triple, |K| <= 3, 20 unique components).  Taylor
 *   coefficients L_A[J] = d^J Phi(X_A).  Truncation |J| + |I| <= 3:
 *       L_A[J] = sum_B sum_{m=0}^{3-|J|} ((-1)^m / m!) sum_{i in {x,y,z}^m}
 *                M_B[i] D[J u i](X_A - X_B),           D[K] = d^K G.
 *   Opening rule (theta = 0.5 with the cell circumradius): two cells of one
 *   level at integer offset o are well separated iff |o|^2 > 12.  A pair is
 *   "far" at level l >= 1 iff it is well separated and its parents are not
 *   (|floor((p + o)/2)|^2 <= 12, p = target cell parity); at level 0 iff it is
 *   well separated.  "Near" pairs (0 < |o|^2 <= 12) are evaluated for leaf
 *   targets only.
 *   Source classes: a cell of a non-leaf node is a multipole source (pass 1);
 *   a cell of a leaf node is a point mass (pass 2); a position not covered by
 *   a node of the target's level but covered by a coarser leaf is a virtual
 *   descendant of that leaf holding 8^-d of its cell mass (pass 2); anything
 *   else (outside the domain, no data) contributes nothing.
 *   Angular-momentum correction (multipole pass, non-leaf targets only):
 *       Lc_A[i] = -(1/6) sum_B sum_{jkl} (M3_B - (m_B/m_A) M3_A)[jkl] D[ijkl].
 *
 * Every loop below runs over full index tuples, exactly as the sums are
 * written, with no blocking or reordering.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NCOMP 20
#define NCOMP4 35
#define NCELL 512

/* ------------------------------------------------------------------------ */
/* multi-index tables                                                        */
/* ------------------------------------------------------------------------ */

static const int RANK_OFF[6] = {0, 1, 4, 10, 20, 35};
static int comp_rank[NCOMP4];
static int comp_idx[NCOMP4][4];     /* sorted index tuple */
static int comp_exp[NCOMP4][3];     /* exponent triple   */
static int exp_comp[5][5][5];       /* exponent triple -> component */
static int tables_ready = 0;

static void build_tables(void) {
    if (tables_ready) return;
    int c = 0;
    for (int k = 0; k <= 4; k++) {
        int i[4] = {0, 0, 0, 0};
        /* nondecreasing tuples of length k over {0,1,2}, lexicographic */
        int total = 1;
        for (int t = 0; t < k; t++) total *= 3;
        for (int code = 0; code < total; code++) {
            int v = code, ok = 1;
            for (int t = k - 1; t >= 0; t--) { i[t] = v % 3; v /= 3; }
            for (int t = 1; t < k; t++) if (i[t] < i[t - 1]) ok = 0;
            if (!ok) continue;
            comp_rank[c] = k;
            int e[3] = {0, 0, 0};
            for (int t = 0; t < k; t++) { comp_idx[c][t] = i[t]; e[i[t]]++; }
            comp_exp[c][0] = e[0]; comp_exp[c][1] = e[1]; comp_exp[c][2] = e[2];
            exp_comp[e[0]][e[1]][e[2]] = c;
            c++;
        }
    }
    tables_ready = 1;
}

/* component of the symmetric tensor addressed by an arbitrary index tuple */
static int comp_of(const int* idx, int k) {
    int e[3] = {0, 0, 0};
    for (int t = 0; t < k; t++) e[idx[t]]++;
    return exp_comp[e[0]][e[1]][e[2]];
}

int oracle_comp_exponents(int c, int* e) {
    build_tables();
    if (c < 0 || c >= NCOMP4) return -1;
    e[0] = comp_exp[c][0]; e[1] = comp_exp[c][1]; e[2] = comp_exp[c][2];
    return comp_rank[c];
}

/* ------------------------------------------------------------------------ */
/* derivatives of G = -1/r                                                   */
/* ------------------------------------------------------------------------ */

/* d^k G / dx_{i1}..dx_{ik} = sum over partial pairings of the k indices of
 * g_{k - #pairs} * prod(delta over pairs) * prod(R over unpaired), with
 * g_0 = -1/r and g_{k} = -(2k - 1) g_{k-1} / r^2 (so d_j g_k = g_{k+1} x_j). */
static double pairing_sum(const int* idx, int k, int pos, unsigned used, int npairs,
                          double prod, const double* R, const double* g) {
    while (pos < k && ((used >> pos) & 1u)) pos++;
    if (pos == k) return g[k - npairs] * prod;
    double s = pairing_sum(idx, k, pos + 1, used | (1u << pos), npairs, prod * R[idx[pos]], R, g);
    for (int q = pos + 1; q < k; q++) {
        if ((used >> q) & 1u) continue;
        if (idx[q] == idx[pos])
            s += pairing_sum(idx, k, pos + 1, used | (1u << pos) | (1u << q), npairs + 1, prod, R, g);
    }
    return s;
}

void oracle_D(const double* R, double* D) {
    build_tables();
    double r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
    double r = sqrt(r2);
    double g[5];
    g[0] = -1.0 / r;
    for (int k = 1; k <= 4; k++) g[k] = -(2.0 * k - 1.0) * g[k - 1] / r2;
    for (int c = 0; c < NCOMP4; c++)
        D[c] = pairing_sum(comp_idx[c], comp_rank[c], 0, 0u, 0, 1.0, R, g);
}

/* Magnitudes of every derivative's terms: the same pairing sum with each
 * term |g_{k - #pairs}| * prod |R| * prod delta taken in absolute value.
 * The passes' S sums treat each derivative as one exact number; a
 * derivative is itself a sum of these terms, and any way of evaluating it
 * rounds by a few units of their magnitude sum, which is the only non-zero
 * scale where the terms cancel to exactly zero.  The passes accumulate
 * SD = sum over the contraction's terms of |coefficient * moment| * Dabs. */
void oracle_D_abs(const double* R, double* Dabs) {
    build_tables();
    double r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
    double r = sqrt(r2);
    double g[5], Ra[3] = {fabs(R[0]), fabs(R[1]), fabs(R[2])};
    g[0] = 1.0 / r;
    for (int k = 1; k <= 4; k++) g[k] = (2.0 * k - 1.0) * g[k - 1] / r2;
    for (int c = 0; c < NCOMP4; c++)
        Dabs[c] = pairing_sum(comp_idx[c], comp_rank[c], 0, 0u, 0, 1.0, Ra, g);
}

/* ------------------------------------------------------------------------ */
/* tree lookup                                                               */
/* ------------------------------------------------------------------------ */

typedef struct {
    int n;
    const int* level;
    const int* coord;
    const uint8_t* is_leaf;
    double h0;
    uint64_t* keys;      /* sorted */
    int* order;          /* node index of each sorted key */
    int max_level;
} otree;

/* A key that is unique over levels 0..21 for 0 <= x, y, z < 2^l: the level's
 * own bit 3l above the coordinates' 3l bits. */
static uint64_t node_key(int l, long x, long y, long z) {
    return ((uint64_t)1 << (3 * l)) | ((uint64_t)x << (2 * l)) | ((uint64_t)y << l) | (uint64_t)z;
}

static otree* key_sort_tree;
static int key_cmp(const void* a, const void* b) {
    int ia = *(const int*)a, ib = *(const int*)b;
    uint64_t ka = node_key(key_sort_tree->level[ia], key_sort_tree->coord[3 * ia],
                           key_sort_tree->coord[3 * ia + 1], key_sort_tree->coord[3 * ia + 2]);
    uint64_t kb = node_key(key_sort_tree->level[ib], key_sort_tree->coord[3 * ib],
                           key_sort_tree->coord[3 * ib + 1], key_sort_tree->coord[3 * ib + 2]);
    return ka < kb ? -1 : (ka > kb ? 1 : 0);
}

static int tree_init(otree* t, int n, const int* level, const int* coord, const uint8_t* is_leaf, double h0) {
    build_tables();
    t->n = n; t->level = level; t->coord = coord; t->is_leaf = is_leaf; t->h0 = h0;
    t->keys = (uint64_t*)malloc(sizeof(uint64_t) * (n > 0 ? n : 1));
    t->order = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
    t->max_level = 0;
    for (int i = 0; i < n; i++) {
        t->order[i] = i;
        if (level[i] > t->max_level) t->max_level = level[i];
    }
    key_sort_tree = t;
    qsort(t->order, n, sizeof(int), key_cmp);
    for (int i = 0; i < n; i++) {
        int j = t->order[i];
        t->keys[i] = node_key(level[j], coord[3 * j], coord[3 * j + 1], coord[3 * j + 2]);
    }
    return 0;
}

static void tree_free(otree* t) { free(t->keys); free(t->order); }

static int tree_find(const otree* t, int l, long x, long y, long z) {
    if (l < 0 || x < 0 || y < 0 || z < 0) return -1;
    long s = 1L << l;
    if (x >= s || y >= s || z >= s) return -1;
    uint64_t k = node_key(l, x, y, z);
    int lo = 0, hi = t->n - 1;
    while (lo <= hi) {
        int mid = (lo + hi) / 2;
        if (t->keys[mid] == k) return t->order[mid];
        if (t->keys[mid] < k) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

static long floordiv(long a, long b) { long q = a / b; if ((a % b != 0) && ((a < 0) != (b < 0))) q--; return q; }

/* Source cell at level-l global cell position q.
 * returns 0: nothing, 1: multipole cell, 2: leaf cell, 3: virtual descendant. */
static int source_lookup(const otree* t, int l, const long* q, int* node, int* cell, double* scale) {
    long s = 8L << l;
    for (int a = 0; a < 3; a++) if (q[a] < 0 || q[a] >= s) return 0;
    int idx = tree_find(t, l, q[0] >> 3, q[1] >> 3, q[2] >> 3);
    if (idx >= 0) {
        *node = idx;
        *cell = (int)((q[0] & 7) + 8 * (q[1] & 7) + 64 * (q[2] & 7));
        *scale = 1.0;
        return t->is_leaf[idx] ? 2 : 1;
    }
    for (int d = 1; d <= l; d++) {
        idx = tree_find(t, l - d, q[0] >> (3 + d), q[1] >> (3 + d), q[2] >> (3 + d));
        if (idx < 0) continue;
        if (!t->is_leaf[idx]) return 0;
        *node = idx;
        *cell = (int)(((q[0] >> d) & 7) + 8 * ((q[1] >> d) & 7) + 64 * ((q[2] >> d) & 7));
        *scale = pow(0.125, d);
        return 3;
    }
    return 0;
}

/* pair selection: returns 1 if offset o is in the stencil of a target cell of
 * level l, global position g (parity p = g mod 2), leaf flag leafT */
static int pair_selected(int l, const long* g, const int* o, int leafT, int* is_far) {
    long n2 = (long)o[0] * o[0] + (long)o[1] * o[1] + (long)o[2] * o[2];
    if (n2 == 0) return 0;
    int far;
    if (l == 0) {
        far = n2 > 12;
    } else {
        long pn2 = 0;
        for (int a = 0; a < 3; a++) {
            long op = floordiv((g[a] & 1) + o[a], 2);
            pn2 += op * op;
        }
        far = (n2 > 12) && (pn2 <= 12);
    }
    int near = n2 <= 12;
    *is_far = far;
    return far || (near && leafT);
}

/* ------------------------------------------------------------------------ */
/* moments                                                                   */
/* ------------------------------------------------------------------------ */

/* raw moments of a uniform cube of side h about its centre:
 * int_{-h/2}^{h/2} t^e dt = h^{e+1} / (2^e (e+1)) for even e, 0 for odd e. */
static double cube_axis_moment(int e, double h) {
    if (e & 1) return 0.0;
    return pow(h, e + 1) / (pow(2.0, e) * (e + 1));
}

static double binom(int n, int k) {
    double r = 1.0;
    for (int i = 1; i <= k; i++) r = r * (n - k + i) / i;
    return r;
}

/* M [n][20][512]: leaf-cube moments from rho for nodes without children,
 * exact M2M shift of the 8 children's cells otherwise. */
int oracle_moments(int n, const int* level, const int* coord, const uint8_t* is_leaf, double h0,
                   const double* rho, double* M) {
    otree t;
    tree_init(&t, n, level, coord, is_leaf, h0);
    for (int l = t.max_level; l >= 0; l--) {
        double h = h0 / pow(2.0, l);
        /* the nodes of one level are independent (each reads only the
         * finished level below and writes only its own cells) */
#pragma omp parallel for schedule(dynamic, 1)
        for (int i = 0; i < n; i++) {
            if (level[i] != l) continue;
            int nchild = 0;
            for (int b = 0; b < 8; b++)
                if (tree_find(&t, l + 1, 2L * coord[3 * i] + (b & 1), 2L * coord[3 * i + 1] + ((b >> 1) & 1),
                              2L * coord[3 * i + 2] + ((b >> 2) & 1)) >= 0) nchild++;
            for (int a = 0; a < NCELL; a++) {
                double* out = M + ((size_t)i * NCOMP) * NCELL + a;
                if (nchild < 8) {
                    for (int c = 0; c < NCOMP; c++) {
                        double v = rho[(size_t)i * NCELL + a];
                        for (int ax = 0; ax < 3; ax++) v *= cube_axis_moment(comp_exp[c][ax], h);
                        out[(size_t)c * NCELL] = v;
                    }
                    continue;
                }
                long gP[3] = {8L * coord[3 * i] + (a & 7), 8L * coord[3 * i + 1] + ((a >> 3) & 7),
                              8L * coord[3 * i + 2] + (a >> 6)};
                double acc[NCOMP];
                for (int c = 0; c < NCOMP; c++) acc[c] = 0.0;
                double hc = h / 2.0;
                for (int b = 0; b < 8; b++) {
                    int bb[3] = {b & 1, (b >> 1) & 1, (b >> 2) & 1};
                    long gc[3];
                    double d[3];
                    for (int ax = 0; ax < 3; ax++) { gc[ax] = 2 * gP[ax] + bb[ax]; d[ax] = (bb[ax] - 0.5) * hc; }
                    int cn = tree_find(&t, l + 1, gc[0] >> 3, gc[1] >> 3, gc[2] >> 3);
                    int cc = (int)((gc[0] & 7) + 8 * (gc[1] & 7) + 64 * (gc[2] & 7));
                    const double* Mc = M + ((size_t)cn * NCOMP) * NCELL + cc;
                    for (int K = 0; K < NCOMP; K++) {
                        const int* e = comp_exp[K];
                        for (int I = 0; I < NCOMP; I++) {
                            const int* f = comp_exp[I];
                            if (f[0] > e[0] || f[1] > e[1] || f[2] > e[2]) continue;
                            double term = Mc[(size_t)I * NCELL];
                            for (int ax = 0; ax < 3; ax++)
                                term *= binom(e[ax], f[ax]) * pow(d[ax], e[ax] - f[ax]);
                            acc[K] += term;
                        }
                    }
                }
                for (int c = 0; c < NCOMP; c++) out[(size_t)c * NCELL] = acc[c];
            }
        }
    }
    tree_free(&t);
    return 0;
}

/* Centre-of-mass variant: C [n][3][512] receives every cell's expansion
 * centre -- the geometric centre for a childless node's uniform cube, the
 * mass-weighted mean of the 8 children's centres otherwise (geometric if the
 * mass is zero) -- and M the moments about it (exact binomial shift of the
 * children's moments by d = C_child - C_parent). */
int oracle_moments_com(int n, const int* level, const int* coord, const uint8_t* is_leaf, double h0,
                       const double* rho, double* M, double* C) {
    otree t;
    tree_init(&t, n, level, coord, is_leaf, h0);
    for (int l = t.max_level; l >= 0; l--) {
        double h = h0 / pow(2.0, l);
        /* the nodes of one level are independent (each reads only the
         * finished level below and writes only its own cells) */
#pragma omp parallel for schedule(dynamic, 1)
        for (int i = 0; i < n; i++) {
            if (level[i] != l) continue;
            int child[8], nchild = 0;
            for (int b = 0; b < 8; b++) {
                child[b] = tree_find(&t, l + 1, 2L * coord[3 * i] + (b & 1), 2L * coord[3 * i + 1] + ((b >> 1) & 1),
                                     2L * coord[3 * i + 2] + ((b >> 2) & 1));
                if (child[b] >= 0) nchild++;
            }
            for (int a = 0; a < NCELL; a++) {
                long gP[3] = {8L * coord[3 * i] + (a & 7), 8L * coord[3 * i + 1] + ((a >> 3) & 7),
                              8L * coord[3 * i + 2] + (a >> 6)};
                double* out = M + ((size_t)i * NCOMP) * NCELL + a;
                double* cen = C + ((size_t)i * 3) * NCELL + a;
                if (nchild < 8) {
                    for (int ax = 0; ax < 3; ax++) cen[(size_t)ax * NCELL] = (gP[ax] + 0.5) * h;
                    for (int c = 0; c < NCOMP; c++) {
                        double v = rho[(size_t)i * NCELL + a];
                        for (int ax = 0; ax < 3; ax++) v *= cube_axis_moment(comp_exp[c][ax], h);
                        out[(size_t)c * NCELL] = v;
                    }
                    continue;
                }
                /* children cells: positions, masses, centres */
                int cn[8], cc[8];
                double mass = 0.0, wsum[3] = {0.0, 0.0, 0.0};
                for (int b = 0; b < 8; b++) {
                    long gc[3] = {2 * gP[0] + (b & 1), 2 * gP[1] + ((b >> 1) & 1), 2 * gP[2] + ((b >> 2) & 1)};
                    cn[b] = tree_find(&t, l + 1, gc[0] >> 3, gc[1] >> 3, gc[2] >> 3);
                    cc[b] = (int)((gc[0] & 7) + 8 * (gc[1] & 7) + 64 * (gc[2] & 7));
                    double mc = M[((size_t)cn[b] * NCOMP) * NCELL + cc[b]];
                    mass += mc;
                    for (int ax = 0; ax < 3; ax++) wsum[ax] += mc * C[((size_t)cn[b] * 3 + ax) * NCELL + cc[b]];
                }
                double XP[3];
                for (int ax = 0; ax < 3; ax++) XP[ax] = (mass != 0.0) ? wsum[ax] / mass : (gP[ax] + 0.5) * h;
                double acc[NCOMP];
                for (int c = 0; c < NCOMP; c++) acc[c] = 0.0;
                for (int b = 0; b < 8; b++) {
                    const double* Mc = M + (size_t)cn[b] * NCOMP * NCELL + cc[b];
                    double d[3];
                    for (int ax = 0; ax < 3; ax++) d[ax] = C[((size_t)cn[b] * 3 + ax) * NCELL + cc[b]] - XP[ax];
                    for (int K = 0; K < NCOMP; K++) {
                        const int* e = comp_exp[K];
                        for (int I = 0; I < NCOMP; I++) {
                            const int* f = comp_exp[I];
                            if (f[0] > e[0] || f[1] > e[1] || f[2] > e[2]) continue;
                            double term = Mc[(size_t)I * NCELL];
                            for (int ax = 0; ax < 3; ax++)
                                term *= binom(e[ax], f[ax]) * pow(d[ax], e[ax] - f[ax]);
                            acc[K] += term;
                        }
                    }
                }
                for (int c = 0; c < NCOMP; c++) out[(size_t)c * NCELL] = acc[c];
                for (int ax = 0; ax < 3; ax++) cen[(size_t)ax * NCELL] = XP[ax];
            }
        }
    }
    tree_free(&t);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* interaction passes                                                        */
/* ------------------------------------------------------------------------ */

/* expansion centre of a source found by source_lookup: from C for real
 * cells, the geometric centre of the virtual cell otherwise */
static void source_centre(const otree* t, int cls, int B, int cb, int l, const long* q, const double* C,
                          double* XB) {
    if (cls == 3 || !C) {
        double h = t->h0 / pow(2.0, l);
        for (int ax = 0; ax < 3; ax++) XB[ax] = (q[ax] + 0.5) * h;
        return;
    }
    for (int ax = 0; ax < 3; ax++) XB[ax] = C[((size_t)B * 3 + ax) * NCELL + cb];
}

static const double INV_FACT[4] = {1.0, 1.0, 0.5, 1.0 / 6.0};

/* Coarse leaf target next to a refined region: a leaf target cell at global
 * position g (level l) whose near source q is a cell of a refined sub-grid
 * is itself refined virtually.  Its 8 children (level l+1, each holding an
 * eighth of the cell) meet the 8 children of q as point masses one level
 * down, and the target's coefficients are the mean of its children's.
 * child_s[cs], child_R[cs][cv][3]: the source children's (node, cell) and
 * the separations X_v - X_s (geometric centres, exact in binary). */
static void refined_pairs(const otree* t, int l, const long* g, const long* q, int (*child_s)[2],
                          double (*child_R)[8][3]) {
    double hc = t->h0 / pow(2.0, l + 1);
    for (int cs = 0; cs < 8; cs++) {
        long qs[3] = {2 * q[0] + (cs & 1), 2 * q[1] + ((cs >> 1) & 1), 2 * q[2] + (cs >> 2)};
        double sc;
        /* in a 2:1-balanced tree these children are leaf cells */
        source_lookup(t, l + 1, qs, &child_s[cs][0], &child_s[cs][1], &sc);
        for (int cv = 0; cv < 8; cv++) {
            long gv[3] = {2 * g[0] + (cv & 1), 2 * g[1] + ((cv >> 1) & 1), 2 * g[2] + (cv >> 2)};
            for (int ax = 0; ax < 3; ax++) child_R[cs][cv][ax] = (double)(gv[ax] - qs[ax]) * hc;
        }
    }
}

/* One target cell of one pass.  pass 1: multipole sources (M), pass 2: point
 * masses (m).  Writes L[20] (+ Lc[3] for pass 1), S = sum of |terms|, and,
 * where SD (SDc) is not NULL, the same sums with each derivative's terms
 * expanded (oracle_D_abs). */
static long long target_pass(const otree* t, int pass, const double* M, const double* m, const double* C,
                             int T, int a, double* L, double* Lc, double* S, double* Sc, double* SD,
                             double* SDc) {
    int l = t->level[T];
    double h = t->h0 / pow(2.0, l);
    long g[3] = {8L * t->coord[3 * T] + (a & 7), 8L * t->coord[3 * T + 1] + ((a >> 3) & 7),
                 8L * t->coord[3 * T + 2] + (a >> 6)};
    int leafT = t->is_leaf[T];
    for (int c = 0; c < NCOMP; c++) { L[c] = 0.0; S[c] = 0.0; }
    for (int i = 0; i < 3; i++) { Lc[i] = 0.0; Sc[i] = 0.0; }
    if (SD) for (int c = 0; c < NCOMP; c++) SD[c] = 0.0;
    if (SDc) for (int i = 0; i < 3; i++) SDc[i] = 0.0;
    double Da[NCOMP4];
    double mA = 0.0;
    if (pass == 1) mA = M[((size_t)T * NCOMP + 0) * NCELL + a];
    long long npairs = 0;
    int o[3];
    for (o[2] = -7; o[2] <= 7; o[2]++)
        for (o[1] = -7; o[1] <= 7; o[1]++)
            for (o[0] = -7; o[0] <= 7; o[0]++) {
                int is_far;
                if (!pair_selected(l, g, o, leafT, &is_far)) continue;
                long q[3] = {g[0] + o[0], g[1] + o[1], g[2] + o[2]};
                int B, cb;
                double scale;
                int cls = source_lookup(t, l, q, &B, &cb, &scale);
                int refined = leafT && !is_far && cls == 1;
                if (pass == 1 && (cls != 1 || refined)) continue;
                if (pass == 2 && cls != 2 && cls != 3 && !refined) continue;
                if (refined) {
                    /* pass 2: the mean over the target's virtual children of the
                     * point-mass contributions of the source's children */
                    int cs_[8][2];
                    double Rc[8][8][3];
                    refined_pairs(t, l, g, q, cs_, Rc);
                    npairs += 1;   /* one stencil pair */
                    for (int cs = 0; cs < 8; cs++) {
                        double ms = m[(size_t)cs_[cs][0] * NCELL + cs_[cs][1]];
                        for (int cv = 0; cv < 8; cv++) {
                            double D[NCOMP4];
                            oracle_D(Rc[cs][cv], D);
                            if (SD) oracle_D_abs(Rc[cs][cv], Da);
                            for (int J = 0; J < NCOMP; J++) {
                                double term = 0.125 * ms * D[J];
                                L[J] += term;
                                S[J] += fabs(term);
                                if (SD) SD[J] += fabs(0.125 * ms) * Da[J];
                            }
                        }
                    }
                    continue;
                }
                double R[3] = {-o[0] * h, -o[1] * h, -o[2] * h};   /* X_A - X_B */
                if (C) {
                    double XB[3];
                    source_centre(t, cls, B, cb, l, q, C, XB);
                    for (int ax = 0; ax < 3; ax++) R[ax] = C[((size_t)T * 3 + ax) * NCELL + a] - XB[ax];
                }
                double D[NCOMP4];
                oracle_D(R, D);
                if (SD || SDc) oracle_D_abs(R, Da);
                npairs++;
                if (pass == 2) {
                    double mass = m[(size_t)B * NCELL + cb] * scale;
                    for (int J = 0; J < NCOMP; J++) {
                        double term = mass * D[J];
                        L[J] += term;
                        S[J] += fabs(term);
                        if (SD) SD[J] += fabs(mass) * Da[J];
                    }
                    continue;
                }
                const double* MB = M + (size_t)B * NCOMP * NCELL + cb;
                for (int J = 0; J < NCOMP; J++) {
                    int nJ = comp_rank[J];
                    for (int mm = 0; mm <= 3 - nJ; mm++) {
                        double cm = ((mm & 1) ? -1.0 : 1.0) * INV_FACT[mm];
                        int total = 1;
                        for (int s = 0; s < mm; s++) total *= 3;
                        for (int code = 0; code < total; code++) {
                            int it[3], full[7];
                            int v = code;
                            for (int s = 0; s < mm; s++) { it[s] = v % 3; v /= 3; }
                            for (int s = 0; s < nJ; s++) full[s] = comp_idx[J][s];
                            for (int s = 0; s < mm; s++) full[nJ + s] = it[s];
                            double cmM = cm * MB[(size_t)comp_of(it, mm) * NCELL];
                            double term = cmM * D[comp_of(full, nJ + mm)];
                            L[J] += term;
                            S[J] += fabs(term);
                            if (SD) SD[J] += fabs(cmM) * Da[comp_of(full, nJ + mm)];
                        }
                    }
                }
                if (!leafT && is_far && mA != 0.0) {
                    double mB = MB[0];
                    for (int i = 0; i < 3; i++) {
                        for (int code = 0; code < 27; code++) {
                            int it[3] = {code % 3, (code / 3) % 3, code / 9};
                            int full[4] = {i, it[0], it[1], it[2]};
                            int c3 = comp_of(it, 3);
                            double M3A = M[((size_t)T * NCOMP + c3) * NCELL + a];
                            double nB = MB[(size_t)c3 * NCELL] - (mB / mA) * M3A;
                            double d4 = D[comp_of(full, 4)];
                            double term = -(1.0 / 6.0) * nB * d4;
                            Lc[i] += term;
                            /* the term has two contributions, the source octupole and
                             * the target octupole: count both in the magnitude sum */
                            Sc[i] += fabs((1.0 / 6.0) * MB[(size_t)c3 * NCELL] * d4) +
                                     fabs((1.0 / 6.0) * (mB / mA) * M3A * d4);
                            if (SDc)
                                SDc[i] += (fabs((1.0 / 6.0) * MB[(size_t)c3 * NCELL]) +
                                           fabs((1.0 / 6.0) * (mB / mA) * M3A)) * Da[comp_of(full, 4)];
                        }
                    }
                }
            }
    return npairs;
}

/* targets: [nt][2] (node, cell) or NULL for every cell of every node in order.
 * L, S: [nt][20]; Lc, Sc: [nt][3] (pass 1 only; may be NULL). */
long long oracle_pass_scales(int n, const int* level, const int* coord, const uint8_t* is_leaf, double h0,
                             const double* M, const double* m, const double* C, int pass, int nt,
                             const int* targets, double* L, double* Lc, double* S, double* Sc, double* SD,
                             double* SDc);

long long oracle_pass(int n, const int* level, const int* coord, const uint8_t* is_leaf, double h0,
                      const double* M, const double* m, int pass, int nt, const int* targets,
                      double* L, double* Lc, double* S, double* Sc) {
    return oracle_pass_scales(n, level, coord, is_leaf, h0, M, m, NULL, pass, nt, targets, L, Lc, S, Sc, NULL,
                              NULL);
}

/* The same with expansion centres C [n][3][512] (NULL: geometric): the pair
 * set is unchanged, R = C_A - C_B. */
long long oracle_pass_centres(int n, const int* level, const int* coord, const uint8_t* is_leaf, double h0,
                              const double* M, const double* m, const double* C, int pass, int nt,
                              const int* targets, double* L, double* Lc, double* S, double* Sc) {
    return oracle_pass_scales(n, level, coord, is_leaf, h0, M, m, C, pass, nt, targets, L, Lc, S, Sc, NULL, NULL);
}

/* The same, with the expanded-derivative magnitude sums SD [nt][20] and SDc
 * [nt][3] too (either may be NULL). */
long long oracle_pass_scales(int n, const int* level, const int* coord, const uint8_t* is_leaf, double h0,
                             const double* M, const double* m, const double* C, int pass, int nt,
                             const int* targets, double* L, double* Lc, double* S, double* Sc, double* SD,
                             double* SDc) {
    otree t;
    tree_init(&t, n, level, coord, is_leaf, h0);
    if (!targets) nt = n * NCELL;
    long long total = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : total)
    for (int k = 0; k < nt; k++) {
        int T = targets ? targets[2 * k] : k / NCELL;
        int a = targets ? targets[2 * k + 1] : k % NCELL;
        double lc[3], sc[3], sdc[3];
        total += target_pass(&t, pass, M, m, C, T, a, L + (size_t)k * NCOMP, lc, S + (size_t)k * NCOMP, sc,
                             SD ? SD + (size_t)k * NCOMP : NULL, SDc ? sdc : NULL);
        if (Lc) for (int i = 0; i < 3; i++) Lc[(size_t)k * 3 + i] = lc[i];
        if (Sc) for (int i = 0; i < 3; i++) Sc[(size_t)k * 3 + i] = sc[i];
        if (SDc) for (int i = 0; i < 3; i++) SDc[(size_t)k * 3 + i] = sdc[i];
    }
    tree_free(&t);
    return total;
}

long long oracle_pass_adjoint_targets(int n, const int* level, const int* coord, const uint8_t* is_leaf,
                                      double h0, int pass, const double* Lbar, double* Mbar, double* mbar,
                                      double* Sbar, int nt, const int* targets);

/* Transposed sums of a pass: walk exactly the pairs of the forward pass and
 * scatter Lbar[A] through the transposed coefficients onto the source.
 * pass 1 -> Mbar [n][20][512] (gradient w.r.t. the stored components of M);
 * pass 2 -> mbar [n][512] (virtual descendants scatter onto their leaf).
 * Sbar (same shape, may be NULL) receives the sum of |terms|. */
int oracle_pass_adjoint(int n, const int* level, const int* coord, const uint8_t* is_leaf, double h0,
                        int pass, const double* Lbar, double* Mbar, double* mbar, double* Sbar) {
    oracle_pass_adjoint_targets(n, level, coord, is_leaf, h0, pass, Lbar, Mbar, mbar, Sbar, 0, NULL);
    return 0;
}

long long oracle_pass_adjoint_centres(int n, const int* level, const int* coord, const uint8_t* is_leaf,
                                      double h0, const double* C, int pass, const double* Lbar, double* Mbar,
                                      double* mbar, double* Sbar, int nt, const int* targets);
long long oracle_pass_adjoint_scales(int n, const int* level, const int* coord, const uint8_t* is_leaf,
                                     double h0, const double* C, int pass, const double* Lbar, double* Mbar,
                                     double* mbar, double* Sbar, double* SDbar, int nt, const int* targets);

/* Same, scattering only from the listed target cells ([nt][2] node, cell);
 * returns the number of pairs walked. */
long long oracle_pass_adjoint_targets(int n, const int* level, const int* coord, const uint8_t* is_leaf,
                                      double h0, int pass, const double* Lbar, double* Mbar, double* mbar,
                                      double* Sbar, int nt, const int* targets) {
    return oracle_pass_adjoint_centres(n, level, coord, is_leaf, h0, NULL, pass, Lbar, Mbar, mbar, Sbar, nt,
                                       targets);
}

/* The same with expansion centres C [n][3][512] held fixed (NULL: geometric):
 * the pairs are those of the forward pass, R = C_A - C_B as there. */
long long oracle_pass_adjoint_centres(int n, const int* level, const int* coord, const uint8_t* is_leaf,
                                      double h0, const double* C, int pass, const double* Lbar, double* Mbar,
                                      double* mbar, double* Sbar, int nt, const int* targets) {
    return oracle_pass_adjoint_scales(n, level, coord, is_leaf, h0, C, pass, Lbar, Mbar, mbar, Sbar, NULL, nt,
                                      targets);
}

/* The same, with SDbar (the shape of Sbar, may be NULL): the magnitude sums
 * with each derivative's terms expanded (oracle_D_abs). */
long long oracle_pass_adjoint_scales(int n, const int* level, const int* coord, const uint8_t* is_leaf,
                                     double h0, const double* C, int pass, const double* Lbar, double* Mbar,
                                     double* mbar, double* Sbar, double* SDbar, int nt, const int* targets) {
    otree t;
    long long npairs = 0;
    tree_init(&t, n, level, coord, is_leaf, h0);
    size_t nout = (pass == 1) ? (size_t)n * NCOMP * NCELL : (size_t)n * NCELL;
    if (pass == 1) memset(Mbar, 0, sizeof(double) * nout);
    else memset(mbar, 0, sizeof(double) * nout);
    if (Sbar) memset(Sbar, 0, sizeof(double) * nout);
    if (SDbar) memset(SDbar, 0, sizeof(double) * nout);
    double Da[NCOMP4];
    long total = targets ? nt : (long)n * NCELL;
    for (long k = 0; k < total; k++) {
        int T = targets ? targets[2 * k] : (int)(k / NCELL);
        int a = targets ? targets[2 * k + 1] : (int)(k % NCELL);
        int l = level[T];
        double h = h0 / pow(2.0, l);
        int leafT = is_leaf[T];
        {
            long g[3] = {8L * coord[3 * T] + (a & 7), 8L * coord[3 * T + 1] + ((a >> 3) & 7),
                         8L * coord[3 * T + 2] + (a >> 6)};
            const double* LA = Lbar + (size_t)T * NCOMP * NCELL + a;
            int o[3];
            for (o[2] = -7; o[2] <= 7; o[2]++)
                for (o[1] = -7; o[1] <= 7; o[1]++)
                    for (o[0] = -7; o[0] <= 7; o[0]++) {
                        int is_far;
                        if (!pair_selected(l, g, o, leafT, &is_far)) continue;
                        long q[3] = {g[0] + o[0], g[1] + o[1], g[2] + o[2]};
                        int B, cb;
                        double scale;
                        int cls = source_lookup(&t, l, q, &B, &cb, &scale);
                        int refined = leafT && !is_far && cls == 1;
                        if (pass == 1 && (cls != 1 || refined)) continue;
                        if (pass == 2 && cls != 2 && cls != 3 && !refined) continue;
                        if (refined) {
                            int cs_[8][2];
                            double Rc[8][8][3];
                            refined_pairs(&t, l, g, q, cs_, Rc);
                            npairs += 1;   /* one stencil pair */
                            for (int cs = 0; cs < 8; cs++) {
                                double acc = 0.0, sacc = 0.0, sdacc = 0.0;
                                for (int cv = 0; cv < 8; cv++) {
                                    double D[NCOMP4];
                                    oracle_D(Rc[cs][cv], D);
                                    if (SDbar) oracle_D_abs(Rc[cs][cv], Da);
                                    for (int J = 0; J < NCOMP; J++) {
                                        acc += 0.125 * LA[(size_t)J * NCELL] * D[J];
                                        sacc += fabs(0.125 * LA[(size_t)J * NCELL] * D[J]);
                                        if (SDbar) sdacc += fabs(0.125 * LA[(size_t)J * NCELL]) * Da[J];
                                    }
                                }
                                mbar[(size_t)cs_[cs][0] * NCELL + cs_[cs][1]] += acc;
                                if (Sbar) Sbar[(size_t)cs_[cs][0] * NCELL + cs_[cs][1]] += sacc;
                                if (SDbar) SDbar[(size_t)cs_[cs][0] * NCELL + cs_[cs][1]] += sdacc;
                            }
                            continue;
                        }
                        npairs++;
                        double R[3] = {-o[0] * h, -o[1] * h, -o[2] * h};
                        if (C) {
                            double XB[3];
                            source_centre(&t, cls, B, cb, l, q, C, XB);
                            for (int ax = 0; ax < 3; ax++) R[ax] = C[((size_t)T * 3 + ax) * NCELL + a] - XB[ax];
                        }
                        double D[NCOMP4];
                        oracle_D(R, D);
                        if (SDbar) oracle_D_abs(R, Da);
                        if (pass == 2) {
                            double acc = 0.0, sacc = 0.0, sdacc = 0.0;
                            for (int J = 0; J < NCOMP; J++) {
                                acc += LA[(size_t)J * NCELL] * D[J];
                                sacc += fabs(LA[(size_t)J * NCELL] * D[J]);
                                if (SDbar) sdacc += fabs(LA[(size_t)J * NCELL]) * Da[J];
                            }
                            mbar[(size_t)B * NCELL + cb] += scale * acc;
                            if (Sbar) Sbar[(size_t)B * NCELL + cb] += scale * sacc;
                            if (SDbar) SDbar[(size_t)B * NCELL + cb] += scale * sdacc;
                            continue;
                        }
                        double* MB = Mbar + (size_t)B * NCOMP * NCELL + cb;
                        for (int J = 0; J < NCOMP; J++) {
                            int nJ = comp_rank[J];
                            double lbar = LA[(size_t)J * NCELL];
                            for (int mm = 0; mm <= 3 - nJ; mm++) {
                                double cm = ((mm & 1) ? -1.0 : 1.0) * INV_FACT[mm];
                                int total = 1;
                                for (int s = 0; s < mm; s++) total *= 3;
                                for (int code = 0; code < total; code++) {
                                    int it[3], full[7];
                                    int v = code;
                                    for (int s = 0; s < mm; s++) { it[s] = v % 3; v /= 3; }
                                    for (int s = 0; s < nJ; s++) full[s] = comp_idx[J][s];
                                    for (int s = 0; s < mm; s++) full[nJ + s] = it[s];
                                    double term = cm * lbar * D[comp_of(full, nJ + mm)];
                                    MB[(size_t)comp_of(it, mm) * NCELL] += term;
                                    const size_t si = (size_t)B * NCOMP * NCELL + (size_t)comp_of(it, mm) * NCELL + cb;
                                    if (Sbar) Sbar[si] += fabs(term);
                                    if (SDbar) SDbar[si] += fabs(cm * lbar) * Da[comp_of(full, nJ + mm)];
                                }
                            }
                        }
                    }
        }
    }
    tree_free(&t);
    return npairs;
}

/* ------------------------------------------------------------------------ */
/* local-expansion shift and the full multilevel solve                       */
/* ------------------------------------------------------------------------ */

/* Taylor shift of a degree-3 local expansion by d:
 * Lc[J] = sum_{q=0}^{3-|J|} (1/q!) sum_{i in {x,y,z}^q} Lp[J u i] d^i */
void oracle_l2l(const double* Lp, const double* d, double* Lc) {
    build_tables();
    for (int J = 0; J < NCOMP; J++) {
        int nJ = comp_rank[J];
        double acc = 0.0;
        for (int q = 0; q <= 3 - nJ; q++) {
            int total = 1;
            for (int s = 0; s < q; s++) total *= 3;
            for (int code = 0; code < total; code++) {
                int it[3], full[7];
                int v = code;
                double dp = 1.0;
                for (int s = 0; s < q; s++) { it[s] = v % 3; v /= 3; dp *= d[it[s]]; }
                for (int s = 0; s < nJ; s++) full[s] = comp_idx[J][s];
                for (int s = 0; s < q; s++) full[nJ + s] = it[s];
                acc += INV_FACT[q] * Lp[comp_of(full, nJ + q)] * dp;
            }
        }
        Lc[J] = acc;
    }
}

/* Full solve: moments (leaf cubes + M2M), both passes at every level, L2L from
 * each parent cell down to its children, level by level from the root.
 * Ltot [n][20][512] receives the total local expansion of every cell; Stot
 * (same shape, may be NULL) the sum of |terms| behind each coefficient: the
 * passes' sums, carried down by the same shift with |d|. */
int oracle_full_solve_com(int n, const int* level, const int* coord, const uint8_t* is_leaf, double h0,
                          const double* rho, int com, double* Ltot, double* Stot);

int oracle_full_solve(int n, const int* level, const int* coord, const uint8_t* is_leaf, double h0,
                      const double* rho, double* Ltot, double* Stot) {
    return oracle_full_solve_com(n, level, coord, is_leaf, h0, rho, 0, Ltot, Stot);
}

/* com = 1: centre-of-mass expansion centres (moments, passes and the L2L
 * shifts between them); com = 0: geometric centres. */
int oracle_full_solve_com(int n, const int* level, const int* coord, const uint8_t* is_leaf, double h0,
                          const double* rho, int com, double* Ltot, double* Stot) {
    otree t;
    tree_init(&t, n, level, coord, is_leaf, h0);
    size_t nn = (size_t)n * NCOMP * NCELL;
    double* M = (double*)malloc(sizeof(double) * nn);
    double* m = (double*)malloc(sizeof(double) * (size_t)n * NCELL);
    double* L1 = (double*)malloc(sizeof(double) * (size_t)n * NCELL * NCOMP);
    double* L2 = (double*)malloc(sizeof(double) * (size_t)n * NCELL * NCOMP);
    double* S = (double*)malloc(sizeof(double) * (size_t)n * NCELL * NCOMP);
    double* S2 = (double*)malloc(sizeof(double) * (size_t)n * NCELL * NCOMP);
    double* C = com ? (double*)malloc(sizeof(double) * (size_t)n * 3 * NCELL) : NULL;
    if (com) oracle_moments_com(n, level, coord, is_leaf, h0, rho, M, C);
    else oracle_moments(n, level, coord, is_leaf, h0, rho, M);
    for (int i = 0; i < n; i++)
        for (int a = 0; a < NCELL; a++) m[(size_t)i * NCELL + a] = M[((size_t)i * NCOMP) * NCELL + a];
    oracle_pass_centres(n, level, coord, is_leaf, h0, M, m, C, 1, 0, NULL, L1, NULL, S, NULL);
    oracle_pass_centres(n, level, coord, is_leaf, h0, M, m, C, 2, 0, NULL, L2, NULL, S2, NULL);
    for (int i = 0; i < n; i++)
        for (int a = 0; a < NCELL; a++)
            for (int c = 0; c < NCOMP; c++) {
                Ltot[((size_t)i * NCOMP + c) * NCELL + a] =
                    L1[((size_t)i * NCELL + a) * NCOMP + c] + L2[((size_t)i * NCELL + a) * NCOMP + c];
                if (Stot)
                    Stot[((size_t)i * NCOMP + c) * NCELL + a] =
                        S[((size_t)i * NCELL + a) * NCOMP + c] + S2[((size_t)i * NCELL + a) * NCOMP + c];
            }
    for (int l = 1; l <= t.max_level; l++) {
        double h = h0 / pow(2.0, l);
        for (int i = 0; i < n; i++) {
            if (level[i] != l) continue;
            for (int a = 0; a < NCELL; a++) {
                long g[3] = {8L * coord[3 * i] + (a & 7), 8L * coord[3 * i + 1] + ((a >> 3) & 7),
                             8L * coord[3 * i + 2] + (a >> 6)};
                long gp[3] = {g[0] >> 1, g[1] >> 1, g[2] >> 1};
                int P = tree_find(&t, l - 1, gp[0] >> 3, gp[1] >> 3, gp[2] >> 3);
                if (P < 0) continue;
                int cp = (int)((gp[0] & 7) + 8 * (gp[1] & 7) + 64 * (gp[2] & 7));
                double Lp[NCOMP], Lc[NCOMP];
                for (int c = 0; c < NCOMP; c++) Lp[c] = Ltot[((size_t)P * NCOMP + c) * NCELL + cp];
                double d[3];
                for (int ax = 0; ax < 3; ax++)
                    d[ax] = com ? C[((size_t)i * 3 + ax) * NCELL + a] - C[((size_t)P * 3 + ax) * NCELL + cp]
                                : ((g[ax] & 1) - 0.5) * h;
                oracle_l2l(Lp, d, Lc);
                for (int c = 0; c < NCOMP; c++) Ltot[((size_t)i * NCOMP + c) * NCELL + a] += Lc[c];
                if (Stot) {
                    double Sp[NCOMP], Sc[NCOMP], ad[3] = {fabs(d[0]), fabs(d[1]), fabs(d[2])};
                    for (int c = 0; c < NCOMP; c++) Sp[c] = Stot[((size_t)P * NCOMP + c) * NCELL + cp];
                    oracle_l2l(Sp, ad, Sc);
                    for (int c = 0; c < NCOMP; c++) Stot[((size_t)i * NCOMP + c) * NCELL + a] += Sc[c];
                }
            }
        }
    }
    free(M); free(m); free(L1); free(L2); free(S); free(S2); free(C);
    tree_free(&t);
    return 0;
}

void oracle_set_threads(int k) {
#ifdef _OPENMP
    omp_set_num_threads(k);
#else
    (void)k;
#endif
}

int oracle_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
