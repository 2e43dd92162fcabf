/*
 * ASKIT oracle: a plain, slow, sequential FP64 CPU restatement of the ASKIT
 * method (March, Xiao & Biros, "ASKIT: Approximate Skeletonization
 * Kernel-Independent Treecode in High Dimensions").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * includes this file; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg load it.  It shares no code, header, table or
 * constant generator with the CUDA path.
 *
 * Every function follows one passage of the paper, cited in its comment.
 * Floating point: inputs are FP32, every computation is FP64, compiled with
 * -ffp-contract=off (no fused multiply-add), sums run in the order written.
 * Where the paper leaves a choice open, the reading taken is stated at the
 * function.
 *
 * Pinning (tests/test_oracle_*.py): each stage is checked against something
 * other than itself -- numpy's Philox for the RNG, libm/mpmath for exp,
 * brute force and numpy.lexsort for kNN, hand-built trees, brute-force set
 * algebra for node lists and sampling, scipy's pivoted QR and numpy's SVD
 * for the ID, and the direct sum for Evaluate in the cases where the paper's
 * algorithm degenerates to it.  No function here is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Counter-based RNG: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11,     */
/* "Parallel random numbers: as easy as 1, 2, 3").  Written from that       */
/* paper's definition; pinned bitwise against numpy.random.Philox.          */
/* ------------------------------------------------------------------------ */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void orc_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(M0, c0, &hi0, &lo0);
        mulhilo64(M1, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        uint64_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The n-th 64-bit word of the stream keyed (k0, k1): block n/4, lane n%4. */
static uint64_t philox_word(uint64_t k0, uint64_t k1, uint64_t c0, uint64_t n)
{
    uint64_t ctr[4] = {c0, n >> 2, 0, 0}, key[2] = {k0, k1}, out[4];
    orc_philox4x64_10(ctr, key, out);
    return out[n & 3];
}

/* ------------------------------------------------------------------------ */
/* Canonical FP64 exponential used to fill the ID's kernel matrices, so    */
/* that pivot choices do not depend on a platform's libm.  Method: Cody &  */
/* Waite range reduction a = n ln2 + r (ln2 split into a 32-bit head and a */
/* tail), degree-13 Taylor polynomial for e^r on |r| <= ln2/2 in Horner    */
/* form, then exact scaling by 2^n.  Arguments below -700 return 0.        */
/* Pinned against libm and mpmath (<= 2 ulp).                              */
/* ------------------------------------------------------------------------ */
double orc_cexp(double a)
{
    if (a < -700.0) return 0.0;
    if (a > 700.0) return INFINITY;
    const double INV_LN2 = 0x1.71547652b82fep+0;
    const double LN2_HEAD = 0x1.62e42ff000000p-1;   /* ln2 to 32 significant bits */
    const double LN2_TAIL = -0x1.718432a1b0e26p-35; /* ln2 - LN2_HEAD */
    double n = nearbyint(a * INV_LN2);
    double r = (a - n * LN2_HEAD) - n * LN2_TAIL;
    /* 1/k! for k = 13 .. 0 */
    static const double C[14] = {
        0x1.6124613a86d09p-33, 0x1.1eed8eff8d898p-29, 0x1.ae64567f544e4p-26,
        0x1.27e4fb7789f5cp-22, 0x1.71de3a556c734p-19, 0x1.a01a01a01a01ap-16,
        0x1.a01a01a01a01ap-13, 0x1.6c16c16c16c17p-10, 0x1.1111111111111p-7,
        0x1.5555555555555p-5,  0x1.5555555555555p-3,  0x1.0000000000000p-1,
        0x1.0000000000000p+0,  0x1.0000000000000p+0};
    double p = C[0];
    for (int k = 1; k < 14; ++k) p = p * r + C[k];
    return ldexp(p, (int)n);
}

/* Squared Euclidean distance (the kernel's argument), FP64 from FP32 data,
 * coordinates in ascending order, no fused multiply-add. */
static double dist2_ff(const float *x, const float *y, int d)
{
    double acc = 0.0;
    for (int k = 0; k < d; ++k) {
        double t = (double)x[k] - (double)y[k];
        acc = acc + t * t;
    }
    return acc;
}

static double dist2_df(const double *x, const float *y, int d)
{
    double acc = 0.0;
    for (int k = 0; k < d; ++k) {
        double t = x[k] - (double)y[k];
        acc = acc + t * t;
    }
    return acc;
}

/* (value, index) lexicographic order used for every tie in the method. */
static int lex_less(double a, int64_t ia, double b, int64_t ib)
{
    return a < b || (a == b && ia < ib);
}

typedef struct { double v; int64_t j; } keyed;
static int keyed_cmp(const void *pa, const void *pb)
{
    const keyed *a = (const keyed *)pa, *b = (const keyed *)pb;
    if (a->v < b->v) return -1;
    if (a->v > b->v) return 1;
    if (a->j < b->j) return -1;
    if (a->j > b->j) return 1;
    return 0;
}
static int i64_cmp(const void *pa, const void *pb)
{
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    return (a > b) - (a < b);
}

/* ------------------------------------------------------------------------ */
/* Direct sum, eq. (1.1): u_i = sum_j K(x_i, x_j) w_j with the Gaussian   */
/* K = exp(-c ||x_i - x_j||^2 / h_j^2) of Section 4 (bandwidth of the     */
/* source point j; c = 1 is the paper's constant, c = 1/2 the usual       */
/* exp(-r^2/2h^2)).  All j, including j = i (K(x,x) = 1).                 */
/* Y == NULL: targets are the points themselves, rows `tgt` of X.         */
/* ------------------------------------------------------------------------ */
void orc_direct(const float *X, int64_t N, int d, const float *hsrc, double c,
                const double *W, int r, const float *Y, const int64_t *tgt,
                int64_t T, double *U)
{
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < T; ++t) {
        const float *x = Y ? Y + (size_t)t * d : X + (size_t)tgt[t] * d;
        for (int q = 0; q < r; ++q) U[(size_t)t * r + q] = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            double D = dist2_ff(x, X + (size_t)j * d, d);
            double h = (double)hsrc[j];
            double k = exp(-(c * D) / (h * h));
            for (int q = 0; q < r; ++q)
                U[(size_t)t * r + q] = U[(size_t)t * r + q] + k * W[(size_t)j * r + q];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Exact kNN (Section 4: exhaustive search used to measure hit rate):     */
/* N_i = the kappa smallest (D(i,j), j) over all j != i.  For queries Y   */
/* (out-of-sample targets) self-exclusion does not apply (excl = -1).     */
/* ------------------------------------------------------------------------ */
static void insert_best(int kappa, int32_t *ids, double *dd, int *cnt, double D, int64_t j)
{
    for (int q = 0; q < *cnt; ++q)
        if (ids[q] == j) return;
    if (*cnt == kappa && !lex_less(D, j, dd[kappa - 1], ids[kappa - 1])) return;
    int pos = (*cnt < kappa) ? *cnt : kappa - 1;
    while (pos > 0 && lex_less(D, j, dd[pos - 1], ids[pos - 1])) {
        dd[pos] = dd[pos - 1];
        ids[pos] = ids[pos - 1];
        --pos;
    }
    dd[pos] = D;
    ids[pos] = (int32_t)j;
    if (*cnt < kappa) ++*cnt;
}

void orc_knn_exact(const float *X, int64_t N, int d, int kappa, const float *Y,
                   const int64_t *qrows, int64_t Q, int32_t *ids, double *dist)
{
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < Q; ++t) {
        const float *x = Y ? Y + (size_t)t * d : X + (size_t)qrows[t] * d;
        int64_t self = Y ? -1 : qrows[t];
        int cnt = 0;
        int32_t *id = ids + (size_t)t * kappa;
        double *dd = dist + (size_t)t * kappa;
        for (int64_t j = 0; j < N; ++j) {
            if (j == self) continue;
            insert_best(kappa, id, dd, &cnt, dist2_ff(x, X + (size_t)j * d, d), j);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Binary tree skeleton shared by the ASKIT tree (Section 2.2, "the binary */
/* tree used in the treecode") and the random-projection trees of the kNN */
/* search.  Heap numbering: root 1, children 2a and 2a+1.  Reading taken:  */
/* every leaf sits at one depth L, the least depth at which every node    */
/* holds no more than `leaf` points (sizes at depth t are ceil(N/2^t) or  */
/* floor(N/2^t)); the left child takes ceil(n/2) points.                  */
/* ------------------------------------------------------------------------ */
int orc_tree_depth(int64_t N, int64_t leaf)
{
    int L = 0;
    while (((N + ((int64_t)1 << L) - 1) >> L) > leaf) ++L;
    return L;
}

/* Split one node's points (ascending id on entry) into left/right by the
 * projections p (one per listed point): order (p_j, j), left = first
 * ceil(n/2); both halves returned in ascending id. */
static void split_by_projection(int64_t *pts, int64_t n, const double *p)
{
    keyed *kv = (keyed *)malloc(sizeof(keyed) * (n ? n : 1));
    for (int64_t q = 0; q < n; ++q) { kv[q].v = p[q]; kv[q].j = pts[q]; }
    qsort(kv, n, sizeof(keyed), keyed_cmp);
    int64_t nl = (n + 1) / 2;
    for (int64_t q = 0; q < n; ++q) pts[q] = kv[q].j;
    qsort(pts, nl, sizeof(int64_t), i64_cmp);
    qsort(pts + nl, n - nl, sizeof(int64_t), i64_cmp);
    free(kv);
}

/* ASKIT tree split rule (Section 2.2, Fig. 3): center x_c (arithmetic   */
/* mean, points summed in ascending id), x_l = the farthest point from    */
/* x_c, x_r = the farthest point from x_l (ties: smallest id), project on */
/* the line (x_l, x_r) with origin x_l, split at the median.              */
static void askit_projection(const float *X, int d, const int64_t *pts, int64_t n, double *p)
{
    double *xc = (double *)calloc(d, sizeof(double));
    for (int k = 0; k < d; ++k) {
        double acc = 0.0;
        for (int64_t q = 0; q < n; ++q) acc = acc + (double)X[(size_t)pts[q] * d + k];
        xc[k] = acc / (double)n;
    }
    int64_t l = -1; double best = -1.0;
    for (int64_t q = 0; q < n; ++q) {
        double D = dist2_df(xc, X + (size_t)pts[q] * d, d);
        if (D > best) { best = D; l = pts[q]; }   /* pts ascending: first max = smallest id */
    }
    int64_t rr = -1; best = -1.0;
    for (int64_t q = 0; q < n; ++q) {
        double D = dist2_ff(X + (size_t)l * d, X + (size_t)pts[q] * d, d);
        if (D > best) { best = D; rr = pts[q]; }
    }
    const float *xl = X + (size_t)l * d, *xr = X + (size_t)rr * d;
    for (int64_t q = 0; q < n; ++q) {
        const float *xj = X + (size_t)pts[q] * d;
        double acc = 0.0;
        for (int k = 0; k < d; ++k) {
            double a = (double)xj[k] - (double)xl[k];
            double b = (double)xr[k] - (double)xl[k];
            acc = acc + a * b;
        }
        p[q] = acc;
    }
    free(xc);
}

/* Random-projection direction of node `node` in RP tree `iter`: Rademacher
 * signs from Philox keyed (seed, iter + 1), counter (node, word/4); bit k%64
 * of word k/64 set means -1.  Projection sum in ascending k. */
static void rp_projection(const float *X, int d, const int64_t *pts, int64_t n,
                          uint64_t seed, int iter, int64_t node, double *p)
{
    double *v = (double *)malloc(sizeof(double) * d);
    for (int k = 0; k < d; ++k) {
        uint64_t w = philox_word(seed, (uint64_t)iter + 1, (uint64_t)node, (uint64_t)(k >> 6));
        v[k] = ((w >> (k & 63)) & 1) ? -1.0 : 1.0;
    }
    for (int64_t q = 0; q < n; ++q) {
        const float *xj = X + (size_t)pts[q] * d;
        double acc = 0.0;
        for (int k = 0; k < d; ++k) acc = acc + v[k] * (double)xj[k];
        p[q] = acc;
    }
    free(v);
}

/* Build a tree of depth L over all N points.  kind 0: ASKIT rule; kind 1:
 * RP rule.  Output: order[N] = point ids in leaf order (left to right, each
 * leaf ascending id), start/size per heap node (arrays of 2^(L+1)). */
static void build_tree(const float *X, int64_t N, int d, int L, int kind, uint64_t seed,
                       int iter, int64_t *order, int64_t *start, int64_t *size)
{
    for (int64_t j = 0; j < N; ++j) order[j] = j;
    start[1] = 0; size[1] = N;
    double *p = (double *)malloc(sizeof(double) * (N ? N : 1));
    for (int t = 0; t < L; ++t) {
        for (int64_t a = (int64_t)1 << t; a < ((int64_t)2 << t); ++a) {
            int64_t *pts = order + start[a];
            int64_t n = size[a];
            if (kind == 0) askit_projection(X, d, pts, n, p);
            else rp_projection(X, d, pts, n, seed, iter, a, p);
            split_by_projection(pts, n, p);
            start[2 * a] = start[a];          size[2 * a] = (n + 1) / 2;
            start[2 * a + 1] = start[a] + (n + 1) / 2; size[2 * a + 1] = n / 2;
        }
    }
    free(p);
}

/* RP-tree kNN (Section 2.2, "Computing nearest neighbors", after Dasgupta */
/* and Freund): for T independent RP trees with leaves of <= rp_leaf       */
/* points, search exhaustively inside each point's leaf, keep the best     */
/* kappa candidates over all iterations.  Result: the kappa smallest       */
/* (D(i,j), j) over the union of i's leaf-mates across the T trees.       */
void orc_knn_rp(const float *X, int64_t N, int d, int kappa, int T, int64_t rp_leaf,
                uint64_t seed, int32_t *ids, double *dist)
{
    int L = orc_tree_depth(N, rp_leaf);
    int64_t nn = (int64_t)2 << L;
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * N);
    int64_t *start = (int64_t *)calloc(nn, sizeof(int64_t));
    int64_t *size = (int64_t *)calloc(nn, sizeof(int64_t));
    int *cnt = (int *)calloc(N, sizeof(int));
    for (int it = 0; it < T; ++it) {
        build_tree(X, N, d, L, 1, seed, it, order, start, size);
        #pragma omp parallel for schedule(dynamic, 1)
        for (int64_t a = (int64_t)1 << L; a < ((int64_t)2 << L); ++a) {
            for (int64_t q = 0; q < size[a]; ++q) {
                int64_t i = order[start[a] + q];
                for (int64_t q2 = 0; q2 < size[a]; ++q2) {
                    int64_t j = order[start[a] + q2];
                    if (j == i) continue;
                    insert_best(kappa, ids + (size_t)i * kappa, dist + (size_t)i * kappa, &cnt[i],
                                dist2_ff(X + (size_t)i * d, X + (size_t)j * d, d), j);
                }
            }
        }
    }
    free(order); free(start); free(size); free(cnt);
}

/* Standalone ASKIT tree for pin tests: perm = point ids in leaf order. */
int orc_askit_tree(const float *X, int64_t N, int d, int64_t m, int64_t *perm)
{
    int L = orc_tree_depth(N, m);
    int64_t nn = (int64_t)2 << L;
    int64_t *start = (int64_t *)calloc(nn, sizeof(int64_t));
    int64_t *size = (int64_t *)calloc(nn, sizeof(int64_t));
    build_tree(X, N, d, L, 0, 0, 0, perm, start, size);
    free(start); free(size);
    return L;
}

/* ------------------------------------------------------------------------ */
/* Interpolative decomposition by column-pivoted Householder QR (Section   */
/* 2.1): K Pi = Q R, skeleton = the first s pivots, P = R11^{-1} R12.      */
/* Reading taken (the paper fixes s; an adaptive rank is future work):    */
/* at step k the column with the largest squared norm of its trailing     */
/* part A[k:, j] (recomputed, no downdating; ties: smallest position) is  */
/* the pivot and |R_kk| its norm; the rank s is the first k with |R_kk| <= */
/* tol |R_00| once k >= s_lo, or the first k with R_kk == 0, or s_hi.     */
/* Householder sign beta = -sign(alpha) ||x||.  A is rows x cols row-major */
/* and is overwritten.  Outputs: piv[cols] (pivot order of the columns),  */
/* P[s][cols-s] row-major, rdiag[s] = R_kk; returns s.                    */
/* ------------------------------------------------------------------------ */
int orc_cpqr_id(double *A, int rows, int cols, double tol, int s_lo, int s_hi,
                int32_t *piv, double *P, double *rdiag)
{
    for (int j = 0; j < cols; ++j) piv[j] = j;
    if (s_hi > rows) s_hi = rows;
    if (s_hi > cols) s_hi = cols;
    if (s_lo > s_hi) s_lo = s_hi;
    double r00 = 0.0;
    int s = s_hi;
    double *v = (double *)malloc(sizeof(double) * (rows ? rows : 1));
    for (int k = 0; k < s_hi; ++k) {
        /* pivot: largest trailing squared norm */
        int p = -1; double best = -1.0;
        for (int j = k; j < cols; ++j) {
            double acc = 0.0;
            for (int i = k; i < rows; ++i) acc = acc + A[(size_t)i * cols + j] * A[(size_t)i * cols + j];
            if (acc > best) { best = acc; p = j; }
        }
        double nrm = sqrt(best);
        if (k == 0) r00 = nrm;
        if (nrm == 0.0 || (k >= s_lo && nrm <= tol * r00)) { s = k; break; }
        if (p != k) {
            for (int i = 0; i < rows; ++i) {
                double t = A[(size_t)i * cols + k];
                A[(size_t)i * cols + k] = A[(size_t)i * cols + p];
                A[(size_t)i * cols + p] = t;
            }
            int32_t t = piv[k]; piv[k] = piv[p]; piv[p] = t;
        }
        /* Householder reflector H = I - tau v v^T with v_k = 1, H x = beta e_k */
        double alpha = A[(size_t)k * cols + k];
        double beta = (alpha >= 0.0) ? -nrm : nrm;
        double tau = (beta - alpha) / beta;
        double scal = alpha - beta;
        v[k] = 1.0;
        for (int i = k + 1; i < rows; ++i) v[i] = A[(size_t)i * cols + k] / scal;
        A[(size_t)k * cols + k] = beta;
        for (int i = k + 1; i < rows; ++i) A[(size_t)i * cols + k] = 0.0;
        rdiag[k] = beta;
        for (int j = k + 1; j < cols; ++j) {
            double dot = 0.0;
            for (int i = k; i < rows; ++i) dot = dot + v[i] * A[(size_t)i * cols + j];
            double tdot = tau * dot;
            for (int i = k; i < rows; ++i) A[(size_t)i * cols + j] = A[(size_t)i * cols + j] - tdot * v[i];
        }
    }
    free(v);
    /* P = R11^{-1} R12 by back substitution, one column of R12 at a time */
    int nr = cols - s;
    for (int j = 0; j < nr; ++j) {
        for (int i = s - 1; i >= 0; --i) {
            double acc = A[(size_t)i * cols + (s + j)];
            for (int t = i + 1; t < s; ++t) acc = acc - A[(size_t)i * cols + t] * P[(size_t)t * nr + j];
            P[(size_t)i * nr + j] = acc / A[(size_t)i * cols + i];
        }
    }
    return s;
}

/* ------------------------------------------------------------------------ */
/* The full ASKIT structure (Algorithm 5): tree, kNN, node neighbor lists, */
/* sampled targets, skeletons, skeleton weights.                          */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t leaf_size, kappa, knn_mode, rp_iters, rp_leaf, s_max, s_min, ell_extra;
    int32_t prune, bw_mode, bw_k, pad_;
    double id_tol, kscale, h;
    uint64_t seed;
} orc_params;

typedef struct {
    int64_t N; int d; int L; int64_t nnodes;
    orc_params prm;
    const float *X;              /* caller's points [N,d], not owned */
    float *hsrc;                 /* [N] bandwidth of each source point */
    int64_t *perm;               /* [N] leaf order -> point id */
    int64_t *leafof;             /* [N] point id -> leaf heap index */
    int64_t *start, *size;       /* per heap node, leaf-order ranges */
    int32_t *knn; double *knnd;  /* [N,kappa] */
    /* per node (index by heap id) */
    int64_t *nl_cnt; int32_t **nl_ids; double **nl_key;     /* node neighbor lists */
    int64_t *ell;  int32_t **trows;                          /* sampled targets T_alpha */
    int64_t *ncol; int32_t **cols;                           /* C_alpha */
    int64_t *sk_s; int32_t **piv; double **P; int32_t **skel; /* ID */
    int r; double **wsk;         /* skeleton weights [s,r] */
    double *W;                   /* [N,r] weights, caller order */
} orc_tree;

static int in_subtree(const orc_tree *t, int64_t leaf, int64_t a)
{
    int da = 0; while (((int64_t)2 << da) <= a) ++da;   /* depth of a */
    return (leaf >> (t->L - da)) == a;
}


typedef struct { int64_t j; double key; } jkey;
static int jkey_by_j(const void *pa, const void *pb)
{
    const jkey *a = (const jkey *)pa, *b = (const jkey *)pb;
    if (a->j != b->j) return (a->j > b->j) - (a->j < b->j);
    return (a->key > b->key) - (a->key < b->key);
}
static int jkey_by_key(const void *pa, const void *pb)
{
    const jkey *a = (const jkey *)pa, *b = (const jkey *)pb;
    if (a->key != b->key) return (a->key > b->key) - (a->key < b->key);
    return (a->j > b->j) - (a->j < b->j);
}

/* Node neighbor lists, Algorithm 2, with the truncation of Section 2.2:  */
/* leaf: N_a = (U_{i in X_a} N_i) \ X_a; internal: (N_l U N_r) \ X_a.     */
/* Reading taken for the truncation key ("distance from their nearest    */
/* neighbor in a"): the minimum D(i,j) over the recorded pairs i in X_a,  */
/* j in N_i; for an internal node the minimum of the children's keys.     */
/* Sorted (key, j), truncated to ell = s_max + ell_extra entries.         */
static void build_node_lists(orc_tree *t)
{
    int64_t ellmax = (int64_t)t->prm.s_max + t->prm.ell_extra;
    int kappa = t->prm.kappa;
    for (int depth = t->L; depth >= 1; --depth) {
        #pragma omp parallel for schedule(dynamic, 1)
        for (int64_t a = (int64_t)1 << depth; a < ((int64_t)2 << depth); ++a) {
            int64_t n = 0;
            jkey *cand;
            if (depth == t->L) {
                cand = (jkey *)malloc(sizeof(jkey) * (t->size[a] * kappa + 1));
                for (int64_t q = 0; q < t->size[a]; ++q) {
                    int64_t i = t->perm[t->start[a] + q];
                    for (int z = 0; z < kappa; ++z) {
                        int64_t j = t->knn[(size_t)i * kappa + z];
                        if (in_subtree(t, t->leafof[j], a)) continue;
                        cand[n].j = j; cand[n].key = t->knnd[(size_t)i * kappa + z]; ++n;
                    }
                }
            } else {
                int64_t ch[2] = {2 * a, 2 * a + 1};
                cand = (jkey *)malloc(sizeof(jkey) * (t->nl_cnt[ch[0]] + t->nl_cnt[ch[1]] + 1));
                for (int c = 0; c < 2; ++c)
                    for (int64_t q = 0; q < t->nl_cnt[ch[c]]; ++q) {
                        int64_t j = t->nl_ids[ch[c]][q];
                        if (in_subtree(t, t->leafof[j], a)) continue;
                        cand[n].j = j; cand[n].key = t->nl_key[ch[c]][q]; ++n;
                    }
            }
            /* one entry per j, carrying its smallest key */
            qsort(cand, n, sizeof(jkey), jkey_by_j);
            int64_t u = 0;
            for (int64_t q = 0; q < n; ++q)
                if (q == 0 || cand[q].j != cand[q - 1].j) cand[u++] = cand[q];
            qsort(cand, u, sizeof(jkey), jkey_by_key);
            if (u > ellmax) u = ellmax;
            t->nl_cnt[a] = u;
            t->nl_ids[a] = (int32_t *)malloc(sizeof(int32_t) * (u + 1));
            t->nl_key[a] = (double *)malloc(sizeof(double) * (u + 1));
            for (int64_t q = 0; q < u; ++q) { t->nl_ids[a][q] = (int32_t)cand[q].j; t->nl_key[a][q] = cand[q].key; }
            free(cand);
        }
    }
}

/* Sampled skeletonization targets, eq. (2.4): T_a = N_a U Sample(X \ (X_a */
/* U N_a), ell_a - |N_a|) without replacement, ell_a = min(s_max +        */
/* ell_extra, N - |X_a|).  Reading taken for the uniform sampling: draw n */
/* of node a is j = floor(u * N / 2^32) with u the top 32 bits of Philox  */
/* word n keyed (seed, 0), counter (a, n/4); j is rejected when it lies in */
/* X_a, in N_a, or was drawn before.  Rows: N_a in key order, then draws. */
static void build_samples(orc_tree *t)
{
    int64_t ellmax = (int64_t)t->prm.s_max + t->prm.ell_extra;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t a = 2; a < t->nnodes; ++a) {
        int64_t ell = ellmax;
        if (t->N - t->size[a] < ell) ell = t->N - t->size[a];
        t->ell[a] = ell;
        t->trows[a] = (int32_t *)malloc(sizeof(int32_t) * (ell + 1));
        int64_t nr = t->nl_cnt[a] < ell ? t->nl_cnt[a] : ell;
        for (int64_t q = 0; q < nr; ++q) t->trows[a][q] = t->nl_ids[a][q];
        for (uint64_t draw = 0; nr < ell; ++draw) {
            uint64_t w = philox_word(t->prm.seed, 0, (uint64_t)a, draw);
            int64_t j = (int64_t)(((w >> 32) * (uint64_t)t->N) >> 32);
            if (in_subtree(t, t->leafof[j], a)) continue;
            int seen = 0;
            for (int64_t q = 0; q < nr && !seen; ++q) seen = (t->trows[a][q] == j);
            if (seen) continue;
            t->trows[a][nr++] = (int32_t)j;
        }
    }
}

/* Skeletonization, Algorithm 3 and Section 2.1: columns C_a = X_a        */
/* (ascending id) at a leaf, S_l then S_r at an internal node; kernel      */
/* matrix K(T_a, C_a) with the canonical exp and the column point's        */
/* bandwidth; ID by pivoted QR with s in [min(s_min, c), min(s_max, c)];   */
/* skeleton S_a = the first s pivots.  The root is never pruned            */
/* (eq. (2.5): it is an ancestor of every point) and is not skeletonized.  */
static void skeletonize(orc_tree *t)
{
    int d = t->d;
    for (int depth = t->L; depth >= 1; --depth) {
        #pragma omp parallel for schedule(dynamic, 1)
        for (int64_t a = (int64_t)1 << depth; a < ((int64_t)2 << depth); ++a) {
            int64_t c;
            int32_t *cols;
            if (depth == t->L) {
                c = t->size[a];
                cols = (int32_t *)malloc(sizeof(int32_t) * (c + 1));
                for (int64_t q = 0; q < c; ++q) cols[q] = (int32_t)t->perm[t->start[a] + q];
            } else {
                int64_t l = 2 * a, r = 2 * a + 1;
                c = t->sk_s[l] + t->sk_s[r];
                cols = (int32_t *)malloc(sizeof(int32_t) * (c + 1));
                for (int64_t q = 0; q < t->sk_s[l]; ++q) cols[q] = t->skel[l][q];
                for (int64_t q = 0; q < t->sk_s[r]; ++q) cols[t->sk_s[l] + q] = t->skel[r][q];
            }
            t->ncol[a] = c; t->cols[a] = cols;
            int64_t ell = t->ell[a];
            double *A = (double *)malloc(sizeof(double) * (ell * c + 1));
            for (int64_t i = 0; i < ell; ++i)
                for (int64_t q = 0; q < c; ++q) {
                    const float *xi = t->X + (size_t)t->trows[a][i] * d;
                    const float *xq = t->X + (size_t)cols[q] * d;
                    double D = dist2_ff(xi, xq, d);
                    double h = (double)t->hsrc[cols[q]];
                    double arg = (t->prm.kscale * D) / (h * h);
                    A[(size_t)i * c + q] = orc_cexp(-arg);
                }
            int s_lo = t->prm.s_min < c ? t->prm.s_min : (int)c;
            int s_hi = t->prm.s_max < c ? t->prm.s_max : (int)c;
            int32_t *piv = (int32_t *)malloc(sizeof(int32_t) * (c + 1));
            double *P = (double *)malloc(sizeof(double) * ((size_t)s_hi * c + 1));
            double *rd = (double *)malloc(sizeof(double) * (c + 1));
            int s = orc_cpqr_id(A, (int)ell, (int)c, t->prm.id_tol, s_lo, s_hi, piv, P, rd);
            free(A); free(rd);
            t->sk_s[a] = s; t->piv[a] = piv; t->P[a] = P;
            t->skel[a] = (int32_t *)malloc(sizeof(int32_t) * (s + 1));
            for (int q = 0; q < s; ++q) t->skel[a][q] = cols[piv[q]];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Build everything Algorithm 5 needs before Evaluate.                     */
/* knn_in: optional caller-given [N,kappa] neighbor ids (the paper's       */
/* N(X) argument); NULL computes them (knn_mode 0 exact, 1 RP trees).      */
/* hsrc_in: per-point bandwidth for bw_mode 1.  bw_mode 0: constant h;     */
/* bw_mode 2: h_j = distance to the bw_k-th neighbor (rounded to FP32).    */
/* ------------------------------------------------------------------------ */
orc_tree *orc_build(const float *X, int64_t N, int d, const orc_params *prm,
                    const float *hsrc_in, const int32_t *knn_in)
{
    orc_tree *t = (orc_tree *)calloc(1, sizeof(orc_tree));
    t->N = N; t->d = d; t->prm = *prm; t->X = X;
    int kappa = prm->kappa;
    t->knn = (int32_t *)malloc(sizeof(int32_t) * N * kappa);
    t->knnd = (double *)malloc(sizeof(double) * N * kappa);
    if (knn_in) {
        memcpy(t->knn, knn_in, sizeof(int32_t) * N * kappa);
        for (int64_t i = 0; i < N; ++i)
            for (int z = 0; z < kappa; ++z)
                t->knnd[i * kappa + z] = dist2_ff(X + (size_t)i * d, X + (size_t)t->knn[i * kappa + z] * d, d);
    } else if (prm->knn_mode == 0) {
        int64_t *rows = (int64_t *)malloc(sizeof(int64_t) * N);
        for (int64_t i = 0; i < N; ++i) rows[i] = i;
        orc_knn_exact(X, N, d, kappa, NULL, rows, N, t->knn, t->knnd);
        free(rows);
    } else {
        orc_knn_rp(X, N, d, kappa, prm->rp_iters, prm->rp_leaf, prm->seed, t->knn, t->knnd);
    }
    t->hsrc = (float *)malloc(sizeof(float) * N);
    for (int64_t j = 0; j < N; ++j) {
        if (prm->bw_mode == 1) t->hsrc[j] = hsrc_in[j];
        else if (prm->bw_mode == 2) t->hsrc[j] = (float)sqrt(t->knnd[j * kappa + (prm->bw_k - 1)]);
        else t->hsrc[j] = (float)prm->h;
    }
    t->L = orc_tree_depth(N, prm->leaf_size);
    t->nnodes = (int64_t)2 << t->L;
    t->perm = (int64_t *)malloc(sizeof(int64_t) * N);
    t->start = (int64_t *)calloc(t->nnodes, sizeof(int64_t));
    t->size = (int64_t *)calloc(t->nnodes, sizeof(int64_t));
    build_tree(X, N, d, t->L, 0, 0, 0, t->perm, t->start, t->size);
    t->leafof = (int64_t *)malloc(sizeof(int64_t) * N);
    for (int64_t a = (int64_t)1 << t->L; a < t->nnodes; ++a)
        for (int64_t q = 0; q < t->size[a]; ++q) t->leafof[t->perm[t->start[a] + q]] = a;
#define ALLOC(f, T) t->f = (T *)calloc(t->nnodes, sizeof(T))
    ALLOC(nl_cnt, int64_t); ALLOC(nl_ids, int32_t *); ALLOC(nl_key, double *);
    ALLOC(ell, int64_t); ALLOC(trows, int32_t *); ALLOC(ncol, int64_t); ALLOC(cols, int32_t *);
    ALLOC(sk_s, int64_t); ALLOC(piv, int32_t *); ALLOC(P, double *); ALLOC(skel, int32_t *);
    ALLOC(wsk, double *);
#undef ALLOC
    if (t->L > 0) {
        build_node_lists(t);
        build_samples(t);
        skeletonize(t);
    }
    return t;
}

/* Skeleton weights, Section 2.1 and Algorithm 3: w~_a = v(S_a) + P_a v(R) */
/* with v = w(X_a) at a leaf and v = [w~_l; w~_r] at an internal node;     */
/* R = the remaining columns in pivot order.  W is [N,r] in point order.  */
void orc_set_weights(orc_tree *t, const double *W, int r)
{
    free(t->W);
    t->r = r;
    t->W = (double *)malloc(sizeof(double) * t->N * r);
    memcpy(t->W, W, sizeof(double) * t->N * r);
    for (int depth = t->L; depth >= 1; --depth) {
        #pragma omp parallel for schedule(dynamic, 1)
        for (int64_t a = (int64_t)1 << depth; a < ((int64_t)2 << depth); ++a) {
            int64_t c = t->ncol[a], s = t->sk_s[a], nr = c - s;
            double *v = (double *)malloc(sizeof(double) * (c * r + 1));
            if (depth == t->L) {
                for (int64_t q = 0; q < c; ++q)
                    for (int z = 0; z < r; ++z) v[q * r + z] = W[(size_t)t->cols[a][q] * r + z];
            } else {
                int64_t l = 2 * a, rr = 2 * a + 1;
                for (int64_t q = 0; q < t->sk_s[l]; ++q)
                    for (int z = 0; z < r; ++z) v[q * r + z] = t->wsk[l][q * r + z];
                for (int64_t q = 0; q < t->sk_s[rr]; ++q)
                    for (int z = 0; z < r; ++z) v[(t->sk_s[l] + q) * r + z] = t->wsk[rr][q * r + z];
            }
            free(t->wsk[a]);
            t->wsk[a] = (double *)malloc(sizeof(double) * (s * r + 1));
            for (int64_t q = 0; q < s; ++q)
                for (int z = 0; z < r; ++z) {
                    double acc = 0.0;
                    for (int64_t u = 0; u < nr; ++u)
                        acc = acc + t->P[a][q * nr + u] * v[(size_t)t->piv[a][s + u] * r + z];
                    t->wsk[a][q * r + z] = v[(size_t)t->piv[a][q] * r + z] + acc;
                }
            free(v);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Evaluate, Algorithm 4, with the neighbor pruning rule eq. (2.5):        */
/* Prune(a, i) holds when no j in {i} U N_i has a among its ancestors     */
/* (a node counts as its own ancestor).  Pruned: K(x_i, S_a) w~_a; leaf:   */
/* K(x_i, X_a) w_a (direct, includes j = i); else right child + left.     */
/* `pset` is the prune set as leaf indices (np entries).                  */
/* near/far count the leaves evaluated directly and the skeletons used.   */
/* ------------------------------------------------------------------------ */
/* `part` selects which terms enter u: 1 the near field (direct leaf sums), */
/* 2 the far field (skeleton sums), 3 both (Algorithm 4 itself).  The paper */
/* reports eps_kappa, the error of the near field alone (Table 4).           */
/* `far_height` (>= 0) restricts the far field to nodes at most that many  */
/* levels above the leaves (Section 3 proposes bounding the level of the   */
/* skeletons used by starting the downward pass a fixed number of levels   */
/* above the leaves): a higher node that would be pruned is descended      */
/* instead, down to that height.  -1: no restriction (Algorithm 4).        */
static void evaluate_rec(const orc_tree *t, const float *x, const int64_t *pset, int np,
                         int64_t a, int depth, double *u, int64_t *near, int64_t *far, int part,
                         int far_height)
{
    int r = t->r, d = t->d;
    int pruned = t->prm.prune;
    if (pruned)
        for (int q = 0; q < np && pruned; ++q)
            if ((pset[q] >> (t->L - depth)) == a) pruned = 0;
    if (depth == 0) pruned = 0;
    if (far_height >= 0 && t->L - depth > far_height) pruned = 0;
    if (pruned) {
        for (int64_t q = 0; q < t->sk_s[a] && (part & 2); ++q) {
            int64_t j = t->skel[a][q];
            double h = (double)t->hsrc[j];
            double k = exp(-(t->prm.kscale * dist2_ff(x, t->X + (size_t)j * d, d)) / (h * h));
            for (int z = 0; z < r; ++z) u[z] = u[z] + k * t->wsk[a][q * r + z];
        }
        ++*far;
        return;
    }
    if (depth == t->L) {
        for (int64_t q = 0; q < t->size[a] && (part & 1); ++q) {
            int64_t j = t->perm[t->start[a] + q];
            double h = (double)t->hsrc[j];
            double k = exp(-(t->prm.kscale * dist2_ff(x, t->X + (size_t)j * d, d)) / (h * h));
            for (int z = 0; z < r; ++z) u[z] = u[z] + k * t->W[(size_t)j * r + z];
        }
        ++*near;
        return;
    }
    evaluate_rec(t, x, pset, np, 2 * a + 1, depth + 1, u, near, far, part, far_height);
    evaluate_rec(t, x, pset, np, 2 * a, depth + 1, u, near, far, part, far_height);
}

/* Adaptive kappa_i (Section 3 suggests choosing kappa per point from the */
/* distance to its farther neighbors).                                     */
/* Reading taken: with a kernel cut a > 0, the prune set keeps the         */
/* neighbors up to the last rank whose kernel value exceeds e^-a, i.e.     */
/* kappa_i = 1 + max{ z : c D(i, N_i[z]) / h^2 < a } (0 if none), with h   */
/* the neighbor's bandwidth and D the stored FP64 squared distance; a <= 0 */
/* keeps all kappa.  Neighbors past kappa_i may then be approximated in   */
/* pruned nodes, where their kernel values are small.                      */
static int kappa_of(const orc_tree *t, const double *dist, const int32_t *ids, double cut)
{
    int kappa = t->prm.kappa;
    if (!(cut > 0.0)) return kappa;
    int ki = 0;
    for (int z = 0; z < kappa; ++z) {
        double h = (double)t->hsrc[ids[z]];
        double arg = (t->prm.kscale * dist[z]) / (h * h);
        if (arg < cut) ki = z + 1;
    }
    return ki;
}

/* In-sample targets: rows tgt[0..T) (point ids); U [T,r].  The prune set */
/* of target i is {i} U N_i (eq. (2.5)).  With prune == 2 (leaf-grouped   */
/* lists) it is the union of {p} U N_p over the points p of i's leaf, so  */
/* every target of a leaf shares one Near and one Far list -- the grouping */
/* Section 3 points to when it notes that the direct nodes of the targets */
/* of one leaf overlap heavily.                                           */
void orc_evaluate_ext(const orc_tree *t, const int64_t *tgt, int64_t T, int part, int far_height,
                      double kappa_cut, double *U, int64_t *near, int64_t *far)
{
    int kappa = t->prm.kappa;
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t q = 0; q < T; ++q) {
        int64_t i = tgt[q];
        int64_t np = 0;
        int64_t *pset;
        if (t->prm.prune == 2) {
            int64_t a = t->leafof[i];
            pset = (int64_t *)malloc(sizeof(int64_t) * t->size[a] * (kappa + 1));
            for (int64_t v = 0; v < t->size[a]; ++v) {
                int64_t p = t->perm[t->start[a] + v];
                int kp = kappa_of(t, t->knnd + (size_t)p * kappa, t->knn + (size_t)p * kappa, kappa_cut);
                pset[np++] = t->leafof[p];
                for (int z = 0; z < kp; ++z) pset[np++] = t->leafof[t->knn[(size_t)p * kappa + z]];
            }
        } else {
            int ki = kappa_of(t, t->knnd + (size_t)i * kappa, t->knn + (size_t)i * kappa, kappa_cut);
            pset = (int64_t *)malloc(sizeof(int64_t) * (kappa + 1));
            pset[np++] = t->leafof[i];
            for (int z = 0; z < ki; ++z) pset[np++] = t->leafof[t->knn[(size_t)i * kappa + z]];
        }
        double *u = U + (size_t)q * t->r;
        for (int z = 0; z < t->r; ++z) u[z] = 0.0;
        int64_t nn = 0, nf = 0;
        evaluate_rec(t, t->X + (size_t)i * t->d, pset, (int)np, 1, 0, u, &nn, &nf, part, far_height);
        if (near) near[q] = nn;
        if (far) far[q] = nf;
        free(pset);
    }
}

void orc_evaluate_part(const orc_tree *t, const int64_t *tgt, int64_t T, int part, double *U,
                       int64_t *near, int64_t *far)
{
    orc_evaluate_ext(t, tgt, T, part, -1, 0.0, U, near, far);
}

void orc_evaluate(const orc_tree *t, const int64_t *tgt, int64_t T, double *U,
                  int64_t *near, int64_t *far)
{
    orc_evaluate_ext(t, tgt, T, 3, -1, 0.0, U, near, far);
}

/* Out-of-sample targets y (the paper takes sources = targets; reading    */
/* taken): the prune set of y is its exact kappa nearest sources N_y (no  */
/* self term); then Algorithm 4 unchanged.  y belongs to no leaf, so the  */
/* leaf-grouped mode (prune == 2) uses the same per-target set here.      */
void orc_evaluate_oos_ext(const orc_tree *t, const float *Y, int64_t T, int far_height, double kappa_cut,
                          double *U, int32_t *knn_out, int64_t *near, int64_t *far)
{
    int kappa = t->prm.kappa, d = t->d;
    int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * T * kappa);
    double *dd = (double *)malloc(sizeof(double) * T * kappa);
    orc_knn_exact(t->X, t->N, d, kappa, Y, NULL, T, ids, dd);
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t q = 0; q < T; ++q) {
        int ky = kappa_of(t, dd + (size_t)q * kappa, ids + (size_t)q * kappa, kappa_cut);
        int64_t *pset = (int64_t *)malloc(sizeof(int64_t) * (kappa + 1));
        for (int z = 0; z < ky; ++z) pset[z] = t->leafof[ids[(size_t)q * kappa + z]];
        double *u = U + (size_t)q * t->r;
        for (int z = 0; z < t->r; ++z) u[z] = 0.0;
        int64_t nn = 0, nf = 0;
        evaluate_rec(t, Y + (size_t)q * d, pset, ky, 1, 0, u, &nn, &nf, 3, far_height);
        if (near) near[q] = nn;
        if (far) far[q] = nf;
        free(pset);
    }
    if (knn_out) memcpy(knn_out, ids, sizeof(int32_t) * T * kappa);
    free(ids); free(dd);
}

void orc_evaluate_oos(const orc_tree *t, const float *Y, int64_t T, double *U,
                      int32_t *knn_out, int64_t *near, int64_t *far)
{
    orc_evaluate_oos_ext(t, Y, T, -1, 0.0, U, knn_out, near, far);
}

/* ------------------------------------------------------------------------ */
/* Pruning statistics of Table 1 (Section 3, which compares distance     */
/* pruning with neighbor pruning): for every point i as a target, the     */
/* number of tree nodes the downward pass visits (Evaluate calls, pruned */
/* nodes included) under                                                   */
/*   neighbor pruning, eq. (2.5): a node is pruned unless it holds i or    */
/*     one of its kappa nearest neighbors (the exact kNN, any kappa);      */
/*   distance pruning: a node alpha with centroid c_alpha and radius       */
/*     R_alpha = max_{x in alpha} ||x - c_alpha|| is pruned when           */
/*     ||x_i - c_alpha|| > rscale R_alpha (Section 3 remarks that R needs */
/*     a scale factor to separate the nodes; rscale = 1 is the plain rule).*/
/* The root is never pruned.  Readings taken: c_alpha is the FP64 mean of  */
/* the node's points summed in leaf order, distances are compared squared */
/* (D(x_i, c) > rscale^2 R^2) in FP64, coordinates in ascending order.    */
/* ------------------------------------------------------------------------ */
static int64_t visit_dist(const float *x, int d, int L, int64_t a, int depth, const double *cent,
                          const double *r2, double rs2)
{
    int64_t v = 1;
    if (depth > 0 && dist2_df(cent + (size_t)a * d, x, d) > rs2 * r2[a]) return v;
    if (depth == L) return v;
    return v + visit_dist(x, d, L, 2 * a, depth + 1, cent, r2, rs2) +
           visit_dist(x, d, L, 2 * a + 1, depth + 1, cent, r2, rs2);
}

static int64_t visit_knn(int L, int64_t a, int depth, const int64_t *pset, int np)
{
    int64_t v = 1;
    int keep = depth == 0;
    for (int q = 0; q < np && !keep; ++q)
        if ((pset[q] >> (L - depth)) == a) keep = 1;
    if (!keep || depth == L) return v;
    return v + visit_knn(L, 2 * a, depth + 1, pset, np) + visit_knn(L, 2 * a + 1, depth + 1, pset, np);
}

int orc_prune_stats(const float *X, int64_t N, int d, int64_t m, int kappa, double rscale,
                    int64_t *visited_knn, int64_t *visited_dist)
{
    int L = orc_tree_depth(N, m);
    int64_t nn = (int64_t)2 << L;
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * N);
    int64_t *start = (int64_t *)calloc(nn, sizeof(int64_t));
    int64_t *size = (int64_t *)calloc(nn, sizeof(int64_t));
    build_tree(X, N, d, L, 0, 0, 0, perm, start, size);
    int64_t *leaf = (int64_t *)malloc(sizeof(int64_t) * N);
    for (int64_t a = (int64_t)1 << L; a < nn; ++a)
        for (int64_t q = 0; q < size[a]; ++q) leaf[perm[start[a] + q]] = a;
    int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * N * kappa);
    double *dd = (double *)malloc(sizeof(double) * N * kappa);
    int64_t *rows = (int64_t *)malloc(sizeof(int64_t) * N);
    for (int64_t i = 0; i < N; ++i) rows[i] = i;
    orc_knn_exact(X, N, d, kappa, NULL, rows, N, ids, dd);
    double *cent = (double *)calloc((size_t)nn * d, sizeof(double));
    double *r2 = (double *)calloc(nn, sizeof(double));
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t a = 1; a < nn; ++a) {
        if (size[a] == 0) continue;
        double *c = cent + (size_t)a * d;
        for (int64_t q = 0; q < size[a]; ++q) {
            const float *x = X + (size_t)perm[start[a] + q] * d;
            for (int k = 0; k < d; ++k) c[k] = c[k] + (double)x[k];
        }
        for (int k = 0; k < d; ++k) c[k] = c[k] / (double)size[a];
        double mx = 0.0;
        for (int64_t q = 0; q < size[a]; ++q) {
            double D = dist2_df(c, X + (size_t)perm[start[a] + q] * d, d);
            if (D > mx) mx = D;
        }
        r2[a] = mx;
    }
    const double rs2 = rscale * rscale;
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < N; ++i) {
        int64_t pset[1 + 4096];
        int np = 0;
        pset[np++] = leaf[i];
        for (int z = 0; z < kappa && z < 4096; ++z) pset[np++] = leaf[ids[(size_t)i * kappa + z]];
        visited_knn[i] = visit_knn(L, 1, 0, pset, np);
        visited_dist[i] = visit_dist(X + (size_t)i * d, d, L, 1, 0, cent, r2, rs2);
    }
    free(perm); free(start); free(size); free(leaf); free(ids); free(dd); free(rows); free(cent); free(r2);
    return L;
}

/* ------------------------------------------------------------------------ */
/* Accessors for tests (copy out; sizes via orc_info).                    */
/* ------------------------------------------------------------------------ */
void orc_info(const orc_tree *t, int64_t *out)
{
    out[0] = t->N; out[1] = t->d; out[2] = t->L; out[3] = t->nnodes;
    int64_t tot_s = 0, tot_nl = 0, tot_ell = 0, tot_p = 0;
    for (int64_t a = 2; a < t->nnodes; ++a) {
        tot_s += t->sk_s[a]; tot_nl += t->nl_cnt[a]; tot_ell += t->ell[a];
        tot_p += t->sk_s[a] * (t->ncol[a] - t->sk_s[a]);
    }
    out[4] = tot_s; out[5] = tot_nl; out[6] = tot_ell; out[7] = tot_p;
}
void orc_get_perm(const orc_tree *t, int64_t *perm) { memcpy(perm, t->perm, sizeof(int64_t) * t->N); }
void orc_get_knn(const orc_tree *t, int32_t *ids, double *dd)
{
    memcpy(ids, t->knn, sizeof(int32_t) * t->N * t->prm.kappa);
    if (dd) memcpy(dd, t->knnd, sizeof(double) * t->N * t->prm.kappa);
}
void orc_get_hsrc(const orc_tree *t, float *h) { memcpy(h, t->hsrc, sizeof(float) * t->N); }
/* per node counts: [nnodes] each */
void orc_get_counts(const orc_tree *t, int64_t *start, int64_t *size, int64_t *nl, int64_t *ell,
                    int64_t *ncol, int64_t *s)
{
    for (int64_t a = 0; a < t->nnodes; ++a) {
        start[a] = t->start[a]; size[a] = t->size[a]; nl[a] = t->nl_cnt[a];
        ell[a] = t->ell[a]; ncol[a] = t->ncol[a]; s[a] = t->sk_s[a];
    }
}
void orc_get_node(const orc_tree *t, int64_t a, int32_t *nl_ids, double *nl_key, int32_t *trows,
                  int32_t *cols, int32_t *piv, int32_t *skel, double *P, double *wsk)
{
    if (nl_ids) memcpy(nl_ids, t->nl_ids[a], sizeof(int32_t) * t->nl_cnt[a]);
    if (nl_key) memcpy(nl_key, t->nl_key[a], sizeof(double) * t->nl_cnt[a]);
    if (trows) memcpy(trows, t->trows[a], sizeof(int32_t) * t->ell[a]);
    if (cols) memcpy(cols, t->cols[a], sizeof(int32_t) * t->ncol[a]);
    if (piv) memcpy(piv, t->piv[a], sizeof(int32_t) * t->ncol[a]);
    if (skel) memcpy(skel, t->skel[a], sizeof(int32_t) * t->sk_s[a]);
    if (P) memcpy(P, t->P[a], sizeof(double) * t->sk_s[a] * (t->ncol[a] - t->sk_s[a]));
    if (wsk && t->wsk[a]) memcpy(wsk, t->wsk[a], sizeof(double) * t->sk_s[a] * t->r);
}

void orc_free(orc_tree *t)
{
    if (!t) return;
    for (int64_t a = 0; a < t->nnodes; ++a) {
        free(t->nl_ids[a]); free(t->nl_key[a]); free(t->trows[a]); free(t->cols[a]);
        free(t->piv[a]); free(t->P[a]); free(t->skel[a]); free(t->wsk[a]);
    }
    free(t->nl_cnt); free(t->nl_ids); free(t->nl_key); free(t->ell); free(t->trows);
    free(t->ncol); free(t->cols); free(t->sk_s); free(t->piv); free(t->P); free(t->skel);
    free(t->wsk); free(t->W); free(t->knn); free(t->knnd); free(t->hsrc); free(t->perm);
    free(t->leafof); free(t->start); free(t->size); free(t);
}

/* OpenMP threads of the oracle's parallel loops (independent targets,   */
/* points or nodes only; results do not depend on it).                     */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
