/*
 * exsum_oracle.c -- CPU oracle for multidimensional included and excluded sums
 * (Xu, Fraser, Leiserson, "Multidimensional Included and Excluded Sums",
 * SIAM ACDA 2021).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, single-threaded
 * restatement of the paper's definitions and algorithms.  It exists to check
 * the CUDA library; it is never called by the library.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.
 * It shares no code, header, table or constant with the CUDA path.
 *
 * Conventions
 *   - Tensors are row-major: dimension d-1 is contiguous, dimension 0 the
 *     slowest.  Coordinates are 0-based (the paper is 1-based).
 *   - Elements are 8-byte cells (union oval): int64 for integer monoids,
 *     double for floating-point monoids.  Narrower inputs are widened
 *     exactly by the caller (int32 -> int64, fp32/bf16 -> double).
 *   - Monoids (Sec. 1, "monoid (S, +, e)"):
 *       ORC_ADD_I64  integer +, wrapping modulo 2^64 (exact, so any
 *                    reassociation gives the same bits; the low 32 bits give
 *                    the wrapping int32 sum)
 *       ORC_MAX_I64  integer max, identity INT64_MIN
 *       ORC_ADD_F64  double +
 *       ORC_MAX_F64  double max, identity -infinity (inputs carry no NaN)
 *   - A box of size k cornered at x is the half-open box [x, x+k) clipped to
 *     the tensor (Sec. 2, colon notation): coordinates outside the tensor
 *     contribute the identity e.
 *
 * Parity status of each entry point (what pins it is in the test suite):
 *   orc_included_brute / orc_excluded_brute / orc_*_at  -- the definition
 *       (Sec. 2, Definition "Included and Excluded Sums"), pinned by closed
 *       forms, invariants and special cases.
 *   orc_bdbs            -- Sec. 3 (BDBS-1D, Fig. "incsum-1d-code"; BDBS in
 *                          arbitrary dimensions), pinned against brute force.
 *   orc_box_complement  -- Sec. 5 (Fig. "exsum-code-full" with the
 *                          subroutines of App. C), pinned against brute force.
 *   orc_corners         -- App. A (corners algorithm), d = 2 and d = 3,
 *                          pinned against brute force; partition checked
 *                          exhaustively.
 *   orc_sat_included    -- Sec. 1 (summed-area table), integer + only.
 *   orc_bdbsc           -- Sec. 1 (BDBS complement, weak), integer + only.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORC_MAX_DIMS 8

enum { ORC_ADD_I64 = 0, ORC_MAX_I64 = 1, ORC_ADD_F64 = 2, ORC_MAX_F64 = 3 };
enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ENOMEM = -2 };

typedef union {
    int64_t i;
    double f;
} oval;

/* Number of applications of the monoid operator since the last reset. */
static uint64_t g_ops = 0;

void orc_reset_ops(void) { g_ops = 0; }
uint64_t orc_get_ops(void) { return g_ops; }

static oval identity(int mon)
{
    oval e;
    switch (mon) {
    case ORC_ADD_I64: e.i = 0; break;
    case ORC_MAX_I64: e.i = INT64_MIN; break;
    case ORC_ADD_F64: e.f = 0.0; break;
    default: e.f = -INFINITY; break;
    }
    return e;
}

/* a (+) b for the chosen monoid; a is the left operand. */
static oval combine(int mon, oval a, oval b)
{
    oval r;
    g_ops++;
    switch (mon) {
    case ORC_ADD_I64: r.i = (int64_t)((uint64_t)a.i + (uint64_t)b.i); break;
    case ORC_MAX_I64: r.i = a.i > b.i ? a.i : b.i; break;
    case ORC_ADD_F64: r.f = a.f + b.f; break;
    default: r.f = a.f > b.f ? a.f : b.f; break;
    }
    return r;
}

static int valid_monoid(int mon) { return mon >= ORC_ADD_I64 && mon <= ORC_MAX_F64; }

/* Checks 1 <= d <= 8, n_i >= 1 and 1 <= k_i <= n_i (Sec. 1: k_i <= n_i). */
static int check_args(int d, const int64_t *n, const int64_t *k, int mon)
{
    int i;
    if (d < 1 || d > ORC_MAX_DIMS || !valid_monoid(mon)) return ORC_EINVAL;
    for (i = 0; i < d; i++) {
        if (n[i] < 1) return ORC_EINVAL;
        if (k && (k[i] < 1 || k[i] > n[i])) return ORC_EINVAL;
    }
    return ORC_OK;
}

static int64_t volume(int d, const int64_t *n)
{
    int64_t v = 1;
    int i;
    for (i = 0; i < d; i++) v *= n[i];
    return v;
}

static void row_major_strides(int d, const int64_t *n, int64_t *st)
{
    int i;
    st[d - 1] = 1;
    for (i = d - 2; i >= 0; i--) st[i] = st[i + 1] * n[i + 1];
}

/* Advances the odometer x over lo[i] <= x[i] < hi[i]; returns 0 when done. */
static int next_coord(int d, int64_t *x, const int64_t *lo, const int64_t *hi)
{
    int i;
    for (i = d - 1; i >= 0; i--) {
        if (++x[i] < hi[i]) return 1;
        x[i] = lo[i];
    }
    return 0;
}

static int64_t offset_of(int d, const int64_t *x, const int64_t *st)
{
    int64_t o = 0;
    int i;
    for (i = 0; i < d; i++) o += x[i] * st[i];
    return o;
}

/* ------------------------------------------------------------------------
 * The definition (Sec. 2): the included sum at x reduces A over the box
 * [x, x+k) clipped to the tensor; the excluded sum reduces A over every
 * coordinate outside that box.
 * ------------------------------------------------------------------------ */

static oval included_at(const oval *A, int d, const int64_t *n, const int64_t *k,
                        int mon, const int64_t *x, const int64_t *st)
{
    int64_t lo[ORC_MAX_DIMS], hi[ORC_MAX_DIMS], y[ORC_MAX_DIMS];
    oval acc = identity(mon);
    int i;
    for (i = 0; i < d; i++) {
        lo[i] = x[i];
        hi[i] = x[i] + k[i] < n[i] ? x[i] + k[i] : n[i];
        y[i] = lo[i];
    }
    do {
        acc = combine(mon, acc, A[offset_of(d, y, st)]);
    } while (next_coord(d, y, lo, hi));
    return acc;
}

static int inside_box(int d, const int64_t *y, const int64_t *x, const int64_t *k)
{
    int i;
    for (i = 0; i < d; i++)
        if (y[i] < x[i] || y[i] >= x[i] + k[i]) return 0;
    return 1;
}

static oval excluded_at(const oval *A, int d, const int64_t *n, const int64_t *k,
                        int mon, const int64_t *x, const int64_t *st)
{
    int64_t lo[ORC_MAX_DIMS], y[ORC_MAX_DIMS];
    oval acc = identity(mon);
    int i;
    for (i = 0; i < d; i++) lo[i] = y[i] = 0;
    do {
        if (!inside_box(d, y, x, k)) acc = combine(mon, acc, A[offset_of(d, y, st)]);
    } while (next_coord(d, y, lo, n));
    return acc;
}

int orc_included_at(const oval *A, int d, const int64_t *n, const int64_t *k, int mon,
                    const int64_t *x, oval *result)
{
    int64_t st[ORC_MAX_DIMS];
    int i;
    if (check_args(d, n, k, mon)) return ORC_EINVAL;
    for (i = 0; i < d; i++)
        if (x[i] < 0 || x[i] >= n[i]) return ORC_EINVAL;
    row_major_strides(d, n, st);
    *result = included_at(A, d, n, k, mon, x, st);
    return ORC_OK;
}

int orc_excluded_at(const oval *A, int d, const int64_t *n, const int64_t *k, int mon,
                    const int64_t *x, oval *result)
{
    int64_t st[ORC_MAX_DIMS];
    int i;
    if (check_args(d, n, k, mon)) return ORC_EINVAL;
    for (i = 0; i < d; i++)
        if (x[i] < 0 || x[i] >= n[i]) return ORC_EINVAL;
    row_major_strides(d, n, st);
    *result = excluded_at(A, d, n, k, mon, x, st);
    return ORC_OK;
}

int orc_included_brute(const oval *A, oval *out, int d, const int64_t *n, const int64_t *k, int mon)
{
    int64_t st[ORC_MAX_DIMS], lo[ORC_MAX_DIMS], x[ORC_MAX_DIMS];
    int i;
    if (check_args(d, n, k, mon)) return ORC_EINVAL;
    row_major_strides(d, n, st);
    for (i = 0; i < d; i++) lo[i] = x[i] = 0;
    do {
        out[offset_of(d, x, st)] = included_at(A, d, n, k, mon, x, st);
    } while (next_coord(d, x, lo, n));
    return ORC_OK;
}

int orc_excluded_brute(const oval *A, oval *out, int d, const int64_t *n, const int64_t *k, int mon)
{
    int64_t st[ORC_MAX_DIMS], lo[ORC_MAX_DIMS], x[ORC_MAX_DIMS];
    int i;
    if (check_args(d, n, k, mon)) return ORC_EINVAL;
    row_major_strides(d, n, st);
    for (i = 0; i < d; i++) lo[i] = x[i] = 0;
    do {
        out[offset_of(d, x, st)] = excluded_at(A, d, n, k, mon, x, st);
    } while (next_coord(d, x, lo, n));
    return ORC_OK;
}

/* ------------------------------------------------------------------------
 * Row iteration.  A "view" is the sub-tensor of the full row-major tensor in
 * which dimensions 0..fixed-1 are pinned (the pinned part is folded into
 * `base`) and dimensions fixed..d-1 range over their full extent.  This is
 * the dimension-reduced tensor of Sec. 5 ("fixes the first i dimensions at
 * n_1, ..., n_i").
 * ------------------------------------------------------------------------ */

typedef void (*row_fn)(oval *row, int64_t stride, int64_t len, int64_t k, int mon, oval *t1, oval *t2);

/* Applies fn to every row along dimension `dim` of the view whose dimensions
 * < fixed are pinned. */
static void for_each_row(oval *base, int d, const int64_t *n, const int64_t *st, int fixed,
                         int dim, int64_t k, int mon, row_fn fn, oval *t1, oval *t2)
{
    int64_t lo[ORC_MAX_DIMS], hi[ORC_MAX_DIMS], x[ORC_MAX_DIMS];
    int i;
    for (i = 0; i < d; i++) {
        lo[i] = 0;
        x[i] = 0;
        hi[i] = (i < fixed || i == dim) ? 1 : n[i];
    }
    do {
        fn(base + offset_of(d, x, st), st[dim], n[dim], k, mon, t1, t2);
    } while (next_coord(d, x, lo, hi));
}

/* Prefix (Sec. 2, Eq. "prefix-sum-def"): in-place running reduction from the
 * first element of the row to the last.  The operands are combined in array
 * order (earlier elements on the left). */
static void prefix_row(oval *r, int64_t s, int64_t len, int64_t k, int mon, oval *t1, oval *t2)
{
    int64_t x;
    (void)k; (void)t1; (void)t2;
    for (x = 1; x < len; x++) r[x * s] = combine(mon, r[(x - 1) * s], r[x * s]);
}

/* Suffix (Sec. 2): the same recursion run from the last element back. */
static void suffix_row(oval *r, int64_t s, int64_t len, int64_t k, int mon, oval *t1, oval *t2)
{
    int64_t x;
    (void)k; (void)t1; (void)t2;
    for (x = len - 2; x >= 0; x--) r[x * s] = combine(mon, r[x * s], r[(x + 1) * s]);
}

/* BDBS-1D (Sec. 3, Fig. "incsum-1d-code"), in place on one row of length len.
 * t1 receives the k-wise prefixes A_p and t2 the k-wise suffixes A_s.
 * When len is not a multiple of k the row is treated as padded with the
 * identity up to the next multiple of k (Sec. 3 footnote), which is the
 * clipped-box semantics of Sec. 2. */
static void bdbs_row(oval *r, int64_t s, int64_t len, int64_t k, int mon, oval *Ap, oval *As)
{
    int64_t b0, end, x;
    /* Range-Prefix-Row: prefix over each block [b0, b0+k). */
    for (b0 = 0; b0 < len; b0 += k) {
        end = b0 + k < len ? b0 + k : len;
        Ap[b0] = r[b0 * s];
        for (x = b0 + 1; x < end; x++) Ap[x] = combine(mon, Ap[x - 1], r[x * s]);
    }
    /* Range-Suffix-Row: suffix over each block. */
    for (b0 = 0; b0 < len; b0 += k) {
        end = b0 + k < len ? b0 + k : len;
        As[end - 1] = r[(end - 1) * s];
        for (x = end - 2; x >= b0; x--) As[x] = combine(mon, r[x * s], As[x + 1]);
    }
    /* Combine-Along-Row: a block start takes its whole-block suffix; any other
     * x combines the suffix of its block with the prefix of the next block up
     * to x+k-1.  In the padded row that prefix ends at the row's last element
     * when x+k-1 runs past it, and is empty when the next block is all
     * padding. */
    for (x = 0; x < len; x++) {
        oval v = As[x];
        if (x % k != 0) {
            int64_t j = x + k - 1;
            int64_t next_block = (x / k + 1) * k;
            if (j < len)
                v = combine(mon, As[x], Ap[j]);
            else if (next_block <= len - 1)
                v = combine(mon, As[x], Ap[len - 1]);
        }
        r[x * s] = v;
    }
}

/* BDBS (Sec. 3, "Generalizing to Arbitrary Dimensions"): the included sum
 * along dimensions 1..d in turn. */
int orc_bdbs(const oval *A, oval *out, int d, const int64_t *n, const int64_t *k, int mon)
{
    int64_t st[ORC_MAX_DIMS], N, maxn = 1;
    oval *Ap, *As;
    int i;
    if (check_args(d, n, k, mon)) return ORC_EINVAL;
    row_major_strides(d, n, st);
    N = volume(d, n);
    for (i = 0; i < d; i++)
        if (n[i] > maxn) maxn = n[i];
    Ap = (oval *)malloc(sizeof(oval) * maxn);
    As = (oval *)malloc(sizeof(oval) * maxn);
    if (!Ap || !As) { free(Ap); free(As); return ORC_ENOMEM; }
    memcpy(out, A, sizeof(oval) * N);
    for (i = 0; i < d; i++) for_each_row(out, d, n, st, 0, i, k[i], mon, bdbs_row, Ap, As);
    free(Ap);
    free(As);
    return ORC_OK;
}

/* ------------------------------------------------------------------------
 * Box-complement (Sec. 5, Fig. "exsum-code" and its full form
 * Fig. "exsum-code-full", with Prefix-Along-Dim, BDBS-Along-Dim and
 * Add-Contribution from App. C).
 * ------------------------------------------------------------------------ */

/* Copies the view with dimensions < fixed pinned at their last index. */
static void copy_view(oval *dst, const oval *src, int d, const int64_t *n, const int64_t *st,
                      int fixed)
{
    int64_t lo[ORC_MAX_DIMS], hi[ORC_MAX_DIMS], x[ORC_MAX_DIMS], o;
    int i;
    for (i = 0; i < d; i++) {
        lo[i] = i < fixed ? n[i] - 1 : 0;
        hi[i] = i < fixed ? n[i] : n[i];
        x[i] = lo[i];
    }
    do {
        o = offset_of(d, x, st);
        dst[o] = src[o];
    } while (next_coord(d, x, lo, hi));
}

/* Add-Contribution (App. C, Fig. "add-contribution-code"): for every x of
 * the output B, B[x] (+)= V[n_1..n_{dim-1} pinned, x_dim + off, x_{dim+1}..]
 * when x_dim + off lies inside [0, n_dim).  The figure writes "=" where the
 * text (Sec. 5, "Adding in the Contribution") means the contribution is added
 * in; the figure also checks only the upper bound, and the lower bound is
 * needed for the prefix step's offset of -1. */
static void add_contribution(oval *B, const oval *V, int d, const int64_t *n, const int64_t *st,
                             int dim, int64_t off, int mon)
{
    int64_t lo[ORC_MAX_DIMS], x[ORC_MAX_DIMS], src[ORC_MAX_DIMS];
    int i;
    for (i = 0; i < d; i++) lo[i] = x[i] = 0;
    do {
        int64_t t = x[dim] + off;
        if (t >= 0 && t < n[dim]) {
            for (i = 0; i < d; i++) src[i] = i < dim ? n[i] - 1 : x[i];
            src[dim] = t;
            {
                int64_t o = offset_of(d, x, st);
                B[o] = combine(mon, B[o], V[offset_of(d, src, st)]);
            }
        }
    } while (next_coord(d, x, lo, n));
}

int orc_box_complement(const oval *A, oval *B, int d, const int64_t *n, const int64_t *k, int mon)
{
    int64_t st[ORC_MAX_DIMS], N, maxn = 1, x;
    oval *Aw, *Apre, *Asuf, *t1, *t2, *pin;
    int i, j;
    if (check_args(d, n, k, mon)) return ORC_EINVAL;
    row_major_strides(d, n, st);
    N = volume(d, n);
    for (i = 0; i < d; i++)
        if (n[i] > maxn) maxn = n[i];
    Aw = (oval *)malloc(sizeof(oval) * N);
    Apre = (oval *)malloc(sizeof(oval) * N);
    Asuf = (oval *)malloc(sizeof(oval) * N);
    t1 = (oval *)malloc(sizeof(oval) * maxn);
    t2 = (oval *)malloc(sizeof(oval) * maxn);
    if (!Aw || !Apre || !Asuf || !t1 || !t2) {
        free(Aw); free(Apre); free(Asuf); free(t1); free(t2);
        return ORC_ENOMEM;
    }
    /* The output starts at the identity; A_p starts as the input. */
    for (x = 0; x < N; x++) B[x] = identity(mon);
    memcpy(Apre, A, sizeof(oval) * N);

    for (i = 0; i < d; i++) {
        /* The view of step i pins dimensions 0..i-1 at their last index, i.e.
         * it holds the reduction of A over those dimensions (A_p carries the
         * prefix of the previous step, whose last slice is the total). */
        int64_t base = 0;
        for (j = 0; j < i; j++) base += (n[j] - 1) * st[j];
        pin = Aw + base;

        /* PREFIX STEP */
        copy_view(Aw, Apre, d, n, st, i);
        copy_view(Asuf, Apre, d, n, st, i);          /* save input to the suffix step */
        for_each_row(pin, d, n, st, i, i, 1, mon, prefix_row, t1, t2);   /* Prefix-Along-Dim */
        copy_view(Apre, Aw, d, n, st, i);            /* save prefix for the next step */
        for (j = i + 1; j < d; j++)                  /* BDBS-Along-Dim for dims > i */
            for_each_row(pin, d, n, st, i, j, k[j], mon, bdbs_row, t1, t2);
        add_contribution(B, Aw, d, n, st, i, -1, mon);

        /* SUFFIX STEP */
        copy_view(Aw, Asuf, d, n, st, i);
        for_each_row(pin, d, n, st, i, i, 1, mon, suffix_row, t1, t2);   /* Suffix-Along-Dim */
        for (j = i + 1; j < d; j++)
            for_each_row(pin, d, n, st, i, j, k[j], mon, bdbs_row, t1, t2);
        add_contribution(B, Aw, d, n, st, i, k[i], mon);
    }
    free(Aw); free(Apre); free(Asuf); free(t1); free(t2);
    return ORC_OK;
}

/* ------------------------------------------------------------------------
 * Corners algorithm (App. A), d = 2 and d = 3.
 *
 * The excluded region of the box at x is split into 2^d disjoint regions,
 * one per string b in {P,S}^d.  Region b constrains every dimension i to one
 * side of a threshold: P means y_i < t_i, S means y_i >= t_i, and t_i is
 * either x_i ("lo") or x_i + k_i ("hi").  With T_b the full-tensor
 * combination of inclusive prefixes (P) and suffixes (S) along each
 * dimension, region b reduces to one element of T_b.
 *
 * The paper gives the 2-D picture only and no higher-dimensional
 * construction.  The threshold choices below are this oracle's own; the test
 * suite checks exhaustively over the 3^d cell pattern (below / inside /
 * above the box in each dimension) that they partition the complement of
 * the box exactly.
 *   d = 2: dimension 1 uses "hi" iff b_2 = S; dimension 2 uses "hi" iff
 *          b_1 = P (a pinwheel around the box).
 *   d = 3: dimension i uses "hi" iff b_{(i mod 3) + 1} = S.
 * ------------------------------------------------------------------------ */

static int corner_uses_hi(int d, int dim, unsigned mask)
{
    /* bit i of mask set <=> b_{i+1} = S */
    if (d == 2) {
        if (dim == 0) return (mask >> 1) & 1u;
        return !((mask >> 0) & 1u);
    }
    return (mask >> ((dim + 1) % 3)) & 1u;
}

int orc_corner_threshold_hi(int d, int dim, unsigned mask)
{
    if ((d != 2 && d != 3) || dim < 0 || dim >= d) return -1;
    return corner_uses_hi(d, dim, mask);
}

int orc_corners(const oval *A, oval *B, int d, const int64_t *n, const int64_t *k, int mon)
{
    int64_t st[ORC_MAX_DIMS], N, lo[ORC_MAX_DIMS], x[ORC_MAX_DIMS], idx[ORC_MAX_DIMS], o;
    oval *T;
    unsigned mask;
    int i;
    if (check_args(d, n, k, mon)) return ORC_EINVAL;
    if (d != 2 && d != 3) return ORC_EINVAL;
    row_major_strides(d, n, st);
    N = volume(d, n);
    T = (oval *)malloc(sizeof(oval) * N);
    if (!T) return ORC_ENOMEM;
    for (o = 0; o < N; o++) B[o] = identity(mon);

    for (mask = 0; mask < (1u << d); mask++) {
        /* T_b: full-tensor prefix (P) or suffix (S) along every dimension. */
        memcpy(T, A, sizeof(oval) * N);
        for (i = 0; i < d; i++)
            for_each_row(T, d, n, st, 0, i, 1, mon, ((mask >> i) & 1u) ? suffix_row : prefix_row,
                         NULL, NULL);
        for (i = 0; i < d; i++) lo[i] = x[i] = 0;
        do {
            int empty = 0;
            for (i = 0; i < d && !empty; i++) {
                int is_suffix = (mask >> i) & 1u;
                int64_t t = corner_uses_hi(d, i, mask) ? x[i] + k[i] : x[i];
                if (!is_suffix) {
                    /* y_i < t  ->  prefix ends at min(t, n_i) - 1 */
                    int64_t e = (t < n[i] ? t : n[i]) - 1;
                    if (e < 0) empty = 1;
                    idx[i] = e;
                } else {
                    /* y_i >= t ->  suffix starts at t */
                    if (t >= n[i]) empty = 1;
                    idx[i] = t;
                }
            }
            if (!empty) {
                o = offset_of(d, x, st);
                B[o] = combine(mon, B[o], T[offset_of(d, idx, st)]);
            }
        } while (next_coord(d, x, lo, n));
    }
    free(T);
    return ORC_OK;
}

/* ------------------------------------------------------------------------
 * Weak algorithms (need an inverse), integer + only.
 * ------------------------------------------------------------------------ */

/* Summed-area table (Sec. 1): d-dimensional inclusive prefix, then
 * inclusion-exclusion over the 2^d corners of each box. */
int orc_sat_included(const oval *A, oval *out, int d, const int64_t *n, const int64_t *k)
{
    int64_t st[ORC_MAX_DIMS], N, lo[ORC_MAX_DIMS], x[ORC_MAX_DIMS], c[ORC_MAX_DIMS];
    oval *S;
    unsigned mask;
    int i;
    if (check_args(d, n, k, ORC_ADD_I64)) return ORC_EINVAL;
    row_major_strides(d, n, st);
    N = volume(d, n);
    S = (oval *)malloc(sizeof(oval) * N);
    if (!S) return ORC_ENOMEM;
    memcpy(S, A, sizeof(oval) * N);
    for (i = 0; i < d; i++) for_each_row(S, d, n, st, 0, i, 1, ORC_ADD_I64, prefix_row, NULL, NULL);
    for (i = 0; i < d; i++) lo[i] = x[i] = 0;
    do {
        uint64_t acc = 0;
        for (mask = 0; mask < (1u << d); mask++) {
            int zero = 0, parity = 0;
            for (i = 0; i < d; i++) {
                if ((mask >> i) & 1u) {
                    c[i] = x[i] - 1;
                    parity ^= 1;
                } else {
                    c[i] = (x[i] + k[i] < n[i] ? x[i] + k[i] : n[i]) - 1;
                }
                if (c[i] < 0) zero = 1;
            }
            if (zero) continue;
            if (parity)
                acc -= (uint64_t)S[offset_of(d, c, st)].i;
            else
                acc += (uint64_t)S[offset_of(d, c, st)].i;
        }
        out[offset_of(d, x, st)].i = (int64_t)acc;
    } while (next_coord(d, x, lo, n));
    free(S);
    return ORC_OK;
}

/* BDBS complement (Sec. 1): total minus the BDBS included sum. */
int orc_bdbsc(const oval *A, oval *out, int d, const int64_t *n, const int64_t *k)
{
    int64_t N, x;
    uint64_t total = 0;
    int rc;
    if (check_args(d, n, k, ORC_ADD_I64)) return ORC_EINVAL;
    N = volume(d, n);
    rc = orc_bdbs(A, out, d, n, k, ORC_ADD_I64);
    if (rc) return rc;
    for (x = 0; x < N; x++) total += (uint64_t)A[x].i;
    for (x = 0; x < N; x++) out[x].i = (int64_t)(total - (uint64_t)out[x].i);
    return ORC_OK;
}
