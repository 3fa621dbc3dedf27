/*
 * exsum_oracle_omp.c -- the box-complement oracle of exsum_oracle.c with its
 * independent loops spread over the host cores by OpenMP.
 *
 * TEST INFRASTRUCTURE ONLY.  It times the all-core CPU baseline of the
 * benchmark; the tests check that its results equal those of the
 * single-threaded oracle bit for bit.  It performs the same steps in the
 * same order as orc_box_complement (Sec. 5, Fig. "exsum-code-full" with the
 * subroutines of App. C): every row of a Prefix-/Suffix-Along-Dim or
 * BDBS-Along-Dim step, and every element of a copy or an Add-Contribution,
 * is still computed by one thread in the same operand order; only different
 * rows (elements) run on different threads.  It shares no code with the
 * CUDA path.  Built without OpenMP it runs on one thread.
 *
 * Conventions: as exsum_oracle.c (row-major, 0-based, 8-byte cells, the
 * monoid codes 0..3 = int +, int max, double +, double max).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORCP_MAX_DIMS 8

typedef union {
    int64_t i;
    double f;
} cell;

static cell ident(int mon)
{
    cell e;
    switch (mon) {
    case 0: e.i = 0; break;
    case 1: e.i = INT64_MIN; break;
    case 2: e.f = 0.0; break;
    default: e.f = -INFINITY; break;
    }
    return e;
}

static cell comb(int mon, cell a, cell b)
{
    cell r;
    switch (mon) {
    case 0: r.i = (int64_t)((uint64_t)a.i + (uint64_t)b.i); break;
    case 1: r.i = a.i > b.i ? a.i : b.i; break;
    case 2: r.f = a.f + b.f; break;
    default: r.f = a.f > b.f ? a.f : b.f; break;
    }
    return r;
}

int orcp_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Offset of the idx-th point of the box [0, ext) (row-major over the
 * dimensions with ext > 1 ... all d of them), strides st. */
static int64_t point_offset(int d, const int64_t *ext, const int64_t *st, int64_t idx)
{
    int64_t o = 0;
    int i;
    for (i = d - 1; i >= 0; i--) {
        const int64_t c = idx % ext[i];
        idx /= ext[i];
        o += c * st[i];
    }
    return o;
}

static void row_prefix(cell *r, int64_t s, int64_t len, int mon)
{
    int64_t x;
    for (x = 1; x < len; x++) r[x * s] = comb(mon, r[(x - 1) * s], r[x * s]);
}

static void row_suffix(cell *r, int64_t s, int64_t len, int mon)
{
    int64_t x;
    for (x = len - 2; x >= 0; x--) r[x * s] = comb(mon, r[x * s], r[(x + 1) * s]);
}

/* BDBS-1D on one row (Sec. 3): block prefixes, block suffixes, combine. */
static void row_bdbs(cell *r, int64_t s, int64_t len, int64_t k, int mon, cell *Ap, cell *As)
{
    int64_t b0, end, x;
    for (b0 = 0; b0 < len; b0 += k) {
        end = b0 + k < len ? b0 + k : len;
        Ap[b0] = r[b0 * s];
        for (x = b0 + 1; x < end; x++) Ap[x] = comb(mon, Ap[x - 1], r[x * s]);
    }
    for (b0 = 0; b0 < len; b0 += k) {
        end = b0 + k < len ? b0 + k : len;
        As[end - 1] = r[(end - 1) * s];
        for (x = end - 2; x >= b0; x--) As[x] = comb(mon, r[x * s], As[x + 1]);
    }
    for (x = 0; x < len; x++) {
        cell v = As[x];
        if (x % k != 0) {
            int64_t j = x + k - 1;
            int64_t next_block = (x / k + 1) * k;
            if (j < len)
                v = comb(mon, As[x], Ap[j]);
            else if (next_block <= len - 1)
                v = comb(mon, As[x], Ap[len - 1]);
        }
        r[x * s] = v;
    }
}

/* kind: 0 prefix, 1 suffix, 2 BDBS with box k.  Rows along `dim` of the
 * view at `pin` whose dimensions < fixed are pinned; one row per thread. */
static void each_row(cell *pin, int d, const int64_t *n, const int64_t *st, int fixed, int dim,
                     int64_t k, int mon, int kind, int64_t maxn)
{
    int64_t ext[ORCP_MAX_DIMS], rows = 1;
    int i;
    for (i = 0; i < d; i++) {
        ext[i] = (i < fixed || i == dim) ? 1 : n[i];
        rows *= ext[i];
    }
#pragma omp parallel
    {
        cell *Ap = kind == 2 ? (cell *)malloc(sizeof(cell) * maxn) : NULL;
        cell *As = kind == 2 ? (cell *)malloc(sizeof(cell) * maxn) : NULL;
        int64_t r;
#pragma omp for schedule(static)
        for (r = 0; r < rows; r++) {
            cell *row = pin + point_offset(d, ext, st, r);
            if (kind == 0)
                row_prefix(row, st[dim], n[dim], mon);
            else if (kind == 1)
                row_suffix(row, st[dim], n[dim], mon);
            else
                row_bdbs(row, st[dim], n[dim], k, mon, Ap, As);
        }
        free(Ap);
        free(As);
    }
}

/* dst = src on the view with dimensions < fixed pinned at their last index. */
static void copy_pinned(cell *dst, const cell *src, int d, const int64_t *n, const int64_t *st, int fixed)
{
    int64_t ext[ORCP_MAX_DIMS], cnt = 1, base = 0, p;
    int i;
    for (i = 0; i < d; i++) {
        ext[i] = i < fixed ? 1 : n[i];
        if (i < fixed) base += (n[i] - 1) * st[i];
        cnt *= ext[i];
    }
#pragma omp parallel for schedule(static)
    for (p = 0; p < cnt; p++) {
        const int64_t o = base + point_offset(d, ext, st, p);
        dst[o] = src[o];
    }
}

/* Add-Contribution (App. C): B[x] (+)= V[n_1..n_{dim-1} pinned, x_dim + off, ...]
 * when x_dim + off lies in [0, n_dim). */
static void add_contrib(cell *B, const cell *V, int d, const int64_t *n, const int64_t *st, int dim,
                        int64_t off, int mon, int64_t N)
{
    int64_t p;
#pragma omp parallel for schedule(static)
    for (p = 0; p < N; p++) {
        int64_t x[ORCP_MAX_DIMS], rest = p, so = 0;
        int i;
        for (i = d - 1; i >= 0; i--) {
            x[i] = rest % n[i];
            rest /= n[i];
        }
        {
            const int64_t t = x[dim] + off;
            if (t < 0 || t >= n[dim]) continue;
            for (i = 0; i < d; i++) so += (i < dim ? n[i] - 1 : (i == dim ? t : x[i])) * st[i];
            B[p] = comb(mon, B[p], V[so]);
        }
    }
}

int orcp_box_complement(const cell *A, cell *B, int d, const int64_t *n, const int64_t *k, int mon)
{
    int64_t st[ORCP_MAX_DIMS], N = 1, maxn = 1, x;
    cell *Aw, *Apre, *Asuf;
    int i, j;
    if (d < 1 || d > ORCP_MAX_DIMS || mon < 0 || mon > 3) return -1;
    for (i = 0; i < d; i++) {
        if (n[i] < 1 || k[i] < 1 || k[i] > n[i]) return -1;
        N *= n[i];
        if (n[i] > maxn) maxn = n[i];
    }
    st[d - 1] = 1;
    for (i = d - 2; i >= 0; i--) st[i] = st[i + 1] * n[i + 1];
    Aw = (cell *)malloc(sizeof(cell) * N);
    Apre = (cell *)malloc(sizeof(cell) * N);
    Asuf = (cell *)malloc(sizeof(cell) * N);
    if (!Aw || !Apre || !Asuf) {
        free(Aw); free(Apre); free(Asuf);
        return -2;
    }
#pragma omp parallel for schedule(static)
    for (x = 0; x < N; x++) {
        B[x] = ident(mon);
        Apre[x] = A[x];
    }
    for (i = 0; i < d; i++) {
        int64_t base = 0;
        cell *pin;
        for (j = 0; j < i; j++) base += (n[j] - 1) * st[j];
        pin = Aw + base;
        /* prefix step */
        copy_pinned(Aw, Apre, d, n, st, i);
        copy_pinned(Asuf, Apre, d, n, st, i);
        each_row(pin, d, n, st, i, i, 1, mon, 0, maxn);
        copy_pinned(Apre, Aw, d, n, st, i);
        for (j = i + 1; j < d; j++) each_row(pin, d, n, st, i, j, k[j], mon, 2, maxn);
        add_contrib(B, Aw, d, n, st, i, -1, mon, N);
        /* suffix step */
        copy_pinned(Aw, Asuf, d, n, st, i);
        each_row(pin, d, n, st, i, i, 1, mon, 1, maxn);
        for (j = i + 1; j < d; j++) each_row(pin, d, n, st, i, j, k[j], mon, 2, maxn);
        add_contrib(B, Aw, d, n, st, i, k[i], mon, N);
    }
    free(Aw); free(Apre); free(Asuf);
    return 0;
}
