/*
 * ddsg_oracle.c -- TEST INFRASTRUCTURE, NOT PRODUCT CODE.
 *
 * A plain, slow, obviously-correct FP64 CPU restatement of the cut-HDMR
 * adaptive-sparse-grid ("DDSG") interpolant of Eftekhari & Scheidegger,
 * "High-Dimensional Dynamic Stochastic Model Representation" (arXiv 2202.06555).
 * It exists only to be compared against the CUDA library. Only tests/,
 * __graft_entry__.smoke() and bench.py's cpu_baseline / reference arm may load
 * it. It shares no code, header or table with the CUDA library.
 *
 * Compiled with -O2 -ffp-contract=off (no FMA contraction) so that every sum
 * is evaluated left to right in round-to-nearest FP64.
 *
 * Conventions (paper Sec. 3.1 with the boundary-augmented basis, the variant
 * the paper's Table 2 grid counts confirm):
 *   level 1 : one node at 1/2, phi == 1 on [0,1]                      (index 1)
 *   level 2 : nodes 0 and 1, phi = max(0, 1 - |2x - i|), i in {0, 2}
 *   level l>=3 : nodes i/2^(l-1), i odd, phi = max(0, 1 - |2^(l-1) x - i|)   (eq. 3.1)
 *   d-linear basis = product over the component's dimensions          (eq. 3.2)
 *   level constraint of a level-L grid: sum_j (l_j - 1) <= L - 1        (eq. 3.5)
 * A component u (|u| = k, dims ascending) owns points p = (l_p, i_p) and
 * surpluses alpha_p in R^m. The empty component (k = 0) has one point whose
 * basis value is the empty product 1 and whose surplus is f(anchor).
 *
 * Parity status of every function is listed in the pin tests
 * (tests/test_oracle_pins.py); all functions below are pinned.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define KMAX 8

/* ------------------------------------------------------------------ */
/* 1D basis (Sec. 3.1, eq. 3.1 with boundary nodes)                    */
/* ------------------------------------------------------------------ */

double orc_phi1d(int l, uint32_t i, double x)
{
    if (l == 1) return 1.0;
    double y = ldexp(x, l - 1);               /* 2^(l-1) x, exact */
    double t = 1.0 - fabs(y - (double)i);
    return t > 0.0 ? t : 0.0;
}

/* Support test in exact arithmetic: phi_{l,i}(x) > 0 as a real number. */
int orc_active1d(int l, uint32_t i, double x)
{
    if (l == 1) return 1;
    double y = ldexp(x, l - 1);
    return (y > (double)i - 1.0) && (y < (double)i + 1.0);
}

/* node position of (l, i) */
double orc_node1d(int l, uint32_t i)
{
    if (l == 1) return 0.5;
    return ldexp((double)i, -(l - 1));
}

/* integral of phi_{l,i} over [0,1] (used by eq. 3.7) */
double orc_int1d(int l, uint32_t i)
{
    (void)i;
    if (l == 1) return 1.0;
    if (l == 2) return 0.25;
    return ldexp(1.0, -(l - 1));
}

/* number of 1D nodes of level l */
static int64_t n1d(int l)
{
    if (l == 1) return 1;
    if (l == 2) return 2;
    return (int64_t)1 << (l - 2);
}

static uint32_t idx1d(int l, int64_t r)   /* r-th node of level l */
{
    if (l == 1) return 1;
    if (l == 2) return (uint32_t)(2 * r);
    return (uint32_t)(2 * r + 1);
}

/* ------------------------------------------------------------------ */
/* Regular sparse grids (eq. 3.5)                                      */
/* ------------------------------------------------------------------ */

/* Enumerate level tuples of k dims with sum(l-1) == s in lexicographic order. */
static int64_t tuples_with_sum(int k, int s, int *out /* cap*k or NULL */)
{
    if (k == 0) return s == 0 ? 1 : 0;
    int64_t cnt = 0;
    int lv[KMAX];
    /* odometer over excess e_j = l_j - 1 >= 0, sum e = s, lexicographic in e */
    for (int j = 0; j < k; ++j) lv[j] = 0;
    lv[k - 1] = s;
    for (;;) {
        if (out) for (int j = 0; j < k; ++j) out[cnt * k + j] = lv[j] + 1;
        ++cnt;
        /* next composition of s into k parts, lexicographically increasing */
        int j = k - 2;
        while (j >= 0) {
            int rest = 0;
            for (int q = j + 1; q < k; ++q) rest += lv[q];
            if (rest > 0) {
                lv[j] += 1;
                rest -= 1;
                for (int q = j + 1; q < k; ++q) lv[q] = 0;
                lv[k - 1] = rest;
                break;
            }
            --j;
        }
        if (j < 0) break;
    }
    return cnt;
}

/* Points of the regular level-L grid of a k-dim component, canonical order:
 * (level sum, level tuple lexicographic, index tuple lexicographic).
 * Returns the number of points; writes levels/indices (npts*KMAX) if non-NULL. */
int64_t orc_regular_grid(int k, int L, uint8_t *levels, uint32_t *indices)
{
    int64_t np = 0;
    int tup[4096 * KMAX];
    for (int s = 0; s <= (k == 0 ? 0 : L - 1); ++s) {
        int64_t nt = tuples_with_sum(k, s, NULL);
        if (nt * k > 4096 * KMAX) return -1;
        tuples_with_sum(k, s, tup);
        for (int64_t t = 0; t < nt; ++t) {
            int *lv = &tup[t * k];
            int64_t tot = 1;
            for (int j = 0; j < k; ++j) tot *= n1d(lv[j]);
            for (int64_t r = 0; r < tot; ++r) {
                if (levels) {
                    int64_t rr = r;
                    for (int j = k - 1; j >= 0; --j) {
                        int64_t nj = n1d(lv[j]);
                        levels[np * KMAX + j] = (uint8_t)lv[j];
                        indices[np * KMAX + j] = idx1d(lv[j], rr % nj);
                        rr /= nj;
                    }
                    for (int j = k; j < KMAX; ++j) {
                        levels[np * KMAX + j] = 0;
                        indices[np * KMAX + j] = 0;
                    }
                }
                ++np;
            }
        }
    }
    return np;
}

/* ------------------------------------------------------------------ */
/* Active-set hash: splitmix64 finalizer (Steele et al. 2014)          */
/* ------------------------------------------------------------------ */

static uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t orc_point_key(int32_t comp, int k, const uint8_t *lv, const uint32_t *ix)
{
    uint64_t key = (uint64_t)(uint32_t)comp;
    for (int j = 0; j < k; ++j)
        key = mix64(key ^ ((uint64_t)lv[j] << 40) ^ (uint64_t)ix[j]);
    return mix64(key + 0x9E3779B97F4A7C15ULL);
}

/* ------------------------------------------------------------------ */
/* Tables of a whole HDMR expansion                                    */
/* ------------------------------------------------------------------ */
/*
 * C components; comp_k[c]; comp_dims[c*KMAX + j] (ascending, 0-based);
 * comp_off[c]..comp_off[c+1] are the points of c in levels/indices/alpha
 * (levels, indices: P*KMAX; alpha: P*m, FP64).
 */

static int is_subset(int ka, const int32_t *a, int kb, const int32_t *b)
{
    /* a subset of b (both ascending) */
    int q = 0;
    for (int j = 0; j < ka; ++j) {
        while (q < kb && b[q] < a[j]) ++q;
        if (q >= kb || b[q] != a[j]) return 0;
        ++q;
    }
    return 1;
}

/* eq. 4.2: b_v = sum over accepted u containing v of (-1)^(|u|-|v|) */
void orc_b_coeffs(int C, const int32_t *comp_k, const int32_t *comp_dims, double *b)
{
    for (int v = 0; v < C; ++v) {
        double s = 0.0;
        for (int u = 0; u < C; ++u) {
            if (comp_k[u] < comp_k[v]) continue;
            if (!is_subset(comp_k[v], &comp_dims[v * KMAX], comp_k[u], &comp_dims[u * KMAX]))
                continue;
            s += ((comp_k[u] - comp_k[v]) % 2) ? -1.0 : 1.0;
        }
        b[v] = s;
    }
}

/* canonical coordinate: (x - lo)/(hi - lo), clamped to [0,1] */
static double canon(double x, double lo, double hi)
{
    double c = (x - lo) / (hi - lo);
    if (c < 0.0) c = 0.0;
    if (c > 1.0) c = 1.0;
    return c;
}

/* value and support test of point p of component c at canonical query xc */
static int point_basis(int k, const int32_t *dims, const uint8_t *lv, const uint32_t *ix,
                       const double *xc, double *phi)
{
    double w = 1.0;
    for (int j = 0; j < k; ++j) {
        double xj = xc[dims[j]];
        if (!orc_active1d(lv[j], ix[j], xj)) { *phi = 0.0; return 0; }
        w *= orc_phi1d(lv[j], ix[j], xj);
    }
    *phi = w;
    return 1;
}

/*
 * Brute-force evaluation (every point of every component is tested; no pruning).
 *   form 0 (paper, eq. 4.2): y = sum_v b_v s_v(x_v),  s_v = sum_{p in G_v} alpha_p phi_p
 *   form 1 (slice-free):     y = sum_u sum_{p in G_u, all l_pj >= 2} alpha_p phi_p
 * Queries x are physical (n*d), mapped to [0,1] by lo/hi and clamped.
 * Outputs (each optional): y (n*m), S = sum of |terms| (n*m),
 * hash = XOR of point keys over summed active points (n), count (n).
 * Components with b_v == 0 are skipped in form 0.
 */
void orc_eval(int d, int m, int C, const int32_t *comp_k, const int32_t *comp_dims,
              const int64_t *comp_off, const uint8_t *levels, const uint32_t *indices,
              const double *alpha, const double *b, const double *lo, const double *hi,
              int form, int64_t n, const double *x, double *y, double *S,
              uint64_t *hash, int32_t *count)
{
    double *xc = (double *)malloc(sizeof(double) * (size_t)d);
    double *acc = (double *)malloc(sizeof(double) * (size_t)m);
    double *sab = (double *)malloc(sizeof(double) * (size_t)m);
    for (int64_t q = 0; q < n; ++q) {
        int finite = 1;
        for (int i = 0; i < d; ++i) {
            if (!isfinite(x[q * d + i]) || !isfinite((x[q * d + i] - lo[i]) / (hi[i] - lo[i])))
                finite = 0;
            xc[i] = canon(x[q * d + i], lo[i], hi[i]);
        }
        if (!finite) {   /* a non-finite coordinate gives a NaN row and an empty active set */
            if (y) for (int j = 0; j < m; ++j) y[q * m + j] = NAN;
            if (S) for (int j = 0; j < m; ++j) S[q * m + j] = NAN;
            if (hash) hash[q] = 0;
            if (count) count[q] = 0;
            continue;
        }
        for (int j = 0; j < m; ++j) { acc[j] = 0.0; sab[j] = 0.0; }
        uint64_t h = 0;
        int32_t cnt = 0;
        for (int c = 0; c < C; ++c) {
            double bc = (form == 0) ? b[c] : 1.0;
            if (form == 0 && bc == 0.0) continue;
            int k = comp_k[c];
            const int32_t *dims = &comp_dims[c * KMAX];
            for (int64_t p = comp_off[c]; p < comp_off[c + 1]; ++p) {
                const uint8_t *lv = &levels[p * KMAX];
                const uint32_t *ix = &indices[p * KMAX];
                if (form == 1) {
                    int interior = 1;
                    for (int j = 0; j < k; ++j) if (lv[j] < 2) interior = 0;
                    if (!interior) continue;
                }
                double phi;
                if (!point_basis(k, dims, lv, ix, xc, &phi)) continue;
                double w = bc * phi;
                for (int j = 0; j < m; ++j) {
                    double t = w * alpha[p * m + j];
                    acc[j] += t;
                    sab[j] += fabs(t);
                }
                h ^= orc_point_key(c, k, lv, ix);
                ++cnt;
            }
        }
        if (y) for (int j = 0; j < m; ++j) y[q * m + j] = acc[j];
        if (S) for (int j = 0; j < m; ++j) S[q * m + j] = sab[j];
        if (hash) hash[q] = h;
        if (count) count[q] = cnt;
    }
    free(xc);
    free(acc);
    free(sab);
}

/* s_c(x) of one component at a canonical query (brute force) */
static void comp_interp(int m, int k, const int32_t *dims, int64_t p0, int64_t p1,
                        const uint8_t *levels, const uint32_t *indices, const double *alpha,
                        const double *xc, double *out)
{
    for (int j = 0; j < m; ++j) out[j] = 0.0;
    for (int64_t p = p0; p < p1; ++p) {
        double phi;
        if (!point_basis(k, dims, &levels[p * KMAX], &indices[p * KMAX], xc, &phi)) continue;
        for (int j = 0; j < m; ++j) out[j] += phi * alpha[p * m + j];
    }
}

/*
 * Literal telescopic sum, eq. 3.16: y = sum_{u in U} sum_{v subset u} (-1)^{|u|-|v|} I f(xbar\x_v),
 * where I f(xbar\x_v) is component v's interpolant. Each subset v of u is looked
 * up in U by its dimension list. Independent of b; for small expansions only.
 * Returns -1 if some subset is missing from U (U not downward closed).
 */
int orc_eval_telescopic(int d, int m, int C, const int32_t *comp_k, const int32_t *comp_dims,
                        const int64_t *comp_off, const uint8_t *levels, const uint32_t *indices,
                        const double *alpha, const double *lo, const double *hi,
                        int64_t n, const double *x, double *y)
{
    double *xc = (double *)malloc(sizeof(double) * (size_t)d);
    double *sv = (double *)malloc(sizeof(double) * (size_t)m);
    int rc = 0;
    for (int64_t q = 0; q < n && rc == 0; ++q) {
        for (int i = 0; i < d; ++i) xc[i] = canon(x[q * d + i], lo[i], hi[i]);
        for (int j = 0; j < m; ++j) y[q * m + j] = 0.0;
        for (int u = 0; u < C && rc == 0; ++u) {
            int k = comp_k[u];
            for (int mask = 0; mask < (1 << k); ++mask) {
                int32_t vd[KMAX];
                int kv = 0;
                for (int j = 0; j < k; ++j)
                    if (mask & (1 << j)) vd[kv++] = comp_dims[u * KMAX + j];
                int v = -1;
                for (int c = 0; c < C; ++c) {
                    if (comp_k[c] != kv) continue;
                    if (kv == 0 || memcmp(&comp_dims[c * KMAX], vd, sizeof(int32_t) * kv) == 0) {
                        v = c;
                        break;
                    }
                }
                if (v < 0) { rc = -1; break; }
                comp_interp(m, kv, &comp_dims[v * KMAX], comp_off[v], comp_off[v + 1],
                            levels, indices, alpha, xc, sv);
                double sg = ((k - kv) % 2) ? -1.0 : 1.0;
                for (int j = 0; j < m; ++j) y[q * m + j] += sg * sv[j];
            }
        }
    }
    free(xc);
    free(sv);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Hierarchization (surplus = value - coarser interpolant, Sec. 3.1)  */
/* ------------------------------------------------------------------ */

static int level_sum(int k, const uint8_t *lv)
{
    int s = 0;
    for (int j = 0; j < k; ++j) s += lv[j] - 1;
    return s;
}

/*
 * For every component and point p, in increasing level sum:
 *   alpha_p = v_p - sum_{q in G_c, levelsum(q) < levelsum(p)} alpha_q phi_q(x_p)
 * values, alpha: P*m. Points of one layer do not interact (finer hats vanish
 * at coarser nodes), so the order inside a layer is irrelevant.
 */
void orc_hierarchize(int m, int C, const int32_t *comp_k, const int64_t *comp_off,
                     const uint8_t *levels, const uint32_t *indices, const double *values,
                     double *alpha)
{
    for (int c = 0; c < C; ++c) {
        int k = comp_k[c];
        int64_t p0 = comp_off[c], p1 = comp_off[c + 1];
        int maxs = 0;
        for (int64_t p = p0; p < p1; ++p) {
            int s = level_sum(k, &levels[p * KMAX]);
            if (s > maxs) maxs = s;
        }
        for (int s = 0; s <= maxs; ++s) {
            for (int64_t p = p0; p < p1; ++p) {
                if (level_sum(k, &levels[p * KMAX]) != s) continue;
                double xp[KMAX];
                for (int j = 0; j < k; ++j)
                    xp[j] = orc_node1d(levels[p * KMAX + j], indices[p * KMAX + j]);
                for (int j = 0; j < m; ++j) alpha[p * m + j] = values[p * m + j];
                for (int64_t q = p0; q < p1; ++q) {
                    if (level_sum(k, &levels[q * KMAX]) >= s) continue;
                    double w = 1.0;
                    int act = 1;
                    for (int j = 0; j < k && act; ++j) {
                        int lq = levels[q * KMAX + j];
                        uint32_t iq = indices[q * KMAX + j];
                        if (!orc_active1d(lq, iq, xp[j])) act = 0;
                        else w *= orc_phi1d(lq, iq, xp[j]);
                    }
                    if (!act) continue;
                    for (int j = 0; j < m; ++j) alpha[p * m + j] -= w * alpha[q * m + j];
                }
            }
        }
    }
}

/* Node coordinates of points p0..p1-1 of a component: out[(p-p0)*k + j]. */
void orc_nodes(int k, int64_t p0, int64_t p1, const uint8_t *levels, const uint32_t *indices,
               double *out)
{
    for (int64_t p = p0; p < p1; ++p)
        for (int j = 0; j < k; ++j)
            out[(p - p0) * k + j] = orc_node1d(levels[p * KMAX + j], indices[p * KMAX + j]);
}

/* ------------------------------------------------------------------ */
/* Adaptive refinement (eq. 3.8)                                       */
/* ------------------------------------------------------------------ */

/* children of (l, i) in 1D: returns count (0..2) */
static int children1d(int l, uint32_t i, uint32_t *ci)
{
    if (l == 1) { ci[0] = 0; ci[1] = 2; return 2; }
    if (l == 2) { ci[0] = (i == 0) ? 1u : 3u; return 1; }
    ci[0] = 2 * i - 1;
    ci[1] = 2 * i + 1;
    return 2;
}

/* parent of (l, i) in 1D, l >= 2 */
static void parent1d(int l, uint32_t i, int *pl, uint32_t *pi)
{
    if (l == 2) { *pl = 1; *pi = 1; return; }
    if (l == 3) { *pl = 2; *pi = (i == 1) ? 0u : 2u; return; }
    *pl = l - 1;
    /* (l, i) with i odd comes from (l-1, i') where i = 2i' +- 1 and i' odd */
    uint32_t a = (i - 1) / 2, bb = (i + 1) / 2;
    *pi = (a & 1u) ? a : bb;
}

typedef struct { uint8_t lv[KMAX]; uint32_t ix[KMAX]; } opt_t;

static int g_sort_k;
static int cmp_pt(const void *A, const void *B)
{
    const opt_t *a = (const opt_t *)A, *b = (const opt_t *)B;
    int k = g_sort_k;
    int sa = level_sum(k, a->lv), sb = level_sum(k, b->lv);
    if (sa != sb) return sa < sb ? -1 : 1;
    for (int j = 0; j < k; ++j)
        if (a->lv[j] != b->lv[j]) return a->lv[j] < b->lv[j] ? -1 : 1;
    for (int j = 0; j < k; ++j)
        if (a->ix[j] != b->ix[j]) return a->ix[j] < b->ix[j] ? -1 : 1;
    return 0;
}

static int64_t find_pt(int k, int64_t p0, int64_t p1, const uint8_t *levels,
                       const uint32_t *indices, const uint8_t *lv, const uint32_t *ix)
{
    for (int64_t p = p0; p < p1; ++p) {
        int eq = 1;
        for (int j = 0; j < k && eq; ++j)
            if (levels[p * KMAX + j] != lv[j] || indices[p * KMAX + j] != ix[j]) eq = 0;
        if (eq) return p;
    }
    return -1;
}

static double linf(int m, const double *a)
{
    double g = 0.0;
    for (int j = 0; j < m; ++j) if (fabs(a[j]) > g) g = fabs(a[j]);
    return g;
}

/*
 * One refinement sweep of one component (eq. 3.8): a point is significant if
 * ||alpha_p||_inf > eps. Every child, in every dimension, of a significant
 * point is a candidate if sum(l-1) <= L-1 and it is not already present.
 *   strict == 0: a candidate is added (any significant parent suffices).
 *   strict == 1: a candidate is dropped if some present parent of it (in any
 *                dimension) is not significant: the stricter reading of
 *                Sec. 3.1, where finer points inside the support of a
 *                rejected point are left out.
 * New points are sorted (level sum, level tuple, index tuple) and written to
 * new_lv/new_ix (cap*KMAX). Returns the number of new points, or -1 if cap is
 * too small.
 */
int64_t orc_refine(int m, int k, int64_t p0, int64_t p1, const uint8_t *levels,
                   const uint32_t *indices, const double *alpha, double eps, int L,
                   int strict, int64_t cap, uint8_t *new_lv, uint32_t *new_ix)
{
    int64_t nc = 0, ccap = 1024;
    opt_t *cand = (opt_t *)malloc(sizeof(opt_t) * (size_t)ccap);
    for (int64_t p = p0; p < p1; ++p) {
        if (!(linf(m, &alpha[p * m]) > eps)) continue;
        for (int j = 0; j < k; ++j) {
            uint32_t ci[2];
            int nch = children1d(levels[p * KMAX + j], indices[p * KMAX + j], ci);
            for (int c = 0; c < nch; ++c) {
                opt_t o;
                memset(&o, 0, sizeof o);
                for (int q = 0; q < k; ++q) {
                    o.lv[q] = levels[p * KMAX + q];
                    o.ix[q] = indices[p * KMAX + q];
                }
                o.lv[j] = (uint8_t)(o.lv[j] + 1);
                o.ix[j] = ci[c];
                if (level_sum(k, o.lv) > L - 1) continue;
                if (find_pt(k, p0, p1, levels, indices, o.lv, o.ix) >= 0) continue;
                if (strict) {
                    int ok = 1;
                    for (int q = 0; q < k && ok; ++q) {
                        if (o.lv[q] < 2) continue;
                        opt_t par = o;
                        int pl;
                        uint32_t pi;
                        parent1d(o.lv[q], o.ix[q], &pl, &pi);
                        par.lv[q] = (uint8_t)pl;
                        par.ix[q] = pi;
                        int64_t pp = find_pt(k, p0, p1, levels, indices, par.lv, par.ix);
                        if (pp >= 0 && !(linf(m, &alpha[pp * m]) > eps)) ok = 0;
                    }
                    if (!ok) continue;
                }
                if (nc == ccap) {
                    ccap *= 2;
                    cand = (opt_t *)realloc(cand, sizeof(opt_t) * (size_t)ccap);
                }
                cand[nc++] = o;
            }
        }
    }
    g_sort_k = k;
    qsort(cand, (size_t)nc, sizeof(opt_t), cmp_pt);
    int64_t nu = 0;
    for (int64_t c = 0; c < nc; ++c) {
        if (nu > 0 && cmp_pt(&cand[c], &cand[nu - 1]) == 0) continue;
        cand[nu++] = cand[c];
    }
    if (nu > cap) { free(cand); return -1; }
    for (int64_t c = 0; c < nu; ++c) {
        for (int j = 0; j < KMAX; ++j) {
            new_lv[c * KMAX + j] = j < k ? cand[c].lv[j] : 0;
            new_ix[c * KMAX + j] = j < k ? cand[c].ix[j] : 0;
        }
    }
    free(cand);
    return nu;
}

/* ------------------------------------------------------------------ */
/* Quadrature (eq. 3.7) of each component interpolant                  */
/* ------------------------------------------------------------------ */

void orc_quadrature(int m, int C, const int32_t *comp_k, const int64_t *comp_off,
                    const uint8_t *levels, const uint32_t *indices, const double *alpha,
                    double *Q /* C*m */)
{
    for (int c = 0; c < C; ++c) {
        for (int j = 0; j < m; ++j) Q[c * m + j] = 0.0;
        for (int64_t p = comp_off[c]; p < comp_off[c + 1]; ++p) {
            double w = 1.0;
            for (int j = 0; j < comp_k[c]; ++j)
                w *= orc_int1d(levels[p * KMAX + j], indices[p * KMAX + j]);
            for (int j = 0; j < m; ++j) Q[c * m + j] += w * alpha[p * m + j];
        }
    }
}

/* ------------------------------------------------------------------ */
/* Pruned active sets: tree descent (Sec. 3.1, eq. 3.3)                */
/* ------------------------------------------------------------------ */

/*
 * The support of a child (one dimension refined one level) lies inside its
 * parent's support, so every active point's parents are active, and every
 * point of a grid built by refinement is reached from the root (1, ..., 1) by
 * a chain of existing parent -> child links. The active set of a query is
 * therefore found by a breadth-first descent that starts at the root and visits
 * a child only from an active parent and only if the child's own hat is
 * nonzero in the refined dimension (its other dimensions equal the parent's).
 * Points are looked up in a per-call copy of each component's points sorted
 * by (levels, indices). Only the index work is computed: the XOR of the point
 * keys and the count of the active points the form sums (form 1: all levels
 * >= 2), exactly as orc_eval's hash and count outputs. Queries run in parallel
 * over `threads` POSIX threads (0: one), each with its own visit stamps.
 * Returns 0, or -1 if a component has no root point (then nothing is written).
 */
typedef struct {
    int32_t comp, k;
    uint8_t lv[KMAX];
    uint32_t ix[KMAX];
    int64_t orig;          /* index of the point in the caller's tables */
} ppt_t;

static int cmp_ppt(const void *A, const void *B)
{
    const ppt_t *a = (const ppt_t *)A, *b = (const ppt_t *)B;
    if (a->comp != b->comp) return a->comp < b->comp ? -1 : 1;
    for (int j = 0; j < a->k; ++j)
        if (a->lv[j] != b->lv[j]) return a->lv[j] < b->lv[j] ? -1 : 1;
    for (int j = 0; j < a->k; ++j)
        if (a->ix[j] != b->ix[j]) return a->ix[j] < b->ix[j] ? -1 : 1;
    return 0;
}

typedef struct {
    int d, C, form;
    const int32_t *comp_k, *comp_dims;
    const int64_t *comp_off;
    const ppt_t *pts;          /* all points, sorted by (component, levels, indices) */
    const int64_t *root;       /* per component: position of its root in pts */
    const double *b, *lo, *hi, *x;
    uint64_t *hash;
    int32_t *count;
    int64_t q0, q1;
    int64_t P;
} prune_job_t;

static int64_t find_sorted(const ppt_t *pts, int64_t p0, int64_t p1, const ppt_t *key)
{
    int64_t lo = p0, hi = p1;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        int c = cmp_ppt(&pts[mid], key);
        if (c == 0) return mid;
        if (c < 0) lo = mid + 1; else hi = mid;
    }
    return -1;
}

static void *prune_worker(void *arg)
{
    prune_job_t *J = (prune_job_t *)arg;
    const int d = J->d;
    int64_t *stamp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(J->P > 0 ? J->P : 1));
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)(J->P > 0 ? J->P : 1));
    double *xc = (double *)malloc(sizeof(double) * (size_t)d);
    for (int64_t i = 0; i < J->P; ++i) stamp[i] = -1;
    for (int64_t q = J->q0; q < J->q1; ++q) {
        int finite = 1;
        for (int i = 0; i < d; ++i) {
            double v = J->x[q * d + i];
            if (!isfinite(v) || !isfinite((v - J->lo[i]) / (J->hi[i] - J->lo[i]))) finite = 0;
            xc[i] = canon(v, J->lo[i], J->hi[i]);
        }
        uint64_t h = 0;
        int32_t cnt = 0;
        if (finite) {
            for (int c = 0; c < J->C; ++c) {
                if (J->form == 0 && J->b[c] == 0.0) continue;
                const int k = J->comp_k[c];
                const int32_t *dims = &J->comp_dims[c * KMAX];
                const int64_t p0 = J->comp_off[c], p1 = J->comp_off[c + 1];
                int64_t head = 0, tail = 0;
                queue[tail++] = J->root[c];
                stamp[J->root[c]] = q;
                while (head < tail) {
                    const ppt_t *p = &J->pts[queue[head++]];
                    int interior = 1;
                    for (int j = 0; j < k; ++j) if (p->lv[j] < 2) interior = 0;
                    if (J->form == 0 || interior) {
                        h ^= orc_point_key(c, k, p->lv, p->ix);
                        ++cnt;
                    }
                    for (int j = 0; j < k; ++j) {
                        uint32_t ci[2];
                        const int nc = children1d(p->lv[j], p->ix[j], ci);
                        for (int t = 0; t < nc; ++t) {
                            if (!orc_active1d(p->lv[j] + 1, ci[t], xc[dims[j]])) continue;
                            ppt_t key = *p;
                            key.lv[j] = (uint8_t)(p->lv[j] + 1);
                            key.ix[j] = ci[t];
                            const int64_t f = find_sorted(J->pts, p0, p1, &key);
                            if (f >= 0 && stamp[f] != q) {
                                stamp[f] = q;
                                queue[tail++] = f;
                            }
                        }
                    }
                }
            }
        }
        if (J->hash) J->hash[q] = h;
        if (J->count) J->count[q] = cnt;
    }
    free(stamp);
    free(queue);
    free(xc);
    return NULL;
}

int orc_active_pruned(int d, int C, const int32_t *comp_k, const int32_t *comp_dims,
                      const int64_t *comp_off, const uint8_t *levels, const uint32_t *indices,
                      const double *b, const double *lo, const double *hi, int form, int64_t n,
                      const double *x, uint64_t *hash, int32_t *count, int threads)
{
    const int64_t P = comp_off[C];
    ppt_t *pts = (ppt_t *)malloc(sizeof(ppt_t) * (size_t)(P > 0 ? P : 1));
    int64_t *root = (int64_t *)malloc(sizeof(int64_t) * (size_t)(C > 0 ? C : 1));
    int rc = 0;
    for (int c = 0; c < C; ++c)
        for (int64_t p = comp_off[c]; p < comp_off[c + 1]; ++p) {
            ppt_t *t = &pts[p];
            memset(t, 0, sizeof *t);
            t->comp = c;
            t->k = comp_k[c];
            for (int j = 0; j < comp_k[c]; ++j) {
                t->lv[j] = levels[p * KMAX + j];
                t->ix[j] = indices[p * KMAX + j];
            }
            t->orig = p;
        }
    qsort(pts, (size_t)P, sizeof(ppt_t), cmp_ppt);
    for (int c = 0; c < C && rc == 0; ++c) {
        ppt_t key;
        memset(&key, 0, sizeof key);
        key.comp = c;
        key.k = comp_k[c];
        for (int j = 0; j < comp_k[c]; ++j) { key.lv[j] = 1; key.ix[j] = 1; }
        root[c] = find_sorted(pts, comp_off[c], comp_off[c + 1], &key);
        if (root[c] < 0) rc = -1;
    }
    if (rc == 0) {
        if (threads < 1) threads = 1;
        if (threads > 256) threads = 256;
        prune_job_t jobs[256];
        pthread_t tid[256];
        for (int t = 0; t < threads; ++t) {
            prune_job_t *J = &jobs[t];
            J->d = d; J->C = C; J->form = form;
            J->comp_k = comp_k; J->comp_dims = comp_dims; J->comp_off = comp_off;
            J->pts = pts; J->root = root; J->b = b; J->lo = lo; J->hi = hi; J->x = x;
            J->hash = hash; J->count = count; J->P = P;
            J->q0 = n * t / threads;
            J->q1 = n * (t + 1) / threads;
        }
        for (int t = 1; t < threads; ++t) pthread_create(&tid[t], NULL, prune_worker, &jobs[t]);
        prune_worker(&jobs[0]);
        for (int t = 1; t < threads; ++t) pthread_join(tid[t], NULL);
    }
    free(pts);
    free(root);
    return rc;
}
