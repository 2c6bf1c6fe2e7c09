/*
 * FP64 CPU oracle for the k-dimensional sliding window DFT, the extension of Richardson &
 * Eddy's 2D Tree SWDFT (arXiv 1707.08213) to k dimensions in Section 4.4.
 *
 * TEST INFRASTRUCTURE ONLY.  The only callers are the tests and bench.py's cpu_baseline leg.
 * The GPU library never includes, links or loads this file, and this file uses no code,
 * header or table of the GPU library.
 *
 * What it computes: for an N_0 x ... x N_{K-1} array x and windows n_0 x ... x n_{K-1}
 * (K <= SWK_MAXK), every window that lies inside the array gets its K-dimensional DFT,
 * Eq. (2) with one more sum per dimension:
 *
 *   a[q; k] = c * sum_{j_0 < n_0} ... sum_{j_{K-1} < n_{K-1}} x[q_0 + j_0, ..., q_{K-1} + j_{K-1}]
 *                 * prod_d w_{n_d}^{-j_d k_d},                 w_n = exp(2*pi*i/n),
 *
 * q_d < P_d = N_d - n_d + 1 (the window ending at p_d = q_d + n_d - 1).  Output layout is
 * row-major [q_0]...[q_{K-1}][k_0]...[k_{K-1}] complex128 (interleaved re, im); the input is
 * row-major complex128.  c = 1/sqrt(prod n_d) is the unitary scale; 1 gives the bare sums.
 *
 * Two evaluation orders of the same sum:
 *   direct     - for every k, the K-fold sum over j exactly as written above;
 *   separable  - the window's DFT taken one axis at a time (the row-column factorisation of
 *                Section 4.2 in K axes): the same sum with its loops nested differently.
 *
 * swt_treekd_f64 is the tree itself, Eq. (kdfswft), in the loop order of Section 4.4's
 * description (dimension, then levels of that dimension, then trees, then nodes), kept
 * apart from the definition so that the tests can check one against the other.
 *
 * Exponentials are tabulated per length as cos/sin(2*pi*j/n), j < n, and indexed by
 * (j*k) mod n, so no phase is evaluated beyond 2*pi.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define SWK_MAXK 4
#define SWK_OK 0
#define SWK_EINVAL (-1)
#define SWK_ENOMEM (-5)

#ifdef _OPENMP
#define SWK_PRAGMA(x) _Pragma(#x)
#else
#define SWK_PRAGMA(x)
#endif

static const double SWK_TWO_PI = 6.283185307179586476925286766559;

/* w[j] = w_n^{-j} = exp(-2*pi*i*j/n), j < n, interleaved. */
static double *kd_omega(int n) {
    double *w = (double *)malloc(sizeof(double) * 2 * (size_t)n);
    if (!w) return NULL;
    for (int j = 0; j < n; ++j) {
        const double ang = SWK_TWO_PI * (double)j / (double)n;
        w[2 * j] = cos(ang);
        w[2 * j + 1] = -sin(ang);
    }
    return w;
}

typedef struct {
    int K;
    int64_t N[SWK_MAXK], P[SWK_MAXK];
    int n[SWK_MAXK];
    int64_t xstride[SWK_MAXK];  /* input element stride of dimension d */
    int64_t kstride[SWK_MAXK];  /* coefficient stride of dimension d inside one window */
    int64_t nn;                 /* coefficients per window */
    int64_t windows;            /* prod P_d */
    double *w[SWK_MAXK];
} kd_geom;

static void kd_free(kd_geom *g) {
    for (int d = 0; d < SWK_MAXK; ++d) free(g->w[d]);
}

static int kd_setup(kd_geom *g, int K, const int64_t *N, const int *n) {
    memset(g, 0, sizeof(*g));
    if (K < 1 || K > SWK_MAXK || !N || !n) return SWK_EINVAL;
    g->K = K;
    g->nn = 1;
    g->windows = 1;
    for (int d = 0; d < K; ++d) {
        if (N[d] < 1 || n[d] < 1 || n[d] > N[d]) return SWK_EINVAL;
        g->N[d] = N[d];
        g->n[d] = n[d];
        g->P[d] = N[d] - n[d] + 1;
        g->nn *= n[d];
        g->windows *= g->P[d];
    }
    g->xstride[K - 1] = 1;
    g->kstride[K - 1] = 1;
    for (int d = K - 2; d >= 0; --d) {
        g->xstride[d] = g->xstride[d + 1] * N[d + 1];
        g->kstride[d] = g->kstride[d + 1] * n[d + 1];
    }
    for (int d = 0; d < K; ++d) {
        g->w[d] = kd_omega(n[d]);
        if (!g->w[d]) {
            kd_free(g);
            return SWK_ENOMEM;
        }
    }
    return SWK_OK;
}

/* Unflatten a row-major index over extents ext[0..K-1]. */
static void kd_unflatten(int64_t flat, int K, const int64_t *ext, int64_t *idx) {
    for (int d = K - 1; d >= 0; --d) {
        idx[d] = flat % ext[d];
        flat /= ext[d];
    }
}

/* One window by the K-fold sum.  q: first sample of the window per dimension. */
static void kd_window_direct(const kd_geom *g, const double *x, const int64_t *q, double c, double *out) {
    const int K = g->K;
    int64_t ext[SWK_MAXK], kk[SWK_MAXK], jj[SWK_MAXK];
    for (int d = 0; d < K; ++d) ext[d] = g->n[d];
    int64_t base = 0;
    for (int d = 0; d < K; ++d) base += q[d] * g->xstride[d];
    for (int64_t kf = 0; kf < g->nn; ++kf) {
        kd_unflatten(kf, K, ext, kk);
        double sr = 0.0, si = 0.0;
        for (int64_t jf = 0; jf < g->nn; ++jf) {
            kd_unflatten(jf, K, ext, jj);
            /* kernel = prod_d w_{n_d}^{-j_d k_d} */
            double er = 1.0, ei = 0.0;
            int64_t off = base;
            for (int d = 0; d < K; ++d) {
                const double *e = g->w[d] + 2 * ((jj[d] * kk[d]) % g->n[d]);
                const double tr = er * e[0] - ei * e[1];
                const double ti = er * e[1] + ei * e[0];
                er = tr;
                ei = ti;
                off += jj[d] * g->xstride[d];
            }
            const double *v = x + 2 * off;
            sr += v[0] * er - v[1] * ei;
            si += v[0] * ei + v[1] * er;
        }
        out[2 * kf] = c * sr;
        out[2 * kf + 1] = c * si;
    }
}

/* One window axis by axis: copy the patch, then replace each line along dimension d by its
 * n_d-point DFT, for d = K-1 down to 0.  buf: 2*nn doubles, line: 2*max n doubles. */
static void kd_window_separable(const kd_geom *g, const double *x, const int64_t *q, double c,
                                double *out, double *line) {
    const int K = g->K;
    int64_t ext[SWK_MAXK], jj[SWK_MAXK];
    for (int d = 0; d < K; ++d) ext[d] = g->n[d];
    int64_t base = 0;
    for (int d = 0; d < K; ++d) base += q[d] * g->xstride[d];
    for (int64_t jf = 0; jf < g->nn; ++jf) {
        kd_unflatten(jf, K, ext, jj);
        int64_t off = base;
        for (int d = 0; d < K; ++d) off += jj[d] * g->xstride[d];
        out[2 * jf] = x[2 * off];
        out[2 * jf + 1] = x[2 * off + 1];
    }
    for (int d = K - 1; d >= 0; --d) {
        const int nd = g->n[d];
        const int64_t st = g->kstride[d];
        for (int64_t start = 0; start < g->nn; ++start) {
            if ((start / st) % nd != 0) continue; /* one line per index with j_d = 0 */
            for (int k = 0; k < nd; ++k) {
                double sr = 0.0, si = 0.0;
                for (int j = 0; j < nd; ++j) {
                    const double *e = g->w[d] + 2 * (((int64_t)j * k) % nd);
                    const double *v = out + 2 * (start + j * st);
                    sr += v[0] * e[0] - v[1] * e[1];
                    si += v[0] * e[1] + v[1] * e[0];
                }
                line[2 * k] = sr;
                line[2 * k + 1] = si;
            }
            for (int k = 0; k < nd; ++k) {
                out[2 * (start + k * st)] = line[2 * k];
                out[2 * (start + k * st) + 1] = line[2 * k + 1];
            }
        }
    }
    for (int64_t i = 0; i < 2 * g->nn; ++i) out[i] *= c;
}

static int kd_max_n(const kd_geom *g) {
    int m = 1;
    for (int d = 0; d < g->K; ++d)
        if (g->n[d] > m) m = g->n[d];
    return m;
}

/* Windows listed in q (count x K, row-major), or every window when q == NULL. */
static int kd_run(const double *x, int K, const int64_t *N, const int *n, double c, int method,
                  int64_t count, const int64_t *q, int nthreads, double *out) {
    kd_geom g;
    int rc = kd_setup(&g, K, N, n);
    if (rc != SWK_OK) return rc;
    if (method != 0 && method != 1) {
        kd_free(&g);
        return SWK_EINVAL;
    }
    if (q) {
        for (int64_t i = 0; i < count; ++i)
            for (int d = 0; d < K; ++d)
                if (q[i * K + d] < 0 || q[i * K + d] >= g.P[d]) {
                    kd_free(&g);
                    return SWK_EINVAL;
                }
    } else {
        count = g.windows;
    }
    const int mx = kd_max_n(&g);
    int failed = 0;
    (void)nthreads;
    SWK_PRAGMA(omp parallel num_threads(nthreads > 0 ? nthreads : 1) reduction(| : failed))
    {
        double *line = (double *)malloc(sizeof(double) * 2 * (size_t)mx);
        if (!line) failed = 1;
        SWK_PRAGMA(omp for schedule(static))
        for (int64_t i = 0; i < count; ++i) {
            if (!line) continue;
            int64_t qq[SWK_MAXK];
            if (q)
                for (int d = 0; d < K; ++d) qq[d] = q[i * K + d];
            else
                kd_unflatten(i, K, g.P, qq);
            double *o = out + 2 * i * g.nn;
            if (method == 0)
                kd_window_direct(&g, x, qq, c, o);
            else
                kd_window_separable(&g, x, qq, c, o, line);
        }
        free(line);
    }
    kd_free(&g);
    return failed ? SWK_ENOMEM : SWK_OK;
}

/* Every window: out holds prod P_d * prod n_d complex. method 0 = direct, 1 = separable. */
int swo_swdftkd(const double *x, int K, const int64_t *N, const int *n, double c, int method,
                int nthreads, double *out) {
    if (!x || !out) return SWK_EINVAL;
    return kd_run(x, K, N, n, c, method, 0, NULL, nthreads, out);
}

/* Windows q[i*K .. i*K+K-1], i < count: out holds count * prod n_d complex. */
int swo_swdftkd_windows(const double *x, int K, const int64_t *N, const int *n, double c,
                        int method, int64_t count, const int64_t *q, int nthreads, double *out) {
    if (!x || !out || !q || count < 0) return SWK_EINVAL;
    return kd_run(x, K, N, n, c, method, count, q, nthreads, out);
}

static int kd_ilog2(int n) {
    int m = 0;
    while ((1 << m) < n) ++m;
    return ((1 << m) == n) ? m : -1;
}

/*
 * The tree of Eq. (kdfswft).  Every array position p carries a tree whose level-l node
 * (i_0, ..., i_{K-1}) is T[p, l, i]; level 0 is the data at node 0.  Dimension c owns levels
 * below_c + 1 .. below_c + m_c, where below_c = sum_{e > c} m_e (the last dimension's levels
 * come first).  At level l = below_c + t of dimension c, with s = 2^(m_c - t) (the paper's
 * s_l^c = 2^(sum_{e >= c} m_e - l)) and h = 2^(t-1):
 *
 *   T[p, l, (0.., i_c, i_{c+1}, ..)] = T[p - s e_c, l-1, (0.., i_c mod h, i_{c+1}, ..)]
 *                                     + Om_c[i_c * s] * T[p, l-1, (0.., i_c mod h, i_{c+1}, ..)]
 *
 * for i_c < 2^t, i_e < n_e (e > c), i_e = 0 (e < c); Om_c[j] = w_{n_c}^{-j}.  The final level
 * at p_d >= n_d - 1 holds the window's K-dimensional DFT in natural k order.  Nodes are
 * stored at sum_d i_d * prod_{e > d} n_e, two level buffers of prod N_d * prod n_d complex.
 * A node whose shifted tree lies outside the array belongs to an incomplete border tree and
 * takes 0 for the missing term; such nodes never reach a complete window.
 * opcount: node evaluations (one complex multiply and one add each), over all positions.
 */
int swt_treekd_f64(const double *x, int K, const int64_t *N, const int *n, double c, double *out,
                   int64_t *opcount) {
    kd_geom g;
    int rc = kd_setup(&g, K, N, n);
    if (rc != SWK_OK) return rc;
    int m[SWK_MAXK];
    for (int d = 0; d < K; ++d) {
        m[d] = kd_ilog2(n[d]);
        if (m[d] < 0) {
            kd_free(&g);
            return SWK_EINVAL;
        }
    }
    int64_t cells = g.nn;
    for (int d = 0; d < K; ++d) cells *= N[d];
    double *prev = (double *)calloc(2 * (size_t)cells, sizeof(double));
    double *cur = (double *)calloc(2 * (size_t)cells, sizeof(double));
    if (!prev || !cur) {
        free(prev);
        free(cur);
        kd_free(&g);
        return SWK_ENOMEM;
    }
    int64_t positions = cells / g.nn;
    for (int64_t pf = 0; pf < positions; ++pf) {
        prev[2 * pf * g.nn] = x[2 * pf];
        prev[2 * pf * g.nn + 1] = x[2 * pf + 1];
    }
    int64_t ops = 0;
    for (int cdim = K - 1; cdim >= 0; --cdim) {
        int64_t inner = 1; /* nodes of the dimensions after cdim: prod_{e > c} n_e */
        for (int e = cdim + 1; e < K; ++e) inner *= n[e];
        const int64_t st = g.kstride[cdim];
        for (int t = 1; t <= m[cdim]; ++t) {
            const int64_t s = (int64_t)1 << (m[cdim] - t);
            const int64_t h = (int64_t)1 << (t - 1);
            for (int64_t pf = 0; pf < positions; ++pf) {
                int64_t p[SWK_MAXK];
                kd_unflatten(pf, K, g.N, p);
                const double *D = prev + 2 * pf * g.nn;
                const double *B = (p[cdim] - s >= 0) ? prev + 2 * (pf - s * g.xstride[cdim]) * g.nn : NULL;
                double *A = cur + 2 * pf * g.nn;
                for (int64_t ic = 0; ic < 2 * h; ++ic) {
                    const double *w = g.w[cdim] + 2 * (ic * s);
                    const int64_t src = (ic % h) * st, dst = ic * st;
                    for (int64_t r = 0; r < inner; ++r) {
                        const double dr = D[2 * (src + r)], di = D[2 * (src + r) + 1];
                        const double br = B ? B[2 * (src + r)] : 0.0, bi = B ? B[2 * (src + r) + 1] : 0.0;
                        A[2 * (dst + r)] = br + (w[0] * dr - w[1] * di);
                        A[2 * (dst + r) + 1] = bi + (w[0] * di + w[1] * dr);
                    }
                }
                ops += 2 * h * inner;
            }
            double *tmp = prev;
            prev = cur;
            cur = tmp;
        }
    }
    for (int64_t wf = 0; wf < g.windows; ++wf) {
        int64_t q[SWK_MAXK];
        kd_unflatten(wf, K, g.P, q);
        int64_t pf = 0;
        for (int d = 0; d < K; ++d) pf += (q[d] + n[d] - 1) * g.xstride[d];
        const double *T = prev + 2 * pf * g.nn;
        for (int64_t k = 0; k < g.nn; ++k) {
            out[2 * (wf * g.nn + k)] = c * T[2 * k];
            out[2 * (wf * g.nn + k) + 1] = c * T[2 * k + 1];
        }
    }
    if (opcount) *opcount = ops;
    free(prev);
    free(cur);
    kd_free(&g);
    return SWK_OK;
}
