/*
 * The 2D Tree SWDFT exactly as the paper lays it out (arXiv 1707.08213, Section 4.2 Eqs.
 * rowfswft2d / colfswft2d, Section 4.3 loop order), on the CPU, in FP64 and FP32.
 *
 * TEST INFRASTRUCTURE ONLY (tests/, __graft_entry__.smoke(), bench.py's cpu_baseline leg).
 * It shares nothing with the GPU library.  It is checked against the direct definition in
 * swdft2d_oracle.c (the paper states the tree reproduces the per-window FFT, Section 4.6),
 * and it is the "plain CPU tree" whose speed the bench reports beside the oracle.
 *
 * Tree T[p0,p1,l,i0,i1] (Section 4.2): level 0 is the data, T[p0,p1,0,0,0] = x[p0,p1].
 *   row levels t = 1..m1, shift s = 2^(m1-t), nodes (0, i1), i1 < 2^t:
 *     T[p,t,0,i1] = T[p0,p1-s,t-1,0,i1 mod 2^(t-1)] + Om1[i1*s] * T[p,t-1,0,i1 mod 2^(t-1)]
 *   column levels v = m1+1..m1+m0, shift s = 2^(m0+m1-v), nodes (i0,i1), i0 < 2^(v-m1), i1 < n1:
 *     T[p,v,i0,i1] = T[p0-s,p1,v-1,i0 mod 2^(v-m1-1),i1] + Om0[i0*s] * T[p,v-1,i0 mod ...,i1]
 *   with Om_d[j] = w_{n_d}^{-j}.  Level m0+m1 at p_i >= n_i-1 holds the window's 2D DFT in
 *   natural (k0,k1) order.
 * Readings taken where the text is loose: the first m1 levels are the dimension-1 ("row")
 * transforms, as the equations say; the column shift exponent uses v; the column-level node
 * ranges are i0 < 2^(v-m1), i1 < n1; memory is 2*N0*N1*n0*n1 complex.
 *
 * Loop order (Section 4.3): levels outermost, then trees p0, p1, then nodes, with two level
 * buffers (previous and current).  A node whose shifted tree lies outside the array belongs
 * to an incomplete border tree (Section 4.7); its missing term is taken as 0 -- such nodes
 * never reach a complete window.
 *
 * opcount (optional): the number of node evaluations, each one complex multiply and one
 * complex add, the paper's unit of work (Eq. windowops).
 * dump_level/dump (optional): a copy of one level's buffer, for the level invariant test.
 * nthreads: OpenMP threads over p0 inside each level when built with -fopenmp (the paper
 * notes the levels-outer order suits parallel work, Section 4.3); results do not depend on it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifdef _OPENMP
#define SWT_PRAGMA(x) _Pragma(#x)
#else
#define SWT_PRAGMA(x)
#endif

static const double SWT_TWO_PI = 6.283185307179586476925286766559;

static int ilog2_exact(int n) {
    int m = 0;
    while ((1 << m) < n) ++m;
    return ((1 << m) == n) ? m : -1;
}

#define SWT_DEFINE_TREE(NAME, REAL)                                                              \
int NAME(const REAL *x, int64_t N0, int64_t N1, int n0, int n1, REAL c, REAL *out,              \
         int64_t *opcount, int dump_level, REAL *dump, int nthreads) {                                          \
    const int m0 = ilog2_exact(n0), m1 = ilog2_exact(n1);                                        \
    (void)nthreads;                                                                              \
    if (m0 < 0 || m1 < 0 || N0 < n0 || N1 < n1 || n0 < 1 || n1 < 1) return -1;                   \
    const int64_t nn = (int64_t)n0 * n1, P0 = N0 - n0 + 1, P1 = N1 - n1 + 1;                     \
    const size_t cells = (size_t)(N0 * N1 * nn);                                                  \
    REAL *prev = (REAL *)calloc(2 * cells, sizeof(REAL));                                        \
    REAL *cur = (REAL *)calloc(2 * cells, sizeof(REAL));                                         \
    REAL *om0 = (REAL *)malloc(sizeof(REAL) * 2 * (size_t)n0);                                   \
    REAL *om1 = (REAL *)malloc(sizeof(REAL) * 2 * (size_t)n1);                                   \
    if (!prev || !cur || !om0 || !om1) {                                                         \
        free(prev); free(cur); free(om0); free(om1); return -5;                                  \
    }                                                                                            \
    for (int j = 0; j < n0; ++j) {                                                               \
        om0[2 * j] = (REAL)cos(SWT_TWO_PI * j / n0);                                             \
        om0[2 * j + 1] = (REAL)(-sin(SWT_TWO_PI * j / n0));                                      \
    }                                                                                            \
    for (int j = 0; j < n1; ++j) {                                                               \
        om1[2 * j] = (REAL)cos(SWT_TWO_PI * j / n1);                                             \
        om1[2 * j + 1] = (REAL)(-sin(SWT_TWO_PI * j / n1));                                      \
    }                                                                                            \
    /* level 0: the data, node (0,0) of every tree */                                            \
    for (int64_t p0 = 0; p0 < N0; ++p0)                                                          \
        for (int64_t p1 = 0; p1 < N1; ++p1) {                                                    \
            prev[2 * ((p0 * N1 + p1) * nn)] = x[2 * (p0 * N1 + p1)];                             \
            prev[2 * ((p0 * N1 + p1) * nn) + 1] = x[2 * (p0 * N1 + p1) + 1];                     \
        }                                                                                        \
    if (dump && dump_level == 0) memcpy(dump, prev, 2 * cells * sizeof(REAL));                   \
    int64_t ops = 0;                                                                             \
    /* row levels t = 1..m1 (Eq. rowfswft2d) */                                                  \
    for (int t = 1; t <= m1; ++t) {                                                              \
        const int64_t s = (int64_t)1 << (m1 - t);                                                \
        const int half = 1 << (t - 1);                                                           \
        SWT_PRAGMA(omp parallel for num_threads(nthreads > 0 ? nthreads : 1) reduction(+ : ops)) \
        for (int64_t p0 = 0; p0 < N0; ++p0) {                                                    \
            for (int64_t p1 = 0; p1 < N1; ++p1) {                                                \
                const REAL *D = prev + 2 * ((p0 * N1 + p1) * nn);                                \
                const REAL *B = (p1 - s >= 0) ? prev + 2 * ((p0 * N1 + (p1 - s)) * nn) : NULL;   \
                REAL *A = cur + 2 * ((p0 * N1 + p1) * nn);                                       \
                for (int i1 = 0; i1 < 2 * half; ++i1) {                                          \
                    const int j = i1 % half;                                                     \
                    const REAL *w = om1 + 2 * ((int64_t)i1 * s);                                 \
                    REAL br = B ? B[2 * j] : (REAL)0, bi = B ? B[2 * j + 1] : (REAL)0;           \
                    A[2 * i1] = br + (w[0] * D[2 * j] - w[1] * D[2 * j + 1]);                    \
                    A[2 * i1 + 1] = bi + (w[0] * D[2 * j + 1] + w[1] * D[2 * j]);                \
                }                                                                                \
                ops += 2 * half;                                                                 \
            }                                                                                    \
        }                                                                                        \
        { REAL *tmp = prev; prev = cur; cur = tmp; }                                             \
        if (dump && dump_level == t) memcpy(dump, prev, 2 * cells * sizeof(REAL));               \
    }                                                                                            \
    /* column levels v = m1+1..m1+m0 (Eq. colfswft2d) */                                         \
    for (int v = m1 + 1; v <= m1 + m0; ++v) {                                                    \
        const int64_t s = (int64_t)1 << (m0 + m1 - v);                                           \
        const int half = 1 << (v - m1 - 1);                                                      \
        SWT_PRAGMA(omp parallel for num_threads(nthreads > 0 ? nthreads : 1) reduction(+ : ops)) \
        for (int64_t p0 = 0; p0 < N0; ++p0) {                                                    \
            for (int64_t p1 = 0; p1 < N1; ++p1) {                                                \
                const REAL *D = prev + 2 * ((p0 * N1 + p1) * nn);                                \
                const REAL *B = (p0 - s >= 0) ? prev + 2 * (((p0 - s) * N1 + p1) * nn) : NULL;   \
                REAL *A = cur + 2 * ((p0 * N1 + p1) * nn);                                       \
                for (int i0 = 0; i0 < 2 * half; ++i0) {                                          \
                    const int j0 = i0 % half;                                                    \
                    const REAL *w = om0 + 2 * ((int64_t)i0 * s);                                 \
                    for (int i1 = 0; i1 < n1; ++i1) {                                            \
                        const int64_t jd = (int64_t)j0 * n1 + i1;                                \
                        REAL br = B ? B[2 * jd] : (REAL)0, bi = B ? B[2 * jd + 1] : (REAL)0;     \
                        A[2 * (i0 * n1 + i1)] = br + (w[0] * D[2 * jd] - w[1] * D[2 * jd + 1]);  \
                        A[2 * (i0 * n1 + i1) + 1] =                                              \
                            bi + (w[0] * D[2 * jd + 1] + w[1] * D[2 * jd]);                      \
                    }                                                                            \
                }                                                                                \
                ops += (int64_t)2 * half * n1;                                                   \
            }                                                                                    \
        }                                                                                        \
        { REAL *tmp = prev; prev = cur; cur = tmp; }                                             \
        if (dump && dump_level == v) memcpy(dump, prev, 2 * cells * sizeof(REAL));               \
    }                                                                                            \
    /* select level m0+m1 of every complete tree, p_i = q_i + n_i - 1 (Section 4.2) */           \
    for (int64_t q0 = 0; q0 < P0; ++q0)                                                          \
        for (int64_t q1 = 0; q1 < P1; ++q1) {                                                    \
            const REAL *T = prev + 2 * (((q0 + n0 - 1) * N1 + (q1 + n1 - 1)) * nn);              \
            REAL *o = out + 2 * ((q0 * P1 + q1) * nn);                                           \
            for (int64_t k = 0; k < nn; ++k) {                                                   \
                o[2 * k] = c * T[2 * k];                                                         \
                o[2 * k + 1] = c * T[2 * k + 1];                                                 \
            }                                                                                    \
        }                                                                                        \
    if (opcount) *opcount = ops;                                                                 \
    free(prev); free(cur); free(om0); free(om1);                                                 \
    return 0;                                                                                    \
}

SWT_DEFINE_TREE(swt_tree2d_f64, double)
SWT_DEFINE_TREE(swt_tree2d_f32, float)
