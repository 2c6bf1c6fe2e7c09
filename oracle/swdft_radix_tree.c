/*
 * The 2D sliding tree with radix-2 or radix-3 levels per axis, on the CPU in FP64.
 *
 * TEST INFRASTRUCTURE ONLY (tests/ and bench.py's cpu_baseline leg).  It shares nothing with
 * the GPU library and is checked against the definition in swdft2d_oracle.c.
 *
 * The paper (arXiv 1707.08213) derives the tree for radix 2 (Section 4.2) and remarks
 * (Section 5) that radix 3 replaces the binary trees by ternary ones, without equations.
 * The recurrence used here, for an axis whose window has n = r^m samples (r = 2 or 3):
 *
 *   level t (t = 1..m) of the tree under position p holds the r^t-point DFT of the samples
 *   x[p - (r^t - 1 - j) * s_t], j < r^t, spaced s_t = r^(m-t) apart and ending at p.  Those
 *   samples split into r interleaved sequences of r^(t-1) samples spaced r * s_t = s_(t-1)
 *   apart; sequence d (d < r) ends at p - (r-1-d) * s_t, so it is level t-1 of the tree at
 *   that position, and the DFT of the whole is
 *
 *     T_t(p)[i] = sum_{d<r} w_{r^t}^{-i d} * T_(t-1)(p - (r-1-d) s_t)[i mod r^(t-1)],  i < r^t,
 *
 *   with w_{r^t}^{-i d} = Om[(i d s_t) mod n], Om[j] = w_n^{-j}.  For r = 2 this is the
 *   paper's Eq. rowfswft2d / colfswft2d.  Level 0 is the data; level m is the window's DFT
 *   in natural order.
 *
 * As in swdft2d_tree_ref.c, the m1 levels of dimension 1 come first, then the m0 levels of
 * dimension 0 (nodes (i0, i1), i1 < n1), levels outermost, two level buffers of
 * N0 N1 n0 n1 complex, and a missing term of an incomplete border tree is taken as 0.
 * opcount: nodes evaluated (each r-1 complex multiply-adds), over all positions.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static const double SWR_TWO_PI = 6.283185307179586476925286766559;

/* n = r^m with r in {2, 3}: returns r and sets *m, or returns 0. */
static int swr_radix(int n, int *m) {
    for (int r = 2; r <= 3; ++r) {
        int k = 0, v = 1;
        while (v < n) {
            v *= r;
            ++k;
        }
        if (v == n) {
            *m = k;
            return n == 1 ? 2 : r;
        }
    }
    return 0;
}

int swt_tree2d_radix_f64(const double *x, int64_t N0, int64_t N1, int n0, int n1, double c, double *out,
                         int64_t *opcount) {
    int m0 = 0, m1 = 0;
    const int r0 = swr_radix(n0, &m0), r1 = swr_radix(n1, &m1);
    if (!r0 || !r1 || n0 < 1 || n1 < 1 || N0 < n0 || N1 < n1) return -1;
    const int64_t nn = (int64_t)n0 * n1, P0 = N0 - n0 + 1, P1 = N1 - n1 + 1;
    const size_t cells = (size_t)(N0 * N1 * nn);
    double *prev = (double *)calloc(2 * cells, sizeof(double));
    double *cur = (double *)calloc(2 * cells, sizeof(double));
    double *om0 = (double *)malloc(sizeof(double) * 2 * (size_t)n0);
    double *om1 = (double *)malloc(sizeof(double) * 2 * (size_t)n1);
    if (!prev || !cur || !om0 || !om1) {
        free(prev);
        free(cur);
        free(om0);
        free(om1);
        return -5;
    }
    for (int j = 0; j < n0; ++j) {
        om0[2 * j] = cos(SWR_TWO_PI * j / n0);
        om0[2 * j + 1] = -sin(SWR_TWO_PI * j / n0);
    }
    for (int j = 0; j < n1; ++j) {
        om1[2 * j] = cos(SWR_TWO_PI * j / n1);
        om1[2 * j + 1] = -sin(SWR_TWO_PI * j / n1);
    }
    for (int64_t p = 0; p < N0 * N1; ++p) {
        prev[2 * p * nn] = x[2 * p];
        prev[2 * p * nn + 1] = x[2 * p + 1];
    }
    int64_t ops = 0;
    /* dimension 1: nodes (0, i1), i1 < r1^t */
    int64_t s = n1, size = 1;
    for (int t = 1; t <= m1; ++t) {
        s /= r1;
        const int64_t half = size; /* r1^(t-1) */
        size *= r1;
        for (int64_t p0 = 0; p0 < N0; ++p0)
            for (int64_t p1 = 0; p1 < N1; ++p1) {
                double *A = cur + 2 * ((p0 * N1 + p1) * nn);
                for (int64_t i = 0; i < size; ++i) {
                    double ar = 0.0, ai = 0.0;
                    for (int d = 0; d < r1; ++d) {
                        const int64_t q = p1 - (int64_t)(r1 - 1 - d) * s;
                        if (q < 0) continue; /* incomplete border tree */
                        const double *T = prev + 2 * ((p0 * N1 + q) * nn + (i % half));
                        const double *w = om1 + 2 * ((i * d * s) % n1);
                        ar += w[0] * T[0] - w[1] * T[1];
                        ai += w[0] * T[1] + w[1] * T[0];
                    }
                    A[2 * i] = ar;
                    A[2 * i + 1] = ai;
                }
                ops += size;
            }
        double *tmp = prev;
        prev = cur;
        cur = tmp;
    }
    /* dimension 0: nodes (i0, i1), i0 < r0^v, i1 < n1 */
    s = n0;
    size = 1;
    for (int v = 1; v <= m0; ++v) {
        s /= r0;
        const int64_t half = size;
        size *= r0;
        for (int64_t p0 = 0; p0 < N0; ++p0)
            for (int64_t p1 = 0; p1 < N1; ++p1) {
                double *A = cur + 2 * ((p0 * N1 + p1) * nn);
                for (int64_t i0 = 0; i0 < size; ++i0)
                    for (int64_t i1 = 0; i1 < n1; ++i1) {
                        double ar = 0.0, ai = 0.0;
                        for (int d = 0; d < r0; ++d) {
                            const int64_t q = p0 - (int64_t)(r0 - 1 - d) * s;
                            if (q < 0) continue;
                            const double *T = prev + 2 * ((q * N1 + p1) * nn + (i0 % half) * n1 + i1);
                            const double *w = om0 + 2 * ((i0 * d * s) % n0);
                            ar += w[0] * T[0] - w[1] * T[1];
                            ai += w[0] * T[1] + w[1] * T[0];
                        }
                        A[2 * (i0 * n1 + i1)] = ar;
                        A[2 * (i0 * n1 + i1) + 1] = ai;
                    }
                ops += size * n1;
            }
        double *tmp = prev;
        prev = cur;
        cur = tmp;
    }
    for (int64_t q0 = 0; q0 < P0; ++q0)
        for (int64_t q1 = 0; q1 < P1; ++q1) {
            const double *T = prev + 2 * (((q0 + n0 - 1) * N1 + (q1 + n1 - 1)) * nn);
            double *o = out + 2 * ((q0 * P1 + q1) * nn);
            for (int64_t k = 0; k < nn; ++k) {
                o[2 * k] = c * T[2 * k];
                o[2 * k + 1] = c * T[2 * k + 1];
            }
        }
    if (opcount) *opcount = ops;
    free(prev);
    free(cur);
    free(om0);
    free(om1);
    return 0;
}

/*
 * Mixed radices within one axis.  The window of an axis has n = r_1 r_2 ... r_L samples and
 * level t of its tree uses radix r_t (2 or 3, in any order).  With N_t = r_1 ... r_t and
 * s_t = n / N_t, level t under position p holds the N_t-point DFT of the samples spaced s_t
 * apart that end at p.  Those samples interleave r_t sequences of N_(t-1) samples spaced
 * r_t s_t = s_(t-1) apart; sequence d ends at p - (r_t - 1 - d) s_t (it is level t-1 of the
 * tree there), so
 *
 *   T_t(p)[i] = sum_{d < r_t} w_{N_t}^{-i d} T_(t-1)(p - (r_t - 1 - d) s_t)[i mod N_(t-1)],
 *
 * w_{N_t}^{-i d} = Om[(i d s_t) mod n], Om[j] = w_n^{-j}: the same recurrence as above with
 * the radix chosen per level (a constant radix gives swt_tree2d_radix_f64).  rad0 / rad1
 * list the radices of dimension 0 / 1 in level order (L0 / L1 entries; L = 0 for n = 1).
 * Same loop order, buffers, border rule and node count as swt_tree2d_radix_f64.
 */
int swt_tree2d_mixed_f64(const double *x, int64_t N0, int64_t N1, const int *rad0, int L0, const int *rad1,
                         int L1, double c, double *out, int64_t *opcount) {
    int n0 = 1, n1 = 1;
    for (int t = 0; t < L0; ++t) {
        if (rad0[t] != 2 && rad0[t] != 3) return -1;
        n0 *= rad0[t];
    }
    for (int t = 0; t < L1; ++t) {
        if (rad1[t] != 2 && rad1[t] != 3) return -1;
        n1 *= rad1[t];
    }
    if (N0 < n0 || N1 < n1) return -1;
    const int64_t nn = (int64_t)n0 * n1, P0 = N0 - n0 + 1, P1 = N1 - n1 + 1;
    const size_t cells = (size_t)(N0 * N1 * nn);
    double *prev = (double *)calloc(2 * cells, sizeof(double));
    double *cur = (double *)calloc(2 * cells, sizeof(double));
    double *om0 = (double *)malloc(sizeof(double) * 2 * (size_t)n0);
    double *om1 = (double *)malloc(sizeof(double) * 2 * (size_t)n1);
    if (!prev || !cur || !om0 || !om1) {
        free(prev);
        free(cur);
        free(om0);
        free(om1);
        return -5;
    }
    for (int j = 0; j < n0; ++j) {
        om0[2 * j] = cos(SWR_TWO_PI * j / n0);
        om0[2 * j + 1] = -sin(SWR_TWO_PI * j / n0);
    }
    for (int j = 0; j < n1; ++j) {
        om1[2 * j] = cos(SWR_TWO_PI * j / n1);
        om1[2 * j + 1] = -sin(SWR_TWO_PI * j / n1);
    }
    for (int64_t p = 0; p < N0 * N1; ++p) {
        prev[2 * p * nn] = x[2 * p];
        prev[2 * p * nn + 1] = x[2 * p + 1];
    }
    int64_t ops = 0;
    /* dimension 1: nodes (0, i1), i1 < N_t */
    int64_t s = n1, size = 1;
    for (int t = 0; t < L1; ++t) {
        const int r = rad1[t];
        s /= r;
        const int64_t prev_size = size; /* N_(t-1) */
        size *= r;
        for (int64_t p0 = 0; p0 < N0; ++p0)
            for (int64_t p1 = 0; p1 < N1; ++p1) {
                double *A = cur + 2 * ((p0 * N1 + p1) * nn);
                for (int64_t i = 0; i < size; ++i) {
                    double ar = 0.0, ai = 0.0;
                    for (int d = 0; d < r; ++d) {
                        const int64_t q = p1 - (int64_t)(r - 1 - d) * s;
                        if (q < 0) continue; /* incomplete border tree */
                        const double *T = prev + 2 * ((p0 * N1 + q) * nn + (i % prev_size));
                        const double *w = om1 + 2 * ((i * d * s) % n1);
                        ar += w[0] * T[0] - w[1] * T[1];
                        ai += w[0] * T[1] + w[1] * T[0];
                    }
                    A[2 * i] = ar;
                    A[2 * i + 1] = ai;
                }
                ops += size;
            }
        double *tmp = prev;
        prev = cur;
        cur = tmp;
    }
    /* dimension 0: nodes (i0, i1), i0 < N_v, i1 < n1 */
    s = n0;
    size = 1;
    for (int v = 0; v < L0; ++v) {
        const int r = rad0[v];
        s /= r;
        const int64_t prev_size = size;
        size *= r;
        for (int64_t p0 = 0; p0 < N0; ++p0)
            for (int64_t p1 = 0; p1 < N1; ++p1) {
                double *A = cur + 2 * ((p0 * N1 + p1) * nn);
                for (int64_t i0 = 0; i0 < size; ++i0)
                    for (int64_t i1 = 0; i1 < n1; ++i1) {
                        double ar = 0.0, ai = 0.0;
                        for (int d = 0; d < r; ++d) {
                            const int64_t q = p0 - (int64_t)(r - 1 - d) * s;
                            if (q < 0) continue;
                            const double *T = prev + 2 * ((q * N1 + p1) * nn + (i0 % prev_size) * n1 + i1);
                            const double *w = om0 + 2 * ((i0 * d * s) % n0);
                            ar += w[0] * T[0] - w[1] * T[1];
                            ai += w[0] * T[1] + w[1] * T[0];
                        }
                        A[2 * (i0 * n1 + i1)] = ar;
                        A[2 * (i0 * n1 + i1) + 1] = ai;
                    }
                ops += size * n1;
            }
        double *tmp = prev;
        prev = cur;
        cur = tmp;
    }
    for (int64_t q0 = 0; q0 < P0; ++q0)
        for (int64_t q1 = 0; q1 < P1; ++q1) {
            const double *T = prev + 2 * (((q0 + n0 - 1) * N1 + (q1 + n1 - 1)) * nn);
            double *o = out + 2 * ((q0 * P1 + q1) * nn);
            for (int64_t k = 0; k < nn; ++k) {
                o[2 * k] = c * T[2 * k];
                o[2 * k + 1] = c * T[2 * k + 1];
            }
        }
    if (opcount) *opcount = ops;
    free(prev);
    free(cur);
    free(om0);
    free(om1);
    return 0;
}
