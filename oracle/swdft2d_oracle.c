/*
 * FP64 CPU oracle for the 2D sliding window DFT of Richardson & Eddy, "The 2D Tree Sliding
 * Window Discrete Fourier Transform" (arXiv 1707.08213).
 *
 * TEST INFRASTRUCTURE ONLY.  The only callers are the tests, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py.  The GPU library never includes, links or loads this file,
 * and this file uses no code, header or table of the GPU library.
 *
 * What it computes is the plain definition, Section 4.1, Eq. (2):
 *
 *   a[p0,p1,k0,k1] = c * sum_{j0<n0} sum_{j1<n1} x[p0-n0+1+j0, p1-n1+1+j1]
 *                        * w_{n0}^{-j0 k0} * w_{n1}^{-j1 k1},      w_n = exp(2*pi*i/n),
 *
 * for every window that lies inside the array (p_i = n_i-1 .. N_i-1).  Windows are stored by
 * their first row/column q_i = p_i - (n_i - 1), so the output is row-major
 * [q0][q1][k0][k1] complex128 (interleaved re, im), q_i < P_i = N_i - n_i + 1.
 * The scale c is a parameter: Eq. (2) uses 1/sqrt(n0 n1); 1 gives the bare sums.
 *
 * Exponentials are tabulated once per transform length as cos/sin(2*pi*((j*k) mod n)/n),
 * so no phase is evaluated at an argument beyond 2*pi.
 *
 * Two evaluation orders of the same sum are offered:
 *   direct     - the double sum over (j0, j1) exactly as Eq. (2) is written;
 *   separable  - the row-column factorisation of Section 4.2 (Eqs. 3-4): first
 *                z[j0,k1] = sum_j1 x[.,.] w_{n1}^{-j1 k1}, then a = sum_j0 z[j0,k1] w_{n0}^{-j0 k0}.
 *                It is the same sum with the j1 loop moved inside; no tree and no FFT.
 *
 * The adjoint A^H (used to check the hand-written adjoint) is the explicit conjugate sum:
 *   g[r,c] = sum over windows q containing (r,c) of c * sum_k G[q,k] * conj(w_{n0}^{-(r-q0)k0} w_{n1}^{-(c-q1)k1}).
 *
 * Compiled with -fopenmp the window loops may run on several threads (nthreads > 1);
 * each window's result is independent, so the arithmetic is identical to one thread.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define SWO_OK 0
#define SWO_EINVAL (-1)
#define SWO_ENOMEM (-5)

static const double SWO_TWO_PI = 6.283185307179586476925286766559;

/* w[j] = w_n^{-j} = exp(-2*pi*i*j/n), j < n, interleaved (re, im). */
static double *omega_table(int n) {
    double *w = (double *)malloc(sizeof(double) * 2 * (size_t)n);
    if (!w) return NULL;
    for (int j = 0; j < n; ++j) {
        double ang = SWO_TWO_PI * (double)j / (double)n;
        w[2 * j] = cos(ang);
        w[2 * j + 1] = -sin(ang);
    }
    return w;
}

static int check_shape(int64_t N0, int64_t N1, int n0, int n1) {
    if (N0 < 1 || N1 < 1 || n0 < 1 || n1 < 1 || n0 > N0 || n1 > N1) return SWO_EINVAL;
    return SWO_OK;
}

/* One window by the direct double sum of Eq. (2).  out: n0*n1 complex. */
static void window_direct(const double *x, int64_t N1, int64_t q0, int64_t q1, int n0, int n1,
                          const double *w0, const double *w1, double c, double *out) {
    for (int k0 = 0; k0 < n0; ++k0) {
        for (int k1 = 0; k1 < n1; ++k1) {
            double sr = 0.0, si = 0.0;
            for (int j0 = 0; j0 < n0; ++j0) {
                const double *e0 = w0 + 2 * (((int64_t)j0 * k0) % n0);
                for (int j1 = 0; j1 < n1; ++j1) {
                    const double *e1 = w1 + 2 * (((int64_t)j1 * k1) % n1);
                    /* kernel = w_{n0}^{-j0k0} * w_{n1}^{-j1k1} */
                    double er = e0[0] * e1[0] - e0[1] * e1[1];
                    double ei = e0[0] * e1[1] + e0[1] * e1[0];
                    const double *v = x + 2 * ((q0 + j0) * N1 + (q1 + j1));
                    sr += v[0] * er - v[1] * ei;
                    si += v[0] * ei + v[1] * er;
                }
            }
            out[2 * (k0 * n1 + k1)] = c * sr;
            out[2 * (k0 * n1 + k1) + 1] = c * si;
        }
    }
}

/* One window by the row-column factorisation (Section 4.2).  z: scratch n0*n1 complex. */
static void window_separable(const double *x, int64_t N1, int64_t q0, int64_t q1, int n0, int n1,
                             const double *w0, const double *w1, double c, double *z, double *out) {
    /* z[j0,k1] = sum_j1 x[q0+j0, q1+j1] w_{n1}^{-j1 k1} */
    for (int j0 = 0; j0 < n0; ++j0) {
        const double *row = x + 2 * ((q0 + j0) * N1 + q1);
        for (int k1 = 0; k1 < n1; ++k1) {
            double sr = 0.0, si = 0.0;
            for (int j1 = 0; j1 < n1; ++j1) {
                const double *e = w1 + 2 * (((int64_t)j1 * k1) % n1);
                sr += row[2 * j1] * e[0] - row[2 * j1 + 1] * e[1];
                si += row[2 * j1] * e[1] + row[2 * j1 + 1] * e[0];
            }
            z[2 * (j0 * n1 + k1)] = sr;
            z[2 * (j0 * n1 + k1) + 1] = si;
        }
    }
    /* a[k0,k1] = sum_j0 z[j0,k1] w_{n0}^{-j0 k0} */
    for (int k0 = 0; k0 < n0; ++k0) {
        for (int k1 = 0; k1 < n1; ++k1) {
            double sr = 0.0, si = 0.0;
            for (int j0 = 0; j0 < n0; ++j0) {
                const double *e = w0 + 2 * (((int64_t)j0 * k0) % n0);
                const double *v = z + 2 * (j0 * n1 + k1);
                sr += v[0] * e[0] - v[1] * e[1];
                si += v[0] * e[1] + v[1] * e[0];
            }
            out[2 * (k0 * n1 + k1)] = c * sr;
            out[2 * (k0 * n1 + k1) + 1] = c * si;
        }
    }
}

/*
 * Every window of an N0 x N1 complex array x (row-major, interleaved).
 * method 0 = direct double sum, 1 = row-column factorisation.
 * out: P0*P1*n0*n1 complex, [q0][q1][k0][k1].
 */
int swo_swdft2d(const double *x, int64_t N0, int64_t N1, int n0, int n1, double c, int method,
                int nthreads, double *out) {
    if (check_shape(N0, N1, n0, n1)) return SWO_EINVAL;
    const int64_t P0 = N0 - n0 + 1, P1 = N1 - n1 + 1;
    double *w0 = omega_table(n0), *w1 = omega_table(n1);
    if (!w0 || !w1) { free(w0); free(w1); return SWO_ENOMEM; }
    int err = SWO_OK;
    (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
#endif
    {
        double *z = (double *)malloc(sizeof(double) * 2 * (size_t)n0 * n1);
        if (!z) {
            err = SWO_ENOMEM;
        } else {
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
            for (int64_t q0 = 0; q0 < P0; ++q0) {
                for (int64_t q1 = 0; q1 < P1; ++q1) {
                    double *o = out + 2 * ((q0 * P1 + q1) * (int64_t)n0 * n1);
                    if (method == 0)
                        window_direct(x, N1, q0, q1, n0, n1, w0, w1, c, o);
                    else
                        window_separable(x, N1, q0, q1, n0, n1, w0, w1, c, z, o);
                }
            }
            free(z);
        }
    }
    free(w0);
    free(w1);
    return err;
}

/* Selected windows (q0s[i], q1s[i]); out: nwin*n0*n1 complex. */
int swo_swdft2d_windows(const double *x, int64_t N0, int64_t N1, int n0, int n1, double c,
                        int method, int64_t nwin, const int64_t *q0s, const int64_t *q1s,
                        int nthreads, double *out) {
    if (check_shape(N0, N1, n0, n1)) return SWO_EINVAL;
    const int64_t P0 = N0 - n0 + 1, P1 = N1 - n1 + 1;
    for (int64_t i = 0; i < nwin; ++i)
        if (q0s[i] < 0 || q0s[i] >= P0 || q1s[i] < 0 || q1s[i] >= P1) return SWO_EINVAL;
    double *w0 = omega_table(n0), *w1 = omega_table(n1);
    if (!w0 || !w1) { free(w0); free(w1); return SWO_ENOMEM; }
    int err = SWO_OK;
    (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
#endif
    {
        double *z = (double *)malloc(sizeof(double) * 2 * (size_t)n0 * n1);
        if (!z) {
            err = SWO_ENOMEM;
        } else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
            for (int64_t i = 0; i < nwin; ++i) {
                double *o = out + 2 * (i * (int64_t)n0 * n1);
                if (method == 0)
                    window_direct(x, N1, q0s[i], q1s[i], n0, n1, w0, w1, c, o);
                else
                    window_separable(x, N1, q0s[i], q1s[i], n0, n1, w0, w1, c, z, o);
            }
            free(z);
        }
    }
    free(w0);
    free(w1);
    return err;
}

/*
 * Adjoint A^H G for an N0 x N1 input: G is P0*P1*n0*n1 complex ([q0][q1][k0][k1]),
 * g is N0*N1 complex.  method 0 = direct sum per pixel contribution,
 * 1 = separable: per window an inverse transform along k0 then k1, then overlap-add.
 * Single-threaded (the overlap-add writes shared pixels).
 */
int swo_swdft2d_adjoint(const double *G, int64_t N0, int64_t N1, int n0, int n1, double c,
                        int method, double *g) {
    if (check_shape(N0, N1, n0, n1)) return SWO_EINVAL;
    const int64_t P0 = N0 - n0 + 1, P1 = N1 - n1 + 1;
    double *w0 = omega_table(n0), *w1 = omega_table(n1);
    double *y = (double *)malloc(sizeof(double) * 2 * (size_t)n0 * n1);
    if (!w0 || !w1 || !y) { free(w0); free(w1); free(y); return SWO_ENOMEM; }
    memset(g, 0, sizeof(double) * 2 * (size_t)(N0 * N1));
    for (int64_t q0 = 0; q0 < P0; ++q0) {
        for (int64_t q1 = 0; q1 < P1; ++q1) {
            const double *Gw = G + 2 * ((q0 * P1 + q1) * (int64_t)n0 * n1);
            if (method == 0) {
                for (int j0 = 0; j0 < n0; ++j0) {
                    for (int j1 = 0; j1 < n1; ++j1) {
                        double sr = 0.0, si = 0.0;
                        for (int k0 = 0; k0 < n0; ++k0) {
                            const double *e0 = w0 + 2 * (((int64_t)j0 * k0) % n0);
                            for (int k1 = 0; k1 < n1; ++k1) {
                                const double *e1 = w1 + 2 * (((int64_t)j1 * k1) % n1);
                                double er = e0[0] * e1[0] - e0[1] * e1[1];
                                double ei = -(e0[0] * e1[1] + e0[1] * e1[0]); /* conjugate */
                                const double *v = Gw + 2 * (k0 * n1 + k1);
                                sr += v[0] * er - v[1] * ei;
                                si += v[0] * ei + v[1] * er;
                            }
                        }
                        double *d = g + 2 * ((q0 + j0) * N1 + (q1 + j1));
                        d[0] += c * sr;
                        d[1] += c * si;
                    }
                }
            } else {
                /* y[j0,k1] = sum_k0 G[k0,k1] conj(w_{n0}^{-j0 k0}) */
                for (int j0 = 0; j0 < n0; ++j0) {
                    for (int k1 = 0; k1 < n1; ++k1) {
                        double sr = 0.0, si = 0.0;
                        for (int k0 = 0; k0 < n0; ++k0) {
                            const double *e = w0 + 2 * (((int64_t)j0 * k0) % n0);
                            const double *v = Gw + 2 * (k0 * n1 + k1);
                            sr += v[0] * e[0] + v[1] * e[1];
                            si += v[1] * e[0] - v[0] * e[1];
                        }
                        y[2 * (j0 * n1 + k1)] = sr;
                        y[2 * (j0 * n1 + k1) + 1] = si;
                    }
                }
                /* g[q0+j0, q1+j1] += c * sum_k1 y[j0,k1] conj(w_{n1}^{-j1 k1}) */
                for (int j0 = 0; j0 < n0; ++j0) {
                    for (int j1 = 0; j1 < n1; ++j1) {
                        double sr = 0.0, si = 0.0;
                        for (int k1 = 0; k1 < n1; ++k1) {
                            const double *e = w1 + 2 * (((int64_t)j1 * k1) % n1);
                            const double *v = y + 2 * (j0 * n1 + k1);
                            sr += v[0] * e[0] + v[1] * e[1];
                            si += v[1] * e[0] - v[0] * e[1];
                        }
                        double *d = g + 2 * ((q0 + j0) * N1 + (q1 + j1));
                        d[0] += c * sr;
                        d[1] += c * si;
                    }
                }
            }
        }
    }
    free(w0);
    free(w1);
    free(y);
    return SWO_OK;
}

/* (A^H G) at selected pixels (rs[i], cs[i]) by the direct sum; out: npix complex. */
int swo_swdft2d_adjoint_pixels(const double *G, int64_t N0, int64_t N1, int n0, int n1, double c,
                               int64_t npix, const int64_t *rs, const int64_t *cs, int nthreads,
                               double *out) {
    if (check_shape(N0, N1, n0, n1)) return SWO_EINVAL;
    const int64_t P0 = N0 - n0 + 1, P1 = N1 - n1 + 1;
    for (int64_t i = 0; i < npix; ++i)
        if (rs[i] < 0 || rs[i] >= N0 || cs[i] < 0 || cs[i] >= N1) return SWO_EINVAL;
    double *w0 = omega_table(n0), *w1 = omega_table(n1);
    if (!w0 || !w1) { free(w0); free(w1); return SWO_ENOMEM; }
    (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads > 0 ? nthreads : 1) schedule(dynamic, 4)
#endif
    for (int64_t i = 0; i < npix; ++i) {
        const int64_t r = rs[i], col = cs[i];
        double sr = 0.0, si = 0.0;
        for (int j0 = 0; j0 < n0; ++j0) {
            const int64_t q0 = r - j0;
            if (q0 < 0 || q0 >= P0) continue;
            for (int j1 = 0; j1 < n1; ++j1) {
                const int64_t q1 = col - j1;
                if (q1 < 0 || q1 >= P1) continue;
                const double *Gw = G + 2 * ((q0 * P1 + q1) * (int64_t)n0 * n1);
                for (int k0 = 0; k0 < n0; ++k0) {
                    const double *e0 = w0 + 2 * (((int64_t)j0 * k0) % n0);
                    for (int k1 = 0; k1 < n1; ++k1) {
                        const double *e1 = w1 + 2 * (((int64_t)j1 * k1) % n1);
                        double er = e0[0] * e1[0] - e0[1] * e1[1];
                        double ei = -(e0[0] * e1[1] + e0[1] * e1[0]);
                        const double *v = Gw + 2 * (k0 * n1 + k1);
                        sr += v[0] * er - v[1] * ei;
                        si += v[0] * ei + v[1] * er;
                    }
                }
            }
        }
        out[2 * i] = c * sr;
        out[2 * i + 1] = c * si;
    }
    free(w0);
    free(w1);
    return SWO_OK;
}

int swo_openmp_available(void) {
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}
