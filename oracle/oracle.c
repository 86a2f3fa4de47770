/*
 * FP64 CPU oracle helpers -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain loops (OpenMP-parallel over independent outputs) used by the Python
 * oracle in this directory.  Nothing in the product library calls or links
 * this file; only tests, the smoke check and the CPU-baseline leg of the
 * benchmark execute it.
 *
 *  - orc_spread2d / orc_spread1d: the Gaussian gridding step of the fast
 *    Gaussian gridding NUFFT (Greengard & Lee) that Sec. III uses for the
 *    Fourier transforms and the Stolt step of Eq. 16.  Each sample at
 *    position x (radians, 2*pi-periodic) adds c * exp(-(x - j*h)^2 / (4 tau))
 *    to the w grid points j = ceil(x/h - w/2) + 0..w-1 (indices mod the grid
 *    size), h = 2*pi / grid size.
 *  - orc_bpa: direct back-projection (Sec. III, the "gold standard"),
 *    o(r) = sum_{t,r,p,k} s * exp(+j k (|T - r| + |R - r|)), Eq. 2 distances.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_C0 299792458.0
#define ORC_2PI 6.283185307179586476925286766559

static long orc_mod(long a, long m) { long r = a % m; return r < 0 ? r + m : r; }

/* 2-D spreading of Nk-vectors.  x[L], y[L] in radians; c[L][Nk];
 * G[Mry][Mrx][Nk] accumulated in place (caller zero-fills).
 * Threads own disjoint k ranges, so there are no write races. */
void orc_spread2d(long L, int Nk, const double *x, const double *y,
                  const double complex *c, int Mrx, int Mry, int w,
                  double taux, double tauy, double complex *G)
{
    const double hx = ORC_2PI / Mrx, hy = ORC_2PI / Mry;
#pragma omp parallel
    {
#ifdef _OPENMP
        const int nt = omp_get_num_threads(), me = omp_get_thread_num();
#else
        const int nt = 1, me = 0;
#endif
        const int k_lo = (int)((long)Nk * me / nt), k_hi = (int)((long)Nk * (me + 1) / nt);
        double *wx = (double *)malloc(sizeof(double) * w);
        double *wy = (double *)malloc(sizeof(double) * w);
        long *jx = (long *)malloc(sizeof(long) * w);
        long *jy = (long *)malloc(sizeof(long) * w);
        if (k_hi > k_lo) {
            for (long l = 0; l < L; ++l) {
                const long jx0 = (long)ceil(x[l] / hx - 0.5 * w);
                const long jy0 = (long)ceil(y[l] / hy - 0.5 * w);
                for (int a = 0; a < w; ++a) {
                    const double dxa = x[l] - (double)(jx0 + a) * hx;
                    const double dya = y[l] - (double)(jy0 + a) * hy;
                    wx[a] = exp(-dxa * dxa / (4.0 * taux));
                    wy[a] = exp(-dya * dya / (4.0 * tauy));
                    jx[a] = orc_mod(jx0 + a, Mrx);
                    jy[a] = orc_mod(jy0 + a, Mry);
                }
                const double complex *cl = c + (size_t)l * Nk;
                for (int b = 0; b < w; ++b) {
                    for (int a = 0; a < w; ++a) {
                        const double wt = wx[a] * wy[b];
                        double complex *g = G + ((size_t)jy[b] * Mrx + (size_t)jx[a]) * Nk;
                        for (int k = k_lo; k < k_hi; ++k) g[k] += wt * cl[k];
                    }
                }
            }
        }
        free(wx); free(wy); free(jx); free(jy);
    }
}

/* 1-D spreading, one independent problem per column.
 * t[ncols][Nk] (radians), c[ncols][Nk]; g[ncols][Mr] accumulated in place. */
void orc_spread1d(long ncols, int Nk, const double *t, const double complex *c,
                  int Mr, int w, double tau, double complex *g)
{
    const double h = ORC_2PI / Mr;
#pragma omp parallel for schedule(static)
    for (long col = 0; col < ncols; ++col) {
        const double *tc = t + (size_t)col * Nk;
        const double complex *cc = c + (size_t)col * Nk;
        double complex *gc = g + (size_t)col * Mr;
        for (int k = 0; k < Nk; ++k) {
            if (cc[k] == 0.0) continue;
            const long j0 = (long)ceil(tc[k] / h - 0.5 * w);
            for (int a = 0; a < w; ++a) {
                const double d = tc[k] - (double)(j0 + a) * h;
                gc[orc_mod(j0 + a, Mr)] += cc[k] * exp(-d * d / (4.0 * tau));
            }
        }
    }
}

/* Direct back-projection at nvox voxels.
 * echo[T][R][P][Nk] complex, pos[P][3], tx[T][3], rx[R][3], freq[Nk] (Hz),
 * vox[nvox][3]; out[nvox]. */
void orc_bpa(int T, int R, int P, int Nk, const double *pos, const double *tx,
             const double *rx, const double *freq, const double complex *echo,
             long nvox, const double *vox, double complex *out)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (long v = 0; v < nvox; ++v) {
        const double X = vox[3 * v], Y = vox[3 * v + 1], Z = vox[3 * v + 2];
        double complex acc = 0.0;
        for (int t = 0; t < T; ++t)
            for (int r = 0; r < R; ++r)
                for (int p = 0; p < P; ++p) {
                    const double ax = pos[3 * p] + tx[3 * t] - X;
                    const double ay = pos[3 * p + 1] + tx[3 * t + 1] - Y;
                    const double az = pos[3 * p + 2] + tx[3 * t + 2] - Z;
                    const double bx = pos[3 * p] + rx[3 * r] - X;
                    const double by = pos[3 * p + 1] + rx[3 * r + 1] - Y;
                    const double bz = pos[3 * p + 2] + rx[3 * r + 2] - Z;
                    const double Rrt = sqrt(ax * ax + ay * ay + az * az) + sqrt(bx * bx + by * by + bz * bz);
                    const double complex *s = echo + (((size_t)t * R + r) * P + p) * Nk;
                    for (int k = 0; k < Nk; ++k) {
                        const double kk = ORC_2PI * freq[k] / ORC_C0;
                        acc += s[k] * cexp(I * kk * Rrt);
                    }
                }
        out[v] = acc;
    }
}
