/*
 * Synthetic MIMO-SAR echo generator (input synthesis only; not part of the
 * imaging method).
 *
 * Forward model of the frequency-domain echo, Sec. II-C, Eq. 9, with the
 * amplitude factor 1/(R_T R_R) and the pulse spectrum P(f) taken as 1:
 *
 *   s(t, r, p, k) = sum_s sigma_s * exp(-j * k_k * (|T_tp - r_s| + |R_rp - r_s|))
 *
 * where k_k = 2*pi*f_k/c, f_k = f0 + k*df, T_tp = pos_p + tx_t and
 * R_rp = pos_p + rx_r (round-trip distance of Eq. 2).  The optional
 * amplitude flag multiplies each term by 1/(|T-r||R-r|) (Eq. 9 as printed).
 *
 * The phase over the uniform frequency grid is generated by a complex
 * rotation recurrence that is re-anchored from an exact sincos every 32
 * steps, which keeps the FP64 phase error below 1e-13 rad.
 *
 * Layout: pos [P][3], tx [T][3], rx [R][3], scat [S][4] = (x, y, z, sigma),
 * out [T][R][P][Nk][2] float (interleaved re, im).  All metres / Hz.
 */
#include <math.h>
#include <stdlib.h>

#define SYNTH_C0 299792458.0

int synth_echo(int T, int R, int P, int Nk,
               const double *pos, const double *tx, const double *rx,
               double f0, double df,
               int S, const double *scat, int amplitude,
               float *out)
{
    if (T < 0 || R < 0 || P < 0 || Nk <= 0 || S < 0) return -1;
    const double two_pi = 6.283185307179586476925286766559;
    const long long L = (long long)T * R * P;
#pragma omp parallel
    {
        double *acc = (double *)malloc(sizeof(double) * 2 * (size_t)Nk);
#pragma omp for schedule(static)
        for (long long l = 0; l < L; ++l) {
            const int p = (int)(l % P);
            const int r = (int)((l / P) % R);
            const int t = (int)(l / ((long long)P * R));
            const double Tx = pos[3 * p + 0] + tx[3 * t + 0];
            const double Ty = pos[3 * p + 1] + tx[3 * t + 1];
            const double Tz = pos[3 * p + 2] + tx[3 * t + 2];
            const double Rx = pos[3 * p + 0] + rx[3 * r + 0];
            const double Ry = pos[3 * p + 1] + rx[3 * r + 1];
            const double Rz = pos[3 * p + 2] + rx[3 * r + 2];
            for (int k = 0; k < 2 * Nk; ++k) acc[k] = 0.0;
            for (int s = 0; s < S; ++s) {
                const double *q = scat + 4 * s;
                const double dTx = Tx - q[0], dTy = Ty - q[1], dTz = Tz - q[2];
                const double dRx = Rx - q[0], dRy = Ry - q[1], dRz = Rz - q[2];
                const double RT = sqrt(dTx * dTx + dTy * dTy + dTz * dTz);
                const double RR = sqrt(dRx * dRx + dRy * dRy + dRz * dRz);
                const double Rrt = RT + RR;
                const double amp = q[3] * (amplitude ? 1.0 / (RT * RR) : 1.0);
                /* rotation by exp(-j * 2*pi*df/c * Rrt) per frequency step */
                const double dphi = -two_pi * df / SYNTH_C0 * Rrt;
                const double cr = cos(dphi), ci = sin(dphi);
                double zr = 0.0, zi = 0.0;
                for (int k = 0; k < Nk; ++k) {
                    if ((k & 31) == 0) {
                        const double phi = -two_pi * (f0 + df * k) / SYNTH_C0 * Rrt;
                        zr = amp * cos(phi);
                        zi = amp * sin(phi);
                    }
                    acc[2 * k] += zr;
                    acc[2 * k + 1] += zi;
                    const double nr = zr * cr - zi * ci;
                    zi = zr * ci + zi * cr;
                    zr = nr;
                }
            }
            float *o = out + (size_t)l * 2 * Nk;
            for (int k = 0; k < 2 * Nk; ++k) o[k] = (float)acc[k];
        }
        free(acc);
    }
    return 0;
}
