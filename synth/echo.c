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
 * steps, which keeps the FP64 phase error below 1e-13 rad; scatterers are
 * processed in blocks of 8 so that the per-frequency update vectorises.
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
            /* scatterers in blocks of SB so the per-frequency update runs
             * across a block (vectorisable); the phase of each scatterer is
             * re-anchored from an exact sincos every 32 frequencies */
            enum { SB = 8 };
            for (int s0 = 0; s0 < S; s0 += SB) {
                const int nb = S - s0 < SB ? S - s0 : SB;
                double Rrt[SB], amp[SB], cr[SB], ci[SB], zr[SB], zi[SB];
                for (int j = 0; j < SB; ++j) {
                    Rrt[j] = 0.0; amp[j] = 0.0; cr[j] = 1.0; ci[j] = 0.0; zr[j] = 0.0; zi[j] = 0.0;
                    if (j >= nb) continue;
                    const double *q = scat + 4 * (s0 + j);
                    const double dTx = Tx - q[0], dTy = Ty - q[1], dTz = Tz - q[2];
                    const double dRx = Rx - q[0], dRy = Ry - q[1], dRz = Rz - q[2];
                    const double RT = sqrt(dTx * dTx + dTy * dTy + dTz * dTz);
                    const double RR = sqrt(dRx * dRx + dRy * dRy + dRz * dRz);
                    Rrt[j] = RT + RR;
                    amp[j] = q[3] * (amplitude ? 1.0 / (RT * RR) : 1.0);
                    /* rotation by exp(-j * 2*pi*df/c * Rrt) per frequency step */
                    const double dphi = -two_pi * df / SYNTH_C0 * Rrt[j];
                    cr[j] = cos(dphi);
                    ci[j] = sin(dphi);
                }
                for (int k0 = 0; k0 < Nk; k0 += 32) {
                    for (int j = 0; j < nb; ++j) {
                        const double phi = -two_pi * (f0 + df * k0) / SYNTH_C0 * Rrt[j];
                        zr[j] = amp[j] * cos(phi);
                        zi[j] = amp[j] * sin(phi);
                    }
                    const int k1 = k0 + 32 < Nk ? k0 + 32 : Nk;
                    for (int k = k0; k < k1; ++k) {
                        double sr = 0.0, si = 0.0;
                        for (int j = 0; j < SB; ++j) {
                            sr += zr[j];
                            si += zi[j];
                            const double nr = zr[j] * cr[j] - zi[j] * ci[j];
                            zi[j] = zr[j] * ci[j] + zi[j] * cr[j];
                            zr[j] = nr;
                        }
                        acc[2 * k] += sr;
                        acc[2 * k + 1] += si;
                    }
                }
            }
            float *o = out + (size_t)l * 2 * Nk;
            for (int k = 0; k < 2 * Nk; ++k) o[k] = (float)acc[k];
        }
        free(acc);
    }
    return 0;
}
