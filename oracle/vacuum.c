/*
 * FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Random numbers, Fourier transforms, Gaussian vacuum initial conditions and
 * binned power spectra:
 *   - Philox-4x32-10 counter-based generator, from its published definition
 *     (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 *     SC'11): 10 rounds of two 32x32->64 multiplies with the Weyl key schedule.
 *   - a plain O(N) per output direct DFT along each axis (no FFT algorithm), with
 *     the paper's convention f(n) = N^-3 sum_k e^{+i 2 pi k.n/N} f(k)
 *     (section "Arbitrary binning and unbinned spectra", Eq. discretePSaux).
 *   - vacuum fluctuations of Eq. QuantumFlucts set through Eq. fpr_influct and
 *     Eq. fpr_influct2, with variance (N/dx)^3 P(k) per mode (Eq. varFandDFgeneral,
 *     Upsilon = 1) split evenly between real and imaginary parts.
 *   - the binned spectrum of Eq. discretePST2 / Eq. UpsilonII (Type I and II).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------- Philox */

static void mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo32(0xD2511F53u, c0, &hi0, &lo0);
        mulhilo32(0xCD9E8D57u, c2, &hi1, &lo1);
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Four standard normals from one Philox block: u = (x + 1/2) 2^-32 in (0,1),
 * then two Box-Muller pairs (u0,u1) and (u2,u3). */
static void gauss4(uint32_t idx, uint32_t field, uint32_t member, uint64_t seed, double z[4])
{
    uint32_t ctr[4] = {idx, field, member, 0u};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    double u[4];
    for (int i = 0; i < 4; ++i) u[i] = ((double)r[i] + 0.5) * (1.0 / 4294967296.0);
    const double two_pi = 6.283185307179586476925286766559;
    double rho0 = sqrt(-2.0 * log(u[0])), rho1 = sqrt(-2.0 * log(u[2]));
    z[0] = rho0 * cos(two_pi * u[1]);
    z[1] = rho0 * sin(two_pi * u[1]);
    z[2] = rho1 * cos(two_pi * u[3]);
    z[3] = rho1 * sin(two_pi * u[3]);
}

/* ---------------------------------------------------------------------- DFT */

/* In-place 3-D DFT, sign = -1: F(k) = sum_n e^{-i 2pi k.n/N} f(n);
 * sign = +1: f(n) = N^-3 sum_k e^{+i 2pi k.n/N} F(k). */
void orc_dft3(int N, int sign, double* re, double* im)
{
    double* cr = malloc(sizeof(double) * N);
    double* ci = malloc(sizeof(double) * N);
    double* tr = malloc(sizeof(double) * N);
    double* ti = malloc(sizeof(double) * N);
    const double two_pi = 6.283185307179586476925286766559;
    for (int j = 0; j < N; ++j) {
        cr[j] = cos(two_pi * j / N);
        ci[j] = sign * sin(two_pi * j / N);
    }
    const int64_t stride[3] = {1, N, (int64_t)N * N};
    for (int axis = 0; axis < 3; ++axis) {
        const int64_t s = stride[axis];
        for (int64_t line = 0; line < (int64_t)N * N; ++line) {
            /* base index of the line: the two other coordinates */
            int64_t u = line % N, v = line / N, base;
            if (axis == 0) base = u * N + v * N * N;
            else if (axis == 1) base = u + v * N * N;
            else base = u + v * N;
            for (int k = 0; k < N; ++k) {
                double sr = 0.0, si = 0.0;
                for (int n = 0; n < N; ++n) {
                    int j = (int)(((int64_t)k * n) % N);
                    double xr = re[base + n * s], xi = im[base + n * s];
                    sr += xr * cr[j] - xi * ci[j];
                    si += xr * ci[j] + xi * cr[j];
                }
                tr[k] = sr;
                ti[k] = si;
            }
            for (int k = 0; k < N; ++k) {
                re[base + k * s] = tr[k];
                im[base + k * s] = ti[k];
            }
        }
    }
    if (sign > 0) {
        const double inv = 1.0 / ((double)N * N * N);
        for (int64_t n = 0; n < (int64_t)N * N * N; ++n) { re[n] *= inv; im[n] *= inv; }
    }
    free(cr); free(ci); free(tr); free(ti);
}

/* ------------------------------------------------------ vacuum initial state */

static int signed_mode(int i, int N) { return (i <= N / 2) ? i : i - N; }

/* Mode value of field f at Fourier index (i,j,k): returns delta f(k) and
 * delta pi(k) = a^(3-alpha) delta f'(k).  The spectrum is Hermitian by
 * construction: of the pair {k, -k} the one with the smaller linear index draws
 * the random numbers, the other takes the complex conjugate; self-conjugate
 * modes keep the real part. */
static void vacuum_mode(const orc_model* m, uint64_t seed, uint32_t member, int f, double kcut, double amp2,
                        double a, double H, double m2eff, int i, int j, int k,
                        double* fr, double* fi, double* pr, double* pim)
{
    const int N = m->N;
    *fr = *fi = *pr = *pim = 0.0;
    const int si = signed_mode(i, N), sj = signed_mode(j, N), sk = signed_mode(k, N);
    if (si == 0 && sj == 0 && sk == 0) return;
    const double dx = m->L / N;
    const double kIR = 6.283185307179586476925286766559 / m->L;
    const double kmod = kIR * sqrt((double)si * si + (double)sj * sj + (double)sk * sk);
    if (kmod > kcut) return;

    const int ci = (N - i) % N, cj = (N - j) % N, ck = (N - k) % N;
    const int64_t idx = ((int64_t)k * N + j) * N + i;
    const int64_t cidx = ((int64_t)ck * N + cj) * N + ci;
    const int64_t draw = idx <= cidx ? idx : cidx;
    double z[4];
    gauss4((uint32_t)draw, (uint32_t)f, member, seed, z);

    /* Eq. QuantumFlucts in program units: P = (omega_star / f_star)^2 / (2 a^2 omega_k),
     * omega_k = sqrt(k^2 + a^2 m^2); variance of each real component = (N/dx)^3 P / 2. */
    const double omega = sqrt(kmod * kmod + a * a * m2eff);
    const double P = amp2 / (2.0 * a * a * omega);
    const double sigma = sqrt(0.5 * pow(N / dx, 3.0) * P);
    const double lr = z[0], li = z[1], rr = z[2], ri = z[3];
    const double isq2 = 0.70710678118654752440084436210485;
    /* Eq. fpr_influct: delta f = (f_l + f_r)/sqrt2 */
    double Fr = sigma * (lr + rr) * isq2, Fi = sigma * (li + ri) * isq2;
    /* Eq. fpr_influct2: delta f' = a^(alpha-1) i omega (f_l - f_r)/sqrt2 - H delta f */
    const double c1 = pow(a, m->alpha - 1.0) * omega * sigma * isq2;
    double Dr = -c1 * (li - ri) - H * Fr;
    double Di = c1 * (lr - rr) - H * Fi;
    const double cp = pow(a, 3.0 - m->alpha);
    double Pr = cp * Dr, Pi = cp * Di;
    if (idx == cidx) { Fi = 0.0; Pi = 0.0; }      /* self-conjugate: real */
    else if (idx != draw) { Fi = -Fi; Pi = -Pi; } /* conjugate partner    */
    *fr = Fr; *fi = Fi; *pr = Pr; *pim = Pi;
}

void orc_vacuum(const orc_model* m, uint64_t seed, uint32_t member, double kcut, double amp2,
                const double* fbar, const double* dfbar, double a0,
                double* phi, double* pi, double* abt)
{
    const int N = m->N;
    const int64_t V = (int64_t)N * N * N;
    const double a = a0;
    const double f0 = fbar[0], f1 = m->nf > 1 ? fbar[1] : 0.0;

    /* homogeneous Hubble rate from the homogeneous energy (Eq. Friedmann2) */
    double rho_h = orc_V(m, f0, f1);
    for (int f = 0; f < m->nf; ++f) rho_h += dfbar[f] * dfbar[f] / (2.0 * pow(a, 2.0 * m->alpha));
    const double H = m->expansion ? sqrt(pow(a, 2.0 * m->alpha) * m->kappa * rho_h / 3.0) : 0.0;

    double* re = malloc(sizeof(double) * (size_t)V);
    double* im = malloc(sizeof(double) * (size_t)V);
    double* pre = malloc(sizeof(double) * (size_t)V);
    double* pim = malloc(sizeof(double) * (size_t)V);
    for (int f = 0; f < m->nf; ++f) {
        const double m2eff = orc_d2V(m, f, f0, f1); /* m^2 = V'' at the homogeneous value */
        for (int k = 0; k < N; ++k)
            for (int j = 0; j < N; ++j)
                for (int i = 0; i < N; ++i) {
                    const int64_t n = ((int64_t)k * N + j) * N + i;
                    vacuum_mode(m, seed, member, f, kcut, amp2, a, H, m2eff, i, j, k,
                                &re[n], &im[n], &pre[n], &pim[n]);
                }
        orc_dft3(N, +1, re, im);
        orc_dft3(N, +1, pre, pim);
        const double pbar = pow(a, 3.0 - m->alpha) * dfbar[f];
        for (int64_t n = 0; n < V; ++n) {
            phi[(int64_t)f * V + n] = fbar[f] + re[n];
            pi[(int64_t)f * V + n] = pbar + pre[n];
        }
    }
    free(re); free(im); free(pre); free(pim);

    abt[0] = a;
    abt[1] = 0.0;
    abt[2] = 0.0;
    if (m->expansion) {
        double e[ORC_NE];
        orc_energies(m, phi, pi, NULL, NULL, abt, e);
        abt[1] = a * sqrt(pow(a, 2.0 * m->alpha) * m->kappa * e[ORC_E_RHO] / 3.0);
    }
}

/* --------------------------------------------------------------- spectrum */

/* Binned spectrum of a real lattice field.  Bin l collects the modes with
 * l = floor(|n~|/dn + 1/2), i.e. |n~| in [l dn - dn/2, l dn + dn/2).  For bin
 * l > 0, with n_l = l dn, k_l = k_IR n_l and S_l = sum of |f(n~)|^2 over the bin:
 *   Type I : Delta = n_l S_l / (N^6 dn)                (exact multiplicity #_l)
 *   Type II: Delta = 4 pi n_l^3 <|f|^2>_l / N^6         (# replaced by 4 pi n_l^2 dn)
 * which is Eq. discretePST2 with Upsilon of Eq. UpsilonII generalised to width dn.
 * Returns the number of bins written (bin 0 holds the zero mode, Delta = 0). */
int orc_spectrum(int N, double L, const double* f, double dn, int type,
                 double* k_out, double* delta_out, double* count_out, int cap)
{
    const int64_t V = (int64_t)N * N * N;
    double* re = malloc(sizeof(double) * (size_t)V);
    double* im = calloc((size_t)V, sizeof(double));
    memcpy(re, f, sizeof(double) * (size_t)V);
    orc_dft3(N, -1, re, im);
    const double nmax = sqrt(3.0) * (N / 2);
    int nb = (int)floor(nmax / dn + 0.5) + 1;
    if (nb > cap) nb = cap;
    double* S = calloc((size_t)nb, sizeof(double));
    double* C = calloc((size_t)nb, sizeof(double));
    for (int k = 0; k < N; ++k)
        for (int j = 0; j < N; ++j)
            for (int i = 0; i < N; ++i) {
                const int si = signed_mode(i, N), sj = signed_mode(j, N), sk = signed_mode(k, N);
                const double nm = sqrt((double)si * si + (double)sj * sj + (double)sk * sk);
                const int l = (int)floor(nm / dn + 0.5);
                if (l >= nb) continue;
                const int64_t n = ((int64_t)k * N + j) * N + i;
                S[l] += re[n] * re[n] + im[n] * im[n];
                C[l] += 1.0;
            }
    const double kIR = 6.283185307179586476925286766559 / L;
    const double N6 = (double)V * (double)V;
    for (int l = 0; l < nb; ++l) {
        const double nl = l * dn;
        k_out[l] = kIR * nl;
        count_out[l] = C[l];
        if (l == 0 || C[l] == 0.0) { delta_out[l] = 0.0; continue; }
        if (type == 1) delta_out[l] = nl * S[l] / (N6 * dn);
        else delta_out[l] = 4.0 * 3.14159265358979323846264338327950 * nl * nl * nl * (S[l] / C[l]) / N6;
    }
    free(re); free(im); free(S); free(C);
    return nb;
}
