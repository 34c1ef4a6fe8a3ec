/*
 * FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Gravitational waves with five traceless auxiliary fields (section "New algorithm for
 * GWs").  The paper evolves v_ij with v_33 = -v_11 - v_22,
 *   v'' + (3 - alpha)(a'/a) v' - a^(-2(1-alpha)) Lap v = 2 / (m_p^2 a^(2(1-alpha))) [Pi_ij - delta_ij Pi / 3],
 * and obtains h_ij(k) = Lambda_ij,lm(k^) v_lm(k) with the TT projector
 * Lambda_ij,lm = P_il P_jm - P_ij P_lm / 2, P_ij = delta_ij - k^_i k^_j.
 * In program variables (pi_v = a^(3-alpha) v', kappa = (f_star/m_p)^2):
 *   v' = a^(alpha-3) pi_v,   pi_v' = a^(1+alpha) Lap v + 2 kappa a^(1+alpha) [Pi_ij - delta_ij Pi / 3].
 * Readings (the discretisation is in the paper's companion review): the scalar source
 * Pi_ij = sum_f dbar_i phi_f dbar_j phi_f with the central difference
 * dbar_i phi = (phi(n+i) - phi(n-i)) / (2 dx); the projector built from the matching lattice
 * momentum kbar_i = sin(k_i dx) / dx; the energy density rho_GW = <h'_ij h'_ij> / (4 kappa a^(2 alpha))
 * (the m_p^2 of the continuum formula is 1/kappa in program units), binned per log k as the
 * scalar spectra: Type I n_l S_l / (N^6 dn), Type II 4 pi n_l^3 <|.|^2>_l / N^6, times
 * 1 / (4 kappa a^(2 alpha)), with S_l the sum over the bin of sum_ij |(Lambda H)_ij|^2 and
 * H = DFT of h' (unnormalised).  Every loop follows the formulas as written.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>

/* component index of (a, b), a <= b, in {11, 12, 13, 22, 23}; 33 is -11 - 22 */
static const int GW_A[5] = {0, 0, 0, 1, 1};
static const int GW_B[5] = {0, 1, 2, 1, 2};

static int64_t gw_site(int N, int x, int y, int z)
{
    x = ((x % N) + N) % N;
    y = ((y % N) + N) % N;
    z = ((z % N) + N) % N;
    return ((int64_t)z * N + y) * N + x;
}

void orc_gw_force(const orc_model* m, const double* phi, const double* gv, double a, double* out)
{
    const int N = m->N;
    const int64_t V = (int64_t)N * N * N;
    const double dx = m->L / N;
    const double cl = pow(a, 1.0 + m->alpha);
    double* lap = malloc(sizeof(double) * (size_t)V);
    for (int c = 0; c < 5; ++c) {
        orc_laplacian(N, dx, gv + (int64_t)c * V, lap);
        for (int64_t n = 0; n < V; ++n) out[(int64_t)c * V + n] = cl * lap[n];
    }
    free(lap);
    for (int z = 0; z < N; ++z)
        for (int y = 0; y < N; ++y)
            for (int x = 0; x < N; ++x) {
                const int64_t n = gw_site(N, x, y, z);
                double Pi[3][3] = {{0}};
                for (int f = 0; f < m->nf; ++f) {
                    const double* p = phi + (int64_t)f * V;
                    const double d[3] = {(p[gw_site(N, x + 1, y, z)] - p[gw_site(N, x - 1, y, z)]) / (2.0 * dx),
                                         (p[gw_site(N, x, y + 1, z)] - p[gw_site(N, x, y - 1, z)]) / (2.0 * dx),
                                         (p[gw_site(N, x, y, z + 1)] - p[gw_site(N, x, y, z - 1)]) / (2.0 * dx)};
                    for (int i = 0; i < 3; ++i)
                        for (int j = 0; j < 3; ++j) Pi[i][j] += d[i] * d[j];
                }
                const double tr = Pi[0][0] + Pi[1][1] + Pi[2][2];
                for (int c = 0; c < 5; ++c) {
                    const int i = GW_A[c], j = GW_B[c];
                    const double S = Pi[i][j] - (i == j ? tr / 3.0 : 0.0);
                    out[(int64_t)c * V + n] += 2.0 * m->kappa * cl * S;
                }
            }
}

static int gw_signed(int i, int N) { return (i <= N / 2) ? i : i - N; }

int orc_gw_spectrum(const orc_model* m, const double* gp, const double* abt, double dn, int type, double* k_out,
                    double* delta_out, double* count_out, int cap)
{
    const int N = m->N;
    const int64_t V = (int64_t)N * N * N;
    const double dx = m->L / N;
    const double a = abt[0];
    const double pi_ = 3.14159265358979323846264338327950;
    const double ca = pow(a, m->alpha - 3.0);  /* h' = a^(alpha-3) pi_v */
    /* the six components h'_ij (symmetric), DFT of each */
    double* re[3][3];
    double* im[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = i; j < 3; ++j) {
            re[i][j] = malloc(sizeof(double) * (size_t)V);
            im[i][j] = calloc((size_t)V, sizeof(double));
            for (int64_t n = 0; n < V; ++n) {
                double v;
                if (i == 2 && j == 2) v = -gp[0 * V + n] - gp[3 * V + n];  /* h'_33 = -h'_11 - h'_22 */
                else {
                    int c = 0;
                    while (!(GW_A[c] == i && GW_B[c] == j)) ++c;
                    v = gp[(int64_t)c * V + n];
                }
                re[i][j][n] = ca * v;
            }
            orc_dft3(N, -1, re[i][j], im[i][j]);
            re[j][i] = re[i][j];
            im[j][i] = im[i][j];
        }
    const double nmax = sqrt(3.0) * (N / 2);
    int nb = (int)floor(nmax / dn + 0.5) + 1;
    if (nb > cap) nb = cap;
    double* S = calloc((size_t)nb, sizeof(double));
    double* C = calloc((size_t)nb, sizeof(double));
    for (int kz = 0; kz < N; ++kz)
        for (int ky = 0; ky < N; ++ky)
            for (int kx = 0; kx < N; ++kx) {
                const int s[3] = {gw_signed(kx, N), gw_signed(ky, N), gw_signed(kz, N)};
                const double nm = sqrt((double)s[0] * s[0] + (double)s[1] * s[1] + (double)s[2] * s[2]);
                const int l = (int)floor(nm / dn + 0.5);
                if (l >= nb) continue;
                C[l] += 1.0;
                double kb[3], k2 = 0.0;
                for (int c = 0; c < 3; ++c) {
                    kb[c] = sin(2.0 * pi_ * s[c] / N) / dx;
                    k2 += kb[c] * kb[c];
                }
                if (k2 <= 0.0) continue;  /* no direction: no TT part */
                double P[3][3];
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) P[i][j] = (i == j ? 1.0 : 0.0) - kb[i] * kb[j] / k2;
                const int64_t n = ((int64_t)kz * N + ky) * N + kx;
                double p = 0.0;
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) {
                        double tr = 0.0, ti = 0.0;  /* (Lambda H)_ij */
                        for (int l2 = 0; l2 < 3; ++l2)
                            for (int mm = 0; mm < 3; ++mm) {
                                const double L = P[i][l2] * P[j][mm] - 0.5 * P[i][j] * P[l2][mm];
                                tr += L * re[l2][mm][n];
                                ti += L * im[l2][mm][n];
                            }
                        p += tr * tr + ti * ti;
                    }
                S[l] += p;
            }
    const double kIR = 2.0 * pi_ / m->L;
    const double N6 = (double)V * (double)V;
    const double pref = 1.0 / (4.0 * m->kappa * pow(a, 2.0 * m->alpha));
    for (int l = 0; l < nb; ++l) {
        const double nl = l * dn;
        k_out[l] = kIR * nl;
        count_out[l] = C[l];
        if (l == 0 || C[l] == 0.0) { delta_out[l] = 0.0; continue; }
        if (type == 1) delta_out[l] = pref * nl * S[l] / (N6 * dn);
        else delta_out[l] = pref * 4.0 * pi_ * nl * nl * nl * (S[l] / C[l]) / N6;
    }
    for (int i = 0; i < 3; ++i)
        for (int j = i; j < 3; ++j) {
            free(re[i][j]);
            free(im[i][j]);
        }
    free(S);
    free(C);
    return nb;
}
