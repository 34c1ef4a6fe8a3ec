/*
 * FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Axion coupled to compact U(1) links (section "ALP-gauge interactions",
 * Eq. AxionInfEOM: phi'' gains +(alpha_L/(a^3 m_p)) E.B, E' gains
 * -(alpha_L/(a m_p)) (phi' B - grad phi x E); the Gauss law becomes
 * div E = -(alpha_L/(a m_p)) grad phi . B), recast in alpha-time and solved with the
 * low-storage Runge-Kutta schemes, as that section prescribes.
 *
 * The paper gives only continuum equations; the lattice equations here are the
 * Euler-Lagrange equations of the lattice Lagrangian (program units, one site):
 *   L = 1/2 a^(3-alpha) phi'^2 - 1/2 a^(1+alpha) sum_i (grad+_i phi)^2 - a^(3+alpha) V(phi)
 *     + ws2 [ 1/2 a^(1-alpha) sum_i E_i^2 - a^(alpha-1) sum_{i<j} (1 - cos theta_ij)/dx^4
 *             + g phi Ebar . Bbar ]
 * with link angles theta_i(n) = dx A_i on n -> n+i, E_i = A_i' on the same link,
 * plaquettes theta_ij(n) = theta_i(n) + theta_j(n+i) - theta_i(n+j) - theta_j(n),
 * Ebar_i(n) = (E_i(n) + E_i(n-i))/2 (two-link average), Bbar_i(n) the average of
 * sin theta_jk/dx^2 over the four plaquettes of the (j,k) plane around n ((i,j,k)
 * cyclic, the "clover"), g = alpha_L sqrt(kappa) (kappa = (f_star/m_p)^2) and
 * ws2 = (omega_star/f_star)^2.  Its equations of motion:
 *   pi'  = a^(1+alpha) Lap phi - a^(3+alpha) V' + ws2 g Ebar.Bbar
 *   d/deta [a^(1-alpha) E_i + g W_i] = -a^(alpha-1) Mag_i + g C_i
 *     W_i(n)   = (phi(n) Bbar_i(n) + phi(n+i) Bbar_i(n+i))/2
 *     Mag_i    = dx d/dtheta_i sum (1 - cos theta_P)/dx^4
 *     C_i      = dx d/dtheta_i sum_m phi(m) Ebar(m).Bbar(m)
 * Gauge invariance makes G(n) = div- [a^(1-alpha) E + g W] a conserved charge of the
 * continuous-time flow (the lattice Gauss law), and the Chern-Simons term drops out
 * of the energy.  All derivatives below are taken literally: every plaquette's
 * derivative is scattered onto its four links.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static int64_t shift(int N, int64_t n, int d, int s)
{
    int c[3];
    c[0] = (int)(n % N);
    c[1] = (int)((n / N) % N);
    c[2] = (int)(n / ((int64_t)N * N));
    c[d] = ((c[d] + s) % N + N) % N;
    return ((int64_t)c[2] * N + c[1]) * N + c[0];
}

/* signed Fourier index: 0..N/2 and -(N/2-1)..-1 */
static int signed_mode_u1(int i, int N) { return (i <= N / 2) ? i : i - N; }

/* theta_ij(n) = theta_i(n) + theta_j(n+i) - theta_i(n+j) - theta_j(n) */
static double plaq(int N, const double* th, int64_t n, int i, int j)
{
    const int64_t V = (int64_t)N * N * N;
    return th[i * V + n] + th[j * V + shift(N, n, i, 1)] - th[i * V + shift(N, n, j, 1)] - th[j * V + n];
}

/* Link rate of a plaquette: d theta_ij(n)/d eta = dx (E_i(n) + E_j(n+i) - E_i(n+j) - E_j(n)) */
static double plaq_rate(int N, double dx, const double* E, int64_t n, int i, int j)
{
    const int64_t V = (int64_t)N * N * N;
    return dx * (E[i * V + n] + E[j * V + shift(N, n, i, 1)] - E[i * V + shift(N, n, j, 1)] - E[j * V + n]);
}

/* Add c * d theta_ij(q)/d theta_l to every link l of the plaquette (i, j) at q. */
static void scatter_plaq(int N, double* F, int64_t q, int i, int j, double c)
{
    const int64_t V = (int64_t)N * N * N;
    F[i * V + q] += c;
    F[j * V + shift(N, q, i, 1)] += c;
    F[i * V + shift(N, q, j, 1)] -= c;
    F[j * V + q] -= c;
}

double orc_u1_magnetic_sum(int N, const double* th)
{
    const int64_t V = (int64_t)N * N * N;
    double s = 0.0;
    /* 1 - cos p written as 2 sin^2(p/2): the same function, without the cancellation
     * that loses every digit when the plaquettes are small (gauge fields grown from zero) */
    for (int64_t n = 0; n < V; ++n)
        for (int i = 0; i < 3; ++i)
            for (int j = i + 1; j < 3; ++j) {
                const double h = sin(0.5 * plaq(N, th, n, i, j));
                s += 2.0 * h * h;
            }
    return s;
}

/* Clover-averaged Bbar_k(m) and its rate, and the two-link Ebar_k(m). */
static void clover_fields(int N, double dx, const double* th, const double* E, double* Bbar, double* Bdot,
                          double* Ebar)
{
    const int64_t V = (int64_t)N * N * N;
    for (int64_t m = 0; m < V; ++m)
        for (int k = 0; k < 3; ++k) {
            const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
            const int64_t q[4] = {m, shift(N, m, k1, -1), shift(N, m, k2, -1), shift(N, shift(N, m, k1, -1), k2, -1)};
            double b = 0.0, bd = 0.0;
            for (int c = 0; c < 4; ++c) {
                const double p = plaq(N, th, q[c], k1, k2);
                b += sin(p);
                if (Bdot) bd += cos(p) * plaq_rate(N, dx, E, q[c], k1, k2);
            }
            Bbar[k * V + m] = b / (4.0 * dx * dx);
            if (Bdot) Bdot[k * V + m] = bd / (4.0 * dx * dx);
            Ebar[k * V + m] = 0.5 * (E[k * V + m] + E[k * V + shift(N, m, k, -1)]);
        }
}

/* Right-hand side of the coupled system at fixed (a, a'). */
static void u1_rhs(const orc_model* m, const double* phi, const double* pi, const double* th, const double* E,
                   double a, double b, double* dphi, double* dpi, double* dth, double* dE)
{
    const int N = m->N;
    const int64_t V = (int64_t)N * N * N;
    const double dx = m->L / N, al = m->alpha;
    const double g = m->alphaL * sqrt(m->kappa);
    double* Bbar = malloc(sizeof(double) * 3 * V);
    double* Bdot = malloc(sizeof(double) * 3 * V);
    double* Ebar = malloc(sizeof(double) * 3 * V);
    double* Mag = calloc((size_t)(3 * V), sizeof(double));
    double* Ccs = calloc((size_t)(3 * V), sizeof(double));
    clover_fields(N, dx, th, E, Bbar, Bdot, Ebar);

    /* scalar: phi' = a^(alpha-3) pi;  pi' = a^(1+alpha) Lap phi - a^(3+alpha) V' + ws2 g Ebar.Bbar */
    orc_kick_force(m, 0, phi, a, dpi);
    for (int64_t n = 0; n < V; ++n) {
        dphi[n] = pow(a, al - 3.0) * pi[n];
        double eb = 0.0;
        for (int k = 0; k < 3; ++k) eb += Ebar[k * V + n] * Bbar[k * V + n];
        dpi[n] += m->ws2 * g * eb;
    }
    /* links: theta_i' = dx E_i */
    for (int64_t l = 0; l < 3 * V; ++l) dth[l] = dx * E[l];

    /* magnetic force: Mag_l = sum_P sin theta_P d theta_P/d theta_l / dx^3 */
    for (int64_t q = 0; q < V; ++q)
        for (int i = 0; i < 3; ++i)
            for (int j = i + 1; j < 3; ++j) scatter_plaq(N, Mag, q, i, j, sin(plaq(N, th, q, i, j)) / (dx * dx * dx));

    /* Chern-Simons force: C_l = dx d/d theta_l sum_m phi(m) sum_k Ebar_k(m) Bbar_k(m) */
    for (int64_t mm = 0; mm < V; ++mm)
        for (int k = 0; k < 3; ++k) {
            const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
            const double coef = dx * phi[mm] * Ebar[k * V + mm] / (4.0 * dx * dx);
            const int64_t q[4] = {mm, shift(N, mm, k1, -1), shift(N, mm, k2, -1),
                                  shift(N, shift(N, mm, k1, -1), k2, -1)};
            for (int c = 0; c < 4; ++c) scatter_plaq(N, Ccs, q[c], k1, k2, coef * cos(plaq(N, th, q[c], k1, k2)));
        }

    /* E_i' = a^(alpha-1) [ -a^(alpha-1) Mag_i + g (C_i - W_i') ] - (1 - alpha) (a'/a) E_i */
    for (int i = 0; i < 3; ++i)
        for (int64_t n = 0; n < V; ++n) {
            const int64_t np = shift(N, n, i, 1);
            const double Wdot = 0.5 * (dphi[n] * Bbar[i * V + n] + phi[n] * Bdot[i * V + n] +
                                       dphi[np] * Bbar[i * V + np] + phi[np] * Bdot[i * V + np]);
            const int64_t l = i * V + n;
            dE[l] = pow(a, al - 1.0) * (-pow(a, al - 1.0) * Mag[l] + g * (Ccs[l] - Wdot)) - (1.0 - al) * (b / a) * E[l];
        }
    free(Bbar); free(Bdot); free(Ebar); free(Mag); free(Ccs);
}

void orc_u1_rhs(const orc_model* m, const double* phi, const double* pi, const double* links, const double* efield,
                const double* abt, double* dphi, double* dpi, double* dlinks, double* defield)
{
    /* without expansion a is frozen, so its rate a' is zero */
    u1_rhs(m, phi, pi, links, efield, abt[0], m->expansion ? abt[1] : 0.0, dphi, dpi, dlinks, defield);
}

/* Lattice Gauss charge G(n) = sum_i [(a^(1-alpha) E_i + g W_i)(n) - (same)(n - i)] / dx. */
void orc_u1_gauss(const orc_model* m, const double* phi, const double* links, const double* efield, double a,
                  double* out)
{
    const int N = m->N;
    const int64_t V = (int64_t)N * N * N;
    const double dx = m->L / N;
    const double g = m->alphaL * sqrt(m->kappa);
    double* Bbar = malloc(sizeof(double) * 3 * V);
    double* Ebar = malloc(sizeof(double) * 3 * V);
    double* P = malloc(sizeof(double) * 3 * V);
    clover_fields(N, dx, links, efield, Bbar, NULL, Ebar);
    for (int i = 0; i < 3; ++i)
        for (int64_t n = 0; n < V; ++n) {
            const int64_t np = shift(N, n, i, 1);
            const double W = 0.5 * (phi[n] * Bbar[i * V + n] + phi[np] * Bbar[i * V + np]);
            P[i * V + n] = pow(a, 1.0 - m->alpha) * efield[i * V + n] + g * W;
        }
    for (int64_t n = 0; n < V; ++n) {
        double s = 0.0;
        for (int i = 0; i < 3; ++i) s += P[i * V + n] - P[i * V + shift(N, n, i, -1)];
        out[n] = s / dx;
    }
    free(Bbar); free(Ebar); free(P);
}

/* One 2N Runge-Kutta step of y = (phi, pi, theta, E, a, a'). */
int orc_rk_coeffs(int scheme, const double** A, const double** B);

void orc_u1_rk_step(const orc_model* m, int scheme, double h, double* phi, double* pi, double* links,
                    double* efield, double* abt)
{
    const int N = m->N;
    const int64_t V = (int64_t)N * N * N;
    const double *A, *B;
    const int S = orc_rk_coeffs(scheme, &A, &B);
    const int64_t nd = 8 * V;  /* phi, pi, 3 links, 3 electric */
    double* k = calloc((size_t)nd, sizeof(double));
    double* F = malloc(sizeof(double) * (size_t)nd);
    double ka = 0.0, kb = 0.0;
    for (int s = 0; s < S; ++s) {
        const double a = abt[0], b = m->expansion ? abt[1] : 0.0;
        double Fa = 0.0, Fb = 0.0;
        if (m->expansion) {
            double e[ORC_NE];
            orc_energies(m, phi, pi, links, efield, abt, e);
            Fa = b;
            Fb = orc_addot(m, a, e[ORC_E_RHO], e[ORC_E_P]);
        }
        u1_rhs(m, phi, pi, links, efield, a, b, F, F + V, F + 2 * V, F + 5 * V);
        double* y[4] = {phi, pi, links, efield};
        const int64_t off[4] = {0, V, 2 * V, 5 * V};
        const int64_t len[4] = {V, V, 3 * V, 3 * V};
        for (int p = 0; p < 4; ++p)
            for (int64_t n = 0; n < len[p]; ++n) {
                k[off[p] + n] = A[s] * k[off[p] + n] + h * F[off[p] + n];
                y[p][n] += B[s] * k[off[p] + n];
            }
        ka = A[s] * ka + h * Fa;
        kb = A[s] * kb + h * Fb;
        abt[0] += B[s] * ka;
        abt[1] += B[s] * kb;
    }
    abt[2] += h;
    free(k);
    free(F);
}

/* ------------------------------------------------------------------ leapfrog */

/* Momentum part of the right-hand side, f(q, a, b, p) = (pi', E'), at positions q = (phi, theta)
 * and momenta p = (pi, E) stored as P[0..V) = pi, P[V..4V) = E_0..2. */
static void u1_momentum_force(const orc_model* m, const double* phi, const double* th, const double* P, double a,
                              double b, double* Fp, double* sphi, double* sth)
{
    const int64_t V = (int64_t)m->N * m->N * m->N;
    u1_rhs(m, phi, P, th, P + V, a, b, sphi, Fp, sth, Fp + V);
}

/* Leapfrog of the axion-U(1) system (section "ALP-gauge interactions": its equations are not
 * canonical in (pi, E), since the E' of Eq. AxionInfEOM depends on phi' and the pi' on E, so
 * a kick at fixed positions is not explicit).  Positions q = (phi, theta, a) and momenta
 * p = (pi, E, a') are staggered as in the generalized Stoermer-Verlet method (Hairer, Lubich
 * and Wanner, Geometric Numerical Integration, section VI.3, its Eq. (3.4) with the momentum
 * force f affine in p), ordered like the scalar velocity-Verlet step of lattice.c:
 *   a'_{1/2} = a'_0 + h/2 a''(a_0, rho_0, p_0)                        (energies of q_0, p_0)
 *   p_{1/2}  = p_0 + h/2 f(q_0, a_0, a'_{1/2}, p_{1/2})                (implicit)
 *   a_1 = a_0 + h a'_{1/2};  phi_1 = phi_0 + h ((a_0+a_1)/2)^(alpha-3) pi_{1/2};
 *   theta_1 = theta_0 + h dx E_{1/2}
 *   p_1      = p_{1/2} + h/2 f(q_1, a_1, a'_{1/2}, p_{1/2})             (explicit)
 *   a'_1     = a'_{1/2} + h/2 a''(a_1, rho_1, p_1).
 * The implicit half-kick is solved by fixed-point iteration, `iters` evaluations of f:
 *   p^(1) = p_0 + h/2 G,   p^(k+1) = p_0 + h/2 f(q_0, a_0, a'_{1/2}, p^(k)),   p_{1/2} = p^(iters),
 * where G is the force of the previous step's closing half-kick (so that p^(1) is the
 * previous half-step momentum advanced by a full kick with the force at q_0), and, in the
 * first step of a call, f(q_0, a_0, a'_0, p_0).  Because f is affine in p, the merged kick
 * of two consecutive half-kicks is p_{n+1/2} = p_{n-1/2} + h f(q_n, (p_{n-1/2} + p_{n+1/2})/2)
 * when iterated to convergence, which is the leapfrog with the coupling at the average of
 * the old and new momenta. */
void orc_u1_leapfrog(const orc_model* m, double h, int nsteps, int iters, double* phi, double* pi, double* links,
                     double* efield, double* abt)
{
    const int N = m->N;
    const int64_t V = (int64_t)N * N * N;
    const double dx = m->L / N, al = m->alpha;
    double* P0 = malloc(sizeof(double) * (size_t)(4 * V));  /* p_n: pi, E_0..2 */
    double* Pk = malloc(sizeof(double) * (size_t)(4 * V));  /* iterate */
    double* G = malloc(sizeof(double) * (size_t)(4 * V));   /* force of the last kick */
    double* F = malloc(sizeof(double) * (size_t)(4 * V));
    double* sphi = malloc(sizeof(double) * (size_t)V);      /* unused rates */
    double* sth = malloc(sizeof(double) * (size_t)(3 * V));
    memcpy(P0, pi, sizeof(double) * (size_t)V);
    memcpy(P0 + V, efield, sizeof(double) * (size_t)(3 * V));
    double a = abt[0], b = m->expansion ? abt[1] : 0.0;
    if (iters < 1) iters = 1;
    u1_momentum_force(m, phi, links, P0, a, b, G, sphi, sth);
    for (int s = 0; s < nsteps; ++s) {
        double e[ORC_NE];
        double bh = b;
        if (m->expansion) {
            const double abt_n[3] = {a, b, abt[2]};
            orc_energies(m, phi, P0, links, P0 + V, abt_n, e);
            bh = b + 0.5 * h * orc_addot(m, a, e[ORC_E_RHO], e[ORC_E_P]);
        }
        for (int64_t l = 0; l < 4 * V; ++l) Pk[l] = P0[l] + 0.5 * h * G[l];
        for (int k = 1; k < iters; ++k) {
            u1_momentum_force(m, phi, links, Pk, a, bh, F, sphi, sth);
            for (int64_t l = 0; l < 4 * V; ++l) Pk[l] = P0[l] + 0.5 * h * F[l];
        }
        const double a1 = m->expansion ? a + h * bh : a;
        const double cd = h * pow(0.5 * (a + a1), al - 3.0);
        for (int64_t n = 0; n < V; ++n) phi[n] += cd * Pk[n];
        for (int64_t l = 0; l < 3 * V; ++l) links[l] += h * dx * Pk[V + l];
        a = a1;
        u1_momentum_force(m, phi, links, Pk, a, bh, G, sphi, sth);
        for (int64_t l = 0; l < 4 * V; ++l) P0[l] = Pk[l] + 0.5 * h * G[l];
        b = bh;
        if (m->expansion) {
            const double abt_n[3] = {a, bh, abt[2]};
            orc_energies(m, phi, P0, links, P0 + V, abt_n, e);
            b = bh + 0.5 * h * orc_addot(m, a, e[ORC_E_RHO], e[ORC_E_P]);
        }
        abt[2] += h;
    }
    memcpy(pi, P0, sizeof(double) * (size_t)V);
    memcpy(efield, P0 + V, sizeof(double) * (size_t)(3 * V));
    abt[0] = a;
    if (m->expansion) abt[1] = b;
    free(P0); free(Pk); free(G); free(F); free(sphi); free(sth);
}

/* --------------------------------------------------------------- gauge spectra */

/* Binned spectra of the U(1) sector (section "ALP-gauge interactions": the spectra of the
 * two chiralities of the gauge field; reading, since the paper gives no definition):
 *   which 0: electric field, sum over i of |E_i(k)|^2;
 *   which 1: magnetic field B_k(n) = sin theta_{k1 k2}(n) / dx^2 (plaquette of normal k,
 *            k1 = k+1, k2 = k+2 mod 3), sum over k of |B_k(k)|^2;
 *   which 2, 3: the + and - chiralities of the gauge potential A_i = theta_i / dx.  A link
 *            field lives at n + e_i/2, so its Fourier amplitude carries the phase
 *            exp(-i k_i dx / 2): A^_i = exp(-i k_i dx/2) DFT(A_i).  The forward-difference
 *            curl is then i kt x A^ with the real lattice momentum kt_l = (2/dx) sin(k_l dx/2).
 *            With kh = kt/|kt| and u, v = kh x u orthonormal and transverse to kt, the
 *            vectors e_s = (u + s i v)/sqrt(2) satisfy i kh x e_s = s e_s (s = +1, -1), and
 *            A_s = conj(e_s) . A^ is the amplitude of chirality s (|A_s|^2 does not depend
 *            on the choice of u).  The zero mode has none.
 * Every mode of the full spectrum is visited; binning and normalisation as orc_spectrum. */
int orc_gauge_spectrum(const orc_model* m, const double* links, const double* efield, int which, double dn,
                       int type, double* k_out, double* delta_out, double* count_out, int cap)
{
    const int N = m->N;
    const int64_t V = (int64_t)N * N * N;
    const double dx = m->L / N;
    const double pi_ = 3.14159265358979323846264338327950;
    double* re[3];
    double* im[3];
    for (int c = 0; c < 3; ++c) {
        re[c] = malloc(sizeof(double) * (size_t)V);
        im[c] = calloc((size_t)V, sizeof(double));
        for (int64_t n = 0; n < V; ++n) {
            if (which == 0) re[c][n] = efield[c * V + n];
            else if (which == 1) re[c][n] = sin(plaq(N, links, n, (c + 1) % 3, (c + 2) % 3)) / (dx * dx);
            else re[c][n] = links[c * V + n] / dx;
        }
        orc_dft3(N, -1, re[c], im[c]);
    }
    const double nmax = sqrt(3.0) * (N / 2);
    int nb = (int)floor(nmax / dn + 0.5) + 1;
    if (nb > cap) nb = cap;
    double* S = calloc((size_t)nb, sizeof(double));
    double* C = calloc((size_t)nb, sizeof(double));
    const double s_hel = which == 2 ? 1.0 : -1.0;
    for (int k = 0; k < N; ++k)
        for (int j = 0; j < N; ++j)
            for (int i = 0; i < N; ++i) {
                const int s[3] = {signed_mode_u1(i, N), signed_mode_u1(j, N), signed_mode_u1(k, N)};
                const double nm = sqrt((double)s[0] * s[0] + (double)s[1] * s[1] + (double)s[2] * s[2]);
                const int l = (int)floor(nm / dn + 0.5);
                if (l >= nb) continue;
                const int64_t n = ((int64_t)k * N + j) * N + i;
                double p = 0.0;
                if (which < 2) {
                    for (int c = 0; c < 3; ++c) p += re[c][n] * re[c][n] + im[c][n] * im[c][n];
                } else {
                    double kt[3], ar[3], ai[3], nk = 0.0;
                    for (int c = 0; c < 3; ++c) {
                        const double half = pi_ * s[c] / N;  /* k_c dx / 2 */
                        kt[c] = 2.0 / dx * sin(half);
                        nk += kt[c] * kt[c];
                        /* A^_c = exp(-i half) (re + i im) */
                        ar[c] = cos(half) * re[c][n] + sin(half) * im[c][n];
                        ai[c] = cos(half) * im[c][n] - sin(half) * re[c][n];
                    }
                    nk = sqrt(nk);
                    if (nk > 0.0) {
                        double kh[3] = {kt[0] / nk, kt[1] / nk, kt[2] / nk};
                        int a = 0;  /* axis least aligned with kh */
                        for (int c = 1; c < 3; ++c)
                            if (fabs(kh[c]) < fabs(kh[a])) a = c;
                        double u[3] = {-kh[a] * kh[0], -kh[a] * kh[1], -kh[a] * kh[2]};
                        u[a] += 1.0;
                        const double nu = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
                        for (int c = 0; c < 3; ++c) u[c] /= nu;
                        const double v[3] = {kh[1] * u[2] - kh[2] * u[1], kh[2] * u[0] - kh[0] * u[2],
                                             kh[0] * u[1] - kh[1] * u[0]};
                        /* A_s = sum_c conj(e_s,c) A^_c, conj(e_s,c) = (u_c - s i v_c) / sqrt(2) */
                        double xr = 0.0, xi = 0.0;
                        for (int c = 0; c < 3; ++c) {
                            xr += u[c] * ar[c] + s_hel * v[c] * ai[c];
                            xi += u[c] * ai[c] - s_hel * v[c] * ar[c];
                        }
                        p = 0.5 * (xr * xr + xi * xi);
                    }
                }
                S[l] += p;
                C[l] += 1.0;
            }
    const double kIR = 2.0 * pi_ / m->L;
    const double N6 = (double)V * (double)V;
    for (int l = 0; l < nb; ++l) {
        const double nl = l * dn;
        k_out[l] = kIR * nl;
        count_out[l] = C[l];
        if (l == 0 || C[l] == 0.0) { delta_out[l] = 0.0; continue; }
        if (type == 1) delta_out[l] = nl * S[l] / (N6 * dn);
        else delta_out[l] = 4.0 * pi_ * nl * nl * nl * (S[l] / C[l]) / N6;
    }
    for (int c = 0; c < 3; ++c) { free(re[c]); free(im[c]); }
    free(S); free(C);
    return nb;
}
