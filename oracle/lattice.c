/*
 * FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Scalar sector of the lattice time step: potential, 7-point Laplacian,
 * forward-difference gradient energy, the volume-averaged energies of
 * Eq. energy-contrib / Eq. rhoLocal, the Friedmann equations (Eq. Friedmann1,
 * Eq. Friedmann2) and the time integrators the paper lists in its section
 * "Non-symplectic evolvers": velocity Verlet (order 2), the order-4 Yoshida
 * composition of it, and the low-storage 2N Runge-Kutta schemes RK3-3 and RK4-5.
 * Everything is plain triple loops in double precision, in the order the
 * equations are written; no blocking, fusion or reordering.  Reduced (d+1)-dimensional
 * lattices (section "Scalar dynamics in 1+1 and 2+1 dimensions", model dims = 1 or 2) are
 * boxes of extent 1 along the missing directions, whose terms the operators leave out.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static int wrap(int i, int N) { return ((i % N) + N) % N; }

#ifdef _OPENMP
#include <omp.h>
int orc_threads(void) { return omp_get_max_threads(); }
#else
int orc_threads(void) { return 1; }
#endif

/* ------------------------------------------------------------------ potential */

double orc_V(const orc_model* m, double f0, double f1)
{
    double v = 0.5 * m->m2[0] * f0 * f0 + 0.25 * m->lam[0] * f0 * f0 * f0 * f0;
    if (m->nf > 1)
        v += 0.5 * m->m2[1] * f1 * f1 + 0.25 * m->lam[1] * f1 * f1 * f1 * f1 + 0.5 * m->g2 * f0 * f0 * f1 * f1;
    return v;
}

double orc_dV(const orc_model* m, int f, double f0, double f1)
{
    if (f == 0) {
        double d = m->m2[0] * f0 + m->lam[0] * f0 * f0 * f0;
        if (m->nf > 1) d += m->g2 * f0 * f1 * f1;
        return d;
    }
    return m->m2[1] * f1 + m->lam[1] * f1 * f1 * f1 + m->g2 * f0 * f0 * f1;
}

double orc_d2V(const orc_model* m, int f, double f0, double f1)
{
    if (f == 0) {
        double d = m->m2[0] + 3.0 * m->lam[0] * f0 * f0;
        if (m->nf > 1) d += m->g2 * f1 * f1;
        return d;
    }
    return m->m2[1] + 3.0 * m->lam[1] * f1 * f1 + m->g2 * f0 * f0;
}

/* ------------------------------------------------------------ lattice operators */

int64_t orc_volume(const orc_model* m)
{
    int nx, ny, nz;
    orc_extents(m, &nx, &ny, &nz);
    return (int64_t)nx * ny * nz;
}

void orc_extents(const orc_model* m, int* nx, int* ny, int* nz)
{
    const int d = (m->dims == 1 || m->dims == 2) ? m->dims : 3;
    *nx = m->N;
    *ny = d >= 2 ? m->N : 1;
    *nz = d >= 3 ? m->N : 1;
}

/* index of (x, y, z) in a box of extents nx, ny (x fastest) */
static int64_t IB(int nx, int ny, int x, int y, int z) { return ((int64_t)z * ny + y) * nx + x; }

/* 7-point Laplacian over the directions of extent > 1 of an nx x ny x nz box */
static void laplacian_box(int nx, int ny, int nz, double dx, const double* f, double* out)
{
    ORC_PAR_FOR
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const double c = f[IB(nx, ny, x, y, z)];
                double s = f[IB(nx, ny, wrap(x + 1, nx), y, z)] + f[IB(nx, ny, wrap(x - 1, nx), y, z)] - 2.0 * c;
                if (ny > 1) s += f[IB(nx, ny, x, wrap(y + 1, ny), z)] + f[IB(nx, ny, x, wrap(y - 1, ny), z)] - 2.0 * c;
                if (nz > 1) s += f[IB(nx, ny, x, y, wrap(z + 1, nz))] + f[IB(nx, ny, x, y, wrap(z - 1, nz))] - 2.0 * c;
                out[IB(nx, ny, x, y, z)] = s / (dx * dx);
            }
}

/* sum_n sum_i [f(n+i) - f(n)]^2 over the directions of extent > 1  (no 1/dx^2) */
static double grad2_box(int nx, int ny, int nz, const double* f)
{
    double s = 0.0;
    ORC_PAR_SUM(s)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const double c = f[IB(nx, ny, x, y, z)];
                const double gx = f[IB(nx, ny, wrap(x + 1, nx), y, z)] - c;
                s += gx * gx;
                if (ny > 1) {
                    const double gy = f[IB(nx, ny, x, wrap(y + 1, ny), z)] - c;
                    s += gy * gy;
                }
                if (nz > 1) {
                    const double gz = f[IB(nx, ny, x, y, wrap(z + 1, nz))] - c;
                    s += gz * gz;
                }
            }
    return s;
}

void orc_laplacian(int N, double dx, const double* f, double* out) { laplacian_box(N, N, N, dx, f, out); }

/* sum_n sum_i [f(n+i) - f(n)]^2  (no 1/dx^2) */
double orc_grad2_sum(int N, const double* f) { return grad2_box(N, N, N, f); }

/* Kick of Eq. singletEOM with pi = a^(3-alpha) phi':
 *   pi' = a^(1+alpha) Lap phi - a^(3+alpha) dV/dphi_f                     */
void orc_kick_force(const orc_model* m, int f, const double* phi, double a, double* out)
{
    const int N = m->N;
    const int64_t V = orc_volume(m);
    const double dx = m->L / N;
    const double* pf = phi + (int64_t)f * V;
    const double* p0 = phi;
    const double* p1 = (m->nf > 1) ? phi + V : NULL;
    int nx, ny, nz;
    orc_extents(m, &nx, &ny, &nz);
    laplacian_box(nx, ny, nz, dx, pf, out);
    const double ca = pow(a, 1.0 + m->alpha), cv = pow(a, 3.0 + m->alpha);
    ORC_PAR_FOR
    for (int64_t n = 0; n < V; ++n)
        out[n] = ca * out[n] - cv * orc_dV(m, f, p0[n], p1 ? p1[n] : 0.0);
}

/* ----------------------------------------------------- energies and Friedmann */

/* Eq. Friedmann1 in program units: a'' = a^(2 alpha + 1) kappa/6 [(2 alpha - 1) rho - 3 p]. */
double orc_addot(const orc_model* m, double a, double rho, double p)
{
    return pow(a, 2.0 * m->alpha + 1.0) * (m->kappa / 6.0) * ((2.0 * m->alpha - 1.0) * rho - 3.0 * p);
}

/* U(1) magnetic energy sum_n sum_{i<j} (1 - cos theta_ij)  (defined in u1.c) */
double orc_u1_magnetic_sum(int N, const double* links);

void orc_energies(const orc_model* m, const double* phi, const double* pi,
                  const double* links, const double* efield, const double* abt, double* out)
{
    const int N = m->N;
    const int64_t V = orc_volume(m);
    const double dx = m->L / N;
    const double a = abt[0], b = abt[1];
    int nx, ny, nz;
    orc_extents(m, &nx, &ny, &nz);
    memset(out, 0, sizeof(double) * ORC_NE);

    for (int f = 0; f < m->nf; ++f) {
        const double* pf = pi + (int64_t)f * V;
        double s = 0.0;
        ORC_PAR_SUM(s)
        for (int64_t n = 0; n < V; ++n) s += pf[n] * pf[n];
        /* K = phi'^2 / (2 a^(2 alpha)) with phi' = a^(alpha-3) pi  ->  pi^2 / (2 a^6) */
        out[ORC_E_K0 + f] = s / (2.0 * pow(a, 6.0) * (double)V);
        /* G = sum_i (grad+_i phi)^2 / (2 a^2) */
        out[ORC_E_G0 + f] = grad2_box(nx, ny, nz, phi + (int64_t)f * V) / (dx * dx) / (2.0 * a * a * (double)V);
    }
    {
        double s = 0.0;
        ORC_PAR_SUM(s)
        for (int64_t n = 0; n < V; ++n) s += orc_V(m, phi[n], m->nf > 1 ? phi[V + n] : 0.0);
        out[ORC_E_V] = s / (double)V;
    }
    if (m->gauge == 1 && links && efield) {
        /* K_U(1) = sum_i E_i^2 / (2 a^(2+2 alpha)),  G_U(1) = sum_{i<j} F_ij^2 / (2 a^4),
         * the lattice F_ij^2/2 being (1 - cos theta_ij)/dx^4; both carry (omega_star / f_star)^2
         * when expressed in the scalar's energy unit f_star^2 omega_star^2.                  */
        double se = 0.0;
        for (int64_t n = 0; n < 3 * V; ++n) se += efield[n] * efield[n];
        out[ORC_E_KEM] = m->ws2 * se / (2.0 * pow(a, 2.0 + 2.0 * m->alpha) * (double)V);
        out[ORC_E_GEM] = m->ws2 * orc_u1_magnetic_sum(N, links) / pow(dx, 4.0) / (pow(a, 4.0) * (double)V);
    }
    const double K = out[ORC_E_K0] + out[ORC_E_K1];
    const double G = out[ORC_E_G0] + out[ORC_E_G1];
    const double U = out[ORC_E_V];
    const double EM = out[ORC_E_KEM] + out[ORC_E_GEM];
    /* Eq. rhoLocal and the pressure below it */
    out[ORC_E_RHO] = K + G + U + EM;
    out[ORC_E_P] = K - G / 3.0 - U + EM / 3.0;
    /* Eq. Friedmann2 as a monitor: |H^2 - a^(2 alpha) kappa rho / 3| / H^2 */
    {
        const double H = b / a;
        const double rhs = pow(a, 2.0 * m->alpha) * m->kappa * out[ORC_E_RHO] / 3.0;
        out[ORC_E_HV] = (H != 0.0) ? fabs(H * H - rhs) / (H * H) : 0.0;
    }
    out[ORC_E_A] = a;
    out[ORC_E_B] = b;
}

/* ----------------------------------------------------------------- integrators */

/* U(1)+axion right-hand side and RK driver (defined in u1.c) */
void orc_u1_rk_step(const orc_model* m, int scheme, double h,
                    double* phi, double* pi, double* links, double* efield, double* abt);

/* One velocity-Verlet step (order 2) of fields and scale factor, ordered
 * symmetrically so that the map is time-reversible:
 *   a'  half-kick with rho(t), p(t);   pi half-kick with a(t);
 *   a   drift by h a';                 phi drift with ((a(t)+a(t+h))/2)^(alpha-3);
 *   pi  half-kick with a(t+h);         a' half-kick with rho(t+h), p(t+h).       */
static void vv_step(const orc_model* m, double h, double* phi, double* pi, double* abt, double* tmp, double* gv,
                    double* gp)
{
    const int64_t V = orc_volume(m);
    double e[ORC_NE];
    double a = abt[0], b = abt[1];
    double* gtmp = gv ? malloc(sizeof(double) * (size_t)(5 * V)) : NULL;

    if (m->expansion) {
        orc_energies(m, phi, pi, NULL, NULL, abt, e);
        b = b + 0.5 * h * orc_addot(m, a, e[ORC_E_RHO], e[ORC_E_P]);
    }
    for (int f = 0; f < m->nf; ++f) {
        orc_kick_force(m, f, phi, a, tmp + (int64_t)f * V);
    }
    if (gv) orc_gw_force(m, phi, gv, a, gtmp);  /* GW half-kick with the fields at t */
    for (int f = 0; f < m->nf; ++f) {
        ORC_PAR_FOR
        for (int64_t n = 0; n < V; ++n) pi[(int64_t)f * V + n] += 0.5 * h * tmp[(int64_t)f * V + n];
    }
    if (gv)
        for (int64_t n = 0; n < 5 * V; ++n) gp[n] += 0.5 * h * gtmp[n];

    const double a1 = m->expansion ? a + h * b : a;
    const double ahalf = 0.5 * (a + a1);
    const double cd = h * pow(ahalf, m->alpha - 3.0);
    ORC_PAR_FOR
    for (int64_t n = 0; n < (int64_t)m->nf * V; ++n) phi[n] += cd * pi[n];
    if (gv)
        for (int64_t n = 0; n < 5 * V; ++n) gv[n] += cd * gp[n];
    a = a1;

    for (int f = 0; f < m->nf; ++f) orc_kick_force(m, f, phi, a, tmp + (int64_t)f * V);
    if (gv) orc_gw_force(m, phi, gv, a, gtmp);  /* and with the fields at t + h */
    for (int f = 0; f < m->nf; ++f) {
        ORC_PAR_FOR
        for (int64_t n = 0; n < V; ++n) pi[(int64_t)f * V + n] += 0.5 * h * tmp[(int64_t)f * V + n];
    }
    if (gv) {
        for (int64_t n = 0; n < 5 * V; ++n) gp[n] += 0.5 * h * gtmp[n];
        free(gtmp);
    }

    if (m->expansion) {
        double abt1[3] = {a, b, abt[2]};
        orc_energies(m, phi, pi, NULL, NULL, abt1, e);
        b = b + 0.5 * h * orc_addot(m, a, e[ORC_E_RHO], e[ORC_E_P]);
    }
    abt[0] = a;
    abt[1] = b;
    abt[2] += h;
}

/* Low-storage (2N) Runge-Kutta coefficients.
 * RK3-3: Williamson, J. Comput. Phys. 35 (1980) 48, third-order three-stage scheme.
 * RK4-5: Carpenter & Kennedy, NASA TM-109112 (1994), fourth-order five-stage scheme
 *        (the paper's ref. for its RK4-5), coefficients as published there.       */
static const double RK33_A[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
static const double RK33_B[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};
static const double RK45_A[5] = {0.0,
                                 -567301805773.0 / 1357537059087.0,
                                 -2404267990393.0 / 2016746695238.0,
                                 -3550918686646.0 / 2091501179385.0,
                                 -1275806237668.0 / 842570457699.0};
static const double RK45_B[5] = {1432997174477.0 / 9575080441755.0,
                                 5161836677717.0 / 13612068292357.0,
                                 1720146321549.0 / 2090206949498.0,
                                 3134564353537.0 / 4481467310338.0,
                                 2277821191437.0 / 14882151754819.0};

/* RK3-4 (reading: the paper names a third-order four-stage low-storage scheme that admits
 * adaptive time steps, and prints no coefficients).  This 2N scheme is fixed by the order
 * conditions alone: the four third-order conditions on its Butcher weights; the state after
 * the third stage being a second-order solution at t + h (its abscissa c_4 = 1 and
 * sum_j a_4j c_j = 1/2), so that y_4 - y_3 = B_4 k estimates the local error with no extra
 * storage; and the z^4 coefficient of the stability function b A^3 1 = 1/24, which makes
 * R(z) the degree-4 Taylor polynomial of e^z (stable on the imaginary axis up to 2 sqrt 2).
 * These seven equations have one real solution; its coefficients, to 25 digits:           */
static const double RK34_A[4] = {0.0, -0.7825460361923582986318837, -2.042914325731224687686953,
                                 -1.799337253940777102361562};
static const double RK34_B[4] = {0.06688758201974096587947945, 2.876554598956718963241208,
                                 0.553465736134398241034173, 0.3912730180961791493159418};

int orc_rk_coeffs(int scheme, const double** A, const double** B)
{
    if (scheme == ORC_RK3_3) { *A = RK33_A; *B = RK33_B; return 3; }
    if (scheme == ORC_RK4_5) { *A = RK45_A; *B = RK45_B; return 5; }
    if (scheme == ORC_RK3_4) { *A = RK34_A; *B = RK34_B; return 4; }
    return 0;
}

double orc_nmc_ricci(const orc_model* m, const double* phi, const double* pi, const double* abt)
{
    const int64_t V = orc_volume(m);
    double e[ORC_NE];
    orc_energies(m, phi, pi, NULL, NULL, abt, e);
    double phidv = 0.0, phi2 = 0.0;
    for (int64_t n = 0; n < V; ++n) {
        phidv += phi[n] * orc_dV(m, 0, phi[n], 0.0);
        phi2 += phi[n] * phi[n];
    }
    phidv /= (double)V;
    phi2 /= (double)V;
    const double dphi2 = 2.0 * e[ORC_E_G0] - 2.0 * e[ORC_E_K0];  /* g^{mu nu} d_mu phi d_nu phi */
    const double F = 1.0 / (1.0 + (6.0 * m->xi - 1.0) * m->xi * m->kappa * phi2);
    return m->kappa * F * ((1.0 - 6.0 * m->xi) * dphi2 + 4.0 * e[ORC_E_V] - 6.0 * m->xi * phidv);
}

/* One 2N-storage RK step of the scalar system y = (phi, pi, a, a'), with
 *   F(y) = (a^(alpha-3) pi, a^(1+alpha) Lap phi - a^(3+alpha) V', a', a''(a, rho(y), p(y))).
 * Per stage s:  k <- A_s k + h F(y);  y <- y + B_s k   (one auxiliary copy per dof).
 * NMC models (Eq. eomNMC, Eq. piadot): the kick of field 0 gains -a^(3+alpha) xi R phi and
 *   a'' = a [a^(2 alpha) R / 6 - (1 - alpha) (a'/a)^2], with R = orc_nmc_ricci(y). */
static double rk_step(const orc_model* m, int scheme, double h, double* phi, double* pi, double* abt)
{
    const int64_t V = orc_volume(m);
    const int64_t nd = (int64_t)m->nf * V;
    const double *A, *B;
    const int S = orc_rk_coeffs(scheme, &A, &B);
    double* kphi = calloc((size_t)nd, sizeof(double));
    double* kpi = calloc((size_t)nd, sizeof(double));
    double* Fpi = malloc(sizeof(double) * (size_t)nd);
    double ka = 0.0, kb = 0.0;
    for (int s = 0; s < S; ++s) {
        const double a = abt[0], b = abt[1];
        double e[ORC_NE];
        double Fa = 0.0, Fb = 0.0;
        const double R = m->nmc ? orc_nmc_ricci(m, phi, pi, abt) : 0.0;
        if (m->expansion) {
            orc_energies(m, phi, pi, NULL, NULL, abt, e);
            Fa = b;
            Fb = m->nmc ? a * (pow(a, 2.0 * m->alpha) * R / 6.0 - (1.0 - m->alpha) * (b / a) * (b / a))
                        : orc_addot(m, a, e[ORC_E_RHO], e[ORC_E_P]);
        }
        for (int f = 0; f < m->nf; ++f) orc_kick_force(m, f, phi, a, Fpi + (int64_t)f * V);
        if (m->nmc) {
            const double c = pow(a, 3.0 + m->alpha) * m->xi * R;
            for (int64_t n = 0; n < V; ++n) Fpi[n] -= c * phi[n];
        }
        const double cd = pow(a, m->alpha - 3.0);
        for (int64_t n = 0; n < nd; ++n) {
            kphi[n] = A[s] * kphi[n] + h * cd * pi[n];
            kpi[n] = A[s] * kpi[n] + h * Fpi[n];
        }
        ka = A[s] * ka + h * Fa;
        kb = A[s] * kb + h * Fb;
        for (int64_t n = 0; n < nd; ++n) {
            phi[n] += B[s] * kphi[n];
            pi[n] += B[s] * kpi[n];
        }
        abt[0] += B[s] * ka;
        abt[1] += B[s] * kb;
    }
    abt[2] += h;
    /* embedded error estimate of the last stage's increment: |y_S - y_(S-1)| / |y_S| */
    double e2 = 0.0, y2 = 0.0;
    for (int64_t n = 0; n < nd; ++n) {
        const double dphi = B[S - 1] * kphi[n], dpi = B[S - 1] * kpi[n];
        e2 += dphi * dphi + dpi * dpi;
        y2 += phi[n] * phi[n] + pi[n] * pi[n];
    }
    free(kphi);
    free(kpi);
    free(Fpi);
    return y2 > 0.0 ? sqrt(e2 / y2) : 0.0;
}

void orc_step_adaptive(const orc_model* m, double* h, double tol, double hmin, double hmax, int nsteps,
                       double* phi, double* pi, double* abt, double* h_used, double* eps_out)
{
    for (int s = 0; s < nsteps; ++s) {
        const double eps = rk_step(m, ORC_RK3_4, *h, phi, pi, abt);
        h_used[s] = *h;
        eps_out[s] = eps;
        double f = eps > 0.0 ? 0.9 * cbrt(tol / eps) : 2.0;
        f = f > 2.0 ? 2.0 : (f < 0.2 ? 0.2 : f);
        double hn = *h * f;
        hn = hn > hmax ? hmax : (hn < hmin ? hmin : hn);
        *h = hn;
    }
}

/* Symmetric composition of order p (Yoshida 1990, section 4): a method of order p-2 applied
 * with steps x1 h, x0 h, x1 h, where x1 = 1/(2 - 2^(1/(p-1))) and x0 = 1 - 2 x1 cancel the
 * leading error term; order 2 is one velocity-Verlet step.  Order 4 gives the three-step
 * Yoshida scheme, orders 6, 8 and 10 take 9, 27 and 81 velocity-Verlet steps. */
static void composed_step(const orc_model* m, int order, double h, double* phi, double* pi, double* abt,
                          double* tmp, double* gv, double* gp)
{
    if (order <= 2) {
        vv_step(m, h, phi, pi, abt, tmp, gv, gp);
        return;
    }
    const double c = pow(2.0, 1.0 / (order - 1));
    const double x1 = 1.0 / (2.0 - c);
    const double x0 = -c / (2.0 - c);
    composed_step(m, order - 2, x1 * h, phi, pi, abt, tmp, gv, gp);
    composed_step(m, order - 2, x0 * h, phi, pi, abt, tmp, gv, gp);
    composed_step(m, order - 2, x1 * h, phi, pi, abt, tmp, gv, gp);
}

void orc_step(const orc_model* m, int scheme, double h, int nsteps,
              double* phi, double* pi, double* links, double* efield, double* abt)
{
    const int64_t V = orc_volume(m);
    if (m->gauge == 1) {
        if (scheme == ORC_VV2) {  /* the leapfrog with three fixed-point evaluations per implicit kick */
            orc_u1_leapfrog(m, h, nsteps, 3, phi, pi, links, efield, abt);
            return;
        }
        for (int s = 0; s < nsteps; ++s) orc_u1_rk_step(m, scheme, h, phi, pi, links, efield, abt);
        return;
    }
    double* tmp = malloc(sizeof(double) * (size_t)(m->nf * V));
    for (int s = 0; s < nsteps; ++s) {
        switch (scheme) {
        case ORC_VV2: vv_step(m, h, phi, pi, abt, tmp, NULL, NULL); break;
        case ORC_YOSHIDA4: composed_step(m, 4, h, phi, pi, abt, tmp, NULL, NULL); break;
        case ORC_YOSHIDA6: composed_step(m, 6, h, phi, pi, abt, tmp, NULL, NULL); break;
        case ORC_YOSHIDA8: composed_step(m, 8, h, phi, pi, abt, tmp, NULL, NULL); break;
        case ORC_YOSHIDA10: composed_step(m, 10, h, phi, pi, abt, tmp, NULL, NULL); break;
        default: rk_step(m, scheme, h, phi, pi, abt); break;
        }
    }
    free(tmp);
}

void orc_step_gw(const orc_model* m, int scheme, double h, int nsteps, double* phi, double* pi, double* gv,
                 double* gp, double* abt)
{
    const int64_t V = (int64_t)m->N * m->N * m->N;
    double* tmp = malloc(sizeof(double) * (size_t)(m->nf * V));
    const int order = scheme == ORC_VV2 ? 2 : scheme == ORC_YOSHIDA4 ? 4 : scheme == ORC_YOSHIDA6 ? 6
                    : scheme == ORC_YOSHIDA8 ? 8 : 10;
    for (int s = 0; s < nsteps; ++s) composed_step(m, order, h, phi, pi, abt, tmp, gv, gp);
    free(tmp);
}
