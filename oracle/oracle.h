/*
 * FP64 CPU oracle of the CosmoLattice-2.0 lattice time step -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference leg
 * may load this code.  It shares nothing with the CUDA path (no headers, no
 * tables, no helpers): it is a second, independent statement of the method,
 * written as plain loops in double precision so that it can be read against the
 * paper equation by equation.
 *
 * Program variables (section "Inherited capabilities", Eq. FieldSpaceTimeNaturalVariables):
 * fields phi~ = phi/f_star, alpha-time eta~, comoving x~.  Momenta are pi = a^(3-alpha) phi'
 * (the canonical choice the paper defers to its companion review), so that
 * Eq. singletEOM becomes
 *      phi' = a^(alpha-3) pi ,      pi' = a^(1+alpha) Lap phi - a^(3+alpha) dV/dphi .
 * The scale factor obeys Eq. Friedmann1 with kappa = (f_star / m_p)^2,
 *      a'' = a^(2 alpha + 1) (kappa/6) [ (2 alpha - 1) rho - 3 p ],
 * and Eq. Friedmann2 (H^2 = a^(2 alpha) kappa rho / 3, H = a'/a) is the monitored constraint.
 *
 * Lattice operators (readings; the paper defers them to its companion review):
 *      Lap f(n)   = sum_i [f(n+i) + f(n-i) - 2 f(n)] / dx^2          (7-point)
 *      grad+_i f  = [f(n+i) - f(n)] / dx                              (forward)
 * Site index: n = (z*N + y)*N + x, x fastest, periodic in every direction.
 *
 * Parity is pinned (tests/test_oracle_*.py) against closed forms, invariants and
 * brute force; no function here is "parity unpinned" unless its comment says so.
 */
#ifndef CL_ORACLE_H
#define CL_ORACLE_H

#include <stdint.h>

/* Loop-parallel build.  liboracle_omp.so (compiled with -fopenmp) exists only to time
 * the oracle on every host core for the CPU baseline: the site loops of the scalar step
 * are split across threads and its sums become OpenMP reductions (so their summation
 * order differs).  liboracle.so, which every test loads, is compiled without OpenMP;
 * there these macros expand to nothing and every loop runs in the order written. */
#ifdef _OPENMP
#define ORC_PRAGMA(x) _Pragma(#x)
#define ORC_PAR_FOR ORC_PRAGMA(omp parallel for schedule(static))
#define ORC_PAR_SUM(v) ORC_PRAGMA(omp parallel for schedule(static) reduction(+ : v))
#else
#define ORC_PAR_FOR
#define ORC_PAR_SUM(v)
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Model description.  Potential in program units (two real singlets phi_0, phi_1):
 *   V = m2[0]/2 phi0^2 + lam[0]/4 phi0^4 + m2[1]/2 phi1^2 + lam[1]/4 phi1^4 + g2/2 phi0^2 phi1^2
 * which covers lambda phi^4, m^2 phi^2 and the phi^2 chi^2 preheating families. */
typedef struct {
    int32_t N;          /* sites per side                                   */
    int32_t nf;         /* number of scalar fields (1 or 2)                 */
    int32_t expansion;  /* 1: self-consistent FLRW; 0: a, a' frozen         */
    int32_t gauge;      /* 0: none; 1: compact U(1) + axion coupling        */
    double L;           /* box side, program units; dx = L/N                */
    double alpha;       /* alpha-time exponent (0 cosmic, 1 conformal)      */
    double kappa;       /* (f_star / m_p)^2                                       */
    double m2[2];
    double lam[2];
    double g2;
    /* gauge sector (gauge == 1): axion coupling alpha_L and the factor
     * (omega_star / f_star)^2 that multiplies E.B in the axion equation.             */
    double alphaL;
    double ws2;
    /* non-minimal coupling xi phi^2 R of field 0 (section "Scalar fields non-minimally
     * coupled to gravity"); Runge-Kutta schemes only, one field, no gauge sector        */
    int32_t nmc;        /* 1: on                                                         */
    double xi;
    /* spatial dimensions of the lattice (section "Scalar dynamics in 1+1 and 2+1 dimensions"):
     * 0 or 3 = N^3 sites; 2 = N^2 and 1 = N sites, the Laplacian and the gradient energy
     * summed over those directions only, everything else unchanged.  Scalar fields only.   */
    int32_t dims;
} orc_model;

/* Sites of the model's lattice, and its extents along x, y, z (1 beyond dims). */
int64_t orc_volume(const orc_model* m);
void orc_extents(const orc_model* m, int* nx, int* ny, int* nz);

/* Indices into the energies vector returned by orc_energies(). */
enum {
    ORC_E_K0 = 0, ORC_E_K1, ORC_E_G0, ORC_E_G1, ORC_E_V,
    ORC_E_KEM, ORC_E_GEM,           /* U(1) electric / magnetic energies  */
    ORC_E_RHO, ORC_E_P, ORC_E_HV,   /* rho, p, Hubble-constraint violation */
    ORC_E_A, ORC_E_B,               /* a and a' the energies refer to      */
    ORC_NE
};

/* Integrators (section "Non-symplectic evolvers" and the symplectic family it lists). */
enum { ORC_VV2 = 0, ORC_YOSHIDA4 = 1, ORC_RK3_3 = 2, ORC_RK4_5 = 3, ORC_YOSHIDA6 = 4, ORC_YOSHIDA8 = 5,
       ORC_YOSHIDA10 = 6, ORC_RK3_4 = 7 };

/* ---- potential and lattice operators ---- */
double orc_V(const orc_model* m, double f0, double f1);
double orc_dV(const orc_model* m, int f, double f0, double f1);
double orc_d2V(const orc_model* m, int f, double f0, double f1);
void   orc_laplacian(int N, double dx, const double* f, double* out);
double orc_grad2_sum(int N, const double* f);
void   orc_kick_force(const orc_model* m, int f, const double* phi, double a, double* out);

/* ---- volume averages and the Friedmann equations ---- */
/* phi, pi: nf arrays of N^3 back to back.  abt = {a, a', t}.  out[ORC_NE]. */
void   orc_energies(const orc_model* m, const double* phi, const double* pi,
                    const double* links, const double* efield,
                    const double* abt, double* out);
double orc_addot(const orc_model* m, double a, double rho, double p);
/* Background Ricci scalar of an NMC model at the state (phi, pi, abt): Eq. eomR in program
 * units, R = kappa F [(1 - 6 xi) <d phi . d phi> + 4 <V> - 6 xi <phi V'>],
 * F = 1 / (1 + (6 xi - 1) xi kappa <phi^2>), <d phi . d phi> = 2 G - 2 K. */
double orc_nmc_ricci(const orc_model* m, const double* phi, const double* pi, const double* abt);

/* ---- time integration ----
 * Scalar models: links = efield = NULL.
 * U(1)+axion models (gauge == 1): nf = 1, links/efield are 3 arrays of N^3
 * (theta_i = dx * A_i on the link n -> n+i, E_i on the same link). */
void orc_step(const orc_model* m, int scheme, double h, int nsteps,
              double* phi, double* pi, double* links, double* efield, double* abt);

/* ---- gravitational waves (gw.c; section "New algorithm for GWs") ----
 * Five traceless auxiliaries v = {v11, v12, v13, v22, v23} (v33 = -v11 - v22), each N^3, and
 * their momenta gp = a^(3-alpha) v' (same layout).  orc_gw_force: the kick
 *   a^(1+alpha) Lap v_ab + 2 kappa a^(1+alpha) [Pi_ab - delta_ab Pi / 3],
 *   Pi_ab = sum_f dbar_a phi_f dbar_b phi_f, dbar the central difference;
 * orc_step_gw: the leapfrog schemes (VV2, Yoshida) of orc_step with the GW fields kicked and
 * drifted alongside the scalars (no backreaction on a);
 * orc_gw_spectrum: d rho_GW / d log k of the TT part of h' = a^(alpha-3) gp, binned as
 * orc_spectrum with the factor 1 / (4 kappa a^(2 alpha)). */
void orc_gw_force(const orc_model* m, const double* phi, const double* gv, double a, double* out);
void orc_step_gw(const orc_model* m, int scheme, double h, int nsteps, double* phi, double* pi, double* gv,
                 double* gp, double* abt);
int orc_gw_spectrum(const orc_model* m, const double* gp, const double* abt, double dn, int type, double* k_out,
                    double* delta_out, double* count_out, int cap);

/* ---- U(1) + axion: right-hand side of the coupled system and the Gauss charge ---- */
void orc_u1_rhs(const orc_model* m, const double* phi, const double* pi, const double* links,
                const double* efield, const double* abt,
                double* dphi, double* dpi, double* dlinks, double* defield);
int orc_gauge_spectrum(const orc_model* m, const double* links, const double* efield, int which, double dn,
                       int type, double* k_out, double* delta_out, double* count_out, int cap);
void orc_u1_gauss(const orc_model* m, const double* phi, const double* links,
                  const double* efield, double a, double* out_gauss /* N^3 */);
/* Leapfrog of the U(1) + axion system (u1.c): positions phi, theta, a at integer steps, the
 * kick of the momenta pi, E at fixed positions implicit (generalized Stoermer-Verlet), solved
 * with `iters` fixed-point evaluations of the momentum force.  orc_step with ORC_VV2 on a
 * gauge model takes iters = 3. */
void orc_u1_leapfrog(const orc_model* m, double h, int nsteps, int iters, double* phi, double* pi,
                     double* links, double* efield, double* abt);

/* ---- random numbers, initial conditions, spectra ---- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void orc_dft3(int N, int sign, double* re, double* im);
void orc_vacuum(const orc_model* m, uint64_t seed, uint32_t member, double kcut, double amp2,
                const double* fbar, const double* dfbar, double a0,
                double* phi, double* pi, double* abt);
int  orc_spectrum(int N, double L, const double* f, double dn, int type,
                  double* k_out, double* delta_out, double* count_out, int cap);

/* ---- convolutional surrogate layers (surrogate.c): periodic 3x3x3 convolutions ----
 * x[n*C + c] site-major; W[(t*cout + co)*cin + ci], tap t = (tz*3 + ty)*3 + tx at offset
 * (tx-1, ty-1, tz-1). */
void orc_conv3d_fwd(int N, int cin, int cout, const double* x, const double* W, const double* b, double* y);
void orc_conv3d_bwd_data(int N, int cin, int cout, const double* dy, const double* W, double* dx);
void orc_conv3d_bwd_weight(int N, int cin, int cout, const double* x, const double* dy, double* dW, double* db);
double orc_act(int act, double u);       /* 0 = ReLU, 1 = GELU (tanh form) */
double orc_act_grad(int act, double u);
void orc_act_array(int act, int64_t n, const double* u, double* h);
void orc_act_bwd_array(int act, int64_t n, const double* u, const double* dh, double* du);

/* Adaptive RK3-4 steps (section "Non-symplectic evolvers": RK3-4 admits adaptive time
 * stepping).  Each step is taken with the current h and always accepted; its embedded error
 * estimate eps = |y_4 - y_3| / |y_4| (2-norms over phi and pi of every field and site; y_3,
 * the state after the third stage, is a second-order solution at t + h) sets the next step,
 *     h <- clamp(h * min(2, max(1/5, 0.9 (tol / eps)^(1/3))), hmin, hmax)   (h * 2 if eps = 0).
 * h_used[s], eps_out[s] (nsteps each) receive the step sizes taken and their estimates;
 * h is updated in place. */
void orc_step_adaptive(const orc_model* m, double* h, double tol, double hmin, double hmax, int nsteps,
                       double* phi, double* pi, double* abt, double* h_used, double* eps_out);

/* Threads the loop-parallel build uses (1 in the serial build). */
int orc_threads(void);

#ifdef __cplusplus
}
#endif
#endif
