/*
 * cl.h -- C ABI of the GB300 (sm_103a) lattice time-step library libcl.so.
 *
 * The library advances CosmoLattice-2.0-style lattice field theories: interacting
 * real scalar singlets, optionally one axion coupled to compact U(1) links, on a
 * periodic N^3 lattice in a self-consistently expanding FLRW background.  All
 * quantities are in the paper's program variables (section "Inherited capabilities
 * from CL 1.X", Eq. FieldSpaceTimeNaturalVariables): phi~ = phi/f_star,
 * d eta~ = a^-alpha omega_star dt, x~ = omega_star x, A~ = A/omega_star.
 *
 * Conventions shared by every call
 *   - Site index n = (z*N + y)*N + x (x fastest), periodic boundaries.  dx = L/N.
 *   - Field momenta are pi = a^(3-alpha) phi', so Eq. singletEOM reads
 *       phi' = a^(alpha-3) pi,   pi' = a^(1+alpha) Lap phi - a^(3+alpha) dV/dphi,
 *     with the 7-point Laplacian; gradient energies use forward differences.
 *   - The scale factor a and its alpha-time derivative a' ("adot") follow
 *     Eq. Friedmann1; Eq. Friedmann2 is monitored (the "Hubble violation").
 *   - Element type of every field array is double for CL_PREC_FP64 and float for
 *     CL_PREC_FP32 and CL_PREC_FP32_KAHAN.  Energies, a, a' and t are always double.
 *   - The library owns all device memory of a lattice.  Caller buffers are only
 *     read or written during the call that receives them (host buffers), or in
 *     stream order on the lattice's stream (device buffers, on_device = 1).
 *   - Work is queued on the CUDA stream given at creation (NULL = legacy default
 *     stream).  cl_step only queues work; device-side failures (a non-finite
 *     energy, a Hubble violation above the limit) are reported by the next
 *     synchronising call: cl_sync, cl_energies, cl_get_state, cl_spectrum.
 *   - No call aborts the process.  Every call returns a cl_status; the text of
 *     the last failure of a handle is available from cl_last_error.
 *   - A handle must not be used from two host threads at the same time.
 */
#ifndef CL_H
#define CL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cl_lattice cl_lattice; /* opaque, owned by the library */

typedef enum {
    CL_OK = 0,
    CL_EINVAL = 1,        /* bad argument: size, enum value, NULL pointer, out-of-range member */
    CL_ENOMEM = 2,        /* device or host allocation failed                                  */
    CL_ECUDA = 3,         /* a CUDA runtime or cuFFT call failed                               */
    CL_ENAN = 4,          /* a volume-averaged energy became non-finite                        */
    CL_ECONSTRAINT = 5,   /* Hubble-constraint violation above the limit set by cl_set_hubble_limit */
    CL_ETIMEOUT = 6,      /* a bounded device wait of a pipelined kernel gave up (reported by
                             the next synchronising call, like CL_ENAN)                        */
    CL_ESTATE = 7,        /* call not valid in the handle's current state                      */
    CL_EUNSUPPORTED = 8   /* valid request that this build does not implement                  */
} cl_status;

/* Precision of field storage and arithmetic.  Reductions, a(t) and a'(t) are FP64 in all modes. */
enum {
    CL_PREC_FP64 = 0,       /* double fields                                            */
    CL_PREC_FP32_KAHAN = 1, /* float fields, compensated (Kahan) drift of every field    */
    CL_PREC_FP32 = 2        /* float fields, plain drift                                 */
};

/* Time integrators (section "Non-symplectic evolvers"). */
enum {
    CL_INT_VV2 = 0,      /* velocity Verlet, O(dt^2), one fused lattice pass per step           */
    CL_INT_YOSHIDA4 = 1, /* Yoshida composition of three VV steps, O(dt^4), three passes/step   */
    CL_INT_RK3_3 = 2,    /* low-storage 2N Runge-Kutta, 3rd order, 3 stages (Williamson 1980)   */
    CL_INT_RK4_5 = 3,    /* low-storage 2N Runge-Kutta, 4th order, 5 stages (Carpenter-Kennedy 1994) */
    /* Higher-order Yoshida compositions (section "Non-symplectic evolvers" lists orders up to
     * 10): the symmetric triple jump applied recursively to VV-2, 3^((p-2)/2) passes/step   */
    CL_INT_YOSHIDA6 = 4,  /* O(dt^6), 9 passes/step   */
    CL_INT_YOSHIDA8 = 5,  /* O(dt^8), 27 passes/step  */
    CL_INT_YOSHIDA10 = 6, /* O(dt^10), 81 passes/step */
    /* low-storage 2N Runge-Kutta, 3rd order, 4 stages, with an embedded second-order solution
     * (the state after its third stage) for adaptive time steps (section "Non-symplectic
     * evolvers" names RK3-4 and its adaptive stepping without printing coefficients; this
     * table is fixed by the third-order conditions, c_4 = 1 with sum_j a_4j c_j = 1/2, and a
     * stability function equal to the degree-4 Taylor polynomial of e^z): see
     * cl_set_adaptive */
    CL_INT_RK3_4 = 7
};

enum { CL_GAUGE_NONE = 0, CL_GAUGE_U1_AXION = 1 };

/* Potentials in program units (cl_set_potential).  All are special cases of
 *   V = m2_0/2 phi0^2 + lam_0/4 phi0^4 + m2_1/2 phi1^2 + lam_1/4 phi1^4 + g2/2 phi0^2 phi1^2. */
enum {
    CL_POT_LPHI4 = 0,    /* params {lam}:       V = lam/4 phi^4                      (1 field)  */
    CL_POT_M2 = 1,       /* params {m2}:        V = m2/2 phi^2                       (1 field)  */
    CL_POT_M2_G2 = 2,    /* params {m2, g2}:    V = m2/2 phi^2 + g2/2 phi^2 chi^2    (2 fields) */
    CL_POT_LPHI4_G2 = 3, /* params {lam, g2}:   V = lam/4 phi^4 + g2/2 phi^2 chi^2   (2 fields) */
    CL_POT_POLY = 4      /* params {m2_0, lam_0, m2_1, lam_1, g2}: the general form above       */
};

/* Field identifiers for cl_set_state / cl_get_state / cl_spectrum. */
enum {
    CL_FIELD_PHI0 = 0, CL_FIELD_PHI1 = 1, /* scalar fields                                  */
    CL_FIELD_PI0 = 2, CL_FIELD_PI1 = 3,   /* their momenta pi = a^(3-alpha) phi'            */
    CL_FIELD_THETA1 = 4, CL_FIELD_THETA2 = 5, CL_FIELD_THETA3 = 6, /* U(1) link angles dx*A_i on n -> n+i */
    CL_FIELD_E1 = 7, CL_FIELD_E2 = 8, CL_FIELD_E3 = 9,            /* electric field A_i' on the same links */
    /* gravitational-wave auxiliaries (cl_enable_gw): v11, v12, v13, v22, v23 (v33 = -v11 - v22)
     * and their momenta a^(3-alpha) v' */
    CL_FIELD_GW_V11 = 10, CL_FIELD_GW_V12 = 11, CL_FIELD_GW_V13 = 12, CL_FIELD_GW_V22 = 13, CL_FIELD_GW_V23 = 14,
    CL_FIELD_GW_P11 = 15, CL_FIELD_GW_P12 = 16, CL_FIELD_GW_P13 = 17, CL_FIELD_GW_P22 = 18, CL_FIELD_GW_P23 = 19
};

/* Batched ensembles (members > 1): B independent lattices of sizes member_N[m]
 * (2..512 each) and boxes member_L[m], each with its own couplings, a, a', t and step
 * count, advanced together by one launch per pass (N and L are then ignored).  They share
 * nfields, precision, integrator (VV-2 or a Yoshida composition), alpha, kappa and dt;
 * gauge must be CL_GAUGE_NONE.  Every call that takes a member addresses one of them; the
 * fields of member m hold member_N[m]^3 elements.  Errors at creation: CL_EINVAL (sizes),
 * CL_EUNSUPPORTED (Runge-Kutta or gauge ensembles). */
typedef struct {
    int32_t N;            /* sites per side, 2 <= N <= 1536 (single lattice; reduced      */
                          /* lattices: N <= 46340 for dims 2, N <= 2^30 for dims 1)          */
    int32_t nfields;      /* scalar fields, 1 or 2 (1 when gauge = CL_GAUGE_U1_AXION)       */
    int32_t precision;    /* CL_PREC_*                                                      */
    int32_t integrator;   /* CL_INT_*                                                       */
    int32_t gauge;        /* CL_GAUGE_*                                                     */
    int32_t expansion;    /* 1: self-consistent expansion (Eq. Friedmann1); 0: a, a' frozen */
    int32_t members;      /* ensemble size B; 0 or 1 = single lattice (see below)           */
    int32_t dims;         /* spatial dimensions: 0 or 3 = N^3 sites; 2 / 1 = the reduced     */
                          /* (2+1) / (1+1)-dimensional lattice of N^2 / N sites (section     */
                          /* "Scalar dynamics in 1+1 and 2+1 dimensions"): Laplacian and     */
                          /* gradient energy over those directions, the rest unchanged;     */
                          /* single lattices of scalar fields only (CL_EUNSUPPORTED with     */
                          /* ensembles or gauge fields; vacuum initial conditions, spectra, */
                          /* GW, non-minimal coupling, autotuner and surrogate refuse them). */
                          /* Field arrays hold N^dims elements, x fastest.                  */
    const int32_t* member_N; /* B per-member sizes (copied) when members > 1, else NULL     */
    const double* member_L;  /* B per-member box sides (copied), or NULL = L for all        */
    double L;             /* box side in program units                                      */
    double alpha;         /* alpha-time exponent (Eq. FLRWmetric): 0 cosmic, 1 conformal    */
    double kappa;         /* (f_star/m_p)^2, sets the strength of Eq. Friedmann1/2          */
    double dt;            /* time step in program units                                     */
    double a0;            /* initial scale factor (a' starts at 0 until set)                */
    void* stream;         /* cudaStream_t used for all work of this handle; NULL = default  */
} cl_lattice_params;

/* Vacuum initial conditions (section "Initial conditions", Eq. QuantumFlucts,
 * Eq. fpr_influct, Eq. fpr_influct2): homogeneous values plus Gaussian modes of
 * variance (N/dx)^3 P(k) per mode, P = amp2 / (2 a^2 omega_k), omega_k^2 = k^2 + a^2 V''(fbar),
 * zero at k = 0 and for |k| > kcut.  Random numbers: Philox-4x32-10 with key = seed
 * and counter = (mode index, field, member, 0). */
typedef struct {
    uint64_t seed;
    double kcut;      /* momentum cut-off in program units (use a huge value for none) */
    double amp2;      /* (omega_star/f_star)^2, the vacuum amplitude in program units  */
    double fbar[2];   /* homogeneous field values                                      */
    double dfbar[2];  /* homogeneous alpha-time derivatives phi'                       */
} cl_vacuum_params;

/* Volume averages at the most recent integer time (Eq. energy-contrib, Eq. rhoLocal). */
typedef struct {
    double t;                 /* alpha-time                                              */
    double a, adot;           /* scale factor and a' at t                                */
    double K[2], G[2];        /* kinetic and gradient energy of each scalar field        */
    double V;                 /* potential energy                                        */
    double KE, GB;            /* U(1) electric and magnetic energies (0 without gauge)   */
    double rho, p;            /* energy density and pressure                             */
    double hubble_violation;  /* |H^2 - a^(2 alpha) kappa rho/3| / H^2, H = a'/a (0 if H = 0) */
    double gauss_violation;   /* U(1): lattice Gauss charge G(n) = sum_i [P_i(n) - P_i(n-i)]/dx,
                                 P = a^(1-alpha) E + g W (Eq. AxionInfEOM's Gauss law), of the
                                 current state: max_n |G(n)| / max_n sum_i (|P_i(n)| + |P_i(n-i)|)/dx;
                                 0 without gauge                                         */
    int64_t step;             /* time steps taken since the state was set                */
    double ricci;             /* background Ricci scalar R (Eq. eomR) of a non-minimally coupled
                                 lattice (cl_set_nonminimal); 0 otherwise                  */
    double gauss_rms_step;    /* U(1), tracked every step: rms Gauss violation of the latest
                                 cl_step step's starting state (the leapfrog's integer-time
                                 starting state, its momenta at the integer time),
                                 dx sqrt(sum_n G(n)^2) / (a^(1-alpha) sqrt(sum_n E(n)^2))   */
    double gauss_rms_max;     /* U(1): the largest gauss_rms_step since the last
                                 cl_set_scalars or cl_init_vacuum                         */
    double dt;                /* the step size the next cl_step step takes (adaptive RK3-4:
                                 set by the controller; otherwise the lattice's dt)       */
    double rk_error;          /* adaptive RK3-4: embedded error estimate of the latest step,
                                 |y_4 - y_3| / |y_4| over phi and pi; 0 otherwise           */
} cl_energy;

/* Create a lattice.  Allocates all device memory (fields, their ping-pong copies,
 * Kahan compensation arrays, reduction scratch) and zeroes it; a = a0, a' = 0, t = 0.
 * Errors: CL_EINVAL (bad sizes/enums/NULL), CL_ENOMEM, CL_ECUDA. *out is NULL on error. */
cl_status cl_init_lattice(cl_lattice** out, const cl_lattice_params* p);

/* Release every resource of the handle (waits for its queued work).  NULL is ignored. */
void cl_free(cl_lattice* l);

/* Set the potential (kind = CL_POT_*).  params holds the kind's values (LPHI4 {lam},
 * M2 {m2}, M2_G2 {m2, g2}, LPHI4_G2 {lam, g2}, POLY {m2_0, lam_0, m2_1, lam_1, g2});
 * for an ensemble either one set shared by every member or members sets back to back.
 * Errors: CL_EINVAL (count, kind, non-finite value, two-field terms on one field). */
cl_status cl_set_potential(cl_lattice* l, int32_t kind, const double* params, int32_t nparams);

/* Copy one field of one member in (set) or out (get).  src/dst hold N^3 elements (the
 * member's N for an ensemble; member -1 = 0 for a single lattice) of the lattice's element type, in host memory (on_device = 0) or device memory (on_device = 1).
 * cl_set_state leaves the handle at an integer time: the next cl_step first opens the
 * leapfrog with a half kick.  cl_get_state returns the values at the most recent
 * integer time (momenta are synchronised on the fly; the evolving state is not altered).
 * Errors: CL_EINVAL (field/member out of range, NULL), CL_ECUDA, CL_ENAN/CL_ECONSTRAINT. */
cl_status cl_set_state(cl_lattice* l, int32_t member, int32_t field, const void* src, int32_t on_device);
cl_status cl_get_state(cl_lattice* l, int32_t member, int32_t field, void* dst, int32_t on_device);

/* Scale factor a, its derivative a' and the time t of one member (member = -1: all).
 * Passing adot = NaN to cl_set_scalars computes a' from Eq. Friedmann2 with the lattice
 * energy (expanding lattices only). */
cl_status cl_set_scalars(cl_lattice* l, int32_t member, double a, double adot, double t);
cl_status cl_get_scalars(cl_lattice* l, int32_t member, double* a, double* adot, double* t);

/* Gaussian vacuum fluctuations over the homogeneous values for every scalar field of
 * one member (member = -1: every member, each with its own Philox counter stream);
 * momenta pi = a^(3-alpha) phi'; a' from Eq. Friedmann2 with the lattice energy.
 * Uses cuFFT; not part of the timed step.  Errors: CL_EINVAL, CL_ECUDA, CL_ENOMEM. */
cl_status cl_init_vacuum(cl_lattice* l, int32_t member, const cl_vacuum_params* v);

/* Queue nsteps time steps of the configured integrator on the handle's stream (replayed
 * from a captured CUDA graph when graphs are enabled).  Returns after queueing.
 * Errors: CL_EINVAL (nsteps < 0), CL_ESTATE (cl_set_potential not called), CL_ECUDA. */
cl_status cl_step(cl_lattice* l, int32_t nsteps);

/* Wait for the handle's queued work; report device-side failures (CL_ENAN, CL_ECONSTRAINT,
 * CL_ETIMEOUT). */
cl_status cl_sync(cl_lattice* l);

/* Copy the energies of `count` members (starting at member 0; 1 <= count <= members, or
 * count = 1 for a single lattice) to host memory `out`.
 * Synchronising.  Errors: CL_EINVAL, CL_ECUDA, CL_ENAN, CL_ECONSTRAINT, CL_ETIMEOUT. */
cl_status cl_energies(cl_lattice* l, cl_energy* out, int32_t count);

/* Binned spectrum of one field (section "Arbitrary binning and unbinned spectra",
 * Eq. discretePST2, Eq. UpsilonII).  Bin l collects modes with floor(|n~|/dn + 1/2) = l;
 * for l > 0, with n_l = l dn and S_l the sum of |f(n~)|^2 over the bin (DFT without
 * normalisation):  type 1: Delta = n_l S_l / (N^6 dn);  type 2: Delta = 4 pi n_l^3 (S_l/#_l) / N^6.
 * k_out[l] = (2 pi / L) n_l, count_out[l] = #_l (number of modes), delta_out[0] = 0.
 * Writes min(cap, bins) host values and sets *nbins to the number of bins of the lattice.
 * Uses cuFFT; synchronising.  Errors: CL_EINVAL, CL_ECUDA, CL_ENOMEM. */
cl_status cl_spectrum(cl_lattice* l, int32_t member, int32_t field, double dn, int32_t type,
                      double* k_out, double* delta_out, double* count_out, int32_t cap, int32_t* nbins);

/* Spectra of the U(1) sector of an axion-U(1) lattice (section "ALP-gauge interactions":
 * the two chiralities of the gauge field are output separately).  which:
 *   CL_GSPEC_E: electric field, sum over i of |E_i(k)|^2;
 *   CL_GSPEC_B: magnetic field B_k(n) = sin P_k(n) / dx^2 (plaquette of normal k at lower corner n);
 *   CL_GSPEC_APLUS / CL_GSPEC_AMINUS: the + / - chirality of the gauge potential
 *     A_i = theta_i / dx: with the half-link phase exp(-i k_i dx / 2) of A^_i and the lattice
 *     momentum kt_l = (2/dx) sin(k_l dx / 2), the power of conj(e_s) . A^ where
 *     i (kt/|kt|) x e_s = s e_s, s = +1 / -1 (the forward-difference curl is i kt x A^).
 * Binning, normalisation, type and outputs as cl_spectrum (state at the current integer time).
 * Uses cuFFT; synchronising.  Errors: CL_EINVAL (no gauge field, bad arguments), CL_ECUDA,
 * CL_ENOMEM. */
enum { CL_GSPEC_E = 0, CL_GSPEC_B = 1, CL_GSPEC_APLUS = 2, CL_GSPEC_AMINUS = 3 };
cl_status cl_gauge_spectrum(cl_lattice* l, int32_t which, double dn, int32_t type, double* k_out, double* delta_out,
                            double* count_out, int32_t cap, int32_t* nbins);

/* Axion-U(1) couplings (gauge = CL_GAUGE_U1_AXION; section "ALP-gauge interactions",
 * Eq. AxionInfEOM): alphaL is the dimensionless coupling alpha_Lambda of the
 * alpha_Lambda/(4 m_p) phi F Ftilde term, ws2 = (omega_star/f_star)^2 the weight of the
 * electromagnetic energy in the scalar's energy unit.  In program units the axion equation
 * gains ws2 g Ebar.Bbar and the electric field -g (phi' Bbar - grad phi x Ebar) with
 * g = alphaL sqrt(kappa).  On the lattice: link angles theta_i = dx A_i and E_i = A_i' on the
 * links n -> n+i (fields CL_FIELD_THETA1..3, CL_FIELD_E1..3, zero at creation),
 * Ebar the two-link average and Bbar the clover average of sin(plaquette)/dx^2; the equations
 * are the Euler-Lagrange equations of the lattice action, so the lattice Gauss law is a
 * conserved charge of the continuous-time flow.  Gauge lattices integrate with
 * CL_INT_RK3_3 / CL_INT_RK4_5 / CL_INT_RK3_4 (as the paper does for this module) or with
 * CL_INT_VV2, a leapfrog with the kick of (pi, E) implicit at fixed positions, since the
 * E' of Eq. AxionInfEOM depends on phi' and the pi' on E: positions (phi, theta, a) at
 * integer steps, momenta (pi, E, a') at half steps in between, and
 *   p_(n+1/2) = p_n + h/2 f(q_n, a_n, a'_(n+1/2), p_(n+1/2))   (implicit half-kick)
 *   q_(n+1)   = q_n + h (drift with p_(n+1/2), a at the midpoint)
 *   p_(n+1)   = p_(n+1/2) + h/2 f(q_(n+1), a_(n+1), a'_(n+1/2), p_(n+1/2))   (explicit)
 * with a' half-kicked by Eq. Friedmann1 at the integer times (the generalized
 * Stoermer-Verlet method: order 2, time-reversible when converged).  The implicit half-kick
 * is solved by three evaluations of f: the first from the previous step's closing force (in
 * the first step of a cl_step call from a written state, the force at that state), two
 * fixed-point iterations after it.  Between calls the leapfrog stays open: the integer-time
 * momenta are kept beside the staggered ones, so reading fields, energies or spectra does
 * not change the trajectory; writing the state or the scalars closes it.  One step is three
 * passes of two launches each (one each with CL_OPT_PASS_VARIANT 3), the rms Gauss violation
 * of every step's integer-time starting state summed by the second pass (the gather form,
 * variant 0, adds one reduction launch) and reported in cl_energy::gauss_rms_step / _max;
 * the first step of a cl_step call from a closed state adds the opening pass.  One axion
 * field, CL_PREC_FP64 or CL_PREC_FP32.  Errors: CL_EINVAL (no gauge field, bad values). */
cl_status cl_set_gauge_coupling(cl_lattice* l, double alphaL, double ws2);

/* Non-minimal coupling xi phi^2 R of the scalar field (section "Scalar fields non-minimally
 * coupled to gravity", Eq. eomNMC, Eq. eomR, Eq. piadot) for a single lattice with one field
 * and a Runge-Kutta integrator (the paper integrates this system with them).  Each stage then
 * first reduces the background Ricci scalar of its state,
 *   R = kappa F [(1 - 6 xi) (2 G - 2 K) + 4 <V> - 6 xi <phi V'>],  F = 1/(1 + (6 xi - 1) xi kappa <phi^2>)
 * (program units, K = <pi^2>/(2 a^6), G = <(grad+ phi)^2>/(2 a^2)); the kick gains
 * -a^(3+alpha) xi R phi and a'' = a [a^(2 alpha) R/6 - (1 - alpha)(a'/a)^2].  The energies keep
 * their minimally coupled form (hubble_violation is then not a constraint of the system; set
 * a' explicitly).  Errors: CL_EINVAL, CL_EUNSUPPORTED. */
cl_status cl_set_nonminimal(cl_lattice* l, double xi);

/* Adaptive time steps of CL_INT_RK3_4 (section "Non-symplectic evolvers": RK3-4 admits
 * adaptive time stepping).  With tol > 0 every cl_step step is taken with the current step
 * size h (starting from the lattice's dt) and always accepted; its last stage reduces the
 * embedded error estimate eps = |y_4 - y_3| / |y_4| (2-norms over phi and pi of every field
 * and site, y_3 the second-order state after the third stage) and sets, on the device,
 *     h <- clamp(h min(2, max(1/5, 0.9 (tol / eps)^(1/3))), h_min, h_max)   (2 h if eps = 0)
 * for the next step, so steps stay graph-replayed with no host round trip.  tol <= 0 returns
 * to the fixed dt.  cl_energies reports the current h (dt) and the latest eps (rk_error).
 * Single lattices of scalar fields (3-D or reduced) without non-minimal coupling.
 * Errors: CL_EINVAL (h_min > h_max, non-positive h_max), CL_EUNSUPPORTED (another
 * integrator, gauge fields, ensembles, non-minimal coupling). */
cl_status cl_set_adaptive(cl_lattice* l, double tol, double h_min, double h_max);

/* Gravitational waves (section "New algorithm for GWs"): five traceless auxiliaries v_ij
 * (v33 = -v11 - v22, fields CL_FIELD_GW_*, zero when enabled) evolved with the leapfrog
 * alongside the scalars:
 *   v' = a^(alpha-3) pi_v,  pi_v' = a^(1+alpha) Lap v + 2 kappa a^(1+alpha) [Pi_ij - delta_ij Pi / 3],
 *   Pi_ij = sum_f dbar_i phi_f dbar_j phi_f  (central differences), no backreaction on a.
 * A single scalar lattice with a leapfrog integrator (VV-2 or Yoshida); one GW launch joins
 * every pass.  Errors: CL_EUNSUPPORTED (ensembles, gauge fields, Runge-Kutta), CL_ENOMEM. */
cl_status cl_enable_gw(cl_lattice* l);

/* Energy spectrum of the gravitational waves, d rho_GW / d log k in program units, of the TT
 * part h_ij(k) = Lambda_ij,lm(kbar) v_lm(k) with kbar_i = sin(k_i dx)/dx:
 *   type 1: n_l S_l / (N^6 dn) / (4 kappa a^(2 alpha)),  type 2: 4 pi n_l^3 (S_l/#_l) / N^6 / (4 kappa a^(2 alpha)),
 * S_l the sum over bin l of sum_ij |(Lambda H')_ij|^2, H' the unnormalised DFT of h' = a^(alpha-3) pi_v
 * (so that summing type 1 over the bins with weight dn/n_l gives rho_GW = <h'_ij h'_ij>_TT / (4 kappa a^(2 alpha))).
 * Binning and outputs as cl_spectrum.  Uses cuFFT; synchronising.  Errors: CL_EINVAL (not
 * enabled, bad arguments), CL_ECUDA, CL_ENOMEM. */
cl_status cl_gw_spectrum(cl_lattice* l, double dn, int32_t type, double* k_out, double* delta_out, double* count_out,
                         int32_t cap, int32_t* nbins);

/* When limit > 0, a Hubble violation above it sets the device status CL_ECONSTRAINT
 * (reported by the next synchronising call).  limit <= 0 disables the check (default). */
cl_status cl_set_hubble_limit(cl_lattice* l, double limit);

/* Options.  CL_OPT_GRAPH: 1 = replay steps from captured CUDA graphs (default), 0 = plain
 * launches.  CL_OPT_TILE_BY: rows per block of the fused scalar pass (0 = library
 * choice).  CL_OPT_TILE_DZ: planes per block (0 = library choice: the y tiles are cut into
 * the same z chunks so that one wave of blocks covers the lattice; -1 = a persistent grid
 * of one wave, each block a balanced contiguous range of planes; for the axion-U(1)
 * kernels, the planes of the z chunk each (x, y) tile marches through, where the staged
 * plaquette launches, whose tiles are twice as tall, split every chunk in two).  CL_OPT_STAGES: TMA stage buffers
 * of the fused pass, 2..6, or -1 for the loader without TMA staging (0 = library choice;
 * rows that are not a multiple of 16 bytes always use the loader without TMA; ensembles
 * clamp to 2..4 with the ring kernel and 3..6 ringless).  On a Runge-Kutta scalar lattice
 * the three options tile the stage kernel instead: CL_OPT_STAGES 3..6 stage buffers of the
 * TMA-staged stage kernel (2 counts as 3; -1 = the direct-load kernel), CL_OPT_TILE_BY its
 * rows per tile, CL_OPT_TILE_DZ its z chunks (0 = the library's: every y tile cut into the
 * same chunks, one wave of blocks; -1 = balanced persistent ranges).
 * CL_OPT_PASS_VARIANT (-1 = library choice, the default): TMA-staged pass kernel, 1 =
 * ringless (the library's choice: each warp drifts the neighbour rows it needs from the
 * stage buffers, no consumer barrier; 16-byte vectors, 2..5 stages (ensembles 3..6), other
 * rows fall back to 0), 0 = drifted rows shared through a ring in shared memory with one
 * consumer barrier per plane.  Both give bit-identical fields on the same tiles.  For an
 * axion-U(1) lattice, two launches per Runge-Kutta stage (plaquette fields through global
 * memory, then the stage) unless 1: 0 = every neighbour gathered from L1/L2, 2 = the
 * neighbourhoods of each plane staged in shared memory by asynchronous copies (the library's
 * choice where N is a multiple of 32, else 0), 1 = one fused launch per stage with the
 * plaquette fields in shared memory (N a multiple of 32; Runge-Kutta only, CL_EUNSUPPORTED
 * with the leapfrog), 3 = the staged neighbourhoods of 2 in one launch per stage or pass, the
 * plaquette fields computed into shared memory (N a multiple of 32).  All agree to rounding,
 * also across a change of form with the axion-U(1) leapfrog open (the first step after a
 * change to 2 adds one plaquette launch that saves sin P and cos P of the open positions,
 * which form 2 keeps from each step's first pass for its other two).  On a
 * (2+1)-dimensional lattice the leapfrog pass is 1 = row marching (the library's choice where N is a multiple of 128 in
 * FP32, 64 in FP64: each warp owns a strip of columns and a chunk of rows and keeps three
 * drifted rows in registers; CL_OPT_TILE_DZ its rows per chunk, CL_OPT_TILE_BY how many rows
 * ahead it prefetches into L2, 0 = library choice) or 0 = one thread per site; both agree to
 * rounding.
 * Errors: CL_EINVAL, CL_EUNSUPPORTED. */
enum { CL_OPT_GRAPH = 0, CL_OPT_TILE_BY = 1, CL_OPT_TILE_DZ = 2, CL_OPT_STAGES = 3, CL_OPT_PASS_VARIANT = 4 };
cl_status cl_set_option(cl_lattice* l, int32_t option, int64_t value);

/* The value in effect for an option after the library's choices: rows per tile, planes per
 * block (-1: persistent ranges), TMA stages (0: loader without TMA staging) and the pass
 * variant that the fused pass runs with.  Ensembles report member 0's tile and the ring
 * variant (0).  value: host pointer, written on success.  Errors: CL_EINVAL. */
cl_status cl_get_option(cl_lattice* l, int32_t option, int64_t* value);

/* Autotuner of the fused leapfrog pass (single lattices and ensembles, no gauge field):
 * times trial passes of candidate tilings -- TMA stage buffers (CL_OPT_STAGES), rows per tile
 * (CL_OPT_TILE_BY), planes per work unit or z chunk (CL_OPT_TILE_DZ) and, for single
 * lattices, the pass kernel (CL_OPT_PASS_VARIANT) -- and keeps the fastest.  A trial pass does the full work of a pass (drift while loading, stencil kick,
 * energies) but writes into the spare buffers and commits nothing: the state, a, a' and t are
 * unchanged.  cache_path (may be NULL): a text file of earlier choices, one JSON object per
 * line, keyed by the lattice's shape, precision and field count; a hit applies the cached
 * choice without trials, a miss appends the new one.  best (may be NULL, else 5 doubles)
 * receives the tiling then in effect (as cl_get_option reports it: stages, 0 for the loader
 * without TMA staging; tile_by; tile_dz, -1 for persistent ranges), the microseconds per trial
 * pass and the pass variant: {stages, tile_by, tile_dz, us, variant}.  Errors: CL_EINVAL (Runge-Kutta or
 * gauge lattice), CL_ESTATE (no potential), CL_ECUDA. */
cl_status cl_autotune(cl_lattice* l, const char* cache_path, double* best);

/* ---- Allocation-free pass (the paper has no counterpart; this serves callers that cannot
 * allocate device memory when they step: code inside an application that owns a fixed memory
 * arena, hosts that forbid allocation after start-up, frameworks that hand over only
 * pre-allocated buffers).
 *
 * cl_fused_pass_noalloc runs one fused pass of the same kernel cl_step uses, on device arrays
 * the caller owns, and allocates nothing: no cudaMalloc/cudaFree and no allocating library
 * call.  One pass drifts phi by `drift` (with a' and a drifted alongside), kicks pi by `kick`,
 * evaluates the energies with pi + energy_kick * F and advances a' by kick * a''.  Velocity
 * Verlet in staggered form is, with h = dt: an opening pass {0, 0, h/2}, then {h, h/2, h} per
 * step; {0, -h/2, -h/2} returns the momenta to the integer time.
 *
 * Scratch (block partials of the energy reduction, the arrival counter, the working copy of
 * a, a', t) lives in one fixed array of static device memory inside the library, 327,936
 * bytes (320 KiB), which every GPU that loads the library holds until the process exits.  It limits a
 * pass to 8192 blocks of the direct-load kernel (larger lattices march more planes per block).
 * A row of the lattice must fit one 512-thread block, as for cl_step: odd N up to 511, even N
 * up to 1024, and in FP32 multiples of 4 up to 1536; other sizes return CL_EINVAL before any
 * work is queued.  The first call on a device looks up that
 * array's device address (with the device current); make that first call before any stream
 * capture.  All calls share the array and each clears what must start at zero: calls whose
 * GPU work overlaps (other streams, other host threads) race and must be serialised by the
 * caller.  Work is queued on `stream`; the call does not synchronise.
 *
 * Arrays: N^3 elements of the precision's type (double for CL_PREC_FP64, float otherwise),
 * site index (z*N + y)*N + x; inputs and outputs must be distinct buffers; c_in/c_out (the
 * Kahan compensations) are used with CL_PREC_FP32_KAHAN only.  scalars: device, 3 doubles
 * {a, a', t}, read and then overwritten with the values after the pass.  energies: device,
 * 14 doubles {t, a, a', K0, K1, G0, G1, V, KE, GB, rho, p, hubble_violation, gauss_violation}
 * at the pass's integer time, or NULL.  status: device, one int32 or NULL; receives the pass's
 * status bits (1: a non-finite energy, as CL_ENAN reports for cl_step).  The call queues work
 * and returns before it runs, so it cannot report that condition itself: read status (or check
 * that energies[rho] is finite) after the stream has run.  Every array must be device (or
 * managed) memory of the current device; no output may overlap an input or another output.
 * Errors: CL_EINVAL (bad descriptor, host pointer, overlapping arrays), CL_ECUDA. */
typedef struct {
    int32_t N, nfields, precision, expansion;
    double L, alpha, kappa;
    double m2[2], lam[2], g2;           /* potential, as for CL_POT_POLY */
    double drift, energy_kick, kick;    /* pass coefficients, already multiplied by dt */
    const void* phi_in[2];
    const void* pi_in[2];
    const void* c_in[2];
    void* phi_out[2];
    void* pi_out[2];
    void* c_out[2];
    double* scalars;
    double* energies;
    void* stream;                       /* cudaStream_t, NULL = legacy default stream */
    int32_t* status;                    /* device, optional: status bits of the pass */
} cl_pass_noalloc_desc;
cl_status cl_fused_pass_noalloc(const cl_pass_noalloc_desc* d);

/* Number of kernel launches queued by the most recent cl_step (graph replays count the
 * kernels inside the graph). */
int64_t cl_last_launch_count(const cl_lattice* l);

const char* cl_strerror(cl_status s);
const char* cl_last_error(const cl_lattice* l);

/* ------------------------------------------------------------------------------------
 * Convolutional surrogate: a learned jump of the lattice state by a fixed number of
 * leapfrog steps (the neural operator of the build's scope; the paper defines no learned
 * component).  A stack of `layers` periodic 3x3x3 convolutions on an N^3 lattice:
 *     h_0 = x,   h_{l+1} = act(conv_l(h_l))  (l < layers-1),
 *     y = x[:, :out_channels] + conv_{layers-1}(h_{layers-1})          (residual jump)
 * with conv_l(h)[n][co] = b_l[co] + sum_t sum_ci W_l[t][co][ci] h[n + o(t)][ci], tap
 * t = (tz*3 + ty)*3 + tx at offset o(t) = (tx-1, ty-1, tz-1), periodic boundaries.
 * Arrays are site-major with channels contiguous: x[n * in_channels + c], site
 * n = (z*N + y)*N + x.  Weights W_l are FP32 [27][cout][cin], biases FP32 [cout].
 *
 * Precision CL_SG_BF16: every layer runs on the tensor cores (tcgen05, BF16 operands, FP32
 * accumulation); the thin first and last layers are zero-padded to 16 channels, the FP32
 * input is rounded to BF16 as it is staged, hidden activations are stored in BF16 and the
 * last layer writes FP32 with the residual; the backward pass computes the data gradients
 * and the weight and bias gradients on the tensor cores too.  N must be a multiple of 16.
 * CL_SG_FP32: every layer on CUDA cores in FP32 (reference mode).
 * The handle owns all device memory; calls are ordered on its stream and synchronise
 * when they copy to or from host memory. */
enum { CL_ACT_RELU = 1, CL_ACT_GELU = 2 };
enum { CL_SG_BF16 = 0, CL_SG_FP32 = 1 };

typedef struct cl_surrogate cl_surrogate;

typedef struct {
    int32_t N;             /* sites per side                                              */
    int32_t in_channels;   /* 1..3, e.g. phi, pi and a constant channel carrying a         */
    int32_t out_channels;  /* 1..in_channels; the residual adds the first ones             */
    int32_t hidden;        /* hidden width: 16, 32 or 48                                   */
    int32_t layers;        /* convolutions, >= 2                                           */
    int32_t activation;    /* CL_ACT_RELU or CL_ACT_GELU (tanh form)                       */
    int32_t precision;     /* CL_SG_BF16 or CL_SG_FP32                                     */
    int32_t reserved;      /* must be 0                                                    */
    void* stream;          /* cudaStream_t for all work of the handle; NULL = own stream    */
} cl_surrogate_params;

/* Errors: CL_EINVAL (sizes, enums), CL_ENOMEM, CL_ECUDA.  Weights start at zero. */
cl_status cl_surrogate_create(cl_surrogate** out, const cl_surrogate_params* p);
void cl_surrogate_free(cl_surrogate* s);
/* Copy layer `layer`'s weights W [27][cout][cin] and bias b [cout] (host FP32) in or out. */
cl_status cl_surrogate_set_weights(cl_surrogate* s, int32_t layer, const float* W, const float* b);
cl_status cl_surrogate_get_weights(cl_surrogate* s, int32_t layer, float* W, float* b);
/* y = network(x): x holds N^3 * in_channels FP32 values, y N^3 * out_channels, both in host
 * memory (on_device = 0) or device memory (1).  Keeps the activations for a backward call. */
cl_status cl_surrogate_forward(cl_surrogate* s, const float* x, float* y, int32_t on_device);
/* Gradients of sum(y * g) for the last forward's input: g holds N^3 * out_channels FP32
 * values (NULL: the gradient left by cl_surrogate_loss); dx (N^3 * in_channels, may be NULL)
 * receives d/dx.  Weight and bias gradients stay
 * on the device (cl_surrogate_get_grads).  Errors: CL_ESTATE without a preceding forward. */
cl_status cl_surrogate_backward(cl_surrogate* s, const float* g, float* dx, int32_t on_device);
cl_status cl_surrogate_get_grads(cl_surrogate* s, int32_t layer, float* dW, float* db);
/* Kernel launches queued by the most recent forward or backward call. */
int64_t cl_surrogate_last_launch_count(const cl_surrogate* s);

/* Training loss of the most recent forward:
 *     L = mean over sites n and output channels c of ((y[n][c] - target[n*stride + c]) / scale[c])^2
 * (scale NULL: 1).  Keeps dL/dy as the output gradient of a following
 * cl_surrogate_backward(s, NULL, ...) and writes L to *loss (synchronising).  target in
 * device (on_device = 1) or host memory; stride >= out_channels.
 * Errors: CL_EINVAL, CL_ESTATE (no forward yet), CL_ECUDA. */
cl_status cl_surrogate_loss(cl_surrogate* s, const float* target, int32_t stride, const float* scale,
                            int32_t on_device, double* loss);
/* One AdamW step (Loshchilov & Hutter, decoupled weight decay) on every layer with the
 * gradients of the most recent backward: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * W -= lr (m/(1-b1^t) / (sqrt(v/(1-b2^t)) + eps) + weight_decay W); biases without decay;
 * t = 1, 2, ...  Rebuilds the tensor-core weight layouts on the device.  Errors: CL_EINVAL. */
cl_status cl_surrogate_adamw(cl_surrogate* s, double lr, double beta1, double beta2, double eps, double weight_decay,
                             int64_t t);
/* Mean and standard deviation (population) of each of the `channels` (<= 3) columns of the
 * device array x (n rows); results to host arrays.  Synchronising. */
cl_status cl_surrogate_channel_stats(cl_surrogate* s, const float* x_dev, int64_t n, int32_t channels, float* mean,
                                     float* stdev);

/* Lattice <-> network (single FP32 lattice, one scalar field, N^3 sites = the network's N).
 * cl_lattice_pack writes x[n] = ((phi - mu[0])/sg[0], (pi - mu[1])/sg[1], (a - mu[2])/sg[2])
 * at the most recent integer time into the device array x (N^3 x 3); cl_lattice_unpack sets
 * phi = mu[0] + sg[0] y[n][0], pi = mu[1] + sg[1] y[n][1] from the device array y (N^3 x 2)
 * (Kahan compensation restarts at zero; a, a', t unchanged).  Errors: CL_EINVAL. */
cl_status cl_lattice_pack(cl_lattice* l, const float* mu, const float* sg, float* x_dev);
cl_status cl_lattice_unpack(cl_lattice* l, const float* mu, const float* sg, const float* y_dev);

/* Advance the lattice by `steps` time steps with one surrogate forward (the learned jump):
 * (phi, pi) from the network applied to the packed state (normalisation mu, sg as above),
 * a and a' advanced over the jump J = steps * dt with a'' of the starting state,
 * a += J a' + J^2 a''/2, a' += J a'' (Eq. Friedmann1).  The jump is accepted when the Hubble
 * violation (Eq. Friedmann2) of the new state is finite and at most hubble_limit; otherwise
 * the starting state is restored and `steps` leapfrog steps of the lattice's integrator are
 * taken instead (the fallback).  *accepted = 1 or 0.  The network needs in_channels 3 and
 * out_channels 2.  Synchronising.  Errors: CL_EINVAL (shapes, precision), CL_ECUDA. */
cl_status cl_surrogate_jump(cl_surrogate* s, cl_lattice* l, int32_t steps, const float* mu, const float* sg,
                            double hubble_limit, int32_t* accepted);
/* Side of the network's lattice (for callers combining a surrogate with a lattice). */
int32_t cl_surrogate_size(const cl_surrogate* s);

#ifdef __cplusplus
}
#endif
#endif /* CL_H */
