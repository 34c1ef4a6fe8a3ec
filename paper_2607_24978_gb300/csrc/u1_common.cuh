// Scale-factor epilogue of the axion-U(1) Runge-Kutta stage, run by one thread of the last
// block to arrive (u1_stage.cu, u1_fused.cu): from the lattice sums w = {sum pi^2,
// sum (grad phi)^2, sum V, sum E^2, sum 2 sin^2(P/2)} of the old state it forms the
// volume averages (Eq. energy-contrib with the EM terms of Eq. AxionInfEOM's energy), writes
// the diagnostics and, unless the pass only measures energies, advances a and a' by the
// stage (k <- A k + h F, y <- y + B k) and the time.
#pragma once

#include <math.h>

#include "cl_internal.cuh"
#include "kernel_common.cuh"

namespace clk {

// Per-step Gauss tracking: from gsum = sum_n (dx G(n))^2, the squared lattice Gauss charge
// of the step's starting state (G = sum_i [P_i(n) - P_i(n - i)] / dx, P = a^(1-alpha) E + g W),
// and e2sum = sum_n sum_i E_i(n)^2, the rms violation relative to the electric term,
//     r = sqrt(gsum) / (a^(1-alpha) sqrt(e2sum))      (0 when gsum = 0),
// stored as the latest value and folded into the running maximum.  One thread.
__device__ __forceinline__ void u1_gauss_track(DevScal* S, double gsum, double e2sum, double ca)
{
    const double r = gsum > 0.0 ? sqrt(gsum) / (ca * sqrt(e2sum)) : 0.0;
    S->gauss[0] = r;
    S->gauss[1] = fmax(S->gauss[1], r);
}

template <typename T>
__device__ __forceinline__ void u1_epilogue(const U1Args<T>& A, const double (&w)[kMaxQ], double a_old, bool first,
                                            bool update, bool expand, uint32_t V)
{
    const double a = a_old;
    DevScal* S = A.scal;
    const double vol = (double)V;
    const double b = expand ? S->b : 0.0;
    const double a2 = a * a, a4 = a2 * a2, a6 = a4 * a2;
    const double K = w[0] / (2.0 * a6 * vol);
    const double G = w[1] / (A.dx * A.dx * 2.0 * a2 * vol);
    const double Vp = w[2] / vol;
    const double KE = A.ws2 * w[3] / (2.0 * apow(a, 2.0 + 2.0 * A.alpha) * vol);
    const double GB = A.ws2 * w[4] / (apow(A.dx, 4.0) * a4 * vol);
    const double rho = K + G + Vp + KE + GB;
    const double p = K - G / 3.0 - Vp + (KE + GB) / 3.0;
    const double a2al = apow(a, 2.0 * A.alpha);
    double bb = b;
    if ((A.flags & P_HUBBLE_INIT) && expand) bb = a * sqrt(a2al * A.kappa * rho / 3.0);
    const double H = bb / a;
    const double hv = H != 0.0 ? fabs(H * H - a2al * A.kappa * rho / 3.0) / (H * H) : 0.0;
    S->diag[D_T] = S->t;
    S->diag[D_A] = a;
    S->diag[D_ADOT] = bb;
    S->diag[D_K0] = K;
    S->diag[D_K1] = 0.0;
    S->diag[D_G0] = G;
    S->diag[D_G1] = 0.0;
    S->diag[D_V] = Vp;
    S->diag[D_KE] = KE;
    S->diag[D_GB] = GB;
    S->diag[D_RHO] = rho;
    S->diag[D_P] = p;
    S->diag[D_HV] = hv;
    if (A.flags & P_HUBBLE_INIT) S->b = bb;
    if (update && expand) {
        const double Fa = b;
        const double Fb = apow(a, 2.0 * A.alpha + 1.0) * (A.kappa / 6.0) * ((2.0 * A.alpha - 1.0) * rho - 3.0 * p);
        const double ka = first ? A.h * Fa : A.A * S->rk[0] + A.h * Fa;
        const double kb = first ? A.h * Fb : A.A * S->rk[1] + A.h * Fb;
        S->rk[0] = ka;
        S->rk[1] = kb;
        S->a = a + A.B * ka;
        S->b = b + A.B * kb;
    }
    if (update && (A.flags & P_COUNT_STEP)) {
        S->t += A.h;
        S->step += 1;
    }
    int st = 0;
    if (!isfinite(rho) || !isfinite(p)) st |= ST_NAN;
    if (first && A.hubble_limit > 0.0 && hv > A.hubble_limit) st |= ST_CONSTRAINT;
    if (st) atomicOr(&S->status, st);
    S->counter = 0u;
}

// Epilogue of a leapfrog pass (U1Args::lf), one thread of the last block.  Pass 1 (the
// closing half-kick of a step merged with the first evaluation of the next step's implicit
// kick) turns the sums w of the integer-time state into the diagnostics, with
// a'_n = a' + le a''(a, rho, p), and kicks the stored a' by lb a''; pass 3 drifts
// a by h a' and counts the step.
template <typename T>
__device__ __forceinline__ void u1_lf_epilogue(const U1Args<T>& A, const double (&w)[kMaxQ], double a, bool expand,
                                               uint32_t V)
{
    DevScal* S = A.scal;
    if (A.lf == 1) {
        const double vol = (double)V;
        const double b = expand ? S->b : 0.0;
        const double a2 = a * a, a4 = a2 * a2, a6 = a4 * a2;
        const double K = w[0] / (2.0 * a6 * vol);
        const double G = w[1] / (A.dx * A.dx * 2.0 * a2 * vol);
        const double Vp = w[2] / vol;
        const double KE = A.ws2 * w[3] / (2.0 * apow(a, 2.0 + 2.0 * A.alpha) * vol);
        const double GB = A.ws2 * w[4] / (apow(A.dx, 4.0) * a4 * vol);
        const double rho = K + G + Vp + KE + GB;
        const double p = K - G / 3.0 - Vp + (KE + GB) / 3.0;
        const double a2al = apow(a, 2.0 * A.alpha);
        const double Fb = expand ? apow(a, 2.0 * A.alpha + 1.0) * (A.kappa / 6.0) * ((2.0 * A.alpha - 1.0) * rho - 3.0 * p)
                                 : 0.0;
        const double bn = b + A.le * Fb;
        const double H = bn / a;
        const double hv = H != 0.0 ? fabs(H * H - a2al * A.kappa * rho / 3.0) / (H * H) : 0.0;
        S->diag[D_T] = S->t;
        S->diag[D_A] = a;
        S->diag[D_ADOT] = bn;
        S->diag[D_K0] = K;
        S->diag[D_K1] = 0.0;
        S->diag[D_G0] = G;
        S->diag[D_G1] = 0.0;
        S->diag[D_V] = Vp;
        S->diag[D_KE] = KE;
        S->diag[D_GB] = GB;
        S->diag[D_RHO] = rho;
        S->diag[D_P] = p;
        S->diag[D_HV] = hv;
        if (expand) S->b = b + A.lb * Fb;
        int st = 0;
        if (!isfinite(rho) || !isfinite(p)) st |= ST_NAN;
        if (A.hubble_limit > 0.0 && hv > A.hubble_limit) st |= ST_CONSTRAINT;
        if (st) atomicOr(&S->status, st);
    } else if (A.lf == 3) {
        if (expand) S->a = a + A.h * S->b;
        S->t += A.h;
        S->step += 1;
    }
    S->counter = 0u;
}

// Drift coefficient of leapfrog pass 3: h ((a + a_1)/2)^(alpha-3), a_1 = a + h a'.
__device__ __forceinline__ double u1_lf_drift(double a, double b, double h, double alpha)
{
    const double a1 = a + h * b;
    return h * apow(0.5 * (a + a1), alpha - 3.0);
}

}  // namespace clk
