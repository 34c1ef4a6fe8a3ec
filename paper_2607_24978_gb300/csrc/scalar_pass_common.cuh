// Per-site arithmetic of the fused scalar pass, shared by the single-lattice kernels
// (scalar_pass.cu, scalar_pass_tma.cuh) and the ensemble kernel (ensemble_pass.cu):
// the pass prefactors, the stencil kick of one row vector, the direct-loader march over
// one tile, and the scale-factor epilogue run by the last block of a lattice.
#pragma once

#include <math.h>

#include "cl_internal.cuh"
#include "kernel_common.cuh"

namespace clk {

// Scalar prefactors of a pass, computed once per block (or work item) by thread 0.
__device__ __forceinline__ void pass_coefficients(const double a_old, const double b_old, const double d,
                                                  const double alpha, const double dx, const bool expand,
                                                  double* s_coef)
{
    const double a_new = expand ? a_old + d * b_old : a_old;
    const double ah = 0.5 * (a_old + a_new);
    s_coef[0] = d * apow(ah, alpha - 3.0);
    s_coef[1] = apow(a_new, 1.0 + alpha) / (dx * dx);
    s_coef[2] = apow(a_new, 3.0 + alpha);
    s_coef[3] = a_new;
}

// The same prefactors computed by lanes 0 of warps 0, 1 and 2 at once (one pow each):
// for kernels that evaluate them once per work item.  Needs at least 65 threads.
__device__ __forceinline__ void pass_coefficients_warps(int tid, const double a_old, const double b_old,
                                                        const double d, const double alpha, const double dx,
                                                        const bool expand, double* s_coef)
{
    if (tid != 0 && tid != 32 && tid != 64) return;
    const double a_new = expand ? a_old + d * b_old : a_old;
    if (tid == 0) {
        s_coef[0] = d * apow(0.5 * (a_old + a_new), alpha - 3.0);
        s_coef[3] = a_new;
    } else if (tid == 32) {
        s_coef[1] = apow(a_new, 1.0 + alpha) / (dx * dx);
    } else {
        s_coef[2] = apow(a_new, 3.0 + alpha);
    }
}

// Kick of one own-row vector of a plane.  S*[f] point at row (r+1) of the centre
// (Sc), lower (Szm) and upper (Szp) planes of field f; rows r and r+2 of the
// centre plane are Sc -/+ N.  Writes pi_out and accumulates K, G, V.
//
// SBP (used by the FP64 direct-load pass, whose speed is set by GB300's FP64 rate, not
// by memory): fewer FP64 operations for the same quantities.  The gradient sum
// sum_n sum_i (phi(n+i) - phi(n))^2 equals -sum_n phi(n) Lap phi(n) dx^2 on the periodic
// lattice (summation by parts), and sum_n Lap phi(n) = 0, so it is accumulated as
// sum_n (C - phi(n)) Lap phi(n) dx^2 with a constant C that every block of the lattice
// takes the same (gC[f]: the drifted field at site 0); subtracting C keeps the products
// small, so the rounding of Lap phi does not swamp the sum.  The potential and its
// derivatives are evaluated in Horner form on phi^2.
template <typename T, int NF, int VW, bool SBP = false>
__device__ __forceinline__ void kick_vector(const T* const (&Sc)[NF], const T* const (&Szm)[NF],
                                            const T* const (&Szp)[NF], int N, int x0, const T (&pin)[NF][VW],
                                            const T cL, const T cV, const T ce, const T ck, const PotCoef<T>& P,
                                            T* const* pi_out, size_t base, Acc<T> (&accK)[NF],
                                            Acc<T> (&accG)[NF], Acc<T>& accV, const T* gC = nullptr)
{
    T phc[NF][VW], lap[NF][VW];
    if constexpr (SBP) {
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            T c[VW], ym[VW], yp[VW], zm[VW], zp[VW];
            vload_smem<T, VW>(c, Sc[f] + x0);
            vload_smem<T, VW>(ym, Sc[f] - N + x0);
            vload_smem<T, VW>(yp, Sc[f] + N + x0);
            vload_smem<T, VW>(zm, Szm[f] + x0);
            vload_smem<T, VW>(zp, Szp[f] + x0);
            const T xm_edge = Sc[f][x0 == 0 ? N - 1 : x0 - 1];
            const T xp_edge = Sc[f][x0 + VW == N ? 0 : x0 + VW];
            const T Cf = gC[f];
            T g = (T)0;
#pragma unroll
            for (int i = 0; i < VW; ++i) {
                const T xm = i == 0 ? xm_edge : c[i - 1];
                const T xp = i == VW - 1 ? xp_edge : c[i + 1];
                lap[f][i] = ((xp + xm) + (yp[i] + ym[i]) + (zp[i] + zm[i])) - (T)6 * c[i];
                g = fma_rn(Cf - c[i], lap[f][i], g);
                phc[f][i] = c[i];
            }
            accG[f].add(g);
        }
        T vsum = (T)0;
        T dV[NF][VW];
#pragma unroll
        for (int i = 0; i < VW; ++i) {
            const T p0 = phc[0][i], P0 = p0 * p0;
            if constexpr (NF > 1) {
                const T p1 = phc[NF - 1][i], P1 = p1 * p1;
                dV[0][i] = p0 * fma_rn(P.l0, P0, fma_rn(P.g2, P1, P.m20));
                dV[NF - 1][i] = p1 * fma_rn(P.l1, P1, fma_rn(P.g2, P0, P.m21));
                vsum += fma_rn(P0, fma_rn(P.q_l0, P0, P.h_m20), P1 * fma_rn(P.q_l1, P1, fma_rn(P.h_g2, P0, P.h_m21)));
            } else {
                dV[0][i] = p0 * fma_rn(P.l0, P0, P.m20);
                vsum += P0 * fma_rn(P.q_l0, P0, P.h_m20);
            }
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            T po[VW], ksum = (T)0;
#pragma unroll
            for (int i = 0; i < VW; ++i) {
                const T F = cL * lap[f][i] - cV * dV[f][i];
                const T pe = pin[f][i] + ce * F;
                po[i] = pin[f][i] + ck * F;
                ksum += pe * pe;
            }
            accK[f].add(ksum);
            vstore<T, VW>(pi_out[f] + base, po);
        }
        accV.add(vsum);
        return;
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        T c[VW], ym[VW], yp[VW], zm[VW], zp[VW];
        vload_smem<T, VW>(c, Sc[f] + x0);
        vload_smem<T, VW>(ym, Sc[f] - N + x0);
        vload_smem<T, VW>(yp, Sc[f] + N + x0);
        vload_smem<T, VW>(zm, Szm[f] + x0);
        vload_smem<T, VW>(zp, Szp[f] + x0);
        const T xm_edge = Sc[f][x0 == 0 ? N - 1 : x0 - 1];
        const T xp_edge = Sc[f][x0 + VW == N ? 0 : x0 + VW];
        T g = (T)0;
#pragma unroll
        for (int i = 0; i < VW; ++i) {
            const T xm = i == 0 ? xm_edge : c[i - 1];
            const T xp = i == VW - 1 ? xp_edge : c[i + 1];
            lap[f][i] = ((xp + xm) + (yp[i] + ym[i]) + (zp[i] + zm[i])) - (T)6 * c[i];
            const T gx = xp - c[i], gy = yp[i] - c[i], gz = zp[i] - c[i];
            g += gx * gx + gy * gy + gz * gz;
            phc[f][i] = c[i];
        }
        accG[f].add(g);
    }
    T vsum = (T)0;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        T po[VW], ksum = (T)0;
#pragma unroll
        for (int i = 0; i < VW; ++i) {
            const T p0 = phc[0][i];
            const T p1 = NF > 1 ? phc[NF - 1][i] : (T)0;
            T dV;
            if (f == 0) dV = p0 * (P.m20 + P.l0 * p0 * p0 + (NF > 1 ? P.g2 * p1 * p1 : (T)0));
            else dV = p1 * (P.m21 + P.l1 * p1 * p1 + P.g2 * p0 * p0);
            const T F = cL * lap[f][i] - cV * dV;
            const T pe = pin[f][i] + ce * F;
            po[i] = pin[f][i] + ck * F;
            ksum += pe * pe;
            if (f == 0) {
                T v = p0 * p0 * (P.h_m20 + P.q_l0 * p0 * p0);
                if (NF > 1) v += p1 * p1 * (P.h_m21 + P.q_l1 * p1 * p1) + P.h_g2 * p0 * p0 * p1 * p1;
                vsum += v;
            }
        }
        accK[f].add(ksum);
        vstore<T, VW>(pi_out[f] + base, po);
    }
    accV.add(vsum);
}

// Array bases of one lattice: read from the `in` buffers, written to the `out` buffers.
template <typename T>
struct FieldSet {
    const T* phi_in[2];
    const T* pi_in[2];
    const T* c_in[2];
    T* phi_out[2];
    T* pi_out[2];
    T* c_out[2];
};

// Pass coefficients of one tile in the element type.
template <typename T>
struct TileCoef {
    T cd, cL, cV, ce, ck;
};

// Direct-loader march over one tile: rows y0 .. y0+R-1 (R <= BY) of the planes
// z0 .. z0+NZ-1 of an N^3 lattice.  A three-slot ring in shared memory (`sm`: NF fields
// x 3 slots x (BY+2) rows x N) holds the drifted field of the planes below, at and above
// the plane being kicked; thread tid < BY*(N/VW) owns one row vector.  Every output is
// written once; loads of the halo rows (and planes) are the only re-reads.  Ends with a
// block barrier, so the ring may be refilled at once.
template <typename T, int NF, bool KAHAN, int VW, bool SBP = false>
__device__ __forceinline__ void march_tile(const FieldSet<T>& F, int N, int BY, int y0, int R, int z0, int NZ,
                                           T* sm, int tid, int nthr, bool do_drift, const TileCoef<T>& C,
                                           const PotCoef<T>& P, Acc<T> (&accK)[NF], Acc<T> (&accG)[NF],
                                           Acc<T>& accV, const T* gC = nullptr)
{
    const int TX = N / VW;
    const int r = tid < BY * TX ? tid / TX : BY, tx = tid < BY * TX ? tid % TX : 0;
    const int slot_stride = (BY + 2) * N, field_stride = 3 * slot_stride;
    const int x0 = tx * VW;

    auto fill = [&](int zrel, int slot, bool write_out, T(&pin)[NF][VW]) {
        int zz = z0 + zrel;
        zz = zz < 0 ? zz + N : (zz >= N ? zz - N : zz);
        if (r < R) {
            const size_t base = ((size_t)zz * N + (y0 + r)) * N + x0;
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                T ph[VW], pv[VW], cv[VW];
                vload<T, VW>(ph, F.phi_in[f] + base);
                vload<T, VW>(pv, F.pi_in[f] + base);
                if (KAHAN) vload<T, VW>(cv, F.c_in[f] + base);
                if (do_drift) {
#pragma unroll
                    for (int i = 0; i < VW; ++i) drift<T, KAHAN>(ph[i], cv[i], pv[i], C.cd);
                }
                vstore<T, VW>(sm + f * field_stride + slot * slot_stride + (r + 1) * N + x0, ph);
                if (write_out) {
                    vstore<T, VW>(F.phi_out[f] + base, ph);
                    if (KAHAN) vstore<T, VW>(F.c_out[f] + base, cv);
                }
#pragma unroll
                for (int i = 0; i < VW; ++i) pin[f][i] = pv[i];
            }
        }
        for (int h = tid; h < 2 * TX; h += nthr) {
            const int sel = h / TX, vx = (h - sel * TX) * VW;
            int y = sel == 0 ? y0 - 1 : y0 + R;
            y = y < 0 ? y + N : (y >= N ? y - N : y);
            const int srow = sel == 0 ? 0 : R + 1;
            const size_t base = ((size_t)zz * N + y) * N + vx;
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                T ph[VW], pv[VW], cv[VW];
                vload<T, VW>(ph, F.phi_in[f] + base);
                if (do_drift) {
                    vload<T, VW>(pv, F.pi_in[f] + base);
                    if (KAHAN) vload<T, VW>(cv, F.c_in[f] + base);
#pragma unroll
                    for (int i = 0; i < VW; ++i) drift<T, KAHAN>(ph[i], cv[i], pv[i], C.cd);
                }
                vstore<T, VW>(sm + f * field_stride + slot * slot_stride + srow * N + vx, ph);
            }
        }
    };

    T pcur[NF][VW], pnext[NF][VW];
    fill(-1, 0, false, pnext);
    fill(0, 1, true, pcur);
    for (int zr = 0; zr < NZ; ++zr) {
        const int sl = zr % 3, sc = (zr + 1) % 3, su = (zr + 2) % 3;
        fill(zr + 1, su, zr + 1 < NZ, pnext);
        __syncthreads();
        if (r < R) {
            const T* Sc[NF];
            const T* Szm[NF];
            const T* Szp[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                Sc[f] = sm + f * field_stride + sc * slot_stride + (r + 1) * N;
                Szm[f] = sm + f * field_stride + sl * slot_stride + (r + 1) * N;
                Szp[f] = sm + f * field_stride + su * slot_stride + (r + 1) * N;
            }
            const size_t base = ((size_t)(z0 + zr) * N + (y0 + r)) * N + x0;
            kick_vector<T, NF, VW, SBP>(Sc, Szm, Szp, N, x0, pcur, C.cL, C.cV, C.ce, C.ck, P, F.pi_out, base, accK,
                                        accG, accV, gC);
        }
#pragma unroll
        for (int f = 0; f < NF; ++f)
#pragma unroll
            for (int i = 0; i < VW; ++i) pcur[f][i] = pnext[f][i];
        __syncthreads();
    }
}

// Energies of a pass from the lattice sums w (sum pi_int^2 per field, sum (grad+ phi)^2
// per field, sum V), its diagnostics, and the update of a, a' and t (Eq. Friedmann1,
// Eq. Friedmann2, Eq. energy-contrib).  One thread; clears the arrival counter.
__device__ inline void scalar_epilogue(DevScal* S, const double (&w)[kMaxQ], double vol, double dx, double a,
                                       double alpha, double kappa, double d, double e, double k, int flags,
                                       double hubble_limit)
{
    // reciprocals once: FP64 divisions are long dependent chains on GB300's FP64 pipe, and this
    // runs on one thread at the end of every pass
    constexpr double third = 1.0 / 3.0, sixth = 1.0 / 6.0;
    const double ivol = 1.0 / vol, ia = 1.0 / a, ia2 = ia * ia, ia6 = ia2 * ia2 * ia2;
    const double ck = 0.5 * ia6 * ivol, cg = 0.5 * ia2 * ivol / (dx * dx);
    const double K0 = w[0] * ck, K1 = w[1] * ck;
    const double G0 = w[2] * cg, G1 = w[3] * cg;
    const double Vp = w[4] * ivol;
    const double K = K0 + K1, G = G0 + G1;
    const double rho = K + G + Vp;
    const double p = K - G * third - Vp;
    const bool expand = (flags & P_EXPANSION) != 0;
    const double a2al = apow(a, 2.0 * alpha);
    double b = S->b;
    if ((flags & P_HUBBLE_INIT) && expand) b = a * sqrt(a2al * kappa * rho * third);
    const double addot = expand ? a2al * a * (kappa * sixth) * ((2.0 * alpha - 1.0) * rho - 3.0 * p) : 0.0;
    const double b_int = b + e * addot;
    const double H = b_int * ia;
    const double hv = H != 0.0 ? fabs(H * H - a2al * kappa * rho * third) / (H * H) : 0.0;
    const double t_int = S->t + d;
    if (flags & P_COMMIT) {
        S->a_prev = S->a;
        S->a = a;
        S->b = b + k * addot;
        S->t = t_int;
        if (flags & P_COUNT_STEP) S->step += 1;
    }
    S->diag[D_T] = t_int;
    S->diag[D_A] = a;
    S->diag[D_ADOT] = b_int;
    S->diag[D_K0] = K0;
    S->diag[D_K1] = K1;
    S->diag[D_G0] = G0;
    S->diag[D_G1] = G1;
    S->diag[D_V] = Vp;
    S->diag[D_KE] = 0.0;
    S->diag[D_GB] = 0.0;
    S->diag[D_RHO] = rho;
    S->diag[D_P] = p;
    S->diag[D_HV] = hv;
    S->diag[D_GV] = 0.0;
    int st = 0;
    if (!isfinite(rho) || !isfinite(p)) st |= ST_NAN;
    if (hubble_limit > 0.0 && hv > hubble_limit) st |= ST_CONSTRAINT;
    if (st) atomicOr(&S->status, st);
    S->counter = 0u;
}

}  // namespace clk
