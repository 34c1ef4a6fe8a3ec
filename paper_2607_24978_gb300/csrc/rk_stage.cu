// One stage of a low-storage (2N) Runge-Kutta scheme for the scalar fields and the
// scale factor (section "Non-symplectic evolvers"; RK3-3 of Williamson 1980 and RK4-5
// of Carpenter & Kennedy 1994).  For the state y = (phi, pi, a, a') with
//
//   F(y) = (a^(alpha-3) pi,  a^(1+alpha) Lap phi - a^(3+alpha) dV/dphi,  a',  a''(a, rho(y), p(y)))
//
// a stage does  k <- A k + h F(y);  y <- y + B k  with one auxiliary array per field
// degree of freedom.  The field part is one launch: each site needs the 7-point
// stencil of the old phi only, so a block marches up z with a three-plane ring of the
// old field in shared memory (full x rows, BY rows plus one halo row each side) and
// reads pi, k_phi, k_pi (and the Kahan compensation of phi) of its own sites straight
// from global memory.  The same launch reduces the volume-averaged energies of the old
// state (FP64 across threads and blocks, fixed order), and the last block to arrive
// uses them for the a' component of F, advancing a, a' and their own k values.  The
// first stage (A = 0) does not read k.  Inputs and outputs are ping-pong buffers.
#include <math.h>

#include "cl_internal.cuh"
#include "kernel_common.cuh"
#include "rk_tma.cuh"

namespace clk {

// Block partials of the old state's energy sums v (K_0, K_1, G_0, G_1, V), then the last
// block to arrive: volume averages, diagnostics, and the (a, a') part of the stage.
// With v2 (sums of pi^2, (grad+ phi)^2, V, phi V', phi^2 of the stage's output state, field 0),
// the last block also writes the background Ricci scalar of that state to scal->rbar, after
// the stage used the one of its input state (partials of v2 after those of v).
template <typename T>
// With P_RK_ERROR, v2 instead carries the sums |B k|^2 and |y|^2 over the degrees of freedom of
// the last stage (adaptive RK3-4): the last block sets the next step size from their ratio.
// h: the step size of this stage.
// acc / acc2: the thread's accumulators of the sums (nullptr: none; acc2 nullptr: no v2).
__device__ __forceinline__ void rk_finish(const RkStageArgs<T>& A, const Acc<T>* const (&acc)[kMaxQ], double a_old,
                                          double h, bool first, double (*s_red)[kMaxQ], int* s_last, int tid, int nthr,
                                          const Acc<T>* const (*acc2)[kMaxQ] = nullptr, int dims = 3)
{
    const int N = A.N;
    double v[kMaxQ], v2b[kMaxQ];
    double (*v2)[kMaxQ] = acc2 ? &v2b : nullptr;
    block_reduce_acc<T, kMaxQ>(acc, v, s_red, tid, nthr);
    if (acc2) block_reduce_acc<T, kMaxQ>(*acc2, v2b, s_red, tid, nthr);
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < kMaxQ; ++q) A.partials[(size_t)blockIdx.x * kMaxQ + q] = v[q];
        if (v2)
#pragma unroll
            for (int q = 0; q < kMaxQ; ++q) A.partials[((size_t)gridDim.x + blockIdx.x) * kMaxQ + q] = (*v2)[q];
        __threadfence();
        const unsigned prev = atomicAdd(&A.scal->counter, 1u);
        *s_last = (prev + 1u == gridDim.x);
    }
    __syncthreads();
    if (!*s_last) return;
    __threadfence();
    if (tid >= 32) return;  // one warp sums the grid's partials, its lane 0 runs the epilogue
    double w[kMaxQ];
    warp_sum_partials<kMaxQ>(A.partials, (int)gridDim.x, tid, w);
    double w2[kMaxQ] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (v2) warp_sum_partials<kMaxQ>(A.partials + (size_t)gridDim.x * kMaxQ, (int)gridDim.x, tid, w2);
    if (tid == 0) {
        DevScal* S = A.scal;
        const double vol = dims == 1 ? (double)N : (dims == 2 ? (double)N * N : (double)N * N * N);
        const double a = a_old, b = S->b;
        const double a2 = a * a, a6 = a2 * a2 * a2;
        const double K0 = w[0] / (2.0 * a6 * vol), K1 = w[1] / (2.0 * a6 * vol);
        const double G0 = w[2] / (A.dx * A.dx * 2.0 * a2 * vol), G1 = w[3] / (A.dx * A.dx * 2.0 * a2 * vol);
        const double Vp = w[4] / vol;
        const double K = K0 + K1, G = G0 + G1;
        const double rho = K + G + Vp, p = K - G / 3.0 - Vp;
        const bool expand = (A.flags & P_EXPANSION) != 0;
        const double a2al = apow(a, 2.0 * A.alpha);
        const double H = b / a;
        const double hv = H != 0.0 ? fabs(H * H - a2al * A.kappa * rho / 3.0) / (H * H) : 0.0;
        S->diag[D_T] = S->t;
        S->diag[D_A] = a;
        S->diag[D_ADOT] = b;
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
        if (expand) {
            const double Fa = b;
            // Eq. Friedmann1, or for a non-minimally coupled field Eq. piadot with R of the state
            const double Fb = A.nmc ? a * (apow(a, 2.0 * A.alpha) * S->rbar / 6.0 - (1.0 - A.alpha) * (b / a) * (b / a))
                                    : apow(a, 2.0 * A.alpha + 1.0) * (A.kappa / 6.0) * ((2.0 * A.alpha - 1.0) * rho - 3.0 * p);
            const double ka = first ? h * Fa : A.A * S->rk[0] + h * Fa;
            const double kb = first ? h * Fb : A.A * S->rk[1] + h * Fb;
            S->rk[0] = ka;
            S->rk[1] = kb;
            S->a = a + A.B * ka;
            S->b = b + A.B * kb;
        }
        if (A.flags & P_COUNT_STEP) {
            S->t += h;
            S->step += 1;
        }
        if (v2 && (A.flags & P_RK_ERROR)) {
            // embedded estimate |y_4 - y_3| / |y_4| and the step-size controller
            const double eps = w2[1] > 0.0 ? sqrt(w2[0] / w2[1]) : 0.0;
            double f = eps > 0.0 ? 0.9 * cbrt(A.tol / eps) : 2.0;
            f = f > 2.0 ? 2.0 : (f < 0.2 ? 0.2 : f);
            double hn = h * f;
            hn = hn > A.hmax ? A.hmax : (hn < A.hmin ? A.hmin : hn);
            S->rk_err = eps;
            S->h = hn;
        } else if (v2) {  // Eq. eomR for the output state, with its scale factor
            const double an = S->a, an2 = an * an;
            const double Kn = w2[0] / (2.0 * an2 * an2 * an2 * vol), Gn = w2[1] / (2.0 * an2 * A.dx * A.dx * vol);
            const double Vn = w2[2] / vol, phidvn = w2[3] / vol, phi2n = w2[4] / vol;
            const double F = 1.0 / (1.0 + (6.0 * A.xi - 1.0) * A.xi * A.kappa * phi2n);
            S->rbar = A.kappa * F * ((1.0 - 6.0 * A.xi) * (2.0 * Gn - 2.0 * Kn) + 4.0 * Vn - 6.0 * A.xi * phidvn);
        }
        int st = 0;
        if (!isfinite(rho) || !isfinite(p)) st |= ST_NAN;
        if (first && A.hubble_limit > 0.0 && hv > A.hubble_limit) st |= ST_CONSTRAINT;
        if (st) atomicOr(&S->status, st);
        S->counter = 0u;
    }
}

// EST: the last stage of an adaptive RK3-4 step, which also sums the embedded error estimate
// (a separate instance keeps that work and its registers out of the other stages).
template <typename T, int NF, bool KAHAN, int VW, bool EST>
__global__ void __launch_bounds__(512) k_rk_stage(const RkStageArgs<T> A)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);  // [NF][3][BY+2][N] old field
    __shared__ double s_coef[6];
    __shared__ double s_red[32][kMaxQ];
    __shared__ int s_last;

    const int N = A.N, BY = A.BY;
    const int TX = N / VW;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int r = tid < BY * TX ? tid / TX : BY, tx = tid < BY * TX ? tid % TX : 0;
    const int slot_stride = (BY + 2) * N, field_stride = 3 * slot_stride;
    const int x0 = tx * VW;
    const bool first = (A.flags & P_FIRST_STAGE) != 0;
    long long u0, u1;
    block_units(N, A.nby, A.DZ, u0, u1);

    if (tid == 0) {
        const double a = A.scal->a;
        const double h = (A.flags & P_DEVICE_H) ? A.scal->h : A.h;  // adaptive steps: the device's h
        s_coef[0] = h * apow(a, A.alpha - 3.0);
        s_coef[1] = h * apow(a, 1.0 + A.alpha) / (A.dx * A.dx);
        s_coef[2] = h * apow(a, 3.0 + A.alpha);
        s_coef[3] = a;
        s_coef[5] = h;
        s_coef[4] = A.nmc ? A.xi * A.scal->rbar : 0.0;  // xi R of the stage's state
    }
    __syncthreads();
    const T cphi = (T)s_coef[0], cL = (T)s_coef[1], cV = (T)s_coef[2], xiR = (T)s_coef[4];
    const T cA = (T)A.A, cB = (T)A.B;
    const PotCoef<T> P(A.m2, A.lam, A.g2);
    Acc<T> accK[NF], accG[NF], accV;
    Acc<T> accE, accY;  // adaptive RK3-4, last stage: |B k|^2 and |y|^2
    constexpr bool est = EST;

    int y0 = 0, z0 = 0, R = 1;
    // Load plane z0 + zrel of own and halo rows of the old fields into ring slot `slot`.
    auto fill = [&](int zrel, int slot) {
        int zz = z0 + zrel;
        zz = zz < 0 ? zz + N : (zz >= N ? zz - N : zz);
        if (r < R) {
            const size_t base = ((size_t)zz * N + (y0 + r)) * N + x0;
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                T ph[VW];
                vload<T, VW>(ph, A.phi_in[f] + base);
                vstore<T, VW>(sm + f * field_stride + slot * slot_stride + (r + 1) * N + x0, ph);
            }
        }
        for (int h = tid; h < NF * 2 * TX; h += nthr) {
            const int f = h / (2 * TX), hv = h - f * 2 * TX;
            const int sel = hv / TX, vx = (hv - sel * TX) * VW;
            int y = sel == 0 ? y0 - 1 : y0 + R;
            y = y < 0 ? y + N : (y >= N ? y - N : y);
            const int srow = sel == 0 ? 0 : R + 1;
            T ph[VW];
            vload<T, VW>(ph, A.phi_in[f] + ((size_t)zz * N + y) * N + vx);
            vstore<T, VW>(sm + f * field_stride + slot * slot_stride + srow * N + vx, ph);
        }
    };

    for (long long u = u0; u < u1;) {
        const int tile = (int)(u / N);
        z0 = (int)(u - (long long)tile * N);
        const int NZ = (int)min((long long)(N - z0), u1 - u);
        y0 = tile * BY;
        R = min(BY, N - y0);
        u += NZ;
        fill(-1, 0);
        fill(0, 1);
        for (int zr = 0; zr < NZ; ++zr) {
            const int sl = zr % 3, sc = (zr + 1) % 3, su = (zr + 2) % 3;
            fill(zr + 1, su);
            __syncthreads();
            if (r < R) {
                const size_t base = ((size_t)(z0 + zr) * N + (y0 + r)) * N + x0;
                T phc[NF][VW], lap[NF][VW];
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    const T* Sc = sm + f * field_stride + sc * slot_stride + (r + 1) * N;
                    const T* Szm = sm + f * field_stride + sl * slot_stride + (r + 1) * N;
                    const T* Szp = sm + f * field_stride + su * slot_stride + (r + 1) * N;
                    T c[VW], ym[VW], yp[VW], zm[VW], zp[VW];
                    vload_smem<T, VW>(c, Sc + x0);
                    vload_smem<T, VW>(ym, Sc - N + x0);
                    vload_smem<T, VW>(yp, Sc + N + x0);
                    vload_smem<T, VW>(zm, Szm + x0);
                    vload_smem<T, VW>(zp, Szp + x0);
                    const T xm_edge = Sc[x0 == 0 ? N - 1 : x0 - 1];
                    const T xp_edge = Sc[x0 + VW == N ? 0 : x0 + VW];
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
                    T pv[VW], kf[VW], kp[VW], cv[VW], ksum = (T)0;
                    vload<T, VW>(pv, A.pi_in[f] + base);
                    if (!first) {
                        vload<T, VW>(kf, A.kphi_in[f] + base);
                        vload<T, VW>(kp, A.kpi_in[f] + base);
                    }
                    if (KAHAN) vload<T, VW>(cv, A.c_in[f] + base);
                    T ph[VW], po[VW], ee = (T)0, ey = (T)0;
#pragma unroll
                    for (int i = 0; i < VW; ++i) {
                        const T p0 = phc[0][i];
                        const T p1 = NF > 1 ? phc[NF - 1][i] : (T)0;
                        T dV;
                        if (f == 0) dV = p0 * (P.m20 + P.l0 * p0 * p0 + (NF > 1 ? P.g2 * p1 * p1 : (T)0)) + xiR * p0;
                        else dV = p1 * (P.m21 + P.l1 * p1 * p1 + P.g2 * p0 * p0);
                        ksum += pv[i] * pv[i];
                        const T fphi = cphi * pv[i];
                        const T fpi = cL * lap[f][i] - cV * dV;
                        kf[i] = first ? fphi : cA * kf[i] + fphi;
                        kp[i] = first ? fpi : cA * kp[i] + fpi;
                        ph[i] = phc[f][i];
                        drift<T, KAHAN>(ph[i], cv[i], kf[i], cB);  // phi += B k_phi (compensated in FP32)
                        po[i] = pv[i] + cB * kp[i];
                        if (est) {
                            const T dp = cB * kf[i], dq = cB * kp[i];
                            ee += dp * dp + dq * dq;
                            ey += ph[i] * ph[i] + po[i] * po[i];
                        }
                        if (f == 0) {
                            T v = p0 * p0 * (P.h_m20 + P.q_l0 * p0 * p0);
                            if (NF > 1) v += p1 * p1 * (P.h_m21 + P.q_l1 * p1 * p1) + P.h_g2 * p0 * p0 * p1 * p1;
                            vsum += v;
                        }
                    }
                    accK[f].add(ksum);
                    if (est) {
                        accE.add(ee);
                        accY.add(ey);
                    }
                    vstore<T, VW>(A.phi_out[f] + base, ph);
                    vstore<T, VW>(A.pi_out[f] + base, po);
                    vstore<T, VW>(A.kphi_out[f] + base, kf);
                    vstore<T, VW>(A.kpi_out[f] + base, kp);
                    if (KAHAN) vstore<T, VW>(A.c_out[f] + base, cv);
                }
                accV.add(vsum);
            }
            __syncthreads();
        }
    }

    // ---- block partials, last block: energies of the old state and the (a, a') stage ----
    const Acc<T>* av[kMaxQ] = {&accK[0], NF > 1 ? &accK[NF - 1] : nullptr, &accG[0], NF > 1 ? &accG[NF - 1] : nullptr,
                               &accV};
    const Acc<T>* ae[kMaxQ] = {&accE, &accY, nullptr, nullptr, nullptr};
    rk_finish(A, av, s_coef[3], s_coef[5], first, s_red, &s_last, tid, nthr, est ? &ae : nullptr);
}

// TMA-staged form of the same stage.  One producer warp copies, plane after plane, the rows
// a tile needs into a ring of S stage buffers with bulk asynchronous copies: the old field's
// rows y0-1 .. y0+R (three copies: the halo rows and the R own rows) and the R own rows of
// pi, the compensation and k_phi, k_pi (the z halo planes: the field only; the first stage:
// no k).  Consumer warps own one x vector of one row each, keep the field of planes j-2,
// j-1, j of their own vector in registers, and at plane j finish plane j-1: the z
// neighbours from registers, the y neighbours and the other arrays from the stage of plane
// j-1, the x neighbours from the adjacent lanes.  A stage is released once its plane was
// finished (the z halos right away), so the producer stays S - 2 planes ahead; the warps
// synchronise through the full / empty mbarriers only, every wait bounded.  The arithmetic
// is that of k_rk_stage, operation for operation.
// For a non-minimally coupled field (A.nmc == 2) the stage also sums the terms of the Ricci
// scalar (Eq. eomR) of its output state, which the next stage needs: pi^2, V, phi V', phi^2
// of the new values at each site and the forward differences of the new field.  Those cross
// the tile's last row, the vector edges and the chunk's last plane, so the stage buffers
// then also hold pi (, c), k_phi of the row y0+R and of the upper halo plane, from which a
// consumer recomputes the new field there with the owner's operations.
template <typename T, int NF, bool KAHAN, int VW, int S, bool EST>
__global__ void __launch_bounds__(480, 1) k_rk_stage_tma(const RkStageArgs<T> A)
{
    constexpr int NOWN = KAHAN ? 4 : 3;  // own-row arrays per field: pi (, c), k_phi, k_pi
    constexpr int OC = KAHAN ? 1 : -1, OKF = KAHAN ? 2 : 1, OKP = KAHAN ? 3 : 2;  // their slots
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t s_full[S];
    __shared__ __align__(8) uint64_t s_empty[S];
    __shared__ double s_coef[6];
    __shared__ double s_red[32][kMaxQ];
    __shared__ int s_last, s_timeout;

    const int N = A.N, BY = A.BY;
    const int TX = N / VW;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int CT = nthr - 32;  // consumer threads (whole warps)
    const int CW = CT / 32;
    const bool producer = tid >= CT;
    const bool own = tid < BY * TX;
    const int r = own ? tid / TX : BY, tx = own ? tid % TX : 0;
    const int x0 = tx * VW;
    // A.nmc == 2: the stage also sums the Ricci-scalar terms of its output state, which needs
    // the new field one row beyond the tile (the own arrays carry the halo row y0+R as row R)
    // and one plane beyond the z chunk (the upper halo plane carries pi, c, k_phi too)
    const bool fuse_r = NF == 1 && A.nmc == 2;
    const int phi_stride = (BY + 2) * N, own_stride = (BY + (fuse_r ? 1 : 0)) * N;
    const int field_stride = phi_stride + NOWN * own_stride;
    const int stage_stride = NF * field_stride;
    T* stage = reinterpret_cast<T*>(smem_raw);
    const bool first = (A.flags & P_FIRST_STAGE) != 0;
    long long u0, u1;
    block_units(N, A.nby, A.DZ, u0, u1);

    if (tid == 0) {
        const double a = A.scal->a;
        const double h = (A.flags & P_DEVICE_H) ? A.scal->h : A.h;  // adaptive steps: the device's h
        s_coef[0] = h * apow(a, A.alpha - 3.0);
        s_coef[1] = h * apow(a, 1.0 + A.alpha) / (A.dx * A.dx);
        s_coef[2] = h * apow(a, 3.0 + A.alpha);
        s_coef[3] = a;
        s_coef[5] = h;
        s_coef[4] = A.nmc ? A.xi * A.scal->rbar : 0.0;  // xi R of the stage's state
#pragma unroll
        for (int k = 0; k < S; ++k) {
            mbar_init(&s_full[k], 1);
            mbar_init(&s_empty[k], CW);
        }
        mbar_fence_init();
        s_timeout = 0;
    }
    __syncthreads();
    Acc<T> accK[NF], accG[NF], accV;
    Acc<T> accE, accY;  // adaptive RK3-4, last stage: |B k|^2 and |y|^2
    constexpr bool est = EST;
    Acc<T> nK, nG, nV, nPV, nP2;  // Ricci terms of the output state (fuse_r)
    auto bounded = [&](uint64_t* bar, uint32_t parity) {
        if (!mbar_wait_bounded(bar, parity, s_timeout ? 1000000ull : 2000000000ull)) s_timeout = 1;
    };

    if (producer) {
        // ---------------------------------------------------------------- producer warp
        const int lane = tid - CT;
        int st = 0, issued = 0;
        uint32_t empty_phase = 0;
        const int nown_in = first ? (KAHAN ? 2 : 1) : NOWN;  // arrays of the own rows read this stage
        for (long long u = u0; u < u1;) {
            const int tile = (int)(u / N);
            const int z0 = (int)(u - (long long)tile * N);
            const int NZ = (int)min((long long)(N - z0), u1 - u);
            const int y0 = tile * BY, R = min(BY, N - y0);
            const int ylo = y0 == 0 ? N - 1 : y0 - 1;
            const int yhi = y0 + R == N ? 0 : y0 + R;
            u += NZ;
            int zz = z0 == 0 ? N - 1 : z0 - 1;
            for (int j = 0; j < NZ + 2; ++j) {
                if (issued >= S) {
                    bounded(&s_empty[st], (empty_phase >> st) & 1u);
                    empty_phase ^= 1u << st;
                }
                // own-row arrays this plane: none for the lower z halo, and for the upper one
                // only what the new field needs when the Ricci terms are fused
                const int nnew = first ? (KAHAN ? 2 : 1) : (KAHAN ? 3 : 2);  // pi (, c) (, k_phi)
                const int nown = j == 0 ? 0 : (j == NZ + 1 ? (fuse_r ? nnew : 0) : nown_in);
                const int nhalo = fuse_r && j > 0 ? nnew : 0;  // the row y0+R of the same arrays
                const int per_field = 3 + nown + nhalo;
                if (lane == 0)
                    mbar_arrive_expect_tx(&s_full[st],
                                          (uint32_t)(NF * (R + 2 + nown * R + nhalo) * N * sizeof(T)));
                __syncwarp();
                if (lane < NF * per_field) {
                    const int f = lane / per_field, part = lane - f * per_field;
                    T* fb = stage + st * stage_stride + f * field_stride;
                    const size_t plane = (size_t)zz * N;
                    if (part < 3) {  // old field: halo row below, own rows, halo row above
                        const T* src = f == 0 ? A.phi_in[0] : A.phi_in[NF - 1];
                        const int y = part == 0 ? ylo : (part == 1 ? y0 : yhi);
                        const int srow = part == 0 ? 0 : (part == 1 ? 1 : R + 1);
                        const int nrows = part == 1 ? R : 1;
                        tma_bulk_g2s(fb + srow * N, src + (plane + y) * N, (uint32_t)(nrows * N * sizeof(T)), &s_full[st]);
                    } else {  // own rows (or the halo row y0+R) of pi (, c), k_phi, k_pi
                        const bool halo = part - 3 >= nown;
                        const int k = halo ? part - 3 - nown : part - 3;
                        const T* src;
                        if (k == 0) src = f == 0 ? A.pi_in[0] : A.pi_in[NF - 1];
                        else if (k == OC) src = f == 0 ? A.c_in[0] : A.c_in[NF - 1];
                        else if (k == OKF) src = f == 0 ? A.kphi_in[0] : A.kphi_in[NF - 1];
                        else src = f == 0 ? A.kpi_in[0] : A.kpi_in[NF - 1];
                        if (halo)
                            tma_bulk_g2s(fb + phi_stride + k * own_stride + R * N, src + (plane + yhi) * N,
                                         (uint32_t)(N * sizeof(T)), &s_full[st]);
                        else
                            tma_bulk_g2s(fb + phi_stride + k * own_stride, src + (plane + y0) * N,
                                         (uint32_t)(R * N * sizeof(T)), &s_full[st]);
                    }
                }
                __syncwarp();
                ++issued;
                st = st + 1 == S ? 0 : st + 1;
                zz = zz + 1 == N ? 0 : zz + 1;
            }
        }
    } else {
        // ---------------------------------------------------------------- consumer warps
        const T cphi = (T)s_coef[0], cL = (T)s_coef[1], cV = (T)s_coef[2], xiR = (T)s_coef[4];
        const T cA = (T)A.A, cB = (T)A.B;
        const PotCoef<T> P(A.m2, A.lam, A.g2);
        const int lane = tid & 31;
        const bool xm_lane = own && lane > 0 && tx > 0;
        const bool xp_lane = own && lane < 31 && tx < TX - 1;
        const int xm_idx = x0 == 0 ? N - 1 : x0 - 1;
        const int xp_idx = x0 + VW == N ? 0 : x0 + VW;
        T zlo[NF][VW], zmid[NF][VW], znew[NF][VW];  // old field of planes j-2, j-1, j
#pragma unroll
        for (int f = 0; f < NF; ++f)
#pragma unroll
            for (int i = 0; i < VW; ++i) zlo[f][i] = zmid[f][i] = znew[f][i] = (T)0;
        // new field 0 of VW elements at phi row rphi, own row rown, column col of stage sbuf: the
        // same operations as the site that owns them (used for the forward differences of the
        // output state across tile rows, vector edges and the z chunk's end)
        auto phi_new = [&](const T* sbuf, int rphi, int rown, int col, T (&out)[VW]) {
            const T* ob = sbuf + phi_stride + rown * N + col;
            T pv[VW], cv[VW], kf[VW];
            vload_smem<T, VW>(out, sbuf + rphi * N + col);
            vload_smem<T, VW>(pv, ob);
            if (KAHAN) vload_smem<T, VW>(cv, ob + (KAHAN ? OC : 0) * own_stride);
            if (!first) vload_smem<T, VW>(kf, ob + OKF * own_stride);
#pragma unroll
            for (int i = 0; i < VW; ++i) {
                const T fphi = cphi * pv[i];
                kf[i] = first ? fphi : cA * kf[i] + fphi;
                drift<T, KAHAN>(out[i], cv[i], kf[i], cB);
            }
        };
        auto phi_new1 = [&](const T* sbuf, int rphi, int rown, int col) {
            const T* ob = sbuf + phi_stride + rown * N + col;
            T ph = sbuf[rphi * N + col], cv = KAHAN ? ob[(KAHAN ? OC : 0) * own_stride] : (T)0;
            const T fphi = cphi * ob[0];
            const T kf = first ? fphi : cA * ob[OKF * own_stride] + fphi;
            drift<T, KAHAN>(ph, cv, kf, cB);
            return ph;
        };
        T nzprev[VW];  // new field of the plane finished before (own vector), for the z differences
#pragma unroll
        for (int i = 0; i < VW; ++i) nzprev[i] = (T)0;
        int st = 0, st_prev = 0;
        uint32_t full_phase = 0;
        auto release = [&](int s_idx) {
            __syncwarp();
            if (lane == 0) mbar_arrive(&s_empty[s_idx]);
        };
        for (long long u = u0; u < u1;) {
            const int tile = (int)(u / N);
            const int z0 = (int)(u - (long long)tile * N);
            const int NZ = (int)min((long long)(N - z0), u1 - u);
            const int y0 = tile * BY, R = min(BY, N - y0);
            u += NZ;
            for (int j = 0; j < NZ + 2; ++j) {
                bounded(&s_full[st], (full_phase >> st) & 1u);
                full_phase ^= 1u << st;
                const T* sb = stage + st * stage_stride;
                if (r < R) {
#pragma unroll
                    for (int f = 0; f < NF; ++f) vload_smem<T, VW>(znew[f], sb + f * field_stride + (r + 1) * N + x0);
                }
                if (j >= 2) {
                    // finish plane j-1 from its stage (sp) and the registers
                    const T* sp = stage + st_prev * stage_stride;
                    T phc[NF][VW], lap[NF][VW];
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        const T xm_s = __shfl_up_sync(0xffffffffu, zmid[f][VW - 1], 1);
                        const T xp_s = __shfl_down_sync(0xffffffffu, zmid[f][0], 1);
                        if (r < R) {
                            const T* fp = sp + f * field_stride;
                            T ym[VW], yp[VW];
                            vload_smem<T, VW>(ym, fp + r * N + x0);
                            vload_smem<T, VW>(yp, fp + (r + 2) * N + x0);
                            const T xm_edge = xm_lane ? xm_s : fp[(r + 1) * N + xm_idx];
                            const T xp_edge = xp_lane ? xp_s : fp[(r + 1) * N + xp_idx];
                            T g = (T)0;
#pragma unroll
                            for (int i = 0; i < VW; ++i) {
                                const T c = zmid[f][i];
                                const T xm = i == 0 ? xm_edge : zmid[f][i - 1];
                                const T xp = i == VW - 1 ? xp_edge : zmid[f][i + 1];
                                lap[f][i] = ((xp + xm) + (yp[i] + ym[i]) + (znew[f][i] + zlo[f][i])) - (T)6 * c;
                                const T gx = xp - c, gy = yp[i] - c, gz = znew[f][i] - c;
                                g += gx * gx + gy * gy + gz * gz;
                                phc[f][i] = c;
                            }
                            accG[f].add(g);
                        }
                    }
                    if (r < R) {
                        const size_t base = ((size_t)(z0 + j - 2) * N + (y0 + r)) * N + x0;
                        T vsum = (T)0;
#pragma unroll
                        for (int f = 0; f < NF; ++f) {
                            const T* ob = sp + f * field_stride + phi_stride + r * N + x0;
                            T pv[VW], kf[VW], kp[VW], cv[VW], ksum = (T)0;
                            vload_smem<T, VW>(pv, ob);
                            if (!first) {
                                vload_smem<T, VW>(kf, ob + OKF * own_stride);
                                vload_smem<T, VW>(kp, ob + OKP * own_stride);
                            }
                            if (KAHAN) vload_smem<T, VW>(cv, ob + (KAHAN ? OC : 0) * own_stride);
                            T ph[VW], po[VW], ee = (T)0, ey = (T)0;
#pragma unroll
                            for (int i = 0; i < VW; ++i) {
                                const T p0 = phc[0][i];
                                const T p1 = NF > 1 ? phc[NF - 1][i] : (T)0;
                                T dV;
                                if (f == 0) dV = p0 * (P.m20 + P.l0 * p0 * p0 + (NF > 1 ? P.g2 * p1 * p1 : (T)0)) + xiR * p0;
                                else dV = p1 * (P.m21 + P.l1 * p1 * p1 + P.g2 * p0 * p0);
                                ksum += pv[i] * pv[i];
                                const T fphi = cphi * pv[i];
                                const T fpi = cL * lap[f][i] - cV * dV;
                                kf[i] = first ? fphi : cA * kf[i] + fphi;
                                kp[i] = first ? fpi : cA * kp[i] + fpi;
                                ph[i] = phc[f][i];
                                drift<T, KAHAN>(ph[i], cv[i], kf[i], cB);  // phi += B k_phi (compensated in FP32)
                                po[i] = pv[i] + cB * kp[i];
                                if (est) {
                                    const T dp = cB * kf[i], dq = cB * kp[i];
                                    ee += dp * dp + dq * dq;
                                    ey += ph[i] * ph[i] + po[i] * po[i];
                                }
                                if (f == 0) {
                                    T v = p0 * p0 * (P.h_m20 + P.q_l0 * p0 * p0);
                                    if (NF > 1) v += p1 * p1 * (P.h_m21 + P.q_l1 * p1 * p1) + P.h_g2 * p0 * p0 * p1 * p1;
                                    vsum += v;
                                }
                            }
                            accK[f].add(ksum);
                            if (est) {
                                accE.add(ee);
                                accY.add(ey);
                            }
                            if (fuse_r && f == 0) {
                                // Ricci terms of the output state at this vector: local ones, and the
                                // forward differences in x and y (z: with the previous plane)
                                const unsigned act = __activemask();
                                const T xs = __shfl_down_sync(act, ph[0], 1);
                                const T xe = xp_lane ? xs : phi_new1(sp, r + 1, r, xp_idx);
                                T yn[VW];
                                phi_new(sp, r + 2, r + 1, x0, yn);
                                T kn = (T)0, gn = (T)0, vn = (T)0, pvn = (T)0, p2n = (T)0;
#pragma unroll
                                for (int i = 0; i < VW; ++i) {
                                    const T c = ph[i], xn = i + 1 < VW ? ph[(i + 1) % VW] : xe;
                                    kn += po[i] * po[i];
                                    gn += (xn - c) * (xn - c) + (yn[i] - c) * (yn[i] - c);
                                    if (j >= 3) gn += (c - nzprev[i]) * (c - nzprev[i]);  // plane below
                                    vn += c * c * (P.h_m20 + P.q_l0 * c * c);
                                    pvn += c * c * (P.m20 + P.l0 * c * c);
                                    p2n += c * c;
                                    nzprev[i] = c;
                                }
                                nK.add(kn);
                                nG.add(gn);
                                nV.add(vn);
                                nPV.add(pvn);
                                nP2.add(p2n);
                            }
                            vstore<T, VW>(A.phi_out[f] + base, ph);
                            vstore<T, VW>(A.pi_out[f] + base, po);
                            vstore<T, VW>(A.kphi_out[f] + base, kf);
                            vstore<T, VW>(A.kpi_out[f] + base, kp);
                            if (KAHAN) vstore<T, VW>(A.c_out[f] + base, cv);
                        }
                        accV.add(vsum);
                    }
                }
                if (fuse_r && j == NZ + 1 && r < R) {
                    // the chunk's last plane: its z difference with the new field above it
                    T up[VW];
                    phi_new(sb, r + 1, r, x0, up);
                    T gn = (T)0;
#pragma unroll
                    for (int i = 0; i < VW; ++i) gn += (up[i] - nzprev[i]) * (up[i] - nzprev[i]);
                    nG.add(gn);
                }
                if (j >= 1) release(st_prev);  // plane j-1: finished (or the lower z halo)
#pragma unroll
                for (int f = 0; f < NF; ++f)
#pragma unroll
                    for (int i = 0; i < VW; ++i) {
                        zlo[f][i] = zmid[f][i];
                        zmid[f][i] = znew[f][i];
                    }
                st_prev = st;
                st = st + 1 == S ? 0 : st + 1;
            }
            release(st_prev);  // the upper z halo of the segment is never finished
        }
    }
    __syncthreads();  // producer and consumers meet; no copy is in flight past this point
    if (tid == 0 && s_timeout) atomicOr(&A.scal->status, ST_TIMEOUT);
    const Acc<T>* av[kMaxQ] = {&accK[0], NF > 1 ? &accK[NF - 1] : nullptr, &accG[0], NF > 1 ? &accG[NF - 1] : nullptr,
                               &accV};
    // the Ricci terms of the output state, or for adaptive RK3-4 (never with them) the estimate
    const Acc<T>* a2[kMaxQ] = {est ? &accE : &nK, est ? &accY : &nG, est ? nullptr : &nV, est ? nullptr : &nPV,
                               est ? nullptr : &nP2};
    rk_finish(A, av, s_coef[3], s_coef[5], first, s_red, &s_last, tid, nthr, fuse_r || est ? &a2 : nullptr);
}

// The stage on a reduced (d+1)-dimensional lattice (section "Scalar dynamics in 1+1 and 2+1
// dimensions"): N^d sites (d = 1, 2; x fastest), the Laplacian and the gradient energy over
// the d directions; one thread per site, grid-stride, the per-site arithmetic of k_rk_stage.
template <typename T, int NF, bool KAHAN>
__global__ void __launch_bounds__(256) k_reduced_rk(const RkStageArgs<T> A, int dims)
{
    __shared__ double s_coef[6];
    __shared__ double s_red[32][kMaxQ];
    __shared__ int s_last;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const bool first = (A.flags & P_FIRST_STAGE) != 0;
    if (tid == 0) {
        const double a = A.scal->a;
        const double h = (A.flags & P_DEVICE_H) ? A.scal->h : A.h;  // adaptive steps: the device's h
        s_coef[0] = h * apow(a, A.alpha - 3.0);
        s_coef[1] = h * apow(a, 1.0 + A.alpha) / (A.dx * A.dx);
        s_coef[2] = h * apow(a, 3.0 + A.alpha);
        s_coef[3] = a;
        s_coef[5] = h;
        s_coef[4] = 0.0;
    }
    __syncthreads();
    const T cphi = (T)s_coef[0], cL = (T)s_coef[1], cV = (T)s_coef[2];
    const T cA = (T)A.A, cB = (T)A.B;
    const PotCoef<T> P(A.m2, A.lam, A.g2);
    const long long N = A.N, V = dims == 1 ? N : N * N;
    Acc<T> accK[NF], accG[NF], accV;
    Acc<T> accE, accY;  // adaptive RK3-4, last stage: |B k|^2 and |y|^2
    const bool est = (A.flags & P_RK_ERROR) != 0;
    for (long long n = blockIdx.x * (long long)nthr + tid; n < V; n += (long long)gridDim.x * nthr) {
        const long long x = n % N, row = n - x;
        const long long xm = row + (x == 0 ? N - 1 : x - 1), xp = row + (x + 1 == N ? 0 : x + 1);
        long long ym = 0, yp = 0;
        if (dims == 2) {
            const long long y = n / N;
            ym = (y == 0 ? N - 1 : y - 1) * N + x;
            yp = (y + 1 == N ? 0 : y + 1) * N + x;
        }
        T phc[NF], lap[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const T* ph = f == 0 ? A.phi_in[0] : A.phi_in[NF - 1];
            const T c = ph[n], xpv = ph[xp], xmv = ph[xm];
            T g = (xpv - c) * (xpv - c);
            if (dims == 2) {
                const T ypv = ph[yp], ymv = ph[ym];
                lap[f] = ((xpv + xmv) + (ypv + ymv)) - (T)4 * c;
                g += (ypv - c) * (ypv - c);
            } else {
                lap[f] = (xpv + xmv) - (T)2 * c;
            }
            accG[f].add(g);
            phc[f] = c;
        }
        const T p0 = phc[0], p1 = NF > 1 ? phc[NF - 1] : (T)0;
        T vsum = (T)0;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const T pv = (f == 0 ? A.pi_in[0] : A.pi_in[NF - 1])[n];
            T kf = first ? (T)0 : (f == 0 ? A.kphi_in[0] : A.kphi_in[NF - 1])[n];
            T kp = first ? (T)0 : (f == 0 ? A.kpi_in[0] : A.kpi_in[NF - 1])[n];
            T cv = KAHAN ? (f == 0 ? A.c_in[0] : A.c_in[NF - 1])[n] : (T)0;
            T dV;
            if (f == 0) dV = p0 * (P.m20 + P.l0 * p0 * p0 + (NF > 1 ? P.g2 * p1 * p1 : (T)0));
            else dV = p1 * (P.m21 + P.l1 * p1 * p1 + P.g2 * p0 * p0);
            const T fphi = cphi * pv;
            const T fpi = cL * lap[f] - cV * dV;
            kf = first ? fphi : cA * kf + fphi;
            kp = first ? fpi : cA * kp + fpi;
            T phn = phc[f];
            drift<T, KAHAN>(phn, cv, kf, cB);  // phi += B k_phi (compensated in FP32)
            accK[f].add(pv * pv);
            const T pn = pv + cB * kp;
            if (est) {
                accE.add(cB * kf * (cB * kf) + cB * kp * (cB * kp));
                accY.add(phn * phn + pn * pn);
            }
            (f == 0 ? A.phi_out[0] : A.phi_out[NF - 1])[n] = phn;
            (f == 0 ? A.pi_out[0] : A.pi_out[NF - 1])[n] = pn;
            (f == 0 ? A.kphi_out[0] : A.kphi_out[NF - 1])[n] = kf;
            (f == 0 ? A.kpi_out[0] : A.kpi_out[NF - 1])[n] = kp;
            if (KAHAN) (f == 0 ? A.c_out[0] : A.c_out[NF - 1])[n] = cv;
            if (f == 0) {
                T v = p0 * p0 * (P.h_m20 + P.q_l0 * p0 * p0);
                if (NF > 1) v += p1 * p1 * (P.h_m21 + P.q_l1 * p1 * p1) + P.h_g2 * p0 * p0 * p1 * p1;
                vsum += v;
            }
        }
        accV.add(vsum);
    }
    const Acc<T>* av[kMaxQ] = {&accK[0], NF > 1 ? &accK[NF - 1] : nullptr, &accG[0], NF > 1 ? &accG[NF - 1] : nullptr,
                               &accV};
    const Acc<T>* ae[kMaxQ] = {&accE, &accY, nullptr, nullptr, nullptr};
    rk_finish(A, av, s_coef[3], s_coef[5], first, s_red, &s_last, tid, nthr, est ? &ae : nullptr, dims);
}

// Background Ricci scalar of a non-minimally coupled field (section "Scalar fields
// non-minimally coupled to gravity", Eq. eomR in program units):
//   R = kappa F [(1 - 6 xi) (2 G - 2 K) + 4 <V> - 6 xi <phi V'>],  F = 1 / (1 + (6 xi - 1) xi kappa <phi^2>),
// with K = <pi^2> / (2 a^6) and G = <(grad+ phi)^2> / (2 a^2) of the state (field 0).  Per-thread
// compensated sums of per-vector partial sums, FP64 across threads and blocks in a fixed order;
// the last block writes R.
template <typename T, int VW>
__global__ void __launch_bounds__(256) k_nmc_ricci(const RkStageArgs<T> A)
{
    __shared__ double s_red[32][kMaxQ];
    __shared__ int s_last;
    const int N = A.N, NV = N / VW;
    const T m2 = (T)A.m2[0], lam = (T)A.lam[0];
    const T* __restrict__ phi = A.phi_in[0];
    const T* __restrict__ pi = A.pi_in[0];
    Acc<T> sK, sG, sV, sPV, sP2;
    // Whole x rows of VW-vectors: tpr threads per row, two vectors each (both loaded before
    // either is summed), rpi rows per block sweep; the +y and +z neighbour rows load
    // coalesced, one division per row.
    int tpr = (NV + 1) / 2;
    tpr = tpr < (int)blockDim.x ? tpr : (int)blockDim.x;
    const int rpi = (int)blockDim.x / tpr;
    const int rr = (int)threadIdx.x / tpr, tx = (int)threadIdx.x - rr * tpr;
    struct Vec { T ph[VW], pv[VW], py[VW], pz[VW], pxe; };
    auto load = [&](Vec& q, size_t rb, size_t ry, size_t rz, int x0) {
        vload<T, VW>(q.ph, phi + rb + x0);
        vload<T, VW>(q.pv, pi + rb + x0);
        vload<T, VW>(q.py, phi + ry + x0);
        vload<T, VW>(q.pz, phi + rz + x0);
        q.pxe = __ldg(phi + rb + (x0 + VW == N ? 0 : x0 + VW));  // x neighbour of the last element
    };
    auto sum = [&](const Vec& q) {
        T k = (T)0, gsum = (T)0, v = (T)0, pvd = (T)0, p2 = (T)0;
#pragma unroll
        for (int i = 0; i < VW; ++i) {
            const T c = q.ph[i], px = i + 1 < VW ? q.ph[(i + 1) % VW] : q.pxe;
            k += q.pv[i] * q.pv[i];
            gsum += (px - c) * (px - c) + (q.py[i] - c) * (q.py[i] - c) + (q.pz[i] - c) * (q.pz[i] - c);
            v += c * c * ((T)0.5 * m2 + (T)0.25 * lam * c * c);
            pvd += c * c * (m2 + lam * c * c);
            p2 += c * c;
        }
        sK.add(k);
        sG.add(gsum);
        sV.add(v);
        sPV.add(pvd);
        sP2.add(p2);
    };
    if (rr < rpi) {
        for (int row = blockIdx.x * rpi + rr; row < N * N; row += gridDim.x * rpi) {
            const int z = row / N, y = row - z * N;
            const size_t rb = (size_t)row * N;
            const size_t ry = ((size_t)z * N + (y + 1 == N ? 0 : y + 1)) * N;
            const size_t rz = ((size_t)(z + 1 == N ? 0 : z + 1) * N + y) * N;
            for (int xv = tx; xv < NV; xv += 2 * tpr) {
                const bool two = xv + tpr < NV;
                Vec a, b;
                load(a, rb, ry, rz, xv * VW);
                if (two) load(b, rb, ry, rz, (xv + tpr) * VW);
                sum(a);
                if (two) sum(b);
            }
        }
    }
    double v[kMaxQ] = {sK.value(), sG.value(), sV.value(), sPV.value(), sP2.value()};
    block_reduce<kMaxQ>(v, s_red, threadIdx.x, blockDim.x);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < kMaxQ; ++q) A.partials[(size_t)blockIdx.x * kMaxQ + q] = v[q];
        __threadfence();
        const unsigned prev = atomicAdd(&A.scal->counter, 1u);
        s_last = (prev + 1u == gridDim.x);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double w[kMaxQ] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
#pragma unroll
        for (int q = 0; q < kMaxQ; ++q) w[q] += __ldcg(&A.partials[(size_t)b * kMaxQ + q]);
    block_reduce<kMaxQ>(w, s_red, threadIdx.x, blockDim.x);
    if (threadIdx.x == 0) {
        DevScal* S = A.scal;
        const double vol = (double)N * N * N, a = S->a, a2 = a * a;
        const double K = w[0] / (2.0 * a2 * a2 * a2 * vol);
        const double G = w[1] / (2.0 * a2 * A.dx * A.dx * vol);
        const double Vp = w[2] / vol, phidv = w[3] / vol, phi2 = w[4] / vol;
        const double F = 1.0 / (1.0 + (6.0 * A.xi - 1.0) * A.xi * A.kappa * phi2);
        S->rbar = A.kappa * F * ((1.0 - 6.0 * A.xi) * (2.0 * G - 2.0 * K) + 4.0 * Vp - 6.0 * A.xi * phidv);
        S->counter = 0u;
    }
}

template <typename T>
static cudaError_t launch_nmc_ricci_t(const RkStageArgs<T>& A, int grid, cudaStream_t s)
{
    constexpr int VW = 16 / sizeof(T);  // 16-byte vectors where the rows allow them
    // one wave of resident blocks (a partial second wave would run at a fraction of the rate)
    static int wave[2] = {0, 0};
    const int vi = A.N % VW == 0 ? 0 : 1;
    if (!wave[vi]) {
        int dev = 0, nsm = 0, occ = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        const cudaError_t e = vi == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_nmc_ricci<T, VW>, 256, 0)
                                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_nmc_ricci<T, 1>, 256, 0);
        if (e != cudaSuccess) return e;
        wave[vi] = (occ > 0 ? occ : 1) * (nsm > 0 ? nsm : 1);
    }
    if (grid > wave[vi]) grid = wave[vi];
    if (vi == 0) k_nmc_ricci<T, VW><<<grid, 256, 0, s>>>(A);
    else k_nmc_ricci<T, 1><<<grid, 256, 0, s>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_nmc_ricci(int precision, const void* args, int grid, cudaStream_t s)
{
    if (grid < 1) return cudaErrorInvalidValue;
    if (precision == CL_PREC_FP64) return launch_nmc_ricci_t(*static_cast<const RkStageArgs<double>*>(args), grid, s);
    return launch_nmc_ricci_t(*static_cast<const RkStageArgs<float>*>(args), grid, s);
}

template <typename T, int NF, bool KAHAN, int VW>
static cudaError_t launch_rk(const RkStageArgs<T>& A, cudaStream_t s)
{
    const int TX = A.N / VW;
    dim3 block(((TX * A.BY + 31) / 32) * 32);
    dim3 grid(A.nby * A.nbz);
    const size_t smem = (size_t)NF * 3 * (A.BY + 2) * A.N * sizeof(T);
    static DevFlag attr_set[2];
    const bool est = (A.flags & P_RK_ERROR) != 0;
    if (!attr_set[est]) {
        cudaError_t e = est ? cudaFuncSetAttribute(k_rk_stage<T, NF, KAHAN, VW, true>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, kPassMaxSmem)
                            : cudaFuncSetAttribute(k_rk_stage<T, NF, KAHAN, VW, false>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, kPassMaxSmem);
        if (e != cudaSuccess) return e;
        attr_set[est] = true;
    }
    if (est) k_rk_stage<T, NF, KAHAN, VW, true><<<grid, block, smem, s>>>(A);
    else k_rk_stage<T, NF, KAHAN, VW, false><<<grid, block, smem, s>>>(A);
    return cudaGetLastError();
}

template <typename T, int NF, bool KAHAN>
static cudaError_t rk_vw(const RkStageArgs<T>& A, int vw, cudaStream_t s)
{
    if (vw == 1) return launch_rk<T, NF, KAHAN, 1>(A, s);
    if (vw == 2) return launch_rk<T, NF, KAHAN, 2>(A, s);
    if constexpr (sizeof(T) == 4) {
        if (vw == 4) return launch_rk<T, NF, KAHAN, 4>(A, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_rk_stage(int precision, int nf, const void* args, int vw, cudaStream_t s)
{
    if (precision == CL_PREC_FP64) {
        const auto& A = *static_cast<const RkStageArgs<double>*>(args);
        return nf == 1 ? rk_vw<double, 1, false>(A, vw, s) : rk_vw<double, 2, false>(A, vw, s);
    }
    const auto& A = *static_cast<const RkStageArgs<float>*>(args);
    if (precision == CL_PREC_FP32_KAHAN)
        return nf == 1 ? rk_vw<float, 1, true>(A, vw, s) : rk_vw<float, 2, true>(A, vw, s);
    return nf == 1 ? rk_vw<float, 1, false>(A, vw, s) : rk_vw<float, 2, false>(A, vw, s);
}

size_t rk_stage_tma_smem(int precision, int nf, int N, int BY, int stages, bool ricci)
{
    const size_t es = precision == CL_PREC_FP64 ? 8 : 4;
    const int nown = precision == CL_PREC_FP32_KAHAN ? 4 : 3;
    return (size_t)stages * nf * ((size_t)(BY + 2) + (size_t)nown * (BY + (ricci ? 1 : 0))) * N * es;
}

template <typename T, int NF, bool KAHAN, int VW>
static cudaError_t launch_rk_tma(const RkStageArgs<T>& A, int stages, cudaStream_t s)
{
    if constexpr (VW * sizeof(T) == 16) {
        const int prec = sizeof(T) == 8 ? CL_PREC_FP64 : (KAHAN ? CL_PREC_FP32_KAHAN : CL_PREC_FP32);
        const int TX = A.N / VW;
        const dim3 block(((TX * A.BY + 31) / 32) * 32 + 32);  // consumers + the producer warp
        const dim3 grid(A.DZ > 0 ? A.nby * A.nbz : A.nbz);
        const size_t smem = rk_stage_tma_smem(prec, NF, A.N, A.BY, stages, A.nmc == 2);
        if (block.x > 480 || smem > (size_t)kPassMaxSmem || A.N % VW != 0 || (A.nmc == 2 && NF != 1))
            return cudaErrorInvalidValue;
        static DevFlag attr[2][7];
        const bool est = (A.flags & P_RK_ERROR) != 0;
        cudaError_t e = cudaSuccess;
#define CL_RKT_CASE(SS)                                                                                         \
    case SS:                                                                                                    \
        if (!attr[est][SS]) {                                                                                   \
            e = est ? cudaFuncSetAttribute(k_rk_stage_tma<T, NF, KAHAN, VW, SS, true>,                          \
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, kPassMaxSmem)           \
                    : cudaFuncSetAttribute(k_rk_stage_tma<T, NF, KAHAN, VW, SS, false>,                         \
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, kPassMaxSmem);          \
            if (e != cudaSuccess) return e;                                                                     \
            attr[est][SS] = true;                                                                               \
        }                                                                                                       \
        if (est) k_rk_stage_tma<T, NF, KAHAN, VW, SS, true><<<grid, block, smem, s>>>(A);                       \
        else k_rk_stage_tma<T, NF, KAHAN, VW, SS, false><<<grid, block, smem, s>>>(A);                          \
        return cudaGetLastError();
        switch (stages) {
            CL_RKT_CASE(3)
            CL_RKT_CASE(4)
            CL_RKT_CASE(5)
            CL_RKT_CASE(6)
        }
#undef CL_RKT_CASE
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_rk_stage_tma(int precision, int nf, const void* args, int vw, int stages, cudaStream_t s)
{
    if (precision == CL_PREC_FP64) {
        const auto& A = *static_cast<const RkStageArgs<double>*>(args);
        if (vw != 2) return cudaErrorInvalidValue;
        return nf == 1 ? launch_rk_tma<double, 1, false, 2>(A, stages, s) : launch_rk_tma<double, 2, false, 2>(A, stages, s);
    }
    const auto& A = *static_cast<const RkStageArgs<float>*>(args);
    if (vw != 4) return cudaErrorInvalidValue;
    if (precision == CL_PREC_FP32_KAHAN)
        return nf == 1 ? launch_rk_tma<float, 1, true, 4>(A, stages, s) : launch_rk_tma<float, 2, true, 4>(A, stages, s);
    return nf == 1 ? launch_rk_tma<float, 1, false, 4>(A, stages, s) : launch_rk_tma<float, 2, false, 4>(A, stages, s);
}

template <typename T, int NF, bool KAHAN>
static cudaError_t launch_reduced_rk_t(const RkStageArgs<T>& A, int dims, int grid, cudaStream_t s)
{
    k_reduced_rk<T, NF, KAHAN><<<grid, 256, 0, s>>>(A, dims);
    return cudaGetLastError();
}

cudaError_t launch_reduced_rk_stage(int precision, int nf, const void* args, int dims, int grid, cudaStream_t s)
{
    if ((dims != 1 && dims != 2) || grid < 1) return cudaErrorInvalidValue;
    if (precision == CL_PREC_FP64) {
        const auto& A = *static_cast<const RkStageArgs<double>*>(args);
        if (A.nmc) return cudaErrorInvalidValue;
        return nf == 1 ? launch_reduced_rk_t<double, 1, false>(A, dims, grid, s)
                       : launch_reduced_rk_t<double, 2, false>(A, dims, grid, s);
    }
    const auto& A = *static_cast<const RkStageArgs<float>*>(args);
    if (A.nmc) return cudaErrorInvalidValue;
    if (precision == CL_PREC_FP32_KAHAN)
        return nf == 1 ? launch_reduced_rk_t<float, 1, true>(A, dims, grid, s)
                       : launch_reduced_rk_t<float, 2, true>(A, dims, grid, s);
    return nf == 1 ? launch_reduced_rk_t<float, 1, false>(A, dims, grid, s)
                   : launch_reduced_rk_t<float, 2, false>(A, dims, grid, s);
}

}  // namespace clk
