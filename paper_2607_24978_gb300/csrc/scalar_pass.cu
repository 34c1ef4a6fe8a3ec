// Fused scalar-field pass of the lattice time step (sm_103a).
//
// One launch advances every site of a lattice by one "pass" of a kick-drift
// integrator in its staggered (leapfrog) form, with per-pass coefficients
// (d, e, k) that express velocity Verlet and the Yoshida-4 composition:
//
//   a_new   = a + d a'                                   (scale-factor drift)
//   phi     = phi + d ((a + a_new)/2)^(alpha-3) pi       (field drift, Kahan-compensated in FP32)
//   F       = a_new^(1+alpha) Lap phi - a_new^(3+alpha) dV/dphi     (Eq. singletEOM kick)
//   pi_int  = pi + e F      -> K, G, V at the pass's integer time (Eq. energy-contrib)
//   pi      = pi + k F
//   a'      = a' + k a''(a_new, rho, p)                  (Eq. Friedmann1, in the last block)
//
// Data layout: one contiguous N^3 array per field, momentum and compensation,
// x fastest, read from one buffer and written to its ping-pong partner.
//
// Tiling: a block owns full x rows (N sites), BY rows in y and DZ planes in z.
// It marches up z keeping a three-plane ring of drifted field values in shared
// memory (own rows plus one halo row on each side); x neighbours wrap inside the
// row, y neighbours come from the halo rows, z neighbours from the ring.  The
// drift is applied once per loaded element and every output is written once.
//
// Two loaders:
//  * TMA-staged (rows of 16-byte multiples): warp 0 copies, for every plane, the
//    own rows plus the two halo rows of every input array with bulk TMA copies
//    (cp.async.bulk, completion on an mbarrier) into a ring of S stage buffers,
//    S-1 planes ahead of the plane being drifted, so loads stay in flight while
//    the block drifts and kicks.  mbarrier waits are bounded (globaltimer) and a
//    timeout is reported through the status word, never a hang.
//  * general (any N): vector loads straight from global memory.
//
// Energies: per-thread sums (compensated FP32 or FP64) -> warp shuffles in FP64 ->
// block partial in FP64 -> the last block to finish reduces the partials in a
// fixed order (deterministic), evaluates rho and p, updates a and a' and writes
// the diagnostics.  No block ever waits for another.
#include <math.h>

#include "cl_internal.cuh"
#include "kernel_common.cuh"

namespace clk {

// Scalar prefactors of a pass, computed once per block by thread 0.
__device__ __forceinline__ void pass_coefficients(const double a_old, const double b_old, const double d,
                                                  const double alpha, const double dx, const bool expand,
                                                  double* s_coef)
{
    const double a_new = expand ? a_old + d * b_old : a_old;
    const double ah = 0.5 * (a_old + a_new);
    s_coef[0] = d * pow(ah, alpha - 3.0);
    s_coef[1] = pow(a_new, 1.0 + alpha) / (dx * dx);
    s_coef[2] = pow(a_new, 3.0 + alpha);
    s_coef[3] = a_new;
}

// Kick of one own-row vector of a plane.  S*[f] point at row (r+1) of the centre
// (Sc), lower (Szm) and upper (Szp) planes of field f; rows r and r+2 of the
// centre plane are Sc -/+ N.  Writes pi_out and accumulates K, G, V.
template <typename T, int NF, int VW>
__device__ __forceinline__ void kick_vector(const T* const (&Sc)[NF], const T* const (&Szm)[NF],
                                            const T* const (&Szp)[NF], int N, int x0, const T (&pin)[NF][VW],
                                            const T cL, const T cV, const T ce, const T ck, const PotCoef<T>& P,
                                            T* const (&pi_out)[2], size_t base, Acc<T> (&accK)[NF],
                                            Acc<T> (&accG)[NF], Acc<T>& accV)
{
    T phc[NF][VW], lap[NF][VW];
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

// Block partials, last-block-done fixed-order reduction and the scalar update.
template <typename T, int NF>
__device__ __forceinline__ void finish_pass(const ScalarPassArgs<T>& A, Acc<T> (&accK)[NF], Acc<T> (&accG)[NF],
                                            Acc<T>& accV, const double* s_coef, double (*s_red)[kMaxQ],
                                            int* s_last, int tid, int nthr, int timeout)
{
    double v[kMaxQ];
    v[0] = accK[0].value();
    v[1] = NF > 1 ? accK[NF - 1].value() : 0.0;
    v[2] = accG[0].value();
    v[3] = NF > 1 ? accG[NF - 1].value() : 0.0;
    v[4] = accV.value();
    block_reduce<kMaxQ>(v, s_red, tid, nthr);
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < kMaxQ; ++q) A.partials[(size_t)blockIdx.x * kMaxQ + q] = v[q];
        if (timeout) atomicOr(&A.scal->status, ST_TIMEOUT);
        __threadfence();
        const unsigned prev = atomicAdd(&A.scal->counter, 1u);
        *s_last = (prev + 1u == gridDim.x);
    }
    __syncthreads();
    if (!*s_last) return;

    __threadfence();
    double w[kMaxQ];
#pragma unroll
    for (int q = 0; q < kMaxQ; ++q) w[q] = 0.0;
    for (int b = tid; b < (int)gridDim.x; b += nthr)
#pragma unroll
        for (int q = 0; q < kMaxQ; ++q) w[q] += __ldcg(&A.partials[(size_t)b * kMaxQ + q]);
    block_reduce<kMaxQ>(w, s_red, tid, nthr);
    if (tid == 0) {
        DevScal* S = A.scal;
        const int N = A.N;
        const double vol = (double)N * N * N;
        const double a = s_coef[3];
        const double a2 = a * a, a6 = a2 * a2 * a2;
        const double K0 = w[0] / (2.0 * a6 * vol), K1 = w[1] / (2.0 * a6 * vol);
        const double G0 = w[2] / (A.dx * A.dx * 2.0 * a2 * vol), G1 = w[3] / (A.dx * A.dx * 2.0 * a2 * vol);
        const double Vp = w[4] / vol;
        const double K = K0 + K1, G = G0 + G1;
        const double rho = K + G + Vp;
        const double p = K - G / 3.0 - Vp;
        const bool expand = (A.flags & P_EXPANSION) != 0;
        const double a2al = pow(a, 2.0 * A.alpha);
        double b = S->b;
        if ((A.flags & P_HUBBLE_INIT) && expand) b = a * sqrt(a2al * A.kappa * rho / 3.0);
        const double addot =
            expand ? pow(a, 2.0 * A.alpha + 1.0) * (A.kappa / 6.0) * ((2.0 * A.alpha - 1.0) * rho - 3.0 * p) : 0.0;
        const double b_int = b + A.e * addot;
        const double H = b_int / a;
        const double hv = H != 0.0 ? fabs(H * H - a2al * A.kappa * rho / 3.0) / (H * H) : 0.0;
        const double t_int = S->t + A.d;
        if (A.flags & P_COMMIT) {
            S->a = a;
            S->b = b + A.k * addot;
            S->t = t_int;
            if (A.flags & P_COUNT_STEP) S->step += 1;
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
        if (A.hubble_limit > 0.0 && hv > A.hubble_limit) st |= ST_CONSTRAINT;
        if (st) atomicOr(&S->status, st);
        S->counter = 0u;
    }
}

// ------------------------------------------------------------------ general loader
template <typename T, int NF, bool KAHAN, int VW>
__global__ void __launch_bounds__(512) k_scalar_pass(const ScalarPassArgs<T> A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    __shared__ double s_coef[4];
    __shared__ double s_red[32][kMaxQ];
    __shared__ int s_last;

    const int N = A.N, BY = A.BY;
    const int TX = N / VW;  // vectors per row
    // Flat mapping: thread tid owns vector tx of row r when tid < BY*TX; the block size is
    // rounded up to whole warps, the extra threads only help with halo rows and reductions.
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int r = tid < BY * TX ? tid / TX : BY, tx = tid < BY * TX ? tid % TX : 0;
    const int slot_stride = (BY + 2) * N, field_stride = 3 * slot_stride;
    const int x0 = tx * VW;
    long long u0, u1;
    block_units(N, A.nby, A.DZ, u0, u1);
    int y0 = 0, z0 = 0, R = 1, NZ = 0;  // current segment, set in the loop below

    if (tid == 0) pass_coefficients(A.scal->a, A.scal->b, A.d, A.alpha, A.dx, (A.flags & P_EXPANSION) != 0, s_coef);
    __syncthreads();
    const T cd = (T)s_coef[0], cL = (T)s_coef[1], cV = (T)s_coef[2];
    const T ce = (T)A.e, ck = (T)A.k;
    const bool do_drift = (A.flags & P_DRIFT) != 0;
    const PotCoef<T> P(A.m2, A.lam, A.g2);
    Acc<T> accK[NF], accG[NF], accV;

    auto fill = [&](int zrel, int slot, bool write_out, T(&pin)[NF][VW]) {
        int zz = z0 + zrel;
        zz = zz < 0 ? zz + N : (zz >= N ? zz - N : zz);
        if (r < R) {
            const size_t base = ((size_t)zz * N + (y0 + r)) * N + x0;
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                T ph[VW], pv[VW], cv[VW];
                vload<T, VW>(ph, A.phi_in[f] + base);
                vload<T, VW>(pv, A.pi_in[f] + base);
                if (KAHAN) vload<T, VW>(cv, A.c_in[f] + base);
                if (do_drift) {
#pragma unroll
                    for (int i = 0; i < VW; ++i) drift<T, KAHAN>(ph[i], cv[i], pv[i], cd);
                }
                vstore<T, VW>(sm + f * field_stride + slot * slot_stride + (r + 1) * N + x0, ph);
                if (write_out) {
                    vstore<T, VW>(A.phi_out[f] + base, ph);
                    if (KAHAN) vstore<T, VW>(A.c_out[f] + base, cv);
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
                vload<T, VW>(ph, A.phi_in[f] + base);
                if (do_drift) {
                    vload<T, VW>(pv, A.pi_in[f] + base);
                    if (KAHAN) vload<T, VW>(cv, A.c_in[f] + base);
#pragma unroll
                    for (int i = 0; i < VW; ++i) drift<T, KAHAN>(ph[i], cv[i], pv[i], cd);
                }
                vstore<T, VW>(sm + f * field_stride + slot * slot_stride + srow * N + vx, ph);
            }
        }
    };

    T pcur[NF][VW], pnext[NF][VW];
    for (long long u = u0; u < u1;) {
    const int tile = (int)(u / N);
    z0 = (int)(u - (long long)tile * N);
    NZ = (int)min((long long)(N - z0), u1 - u);
    y0 = tile * BY;
    R = min(BY, N - y0);
    u += NZ;
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
            kick_vector<T, NF, VW>(Sc, Szm, Szp, N, x0, pcur, cL, cV, ce, ck, P, A.pi_out, base, accK, accG, accV);
        }
#pragma unroll
        for (int f = 0; f < NF; ++f)
#pragma unroll
            for (int i = 0; i < VW; ++i) pcur[f][i] = pnext[f][i];
        __syncthreads();
    }
    }  // segments
    finish_pass<T, NF>(A, accK, accG, accV, s_coef, s_red, &s_last, tid, nthr, 0);
}

#include "scalar_pass_tma.cuh"

// ------------------------------------------------------------------ launchers
size_t scalar_pass_smem_bytes(int precision, int nf, int N, int BY, int stages)
{
    const size_t es = precision == CL_PREC_FP64 ? 8 : 4;
    const size_t rows = (size_t)(BY + 2) * N * es;
    if (stages <= 0) return (size_t)nf * 3 * rows;  // direct loader: three-plane ring
    // TMA loader: three-slot ring of drifted fields plus the stage buffers
    const size_t narr = (size_t)nf * (precision == CL_PREC_FP32_KAHAN ? 3 : 2);
    return (size_t)nf * 3 * rows + (size_t)stages * narr * rows;
}

template <typename K>
static cudaError_t allow_smem(K kernel)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kPassMaxSmem);
}

// Launch the pass, or (occ != nullptr) report how many blocks of it fit on one SM.
template <typename T, int NF, bool KAHAN, int VW>
static cudaError_t launch_one(const ScalarPassArgs<T>& A, cudaStream_t s, int* occ)
{
    const int prec = sizeof(T) == 8 ? CL_PREC_FP64 : (KAHAN ? CL_PREC_FP32_KAHAN : CL_PREC_FP32);
    const int TX = A.N / VW;
    dim3 block(((TX * A.BY + 31) / 32) * 32 + (A.stages > 0 ? 32 : 0));  // + producer warp
    dim3 grid(A.DZ > 0 ? A.nby * A.nbz : A.grid);  // DZ < 0: balanced persistent ranges
    const size_t smem = scalar_pass_smem_bytes(prec, NF, A.N, A.BY, A.stages);
    static bool attr_set[8] = {false, false, false, false, false, false, false, false};
    const int si = A.stages < 0 ? 0 : (A.stages > 7 ? 7 : A.stages);
    cudaError_t e = cudaSuccess;
    if (!attr_set[si]) {
        switch (A.stages) {
        case 2: e = allow_smem(k_scalar_pass_tma<T, NF, KAHAN, VW, 2>); break;
        case 3: e = allow_smem(k_scalar_pass_tma<T, NF, KAHAN, VW, 3>); break;
        case 4: e = allow_smem(k_scalar_pass_tma<T, NF, KAHAN, VW, 4>); break;
        case 5: e = allow_smem(k_scalar_pass_tma<T, NF, KAHAN, VW, 5>); break;
        case 6: e = allow_smem(k_scalar_pass_tma<T, NF, KAHAN, VW, 6>); break;
        default: e = allow_smem(k_scalar_pass<T, NF, KAHAN, VW>); break;
        }
        if (e != cudaSuccess) return e;
        attr_set[si] = true;
    }
    if (occ) {
        switch (A.stages) {
        case 2: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_scalar_pass_tma<T, NF, KAHAN, VW, 2>, block.x, smem);
        case 3: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_scalar_pass_tma<T, NF, KAHAN, VW, 3>, block.x, smem);
        case 4: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_scalar_pass_tma<T, NF, KAHAN, VW, 4>, block.x, smem);
        case 5: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_scalar_pass_tma<T, NF, KAHAN, VW, 5>, block.x, smem);
        case 6: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_scalar_pass_tma<T, NF, KAHAN, VW, 6>, block.x, smem);
        default: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_scalar_pass<T, NF, KAHAN, VW>, block.x, smem);
        }
    }
    switch (A.stages) {
    case 2: k_scalar_pass_tma<T, NF, KAHAN, VW, 2><<<grid, block, smem, s>>>(A); break;
    case 3: k_scalar_pass_tma<T, NF, KAHAN, VW, 3><<<grid, block, smem, s>>>(A); break;
    case 4: k_scalar_pass_tma<T, NF, KAHAN, VW, 4><<<grid, block, smem, s>>>(A); break;
    case 5: k_scalar_pass_tma<T, NF, KAHAN, VW, 5><<<grid, block, smem, s>>>(A); break;
    case 6: k_scalar_pass_tma<T, NF, KAHAN, VW, 6><<<grid, block, smem, s>>>(A); break;
    default: k_scalar_pass<T, NF, KAHAN, VW><<<grid, block, smem, s>>>(A); break;
    }
    return cudaGetLastError();
}

template <typename T, int NF, bool KAHAN>
static cudaError_t dispatch_vw(const ScalarPassArgs<T>& A, int vw, cudaStream_t s, int* occ)
{
    if (vw == 1) return launch_one<T, NF, KAHAN, 1>(A, s, occ);
    if (vw == 2) return launch_one<T, NF, KAHAN, 2>(A, s, occ);
    if constexpr (sizeof(T) == 4) {
        if (vw == 4) return launch_one<T, NF, KAHAN, 4>(A, s, occ);
    }
    return cudaErrorInvalidValue;
}

static cudaError_t dispatch(int precision, int nf, const void* args, int vw, cudaStream_t s, int* occ)
{
    if (precision == CL_PREC_FP64) {
        const auto& A = *static_cast<const ScalarPassArgs<double>*>(args);
        return nf == 1 ? dispatch_vw<double, 1, false>(A, vw, s, occ) : dispatch_vw<double, 2, false>(A, vw, s, occ);
    }
    const auto& A = *static_cast<const ScalarPassArgs<float>*>(args);
    if (precision == CL_PREC_FP32_KAHAN)
        return nf == 1 ? dispatch_vw<float, 1, true>(A, vw, s, occ) : dispatch_vw<float, 2, true>(A, vw, s, occ);
    return nf == 1 ? dispatch_vw<float, 1, false>(A, vw, s, occ) : dispatch_vw<float, 2, false>(A, vw, s, occ);
}

cudaError_t launch_scalar_pass(int precision, int nf, const void* args, int vw, cudaStream_t s)
{
    return dispatch(precision, nf, args, vw, s, nullptr);
}

cudaError_t scalar_pass_blocks_per_sm(int precision, int nf, const void* args, int vw, int* blocks)
{
    return dispatch(precision, nf, args, vw, nullptr, blocks);
}

int scalar_pass_vector_width(int precision, int N)
{
    if (precision != CL_PREC_FP64 && N % 4 == 0) return 4;
    if (N % 2 == 0) return 2;
    return 1;
}

bool scalar_pass_tma_ok(int precision, int N)
{
    const int es = precision == CL_PREC_FP64 ? 8 : 4;
    return (N * es) % 16 == 0;
}

size_t scalar_pass_smem(int precision, int nf, int N, int BY)
{
    return scalar_pass_smem_bytes(precision, nf, N, BY, 0);
}

int scalar_pass_threads(int precision, int N, int BY)
{
    const int t = N / scalar_pass_vector_width(precision, N) * BY;
    return ((t + 31) / 32) * 32;
}

}  // namespace clk
