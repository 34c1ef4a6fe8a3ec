// Fused scalar pass over a batched ensemble of independent lattices (sm_103a).
//
// Many small lattices (each with its own size, box, couplings, a and a') advance by one
// pass of the staggered kick-drift scheme in a single persistent launch.  The work is a
// table of items, each BY full x rows times DZ planes of one member; block b takes the
// items b, b + grid, b + 2 grid, ... of a schedule (largest first) and runs the same per-site arithmetic as the
// single-lattice direct loader on it (drift while loading, stencil kick, energies).
// Reductions: every item writes its FP64 partial sums; the block that completes the last
// item of a member (an arrival counter per member) sums that member's partials in a fixed
// order and runs the member's scale-factor epilogue.  Reading a, a' happens at item
// start, before the item's arrival, so the epilogue never races a reader.
#include <math.h>

#include "cl_internal.cuh"
#include "kernel_common.cuh"
#include "scalar_pass_common.cuh"
#include "tma_pipeline.cuh"

namespace clk {

template <typename T, int NF, bool KAHAN, int VW>
__global__ void __launch_bounds__(kEnsThreads) k_ensemble_pass(const EnsPassArgs<T> A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    __shared__ double s_coef[4];
    __shared__ double s_red[32][kMaxQ];
    __shared__ int s_last;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const bool do_drift = (A.flags & P_DRIFT) != 0;
    const bool expand = (A.flags & P_EXPANSION) != 0;

    for (int k = blockIdx.x; k < A.item_end - A.item_begin; k += gridDim.x) {
        const int it = A.sched ? A.sched[k] : A.item_begin + k;
        const EnsItem I = A.items[it];
        const EnsMember& M = A.members[I.member];
        const int N = M.N, BY = M.BY;
        const double dx = M.dx;
        DevScal* S = A.scal + I.member;
        pass_coefficients_warps(tid, S->a, S->b, A.d, A.alpha, dx, expand, s_coef);
        __syncthreads();
        const TileCoef<T> C{(T)s_coef[0], (T)s_coef[1], (T)s_coef[2], (T)A.e, (T)A.k};
        const PotCoef<T> P(M.m2, M.lam, M.g2);
        const long long off = M.off;
        FieldSet<T> F{};
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            F.phi_in[f] = A.phi_in[f] + off;
            F.pi_in[f] = A.pi_in[f] + off;
            F.c_in[f] = KAHAN ? A.c_in[f] + off : nullptr;
            F.phi_out[f] = A.phi_out[f] + off;
            F.pi_out[f] = A.pi_out[f] + off;
            F.c_out[f] = KAHAN ? A.c_out[f] + off : nullptr;
        }
        Acc<T> accK[NF], accG[NF], accV;
        const int R = min(BY, N - I.y0), NZ = min(M.DZ, N - I.z0);
        march_tile<T, NF, KAHAN, VW>(F, N, BY, I.y0, R, I.z0, NZ, sm, tid, nthr, do_drift, C, P, accK, accG, accV);

        double v[kMaxQ];
        const Acc<T>* av[kMaxQ] = {&accK[0], NF > 1 ? &accK[NF - 1] : nullptr, &accG[0],
                                   NF > 1 ? &accG[NF - 1] : nullptr, &accV};
        block_reduce_acc<T, kMaxQ>(av, v, s_red, tid, nthr);
        if (tid == 0) {
#pragma unroll
            for (int q = 0; q < kMaxQ; ++q) A.partials[(size_t)it * kMaxQ + q] = v[q];
            __threadfence();
            const unsigned prev = atomicAdd(&S->counter, 1u);
            s_last = (prev + 1u == (unsigned)M.nitems);
        }
        __syncthreads();
        if (s_last && tid < 32) {  // block-uniform; one warp sums the member's item partials
            __threadfence();
            double w[kMaxQ];
            warp_sum_partials<kMaxQ>(A.partials + (size_t)M.item0 * kMaxQ, M.nitems, tid, w);
            if (tid == 0)
                scalar_epilogue(S, w, (double)N * N * N, dx, s_coef[3], A.alpha, A.kappa, A.d, A.e, A.k, A.flags,
                                A.hubble_limit);
        }
        __syncthreads();  // s_coef and s_last are rewritten by the next item
    }
}

// TMA-staged variant (every member's rows a multiple of 16 bytes): one producer warp
// streams the planes of the block's items, item after item, into a ring of S stage
// buffers; kEnsThreads consumer threads drift and kick them with the register z-march of
// the single-lattice kernel.  Stage buffers and ring slots have the size of the largest
// member tile, so a change of member between items never moves a buffer that another
// warp may still use; the full/empty mbarriers order the stages and the consumers'
// named barriers order the ring, exactly as within one lattice.  Per item the consumers
// evaluate the member's pass prefactors, reduce the item's partial sums on named barrier
// 2 and, for a member's last item, run the member's epilogue.  All waits are bounded; a
// timeout is reported through the status word of member 0.
// NR (ringless): no ring and no per-plane barrier; each warp re-drifts the y-neighbour rows
// it needs from the previous plane's stage, which it releases only after that plane's kick
// (the producer then runs S - 2 planes ahead).
template <typename T, int NF, bool KAHAN, int VW, int S, bool NR>
__global__ void __launch_bounds__(kEnsTmaThreads, NF == 1 ? 2 : 1) k_ensemble_pass_tma(const EnsPassArgs<T> A)
{
    constexpr int RING = 3;
    constexpr int KPF = KAHAN ? 3 : 2;
    constexpr int NARR = NF * KPF;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t s_full[S];
    __shared__ __align__(8) uint64_t s_empty[S];
    __shared__ double s_coef[4];
    __shared__ double s_red[32][kMaxQ];
    __shared__ int s_last, s_timeout;
    const int tid = threadIdx.x;
    constexpr int CT = kEnsThreads, CW = CT / 32;
    const bool producer = tid >= CT;
    T* stage = reinterpret_cast<T*>(smem_raw);
    T* ring = stage + S * A.stage_stride;
    const bool do_drift = (A.flags & P_DRIFT) != 0;
    const bool expand = (A.flags & P_EXPANSION) != 0;

    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < S; ++s) {
            mbar_init(&s_full[s], 1);
            mbar_init(&s_empty[s], CW);
        }
        mbar_fence_init();
        s_timeout = 0;
    }
    __syncthreads();

    if (producer) {
        const int lane = tid - CT;
        int st = 0;
        uint32_t empty_phase = 0;
        int issued = 0;
        for (int k = blockIdx.x; k < A.item_end - A.item_begin; k += gridDim.x) {
            const int it = A.sched ? A.sched[k] : A.item_begin + k;
            const EnsItem I = A.items[it];
            const EnsMember& M = A.members[I.member];
            const int N = M.N, BY = M.BY, y0 = I.y0, z0 = I.z0;
            const int R = min(BY, N - y0), NZ = min(M.DZ, N - z0);
            const int ylo = y0 == 0 ? N - 1 : y0 - 1;
            const int yhi = y0 + R == N ? 0 : y0 + R;
            const int arr_stride = (BY + 2) * N;
            const uint32_t plane_bytes = (uint32_t)(NARR * (R + 2) * N * sizeof(T));
            const long long off = M.off;
            FieldSet<T> F{};
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                F.phi_in[f] = A.phi_in[f] + off;
                F.pi_in[f] = A.pi_in[f] + off;
                F.c_in[f] = KAHAN ? A.c_in[f] + off : nullptr;
            }
            int zz = z0 == 0 ? N - 1 : z0 - 1;
            for (int j = 0; j < NZ + 2; ++j) {
                if (issued >= S) {
                    if (!mbar_wait_bounded(&s_empty[st], (empty_phase >> st) & 1u,
                                           s_timeout ? 1000000ull : 2000000000ull))
                        s_timeout = 1;
                    empty_phase ^= 1u << st;
                }
                if (lane == 0) mbar_arrive_expect_tx(&s_full[st], plane_bytes);
                __syncwarp();
                tma_issue_plane<T, NF, KAHAN>(lane, stage + st * A.stage_stride, arr_stride, F, N, zz, y0, R, ylo, yhi,
                                              &s_full[st]);
                __syncwarp();
                ++issued;
                st = st + 1 == S ? 0 : st + 1;
                zz = zz + 1 == N ? 0 : zz + 1;
            }
        }
    } else {
        int st = 0, st_prev = 0;
        uint32_t full_phase = 0;
        int rnew = 0, rmid = RING - 1;
        const int lane = tid & 31;
        auto release = [&](int s_idx) {
            __syncwarp();
            if (lane == 0) mbar_arrive(&s_empty[s_idx]);
        };
        ZMarch<T, NF, VW> Z;
        for (int k = blockIdx.x; k < A.item_end - A.item_begin; k += gridDim.x) {
            const int it = A.sched ? A.sched[k] : A.item_begin + k;
            const EnsItem I = A.items[it];
            const EnsMember& M = A.members[I.member];
            const int N = M.N, BY = M.BY, y0 = I.y0, z0 = I.z0;
            const int R = min(BY, N - y0), NZ = min(M.DZ, N - z0);
            const double dx = M.dx;
            DevScal* Sm = A.scal + I.member;
            pass_coefficients_warps(tid, Sm->a, Sm->b, A.d, A.alpha, dx, expand, s_coef);
            named_barrier_sync(2, CT);
            const TileCoef<T> C{(T)s_coef[0], (T)s_coef[1], (T)s_coef[2], (T)A.e, (T)A.k};
            const PotCoef<T> P(M.m2, M.lam, M.g2);
            const OutArrays<EnsPassArgs<T>> Out{A, M.off};
            const TileGeom G(N, VW, BY, R, tid);
            const size_t plane = (size_t)N * N;
            const size_t row_off = (size_t)(y0 + G.r) * N + G.x0;
            Acc<T> accK[NF], accG[NF], accV;
            int zz = z0 == 0 ? N - 1 : z0 - 1;
            for (int j = 0; j < NZ + 2; ++j) {
                if (!mbar_wait_bounded(&s_full[st], (full_phase >> st) & 1u, s_timeout ? 1000000ull : 2000000000ull))
                    s_timeout = 1;
                full_phase ^= 1u << st;
                if constexpr (NR) {
                    tma_consume_plane_nr<T, NF, KAHAN, VW>(G, stage + st * A.stage_stride,
                                                           stage + st_prev * A.stage_stride, do_drift,
                                                           j >= 1 && j <= NZ, j >= 2, (size_t)zz * plane + row_off,
                                                           (size_t)(z0 + j - 2) * plane + row_off, Out, C, P, Z, accK,
                                                           accG, accV);
                    if (j >= 1) release(st_prev);  // plane j-1: kicked (or the lower z halo, never kicked)
                } else {
                    tma_consume_plane<T, NF, KAHAN, VW>(G, stage + st * A.stage_stride, ring + rnew * A.ring_slot,
                                                        ring + rmid * A.ring_slot, tid, CT, do_drift,
                                                        j >= 1 && j <= NZ, j >= 2, (size_t)zz * plane + row_off,
                                                        (size_t)(z0 + j - 2) * plane + row_off, Out, C, P, Z, accK,
                                                        accG, accV, &s_empty[st]);
                    rmid = rnew;
                    rnew = rnew + 1 == RING ? 0 : rnew + 1;
                }
                st_prev = st;
                st = st + 1 == S ? 0 : st + 1;
                zz = zz + 1 == N ? 0 : zz + 1;
            }
            if constexpr (NR) release(st_prev);  // the upper z halo of the item is never kicked
            // item partials; the member's last item reduces them in a fixed order
            double v[kMaxQ];
            const Acc<T>* av[kMaxQ] = {&accK[0], NF > 1 ? &accK[NF - 1] : nullptr, &accG[0],
                                       NF > 1 ? &accG[NF - 1] : nullptr, &accV};
            group_reduce_acc<T, kMaxQ>(av, v, s_red, tid, CT, 2);
            if (tid == 0) {
#pragma unroll
                for (int q = 0; q < kMaxQ; ++q) A.partials[(size_t)it * kMaxQ + q] = v[q];
                __threadfence();
                const unsigned prev = atomicAdd(&Sm->counter, 1u);
                s_last = (prev + 1u == (unsigned)M.nitems);
            }
            named_barrier_sync(2, CT);
            if (s_last && tid < 32) {  // uniform over the consumers; one warp sums the item partials
                __threadfence();
                double w[kMaxQ];
                warp_sum_partials<kMaxQ>(A.partials + (size_t)M.item0 * kMaxQ, M.nitems, tid, w);
                if (tid == 0)
                    scalar_epilogue(Sm, w, (double)N * N * N, dx, s_coef[3], A.alpha, A.kappa, A.d, A.e, A.k, A.flags,
                                    A.hubble_limit);
            }
            named_barrier_sync(2, CT);  // s_coef, s_red and s_last are rewritten by the next item
        }
    }
    __syncthreads();  // producer and consumers meet; no copy is in flight past this point
    if (tid == 0 && s_timeout) atomicOr(&A.scal[0].status, ST_TIMEOUT);
}

template <typename K>
static cudaError_t ens_smem_attr(K kernel)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kPassMaxSmem);
}

template <typename K, typename T>
static cudaError_t ens_launch(K kernel, int threads, const void* args, int grid, size_t smem, cudaStream_t s,
                              int* occ, DevFlag& attr)
{
    if (!attr) {
        cudaError_t e = ens_smem_attr(kernel);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    if (occ) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, kernel, threads, smem);
    kernel<<<grid, threads, smem, s>>>(*static_cast<const EnsPassArgs<T>*>(args));
    return cudaGetLastError();
}

// stages: 0 = direct loader, 2..4 = TMA stage buffers with the ring, 3..6 ringless (variant 1)
template <typename T, int NF, bool KAHAN, int VW>
static cudaError_t ens_one(const void* args, int stages, int variant, int grid, size_t smem, cudaStream_t s, int* occ)
{
    static DevFlag attr[2][7];
    if (stages <= 0) return ens_launch<decltype(&k_ensemble_pass<T, NF, KAHAN, VW>), T>(
        k_ensemble_pass<T, NF, KAHAN, VW>, kEnsThreads, args, grid, smem, s, occ, attr[0][0]);
    if constexpr (VW * sizeof(T) == 16) {  // 16-byte vectors: every member row is a 16-byte multiple
#define CL_ENS_CASE(SS, NRV)                                                                                  \
        if (stages == SS && variant == (NRV ? 1 : 0))                                                        \
            return ens_launch<decltype(&k_ensemble_pass_tma<T, NF, KAHAN, VW, SS, NRV>), T>(                 \
                k_ensemble_pass_tma<T, NF, KAHAN, VW, SS, NRV>, kEnsTmaThreads, args, grid, smem, s, occ,    \
                attr[NRV ? 1 : 0][SS]);
        CL_ENS_CASE(2, false)
        CL_ENS_CASE(3, false)
        CL_ENS_CASE(4, false)
        CL_ENS_CASE(3, true)
        CL_ENS_CASE(4, true)
        CL_ENS_CASE(5, true)
        CL_ENS_CASE(6, true)
#undef CL_ENS_CASE
    }
    return cudaErrorInvalidValue;
}

template <typename T, int NF, bool KAHAN>
static cudaError_t ens_vw(const void* args, int vw, int stages, int variant, int grid, size_t smem, cudaStream_t s,
                          int* occ)
{
    if (vw == 1) return ens_one<T, NF, KAHAN, 1>(args, stages, variant, grid, smem, s, occ);
    if (vw == 2) return ens_one<T, NF, KAHAN, 2>(args, stages, variant, grid, smem, s, occ);
    if constexpr (sizeof(T) == 4) {
        if (vw == 4) return ens_one<T, NF, KAHAN, 4>(args, stages, variant, grid, smem, s, occ);
    }
    return cudaErrorInvalidValue;
}

static cudaError_t ens_dispatch(int precision, int nf, const void* args, int vw, int stages, int variant, int grid,
                                size_t smem, cudaStream_t s, int* occ)
{
    if (precision == CL_PREC_FP64)
        return nf == 1 ? ens_vw<double, 1, false>(args, vw, stages, variant, grid, smem, s, occ)
                       : ens_vw<double, 2, false>(args, vw, stages, variant, grid, smem, s, occ);
    if (precision == CL_PREC_FP32_KAHAN)
        return nf == 1 ? ens_vw<float, 1, true>(args, vw, stages, variant, grid, smem, s, occ)
                       : ens_vw<float, 2, true>(args, vw, stages, variant, grid, smem, s, occ);
    return nf == 1 ? ens_vw<float, 1, false>(args, vw, stages, variant, grid, smem, s, occ)
                   : ens_vw<float, 2, false>(args, vw, stages, variant, grid, smem, s, occ);
}

cudaError_t launch_ensemble_pass(int precision, int nf, const void* args, int vw, int grid, size_t smem,
                                 cudaStream_t s)
{
    if (grid < 1) return cudaSuccess;
    int stages, variant;
    if (precision == CL_PREC_FP64) {
        const auto* A = static_cast<const EnsPassArgs<double>*>(args);
        stages = A->stages;
        variant = A->variant;
    } else {
        const auto* A = static_cast<const EnsPassArgs<float>*>(args);
        stages = A->stages;
        variant = A->variant;
    }
    return ens_dispatch(precision, nf, args, vw, stages, variant, grid, smem, s, nullptr);
}

cudaError_t ensemble_pass_blocks_per_sm(int precision, int nf, int vw, int stages, int variant, size_t smem,
                                        int* blocks)
{
    return ens_dispatch(precision, nf, nullptr, vw, stages, variant, 0, smem, nullptr, blocks);
}

}  // namespace clk
