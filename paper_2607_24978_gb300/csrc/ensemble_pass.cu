// Fused scalar pass over a batched ensemble of independent lattices (sm_103a).
//
// Many small lattices (each with its own size, box, couplings, a and a') advance by one
// pass of the staggered kick-drift scheme in a single persistent launch.  The work is a
// table of items, each BY full x rows times DZ planes of one member; block b takes items
// b, b + grid, b + 2 grid, ... and runs the same per-site arithmetic as the
// single-lattice direct loader on it (drift while loading, stencil kick, energies).
// Reductions: every item writes its FP64 partial sums; the block that completes the last
// item of a member (an arrival counter per member) sums that member's partials in a fixed
// order and runs the member's scale-factor epilogue.  Reading a, a' happens at item
// start, before the item's arrival, so the epilogue never races a reader.
#include <math.h>

#include "cl_internal.cuh"
#include "kernel_common.cuh"
#include "scalar_pass_common.cuh"

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

    for (int it = A.item_begin + blockIdx.x; it < A.item_end; it += gridDim.x) {
        const EnsItem I = A.items[it];
        const EnsMember& M = A.members[I.member];
        const int N = M.N, BY = M.BY;
        const double dx = M.dx;
        DevScal* S = A.scal + I.member;
        if (tid == 0) pass_coefficients(S->a, S->b, A.d, A.alpha, dx, expand, s_coef);
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
        v[0] = accK[0].value();
        v[1] = NF > 1 ? accK[NF - 1].value() : 0.0;
        v[2] = accG[0].value();
        v[3] = NF > 1 ? accG[NF - 1].value() : 0.0;
        v[4] = accV.value();
        block_reduce<kMaxQ>(v, s_red, tid, nthr);
        if (tid == 0) {
#pragma unroll
            for (int q = 0; q < kMaxQ; ++q) A.partials[(size_t)it * kMaxQ + q] = v[q];
            __threadfence();
            const unsigned prev = atomicAdd(&S->counter, 1u);
            s_last = (prev + 1u == (unsigned)M.nitems);
        }
        __syncthreads();
        if (s_last) {  // block-uniform
            __threadfence();
            double w[kMaxQ];
#pragma unroll
            for (int q = 0; q < kMaxQ; ++q) w[q] = 0.0;
            for (int b = tid; b < M.nitems; b += nthr)
#pragma unroll
                for (int q = 0; q < kMaxQ; ++q) w[q] += __ldcg(&A.partials[(size_t)(M.item0 + b) * kMaxQ + q]);
            block_reduce<kMaxQ>(w, s_red, tid, nthr);
            if (tid == 0)
                scalar_epilogue(S, w, (double)N * N * N, dx, s_coef[3], A.alpha, A.kappa, A.d, A.e, A.k, A.flags,
                                A.hubble_limit);
        }
        __syncthreads();  // s_coef and s_last are rewritten by the next item
    }
}

template <typename K>
static cudaError_t ens_smem_attr(K kernel)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kPassMaxSmem);
}

template <typename T, int NF, bool KAHAN, int VW>
static cudaError_t ens_one(const void* args, int grid, size_t smem, cudaStream_t s, int* occ)
{
    auto kernel = k_ensemble_pass<T, NF, KAHAN, VW>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = ens_smem_attr(kernel);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    if (occ) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, kernel, kEnsThreads, smem);
    kernel<<<grid, kEnsThreads, smem, s>>>(*static_cast<const EnsPassArgs<T>*>(args));
    return cudaGetLastError();
}

template <typename T, int NF, bool KAHAN>
static cudaError_t ens_vw(const void* args, int vw, int grid, size_t smem, cudaStream_t s, int* occ)
{
    if (vw == 1) return ens_one<T, NF, KAHAN, 1>(args, grid, smem, s, occ);
    if (vw == 2) return ens_one<T, NF, KAHAN, 2>(args, grid, smem, s, occ);
    if constexpr (sizeof(T) == 4) {
        if (vw == 4) return ens_one<T, NF, KAHAN, 4>(args, grid, smem, s, occ);
    }
    return cudaErrorInvalidValue;
}

static cudaError_t ens_dispatch(int precision, int nf, const void* args, int vw, int grid, size_t smem,
                                cudaStream_t s, int* occ)
{
    if (precision == CL_PREC_FP64)
        return nf == 1 ? ens_vw<double, 1, false>(args, vw, grid, smem, s, occ)
                       : ens_vw<double, 2, false>(args, vw, grid, smem, s, occ);
    if (precision == CL_PREC_FP32_KAHAN)
        return nf == 1 ? ens_vw<float, 1, true>(args, vw, grid, smem, s, occ)
                       : ens_vw<float, 2, true>(args, vw, grid, smem, s, occ);
    return nf == 1 ? ens_vw<float, 1, false>(args, vw, grid, smem, s, occ)
                   : ens_vw<float, 2, false>(args, vw, grid, smem, s, occ);
}

cudaError_t launch_ensemble_pass(int precision, int nf, const void* args, int vw, int grid, size_t smem,
                                 cudaStream_t s)
{
    if (grid < 1) return cudaSuccess;
    return ens_dispatch(precision, nf, args, vw, grid, smem, s, nullptr);
}

cudaError_t ensemble_pass_blocks_per_sm(int precision, int nf, int vw, size_t smem, int* blocks)
{
    return ens_dispatch(precision, nf, nullptr, vw, 0, smem, nullptr, blocks);
}

}  // namespace clk
