// CUDA-core pieces of the convolutional surrogate: the thin first and last layers (3 -> C
// and C -> 2 channels, with the residual jump), their data gradients, the FP32 reference
// mode of every layer, and the weight / bias gradients.  Conventions in
// surrogate_common.cuh.
#include <cuda_bf16.h>
#include <stdint.h>

#include "cl_internal.cuh"
#include "kernel_common.cuh"
#include "surrogate_common.cuh"

namespace clk {

__device__ __forceinline__ float load_act(const void* p, int bf16, size_t i)
{
    return bf16 ? __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(p)[i]) : reinterpret_cast<const float*>(p)[i];
}

template <int COUT>
__global__ void __launch_bounds__(128) k_conv_cc(const ConvCCArgs A)
{
    const uint32_t N = (uint32_t)A.N, V = N * N * N;
    const int cin = A.cin;
    for (uint32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < V; n += gridDim.x * blockDim.x) {
        const uint32_t x = n % N, r = n / N, y = r % N, z = r / N;
        float acc[COUT];
#pragma unroll
        for (int co = 0; co < COUT; ++co) acc[co] = A.bias ? __ldg(A.bias + co) : 0.f;
        for (int t = 0; t < 27; ++t) {
            const uint32_t xs = (x + N + t % 3 - 1) % N, ys = (y + N + (t / 3) % 3 - 1) % N, zs = (z + N + t / 9 - 1) % N;
            const size_t m = ((size_t)zs * N + ys) * N + xs;
            for (int ci = 0; ci < cin; ++ci) {
                const float v = act_f(A.in_act, load_act(A.in, A.in_bf16, m * cin + ci));
                const float* w = A.flip ? A.w + ((size_t)(26 - t) * cin + ci) * COUT : A.w + (size_t)t * COUT * cin + ci;
#pragma unroll
                for (int co = 0; co < COUT; ++co) acc[co] += __ldg(A.flip ? w + co : w + (size_t)co * cin) * v;
            }
        }
        if (A.resid) {
            for (int co = 0; co < A.resid_c && co < COUT; ++co) acc[co] += A.resid[(size_t)n * A.resid_stride + co];
        }
        if (A.gate_act) {
#pragma unroll
            for (int co = 0; co < COUT; ++co)
                acc[co] *= act_grad_f(A.gate_act, load_act(A.gate, A.gate_bf16, (size_t)n * COUT + co));
        }
        if (A.out_bf16) {
            __nv_bfloat16* o = reinterpret_cast<__nv_bfloat16*>(A.out) + (size_t)n * COUT;
#pragma unroll
            for (int co = 0; co < COUT; ++co) o[co] = __float2bfloat16_rn(acc[co]);
        } else {
            float* o = reinterpret_cast<float*>(A.out) + (size_t)n * COUT;
#pragma unroll
            for (int co = 0; co < COUT; ++co) o[co] = acc[co];
        }
    }
}

cudaError_t launch_conv_cc(const ConvCCArgs& A, cudaStream_t s)
{
    const int64_t V = (int64_t)A.N * A.N * A.N;
    int64_t blocks = (V + 127) / 128;
    if (blocks > 152 * 32) blocks = 152 * 32;
    const int g = (int)blocks;
    switch (A.cout) {
    case 2: k_conv_cc<2><<<g, 128, 0, s>>>(A); break;
    case 3: k_conv_cc<3><<<g, 128, 0, s>>>(A); break;
    case 16: k_conv_cc<16><<<g, 128, 0, s>>>(A); break;
    case 32: k_conv_cc<32><<<g, 128, 0, s>>>(A); break;
    case 48: k_conv_cc<48><<<g, 128, 0, s>>>(A); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- weight gradients
constexpr int kDwSites = 32;  // sites staged per batch

// Block (chunk c, tap t): partial[c][t][co][ci] over the chunk's sites; blocks of tap 0
// also write the bias partials partial[c][27 * cout * cin + co].
__global__ void __launch_bounds__(256) k_conv_dw(const ConvDWArgs A)
{
    extern __shared__ float sdw[];
    const int cin = A.cin, cout = A.cout;
    float* gs = sdw;                      // [kDwSites][cout]
    float* hs = sdw + kDwSites * cout;    // [kDwSites][cin]
    const uint32_t N = (uint32_t)A.N, V = N * N * N;
    const int c = blockIdx.x, t = blockIdx.y;
    const uint32_t s0 = (uint32_t)((uint64_t)V * c / A.chunks), s1 = (uint32_t)((uint64_t)V * (c + 1) / A.chunks);
    const int ox = t % 3 - 1, oy = (t / 3) % 3 - 1, oz = t / 9 - 1;
    const int npair = cout * cin;
    constexpr int PMAX = 9;  // pairs per thread: cout * cin <= 256 * 9
    float acc[PMAX], bacc = 0.f;
#pragma unroll
    for (int k = 0; k < PMAX; ++k) acc[k] = 0.f;
    for (uint32_t b = s0; b < s1; b += kDwSites) {
        const int nb = (int)min((uint32_t)kDwSites, s1 - b);
        for (int i = threadIdx.x; i < nb * cout; i += blockDim.x) {
            const int s = i / cout, co = i - s * cout;
            gs[i] = load_act(A.g, A.g_bf16, (size_t)(b + s) * cout + co);
        }
        for (int i = threadIdx.x; i < nb * cin; i += blockDim.x) {
            const int s = i / cin, ci = i - s * cin;
            const uint32_t n = b + s;
            const uint32_t x = n % N, r = n / N, y = r % N, z = r / N;
            const uint32_t m = (((z + N + oz) % N) * N + (y + N + oy) % N) * N + (x + N + ox) % N;
            hs[i] = act_f(A.h_act, load_act(A.h, A.h_bf16, (size_t)m * cin + ci));
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < PMAX; ++k) {
            const int p = threadIdx.x + k * blockDim.x;
            if (p < npair) {
                const int co = p / cin, ci = p - co * cin;
                float a = acc[k];
                for (int s = 0; s < nb; ++s) a += gs[s * cout + co] * hs[s * cin + ci];
                acc[k] = a;
            }
        }
        if (t == 0 && (int)threadIdx.x < cout)
            for (int s = 0; s < nb; ++s) bacc += gs[s * cout + threadIdx.x];
        __syncthreads();
    }
    float* P = A.partial + (size_t)c * (27 * npair + cout);
#pragma unroll
    for (int k = 0; k < PMAX; ++k) {
        const int p = threadIdx.x + k * blockDim.x;
        if (p < npair) P[(size_t)t * npair + p] = acc[k];
    }
    if (t == 0 && (int)threadIdx.x < cout) P[27 * npair + threadIdx.x] = bacc;
}

__global__ void k_conv_dw_reduce(const ConvDWArgs A)
{
    const int npair = A.cout * A.cin, total = 27 * npair + A.cout;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int c = 0; c < A.chunks; ++c) s += A.partial[(size_t)c * total + i];  // fixed order
        if (i < 27 * npair) A.dW[i] = s;
        else A.db[i - 27 * npair] = s;
    }
}

int conv_dw_chunks(int N)
{
    const int64_t V = (int64_t)N * N * N;
    int64_t c = V / 4096;  // at least 4096 sites per chunk
    if (c < 1) c = 1;
    if (c > 24) c = 24;    // 27 x 24 blocks: about four waves
    return (int)c;
}

cudaError_t launch_conv_dw(const ConvDWArgs& A, cudaStream_t s)
{
    if (A.cout * A.cin > 256 * 9) return cudaErrorInvalidValue;
    const size_t smem = sizeof(float) * kDwSites * (A.cout + A.cin);
    k_conv_dw<<<dim3(A.chunks, 27), 256, smem, s>>>(A);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int total = 27 * A.cout * A.cin + A.cout;
    k_conv_dw_reduce<<<(total + 255) / 256, 256, 0, s>>>(A);
    return cudaGetLastError();
}

}  // namespace clk
