// Weight gradients of a hidden surrogate layer (C -> C channels, C = 16, 32 or 48) on the
// tensor cores (tcgen05, BF16 operands, FP32 accumulation in TMEM):
//
//   dW[t][co][ci] = sum_n g[n][co] h[n + o(t)][ci],    t = (tz*3 + ty)*3 + tx, o = (tx-1, ty-1, tz-1)
//
// with g the gradient of the layer's output and h its (activated) input, both BF16
// [site][C].  The sites are the reduction (K) dimension, so both operands are read
// MN-major: shared memory holds 16-byte entries (8 channels of one site) laid out
// [channel group][site], where eight consecutive sites form one 128-byte core matrix and
// a one-site shift of a tap is a 16-byte shift of the descriptor's start address.
//
// A work unit is one x row (z, y) of N sites, split into K chunks of 16 sites.  Per chunk
// and x tap (three MMAs, M = 128, N = 3C, K = 16):
//  * B (N rows) is h of the three rows y-1, y, y+1 of one plane, staged [row][group][x]
//    with a one-site periodic halo in x: the 3C rows (y tap, input channel) are evenly
//    strided, so the three y taps are one MMA;
//  * A (M = 128 rows) is g of row (z, y) in rows 0-63 (channels padded to 64 with zeros)
//    and, in the first block group, g of row (z-1, y) in rows 64-127.
// The first group stages h of plane z-1: rows 0-63 accumulate the tz = 0 taps of output
// plane z and rows 64-127 the tz = 1 taps of plane z-1 (each plane is the z-1 of exactly
// one unit, periodic in z).  The second group stages h of plane z+1 (tz = 2; its rows
// 64-127 stay zero).  A block accumulates its units in TMEM (three x taps x 3C columns)
// and writes one partial per tap; a second kernel sums the partials in a fixed order.
//
// Warp roles, synchronised by mbarriers only: warp 0, lane 0 issues the MMAs; warps 1-3
// stage units with cp.async into a ring of slots; warps 4-7 read the accumulators back at
// the end.  All waits are bounded and report through the status word.
#include <cuda_bf16.h>
#include <stdint.h>

#include "cl_internal.cuh"
#include "kernel_common.cuh"
#include "surrogate_common.cuh"
#include "tcgen05_ops.cuh"

namespace clk {

constexpr int kDwMaxSlots = 4;
constexpr int kDwStage = 96;  // staging threads (warps 1-3)

// 16-byte entries of one slot: A (16 channel blocks of N + 1 sites, the +1 spreads the
// blocks over the shared-memory banks) and B (3 rows x C/8 groups x N + 2 sites).
__host__ __device__ inline int dw_a_entries(int N) { return 16 * (N + 1); }
__host__ __device__ inline int dw_slot_entries(int C, int N) { return dw_a_entries(N) + 3 * (C / 8) * (N + 2); }

template <int C>
struct DwTCShape {
    static constexpr int CG = C / 8;        // channel groups of a site
    static constexpr int NT = 3 * C;        // MMA N: three y taps x C input channels
    static constexpr int TMEM_COLS = 3 * NT <= 256 ? 256 : 512;  // three x taps
};

template <int C>
__global__ void __launch_bounds__(256, 1) k_conv_dw_tc(const ConvDWTCArgs A)
{
    using S = DwTCShape<C>;
    constexpr int CG = S::CG, NT = S::NT;
    extern __shared__ __align__(128) uint4 smem[];
    __shared__ __align__(8) uint64_t s_full[kDwMaxSlots];   // unit staged in the slot (96 arrivals)
    __shared__ __align__(8) uint64_t s_freeb[kDwMaxSlots];  // slot's unit read by its MMAs (commit)
    __shared__ __align__(8) uint64_t s_done;                // every MMA of the block complete (commit)
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = A.N, NS = A.nslot, grp = blockIdx.y;
    const int AST = N + 1, BST = N + 2;  // entries between channel blocks of A, groups of B
    const int AENT = dw_a_entries(N), SLOT = dw_slot_entries(C, N);
    const long long units = (long long)N * N;
    const long long u0 = units * blockIdx.x / gridDim.x, u1 = units * (blockIdx.x + 1) / gridDim.x;
    const int nblk_a = grp == 0 ? 2 : 1;  // g rows staged into A (rows 0-63, and 64-127)

    // zero the padding channel blocks of A once: the staging warps never write them
    for (int s = 0; s < NS; ++s) {
        uint4* sa = smem + (size_t)s * SLOT;
        for (int e = tid; e < 16 * AST; e += blockDim.x) {
            const int b = e / AST;
            const bool used = (b < CG) || (nblk_a == 2 && b >= 8 && b < 8 + CG);
            if (!used) sa[e] = make_uint4(0u, 0u, 0u, 0u);
        }
    }
    if (tid == 0) {
        for (int k = 0; k < NS; ++k) {
            mbar_init(&s_full[k], kDwStage);
            mbar_init(&s_freeb[k], 1);
        }
        mbar_init(&s_done, 1);
        mbar_fence_init();
        s_fail = 0;
    }
    if (warp == 0) {
        tmem_alloc(&s_tmem, S::TMEM_COLS);
        tmem_relinquish();
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = s_tmem;
    auto wait = [&](uint64_t* bar, uint32_t& phases, int bit) {
        if (!mbar_wait_bounded(bar, (phases >> bit) & 1u, s_fail ? 1000000ull : 2000000000ull)) s_fail = 1;
        phases ^= 1u << bit;
    };

    if (warp == 0) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint32_t full_ph = 0;
            int seq = 0;
            constexpr uint32_t idesc = idesc_bf16_mn(128, NT);
            const uint32_t sbo_a = (uint32_t)AST * 16, sbo_b = (uint32_t)BST * 16;
            for (long long u = u0; u < u1; ++u, ++seq) {
                const int slot = seq % NS;
                wait(&s_full[slot], full_ph, slot);
                tc_fence_after();
                const uint32_t a0 = smem_u32(smem + (size_t)slot * SLOT), b0 = a0 + (uint32_t)AENT * 16;
#pragma unroll 1
                for (int kc = 0; kc < N / 16; ++kc) {
                    const uint64_t adesc = smem_desc(a0 + kc * 256, 128, sbo_a);
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx)
                        tc_mma(tbase + dx * NT, adesc, smem_desc(b0 + (kc * 16 + dx) * 16, 128, sbo_b), idesc,
                               (u == u0 && kc == 0) ? 0u : 1u);
                }
                tc_commit(&s_freeb[slot]);  // the slot may be restaged once these MMAs completed
            }
            if (u1 > u0) tc_commit(&s_done);
        }
        __syncwarp();
    } else if (warp < 4) {
        // ------------------------------------------------------------ staging warps
        const int st = tid - 32;
        const __nv_bfloat16* g = A.g;
        const __nv_bfloat16* h = A.h;
        const int dzh = grp == 0 ? -1 : 1;  // plane of h relative to the unit
        uint32_t free_ph = 0;
        int seq = 0, pend_slot = -1;
        const int na = nblk_a * CG * N, nb = 3 * CG * BST;
        auto land = [&](int slot) {
            fence_proxy_async_smem();
            mbar_arrive(&s_full[slot]);
        };
        for (long long u = u0; u < u1; ++u, ++seq) {
            const int slot = seq % NS;
            if (seq >= NS) wait(&s_freeb[slot], free_ph, slot);
            const int z = (int)(u / N), y = (int)(u - (long long)z * N);
            uint4* sa = smem + (size_t)slot * SLOT;
            uint4* sb = sa + AENT;
            // A: g of row (z, y) into channel blocks 0.., and of row (z-1, y) into blocks 8..
            for (int e = st; e < na; e += kDwStage) {
                const int half = e / (CG * N), r = e - half * (CG * N);
                const int cg = r % CG, x = r / CG;
                const int zz = half == 0 ? z : (z == 0 ? N - 1 : z - 1);
                const size_t site = ((size_t)zz * N + y) * N + x;
                cp_async16(sa + (half * 8 + cg) * AST + x, g + site * C + cg * 8);
            }
            // B: h of rows y-1, y, y+1 of plane z + dzh, x from -1 to N (periodic)
            const int zh = (z + dzh + N) % N;
            for (int e = st; e < nb; e += kDwStage) {
                const int cg = e % CG, r = e / CG;
                const int p = r % BST, dy = r / BST;
                const int yy = (y + dy - 1 + N) % N, xx = p == 0 ? N - 1 : (p == N + 1 ? 0 : p - 1);
                const size_t site = ((size_t)zh * N + yy) * N + xx;
                cp_async16(sb + (dy * CG + cg) * BST + p, h + site * C + cg * 8);
            }
            cp_async_commit();
            if (pend_slot >= 0) {  // the previous unit's copies have landed once one group is left
                cp_async_wait1();
                land(pend_slot);
            }
            pend_slot = slot;
        }
        if (pend_slot >= 0) {
            cp_async_wait0();
            land(pend_slot);
        }
    } else {
        // ------------------------------------------------------------ epilogue warps
        const int q = warp & 3;           // TMEM lane quarter of this warp
        const int r = 32 * q + lane;      // accumulator row
        const int half = r >> 6, co = r & 63;
        const bool any = u1 > u0;
        uint32_t done_ph = 0;
        if (any) {
            wait(&s_done, done_ph, 0);
            tc_fence_after();
        }
        const bool valid = co < C && (grp == 0 || half == 0);
        float* P = grp == 0 ? A.part0 + (size_t)blockIdx.x * 18 * C * C : A.part1 + (size_t)blockIdx.x * 9 * C * C;
#pragma unroll 1
        for (int dx = 0; dx < 3; ++dx) {
#pragma unroll 1
            for (int c16 = 0; c16 < NT / 16; ++c16) {
                uint32_t raw[16];
                if (any) {
                    tmem_ld16(tbase + ((uint32_t)(32 * q) << 16) + dx * NT + c16 * 16, raw);
                    tmem_wait<16>(raw);
                } else {
#pragma unroll
                    for (int e = 0; e < 16; ++e) raw[e] = 0u;
                }
                if (valid) {
                    const int col = c16 * 16, dy = col / C, ci0 = col - dy * C;
                    const int tl = (half * 3 + dy) * 3 + dx;  // tap within the group's planes
                    float4* o = reinterpret_cast<float4*>(P + ((size_t)tl * C + co) * C + ci0);
#pragma unroll
                    for (int v = 0; v < 4; ++v)
                        o[v] = make_float4(__uint_as_float(raw[4 * v]), __uint_as_float(raw[4 * v + 1]),
                                           __uint_as_float(raw[4 * v + 2]), __uint_as_float(raw[4 * v + 3]));
                }
            }
        }
        tc_fence_before();
    }
    __syncthreads();  // the epilogue waited for every MMA; no copy is in flight
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tbase, S::TMEM_COLS);
    if (tid == 0 && s_fail) atomicOr(A.status, ST_TIMEOUT);
}

// dW[t] = sum over the blocks of the group owning plane tz of their partials (fixed order);
// db[co] = sum over the bias partials (fixed order).
__global__ void k_conv_dw_tc_reduce(const ConvDWTCArgs A, int C)
{
    const int cc = C * C, total = 27 * cc + C;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        if (i < 18 * cc) {
            float s = 0.f;
            for (int b = 0; b < A.nb; ++b) s += A.part0[(size_t)b * 18 * cc + i];
            A.dW[i] = s;
        } else if (i < 27 * cc) {
            float s = 0.f;
            for (int b = 0; b < A.nb; ++b) s += A.part1[(size_t)b * 9 * cc + (i - 18 * cc)];
            A.dW[i] = s;
        } else {
            const int co = i - 27 * cc;
            double s = 0.0;
            for (int b = 0; b < A.nbias; ++b) s += A.bpart[(size_t)b * C + co];
            A.db[co] = (float)s;
        }
    }
}

// Bias gradient partials: block b sums g[n][co] over its range of sites (FP64).
__global__ void __launch_bounds__(256) k_conv_db_partial(const ConvDWTCArgs A, int C)
{
    __shared__ double s_acc[256];
    const long long V = (long long)A.N * A.N * A.N;
    const long long s0 = V * blockIdx.x / gridDim.x, s1 = V * (blockIdx.x + 1) / gridDim.x;
    const int lanes = 256 / C;  // threads per channel
    const int co = threadIdx.x % C, k = threadIdx.x / C;
    double acc = 0.0;
    if (k < lanes)
        for (long long n = s0 + k; n < s1; n += lanes) acc += (double)__bfloat162float(A.g[n * C + co]);
    s_acc[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < C) {
        double s = 0.0;
        for (int j = 0; j < lanes; ++j) s += s_acc[j * C + threadIdx.x];  // fixed order
        A.bpart[(size_t)blockIdx.x * C + threadIdx.x] = s;
    }
}

size_t conv_dw_tc_smem(int C, int N, int nslot) { return (size_t)nslot * dw_slot_entries(C, N) * 16; }

int conv_dw_tc_slots(int C, int N)
{
    if ((C != 16 && C != 32 && C != 48) || N < 16 || N % 16 != 0) return 0;
    for (int s = kDwMaxSlots; s >= 2; --s)
        if (conv_dw_tc_smem(C, N, s) <= (size_t)kPassMaxSmem) return s;
    return 0;
}

template <int C>
static cudaError_t launch_dw_tc_t(const ConvDWTCArgs& A, cudaStream_t s)
{
    const size_t smem = conv_dw_tc_smem(C, A.N, A.nslot);
    cudaError_t e = cudaFuncSetAttribute(k_conv_dw_tc<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_conv_dw_tc<C><<<dim3(A.nb, 2), 256, smem, s>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_conv_dw_tc(int C, const ConvDWTCArgs& A, cudaStream_t s)
{
    if (A.nslot < 2 || A.nslot > kDwMaxSlots || A.nslot > conv_dw_tc_slots(C, A.N) || A.nb < 1 || A.nbias < 1 ||
        C * C * 27 + C > (1 << 30))
        return cudaErrorInvalidValue;
    cudaError_t e;
    switch (C) {
    case 16: e = launch_dw_tc_t<16>(A, s); break;
    case 32: e = launch_dw_tc_t<32>(A, s); break;
    case 48: e = launch_dw_tc_t<48>(A, s); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    k_conv_db_partial<<<A.nbias, 256, 0, s>>>(A, C);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int total = 27 * C * C + C;
    k_conv_dw_tc_reduce<<<(total + 255) / 256, 256, 0, s>>>(A, C);
    return cudaGetLastError();
}

}  // namespace clk
