// Tensor-core (tcgen05) periodic 3x3x3 convolution of the surrogate's hidden layers,
// C input and C output channels (C = 16, 32 or 48), BF16 operands, FP32 accumulation.
//
// Implicit GEMM: for an 8 x 16 (x, y) tile of output sites of one plane, D[128 x C] =
// sum over the 27 taps and the C/16 K-chunks of A_tap[128 x 16] B_tap[16 x C], one
// tcgen05.mma (M = 128, N = C, K = 16) each.  Rows of A are output sites (row = x + 8 y),
// so the A operand of a tap is the staged input plane read at an (x, y) offset: the input
// planes live in shared memory as 16-byte entries (8 channels of one site) laid out
// [channel group][y][x] over the tile plus a one-site halo, which is the no-swizzle
// K-major core-matrix layout (eight consecutive x form one 128-byte core matrix; the
// next channel group is the next core matrix along K, the next y row the next along M).
// Every tap is therefore only a different descriptor start address.  The weights of all
// 27 taps stay in shared memory for the whole kernel in the same layout
// ([tap][channel-in group][channel-out group][8 out][8 in]).
//
// A block owns tiles of z-columns: it stages the input planes z-1, z, z+1 into a ring of
// four slots and marches up z.  One thread issues the 27 C/16 MMAs of a plane into one of
// two TMEM accumulators and commits them to that accumulator's mbarrier; meanwhile all
// threads stage plane z+2 and read back (tcgen05.ld) the previous plane's accumulator,
// finish it (bias, or the activation derivative of the backward pass) and store it as
// BF16.  All mbarrier waits are bounded and report through the status word.
#include <cuda_bf16.h>
#include <stdint.h>

#include "cl_internal.cuh"
#include "kernel_common.cuh"
#include "surrogate_common.cuh"

namespace clk {

// ---------------------------------------------------------------- tcgen05 wrappers
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[smem] B[smem], kind::f16 (BF16 x BF16 -> FP32), issued by one thread.
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// Arrive on `bar` once every MMA issued so far by this thread has completed.
__device__ __forceinline__ void tc_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// Eight consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8])
{
    uint32_t r0, r1, r2, r3, r4, r5, r6, r7;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3), "=r"(r4), "=r"(r5), "=r"(r6), "=r"(r7)
                 : "r"(taddr));
    // the registers are valid only after the wait; tie them to it
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r0), "+r"(r1), "+r"(r2), "+r"(r3), "+r"(r4), "+r"(r5), "+r"(r6), "+r"(r7)::"memory");
    v[0] = __uint_as_float(r0); v[1] = __uint_as_float(r1); v[2] = __uint_as_float(r2); v[3] = __uint_as_float(r3);
    v[4] = __uint_as_float(r4); v[5] = __uint_as_float(r5); v[6] = __uint_as_float(r6); v[7] = __uint_as_float(r7);
}

// Shared-memory matrix descriptor, no swizzle: start address, the byte offset between
// core matrices along K (leading) and along M/N (stride), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ---------------------------------------------------------------- the kernel
template <int C>
struct ConvTCShape {
    static constexpr int KG = C / 8;              // 16-byte channel groups of a site
    static constexpr int KC = C / 16;             // K chunks of one tap
    static constexpr int HX = kSgTileX + 2, HY = kSgTileY + 2;
    static constexpr int PLANE = KG * HY * HX;    // 16-byte entries of one staged plane
    static constexpr int NSLOT = 4;
    static constexpr int WENT = 27 * KG * C;      // 16-byte entries of the weights
    static constexpr int BUF = C <= 16 ? 16 : (C <= 32 ? 32 : 64);  // TMEM columns per accumulator
    static constexpr int TMEM_COLS = 2 * BUF < 32 ? 32 : 2 * BUF;
    static constexpr size_t SMEM = (size_t)(NSLOT * PLANE + WENT) * 16;
};

template <int C>
__global__ void __launch_bounds__(256, 1) k_conv_tc(const ConvTCArgs A)
{
    using S = ConvTCShape<C>;
    constexpr int KG = S::KG, KC = S::KC, HX = S::HX, HY = S::HY, PLANE = S::PLANE;
    constexpr uint32_t LBO_A = HY * HX * 16, SBO_A = HX * 16;
    constexpr uint32_t LBO_B = (C / 8) * 128, SBO_B = 128;
    constexpr uint32_t IDESC = idesc_bf16(128, C);
    extern __shared__ __align__(128) uint4 smem[];
    uint4* sA = smem;                       // [NSLOT][KG][HY][HX]
    uint4* sB = smem + S::NSLOT * PLANE;    // [27][KG][C/8][8]
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = A.N;
    const int ntx = N / kSgTileX, nty = N / kSgTileY, nzc = (N + A.DZ - 1) / A.DZ;
    const int units = ntx * nty * nzc;

    for (int i = tid; i < S::WENT; i += blockDim.x) sB[i] = __ldg(reinterpret_cast<const uint4*>(A.wfmt) + i);
    if (tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
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
    uint32_t phase = 0;  // bit b: parity of the next completion of s_bar[b]
    uint32_t step = 0;   // planes issued by this block (accumulator = step & 1)

    for (int unit = blockIdx.x; unit < units; unit += gridDim.x) {
        const int tx = unit % ntx, ty = (unit / ntx) % nty, tz = unit / (ntx * nty);
        const int x0 = tx * kSgTileX, y0 = ty * kSgTileY, z0 = tz * A.DZ;
        const int nz = min(A.DZ, N - z0);

        // stage input plane p (periodic) into slot (p + 4) & 3, applying the input activation
        auto stage = [&](int p) {
            const int zz = ((p % N) + N) % N;
            uint4* dst = sA + ((p + 4) & 3) * PLANE;
            for (int i = tid; i < PLANE; i += blockDim.x) {
                const int kg = i % KG, s = i / KG;
                const int hx = s % HX, hy = s / HX;
                int gx = x0 - 1 + hx, gy = y0 - 1 + hy;
                gx = gx < 0 ? gx + N : (gx >= N ? gx - N : gx);
                gy = gy < 0 ? gy + N : (gy >= N ? gy - N : gy);
                const size_t site = ((size_t)zz * N + gy) * N + gx;
                uint4 v = __ldg(reinterpret_cast<const uint4*>(A.in + site * C) + kg);
                if (A.in_act) v = act_bf16x8(A.in_act, v);
                dst[(kg * HY + hy) * HX + hx] = v;
            }
        };
        // finish the accumulator of plane zp: 8 warps, warp w reads TMEM lanes 32 (w & 3) ..
        // and the column half (w >> 2)
        auto epilogue = [&](int zp, uint32_t buf) {
            const int q = warp & 3, half = warp >> 2;
            const int r = 32 * q + lane;
            const size_t site = ((size_t)zp * N + (y0 + (r >> 3))) * N + (x0 + (r & 7));
            constexpr int CH = C / 2;
#pragma unroll
            for (int c8 = 0; c8 < CH / 8; ++c8) {
                const int c0 = half * CH + c8 * 8;
                float v[8];
                tmem_ld8(tbase + ((uint32_t)(32 * q) << 16) + buf * S::BUF + c0, v);
                if (A.bias) {
#pragma unroll
                    for (int e = 0; e < 8; ++e) v[e] += __ldg(A.bias + c0 + e);
                }
                if (A.gate_act) {
                    const uint4 gv = __ldg(reinterpret_cast<const uint4*>(A.gate + site * C + c0));
                    float gf[8];
                    unpack_bf16x8(gv, gf);
#pragma unroll
                    for (int e = 0; e < 8; ++e) v[e] *= act_grad_f(A.gate_act, gf[e]);
                }
                reinterpret_cast<uint4*>(A.out + site * C + c0)[0] = pack_bf16x8(v);
            }
        };

        stage(z0 - 1);
        stage(z0);
        stage(z0 + 1);
        fence_proxy_async_smem();
        __syncthreads();
        for (int j = 0; j < nz; ++j) {
            const int z = z0 + j;
            const uint32_t buf = step & 1;
            if (tid == 0) {
                tc_fence_after();
                const uint32_t d = tbase + buf * S::BUF;
                uint32_t acc = 0;
#pragma unroll 1
                for (int t = 0; t < 27; ++t) {
                    const int ox = t % 3, oy = (t / 3) % 3, oz = t / 9;
                    const uint32_t a0 = smem_u32(sA + ((z + oz - 1 + 4) & 3) * PLANE + oy * HX + ox);
                    const uint32_t b0 = smem_u32(sB + t * KG * (C / 8) * 8);
#pragma unroll
                    for (int kc = 0; kc < KC; ++kc) {
                        tc_mma(d, smem_desc(a0 + kc * 2 * LBO_A, LBO_A, SBO_A), smem_desc(b0 + kc * 2 * LBO_B, LBO_B, SBO_B),
                               IDESC, acc);
                        acc = 1;
                    }
                }
                tc_commit(&s_bar[buf]);
            }
            if (j >= 1) {  // previous plane: wait for its MMAs, then finish it
                const uint32_t pb = buf ^ 1;
                if (!mbar_wait_bounded(&s_bar[pb], (phase >> pb) & 1u, s_fail ? 1000000ull : 2000000000ull)) s_fail = 1;
                phase ^= 1u << pb;
                tc_fence_after();
                epilogue(z - 1, pb);
            }
            // the slot of plane z+2 held plane z-2, last read by the MMAs just waited for
            if (j + 1 < nz) stage(z + 2);
            fence_proxy_async_smem();
            tc_fence_before();
            __syncthreads();
            ++step;
        }
        {  // last plane of the unit
            const uint32_t pb = (step - 1) & 1;
            if (!mbar_wait_bounded(&s_bar[pb], (phase >> pb) & 1u, s_fail ? 1000000ull : 2000000000ull)) s_fail = 1;
            phase ^= 1u << pb;
            tc_fence_after();
            epilogue(z0 + nz - 1, pb);
            tc_fence_before();
            __syncthreads();  // every MMA of the unit is complete: the ring may be refilled
        }
    }
    if (warp == 0) tmem_dealloc(tbase, S::TMEM_COLS);
    if (tid == 0 && s_fail) atomicOr(A.status, ST_TIMEOUT);
}

template <int C>
static cudaError_t launch_conv_tc_c(const ConvTCArgs& A, int grid, cudaStream_t s)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_conv_tc<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)ConvTCShape<C>::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_conv_tc<C><<<grid, 256, ConvTCShape<C>::SMEM, s>>>(A);
    return cudaGetLastError();
}

size_t conv_tc_smem(int C)
{
    return C == 16 ? ConvTCShape<16>::SMEM : (C == 32 ? ConvTCShape<32>::SMEM : ConvTCShape<48>::SMEM);
}

cudaError_t launch_conv_tc(int C, const ConvTCArgs& A, int grid, cudaStream_t s)
{
    if (C == 16) return launch_conv_tc_c<16>(A, grid, s);
    if (C == 32) return launch_conv_tc_c<32>(A, grid, s);
    if (C == 48) return launch_conv_tc_c<48>(A, grid, s);
    return cudaErrorInvalidValue;
}

}  // namespace clk
