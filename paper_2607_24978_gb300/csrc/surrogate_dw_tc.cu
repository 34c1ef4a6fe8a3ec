// Weight gradients of a surrogate layer (CI -> CO channels, padded to CIP, COP = 16, 32 or
// 48) on the tensor cores (tcgen05, BF16 operands, FP32 accumulation in TMEM):
//
//   dW[t][co][ci] = sum_n g[n][co] h[n + o(t)][ci],    t = (tz*3 + ty)*3 + tx, o = (tx-1, ty-1, tz-1)
//
// with g the gradient of the layer's output and h its (activated) input: BF16 [site][C]
// activations, or the thin FP32 network input / loss gradient, converted to BF16 and
// zero-padded while staged.  The sites are the reduction (K) dimension, so both operands are read
// MN-major: shared memory holds 16-byte entries (8 channels of one site) laid out
// [channel group][site], where eight consecutive sites form one 128-byte core matrix and
// a one-site shift of a tap is a 16-byte shift of the descriptor's start address.
//
// A work unit is one x row (z, y) of N sites, split into K chunks of 16 sites.  Per chunk
// and x tap (three MMAs, M = 128, N = 3 CIP, K = 16):
//  * B (N rows) is h of the three rows y-1, y, y+1 of one plane, staged [row][group][x]
//    with a one-site periodic halo in x: the 3 CIP rows (y tap, input channel) are evenly
//    strided, so the three y taps are one MMA (N = 3 CIP);
//  * A (M = 128 rows) is g of row (z, y) in rows 0-63 (channels padded with zeros) and, in
//    the first block group, g of row (z-1, y) in rows 64-127.
// The first group stages h of plane z-1: rows 0-63 accumulate the tz = 0 taps of output
// plane z and rows 64-127 the tz = 1 taps of plane z-1 (each plane is the z-1 of exactly
// one unit, periodic in z).  The second group stages h of plane z+1 (tz = 2; its rows
// 64-127 stay zero).  B carries one more channel block that holds the constant 1 (and a
// zero block to round N up to a multiple of 16): the first x tap's MMA (N = 3 CIP + 16)
// then also accumulates db[co] = sum_n g[n][co].  A block accumulates its units in TMEM
// and writes one partial per tap (and per bias); a second kernel sums the partials in a
// fixed order.
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
// blocks over the shared-memory banks) and B (3 rows x CIP/8 groups, then the ones block and
// a zero block, of N + 2 sites each).
__host__ __device__ inline int dw_a_entries(int N) { return 16 * (N + 1); }
__host__ __device__ inline int dw_slot_entries(int CIP, int N) { return dw_a_entries(N) + (3 * (CIP / 8) + 2) * (N + 2); }

template <int CIP, int COP>
struct DwTCShape {
    static constexpr int CGA = COP / 8;     // channel groups of g (A, per half)
    static constexpr int CG = CIP / 8;      // channel groups of h (B)
    static constexpr int NT = 3 * CIP;      // MMA N of an x tap: three y taps x CIP input channels
    static constexpr int NT1 = NT + 16;     // first x tap: plus the ones (bias) block
    static constexpr int COLS = NT1 + 2 * NT;
    static constexpr int TMEM_COLS = COLS <= 256 ? 256 : 512;
    static_assert(COLS <= 512, "accumulators exceed TMEM");
    static_assert(kDwStage % CGA == 0 && kDwStage % CG == 0, "staging threads per channel group");
};

// 16-byte entry of 8 channels (from channel c0) of FP32 site data with `nc` channels, BF16,
// zero beyond nc.
__device__ __forceinline__ uint4 f32_entry(const float* site, int nc, int c0)
{
    float f[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) f[c] = c0 + c < nc ? __ldg(site + c0 + c) : 0.f;
    return pack_bf16x8(f);
}

template <int CIP, int COP, bool GF32, bool HF32>
__global__ void __launch_bounds__(256, 1) k_conv_dw_tc(const ConvDWTCArgs A)
{
    using S = DwTCShape<CIP, COP>;
    constexpr int CGA = S::CGA, CG = S::CG, NT = S::NT, NT1 = S::NT1;
    extern __shared__ __align__(128) uint4 smem[];
    __shared__ __align__(8) uint64_t s_full[kDwMaxSlots];   // unit staged in the slot (96 arrivals)
    __shared__ __align__(8) uint64_t s_freeb[kDwMaxSlots];  // slot's unit read by its MMAs (commit)
    __shared__ __align__(8) uint64_t s_done;                // every MMA of the block complete (commit)
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = A.N, NS = A.nslot, grp = blockIdx.y;
    const int AST = N + 1, BST = N + 2;  // entries between channel blocks of A, of B
    const int AENT = dw_a_entries(N), SLOT = dw_slot_entries(CIP, N);
    const long long units = (long long)N * N;
    const long long u0 = units * blockIdx.x / gridDim.x, u1 = units * (blockIdx.x + 1) / gridDim.x;
    const int nblk_a = grp == 0 ? 2 : 1;  // g rows staged into A (rows 0-63, and 64-127)

    // constant blocks, written once: the padding channel blocks of A (zero), and the ones
    // block (channel 0 = 1) and zero block that follow the h rows in B
    for (int s = 0; s < NS; ++s) {
        uint4* sa = smem + (size_t)s * SLOT;
        for (int e = tid; e < 16 * AST; e += blockDim.x) {
            const int b = e / AST;
            const bool used = (b < CGA) || (nblk_a == 2 && b >= 8 && b < 8 + CGA);
            if (!used) sa[e] = make_uint4(0u, 0u, 0u, 0u);
        }
        uint4* sk = sa + AENT + 3 * CG * BST;
        const uint4 one = make_uint4(0x3F80u, 0u, 0u, 0u);  // BF16 1.0 in channel 0
        for (int e = tid; e < 2 * BST; e += blockDim.x) sk[e] = e < BST ? one : make_uint4(0u, 0u, 0u, 0u);
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
        // accumulator columns: x tap 0 (with the bias block) [0, NT1), x tap 1 [NT1, NT1 + NT),
        // x tap 2 [NT1 + NT, NT1 + 2 NT)
        if (lane == 0) {
            uint32_t full_ph = 0;
            int seq = 0;
            constexpr uint32_t idesc0 = idesc_bf16_mn(128, NT1), idesc = idesc_bf16_mn(128, NT);
            const uint32_t sbo_a = (uint32_t)AST * 16, sbo_b = (uint32_t)BST * 16;
            for (long long u = u0; u < u1; ++u, ++seq) {
                const int slot = seq % NS;
                wait(&s_full[slot], full_ph, slot);
                tc_fence_after();
                const uint32_t a0 = smem_u32(smem + (size_t)slot * SLOT), b0 = a0 + (uint32_t)AENT * 16;
#pragma unroll 1
                for (int kc = 0; kc < N / 16; ++kc) {
                    const uint64_t adesc = smem_desc(a0 + kc * 256, 128, sbo_a);
                    const uint32_t acc = (u == u0 && kc == 0) ? 0u : 1u;
                    tc_mma(tbase, adesc, smem_desc(b0 + kc * 256, 128, sbo_b), idesc0, acc);
                    tc_mma(tbase + NT1, adesc, smem_desc(b0 + kc * 256 + 16, 128, sbo_b), idesc, acc);
                    tc_mma(tbase + NT1 + NT, adesc, smem_desc(b0 + kc * 256 + 32, 128, sbo_b), idesc, acc);
                }
                tc_commit(&s_freeb[slot]);  // the slot may be restaged once these MMAs completed
            }
            if (u1 > u0) tc_commit(&s_done);
        }
        __syncwarp();
    } else if (warp < 4) {
        // ------------------------------------------------------------ staging warps
        // Each thread keeps one channel group (its index mod the groups of a site) and steps
        // through the sites: no division in the loops.
        const int st = tid - 32;
        const int dzh = grp == 0 ? -1 : 1;  // plane of h relative to the unit
        constexpr int SXA = kDwStage / CGA, SXB = kDwStage / CG;
        const int cga = st % CGA, xa0 = st / CGA;
        const int cgb = st % CG, pb0 = st / CG;
        uint32_t free_ph = 0;
        int seq = 0, pend_slot = -1;
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
            for (int half = 0; half < nblk_a; ++half) {
                const int zz = half == 0 ? z : (z == 0 ? N - 1 : z - 1);
                const size_t row = ((size_t)zz * N + y) * N;
                uint4* d = sa + (half * 8 + cga) * AST;
                for (int x = xa0; x < N; x += SXA) {
                    if (!GF32) cp_async16(d + x, reinterpret_cast<const __nv_bfloat16*>(A.g) + (row + x) * COP + cga * 8);
                    else d[x] = f32_entry(reinterpret_cast<const float*>(A.g) + (row + x) * A.g_c, A.g_c, cga * 8);
                }
            }
            // B: h of rows y-1, y, y+1 of plane z + dzh, x from -1 to N (periodic)
            const int zh = z + dzh < 0 ? N - 1 : (z + dzh >= N ? 0 : z + dzh);
#pragma unroll
            for (int dy = 0; dy < 3; ++dy) {
                const int yy = y + dy - 1 < 0 ? N - 1 : (y + dy - 1 >= N ? 0 : y + dy - 1);
                const size_t row = ((size_t)zh * N + yy) * N;
                uint4* d = sb + (dy * CG + cgb) * BST;
                for (int p = pb0; p < BST; p += SXB) {
                    const int xx = p == 0 ? N - 1 : (p == N + 1 ? 0 : p - 1);
                    if (!HF32) cp_async16(d + p, reinterpret_cast<const __nv_bfloat16*>(A.h) + (row + xx) * CIP + cgb * 8);
                    else d[p] = f32_entry(reinterpret_cast<const float*>(A.h) + (row + xx) * A.h_c, A.h_c, cgb * 8);
                }
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
        const bool valid = co < COP && (grp == 0 || half == 0);
        float* P = grp == 0 ? A.part0 + (size_t)blockIdx.x * 18 * COP * CIP : A.part1 + (size_t)blockIdx.x * 9 * COP * CIP;
        auto load16 = [&](int col, uint32_t (&raw)[16]) {
            if (any) {
                tmem_ld16(tbase + ((uint32_t)(32 * q) << 16) + col, raw);
                tmem_wait<16>(raw);
            } else {
#pragma unroll
                for (int e = 0; e < 16; ++e) raw[e] = 0u;
            }
        };
#pragma unroll 1
        for (int dx = 0; dx < 3; ++dx) {
            const int cbase = dx == 0 ? 0 : NT1 + (dx - 1) * NT;
#pragma unroll 1
            for (int c16 = 0; c16 < NT / 16; ++c16) {
                uint32_t raw[16];
                load16(cbase + c16 * 16, raw);
                if (valid) {
                    const int col = c16 * 16, dy = col / CIP, ci0 = col - dy * CIP;
                    const int tl = (half * 3 + dy) * 3 + dx;  // tap within the group's planes
                    float4* o = reinterpret_cast<float4*>(P + ((size_t)tl * COP + co) * CIP + ci0);
#pragma unroll
                    for (int v = 0; v < 4; ++v)
                        o[v] = make_float4(__uint_as_float(raw[4 * v]), __uint_as_float(raw[4 * v + 1]),
                                           __uint_as_float(raw[4 * v + 2]), __uint_as_float(raw[4 * v + 3]));
                }
            }
        }
        {  // the ones column: sum of g over this block's sites (the second group's rows 0-63)
            uint32_t raw[16];
            load16(NT, raw);
            if (grp == 1 && half == 0 && co < COP) A.bpart[(size_t)blockIdx.x * COP + co] = __uint_as_float(raw[0]);
        }
        tc_fence_before();
    }
    __syncthreads();  // the epilogue waited for every MMA; no copy is in flight
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tbase, S::TMEM_COLS);
    if (tid == 0 && s_fail) atomicOr(A.status, ST_TIMEOUT);
}

// dW[t][co][ci] (CO x CI real channels) = sum over the blocks of the group owning plane tz
// of their padded partials, db[co] = sum of the bias partials (fixed orders).
__global__ void k_conv_dw_tc_reduce(const ConvDWTCArgs A, int CIP, int COP)
{
    const int cc = A.CO * A.CI, pp = COP * CIP, total = 27 * cc + A.CO;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        if (i < 27 * cc) {
            const int t = i / cc, r = i - t * cc, co = r / A.CI, ci = r - co * A.CI;
            float s = 0.f;
            if (t < 18) {
                const size_t j = (size_t)t * pp + co * CIP + ci;
                for (int b = 0; b < A.nb; ++b) s += A.part0[(size_t)b * 18 * pp + j];
            } else {
                const size_t j = (size_t)(t - 18) * pp + co * CIP + ci;
                for (int b = 0; b < A.nb; ++b) s += A.part1[(size_t)b * 9 * pp + j];
            }
            A.dW[i] = s;
        } else {
            const int co = i - 27 * cc;
            double s = 0.0;
            for (int b = 0; b < A.nb; ++b) s += A.bpart[(size_t)b * COP + co];
            A.db[co] = (float)s;
        }
    }
}

size_t conv_dw_tc_smem(int CIP, int N, int nslot) { return (size_t)nslot * dw_slot_entries(CIP, N) * 16; }

int conv_dw_tc_slots(int CIP, int N)
{
    if ((CIP != 16 && CIP != 32 && CIP != 48) || N < 16 || N % 16 != 0) return 0;
    for (int s = kDwMaxSlots; s >= 2; --s)
        if (conv_dw_tc_smem(CIP, N, s) <= (size_t)kPassMaxSmem) return s;
    return 0;
}

template <int CIP, int COP, bool GF32, bool HF32>
static cudaError_t launch_dw_tc_t(const ConvDWTCArgs& A, cudaStream_t s)
{
    const size_t smem = conv_dw_tc_smem(CIP, A.N, A.nslot);
    cudaError_t e = cudaFuncSetAttribute(k_conv_dw_tc<CIP, COP, GF32, HF32>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_conv_dw_tc<CIP, COP, GF32, HF32><<<dim3(A.nb, 2), 256, smem, s>>>(A);
    return cudaGetLastError();
}

// (CIP, COP, FP32 g, FP32 h): hidden layers, the first layer (FP32 network input) and the
// last layer (FP32 loss gradient) of hidden widths 16, 32 and 48
#define CL_DW_SHAPES(X)                                                                            \
    X(16, 16, false, false) X(32, 32, false, false) X(48, 48, false, false) X(16, 16, false, true) \
    X(16, 32, false, true) X(16, 48, false, true) X(16, 16, true, false) X(32, 16, true, false)   \
    X(48, 16, true, false)

cudaError_t launch_conv_dw_tc(int CIP, int COP, const ConvDWTCArgs& A, cudaStream_t s)
{
    if (A.nslot < 2 || A.nslot > kDwMaxSlots || A.nslot > conv_dw_tc_slots(CIP, A.N) || A.nb < 1 || A.CI < 1 ||
        A.CI > CIP || A.CO < 1 || A.CO > COP || (A.h_f32 && A.h_c != A.CI) || (A.g_f32 && A.g_c != A.CO) ||
        (!A.h_f32 && A.CI != CIP) || (!A.g_f32 && A.CO != COP) || (A.g_f32 && A.h_f32))
        return cudaErrorInvalidValue;
    cudaError_t e = cudaErrorInvalidValue;
    const bool gf = A.g_f32 != 0, hf = A.h_f32 != 0;
#define CL_DW_LAUNCH(a, b, c, d) \
    if (CIP == a && COP == b && gf == c && hf == d) e = launch_dw_tc_t<a, b, c, d>(A, s);
    CL_DW_SHAPES(CL_DW_LAUNCH)
#undef CL_DW_LAUNCH
    if (e != cudaSuccess) return e;
    const int total = 27 * A.CO * A.CI + A.CO;
    k_conv_dw_tc_reduce<<<(total + 255) / 256, 256, 0, s>>>(A, CIP, COP);
    return cudaGetLastError();
}

}  // namespace clk
