// Tensor-core (tcgen05) periodic 3x3x3 convolution of the surrogate's layers: CI input and
// CO output channels (16, 32 or 48; the thin first and last layers are zero-padded to 16),
// BF16 operands, FP32 accumulation.
//
// Implicit GEMM: for an 8 x 16 (x, y) tile of output sites of one plane, D[128 x CO] =
// sum over the 27 taps and the CI/16 K-chunks of A_tap[128 x 16] B_tap[16 x CO], one
// tcgen05.mma (M = 128, N = CO, K = 16) each.  Rows of A are output sites (row = x + 8 y),
// so the A operand of a tap is the staged input plane read at an (x, y) offset: the input
// planes live in shared memory as 16-byte entries (8 channels of one site) laid out
// [channel group][y][x] over the tile plus a one-site halo, which is the no-swizzle
// K-major core-matrix layout (eight consecutive x form one 128-byte core matrix; the
// next channel group is the next core matrix along K, the next y row the next along M).
// Every tap is therefore only a different descriptor start address.  The weights of all
// 27 taps stay in shared memory for the whole kernel in the same layout
// ([tap][channel-in group][channel-out group][8 out][8 in]).
//
// A block owns tiles of z-columns and marches up z through a ring of five staged input
// planes, with three warp roles synchronised by mbarriers only:
//  * warp 0, lane 0, issues the 27 * CI/16 MMAs of an output plane into one of two TMEM
//    accumulators once the three input planes are staged and the accumulator was read
//    back, and commits them to the accumulator's "done" barrier and to the "free" barrier
//    of every ring slot whose plane they read last;
//  * warps 1-3 stage input planes into free slots, two planes in flight: a BF16 input with
//    one 5-D tensor copy per plane (the view (8 channels, x, y, channel group, z) lands the
//    box directly in the [group][y][x] layout; zeros outside the lattice, after which the
//    periodic halo entries of boundary tiles are patched with plain loads), the thin FP32
//    input with converting loads; they apply the input activation in place once a plane
//    landed, and arrive on its "full" barrier;
//  * warps 4-7 (one per TMEM lane quarter) read an accumulator back (tcgen05.ld), release
//    it, and finish the plane (bias / residual or activation derivative) into global memory.
// Every barrier is waited for once per phase in order, so no waiter can miss a phase.  All
// waits are bounded and report through the status word.
#include <cuda_bf16.h>
#include <stdint.h>

#include "cl_internal.cuh"
#include "kernel_common.cuh"
#include "surrogate_common.cuh"
#include "tcgen05_ops.cuh"

#include <cudaTypedefs.h>

namespace clk {

// ---------------------------------------------------------------- the kernel
template <int CI, int CO>
struct ConvTCShape {
    static constexpr int KG = CI / 8;             // 16-byte channel groups of an input site
    static constexpr int KC = CI / 16;            // K chunks of one tap
    static constexpr int NG = CO / 8;             // 8-channel output groups
    static constexpr int HX = kSgTileX + 2, HY = kSgTileY + 2;
    static constexpr int PLANE = KG * HY * HX;    // 16-byte entries of one staged plane
    static constexpr int NSLOT = 5;
    static constexpr int WENT = 27 * KG * CO;     // 16-byte entries of the weights
    static constexpr int TMEM_COLS = 512;         // whole TMEM: a ring of accumulators
    static constexpr int NACC = TMEM_COLS / CO;   // accumulators of CO columns in the ring
    static constexpr size_t SMEM = (size_t)(NSLOT * PLANE + WENT) * 16;
};

template <int CI, int CO>
__global__ void __launch_bounds__(256, 1) k_conv_tc(const __grid_constant__ ConvTCArgs A)
{
    using S = ConvTCShape<CI, CO>;
    constexpr int KG = S::KG, KC = S::KC, NG = S::NG, HX = S::HX, HY = S::HY, PLANE = S::PLANE, NSLOT = S::NSLOT;
    constexpr uint32_t LBO_A = HY * HX * 16, SBO_A = HX * 16;
    constexpr uint32_t LBO_B3 = 3 * NG * 128, SBO_B = 128;  // weights [t9][kg][oz][ng][8][8]
    constexpr int NSTAGE = 96;  // staging threads (warps 1..3)
    extern __shared__ __align__(128) uint4 smem[];
    uint4* sA = smem;                  // [NSLOT][KG][HY][HX]
    uint4* sB = smem + NSLOT * PLANE;  // [9 (oy, ox)][KG][3 (oz)][NG][8]
    __shared__ __align__(8) uint64_t s_full[NSLOT];   // plane staged in the slot (96 arrivals)
    __shared__ __align__(8) uint64_t s_tma[NSLOT];    // tensor copy of the plane landed (bytes)
    __shared__ __align__(8) uint64_t s_freeb[NSLOT];  // slot's plane read by its last MMA (commit)
    __shared__ __align__(8) uint64_t s_done[S::NACC];     // accumulator complete (commit)
    __shared__ __align__(8) uint64_t s_accfree[S::NACC];  // accumulator read back (4 epilogue warps)
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    __shared__ float s_bias[CO];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = A.N;
    const int ntx = N / kSgTileX, nty = N / kSgTileY, nzc = (N + A.DZ - 1) / A.DZ;
    const int units = ntx * nty * nzc;

    for (int i = tid; i < S::WENT; i += blockDim.x) sB[i] = __ldg(reinterpret_cast<const uint4*>(A.wfmt) + i);
    for (int i = tid; i < CO; i += blockDim.x) s_bias[i] = A.bias ? __ldg(A.bias + i) : 0.f;
    if (tid == 0) {
        for (int k = 0; k < NSLOT; ++k) {
            mbar_init(&s_full[k], NSTAGE);
            mbar_init(&s_freeb[k], 1);
            mbar_init(&s_tma[k], 1);
        }
        for (int k = 0; k < S::NACC; ++k) {
            mbar_init(&s_done[k], 1);
            mbar_init(&s_accfree[k], 4);
        }
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
    auto unit_geom = [&](int unit, int& x0, int& y0, int& z0, int& nz) {
        const int tx = unit % ntx, ty = (unit / ntx) % nty, tz = unit / (ntx * nty);
        x0 = tx * kSgTileX;
        y0 = ty * kSgTileY;
        z0 = tz * A.DZ;
        nz = min(A.DZ, N - z0);
    };

    if (warp == 0) {
        // ------------------------------------------------------------ MMA issuer
        // Input plane i of a unit contributes, through tap plane oz, to output plane
        // k = i - oz.  The three z taps read the same A tile (the input plane at an (x, y)
        // offset), so one MMA with N = (oz range) * CO covers them, writing the accumulators
        // of outputs k = i, i-1, i-2.  Accumulator of output c (block-wide count) is ring slot
        // acc_slot(c) = (NACC - 1 - c) mod NACC: consecutive oz map to consecutive slots,
        // except where the ring wraps (the MMA is split there).  An output's first
        // contribution (i = k, oz = 0) overwrites, all others accumulate.
        if (lane == 0) {
            constexpr int NA = S::NACC;
            uint32_t full_ph = 0, accfree_ph = 0;
            uint32_t seq = 0, cbase = 0;  // staged planes and outputs of earlier units
            auto acc_slot = [&](uint32_t c) { return (int)(NA - 1 - (int)(c % NA)); };
            for (int unit = blockIdx.x; unit < units; unit += gridDim.x) {
                int x0, y0, z0, nz;
                unit_geom(unit, x0, y0, z0, nz);
                for (int i = 0; i < nz + 2; ++i) {
                    const int slot = (int)((seq + i) % NSLOT);
                    wait(&s_full[slot], full_ph, slot);
                    const int lo = max(0, i - nz + 1), hi = min(2, i);
                    if (i <= nz - 1) {  // output cbase + i starts here: its accumulator must be free
                        const uint32_t c = cbase + i;
                        if (c >= (uint32_t)NA) wait(&s_accfree[acc_slot(c)], accfree_ph, acc_slot(c));
                    }
                    tc_fence_after();
                    const uint32_t a_plane = smem_u32(sA + slot * PLANE);
                    // MMAs of taps oz in [a, b] (contiguous accumulators) for one (ox, oy, kc)
                    auto mma_run = [&](uint32_t a_addr, uint32_t b_tap, int a, int b, uint32_t accum) {
                        const int sl = acc_slot(cbase + i - a);
                        const uint32_t bdesc_addr = b_tap + a * NG * 128;
                        const int n = (b - a + 1) * CO;
                        tc_mma(tbase + sl * CO, smem_desc(a_addr, LBO_A, SBO_A), smem_desc(bdesc_addr, LBO_B3, SBO_B),
                               idesc_bf16(128, n), accum);
                    };
                    auto mma_range = [&](uint32_t a_addr, uint32_t b_tap, int a, int b, uint32_t accum) {
                        // split where the accumulator ring wraps
                        const int sl = acc_slot(cbase + i - a);
                        const int room = NA - sl;  // slots before the wrap
                        if (b - a + 1 <= room) {
                            mma_run(a_addr, b_tap, a, b, accum);
                        } else {
                            mma_run(a_addr, b_tap, a, a + room - 1, accum);
                            mma_run(a_addr, b_tap, a + room, b, accum);
                        }
                    };
#pragma unroll 1
                    for (int t9 = 0; t9 < 9; ++t9) {
                        const int ox = t9 % 3, oy = t9 / 3;
                        const uint32_t a0 = a_plane + (oy * HX + ox) * 16;
#pragma unroll
                        for (int kc = 0; kc < KC; ++kc) {
                            const uint32_t a_addr = a0 + kc * 2 * LBO_A;
                            const uint32_t b_tap = smem_u32(sB) + ((t9 * KG + 2 * kc) * 3 * NG) * 128;
                            if (t9 == 0 && kc == 0 && lo == 0) {
                                mma_range(a_addr, b_tap, 0, 0, 0);  // first contribution to output i
                                if (hi >= 1) mma_range(a_addr, b_tap, 1, hi, 1);
                            } else {
                                mma_range(a_addr, b_tap, lo, hi, 1);
                            }
                        }
                    }
                    tc_commit(&s_freeb[slot]);  // the staged plane was read by this plane's MMAs only
                    if (i >= 2) tc_commit(&s_done[acc_slot(cbase + i - 2)]);  // output i-2 complete
                }
                seq += nz + 2;
                cbase += nz;
            }
        }
        __syncwarp();
    } else if (warp < 4) {
        // ------------------------------------------------------------ staging warps
        const int st = tid - 32;
        uint32_t free_ph = 0, tma_ph = 0;
        uint32_t seq = 0;
        int pend_slot = -1, pend_x0 = 0, pend_y0 = 0, pend_z = 0;  // the plane whose copies are still landing
        const bool tma = A.in_tma && !A.in_f32;
        // The plane in `slot` (tile x0, y0, plane z) has landed: periodic halo entries the
        // tensor copy filled with zeros, the input activation, then publish.
        auto land = [&](int slot, int x0, int y0, int z) {
            uint4* dst = sA + slot * PLANE;
            if (tma) {
                wait(&s_tma[slot], tma_ph, slot);
                const int lx = x0 == 0, rx = x0 + kSgTileX == N, ly = y0 == 0, ry = y0 + kSgTileY == N;
                const int ncol = lx + rx, nrow = ly + ry;
                const int nent = (ncol * HY + nrow * HX) * KG;
                const __nv_bfloat16* in = reinterpret_cast<const __nv_bfloat16*>(A.in);
                for (int e = st; e < nent; e += NSTAGE) {
                    int hx, hy, kg;
                    if (e < ncol * HY * KG) {  // a halo column, every row
                        const int c = e / (HY * KG), rem = e - c * (HY * KG);
                        hx = (c == 0 && lx) ? 0 : HX - 1;
                        hy = rem / KG;
                        kg = rem - hy * KG;
                    } else {  // a halo row, every column
                        const int e2 = e - ncol * HY * KG;
                        const int c = e2 / (HX * KG), rem = e2 - c * (HX * KG);
                        hy = (c == 0 && ly) ? 0 : HY - 1;
                        hx = rem / KG;
                        kg = rem - hx * KG;
                    }
                    int gx = x0 - 1 + hx, gy = y0 - 1 + hy;
                    gx = gx < 0 ? gx + N : (gx >= N ? gx - N : gx);
                    gy = gy < 0 ? gy + N : (gy >= N ? gy - N : gy);
                    const size_t site = ((size_t)z * N + gy) * N + gx;
                    dst[(kg * HY + hy) * HX + hx] = __ldg(reinterpret_cast<const uint4*>(in + site * CI + kg * 8));
                }
            }
            if (!A.in_f32 && A.in_act) {
                if (tma) named_barrier_sync(1, NSTAGE);  // every patch is in place
                for (int e = st; e < PLANE; e += NSTAGE) {
                    const int kg = e % KG, s2 = e / KG;
                    uint4* d = dst + (kg * HY + s2 / HX) * HX + s2 % HX;
                    *d = act_bf16x8(A.in_act, *d);
                }
            }
            fence_proxy_async_smem();
            mbar_arrive(&s_full[slot]);
        };
        constexpr int EMAX = (PLANE + NSTAGE - 1) / NSTAGE;  // entries of a plane per staging thread
        for (int unit = blockIdx.x; unit < units; unit += gridDim.x) {
            int x0, y0, z0, nz;
            unit_geom(unit, x0, y0, z0, nz);
            // this thread's entries of a plane (copies without the tensor map): shared-memory
            // entry and site within the plane
            int soff[EMAX], goff[EMAX];
#pragma unroll
            for (int q = 0; q < EMAX; ++q) {
                const int e = st + q * NSTAGE;
                const int kg = e % KG, s2 = e / KG;
                const int hx = s2 % HX, hy = s2 / HX;
                int gx = x0 - 1 + hx, gy = y0 - 1 + hy;
                gx = gx < 0 ? gx + N : (gx >= N ? gx - N : gx);
                gy = gy < 0 ? gy + N : (gy >= N ? gy - N : gy);
                soff[q] = (kg * HY + hy) * HX + hx;
                goff[q] = gy * N + gx;
            }
            for (int i = 0; i < nz + 2; ++i, ++seq) {
                const int slot = (int)(seq % NSLOT);
                if (seq >= NSLOT) wait(&s_freeb[slot], free_ph, slot);
                const int p = z0 - 1 + i;
                const int pz = ((p % N) + N) % N;
                const size_t zbase = (size_t)pz * N * N;
                uint4* dst = sA + slot * PLANE;
                if (tma) {
                    if (st == 0) {  // one tensor copy: the plane with its halo (zeros outside the box)
                        mbar_arrive_expect_tx(&s_tma[slot], (uint32_t)(PLANE * 16));
                        asm volatile(
                            "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                            " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(dst)),
                            "l"(reinterpret_cast<uint64_t>(&A.in_map)), "r"(0), "r"(x0 - 1), "r"(y0 - 1), "r"(0), "r"(pz),
                            "r"(smem_u32(&s_tma[slot]))
                            : "memory");
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < EMAX; ++q) {
                        const int e = st + q * NSTAGE;
                        if (e >= PLANE) break;
                        const int kg = e % KG;
                        const size_t site = zbase + goff[q];
                        if (!A.in_f32) {
                            cp_async16(dst + soff[q], reinterpret_cast<const __nv_bfloat16*>(A.in) + site * CI + kg * 8);
                        } else {  // thin FP32 input: convert and zero-pad to CI channels
                            float f[8];
#pragma unroll
                            for (int c = 0; c < 8; ++c) {
                                const int ch = kg * 8 + c;
                                f[c] = ch < A.in_c ? __ldg(reinterpret_cast<const float*>(A.in) + site * A.in_c + ch) : 0.f;
                            }
                            dst[soff[q]] = pack_bf16x8(f);
                        }
                    }
                    cp_async_commit();
                }
                if (pend_slot >= 0) {  // the previous plane: landed once one group is left
                    if (!tma) cp_async_wait1();
                    land(pend_slot, pend_x0, pend_y0, pend_z);
                }
                pend_slot = slot;
                pend_x0 = x0;
                pend_y0 = y0;
                pend_z = pz;
            }
        }
        if (pend_slot >= 0) {
            if (!tma) cp_async_wait0();
            land(pend_slot, pend_x0, pend_y0, pend_z);
        }
    } else {
        // ------------------------------------------------------------ epilogue warps
        const int q = warp & 3;  // TMEM lane quarter of this warp
        const int r = 32 * q + lane;
        uint32_t done_ph = 0, c = 0;
        for (int unit = blockIdx.x; unit < units; unit += gridDim.x) {
            int x0, y0, z0, nz;
            unit_geom(unit, x0, y0, z0, nz);
            for (int k = 0; k < nz; ++k, ++c) {
                const int buf = (int)(S::NACC - 1 - (int)(c % S::NACC));  // accumulator slot of output c
                wait(&s_done[buf], done_ph, buf);
                tc_fence_after();
                uint32_t raw[CO];
#pragma unroll
                for (int c16 = 0; c16 < CO / 16; ++c16)
                    tmem_ld16(tbase + ((uint32_t)(32 * q) << 16) + buf * CO + c16 * 16,
                              *reinterpret_cast<uint32_t(*)[16]>(raw + c16 * 16));
                tmem_wait<CO>(raw);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&s_accfree[buf]);  // the accumulator may be overwritten
                float v[CO];
#pragma unroll
                for (int e = 0; e < CO; ++e) v[e] = __uint_as_float(raw[e]) + s_bias[e];
                const size_t site = ((size_t)(z0 + k) * N + (y0 + (r >> 3))) * N + (x0 + (r & 7));
                if (A.gate_act) {
#pragma unroll
                    for (int c8 = 0; c8 < CO / 8; ++c8) {
                        float gf[8];
                        unpack_bf16x8(__ldg(reinterpret_cast<const uint4*>(A.gate + site * CO + c8 * 8)), gf);
#pragma unroll
                        for (int e = 0; e < 8; ++e) v[c8 * 8 + e] *= act_grad_f(A.gate_act, gf[e]);
                    }
                }
                if (A.out_f32) {
                    float* o = reinterpret_cast<float*>(A.out) + site * A.out_c;
#pragma unroll
                    for (int e = 0; e < CO; ++e)  // constant indices keep v in registers
                        if (e < A.out_c) o[e] = v[e] + (A.resid ? A.resid[site * A.resid_stride + e] : 0.f);
                } else {
                    uint4* o = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(A.out) + site * CO);
                    uint4* op = A.out_pre ? reinterpret_cast<uint4*>(A.out_pre + site * CO) : nullptr;
#pragma unroll
                    for (int c8 = 0; c8 < CO / 8; ++c8) {
                        float f8[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) f8[e] = v[c8 * 8 + e];
                        if (op) op[c8] = pack_bf16x8(f8);
                        if (A.out_act) {
#pragma unroll
                            for (int e = 0; e < 8; ++e) f8[e] = act_f(A.out_act, f8[e]);
                        }
                        o[c8] = pack_bf16x8(f8);
                    }
                }
            }
        }
    }
    __syncthreads();  // every MMA was waited for by the epilogue warps; no copy is in flight
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tbase, S::TMEM_COLS);
    if (tid == 0 && s_fail) atomicOr(A.status, ST_TIMEOUT);
}

template <int CI, int CO>
static cudaError_t launch_conv_tc_t(const ConvTCArgs& A, int grid, cudaStream_t s)
{
    static DevFlag attr;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_conv_tc<CI, CO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)ConvTCShape<CI, CO>::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_conv_tc<CI, CO><<<grid, 256, ConvTCShape<CI, CO>::SMEM, s>>>(A);
    return cudaGetLastError();
}

void conv_tc_encode_input(ConvTCArgs& A, int CI)
{
    A.in_tma = 0;
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    if (!encode || A.in_f32 || !A.in || ((uintptr_t)A.in & 15u)) return;
    const cuuint64_t N = (cuuint64_t)A.N, es = 2;
    // dimensions: 8 channels (contiguous), x, y, channel group, z; strides of dims 1..4 in bytes
    const cuuint64_t dims[5] = {8, N, N, (cuuint64_t)(CI / 8), N};
    const cuuint64_t strides[4] = {CI * es, N * CI * es, 8 * es, N * N * CI * es};
    const cuuint32_t box[5] = {8, (cuuint32_t)(kSgTileX + 2), (cuuint32_t)(kSgTileY + 2), (cuuint32_t)(CI / 8), 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    if (encode(&A.in_map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(A.in), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
        A.in_tma = 1;
}

#define CL_TC_SHAPES(X) X(16, 16) X(32, 32) X(48, 48) X(16, 32) X(16, 48) X(32, 16) X(48, 16)

size_t conv_tc_smem(int CI, int CO)
{
#define CL_SMEM(a, b) \
    if (CI == a && CO == b) return ConvTCShape<a, b>::SMEM;
    CL_TC_SHAPES(CL_SMEM)
#undef CL_SMEM
    return 0;
}

cudaError_t launch_conv_tc(int CI, int CO, const ConvTCArgs& A, int grid, cudaStream_t s)
{
#define CL_LAUNCH(a, b) \
    if (CI == a && CO == b) return launch_conv_tc_t<a, b>(A, grid, s);
    CL_TC_SHAPES(CL_LAUNCH)
#undef CL_LAUNCH
    return cudaErrorInvalidValue;
}

}  // namespace clk
