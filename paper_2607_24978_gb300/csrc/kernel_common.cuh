// Device helpers shared by the lattice kernels (vector access, exact rounding,
// per-thread accumulators, fixed-order block reductions, TMA bulk copies and
// bounded mbarrier waits).
#pragma once

#include <stdint.h>

#include "cl_internal.cuh"

namespace clk {

template <typename T, int VW> struct VT;
template <> struct VT<float, 4> { using type = float4; };
template <> struct VT<float, 2> { using type = float2; };
template <> struct VT<float, 1> { using type = float; };
template <> struct VT<double, 2> { using type = double2; };
template <> struct VT<double, 1> { using type = double; };

template <typename T, int VW>
__device__ __forceinline__ void vload(T (&d)[VW], const T* __restrict__ p)
{
    using V = typename VT<T, VW>::type;
    V v = __ldg(reinterpret_cast<const V*>(p));
    const T* q = reinterpret_cast<const T*>(&v);
#pragma unroll
    for (int i = 0; i < VW; ++i) d[i] = q[i];
}

template <typename T, int VW>
__device__ __forceinline__ void vload_smem(T (&d)[VW], const T* p)
{
    using V = typename VT<T, VW>::type;
    V v = *reinterpret_cast<const V*>(p);
    const T* q = reinterpret_cast<const T*>(&v);
#pragma unroll
    for (int i = 0; i < VW; ++i) d[i] = q[i];
}

template <typename T, int VW>
__device__ __forceinline__ void vstore(T* p, const T (&s)[VW])
{
    using V = typename VT<T, VW>::type;
    V v;
    T* q = reinterpret_cast<T*>(&v);
#pragma unroll
    for (int i = 0; i < VW; ++i) q[i] = s[i];
    *reinterpret_cast<V*>(p) = v;
}

// a^e for the powers of the scale factor in the equations of motion (e = alpha + const).
// Integer exponents -- alpha = 0 or 1, the usual choices -- by repeated multiplication, a
// handful of FP64 operations; other exponents by pow.  On GB300's narrow FP64 pipe the
// accurate pow routine takes microseconds on the single thread that evaluates a pass's
// coefficients while the rest of its block waits, so each pass paid several of them.
__device__ __forceinline__ double apow(double a, double e)
{
    const double r = rint(e);
    if (r == e && fabs(r) <= 16.0) {
        int n = (int)r;
        const bool neg = n < 0;
        if (neg) n = -n;
        double p = 1.0, b = a;
        while (n) {
            if (n & 1) p *= b;
            b *= b;
            n >>= 1;
        }
        return neg ? 1.0 / p : p;
    }
    return pow(a, e);
}

// Explicitly rounded operations: the drift of a halo element must be bit-identical
// to the owner's drift of the same element, so no contraction choice is left to
// the compiler.
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }

// Fetch the 128-byte line holding p into L2 (no register result; a hint).
__device__ __forceinline__ void prefetch_l2(const void* p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// phi += cd * pi, with Kahan compensation c when KAHAN.
template <typename T, bool KAHAN>
__device__ __forceinline__ void drift(T& phi, T& c, T pi, T cd)
{
    if (KAHAN) {
        const T y = fma_rn(cd, pi, -c);
        const T t = add_rn(phi, y);
        c = sub_rn(sub_rn(t, phi), y);
        phi = t;
    } else {
        phi = fma_rn(cd, pi, phi);
    }
}

// Per-thread accumulator: compensated float sum for FP32 fields, plain double for FP64.
template <typename T> struct Acc;
template <> struct Acc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        const float y = __fsub_rn(x, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};
template <> struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double value() const { return s; }
};

// Sum v[q] over the block; the result is valid in thread 0.  Fixed reduction order.
template <int Q>
__device__ __forceinline__ void block_reduce(double (&v)[Q], double (*s_red)[kMaxQ], int tid, int nthr)
{
#pragma unroll
    for (int q = 0; q < Q; ++q)
        for (int off = 16; off > 0; off >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], off);
    const int warp = tid >> 5, lane = tid & 31, nw = (nthr + 31) >> 5;
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < Q; ++q) s_red[warp][q] = v[q];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            double x = lane < nw ? s_red[lane][q] : 0.0;
            for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
            v[q] = x;
        }
    }
    __syncthreads();
}

// Float-pair (hi + lo) addition with the two-sum error term, for the warp-level stage of the
// FP32 passes' energy sums: about 44 significant bits on the FP32 pipe.  GB300 executes FP64
// additions two lanes per SM and cycle, so a warp butterfly of doubles on every lane is slow
// on the critical path of each block's reduction; in pairs the warp stage costs no FP64 work.
struct F2 {
    float hi, lo;
};
__device__ __forceinline__ F2 f2_add(F2 a, F2 b)
{
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float h = __fadd_rn(s, e);
    return {h, __fsub_rn(e, __fsub_rn(h, s))};
}

// Sum over the block of per-thread values hi[q] + lo[q] (e.g. a compensated FP32 sum s - c),
// the result in FP64, valid in thread 0.  Each warp adds its lanes as float pairs, lane 0
// converts once to FP64, warp 0 adds the warps in FP64.  Fixed reduction order.
template <int Q>
__device__ __forceinline__ void block_reduce_pairs(const float (&hi)[Q], const float (&lo)[Q], double (&v)[Q],
                                                   double (*s_red)[kMaxQ], int tid, int nthr)
{
    const int warp = tid >> 5, lane = tid & 31, nw = (nthr + 31) >> 5;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        F2 x{hi[q], lo[q]};
        for (int off = 16; off > 0; off >>= 1) {
            const F2 o{__shfl_xor_sync(0xffffffffu, x.hi, off), __shfl_xor_sync(0xffffffffu, x.lo, off)};
            x = f2_add(x, o);
        }
        if (lane == 0) s_red[warp][q] = (double)x.hi + (double)x.lo;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            double x = lane < nw ? s_red[lane][q] : 0.0;
            for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
            v[q] = x;
        }
    }
    __syncthreads();
}

// Sum of the grid's block partials partials[b * kMaxQ + q] (b < nb) by one warp, in FP64 and a
// fixed order (each lane adds the blocks b = lane, lane + 32, ... in turn, then a butterfly);
// call with all 32 lanes of the warp; the result is valid in every lane.
template <int Q>
__device__ __forceinline__ void warp_sum_partials(const double* partials, int nb, int lane, double (&w)[Q])
{
#pragma unroll
    for (int q = 0; q < Q; ++q) w[q] = 0.0;
    for (int b = lane; b < nb; b += 32)
#pragma unroll
        for (int q = 0; q < Q; ++q) w[q] += __ldcg(&partials[(size_t)b * kMaxQ + q]);
#pragma unroll
    for (int q = 0; q < Q; ++q)
        for (int off = 16; off > 0; off >>= 1) w[q] += __shfl_xor_sync(0xffffffffu, w[q], off);
}

// Block sum of per-thread accumulators acc[q] (nullptr: 0) into v[q], valid in thread 0:
// compensated FP32 accumulators (their s - c) through the float-pair warp stage, FP64 ones
// through block_reduce.
template <typename T, int Q>
__device__ __forceinline__ void block_reduce_acc(const Acc<T>* const (&acc)[Q], double (&v)[Q],
                                                 double (*s_red)[kMaxQ], int tid, int nthr)
{
    if constexpr (sizeof(T) == 4) {
        float hi[Q], lo[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            hi[q] = acc[q] ? acc[q]->s : 0.f;
            lo[q] = acc[q] ? -acc[q]->c : 0.f;
        }
        block_reduce_pairs<Q>(hi, lo, v, s_red, tid, nthr);
    } else {
#pragma unroll
        for (int q = 0; q < Q; ++q) v[q] = acc[q] ? acc[q]->value() : 0.0;
        block_reduce<Q>(v, s_red, tid, nthr);
    }
}

// block_reduce over the first nthr threads only (a multiple of 32), synchronising on the
// named barrier `bar` instead of the whole block.
template <int Q>
__device__ __forceinline__ void group_reduce(double (&v)[Q], double (*s_red)[kMaxQ], int tid, int nthr, int bar)
{
#pragma unroll
    for (int q = 0; q < Q; ++q)
        for (int off = 16; off > 0; off >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], off);
    const int warp = tid >> 5, lane = tid & 31, nw = nthr >> 5;
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < Q; ++q) s_red[warp][q] = v[q];
    asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nthr) : "memory");
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            double x = lane < nw ? s_red[lane][q] : 0.0;
            for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
            v[q] = x;
        }
    }
    asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nthr) : "memory");
}

// group_reduce of per-thread accumulators acc[q] (nullptr: 0): compensated FP32 ones through
// a float-pair warp stage, FP64 ones as group_reduce does.  Valid in thread 0 of the group.
template <typename T, int Q>
__device__ __forceinline__ void group_reduce_acc(const Acc<T>* const (&acc)[Q], double (&v)[Q],
                                                 double (*s_red)[kMaxQ], int tid, int nthr, int bar)
{
    if constexpr (sizeof(T) == 4) {
        const int warp = tid >> 5, lane = tid & 31, nw = nthr >> 5;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            F2 x{acc[q] ? acc[q]->s : 0.f, acc[q] ? -acc[q]->c : 0.f};
            for (int off = 16; off > 0; off >>= 1) {
                const F2 o{__shfl_xor_sync(0xffffffffu, x.hi, off), __shfl_xor_sync(0xffffffffu, x.lo, off)};
                x = f2_add(x, o);
            }
            if (lane == 0) s_red[warp][q] = (double)x.hi + (double)x.lo;
        }
        asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nthr) : "memory");
        if (warp == 0) {
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                double x = lane < nw ? s_red[lane][q] : 0.0;
                for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
                v[q] = x;
            }
        }
        asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nthr) : "memory");
    } else {
#pragma unroll
        for (int q = 0; q < Q; ++q) v[q] = acc[q] ? acc[q]->value() : 0.0;
        group_reduce<Q>(v, s_red, tid, nthr, bar);
    }
}

// ---------------------------------------------------------------- lattice tiling and potential

// Work units are (y tile, z plane) pairs in tile-major order, U = nby * N of them.
// Fixed chunks (DZ > 0): block b owns tile b % nby, planes [bz DZ, bz DZ + DZ) with
// bz = b / nby.  Persistent (DZ < 0): block b owns the contiguous balanced range
// [b U / G, (b+1) U / G) of a grid of G blocks, so every SM gets the same number of
// planes and a block's pipeline restarts only where its range crosses a tile.
// (The host turns "automatic" DZ into a fixed DZ; the kernels only see DZ > 0 or DZ < 0.)
__device__ __forceinline__ void block_units(int N, int nby, int DZ, long long& u0, long long& u1)
{
    if (DZ > 0) {
        const int by = blockIdx.x % nby, bz = blockIdx.x / nby;
        u0 = (long long)by * N + (long long)bz * DZ;
        u1 = u0 + min(DZ, N - bz * DZ);
    } else {
        const long long U = (long long)nby * N;
        u0 = U * blockIdx.x / gridDim.x;
        u1 = U * (blockIdx.x + 1) / gridDim.x;
    }
}

template <typename T>
struct PotCoef {
    T m20, m21, l0, l1, g2, h_m20, h_m21, q_l0, q_l1, h_g2;
    __device__ __forceinline__ PotCoef(const double (&m2)[2], const double (&lam)[2], double g)
        : m20((T)m2[0]), m21((T)m2[1]), l0((T)lam[0]), l1((T)lam[1]), g2((T)g), h_m20((T)(0.5 * m2[0])),
          h_m21((T)(0.5 * m2[1])), q_l0((T)(0.25 * lam[0])), q_l1((T)(0.25 * lam[1])), h_g2((T)(0.5 * g))
    {
    }
};

// ---------------------------------------------------------------- TMA / mbarrier

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make initialised barriers visible to the asynchronous (TMA) proxy.
__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Barrier among the first `count` threads of the block (count a multiple of 32).
__device__ __forceinline__ void named_barrier_sync(int id, int count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Generic-proxy accesses to shared memory before this point are ordered before later
// asynchronous-proxy (TMA) writes to it.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// One bulk (non-tensor) TMA copy global -> shared, completing on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void tma_bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ uint64_t global_timer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of `bar` to complete, giving up after limit_ns.
// Returns false on timeout (the caller records it; it never spins unbounded).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns)
{
    uint32_t done = 0;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    const uint64_t t0 = global_timer_ns();
    while (true) {
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if (global_timer_ns() - t0 > limit_ns) return false;
    }
}

}  // namespace clk
