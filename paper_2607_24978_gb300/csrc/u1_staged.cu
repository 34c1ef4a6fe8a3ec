// Shared-memory staged forms of the two axion-U(1) launches of a Runge-Kutta stage: the
// plaquette fields, then the stage.  The equations, the lattice Chern-Simons discretisation,
// the 2N-RK update and the energy sums are those of u1_stage.cu (section "ALP-gauge
// interactions", Eq. AxionInfEOM), evaluated in the same order, except that the plaquette
// launch takes sin P, cos P and sin^2(P/2) from one sincos of P/2 (sin P = 2 s c,
// cos P = 1 - 2 s^2).
//
// The gather kernels of u1_stage.cu read 40 to 110 neighbour values per site from L1/L2
// into registers; a thread can only keep as many loads in flight as it has registers, and
// both kernels stall on memory latency at a fraction of the HBM bandwidth.  Here a block
// owns a 32 x TY tile of (x, y) (stage launches: TY = 16 in FP32, 8 in FP64; plaquette
// launches, which stage fewer arrays: twice that, over half the z chunk, so that both
// launch the same blocks; one site per consumer thread) and marches up its z chunk with planes z-1, z, z+1 of every array that is read at a
// neighbour in shared memory: rows y0-1 .. y0+TY and columns x0-VE .. x0+31+VE (VE elements
// per 16 bytes, so that every row is whole 16-byte units; only the first and last columns
// are read).  Warp roles, synchronised by mbarriers only:
//  * six producer warps copy plane after plane into a ring of five slots with 16-byte
//    asynchronous copies (cp.async; the source of every 16-byte unit of a plane, periodic
//    wrap included, is tabulated in shared memory once per block), and each lane's copies
//    arrive on the slot's "full" barrier when they have landed (measured at 192^3 FP32: one
//    producer warp, 2.5 Gsite-updates/s; two, 4.3; four, 6.3; six, 6.7; eight, 6.4;
//    single bulk copies of each staged row, 1.1: many small bulk copies are slow);
//  * TY consumer warps (one row of the tile each) wait for the planes they need, compute the
//    site, and release a slot once they have read it for the last time (its "empty" barrier
//    counts one arrival per consumer warp), so no warp waits for another one's work.
// Arrays read only at the site itself (theta and the Runge-Kutta auxiliaries) are loaded by
// the consumers straight from global memory, one plane ahead.  Every wait is bounded and
// reports through the status word.  Needs N % 32 == 0; other sizes use the gather kernels.
#include <math.h>

#include "cl_internal.cuh"
#include "kernel_common.cuh"
#include "u1_common.cuh"
#include "u1_staged.cuh"

namespace clk {

// Tile geometry: TX x TY sites a block, RW tile rows a consumer warp (rows w, w + CW, ...),
// PWARPS producer warps; SPLIT z parts of every z chunk of the stage grid, so that a geometry
// with SPLIT times taller tiles launches the same number of blocks over the same chunks.
template <typename T_, int TY_, int PWARPS_, int SPLIT_, int RW_>
struct U1SGeomT {
    using T = T_;
    static constexpr int TX = 32;
    static constexpr int TY = TY_;
    static constexpr int RW = RW_;
    static constexpr int CW = TY / RW;         // consumer warps
    static constexpr int PWARPS = PWARPS_;     // producer warps
    static constexpr int SPLIT = SPLIT_;
    static constexpr int PL = 32 * PWARPS;     // producer lanes
    static constexpr int NT = 32 * (CW + PWARPS);  // threads of a block (consumers, then the producers)
    static constexpr int VE = 16 / (int)sizeof(T);
    static constexpr int PW = TX + 2 * VE;     // staged columns x0 - VE .. x0 + TX + VE - 1
    static constexpr int PH = TY + 2;          // staged rows y0 - 1 .. y0 + TY
    static constexpr int ARR = PH * PW;        // elements of one array plane
    static constexpr int CPR = PW / VE;        // 16-byte units of a staged row
    static constexpr int SLOTS = 5;
    static_assert(TY % RW == 0 && NT <= 1024, "tile rows a warp; threads a block");
};

// the stage launches: 32 x 16 tiles in FP32, 32 x 8 in FP64, six producer warps
template <typename T>
using U1SGeom = U1SGeomT<T, sizeof(T) == 4 ? 16 : 8, 6, 1, 1>;
// the plaquette launches, which stage half as many arrays: tiles twice as tall over half z
// chunks, six producer warps, and in FP32 two sites a consumer thread (two independent
// chains of shared-memory loads and trigonometry; measured at 192^3 FP32 with one site a
// thread in 32 x 16 tiles: 113 us a launch, 61% of the issue slots active; this geometry:
// 104 us, 10% fewer instructions; with four producer warps: 121 us, the consumers waiting on
// the copies)
template <typename T>
using U1PGeom = U1SGeomT<T, 2 * U1SGeom<T>::TY, 6, 2, sizeof(T) == 4 ? 2 : 1>;

// arrays staged by the plaquette launch and by the stage launch, in slot order
enum { PQ_PHI = 0, PQ_TH = 1, PQ_E = 4, PQ_NA = 7 };
enum { SG_PHI = 0, SG_PI = 1, SG_E = 2, SG_SP = 5, SG_RP = 8, SG_Z = 11, SG_NA = 14 };

// 16-byte units of one staged plane of NA arrays, and the producer lanes' share of them
template <typename G, int NA>
struct U1SUnits {
    static constexpr int CH = NA * G::PH * G::CPR;
    static constexpr int PER_LANE = (CH + G::PL - 1) / G::PL;
};

// dynamic shared memory: the ring of plane slots, then the unit table (two words a unit)
template <typename G, int NA>
constexpr size_t u1s_smem_bytes()
{
    return (size_t)G::SLOTS * NA * G::ARR * sizeof(typename G::T) + (size_t)G::PL * U1SUnits<G, NA>::PER_LANE * 8;
}
// (every launch's dynamic shared memory, with 2 KB for its static arrays, fits one block)
static_assert(u1s_smem_bytes<U1PGeom<float>, PQ_NA>() + 2048 <= (size_t)kPassMaxSmem, "plaquette ring (FP32)");
static_assert(u1s_smem_bytes<U1PGeom<double>, PQ_NA>() + 2048 <= (size_t)kPassMaxSmem, "plaquette ring (FP64)");
static_assert(u1s_smem_bytes<U1SGeom<float>, SG_NA>() + 2048 <= (size_t)kPassMaxSmem, "stage ring (FP32)");
static_assert(u1s_smem_bytes<U1SGeom<double>, SG_NA>() + 2048 <= (size_t)kPassMaxSmem, "stage ring (FP64)");

// Tile and z range of this block: part bz % SPLIT of the z chunk bz / SPLIT (dz planes; the
// last chunk may be shorter).  A part may be empty (nz = 0) when its chunk has fewer planes
// than SPLIT; its block stages the two halo planes and writes nothing.
template <typename G>
struct U1STile {
    uint32_t N, x0, y0, z0, nz;
    __device__ __forceinline__ U1STile(uint32_t N_, uint32_t dz) : N(N_)
    {
        const uint32_t ntx = N / G::TX, nty = N / G::TY;
        uint32_t b = blockIdx.x;
        const uint32_t bx = b % ntx;
        b /= ntx;
        const uint32_t by = b % nty, bz = b / nty;
        x0 = bx * G::TX;
        y0 = by * G::TY;
        const uint32_t c0 = (bz / G::SPLIT) * dz;
        const uint32_t cn = c0 + dz < N ? dz : N - c0;
        const uint32_t per = (cn + G::SPLIT - 1) / G::SPLIT, skip = (bz % G::SPLIT) * per;
        z0 = c0 + skip;
        nz = cn > skip ? (cn - skip < per ? cn - skip : per) : 0u;
    }
};

// Unit table of the producer lanes: unit i of lane l (l + 32 i of the plane) is array a at
// staged row r, 16-byte column unit u; its entry holds (a << 16 | element offset in the slot)
// and the element offset of its source in a plane of the array (periodic wrap applied).
template <typename G, int NA>
__device__ __forceinline__ void u1s_build_units(uint2* table, const U1STile<G>& t, int tid, int nthr)
{
    using U = U1SUnits<G, NA>;
    const int N = (int)t.N;
    for (int e = tid; e < G::PL * U::PER_LANE; e += nthr) {
        const int lane = e % G::PL, i = e / G::PL, c = lane + G::PL * i;
        uint2 v = make_uint2(0xffffffffu, 0u);
        if (c < U::CH) {
            const int a = c / (G::PH * G::CPR), rem = c - a * (G::PH * G::CPR);
            const int r = rem / G::CPR, u = rem - r * G::CPR;
            int gy = (int)t.y0 - 1 + r, gx = (int)t.x0 - G::VE + u * G::VE;  // in [-1, N] and [-VE, N]
            gy = gy < 0 ? gy + N : (gy >= N ? gy - N : gy);
            gx = gx < 0 ? gx + N : (gx >= N ? gx - N : gx);
            v.x = ((uint32_t)a << 16) | (uint32_t)(a * G::ARR + r * G::PW + u * G::VE);
            v.y = (uint32_t)gy * (uint32_t)N + (uint32_t)gx;
        }
        table[i * G::PL + lane] = v;
    }
}

__device__ __forceinline__ void cp_async16_cg(void* smem_dst, const void* gsrc)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem_dst)), "l"(gsrc) : "memory");
}

// This lane's cp.async copies, issued before, arrive on bar once they have landed (the
// barrier's expected count includes the arrival).
__device__ __forceinline__ void cp_async_arrive_noinc(uint64_t* bar)
{
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Producer lane: its units of plane z0 - 1 + q (periodic) of the arrays src[] into slot,
// arriving on full when they have landed.
template <typename G, int NA, typename T = typename G::T>
__device__ __forceinline__ void u1s_copy_plane(int lane, T* slot, const T* const* src, const uint2* table,
                                               const U1STile<G>& t, int q, uint64_t* full)
{
    const int N = (int)t.N;
    int z = (int)t.z0 - 1 + q;
    z = z < 0 ? z + N : (z >= N ? z - N : z);
    const size_t zoff = (size_t)z * t.N * t.N;
#pragma unroll 4
    for (int i = 0; i < U1SUnits<G, NA>::PER_LANE; ++i) {
        const uint2 v = table[i * G::PL + lane];
        if (v.x != 0xffffffffu) cp_async16_cg(slot + (v.x & 0xffffu), src[v.x >> 16] + zoff + v.y);
    }
    cp_async_arrive_noinc(full);
}

// Neighbourhood of a consumer's site in the three staged planes (z-1, z, z+1).
template <typename G>
struct U1SNb {
    using T = typename G::T;
    const T* p[3];
    __device__ __forceinline__ T operator()(int a, int ox, int oy, int oz) const
    {
        return p[oz + 1][a * G::ARR + oy * G::PW + ox];
    }
    __device__ __forceinline__ T at(int a, const int (&o)[3]) const { return (*this)(a, o[0], o[1], o[2]); }
    // clover sum of array a (normal k) over the four plaquettes around the site at offset o
    __device__ __forceinline__ T clover(int a, int k, int ox, int oy, int oz) const
    {
        const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
        const int o[3] = {ox, oy, oz};
        int b[3] = {ox, oy, oz}, c[3] = {ox, oy, oz};
        b[k1] -= 1;
        c[k2] -= 1;
        int d[3] = {b[0], b[1], b[2]};
        d[k2] -= 1;
        return (at(a, o) + at(a, b)) + (at(a, c) + at(a, d));
    }
};

// Ring bookkeeping shared by both kernels: the producer loop and the consumers' waits and
// releases.  Plane q of the chunk lives in slot q % SLOTS; consumers read planes j, j+1, j+2
// for output plane j and release plane j afterwards (the last two planes after the loop).
template <typename G, int NA>
struct U1SRing {
    using T = typename G::T;
    static constexpr size_t SLOT = (size_t)NA * G::ARR;
    T* sm;
    const uint2* table;
    uint64_t* full;
    uint64_t* empty;
    int* fail;
    __device__ __forceinline__ bool wait(uint64_t* bar, uint32_t parity) const
    {
        if (mbar_wait_bounded(bar, parity, *fail ? 1000000ull : 2000000000ull)) return true;
        *fail = 1;
        return false;
    }
    // producer warp: every plane of the chunk
    __device__ __forceinline__ void produce(int lane, const T* const* src, const U1STile<G>& t) const
    {
        const int nq = (int)t.nz + 2;
        for (int q = 0; q < nq; ++q) {
            const int st = q % G::SLOTS;
            if (q >= G::SLOTS) wait(&empty[st], (uint32_t)((q / G::SLOTS - 1) & 1));
            u1s_copy_plane<G, NA>(lane, sm + st * SLOT, src, table, t, q, &full[st]);
        }
        // copies still in flight (only after a timeout, when consumers stopped waiting)
        if (*fail && lane == 0)
            for (int q = max(0, nq - G::SLOTS); q < nq; ++q)
                mbar_wait_bounded(&full[q % G::SLOTS], (uint32_t)((q / G::SLOTS) & 1), 1000000ull);
    }
    __device__ __forceinline__ void acquire(int q) const { wait(&full[q % G::SLOTS], (uint32_t)((q / G::SLOTS) & 1)); }
    __device__ __forceinline__ void release(int q, int lane) const
    {
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[q % G::SLOTS]);
    }
    // the three planes of output plane j at the consumer's site (row ly, column lx)
    __device__ __forceinline__ U1SNb<G> nb(int j, int lx, int ly) const
    {
        const int t0 = (ly + 1) * G::PW + lx + G::VE;
        U1SNb<G> n;
#pragma unroll
        for (int i = 0; i < 3; ++i) n.p[i] = sm + ((j + i) % G::SLOTS) * SLOT + t0;
        return n;
    }
};

// unit offset vector along axis d with sign s
#define U1S_E(d, s) ((d) == 0 ? (s) : 0), ((d) == 1 ? (s) : 0), ((d) == 2 ? (s) : 0)

template <typename T>
__global__ void __launch_bounds__(U1PGeom<T>::NT, 1) k_u1s_plaquettes(const U1Args<T> A)
{
    using G = U1PGeom<T>;
    constexpr int NA = PQ_NA;
    extern __shared__ __align__(128) unsigned char u1s_dyn[];
    __shared__ const T* s_src[NA];
    __shared__ __align__(8) uint64_t s_full[G::SLOTS], s_empty[G::SLOTS];
    __shared__ double s_red[G::NT / 32][kMaxQ];  // a row for every warp; the sum takes the consumers'
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        s_src[PQ_PHI] = A.phi_in;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            s_src[PQ_TH + k] = A.th_in[k];
            s_src[PQ_E + k] = A.E_in[k];
        }
        for (int k = 0; k < G::SLOTS; ++k) {
            mbar_init(&s_full[k], G::PL);  // the producer lanes' copies
            mbar_init(&s_empty[k], G::CW);
        }
        mbar_fence_init();
        s_fail = 0;
    }
    __syncthreads();
    const U1STile<G> t((uint32_t)A.N, (uint32_t)A.dz);
    T* ring_sm = reinterpret_cast<T*>(u1s_dyn);
    uint2* table = reinterpret_cast<uint2*>(ring_sm + G::SLOTS * NA * G::ARR);
    u1s_build_units<G, NA>(table, t, tid, G::NT);
    __syncthreads();
    const U1SRing<G, NA> ring{ring_sm, table, s_full, s_empty, &s_fail};
    Acc<T> accGB;
    if (warp >= G::CW) {
        ring.produce(tid - 32 * G::CW, s_src, t);
    } else {
        const uint32_t N = t.N;
        const T dx = (T)A.dx;
        ring.acquire(0);
        ring.acquire(1);
        for (int j = 0; j < (int)t.nz; ++j) {
            ring.acquire(j + 2);
            T o_s[G::RW][3], o_r[G::RW][3], o_z[G::RW][3], o_c[G::RW][3];
#pragma unroll
            for (int r = 0; r < G::RW; ++r)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const U1SNb<G> S = ring.nb(j, lane, warp + r * G::CW);
                const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
                const T P = S(PQ_TH + k1, 0, 0, 0) + S(PQ_TH + k2, U1S_E(k1, 1)) - S(PQ_TH + k1, U1S_E(k2, 1)) -
                            S(PQ_TH + k2, 0, 0, 0);
                const T R = dx * (S(PQ_E + k1, 0, 0, 0) + S(PQ_E + k2, U1S_E(k1, 1)) - S(PQ_E + k1, U1S_E(k2, 1)) -
                                  S(PQ_E + k2, 0, 0, 0));
                T sh, ch;  // sin, cos of P / 2
                if constexpr (sizeof(T) == 4) sincosf((T)0.5 * P, &sh, &ch);
                else sincos((T)0.5 * P, &sh, &ch);
                const T sp = (T)2 * sh * ch, cp = (T)1 - (T)2 * sh * sh;
                // X_k = phi Ebar_k at the corners n, n + e_k1, n + e_k2, n + e_k1 + e_k2
                const int e1[3] = {U1S_E(k1, 1)}, e2[3] = {U1S_E(k2, 1)}, ek[3] = {U1S_E(k, 1)};
                auto X = [&](int ox, int oy, int oz) {
                    return S(PQ_PHI, ox, oy, oz) *
                           (S(PQ_E + k, ox, oy, oz) + S(PQ_E + k, ox - ek[0], oy - ek[1], oz - ek[2]));
                };
                const T qs = X(0, 0, 0) + X(e1[0], e1[1], e1[2]) + X(e2[0], e2[1], e2[2]) +
                             X(e1[0] + e2[0], e1[1] + e2[1], e1[2] + e2[2]);
                o_s[r][k] = sp;
                o_r[r][k] = cp * R;
                o_z[r][k] = cp * ((T)0.5 * qs);
                o_c[r][k] = cp;
                accGB.add((T)2 * sh * sh);
            }
            ring.release(j, lane);
#pragma unroll
            for (int r = 0; r < G::RW; ++r) {
                const uint32_t n = ((t.z0 + j) * N + t.y0 + warp + r * G::CW) * N + t.x0 + lane;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    A.sP[k][n] = o_s[r][k];
                    A.rP[k][n] = o_r[r][k];
                    A.Z[k][n] = o_z[r][k];
                    if (A.cP[0]) A.cP[k][n] = o_c[r][k];  // cos P, for the rates launches of the same link angles
                }
            }
        }
        ring.release((int)t.nz, lane);
        ring.release((int)t.nz + 1, lane);
    }
    __syncthreads();  // producer and consumers meet; no copy is in flight past this point
    double v[1];
    const Acc<T>* av[1] = {&accGB};
    block_reduce_acc<T, 1>(av, v, s_red, tid, 32 * G::CW);  // (the producers' sums are zero)
    if (tid == 0) {
        A.partials[(size_t)gridDim.x * kMaxQ + blockIdx.x] = v[0];
        if (s_fail) atomicOr(&A.scal->status, ST_TIMEOUT);
    }
}

// The E-dependent plaquette fields of link angles whose cos P a plaquette launch saved
// (A.cP): cos P dP/dt and cos P times the corner sum of phi Ebar_k, from the staged phi and E
// (four arrays instead of seven, no trigonometry); sin P and the magnetic energy stay from
// that launch.  The leapfrog's second and third passes evaluate the force at the positions
// of the previous pass 1, whose plaquette launch saved cos P.
enum { RQ_PHI = 0, RQ_E = 1, RQ_NA = 4 };

template <typename T>
__global__ void __launch_bounds__(U1PGeom<T>::NT, 1) k_u1s_plaquette_rates(const U1Args<T> A)
{
    using G = U1PGeom<T>;
    constexpr int NA = RQ_NA;
    extern __shared__ __align__(128) unsigned char u1s_dyn[];
    __shared__ const T* s_src[NA];
    __shared__ __align__(8) uint64_t s_full[G::SLOTS], s_empty[G::SLOTS];
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        s_src[RQ_PHI] = A.phi_in;
#pragma unroll
        for (int k = 0; k < 3; ++k) s_src[RQ_E + k] = A.E_in[k];
        for (int k = 0; k < G::SLOTS; ++k) {
            mbar_init(&s_full[k], G::PL);  // the producer lanes' copies
            mbar_init(&s_empty[k], G::CW);
        }
        mbar_fence_init();
        s_fail = 0;
    }
    __syncthreads();
    const U1STile<G> t((uint32_t)A.N, (uint32_t)A.dz);
    T* ring_sm = reinterpret_cast<T*>(u1s_dyn);
    uint2* table = reinterpret_cast<uint2*>(ring_sm + G::SLOTS * NA * G::ARR);
    u1s_build_units<G, NA>(table, t, tid, G::NT);
    __syncthreads();
    const U1SRing<G, NA> ring{ring_sm, table, s_full, s_empty, &s_fail};
    if (warp >= G::CW) {
        ring.produce(tid - 32 * G::CW, s_src, t);
    } else {
        const uint32_t N = t.N;
        const T dx = (T)A.dx;
        // cos P of the sites' three plaquettes, loaded one plane ahead
        T cc[G::RW][3];
        auto load_c = [&](uint32_t m) {
#pragma unroll
            for (int r = 0; r < G::RW; ++r)
#pragma unroll
                for (int k = 0; k < 3; ++k) cc[r][k] = A.cP[k][m + (uint32_t)(r * G::CW) * N];
        };
        if (t.nz > 0) load_c((t.z0 * N + t.y0 + warp) * N + t.x0 + lane);
        ring.acquire(0);
        ring.acquire(1);
        for (int j = 0; j < (int)t.nz; ++j) {
            ring.acquire(j + 2);
            const uint32_t n = ((t.z0 + j) * N + t.y0 + warp) * N + t.x0 + lane;  // row warp; row warp + r CW at + r CW N
            T cp3[G::RW][3];
#pragma unroll
            for (int r = 0; r < G::RW; ++r)
#pragma unroll
                for (int k = 0; k < 3; ++k) cp3[r][k] = cc[r][k];
            if (j + 1 < (int)t.nz) load_c(n + N * N);
            T o_r[G::RW][3], o_z[G::RW][3];
#pragma unroll
            for (int r = 0; r < G::RW; ++r)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const U1SNb<G> S = ring.nb(j, lane, warp + r * G::CW);
                const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
                const T R = dx * (S(RQ_E + k1, 0, 0, 0) + S(RQ_E + k2, U1S_E(k1, 1)) - S(RQ_E + k1, U1S_E(k2, 1)) -
                                  S(RQ_E + k2, 0, 0, 0));
                const int e1[3] = {U1S_E(k1, 1)}, e2[3] = {U1S_E(k2, 1)}, ek[3] = {U1S_E(k, 1)};
                auto X = [&](int ox, int oy, int oz) {
                    return S(RQ_PHI, ox, oy, oz) *
                           (S(RQ_E + k, ox, oy, oz) + S(RQ_E + k, ox - ek[0], oy - ek[1], oz - ek[2]));
                };
                const T qs = X(0, 0, 0) + X(e1[0], e1[1], e1[2]) + X(e2[0], e2[1], e2[2]) +
                             X(e1[0] + e2[0], e1[1] + e2[1], e1[2] + e2[2]);
                o_r[r][k] = cp3[r][k] * R;
                o_z[r][k] = cp3[r][k] * ((T)0.5 * qs);
            }
            ring.release(j, lane);
#pragma unroll
            for (int r = 0; r < G::RW; ++r)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    A.rP[k][n + (uint32_t)(r * G::CW) * N] = o_r[r][k];
                    A.Z[k][n + (uint32_t)(r * G::CW) * N] = o_z[r][k];
                }
        }
        ring.release((int)t.nz, lane);
        ring.release((int)t.nz + 1, lane);
    }
    __syncthreads();  // producer and consumers meet; no copy is in flight past this point
    if (tid == 0 && s_fail) atomicOr(&A.scal->status, ST_TIMEOUT);
}

// TRACK: the first stage of a step, which also sums the squared lattice Gauss charge of its
// input state (the state at the step's start), so that the Gauss constraint is tracked each
// step; a separate instance keeps that work, and its registers, out of the other stages.
// LF: the passes of the leapfrog (U1Args::lf) instead of a Runge-Kutta stage.
template <typename T, bool TRACK, bool LF>
__global__ void __launch_bounds__(U1SGeom<T>::NT, 1) k_u1s_stage(const U1Args<T> A)
{
    using G = U1SGeom<T>;
    constexpr int NA = SG_NA;
    extern __shared__ __align__(128) unsigned char u1s_dyn[];
    __shared__ const T* s_src[NA];
    __shared__ __align__(8) uint64_t s_full[G::SLOTS], s_empty[G::SLOTS];
    __shared__ double s_coef[8];
    __shared__ double s_red[32][kMaxQ];
    __shared__ int s_last, s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool first = !LF && (A.flags & P_FIRST_STAGE) != 0;
    const int lf = LF ? A.lf : 0;
    const bool update = (A.flags & P_ENERGY_ONLY) == 0;
    constexpr bool track = TRACK;
    const bool expand = (A.flags & P_EXPANSION) != 0;
    if (tid == 0) {
        const double a = A.scal->a, b = expand ? A.scal->b : 0.0;
        s_coef[0] = apow(a, A.alpha - 3.0);                 // phi' = c0 pi
        s_coef[1] = apow(a, 1.0 + A.alpha) / (A.dx * A.dx);  // Laplacian
        s_coef[2] = apow(a, 3.0 + A.alpha);                 // potential
        s_coef[3] = apow(a, A.alpha - 1.0);                 // E' prefactor
        s_coef[4] = (1.0 - A.alpha) * b / a;               // electric friction
        s_coef[5] = a;
        s_coef[6] = apow(a, 1.0 - A.alpha);                 // a^(1-alpha) E in the Gauss charge
        s_coef[7] = LF && A.lf == 3 ? u1_lf_drift(a, b, A.h, A.alpha) : 0.0;  // leapfrog drift of phi
        s_src[SG_PHI] = A.phi_in;
        s_src[SG_PI] = A.pi_in;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            s_src[SG_E + k] = A.E_in[k];
            s_src[SG_SP + k] = A.sP[k];
            s_src[SG_RP + k] = A.rP[k];
            s_src[SG_Z + k] = A.Z[k];
        }
        for (int k = 0; k < G::SLOTS; ++k) {
            mbar_init(&s_full[k], G::PL);  // the producer lanes' copies
            mbar_init(&s_empty[k], G::CW);
        }
        mbar_fence_init();
        s_fail = 0;
    }
    __syncthreads();
    const U1STile<G> t((uint32_t)A.N, (uint32_t)A.dz);
    T* ring_sm = reinterpret_cast<T*>(u1s_dyn);
    uint2* table = reinterpret_cast<uint2*>(ring_sm + G::SLOTS * NA * G::ARR);
    u1s_build_units<G, NA>(table, t, tid, G::NT);
    __syncthreads();
    const U1SRing<G, NA> ring{ring_sm, table, s_full, s_empty, &s_fail};
    const uint32_t N = t.N, V = N * N * N;
    Acc<T> accK, accG, accV, accKE, accGs;
    if (warp >= G::CW) {
        ring.produce(tid - 32 * G::CW, s_src, t);
    } else {
        const T c_dphi = (T)s_coef[0], cL = (T)s_coef[1], cV = (T)s_coef[2], cE = (T)s_coef[3], cfr = (T)s_coef[4];
        const T ca = (T)s_coef[6];
        const T g = (T)A.g, ws2 = (T)A.ws2, dx = (T)A.dx, m2 = (T)A.m2, lam = (T)A.lam;
        const T inv_dx3 = (T)(1.0 / (A.dx * A.dx * A.dx)), inv4dx = (T)(0.25 / A.dx);
        const T inv4dx2 = (T)(0.25 / (A.dx * A.dx));
        const T h = (T)A.h, cA = (T)A.A, cB = (T)A.B;
        const T le = (T)A.le, lk = (T)A.lk, cdrift = (T)s_coef[7], hdx = (T)(A.h * A.dx);
        // site-only arrays (theta, the RK auxiliaries or the leapfrog's base momenta), loaded
        // one plane ahead
        T thc[3] = {}, kc[8] = {};
        auto load_site = [&](uint32_t m) {
            if constexpr (LF) {
                if (lf == 3) {
#pragma unroll
                    for (int i = 0; i < 3; ++i) thc[i] = A.th_in[i][m];
                }
                if (lf >= 2) {
                    kc[1] = A.k_in[1][m];
#pragma unroll
                    for (int i = 0; i < 3; ++i) kc[5 + i] = A.k_in[5 + i][m];
                }
            } else {
#pragma unroll
                for (int i = 0; i < 3; ++i) thc[i] = A.th_in[i][m];
#pragma unroll
                for (int q = 0; q < 8; ++q) kc[q] = first ? (T)0 : A.k_in[q][m];
            }
        };
        if (update) load_site((t.z0 * N + t.y0 + warp) * N + t.x0 + lane);
        ring.acquire(0);
        ring.acquire(1);
        for (int j = 0; j < (int)t.nz; ++j) {
            ring.acquire(j + 2);
            const U1SNb<G> S = ring.nb(j, lane, warp);
            const uint32_t n = ((t.z0 + j) * N + t.y0 + warp) * N + t.x0 + lane;
            T thv[3], kv[8];
#pragma unroll
            for (int i = 0; i < 3; ++i) thv[i] = thc[i];
#pragma unroll
            for (int q = 0; q < 8; ++q) kv[q] = kc[q];
            if (update && j + 1 < (int)t.nz) load_site(n + N * N);
            if (update && j + 2 < (int)t.nz) {
                // the site-only arrays of the plane after next into L2 (one 128-byte row a
                // lane), so that the loads one plane ahead wait on L2 rather than DRAM
                const T* pf = nullptr;
                if constexpr (LF) {
                    if (lane < 3) pf = lf == 3 ? A.th_in[lane] : nullptr;
                    else if (lane == 3) pf = lf >= 2 ? A.k_in[1] : nullptr;
                    else if (lane < 7) pf = lf >= 2 ? A.k_in[1 + lane] : nullptr;
                } else {
                    if (lane < 3) pf = A.th_in[lane];
                    else if (lane < 11 && !first) pf = A.k_in[lane - 3];
                }
                if (pf) prefetch_l2(pf + n + 2 * N * N);
            }

            // scalar sector
            const T ph = S(SG_PHI, 0, 0, 0), pv = S(SG_PI, 0, 0, 0);
            const T pxp = S(SG_PHI, 1, 0, 0), pxm = S(SG_PHI, -1, 0, 0);
            const T pyp = S(SG_PHI, 0, 1, 0), pym = S(SG_PHI, 0, -1, 0);
            const T pzp = S(SG_PHI, 0, 0, 1), pzm = S(SG_PHI, 0, 0, -1);
            const T lap = ((pxp + pxm) + (pyp + pym) + (pzp + pzm)) - (T)6 * ph;
            const T dV = ph * (m2 + lam * ph * ph);
            T eb = (T)0, e2 = (T)0;
            T Ecur[3], Bn[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                Ecur[k] = S(SG_E + k, 0, 0, 0);
                Bn[k] = inv4dx2 * S.clover(SG_SP + k, k, 0, 0, 0);
                eb += (T)0.5 * (Ecur[k] + S(SG_E + k, U1S_E(k, -1))) * Bn[k];
                e2 += Ecur[k] * Ecur[k];
            }
            const T F_phi = c_dphi * pv;
            const T F_pi = cL * lap - cV * dV + ws2 * g * eb;
            if (!LF) {  // (leapfrog pass 1 sums the kinetic energies of its output momenta)
                accK.add(pv * pv);
                accKE.add(e2);
            }
            if (!LF || lf == 1) {
                accG.add((pxp - ph) * (pxp - ph) + (pyp - ph) * (pyp - ph) + (pzp - ph) * (pzp - ph));
                accV.add(ph * ph * ((T)0.5 * m2 + (T)0.25 * lam * ph * ph));
            }
            if (update) {
                if constexpr (TRACK) {
                    // dx times the lattice Gauss charge sum_i [P_i(n) - P_i(n - i)] of the input
                    // state, P_i = a^(1-alpha) E_i + g W_i (the phi B terms at n cancel).  The
                    // leapfrog's second pass tracks the integer-time state of the step's start:
                    // its positions are staged, its electric field is the base (site and the
                    // three lower neighbours, loaded here)
                    T ec[3], em[3];
                    if constexpr (LF) {
                        const uint32_t x = t.x0 + lane, y = t.y0 + warp, z = t.z0 + j;
                        const uint32_t nm[3] = {x == 0 ? n + N - 1 : n - 1, y == 0 ? n + (N - 1) * N : n - N,
                                                z == 0 ? n + (N - 1) * N * N : n - N * N};
#pragma unroll
                        for (int i = 0; i < 3; ++i) {
                            ec[i] = kv[5 + i];
                            em[i] = A.k_in[5 + i][nm[i]];
                        }
                        accKE.add(ec[0] * ec[0] + ec[1] * ec[1] + ec[2] * ec[2]);
                    } else {
#pragma unroll
                        for (int i = 0; i < 3; ++i) {
                            ec[i] = Ecur[i];
                            em[i] = S(SG_E + i, U1S_E(i, -1));
                        }
                    }
                    T gd = (T)0;
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        const T Bpi = inv4dx2 * S.clover(SG_SP + i, i, U1S_E(i, 1));
                        const T Bmi = inv4dx2 * S.clover(SG_SP + i, i, U1S_E(i, -1));
                        gd += ca * (ec[i] - em[i]) +
                              (T)0.5 * g * (S(SG_PHI, U1S_E(i, 1)) * Bpi - S(SG_PHI, U1S_E(i, -1)) * Bmi);
                    }
                    accGs.add(gd * gd);
                }
                // link forces
                T F_E[3];
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const int ip = (i + 1) % 3, im = (i + 2) % 3;
                    const T mag = (S(SG_SP + im, 0, 0, 0) - S(SG_SP + im, U1S_E(ip, -1))) -
                                  (S(SG_SP + ip, 0, 0, 0) - S(SG_SP + ip, U1S_E(im, -1)));
                    const T cs = (S(SG_Z + im, 0, 0, 0) - S(SG_Z + im, U1S_E(ip, -1))) +
                                 (S(SG_Z + ip, U1S_E(im, -1)) - S(SG_Z + ip, 0, 0, 0));
                    const T Bdn = inv4dx2 * S.clover(SG_RP + i, i, 0, 0, 0);
                    const T Bni = inv4dx2 * S.clover(SG_SP + i, i, U1S_E(i, 1));
                    const T Bdni = inv4dx2 * S.clover(SG_RP + i, i, U1S_E(i, 1));
                    const T wdot = (T)0.5 * (F_phi * Bn[i] + ph * Bdn + c_dphi * S(SG_PI, U1S_E(i, 1)) * Bni +
                                             S(SG_PHI, U1S_E(i, 1)) * Bdni);
                    F_E[i] = cE * (-cE * mag * inv_dx3 + g * (cs * inv4dx - wdot)) - cfr * Ecur[i];
                }
                ring.release(j, lane);
                if constexpr (LF) {
                    if (lf == 1) {  // closing half-kick (integer-time momenta) and the first iterate
                        T En[3], Eo[3], en2 = (T)0;
#pragma unroll
                        for (int i = 0; i < 3; ++i) {
                            En[i] = Ecur[i] + le * F_E[i];
                            Eo[i] = Ecur[i] + lk * F_E[i];
                            en2 += En[i] * En[i];
                        }
                        const T pn = pv + le * F_pi;
                        accK.add(pn * pn);
                        accKE.add(en2);
                        A.k_out[1][n] = pn;
                        A.pi_out[n] = pv + lk * F_pi;
#pragma unroll
                        for (int i = 0; i < 3; ++i) {
                            A.k_out[5 + i][n] = En[i];
                            A.E_out[i][n] = Eo[i];
                        }
                    } else {  // an iterate of the implicit kick from the base momenta
                        const T po = kv[1] + lk * F_pi;
                        T Eo[3];
#pragma unroll
                        for (int i = 0; i < 3; ++i) Eo[i] = kv[5 + i] + lk * F_E[i];
                        if (lf == 3) {
                            A.phi_out[n] = ph + cdrift * po;
#pragma unroll
                            for (int i = 0; i < 3; ++i) A.th_out[i][n] = thv[i] + hdx * Eo[i];
                        }
                        A.pi_out[n] = po;
#pragma unroll
                        for (int i = 0; i < 3; ++i) A.E_out[i][n] = Eo[i];
                    }
                    continue;
                }
                // 2N Runge-Kutta update of the eight degrees of freedom of this site
                const T F[8] = {F_phi, F_pi, dx * Ecur[0], dx * Ecur[1], dx * Ecur[2], F_E[0], F_E[1], F_E[2]};
                const T y[8] = {ph, pv, thv[0], thv[1], thv[2], Ecur[0], Ecur[1], Ecur[2]};
                T kq[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) kq[q] = first ? h * F[q] : cA * kv[q] + h * F[q];
                T* out[8] = {A.phi_out, A.pi_out, A.th_out[0], A.th_out[1], A.th_out[2], A.E_out[0], A.E_out[1],
                             A.E_out[2]};
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    A.k_out[q][n] = kq[q];
                    out[q][n] = y[q] + cB * kq[q];
                }
            } else {
                ring.release(j, lane);
            }
        }
        ring.release((int)t.nz, lane);
        ring.release((int)t.nz + 1, lane);
    }
    __syncthreads();  // producer and consumers meet; no copy is in flight past this point

    // ---- block partials; last block: energies of the old state and the (a, a') stage ----
    // slot 4 of the stage's partials carries the Gauss sum (the magnetic energy's partials
    // follow in the plaquette launch's region)
    double v[kMaxQ];
    const Acc<T>* av[kMaxQ] = {&accK, &accG, &accV, &accKE, &accGs};
    block_reduce_acc<T, kMaxQ>(av, v, s_red, tid, G::NT);
    if (tid == 0) {
        if (s_fail) atomicOr(&A.scal->status, ST_TIMEOUT);
#pragma unroll
        for (int q = 0; q < kMaxQ; ++q) A.partials[(size_t)blockIdx.x * kMaxQ + q] = v[q];
        __threadfence();
        const unsigned prev = atomicAdd(&A.scal->counter, 1u);
        s_last = (prev + 1u == gridDim.x);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (tid >= 32) return;  // one warp sums the grid's partials, its lane 0 runs the epilogue
    double ws[kMaxQ];  // the stage's sums; slot 4 is the Gauss sum
    warp_sum_partials<kMaxQ>(A.partials, (int)gridDim.x, tid, ws);
    double gb = 0.0;  // the magnetic energy from the plaquette launch (same grid, one value a block)
    for (int b = tid; b < (int)gridDim.x; b += 32) gb += __ldcg(&A.partials[(size_t)gridDim.x * kMaxQ + b]);
    for (int off = 16; off > 0; off >>= 1) gb += __shfl_xor_sync(0xffffffffu, gb, off);
    double w[kMaxQ] = {ws[0], ws[1], ws[2], ws[3], gb};
    double wg[1] = {ws[kMaxQ - 1]};
    if (tid == 0) {
        if (track) u1_gauss_track(A.scal, wg[0], w[3], s_coef[6]);
        if (LF) u1_lf_epilogue(A, w, s_coef[5], expand, V);
        else u1_epilogue(A, w, s_coef[5], first, update, expand, V);
    }
}

// ---------------------------------------------------------------- fused staged stage
// One launch per stage (or leapfrog pass): the plaquette fields live in shared memory instead
// of going through global memory.  The producer warps stage the eight raw arrays (phi, pi,
// theta_1..3, E_1..3) plane by plane as above; the consumer warps, for output plane z, first
// compute the plaquettes of normal x and y at plane z and of normal z at plane z + 1 over the
// tile and the halo the stage reads (one consumer barrier per plane separates writers from
// readers), then run the stage of plane z with every
// plaquette field from shared memory and theta from the staged planes.  Ranges (relative to
// the tile origin): normal x, columns -1..32, rows -1..TY-1; normal y, columns -1..31, rows
// -1..TY; normal z, columns -1..31, rows -1..TY-1 (column -1 of normal x and row -1 of normal
// y only for the Gauss charge, which needs the clover field at n - e_i; row -1 of normal y
// has no Chern-Simons field, whose corner sum would reach row -2).  The magnetic energy of a
// plaquette is counted by the block that owns its corner.  The plaquette planes rotate through
// four slots: a warp that runs one plane ahead writes a slot that no warp still on the previous
// plane reads (that plane's stage reads the slots of its planes z - 1 .. z + 1).
template <typename T>
struct U1FPq {
    using G = U1SGeom<T>;
    static constexpr int X = G::TX + 2;            // columns -1 .. TX
    static constexpr int Y = G::TY + 2;            // rows -1 .. TY
    static constexpr int PLANE = X * Y;            // one field of one orientation
    static constexpr int SLOT = 9 * PLANE;         // three orientations x (sin P, cos P dP/dt, Z)
    static constexpr int NSLOT = 4;
};

template <typename T>
constexpr size_t u1f_smem_bytes()
{
    return u1s_smem_bytes<U1SGeom<T>, 8>() + (size_t)U1FPq<T>::NSLOT * U1FPq<T>::SLOT * sizeof(T);
}

enum { FR_PHI = 0, FR_PI = 1, FR_TH = 2, FR_E = 5, FR_NA = 8 };

// Raw staged planes c - 1, c, c + 1 (chunk-relative plane indices) around the point at tile
// offset (lx, ly) (lx in -VE .. TX + VE - 1, ly in -1 .. TY).
template <typename T>
__device__ __forceinline__ U1SNb<U1SGeom<T>> u1f_raw(const T* ring, int c, int lx, int ly)
{
    using G = U1SGeom<T>;
    constexpr size_t SL = (size_t)FR_NA * G::ARR;
    const int t0 = (ly + 1) * G::PW + lx + G::VE;
    U1SNb<U1SGeom<T>> n;
#pragma unroll
    for (int i = 0; i < 3; ++i) n.p[i] = ring + ((c - 1 + i + G::SLOTS) % G::SLOTS) * SL + t0;
    return n;
}

// Plaquette fields around a site at tile offset (lx, ly) of the output plane whose
// chunk-relative index is c (plaquette planes c - 1 .. c + 1 for the offsets oz = -1 .. 1).
template <typename T>
struct U1FQ {
    const T* pq;
    int c, lx, ly;
    __device__ __forceinline__ T operator()(int k, int f, int ox, int oy, int oz) const
    {
        using P = U1FPq<T>;
        return pq[((c + oz) % P::NSLOT) * P::SLOT + (k * 3 + f) * P::PLANE + (ly + oy + 1) * P::X + lx + ox + 1];
    }
    // clover sum of field f of normal k over the four plaquettes around offset o
    __device__ __forceinline__ T clover(int f, int k, int ox, int oy, int oz) const
    {
        const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
        int b[3] = {ox, oy, oz}, d[3] = {ox, oy, oz}, e[3];
        b[k1] -= 1;
        d[k2] -= 1;
        e[0] = b[0]; e[1] = b[1]; e[2] = b[2];
        e[k2] -= 1;
        return ((*this)(k, f, ox, oy, oz) + (*this)(k, f, b[0], b[1], b[2])) +
               ((*this)(k, f, d[0], d[1], d[2]) + (*this)(k, f, e[0], e[1], e[2]));
    }
};

// Plaquettes of normal K at plane c (chunk-relative), into slot c % 4; `count` adds the
// magnetic energy of the corners this block owns; with_z: the Chern-Simons field too (normal
// z needs raw plane c - 1 for it).  K is a template parameter so that every offset folds.
template <typename T, int K>
__device__ __forceinline__ void u1f_plaquettes(T* pq, const T* ring, int c, bool with_z, bool count, T dx, int ctid,
                                               Acc<T>& accGB)
{
    using G = U1SGeom<T>;
    using P = U1FPq<T>;
    constexpr int NT = 32 * G::CW;
    // corners: normal x columns -1..TX, rows -1..TY-1; normal y columns -1..TX-1, rows -1..TY;
    // normal z columns -1..TX-1, rows -1..TY-1 (tile offsets; xo, yo count from -1)
    constexpr int W = K == 0 ? G::TX + 2 : G::TX + 1;
    constexpr int H = K == 1 ? G::TY + 2 : G::TY + 1;
    constexpr int K1 = (K + 1) % 3, K2 = (K + 2) % 3;
    constexpr int e1x = K1 == 0, e1y = K1 == 1, e1z = K1 == 2;
    constexpr int e2x = K2 == 0, e2y = K2 == 1, e2z = K2 == 2;
    constexpr int ekx = K == 0, eky = K == 1, ekz = K == 2;
    T* slot = pq + (c % P::NSLOT) * P::SLOT + (K * 3) * P::PLANE;
    for (int w = ctid; w < W * H; w += NT) {
        const int xo = w % W, yo = w / W;
        const U1SNb<U1SGeom<T>> S = u1f_raw<T>(ring, c, xo - 1, yo - 1);
        const T Pl = S(FR_TH + K1, 0, 0, 0) + S(FR_TH + K2, e1x, e1y, e1z) - S(FR_TH + K1, e2x, e2y, e2z) -
                     S(FR_TH + K2, 0, 0, 0);
        const T R = dx * (S(FR_E + K1, 0, 0, 0) + S(FR_E + K2, e1x, e1y, e1z) - S(FR_E + K1, e2x, e2y, e2z) -
                          S(FR_E + K2, 0, 0, 0));
        T sh, ch;  // sin, cos of P / 2
        if constexpr (sizeof(T) == 4) sincosf((T)0.5 * Pl, &sh, &ch);
        else sincos((T)0.5 * Pl, &sh, &ch);
        const T sp = (T)2 * sh * ch, cp = (T)1 - (T)2 * sh * sh;
        // the corner sum of phi Ebar_k reaches one row / plane below the corner along k: not
        // formed for row -1 of normal y (never read) nor when the plane below is not staged
        T z = (T)0;
        if ((K != 1 || yo > 0) && (K != 2 || with_z)) {
            auto X = [&](int ox, int oy, int oz) {
                return S(FR_PHI, ox, oy, oz) * (S(FR_E + K, ox, oy, oz) + S(FR_E + K, ox - ekx, oy - eky, oz - ekz));
            };
            const T qs = X(0, 0, 0) + X(e1x, e1y, e1z) + X(e2x, e2y, e2z) + X(e1x + e2x, e1y + e2y, e1z + e2z);
            z = cp * ((T)0.5 * qs);
        }
        const int at = yo * P::X + xo;
        slot[at] = sp;
        slot[at + P::PLANE] = cp * R;
        slot[at + 2 * P::PLANE] = z;
        // owned corners: tile columns 0..TX-1, rows 0..TY-1
        if (count && xo >= 1 && xo <= G::TX && yo >= 1 && yo <= G::TY) accGB.add((T)2 * sh * sh);
    }
}

__device__ __forceinline__ void u1f_consumer_barrier(int nthreads)
{
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

template <typename T, bool TRACK, bool LF>
__global__ void __launch_bounds__(U1SGeom<T>::NT, 1) k_u1f_stage(const U1Args<T> A)
{
    using G = U1SGeom<T>;
    constexpr int NA = FR_NA;
    extern __shared__ __align__(128) unsigned char u1s_dyn[];
    __shared__ const T* s_src[NA];
    __shared__ __align__(8) uint64_t s_full[G::SLOTS], s_empty[G::SLOTS];
    __shared__ double s_coef[8];
    __shared__ double s_red[32][kMaxQ];
    __shared__ int s_last, s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool first = !LF && (A.flags & P_FIRST_STAGE) != 0;
    const int lf = LF ? A.lf : 0;
    const bool update = (A.flags & P_ENERGY_ONLY) == 0;
    constexpr bool track = TRACK;
    const bool expand = (A.flags & P_EXPANSION) != 0;
    if (tid == 0) {
        const double a = A.scal->a, b = expand ? A.scal->b : 0.0;
        s_coef[0] = apow(a, A.alpha - 3.0);                 // phi' = c0 pi
        s_coef[1] = apow(a, 1.0 + A.alpha) / (A.dx * A.dx);  // Laplacian
        s_coef[2] = apow(a, 3.0 + A.alpha);                 // potential
        s_coef[3] = apow(a, A.alpha - 1.0);                 // E' prefactor
        s_coef[4] = (1.0 - A.alpha) * b / a;               // electric friction
        s_coef[5] = a;
        s_coef[6] = apow(a, 1.0 - A.alpha);                 // a^(1-alpha) E in the Gauss charge
        s_coef[7] = LF && A.lf == 3 ? u1_lf_drift(a, b, A.h, A.alpha) : 0.0;  // leapfrog drift of phi
        s_src[FR_PHI] = A.phi_in;
        s_src[FR_PI] = A.pi_in;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            s_src[FR_TH + k] = A.th_in[k];
            s_src[FR_E + k] = A.E_in[k];
        }
        for (int k = 0; k < G::SLOTS; ++k) {
            mbar_init(&s_full[k], G::PL);  // the producer lanes' copies
            mbar_init(&s_empty[k], G::CW);
        }
        mbar_fence_init();
        s_fail = 0;
    }
    __syncthreads();
    const U1STile<G> t((uint32_t)A.N, (uint32_t)A.dz);
    T* ring_sm = reinterpret_cast<T*>(u1s_dyn);
    uint2* table = reinterpret_cast<uint2*>(ring_sm + G::SLOTS * NA * G::ARR);
    T* pq = reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(u1s_dyn) + u1s_smem_bytes<G, NA>());
    u1s_build_units<G, NA>(table, t, tid, G::NT);
    __syncthreads();
    const U1SRing<G, NA> ring{ring_sm, table, s_full, s_empty, &s_fail};
    const uint32_t N = t.N, V = N * N * N;
    Acc<T> accK, accG, accV, accKE, accGs, accGB;
    if (warp >= G::CW) {
        ring.produce(tid - 32 * G::CW, s_src, t);
    } else {
        const T c_dphi = (T)s_coef[0], cL = (T)s_coef[1], cV = (T)s_coef[2], cE = (T)s_coef[3], cfr = (T)s_coef[4];
        const T ca = (T)s_coef[6];
        const T g = (T)A.g, ws2 = (T)A.ws2, dx = (T)A.dx, m2 = (T)A.m2, lam = (T)A.lam;
        const T inv_dx3 = (T)(1.0 / (A.dx * A.dx * A.dx)), inv4dx = (T)(0.25 / A.dx);
        const T inv4dx2 = (T)(0.25 / (A.dx * A.dx));
        const T h = (T)A.h, cA = (T)A.A, cB = (T)A.B;
        const T le = (T)A.le, lk = (T)A.lk, cdrift = (T)s_coef[7], hdx = (T)(A.h * A.dx);
        const int nz = (int)t.nz;
        // site-only arrays (the Runge-Kutta auxiliaries or the leapfrog's base momenta), loaded
        // one plane ahead
        T kc[8] = {};
        auto load_site = [&](uint32_t m) {
            if constexpr (LF) {
                if (lf >= 2) {
                    kc[1] = A.k_in[1][m];
#pragma unroll
                    for (int i = 0; i < 3; ++i) kc[5 + i] = A.k_in[5 + i][m];
                }
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) kc[q] = first ? (T)0 : A.k_in[q][m];
            }
        };
        if (update) load_site((t.z0 * N + t.y0 + warp) * N + t.x0 + lane);
        // plaquette planes before the march: normal x and y at plane z0 - 1, normal z at z0
        // (and, for the Gauss charge, its sin P at z0 - 1)
        ring.acquire(0);
        ring.acquire(1);
        u1f_plaquettes<T, 0>(pq, ring_sm, 0, true, false, dx, tid, accGB);
        u1f_plaquettes<T, 1>(pq, ring_sm, 0, true, false, dx, tid, accGB);
        if (TRACK) u1f_plaquettes<T, 2>(pq, ring_sm, 0, false, false, dx, tid, accGB);
        u1f_plaquettes<T, 2>(pq, ring_sm, 1, true, nz > 0, dx, tid, accGB);
        for (int j = 0; j < nz; ++j) {
            ring.acquire(j + 2);
            // normal x, y at plane z0 + j (chunk-relative j + 1), normal z at plane z0 + j + 1
            u1f_plaquettes<T, 0>(pq, ring_sm, j + 1, true, true, dx, tid, accGB);
            u1f_plaquettes<T, 1>(pq, ring_sm, j + 1, true, true, dx, tid, accGB);
            u1f_plaquettes<T, 2>(pq, ring_sm, j + 2, true, j + 1 < nz, dx, tid, accGB);
            u1f_consumer_barrier(32 * G::CW);
            const U1SNb<U1SGeom<T>> S = u1f_raw<T>(ring_sm, j + 1, lane, warp);
            const U1FQ<T> Q{pq, j + 1, lane, warp};
            const uint32_t n = ((t.z0 + j) * N + t.y0 + warp) * N + t.x0 + lane;
            T kv[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) kv[q] = kc[q];
            if (update && j + 1 < nz) load_site(n + N * N);

            // scalar sector
            const T ph = S(FR_PHI, 0, 0, 0), pv = S(FR_PI, 0, 0, 0);
            const T pxp = S(FR_PHI, 1, 0, 0), pxm = S(FR_PHI, -1, 0, 0);
            const T pyp = S(FR_PHI, 0, 1, 0), pym = S(FR_PHI, 0, -1, 0);
            const T pzp = S(FR_PHI, 0, 0, 1), pzm = S(FR_PHI, 0, 0, -1);
            const T lap = ((pxp + pxm) + (pyp + pym) + (pzp + pzm)) - (T)6 * ph;
            const T dV = ph * (m2 + lam * ph * ph);
            T eb = (T)0, e2 = (T)0;
            T Ecur[3], Bn[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                Ecur[k] = S(FR_E + k, 0, 0, 0);
                Bn[k] = inv4dx2 * Q.clover(0, k, 0, 0, 0);
                eb += (T)0.5 * (Ecur[k] + S(FR_E + k, U1S_E(k, -1))) * Bn[k];
                e2 += Ecur[k] * Ecur[k];
            }
            const T F_phi = c_dphi * pv;
            const T F_pi = cL * lap - cV * dV + ws2 * g * eb;
            if (!LF) {  // (leapfrog pass 1 sums the kinetic energies of its output momenta)
                accK.add(pv * pv);
                accKE.add(e2);
            }
            if (!LF || lf == 1) {
                accG.add((pxp - ph) * (pxp - ph) + (pyp - ph) * (pyp - ph) + (pzp - ph) * (pzp - ph));
                accV.add(ph * ph * ((T)0.5 * m2 + (T)0.25 * lam * ph * ph));
            }
            if (update) {
                if constexpr (TRACK) {
                    // dx times the lattice Gauss charge of the input state (the leapfrog's:
                    // the integer-time state, its electric field the base momenta)
                    T ec[3], em[3];
                    if constexpr (LF) {
                        const uint32_t x = t.x0 + lane, y = t.y0 + warp, z = t.z0 + j;
                        const uint32_t nm[3] = {x == 0 ? n + N - 1 : n - 1, y == 0 ? n + (N - 1) * N : n - N,
                                                z == 0 ? n + (N - 1) * N * N : n - N * N};
#pragma unroll
                        for (int i = 0; i < 3; ++i) {
                            ec[i] = kv[5 + i];
                            em[i] = A.k_in[5 + i][nm[i]];
                        }
                        accKE.add(ec[0] * ec[0] + ec[1] * ec[1] + ec[2] * ec[2]);
                    } else {
#pragma unroll
                        for (int i = 0; i < 3; ++i) {
                            ec[i] = Ecur[i];
                            em[i] = S(FR_E + i, U1S_E(i, -1));
                        }
                    }
                    T gd = (T)0;
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        const T Bpi = inv4dx2 * Q.clover(0, i, U1S_E(i, 1));
                        const T Bmi = inv4dx2 * Q.clover(0, i, U1S_E(i, -1));
                        gd += ca * (ec[i] - em[i]) +
                              (T)0.5 * g * (S(FR_PHI, U1S_E(i, 1)) * Bpi - S(FR_PHI, U1S_E(i, -1)) * Bmi);
                    }
                    accGs.add(gd * gd);
                }
                // link forces
                T F_E[3];
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const int ip = (i + 1) % 3, im = (i + 2) % 3;
                    const T mag = (Q(im, 0, 0, 0, 0) - Q(im, 0, U1S_E(ip, -1))) - (Q(ip, 0, 0, 0, 0) - Q(ip, 0, U1S_E(im, -1)));
                    const T cs = (Q(im, 2, 0, 0, 0) - Q(im, 2, U1S_E(ip, -1))) + (Q(ip, 2, U1S_E(im, -1)) - Q(ip, 2, 0, 0, 0));
                    const T Bdn = inv4dx2 * Q.clover(1, i, 0, 0, 0);
                    const T Bni = inv4dx2 * Q.clover(0, i, U1S_E(i, 1));
                    const T Bdni = inv4dx2 * Q.clover(1, i, U1S_E(i, 1));
                    const T wdot = (T)0.5 * (F_phi * Bn[i] + ph * Bdn + c_dphi * S(FR_PI, U1S_E(i, 1)) * Bni +
                                             S(FR_PHI, U1S_E(i, 1)) * Bdni);
                    F_E[i] = cE * (-cE * mag * inv_dx3 + g * (cs * inv4dx - wdot)) - cfr * Ecur[i];
                }
                const T thv[3] = {S(FR_TH + 0, 0, 0, 0), S(FR_TH + 1, 0, 0, 0), S(FR_TH + 2, 0, 0, 0)};
                ring.release(j, lane);
                if constexpr (LF) {
                    if (lf == 1) {  // closing half-kick (integer-time momenta) and the first iterate
                        T En[3], Eo[3], en2 = (T)0;
#pragma unroll
                        for (int i = 0; i < 3; ++i) {
                            En[i] = Ecur[i] + le * F_E[i];
                            Eo[i] = Ecur[i] + lk * F_E[i];
                            en2 += En[i] * En[i];
                        }
                        const T pn = pv + le * F_pi;
                        accK.add(pn * pn);
                        accKE.add(en2);
                        A.k_out[1][n] = pn;
                        A.pi_out[n] = pv + lk * F_pi;
#pragma unroll
                        for (int i = 0; i < 3; ++i) {
                            A.k_out[5 + i][n] = En[i];
                            A.E_out[i][n] = Eo[i];
                        }
                    } else {  // an iterate of the implicit kick from the base momenta
                        const T po = kv[1] + lk * F_pi;
                        T Eo[3];
#pragma unroll
                        for (int i = 0; i < 3; ++i) Eo[i] = kv[5 + i] + lk * F_E[i];
                        if (lf == 3) {
                            A.phi_out[n] = ph + cdrift * po;
#pragma unroll
                            for (int i = 0; i < 3; ++i) A.th_out[i][n] = thv[i] + hdx * Eo[i];
                        }
                        A.pi_out[n] = po;
#pragma unroll
                        for (int i = 0; i < 3; ++i) A.E_out[i][n] = Eo[i];
                    }
                } else {
                    // 2N Runge-Kutta update of the eight degrees of freedom of this site
                    const T F[8] = {F_phi, F_pi, dx * Ecur[0], dx * Ecur[1], dx * Ecur[2], F_E[0], F_E[1], F_E[2]};
                    const T y[8] = {ph, pv, thv[0], thv[1], thv[2], Ecur[0], Ecur[1], Ecur[2]};
                    T kq[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) kq[q] = first ? h * F[q] : cA * kv[q] + h * F[q];
                    T* out[8] = {A.phi_out, A.pi_out, A.th_out[0], A.th_out[1], A.th_out[2], A.E_out[0], A.E_out[1],
                                 A.E_out[2]};
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        A.k_out[q][n] = kq[q];
                        out[q][n] = y[q] + cB * kq[q];
                    }
                }
            } else {
                ring.release(j, lane);
            }
        }
        ring.release(nz, lane);
        ring.release(nz + 1, lane);
    }
    __syncthreads();  // producer and consumers meet; no copy is in flight past this point

    // ---- block partials; last block: energies of the old state and the (a, a') stage ----
    // the stage's five sums (slot 4 the Gauss sum), the magnetic energy after them (one value a
    // block, as the plaquette launch of the two-launch form leaves it)
    double v[kMaxQ];
    const Acc<T>* av[kMaxQ] = {&accK, &accG, &accV, &accKE, &accGs};
    block_reduce_acc<T, kMaxQ>(av, v, s_red, tid, G::NT);
    double vb[1];
    const Acc<T>* ab[1] = {&accGB};
    block_reduce_acc<T, 1>(ab, vb, s_red, tid, G::NT);
    if (tid == 0) {
        if (s_fail) atomicOr(&A.scal->status, ST_TIMEOUT);
#pragma unroll
        for (int q = 0; q < kMaxQ; ++q) A.partials[(size_t)blockIdx.x * kMaxQ + q] = v[q];
        A.partials[(size_t)gridDim.x * kMaxQ + blockIdx.x] = vb[0];
        __threadfence();
        const unsigned prev = atomicAdd(&A.scal->counter, 1u);
        s_last = (prev + 1u == gridDim.x);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (tid >= 32) return;  // one warp sums the grid's partials, its lane 0 runs the epilogue
    double ws[kMaxQ];
    warp_sum_partials<kMaxQ>(A.partials, (int)gridDim.x, tid, ws);
    double gb = 0.0;
    for (int b = tid; b < (int)gridDim.x; b += 32) gb += __ldcg(&A.partials[(size_t)gridDim.x * kMaxQ + b]);
    for (int off = 16; off > 0; off >>= 1) gb += __shfl_xor_sync(0xffffffffu, gb, off);
    double w[kMaxQ] = {ws[0], ws[1], ws[2], ws[3], gb};
    if (tid == 0) {
        if (track) u1_gauss_track(A.scal, ws[kMaxQ - 1], w[3], s_coef[6]);
        if (LF) u1_lf_epilogue(A, w, s_coef[5], expand, V);
        else u1_epilogue(A, w, s_coef[5], first, update, expand, V);
    }
}

#undef U1S_E

bool u1_staged_ok(int N) { return N >= 32 && N % 32 == 0; }

int u1_staged_blocks(int precision, int N, int dz)
{
    const int ty = precision == CL_PREC_FP64 ? U1SGeom<double>::TY : U1SGeom<float>::TY;
    return (N / 32) * (N / ty) * ((N + dz - 1) / dz);
}

// z chunk of the staged launches: one block per SM at a time, so the chunk count minimises
// waves x (planes + 2 halo planes) of the busiest SM.
int u1_staged_dz(int precision, int N, int nsm)
{
    const int ty = precision == CL_PREC_FP64 ? U1SGeom<double>::TY : U1SGeom<float>::TY;
    const long long tiles = (long long)(N / 32) * (N / ty);
    long long best = -1;
    int best_dz = N;
    for (int nbz = 1; nbz <= N; ++nbz) {
        const int dz = (N + nbz - 1) / nbz;
        if ((N + dz - 1) / dz != nbz) continue;  // same chunks as a smaller count
        const long long waves = (tiles * nbz + nsm - 1) / nsm;
        const long long cost = waves * (dz + 2);
        if (best < 0 || cost < best) {
            best = cost;
            best_dz = dz;
        }
    }
    return best_dz;
}

template <typename T>
static cudaError_t launch_u1s_t(const U1Args<T>& A, int what, cudaStream_t s)
{
    using G = U1SGeom<T>;
    if (!u1_staged_ok(A.N) || A.dz < 1 || A.dz > A.N) return cudaErrorInvalidValue;
    const int grid = u1_staged_blocks(sizeof(T) == 8 ? CL_PREC_FP64 : CL_PREC_FP32, A.N, A.dz);
    static DevFlag attr[5];
    if (what == 0) {
        constexpr size_t smem = u1s_smem_bytes<U1PGeom<T>, PQ_NA>();
        if (!attr[0]) {
            const cudaError_t e =
                cudaFuncSetAttribute(k_u1s_plaquettes<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            attr[0] = true;
        }
        k_u1s_plaquettes<T><<<grid, U1PGeom<T>::NT, smem, s>>>(A);
    } else if (what == 3) {
        constexpr size_t smem = u1s_smem_bytes<U1PGeom<T>, RQ_NA>();
        if (!A.cP[0] || !A.cP[1] || !A.cP[2]) return cudaErrorInvalidValue;
        static DevFlag rattr;
        if (!rattr) {
            const cudaError_t e =
                cudaFuncSetAttribute(k_u1s_plaquette_rates<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            rattr = true;
        }
        k_u1s_plaquette_rates<T><<<grid, U1PGeom<T>::NT, smem, s>>>(A);
    } else if (what == 2) {
        constexpr size_t smem = u1f_smem_bytes<T>();
        const int form = A.lf ? (A.lf == 2 ? 4 : 3) : ((A.flags & P_FIRST_STAGE) && !(A.flags & P_ENERGY_ONLY) ? 2 : 1);
        static DevFlag fattr[5];
        if (!fattr[form]) {
            const int sm = (int)smem;
            const cudaError_t e =
                form == 4   ? cudaFuncSetAttribute(k_u1f_stage<T, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)
                : form == 3 ? cudaFuncSetAttribute(k_u1f_stage<T, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)
                : form == 2 ? cudaFuncSetAttribute(k_u1f_stage<T, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)
                            : cudaFuncSetAttribute(k_u1f_stage<T, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            if (e != cudaSuccess) return e;
            fattr[form] = true;
        }
        if (form == 4) k_u1f_stage<T, true, true><<<grid, G::NT, smem, s>>>(A);
        else if (form == 3) k_u1f_stage<T, false, true><<<grid, G::NT, smem, s>>>(A);
        else if (form == 2) k_u1f_stage<T, true, false><<<grid, G::NT, smem, s>>>(A);
        else k_u1f_stage<T, false, false><<<grid, G::NT, smem, s>>>(A);
    } else {
        constexpr size_t smem = u1s_smem_bytes<U1SGeom<T>, SG_NA>();
        // forms: 1 a Runge-Kutta stage, 2 the first stage of a step (Gauss tracking), 3 a
        // leapfrog pass, 4 the leapfrog's second pass (Gauss tracking)
        const int form = A.lf ? (A.lf == 2 ? 4 : 3) : ((A.flags & P_FIRST_STAGE) && !(A.flags & P_ENERGY_ONLY) ? 2 : 1);
        if (!attr[form]) {
            const int sm = (int)smem;
            const cudaError_t e =
                form == 4   ? cudaFuncSetAttribute(k_u1s_stage<T, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)
                : form == 3 ? cudaFuncSetAttribute(k_u1s_stage<T, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)
                : form == 2 ? cudaFuncSetAttribute(k_u1s_stage<T, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)
                            : cudaFuncSetAttribute(k_u1s_stage<T, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            if (e != cudaSuccess) return e;
            attr[form] = true;
        }
        if (form == 4) k_u1s_stage<T, true, true><<<grid, G::NT, smem, s>>>(A);
        else if (form == 3) k_u1s_stage<T, false, true><<<grid, G::NT, smem, s>>>(A);
        else if (form == 2) k_u1s_stage<T, true, false><<<grid, G::NT, smem, s>>>(A);
        else k_u1s_stage<T, false, false><<<grid, G::NT, smem, s>>>(A);
    }
    return cudaGetLastError();
}

cudaError_t launch_u1_staged(int precision, const void* args, int what, cudaStream_t s)
{
    if (precision == CL_PREC_FP64) return launch_u1s_t(*static_cast<const U1Args<double>*>(args), what, s);
    return launch_u1s_t(*static_cast<const U1Args<float>*>(args), what, s);
}

}  // namespace clk
