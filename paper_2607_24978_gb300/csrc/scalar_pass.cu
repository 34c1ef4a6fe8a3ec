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
#include "scalar_pass_common.cuh"

namespace clk {

// Block partials, last-block-done fixed-order reduction and the scalar update (vol: the
// lattice's sites).
template <typename T, int NF>
__device__ __forceinline__ void finish_pass_vol(const ScalarPassArgs<T>& A, Acc<T> (&accK)[NF], Acc<T> (&accG)[NF],
                                                Acc<T>& accV, const double* s_coef, double (*s_red)[kMaxQ],
                                                int* s_last, int tid, int nthr, int timeout, double vol)
{
    double v[kMaxQ];
    if constexpr (sizeof(T) == 4) {  // compensated FP32 sums s - c: the warp stage in float pairs
        const float hi[kMaxQ] = {accK[0].s, NF > 1 ? accK[NF - 1].s : 0.f, accG[0].s, NF > 1 ? accG[NF - 1].s : 0.f,
                                 accV.s};
        const float lo[kMaxQ] = {-accK[0].c, NF > 1 ? -accK[NF - 1].c : 0.f, -accG[0].c,
                                 NF > 1 ? -accG[NF - 1].c : 0.f, -accV.c};
        block_reduce_pairs<kMaxQ>(hi, lo, v, s_red, tid, nthr);
    } else {
        v[0] = accK[0].value();
        v[1] = NF > 1 ? accK[NF - 1].value() : 0.0;
        v[2] = accG[0].value();
        v[3] = NF > 1 ? accG[NF - 1].value() : 0.0;
        v[4] = accV.value();
        block_reduce<kMaxQ>(v, s_red, tid, nthr);
    }
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
    if (tid >= 32) return;  // one warp sums the grid's partials, its lane 0 runs the epilogue
    double w[kMaxQ];
    warp_sum_partials<kMaxQ>(A.partials, (int)gridDim.x, tid, w);
    if (tid == 0)
        scalar_epilogue(A.scal, w, vol, A.dx, s_coef[3], A.alpha, A.kappa, A.d, A.e, A.k, A.flags, A.hubble_limit);
}

// The same for an N^3 lattice.
template <typename T, int NF>
__device__ __forceinline__ void finish_pass(const ScalarPassArgs<T>& A, Acc<T> (&accK)[NF], Acc<T> (&accG)[NF],
                                            Acc<T>& accV, const double* s_coef, double (*s_red)[kMaxQ],
                                            int* s_last, int tid, int nthr, int timeout)
{
    finish_pass_vol<T, NF>(A, accK, accG, accV, s_coef, s_red, s_last, tid, nthr, timeout, (double)A.N * A.N * A.N);
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
    // Flat mapping: thread tid owns one row vector when tid < BY*(N/VW); the block size is
    // rounded up to whole warps, the extra threads only help with halo rows and reductions.
    const int tid = threadIdx.x, nthr = blockDim.x;
    long long u0, u1;
    block_units(N, A.nby, A.DZ, u0, u1);

    // FP64: the summation-by-parts gradient sum (see kick_vector) needs one constant per field
    // that every block takes alike: the drifted field at site 0, computed here by each block
    // with the drift's own operation.
    constexpr bool SBP = sizeof(T) == 8 && !KAHAN;
    __shared__ T s_gC[2];
    if (tid == 0) {
        pass_coefficients(A.scal->a, A.scal->b, A.d, A.alpha, A.dx, (A.flags & P_EXPANSION) != 0, s_coef);
        if (SBP)
            for (int f = 0; f < NF; ++f) {
                T ph = A.phi_in[f][0], c0 = (T)0;
                if (A.flags & P_DRIFT) drift<T, false>(ph, c0, A.pi_in[f][0], (T)s_coef[0]);
                s_gC[f] = ph;
            }
    }
    __syncthreads();
    const TileCoef<T> C{(T)s_coef[0], (T)s_coef[1], (T)s_coef[2], (T)A.e, (T)A.k};
    const bool do_drift = (A.flags & P_DRIFT) != 0;
    const PotCoef<T> P(A.m2, A.lam, A.g2);
    const FieldSet<T> F{{A.phi_in[0], A.phi_in[1]}, {A.pi_in[0], A.pi_in[1]}, {A.c_in[0], A.c_in[1]},
                        {A.phi_out[0], A.phi_out[1]}, {A.pi_out[0], A.pi_out[1]}, {A.c_out[0], A.c_out[1]}};
    Acc<T> accK[NF], accG[NF], accV;
    T gC[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) gC[f] = SBP ? s_gC[f] : (T)0;

    // segments of this block's unit range: one y tile, consecutive z planes
    for (long long u = u0; u < u1;) {
        const int tile = (int)(u / N);
        const int z0 = (int)(u - (long long)tile * N);
        const int NZ = (int)min((long long)(N - z0), u1 - u);
        const int y0 = tile * BY;
        const int R = min(BY, N - y0);
        u += NZ;
        march_tile<T, NF, KAHAN, VW, SBP>(F, N, BY, y0, R, z0, NZ, sm, tid, nthr, do_drift, C, P, accK, accG, accV,
                                          gC);
    }
    finish_pass<T, NF>(A, accK, accG, accV, s_coef, s_red, &s_last, tid, nthr, 0);
}

#include "scalar_pass_tma.cuh"
#include "scalar_pass_tma_nr.cuh"

// ------------------------------------------------------------------ reduced lattices
// The fused pass on a reduced (d+1)-dimensional lattice (section "Scalar dynamics in 1+1 and
// 2+1 dimensions"): N^d sites (d = 1, 2; x fastest), the Laplacian and the gradient energy
// summed over the d directions, everything else as on N^3 sites.  One thread per site,
// grid-stride: the old field is drifted at the site and again at each of its 2d neighbours
// (the same compensated operations as the owning thread), then kicked.
template <typename T, int NF, bool KAHAN>
__global__ void __launch_bounds__(256) k_reduced_pass(const ScalarPassArgs<T> A, int dims)
{
    __shared__ double s_coef[4];
    __shared__ double s_red[32][kMaxQ];
    __shared__ int s_last;
    const int tid = threadIdx.x, nthr = blockDim.x;
    if (tid == 0) pass_coefficients(A.scal->a, A.scal->b, A.d, A.alpha, A.dx, (A.flags & P_EXPANSION) != 0, s_coef);
    __syncthreads();
    const T cd = (T)s_coef[0], cL = (T)s_coef[1], cV = (T)s_coef[2], ce = (T)A.e, ck = (T)A.k;
    const bool do_drift = (A.flags & P_DRIFT) != 0;
    const PotCoef<T> P(A.m2, A.lam, A.g2);
    const long long N = A.N, V = dims == 1 ? N : N * N;
    Acc<T> accK[NF], accG[NF], accV;
    // field f (constant-index selects of the argument arrays) drifted at site m
    auto drifted = [&](int f, long long m, T& cv, T& pv) {
        const T* ph_in = f == 0 ? A.phi_in[0] : A.phi_in[NF - 1];
        const T* pi_in = f == 0 ? A.pi_in[0] : A.pi_in[NF - 1];
        const T* c_in = f == 0 ? A.c_in[0] : A.c_in[NF - 1];
        T ph = ph_in[m];
        pv = pi_in[m];
        cv = KAHAN ? c_in[m] : (T)0;
        if (do_drift) drift<T, KAHAN>(ph, cv, pv, cd);
        return ph;
    };
    for (long long n = blockIdx.x * (long long)nthr + tid; n < V; n += (long long)gridDim.x * nthr) {
        const long long x = n % N, row = n - x;
        const long long xm = row + (x == 0 ? N - 1 : x - 1), xp = row + (x + 1 == N ? 0 : x + 1);
        long long ym = 0, yp = 0;
        if (dims == 2) {
            const long long y = n / N;
            ym = (y == 0 ? N - 1 : y - 1) * N + x;
            yp = (y + 1 == N ? 0 : y + 1) * N + x;
        }
        T phc[NF], lap[NF], pin[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            T cv, pv, c2, p2;
            const T c = drifted(f, n, cv, pv);
            const T xpv = drifted(f, xp, c2, p2), xmv = drifted(f, xm, c2, p2);
            T g = (xpv - c) * (xpv - c);
            if (dims == 2) {
                const T ypv = drifted(f, yp, c2, p2), ymv = drifted(f, ym, c2, p2);
                lap[f] = ((xpv + xmv) + (ypv + ymv)) - (T)4 * c;
                g += (ypv - c) * (ypv - c);
            } else {
                lap[f] = (xpv + xmv) - (T)2 * c;
            }
            accG[f].add(g);
            phc[f] = c;
            pin[f] = pv;
            (f == 0 ? A.phi_out[0] : A.phi_out[NF - 1])[n] = c;
            if (KAHAN) (f == 0 ? A.c_out[0] : A.c_out[NF - 1])[n] = cv;
        }
        const T p0 = phc[0], p1 = NF > 1 ? phc[NF - 1] : (T)0;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            T dV;
            if (f == 0) dV = p0 * (P.m20 + P.l0 * p0 * p0 + (NF > 1 ? P.g2 * p1 * p1 : (T)0));
            else dV = p1 * (P.m21 + P.l1 * p1 * p1 + P.g2 * p0 * p0);
            const T F = cL * lap[f] - cV * dV;
            const T pe = pin[f] + ce * F;
            accK[f].add(pe * pe);
            (f == 0 ? A.pi_out[0] : A.pi_out[NF - 1])[n] = pin[f] + ck * F;
        }
        T v = p0 * p0 * (P.h_m20 + P.q_l0 * p0 * p0);
        if (NF > 1) v += p1 * p1 * (P.h_m21 + P.q_l1 * p1 * p1) + P.h_g2 * p0 * p0 * p1 * p1;
        accV.add(v);
    }
    finish_pass_vol<T, NF>(A, accK, accG, accV, s_coef, s_red, &s_last, tid, nthr, 0, (double)V);
}

// The (2+1)-dimensional pass with row marching (N a multiple of 32 VW): warp w owns a strip of
// 32 VW columns (lane l the VW columns from 32 VW s + VW l, loaded as one 16-byte vector) and
// a chunk of rows [y0, y0 + dy), and marches up its rows keeping the drifted rows y - 1, y,
// y + 1 of every field in registers.  Each input row is loaded and drifted once per strip
// (the two halo rows of a chunk twice, by the neighbouring chunks), with the same compensated
// operations as k_reduced_pass, and its own rows' drifted fields are stored at once; the
// momenta of a row are read again for its kick one row later (L1 hits); the x neighbours of a lane's vector come from its own
// registers, from the neighbouring lanes (shuffles) and, at the strip's ends, from one column
// that the first and the last lane load and drift.  Lattice sums, stores and the epilogue as in
// k_reduced_pass.  Units (strip, chunk) beyond the grid's warps are left to no one: the grid
// is ceil(strips x chunks / 8) blocks of 8 warps.
template <typename T, int NF, bool KAHAN, int VW>
__global__ void __launch_bounds__(256, 3) k_plane_pass(const ScalarPassArgs<T> A, int dy, int pd)
{
    __shared__ double s_coef[4];
    __shared__ double s_red[32][kMaxQ];
    __shared__ int s_last;
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31;
    if (tid == 0) pass_coefficients(A.scal->a, A.scal->b, A.d, A.alpha, A.dx, (A.flags & P_EXPANSION) != 0, s_coef);
    __syncthreads();
    const T cd = (T)s_coef[0], cL = (T)s_coef[1], cV = (T)s_coef[2], ce = (T)A.e, ck = (T)A.k;
    const bool do_drift = (A.flags & P_DRIFT) != 0;
    const PotCoef<T> P(A.m2, A.lam, A.g2);
    const int N = A.N, SW = 32 * VW, nstrips = N / SW, nchunks = (N + dy - 1) / dy;
    const int unit = blockIdx.x * (nthr >> 5) + (tid >> 5);
    Acc<T> accK[NF], accG[NF], accV;
    if (unit < nstrips * nchunks) {  // warp-uniform
        const int strip = unit % nstrips, chunk = unit / nstrips;
        const int xs = strip * SW, x0 = xs + lane * VW;
        const int xe = lane == 0 ? (xs == 0 ? N - 1 : xs - 1) : (xs + SW == N ? 0 : xs + SW);  // edge column
        const bool edge_lane = lane == 0 || lane == 31;
        const int y0 = chunk * dy, y1 = min(y0 + dy, N);
        // row y of field f, drifted: the lane's vector (stored at once, with its compensation,
        // when the row is one of the chunk's own) and, on the edge lanes, the edge column
        auto load_row = [&](int f, int y, bool own, T (&ph)[VW], T& pe) {
            const size_t row = (size_t)y * N;
            const T* ph_in = f == 0 ? A.phi_in[0] : A.phi_in[NF - 1];
            const T* pi_in = f == 0 ? A.pi_in[0] : A.pi_in[NF - 1];
            const T* c_in = f == 0 ? A.c_in[0] : A.c_in[NF - 1];
            T pv[VW], cv[VW];
            vload<T, VW>(ph, ph_in + row + x0);
            vload<T, VW>(pv, pi_in + row + x0);
            if (KAHAN) vload<T, VW>(cv, c_in + row + x0);
            else {
#pragma unroll
                for (int i = 0; i < VW; ++i) cv[i] = (T)0;
            }
            T eph = (T)0, epv = (T)0, ecv = (T)0;
            if (edge_lane) {
                eph = ph_in[row + xe];
                epv = pi_in[row + xe];
                ecv = KAHAN ? c_in[row + xe] : (T)0;
            }
            if (do_drift) {
#pragma unroll
                for (int i = 0; i < VW; ++i) drift<T, KAHAN>(ph[i], cv[i], pv[i], cd);
                drift<T, KAHAN>(eph, ecv, epv, cd);
            }
            pe = eph;
            if (own) {
                vstore<T, VW>((f == 0 ? A.phi_out[0] : A.phi_out[NF - 1]) + row + x0, ph);
                if (KAHAN) vstore<T, VW>((f == 0 ? A.c_out[0] : A.c_out[NF - 1]) + row + x0, cv);
            }
        };
        T prv[NF][VW], cur[NF][VW], cedge[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            T e;
            load_row(f, y0 == 0 ? N - 1 : y0 - 1, false, prv[f], e);
            load_row(f, y0, true, cur[f], cedge[f]);
        }
        for (int y = y0; y < y1; ++y) {
            const int yn = y + 1 == N ? 0 : y + 1;
            if (pd > 0 && (lane & 7) == 0 && y + 1 + pd <= y1) {
                // the row pd ahead into L2 (one 128-byte line a lane of eight), so that its
                // loads wait on L2 rather than DRAM
                int yq = y + 1 + pd;
                yq = yq >= N ? yq - N : yq;
                const size_t off = (size_t)yq * N + x0;
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    prefetch_l2((f == 0 ? A.phi_in[0] : A.phi_in[NF - 1]) + off);
                    prefetch_l2((f == 0 ? A.pi_in[0] : A.pi_in[NF - 1]) + off);
                    if (KAHAN) prefetch_l2((f == 0 ? A.c_in[0] : A.c_in[NF - 1]) + off);
                }
            }
            T nxt[NF][VW], nedge[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) load_row(f, yn, y + 1 < y1, nxt[f], nedge[f]);
            T lap[NF][VW];
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                // x neighbours of the lane's first and last columns
                const T left_l = __shfl_up_sync(0xffffffffu, cur[f][VW - 1], 1);
                const T right_l = __shfl_down_sync(0xffffffffu, cur[f][0], 1);
                const T left = lane == 0 ? cedge[f] : left_l;
                const T right = lane == 31 ? cedge[f] : right_l;
#pragma unroll
                for (int i = 0; i < VW; ++i) {
                    const T c = cur[f][i];
                    const T xm = i > 0 ? cur[f][i - 1] : left;
                    const T xp = i + 1 < VW ? cur[f][i + 1] : right;
                    const T yp = nxt[f][i], ym = prv[f][i];
                    lap[f][i] = ((xp + xm) + (yp + ym)) - (T)4 * c;
                    accG[f].add((xp - c) * (xp - c) + (yp - c) * (yp - c));
                }
            }
            // the kick: pi of row y again (loaded with the row one step earlier, an L1 hit)
            const size_t base = (size_t)y * N + x0;
            T pin[NF][VW];
#pragma unroll
            for (int f = 0; f < NF; ++f) vload<T, VW>(pin[f], (f == 0 ? A.pi_in[0] : A.pi_in[NF - 1]) + base);
#pragma unroll
            for (int i = 0; i < VW; ++i) {
                const T p0 = cur[0][i], p1 = NF > 1 ? cur[NF - 1][i] : (T)0;
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    T dV;
                    if (f == 0) dV = p0 * (P.m20 + P.l0 * p0 * p0 + (NF > 1 ? P.g2 * p1 * p1 : (T)0));
                    else dV = p1 * (P.m21 + P.l1 * p1 * p1 + P.g2 * p0 * p0);
                    const T F = cL * lap[f][i] - cV * dV;
                    const T pe = pin[f][i] + ce * F;
                    accK[f].add(pe * pe);
                    pin[f][i] = pin[f][i] + ck * F;
                }
                T v = p0 * p0 * (P.h_m20 + P.q_l0 * p0 * p0);
                if (NF > 1) v += p1 * p1 * (P.h_m21 + P.q_l1 * p1 * p1) + P.h_g2 * p0 * p0 * p1 * p1;
                accV.add(v);
            }
#pragma unroll
            for (int f = 0; f < NF; ++f) vstore<T, VW>((f == 0 ? A.pi_out[0] : A.pi_out[NF - 1]) + base, pin[f]);
#pragma unroll
            for (int f = 0; f < NF; ++f) {
#pragma unroll
                for (int i = 0; i < VW; ++i) {
                    prv[f][i] = cur[f][i];
                    cur[f][i] = nxt[f][i];
                }
                cedge[f] = nedge[f];
            }
        }
    }
    finish_pass_vol<T, NF>(A, accK, accG, accV, s_coef, s_red, &s_last, tid, nthr, 0, (double)N * N);
}

template <typename T, int NF, bool KAHAN>
static cudaError_t launch_plane_t(const ScalarPassArgs<T>& A, int dy, int pd, int grid, cudaStream_t s)
{
    constexpr int VW = 16 / (int)sizeof(T);
    if (A.N % (32 * VW) != 0 || dy < 1 || pd < 0 || grid < 1) return cudaErrorInvalidValue;
    k_plane_pass<T, NF, KAHAN, VW><<<grid, 256, 0, s>>>(A, dy, pd);
    return cudaGetLastError();
}

bool plane_pass_ok(int precision, int N) { return N % (precision == CL_PREC_FP64 ? 64 : 128) == 0; }

cudaError_t launch_plane_pass(int precision, int nf, const void* args, int dy, int pd, int grid, cudaStream_t s)
{
    if (precision == CL_PREC_FP64) {
        const auto& A = *static_cast<const ScalarPassArgs<double>*>(args);
        return nf == 1 ? launch_plane_t<double, 1, false>(A, dy, pd, grid, s)
                       : launch_plane_t<double, 2, false>(A, dy, pd, grid, s);
    }
    const auto& A = *static_cast<const ScalarPassArgs<float>*>(args);
    if (precision == CL_PREC_FP32_KAHAN)
        return nf == 1 ? launch_plane_t<float, 1, true>(A, dy, pd, grid, s) : launch_plane_t<float, 2, true>(A, dy, pd, grid, s);
    return nf == 1 ? launch_plane_t<float, 1, false>(A, dy, pd, grid, s) : launch_plane_t<float, 2, false>(A, dy, pd, grid, s);
}

template <typename T, int NF, bool KAHAN>
static cudaError_t launch_reduced_t(const ScalarPassArgs<T>& A, int dims, int grid, cudaStream_t s)
{
    k_reduced_pass<T, NF, KAHAN><<<grid, 256, 0, s>>>(A, dims);
    return cudaGetLastError();
}

cudaError_t launch_reduced_pass(int precision, int nf, const void* args, int dims, int grid, cudaStream_t s)
{
    if ((dims != 1 && dims != 2) || grid < 1) return cudaErrorInvalidValue;
    if (precision == CL_PREC_FP64) {
        const auto& A = *static_cast<const ScalarPassArgs<double>*>(args);
        return nf == 1 ? launch_reduced_t<double, 1, false>(A, dims, grid, s) : launch_reduced_t<double, 2, false>(A, dims, grid, s);
    }
    const auto& A = *static_cast<const ScalarPassArgs<float>*>(args);
    if (precision == CL_PREC_FP32_KAHAN)
        return nf == 1 ? launch_reduced_t<float, 1, true>(A, dims, grid, s) : launch_reduced_t<float, 2, true>(A, dims, grid, s);
    return nf == 1 ? launch_reduced_t<float, 1, false>(A, dims, grid, s) : launch_reduced_t<float, 2, false>(A, dims, grid, s);
}

// ------------------------------------------------------------------ launchers
size_t scalar_pass_smem_bytes(int precision, int nf, int N, int BY, int stages, int variant)
{
    const size_t es = precision == CL_PREC_FP64 ? 8 : 4;
    const size_t rows = (size_t)(BY + 2) * N * es;
    if (stages <= 0) return (size_t)nf * 3 * rows;  // direct loader: three-plane ring
    const size_t narr = (size_t)nf * (precision == CL_PREC_FP32_KAHAN ? 3 : 2);
    if (variant == 1) return (size_t)stages * narr * rows;  // ringless: the stage buffers only
    // TMA loader: three-slot ring of drifted fields plus the stage buffers
    return (size_t)nf * 3 * rows + (size_t)stages * narr * rows;
}

template <typename K>
static cudaError_t allow_smem(K kernel)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kPassMaxSmem);
}

// Launch the pass, or (occ != nullptr) report how many blocks of it fit on one SM.
// Ringless TMA kernel (16-byte vectors only), S = 2..5 stages.
template <typename T, int NF, bool KAHAN, int VW>
static cudaError_t launch_nr(const ScalarPassArgs<T>& A, dim3 grid, dim3 block, size_t smem, cudaStream_t s, int* occ)
{
    if constexpr (VW * sizeof(T) == 16) {
        static DevFlag attr[6];
        const int S = A.stages;
        if (S < 2 || S > 5) return cudaErrorInvalidValue;
        cudaError_t e = cudaSuccess;
#define CL_NR_CASE(SS)                                                                                             \
    case SS:                                                                                                       \
        if (!attr[SS]) {                                                                                           \
            e = cudaFuncSetAttribute(k_scalar_pass_tma_nr<T, NF, KAHAN, VW, SS>,                                  \
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, kPassMaxSmem);                    \
            if (e != cudaSuccess) return e;                                                                        \
            attr[SS] = true;                                                                                       \
        }                                                                                                          \
        if (occ)                                                                                                   \
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_scalar_pass_tma_nr<T, NF, KAHAN, VW, SS>, \
                                                                 block.x, smem);                                   \
        k_scalar_pass_tma_nr<T, NF, KAHAN, VW, SS><<<grid, block, smem, s>>>(A);                                  \
        return cudaGetLastError();
        switch (S) {
            CL_NR_CASE(2)
            CL_NR_CASE(3)
            CL_NR_CASE(4)
            CL_NR_CASE(5)
        }
#undef CL_NR_CASE
    }
    return cudaErrorInvalidValue;
}

template <typename T, int NF, bool KAHAN, int VW>
static cudaError_t launch_one(const ScalarPassArgs<T>& A, cudaStream_t s, int* occ)
{
    const int prec = sizeof(T) == 8 ? CL_PREC_FP64 : (KAHAN ? CL_PREC_FP32_KAHAN : CL_PREC_FP32);
    const int TX = A.N / VW;
    dim3 block(((TX * A.BY + 31) / 32) * 32 + (A.stages > 0 ? 32 : 0));  // + producer warp
    dim3 grid(A.DZ > 0 ? A.nby * A.nbz : A.grid);  // DZ < 0: balanced persistent ranges
    const size_t smem = scalar_pass_smem_bytes(prec, NF, A.N, A.BY, A.stages, A.variant);
    if (A.variant == 1 && A.stages > 0) return launch_nr<T, NF, KAHAN, VW>(A, grid, block, smem, s, occ);
    static DevFlag attr_set[8];
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
