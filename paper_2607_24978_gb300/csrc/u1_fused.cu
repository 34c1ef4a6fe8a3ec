// Fused axion-U(1) Runge-Kutta stage: the plaquette fields and the stage in one pass (the
// equations, the lattice Chern-Simons discretisation and the 2N-RK update are those of
// u1_stage.cu: section "ALP-gauge interactions", Eq. AxionInfEOM).
//
// The two-launch form writes nine per-site plaquette fields (sin P, cos P dP/dt and
// cos P times the corner sum of phi Ebar, for the three plane orientations) and reads them
// back around every site: 144 bytes of HBM traffic per site beyond the 128 that the stage
// itself has to move, and two latency-bound gathers.  Here a block owns a 32 x 8 tile of
// (x, y) and marches up its planes with
//   * the raw fields phi, pi, theta_i, E_i of the planes z-1, z, z+1 in shared memory with
//     a one-site halo in x and y (a ring of four planes: plane z+2 lands by cp.async while
//     plane z is computed);
//   * the plaquette fields of the two planes each orientation needs (normal x and y: z-1,
//     z; normal z: z, z+1) in a two-plane ring, computed once per plane over the tile and
//     the part of the halo the stage reads: 33 x 9 plaquettes per orientation and plane.
// Every neighbour the stage gathers then comes from shared memory, and the HBM traffic is
// the compulsory one (the eight degrees of freedom and their eight auxiliaries, read and
// written once, plus halo rows that hit L2).  The magnetic energy of a plaquette is counted
// by the block that owns its lower corner.  Sizes must be multiples of the tile (N % 32 == 0);
// other sizes use the two-launch form.
#include <math.h>

#include "cl_internal.cuh"
#include "kernel_common.cuh"
#include "u1_common.cuh"

namespace clk {

// 4- or 8-byte asynchronous copy global -> shared (L1-cached)
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem_dst, const T* gsrc)
{
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "element size");
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(smem_dst)), "l"(gsrc), "n"(sizeof(T))
                 : "memory");
}

constexpr int kFX = 32, kFY = 8;               // tile: one site per thread and plane
constexpr int kFHX = kFX + 2, kFHY = kFY + 2;  // raw planes with a one-site halo
constexpr int kFPX = kFX + 1, kFPY = kFY + 1;  // plaquette planes
constexpr int kFRaw = 8;                       // phi, pi, theta_0..2, E_0..2
constexpr int kFThreads = kFX * kFY;
constexpr int kFRawArr = kFHY * kFHX;           // elements of one raw array of a plane
constexpr int kFRawPlane = kFRaw * kFRawArr;    // elements of one raw plane
constexpr int kFPQ = kFPY * kFPX;               // plaquettes of one orientation and plane
constexpr int kFPQ3 = 3 * kFPQ;                 // sP, rP, Z of one orientation
constexpr int kFLoads = (kFRawPlane + kFThreads - 1) / kFThreads;
enum { FR_PHI = 0, FR_PI = 1, FR_TH = 2, FR_E = 5 };

constexpr int kFSlots = 4;                     // raw plane slots

template <typename T>
struct U1FusedSmem {
    T raw[kFSlots][kFRaw][kFHY][kFHX];  // raw fields, plane slots
    T pq[2][3][3][kFPY][kFPX];    // plaquette fields [ring][normal k][sP, rP, Z][y][x]
};

// Plaquette fields of normal K at the plaquette whose lower corner q is at r0 in its raw
// plane (r1: the same site in the plane above, rm: below): writes sin P, cos P dP/dt and
// cos P * (sum over the corners of phi Ebar_K) / 2 to out[0], out[kFPQ], out[2 kFPQ] and
// returns P.  Every offset is a compile-time constant.
template <typename T, int K>
__device__ __forceinline__ void plaq_site(const T* r0, const T* r1, const T* rm, T dx, T* out, T& P)
{
    constexpr int k1 = (K + 1) % 3, k2 = (K + 2) % 3;
    constexpr int o1 = k1 == 0 ? 1 : (k1 == 1 ? kFHX : 0), p1 = k1 == 2 ? 1 : 0;  // + e_k1
    constexpr int o2 = k2 == 0 ? 1 : (k2 == 1 ? kFHX : 0), p2 = k2 == 2 ? 1 : 0;  // + e_k2
    constexpr int ok = K == 0 ? 1 : (K == 1 ? kFHX : 0), pk = K == 2 ? 1 : 0;      // e_K
    auto V = [&](int arr, int off, int pl) -> T { return (pl == 0 ? r0 : (pl > 0 ? r1 : rm))[arr * kFRawArr + off]; };
    P = V(FR_TH + k1, 0, 0) + V(FR_TH + k2, o1, p1) - V(FR_TH + k1, o2, p2) - V(FR_TH + k2, 0, 0);
    const T R = dx * (V(FR_E + k1, 0, 0) + V(FR_E + k2, o1, p1) - V(FR_E + k1, o2, p2) - V(FR_E + k2, 0, 0));
    T sp, cp;
    if constexpr (sizeof(T) == 4) sincosf(P, &sp, &cp);
    else sincos(P, &sp, &cp);
    // X_K = phi Ebar_K at the four corners; Ebar_K(c) = (E_K(c) + E_K(c - e_K)) / 2
    const T q = V(FR_PHI, 0, 0) * (V(FR_E + K, 0, 0) + V(FR_E + K, -ok, -pk)) +
                V(FR_PHI, o1, p1) * (V(FR_E + K, o1, p1) + V(FR_E + K, o1 - ok, p1 - pk)) +
                V(FR_PHI, o2, p2) * (V(FR_E + K, o2, p2) + V(FR_E + K, o2 - ok, p2 - pk)) +
                V(FR_PHI, o1 + o2, p1 + p2) * (V(FR_E + K, o1 + o2, p1 + p2) + V(FR_E + K, o1 + o2 - ok, p1 + p2 - pk));
    out[0] = sp;
    out[kFPQ] = cp * R;
    out[2 * kFPQ] = cp * ((T)0.5 * q);
}

template <typename T>
__global__ void __launch_bounds__(kFThreads, sizeof(T) == 4 ? 3 : 2) k_u1_fused(const U1Args<T> A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    U1FusedSmem<T>& S = *reinterpret_cast<U1FusedSmem<T>*>(smem_raw);
    __shared__ double s_coef[6];
    __shared__ double s_red[32][kMaxQ];
    __shared__ int s_last;
    const uint32_t N = (uint32_t)A.N, V = N * N * N;
    const int tid = threadIdx.x;
    const int tx = tid % kFX, ty = tid / kFX;
    const bool first = (A.flags & P_FIRST_STAGE) != 0;
    const bool update = (A.flags & P_ENERGY_ONLY) == 0;
    const bool expand = (A.flags & P_EXPANSION) != 0;
    const uint32_t ntx = N / kFX, nty = N / kFY;
    const uint32_t bx = blockIdx.x % ntx, by = (blockIdx.x / ntx) % nty, bz = blockIdx.x / (ntx * nty);
    const uint32_t x0 = bx * kFX, y0 = by * kFY;
    const uint32_t z0 = bz * (uint32_t)A.dz, z1 = min(z0 + (uint32_t)A.dz, N);
    if (tid == 0) {
        const double a = A.scal->a, b = expand ? A.scal->b : 0.0;
        s_coef[0] = apow(a, A.alpha - 3.0);                     // phi' = c0 pi
        s_coef[1] = apow(a, 1.0 + A.alpha) / (A.dx * A.dx);      // Laplacian
        s_coef[2] = apow(a, 3.0 + A.alpha);                     // potential
        s_coef[3] = apow(a, A.alpha - 1.0);                     // E' prefactor
        s_coef[4] = (1.0 - A.alpha) * b / a;                   // electric friction
        s_coef[5] = a;
    }
    const T dx = (T)A.dx;

    // ---- asynchronous copies of raw plane p (periodic) into slot sl: this thread's
    // elements e = tid + i * 256 (one cp.async group per call)
    auto load_plane = [&](uint32_t p, int sl) {
        const uint32_t pz = p % N;
        T* dst = &S.raw[sl][0][0][0];
#pragma unroll
        for (int i = 0; i < kFLoads; ++i) {
            const int e = tid + i * kFThreads;
            if (e < kFRawPlane) {
                const int arr = e / (kFHY * kFHX), r = e - arr * (kFHY * kFHX);
                const int ry = r / kFHX, rx = r - ry * kFHX;
                const uint32_t gx = (x0 + N - 1 + (uint32_t)rx) % N, gy = (y0 + N - 1 + (uint32_t)ry) % N;
                // selected from the kernel parameters (no pointer table in registers)
                const T* base = arr == 0 ? A.phi_in : arr == 1 ? A.pi_in : arr == 2 ? A.th_in[0] : arr == 3 ? A.th_in[1]
                              : arr == 4 ? A.th_in[2] : arr == 5 ? A.E_in[0] : arr == 6 ? A.E_in[1] : A.E_in[2];
                cp_async_elem(dst + e, base + ((size_t)pz * N + gy) * N + gx);
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };

    // ---- plaquette fields: this thread's plaquettes i = tid + 256 j of the 3 x 33 x 9 per
    // plane pair (normal x and y at plane qz01, normal z at plane qz01 + 1).  r01: raw slot of
    // plane qz01, r01p of qz01 + 1 (normal x, y); r2: slot of the normal-z plane, r2m of the
    // plane below it.  count01 / count2: add the owned plaquettes' magnetic energy.
    Acc<T> accGB;
    auto plaquettes = [&](const T* r01, const T* r01p, const T* r2, const T* r2m, T* pqr, bool count01, bool count2) {
#pragma unroll
        for (int j = 0; j < (3 * kFPQ + kFThreads - 1) / kFThreads; ++j) {
            const int i = tid + j * kFThreads;
            if (i >= 3 * kFPQ) break;
            const int k = i >= 2 * kFPQ ? 2 : (i >= kFPQ ? 1 : 0), pos = i - k * kFPQ;
            const int py = pos / kFPX, px = pos - py * kFPX;
            T P;
            bool owned;
            if (k == 0) {
                plaq_site<T, 0>(r01 + py * kFHX + px + 1, r01p + py * kFHX + px + 1, nullptr, dx, pqr + pos, P);
                owned = count01 && px < kFX && py >= 1;
            } else if (k == 1) {
                plaq_site<T, 1>(r01 + (py + 1) * kFHX + px, r01p + (py + 1) * kFHX + px, nullptr, dx,
                                pqr + kFPQ3 + pos, P);
                owned = count01 && px >= 1 && py < kFY;
            } else {
                plaq_site<T, 2>(r2 + py * kFHX + px, nullptr, r2m + py * kFHX + px, dx, pqr + 2 * kFPQ3 + pos, P);
                owned = count2 && px >= 1 && py >= 1;
            }
            if (owned) {  // the plaquette's lower corner lies in the tile
                const T sh = sin((T)0.5 * P);
                accGB.add((T)2 * sh * sh);
            }
        }
    };
    auto raw_slot = [&](int sl) -> const T* { return &S.raw[sl][0][0][0]; };

    // ---- prologue: raw planes z0-1, z0, z0+1 in slots 0, 1, 2; plaquettes of normal x, y at
    // plane z0-1 and of normal z at plane z0 in ring slot 1
    for (int j = 0; j < 3; ++j) load_plane(z0 + N - 1 + (uint32_t)j, j);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    // normal x, y at plane z0-1 (slot 0, plane + 1 in slot 1), normal z at plane z0 (slot 1,
    // plane - 1 in slot 0), into ring slot 1
    plaquettes(raw_slot(0), raw_slot(1), raw_slot(1), raw_slot(0), &S.pq[1][0][0][0][0], false, true);
    const T c_dphi = (T)s_coef[0], cL = (T)s_coef[1], cV = (T)s_coef[2], cE = (T)s_coef[3], cfr = (T)s_coef[4];
    const T g = (T)A.g, ws2 = (T)A.ws2, m2 = (T)A.m2, lam = (T)A.lam;
    const T inv_dx3 = (T)(1.0 / (A.dx * A.dx * A.dx)), inv4dx = (T)(0.25 / A.dx), inv4dx2 = (T)(0.25 / (A.dx * A.dx));
    const T h = (T)A.h, cA = (T)A.A, cB = (T)A.B;
    Acc<T> accK, accG, accV, accKE;

    const uint32_t nz = z1 - z0;
    for (uint32_t s = 0; s < nz; ++s) {
        const uint32_t z = z0 + s;
        // slots of planes z-1, z, z+1 (plane z0 - 1 + j in slot j mod 4)
        const int sm = (int)(s % kFSlots), s0 = (int)((s + 1) % kFSlots), sp = (int)((s + 2) % kFSlots);
        const int cur = (int)(s & 1), prev = cur ^ 1;
        // plane z+2 lands in the slot of plane z-2 (read last in the previous step)
        const bool more = s + 1 < nz;
        if (more) load_plane(z + 2, (int)((s + 3) % kFSlots));
        // plaquettes of normal x, y at plane z and of normal z at plane z+1 (counted below z1)
        plaquettes(raw_slot(s0), raw_slot(sp), raw_slot(sp), raw_slot(s0), &S.pq[cur][0][0][0][0], true, s + 1 < nz);
        __syncthreads();

        // ---- the stage at site (x0 + tx, y0 + ty, z) ----
        // this thread's site in the raw planes z-1, z, z+1 and the plaquette ring slots; every
        // neighbour below is a constant offset from these
        const T* rm = &S.raw[sm][0][ty + 1][tx + 1];
        const T* r0 = &S.raw[s0][0][ty + 1][tx + 1];
        const T* rp = &S.raw[sp][0][ty + 1][tx + 1];
        const T* pc = &S.pq[cur][0][0][ty][tx];
        const T* pv_ = &S.pq[prev][0][0][ty][tx];
        auto RW = [&](int arr, int d0, int d1, int d2) -> T {
            return (d2 == 0 ? r0 : (d2 > 0 ? rp : rm))[arr * kFRawArr + d1 * kFHX + d0];
        };
        // plaquette field f of normal k at the site offset by (d0, d1, d2)
        auto PQ = [&](int k, int f, int d0, int d1, int d2) -> T {
            const bool c = k < 2 ? d2 == 0 : d2 == 1;
            return (c ? pc : pv_)[k * kFPQ3 + f * kFPQ + (d1 + (k == 1 ? 0 : 1)) * kFPX + d0 + (k == 0 ? 0 : 1)];
        };
        auto dir = [](int d, int& d0, int& d1, int& d2, int sgn) {
            d0 += sgn * (d == 0);
            d1 += sgn * (d == 1);
            d2 += sgn * (d == 2);
        };
        // clover sum of field f of normal k around the site offset by o
        auto clover = [&](int k, int f, int o0, int o1, int o2) -> T {
            const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
            int b0 = o0, b1 = o1, b2 = o2, c0 = o0, c1 = o1, c2 = o2;
            dir(k1, b0, b1, b2, -1);
            dir(k2, c0, c1, c2, -1);
            int e0 = b0, e1 = b1, e2 = b2;
            dir(k2, e0, e1, e2, -1);
            return (PQ(k, f, o0, o1, o2) + PQ(k, f, b0, b1, b2)) + (PQ(k, f, c0, c1, c2) + PQ(k, f, e0, e1, e2));
        };
        const T ph = RW(FR_PHI, 0, 0, 0), pv = RW(FR_PI, 0, 0, 0);
        const T pxp = RW(FR_PHI, 1, 0, 0), pxm = RW(FR_PHI, -1, 0, 0);
        const T pyp = RW(FR_PHI, 0, 1, 0), pym = RW(FR_PHI, 0, -1, 0);
        const T pzp = RW(FR_PHI, 0, 0, 1), pzm = RW(FR_PHI, 0, 0, -1);
        const T lap = ((pxp + pxm) + (pyp + pym)) + (pzp + pzm) - (T)6 * ph;
        const T dV = ph * (m2 + lam * ph * ph);
        T eb = (T)0, e2 = (T)0;
        T Ecur[3], Bn[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            int d0 = 0, d1 = 0, d2 = 0;
            dir(k, d0, d1, d2, -1);
            Ecur[k] = RW(FR_E + k, 0, 0, 0);
            Bn[k] = inv4dx2 * clover(k, 0, 0, 0, 0);
            eb += (T)0.5 * (Ecur[k] + RW(FR_E + k, d0, d1, d2)) * Bn[k];
            e2 += Ecur[k] * Ecur[k];
        }
        const T F_phi = c_dphi * pv;
        const T F_pi = cL * lap - cV * dV + ws2 * g * eb;
        accK.add(pv * pv);
        accG.add((pxp - ph) * (pxp - ph) + (pyp - ph) * (pyp - ph) + (pzp - ph) * (pzp - ph));
        accV.add(ph * ph * ((T)0.5 * m2 + (T)0.25 * lam * ph * ph));
        accKE.add(e2);
        if (update) {
            T F_E[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const int ip = (i + 1) % 3, im = (i + 2) % 3;
                int a0 = 0, a1 = 0, a2 = 0, b0 = 0, b1 = 0, b2 = 0, c0 = 0, c1 = 0, c2 = 0;
                dir(ip, a0, a1, a2, -1);  // -e_ip
                dir(im, b0, b1, b2, -1);  // -e_im
                dir(i, c0, c1, c2, 1);    // +e_i
                const T mag = (PQ(im, 0, 0, 0, 0) - PQ(im, 0, a0, a1, a2)) - (PQ(ip, 0, 0, 0, 0) - PQ(ip, 0, b0, b1, b2));
                const T cs = (PQ(im, 2, 0, 0, 0) - PQ(im, 2, a0, a1, a2)) + (PQ(ip, 2, b0, b1, b2) - PQ(ip, 2, 0, 0, 0));
                const T Bdn = inv4dx2 * clover(i, 1, 0, 0, 0);
                const T Bni = inv4dx2 * clover(i, 0, c0, c1, c2);
                const T Bdni = inv4dx2 * clover(i, 1, c0, c1, c2);
                const T wdot = (T)0.5 * (F_phi * Bn[i] + ph * Bdn + c_dphi * RW(FR_PI, c0, c1, c2) * Bni +
                                         RW(FR_PHI, c0, c1, c2) * Bdni);
                F_E[i] = cE * (-cE * mag * inv_dx3 + g * (cs * inv4dx - wdot)) - cfr * Ecur[i];
            }
            const size_t n = ((size_t)z * N + (y0 + ty)) * N + (x0 + tx);
            // k <- A k + h F(y); y <- y + B k for the eight degrees of freedom of the site
            auto rk = [&](int q, T Fq, T yq, T* yout) {
                const T kq = first ? h * Fq : cA * A.k_in[q][n] + h * Fq;
                A.k_out[q][n] = kq;
                yout[n] = yq + cB * kq;
            };
            rk(0, F_phi, ph, A.phi_out);
            rk(1, F_pi, pv, A.pi_out);
            rk(2, dx * Ecur[0], RW(FR_TH, 0, 0, 0), A.th_out[0]);
            rk(3, dx * Ecur[1], RW(FR_TH + 1, 0, 0, 0), A.th_out[1]);
            rk(4, dx * Ecur[2], RW(FR_TH + 2, 0, 0, 0), A.th_out[2]);
            rk(5, F_E[0], Ecur[0], A.E_out[0]);
            rk(6, F_E[1], Ecur[1], A.E_out[1]);
            rk(7, F_E[2], Ecur[2], A.E_out[2]);
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");  // this thread's copies of plane z+2
        __syncthreads();  // plane z+2 complete; the plaquette slot read as "prev" is free
    }

    // ---- block partials; last block: energies of the old state and the (a, a') stage ----
    double v[kMaxQ] = {accK.value(), accG.value(), accV.value(), accKE.value(), accGB.value()};
    block_reduce<kMaxQ>(v, s_red, tid, kFThreads);
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < kMaxQ; ++q) A.partials[(size_t)blockIdx.x * kMaxQ + q] = v[q];
        __threadfence();
        const unsigned prev = atomicAdd(&A.scal->counter, 1u);
        s_last = (prev + 1u == gridDim.x);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double w[kMaxQ] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = tid; b < (int)gridDim.x; b += kFThreads)
#pragma unroll
        for (int q = 0; q < kMaxQ; ++q) w[q] += __ldcg(&A.partials[(size_t)b * kMaxQ + q]);
    block_reduce<kMaxQ>(w, s_red, tid, kFThreads);
    if (tid == 0) u1_epilogue(A, w, s_coef[5], first, update, expand, V);
}

bool u1_fused_ok(int N) { return N >= kFX && N % kFX == 0 && N % kFY == 0; }

int u1_fused_grid(int N, int dz) { return (N / kFX) * (N / kFY) * ((N + dz - 1) / dz); }

template <typename T>
static cudaError_t u1_fused_attr()
{
    static DevFlag done;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_u1_fused<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(U1FusedSmem<T>));
    if (e == cudaSuccess) done = true;
    return e;
}

cudaError_t u1_fused_blocks_per_sm(int precision, int* blocks)
{
    if (precision == CL_PREC_FP64) {
        cudaError_t e = u1_fused_attr<double>();
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_u1_fused<double>, kFThreads,
                                                             sizeof(U1FusedSmem<double>));
    }
    cudaError_t e = u1_fused_attr<float>();
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_u1_fused<float>, kFThreads,
                                                         sizeof(U1FusedSmem<float>));
}

template <typename T>
static cudaError_t launch_fused_t(const U1Args<T>& A, cudaStream_t s)
{
    if (!u1_fused_ok(A.N) || A.dz < 1 || A.dz > A.N) return cudaErrorInvalidValue;
    cudaError_t e = u1_fused_attr<T>();
    if (e != cudaSuccess) return e;
    k_u1_fused<T><<<u1_fused_grid(A.N, A.dz), kFThreads, sizeof(U1FusedSmem<T>), s>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_u1_fused(int precision, const void* args, cudaStream_t s)
{
    if (precision == CL_PREC_FP64) return launch_fused_t(*static_cast<const U1Args<double>*>(args), s);
    return launch_fused_t(*static_cast<const U1Args<float>*>(args), s);
}

}  // namespace clk
