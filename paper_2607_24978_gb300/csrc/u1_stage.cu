// Axion coupled to compact U(1) links: one 2N Runge-Kutta stage (section "ALP-gauge
// interactions", Eq. AxionInfEOM, recast in alpha-time and integrated with the
// low-storage Runge-Kutta schemes as that section prescribes).
//
// Lattice fields: the axion phi and its momentum pi = a^(3-alpha) phi' on sites; link
// angles theta_i(n) = dx A_i and electric fields E_i(n) = A_i' on the links n -> n+i.
// The equations are the Euler-Lagrange equations of a lattice Lagrangian whose
// Chern-Simons term is g phi(n) Ebar(n).Bbar(n), Ebar_i(n) = (E_i(n) + E_i(n-i))/2 and
// Bbar_i(n) the average of sin theta_jk / dx^2 over the four (j,k)-plaquettes around n
// ((i,j,k) cyclic), g = alpha_L sqrt(kappa), ws2 = (omega_star/f_star)^2:
//
//   phi' = a^(alpha-3) pi
//   pi'  = a^(1+alpha) Lap phi - a^(3+alpha) V'(phi) + ws2 g Ebar.Bbar
//   theta_i' = dx E_i
//   E_i' = a^(alpha-1) [ -a^(alpha-1) Mag_i + g (C_i - W_i') ] - (1-alpha) (a'/a) E_i
//     Mag_i(n) = sum_{j!=i} [sin theta_ij(n) - sin theta_ij(n-j)] / dx^3
//     C_i(n)   = sum over the four plaquettes P through the link of
//                +-cos theta_P * (sum of phi Ebar_k over the four corners of P) / (4 dx),
//                k the direction normal to P (the link derivative of sum phi Ebar.Bbar)
//     W_i(n)   = (phi(n) Bbar_i(n) + phi(n+i) Bbar_i(n+i)) / 2
//
// Two launches per stage.  k_u1_plaquettes evaluates every plaquette once: for the
// plaquette P_k(n) with normal k (spanned by k1 = k+1, k2 = k+2, lower corner n) it
// stores sin P_k, cos P_k * dP_k/dt and Z_k = cos P_k * (sum of X_k = phi Ebar_k over
// the plaquette's four corners), and reduces the magnetic energy 2 sin^2(P_k / 2)
// (= 1 - cos P_k without cancellation at small angles).  k_u1_stage gathers the forces
// from those fields inside the 3x3x3 neighbourhood of each site (clover averages, the
// magnetic curl, the Chern-Simons sums), performs k <- A k + h F(y), y <- y + B k for
// the eight degrees of freedom of the site, and reduces the other energies of the old
// state (FP64 across threads and blocks, fixed order); its last block advances a, a' and
// their auxiliaries.  k_u1_gauss reduces the lattice Gauss charge
// div-[a^(1-alpha) E + g W] for the diagnostics.
//
// Work decomposition (all three kernels): block b owns a 32 x 8 tile in (x, y) of the
// planes [bz dz, bz dz + dz) (dz chosen by the library); thread (lane, warp) owns column x = 32 bx + lane of row
// y = 8 by + warp and marches up the planes, so most y and z neighbours it gathers were
// loaded by its own block shortly before (L1 hits).  Linear indices fit 32 bits for
// N <= 1536; coordinates and their periodic neighbours are formed once per site.
#include <math.h>

#include "cl_internal.cuh"
#include "kernel_common.cuh"
#include "u1_common.cuh"

namespace clk {

// The tile of this block and this thread's column and row in it.
struct U1Tile {
    uint32_t x, y, z0, z1;
    bool active;
    __device__ __forceinline__ U1Tile(uint32_t N, uint32_t dz)
    {
        const uint32_t ntx = (N + 31) / 32, nty = (N + 7) / 8;
        uint32_t b = blockIdx.x;
        const uint32_t bx = b % ntx;
        b /= ntx;
        const uint32_t by = b % nty, bz = b / nty;
        x = bx * 32 + (threadIdx.x & 31);
        y = by * 8 + (threadIdx.x >> 5);
        z0 = bz * dz;
        z1 = z0 + dz < N ? z0 + dz : N;
        active = x < N && y < N;
    }
};

// A site and its periodic neighbours at offsets -1, 0, +1 along each axis.
struct Nbhd {
    uint32_t N, cx[3], cy[3], cz[3];
    __device__ __forceinline__ Nbhd(uint32_t x, uint32_t y, uint32_t z, uint32_t N_) : N(N_)
    {
        cx[0] = x == 0 ? N_ - 1 : x - 1; cx[1] = x; cx[2] = x + 1 == N_ ? 0 : x + 1;
        cy[0] = y == 0 ? N_ - 1 : y - 1; cy[1] = y; cy[2] = y + 1 == N_ ? 0 : y + 1;
        cz[0] = z == 0 ? N_ - 1 : z - 1; cz[1] = z; cz[2] = z + 1 == N_ ? 0 : z + 1;
    }
    // site at offset o (each component -1, 0 or +1)
    __device__ __forceinline__ uint32_t at(const int (&o)[3]) const
    {
        return (cz[o[2] + 1] * N + cy[o[1] + 1]) * N + cx[o[0] + 1];
    }
};

// Offset vector: sa e_da + sb e_db + sc e_dc (direction indices 0..2, signs -1, 0, +1).
struct Off {
    int o[3];
    __device__ __forceinline__ Off(int da = 0, int sa = 0, int db = 0, int sb = 0, int dc = 0, int sc = 0)
    {
        o[0] = o[1] = o[2] = 0;
        o[da] += sa;
        o[db] += sb;
        o[dc] += sc;
    }
};

template <typename T>
__global__ void __launch_bounds__(256) k_u1_plaquettes(const U1Args<T> A)
{
    __shared__ double s_red[32][kMaxQ];
    const uint32_t N = (uint32_t)A.N;
    const T dx = (T)A.dx;
    Acc<T> accGB;
    const U1Tile tile(N, (uint32_t)A.dz);
    for (uint32_t z = tile.z0; z < tile.z1; ++z) {
        if (!tile.active) break;
        const uint32_t n = (z * N + tile.y) * N + tile.x;
        const Nbhd s(tile.x, tile.y, z, N);
        // every load of the site precedes its stores (outputs may not be assumed disjoint
        // from inputs by the compiler, so an early store would serialise the loads)
        T o_s[3], o_r[3], o_z[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
            const uint32_t n1 = s.at(Off(k1, 1).o), n2 = s.at(Off(k2, 1).o), n12 = s.at(Off(k1, 1, k2, 1).o);
            const T P = A.th_in[k1][n] + A.th_in[k2][n1] - A.th_in[k1][n2] - A.th_in[k2][n];
            const T R = dx * (A.E_in[k1][n] + A.E_in[k2][n1] - A.E_in[k1][n2] - A.E_in[k2][n]);
            T sp, cp;
            if constexpr (sizeof(T) == 4) sincosf(P, &sp, &cp);
            else sincos(P, &sp, &cp);
            // X_k = phi Ebar_k at the four corners; Ebar_k(q) = (E_k(q) + E_k(q - e_k)) / 2
            const uint32_t m0 = s.at(Off(k, -1).o), m1 = s.at(Off(k1, 1, k, -1).o), m2 = s.at(Off(k2, 1, k, -1).o),
                           m12 = s.at(Off(k1, 1, k2, 1, k, -1).o);
            const T q = A.phi_in[n] * (A.E_in[k][n] + A.E_in[k][m0]) + A.phi_in[n1] * (A.E_in[k][n1] + A.E_in[k][m1]) +
                        A.phi_in[n2] * (A.E_in[k][n2] + A.E_in[k][m2]) +
                        A.phi_in[n12] * (A.E_in[k][n12] + A.E_in[k][m12]);
            o_s[k] = sp;
            o_r[k] = cp * R;
            o_z[k] = cp * ((T)0.5 * q);
            const T sh = sin((T)0.5 * P);
            accGB.add((T)2 * sh * sh);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            A.sP[k][n] = o_s[k];
            A.rP[k][n] = o_r[k];
            A.Z[k][n] = o_z[k];
        }
    }
    double v[1] = {accGB.value()};
    block_reduce<1>(v, s_red, threadIdx.x, blockDim.x);
    if (threadIdx.x == 0) A.partials[(size_t)gridDim.x * kMaxQ + blockIdx.x] = v[0];
}

// Clover sum of f_k over the four plaquettes with normal k around site q (offset oq).
template <typename T>
__device__ __forceinline__ T clover(const T* const f, const Nbhd& s, const Off& oq, int k)
{
    const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
    Off b = oq, c = oq;
    b.o[k1] -= 1;
    c.o[k2] -= 1;
    Off d = b;
    d.o[k2] -= 1;
    return (f[s.at(oq.o)] + f[s.at(b.o)]) + (f[s.at(c.o)] + f[s.at(d.o)]);
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) k_u1_stage(const U1Args<T> A)
{
    __shared__ double s_coef[7];
    __shared__ double s_red[32][kMaxQ];
    __shared__ int s_last;
    const uint32_t N = (uint32_t)A.N, V = N * N * N;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const bool first = (A.flags & P_FIRST_STAGE) != 0;
    const bool update = (A.flags & P_ENERGY_ONLY) == 0;
    const bool expand = (A.flags & P_EXPANSION) != 0;
    if (tid == 0) {
        const double a = A.scal->a, b = expand ? A.scal->b : 0.0;
        s_coef[0] = apow(a, A.alpha - 3.0);                     // phi' = c0 pi
        s_coef[1] = apow(a, 1.0 + A.alpha) / (A.dx * A.dx);      // Laplacian
        s_coef[2] = apow(a, 3.0 + A.alpha);                     // potential
        s_coef[3] = apow(a, A.alpha - 1.0);                     // E' prefactor
        s_coef[4] = (1.0 - A.alpha) * b / a;                   // electric friction
        s_coef[5] = a;
        s_coef[6] = A.lf == 3 ? u1_lf_drift(a, b, A.h, A.alpha) : 0.0;  // leapfrog drift of phi
    }
    __syncthreads();
    const T c_dphi = (T)s_coef[0], cL = (T)s_coef[1], cV = (T)s_coef[2], cE = (T)s_coef[3], cfr = (T)s_coef[4];
    const int lf = A.lf;
    const T le = (T)A.le, lk = (T)A.lk, cdrift = (T)s_coef[6], hdx = (T)(A.h * A.dx);
    const T g = (T)A.g, ws2 = (T)A.ws2, dx = (T)A.dx, m2 = (T)A.m2, lam = (T)A.lam;
    const T inv_dx3 = (T)(1.0 / (A.dx * A.dx * A.dx)), inv4dx = (T)(0.25 / A.dx), inv4dx2 = (T)(0.25 / (A.dx * A.dx));
    const T h = (T)A.h, cA = (T)A.A, cB = (T)A.B;
    Acc<T> accK, accG, accV, accKE;

    const U1Tile tile(N, (uint32_t)A.dz);
    for (uint32_t z = tile.z0; z < tile.z1; ++z) {
        if (!tile.active) break;
        const uint32_t n = (z * N + tile.y) * N + tile.x;
        const Nbhd s(tile.x, tile.y, z, N);
        const T ph = A.phi_in[n], pv = A.pi_in[n];
        // scalar sector
        const T pxp = A.phi_in[s.at(Off(0, 1).o)], pxm = A.phi_in[s.at(Off(0, -1).o)];
        const T pyp = A.phi_in[s.at(Off(1, 1).o)], pym = A.phi_in[s.at(Off(1, -1).o)];
        const T pzp = A.phi_in[s.at(Off(2, 1).o)], pzm = A.phi_in[s.at(Off(2, -1).o)];
        const T lap = ((pxp + pxm) + (pyp + pym) + (pzp + pzm)) - (T)6 * ph;
        const T dV = ph * (m2 + lam * ph * ph);
        T eb = (T)0, e2 = (T)0;
        T Ecur[3], Bn[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            Ecur[k] = A.E_in[k][n];
            Bn[k] = inv4dx2 * clover(A.sP[k], s, Off(), k);
            eb += (T)0.5 * (Ecur[k] + A.E_in[k][s.at(Off(k, -1).o)]) * Bn[k];
            e2 += Ecur[k] * Ecur[k];
        }
        const T F_phi = c_dphi * pv;
        const T F_pi = cL * lap - cV * dV + ws2 * g * eb;
        if (lf == 0) {  // (leapfrog pass 1 sums the kinetic energies of its output momenta)
            accK.add(pv * pv);
            accKE.add(e2);
        }
        accG.add((pxp - ph) * (pxp - ph) + (pyp - ph) * (pyp - ph) + (pzp - ph) * (pzp - ph));
        accV.add(ph * ph * ((T)0.5 * m2 + (T)0.25 * lam * ph * ph));
        if (!update) continue;

        // link forces
        T F_E[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int ip = (i + 1) % 3, im = (i + 2) % 3;
            // magnetic: sum_{j != i} sin theta_ij(n) - sin theta_ij(n - j); theta_{i,ip} has normal im,
            // theta_{im,i} normal ip
            const T mag = (A.sP[im][n] - A.sP[im][s.at(Off(ip, -1).o)]) - (A.sP[ip][n] - A.sP[ip][s.at(Off(im, -1).o)]);
            // Chern-Simons: the four plaquettes through the link
            const T cs = (A.Z[im][n] - A.Z[im][s.at(Off(ip, -1).o)]) + (A.Z[ip][s.at(Off(im, -1).o)] - A.Z[ip][n]);
            // W_i' from the clover fields at n and n + i
            const Off oi(i, 1);
            const uint32_t ni = s.at(oi.o);
            const T Bdn = inv4dx2 * clover(A.rP[i], s, Off(), i);
            const T Bni = inv4dx2 * clover(A.sP[i], s, oi, i);
            const T Bdni = inv4dx2 * clover(A.rP[i], s, oi, i);
            const T wdot = (T)0.5 * (F_phi * Bn[i] + ph * Bdn + c_dphi * A.pi_in[ni] * Bni + A.phi_in[ni] * Bdni);
            F_E[i] = cE * (-cE * mag * inv_dx3 + g * (cs * inv4dx - wdot)) - cfr * Ecur[i];
        }
        if (lf == 1) {  // leapfrog: closing half-kick (integer-time momenta) and the first iterate
            const T pn = pv + le * F_pi;
            const T po = pv + lk * F_pi;
            T En[3], Eo[3], en2 = (T)0;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                En[i] = Ecur[i] + le * F_E[i];
                Eo[i] = Ecur[i] + lk * F_E[i];
                en2 += En[i] * En[i];
            }
            accK.add(pn * pn);
            accKE.add(en2);
            A.k_out[1][n] = pn;
            A.pi_out[n] = po;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                A.k_out[5 + i][n] = En[i];
                A.E_out[i][n] = Eo[i];
            }
            continue;
        }
        if (lf != 0) {  // leapfrog: an iterate of the implicit kick from the base momenta
            const T po = A.k_in[1][n] + lk * F_pi;
            T Eo[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) Eo[i] = A.k_in[5 + i][n] + lk * F_E[i];
            if (lf == 3) {
                const T th[3] = {A.th_in[0][n], A.th_in[1][n], A.th_in[2][n]};
                A.phi_out[n] = ph + cdrift * po;
#pragma unroll
                for (int i = 0; i < 3; ++i) A.th_out[i][n] = th[i] + hdx * Eo[i];
            }
            A.pi_out[n] = po;
#pragma unroll
            for (int i = 0; i < 3; ++i) A.E_out[i][n] = Eo[i];
            continue;
        }
        // 2N Runge-Kutta update of the eight degrees of freedom of this site (all loads
        // first, then the stores)
        const T F[8] = {F_phi, F_pi, dx * Ecur[0], dx * Ecur[1], dx * Ecur[2], F_E[0], F_E[1], F_E[2]};
        const T y[8] = {ph, pv, A.th_in[0][n], A.th_in[1][n], A.th_in[2][n], Ecur[0], Ecur[1], Ecur[2]};
        T kq[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) kq[q] = first ? h * F[q] : cA * A.k_in[q][n] + h * F[q];
        T* out[8] = {A.phi_out, A.pi_out, A.th_out[0], A.th_out[1], A.th_out[2], A.E_out[0], A.E_out[1], A.E_out[2]};
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            A.k_out[q][n] = kq[q];
            out[q][n] = y[q] + cB * kq[q];
        }
    }

    // ---- block partials; last block: energies of the old state and the (a, a') stage ----
    double v[kMaxQ] = {accK.value(), accG.value(), accV.value(), accKE.value(), 0.0};
    block_reduce<kMaxQ>(v, s_red, tid, nthr);
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
    for (int b = tid; b < (int)gridDim.x; b += nthr) {
#pragma unroll
        for (int q = 0; q < kMaxQ - 1; ++q) w[q] += __ldcg(&A.partials[(size_t)b * kMaxQ + q]);
        w[kMaxQ - 1] += __ldcg(&A.partials[(size_t)gridDim.x * kMaxQ + b]);  // plaquette launch, same grid
    }
    block_reduce<kMaxQ>(w, s_red, tid, nthr);
    if (tid == 0) {
        if (lf) u1_lf_epilogue(A, w, s_coef[5], expand, V);
        else u1_epilogue(A, w, s_coef[5], first, update, expand, V);
    }
}

// Lattice Gauss charge G(n) = sum_i [P_i(n) - P_i(n - i)] / dx, P = a^(1-alpha) E + g W.
// mode 0 writes diag[D_GV] = max_n |G(n)| / max_n sum_i (|P_i(n)| + |P_i(n - i)|) / dx;
// mode 1 (per-step tracking, for the launch forms whose stage does not sum it itself) the
// rms violation sqrt(sum_n (dx G)^2) / (a^(1-alpha) sqrt(sum_n E^2)) into DevScal::gauss.
template <typename T>
__global__ void __launch_bounds__(256) k_u1_gauss(const U1Args<T> A, int mode)
{
    __shared__ double s_red[32][kMaxQ];
    __shared__ int s_last;
    const uint32_t N = (uint32_t)A.N;
    const int tid = threadIdx.x, nthr = blockDim.x;
    // per-site arithmetic in the field precision (GB300's FP64 rate would make this
    // diagnostic cost a millisecond at 192^3 in double), the maxima and sums in double
    const T ca = (T)apow(A.scal->a, 1.0 - A.alpha);
    const T b4 = (T)(0.25 / (A.dx * A.dx)), gh = (T)(0.5 * A.g);
    double gmax = 0.0, smax = 0.0, gsq = 0.0, e2 = 0.0;
    const U1Tile tile(N, (uint32_t)A.dz);
    for (uint32_t z = tile.z0; z < tile.z1; ++z) {
        if (!tile.active) break;
        const uint32_t n = (z * N + tile.y) * N + tile.x;
        const Nbhd s(tile.x, tile.y, z, N);
        T G = (T)0, sc = (T)0, ee = (T)0;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const Off op(i, 1), om(i, -1);
            const uint32_t np = s.at(op.o), nm = s.at(om.o);
            const T Bn = b4 * clover(A.sP[i], s, Off(), i);
            const T Bp = b4 * clover(A.sP[i], s, op, i);
            const T Bm = b4 * clover(A.sP[i], s, om, i);
            const T Pn = ca * A.E_in[i][n] + gh * (A.phi_in[n] * Bn + A.phi_in[np] * Bp);
            const T Pm = ca * A.E_in[i][nm] + gh * (A.phi_in[nm] * Bm + A.phi_in[n] * Bn);
            G += Pn - Pm;
            sc += fabs(Pn) + fabs(Pm);
            ee += A.E_in[i][n] * A.E_in[i][n];
        }
        gmax = fmax(gmax, fabs((double)G) / A.dx);
        smax = fmax(smax, (double)sc / A.dx);
        gsq += (double)G * (double)G;
        e2 += (double)ee;
    }
    if (mode == 1) {  // sums in a fixed order, then the last block stores the tracked value
        double v[2] = {gsq, e2};
        block_reduce<2>(v, s_red, tid, nthr);
        if (tid == 0) {
            A.partials[(size_t)blockIdx.x * kMaxQ + 0] = v[0];
            A.partials[(size_t)blockIdx.x * kMaxQ + 1] = v[1];
            __threadfence();
            const unsigned prev = atomicAdd(&A.scal->counter, 1u);
            s_last = (prev + 1u == gridDim.x);
        }
        __syncthreads();
        if (!s_last) return;
        __threadfence();
        double w[2] = {0.0, 0.0};
        for (int b = tid; b < (int)gridDim.x; b += nthr) {
            w[0] += __ldcg(&A.partials[(size_t)b * kMaxQ + 0]);
            w[1] += __ldcg(&A.partials[(size_t)b * kMaxQ + 1]);
        }
        block_reduce<2>(w, s_red, tid, nthr);
        if (tid == 0) {
            u1_gauss_track(A.scal, w[0], w[1], ca);
            A.scal->counter = 0u;
        }
        return;
    }
    // block maxima (fixed order), then the last block combines them
    for (int off = 16; off > 0; off >>= 1) {
        gmax = fmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, off));
        smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, off));
    }
    const int warp = tid >> 5, lane = tid & 31, nw = (nthr + 31) >> 5;
    if (lane == 0) {
        s_red[warp][0] = gmax;
        s_red[warp][1] = smax;
    }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < nw; ++w) {
            gmax = fmax(gmax, s_red[w][0]);
            smax = fmax(smax, s_red[w][1]);
        }
        A.partials[(size_t)blockIdx.x * kMaxQ + 0] = gmax;
        A.partials[(size_t)blockIdx.x * kMaxQ + 1] = smax;
        __threadfence();
        const unsigned prev = atomicAdd(&A.scal->counter, 1u);
        s_last = (prev + 1u == gridDim.x);
    }
    __syncthreads();
    if (!s_last || tid != 0) return;
    __threadfence();
    double G = 0.0, Sc = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) {
        G = fmax(G, __ldcg(&A.partials[(size_t)b * kMaxQ + 0]));
        Sc = fmax(Sc, __ldcg(&A.partials[(size_t)b * kMaxQ + 1]));
    }
    A.scal->diag[D_GV] = Sc > 0.0 ? G / Sc : 0.0;
    A.scal->counter = 0u;
}

// Grid of all three kernels (the stage kernel reads the plaquette kernel's partials by
// block index, so both use this grid).
static int u1_grid(int N, int dz)
{
    return ((N + 31) / 32) * ((N + 7) / 8) * ((N + dz - 1) / dz);
}

template <typename T>
static cudaError_t launch_u1_t(const U1Args<T>& A, int what, cudaStream_t s)
{
    if (A.dz < 1 || A.dz > A.N) return cudaErrorInvalidValue;
    const int grid = u1_grid(A.N, A.dz);
    if (what == 0) k_u1_plaquettes<T><<<grid, 256, 0, s>>>(A);
    else if (what == 1) k_u1_stage<T><<<grid, 256, 0, s>>>(A);
    else k_u1_gauss<T><<<grid, 256, 0, s>>>(A, what == 3 ? 1 : 0);
    return cudaGetLastError();
}

int u1_grid_blocks(int N, int dz) { return u1_grid(N, dz); }

cudaError_t launch_u1(int precision, const void* args, int what, cudaStream_t s)
{
    if (precision == CL_PREC_FP64) return launch_u1_t(*static_cast<const U1Args<double>*>(args), what, s);
    return launch_u1_t(*static_cast<const U1Args<float>*>(args), what, s);
}

}  // namespace clk
