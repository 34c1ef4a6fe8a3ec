// Gravitational waves with five traceless auxiliary fields (section "New algorithm for
// GWs"): v = {v11, v12, v13, v22, v23} (v33 = -v11 - v22) and pi_v = a^(3-alpha) v', with
//   v' = a^(alpha-3) pi_v,   pi_v' = a^(1+alpha) Lap v + 2 kappa a^(1+alpha) [Pi_ij - delta_ij Pi / 3],
//   Pi_ij = sum_f dbar_i phi_f dbar_j phi_f  (central differences),
// evolved by the leapfrog alongside the scalars.  One GW pass runs after each fused scalar
// pass with the same coefficients (d, k): it reads the scalars that pass drifted (its output)
// for the source, drifts v, and kicks pi_v, with the pass's prefactors formed from a before
// and after the pass (DevScal::a_prev, a) exactly as the scalar pass formed them.  The GW
// fields do not act back on the scalars or on a.
//
// Work decomposition as the Runge-Kutta stage kernel: a block owns BY full x rows and a
// range of planes and marches up z with a three-plane ring of the drifted scalars and v
// (own rows plus one halo row each side) in shared memory.
//
// The energy spectrum of the TT part of h' = a^(alpha-3) pi_v (k_gw_bins): five D2Z
// transforms, h'_33 = -h'_11 - h'_22 by linearity, the projector Lambda(kbar) with
// kbar_i = sin(k_i dx) / dx (the momentum of the central difference), and shell binning over
// the half spectrum with each unstored conjugate partner evaluated from the conjugated
// amplitudes and its own momentum.
#include <math.h>

#include "cl_internal.cuh"
#include "kernel_common.cuh"
#include "scalar_pass_common.cuh"

namespace clk {

constexpr int kGwC = 5;  // stored components

template <typename T, int NF, bool KAHAN, int VW>
__global__ void __launch_bounds__(256) k_gw_pass(const GwPassArgs<T> A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);  // [NF + 5][3][BY+2][N]: drifted phi_f, then v_c
    __shared__ double s_coef[4];
    const int N = A.N, BY = A.BY;
    const int TX = N / VW;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int r = tid < BY * TX ? tid / TX : BY, tx = tid < BY * TX ? tid % TX : 0;
    const int slot_stride = (BY + 2) * N, field_stride = 3 * slot_stride;
    const int x0 = tx * VW;
    const bool do_drift = (A.flags & P_DRIFT) != 0;
    long long u0, u1;
    block_units(N, A.nby, A.DZ, u0, u1);
    if (tid == 0) {
        // the scalar pass's prefactors: a_new = a_old + d a' is what it committed
        const bool expand = (A.flags & P_EXPANSION) != 0;
        const double a_new = A.scal->a, a_old = expand ? A.scal->a_prev : a_new;
        s_coef[0] = A.d * apow(0.5 * (a_old + a_new), A.alpha - 3.0);
        s_coef[1] = apow(a_new, 1.0 + A.alpha) / (A.dx * A.dx);
    }
    __syncthreads();
    const T cd = (T)s_coef[0], cL = (T)s_coef[1];
    const T cS = (T)(2.0 * A.kappa * s_coef[1] * A.dx * A.dx);  // 2 kappa a_new^(1+alpha)
    const T ck = (T)A.k, inv2dx = (T)(0.5 / A.dx);

    int y0 = 0, z0 = 0, R = 1;
    // drifted fields of plane z0 + zrel (own and halo rows) into ring slot `slot`
    auto fill = [&](int zrel, int slot) {
        int zz = z0 + zrel;
        zz = zz < 0 ? zz + N : (zz >= N ? zz - N : zz);
        auto row = [&](int y, int srow, int vx) {
            const size_t g = ((size_t)zz * N + y) * N + vx;
#pragma unroll
            for (int f = 0; f < NF; ++f) {  // already drifted by the scalar pass
                T ph[VW];
                vload<T, VW>(ph, A.phi_in[f] + g);
                vstore<T, VW>(sm + f * field_stride + slot * slot_stride + srow * N + vx, ph);
            }
#pragma unroll
            for (int c = 0; c < kGwC; ++c) {
                T v[VW], pv[VW];
                vload<T, VW>(v, A.v_in[c] + g);
                if (do_drift) {
                    vload<T, VW>(pv, A.pv_in[c] + g);
#pragma unroll
                    for (int i = 0; i < VW; ++i) v[i] = fma_rn(cd, pv[i], v[i]);
                }
                vstore<T, VW>(sm + (NF + c) * field_stride + slot * slot_stride + srow * N + vx, v);
            }
        };
        if (r < R) row(y0 + r, r + 1, x0);
        for (int h = tid; h < 2 * TX; h += nthr) {
            const int sel = h / TX, vx = (h - sel * TX) * VW;
            int y = sel == 0 ? y0 - 1 : y0 + R;
            y = y < 0 ? y + N : (y >= N ? y - N : y);
            row(y, sel == 0 ? 0 : R + 1, vx);
        }
    };

    // the own rows of plane z0 + zrel into L2 (one 128-byte line per lane that starts one), so
    // that the fill one plane later waits on L2 rather than DRAM; the halo rows are other
    // tiles' own rows
    auto prefetch_plane = [&](int zrel) {
        if (r >= R || ((x0 * (int)sizeof(T)) & 127) != 0) return;
        int zz = z0 + zrel;
        zz = zz < 0 ? zz + N : (zz >= N ? zz - N : zz);
        const size_t g = ((size_t)zz * N + (y0 + r)) * N + x0;
#pragma unroll
        for (int f = 0; f < NF; ++f) prefetch_l2(A.phi_in[f] + g);
#pragma unroll
        for (int c = 0; c < kGwC; ++c) {
            prefetch_l2(A.v_in[c] + g);
            if (do_drift) prefetch_l2(A.pv_in[c] + g);
        }
    };

    for (long long u = u0; u < u1;) {
        const int tile = (int)(u / N);
        z0 = (int)(u - (long long)tile * N);
        const int NZ = (int)min((long long)(N - z0), u1 - u);
        y0 = tile * BY;
        R = min(BY, N - y0);
        u += NZ;
        fill(-1, 0);
        fill(0, 1);
        for (int zr = 0; zr < NZ; ++zr) {
            const int sl = zr % 3, sc = (zr + 1) % 3, su = (zr + 2) % 3;
            if (zr + 2 <= NZ) prefetch_plane(zr + 2);
            fill(zr + 1, su);
            __syncthreads();
            if (r < R) {
                const size_t base = ((size_t)(z0 + zr) * N + (y0 + r)) * N + x0;
                // central differences of the drifted scalars: Pi_ij summed over the fields
                T Pi[6][VW];  // 00, 01, 02, 11, 12, 22
#pragma unroll
                for (int q = 0; q < 6; ++q)
#pragma unroll
                    for (int i = 0; i < VW; ++i) Pi[q][i] = (T)0;
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    const T* Sc = sm + f * field_stride + sc * slot_stride + (r + 1) * N;
                    const T* Szm = sm + f * field_stride + sl * slot_stride + (r + 1) * N;
                    const T* Szp = sm + f * field_stride + su * slot_stride + (r + 1) * N;
                    T c[VW], ym[VW], yp[VW], zm[VW], zp[VW];
                    vload_smem<T, VW>(c, Sc + x0);
                    vload_smem<T, VW>(ym, Sc - N + x0);
                    vload_smem<T, VW>(yp, Sc + N + x0);
                    vload_smem<T, VW>(zm, Szm + x0);
                    vload_smem<T, VW>(zp, Szp + x0);
                    const T xm_edge = Sc[x0 == 0 ? N - 1 : x0 - 1];
                    const T xp_edge = Sc[x0 + VW == N ? 0 : x0 + VW];
#pragma unroll
                    for (int i = 0; i < VW; ++i) {
                        const T xm = i == 0 ? xm_edge : c[i - 1];
                        const T xp = i == VW - 1 ? xp_edge : c[i + 1];
                        const T d0 = (xp - xm) * inv2dx, d1 = (yp[i] - ym[i]) * inv2dx, d2 = (zp[i] - zm[i]) * inv2dx;
                        Pi[0][i] += d0 * d0;
                        Pi[1][i] += d0 * d1;
                        Pi[2][i] += d0 * d2;
                        Pi[3][i] += d1 * d1;
                        Pi[4][i] += d1 * d2;
                        Pi[5][i] += d2 * d2;
                    }
                }
#pragma unroll
                for (int c = 0; c < kGwC; ++c) {
                    const T* Sc = sm + (NF + c) * field_stride + sc * slot_stride + (r + 1) * N;
                    const T* Szm = sm + (NF + c) * field_stride + sl * slot_stride + (r + 1) * N;
                    const T* Szp = sm + (NF + c) * field_stride + su * slot_stride + (r + 1) * N;
                    T vc[VW], ym[VW], yp[VW], zm[VW], zp[VW], pv[VW], po[VW];
                    vload_smem<T, VW>(vc, Sc + x0);
                    vload_smem<T, VW>(ym, Sc - N + x0);
                    vload_smem<T, VW>(yp, Sc + N + x0);
                    vload_smem<T, VW>(zm, Szm + x0);
                    vload_smem<T, VW>(zp, Szp + x0);
                    vload<T, VW>(pv, A.pv_in[c] + base);
                    const T xm_edge = Sc[x0 == 0 ? N - 1 : x0 - 1];
                    const T xp_edge = Sc[x0 + VW == N ? 0 : x0 + VW];
#pragma unroll
                    for (int i = 0; i < VW; ++i) {
                        const T xm = i == 0 ? xm_edge : vc[i - 1];
                        const T xp = i == VW - 1 ? xp_edge : vc[i + 1];
                        const T lap = ((xp + xm) + (yp[i] + ym[i]) + (zp[i] + zm[i])) - (T)6 * vc[i];
                        const T tr = Pi[0][i] + Pi[3][i] + Pi[5][i];
                        // components 11, 12, 13, 22, 23 of Pi - delta tr / 3
                        const T S = c == 0 ? Pi[0][i] - tr / (T)3
                                  : c == 1 ? Pi[1][i]
                                  : c == 2 ? Pi[2][i]
                                  : c == 3 ? Pi[3][i] - tr / (T)3
                                           : Pi[4][i];
                        po[i] = pv[i] + ck * (cL * lap + cS * S);
                    }
                    vstore<T, VW>(A.v_out[c] + base, vc);
                    vstore<T, VW>(A.pv_out[c] + base, po);
                }
            }
            __syncthreads();
        }
    }
}

template <typename T, int NF, bool KAHAN, int VW>
static cudaError_t launch_gw_t(const GwPassArgs<T>& A, cudaStream_t s)
{
    const size_t smem = (size_t)(NF + kGwC) * 3 * (A.BY + 2) * A.N * sizeof(T);
    static DevFlag attr;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_gw_pass<T, NF, KAHAN, VW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             kPassMaxSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    if (smem > (size_t)kPassMaxSmem) return cudaErrorInvalidValue;
    const int threads = ((A.BY * (A.N / VW) + 31) / 32) * 32;
    k_gw_pass<T, NF, KAHAN, VW><<<A.nby * A.nbz, threads, smem, s>>>(A);
    return cudaGetLastError();
}

template <typename T, int NF, bool KAHAN>
static cudaError_t launch_gw_vw(const GwPassArgs<T>& A, int vw, cudaStream_t s)
{
    if (vw == 1) return launch_gw_t<T, NF, KAHAN, 1>(A, s);
    if (vw == 2) return launch_gw_t<T, NF, KAHAN, 2>(A, s);
    if constexpr (sizeof(T) == 4) {
        if (vw == 4) return launch_gw_t<T, NF, KAHAN, 4>(A, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_gw_pass(int precision, int nf, const void* args, int vw, cudaStream_t s)
{
    if (precision == CL_PREC_FP64) {
        const auto& A = *static_cast<const GwPassArgs<double>*>(args);
        return nf == 1 ? launch_gw_vw<double, 1, false>(A, vw, s) : launch_gw_vw<double, 2, false>(A, vw, s);
    }
    const auto& A = *static_cast<const GwPassArgs<float>*>(args);
    if (precision == CL_PREC_FP32_KAHAN)
        return nf == 1 ? launch_gw_vw<float, 1, true>(A, vw, s) : launch_gw_vw<float, 2, true>(A, vw, s);
    return nf == 1 ? launch_gw_vw<float, 1, false>(A, vw, s) : launch_gw_vw<float, 2, false>(A, vw, s);
}

size_t gw_pass_smem(int nf, int N, int BY, int es) { return (size_t)(nf + kGwC) * 3 * (BY + 2) * N * es; }

// ---------------------------------------------------------------- GW energy spectrum

__device__ __forceinline__ int gw_signed(int i, int N) { return i <= N / 2 ? i : i - N; }

// TT power sum_ij |(Lambda H)_ij|^2 of mode s with the five stored amplitudes h[5]
__device__ double gw_tt_power(const int (&s)[3], const double2 (&h)[5], int N, double dx)
{
    double kb[3], k2 = 0.0;
    for (int c = 0; c < 3; ++c) {
        kb[c] = sin(2.0 * M_PI * s[c] / N) / dx;
        k2 += kb[c] * kb[c];
    }
    if (k2 <= 0.0) return 0.0;
    double P[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) P[i][j] = (i == j ? 1.0 : 0.0) - kb[i] * kb[j] / k2;
    // the symmetric 3 x 3 amplitude with H_33 = -H_11 - H_22
    double2 H[3][3];
    H[0][0] = h[0];
    H[0][1] = H[1][0] = h[1];
    H[0][2] = H[2][0] = h[2];
    H[1][1] = h[3];
    H[1][2] = H[2][1] = h[4];
    H[2][2] = make_double2(-h[0].x - h[3].x, -h[0].y - h[3].y);
    double p = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double tr = 0.0, ti = 0.0;
            for (int l = 0; l < 3; ++l)
                for (int m = 0; m < 3; ++m) {
                    const double L = P[i][l] * P[j][m] - 0.5 * P[i][j] * P[l][m];
                    tr += L * H[l][m].x;
                    ti += L * H[l][m].y;
                }
            p += tr * tr + ti * ti;
        }
    return p;
}

__global__ void k_gw_bins(const double2* __restrict__ F, int N, double dx, double dn, int nbins, double* S, double* C,
                          int use_smem)
{
    extern __shared__ double sh[];
    double* sS = sh;
    double* sC = sh + nbins;
    if (use_smem) {
        for (int l = threadIdx.x; l < 2 * nbins; l += blockDim.x) sh[l] = 0.0;
        __syncthreads();
    }
    const int NH = N / 2 + 1;
    const int64_t total = (int64_t)N * N * NH;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % NH);
        const int j = (int)((q / NH) % N);
        const int k = (int)(q / ((int64_t)NH * N));
        const int s[3] = {i, gw_signed(j, N), gw_signed(k, N)};
        const double nm = sqrt((double)s[0] * s[0] + (double)s[1] * s[1] + (double)s[2] * s[2]);
        const int l = (int)floor(nm / dn + 0.5);
        if (l >= nbins) continue;
        double2 h[5];
        for (int c = 0; c < 5; ++c) h[c] = F[(size_t)c * total + q];
        double p = gw_tt_power(s, h, N, dx), w = 1.0;
        if (i != 0 && 2 * i != N) {  // the unstored conjugate partner -k
            const int sp[3] = {-i, gw_signed((N - j) % N, N), gw_signed((N - k) % N, N)};
            double2 hc[5];
            for (int c = 0; c < 5; ++c) hc[c] = make_double2(h[c].x, -h[c].y);
            p += gw_tt_power(sp, hc, N, dx);
            w = 2.0;
        }
        if (use_smem) {
            atomicAdd(&sS[l], p);
            atomicAdd(&sC[l], w);
        } else {
            atomicAdd(&S[l], p);
            atomicAdd(&C[l], w);
        }
    }
    if (use_smem) {
        __syncthreads();
        for (int l = threadIdx.x; l < nbins; l += blockDim.x)
            if (sC[l] != 0.0) {
                atomicAdd(&S[l], sS[l]);
                atomicAdd(&C[l], sC[l]);
            }
    }
}

cudaError_t launch_gw_bins(const double2* F, int N, double dx, double dn, int nbins, double* S, double* C,
                           cudaStream_t s)
{
    const int64_t total = (int64_t)N * N * (N / 2 + 1);
    const size_t smem = (size_t)2 * nbins * sizeof(double);
    const int use_smem = smem <= 40 * 1024;
    const int threads = 256;
    const int blocks = (int)((total + threads - 1) / threads < 152 * 8 ? (total + threads - 1) / threads : 152 * 8);
    k_gw_bins<<<blocks, threads, use_smem ? smem : 0, s>>>(F, N, dx, dn, nbins, S, C, use_smem);
    return cudaGetLastError();
}

}  // namespace clk
