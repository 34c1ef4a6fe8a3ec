// Vacuum initial conditions and binned spectra (sm_103a).  Not part of the timed step.
//
// Initial conditions (section "Initial conditions", Eq. QuantumFlucts, Eq. fpr_influct,
// Eq. fpr_influct2): for every Fourier mode k (zero mode and |k| > kcut excluded), the
// left- and right-mover amplitudes f_l, f_r are complex Gaussians whose real and
// imaginary parts have variance (N/dx)^3 P(k) / 2 with P = amp2 / (2 a^2 omega_k),
// omega_k = sqrt(k^2 + a^2 m^2).  Then
//     delta f  = (f_l + f_r)/sqrt2,
//     delta f' = a^(alpha-1) i omega_k (f_l - f_r)/sqrt2 - H delta f,
//     delta pi = a^(3-alpha) delta f'.
// The random numbers come from Philox-4x32-10 (Salmon et al., SC'11) keyed by the
// seed with counter (mode index, field, member, 0), four standard normals per mode
// from two Box-Muller pairs.  Of each pair {k, -k} the mode with the smaller linear
// index draws the numbers and its partner is the complex conjugate, so the field is
// real; self-conjugate modes keep the real part.  The kernel fills the half spectrum
// kx in [0, N/2] consumed by cuFFT's complex-to-real transform.
//
// Spectra (section "Arbitrary binning and unbinned spectra", Eq. discretePST2,
// Eq. UpsilonII): real-to-complex transform, then shell binning of |F|^2 with weight
// 2 for the modes whose conjugate partner is not stored in the half spectrum.
#include <math.h>

#include "cl_internal.cuh"

namespace clk {

__device__ __forceinline__ void philox4x32_10(uint32_t (&c)[4], uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
        const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

__device__ __forceinline__ int signed_index(int i, int N) { return i <= N / 2 ? i : i - N; }

__global__ void k_vacuum_modes(const VacuumModeArgs A, double2* __restrict__ fk, double2* __restrict__ pk)
{
    const int N = A.N, NH = N / 2 + 1;
    const int64_t total = (int64_t)N * N * NH;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % NH);
        const int j = (int)((q / NH) % N);
        const int k = (int)(q / ((int64_t)NH * N));
        double2 F = make_double2(0.0, 0.0), P = make_double2(0.0, 0.0);
        const int si = signed_index(i, N), sj = signed_index(j, N), sk = signed_index(k, N);
        const double kIR = 2.0 * M_PI / A.L;
        const double kmod = kIR * sqrt((double)si * si + (double)sj * sj + (double)sk * sk);
        if (!(si == 0 && sj == 0 && sk == 0) && kmod <= A.kcut) {
            const int ci = (N - i) % N, cj = (N - j) % N, ck = (N - k) % N;
            const int64_t idx = ((int64_t)k * N + j) * N + i;
            const int64_t cidx = ((int64_t)ck * N + cj) * N + ci;
            const int64_t draw = idx < cidx ? idx : cidx;
            uint32_t c[4] = {(uint32_t)draw, (uint32_t)A.field, A.member, 0u};
            philox4x32_10(c, (uint32_t)(A.seed & 0xffffffffu), (uint32_t)(A.seed >> 32));
            const double inv32 = 1.0 / 4294967296.0;
            const double u0 = ((double)c[0] + 0.5) * inv32, u1 = ((double)c[1] + 0.5) * inv32;
            const double u2 = ((double)c[2] + 0.5) * inv32, u3 = ((double)c[3] + 0.5) * inv32;
            const double r0 = sqrt(-2.0 * log(u0)), r1 = sqrt(-2.0 * log(u2));
            double s1, c1, s3, c3;
            sincospi(2.0 * u1, &s1, &c1);
            sincospi(2.0 * u3, &s3, &c3);
            const double lr = r0 * c1, li = r0 * s1, rr = r1 * c3, ri = r1 * s3;
            const double dx = A.L / N;
            const double omega = sqrt(kmod * kmod + A.a * A.a * A.m2eff);
            const double Pk = A.amp2 / (2.0 * A.a * A.a * omega);
            const double vol = (double)N / dx;
            const double sigma = sqrt(0.5 * vol * vol * vol * Pk);
            const double isq2 = 0.70710678118654752440;
            F.x = sigma * (lr + rr) * isq2;
            F.y = sigma * (li + ri) * isq2;
            const double cw = pow(A.a, A.alpha - 1.0) * omega * sigma * isq2;
            const double cp = pow(A.a, 3.0 - A.alpha);
            P.x = cp * (-cw * (li - ri) - A.H * F.x);
            P.y = cp * (cw * (lr - rr) - A.H * F.y);
            if (idx == cidx) {
                F.y = 0.0;
                P.y = 0.0;
            } else if (idx != draw) {
                F.y = -F.y;
                P.y = -P.y;
            }
        }
        fk[q] = F;
        pk[q] = P;
    }
}

cudaError_t launch_vacuum_modes(const VacuumModeArgs& a, double2* fk, double2* pk, cudaStream_t s)
{
    const int64_t total = (int64_t)a.N * a.N * (a.N / 2 + 1);
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((total + threads - 1) / threads, 152 * 32);
    k_vacuum_modes<<<blocks, threads, 0, s>>>(a, fk, pk);
    return cudaGetLastError();
}

template <typename T>
__global__ void k_real_to_field(const double* __restrict__ in, T* __restrict__ out, double base, double scale,
                                int64_t n)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        out[q] = (T)(base + scale * in[q]);
}

template <typename T>
__global__ void k_field_to_double(const T* __restrict__ in, double* __restrict__ out, int64_t n)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        out[q] = (double)in[q];
}

template <typename T>
__global__ void k_fill(T* __restrict__ p, int64_t n, T v)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        p[q] = v;
}

static int grid_for(int64_t n, int threads)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, 152 * 32));
}

cudaError_t launch_real_to_field(int precision, const double* in, void* out, double base, double scale, int64_t n,
                                 cudaStream_t s)
{
    if (precision == CL_PREC_FP64)
        k_real_to_field<double><<<grid_for(n, 256), 256, 0, s>>>(in, (double*)out, base, scale, n);
    else
        k_real_to_field<float><<<grid_for(n, 256), 256, 0, s>>>(in, (float*)out, base, scale, n);
    return cudaGetLastError();
}

cudaError_t launch_field_to_double(int precision, const void* in, double* out, int64_t n, cudaStream_t s)
{
    if (precision == CL_PREC_FP64)
        k_field_to_double<double><<<grid_for(n, 256), 256, 0, s>>>((const double*)in, out, n);
    else
        k_field_to_double<float><<<grid_for(n, 256), 256, 0, s>>>((const float*)in, out, n);
    return cudaGetLastError();
}

cudaError_t launch_fill(void* p, int precision, int64_t n, double v, cudaStream_t s)
{
    if (precision == CL_PREC_FP64)
        k_fill<double><<<grid_for(n, 256), 256, 0, s>>>((double*)p, n, v);
    else
        k_fill<float><<<grid_for(n, 256), 256, 0, s>>>((float*)p, n, (float)v);
    return cudaGetLastError();
}

// Shell binning over the half spectrum.  Block-local histograms in shared memory when
// they fit, then one atomic per bin and block.
__global__ void k_spectrum_bins(const double2* __restrict__ F, int N, double dn, int nbins, double* S, double* C,
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
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % NH);
        const int j = (int)((q / NH) % N);
        const int k = (int)(q / ((int64_t)NH * N));
        const int si = i, sj = signed_index(j, N), sk = signed_index(k, N);
        const double nm = sqrt((double)si * si + (double)sj * sj + (double)sk * sk);
        const int l = (int)floor(nm / dn + 0.5);
        if (l >= nbins) continue;
        // modes 0 < i < N/2 stand for themselves and their conjugate partner (-i)
        const double w = (i == 0 || 2 * i == N) ? 1.0 : 2.0;
        const double2 v = F[q];
        const double p = w * (v.x * v.x + v.y * v.y);
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
        for (int l = threadIdx.x; l < nbins; l += blockDim.x) {
            if (sC[l] != 0.0) {
                atomicAdd(&S[l], sS[l]);
                atomicAdd(&C[l], sC[l]);
            }
        }
    }
}

cudaError_t launch_spectrum_bins(const double2* F, int N, double dn, int nbins, double* S, double* C,
                                 cudaStream_t s)
{
    const int64_t total = (int64_t)N * N * (N / 2 + 1);
    const size_t smem = (size_t)2 * nbins * sizeof(double);
    const int use_smem = smem <= 40 * 1024;
    const int threads = 512;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((total + threads - 1) / threads, 152 * 4));
    k_spectrum_bins<<<blocks, threads, use_smem ? smem : 0, s>>>(F, N, dn, nbins, S, C, use_smem);
    return cudaGetLastError();
}

__global__ void k_spectrum_finish(const double* S, const double* C, int N, double L, double dn, int type, int nbins,
                                  double* k_out, double* delta_out)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nbins) return;
    const double nl = l * dn;
    const double N3 = (double)N * N * N;
    const double N6 = N3 * N3;
    k_out[l] = 2.0 * M_PI / L * nl;
    double d = 0.0;
    if (l > 0 && C[l] > 0.0) d = type == 1 ? nl * S[l] / (N6 * dn) : 4.0 * M_PI * nl * nl * nl * (S[l] / C[l]) / N6;
    delta_out[l] = d;
}

cudaError_t launch_spectrum_finish(const double* S, const double* C, int N, double L, double dn, int type,
                                   int nbins, double* k_out, double* delta_out, cudaStream_t s)
{
    k_spectrum_finish<<<(nbins + 127) / 128, 128, 0, s>>>(S, C, N, L, dn, type, nbins, k_out, delta_out);
    return cudaGetLastError();
}

}  // namespace clk
