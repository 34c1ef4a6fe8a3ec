// Spectra of the U(1) sector (section "ALP-gauge interactions": the spectra of the two
// chiralities of the gauge field, output separately), outside the time step:
//   electric field E_i; magnetic field B_k(n) = sin P_k(n) / dx^2 (plaquette of normal k at
//   lower corner n); and the + / - chiralities of the gauge potential A_i = theta_i / dx.
// A link field lives at n + e_i / 2: its Fourier amplitude carries exp(-i k_i dx / 2), and
// the forward-difference curl becomes i kt x A^ with the real lattice momentum
// kt_l = (2 / dx) sin(k_l dx / 2).  With kh = kt / |kt| and u, v = kh x u orthonormal and
// transverse to kt, e_s = (u + s i v) / sqrt(2) satisfies i kh x e_s = s e_s, and the
// chirality-s amplitude is conj(e_s) . A^ (its modulus does not depend on u).
//
// The three component fields are transformed with cuFFT (D2Z, half spectrum); the binning
// kernel visits each stored mode and, for 0 < kx < N/2, also its conjugate partner
// (-k, with Nyquist components kept at +N/2), whose chirality power it evaluates from the
// conjugated amplitude and the partner's own lattice momentum: every mode of the full
// spectrum is counted once.  Normalisation as the scalar spectra (vacuum.cu).
#include <math.h>

#include "cl_internal.cuh"

namespace clk {

__device__ __forceinline__ int gs_signed(int i, int N) { return i <= N / 2 ? i : i - N; }

template <typename T>
__global__ void k_gauge_fields(GaugeSpecArgs<T> A, double* __restrict__ out)
{
    const int N = A.N;
    const int64_t V = (int64_t)N * N * N;
    const double inv_dx2 = 1.0 / (A.dx * A.dx), inv_dx = 1.0 / A.dx;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < V; n += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(n % N), y = (int)((n / N) % N), z = (int)(n / ((int64_t)N * N));
        for (int c = 0; c < 3; ++c) {
            double v;
            if (A.which == 0) {
                v = (double)A.E[c][n];
            } else if (A.which == 1) {
                // P_c(n) = theta_c1(n) + theta_c2(n + e_c1) - theta_c1(n + e_c2) - theta_c2(n)
                const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
                int q1[3] = {x, y, z}, q2[3] = {x, y, z};
                q1[c1] = q1[c1] + 1 == N ? 0 : q1[c1] + 1;
                q2[c2] = q2[c2] + 1 == N ? 0 : q2[c2] + 1;
                const int64_t n1 = ((int64_t)q1[2] * N + q1[1]) * N + q1[0];
                const int64_t n2 = ((int64_t)q2[2] * N + q2[1]) * N + q2[0];
                const double P = (double)A.th[c1][n] + (double)A.th[c2][n1] - (double)A.th[c1][n2] - (double)A.th[c2][n];
                v = sin(P) * inv_dx2;
            } else {
                v = (double)A.th[c][n] * inv_dx;
            }
            out[c * V + n] = v;
        }
    }
}

// Power of mode s (signed indices) with component amplitudes f[3]: sum |f_c|^2 (which 0, 1)
// or the chirality power |conj(e_s) . A^|^2 (which 2: +, 3: -).
__device__ double gs_power(int which, const int (&s)[3], const double2 (&f)[3], int N, double dx)
{
    if (which < 2) {
        double p = 0.0;
        for (int c = 0; c < 3; ++c) p += f[c].x * f[c].x + f[c].y * f[c].y;
        return p;
    }
    double kt[3], ar[3], ai[3], nk = 0.0;
    for (int c = 0; c < 3; ++c) {
        const double half = M_PI * s[c] / N;  // k_c dx / 2
        double sh, ch;
        sincos(half, &sh, &ch);
        kt[c] = 2.0 / dx * sh;
        nk += kt[c] * kt[c];
        ar[c] = ch * f[c].x + sh * f[c].y;  // exp(-i half) f
        ai[c] = ch * f[c].y - sh * f[c].x;
    }
    if (nk <= 0.0) return 0.0;
    nk = sqrt(nk);
    const double kh[3] = {kt[0] / nk, kt[1] / nk, kt[2] / nk};
    int a = 0;  // the axis least aligned with kh
    for (int c = 1; c < 3; ++c)
        if (fabs(kh[c]) < fabs(kh[a])) a = c;
    double u[3] = {-kh[a] * kh[0], -kh[a] * kh[1], -kh[a] * kh[2]};
    u[a] += 1.0;
    const double nu = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    for (int c = 0; c < 3; ++c) u[c] /= nu;
    const double v[3] = {kh[1] * u[2] - kh[2] * u[1], kh[2] * u[0] - kh[0] * u[2], kh[0] * u[1] - kh[1] * u[0]};
    const double sg = which == 2 ? 1.0 : -1.0;
    double xr = 0.0, xi = 0.0;
    for (int c = 0; c < 3; ++c) {
        xr += u[c] * ar[c] + sg * v[c] * ai[c];
        xi += u[c] * ai[c] - sg * v[c] * ar[c];
    }
    return 0.5 * (xr * xr + xi * xi);
}

__global__ void k_gauge_bins(const double2* __restrict__ F, int N, double dx, int which, double dn, int nbins,
                             double* S, double* C, int use_smem)
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
        const int s[3] = {i, gs_signed(j, N), gs_signed(k, N)};
        const double nm = sqrt((double)s[0] * s[0] + (double)s[1] * s[1] + (double)s[2] * s[2]);
        const int l = (int)floor(nm / dn + 0.5);
        if (l >= nbins) continue;
        double2 f[3];
        for (int c = 0; c < 3; ++c) f[c] = F[(size_t)c * total + q];
        double p = gs_power(which, s, f, N, dx), w = 1.0;
        if (i != 0 && 2 * i != N) {  // the conjugate partner -k is not stored
            const int sp[3] = {-i, gs_signed((N - j) % N, N), gs_signed((N - k) % N, N)};
            double2 fc[3];
            for (int c = 0; c < 3; ++c) fc[c] = make_double2(f[c].x, -f[c].y);
            p += gs_power(which, sp, fc, N, dx);
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
        for (int l = threadIdx.x; l < nbins; l += blockDim.x) {
            if (sC[l] != 0.0) {
                atomicAdd(&S[l], sS[l]);
                atomicAdd(&C[l], sC[l]);
            }
        }
    }
}

template <typename T>
static cudaError_t launch_gauge_fields_t(const GaugeSpecArgs<T>& A, double* out, cudaStream_t s)
{
    const int64_t V = (int64_t)A.N * A.N * A.N;
    const int blocks = (int)(V < 152 * 8 * 256 ? (V + 255) / 256 : 152 * 8);
    k_gauge_fields<T><<<blocks, 256, 0, s>>>(A, out);
    return cudaGetLastError();
}

cudaError_t launch_gauge_fields(int precision, const void* args, double* out, cudaStream_t s)
{
    if (precision == CL_PREC_FP64) return launch_gauge_fields_t(*static_cast<const GaugeSpecArgs<double>*>(args), out, s);
    return launch_gauge_fields_t(*static_cast<const GaugeSpecArgs<float>*>(args), out, s);
}

cudaError_t launch_gauge_bins(const double2* F, int N, double dx, int which, double dn, int nbins, double* S,
                              double* C, cudaStream_t s)
{
    const int64_t total = (int64_t)N * N * (N / 2 + 1);
    const size_t smem = (size_t)2 * nbins * sizeof(double);
    const int use_smem = smem <= 40 * 1024;
    const int threads = 256;
    const int blocks = (int)((total + threads - 1) / threads < 152 * 8 ? (total + threads - 1) / threads : 152 * 8);
    k_gauge_bins<<<blocks, threads, use_smem ? smem : 0, s>>>(F, N, dx, which, dn, nbins, S, C, use_smem);
    return cudaGetLastError();
}

}  // namespace clk
