// Training and application kernels of the convolutional surrogate: the loss and its
// gradient, the AdamW update, the tensor-core weight layout built on the device, channel
// statistics of packed inputs, and the packing of a lattice state into network input and
// back.  Conventions in surrogate_common.cuh.
#include <cuda_bf16.h>
#include <stdint.h>

#include "cl_internal.cuh"
#include "kernel_common.cuh"
#include "surrogate_common.cuh"
#include "surrogate_train.cuh"

namespace clk {

constexpr int kRedThreads = 256;

static int red_grid(int64_t n)
{
    int64_t b = (n + kRedThreads - 1) / kRedThreads;
    return (int)(b < 1 ? 1 : (b > 1024 ? 1024 : b));
}

// ---------------------------------------------------------------- loss
// L = (1 / (n C)) sum_n sum_c ((y[n][c] - t[n * tstride + c]) / scale[c])^2
// g[n][c] = 2 (y - t) / (scale[c]^2 n C); per-block FP64 partials of L.
__global__ void __launch_bounds__(kRedThreads) k_loss(const LossArgs A)
{
    __shared__ double s_red[32][kMaxQ];
    const int64_t total = A.n * A.C;
    const double inv = 1.0 / (double)total;
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t n = i / A.C;
        const int c = (int)(i - n * A.C);
        const float sc = A.scale ? A.scale[c] : 1.f;
        const float d = (A.y[i] - A.t[n * A.tstride + c]) / sc;
        acc += (double)d * d;
        A.g[i] = (float)(2.0 * inv) * d / sc;
    }
    double v[1] = {acc * inv};
    block_reduce<1>(v, s_red, threadIdx.x, blockDim.x);
    if (threadIdx.x == 0) A.partial[blockIdx.x] = v[0];
}

__global__ void k_sum_partials(const double* p, int n, double* out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += p[i];  // fixed order
        *out = s;
    }
}

cudaError_t launch_loss(const LossArgs& A, double* result, cudaStream_t s)
{
    const int g = red_grid(A.n * A.C);
    k_loss<<<g, kRedThreads, 0, s>>>(A);
    k_sum_partials<<<1, 32, 0, s>>>(A.partial, g, result);
    return cudaGetLastError();
}

int loss_partials(int64_t n) { return red_grid(n); }

// ---------------------------------------------------------------- AdamW
__global__ void k_adamw(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                        float* __restrict__ v, int64_t n, AdamArgs A, float decay)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = A.b1 * m[i] + (1.f - A.b1) * gi;
        const float vi = A.b2 * v[i] + (1.f - A.b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float mh = mi * A.c1, vh = vi * A.c2;  // bias corrections 1/(1 - b^t)
        w[i] -= A.lr * (mh / (sqrtf(vh) + A.eps) + decay * w[i]);
    }
}

cudaError_t launch_adamw(float* w, const float* g, float* m, float* v, int64_t n, const AdamArgs& A, bool decay,
                         cudaStream_t s)
{
    k_adamw<<<red_grid(n), kRedThreads, 0, s>>>(w, g, m, v, n, A, decay ? A.wd : 0.f);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- tensor-core layout
// out[t9][ci/8][oz][co/8][co%8][ci%8] (padded to CIp x COp, BF16) from W[t][co][ci] (CO x CI),
// or, adjoint, from Wk[t][a][c] = W[26 - t][c][a] (the layer's output channels become the input).
__global__ void k_format_tc(const float* __restrict__ W, int CO, int CI, int COp, int CIp, int adjoint,
                            __nv_bfloat16* __restrict__ out)
{
    const int KG = CIp / 8, NG = COp / 8;
    const int64_t total = (int64_t)27 * COp * CIp;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = i;
        const int e = (int)(r % 8); r /= 8;
        const int row = (int)(r % 8); r /= 8;
        const int ng = (int)(r % NG); r /= NG;
        const int oz = (int)(r % 3); r /= 3;
        const int kg = (int)(r % KG); r /= KG;
        const int t9 = (int)r;
        const int t = oz * 9 + t9, co = ng * 8 + row, ci = kg * 8 + e;
        float v = 0.f;
        if (!adjoint) {
            if (co < CO && ci < CI) v = W[((int64_t)t * CO + co) * CI + ci];
        } else {  // kernel channels: out = layer input (co < CO here is the layer's cin), in = layer output
            if (co < CO && ci < CI) v = W[((int64_t)(26 - t) * CI + ci) * CO + co];
        }
        out[i] = __float2bfloat16_rn(v);
    }
}

cudaError_t launch_format_tc(const float* W, int CO, int CI, int COp, int CIp, int adjoint, __nv_bfloat16* out,
                             cudaStream_t s)
{
    k_format_tc<<<red_grid((int64_t)27 * COp * CIp), kRedThreads, 0, s>>>(W, CO, CI, COp, CIp, adjoint, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- channel statistics
// FP64 per-block sums of x and x^2 for each channel (C <= 3), then a fixed-order total.
__global__ void __launch_bounds__(kRedThreads) k_channel_sums(const float* x, int64_t n, int C, double* partial)
{
    __shared__ double s_red[32][kMaxQ];
    double v[kMaxQ] = {0, 0, 0, 0, 0};
    double sq[3] = {0, 0, 0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int c = 0; c < C; ++c) {
            const double a = x[i * C + c];
            v[c] += a;
            sq[c] += a * a;
        }
    // channel sums in v[0..2], squares in v[3..4] and a second pass for the third
    double w[kMaxQ] = {v[0], v[1], v[2], sq[0], sq[1]};
    block_reduce<kMaxQ>(w, s_red, threadIdx.x, blockDim.x);
    double w2[1] = {sq[2]};
    block_reduce<1>(w2, s_red, threadIdx.x, blockDim.x);
    if (threadIdx.x == 0) {
        for (int q = 0; q < 5; ++q) partial[blockIdx.x * 6 + q] = w[q];
        partial[blockIdx.x * 6 + 5] = w2[0];
    }
}

__global__ void k_channel_finish(const double* partial, int nb, int64_t n, int C, float* mean, float* stdev)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s[3] = {0, 0, 0}, q[3] = {0, 0, 0};
    for (int b = 0; b < nb; ++b) {  // fixed order
        for (int c = 0; c < 3; ++c) s[c] += partial[b * 6 + c];
        q[0] += partial[b * 6 + 3];
        q[1] += partial[b * 6 + 4];
        q[2] += partial[b * 6 + 5];
    }
    for (int c = 0; c < C; ++c) {
        const double mu = s[c] / (double)n;
        const double var = q[c] / (double)n - mu * mu;
        mean[c] = (float)mu;
        stdev[c] = (float)sqrt(var > 0.0 ? var : 0.0);
    }
}

cudaError_t launch_channel_stats(const float* x, int64_t n, int C, double* partial, float* mean, float* stdev,
                                 cudaStream_t s)
{
    const int g = red_grid(n);
    k_channel_sums<<<g, kRedThreads, 0, s>>>(x, n, C, partial);
    k_channel_finish<<<1, 32, 0, s>>>(partial, g, n, C, mean, stdev);
    return cudaGetLastError();
}

int channel_stats_partials(int64_t n) { return red_grid(n) * 6; }

// ---------------------------------------------------------------- lattice <-> network
// x[n][0] = (phi - mu0)/sg0, x[n][1] = (pi - mu1)/sg1, x[n][2] = (a - mu2)/sg2 (C = 3)
__global__ void k_pack(const float* __restrict__ phi, const float* __restrict__ pi, const double* a_dev, int64_t n,
                       int C, Norm3 nm, float* __restrict__ x)
{
    const float a = a_dev ? (float)*a_dev : 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float* o = x + i * C;
        o[0] = (phi[i] - nm.mu[0]) / nm.sg[0];
        if (C > 1) o[1] = (pi[i] - nm.mu[1]) / nm.sg[1];
        if (C > 2) o[2] = (a - nm.mu[2]) / nm.sg[2];
    }
}

cudaError_t launch_pack(const float* phi, const float* pi, const double* a_dev, int64_t n, int C, const Norm3& nm,
                        float* x, cudaStream_t s)
{
    k_pack<<<red_grid(n), kRedThreads, 0, s>>>(phi, pi, a_dev, n, C, nm, x);
    return cudaGetLastError();
}

// phi = mu0 + sg0 y[n][0], pi = mu1 + sg1 y[n][1]; the Kahan compensation (if any) restarts at 0
__global__ void k_unpack(const float* __restrict__ y, int64_t n, int ystride, Norm3 nm, float* __restrict__ phi,
                         float* __restrict__ pi, float* __restrict__ c)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        phi[i] = nm.mu[0] + nm.sg[0] * y[i * ystride];
        pi[i] = nm.mu[1] + nm.sg[1] * y[i * ystride + 1];
        if (c) c[i] = 0.f;
    }
}

cudaError_t launch_unpack(const float* y, int64_t n, int ystride, const Norm3& nm, float* phi, float* pi, float* c,
                          cudaStream_t s)
{
    k_unpack<<<red_grid(n), kRedThreads, 0, s>>>(y, n, ystride, nm, phi, pi, c);
    return cudaGetLastError();
}

}  // namespace clk
