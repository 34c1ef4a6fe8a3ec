// Launch interfaces of surrogate_train.cu (training and application kernels).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace clk {

struct LossArgs {
    const float* y;       // prediction, n x C
    const float* t;       // target, n rows of tstride values (first C used)
    const float* scale;   // C per-channel scales, or nullptr
    float* g;             // dL/dy, n x C
    double* partial;      // per-block partial losses
    int64_t n;
    int C, tstride;
};
cudaError_t launch_loss(const LossArgs& A, double* result, cudaStream_t s);
int loss_partials(int64_t n);

struct AdamArgs {
    float lr, b1, b2, eps, wd;
    float c1, c2;  // 1 / (1 - b1^t), 1 / (1 - b2^t)
};
cudaError_t launch_adamw(float* w, const float* g, float* m, float* v, int64_t n, const AdamArgs& A, bool decay,
                         cudaStream_t s);
cudaError_t launch_format_tc(const float* W, int CO, int CI, int COp, int CIp, int adjoint, __nv_bfloat16* out,
                             cudaStream_t s);

cudaError_t launch_channel_stats(const float* x, int64_t n, int C, double* partial, float* mean, float* stdev,
                                 cudaStream_t s);
int channel_stats_partials(int64_t n);

struct Norm3 {
    float mu[3], sg[3];
};
cudaError_t launch_pack(const float* phi, const float* pi, const double* a_dev, int64_t n, int C, const Norm3& nm,
                        float* x, cudaStream_t s);
cudaError_t launch_unpack(const float* y, int64_t n, int ystride, const Norm3& nm, float* phi, float* pi, float* c,
                          cudaStream_t s);

}  // namespace clk

// Stream of a surrogate handle (for ordering work of a lattice after the surrogate's).
struct cl_surrogate;
cudaStream_t surrogate_stream(const cl_surrogate* s);
