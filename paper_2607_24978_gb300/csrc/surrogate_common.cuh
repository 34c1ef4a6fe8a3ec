// Shared declarations of the convolutional surrogate (surrogate_tc.cu, surrogate_cc.cu,
// surrogate_api.cu).  Activations are site-major with channels contiguous (x fastest,
// periodic); weights of a layer are W[27][cout][cin] with tap t = (tz*3 + ty)*3 + tx at
// offset (tx-1, ty-1, tz-1).  Hidden activations are stored as BF16 pre-activations u;
// the consumer of u applies the activation (ReLU or the tanh form of GELU) as it loads.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace clk {

constexpr int kSgTileX = 8, kSgTileY = 16;  // output tile of one tensor-core MMA (M = 128 sites)

enum : int { SG_ACT_NONE = 0, SG_ACT_RELU = 1, SG_ACT_GELU = 2 };

__device__ __forceinline__ float act_f(int act, float u)
{
    if (act == SG_ACT_RELU) return u > 0.f ? u : 0.f;
    if (act == SG_ACT_GELU) {
        const float c = 0.7978845608028654f;  // sqrt(2/pi)
        return 0.5f * u * (1.f + tanhf(c * (u + 0.044715f * u * u * u)));
    }
    return u;
}

__device__ __forceinline__ float act_grad_f(int act, float u)
{
    if (act == SG_ACT_RELU) return u > 0.f ? 1.f : 0.f;
    if (act == SG_ACT_GELU) {
        const float c = 0.7978845608028654f;
        const float th = tanhf(c * (u + 0.044715f * u * u * u));
        return 0.5f * (1.f + th) + 0.5f * u * (1.f - th * th) * c * (1.f + 3.f * 0.044715f * u * u);
    }
    return 1.f;
}

__device__ __forceinline__ void unpack_bf16x8(const uint4 v, float (&f)[8])
{
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 p = __bfloat1622float2(h[i]);
        f[2 * i] = p.x;
        f[2 * i + 1] = p.y;
    }
}

__device__ __forceinline__ uint4 pack_bf16x8(const float (&f)[8])
{
    uint4 v;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&v);
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
    return v;
}

__device__ __forceinline__ uint4 act_bf16x8(int act, const uint4 v)
{
    float f[8];
    unpack_bf16x8(v, f);
#pragma unroll
    for (int i = 0; i < 8; ++i) f[i] = act_f(act, f[i]);
    return pack_bf16x8(f);
}

// Tensor-core convolution layer with CI input and CO output channels (16, 32 or 48;
// thinner layers are zero-padded to 16):
//   out = act_out(conv(act_in(in)) + bias) (+ resid)   (forward)
//   out = conv(in) * act'(gate)                        (data gradient, adjoint weights)
struct ConvTCArgs {
    CUtensorMap in_map;         // when in_tma: BF16 `in` viewed as (8 channels, x, y, channel group, z), so that
    int in_tma;                 //   one box lands a staged plane in the [group][y][x] layout of the MMA operand
    const void* in;             // BF16 [N^3][CI], or FP32 [N^3][in_c] when in_f32 (padded with zeros)
    int in_f32, in_c;
    const __nv_bfloat16* wfmt;  // weights in the tensor-core layout [27][CI/8][CO/8][8][8]
    const float* bias;          // CO values, or nullptr
    const __nv_bfloat16* gate;  // BF16 [N^3][CO] pre-activations whose derivative multiplies out, or nullptr
    void* out;                  // BF16 [N^3][CO], or FP32 [N^3][out_c] (first out_c channels) when out_f32
    int out_f32, out_c;
    const float* resid;         // FP32 residual added to the out_c channels (stride resid_stride), or nullptr
    int resid_stride;
    int* status;                // ST_TIMEOUT on a bounded wait that gave up
    int N;                      // multiple of 16
    int DZ;                     // planes per work unit
    int in_act;                 // activation applied to a BF16 `in` while staging
    int gate_act;               // activation whose derivative gates the output (0: none);
                                // ReLU gates may be post-activation values (h > 0 iff u > 0)
    int out_act;                // activation applied before a BF16 store (forward hidden layers)
    __nv_bfloat16* out_pre;     // BF16 [N^3][CO] pre-activation copy of out (GELU backward), or nullptr
};
size_t conv_tc_smem(int CI, int CO);
cudaError_t launch_conv_tc(int CI, int CO, const ConvTCArgs& A, int grid, cudaStream_t s);
// Encode A.in_map for a BF16 input of CI channels on an N^3 lattice (sets A.in_tma; leaves it
// 0 when the driver's encoder is unavailable or refuses the view).
void conv_tc_encode_input(ConvTCArgs& A, int CI);

// CUDA-core convolution for the thin layers (and the FP32 reference mode): each thread
// computes all cout outputs of one site.
//   out[n][co] = bias[co] + sum_t sum_ci w(t, co, ci) act_in(in[n + o(t)][ci])
//                (+ resid[n][co] for co < resid_c) ; times act'(gate[n][co]) when gate_act
// with w(t, co, ci) = W[t][co][ci], or W[26 - t][ci][co] when flip (the adjoint).
struct ConvCCArgs {
    const void* in;             // float or BF16 by in_bf16
    int in_bf16, in_act;
    int cin, cout;
    const float* w;             // FP32 weights of the layer, [27][cout][cin] (flip: [27][cin][cout])
    int flip;
    const float* bias;          // or nullptr
    const void* gate;           // float or BF16 by gate_bf16, or nullptr
    int gate_bf16, gate_act;
    const float* resid;         // FP32 residual source with resid_stride channels, or nullptr
    int resid_c, resid_stride;
    void* out;                  // float or BF16 by out_bf16
    int out_bf16;
    int N;
};
cudaError_t launch_conv_cc(const ConvCCArgs& A, cudaStream_t s);

// Weight and bias gradients on CUDA cores: dW[t][co][ci] = sum_n g[n][co] act(h[n + o(t)][ci]),
// db[co] = sum_n g[n][co]; per-chunk partials, then a fixed-order reduction (deterministic).
struct ConvDWArgs {
    const void* h;              // layer input (float or BF16 pre-activation)
    int h_bf16, h_act;
    const void* g;              // output gradient (float or BF16)
    int g_bf16;
    int cin, cout, N;
    float* partial;             // [chunks][27 * cout * cin + cout]
    int chunks;
    float* dW;                  // [27][cout][cin]
    float* db;                  // [cout]
};
int conv_dw_chunks(int N);
cudaError_t launch_conv_dw(const ConvDWArgs& A, cudaStream_t s);

// Weight and bias gradients of a layer on the tensor cores (channels padded to CIP, COP =
// 16, 32 or 48; at most one of g and h FP32): dW[t][co][ci] = sum_n g[n][co] h[n + o(t)][ci],
// db[co] = sum_n g[n][co]; block partials, then fixed-order sums (deterministic).
struct ConvDWTCArgs {
    const void* h;              // layer input: BF16 [N^3][CIP] activations, or FP32 [N^3][h_c]
    int h_f32, h_c;
    const void* g;              // output gradient: BF16 [N^3][COP], or FP32 [N^3][g_c]
    int g_f32, g_c;
    int CI, CO;                 // real channels (the padded ones read as zeros)
    int N;                      // multiple of 16
    int nslot;                  // staging slots, 2 .. conv_dw_tc_slots(CIP, N)
    int nb;                     // blocks per tap group (grid nb x 2)
    float* part0;               // [nb][18][COP][CIP]: taps of planes tz = 0, 1
    float* part1;               // [nb][9][COP][CIP]: taps of plane tz = 2
    float* bpart;               // [nb][COP]: bias partials
    float* dW;                  // [27][CO][CI]
    float* db;                  // [CO]
    int* status;                // ST_TIMEOUT on a bounded wait that gave up
};
int conv_dw_tc_slots(int CIP, int N);  // 0: shape not supported on the tensor cores
size_t conv_dw_tc_smem(int CIP, int N, int nslot);
cudaError_t launch_conv_dw_tc(int CIP, int COP, const ConvDWTCArgs& A, cudaStream_t s);

}  // namespace clk
