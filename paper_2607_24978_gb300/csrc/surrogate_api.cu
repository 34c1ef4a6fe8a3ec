// C ABI of the convolutional surrogate: parameters, activations and gradients on the
// device, and the order of the layer launches (surrogate_tc.cu, surrogate_cc.cu).
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "cl_internal.cuh"
#include "surrogate_common.cuh"
#include "surrogate_train.cuh"

using namespace clk;

struct cl_surrogate {
    cl_surrogate_params p{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int nsm = 152;
    int64_t V = 0;
    std::vector<int> cin, cout;        // per layer
    std::vector<float*> W, b;          // FP32 weights [27][cout][cin] and biases
    std::vector<float*> dW, db;        // their gradients
    std::vector<__nv_bfloat16*> wf;    // tensor-core layout of each layer (forward), BF16 mode
    std::vector<__nv_bfloat16*> wb;    // tensor-core layout of the adjoint (data gradient), layers >= 1
    std::vector<float*> bpad;          // biases zero-padded to the tensor-core output width
    float* x = nullptr;                // last forward input (FP32, N^3 x in)
    float* y = nullptr;                // output (FP32, N^3 x out)
    float* g = nullptr;                // output gradient (FP32)
    float* dx = nullptr;               // input gradient (FP32)
    // outputs of layers 0 .. layers-2: FP32 mode stores the pre-activations u_l; BF16 mode
    // stores the activations h_l = act(u_l) (the next layer's input as is) and, for GELU,
    // the pre-activations in upre (ReLU's derivative follows from h: h > 0 iff u > 0)
    std::vector<void*> u;
    std::vector<void*> upre;
    void* du[2] = {nullptr, nullptr};  // gradient ping-pong (BF16 or FP32)
    float* partial = nullptr;          // weight-gradient partials
    int chunks = 1;
    // tensor-core weight gradients (BF16 mode): blocks per tap group and their partials
    // (weights of the two tap groups, biases)
    int dw_nb = 0;
    float *dw_part0 = nullptr, *dw_part1 = nullptr, *dw_bpart = nullptr;
    int* status = nullptr;
    bool have_forward = false, have_loss = false;
    int64_t launches = 0;
    std::vector<float*> mW, vW, mb, vb;  // AdamW moments
    double* red = nullptr;             // reduction scratch (loss, statistics)
    size_t red_cap = 0;
};

namespace {

bool bf16_mode(const cl_surrogate* s) { return s->p.precision == CL_SG_BF16; }
size_t act_bytes(const cl_surrogate* s) { return bf16_mode(s) ? 2 : 4; }

// Tensor-core width of a channel count: 16, 32 or 48 (thin layers are zero-padded).
int tc_width(int c) { return c <= 16 ? 16 : (c <= 32 ? 32 : 48); }

// Tensor-core layout of weights Wk[t][co][ci] (co < CO, ci < CI real channels), padded to
// CIp x COp, tap t = oz * 9 + t9: [t9][ci/8][oz][co/8][co%8][ci%8], BF16, zeros in the
// padding (one MMA covers the three z taps of an (x, y) tap with N = 3 COp).
void format_tc(const float* Wk, int CO, int CI, int COp, int CIp, std::vector<__nv_bfloat16>& out)
{
    const int KG = CIp / 8, NG = COp / 8;
    out.assign((size_t)27 * COp * CIp, __float2bfloat16(0.f));
    for (int t = 0; t < 27; ++t) {
        const int oz = t / 9, t9 = t % 9;
        for (int co = 0; co < CO; ++co)
            for (int ci = 0; ci < CI; ++ci) {
                const size_t i = (((((size_t)t9 * KG + ci / 8) * 3 + oz) * NG + co / 8) * 8 + co % 8) * 8 + ci % 8;
                out[i] = __float2bfloat16(Wk[((size_t)t * CO + co) * CI + ci]);
            }
    }
}

cl_status check(cudaError_t e) { return e == cudaSuccess ? CL_OK : CL_ECUDA; }

cl_status read_status(cl_surrogate* s)
{
    int st = 0;
    if (cudaMemcpyAsync(&st, s->status, sizeof(int), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return CL_ECUDA;
    if (st) {
        cudaMemsetAsync(s->status, 0, sizeof(int), s->stream);
        if (st & ST_TIMEOUT) return CL_ETIMEOUT;
    }
    return CL_OK;
}

int tc_grid(const cl_surrogate* s, int DZ)
{
    const int N = s->p.N;
    const int units = (N / kSgTileX) * (N / kSgTileY) * ((N + DZ - 1) / DZ);
    return units < s->nsm ? units : s->nsm;
}

constexpr int kTcDZ = 16;

// Convolution of layer l (forward): in -> out with the input activation in_act.
cl_status conv_forward(cl_surrogate* s, int l, const void* in, int in_bf16, int in_act, void* out, int out_bf16,
                       const float* resid, int out_act = 0, void* out_pre = nullptr)
{
    if (bf16_mode(s)) {  // every forward layer on the tensor cores
        ConvTCArgs A{};
        A.in = in;
        A.in_f32 = in_bf16 ? 0 : 1;
        A.in_c = s->cin[l];
        A.wfmt = s->wf[l];
        A.bias = s->bpad[l];
        A.out = out;
        A.out_f32 = out_bf16 ? 0 : 1;
        A.out_c = s->cout[l];
        A.resid = resid;
        A.resid_stride = s->p.in_channels;
        A.status = s->status;
        A.N = s->p.N;
        A.DZ = kTcDZ < s->p.N ? kTcDZ : s->p.N;
        A.in_act = in_act;
        A.out_act = out_act;
        A.out_pre = (__nv_bfloat16*)out_pre;
        conv_tc_encode_input(A, tc_width(s->cin[l]));
        ++s->launches;
        return check(launch_conv_tc(tc_width(s->cin[l]), tc_width(s->cout[l]), A, tc_grid(s, A.DZ), s->stream));
    }
    ConvCCArgs A{};
    A.in = in;
    A.in_bf16 = in_bf16;
    A.in_act = in_act;
    A.cin = s->cin[l];
    A.cout = s->cout[l];
    A.w = s->W[l];
    A.bias = s->b[l];
    A.resid = resid;
    A.resid_c = resid ? s->p.out_channels : 0;
    A.resid_stride = s->p.in_channels;
    A.out = out;
    A.out_bf16 = out_bf16;
    A.N = s->p.N;
    ++s->launches;
    return check(launch_conv_cc(A, s->stream));
}

}  // namespace

extern "C" {

void cl_surrogate_free(cl_surrogate* s)
{
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    for (auto* p : s->W) cudaFree(p);
    for (auto* p : s->b) cudaFree(p);
    for (auto* p : s->dW) cudaFree(p);
    for (auto* p : s->db) cudaFree(p);
    for (auto* p : s->wf) cudaFree(p);
    for (auto* p : s->wb) cudaFree(p);
    for (auto* p : s->bpad) cudaFree(p);
    for (auto* p : s->u) cudaFree(p);
    for (auto* p : s->upre) cudaFree(p);
    cudaFree(s->du[0]);
    cudaFree(s->du[1]);
    cudaFree(s->x);
    cudaFree(s->y);
    cudaFree(s->g);
    cudaFree(s->dx);
    cudaFree(s->partial);
    cudaFree(s->dw_part0);
    cudaFree(s->dw_part1);
    cudaFree(s->dw_bpart);
    cudaFree(s->status);
    for (auto* p : s->mW) cudaFree(p);
    for (auto* p : s->vW) cudaFree(p);
    for (auto* p : s->mb) cudaFree(p);
    for (auto* p : s->vb) cudaFree(p);
    cudaFree(s->red);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
}

cl_status cl_surrogate_create(cl_surrogate** out, const cl_surrogate_params* p)
{
    if (!out) return CL_EINVAL;
    *out = nullptr;
    if (!p || p->reserved != 0 || p->N < 2 || p->N > 512 || p->in_channels < 1 || p->in_channels > 3 ||
        p->out_channels < 1 || p->out_channels > p->in_channels || p->layers < 2 ||
        (p->hidden != 16 && p->hidden != 32 && p->hidden != 48) ||
        (p->activation != CL_ACT_RELU && p->activation != CL_ACT_GELU) ||
        (p->precision != CL_SG_BF16 && p->precision != CL_SG_FP32))
        return CL_EINVAL;
    if (p->precision == CL_SG_BF16 && p->N % 16 != 0) return CL_EINVAL;
    cl_surrogate* s = new (std::nothrow) cl_surrogate();
    if (!s) return CL_ENOMEM;
    s->p = *p;
    s->V = (int64_t)p->N * p->N * p->N;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&s->nsm, cudaDevAttrMultiProcessorCount, dev);
    if (p->stream) {
        s->stream = (cudaStream_t)p->stream;
    } else {
        if (cudaStreamCreate(&s->stream) != cudaSuccess) {
            delete s;
            return CL_ECUDA;
        }
        s->own_stream = true;
    }
    const int L = p->layers;
    bool ok = true;
    for (int l = 0; l < L; ++l) {
        const int ci = l == 0 ? p->in_channels : p->hidden;
        const int co = l == L - 1 ? p->out_channels : p->hidden;
        s->cin.push_back(ci);
        s->cout.push_back(co);
        float *w = nullptr, *bb = nullptr, *gw = nullptr, *gb = nullptr;
        const size_t nw = (size_t)27 * co * ci;
        ok = ok && cudaMalloc(&w, nw * 4) == cudaSuccess && cudaMalloc(&bb, co * 4) == cudaSuccess &&
             cudaMalloc(&gw, nw * 4) == cudaSuccess && cudaMalloc(&gb, co * 4) == cudaSuccess;
        s->W.push_back(w);
        s->b.push_back(bb);
        s->dW.push_back(gw);
        s->db.push_back(gb);
        float *m1 = nullptr, *v1 = nullptr, *m2 = nullptr, *v2 = nullptr;
        ok = ok && cudaMalloc(&m1, nw * 4) == cudaSuccess && cudaMalloc(&v1, nw * 4) == cudaSuccess &&
             cudaMalloc(&m2, co * 4) == cudaSuccess && cudaMalloc(&v2, co * 4) == cudaSuccess &&
             cudaMemset(m1, 0, nw * 4) == cudaSuccess && cudaMemset(v1, 0, nw * 4) == cudaSuccess &&
             cudaMemset(m2, 0, co * 4) == cudaSuccess && cudaMemset(v2, 0, co * 4) == cudaSuccess;
        s->mW.push_back(m1);
        s->vW.push_back(v1);
        s->mb.push_back(m2);
        s->vb.push_back(v2);
        if (ok) {
            cudaMemset(w, 0, nw * 4);
            cudaMemset(bb, 0, co * 4);
        }
        __nv_bfloat16 *f = nullptr, *fb = nullptr;
        float* bp = nullptr;
        if (ok && p->precision == CL_SG_BF16) {
            const size_t np = (size_t)27 * tc_width(co) * tc_width(ci);
            ok = cudaMalloc(&f, np * 2) == cudaSuccess && cudaMemset(f, 0, np * 2) == cudaSuccess &&
                 cudaMalloc(&bp, tc_width(co) * 4) == cudaSuccess && cudaMemset(bp, 0, tc_width(co) * 4) == cudaSuccess;
            if (ok && l > 0)
                ok = cudaMalloc(&fb, np * 2) == cudaSuccess && cudaMemset(fb, 0, np * 2) == cudaSuccess;
        }
        s->wf.push_back(f);
        s->wb.push_back(fb);
        s->bpad.push_back(bp);
        if (l < L - 1) {
            void *uu = nullptr, *up = nullptr;
            ok = ok && cudaMalloc(&uu, (size_t)s->V * p->hidden * act_bytes(s)) == cudaSuccess;
            if (ok && p->precision == CL_SG_BF16 && p->activation == CL_ACT_GELU)
                ok = cudaMalloc(&up, (size_t)s->V * p->hidden * 2) == cudaSuccess;
            s->u.push_back(uu);
            s->upre.push_back(up);
        }
    }
    s->chunks = conv_dw_chunks(p->N);
    const size_t part = (size_t)s->chunks * (27 * (size_t)p->hidden * p->hidden + p->hidden);
    ok = ok && cudaMalloc(&s->du[0], (size_t)s->V * p->hidden * act_bytes(s)) == cudaSuccess &&
         cudaMalloc(&s->du[1], (size_t)s->V * p->hidden * act_bytes(s)) == cudaSuccess &&
         cudaMalloc(&s->x, (size_t)s->V * p->in_channels * 4) == cudaSuccess &&
         cudaMalloc(&s->y, (size_t)s->V * p->out_channels * 4) == cudaSuccess &&
         cudaMalloc(&s->g, (size_t)s->V * p->out_channels * 4) == cudaSuccess &&
         cudaMalloc(&s->dx, (size_t)s->V * p->in_channels * 4) == cudaSuccess &&
         cudaMalloc(&s->partial, part * 4) == cudaSuccess && cudaMalloc(&s->status, sizeof(int)) == cudaSuccess &&
         cudaMemset(s->status, 0, sizeof(int)) == cudaSuccess;
    if (ok && p->precision == CL_SG_BF16 && conv_dw_tc_slots(16, p->N) >= 2) {
        // weight gradients on the tensor cores: about 64 or more rows per block, two tap
        // groups sharing the SMs; partials sized for the widest layer (hidden x hidden)
        const int C = p->hidden;
        const int64_t rows = (int64_t)p->N * p->N;
        int64_t nb = rows / 64;
        nb = nb < 1 ? 1 : (nb > s->nsm / 2 ? s->nsm / 2 : nb);
        s->dw_nb = (int)(nb < 1 ? 1 : nb);
        ok = cudaMalloc(&s->dw_part0, (size_t)s->dw_nb * 18 * C * C * 4) == cudaSuccess &&
             cudaMalloc(&s->dw_part1, (size_t)s->dw_nb * 9 * C * C * 4) == cudaSuccess &&
             cudaMalloc(&s->dw_bpart, (size_t)s->dw_nb * C * 4) == cudaSuccess;
    }
    if (!ok || cudaDeviceSynchronize() != cudaSuccess) {
        cl_surrogate_free(s);
        return CL_ENOMEM;
    }
    *out = s;
    return CL_OK;
}

cl_status cl_surrogate_set_weights(cl_surrogate* s, int32_t layer, const float* W, const float* b)
{
    if (!s || layer < 0 || layer >= (int)s->cin.size() || !W || !b) return CL_EINVAL;
    const int ci = s->cin[layer], co = s->cout[layer];
    const size_t nw = (size_t)27 * co * ci;
    for (size_t i = 0; i < nw; ++i)
        if (!isfinite(W[i])) return CL_EINVAL;
    if (cudaMemcpyAsync(s->W[layer], W, nw * 4, cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
        cudaMemcpyAsync(s->b[layer], b, co * 4, cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
        return CL_ECUDA;
    if (s->wf[layer]) {
        // forward layout (CI -> CO), and the adjoint's (CO -> CI): Wk[t][a][c] = W[26 - t][c][a]
        const int cip = tc_width(ci), cop = tc_width(co);
        std::vector<__nv_bfloat16> f, fb;
        format_tc(W, co, ci, cop, cip, f);
        if (cudaMemcpyAsync(s->wf[layer], f.data(), f.size() * 2, cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
            cudaMemcpyAsync(s->bpad[layer], b, co * 4, cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
            return CL_ECUDA;
        if (s->wb[layer]) {
            std::vector<float> Wa(nw);
            for (int t = 0; t < 27; ++t)
                for (int a = 0; a < ci; ++a)
                    for (int c = 0; c < co; ++c)
                        Wa[((size_t)t * ci + a) * co + c] = W[((size_t)(26 - t) * co + c) * ci + a];
            format_tc(Wa.data(), ci, co, cip, cop, fb);
            if (cudaMemcpyAsync(s->wb[layer], fb.data(), fb.size() * 2, cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
                return CL_ECUDA;
        }
        if (cudaStreamSynchronize(s->stream) != cudaSuccess) return CL_ECUDA;  // host staging vectors go out of scope
    }
    return cudaStreamSynchronize(s->stream) == cudaSuccess ? CL_OK : CL_ECUDA;
}

cl_status cl_surrogate_get_weights(cl_surrogate* s, int32_t layer, float* W, float* b)
{
    if (!s || layer < 0 || layer >= (int)s->cin.size() || !W || !b) return CL_EINVAL;
    const size_t nw = (size_t)27 * s->cout[layer] * s->cin[layer];
    if (cudaMemcpyAsync(W, s->W[layer], nw * 4, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
        cudaMemcpyAsync(b, s->b[layer], s->cout[layer] * 4, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
        return CL_ECUDA;
    return cudaStreamSynchronize(s->stream) == cudaSuccess ? CL_OK : CL_ECUDA;
}

cl_status cl_surrogate_forward(cl_surrogate* s, const float* x, float* y, int32_t on_device)
{
    if (!s || !x || !y) return CL_EINVAL;
    s->launches = 0;
    const size_t nx = (size_t)s->V * s->p.in_channels * 4, ny = (size_t)s->V * s->p.out_channels * 4;
    if (cudaMemcpyAsync(s->x, x, nx, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->stream) !=
        cudaSuccess)
        return CL_ECUDA;
    const int L = (int)s->cin.size(), act = s->p.activation;
    cl_status st = CL_OK;
    if (bf16_mode(s)) {  // stored tensors are activations; GELU also keeps the pre-activations
        st = conv_forward(s, 0, s->x, 0, 0, s->u[0], 1, nullptr, act, s->upre[0]);
        for (int l = 1; st == CL_OK && l < L - 1; ++l)
            st = conv_forward(s, l, s->u[l - 1], 1, 0, s->u[l], 1, nullptr, act, s->upre[l]);
        if (st == CL_OK) st = conv_forward(s, L - 1, s->u[L - 2], 1, 0, s->y, 0, s->x);
    } else {
        st = conv_forward(s, 0, s->x, 0, 0, s->u[0], 0, nullptr);
        for (int l = 1; st == CL_OK && l < L - 1; ++l) st = conv_forward(s, l, s->u[l - 1], 0, act, s->u[l], 0, nullptr);
        if (st == CL_OK) st = conv_forward(s, L - 1, s->u[L - 2], 0, act, s->y, 0, s->x);
    }
    if (st != CL_OK) return st;
    if (cudaMemcpyAsync(y, s->y, ny, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->stream) !=
        cudaSuccess)
        return CL_ECUDA;
    s->have_forward = true;
    if (!on_device) return read_status(s);
    return CL_OK;
}

cl_status cl_surrogate_backward(cl_surrogate* s, const float* g, float* dx, int32_t on_device)
{
    if (!s) return CL_EINVAL;
    if (!s->have_forward || (!g && !s->have_loss)) return CL_ESTATE;
    s->launches = 0;
    const int L = (int)s->cin.size(), act = s->p.activation;
    const int ab = bf16_mode(s) ? 1 : 0;
    const size_t ng = (size_t)s->V * s->p.out_channels * 4;
    if (g && cudaMemcpyAsync(s->g, g, ng, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                             s->stream) != cudaSuccess)
        return CL_ECUDA;
    auto wgrad = [&](int l, const void* h, int h_bf16, int h_act, const void* gg, int g_bf16) {
        // BF16 mode: every layer's weight gradients on the tensor cores (the thin FP32 network
        // input and loss gradient are rounded to BF16 while staged, as in the forward)
        const int cip = tc_width(s->cin[l]), cop = tc_width(s->cout[l]);
        if (s->dw_nb > 0 && !h_act && conv_dw_tc_slots(cip, s->p.N) >= 2) {
            ConvDWTCArgs A{};
            A.h = h;
            A.h_f32 = h_bf16 ? 0 : 1;
            A.h_c = s->cin[l];
            A.g = gg;
            A.g_f32 = g_bf16 ? 0 : 1;
            A.g_c = s->cout[l];
            A.CI = s->cin[l];
            A.CO = s->cout[l];
            A.N = s->p.N;
            A.nslot = conv_dw_tc_slots(cip, s->p.N);
            A.nb = s->dw_nb;
            A.part0 = s->dw_part0;
            A.part1 = s->dw_part1;
            A.bpart = s->dw_bpart;
            A.dW = s->dW[l];
            A.db = s->db[l];
            A.status = s->status;
            s->launches += 2;
            return check(launch_conv_dw_tc(cip, cop, A, s->stream));
        }
        ConvDWArgs A{};
        A.h = h;
        A.h_bf16 = h_bf16;
        A.h_act = h_act;
        A.g = gg;
        A.g_bf16 = g_bf16;
        A.cin = s->cin[l];
        A.cout = s->cout[l];
        A.N = s->p.N;
        A.partial = s->partial;
        A.chunks = s->chunks;
        A.dW = s->dW[l];
        A.db = s->db[l];
        s->launches += 2;
        return check(launch_conv_dw(A, s->stream));
    };
    // adjoint of layer l: from the gradient of its output (gin, cin' = cout_l) to the gradient
    // of its input's pre-activation (gated by act'(gate)) or of the network input
    auto dgrad = [&](int l, const void* gin, int gin_bf16, void* gout, int gout_bf16, const void* gate, int gate_bf16,
                     int gate_act, const float* resid) {
        if (ab && l > 0) {  // adjoint of layer l on the tensor cores: cout_l -> cin_l channels
            ConvTCArgs A{};
            A.in = gin;
            A.in_f32 = gin_bf16 ? 0 : 1;
            A.in_c = s->cout[l];
            A.wfmt = s->wb[l];
            A.gate = (const __nv_bfloat16*)gate;
            A.gate_act = gate_act;
            A.out = gout;
            A.out_f32 = gout_bf16 ? 0 : 1;
            A.out_c = s->cin[l];
            A.status = s->status;
            A.N = s->p.N;
            A.DZ = kTcDZ < s->p.N ? kTcDZ : s->p.N;
            conv_tc_encode_input(A, tc_width(s->cout[l]));
            ++s->launches;
            return check(launch_conv_tc(tc_width(s->cout[l]), tc_width(s->cin[l]), A, tc_grid(s, A.DZ), s->stream));
        }
        ConvCCArgs A{};
        A.in = gin;
        A.in_bf16 = gin_bf16;
        A.cin = s->cout[l];
        A.cout = s->cin[l];
        A.w = s->W[l];
        A.flip = 1;
        A.gate = gate;
        A.gate_bf16 = gate_bf16;
        A.gate_act = gate_act;
        A.resid = resid;
        A.resid_c = resid ? s->p.out_channels : 0;
        A.resid_stride = s->p.out_channels;
        A.out = gout;
        A.out_bf16 = gout_bf16;
        A.N = s->p.N;
        ++s->launches;
        return check(launch_conv_cc(A, s->stream));
    };
    // layer inputs h_l = act(u_l): stored as is in BF16 mode, activated on load in FP32 mode;
    // activation-derivative gates: h (ReLU) or the pre-activations (GELU) in BF16 mode
    const int h_act = ab ? 0 : act;
    auto gate_of = [&](int l) -> const void* { return ab && act == CL_ACT_GELU ? s->upre[l] : s->u[l]; };
    // last layer: input h_{L-2}, output gradient g (FP32)
    cl_status st = wgrad(L - 1, s->u[L - 2], ab, h_act, s->g, 0);
    int cur = 0;
    if (st == CL_OK) st = dgrad(L - 1, s->g, 0, s->du[cur], ab, gate_of(L - 2), ab, act, nullptr);
    for (int l = L - 2; st == CL_OK && l >= 1; --l) {
        st = wgrad(l, s->u[l - 1], ab, h_act, s->du[cur], ab);
        if (st == CL_OK) st = dgrad(l, s->du[cur], ab, s->du[cur ^ 1], ab, gate_of(l - 1), ab, act, nullptr);
        cur ^= 1;
    }
    if (st == CL_OK) st = wgrad(0, s->x, 0, 0, s->du[cur], ab);
    if (st == CL_OK && dx) {
        // d/dx: adjoint of layer 0 plus the residual path (g on the first out_channels)
        st = dgrad(0, s->du[cur], ab, s->dx, 0, nullptr, 0, 0, s->g);
        if (st == CL_OK &&
            cudaMemcpyAsync(dx, s->dx, (size_t)s->V * s->p.in_channels * 4,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
            st = CL_ECUDA;
    }
    if (st != CL_OK) return st;
    return read_status(s);
}

cl_status cl_surrogate_get_grads(cl_surrogate* s, int32_t layer, float* dW, float* db)
{
    if (!s || layer < 0 || layer >= (int)s->cin.size() || !dW || !db) return CL_EINVAL;
    const size_t nw = (size_t)27 * s->cout[layer] * s->cin[layer];
    if (cudaMemcpyAsync(dW, s->dW[layer], nw * 4, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
        cudaMemcpyAsync(db, s->db[layer], s->cout[layer] * 4, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
        return CL_ECUDA;
    return cudaStreamSynchronize(s->stream) == cudaSuccess ? CL_OK : CL_ECUDA;
}

int64_t cl_surrogate_last_launch_count(const cl_surrogate* s) { return s ? s->launches : 0; }

int32_t cl_surrogate_size(const cl_surrogate* s) { return s ? s->p.N : 0; }

}  // extern "C"

cudaStream_t surrogate_stream(const cl_surrogate* s) { return s ? s->stream : nullptr; }

extern "C" {

static cl_status ensure_red(cl_surrogate* s, size_t n)
{
    if (n + 1 <= s->red_cap) return CL_OK;
    cudaFree(s->red);
    s->red = nullptr;
    s->red_cap = 0;
    if (cudaMalloc(&s->red, (n + 1) * sizeof(double)) != cudaSuccess) return CL_ENOMEM;
    s->red_cap = n + 1;
    return CL_OK;
}

cl_status cl_surrogate_loss(cl_surrogate* s, const float* target, int32_t stride, const float* scale,
                            int32_t on_device, double* loss)
{
    if (!s || !target || !loss || stride < s->p.out_channels) return CL_EINVAL;
    if (!s->have_forward) return CL_ESTATE;
    const int C = s->p.out_channels;
    const int64_t n = s->V;
    const int np = loss_partials(n);
    cl_status st = ensure_red(s, (size_t)np + 8);
    if (st != CL_OK) return st;
    // target and scale in device memory: the target goes to the (idle) input-gradient buffer
    const float* td = target;
    if (!on_device) {  // host targets are staged in the input-gradient buffer (N^3 x in_channels)
        if (stride > s->p.in_channels) return CL_EINVAL;
        if (cudaMemcpyAsync(s->dx, target, (size_t)n * stride * 4, cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
            return CL_ECUDA;
        td = s->dx;
    }
    float* sc = nullptr;
    if (scale) {
        sc = reinterpret_cast<float*>(s->red + np + 1);
        if (cudaMemcpyAsync(sc, scale, C * 4, cudaMemcpyHostToDevice, s->stream) != cudaSuccess) return CL_ECUDA;
    }
    LossArgs A{};
    A.y = s->y;
    A.t = td;
    A.scale = sc;
    A.g = s->g;
    A.partial = s->red;
    A.n = n;
    A.C = C;
    A.tstride = stride;
    double* res = s->red + np;
    if (launch_loss(A, res, s->stream) != cudaSuccess) return CL_ECUDA;
    if (cudaMemcpyAsync(loss, res, sizeof(double), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return CL_ECUDA;
    s->have_loss = true;
    return CL_OK;
}

cl_status cl_surrogate_adamw(cl_surrogate* s, double lr, double beta1, double beta2, double eps, double weight_decay,
                             int64_t t)
{
    if (!s || t < 1 || !(lr >= 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0) ||
        !(weight_decay >= 0))
        return CL_EINVAL;
    AdamArgs A{};
    A.lr = (float)lr;
    A.b1 = (float)beta1;
    A.b2 = (float)beta2;
    A.eps = (float)eps;
    A.wd = (float)weight_decay;
    A.c1 = (float)(1.0 / (1.0 - pow(beta1, (double)t)));
    A.c2 = (float)(1.0 / (1.0 - pow(beta2, (double)t)));
    for (size_t l = 0; l < s->cin.size(); ++l) {
        const int ci = s->cin[l], co = s->cout[l];
        const int64_t nw = (int64_t)27 * co * ci;
        if (launch_adamw(s->W[l], s->dW[l], s->mW[l], s->vW[l], nw, A, true, s->stream) != cudaSuccess ||
            launch_adamw(s->b[l], s->db[l], s->mb[l], s->vb[l], co, A, false, s->stream) != cudaSuccess)
            return CL_ECUDA;
        if (s->wf[l]) {
            const int cip = tc_width(ci), cop = tc_width(co);
            if (launch_format_tc(s->W[l], co, ci, cop, cip, 0, s->wf[l], s->stream) != cudaSuccess ||
                cudaMemcpyAsync(s->bpad[l], s->b[l], co * 4, cudaMemcpyDeviceToDevice, s->stream) != cudaSuccess)
                return CL_ECUDA;
            if (s->wb[l] && launch_format_tc(s->W[l], ci, co, cip, cop, 1, s->wb[l], s->stream) != cudaSuccess)
                return CL_ECUDA;
        }
    }
    return CL_OK;
}

cl_status cl_surrogate_channel_stats(cl_surrogate* s, const float* x_dev, int64_t n, int32_t channels, float* mean,
                                     float* stdev)
{
    if (!s || !x_dev || n < 1 || channels < 1 || channels > 3 || !mean || !stdev) return CL_EINVAL;
    const int np = channel_stats_partials(n);
    cl_status st = ensure_red(s, (size_t)np + 8);
    if (st != CL_OK) return st;
    float* dm = reinterpret_cast<float*>(s->red + np);
    float* ds = dm + 4;
    if (launch_channel_stats(x_dev, n, channels, s->red, dm, ds, s->stream) != cudaSuccess) return CL_ECUDA;
    if (cudaMemcpyAsync(mean, dm, channels * 4, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
        cudaMemcpyAsync(stdev, ds, channels * 4, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return CL_ECUDA;
    return CL_OK;
}

}  // extern "C"
