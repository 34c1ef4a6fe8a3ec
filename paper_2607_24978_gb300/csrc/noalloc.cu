// Allocation-free entry point: one fused scalar pass on caller-owned device arrays.
//
// Some callers cannot allocate device memory at the time they step a lattice: code
// running inside an application that owns a fixed memory arena or pool, embedded or
// real-time hosts that forbid allocation after start-up, or frameworks that hand the
// library only pre-allocated buffers.  cl_fused_pass_noalloc serves them: it runs the
// same fused-pass kernel as cl_step on arrays the caller provides, and keeps its
// scratch (the block partials of the energy reduction, the arrival counter and the
// working copy of a, a', t) in a fixed array of static device memory that every GPU
// loading the library reserves until the process exits.
//
// The array's host-side name is not a device address, so the address used for the
// kernels is fetched once per device with cudaGetSymbolAddress (with that device
// current) the first time the entry point runs there.  Every call shares the array:
// calls whose work overlaps on the GPU (other streams, other host threads) race, and
// each call clears the part that must start at zero.
#include <mutex>

#include "cl_internal.cuh"

using namespace clk;

namespace {

constexpr int kNoAllocMaxBlocks = 8192;  // largest grid the scratch can serve
constexpr size_t kScalBytes = (sizeof(DevScal) + 255) / 256 * 256;
constexpr size_t kNoAllocScratchBytes = kScalBytes + (size_t)kNoAllocMaxBlocks * kMaxQ * sizeof(double);

// DevScal at offset 0, then kNoAllocMaxBlocks * kMaxQ doubles of block partials.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Address of the scratch array on the current device (set-up once per device).
cudaError_t scratch_address(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

// Load the caller's a, a', t into the scratch DevScal and clear counter and status.
__global__ void k_noalloc_load(DevScal* S, const double* __restrict__ abt)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        S->a = abt[0];
        S->b = abt[1];
        S->t = abt[2];
        S->step = 0;
        S->counter = 0u;
        S->status = 0;
        for (int i = 0; i < D_NDIAG; ++i) S->diag[i] = 0.0;
    }
}

// Copy the updated a, a', t, the pass's energies and its status bits back to the caller.
__global__ void k_noalloc_store(const DevScal* S, double* __restrict__ abt, double* __restrict__ energies,
                                int32_t* __restrict__ status)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        abt[0] = S->a;
        abt[1] = S->b;
        abt[2] = S->t;
        if (energies)
            for (int i = 0; i < D_NDIAG; ++i) energies[i] = S->diag[i];
        if (status) *status = S->status;
    }
}

// True when p is device (or managed) memory that the current device can address.
bool on_current_device(const void* p, int dev)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();  // clear the sticky-free error of an unknown pointer
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

bool overlap(const void* a, const void* b, size_t bytes)
{
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + bytes && y < x + bytes;
}

template <typename T>
void fill_args(ScalarPassArgs<T>& A, const cl_pass_noalloc_desc* d)
{
    for (int f = 0; f < d->nfields; ++f) {
        A.phi_in[f] = (const T*)d->phi_in[f];
        A.pi_in[f] = (const T*)d->pi_in[f];
        A.c_in[f] = (const T*)d->c_in[f];
        A.phi_out[f] = (T*)d->phi_out[f];
        A.pi_out[f] = (T*)d->pi_out[f];
        A.c_out[f] = (T*)d->c_out[f];
    }
}

}  // namespace

extern "C" cl_status cl_fused_pass_noalloc(const cl_pass_noalloc_desc* d)
{
    if (!d) return CL_EINVAL;
    const int N = d->N, nf = d->nfields, prec = d->precision;
    if (N < 2 || N > 1536 || nf < 1 || nf > 2 || prec < 0 || prec > 2 || !(d->L > 0) || !d->scalars)
        return CL_EINVAL;
    const bool kahan = prec == CL_PREC_FP32_KAHAN;
    for (int f = 0; f < nf; ++f) {
        if (!d->phi_in[f] || !d->pi_in[f] || !d->phi_out[f] || !d->pi_out[f]) return CL_EINVAL;
        if (kahan && (!d->c_in[f] || !d->c_out[f])) return CL_EINVAL;
    }
    if (nf == 1 && (d->m2[1] != 0 || d->lam[1] != 0 || d->g2 != 0)) return CL_EINVAL;

    // Tiling of the direct-load kernel: full x rows, BY rows per block, DZ planes per block,
    // with the grid kept within the scratch's block capacity.  A row of N / VW threads must
    // fit the kernel's 512-thread blocks (the same rule as cl_step's set-up): odd N up to
    // 512, even N up to 1024, and in FP32 multiples of 4 up to 1536.
    const int VW = scalar_pass_vector_width(prec, N);
    const int TX = N / VW;
    int BY = TX >= 256 ? 1 : 256 / TX;
    if (BY > N) BY = N;
    while (BY > 1 && scalar_pass_threads(prec, N, BY) > 512) --BY;
    while (BY > 1 && scalar_pass_smem_bytes(prec, nf, N, BY, 0) > (size_t)kPassMaxSmem) --BY;
    if (scalar_pass_threads(prec, N, BY) > 512) return CL_EINVAL;
    if (scalar_pass_smem_bytes(prec, nf, N, BY, 0) > (size_t)kPassMaxSmem) return CL_EINVAL;

    // Every array must be memory of the current device, and no output may overlap an input
    // or another output (inputs are read while outputs are written).
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CL_ECUDA;
    const size_t bytes = (size_t)N * N * N * (prec == CL_PREC_FP64 ? sizeof(double) : sizeof(float));
    const void* ins[6];
    const void* outs[6];
    int nin = 0, nout = 0;
    for (int f = 0; f < nf; ++f) {
        ins[nin++] = d->phi_in[f];
        ins[nin++] = d->pi_in[f];
        outs[nout++] = d->phi_out[f];
        outs[nout++] = d->pi_out[f];
        if (kahan) {
            ins[nin++] = d->c_in[f];
            outs[nout++] = d->c_out[f];
        }
    }
    for (int i = 0; i < nin; ++i)
        if (!on_current_device(ins[i], dev)) return CL_EINVAL;
    for (int i = 0; i < nout; ++i) {
        if (!on_current_device(outs[i], dev)) return CL_EINVAL;
        for (int j = 0; j < nin; ++j)
            if (overlap(outs[i], ins[j], bytes)) return CL_EINVAL;
        for (int j = 0; j < i; ++j)
            if (overlap(outs[i], outs[j], bytes)) return CL_EINVAL;
    }
    if (!on_current_device(d->scalars, dev)) return CL_EINVAL;
    if (d->energies && !on_current_device(d->energies, dev)) return CL_EINVAL;
    if (d->status && !on_current_device(d->status, dev)) return CL_EINVAL;
    const int nby = (N + BY - 1) / BY;
    if (nby > kNoAllocMaxBlocks) return CL_EINVAL;  // beyond the scratch capacity
    int nbz = (N + 15) / 16;
    if ((int64_t)nby * nbz > kNoAllocMaxBlocks) nbz = kNoAllocMaxBlocks / nby;
    const int DZ = (N + nbz - 1) / nbz;
    nbz = (N + DZ - 1) / DZ;

    void* scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return CL_ECUDA;
    DevScal* S = (DevScal*)scratch;
    double* partials = (double*)((unsigned char*)scratch + kScalBytes);
    cudaStream_t s = (cudaStream_t)d->stream;

    const int flags = P_COMMIT | (d->drift != 0.0 ? P_DRIFT : 0) | (d->expansion ? P_EXPANSION : 0);
    k_noalloc_load<<<1, 32, 0, s>>>(S, d->scalars);
    if (cudaGetLastError() != cudaSuccess) return CL_ECUDA;
    cudaError_t e;
    if (prec == CL_PREC_FP64) {
        ScalarPassArgs<double> A{};
        fill_args(A, d);
        A.scal = S; A.partials = partials;
        A.N = N; A.BY = BY; A.DZ = DZ; A.nby = nby; A.nbz = nbz;
        A.dx = d->L / N; A.alpha = d->alpha; A.kappa = d->kappa;
        A.d = d->drift; A.e = d->energy_kick; A.k = d->kick;
        for (int f = 0; f < 2; ++f) { A.m2[f] = d->m2[f]; A.lam[f] = d->lam[f]; }
        A.g2 = d->g2; A.hubble_limit = 0.0; A.flags = flags; A.stages = 0; A.grid = nby * nbz;
        e = launch_scalar_pass(prec, nf, &A, VW, s);
    } else {
        ScalarPassArgs<float> A{};
        fill_args(A, d);
        A.scal = S; A.partials = partials;
        A.N = N; A.BY = BY; A.DZ = DZ; A.nby = nby; A.nbz = nbz;
        A.dx = d->L / N; A.alpha = d->alpha; A.kappa = d->kappa;
        A.d = d->drift; A.e = d->energy_kick; A.k = d->kick;
        for (int f = 0; f < 2; ++f) { A.m2[f] = d->m2[f]; A.lam[f] = d->lam[f]; }
        A.g2 = d->g2; A.hubble_limit = 0.0; A.flags = flags; A.stages = 0; A.grid = nby * nbz;
        e = launch_scalar_pass(prec, nf, &A, VW, s);
    }
    if (e != cudaSuccess) return CL_ECUDA;
    k_noalloc_store<<<1, 32, 0, s>>>(S, d->scalars, d->energies, d->status);
    if (cudaGetLastError() != cudaSuccess) return CL_ECUDA;
    return CL_OK;
}
