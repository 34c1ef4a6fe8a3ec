// Internal declarations of libcl.so (CUDA sm_103a).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/cl.h"

namespace clk {

// A set-once flag kept per CUDA device, for kernel attributes (a function attribute
// set with one device current does not carry over to another device).  Reading and
// setting it refer to the current device; devices numbered 64 and above always read
// false, so their attribute is set again on every call.
struct DevFlag {
    std::atomic<unsigned long long> bits{0ull};
    static int current()
    {
        int d = 0;
        return cudaGetDevice(&d) == cudaSuccess ? d : 64;
    }
    operator bool() const
    {
        const int d = current();
        return d < 64 && ((bits.load(std::memory_order_acquire) >> d) & 1ull);
    }
    DevFlag& operator=(bool v)
    {
        const int d = current();
        if (d < 64) {
            if (v) bits.fetch_or(1ull << d, std::memory_order_acq_rel);
            else bits.fetch_and(~(1ull << d), std::memory_order_acq_rel);
        }
        return *this;
    }
};

// Status bits of the device status word.
enum : int { ST_NAN = 1, ST_CONSTRAINT = 2, ST_TIMEOUT = 4 };

// Diagnostics written by the last block of every fused pass (energies at the pass's
// integer time).  Index names follow cl_energy.
enum {
    D_T = 0, D_A, D_ADOT, D_K0, D_K1, D_G0, D_G1, D_V, D_KE, D_GB, D_RHO, D_P, D_HV, D_GV, D_NDIAG
};

// Device-resident scalar state of one lattice (one ensemble member).
struct DevScal {
    double a;       // scale factor at the time of the stored field values
    double b;       // a' at the staggered (open) or integer (closed) position
    double t;       // alpha-time of the stored field values
    double diag[D_NDIAG];
    long long step;
    unsigned int counter;  // last-block-done arrival counter; the last block resets it to 0
    int status;            // ST_* bits, sticky until read by the host
    double rk[2];          // 2N Runge-Kutta auxiliaries of a and a' (k_a, k_a')
    double rbar;           // background Ricci scalar of the state (non-minimally coupled lattices)
    double gauss[2];       // U(1): rms Gauss violation of the latest step's starting state, and
                           // its maximum over the steps since the state was set
    double h;              // adaptive RK3-4: the step size of the next step (P_DEVICE_H)
    double rk_err;         // adaptive RK3-4: error estimate of the latest step
    double a_prev;         // leapfrog: a before the latest committed scalar pass (the GW pass
                           // that follows it forms the pass's midpoint a from it and a)
};

// Flags of one fused scalar pass.
enum : int {
    P_DRIFT = 1,        // apply the drift phi += d a_half^(alpha-3) pi before the kick
    P_COMMIT = 2,       // update a, a', t and step in DevScal (else only diag)
    P_EXPANSION = 4,    // self-consistent expansion (Eq. Friedmann1)
    P_HUBBLE_INIT = 8,  // set a' from Eq. Friedmann2 with this pass's energies first
    P_COUNT_STEP = 16,  // this pass ends a time step
    P_FIRST_STAGE = 32, // Runge-Kutta: first stage of a step (A = 0, k is not read)
    P_ENERGY_ONLY = 64, // reduce the energies of the state, update nothing else
    P_DEVICE_H = 128,   // Runge-Kutta: take the step size from DevScal::h, not from the arguments
    P_RK_ERROR = 256,   // Runge-Kutta, last stage: reduce the embedded error estimate
                        //   |B k| / |y| and set DevScal::h of the next step (adaptive RK3-4)
};

// Largest dynamic shared memory a fused-pass block may use (227 KB per block on sm_103a,
// less the kernels' static shared memory).
constexpr int kPassMaxSmem = 227 * 1024 - 2048;

// Quantities reduced by the scalar pass: per field sum pi^2 and sum (grad+ phi)^2, and sum V.
constexpr int kMaxQ = 5;

template <typename T>
struct ScalarPassArgs {
    const T* phi_in[2];
    const T* pi_in[2];
    const T* c_in[2];
    T* phi_out[2];
    T* pi_out[2];
    T* c_out[2];
    DevScal* scal;
    double* partials;   // [gridDim.x][kMaxQ]
    int N, BY, DZ, nby, nbz;
    double dx, alpha, kappa;
    double d, e, k;     // drift, energy-kick and kick coefficients of this pass (already x dt)
    double m2[2], lam[2], g2;
    double hubble_limit;
    int flags;
    int stages;         // TMA stage buffers (2..6), 0 = general loader
    int grid;           // persistent grid size (used when DZ < 0)
    int variant;        // TMA kernel: 0 = shared ring of drifted rows, 1 = ringless
};

// Launch one fused scalar pass (drift -> stencil kick -> energies -> scale-factor update).
// Returns the CUDA error of the launch.
cudaError_t launch_scalar_pass(int precision, int nf, const void* args, int vw, cudaStream_t s);
// The same pass on a reduced lattice of N^dims sites (dims = 1, 2), `grid` blocks of 256
// threads (partials[grid][kMaxQ]).
cudaError_t launch_reduced_pass(int precision, int nf, const void* args, int dims, int grid, cudaStream_t s);
// (2+1)-dimensional pass with row marching (scalar_pass.cu): N a multiple of 32 x (16 bytes /
// element size) (plane_pass_ok); dy rows per chunk; pd > 0 prefetches the row pd ahead into L2;
// grid = ceil((N / (32 VW)) x ceil(N / dy) / 8) blocks of 256 threads (one warp per strip and
// chunk).  Same results as launch_reduced_pass.
bool plane_pass_ok(int precision, int N);
cudaError_t launch_plane_pass(int precision, int nf, const void* args, int dy, int pd, int grid, cudaStream_t s);
// Resident blocks per SM of the pass configured by args (tiles, stages).
cudaError_t scalar_pass_blocks_per_sm(int precision, int nf, const void* args, int vw, int* blocks);
int scalar_pass_vector_width(int precision, int N);
size_t scalar_pass_smem(int precision, int nf, int N, int BY);
size_t scalar_pass_smem_bytes(int precision, int nf, int N, int BY, int stages, int variant = 0);
bool scalar_pass_tma_ok(int precision, int N);
int scalar_pass_threads(int precision, int N, int BY);

// One 2N Runge-Kutta stage of the scalar fields and the scale factor.
template <typename T>
struct RkStageArgs {
    const T* phi_in[2];
    const T* pi_in[2];
    const T* c_in[2];
    const T* kphi_in[2];
    const T* kpi_in[2];
    T* phi_out[2];
    T* pi_out[2];
    T* c_out[2];
    T* kphi_out[2];
    T* kpi_out[2];
    DevScal* scal;
    double* partials;   // [gridDim.x][kMaxQ]
    int N, BY, DZ, nby, nbz;
    double dx, alpha, kappa;
    double A, B, h;     // stage coefficients and the step size
    double m2[2], lam[2], g2;
    double hubble_limit;
    double tol, hmin, hmax;  // adaptive step-size control (P_RK_ERROR)
    int flags;          // P_EXPANSION, P_FIRST_STAGE, P_COUNT_STEP, P_DEVICE_H, P_RK_ERROR
    int nmc;            // non-minimal coupling xi phi^2 R of field 0 (one field): the kick and a''
    double xi;          //   use scal->rbar, written by launch_nmc_ricci for the same state
};
cudaError_t launch_rk_stage(int precision, int nf, const void* args, int vw, cudaStream_t s);
// Gravitational waves (gw_pass.cu): five traceless auxiliaries v = {v11, v12, v13, v22,
// v23} and their momenta, kicked and drifted by one pass after each fused scalar pass with
// the same coefficients; that pass's output (the drifted scalars) provides the source.
template <typename T>
struct GwPassArgs {
    const T* phi_in[2];  // the scalars drifted by this pass: the scalar pass's output
    const T* v_in[5];
    const T* pv_in[5];
    T* v_out[5];
    T* pv_out[5];
    const DevScal* scal;
    int N, BY, DZ, nby, nbz;
    double dx, alpha, kappa;
    double d, k;        // pass coefficients (already x dt), as in ScalarPassArgs; the pass
                        // runs after the scalar pass of the same coefficients
    int flags;          // P_DRIFT, P_EXPANSION
};
cudaError_t launch_gw_pass(int precision, int nf, const void* args, int vw, cudaStream_t s);
size_t gw_pass_smem(int nf, int N, int BY, int es);
// TT energy spectrum sums of the five transformed momenta F[5][N][N][N/2+1] (h'_33 = -h'_11 - h'_22)
cudaError_t launch_gw_bins(const double2* F, int N, double dx, double dn, int nbins, double* S, double* C,
                           cudaStream_t s);

// Background Ricci scalar (Eq. eomR) of the state phi_in, pi_in (field 0) into scal->rbar:
// `grid` blocks, partials[grid][kMaxQ].
cudaError_t launch_nmc_ricci(int precision, const void* args, int grid, cudaStream_t s);

// Axion + compact U(1) links, one 2N Runge-Kutta stage (u1_stage.cu).  Degrees of
// freedom per site, in k order: phi, pi, theta_1..3, E_1..3.
template <typename T>
struct U1Args {
    const T* phi_in;
    const T* pi_in;
    const T* th_in[3];
    const T* E_in[3];
    const T* k_in[8];
    T* phi_out;
    T* pi_out;
    T* th_out[3];
    T* E_out[3];
    T* k_out[8];
    T* sP[3];     // per-site plaquette fields written by the plaquette launch (normal k):
    T* rP[3];     //   sin P_k, cos P_k * dP_k/dt, and cos P_k times the corner sum of phi Ebar_k
    T* Z[3];
    DevScal* scal;
    double* partials;
    int N;
    double dx, alpha, kappa, g, ws2, m2, lam;
    double A, B, h;
    double hubble_limit;
    int flags;    // P_EXPANSION, P_FIRST_STAGE, P_COUNT_STEP, P_ENERGY_ONLY, P_HUBBLE_INIT
    int dz;       // planes per block (all three kernels)
    // Leapfrog passes (lf != 0; the stage launch only, the plaquette launch is unchanged).
    // The force f = (pi', E') is evaluated at positions (phi, theta, a) with the momenta of
    // pi_in / E_in and a' = scal->b; p~ denotes those momenta, base those of k_in[1], k_in[5..7].
    //   lf 1: k_out[1], k_out[5..7] = p~ + le f (the integer-time momenta, whose energies are
    //         reduced), pi_out / E_out = p~ + lk f; a' += lb a''(rho), diag a' = a' + le a''
    //   lf 2: pi_out / E_out = base + lk f
    //   lf 3: as 2, then phi_out = phi + h ((a + a_1)/2)^(alpha-3) pi_out, theta_out = theta
    //         + h dx E_out with a_1 = a + h a'; a = a_1, t += h, step += 1
    int lf;
    double le, lk, lb;
    // cos P of every plaquette (normal k, lower corner n), saved by a plaquette launch when
    // non-null; the staged "rates" launch (launch_u1_staged what 3) reads it back and forms
    // only the fields that depend on E (cos P dP/dt and the Chern-Simons corner sums) for
    // the same link angles, keeping sin P from the launch that saved it
    T* cP[3];
};
// what: 0 = plaquette fields, 1 = stage (or energies with P_ENERGY_ONLY), 2 = Gauss diagnostic,
// 3 = rms Gauss violation of the state into DevScal::gauss (the staged stage launch computes
// it itself in the first stage of every step).
// The plaquette launch writes its magnetic-energy partials after the stage's, at
// partials[u1_grid_blocks(N, dz) * kMaxQ + block].
cudaError_t launch_u1(int precision, const void* args, int what, cudaStream_t s);
int u1_grid_blocks(int N, int dz);
// Fused stage (u1_fused.cu): plaquettes and stage in one launch, grid u1_grid_blocks(N, dz),
// its partials (all five sums) at partials[block * kMaxQ]; needs u1_fused_ok(N).
bool u1_fused_ok(int N);
cudaError_t launch_u1_fused(int precision, const void* args, cudaStream_t s);
cudaError_t u1_fused_blocks_per_sm(int precision, int* blocks);

// Batched ensemble of independent lattices (ensemble_pass.cu).  Every array class (phi,
// pi, compensation, per field and buffer) is one arena holding the members back to back,
// each starting on a 256-byte boundary.  A work item is BY full x rows times DZ planes of
// one member; items of a member are consecutive in the item table.
constexpr int kEnsThreads = 256;
struct EnsMember {
    long long off;       // element offset of the member's arrays in every arena
    int N, BY, DZ;       // sites per side and the tile of one work item
    int item0, nitems;   // the member's work items [item0, item0 + nitems)
    double dx;
    double m2[2], lam[2], g2;
};
struct EnsItem {
    int member, y0, z0, pad;
};
template <typename T>
struct EnsPassArgs {
    const T* phi_in[2];
    const T* pi_in[2];
    const T* c_in[2];
    T* phi_out[2];
    T* pi_out[2];
    T* c_out[2];
    const EnsMember* members;
    const EnsItem* items;
    const int* sched;     // processing order of all items (nullptr: items item_begin.. in order)
    DevScal* scal;        // one per member
    double* partials;     // [items][kMaxQ]
    int item_begin, item_end;
    double alpha, kappa;
    double d, e, k;       // pass coefficients (already x dt), as in ScalarPassArgs
    double hubble_limit;
    int flags;
    int stages;           // TMA stage buffers (ring 2..4, ringless 3..6) or 0 for the direct loader
    int stage_stride;     // elements of one stage buffer (largest member tile)
    int ring_slot;        // elements of one ring slot of drifted fields (largest member tile)
    int variant;          // TMA kernel: 0 = ring of drifted rows, 1 = ringless
};
constexpr int kEnsTmaThreads = kEnsThreads + 32;  // consumers + one producer warp
// One pass over the items [item_begin, item_end) with `grid` persistent blocks.
cudaError_t launch_ensemble_pass(int precision, int nf, const void* args, int vw, int grid, size_t smem,
                                 cudaStream_t s);
cudaError_t ensemble_pass_blocks_per_sm(int precision, int nf, int vw, int stages, int variant, size_t smem,
                                        int* blocks);

// Vacuum initial conditions: fills the half spectrum (kx in [0, N/2]) of delta f and
// delta pi for one field into two complex-double buffers of N*N*(N/2+1) entries.
struct VacuumModeArgs {
    int N, field;
    uint32_t member;
    uint64_t seed;
    double L, kcut, amp2, a, alpha, H, m2eff;
};
cudaError_t launch_vacuum_modes(const VacuumModeArgs& a, double2* fk, double2* pk, cudaStream_t s);
// out[n] = base + scale * in[n], converted to the field's element type.
cudaError_t launch_real_to_field(int precision, const double* in, void* out, double base, double scale,
                                 int64_t n, cudaStream_t s);
cudaError_t launch_field_to_double(int precision, const void* in, double* out, int64_t n, cudaStream_t s);

// Spectra of the U(1) sector (gauge_spectrum.cu): the three component fields of `which`
// (0 electric, 1 magnetic, 2 / 3 the gauge potential for the + / - chirality) as doubles
// [3][N^3], and the shell binning of their D2Z transforms F[3][N][N][N/2+1].
template <typename T>
struct GaugeSpecArgs {
    const T* th[3];
    const T* E[3];
    int N;
    double dx;
    int which;
};
cudaError_t launch_gauge_fields(int precision, const void* args, double* out, cudaStream_t s);
cudaError_t launch_gauge_bins(const double2* F, int N, double dx, int which, double dn, int nbins, double* S,
                              double* C, cudaStream_t s);
// Shell binning of |F|^2 over a real-to-complex half spectrum: S[l], C[l] (zeroed by the caller).
cudaError_t launch_spectrum_bins(const double2* F, int N, double dn, int nbins, double* S, double* C,
                                 cudaStream_t s);
// delta[l] from S, C per the spectrum formula of cl_spectrum.
cudaError_t launch_spectrum_finish(const double* S, const double* C, int N, double L, double dn, int type,
                                   int nbins, double* k_out, double* delta_out, cudaStream_t s);
cudaError_t launch_fill(void* p, int precision, int64_t n, double v, cudaStream_t s);

}  // namespace clk
