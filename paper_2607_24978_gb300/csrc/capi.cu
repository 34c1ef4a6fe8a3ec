// C ABI of libcl.so: handle management, state transfer, the integrator schedules and
// CUDA-graph replay.  Every arithmetic step of the evolution runs in the kernels of
// this folder; the host code here only orders launches and moves buffers.
#include <cufft.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <string>
#include <new>
#include <vector>

#include "cl_internal.cuh"
#include "surrogate_train.cuh"
#include "rk_tma.cuh"
#include "u1_staged.cuh"

using namespace clk;

namespace {

constexpr int kMaxN = 1536;
constexpr int kMaxMembers = 1 << 16;  // ensemble members per handle
constexpr int kEnsMaxN = 512;         // sites per side of one ensemble member
// resident blocks per SM of the U(1) stage kernel (its launch bounds: FP32, FP64)
constexpr int kU1BlocksPerSM32 = 4, kU1BlocksPerSM64 = 2;

// One pass of a kick-drift scheme in staggered form (see scalar_pass.cu):
// drift by d, energies with pi + e F, kick by k.
struct PassCoef {
    double d, e, k;   // leapfrog pass: drift, energy-kick and kick coefficients
    int flags;
    int rk = 0;       // 1: a 2N Runge-Kutta stage with coefficients A, B instead
    double A = 0.0, B = 0.0;
    int lf = 0;       // 1..3: a pass of the axion-U(1) leapfrog (U1Args::lf) with le, lk, lb
    double le = 0.0, lk = 0.0, lb = 0.0;
    bool flip = true;  // the pass leaves the state in the other buffer
};

bool is_rk(int integrator)
{
    return integrator == CL_INT_RK3_3 || integrator == CL_INT_RK4_5 || integrator == CL_INT_RK3_4;
}

}  // namespace

struct cl_lattice {
    cl_lattice_params p{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int N = 0, nf = 1, es = 8, VW = 1, BY = 1, DZ = 1, nby = 1, nbz = 1, stages = 0, grid = 1;
    int64_t V = 0;
    double dx = 1.0;
    void* phi[2][2] = {};  // [field][buffer]
    void* pi[2][2] = {};
    void* cc[2][2] = {};
    void* kphi[2][2] = {};  // Runge-Kutta auxiliaries (RK integrators only)
    void* kpi[2][2] = {};
    int rk_BY = 1, rk_DZ = 1, rk_nby = 1, rk_nbz = 1;
    int rk_stages = 0;              // TMA-staged Runge-Kutta kernel with this many stages (0: direct loads)
    int variant = 0;          // TMA pass kernel in use (0 ring, 1 ringless)
    bool gauge = false;       // axion + compact U(1) links (one scalar field, Runge-Kutta)
    void* th[3][2] = {};      // link angles theta_i
    void* ef[3][2] = {};      // electric fields E_i
    void* ku1[8][2] = {};     // Runge-Kutta auxiliaries of phi, pi, theta_1..3, E_1..3
    void* u1s[9] = {};        // per-site scratch: Bbar_1..3, their rates, phi Ebar_1..3
    double alphaL = 0.0, ws2 = 0.0;
    int cur = 0;
    DevScal* scal = nullptr;
    double* partials = nullptr;
    int partials_cap = 0;
    double m2[2] = {0, 0}, lam[2] = {0, 0}, g2 = 0;
    bool potential_set = false;
    bool open = false;
    bool diag_valid = false;
    double hubble_limit = 0.0;
    bool use_graph = true;
    int opt_BY = 0, opt_DZ = 0, opt_stages = 0, opt_variant = -1;  // -1: library choice
    int u1_dz = 8;                  // planes per block of the U(1) kernels
    int u1_gdz = 8;                 // planes per block of the gather kernels beside staged ones
    bool u1_fused = false;          // U(1) stage as one fused launch (plaquettes in shared memory)
    bool u1_staged = false;         // U(1) launches with shared-memory staged neighbourhoods
    bool u1_sfused = false;         //   as one launch, the plaquette fields in shared memory
    bool u1_lf_pq = false;          // axion-U(1) leapfrog: sin P, cos P of the current positions
                                    //   saved by a staged pass (ku1 slots 2..4)
    int dims = 3;                   // spatial dimensions (1, 2: reduced lattice of N^dims sites)
    int red_grid = 1;               // blocks of the reduced-lattice kernels
    int red_dy = 0, red_pgrid = 0;  // (2+1) row-marching pass: rows per chunk and blocks (0: not used)
    int red_pd = 0;                 //   and the rows ahead of its L2 prefetch (0: none)
    bool nmc = false;               // non-minimal coupling xi phi^2 R of field 0 (Runge-Kutta)
    bool rbar_valid = false;        // scal->rbar holds the Ricci scalar of the current state
    double xi = 0.0;
    double adapt_tol = 0.0;         // adaptive RK3-4 steps when > 0 (the step size lives in scal->h)
    double adapt_hmin = 0.0, adapt_hmax = 0.0;
    bool gw = false;                // gravitational-wave auxiliaries evolved with the leapfrog
    void* gv[5][2] = {};            // v11, v12, v13, v22, v23 (ping-pong)
    void* gpv[5][2] = {};           // their momenta a^(3-alpha) v'
    int gw_BY = 1, gw_DZ = 1, gw_nby = 1, gw_nbz = 1;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int64_t last_launches = 0;
    // batched ensemble (members > 1): per-member sizes, boxes, arena offsets and couplings
    int members = 1;
    std::vector<int> mN;
    std::vector<double> mL;
    std::vector<long long> moff;
    std::vector<double> mpot;       // 5 per member: m2_0, lam_0, m2_1, lam_1, g2
    std::vector<EnsMember> hmem;
    std::vector<EnsItem> hitems;
    EnsMember* d_members = nullptr;
    EnsItem* d_items = nullptr;
    int* d_sched = nullptr;         // items by decreasing size
    int nitems = 0, ens_grid = 0, ens_stages = 0, ens_stage_stride = 0, ens_ring_slot = 0, ens_variant = 0;
    float* sg_buf = nullptr;        // surrogate jumps: packed input (3 V), output (2 V), snapshot (3 V)
    size_t ens_smem = 0;
    char err[512] = {0};
};

namespace {

cl_status fail(cl_lattice* l, cl_status s, const char* fmt, ...)
{
    if (l) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(l->err, sizeof(l->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

#define CUDA_TRY(l, call)                                                                                   \
    do {                                                                                                    \
        cudaError_t e_ = (call);                                                                            \
        if (e_ != cudaSuccess) return fail((l), CL_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

bool is_fp64(const cl_lattice* l) { return l->p.precision == CL_PREC_FP64; }
bool has_kahan(const cl_lattice* l) { return l->p.precision == CL_PREC_FP32_KAHAN; }
bool is_ens(const cl_lattice* l) { return l->members > 1; }
// axion-U(1) lattice integrated with the leapfrog (the only leapfrog a gauge lattice accepts)
bool is_u1_lf(const cl_lattice* l) { return l->gauge && !is_rk(l->p.integrator); }
int mem_N(const cl_lattice* l, int m) { return is_ens(l) ? l->mN[m] : l->N; }
int64_t mem_V(const cl_lattice* l, int m)
{
    const int64_t n = mem_N(l, m);
    if (!is_ens(l) && l->dims < 3) return l->dims == 1 ? n : n * n;  // reduced lattice
    return n * n * n;
}
size_t mem_off_bytes(const cl_lattice* l, int m) { return is_ens(l) ? (size_t)l->moff[m] * l->es : 0; }
double mem_L(const cl_lattice* l, int m) { return is_ens(l) ? l->mL[m] : l->p.L; }
bool member_ok(const cl_lattice* l, int m) { return m >= 0 && m < l->members; }

void invalidate_graphs(cl_lattice* l)
{
    for (auto& g : l->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

cl_status query_blocks_per_sm(cl_lattice* l, int* per_sm);

cl_status grow_partials(cl_lattice* l, int nblocks)
{
    if (nblocks > l->partials_cap) {
        if (l->partials) cudaFree(l->partials);
        l->partials = nullptr;
        if (cudaMalloc(&l->partials, sizeof(double) * kMaxQ * (size_t)nblocks) != cudaSuccess)
            return fail(l, CL_ENOMEM, "cannot allocate %d reduction partials", nblocks);
        l->partials_cap = nblocks;
    }
    return CL_OK;
}

// Copy the per-member couplings into the descriptor table and upload it.
cl_status upload_members(cl_lattice* l)
{
    for (int m = 0; m < l->members; ++m) {
        EnsMember& M = l->hmem[m];
        const double* q = &l->mpot[5 * (size_t)m];
        M.m2[0] = q[0]; M.lam[0] = q[1]; M.m2[1] = q[2]; M.lam[1] = q[3]; M.g2 = q[4];
    }
    CUDA_TRY(l, cudaMemcpy(l->d_members, l->hmem.data(), sizeof(EnsMember) * l->hmem.size(), cudaMemcpyHostToDevice));
    return CL_OK;
}

// Ensemble work items.  Per member: BY full rows (as many as one block's threads cover)
// by all N planes (or CL_OPT_TILE_DZ planes), both balanced within the member; long items
// amortise the per-item pipeline start and epilogue (measured: 16-plane items ran at 37%
// of HBM bandwidth, whole columns at 67% on 32..64^3 members).  The items of a member are
// consecutive in the table (their partials are reduced in that order); blocks take items
// in order of decreasing size (largest first balances the persistent grid's tail).  The
// persistent grid is one wave of resident blocks.
cl_status ens_tiles(cl_lattice* l)
{
    const int B = l->members, prec = l->p.precision;
    l->hmem.assign(B, EnsMember{});
    l->hitems.clear();
    size_t smem = 0;
    int64_t stage_max = 0, ring_max = 0;
    const int narr = l->nf * (has_kahan(l) ? 3 : 2);
    for (int m = 0; m < B; ++m) {
        const int N = l->mN[m], TX = N / l->VW;
        int BY = kEnsThreads / TX;
        if (l->opt_BY > 0 && l->opt_BY < BY) BY = l->opt_BY;
        if (BY > N) BY = N;
        if (BY < 1) BY = 1;
        const int nby = (N + BY - 1) / BY;
        BY = (N + nby - 1) / nby;
        int DZ = l->opt_DZ > 0 ? l->opt_DZ : N;
        if (DZ > N) DZ = N;
        if (DZ < 1) DZ = 1;
        const int nbz = (N + DZ - 1) / DZ;
        DZ = (N + nbz - 1) / nbz;
        EnsMember& M = l->hmem[m];
        M.off = l->moff[m];
        M.N = N;
        M.BY = BY;
        M.DZ = DZ;
        M.item0 = (int)l->hitems.size();
        M.nitems = nby * nbz;
        M.dx = l->mL[m] / N;
        if ((nby - 1) * BY >= N || (nbz - 1) * DZ >= N) return fail(l, CL_EINVAL, "ensemble tiling error");
        for (int bz = 0; bz < nbz; ++bz)
            for (int by = 0; by < nby; ++by) l->hitems.push_back({m, by * BY, bz * DZ, 0});
        const size_t sm = (size_t)l->nf * 3 * (BY + 2) * N * l->es;
        if (sm > smem) smem = sm;
        if ((int64_t)narr * (BY + 2) * N > stage_max) stage_max = (int64_t)narr * (BY + 2) * N;
        if ((int64_t)l->nf * (BY + 2) * N > ring_max) ring_max = (int64_t)l->nf * (BY + 2) * N;
    }
    if (smem > (size_t)kPassMaxSmem) return fail(l, CL_EINVAL, "ensemble member too large for the pass tiling");
    // TMA staging when every member row is a multiple of 16 bytes (16-byte vectors): the
    // ringless kernel (default; 3..6 stages, no ring of drifted rows) or the ring kernel
    // (2..4 stages); by default as many stages (up to 5 / 4) as leave room for two blocks
    // per SM
    int stages = 0, var = 0;
    if (l->opt_stages >= 0 && l->VW * l->es == 16) {
        var = l->opt_variant != 0 ? 1 : 0;
        const int smin = var ? 3 : 2, smax = var ? 6 : 4;
        auto bytes = [&](int S) { return (size_t)(S * stage_max + (var ? 0 : 3 * ring_max)) * l->es; };
        if (l->opt_stages >= 2) {
            const int S = l->opt_stages < smin ? smin : (l->opt_stages > smax ? smax : l->opt_stages);
            stages = bytes(S) <= (size_t)kPassMaxSmem ? S : 0;
        } else {
            for (int S = var ? 5 : 4; S >= smin && !stages; --S)
                if (bytes(S) <= (size_t)kPassMaxSmem / 2) stages = S;
        }
        if (stages) smem = bytes(stages);
    }
    if (!stages) var = 0;
    l->ens_stages = stages;
    l->ens_variant = var;
    l->ens_stage_stride = (int)stage_max;
    l->ens_ring_slot = (int)ring_max;
    l->nitems = (int)l->hitems.size();
    l->ens_smem = smem;
    if (l->d_items) cudaFree(l->d_items);
    l->d_items = nullptr;
    if (l->d_sched) cudaFree(l->d_sched);
    l->d_sched = nullptr;
    if (!l->d_members && cudaMalloc(&l->d_members, sizeof(EnsMember) * B) != cudaSuccess)
        return fail(l, CL_ENOMEM, "cannot allocate the member table");
    if (cudaMalloc(&l->d_items, sizeof(EnsItem) * l->hitems.size()) != cudaSuccess)
        return fail(l, CL_ENOMEM, "cannot allocate the item table");
    CUDA_TRY(l, cudaMemcpy(l->d_items, l->hitems.data(), sizeof(EnsItem) * l->hitems.size(), cudaMemcpyHostToDevice));
    {
        std::vector<int> order(l->hitems.size());
        std::vector<int64_t> size(l->hitems.size());
        for (size_t i = 0; i < order.size(); ++i) {
            const EnsItem& I = l->hitems[i];
            const EnsMember& M = l->hmem[I.member];
            const int R = M.BY < M.N - I.y0 ? M.BY : M.N - I.y0, NZ = M.DZ < M.N - I.z0 ? M.DZ : M.N - I.z0;
            order[i] = (int)i;
            size[i] = (int64_t)R * NZ * M.N;
        }
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return size[a] > size[b]; });
        if (cudaMalloc(&l->d_sched, sizeof(int) * order.size()) != cudaSuccess)
            return fail(l, CL_ENOMEM, "cannot allocate the item schedule");
        CUDA_TRY(l, cudaMemcpy(l->d_sched, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice));
    }
    cl_status s = upload_members(l);
    if (s != CL_OK) return s;
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
        return fail(l, CL_ECUDA, "cannot query the SM count");
    CUDA_TRY(l, ensemble_pass_blocks_per_sm(prec, l->nf, l->VW, stages, var, smem, &per_sm));
    if (per_sm < 1) return fail(l, CL_EINVAL, "ensemble pass does not fit on an SM");
    const int64_t wave = (int64_t)per_sm * nsm;
    l->ens_grid = (int)(wave < l->nitems ? wave : l->nitems);
    s = grow_partials(l, l->nitems);
    if (s != CL_OK) return s;
    invalidate_graphs(l);
    return CL_OK;
}

cl_status choose_tiles(cl_lattice* l)
{
    if (is_ens(l)) return ens_tiles(l);
    if (l->dims < 3) {
        // reduced lattice: one thread per site, at most eight blocks per SM
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
            return fail(l, CL_ECUDA, "cannot query the SM count");
        const int64_t blocks = (l->V + 255) / 256;
        l->red_grid = (int)(blocks < 8 * (int64_t)nsm ? blocks : 8 * (int64_t)nsm);
        l->VW = 1;
        // (2+1) leapfrog passes: the row-marching kernel where the strips divide N (the library's
        // choice, pass variant 1), else one thread per site (variant 0).  By default one wave of
        // warps (three 256-thread blocks per SM, its launch bounds): enough chunks of rows that
        // strips x chunks fills it, at least 8 rows a chunk (the two halo rows of a chunk are
        // loaded twice; measured at 4096^2: 36 rows, one wave, 0.70 of HBM; 18 rows, two waves,
        // 0.65; 24 rows, 1.5 waves, 0.55); CL_OPT_TILE_DZ > 0 sets the rows per chunk
        l->red_dy = 0;
        l->red_pgrid = 0;
        l->variant = 0;
        if (l->dims == 2 && l->opt_variant != 0 && plane_pass_ok(l->p.precision, l->N)) {
            const int64_t N = l->N, strips = N / (l->p.precision == CL_PREC_FP64 ? 64 : 128);
            const int64_t target = 24 * (int64_t)nsm;
            int64_t chunks = (target + strips - 1) / strips;
            if (chunks > N) chunks = N;
            int64_t dy = (N + chunks - 1) / chunks;
            if (dy < 8) dy = N < 8 ? N : 8;
            if (l->opt_DZ > 0) dy = l->opt_DZ > N ? N : l->opt_DZ;
            // the next row but one prefetched into L2 while the next is loaded (measured at
            // 4096^2 FP32 + Kahan, two fields: 0.70 of HBM without, 0.77 one row ahead, 0.61-0.68
            // two to eight rows ahead); CL_OPT_TILE_BY > 0 sets the distance
            l->red_pd = l->opt_BY > 0 ? l->opt_BY : 1;
            chunks = (N + dy - 1) / dy;
            l->red_dy = (int)dy;
            l->red_pgrid = (int)((strips * chunks + 7) / 8);
            l->variant = 1;
        }
        const int pblocks = l->red_pgrid > l->red_grid ? l->red_pgrid : l->red_grid;
        // adaptive RK3-4: a second set of partials for the error estimate
        cl_status s = grow_partials(l, pblocks * (l->p.integrator == CL_INT_RK3_4 ? 2 : 1));
        if (s != CL_OK) return s;
        invalidate_graphs(l);
        return CL_OK;
    }
    const int N = l->N, prec = l->p.precision;
    l->VW = scalar_pass_vector_width(prec, N);
    const int TX = N / l->VW;
    // TMA staging needs rows of 16-byte multiples.  Default: as many stages as fit one
    // block per SM in shared memory (loads kept in flight are what the pass needs).
    // The TMA kernel adds a producer warp to the consumer threads; blocks stay <= 512 threads.
    // FP64 passes are bound by GB300's FP64 rate, not by memory: they default to the
    // direct loader, which measured faster for them.
    bool tma = l->opt_stages >= 0 && scalar_pass_tma_ok(prec, N) && scalar_pass_threads(prec, N, 1) <= 480 &&
               !(prec == CL_PREC_FP64 && l->opt_stages == 0);
    // ringless variant (16-byte vectors): at most 448 consumers (blocks of <= 480 threads)
    const bool want_nr = tma && l->opt_variant != 0 && l->VW * l->es == 16;
    const int max_consumers = want_nr ? 448 : (tma ? 480 : 512);
    // Default tile: as many rows as the consumer threads allow (more warps per SM), with
    // three TMA stages; measured best on GB300 for 256^3 and 512^3 lattices.
    int BY = l->opt_BY > 0 ? l->opt_BY : (tma ? max_consumers / TX : (TX >= 256 ? 1 : 256 / TX));
    if (BY > N) BY = N;
    if (BY < 1) BY = 1;
    while (BY > 1 && scalar_pass_threads(prec, N, BY) > max_consumers) --BY;
    int stages = 0;
    // ringless TMA variant: 16-byte vectors only, 2..5 stages
    const int var = want_nr ? 1 : 0;
    if (tma) {
        const int smax = var ? 5 : 6;
        stages = l->opt_stages > 0 ? (l->opt_stages > smax ? smax : l->opt_stages) : (var ? 4 : 3);
        if (l->opt_BY <= 0)
            while (BY > 1 && scalar_pass_smem_bytes(prec, l->nf, N, BY, stages, var) > (size_t)kPassMaxSmem) --BY;
        while (BY > 1 && scalar_pass_smem_bytes(prec, l->nf, N, BY, 2, var) > (size_t)kPassMaxSmem) BY /= 2;
        while (stages > 2 && scalar_pass_smem_bytes(prec, l->nf, N, BY, stages, var) > (size_t)kPassMaxSmem) --stages;
        if (scalar_pass_smem_bytes(prec, l->nf, N, BY, stages, var) > (size_t)kPassMaxSmem) stages = 0;
        // a fifth ringless stage where it fits beside the same tile (one field: measured at
        // 256^3 FP32 + Kahan 0.70 -> 0.75 of HBM for VV-2; two fields at 256^3 do not fit it)
        if (l->opt_stages <= 0 && var && stages == 4 &&
            scalar_pass_smem_bytes(prec, l->nf, N, BY, 5, var) <= (size_t)kPassMaxSmem)
            stages = 5;
    }
    const int var_eff = stages > 0 ? var : 0;
    while (BY > 1 && scalar_pass_smem_bytes(prec, l->nf, N, BY, stages, var_eff) > (size_t)kPassMaxSmem) BY /= 2;
    if (scalar_pass_threads(prec, N, BY) > 512 ||
        scalar_pass_smem_bytes(prec, l->nf, N, BY, stages, var_eff) > (size_t)kPassMaxSmem)
        return fail(l, CL_EINVAL, "lattice too large for the fused pass tiling (N=%d)", N);
    l->variant = var_eff;
    const int nby = (N + BY - 1) / BY;
    l->BY = BY;
    l->stages = stages;
    l->nby = nby;
    // resident blocks of one wave
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
        return fail(l, CL_ECUDA, "cannot query the SM count");
    l->DZ = N;
    l->nbz = 1;
    l->grid = 1;
    cl_status s = query_blocks_per_sm(l, &per_sm);
    if (s != CL_OK) return s;
    if (per_sm < 1) per_sm = 1;
    const int64_t wave = (int64_t)per_sm * nsm;
    int DZ;
    if (l->opt_DZ > 0) {
        DZ = l->opt_DZ > N ? N : l->opt_DZ;  // fixed chunks
    } else if (l->opt_DZ < 0 || (prec == CL_PREC_FP64 && stages == 0)) {
        // balanced persistent ranges over one wave; the default for FP64 direct-load passes,
        // which are bound by the FP64 rate: every SM gets the same share (at 256^3 the lockstep
        // chunks left 48 of 152 SMs with one block instead of two)
        DZ = -1;
    } else {
        // lockstep: every y tile split into the same z chunks, so the blocks of neighbouring
        // tiles march through the same planes together (halo rows hit L2).  The chunk count
        // minimises waves x (planes + 2 halo planes) of the busiest SM: one wave where the
        // tiles allow it (256^3: 37 tiles x 4 chunks), else several evenly filled waves (512^3
        // two-row tiles: 256 x 4 chunks, 6.9 waves, measured 0.80 of HBM against 0.74 with
        // whole-z blocks in 1.7 waves and 0.76 with 8 chunks)
        int64_t best_cost = -1, best_nbz = 1;
        for (int64_t nbz = 1; nbz <= N; ++nbz) {
            const int64_t dz = (N + nbz - 1) / nbz;
            if ((N + dz - 1) / dz != nbz) continue;  // the same chunks as a smaller count
            const int64_t waves = (nby * nbz + wave - 1) / wave;
            const int64_t cost = waves * (dz + 2);
            if (best_cost < 0 || cost < best_cost) {
                best_cost = cost;
                best_nbz = nbz;
            }
        }
        DZ = (int)((N + best_nbz - 1) / best_nbz);
    }
    l->DZ = DZ;
    l->nbz = DZ > 0 ? (N + DZ - 1) / DZ : 1;
    int nblocks = l->nby * l->nbz;
    if (DZ < 0) {
        const int64_t units = (int64_t)nby * N;
        nblocks = (int)(units < wave ? units : wave);
        l->grid = nblocks;
    }
    if (l->gw) {
        // GW pass (direct loads, as the Runge-Kutta stage kernel): about 256 threads per block,
        // two blocks per SM, the y tiles cut into z chunks so that about one wave covers the
        // lattice.  (Measured at 256^3 FP32, two fields, Yoshida-4: 10.5 Gsite-updates/s; a pass
        // with four cp.async plane stages of 2-row tiles, one block per SM, 6.2 with 8 warps and
        // 8.0 with 16: the pass is bound by its latency-exposed arithmetic, not by its loads.)
        int gby = TX >= 256 ? 1 : 256 / TX;
        if (gby > N) gby = N;
        while (gby > 1 && gw_pass_smem(l->nf, N, gby, l->es) > (size_t)kPassMaxSmem / 2) --gby;
        if (gw_pass_smem(l->nf, N, gby, l->es) > (size_t)kPassMaxSmem)
            return fail(l, CL_EINVAL, "lattice too large for the GW pass tiling (N=%d)", N);
        l->gw_BY = gby;
        l->gw_nby = (N + gby - 1) / gby;
        int64_t nbz = (2 * (int64_t)nsm) / l->gw_nby;
        if (nbz < 1) nbz = 1;
        if (nbz > N) nbz = N;
        l->gw_DZ = (int)((N + nbz - 1) / nbz);
        l->gw_nbz = (N + l->gw_DZ - 1) / l->gw_DZ;
    }
    l->rk_stages = 0;
    if (is_rk(l->p.integrator) && l->VW * l->es == 16 && N % l->VW == 0 && l->opt_stages != -1) {
        // TMA-staged Runge-Kutta kernel (the library's choice for 16-byte vectors): up to 448
        // consumer threads, the tallest tile whose stage ring holds three or more stages (the
        // deepest that fits), one block per SM.  Measured at 256^3, two fields, FP32 + Kahan,
        // RK4-5 (persistent ranges): 7 rows x 3 stages 13.8 Gsite-updates/s, 5 x 4 13.5, 4 x 5
        // 12.8; the direct-load kernel 9.7.
        // CL_OPT_TILE_BY / CL_OPT_STAGES / CL_OPT_TILE_DZ override.
        int by_max = 448 / TX < 1 ? 1 : 448 / TX;
        if (by_max > N) by_max = N;
        const bool ricci = l->nmc && l->nf == 1;  // the stage also sums the Ricci terms of its output
        // two sets of partials with the Ricci terms, and for the error estimate of adaptive RK3-4
        const int psets = ricci || l->p.integrator == CL_INT_RK3_4 ? 2 : 1;
        auto fits = [&](int by, int st) { return rk_stage_tma_smem(prec, l->nf, N, by, st, ricci) <= (size_t)kPassMaxSmem; };
        auto most_stages = [&](int by) {  // the deepest ring (3..6) a tile of by rows allows, or 0
            for (int st = 6; st >= 3; --st)
                if (fits(by, st)) return st;
            return 0;
        };
        int best_by = 0, best_s = 0;
        if (l->opt_BY > 0) {  // the given rows (and stages, or the deepest ring)
            const int by = l->opt_BY < by_max ? l->opt_BY : by_max;
            const int want = l->opt_stages > 0 ? (l->opt_stages < 3 ? 3 : l->opt_stages) : 0;
            const int st = want ? (fits(by, want) ? want : 0) : most_stages(by);
            if (st) best_by = by, best_s = st;
        } else if (l->opt_stages > 0) {  // the given stages (at least three), the tallest tile
            const int want = l->opt_stages < 3 ? 3 : l->opt_stages;
            for (int by = by_max; by >= 1 && !best_by; --by)
                if (fits(by, want)) best_by = by, best_s = want;
        } else {  // the tallest tile, with the deepest ring it allows
            for (int by = by_max; by >= 1 && !best_by; --by)
                if (most_stages(by)) best_by = by, best_s = most_stages(by);
        }
        if (best_by) {
            l->rk_stages = best_s;
            l->rk_BY = best_by;
            l->rk_nby = (N + best_by - 1) / best_by;
            if (l->opt_DZ >= 0) {
                // fixed z chunks; by default every y tile cut into the same chunks, one block
                // per SM in one wave, so neighbouring tiles march through the same planes
                // together and their halo rows hit L2 (measured at 256^3, two fields, RK4-5:
                // 14.4 Gsite-updates/s, against 13.7 with balanced persistent ranges)
                int dz = l->opt_DZ;
                if (dz == 0) {
                    int64_t nbz = (int64_t)nsm / l->rk_nby;
                    if (nbz < 1) nbz = 1;
                    if (nbz > N) nbz = N;
                    dz = (int)((N + nbz - 1) / nbz);
                }
                l->rk_DZ = dz > N ? N : dz;
                l->rk_nbz = (N + l->rk_DZ - 1) / l->rk_DZ;
                const int grid = l->rk_nby * l->rk_nbz * psets;
                if (grid > nblocks) nblocks = grid;
            } else {  // balanced persistent ranges over one wave
                const int64_t units = (int64_t)l->rk_nby * N;
                l->rk_DZ = -1;
                l->rk_nbz = (int)(units < nsm ? units : nsm);  // the grid
                if (l->rk_nbz * psets > nblocks) nblocks = l->rk_nbz * psets;
            }
        }
    }
    if (is_rk(l->p.integrator) && l->rk_stages == 0) {
        // Runge-Kutta stage kernel (direct loads): about 256 threads per block, two blocks per
        // SM, the y tiles cut into the same z chunks so that about one wave covers the lattice
        int rby = TX >= 256 ? 1 : 256 / TX;
        if (rby > N) rby = N;
        const size_t es = (size_t)l->es;
        while (rby > 1 && (size_t)l->nf * 3 * (rby + 2) * N * es > (size_t)kPassMaxSmem / 2) --rby;
        l->rk_BY = rby;
        l->rk_nby = (N + rby - 1) / rby;
        int64_t nbz = (2 * (int64_t)nsm) / l->rk_nby;
        if (nbz < 1) nbz = 1;
        if (nbz > N) nbz = N;
        l->rk_DZ = (int)((N + nbz - 1) / nbz);
        l->rk_nbz = (N + l->rk_DZ - 1) / l->rk_DZ;
        const int psets = l->p.integrator == CL_INT_RK3_4 ? 2 : 1;  // error estimate of adaptive RK3-4
        if (l->rk_nby * l->rk_nbz * psets > nblocks) nblocks = l->rk_nby * l->rk_nbz * psets;
    }
    if (l->gauge) {
        // U(1) kernels: 32 x 8 tiles marching through u1_dz planes each; by default the z
        // chunks are cut so that the tiles fill one wave of resident blocks (long marches
        // amortise each block's reduction; measured at 192^3 FP32: 0.29 of HBM with 48-plane
        // chunks in one wave of 4 blocks per SM, 0.21 with 8-plane chunks)
        const int tiles = ((N + 31) / 32) * ((N + 7) / 8);
        // the fused stage only on request: measured slower than the two launches at 192^3
        // (3.96 against 5.12 Gsite-updates/s; both latency-bound)
        l->u1_fused = l->opt_variant == 1 && u1_fused_ok(N) && !is_u1_lf(l);
        // the staged launches (neighbourhoods in shared memory) are the library's choice
        // where the tiles divide N
        l->u1_staged = (l->opt_variant == -1 || l->opt_variant == 2 || l->opt_variant == 3) && u1_staged_ok(N);
        l->u1_sfused = l->u1_staged && l->opt_variant == 3;
        int bps = prec == CL_PREC_FP64 ? kU1BlocksPerSM64 : kU1BlocksPerSM32;
        if (l->u1_fused) {
            CUDA_TRY(l, u1_fused_blocks_per_sm(prec, &bps));
            if (bps < 1) bps = 1;
        }
        int64_t nbz = (int64_t)bps * nsm / tiles;
        if (nbz < 1) nbz = 1;
        if (nbz > N) nbz = N;
        const int auto_dz = l->u1_staged ? u1_staged_dz(prec, N, nsm) : (int)((N + nbz - 1) / nbz);
        l->u1_dz = l->opt_DZ > 0 ? (l->opt_DZ > N ? N : l->opt_DZ) : auto_dz;
        // the gather kernels that run beside the staged launches (the Gauss diagnostic and its
        // plaquette fields) keep the gather form's one-wave chunks
        l->u1_gdz = l->u1_staged ? (int)((N + nbz - 1) / nbz) : l->u1_dz;
        if (2 * u1_grid_blocks(N, l->u1_dz) > nblocks) nblocks = 2 * u1_grid_blocks(N, l->u1_dz);  // stage + plaquette partials
        if (2 * u1_grid_blocks(N, l->u1_gdz) > nblocks) nblocks = 2 * u1_grid_blocks(N, l->u1_gdz);
        if (l->u1_staged && 2 * u1_staged_blocks(prec, N, l->u1_dz) > nblocks)
            nblocks = 2 * u1_staged_blocks(prec, N, l->u1_dz);
    }
    s = grow_partials(l, nblocks);
    if (s != CL_OK) return s;
    invalidate_graphs(l);
    return CL_OK;
}

// Launch one fused pass reading buffer `in` and writing buffer `out`
// (occ != nullptr: only report resident blocks per SM of this configuration).
cl_status run_pass_impl(cl_lattice* l, const PassCoef& pc, int in, int out, int* occ)
{
    const int flags = pc.flags | (l->p.expansion ? P_EXPANSION : 0);
    cudaError_t e;
    if (is_fp64(l)) {
        ScalarPassArgs<double> A{};
        for (int f = 0; f < l->nf; ++f) {
            A.phi_in[f] = (const double*)l->phi[f][in];
            A.pi_in[f] = (const double*)l->pi[f][in];
            A.phi_out[f] = (double*)l->phi[f][out];
            A.pi_out[f] = (double*)l->pi[f][out];
        }
        A.scal = l->scal;
        A.partials = l->partials;
        A.N = l->N; A.BY = l->BY; A.DZ = l->DZ; A.nby = l->nby; A.nbz = l->nbz;
        A.dx = l->dx; A.alpha = l->p.alpha; A.kappa = l->p.kappa;
        A.d = pc.d; A.e = pc.e; A.k = pc.k;
        for (int f = 0; f < 2; ++f) { A.m2[f] = l->m2[f]; A.lam[f] = l->lam[f]; }
        A.g2 = l->g2;
        A.hubble_limit = l->hubble_limit;
        A.flags = flags;
        A.stages = l->stages;
        A.grid = l->grid;
        A.variant = l->variant;
        e = l->dims < 3 ? (occ ? (*occ = 1, cudaSuccess)
                           : l->red_dy > 0 ? launch_plane_pass(l->p.precision, l->nf, &A, l->red_dy, l->red_pd, l->red_pgrid, l->stream)
                                           : launch_reduced_pass(l->p.precision, l->nf, &A, l->dims, l->red_grid, l->stream))
            : occ ? scalar_pass_blocks_per_sm(l->p.precision, l->nf, &A, l->VW, occ)
                  : launch_scalar_pass(l->p.precision, l->nf, &A, l->VW, l->stream);
    } else {
        ScalarPassArgs<float> A{};
        for (int f = 0; f < l->nf; ++f) {
            A.phi_in[f] = (const float*)l->phi[f][in];
            A.pi_in[f] = (const float*)l->pi[f][in];
            A.c_in[f] = (const float*)l->cc[f][in];
            A.phi_out[f] = (float*)l->phi[f][out];
            A.pi_out[f] = (float*)l->pi[f][out];
            A.c_out[f] = (float*)l->cc[f][out];
        }
        A.scal = l->scal;
        A.partials = l->partials;
        A.N = l->N; A.BY = l->BY; A.DZ = l->DZ; A.nby = l->nby; A.nbz = l->nbz;
        A.dx = l->dx; A.alpha = l->p.alpha; A.kappa = l->p.kappa;
        A.d = pc.d; A.e = pc.e; A.k = pc.k;
        for (int f = 0; f < 2; ++f) { A.m2[f] = l->m2[f]; A.lam[f] = l->lam[f]; }
        A.g2 = l->g2;
        A.hubble_limit = l->hubble_limit;
        A.flags = flags;
        A.stages = l->stages;
        A.grid = l->grid;
        A.variant = l->variant;
        e = l->dims < 3 ? (occ ? (*occ = 1, cudaSuccess)
                           : l->red_dy > 0 ? launch_plane_pass(l->p.precision, l->nf, &A, l->red_dy, l->red_pd, l->red_pgrid, l->stream)
                                           : launch_reduced_pass(l->p.precision, l->nf, &A, l->dims, l->red_grid, l->stream))
            : occ ? scalar_pass_blocks_per_sm(l->p.precision, l->nf, &A, l->VW, occ)
                  : launch_scalar_pass(l->p.precision, l->nf, &A, l->VW, l->stream);
    }
    if (e != cudaSuccess) return fail(l, CL_ECUDA, "scalar pass launch failed: %s", cudaGetErrorString(e));
    return CL_OK;
}

// One 2N Runge-Kutta stage reading buffer `in` and writing buffer `out`.
// Blocks of the Ricci reduction (whole x rows each): at most one per row, 8 per SM.
int nmc_grid(const cl_lattice* l)
{
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int64_t g = (int64_t)l->N * l->N;
    if (g > 8 * (int64_t)nsm) g = 8 * (int64_t)nsm;
    return (int)(g < 1 ? 1 : g);
}

// Non-minimal stages that carry the Ricci scalar themselves (TMA-staged stage kernel, one field).
bool nmc_fused(const cl_lattice* l) { return l->nmc && l->nf == 1 && l->rk_stages > 0; }

template <typename T>
cl_status run_rk_stage_t(cl_lattice* l, const PassCoef& pc, int in, int out)
{
    RkStageArgs<T> A{};
    for (int f = 0; f < l->nf; ++f) {
        A.phi_in[f] = (const T*)l->phi[f][in];
        A.pi_in[f] = (const T*)l->pi[f][in];
        A.c_in[f] = (const T*)l->cc[f][in];
        A.kphi_in[f] = (const T*)l->kphi[f][in];
        A.kpi_in[f] = (const T*)l->kpi[f][in];
        A.phi_out[f] = (T*)l->phi[f][out];
        A.pi_out[f] = (T*)l->pi[f][out];
        A.c_out[f] = (T*)l->cc[f][out];
        A.kphi_out[f] = (T*)l->kphi[f][out];
        A.kpi_out[f] = (T*)l->kpi[f][out];
    }
    A.scal = l->scal;
    A.partials = l->partials;
    A.N = l->N; A.BY = l->rk_BY; A.DZ = l->rk_DZ; A.nby = l->rk_nby; A.nbz = l->rk_nbz;
    A.dx = l->dx; A.alpha = l->p.alpha; A.kappa = l->p.kappa;
    A.A = pc.A; A.B = pc.B; A.h = l->p.dt;
    for (int f = 0; f < 2; ++f) { A.m2[f] = l->m2[f]; A.lam[f] = l->lam[f]; }
    A.g2 = l->g2;
    A.hubble_limit = l->hubble_limit;
    A.tol = l->adapt_tol; A.hmin = l->adapt_hmin; A.hmax = l->adapt_hmax;
    A.flags = pc.flags | (l->p.expansion ? P_EXPANSION : 0);
    // with the TMA-staged kernel the stage itself leaves the Ricci scalar of its output state
    // (the next stage's input) in scal->rbar; otherwise a reduction launch precedes each stage
    const bool fused = nmc_fused(l);
    A.nmc = l->nmc ? (fused ? 2 : 1) : 0;
    A.xi = l->xi;
    if (l->nmc && !fused) {  // the Ricci scalar of the stage's state first
        cudaError_t e = launch_nmc_ricci(l->p.precision, &A, nmc_grid(l), l->stream);
        if (e != cudaSuccess) return fail(l, CL_ECUDA, "Ricci reduction launch failed: %s", cudaGetErrorString(e));
    }
    cudaError_t e = l->dims < 3 ? launch_reduced_rk_stage(l->p.precision, l->nf, &A, l->dims, l->red_grid, l->stream)
                    : l->rk_stages > 0 ? launch_rk_stage_tma(l->p.precision, l->nf, &A, l->VW, l->rk_stages, l->stream)
                                       : launch_rk_stage(l->p.precision, l->nf, &A, l->VW, l->stream);
    if (e != cudaSuccess) return fail(l, CL_ECUDA, "Runge-Kutta stage launch failed: %s", cudaGetErrorString(e));
    return CL_OK;
}

cl_status run_u1(cl_lattice* l, int what, double cA, double cB, int flags, int in, int out);
cl_status run_u1_lf(cl_lattice* l, const PassCoef& pc, int s);

// The GW pass of a leapfrog pass with coefficients pc, buffers in -> out.
template <typename T>
cl_status run_gw_pass_t(cl_lattice* l, const PassCoef& pc, int in, int out)
{
    GwPassArgs<T> A{};
    for (int f = 0; f < l->nf; ++f) A.phi_in[f] = (const T*)l->phi[f][out];  // drifted by the scalar pass
    for (int c = 0; c < 5; ++c) {
        A.v_in[c] = (const T*)l->gv[c][in];
        A.pv_in[c] = (const T*)l->gpv[c][in];
        A.v_out[c] = (T*)l->gv[c][out];
        A.pv_out[c] = (T*)l->gpv[c][out];
    }
    A.scal = l->scal;
    A.N = l->N; A.BY = l->gw_BY; A.DZ = l->gw_DZ; A.nby = l->gw_nby; A.nbz = l->gw_nbz;
    A.dx = l->dx; A.alpha = l->p.alpha; A.kappa = l->p.kappa;
    A.d = pc.d; A.k = pc.k;
    A.flags = (pc.flags & P_DRIFT) | (l->p.expansion ? P_EXPANSION : 0);
    cudaError_t e = launch_gw_pass(l->p.precision, l->nf, &A, l->VW, l->stream);
    if (e != cudaSuccess) return fail(l, CL_ECUDA, "GW pass launch failed: %s", cudaGetErrorString(e));
    return CL_OK;
}

// Background Ricci scalar of the current state of a non-minimally coupled lattice into scal->rbar.
template <typename T>
cl_status nmc_ricci_t(cl_lattice* l)
{
    RkStageArgs<T> A{};
    A.phi_in[0] = (const T*)l->phi[0][l->cur];
    A.pi_in[0] = (const T*)l->pi[0][l->cur];
    A.scal = l->scal;
    A.partials = l->partials;
    A.N = l->N;
    A.dx = l->dx; A.alpha = l->p.alpha; A.kappa = l->p.kappa;
    A.m2[0] = l->m2[0]; A.lam[0] = l->lam[0];
    A.nmc = 1;
    A.xi = l->xi;
    cudaError_t e = launch_nmc_ricci(l->p.precision, &A, nmc_grid(l), l->stream);
    if (e != cudaSuccess) return fail(l, CL_ECUDA, "Ricci reduction launch failed: %s", cudaGetErrorString(e));
    return CL_OK;
}

// One ensemble pass over the members [m0, m1) reading buffer `in` and writing `out`.
template <typename T>
cl_status run_ens_pass_t(cl_lattice* l, const PassCoef& pc, int in, int out, int m0, int m1)
{
    EnsPassArgs<T> A{};
    for (int f = 0; f < l->nf; ++f) {
        A.phi_in[f] = (const T*)l->phi[f][in];
        A.pi_in[f] = (const T*)l->pi[f][in];
        A.c_in[f] = (const T*)l->cc[f][in];
        A.phi_out[f] = (T*)l->phi[f][out];
        A.pi_out[f] = (T*)l->pi[f][out];
        A.c_out[f] = (T*)l->cc[f][out];
    }
    A.members = l->d_members;
    A.items = l->d_items;
    A.sched = (m0 == 0 && m1 == l->members) ? l->d_sched : nullptr;  // whole passes: largest items first
    A.scal = l->scal;
    A.partials = l->partials;
    A.item_begin = l->hmem[m0].item0;
    A.item_end = l->hmem[m1 - 1].item0 + l->hmem[m1 - 1].nitems;
    A.alpha = l->p.alpha; A.kappa = l->p.kappa;
    A.d = pc.d; A.e = pc.e; A.k = pc.k;
    A.hubble_limit = l->hubble_limit;
    A.flags = pc.flags | (l->p.expansion ? P_EXPANSION : 0);
    A.stages = l->ens_stages;
    A.stage_stride = l->ens_stage_stride;
    A.ring_slot = l->ens_ring_slot;
    A.variant = l->ens_variant;
    const int n = A.item_end - A.item_begin;
    const int grid = n < l->ens_grid ? n : l->ens_grid;
    cudaError_t e = launch_ensemble_pass(l->p.precision, l->nf, &A, l->VW, grid, l->ens_smem, l->stream);
    if (e != cudaSuccess) return fail(l, CL_ECUDA, "ensemble pass launch failed: %s", cudaGetErrorString(e));
    return CL_OK;
}

cl_status run_ens_pass(cl_lattice* l, const PassCoef& pc, int in, int out, int m0, int m1)
{
    return is_fp64(l) ? run_ens_pass_t<double>(l, pc, in, out, m0, m1) : run_ens_pass_t<float>(l, pc, in, out, m0, m1);
}

cl_status run_pass(cl_lattice* l, const PassCoef& pc, int in, int out)
{
    if (is_ens(l)) return run_ens_pass(l, pc, in, out, 0, l->members);
    if (pc.lf) return run_u1_lf(l, pc, in);                              // axion + U(1) leapfrog pass
    if (pc.rk == 2) return run_u1(l, 1, pc.A, pc.B, pc.flags, in, out);  // axion + U(1) stage
    if (pc.rk) return is_fp64(l) ? run_rk_stage_t<double>(l, pc, in, out) : run_rk_stage_t<float>(l, pc, in, out);
    cl_status s = run_pass_impl(l, pc, in, out, nullptr);
    if (s == CL_OK && l->gw)  // the GW auxiliaries after it, from the scalars it drifted
        s = is_fp64(l) ? run_gw_pass_t<double>(l, pc, in, out) : run_gw_pass_t<float>(l, pc, in, out);
    return s;
}

// Low-storage 2N Runge-Kutta coefficients (A_s, B_s), as published:
// RK3-3: Williamson, J. Comput. Phys. 35 (1980) 48.
// RK4-5: Carpenter & Kennedy, NASA TM-109112 (1994), the five-stage fourth-order scheme.
// RK3-4: the four-stage third-order 2N scheme whose third-stage state is a second-order
//   solution at t + h (c_4 = 1, sum_j a_4j c_j = 1/2) and whose stability function is the
//   degree-4 Taylor polynomial of e^z (b A^3 1 = 1/24); the paper names the scheme without
//   its coefficients, and these seven conditions fix them (one real solution).
void rk_tables(int integrator, std::vector<double>& A, std::vector<double>& B)
{
    if (integrator == CL_INT_RK3_3) {
        A = {0.0, -5.0 / 9.0, -153.0 / 128.0};
        B = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};
    } else if (integrator == CL_INT_RK3_4) {
        A = {0.0, -0.7825460361923582986318837, -2.042914325731224687686953, -1.799337253940777102361562};
        B = {0.06688758201974096587947945, 2.876554598956718963241208, 0.553465736134398241034173,
             0.3912730180961791493159418};
    } else {
        A = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
             -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
        B = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
             1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
             2277821191437.0 / 14882151754819.0};
    }
}

cl_status query_blocks_per_sm(cl_lattice* l, int* per_sm)
{
    return run_pass_impl(l, {0.0, 0.0, 0.0, 0}, 0, 1, per_sm);
}

// Yoshida (1990) fourth-order weights.
// Order of a leapfrog-family integrator (2 for VV-2, 4..10 for the Yoshida compositions).
int leapfrog_order(int integrator)
{
    switch (integrator) {
    case CL_INT_YOSHIDA4: return 4;
    case CL_INT_YOSHIDA6: return 6;
    case CL_INT_YOSHIDA8: return 8;
    case CL_INT_YOSHIDA10: return 10;
    default: return 2;
    }
}

// Time weights of the velocity-Verlet substeps of one step: Yoshida's symmetric triple
// jump (Yoshida 1990, section 4) applied recursively, S_{p+2}(h) = S_p(x1 h) S_p(x0 h) S_p(x1 h)
// with x1 = 1 / (2 - 2^(1/(p+1))) and x0 = 1 - 2 x1, starting from VV-2 (p = 2): 3^((p-2)/2)
// substeps for order p.
void composition_weights(int order, std::vector<double>& w)
{
    w.assign(1, 1.0);
    for (int p = 2; p < order; p += 2) {
        const double c = pow(2.0, 1.0 / (p + 1));
        const double x1 = 1.0 / (2.0 - c), x0 = -c / (2.0 - c);
        std::vector<double> n;
        n.reserve(3 * w.size());
        for (double x : {x1, x0, x1})
            for (double v : w) n.push_back(x * v);
        w.swap(n);
    }
}

// Pass schedule of one time step in staggered form, and the opening half-kick.
std::vector<PassCoef> step_schedule(const cl_lattice* l)
{
    const double h = l->p.dt;
    std::vector<PassCoef> s;
    if (is_u1_lf(l)) {
        // axion-U(1) leapfrog: the second and third evaluations of the implicit kick (the
        // third with the drift), then the closing half-kick of the step merged with the first
        // evaluation of the next step's kick
        PassCoef b{0.0, 0.0, 0.0, 0}, c{0.0, 0.0, 0.0, P_COUNT_STEP}, a{0.0, 0.0, 0.0, 0};
        b.lf = 2; b.lk = 0.5 * h; b.flip = false;
        c.lf = 3; c.lk = 0.5 * h;
        a.lf = 1; a.le = 0.5 * h; a.lk = h; a.lb = h; a.flip = false;
        s = {b, c, a};
        return s;
    }
    if (is_rk(l->p.integrator)) {
        std::vector<double> A, B;
        rk_tables(l->p.integrator, A, B);
        // adaptive RK3-4: every stage takes h from the device, the last one sets the next h
        const int adapt = l->adapt_tol > 0.0 ? P_DEVICE_H : 0;
        for (size_t i = 0; i < A.size(); ++i) {
            PassCoef pc{0.0, 0.0, 0.0, (i == 0 ? P_FIRST_STAGE : 0) | (i + 1 == A.size() ? P_COUNT_STEP : 0) | adapt |
                                           (adapt && i + 1 == A.size() ? P_RK_ERROR : 0)};
            pc.rk = l->gauge ? 2 : 1;
            pc.A = A[i];
            pc.B = B[i];
            s.push_back(pc);
        }
    } else {
        // substep i: drift w_i h; the closing half-kick of substep i merged with the opening
        // half-kick of substep i+1 (of the next step's first substep after the last one)
        std::vector<double> w;
        composition_weights(leapfrog_order(l->p.integrator), w);
        const size_t S = w.size();
        for (size_t i = 0; i < S; ++i) {
            const double wn = i + 1 < S ? w[i + 1] : w[0];
            s.push_back({w[i] * h, 0.5 * w[i] * h, 0.5 * (w[i] + wn) * h,
                         P_DRIFT | P_COMMIT | (i + 1 == S ? P_COUNT_STEP : 0)});
        }
    }
    return s;
}

double open_kick(const cl_lattice* l)
{
    std::vector<double> w;
    composition_weights(leapfrog_order(l->p.integrator), w);
    return 0.5 * w[0] * l->p.dt;
}

cl_status open_leapfrog(cl_lattice* l)
{
    if (l->open) return CL_OK;
    if (is_u1_lf(l)) {  // integer-time momenta kept, the first evaluation of the implicit kick
        PassCoef o{0.0, 0.0, 0.0, 0};
        o.lf = 1; o.le = 0.0; o.lk = 0.5 * l->p.dt; o.lb = 0.5 * l->p.dt;
        cl_status s = run_u1_lf(l, o, l->cur);
        if (s != CL_OK) return s;
        l->open = true;
        l->diag_valid = true;
        return CL_OK;
    }
    const double hk = open_kick(l);
    cl_status s = run_pass(l, {0.0, 0.0, hk, P_COMMIT}, l->cur, l->cur ^ 1);
    if (s != CL_OK) return s;
    l->cur ^= 1;
    l->open = true;
    l->diag_valid = true;
    return CL_OK;
}

// Synchronise the momenta to the integer time.  commit = true makes it the state.
cl_status close_leapfrog(cl_lattice* l, bool commit)
{
    if (!l->open) return CL_OK;
    if (is_u1_lf(l)) {
        // the open state keeps the integer-time momenta (ku1 slots 1, 5..7) and a' of the
        // integer time in the diagnostics: committing copies them into the state
        if (!commit) return CL_OK;
        const size_t bytes = (size_t)l->V * l->es;
        CUDA_TRY(l, cudaMemcpyAsync(l->pi[0][l->cur], l->ku1[1][l->cur], bytes, cudaMemcpyDeviceToDevice, l->stream));
        for (int i = 0; i < 3; ++i)
            CUDA_TRY(l, cudaMemcpyAsync(l->ef[i][l->cur], l->ku1[5 + i][l->cur], bytes, cudaMemcpyDeviceToDevice,
                                        l->stream));
        CUDA_TRY(l, cudaMemcpyAsync(&l->scal->b, &l->scal->diag[D_ADOT], sizeof(double), cudaMemcpyDeviceToDevice,
                                    l->stream));
        l->open = false;
        return CL_OK;
    }
    const double hk = open_kick(l);
    cl_status s = run_pass(l, {0.0, -hk, -hk, commit ? P_COMMIT : 0}, l->cur, l->cur ^ 1);
    if (s != CL_OK) return s;
    if (commit) {
        l->cur ^= 1;
        l->open = false;
    }
    l->diag_valid = true;
    return CL_OK;
}

template <typename T>
void u1_fill(cl_lattice* l, U1Args<T>& A, int in, int out)
{
    A.phi_in = (const T*)l->phi[0][in];
    A.pi_in = (const T*)l->pi[0][in];
    A.phi_out = (T*)l->phi[0][out];
    A.pi_out = (T*)l->pi[0][out];
    for (int i = 0; i < 3; ++i) {
        A.th_in[i] = (const T*)l->th[i][in];
        A.E_in[i] = (const T*)l->ef[i][in];
        A.th_out[i] = (T*)l->th[i][out];
        A.E_out[i] = (T*)l->ef[i][out];
        A.sP[i] = (T*)l->u1s[i];
        A.rP[i] = (T*)l->u1s[3 + i];
        A.Z[i] = (T*)l->u1s[6 + i];
    }
    for (int q = 0; q < 8; ++q) {
        A.k_in[q] = (const T*)l->ku1[q][in];
        A.k_out[q] = (T*)l->ku1[q][out];
    }
    A.scal = l->scal;
    A.partials = l->partials;
    A.N = l->N;
    A.dx = l->dx; A.alpha = l->p.alpha; A.kappa = l->p.kappa;
    A.g = l->alphaL * sqrt(l->p.kappa);
    A.ws2 = l->ws2;
    A.m2 = l->m2[0]; A.lam = l->lam[0];
    A.h = l->p.dt;
    A.hubble_limit = l->hubble_limit;
    A.dz = l->u1_dz;
}

// Component fields of a gauge spectrum (current buffer) as doubles.
template <typename T>
cudaError_t gauge_fields_t(cl_lattice* l, int which, double* out)
{
    GaugeSpecArgs<T> A{};
    for (int i = 0; i < 3; ++i) {
        A.th[i] = (const T*)l->th[i][l->cur];
        A.E[i] = (const T*)(is_u1_lf(l) && l->open ? l->ku1[5 + i][l->cur] : l->ef[i][l->cur]);
    }
    A.N = l->N;
    A.dx = l->dx;
    A.which = which;
    return launch_gauge_fields(l->p.precision, &A, out, l->stream);
}

// U(1) launches on buffer `in` (-> `out`): what = 1 stage (or energies), 2 Gauss diagnostic.
template <typename T>
cl_status run_u1_t(cl_lattice* l, int what, double cA, double cB, int flags, int in, int out)
{
    U1Args<T> A{};
    u1_fill(l, A, in, out);
    if (is_u1_lf(l) && l->open) {  // the integer-time momenta of the open leapfrog
        A.pi_in = (const T*)l->ku1[1][in];
        for (int i = 0; i < 3; ++i) A.E_in[i] = (const T*)l->ku1[5 + i][in];
    }
    A.A = cA;
    A.B = cB;
    A.flags = flags | (l->p.expansion ? P_EXPANSION : 0);
    cudaError_t e;
    // Gauss tracking in the first stage of every step: the staged stage sums it itself; the
    // other forms launch the rms Gauss reduction on the step's starting state (after the
    // plaquette fields of that state, which the fused stage does not write)
    const bool track = what == 1 && (flags & P_FIRST_STAGE) && !(flags & P_ENERGY_ONLY) && !l->u1_staged;
    if (what == 1 && l->u1_fused) {
        e = cudaSuccess;
        if (track) {
            e = launch_u1(l->p.precision, &A, 0, l->stream);
            if (e == cudaSuccess) e = launch_u1(l->p.precision, &A, 3, l->stream);
        }
        if (e == cudaSuccess) e = launch_u1_fused(l->p.precision, &A, l->stream);  // plaquettes and stage in one launch
    } else if (what == 1 && l->u1_sfused) {
        e = launch_u1_staged(l->p.precision, &A, 2, l->stream);  // plaquette fields in shared memory
    } else if (what == 1 && l->u1_staged) {
        e = launch_u1_staged(l->p.precision, &A, 0, l->stream);  // plaquette fields first
        if (e == cudaSuccess) e = launch_u1_staged(l->p.precision, &A, 1, l->stream);
    } else {
        if (l->u1_staged) A.dz = l->u1_gdz;  // gather kernels beside the staged launches
        e = launch_u1(l->p.precision, &A, 0, l->stream);  // plaquette fields first
        if (e == cudaSuccess && track) e = launch_u1(l->p.precision, &A, 3, l->stream);
        if (e == cudaSuccess) e = launch_u1(l->p.precision, &A, what, l->stream);
    }
    if (e != cudaSuccess) return fail(l, CL_ECUDA, "U(1) launch failed: %s", cudaGetErrorString(e));
    return CL_OK;
}

cl_status run_u1(cl_lattice* l, int what, double cA, double cB, int flags, int in, int out)
{
    return is_fp64(l) ? run_u1_t<double>(l, what, cA, cB, flags, in, out)
                      : run_u1_t<float>(l, what, cA, cB, flags, in, out);
}

// One pass of the axion-U(1) leapfrog (U1Args::lf) on the state whose positions are in buffer s:
//   lf 1: the force at the momenta of s; integer-time momenta into ku1[.][s] (slots 1, 5..7),
//         the first iterate of the implicit kick into the momenta of s^1
//   lf 2: the force at the iterate in the momenta of s^1, base ku1[.][s] -> momenta of s; and
//         the rms Gauss violation of the integer-time state (positions of s, momenta ku1[.][s])
//   lf 3: the force at the iterate in the momenta of s, base ku1[.][s] -> momenta of s^1, and
//         the positions drifted with them into s^1
template <typename T>
cl_status run_u1_lf_t(cl_lattice* l, const PassCoef& pc, int s)
{
    // sin P and cos P saved by the previous pass (invalid after any other form's pass, e.g.
    // when the pass variant changed with the leapfrog open)
    const bool pq_saved = l->u1_lf_pq;
    l->u1_lf_pq = false;
    U1Args<T> A{};
    u1_fill(l, A, s, s ^ 1);
    const int pin = pc.lf == 2 ? (s ^ 1) : s;
    const int pout = pc.lf == 2 ? s : (s ^ 1);
    A.pi_in = (const T*)l->pi[0][pin];
    A.pi_out = (T*)l->pi[0][pout];
    for (int i = 0; i < 3; ++i) {
        A.E_in[i] = (const T*)l->ef[i][pin];
        A.E_out[i] = (T*)l->ef[i][pout];
    }
    for (int q = 0; q < 8; ++q) {
        A.k_in[q] = (const T*)l->ku1[q][s];
        A.k_out[q] = (T*)l->ku1[q][s];
    }
    A.lf = pc.lf;
    A.le = pc.le;
    A.lk = pc.lk;
    A.lb = pc.lb;
    A.flags = pc.flags | (l->p.expansion ? P_EXPANSION : 0);
    const int prec = l->p.precision;
    if (l->u1_sfused) {  // one launch: plaquette fields in shared memory, Gauss summed in pass 2
        const cudaError_t ef = launch_u1_staged(prec, &A, 2, l->stream);
        if (ef != cudaSuccess) return fail(l, CL_ECUDA, "U(1) leapfrog launch failed: %s", cudaGetErrorString(ef));
        return CL_OK;
    }
    int pq = 0;  // plaquette launch: 0 full, 3 the E-dependent fields only (staged form)
    if (l->u1_staged) {
        // the three passes of a step evaluate the force at the positions of the previous
        // pass 1: its plaquette launch keeps sin P and cos P in arrays of their own (free
        // auxiliary slots, untouched by the diagnostic launches), so passes 2 and 3 form only
        // cos P dP/dt and the Chern-Simons sums
        for (int i = 0; i < 3; ++i) {
            A.sP[i] = (T*)l->ku1[2 + i][1];
            A.cP[i] = (T*)l->ku1[2 + i][0];
        }
        pq = pc.lf != 1 && pq_saved ? 3 : 0;
    }
    cudaError_t e = l->u1_staged ? launch_u1_staged(prec, &A, pq, l->stream) : launch_u1(prec, &A, 0, l->stream);
    if (e == cudaSuccess && pc.lf == 2 && !l->u1_staged) {
        // Gauss tracking of the step's integer-time starting state (positions of s, the
        // plaquette fields just computed from them, momenta ku1[.][s]); the staged second
        // pass sums it itself
        U1Args<T> G = A;
        G.pi_in = (const T*)l->ku1[1][s];
        for (int i = 0; i < 3; ++i) G.E_in[i] = (const T*)l->ku1[5 + i][s];
        e = launch_u1(prec, &G, 3, l->stream);
    }
    if (e == cudaSuccess) e = l->u1_staged ? launch_u1_staged(prec, &A, 1, l->stream) : launch_u1(prec, &A, 1, l->stream);
    if (e != cudaSuccess) return fail(l, CL_ECUDA, "U(1) leapfrog launch failed: %s", cudaGetErrorString(e));
    l->u1_lf_pq = l->u1_staged && pc.lf != 3;  // pass 3 drifts the positions
    return CL_OK;
}

cl_status run_u1_lf(cl_lattice* l, const PassCoef& pc, int s)
{
    return is_fp64(l) ? run_u1_lf_t<double>(l, pc, s) : run_u1_lf_t<float>(l, pc, s);
}

// sin P and cos P of the open leapfrog's positions (buffer cur) into the slots that the staged
// passes 2 and 3 read, when the pass that should have saved them ran in another form (the pass
// variant changed with the leapfrog open); one plaquette launch, outside any step graph.
template <typename T>
cl_status u1_lf_save_pq_t(cl_lattice* l)
{
    U1Args<T> A{};
    u1_fill(l, A, l->cur, l->cur ^ 1);
    for (int i = 0; i < 3; ++i) {
        A.sP[i] = (T*)l->ku1[2 + i][1];
        A.cP[i] = (T*)l->ku1[2 + i][0];
    }
    A.flags = l->p.expansion ? P_EXPANSION : 0;
    const cudaError_t e = launch_u1_staged(l->p.precision, &A, 0, l->stream);
    if (e != cudaSuccess) return fail(l, CL_ECUDA, "U(1) plaquette launch failed: %s", cudaGetErrorString(e));
    l->u1_lf_pq = true;
    return CL_OK;
}

// Energies of members [m0, m1) of an ensemble only (a' from Eq. Friedmann2 with P_HUBBLE_INIT).
cl_status energy_pass_members(cl_lattice* l, int flags, int m0, int m1)
{
    return run_ens_pass(l, {0.0, 0.0, 0.0, flags}, l->cur, l->cur ^ 1, m0, m1);
}

cl_status energy_pass(cl_lattice* l, int extra_flags)
{
    if (is_u1_lf(l) && l->open) {  // the energy launch reads a closed state
        cl_status c = close_leapfrog(l, true);
        if (c != CL_OK) return c;
    }
    cl_status s = l->gauge ? run_u1(l, 1, 0.0, 0.0, P_ENERGY_ONLY | (extra_flags & P_HUBBLE_INIT), l->cur, l->cur ^ 1)
                           : run_pass(l, {0.0, 0.0, 0.0, extra_flags}, l->cur, l->cur ^ 1);
    if (s != CL_OK) return s;
    if (l->nmc) {  // the background Ricci scalar of the same state
        s = is_fp64(l) ? nmc_ricci_t<double>(l) : nmc_ricci_t<float>(l);
        if (s != CL_OK) return s;
        l->rbar_valid = true;
    }
    l->diag_valid = true;
    return CL_OK;
}

// Copy the scalar state of every member to `host`; report and clear the device status.
cl_status read_status(cl_lattice* l, std::vector<DevScal>& host)
{
    host.resize(l->members);
    CUDA_TRY(l, cudaMemcpyAsync(host.data(), l->scal, sizeof(DevScal) * host.size(), cudaMemcpyDeviceToHost,
                                l->stream));
    CUDA_TRY(l, cudaStreamSynchronize(l->stream));
    int st = 0;
    for (int m = 0; m < l->members; ++m)
        if (host[m].status) {
            st |= host[m].status;
            CUDA_TRY(l, cudaMemsetAsync(&l->scal[m].status, 0, sizeof(int), l->stream));
        }
    if (st) {
        CUDA_TRY(l, cudaStreamSynchronize(l->stream));
        if (st & ST_TIMEOUT) return fail(l, CL_ETIMEOUT, "a bounded device wait gave up (copy pipeline)");
        if (st & ST_NAN) return fail(l, CL_ENAN, "a volume-averaged energy became non-finite");
        if (st & ST_CONSTRAINT) return fail(l, CL_ECONSTRAINT, "Hubble-constraint violation above %g", l->hubble_limit);
    }
    return CL_OK;
}

// 0 = scalar field f, 1 = its momentum, 2 = link angle theta_f, 3 = electric field E_f.
int field_kind(const cl_lattice* l, int field, int* f)
{
    if (l->gw && field >= CL_FIELD_GW_V11 && field <= CL_FIELD_GW_V23) {
        *f = field - CL_FIELD_GW_V11;
        return 4;
    }
    if (l->gw && field >= CL_FIELD_GW_P11 && field <= CL_FIELD_GW_P23) {
        *f = field - CL_FIELD_GW_P11;
        return 5;
    }
    if (field == CL_FIELD_PHI0 || field == CL_FIELD_PHI1) {
        *f = field - CL_FIELD_PHI0;
        return *f < l->nf ? 0 : -1;
    }
    if (field == CL_FIELD_PI0 || field == CL_FIELD_PI1) {
        *f = field - CL_FIELD_PI0;
        return *f < l->nf ? 1 : -1;
    }
    if (l->gauge && field >= CL_FIELD_THETA1 && field <= CL_FIELD_THETA3) {
        *f = field - CL_FIELD_THETA1;
        return 2;
    }
    if (l->gauge && field >= CL_FIELD_E1 && field <= CL_FIELD_E3) {
        *f = field - CL_FIELD_E1;
        return 3;
    }
    return -1;
}

void* field_buffer(cl_lattice* l, int kind, int f, int buf)
{
    switch (kind) {
    case 0: return l->phi[f][buf];
    case 1: return l->pi[f][buf];
    case 2: return l->th[f][buf];
    case 4: return l->gv[f][buf];
    case 5: return l->gpv[f][buf];
    default: return l->ef[f][buf];
    }
}

}  // namespace

extern "C" {

const char* cl_strerror(cl_status s)
{
    switch (s) {
    case CL_OK: return "ok";
    case CL_EINVAL: return "invalid argument";
    case CL_ENOMEM: return "out of memory";
    case CL_ECUDA: return "CUDA error";
    case CL_ENAN: return "non-finite energy";
    case CL_ECONSTRAINT: return "constraint violation above limit";
    case CL_ETIMEOUT: return "device wait timed out";
    case CL_ESTATE: return "call not valid in this state";
    case CL_EUNSUPPORTED: return "not supported by this build";
    }
    return "unknown status";
}

const char* cl_last_error(const cl_lattice* l) { return l ? l->err : "null handle"; }

int64_t cl_last_launch_count(const cl_lattice* l) { return l ? l->last_launches : 0; }

void cl_free(cl_lattice* l)
{
    if (!l) return;
    if (l->stream) cudaStreamSynchronize(l->stream);
    invalidate_graphs(l);
    for (int f = 0; f < 2; ++f)
        for (int b = 0; b < 2; ++b) {
            if (l->phi[f][b]) cudaFree(l->phi[f][b]);
            if (l->pi[f][b]) cudaFree(l->pi[f][b]);
            if (l->cc[f][b]) cudaFree(l->cc[f][b]);
            if (l->kphi[f][b]) cudaFree(l->kphi[f][b]);
            if (l->kpi[f][b]) cudaFree(l->kpi[f][b]);
        }
    for (int b = 0; b < 2; ++b) {
        for (int i = 0; i < 3; ++i) {
            if (l->th[i][b]) cudaFree(l->th[i][b]);
            if (l->ef[i][b]) cudaFree(l->ef[i][b]);
        }
        for (int q = 0; q < 8; ++q)
            if (l->ku1[q][b]) cudaFree(l->ku1[q][b]);
        for (int c = 0; c < 5; ++c) {
            if (l->gv[c][b]) cudaFree(l->gv[c][b]);
            if (l->gpv[c][b]) cudaFree(l->gpv[c][b]);
        }
    }
    for (int q = 0; q < 9; ++q)
        if (l->u1s[q]) cudaFree(l->u1s[q]);
    if (l->scal) cudaFree(l->scal);
    if (l->partials) cudaFree(l->partials);
    if (l->sg_buf) cudaFree(l->sg_buf);
    if (l->d_members) cudaFree(l->d_members);
    if (l->d_items) cudaFree(l->d_items);
    if (l->d_sched) cudaFree(l->d_sched);
    if (l->own_stream && l->stream) cudaStreamDestroy(l->stream);
    delete l;
}

cl_status cl_init_lattice(cl_lattice** out, const cl_lattice_params* p)
{
    if (!out) return CL_EINVAL;
    *out = nullptr;
    if (!p) return CL_EINVAL;
    const bool ens = p->members > 1;
    if (ens) {
        // batched ensemble of independent lattices: leapfrog schemes, scalar fields only
        if (p->members > kMaxMembers || !p->member_N) return CL_EINVAL;
        if (p->gauge != CL_GAUGE_NONE || is_rk(p->integrator)) return CL_EUNSUPPORTED;
        for (int m = 0; m < p->members; ++m) {
            if (p->member_N[m] < 2 || p->member_N[m] > kEnsMaxN) return CL_EINVAL;
            if (p->member_L && !(p->member_L[m] > 0)) return CL_EINVAL;
        }
    }
    if (p->members < 0) return CL_EINVAL;
    // largest N: 32-bit site indices for N^3 lattices; N^2 < 2^31 on the (2+1) lattice
    const int dims_in = (p->dims == 1 || p->dims == 2) ? p->dims : 3;
    const long long max_n = dims_in == 3 ? kMaxN : (dims_in == 2 ? 46340 : (1ll << 30));
    if ((!ens && (p->N < 2 || p->N > max_n)) || p->nfields < 1 || p->nfields > 2 || p->precision < 0 || p->precision > 2 ||
        p->integrator < 0 || p->integrator > CL_INT_RK3_4 || p->gauge < 0 || p->gauge > 1 || !(p->L > 0) || !(p->dt > 0) ||
        !(p->a0 > 0) || p->dims < 0 || p->dims > 3)
        return CL_EINVAL;
    // reduced (d+1)-dimensional lattices: single lattices of scalar fields
    if (p->dims == 1 || p->dims == 2) {
        if (ens || p->gauge != CL_GAUGE_NONE) return CL_EUNSUPPORTED;
    }
    if (p->gauge == CL_GAUGE_U1_AXION) {
        // the paper integrates the axion-gauge module with Runge-Kutta; one axion field;
        // fields stored in FP64 or plain FP32
        if (p->nfields != 1) return CL_EINVAL;
        // the Runge-Kutta schemes, or the leapfrog with an implicit momentum kick (order 2)
        if ((!is_rk(p->integrator) && p->integrator != CL_INT_VV2) || p->precision == CL_PREC_FP32_KAHAN)
            return CL_EUNSUPPORTED;
    }
    cl_lattice* l = new (std::nothrow) cl_lattice();
    if (!l) return CL_ENOMEM;
    l->p = *p;
    l->p.member_N = nullptr;
    l->p.member_L = nullptr;
    l->nf = p->nfields;
    l->es = p->precision == CL_PREC_FP64 ? 8 : 4;
    l->dims = (p->dims == 1 || p->dims == 2) ? p->dims : 3;
    if (ens) {
        // members back to back in every arena, each on a 256-byte boundary; one vector
        // width for all members (the widest that divides every size)
        const int B = p->members;
        l->members = B;
        l->mN.assign(p->member_N, p->member_N + B);
        l->mL.resize(B);
        l->moff.resize(B);
        l->mpot.assign(5 * (size_t)B, 0.0);
        const int64_t align = 256 / l->es;
        int64_t off = 0;
        int vw = p->precision == CL_PREC_FP64 ? 2 : 4, nmax = 0;
        for (int m = 0; m < B; ++m) {
            const int n = l->mN[m];
            l->mL[m] = p->member_L ? p->member_L[m] : p->L;
            l->moff[m] = off;
            off += ((int64_t)n * n * n + align - 1) / align * align;
            while (n % vw) vw /= 2;
            if (n > nmax) nmax = n;
        }
        for (int m = 0; m < B; ++m)
            if (l->mN[m] / vw > kEnsThreads) {
                delete l;
                return CL_EINVAL;
            }
        l->VW = vw;
        l->N = nmax;
        l->V = off;
        l->dx = l->mL[0] / l->mN[0];
    } else {
        l->N = p->N;
        l->V = l->dims == 1 ? (int64_t)p->N : (l->dims == 2 ? (int64_t)p->N * p->N : (int64_t)p->N * p->N * p->N);
        l->dx = p->L / p->N;
    }
    if (p->stream) {
        l->stream = (cudaStream_t)p->stream;
    } else {
        // a blocking stream: ordered with the legacy default stream, and capturable
        if (cudaStreamCreate(&l->stream) != cudaSuccess) {
            delete l;
            return CL_ECUDA;
        }
        l->own_stream = true;
    }
    const size_t bytes = (size_t)l->V * l->es;
    for (int f = 0; f < l->nf; ++f)
        for (int b = 0; b < 2; ++b) {
            if (cudaMalloc(&l->phi[f][b], bytes) != cudaSuccess || cudaMalloc(&l->pi[f][b], bytes) != cudaSuccess ||
                (has_kahan(l) && cudaMalloc(&l->cc[f][b], bytes) != cudaSuccess) ||
                (is_rk(p->integrator) && (cudaMalloc(&l->kphi[f][b], bytes) != cudaSuccess ||
                                          cudaMalloc(&l->kpi[f][b], bytes) != cudaSuccess))) {
                cl_free(l);
                return CL_ENOMEM;
            }
            cudaMemsetAsync(l->phi[f][b], 0, bytes, l->stream);
            cudaMemsetAsync(l->pi[f][b], 0, bytes, l->stream);
            if (has_kahan(l)) cudaMemsetAsync(l->cc[f][b], 0, bytes, l->stream);
        }
    if (p->gauge == CL_GAUGE_U1_AXION) {
        l->gauge = true;
        bool ok = true;
        for (int b = 0; b < 2 && ok; ++b) {
            for (int i = 0; i < 3 && ok; ++i) {
                ok = cudaMalloc(&l->th[i][b], bytes) == cudaSuccess && cudaMalloc(&l->ef[i][b], bytes) == cudaSuccess;
                if (ok) {
                    cudaMemsetAsync(l->th[i][b], 0, bytes, l->stream);
                    cudaMemsetAsync(l->ef[i][b], 0, bytes, l->stream);
                }
            }
            for (int q = 0; q < 8 && ok; ++q) ok = cudaMalloc(&l->ku1[q][b], bytes) == cudaSuccess;
        }
        for (int q = 0; q < 9 && ok; ++q) ok = cudaMalloc(&l->u1s[q], bytes) == cudaSuccess;
        if (!ok) {
            cl_free(l);
            return CL_ENOMEM;
        }
    }
    if (cudaMalloc(&l->scal, sizeof(DevScal) * l->members) != cudaSuccess) {
        cl_free(l);
        return CL_ENOMEM;
    }
    std::vector<DevScal> h(l->members, DevScal{});
    for (auto& x : h) {
        x.a = p->a0;
        x.h = p->dt;
    }
    cudaMemcpyAsync(l->scal, h.data(), sizeof(DevScal) * h.size(), cudaMemcpyHostToDevice, l->stream);
    const cl_status ts = choose_tiles(l);
    if (ts != CL_OK) {
        cl_free(l);
        return ts == CL_EINVAL ? CL_EINVAL : CL_ENOMEM;
    }
    if (cudaStreamSynchronize(l->stream) != cudaSuccess) {
        cl_free(l);
        return CL_ECUDA;
    }
    *out = l;
    return CL_OK;
}

cl_status cl_set_potential(cl_lattice* l, int32_t kind, const double* params, int32_t nparams)
{
    if (!l) return CL_EINVAL;
    if (!params) return fail(l, CL_EINVAL, "params is NULL");
    int per = 0;  // values per member
    switch (kind) {
    case CL_POT_LPHI4: case CL_POT_M2: per = 1; break;
    case CL_POT_M2_G2: case CL_POT_LPHI4_G2: per = 2; break;
    case CL_POT_POLY: per = 5; break;
    default: return fail(l, CL_EINVAL, "unknown potential kind %d", kind);
    }
    if (nparams != per && !(is_ens(l) && nparams == per * l->members))
        return fail(l, CL_EINVAL, "potential kind %d takes %d values (per member for an ensemble)", kind, per);
    if ((kind == CL_POT_M2_G2 || kind == CL_POT_LPHI4_G2) && l->nf != 2)
        return fail(l, CL_EINVAL, "this potential needs two fields");
    std::vector<double> pot(5 * (size_t)l->members, 0.0);
    for (int m = 0; m < l->members; ++m) {
        const double* q = params + (nparams == per ? 0 : (size_t)per * m);
        double* c = &pot[5 * (size_t)m];  // m2_0, lam_0, m2_1, lam_1, g2
        switch (kind) {
        case CL_POT_LPHI4: c[1] = q[0]; break;
        case CL_POT_M2: c[0] = q[0]; break;
        case CL_POT_M2_G2: c[0] = q[0]; c[4] = q[1]; break;
        case CL_POT_LPHI4_G2: c[1] = q[0]; c[4] = q[1]; break;
        default: for (int i = 0; i < 5; ++i) c[i] = q[i]; break;
        }
        for (int i = 0; i < 5; ++i)
            if (!isfinite(c[i])) return fail(l, CL_EINVAL, "non-finite coupling");
        if (l->nf == 1 && (c[2] != 0 || c[3] != 0 || c[4] != 0))
            return fail(l, CL_EINVAL, "second-field couplings on a one-field lattice");
    }
    l->m2[0] = pot[0]; l->lam[0] = pot[1]; l->m2[1] = pot[2]; l->lam[1] = pot[3]; l->g2 = pot[4];
    if (is_ens(l)) {
        l->mpot = pot;
        cl_status s = upload_members(l);
        if (s != CL_OK) return s;
    }
    l->potential_set = true;
    l->diag_valid = false;
    l->rbar_valid = false;
    invalidate_graphs(l);
    return CL_OK;
}

cl_status cl_set_state(cl_lattice* l, int32_t member, int32_t field, const void* src, int32_t on_device)
{
    if (!l) return CL_EINVAL;
    if (!is_ens(l) && member == -1) member = 0;
    if (!member_ok(l, member)) return fail(l, CL_EINVAL, "member %d out of range", member);
    if (!src) return fail(l, CL_EINVAL, "src is NULL");
    int f = 0;
    const int kind = field_kind(l, field, &f);
    if (kind < 0) return fail(l, CL_EINVAL, "field %d not present", field);
    cl_status s = close_leapfrog(l, true);
    if (s != CL_OK) return s;
    const size_t bytes = (size_t)mem_V(l, member) * l->es, off = mem_off_bytes(l, member);
    void* dst = (char*)field_buffer(l, kind, f, l->cur) + off;
    CUDA_TRY(l, cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                l->stream));
    if (kind == 0 && has_kahan(l)) CUDA_TRY(l, cudaMemsetAsync((char*)l->cc[f][l->cur] + off, 0, bytes, l->stream));
    if (!on_device) CUDA_TRY(l, cudaStreamSynchronize(l->stream));
    l->diag_valid = false;
    l->rbar_valid = false;
    return CL_OK;
}

cl_status cl_get_state(cl_lattice* l, int32_t member, int32_t field, void* dst, int32_t on_device)
{
    if (!l) return CL_EINVAL;
    if (!member_ok(l, member)) return fail(l, CL_EINVAL, "member %d out of range", member);
    if (!dst) return fail(l, CL_EINVAL, "dst is NULL");
    int f = 0;
    const int kind = field_kind(l, field, &f);
    if (kind < 0) return fail(l, CL_EINVAL, "field %d not present", field);
    int buf = l->cur;
    const void* fb = nullptr;
    if (l->open && is_u1_lf(l)) {  // the open axion-U(1) leapfrog keeps the integer-time momenta
        if (kind == 1) fb = l->ku1[1][l->cur];
        else if (kind == 3) fb = l->ku1[5 + f][l->cur];
    } else if (l->open && (kind == 1 || kind == 5)) {
        cl_status s = close_leapfrog(l, false);  // integer-time momenta into the spare buffer
        if (s != CL_OK) return s;
        buf = l->cur ^ 1;
    }
    if (!fb) fb = field_buffer(l, kind, f, buf);
    const size_t bytes = (size_t)mem_V(l, member) * l->es;
    const void* srcp = (const char*)fb + mem_off_bytes(l, member);
    CUDA_TRY(l, cudaMemcpyAsync(dst, srcp, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                l->stream));
    std::vector<DevScal> h;
    return read_status(l, h);
}

cl_status cl_set_scalars(cl_lattice* l, int32_t member, double a, double adot, double t)
{
    if (!l) return CL_EINVAL;
    if (member != -1 && !member_ok(l, member)) return fail(l, CL_EINVAL, "member %d out of range", member);
    if (!(a > 0) || !isfinite(a)) return fail(l, CL_EINVAL, "a must be positive");
    cl_status s = close_leapfrog(l, true);
    if (s != CL_OK) return s;
    std::vector<DevScal> h;
    s = read_status(l, h);
    if (s != CL_OK) return s;
    const int m0 = member < 0 ? 0 : member, m1 = member < 0 ? l->members : member + 1;
    for (int m = m0; m < m1; ++m) {
        h[m].a = a;
        h[m].b = isnan(adot) ? 0.0 : adot;
        h[m].t = t;
        h[m].gauss[0] = h[m].gauss[1] = 0.0;  // Gauss tracking restarts with the new state
    }
    CUDA_TRY(l, cudaMemcpyAsync(l->scal, h.data(), sizeof(DevScal) * h.size(), cudaMemcpyHostToDevice, l->stream));
    CUDA_TRY(l, cudaStreamSynchronize(l->stream));
    l->diag_valid = false;
    l->rbar_valid = false;
    if (isnan(adot) && l->p.expansion) {
        if (is_ens(l) && member >= 0) return energy_pass_members(l, P_HUBBLE_INIT | P_COMMIT, m0, m1);
        return energy_pass(l, P_HUBBLE_INIT | P_COMMIT);
    }
    return CL_OK;
}

cl_status cl_get_scalars(cl_lattice* l, int32_t member, double* a, double* adot, double* t)
{
    if (!l) return CL_EINVAL;
    if (!member_ok(l, member)) return fail(l, CL_EINVAL, "member %d out of range", member);
    if (l->open && !is_u1_lf(l)) {
        cl_status s = close_leapfrog(l, false);
        if (s != CL_OK) return s;
    } else if (!l->diag_valid) {
        cl_status s = energy_pass(l, 0);
        if (s != CL_OK) return s;
    }
    std::vector<DevScal> h;
    cl_status s = read_status(l, h);
    if (s != CL_OK) return s;
    if (a) *a = h[member].diag[D_A];
    if (adot) *adot = h[member].diag[D_ADOT];
    if (t) *t = h[member].diag[D_T];
    return CL_OK;
}

cl_status cl_set_gauge_coupling(cl_lattice* l, double alphaL, double ws2)
{
    if (!l) return CL_EINVAL;
    if (!l->gauge) return fail(l, CL_EINVAL, "the lattice has no gauge field");
    if (!isfinite(alphaL) || !isfinite(ws2) || ws2 < 0) return fail(l, CL_EINVAL, "bad gauge coupling");
    l->alphaL = alphaL;
    l->ws2 = ws2;
    l->diag_valid = false;
    l->rbar_valid = false;
    invalidate_graphs(l);
    return CL_OK;
}

cl_status cl_set_nonminimal(cl_lattice* l, double xi)
{
    if (!l) return CL_EINVAL;
    if (l->dims < 3) return fail(l, CL_EUNSUPPORTED, "the non-minimal coupling is not available on a reduced (1+1)/(2+1) lattice");
    if (is_ens(l) || l->gauge || l->nf != 1 || !is_rk(l->p.integrator))
        return fail(l, CL_EUNSUPPORTED, "the non-minimal coupling needs one scalar field and a Runge-Kutta integrator");
    if (l->adapt_tol > 0.0)
        return fail(l, CL_EUNSUPPORTED, "the non-minimal coupling is not available with adaptive steps");
    if (!isfinite(xi)) return fail(l, CL_EINVAL, "xi must be finite");
    cl_status s = grow_partials(l, nmc_grid(l));
    if (s != CL_OK) return s;
    l->nmc = true;
    l->xi = xi;
    l->diag_valid = false;
    l->rbar_valid = false;
    invalidate_graphs(l);
    return choose_tiles(l);  // the stage kernel's buffers grow by the rows of the Ricci terms
}

cl_status cl_set_adaptive(cl_lattice* l, double tol, double h_min, double h_max)
{
    if (!l) return CL_EINVAL;
    if (l->p.integrator != CL_INT_RK3_4 || is_ens(l) || l->gauge || l->nmc)
        return fail(l, CL_EUNSUPPORTED, "adaptive steps need a single scalar lattice integrated with RK3-4 "
                                        "(no gauge field, no non-minimal coupling)");
    if (!isfinite(tol) || !isfinite(h_min) || !isfinite(h_max))
        return fail(l, CL_EINVAL, "tolerance and step bounds must be finite");
    const bool on = tol > 0.0;
    if (on && (!(h_max > 0.0) || h_min < 0.0 || h_min > h_max))
        return fail(l, CL_EINVAL, "need 0 <= h_min <= h_max and h_max > 0");
    std::vector<DevScal> h;
    cl_status s = read_status(l, h);
    if (s != CL_OK) return s;
    if (on && !(l->adapt_tol > 0.0)) {  // start from the lattice's dt (within the bounds)
        double h0 = l->p.dt;
        h0 = h0 > h_max ? h_max : (h0 < h_min ? h_min : h0);
        h[0].h = h0;
        h[0].rk_err = 0.0;
        CUDA_TRY(l, cudaMemcpyAsync(l->scal, h.data(), sizeof(DevScal), cudaMemcpyHostToDevice, l->stream));
        CUDA_TRY(l, cudaStreamSynchronize(l->stream));
    }
    l->adapt_tol = on ? tol : 0.0;
    l->adapt_hmin = on ? h_min : 0.0;
    l->adapt_hmax = on ? h_max : 0.0;
    invalidate_graphs(l);  // the stage flags change
    return CL_OK;
}

cl_status cl_enable_gw(cl_lattice* l)
{
    if (!l) return CL_EINVAL;
    if (l->dims < 3) return fail(l, CL_EUNSUPPORTED, "the GW sector is not available on a reduced (1+1)/(2+1) lattice");
    if (is_ens(l) || l->gauge || is_rk(l->p.integrator))
        return fail(l, CL_EUNSUPPORTED, "gravitational waves need a single scalar lattice with a leapfrog integrator");
    if (l->gw) return CL_OK;
    cl_status s = close_leapfrog(l, true);
    if (s != CL_OK) return s;
    const size_t bytes = (size_t)l->N * l->N * l->N * l->es;
    for (int c = 0; c < 5; ++c)
        for (int b = 0; b < 2; ++b) {
            if (cudaMalloc(&l->gv[c][b], bytes) != cudaSuccess || cudaMalloc(&l->gpv[c][b], bytes) != cudaSuccess)
                return fail(l, CL_ENOMEM, "GW field allocation failed");
            CUDA_TRY(l, cudaMemsetAsync(l->gv[c][b], 0, bytes, l->stream));
            CUDA_TRY(l, cudaMemsetAsync(l->gpv[c][b], 0, bytes, l->stream));
        }
    l->gw = true;
    s = choose_tiles(l);
    if (s != CL_OK) return s;
    CUDA_TRY(l, cudaStreamSynchronize(l->stream));
    invalidate_graphs(l);
    return CL_OK;
}

cl_status cl_gw_spectrum(cl_lattice* l, double dn, int32_t type, double* k_out, double* delta_out, double* count_out,
                         int32_t cap, int32_t* nbins)
{
    if (!l) return CL_EINVAL;
    if (!l->gw) return fail(l, CL_EINVAL, "gravitational waves are not enabled (cl_enable_gw)");
    if (!(dn > 0) || (type != 1 && type != 2) || cap < 0 || (cap > 0 && (!k_out || !delta_out || !count_out)))
        return fail(l, CL_EINVAL, "GW spectrum: bad arguments");
    const int N = l->N;
    const int64_t V = (int64_t)N * N * N;
    const int nb = (int)floor(sqrt(3.0) * (N / 2) / dn + 0.5) + 1;
    if (nbins) *nbins = nb;
    if (cap == 0) return CL_OK;
    int buf = l->cur;
    if (l->open) {  // integer-time momenta (and a) into the spare buffer / diagnostics
        cl_status s = close_leapfrog(l, false);
        if (s != CL_OK) return s;
        buf = l->cur ^ 1;
    }
    std::vector<DevScal> hs;
    cl_status st = read_status(l, hs);
    if (st != CL_OK) return st;
    const double a = hs[0].a;  // a at the integer time (the staggered form keeps a there)
    const size_t nh = (size_t)N * N * (N / 2 + 1);
    double* real = nullptr;
    double2* F = nullptr;
    double* bins = nullptr;  // S[nb], C[nb], k[nb], delta[nb]
    cufftHandle plan = 0;
    if (cudaMalloc(&real, (size_t)V * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&F, 5 * nh * sizeof(double2)) != cudaSuccess || cudaMalloc(&bins, 4 * (size_t)nb * sizeof(double)) != cudaSuccess)
        st = fail(l, CL_ENOMEM, "GW spectrum scratch allocation failed");
    if (st == CL_OK && cufftPlan3d(&plan, N, N, N, CUFFT_D2Z) != CUFFT_SUCCESS) st = fail(l, CL_ECUDA, "cufftPlan3d failed");
    if (st == CL_OK && cufftSetStream(plan, l->stream) != CUFFT_SUCCESS) st = fail(l, CL_ECUDA, "cufftSetStream failed");
    for (int c = 0; c < 5 && st == CL_OK; ++c) {
        // h' = a^(alpha-3) pi_v: the factor is applied to the binned sums below
        if (launch_field_to_double(l->p.precision, l->gpv[c][buf], real, V, l->stream) != cudaSuccess)
            st = fail(l, CL_ECUDA, "field conversion failed");
        else if (cufftExecD2Z(plan, real, (cufftDoubleComplex*)(F + c * nh)) != CUFFT_SUCCESS)
            st = fail(l, CL_ECUDA, "D2Z failed");
    }
    if (st == CL_OK && cudaMemsetAsync(bins, 0, 2 * (size_t)nb * sizeof(double), l->stream) != cudaSuccess)
        st = fail(l, CL_ECUDA, "memset failed");
    if (st == CL_OK && launch_gw_bins(F, N, l->dx, dn, nb, bins, bins + nb, l->stream) != cudaSuccess)
        st = fail(l, CL_ECUDA, "binning failed");
    if (st == CL_OK &&
        launch_spectrum_finish(bins, bins + nb, N, l->p.L, dn, type, nb, bins + 2 * nb, bins + 3 * nb, l->stream) != cudaSuccess)
        st = fail(l, CL_ECUDA, "spectrum finish failed");
    std::vector<double> h(4 * (size_t)nb);
    if (st == CL_OK && cudaMemcpyAsync(h.data(), bins, 4 * (size_t)nb * sizeof(double), cudaMemcpyDeviceToHost, l->stream) != cudaSuccess)
        st = fail(l, CL_ECUDA, "copy failed");
    if (st == CL_OK && cudaStreamSynchronize(l->stream) != cudaSuccess) st = fail(l, CL_ECUDA, "sync failed");
    if (st == CL_OK) {
        // |h'|^2 = a^(2(alpha-3)) |pi_v|^2, times 1 / (4 kappa a^(2 alpha))
        const double ca = pow(a, 2.0 * (l->p.alpha - 3.0)) / (4.0 * l->p.kappa * pow(a, 2.0 * l->p.alpha));
        const int n = cap < nb ? cap : nb;
        for (int i = 0; i < n; ++i) {
            count_out[i] = h[nb + i];
            k_out[i] = h[2 * nb + i];
            delta_out[i] = ca * h[3 * nb + i];
        }
    }
    if (plan) cufftDestroy(plan);
    if (real) cudaFree(real);
    if (F) cudaFree(F);
    if (bins) cudaFree(bins);
    return st;
}

cl_status cl_set_hubble_limit(cl_lattice* l, double limit)
{
    if (!l) return CL_EINVAL;
    l->hubble_limit = limit;
    invalidate_graphs(l);
    return CL_OK;
}

cl_status cl_get_option(cl_lattice* l, int32_t option, int64_t* value)
{
    if (!l || !value) return CL_EINVAL;
    const bool ens = is_ens(l);
    switch (option) {
    case CL_OPT_GRAPH: *value = l->use_graph ? 1 : 0; return CL_OK;
    case CL_OPT_TILE_BY: *value = ens ? l->hmem[0].BY : (is_rk(l->p.integrator) && !l->gauge ? l->rk_BY : l->BY); return CL_OK;
    case CL_OPT_TILE_DZ:
        *value = ens ? l->hmem[0].DZ
                     : (l->gauge ? l->u1_dz : (l->dims < 3 ? l->red_dy : (is_rk(l->p.integrator) ? l->rk_DZ : l->DZ)));
        return CL_OK;
    case CL_OPT_STAGES:
        *value = ens ? l->ens_stages : (is_rk(l->p.integrator) && !l->gauge ? (l->rk_stages > 0 ? l->rk_stages : -1) : l->stages);
        return CL_OK;
    case CL_OPT_PASS_VARIANT:
        *value = ens ? l->ens_variant : (l->gauge ? (l->u1_fused ? 1 : (l->u1_sfused ? 3 : (l->u1_staged ? 2 : 0))) : l->variant);
        return CL_OK;
    }
    return fail(l, CL_EINVAL, "unknown option %d", option);
}

cl_status cl_set_option(cl_lattice* l, int32_t option, int64_t value)
{
    if (!l) return CL_EINVAL;
    switch (option) {
    case CL_OPT_GRAPH: l->use_graph = value != 0; return CL_OK;
    case CL_OPT_TILE_BY:
        if (value < 0 || value > l->N) return fail(l, CL_EINVAL, "tile BY out of range");
        l->opt_BY = (int)value;
        return choose_tiles(l);
    case CL_OPT_TILE_DZ:
        if (value < -1 || value > l->N) return fail(l, CL_EINVAL, "tile DZ out of range");
        l->opt_DZ = (int)value;
        return choose_tiles(l);
    case CL_OPT_PASS_VARIANT:
        if (value < -1 || value > (l->gauge ? 3 : 1))
            return fail(l, CL_EINVAL, "pass variant must be -1, 0 or 1 (2, 3 on an axion-U(1) lattice)");
        if (value == 1 && is_u1_lf(l))
            return fail(l, CL_EUNSUPPORTED, "the axion-U(1) leapfrog has no fused pass form");
        l->opt_variant = (int)value;
        return choose_tiles(l);
    case CL_OPT_STAGES:
        if (value < -1 || value == 1 || value > 6) return fail(l, CL_EINVAL, "stages must be -1, 0 or 2..6");
        l->opt_stages = (int)value;
        return choose_tiles(l);
    }
    return fail(l, CL_EINVAL, "unknown option %d", option);
}

// ---------------------------------------------------------------- autotuner
// The tiling in effect (after the library's own choices for the 0 = "library choice" values
// a candidate may carry) and the time per trial pass, into best[5].
static void report_tiles(const cl_lattice* l, double us, double* best)
{
    if (!best) return;
    const bool ens = is_ens(l);
    best[0] = ens ? l->ens_stages : l->stages;
    best[1] = ens ? l->hmem[0].BY : l->BY;
    best[2] = ens ? l->hmem[0].DZ : l->DZ;
    best[3] = us;
    best[4] = ens ? l->ens_variant : l->variant;
}

static std::string tune_key(const cl_lattice* l)
{
    char buf[256];
    if (!is_ens(l)) {
        snprintf(buf, sizeof(buf), "single N=%d nf=%d prec=%d", l->N, l->nf, l->p.precision);
    } else {
        uint64_t h = 1469598103934665603ull;  // FNV-1a over the member sizes
        for (int n : l->mN) {
            h ^= (uint64_t)n;
            h *= 1099511628211ull;
        }
        snprintf(buf, sizeof(buf), "ensemble B=%d sizes=%016llx nf=%d prec=%d", l->members, (unsigned long long)h, l->nf,
                 l->p.precision);
    }
    return buf;
}

static cl_status apply_tiles(cl_lattice* l, int stages, int by, int dz, int variant)
{
    l->opt_stages = stages;
    l->opt_BY = by;
    l->opt_DZ = dz;
    l->opt_variant = variant;
    return choose_tiles(l);
}

// Average duration (microseconds) of `n` trial passes after `warm` untimed ones.
static cl_status time_trials(cl_lattice* l, int warm, int n, double* us)
{
    const PassCoef pc{l->p.dt, 0.5 * l->p.dt, l->p.dt, P_DRIFT};  // no P_COMMIT: the state is untouched
    for (int i = 0; i < warm; ++i) {
        cl_status s = run_pass(l, pc, l->cur, l->cur ^ 1);
        if (s != CL_OK) return s;
    }
    cudaEvent_t a, b;
    CUDA_TRY(l, cudaEventCreate(&a));
    CUDA_TRY(l, cudaEventCreate(&b));
    cudaEventRecord(a, l->stream);
    cl_status s = CL_OK;
    for (int i = 0; i < n && s == CL_OK; ++i) s = run_pass(l, pc, l->cur, l->cur ^ 1);
    cudaEventRecord(b, l->stream);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *us = 1e3 * ms / n;
    return s;
}

cl_status cl_autotune(cl_lattice* l, const char* cache_path, double* best)
{
    if (!l) return CL_EINVAL;
    if (l->dims < 3) return fail(l, CL_EUNSUPPORTED, "the autotuner is not available on a reduced (1+1)/(2+1) lattice");
    if (is_rk(l->p.integrator) || l->gauge) return fail(l, CL_EINVAL, "the autotuner covers the leapfrog pass only");
    if (!l->potential_set) return fail(l, CL_ESTATE, "cl_set_potential has not been called");
    const std::string key = tune_key(l);
    if (cache_path) {
        if (FILE* f = fopen(cache_path, "r")) {
            char line[512];
            int hit = 0, st = 0, by = 0, dz = 0, var = 1;
            double us = 0.0;
            while (fgets(line, sizeof(line), f)) {
                const char* k = strstr(line, "\"key\": \"");
                if (!k) continue;
                k += 8;
                const char* e = strchr(k, '"');
                if (!e || std::string(k, e - k) != key) continue;
                if (sscanf(e, "\", \"stages\": %d, \"by\": %d, \"dz\": %d, \"variant\": %d, \"us\": %lf", &st, &by, &dz,
                           &var, &us) == 5)
                    hit = 1;
            }
            fclose(f);
            if (hit && apply_tiles(l, st, by, dz, var) == CL_OK) {
                report_tiles(l, us, best);
                l->diag_valid = false;
                l->rbar_valid = false;
                return CL_OK;
            }
        }
    }
    // candidates
    // candidates {stages, BY, DZ, pass variant}
    std::vector<std::array<int, 4>> cand;
    if (is_ens(l)) {
        // {stages, variant}: the direct loader, the ring kernel and the ringless kernel
        const int sv_list[][2] = {{-1, 1}, {2, 0}, {3, 0}, {4, 0}, {3, 1}, {4, 1}, {5, 1}, {6, 1}};
        const int dz_list[] = {0, 32, 16};
        for (const auto& sv : sv_list)
            for (int dz : dz_list)
                for (int by : {0, 8}) cand.push_back({sv[0], by, dz, sv[1]});
    } else {
        cl_status s0 = apply_tiles(l, 0, 0, 0, 1);
        if (s0 != CL_OK) return s0;
        const int by_auto = l->BY;
        const bool nr_ok = l->VW * l->es == 16;  // the ringless kernel takes 16-byte vectors
        std::vector<int> st_list = {-1, 0};
        if (scalar_pass_tma_ok(l->p.precision, l->N))
            for (int st = 2; st <= 6; ++st) st_list.push_back(st);
        for (int st : st_list)
            for (int var : {0, 1}) {
                if (var == 1 && (!nr_ok || st < 0 || st > 5)) continue;
                for (int dz : {0, -1})
                    for (int by : {0, by_auto > 1 ? by_auto / 2 : 0}) {
                        std::array<int, 4> c = {st, by, dz, var};
                        if (std::find(cand.begin(), cand.end(), c) == cand.end()) cand.push_back(c);
                    }
            }
    }
    double best_us = 1e300;
    std::array<int, 4> best_c = {0, 0, 0, 1};
    for (const auto& c : cand) {
        if (apply_tiles(l, c[0], c[1], c[2], c[3]) != CL_OK) continue;
        double us = 0.0;
        if (time_trials(l, 2, 5, &us) != CL_OK) continue;
        if (us < best_us) {
            best_us = us;
            best_c = c;
        }
    }
    cl_status s = apply_tiles(l, best_c[0], best_c[1], best_c[2], best_c[3]);
    if (s != CL_OK) return s;
    CUDA_TRY(l, cudaStreamSynchronize(l->stream));
    l->diag_valid = false;
    l->rbar_valid = false;
    if (cache_path && best_us < 1e300) {
        if (FILE* f = fopen(cache_path, "a")) {
            fprintf(f, "{\"key\": \"%s\", \"stages\": %d, \"by\": %d, \"dz\": %d, \"variant\": %d, \"us\": %.3f}\n",
                    key.c_str(), best_c[0], best_c[1], best_c[2], best_c[3], best_us);
            fclose(f);
        }
    }
    report_tiles(l, best_us, best);
    return CL_OK;
}

cl_status cl_step(cl_lattice* l, int32_t nsteps)
{
    if (!l) return CL_EINVAL;
    if (nsteps < 0) return fail(l, CL_EINVAL, "nsteps < 0");
    if (!l->potential_set) return fail(l, CL_ESTATE, "cl_set_potential has not been called");
    l->last_launches = 0;
    if (nsteps == 0) return CL_OK;
    const bool rk = is_rk(l->p.integrator);  // Runge-Kutta states stay at integer times
    if (!l->open && !rk) {
        cl_status s = open_leapfrog(l);
        if (s != CL_OK) return s;
        l->last_launches += is_u1_lf(l) ? (l->u1_sfused ? 1 : 2) : (l->gw ? 2 : 1);
    } else if (is_u1_lf(l) && l->u1_staged && !l->u1_sfused && !l->u1_lf_pq) {
        cl_status s = is_fp64(l) ? u1_lf_save_pq_t<double>(l) : u1_lf_save_pq_t<float>(l);
        if (s != CL_OK) return s;
        l->last_launches += 1;
    }
    const std::vector<PassCoef> sched = step_schedule(l);
    const int pps = (int)sched.size();
    int flips = 0;  // buffer swaps of one step
    for (const auto& pc : sched) flips += pc.flip ? 1 : 0;
    const bool nmc_f = nmc_fused(l);
    if (nmc_f && !l->rbar_valid) {  // the fused stages carry the Ricci scalar from stage to stage
        cl_status s = is_fp64(l) ? nmc_ricci_t<double>(l) : nmc_ricci_t<float>(l);
        if (s != CL_OK) return s;
        l->last_launches += 1;
    }
    // the fused stages leave R of the final state behind; stages with a reduction launch leave
    // that of their last input state
    l->rbar_valid = nmc_f;
    for (int i = 0; i < nsteps; ++i) {
        if (l->use_graph) {
            const int par = l->cur;
            if (!l->graph[par]) {
                cudaGraph_t g;
                CUDA_TRY(l, cudaStreamBeginCapture(l->stream, cudaStreamCaptureModeThreadLocal));
                int c = par;
                cl_status s = CL_OK;
                for (const auto& pc : sched) {
                    s = run_pass(l, pc, c, c ^ 1);
                    if (s != CL_OK) break;
                    if (pc.flip) c ^= 1;
                }
                cudaError_t ee = cudaStreamEndCapture(l->stream, &g);
                if (s != CL_OK) return s;
                if (ee != cudaSuccess) return fail(l, CL_ECUDA, "graph capture failed: %s", cudaGetErrorString(ee));
                ee = cudaGraphInstantiate(&l->graph[par], g, 0);
                cudaGraphDestroy(g);
                if (ee != cudaSuccess) return fail(l, CL_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(ee));
            }
            CUDA_TRY(l, cudaGraphLaunch(l->graph[par], l->stream));
            l->cur = (flips & 1) ? par ^ 1 : par;
        } else {
            for (const auto& pc : sched) {
                cl_status s = run_pass(l, pc, l->cur, l->cur ^ 1);
                if (s != CL_OK) return s;
                if (pc.flip) l->cur ^= 1;
            }
        }
        // two-launch gauge stages (helper + stage), non-minimally coupled stages (Ricci + stage)
        // and leapfrog passes with gravitational waves (GW pass + scalar pass)
        l->last_launches += (l->gauge && !l->u1_fused && !l->u1_sfused) || (l->nmc && !nmc_f) || l->gw ? 2 * pps : pps;
        // per-step Gauss tracking launches of the U(1) forms whose stage does not sum it itself
        if (is_u1_lf(l)) l->last_launches += l->u1_staged ? 0 : 1;
        else if (l->gauge && !l->u1_staged) l->last_launches += l->u1_fused ? 2 : 1;
    }
    // a leapfrog step ends with the energies of its integer time; a Runge-Kutta stage
    // reports those of the state it started from, so they are recomputed on demand
    l->diag_valid = !rk;
    return CL_OK;
}

cl_status cl_sync(cl_lattice* l)
{
    if (!l) return CL_EINVAL;
    std::vector<DevScal> h;
    return read_status(l, h);
}

cl_status cl_energies(cl_lattice* l, cl_energy* out, int32_t count)
{
    if (!l) return CL_EINVAL;
    if (!out || count < 1 || count > l->members) return fail(l, CL_EINVAL, "energies: bad output or count");
    if (!l->diag_valid) {
        cl_status s = energy_pass(l, 0);
        if (s != CL_OK) return s;
    }
    if (l->gauge) {  // lattice Gauss charge of the current state
        cl_status s = run_u1(l, 2, 0.0, 0.0, 0, l->cur, l->cur ^ 1);
        if (s != CL_OK) return s;
    }
    std::vector<DevScal> hv;
    cl_status s = read_status(l, hv);
    for (int m = 0; m < count; ++m) {
        const DevScal& h = hv[m];
        cl_energy* o = out + m;
        memset(o, 0, sizeof(cl_energy));
        o->t = h.diag[D_T];
        o->a = h.diag[D_A];
        o->adot = h.diag[D_ADOT];
        o->K[0] = h.diag[D_K0];
        o->K[1] = h.diag[D_K1];
        o->G[0] = h.diag[D_G0];
        o->G[1] = h.diag[D_G1];
        o->V = h.diag[D_V];
        o->KE = h.diag[D_KE];
        o->GB = h.diag[D_GB];
        o->rho = h.diag[D_RHO];
        o->p = h.diag[D_P];
        o->hubble_violation = h.diag[D_HV];
        o->gauss_violation = h.diag[D_GV];
        o->gauss_rms_step = l->gauge ? h.gauss[0] : 0.0;
        o->gauss_rms_max = l->gauge ? h.gauss[1] : 0.0;
        o->dt = l->adapt_tol > 0.0 ? h.h : l->p.dt;
        o->rk_error = l->adapt_tol > 0.0 ? h.rk_err : 0.0;
        o->step = h.step;
        o->ricci = l->nmc ? h.rbar : 0.0;
    }
    return s;
}

cl_status cl_init_vacuum(cl_lattice* l, int32_t member, const cl_vacuum_params* v)
{
    if (!l) return CL_EINVAL;
    if (l->dims < 3) return fail(l, CL_EUNSUPPORTED, "the vacuum initial condition is not available on a reduced (1+1)/(2+1) lattice");
    if (!v) return fail(l, CL_EINVAL, "vacuum params NULL");
    if (member != -1 && !member_ok(l, member)) return fail(l, CL_EINVAL, "member %d out of range", member);
    if (!l->potential_set) return fail(l, CL_ESTATE, "cl_set_potential has not been called");
    const int m0 = member < 0 ? 0 : member, m1 = member < 0 ? l->members : member + 1;
    const int nf = l->nf;
    const double a = l->p.a0, al = l->p.alpha;
    int nmax = 0;
    for (int m = m0; m < m1; ++m) nmax = mem_N(l, m) > nmax ? mem_N(l, m) : nmax;
    const size_t nh_max = (size_t)nmax * nmax * (nmax / 2 + 1);
    double2 *fk = nullptr, *pk = nullptr;
    double* real = nullptr;
    std::vector<std::pair<int, cufftHandle>> plans;  // one Z2D plan per member size
    cl_status st = CL_OK;
    if (cudaMalloc(&fk, nh_max * sizeof(double2)) != cudaSuccess || cudaMalloc(&pk, nh_max * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&real, (size_t)nmax * nmax * nmax * sizeof(double)) != cudaSuccess) {
        st = fail(l, CL_ENOMEM, "vacuum scratch allocation failed");
    }
    if (st == CL_OK) st = close_leapfrog(l, true);
    for (int m = m0; st == CL_OK && m < m1; ++m) {
        const int N = mem_N(l, m);
        const int64_t V = mem_V(l, m);
        const size_t off = mem_off_bytes(l, m);
        const double* c = is_ens(l) ? &l->mpot[5 * (size_t)m] : nullptr;
        const double m2_0 = c ? c[0] : l->m2[0], lam_0 = c ? c[1] : l->lam[0];
        const double m2_1 = c ? c[2] : l->m2[1], lam_1 = c ? c[3] : l->lam[1], g2 = c ? c[4] : l->g2;
        // homogeneous energy and Hubble rate (Eq. Friedmann2) for the momentum modes
        const double f0 = v->fbar[0], f1 = nf > 1 ? v->fbar[1] : 0.0;
        double rho_h = 0.5 * m2_0 * f0 * f0 + 0.25 * lam_0 * f0 * f0 * f0 * f0 + 0.5 * m2_1 * f1 * f1 +
                       0.25 * lam_1 * f1 * f1 * f1 * f1 + 0.5 * g2 * f0 * f0 * f1 * f1;
        for (int f = 0; f < nf; ++f) rho_h += v->dfbar[f] * v->dfbar[f] / (2.0 * pow(a, 2.0 * al));
        const double H = l->p.expansion ? sqrt(pow(a, 2.0 * al) * l->p.kappa * rho_h / 3.0) : 0.0;
        cufftHandle plan = 0;
        for (const auto& pp : plans)
            if (pp.first == N) plan = pp.second;
        if (!plan) {
            if (cufftPlan3d(&plan, N, N, N, CUFFT_Z2D) != CUFFT_SUCCESS) { st = fail(l, CL_ECUDA, "cufftPlan3d failed"); break; }
            plans.push_back({N, plan});
            if (cufftSetStream(plan, l->stream) != CUFFT_SUCCESS) { st = fail(l, CL_ECUDA, "cufftSetStream failed"); break; }
        }
        for (int f = 0; f < nf; ++f) {
            VacuumModeArgs A{};
            A.N = N; A.field = f; A.member = (uint32_t)m; A.seed = v->seed;
            A.L = mem_L(l, m); A.kcut = v->kcut; A.amp2 = v->amp2; A.a = a; A.alpha = al; A.H = H;
            A.m2eff = f == 0 ? m2_0 + 3.0 * lam_0 * f0 * f0 + g2 * f1 * f1 : m2_1 + 3.0 * lam_1 * f1 * f1 + g2 * f0 * f0;
            cudaError_t e = launch_vacuum_modes(A, fk, pk, l->stream);
            if (e != cudaSuccess) { st = fail(l, CL_ECUDA, "vacuum modes: %s", cudaGetErrorString(e)); break; }
            const double inv = 1.0 / (double)V;  // f(n) = N^-3 sum_k e^{+ikn} f(k)
            if (cufftExecZ2D(plan, (cufftDoubleComplex*)fk, real) != CUFFT_SUCCESS) { st = fail(l, CL_ECUDA, "Z2D failed"); break; }
            e = launch_real_to_field(l->p.precision, real, (char*)l->phi[f][l->cur] + off, v->fbar[f], inv, V, l->stream);
            if (e != cudaSuccess) { st = fail(l, CL_ECUDA, "convert: %s", cudaGetErrorString(e)); break; }
            if (cufftExecZ2D(plan, (cufftDoubleComplex*)pk, real) != CUFFT_SUCCESS) { st = fail(l, CL_ECUDA, "Z2D failed"); break; }
            e = launch_real_to_field(l->p.precision, real, (char*)l->pi[f][l->cur] + off, pow(a, 3.0 - al) * v->dfbar[f],
                                     inv, V, l->stream);
            if (e != cudaSuccess) { st = fail(l, CL_ECUDA, "convert: %s", cudaGetErrorString(e)); break; }
            if (has_kahan(l)) cudaMemsetAsync((char*)l->cc[f][l->cur] + off, 0, (size_t)V * l->es, l->stream);
        }
    }
    if (st == CL_OK) {
        std::vector<DevScal> h;
        st = read_status(l, h);
        if (st == CL_OK) {
            for (int m = m0; m < m1; ++m) {
                h[m] = DevScal{};
                h[m].a = a;
                h[m].h = l->p.dt;
            }
            cudaError_t e = cudaMemcpyAsync(l->scal, h.data(), sizeof(DevScal) * h.size(), cudaMemcpyHostToDevice, l->stream);
            if (e != cudaSuccess) st = fail(l, CL_ECUDA, "scalar upload: %s", cudaGetErrorString(e));
            if (st == CL_OK && cudaStreamSynchronize(l->stream) != cudaSuccess) st = fail(l, CL_ECUDA, "sync failed");
        }
    }
    if (st == CL_OK) {
        l->diag_valid = false;
        l->rbar_valid = false;
        st = is_ens(l) ? energy_pass_members(l, P_HUBBLE_INIT | P_COMMIT, m0, m1) : energy_pass(l, P_HUBBLE_INIT | P_COMMIT);
        if (st == CL_OK && !is_ens(l)) l->diag_valid = true;
    }
    if (st == CL_OK && cudaStreamSynchronize(l->stream) != cudaSuccess) st = fail(l, CL_ECUDA, "sync failed");
    if (st != CL_OK) cudaStreamSynchronize(l->stream);
    for (const auto& pp : plans) cufftDestroy(pp.second);
    if (fk) cudaFree(fk);
    if (pk) cudaFree(pk);
    if (real) cudaFree(real);
    l->open = false;
    return st;
}

cl_status cl_spectrum(cl_lattice* l, int32_t member, int32_t field, double dn, int32_t type, double* k_out,
                      double* delta_out, double* count_out, int32_t cap, int32_t* nbins)
{
    if (!l) return CL_EINVAL;
    if (l->dims < 3) return fail(l, CL_EUNSUPPORTED, "the spectrum is not available on a reduced (1+1)/(2+1) lattice");
    if (!member_ok(l, member)) return fail(l, CL_EINVAL, "member %d out of range", member);
    if (!(dn > 0) || (type != 1 && type != 2) || cap < 0 || (cap > 0 && (!k_out || !delta_out || !count_out)))
        return fail(l, CL_EINVAL, "spectrum: bad arguments");
    int f = 0;
    const int kind = field_kind(l, field, &f);
    if (kind < 0) return fail(l, CL_EINVAL, "field %d not present", field);
    const int N = mem_N(l, member);
    const int64_t V = mem_V(l, member);
    const int nb = (int)floor(sqrt(3.0) * (N / 2) / dn + 0.5) + 1;
    if (nbins) *nbins = nb;
    if (cap == 0) return CL_OK;
    int buf = l->cur;
    const void* fb = kind == 0 ? l->phi[f][buf] : l->pi[f][buf];
    if (l->open && kind == 1 && is_u1_lf(l)) {
        fb = l->ku1[1][l->cur];  // the open axion-U(1) leapfrog keeps the integer-time momenta
    } else if (l->open && kind == 1) {
        cl_status s = close_leapfrog(l, false);
        if (s != CL_OK) return s;
        buf = l->cur ^ 1;
        fb = l->pi[f][buf];
    }
    const void* src = (const char*)fb + mem_off_bytes(l, member);
    const size_t nh = (size_t)N * N * (N / 2 + 1);
    double* real = nullptr;
    double2* F = nullptr;
    double* bins = nullptr;  // S[nb], C[nb], k[nb], delta[nb]
    cufftHandle plan = 0;
    cl_status st = CL_OK;
    if (cudaMalloc(&real, (size_t)V * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&F, nh * sizeof(double2)) != cudaSuccess || cudaMalloc(&bins, 4 * (size_t)nb * sizeof(double)) != cudaSuccess)
        st = fail(l, CL_ENOMEM, "spectrum scratch allocation failed");
    if (st == CL_OK && cufftPlan3d(&plan, N, N, N, CUFFT_D2Z) != CUFFT_SUCCESS) st = fail(l, CL_ECUDA, "cufftPlan3d failed");
    if (st == CL_OK && cufftSetStream(plan, l->stream) != CUFFT_SUCCESS) st = fail(l, CL_ECUDA, "cufftSetStream failed");
    if (st == CL_OK && launch_field_to_double(l->p.precision, src, real, V, l->stream) != cudaSuccess)
        st = fail(l, CL_ECUDA, "field conversion failed");
    if (st == CL_OK && cufftExecD2Z(plan, real, (cufftDoubleComplex*)F) != CUFFT_SUCCESS) st = fail(l, CL_ECUDA, "D2Z failed");
    if (st == CL_OK && cudaMemsetAsync(bins, 0, 2 * (size_t)nb * sizeof(double), l->stream) != cudaSuccess)
        st = fail(l, CL_ECUDA, "memset failed");
    if (st == CL_OK && launch_spectrum_bins(F, N, dn, nb, bins, bins + nb, l->stream) != cudaSuccess)
        st = fail(l, CL_ECUDA, "binning failed");
    if (st == CL_OK &&
        launch_spectrum_finish(bins, bins + nb, N, mem_L(l, member), dn, type, nb, bins + 2 * nb, bins + 3 * nb, l->stream) != cudaSuccess)
        st = fail(l, CL_ECUDA, "spectrum finish failed");
    std::vector<double> h(4 * (size_t)nb);
    if (st == CL_OK && cudaMemcpyAsync(h.data(), bins, 4 * (size_t)nb * sizeof(double), cudaMemcpyDeviceToHost, l->stream) != cudaSuccess)
        st = fail(l, CL_ECUDA, "copy failed");
    if (st == CL_OK && cudaStreamSynchronize(l->stream) != cudaSuccess) st = fail(l, CL_ECUDA, "sync failed");
    if (st == CL_OK) {
        const int n = cap < nb ? cap : nb;
        for (int i = 0; i < n; ++i) {
            count_out[i] = h[nb + i];
            k_out[i] = h[2 * nb + i];
            delta_out[i] = h[3 * nb + i];
        }
    }
    if (plan) cufftDestroy(plan);
    if (real) cudaFree(real);
    if (F) cudaFree(F);
    if (bins) cudaFree(bins);
    return st;
}

cl_status cl_gauge_spectrum(cl_lattice* l, int32_t which, double dn, int32_t type, double* k_out, double* delta_out,
                            double* count_out, int32_t cap, int32_t* nbins)
{
    if (!l) return CL_EINVAL;
    if (!l->gauge) return fail(l, CL_EINVAL, "gauge spectra need an axion-U(1) lattice");
    if (which < 0 || which > 3 || !(dn > 0) || (type != 1 && type != 2) || cap < 0 ||
        (cap > 0 && (!k_out || !delta_out || !count_out)))
        return fail(l, CL_EINVAL, "gauge spectrum: bad arguments");
    const int N = l->N;
    const int64_t V = (int64_t)N * N * N;
    const int nb = (int)floor(sqrt(3.0) * (N / 2) / dn + 0.5) + 1;
    if (nbins) *nbins = nb;
    if (cap == 0) return CL_OK;
    const size_t nh = (size_t)N * N * (N / 2 + 1);
    double* real = nullptr;
    double2* F = nullptr;
    double* bins = nullptr;  // S[nb], C[nb], k[nb], delta[nb]
    cufftHandle plan = 0;
    cl_status st = CL_OK;
    if (cudaMalloc(&real, 3 * (size_t)V * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&F, 3 * nh * sizeof(double2)) != cudaSuccess || cudaMalloc(&bins, 4 * (size_t)nb * sizeof(double)) != cudaSuccess)
        st = fail(l, CL_ENOMEM, "gauge spectrum scratch allocation failed");
    if (st == CL_OK && cufftPlan3d(&plan, N, N, N, CUFFT_D2Z) != CUFFT_SUCCESS) st = fail(l, CL_ECUDA, "cufftPlan3d failed");
    if (st == CL_OK && cufftSetStream(plan, l->stream) != CUFFT_SUCCESS) st = fail(l, CL_ECUDA, "cufftSetStream failed");
    if (st == CL_OK) {
        const cudaError_t e = is_fp64(l) ? gauge_fields_t<double>(l, which, real) : gauge_fields_t<float>(l, which, real);
        if (e != cudaSuccess) st = fail(l, CL_ECUDA, "gauge field conversion failed");
    }
    for (int c = 0; c < 3 && st == CL_OK; ++c)
        if (cufftExecD2Z(plan, real + c * V, (cufftDoubleComplex*)(F + c * nh)) != CUFFT_SUCCESS)
            st = fail(l, CL_ECUDA, "D2Z failed");
    if (st == CL_OK && cudaMemsetAsync(bins, 0, 2 * (size_t)nb * sizeof(double), l->stream) != cudaSuccess)
        st = fail(l, CL_ECUDA, "memset failed");
    if (st == CL_OK && launch_gauge_bins(F, N, l->dx, which, dn, nb, bins, bins + nb, l->stream) != cudaSuccess)
        st = fail(l, CL_ECUDA, "binning failed");
    if (st == CL_OK &&
        launch_spectrum_finish(bins, bins + nb, N, l->p.L, dn, type, nb, bins + 2 * nb, bins + 3 * nb, l->stream) != cudaSuccess)
        st = fail(l, CL_ECUDA, "spectrum finish failed");
    std::vector<double> h(4 * (size_t)nb);
    if (st == CL_OK && cudaMemcpyAsync(h.data(), bins, 4 * (size_t)nb * sizeof(double), cudaMemcpyDeviceToHost, l->stream) != cudaSuccess)
        st = fail(l, CL_ECUDA, "copy failed");
    if (st == CL_OK && cudaStreamSynchronize(l->stream) != cudaSuccess) st = fail(l, CL_ECUDA, "sync failed");
    if (st == CL_OK) {
        const int n = cap < nb ? cap : nb;
        for (int i = 0; i < n; ++i) {
            count_out[i] = h[nb + i];
            k_out[i] = h[2 * nb + i];
            delta_out[i] = h[3 * nb + i];
        }
    }
    if (plan) cufftDestroy(plan);
    if (real) cudaFree(real);
    if (F) cudaFree(F);
    if (bins) cudaFree(bins);
    return st;
}

// ---------------------------------------------------------------- surrogate coupling
static cl_status check_sg_lattice(cl_lattice* l)
{
    if (is_ens(l) || l->gauge || l->nf != 1 || is_fp64(l)) return fail(l, CL_EINVAL, "surrogate coupling needs a single FP32 one-field lattice");
    return CL_OK;
}

static Norm3 make_norm(const float* mu, const float* sg, int C)
{
    Norm3 nm{};
    for (int c = 0; c < 3; ++c) {
        nm.mu[c] = c < C ? mu[c] : 0.f;
        nm.sg[c] = c < C ? sg[c] : 1.f;
    }
    return nm;
}

cl_status cl_lattice_pack(cl_lattice* l, const float* mu, const float* sg, float* x_dev)
{
    if (!l) return CL_EINVAL;
    if (l->dims < 3) return fail(l, CL_EUNSUPPORTED, "the surrogate is not available on a reduced (1+1)/(2+1) lattice");
    if (!mu || !sg || !x_dev) return fail(l, CL_EINVAL, "pack: NULL argument");
    cl_status st = check_sg_lattice(l);
    if (st != CL_OK) return st;
    for (int c = 0; c < 3; ++c)
        if (!(sg[c] != 0.f) || !isfinite(sg[c]) || !isfinite(mu[c])) return fail(l, CL_EINVAL, "pack: bad normalisation");
    st = close_leapfrog(l, true);
    if (st != CL_OK) return st;
    CUDA_TRY(l, launch_pack((const float*)l->phi[0][l->cur], (const float*)l->pi[0][l->cur], &l->scal->a, l->V, 3,
                            make_norm(mu, sg, 3), x_dev, l->stream));
    return CL_OK;
}

cl_status cl_lattice_unpack(cl_lattice* l, const float* mu, const float* sg, const float* y_dev)
{
    if (!l) return CL_EINVAL;
    if (l->dims < 3) return fail(l, CL_EUNSUPPORTED, "the surrogate is not available on a reduced (1+1)/(2+1) lattice");
    if (!mu || !sg || !y_dev) return fail(l, CL_EINVAL, "unpack: NULL argument");
    cl_status st = check_sg_lattice(l);
    if (st != CL_OK) return st;
    st = close_leapfrog(l, true);
    if (st != CL_OK) return st;
    CUDA_TRY(l, launch_unpack(y_dev, l->V, 2, make_norm(mu, sg, 2), (float*)l->phi[0][l->cur], (float*)l->pi[0][l->cur],
                              has_kahan(l) ? (float*)l->cc[0][l->cur] : nullptr, l->stream));
    l->diag_valid = false;
    l->rbar_valid = false;
    return CL_OK;
}

cl_status cl_surrogate_jump(cl_surrogate* s, cl_lattice* l, int32_t steps, const float* mu, const float* sg,
                            double hubble_limit, int32_t* accepted)
{
    if (!l) return CL_EINVAL;
    if (l->dims < 3) return fail(l, CL_EUNSUPPORTED, "the surrogate jump is not available on a reduced (1+1)/(2+1) lattice");
    if (!s || !mu || !sg || !accepted || steps < 1) return fail(l, CL_EINVAL, "jump: bad arguments");
    cl_status st = check_sg_lattice(l);
    if (st != CL_OK) return st;
    if (cl_surrogate_size(s) != l->N) return fail(l, CL_EINVAL, "jump: network and lattice sizes differ");
    *accepted = 0;
    st = close_leapfrog(l, true);
    if (st == CL_OK && !l->diag_valid) st = energy_pass(l, 0);
    std::vector<DevScal> h;
    if (st == CL_OK) st = read_status(l, h);
    if (st != CL_OK) return st;
    const DevScal h0 = h[0];
    const size_t V = (size_t)l->V;
    if (!l->sg_buf && cudaMalloc(&l->sg_buf, 8 * V * sizeof(float)) != cudaSuccess)
        return fail(l, CL_ENOMEM, "jump: scratch allocation failed");
    float* x = l->sg_buf;
    float* y = x + 3 * V;
    float* snap = y + 2 * V;
    const int cur = l->cur;
    float* ph = (float*)l->phi[0][cur];
    float* pv = (float*)l->pi[0][cur];
    float* cv = has_kahan(l) ? (float*)l->cc[0][cur] : nullptr;
    CUDA_TRY(l, cudaMemcpyAsync(snap, ph, V * 4, cudaMemcpyDeviceToDevice, l->stream));
    CUDA_TRY(l, cudaMemcpyAsync(snap + V, pv, V * 4, cudaMemcpyDeviceToDevice, l->stream));
    if (cv) CUDA_TRY(l, cudaMemcpyAsync(snap + 2 * V, cv, V * 4, cudaMemcpyDeviceToDevice, l->stream));
    // the learned jump of (phi, pi)
    CUDA_TRY(l, launch_pack(ph, pv, &l->scal->a, l->V, 3, make_norm(mu, sg, 3), x, l->stream));
    CUDA_TRY(l, cudaStreamSynchronize(l->stream));
    st = cl_surrogate_forward(s, x, y, 1);
    if (st != CL_OK) return fail(l, st, "jump: surrogate forward failed");
    CUDA_TRY(l, cudaStreamSynchronize(surrogate_stream(s)));  // y is written on the surrogate's stream
    CUDA_TRY(l, launch_unpack(y, l->V, 2, make_norm(mu, sg, 2), ph, pv, cv, l->stream));
    // a, a' over the jump with a'' of the starting state (Eq. Friedmann1)
    const double J = (double)steps * l->p.dt, al = l->p.alpha;
    const double a = h0.diag[D_A], b = h0.diag[D_ADOT], rho = h0.diag[D_RHO], p = h0.diag[D_P];
    const double addot =
        l->p.expansion ? pow(a, 2.0 * al + 1.0) * (l->p.kappa / 6.0) * ((2.0 * al - 1.0) * rho - 3.0 * p) : 0.0;
    DevScal hn = h0;
    hn.a = l->p.expansion ? a + J * b + 0.5 * J * J * addot : a;
    hn.b = l->p.expansion ? b + J * addot : b;
    hn.t = h0.diag[D_T] + J;
    hn.step = h0.step + steps;
    hn.status = 0;
    CUDA_TRY(l, cudaMemcpyAsync(l->scal, &hn, sizeof(DevScal), cudaMemcpyHostToDevice, l->stream));
    st = energy_pass(l, 0);
    if (st == CL_OK) st = read_status(l, h);
    if (st != CL_OK && st != CL_ENAN) return st;
    const double hv = h[0].diag[D_HV];
    if (st == CL_OK && isfinite(h[0].diag[D_RHO]) && isfinite(hv) && hv <= hubble_limit) {
        *accepted = 1;
        return CL_OK;
    }
    // fallback: restore the starting state and take the leapfrog steps
    CUDA_TRY(l, cudaMemcpyAsync(ph, snap, V * 4, cudaMemcpyDeviceToDevice, l->stream));
    CUDA_TRY(l, cudaMemcpyAsync(pv, snap + V, V * 4, cudaMemcpyDeviceToDevice, l->stream));
    if (cv) CUDA_TRY(l, cudaMemcpyAsync(cv, snap + 2 * V, V * 4, cudaMemcpyDeviceToDevice, l->stream));
    DevScal hr = h0;
    hr.status = 0;
    CUDA_TRY(l, cudaMemcpyAsync(l->scal, &hr, sizeof(DevScal), cudaMemcpyHostToDevice, l->stream));
    CUDA_TRY(l, cudaStreamSynchronize(l->stream));
    l->diag_valid = false;
    l->rbar_valid = false;
    st = cl_step(l, steps);
    if (st == CL_OK) st = cl_sync(l);
    return st;
}

}  // extern "C"
