// Axion coupled to compact U(1) links: one 2N Runge-Kutta stage (section "ALP-gauge
// interactions", Eq. AxionInfEOM, recast in alpha-time and integrated with the
// low-storage Runge-Kutta schemes as that section prescribes).
//
// Lattice fields: the axion phi and its momentum pi = a^(3-alpha) phi' on sites; link
// angles theta_i(n) = dx A_i and electric fields E_i(n) = A_i' on the links n -> n+i.
// The equations are the Euler-Lagrange equations of a lattice Lagrangian whose
// Chern-Simons term is g phi(n) Ebar(n).Bbar(n), Ebar_i(n) = (E_i(n) + E_i(n-i))/2 and
// Bbar_i(n) the average of sin theta_jk / dx^2 over the four (j,k)-plaquettes around n
// ((i,j,k) cyclic), g = alpha_L sqrt(kappa), ws2 = (omega_star/f_star)^2:
//
//   phi' = a^(alpha-3) pi
//   pi'  = a^(1+alpha) Lap phi - a^(3+alpha) V'(phi) + ws2 g Ebar.Bbar
//   theta_i' = dx E_i
//   E_i' = a^(alpha-1) [ -a^(alpha-1) Mag_i + g (C_i - W_i') ] - (1-alpha) (a'/a) E_i
//     Mag_i(n) = sum_{j!=i} [sin theta_ij(n) - sin theta_ij(n-j)] / dx^3
//     C_i(n)   = sum over the four plaquettes P through the link of
//                +-cos theta_P * (sum of phi Ebar_k over the four corners of P) / (4 dx),
//                k the direction normal to P (the link derivative of sum phi Ebar.Bbar)
//     W_i(n)   = (phi(n) Bbar_i(n) + phi(n+i) Bbar_i(n+i)) / 2
//
// Two launches per stage.  k_u1_helpers stores, per site, Bbar_k, its rate and
// X_k = phi Ebar_k; k_u1_stage gathers the forces from them, performs
// k <- A k + h F(y), y <- y + B k for all eight degrees of freedom per site, and
// reduces the energies of the old state (FP64 across threads and blocks, fixed
// order); the last block advances a, a' and their auxiliaries.  k_u1_gauss reduces
// the lattice Gauss charge div-[a^(1-alpha) E + g W] for the diagnostics.
#include <math.h>

#include "cl_internal.cuh"
#include "kernel_common.cuh"

namespace clk {

struct Site {
    int x, y, z, N;
    __device__ __forceinline__ Site(int64_t n, int N_) : N(N_)
    {
        x = (int)(n % N_);
        y = (int)((n / N_) % N_);
        z = (int)(n / ((int64_t)N_ * N_));
    }
    __device__ __forceinline__ int64_t at(int dx_, int dy_, int dz_) const
    {
        int xx = x + dx_, yy = y + dy_, zz = z + dz_;
        xx = xx < 0 ? xx + N : (xx >= N ? xx - N : xx);
        yy = yy < 0 ? yy + N : (yy >= N ? yy - N : yy);
        zz = zz < 0 ? zz + N : (zz >= N ? zz - N : zz);
        return ((int64_t)zz * N + yy) * N + xx;
    }
    // site shifted by s along direction d, then by t along e
    __device__ __forceinline__ int64_t sh(int d, int s, int e = 0, int t = 0) const
    {
        int o[3] = {0, 0, 0};
        o[d] += s;
        o[e] += t;
        return at(o[0], o[1], o[2]);
    }
};

template <typename T>
__device__ __forceinline__ T plaq(const U1Args<T>& A, const Site& s, int64_t q, int i, int j)
{
    const Site sq(q, s.N);
    return A.th_in[i][q] + A.th_in[j][sq.sh(i, 1)] - A.th_in[i][sq.sh(j, 1)] - A.th_in[j][q];
}

template <typename T>
__device__ __forceinline__ T plaq_rate(const U1Args<T>& A, const Site& s, int64_t q, int i, int j)
{
    const Site sq(q, s.N);
    return (T)A.dx * (A.E_in[i][q] + A.E_in[j][sq.sh(i, 1)] - A.E_in[i][sq.sh(j, 1)] - A.E_in[j][q]);
}

template <typename T>
__global__ void __launch_bounds__(256) k_u1_helpers(const U1Args<T> A)
{
    const int N = A.N;
    const int64_t V = (int64_t)N * N * N;
    const T inv4dx2 = (T)(0.25 / (A.dx * A.dx));
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < V; m += (int64_t)gridDim.x * blockDim.x) {
        const Site s(m, N);
        const T ph = A.phi_in[m];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
            const int64_t q[4] = {m, s.sh(k1, -1), s.sh(k2, -1), s.sh(k1, -1, k2, -1)};
            T b = (T)0, bd = (T)0;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const T p = plaq(A, s, q[c], k1, k2);
                b += sin(p);
                bd += cos(p) * plaq_rate(A, s, q[c], k1, k2);
            }
            A.Bbar[k][m] = b * inv4dx2;
            A.Bdot[k][m] = bd * inv4dx2;
            A.X[k][m] = ph * (T)0.5 * (A.E_in[k][m] + A.E_in[k][s.sh(k, -1)]);
        }
    }
}

// Sum of X_k over the four corners q, q+e_k1, q+e_k2, q+e_k1+e_k2 of the plaquette at q.
template <typename T>
__device__ __forceinline__ T corner_sum(const U1Args<T>& A, int64_t q, int k, int k1, int k2)
{
    const Site sq(q, A.N);
    return A.X[k][q] + A.X[k][sq.sh(k1, 1)] + A.X[k][sq.sh(k2, 1)] + A.X[k][sq.sh(k1, 1, k2, 1)];
}

template <typename T>
__global__ void __launch_bounds__(256) k_u1_stage(const U1Args<T> A)
{
    __shared__ double s_coef[6];
    __shared__ double s_red[32][kMaxQ];
    __shared__ int s_last;
    const int N = A.N;
    const int64_t V = (int64_t)N * N * N;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const bool first = (A.flags & P_FIRST_STAGE) != 0;
    const bool update = (A.flags & P_ENERGY_ONLY) == 0;
    const bool expand = (A.flags & P_EXPANSION) != 0;
    if (tid == 0) {
        const double a = A.scal->a, b = expand ? A.scal->b : 0.0;
        s_coef[0] = pow(a, A.alpha - 3.0);                     // phi' = c0 pi
        s_coef[1] = pow(a, 1.0 + A.alpha) / (A.dx * A.dx);      // Laplacian
        s_coef[2] = pow(a, 3.0 + A.alpha);                     // potential
        s_coef[3] = pow(a, A.alpha - 1.0);                     // E' prefactor
        s_coef[4] = (1.0 - A.alpha) * b / a;                   // electric friction
        s_coef[5] = a;
    }
    __syncthreads();
    const T c_dphi = (T)s_coef[0], cL = (T)s_coef[1], cV = (T)s_coef[2], cE = (T)s_coef[3], cfr = (T)s_coef[4];
    const T g = (T)A.g, ws2 = (T)A.ws2, dx = (T)A.dx, m2 = (T)A.m2, lam = (T)A.lam;
    const T inv_dx3 = (T)(1.0 / (A.dx * A.dx * A.dx)), inv4dx = (T)(0.25 / A.dx);
    const T h = (T)A.h, cA = (T)A.A, cB = (T)A.B;
    Acc<T> accK, accG, accV, accKE, accGB;

    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + tid; n < V; n += (int64_t)gridDim.x * blockDim.x) {
        const Site s(n, N);
        const T ph = A.phi_in[n], pv = A.pi_in[n];
        // scalar sector
        const T pxp = A.phi_in[s.sh(0, 1)], pxm = A.phi_in[s.sh(0, -1)];
        const T pyp = A.phi_in[s.sh(1, 1)], pym = A.phi_in[s.sh(1, -1)];
        const T pzp = A.phi_in[s.sh(2, 1)], pzm = A.phi_in[s.sh(2, -1)];
        const T lap = ((pxp + pxm) + (pyp + pym) + (pzp + pzm)) - (T)6 * ph;
        const T dV = ph * (m2 + lam * ph * ph);
        T eb = (T)0, e2 = (T)0;
        T Ecur[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            Ecur[k] = A.E_in[k][n];
            eb += (T)0.5 * (Ecur[k] + A.E_in[k][s.sh(k, -1)]) * A.Bbar[k][n];
            e2 += Ecur[k] * Ecur[k];
        }
        const T F_phi = c_dphi * pv;
        const T F_pi = cL * lap - cV * dV + ws2 * g * eb;
        T gb = (T)0;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = i + 1; j < 3; ++j) gb += (T)1 - cos(plaq(A, s, n, i, j));
        accK.add(pv * pv);
        accG.add((pxp - ph) * (pxp - ph) + (pyp - ph) * (pyp - ph) + (pzp - ph) * (pzp - ph));
        accV.add(ph * ph * ((T)0.5 * m2 + (T)0.25 * lam * ph * ph));
        accKE.add(e2);
        accGB.add(gb);
        if (!update) continue;

        // link forces
        T F_th[3], F_E[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int ip = (i + 1) % 3, im = (i + 2) % 3;
            // magnetic: sum_{j != i} sin theta_ij(n) - sin theta_ij(n - j), theta_ji = -theta_ij
            T mag = sin(plaq(A, s, n, i, ip)) - sin(plaq(A, s, s.sh(ip, -1), i, ip)) -
                    sin(plaq(A, s, n, im, i)) + sin(plaq(A, s, s.sh(im, -1), im, i));
            // Chern-Simons: plaquettes (i, i+1) normal to i+2 and (i+2, i) normal to i+1
            const int64_t qa = s.sh(ip, -1), qb = s.sh(im, -1);
            const T cs = cos(plaq(A, s, n, i, ip)) * corner_sum(A, n, im, i, ip) -
                         cos(plaq(A, s, qa, i, ip)) * corner_sum(A, qa, im, i, ip) +
                         cos(plaq(A, s, qb, im, i)) * corner_sum(A, qb, ip, im, i) -
                         cos(plaq(A, s, n, im, i)) * corner_sum(A, n, ip, im, i);
            const int64_t ni = s.sh(i, 1);
            const T wdot = (T)0.5 * (F_phi * A.Bbar[i][n] + ph * A.Bdot[i][n] +
                                     c_dphi * A.pi_in[ni] * A.Bbar[i][ni] + A.phi_in[ni] * A.Bdot[i][ni]);
            F_E[i] = cE * (-cE * mag * inv_dx3 + g * (cs * inv4dx - wdot)) - cfr * Ecur[i];
            F_th[i] = dx * Ecur[i];
        }
        // 2N Runge-Kutta update of the eight degrees of freedom of this site
        const T F[8] = {F_phi, F_pi, F_th[0], F_th[1], F_th[2], F_E[0], F_E[1], F_E[2]};
        const T y[8] = {ph, pv, A.th_in[0][n], A.th_in[1][n], A.th_in[2][n], Ecur[0], Ecur[1], Ecur[2]};
        T* out[8] = {A.phi_out, A.pi_out, A.th_out[0], A.th_out[1], A.th_out[2], A.E_out[0], A.E_out[1], A.E_out[2]};
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const T kq = first ? h * F[q] : cA * A.k_in[q][n] + h * F[q];
            A.k_out[q][n] = kq;
            out[q][n] = y[q] + cB * kq;
        }
    }

    // ---- block partials; last block: energies of the old state and the (a, a') stage ----
    double v[kMaxQ] = {accK.value(), accG.value(), accV.value(), accKE.value(), accGB.value()};
    block_reduce<kMaxQ>(v, s_red, tid, nthr);
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < kMaxQ; ++q) A.partials[(size_t)blockIdx.x * kMaxQ + q] = v[q];
        __threadfence();
        const unsigned prev = atomicAdd(&A.scal->counter, 1u);
        s_last = (prev + 1u == gridDim.x);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double w[kMaxQ] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = tid; b < (int)gridDim.x; b += nthr)
#pragma unroll
        for (int q = 0; q < kMaxQ; ++q) w[q] += __ldcg(&A.partials[(size_t)b * kMaxQ + q]);
    block_reduce<kMaxQ>(w, s_red, tid, nthr);
    if (tid == 0) {
        DevScal* S = A.scal;
        const double vol = (double)V;
        const double a = s_coef[5], b = expand ? S->b : 0.0;
        const double a2 = a * a, a4 = a2 * a2, a6 = a4 * a2;
        const double K = w[0] / (2.0 * a6 * vol);
        const double G = w[1] / (A.dx * A.dx * 2.0 * a2 * vol);
        const double Vp = w[2] / vol;
        const double KE = A.ws2 * w[3] / (2.0 * pow(a, 2.0 + 2.0 * A.alpha) * vol);
        const double GB = A.ws2 * w[4] / (pow(A.dx, 4.0) * a4 * vol);
        const double rho = K + G + Vp + KE + GB;
        const double p = K - G / 3.0 - Vp + (KE + GB) / 3.0;
        const double a2al = pow(a, 2.0 * A.alpha);
        double bb = b;
        if ((A.flags & P_HUBBLE_INIT) && expand) bb = a * sqrt(a2al * A.kappa * rho / 3.0);
        const double H = bb / a;
        const double hv = H != 0.0 ? fabs(H * H - a2al * A.kappa * rho / 3.0) / (H * H) : 0.0;
        S->diag[D_T] = S->t;
        S->diag[D_A] = a;
        S->diag[D_ADOT] = bb;
        S->diag[D_K0] = K;
        S->diag[D_K1] = 0.0;
        S->diag[D_G0] = G;
        S->diag[D_G1] = 0.0;
        S->diag[D_V] = Vp;
        S->diag[D_KE] = KE;
        S->diag[D_GB] = GB;
        S->diag[D_RHO] = rho;
        S->diag[D_P] = p;
        S->diag[D_HV] = hv;
        if (A.flags & P_HUBBLE_INIT) S->b = bb;
        if (update && expand) {
            const double Fa = b;
            const double Fb = pow(a, 2.0 * A.alpha + 1.0) * (A.kappa / 6.0) * ((2.0 * A.alpha - 1.0) * rho - 3.0 * p);
            const double ka = first ? A.h * Fa : A.A * S->rk[0] + A.h * Fa;
            const double kb = first ? A.h * Fb : A.A * S->rk[1] + A.h * Fb;
            S->rk[0] = ka;
            S->rk[1] = kb;
            S->a = a + A.B * ka;
            S->b = b + A.B * kb;
        }
        if (update && (A.flags & P_COUNT_STEP)) {
            S->t += A.h;
            S->step += 1;
        }
        int st = 0;
        if (!isfinite(rho) || !isfinite(p)) st |= ST_NAN;
        if (first && A.hubble_limit > 0.0 && hv > A.hubble_limit) st |= ST_CONSTRAINT;
        if (st) atomicOr(&S->status, st);
        S->counter = 0u;
    }
}

// Lattice Gauss charge G(n) = sum_i [P_i(n) - P_i(n - i)] / dx, P = a^(1-alpha) E + g W.
// Writes diag[D_GV] = max_n |G(n)| / max_n sum_i (|P_i(n)| + |P_i(n - i)|) / dx.
template <typename T>
__global__ void __launch_bounds__(256) k_u1_gauss(const U1Args<T> A)
{
    __shared__ double s_red[32][kMaxQ];
    __shared__ int s_last;
    const int N = A.N;
    const int64_t V = (int64_t)N * N * N;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const double ca = pow(A.scal->a, 1.0 - A.alpha);
    double gmax = 0.0, smax = 0.0;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + tid; n < V; n += (int64_t)gridDim.x * blockDim.x) {
        const Site s(n, N);
        double G = 0.0, sc = 0.0;
        for (int i = 0; i < 3; ++i) {
            const int64_t np = s.sh(i, 1), nm = s.sh(i, -1);
            const double Pn = ca * (double)A.E_in[i][n] +
                              A.g * 0.5 * ((double)A.phi_in[n] * A.Bbar[i][n] + (double)A.phi_in[np] * A.Bbar[i][np]);
            const double Pm = ca * (double)A.E_in[i][nm] +
                              A.g * 0.5 * ((double)A.phi_in[nm] * A.Bbar[i][nm] + (double)A.phi_in[n] * A.Bbar[i][n]);
            G += Pn - Pm;
            sc += fabs(Pn) + fabs(Pm);
        }
        gmax = fmax(gmax, fabs(G) / A.dx);
        smax = fmax(smax, sc / A.dx);
    }
    // block maxima (fixed order), then the last block combines them
    for (int off = 16; off > 0; off >>= 1) {
        gmax = fmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, off));
        smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, off));
    }
    const int warp = tid >> 5, lane = tid & 31, nw = (nthr + 31) >> 5;
    if (lane == 0) {
        s_red[warp][0] = gmax;
        s_red[warp][1] = smax;
    }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < nw; ++w) {
            gmax = fmax(gmax, s_red[w][0]);
            smax = fmax(smax, s_red[w][1]);
        }
        A.partials[(size_t)blockIdx.x * kMaxQ + 0] = gmax;
        A.partials[(size_t)blockIdx.x * kMaxQ + 1] = smax;
        __threadfence();
        const unsigned prev = atomicAdd(&A.scal->counter, 1u);
        s_last = (prev + 1u == gridDim.x);
    }
    __syncthreads();
    if (!s_last || tid != 0) return;
    __threadfence();
    double G = 0.0, Sc = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) {
        G = fmax(G, __ldcg(&A.partials[(size_t)b * kMaxQ + 0]));
        Sc = fmax(Sc, __ldcg(&A.partials[(size_t)b * kMaxQ + 1]));
    }
    A.scal->diag[D_GV] = Sc > 0.0 ? G / Sc : 0.0;
    A.scal->counter = 0u;
}

static int u1_grid(int N)
{
    const int64_t V = (int64_t)N * N * N;
    int64_t b = (V + 255) / 256;
    return (int)(b < 152 * 16 ? b : 152 * 16);
}

template <typename T>
static cudaError_t launch_u1_t(const U1Args<T>& A, int what, cudaStream_t s)
{
    const int grid = u1_grid(A.N);
    if (what == 0) k_u1_helpers<T><<<grid, 256, 0, s>>>(A);
    else if (what == 1) k_u1_stage<T><<<grid, 256, 0, s>>>(A);
    else k_u1_gauss<T><<<grid, 256, 0, s>>>(A);
    return cudaGetLastError();
}

int u1_grid_blocks(int N) { return u1_grid(N); }

cudaError_t launch_u1(int precision, const void* args, int what, cudaStream_t s)
{
    if (precision == CL_PREC_FP64) return launch_u1_t(*static_cast<const U1Args<double>*>(args), what, s);
    return launch_u1_t(*static_cast<const U1Args<float>*>(args), what, s);
}

}  // namespace clk
