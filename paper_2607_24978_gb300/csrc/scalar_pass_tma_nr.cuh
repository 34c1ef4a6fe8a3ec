// Ringless variant of the TMA-staged fused pass (included by scalar_pass.cu after the
// ring kernel).  Same producer and stage protocol, but no shared ring of drifted fields
// and no per-plane consumer barrier: a consumer warp drifts its own row of plane j into
// registers, then kicks plane j-1 with the y-neighbour rows drifted again on the fly from
// that plane's stage buffer (the same deterministic drift the owning warp applied, so the
// values agree bit for bit).  A stage is therefore held until its plane was kicked: every
// consumer warp arrives on its "empty" barrier after the kick (the planes that are never
// kicked, the two z halos of a segment, right away), and the producer stays S - 2 planes
// ahead.  Warps synchronise only through the full/empty mbarriers; all waits are bounded.

template <typename T, int NF, bool KAHAN, int VW, int S>
__global__ void __launch_bounds__(480, 1) k_scalar_pass_tma_nr(const ScalarPassArgs<T> A)
{
    constexpr int KPF = KAHAN ? 3 : 2;  // arrays per field in a stage: phi, pi (, c)
    constexpr int NARR = NF * KPF;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t s_full[S];
    __shared__ __align__(8) uint64_t s_empty[S];
    __shared__ double s_coef[4];
    __shared__ double s_red[32][kMaxQ];
    __shared__ int s_last, s_timeout;

    const int N = A.N, BY = A.BY;
    const int TX = N / VW;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int CT = nthr - 32;        // consumer threads (whole warps)
    const int CW = CT / 32;          // consumer warps
    const bool producer = tid >= CT;
    const int r = tid < BY * TX ? tid / TX : BY, tx = tid < BY * TX ? tid % TX : 0;
    const int x0 = tx * VW;
    const int arr_stride = (BY + 2) * N;  // elements of one array in one stage
    const int stage_stride = NARR * arr_stride;
    T* stage = reinterpret_cast<T*>(smem_raw);
    long long u0, u1;
    block_units(N, A.nby, A.DZ, u0, u1);

    if (tid == 0) {
        pass_coefficients(A.scal->a, A.scal->b, A.d, A.alpha, A.dx, (A.flags & P_EXPANSION) != 0, s_coef);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            mbar_init(&s_full[s], 1);
            mbar_init(&s_empty[s], CW);
        }
        mbar_fence_init();
        s_timeout = 0;
    }
    __syncthreads();
    Acc<T> accK[NF], accG[NF], accV;

    if (producer) {
        // ---------------------------------------------------------------- producer warp
        const int lane = tid - CT;
        int st = 0;
        uint32_t empty_phase = 0;
        int issued = 0;
        for (long long u = u0; u < u1;) {
            const int tile = (int)(u / N);
            const int z0 = (int)(u - (long long)tile * N);
            const int NZ = (int)min((long long)(N - z0), u1 - u);
            const int y0 = tile * BY, R = min(BY, N - y0);
            const int ylo = y0 == 0 ? N - 1 : y0 - 1;
            const int yhi = y0 + R == N ? 0 : y0 + R;
            const uint32_t plane_bytes = (uint32_t)(NARR * (R + 2) * N * sizeof(T));
            u += NZ;
            int zz = z0 == 0 ? N - 1 : z0 - 1;
            for (int j = 0; j < NZ + 2; ++j) {
                if (issued >= S) {
                    if (!mbar_wait_bounded(&s_empty[st], (empty_phase >> st) & 1u,
                                           s_timeout ? 1000000ull : 2000000000ull))
                        s_timeout = 1;
                    empty_phase ^= 1u << st;
                }
                if (lane == 0) mbar_arrive_expect_tx(&s_full[st], plane_bytes);
                __syncwarp();
                if (lane < 3 * NARR) {
                    const int a = lane / 3, part = lane - 3 * (lane / 3);
                    const int f = a / KPF, kind = a - KPF * (a / KPF);
                    const T* src = kind == 0 ? A.phi_in[f] : (kind == 1 ? A.pi_in[f] : A.c_in[f]);
                    const int y = part == 0 ? ylo : (part == 1 ? y0 : yhi);
                    const int srow = part == 0 ? 0 : (part == 1 ? 1 : R + 1);
                    const int nrows = part == 1 ? R : 1;
                    T* dst = stage + st * stage_stride + a * arr_stride + srow * N;
                    tma_bulk_g2s(dst, src + ((size_t)zz * N + y) * N, (uint32_t)(nrows * N * sizeof(T)), &s_full[st]);
                }
                __syncwarp();
                ++issued;
                st = st + 1 == S ? 0 : st + 1;
                zz = zz + 1 == N ? 0 : zz + 1;
            }
        }
    } else {
        // ---------------------------------------------------------------- consumer warps
        const T cd = (T)s_coef[0], cL = (T)s_coef[1], cV = (T)s_coef[2];
        const T ce = (T)A.e, ck = (T)A.k;
        const bool do_drift = (A.flags & P_DRIFT) != 0;
        const PotCoef<T> P(A.m2, A.lam, A.g2);
        const int lane = tid & 31;
        const bool own = tid < BY * TX;
        const bool xm_lane = own && lane > 0 && tx > 0;
        const bool xp_lane = own && lane < 31 && tx < TX - 1;
        const int xm_idx = x0 == 0 ? N - 1 : x0 - 1;
        const int xp_idx = x0 + VW == N ? 0 : x0 + VW;
        T pcur[NF][VW], pnext[NF][VW];
        T zlo[NF][VW], zmid[NF][VW], znew[NF][VW];  // drifted own vector of planes j-2, j-1, j
        int st = 0, st_prev = 0;  // stages of planes j and j-1
        uint32_t full_phase = 0;
        const size_t plane = (size_t)N * N;
        // drifted value of field f at (stage row srow, column x) of stage buffer sb
        auto drifted1 = [&](const T* sb, int f, int srow, int x) -> T {
            const T* sa = sb + f * KPF * arr_stride + srow * N + x;
            T ph = sa[0];
            if (do_drift) {
                T cv = KAHAN ? sa[2 * arr_stride] : (T)0;
                drift<T, KAHAN>(ph, cv, sa[arr_stride], cd);
            }
            return ph;
        };
        auto release = [&](int s_idx) {
            __syncwarp();
            if (lane == 0) mbar_arrive(&s_empty[s_idx]);
        };
        for (long long u = u0; u < u1;) {
            const int tile = (int)(u / N);
            const int z0 = (int)(u - (long long)tile * N);
            const int NZ = (int)min((long long)(N - z0), u1 - u);
            const int y0 = tile * BY, R = min(BY, N - y0);
            u += NZ;
            int zz = z0 == 0 ? N - 1 : z0 - 1;
            const size_t row_off = (size_t)(y0 + r) * N + x0;
            for (int j = 0; j < NZ + 2; ++j) {
                if (!mbar_wait_bounded(&s_full[st], (full_phase >> st) & 1u, s_timeout ? 1000000ull : 2000000000ull))
                    s_timeout = 1;
                full_phase ^= 1u << st;
                const T* sb = stage + st * stage_stride;
                const bool write_out = j >= 1 && j <= NZ;
                if (r < R) {  // own row of plane j: drift, write out, keep in registers
                    const size_t base = (size_t)zz * plane + row_off;
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        T pv[VW], cv[VW];
                        const T* sa = sb + f * KPF * arr_stride + (r + 1) * N + x0;
                        vload_smem<T, VW>(znew[f], sa);
                        vload_smem<T, VW>(pv, sa + arr_stride);
                        if (KAHAN) vload_smem<T, VW>(cv, sa + 2 * arr_stride);
                        if (do_drift) {
#pragma unroll
                            for (int i = 0; i < VW; ++i) drift<T, KAHAN>(znew[f][i], cv[i], pv[i], cd);
                        }
                        if (write_out) {
                            vstore<T, VW>(A.phi_out[f] + base, znew[f]);
                            if (KAHAN) vstore<T, VW>(A.c_out[f] + base, cv);
                        }
#pragma unroll
                        for (int i = 0; i < VW; ++i) pnext[f][i] = pv[i];
                    }
                }
                if (j >= 2) {
                    // kick plane j-1: centre zmid, z neighbours zlo / znew, y neighbours drifted
                    // again from the stage of plane j-1
                    const T* sp = stage + st_prev * stage_stride;
                    T phc[NF][VW], lap[NF][VW];
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        T xm_s = __shfl_up_sync(0xffffffffu, zmid[f][VW - 1], 1);
                        T xp_s = __shfl_down_sync(0xffffffffu, zmid[f][0], 1);
                        if (r < R) {
                            T ym[VW], yp[VW];
                            {
                                T pvm[VW], cvm[VW], pvp[VW], cvp[VW];
                                const T* am = sp + f * KPF * arr_stride + r * N + x0;
                                const T* ap = sp + f * KPF * arr_stride + (r + 2) * N + x0;
                                vload_smem<T, VW>(ym, am);
                                vload_smem<T, VW>(yp, ap);
                                if (do_drift) {
                                    vload_smem<T, VW>(pvm, am + arr_stride);
                                    vload_smem<T, VW>(pvp, ap + arr_stride);
                                    if (KAHAN) {
                                        vload_smem<T, VW>(cvm, am + 2 * arr_stride);
                                        vload_smem<T, VW>(cvp, ap + 2 * arr_stride);
                                    }
#pragma unroll
                                    for (int i = 0; i < VW; ++i) {
                                        drift<T, KAHAN>(ym[i], cvm[i], pvm[i], cd);
                                        drift<T, KAHAN>(yp[i], cvp[i], pvp[i], cd);
                                    }
                                }
                            }
                            const T xm_edge = xm_lane ? xm_s : drifted1(sp, f, r + 1, xm_idx);
                            const T xp_edge = xp_lane ? xp_s : drifted1(sp, f, r + 1, xp_idx);
                            T gsum = (T)0;
#pragma unroll
                            for (int i = 0; i < VW; ++i) {
                                const T c = zmid[f][i];
                                const T xm = i == 0 ? xm_edge : zmid[f][i - 1];
                                const T xp = i == VW - 1 ? xp_edge : zmid[f][i + 1];
                                lap[f][i] = ((xp + xm) + (yp[i] + ym[i]) + (znew[f][i] + zlo[f][i])) - (T)6 * c;
                                const T gx = xp - c, gy = yp[i] - c, gz = znew[f][i] - c;
                                gsum += gx * gx + gy * gy + gz * gz;
                                phc[f][i] = c;
                            }
                            accG[f].add(gsum);
                        }
                    }
                    if (r < R) {
                        const size_t base = (size_t)(z0 + j - 2) * plane + row_off;
                        T vsum = (T)0;
#pragma unroll
                        for (int f = 0; f < NF; ++f) {
                            T po[VW], ksum = (T)0;
#pragma unroll
                            for (int i = 0; i < VW; ++i) {
                                const T p0 = phc[0][i];
                                const T p1 = NF > 1 ? phc[NF - 1][i] : (T)0;
                                T dV;
                                if (f == 0) dV = p0 * (P.m20 + P.l0 * p0 * p0 + (NF > 1 ? P.g2 * p1 * p1 : (T)0));
                                else dV = p1 * (P.m21 + P.l1 * p1 * p1 + P.g2 * p0 * p0);
                                const T F = cL * lap[f][i] - cV * dV;
                                const T pe = pcur[f][i] + ce * F;
                                po[i] = pcur[f][i] + ck * F;
                                ksum += pe * pe;
                                if (f == 0) {
                                    T v = p0 * p0 * (P.h_m20 + P.q_l0 * p0 * p0);
                                    if (NF > 1) v += p1 * p1 * (P.h_m21 + P.q_l1 * p1 * p1) + P.h_g2 * p0 * p0 * p1 * p1;
                                    vsum += v;
                                }
                            }
                            accK[f].add(ksum);
                            vstore<T, VW>(A.pi_out[f] + base, po);
                        }
                        accV.add(vsum);
                    }
                }
                if (j >= 1) release(st_prev);  // plane j-1: kicked (or the lower z halo, never kicked)
#pragma unroll
                for (int f = 0; f < NF; ++f)
#pragma unroll
                    for (int i = 0; i < VW; ++i) {
                        zlo[f][i] = zmid[f][i];
                        zmid[f][i] = znew[f][i];
                        pcur[f][i] = pnext[f][i];
                    }
                st_prev = st;
                st = st + 1 == S ? 0 : st + 1;
                zz = zz + 1 == N ? 0 : zz + 1;
            }
            release(st_prev);  // the upper z halo of the segment is never kicked
        }
    }
    __syncthreads();  // producer and consumers meet; no copy is in flight past this point
    finish_pass<T, NF>(A, accK, accG, accV, s_coef, s_red, &s_last, tid, nthr, s_timeout);
}
