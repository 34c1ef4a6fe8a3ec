// TMA-staged, warp-specialized variant of the fused scalar pass with register
// z-marching (included by scalar_pass.cu after the shared device functions).
//
// Block = C consumer warps (own rows: thread (r, tx) owns vector tx of row r) plus one
// producer warp.  The producer copies every plane (own rows and the two halo rows of
// every input array) into a ring of S stage buffers with bulk TMA copies that complete
// on the stage's "full" mbarrier; it refills a stage once every consumer warp has
// arrived on the stage's "empty" mbarrier.  It runs ahead over all segments of the
// block, so the next segment's planes are already in flight when a segment ends.
//
// Consumers drift plane j from its stage (own rows into registers, own and halo rows
// into a 3-slot ring of drifted fields), meet on one named barrier, then kick plane
// j-1.  Each thread keeps the drifted values of its own vector for planes j-2, j-1, j
// in registers (z-marching), takes x neighbours from the neighbouring lanes by warp
// shuffles (shared memory only across warp or row edges) and reads just the two y
// neighbour vectors from the ring.  With three ring slots the drift of plane j+1 never
// touches the slot the kick of plane j-1 reads, so one consumer barrier per plane
// suffices.  Halo-row drift work is spread evenly over the consumer threads.  All
// mbarrier waits are bounded.  (The ensemble kernel runs the same protocol through the
// shared steps of tma_pipeline.cuh; this kernel keeps its own inline copy, which measured
// about 2% faster on the 256^3 two-field pass than the version built on those steps.)

template <typename T, int NF, bool KAHAN, int VW, int S>
__global__ void __launch_bounds__(512, 1) k_scalar_pass_tma(const ScalarPassArgs<T> A)
{
    constexpr int KPF = KAHAN ? 3 : 2;  // arrays per field in a stage: phi, pi (, c)
    constexpr int NARR = NF * KPF;
    constexpr int RING = 3;
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
    const int arr_stride = (BY + 2) * N;  // elements of one array in one stage / ring slot
    const int stage_stride = NARR * arr_stride;
    T* stage = reinterpret_cast<T*>(smem_raw);
    T* ring = stage + S * stage_stride;  // [RING][NF][BY+2][N] drifted fields
    const int ring_slot = NF * arr_stride;
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
        int st = 0;                // stage of the next plane
        uint32_t empty_phase = 0;  // bit s: parity of the next phase of s_empty[s] to wait for
        int issued = 0;            // planes issued so far (the first S need no wait)
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
                if (issued >= S) {  // wait until every consumer warp released the previous use
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
        // x neighbours from the adjacent lane when it holds the adjacent vector of the same row
        const bool own = tid < BY * TX;
        const bool xm_lane = own && lane > 0 && tx > 0;
        const bool xp_lane = own && lane < 31 && tx < TX - 1;
        const int xm_idx = x0 == 0 ? N - 1 : x0 - 1;
        const int xp_idx = x0 + VW == N ? 0 : x0 + VW;
        T pcur[NF][VW], pnext[NF][VW];
        T zlo[NF][VW], zmid[NF][VW], znew[NF][VW];  // drifted own vector of planes j-2, j-1, j
        int st = 0;               // stage of the next plane
        uint32_t full_phase = 0;  // bit s: parity of the next phase of s_full[s]
        int rnew = 0, rmid = RING - 1;  // ring slots of planes j and j-1
        const size_t plane = (size_t)N * N;
        for (long long u = u0; u < u1;) {
            const int tile = (int)(u / N);
            const int z0 = (int)(u - (long long)tile * N);
            const int NZ = (int)min((long long)(N - z0), u1 - u);
            const int y0 = tile * BY, R = min(BY, N - y0);
            u += NZ;
            int zz = z0 == 0 ? N - 1 : z0 - 1;                       // plane of iteration j
            const size_t row_off = (size_t)(y0 + r) * N + x0;          // own vector within a plane
            for (int j = 0; j < NZ + 2; ++j) {
                if (!mbar_wait_bounded(&s_full[st], (full_phase >> st) & 1u, s_timeout ? 1000000ull : 2000000000ull))
                    s_timeout = 1;
                full_phase ^= 1u << st;
                const T* sb = stage + st * stage_stride;
                T* rs = ring + rnew * ring_slot;
                const bool write_out = j >= 1 && j <= NZ;
                if (r < R) {  // own rows: drift, write out, keep field and momenta in registers
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
                        vstore<T, VW>(rs + f * arr_stride + (r + 1) * N + x0, znew[f]);
                        if (write_out) {
                            vstore<T, VW>(A.phi_out[f] + base, znew[f]);
                            if (KAHAN) vstore<T, VW>(A.c_out[f] + base, cv);
                        }
#pragma unroll
                        for (int i = 0; i < VW; ++i) pnext[f][i] = pv[i];
                    }
                }
                // halo rows: NF * 2 * TX vector items spread over all consumer threads
                for (int h = tid; h < NF * 2 * TX; h += CT) {
                    const int f = h / (2 * TX), hv = h - f * 2 * TX;
                    const int sel = hv / TX, vx = (hv - sel * TX) * VW;
                    const int srow = sel == 0 ? 0 : R + 1;
                    T ph[VW], pv[VW], cv[VW];
                    const T* sa = sb + f * KPF * arr_stride + srow * N + vx;
                    vload_smem<T, VW>(ph, sa);
                    if (do_drift) {
                        vload_smem<T, VW>(pv, sa + arr_stride);
                        if (KAHAN) vload_smem<T, VW>(cv, sa + 2 * arr_stride);
#pragma unroll
                        for (int i = 0; i < VW; ++i) drift<T, KAHAN>(ph[i], cv[i], pv[i], cd);
                    }
                    vstore<T, VW>(rs + f * arr_stride + srow * N + vx, ph);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&s_empty[st]);  // this warp is done with the stage
                named_barrier_sync(1, CT);                   // ring slot rnew complete
                if (j >= 2) {
                    // kick plane j-1: centre zmid, z neighbours zlo / znew in registers
                    const T* rc = ring + rmid * ring_slot;
                    T phc[NF][VW], lap[NF][VW];
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        // every consumer lane takes part in the shuffles (idle lanes pass junk)
                        T xm_s = __shfl_up_sync(0xffffffffu, zmid[f][VW - 1], 1);
                        T xp_s = __shfl_down_sync(0xffffffffu, zmid[f][0], 1);
                        if (r < R) {
                            const T* Sc = rc + f * arr_stride + (r + 1) * N;
                            T ym[VW], yp[VW];
                            vload_smem<T, VW>(ym, Sc - N + x0);
                            vload_smem<T, VW>(yp, Sc + N + x0);
                            const T xm_edge = xm_lane ? xm_s : Sc[xm_idx];
                            const T xp_edge = xp_lane ? xp_s : Sc[xp_idx];
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
                // march the register window up one plane
#pragma unroll
                for (int f = 0; f < NF; ++f)
#pragma unroll
                    for (int i = 0; i < VW; ++i) {
                        zlo[f][i] = zmid[f][i];
                        zmid[f][i] = znew[f][i];
                        pcur[f][i] = pnext[f][i];
                    }
                rmid = rnew;
                rnew = rnew + 1 == RING ? 0 : rnew + 1;
                st = st + 1 == S ? 0 : st + 1;
                zz = zz + 1 == N ? 0 : zz + 1;
            }
        }
    }
    __syncthreads();  // producer and consumers meet; no copy is in flight past this point
    finish_pass<T, NF>(A, accK, accG, accV, s_coef, s_red, &s_last, tid, nthr, s_timeout);
}
