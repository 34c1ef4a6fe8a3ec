// Steps of the TMA-staged, warp-specialized scalar pass as used by the ensemble kernel
// (ensemble_pass.cu): the producer's bulk copies of one plane and the consumers' drift /
// kick of one plane, with a ring of drifted rows or ringless.  Same protocol and register
// z-march as the single-lattice kernels (scalar_pass_tma.cuh and scalar_pass_tma_nr.cuh,
// which keep inline copies of these steps).
#pragma once

#include "cl_internal.cuh"
#include "kernel_common.cuh"
#include "scalar_pass_common.cuh"

namespace clk {

// Producer: the bulk copies of one plane zz of a tile -- own rows y0 .. y0+R-1 and the
// halo rows ylo, yhi -- of every input array into the stage buffer sb, laid out
// [array][BY+2 rows][N] with arrays arr_stride apart.  Lane l < 3 * arrays issues one copy.
template <typename T, int NF, bool KAHAN>
__device__ __forceinline__ void tma_issue_plane(int lane, T* sb, int arr_stride, const FieldSet<T>& F, int N, int zz,
                                                int y0, int R, int ylo, int yhi, uint64_t* full)
{
    constexpr int KPF = KAHAN ? 3 : 2;  // arrays per field in a stage: phi, pi (, c)
    constexpr int NARR = NF * KPF;
    if (lane < 3 * NARR) {
        const int a = lane / 3, part = lane - 3 * (lane / 3);
        const int f = a / KPF, kind = a - KPF * (a / KPF);
        // selects with constant indices only (a dynamic index would put F in local memory)
        const T* src = f == 0 ? (kind == 0 ? F.phi_in[0] : (kind == 1 ? F.pi_in[0] : F.c_in[0]))
                              : (kind == 0 ? F.phi_in[NF - 1] : (kind == 1 ? F.pi_in[NF - 1] : F.c_in[NF - 1]));
        const int y = part == 0 ? ylo : (part == 1 ? y0 : yhi);
        const int srow = part == 0 ? 0 : (part == 1 ? 1 : R + 1);
        const int nrows = part == 1 ? R : 1;
        T* dst = sb + a * arr_stride + srow * N;
        tma_bulk_g2s(dst, src + ((size_t)zz * N + y) * N, (uint32_t)(nrows * N * sizeof(T)), full);
    }
}

// Consumer geometry of one tile: thread (r, tx) owns vector tx of row r.
struct TileGeom {
    int N, TX, r, R, x0, xm_idx, xp_idx, arr_stride;
    bool xm_lane, xp_lane;  // x neighbour held by the adjacent lane (same row)
    __device__ __forceinline__ TileGeom(int N_, int VW, int BY, int R_, int tid)
    {
        N = N_;
        TX = N_ / VW;
        const bool own = tid < BY * TX;
        r = own ? tid / TX : BY;
        const int tx = own ? tid % TX : 0;
        R = R_;
        x0 = tx * VW;
        const int lane = tid & 31;
        xm_lane = own && lane > 0 && tx > 0;
        xp_lane = own && lane < 31 && tx < TX - 1;
        xm_idx = x0 == 0 ? N_ - 1 : x0 - 1;
        xp_idx = x0 + VW == N_ ? 0 : x0 + VW;
        arr_stride = (BY + 2) * N_;
    }
};

// Registers of the consumer z-march: drifted own vector of planes j-2, j-1, j and the
// momenta of planes j-1 (pcur) and j (pnext).
template <typename T, int NF, int VW>
struct ZMarch {
    T zlo[NF][VW], zmid[NF][VW], znew[NF][VW], pcur[NF][VW], pnext[NF][VW];
};

// Output arrays of the consumers, read from the kernel's parameters at each use (holding
// them in registers costs the z-march registers): phi(f), pi(f), c(f) for a single lattice
// and, with the member's element offset, for an ensemble member.
template <typename Args>
struct OutArrays {
    const Args& A;
    long long off;
    __device__ __forceinline__ auto phi(int f) const { return A.phi_out[f] + off; }
    __device__ __forceinline__ auto pi(int f) const { return A.pi_out[f] + off; }
    __device__ __forceinline__ auto c(int f) const { return A.c_out[f] + off; }
};

// Consumer step j of a tile: drift the plane in stage sb (own rows into registers and the
// new ring slot rs, halo rows into rs), write its phi (and c) at base_new when write_out,
// release the stage, meet the other consumers on named barrier 1, then (kick) kick the
// previous plane from ring slot rc and registers and write its pi at base_kick.
template <typename T, int NF, bool KAHAN, int VW, class Out>
__device__ __forceinline__ void tma_consume_plane(const TileGeom& G, const T* sb, T* rs, const T* rc, int tid, int CT,
                                                  bool do_drift, bool write_out, bool kick, size_t base_new,
                                                  size_t base_kick, const Out& F, const TileCoef<T>& C,
                                                  const PotCoef<T>& P, ZMarch<T, NF, VW>& Z, Acc<T> (&accK)[NF],
                                                  Acc<T> (&accG)[NF], Acc<T>& accV, uint64_t* empty)
{
    constexpr int KPF = KAHAN ? 3 : 2;
    const int N = G.N, r = G.r, R = G.R, x0 = G.x0, TX = G.TX, arr_stride = G.arr_stride;
    const int lane = tid & 31;
    if (r < R) {  // own rows: drift, write out, keep field and momenta in registers
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            T pv[VW], cv[VW];
            const T* sa = sb + f * KPF * arr_stride + (r + 1) * N + x0;
            vload_smem<T, VW>(Z.znew[f], sa);
            vload_smem<T, VW>(pv, sa + arr_stride);
            if (KAHAN) vload_smem<T, VW>(cv, sa + 2 * arr_stride);
            if (do_drift) {
#pragma unroll
                for (int i = 0; i < VW; ++i) drift<T, KAHAN>(Z.znew[f][i], cv[i], pv[i], C.cd);
            }
            vstore<T, VW>(rs + f * arr_stride + (r + 1) * N + x0, Z.znew[f]);
            if (write_out) {
                vstore<T, VW>(F.phi(f) + base_new, Z.znew[f]);
                if (KAHAN) vstore<T, VW>(F.c(f) + base_new, cv);
            }
#pragma unroll
            for (int i = 0; i < VW; ++i) Z.pnext[f][i] = pv[i];
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
            for (int i = 0; i < VW; ++i) drift<T, KAHAN>(ph[i], cv[i], pv[i], C.cd);
        }
        vstore<T, VW>(rs + f * arr_stride + srow * N + vx, ph);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(empty);  // this warp is done with the stage
    named_barrier_sync(1, CT);          // ring slot rs complete
    if (kick) {
        // kick the previous plane: centre zmid, z neighbours zlo / znew in registers
        T phc[NF][VW], lap[NF][VW];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            // every consumer lane takes part in the shuffles (idle lanes pass junk)
            T xm_s = __shfl_up_sync(0xffffffffu, Z.zmid[f][VW - 1], 1);
            T xp_s = __shfl_down_sync(0xffffffffu, Z.zmid[f][0], 1);
            if (r < R) {
                const T* Sc = rc + f * arr_stride + (r + 1) * N;
                T ym[VW], yp[VW];
                vload_smem<T, VW>(ym, Sc - N + x0);
                vload_smem<T, VW>(yp, Sc + N + x0);
                const T xm_edge = G.xm_lane ? xm_s : Sc[G.xm_idx];
                const T xp_edge = G.xp_lane ? xp_s : Sc[G.xp_idx];
                T gsum = (T)0;
#pragma unroll
                for (int i = 0; i < VW; ++i) {
                    const T c = Z.zmid[f][i];
                    const T xm = i == 0 ? xm_edge : Z.zmid[f][i - 1];
                    const T xp = i == VW - 1 ? xp_edge : Z.zmid[f][i + 1];
                    lap[f][i] = ((xp + xm) + (yp[i] + ym[i]) + (Z.znew[f][i] + Z.zlo[f][i])) - (T)6 * c;
                    const T gx = xp - c, gy = yp[i] - c, gz = Z.znew[f][i] - c;
                    gsum += gx * gx + gy * gy + gz * gz;
                    phc[f][i] = c;
                }
                accG[f].add(gsum);
            }
        }
        if (r < R) {
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
                    const T Fk = C.cL * lap[f][i] - C.cV * dV;
                    const T pe = Z.pcur[f][i] + C.ce * Fk;
                    po[i] = Z.pcur[f][i] + C.ck * Fk;
                    ksum += pe * pe;
                    if (f == 0) {
                        T v = p0 * p0 * (P.h_m20 + P.q_l0 * p0 * p0);
                        if (NF > 1) v += p1 * p1 * (P.h_m21 + P.q_l1 * p1 * p1) + P.h_g2 * p0 * p0 * p1 * p1;
                        vsum += v;
                    }
                }
                accK[f].add(ksum);
                vstore<T, VW>(F.pi(f) + base_kick, po);
            }
            accV.add(vsum);
        }
    }
    // march the register window up one plane
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int i = 0; i < VW; ++i) {
            Z.zlo[f][i] = Z.zmid[f][i];
            Z.zmid[f][i] = Z.znew[f][i];
            Z.pcur[f][i] = Z.pnext[f][i];
        }
}

// Ringless consumer step j of a tile (no ring, no named barrier): drift this thread's own
// row of the plane in stage sb into registers and write its phi (and c) at base_new when
// write_out; then (kick) kick the previous plane, whose stage sp is still held, drifting the
// y-neighbour rows again from sp with the same compensated arithmetic as their owners (so
// the values agree bit for bit) and taking x neighbours from adjacent lanes or, at row and
// warp ends, one drifted value from sp.  The caller releases sp after this step.
template <typename T, int NF, bool KAHAN, int VW, class Out>
__device__ __forceinline__ void tma_consume_plane_nr(const TileGeom& G, const T* sb, const T* sp, bool do_drift,
                                                     bool write_out, bool kick, size_t base_new, size_t base_kick,
                                                     const Out& F, const TileCoef<T>& C, const PotCoef<T>& P,
                                                     ZMarch<T, NF, VW>& Z, Acc<T> (&accK)[NF], Acc<T> (&accG)[NF],
                                                     Acc<T>& accV)
{
    constexpr int KPF = KAHAN ? 3 : 2;
    const int N = G.N, r = G.r, R = G.R, x0 = G.x0, arr_stride = G.arr_stride;
    // drifted value of field f at (stage row srow, column x) of stage buffer b
    auto drifted1 = [&](const T* b, int f, int srow, int x) -> T {
        const T* sa = b + f * KPF * arr_stride + srow * N + x;
        T ph = sa[0];
        if (do_drift) {
            T cv = KAHAN ? sa[2 * arr_stride] : (T)0;
            drift<T, KAHAN>(ph, cv, sa[arr_stride], C.cd);
        }
        return ph;
    };
    if (r < R) {  // own row of plane j: drift, write out, keep field and momenta in registers
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            T pv[VW], cv[VW];
            const T* sa = sb + f * KPF * arr_stride + (r + 1) * N + x0;
            vload_smem<T, VW>(Z.znew[f], sa);
            vload_smem<T, VW>(pv, sa + arr_stride);
            if (KAHAN) vload_smem<T, VW>(cv, sa + 2 * arr_stride);
            if (do_drift) {
#pragma unroll
                for (int i = 0; i < VW; ++i) drift<T, KAHAN>(Z.znew[f][i], cv[i], pv[i], C.cd);
            }
            if (write_out) {
                vstore<T, VW>(F.phi(f) + base_new, Z.znew[f]);
                if (KAHAN) vstore<T, VW>(F.c(f) + base_new, cv);
            }
#pragma unroll
            for (int i = 0; i < VW; ++i) Z.pnext[f][i] = pv[i];
        }
    }
    if (kick) {
        T phc[NF][VW], lap[NF][VW];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            // every consumer lane takes part in the shuffles (idle lanes pass junk)
            T xm_s = __shfl_up_sync(0xffffffffu, Z.zmid[f][VW - 1], 1);
            T xp_s = __shfl_down_sync(0xffffffffu, Z.zmid[f][0], 1);
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
                            drift<T, KAHAN>(ym[i], cvm[i], pvm[i], C.cd);
                            drift<T, KAHAN>(yp[i], cvp[i], pvp[i], C.cd);
                        }
                    }
                }
                const T xm_edge = G.xm_lane ? xm_s : drifted1(sp, f, r + 1, G.xm_idx);
                const T xp_edge = G.xp_lane ? xp_s : drifted1(sp, f, r + 1, G.xp_idx);
                T gsum = (T)0;
#pragma unroll
                for (int i = 0; i < VW; ++i) {
                    const T c = Z.zmid[f][i];
                    const T xm = i == 0 ? xm_edge : Z.zmid[f][i - 1];
                    const T xp = i == VW - 1 ? xp_edge : Z.zmid[f][i + 1];
                    lap[f][i] = ((xp + xm) + (yp[i] + ym[i]) + (Z.znew[f][i] + Z.zlo[f][i])) - (T)6 * c;
                    const T gx = xp - c, gy = yp[i] - c, gz = Z.znew[f][i] - c;
                    gsum += gx * gx + gy * gy + gz * gz;
                    phc[f][i] = c;
                }
                accG[f].add(gsum);
            }
        }
        if (r < R) {
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
                    const T Fk = C.cL * lap[f][i] - C.cV * dV;
                    const T pe = Z.pcur[f][i] + C.ce * Fk;
                    po[i] = Z.pcur[f][i] + C.ck * Fk;
                    ksum += pe * pe;
                    if (f == 0) {
                        T v = p0 * p0 * (P.h_m20 + P.q_l0 * p0 * p0);
                        if (NF > 1) v += p1 * p1 * (P.h_m21 + P.q_l1 * p1 * p1) + P.h_g2 * p0 * p0 * p1 * p1;
                        vsum += v;
                    }
                }
                accK[f].add(ksum);
                vstore<T, VW>(F.pi(f) + base_kick, po);
            }
            accV.add(vsum);
        }
    }
    // march the register window up one plane
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int i = 0; i < VW; ++i) {
            Z.zlo[f][i] = Z.zmid[f][i];
            Z.zmid[f][i] = Z.znew[f][i];
            Z.pcur[f][i] = Z.pnext[f][i];
        }
}

}  // namespace clk
