// TMA-staged Runge-Kutta stage (rk_stage.cu): host-side entry points.
#pragma once

#include "cl_internal.cuh"

namespace clk {

// Dynamic shared memory of `stages` stage buffers: per field, the old field's rows y0-1 ..
// y0+BY and BY own rows of pi, the compensation (FP32 + Kahan) and k_phi, k_pi, one row more
// of the latter when the stage also sums the Ricci terms of its output (`ricci`).
size_t rk_stage_tma_smem(int precision, int nf, int N, int BY, int stages, bool ricci);
// One stage with the TMA-staged kernel: 16-byte vectors (vw * element size == 16), 3..6
// stages; work units as block_units (A.DZ > 0: grid A.nby * A.nbz; A.DZ < 0: grid A.nbz
// blocks with balanced ranges).  A.nmc == 2 (one field only): the non-minimal stage that also
// writes the background Ricci scalar of its output state to scal->rbar (partials: two sets of
// kMaxQ per block).
cudaError_t launch_rk_stage_tma(int precision, int nf, const void* args, int vw, int stages, cudaStream_t s);
// One stage on a reduced lattice of N^dims sites (dims = 1, 2; no non-minimal coupling),
// `grid` blocks of 256 threads (partials[grid][kMaxQ]).
cudaError_t launch_reduced_rk_stage(int precision, int nf, const void* args, int dims, int grid, cudaStream_t s);

}  // namespace clk
