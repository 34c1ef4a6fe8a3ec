// Shared-memory staged axion-U(1) launches (u1_staged.cu).
#pragma once

#include "cl_internal.cuh"

namespace clk {

// what 0 = plaquette fields (and cos P into args cP when that is non-null), 1 = stage (or
// energies with P_ENERGY_ONLY), 2 = the fused stage (plaquette fields in shared memory, no
// plaquette launch), 3 = the E-dependent plaquette fields from a saved cos P (args cP), with
// the partial layout of
// launch_u1, on u1_staged_blocks(precision, N, dz) blocks of 32 x 16 (FP32) or 32 x 8 (FP64)
// tiles, each marching through dz planes; needs u1_staged_ok(N).
bool u1_staged_ok(int N);
int u1_staged_blocks(int precision, int N, int dz);
// The library's z chunk: one block per SM at a time, waves x (planes + 2) minimised.
int u1_staged_dz(int precision, int N, int nsm);
cudaError_t launch_u1_staged(int precision, const void* args, int what, cudaStream_t s);

}  // namespace clk
