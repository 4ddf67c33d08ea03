// Tensor-core (tcgen05) k-means assignment for the TF32 and BF16 modes.
// Internal header (not part of the ABI).
#pragma once

#include "common.cuh"

namespace cabs {

// Operand width (d rounded up to the 128-byte K chunk) and the conversion of
// an FP32 row-major matrix (rows x d) to K-major BF16 or TF32 operand rows of
// Kp elements, zero-padded; shared by the tensor-core assignment and snap.
int tc_kp_of(int d, bool tf32);
cabs_status tc_to_operand(const float* X, int64_t rows, int d, int Kp, bool tf32, void* out, const char* name,
                          cudaStream_t stream);

// CTAs of the assignment grid for M points.
int tc_assign_blocks(int64_t M);
// Extra workspace (operand copies, re-check flags) carved after the FP32 k-means slices.
void tc_assign_carve(Carve& cv, int64_t M, int d, int k2);
// labels[l] = argmin_j |z_j|^2 - 2 x_l.z_j with the contraction on tensor cores;
// rows whose two best distances are within the operand rounding bound are
// recomputed in FP32 (counted in *d_recheck).
// prep_points: convert the points to the operand format (once per k-means run).
cabs_status tc_assign_launch(const float* X, int64_t M, int d, const float* Z, const float* zn, int k2,
                             const float* xn, const float* w, int* labels, int* d_recheck, bool bf16,
                             bool prep_points, void* tcws, cudaStream_t stream);

}  // namespace cabs
