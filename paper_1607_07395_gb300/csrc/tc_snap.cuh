// Tensor-core (tcgen05) candidate search of the snap for the BF16 and TF32
// modes. Internal header (not part of the ABI).
#pragma once

#include "common.cuh"

namespace cabs {

// Whether the tensor-core candidate search handles these sizes.
bool tc_snap_supported(int64_t M, int d, int k2, bool tf32);
// Workspace of tc_snap_candidates.
size_t tc_snap_ws_bytes(int64_t M, int d, int k2);
// For every centre j < k2: its 8 nearest rows of X (M x d, FP32) by direct
// FP32 distance (summed in dimension order, as the CUDA-core candidate
// kernel does) among the 32 best by the tensor-core ranking |x|^2 - 2 x.z,
// in (distance, row) order: top_d[j * 8 + t], top_r[j * 8 + t] (rows past the
// end, if M < 8, are 0x7fffffff with an infinite distance).
cabs_status tc_snap_candidates(const float* X, int64_t M, int d, const float* Z, int k2, bool tf32, float* top_d,
                               int* top_r, void* ws, size_t ws_bytes, cudaStream_t stream);

}  // namespace cabs
