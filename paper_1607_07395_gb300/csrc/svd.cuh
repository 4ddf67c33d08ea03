// FP64-accurate SVD of the k x k core matrix (internal).
#pragma once

#include "common.cuh"
#include "grid_sync.cuh"

namespace cabs {

struct SvdWs {
  double *U[2], *V[2];                 // column-major iterates
  double *P, *T, *UtU, *VtV, *F, *G;   // k x k scratch
  double* d;                           // current singular value estimates
  unsigned long long* maxoff;          // per-iteration max |F|, |G| (i != j), then max |T_ij| over pairs kept undiagonalised (as ordered bits)
  int* done_iter;                      // first converged iteration, or INT_MAX
  int *pos, *rank_tmp;                 // descending position of each value; kept rank
  GridBarrier* bar;
  double *Wc, *Vc;                     // FP64 Jacobi fallback scratch
  float* qr;                           // FP32 phase: preconditioning QR reflectors
};

SvdWs carve_svd(Carve& cv, int k);

// W (k x k row-major, FP64) -> sig (k, descending), Uw, Vw (k x k row-major,
// column r = r-th singular vector, zero beyond the kept rank), *rank, *sweeps
// (FP32 Jacobi sweeps), *refine (FP64 refinement iterations, -1 when the FP64
// Jacobi fallback ran; may be NULL). The refinement may stop with a pair of
// values undiagonalised when both are at or below
// max(trunc_rtol, k 2^-52, resolve_rtol) sigma_1, or when its off-diagonal
// entries of U^T W V are at most max(1e-13, resolve_rtol) sigma_1:
// resolve_rtol = 0 for a W that is exact in FP64; the callers pass
// kResolveReduced for data carried in FP32 or less, whose own rounding is
// far above that level.
constexpr double kResolveReduced = 9.5367431640625e-07;  // 2^-20
cabs_status launch_svd(const double* W, int k, double trunc_rtol, double resolve_rtol, double* sig, double* Uw,
                       double* Vw, int* rank,
                       int* sweeps, int* refine, int* status, const SvdWs& w, cudaStream_t stream);

// One-CTA FP64 one-sided Jacobi; does nothing if *done_iter != INT_MAX
// (done_iter may be NULL: always run).
cabs_status launch_svd_jacobi_f64(const double* W, int k, double trunc_rtol, const int* done_iter, double* Wc,
                                  double* Vc, double* sig, double* Uw, double* Vw, int* rank, int* sweeps, int* status,
                                  cudaStream_t stream);

}  // namespace cabs
