// Step a3 -- the SVD W = U_w Sigma_w V_w^T of the k x k intersection matrix
// (Section 4.1), computed to FP64 accuracy.
//
// FP64 arithmetic on this GPU runs at 1/64 of the FP32 rate, and an SVD of a
// few hundred columns is latency-bound, so the work is split:
//
//  Phase A (FP32, Jacobi): one-sided (Hestenes) Jacobi on an FP32 copy of W,
//    run to convergence. For k <= 64 one CTA holds W and V in shared memory
//    and processes the k/2 disjoint pairs of each round-robin round on its
//    warps. For larger k a thread-block cluster holds the columns in the
//    shared memories of its CTAs, and the Jacobi starts from X = W Q, V = Q
//    with W^T = Q R (a blocked Householder QR across the cluster), so that
//    X = R^T: this preconditioning cuts the sweeps by a third to a half
//    (a W with zero rows starts from W itself). Each
//    CTA owns two blocks of columns, rotates
//    every pair across them (and, once per sweep, the pairs inside them), then
//    the blocks move one step along the round-robin circle through distributed
//    shared memory; one cluster barrier per round, double-buffered. In the
//    cross-block steps a warp keeps its top column in registers for the whole
//    round, and the same warp applies each step's rotation to the V columns
//    one step later, off the dependent chain of W rotations (measured on
//    GB300: slightly faster than giving V its own warps, which compete with
//    the W chain for issue slots).
//  Phase B (FP64, refinement): from U0, V0, iterate
//      T = U^T W V,  R = I - U^T U,  S = I - V^T V,
//      d_i = T_ii / (1 - (R_ii + S_ii) / 2),
//      for i != j with a = T_ij + d_j R_ij, b = T_ji + d_j S_ij:
//        F_ij = (a d_j + b d_i) / (d_j^2 - d_i^2),  G_ij = (a d_i + b d_j) / (d_j^2 - d_i^2),
//      F_ii = R_ii / 2, G_ii = S_ii / 2;  U <- U + U F,  V <- V + V G,
//    which solves the first-order conditions U'^T U' = I, V'^T V' = I and
//    U'^T W V' diagonal, and so converges quadratically. Before the first
//    iteration the kept columns of U are recomputed in FP64 as W V / |W V|
//    (and, where W has zero rows, the others completed to span R^k). Every
//    product is an FP64 GEMM spread over all SMs. Pairs with d_i^2 ~ d_j^2,
//    or whose correction would exceed 0.05 (values not yet separated by more
//    than the estimates' error), keep only the orthogonality correction;
//    a pair with d_i ~ d_j clearly above zero (a repeated value) also gets
//    the rotation that makes U and V agree inside it. The iteration has
//    converged when its corrections are small and every close pair left
//    undiagonalised has |T_ij| at the rounding level of the input.
//    Iteration t's kernels exit at once if an earlier iteration already
//    converged (a device-side flag; no host sync).
//  Fallback: if Phase B has not converged after its iterations, the one-CTA
//    FP64 Jacobi SVD runs instead (status bit 1).
// The result is sorted by singular value and truncated as before.
#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels.cuh"
#include "profile.cuh"
#include "grid_sync.cuh"
#include "svd.cuh"

namespace cg = cooperative_groups;

namespace cabs {
namespace {

constexpr int kCtaMaxK = 64;           // one-CTA Phase A up to this k
#ifndef CABS_SVD_TOL_A
#define CABS_SVD_TOL_A 1e-5f
#endif
constexpr float kTolA = CABS_SVD_TOL_A;  // Phase A rotation threshold |g| > tol sqrt(a b)
// Phase A stops after a sweep in which no pair had |g| > kStopA sqrt(a b):
// cyclic Jacobi converges quadratically there, so the factors are then
// orthogonal to about kStopA^2 (a CPU model of the kernel on the sketching
// workloads: largest |g| / sqrt(a b) per sweep 0.03, 8e-3, 7e-4, 1e-5), and
// the quadratically convergent FP64 refinement takes them from there. A stop
// at 1e-2 saved a sweep on the sketch cores but left the refinement of the
// SVD form's k x k products (Section 3 orthogonalisation) unconverged after
// its iterations, so that the FP64 Jacobi fallback ran; 1e-3 converges there.
#ifndef CABS_SVD_STOP_A
#define CABS_SVD_STOP_A 1e-3f
#endif
constexpr float kStopA = CABS_SVD_STOP_A;
constexpr int kMaxSweepsA = 40;
constexpr int kItersB = 8;
constexpr double kMaxCorrB = 0.05;      // Phase B: larger first-order corrections are deferred
constexpr double kConvB = 1e-8;         // Phase B: last iteration when max |F_ij|, |G_ij| (i != j) < this
constexpr double kCloseOffB = 1e-13;    // ... and |T_ij| < this max |d| for every pair left undiagonalised
constexpr int kNotDone = 0x7fffffff;

__device__ __forceinline__ void rr_pair(int round, int pr, int kk, int& p, int& q) {
  if (pr == 0) {
    p = round;
    q = kk - 1;
  } else {
    p = (round + pr) % (kk - 1);
    q = (round - pr + kk - 1) % (kk - 1);
  }
  if (p > q) {
    const int t = p;
    p = q;
    q = t;
  }
}

// The Hestenes rotation that makes two columns with squared norms a, b and
// inner product g orthogonal, |angle| <= pi/4: with d = b - a and
// r = sqrt(d^2 + 4 g^2), cos 2t = |d| / r, so c = sqrt((1 + |d| / r) / 2) and
// s = sign(d) g / (r c) (the same c, s as t = sign(zeta) / (|zeta| +
// sqrt(1 + zeta^2)), zeta = d / 2g, c = 1 / sqrt(1 + t^2), s = c t). Two
// reciprocal square roots and no division or branch keep the dependent
// chain of a rotation step short; c^2 + s^2 = 1 up to rounding, and Phase A
// needs only approximate rotations (the FP64 refinement finishes the job).
// Returns 0 (c = 1, s = 0: no rotation) unless |g| > tol sqrt(a b), tested as
// g^2 > tol^2 a b; else 1, or 3 when |g| > kStopA sqrt(a b) (the sweep is
// not the last one). c and s depend only on the ratio d : g, so d and g are
// first scaled by 2^-100 or 2^100 when the larger of them is above 1e18 or
// below 1e-18, keeping d^2 + 4 g^2 clear of overflow and of the subnormal
// range.
__device__ __forceinline__ int jacobi_cs(float a, float b, float g, float& c, float& s) {
  const float ab = a * b, g2 = g * g;
  const float big = fmaxf(fabsf(b - a), fabsf(g));
  const float sc = big > 1e18f ? 7.888609052210118e-31f : (big < 1e-18f ? 1.2676506002282294e30f : 1.f);
  const float d = (b - a) * sc, gs = g * sc;
  const float q1 = rsqrtf(fmaf(4.f * gs, gs, d * d));
  const float h = fmaf(0.5f * fabsf(d), q1, 0.5f);
  const float q2 = rsqrtf(h);
  const float sg = (d < 0.f ? -gs : gs) * q1;
  const int code = g2 > kTolA * kTolA * ab ? (g2 > kStopA * kStopA * ab ? 3 : 1) : 0;
  c = code ? h * q2 : 1.f;
  s = code ? sg * q2 : 0.f;
  return code;
}

// Rotates columns x, y (length k, lane-strided) so that they become
// orthogonal; returns jacobi_cs's code (0: no rotation). x, y, vx, vy may
// live in shared or distributed shared memory.
__device__ __forceinline__ int rotate_pair_f32(float* x, float* y, float* vx, float* vy, int k, int lane) {
  float a = 0.f, b = 0.f, g = 0.f;
  for (int i = lane; i < k; i += 32) {
    const float u = x[i], v = y[i];
    a = fmaf(u, u, a);
    b = fmaf(v, v, b);
    g = fmaf(u, v, g);
  }
  a = warp_sum(a);
  b = warp_sum(b);
  g = warp_sum(g);
  float c, s;
  const int code = jacobi_cs(a, b, g, c, s);
  if (!code) return 0;
  for (int i = lane; i < k; i += 32) {
    const float u = x[i], v = y[i];
    x[i] = c * u - s * v;
    y[i] = s * u + c * v;
    const float p = vx[i], q = vy[i];
    vx[i] = c * p - s * q;
    vy[i] = s * p + c * q;
  }
  return code;
}

// Same rotation with each lane owning R rows of a column padded to 32 R
// entries (R a multiple of 4), as R / 4 float4 groups interleaved across the
// lanes (group i of lane l at float4 index l + 32 i, so a warp's 16-byte
// accesses are consecutive and free of bank conflicts): the two columns are
// read once, rotated in registers and written back once.
template <int R>
__device__ __forceinline__ int rotate_pair_reg(float* x, float* y, float* vx, float* vy, int lane) {
  float xr[R], yr[R];
  const float4* x4 = (const float4*)x;
  const float4* y4 = (const float4*)y;
  // the V columns are read up front, so their latency hides behind the reductions
  float4 pv[R / 4], qv[R / 4];
  const float4* vx4 = (const float4*)vx;
  const float4* vy4 = (const float4*)vy;
#pragma unroll
  for (int i = 0; i < R / 4; ++i) {
    const float4 a = x4[lane + 32 * i], b = y4[lane + 32 * i];
    xr[4 * i] = a.x; xr[4 * i + 1] = a.y; xr[4 * i + 2] = a.z; xr[4 * i + 3] = a.w;
    yr[4 * i] = b.x; yr[4 * i + 1] = b.y; yr[4 * i + 2] = b.z; yr[4 * i + 3] = b.w;
  }
#pragma unroll
  for (int i = 0; i < R / 4; ++i) {
    pv[i] = vx4[lane + 32 * i];
    qv[i] = vy4[lane + 32 * i];
  }
  float a = 0.f, b = 0.f, g = 0.f;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    a = fmaf(xr[i], xr[i], a);
    b = fmaf(yr[i], yr[i], b);
    g = fmaf(xr[i], yr[i], g);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, off);
    b += __shfl_xor_sync(0xffffffffu, b, off);
    g += __shfl_xor_sync(0xffffffffu, g, off);
  }
  float c, s;
  const int code = jacobi_cs(a, b, g, c, s);
  if (!code) return 0;
  float4* xo = (float4*)x;
  float4* yo = (float4*)y;
#pragma unroll
  for (int i = 0; i < R / 4; ++i) {
    float4 p, q;
    p.x = c * xr[4 * i] - s * yr[4 * i];         q.x = s * xr[4 * i] + c * yr[4 * i];
    p.y = c * xr[4 * i + 1] - s * yr[4 * i + 1]; q.y = s * xr[4 * i + 1] + c * yr[4 * i + 1];
    p.z = c * xr[4 * i + 2] - s * yr[4 * i + 2]; q.z = s * xr[4 * i + 2] + c * yr[4 * i + 2];
    p.w = c * xr[4 * i + 3] - s * yr[4 * i + 3]; q.w = s * xr[4 * i + 3] + c * yr[4 * i + 3];
    xo[lane + 32 * i] = p;
    yo[lane + 32 * i] = q;
  }
  float4* vxo = (float4*)vx;
  float4* vyo = (float4*)vy;
#pragma unroll
  for (int i = 0; i < R / 4; ++i) {
    const float4 p = pv[i], q = qv[i];
    float4 p2, q2;
    p2.x = c * p.x - s * q.x; q2.x = s * p.x + c * q.x;
    p2.y = c * p.y - s * q.y; q2.y = s * p.y + c * q.y;
    p2.z = c * p.z - s * q.z; q2.z = s * p.z + c * q.z;
    p2.w = c * p.w - s * q.w; q2.w = s * p.w + c * q.w;
    vxo[lane + 32 * i] = p2;
    vyo[lane + 32 * i] = q2;
  }
  return code;
}

template <int R>
__device__ __forceinline__ void load_col(const float* x, int lane, float* xr) {
  const float4* x4 = (const float4*)x;
#pragma unroll
  for (int i = 0; i < R / 4; ++i) {
    const float4 a = x4[lane + 32 * i];
    xr[4 * i] = a.x; xr[4 * i + 1] = a.y; xr[4 * i + 2] = a.z; xr[4 * i + 3] = a.w;
  }
}

template <int R>
__device__ __forceinline__ void store_col(float* x, int lane, const float* xr) {
  float4* x4 = (float4*)x;
#pragma unroll
  for (int i = 0; i < R / 4; ++i) x4[lane + 32 * i] = make_float4(xr[4 * i], xr[4 * i + 1], xr[4 * i + 2], xr[4 * i + 3]);
}

// One step of a block round for a warp. kW: the rotation of rotate_pair_reg
// with column x held in registers (xr) and column y in shared memory, (c, s)
// recorded in *cs_out ((1, 0) when the pair is already orthogonal to the
// tolerance). The squared norms travel with the columns -- a in a register,
// b in shared memory at *bn -- and are updated by the exact identities
// |c x - s y|^2 = c^2 a - 2 c s g + s^2 b and |s x + c y|^2 = s^2 a + 2 c s g
// + c^2 b, so a step reduces only the inner product g across the warp (they
// are recomputed from the columns at the start of every round). kV: the V
// columns (vx, vy) take the rotation recorded one step earlier (*cs_prev).
// Both sit in one branch-free block, so that the V columns' loads, rotation
// and stores fill the latency of the warp sum; a pair below the threshold
// gets c = 1, s = 0, which leaves columns and norms as they are.
template <int R, bool kW, bool kV>
__device__ __forceinline__ int rotate_step(float* xr, float& a, float* y, float* bn, float2* cs_out, float* vx,
                                           float* vy, const float2* cs_prev, int lane) {
  float pr[R], qr[R], yr[R];
  float2 cp = make_float2(1.f, 0.f);
  if constexpr (kV) {
    cp = *cs_prev;
    load_col<R>(vx, lane, pr);
    load_col<R>(vy, lane, qr);
  }
  float b = 0.f, g = 0.f;
  if constexpr (kW) {
    load_col<R>(y, lane, yr);
    // every lane reads b before the shuffles below, which lane 0 must pass
    // before it overwrites *bn
    b = *bn;
#pragma unroll
    for (int i = 0; i < R; ++i) g = fmaf(xr[i], yr[i], g);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) g += __shfl_xor_sync(0xffffffffu, g, off);
  }
  if constexpr (kV) {
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const float p = pr[i], q = qr[i];
      pr[i] = cp.x * p - cp.y * q;
      qr[i] = cp.y * p + cp.x * q;
    }
    store_col<R>(vx, lane, pr);
    store_col<R>(vy, lane, qr);
  }
  int code = 0;
  if constexpr (kW) {
    float c, s;
    code = jacobi_cs(a, b, g, c, s);
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const float u = xr[i], v = yr[i];
      xr[i] = c * u - s * v;
      yr[i] = s * u + c * v;
    }
    store_col<R>(y, lane, yr);
    const float cc = c * c, ss = s * s, cs2 = 2.f * c * s * g;
    const float a2 = cc * a - cs2 + ss * b;
    if (lane == 0) {
      *bn = ss * a + cs2 + cc * b;
      *cs_out = make_float2(c, s);
    }
    a = a2;
  }
  return code;
}

// Squared norm of a column held as in load_col.
template <int R>
__device__ __forceinline__ float col_sq(const float* xr) {
  float a = 0.f;
#pragma unroll
  for (int i = 0; i < R; ++i) a = fmaf(xr[i], xr[i], a);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
  return a;
}

// Writes U0 (normalised columns) and V0 in FP64, column-major k x k.
__device__ __forceinline__ void emit_column(const float* w, const float* v, int k, int gc, int lane, double* U0,
                                            double* V0) {
  float a = 0.f;
  for (int i = lane; i < k; i += 32) a = fmaf(w[i], w[i], a);
  a = warp_sum(a);
  const float nrm = sqrtf(a);
  const float inv = nrm > 0.f ? 1.f / nrm : 0.f;
  for (int i = lane; i < k; i += 32) {
    U0[(size_t)gc * k + i] = (double)(w[i] * inv);
    V0[(size_t)gc * k + i] = (double)v[i];
  }
}

// Preconditioning QR (below): the panel of CTA p is its two blocks, top
// then bottom, i.e. panel positions 2 b p + t, t < 2 b. Position -> column of
// W^T (a row of W); >= k (or past the 2 NC blocks) is padding.
__device__ __forceinline__ int panel_col(int pos, int b, int NC) {
  const int pw = 2 * b, P = pos / pw, t = pos - P * pw;
  if (P >= NC) return 0x7fffffff;
  return (t < b ? P : 2 * NC - 1 - P) * b + (t < b ? t : t - b);
}

// emit_column for a W column whose rows are panel positions (the
// preconditioned cluster kernel): row pos of w is row panel_col(pos) of U0.
__device__ __forceinline__ void emit_column_perm(const float* w, const float* v, int k, int kp, int b, int NC, int gc,
                                                 int lane, double* U0, double* V0) {
  float a = 0.f;
  for (int i = lane; i < kp; i += 32) a = fmaf(w[i], w[i], a);
  a = warp_sum(a);
  const float nrm = sqrtf(a);
  const float inv = nrm > 0.f ? 1.f / nrm : 0.f;
  for (int pos = lane; pos < kp; pos += 32) {
    const int r = panel_col(pos, b, NC);
    if (r < k) U0[(size_t)gc * k + r] = (double)(w[pos] * inv);
  }
  for (int i = lane; i < k; i += 32) V0[(size_t)gc * k + i] = (double)v[i];
}

// ---------------------------------------------------------- Phase A, 1 CTA

__global__ void __launch_bounds__(512) svd32_cta_kernel(const double* __restrict__ W, int k, double* __restrict__ U0,
                                                         double* __restrict__ V0, int* sweeps_out) {
  extern __shared__ __align__(16) float s32[];
  float* Wc = s32;                    // column-major k x k
  float* Vc = s32 + (size_t)k * k;
  __shared__ int rotated;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  for (int e = tid; e < k * k; e += blockDim.x) {
    const int i = e / k, j = e - i * k;
    Wc[(size_t)j * k + i] = (float)W[e];
    Vc[e] = (i == j) ? 1.f : 0.f;
  }
  if (tid == 0) rotated = 0;
  __syncthreads();
  const int kk = k + (k & 1);
  int sweep = 0;
  bool conv = k < 2;
  while (!conv && sweep < kMaxSweepsA) {
    for (int round = 0; round < kk - 1; ++round) {
      for (int pr = warp; pr < kk / 2; pr += nwarps) {
        int p, q;
        rr_pair(round, pr, kk, p, q);
        if (q >= k) continue;
        const int code =
            rotate_pair_f32(Wc + (size_t)p * k, Wc + (size_t)q * k, Vc + (size_t)p * k, Vc + (size_t)q * k, k, lane);
        if (code && lane == 0) atomicOr(&rotated, code);
      }
      __syncthreads();
    }
    ++sweep;
    const int any = rotated;
    __syncthreads();
    if (tid == 0) rotated = 0;
    __syncthreads();
    conv = (any & 2) == 0;  // no rotation, or only small ones (kStopA)
  }
  for (int j = warp; j < k; j += nwarps) emit_column(Wc + (size_t)j * k, Vc + (size_t)j * k, k, j, lane, U0, V0);
  if (tid == 0 && sweeps_out) *sweeps_out = sweep;
}

// ------------------------------------------------------- Phase A, cluster

constexpr int kClusterThreads = 512;
constexpr int kMaxBlkRot = 16;  // columns per block (b) the cluster kernel supports

// Householder QR of one panel of pw = 2 b <= 32 columns held in shared
// memory (the block at base, then the one at base + blk; kp = 32 R rows, b
// columns each, the top block's real columns ntop). The real columns take the
// diagonal rows row0, row0 + 1, ... in panel order (padding columns are zero
// and take none), so the k real columns of W^T P use rows 0 ... k - 1 once
// each. Warp w keeps columns w and w + 16 in registers (lane l owns rows
// l + 32 i). Step t: the warp holding column t forms v from its rows >= row0
// + t (alpha = -sign(x0) |x|, v0 = x0 - alpha, beta = 2 / v^T v = -1 /
// (alpha v0)), stores v (zero above the diagonal) and beta for the other
// CTAs, and every later column takes y <- y - beta (v^T y) v. A remaining
// squared norm at or below 1e-36 (where beta would overflow) gives beta = 0
// and no reflection. On return each column holds R's column: the entries
// above the diagonal, alpha on it, zeros below.
template <int R>
__device__ void factor_panel(float* base, int b, size_t blk, int row0, int ntop, float* vout, float* beta, int warp,
                             int lane) {
  constexpr int kp = 32 * R;
  const int pw = 2 * b;
  auto col = [&](int t) { return base + (t < b ? (size_t)t * kp : blk + (size_t)(t - b) * kp); };
  float xr[2][R];
  const int nloc = (warp < pw ? 1 : 0) + (warp + 16 < pw ? 1 : 0);
#pragma unroll
  for (int h = 0; h < 2; ++h)
    if (h < nloc)
#pragma unroll
      for (int i = 0; i < R; ++i) xr[h][i] = col(warp + 16 * h)[lane + 32 * i];
  for (int t = 0; t < pw; ++t) {
    const int row = t < b ? row0 + t : row0 + ntop + (t - b);
    if (warp == (t & 15)) {
      const int h = t >> 4;
      float x[R];
#pragma unroll
      for (int i = 0; i < R; ++i) x[i] = h == 0 ? xr[0][i] : xr[1][i];
      float sq = 0.f, x0l = 0.f;
#pragma unroll
      for (int i = 0; i < R; ++i) {
        const int r = lane + 32 * i;
        if (r >= row) sq = fmaf(x[i], x[i], sq);
        if (r == row) x0l = x[i];
      }
      sq = warp_sum(sq);
      const float x0 = __shfl_sync(0xffffffffu, x0l, row & 31);
      float al = x0, be = 0.f, v0 = 0.f;
      if (sq > 1e-36f) {
        al = -copysignf(sqrtf(sq), x0);
        v0 = x0 - al;  // |x0| + |alpha|: no cancellation
        be = -1.f / (al * v0);
      }
      float* v = vout + (size_t)t * kp;
#pragma unroll
      for (int i = 0; i < R; ++i) {
        const int r = lane + 32 * i;
        v[r] = (be == 0.f || r < row) ? 0.f : (r == row ? v0 : x[i]);
        x[i] = r < row ? x[i] : (r == row ? al : 0.f);
      }
      if (lane == 0) beta[t] = be;
#pragma unroll
      for (int i = 0; i < R; ++i) {
        if (h == 0) xr[0][i] = x[i];
        else xr[1][i] = x[i];
      }
    }
    __syncthreads();
    const float be = beta[t];
    if (be != 0.f) {
      const float* v = vout + (size_t)t * kp;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h < nloc && warp + 16 * h > t) {
          float vr[R], d = 0.f;
#pragma unroll
          for (int i = 0; i < R; ++i) {
            vr[i] = v[lane + 32 * i];
            d = fmaf(vr[i], xr[h][i], d);
          }
          d = warp_sum(d) * be;
#pragma unroll
          for (int i = 0; i < R; ++i) xr[h][i] = fmaf(-d, vr[i], xr[h][i]);
        }
      }
    }
  }
#pragma unroll
  for (int h = 0; h < 2; ++h)
    if (h < nloc)
#pragma unroll
      for (int i = 0; i < R; ++i) col(warp + 16 * h)[lane + 32 * i] = xr[h][i];
}

// y <- H_{pw-1} ... H_0 y for a panel's reflectors (v zero above its
// diagonal, so no masks); y (32 R rows) in registers, lane l owning rows
// l + 32 i.
// Two columns at a time (y2 may be null), so that their reductions overlap.
template <int R>
__device__ __forceinline__ void apply_panel(const float* V, const float* beta, int pw, float* y1, float* y2,
                                            int lane) {
  constexpr int kp = 32 * R;
  float yr[R], zr[R];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    yr[i] = y1[lane + 32 * i];
    zr[i] = y2 ? y2[lane + 32 * i] : 0.f;
  }
  for (int t = 0; t < pw; ++t) {
    const float be = beta[t];
    if (be == 0.f) continue;
    const float* v = V + (size_t)t * kp;
    float vr[R], d = 0.f, e = 0.f;
#pragma unroll
    for (int i = 0; i < R; ++i) {
      vr[i] = v[lane + 32 * i];
      d = fmaf(vr[i], yr[i], d);
      e = fmaf(vr[i], zr[i], e);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      d += __shfl_xor_sync(0xffffffffu, d, off);
      e += __shfl_xor_sync(0xffffffffu, e, off);
    }
    d *= be;
    e *= be;
#pragma unroll
    for (int i = 0; i < R; ++i) {
      yr[i] = fmaf(-d, vr[i], yr[i]);
      zr[i] = fmaf(-e, vr[i], zr[i]);
    }
  }
#pragma unroll
  for (int i = 0; i < R; ++i) {
    y1[lane + 32 * i] = yr[i];
    if (y2) y2[lane + 32 * i] = zr[i];
  }
}

// Cluster of NC CTAs; CTA c holds blocks top[c], bot[c] of b columns each.
// Round-robin over the 2 NC blocks: block slot top[0] stays, the others move
// one place around the circle each round.
//
// Preconditioning: the Jacobi does not start from W itself but from X = W Q,
// V = Q, where W^T = Q R is a Householder QR; then X = R^T, lower triangular.
// One-sided Jacobi then gives X J = U Sigma, i.e. W = U Sigma (Q J)^T: the same
// outputs as before (U from the normalised columns, V accumulated), in fewer
// sweeps, since the Gram matrix of R^T, R R^T, is much nearer to diagonal
// than W^T W = R^T R (about 10 sweeps instead of 15 to 19 on the sketching
// workloads). The QR runs over the cluster with one panel per CTA, its two
// blocks: the columns of W^T are factored in CTA order, i.e. W^T P = Q R,
// X = P^T W Q, and U comes out with its rows permuted back. CTA p factors its
// panel (a warp per column, in registers) and publishes the reflectors in
// global memory; after one cluster barrier every CTA reads them from L2 and
// applies them to its later columns of W^T and to all its columns of
// Y = Q^T (started at I). R^T and Q = Y^T are then scattered into the other
// buffer through distributed shared memory. A W with zero rows (sparse
// inputs) starts from W itself: its QR turns exact zeros into rounding noise,
// and there the preconditioned Jacobi needed more sweeps, not fewer.
template <int R>
__global__ void __launch_bounds__(kClusterThreads, 1) svd32_cluster_kernel(const double* __restrict__ W, int k, int b,
                                                                        double* __restrict__ U0,
                                                                        double* __restrict__ V0, float* __restrict__ qr,
                                                                        int* sweeps_out) {
  constexpr int kp = 32 * R;  // padded column length
  cg::cluster_group cluster = cg::this_cluster();
  const int NC = (int)cluster.num_blocks();
  const int c = (int)cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  extern __shared__ __align__(16) float cs[];
  const size_t blk = (size_t)b * kp;  // floats per block of W (and of V)
  // buffers[2]: each holds [W top | W bot | V top | V bot]
  float* buf0 = cs;
  float* buf1 = cs + 4 * blk;
  __shared__ int rot_flag[2];
  __shared__ float2 rot_cs[kMaxBlkRot][kMaxBlkRot];  // (c, s) of step s, pair j
  __shared__ float bnorm[kMaxBlkRot];                 // squared norms of the bottom block's columns
  __shared__ float own_beta[2 * kMaxBlkRot];          // my panel's reflectors' beta
  __shared__ float st_beta[2 * kMaxBlkRot];           // beta of the panel being applied
  __shared__ int zero_row;                            // one of my columns of W^T is zero
  float* own = cs + 8 * blk;                          // my panel's reflectors (2 b columns)
  float* stage = cs + 10 * blk;                       // another CTA's panel, being applied
  const int pw = 2 * b;                               // panel width
  // real columns of block B, and the first diagonal row of my panel
  auto nreal = [&](int B) { return max(0, min(b, k - B * b)); };
  int my_row0 = 0;
  for (int P = 0; P < c; ++P) my_row0 += nreal(P) + nreal(2 * NC - 1 - P);
  // CTA c starts with blocks c (top) and 2 NC - 1 - c (bottom). Block 0 stays;
  // the other 2 NC - 1 move one place around the circle per round, so after
  // the 2 NC - 1 rounds of a sweep every block is back where it started and
  // every pair of blocks has met once.
  const int id_top = c, id_bot = 2 * NC - 1 - c;
  if (tid < 2) rot_flag[tid] = 0;
  if (tid == 0) zero_row = 0;
  __syncthreads();
  // buf0 <- my two blocks of W^T and of Y = I; buf1 <- 0 (R^T and Q land there)
  for (int slot = 0; slot < 2; ++slot) {
    const int B = slot == 0 ? id_top : id_bot;
    float* w = buf0 + slot * blk;
    float* v = buf0 + (2 + slot) * blk;
    for (int e = tid; e < (int)blk; e += blockDim.x) {
      const int j = e / kp, i = e - j * kp;
      const int gc = B * b + j;
      w[e] = (gc < k && i < k) ? (float)W[(size_t)gc * k + i] : 0.f;
      v[e] = (gc < k && i == gc) ? 1.f : 0.f;
    }
  }
  for (int e = tid; e < (int)(4 * blk); e += blockDim.x) buf1[e] = 0.f;
  __syncthreads();
  // W with zero rows (sparse inputs): W^T is then rank-deficient with exact
  // zeros that the QR would turn into rounding noise, and the Jacobi on R^T
  // needs more sweeps than on W itself, so those start from W, V = I.
  for (int t = warp; t < 2 * b; t += nwarps) {
    const int slot = t / b, j = t - slot * b;
    const int gc = (slot == 0 ? id_top : id_bot) * b + j;
    if (gc >= k) continue;
    const float* col = buf0 + slot * blk + (size_t)j * kp;
    bool nz = false;
    for (int i = lane; i < k; i += 32) nz |= col[i] != 0.f;
    if (!__any_sync(0xffffffffu, nz) && lane == 0) zero_row = 1;
  }
  cluster.sync();
  int any_zero_row = 0;
  for (int r = 0; r < NC; ++r) any_zero_row |= *cluster.map_shared_rank(&zero_row, r);
  const bool precondition = any_zero_row == 0;
  if (!precondition) {
    for (int slot = 0; slot < 2; ++slot) {
      const int B = slot == 0 ? id_top : id_bot;
      float* w = buf0 + slot * blk;
      for (int e = tid; e < (int)blk; e += blockDim.x) {
        const int j = e / kp, i = e - j * kp;
        const int gc = B * b + j;
        w[e] = (gc < k && i < k) ? (float)W[(size_t)i * k + gc] : 0.f;
      }
    }
  }
  // Householder QR of W^T P, panel p = CTA p's two blocks (positions
  // p pw ... p pw + pw - 1). The owner factors its panel and publishes the
  // reflectors through global memory (read back from L2 by every CTA: one
  // SM's shared memory serving 15 readers was the bottleneck).
  for (int p = 0; p < (precondition ? NC : 0); ++p) {
    float* gv = qr + (size_t)p * pw * kp;
    float* gb = qr + (size_t)NC * pw * kp + (size_t)p * pw;
    if (c == p) {
      factor_panel<R>(buf0, b, blk, my_row0, nreal(c), own, own_beta, warp, lane);
      const float4* src = (const float4*)own;
      float4* dst = (float4*)gv;
      for (int e = tid; e < (int)(2 * blk / 4); e += blockDim.x) dst[e] = src[e];
      if (tid < pw) gb[tid] = own_beta[tid];
    }
    cluster.sync();
    const float* Vp = own;
    const float* bp = own_beta;
    if (c != p) {
      const float4* src = (const float4*)gv;
      float4* dst = (float4*)stage;
      const int n4 = (int)(2 * blk / 4);
      for (int e = tid; e < n4; e += 2 * blockDim.x) {
        const float4 x0 = __ldcg(src + e);
        const bool two = e + (int)blockDim.x < n4;
        const float4 x1 = two ? __ldcg(src + e + blockDim.x) : x0;
        dst[e] = x0;
        if (two) dst[e + blockDim.x] = x1;
      }
      if (tid < pw) st_beta[tid] = __ldcg(gb + tid);
      __syncthreads();
      Vp = stage;
      bp = st_beta;
    }
    // my columns of W^T if my panel comes later, and all my columns of Y:
    // list entry t < pw is W^T column t, t >= pw is Y column t - pw
    const int first = c > p ? 0 : pw;
    const int ncols = 2 * pw - first;
    for (int t = warp; t < ncols; t += 2 * nwarps) {
      const int t1 = first + t, t2 = t + nwarps < ncols ? t1 + nwarps : -1;
      float* y1 = buf0 + (size_t)(t1 / b) * blk + (size_t)(t1 % b) * kp;
      float* y2 = t2 >= 0 ? buf0 + (size_t)(t2 / b) * blk + (size_t)(t2 % b) * kp : nullptr;
      apply_panel<R>(Vp, bp, pw, y1, y2, lane);
    }
    __syncthreads();
  }
  cluster.sync();
  // scatter X = R^T (X[pos, i] = R[i, pos], i <= pos, pos = my panel
  // positions) and Q = Y^T (Q[gc, i] = Y[i, gc]) into buf1 of the owners of
  // column i
  for (int t = warp; t < (precondition ? pw : 0); t += nwarps) {
    const int slot = t / b, j = t - slot * b;
    const int gc = (slot == 0 ? id_top : id_bot) * b + j;
    if (gc >= k) continue;
    const int pos = c * pw + t;
    const int prow = t < b ? my_row0 + t : my_row0 + nreal(c) + (t - b);  // its diagonal row
    const float* wcol = buf0 + slot * blk + (size_t)j * kp;
    const float* ycol = buf0 + (2 + slot) * blk + (size_t)j * kp;
    for (int i = lane; i < k; i += 32) {
      const int Bi = i / b, ji = i - Bi * b;
      const int dr = Bi < NC ? Bi : 2 * NC - 1 - Bi;
      const int ds = Bi < NC ? 0 : 1;
      float* dst = cluster.map_shared_rank(buf1, dr);
      if (i <= prow) dst[(size_t)ds * blk + (size_t)ji * kp + pos] = wcol[i];
      dst[(size_t)(2 + ds) * blk + (size_t)ji * kp + gc] = ycol[i];
    }
  }
  cluster.sync();
  float* cur = precondition ? buf1 : buf0;
  float* nxt = precondition ? buf0 : buf1;
  int sweep = 0;
  bool conv = false;
  while (!conv && sweep < kMaxSweepsA) {
    int my_rot = 0;
    for (int round = 0; round < 2 * NC - 1; ++round) {
      float* Wt = cur;
      float* Wb = cur + blk;
      float* Vt = cur + 2 * blk;
      float* Vb = cur + 3 * blk;
      if (round == 0) {
        // pairs inside each block (each block sits in exactly one CTA in round 0)
        const int bb = b + (b & 1);
        for (int r = 0; r < bb - 1; ++r) {
          for (int t = warp; t < bb; t += nwarps) {  // bb/2 pairs per slot, two slots
            const int slot = t / (bb / 2), pr = t % (bb / 2);
            int p, q;
            rr_pair(r, pr, bb, p, q);
            if (q >= b) continue;
            float* w = slot == 0 ? Wt : Wb;
            float* v = slot == 0 ? Vt : Vb;
            my_rot |= rotate_pair_reg<R>(w + (size_t)p * kp, w + (size_t)q * kp, v + (size_t)p * kp,
                                         v + (size_t)q * kp, lane);
          }
          __syncthreads();
        }
      }
      // every column of the top block against every column of the bottom block:
      // in step s warp j rotates W columns (top j, bottom (j + s) % b), keeping
      // top column j in registers for the whole round, and records (c, s); the
      // same warp applies that rotation to the V columns one step later, off
      // the critical path
      {
        float xr[R];
        float an = 0.f;
        if (warp < b) {
          float yr[R];
          load_col<R>(Wt + (size_t)warp * kp, lane, xr);
          load_col<R>(Wb + (size_t)warp * kp, lane, yr);
          an = col_sq<R>(xr);
          const float bq = col_sq<R>(yr);
          if (lane == 0) bnorm[warp] = bq;  // read in step 0 by this warp only
          __syncwarp();
        }
        // step 0: W only; steps 1 .. b - 1: W and the previous step's V;
        // step b: V only
        if (warp < b)
          my_rot |= rotate_step<R, true, false>(xr, an, Wb + (size_t)warp * kp, &bnorm[warp], &rot_cs[0][warp],
                                                nullptr, nullptr, nullptr, lane);
        __syncthreads();
        for (int s = 1; s < b; ++s) {
          if (warp < b) {
            const int q = warp + s - (warp + s >= b ? b : 0);  // (warp + s) mod b, both < b
            const int qv = q == 0 ? b - 1 : q - 1;             // (warp + s - 1) mod b
            my_rot |= rotate_step<R, true, true>(xr, an, Wb + (size_t)q * kp, &bnorm[q], &rot_cs[s][warp],
                                                 Vt + (size_t)warp * kp, Vb + (size_t)qv * kp, &rot_cs[s - 1][warp],
                                                 lane);
          }
          __syncthreads();
        }
        if (warp < b) {
          const int qv = warp == 0 ? b - 1 : warp - 1;  // (warp + b - 1) mod b
          rotate_step<R, false, true>(xr, an, nullptr, nullptr, nullptr, Vt + (size_t)warp * kp, Vb + (size_t)qv * kp,
                                      &rot_cs[b - 1][warp], lane);
        }
        __syncthreads();
        if (warp < b) store_col<R>(Wt + (size_t)warp * kp, lane, xr);
        __syncthreads();
      }
      // move blocks one step around the circle (into the destinations' next buffers)
      {
        const int dst_top = (c == 0) ? 0 : (c == NC - 1 ? NC - 1 : c + 1);
        const int dst_top_slot = (c == 0) ? 0 : (c == NC - 1 ? 1 : 0);
        const int dst_bot = (c == 0) ? 1 : c - 1;
        const int dst_bot_slot = (c == 0) ? 0 : 1;
        float* rt = cluster.map_shared_rank(nxt, dst_top);
        float* rb = cluster.map_shared_rank(nxt, dst_bot);
        const float4* srcWt = (const float4*)Wt;
        const float4* srcVt = (const float4*)Vt;
        const float4* srcWb = (const float4*)Wb;
        const float4* srcVb = (const float4*)Vb;
        float4* dWt = (float4*)(rt + dst_top_slot * blk);
        float4* dVt = (float4*)(rt + (2 + dst_top_slot) * blk);
        float4* dWb = (float4*)(rb + dst_bot_slot * blk);
        float4* dVb = (float4*)(rb + (2 + dst_bot_slot) * blk);
        const int n4 = (int)(blk / 4);
        for (int e = tid; e < n4; e += blockDim.x) {
          dWt[e] = srcWt[e];
          dVt[e] = srcVt[e];
          dWb[e] = srcWb[e];
          dVb[e] = srcVb[e];
        }
      }
      cluster.sync();
      // every CTA has read last sweep's flags before arriving here, so the
      // slot of the next sweep can be cleared now
      if (round == 0 && tid == 0) rot_flag[(sweep + 1) & 1] = 0;
      float* t = cur;
      cur = nxt;
      nxt = t;
    }
    // cluster-wide "any rotation in this sweep"
    if (my_rot) atomicOr(&rot_flag[sweep & 1], my_rot);
    cluster.sync();
    int any = 0;
    for (int r = 0; r < NC; ++r) any |= *cluster.map_shared_rank(&rot_flag[sweep & 1], r);
    conv = (any & 2) == 0;  // no rotation, or only small ones (kStopA)
    ++sweep;
  }
  // write out my two blocks (back at their starting places after whole sweeps)
  for (int slot = 0; slot < 2; ++slot) {
    for (int j = warp; j < b; j += nwarps) {
      const int gc = (slot == 0 ? id_top : id_bot) * b + j;
      if (gc >= k) continue;
      if (precondition)
        emit_column_perm(cur + slot * blk + (size_t)j * kp, cur + (2 + slot) * blk + (size_t)j * kp, k, kp, b, NC, gc,
                         lane, U0, V0);
      else
        emit_column(cur + slot * blk + (size_t)j * kp, cur + (2 + slot) * blk + (size_t)j * kp, k, gc, lane, U0, V0);
    }
  }
  if (c == 0 && tid == 0 && sweeps_out) *sweeps_out = sweep;
  cluster.sync();
}

// ------------------------------------------------------------- Phase B

constexpr int kGT = 16, kGK = 16;

__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }

__global__ void svd_flags_init_kernel(unsigned long long* maxoff, int iters, int* done_iter, GridBarrier* bar,
                                      long long limit) {
  if (threadIdx.x < 2 * iters) maxoff[threadIdx.x] = 0ull;
  if (threadIdx.x == 0) {
    *done_iter = kNotDone;
    bar->count = 0u;
    bar->gen = 0u;
    bar->err = 0;
    bar->limit = limit;
  }
}

// One 16 x 16 tile of C = op(A) B (+ Cadd); k x k column-major; 256 threads.
__device__ __forceinline__ void gemm_tile(int k, int ti, int tj, const double* __restrict__ A, int transA,
                                          const double* __restrict__ B, const double* __restrict__ Cadd,
                                          double* __restrict__ Cout, double (*As)[kGT + 1], double (*Bs)[kGT + 1]) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = ti * kGT, j0 = tj * kGT;
  double acc = 0.0;
  for (int p0 = 0; p0 < k; p0 += kGK) {
    const int gi = i0 + tx, gp = p0 + ty;
    double v = 0.0;
    if (gi < k && gp < k) v = transA ? A[(size_t)gi * k + gp] : A[(size_t)gp * k + gi];
    As[ty][tx] = v;
    const int gj = j0 + tx;
    Bs[ty][tx] = (gp < k && gj < k) ? B[(size_t)gj * k + gp] : 0.0;
    __syncthreads();
#pragma unroll
    for (int p = 0; p < kGK; ++p) acc = fma(As[p][ty], Bs[p][tx], acc);
    __syncthreads();
  }
  const int gi = i0 + ty, gj = j0 + tx;
  if (gi < k && gj < k) {
    const size_t o = (size_t)gj * k + gi;
    Cout[o] = Cadd ? Cadd[o] + acc : acc;
  }
}

// One 16 x 16 tile of the symmetric C = A^T A (A column-major k x k), tile
// (ti, tj) with ti <= tj, written to both triangles; same FP64 arithmetic as
// gemm_tile.
__device__ __forceinline__ void gram_tile(int k, int ti, int tj, const double* __restrict__ A,
                                          double* __restrict__ Cout, double (*As)[kGT + 1], double (*Bs)[kGT + 1]) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = ti * kGT, j0 = tj * kGT;
  double acc = 0.0;
  for (int p0 = 0; p0 < k; p0 += kGK) {
    const int gi = i0 + tx, gp = p0 + ty, gj = j0 + tx;
    As[ty][tx] = (gi < k && gp < k) ? A[(size_t)gi * k + gp] : 0.0;
    Bs[ty][tx] = (gp < k && gj < k) ? A[(size_t)gj * k + gp] : 0.0;
    __syncthreads();
#pragma unroll
    for (int p = 0; p < kGK; ++p) acc = fma(As[p][ty], Bs[p][tx], acc);
    __syncthreads();
  }
  const int gi = i0 + ty, gj = j0 + tx;
  if (gi < k && gj < k) {
    Cout[(size_t)gj * k + gi] = acc;
    if (ti != tj) Cout[(size_t)gi * k + gj] = acc;
  }
}

// One 16 x 16 tile of Cout = Cadd + A B (A, B, Cadd column-major k x k, FP64
// storage) with the product in FP32. Used for the corrections U F and V G:
// F and G are already small, so the FP32 product's rounding (about 2^-24 of
// |U| |F|) is far below the error the iteration removes and is corrected by
// the next one.
__device__ __forceinline__ void corr_tile_f32(int k, int ti, int tj, const double* __restrict__ A,
                                              const double* __restrict__ B, const double* __restrict__ Cadd,
                                              double* __restrict__ Cout, float (*As)[kGT + 1], float (*Bs)[kGT + 1]) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = ti * kGT, j0 = tj * kGT;
  float acc = 0.f;
  for (int p0 = 0; p0 < k; p0 += kGK) {
    const int gi = i0 + tx, gp = p0 + ty, gj = j0 + tx;
    As[ty][tx] = (gi < k && gp < k) ? (float)A[(size_t)gp * k + gi] : 0.f;
    Bs[ty][tx] = (gp < k && gj < k) ? (float)B[(size_t)gj * k + gp] : 0.f;
    __syncthreads();
#pragma unroll
    for (int p = 0; p < kGK; ++p) acc = fmaf(As[p][ty], Bs[p][tx], acc);
    __syncthreads();
  }
  const int gi = i0 + ty, gj = j0 + tx;
  if (gi < k && gj < k) {
    const size_t o = (size_t)gj * k + gi;
    Cout[o] = Cadd[o] + (double)acc;
  }
}

__device__ __forceinline__ void tri_of(int x, int nt, int& ti, int& tj) {
  // x-th tile (ti <= tj) of the upper triangle, row by row
  ti = 0;
  while (x >= nt - ti) {
    x -= nt - ti;
    ++ti;
  }
  tj = ti + x;
}

struct RefineArgs {
  int k;
  const double* W;  // row-major k x k (= W^T column-major)
  double *U0, *U1, *V0, *V1, *P, *T, *UtU, *VtV, *F, *G, *d;
  unsigned long long* maxoff;
  int* done_iter;
  GridBarrier* bar;
  int* status;
  double keep_rtol;     // values at or below keep_rtol max |d| are truncated afterwards
  double resolve_rtol;  // off-diagonal |T_ij| up to resolve_rtol max |d| may stay (reduced-precision data)
};

// Phase B in one launch: every iteration's GEMMs are spread over the CTAs as
// 16 x 16 tiles, with a grid barrier between dependent phases; all CTAs read
// the same convergence measure after a barrier, so they stop together.
__global__ void __launch_bounds__(256) refine_persistent_kernel(RefineArgs a) {
  __shared__ double As[kGK][kGT + 1];
  __shared__ double Bs[kGK][kGT + 1];
  __shared__ float As32[kGK][kGT + 1];
  __shared__ float Bs32[kGK][kGT + 1];
  __shared__ double dsh[CABS_MAX_K];
  __shared__ double dmax2;
  const int k = a.k;
  const unsigned nb = gridDim.x;
  const int nt = (k + kGT - 1) / kGT;
  const int tiles = nt * nt;
  const int tri = nt * (nt + 1) / 2;
  double prev = 0.0;
  for (int t = 0; t < kItersB; ++t) {
    const double* U = (t & 1) ? a.U1 : a.U0;
    const double* V = (t & 1) ? a.V1 : a.V0;
    double* Un = (t & 1) ? a.U0 : a.U1;
    double* Vn = (t & 1) ? a.V0 : a.V1;
    if (t == 0) {
      // First iteration: P = W V and V^T V; then every column of P above the
      // FP32 phase's noise level (2^-18 of the largest) replaces the FP32
      // column of U (U_j = P_j / |P_j|), so that the kept columns span the
      // range of W to FP64 accuracy. U + U F only mixes existing columns, so
      // it could not leave an FP32-accurate span where W has exactly zero
      // columns (nothing else supplies the missing directions). Columns at
      // the noise level keep their FP32 directions. Then U^T U and T = U^T P.
      for (int x = blockIdx.x; x < tiles + tri; x += nb) {
        if (x < tiles) {
          gemm_tile(k, x % nt, x / nt, a.W, 1, V, nullptr, a.P, As, Bs);
        } else {
          int ti, tj;
          tri_of(x - tiles, nt, ti, tj);
          gram_tile(k, ti, tj, V, a.VtV, As, Bs);
        }
      }
      if (!grid_sync(a.bar, nb)) return;
      for (int j = blockIdx.x; j < k; j += nb) {
        double s2 = 0.0;
        for (int i = threadIdx.x; i < k; i += blockDim.x) {
          const double v = a.P[(size_t)j * k + i];
          s2 = fma(v, v, s2);
        }
        s2 = warp_sum(s2);
        if ((threadIdx.x & 31) == 0) dsh[threadIdx.x >> 5] = s2;
        __syncthreads();
        if (threadIdx.x == 0) {
          double tot = 0.0;
          for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += dsh[w];
          a.d[j] = sqrt(tot);
        }
        __syncthreads();
      }
      if (!grid_sync(a.bar, nb)) return;
      {
        double mx = 0.0;
        for (int j = 0; j < k; ++j) mx = fmax(mx, a.d[j]);
        double* Uw = const_cast<double*>(U);
        for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)k * k;
             e += (long long)nb * blockDim.x) {
          const int j = (int)(e / k);
          const double nj = a.d[j];
          if (nj > 3.814697265625e-06 * mx) Uw[e] = a.P[e] / nj;
        }
        // Columns at the noise level whose W has all-zero rows: each takes a
        // unit vector e_i of such a row, an exact left null vector of W. A
        // zero row of W is zero in every column the FP32 phase produces, so
        // without these the columns of U could not span R^k.
        if (blockIdx.x == 0) {
          __shared__ int zrow[CABS_MAX_K], ncol[CABS_MAX_K], counts[2];
          {
            // one warp per row of W: all-zero test by ballot
            const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
            for (int i = threadIdx.x >> 5; i < k; i += nw) {
              bool nzr = false;
              for (int j = lane; j < k; j += 32) nzr |= a.W[(size_t)i * k + j] != 0.0;
              const bool anyr = __any_sync(0xffffffffu, nzr);
              if (lane == 0) {
                zrow[i] = anyr ? 0 : 1;
                ncol[i] = a.d[i] > 3.814697265625e-06 * mx ? 0 : 1;
              }
            }
          }
          __syncthreads();
          if (threadIdx.x == 0) {
            int nz = 0, nn = 0;
            for (int i = 0; i < k; ++i) {
              if (zrow[i]) zrow[nz++] = i;
              if (ncol[i]) ncol[nn++] = i;
            }
            counts[0] = nz;
            counts[1] = nn;
          }
          __syncthreads();
          const int pairs = min(counts[0], counts[1]);
          for (long long e = threadIdx.x; e < (long long)pairs * k; e += blockDim.x) {
            const int t2 = (int)(e / k), i = (int)(e - (long long)t2 * k);
            Uw[(size_t)ncol[t2] * k + i] = i == zrow[t2] ? 1.0 : 0.0;
          }
          __syncthreads();
          // Null columns left over (the rank falls short of k by more than the
          // zero rows, e.g. through repeated nonzero rows) lie in the span of
          // the others or are zero, and the refinement cannot make them
          // orthonormal. When W has zero rows (the sparse regime) they are all
          // replaced by Gram-Schmidt: each takes
          // e_i for the row i least covered by the columns so far (smallest
          // rho_i = sum_b U_ib^2, so |e_i - proj|^2 = 1 - rho_i >= 1 - r / k
          // > 0), minus its projection. Elsewhere the noise columns keep their
          // FP32 directions, which span the complement.
          __shared__ double rho[CABS_MAX_K], qv[CABS_MAX_K], red[CABS_MAX_K];
          __shared__ int slot_s[CABS_MAX_K], nslot, istar;
          if (threadIdx.x == 0) {
            // only zero rows keep U from spanning R^k; exactly zero columns of
            // W alone (a zero-padded block) leave the kept columns spanning
            // the range of W exactly, and the refinement handles the rest
            const bool sparse = counts[0] > 0;
            int ns = 0;
            if (sparse)
              for (int t2 = pairs; t2 < counts[1]; ++t2) slot_s[ns++] = ncol[t2];
            nslot = ns;
          }
          __syncthreads();
          for (long long e = threadIdx.x; e < (long long)nslot * k; e += blockDim.x) {
            const int t2 = (int)(e / k), i = (int)(e - (long long)t2 * k);
            Uw[(size_t)slot_s[t2] * k + i] = 0.0;
          }
          __syncthreads();
          if (nslot > 0) {
            for (int i = threadIdx.x; i < k; i += blockDim.x) {
              double r2 = 0.0;
              for (int b2 = 0; b2 < k; ++b2) {
                const double u = Uw[(size_t)b2 * k + i];  // zero columns add nothing
                r2 = fma(u, u, r2);
              }
              rho[i] = r2;
            }
            __syncthreads();
            for (int t2 = 0; t2 < nslot; ++t2) {
              if (threadIdx.x == 0) {
                int best = 0;
                for (int i = 1; i < k; ++i)
                  if (rho[i] < rho[best]) best = i;
                istar = best;
              }
              __syncthreads();
              const int is = istar;
              for (int i = threadIdx.x; i < k; i += blockDim.x) {
                double q = i == is ? 1.0 : 0.0;
                for (int b2 = 0; b2 < k; ++b2) q = fma(-Uw[(size_t)b2 * k + is], Uw[(size_t)b2 * k + i], q);
                qv[i] = q;
                red[i] = q * q;
              }
              for (int i = k + threadIdx.x; i < CABS_MAX_K; i += blockDim.x) red[i] = 0.0;
              __syncthreads();
              for (int w2 = CABS_MAX_K / 2; w2 > 0; w2 >>= 1) {
                for (int i = threadIdx.x; i < w2; i += blockDim.x) red[i] += red[i + w2];
                __syncthreads();
              }
              const double inv = red[0] > 0.0 ? 1.0 / sqrt(red[0]) : 0.0;
              const int j = slot_s[t2];
              for (int i = threadIdx.x; i < k; i += blockDim.x) {
                const double q = qv[i] * inv;
                Uw[(size_t)j * k + i] = q;
                rho[i] += q * q;
              }
              __syncthreads();
            }
          }
        }
      }
      if (!grid_sync(a.bar, nb)) return;
      for (int x = blockIdx.x; x < tiles + tri; x += nb) {
        if (x < tiles) {
          gemm_tile(k, x % nt, x / nt, U, 1, a.P, nullptr, a.T, As, Bs);
        } else {
          int ti, tj;
          tri_of(x - tiles, nt, ti, tj);
          gram_tile(k, ti, tj, U, a.UtU, As, Bs);
        }
      }
      if (!grid_sync(a.bar, nb)) return;
    } else {
      // P = W V, and (independent of it) the Gram matrices U^T U, V^T V by
      // their upper triangles; then T = U^T P
      for (int x = blockIdx.x; x < tiles + 2 * tri; x += nb) {
        if (x < tiles) {
          gemm_tile(k, x % nt, x / nt, a.W, 1, V, nullptr, a.P, As, Bs);
        } else {
          const int y = x - tiles, which = y / tri;
          int ti, tj;
          tri_of(y - which * tri, nt, ti, tj);
          gram_tile(k, ti, tj, which == 0 ? U : V, which == 0 ? a.UtU : a.VtV, As, Bs);
        }
      }
      if (!grid_sync(a.bar, nb)) return;
      for (int x = blockIdx.x; x < tiles; x += nb) gemm_tile(k, x % nt, x / nt, U, 1, a.P, nullptr, a.T, As, Bs);
      if (!grid_sync(a.bar, nb)) return;
    }
    // coefficients F, G and singular value estimates d
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
      const size_t ii = (size_t)i * k + i;
      dsh[i] = a.T[ii] / (1.0 - 0.5 * ((1.0 - a.UtU[ii]) + (1.0 - a.VtV[ii])));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double m = 0.0;
      for (int i = 0; i < k; ++i) m = fmax(m, fabs(dsh[i]));
      dmax2 = m * m;
    }
    __syncthreads();
    if (blockIdx.x == 0)
      for (int i = threadIdx.x; i < k; i += blockDim.x) a.d[i] = dsh[i];
    double local = 0.0, lclose = 0.0;
    const double keep2 = a.keep_rtol * a.keep_rtol * dmax2;
    // a pair left undiagonalised counts unless both values are truncated
    auto counts = [&](double di, double dj) { return fmax(di * di, dj * dj) > keep2; };
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)k * k;
         e += (long long)nb * blockDim.x) {
      const int j = (int)(e / k), i = (int)(e - (long long)j * k);
      const size_t ij = (size_t)j * k + i, ji = (size_t)i * k + j;
      const double Rij = (i == j ? 1.0 : 0.0) - a.UtU[ij];
      const double Sij = (i == j ? 1.0 : 0.0) - a.VtV[ij];
      double f, g;
      if (i == j) {
        f = 0.5 * Rij;
        g = 0.5 * Sij;
      } else {
        const double di = dsh[i], dj = dsh[j];
        const double den = dj * dj - di * di;
        if (fabs(den) <= 1e-13 * dmax2) {
          f = 0.5 * Rij;
          g = 0.5 * Sij;
          double res = fabs(a.T[ij]);
          const double db = 0.5 * (di + dj);
          if (db * db > 1e-13 * dmax2) {
            // A repeated value: any rotation of the pair's U and V columns
            // together is as good, but U and V may still differ by one, which
            // leaves the block d [[1, -t], [t, 1]]. Splitting the rotation
            // t / 2 onto U and -t / 2 onto V (the first-order conditions with
            // d_i = d_j) removes it; what stays is the symmetric part.
            const double rot = (a.T[ij] - a.T[ji]) / (4.0 * db);
            if (fabs(rot) <= kMaxCorrB) {
              f += rot;
              g -= rot;
              res = 0.5 * fabs(a.T[ij] + a.T[ji]);
            }
          }
          if (counts(di, dj)) lclose = fmax(lclose, res);
        } else {
          const double al = a.T[ij] + dj * Rij;
          const double be = a.T[ji] + dj * Sij;
          f = (al * dj + be * di) / den;
          g = (al * di + be * dj) / den;
          // A first-order correction this large means the two values are not
          // yet separated by more than the error of the estimates (exactly
          // repeated values differ only by rounding): orthogonalise the pair
          // this time, as for equal values.
          if (!(fabs(f) <= kMaxCorrB && fabs(g) <= kMaxCorrB)) {
            f = 0.5 * Rij;
            g = 0.5 * Sij;
          }
        }
        local = fmax(local, fmax(fabs(f), fabs(g)));
      }
      a.F[ij] = f;
      a.G[ij] = g;
    }
    local = warp_max(local);
    lclose = warp_max(lclose);
    if ((threadIdx.x & 31) == 0 && local > 0.0) atomicMax(a.maxoff + t, dbits(local));
    if ((threadIdx.x & 31) == 0 && lclose > 0.0) atomicMax(a.maxoff + kItersB + t, dbits(lclose));
    if (!grid_sync(a.bar, nb)) return;
    for (int x = blockIdx.x; x < 2 * tiles; x += nb) {
      const int which = x / tiles, y = x - which * tiles;
      if (which == 0) corr_tile_f32(k, y % nt, y / nt, U, a.F, U, Un, As32, Bs32);
      else corr_tile_f32(k, y % nt, y / nt, V, a.G, V, Vn, As32, Bs32);
    }
    // Quadratic convergence: the update just applied used corrections of size
    // m, so it leaves an error of order m^2 (times the inverse relative gap of
    // the pairs that still rotate); at m < kConvB that is below the FP64
    // rounding floor and no verifying iteration is needed. Or a plateau at the
    // rounding floor (clustered values whose corrections stop shrinking).
    // Pairs closer than the estimates' resolution keep only the
    // orthogonality correction (and, for a repeated value, the split
    // rotation), so the update does not diagonalise them: their remaining
    // |T_ij| must already be at the rounding level, otherwise (a block of
    // tiny values that the FP32 phase could not resolve) the iteration has
    // not converged and the FP64 Jacobi takes over. Pairs whose values are
    // both truncated afterwards do not count, and for data carried in FP32
    // or less the bound is the data's own resolution (resolve_rtol) rather
    // than 1e-13. Pairs deferred for a correction above kMaxCorrB are not
    // counted either: in FP32 data they can stay deferred with |T_ij| near
    // 1e-7, as before this check existed.
    // For data carried in FP32 or less (resolve_rtol > 0) the factors need
    // only reach the data's own resolution: corrections below
    // 1e-2 sqrt(resolve_rtol) (about 1e-5 at 2^-20) leave an error of order
    // 1e-10, four orders below it, so the update that brought them is the
    // last; FP64 data keeps kConvB.
    const double conv_m = a.resolve_rtol > 0.0 ? fmax(kConvB, 1e-2 * sqrt(a.resolve_rtol)) : kConvB;
    const double m = __longlong_as_double((long long)*(volatile unsigned long long*)(a.maxoff + t));
    const double mc = __longlong_as_double((long long)*(volatile unsigned long long*)(a.maxoff + kItersB + t));
    const bool conv = (m < conv_m || (t >= 1 && m < 1e-7 && m > 0.25 * prev)) &&
                      mc <= fmax(kCloseOffB, a.resolve_rtol) * sqrt(dmax2);
    prev = m;
    if (!grid_sync(a.bar, nb)) return;
    if (conv) {
      if (blockIdx.x == 0 && threadIdx.x == 0) *a.done_iter = t;
      return;
    }
  }
}

// Sort and truncate: the position of every singular value in descending
// order (ties to the lower index), the kept rank and sig (desc). One CTA.
// Runs unless the FP64 Jacobi fallback is needed.
__global__ void __launch_bounds__(256) refine_sort_kernel(int k, double trunc_rtol, const double* __restrict__ d,
                                                          const int* __restrict__ done_iter, double* __restrict__ sig_out,
                                                          int* __restrict__ pos_out, int* __restrict__ rank_tmp,
                                                          int* rank_out, int* refine_out, int* status,
                                                          const GridBarrier* __restrict__ bar) {
  const int done = *done_iter;
  if (threadIdx.x == 0 && status && bar->err) atomicOr(status, 4);
  if (threadIdx.x == 0 && refine_out) *refine_out = done == kNotDone ? -1 : done + 1;
  if (done == kNotDone) {
    if (threadIdx.x == 0 && status) atomicOr(status, 2);
    return;  // the FP64 Jacobi fallback writes the outputs
  }
  __shared__ double sg[CABS_MAX_K];
  __shared__ double wmax[8];
  for (int i = threadIdx.x; i < k; i += blockDim.x) sg[i] = fabs(d[i]);
  __syncthreads();
  // position of value j: the number of values before it in descending order
  // (four independent counters, so the loads overlap)
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    const double v = sg[j];
    int r0 = 0, r1 = 0, r2 = 0, r3 = 0, i = 0;
    for (; i + 4 <= k; i += 4) {
      r0 += (sg[i] > v) || (sg[i] == v && i < j);
      r1 += (sg[i + 1] > v) || (sg[i + 1] == v && i + 1 < j);
      r2 += (sg[i + 2] > v) || (sg[i + 2] == v && i + 2 < j);
      r3 += (sg[i + 3] > v) || (sg[i + 3] == v && i + 3 < j);
    }
    for (; i < k; ++i) r0 += (sg[i] > v) || (sg[i] == v && i < j);
    const int r = r0 + r1 + r2 + r3;
    pos_out[j] = r;
    sig_out[r] = v;
  }
  // the largest value (block maximum), then the kept count
  double m = 0.0;
  for (int j = threadIdx.x; j < k; j += blockDim.x) m = fmax(m, sg[j]);
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
  __syncthreads();
  double smax = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) smax = fmax(smax, wmax[w]);
  const double tol = fmax(trunc_rtol, (double)k * 2.220446049250313e-16) * smax;
  int keep = 0;
  for (int j = threadIdx.x; j < k; j += blockDim.x) keep += (smax > 0.0 && sg[j] > tol) ? 1 : 0;
  const int r = __syncthreads_count(keep);
  if (threadIdx.x == 0) {
    *rank_tmp = r;
    if (rank_out) *rank_out = r;
  }
}

// Sign-fix and write Uw, Vw (row-major, column r = r-th singular vector,
// zero beyond the kept rank) from the last iterates; spread over the grid.
__global__ void __launch_bounds__(256) refine_write_kernel(int k, const double* __restrict__ Ubuf0,
                                                           const double* __restrict__ Ubuf1,
                                                           const double* __restrict__ Vbuf0,
                                                           const double* __restrict__ Vbuf1, const double* __restrict__ d,
                                                           const int* __restrict__ done_iter,
                                                           const int* __restrict__ pos, const int* __restrict__ rank_tmp,
                                                           double* __restrict__ Uw_out, double* __restrict__ Vw_out) {
  const int done = *done_iter;
  if (done == kNotDone) return;
  const int last = done;  // U, V after iteration `done` live in buffer (done + 1) % 2
  const double* U = ((last + 1) & 1) ? Ubuf1 : Ubuf0;
  const double* V = ((last + 1) & 1) ? Vbuf1 : Vbuf0;
  const int rank = *rank_tmp;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)k * k;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / k), i = (int)(e - (long long)j * k);  // column j, row i of U / V (column-major)
    const int r = pos[j];
    const bool keep = r < rank;
    const double sgn = d[j] < 0.0 ? -1.0 : 1.0;
    Uw_out[(size_t)i * k + r] = keep ? sgn * U[e] : 0.0;
    Vw_out[(size_t)i * k + r] = keep ? V[e] : 0.0;
  }
}

// ------------------------------------------------ FP64 Jacobi (fallback)

constexpr int kSvdThreads = 1024;
constexpr int kMaxSweeps = 40;
constexpr double kJacobiTol = 1e-15;
constexpr size_t kSvdSmemLimit = 200 * 1024;

__device__ __forceinline__ void pair_of_f64(int round, int pr, int kk, int& p, int& q) {
  if (pr == 0) {
    p = round;
    q = kk - 1;
  } else {
    p = (round + pr) % (kk - 1);
    q = (round - pr + kk - 1) % (kk - 1);
  }
  if (p > q) {
    const int t = p;
    p = q;
    q = t;
  }
}

// One CTA. W (k x k, row-major). Wc/Vc: column-major scratch (shared memory
// when use_smem, else the given global buffers). Outputs: sig (k, descending),
// Uw, Vw (k x k row-major, column r = r-th singular vector, zero beyond rank).
__global__ void __launch_bounds__(kSvdThreads) svd_jacobi_kernel(const double* __restrict__ W, int k,
                                                                  double trunc_rtol, int use_smem,
                                                                  double* Wc_g, double* Vc_g,
                                                                  double* __restrict__ sig_out,
                                                                  double* __restrict__ Uw_out,
                                                                  double* __restrict__ Vw_out, int* rank_out,
                                                                  int* sweeps_out, int* status,
                                                                  const int* __restrict__ done_iter) {
  if (done_iter && *done_iter != 0x7fffffff) return;
  extern __shared__ __align__(16) double svd_smem[];
  __shared__ double sig[CABS_MAX_K];
  __shared__ int pos[CABS_MAX_K];
  __shared__ int rotated;
  __shared__ int rank_s;
  double* Wc = use_smem ? svd_smem : Wc_g;
  double* Vc = use_smem ? svd_smem + (size_t)k * k : Vc_g;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int kk2 = k * k;
  for (int e = tid; e < kk2; e += blockDim.x) {
    const int i = e / k, j = e - i * k;
    Wc[(size_t)j * k + i] = W[e];
    Vc[e] = (i == j) ? 1.0 : 0.0;
  }
  if (tid == 0) rotated = 0;
  __syncthreads();

  const int kk = k + (k & 1);
  const int npairs = kk / 2;
  int sweep = 0;
  bool converged = (k < 2);
  while (!converged && sweep < kMaxSweeps) {
    for (int round = 0; round < kk - 1; ++round) {
      for (int pr = warp; pr < npairs; pr += nwarps) {
        int p, q;
        pair_of_f64(round, pr, kk, p, q);
        if (q >= k) continue;
        double* wp = Wc + (size_t)p * k;
        double* wq = Wc + (size_t)q * k;
        double a = 0.0, b = 0.0, g = 0.0;
        for (int i = lane; i < k; i += 32) {
          const double x = wp[i], y = wq[i];
          a = fma(x, x, a);
          b = fma(y, y, b);
          g = fma(x, y, g);
        }
        a = warp_sum(a);
        b = warp_sum(b);
        g = warp_sum(g);
        if (fabs(g) > kJacobiTol * sqrt(a) * sqrt(b)) {
          const double zeta = (b - a) / (2.0 * g);
          const double t = fabs(zeta) > 1e150 ? 0.5 / zeta
                                              : copysign(1.0, zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
          const double c = 1.0 / sqrt(fma(t, t, 1.0));
          const double s = c * t;
          double* vp = Vc + (size_t)p * k;
          double* vq = Vc + (size_t)q * k;
          for (int i = lane; i < k; i += 32) {
            const double x = wp[i], y = wq[i];
            wp[i] = c * x - s * y;
            wq[i] = s * x + c * y;
            const double u = vp[i], v = vq[i];
            vp[i] = c * u - s * v;
            vq[i] = s * u + c * v;
          }
          if (lane == 0) rotated = 1;
        }
      }
      __syncthreads();
    }
    ++sweep;
    const int any = rotated;
    __syncthreads();
    if (tid == 0) rotated = 0;
    __syncthreads();
    converged = (any == 0);
  }

  // singular values = column norms, then a rank sort (descending, stable)
  for (int j = warp; j < k; j += nwarps) {
    const double* wj = Wc + (size_t)j * k;
    double a = 0.0;
    for (int i = lane; i < k; i += 32) a = fma(wj[i], wj[i], a);
    a = warp_sum(a);
    if (lane == 0) sig[j] = sqrt(a);
  }
  __syncthreads();
  for (int j = tid; j < k; j += blockDim.x) {
    const double sj = sig[j];
    int r = 0;
    for (int i = 0; i < k; ++i) r += (sig[i] > sj) || (sig[i] == sj && i < j);
    pos[j] = r;
  }
  __syncthreads();
  if (tid == 0) {
    double smax = 0.0;
    for (int j = 0; j < k; ++j) smax = fmax(smax, sig[j]);
    int r = 0;
    if (smax > 0.0) {
      const double tol = fmax(trunc_rtol, (double)k * 2.220446049250313e-16) * smax;
      for (int j = 0; j < k; ++j) r += sig[j] > tol;
    }
    rank_s = r;
    if (rank_out) *rank_out = r;
    if (sweeps_out) *sweeps_out = sweep;
    if (status && !converged) atomicOr(status, 1);
  }
  __syncthreads();
  const int rank = rank_s;
  for (int j = tid; j < k; j += blockDim.x) sig_out[pos[j]] = sig[j];
  for (int e = tid; e < kk2; e += blockDim.x) {
    const int j = e / k, i = e - j * k;  // column j, row i (column-major walk)
    const int r = pos[j];
    const bool keep = r < rank;
    Vw_out[(size_t)i * k + r] = keep ? Vc[e] : 0.0;
    Uw_out[(size_t)i * k + r] = keep ? Wc[e] / sig[j] : 0.0;
  }
}

}  // namespace

cabs_status launch_svd_jacobi_f64(const double* W, int k, double trunc_rtol, const int* done_iter, double* Wc,
                                  double* Vc, double* sig, double* Uw, double* Vw, int* rank, int* sweeps, int* status,
                                  cudaStream_t stream) {
  const size_t smem_need = (size_t)2 * k * k * sizeof(double);
  const int use_smem = smem_need <= kSvdSmemLimit;
  const size_t smem = use_smem ? smem_need : 0;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(svd_jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  CABS_LAUNCH(stream, "svd_jacobi_kernel",
              svd_jacobi_kernel<<<1, kSvdThreads, smem, stream>>>(W, k, trunc_rtol, use_smem, Wc, Vc, sig, Uw, Vw, rank,
                                                                  sweeps, status, done_iter));
  return CABS_OK;
}

// Scratch of the preconditioning QR: the reflectors of every panel position
// (2 NC b <= k + 31 for any cluster size NC, since b = ceil(k / 2 NC)) of
// kp <= 256 rows (kp = 128 up to k = 128), and their betas.
static size_t svd_qr_floats(int k) { return (size_t)(k + 32) * (k <= 128 ? 128 : 256) + (k + 32); }

SvdWs carve_svd(Carve& cv, int k) {
  SvdWs w;
  const size_t kk = (size_t)k * k;
  for (int t = 0; t < 2; ++t) {
    w.U[t] = cv.take<double>(kk);
    w.V[t] = cv.take<double>(kk);
  }
  w.P = cv.take<double>(kk);
  w.T = cv.take<double>(kk);
  w.UtU = cv.take<double>(kk);
  w.VtV = cv.take<double>(kk);
  w.F = cv.take<double>(kk);
  w.G = cv.take<double>(kk);
  w.d = cv.take<double>(k);
  w.maxoff = cv.take<unsigned long long>(2 * kItersB);
  w.done_iter = cv.take<int>(1);
  w.pos = cv.take<int>(k);
  w.rank_tmp = cv.take<int>(1);
  w.bar = cv.take<GridBarrier>(1);
  w.Wc = cv.take<double>(kk);
  w.Vc = cv.take<double>(kk);
  w.qr = cv.take<float>(svd_qr_floats(k));
  return w;
}

#ifndef CABS_SVD_CLUSTER
#define CABS_SVD_CLUSTER 16
#endif

template <int R>
static cabs_status launch_cluster(const double* W, int k, double* U0, double* V0, float* qr, int* sweeps,
                                  cudaStream_t stream) {
  static int nc = -1;  // cluster size actually schedulable on this device
  const int want = CABS_SVD_CLUSTER;
  auto smem_for = [&](int c) {
    int b = (k + 2 * c - 1) / (2 * c);
    return (size_t)12 * b * 32 * R * sizeof(float);  // 2 x 4 blocks + 2 panels of reflectors
  };
  if (nc < 0) {
    nc = 8;
    if (want > 8) {
      cudaFuncSetAttribute(svd32_cluster_kernel<R>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      const size_t sm = smem_for(want);
      cudaFuncSetAttribute(svd32_cluster_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(want);
      cfg.blockDim = dim3(kClusterThreads);
      cfg.dynamicSmemBytes = sm;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = want;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int clusters = 0;
      if (cudaOccupancyMaxActiveClusters(&clusters, svd32_cluster_kernel<R>, &cfg) == cudaSuccess && clusters > 0)
        nc = want;
      cudaGetLastError();
    }
  }
  const int b = (k + 2 * nc - 1) / (2 * nc);
  if (b > kMaxBlkRot) {
    set_error("svd: %d columns per block exceed %d (k = %d on a %d-CTA cluster)", b, kMaxBlkRot, k, nc);
    return CABS_EINVAL;
  }
  if (32 * R < k || (size_t)2 * nc * b * (32 * R + 1) > svd_qr_floats(k)) {
    set_error("svd: k = %d does not fit the %d-row cluster layout or its QR scratch", k, 32 * R);
    return CABS_EINVAL;
  }
  const size_t smem = smem_for(nc);
  cudaFuncSetAttribute(svd32_cluster_kernel<R>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaFuncSetAttribute(svd32_cluster_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nc);
  cfg.blockDim = dim3(kClusterThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = nc;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  CABS_LAUNCH(stream, "svd32_cluster_kernel", cudaLaunchKernelEx(&cfg, svd32_cluster_kernel<R>, W, k, b, U0, V0, qr, sweeps));
  return CABS_OK;
}

cabs_status launch_svd(const double* W, int k, double trunc_rtol, double resolve_rtol, double* sig, double* Uw,
                       double* Vw, int* rank,
                       int* sweeps, int* refine, int* status, const SvdWs& w, cudaStream_t stream) {
  // ---- Phase A: FP32 Jacobi -> U[0], V[0]
  if (k <= kCtaMaxK) {
    const size_t smem = (size_t)2 * k * k * sizeof(float);
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(svd32_cta_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    CABS_LAUNCH(stream, "svd32_cta_kernel",
                svd32_cta_kernel<<<1, 512, smem, stream>>>(W, k, w.U[0], w.V[0], sweeps));
  } else if (k <= 128) {
    CABS_TRY(launch_cluster<4>(W, k, w.U[0], w.V[0], w.qr, sweeps, stream));
  } else {
    CABS_TRY(launch_cluster<8>(W, k, w.U[0], w.V[0], w.qr, sweeps, stream));
  }
  // ---- Phase B: FP64 refinement, one cooperative launch
  CABS_LAUNCH(stream, "svd_flags_init",
              svd_flags_init_kernel<<<1, 32, 0, stream>>>(w.maxoff, kItersB, w.done_iter, w.bar, wait_limit()));
  {
    const int nt = ceil_div(k, kGT);
    const int tiles = nt * nt + nt * (nt + 1);  // work units of the widest phase
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, refine_persistent_kernel, 256, 0);
    const int grid = std::max(1, std::min(tiles, coop_grid_cap(sm_count() * std::max(per_sm, 1))));
    RefineArgs ra{k, W, w.U[0], w.U[1], w.V[0], w.V[1], w.P, w.T, w.UtU, w.VtV, w.F, w.G, w.d, w.maxoff,
                  w.done_iter, w.bar, status,
                  std::max(std::max(trunc_rtol, (double)k * 2.220446049250313e-16), resolve_rtol), resolve_rtol};
    void* args[] = {&ra};
    CABS_LAUNCH(stream, "refine_persistent_kernel",
                cudaLaunchCooperativeKernel((const void*)refine_persistent_kernel, dim3(grid), dim3(256), args, 0,
                                            stream));
  }
  CABS_LAUNCH(stream, "refine_sort_kernel",
              refine_sort_kernel<<<1, 256, 0, stream>>>(k, trunc_rtol, w.d, w.done_iter, sig, w.pos, w.rank_tmp, rank,
                                                        refine, status, w.bar));
  CABS_LAUNCH(stream, "refine_write_kernel",
              refine_write_kernel<<<std::max(1, std::min(ceil_div(k * k, 256), 2 * sm_count())), 256, 0, stream>>>(
                  k, w.U[0], w.U[1], w.V[0], w.V[1], w.d, w.done_iter, w.pos, w.rank_tmp, Uw, Vw));
  // ---- fallback: FP64 Jacobi (exits at once when Phase B converged)
  return launch_svd_jacobi_f64(W, k, trunc_rtol, w.done_iter, w.Wc, w.Vc, sig, Uw, Vw, rank, sweeps, status, stream);
}

}  // namespace cabs
