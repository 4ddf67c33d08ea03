// Step a5 -- weighted k-means sampling on the pilot embeddings (Section 3.2,
// Eq. wkmeans; Algorithm 2, step 3).
//
// Objective: sum_l w_l |x_l - z_s(l)|^2 with w_l = Upsilon(|x_l|) = |x_l|^p.
// Each iteration assigns every point to its nearest centre (ties to the lower
// centre index) and moves each centre to the weighted mean of its members;
// a centre with no weight keeps its position. Centres start at the points
// given by init_rows (the pilot rows, in draw order).
//
// Assignment kernels
//   FP64: direct differences sum_q (x_q - z_q)^2, summed in dimension order.
//   FP32: expansion |z|^2 - 2 x.z (|x|^2 is common to a row), a register-tiled
//         CUDA-core contraction: a CTA holds 64 points x all (<= 256)
//         centres, each thread 8 x 8 accumulators; the row argmin is a
//         warp-shuffle reduction over the 32 lanes that share a point row.
//   TF32/BF16: tensor-core contraction (separate kernel file), with near ties
//         re-checked in FP32.
// Update: a stable counting sort of the labels lists each centre's members in
// index order; four CTAs per centre sum contiguous parts of that list (16
// warps each, warp sums in warp order) and a combine kernel adds the parts in
// order, so the centres do not depend on scheduling.
// Energies (weighted encoding errors) are per-CTA FP64 partials summed in a
// fixed order.
#include "common.cuh"
#include "kernels.cuh"
#include "profile.cuh"
#include "tc_assign.cuh"

namespace cabs {
namespace {

// -------------------------------------------------------------- helpers

template <typename T>
__global__ void point_prep_kernel(const T* __restrict__ X, long long M, int d, float p, T* __restrict__ xn,
                                  T* __restrict__ w) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long l = warp; l < M; l += nwarps) {
    T s = T(0);
    for (int q = lane; q < d; q += 32) s = fma(X[l * d + q], X[l * d + q], s);
    s = warp_sum(s);
    if (lane == 0) {
      xn[l] = s;
      w[l] = (p == 0.0f) ? T(1) : (T)pow((double)dev_sqrt<T>(s), (double)p);
    }
  }
}

template <typename T>
__global__ void init_centres_kernel(const T* __restrict__ X, long long M, int d, const int* __restrict__ rows,
                                    int k2, T* __restrict__ Z) {
  const int j = blockIdx.x;
  if (j >= k2) return;
  const long long l = min(max((long long)rows[j], 0ll), M - 1);
  for (int q = threadIdx.x; q < d; q += blockDim.x) Z[(size_t)j * d + q] = X[l * d + q];
}

template <typename T>
__global__ void centre_norms_kernel(const T* __restrict__ Z, int k2, int d, T* __restrict__ zn) {
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (j >= k2) return;
  T s = T(0);
  for (int q = lane; q < d; q += 32) s = fma(Z[(size_t)j * d + q], Z[(size_t)j * d + q], s);
  s = warp_sum(s);
  if (lane == 0) zn[j] = s;
}

// ------------------------------------------------------ FP32 assignment

constexpr int kAM = 64;   // points per CTA tile
constexpr int kAK = 16;   // dimensions per stage
constexpr int kAN = 256;  // centres per CTA (all of them)

__global__ void __launch_bounds__(256) assign_f32_kernel(const float* __restrict__ X, long long M, int d,
                                                         const float* __restrict__ Z, const float* __restrict__ zn,
                                                         int k2, int* __restrict__ labels) {
  __shared__ __align__(16) float xs[kAK][kAM + 4];
  __shared__ __align__(16) float zs[kAK][kAN + 4];
  const int tid = threadIdx.x, ty = tid >> 5, tx = tid & 31;
  const long long m0 = (long long)blockIdx.x * kAM;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[i][c] = 0.f;
  for (int q0 = 0; q0 < d; q0 += kAK) {
    {
      const int p = tid >> 2, qq = (tid & 3) * 4;
      const long long l = m0 + p;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int q = q0 + qq + e;
        xs[qq + e][p] = (l < M && q < d) ? X[l * d + q] : 0.f;
      }
      const int j = tid;
#pragma unroll
      for (int e = 0; e < kAK; ++e) {
        const int q = q0 + e;
        zs[e][j] = (j < k2 && q < d) ? Z[(size_t)j * d + q] : 0.f;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kAK; ++kk) {
      float a[8], b[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = xs[kk][ty * 8 + i];
#pragma unroll
      for (int c = 0; c < 8; ++c) b[c] = zs[kk][tx + 32 * c];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[i][c] = fmaf(a[i], b[c], acc[i][c]);
    }
    __syncthreads();
  }
  float znr[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int j = tx + 32 * c;
    znr[c] = j < k2 ? zn[j] : 0.f;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const long long l = m0 + ty * 8 + i;
    float best = pos_inf<float>();
    int bj = 0x7fffffff;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int j = tx + 32 * c;
      const float dist = fmaf(-2.f, acc[i][c], znr[c]);
      if (j < k2 && dist < best) {
        best = dist;
        bj = j;
      }
    }
    warp_argmin(best, bj);
    if (tx == 0 && l < M) labels[l] = bj;
  }
}

// ------------------------------------------------------ FP64 assignment

constexpr int kDM = 32;  // points per CTA
constexpr int kDG = 8;   // centres per stage (one per thread group lane)

__global__ void __launch_bounds__(256) assign_f64_kernel(const double* __restrict__ X, long long M, int d,
                                                         const double* __restrict__ Z, int k2,
                                                         const double* __restrict__ w, int* __restrict__ labels,
                                                         double* __restrict__ part_e) {
  extern __shared__ __align__(16) double dsm[];
  const int ld = d + 1;
  double* xs = dsm;             // kDM x ld
  double* zs = dsm + kDM * ld;  // kDG x ld
  __shared__ double esum[8];
  const int tid = threadIdx.x, pl = tid >> 3, g = tid & 7;
  const long long m0 = (long long)blockIdx.x * kDM;
  for (int e = tid; e < kDM * d; e += blockDim.x) {
    const int p = e / d, q = e - p * d;
    const long long l = m0 + p;
    xs[p * ld + q] = l < M ? X[l * d + q] : 0.0;
  }
  double best = pos_inf<double>();
  int bj = 0x7fffffff;
  for (int c0 = 0; c0 < k2; c0 += kDG) {
    __syncthreads();
    for (int e = tid; e < kDG * d; e += blockDim.x) {
      const int jj = e / d, q = e - jj * d;
      const int j = c0 + jj;
      zs[jj * ld + q] = j < k2 ? Z[(size_t)j * d + q] : 0.0;
    }
    __syncthreads();
    const int j = c0 + g;
    if (j < k2) {
      double s = 0.0;
      const double* xr = xs + pl * ld;
      const double* zr = zs + g * ld;
      for (int q = 0; q < d; ++q) {
        const double t = xr[q] - zr[q];
        s = fma(t, t, s);
      }
      if (s < best) {
        best = s;
        bj = j;
      }
    }
  }
#pragma unroll
  for (int off = 4; off > 0; off >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, best, off);
    const int oi = __shfl_xor_sync(0xffffffffu, bj, off);
    if (lex_less(ov, oi, best, bj)) {
      best = ov;
      bj = oi;
    }
  }
  const long long l = m0 + pl;
  double e = 0.0;
  if (g == 0 && l < M) {
    labels[l] = bj;
    e = w[l] * best;
  }
  e = warp_sum(e);
  if ((tid & 31) == 0) esum[tid >> 5] = e;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int i = 0; i < 8; ++i) s += esum[i];
    part_e[blockIdx.x] = s;
  }
}

// ---------------------------------------------------- exact energies
// Weighted encoding error sum_l w_l |x_l - z_s(l)|^2 by direct differences,
// one warp per point (lanes over dimensions); CTA b sums a fixed contiguous
// range of points, so the partial sums do not depend on scheduling.

template <typename T>
__global__ void __launch_bounds__(256) energy_exact_kernel(const T* __restrict__ X, long long M, int d,
                                                           const T* __restrict__ Z, int k2,
                                                           const int* __restrict__ labels, const T* __restrict__ w,
                                                           double* __restrict__ part) {
  __shared__ double red[8];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const long long lo = M * blockIdx.x / gridDim.x, hi = M * (blockIdx.x + 1) / gridDim.x;
  double acc = 0.0;
  for (long long l0 = lo + 4 * wi; l0 < hi; l0 += 32) {
    T s4[4];
    int j4[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      j4[u] = l0 + u < hi ? min(max(labels[l0 + u], 0), k2 - 1) : 0;
      s4[u] = T(0);
    }
    for (int q = lane; q < d; q += 32) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (l0 + u < hi) {
          const T t = X[(l0 + u) * d + q] - Z[(size_t)j4[u] * d + q];
          s4[u] = fma(t, t, s4[u]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const T sv = warp_sum(s4[u]);
      if (lane == 0 && l0 + u < hi) acc += (double)w[l0 + u] * (double)sv;
    }
  }
  if (lane == 0) red[wi] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < 8; ++i) t += red[i];
    part[blockIdx.x] = t;
  }
}

// ------------------------------------------------------------- update

constexpr int kUWarps = 16;
constexpr int kUMaxPerLane = CABS_MAX_K / 32;

// ------------------------------------------------ members by centre
// The update reads each centre's members from a stable counting sort of the
// labels (index order within a centre) instead of scanning all labels once
// per centre: per-chunk histograms, an offset table, a stable scatter, then
// one CTA per centre over its own members only.

constexpr int kSortChunk = 256;  // points per histogram / scatter chunk

__global__ void __launch_bounds__(256) label_hist_kernel(const int* __restrict__ labels, long long M, int k2,
                                                         int* __restrict__ chunk_cnt) {
  __shared__ int h[CABS_MAX_K];
  for (int j = threadIdx.x; j < k2; j += blockDim.x) h[j] = 0;
  __syncthreads();
  const long long lo = (long long)blockIdx.x * kSortChunk, hi = min(M, lo + kSortChunk);
  for (long long l = lo + threadIdx.x; l < hi; l += blockDim.x) {
    const int j = labels[l];
    if (j >= 0 && j < k2) atomicAdd(&h[j], 1);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < k2; j += blockDim.x) chunk_cnt[(size_t)blockIdx.x * k2 + j] = h[j];
}

// One CTA of 4 CABS_MAX_K threads: chunk_off[c][j] = start of chunk c's
// members of centre j in the sorted order; base[j], cnt[j] = centre j's
// range. Four threads per centre each take a quarter of the chunks (so the
// count loads of one centre are spread over four threads); the centre totals
// are scanned by warp shuffles and a scan of the warp totals.
constexpr int kOffParts = 4;
__global__ void __launch_bounds__(kOffParts * CABS_MAX_K) label_offsets_kernel(const int* __restrict__ chunk_cnt,
                                                                               int chunks, int k2,
                                                                               int* __restrict__ chunk_off,
                                                                               int* __restrict__ base,
                                                                               int* __restrict__ cnt) {
  __shared__ int ptot[kOffParts][CABS_MAX_K];  // each part's count of each centre
  __shared__ int pref[CABS_MAX_K];             // exclusive prefix of the centre totals inside their warp
  __shared__ int wtot[CABS_MAX_K / 32];        // warp totals, then their inclusive scan
  const int j = threadIdx.x % CABS_MAX_K, part = threadIdx.x / CABS_MAX_K;
  const int lane = j & 31, w = j >> 5;
  const int c0 = (int)((long long)chunks * part / kOffParts), c1 = (int)((long long)chunks * (part + 1) / kOffParts);
  int tp = 0;
  if (j < k2) {
#pragma unroll 8
    for (int c = c0; c < c1; ++c) tp += chunk_cnt[(size_t)c * k2 + j];
  }
  ptot[part][j] = tp;
  __syncthreads();
  int t = 0;
  for (int q = 0; q < kOffParts; ++q) t += ptot[q][j];  // centre j's total (every part)
  if (part == 0) {
    int incl = t;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int o = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += o;
    }
    if (lane == 31) wtot[w] = incl;
    pref[j] = incl - t;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    int x = lane < CABS_MAX_K / 32 ? wtot[lane] : 0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int o = __shfl_up_sync(0xffffffffu, x, off);
      if (lane >= off) x += o;
    }
    if (lane < CABS_MAX_K / 32) wtot[lane] = x;
  }
  __syncthreads();
  if (j < k2) {
    int run = pref[j] + (w > 0 ? wtot[w - 1] : 0);  // start of centre j
    if (part == 0) {
      base[j] = run;
      cnt[j] = t;
    }
    for (int q = 0; q < part; ++q) run += ptot[q][j];  // the earlier parts' members of centre j
#pragma unroll 8
    for (int c = c0; c < c1; ++c) {
      chunk_off[(size_t)c * k2 + j] = run;
      run += chunk_cnt[(size_t)c * k2 + j];
    }
  }
}

// One warp per chunk, 32 points at a time in index order: a point's slot is
// its centre's running offset plus its rank among the batch's points of the
// same centre (stable).
__global__ void __launch_bounds__(32) label_scatter_kernel(const int* __restrict__ labels, long long M, int k2,
                                                           const int* __restrict__ chunk_off, int* __restrict__ perm) {
  __shared__ int run[CABS_MAX_K];
  const int lane = threadIdx.x;
  for (int j = lane; j < k2; j += 32) run[j] = chunk_off[(size_t)blockIdx.x * k2 + j];
  __syncwarp();
  const long long lo = (long long)blockIdx.x * kSortChunk, hi = min(M, lo + kSortChunk);
  for (long long b = lo; b < hi; b += 32) {
    const long long l = b + lane;
    int j = l < hi ? labels[l] : -1;
    if (j >= k2) j = -1;
    const unsigned act = __ballot_sync(0xffffffffu, j >= 0);
    if (j >= 0) {
      const unsigned peers = __match_any_sync(act, j);
      const int rank = __popc(peers & ((1u << lane) - 1u));
      perm[run[j] + rank] = (int)l;
      __syncwarp(act);
      if (lane == 31 - __clz(peers)) run[j] += __popc(peers);
    }
    __syncwarp();
  }
}

// CTA (j, p) over part p of centre j's members perm[base_j, base_j + cnt_j)
// (kUParts parts, so a large cluster -- sparse inputs put every empty row in
// one -- spreads over several SMs): warp i takes the i-th contiguous piece of
// the part, in order, and the warps' sums are added in warp order. The part
// sums go to `part`; update_combine_kernel adds the parts in order
// (deterministic) and forms the weighted mean (an empty cluster keeps its
// centre), the count and, with energy, sum w_l |x_l - z_j|^2 with the centre
// the assignment used.
constexpr int kUParts = 4;

template <typename T>
__global__ void __launch_bounds__(kUWarps * 32, sizeof(T) == 4 ? 2 : 1) update_sorted_kernel(
    const T* __restrict__ X, int d, const int* __restrict__ perm, const int* __restrict__ base,
    const int* __restrict__ cnt_in, const T* __restrict__ w, const T* __restrict__ Zcur, T* __restrict__ part,
    double* __restrict__ part_e, bool want_e) {
  __shared__ T accs[kUWarps][CABS_MAX_K];
  __shared__ T zc[CABS_MAX_K];
  __shared__ T wsums[kUWarps];
  __shared__ double esums[kUWarps];
  const int j = blockIdx.x, pp = blockIdx.y, k2 = gridDim.x;
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const long long nm = cnt_in[j];
  const long long p_lo = base[j] + nm * pp / kUParts, p_hi = base[j] + nm * (pp + 1) / kUParts;
  const long long pn = p_hi - p_lo;
  const long long lo = p_lo + pn * wi / kUWarps, hi = p_lo + pn * (wi + 1) / kUWarps;
  for (int q = threadIdx.x; q < CABS_MAX_K; q += blockDim.x) zc[q] = q < d ? Zcur[(size_t)j * d + q] : T(0);
  __syncthreads();
  T acc[kUMaxPerLane];
#pragma unroll
  for (int s2 = 0; s2 < kUMaxPerLane; ++s2) acc[s2] = T(0);
  T wsum = T(0), esum = T(0);
  for (long long e0 = lo; e0 < hi; e0 += 4) {
    long long ls[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) ls[u] = e0 + u < hi ? (long long)perm[e0 + u] : -1;
    T xv[4][kUMaxPerLane];
    T wv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      wv[u] = ls[u] >= 0 ? w[ls[u]] : T(0);
#pragma unroll
      for (int s2 = 0; s2 < kUMaxPerLane; ++s2) {
        const int q = lane + 32 * s2;
        xv[u][s2] = (ls[u] >= 0 && q < d) ? X[ls[u] * d + q] : T(0);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (ls[u] >= 0) {
#pragma unroll
        for (int s2 = 0; s2 < kUMaxPerLane; ++s2) acc[s2] = fma(wv[u], xv[u][s2], acc[s2]);
        if (want_e) {
          T ee = T(0);
#pragma unroll
          for (int s2 = 0; s2 < kUMaxPerLane; ++s2) {
            const T t = xv[u][s2] - zc[lane + 32 * s2];
            ee = fma(t, t, ee);
          }
          esum = fma(wv[u], ee, esum);
        }
        wsum += wv[u];
      }
    }
  }
#pragma unroll
  for (int s2 = 0; s2 < kUMaxPerLane; ++s2) accs[wi][lane + 32 * s2] = acc[s2];
  const T ew = warp_sum(esum);
  if (lane == 0) {
    wsums[wi] = wsum;
    esums[wi] = (double)ew;
  }
  __syncthreads();
  // part layout: [p][j][d + 1]: the d sums and the weight sum; energy in part_e[p][j]
  T* out = part + ((size_t)pp * k2 + j) * (d + 1);
  for (int q = threadIdx.x; q < d; q += blockDim.x) {
    T sq = T(0);
    for (int i = 0; i < kUWarps; ++i) sq += accs[i][q];
    out[q] = sq;
  }
  if (threadIdx.x == 0) {
    T W = T(0);
    double e = 0.0;
    for (int i = 0; i < kUWarps; ++i) {
      W += wsums[i];
      e += esums[i];
    }
    out[d] = W;
    part_e[(size_t)pp * k2 + j] = e;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) update_combine_kernel(const T* __restrict__ part,
                                                             const double* __restrict__ part_e, int d,
                                                             const int* __restrict__ cnt_in,
                                                             const T* __restrict__ Zcur, T* __restrict__ Znext,
                                                             int* __restrict__ counts, double* __restrict__ energy) {
  const int j = blockIdx.x, k2 = gridDim.x;
  T W = T(0);
  for (int pp = 0; pp < kUParts; ++pp) W += part[((size_t)pp * k2 + j) * (d + 1) + d];
  for (int q = threadIdx.x; q < d; q += blockDim.x) {
    T sq = T(0);
    for (int pp = 0; pp < kUParts; ++pp) sq += part[((size_t)pp * k2 + j) * (d + 1) + q];
    Znext[(size_t)j * d + q] = W > T(0) ? sq / W : Zcur[(size_t)j * d + q];
  }
  if (threadIdx.x == 0) {
    if (counts) counts[j] = cnt_in[j];
    if (energy) {
      double e = 0.0;
      for (int pp = 0; pp < kUParts; ++pp) e += part_e[(size_t)pp * k2 + j];
      energy[j] = e;
    }
  }
}

__global__ void max_count_kernel(const int* __restrict__ counts, int k2, int* __restrict__ out) {
  __shared__ int mx[256];
  int m = 0;
  for (int j = threadIdx.x; j < k2; j += blockDim.x) m = max(m, counts[j]);
  mx[threadIdx.x] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    int r = 0;
    for (int i = 0; i < (int)blockDim.x; ++i) r = max(r, mx[i]);
    *out = r;
  }
}

__global__ void energy_reduce_kernel(const double* __restrict__ part, int nb, int iters, double* __restrict__ out) {
  const int t = threadIdx.x;
  if (t >= iters) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[(size_t)t * nb + b];
  out[t] = s;
}

template <typename T>
__global__ void copy_kernel(const T* __restrict__ a, T* __restrict__ b, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = a[i];
}

// ---------------------------------------------------------- workspace

struct KmWs {
  void *xn, *w, *Za, *Zb, *zn, *tc;
  int *labels, *counts, *T;
  int *chunk_cnt, *chunk_off, *perm, *lbase, *lcnt;  // members by centre
  void* upart;                                        // per-part sums of the update
  double* upart_e;                                    //   and their energies
  double *part_e, *energy;
};

int sort_chunks(int64_t M) { return (int)((M + kSortChunk - 1) / kSortChunk); }

// Partial energies per iteration: the FP64 assignment kernel writes one per
// CTA of its grid; in the other modes the update writes one per centre.
int energy_parts(int64_t M, int k2, int prec) {
  if (prec == CABS_PREC_FP64) return ceil_div(M, kDM);
  return k2;
}

// Grid of the exact-energy kernel (the encoding error of given representatives).
int energy_blocks(int64_t M) { return std::max(1, std::min(ceil_div(M, 64), sm_count() * 4)); }

KmWs carve_km(Carve& cv, int64_t M, int d, int k2, int iters, int prec) {
  const size_t eb = elem_bytes(prec);
  KmWs w;
  w.xn = cv.take<char>(M * eb);
  w.w = cv.take<char>(M * eb);
  w.Za = cv.take<char>((size_t)k2 * d * eb);
  w.Zb = cv.take<char>((size_t)k2 * d * eb);
  w.zn = cv.take<char>((size_t)k2 * eb);
  w.labels = cv.take<int>(M);
  w.counts = cv.take<int>(k2);
  w.T = cv.take<int>(1);
  w.part_e = cv.take<double>((size_t)std::max(iters, 1) * std::max(energy_parts(M, k2, prec), energy_blocks(M)));
  w.energy = cv.take<double>(std::max(iters, 1));
  w.chunk_cnt = cv.take<int>((size_t)sort_chunks(M) * k2);
  w.chunk_off = cv.take<int>((size_t)sort_chunks(M) * k2);
  w.perm = cv.take<int>(M);
  w.lbase = cv.take<int>(k2);
  w.lcnt = cv.take<int>(k2);
  w.upart = cv.take<char>((size_t)kUParts * k2 * (d + 1) * eb);
  w.upart_e = cv.take<double>((size_t)kUParts * k2);
  w.tc = nullptr;
  if (prec == CABS_PREC_TF32 || prec == CABS_PREC_BF16) {
    w.tc = cv.base ? cv.base + cv.used : nullptr;
    tc_assign_carve(cv, M, d, k2);
  }
  return w;
}

template <typename T>
cabs_status assign_once(const T* X, int64_t M, int d, const T* Z, int k2, int prec, const T* xn, const T* w, T* zn,
                        int* labels, double* part_e, int* d_recheck, bool first, void* tcws, cudaStream_t stream);

template <>
cabs_status assign_once<double>(const double* X, int64_t M, int d, const double* Z, int k2, int prec,
                                const double* xn, const double* w, double* zn, int* labels, double* part_e,
                                int* d_recheck, bool first, void* tcws, cudaStream_t stream) {
  const int nb = ceil_div(M, kDM);
  const size_t smem = (size_t)(kDM + kDG) * (d + 1) * sizeof(double);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(assign_f64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  CABS_LAUNCH(stream, "assign_f64_kernel", assign_f64_kernel<<<nb, 256, smem, stream>>>(X, M, d, Z, k2, w, labels, part_e));
  return CABS_OK;
}

template <>
cabs_status assign_once<float>(const float* X, int64_t M, int d, const float* Z, int k2, int prec, const float* xn,
                               const float* w, float* zn, int* labels, double* part_e, int* d_recheck, bool first,
                               void* tcws, cudaStream_t stream) {
  CABS_LAUNCH(stream, "centre_norms_kernel", centre_norms_kernel<float><<<ceil_div(k2, 8), 256, 0, stream>>>(Z, k2, d, zn));
  if (prec == CABS_PREC_FP32) {
    CABS_LAUNCH(stream, "assign_f32_kernel",
                assign_f32_kernel<<<ceil_div(M, kAM), 256, 0, stream>>>(X, M, d, Z, zn, k2, labels));
  } else {
    CABS_TRY(tc_assign_launch(X, M, d, Z, zn, k2, xn, w, labels, d_recheck, prec == CABS_PREC_BF16, first, tcws,
                              stream));
  }
  (void)part_e;  // the update pass adds up this iteration's energy
  return CABS_OK;
}

template <typename T>
cabs_status kmeans_typed(const T* X, int64_t M, int d, const int* init_rows, int k2, int iters, int prec, float p,
                         int* labels_out, T* centres, double* energy, int* d_T, int* d_recheck, void* ws,
                         size_t ws_bytes, cudaStream_t stream) {
  Carve cv(ws, ws_bytes);
  KmWs w = carve_km(cv, M, d, k2, iters, prec);
  void* tcws = w.tc;
  if (!cv.fits()) {
    set_error("k-means workspace too small: need %zu bytes, got %zu", cv.used, ws_bytes);
    return CABS_ENOMEM;
  }
  const int sms = sm_count();
  T* xn = (T*)w.xn;
  T* wt = (T*)w.w;
  CABS_LAUNCH(stream, "point_prep_kernel", point_prep_kernel<T><<<std::max(1, std::min(ceil_div(M, 8), sms * 16)), 256, 0, stream>>>(X, M, d, p, xn, wt));
  T* Zc = (T*)w.Za;
  T* Zn = (T*)w.Zb;
  CABS_LAUNCH(stream, "init_centres_kernel", init_centres_kernel<T><<<k2, 128, 0, stream>>>(X, M, d, init_rows, k2, Zc));
  const int nb = energy_parts(M, k2, prec);
  for (int t = 0; t < iters; ++t) {
    int* lab = labels_out ? labels_out + (size_t)t * M : w.labels;
    double* pe = w.part_e + (size_t)t * nb;
    CABS_TRY(assign_once<T>(X, M, d, Zc, k2, prec, xn, wt, (T*)w.zn, lab, pe, d_recheck, t == 0, tcws, stream));
    const int ch = sort_chunks(M);
    CABS_LAUNCH(stream, "label_hist_kernel", label_hist_kernel<<<ch, 256, 0, stream>>>(lab, M, k2, w.chunk_cnt));
    CABS_LAUNCH(stream, "label_offsets_kernel",
                label_offsets_kernel<<<1, kOffParts * CABS_MAX_K, 0, stream>>>(w.chunk_cnt, ch, k2, w.chunk_off, w.lbase, w.lcnt));
    CABS_LAUNCH(stream, "label_scatter_kernel",
                label_scatter_kernel<<<ch, 32, 0, stream>>>(lab, M, k2, w.chunk_off, w.perm));
    CABS_LAUNCH(stream, "update_kernel",
                update_sorted_kernel<T><<<dim3(k2, kUParts), kUWarps * 32, 0, stream>>>(
                    X, d, w.perm, w.lbase, w.lcnt, wt, Zc, (T*)w.upart, w.upart_e, prec != CABS_PREC_FP64));
    CABS_LAUNCH(stream, "update_combine_kernel",
                update_combine_kernel<T><<<k2, 256, 0, stream>>>((const T*)w.upart, w.upart_e, d, w.lcnt, Zc, Zn,
                                                                 w.counts,
                                                                 prec == CABS_PREC_FP64 ? nullptr : pe));
    T* tmp = Zc;
    Zc = Zn;
    Zn = tmp;
  }
  if (iters > 0) {
    if (energy) {
      CABS_LAUNCH(stream, "energy_reduce_kernel", energy_reduce_kernel<<<1, 64, 0, stream>>>(w.part_e, nb, iters, energy));
    }
    if (d_T) {
      CABS_LAUNCH(stream, "max_count_kernel", max_count_kernel<<<1, 256, 0, stream>>>(w.counts, k2, d_T));
    }
  }
  CABS_LAUNCH(stream, "copy_kernel", copy_kernel<T><<<std::max(1, ceil_div((int64_t)k2 * d, 256)), 256, 0, stream>>>(Zc, centres, (long long)k2 * d));
  return CABS_OK;
}

template <typename T>
cabs_status enc_err_typed(const T* X, int64_t M, int d, const int* reps, int k2, int prec, float p, double* out,
                          void* ws, size_t ws_bytes, cudaStream_t stream) {
  Carve cv(ws, ws_bytes);
  KmWs w = carve_km(cv, M, d, k2, 1, prec);
  void* tcws = w.tc;
  if (!cv.fits()) {
    set_error("encoding-error workspace too small");
    return CABS_ENOMEM;
  }
  const int sms = sm_count();
  CABS_LAUNCH(stream, "point_prep_kernel", point_prep_kernel<T><<<std::max(1, std::min(ceil_div(M, 8), sms * 16)), 256, 0, stream>>>(X, M, d, p, (T*)w.xn,
                                                                                           (T*)w.w));
  CABS_LAUNCH(stream, "init_centres_kernel", init_centres_kernel<T><<<k2, 128, 0, stream>>>(X, M, d, reps, k2, (T*)w.Za));
  CABS_TRY(assign_once<T>(X, M, d, (T*)w.Za, k2, prec, (T*)w.xn, (T*)w.w, (T*)w.zn, w.labels, w.part_e, nullptr,
                          true, tcws, stream));
  int nb = energy_parts(M, k2, prec);
  if (prec != CABS_PREC_FP64) {
    nb = energy_blocks(M);
    CABS_LAUNCH(stream, "energy_exact_kernel",
                energy_exact_kernel<T><<<nb, 256, 0, stream>>>(X, M, d, (T*)w.Za, k2, w.labels, (T*)w.w, w.part_e));
  }
  CABS_LAUNCH(stream, "energy_reduce_kernel", energy_reduce_kernel<<<1, 64, 0, stream>>>(w.part_e, nb, 1, out));
  return CABS_OK;
}

}  // namespace

size_t kmeans_ws_bytes(int64_t M, int d, int k2, int iters, int prec) {
  Carve cv;
  carve_km(cv, M, d, k2, iters, prec);
  return cv.used;
}

cabs_status launch_kmeans(const void* X, int64_t M, int d, const int* init_rows, int k2, int iters, int prec,
                          float upsilon_pow, int* labels, void* centres, double* energy, int* d_T, int* d_recheck,
                          void* ws, size_t ws_bytes, cudaStream_t stream) {
  if (prec == CABS_PREC_FP64)
    return kmeans_typed<double>((const double*)X, M, d, init_rows, k2, iters, prec, upsilon_pow, labels,
                                (double*)centres, energy, d_T, d_recheck, ws, ws_bytes, stream);
  return kmeans_typed<float>((const float*)X, M, d, init_rows, k2, iters, prec, upsilon_pow, labels, (float*)centres,
                             energy, d_T, d_recheck, ws, ws_bytes, stream);
}

cabs_status launch_encoding_error(const void* X, int64_t M, int d, const int* reps, int k2, int prec,
                                  float upsilon_pow, double* out, void* ws, size_t ws_bytes, cudaStream_t stream) {
  if (prec == CABS_PREC_FP64)
    return enc_err_typed<double>((const double*)X, M, d, reps, k2, prec, upsilon_pow, out, ws, ws_bytes, stream);
  return enc_err_typed<float>((const float*)X, M, d, reps, k2, prec, upsilon_pow, out, ws, ws_bytes, stream);
}

}  // namespace cabs
