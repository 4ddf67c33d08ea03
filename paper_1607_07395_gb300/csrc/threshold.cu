// Follow-up selection by hard threshold (Section 5, follow-up variant (f)):
// the k2 rows of an embedding X (P or Q) with the largest norm, ties to the
// lower row index, returned in ascending order. It replaces the weighted
// k-means and the snap of Algorithm 2, step 3 when CABS_FLAG_HARD_THRESHOLD
// is set.
//
//  1. sq_norms_kernel: squared row norms summed in dimension order, one
//     multiply and one add per term (as a plain loop would), so FP64 keys
//     equal those of a sequential FP64 sum bit for bit. A warp stages 32 rows
//     x 32 dimensions through shared memory so the loads are coalesced while
//     each lane sums one row. Non-negative floats order like their bit
//     patterns, so the bits are the selection keys.
//  Leverage-score variant (Section 5, follow-up variant (e)): lev_keys_kernel
//     takes the leverage score l_i = |X_i|^2 of each row of an orthonormal
//     factor X (FP64 sum) and the A-Res key of Efraimidis and Spirakis (2006),
//     u_i^(1/l_i), ranked through the increasing map l_i / (-ln u_i) in FP64,
//     with u_i = ((r_i >> 11) + 1/2) 2^-53 and r_i = word 0 of
//     Philox((i, 0, 0, 0), (seed, tag)); the k2 largest keys are a draw of k2
//     distinct rows with probabilities proportional to l.
//  2. select_topk_kernel (one CTA): a radix select finds the k2-th largest
//     key T, 8 bits at a time with warp-aggregated shared-memory histograms;
//     then one pass in index order keeps every row with key > T and the
//     lowest-indexed rows with key == T, placing each by a block-wide scan,
//     which yields the rows already sorted.
#include "common.cuh"
#include "kernels.cuh"
#include "profile.cuh"

namespace cabs {
namespace {

constexpr int kSelThreads = 1024;

template <typename T>
__device__ __forceinline__ unsigned long long key_bits(T v);
template <>
__device__ __forceinline__ unsigned long long key_bits<float>(float v) {
  return (unsigned long long)__float_as_uint(v);
}
template <>
__device__ __forceinline__ unsigned long long key_bits<double>(double v) {
  return (unsigned long long)__double_as_longlong(v);
}

__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

constexpr int kNormThreads = 128;

template <typename T>
__global__ void __launch_bounds__(kNormThreads) sq_norms_kernel(const T* __restrict__ X, long long M, int d,
                                                                unsigned long long* __restrict__ key) {
  __shared__ T tile[kNormThreads / 32][32][33];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long r0 = ((long long)blockIdx.x * (blockDim.x >> 5) + wi) * 32; r0 < M; r0 += nwarps * 32) {
    T s = T(0);
    for (int q0 = 0; q0 < d; q0 += 32) {
#pragma unroll 4
      for (int r = 0; r < 32; ++r) {
        const long long l = r0 + r;
        tile[wi][r][lane] = (l < M && q0 + lane < d) ? X[l * d + q0 + lane] : T(0);
      }
      __syncwarp();
      const int qn = min(32, d - q0);
      for (int q = 0; q < qn; ++q) {
        const T x = tile[wi][lane][q];
        s = add_rn(s, mul_rn(x, x));
      }
      __syncwarp();
    }
    if (r0 + lane < M) key[r0 + lane] = key_bits<T>(s);
  }
}

template <typename T>
__global__ void __launch_bounds__(kNormThreads) lev_keys_kernel(const T* __restrict__ X, long long M, int d,
                                                                uint64_t seed, int tag,
                                                                unsigned long long* __restrict__ key) {
  __shared__ T tile[kNormThreads / 32][32][33];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long r0 = ((long long)blockIdx.x * (blockDim.x >> 5) + wi) * 32; r0 < M; r0 += nwarps * 32) {
    double s = 0.0;
    for (int q0 = 0; q0 < d; q0 += 32) {
#pragma unroll 4
      for (int r = 0; r < 32; ++r) {
        const long long l = r0 + r;
        tile[wi][r][lane] = (l < M && q0 + lane < d) ? X[l * d + q0 + lane] : T(0);
      }
      __syncwarp();
      const int qn = min(32, d - q0);
      for (int q = 0; q < qn; ++q) {
        const double x = (double)tile[wi][lane][q];
        s = fma(x, x, s);
      }
      __syncwarp();
    }
    const long long i = r0 + lane;
    if (i < M) {
      const uint64_t r = philox4x64_10((uint64_t)i, 0, 0, 0, seed, (uint64_t)tag).v[0];
      const double u = ((double)(r >> 11) + 0.5) * 1.1102230246251565e-16;  // 2^-53
      key[i] = (unsigned long long)__double_as_longlong(s / -log(u));
    }
  }
}

// Block-wide exclusive scan of one flag per thread; returns the prefix and
// writes the block total to *total (all threads).
__device__ __forceinline__ int block_scan(int v, int* warp_sums, int* total) {
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int o = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += o;
  }
  if (lane == 31) warp_sums[wi] = incl;
  __syncthreads();
  if (wi == 0) {
    const int w = lane < (kSelThreads >> 5) ? warp_sums[lane] : 0;
    int wincl = w;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int o = __shfl_up_sync(0xffffffffu, wincl, off);
      if (lane >= off) wincl += o;
    }
    warp_sums[lane] = wincl - w;  // exclusive prefix of the warps
    if (lane == 31) warp_sums[32] = wincl;
  }
  __syncthreads();
  const int r = warp_sums[wi] + incl - v;
  *total = warp_sums[32];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kSelThreads) select_topk_kernel(const unsigned long long* __restrict__ key,
                                                                  long long M, int k2, int top_shift,
                                                                  int* __restrict__ sorted) {
  __shared__ unsigned int hist[256];
  __shared__ unsigned long long prefix_s;
  __shared__ long long want_s;
  __shared__ int warp_sums[33];
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) {
    prefix_s = 0ull;
    want_s = k2;  // rank (from the top) of the key sought inside the current prefix group
  }
  unsigned long long mask = 0ull;
  for (int shift = top_shift; shift >= 0; shift -= 8) {
    for (int b = tid; b < 256; b += blockDim.x) hist[b] = 0u;
    __syncthreads();
    const unsigned long long prefix = prefix_s;
    for (long long i0 = 0; i0 < M; i0 += blockDim.x) {
      const long long i = i0 + tid;
      const unsigned long long k = i < M ? key[i] : 0ull;
      const bool in = i < M && (k & mask) == prefix;
      const unsigned bin = (unsigned)((k >> shift) & 255ull);
      // one shared atomic per distinct bin of the warp
      const unsigned act = __ballot_sync(0xffffffffu, in);
      if (in) {
        const unsigned peers = __match_any_sync(act, bin);
        if ((int)(__ffs(peers) - 1) == lane) atomicAdd(&hist[bin], (unsigned)__popc(peers));
      }
    }
    __syncthreads();
    if (tid == 0) {
      long long cum = 0;
      const long long want = want_s;
      for (int b = 255; b >= 0; --b) {
        if (cum + hist[b] >= want) {
          want_s = want - cum;
          prefix_s = prefix | ((unsigned long long)b << shift);
          break;
        }
        cum += hist[b];
      }
    }
    mask |= 255ull << shift;
    __syncthreads();
  }
  const unsigned long long T = prefix_s;
  const long long take_eq = want_s;  // rows with key == T to keep, lowest indices first
  long long out_base = 0, eq_seen = 0;
  for (long long i0 = 0; i0 < M; i0 += blockDim.x) {
    const long long i = i0 + tid;
    const unsigned long long k = i < M ? key[i] : 0ull;
    const int eq = (i < M && k == T) ? 1 : 0;
    int eq_total;
    const int eq_rank = block_scan(eq, warp_sums, &eq_total);
    const int inc = ((i < M && k > T) || (eq && eq_seen + eq_rank < take_eq)) ? 1 : 0;
    int inc_total;
    const int pos = block_scan(inc, warp_sums, &inc_total);
    if (inc && out_base + pos < k2) sorted[out_base + pos] = (int)i;
    out_base += inc_total;
    eq_seen += eq_total;
  }
}

template <typename T>
cabs_status threshold_typed(const T* X, int64_t M, int d, int k2, int* sorted, void* ws, size_t ws_bytes,
                            cudaStream_t stream) {
  if (ws_bytes < (size_t)M * sizeof(unsigned long long)) {
    set_error("threshold workspace too small: need %zu bytes, got %zu", (size_t)M * 8, ws_bytes);
    return CABS_ENOMEM;
  }
  unsigned long long* key = (unsigned long long*)ws;
  const int blocks = std::max(1, std::min(ceil_div(M, kNormThreads), sm_count() * 8));
  CABS_LAUNCH(stream, "sq_norms_kernel", sq_norms_kernel<T><<<blocks, kNormThreads, 0, stream>>>(X, M, d, key));
  const int top_shift = sizeof(T) == 8 ? 56 : 24;
  CABS_LAUNCH(stream, "select_topk_kernel",
              select_topk_kernel<<<1, kSelThreads, 0, stream>>>(key, M, k2, top_shift, sorted));
  return CABS_OK;
}

template <typename T>
cabs_status leverage_typed(const T* X, int64_t M, int d, int k2, uint64_t seed, int tag, int* sorted, void* ws,
                           size_t ws_bytes, cudaStream_t stream) {
  if (ws_bytes < (size_t)M * sizeof(unsigned long long)) {
    set_error("leverage workspace too small: need %zu bytes, got %zu", (size_t)M * 8, ws_bytes);
    return CABS_ENOMEM;
  }
  unsigned long long* key = (unsigned long long*)ws;
  const int blocks = std::max(1, std::min(ceil_div(M, kNormThreads), sm_count() * 8));
  CABS_LAUNCH(stream, "lev_keys_kernel",
              lev_keys_kernel<T><<<blocks, kNormThreads, 0, stream>>>(X, M, d, seed, tag, key));
  CABS_LAUNCH(stream, "select_topk_kernel",
              select_topk_kernel<<<1, kSelThreads, 0, stream>>>(key, M, k2, 56, sorted));
  return CABS_OK;
}

}  // namespace

cabs_status launch_leverage_select(const void* X, int64_t M, int d, int k2, bool elem_f64, uint64_t seed, int tag,
                                   int* sorted, void* ws, size_t ws_bytes, cudaStream_t stream) {
  if (elem_f64) return leverage_typed<double>((const double*)X, M, d, k2, seed, tag, sorted, ws, ws_bytes, stream);
  return leverage_typed<float>((const float*)X, M, d, k2, seed, tag, sorted, ws, ws_bytes, stream);
}

size_t threshold_ws_bytes(int64_t M) { return align256((size_t)M * sizeof(unsigned long long)); }

cabs_status launch_threshold(const void* X, int64_t M, int d, int k2, int prec, int* sorted, void* ws,
                             size_t ws_bytes, cudaStream_t stream) {
  if (prec == CABS_PREC_FP64)
    return threshold_typed<double>((const double*)X, M, d, k2, sorted, ws, ws_bytes, stream);
  return threshold_typed<float>((const float*)X, M, d, k2, sorted, ws, ws_bytes, stream);
}

}  // namespace cabs
