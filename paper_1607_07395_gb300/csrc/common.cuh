// Shared helpers of libcabs: status plumbing, the Philox4x64-10 counter-based
// generator, small device utilities. Internal header (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <algorithm>

#include "cabs.h"

namespace cabs {

// ---------------------------------------------------------------- status

// Records a message for the calling thread (read back by cabs_last_error).
void set_error(const char* fmt, ...);
void clear_error();
const char* last_error();

// Converts a pending CUDA error (launch or asynchronous) into CABS_ECUDA.
cabs_status check_cuda(const char* what);

#define CABS_TRY(expr)                        \
  do {                                        \
    cabs_status _s = (expr);                  \
    if (_s != CABS_OK) return _s;             \
  } while (0)

#define CABS_REQUIRE(cond, ...)               \
  do {                                        \
    if (!(cond)) {                            \
      ::cabs::set_error(__VA_ARGS__);         \
      return CABS_EINVAL;                     \
    }                                         \
  } while (0)

#define CABS_LAUNCHED(what) CABS_TRY(::cabs::check_cuda(what))

// ------------------------------------------------------------- workspace

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Carves 256-byte-aligned slices off a caller-provided device buffer.
struct Carve {
  char* base;
  size_t used;
  size_t cap;
  explicit Carve(void* p = nullptr, size_t c = 0) : base((char*)p), used(0), cap(c) {}
  template <typename T>
  T* take(size_t count) {
    size_t bytes = align256(count * sizeof(T));
    T* out = base ? (T*)(base + used) : nullptr;
    used += bytes;
    return out;
  }
  bool fits() const { return used <= cap; }
};

// ----------------------------------------------------------------- Philox
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds, each two
// 64x64->128-bit products of counter words 0 and 2 with fixed multipliers;
// the key is bumped by two Weyl constants between rounds.

constexpr uint64_t kPhiloxM0 = 0xD2E7470EE14C6C93ull;
constexpr uint64_t kPhiloxM1 = 0xCA5A826395121157ull;
constexpr uint64_t kPhiloxW0 = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kPhiloxW1 = 0xBB67AE8584CAA73Bull;

__host__ __device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * (unsigned __int128)b) >> 64);
#endif
}

struct U64x4 {
  uint64_t v[4];
};

__host__ __device__ __forceinline__ U64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                                        uint64_t k0, uint64_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t hi0 = mulhi64(kPhiloxM0, c0), lo0 = kPhiloxM0 * c0;
    const uint64_t hi1 = mulhi64(kPhiloxM1, c2), lo1 = kPhiloxM1 * c2;
    const uint64_t n0 = hi1 ^ c1 ^ k0;
    const uint64_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
  U64x4 o;
  o.v[0] = c0;
  o.v[1] = c1;
  o.v[2] = c2;
  o.v[3] = c3;
  return o;
}

// ------------------------------------------------------------ CSR sources

// Position of column j in the sorted col_idx[lo, hi), or -1.
__device__ __forceinline__ long long csr_find(const int* __restrict__ col_idx, long long lo, long long hi, int j) {
  while (lo < hi) {
    const long long mid = (lo + hi) >> 1;
    const int c = col_idx[mid];
    if (c == j) return mid;
    if (c < j) lo = mid + 1;
    else hi = mid;
  }
  return -1;
}

// The stored range [lo, hi) of row i, clamped to [0, nnz].
__device__ __forceinline__ void csr_row_range(const long long* __restrict__ row_ptr, long long nnz, long long i,
                                              long long& lo, long long& hi) {
  lo = min(max(row_ptr[i], 0ll), nnz);
  hi = min(max(row_ptr[i + 1], lo), nnz);
}

// ------------------------------------------------------------ elem types

template <typename T>
struct ElemOf;
inline bool prec_is_f64(int prec) { return prec == CABS_PREC_FP64; }
inline size_t elem_bytes(int prec) { return prec_is_f64(prec) ? 8 : 4; }

template <typename T>
__device__ __forceinline__ T dev_exp(T x);
template <>
__device__ __forceinline__ float dev_exp<float>(float x) { return expf(x); }
template <>
__device__ __forceinline__ double dev_exp<double>(double x) { return exp(x); }

template <typename T>
__device__ __forceinline__ T dev_sqrt(T x);
template <>
__device__ __forceinline__ float dev_sqrt<float>(float x) { return sqrtf(x); }
template <>
__device__ __forceinline__ double dev_sqrt<double>(double x) { return sqrt(x); }

template <typename T>
__device__ __forceinline__ T pos_inf();
template <>
__device__ __forceinline__ float pos_inf<float>() { return __int_as_float(0x7f800000); }
template <>
__device__ __forceinline__ double pos_inf<double>() { return __longlong_as_double(0x7ff0000000000000ll); }

// Lexicographic (value, index) minimum: ties go to the lower index.
template <typename T>
__device__ __forceinline__ bool lex_less(T a, int ia, T b, int ib) {
  return a < b || (a == b && ia < ib);
}

template <typename T>
__device__ __forceinline__ void warp_argmin(T& v, int& idx) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    T ov = __shfl_xor_sync(0xffffffffu, v, off);
    int oi = __shfl_xor_sync(0xffffffffu, idx, off);
    if (lex_less(ov, oi, v, idx)) {
      v = ov;
      idx = oi;
    }
  }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, off));
  return v;
}

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Number of SMs of the current device (cached per device).
int sm_count();

// Largest grid for a kernel whose CTAs wait on one another (a cooperative
// launch with a grid barrier). Alone, such a kernel may fill the GPU; while
// `sharers` sketches run concurrently (batched lanes, serving slots), its CTAs
// would otherwise sit at the barrier holding SMs until the other sketches'
// kernels drain, so the grid is divided among the sharers. The work split
// does not change any result.
int coop_grid_cap(int full);
struct SharersScope {
  explicit SharersScope(int sharers);
  ~SharersScope();
  int prev;
};

// Launch shapes of the tunable kernels for the sketch being enqueued on the
// calling thread (cabs_tune of the ABI, 0 = the kernel's default). The ABI
// layer looks up the shape bucket of each sketch in its context's table and
// holds a TuneScope while it enqueues that sketch. No choice here changes a
// result: only which thread computes which output.
const cabs_tune& current_tune();
struct TuneScope {
  explicit TuneScope(const cabs_tune& t);
  ~TuneScope();
  cabs_tune prev;
};

}  // namespace cabs
