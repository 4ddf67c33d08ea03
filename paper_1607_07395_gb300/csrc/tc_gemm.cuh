// Persistent warp-specialised tensor-core contraction C = A B^T with a fused
// epilogue (internal header).
//
// Work unit u = (column block cb, row tile rt), ordered column-block-major;
// a CTA takes a contiguous range of units, so its resident B block (BN rows
// of B, all of K) changes rarely. Roles inside a CTA:
//   warp 0 lane 0  producer: TMA loads of the resident B block (when cb
//                  changes) and of A row tiles (128 rows x one 128-byte K
//                  chunk per stage) into a kStages-deep ring;
//   warp 1 lane 0  MMA issuer: for each unit, 4 MMAs per K chunk
//                  (M = 128, N = BN, K = 32 bytes each) into one of two TMEM
//                  accumulators, commits to free ring stages and to hand the
//                  accumulator to the epilogue;
//   warp 2         allocates / frees TMEM;
//   warps 4..11    epilogue (kernel-specific): lane = TMEM lane = tile row,
//                  warps w and w + 4 split the BN columns in halves.
// All waits are bounded (tc::mbar_wait); on a timeout every role leaves its
// loop, the CTA records an error and frees its TMEM.
#pragma once

#include "tc_common.cuh"

namespace cabs {
namespace tc {

constexpr int kBM = 128;
constexpr int kStages = 4;
constexpr int kThreads = 384;
constexpr int kEpiWarp0 = 4;
constexpr int kEpiWarps = 8;

struct alignas(8) Barriers {
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t bfull;
  uint64_t bempty;
  uint64_t accfull[2];
  uint64_t accempty[2];
  uint32_t tmem_base;
  int abort;
};

// Dynamic shared memory layout: [B resident: nch x BN x 128 B][A ring: kSt x 128 x 128 B]
// (kSt <= kStages ring stages; a kernel may append its own buffers after it).
template <int kSt = kStages>
__host__ __device__ constexpr size_t smem_bytes(int nch, int BN) {
  return (size_t)nch * BN * 128 + (size_t)kSt * kBM * 128 + 1024 /* alignment slack */;
}

__device__ __forceinline__ void unit_of(int u, int MT, int& cb, int& rt) {
  cb = u / MT;
  rt = u - cb * MT;
}

template <int BN, int kSt = kStages>
__device__ __forceinline__ void producer_loop(const CUtensorMap* tmA, const CUtensorMap* tmB, uint8_t* Bres,
                                              uint8_t* Aring, Barriers* bars, int u0, int u1, int MT, int nch,
                                              int kc_elems) {
  volatile int* abort = &bars->abort;
  int cur_cb = -1;
  uint32_t bphase = 0;
  int s = 0;
  uint32_t ph = 0;
  for (int u = u0; u < u1; ++u) {
    int cb, rt;
    unit_of(u, MT, cb, rt);
    if (cb != cur_cb) {
      if (cur_cb >= 0) {
        if (!mbar_wait(&bars->bempty, bphase, abort)) return;
        bphase ^= 1;
      }
      mbar_expect_tx(&bars->bfull, (uint32_t)(nch * BN * 128));
      for (int c = 0; c < nch; ++c) tma_load_2d(Bres + (size_t)c * BN * 128, tmB, &bars->bfull, c * kc_elems, cb * BN);
      cur_cb = cb;
    }
    for (int c = 0; c < nch; ++c) {
      if (!mbar_wait(&bars->empty[s], ph ^ 1, abort)) return;
      mbar_expect_tx(&bars->full[s], (uint32_t)(kBM * 128));
      tma_load_2d(Aring + (size_t)s * kBM * 128, tmA, &bars->full[s], c * kc_elems, rt * kBM);
      if (++s == kSt) {
        s = 0;
        ph ^= 1;
      }
    }
  }
}

template <bool kTF32, int BN, int kSt = kStages>
__device__ __forceinline__ void mma_loop(uint8_t* Bres, uint8_t* Aring, Barriers* bars, int u0, int u1, int MT,
                                         int nch) {
  volatile int* abort = &bars->abort;
  constexpr uint32_t idesc = instr_desc(kTF32, kBM, BN);
  const uint32_t tbase = bars->tmem_base;
  int cur_cb = -1;
  uint32_t bphase = 0;
  int s = 0;
  uint32_t ph = 0;
  int ab = 0;
  uint32_t accph[2] = {0, 0};
  const uint32_t bres = smem_u32(Bres), aring = smem_u32(Aring);
  for (int u = u0; u < u1; ++u) {
    int cb, rt;
    unit_of(u, MT, cb, rt);
    if (cb != cur_cb) {
      if (cur_cb >= 0) mma_commit(&bars->bempty);  // old B block free once its MMAs are done
      if (!mbar_wait(&bars->bfull, bphase, abort)) return;
      bphase ^= 1;
      cur_cb = cb;
    }
    if (!mbar_wait(&bars->accempty[ab], accph[ab] ^ 1, abort)) return;
    fence_after_sync();
    const uint32_t dt = tbase + (uint32_t)(ab * BN);
    for (int c = 0; c < nch; ++c) {
      if (!mbar_wait(&bars->full[s], ph, abort)) return;
      fence_after_sync();
      const uint32_t a0 = aring + (uint32_t)(s * kBM * 128);
      const uint32_t b0 = bres + (uint32_t)(c * BN * 128);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        mma<kTF32>(dt, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), idesc, (c > 0 || kk > 0) ? 1u : 0u);
      mma_commit(&bars->empty[s]);
      if (++s == kSt) {
        s = 0;
        ph ^= 1;
      }
    }
    mma_commit(&bars->accfull[ab]);
    accph[ab] ^= 1;
    ab ^= 1;
  }
}

// Common prologue: carve shared memory, init barriers, allocate 2 x BN TMEM columns.
template <int BN>
__device__ __forceinline__ void setup(uint8_t* smem_raw, int nch, uint8_t*& Bres, uint8_t*& Aring, Barriers* bars) {
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  Bres = base;
  Aring = base + (size_t)nch * BN * 128;
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&bars->full[i], 1);
      mbar_init(&bars->empty[i], 1);
    }
    mbar_init(&bars->bfull, 1);
    mbar_init(&bars->bempty, 1);
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bars->accfull[i], 1);
      mbar_init(&bars->accempty[i], kEpiWarps);
    }
    bars->abort = 0;
    fence_barrier_init();
  }
  if (warp == 2) tmem_alloc(&bars->tmem_base, (uint32_t)(2 * BN));
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
}

template <int BN>
__device__ __forceinline__ void teardown(Barriers* bars, int* err) {
  fence_before_sync();
  __syncthreads();
  if (threadIdx.x == 0 && bars->abort && err) atomicOr(err, 4);
  if ((threadIdx.x >> 5) == 2) {
    fence_after_sync();
    tmem_dealloc(bars->tmem_base, (uint32_t)(2 * BN));
  }
}

}  // namespace tc
}  // namespace cabs
