// Step a5 on tensor cores -- the k-means assignment of Eq. (wkmeans) for the
// BF16 and TF32 modes.
//
// The distance contraction x . z for all points x (rows of P or Q) and all
// k2 <= 256 centres z is one tcgen05 MMA chain per 128-point tile: points
// stream through a TMA ring, the centres stay resident in shared memory, and
// a 128 x 256 FP32 accumulator sits in TMEM (two of them, so the epilogue of
// one tile overlaps the MMAs of the next). 256 TF32 centres of width above
// 128 do not fit in shared memory: there the centres form two column blocks
// of 128, each unit (row tile, block) keeps its block's two best per row,
// and a per-row pass merges the blocks in order.
// Epilogue warps read a row of accumulators per thread and form
// |z|^2 - 2 x . z, keeping the best and second-best centre; warps holding
// the two column halves of a row merge through shared memory. When the two
// best are closer than the rounding bound of the operands
// (1.25 * 4u |x| (|z_a| + |z_b|); u = 2^-8 for BF16, which keeps 8 significant
// bits and rounds to nearest, and 2^-10 for TF32, whose 11 significant bits
// the tensor core may take by truncation), the
// row is flagged and a separate coalesced pass recomputes both distances in
// FP32 by direct differences; the smaller wins (ties to the lower index). The weighted encoding error is computed afterwards by
// a separate pass with direct differences (k-means kernel file).
#include <cuda_bf16.h>

#include "kernels.cuh"
#include "profile.cuh"
#include "tc_assign.cuh"
#include "tc_gemm.cuh"

namespace cabs {
namespace {

constexpr int kBN = 256;

template <bool kTF32>
struct AsgCfg {
  static constexpr int KC = kTF32 ? 32 : 64;
  static constexpr int ES = kTF32 ? 4 : 2;
};

template <bool kTF32>
// Eight consecutive operand entries of one row per thread (Kp is a multiple
// of 32, so a group never straddles rows): two 16-byte loads when d is a
// multiple of 4 and the group lies inside the row, and one 16-byte (BF16) or
// two (TF32) stores; entries at or beyond d are zero.
__global__ void to_operand_kernel(const float* __restrict__ X, long long rows, int d, int Kp, void* __restrict__ out) {
  const long long groups = rows * (Kp / 8);
  const bool vec = (d & 3) == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0;
  for (long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x; gi < groups;
       gi += (long long)gridDim.x * blockDim.x) {
    const long long e0 = gi * 8;
    const long long r = e0 / Kp;
    const int q0 = (int)(e0 - r * Kp);
    const float* src = X + r * d + q0;
    float v[8];
    if (vec && q0 + 8 <= d) {
      const float4 a = *reinterpret_cast<const float4*>(src);
      const float4 b = *reinterpret_cast<const float4*>(src + 4);
      v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
      v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i) v[i] = q0 + i < d ? src[i] : 0.f;
    }
    if constexpr (kTF32) {
      float4* o = reinterpret_cast<float4*>((float*)out + e0);
      o[0] = make_float4(v[0], v[1], v[2], v[3]);
      o[1] = make_float4(v[4], v[5], v[6], v[7]);
    } else {
      __align__(16) __nv_bfloat16 h[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) h[i] = __float2bfloat16_rn(v[i]);
      *reinterpret_cast<uint4*>((__nv_bfloat16*)out + e0) = *reinterpret_cast<const uint4*>(h);
    }
  }
}

struct Best2 {
  float b1, b2;
  int j1, j2;
};

__device__ __forceinline__ void best2_push(Best2& s, float v, int j) {
  if (v < s.b1 || (v == s.b1 && j < s.j1)) {
    s.b2 = s.b1;
    s.j2 = s.j1;
    s.b1 = v;
    s.j1 = j;
  } else if (v < s.b2 || (v == s.b2 && j < s.j2)) {
    s.b2 = v;
    s.j2 = j;
  }
}

// Near-tie bound of the two best distances of a row (see the file comment).
template <bool kTF32>
__device__ __forceinline__ int near_tie_alt(const Best2& s, int k2, float xl, const float* __restrict__ zn) {
  // the difference of two rounded contractions 2 x.z_a - 2 x.z_b is off by at
  // most 4 u |x| (|z_a| + |z_b|) for operand rounding u (2^-8 BF16, 2^-10
  // TF32); a 1.25x margin covers the FP32 accumulation
  constexpr float rel = kTF32 ? 0.0048828125f : 0.01953125f;
  if (s.j2 >= k2) return -1;
  const float bound = rel * sqrtf(fmaxf(xl, 0.f)) * (sqrtf(fmaxf(zn[s.j1], 0.f)) + sqrtf(fmaxf(zn[s.j2], 0.f)));
  return s.b2 - s.b1 <= bound ? s.j2 : -1;
}

// One CTA per SM over units (column block cb, row tile rt), column-block
// major. BN = 256: every centre in one column block, labels written
// directly. BN = 128 (TF32 with d > 128, where 256 resident TF32 centres do
// not fit in shared memory): each unit leaves its block's best and second
// best per row in part[l * ncb + cb], merged by tc_assign_merge_kernel.
template <bool kTF32, int BN>
__global__ void __launch_bounds__(tc::kThreads, 1)
    tc_assign_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     const float* __restrict__ zn, const float* __restrict__ xn, int M, int k2, int nch, int MT,
                     int units, int* __restrict__ labels, int* __restrict__ alt, Best2* __restrict__ part, int ncb,
                     int* err) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ tc::Barriers bars;
  __shared__ Best2 xchg[4][32];
  __shared__ float zn_s[kBN];  // |z_j|^2, +inf past k2 (such columns never win)
  for (int j = threadIdx.x; j < kBN; j += blockDim.x) zn_s[j] = j < k2 ? zn[j] : __int_as_float(0x7f800000);
  uint8_t *Bres, *Aring;
  tc::setup<BN>(smem_raw, nch, Bres, Aring, &bars);  // its __syncthreads publishes zn_s
  const int u0 = (int)((long long)units * blockIdx.x / gridDim.x);
  const int u1 = (int)((long long)units * (blockIdx.x + 1) / gridDim.x);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    if (lane == 0) {
      tc::prefetch_tmap(&tmA);
      tc::prefetch_tmap(&tmB);
      tc::producer_loop<BN>(&tmA, &tmB, Bres, Aring, &bars, u0, u1, MT, nch, AsgCfg<kTF32>::KC);
    }
  } else if (warp == 1) {
    if (lane == 0) tc::mma_loop<kTF32, BN>(Bres, Aring, &bars, u0, u1, MT, nch);
  } else if (warp >= tc::kEpiWarp0) {
    const int e = warp - tc::kEpiWarp0;
    const int sub = warp & 3, half = e >> 2;
    const int row = sub * 32 + lane;
    int ab = 0;
    uint32_t accph[2] = {0, 0};
    for (int u = u0; u < u1; ++u) {
      const int cb = u / MT, rt = u - cb * MT;
      // every epilogue warp must leave together: they share named barrier 1
      const int fail = tc::mbar_wait(&bars.accfull[ab], accph[ab], &bars.abort) ? 0 : 1;
      int anyfail;
      asm volatile(
          "{\n\t.reg .pred p, q;\n\tsetp.ne.s32 q, %1, 0;\n\t"
          "bar.red.or.pred p, 1, %2, q;\n\tselp.s32 %0, 1, 0, p;\n\t}"
          : "=r"(anyfail)
          : "r"(fail), "n"(tc::kEpiWarps * 32));
      if (anyfail) break;
      accph[ab] ^= 1;
      tc::fence_after_sync();
      Best2 s{__int_as_float(0x7f800000), __int_as_float(0x7f800000), 0x7fffffff, 0x7fffffff};
      // this half's columns in groups of 32, the next group loading from
      // TMEM while the current one is scanned; within a thread the centre
      // index only grows, so a strict < keeps the lower index on ties
      constexpr int kGroups = BN / 2 / 32;
      const int c_half = cb * BN + half * (BN / 2);  // first centre of this half
      const int ng = min(kGroups, max(0, (k2 - c_half + 31) / 32));  // warp-uniform
      const uint32_t taddr = bars.tmem_base + (uint32_t)(ab * BN + half * (BN / 2)) + ((uint32_t)(sub * 32) << 16);
      uint32_t r[2][32];
      if (ng > 0) tc::tmem_ld32_issue(taddr, r[0]);
#pragma unroll
      for (int j = 0; j < kGroups; ++j) {
        if (j < ng) {
          tc::tmem_ld_wait(r[j & 1]);
          if (j + 1 < ng) tc::tmem_ld32_issue(taddr + (uint32_t)((j + 1) * 32), r[(j + 1) & 1]);
          const int c0 = c_half + j * 32;
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            const float dv = fmaf(-2.f, __uint_as_float(r[j & 1][q]), zn_s[c0 + q]);
            const bool lt1 = dv < s.b1, lt2 = dv < s.b2;
            s.b2 = lt1 ? s.b1 : (lt2 ? dv : s.b2);
            s.j2 = lt1 ? s.j1 : (lt2 ? c0 + q : s.j2);
            s.b1 = lt1 ? dv : s.b1;
            s.j1 = lt1 ? c0 + q : s.j1;
          }
        }
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bars.accempty[ab]);
      ab ^= 1;
      // merge the two column halves of each row (warps w and w + 4)
      if (half == 1) xchg[sub][lane] = s;
      asm volatile("bar.sync 1, %0;" ::"n"(tc::kEpiWarps * 32));
      if (half == 0) {
        const Best2 o = xchg[sub][lane];
        best2_push(s, o.b1, o.j1);
        best2_push(s, o.b2, o.j2);
        const long long l = (long long)rt * tc::kBM + row;
        if (l < M) {
          if (part) {
            part[l * ncb + cb] = s;
          } else {
            labels[l] = s.j1;
            alt[l] = near_tie_alt<kTF32>(s, k2, xn[l], zn);
          }
        }
      }
      asm volatile("bar.sync 1, %0;" ::"n"(tc::kEpiWarps * 32));
    }
  }
  tc::teardown<BN>(&bars, err);
}

// Per row: the column blocks' best and second best merged in block order
// (ties to the lower centre), then the label and the near-tie flag.
template <bool kTF32>
__global__ void __launch_bounds__(256) tc_assign_merge_kernel(const Best2* __restrict__ part, int ncb, long long M,
                                                              int k2, const float* __restrict__ xn,
                                                              const float* __restrict__ zn, int* __restrict__ labels,
                                                              int* __restrict__ alt) {
  for (long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x; l < M; l += (long long)gridDim.x * blockDim.x) {
    Best2 s = part[l * ncb];
    for (int cb = 1; cb < ncb; ++cb) {
      const Best2 o = part[l * ncb + cb];
      best2_push(s, o.b1, o.j1);
      best2_push(s, o.b2, o.j2);
    }
    labels[l] = s.j1;
    alt[l] = near_tie_alt<kTF32>(s, k2, xn[l], zn);
  }
}

// Rows whose two best centres were closer than the operand rounding bound:
// both distances again in FP32 by direct differences (one warp per row, lanes
// over dimensions, coalesced); the smaller wins, ties to the lower index. A
// CTA covers 256 rows at a time: their flagged rows are gathered into a
// shared list and dealt out to the 8 warps, so that no warp walks many
// flagged rows one after another (each row's decision is independent).
__global__ void __launch_bounds__(256) assign_resolve_kernel(const float* __restrict__ X, long long M, int d,
                                                             const float* __restrict__ Z, int* __restrict__ labels,
                                                             const int* __restrict__ alt, int* rechecks) {
  __shared__ int list[256];
  __shared__ int cnt;
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int nre = 0;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < M; base += (long long)gridDim.x * blockDim.x) {
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    const long long l = base + threadIdx.x;
    if (l < M && alt[l] >= 0) list[atomicAdd(&cnt, 1)] = threadIdx.x;
    __syncthreads();
    const int n = cnt;
    for (int e = wi; e < n; e += nw) {
      const long long r = base + list[e];
      const int j1 = labels[r], j2 = alt[r];
      float s1 = 0.f, s2 = 0.f;
      // unrolled so that a row's loads (d <= 256: 8 per operand) are all in flight at once
#pragma unroll 8
      for (int q = lane; q < d; q += 32) {
        const float x = __ldg(X + r * d + q);
        const float t1 = x - __ldg(Z + (size_t)j1 * d + q);
        const float t2 = x - __ldg(Z + (size_t)j2 * d + q);
        s1 = fmaf(t1, t1, s1);
        s2 = fmaf(t2, t2, s2);
      }
      s1 = warp_sum(s1);
      s2 = warp_sum(s2);
      if (lane == 0) {
        ++nre;
        if (s2 < s1 || (s2 == s1 && j2 < j1)) labels[r] = j2;
      }
    }
    __syncthreads();  // the list is rebuilt for the next 256 rows
  }
  if (lane == 0 && nre && rechecks) atomicAdd(rechecks, nre);
}

struct TcWs {
  void *Pp, *Zp;
  int *alt, *err;
  Best2* part;  // per-row, per-column-block best two (two-block TF32 form)
};

int kp_of(int d, bool tf32) {
  const int KC = tf32 ? 32 : 64;
  return (d + KC - 1) / KC * KC;
}

// Centres per column block: all 256 when their operand block fits in 128 KB
// of shared memory (BF16 up to d = 256, TF32 up to d = 128), else 128. The
// launch shape may also choose 128 (half the MMA columns when k2 <= 128;
// the per-row merge of two blocks keeps the same answer).
int block_n(int d, bool tf32) { return (size_t)kp_of(d, tf32) / (tf32 ? 32 : 64) * kBN * 128 > 128 * 1024 ? 128 : kBN; }

TcWs carve_tc(Carve& cv, int64_t M, int d, int k2, bool tf32) {
  const int Kp = kp_of(d, tf32);
  const int es = tf32 ? 4 : 2;
  TcWs w;
  w.Pp = cv.take<char>((size_t)M * Kp * es);
  w.Zp = cv.take<char>((size_t)kBN * Kp * es);
  w.alt = cv.take<int>(M);
  w.err = cv.take<int>(1);
  w.part = cv.take<Best2>((size_t)M * (kBN / 128));
  return w;
}

template <bool kTF32, int BN>
cabs_status launch_assign(const CUtensorMap& tmA, const CUtensorMap& tmB, const float* zn, const float* xn, int64_t M,
                          int k2, int nch, int* labels, TcWs& t, cudaStream_t stream) {
  const int MT = ceil_div(M, tc::kBM);
  const int ncb = ceil_div(k2, BN);
  const int units = MT * ncb;
  const int grid = std::max(1, std::min(units, sm_count()));
  const size_t smem = tc::smem_bytes(nch, BN);
  cudaFuncSetAttribute(tc_assign_kernel<kTF32, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  Best2* part = BN == kBN ? nullptr : t.part;
  CABS_LAUNCH(stream, "tc_assign_kernel",
              (tc_assign_kernel<kTF32, BN><<<grid, tc::kThreads, smem, stream>>>(
                  tmA, tmB, zn, xn, (int)M, k2, nch, MT, units, labels, t.alt, part, ncb, t.err)));
  if (part)
    CABS_LAUNCH(stream, "tc_assign_merge_kernel",
                tc_assign_merge_kernel<kTF32><<<std::max(1, std::min(ceil_div(M, 256), sm_count() * 4)), 256, 0,
                                                stream>>>(part, ncb, M, k2, xn, zn, labels, t.alt));
  return CABS_OK;
}

template <bool kTF32>
cabs_status tc_assign_typed(const float* X, int64_t M, int d, const float* Z, const float* zn, int k2, const float* xn,
                            const float* w, int* labels, int* d_recheck, bool prep_points, void* tcws,
                            cudaStream_t stream) {
  (void)w;
  Carve cv(tcws, (size_t)-1);
  TcWs t = carve_tc(cv, M, d, k2, kTF32);
  const int Kp = kp_of(d, kTF32);
  const int nch = Kp / AsgCfg<kTF32>::KC;
  // 128 where 256 resident centres do not fit, else the launch shape's choice
  const int BN = block_n(d, kTF32) == 128 || current_tune().assign_bn == 128 ? 128 : kBN;
  const int sms = sm_count();
  if (prep_points)
    CABS_LAUNCH(stream, "tc_assign_points_prep",
                to_operand_kernel<kTF32><<<std::max(1, std::min(ceil_div(M * Kp / 8, 256), sms * 8)), 256, 0, stream>>>(
                    X, M, d, Kp, t.Pp));
  CABS_LAUNCH(stream, "tc_assign_centres_prep",
              to_operand_kernel<kTF32><<<std::max(1, ceil_div((int64_t)kBN * Kp / 8, 256)), 256, 0, stream>>>(
                  Z, k2, d, Kp, t.Zp));
  if (cudaMemsetAsync(t.err, 0, sizeof(int), stream) != cudaSuccess) return check_cuda("tc_assign err clear");
  CUtensorMap tmA, tmB;
  const int dt = kTF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  CABS_TRY(make_tmap_2d(&tmA, t.Pp, dt, M, Kp, (uint64_t)Kp * AsgCfg<kTF32>::ES, AsgCfg<kTF32>::KC, tc::kBM));
  // rows of a block's box at or beyond k2 lie outside the map and load as zeros
  CABS_TRY(make_tmap_2d(&tmB, t.Zp, dt, k2, Kp, (uint64_t)Kp * AsgCfg<kTF32>::ES, AsgCfg<kTF32>::KC, BN));
  if (BN == kBN)
    CABS_TRY((launch_assign<kTF32, kBN>(tmA, tmB, zn, xn, M, k2, nch, labels, t, stream)));
  else
    CABS_TRY((launch_assign<kTF32, 128>(tmA, tmB, zn, xn, M, k2, nch, labels, t, stream)));
  CABS_LAUNCH(stream, "assign_resolve_kernel",
              assign_resolve_kernel<<<std::max(1, std::min(ceil_div(M, 256), sms * 8)), 256, 0, stream>>>(
                  X, M, d, Z, labels, t.alt, d_recheck));
  return CABS_OK;
}

}  // namespace

int tc_kp_of(int d, bool tf32) { return kp_of(d, tf32); }

cabs_status tc_to_operand(const float* X, int64_t rows, int d, int Kp, bool tf32, void* out, const char* name,
                          cudaStream_t stream) {
  const int blocks = std::max(1, std::min(ceil_div(rows * Kp / 8, 256), sm_count() * 8));
  if (tf32)
    CABS_LAUNCH(stream, name, to_operand_kernel<true><<<blocks, 256, 0, stream>>>(X, rows, d, Kp, out));
  else
    CABS_LAUNCH(stream, name, to_operand_kernel<false><<<blocks, 256, 0, stream>>>(X, rows, d, Kp, out));
  return CABS_OK;
}

int tc_assign_blocks(int64_t M) { return std::max(1, std::min(ceil_div(M, tc::kBM), sm_count())); }

void tc_assign_carve(Carve& cv, int64_t M, int d, int k2) {
  // sized for the wider (TF32) operands so either mode fits
  carve_tc(cv, M, d, k2, true);
}

cabs_status tc_assign_launch(const float* X, int64_t M, int d, const float* Z, const float* zn, int k2,
                             const float* xn, const float* w, int* labels, int* d_recheck, bool bf16,
                             bool prep_points, void* tcws, cudaStream_t stream) {
  if (bf16) return tc_assign_typed<false>(X, M, d, Z, zn, k2, xn, w, labels, d_recheck, prep_points, tcws, stream);
  return tc_assign_typed<true>(X, M, d, Z, zn, k2, xn, w, labels, d_recheck, prep_points, tcws, stream);
}

}  // namespace cabs
