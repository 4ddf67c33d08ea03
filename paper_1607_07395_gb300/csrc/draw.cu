// Step a1 -- pilot sampling of k distinct rows or columns (Algorithm 2, step 1).
//
// The paper only says the pilot rows and columns are drawn at random; here a
// draw is a partial Fisher-Yates shuffle of a virtual identity array
// a[0..N): step i swaps a[i] and a[j], j = i + hi64(r_i * (N - i)), where r_i
// is word 0 of Philox4x64-10 at counter (i, 0, 0, 0) under key (seed, tag).
// a[0..k) in draw order and sorted ascending are returned.
//
// One CTA per draw. All k random words come from Philox in parallel; the k
// swaps are inherently sequential and run on one thread against an
// open-addressing hash map in shared memory that holds only the positions
// that were touched (at most 2k of them); the sort is a bitonic network over
// all threads.
#include "common.cuh"
#include "kernels.cuh"
#include "profile.cuh"

namespace cabs {
namespace {

constexpr int kDrawThreads = 256;
constexpr int kEmpty = -1;

__host__ __device__ inline int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

__device__ __forceinline__ unsigned hash_pos(int pos, unsigned mask) {
  return ((unsigned)pos * 2654435761u) & mask;
}

// Returns the slot holding `pos`, or the empty slot where it would go.
__device__ __forceinline__ unsigned probe(const int* keys, int pos, unsigned mask) {
  unsigned h = hash_pos(pos, mask);
  while (keys[h] != kEmpty && keys[h] != pos) h = (h + 1) & mask;
  return h;
}

struct DrawJob {
  uint64_t seed;
  int tag;
  int k;
  long long N;
  int* drawn;
  int* sorted;
};

__global__ void __launch_bounds__(kDrawThreads) draw_kernel(DrawJob j0, DrawJob j1) {
  const DrawJob job = blockIdx.x == 0 ? j0 : j1;
  const int k = job.k;
  if (k <= 0) return;
  const int H = next_pow2(4 * k);  // hash capacity: >= 2x the at most 2k live keys
  const int P = next_pow2(k);      // sort width
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* r = (uint64_t*)smem;
  int* keys = (int*)(r + k);
  int* vals = keys + H;
  int* srt = vals + H;

  for (int i = threadIdx.x; i < k; i += blockDim.x)
    r[i] = philox4x64_10((uint64_t)i, 0, 0, 0, job.seed, (uint64_t)job.tag).v[0];
  for (int h = threadIdx.x; h < H; h += blockDim.x) keys[h] = kEmpty;
  __syncthreads();

  if (threadIdx.x == 0) {
    const unsigned mask = (unsigned)H - 1u;
    for (int i = 0; i < k; ++i) {
      const long long span = job.N - i;
      const int j = i + (int)mulhi64(r[i], (uint64_t)span);
      const unsigned si = probe(keys, i, mask);
      const int vi = keys[si] == kEmpty ? i : vals[si];
      const unsigned sj = probe(keys, j, mask);
      const int vj = keys[sj] == kEmpty ? j : vals[sj];
      // position j now holds a[i]; position i is final and never read again
      keys[sj] = j;
      vals[sj] = vi;
      job.drawn[i] = vj;
      srt[i] = vj;
    }
  }
  __syncthreads();
  for (int i = k + threadIdx.x; i < P; i += blockDim.x) srt[i] = 0x7fffffff;
  __syncthreads();
  // bitonic sort, ascending
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < P; t += blockDim.x) {
        const int partner = t ^ stride;
        if (partner > t) {
          const bool up = (t & size) == 0;
          const int a = srt[t], b = srt[partner];
          if ((a > b) == up) {
            srt[t] = b;
            srt[partner] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < k; i += blockDim.x) job.sorted[i] = srt[i];
}

size_t draw_smem(int k) {
  if (k <= 0) return 0;
  const int H = next_pow2(4 * k), P = next_pow2(k);
  return (size_t)k * 8 + (size_t)H * 8 + (size_t)P * 4;
}

}  // namespace

cabs_status launch_draw2(uint64_t seed, int tag0, long long N0, int k0, int* drawn0, int* sorted0, int tag1,
                         long long N1, int k1, int* drawn1, int* sorted1, cudaStream_t stream) {
  DrawJob a{seed, tag0, k0, N0, drawn0, sorted0};
  DrawJob b{seed, tag1, k1, N1, drawn1, sorted1};
  const int jobs = k1 > 0 ? 2 : 1;
  size_t smem = draw_smem(k0);
  if (jobs == 2 && draw_smem(k1) > smem) smem = draw_smem(k1);
  if (smem > 48 * 1024) {
    cudaFuncSetAttribute(draw_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  CABS_LAUNCH(stream, "draw_kernel", draw_kernel<<<jobs, kDrawThreads, smem, stream>>>(a, b));
  return CABS_OK;
}

}  // namespace cabs
