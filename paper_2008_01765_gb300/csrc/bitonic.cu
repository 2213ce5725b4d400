// Bitonic sorting network on the GPU (Batcher 1968): the oblivious-sort comparator of Table 1
// (n log^2 n work, 1/4 n log^2 n comparisons). Records are ordered by (key, payload).
//
// Stages whose partner distance j is below the shared-memory block (128 KB of records) run inside
// shared memory, all of them in one launch per merge size. The others run up to four at a time:
// a thread holds the 2^m records of one m-dimensional sub-cube of the index bits j .. j/2^(m-1)
// in registers and applies the m compare-exchange stages there, so one pass over the array does
// m stages (all of its records share the merge direction, set by bit kk above the cube).
#include "common.cuh"
#include "internal.h"

namespace bos {

namespace {

constexpr uint32_t kBlockBytes = 128u << 10;  // shared-memory block: 8192 16-byte records
constexpr int kThreads = 1024;

template <int R>
__device__ __forceinline__ bool rec_less(const typename RecT<R>::T& a, const typename RecT<R>::T& b);
template <>
__device__ __forceinline__ bool rec_less<8>(const uint2& a, const uint2& b) {
  return a.x < b.x || (a.x == b.x && a.y < b.y);
}
template <>
__device__ __forceinline__ bool rec_less<16>(const uint4& a, const uint4& b) {
  const unsigned long long ka = (unsigned long long)a.x | ((unsigned long long)a.y << 32);
  const unsigned long long kb = (unsigned long long)b.x | ((unsigned long long)b.y << 32);
  if (ka != kb) return ka < kb;
  const unsigned long long pa = (unsigned long long)a.z | ((unsigned long long)a.w << 32);
  const unsigned long long pb = (unsigned long long)b.z | ((unsigned long long)b.w << 32);
  return pa < pb;
}

// Sort (kFull) or merge (k given, partner distances < block) one block of `bs` records in
// shared memory. Element i's direction in merge size kk is ascending iff (global i & kk) == 0.
template <int R, bool kFull>
__global__ void __launch_bounds__(kThreads) bitonic_block_kernel(const void* in, void* out, uint32_t bs,
                                                                 uint64_t kmerge) {
  using Rec = typename RecT<R>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  Rec* s = reinterpret_cast<Rec*>(smem);
  const uint64_t base = (uint64_t)blockIdx.x * bs;
  const Rec* src = reinterpret_cast<const Rec*>(in) + base;
  Rec* dst = reinterpret_cast<Rec*>(out) + base;
  for (uint32_t x = threadIdx.x; x < bs; x += kThreads) s[x] = src[x];
  __syncthreads();
  const uint64_t kk_lo = kFull ? 2 : kmerge;
  const uint64_t kk_hi = kFull ? bs : kmerge;
  for (uint64_t kk = kk_lo; kk <= kk_hi; kk <<= 1) {
    for (uint32_t j = (uint32_t)((kk >> 1) < (bs >> 1) ? (kk >> 1) : (bs >> 1)); j > 0; j >>= 1) {
      for (uint32_t p = threadIdx.x; p < bs / 2; p += kThreads) {
        const uint32_t i = 2 * p - (p & (j - 1));  // i has bit j clear
        const uint32_t l = i | j;
        const bool asc = ((base + i) & kk) == 0;
        const Rec a = s[i], b = s[l];
        if (asc ? rec_less<R>(b, a) : rec_less<R>(a, b)) {
          s[i] = b;
          s[l] = a;
        }
      }
      __syncthreads();
    }
  }
  for (uint32_t x = threadIdx.x; x < bs; x += kThreads) dst[x] = s[x];
}

// M = 2^m records per thread: the sub-cube {i0 + c * jlo : c < M}, i0 with the m cube bits clear.
// Stages jj = M/2 .. 1 (times jlo) compare-exchange inside the cube, in registers.
template <int R, int M>
__global__ void __launch_bounds__(256) bitonic_cube_kernel(void* data, uint64_t n, uint64_t kk, uint64_t jlo) {
  using Rec = typename RecT<R>::T;
  Rec* d = reinterpret_cast<Rec*>(data);
  const uint32_t lg = (uint32_t)__ffsll((long long)jlo) - 1;  // jlo is a power of two
  for (uint64_t p = (uint64_t)blockIdx.x * 256 + threadIdx.x; p < n / M; p += (uint64_t)gridDim.x * 256) {
    // insert log2(M) zero bits at bit lg of p
    const uint64_t low = p & (jlo - 1), high = p >> lg;
    const uint64_t i0 = low | (high << (lg + __ffs(M) - 1));
    const bool asc = (i0 & kk) == 0;
    Rec e[M];
#pragma unroll
    for (int c = 0; c < M; ++c) e[c] = d[i0 + (uint64_t)c * jlo];
#pragma unroll
    for (int jj = M / 2; jj > 0; jj >>= 1) {
#pragma unroll
      for (int c = 0; c < M; ++c) {
        if ((c & jj) == 0) {
          const Rec a = e[c], b = e[c | jj];
          if (asc ? rec_less<R>(b, a) : rec_less<R>(a, b)) {
            e[c] = b;
            e[c | jj] = a;
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < M; ++c) d[i0 + (uint64_t)c * jlo] = e[c];
  }
}

template <int R, int M>
cudaError_t launch_cube(void* data, uint64_t n, uint64_t kk, uint64_t jlo, cudaStream_t st) {
  const uint64_t need = (n / M + 255) / 256;
  const unsigned grid = (unsigned)(need < 152ull * 8 ? need : 152ull * 8);
  bitonic_cube_kernel<R, M><<<grid, 256, 0, st>>>(data, n, kk, jlo);
  return cudaGetLastError();
}

template <int R>
cudaError_t run(const void* in, void* out, uint64_t n, cudaStream_t st) {
  using Rec = typename RecT<R>::T;
  const uint32_t kBlock = kBlockBytes / sizeof(Rec);
  const uint32_t bs = (uint32_t)(n < kBlock ? n : kBlock);
  const uint32_t smem = bs * sizeof(Rec);
  cudaError_t e = set_smem_optin(bitonic_block_kernel<R, true>);
  if (e != cudaSuccess) return e;
  e = set_smem_optin(bitonic_block_kernel<R, false>);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)(n / bs);
  bitonic_block_kernel<R, true><<<blocks, kThreads, smem, st>>>(in, out, bs, 0);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (uint64_t kk = 2ull * bs; kk <= n; kk <<= 1) {
    // stages j = kk/2 .. bs, up to four per pass
    for (uint64_t j = kk >> 1; j >= bs;) {
      uint32_t m = 0;
      while (m < 4 && (j >> m) >= bs) ++m;
      const uint64_t jlo = j >> (m - 1);
      switch (m) {
        case 4: e = launch_cube<R, 16>(out, n, kk, jlo, st); break;
        case 3: e = launch_cube<R, 8>(out, n, kk, jlo, st); break;
        case 2: e = launch_cube<R, 4>(out, n, kk, jlo, st); break;
        default: e = launch_cube<R, 2>(out, n, kk, jlo, st); break;
      }
      if (e != cudaSuccess) return e;
      j = jlo >> 1;
    }
    bitonic_block_kernel<R, false><<<blocks, kThreads, smem, st>>>(out, out, bs, kk);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_bitonic(const void* in, void* out, uint64_t n, int R, cudaStream_t st) {
  if (n <= 1) {
    if (n == 1) return cudaMemcpyAsync(out, in, R, cudaMemcpyDeviceToDevice, st);
    return cudaSuccess;
  }
  return R == 8 ? run<8>(in, out, n, st) : run<16>(in, out, n, st);
}

}  // namespace bos
