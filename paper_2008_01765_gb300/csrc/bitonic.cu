// Bitonic sorting network on the GPU (Batcher 1968): the oblivious-sort comparator of Table 1
// (n log^2 n work, 1/4 n log^2 n comparisons). Records are ordered by (key, payload).
//
// Stages whose partner distance j is below the shared-memory block (4096 records) run inside
// shared memory, all of them in one launch per merge size; the others are one global
// compare-exchange launch each.
#include "common.cuh"
#include "internal.h"

namespace bos {

namespace {

constexpr uint32_t kBlock = 4096;
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

template <int R>
__global__ void __launch_bounds__(256) bitonic_global_kernel(void* data, uint64_t n, uint64_t kk, uint64_t j) {
  using Rec = typename RecT<R>::T;
  Rec* d = reinterpret_cast<Rec*>(data);
  for (uint64_t p = (uint64_t)blockIdx.x * 256 + threadIdx.x; p < n / 2; p += (uint64_t)gridDim.x * 256) {
    const uint64_t i = 2 * p - (p & (j - 1));
    const uint64_t l = i | j;
    const bool asc = (i & kk) == 0;
    const Rec a = d[i], b = d[l];
    if (asc ? rec_less<R>(b, a) : rec_less<R>(a, b)) {
      d[i] = b;
      d[l] = a;
    }
  }
}

template <int R>
cudaError_t run(const void* in, void* out, uint64_t n, cudaStream_t st) {
  using Rec = typename RecT<R>::T;
  const uint32_t bs = (uint32_t)(n < kBlock ? n : kBlock);
  const uint32_t smem = bs * sizeof(Rec);
  cudaError_t e = set_smem_optin(bitonic_block_kernel<R, true>);
  if (e != cudaSuccess) return e;
  e = set_smem_optin(bitonic_block_kernel<R, false>);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)(n / bs);
  bitonic_block_kernel<R, true><<<blocks, kThreads, smem, st>>>(in, out, bs, 0);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const uint64_t pairs = n / 2;
  const uint64_t gneed = (pairs + 255) / 256;
  const unsigned ggrid = (unsigned)(gneed < 152ull * 16 ? gneed : 152ull * 16);
  for (uint64_t kk = 2ull * bs; kk <= n; kk <<= 1) {
    for (uint64_t j = kk >> 1; j >= bs; j >>= 1) {
      bitonic_global_kernel<R><<<ggrid, 256, 0, st>>>(out, n, kk, j);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
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
