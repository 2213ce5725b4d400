// Stable LSD radix sort on the record key (the non-oblivious sort of Section 3.3), sm_103a.
//
// Onesweep organisation: one histogram pass gives the counts of all 8-bit digits at once; each
// digit then takes one pass that ranks a tile of records stably per digit (one ballot per digit
// bit + per-warp counters), finds the tile's global offset per digit by decoupled look-back over
// the tiles in ticket order, stages the tile in shared memory in digit order and writes it out
// in runs.
// A digit on which every key agrees is skipped (the pass would be the identity); the buffers
// alternate so that the last pass that runs writes the final output.
#include "common.cuh"
#include "internal.h"
#include "radix_tile.cuh"

namespace bos {

namespace {

constexpr int kHistCtas = 4 * 152;

// Counts of every 8-bit digit of the keys in records [lo, hi), added to a.hist.
template <int R>
__device__ __forceinline__ void radix_hist_body(const RadixArgs& a, uint64_t lo, uint64_t hi, uint64_t step) {
  using Rec = typename RecT<R>::T;
  constexpr int D = RecT<R>::kDigits;
  __shared__ uint32_t h[D][256];
  for (int x = threadIdx.x; x < D * 256; x += kThreads) (&h[0][0])[x] = 0;
  __syncthreads();
  const Rec* in = reinterpret_cast<const Rec*>(a.in);
  for (uint64_t idx = lo + threadIdx.x; idx < hi; idx += step) {
    const auto key = RecT<R>::key(in[idx]);
#pragma unroll
    for (int d = 0; d < D; ++d) atomicAdd(&h[d][(key >> (8 * d)) & 255u], 1u);
  }
  __syncthreads();
  for (int x = threadIdx.x; x < D * 256; x += kThreads) {
    const uint32_t c = (&h[0][0])[x];
    if (c) atomicAdd(a.hist + x, c);
  }
}

template <int R>
__global__ void __launch_bounds__(kThreads) radix_hist_kernel(RadixArgs a) {
  // grid-stride over the whole array: block b handles b*kThreads + j*gridDim*kThreads + tid
  const uint64_t step = (uint64_t)gridDim.x * kThreads;
  radix_hist_body<R>(a, (uint64_t)blockIdx.x * kThreads, a.n, step);
}

// Batched: block b counts chunk b - first[j] (kTile records) of array j.
template <int R>
__global__ void __launch_bounds__(kThreads) radix_hist_batched_kernel(BatchRadix br) {
  __shared__ uint32_t j_s;
  __shared__ unsigned long long c_s;
  if (threadIdx.x == 0) {
    uint32_t lo = 0, hi = br.narr;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (br.first[mid] <= blockIdx.x) lo = mid; else hi = mid;
    }
    j_s = lo;
    c_s = blockIdx.x - br.first[lo];
  }
  __syncthreads();
  const RadixArgs& a = br.args[j_s];
  const uint64_t lo = c_s * kTile, hi = lo + kTile < a.n ? lo + kTile : a.n;
  radix_hist_body<R>(a, lo, hi, kThreads);
}

// Per digit: exclusive offsets of the 256 digit values, and whether the digit is live.
__device__ __forceinline__ void radix_prep_body(const RadixArgs& a, int d) {
  __shared__ uint32_t s[256];
  __shared__ uint32_t any_full;
  const int v = threadIdx.x;
  const uint32_t c = a.hist[d * 256 + v];
  s[v] = c;
  if (v == 0) any_full = 0;
  __syncthreads();
  if ((uint64_t)c == a.n) any_full = 1;
  // inclusive scan (Hillis-Steele)
  for (int o = 1; o < 256; o <<= 1) {
    const uint32_t y = v >= o ? s[v - o] : 0;
    __syncthreads();
    s[v] += y;
    __syncthreads();
  }
  a.dbase[d * 256 + v] = s[v] - c;
  if (v == 0 && !any_full) atomicOr(&a.ctrl->radix_live, 1u << d);
}

template <int R>
__global__ void __launch_bounds__(256) radix_prep_kernel(RadixArgs a) {
  radix_prep_body(a, blockIdx.x);
}

// Batched: block b = (array b / D, digit b % D).
template <int R>
__global__ void __launch_bounds__(256) radix_prep_batched_kernel(BatchRadix br) {
  constexpr int D = RecT<R>::kDigits;
  radix_prep_body(br.args[blockIdx.x / D], blockIdx.x % D);
}

// One tile of one live digit of the LSD chain (the whole CTA).
template <int R>
__device__ __forceinline__ void radix_pass_body(const RadixArgs& a, uint32_t digit, uint64_t tile) {
  using Rec = typename RecT<R>::T;
  const uint32_t live = a.ctrl->radix_live;
  // Buffer chain: X_nlive = buf0 (output); X_j alternates backwards. This pass maps X_c -> X_c+1.
  const uint32_t nlive = __popc(live);
  const uint32_t c = __popc(live & ((1u << digit) - 1));
  auto X = [&](uint32_t j) -> Rec* {
    return reinterpret_cast<Rec*>(((nlive - j) & 1) ? a.buf1 : a.buf0);
  };
  radix_tile<R>(X(c), X(c + 1), a.n, tile, 8 * digit, digit + 1, a.status, a.dbase + digit * 256, a.n, a.ctrl);
}

template <int R>
// Persistent: CTAs take tiles by ticket until none is left (tiles start in ticket order, so every
// look-back waits only on tiles already taken by running CTAs).
__global__ void __launch_bounds__(kThreads, 2) radix_pass_kernel(RadixArgs a, uint32_t digit) {
  __shared__ unsigned long long t_s;
  // a constant digit is skipped; so is every LSD pass when the hybrid sort runs instead
  if (!((a.ctrl->radix_live >> digit) & 1u) || a.ctrl->sort_mode) return;
  const uint64_t tiles = (a.n + kTile - 1) / kTile;
  while (true) {
    if (threadIdx.x == 0) t_s = atomicAdd(&a.ctrl->tickets[a.ticket_base + digit], 1u);
    __syncthreads();
    const unsigned long long t = t_s;
    if (t >= tiles) break;
    radix_pass_body<R>(a, digit, t);
    __syncthreads();
  }
}

// Batched: tickets over all tiles of all arrays; ticket t is tile t - first[j] of array j, so
// inside every array the tiles start in order (the look-back stops at the array's tile 0).
template <int R>
__global__ void __launch_bounds__(kThreads, 2) radix_pass_batched_kernel(BatchRadix br, uint32_t digit) {
  __shared__ unsigned long long t_s;
  __shared__ uint32_t j_s;
  if (threadIdx.x == 0) {
    const uint64_t t = atomicAdd(br.ticket + digit, 1u);
    uint32_t lo = 0, hi = br.narr;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (br.first[mid] <= t) lo = mid; else hi = mid;
    }
    j_s = lo;
    t_s = t - br.first[lo];
  }
  __syncthreads();
  const RadixArgs& a = br.args[j_s];
  if (!((a.ctrl->radix_live >> digit) & 1u)) return;
  radix_pass_body<R>(a, digit, t_s);
}

template <int R>
uint32_t pass_smem() {
  return radix_tile_smem<R>();
}

}  // namespace

uint64_t radix_tiles(uint64_t n, int) { return (n + kTile - 1) / kTile; }

cudaError_t launch_radix_hist(const RadixArgs& a, int R, cudaStream_t st) {
  const uint64_t need = (a.n + kThreads - 1) / kThreads;
  const unsigned grid = (unsigned)(need < (uint64_t)kHistCtas ? (need ? need : 1) : kHistCtas);
  if (R == 8)
    radix_hist_kernel<8><<<grid, kThreads, 0, st>>>(a);
  else
    radix_hist_kernel<16><<<grid, kThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_radix_batched(const BatchRadix& br, int R, int stage, uint32_t digit, cudaStream_t st) {
  if (br.narr == 0) return cudaSuccess;
  if (stage == 0) {  // histograms: one block per chunk of kTile records
    if (br.nblocks == 0) return cudaSuccess;
    if (R == 8)
      radix_hist_batched_kernel<8><<<(unsigned)br.nblocks, kThreads, 0, st>>>(br);
    else
      radix_hist_batched_kernel<16><<<(unsigned)br.nblocks, kThreads, 0, st>>>(br);
  } else if (stage == 1) {  // digit offsets
    if (R == 8)
      radix_prep_batched_kernel<8><<<br.narr * RecT<8>::kDigits, 256, 0, st>>>(br);
    else
      radix_prep_batched_kernel<16><<<br.narr * RecT<16>::kDigits, 256, 0, st>>>(br);
  } else {  // one digit pass over every array's tiles
    if (br.nblocks == 0) return cudaSuccess;
    if (R == 8) {
      const uint32_t sm = pass_smem<8>();
      cudaError_t e = set_smem_optin(radix_pass_batched_kernel<8>);
      if (e != cudaSuccess) return e;
      radix_pass_batched_kernel<8><<<(unsigned)br.nblocks, kThreads, sm, st>>>(br, digit);
    } else {
      const uint32_t sm = pass_smem<16>();
      cudaError_t e = set_smem_optin(radix_pass_batched_kernel<16>);
      if (e != cudaSuccess) return e;
      radix_pass_batched_kernel<16><<<(unsigned)br.nblocks, kThreads, sm, st>>>(br, digit);
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_radix_prep(const RadixArgs& a, int R, cudaStream_t st) {
  if (R == 8)
    radix_prep_kernel<8><<<RecT<8>::kDigits, 256, 0, st>>>(a);
  else
    radix_prep_kernel<16><<<RecT<16>::kDigits, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_radix_pass(const RadixArgs& a, int R, uint32_t digit, cudaStream_t st) {
  const uint64_t tiles = radix_tiles(a.n, R);
  if (tiles == 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaError_t e0 = cudaGetDevice(&dev);
  if (e0 == cudaSuccess) e0 = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e0 != cudaSuccess) return e0;
  const unsigned grid = (unsigned)(tiles < 2ull * sms ? tiles : 2ull * sms);  // two CTAs per SM
  if (R == 8) {
    const uint32_t sm = pass_smem<8>();
    cudaError_t e = set_smem_optin(radix_pass_kernel<8>);
    if (e != cudaSuccess) return e;
    radix_pass_kernel<8><<<grid, kThreads, sm, st>>>(a, digit);
  } else {
    const uint32_t sm = pass_smem<16>();
    cudaError_t e = set_smem_optin(radix_pass_kernel<16>);
    if (e != cudaSuccess) return e;
    radix_pass_kernel<16><<<grid, kThreads, sm, st>>>(a, digit);
  }
  return cudaGetLastError();
}

}  // namespace bos
