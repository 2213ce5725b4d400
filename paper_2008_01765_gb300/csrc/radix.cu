// Stable LSD radix sort on the record key (the non-oblivious sort of Section 3.3), sm_103a.
//
// Onesweep organisation: one histogram pass gives the counts of all 8-bit digits at once; each
// digit then takes one pass that ranks a tile of records stably per digit (warp match + per-warp
// counters), finds the tile's global offset per digit by decoupled look-back over the tiles in
// ticket order, stages the tile in shared memory in digit order and writes it out in runs.
// A digit on which every key agrees is skipped (the pass would be the identity); the buffers
// alternate so that the last pass that runs writes the final output.
#include "common.cuh"
#include "internal.h"

namespace bos {

namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 8;
constexpr uint32_t kTile = kThreads * kItems;
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

// One tile (kTile records) of a stable scatter by one 8-bit digit (the whole CTA).
//   src, n        the records of the segment being sorted (tile t covers [t*kTile, ...))
//   dst, dbase    output: records with digit value v go to dst[dbase[v] + rank among them];
//                 nout bounds the output (a position at or past it is never written)
//   status        the segment's look-back words, 256 per tile, tile 0 first
// Ranking is stable: warp-contiguous positions, lane-striped per item, ranked item by item with
// per-warp counters; a tile's counts are published at once and its global offsets come from the
// decoupled look-back over the preceding tiles of the segment.
template <int R>
__device__ __forceinline__ void radix_tile(const typename RecT<R>::T* src, typename RecT<R>::T* dst, uint64_t n,
                                           uint64_t tile, uint32_t shift, uint32_t tag, unsigned long long* status,
                                           const unsigned long long* dbase, uint64_t nout, Ctrl* ctrl) {
  using Rec = typename RecT<R>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  Rec* stage = reinterpret_cast<Rec*>(smem);                                   // [kTile]
  uint32_t* wcnt = reinterpret_cast<uint32_t*>(smem + kTile * sizeof(Rec));    // [kWarps][257]
  uint32_t* lstart = wcnt + kWarps * 257;                                      // [257]
  uint32_t* half0 = lstart + 257;                                              // [256]
  uint32_t* half1 = half0 + 256;                                               // [256]
  uint32_t* wsum = half1 + 256;                                                // [8]
  unsigned long long* gstart = reinterpret_cast<unsigned long long*>(wsum + 9);  // [256], 8-byte aligned

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int x = tid; x < kWarps * 257; x += kThreads) wcnt[x] = 0;
  __syncthreads();
  const uint64_t t0 = tile * kTile;
  const uint32_t lt_mask = lanemask_lt();

  Rec rc[kItems];
  uint32_t dr[kItems];  // digit (bits 0..8, 256 = none) | rank inside the warp << 9
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    const uint64_t idx = t0 + warp * 32 * kItems + it * 32 + lane;
    dr[it] = 256;
    if (idx < n) {
      rc[it] = src[idx];
      dr[it] = (uint32_t)(RecT<R>::key(rc[it]) >> shift) & 255u;
    }
  }
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    const uint32_t d = dr[it];
    const uint32_t peers = ballot_peers(d, 9);  // 9 bits: 256 = no item
    const uint32_t lt = __popc(peers & lt_mask);
    const uint32_t r = wcnt[warp * 257 + d] + lt;
    __syncwarp();
    if (lt == 0) wcnt[warp * 257 + d] += __popc(peers);
    __syncwarp();
    dr[it] = d | (r << 9);
  }
  __syncthreads();
  // Offsets: thread (h, v) with v = tid & 255 sums digit v over warps 8h..8h+7; the tile count of
  // v is the sum of both halves; an exclusive scan over v gives the tile-local start lstart[v];
  // wcnt[w][v] becomes the tile-local start of warp w's items with digit v.
  const uint32_t v = tid & 255u, h = tid >> 8;
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += wcnt[(h * 8 + j) * 257 + v];
  (h ? half1 : half0)[v] = s;
  __syncthreads();
  const uint32_t below = h ? half0[v] : 0u;  // digit v's items in warps 0..7
  const uint32_t total_v = half0[v] + half1[v];
  uint32_t incl = total_v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += y;
  }
  if (h == 0 && lane == 31) wsum[warp] = incl;
  __syncthreads();
  uint32_t excl = incl - total_v;
  for (int w = 0; w < (warp & 7); ++w) excl += wsum[w];
  if (h == 0) {
    lstart[v] = excl;
    st_status(status + tile * 256 + v, st_word(tile == 0 ? kStIncl : kStAgg, tag, total_v));
    if (v == 255) lstart[256] = excl + total_v;
  }
  {
    uint32_t run = excl + below;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint32_t x = wcnt[(h * 8 + j) * 257 + v];
      wcnt[(h * 8 + j) * 257 + v] = run;
      run += x;
    }
  }
  __syncthreads();
  // stage the tile in digit order (independent of the global prefix)
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    const uint32_t d = dr[it] & 511u;
    if (d < 256) stage[wcnt[warp * 257 + d] + (dr[it] >> 9)] = rc[it];
  }
  // global offset of every digit value: decoupled look-back over the segment's preceding tiles
  if (tid < 256) {
    unsigned long long pre = 0;
    if (tile > 0) {
      pre = lookback_window<8>(status + tid, tile, 256, tag, ctrl);
      st_status(status + tile * 256 + tid, st_word(kStIncl, tag, pre + total_v));
    }
    gstart[tid] = dbase[tid] + pre - lstart[tid];  // output index of stage[j] with digit v: gstart[v] + j
  }
  __syncthreads();
  const uint32_t total = lstart[256];
  for (uint32_t j = tid; j < total; j += kThreads) {
    const Rec r = stage[j];
    const uint32_t dv = (uint32_t)(RecT<R>::key(r) >> shift) & 255u;
    const uint64_t pos = gstart[dv] + j;
    if (pos < nout) dst[pos] = r;
  }
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
__global__ void __launch_bounds__(kThreads, 2) radix_pass_kernel(RadixArgs a, uint32_t digit) {
  __shared__ unsigned long long t_s;
  if (!((a.ctrl->radix_live >> digit) & 1u)) return;
  if (threadIdx.x == 0) t_s = atomicAdd(&a.ctrl->tickets[a.ticket_base + digit], 1u);
  __syncthreads();
  radix_pass_body<R>(a, digit, t_s);
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
  using Rec = typename RecT<R>::T;
  return kTile * sizeof(Rec) + (kWarps * 257 + 257 + 512 + 9) * 4 + 256 * 8;
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
  const unsigned grid = (unsigned)radix_tiles(a.n, R);
  if (grid == 0) return cudaSuccess;
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
