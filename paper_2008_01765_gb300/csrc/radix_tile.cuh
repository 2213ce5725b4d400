// One tile of a stable scatter by one 8-bit digit (onesweep organisation), shared by the LSD
// radix sort (radix.cu) and the MSD partition passes of the hybrid sort (sort_hybrid.cu).
#pragma once
#include "common.cuh"

namespace bos {
namespace rtile {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 8;
constexpr uint32_t kTile = kThreads * kItems;

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
  const bool full = t0 + kTile <= n;  // every item present: eight ballots decide a digit
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    const uint32_t d = dr[it];
    const uint32_t peers = full ? ballot_peers(d, 8) : ballot_peers(d, 9);  // 9 bits: 256 = no item
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

template <int R>
inline uint32_t radix_tile_smem() {
  using Rec = typename RecT<R>::T;
  return kTile * sizeof(Rec) + (kWarps * 257 + 257 + 512 + 9) * 4 + 256 * 8;
}

}  // namespace rtile
using namespace rtile;
}  // namespace bos
