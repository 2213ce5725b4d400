// In-bin permutation table of the fused LAST pass (Section 3.2), sm_103a.
//
// Final bucket b ends the butterfly with its m reals at slots 0..m-1 in stable order. Slot s has
// the key r(b, s) = (w0 << 32 | w1) of Philox(b*Z + s, attempt, stream 1), and the reals leave
// the bucket ordered by (r, s). The keys depend on neither the data nor the routing, so this
// kernel sorts each final bucket's slots by (r, s) ahead of the LAST pass, at full occupancy,
// and the LAST pass (one CTA per SM, bound by its routing) only filters its rows.
//
// Row b of the table lists slots in key order, Z entries of u16. The LAST pass keeps the entries
// below m; dropping the others keeps their relative order, so either of two rows serves:
//   * reals only (the pass has input tags): the kernel reads the LAST pass's input tags, counts
//     m for each final bucket exactly as the LAST pass will (the label digit of every real),
//     sorts slots 0..m-1 and pads the row with 0xFFFF;
//   * all slots (a single pass that draws the labels itself): slots 0..Z-1 sorted.
// A bucket's slots are sorted by the top 9 bits of w0 (counts, exclusive scan, placement), then
// each bin's few slots are put in (w0, w1, s) order in place by one thread.
#include "common.cuh"
#include "internal.h"

namespace bos {

namespace {

constexpr int kPT = 256;      // threads per CTA
constexpr int kPBins = 512;  // bins: top 9 bits of w0
constexpr int kShift = 23;
constexpr int kPer = kPBins / kPT;  // bins per thread in the scan
constexpr uint32_t kMaxK = 12;      // final buckets per LAST subproblem: at most 2^12

// Slot s3 sorts before slot s2 (same bucket, base = b*Z, equal w0): smaller w1, or equal w1 and
// s3 < s2. Rare (equal 32-bit words), so out of line.
__device__ __noinline__ bool tie_less(uint64_t base, uint32_t s3, uint32_t s2, uint32_t attempt, uint64_t seed) {
  const uint32_t l2 = philox_at(base + s2, attempt, 1, seed).w1;
  const uint32_t l3 = philox_at(base + s3, attempt, 1, seed).w1;
  return (l3 < l2) || (l3 == l2 && s3 < s2);
}

uint32_t table_smem(uint32_t Z, uint32_t D) { return Z * 4 + kPBins * 4 + Z * 2 + (16 + D) * 4; }

template <bool TRACE>
__global__ void __launch_bounds__(kPT) perm_table_kernel(PermTableArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t Z = a.Z;
  uint32_t* key = reinterpret_cast<uint32_t*>(smem);                 // [Z] w0 of each slot
  uint32_t* cur = key + Z;                                           // [kPBins]
  uint16_t* mem = reinterpret_cast<uint16_t*>(cur + kPBins);         // [Z] slots by bin, then in key order
  uint32_t* wsum = reinterpret_cast<uint32_t*>(mem + Z);             // [8]
  uint32_t* mcnt = wsum + 16;                                        // [D] reals per final bucket
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lt_mask = lanemask_lt();

  // unit = a LAST subproblem (D final buckets) with tags, one bucket without
  const bool tagged = a.tag != nullptr;
  const uint32_t D = tagged ? 1u << a.k : 1u;
  const uint64_t units = tagged ? a.B >> a.k : a.B;
  const uint32_t shift = a.L - a.i - a.k;  // the LAST pass's routing digit: label bits [shift, shift+k)

  for (uint64_t q = blockIdx.x; q < units; q += gridDim.x) {
    if (tagged) {
      // m of each final bucket q*D + u: the reals of input buckets s*2^i + t (s < D, q = G*2^i + t)
      // whose digit is u, as the LAST pass counts them (capped at Z there as here)
      for (uint32_t x = tid; x < D; x += kPT) mcnt[x] = 0;
      __syncthreads();
      const uint64_t t = q & ((1ull << a.i) - 1), G = q >> a.i;
      for (uint32_t s = 0; s < D; ++s) {
        const uint64_t gb = (G << (a.i + a.k)) + ((uint64_t)s << a.i) + t;
        if (tid == 0) trace_log<TRACE>(a.trace, kRead, a.buf_tag, Z * 4, gb * Z * 4);
        for (uint32_t sl = tid; sl < Z; sl += kPT) {  // Z is a multiple of 32: whole warps
          const uint32_t tg = a.tag[gb * Z + sl];
          const bool real = tg != kDummy;
          const uint32_t u = real ? (tg >> shift) & (D - 1) : D;
          const uint32_t peers = __match_any_sync(0xFFFFFFFFu, u);
          if (real && (peers & lt_mask) == 0) atomicAdd(&mcnt[u], (uint32_t)__popc(peers));
        }
      }
      __syncthreads();
    }
    for (uint32_t u = 0; u < D; ++u) {
      const uint64_t b = q * D + u, base = b * Z;
      const uint32_t m = tagged ? min(mcnt[u], Z) : Z;
      for (int x = tid; x < kPBins; x += kPT) cur[x] = 0;
      __syncthreads();
      for (uint32_t s0 = tid; s0 < m; s0 += 4 * kPT) {  // up to four independent Philox chains per step
        uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (s0 + c * kPT < m) w[c] = philox_at(base + s0 + c * kPT, a.attempt, 1, a.seed).w0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const uint32_t s = s0 + c * kPT;
          if (s < m) {
            key[s] = w[c];
            atomicAdd(&cur[w[c] >> kShift], 1u);
          }
        }
      }
      __syncthreads();
      {  // exclusive scan of the bin counts: kPer consecutive bins per thread
        uint32_t v[kPer], sum = 0;
#pragma unroll
        for (int e = 0; e < kPer; ++e) {
          v[e] = cur[tid * kPer + e];
          sum += v[e];
        }
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
          if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        uint32_t run = incl - sum;
        for (int w2 = 0; w2 < warp; ++w2) run += wsum[w2];
#pragma unroll
        for (int e = 0; e < kPer; ++e) {
          cur[tid * kPer + e] = run;
          run += v[e];
        }
      }
      __syncthreads();
      for (uint32_t s = tid; s < m; s += kPT) mem[atomicAdd(&cur[key[s] >> kShift], 1u)] = (uint16_t)s;
      for (uint32_t s = m + tid; s < Z; s += kPT) mem[s] = 0xFFFFu;  // no real at these ranks
      __syncthreads();
      // cur[bin] is now the end of the bin and a bin starts where the previous one ends; each
      // bin's few members are put in (w0, w1, s) order in place by one thread (insertion sort)
      for (uint32_t bin = tid; bin < kPBins; bin += kPT) {
        const uint32_t start = bin ? cur[bin - 1] : 0u, end = cur[bin];
        for (uint32_t i = start + 1; i < end; ++i) {
          const uint32_t v = mem[i], kv = key[v];
          uint32_t j = i;
          while (j > start) {
            const uint32_t w = mem[j - 1], kw = key[w];
            if (!(kv < kw || (kv == kw && tie_less(base, v, w, a.attempt, a.seed)))) break;
            mem[j] = (uint16_t)w;
            --j;
          }
          mem[j] = (uint16_t)v;
        }
      }
      __syncthreads();
      // Z is a multiple of 32: the bucket's row is whole 16-byte words, 16-byte aligned
      uint4* dst = reinterpret_cast<uint4*>(a.ord + base);
      const uint4* src = reinterpret_cast<const uint4*>(mem);
      for (uint32_t x = tid; x < Z / 8; x += kPT) dst[x] = src[x];
      if (tid == 0) trace_log<TRACE>(a.trace, kWrite, kBufPerm, Z * 2, base * 2);
      __syncthreads();  // the next bucket reuses every array
    }
  }
}

}  // namespace

cudaError_t launch_perm_table(const PermTableArgs& a, cudaStream_t st, bool trace) {
  if (a.B == 0) return cudaSuccess;
  if (a.Z % 32 != 0 || a.Z > 4096 || (a.tag && a.k > kMaxK)) return cudaErrorInvalidValue;
  const uint32_t sm = table_smem(a.Z, a.tag ? 1u << a.k : 1u);
  int dev = 0, sms = 0, occ = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = trace ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, perm_table_kernel<true>, kPT, sm)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, perm_table_kernel<false>, kPT, sm);
  if (e != cudaSuccess) return e;
  const uint64_t units = a.tag ? a.B >> a.k : a.B;
  const uint64_t want = (uint64_t)sms * (occ > 0 ? occ : 1);
  const unsigned grid = (unsigned)(units < want ? units : want);
  if (trace)
    perm_table_kernel<true><<<grid, kPT, sm, st>>>(a);
  else
    perm_table_kernel<false><<<grid, kPT, sm, st>>>(a);
  return cudaGetLastError();
}

}  // namespace bos
