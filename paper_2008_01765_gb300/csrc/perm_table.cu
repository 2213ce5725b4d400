// In-bin permutation table of the fused LAST pass (Section 3.2), sm_103a.
//
// Final bucket b ends the butterfly with its m reals at slots 0..m-1 in stable order. Slot s has
// the key r(b, s) = (w0 << 32 | w1) of Philox(b*Z + s, attempt, stream 1), and the reals leave
// the bucket ordered by (r, s). The keys depend on neither the data nor the routing, so this
// kernel sorts each final bucket's slots by (r, s) ahead of the LAST pass, at full occupancy,
// and the LAST pass only filters its rows.
//
// Row b of the table lists slots in key order, Z entries of u16. The LAST pass keeps the entries
// below m; dropping the others keeps their relative order, so either of two rows serves:
//   * reals only (the pass has input tags): the CTA reads the LAST subproblem's input tags and
//     counts m for each of its final buckets exactly as the LAST pass will (the label digit of
//     every real), then sorts slots 0..m-1 and pads the row with 0xFFFF;
//   * all slots (a single pass that draws the labels itself): slots 0..Z-1 sorted.
// One warp sorts one final bucket with no block-wide barrier: it draws the keys, counts the top 8
// bits of w0 into 256 bins of its own, scans them, places each slot in its bin, and puts each
// slot at its bin's start plus its rank among the bin's few members (compared by (w0, w1, s)).
#include "common.cuh"
#include "internal.h"

namespace bos {

namespace {

constexpr int kPBins = 256;        // bins: top 8 bits of w0
constexpr int kShift = 24;
constexpr uint32_t kMaxK = 12;     // final buckets per LAST subproblem: at most 2^12

// Slot s3 sorts before slot s2 (same bucket, base = b*Z, equal w0): smaller w1, or equal w1 and
// s3 < s2. Rare (equal 32-bit words), so out of line.
__device__ __noinline__ bool tie_less(uint64_t base, uint32_t s3, uint32_t s2, uint32_t attempt, uint64_t seed) {
  const uint32_t l2 = philox_at(base + s2, attempt, 1, seed).w1;
  const uint32_t l3 = philox_at(base + s3, attempt, 1, seed).w1;
  return (l3 < l2) || (l3 == l2 && s3 < s2);
}

// warps per CTA and shared memory: per warp Z keys (u32), Z placed slots and Z row entries (u16),
// 256 bins; per CTA the final-bucket loads of one LAST subproblem
__host__ __device__ inline uint32_t table_warps(uint32_t Z) { return Z <= 1024 ? 8u : (Z <= 2048 ? 4u : 2u); }
__host__ __device__ inline uint32_t warp_bytes(uint32_t Z) { return Z * 8 + kPBins * 4; }
uint32_t table_smem(uint32_t Z, uint32_t D) { return table_warps(Z) * warp_bytes(Z) + D * 4; }

template <bool TRACE>
__global__ void __launch_bounds__(256) perm_table_kernel(PermTableArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t Z = a.Z, W = table_warps(Z);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nthreads = (int)W * 32;
  unsigned char* wbase = smem + warp * warp_bytes(Z);
  uint32_t* key = reinterpret_cast<uint32_t*>(wbase);               // [Z] w0 of each slot
  uint32_t* bins = key + Z;                                         // [kPBins] starts, then ends
  uint16_t* placed = reinterpret_cast<uint16_t*>(bins + kPBins);    // [Z] slots grouped by bin
  uint16_t* row = placed + Z;                                       // [Z] the sorted row
  uint32_t* mcnt = reinterpret_cast<uint32_t*>(smem + W * warp_bytes(Z));  // [D] reals per final bucket
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
      for (uint32_t x = tid; x < D; x += nthreads) mcnt[x] = 0;
      __syncthreads();
      const uint64_t t = q & ((1ull << a.i) - 1), G = q >> a.i;
      for (uint32_t s = warp; s < D; s += W) {
        const uint64_t gb = (G << (a.i + a.k)) + ((uint64_t)s << a.i) + t;
        if (lane == 0) trace_log<TRACE>(a.trace, kRead, a.buf_tag, Z * 4, gb * Z * 4);
        const uint4* tg4 = reinterpret_cast<const uint4*>(a.tag + gb * Z);  // Z multiple of 32: 16-byte rows
        // every lane runs every step (the match below needs the whole warp), past the row as dummies
        for (uint32_t c0 = 0; c0 < Z / 4; c0 += 32) {
          const uint32_t c = c0 + lane;
          const uint4 v = c < Z / 4 ? tg4[c] : make_uint4(kDummy, kDummy, kDummy, kDummy);
          const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const bool real = w[e] != kDummy;
            const uint32_t u = real ? (w[e] >> shift) & (D - 1) : D;
            const uint32_t peers = __match_any_sync(0xFFFFFFFFu, u);
            if (real && (peers & lt_mask) == 0) atomicAdd(&mcnt[u], (uint32_t)__popc(peers));
          }
        }
      }
      __syncthreads();
    }
    for (uint32_t u = warp; u < D; u += W) {
      const uint64_t b = q * D + u, base = b * Z;
      const uint32_t m = tagged ? min(mcnt[u], Z) : Z;
      for (int x = lane; x < kPBins; x += 32) bins[x] = 0;
      __syncwarp();
      // keys and bin counts (four independent Philox chains per lane per step)
      for (uint32_t s0 = lane; s0 < m; s0 += 128) {
        uint32_t w[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) w[c] = s0 + c * 32 < m ? philox_at(base + s0 + c * 32, a.attempt, 1, a.seed).w0 : 0u;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const uint32_t s = s0 + c * 32;
          if (s < m) {
            key[s] = w[c];
            atomicAdd(&bins[w[c] >> kShift], 1u);
          }
        }
      }
      __syncwarp();
      {  // exclusive scan of the bins: eight consecutive bins per lane
        uint32_t v[kPBins / 32], sum = 0;
#pragma unroll
        for (int e = 0; e < kPBins / 32; ++e) {
          v[e] = bins[lane * (kPBins / 32) + e];
          sum += v[e];
        }
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
          if (lane >= o) incl += y;
        }
        uint32_t run = incl - sum;
#pragma unroll
        for (int e = 0; e < kPBins / 32; ++e) {
          bins[lane * (kPBins / 32) + e] = run;
          run += v[e];
        }
      }
      __syncwarp();
      // slots grouped by bin (any order inside a bin); bins[] becomes each bin's end
      for (uint32_t s = lane; s < m; s += 32) placed[atomicAdd(&bins[key[s] >> kShift], 1u)] = (uint16_t)s;
      __syncwarp();
      // each slot's final place: its bin's start plus the members of the bin that sort before it
      for (uint32_t s = lane; s < m; s += 32) {
        const uint32_t ks = key[s], bin = ks >> kShift;
        const uint32_t start = bin ? bins[bin - 1] : 0u, end = bins[bin];
        uint32_t rank = 0;
        for (uint32_t e = start; e < end; ++e) {
          const uint32_t o = placed[e], ko = key[o];
          rank += (ko < ks || (ko == ks && o != s && tie_less(base, o, s, a.attempt, a.seed))) ? 1u : 0u;
        }
        row[start + rank] = (uint16_t)s;
      }
      for (uint32_t s = m + lane; s < Z; s += 32) row[s] = 0xFFFFu;  // no real at these ranks
      __syncwarp();
      // Z is a multiple of 32: the bucket's row is whole 16-byte words, 16-byte aligned
      uint4* dst = reinterpret_cast<uint4*>(a.ord + base);
      const uint4* src = reinterpret_cast<const uint4*>(row);
      for (uint32_t x = lane; x < Z / 8; x += 32) dst[x] = src[x];
      if (lane == 0) trace_log<TRACE>(a.trace, kWrite, kBufPerm, Z * 2, base * 2);
      __syncwarp();  // the warp's next bucket reuses its arrays
    }
    if (tagged) __syncthreads();  // mcnt is reset by the next subproblem
  }
}

}  // namespace

cudaError_t launch_perm_table(const PermTableArgs& a, cudaStream_t st, bool trace) {
  if (a.B == 0) return cudaSuccess;
  if (a.Z % 32 != 0 || a.Z > 4096 || (a.tag && a.k > kMaxK)) return cudaErrorInvalidValue;
  const uint32_t sm = table_smem(a.Z, a.tag ? 1u << a.k : 1u), nt = table_warps(a.Z) * 32;
  int dev = 0, sms = 0, occ = 0;
  cudaError_t e = trace ? set_smem_optin(perm_table_kernel<true>) : set_smem_optin(perm_table_kernel<false>);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = trace ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, perm_table_kernel<true>, nt, sm)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, perm_table_kernel<false>, nt, sm);
  if (e != cudaSuccess) return e;
  const uint64_t units = a.tag ? a.B >> a.k : a.B;
  const uint64_t want = (uint64_t)sms * (occ > 0 ? occ : 1);
  const unsigned grid = (unsigned)(units < want ? units : want);
  if (trace)
    perm_table_kernel<true><<<grid, nt, sm, st>>>(a);
  else
    perm_table_kernel<false><<<grid, nt, sm, st>>>(a);
  return cudaGetLastError();
}

}  // namespace bos
