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
//   * reals only (the pass has input tags): final_load_kernel reads the LAST pass's input tags and
//     counts m for every final bucket exactly as the LAST pass will (the label digit of every
//     real); the table kernel sorts slots 0..m-1 and pads the row with 0xFFFF;
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
// 256 bins
__host__ __device__ inline uint32_t table_warps(uint32_t Z) { return Z <= 1024 ? 8u : (Z <= 2048 ? 4u : 2u); }
__host__ __device__ inline uint32_t warp_bytes(uint32_t Z) { return Z * 8 + kPBins * 4; }
uint32_t table_smem(uint32_t Z) { return table_warps(Z) * warp_bytes(Z); }

constexpr int kLT = 256;     // threads of the load-count kernel
constexpr int kLUnroll = 8;  // 16-byte tag loads in flight per thread

// load[q*D + u] = reals of LAST subproblem q whose routing digit is u, for every subproblem q:
// the reals of its input buckets s*2^i + t (s < D, q = G*2^i + t) with label bits [shift, shift+k)
// equal to u, as the LAST pass counts them.
template <bool TRACE>
__global__ void __launch_bounds__(kLT) final_load_kernel(PermTableArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* mcnt = reinterpret_cast<uint32_t*>(smem);
  const uint32_t Z = a.Z, D = 1u << a.k, cpb = Z / 4;  // 16-byte chunks per input bucket
  const uint32_t shift = a.L - a.i - a.k;
  const uint64_t units = a.B >> a.k;
  const int tid = threadIdx.x;
  for (uint64_t q = blockIdx.x; q < units; q += gridDim.x) {
    for (uint32_t x = tid; x < D; x += kLT) mcnt[x] = 0;
    __syncthreads();
    const uint64_t t = q & ((1ull << a.i) - 1), G = q >> a.i;
    if (TRACE && tid == 0)
      for (uint32_t s = 0; s < D; ++s)
        trace_log<TRACE>(a.trace, kRead, a.buf_tag, Z * 4, ((G << (a.i + a.k)) + ((uint64_t)s << a.i) + t) * Z * 4);
    const uint32_t nchunk = D * cpb;
    for (uint32_t c0 = tid; c0 < nchunk; c0 += kLT * kLUnroll) {
      uint4 v[kLUnroll];
#pragma unroll
      for (int e = 0; e < kLUnroll; ++e) {
        const uint32_t c = c0 + e * kLT;
        v[e] = make_uint4(kDummy, kDummy, kDummy, kDummy);
        if (c < nchunk) {
          const uint32_t s = c / cpb, off = c - s * cpb;
          const uint64_t gb = (G << (a.i + a.k)) + ((uint64_t)s << a.i) + t;
          v[e] = reinterpret_cast<const uint4*>(a.tag + gb * Z)[off];  // Z multiple of 32: aligned
        }
      }
#pragma unroll
      for (int e = 0; e < kLUnroll; ++e) {
        const uint32_t w[4] = {v[e].x, v[e].y, v[e].z, v[e].w};
#pragma unroll
        for (int f = 0; f < 4; ++f)
          if (w[f] != kDummy) atomicAdd(&mcnt[(w[f] >> shift) & (D - 1)], 1u);
      }
    }
    __syncthreads();
    for (uint32_t x = tid; x < D; x += kLT) a.load[q * D + x] = mcnt[x];
    __syncthreads();  // mcnt is cleared for the next subproblem
  }
}

template <bool TRACE>
__global__ void __launch_bounds__(256, 3) perm_table_kernel(PermTableArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t Z = a.Z, W = table_warps(Z);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned char* wbase = smem + warp * warp_bytes(Z);
  uint32_t* key = reinterpret_cast<uint32_t*>(wbase);               // [Z] w0 of each slot
  uint32_t* bins = key + Z;                                         // [kPBins] starts, then ends
  uint16_t* placed = reinterpret_cast<uint16_t*>(bins + kPBins);    // [Z] slots grouped by bin
  uint16_t* row = placed + Z;                                       // [Z] the sorted row
  const bool tagged = a.tag != nullptr;

  for (uint64_t b = (uint64_t)blockIdx.x * W + warp; b < a.B; b += (uint64_t)gridDim.x * W) {
    const uint64_t base = (a.bucket0 + b) * Z;  // the keys' counters use the global bucket
    const uint32_t m = tagged ? min(a.load[b], Z) : Z;
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
    // slots grouped by bin (any order inside a bin); bins[] becomes each bin's end. Four slots
    // per lane per step: independent chains.
    for (uint32_t s0 = lane; s0 < m; s0 += 128) {
      uint32_t p[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const uint32_t s = s0 + c * 32;
        p[c] = s < m ? atomicAdd(&bins[key[s] >> kShift], 1u) : 0u;
      }
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (s0 + c * 32 < m) placed[p[c]] = (uint16_t)(s0 + c * 32);
    }
    __syncwarp();
    // each slot's final place: its bin's start plus the members of the bin that sort before it
    for (uint32_t s0 = lane; s0 < m; s0 += 128) {
      uint32_t ks[4], start[4], end[4], rank[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const uint32_t s = s0 + c * 32;
        ks[c] = s < m ? key[s] : 0u;
        const uint32_t bin = ks[c] >> kShift;
        start[c] = s < m && bin ? bins[bin - 1] : 0u;
        end[c] = s < m ? bins[bin] : 0u;
        rank[c] = 0;
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const uint32_t s = s0 + c * 32;
        for (uint32_t e = start[c]; e < end[c]; ++e) {
          const uint32_t o = placed[e], ko = key[o];
          rank[c] += (ko < ks[c] || (ko == ks[c] && o != s && tie_less(base, o, s, a.attempt, a.seed))) ? 1u : 0u;
        }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (s0 + c * 32 < m) row[start[c] + rank[c]] = (uint16_t)(s0 + c * 32);
    }
    for (uint32_t s = m + lane; s < Z; s += 32) row[s] = 0xFFFFu;  // no real at these ranks
    __syncwarp();
    // Z is a multiple of 32: the bucket's row is whole 16-byte words, 16-byte aligned
    uint4* dst = reinterpret_cast<uint4*>(a.ord + b * Z);
    const uint4* src = reinterpret_cast<const uint4*>(row);
    for (uint32_t x = lane; x < Z / 8; x += 32) dst[x] = src[x];
    if (lane == 0) trace_log<TRACE>(a.trace, kWrite, kBufPerm, Z * 2, b * Z * 2);
    __syncwarp();  // the warp's next bucket reuses its arrays
  }
}

}  // namespace

template <bool TRACE>
cudaError_t perm_table_launch(const PermTableArgs& a, cudaStream_t st) {
  int dev = 0, sms = 0, occ = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (a.tag) {  // final loads first
    const uint32_t D = 1u << a.k;
    const uint32_t sm = D * 4;
    if ((e = set_smem_optin(final_load_kernel<TRACE>)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, final_load_kernel<TRACE>, kLT, sm)) != cudaSuccess)
      return e;
    const uint64_t units = a.B >> a.k, want = (uint64_t)sms * (occ > 0 ? occ : 1);
    final_load_kernel<TRACE><<<(unsigned)(units < want ? units : want), kLT, sm, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const uint32_t sm = table_smem(a.Z), W = table_warps(a.Z);
  if ((e = set_smem_optin(perm_table_kernel<TRACE>)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, perm_table_kernel<TRACE>, W * 32, sm)) != cudaSuccess)
    return e;
  const uint64_t need = (a.B + W - 1) / W, want = (uint64_t)sms * (occ > 0 ? occ : 1);
  perm_table_kernel<TRACE><<<(unsigned)(need < want ? need : want), W * 32, sm, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_perm_table(const PermTableArgs& a, cudaStream_t st, bool trace) {
  if (a.B == 0) return cudaSuccess;
  if (a.Z % 32 != 0 || a.Z > 4096 || (a.tag && (a.k > kMaxK || !a.load))) return cudaErrorInvalidValue;
  return trace ? perm_table_launch<true>(a, st) : perm_table_launch<false>(a, st);
}

}  // namespace bos
