// The ORP with O(1) client storage (Section 4.1), sm_103a: every MergeSplit is one bitonic sort of
// its two buckets, and every final bucket is permuted by one bitonic sort, so the schedule of
// shared-memory and global accesses depends on neither the data nor the labels.
//
//   place:  bucket j <- group j (Algorithm 3.1), labels drawn, padded with dummies.
//   level i (one launch each, i = 0 .. L-1): the CTA of pair j reads buckets a = j' + j and
//           a + 2^i, counts the reals going to each side (bit L-1-i of the label), gives the
//           first Z - c0 dummies side 0 and the rest side 1, and bitonic-sorts the 2Z slots by
//           (side, dummy, position); the first Z slots are bucket 2j, the next Z bucket 2j+1.
//           Reals keep their slot order on each side, so this is the stable MergeSplit.
//   final:  each final bucket is bitonic-sorted by (dummy, r, s), r the Section 3.2 key of slot s;
//           its m reals come first, in the in-bin permutation's order.
//   strip:  an exclusive scan of the loads m places every bucket's reals in the output.
// Keys are unique (positions and slots break ties), so no collision retry is needed; the
// permutation equals the fused path's, and so does every result.
#include "common.cuh"
#include "internal.h"

namespace bos {

namespace {

constexpr int kOT = 512;  // threads per CTA

__host__ __device__ inline uint32_t pow2_at_least(uint32_t x) {
  uint32_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

// Bitonic network over N (a power of two) slots held in shared memory as (key, tag, record); the
// compare-exchange schedule is fixed by N. Ascending by key; all threads of the CTA take part.
template <int R, typename K>
__device__ void bitonic_slots(K* key, uint32_t* tag, typename RecT<R>::T* rec, uint32_t N) {
  for (uint32_t size = 2; size <= N; size <<= 1) {
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      __syncthreads();
      for (uint32_t t = threadIdx.x; t < N / 2; t += blockDim.x) {
        const uint32_t lo = 2 * stride * (t / stride) + (t % stride), hi = lo + stride;
        const bool up = (lo & size) == 0;
        const K a = key[lo], b = key[hi];
        if ((b < a) == up) {
          key[lo] = b;
          key[hi] = a;
          const uint32_t tg = tag[lo];
          tag[lo] = tag[hi];
          tag[hi] = tg;
          const typename RecT<R>::T r = rec[lo];
          rec[lo] = rec[hi];
          rec[hi] = r;
        }
      }
    }
  }
  __syncthreads();
}

// Exclusive prefix over the CTA of one value per thread; the total comes back in *total.
__device__ uint32_t block_excl_scan(uint32_t v, uint32_t* ws, uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += y;
  }
  __syncthreads();
  if (lane == 31) ws[warp] = incl;
  __syncthreads();
  uint32_t before = 0, all = 0;
  for (int w = 0; w < nw; ++w) {
    const uint32_t x = ws[w];
    before += w < warp ? x : 0u;
    all += x;
  }
  *total = all;
  return before + incl - v;
}

template <int R, bool TRACE>
__global__ void obl_place_kernel(ObliviousArgs a) {
  using Rec = typename RecT<R>::T;
  const Rec* in = reinterpret_cast<const Rec*>(a.in);
  Rec* orec = reinterpret_cast<Rec*>(a.rec[0]);
  const uint64_t slots = a.B * a.Z;
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < slots; x += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t j = x / a.Z, s = x - j * a.Z;
    const uint64_t lo = (j * a.n) >> a.L, hi = ((j + 1) * a.n) >> a.L;  // group j, B = 2^L
    Rec r = RecT<R>::zero();
    uint32_t tg = kDummy;
    if (lo + s < hi) {
      r = in[lo + s];
      tg = label_of(lo + s, a.seed, a.attempt, a.L);
      trace_log<TRACE>(a.trace, kRead, kBufIn, R, (lo + s) * R);
    }
    orec[x] = r;
    a.tag[0][x] = tg;
    trace_log<TRACE>(a.trace, kWrite, kBufRecA, R, x * R);
    trace_log<TRACE>(a.trace, kWrite, kBufTagA, 4, x * 4);
  }
}

template <int R>
__host__ __device__ inline uint32_t level_smem(uint32_t Z) {
  const uint32_t N = pow2_at_least(2 * Z);
  return N * (uint32_t)sizeof(typename RecT<R>::T) + N * 4 + N * 4 + 64 * 4;
}

template <int R, bool TRACE>
__global__ void __launch_bounds__(kOT) obl_level_kernel(ObliviousArgs a, uint32_t i, uint32_t src) {
  using Rec = typename RecT<R>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t Z = a.Z, N = pow2_at_least(2 * Z), bit = a.L - 1 - i;
  Rec* rec = reinterpret_cast<Rec*>(smem);
  uint32_t* key = reinterpret_cast<uint32_t*>(rec + N);
  uint32_t* tag = key + N;
  uint32_t* ws = tag + N;  // [32] warp sums, [32..34] counts
  const Rec* irec = reinterpret_cast<const Rec*>(a.rec[src]);
  const uint32_t* itag = a.tag[src];
  Rec* orec = reinterpret_cast<Rec*>(a.rec[src ^ 1]);
  uint32_t* otag = a.tag[src ^ 1];
  const uint32_t bufr = src ? kBufRecB : kBufRecA, buft = src ? kBufTagB : kBufTagA;
  const uint32_t per = (N + kOT - 1) / kOT;  // slots per thread in the counting scans

  for (uint64_t j = blockIdx.x; j < a.B / 2; j += gridDim.x) {
    const uint64_t jp = (j >> i) << i, ia = jp + j, ib = ia + (1ull << i);
    for (uint32_t p = threadIdx.x; p < N; p += kOT) {
      if (p < 2 * Z) {
        const uint64_t g = (p < Z ? ia : ib) * Z + (p < Z ? p : p - Z);
        rec[p] = irec[g];
        tag[p] = itag[g];
      } else {
        tag[p] = kDummy;
      }
    }
    if (threadIdx.x == 0) {
      trace_log<TRACE>(a.trace, kRead, bufr, Z * R, ia * Z * R);
      trace_log<TRACE>(a.trace, kRead, buft, Z * 4, ia * Z * 4);
      trace_log<TRACE>(a.trace, kRead, bufr, Z * R, ib * Z * R);
      trace_log<TRACE>(a.trace, kRead, buft, Z * 4, ib * Z * 4);
    }
    __syncthreads();
    // reals per side and each dummy's rank among the dummies (thread t scans slots [t*per, ...))
    uint32_t c0 = 0, c1 = 0, nd = 0;
    for (uint32_t p = threadIdx.x * per; p < (threadIdx.x + 1) * per && p < 2 * Z; ++p) {
      const uint32_t tg = tag[p];
      if (tg == kDummy) ++nd;
      else if ((tg >> bit) & 1u) ++c1;
      else ++c0;
    }
    uint32_t tot0, tot1, totd;
    block_excl_scan(c0, ws, &tot0);
    block_excl_scan(c1, ws, &tot1);
    uint32_t drank = block_excl_scan(nd, ws, &totd);
    if (threadIdx.x == 0 && (tot0 > Z || tot1 > Z)) atomicExch(&a.ctrl->overflow, 1u);
    const uint32_t zero_dummies = tot0 < Z ? Z - tot0 : 0u;  // dummies that fill bucket 2j
    for (uint32_t p = threadIdx.x * per; p < (threadIdx.x + 1) * per && p < N; ++p) {
      uint32_t k = 0xFFFFFFFFu;  // padding slots sort last
      if (p < 2 * Z) {
        const uint32_t tg = tag[p];
        uint32_t side, dummy = 0;
        if (tg == kDummy) {
          dummy = 1;
          side = drank++ < zero_dummies ? 0u : 1u;
        } else {
          side = (tg >> bit) & 1u;
        }
        k = (side << 31) | (dummy << 30) | p;
      }
      key[p] = k;
    }
    bitonic_slots<R>(key, tag, rec, N);
    for (uint32_t p = threadIdx.x; p < 2 * Z; p += kOT) {
      const uint64_t g = (p < Z ? 2 * j : 2 * j + 1) * Z + (p < Z ? p : p - Z);
      const bool dummy = tag[p] == kDummy;
      orec[g] = dummy ? RecT<R>::zero() : rec[p];
      otag[g] = tag[p];
    }
    if (threadIdx.x == 0) {
      trace_log<TRACE>(a.trace, kWrite, src ? kBufRecA : kBufRecB, Z * R, 2 * j * Z * R);
      trace_log<TRACE>(a.trace, kWrite, src ? kBufTagA : kBufTagB, Z * 4, 2 * j * Z * 4);
      trace_log<TRACE>(a.trace, kWrite, src ? kBufRecA : kBufRecB, Z * R, (2 * j + 1) * Z * R);
      trace_log<TRACE>(a.trace, kWrite, src ? kBufTagA : kBufTagB, Z * 4, (2 * j + 1) * Z * 4);
    }
    __syncthreads();  // the next pair reuses shared memory
  }
}

template <int R>
__host__ __device__ inline uint32_t final_smem(uint32_t Z) {
  const uint32_t N = pow2_at_least(Z);
  return N * (uint32_t)sizeof(typename RecT<R>::T) + N * 8 + N * 4 + 64 * 4;
}

// Final bucket b: bitonic sort by (dummy, r, s); the m reals come first, in permuted order. The
// bucket is written back in that order and m goes to load[b].
template <int R, bool TRACE>
__global__ void __launch_bounds__(kOT) obl_final_kernel(ObliviousArgs a, uint32_t src) {
  using Rec = typename RecT<R>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t Z = a.Z, N = pow2_at_least(Z);
  Rec* rec = reinterpret_cast<Rec*>(smem);
  unsigned long long* key = reinterpret_cast<unsigned long long*>(rec + N);  // [N] packed (r high, then s)
  uint32_t* tag = reinterpret_cast<uint32_t*>(key + N);
  uint32_t* ws = tag + N;
  Rec* brec = reinterpret_cast<Rec*>(a.rec[src]);
  uint32_t* btag = a.tag[src];
  const uint32_t bufr = src ? kBufRecB : kBufRecA, buft = src ? kBufTagB : kBufTagA;
  for (uint64_t b = blockIdx.x; b < a.B; b += gridDim.x) {
    for (uint32_t s = threadIdx.x; s < N; s += kOT) {
      if (s < Z) {
        rec[s] = brec[b * Z + s];
        tag[s] = btag[b * Z + s];
      } else {
        tag[s] = kDummy;
      }
    }
    if (threadIdx.x == 0) {
      trace_log<TRACE>(a.trace, kRead, bufr, Z * R, b * Z * R);
      trace_log<TRACE>(a.trace, kRead, buft, Z * 4, b * Z * 4);
    }
    __syncthreads();
    uint32_t m = 0, cnt = 0;
    for (uint32_t s = threadIdx.x; s < N; s += kOT) cnt += (s < Z && tag[s] != kDummy) ? 1u : 0u;
    block_excl_scan(cnt, ws, &m);
    // The reals are slots 0..m-1. A real's key holds r's top 51 bits, a zero bit and s (12 bits,
    // Z <= 4096), so every real sorts before the dummies and padding (key ~0); reals whose top 51
    // bits agree are put in (r, s) order below.
    for (uint32_t s = threadIdx.x; s < N; s += kOT) {
      unsigned long long k = ~0ull;
      if (s < m) {
        const PhiloxOut w = philox_at(b * Z + s, a.attempt, 1, a.seed);
        const unsigned long long r = ((unsigned long long)w.w0 << 32) | w.w1;
        k = ((r >> 13) << 13) | s;
      }
      key[s] = k;
    }
    bitonic_slots<R>(key, tag, rec, N);
    // equal top 51 bits of r (rare): order the run by the whole (r, s), one thread per run
    for (uint32_t x = threadIdx.x; x < m; x += kOT) {
      if (x > 0 && (key[x - 1] >> 13) == (key[x] >> 13)) continue;
      uint32_t e = x + 1;
      while (e < m && (key[e] >> 13) == (key[x] >> 13)) ++e;
      for (uint32_t u = x + 1; u < e; ++u) {  // insertion sort of the (rare) run by (r, s)
        for (uint32_t v = u; v > x; --v) {
          const uint32_t s1 = (uint32_t)(key[v - 1] & 0xFFFu), s2 = (uint32_t)(key[v] & 0xFFFu);
          const PhiloxOut w1 = philox_at(b * Z + s1, a.attempt, 1, a.seed), w2 = philox_at(b * Z + s2, a.attempt, 1, a.seed);
          const unsigned long long r1 = ((unsigned long long)w1.w0 << 32) | w1.w1;
          const unsigned long long r2 = ((unsigned long long)w2.w0 << 32) | w2.w1;
          if (r1 < r2 || (r1 == r2 && s1 < s2)) break;
          const unsigned long long tk = key[v - 1];
          key[v - 1] = key[v];
          key[v] = tk;
          const uint32_t tt = tag[v - 1];
          tag[v - 1] = tag[v];
          tag[v] = tt;
          const Rec tr = rec[v - 1];
          rec[v - 1] = rec[v];
          rec[v] = tr;
        }
      }
    }
    __syncthreads();
    for (uint32_t s = threadIdx.x; s < Z; s += kOT) {
      brec[b * Z + s] = rec[s];
      btag[b * Z + s] = tag[s];
    }
    if (threadIdx.x == 0) {
      a.load[b] = m;
      trace_log<TRACE>(a.trace, kWrite, bufr, Z * R, b * Z * R);
      trace_log<TRACE>(a.trace, kWrite, buft, Z * 4, b * Z * 4);
    }
    __syncthreads();
  }
}

// Exclusive scan of the B loads into off (two levels: blocks of kScanBlock, then their sums).
constexpr uint32_t kScanPer = 8, kScanBlock = kOT * kScanPer;

__global__ void __launch_bounds__(kOT) obl_scan_local_kernel(const uint32_t* load, uint32_t* off, uint32_t* part,
                                                             uint64_t B) {
  __shared__ uint32_t ws[64];
  const uint64_t base = (uint64_t)blockIdx.x * kScanBlock + threadIdx.x * kScanPer;
  uint32_t v[kScanPer], sum = 0;
#pragma unroll
  for (uint32_t e = 0; e < kScanPer; ++e) {
    v[e] = base + e < B ? load[base + e] : 0u;
    sum += v[e];
  }
  uint32_t total;
  uint32_t run = block_excl_scan(sum, ws, &total);
#pragma unroll
  for (uint32_t e = 0; e < kScanPer; ++e) {
    if (base + e < B) off[base + e] = run;
    run += v[e];
  }
  if (threadIdx.x == 0) part[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kOT) obl_scan_parts_kernel(uint32_t* part, uint32_t nparts) {
  __shared__ uint32_t ws[64];
  uint32_t carry = 0;
  for (uint32_t b0 = 0; b0 < nparts; b0 += kOT) {
    const uint32_t x = b0 + threadIdx.x;
    const uint32_t v = x < nparts ? part[x] : 0u;
    uint32_t total;
    const uint32_t e = block_excl_scan(v, ws, &total);
    if (x < nparts) part[x] = carry + e;
    carry += total;
    __syncthreads();
  }
}

template <int R, bool TRACE>
__global__ void obl_strip_kernel(ObliviousArgs a, uint32_t src) {
  using Rec = typename RecT<R>::T;
  const Rec* brec = reinterpret_cast<const Rec*>(a.rec[src]);
  Rec* out = reinterpret_cast<Rec*>(a.out0);
  if (a.out_sel && sort_passes_odd(a.ctrl)) out = reinterpret_cast<Rec*>(a.out1);
  const uint32_t out_buf = (out == reinterpret_cast<Rec*>(a.out0)) ? kBufOut : kBufTmp;
  const uint32_t bufr = src ? kBufRecB : kBufRecA;
  for (uint64_t b = blockIdx.x; b < a.B; b += gridDim.x) {
    const uint64_t o = (uint64_t)a.off[b] + a.part[b / kScanBlock];
    const uint32_t m = a.load[b];
    for (uint32_t x = threadIdx.x; x < m; x += blockDim.x) {
      if (o + x < a.n) {
        out[o + x] = brec[b * a.Z + x];
        trace_log<TRACE>(a.trace, kRead, bufr, R, (b * a.Z + x) * R);
        trace_log<TRACE>(a.trace, kWrite, out_buf, R, (o + x) * R);
      }
    }
  }
}

template <int R, bool TRACE>
cudaError_t oblivious_r(const ObliviousArgs& a, cudaStream_t st) {
  cudaError_t e;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const uint64_t slots = a.B * a.Z;
  obl_place_kernel<R, TRACE><<<(unsigned)((slots + 255) / 256 < (uint64_t)sms * 16 ? (slots + 255) / 256 : (uint64_t)sms * 16), 256, 0,
                               st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  uint32_t src = 0;
  const uint32_t lsm = level_smem<R>(a.Z), fsm = final_smem<R>(a.Z);
  if ((e = set_smem_optin(obl_level_kernel<R, TRACE>)) != cudaSuccess) return e;
  if ((e = set_smem_optin(obl_final_kernel<R, TRACE>)) != cudaSuccess) return e;
  int occ = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, obl_level_kernel<R, TRACE>, kOT, lsm)) != cudaSuccess)
    return e;
  const uint64_t lgrid = (uint64_t)sms * (occ > 0 ? occ : 1);
  for (uint32_t i = 0; i < a.L; ++i) {
    obl_level_kernel<R, TRACE><<<(unsigned)(a.B / 2 < lgrid ? a.B / 2 : lgrid), kOT, lsm, st>>>(a, i, src);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    src ^= 1u;
  }
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, obl_final_kernel<R, TRACE>, kOT, fsm)) != cudaSuccess)
    return e;
  const uint64_t fgrid = (uint64_t)sms * (occ > 0 ? occ : 1);
  obl_final_kernel<R, TRACE><<<(unsigned)(a.B < fgrid ? a.B : fgrid), kOT, fsm, st>>>(a, src);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const uint32_t nparts = (uint32_t)((a.B + kScanBlock - 1) / kScanBlock);
  obl_scan_local_kernel<<<nparts, kOT, 0, st>>>(a.load, a.off, a.part, a.B);
  obl_scan_parts_kernel<<<1, kOT, 0, st>>>(a.part, nparts);
  obl_strip_kernel<R, TRACE><<<(unsigned)(a.B < (uint64_t)sms * 8 ? a.B : (uint64_t)sms * 8), 256, 0, st>>>(a, src);
  return cudaGetLastError();
}

}  // namespace

uint32_t oblivious_smem_bytes(int R, uint32_t Z) {
  return R == 8 ? (level_smem<8>(Z) > final_smem<8>(Z) ? level_smem<8>(Z) : final_smem<8>(Z))
                : (level_smem<16>(Z) > final_smem<16>(Z) ? level_smem<16>(Z) : final_smem<16>(Z));
}

cudaError_t launch_oblivious_orp(const ObliviousArgs& a, int R, cudaStream_t st, bool trace) {
  if (R == 8) return trace ? oblivious_r<8, true>(a, st) : oblivious_r<8, false>(a, st);
  return trace ? oblivious_r<16, true>(a, st) : oblivious_r<16, false>(a, st);
}

}  // namespace bos
