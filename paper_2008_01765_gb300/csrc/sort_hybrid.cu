// Hybrid radix sort of the ORP's output (Section 3.3: after the ORP, any non-oblivious sort). Its
// result is the stable sort by key of the ORP output, the same as the LSD radix sort's; it moves
// the records over HBM fewer times when the keys spread over the top digits.
//
//   1. histogram: one read of the keys gives the counts of every 8-bit digit and of the top two
//      digits together (65536 groups);
//   2. plan (one CTA): mode 1 when all n records fit one CTA's on-chip sort (kCap records); mode 2
//      when every value of the most significant varying digit dA holds at most kCap records;
//      mode 3 when dA and dB (the next varying digit) are the key's top two digits and every
//      (dA, dB) group holds at most kCap; otherwise mode 0, and the LSD passes run instead.
//      Consecutive groups are packed into ranges of whole groups holding at most kCap records;
//   3. modes 2, 3: a stable partition of the whole array by dA (the onesweep tile of the LSD pass);
//   4. mode 3: a stable partition by dB inside every dA bucket (tiles per bucket, the look-back
//      stopping at the bucket's first tile);
//   5. every range is sorted on chip by (key, position) and its records gathered into place: a
//      range of at most 1024 records by one warp in registers, a larger one by a CTA (a stable
//      partition by the range's top varying digit in shared memory, then a warp sort of every
//      sub-bucket; LSD passes over the varying digits when that does not fit).
// The partitions are stable and a range holds whole groups in key order, so sorting every range
// by key sorts the array; ties keep the ORP's order. HBM passes: the mode's count (1 to 3) plus
// the histogram, against 1 + the live digits for the LSD sort.
#include "common.cuh"
#include "internal.h"
#include "radix_tile.cuh"

namespace bos {

namespace {

constexpr int kJThreads = 1024;          // histogram CTA (one per SM: its shared memory holds the groups)
constexpr uint32_t kGroups = 65536;      // top two digits
constexpr int kPlanThreads = 1024;
constexpr int kLThreads = 512;           // local sort CTA
constexpr int kLWarps = kLThreads / 32;
constexpr uint32_t kLocalMaxCtas = 192;  // spill buffers in the workspace (one per CTA)
constexpr uint32_t kTagMsd1 = 12, kTagMsd2 = 13;
constexpr uint32_t kTicketMsd1 = 10, kTicketMsd2 = 11, kTicketLocal = 12;
constexpr uint32_t kWarpMax = 256;        // largest sub-bucket one warp sorts in registers
constexpr int kSThreads = 256;            // warp-per-range kernel
constexpr uint32_t kSmallMax = 1024;      // ranges of at most this many records: one warp each
constexpr uint32_t kRangeList = 65537;    // the small ranges' list starts here in ridx
constexpr uint32_t kTicketSmall = 13;     // and 14
static_assert(kGroups <= 64u * kPlanThreads, "the plan keeps one bit per range in a 64-bit word");

template <int R> struct Local;
template <> struct Local<16> { static constexpr uint32_t kCap = 19456; };  // 10 B per record on chip
template <> struct Local<8> { static constexpr uint32_t kCap = 28672; };   // 6 B per record on chip

__host__ __device__ constexpr uint32_t al16(uint32_t x) { return (x + 15u) & ~15u; }

// Shared memory of the local sort: keys [kCap], positions (u16) [kCap], two per-warp digit count
// tables [2][kLWarps][257], the count scan's scratch [512 + 8], the key AND/OR of every warp, misc
// [4], the sub-bucket starts [257].
template <int R>
__host__ __device__ constexpr uint32_t local_smem_bytes() {
  using Key = typename RecT<R>::Key;
  return al16(Local<R>::kCap * (uint32_t)(sizeof(Key) + 2)) + 2 * kLWarps * 257 * 4 + (512 + 8) * 4 +
         2 * kLWarps * (uint32_t)sizeof(Key) + 16 + 257 * 4;
}
static_assert(local_smem_bytes<16>() <= 232448 - 1024, "local sort shared memory");
static_assert(local_smem_bytes<8>() <= 232448 - 1024, "local sort shared memory");

template <int R>
__device__ __forceinline__ typename RecT<R>::T* sort_buf(const HybridArgs& a, uint32_t passes, uint32_t j) {
  // buffer chain of the sort: X_passes = output, alternating backwards (X_0 is the ORP's target)
  return reinterpret_cast<typename RecT<R>::T*>(((passes - j) & 1u) ? a.buf1 : a.buf0);
}

// Key of record p (its first key_bytes bytes, little-endian), read without the payload.
template <int R>
__device__ __forceinline__ typename RecT<R>::Key load_key(const typename RecT<R>::T* p) {
  return *reinterpret_cast<const typename RecT<R>::Key*>(p);
}

// ---- 1. histogram ---------------------------------------------------------------------------

// The group counters are 16 bits, two to a shared-memory word; an increment that takes one to
// 2^15 moves 2^15 to the group's global counter, so a half never carries into its neighbour.
template <int R>
__device__ __forceinline__ void count_key(typename RecT<R>::Key key, uint32_t* h, uint32_t* jp, uint32_t* joint) {
  constexpr int D = RecT<R>::kDigits;
#pragma unroll
  for (int d = 0; d < D; ++d) atomicAdd(&h[d * 256 + (uint32_t)((key >> (8 * d)) & 255u)], 1u);
  const uint32_t g = (uint32_t)(key >> (8 * (D - 2))) & 0xFFFFu;
  const uint32_t sh = (g & 1u) << 4;
  const uint32_t old = atomicAdd(&jp[g >> 1], 1u << sh);
  if (((old >> sh) & 0xFFFFu) == 0x7FFFu) {
    atomicSub(&jp[g >> 1], 0x8000u << sh);
    atomicAdd(joint + g, 0x8000u);
  }
}

template <int R>
__global__ void __launch_bounds__(kJThreads, 1) hybrid_hist_kernel(HybridArgs a) {
  using Rec = typename RecT<R>::T;
  using Key = typename RecT<R>::Key;
  constexpr int D = RecT<R>::kDigits;
  extern __shared__ __align__(16) uint32_t hsm[];
  uint32_t* h = hsm;             // [D][256]
  uint32_t* jp = hsm + D * 256;  // [kGroups / 2]
  for (uint32_t x = threadIdx.x; x < D * 256 + kGroups / 2; x += kJThreads) hsm[x] = 0;
  __syncthreads();
  const Rec* in = reinterpret_cast<const Rec*>(a.in);
  const uint64_t step = (uint64_t)gridDim.x * kJThreads;
  uint64_t idx = (uint64_t)blockIdx.x * kJThreads + threadIdx.x;
  for (; idx + 3 * step < a.n; idx += 4 * step) {  // four loads in flight per thread
    Key k[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) k[u] = load_key<R>(in + idx + u * step);
#pragma unroll
    for (int u = 0; u < 4; ++u) count_key<R>(k[u], h, jp, a.joint);
  }
  for (; idx < a.n; idx += step) count_key<R>(load_key<R>(in + idx), h, jp, a.joint);
  __syncthreads();
  for (uint32_t x = threadIdx.x; x < D * 256; x += kJThreads)
    if (h[x]) atomicAdd(a.hist + x, h[x]);
  for (uint32_t w = threadIdx.x; w < kGroups / 2; w += kJThreads) {
    const uint32_t v = jp[w];
    if (v & 0xFFFFu) atomicAdd(a.joint + 2 * w, v & 0xFFFFu);
    if (v >> 16) atomicAdd(a.joint + 2 * w + 1, v >> 16);
  }
}

// ---- 2. plan --------------------------------------------------------------------------------

// Exclusive scan of one value per thread over the CTA (kPlanThreads threads); *total gets the sum.
__device__ __forceinline__ unsigned long long plan_scan(unsigned long long v, unsigned long long* s_w,
                                                        unsigned long long* total) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  unsigned long long incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= (uint32_t)o) incl += y;
  }
  if (lane == 31) s_w[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    unsigned long long t = s_w[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, t, o);
      if (lane >= (uint32_t)o) t += y;
    }
    s_w[lane] = t;
  }
  __syncthreads();
  const unsigned long long ex = incl - v + (warp ? s_w[warp - 1] : 0ull);
  *total = s_w[31];
  __syncthreads();
  return ex;
}

template <int R>
__global__ void __launch_bounds__(kPlanThreads) sort_plan_kernel(HybridArgs a) {
  constexpr int D = RecT<R>::kDigits;
  constexpr uint32_t kCap = Local<R>::kCap;
  __shared__ uint32_t s_max[8], s_jmax, s_mode, s_dA, s_dB;
  __shared__ unsigned long long s_w[32];
  const uint32_t tid = threadIdx.x;
  if (tid < 8) s_max[tid] = 0;
  if (tid == 0) s_jmax = 0;
  __syncthreads();
  for (uint32_t x = tid; x < D * 256; x += kPlanThreads) atomicMax(&s_max[x >> 8], a.hist[x]);
  uint32_t jm = 0;
  for (uint32_t x = tid; x < kGroups; x += kPlanThreads) jm = a.joint[x] > jm ? a.joint[x] : jm;
  atomicMax(&s_jmax, jm);
  __syncthreads();
  if (tid == 0) {
    int dA = -1, dB = -1;
    for (int d = D - 1; d >= 0; --d)
      if ((uint64_t)s_max[d] < a.n) {  // some key differs in digit d
        if (dA < 0) dA = d;
        else if (dB < 0) dB = d;
      }
    uint32_t mode = 0;
    if (a.n >= 2 && dA >= 0) {
      if (a.n <= kCap) mode = 1;
      else if (s_max[dA] <= kCap) mode = 2;
      else if (dA == D - 1 && dB == D - 2 && s_jmax <= kCap) mode = 3;
    }
    s_mode = mode;
    s_dA = dA < 0 ? 0u : (uint32_t)dA;
    s_dB = dB < 0 ? 0u : (uint32_t)dB;
    a.meta[0] = mode;
    a.meta[1] = s_dA;
    a.meta[2] = s_dB;
    a.meta[3] = 0;
  }
  __syncthreads();
  const uint32_t mode = s_mode, dA = s_dA;
  if (mode == 0) {
    if (tid == 0) a.ctrl->sort_mode = 0;
    return;
  }
  // groups: the whole array (mode 1), the values of dA (mode 2), the (dA, dB) pairs (mode 3)
  const uint32_t G = mode == 1 ? 1u : mode == 2 ? 256u : kGroups;
  const uint64_t gmax = mode == 1 ? a.n : mode == 2 ? s_max[dA] : s_jmax;
  auto count = [&](uint32_t g) -> uint64_t {
    return mode == 1 ? a.n : mode == 2 ? (uint64_t)a.hist[dA * 256 + g] : (uint64_t)a.joint[g];
  };
  // Ranges. Groups of more than kWarpMax records each get a range of their own (with the empty
  // groups after it), so the on-chip sort splits them by the next digit into small sub-buckets.
  // Smaller groups are packed: a range is a run of consecutive groups whose starts fall in one
  // window of S records (at most S - 1 + gmax <= kCap records), broken at every top-digit value
  // in mode 3, so that the groups are the on-chip sort's sub-buckets.
  const bool single = gmax > kWarpMax;
  const uint64_t S = (uint64_t)kCap - gmax + 1;
  auto starts = [&](uint32_t g, uint64_t gs) -> bool {
    if (g == 0) return true;
    if (single) return count(g) > 0;
    return (mode == 3 && (g & 255u) == 0) || gs / S != (gs - count(g - 1)) / S;
  };
  const uint32_t per = (G + kPlanThreads - 1) / kPlanThreads;
  const uint32_t g0 = tid * per < G ? tid * per : G, g1 = g0 + per < G ? g0 + per : G;
  unsigned long long sum = 0, total = 0;
  for (uint32_t g = g0; g < g1; ++g) sum += count(g);
  const unsigned long long ex = plan_scan(sum, s_w, &total);
  unsigned long long gs = ex;
  uint32_t nr = 0;
  for (uint32_t g = g0; g < g1; ++g) {
    a.gstart[g] = gs;
    nr += starts(g, gs) ? 1u : 0u;
    gs += count(g);
  }
  if (tid == 0) a.gstart[G] = total;
  unsigned long long nranges = 0;
  unsigned long long rx = plan_scan(nr, s_w, &nranges);
  gs = ex;
  for (uint32_t g = g0; g < g1; ++g) {
    if (starts(g, gs)) a.rlist[rx++] = g;
    gs += count(g);
  }
  if (tid == 0) {
    a.rlist[nranges] = G;
    a.meta[3] = (uint32_t)nranges;
  }
  __syncthreads();  // the range list and the group starts are written
  {  // ranges of at most kSmallMax records go to the warp kernel, larger ones to the CTA kernel
    const uint32_t NR = (uint32_t)nranges, rper = (NR + kPlanThreads - 1) / kPlanThreads;
    const uint32_t r0 = tid * rper < NR ? tid * rper : NR, r1 = r0 + rper < NR ? r0 + rper : NR;
    // at most 64 ranges per thread (at most 65536 ranges): one bit each, set for a small range
    unsigned long long small = 0;
#pragma unroll 8
    for (uint32_t r = r0; r < r1; ++r)
      if (a.gstart[a.rlist[r + 1]] - a.gstart[a.rlist[r]] <= kSmallMax) small |= 1ull << (r - r0);
    unsigned long long tsm = 0, tbg = 0;
    const unsigned long long nsm = (unsigned long long)__popcll(small);
    unsigned long long xs = plan_scan(nsm, s_w, &tsm);
    unsigned long long xb = plan_scan((r1 - r0) - nsm, s_w, &tbg);
    for (uint32_t r = r0; r < r1; ++r) {
      if ((small >> (r - r0)) & 1ull)
        a.ridx[kRangeList + xs++] = r;
      else
        a.ridx[xb++] = r;
    }
    if (tid == 0) {
      a.meta[4] = (uint32_t)tbg;
      a.meta[5] = (uint32_t)tsm;
    }
  }
  if (mode == 3) {  // MSD2 tiles: every dA bucket is cut into tiles of its own
    const uint64_t tb = tid < 256 ? ((uint64_t)a.hist[dA * 256 + tid] + kTile - 1) / kTile : 0ull;
    unsigned long long ttot = 0;
    const unsigned long long tx = plan_scan(tb, s_w, &ttot);
    if (tid < 256) a.first[tid] = tx;
    if (tid == 0) a.first[256] = ttot;
  }
  __syncthreads();
  if (tid == 0) a.ctrl->sort_mode = mode;
}

// ---- 3, 4. MSD partitions ---------------------------------------------------------------------
// Persistent, like the LSD pass: CTAs take tiles by ticket, so a launch whose mode does not run
// it costs one early return per CTA.

template <int R>
__global__ void __launch_bounds__(kThreads, 2) msd1_kernel(HybridArgs a) {
  const uint32_t mode = a.ctrl->sort_mode;
  if (mode < 2) return;
  __shared__ unsigned long long t_s;
  const uint32_t dA = a.meta[1];
  const uint64_t tiles = (a.n + kTile - 1) / kTile;
  while (true) {
    if (threadIdx.x == 0) t_s = atomicAdd(&a.ctrl->tickets[kTicketMsd1], 1u);
    __syncthreads();
    const unsigned long long t = t_s;
    if (t >= tiles) break;
    radix_tile<R>(sort_buf<R>(a, mode, 0), sort_buf<R>(a, mode, 1), a.n, t, 8 * dA, kTagMsd1, a.status,
                  a.dbase + dA * 256, a.n, a.ctrl);
    __syncthreads();
  }
}

template <int R>
__global__ void __launch_bounds__(kThreads, 2) msd2_kernel(HybridArgs a) {
  if (a.ctrl->sort_mode != 3) return;
  __shared__ unsigned long long t_s;
  __shared__ uint32_t b_s;
  const uint32_t dA = a.meta[1], dB = a.meta[2];
  const unsigned long long tiles = a.first[256];
  while (true) {
    if (threadIdx.x == 0) {
      const unsigned long long t = atomicAdd(&a.ctrl->tickets[kTicketMsd2], 1u);
      uint32_t lo = 0, hi = 256;  // the dA bucket of tile t: the last b with first[b] <= t
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (a.first[mid] <= t) lo = mid; else hi = mid;
      }
      t_s = t;
      b_s = lo;
    }
    __syncthreads();
    const unsigned long long t = t_s;
    if (t >= tiles) break;
    const uint32_t b = b_s;
    const uint64_t lo = a.dbase[dA * 256 + b];
    const uint64_t nb = a.hist[dA * 256 + b];
    // group (b, v) starts at gstart[b * 256 + v]: the absolute base of digit value v in this bucket
    radix_tile<R>(sort_buf<R>(a, 3, 1) + lo, sort_buf<R>(a, 3, 2), nb, t - a.first[b], 8 * dB, kTagMsd2,
                  a.status + a.first[b] * 256, a.gstart + b * 256, a.n, a.ctrl);
    __syncthreads();
  }
}

// ---- 5. on-chip sort of every range ----------------------------------------------------------

// Per-warp counts -> per-warp output starts, in place: wc[w][v] becomes the position of warp w's
// first item with digit value v (all items of smaller values first, then those of earlier warps).
__device__ __forceinline__ void local_scan(uint32_t* wc, uint32_t* half, uint32_t* wsum) {
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t v = tid & 255u, h = tid >> 8;  // thread (h, v) covers warps 8h .. 8h+7
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += wc[(h * 8 + j) * 257 + v];
  half[h * 256 + v] = s;
  __syncthreads();
  const uint32_t tot = half[v] + half[256 + v];
  uint32_t incl = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= (uint32_t)o) incl += y;
  }
  if (h == 0 && lane == 31) wsum[warp] = incl;
  __syncthreads();
  uint32_t run = incl - tot + (h ? half[v] : 0u);
  for (uint32_t w = 0; w < (warp & 7u); ++w) run += wsum[w];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint32_t x = wc[(h * 8 + j) * 257 + v];
    wc[(h * 8 + j) * 257 + v] = run;
    run += x;
  }
  __syncthreads();
}

// Ascending bitonic sort of the s <= 32 * EPL words at base, in registers: lane l holds elements
// l * EPL .. l * EPL + EPL - 1, so the stages with partner distance below EPL stay in registers.
// Positions past s hold the largest word, which no entry equals (entries are distinct).
template <typename W, int EPL>
__device__ __forceinline__ void warp_sort(W* base, uint32_t s, uint32_t lane) {
  W v[EPL];
#pragma unroll
  for (int r = 0; r < EPL; ++r) {
    const uint32_t e = lane * EPL + r;
    v[r] = e < s ? base[e] : ~W(0);
  }
#pragma unroll
  for (int kk = 2; kk <= 32 * EPL; kk <<= 1) {
#pragma unroll
    for (int j = kk >> 1; j > 0; j >>= 1) {
      if (j < EPL) {  // partners in the same lane: elements r and r ^ j
#pragma unroll
        for (int r = 0; r < EPL; ++r) {
          if ((r & j) == 0) {
            const bool up = ((lane * EPL + (uint32_t)r) & (uint32_t)kk) == 0;
            const W x = v[r], y = v[r | j];
            const bool sw = (y < x) == up;
            v[r] = sw ? y : x;
            v[r | j] = sw ? x : y;
          }
        }
      } else {  // partners in lane ^ (j / EPL), same r
        const uint32_t lj = (uint32_t)j / EPL;
#pragma unroll
        for (int r = 0; r < EPL; ++r) {
          const W o = __shfl_xor_sync(0xFFFFFFFFu, v[r], lj);
          const bool up = ((lane * EPL + (uint32_t)r) & (uint32_t)kk) == 0;
          const bool keep_min = ((lane & lj) == 0) == up;
          if ((o < v[r]) == keep_min) v[r] = o;
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < EPL; ++r) {
    const uint32_t e = lane * EPL + r;
    if (e < s) base[e] = v[r];
  }
}

// Lanes of the warp with this lane's digit value (0..255, or 256 = no item). A full row of the
// warp has no empty lane, so eight ballots decide it.
__device__ __forceinline__ uint32_t row_peers(uint32_t dg, bool full) {
  return full ? ballot_peers(dg, 8) : ballot_peers(dg, 9);
}

// Per-warp counts of digit d of the keys at positions [wlo, whi) (shared-memory atomics on the warp's
// own counters: counts need no ranks).
template <int R>
__device__ __forceinline__ void local_count(const typename RecT<R>::T* in, uint32_t* wc, uint32_t d, uint32_t wlo,
                                            uint32_t whi, uint32_t lane, uint32_t warp) {
  for (uint32_t b = wlo; b < whi; b += 32) {
    const uint32_t j = b + lane;
    const bool valid = j < whi;
    if (valid) atomicAdd(&wc[warp * 257 + (uint32_t)((load_key<R>(in + j) >> (8 * d)) & 255u)], 1u);
  }
}

// One range of at most kCap records, sorted by key (stable). Fast form: one stable partition of
// the range by its most significant varying digit dC into shared memory, each entry packed as
// (key bits below dC, position) in one key-sized word, then every sub-bucket (at most 256
// entries) sorted by a warp in registers; the packed words are distinct, so that order is the
// stable one. Otherwise (the packed word would not fit, or a sub-bucket is larger): LSD passes
// over the varying digits, alternating between shared memory and the CTA's spill buffers.
template <int R>
__global__ void __launch_bounds__(kLThreads, 1) local_sort_kernel(HybridArgs a) {
  using Rec = typename RecT<R>::T;
  using Key = typename RecT<R>::Key;
  constexpr int D = RecT<R>::kDigits;
  constexpr uint32_t kCap = Local<R>::kCap;
  constexpr uint32_t kU = 8;  // rows of a warp whose loads are in flight together
  const uint32_t mode = a.ctrl->sort_mode;
  if (mode == 0) return;
  extern __shared__ __align__(16) unsigned char lsm[];
  Key* SK = reinterpret_cast<Key*>(lsm);
  uint16_t* SI = reinterpret_cast<uint16_t*>(lsm + kCap * sizeof(Key));
  uint32_t* WC = reinterpret_cast<uint32_t*>(lsm + al16(kCap * (uint32_t)(sizeof(Key) + 2)));
  uint32_t* half = WC + 2 * kLWarps * 257;
  uint32_t* wsum = half + 512;
  Key* red = reinterpret_cast<Key*>(wsum + 8);
  uint32_t* misc = reinterpret_cast<uint32_t*>(red + 2 * kLWarps);
  uint32_t* sub = misc + 4;
  // this CTA's spill buffers: the even LSD passes write them (they stay in L2 for the next pass)
  Key* GK = reinterpret_cast<Key*>(a.scratch + (size_t)blockIdx.x * kCap * (sizeof(Key) + 2));
  uint16_t* GI = reinterpret_cast<uint16_t*>(GK + kCap);
  const Rec* src = sort_buf<R>(a, mode, mode - 1);
  Rec* dst = sort_buf<R>(a, mode, mode);
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t lt_mask = lanemask_lt();
  const uint32_t nbig = a.meta[4];  // this kernel's ranges: those of more than kSmallMax records
  // the digit read 1 counts: the top varying digit of a one-group range under this mode
  const uint32_t dspec = mode == 3 ? D - 3 : mode == 2 ? D - 2 : D - 1;

  while (true) {
    if (tid == 0) misc[0] = atomicAdd(&a.ctrl->tickets[kTicketLocal], 1u);
    __syncthreads();
    const uint32_t ti = misc[0];
    if (ti >= nbig) break;
    const uint32_t r = a.ridx[ti];
    const uint64_t lo = a.gstart[a.rlist[r]];
    const uint64_t m64 = a.gstart[a.rlist[r + 1]] - lo;
    if (m64 == 0 || m64 > kCap) {  // empty; or more than the plan allows (never: the counts bound it)
      if (m64 > kCap && tid == 0) atomicExch(&a.ctrl->bad, 1u);
      __syncthreads();
      continue;
    }
    const uint32_t m = (uint32_t)m64;
    const Rec* in = src + lo;
    Rec* out = dst + lo;
    // warp w orders the positions [w c, (w+1) c) of the current order, c a multiple of 32
    const uint32_t c = ((m + kLWarps - 1) / kLWarps + 31u) & ~31u;
    const uint32_t cmagic = 0xFFFFFFFFu / c + 1u;  // __umulhi(pos, cmagic) = pos / c for pos < 2^16
    const uint32_t wlo = warp * c < m ? warp * c : m, whi = wlo + c < m ? wlo + c : m;
    uint32_t* wc = WC;
    uint32_t* wn = WC + kLWarps * 257;
    for (uint32_t x = tid; x < kLWarps * 257; x += kLThreads) wc[x] = 0;
    __syncthreads();
    // read 1: the key AND / OR over the range, and each warp's counts of digit dspec
    Key kand = ~Key(0), kor = Key(0);
    for (uint32_t b0 = wlo; b0 < whi; b0 += 32 * kU) {
      Key kk[kU];
#pragma unroll
      for (uint32_t u = 0; u < kU; ++u) {
        const uint32_t j = b0 + u * 32 + lane;
        kk[u] = j < whi ? load_key<R>(in + j) : Key(0);
      }
#pragma unroll
      for (uint32_t u = 0; u < kU; ++u) {
        if (b0 + u * 32 >= whi) break;
        const uint32_t j = b0 + u * 32 + lane;
        const bool valid = j < whi;
        if (valid) {
          kand &= kk[u];
          kor |= kk[u];
        }
        // counts only (no ranks): one shared-memory atomic per key on the warp's own counters
        if (valid) atomicAdd(&wc[warp * 257 + (uint32_t)((kk[u] >> (8 * dspec)) & 255u)], 1u);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      kand &= __shfl_xor_sync(0xFFFFFFFFu, kand, o);
      kor |= __shfl_xor_sync(0xFFFFFFFFu, kor, o);
    }
    if (lane == 0) {
      red[warp] = kand;
      red[kLWarps + warp] = kor;
    }
    __syncthreads();
    Key band = ~Key(0), bor = Key(0);
    for (int w = 0; w < kLWarps; ++w) {
      band &= red[w];
      bor |= red[kLWarps + w];
    }
    const Key vary = band ^ bor;
    uint32_t vm = 0;  // digits that vary inside the range
#pragma unroll
    for (int d = 0; d < D; ++d)
      if ((vary >> (8 * d)) & 255u) vm |= 1u << d;
    if (vm == 0) {  // every key equal: the range is already in order
      for (uint32_t j0 = tid; j0 < m; j0 += 4 * kLThreads) {
        Rec v[4];
#pragma unroll
        for (uint32_t u = 0; u < 4; ++u)
          if (j0 + u * kLThreads < m) v[u] = in[j0 + u * kLThreads];
#pragma unroll
        for (uint32_t u = 0; u < 4; ++u)
          if (j0 + u * kLThreads < m) out[j0 + u * kLThreads] = v[u];
      }
      __syncthreads();
      continue;
    }
    uint32_t counted = dspec;  // the digit wc holds counts of
    const uint32_t dC = 31u - (uint32_t)__clz(vm);
    bool fast = 8 * dC + 16 <= 8 * sizeof(Key);
    if (fast) {
      if (dC != counted) {
        for (uint32_t x = tid; x < kLWarps * 257; x += kLThreads) wc[x] = 0;
        __syncthreads();
        local_count<R>(in, wc, dC, wlo, whi, lane, warp);
        __syncthreads();
        counted = dC;
      }
      local_scan(wc, half, wsum);
      // sub-bucket v = [sub[v], sub[v + 1]): warp 0's start of digit value v
      if (tid < 256) sub[tid] = wc[tid];
      if (tid == 0) sub[256] = m;
      const uint32_t tot = tid < 256 ? half[tid] + half[256 + tid] : 0u;
      fast = !__syncthreads_or(tot > kWarpMax);
      counted = 0xFFFFFFFFu;  // wc now holds starts, not counts
    }
    if (fast) {
      // stable partition by dC from the records (the shared keys are overwritten by the packed
      // words): word = (key bits below dC) << 16 | position
      const Key low = (Key)((((unsigned long long)1) << (8 * dC)) - 1ull);
      for (uint32_t b0 = wlo; b0 < whi; b0 += 32 * kU) {
        Key kk[kU];
#pragma unroll
        for (uint32_t u = 0; u < kU; ++u) {
          const uint32_t j = b0 + u * 32 + lane;
          kk[u] = j < whi ? load_key<R>(in + j) : Key(0);
        }
#pragma unroll
        for (uint32_t u = 0; u < kU; ++u) {
          if (b0 + u * 32 >= whi) break;
          const uint32_t j = b0 + u * 32 + lane;
          const bool valid = j < whi;
          const uint32_t dg = valid ? (uint32_t)((kk[u] >> (8 * dC)) & 255u) : 256u;
          const uint32_t peers = row_peers(dg, b0 + u * 32 + 32 <= whi);
          const uint32_t lt = __popc(peers & lt_mask);
          const uint32_t base = wc[warp * 257 + dg];
          __syncwarp();
          if (valid && lt == 0) wc[warp * 257 + dg] = base + __popc(peers);
          __syncwarp();
          if (valid) SK[base + lt] = ((kk[u] & low) << 16) | (Key)j;
        }
      }
      if (tid == 0) misc[1] = 0;
      __syncthreads();
      while (true) {  // warps take sub-buckets as they free up (their sizes differ)
        uint32_t v = 0;
        if (lane == 0) v = atomicAdd(&misc[1], 1u);
        v = __shfl_sync(0xFFFFFFFFu, v, 0);
        if (v >= 256) break;
        const uint32_t s0 = sub[v], sz = sub[v + 1] - s0;
        if (sz <= 1) continue;
        if (sz <= 32) warp_sort<Key, 1>(SK + s0, sz, lane);
        else if (sz <= 64) warp_sort<Key, 2>(SK + s0, sz, lane);
        else if (sz <= 128) warp_sort<Key, 4>(SK + s0, sz, lane);
        else warp_sort<Key, 8>(SK + s0, sz, lane);
      }
      __syncthreads();
      for (uint32_t j0 = tid; j0 < m; j0 += 4 * kLThreads) {
        Rec v[4];
#pragma unroll
        for (uint32_t u = 0; u < 4; ++u)
          if (j0 + u * kLThreads < m) v[u] = in[(uint32_t)(SK[j0 + u * kLThreads] & 0xFFFFu)];
#pragma unroll
        for (uint32_t u = 0; u < 4; ++u)
          if (j0 + u * kLThreads < m) out[j0 + u * kLThreads] = v[u];
      }
      __syncthreads();
      continue;
    }
    // LSD passes over the varying digits. Pass q moves (key, position) from the shared buffers to
    // the spill buffers (q even) or back (q odd), stably by digit d, and counts the next digit for
    // the warp that will read each position.
    for (uint32_t j = tid; j < m; j += kLThreads) {  // keys and positions into shared memory
      SK[j] = load_key<R>(in + j);
      SI[j] = (uint16_t)j;
    }
    uint32_t d = (uint32_t)__ffs(vm) - 1;
    vm &= vm - 1;
    if (d != counted) {
      for (uint32_t x = tid; x < kLWarps * 257; x += kLThreads) wc[x] = 0;
      __syncthreads();
      local_count<R>(in, wc, d, wlo, whi, lane, warp);
    }
    __syncthreads();
    uint32_t q = 0;
    while (true) {
      const bool more = vm != 0;
      const uint32_t dn = more ? (uint32_t)__ffs(vm) - 1 : 0u;
      local_scan(wc, half, wsum);
      if (more) {
        for (uint32_t x = tid; x < kLWarps * 257; x += kLThreads) wn[x] = 0;
        __syncthreads();
      }
      const Key* sk = (q & 1u) ? GK : SK;
      const uint16_t* si = (q & 1u) ? GI : SI;
      Key* dk = (q & 1u) ? SK : GK;
      uint16_t* di = (q & 1u) ? SI : GI;
      for (uint32_t b0 = wlo; b0 < whi; b0 += 32 * kU) {
        Key kk[kU];
        uint32_t ii[kU];
#pragma unroll
        for (uint32_t u = 0; u < kU; ++u) {
          const uint32_t j = b0 + u * 32 + lane;
          kk[u] = j < whi ? sk[j] : Key(0);
          ii[u] = j < whi ? si[j] : 0u;
        }
#pragma unroll
        for (uint32_t u = 0; u < kU; ++u) {
          if (b0 + u * 32 >= whi) break;
          const bool valid = b0 + u * 32 + lane < whi;
          const uint32_t dg = valid ? (uint32_t)((kk[u] >> (8 * d)) & 255u) : 256u;
          const uint32_t peers = row_peers(dg, b0 + u * 32 + 32 <= whi);
          const uint32_t lt = __popc(peers & lt_mask);
          const uint32_t base = wc[warp * 257 + dg];
          __syncwarp();
          if (valid && lt == 0) wc[warp * 257 + dg] = base + __popc(peers);
          __syncwarp();
          if (valid) {
            const uint32_t pos = base + lt;
            dk[pos] = kk[u];
            di[pos] = (uint16_t)ii[u];
            if (more)
              atomicAdd(&wn[__umulhi(pos, cmagic) * 257 + (uint32_t)((kk[u] >> (8 * dn)) & 255u)], 1u);
          }
        }
      }
      __syncthreads();
      ++q;
      if (!more) break;
      uint32_t* t = wc;
      wc = wn;
      wn = t;
      d = dn;
      vm &= vm - 1;
    }
    // gather the records in key order: the last pass (q - 1) wrote the spill buffers when q - 1
    // is even, the shared ones when it is odd
    const uint16_t* fi = ((q - 1) & 1u) ? SI : GI;
    for (uint32_t j0 = tid; j0 < m; j0 += 4 * kLThreads) {
      Rec v[4];
#pragma unroll
      for (uint32_t u = 0; u < 4; ++u)
        if (j0 + u * kLThreads < m) v[u] = in[fi[j0 + u * kLThreads]];
#pragma unroll
      for (uint32_t u = 0; u < 4; ++u)
        if (j0 + u * kLThreads < m) out[j0 + u * kLThreads] = v[u];
    }
    __syncthreads();
  }
}

// Ascending bitonic sort of (key, position) pairs in registers, the same network as warp_sort:
// lane l holds elements l * EPL .. l * EPL + EPL - 1. Positions are distinct; padding is the
// largest pair. The stage loops stay rolled (one body per partner distance below EPL and one for
// the distances across lanes), so the code of every size fits the instruction cache.
template <typename Key>
__device__ __forceinline__ bool pair_less(Key ka, uint32_t xa, Key kb, uint32_t xb) {
  return ka < kb || (ka == kb && xa < xb);
}

template <typename Key, int EPL, int J>
__device__ __forceinline__ void pair_stage_lane(Key (&k)[EPL], uint32_t (&x)[EPL], uint32_t lane, uint32_t kk) {
  if constexpr (J < EPL) {
#pragma unroll
    for (int r = 0; r < EPL; ++r) {
      if ((r & J) == 0) {
        const bool up = ((lane * EPL + (uint32_t)r) & kk) == 0;
        const bool sw = pair_less(k[r | J], x[r | J], k[r], x[r]) == up;
        const Key tk = k[r];
        const uint32_t tx = x[r];
        k[r] = sw ? k[r | J] : k[r];
        x[r] = sw ? x[r | J] : x[r];
        k[r | J] = sw ? tk : k[r | J];
        x[r | J] = sw ? tx : x[r | J];
      }
    }
  }
}

template <typename Key, int EPL>
__device__ __forceinline__ void pair_stage_cross(Key (&k)[EPL], uint32_t (&x)[EPL], uint32_t lane, uint32_t kk,
                                                 uint32_t lj) {
#pragma unroll
  for (int r = 0; r < EPL; ++r) {
    const Key ok = __shfl_xor_sync(0xFFFFFFFFu, k[r], lj);
    const uint32_t ox = __shfl_xor_sync(0xFFFFFFFFu, x[r], lj);
    const bool up = ((lane * EPL + (uint32_t)r) & kk) == 0;
    const bool keep_min = ((lane & lj) == 0) == up;
    if (pair_less(ok, ox, k[r], x[r]) == keep_min) {
      k[r] = ok;
      x[r] = ox;
    }
  }
}

template <typename Key, int EPL>
__device__ __forceinline__ void warp_sort_pairs(Key (&k)[EPL], uint32_t (&x)[EPL], uint32_t lane) {
#pragma unroll 1
  for (uint32_t kk = 2; kk <= 32u * EPL; kk <<= 1) {
#pragma unroll 1
    for (uint32_t j = kk >> 1; j > 0; j >>= 1) {
      if (j >= (uint32_t)EPL) pair_stage_cross<Key, EPL>(k, x, lane, kk, j / EPL);
      else if (j == 1) pair_stage_lane<Key, EPL, 1>(k, x, lane, kk);
      else if (j == 2) pair_stage_lane<Key, EPL, 2>(k, x, lane, kk);
      else if (j == 4) pair_stage_lane<Key, EPL, 4>(k, x, lane, kk);
      else if (j == 8) pair_stage_lane<Key, EPL, 8>(k, x, lane, kk);
      else pair_stage_lane<Key, EPL, 16>(k, x, lane, kk);
    }
  }
}

// One range of m <= 32 * EPL records sorted by one warp: keys and positions into registers (in
// any arrangement: the network sorts them all), sorted, the order through shared memory, then the
// records gathered into place with coalesced writes.
template <int R, int EPL>
__device__ __forceinline__ void small_range(const typename RecT<R>::T* in, typename RecT<R>::T* out, uint32_t m,
                                            uint16_t* sidx, uint32_t lane) {
  using Key = typename RecT<R>::Key;
  Key k[EPL];
  uint32_t x[EPL];
#pragma unroll
  for (int r = 0; r < EPL; ++r) {
    const uint32_t e = (uint32_t)r * 32 + lane;
    k[r] = e < m ? load_key<R>(in + e) : ~Key(0);
    x[r] = e < m ? e : 0xFFFFFFFFu;
  }
  warp_sort_pairs<Key, EPL>(k, x, lane);
#pragma unroll
  for (int r = 0; r < EPL; ++r) {
    const uint32_t e = lane * EPL + (uint32_t)r;
    if (e < m) sidx[e] = (uint16_t)x[r];
  }
  __syncwarp();
  for (uint32_t e = lane; e < m; e += 32) out[e] = in[sidx[e]];
  __syncwarp();
}

// The ranges of at most kSmallMax records (many small groups: n between about 2^22 and 2^28 for
// 16-byte records), a warp each, taken by ticket; no block-wide barrier. Two launches share the
// list: BIG = false sorts the ranges of at most 512 records (16 pairs per lane at most, so more
// warps fit an SM), BIG = true those of 513 to 1024 (32 pairs per lane).
template <int R, bool BIG>
__global__ void __launch_bounds__(kSThreads) local_small_kernel(HybridArgs a) {
  using Rec = typename RecT<R>::T;
  constexpr uint32_t kMax = BIG ? 1024u : 512u;
  const uint32_t mode = a.ctrl->sort_mode;
  if (mode == 0) return;
  __shared__ uint16_t sidx[kSThreads / 32][kMax];
  const Rec* src = sort_buf<R>(a, mode, mode - 1);
  Rec* dst = sort_buf<R>(a, mode, mode);
  const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
  const uint32_t nsmall = a.meta[5];
  while (true) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(&a.ctrl->tickets[BIG ? kTicketSmall + 1 : kTicketSmall], 1u);
    t = __shfl_sync(0xFFFFFFFFu, t, 0);
    if (t >= nsmall) break;
    const uint32_t r = a.ridx[kRangeList + t];
    const uint64_t lo = a.gstart[a.rlist[r]];
    const uint64_t m64 = a.gstart[a.rlist[r + 1]] - lo;
    if (m64 > kSmallMax) {  // never: the plan lists only small ranges here
      if (lane == 0) atomicExch(&a.ctrl->bad, 1u);
      continue;
    }
    const uint32_t m = (uint32_t)m64;
    if (m == 0 || (m > 512) != BIG) continue;  // the other launch's range
    if constexpr (BIG) {
      small_range<R, 32>(src + lo, dst + lo, m, sidx[w], lane);
    } else {
      if (m <= 32) small_range<R, 1>(src + lo, dst + lo, m, sidx[w], lane);
      else if (m <= 64) small_range<R, 2>(src + lo, dst + lo, m, sidx[w], lane);
      else if (m <= 128) small_range<R, 4>(src + lo, dst + lo, m, sidx[w], lane);
      else if (m <= 256) small_range<R, 8>(src + lo, dst + lo, m, sidx[w], lane);
      else small_range<R, 16>(src + lo, dst + lo, m, sidx[w], lane);
    }
  }
}

int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return sms;
}

template <int R>
cudaError_t launch_r(const HybridArgs& a, int stage, cudaStream_t st) {
  constexpr int D = RecT<R>::kDigits;
  cudaError_t e = cudaSuccess;
  const int sms = device_sms();
  if (sms <= 0) return cudaErrorInvalidDevice;
  switch (stage) {
    case 0: {
      const uint32_t smem = (D * 256 + kGroups / 2) * 4;
      if ((e = cudaFuncSetAttribute(hybrid_hist_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
          cudaSuccess)
        return e;
      const uint64_t need = (a.n + kJThreads - 1) / kJThreads;
      const unsigned grid = (unsigned)(need < (uint64_t)sms ? (need ? need : 1) : (uint64_t)sms);
      hybrid_hist_kernel<R><<<grid, kJThreads, smem, st>>>(a);
      break;
    }
    case 1:
      sort_plan_kernel<R><<<1, kPlanThreads, 0, st>>>(a);
      break;
    case 2:
    case 3: {
      const uint32_t smem = radix_tile_smem<R>();
      const uint64_t tiles = radix_tiles(a.n, R) + (stage == 3 ? 256u : 0u);  // upper bound for stage 3
      const unsigned grid = (unsigned)(tiles < 2ull * sms ? tiles : 2ull * sms);  // two CTAs per SM
      if (stage == 2) {
        if ((e = set_smem_optin(msd1_kernel<R>)) != cudaSuccess) return e;
        msd1_kernel<R><<<grid, kThreads, smem, st>>>(a);
      } else {
        if ((e = set_smem_optin(msd2_kernel<R>)) != cudaSuccess) return e;
        msd2_kernel<R><<<grid, kThreads, smem, st>>>(a);
      }
      break;
    }
    default: {
      local_small_kernel<R, false><<<(unsigned)sms * 8, kSThreads, 0, st>>>(a);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      local_small_kernel<R, true><<<(unsigned)sms * 4, kSThreads, 0, st>>>(a);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      const uint32_t smem = local_smem_bytes<R>();
      if ((e = cudaFuncSetAttribute(local_sort_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
          cudaSuccess)
        return e;
      const unsigned grid = a.local_ctas < (uint32_t)sms ? a.local_ctas : (unsigned)sms;
      local_sort_kernel<R><<<grid, kLThreads, smem, st>>>(a);
      break;
    }
  }
  return cudaGetLastError();
}

}  // namespace

uint32_t hybrid_local_ctas(uint64_t n, int R) {
  const uint64_t cap = R == 8 ? Local<8>::kCap : Local<16>::kCap;
  const uint64_t want = (n + cap / 2 - 1) / (cap / 2);
  return (uint32_t)(want < 1 ? 1 : want > kLocalMaxCtas ? kLocalMaxCtas : want);
}

size_t hybrid_spill_bytes(uint64_t n, int R) {
  const size_t per = R == 8 ? (size_t)Local<8>::kCap * 6 : (size_t)Local<16>::kCap * 10;
  return per * hybrid_local_ctas(n, R);
}

uint32_t hybrid_cap(int R) { return R == 8 ? Local<8>::kCap : Local<16>::kCap; }

cudaError_t launch_hybrid(const HybridArgs& a, int R, int stage, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  return R == 8 ? launch_r<8>(a, stage, st) : launch_r<16>(a, stage, st);
}

}  // namespace bos
