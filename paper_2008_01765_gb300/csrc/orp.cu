// Bucket ORP passes (Algorithm 3.1 + Section 3.2) for sm_103a.
//
// One kernel template runs one HBM pass that applies k consecutive butterfly levels
// i .. i+k-1 of Algorithm 3.1. Level i pairs bucket j'+j with j'+j+2^i and routes on label bit
// L-1-i; k consecutive levels decompose into B/2^k independent subproblems. Subproblem
// q = G*2^i + t reads the 2^k buckets G*2^(i+k) + s*2^i + t (s < 2^k, stride 2^i, Z slots each)
// and writes the 2^k contiguous buckets q*2^k + u (u < 2^k), where u is label bits
// [L-1-i .. L-i-k]. Inside a bucket the order is stable: reals by (s, slot), then dummies, so
// the result equals k applications of the stable MergeSplit. With k = 1 this is the plain form
// (one level per launch).
//
// The CTA holds the 2^k output buckets in shared memory (the paper's private client storage,
// Section 3.1). Every global access of the pass has an address that depends only on
// (n, Z, k, i, q): whole input buckets are read, whole output buckets are written. The
// label-dependent movement happens in shared memory only.
//
// FIRST pass: the input buckets are the groups of the input array (Algorithm 3.1, "evenly
// divide X into B groups ... pad with dummies"); labels are drawn here from Philox stream 0.
// LAST pass: the routed final buckets are permuted in place (Section 3.2: "randomly permute each
// bucket ... incorporated with the last level", Section 3.4), dummies are dropped, and the reals
// are written contiguously at the prefix of the final loads, found by decoupled look-back over
// the subproblems (the loads depend on the labels only, never on the data, Lemma 3.3).
//
// Overflow (Algorithm 3.1, MergeSplit: more than Z reals in an output bucket) is checked for
// every level inside the pass from per-input-bucket digit counts, and raises ctrl->overflow.
#include "common.cuh"
#include "internal.h"

namespace bos {

namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 4;
constexpr int kChunk = kThreads * kItems;
constexpr int kPermWarps = 8;  // warps that build the in-bin permutations in the LAST pass

struct SmemLayout {
  uint32_t tile_rec, tile_tag, wcnt, base, hist, inv, perm, perm_stride, moff, misc, total;
};

__host__ __device__ inline uint32_t align_up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

// Per-warp scratch of the in-bin permutation: 256 bin starts + 256 bin cursors (u32) and Z
// member slots (u16); the stride is rounded to 16 bytes so every warp's u32 arrays stay aligned
// for any Z.
__host__ __device__ inline uint32_t perm_stride(uint32_t Z) { return align_up(2 * 256 * 4 + Z * 2, 16); }

__host__ __device__ inline SmemLayout smem_layout(int R, uint32_t Z, uint32_t k, bool last) {
  SmemLayout l{};
  const uint32_t D = 1u << k;
  const uint32_t S = D * Z;
  uint32_t off = 0;
  l.tile_rec = off; off = align_up(off + S * R, 16);
  l.tile_tag = off; off = align_up(off + S * 4, 16);
  l.wcnt = off;     off = align_up(off + 2 * kWarps * (D + 1) * 4, 16);  // double-buffered
  l.base = off;     off = align_up(off + (D + 1) * 4, 16);
  l.hist = off;     off = align_up(off + D * D * 4, 16);
  if (last) {
    l.inv = off;  off = align_up(off + S * 2, 16);
    l.perm_stride = perm_stride(Z);
    l.perm = off; off = align_up(off + kPermWarps * l.perm_stride, 16);
    l.moff = off; off = align_up(off + (D + 1) * 4, 16);
  }
  l.misc = off; off = align_up(off + 64, 16);
  l.total = off;
  return l;
}

template <int R>
__device__ __forceinline__ void load_rec(typename RecT<R>::T& dst, const void* base, uint64_t idx) {
  dst = reinterpret_cast<const typename RecT<R>::T*>(base)[idx];
}

// One subproblem q of one pass (the whole CTA).
template <int R, int MODE, bool TRACE>
__device__ __forceinline__ void orp_pass_body(const PassArgs& a, uint64_t q) {
  using Rec = typename RecT<R>::T;
  constexpr bool FIRST = MODE & kModeFirst;
  constexpr bool LAST = MODE & kModeLast;
  extern __shared__ __align__(16) unsigned char smem[];

  const uint32_t Z = a.Z, k = a.k, D = 1u << k;
  const uint32_t S = D * Z;
  const SmemLayout lay = smem_layout(R, Z, k, LAST);
  Rec* tile_rec = reinterpret_cast<Rec*>(smem + lay.tile_rec);
  uint32_t* tile_tag = reinterpret_cast<uint32_t*>(smem + lay.tile_tag);
  uint32_t* wcnt = reinterpret_cast<uint32_t*>(smem + lay.wcnt);  // [2][kWarps][D+1]
  uint32_t* base = reinterpret_cast<uint32_t*>(smem + lay.base);  // [D+1] running digit counts
  uint32_t* hist = reinterpret_cast<uint32_t*>(smem + lay.hist);  // [D][D] input bucket x digit
  uint32_t* misc = reinterpret_cast<uint32_t*>(smem + lay.misc);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t wstride = D + 1;

  const uint32_t i = a.i;
  const uint64_t t = q & ((1ull << i) - 1);
  const uint64_t G = q >> i;
  const uint32_t shift = a.L - i - k;  // routing digit = label bits [shift, shift+k)

  for (uint32_t x = tid; x < 2 * kWarps * wstride; x += kThreads) wcnt[x] = 0;
  for (uint32_t x = tid; x <= D; x += kThreads) base[x] = 0;
  for (uint32_t x = tid; x < D * D; x += kThreads) hist[x] = 0;
  __syncthreads();

  const uint32_t lt_mask = lanemask_lt();
  int buf = 0;
  for (uint32_t cbase = 0; cbase < S; cbase += kChunk, buf ^= 1) {
    uint32_t* wc = wcnt + buf * kWarps * wstride;
    uint32_t* wc_other = wcnt + (buf ^ 1) * kWarps * wstride;
    Rec rc[kItems];
    uint32_t tg[kItems], rk[kItems], dg[kItems];
    // ---- load kItems slots per thread: warp-contiguous, lane-striped positions ----
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
      const uint32_t p = cbase + warp * 32 * kItems + it * 32 + lane;
      tg[it] = kDummy;
      rc[it] = RecT<R>::zero();
      if (p < S) {
        const uint32_t s = p / Z, sl = p - s * Z;
        if constexpr (FIRST) {
          const uint64_t j = a.bucket0 + q * D + s;  // group index (i = 0); B = 2^L
          const uint64_t lo = (j * a.n) >> a.L, hi = ((j + 1) * a.n) >> a.L;
          if (lo + sl < hi) {
            const uint64_t idx = lo + sl;
            load_rec<R>(rc[it], a.in, idx);
            trace_log<TRACE>(a.trace, kRead, kBufIn, R, idx * R);
            tg[it] = label_of(idx, a.seed, a.attempt, a.L);
          }
        } else {
          const uint64_t bucket = (G << (i + k)) + ((uint64_t)s << i) + t;
          const uint64_t off = bucket * Z + sl;
          tg[it] = a.in_tag[off];
          load_rec<R>(rc[it], a.in_rec, off);
          trace_log<TRACE>(a.trace, kRead, a.buf_in_tag, 4, off * 4);
          trace_log<TRACE>(a.trace, kRead, a.buf_in_rec, R, off * R);
        }
      }
    }
    // ---- stable rank within the warp per digit (match + running per-warp counters) ----
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
      const uint32_t p = cbase + warp * 32 * kItems + it * 32 + lane;
      const bool real = tg[it] != kDummy;
      const uint32_t u = real ? ((tg[it] >> shift) & (D - 1)) : D;
      dg[it] = u;
      const uint32_t peers = __match_any_sync(0xFFFFFFFFu, u);
      const uint32_t lt = __popc(peers & lt_mask);
      rk[it] = wc[warp * wstride + u] + lt;
      const uint32_t s_loc = (p < S) ? p / Z : 0;
      const uint32_t key2 = real ? s_loc * D + u : 0xFFFFFFFFu;
      const uint32_t peers2 = __match_any_sync(0xFFFFFFFFu, key2);
      __syncwarp();
      if (lt == 0) wc[warp * wstride + u] += __popc(peers);
      if (real && (peers2 & lt_mask) == 0) atomicAdd(&hist[key2], (uint32_t)__popc(peers2));
      __syncwarp();
    }
    __syncthreads();
    // ---- exclusive offsets over warps per digit; advance running counts; clear other buffer ----
    for (uint32_t d = tid; d < D; d += kThreads) {
      uint32_t run = base[d];
      for (int w = 0; w < kWarps; ++w) {
        const uint32_t x = wc[w * wstride + d];
        wc[w * wstride + d] = run;
        run += x;
      }
      base[d] = run;
    }
    for (uint32_t x = tid; x < kWarps * wstride; x += kThreads) wc_other[x] = 0;
    __syncthreads();
    // ---- scatter into the output tile (shared memory) ----
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
      if (tg[it] != kDummy) {
        const uint32_t u = dg[it];
        const uint32_t dest = wc[warp * wstride + u] + rk[it];
        if (dest < Z) {
          tile_rec[u * Z + dest] = rc[it];
          tile_tag[u * Z + dest] = tg[it];
        }
      }
    }
  }
  __syncthreads();

  // ---- overflow: every bucket of levels i+1 .. i+k inside this subproblem ----
  // level i+l bucket (sigma, pi): inputs s in [sigma 2^l, (sigma+1) 2^l), digits with prefix pi.
  for (uint32_t x = tid; x < k * D; x += kThreads) {
    const uint32_t l = x / D + 1, bkt = x % D;
    const uint32_t sigma = bkt >> l, pi = bkt & ((1u << l) - 1);
    uint32_t c = 0;
    for (uint32_t s = sigma << l; s < ((sigma + 1) << l); ++s)
      for (uint32_t u = pi << (k - l); u < ((pi + 1) << (k - l)); ++u) c += hist[s * D + u];
    if (c > Z) atomicExch(&a.ctrl->overflow, 1u);
  }

  if constexpr (!LAST) {
    // ---- pad with dummies, write the 2^k output buckets (contiguous) ----
    for (uint32_t x = tid; x < S; x += kThreads) {
      const uint32_t u = x / Z, sl = x - u * Z;
      if (sl >= base[u]) {
        tile_tag[x] = kDummy;
        tile_rec[x] = RecT<R>::zero();
      }
    }
    __syncthreads();
    Rec* out_rec = reinterpret_cast<Rec*>(a.out_rec) + q * S;
    uint32_t* out_tag = a.out_tag + q * S;
    for (uint32_t x = tid; x < S; x += kThreads) {
      out_rec[x] = tile_rec[x];
      out_tag[x] = tile_tag[x];
      trace_log<TRACE>(a.trace, kWrite, a.buf_out_rec, R, (q * S + x) * R);
      trace_log<TRACE>(a.trace, kWrite, a.buf_out_tag, 4, (q * S + x) * 4);
    }
  } else {
    // ---- Section 3.2: in-bin permutation of every final bucket b = q*2^k + u ----
    uint16_t* inv = reinterpret_cast<uint16_t*>(smem + lay.inv);
    uint32_t* moff = reinterpret_cast<uint32_t*>(smem + lay.moff);
    if (warp < kPermWarps) {
      unsigned char* pw = smem + lay.perm + warp * lay.perm_stride;
      uint32_t* bin_start = reinterpret_cast<uint32_t*>(pw);
      uint32_t* bin_cur = bin_start + 256;
      uint16_t* members = reinterpret_cast<uint16_t*>(bin_cur + 256);
      for (uint32_t u = warp; u < D; u += kPermWarps) {
        const uint32_t m = min(base[u], Z);
        const uint64_t b = a.bucket0 + q * D + u;  // global bucket: the key's counter
        uint32_t* rhi = tile_tag + u * Z;  // tags are dead in the last pass: reuse as key store
        for (int x = lane; x < 256; x += 32) bin_cur[x] = 0;
        __syncwarp();
        for (uint32_t s = lane; s < m; s += 32) {
          const uint32_t h = philox_at(b * Z + s, a.attempt, 1, a.seed).w0;
          rhi[s] = h;
          atomicAdd(&bin_cur[h >> 24], 1u);
        }
        __syncwarp();
        // exclusive scan over 256 bins: lane owns bins [8 lane, 8 lane + 8)
        uint32_t v[8], sum = 0;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          v[e] = bin_cur[lane * 8 + e];
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
        for (int e = 0; e < 8; ++e) {
          bin_start[lane * 8 + e] = run;
          bin_cur[lane * 8 + e] = run;
          run += v[e];
        }
        __syncwarp();
        for (uint32_t s = lane; s < m; s += 32) {
          const uint32_t pos = atomicAdd(&bin_cur[rhi[s] >> 24], 1u);
          members[pos] = (uint16_t)s;
        }
        __syncwarp();
        for (uint32_t s = lane; s < m; s += 32) {
          const uint32_t h = rhi[s], bin = h >> 24;
          const uint32_t st = bin_start[bin], en = bin_cur[bin];
          uint32_t r = st;
          for (uint32_t x = st; x < en; ++x) {
            const uint32_t s2 = members[x];
            if (s2 == s) continue;
            const uint32_t h2 = rhi[s2];
            bool less = h2 < h;
            if (h2 == h) {  // equal high words: compare the low words, then the slot
              const uint32_t l1 = philox_at(b * Z + s, a.attempt, 1, a.seed).w1;
              const uint32_t l2 = philox_at(b * Z + s2, a.attempt, 1, a.seed).w1;
              less = (l2 < l1) || (l2 == l1 && s2 < s);
            }
            r += less;
          }
          inv[u * Z + r] = (uint16_t)s;
        }
        __syncwarp();
      }
    }
    if (tid == 0) {
      uint32_t run = 0;
      for (uint32_t u = 0; u < D; ++u) {
        moff[u] = run;
        run += min(base[u], Z);
      }
      moff[D] = run;
      // decoupled look-back for this subproblem's output offset
      const unsigned long long total = run;
      unsigned long long prefix = 0;
      const bool skip = a.skip_publish && q == 0;
      if (q == 0) {
        if (!skip) st_status(a.status, st_word(kStIncl, 0, total));
      } else {
        st_status(a.status + q, st_word(kStAgg, 0, total));
        prefix = lookback_window<8>(a.status, q, 1, 0, a.ctrl);
        st_status(a.status + q, st_word(kStIncl, 0, prefix + total));
      }
      misc[1] = (uint32_t)prefix;
      misc[2] = (uint32_t)(prefix >> 32);
    }
    __syncthreads();
    const uint64_t prefix = (uint64_t)misc[1] | ((uint64_t)misc[2] << 32);
    const uint32_t total = moff[D];
    Rec* out = reinterpret_cast<Rec*>(a.out0);
    if (a.out_sel && sort_passes_odd(a.ctrl)) out = reinterpret_cast<Rec*>(a.out1);
    const uint32_t out_buf = (out == reinterpret_cast<Rec*>(a.out0)) ? kBufOut : kBufTmp;
    for (uint32_t j = tid; j < total; j += kThreads) {
      // bucket u with moff[u] <= j < moff[u+1] (binary search over D+1 offsets)
      uint32_t lo = 0, hi = D;
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (moff[mid] <= j) lo = mid; else hi = mid;
      }
      const uint32_t s = inv[lo * Z + (j - moff[lo])];
      if (prefix + j < a.n) {
        out[prefix + j] = tile_rec[lo * Z + s];
        trace_log<TRACE>(a.trace, kWrite, out_buf, R, (prefix + j) * R);
      }
    }
  }
}

// Single array: one CTA per subproblem; the LAST pass takes subproblems by ticket so that every
// look-back predecessor has already started (no CTA waits on one that is not yet resident).
template <int R, int MODE, bool TRACE>
__global__ void __launch_bounds__(kThreads, 1) orp_pass_kernel(PassArgs a) {
  __shared__ unsigned long long q_s;
  uint64_t q = blockIdx.x;
  if constexpr ((MODE & kModeLast) != 0) {
    if (threadIdx.x == 0) q_s = atomicAdd(&a.ctrl->tickets[a.ticket_slot], 1u);
    __syncthreads();
    q = q_s;
  }
  orp_pass_body<R, MODE, TRACE>(a, q);
}

// Many arrays in one launch: block (or ticket) b is subproblem b - first[j] of array j, where
// first[] holds the running sum of the arrays' subproblem counts. LAST passes take tickets over
// the whole launch, so inside every array the subproblems start in order.
template <int R, int MODE, bool TRACE>
__global__ void __launch_bounds__(kThreads, 1) orp_pass_batched_kernel(BatchPass bp) {
  __shared__ unsigned long long q_s;
  __shared__ uint32_t j_s;
  if (threadIdx.x == 0) {
    const uint64_t t = (MODE & kModeLast) ? (uint64_t)atomicAdd(bp.ticket, 1u) : (uint64_t)blockIdx.x;
    uint32_t lo = 0, hi = bp.narr;  // largest j with first[j] <= t
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (bp.first[mid] <= t) lo = mid; else hi = mid;
    }
    j_s = lo;
    q_s = t - bp.first[lo];
  }
  __syncthreads();
  const PassArgs a = bp.args[j_s];
  orp_pass_body<R, MODE, TRACE>(a, q_s);
}

}  // namespace

uint32_t orp_smem_bytes(int R, uint32_t Z, uint32_t k, bool last) {
  return smem_layout(R, Z, k, last).total;
}

template <int R, int MODE, bool TRACE>
static cudaError_t launch_mode(const PassArgs& a, uint64_t grid, cudaStream_t st) {
  const uint32_t smem = smem_layout(R, a.Z, a.k, MODE & kModeLast).total;
  auto kern = orp_pass_kernel<R, MODE, TRACE>;
  cudaError_t e = set_smem_optin(kern);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <int R, bool TRACE>
static cudaError_t launch_r(const PassArgs& a, int mode, uint64_t grid, cudaStream_t st) {
  switch (mode) {
    case 0: return launch_mode<R, 0, TRACE>(a, grid, st);
    case kModeFirst: return launch_mode<R, kModeFirst, TRACE>(a, grid, st);
    case kModeLast: return launch_mode<R, kModeLast, TRACE>(a, grid, st);
    default: return launch_mode<R, kModeFirst | kModeLast, TRACE>(a, grid, st);
  }
}

template <int R, int MODE, bool TRACE>
static cudaError_t batched_mode(const BatchPass& bp, uint32_t smem, cudaStream_t st) {
  auto kern = orp_pass_batched_kernel<R, MODE, TRACE>;
  cudaError_t e = set_smem_optin(kern);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)bp.nblocks, kThreads, smem, st>>>(bp);
  return cudaGetLastError();
}

template <int R, bool TRACE>
static cudaError_t batched_r(const BatchPass& bp, int mode, uint32_t smem, cudaStream_t st) {
  switch (mode) {
    case 0: return batched_mode<R, 0, TRACE>(bp, smem, st);
    case kModeFirst: return batched_mode<R, kModeFirst, TRACE>(bp, smem, st);
    case kModeLast: return batched_mode<R, kModeLast, TRACE>(bp, smem, st);
    default: return batched_mode<R, kModeFirst | kModeLast, TRACE>(bp, smem, st);
  }
}

cudaError_t launch_orp_pass_batched(const BatchPass& bp, int mode, uint32_t smem, cudaStream_t st, int R,
                                    bool trace) {
  if (bp.nblocks == 0) return cudaSuccess;
  if (R == 8) return trace ? batched_r<8, true>(bp, mode, smem, st) : batched_r<8, false>(bp, mode, smem, st);
  return trace ? batched_r<16, true>(bp, mode, smem, st) : batched_r<16, false>(bp, mode, smem, st);
}

cudaError_t launch_orp_pass(const PassArgs& a, int mode, uint64_t grid, cudaStream_t st, int R, bool trace) {
  if (R == 8) return trace ? launch_r<8, true>(a, mode, grid, st) : launch_r<8, false>(a, mode, grid, st);
  return trace ? launch_r<16, true>(a, mode, grid, st) : launch_r<16, false>(a, mode, grid, st);
}

}  // namespace bos
