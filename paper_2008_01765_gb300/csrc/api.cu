// C ABI of libbos (declared in include/bos.h): argument checks, pass planning, workspace layout
// and the attempt loop of Algorithm 3.1 (retry with a fresh attempt counter on overflow).
#include <atomic>
#include <cstring>
#include <mutex>
#include <utility>
#include <vector>

#include "bos.h"
#include "internal.h"

namespace bos {
namespace {

constexpr uint32_t kMaxSmem = 232448 - 1024;  // opt-in shared memory per CTA (sm_100/103) less static use
constexpr uint32_t kMaxK = 6;          // per-pass digit-count table is (2^k)^2 words
constexpr uint32_t kMaxPasses = 32;
constexpr uint32_t kMaxLevels = 32;  // L < 32: slot indexes are 32-bit
constexpr uint32_t kDefaultAttempts = 8;

// Process-wide debug state. The trace buffer is read once per call under g_state_mu, so an
// attach from one thread never tears a call's copy; the profiling events and totals are updated
// under the same mutex and the launch counter is atomic, so calls from several host threads
// (the serving loop's workers) are safe while profiling is on (their launches are then timed in
// whatever order the threads record them).
std::mutex g_state_mu;
Trace g_trace{nullptr, 0, 0};
Trace trace_snapshot() {
  std::lock_guard<std::mutex> g(g_state_mu);
  return g_trace;
}

// ---- opt-in kernel timing (bos_profile_enable / bos_profile_read) ----
enum KClass { kKFirst, kKMid, kKLast, kKSingle, kKHist, kKPrep, kKRadix, kKRadixSkipped, kKBitonic, kKPerm,
              kKMergeBlock, kKMerge, kKOblivious, kKMsd, kKLocal, kKCount };
const char* const kKNames[kKCount] = {"orp_pass_first", "orp_pass_mid", "orp_pass_last", "orp_pass_single",
                                     "radix_hist", "radix_prep", "radix_pass", "radix_pass_skipped",
                                     "bitonic", "perm_table", "merge_block", "merge_pass", "orp_oblivious",
                                     "sort_partition", "sort_local"};
constexpr int kMaxEv = 1024;
struct Prof {
  std::atomic<bool> on{false};
  bool created = false;
  cudaEvent_t ev[2 * kMaxEv];
  int pending = 0;
  int cls[kMaxEv];
  double bytes[kMaxEv];
  uint32_t digit[kMaxEv];
  uint64_t launches[kKCount] = {};
  double ms[kKCount] = {};
  double alg_bytes[kKCount] = {};
  std::atomic<uint64_t> total_launches{0};
};
Prof g_prof;

// Zeroes bytes at p on stream st with a kernel. The library's workspace resets are kernels, not
// cudaMemsetAsync: a memset can wait behind a large copy that another stream has in flight (the
// next step's input or the previous step's output in a pipelined caller).
__global__ void zero_kernel(unsigned char* p, size_t bytes) {
  const size_t head0 = (16 - ((uintptr_t)p & 15)) & 15;
  const size_t head = head0 < bytes ? head0 : bytes;
  const size_t body = (bytes - head) / 16;
  uint4* q = reinterpret_cast<uint4*>(p + head);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < body; i += (size_t)gridDim.x * blockDim.x)
    q[i] = make_uint4(0, 0, 0, 0);
  if (blockIdx.x == 0 && threadIdx.x < 16) {
    if (threadIdx.x < head) p[threadIdx.x] = 0;
    const size_t t = head + body * 16 + threadIdx.x;
    if (t < bytes) p[t] = 0;
  }
}

// Records an event pair around one launch when profiling is on. Returns the slot or -1.
int prof_begin(cudaStream_t st, int cls, double bytes, uint32_t digit = 0) {
  g_prof.total_launches.fetch_add(1, std::memory_order_relaxed);
  if (!g_prof.on) return -1;
  std::lock_guard<std::mutex> g(g_state_mu);
  if (!g_prof.on || g_prof.pending >= kMaxEv) return -1;
  const int i = g_prof.pending++;
  g_prof.cls[i] = cls;
  g_prof.bytes[i] = bytes;
  g_prof.digit[i] = digit;
  cudaEventRecord(g_prof.ev[2 * i], st);
  return i;
}
void prof_end(int i, cudaStream_t st) {
  if (i >= 0) cudaEventRecord(g_prof.ev[2 * i + 1], st);
}
// Launches that run inside another launch's profile event still count as launches.
void count_launches(uint64_t k) { g_prof.total_launches.fetch_add(k, std::memory_order_relaxed); }

cudaError_t zero_async(void* p, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return cudaSuccess;
  const size_t words = bytes / 16 + 1;
  const size_t blocks = (words + 255) / 256;
  const unsigned grid = (unsigned)(blocks < 4096 ? blocks : 4096);
  g_prof.total_launches.fetch_add(1, std::memory_order_relaxed);
  zero_kernel<<<grid, 256, 0, st>>>(static_cast<unsigned char*>(p), bytes);
  return cudaGetLastError();
}
// Folds the finished event pairs into the per-class totals (the stream has been synchronised).
// A launch that returned at once (a constant digit; the LSD passes when the hybrid sort ran; a
// hybrid stage its mode does not run) counts as a skipped radix pass.
void prof_collect(uint32_t radix_live, uint32_t sort_mode) {
  std::lock_guard<std::mutex> g(g_state_mu);
  int keep = 0;  // pairs whose end has not been reached yet (another thread's stream) stay pending
  for (int i = 0; i < g_prof.pending; ++i) {
    float ms = 0.f;
    const cudaError_t e = cudaEventElapsedTime(&ms, g_prof.ev[2 * i], g_prof.ev[2 * i + 1]);
    if (e == cudaErrorNotReady) {
      (void)cudaGetLastError();
      std::swap(g_prof.ev[2 * keep], g_prof.ev[2 * i]);
      std::swap(g_prof.ev[2 * keep + 1], g_prof.ev[2 * i + 1]);
      g_prof.cls[keep] = g_prof.cls[i];
      g_prof.bytes[keep] = g_prof.bytes[i];
      g_prof.digit[keep] = g_prof.digit[i];
      ++keep;
      continue;
    }
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      continue;
    }
    int c = g_prof.cls[i];
    if (c == kKRadix && (!((radix_live >> g_prof.digit[i]) & 1u) || sort_mode)) c = kKRadixSkipped;
    if (c == kKMsd && sort_mode < g_prof.digit[i]) c = kKRadixSkipped;  // stage 2 runs in modes 2, 3; stage 3 in 3
    if (c == kKLocal && sort_mode == 0) c = kKRadixSkipped;
    g_prof.launches[c]++;
    g_prof.ms[c] += ms;
    g_prof.alg_bytes[c] += c == kKRadixSkipped ? 0.0 : g_prof.bytes[i];
  }
  g_prof.pending = keep;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Plan {
  int R = 16;
  uint32_t key_bytes = 8, Z = 0, L = 0, npass = 0, digits = 8;
  uint64_t n = 0, B = 1;
  bool fast = false;  // persistent cluster kernel (Z multiple of 32) instead of the generic one
  uint32_t pass_k[kMaxPasses] = {};
  uint32_t pass_i[kMaxPasses] = {};
  uint32_t pass_C[kMaxPasses] = {};
  bool pass_stream[kMaxPasses] = {};  // first / middle pass run by the streaming kernel (orp_stream.cu)
  // workspace offsets
  size_t off_ctrl = 0, off_rec[2] = {0, 0}, off_tag[2] = {0, 0}, off_status = 0;
  size_t off_tmp = 0, off_hist = 0, off_dbase = 0, off_rstatus = 0, off_ord = 0, off_load = 0, total = 0;
  size_t off_joint = 0, off_gstart = 0, off_rlist = 0, off_first = 0, off_meta = 0, off_spill = 0, off_ridx = 0;
  uint64_t orp_tiles = 0, radix_tiles = 0;
};

uint32_t max_k(int R, uint32_t Z, bool last) {
  uint32_t best = 0;
  for (uint32_t k = 1; k <= kMaxK; ++k)
    if (orp_smem_bytes(R, Z, k, last) <= kMaxSmem) best = k;
  return best;
}

constexpr uint32_t kMaxKFast = 8;

uint32_t max_k_fast(int R, uint32_t Z, uint32_t C, bool last) {
  uint32_t best = 0;
  for (uint32_t k = 1; k <= kMaxKFast; ++k)
    if ((1u << k) >= C && orp_fast_smem_bytes(R, Z, k, C, last) <= kMaxSmem) best = k;
  return best;
}

// Splits L levels into passes of at most kmid levels, the last one at most klast; the fewest
// passes, sizes balanced. Returns the pass count (0 if more than kMaxPasses would be needed).
uint32_t split_levels(uint32_t L, uint32_t kmid, uint32_t klast, uint32_t* pass_k) {
  if (kmid == 0 || klast == 0) return 0;
  for (uint32_t np = 1; np <= kMaxPasses; ++np) {
    const uint32_t kl = klast < (L + np - 1) / np ? klast : (L + np - 1) / np;
    const uint32_t rest = L - (kl < L ? kl : L);
    if (rest <= (np - 1) * kmid) {
      if (pass_k) {
        pass_k[np - 1] = L - rest;
        for (uint32_t x = 0; x + 1 < np; ++x) pass_k[x] = rest / (np - 1) + (x < rest % (np - 1));
      }
      return np;
    }
  }
  return 0;
}

bos_status make_plan(uint64_t n, const bos_params* p, bool sort, Plan* pl, uint32_t max_C = 16) {
  if (!p) return BOS_ERR_INVALID;
  if (!((p->rec_bytes == 8 && p->key_bytes == 4) || (p->rec_bytes == 16 && p->key_bytes == 8)))
    return BOS_ERR_INVALID;
  if (p->Z < 2 || p->Z > 4096) return BOS_ERR_INVALID;
  if (n >= (1ull << 31)) return BOS_ERR_INVALID;
  pl->R = (int)p->rec_bytes;
  pl->key_bytes = p->key_bytes;
  pl->digits = p->key_bytes;
  pl->Z = p->Z;
  pl->n = n;
  uint64_t B = 1;
  uint32_t L = 0;
  while (B * p->Z < 2 * n) {
    B <<= 1;
    ++L;
  }
  if (B * p->Z >= (1ull << 32)) return BOS_ERR_INVALID;  // slot indices are 32-bit inside a pass
  pl->B = B;
  pl->L = L;
  pl->fast = (p->Z % 32 == 0) && !(p->flags & BOS_FLAG_GENERIC);
  if (p->flags & BOS_FLAG_NO_CLUSTER) max_C = 1;
  const uint32_t cap = (p->flags >> 16) & 0x1Fu;
  if (cap && cap < max_C) max_C = cap;
  if (pl->fast && L > 0) {  // no cluster size fits this Z: the generic kernel takes it
    bool any = false;
    for (uint32_t C = 1; C <= max_C && !any; C <<= 1)
      any = max_k_fast(pl->R, p->Z, C, false) && max_k_fast(pl->R, p->Z, C, true);
    if (!any) pl->fast = false;
  }
  if (L == 0) {
    const uint32_t sm = pl->fast ? orp_fast_smem_bytes(pl->R, p->Z, 0, 1, true) : orp_smem_bytes(pl->R, p->Z, 0, true);
    if (sm > kMaxSmem) return BOS_ERR_INVALID;
    pl->npass = 1;
    pl->pass_k[0] = 0;
    pl->pass_C[0] = 1;
  } else if (!pl->fast) {
    // Split the L levels into passes: at most kmid levels per pass, klast in the last pass.
    uint32_t kmid = max_k(pl->R, p->Z, false), klast = max_k(pl->R, p->Z, true);
    if (p->k) {
      kmid = kmid < p->k ? kmid : p->k;
      klast = klast < p->k ? klast : p->k;
    }
    pl->npass = split_levels(L, kmid, klast, pl->pass_k);
    if (!pl->npass) return BOS_ERR_INVALID;
    for (uint32_t x = 0; x < pl->npass; ++x) pl->pass_C[x] = 1;
  } else if (p->flags & BOS_FLAG_FEWEST_PASSES) {
    // Fewest passes over the cluster sizes C (ties: the smaller C), then per pass the smallest
    // C that holds its k levels.
    uint32_t best_np = 0, best_C = 1;
    for (uint32_t C = 1; C <= max_C; C <<= 1) {
      uint32_t kmid = max_k_fast(pl->R, p->Z, C, false), klast = max_k_fast(pl->R, p->Z, C, true);
      if (p->k) {
        kmid = kmid < p->k ? kmid : p->k;
        klast = klast < p->k ? klast : p->k;
      }
      const uint32_t np = split_levels(L, kmid, klast, nullptr);
      if (np && (!best_np || np < best_np)) {
        best_np = np;
        best_C = C;
      }
    }
    if (!best_np) return BOS_ERR_INVALID;
    uint32_t kmid = max_k_fast(pl->R, p->Z, best_C, false), klast = max_k_fast(pl->R, p->Z, best_C, true);
    if (p->k) {
      kmid = kmid < p->k ? kmid : p->k;
      klast = klast < p->k ? klast : p->k;
    }
    pl->npass = split_levels(L, kmid, klast, pl->pass_k);
    for (uint32_t x = 0; x < pl->npass; ++x) {
      const bool last = x + 1 == pl->npass;
      uint32_t C = 1;
      while (C < best_C && (pl->pass_k[x] > max_k_fast(pl->R, p->Z, C, last) || (1u << pl->pass_k[x]) < C)) C <<= 1;
      pl->pass_C[x] = C;
    }
  } else {
    // Cost model from GB300 measurements of the persistent kernel: the time of one pass by role
    // and cluster size C, relative to a cluster-free middle pass (n = 2^30 16-byte records,
    // Z = 1024; each pass applying the most levels its C holds: 3, 4, 5, 6, 7). A cluster applies
    // more levels per pass, but its cluster barriers slow each subproblem; the first pass also
    // draws labels, the last one also writes the compacted output. Each pass takes the smallest
    // C that holds its levels; the first and last pass sizes are enumerated and the middle levels
    // split by dynamic programming. Ties go to fewer passes.
    static const double kMid[5] = {1.0, 1.371, 1.623, 1.919, 2.49};  // C = 1, 2, 4, 8, 16
    static const double kFirst[5] = {1.269, 1.496, 1.667, 2.168, 2.63};
    static const double kLast[5] = {1.219, 1.459, 1.723, 2.212, 2.63};
    // Streaming kernel, k up to 8-9: set so that a streaming plan wins where it saves a pass. Its
    // measured ratios at n = 2^30, Z = 1024 are 1.76 (first, k = 8) and 1.92 (paired middle), and
    // with those the streaming plan still wins there; at small Z they would pick cluster plans
    // that were never measured against it.
    static const double kStreamFirst = 0.85, kStreamMid = 1.15;
    const uint32_t kcap = p->k ? p->k : kMaxKFast;
    auto c_for = [&](uint32_t k, bool last) -> uint32_t {  // smallest C holding k levels; 0: none
      if (k > kcap) return 0;
      for (uint32_t C = 1; C <= max_C; C <<= 1)
        if ((1u << k) >= C && k <= max_k_fast(pl->R, p->Z, C, last)) return C;
      return 0;
    };
    auto ci = [](uint32_t C) { return (uint32_t)__builtin_ctz(C); };
    uint32_t ks = max_k_fast(pl->R, p->Z, 1, true);  // single FIRST+LAST pass (no cluster)
    if (p->k) ks = ks < p->k ? ks : p->k;
    if (ks == 0) return BOS_ERR_INVALID;  // (checked above)
    if (L <= ks) {
      pl->npass = 1;
      pl->pass_k[0] = L;
      pl->pass_C[0] = 1;
    } else {
      // best[M]: cheapest split of M middle levels (cost, passes, first pass size)
      double best[kMaxLevels + 1];
      uint32_t npb[kMaxLevels + 1], take[kMaxLevels + 1];
      best[0] = 0.0;
      npb[0] = 0;
      take[0] = 0;
      for (uint32_t M = 1; M <= L; ++M) {
        best[M] = 1e30;
        npb[M] = 0;
        take[M] = 0;
        for (uint32_t k = 1; k <= M; ++k) {
          const uint32_t C = c_for(k, false);
          if (!C || best[M - k] >= 1e29) continue;
          const double c = kMid[ci(C)] + best[M - k];
          const uint32_t np = npb[M - k] + 1;
          if (c < best[M] - 1e-9 || (c < best[M] + 1e-9 && np < npb[M])) {
            best[M] = c;
            npb[M] = np;
            take[M] = k;
          }
        }
      }
      double bc = 1e30;
      uint32_t bf = 0, bl = 0, bnp = 0;
      for (uint32_t f = 1; f < L; ++f) {
        const uint32_t Cf = c_for(f, false);
        if (!Cf) continue;
        for (uint32_t l = 1; f + l <= L; ++l) {
          const uint32_t Cl = c_for(l, true), M = L - f - l;
          if (!Cl || best[M] >= 1e29 || 2 + npb[M] > kMaxPasses) continue;
          const double c = kFirst[ci(Cf)] + kLast[ci(Cl)] + best[M];
          const uint32_t np = 2 + npb[M];
          if (c < bc - 1e-9 || (c < bc + 1e-9 && np < bnp)) {
            bc = c;
            bf = f;
            bl = l;
            bnp = np;
          }
        }
      }
      if (!bf) return BOS_ERR_INVALID;
      pl->npass = bnp;
      pl->pass_k[0] = bf;
      pl->pass_C[0] = c_for(bf, false);
      uint32_t M = L - bf - bl, x = 1;
      while (M) {
        pl->pass_k[x] = take[M];
        pl->pass_C[x] = c_for(take[M], false);
        M -= take[M];
        ++x;
      }
      pl->pass_k[bnp - 1] = bl;
      pl->pass_C[bnp - 1] = c_for(bl, true);
      // The streaming kernel (orp_stream.cu) takes the first and middle passes when that is
      // cheaper: up to 8-9 levels a pass with no cluster, the last pass stays the cluster kernel
      // (it needs its final buckets whole for the in-bin permutation). Costs in the same unit.
      const uint32_t kmin = orp_stream_min_k();
      // An automatic plan keeps a batch to about 8 reals per output bucket on average (Z / 2^k in
      // the first pass, Z / 2^(k+1) in a middle pass): more overrun the rings and the batch is
      // redone in small rounds. A caller-given k is taken as given.
      uint32_t lz = 0;
      while ((1u << lz) < p->Z) ++lz;
      const uint32_t kminf = p->k ? kmin : (lz >= 3 && lz - 3 > kmin ? lz - 3 : kmin);
      const uint32_t kminm = p->k ? kmin : (lz >= 4 && lz - 4 > kmin ? lz - 4 : kmin);
      uint32_t ksf = (p->flags & BOS_FLAG_NO_STREAM) ? 0u : orp_stream_max_k(pl->R, p->Z, true, kMaxSmem);
      uint32_t ksm = ksf ? orp_stream_max_k(pl->R, p->Z, false, kMaxSmem) : 0u;
      if (p->k) {  // a caller-given k caps every pass (k = 1 is the plain form)
        ksf = p->k >= kmin && ksf ? (ksf < p->k ? ksf : p->k) : 0u;
        ksm = p->k >= kmin && ksm ? (ksm < p->k ? ksm : p->k) : 0u;
      }
      if (ksf < kminf) ksf = 0;
      if (ksm < kminm) ksm = 0;
      double sbest = 1e30;
      uint32_t sl = 0, snp = 0;
      for (uint32_t l = 1; ksf && l < L; ++l) {
        const uint32_t Cl = c_for(l, true), S = L - l;
        if (!Cl) continue;
        for (uint32_t np = 1; np + 1 <= kMaxPasses; ++np) {
          if (S < kminf + (np - 1) * kminm || (np > 1 && !ksm)) continue;
          if (S > ksf + (np - 1) * ksm) continue;
          const double c = kStreamFirst + (np - 1) * kStreamMid + kLast[ci(Cl)];
          if (c < sbest - 1e-9) {
            sbest = c;
            sl = l;
            snp = np;
          }
          break;  // more stream passes only cost more
        }
      }
      if (sl && sbest < bc - 1e-9) {
        const uint32_t S = L - sl;
        pl->npass = snp + 1;
        // balanced split of S levels over snp passes, the first at most ksf, the others ksm
        for (uint32_t x = 0; x < snp; ++x) {
          pl->pass_k[x] = S / snp + (x < S % snp ? 1u : 0u);
          pl->pass_C[x] = 1;
          pl->pass_stream[x] = true;
        }
        while (pl->pass_k[0] > ksf) {  // move levels from the first pass to the middle ones
          for (uint32_t x = 1; x < snp && pl->pass_k[0] > ksf; ++x)
            if (pl->pass_k[x] < ksm) {
              pl->pass_k[x]++;
              pl->pass_k[0]--;
            }
        }
        pl->pass_k[snp] = sl;
        pl->pass_C[snp] = c_for(sl, true);
        pl->pass_stream[snp] = false;
      }
    }
  }
  uint32_t lvl = 0;
  for (uint32_t x = 0; x < pl->npass; ++x) {
    pl->pass_i[x] = lvl;
    lvl += pl->pass_k[x];
  }
  // workspace (independent of k and of the kernel choice)
  const uint64_t slots = B * p->Z;
  size_t off = 0;
  pl->off_ctrl = off; off = align256(off + sizeof(Ctrl));
  // two slot arrays whenever L >= 2 (the plain form needs both), so the size does not depend on k
  const uint32_t arrays = (L >= 2 || (p->flags & BOS_FLAG_OBLIVIOUS_SPLIT)) ? 2 : L;
  for (uint32_t x = 0; x < arrays; ++x) {
    pl->off_rec[x] = off; off = align256(off + slots * pl->R);
    pl->off_tag[x] = off; off = align256(off + slots * 4);
  }
  pl->orp_tiles = B >> pl->pass_k[pl->npass - 1];
  pl->off_ord = off; off = align256(off + slots * 2);  // in-bin permutation table (u16 per slot)
  pl->off_load = off; off = align256(off + B * 4);     // final loads, counted for the table
  // sized for the largest last pass (k = 1) so the workspace does not depend on k
  pl->off_status = off; off = align256(off + B * 8);
  if (sort) {
    pl->radix_tiles = radix_tiles(n, pl->R);
    pl->off_tmp = off;     off = align256(off + n * pl->R);
    pl->off_hist = off;    off = align256(off + pl->digits * 256 * 4);
    pl->off_dbase = off;   off = align256(off + pl->digits * 256 * 8);
    // look-back words: the LSD passes' tiles, or the hybrid sort's second partition (whose tiles
    // restart at every top-digit bucket: at most 256 more)
    pl->off_rstatus = off; off = align256(off + (pl->radix_tiles + 256) * 256 * 8);
    pl->off_joint = off;   off = align256(off + 65536 * 4);
    pl->off_gstart = off;  off = align256(off + 65537 * 8);
    pl->off_rlist = off;   off = align256(off + 65537 * 4);
    pl->off_first = off;   off = align256(off + 257 * 8);
    pl->off_meta = off;    off = align256(off + 32);
    pl->off_ridx = off;    off = align256(off + 2 * 65537 * 4);
    pl->off_spill = off;   off = align256(off + hybrid_spill_bytes(n, pl->R));
  }
  pl->total = off;
  return BOS_OK;
}

// Occupancy of a fast-kernel configuration on the current device (cached per configuration).
int fast_occupancy_cached(int R, int mode, uint32_t Z, uint32_t k, uint32_t C) {
  struct Entry { int dev, R, mode; uint32_t Z, k, C; int occ; };
  static std::mutex mu;
  static Entry cache[256];
  static int used = 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  {
    std::lock_guard<std::mutex> g(mu);
    for (int x = 0; x < used; ++x) {
      const Entry& e = cache[x];
      if (e.dev == dev && e.R == R && e.mode == mode && e.Z == Z && e.k == k && e.C == C) return e.occ;
    }
  }
  const int occ = orp_fast_occupancy(R, mode, Z, k, C);
  std::lock_guard<std::mutex> g(mu);
  if (used < 256) cache[used++] = Entry{dev, R, mode, Z, k, C, occ};
  return occ;
}

// Plan for this device: the largest cluster size whose every pass can be scheduled.
bos_status device_plan(uint64_t n, const bos_params* p, bool sort, Plan* pl) {
  for (uint32_t max_C = 16;; max_C >>= 1) {
    const bos_status s = make_plan(n, p, sort, pl, max_C);
    if (s != BOS_OK || !pl->fast || n == 0) return s;
    bool ok = true;
    for (uint32_t x = 0; x < pl->npass && ok; ++x) {
      const int mode = (x == 0 ? kModeFirst : 0) | (x + 1 == pl->npass ? kModeLast : 0);
      if (pl->pass_stream[x]) continue;  // streaming passes: one CTA per SM, sized by the planner
      ok = fast_occupancy_cached(pl->R, mode, pl->Z, pl->pass_k[x], pl->pass_C[x]) > 0;
    }
    if (ok) return BOS_OK;
    if (max_C == 1) {  // the fast kernel cannot run here: use the generic one
      bos_params q = *p;
      q.flags |= BOS_FLAG_GENERIC;
      return make_plan(n, &q, sort, pl, 1);
    }
  }
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return na && nb && x < y + nb && y < x + na;
}

#define BOS_CUDA(call)                   \
  do {                                   \
    if ((call) != cudaSuccess) {         \
      (void)cudaGetLastError();          \
      return BOS_ERR_CUDA;               \
    }                                    \
  } while (0)

bos_status run(const void* d_in, void* d_out, uint64_t n, const bos_params* p, void* d_ws,
               size_t ws_bytes, void* stream, bos_info* info, bool sort) {
  Plan pl;
  const bool plan_only = p && (p->flags & BOS_FLAG_PLAN_ONLY);
  bos_status s = (n && !plan_only) ? device_plan(n, p, sort, &pl) : make_plan(n, p, sort, &pl);
  if (s != BOS_OK) return s;
  if (info) {
    info->attempts = 0;
    info->L = pl.L;
    info->passes = pl.npass;
    info->radix_passes = 0;
    info->B = pl.B;
    info->max_cluster = 1;
    info->max_k = 0;
    info->stream_passes = 0;
    info->sort_mode = 0;
    for (uint32_t x = 0; x < pl.npass; ++x) {
      info->stream_passes += pl.pass_stream[x] ? 1u : 0u;
      info->max_cluster = pl.pass_C[x] > info->max_cluster ? pl.pass_C[x] : info->max_cluster;
      info->max_k = pl.pass_k[x] > info->max_k ? pl.pass_k[x] : info->max_k;
    }
  }
  if (n == 0 || plan_only) return BOS_OK;
  const size_t bytes = n * pl.R;
  if (!d_in || !d_out || !d_ws) return BOS_ERR_INVALID;
  if (((uintptr_t)d_in % pl.R) || ((uintptr_t)d_out % pl.R) || ((uintptr_t)d_ws & 255)) return BOS_ERR_INVALID;
  if (ws_bytes < pl.total) return BOS_ERR_WORKSPACE;
  if (overlaps(d_out, bytes, d_in, bytes) || overlaps(d_out, bytes, d_ws, ws_bytes)) return BOS_ERR_INVALID;

  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)d_ws;
  Ctrl* ctrl = (Ctrl*)(ws + pl.off_ctrl);
  const uint32_t max_attempts = p->max_attempts ? p->max_attempts : kDefaultAttempts;
  const uint32_t forced = (p->flags >> 8) & 0xFFu;
  const Trace tr = trace_snapshot();
  const bool trace = tr.buf != nullptr;

  // the comparison sort (stable merge) in place of the radix sort; its block-sorted runs start
  // in the buffer that leaves the last merge pass's output in d_out
  const bool merge = sort && (p->flags & BOS_FLAG_MERGE_SORT);
  void* merge_first = merge ? ((merge_passes(n) & 1) ? (void*)(ws + pl.off_tmp) : d_out) : nullptr;
  MergeHooks hooks{};
  hooks.begin = [](cudaStream_t s2, int stage, double b) { return prof_begin(s2, stage ? kKMerge : kKMergeBlock, b); };
  hooks.end = [](int slot, cudaStream_t s2) { prof_end(slot, s2); };
  // Section 4.1's form of the ORP (bitonic MergeSplits, one launch per level) in place of the
  // fused passes; its strip picks the output buffer the way the fused LAST pass does
  const bool oblivious = (p->flags & BOS_FLAG_OBLIVIOUS_SPLIT) != 0;
  if (oblivious && oblivious_smem_bytes(pl.R, pl.Z) > kMaxSmem) return BOS_ERR_INVALID;
  ObliviousArgs oa{};
  if (oblivious) {
    oa.in = d_in;
    oa.out0 = merge ? merge_first : d_out;
    oa.out1 = merge ? merge_first : (sort ? (void*)(ws + pl.off_tmp) : d_out);
    oa.out_sel = (sort && !merge) ? 1u : 0u;
    for (int x = 0; x < 2; ++x) {
      oa.rec[x] = ws + pl.off_rec[x];
      oa.tag[x] = (uint32_t*)(ws + pl.off_tag[x]);
    }
    oa.load = (uint32_t*)(ws + pl.off_status);  // B words each: loads, then offsets
    oa.off = oa.load + pl.B;
    oa.part = (uint32_t*)(ws + pl.off_ord);
    oa.n = n;
    oa.B = pl.B;
    oa.Z = pl.Z;
    oa.L = pl.L;
    oa.seed = p->seed;
    oa.ctrl = ctrl;
    oa.trace = tr;
  }

  RadixArgs ra{};
  if (sort && !merge) {
    ra.in = d_in;
    ra.buf0 = d_out;
    ra.buf1 = ws + pl.off_tmp;
    ra.n = n;
    ra.hist = (uint32_t*)(ws + pl.off_hist);
    ra.dbase = (unsigned long long*)(ws + pl.off_dbase);
    ra.status = (unsigned long long*)(ws + pl.off_rstatus);
    ra.ctrl = ctrl;
    ra.ticket_base = 1;
  }
  // the hybrid radix sort (partitions on the top digits, then on-chip sorts) unless the LSD sort
  // is asked for; its plan kernel picks the LSD passes by itself when a group is too large
  const bool hybrid = sort && !merge && !(p->flags & BOS_FLAG_LSD_SORT);
  HybridArgs ha{};
  if (hybrid) {
    ha.in = d_in;
    ha.buf0 = d_out;
    ha.buf1 = ws + pl.off_tmp;
    ha.n = n;
    ha.hist = ra.hist;
    ha.dbase = ra.dbase;
    ha.joint = (uint32_t*)(ws + pl.off_joint);
    ha.gstart = (unsigned long long*)(ws + pl.off_gstart);
    ha.rlist = (uint32_t*)(ws + pl.off_rlist);
    ha.first = (unsigned long long*)(ws + pl.off_first);
    ha.meta = (uint32_t*)(ws + pl.off_meta);
    ha.ridx = (uint32_t*)(ws + pl.off_ridx);
    ha.status = ra.status;
    ha.scratch = (unsigned char*)(ws + pl.off_spill);
    ha.local_ctas = hybrid_local_ctas(n, pl.R);
    ha.ctrl = ctrl;
  }

  for (uint32_t attempt = 0; attempt < max_attempts; ++attempt) {
    BOS_CUDA(zero_async(ctrl, sizeof(Ctrl), st));
    BOS_CUDA(zero_async(ws + pl.off_status, pl.orp_tiles * 8, st));
    if (sort && !merge) {
      BOS_CUDA(zero_async(ra.hist, pl.digits * 256 * 4, st));
      BOS_CUDA(zero_async(ra.status, (pl.radix_tiles + (hybrid ? 256 : 0)) * 256 * 8, st));
      int ev = prof_begin(st, kKHist, (double)n * pl.key_bytes);
      if (hybrid) {
        BOS_CUDA(zero_async(ha.joint, 65536 * 4, st));
        BOS_CUDA(launch_hybrid(ha, pl.R, 0, st));
      } else {
        BOS_CUDA(launch_radix_hist(ra, pl.R, st));
      }
      prof_end(ev, st);
      ev = prof_begin(st, kKPrep, 0.0);
      BOS_CUDA(launch_radix_prep(ra, pl.R, st));
      if (hybrid) {
        BOS_CUDA(launch_hybrid(ha, pl.R, 1, st));
        count_launches(1);  // the plan kernel, inside the prep event
      }
      prof_end(ev, st);
    }
    if (oblivious) {
      oa.attempt = attempt;
      const double slot_bytes = (double)pl.B * pl.Z * (pl.R + 4);
      const int ev = prof_begin(st, kKOblivious, 2.0 * n * pl.R + slot_bytes * (2.0 * pl.L + 3.0));
      BOS_CUDA(launch_oblivious_orp(oa, pl.R, st, trace));
      prof_end(ev, st);
    }
    for (uint32_t x = 0; x < (oblivious ? 0u : pl.npass); ++x) {
      PassArgs a{};
      const bool first = x == 0, last = x + 1 == pl.npass;
      const uint32_t src = (x + 1) & 1, dst = x & 1;  // pass x reads array (x-1)&1, writes x&1
      a.in = d_in;
      if (!first) {
        a.in_rec = ws + pl.off_rec[src];
        a.in_tag = (const uint32_t*)(ws + pl.off_tag[src]);
        a.buf_in_rec = src ? kBufRecB : kBufRecA;
        a.buf_in_tag = src ? kBufTagB : kBufTagA;
      }
      if (!last) {
        a.out_rec = ws + pl.off_rec[dst];
        a.out_tag = (uint32_t*)(ws + pl.off_tag[dst]);
        a.buf_out_rec = dst ? kBufRecB : kBufRecA;
        a.buf_out_tag = dst ? kBufTagB : kBufTagA;
      } else {
        a.out0 = d_out;
        a.out1 = sort ? ws + pl.off_tmp : d_out;
        a.out_sel = sort ? 1u : 0u;
        if (merge) {
          a.out0 = a.out1 = merge_first;
          a.out_sel = 0u;
        }
        a.status = (unsigned long long*)(ws + pl.off_status);
        a.skip_publish = (p->flags & BOS_FLAG_SKIP_PUBLISH) ? 1u : 0u;
        a.ord = (const uint16_t*)(ws + pl.off_ord);
      }
      a.n = n;
      a.B = pl.B;
      a.Z = pl.Z;
      a.L = pl.L;
      a.i = pl.pass_i[x];
      a.k = pl.pass_k[x];
      a.attempt = attempt;
      a.seed = p->seed;
      a.ctrl = ctrl;
      a.ticket_slot = 0;
      a.trace = tr;
      const int mode = (first ? kModeFirst : 0) | (last ? kModeLast : 0);
      // algorithmic bytes: whole slot arrays in and out, the input and output records once
      const double slot_bytes = (double)pl.B * pl.Z * (pl.R + 4);
      const double in_b = (first ? (double)n * pl.R : slot_bytes) + (last && pl.fast ? (double)pl.B * pl.Z * 2 : 0.0);
      const double out_b = last ? (double)n * pl.R : slot_bytes;
      const int cls = first && last ? kKSingle : first ? kKFirst : last ? kKLast : kKMid;
      if (last && pl.fast) {  // the LAST pass's in-bin permutation table for this attempt
        PermTableArgs ta{};
        ta.ord = (uint16_t*)(ws + pl.off_ord);
        ta.load = (uint32_t*)(ws + pl.off_load);
        ta.tag = first ? nullptr : a.in_tag;  // a single pass has no input tags: rows of all Z slots
        ta.B = pl.B;
        ta.Z = pl.Z;
        ta.attempt = attempt;
        ta.i = a.i;
        ta.k = a.k;
        ta.L = pl.L;
        ta.buf_tag = a.buf_in_tag;
        ta.seed = p->seed;
        ta.trace = tr;
        const double tb = (double)pl.B * pl.Z * (2.0 + (first ? 0.0 : 4.0));  // rows out, tags in
        const int evt = prof_begin(st, kKPerm, tb);
        BOS_CUDA(launch_perm_table(ta, st, trace));
        count_launches(1);  // final loads and table: two kernels in one event
        prof_end(evt, st);
      }
      const int ev = prof_begin(st, cls, in_b + out_b);
      if (pl.pass_stream[x])
        BOS_CUDA(launch_orp_stream(a, first, st, pl.R, trace));
      else if (pl.fast)
        BOS_CUDA(launch_orp_fast(a, mode, pl.pass_C[x], 0, st, pl.R, trace));
      else
        BOS_CUDA(launch_orp_pass(a, mode, pl.B >> a.k, st, pl.R, trace));
      prof_end(ev, st);
    }
    if (merge)
      BOS_CUDA(launch_merge_sort(merge_first, d_out, ws + pl.off_tmp, n, pl.R, (uint64_t*)(ws + pl.off_rstatus), st,
                                 hooks));
    else if (sort) {
      if (hybrid)  // each stage returns at once unless the plan's mode runs it
        for (int stage = 2; stage <= 4; ++stage) {
          const int ev = prof_begin(st, stage == 4 ? kKLocal : kKMsd, 2.0 * n * pl.R, (uint32_t)stage);
          BOS_CUDA(launch_hybrid(ha, pl.R, stage, st));
          if (stage == 4) count_launches(2);  // two warp-per-range launches and the CTA one
          prof_end(ev, st);
        }
      for (uint32_t d = 0; d < pl.digits; ++d) {  // skipped when the hybrid sort runs
        const int ev = prof_begin(st, kKRadix, 2.0 * n * pl.R, d);
        BOS_CUDA(launch_radix_pass(ra, pl.R, d, st));
        prof_end(ev, st);
      }
    }
    Ctrl h{};
    BOS_CUDA(cudaMemcpyAsync(&h, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    BOS_CUDA(cudaStreamSynchronize(st));
    if (g_prof.on) prof_collect(h.radix_live, h.sort_mode);
    if (info) {
      info->attempts = attempt + 1;
      info->sort_mode = h.sort_mode;
      info->radix_passes = h.sort_mode ? h.sort_mode : (uint32_t)__builtin_popcount(h.radix_live);
    }
    if (h.timeout) return BOS_ERR_TIMEOUT;
    if (h.bad) return BOS_ERR_CUDA;
    if (h.overflow || attempt < forced) continue;
    return BOS_OK;
  }
  return BOS_ERR_OVERFLOW;
}

// ============================================================================================
// Batched ORP / sort: many independent arrays through one fixed sequence of launches (one per
// butterfly pass index and mode, one per radix stage), suitable for capture into a CUDA graph.
// Every array uses the one-CTA-per-subproblem pass kernel; its plan, seed and Z are its own, so
// its result equals bos_orp / bos_sort of that array alone.
// ============================================================================================
constexpr uint32_t kBatchMaxPass = 16;
constexpr size_t kBatchHeader = 1024;  // launch tickets (zeroed with the control blocks)

struct BatchIn {
  const void* d_in;
  void* d_out;
  const uint64_t* off;
  uint32_t num;
  const uint64_t* seeds;
  const uint32_t* Zs;
  const uint8_t* ops;
  bos_params base;
};

struct BatchArr {
  Plan pl;
  bool sort = false;
  size_t zero_off = 0, data_off = 0;  // per-array regions
  size_t st_off = 0, hist_off = 0, rst_off = 0;                      // inside the zero region
  size_t rec_off[2] = {0, 0}, tag_off[2] = {0, 0}, tmp_off = 0, dbase_off = 0;  // data region
};

struct BatchLayout {
  std::vector<BatchArr> arr;
  size_t ctrl_off = 0, zero_end = 0, desc_off = 0, desc_bytes = 0, data_off = 0, total = 0;
  int R = 8;
  uint32_t maxpass = 0, digits = 4;
};

bos_status batch_layout(const BatchIn& b, BatchLayout* L) {
  if (!b.off || (!b.seeds && b.num) || (!b.ops && b.num)) return BOS_ERR_INVALID;
  L->R = (int)b.base.rec_bytes;
  L->digits = b.base.key_bytes;
  L->arr.assign(b.num, BatchArr{});
  size_t off = 0;
  off += kBatchHeader;
  L->ctrl_off = off;
  off += (size_t)b.num * sizeof(Ctrl);
  for (uint32_t j = 0; j < b.num; ++j) {
    if (b.off[j + 1] < b.off[j]) return BOS_ERR_INVALID;
    BatchArr& a = L->arr[j];
    bos_params p = b.base;
    p.flags = (p.flags | BOS_FLAG_GENERIC) & ~BOS_FLAG_SKIP_PUBLISH;
    if (b.Zs) p.Z = b.Zs[j];
    a.sort = b.ops[j] != 0;
    const bos_status s = make_plan(b.off[j + 1] - b.off[j], &p, a.sort, &a.pl);
    if (s != BOS_OK) return s;
    if (a.pl.npass > kBatchMaxPass) return BOS_ERR_INVALID;
    L->maxpass = a.pl.npass > L->maxpass ? a.pl.npass : L->maxpass;
    a.zero_off = off;
    a.st_off = off; off = align256(off + a.pl.B * 8);
    if (a.sort) {
      a.hist_off = off; off = align256(off + L->digits * 256 * 4);
      a.rst_off = off;  off = align256(off + radix_tiles(a.pl.n, L->R) * 256 * 8);
    }
  }
  L->zero_end = off;
  // descriptors: PassArgs for every (array, pass), RadixArgs per array, prefix arrays
  L->desc_off = off;
  size_t dsz = 0;
  for (uint32_t j = 0; j < b.num; ++j) dsz += L->arr[j].pl.npass * sizeof(PassArgs);
  dsz += (size_t)b.num * sizeof(RadixArgs);
  dsz += (size_t)(kBatchMaxPass * 4 + 2) * (b.num + 1) * sizeof(uint64_t);
  L->desc_bytes = align256(dsz);
  off = align256(off + L->desc_bytes);
  L->data_off = off;
  for (uint32_t j = 0; j < b.num; ++j) {
    BatchArr& a = L->arr[j];
    const uint64_t slots = a.pl.B * a.pl.Z;
    const uint32_t arrays = a.pl.L >= 2 ? 2 : a.pl.L;
    a.data_off = off;
    for (uint32_t x = 0; x < arrays; ++x) {
      a.rec_off[x] = off; off = align256(off + slots * L->R);
      a.tag_off[x] = off; off = align256(off + slots * 4);
    }
    if (a.sort) {
      a.tmp_off = off;   off = align256(off + a.pl.n * L->R);
      a.dbase_off = off; off = align256(off + L->digits * 256 * 8);
    }
  }
  L->total = off;
  return BOS_OK;
}

// One launch of the sequence: an ORP pass (index, mode) or a radix stage.
struct BatchLaunch {
  int kind;  // 0 = ORP pass, 1 = radix histogram, 2 = radix offsets, 3 = radix digit pass
  int mode;
  uint32_t digit, smem;
  BatchPass bp;
  BatchRadix br;
};

// Builds the launch sequence for the arrays in `sel` (attempt[j] each) and, when `desc` is not
// null, the descriptor bytes to copy into the workspace's descriptor region.
bos_status batch_build(const BatchIn& b, const BatchLayout& L, char* ws, const std::vector<uint32_t>& sel,
                       const std::vector<uint32_t>& attempt, std::vector<BatchLaunch>* launches,
                       std::vector<char>* desc) {
  launches->clear();
  if (desc) desc->assign(L.desc_bytes, 0);
  const Trace tr = trace_snapshot();  // the trace buffer the descriptors carry (debug)
  size_t dpos = 0;
  auto dev = [&](size_t pos) { return ws + L.desc_off + pos; };
  uint32_t ticket_slot = 0;
  uint32_t* tickets = (uint32_t*)ws;  // header
  const int R = L.R;
  // radix descriptors (sort arrays among sel, in sel order)
  std::vector<uint32_t> sorts;
  for (uint32_t j : sel)
    if (L.arr[j].sort && L.arr[j].pl.n) sorts.push_back(j);
  const size_t ra_pos = dpos;
  dpos += sorts.size() * sizeof(RadixArgs);
  const size_t rfirst_pos = dpos;
  dpos += (sorts.size() + 1) * sizeof(uint64_t);
  {
    uint64_t acc = 0;
    for (size_t x = 0; x < sorts.size(); ++x) {
      const uint32_t j = sorts[x];
      const BatchArr& a = L.arr[j];
      RadixArgs ra{};
      ra.in = (const char*)b.d_in + b.off[j] * R;
      ra.buf0 = (char*)b.d_out + b.off[j] * R;
      ra.buf1 = ws + a.tmp_off;
      ra.n = a.pl.n;
      ra.hist = (uint32_t*)(ws + a.hist_off);
      ra.dbase = (unsigned long long*)(ws + a.dbase_off);
      ra.status = (unsigned long long*)(ws + a.rst_off);
      ra.ctrl = (Ctrl*)(ws + L.ctrl_off + (size_t)j * sizeof(Ctrl));
      ra.ticket_base = 0;
      if (desc) {
        std::memcpy(desc->data() + ra_pos + x * sizeof(RadixArgs), &ra, sizeof(ra));
        std::memcpy(desc->data() + rfirst_pos + x * sizeof(uint64_t), &acc, sizeof(acc));
      }
      acc += radix_tiles(a.pl.n, R);
    }
    if (desc) std::memcpy(desc->data() + rfirst_pos + sorts.size() * sizeof(uint64_t), &acc, sizeof(acc));
    BatchRadix br{};
    br.args = (const RadixArgs*)dev(ra_pos);
    br.first = (const uint64_t*)dev(rfirst_pos);
    br.narr = (uint32_t)sorts.size();
    br.nblocks = acc;
    br.ticket = tickets + ticket_slot;
    ticket_slot += L.digits;
    if (!sorts.empty()) {
      launches->push_back(BatchLaunch{1, 0, 0, 0, BatchPass{}, br});
      launches->push_back(BatchLaunch{2, 0, 0, 0, BatchPass{}, br});
    }
    // the digit passes come after the ORP passes (pushed at the end)
    for (uint32_t p = 0; p < L.maxpass; ++p) {
      for (int mode : {kModeFirst | kModeLast, kModeFirst, 0, kModeLast}) {
        std::vector<uint32_t> js;
        for (uint32_t j : sel) {
          const BatchArr& a = L.arr[j];
          if (a.pl.n == 0 || p >= a.pl.npass) continue;
          const int m = (p == 0 ? kModeFirst : 0) | (p + 1 == a.pl.npass ? kModeLast : 0);
          if (m == mode) js.push_back(j);
        }
        if (js.empty()) continue;
        const size_t args_pos = dpos;
        dpos += js.size() * sizeof(PassArgs);
        const size_t first_pos = dpos;
        dpos += (js.size() + 1) * sizeof(uint64_t);
        uint64_t acc2 = 0;
        uint32_t smem = 0;
        for (size_t x = 0; x < js.size(); ++x) {
          const uint32_t j = js[x];
          const BatchArr& a = L.arr[j];
          PassArgs pa{};
          const bool first = p == 0, last = p + 1 == a.pl.npass;
          const uint32_t src = (p + 1) & 1, dst = p & 1;
          pa.in = (const char*)b.d_in + b.off[j] * R;
          if (!first) {
            pa.in_rec = ws + a.rec_off[src];
            pa.in_tag = (const uint32_t*)(ws + a.tag_off[src]);
          }
          if (!last) {
            pa.out_rec = ws + a.rec_off[dst];
            pa.out_tag = (uint32_t*)(ws + a.tag_off[dst]);
          } else {
            pa.out0 = (char*)b.d_out + b.off[j] * R;
            pa.out1 = a.sort ? ws + a.tmp_off : pa.out0;
            pa.out_sel = a.sort ? 1u : 0u;
            pa.status = (unsigned long long*)(ws + a.st_off);
          }
          pa.n = a.pl.n;
          pa.B = a.pl.B;
          pa.Z = a.pl.Z;
          pa.L = a.pl.L;
          pa.i = a.pl.pass_i[p];
          pa.k = a.pl.pass_k[p];
          pa.attempt = attempt[j];
          pa.seed = b.seeds[j];
          pa.ctrl = (Ctrl*)(ws + L.ctrl_off + (size_t)j * sizeof(Ctrl));
          pa.trace = tr;
          pa.buf_in_rec = src ? kBufRecB : kBufRecA;
          pa.buf_in_tag = src ? kBufTagB : kBufTagA;
          pa.buf_out_rec = dst ? kBufRecB : kBufRecA;
          pa.buf_out_tag = dst ? kBufTagB : kBufTagA;
          const uint32_t sm = orp_smem_bytes(R, pa.Z, pa.k, last);
          smem = sm > smem ? sm : smem;
          if (desc) {
            std::memcpy(desc->data() + args_pos + x * sizeof(PassArgs), &pa, sizeof(pa));
            std::memcpy(desc->data() + first_pos + x * sizeof(uint64_t), &acc2, sizeof(acc2));
          }
          acc2 += a.pl.B >> pa.k;
        }
        if (desc) std::memcpy(desc->data() + first_pos + js.size() * sizeof(uint64_t), &acc2, sizeof(acc2));
        BatchPass bp{};
        bp.args = (const PassArgs*)dev(args_pos);
        bp.first = (const uint64_t*)dev(first_pos);
        bp.narr = (uint32_t)js.size();
        bp.nblocks = acc2;
        bp.ticket = tickets + ticket_slot++;
        if (ticket_slot * 4 > kBatchHeader) return BOS_ERR_INVALID;
        launches->push_back(BatchLaunch{0, mode, 0, smem, bp, BatchRadix{}});
      }
    }
    if (!sorts.empty())
      for (uint32_t d = 0; d < L.digits; ++d) launches->push_back(BatchLaunch{3, 0, d, 0, BatchPass{}, br});
  }
  if (dpos > L.desc_bytes) return BOS_ERR_INVALID;
  return BOS_OK;
}

bos_status batch_enqueue(const BatchLayout& L, char* ws, const std::vector<BatchLaunch>& launches, cudaStream_t st) {
  BOS_CUDA(zero_async(ws, L.zero_end, st));
  const bool trace = trace_snapshot().buf != nullptr;
  for (const BatchLaunch& l : launches) {
    if (l.kind == 0) {
      BOS_CUDA(launch_orp_pass_batched(l.bp, l.mode, l.smem, st, L.R, trace));
    } else {
      BOS_CUDA(launch_radix_batched(l.br, L.R, l.kind - 1, l.digit, st));
    }
  }
  return BOS_OK;
}

bos_status batch_check_in(const BatchIn& b, const BatchLayout& L, void* d_ws, size_t ws_bytes) {
  if (!d_ws || ((uintptr_t)d_ws & 255)) return BOS_ERR_INVALID;
  if (ws_bytes < L.total) return BOS_ERR_WORKSPACE;
  const uint64_t nrec = b.num ? b.off[b.num] : 0;
  if (nrec && (!b.d_in || !b.d_out)) return BOS_ERR_INVALID;
  if (((uintptr_t)b.d_in % L.R) || ((uintptr_t)b.d_out % L.R)) return BOS_ERR_INVALID;
  const size_t bytes = nrec * L.R;
  if (overlaps(b.d_out, bytes, b.d_in, bytes) || overlaps(b.d_out, bytes, d_ws, ws_bytes)) return BOS_ERR_INVALID;
  return BOS_OK;
}

// Writes the descriptors of `sel` (synchronous copy from host memory).
bos_status batch_prepare(const BatchIn& b, const BatchLayout& L, char* ws, const std::vector<uint32_t>& sel,
                         const std::vector<uint32_t>& attempt, std::vector<BatchLaunch>* launches,
                         cudaStream_t st) {
  std::vector<char> desc;
  bos_status s = batch_build(b, L, ws, sel, attempt, launches, &desc);
  if (s != BOS_OK) return s;
  BOS_CUDA(cudaMemcpyAsync(ws + L.desc_off, desc.data(), desc.size(), cudaMemcpyHostToDevice, st));
  BOS_CUDA(cudaStreamSynchronize(st));
  return BOS_OK;
}

std::vector<uint32_t> all_arrays(uint32_t num) {
  std::vector<uint32_t> v(num);
  for (uint32_t j = 0; j < num; ++j) v[j] = j;
  return v;
}

// After an enqueue: reads every array's flags; arrays that overflowed run again (as a smaller
// batch) with the next attempt counter, up to max_attempts; then the descriptors of the full
// batch (attempt 0) are written back so a captured graph stays valid.
bos_status batch_collect(const BatchIn& b, const BatchLayout& L, char* ws, cudaStream_t st, uint32_t* h_attempts) {
  const uint32_t max_attempts = b.base.max_attempts ? b.base.max_attempts : kDefaultAttempts;
  std::vector<uint32_t> attempt(b.num, 0);
  std::vector<Ctrl> h(b.num);
  std::vector<uint32_t> sel = all_arrays(b.num), launched_retry;
  bos_status result = BOS_OK;
  for (uint32_t round = 0;; ++round) {
    if (b.num) BOS_CUDA(cudaMemcpyAsync(h.data(), ws + L.ctrl_off, b.num * sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    BOS_CUDA(cudaStreamSynchronize(st));
    std::vector<uint32_t> failed;
    for (uint32_t j : sel) {
      if (L.arr[j].pl.n == 0) continue;
      if (h[j].timeout) result = BOS_ERR_TIMEOUT;
      if (h[j].overflow) failed.push_back(j);
    }
    if (result != BOS_OK || failed.empty()) break;
    for (uint32_t j : failed) attempt[j]++;
    bool exhausted = false;
    for (uint32_t j : failed) exhausted |= attempt[j] >= max_attempts;
    if (exhausted) {
      result = BOS_ERR_OVERFLOW;
      break;
    }
    std::vector<BatchLaunch> launches;
    bos_status s = batch_prepare(b, L, ws, failed, attempt, &launches, st);
    if (s != BOS_OK) return s;
    if ((s = batch_enqueue(L, ws, launches, st)) != BOS_OK) return s;
    sel = failed;
    launched_retry = failed;
  }
  if (h_attempts)
    for (uint32_t j = 0; j < b.num; ++j) h_attempts[j] = L.arr[j].pl.n ? attempt[j] + 1 : 0;
  if (!launched_retry.empty()) {  // restore the full batch's descriptors
    std::vector<BatchLaunch> launches;
    const bos_status s = batch_prepare(b, L, ws, all_arrays(b.num), std::vector<uint32_t>(b.num, 0), &launches, st);
    if (s != BOS_OK) return s;
  }
  return result;
}

}  // namespace

// ============================================================================================
// Shard plan: Algorithm 3.1 over G = 2^g ranks with one fixed exchange (the multi-GPU form of the
// butterfly). Rank r holds buckets [r Bl, (r+1) Bl), Bl = B / G: levels 0 .. L-g-1 pair buckets
// inside aligned blocks of at most Bl and run locally (the rank's passes over its buckets, with
// global label bits and group ranges); then rank s sends rank d its local buckets
// [d Bl/G, (d+1) Bl/G) (whole buckets: volume and addresses do not depend on the data); rank d's
// received buckets, s-major, are the inputs of the subproblems t in [d Bl/G, (d+1) Bl/G) of the
// last g levels, which one fused LAST pass runs (local level count L - g, so the routing digit is
// the label's low g bits), leaving rank d its final buckets [d Bl, (d+1) Bl), permuted by the
// Section 3.2 keys of their global indexes and stripped of dummies.
// ============================================================================================
namespace {

struct ShardPlan {
  Plan lp;            // the local levels as a plan over Bl buckets (its workspace layout)
  uint64_t B = 0, Bl = 0;
  uint32_t L = 0, g = 0, G = 0, kC = 1;  // kC: cluster size of the final pass (Z multiple of 32)
  bool fast_final = false;
  size_t send_rec = 0, send_tag = 0, recv_rec = 0, recv_tag = 0, chunk_rec = 0, chunk_tag = 0;
};

bos_status shard_plan(uint64_t n, uint32_t G, const bos_params* p, ShardPlan* sp) {
  if (!p || G < 2 || (G & (G - 1)) || (p->flags & (BOS_FLAG_OBLIVIOUS_SPLIT | BOS_FLAG_MERGE_SORT))) return BOS_ERR_INVALID;
  Plan full;
  bos_status s = make_plan(n, p, false, &full);
  if (s != BOS_OK) return s;
  uint32_t g = 0;
  while ((1u << g) < G) ++g;
  if ((uint64_t)G * G > full.B) return BOS_ERR_INVALID;  // every rank sends every rank a whole bucket
  sp->B = full.B;
  sp->L = full.L;
  sp->g = g;
  sp->G = G;
  sp->Bl = full.B / G;
  // the local levels: a plan over Bl buckets of L - g levels (n' fills them exactly)
  bos_params q = *p;
  q.flags &= ~(uint32_t)BOS_FLAG_PLAN_ONLY;
  s = make_plan(sp->Bl * p->Z / 2, &q, false, &sp->lp);
  if (s != BOS_OK) return s;
  if (sp->lp.B != sp->Bl || sp->lp.L != full.L - g) return BOS_ERR_INVALID;
  // the final pass: g levels in one LAST pass
  sp->fast_final = sp->lp.fast;
  if (sp->fast_final) {
    uint32_t C = 1;
    while (C <= 16 && (g > max_k_fast(sp->lp.R, p->Z, C, true) || (1u << g) < C)) C <<= 1;
    if (C > 16) sp->fast_final = false; else sp->kC = C;
  }
  if (!sp->fast_final && g > max_k(sp->lp.R, p->Z, true)) return BOS_ERR_INVALID;
  // the local step leaves its buckets in slot array (passes - 1) & 1; the exchange fills the other
  const uint32_t last = (sp->lp.npass - 1) & 1, other = last ^ 1;
  if (sp->lp.L < 2) return BOS_ERR_INVALID;  // both slot arrays exist only when L - g >= 2
  sp->send_rec = sp->lp.off_rec[last];
  sp->send_tag = sp->lp.off_tag[last];
  sp->recv_rec = sp->lp.off_rec[other];
  sp->recv_tag = sp->lp.off_tag[other];
  sp->chunk_rec = (size_t)(sp->Bl / G) * p->Z * sp->lp.R;
  sp->chunk_tag = (size_t)(sp->Bl / G) * p->Z * 4;
  return BOS_OK;
}

}  // namespace

size_t orp_workspace_bytes(uint64_t n, const bos_params* p) {
  Plan pl;
  if (make_plan(n, p, false, &pl) != BOS_OK) return 0;
  return n ? pl.total : 0;
}

bos_status orp_with_workspace(const void* d_in, void* d_out, uint64_t n, const bos_params* p,
                              void* d_ws, size_t ws_bytes, void* stream, bos_info* info) {
  return run(d_in, d_out, n, p, d_ws, ws_bytes, stream, info, false);
}

}  // namespace bos

using namespace bos;

extern "C" {

size_t bos_workspace_bytes(uint64_t n, const bos_params* p) {
  Plan pl;
  if (make_plan(n, p, true, &pl) != BOS_OK) return 0;
  return n ? pl.total : 0;
}

bos_status bos_orp(const void* d_in, void* d_out, uint64_t n, const bos_params* p, void* d_ws,
                   size_t ws_bytes, void* stream, bos_info* info) {
  return run(d_in, d_out, n, p, d_ws, ws_bytes, stream, info, false);
}

bos_status bos_sort(const void* d_in, void* d_out, uint64_t n, const bos_params* p, void* d_ws,
                    size_t ws_bytes, void* stream, bos_info* info) {
  return run(d_in, d_out, n, p, d_ws, ws_bytes, stream, info, true);
}

size_t bos_batched_workspace_bytes(const uint64_t* h_offsets, uint32_t num, const uint32_t* h_Z,
                                   const uint8_t* h_ops, const bos_params* base) {
  if (!h_offsets || !base || (num && !h_ops)) return 0;
  std::vector<uint64_t> seeds(num, 0);
  BatchIn b{nullptr, nullptr, h_offsets, num, seeds.data(), h_Z, h_ops, *base};
  BatchLayout L;
  if (batch_layout(b, &L) != BOS_OK) return 0;
  return L.total;
}

bos_status bos_batched_prepare(const void* d_in, void* d_out, const uint64_t* h_offsets, uint32_t num,
                               const uint64_t* h_seeds, const uint32_t* h_Z, const uint8_t* h_ops,
                               const bos_params* base, void* d_ws, size_t ws_bytes, void* stream) {
  if (!base) return BOS_ERR_INVALID;
  BatchIn b{d_in, d_out, h_offsets, num, h_seeds, h_Z, h_ops, *base};
  BatchLayout L;
  bos_status s = batch_layout(b, &L);
  if (s != BOS_OK) return s;
  if ((s = batch_check_in(b, L, d_ws, ws_bytes)) != BOS_OK) return s;
  std::vector<BatchLaunch> launches;
  return batch_prepare(b, L, (char*)d_ws, all_arrays(num), std::vector<uint32_t>(num, 0), &launches,
                       (cudaStream_t)stream);
}

bos_status bos_batched_enqueue(const void* d_in, void* d_out, const uint64_t* h_offsets, uint32_t num,
                               const uint64_t* h_seeds, const uint32_t* h_Z, const uint8_t* h_ops,
                               const bos_params* base, void* d_ws, size_t ws_bytes, void* stream) {
  if (!base) return BOS_ERR_INVALID;
  BatchIn b{d_in, d_out, h_offsets, num, h_seeds, h_Z, h_ops, *base};
  BatchLayout L;
  bos_status s = batch_layout(b, &L);
  if (s != BOS_OK) return s;
  if ((s = batch_check_in(b, L, d_ws, ws_bytes)) != BOS_OK) return s;
  std::vector<BatchLaunch> launches;
  if ((s = batch_build(b, L, (char*)d_ws, all_arrays(num), std::vector<uint32_t>(num, 0), &launches, nullptr)) != BOS_OK)
    return s;
  return batch_enqueue(L, (char*)d_ws, launches, (cudaStream_t)stream);
}

bos_status bos_batched_collect(const void* d_in, void* d_out, const uint64_t* h_offsets, uint32_t num,
                               const uint64_t* h_seeds, const uint32_t* h_Z, const uint8_t* h_ops,
                               const bos_params* base, void* d_ws, size_t ws_bytes, void* stream,
                               uint32_t* h_attempts) {
  if (!base) return BOS_ERR_INVALID;
  BatchIn b{d_in, d_out, h_offsets, num, h_seeds, h_Z, h_ops, *base};
  BatchLayout L;
  bos_status s = batch_layout(b, &L);
  if (s != BOS_OK) return s;
  if ((s = batch_check_in(b, L, d_ws, ws_bytes)) != BOS_OK) return s;
  return batch_collect(b, L, (char*)d_ws, (cudaStream_t)stream, h_attempts);
}

bos_status bos_sort_batched(const void* d_in, void* d_out, const uint64_t* h_offsets, uint32_t num,
                            const uint64_t* h_seeds, const uint32_t* h_Z, const uint8_t* h_ops,
                            const bos_params* base, void* d_ws, size_t ws_bytes, void* stream,
                            uint32_t* h_attempts) {
  bos_status s = bos_batched_prepare(d_in, d_out, h_offsets, num, h_seeds, h_Z, h_ops, base, d_ws, ws_bytes, stream);
  if (s != BOS_OK) return s;
  s = bos_batched_enqueue(d_in, d_out, h_offsets, num, h_seeds, h_Z, h_ops, base, d_ws, ws_bytes, stream);
  if (s != BOS_OK) return s;
  return bos_batched_collect(d_in, d_out, h_offsets, num, h_seeds, h_Z, h_ops, base, d_ws, ws_bytes, stream,
                             h_attempts);
}

bos_status bos_shard_layout(uint64_t n, uint32_t G, const bos_params* p, bos_shard_layout_t* out) {
  ShardPlan sp;
  const bos_status s = shard_plan(n, G, p, &sp);
  if (s != BOS_OK || !out) return s != BOS_OK ? s : BOS_ERR_INVALID;
  out->B = sp.B;
  out->B_local = sp.Bl;
  out->L = sp.L;
  out->g = sp.g;
  out->local_passes = sp.lp.npass;
  out->ws_bytes = sp.lp.total;
  out->send_rec_offset = sp.send_rec;
  out->send_tag_offset = sp.send_tag;
  out->recv_rec_offset = sp.recv_rec;
  out->recv_tag_offset = sp.recv_tag;
  out->chunk_rec_bytes = sp.chunk_rec;
  out->chunk_tag_bytes = sp.chunk_tag;
  out->out_capacity = sp.Bl * p->Z;
  return BOS_OK;
}

bos_status bos_shard_input_range(uint64_t n, uint32_t G, uint32_t r, const bos_params* p, uint64_t* lo,
                                 uint64_t* hi) {
  ShardPlan sp;
  const bos_status s = shard_plan(n, G, p, &sp);
  if (s != BOS_OK) return s;
  if (r >= G || !lo || !hi) return BOS_ERR_INVALID;
  *lo = ((uint64_t)r * sp.Bl * n) >> sp.L;
  *hi = ((uint64_t)(r + 1) * sp.Bl * n) >> sp.L;
  return BOS_OK;
}

bos_status bos_shard_local(const void* d_in, uint64_t n, uint32_t G, uint32_t r, const bos_params* p,
                           uint32_t attempt, void* d_ws, size_t ws_bytes, void* stream) {
  ShardPlan sp;
  bos_status s = shard_plan(n, G, p, &sp);
  if (s != BOS_OK) return s;
  if (r >= G || !d_ws || ((uintptr_t)d_ws & 255) || (!d_in && n)) return BOS_ERR_INVALID;
  if (ws_bytes < sp.lp.total) return BOS_ERR_WORKSPACE;
  const Plan& pl = sp.lp;
  if ((uintptr_t)d_in % pl.R) return BOS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)d_ws;
  Ctrl* ctrl = (Ctrl*)(ws + pl.off_ctrl);
  const uint64_t lo = ((uint64_t)r * sp.Bl * n) >> sp.L;
  const Trace tr = trace_snapshot();
  BOS_CUDA(zero_async(ctrl, sizeof(Ctrl), st));
  for (uint32_t x = 0; x < pl.npass; ++x) {
    PassArgs a{};
    const bool first = x == 0;
    const uint32_t src = (x + 1) & 1, dst = x & 1;
    // the rank's input slice starts at global record lo: the kernels index records globally
    a.in = (const char*)d_in - lo * pl.R;
    if (!first) {
      a.in_rec = ws + pl.off_rec[src];
      a.in_tag = (const uint32_t*)(ws + pl.off_tag[src]);
      a.buf_in_rec = src ? kBufRecB : kBufRecA;
      a.buf_in_tag = src ? kBufTagB : kBufTagA;
    }
    a.out_rec = ws + pl.off_rec[dst];
    a.out_tag = (uint32_t*)(ws + pl.off_tag[dst]);
    a.buf_out_rec = dst ? kBufRecB : kBufRecA;
    a.buf_out_tag = dst ? kBufTagB : kBufTagA;
    a.n = n;
    a.B = sp.Bl;
    a.Z = pl.Z;
    a.L = sp.L;  // global label width: levels 0 .. L-g-1 route on its top bits
    a.i = pl.pass_i[x];
    a.k = pl.pass_k[x];
    a.attempt = attempt;
    a.seed = p->seed;
    a.ctrl = ctrl;
    a.trace = tr;
    a.bucket0 = (uint64_t)r * sp.Bl;
    const int mode = first ? kModeFirst : 0;
    if (pl.pass_stream[x])
      BOS_CUDA(launch_orp_stream(a, first, st, pl.R, tr.buf != nullptr));
    else if (pl.fast)
      BOS_CUDA(launch_orp_fast(a, mode, pl.pass_C[x], 0, st, pl.R, tr.buf != nullptr));
    else
      BOS_CUDA(launch_orp_pass(a, mode, sp.Bl >> a.k, st, pl.R, tr.buf != nullptr));
  }
  return BOS_OK;
}

bos_status bos_shard_final(uint64_t n, uint32_t G, uint32_t r, const bos_params* p, uint32_t attempt,
                           void* d_out, uint64_t out_cap, void* d_ws, size_t ws_bytes, void* stream,
                           uint64_t* h_count, uint32_t* h_overflow) {
  ShardPlan sp;
  bos_status s = shard_plan(n, G, p, &sp);
  if (s != BOS_OK) return s;
  if (r >= G || !d_ws || ((uintptr_t)d_ws & 255) || !d_out || !h_count || !h_overflow) return BOS_ERR_INVALID;
  if (ws_bytes < sp.lp.total) return BOS_ERR_WORKSPACE;
  const Plan& pl = sp.lp;
  if ((uintptr_t)d_out % pl.R || overlaps(d_out, out_cap * pl.R, d_ws, ws_bytes)) return BOS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)d_ws;
  Ctrl* ctrl = (Ctrl*)(ws + pl.off_ctrl);
  const Trace tr = trace_snapshot();
  const uint64_t nsub = sp.Bl >> sp.g;
  // the local step's overflow flag stays; the tickets and look-back words start at zero
  BOS_CUDA(zero_async(&ctrl->tickets[0], sizeof(ctrl->tickets), st));
  BOS_CUDA(zero_async(ws + pl.off_status, nsub * 8, st));
  PassArgs a{};
  a.in_rec = ws + sp.recv_rec;
  a.in_tag = (const uint32_t*)(ws + sp.recv_tag);
  a.buf_in_rec = sp.recv_rec == pl.off_rec[1] ? kBufRecB : kBufRecA;
  a.buf_in_tag = sp.recv_rec == pl.off_rec[1] ? kBufTagB : kBufTagA;
  a.out0 = a.out1 = d_out;
  a.out_sel = 0;
  a.status = (unsigned long long*)(ws + pl.off_status);
  a.ord = (const uint16_t*)(ws + pl.off_ord);
  a.n = out_cap;  // bound of the output positions
  a.B = sp.Bl;
  a.Z = pl.Z;
  a.L = sp.L - sp.g;  // local level count: the routing digit is the label's low g bits
  a.i = sp.L - 2 * sp.g;
  a.k = sp.g;
  a.attempt = attempt;
  a.seed = p->seed;
  a.ctrl = ctrl;
  a.trace = tr;
  a.bucket0 = (uint64_t)r * sp.Bl;
  if (sp.fast_final) {
    PermTableArgs ta{};
    ta.bucket0 = a.bucket0;
    ta.ord = (uint16_t*)(ws + pl.off_ord);
    ta.tag = a.in_tag;
    ta.load = (uint32_t*)(ws + pl.off_load);
    ta.B = sp.Bl;
    ta.Z = pl.Z;
    ta.attempt = attempt;
    ta.i = a.i;
    ta.k = a.k;
    ta.L = a.L;
    ta.buf_tag = a.buf_in_tag;
    ta.seed = p->seed;
    ta.trace = tr;
    BOS_CUDA(launch_perm_table(ta, st, tr.buf != nullptr));
    BOS_CUDA(launch_orp_fast(a, kModeLast, sp.kC, 0, st, pl.R, tr.buf != nullptr));
  } else {
    BOS_CUDA(launch_orp_pass(a, kModeLast, nsub, st, pl.R, tr.buf != nullptr));
  }
  Ctrl h{};
  unsigned long long last = 0;
  BOS_CUDA(cudaMemcpyAsync(&h, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
  BOS_CUDA(cudaMemcpyAsync(&last, ws + pl.off_status + (nsub - 1) * 8, 8, cudaMemcpyDeviceToHost, st));
  BOS_CUDA(cudaStreamSynchronize(st));
  if (h.timeout) return BOS_ERR_TIMEOUT;
  *h_overflow = h.overflow ? 1u : 0u;
  *h_count = last & kStValue;  // the last subproblem's inclusive prefix: the rank's reals
  if (!h.overflow && *h_count > out_cap) return BOS_ERR_INVALID;
  return BOS_OK;
}

bos_status bos_orp_out_of_core_bytes(uint64_t n, uint32_t G, const bos_params* p, size_t* dev_bytes,
                                     size_t* host_bytes) {
  ShardPlan sp;
  const bos_status s = shard_plan(n, G, p, &sp);
  if (s != BOS_OK) return s;
  if (!dev_bytes || !host_bytes) return BOS_ERR_INVALID;
  const uint64_t slice = (((sp.Bl * n) >> sp.L) + 2);  // input records of one rank, at most
  *dev_bytes = align256(sp.lp.total) + align256(slice * sp.lp.R) + align256(sp.Bl * p->Z * (uint64_t)sp.lp.R);
  *host_bytes = (size_t)G * G * (sp.chunk_rec + sp.chunk_tag);
  return BOS_OK;
}

bos_status bos_orp_out_of_core(const void* h_in, void* h_out, uint64_t n, const bos_params* p, uint32_t G,
                               void* d_buf, size_t dev_bytes, void* h_stage, size_t host_bytes, void* stream,
                               bos_info* info) {
  ShardPlan sp;
  bos_status s = shard_plan(n, G, p, &sp);
  if (s != BOS_OK) return s;
  size_t need_dev = 0, need_host = 0;
  bos_orp_out_of_core_bytes(n, G, p, &need_dev, &need_host);
  if (!h_in || !h_out || !d_buf || !h_stage || ((uintptr_t)d_buf & 255)) return BOS_ERR_INVALID;
  if (dev_bytes < need_dev || host_bytes < need_host) return BOS_ERR_WORKSPACE;
  const uint32_t R = sp.lp.R;
  const size_t ws_bytes = align256(sp.lp.total);
  const uint64_t slice = ((sp.Bl * n) >> sp.L) + 2;
  char* d_ws = (char*)d_buf;
  char* d_in = d_ws + ws_bytes;
  char* d_part = d_in + align256(slice * R);
  cudaStream_t st = (cudaStream_t)stream;
  const size_t per_rank = (size_t)G * (sp.chunk_rec + sp.chunk_tag);  // host: rank r's send regions
  char* hs = (char*)h_stage;
  const uint32_t max_attempts = p->max_attempts ? p->max_attempts : kDefaultAttempts;
  if (info) {
    info->L = sp.L;
    info->B = sp.B;
    info->passes = sp.lp.npass + 1;
    info->radix_passes = 0;
    info->max_cluster = sp.kC;
    info->max_k = sp.g;
    info->stream_passes = 0;
    for (uint32_t x = 0; x < sp.lp.npass; ++x) {
      info->max_k = sp.lp.pass_k[x] > info->max_k ? sp.lp.pass_k[x] : info->max_k;
      info->stream_passes += sp.lp.pass_stream[x] ? 1u : 0u;
    }
  }
  for (uint32_t attempt = 0; attempt < max_attempts; ++attempt) {
    // every rank's local levels; its send regions (G chunks of records, then of tags) to the host
    for (uint32_t r = 0; r < G; ++r) {
      uint64_t lo = 0, hi = 0;
      bos_shard_input_range(n, G, r, p, &lo, &hi);
      if (hi > lo) BOS_CUDA(cudaMemcpyAsync(d_in, (const char*)h_in + lo * R, (hi - lo) * R, cudaMemcpyHostToDevice, st));
      if ((s = bos_shard_local(d_in, n, G, r, p, attempt, d_ws, ws_bytes, stream)) != BOS_OK) return s;
      BOS_CUDA(cudaMemcpyAsync(hs + r * per_rank, d_ws + sp.send_rec, G * sp.chunk_rec, cudaMemcpyDeviceToHost, st));
      BOS_CUDA(cudaMemcpyAsync(hs + r * per_rank + G * sp.chunk_rec, d_ws + sp.send_tag, G * sp.chunk_tag,
                               cudaMemcpyDeviceToHost, st));
      // the local step's overflow flag is kept on the host: the next rank reuses the workspace
      Ctrl h{};
      BOS_CUDA(cudaMemcpyAsync(&h, d_ws + sp.lp.off_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
      BOS_CUDA(cudaStreamSynchronize(st));
      if (h.timeout) return BOS_ERR_TIMEOUT;
      if (h.overflow) goto next_attempt;  // the attempt fails everywhere
    }
    {
      // every rank's received chunks from the host, its last levels, its part to the host output
      uint64_t offset = 0;
      bool over = false;
      for (uint32_t d = 0; d < G && !over; ++d) {
        for (uint32_t r = 0; r < G; ++r) {
          BOS_CUDA(cudaMemcpyAsync(d_ws + sp.recv_rec + r * sp.chunk_rec, hs + r * per_rank + d * sp.chunk_rec,
                                   sp.chunk_rec, cudaMemcpyHostToDevice, st));
          BOS_CUDA(cudaMemcpyAsync(d_ws + sp.recv_tag + r * sp.chunk_tag,
                                   hs + r * per_rank + G * sp.chunk_rec + d * sp.chunk_tag, sp.chunk_tag,
                                   cudaMemcpyHostToDevice, st));
        }
        BOS_CUDA(zero_async(d_ws + sp.lp.off_ctrl, sizeof(Ctrl), st));
        uint64_t count = 0;
        uint32_t ovf = 0;
        if ((s = bos_shard_final(n, G, d, p, attempt, d_part, sp.Bl * p->Z, d_ws, ws_bytes, stream, &count, &ovf)) !=
            BOS_OK)
          return s;
        if (ovf) {
          over = true;
          break;
        }
        if (offset + count > n) return BOS_ERR_INVALID;
        if (count) BOS_CUDA(cudaMemcpyAsync((char*)h_out + offset * R, d_part, count * R, cudaMemcpyDeviceToHost, st));
        offset += count;
      }
      BOS_CUDA(cudaStreamSynchronize(st));
      if (!over) {
        if (info) info->attempts = attempt + 1;
        return offset == n ? BOS_OK : BOS_ERR_INVALID;
      }
    }
  next_attempt:;
  }
  if (info) info->attempts = max_attempts;
  return BOS_ERR_OVERFLOW;
}

bos_status bos_bitonic_sort(const void* d_in, void* d_out, uint64_t n, uint32_t rec_bytes,
                            uint32_t key_bytes, void* stream) {
  if (!((rec_bytes == 8 && key_bytes == 4) || (rec_bytes == 16 && key_bytes == 8))) return BOS_ERR_INVALID;
  if (n & (n - 1)) return BOS_ERR_INVALID;
  if (n == 0) return BOS_OK;
  if (!d_in || !d_out || ((uintptr_t)d_in & 15) || ((uintptr_t)d_out & 15)) return BOS_ERR_INVALID;
  if (d_in != d_out && overlaps(d_in, n * rec_bytes, d_out, n * rec_bytes)) return BOS_ERR_INVALID;
  const int ev = prof_begin((cudaStream_t)stream, kKBitonic, 0.0);
  const cudaError_t e = launch_bitonic(d_in, d_out, n, (int)rec_bytes, (cudaStream_t)stream);
  prof_end(ev, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return BOS_ERR_CUDA;
  }
  return BOS_OK;
}

bos_status bos_trace_attach(void* d_buf, size_t bytes) {
  std::lock_guard<std::mutex> g(g_state_mu);
  if (d_buf == nullptr) {
    g_trace = Trace{nullptr, 0, 0};
    return BOS_OK;
  }
  if (((uintptr_t)d_buf & 15) || bytes < 32) return BOS_ERR_INVALID;
  g_trace = Trace{(unsigned long long*)d_buf, (unsigned long long)(bytes / 16 - 1), 0};
  return BOS_OK;
}

bos_status bos_trace_attach_digest(void* d_buf, size_t bytes) {
  std::lock_guard<std::mutex> g(g_state_mu);
  if (d_buf == nullptr) {
    g_trace = Trace{nullptr, 0, 0};
    return BOS_OK;
  }
  if (((uintptr_t)d_buf & 15) || bytes < 256 * 16) return BOS_ERR_INVALID;
  g_trace = Trace{(unsigned long long*)d_buf, 0, 1};
  return BOS_OK;
}

const char* bos_status_str(bos_status s) {
  switch (s) {
    case BOS_OK: return "ok";
    case BOS_ERR_INVALID: return "invalid argument";
    case BOS_ERR_OVERFLOW: return "bucket overflow on every attempt";
    case BOS_ERR_WORKSPACE: return "workspace too small";
    case BOS_ERR_CUDA: return "CUDA error";
    case BOS_ERR_TIMEOUT: return "device-side wait timed out";
  }
  return "unknown status";
}

uint32_t bos_version(void) { return (0u << 16) | 1u; }

bos_status bos_profile_enable(int on) {
  std::lock_guard<std::mutex> g(g_state_mu);
  if (on && !g_prof.created) {
    for (int i = 0; i < 2 * kMaxEv; ++i)
      if (cudaEventCreate(&g_prof.ev[i]) != cudaSuccess) {
        (void)cudaGetLastError();
        return BOS_ERR_CUDA;
      }
    g_prof.created = true;
  }
  g_prof.on = on != 0;
  g_prof.pending = 0;
  for (int c = 0; c < kKCount; ++c) {
    g_prof.launches[c] = 0;
    g_prof.ms[c] = 0.0;
    g_prof.alg_bytes[c] = 0.0;
  }
  g_prof.total_launches = 0;
  return BOS_OK;
}

uint32_t bos_profile_read(bos_kernel_stat* out, uint32_t max, uint64_t* total_launches) {
  {  // bitonic calls do not synchronise: finish their events here
    std::unique_lock<std::mutex> g(g_state_mu);
    for (int i = 0; i < g_prof.pending; ++i) cudaEventSynchronize(g_prof.ev[2 * i + 1]);
  }
  prof_collect(0xFFFFFFFFu, 0u);
  std::lock_guard<std::mutex> g(g_state_mu);
  if (total_launches) *total_launches = g_prof.total_launches;
  uint32_t m = 0;
  for (int c = 0; c < kKCount && m < max; ++c) {
    if (!g_prof.launches[c]) continue;
    std::strncpy(out[m].name, kKNames[c], sizeof(out[m].name) - 1);
    out[m].name[sizeof(out[m].name) - 1] = 0;
    out[m].launches = (uint32_t)g_prof.launches[c];
    out[m].ms = g_prof.ms[c];
    out[m].bytes = g_prof.alg_bytes[c];
    ++m;
  }
  return m;
}

}  // extern "C"
