// C ABI of libbos (declared in include/bos.h): argument checks, pass planning, workspace layout
// and the attempt loop of Algorithm 3.1 (retry with a fresh attempt counter on overflow).
#include <cstring>
#include <mutex>

#include "bos.h"
#include "internal.h"

namespace bos {
namespace {

constexpr uint32_t kMaxSmem = 232448;  // opt-in dynamic shared memory per CTA on sm_100/103
constexpr uint32_t kMaxK = 6;          // per-pass digit-count table is (2^k)^2 words
constexpr uint32_t kMaxPasses = 32;
constexpr uint32_t kDefaultAttempts = 8;

Trace g_trace{nullptr, 0};

// ---- opt-in kernel timing (bos_profile_enable / bos_profile_read) ----
enum KClass { kKFirst, kKMid, kKLast, kKSingle, kKHist, kKPrep, kKRadix, kKRadixSkipped, kKBitonic, kKCount };
const char* const kKNames[kKCount] = {"orp_pass_first", "orp_pass_mid", "orp_pass_last", "orp_pass_single",
                                     "radix_hist", "radix_prep", "radix_pass", "radix_pass_skipped",
                                     "bitonic"};
constexpr int kMaxEv = 1024;
struct Prof {
  bool on = false;
  bool created = false;
  cudaEvent_t ev[2 * kMaxEv];
  int pending = 0;
  int cls[kMaxEv];
  double bytes[kMaxEv];
  uint32_t digit[kMaxEv];
  uint64_t launches[kKCount] = {};
  double ms[kKCount] = {};
  double alg_bytes[kKCount] = {};
  uint64_t total_launches = 0;
};
Prof g_prof;

// Records an event pair around one launch when profiling is on. Returns the slot or -1.
int prof_begin(cudaStream_t st, int cls, double bytes, uint32_t digit = 0) {
  g_prof.total_launches++;
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
// Folds the finished event pairs into the per-class totals (the stream has been synchronised).
void prof_collect(uint32_t radix_live) {
  for (int i = 0; i < g_prof.pending; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, g_prof.ev[2 * i], g_prof.ev[2 * i + 1]) != cudaSuccess) continue;
    int c = g_prof.cls[i];
    if (c == kKRadix && !((radix_live >> g_prof.digit[i]) & 1u)) c = kKRadixSkipped;
    g_prof.launches[c]++;
    g_prof.ms[c] += ms;
    g_prof.alg_bytes[c] += c == kKRadixSkipped ? 0.0 : g_prof.bytes[i];
  }
  g_prof.pending = 0;
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
  // workspace offsets
  size_t off_ctrl = 0, off_rec[2] = {0, 0}, off_tag[2] = {0, 0}, off_status = 0;
  size_t off_tmp = 0, off_hist = 0, off_dbase = 0, off_rstatus = 0, total = 0;
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
    // Cost model from GB300 measurements of the persistent kernel (time per slot of a butterfly
    // pass relative to the cluster-free kernel): a cluster applies more levels per pass but its
    // two cluster barriers per subproblem slow each pass. The first and the last pass (which
    // also draw labels or build the in-bin permutations) run without clusters; the middle levels
    // take the cluster size with the lowest total cost. Ties go to fewer passes.
    static const double kRel[5] = {1.0, 1.09, 1.37, 1.63, 2.46};  // C = 1, 2, 4, 8, 16
    uint32_t kf = max_k_fast(pl->R, p->Z, 1, false), kl = max_k_fast(pl->R, p->Z, 1, true);
    uint32_t ks = kl;  // single FIRST+LAST pass
    if (p->k) {
      kf = kf < p->k ? kf : p->k;
      kl = kl < p->k ? kl : p->k;
      ks = ks < p->k ? ks : p->k;
    }
    if (kf == 0 || kl == 0) return BOS_ERR_INVALID;  // (checked above)
    if (L <= ks) {
      pl->npass = 1;
      pl->pass_k[0] = L;
      pl->pass_C[0] = 1;
    } else {
      double best = 1e30;
      uint32_t best_f = 0, best_l = 0, best_C = 1, best_m = 0;
      for (uint32_t f = 1; f <= kf && f < L; ++f) {
        for (uint32_t l = 1; l <= kl && f + l <= L; ++l) {
          const uint32_t M = L - f - l;
          for (uint32_t ci = 0, C = 1; C <= max_C; ++ci, C <<= 1) {
            uint32_t km = max_k_fast(pl->R, p->Z, C, false);
            if (p->k) km = km < p->k ? km : p->k;
            if (M > 0 && km == 0) continue;
            const uint32_t m = M ? (M + km - 1) / km : 0;
            const double cost = 2.0 + m * (M ? kRel[ci] : 0.0) - 1e-3 * (f + l);
            if (cost < best - 1e-9) {
              best = cost;
              best_f = f;
              best_l = l;
              best_C = C;
              best_m = m;
            }
            if (!M) break;
          }
        }
      }
      if (best_f == 0 || 2 + best_m > kMaxPasses) return BOS_ERR_INVALID;
      const uint32_t M = L - best_f - best_l;
      pl->npass = 2 + best_m;
      pl->pass_k[0] = best_f;
      pl->pass_C[0] = 1;
      for (uint32_t x = 0; x < best_m; ++x) {
        pl->pass_k[1 + x] = M / best_m + (x < M % best_m);
        uint32_t C = 1;  // smallest cluster that holds this pass's levels
        while (C < best_C && (pl->pass_k[1 + x] > max_k_fast(pl->R, p->Z, C, false) || (1u << pl->pass_k[1 + x]) < C))
          C <<= 1;
        pl->pass_C[1 + x] = C;
      }
      pl->pass_k[pl->npass - 1] = best_l;
      pl->pass_C[pl->npass - 1] = 1;
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
  const uint32_t arrays = L >= 2 ? 2 : L;
  for (uint32_t x = 0; x < arrays; ++x) {
    pl->off_rec[x] = off; off = align256(off + slots * pl->R);
    pl->off_tag[x] = off; off = align256(off + slots * 4);
  }
  pl->orp_tiles = B >> pl->pass_k[pl->npass - 1];
  // sized for the largest last pass (k = 1) so the workspace does not depend on k
  pl->off_status = off; off = align256(off + B * 8);
  if (sort) {
    pl->radix_tiles = radix_tiles(n, pl->R);
    pl->off_tmp = off;     off = align256(off + n * pl->R);
    pl->off_hist = off;    off = align256(off + pl->digits * 256 * 4);
    pl->off_dbase = off;   off = align256(off + pl->digits * 256 * 8);
    pl->off_rstatus = off; off = align256(off + pl->radix_tiles * 256 * 8);
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
  bos_status s = n ? device_plan(n, p, sort, &pl) : make_plan(n, p, sort, &pl);
  if (s != BOS_OK) return s;
  if (info) {
    info->attempts = 0;
    info->L = pl.L;
    info->passes = pl.npass;
    info->radix_passes = 0;
    info->B = pl.B;
    info->max_cluster = 1;
    info->max_k = 0;
    for (uint32_t x = 0; x < pl.npass; ++x) {
      info->max_cluster = pl.pass_C[x] > info->max_cluster ? pl.pass_C[x] : info->max_cluster;
      info->max_k = pl.pass_k[x] > info->max_k ? pl.pass_k[x] : info->max_k;
    }
  }
  if (n == 0) return BOS_OK;
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
  const bool trace = g_trace.buf != nullptr;

  RadixArgs ra{};
  if (sort) {
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

  for (uint32_t attempt = 0; attempt < max_attempts; ++attempt) {
    BOS_CUDA(cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st));
    BOS_CUDA(cudaMemsetAsync(ws + pl.off_status, 0, pl.orp_tiles * 8, st));
    if (sort) {
      BOS_CUDA(cudaMemsetAsync(ra.hist, 0, pl.digits * 256 * 4, st));
      BOS_CUDA(cudaMemsetAsync(ra.status, 0, pl.radix_tiles * 256 * 8, st));
      int ev = prof_begin(st, kKHist, (double)n * pl.key_bytes);
      BOS_CUDA(launch_radix_hist(ra, pl.R, st));
      prof_end(ev, st);
      ev = prof_begin(st, kKPrep, 0.0);
      BOS_CUDA(launch_radix_prep(ra, pl.R, st));
      prof_end(ev, st);
    }
    for (uint32_t x = 0; x < pl.npass; ++x) {
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
        a.status = (unsigned long long*)(ws + pl.off_status);
        a.skip_publish = (p->flags & BOS_FLAG_SKIP_PUBLISH) ? 1u : 0u;
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
      a.trace = g_trace;
      const int mode = (first ? kModeFirst : 0) | (last ? kModeLast : 0);
      // algorithmic bytes: whole slot arrays in and out, the input and output records once
      const double slot_bytes = (double)pl.B * pl.Z * (pl.R + 4);
      const double in_b = first ? (double)n * pl.R : slot_bytes;
      const double out_b = last ? (double)n * pl.R : slot_bytes;
      const int cls = first && last ? kKSingle : first ? kKFirst : last ? kKLast : kKMid;
      const int ev = prof_begin(st, cls, in_b + out_b);
      if (pl.fast)
        BOS_CUDA(launch_orp_fast(a, mode, pl.pass_C[x], 0, st, pl.R, trace));
      else
        BOS_CUDA(launch_orp_pass(a, mode, pl.B >> a.k, st, pl.R, trace));
      prof_end(ev, st);
    }
    if (sort)
      for (uint32_t d = 0; d < pl.digits; ++d) {
        const int ev = prof_begin(st, kKRadix, 2.0 * n * pl.R, d);
        BOS_CUDA(launch_radix_pass(ra, pl.R, d, st));
        prof_end(ev, st);
      }
    Ctrl h{};
    BOS_CUDA(cudaMemcpyAsync(&h, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    BOS_CUDA(cudaStreamSynchronize(st));
    if (g_prof.on) prof_collect(h.radix_live);
    if (info) {
      info->attempts = attempt + 1;
      info->radix_passes = (uint32_t)__builtin_popcount(h.radix_live);
    }
    if (h.timeout) return BOS_ERR_TIMEOUT;
    if (h.overflow || attempt < forced) continue;
    return BOS_OK;
  }
  return BOS_ERR_OVERFLOW;
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
                                   const bos_params* base) {
  if (!h_offsets || !base) return 0;
  size_t best = 0;
  for (uint32_t j = 0; j < num; ++j) {
    bos_params p = *base;
    if (h_Z) p.Z = h_Z[j];
    const size_t w = bos_workspace_bytes(h_offsets[j + 1] - h_offsets[j], &p);
    best = w > best ? w : best;
  }
  return best;
}

bos_status bos_sort_batched(const void* d_in, void* d_out, const uint64_t* h_offsets, uint32_t num,
                            const uint64_t* h_seeds, const uint32_t* h_Z, const uint8_t* h_ops,
                            const bos_params* base, void* d_ws, size_t ws_bytes, void* stream,
                            uint32_t* h_attempts) {
  if (!h_offsets || !h_seeds || !h_ops || !base) return BOS_ERR_INVALID;
  for (uint32_t j = 0; j < num; ++j) {
    if (h_offsets[j + 1] < h_offsets[j]) return BOS_ERR_INVALID;
    bos_params p = *base;
    p.seed = h_seeds[j];
    if (h_Z) p.Z = h_Z[j];
    const uint64_t n = h_offsets[j + 1] - h_offsets[j];
    const size_t off = h_offsets[j] * base->rec_bytes;
    bos_info info{};
    const bos_status s = run((const char*)d_in + off, (char*)d_out + off, n, &p, d_ws, ws_bytes, stream,
                             &info, h_ops[j] != 0);
    if (h_attempts) h_attempts[j] = info.attempts;
    if (s != BOS_OK) return s;
  }
  return BOS_OK;
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
  if (d_buf == nullptr) {
    g_trace = Trace{nullptr, 0};
    return BOS_OK;
  }
  if (((uintptr_t)d_buf & 15) || bytes < 32) return BOS_ERR_INVALID;
  g_trace = Trace{(unsigned long long*)d_buf, (unsigned long long)(bytes / 16 - 1)};
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
  if (g_prof.pending) {  // bitonic calls do not synchronise: finish their events here
    for (int i = 0; i < g_prof.pending; ++i) cudaEventSynchronize(g_prof.ev[2 * i + 1]);
    prof_collect(0xFFFFFFFFu);
  }
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
