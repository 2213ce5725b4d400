// Oracle for bucket oblivious random permutation (ORP) and bucket oblivious sort.
//
// TEST INFRASTRUCTURE ONLY. This file is a plain, slow C++17 restatement of what the method
// computes, written from the paper (Asharov, Chan, Nayak, Pass, Ren, Shi,
// "Bucket Oblivious Sort: An Extremely Simple Oblivious Sort", SOSA 2020). Only the tests, the
// package's smoke check and the benchmark's CPU-baseline leg may load it. It shares no code,
// header, table or helper with the CUDA library; the two meet only through seeded inputs.
//
// Parity is pinned for every function here (see the tests): Philox against cuRAND's host
// generator, the literal butterfly against its closed form (a stable counting sort by label),
// the overflow test against its closed form and the binomial bounds of Lemma 3.2, the ORP
// against uniformity over all permutations (Lemma 3.3), the access count against Section 3.4,
// the sort against std::stable_sort / an LSD radix sort, the bitonic network against std::sort.
// Everything runs on one thread except or_sort_threads, the same literal algorithm with the
// independent work of each step split across std::threads (the threaded CPU baseline), which is
// pinned equal to the one-thread or_sort.
//
// Conventions (the paper leaves them open; each reading is listed in the design notes):
//   * B is the smallest power of two with B*Z >= 2n (Algorithm 3.1), L = log2 B.
//   * Group j of the input is [floor(j n / B), floor((j+1) n / B)) (Algorithm 3.1, "evenly divide").
//   * Level i routes on bit L-1-i of the L-bit label, the (i+1)-st most significant bit.
//   * MergeSplit is stable: reals of A_0 in slot order, then reals of A_1, then dummies.
//   * Labels: the top L bits of word 0 of Philox4x32-10(counter = (lo i, hi i, attempt, 0),
//     key = (lo seed, hi seed)). In-bin permutation: final bucket b, slot s gets the 64-bit
//     key (w0 << 32 | w1) of Philox4x32-10(counter = (lo(bZ+s), hi(bZ+s), attempt, 1)); the
//     reals are ordered by (key, s).
//   * Overflow ("more than Z" reals in a MergeSplit output) aborts the attempt; the next attempt
//     uses attempt+1 in every Philox counter.
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

// ---------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
// SC 2011): ten rounds of two 32x32->64 multiplies on counter words 0 and 2, the high halves
// mixed with the other two counter words and the round key; the key is bumped by the Weyl
// constants between rounds.
// ---------------------------------------------------------------------------------------------
constexpr uint32_t kMul0 = 0xD2511F53u;
constexpr uint32_t kMul1 = 0xCD9E8D57u;
constexpr uint32_t kWeyl0 = 0x9E3779B9u;
constexpr uint32_t kWeyl1 = 0xBB67AE85u;

void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += kWeyl0;
      k1 += kWeyl1;
    }
    const uint64_t p0 = (uint64_t)kMul0 * c0;
    const uint64_t p1 = (uint64_t)kMul1 * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n1 = lo1;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    const uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void philox_at(uint64_t index, uint32_t attempt, uint32_t stream, uint64_t seed, uint32_t out[4]) {
  const uint32_t ctr[4] = {(uint32_t)index, (uint32_t)(index >> 32), attempt, stream};
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  philox4x32_10(ctr, key, out);
}

// ---------------------------------------------------------------------------------------------
// Geometry (Algorithm 3.1): B = smallest power of two >= 2n/Z, i.e. the smallest power of two
// with B*Z >= 2n; L = log2 B.
// ---------------------------------------------------------------------------------------------
void geometry(uint64_t n, uint32_t Z, uint64_t* B, uint32_t* L) {
  uint64_t b = 1;
  uint32_t l = 0;
  while (b * (uint64_t)Z < 2 * n) {
    b <<= 1;
    ++l;
  }
  *B = b;
  *L = l;
}

// Random bin label of element i (Algorithm 3.1, "assign a uniformly random key in [0, B-1]").
uint32_t label_of(uint64_t i, uint64_t seed, uint32_t attempt, uint32_t L) {
  if (L == 0) return 0;
  uint32_t w[4];
  philox_at(i, attempt, 0, seed, w);
  return w[0] >> (32 - L);
}

// Group boundaries: group j = [floor(j n / B), floor((j+1) n / B)).
uint64_t group_lo(uint64_t j, uint64_t n, uint64_t B) {
  // j*n fits in 64 bits for every supported size (j < 2^32, n < 2^32).
  return (j * n) / B;
}

struct Slot {
  bool real;
  uint32_t label;
  uint64_t src;  // index of the element in the input array (carried so the record is copied once)
};

struct Counters {
  uint64_t reads = 0;
  uint64_t writes = 0;
};

// Trace entry: bit 63 = write, bits 56..62 = array index (level of A^(level)), bits 24..55 =
// bucket, bits 0..23 = slot.
struct Tracer {
  uint64_t* buf = nullptr;
  uint64_t cap = 0;
  uint64_t len = 0;
  void log(bool write, uint32_t level, uint64_t bucket, uint32_t slot) {
    if (buf && len < cap)
      buf[len] = ((uint64_t)write << 63) | ((uint64_t)(level & 0x7F) << 56) |
                 ((bucket & 0xFFFFFFFFull) << 24) | (uint64_t)(slot & 0xFFFFFF);
    ++len;
  }
};

// MergeSplit(A_0, A_1, i) of Algorithm 3.1. Reals whose routing bit is 0 go to A'_0, the rest to
// A'_1, each side stable (A_0's reals in slot order, then A_1's). Returns false on overflow,
// i.e. when either side receives more than Z reals.
bool merge_split(const Slot* a0, const Slot* a1, Slot* o0, Slot* o1, uint32_t Z, uint32_t bit,
                 Counters* cnt, Tracer* tr, uint32_t level, uint64_t ia0, uint64_t ia1,
                 uint64_t io0, uint64_t io1) {
  std::vector<Slot> side0, side1;
  const Slot* ins[2] = {a0, a1};
  const uint64_t in_ids[2] = {ia0, ia1};
  for (int h = 0; h < 2; ++h) {
    for (uint32_t s = 0; s < Z; ++s) {
      const Slot x = ins[h][s];
      cnt->reads++;
      if (tr) tr->log(false, level, in_ids[h], s);
      if (!x.real) continue;
      if ((x.label >> bit) & 1u)
        side1.push_back(x);
      else
        side0.push_back(x);
    }
  }
  if (side0.size() > Z || side1.size() > Z) return false;
  Slot* outs[2] = {o0, o1};
  const std::vector<Slot>* sides[2] = {&side0, &side1};
  const uint64_t out_ids[2] = {io0, io1};
  for (int h = 0; h < 2; ++h) {
    for (uint32_t s = 0; s < Z; ++s) {
      if (s < sides[h]->size())
        outs[h][s] = (*sides[h])[s];
      else
        outs[h][s] = Slot{false, 0, 0};
      cnt->writes++;
      if (tr) tr->log(true, level + 1, out_ids[h], s);
    }
  }
  return true;
}

// Literal Algorithm 3.1 for one attempt. On success, `final_buckets` holds A^(log B): B buckets
// of Z slots. Two arrays are used in turn for A^(i) and A^(i+1) (they hold the same contents as
// the paper's log B + 1 arrays).
bool bin_assignment_literal(uint64_t n, uint32_t Z, uint64_t seed, uint32_t attempt,
                            std::vector<Slot>* final_buckets, Counters* cnt, Tracer* tr) {
  uint64_t B;
  uint32_t L;
  geometry(n, Z, &B, &L);
  std::vector<Slot> cur(B * Z), nxt(B * Z);
  // Put group j into A^(0)_j and pad it with dummies to Z slots.
  for (uint64_t j = 0; j < B; ++j) {
    const uint64_t lo = group_lo(j, n, B), hi = group_lo(j + 1, n, B);
    for (uint32_t s = 0; s < Z; ++s) {
      if (lo + s < hi)
        cur[j * Z + s] = Slot{true, label_of(lo + s, seed, attempt, L), lo + s};
      else
        cur[j * Z + s] = Slot{false, 0, 0};
    }
  }
  for (uint32_t i = 0; i < L; ++i) {
    const uint32_t bit = L - 1 - i;
    for (uint64_t j = 0; j < B / 2; ++j) {
      const uint64_t jp = (j >> i) << i;  // j' = floor(j / 2^i) * 2^i
      const uint64_t a = jp + j, b = jp + j + (1ull << i);
      if (!merge_split(&cur[a * Z], &cur[b * Z], &nxt[(2 * j) * Z], &nxt[(2 * j + 1) * Z], Z, bit,
                       cnt, tr, i, a, b, 2 * j, 2 * j + 1))
        return false;
    }
    std::swap(cur, nxt);
  }
  *final_buckets = std::move(cur);
  return true;
}

// Closed form of the butterfly (Figure 1 caption: after level i every 2^i consecutive buckets
// are semi-sorted by the top i label bits). The level-i bucket G*2^i + t holds exactly the
// reals of groups [G 2^i, (G+1) 2^i) whose top i label bits equal t, in input order. So the
// attempt overflows iff one of those counts exceeds Z, and the final bucket b holds the elements
// with label b in input order (a stable counting sort by label).
bool overflow_closed(uint64_t n, uint32_t Z, uint64_t seed, uint32_t attempt) {
  uint64_t B;
  uint32_t L;
  geometry(n, Z, &B, &L);
  std::vector<uint32_t> labels(n);
  std::vector<uint64_t> group(n);
  for (uint64_t j = 0; j < B; ++j)
    for (uint64_t e = group_lo(j, n, B); e < group_lo(j + 1, n, B); ++e) group[e] = j;
  for (uint64_t e = 0; e < n; ++e) labels[e] = label_of(e, seed, attempt, L);
  for (uint32_t i = 1; i <= L; ++i) {
    std::vector<uint64_t> count(B, 0);
    for (uint64_t e = 0; e < n; ++e) {
      const uint64_t G = group[e] >> i;
      const uint64_t t = labels[e] >> (L - i);
      if (++count[(G << i) | t] > Z) return true;
    }
  }
  return false;
}

bool bin_assignment_closed(uint64_t n, uint32_t Z, uint64_t seed, uint32_t attempt,
                           std::vector<Slot>* final_buckets) {
  if (overflow_closed(n, Z, seed, attempt)) return false;
  uint64_t B;
  uint32_t L;
  geometry(n, Z, &B, &L);
  std::vector<uint64_t> fill(B, 0);
  final_buckets->assign(B * Z, Slot{false, 0, 0});
  for (uint64_t e = 0; e < n; ++e) {
    const uint32_t b = label_of(e, seed, attempt, L);
    (*final_buckets)[b * Z + fill[b]] = Slot{true, b, e};
    fill[b]++;
  }
  return true;
}

// Section 3.2: strip the dummies of every final bucket (they follow the reals), permute each
// bucket randomly and concatenate. The permutation of bucket b orders its m reals by the key
// (r(b,s), s), r(b,s) = 64-bit Philox stream-1 word pair at position b*Z + s.
void permute_and_strip(const std::vector<Slot>& fin, uint64_t B, uint32_t Z, uint64_t seed,
                       uint32_t attempt, const uint8_t* in, uint8_t* out, uint32_t rec_bytes,
                       uint32_t* loads) {
  uint64_t pos = 0;
  for (uint64_t b = 0; b < B; ++b) {
    uint32_t m = 0;
    while (m < Z && fin[b * Z + m].real) ++m;
    if (loads) loads[b] = m;
    std::vector<std::pair<uint64_t, uint32_t>> keyed(m);
    for (uint32_t s = 0; s < m; ++s) {
      uint32_t w[4];
      philox_at(b * Z + s, attempt, 1, seed, w);
      keyed[s] = {((uint64_t)w[0] << 32) | w[1], s};
    }
    std::sort(keyed.begin(), keyed.end());
    for (uint32_t j = 0; j < m; ++j) {
      const Slot& x = fin[b * Z + keyed[j].second];
      std::memcpy(out + (pos + j) * rec_bytes, in + x.src * rec_bytes, rec_bytes);
    }
    pos += m;
  }
}

uint64_t key_of(const uint8_t* rec, uint32_t key_bytes) {
  if (key_bytes == 4) {
    uint32_t k;
    std::memcpy(&k, rec, 4);
    return k;
  }
  uint64_t k;
  std::memcpy(&k, rec, 8);
  return k;
}

uint64_t payload_of(const uint8_t* rec, uint32_t rec_bytes, uint32_t key_bytes) {
  uint64_t p = 0;
  std::memcpy(&p, rec + key_bytes, std::min<uint32_t>(8, rec_bytes - key_bytes));
  return p;
}

// Runs f(lo, hi) on `threads` std::threads over contiguous ranges of [0, count).
template <typename F>
void parallel_ranges(uint64_t count, uint32_t threads, F f) {
  if (threads <= 1 || count < 2) {
    f(0, count);
    return;
  }
  std::vector<std::thread> pool;
  for (uint32_t t = 0; t < threads; ++t) {
    const uint64_t lo = count * t / threads, hi = count * (t + 1) / threads;
    if (lo < hi) pool.emplace_back(f, lo, hi);
  }
  for (auto& th : pool) th.join();
}

// Literal Algorithm 3.1 as bin_assignment_literal, with the placement of the groups and the
// B/2 MergeSplits of every level (independent of one another) split across threads.
bool bin_assignment_literal_mt(uint64_t n, uint32_t Z, uint64_t seed, uint32_t attempt,
                               std::vector<Slot>* final_buckets, uint32_t threads) {
  uint64_t B;
  uint32_t L;
  geometry(n, Z, &B, &L);
  std::vector<Slot> cur(B * Z), nxt(B * Z);
  parallel_ranges(B, threads, [&](uint64_t j0, uint64_t j1) {
    for (uint64_t j = j0; j < j1; ++j) {
      const uint64_t lo = group_lo(j, n, B), hi = group_lo(j + 1, n, B);
      for (uint32_t s = 0; s < Z; ++s)
        cur[j * Z + s] = lo + s < hi ? Slot{true, label_of(lo + s, seed, attempt, L), lo + s} : Slot{false, 0, 0};
    }
  });
  for (uint32_t i = 0; i < L; ++i) {
    const uint32_t bit = L - 1 - i;
    std::atomic<bool> failed{false};
    parallel_ranges(B / 2, threads, [&](uint64_t j0, uint64_t j1) {
      Counters cnt;
      for (uint64_t j = j0; j < j1 && !failed.load(std::memory_order_relaxed); ++j) {
        const uint64_t jp = (j >> i) << i;
        const uint64_t a = jp + j, b = jp + j + (1ull << i);
        if (!merge_split(&cur[a * Z], &cur[b * Z], &nxt[(2 * j) * Z], &nxt[(2 * j + 1) * Z], Z, bit,
                         &cnt, nullptr, i, a, b, 2 * j, 2 * j + 1))
          failed.store(true);
      }
    });
    if (failed.load()) return false;
    std::swap(cur, nxt);
  }
  *final_buckets = std::move(cur);
  return true;
}

// permute_and_strip with the buckets split across threads (offsets from the loads first).
void permute_and_strip_mt(const std::vector<Slot>& fin, uint64_t B, uint32_t Z, uint64_t seed,
                          uint32_t attempt, const uint8_t* in, uint8_t* out, uint32_t rec_bytes,
                          uint32_t threads) {
  std::vector<uint64_t> start(B + 1, 0);
  for (uint64_t b = 0; b < B; ++b) {
    uint32_t m = 0;
    while (m < Z && fin[b * Z + m].real) ++m;
    start[b + 1] = start[b] + m;
  }
  parallel_ranges(B, threads, [&](uint64_t b0, uint64_t b1) {
    for (uint64_t b = b0; b < b1; ++b) {
      const uint32_t m = (uint32_t)(start[b + 1] - start[b]);
      std::vector<std::pair<uint64_t, uint32_t>> keyed(m);
      for (uint32_t s = 0; s < m; ++s) {
        uint32_t w[4];
        philox_at(b * Z + s, attempt, 1, seed, w);
        keyed[s] = {((uint64_t)w[0] << 32) | w[1], s};
      }
      std::sort(keyed.begin(), keyed.end());
      for (uint32_t j = 0; j < m; ++j)
        std::memcpy(out + (start[b] + j) * rec_bytes, in + fin[b * Z + keyed[j].second].src * rec_bytes, rec_bytes);
    }
  });
}

// Stable LSD radix sort on 8-bit digits with each pass split across threads: every thread
// counts its contiguous range, the offsets are the per-digit prefix over (digit, thread), and
// every thread scatters its range in order (so equal digits keep their order).
void radix_sort_mt(uint8_t* r, uint64_t n, uint32_t rec_bytes, uint32_t key_bytes, uint32_t threads) {
  if (threads < 1) threads = 1;
  std::vector<uint8_t> tmp(n * rec_bytes);
  uint8_t* src = r;
  uint8_t* dst = tmp.data();
  std::vector<uint64_t> cnt((size_t)threads * 256);
  for (uint32_t d = 0; d < key_bytes; ++d) {
    std::fill(cnt.begin(), cnt.end(), 0);
    parallel_ranges(threads, threads, [&](uint64_t t0, uint64_t t1) {
      for (uint64_t t = t0; t < t1; ++t)
        for (uint64_t i = n * t / threads; i < n * (t + 1) / threads; ++i) cnt[t * 256 + src[i * rec_bytes + d]]++;
    });
    uint64_t run = 0;
    for (int v = 0; v < 256; ++v)
      for (uint32_t t = 0; t < threads; ++t) {
        const uint64_t c = cnt[(size_t)t * 256 + v];
        cnt[(size_t)t * 256 + v] = run;
        run += c;
      }
    parallel_ranges(threads, threads, [&](uint64_t t0, uint64_t t1) {
      for (uint64_t t = t0; t < t1; ++t)
        for (uint64_t i = n * t / threads; i < n * (t + 1) / threads; ++i) {
          const uint8_t v = src[i * rec_bytes + d];
          std::memcpy(dst + (cnt[t * 256 + v]++) * rec_bytes, src + i * rec_bytes, rec_bytes);
        }
    });
    std::swap(src, dst);
  }
  if (src != r) std::memcpy(r, src, n * rec_bytes);
}

struct OrpInfo {
  uint32_t attempts;
  uint32_t L;
  uint64_t B;
  uint64_t slot_reads;   // MergeSplit slot reads of the successful attempt
  uint64_t slot_writes;  // MergeSplit slot writes of the successful attempt
};

}  // namespace

extern "C" {

enum { OR_OK = 0, OR_ERR_INVALID = 1, OR_ERR_OVERFLOW = 2 };

void or_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  philox4x32_10(ctr, key, out);
}

void or_philox_many(uint64_t count, const uint32_t* ctrs, const uint32_t* keys, uint32_t* out) {
  for (uint64_t i = 0; i < count; ++i) philox4x32_10(ctrs + 4 * i, keys + 2 * i, out + 4 * i);
}

void or_geometry(uint64_t n, uint32_t Z, uint64_t* B, uint32_t* L) { geometry(n, Z, B, L); }

// Test hook: the boundaries out[j] = group_lo(j), j = 0..B, of the B groups Algorithm 3.1's
// placement divides the input into (the literal and closed forms both place by these).
void or_group_bounds(uint64_t n, uint32_t Z, uint64_t* out) {
  uint64_t B;
  uint32_t L;
  geometry(n, Z, &B, &L);
  for (uint64_t j = 0; j <= B; ++j) out[j] = group_lo(j, n, B);
}

void or_labels(uint64_t n, uint64_t seed, uint32_t attempt, uint32_t L, uint32_t* out) {
  for (uint64_t i = 0; i < n; ++i) out[i] = label_of(i, seed, attempt, L);
}

// Overflow of one attempt, by running the literal butterfly (method 0) or the closed form (1).
int or_overflow(uint64_t n, uint32_t Z, uint64_t seed, uint32_t attempt, int method) {
  if (method == 1) return overflow_closed(n, Z, seed, attempt) ? 1 : 0;
  std::vector<Slot> fin;
  Counters c;
  return bin_assignment_literal(n, Z, seed, attempt, &fin, &c, nullptr) ? 0 : 1;
}

// Number of seeds in [seed0, seed0 + nseeds) whose attempt `attempt` overflows.
uint64_t or_overflow_count(uint64_t n, uint32_t Z, uint64_t seed0, uint64_t nseeds,
                           uint32_t attempt, int method) {
  uint64_t c = 0;
  for (uint64_t s = 0; s < nseeds; ++s) c += (uint64_t)or_overflow(n, Z, seed0 + s, attempt, method);
  return c;
}

// Bucket ORP (Section 3.2) of n records of rec_bytes each. method 0 runs the literal
// Algorithm 3.1; method 1 its closed form. Attempts first_attempt .. max_attempts-1 are tried
// in order (or_orp starts at attempt 0). `loads` (nullable, B entries) receives the final
// bucket loads; `trace` (nullable) receives the literal run's access trace of the successful
// attempt (trace_len gets the full length even if it exceeds trace_cap).
int or_orp_from(const void* in, void* out, uint64_t n, uint32_t rec_bytes, uint32_t Z,
                uint64_t seed, uint32_t first_attempt, uint32_t max_attempts, int method,
                OrpInfo* info, uint32_t* loads, uint64_t* trace, uint64_t trace_cap,
                uint64_t* trace_len) {
  if (Z < 1 || (rec_bytes != 8 && rec_bytes != 16) || max_attempts < 1) return OR_ERR_INVALID;
  uint64_t B;
  uint32_t L;
  geometry(n, Z, &B, &L);
  if (info) {
    info->B = B;
    info->L = L;
  }
  for (uint32_t a = first_attempt; a < max_attempts; ++a) {
    std::vector<Slot> fin;
    Counters cnt;
    Tracer tr;
    tr.buf = trace;
    tr.cap = trace_cap;
    const bool ok = method == 1 ? bin_assignment_closed(n, Z, seed, a, &fin)
                                : bin_assignment_literal(n, Z, seed, a, &fin, &cnt,
                                                         trace ? &tr : nullptr);
    if (!ok) continue;
    permute_and_strip(fin, B, Z, seed, a, (const uint8_t*)in, (uint8_t*)out, rec_bytes, loads);
    if (info) {
      info->attempts = a + 1;
      info->slot_reads = cnt.reads;
      info->slot_writes = cnt.writes;
    }
    if (trace_len) *trace_len = tr.len;
    return OR_OK;
  }
  if (info) info->attempts = max_attempts;
  return OR_ERR_OVERFLOW;
}

int or_orp(const void* in, void* out, uint64_t n, uint32_t rec_bytes, uint32_t Z, uint64_t seed,
           uint32_t max_attempts, int method, OrpInfo* info, uint32_t* loads, uint64_t* trace,
           uint64_t trace_cap, uint64_t* trace_len) {
  return or_orp_from(in, out, n, rec_bytes, Z, seed, 0, max_attempts, method, info, loads, trace,
                     trace_cap, trace_len);
}

// Sampled ORP output at any size (Section 3.2 restated bucket by bucket, from the closed form of
// the butterfly): for attempt `attempt`, final bucket b holds the elements labelled b in input
// order; the output places bucket b at the sum of the loads of the buckets before it, its reals
// ordered by the in-bin keys (r(b,s), s). For each requested bucket the call returns its output
// offset and load, and appends the input indices of its reals in output order to `src`.
// Returns OR_ERR_INVALID when `src` is too small. (No overflow check: callers sample runs that
// reported no overflow.)
int or_orp_sample(uint64_t n, uint32_t Z, uint64_t seed, uint32_t attempt, const uint64_t* buckets,
                  uint32_t nb, uint64_t* offset, uint32_t* load, uint64_t* src, uint64_t cap) {
  uint64_t B;
  uint32_t L;
  geometry(n, Z, &B, &L);
  std::vector<uint32_t> labels(n);
  std::vector<uint64_t> loads(B, 0);
  for (uint64_t i = 0; i < n; ++i) {
    labels[i] = label_of(i, seed, attempt, L);
    loads[labels[i]]++;
  }
  std::vector<uint64_t> starts(B + 1, 0);
  for (uint64_t b = 0; b < B; ++b) starts[b + 1] = starts[b] + loads[b];
  // members of every sampled bucket, in input order (one scan)
  std::vector<int64_t> which(B, -1);
  for (uint32_t x = 0; x < nb; ++x) {
    if (buckets[x] >= B) return OR_ERR_INVALID;
    which[buckets[x]] = x;
  }
  std::vector<std::vector<uint64_t>> mem(nb);
  for (uint64_t i = 0; i < n; ++i)
    if (which[labels[i]] >= 0) mem[which[labels[i]]].push_back(i);
  uint64_t pos = 0;
  for (uint32_t x = 0; x < nb; ++x) {
    const uint64_t b = buckets[x];
    offset[x] = starts[b];
    load[x] = (uint32_t)loads[b];
    const std::vector<uint64_t>& members = mem[which[b]];
    const uint32_t m = (uint32_t)members.size();
    std::vector<std::pair<uint64_t, uint32_t>> keyed(m);
    for (uint32_t s = 0; s < m; ++s) {
      uint32_t w[4];
      philox_at(b * Z + s, attempt, 1, seed, w);
      keyed[s] = {((uint64_t)w[0] << 32) | w[1], s};
    }
    std::sort(keyed.begin(), keyed.end());
    if (pos + m > cap) return OR_ERR_INVALID;
    for (uint32_t j = 0; j < m; ++j) src[pos + j] = members[keyed[j].second];
    pos += m;
  }
  return OR_OK;
}

// ORP of one small array under `count` consecutive seeds; out receives count * n records.
int or_orp_many(const void* in, void* out, uint64_t n, uint32_t rec_bytes, uint32_t Z,
                uint64_t seed0, uint64_t count, uint32_t max_attempts, int method,
                uint32_t* attempts_out) {
  for (uint64_t s = 0; s < count; ++s) {
    OrpInfo info{};
    const int st = or_orp(in, (uint8_t*)out + s * n * rec_bytes, n, rec_bytes, Z, seed0 + s,
                          max_attempts, method, &info, nullptr, nullptr, 0, nullptr);
    if (attempts_out) attempts_out[s] = info.attempts;
    if (st != OR_OK) return st;
  }
  return OR_OK;
}

// Stable ascending sort by the unsigned key at offset 0 (std::stable_sort).
void or_stable_sort(void* recs, uint64_t n, uint32_t rec_bytes, uint32_t key_bytes) {
  uint8_t* r = (uint8_t*)recs;
  std::vector<uint64_t> idx(n);
  for (uint64_t i = 0; i < n; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](uint64_t a, uint64_t b) {
    return key_of(r + a * rec_bytes, key_bytes) < key_of(r + b * rec_bytes, key_bytes);
  });
  std::vector<uint8_t> tmp(n * rec_bytes);
  for (uint64_t i = 0; i < n; ++i) std::memcpy(&tmp[i * rec_bytes], r + idx[i] * rec_bytes, rec_bytes);
  std::memcpy(r, tmp.data(), tmp.size());
}

// Stable LSD radix sort by key, 8-bit digits, least significant first (a second, independent
// sort used to cross-check std::stable_sort).
void or_radix_sort(void* recs, uint64_t n, uint32_t rec_bytes, uint32_t key_bytes) {
  uint8_t* r = (uint8_t*)recs;
  std::vector<uint8_t> tmp(n * rec_bytes);
  uint8_t* src = r;
  uint8_t* dst = tmp.data();
  for (uint32_t d = 0; d < key_bytes; ++d) {
    uint64_t count[257] = {0};
    for (uint64_t i = 0; i < n; ++i) count[src[i * rec_bytes + d] + 1]++;
    for (int v = 0; v < 256; ++v) count[v + 1] += count[v];
    for (uint64_t i = 0; i < n; ++i) {
      const uint8_t v = src[i * rec_bytes + d];
      std::memcpy(dst + (count[v]++) * rec_bytes, src + i * rec_bytes, rec_bytes);
    }
    std::swap(src, dst);
  }
  if (src != r) std::memcpy(r, src, n * rec_bytes);
}

// Bucket oblivious sort (Section 3.3): ORP, then a non-oblivious stable sort by key. method
// selects the ORP form (0 literal, 1 closed form); sorter 0 = std::stable_sort, 1 = LSD radix.
int or_sort(const void* in, void* out, uint64_t n, uint32_t rec_bytes, uint32_t key_bytes,
            uint32_t Z, uint64_t seed, uint32_t max_attempts, int method, int sorter,
            OrpInfo* info) {
  if (key_bytes != 4 && key_bytes != 8) return OR_ERR_INVALID;
  if (key_bytes >= rec_bytes) return OR_ERR_INVALID;
  const int st = or_orp(in, out, n, rec_bytes, Z, seed, max_attempts, method, info, nullptr,
                        nullptr, 0, nullptr);
  if (st != OR_OK) return st;
  if (sorter == 1)
    or_radix_sort(out, n, rec_bytes, key_bytes);
  else
    or_stable_sort(out, n, rec_bytes, key_bytes);
  return OR_OK;
}

// or_sort (literal ORP, then the LSD radix sort) with the work of each step split across
// `threads` std::threads: the threaded CPU baseline. Same output as or_sort(method 0, sorter 1).
int or_sort_threads(const void* in, void* out, uint64_t n, uint32_t rec_bytes, uint32_t key_bytes,
                    uint32_t Z, uint64_t seed, uint32_t max_attempts, uint32_t threads, OrpInfo* info) {
  if (key_bytes != 4 && key_bytes != 8) return OR_ERR_INVALID;
  if (key_bytes >= rec_bytes || (rec_bytes != 8 && rec_bytes != 16) || Z < 1 || max_attempts < 1)
    return OR_ERR_INVALID;
  uint64_t B;
  uint32_t L;
  geometry(n, Z, &B, &L);
  if (info) {
    info->B = B;
    info->L = L;
  }
  for (uint32_t a = 0; a < max_attempts; ++a) {
    std::vector<Slot> fin;
    if (!bin_assignment_literal_mt(n, Z, seed, a, &fin, threads)) continue;
    permute_and_strip_mt(fin, B, Z, seed, a, (const uint8_t*)in, (uint8_t*)out, rec_bytes, threads);
    radix_sort_mt((uint8_t*)out, n, rec_bytes, key_bytes, threads);
    if (info) {
      info->attempts = a + 1;
      info->slot_reads = 2ull * B * Z * L;
      info->slot_writes = 2ull * B * Z * L;
    }
    return OR_OK;
  }
  if (info) info->attempts = max_attempts;
  return OR_ERR_OVERFLOW;
}

// Bitonic sorting network (Batcher 1968; the comparator of Table 1) on n = 2^m records,
// ordered by (key, payload). Returns OR_ERR_INVALID when n is not a power of two.
int or_bitonic_sort(void* recs, uint64_t n, uint32_t rec_bytes, uint32_t key_bytes) {
  if (n & (n - 1)) return OR_ERR_INVALID;
  uint8_t* r = (uint8_t*)recs;
  std::vector<uint8_t> t(rec_bytes);
  auto less = [&](uint64_t a, uint64_t b) {
    const uint64_t ka = key_of(r + a * rec_bytes, key_bytes), kb = key_of(r + b * rec_bytes, key_bytes);
    if (ka != kb) return ka < kb;
    return payload_of(r + a * rec_bytes, rec_bytes, key_bytes) <
           payload_of(r + b * rec_bytes, rec_bytes, key_bytes);
  };
  for (uint64_t k = 2; k <= n; k <<= 1) {
    for (uint64_t j = k >> 1; j > 0; j >>= 1) {
      for (uint64_t i = 0; i < n; ++i) {
        const uint64_t l = i ^ j;
        if (l <= i) continue;
        const bool ascending = (i & k) == 0;
        if (ascending ? less(l, i) : less(i, l)) {
          std::memcpy(t.data(), r + i * rec_bytes, rec_bytes);
          std::memcpy(r + i * rec_bytes, r + l * rec_bytes, rec_bytes);
          std::memcpy(r + l * rec_bytes, t.data(), rec_bytes);
        }
      }
    }
  }
  return OR_OK;
}

}  // extern "C"
