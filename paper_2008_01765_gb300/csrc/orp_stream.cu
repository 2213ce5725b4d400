// Streaming bucket ORP pass (sm_103a): the first pass and the middle passes of a fused plan.
//
// A pass applies k butterfly levels of Algorithm 3.1 (levels i..i+k-1): subproblem
// q = G*2^i + t reads the input buckets G*2^(i+k) + s*2^i + t (s < 2^k) and writes the contiguous
// output buckets q*2^k + u, each real going to u = label bits [L-1-i .. L-i-k], stable by (s, slot),
// then dummies (the MergeSplit order of the butterfly; Figure 1).
//
// The persistent-cluster kernel (orp_fast.cu) holds all 2^k output buckets on chip, which caps k
// by shared memory. This kernel streams instead: one CTA takes a whole subproblem and reads its
// input in order, in batches brought in by TMA bulk copies through a ring of stages: in the first
// pass a batch is two groups of input records (three stages); in a middle pass it is two input
// buckets (four one-bucket stages) when they fit, else one (three stages), so that the per-batch
// work (barriers, flushes, counter upkeep) is shared by about Z reals. Every output bucket owns a
// small ring of kRing slots in shared memory; a real is appended to its bucket's ring at its
// stable rank, and whenever a ring holds a whole chunk of kChunk slots the chunk leaves for HBM
// (coalesced 16-byte stores). At the end of the subproblem every bucket's last partial chunk is padded with dummies
// and its remaining chunks are written as dummies. So shared memory bounds the chunk buffers, not
// the subproblem, and one pass applies up to 9 levels with no cluster.
//
// Obliviousness (Section 3.1): reads are whole input buckets (or the whole input range of the
// groups); writes are whole chunks of kChunk slots, and every chunk of every output bucket is
// written exactly once. The multiset of addresses is therefore a function of (n, Z, k, pass) alone;
// only the order in which chunks leave depends on the labels, as in every GPU schedule here.
//
// Ranking inside a batch: each real takes a tentative ring position from a shared-memory atomic on
// its bucket's counter and records its slot index there; after a barrier a real whose bucket got
// several reals in this batch counts how many of them have a smaller slot index (usually zero to
// three), which is its stable rank. If a batch would add more reals to a ring than it has room
// for (rare: a ring keeps at most kChunk-1 slots between batches), the batch is redone in smaller
// rounds: halved while a round would overflow, kSub slots at the least.
//
// Overflow (MergeSplit receives more than Z reals, Lemma 3.2): the level-(i+l) buckets of the
// subproblem (l = 1..k-1) gather 2^l consecutive input buckets (2^(l-1) batches of the first pass)
// and the digits with a common l-bit prefix; per-batch digit counts are folded into one counter
// per (level, prefix) and checked at the end of each block. The final level is the ring's fill.
#include "common.cuh"
#include "internal.h"

namespace bos {
namespace {

constexpr int kST = 1024;
constexpr int kSW = kST / 32;
constexpr uint32_t kChunk = 8;         // slots per HBM write (128 B of 16-byte records)
constexpr uint32_t kRing = 24;         // ring slots per output bucket
constexpr uint32_t kRingStride = 25;   // ring pitch in shared memory (odd: spreads the banks)
constexpr uint32_t kStages = 3;        // input stages (first pass: batches; middle: buckets)
constexpr uint32_t kStagesPaired = 4;  // middle pass taking two input buckets per batch
constexpr uint32_t kSmemLimit = 232448 - 1024;  // opt-in shared memory per CTA less static use
constexpr uint32_t kMaxItems = 2;      // slots per thread per batch: Z <= 2048
constexpr uint32_t kSub = 16;          // slots per round when a batch is redone (7 + 16 <= kRing)
constexpr uint32_t kMinK = 5, kMaxK = 9;

struct StreamLayout {
  uint32_t ring_rec, ring_tag, aux, stage, stage_bytes, fill, done, cnt, lv, misc, total;
  uint32_t stages, pair;  // input stages; middle pass: two input buckets per batch (pair = 1)
};

__host__ __device__ inline uint32_t st_align(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline StreamLayout stream_layout_n(int R, uint32_t Z, uint32_t k, bool first, uint32_t stages,
                                                        uint32_t pair) {
  const uint32_t D = 1u << k;
  StreamLayout l{};
  l.stages = stages;
  l.pair = pair;
  uint32_t off = 0;
  l.ring_rec = off;
  off = st_align(off + D * kRingStride * R, 16);
  l.ring_tag = off;
  off = st_align(off + D * kRingStride * 4, 16);
  l.aux = off;
  off = st_align(off + D * kRingStride * 2, 16);
  // first pass: up to Z input records (two groups of at most Z/2) plus one record of alignment;
  // middle pass: one input bucket (tags, then records)
  l.stage_bytes = first ? st_align((Z + 2) * R, 128) : st_align(Z * (4 + R), 128);
  l.stage = st_align(off, 128);
  off = l.stage + stages * l.stage_bytes;
  l.fill = off;
  off += D * 4;
  l.done = off;
  off += D * 4;
  l.cnt = off;
  off += 2 * D * 4;
  l.lv = off;
  off += D * 4;
  l.misc = st_align(off, 16);
  off = l.misc + 64;
  l.total = off;
  return l;
}

// The middle pass takes two input buckets per batch (four single-bucket stages) when Z fits one
// item per thread per bucket, a batch's about Z reals average at most 8 per output bucket (more
// would overrun the rings) and the stages fit; otherwise one bucket per batch, three stages.
__host__ __device__ inline StreamLayout stream_layout(int R, uint32_t Z, uint32_t k, bool first) {
  if (!first && Z <= (uint32_t)kST && Z <= (8u << k)) {
    const StreamLayout p = stream_layout_n(R, Z, k, false, kStagesPaired, 1);
    if (p.total <= kSmemLimit) return p;
  }
  return stream_layout_n(R, Z, k, first, kStages, 0);
}

template <int R, bool FIRST, bool TRACE>
__global__ void __launch_bounds__(kST, 1) orp_stream_kernel(PassArgs a) {
  using Rec = typename RecT<R>::T;
  extern __shared__ __align__(128) unsigned char smem[];
  const uint32_t Z = a.Z, k = a.k, D = 1u << k, L = a.L, i = a.i;
  const uint32_t shift = L - i - k;
  const StreamLayout lay = stream_layout(R, Z, k, FIRST);
  Rec* ring_rec = reinterpret_cast<Rec*>(smem + lay.ring_rec);
  uint32_t* ring_tag = reinterpret_cast<uint32_t*>(smem + lay.ring_tag);
  uint16_t* aux = reinterpret_cast<uint16_t*>(smem + lay.aux);
  uint32_t* fill = reinterpret_cast<uint32_t*>(smem + lay.fill);  // reals appended per bucket
  uint32_t* done = reinterpret_cast<uint32_t*>(smem + lay.done);  // chunks written per bucket
  uint32_t* cnt = reinterpret_cast<uint32_t*>(smem + lay.cnt);    // [2][D] reals per round
  uint32_t* lv = reinterpret_cast<uint32_t*>(smem + lay.lv);      // level l, prefix p: lv[2^l - 2 + p]
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem + lay.misc);  // [lay.stages]
  volatile uint32_t* flag = reinterpret_cast<volatile uint32_t*>(smem + lay.misc + 32);  // [2]

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t nsub = a.B >> k;
  // units: what one stage holds (first pass: a batch of two groups; middle pass: one input
  // bucket); a batch is one unit, or two input buckets when the middle pass is paired
  const uint32_t NU = FIRST ? D / 2 : D;  // units per subproblem
  const uint32_t upb = (!FIRST && lay.pair) ? 2u : 1u;
  const uint32_t NB = NU / upb;  // batches per subproblem
  const uint32_t nst = lay.stages;
  const uint64_t mysub = blockIdx.x < nsub ? (nsub - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const uint64_t nbatch = mysub * NB, nunits = mysub * NU;
  const Rec* in_first = reinterpret_cast<const Rec*>(a.in);
  const Rec* in_rec = reinterpret_cast<const Rec*>(a.in_rec);
  Rec* out_rec = reinterpret_cast<Rec*>(a.out_rec);
  uint32_t* out_tag = a.out_tag;

  for (uint32_t x = tid; x < D; x += kST) {
    fill[x] = 0;
    done[x] = 0;
    cnt[x] = 0;
    cnt[D + x] = 0;
    lv[x] = 0;
  }
  if (tid == 0) {
    for (uint32_t s = 0; s < nst; ++s) mbar_init(smem_u32(bars + s), 1);
    flag[0] = flag[1] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // first pass: batch s of subproblem q = groups q*D + 2s and q*D + 2s + 1 (B = 2^L)
  auto first_range = [&](uint64_t q, uint32_t s, uint64_t& lo, uint64_t& hi) {
    const uint64_t g0 = a.bucket0 + q * D + 2ull * s;
    lo = (g0 * a.n) >> L;
    hi = ((g0 + 2) * a.n) >> L;
  };
  // Input records [lo, hi) of a first-pass batch sit at stage index soff + (record - lo); the
  // bulk copy takes [lo2, hi2), the largest sub-range whose global and shared addresses are both
  // 16-byte aligned (d_in is only guaranteed rec_bytes alignment).
  const uint32_t in_odd = R == 8 ? (uint32_t)((reinterpret_cast<uintptr_t>(a.in) >> 3) & 1u) : 0u;
  auto first_bulk = [&](uint64_t lo, uint64_t hi, uint64_t& lo2, uint64_t& hi2, uint32_t& soff) {
    if (R == 8) {
      lo2 = lo + ((lo + in_odd) & 1u);  // (d_in + 8 * lo2) is a multiple of 16
      hi2 = hi - ((hi + in_odd) & 1u);
      soff = (uint32_t)((lo2 - lo) & 1u);  // so that lo2's stage index is even
    } else {
      lo2 = lo;
      hi2 = hi;
      soff = 0;
    }
  };
  auto in_bucket = [&](uint64_t q, uint32_t s) -> uint64_t {
    const uint64_t t = q & ((1ull << i) - 1), G = q >> i;
    return (G << (i + k)) + ((uint64_t)s << i) + t;
  };
  // TMA of batch s of subproblem q into stage st (thread 0)
  auto issue = [&](uint64_t q, uint32_t s, uint32_t st) {
    const uint32_t bar = smem_u32(bars + st);
    const uint32_t dst = smem_u32(smem + lay.stage + st * lay.stage_bytes);
    if constexpr (FIRST) {
      uint64_t lo, hi;
      first_range(q, s, lo, hi);
      // a bulk copy starts and ends on 16-byte addresses: 8-byte records at the odd ends are
      // loaded by a thread (first_bulk)
      uint64_t lo2, hi2;
      uint32_t soff;
      first_bulk(lo, hi, lo2, hi2, soff);
      const uint32_t bytes = hi2 > lo2 ? (uint32_t)((hi2 - lo2) * R) : 0u;
      mbar_expect_tx(bar, bytes);
      if (bytes) tma_load(dst + (uint32_t)((lo2 - lo + soff) * R), in_first + lo2, bytes, bar);
      trace_log<TRACE>(a.trace, kRead, kBufIn, (uint32_t)((hi - lo) * R), lo * R);
    } else {
      const uint64_t bk = in_bucket(q, s);
      mbar_expect_tx(bar, Z * (4 + R));
      tma_load(dst, a.in_tag + bk * Z, Z * 4, bar);
      tma_load(dst + Z * 4, in_rec + bk * Z, Z * R, bar);
      trace_log<TRACE>(a.trace, kRead, a.buf_in_tag, Z * 4, bk * Z * 4);
      trace_log<TRACE>(a.trace, kRead, a.buf_in_rec, Z * R, bk * Z * R);
    }
  };

  // Writes every whole chunk of the subproblem's output buckets not yet written (done[u] counts
  // the chunks written; chunks at or past Z are never written: that bucket overflowed).
  auto flush_chunks = [&](uint64_t obase) {
    const uint32_t jj = lane & 7, grp = lane >> 3;
    for (uint32_t ub = 0; ub < D; ub += 32 * kSW) {
      const uint32_t u = ub + lane * kSW + warp;
      uint32_t d = 0, nch = 0;
      if (u < D) {
        d = done[u];
        const uint32_t c1 = min(fill[u] / kChunk, Z / kChunk);
        nch = c1 > d ? c1 - d : 0u;
      }
      uint32_t mask = __ballot_sync(0xFFFFFFFFu, nch > 0);
      while (mask) {
        uint32_t mm = mask;  // this 8-lane group serves the grp-th set lane of the mask
        for (uint32_t z = 0; z < grp && mm; ++z) mm &= mm - 1;
        const int src = mm ? __ffs(mm) - 1 : 0;
        const uint32_t su = __shfl_sync(0xFFFFFFFFu, u, src), sd = __shfl_sync(0xFFFFFFFFu, d, src);
        if (mm) {
          const uint32_t slot = sd * kChunk + jj, pos = su * kRingStride + slot % kRing;
          const uint64_t o = (obase + su) * Z + slot;
          out_rec[o] = ring_rec[pos];
          out_tag[o] = ring_tag[pos];
          if (jj == 0) {
            trace_log<TRACE>(a.trace, kWrite, a.buf_out_rec, kChunk * R, o * R);
            trace_log<TRACE>(a.trace, kWrite, a.buf_out_tag, kChunk * 4, o * 4);
          }
        }
        uint32_t rest = mask;  // the (up to) four lowest set lanes were served
        for (int z = 0; z < 4 && rest; ++z) rest &= rest - 1;
        if ((mask ^ rest) >> lane & 1u) {
          ++d;
          --nch;
        }
        mask = __ballot_sync(0xFFFFFFFFu, nch > 0);
      }
      if (u < D) done[u] = d;
    }
  };

  // Unit cursor (q, unit, stage), advanced without division; thread 0 keeps it nst units ahead
  // of the batches for the TMA issue.
  uint64_t iq = blockIdx.x;
  uint32_t is = 0, ist = 0;
  uint64_t issued = 0;
  auto issue_next = [&]() {
    issue(iq, is, ist);
    ++issued;
    if (++is == NU) {
      is = 0;
      iq += gridDim.x;
    }
    if (++ist == nst) ist = 0;
  };
  if (tid == 0)
    while (issued < nst && issued < nunits) issue_next();

  uint64_t q = blockIdx.x;
  uint32_t s = 0, st = 0, par = 0;  // batch s of subproblem q; stage and parity of its first unit
  for (uint64_t g = 0; g < nbatch; ++g) {
    const uint32_t pb = (uint32_t)(g & 1);
    const uint32_t st1 = st + 1 == nst ? 0u : st + 1, par1 = st + 1 == nst ? par ^ 1u : par;
    unsigned char* stg = smem + lay.stage + st * lay.stage_bytes;
    unsigned char* stg1 = smem + lay.stage + st1 * lay.stage_bytes;  // paired: the second bucket
    const uint32_t* stag = reinterpret_cast<const uint32_t*>(stg);
    const uint32_t* stag1 = reinterpret_cast<const uint32_t*>(stg1);
    Rec* srec = reinterpret_cast<Rec*>(FIRST ? stg : stg + Z * 4);
    Rec* srec1 = reinterpret_cast<Rec*>(stg1 + Z * 4);
    uint64_t lo = 0, hi = 0;
    uint32_t nslot = upb * Z, soff = 0;
    if constexpr (FIRST) {
      first_range(q, s, lo, hi);
      nslot = (uint32_t)(hi - lo);
      uint64_t lo2, hi2;
      first_bulk(lo, hi, lo2, hi2, soff);
      if (R == 8 && tid == kST - 1) {  // the records the bulk copy leaves out (odd ends)
        if (hi2 <= lo2) {  // at most two records, no bulk part
          for (uint32_t x = 0; x < nslot; ++x) srec[soff + x] = in_first[lo + x];
        } else {
          if (lo2 > lo) srec[soff] = in_first[lo];
          if (hi2 < hi) srec[soff + nslot - 1] = in_first[hi - 1];
        }
      }
    } else {
      mbar_wait(smem_u32(bars + st), par, a.ctrl);
      if (upb == 2) mbar_wait(smem_u32(bars + st1), par1, a.ctrl);
    }
    const uint64_t obase = q * D;
    uint32_t* cntp = cnt + pb * D;

    // One round over batch slots [rlo, rhi). check: give up (false) if a ring would overflow.
    auto round = [&](uint32_t rlo, uint32_t rhi, bool check) -> bool {
      uint32_t iu[kMaxItems], ifl[kMaxItems], itg[kMaxItems];
      // ---- A: tentative positions (atomics) and each real's slot index at its position ----
#pragma unroll
      for (uint32_t j = 0; j < kMaxItems; ++j) {
        const uint32_t x = rlo + tid + j * kST;
        iu[j] = D;
        ifl[j] = 0;
        itg[j] = kDummy;
        if (x < rhi) {
          uint32_t tg;
          if constexpr (FIRST)
            tg = label_of(lo + x, a.seed, a.attempt, L);
          else
            tg = x < Z ? stag[x] : stag1[x - Z];  // paired: slots Z.. are the second bucket's
          itg[j] = tg;
          if (tg != kDummy) {
            const uint32_t u = (tg >> shift) & (D - 1);
            const uint32_t f = fill[u];
            const uint32_t t = atomicAdd(&cntp[u], 1u);
            aux[u * kRingStride + (f + t) % kRing] = (uint16_t)x;
            if (check && t + (f - kChunk * done[u]) >= kRing) flag[pb] = 1u;
            iu[j] = u;
            ifl[j] = f;
          }
        }
      }
      __syncthreads();
      if (check && flag[pb]) {  // a ring would overflow: undo the counts and clear the flag
#pragma unroll
        for (uint32_t j = 0; j < kMaxItems; ++j)
          if (iu[j] < D) cntp[iu[j]] = 0u;
        __syncthreads();  // every thread has seen the flag
        if (tid == 0) flag[pb] = 0u;
        __syncthreads();  // cleared before the next round can raise it
        return false;
      }
      if constexpr (FIRST) mbar_wait(smem_u32(bars + st), par, a.ctrl);
      // ---- B: stable rank, append to the ring ----
#pragma unroll
      for (uint32_t j = 0; j < kMaxItems; ++j) {
        if (iu[j] < D) {
          const uint32_t u = iu[j], f = ifl[j], x = rlo + tid + j * kST, c = cntp[u];
          uint32_t r = 0;
          if (c > 1)
            for (uint32_t cc = 0; cc < c; ++cc) r += aux[u * kRingStride + (f + cc) % kRing] < x ? 1u : 0u;
          const uint32_t pos = u * kRingStride + (f + r) % kRing;
          ring_rec[pos] = (FIRST || x < Z) ? srec[soff + x] : srec1[x - Z];
          ring_tag[pos] = itg[j];
          if (r == 0) fill[u] = f + c;
        }
      }
      // level counters: per-digit counts of this round summed over groups of 2^g digits
      if ((uint32_t)tid < D) {
        uint32_t v = cntp[tid];
        for (uint32_t gsz = 1; gsz < k; ++gsz) {
          const uint32_t l = k - gsz;
          if (gsz <= 5) {
            v += __shfl_xor_sync(0xFFFFFFFFu, v, 1u << (gsz - 1));
            if ((tid & ((1u << gsz) - 1)) == 0 && v) lv[(1u << l) - 2 + (tid >> gsz)] += v;
          } else if (lane == 0 && v) {
            atomicAdd(&lv[(1u << l) - 2 + (tid >> gsz)], v);
          }
        }
      }
      __syncthreads();
      // ---- C: write the completed chunks. Lane l of warp w watches bucket l * kSW + w; the
      // buckets with a whole unwritten chunk are served four at a time (8 lanes per chunk) ----
      flush_chunks(obase);
      if ((uint32_t)tid < D) cntp[tid] = 0;
      return true;
    };

    if (!round(0, nslot, true)) {
      // a ring would overflow: redo the batch in smaller rounds, halving after every round that
      // would overflow (kSub slots at the least, which no ring can overflow) and doubling after
      // every round that fits
      uint32_t sz = nslot / 2 > kSub ? nslot / 2 : kSub;
      for (uint32_t sb = 0; sb < nslot;) {
        const uint32_t hi = sb + sz < nslot ? sb + sz : nslot;
        if (round(sb, hi, sz > kSub)) {
          sb = hi;
          sz = 2 * sz < nslot ? 2 * sz : nslot;
          __syncthreads();  // the next round reuses this round's counters
        } else {
          sz = sz / 2 > kSub ? sz / 2 : kSub;
        }
      }
    }
    // ---- after the batch: its stage is free; level blocks that end here are checked ----
    if (tid == 0) {
      flag[pb] = 0u;
      for (uint32_t x = 0; x < upb; ++x)
        if (issued < nunits) issue_next();
    }
    {  // level l's blocks end after every 2^l input buckets: 2^(l-1) batches of two (first pass,
      // paired middle pass), 2^l batches of one
      const uint32_t e = (FIRST || upb == 2) ? __ffs(~s) : __ffs(~s) - 1;  // levels 1..e end here
      const uint32_t lmax = e < k - 1 ? e : k - 1;
      for (uint32_t t = tid; t + 2 < (2u << lmax); t += kST) {
        if (lv[t] > Z) atomicExch(&a.ctrl->overflow, 1u);
        lv[t] = 0;
      }
    }
    if (s == NB - 1) {
      __syncthreads();  // every chunk written by the flushes is counted in done[]
      // ---- end of the subproblem: the last partial chunk of every bucket padded with dummies,
      // then its remaining chunks as dummies; the final loads are checked against Z ----
      for (uint32_t u = warp; u < D; u += kSW) {
        const uint32_t f = fill[u], d = done[u];
        if (lane == 0 && f > Z) atomicExch(&a.ctrl->overflow, 1u);
        const uint64_t ob = (obase + u) * Z;
        for (uint32_t slot = d * kChunk + lane; slot < Z; slot += 32) {
          const bool real = slot < f;
          const uint32_t pos = u * kRingStride + slot % kRing;
          out_rec[ob + slot] = real ? ring_rec[pos] : RecT<R>::zero();
          out_tag[ob + slot] = real ? ring_tag[pos] : kDummy;
          if ((slot & (kChunk - 1)) == 0) {
            trace_log<TRACE>(a.trace, kWrite, a.buf_out_rec, kChunk * R, (ob + slot) * R);
            trace_log<TRACE>(a.trace, kWrite, a.buf_out_tag, kChunk * 4, (ob + slot) * 4);
          }
        }
        __syncwarp();
        if (lane == 0) {
          fill[u] = 0;
          done[u] = 0;
        }
      }
      __syncthreads();
    }
    if (++s == NB) {
      s = 0;
      q += gridDim.x;
    }
    for (uint32_t x = 0; x < upb; ++x)
      if (++st == nst) {
        st = 0;
        par ^= 1u;
      }
  }
}

template <int R, bool FIRST, bool TRACE>
cudaError_t stream_launch(const PassArgs& a, cudaStream_t st) {
  const uint32_t smem = stream_layout(R, a.Z, a.k, FIRST).total;
  auto kern = orp_stream_kernel<R, FIRST, TRACE>;
  cudaError_t e = set_smem_optin(kern);
  if (e != cudaSuccess) return e;
  int per_sm = 0, sms = 0, dev = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kST, smem)) != cudaSuccess) return e;
  if (per_sm <= 0) return cudaErrorInvalidConfiguration;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const uint64_t nsub = a.B >> a.k;
  uint64_t grid = (uint64_t)per_sm * sms;
  if (grid > nsub) grid = nsub;
  if (grid == 0) return cudaSuccess;
  kern<<<(unsigned)grid, kST, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace


uint32_t orp_stream_smem_bytes(int R, uint32_t Z, uint32_t k, bool first) {
  return stream_layout(R, Z, k, first).total;
}

uint32_t orp_stream_max_k(int R, uint32_t Z, bool first, uint32_t smem_limit) {
  if (Z % 32 != 0 || Z > kMaxItems * kST) return 0;
  uint32_t best = 0;
  for (uint32_t k = kMinK; k <= kMaxK; ++k)
    if (stream_layout(R, Z, k, first).total <= smem_limit) best = k;
  return best;
}

cudaError_t launch_orp_stream(const PassArgs& a, bool first, cudaStream_t st, int R, bool trace) {
  if (a.k < kMinK || a.k > kMaxK || a.Z % 32 != 0 || a.Z > kMaxItems * kST || a.i + a.k > a.L)
    return cudaErrorInvalidValue;
  if (R == 8) {
    if (first) return trace ? stream_launch<8, true, true>(a, st) : stream_launch<8, true, false>(a, st);
    return trace ? stream_launch<8, false, true>(a, st) : stream_launch<8, false, false>(a, st);
  }
  if (first) return trace ? stream_launch<16, true, true>(a, st) : stream_launch<16, true, false>(a, st);
  return trace ? stream_launch<16, false, true>(a, st) : stream_launch<16, false, false>(a, st);
}

}  // namespace bos
