// Bucket ORP passes, persistent and cluster-wide (sm_103a). Used when Z is a multiple of 32.
//
// Same computation as orp.cu (k butterfly levels of Algorithm 3.1 per HBM pass; subproblem
// q = G*2^i + t reads input buckets G*2^(i+k) + s*2^i + t, s < 2^k, and writes the contiguous
// output buckets q*2^k + u, u = label bits [L-1-i .. L-i-k], stable by (s, slot)), organised for
// GB300:
//   * A cluster of C CTAs (C = 1..16) works on one subproblem; CTA c owns the input buckets and
//     the output buckets [c*Dc, (c+1)*Dc), Dc = 2^k / C. Its output buckets live in its shared
//     memory; reals routed to another CTA's bucket are stored there through distributed shared
//     memory. C CTAs hold C times the client storage of one, so one pass applies more levels.
//   * The kernel is persistent: each cluster loops over subproblems. Input tags arrive by TMA
//     bulk copies (prefetched one subproblem ahead); records are loaded into registers at the
//     start of a subproblem so their latency overlaps the counting and the cluster exchange;
//     the finished tile leaves by TMA bulk stores while the next subproblem starts.
//   * Ranking is stable and warp-local: each warp owns a contiguous run of rows (32 slots) of
//     the CTA's input stream, finds the peers of each slot with the match instruction (a warp
//     holds at most 2^k + 1 distinct digits), and keeps running per-digit counters; a
//     per-(warp, digit) prefix over warps and CTAs gives every real its output slot.
// Every global address depends only on (n, Z, k, C, pass, subproblem): whole input buckets are
// read, whole output buckets are written (Section 3.1). Label-dependent movement stays in shared
// memory (local or distributed).
//
// LAST pass: each final bucket's in-bin permutation (Section 3.2) arrives as a row of the table
// that perm_table.cu sorted ahead of the pass (slots in key order, TMA-loaded per subproblem);
// after the routing each CTA writes its reals compacted, in row order without the entries >= the
// bucket's load, at the prefix of the final loads found by a decoupled look-back over the
// subproblems (ticket order).
#include "common.cuh"
#include "internal.h"

namespace bos {

namespace {

constexpr int kT = 512;
constexpr int kW = kT / 32;
constexpr int kRowsMax = 16;  // rows of 32 slots a warp keeps in registers per round

__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_id_x() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_count_x() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t mapa(uint32_t local, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_cluster_u32(uint32_t addr, uint32_t v) {
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void st_cluster_u64(uint32_t addr, unsigned long long v) {
  asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
}
__device__ __forceinline__ void st_cluster_rec(uint32_t addr, const uint2& v) {
  asm volatile("st.shared::cluster.v2.u32 [%0], {%1, %2};" ::"r"(addr), "r"(v.x), "r"(v.y) : "memory");
}
__device__ __forceinline__ void st_cluster_rec(uint32_t addr, const uint4& v) {
  asm volatile("st.shared::cluster.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z),
               "r"(v.w)
               : "memory");
}

struct FastLayout {
  uint32_t tile_rec, tile_tag, tags, rc, h, aggs, tot, moff, misc, total;
  uint32_t perm, perm_bytes;  // LAST: in-bin permutation scratch
};

__host__ __device__ inline uint32_t fl_align(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline FastLayout fast_layout(int R, uint32_t Z, uint32_t k, uint32_t C, bool last) {
  FastLayout l{};
  const uint32_t D = 1u << k, Dc = D / C, S = Dc * Z;
  uint32_t off = 0;
  l.tile_rec = off; off = fl_align(off + S * R, 128);
  l.tile_tag = off; off = fl_align(off + S * 4, 128);   // LAST: inverse permutations (u16)
  l.tags = off;     off = fl_align(off + S * 4, 128);   // staged input tags of the CTA
  l.rc = off;       off = fl_align(off + kW * D * 4, 16);
  l.h = off;        off = fl_align(off + Dc * D * 4, 16);
  l.aggs = off;     off = fl_align(off + C * D * 4, 16);
  l.tot = off;      off = fl_align(off + D * 4, 16);
  l.moff = off;     off = fl_align(off + (Dc + 1) * 4, 16);
  l.misc = off;     off = fl_align(off + 128, 16);
  // LAST: the CTA's rows of the in-bin permutation table (u16 per slot) use the tag tile; the
  // filter keeps one count per 32 table entries and one partial sum per warp.
  l.perm_bytes = 0;
  l.perm = off;
  if (last) {
    l.perm_bytes = (S / 32 + kW) * 4;
    off = fl_align(off + l.perm_bytes, 16);
  }
  l.total = off;
  return l;
}

// misc words
constexpr int kMiscBar = 0;     // mbarrier (8 bytes)
constexpr int kMiscNext = 2;    // next subproblem (u64 in words 2..3)
constexpr int kMiscPrefix = 4;  // LAST: subproblem output prefix (u64 in words 4..5)
constexpr int kMiscBefore = 8;  // LAST: reals of the lower-ranked CTAs of the subproblem
constexpr int kMiscTotal = 10;  // LAST: reals of the subproblem (u64 in words 10..11)
constexpr int kMiscBarOrd = 12;  // LAST: mbarrier of the permutation table rows (8 bytes)

template <int R, int MODE, bool CL, bool TRACE>
__global__ void __launch_bounds__(kT, 1) orp_fast_kernel(PassArgs a, uint32_t C) {
  using Rec = typename RecT<R>::T;
  constexpr bool FIRST = MODE & kModeFirst;
  constexpr bool LAST = MODE & kModeLast;
  extern __shared__ __align__(128) unsigned char smem[];

  const uint32_t Z = a.Z, k = a.k, D = 1u << k, Dc = D / C, S = Dc * Z;
  const uint32_t rows_per_bucket = Z >> 5, NR = S >> 5;
  const FastLayout lay = fast_layout(R, Z, k, C, LAST);
  Rec* tile_rec = reinterpret_cast<Rec*>(smem + lay.tile_rec);
  uint32_t* tile_tag = reinterpret_cast<uint32_t*>(smem + lay.tile_tag);
  uint16_t* ordl = reinterpret_cast<uint16_t*>(smem + lay.tile_tag);  // LAST: own table rows
  uint32_t* tags = reinterpret_cast<uint32_t*>(smem + lay.tags);
  uint32_t* rc = reinterpret_cast<uint32_t*>(smem + lay.rc);      // [kW][D]
  uint32_t* h = reinterpret_cast<uint32_t*>(smem + lay.h);        // [Dc][D]
  uint32_t* aggs = reinterpret_cast<uint32_t*>(smem + lay.aggs);  // [C][D]
  uint32_t* tot = reinterpret_cast<uint32_t*>(smem + lay.tot);    // [D]
  uint32_t* misc = reinterpret_cast<uint32_t*>(smem + lay.misc);
  const uint32_t bar = smem_u32(misc + kMiscBar);
  const uint32_t bar_ord = smem_u32(misc + kMiscBarOrd);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lt_mask = lanemask_lt();
  const uint32_t crank = CL ? cluster_ctarank() : 0u;
  const uint64_t cid = CL ? cluster_id_x() : blockIdx.x;
  const uint64_t ncl = CL ? cluster_count_x() : gridDim.x;
  const uint32_t i = a.i, L = a.L;
  const uint32_t shift = L - i - k;
  const uint64_t nsub = a.B >> k;
  const uint32_t r0 = (uint32_t)(((uint64_t)warp * NR) / kW), r1 = (uint32_t)(((uint64_t)(warp + 1) * NR) / kW);
  const uint32_t nrows = r1 - r0;
  // this warp's first row as (own input bucket, row inside it); later rows advance incrementally
  const uint32_t sp0 = r0 / rows_per_bucket, rr0 = r0 - sp0 * rows_per_bucket;
  const uint32_t lg_dc = (uint32_t)(__ffs(Dc) - 1);  // Dc is a power of two
  const Rec* in_rec = reinterpret_cast<const Rec*>(FIRST ? a.in : a.in_rec);

  // ---- set-up ----
  if (tid == 0) {
    mbar_init(bar, 1);
    if constexpr (LAST) mbar_init(bar_ord, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (uint32_t x = tid; x < kW * D; x += kT) rc[x] = 0;
  for (uint32_t x = tid; x < Dc * D; x += kT) h[x] = 0;
  // first subproblem: static for the butterfly passes, ticket for the LAST pass
  // (LAST with clusters: only rank 0 writes the word, into every CTA, so a late local write can
  // never overwrite the ticket it pushed)
  if (tid == 0 && (!LAST || !CL || crank == 0)) {
    uint64_t q0 = cid;
    if constexpr (LAST) q0 = atomicAdd(&a.ctrl->tickets[a.ticket_slot], 1u);
    *reinterpret_cast<unsigned long long*>(misc + kMiscNext) = q0;
  }
  __syncthreads();
  if constexpr (LAST && CL) {
    // rank 0's ticket to every CTA of the cluster
    if (tid == 0 && crank == 0) {
      const unsigned long long q0 = *reinterpret_cast<unsigned long long*>(misc + kMiscNext);
      for (uint32_t c = 1; c < C; ++c) st_cluster_u64(mapa(smem_u32(misc + kMiscNext), c), q0);
    }
  }
  if constexpr (CL) cluster_sync();

  uint64_t q = *reinterpret_cast<unsigned long long*>(misc + kMiscNext);
  uint32_t parity = 0, parity_ord = 0;

  // input bucket (global index) of own input bucket s' of subproblem qq
  auto in_bucket = [&](uint64_t qq, uint32_t sp) -> uint64_t {
    const uint64_t t = qq & ((1ull << i) - 1), G = qq >> i;
    return (G << (i + k)) + ((uint64_t)(crank * Dc + sp) << i) + t;
  };
  // TMA of the CTA's input tags for subproblem qq (butterfly passes after the first)
  auto issue_tags = [&](uint64_t qq) {
    if constexpr (!FIRST) {
      if (tid == 0 && qq < nsub) {
        mbar_expect_tx(bar, S * 4);
        for (uint32_t sp = 0; sp < Dc; ++sp) {
          const uint64_t bk = in_bucket(qq, sp);
          tma_load(smem_u32(tags + sp * Z), a.in_tag + bk * Z, Z * 4, bar);
          trace_log<TRACE>(a.trace, kRead, a.buf_in_tag, Z * 4, bk * Z * 4);
        }
      }
    }
  };
  // Records of this warp's rows go to registers at the start of a subproblem; their latency
  // overlaps the counting and the exchange.
  // Row cursor: (sp, rr) = own input bucket and row inside it; base = that bucket's first slot
  // in the input array (FIRST: its group's first record; lim = the group's size).
  auto bucket_base = [&](uint64_t qq, uint32_t sp, uint64_t& base, uint32_t& lim) {
    if constexpr (FIRST) {
      const uint64_t g = a.bucket0 + qq * D + crank * Dc + sp;
      const uint64_t lo = (g * a.n) >> L, hi = ((g + 1) * a.n) >> L;  // group g, B = 2^L
      base = lo;
      lim = (uint32_t)(hi - lo);
    } else {
      base = in_bucket(qq, sp) * Z;
      lim = Z;
    }
  };
  auto load_rows = [&](uint64_t qq, uint32_t first, uint32_t count, Rec* dst) {
    uint32_t sp = sp0, rr = rr0 + first;
    while (rr >= rows_per_bucket) {
      rr -= rows_per_bucket;
      ++sp;
    }
    uint64_t base;
    uint32_t lim;
    bucket_base(qq, sp, base, lim);
#pragma unroll
    for (int j = 0; j < kRowsMax; ++j) {
      if ((uint32_t)j < count) {
        const uint32_t sl = rr * 32 + lane;
        dst[j] = RecT<R>::zero();
        if (sl < lim) {
          dst[j] = in_rec[base + sl];
          trace_log<TRACE>(a.trace, kRead, FIRST ? (uint32_t)kBufIn : a.buf_in_rec, R, (base + sl) * R);
        }
        if (++rr == rows_per_bucket) {
          rr = 0;
          ++sp;
          if ((uint32_t)j + 1 < count) bucket_base(qq, sp, base, lim);
        }
      }
    }
  };
  Rec rr[kRowsMax];
  const uint32_t rows0 = nrows < (uint32_t)kRowsMax ? nrows : (uint32_t)kRowsMax;
  issue_tags(q);

  while (q < nsub) {
    if constexpr (LAST) {
      // the table rows of own final buckets q*2^k + crank*Dc + up, up < Dc: one contiguous run
      // (the tag tile is free: the previous subproblem's filter ended with a barrier)
      if (tid == 0) {
        const uint64_t first = (q * D + crank * Dc) * (uint64_t)Z;
        mbar_expect_tx(bar_ord, S * 2);
        tma_load(smem_u32(ordl), a.ord + first, S * 2, bar_ord);
        trace_log<TRACE>(a.trace, kRead, kBufPerm, S * 2, first * 2);
      }
    }
    load_rows(q, 0, rows0, rr);
    // FIRST: labels into the tag stage; later passes: wait for the tags' TMA
    if constexpr (FIRST) {
      // Rows past a group's records hold only dummies (each warp writes its own); the rows with
      // records are spread over all warps, two per step, so the labels' Philox chains overlap.
      {
        uint32_t sp = sp0, rrow = rr0;
        uint64_t base;
        uint32_t lim;
        bucket_base(q, sp, base, lim);
        for (uint32_t row = r0; row < r1; ++row) {
          if (rrow * 32 >= lim) tags[row * 32 + lane] = kDummy;
          if (++rrow == rows_per_bucket) {
            rrow = 0;
            ++sp;
            if (row + 1 < r1) bucket_base(q, sp, base, lim);
          }
        }
      }
      // Data row d of the CTA lies in the first own bucket whose data rows, summed from bucket 0,
      // exceed d. A thread's d only grows, so one cursor (bucket spc, its first data row dst)
      // walks the buckets once.
      uint32_t spc = 0, dst = 0, limc;
      uint64_t basec;
      bucket_base(q, 0, basec, limc);
      auto data_row = [&](uint32_t d, uint32_t& row, uint64_t& base, uint32_t& lim) -> bool {
        while (d >= dst + ((limc + 31) >> 5)) {
          dst += (limc + 31) >> 5;
          if (++spc >= Dc) return false;
          bucket_base(q, spc, basec, limc);
        }
        row = spc * rows_per_bucket + (d - dst);
        base = basec;
        lim = limc;
        return true;
      };
      for (uint32_t d0 = warp;; d0 += 2 * kW) {
        uint32_t row0 = 0, row1 = 0, lim0 = 0, lim1 = 0;
        uint64_t base0 = 0, base1 = 0;
        if (!data_row(d0, row0, base0, lim0)) break;
        const bool v1 = data_row(d0 + kW, row1, base1, lim1);
        const uint32_t sl0 = (row0 - (row0 / rows_per_bucket) * rows_per_bucket) * 32 + lane;
        if (v1) {
          const uint32_t sl1 = (row1 - (row1 / rows_per_bucket) * rows_per_bucket) * 32 + lane;
          const uint32_t t0 = label_of(base0 + sl0, a.seed, a.attempt, L);
          const uint32_t t1 = label_of(base1 + sl1, a.seed, a.attempt, L);
          tags[row0 * 32 + lane] = sl0 < lim0 ? t0 : kDummy;
          tags[row1 * 32 + lane] = sl1 < lim1 ? t1 : kDummy;
        } else {
          const uint32_t t0 = label_of(base0 + sl0, a.seed, a.attempt, L);
          tags[row0 * 32 + lane] = sl0 < lim0 ? t0 : kDummy;
          break;
        }
      }
      __syncthreads();  // rows were labelled by other warps
    } else {
      mbar_wait(bar, parity, a.ctrl);
      parity ^= 1u;
    }

    // ---- phase 1: per-warp digit counts and per-input-bucket digit counts (atomics) ----
    uint32_t* rcw = rc + warp * D;
    {
      uint32_t sp = sp0, rrow = rr0;
      for (uint32_t row = r0; row < r1; ++row) {
        const uint32_t tg = tags[row * 32 + lane];
        if (tg != kDummy) {
          const uint32_t u = (tg >> shift) & (D - 1);
          atomicAdd(&rcw[u], 1u);
          atomicAdd(&h[sp * D + u], 1u);
        }
        if (++rrow == rows_per_bucket) {
          rrow = 0;
          ++sp;
        }
      }
    }
    __syncthreads();

    // ---- phase 2: CTA aggregates, exchange across the cluster, offsets, overflow ----
    for (uint32_t u = tid; u < D; u += kT) {
      uint32_t run = 0;
      for (int w = 0; w < kW; ++w) {
        const uint32_t x = rc[w * D + u];
        rc[w * D + u] = run;
        run += x;
      }
      if constexpr (CL) {
        const uint32_t local = smem_u32(aggs + crank * D + u);
        for (uint32_t c = 0; c < C; ++c) st_cluster_u32(mapa(local, c), run);
      } else {
        aggs[u] = run;
      }
    }
    // the previous tile must have left shared memory before anyone writes into it again
    if (tid == 0) tma_store_wait_read();
    if constexpr (CL)
      cluster_sync();
    else
      __syncthreads();
    for (uint32_t u = tid; u < D; u += kT) {
      uint32_t base = 0, total = 0;
      for (uint32_t c = 0; c < C; ++c) {
        const uint32_t x = aggs[c * D + u];
        if constexpr (CL) base += c < crank ? x : 0u;  // no earlier CTA without a cluster
        total += x;
      }
      tot[u] = total;
      for (int w = 0; w < kW; ++w) rc[w * D + u] += base;
    }
    __syncthreads();
    // overflow (MergeSplit: more than Z reals) at every level i+l, l = 1..k, of this subproblem.
    // Level-(i+l) bucket (sigma, pi) gathers input buckets [sigma 2^l, (sigma+1) 2^l) and the
    // digits with l-bit prefix pi. Rows of h (own input buckets) and of aggs (whole CTAs) are
    // turned into inclusive prefix sums over the digit, one warp per row; a bucket's count is
    // then a difference per input bucket (inside this CTA) or per CTA (wider blocks, checked by
    // the CTA that holds the block's first input bucket).
    for (uint32_t row = warp; row < Dc + C; row += kW) {
      uint32_t* hr = row < Dc ? h + row * D : aggs + (row - Dc) * D;
      uint32_t carry = 0;
      for (uint32_t u0 = 0; u0 < D; u0 += 32) {
        const uint32_t u = u0 + lane;
        uint32_t v = u < D ? hr[u] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, v, o);
          if (lane >= o) v += y;
        }
        v += carry;
        if (u < D) hr[u] = v;
        carry = __shfl_sync(0xFFFFFFFFu, v, 31);
      }
    }
    __syncthreads();
    for (uint32_t x = tid; x < k * D; x += kT) {
      const uint32_t l = x / D + 1, bkt = x - (l - 1) * D;
      const uint32_t sigma = bkt >> l, pi = bkt & ((1u << l) - 1);
      const uint32_t s_lo = sigma << l, s_hi = (sigma + 1) << l;
      const uint32_t u_lo = pi << (k - l), u_hi = (pi + 1) << (k - l);
      uint32_t cnt = 0;
      bool mine = false;
      if ((1u << l) <= Dc) {
        if (s_lo >= crank * Dc && s_lo < (crank + 1) * Dc) {
          mine = true;
          for (uint32_t s = s_lo; s < s_hi; ++s) {
            const uint32_t* hr = h + (s - crank * Dc) * D;
            cnt += hr[u_hi - 1] - (u_lo ? hr[u_lo - 1] : 0u);
          }
        }
      } else if (s_lo == crank * Dc) {
        mine = true;
        for (uint32_t c = s_lo / Dc; c < s_hi / Dc; ++c) {
          const uint32_t* ar = aggs + c * D;
          cnt += ar[u_hi - 1] - (u_lo ? ar[u_lo - 1] : 0u);
        }
      }
      if (mine && cnt > Z) atomicExch(&a.ctrl->overflow, 1u);
    }
    __syncthreads();
    for (uint32_t x = tid; x < Dc * D; x += kT) h[x] = 0;  // read above; next use after a barrier

    if constexpr (LAST) {
      // ---- publish this subproblem's reals (rank 0, one thread): the look-back that gives its
      // output offset runs after the routing, when the predecessors have had time to finish ----
      if (crank == 0 && tid == kT - 32) {
        unsigned long long total = 0;
        for (uint32_t u = 0; u < D; ++u) total += min(tot[u], Z);
        const bool skip = a.skip_publish && q == 0;
        if (!skip) st_status(a.status + q, st_word(q == 0 ? kStIncl : kStAgg, 0, total));
        *reinterpret_cast<unsigned long long*>(misc + kMiscTotal) = total;
      }
    }

    // ---- phase 3: route every real to its output slot (own tile or a peer's tile) ----
    for (uint32_t base_row = 0; base_row < nrows; base_row += kRowsMax) {
      const uint32_t cnt = nrows - base_row < (uint32_t)kRowsMax ? nrows - base_row : (uint32_t)kRowsMax;
      if (base_row > 0) load_rows(q, base_row, cnt, rr);  // further rounds: the next rows' records
#pragma unroll
      for (int j = 0; j < kRowsMax; ++j) {
        if ((uint32_t)j < cnt) {
          const uint32_t row = r0 + base_row + j;
          const uint32_t tg = tags[row * 32 + lane];
          const bool real = tg != kDummy;
          const uint32_t u = (tg >> shift) & (D - 1);
          const uint32_t peers = __match_any_sync(0xFFFFFFFFu, real ? u : 0xFFFFFFFFu);
          const uint32_t lt = __popc(peers & lt_mask);
          const uint32_t dst = real ? rcw[u] + lt : 0u;
          __syncwarp();
          if (real && lt == 0) rcw[u] += __popc(peers);
          if (real && dst < Z) {
            const uint32_t owner = u >> lg_dc, up = u & (Dc - 1);
            const uint32_t slot = up * Z + dst;
            if constexpr (CL) {
              st_cluster_rec(mapa(smem_u32(tile_rec + slot), owner), rr[j]);
              if constexpr (!LAST) st_cluster_u32(mapa(smem_u32(tile_tag + slot), owner), tg);
            } else {
              tile_rec[slot] = rr[j];
              if constexpr (!LAST) tile_tag[slot] = tg;
            }
          }
          __syncwarp();
        }
      }
    }
    if constexpr (LAST) {
      // ---- decoupled look-back of the subproblem's output offset (rank 0, one thread) ----
      if (crank == 0 && tid == kT - 32) {
        unsigned long long prefix = 0;
        if (q > 0) {
          const unsigned long long total = *reinterpret_cast<unsigned long long*>(misc + kMiscTotal);
          prefix = lookback_window<8>(a.status, q, 1, 0, a.ctrl);
          st_status(a.status + q, st_word(kStIncl, 0, prefix + total));
        }
        if constexpr (CL) {
          const uint32_t local = smem_u32(misc + kMiscPrefix);
          for (uint32_t c = 0; c < C; ++c) st_cluster_u64(mapa(local, c), prefix);
        } else {
          *reinterpret_cast<unsigned long long*>(misc + kMiscPrefix) = prefix;
        }
      }
    }
    // next subproblem index
    if (tid == 0) {
      uint64_t qn = q + ncl;
      if constexpr (LAST) {
        if (crank == 0) qn = atomicAdd(&a.ctrl->tickets[a.ticket_slot], 1u);
        if constexpr (CL) {
          if (crank == 0)
            for (uint32_t c = 0; c < C; ++c) st_cluster_u64(mapa(smem_u32(misc + kMiscNext), c), qn);
        } else {
          *reinterpret_cast<unsigned long long*>(misc + kMiscNext) = qn;
        }
      } else {
        *reinterpret_cast<unsigned long long*>(misc + kMiscNext) = qn;
      }
    }
    for (uint32_t x = lane; x < D; x += 32) rcw[x] = 0;  // this warp's counters for the next subproblem
    if constexpr (CL)
      cluster_sync();  // every remote store into this CTA's tile has landed
    else
      __syncthreads();
    const uint64_t qnext = *reinterpret_cast<unsigned long long*>(misc + kMiscNext);
    issue_tags(qnext);  // the tag stage is free: prefetch the next subproblem's tags
    // The next subproblem's first records are requested once this thread's tile writes are fenced
    // for the TMA store (the proxy fence would otherwise wait for these loads too).

    if constexpr (!LAST) {
      // ---- phase 4: pad with dummies, TMA the Dc contiguous output buckets out ----
      for (uint32_t up = 0; up < Dc; ++up) {
        const uint32_t first = min(tot[crank * Dc + up], Z);
        for (uint32_t sl = first + tid; sl < Z; sl += kT) {
          tile_tag[up * Z + sl] = kDummy;
          tile_rec[up * Z + sl] = RecT<R>::zero();
        }
      }
      fence_proxy_async();
      __syncthreads();
      if (tid == 0) {
        const uint64_t obase = (q * D + crank * Dc) * (uint64_t)Z;
        tma_store(reinterpret_cast<Rec*>(a.out_rec) + obase, smem_u32(tile_rec), S * R);
        tma_store(a.out_tag + obase, smem_u32(tile_tag), S * 4);
        tma_store_commit();
        trace_log<TRACE>(a.trace, kWrite, a.buf_out_rec, S * R, obase * R);
        trace_log<TRACE>(a.trace, kWrite, a.buf_out_tag, S * 4, obase * 4);
      }
    } else {
      // ---- LAST: write own reals compacted, in permuted order ----
      // Bucket up's reals sit at slots s < m = min(tot, Z); its table row lists all Z slots in key
      // order, so its output is the row with the entries >= m dropped. Every 32 entries give one
      // ballot; an exclusive scan of the ballot counts over the CTA's rows places them.
      if (tid == 0) {
        uint32_t before = 0;  // reals of lower-ranked CTAs of this subproblem
        for (uint32_t u = 0; u < crank * Dc; ++u) before += min(tot[u], Z);
        misc[kMiscBefore] = before;
      }
      uint32_t* ccnt = reinterpret_cast<uint32_t*>(smem + lay.perm);  // [S/32]
      uint32_t* cw = ccnt + S / 32;                                     // [kW]
      const uint32_t cpb = Z >> 5, nch = S >> 5;                        // chunks per bucket, in all
      mbar_wait(bar_ord, parity_ord, a.ctrl);
      parity_ord ^= 1u;
      for (uint32_t c = warp; c < nch; c += kW) {
        const uint32_t up = c / cpb, m = min(tot[crank * Dc + up], Z);
        const uint32_t keep = __ballot_sync(0xFFFFFFFFu, ordl[c * 32 + lane] < m);
        if (lane == 0) ccnt[c] = __popc(keep);
      }
      __syncthreads();
      {  // exclusive scan of ccnt: thread t takes chunks [t*per, (t+1)*per)
        const uint32_t per = (nch + kT - 1) / kT, c0 = tid * per, c1 = min(c0 + per, nch);
        uint32_t sum = 0;
        for (uint32_t c = c0; c < c1; ++c) sum += ccnt[c];
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
          if (lane >= o) incl += y;
        }
        if (lane == 31) cw[warp] = incl;
        __syncthreads();
        uint32_t run = incl - sum;
        for (int w = 0; w < warp; ++w) run += cw[w];
        for (uint32_t c = c0; c < c1; ++c) {
          const uint32_t x = ccnt[c];
          ccnt[c] = run;
          run += x;
        }
      }
      __syncthreads();
      const uint64_t gofs = *reinterpret_cast<unsigned long long*>(misc + kMiscPrefix) + misc[kMiscBefore];
      Rec* out = reinterpret_cast<Rec*>(a.out0);
      if (a.out_sel && sort_passes_odd(a.ctrl)) out = reinterpret_cast<Rec*>(a.out1);
      const uint32_t out_buf = (out == reinterpret_cast<Rec*>(a.out0)) ? kBufOut : kBufTmp;
      for (uint32_t c = warp; c < nch; c += kW) {
        const uint32_t up = c / cpb, m = min(tot[crank * Dc + up], Z);
        const uint32_t s = ordl[c * 32 + lane];
        const bool real = s < m;
        const uint32_t keep = __ballot_sync(0xFFFFFFFFu, real);
        const uint64_t pos = gofs + ccnt[c] + __popc(keep & lt_mask);
        if (real && pos < a.n) {
          out[pos] = tile_rec[up * Z + s];
          trace_log<TRACE>(a.trace, kWrite, out_buf, R, pos * R);
        }
      }
      __syncthreads();  // the tile, the table rows and the counts are reused by the next subproblem
    }
    q = qnext;
  }
  if (tid == 0) tma_store_wait_all();
  if constexpr (CL) cluster_sync();  // no CTA leaves while a peer may still address its memory
}

}  // namespace

uint32_t orp_fast_smem_bytes(int R, uint32_t Z, uint32_t k, uint32_t C, bool last) {
  return fast_layout(R, Z, k, C, last).total;
}

template <int R, int MODE, bool CL, bool TRACE>
static cudaError_t fast_launch_mode(const PassArgs& a, uint32_t C, uint32_t max_clusters, cudaStream_t st) {
  const uint32_t smem = fast_layout(R, a.Z, a.k, C, MODE & kModeLast).total;
  auto kern = orp_fast_kernel<R, MODE, CL, TRACE>;
  cudaError_t e = set_smem_optin(kern);
  if (e != cudaSuccess) return e;
  const uint64_t nsub = a.B >> a.k;
  cudaLaunchConfig_t cfg{};
  cfg.blockDim = dim3(kT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  if (CL) {
    if (C > 8) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    cfg.gridDim = dim3(C, 1, 1);
    e = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg);
    if (e != cudaSuccess) return e;
    if (nclusters <= 0) return cudaErrorInvalidConfiguration;
    uint64_t g = (uint64_t)nclusters;
    if (max_clusters && g > max_clusters) g = max_clusters;
    if (g > nsub) g = nsub;
    cfg.gridDim = dim3((unsigned)(g * C), 1, 1);
  } else {
    int per_sm = 0, sms = 0, dev = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kT, smem);
    if (e != cudaSuccess) return e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    uint64_t g = (uint64_t)(per_sm > 0 ? per_sm : 1) * sms;
    if (max_clusters && g > max_clusters) g = max_clusters;
    if (g > nsub) g = nsub;
    cfg.gridDim = dim3((unsigned)g, 1, 1);
  }
  return cudaLaunchKernelEx(&cfg, kern, a, C);
}

template <int R, bool CL, bool TRACE>
static cudaError_t fast_launch_r(const PassArgs& a, int mode, uint32_t C, uint32_t maxc, cudaStream_t st) {
  switch (mode) {
    case 0: return fast_launch_mode<R, 0, CL, TRACE>(a, C, maxc, st);
    case kModeFirst: return fast_launch_mode<R, kModeFirst, CL, TRACE>(a, C, maxc, st);
    case kModeLast: return fast_launch_mode<R, kModeLast, CL, TRACE>(a, C, maxc, st);
    default: return fast_launch_mode<R, kModeFirst | kModeLast, CL, TRACE>(a, C, maxc, st);
  }
}

template <int R, int MODE, bool CL>
static int fast_occupancy(uint32_t Z, uint32_t k, uint32_t C) {
  const uint32_t smem = fast_layout(R, Z, k, C, MODE & kModeLast).total;
  auto kern = orp_fast_kernel<R, MODE, CL, false>;
  if (set_smem_optin(kern) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  if (!CL) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kT, smem) != cudaSuccess) {
      (void)cudaGetLastError();
      return 0;
    }
    return per_sm;
  }
  if (C > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg{};
  cfg.blockDim = dim3(kT, 1, 1);
  cfg.gridDim = dim3(C, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return n;
}

template <int R>
static int fast_occupancy_r(int mode, uint32_t Z, uint32_t k, uint32_t C) {
  const bool cl = C > 1;
  switch (mode) {
    case 0: return cl ? fast_occupancy<R, 0, true>(Z, k, C) : fast_occupancy<R, 0, false>(Z, k, C);
    case kModeFirst: return cl ? fast_occupancy<R, kModeFirst, true>(Z, k, C) : fast_occupancy<R, kModeFirst, false>(Z, k, C);
    case kModeLast: return cl ? fast_occupancy<R, kModeLast, true>(Z, k, C) : fast_occupancy<R, kModeLast, false>(Z, k, C);
    default:
      return cl ? fast_occupancy<R, kModeFirst | kModeLast, true>(Z, k, C)
                : fast_occupancy<R, kModeFirst | kModeLast, false>(Z, k, C);
  }
}

int orp_fast_occupancy(int R, int mode, uint32_t Z, uint32_t k, uint32_t C) {
  return R == 8 ? fast_occupancy_r<8>(mode, Z, k, C) : fast_occupancy_r<16>(mode, Z, k, C);
}

cudaError_t launch_orp_fast(const PassArgs& a, int mode, uint32_t C, uint32_t max_clusters, cudaStream_t st,
                            int R, bool trace) {
  const bool cl = C > 1;
  if (R == 8) {
    if (cl) return trace ? fast_launch_r<8, true, true>(a, mode, C, max_clusters, st)
                         : fast_launch_r<8, true, false>(a, mode, C, max_clusters, st);
    return trace ? fast_launch_r<8, false, true>(a, mode, C, max_clusters, st)
                 : fast_launch_r<8, false, false>(a, mode, C, max_clusters, st);
  }
  if (cl) return trace ? fast_launch_r<16, true, true>(a, mode, C, max_clusters, st)
                       : fast_launch_r<16, true, false>(a, mode, C, max_clusters, st);
  return trace ? fast_launch_r<16, false, true>(a, mode, C, max_clusters, st)
               : fast_launch_r<16, false, false>(a, mode, C, max_clusters, st);
}

}  // namespace bos
