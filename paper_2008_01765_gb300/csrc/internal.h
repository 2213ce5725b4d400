// Internal interfaces between the host orchestration (api.cu) and the kernel files.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "bos.h"
#include "common.cuh"

namespace bos {

constexpr int kModeFirst = 1;
constexpr int kModeLast = 2;

struct PassArgs {
  const void* in;           // FIRST: input records
  const void* in_rec;       // otherwise: slot records of the previous array
  const uint32_t* in_tag;   // otherwise: slot tags of the previous array
  void* out_rec;            // not LAST: slot records of the next array
  uint32_t* out_tag;        // not LAST: slot tags of the next array
  void* out0;               // LAST: output records
  void* out1;               // LAST: alternate output (sort scratch), see out_sel
  uint32_t out_sel;         // LAST: 1 = write out1 when an odd number of radix passes will run
  uint32_t skip_publish;    // debug: subproblem 0 of the LAST pass never publishes
  uint64_t n, B;
  uint32_t Z, L, i, k, attempt, ticket_slot;
  uint64_t seed;
  Ctrl* ctrl;
  unsigned long long* status;  // LAST: look-back words, one per subproblem
  uint32_t buf_in_rec, buf_in_tag, buf_out_rec, buf_out_tag;  // trace buffer ids
  Trace trace;
  const uint16_t* ord;      // LAST (persistent kernel): in-bin permutation table, B*Z slot indexes
  uint64_t bucket0;         // global index of local bucket 0 (a shard's buckets; 0 otherwise): the
                            // first pass's groups and the in-bin permutation keys use global indexes
};

// In-bin permutation table (perm_table.cu): row b < B lists final bucket b's slots in the order
// of the Section 3.2 keys of (b, attempt, seed), ord[b*Z + rank] = slot. With the LAST pass's
// input tags (tag != null; levels i..i+k-1 of L) a row holds the bucket's m real slots, then
// 0xFFFF, m counted first into load[b] by a kernel of its own; without them, all Z slots. Z a
// multiple of 32, <= 4096; k <= 12.
struct PermTableArgs {
  uint64_t bucket0;      // global index of local bucket 0 (the keys use global bucket indexes)
  uint16_t* ord;
  const uint32_t* tag;
  uint32_t* load;        // [B] reals per final bucket (workspace), written and read here
  uint64_t B;
  uint32_t Z, attempt, i, k, L, buf_tag;
  uint64_t seed;
  Trace trace;
};
cudaError_t launch_perm_table(const PermTableArgs& a, cudaStream_t st, bool trace);

uint32_t orp_smem_bytes(int R, uint32_t Z, uint32_t k, bool last);

// One launch of the one-CTA-per-subproblem pass over many arrays (batched ORP).
struct BatchPass {
  const PassArgs* args;   // device: one entry per array in this launch
  const uint64_t* first;  // device: running sum of subproblem counts, narr + 1 entries
  uint32_t narr;
  uint64_t nblocks;       // = first[narr]
  uint32_t* ticket;       // device: zeroed counter (LAST passes)
};
cudaError_t launch_orp_pass_batched(const BatchPass& bp, int mode, uint32_t smem, cudaStream_t st, int R,
                                    bool trace);
cudaError_t launch_orp_pass(const PassArgs& a, int mode, uint64_t grid, cudaStream_t st, int R,
                            bool trace);

// Persistent, cluster-wide ORP pass (orp_fast.cu); Z must be a multiple of 32.
uint32_t orp_fast_smem_bytes(int R, uint32_t Z, uint32_t k, uint32_t C, bool last);
// Co-resident clusters (C > 1) or CTAs per SM (C = 1) of that configuration; 0 = cannot run.
int orp_fast_occupancy(int R, int mode, uint32_t Z, uint32_t k, uint32_t C);
cudaError_t launch_orp_fast(const PassArgs& a, int mode, uint32_t C, uint32_t max_clusters, cudaStream_t st,
                            int R, bool trace);

// Streaming first / middle ORP pass (orp_stream.cu): one CTA per subproblem, input buckets
// through a TMA ring, output chunks write-combined in shared memory; Z a multiple of 32, <= 2048.
uint32_t orp_stream_smem_bytes(int R, uint32_t Z, uint32_t k, bool first);
// Most levels a streaming pass holds in smem_limit bytes (0: the kernel cannot take this Z).
uint32_t orp_stream_max_k(int R, uint32_t Z, bool first, uint32_t smem_limit);
inline uint32_t orp_stream_min_k() { return 5; }
cudaError_t launch_orp_stream(const PassArgs& a, bool first, cudaStream_t st, int R, bool trace);

// The ORP with O(1) client storage (oblivious.cu, Section 4.1): bitonic-sort MergeSplits, one
// launch per level, bitonic in-bin permutations, a scan of the loads and the strip.
struct ObliviousArgs {
  const void* in;        // n input records
  void* out0;            // n output records
  void* out1;            // alternate output (sort scratch); used when out_sel and an odd number of
  uint32_t out_sel;      // radix passes will run (as the fused LAST pass chooses)
  void* rec[2];          // slot record arrays (B*Z each), used in turn
  uint32_t* tag[2];      // slot tag arrays
  uint32_t* load;        // [B] reals per final bucket
  uint32_t* off;         // [B] output offsets inside scan blocks
  uint32_t* part;        // [B / 4096 + 1] scan block offsets
  uint64_t n, B;
  uint32_t Z, L, attempt;
  uint64_t seed;
  Ctrl* ctrl;
  Trace trace;
};
uint32_t oblivious_smem_bytes(int R, uint32_t Z);
cudaError_t launch_oblivious_orp(const ObliviousArgs& a, int R, cudaStream_t st, bool trace);

// Stable merge sort by key (mergesort.cu): runs of 2048 sorted in shared memory, then merge
// passes that double the run width. The result lands in buf0; the block-sorted runs are written
// to buf0 when merge_passes(n) is even and to buf1 when it is odd, so `in` may be that buffer.
// split: merge_split_entries(n) u64 of scratch. hooks (optional) bracket the block sort (stage 0)
// and each merge pass (stage 1) with the algorithmic bytes.
struct MergeHooks {
  int (*begin)(cudaStream_t st, int stage, double bytes);
  void (*end)(int slot, cudaStream_t st);
};
uint32_t merge_passes(uint64_t n);
uint64_t merge_split_entries(uint64_t n);
cudaError_t launch_merge_sort(const void* in, void* buf0, void* buf1, uint64_t n, int R, uint64_t* split,
                              cudaStream_t st, const MergeHooks& hooks);

// LSD radix sort (radix.cu)
struct RadixArgs {
  const void* in;                 // histogram source (any order of the same multiset)
  void* buf0;                     // final output
  void* buf1;                     // scratch of n records
  uint64_t n;
  uint32_t* hist;                 // [digits][256]
  unsigned long long* dbase;      // [digits][256] exclusive digit offsets
  unsigned long long* status;     // [tiles][256] look-back words
  Ctrl* ctrl;
  uint32_t ticket_base;
};
uint64_t radix_tiles(uint64_t n, int R);

// Hybrid radix sort (sort_hybrid.cu): MSD partitions on the top one or two digits, then an on-chip
// sort of every range of groups; falls back to the LSD passes (ctrl->sort_mode = 0) when a group
// exceeds hybrid_cap(R) records. stage: 0 histogram (hist and joint), 1 plan, 2 partition by the
// top varying digit, 3 partition by the next one inside every bucket, 4 the on-chip sort.
struct HybridArgs {
  const void* in;                   // histogram source (the ORP's input: the same multiset of keys)
  void* buf0;                       // final output
  void* buf1;                       // scratch of n records
  uint64_t n;
  uint32_t* hist;                   // [digits][256] digit counts (shared with the LSD path)
  const unsigned long long* dbase;  // [digits][256] exclusive digit offsets (radix prep)
  uint32_t* joint;                  // [65536] counts of the top two digits
  unsigned long long* gstart;       // [65537] group starts
  uint32_t* rlist;                  // [65537] first group of every range
  unsigned long long* first;        // [257] partition tiles before every top-digit bucket
  uint32_t* meta;                   // [8] mode, top varying digit, next varying digit, ranges,
                                    // large ranges, small ranges
  uint32_t* ridx;                   // [2][65537] the large ranges, then (at 65537) the small ones
  unsigned long long* status;       // look-back words for radix_tiles(n) + 256 tiles
  unsigned char* scratch;           // hybrid_spill_bytes(n, R): one spill buffer per on-chip-sort CTA
  uint32_t local_ctas;              // = hybrid_local_ctas(n, R)
  Ctrl* ctrl;
};
uint32_t hybrid_cap(int R);
uint32_t hybrid_local_ctas(uint64_t n, int R);
size_t hybrid_spill_bytes(uint64_t n, int R);
cudaError_t launch_hybrid(const HybridArgs& a, int R, int stage, cudaStream_t st);
// Radix stages over many arrays in one launch (batched sort).
struct BatchRadix {
  const RadixArgs* args;  // device: one entry per array
  const uint64_t* first;  // device: running sum of tiles (kTile records each), narr + 1 entries
  uint32_t narr;
  uint64_t nblocks;       // = first[narr]
  uint32_t* ticket;       // device: one zeroed counter per digit
};
// stage 0 = histograms, 1 = digit offsets, 2 = the pass of `digit`
cudaError_t launch_radix_batched(const BatchRadix& br, int R, int stage, uint32_t digit, cudaStream_t st);
cudaError_t launch_radix_hist(const RadixArgs& a, int R, cudaStream_t st);
cudaError_t launch_radix_prep(const RadixArgs& a, int R, cudaStream_t st);
cudaError_t launch_radix_pass(const RadixArgs& a, int R, uint32_t digit, cudaStream_t st);

// Bucket ORP with a caller-chosen workspace (api.cu); workspace bytes of the ORP alone.
size_t orp_workspace_bytes(uint64_t n, const bos_params* p);
bos_status orp_with_workspace(const void* d_in, void* d_out, uint64_t n, const bos_params* p,
                              void* d_ws, size_t ws_bytes, void* stream, bos_info* info);

// Bitonic comparator (bitonic.cu)
cudaError_t launch_bitonic(const void* in, void* out, uint64_t n, int R, cudaStream_t st);

}  // namespace bos
