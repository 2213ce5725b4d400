/*
 * bos.h - C ABI of the GB300 bucket oblivious random permutation (ORP) and bucket oblivious
 * sort library (libbos.so).
 *
 * The method is the one of Asharov, Chan, Nayak, Pass, Ren, Shi, "Bucket Oblivious Sort: An
 * Extremely Simple Oblivious Sort" (SOSA 2020):
 *   - Algorithm 3.1 (oblivious random bin assignment): every record gets a uniformly random
 *     label in [0, B), the input is split evenly into B buckets of Z slots padded with dummies,
 *     and log2 B butterfly levels of MergeSplit route each record to the bucket of its label.
 *   - Section 3.2 (bucket ORP): the dummies are stripped, each final bucket is permuted at
 *     random and the buckets are concatenated.
 *   - Section 3.3 (bucket oblivious sort): the ORP output is sorted by a non-oblivious sort
 *     (here a stable LSD radix sort on the key).
 *
 * Records are opaque blocks of rec_bytes bytes (8 or 16). The key is the unsigned little-endian
 * integer of key_bytes bytes (4 for 8-byte records, 8 for 16-byte records) at offset 0; the
 * rest of the record is payload and is never compared.
 *
 * Conventions for every entry point:
 *   - Every pointer named d_* is a device pointer owned by the caller. No call allocates or
 *     frees device memory, prints or aborts; errors are reported by status (host-side scratch of
 *     the batched calls is ordinary heap memory). The library image itself holds one fixed
 *     device array, the BOS_NOALLOC_SCRATCH_BYTES scratch of bos_orp_noalloc, on every GPU
 *     where its kernels are loaded.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream). Work is stream-ordered.
 *     bos_orp / bos_sort / bos_sort_batched synchronise `stream` once per attempt to read the
 *     overflow flag (Algorithm 3.1, MergeSplit aborts on overflow; the call retries with a
 *     fresh attempt counter, up to max_attempts).
 *   - Results are a deterministic function of (input, n, Z, seed, rec_bytes, key_bytes) only:
 *     they do not depend on k, on the block shape, on batching or on concurrency.
 *   - d_out must not overlap d_in or the workspace (BOS_ERR_INVALID otherwise). n = 0 is a
 *     no-op that returns BOS_OK.
 */
#ifndef BOS_H_
#define BOS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BOS_OK = 0,
  BOS_ERR_INVALID = 1,   /* bad argument (size, alignment, widths, aliasing, null pointer) */
  BOS_ERR_OVERFLOW = 2,  /* every one of max_attempts attempts overflowed a bucket */
  BOS_ERR_WORKSPACE = 3, /* ws_bytes smaller than bos_workspace_bytes() */
  BOS_ERR_CUDA = 4,      /* a CUDA runtime call or kernel launch failed */
  BOS_ERR_TIMEOUT = 5    /* a bounded device-side wait gave up (the results are not valid) */
} bos_status;

/* flags */
#define BOS_FLAG_NONE 0u
/* Debug: report overflow for the first (flags >> 8) & 0xFF attempts, so the retry path runs
 * without a tiny Z. The results are still those of the first attempt not forced to fail. */
#define BOS_FLAG_FORCE_OVERFLOW(n) (((uint32_t)(n) & 0xFFu) << 8)
/* Debug: one look-back producer skips its publish, so the bounded wait must time out and the
 * call must return BOS_ERR_TIMEOUT (tests the failure path without hanging a GPU). */
#define BOS_FLAG_SKIP_PUBLISH 0x1u
/* Use the one-CTA-per-subproblem pass kernel even when Z is a multiple of 32 (comparison and
 * tests; the result is the same). */
#define BOS_FLAG_GENERIC 0x2u
/* Do not use thread-block clusters (C = 1): fewer levels per pass, same result. */
#define BOS_FLAG_NO_CLUSTER 0x4u
/* Fill *info with the plan for these arguments (B, L, passes, k, cluster size) and return
 * without touching the device (pointers may be NULL). */
#define BOS_FLAG_PLAN_ONLY 0x10u
/* Plan the fewest passes (largest clusters) instead of the measured-cost plan; same result. */
#define BOS_FLAG_FEWEST_PASSES 0x8u
/* bos_sort: sort the ORP's output with a stable GPU merge sort (comparison-based, as Section 3.3
 * composes the ORP with a comparison sort) instead of the LSD radix sort. Same result. */
#define BOS_FLAG_MERGE_SORT 0x20u
/* bos_orp, bos_sort: the ORP in the O(1)-client-storage form of Section 4.1. Every MergeSplit is one
 * bitonic sort of its two buckets (one launch per level), and every final bucket is permuted by one
 * bitonic sort, so the access schedule depends on neither the data nor the labels. Same result;
 * much slower. */
#define BOS_FLAG_OBLIVIOUS_SPLIT 0x40u
/* Do not use the streaming pass kernel for the first and middle passes of the automatic plan
 * (comparison and tests; the result is the same). */
#define BOS_FLAG_NO_STREAM 0x80u
/* Largest thread-block cluster a pass may use (1, 2, 4, 8 or 16; 0 = the library's choice).
 * Tuning only: the result never depends on it. */
#define BOS_FLAG_MAX_CLUSTER(c) (((uint32_t)(c) & 0x1Fu) << 16)
/* bos_sort: the LSD radix sort (one pass per live 8-bit digit) instead of the hybrid radix sort
 * (partitions on the top one or two digits, then an on-chip sort of every group of records that
 * share them). Same result. The hybrid sort falls back to the LSD passes by itself whenever a
 * group would exceed one CTA's on-chip capacity. */
#define BOS_FLAG_LSD_SORT 0x200000u

typedef struct {
  uint32_t rec_bytes;    /* 8 or 16 */
  uint32_t key_bytes;    /* 4 (rec 8) or 8 (rec 16) */
  uint32_t Z;            /* bucket size, 2 <= Z <= 4096 for 8-byte and <= 2048 for 16-byte records
                            (one bucket pair must fit in shared memory); Section 3.4 suggests 512 */
  uint32_t k;            /* butterfly levels fused per HBM pass; 0 = automatic, 1 = plain form
                            (one launch per level). Never changes the result. */
  uint32_t max_attempts; /* overflow retries; 0 = default (8) */
  uint32_t flags;        /* BOS_FLAG_* */
  uint64_t seed;         /* Philox key of the labels and of the in-bin permutation */
} bos_params;

typedef struct {
  uint32_t attempts; /* attempts run (1 unless an overflow forced a retry) */
  uint32_t L;        /* log2 B, the number of butterfly levels */
  uint32_t passes;   /* HBM passes of the ORP in the last attempt */
  uint32_t radix_passes; /* HBM passes of the sort after the ORP, histogram excluded: one per live
                            8-bit digit for the LSD sort (digits where all keys agree are skipped),
                            1 to 3 for the hybrid sort */
  uint64_t B;        /* number of buckets: smallest power of two with B * Z >= 2n */
  uint32_t max_cluster; /* largest thread-block cluster used by a pass (1 = no clusters) */
  uint32_t max_k;    /* most butterfly levels fused into one pass */
  uint32_t stream_passes; /* passes run by the streaming kernel (first and middle passes) */
  uint32_t sort_mode; /* bos_sort's radix sort: 0 LSD; 1 on-chip only; 2 one partition + on-chip;
                         3 two partitions + on-chip */
} bos_info;

/* Bytes of device workspace bos_orp / bos_sort need for n records under *p (0 for n = 0):
 * the two bucket arrays of Algorithm 3.1 (B * Z slots each, the paper's log B + 1 arrays used in
 * turn), the in-bin permutation table of Section 3.2 and, for bos_sort, the radix sort's scratch
 * (Section 3.3). Returns 0 and sets nothing on invalid parameters. */
size_t bos_workspace_bytes(uint64_t n, const bos_params* p);

/* Bucket ORP (Algorithm 3.1 + Section 3.2): d_out[0..n) = d_in permuted uniformly at random
 * (determined by p->seed). d_in: n * rec_bytes bytes, read only, aligned to rec_bytes. d_out: n *
 * rec_bytes bytes, aligned to rec_bytes. d_ws: ws_bytes >= bos_workspace_bytes(n, p), 256-byte
 * aligned; its contents on entry do not matter. info may be NULL. */
bos_status bos_orp(const void* d_in, void* d_out, uint64_t n, const bos_params* p, void* d_ws,
                   size_t ws_bytes, void* stream, bos_info* info);

/* Bucket ORP for callers that cannot allocate device memory (the paper has no counterpart; this
 * is a deployment aid). Some callers cannot provide the workspace bos_orp needs: code running
 * inside a custom device allocator or its callbacks (allocating there would re-enter the
 * allocator), and plugins whose host owns all device memory and forbids them to allocate.
 * bos_orp_noalloc gives the same result as bos_orp for the same arguments but takes its workspace
 * from a scratch array compiled into the library:
 *   - size: BOS_NOALLOC_SCRATCH_BYTES (64 MiB) of device memory, held on every GPU where the
 *     library's kernels are loaded until the process exits. n is accepted while the ORP's
 *     workspace for n fits; otherwise the call returns BOS_ERR_WORKSPACE and touches nothing.
 *     (bos_workspace_bytes(n, p) <= BOS_NOALLOC_SCRATCH_BYTES is a sufficient check; with
 *     Z = 512 every n <= 2^19 fits for 16-byte records and every n <= 2^20 for 8-byte records.)
 *   - no allocation: the call makes no cudaMalloc / cudaFree or other allocating call. Every call
 *     looks up the scratch's device address on the current device (cudaGetSymbolAddress); on the
 *     first call on a device that lookup also loads the library's kernels there.
 *   - synchronisation: like bos_orp, the call synchronises `stream` after every attempt to read
 *     the overflow flag (Algorithm 3.1's MergeSplit abort), so it blocks the host until the ORP
 *     has finished and must not be issued on a stream that is being captured.
 *   - sharing: every call on a device uses the same scratch, which keeps the previous call's
 *     contents (the call clears what must start at zero itself). Calls whose GPU work overlaps
 *     (different streams, or host threads) race on the scratch and give wrong results: order
 *     them on one stream or serialise them.
 * Arguments as for bos_orp. */
#define BOS_NOALLOC_SCRATCH_BYTES (64u << 20)
bos_status bos_orp_noalloc(const void* d_in, void* d_out, uint64_t n, const bos_params* p,
                           void* stream, bos_info* info);

/* Bucket oblivious sort (Section 3.3): the ORP of d_in followed by a stable ascending LSD radix
 * sort on the key, so equal keys keep their ORP order. Same arguments as bos_orp. */
bos_status bos_sort(const void* d_in, void* d_out, uint64_t n, const bos_params* p, void* d_ws,
                    size_t ws_bytes, void* stream, bos_info* info);

/* Batched ORP / sort of `num` independent arrays stored back to back (no counterpart in the
 * paper; the many-arrays form of the same method). Array j occupies records [h_offsets[j],
 * h_offsets[j+1]) of d_in and of d_out, is processed with seed h_seeds[j], Z = h_Z[j] (or
 * base->Z when h_Z is NULL) and op h_ops[j] (0 = ORP, 1 = sort). Its result equals bos_orp /
 * bos_sort of that array alone with the same seed and Z. h_attempts (nullable, num entries)
 * receives the attempts of each array (0 for an empty array). Host arrays are read during the
 * call only. All arrays go through one fixed sequence of launches (a memset, the radix
 * histograms and offsets, one launch per butterfly pass index and mode, one per radix digit);
 * arrays that overflowed run again as a smaller batch with the next attempt counter.
 *
 * bos_sort_batched = bos_batched_prepare + bos_batched_enqueue + bos_batched_collect:
 *   - prepare writes the launch descriptors into d_ws (a synchronous copy);
 *   - enqueue only issues that launch sequence on `stream` (no copy, no synchronisation), so it
 *     can be captured into a CUDA graph and replayed for the same batch;
 *   - collect synchronises `stream`, reads every array's overflow flag, reruns the arrays that
 *     overflowed and writes the full batch's descriptors back (so a captured graph stays valid).
 * The three calls take the same arguments (d_ws must be the same buffer). */
size_t bos_batched_workspace_bytes(const uint64_t* h_offsets, uint32_t num, const uint32_t* h_Z,
                                   const uint8_t* h_ops, const bos_params* base);
bos_status bos_sort_batched(const void* d_in, void* d_out, const uint64_t* h_offsets,
                            uint32_t num, const uint64_t* h_seeds, const uint32_t* h_Z,
                            const uint8_t* h_ops, const bos_params* base, void* d_ws,
                            size_t ws_bytes, void* stream, uint32_t* h_attempts);
bos_status bos_batched_prepare(const void* d_in, void* d_out, const uint64_t* h_offsets,
                               uint32_t num, const uint64_t* h_seeds, const uint32_t* h_Z,
                               const uint8_t* h_ops, const bos_params* base, void* d_ws,
                               size_t ws_bytes, void* stream);
bos_status bos_batched_enqueue(const void* d_in, void* d_out, const uint64_t* h_offsets,
                               uint32_t num, const uint64_t* h_seeds, const uint32_t* h_Z,
                               const uint8_t* h_ops, const bos_params* base, void* d_ws,
                               size_t ws_bytes, void* stream);
bos_status bos_batched_collect(const void* d_in, void* d_out, const uint64_t* h_offsets,
                               uint32_t num, const uint64_t* h_seeds, const uint32_t* h_Z,
                               const uint8_t* h_ops, const bos_params* base, void* d_ws,
                               size_t ws_bytes, void* stream, uint32_t* h_attempts);

/* Shard plan: the bucket ORP of one array over G = 2^g ranks (GPUs) with one fixed exchange
 * (the multi-GPU form of Algorithm 3.1's butterfly; the paper has no multi-GPU section). Rank r
 * holds buckets [r Bl, (r+1) Bl), Bl = B / G, and the input records of their groups,
 * [bos_shard_input_range). Steps of one attempt (every rank uses the same attempt counter):
 *   1. bos_shard_local: levels 0 .. L-g-1, which pair buckets inside aligned blocks of at most Bl
 *      buckets, on the rank's own buckets; its buckets end in the send region of its workspace.
 *   2. the exchange (the caller's: one all-to-all of whole buckets, NCCL or peer copies): rank s
 *      sends rank d the chunk d of its send region (chunk_rec_bytes of records at
 *      send_rec_offset + d * chunk_rec_bytes, chunk_tag_bytes of tags at send_tag_offset +
 *      d * chunk_tag_bytes) into chunk s of rank d's receive region (recv_*_offset + s * chunk).
 *      Its volume and addresses do not depend on the data, so the plan stays oblivious.
 *   3. bos_shard_final: the last g levels on the received buckets in one fused pass, the in-bin
 *      permutation of Section 3.2 (keys of the global bucket indexes) and the strip; the rank's
 *      reals (its final buckets [r Bl, (r+1) Bl) in order) go to d_out, *h_count of them, and
 *      *h_overflow tells whether any MergeSplit of the attempt on this rank overflowed.
 * If any rank overflowed (a max-reduction), every rank repeats with attempt + 1; otherwise rank
 * r's part belongs at the sum of the counts of ranks < r. The parts, put together, equal bos_orp of
 * the whole array with the same seed, and the attempts agree. Requirements: G a power of two with
 * G^2 <= B and L - g >= 2; flags other than the Section 4.1 form and the merge sort as for
 * bos_orp (BOS_ERR_INVALID otherwise). Workspace per rank: ws_bytes, 256-byte aligned; d_out
 * holds out_capacity records. Both steps are stream-ordered; bos_shard_final synchronises
 * `stream` to read the flag and the count. */
typedef struct {
  uint64_t B, B_local;   /* buckets in all, buckets per rank */
  uint32_t L, g;         /* log2 B, log2 G */
  uint32_t local_passes; /* HBM passes of step 1 */
  size_t ws_bytes;       /* workspace bytes per rank */
  size_t send_rec_offset, send_tag_offset, recv_rec_offset, recv_tag_offset;  /* in the workspace */
  size_t chunk_rec_bytes, chunk_tag_bytes;  /* one rank-to-rank chunk of the exchange */
  uint64_t out_capacity; /* records d_out must hold for bos_shard_final */
} bos_shard_layout_t;
bos_status bos_shard_layout(uint64_t n, uint32_t G, const bos_params* p, bos_shard_layout_t* out);
/* Input records [*lo, *hi) of rank r: the groups of its buckets (Algorithm 3.1's placement). */
bos_status bos_shard_input_range(uint64_t n, uint32_t G, uint32_t r, const bos_params* p, uint64_t* lo,
                                 uint64_t* hi);
/* d_in: rank r's input records (its range only, aligned to rec_bytes). */
bos_status bos_shard_local(const void* d_in, uint64_t n, uint32_t G, uint32_t r, const bos_params* p,
                           uint32_t attempt, void* d_ws, size_t ws_bytes, void* stream);
bos_status bos_shard_final(uint64_t n, uint32_t G, uint32_t r, const bos_params* p, uint32_t attempt,
                           void* d_out, uint64_t out_cap, void* d_ws, size_t ws_bytes, void* stream,
                           uint64_t* h_count, uint32_t* h_overflow);

/* Out-of-core bucket ORP: n records in host memory, more than the device can hold (Section 4.3's
 * setting, where the data live in a slower, larger memory and are accessed in large contiguous
 * runs). The shard plan above runs its G ranks one after another on the current GPU, each rank's
 * data staying in host memory between its steps: rank r's input range goes in, its local levels
 * run, its send regions go to h_stage; then, for every rank d, its chunks are gathered from
 * h_stage, its last levels, in-bin permutation and strip run, and its part goes to h_out at the
 * sum of the earlier parts. Every host access is a contiguous run of whole buckets (their volume
 * and addresses do not depend on the data). Same result as bos_orp for the same arguments.
 * h_in, h_out: n records of host memory (pinned for full copy bandwidth); d_buf: dev_bytes of
 * device memory (256-byte aligned); h_stage: host_bytes of host memory; both from
 * bos_orp_out_of_core_bytes. G as for the shard plan. Synchronises `stream`. */
bos_status bos_orp_out_of_core_bytes(uint64_t n, uint32_t G, const bos_params* p, size_t* dev_bytes,
                                     size_t* host_bytes);
bos_status bos_orp_out_of_core(const void* h_in, void* h_out, uint64_t n, const bos_params* p, uint32_t G,
                               void* d_buf, size_t dev_bytes, void* h_stage, size_t host_bytes, void* stream,
                               bos_info* info);

/* GPU bitonic sorting network (Table 1's comparator; not oblivious-sort output compatible:
 * equal keys are ordered by payload). n must be a power of two (BOS_ERR_INVALID otherwise).
 * Sorts d_in into d_out by (key, payload) ascending. Needs no workspace. */
bos_status bos_bitonic_sort(const void* d_in, void* d_out, uint64_t n, uint32_t rec_bytes,
                            uint32_t key_bytes, void* stream);

/* Debug address trace (obliviousness check, Section 3.1 and Lemma 3.3). While attached, every
 * global-memory access of the ORP kernels is appended to d_buf as two uint64 words
 * {(kind << 56) | (buffer << 48) | bytes, byte offset within that buffer}; word 0 of d_buf
 * counts the entries written (entries beyond the buffer's capacity are counted, not stored).
 * kind: 1 = read, 2 = write. buffer: 0 = input, 1 = slot records A, 2 = slot tags A,
 * 3 = slot records B, 4 = slot tags B, 5 = output, 6 = sort scratch in the workspace,
 * 7 = in-bin permutation table in the workspace. Attach NULL to detach. The trace run uses
 * separate kernel instances; the results are identical. The buffer is process-wide: every call
 * that starts while it is attached, from any host thread, appends to it (each call reads the
 * attachment once when it starts); attach and detach between calls to trace one call alone. */
bos_status bos_trace_attach(void* d_buf, size_t bytes);

/* Debug address-trace digest (obliviousness check at sizes whose full trace would not fit,
 * Section 3.1 and Lemma 3.3). While attached, every access the trace above would record is folded
 * into d_buf instead: d_buf holds 256 slots of two uint64 words, and slot (SM id mod 256) counts
 * its entries in word 0 and adds SplitMix64's mix of the entry (mix(word0 ^ mix(offset))) to word 1
 * modulo 2^64. The sums over all slots of both words depend only on the multiset of entries. The
 * caller zeroes the buffer first; bytes >= 4096. Attach NULL (to either attach call) to detach.
 * Same sharing rule as bos_trace_attach. The batched calls carry the buffer attached when their
 * descriptors were written (bos_batched_prepare) and log while one is attached at enqueue. */
bos_status bos_trace_attach_digest(void* d_buf, size_t bytes);

/* Self-test hook for the random source (Philox4x32-10, Salmon et al. SC 2011) that draws the
 * labels of Algorithm 3.1 and the in-bin permutation keys of Section 3.2. For i < n it writes
 * the library's Philox of counter d_ctr[4i..4i+3] and key d_key[2i..2i+1] to d_out[4i..4i+3],
 * and, when d_out_curand is not NULL, cuRAND's curand_Philox4x32_10 of the same inputs to
 * d_out_curand. All buffers are device memory owned by the caller. */
bos_status bos_selftest_philox(const uint32_t* d_ctr, const uint32_t* d_key, uint32_t* d_out,
                               uint32_t* d_out_curand, uint64_t n, void* stream);

/* Kernel timing for benchmarks (no counterpart in the paper). While enabled, every launch of
 * bos_orp / bos_sort / bos_bitonic_sort is bracketed by CUDA events recorded on the call's
 * stream; each kernel class accumulates its launches, device milliseconds and algorithmic bytes
 * (whole slot arrays read and written by a butterfly pass; records read and written by a radix
 * pass; keys read by the histogram). bos_profile_enable creates its events on the first call
 * (CUDA events, no device memory) and resets the totals. The totals are process-wide: calls from
 * several host threads may run while profiling is on (the counters are guarded, and a pair of
 * events whose launch has not finished when another thread collects stays pending); switching
 * profiling on or off, or reading the totals, while other threads run calls mixes their launches
 * into the figures. */
typedef struct {
  char name[32];     /* orp_pass_first, orp_pass_mid, orp_pass_last, orp_pass_single, radix_hist,
                        radix_prep, radix_pass, radix_pass_skipped, bitonic */
  uint32_t launches;
  double ms;         /* summed device time */
  double bytes;      /* summed algorithmic bytes */
} bos_kernel_stat;
bos_status bos_profile_enable(int on);
/* Fills up to max entries (classes with at least one launch); *total_launches (nullable) gets the
 * number of kernel launches counted since the last enable. Returns the entries written. */
uint32_t bos_profile_read(bos_kernel_stat* out, uint32_t max, uint64_t* total_launches);

/* Text of a status code (no counterpart in the paper). */
const char* bos_status_str(bos_status s);

/* Library version, (major << 16) | minor. */
uint32_t bos_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BOS_H_ */
