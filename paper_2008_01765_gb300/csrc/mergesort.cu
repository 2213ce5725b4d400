// Stable merge sort by key, sm_103a: the comparison-based sort that Section 3.3 composes with the
// ORP (any non-oblivious comparison sort after the permutation gives an oblivious sort; its
// accesses depend only on the relative order of the keys, which the ORP has made random).
//
// Block sort: a CTA sorts a tile of kBT records: eight per thread sorted in registers by
// adjacent exchanges, then rounds of pairwise merges of sorted runs in shared memory.
// Merge passes: runs of width w become runs of 2w. A partition kernel finds, for every output
// chunk of kMC records, how many of its predecessors in the pair come from the left run (merge
// path: a binary search on the chunk's diagonal); a CTA then loads its two input ranges, merges
// them in shared memory and writes the chunk. Equal keys always take the left run first, so the
// sort is stable: equal keys keep the order they had after the ORP.
#include "common.cuh"
#include "internal.h"

namespace bos {

namespace {

constexpr int kMT = 256;               // threads per CTA
constexpr int kMI = 8;                 // records per thread
constexpr uint32_t kBT = kMT * kMI;    // block-sorted run (2048 records)
constexpr uint32_t kMC = kMT * kMI;    // merge chunk (2048 records); runs are at least kMC long

// Merge path: of the first d outputs of the stable merge of A[0..na) and B[0..nb) (A first on
// equal keys), how many come from A.
template <int R, typename PA, typename PB>
__device__ __forceinline__ uint32_t merge_split(PA A, uint32_t na, PB B, uint32_t nb, uint32_t d) {
  uint32_t lo = d > nb ? d - nb : 0u, hi = d < na ? d : na;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (!(RecT<R>::key(B[d - 1 - mid]) < RecT<R>::key(A[mid])))  // A[mid] goes before B[d-1-mid]
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// The next `cnt` outputs of the stable merge from positions (i, j), into v.
template <int R>
__device__ __forceinline__ void merge_run(const typename RecT<R>::T* A, uint32_t na, const typename RecT<R>::T* B,
                                          uint32_t nb, uint32_t i, uint32_t j, uint32_t cnt,
                                          typename RecT<R>::T (&v)[kMI]) {
#pragma unroll
  for (int x = 0; x < kMI; ++x) {
    if ((uint32_t)x < cnt) {
      const bool takeA = j >= nb || (i < na && !(RecT<R>::key(B[j]) < RecT<R>::key(A[i])));
      v[x] = takeA ? A[i] : B[j];
      i += takeA;
      j += !takeA;
    }
  }
}

template <int R>
__global__ void __launch_bounds__(kMT) merge_block_kernel(const typename RecT<R>::T* in, typename RecT<R>::T* out,
                                                          uint64_t n) {
  using Rec = typename RecT<R>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  Rec* buf = reinterpret_cast<Rec*>(smem);  // [kBT]
  const int tid = threadIdx.x;
  const uint64_t t0 = (uint64_t)blockIdx.x * kBT;
  const uint32_t cnt = (uint32_t)(n - t0 < kBT ? n - t0 : kBT);
  for (uint32_t x = tid; x < cnt; x += kMT) buf[x] = in[t0 + x];
  __syncthreads();
  const uint32_t o = tid * kMI;
  const uint32_t m = o < cnt ? (cnt - o < (uint32_t)kMI ? cnt - o : (uint32_t)kMI) : 0u;
  Rec v[kMI];
#pragma unroll
  for (int x = 0; x < kMI; ++x)
    if ((uint32_t)x < m) v[x] = buf[o + x];
  // odd-even transposition: exchanging only strictly out-of-order neighbours keeps it stable
#pragma unroll
  for (int r = 0; r < kMI; ++r) {
#pragma unroll
    for (int x = r & 1; x + 1 < kMI; x += 2) {
      if ((uint32_t)(x + 1) < m && RecT<R>::key(v[x + 1]) < RecT<R>::key(v[x])) {
        const Rec t = v[x];
        v[x] = v[x + 1];
        v[x + 1] = t;
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int x = 0; x < kMI; ++x)
    if ((uint32_t)x < m) buf[o + x] = v[x];
  __syncthreads();
  for (uint32_t w = kMI; w < kBT; w <<= 1) {  // runs of w -> runs of 2w
    if (m) {
      const uint32_t pb = o / (2 * w) * (2 * w), b0 = pb + w;
      const uint32_t na = cnt - pb < w ? cnt - pb : w;
      const uint32_t nb = b0 < cnt ? (cnt - b0 < w ? cnt - b0 : w) : 0u;
      const uint32_t d = o - pb;
      const uint32_t i = merge_split<R>(buf + pb, na, buf + b0, nb, d);
      merge_run<R>(buf + pb, na, buf + b0, nb, i, d - i, m, v);
    }
    __syncthreads();  // every read of this round is done
#pragma unroll
    for (int x = 0; x < kMI; ++x)
      if ((uint32_t)x < m) buf[o + x] = v[x];
    __syncthreads();
  }
  for (uint32_t x = tid; x < cnt; x += kMT) out[t0 + x] = buf[x];
}

// For every chunk c (output positions [c*kMC, ...)), the global index of its first left-run
// element: split[c] = a0 + (left-run records among the pair's first d outputs). c = nchunks gives n.
template <int R>
__global__ void merge_partition_kernel(const typename RecT<R>::T* in, uint64_t n, uint64_t w, uint64_t* split,
                                       uint64_t nchunks) {
  const uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c > nchunks) return;
  const uint64_t o = c * kMC < n ? c * kMC : n;
  const uint64_t pb = o / (2 * w) * (2 * w), b0 = pb + w;
  const uint32_t na = (uint32_t)(n - pb < w ? n - pb : w);
  const uint32_t nb = (uint32_t)(b0 < n ? (n - b0 < w ? n - b0 : w) : 0u);
  split[c] = pb + merge_split<R>(in + pb, na, in + b0, nb, (uint32_t)(o - pb));
}

// One chunk of one merge pass (runs of w >= kMC, so a chunk lies inside one pair of runs).
template <int R>
__global__ void __launch_bounds__(kMT) merge_pass_kernel(const typename RecT<R>::T* in, typename RecT<R>::T* out,
                                                         uint64_t n, uint64_t w, const uint64_t* split) {
  using Rec = typename RecT<R>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  Rec* src = reinterpret_cast<Rec*>(smem);  // [kMC] the chunk's two input ranges
  Rec* dst = src + kMC;                     // [kMC] the merged chunk
  const int tid = threadIdx.x;
  const uint64_t c = blockIdx.x, o0 = c * kMC, o1 = o0 + kMC < n ? o0 + kMC : n;
  const uint64_t pb = o0 / (2 * w) * (2 * w), pe = pb + 2 * w < n ? pb + 2 * w : n, b0 = pb + w;
  const uint64_t na = n - pb < w ? n - pb : w;
  const uint64_t a_lo = split[c], a_hi = o1 == pe ? pb + na : split[c + 1];
  const uint64_t b_lo = b0 + ((o0 - pb) - (a_lo - pb)), b_hi = b0 + ((o1 - pb) - (a_hi - pb));
  const uint32_t la = (uint32_t)(a_hi - a_lo), lb = (uint32_t)(b_hi - b_lo);  // la + lb = o1 - o0
  for (uint32_t x = tid; x < la; x += kMT) src[x] = in[a_lo + x];
  for (uint32_t x = tid; x < lb; x += kMT) src[la + x] = in[b_lo + x];
  __syncthreads();
  const uint32_t cnt = (uint32_t)(o1 - o0), o = tid * kMI;
  if (o < cnt) {
    const uint32_t m = cnt - o < (uint32_t)kMI ? cnt - o : (uint32_t)kMI;
    const uint32_t i = merge_split<R>(src, la, src + la, lb, o);
    Rec v[kMI];
    merge_run<R>(src, la, src + la, lb, i, o - i, m, v);
#pragma unroll
    for (int x = 0; x < kMI; ++x)
      if ((uint32_t)x < m) dst[o + x] = v[x];
  }
  __syncthreads();
  for (uint32_t x = tid; x < cnt; x += kMT) out[o0 + x] = dst[x];
}

template <int R>
cudaError_t merge_sort_r(const void* in, void* buf0, void* buf1, uint64_t n, uint64_t* split, cudaStream_t st,
                         const MergeHooks& hooks) {
  using Rec = typename RecT<R>::T;
  const uint32_t passes = merge_passes(n);
  // the block-sorted runs go where an even number of merge passes leaves the result in buf0
  Rec* cur = reinterpret_cast<Rec*>((passes & 1) ? buf1 : buf0);
  Rec* oth = reinterpret_cast<Rec*>((passes & 1) ? buf0 : buf1);
  cudaError_t e = cudaSuccess;
  {
    const uint64_t grid = (n + kBT - 1) / kBT;
    const int ev = hooks.begin ? hooks.begin(st, 0, 2.0 * n * R) : -1;
    merge_block_kernel<R><<<(unsigned)grid, kMT, kBT * sizeof(Rec), st>>>(reinterpret_cast<const Rec*>(in), cur, n);
    if (hooks.end) hooks.end(ev, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if ((e = set_smem_optin(merge_pass_kernel<R>)) != cudaSuccess) return e;
  const uint64_t nchunks = (n + kMC - 1) / kMC;
  for (uint64_t w = kBT; w < n; w <<= 1) {
    const int ev = hooks.begin ? hooks.begin(st, 1, 2.0 * n * R) : -1;
    merge_partition_kernel<R><<<(unsigned)((nchunks + 1 + 255) / 256), 256, 0, st>>>(cur, n, w, split, nchunks);
    merge_pass_kernel<R><<<(unsigned)nchunks, kMT, 2 * kMC * sizeof(Rec), st>>>(cur, oth, n, w, split);
    if (hooks.end) hooks.end(ev, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    Rec* t = cur;
    cur = oth;
    oth = t;
  }
  return cudaSuccess;
}

}  // namespace

uint32_t merge_passes(uint64_t n) {
  uint32_t p = 0;
  for (uint64_t w = kBT; w < n; w <<= 1) ++p;
  return p;
}

uint64_t merge_split_entries(uint64_t n) { return (n + kMC - 1) / kMC + 1; }

cudaError_t launch_merge_sort(const void* in, void* buf0, void* buf1, uint64_t n, int R, uint64_t* split,
                              cudaStream_t st, const MergeHooks& hooks) {
  if (n == 0) return cudaSuccess;
  return R == 8 ? merge_sort_r<8>(in, buf0, buf1, n, split, st, hooks)
                : merge_sort_r<16>(in, buf0, buf1, n, split, st, hooks);
}

}  // namespace bos
