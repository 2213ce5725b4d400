// Self-test hook: evaluates the library's own Philox4x32-10 (the source of the labels of
// Algorithm 3.1 and of the in-bin permutation of Section 3.2) on caller-given counters and keys,
// and, beside it, cuRAND's device function curand_Philox4x32_10 on the same inputs, so a test can
// compare both against each other and against an independent host implementation.
#include <curand_kernel.h>

#include "bos.h"
#include "common.cuh"

namespace {

__global__ void philox_selftest_kernel(const uint32_t* ctr, const uint32_t* key, uint32_t* out,
                                       uint32_t* out_ref, uint64_t n) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t* c = ctr + 4 * i;
    const uint32_t* k = key + 2 * i;
    const bos::PhiloxOut o = bos::philox4x32_10(c[0], c[1], c[2], c[3], k[0], k[1]);
    out[4 * i + 0] = o.w0;
    out[4 * i + 1] = o.w1;
    out[4 * i + 2] = o.w2;
    out[4 * i + 3] = o.w3;
    if (out_ref) {
      const uint4 r = curand_Philox4x32_10(make_uint4(c[0], c[1], c[2], c[3]), make_uint2(k[0], k[1]));
      out_ref[4 * i + 0] = r.x;
      out_ref[4 * i + 1] = r.y;
      out_ref[4 * i + 2] = r.z;
      out_ref[4 * i + 3] = r.w;
    }
  }
}

}  // namespace

extern "C" bos_status bos_selftest_philox(const uint32_t* d_ctr, const uint32_t* d_key,
                                          uint32_t* d_out, uint32_t* d_out_curand, uint64_t n,
                                          void* stream) {
  if (n == 0) return BOS_OK;
  if (!d_ctr || !d_key || !d_out) return BOS_ERR_INVALID;
  const uint64_t blocks = (n + 255) / 256;
  philox_selftest_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, (cudaStream_t)stream>>>(
      d_ctr, d_key, d_out, d_out_curand, n);
  if (cudaGetLastError() != cudaSuccess) return BOS_ERR_CUDA;
  return BOS_OK;
}
