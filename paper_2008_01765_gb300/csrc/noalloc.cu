// bos_orp_noalloc: the bucket ORP for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the point where they need a
// permutation: code that runs inside a custom device allocator or its callbacks (allocating there
// would re-enter the allocator), and plugin hosts that own all device memory and forbid their
// guests to allocate. bos_orp needs a workspace the caller allocates; this entry point uses
// instead a fixed scratch array that is part of the library image, so the caller passes only its
// input and output.
//
// The scratch is a file-scope __device__ array. Host code cannot use its name as an address (the
// host-side symbol is only a stand-in), so every call looks the device address up with
// cudaGetSymbolAddress on the current device. That lookup is cheap and allocates nothing; looking
// it up per call (not once per device) keeps the address right after a device reset or under
// another context of the same device, where the module is loaded anew. The array is shared by
// every call on a device and keeps the previous call's contents; the ORP clears its control
// block and look-back words itself at the start of every attempt, and every other byte it reads
// was written earlier in the same call.
#include "bos.h"
#include "internal.h"

namespace {

static __device__ __align__(256) unsigned char g_scratch[BOS_NOALLOC_SCRATCH_BYTES];

// Device address of g_scratch on the current device.
bos_status scratch_address(void** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) {
    (void)cudaGetLastError();
    return BOS_ERR_CUDA;
  }
  *out = p;
  return BOS_OK;
}

}  // namespace

extern "C" bos_status bos_orp_noalloc(const void* d_in, void* d_out, uint64_t n, const bos_params* p,
                                      void* stream, bos_info* info) {
  if (!p) return BOS_ERR_INVALID;
  const size_t need = bos::orp_workspace_bytes(n, p);
  if (n && need == 0) return BOS_ERR_INVALID;        // invalid parameters
  if (need > BOS_NOALLOC_SCRATCH_BYTES) return BOS_ERR_WORKSPACE;  // n too large for the scratch
  void* ws = nullptr;
  if (n) {
    const bos_status s = scratch_address(&ws);
    if (s != BOS_OK) return s;
  }
  return bos::orp_with_workspace(d_in, d_out, n, p, ws, BOS_NOALLOC_SCRATCH_BYTES, stream, info);
}
