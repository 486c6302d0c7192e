// standalone_noalloc.cu -- dtb_spike_compact_noalloc: the kernel-level spike
// compaction of dtb_spike_compact, for callers that must not allocate.
//
// Some callers cannot allocate device memory while they run this step.  A
// host framework may own the whole device heap through its own pool.  A hard
// real-time loop may forbid calls that can block or synchronise the device,
// as cudaMalloc and cudaFree can.  A plugin may be handed buffers but have
// no allocator of its own.  This variant keeps its scratch (the per-block
// spike counts and two 8-byte words) in a fixed file-scope device array.
// Every GPU that loads the library holds that array until the process
// exits; no call allocates or frees anything.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "dtb.h"
#include "dtb_device.cuh"
#include "dtb_launch.h"

namespace {

// 4 bytes per 1024 neurons for DTB_NOALLOC_MAX_NEURONS neurons, plus 16 bytes.
constexpr size_t kScratchBytes = (size_t)4 * (DTB_NOALLOC_MAX_NEURONS / 1024) + 16;
static __device__ __align__(256) unsigned char g_compact_scratch[kScratchBytes];

// Device address of the scratch array on the current device.  Host code may
// not use the symbol itself as a pointer.  It is looked up on every call (a
// host-side lookup that allocates nothing), so that a device reset, after
// which the module is loaded again and the array may move, leaves no stale
// address behind.
cudaError_t scratch_address(void** out) { return cudaGetSymbolAddress(out, g_compact_scratch); }

}  // namespace

extern "C" dtb_status dtb_spike_compact_noalloc(const uint32_t* d_bits, int64_t n, int32_t* d_ids,
                                                int32_t* d_count, void* stream) {
  if (!d_bits || !d_ids || !d_count) {
    return dtb::set_last_error(DTB_EINVAL, "dtb_spike_compact_noalloc: NULL buffer");
  }
  if (n < 1 || n > DTB_NOALLOC_MAX_NEURONS) {
    return dtb::set_last_error(DTB_EINVAL, "dtb_spike_compact_noalloc: n must be in 1.." +
                                               std::to_string(DTB_NOALLOC_MAX_NEURONS) +
                                               " (the size of its fixed scratch); use dtb_spike_compact for larger n");
  }
  void* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) {
    return dtb::set_last_error(DTB_ECUDA, std::string("dtb_spike_compact_noalloc: cudaGetSymbolAddress: ") +
                                              cudaGetErrorString(e));
  }
  e = dtb::compact_bits(d_bits, n, d_ids, d_count, scratch, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    return dtb::set_last_error(DTB_ECUDA, std::string("dtb_spike_compact_noalloc: ") + cudaGetErrorString(e));
  }
  return DTB_OK;
}
