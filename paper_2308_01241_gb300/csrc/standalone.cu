// standalone.cu -- the spike compaction of the step as a kernel-level entry
// point on caller-given device buffers ("collect spikes sequence", section
// V.B): a spike bit set in, ascending spike ids and their count out.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dtb.h"
#include "dtb_device.cuh"
#include "dtb_launch.h"

namespace dtb {
namespace {

// One warp per 1024-bit block: the block's spike count.
__global__ void block_count_kernel(const uint32_t* bits, int32_t nblk, int32_t* blk_cnt) {
  const int32_t b = (int32_t)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (b >= nblk) return;
  const int lane = threadIdx.x & 31;
  const int c = __reduce_add_sync(0xFFFFFFFFu, __popc(bits[(int64_t)b * 32 + lane]));
  if (lane == 0) blk_cnt[b] = c;
}

}  // namespace

// Count + compaction on a DevNet view of caller buffers; scratch holds the
// block counts [nblk] followed by two 8-byte words (log position, spike sum).
cudaError_t compact_bits(const uint32_t* bits, int64_t n, int32_t* ids, int32_t* count, void* scratch,
                         cudaStream_t st) {
  DevNet g{};
  g.n = n;
  g.nblk = (int32_t)((n + kNeuronsPerBlock - 1) / kNeuronsPerBlock);
  g.npad = (int64_t)g.nblk * kNeuronsPerBlock;
  g.ntiles = (g.nblk + kCompactBlocksPerTile - 1) / kCompactBlocksPerTile;
  g.flags = const_cast<uint32_t*>(bits);
  g.blk_cnt = (int32_t*)scratch;
  int64_t* words = (int64_t*)((char*)scratch + compact_scratch_bytes(n) - 16);
  g.log_pos = words;
  g.spikes = (unsigned long long*)(words + 1);
  g.log_ids = nullptr;
  g.log_cap = 0;
  g.spk = ids;
  g.n_spk = count;
  cudaError_t e = cudaMemsetAsync(words, 0, 16, st);
  if (e != cudaSuccess) return e;
  block_count_kernel<<<(unsigned)((g.nblk * 32 + 255) / 256), 256, 0, st>>>(bits, g.nblk, g.blk_cnt);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_spike_compact(g, 0, st, 1);
}

size_t compact_scratch_bytes(int64_t n) {
  const int64_t nblk = (n + kNeuronsPerBlock - 1) / kNeuronsPerBlock;
  return (size_t)(((4 * nblk + 15) / 16) * 16 + 16);
}

}  // namespace dtb
