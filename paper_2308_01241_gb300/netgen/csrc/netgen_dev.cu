/*
 * netgen_dev.cu -- device side of the seeded synthetic network generator
 * (input generator; see netgen_core.h).  Builds the outgoing CSR of a network
 * too large to stage on the host (20M neurons x 500 inputs) directly in device
 * memory, from the same per-synapse draws as the host pull form:
 *   1. count the outgoing synapses of every neuron,
 *   2. exclusive scan -> row pointers,
 *   3. fill: every (neuron, input) pair writes its entry into its source row.
 * The order inside a row is not fixed (atomic slot claims); the simulated
 * result does not depend on it.
 */
#include <cuda_runtime.h>
#include <cub/device/device_scan.cuh>
#include <stdint.h>

#include "netgen_core.h"

namespace {

__device__ __forceinline__ int32_t voxel_of(const dg_net& g, int64_t i) {
  int32_t lo = 0, hi = g.nv - 1;
  while (lo < hi) {
    int32_t mid = (lo + hi + 1) >> 1;
    if (g.vstart[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void count_kernel(dg_net g, uint32_t* cnt) {
  const int64_t total = g.n * (int64_t)g.K;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
    const int64_t i = e / g.K;
    const int32_t k = (int32_t)(e - i * g.K);
    int32_t p, c;
    uint32_t b;
    dg_synapse(&g, i, voxel_of(g, i), k, &p, &c, &b);
    atomicAdd(&cnt[p], 1u);
  }
}

__global__ void widen_kernel(const uint32_t* cnt, int64_t* row_ptr, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) row_ptr[i] = cnt[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) row_ptr[n] = 0;
}

template <typename W>
__global__ void fill_kernel(dg_net g, const int64_t* row_ptr, uint32_t* fill, uint32_t* word, W* w,
                            const W* wtable) {
  const int64_t total = g.n * (int64_t)g.K;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
    const int64_t i = e / g.K;
    const int32_t k = (int32_t)(e - i * g.K);
    int32_t p, c;
    uint32_t b;
    dg_synapse(&g, i, voxel_of(g, i), k, &p, &c, &b);
    const int64_t q = row_ptr[p] + atomicAdd(&fill[p], 1u);
    word[q] = (uint32_t)i | ((uint32_t)c << 30);
    w[q] = wtable[b];
  }
}

// Warp per row: s = the smallest shift with round(max|w| / 2^s) <= 127, then
// q = sign(w) * round(|w| / 2^s) (halves rounded away from zero).
__global__ void quantize_int8_kernel(const int64_t* row_ptr, const int32_t* w32, int64_t n, int8_t* q8,
                                     uint8_t* row_shift) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = gw; r < n; r += nw) {
    const int64_t a = row_ptr[r], b = row_ptr[r + 1];
    uint32_t mx = 0;
    for (int64_t e = a + lane; e < b; e += 32) {
      const int32_t w = w32[e];
      const uint32_t m = (uint32_t)(w < 0 ? -(int64_t)w : w);
      mx = m > mx ? m : mx;
    }
    for (int o = 16; o > 0; o >>= 1) {
      const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, mx, o);
      mx = y > mx ? y : mx;
    }
    int s = 0;
    while (s < 31 && ((uint64_t)mx + ((1ull << s) >> 1)) >> s > 127) s++;
    if (lane == 0) row_shift[r] = (uint8_t)s;
    for (int64_t e = a + lane; e < b; e += 32) {
      const int32_t w = w32[e];
      const uint64_t m = (uint64_t)(w < 0 ? -(int64_t)w : w);
      const int32_t q = (int32_t)((m + ((1ull << s) >> 1)) >> s);
      q8[e] = (int8_t)(w < 0 ? -q : q);
    }
  }
}

}  // namespace

extern "C" {

/* int8 weights with one power-of-two scale per row from int32 weights:
 * w ~= q8 << row_shift.  All pointers are device memory.  Returns 0 or a
 * cudaError_t value. */
int dg_dev_quantize_int8(const int64_t* d_row_ptr, const int32_t* d_w32, int64_t n, int8_t* d_q8,
                         uint8_t* d_row_shift, void* stream_) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  quantize_int8_kernel<<<sms * 8, 256, 0, (cudaStream_t)stream_>>>(d_row_ptr, d_w32, n, d_q8, d_row_shift);
  return (int)cudaGetLastError();
}

/* Device CSR of the whole network.  g holds DEVICE pointers.  d_row_ptr is
 * int64[n+1]; d_word uint32[n*K]; d_w is [n*K] of w_bytes-wide entries taken
 * from d_wtable[4096]; d_cnt and d_fill are uint32[n] scratch.  Returns 0 or
 * a cudaError_t code. */
int dg_dev_build(const dg_net* g, int64_t* d_row_ptr, uint32_t* d_word, void* d_w, const void* d_wtable,
                 int w_bytes, uint32_t* d_cnt, uint32_t* d_fill, void* stream_) {
  cudaStream_t stream = (cudaStream_t)stream_;
  const int64_t n = g->n;
  const int threads = 256;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 8;
  cudaError_t err;
  if ((err = cudaMemsetAsync(d_cnt, 0, (size_t)n * 4, stream)) != cudaSuccess) return (int)err;
  if ((err = cudaMemsetAsync(d_fill, 0, (size_t)n * 4, stream)) != cudaSuccess) return (int)err;
  count_kernel<<<blocks, threads, 0, stream>>>(*g, d_cnt);
  widen_kernel<<<blocks, threads, 0, stream>>>(d_cnt, d_row_ptr, n);
  size_t tmp_bytes = 0;
  cub::DeviceScan::ExclusiveSum(nullptr, tmp_bytes, d_row_ptr, d_row_ptr, n + 1, stream);
  void* tmp = nullptr;
  if ((err = cudaMallocAsync(&tmp, tmp_bytes, stream)) != cudaSuccess) return (int)err;
  cub::DeviceScan::ExclusiveSum(tmp, tmp_bytes, d_row_ptr, d_row_ptr, n + 1, stream);
  cudaFreeAsync(tmp, stream);
  switch (w_bytes) {
    case 1: fill_kernel<int8_t><<<blocks, threads, 0, stream>>>(*g, d_row_ptr, d_fill, d_word, (int8_t*)d_w, (const int8_t*)d_wtable); break;
    case 2: fill_kernel<int16_t><<<blocks, threads, 0, stream>>>(*g, d_row_ptr, d_fill, d_word, (int16_t*)d_w, (const int16_t*)d_wtable); break;
    case 4: fill_kernel<int32_t><<<blocks, threads, 0, stream>>>(*g, d_row_ptr, d_fill, d_word, (int32_t*)d_w, (const int32_t*)d_wtable); break;
    default: return (int)cudaErrorInvalidValue;
  }
  err = cudaGetLastError();
  return (int)err;
}

}
