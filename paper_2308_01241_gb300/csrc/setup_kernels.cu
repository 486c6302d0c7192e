// setup_kernels.cu -- kernels run once per network (initial state, synapse
// table validation and int32 overflow bound) and the Philox test hook.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dtb_device.cuh"
#include "dtb_launch.h"

namespace dtb {
namespace {

// V0 = Vreset + (Vth - Vreset) * ((word >> 8) * 2^-24), word = Philox({i/4, 0, 0, INIT})[i mod 4].
__global__ void init_voltage_kernel(DevNet g, uint32_t k0, uint32_t k1) {
  const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (i0 >= g.npad) return;
  const uint4 r = philox4x32_10(make_uint4((uint32_t)(i0 >> 2), 0u, 0u, kTagInit), k0, k1);
  const uint32_t rq[4] = {r.x, r.y, r.z, r.w};
  float out[4];
  int32_t v = g.blk_vox[i0 / kNeuronsPerBlock];
#pragma unroll
  for (int q = 0; q < 4; q++) {
    while (v + 1 < g.nv && g.vstart[v + 1] <= i0 + q) v++;
    const VoxConst* c = g.vc + v;
    const float u = __fmul_rn((float)(rq[q] >> 8), 5.9604644775390625e-08f);  // 2^-24, exact
    const float span = __fsub_rn(c->Vth, c->Vreset);
    out[q] = __fadd_rn(c->Vreset, __fmul_rn(span, u));
  }
  *reinterpret_cast<float4*>(g.V + i0) = make_float4(out[0], out[1], out[2], out[3]);
}

template <int WFMT>
__device__ __forceinline__ int64_t acc_weight(const DevNet& g, int64_t e, int shift) {
  if (WFMT == 0) return (int64_t)reinterpret_cast<const int16_t*>(g.w)[e] * ((int64_t)1 << shift);
  if (WFMT == 1) return (int64_t)reinterpret_cast<const int32_t*>(g.w)[e] * ((int64_t)1 << shift);
  if (WFMT == 2) {
    const uint32_t b = (uint32_t)reinterpret_cast<const unsigned short*>(g.w)[e] << 16;
    const float x = __fmul_rn(__uint_as_float(b), 65536.0f);
    if (!(fabsf(x) < 2147483520.0f)) return (int64_t)1 << 40;
    return (int64_t)__float2int_rn(x);
  }
  return (int64_t)reinterpret_cast<const signed char*>(g.w)[e] * ((int64_t)1 << shift);
}

// Warp per row.  Rows must be ascending and within [0, nnz]; every entry's
// target < n and class < nch; |w_acc| summed per (target, channel).
template <int WFMT>
__global__ void check_kernel(DevNet g, unsigned long long* insum, int* bad) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = gw; s < g.n; s += nw) {
    const int64_t r0 = g.row_ptr[s], r1 = g.row_ptr[s + 1];
    if (r1 < r0) {
      if (lane == 0) atomicOr(bad, 1);
      continue;
    }
    const int shift = WFMT == 3 ? g.wshift + (g.row_shift ? g.row_shift[s] : 0) : g.wshift;
    if (WFMT == 3 && shift > 30 && r1 > r0) {  // a shifted int8 weight must stay an int32
      if (lane == 0) atomicOr(bad, 4);
      continue;
    }
    for (int64_t e = r0 + lane; e < r1; e += 32) {
      const uint32_t wd = g.word[e];
      const int64_t tgt = wd & 0x3FFFFFFFu;
      const int32_t c = (int32_t)(wd >> 30);
      if (tgt >= g.n || c >= g.nch) {
        atomicOr(bad, 2);
        continue;
      }
      int64_t w = acc_weight<WFMT>(g, e, shift);
      if (w > 2147483647LL || w < -2147483648LL) {
        atomicOr(bad, 4);
        continue;
      }
      if (w < 0) w = -w;
      atomicAdd(insum + (int64_t)c * g.npad + tgt, (unsigned long long)w);
    }
  }
}

// Warp per row: the delay of every synapse, delay[vox(source)][vox(target)].
// Work items per neuron, ceil(row length / kItemEvents), one byte each; a
// count above 255 sets *too_long.
__global__ void item_count_kernel(DevNet g, uint8_t* out, int32_t* too_long) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.npad; i += stride) {
    int64_t c = 0;
    if (i < g.n) c = (g.row_ptr[i + 1] - g.row_ptr[i] + kItemEvents - 1) / kItemEvents;
    if (c > 255) {
      atomicOr(too_long, 1);
      c = 255;
    }
    out[i] = (uint8_t)c;
  }
}

__global__ void delay_fill_kernel(DevNet g, uint8_t* out) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = gw; s < g.n; s += nw) {
    const uint8_t* drow = g.delay + (int64_t)voxel_of(g, (int32_t)s) * g.nv;
    const int64_t r0 = g.row_ptr[s], r1 = g.row_ptr[s + 1];
    for (int64_t e = r0 + lane; e < r1; e += 32) out[e] = drow[voxel_of(g, (int32_t)(g.word[e] & 0x3FFFFFFFu))];
  }
}

// Sort key of a packed record (word = target | class << 30, y = weight code |
// delay << 16): delay, then target, then class and code.  It is a lossless
// repacking, so the record is recovered from the key.
__device__ __forceinline__ unsigned long long record_key(uint32_t wd, uint32_t y) {
  return ((unsigned long long)(y >> 16) << 48) | ((unsigned long long)(wd & 0x3FFFFFFFu) << 18) |
         ((unsigned long long)(wd >> 30) << 16) | (unsigned long long)(y & 0xFFFFu);
}
__device__ __forceinline__ uint2 key_record(unsigned long long k) {
  return make_uint2((uint32_t)((k >> 18) & 0x3FFFFFFFu) | ((uint32_t)((k >> 16) & 3u) << 30),
                    (uint32_t)(k & 0xFFFFu) | ((uint32_t)(k >> 48) << 16));
}

// Bitonic sort of 32 * R keys held by one warp, element i = r * 32 + lane in
// register r of lane `lane`: distances below 32 exchange across lanes,
// larger ones inside a lane.  Ascending.
template <int R>
__device__ __forceinline__ void warp_bitonic_sort(unsigned long long (&v)[R], int lane) {
#pragma unroll
  for (int k = 2; k <= 32 * R; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j >= 32) {
        const int jj = j >> 5;
#pragma unroll
        for (int r = 0; r < R; r++) {
          if ((r & jj) == 0) {
            const bool asc = ((r * 32) & k) == 0;  // k >= 64 > lane: bit k of i is bit k of r * 32
            const unsigned long long a = v[r], b = v[r | jj];
            const bool sw = asc ? (a > b) : (a < b);
            v[r] = sw ? b : a;
            v[r | jj] = sw ? a : b;
          }
        }
      } else {
        const bool lower = (lane & j) == 0;  // my element has the lower index of its pair
#pragma unroll
        for (int r = 0; r < R; r++) {
          const bool asc = (((r * 32) | lane) & k) == 0;
          const unsigned long long o = __shfl_xor_sync(0xFFFFFFFFu, v[r], j);
          const bool take_min = lower == asc;
          v[r] = take_min ? (o < v[r] ? o : v[r]) : (o > v[r] ? o : v[r]);
        }
      }
    }
  }
}

// Run key of a packed record (word, code | delay << 16): the arrival step's
// queue for delay d > 1, the target region's bin for delay 1 in bins mode
// (every delay-1 event shares one key in the event-queue mode).
__device__ __forceinline__ uint32_t record_run_key(uint2 rec, bool bins) {
  const uint32_t d = (rec.y >> 16) & 0xFFu;
  if (d > 1) return d;
  return bins ? (kRunRegion | ((rec.x & 0x3FFFFFFFu) >> kRegionShift)) : kRunRegion;
}

// Warp per row: the packed record of every synapse, (word, weight code |
// delay << 16), the delay from the voxel-pair table.  Each chunk of
// kItemEvents synapses (one delivery work item) is then sorted by delay and
// target, so that its events wait in few places (runs), and the chunk's run
// count goes to counts[chunk_base[row] + k].  The order of a row's synapses
// changes no result: the sums are exact integers.
template <int WFMT>
__global__ void __launch_bounds__(256) pack_fill_kernel(DevNet g, uint2* out, int32_t* counts) {
  constexpr int R = kItemEvents / 32;
  const int lane = threadIdx.x & 31;
  const bool bins = g.mode == kModeBins;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = gw; s < g.n; s += nw) {
    const uint8_t* drow = g.delay + (int64_t)voxel_of(g, (int32_t)s) * g.nv;
    const int shift = WFMT == 3 ? g.wshift + (g.row_shift ? g.row_shift[s] : 0) : g.wshift;
    const int64_t r0 = g.row_ptr[s], r1 = g.row_ptr[s + 1];
    int64_t chunk = g.chunk_base[s];
    for (int64_t c0 = r0; c0 < r1; c0 += kItemEvents, chunk++) {
      unsigned long long v[R];
#pragma unroll
      for (int r = 0; r < R; r++) {
        const int64_t e = c0 + r * 32 + lane;
        v[r] = ~0ull;  // padding sorts last
        if (e < r1) {
          const uint32_t wd = g.word[e];
          const uint32_t d = drow[voxel_of(g, (int32_t)(wd & 0x3FFFFFFFu))];
          v[r] = record_key(wd, weight_code<WFMT>(g.w, e, shift) | (d << 16));
        }
      }
      warp_bitonic_sort<R>(v, lane);
      int runs = 0;
      uint32_t last = 0xFFFFFFFFu;  // key of the element before this round's first
#pragma unroll
      for (int r = 0; r < R; r++) {
        const int64_t e = c0 + r * 32 + lane;
        const bool valid = e < r1;
        const uint2 rec = key_record(v[r]);
        const uint32_t k = valid ? record_run_key(rec, bins) : 0xFFFFFFFFu;
        uint32_t left = __shfl_up_sync(0xFFFFFFFFu, k, 1);
        if (lane == 0) left = last;
        runs += __popc(__ballot_sync(0xFFFFFFFFu, valid && k != left));
        last = __shfl_sync(0xFFFFFFFFu, k, 31);
        if (valid) out[e] = rec;
      }
      if (lane == 0) counts[chunk] = runs;
    }
  }
}

// Warp per row, after pack_fill and the run pointers: every chunk's run
// records (key | start << 14 | (length - 1) << 23) at runs[run_ptr[chunk]..],
// and each packed record's delay byte replaced by its run's index.
__global__ void __launch_bounds__(256) run_fill_kernel(DevNet g, uint2* pack, const int64_t* run_ptr,
                                                       uint32_t* runs) {
  constexpr int R = kItemEvents / 32;
  const int lane = threadIdx.x & 31;
  const bool bins = g.mode == kModeBins;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = gw; s < g.n; s += nw) {
    const int64_t r0 = g.row_ptr[s], r1 = g.row_ptr[s + 1];
    int64_t chunk = g.chunk_base[s];
    for (int64_t c0 = r0; c0 < r1; c0 += kItemEvents, chunk++) {
      uint32_t k[R];
      uint2 rec[R];
#pragma unroll
      for (int r = 0; r < R; r++) {
        const int64_t e = c0 + r * 32 + lane;
        rec[r] = e < r1 ? pack[e] : make_uint2(0u, 0u);
        k[r] = e < r1 ? record_run_key(rec[r], bins) : 0xFFFFFFFFu;
      }
      uint32_t* out = runs + run_ptr[chunk];
      int before = 0;  // runs that start before this round
      bool tail[R];
      int idx[R];
#pragma unroll
      for (int r = 0; r < R; r++) {
        uint32_t left = __shfl_up_sync(0xFFFFFFFFu, k[r], 1);
        const uint32_t prev_last = r > 0 ? __shfl_sync(0xFFFFFFFFu, k[r > 0 ? r - 1 : 0], 31) : 0xFFFFFFFFu;
        if (lane == 0) left = prev_last;
        uint32_t right = __shfl_down_sync(0xFFFFFFFFu, k[r], 1);
        const uint32_t next_first = r + 1 < R ? __shfl_sync(0xFFFFFFFFu, k[r + 1 < R ? r + 1 : r], 0) : 0xFFFFFFFFu;
        if (lane == 31) right = next_first;
        const bool valid = k[r] != 0xFFFFFFFFu;
        const bool head = valid && k[r] != left;
        tail[r] = valid && k[r] != right;
        const unsigned hb = __ballot_sync(0xFFFFFFFFu, head);
        idx[r] = before + __popc(hb & (0xFFFFFFFFu >> (31 - lane))) - 1;
        if (head) out[idx[r]] = k[r] | ((uint32_t)(r * 32 + lane) << 14);
        before += __popc(hb);
      }
      __syncwarp();
#pragma unroll
      for (int r = 0; r < R; r++) {
        const int64_t e = c0 + r * 32 + lane;
        if (tail[r]) {
          const uint32_t h = out[idx[r]];
          out[idx[r]] = h | ((uint32_t)(r * 32 + lane - run_start(h)) << 23);
        }
        if (e < r1) pack[e] = make_uint2(rec[r].x, (rec[r].y & 0xFFFFu) | ((uint32_t)idx[r] << 16));
      }
      __syncwarp();
    }
  }
}

__global__ void max_kernel(const unsigned long long* a, int64_t m, unsigned long long* out) {
  unsigned long long best = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    best = a[i] > best ? a[i] : best;
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long x = __shfl_xor_sync(0xFFFFFFFFu, best, o);
    best = x > best ? x : best;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(out, best);
}

// One block row per (slot, channel) pair; int64 sums by two's-complement adds.
__global__ void ring_sums_kernel(DevNet g, unsigned long long* sums) {
  const int64_t pair = blockIdx.y;
  const int32_t* row = g.ring + pair * g.npad;
  long long acc = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x)
    acc += row[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(sums + pair, (unsigned long long)acc);
}

__global__ void ring_gather_kernel(DevNet g, const int64_t* idx, int64_t m, int32_t* out) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per = (int64_t)g.D * g.nch;
  if (k >= m * per) return;
  const int64_t r = k / per, sc = k - r * per;  // sc = slot * nch + c
  out[k] = g.ring[sc * g.npad + idx[r]];
}

// ---- event-queue mode: the dense ring view of the pending events ----
// Queue x (x != t mod D) holds the events arriving at the step congruent to x;
// the one-slot accumulator holds slot t mod D (t = the next step to run).
// Bins mode: every queue is a slot (x_acc = -1) and its events carry weight
// codes.
__device__ __forceinline__ int32_t queued_weight(const DevNet& g, uint32_t w) {
  return g.mode == kModeBins ? decode_weight(w, g.wfmt, g.wshift) : (int32_t)w;
}

// Test hook of the counters: every queue (blockIdx.y < D) and, in bins mode,
// every bin (blockIdx.y = D + parity * n_reg + region) gets its unused
// entries filled with placeholder events of weight 0 (target 0, class 0,
// weight code 0), then its count set to value (>= its capacity).
__global__ void preset_counters_kernel(DevNet g, unsigned long long value) {
  const int64_t y = blockIdx.y;
  const bool queue = y < g.D;
  const int64_t cap = queue ? g.qcap : g.bcap;
  unsigned long long* cnt = queue ? g.qcnt + y * kQcntStride : g.bcnt + (y - g.D) * kBcntStride;
  const int64_t used = (int64_t)min(*cnt, (unsigned long long)cap);
  for (int64_t i = used + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += (int64_t)gridDim.x * blockDim.x) {
    if (queue) g.q[y * g.qcap + i] = make_uint2(0u, 0u);
    else if (g.ev8) reinterpret_cast<uint2*>(g.bins)[(y - g.D) * g.bcap + i] = make_uint2(0u, 0u);
    else g.bins[(y - g.D) * g.bcap + i] = 0u;
  }
}

__global__ void set_counters_kernel(DevNet g, unsigned long long value) {
  const int64_t y = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nb = g.mode == kModeBins ? 2 * (int64_t)g.n_reg : 0;
  if (y < g.D) g.qcnt[y * kQcntStride] = value;
  else if (y < g.D + nb) g.bcnt[(y - g.D) * kBcntStride] = value;
}

__global__ void queue_to_dense_kernel(DevNet g, int32_t* dense, int32_t x_acc) {
  const int32_t x = blockIdx.y;
  if (x == x_acc) return;
  const int64_t cnt = (int64_t)min(g.qcnt[x * kQcntStride], (unsigned long long)g.qcap);
  const uint2* q = g.q + (int64_t)x * g.qcap;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
    const uint2 e = q[i];
    atomicAdd(dense + ((int64_t)x * g.nch + (e.x >> 30)) * g.npad + (e.x & 0x3FFFFFFFu), queued_weight(g, e.y));
  }
}

__global__ void dense_to_queue_kernel(DevNet g, const int32_t* dense, int32_t x_acc) {
  const int32_t x = blockIdx.y;
  if (x == x_acc) return;
  const int64_t per = (int64_t)g.nch * g.npad;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < per; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = (int32_t)(k / g.npad);
    const int64_t i = k - (int64_t)c * g.npad;
    const int32_t w = dense[(int64_t)x * per + k];
    if (w == 0 || i >= g.n) continue;
    const unsigned long long pos = atomicAdd(g.qcnt + x * kQcntStride, 1ull);
    if (pos >= (unsigned long long)g.qcap) {
      atomicAdd(g.spill + (int64_t)x * per + k, w);
      g.spill_dirty[x] = 1;
      continue;
    }
    g.q[(int64_t)x * g.qcap + pos] = make_uint2((uint32_t)i | ((uint32_t)c << 30), (uint32_t)w);
  }
}

__global__ void queue_sums_kernel(DevNet g, unsigned long long* sums, int32_t x_acc) {
  const int32_t x = blockIdx.y;
  if (x == x_acc) return;
  const int64_t cnt = (int64_t)min(g.qcnt[x * kQcntStride], (unsigned long long)g.qcap);
  const uint2* q = g.q + (int64_t)x * g.qcap;
  long long acc[4] = {0, 0, 0, 0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
    const uint2 e = q[i];
    acc[e.x >> 30] += queued_weight(g, e.y);
  }
  for (int c = 0; c < 4; c++) {
    long long a = acc[c];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
    if ((threadIdx.x & 31) == 0 && a != 0 && c < g.nch) atomicAdd(sums + x * g.nch + c, (unsigned long long)a);
  }
}

// out [m][D][nch]: map [n] gives the row of a requested neuron (or -1).
__global__ void queue_gather_kernel(DevNet g, const int32_t* map, int32_t* out, int32_t x_acc) {
  const int32_t x = blockIdx.y;
  if (x == x_acc) return;
  const int64_t cnt = (int64_t)min(g.qcnt[x * kQcntStride], (unsigned long long)g.qcap);
  const uint2* q = g.q + (int64_t)x * g.qcap;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
    const uint2 e = q[i];
    const int32_t r = map[e.x & 0x3FFFFFFFu];
    if (r >= 0) atomicAdd(out + ((int64_t)r * g.D + x) * g.nch + (e.x >> 30), queued_weight(g, e.y));
  }
}

// Bins mode: between calls the bins of parity x mod 2 hold the delay-1 events
// of the last delivery, due at step x (the next step to run, ring slot x mod D).
// The three views of the dense ring add them in: into a dense ring, into the
// per-slot sums, into the gathered entries of the neurons in map.
__device__ __forceinline__ void bin_event(const DevNet& g, const uint32_t* bin, int64_t e, uint32_t& loc,
                                          int32_t& w) {
  if (g.ev8) {
    const uint2 v = reinterpret_cast<const uint2*>(bin)[e];
    loc = v.x;
    w = decode_weight(v.y, g.wfmt, g.wshift);
  } else {
    const uint32_t v = bin[e];
    loc = v & 0xFFFFu;
    w = decode_weight(v >> 16, g.wfmt, g.wshift);
  }
}

__global__ void bins_view_kernel(DevNet g, int64_t x, int32_t* dense, unsigned long long* sums, const int32_t* map,
                                 int32_t* out) {
  const int r = blockIdx.y;
  const int par = (int)(x & 1);
  const int32_t slot = (int32_t)(x % g.D);
  const int ew = g.ev8 ? 2 : 1;
  const int64_t cnt = (int64_t)min(g.bcnt[((int64_t)par * g.n_reg + r) * kBcntStride], (unsigned long long)g.bcap);
  const uint32_t* bin = g.bins + ((int64_t)par * g.n_reg + r) * g.bcap * ew;
  long long acc[4] = {0, 0, 0, 0};
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x) {
    uint32_t loc;
    int32_t w;
    bin_event(g, bin, e, loc, w);
    const uint32_t cls = (loc >> kRegionShift) & 3u;
    const int64_t tgt = (int64_t)r * kRegionNeurons + (loc & (kRegionNeurons - 1));
    if (dense) atomicAdd(dense + ((int64_t)slot * g.nch + cls) * g.npad + tgt, w);
    if (sums) acc[cls] += w;
    if (map) {
      const int32_t row = map[tgt];
      if (row >= 0) atomicAdd(out + ((int64_t)row * g.D + slot) * g.nch + cls, w);
    }
  }
  if (sums)
    for (int c = 0; c < 4; c++) {
      long long a = acc[c];
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
      if ((threadIdx.x & 31) == 0 && a != 0 && c < g.nch) atomicAdd(sums + slot * g.nch + c, (unsigned long long)a);
    }
}

__global__ void acc_gather_kernel(DevNet g, const int64_t* idx, int64_t m, int32_t* out, int32_t x_acc) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m * g.nch) return;
  const int64_t r = k / g.nch;
  const int32_t c = (int32_t)(k - r * g.nch);
  out[(r * g.D + x_acc) * g.nch + c] += g.ring[(int64_t)c * g.npad + idx[r]];
}

__global__ void add_kernel(int32_t* dst, const int32_t* src, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] += src[i];
}

__global__ void map_kernel(const int64_t* idx, int64_t m, int32_t* map) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < m) map[idx[r]] = (int32_t)r;
}

__global__ void philox_kernel(const uint4* ctr, const uint2* key, uint4* out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = philox4x32_10(ctr[i], key[i].x, key[i].y);
}

}  // namespace

cudaError_t launch_init_voltage(const DevNet& g, uint64_t init_seed, cudaStream_t st) {
  const int64_t threads = g.npad / 4;
  init_voltage_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(g, (uint32_t)init_seed,
                                                                          (uint32_t)(init_seed >> 32));
  return cudaGetLastError();
}

cudaError_t launch_check_synapses(const DevNet& g, unsigned long long* insum, int* bad,
                                  unsigned long long* max_insum, cudaStream_t st) {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 8;
  switch (g.wfmt) {
    case 0: check_kernel<0><<<blocks, 256, 0, st>>>(g, insum, bad); break;
    case 1: check_kernel<1><<<blocks, 256, 0, st>>>(g, insum, bad); break;
    case 2: check_kernel<2><<<blocks, 256, 0, st>>>(g, insum, bad); break;
    default: check_kernel<3><<<blocks, 256, 0, st>>>(g, insum, bad); break;
  }
  max_kernel<<<blocks, 256, 0, st>>>(insum, (int64_t)g.nch * g.npad, max_insum);
  return cudaGetLastError();
}

cudaError_t launch_ring_sums(const DevNet& g, unsigned long long* sums, cudaStream_t st) {
  dim3 grid(64, (unsigned)(g.D * g.nch));
  ring_sums_kernel<<<grid, 256, 0, st>>>(g, sums);
  return cudaGetLastError();
}

cudaError_t launch_ring_gather(const DevNet& g, const int64_t* idx, int64_t m, int32_t* out, cudaStream_t st) {
  const int64_t total = m * g.D * g.nch;
  if (total <= 0) return cudaSuccess;
  ring_gather_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(g, idx, m, out);
  return cudaGetLastError();
}

cudaError_t launch_queue_to_dense(const DevNet& g, int32_t* dense, int32_t x_acc, cudaStream_t st) {
  queue_to_dense_kernel<<<dim3(64, (unsigned)g.D), 256, 0, st>>>(g, dense, x_acc);
  return cudaGetLastError();
}

cudaError_t launch_bins_view(const DevNet& g, int64_t x, int32_t* dense, unsigned long long* sums,
                             const int32_t* map, int32_t* out, cudaStream_t st) {
  if (g.mode != kModeBins || g.n_reg < 1) return cudaSuccess;
  bins_view_kernel<<<dim3(8, (unsigned)g.n_reg), 256, 0, st>>>(g, x, dense, sums, map, out);
  return cudaGetLastError();
}

cudaError_t launch_add(int32_t* dst, const int32_t* src, int64_t n, cudaStream_t st) {
  add_kernel<<<1024, 256, 0, st>>>(dst, src, n);
  return cudaGetLastError();
}

cudaError_t launch_preset_counters(const DevNet& g, unsigned long long value, cudaStream_t st) {
  const int64_t rows = g.D + (g.mode == kModeBins ? 2 * (int64_t)g.n_reg : 0);
  preset_counters_kernel<<<dim3(8, (unsigned)rows), 256, 0, st>>>(g, value);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  set_counters_kernel<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(g, value);  // after every fill has read its count
  return cudaGetLastError();
}

cudaError_t launch_dense_to_queue(const DevNet& g, const int32_t* dense, int32_t x_acc, cudaStream_t st) {
  dense_to_queue_kernel<<<dim3(64, (unsigned)g.D), 256, 0, st>>>(g, dense, x_acc);
  return cudaGetLastError();
}

cudaError_t launch_queue_sums(const DevNet& g, unsigned long long* sums, int32_t x_acc, cudaStream_t st) {
  queue_sums_kernel<<<dim3(64, (unsigned)g.D), 256, 0, st>>>(g, sums, x_acc);
  return cudaGetLastError();
}

cudaError_t launch_queue_gather(const DevNet& g, const int64_t* idx, int64_t m, int32_t* map, int32_t* out,
                                int32_t x_acc, cudaStream_t st) {
  // map: int32 [n], all -1 on entry.  out starts as the spill ring's entries.
  {
    DevNet sp = g;
    sp.ring = g.spill;
    const int64_t total = m * g.D * g.nch;
    ring_gather_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(sp, idx, m, out);
  }
  map_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(idx, m, map);
  queue_gather_kernel<<<dim3(64, (unsigned)g.D), 256, 0, st>>>(g, map, out, x_acc);
  if (x_acc >= 0) acc_gather_kernel<<<(unsigned)((m * g.nch + 255) / 256), 256, 0, st>>>(g, idx, m, out, x_acc);
  return cudaGetLastError();
}

// The bounded wait of the neuron update's pipeline on an mbarrier: with
// arrive = 0 nothing ever arrives, so the wait gives up after max_cycles and
// the kernel reports it in *status (1); with arrive = 1 the barrier completes
// first and *status is 0.  No asynchronous copy is involved.
__global__ void bounded_wait_kernel(long long max_cycles, int32_t arrive, int32_t* status) {
  __shared__ uint64_t bar;
  mbar_init(&bar, 1);
  fence_mbar_init();
  if (arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar)) : "memory");
  *status = mbar_wait_bounded(&bar, 0, max_cycles) ? 0 : 1;
}

cudaError_t launch_bounded_wait(long long max_cycles, int32_t arrive, int32_t* status, cudaStream_t st) {
  bounded_wait_kernel<<<1, 1, 0, st>>>(max_cycles, arrive, status);
  return cudaGetLastError();
}

cudaError_t launch_item_count(const DevNet& g, uint8_t* out, int32_t* too_long, cudaStream_t st) {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  item_count_kernel<<<sms * 4, 256, 0, st>>>(g, out, too_long);
  return cudaGetLastError();
}

cudaError_t launch_delay_fill(const DevNet& g, uint8_t* out, cudaStream_t st) {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  delay_fill_kernel<<<sms * 8, 256, 0, st>>>(g, out);
  return cudaGetLastError();
}

cudaError_t launch_pack_fill(const DevNet& g, uint2* out, int32_t* counts, cudaStream_t st) {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  switch (g.wfmt) {
    case 0: pack_fill_kernel<0><<<sms * 8, 256, 0, st>>>(g, out, counts); break;
    case 2: pack_fill_kernel<2><<<sms * 8, 256, 0, st>>>(g, out, counts); break;
    case 3: pack_fill_kernel<3><<<sms * 8, 256, 0, st>>>(g, out, counts); break;
    default: return cudaErrorInvalidValue;  // int32 weights do not fit a 16-bit code
  }
  return cudaGetLastError();
}

cudaError_t launch_run_fill(const DevNet& g, uint2* pack, const int64_t* run_ptr, uint32_t* runs, cudaStream_t st) {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  run_fill_kernel<<<sms * 8, 256, 0, st>>>(g, pack, run_ptr, runs);
  return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  philox_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(reinterpret_cast<const uint4*>(ctr),
                                                              reinterpret_cast<const uint2*>(key),
                                                              reinterpret_cast<uint4*>(out), n);
  return cudaGetLastError();
}

}  // namespace dtb
