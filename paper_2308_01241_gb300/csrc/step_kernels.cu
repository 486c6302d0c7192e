// step_kernels.cu -- the four kernels of one simulation step and their launchers.
//
//   neuron_update  Eq. 1 by explicit Euler (sections III.B, VI.A), Poisson drive,
//                  threshold / reset / refractory; spike bits by warp ballot
//   spike_compact  ascending spike ids from the bits: per-block counts,
//                  prefix sums, popc ranks ("collect spikes sequence", IV.B)
//   spike_deliver  outgoing CSR rows of the spiking neurons -> int32 adds into
//                  the delay ring (J sums of section IV.B)
//   bold_step      Balloon-Windkessel per voxel (section IV.E, Friston 2000)
//
// Every floating-point operation of the neuron update is an explicit
// round-to-nearest intrinsic, in the order the header dtb.h states, so no
// multiply-add is ever fused and the result is bit-identical to the C oracle.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dtb_device.cuh"
#include "dtb_launch.h"

namespace dtb {
namespace {

__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }

// One neuron, one step.  A[] are the consumed accumulators, u the Philox word.
template <int NCH>
__device__ __forceinline__ bool update_neuron(const DevNet& g, const VoxConst& c, float& V, float (&jj)[4],
                                              uint32_t& ref, const int32_t (&A)[NCH], uint32_t u) {
  int32_t k = 0;
#pragma unroll
  for (int m = 0; m < kMaxPoisson; m++)
    if (m < g.M) k += (u >= g.T[m]) ? 1 : 0;
  int32_t in[4];
  if (NCH == 2) {
    in[0] = A[0] + k * g.w_ext;
    in[1] = A[0];
    in[2] = A[1];
    in[3] = A[1];
  } else {
    in[0] = A[0] + k * g.w_ext;
    in[1] = A[1 % NCH];
    in[2] = A[2 % NCH];
    in[3] = A[3 % NCH];
  }
  const float SC = 1.52587890625e-05f;  // 2^-16
  float a[4];
#pragma unroll
  for (int q = 0; q < 4; q++) a[q] = fmul(__int2float_rn(in[q]), SC);
  float s = 0.0f;
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const float x = fsub(V, c.E[q]);
    const float y = fmul(c.kU[q], jj[q]);
    s = fadd(s, fmul(y, x));
  }
  float Vn = fsub(V, fmul(c.kL, fsub(V, c.EL)));
  Vn = fsub(Vn, s);
  Vn = fadd(Vn, c.kI);
#pragma unroll
  for (int q = 0; q < 4; q++) jj[q] = fadd(fmul(c.dJ[q], jj[q]), a[q]);
  bool spike = false;
  if (ref > 0) {
    ref -= 1;
    Vn = c.Vreset;
  } else if (Vn >= c.Vth) {
    spike = true;
    Vn = c.Vreset;
    ref = (uint32_t)c.ref_steps;
  }
  V = Vn;
  return spike;
}

__device__ __forceinline__ VoxConst load_vc(const VoxConst* p) {
  VoxConst c;
  const float4* s = reinterpret_cast<const float4*>(p);
  float4* d = reinterpret_cast<float4*>(&c);
#pragma unroll
  for (int q = 0; q < 5; q++) d[q] = __ldg(s + q);
  return c;
}

// 256 threads x 4 consecutive neurons.  One Philox call per thread gives the
// four neurons' drive words.  Spike bits: 4-bit nibbles OR-ed across groups
// of 8 lanes into 32-bit words (word w holds neurons 32w .. 32w+31).
template <int NCH>
__global__ void __launch_bounds__(kUpdateThreads) neuron_update_kernel(DevNet g, int32_t t_rel) {
  const int64_t t = *g.t_base + t_rel;
  const int64_t slot = t % g.D;
  const int64_t i0 = ((int64_t)blockIdx.x * kUpdateThreads + threadIdx.x) * 4;
  const int64_t np = g.npad;

  float4 V4 = *reinterpret_cast<const float4*>(g.V + i0);
  float4 J4[4];
#pragma unroll
  for (int q = 0; q < 4; q++) J4[q] = *reinterpret_cast<const float4*>(g.j + q * np + i0);
  uint32_t ref4 = *reinterpret_cast<const uint32_t*>(g.ref + i0);
  int32_t* acc = g.ring + slot * NCH * np + i0;
  int4 A4[NCH];
#pragma unroll
  for (int c = 0; c < NCH; c++) {
    A4[c] = *reinterpret_cast<const int4*>(acc + c * np);
    *reinterpret_cast<int4*>(acc + c * np) = make_int4(0, 0, 0, 0);
  }
  const uint4 r = philox4x32_10(make_uint4((uint32_t)(i0 >> 2), (uint32_t)t, (uint32_t)((uint64_t)t >> 32), kTagDrive),
                                g.key0, g.key1);

  int32_t v = g.blk_vox[blockIdx.x];
  while (v + 1 < g.nv && g.vstart[v + 1] <= i0) v++;
  int32_t v3 = v;
  while (v3 + 1 < g.nv && g.vstart[v3 + 1] <= i0 + 3) v3++;
  VoxConst c = load_vc(g.vc + v);

  float Vq[4] = {V4.x, V4.y, V4.z, V4.w};
  float Jq[4][4] = {{J4[0].x, J4[1].x, J4[2].x, J4[3].x},
                    {J4[0].y, J4[1].y, J4[2].y, J4[3].y},
                    {J4[0].z, J4[1].z, J4[2].z, J4[3].z},
                    {J4[0].w, J4[1].w, J4[2].w, J4[3].w}};
  const uint32_t uq[4] = {r.x, r.y, r.z, r.w};
  uint32_t nib = 0;
#pragma unroll
  for (int q = 0; q < 4; q++) {
    if (v != v3) {
      int32_t vq = v;
      while (vq + 1 < g.nv && g.vstart[vq + 1] <= i0 + q) vq++;
      c = load_vc(g.vc + vq);
    }
    int32_t Aq[NCH];
#pragma unroll
    for (int cc = 0; cc < NCH; cc++) {
      const int4 a = A4[cc];
      Aq[cc] = q == 0 ? a.x : q == 1 ? a.y : q == 2 ? a.z : a.w;
    }
    uint32_t rq = (ref4 >> (8 * q)) & 0xFFu;
    const bool sp = update_neuron<NCH>(g, c, Vq[q], Jq[q], rq, Aq, uq[q]);
    ref4 = (ref4 & ~(0xFFu << (8 * q))) | (rq << (8 * q));
    if (sp && i0 + q < g.n) nib |= 1u << q;
  }
  *reinterpret_cast<float4*>(g.V + i0) = make_float4(Vq[0], Vq[1], Vq[2], Vq[3]);
#pragma unroll
  for (int q = 0; q < 4; q++)
    *reinterpret_cast<float4*>(g.j + q * np + i0) = make_float4(Jq[0][q], Jq[1][q], Jq[2][q], Jq[3][q]);
  *reinterpret_cast<uint32_t*>(g.ref + i0) = ref4;

  const int lane = threadIdx.x & 31;
  uint32_t word = nib << (4 * (lane & 7));
  word |= __shfl_xor_sync(0xFFFFFFFFu, word, 1);
  word |= __shfl_xor_sync(0xFFFFFFFFu, word, 2);
  word |= __shfl_xor_sync(0xFFFFFFFFu, word, 4);
  if ((lane & 7) == 0) g.flags[(i0 >> 5)] = word;  // i0 of lane 8q is the first neuron of word q
  int cnt = __popc(nib);
  cnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
  __shared__ int s_cnt[kUpdateThreads / 32];
  if (lane == 0) s_cnt[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int tot = 0;
#pragma unroll
    for (int w = 0; w < kUpdateThreads / 32; w++) tot += s_cnt[w];
    g.blk_cnt[blockIdx.x] = tot;
  }
}

// Compaction: CTA = tile of 64 neuron blocks (65,536 neurons).  The tile's
// base offset is the sum of all earlier blocks' counts (re-read from L2 by
// every CTA: no inter-CTA waiting), then a warp scan over the tile's blocks
// and a popc rank inside each 32-neuron word.
__global__ void __launch_bounds__(256) spike_compact_kernel(DevNet g) {
  const int tile = blockIdx.x;
  const int b0 = tile * kCompactBlocksPerTile;
  const int b1 = min(b0 + kCompactBlocksPerTile, g.nblk);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ int s_part[8];
  __shared__ int s_boff[kCompactBlocksPerTile + 1];

  int part = 0;
  for (int b = threadIdx.x; b < b0; b += 256) part += g.blk_cnt[b];
  part = __reduce_add_sync(0xFFFFFFFFu, part);
  if (lane == 0) s_part[warp] = part;
  if (warp == 0) {
    // exclusive scan of this tile's block counts, two per lane
    const int bi = b0 + 2 * lane;
    const int c0 = bi < b1 ? g.blk_cnt[bi] : 0;
    const int c1 = bi + 1 < b1 ? g.blk_cnt[bi + 1] : 0;
    int x = c0 + c1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    const int excl = x - c0 - c1;
    s_boff[2 * lane] = excl;
    s_boff[2 * lane + 1] = excl + c0;
    if (lane == 31) s_boff[kCompactBlocksPerTile] = x;
  }
  __syncthreads();
  int base = 0;
#pragma unroll
  for (int w = 0; w < 8; w++) base += s_part[w];

  const int64_t lp = *g.log_pos;
  for (int b = b0 + warp; b < b1; b += 8) {
    const uint32_t fw = g.flags[(int64_t)b * 32 + lane];
    const int c = __popc(fw);
    int x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    int pos = base + s_boff[b - b0] + x - c;
    uint32_t bits = fw;
    const int32_t id0 = (b * 32 + lane) * 32;
    while (bits) {
      const int bit = __ffs(bits) - 1;
      bits &= bits - 1;
      const int32_t id = id0 + bit;
      g.spk[pos] = id;
      if (lp + pos < g.log_cap) g.log_ids[lp + pos] = id;
      pos++;
    }
  }
  if (tile == gridDim.x - 1 && threadIdx.x == 0) {
    const int total = base + s_boff[kCompactBlocksPerTile];
    *g.n_spk = total;
    atomicAdd(g.spikes, (unsigned long long)total);
  }
}

template <int WFMT>
__device__ __forceinline__ int32_t stored_weight(const void* w, int64_t e, int shift) {
  if (WFMT == 0) return (int32_t)__ldg(reinterpret_cast<const int16_t*>(w) + e) * (1 << shift);
  if (WFMT == 1) return __ldg(reinterpret_cast<const int32_t*>(w) + e) * (1 << shift);
  if (WFMT == 2) {
    const uint32_t b = (uint32_t)__ldg(reinterpret_cast<const unsigned short*>(w) + e) << 16;
    return __float2int_rn(__fmul_rn(__uint_as_float(b), 65536.0f));
  }
  return (int32_t)__ldg(reinterpret_cast<const signed char*>(w) + e) * (1 << shift);
}

// Delivery: one warp per spike (grid-stride over the spike list), lanes
// stride over the row, four synapses in flight per lane.  The add is a
// fire-and-forget reduction at L2, so the order of adds does not matter.
template <int WFMT, int NCH>
__global__ void __launch_bounds__(256) spike_deliver_kernel(DevNet g, int32_t t_rel) {
  const int64_t t = *g.t_base + t_rel;
  const int32_t tm = (int32_t)(t % g.D);
  const int32_t n_spk = *g.n_spk;
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t np = g.npad;
  unsigned long long ev = 0;
  for (int64_t si = gw; si < n_spk; si += nw) {
    const int32_t s = g.spk[si];
    const int64_t r0 = g.row_ptr[s], r1 = g.row_ptr[s + 1];
    ev += (unsigned long long)(r1 - r0);
    const int32_t vs = voxel_of(g, s);
    const uint8_t* drow = g.delay + (int64_t)vs * g.nv;
    const int shift = WFMT == 3 ? g.wshift + (g.row_shift ? g.row_shift[s] : 0) : g.wshift;
    for (int64_t e0 = r0 + lane; e0 < r1; e0 += 4 * 32) {
      uint32_t wd[4];
      int32_t wa[4];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const int64_t e = e0 + u * 32;
        wd[u] = e < r1 ? __ldg(g.word + e) : 0xFFFFFFFFu;
        wa[u] = e < r1 ? stored_weight<WFMT>(g.w, e, shift) : 0;
      }
#pragma unroll
      for (int u = 0; u < 4; u++) {
        if (wd[u] == 0xFFFFFFFFu) continue;
        const int32_t tgt = (int32_t)(wd[u] & 0x3FFFFFFFu);
        const int32_t cls = (int32_t)(wd[u] >> 30);
        const int32_t vt = voxel_of(g, tgt);
        int32_t sl = tm + (int32_t)__ldg(drow + vt);
        if (sl >= g.D) sl -= g.D;
        atomicAdd(g.ring + ((int64_t)sl * NCH + cls) * np + tgt, wa[u]);
      }
    }
  }
  if (lane == 0 && ev) atomicAdd(g.events, ev);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    // spike-log bookkeeping of this step (compaction of the next step reads it)
    const int64_t lp = *g.log_pos;
    int64_t nxt = lp + n_spk;
    if (nxt > g.log_cap) {
      nxt = g.log_cap;
      *g.log_trunc = 1;
    }
    const int32_t cs = *g.call_steps;
    g.step_off[cs + 1] = nxt;
    *g.log_pos = nxt;
    *g.call_steps = cs + 1;
  }
}

__device__ __forceinline__ int lower_bound(const int32_t* a, int n, int32_t x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Balloon-Windkessel, one thread per voxel.  z = spikes / (n_v * dt) in Hz,
// counted by binary search of the voxel's id range in the ascending list.
__global__ void bold_step_kernel(DevNet g, int32_t t_rel) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= g.nv) return;
  const int64_t t = *g.t_base + t_rel;
  const int n_spk = *g.n_spk;
  const int cnt = lower_bound(g.spk, n_spk, g.vstart[v + 1]) - lower_bound(g.spk, n_spk, g.vstart[v]);
  const float z = (float)cnt * g.inv_nvox[v];
  const BoldConst& b = g.bc;
  const int nv = g.nv;
  float s = g.bold[v], f = g.bold[nv + v], vv = g.bold[2 * nv + v], q = g.bold[3 * nv + v];
  const float fout = powf(vv, b.inv_alpha);
  const float Ef = 1.0f - expf(b.ln_1mE0 / f);
  const float ds = b.eps * z - s * b.inv_tau_s - (f - 1.0f) * b.inv_tau_f;
  const float df = s;
  const float dv = (f - fout) * b.inv_tau_0;
  const float dq = (f * Ef * b.inv_E0 - fout * q / vv) * b.inv_tau_0;
  s += b.dt_s * ds;
  f += b.dt_s * df;
  vv += b.dt_s * dv;
  q += b.dt_s * dq;
  const float y = b.V0 * (b.k1 * (1.0f - q) + b.k2 * (1.0f - q / vv) + b.k3 * (1.0f - vv));
  g.bold[v] = s;
  g.bold[nv + v] = f;
  g.bold[2 * nv + v] = vv;
  g.bold[3 * nv + v] = q;
  g.bold[4 * nv + v] = y;
  if (g.bold_every > 0 && (t + 1) % g.bold_every == 0) {
    const int64_t idx = (t + 1) / g.bold_every - 1;
    g.bold_log[(idx % g.bold_cap) * nv + v] = y;
  }
}

__global__ void advance_kernel(int64_t* t_base, int32_t k) { *t_base += k; }

__global__ void begin_call_kernel(DevNet g) {
  *g.log_pos = 0;
  *g.call_steps = 0;
  *g.log_trunc = 0;
  g.step_off[0] = 0;
}

}  // namespace

cudaError_t launch_neuron_update(const DevNet& g, int32_t t_rel, cudaStream_t st) {
  const int blocks = (int)(g.npad / kNeuronsPerBlock);
  if (g.nch == 2) neuron_update_kernel<2><<<blocks, kUpdateThreads, 0, st>>>(g, t_rel);
  else neuron_update_kernel<4><<<blocks, kUpdateThreads, 0, st>>>(g, t_rel);
  return cudaGetLastError();
}

cudaError_t launch_spike_compact(const DevNet& g, cudaStream_t st) {
  spike_compact_kernel<<<g.ntiles, 256, 0, st>>>(g);
  return cudaGetLastError();
}

cudaError_t launch_spike_deliver(const DevNet& g, int32_t t_rel, int blocks, cudaStream_t st) {
#define DTB_DELIVER(W, C) spike_deliver_kernel<W, C><<<blocks, 256, 0, st>>>(g, t_rel)
  if (g.nch == 2) {
    switch (g.wfmt) {
      case 0: DTB_DELIVER(0, 2); break;
      case 1: DTB_DELIVER(1, 2); break;
      case 2: DTB_DELIVER(2, 2); break;
      default: DTB_DELIVER(3, 2); break;
    }
  } else {
    switch (g.wfmt) {
      case 0: DTB_DELIVER(0, 4); break;
      case 1: DTB_DELIVER(1, 4); break;
      case 2: DTB_DELIVER(2, 4); break;
      default: DTB_DELIVER(3, 4); break;
    }
  }
#undef DTB_DELIVER
  return cudaGetLastError();
}

cudaError_t launch_bold_step(const DevNet& g, int32_t t_rel, cudaStream_t st) {
  bold_step_kernel<<<(g.nv + 127) / 128, 128, 0, st>>>(g, t_rel);
  return cudaGetLastError();
}

cudaError_t launch_advance(const DevNet& g, int32_t k, cudaStream_t st) {
  advance_kernel<<<1, 1, 0, st>>>(g.t_base, k);
  return cudaGetLastError();
}

cudaError_t launch_begin_call(const DevNet& g, cudaStream_t st) {
  begin_call_kernel<<<1, 1, 0, st>>>(g);
  return cudaGetLastError();
}

int deliver_blocks_per_sm() {
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, spike_deliver_kernel<0, 2>, 256, 0);
  return n > 0 ? n : 1;
}

}  // namespace dtb
