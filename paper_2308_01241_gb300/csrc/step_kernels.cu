// step_kernels.cu -- the four kernels of one simulation step and their launchers.
//
//   neuron_update  Eq. 1 by explicit Euler (sections III.B, VI.A), Poisson drive,
//                  threshold / reset / refractory; spike bits by warp ballot
//   spike_compact  ascending spike ids from the bits: per-block counts,
//                  prefix sums, popc ranks ("collect spikes sequence", V.B)
//   spike_deliver  outgoing CSR rows of the spiking neurons -> int32 adds into
//                  the delay ring (J sums of section V.B)
//   bold_step      Balloon-Windkessel per voxel (section V.E, Friston 2000)
//
// Every floating-point operation of the neuron update is an explicit
// round-to-nearest intrinsic, in the order the header dtb.h states, so no
// multiply-add is ever fused and the result is bit-identical to the C oracle.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "dtb_device.cuh"
#include "dtb_launch.h"

namespace dtb {
namespace {

__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }

// One neuron, one step, in two parts that touch disjoint state:
//   j part: consume the arrivals A[] of a step and its Poisson word u,
//           j_u <- dJ_u j_u + a_u;
//   V part: V from V and j (the j of the start of the step), OU current,
//           refractory period and threshold; returns the spike.
// The plain step of the paper's order is V part then j part at the same t.
// Applying the j part of step t-1 right before the V part of step t gives
// the same numbers (each operation sees the same operands).
template <int NCH>
__device__ __forceinline__ void update_j(const DevNet& g, const VoxConst& c, float (&jj)[4], const int32_t (&A)[NCH],
                                         uint32_t u) {
  // k = #{m < M : u >= T_m}.  T is ascending, so past the first threshold u
  // is below, none of the later ones counts: four compares cover all but a
  // fraction P(K >= 4) (6e-5 at 2 kHz x 0.1 ms) of the draws
  int32_t k = 0;
#pragma unroll
  for (int m = 0; m < 4; m++)
    if (m < g.M) k += (u >= g.T[m]) ? 1 : 0;
  if (g.M > 4 && u >= g.T[3]) {
#pragma unroll
    for (int m = 4; m < kMaxPoisson; m++)
      if (m < g.M) k += (u >= g.T[m]) ? 1 : 0;
  }
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
#pragma unroll
  for (int q = 0; q < 4; q++) jj[q] = fadd(fmul(c.dJ[q], jj[q]), fmul(__int2float_rn(in[q]), SC));
}

template <bool OU>
__device__ __forceinline__ bool update_v(const DevNet& g, const VoxConst& c, float& V, const float (&jj)[4],
                                         uint32_t& ref, float& I, int64_t i, int64_t t) {
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
  if (OU) {
    // the current of this step into V, then its Euler-Maruyama step; the
    // normal is the centred sum of the four words of one Philox call
    Vn = fadd(Vn, fmul(c.kO, I));
    const uint4 r = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)t, (uint32_t)((uint64_t)t >> 32), kTagOU),
                                  g.key0, g.key1);
    const long long S = (long long)((unsigned long long)r.x + r.y + r.z + r.w) - (1LL << 33);
    const float xi = fmul(__ll2float_rn(S), g.ou_xi);
    I = fadd(fadd(fmul(g.ou_d, I), g.ou_c), fmul(g.ou_s, xi));
  }
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

// Persistent, TMA-fed neuron update.  A CTA of 256 threads owns the tiles
// blockIdx.x, blockIdx.x + gridDim.x, ... of 1024 neurons each.  One thread
// streams each tile's state rows (V, j[4], ref, the ring slot's NCH rows:
// 29 KB for two channels) into a ring of S shared-memory stages with 1D bulk
// copies, S tiles ahead of the compute; every thread then updates its four
// consecutive neurons from shared memory and writes V, j, ref, zeroed
// accumulators and spike bits straight to HBM with 128-bit stores.  One
// Philox call per thread gives the four neurons' drive words.  Spike bits:
// 4-bit nibbles OR-ed across groups of 8 lanes into 32-bit words (word w
// holds neurons 32w .. 32w+31); one spike count per tile.  With the OU drive
// the stage also carries the tile's OU currents (4 KB more).
//
// Bins mode (BINS): there is no dense accumulator.  A CTA owns the regions
// blockIdx.x, blockIdx.x + gridDim.x, ... of kRegionTiles consecutive tiles.
// At the start of a region its threads add the region's bin of arrival events
// into an int32 [NCH][kRegionNeurons] array in shared memory (exact integer
// sums, any order); each neuron then takes its arrivals from that array and
// clears them.  The bin (up to kEvBufWords words) is staged in shared memory
// by one bulk copy issued a region ahead, so adding it waits on no global
// load.  Three resident CTAs per SM (two stages each) let one CTA add its
// region's events while the others stream tiles.
template <int NCH, bool OU, bool BINS>
struct Stage {
  // bins mode stages V, ref (and I) and loads each thread's j straight into
  // registers, so that three CTAs fit on an SM
  static constexpr uint32_t kV = 0, kJ = 4096, kRef = BINS ? 4096 : kJ + 4 * 4096, kAcc = kRef + 1024;
  static constexpr uint32_t kI = kAcc + (BINS ? 0 : NCH * 4096);
  static constexpr uint32_t kVC = kI + (OU ? 4096 : 0);  // the tile's VoxConst (80 B)
  static constexpr uint32_t kNit = kVC + sizeof(VoxConst);  // work items per neuron (1 B each)
  static constexpr uint32_t kBytes = kNit + kNeuronsPerBlock;  // one tile
  // bins mode: the region's arrival sums and its staged bin sit in front of the stages
  static constexpr uint32_t kRegionAcc = BINS ? NCH * kRegionNeurons * 4 : 0;
  static constexpr uint32_t kFront = BINS ? kRegionAcc + kEvBufWords * 4 : 0;
  static constexpr uint32_t bytes(int S) { return kFront + S * kBytes; }
};
constexpr int kMaxRegionsPerCta = 128;  // bins mode: the launcher keeps grid * 128 >= regions

// upd: kUpdFull (V part then j part of step t), kUpdJV (j part of step t-1,
// then V part of step t), kUpdV (V part of step t only), kUpdJ (j part of
// step t only).  The j part consumes the arrivals of its step x: slot x mod D
// of the ring, slot x mod 2 of the event-queue mode's accumulator, or the
// bins of parity x mod 2 in bins mode.
template <int NCH, int S, bool OU, bool BINS>
__global__ void __launch_bounds__(kUpdateThreads, BINS ? 3 : 2)
    neuron_update_kernel(DevNet g, int32_t t_rel, int32_t upd) {
  using St = Stage<NCH, OU, BINS>;
  constexpr int kThr = kUpdateThreads;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* stages = smem + St::kFront;
  int32_t* racc = reinterpret_cast<int32_t*>(smem);  // bins mode: [NCH][kRegionNeurons]
  uint32_t* ebuf = reinterpret_cast<uint32_t*>(smem + St::kRegionAcc);  // bins mode: staged bin
  __shared__ uint64_t bar[S];    // stage k % S holds my k-th tile
  __shared__ uint64_t empty[S];  // every warp has taken what it needs from stage k % S
  __shared__ uint64_t ebar;                          // bins mode: the staged bin landed
  __shared__ uint32_t s_rcnt[BINS ? kMaxRegionsPerCta : 1];  // bins mode: events in my regions' bins
  __shared__ int s_cnt[2][kThr / 32];
  __shared__ int s_items[2][kThr / 32];
  const int64_t t = *g.t_base + t_rel;
  const bool do_v = upd != kUpdJ, do_j = upd != kUpdV, j_first = upd == kUpdJV;
  const int64_t x = j_first ? t - 1 : t;  // the step whose arrivals the j part consumes
  const int64_t np = g.npad;
  int32_t* acc_slot = BINS ? nullptr : g.ring + (g.mode ? (x & 1) : x % g.D) * NCH * np;
  const int ntile = g.nblk;
  // n_mine: my tiles
  int n_mine, r_mine = 0;
  if (BINS) {  // whole regions; only the network's last one may be short
    const int nreg = g.n_reg;
    r_mine = (int)blockIdx.x < nreg ? (nreg - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int r_last = (int)blockIdx.x + (r_mine - 1) * (int)gridDim.x;
    n_mine = r_mine ? (r_mine - 1) * kRegionTiles + min(kRegionTiles, ntile - r_last * kRegionTiles) : 0;
  } else {
    n_mine = (int)blockIdx.x < ntile ? (ntile - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  }
  // my k-th tile
  auto tile_of = [&](int k) {
    return BINS ? ((int)blockIdx.x + (k / kRegionTiles) * (int)gridDim.x) * kRegionTiles + k % kRegionTiles
                : (int)blockIdx.x + k * (int)gridDim.x;
  };
  const int tid = threadIdx.x, lane = tid & 31;
  const bool spilled = do_j && g.mode && g.spill_dirty[x % g.D];

  const uint64_t once = l2_evict_first();  // state is read and written once per step
  auto issue = [&](int k) {  // one thread: bulk loads of my k-th tile into stage k % S
    uint64_t* b = &bar[k % S];
    const int tl = tile_of(k);
    const int64_t base = (int64_t)tl * kNeuronsPerBlock;
    unsigned char* st = stages + (size_t)(k % S) * St::kBytes;
    mbar_expect_tx(b, St::kBytes);
    bulk_g2s_hint(st + St::kV, g.V + base, 4096, b, once);
    if (!BINS) {
#pragma unroll
      for (int q = 0; q < 4; q++) bulk_g2s_hint(st + St::kJ + q * 4096, g.j + q * np + base, 4096, b, once);
    }
    bulk_g2s_hint(st + St::kRef, g.ref + base, 1024, b, once);
    if (!BINS) {
#pragma unroll
      for (int c = 0; c < NCH; c++) bulk_g2s_hint(st + St::kAcc + c * 4096, acc_slot + c * np + base, 4096, b, once);
    }
    if (OU) bulk_g2s_hint(st + St::kI, g.Iou + base, 4096, b, once);
    bulk_g2s(st + St::kVC, g.tile_vc + tl, sizeof(VoxConst), b);
    bulk_g2s_hint(st + St::kNit, g.nitem + base, kNeuronsPerBlock, b, once);
  };
  // bins mode: the bin of my m-th region, parity of step x
  const int par = (int)(x & 1);
  const int ew = g.ev8 ? 2 : 1;
  auto bin_of = [&](int m) {
    return g.bins + ((int64_t)par * g.n_reg + (int)blockIdx.x + m * (int)gridDim.x) * g.bcap * ew;
  };
  auto issue_ev = [&](int m) {  // one thread: bulk copy of my m-th region's bin (up to kEvBufWords words)
    const uint32_t words = min(s_rcnt[m] * (uint32_t)ew, (uint32_t)kEvBufWords);
    const uint32_t bytes = (words * 4u + 15u) & ~15u;  // within the bin: its size is a multiple of 16 bytes
    mbar_expect_tx(&ebar, bytes);
    if (bytes) bulk_g2s_hint(ebuf, bin_of(m), bytes, &ebar, once);
  };

  // thread 0: the spike and work-item counts of my kk-th tile
  auto store_counts = [&](int kk) {
    int tot = 0, toti = 0;
#pragma unroll
    for (int w = 0; w < kThr / 32; w++) {
      tot += s_cnt[kk & 1][w];
      toti += s_items[kk & 1][w];
    }
    g.blk_cnt[tile_of(kk)] = tot;
    g.blk_items[tile_of(kk)] = toti;
  };

  if (tid == 0) {
#pragma unroll
    for (int q = 0; q < S; q++) {
      mbar_init(&bar[q], 1);
      mbar_init(&empty[q], kThr / 32);
    }
    if (BINS) mbar_init(&ebar, 1);
    fence_mbar_init();
  }
  if (BINS) {
    int4* z = reinterpret_cast<int4*>(racc);
    for (int q = tid; q < NCH * kRegionNeurons / 4; q += kThr) z[q] = make_int4(0, 0, 0, 0);
    if (do_j)
      for (int m = tid; m < r_mine; m += kThr)
        s_rcnt[m] = (uint32_t)min(g.bcnt[((int64_t)par * g.n_reg + (int)blockIdx.x + m * (int)gridDim.x) * kBcntStride],
                                  (unsigned long long)g.bcap);
  }
  __syncthreads();
  if (tid == 0) {
    if (BINS && do_j && r_mine > 0) issue_ev(0);
    for (int k = 0; k < S && k < n_mine; k++) issue(k);
  }

  int k = 0;
  int ev_pending = BINS && do_j && r_mine > 0 ? 0 : -1;  // tid 0: the region whose staged bin is in flight
  for (; k < n_mine; k++) {
    const int tile = tile_of(k);
    const int64_t i0 = (int64_t)tile * kNeuronsPerBlock + tid * 4;
    if (BINS && do_j && k % kRegionTiles == 0) {
      // the region's arrivals of step x into shared memory; racc is all zero
      // here (cleared at the start and by every tile's consumers)
      const int m = k / kRegionTiles;
      if (!__syncthreads_and(mbar_wait_bounded(&ebar, (uint32_t)m & 1u))) {
        if (tid == 0) atomicOr(g.err, 1);
        break;
      }
      ev_pending = -1;
      const int cnt = (int)s_rcnt[m];
      const int nbuf = min(cnt, kEvBufWords / ew);
      const uint32_t* evg = bin_of(m);
      const int32_t wfmt = g.wfmt, wsh = g.wshift;
      for (int e = tid; e < cnt; e += kThr) {
        uint32_t a, c;
        if (ew == 1) {
          a = e < nbuf ? ebuf[e] : __ldcs(evg + e);
          c = a >> 16;
        } else {
          const uint2 v = e < nbuf ? reinterpret_cast<const uint2*>(ebuf)[e]
                                   : __ldcs(reinterpret_cast<const uint2*>(evg) + e);
          a = v.x;
          c = v.y;
        }
        atomicAdd(racc + ((a >> kRegionShift) & 3u) * kRegionNeurons + (a & (kRegionNeurons - 1)),
                  decode_weight(c, wfmt, wsh));
      }
      __syncthreads();
      if (tid == 0) {
        // the bin is free for the step two later; the staging buffer for the next region
        g.bcnt[((int64_t)par * g.n_reg + (int)blockIdx.x + m * (int)gridDim.x) * kBcntStride] = 0;
        if (m + 1 < r_mine) {
          fence_proxy_async_smem();
          issue_ev(m + 1);
          ev_pending = m + 1;
        }
      }
    }
    // the drive words depend only on (i, x): drawn while the stage is in flight
    uint4 r = make_uint4(0u, 0u, 0u, 0u);
    if (do_j)
      r = philox4x32_10(make_uint4((uint32_t)(i0 >> 2), (uint32_t)x, (uint32_t)((uint64_t)x >> 32), kTagDrive),
                        g.key0, g.key1);
    float4 J4[4];
    if (BINS) {  // bins mode: my four neurons' j rows, loaded while the stage is in flight
#pragma unroll
      for (int q = 0; q < 4; q++) J4[q] = ld_hint(reinterpret_cast<const float4*>(g.j + q * np + i0), once);
    }
    const bool ok = __syncthreads_and(mbar_wait_bounded(&bar[k % S], (uint32_t)(k / S) & 1u));
    if (!ok) {
      if (tid == 0) atomicOr(g.err, 1);
      break;
    }
    if (tid == 0 && k > 0) store_counts(k - 1);  // every warp wrote them before this barrier
    const unsigned char* st = stages + (size_t)(k % S) * St::kBytes;
    // everything this tile takes from the stage, into registers; then the
    // stage is handed back and refilled while the neurons are updated
    const float4 V4 = reinterpret_cast<const float4*>(st + St::kV)[tid];
    if (!BINS) {
#pragma unroll
      for (int q = 0; q < 4; q++) J4[q] = reinterpret_cast<const float4*>(st + St::kJ + q * 4096)[tid];
    }
    uint32_t ref4 = reinterpret_cast<const uint32_t*>(st + St::kRef)[tid];
    int4 A4[NCH];
    if (!BINS) {
#pragma unroll
      for (int cc = 0; cc < NCH; cc++) A4[cc] = reinterpret_cast<const int4*>(st + St::kAcc + cc * 4096)[tid];
    }
    const float4 I4 = OU ? reinterpret_cast<const float4*>(st + St::kI)[tid] : make_float4(0.f, 0.f, 0.f, 0.f);
    const uint32_t ni4 = reinterpret_cast<const uint32_t*>(st + St::kNit)[tid];
    const VoxConst* tvc = reinterpret_cast<const VoxConst*>(st + St::kVC);
    const bool first_vox = tid * 4 + 3 < tvc->n_first;
    VoxConst c;
    if (first_vox) c = *tvc;
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[k % S]);
    if (tid == 0 && k + S < n_mine) {
      if (mbar_wait_bounded(&empty[k % S], (uint32_t)(k / S) & 1u)) {
        fence_proxy_async_smem();  // the stage's generic reads before the async refill
        issue(k + S);
      } else {
        atomicOr(g.err, 1);  // the refill is not issued: its wait gives up too
      }
    }
    uint32_t nib = 0;
    int nit = 0;  // delivery work items of my spiking neurons
    {
      if (BINS) {
        const int off = (k % kRegionTiles) * kNeuronsPerBlock + tid * 4;
#pragma unroll
        for (int cc = 0; cc < NCH; cc++) {
          int4* p = reinterpret_cast<int4*>(racc + cc * kRegionNeurons + off);
          A4[cc] = *p;
          if (do_j) *p = make_int4(0, 0, 0, 0);
        }
      }
      if (spilled) {  // event-queue and bins modes after a queue or bin overflowed: the spill slot adds in (rare)
        int32_t* sp = g.spill + (x % g.D) * NCH * np + i0;
#pragma unroll
        for (int cc = 0; cc < NCH; cc++) {
          const int4 y = *reinterpret_cast<const int4*>(sp + cc * np);
          *reinterpret_cast<int4*>(sp + cc * np) = make_int4(0, 0, 0, 0);
          A4[cc] = make_int4(A4[cc].x + y.x, A4[cc].y + y.y, A4[cc].z + y.z, A4[cc].w + y.w);
        }
      }
      // constants: the tile's copy when my four neurons lie in its first voxel
      // (no global load), else looked up per neuron
      int32_t v = 0, v3 = 0;
      if (!first_vox) {
        v = g.blk_vox[tile];
        while (v + 1 < g.nv && g.vstart[v + 1] <= i0) v++;
        v3 = v;
        while (v3 + 1 < g.nv && g.vstart[v3 + 1] <= i0 + 3) v3++;
        c = load_vc(g.vc + v);
      }

      float Vq[4] = {V4.x, V4.y, V4.z, V4.w};
      float Jq[4][4] = {{J4[0].x, J4[1].x, J4[2].x, J4[3].x},
                        {J4[0].y, J4[1].y, J4[2].y, J4[3].y},
                        {J4[0].z, J4[1].z, J4[2].z, J4[3].z},
                        {J4[0].w, J4[1].w, J4[2].w, J4[3].w}};
      const uint32_t uq[4] = {r.x, r.y, r.z, r.w};
      float Iq[4] = {I4.x, I4.y, I4.z, I4.w};
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
        if (j_first) update_j<NCH>(g, c, Jq[q], Aq, uq[q]);
        bool sp = false;
        if (do_v) sp = update_v<OU>(g, c, Vq[q], Jq[q], rq, Iq[q], i0 + q, t);
        if (do_j && !j_first) update_j<NCH>(g, c, Jq[q], Aq, uq[q]);
        ref4 = (ref4 & ~(0xFFu << (8 * q))) | (rq << (8 * q));
        if (sp && i0 + q < g.n) nib |= 1u << q;
      }
      if (do_v) {
        st_hint(reinterpret_cast<float4*>(g.V + i0), make_float4(Vq[0], Vq[1], Vq[2], Vq[3]), once);
        st_hint(reinterpret_cast<uint32_t*>(g.ref + i0), ref4, once);
        if (OU) st_hint(reinterpret_cast<float4*>(g.Iou + i0), make_float4(Iq[0], Iq[1], Iq[2], Iq[3]), once);
      }
      if (do_j) {
#pragma unroll
        for (int q = 0; q < 4; q++)
          st_hint(reinterpret_cast<float4*>(g.j + q * np + i0), make_float4(Jq[0][q], Jq[1][q], Jq[2][q], Jq[3][q]),
                  once);
        if (!BINS) {
#pragma unroll
          for (int cc = 0; cc < NCH; cc++) *reinterpret_cast<int4*>(acc_slot + cc * np + i0) = make_int4(0, 0, 0, 0);
        }
      }
      if (nib) {
#pragma unroll
        for (int q = 0; q < 4; q++)
          if ((nib >> q) & 1u) {
            if (g.nitem_ok) {
              nit += (int)((ni4 >> (8 * q)) & 0xFFu);
            } else {
              const int64_t len = g.row_ptr[i0 + q + 1] - g.row_ptr[i0 + q];
              nit += (int)((len + kItemEvents - 1) / kItemEvents);
            }
          }
      }
    }
    uint32_t word = nib << (4 * (lane & 7));
    word |= __shfl_xor_sync(0xFFFFFFFFu, word, 1);
    word |= __shfl_xor_sync(0xFFFFFFFFu, word, 2);
    word |= __shfl_xor_sync(0xFFFFFFFFu, word, 4);
    if ((lane & 7) == 0) g.flags[i0 >> 5] = word;  // i0 of lane 8q is the first neuron of word q
    const int cnt = __reduce_add_sync(0xFFFFFFFFu, __popc(nib));
    nit = __reduce_add_sync(0xFFFFFFFFu, nit);
    if (lane == 0) {  // summed by thread 0 after the next barrier
      s_cnt[k & 1][tid >> 5] = cnt;
      s_items[k & 1][tid >> 5] = nit;
    }
  }
  __syncthreads();
  if (tid == 0 && k == n_mine && n_mine > 0) store_counts(n_mine - 1);
  if (k < n_mine && tid == 0) {
    // gave up: let the copies still in flight land before the CTA exits
    for (int q = k; q < n_mine && q < k + S; q++) (void)mbar_wait_bounded(&bar[q % S], (uint32_t)(q / S) & 1u);
    if (ev_pending >= 0) (void)mbar_wait_bounded(&ebar, (uint32_t)ev_pending & 1u);
  }
}

// ==== end of the neuron update ====  A recorded DRAM traffic of the update
// kernel is keyed by a hash of this file up to this line and of dtb_device.cuh.
__device__ __forceinline__ int warp_incl_scan(int x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Work items of neuron id's row (ceil(len / kItemEvents)), from the per-neuron
// byte when every row fits in it, else from the row bounds.
__device__ __forceinline__ int items_of(const DevNet& g, int32_t id) {
  if (g.nitem_ok) return (int)__ldg(g.nitem + id);
  const int64_t len = __ldg(g.row_ptr + id + 1) - __ldg(g.row_ptr + id);
  return (int)((len + kItemEvents - 1) / kItemEvents);
}

// Block-wide exclusive scan of one value per thread (256 threads); returns the
// thread's exclusive prefix and sets *total.  Two barriers; s holds 8 ints.
__device__ __forceinline__ int block_excl_scan(int x, int* s, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int inc = warp_incl_scan(x, lane);
  if (lane == 31) s[warp] = inc;
  __syncthreads();
  int before = 0, all = 0;
#pragma unroll
  for (int k = 0; k < 8; k++) {
    const int v = s[k];
    if (k < warp) before += v;
    all += v;
  }
  __syncthreads();
  *total = all;
  return before + inc - x;
}

// Compaction: CTA = tile of 64 neuron blocks (65,536 neurons, 2,048 spike-bit
// words).  Thread i owns words 8i .. 8i+7, so thread order is neuron order and
// one block scan ranks the ids.  The tile's base offsets are sums of all
// earlier blocks' counts, re-read from L2 by every CTA: no inter-CTA waiting.
// Work items are then built in rounds of up to kRound spikes: the round's ids
// go to shared memory in rank order, one thread per spike looks up its item
// count, a block scan places the items, and one thread per item (its spike
// found by binary search over the scan) looks up its chunk's run table.  No
// thread walks a chain of lookups per spike or per item, so a tile with a
// crowded word or a row of many items costs a few memory latencies, not one
// per spike.
// spill_rel: the neuron update before this compaction consumed the arrivals
// of step t + spill_rel (0 or -1; 1: none), whose spill flag is cleared here.
__global__ void __launch_bounds__(256) spike_compact_kernel(DevNet g, int32_t t_rel, int32_t spill_rel) {
  constexpr int kWords = 8;    // spike-bit words per thread
  constexpr int kRound = 1024; // spikes per round of item building
  const int tile = blockIdx.x;
  const int b0 = tile * kCompactBlocksPerTile;
  const int words = min(kCompactBlocksPerTile, g.nblk - b0) * 32;  // a multiple of kWords
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool with_items = g.items != nullptr;
  __shared__ int s_part[8], s_ipart[8], s_scan[8];
  __shared__ int32_t s_id[kRound];
  __shared__ int s_it[kRound + 1];

  uint32_t w[kWords];
  const int w0 = tid * kWords;
  if (w0 < words) {
    const uint4* f = reinterpret_cast<const uint4*>(g.flags + (int64_t)b0 * 32 + w0);
    const uint4 x = f[0], y = f[1];
    w[0] = x.x; w[1] = x.y; w[2] = x.z; w[3] = x.w;
    w[4] = y.x; w[5] = y.y; w[6] = y.z; w[7] = y.w;
  } else {
#pragma unroll
    for (int k = 0; k < kWords; k++) w[k] = 0u;
  }

  // the counts of all earlier blocks (b0 is a multiple of 64): 16-byte loads,
  // several in flight per thread, so that the last tiles (tens of thousands
  // of earlier blocks) do not wait on a chain of L2 round trips
  int part = 0, ipart = 0;
  {
    const int4* c4 = reinterpret_cast<const int4*>(g.blk_cnt);
    const int4* i4 = reinterpret_cast<const int4*>(g.blk_items);
    const int n4 = b0 >> 2;
#pragma unroll 4
    for (int q = tid; q < n4; q += 256) {
      const int4 v = c4[q];
      part += (v.x + v.y) + (v.z + v.w);
      if (with_items) {
        const int4 u = i4[q];
        ipart += (u.x + u.y) + (u.z + u.w);
      }
    }
  }
  part = __reduce_add_sync(0xFFFFFFFFu, part);
  ipart = __reduce_add_sync(0xFFFFFFFFu, ipart);
  if (lane == 0) {
    s_part[warp] = part;
    s_ipart[warp] = ipart;
  }

  const int32_t id0 = (b0 * 32 + w0) * 32;  // first neuron of this thread's words
  int c = 0;
#pragma unroll
  for (int k = 0; k < kWords; k++) c += __popc(w[k]);
  int tot;
  const int r0 = block_excl_scan(c, s_scan, &tot);  // its barriers also publish s_part, s_ipart
  int base = 0, ibase = 0;
#pragma unroll
  for (int k = 0; k < 8; k++) {
    base += s_part[k];
    ibase += s_ipart[k];
  }

  if (c) {
    const int64_t lp = *g.log_pos;
    int pos = base + r0;
#pragma unroll
    for (int k = 0; k < kWords; k++)
      for (uint32_t bits = w[k]; bits; bits &= bits - 1) {
        const int32_t id = id0 + 32 * k + __ffs(bits) - 1;
        g.spk[pos] = id;
        if (lp + pos < g.log_cap) g.log_ids[lp + pos] = id;
        pos++;
      }
  }

  int itot = 0;
  if (with_items) {
    for (int lo = 0; lo < tot; lo += kRound) {
      const int nr = min(kRound, tot - lo);
      // this round's ids in rank order
      if (c && r0 < lo + kRound && r0 + c > lo) {
        int r = r0;
#pragma unroll
        for (int k = 0; k < kWords; k++)
          for (uint32_t bits = w[k]; bits; bits &= bits - 1, r++)
            if (r >= lo && r < lo + kRound) s_id[r - lo] = id0 + 32 * k + __ffs(bits) - 1;
      }
      __syncthreads();
      // item counts, four spikes per thread (consecutive, for the scan), loads in flight together
      int cnt[4], sum = 0;
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const int j = 4 * tid + q;
        cnt[q] = j < nr ? items_of(g, s_id[j]) : 0;
      }
#pragma unroll
      for (int q = 0; q < 4; q++) sum += cnt[q];
      int rtot;
      int e = block_excl_scan(sum, s_scan, &rtot);
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const int j = 4 * tid + q;
        if (j < nr) s_it[j] = e;
        e += cnt[q];
      }
      if (tid == 0) s_it[nr] = rtot;
      __syncthreads();
      // one thread per item of the round
      for (int j = tid; j < rtot; j += 256) {
        int lo_k = 0, hi_k = nr - 1;  // the last spike whose first item is <= j
        while (lo_k < hi_k) {
          const int mid = (lo_k + hi_k + 1) >> 1;
          if (s_it[mid] <= j) lo_k = mid;
          else hi_k = mid - 1;
        }
        const int32_t id = s_id[lo_k];
        const int64_t q = j - s_it[lo_k];
        const int64_t rb = __ldg(g.row_ptr + id), len = __ldg(g.row_ptr + id + 1) - rb;
        const int64_t cb = g.run_ptr ? __ldg(g.chunk_base + id) : 0;
        WorkItem it;
        it.e0 = rb + q * kItemEvents;
        it.len = (int32_t)min(len - q * kItemEvents, (int64_t)kItemEvents);
        it.src = id;
        it.rp0 = 0;
        it.nr = 0;
        it.pad = 0;
        if (g.run_ptr) {  // the chunk's run table, so that delivery needs no further lookup
          it.rp0 = __ldg(g.run_ptr + cb + q);
          it.nr = (int32_t)(__ldg(g.run_ptr + cb + q + 1) - it.rp0);
        }
        g.items[ibase + itot + j] = it;
      }
      itot += rtot;
      __syncthreads();  // s_id and s_it are rewritten by the next round
    }
  }
  if (tile == 0 && tid == 0 && g.mode && spill_rel <= 0) {
    const int64_t x = *g.t_base + t_rel + spill_rel;  // the neuron update consumed spill slot x mod D
    g.spill_dirty[x % g.D] = 0;
  }
  if (tile == gridDim.x - 1 && tid == 0) {
    const int total = base + tot;
    *g.n_spk = total;
    if (with_items) *g.n_items = ibase + itot;
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

// Delivery: one warp per work item (up to 512 synapses of one spiking row;
// grid-stride over the item list), lanes stride over the item, four synapses
// in flight per lane.  The add is a fire-and-forget reduction at L2, so the
// order of adds does not matter.
template <int WFMT, int NCH>
__global__ void __launch_bounds__(256) spike_deliver_kernel(DevNet g, int32_t t_rel) {
  const int64_t t = *g.t_base + t_rel;
  const int32_t tm = (int32_t)(t % g.D);
  const int32_t n_spk = *g.n_spk;
  const int32_t n_items = *g.n_items;
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t np = g.npad;
  unsigned long long ev = 0;
  __shared__ unsigned long long s_ev;  // one events atomic per block, not per warp
  if (threadIdx.x == 0) s_ev = 0;
  __syncthreads();
  for (int64_t ii = gw; ii < n_items; ii += nw) {
    const WorkItem item = g.items[ii];
    const int32_t s = item.src;
    const int64_t r0 = item.e0, r1 = r0 + item.len;
    ev += (unsigned long long)(r1 - r0);
    const int shift = WFMT == 3 ? g.wshift + (g.row_shift ? g.row_shift[s] : 0) : g.wshift;
    for (int64_t e0 = r0 + lane; e0 < r1; e0 += 4 * 32) {
      uint32_t wd[4];
      int32_t wa[4];
      int32_t dd[4];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const int64_t e = e0 + u * 32;
        wd[u] = e < r1 ? __ldg(g.word + e) : 0xFFFFFFFFu;
        wa[u] = e < r1 ? stored_weight<WFMT>(g.w, e, shift) : 0;
        dd[u] = e < r1 ? (int32_t)__ldg(g.syn_delay + e) : 0;
      }
#pragma unroll
      for (int u = 0; u < 4; u++) {
        if (wd[u] == 0xFFFFFFFFu) continue;
        const int32_t tgt = (int32_t)(wd[u] & 0x3FFFFFFFu);
        const int32_t cls = (int32_t)(wd[u] >> 30);
        int32_t sl = tm + dd[u];
        if (sl >= g.D) sl -= g.D;
        atomicAdd(g.ring + ((int64_t)sl * NCH + cls) * np + tgt, wa[u]);
      }
    }
  }
  if (lane == 0 && ev) atomicAdd(&s_ev, ev);
  __syncthreads();
  if (threadIdx.x == 0 && s_ev) atomicAdd(g.events, s_ev);
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

// Event-queue and bins delivery.  A CTA takes batches of kQBatch work items
// (one warp per item).  Each lane loads its up to 16 synapses of the item in
// one round (lane l holds synapses l, l + 32, ...), so one memory latency
// covers the item.  Every event then has a key: the arrival step's queue
// (delay d > 1), or in bins mode, for delay-1 events, the target region's bin
// of step t + 1 (their targets lie in the source's voxel: a window of kWin
// regions around the source region, per warp).  Delay-1 events of the
// event-queue mode are reduced straight into the accumulator of step t + 1.
//   pass 1: the 32 synapses a warp holds in one round form runs of equal keys
//           (consecutive lanes; packed rows are sorted by delay and target in
//           every chunk of an item, so runs are long); the run's first lane
//           adds the run's length to the key's batch count in shared memory
//           and learns the run's offset among the batch's events of that key;
//   then:   one global atomic per key of the batch reserves the key's range of
//           its queue or bin, and a block scan places the keys' events one
//           after the other in a shared-memory staging buffer;
//   pass 2: every event goes to its staging slot; then consecutive threads
//           write the staged events out, so that each key's run goes to its
//           queue or bin in coalesced stores.
// Events at or beyond a queue's or bin's capacity are added into the dense
// spill ring instead.  Delay-1 events outside a warp's window reserve one by
// one.  Three barriers per batch.
constexpr int kQBatch = 8;
constexpr int kWin = 64;

// Typed start of an item's stored weights (element e0 of the weight array).
template <int WFMT>
__device__ __forceinline__ const void* weight_row(const void* w, int64_t e0) {
  constexpr int kBytes = WFMT == 1 ? 4 : WFMT == 3 ? 1 : 2;
  return reinterpret_cast<const char*>(w) + e0 * kBytes;
}

// Exclusive scan of a[0 .. n) into out by the 256 threads of a CTA, each a
// contiguous chunk of at most 4 (n <= 1024); returns the total.  a is read
// before the scan's barrier only, so callers may change it afterwards.
__device__ __forceinline__ int deliver_block_scan(const int* a, int* out, int n, int* s_warp) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int per = (n + 255) / 256;
  const int r0 = tid * per;
  int v[4];
  int sum = 0;
#pragma unroll
  for (int q = 0; q < 4; q++) {
    v[q] = q < per && r0 + q < n ? a[r0 + q] : 0;
    sum += v[q];
  }
  int x = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  int before = 0, total = 0;
#pragma unroll
  for (int w = 0; w < 8; w++) {
    const int t = s_warp[w];
    before += w < warp ? t : 0;
    total += t;
  }
  int run = before + x - sum;
#pragma unroll
  for (int q = 0; q < 4; q++)
    if (q < per && r0 + q < n) {
      out[r0 + q] = run;
      run += v[q];
    }
  return total;
}

template <int WFMT, int NCH, bool BINS>
__global__ void __launch_bounds__(256, 3) spike_deliver_queue_kernel(DevNet g, int32_t t_rel) {
  constexpr int kPer = kItemEvents / 32;  // synapses of an item per lane
  constexpr int kDelayKeys = 256;         // keys 0 .. 255: the queue of arrival step t + key
  constexpr int kKeys = kDelayKeys + (BINS ? kQBatch * kWin : 0);  // then warp w's window region r: 256 + w * kWin + r
  constexpr int kStage = kQBatch * kItemEvents;
  extern __shared__ __align__(16) unsigned char dsm[];
  uint2* stage = reinterpret_cast<uint2*>(dsm);                           // [kStage] staged events
  unsigned short* skey = reinterpret_cast<unsigned short*>(stage + kStage);  // [kStage] their keys
  int* hist = reinterpret_cast<int*>(skey + kStage);                      // [kKeys] events per key in the batch
  int* sbase = hist + kKeys;                                              // [kKeys] staging offset of each key
  unsigned int* gbase = reinterpret_cast<unsigned int*>(sbase + kKeys);   // [kKeys] reserved start (clamped to capacity)
  __shared__ int s_warp[8];
  __shared__ int s_wlo[2][kQBatch];  // bins mode: first region of each warp's window, by batch parity
  __shared__ unsigned long long s_ev;  // one events atomic per block, not per warp
  const int64_t t = *g.t_base + t_rel;
  const int32_t tm = (int32_t)(t % g.D);
  const int32_t n_spk = *g.n_spk;
  const int32_t n_items = *g.n_items;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t np = g.npad;
  const long long qcap = g.qcap;
  int32_t* acc1 = BINS ? nullptr : g.ring + ((t + 1) & 1) * NCH * np;  // arrivals of step t + 1
  unsigned long long ev = 0;
  if (threadIdx.x == 0) s_ev = 0;
  for (int k = threadIdx.x; k < kKeys; k += blockDim.x) hist[k] = 0;
  const int par1 = (int)((t + 1) & 1);  // bins mode: parity of step t + 1
  unsigned long long* bc1 = BINS ? g.bcnt + (int64_t)par1 * g.n_reg * kBcntStride : nullptr;
  const int ew = BINS && g.ev8 ? 2 : 1;
  uint32_t* bins1 = BINS ? g.bins + (int64_t)par1 * g.n_reg * g.bcap * ew : nullptr;
  const uint64_t once = l2_evict_first();  // a row is read once per spike
  __syncthreads();
  const int nbatch = (n_items + kQBatch - 1) / kQBatch;
  int bp = 0;  // batch parity
  for (int b = blockIdx.x; b < nbatch; b += gridDim.x, bp ^= 1) {
    const int ii = b * kQBatch + warp;
    const bool has = ii < n_items;
    // the whole item in registers: lane holds synapses lane + 32 u
    uint32_t wd[kPer], cd[kPer];  // word; weight code | delay << 24 (delay 0: no synapse)
    uint32_t off2[kPer / 2];      // two 16-bit offsets per word: an event's place among its key's batch events
#pragma unroll
    for (int u = 0; u < kPer; u++) {
      wd[u] = 0u;
      cd[u] = 0u;
    }
    int len = 0, wlo = 0;
    if (has) {
      const WorkItem item = g.items[ii];
      len = item.len;
      if (BINS) wlo = max((item.src >> kRegionShift) - kWin / 2, 0);
      if (lane == 0) ev += (unsigned long long)len;
      // word, delay and weight rows (networks with packed records and run tables,
      // those with a 16-bit weight code, use the run-table kernel instead)
      const uint32_t* wrow = g.word + item.e0;
      const uint8_t* drow = g.syn_delay + item.e0;
      const void* wtrow = weight_row<WFMT>(g.w, item.e0);
      const int shift = WFMT == 3 ? g.wshift + (g.row_shift ? g.row_shift[item.src] : 0) : g.wshift;
#pragma unroll
      for (int u = 0; u < kPer; u++) {
        const int j = lane + 32 * u;
        const bool in = j < len;
        wd[u] = in ? ldg_hint(wrow + j, once) : 0u;
        const uint32_t d = in ? (uint32_t)__ldg(drow + j) : 0u;
        // int32 weights do not fit beside the delay: they are re-read where they are needed
        cd[u] = d << 24;
        if (in && WFMT != 1) cd[u] |= weight_code<WFMT>(wtrow, j, shift);
      }
    }
    if (BINS && lane == 0) s_wlo[bp][warp] = wlo;
    // pass 1: runs of equal keys -> one shared atomic per run
#pragma unroll
    for (int u = 0; u < kPer; u++) {
      const uint32_t d = cd[u] >> 24;
      const int32_t tgt = (int32_t)(wd[u] & 0x3FFFFFFFu);
      int key = -1;
      if (d > 1) {
        key = (int)d;
      } else if (d == 1) {
        if (BINS) {
          const int w = (tgt >> kRegionShift) - wlo;
          if (w >= 0 && w < kWin) {
            key = kDelayKeys + warp * kWin + w;
          } else {  // outside the window: reserve alone (rare)
            const int r = tgt >> kRegionShift;
            const int64_t pos = (int64_t)min(atomicAdd(bc1 + (int64_t)r * kBcntStride, 1ull), (unsigned long long)g.bcap);
            const uint32_t loc = (uint32_t)(tgt & (kRegionNeurons - 1)) | ((wd[u] >> 30) << kRegionShift);
            const uint32_t code = WFMT == 1 ? (uint32_t)weight_code<1>(g.w, g.items[ii].e0 + lane + 32 * u, 0)
                                            : (cd[u] & 0xFFFFu);
            if (pos < g.bcap) {
              if (ew == 2) reinterpret_cast<uint2*>(bins1)[(int64_t)r * g.bcap + pos] = make_uint2(loc, code);
              else bins1[(int64_t)r * g.bcap + pos] = loc | (code << 16);
            } else {
              int32_t sl = tm + 1;
              if (sl >= g.D) sl -= g.D;
              atomicAdd(g.spill + ((int64_t)sl * NCH + (wd[u] >> 30)) * np + tgt, decode_weight(code, WFMT, g.wshift));
              g.spill_dirty[sl] = 1;
            }
          }
        } else {  // event-queue mode: straight into the accumulator of step t + 1
          const int32_t wa = WFMT == 1 ? stored_weight<1>(g.w, g.items[ii].e0 + lane + 32 * u, g.wshift)
                                       : decode_weight(cd[u] & 0xFFFFu, WFMT, g.wshift);
          atomicAdd(acc1 + (int64_t)(wd[u] >> 30) * np + tgt, wa);
        }
      }
      const int left = __shfl_up_sync(0xFFFFFFFFu, key, 1);
      const bool head = key >= 0 && (lane == 0 || left != key);
      const unsigned heads = __ballot_sync(0xFFFFFFFFu, head);
      const unsigned ends = heads | __ballot_sync(0xFFFFFFFFu, key < 0);
      int run_off = 0;
      if (head) {
        const unsigned above = lane == 31 ? 0u : (ends >> (lane + 1)) << (lane + 1);
        const int nb = above ? __ffs(above) - 1 : 32;
        run_off = atomicAdd(&hist[key], nb - lane);
      }
      const int my_head = 31 - __clz(heads & (0xFFFFFFFFu >> (31 - lane)));
      const int o = __shfl_sync(0xFFFFFFFFu, run_off, my_head & 31) + (lane - my_head);
      const uint32_t o16 = key >= 0 ? (uint32_t)o : 0u;
      if (u & 1) off2[u >> 1] |= o16 << 16;
      else off2[u >> 1] = o16;
    }
    __syncthreads();
    // reservations of the batch's keys and their places in the staging buffer
    const int total = deliver_block_scan(hist, sbase, kKeys, s_warp);
    for (int k = threadIdx.x; k < kKeys; k += blockDim.x) {
      const int h = hist[k];
      if (h > 0) {
        if (k < kDelayKeys) {
          int32_t sl = tm + k;
          if (sl >= g.D) sl -= g.D;
          const unsigned long long p = atomicAdd(g.qcnt + sl * kQcntStride, (unsigned long long)h);
          if (p + (unsigned long long)h > (unsigned long long)qcap) g.spill_dirty[sl] = 1;  // the tail spills
          gbase[k] = (unsigned int)min(p, (unsigned long long)qcap);
        } else if (BINS) {
          const int w = k - kDelayKeys;
          const int r = s_wlo[bp][w / kWin] + w % kWin;
          gbase[k] = (unsigned int)min(atomicAdd(bc1 + (int64_t)r * kBcntStride, (unsigned long long)h),
                                       (unsigned long long)g.bcap);
        }
        hist[k] = 0;  // for the next batch (every warp is past its pass 1)
      }
    }
    __syncthreads();
    // pass 2a: every keyed event into its staging slot
    if (has) {
#pragma unroll
      for (int u = 0; u < kPer; u++) {
        const uint32_t d = cd[u] >> 24;
        if (d == 0 || (!BINS && d == 1)) continue;
        const int32_t tgt = (int32_t)(wd[u] & 0x3FFFFFFFu);
        int key;
        if (d > 1) {
          key = (int)d;
        } else {
          const int w = (tgt >> kRegionShift) - wlo;
          if (w < 0 || w >= kWin) continue;
          key = kDelayKeys + warp * kWin + w;
        }
        const int at = sbase[key] + (int)((off2[u >> 1] >> (16 * (u & 1))) & 0xFFFFu);
        // bins mode queues and bins carry the weight code, the event-queue mode
        // its accumulator value
        uint32_t v = cd[u] & 0xFFFFu;
        if (WFMT == 1) {
          const int64_t e = g.items[ii].e0 + lane + 32 * u;
          v = BINS ? weight_code<1>(g.w, e, 0) : (uint32_t)stored_weight<1>(g.w, e, g.wshift);
        } else if (!BINS) {
          v = (uint32_t)decode_weight(v, WFMT, g.wshift);
        }
        if (BINS && d == 1) {
          const uint32_t loc = (uint32_t)(tgt & (kRegionNeurons - 1)) | ((wd[u] >> 30) << kRegionShift);
          stage[at] = make_uint2(loc, v);
        } else {
          stage[at] = make_uint2(wd[u], v);
        }
        skey[at] = (unsigned short)key;
      }
    }
    __syncthreads();
    // pass 2b: consecutive threads write each key's run out
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
      const int key = skey[i];
      const uint2 e = stage[i];
      const int64_t pos = (int64_t)gbase[key] + (i - sbase[key]);
      if (key < kDelayKeys) {
        int32_t sl = tm + key;
        if (sl >= g.D) sl -= g.D;
        if (pos < qcap) {
          g.q[(int64_t)sl * qcap + pos] = e;
        } else {
          atomicAdd(g.spill + ((int64_t)sl * NCH + (e.x >> 30)) * np + (e.x & 0x3FFFFFFFu),
                    BINS ? decode_weight(e.y, WFMT, g.wshift) : (int32_t)e.y);
        }
      } else if (BINS) {
        const int w = key - kDelayKeys;
        const int r = s_wlo[bp][w / kWin] + w % kWin;
        if (pos < g.bcap) {
          if (ew == 2) reinterpret_cast<uint2*>(bins1)[(int64_t)r * g.bcap + pos] = e;
          else bins1[(int64_t)r * g.bcap + pos] = e.x | (e.y << 16);
        } else {
          int32_t sl = tm + 1;
          if (sl >= g.D) sl -= g.D;
          const int64_t tg = (int64_t)r * kRegionNeurons + (e.x & (kRegionNeurons - 1));
          atomicAdd(g.spill + ((int64_t)sl * NCH + ((e.x >> kRegionShift) & 3u)) * np + tg,
                    decode_weight(e.y, WFMT, g.wshift));
          g.spill_dirty[sl] = 1;
        }
      }
    }
  }
  if (lane == 0 && ev) atomicAdd(&s_ev, ev);
  __syncthreads();
  if (threadIdx.x == 0 && s_ev) atomicAdd(g.events, s_ev);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
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

// Delivery over the run tables (queue and bins modes with packed records,
// whose chunks are sorted by delay and target).  A CTA takes batches of
// kQBatch work items, one warp per item (one chunk), in a two-stage pipeline:
// while the events of batch b go out, batch b + 1 is counted and reserved.
//   pass 1: the warp's lanes take the chunk's runs (a few dozen); each run
//           adds its length to its key's batch count in shared memory, which
//           returns the run's offset among the batch's events of that key
//           (keys: the queue of arrival step t + d, or in bins mode the bin of
//           a target region of step t + 1 inside the warp's window of kWin
//           regions; a delay-1 run outside the window reserves its own range
//           and is written right away; in the event-queue mode delay-1 events
//           are reduced into the accumulator of step t + 1).  The first run of
//           a key puts the key on the batch's list of active keys;
//   reservation: one thread per active key reserves the key's range with one
//           global atomic;
//   pass 2: every event's record names its run; its position is the key's
//           reserved start + the run's offset + its place in the run.
//           Consecutive events of a run go to consecutive positions.
// Iteration b: load batch b's records; pass 1 of batch b + 1; load the first
// run entries of batch b + 2; barrier; issue the reservations of batch b + 1;
// pass 2 of batch b; store the reserved positions of batch b + 1; barrier.
// So a batch's record and run loads and its reservation round trip overlap
// the other batch's work instead of adding up.  Every per-key and per-run
// array is double-buffered by batch parity; the work items (two ahead) rotate
// through three shared slots.
template <bool BINS>
struct RunsSmem {
  static constexpr int kKeys = 256 + (BINS ? kQBatch * kWin : 0);
  static constexpr size_t kHist = 0;                                           // int [2][kKeys]
  static constexpr size_t kPtr = kHist + 2 * kKeys * 4;                        // u64 [2][kKeys]
  static constexpr size_t kRoom = kPtr + 2 * kKeys * 8;                        // u32 [2][kKeys]
  static constexpr size_t kRinfo = kRoom + 2 * kKeys * 4;                      // u32 [2][kQBatch][kItemEvents]
  static constexpr size_t kActive = kRinfo + 2 * kQBatch * kItemEvents * 4;    // u16 [2][kKeys]
  static constexpr size_t kBytes = kActive + 2 * kKeys * 2;
};

// Rare paths of the run-table delivery, kept out of line so that the unrolled
// per-event code stays small.  An event beyond its queue's or bin's capacity
// goes into the dense spill slot sl of its arrival step (exact int32 add).
template <int WFMT, int NCH>
__device__ __noinline__ void spill_event(const DevNet& g, int32_t sl, uint32_t word, uint32_t code, bool mark) {
  atomicAdd(g.spill + ((int64_t)sl * NCH + (word >> 30)) * g.npad + (word & 0x3FFFFFFFu), decode_weight(code, WFMT, g.wshift));
  if (mark) g.spill_dirty[sl] = 1;
}

// A delay-1 run whose target region lies outside the warp's window: its own
// range of the region's bin of step t + 1, written right away.
template <int WFMT, int NCH>
__device__ __forceinline__ void direct_run(const DevNet& g, const uint2* prow, int start, int len, int region,
                                        unsigned long long* bc1, uint32_t* bins1, int32_t s1) {
  const int64_t p0 = (int64_t)atomicAdd(bc1 + (int64_t)region * kBcntStride, (unsigned long long)len);
  for (int q = 0; q < len; q++) {
    const uint2 e = prow[start + q];
    const uint32_t tgt = e.x & 0x3FFFFFFFu, code = e.y & 0xFFFFu;
    const uint32_t loc = (tgt & (kRegionNeurons - 1)) | ((e.x >> 30) << kRegionShift);
    if (p0 + q < g.bcap) bins1[(int64_t)region * g.bcap + p0 + q] = loc | (code << 16);
    else spill_event<WFMT, NCH>(g, s1, e.x, code, true);
  }
}

template <int WFMT, int NCH, bool BINS>
__global__ void __launch_bounds__(256, 3) spike_deliver_runs_kernel(DevNet g, int32_t t_rel) {
  using L = RunsSmem<BINS>;
  constexpr int kPer = kItemEvents / 32;
  constexpr int kDelayKeys = 256;
  constexpr int kKeys = L::kKeys;
  constexpr uint32_t kReduce = 1022u, kDirect = 1023u;  // delay-1 runs reduced / written in pass 1
  extern __shared__ __align__(16) unsigned char dsm[];
  int* hist = reinterpret_cast<int*>(dsm + L::kHist);
  unsigned long long* kptr = reinterpret_cast<unsigned long long*>(dsm + L::kPtr);  // key's reserved start (address)
  unsigned int* kroom = reinterpret_cast<unsigned int*>(dsm + L::kRoom);  // positions left in its queue or bin
  uint32_t* rinfo = reinterpret_cast<uint32_t*>(dsm + L::kRinfo);  // per run: key | (offset - start + 512) << 10
  unsigned short* active = reinterpret_cast<unsigned short*>(dsm + L::kActive);
  __shared__ int n_active[2];
  __shared__ int s_wlo[2][kQBatch];
  __shared__ __align__(16) WorkItem s_item[3][kQBatch];
  __shared__ unsigned long long s_ev;
  const int64_t t = *g.t_base + t_rel;
  const int32_t tm = (int32_t)(t % g.D);
  const int32_t n_spk = *g.n_spk;
  const int32_t n_items = *g.n_items;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t np = g.npad;
  const long long qcap = g.qcap;
  int32_t* acc1 = BINS ? nullptr : g.ring + ((t + 1) & 1) * NCH * np;  // arrivals of step t + 1
  unsigned long long ev = 0;
  if (tid == 0) {
    s_ev = 0;
    n_active[0] = n_active[1] = 0;
  }
  for (int k = tid; k < 2 * kKeys; k += 256) hist[k] = 0;
  const int par1 = (int)((t + 1) & 1);  // bins mode: parity of step t + 1
  unsigned long long* bc1 = BINS ? g.bcnt + (int64_t)par1 * g.n_reg * kBcntStride : nullptr;
  uint32_t* bins1 = BINS ? g.bins + (int64_t)par1 * g.n_reg * g.bcap : nullptr;  // 4-byte events (16-bit codes)
  const uint64_t once = l2_evict_first();  // a row is read once per spike
  const int nbatch = (n_items + kQBatch - 1) / kQBatch;
  const int G = (int)gridDim.x;

  // the warp's work item of batch b, one 4-byte word per lane (len 0: none)
  auto item_word = [&](int b) -> int32_t {
    const int i = b * kQBatch + warp;
    return (lane < 8 && b < nbatch && i < n_items) ? reinterpret_cast<const int32_t*>(g.items + i)[lane] : 0;
  };
  auto put_item = [&](int slot, int32_t w) {
    if (lane < 8) reinterpret_cast<int32_t*>(&s_item[slot][warp])[lane] = w;
    __syncwarp();
  };

  // pass 1 of a batch of parity p whose item sits in slot sl
  constexpr int kRunsAhead = 2;  // run entries per lane loaded one iteration ahead of pass 1
  auto pass1 = [&](int sl, int p, const uint32_t (&rr)[kRunsAhead]) {
    const WorkItem& it = s_item[sl][warp];
    const int len = it.len;
    int wlo = 0;
    if (len > 0) {
      if (BINS) wlo = max((it.src >> kRegionShift) - kWin / 2, 0);
      const uint2* prow = g.syn_pack + it.e0;
      const int64_t rp0 = it.rp0;
      const int nr = it.nr;
      int* hp = hist + p * kKeys;
      uint32_t* ri = rinfo + (p * kQBatch + warp) * kItemEvents;
      unsigned short* act = active + p * kKeys;
      auto take_run = [&](int r, uint32_t run) {
        const uint32_t key = run_key(run);
        const int start = run_start(run), Ln = run_len(run);
        uint32_t ki;
        if (key & kRunRegion) {
          if (!BINS) {
            ki = kReduce;
          } else {
            const int region = (int)(key & (kRunRegion - 1u));
            const int w = region - wlo;
            if (w >= 0 && w < kWin) {
              ki = (uint32_t)(kDelayKeys + warp * kWin + w);
            } else {  // outside the window: its own range, written now (rare)
              ki = kDirect;
              direct_run<WFMT, NCH>(g, prow, start, Ln, region, bc1, bins1, tm + 1 >= g.D ? tm + 1 - g.D : tm + 1);
            }
          }
        } else {
          ki = key;  // the queue of arrival step t + key
        }
        int off = 0;
        if (ki < (uint32_t)kKeys) {
          off = atomicAdd(&hp[ki], Ln);
          if (off == 0) act[atomicAdd(&n_active[p], 1)] = (unsigned short)ki;  // the key's first run
        }
        ri[r] = ki | ((uint32_t)(off - start + 512) << 10);
      };
#pragma unroll
      for (int q = 0; q < kRunsAhead; q++)
        if (lane + 32 * q < nr) take_run(lane + 32 * q, rr[q]);
      for (int r = lane + 32 * kRunsAhead; r < nr; r += 32) take_run(r, __ldg(g.runs + rp0 + r));
    }
    if (BINS && lane == 0) s_wlo[p][warp] = wlo;
  };

  // the counter a key of a batch of parity p reserves on
  auto key_counter = [&](int k, int p) -> unsigned long long* {
    if (k < kDelayKeys) {
      int32_t sl = tm + k;
      if (sl >= g.D) sl -= g.D;
      return g.qcnt + sl * kQcntStride;
    }
    const int w = k - kDelayKeys;
    return bc1 + (int64_t)(s_wlo[p][w / kWin] + w % kWin) * kBcntStride;
  };
  // the reserved start of a key (h events from position got on) for pass 2
  auto store_key = [&](int k, int p, unsigned long long got, int h) {
    if (k < kDelayKeys) {
      int32_t sl = tm + k;
      if (sl >= g.D) sl -= g.D;
      if (got + (unsigned long long)h > (unsigned long long)qcap) g.spill_dirty[sl] = 1;  // the tail spills
      const unsigned long long p0 = min(got, (unsigned long long)qcap);
      kptr[p * kKeys + k] = reinterpret_cast<unsigned long long>(g.q + (int64_t)sl * qcap + (int64_t)p0);
      kroom[p * kKeys + k] = (unsigned int)((unsigned long long)qcap - p0);
    } else if (BINS) {
      const int w = k - kDelayKeys;
      const int r = s_wlo[p][w / kWin] + w % kWin;
      const unsigned long long p0 = min(got, (unsigned long long)g.bcap);
      kptr[p * kKeys + k] = reinterpret_cast<unsigned long long>(bins1 + (int64_t)r * g.bcap + (int64_t)p0);
      kroom[p * kKeys + k] = (unsigned int)((unsigned long long)g.bcap - p0);
    }
  };

  // pass 2 of a batch of parity p: every event to its place
  auto pass2 = [&](int len, const uint2 (&rec)[kPer], int p) {
    const uint32_t* ri = rinfo + (p * kQBatch + warp) * kItemEvents;
    const unsigned long long* kp = kptr + p * kKeys;
    const unsigned int* kr = kroom + p * kKeys;
#pragma unroll
    for (int u = 0; u < kPer; u++) {
      const int pos = lane + 32 * u;
      if (pos >= len) continue;
      const uint2 e = rec[u];
      const uint32_t info = ri[(e.y >> 16) & 511u];
      const uint32_t ki = info & 1023u;
      const uint32_t o = (info >> 10) + (uint32_t)pos - 512u;  // >= 0: a run's offset + the place in it
      if (ki >= (uint32_t)kKeys) {
        if (!BINS && ki == kReduce)
          atomicAdd(acc1 + (int64_t)(e.x >> 30) * np + (e.x & 0x3FFFFFFFu), decode_weight(e.y & 0xFFFFu, WFMT, g.wshift));
        continue;  // kDirect: written in pass 1
      }
      if (o < kr[ki]) {
        if (ki < (uint32_t)kDelayKeys) {
          const uint32_t v = BINS ? (e.y & 0xFFFFu) : (uint32_t)decode_weight(e.y & 0xFFFFu, WFMT, g.wshift);
          reinterpret_cast<uint2*>(kp[ki])[o] = make_uint2(e.x, v);
        } else {  // bins event: local target | class << 12 | code << 16
          reinterpret_cast<uint32_t*>(kp[ki])[o] =
              (e.x & (kRegionNeurons - 1)) | ((e.x >> (30 - kRegionShift)) & (3u << kRegionShift)) | (e.y << 16);
        }
      } else {  // beyond the capacity: the spill ring of the arrival step (rare)
        int32_t sl = tm + (ki < (uint32_t)kDelayKeys ? (int32_t)ki : 1);
        if (sl >= g.D) sl -= g.D;
        spill_event<WFMT, NCH>(g, sl, e.x, e.y & 0xFFFFu, ki >= (uint32_t)kDelayKeys);
      }
    }
  };

  // The first iteration has no current batch (slot 0 stays empty): it only
  // counts and reserves the CTA's first batch.
  put_item(0, 0);
  put_item(1, item_word((int)blockIdx.x));
  // the first runs of the next pass-1 batch, loaded an iteration ahead (its item
  // is the one two batches ahead, loaded at the start of the iteration before)
  uint32_t rn[kRunsAhead];
  auto load_runs = [&](int64_t rp0, int nr) {
#pragma unroll
    for (int q = 0; q < kRunsAhead; q++) rn[q] = lane + 32 * q < nr ? __ldg(g.runs + rp0 + lane + 32 * q) : 0u;
  };
  load_runs(s_item[1][warp].rp0, s_item[1][warp].len > 0 ? s_item[1][warp].nr : 0);
  __syncthreads();  // hist and n_active are clear
  int b = (int)blockIdx.x - G, bp = 1, sc = 0;  // batch, its parity, the slot of its item
  for (; b < nbatch; b += G, bp ^= 1, sc = sc == 2 ? 0 : sc + 1) {
    const int bn = b + G, p1 = bp ^ 1;
    const int sn = sc == 2 ? 0 : sc + 1, snn = sn == 2 ? 0 : sn + 1;
    // batch b's records, and the item two batches ahead
    const int len = s_item[sc][warp].len;
    uint2 rec[kPer];
    {
      const uint2* prow = g.syn_pack + s_item[sc][warp].e0;
#pragma unroll
      for (int u = 0; u < kPer; u++) {
        const int j = lane + 32 * u;
        rec[u] = j < len ? ldg_hint(prow + j, once) : make_uint2(0u, 0u);
      }
    }
    const int32_t wnn = item_word(bn + G);
    if (bn < nbatch) pass1(sn, p1, rn);
    {  // the runs of batch bn + G from its item's words (rp0: words 2-3, len: 4, nr: 6)
      const uint32_t lo = (uint32_t)__shfl_sync(0xFFFFFFFFu, wnn, 2), hi = (uint32_t)__shfl_sync(0xFFFFFFFFu, wnn, 3);
      const int lenn = __shfl_sync(0xFFFFFFFFu, wnn, 4), nrn = __shfl_sync(0xFFFFFFFFu, wnn, 6);
      load_runs((int64_t)(((uint64_t)hi << 32) | lo), lenn > 0 ? nrn : 0);
    }
    __syncthreads();
    // reservations of batch b + 1: a thread's first key stays in flight until
    // after pass 2 of batch b; further keys (more than 256) are stored now
    int rk = -1, rh = 0;
    unsigned long long rg = 0;
    if (bn < nbatch) {
      const int na = n_active[p1];
      if (tid < na) {
        rk = active[p1 * kKeys + tid];
        rh = hist[p1 * kKeys + rk];
        hist[p1 * kKeys + rk] = 0;
        rg = atomicAdd(key_counter(rk, p1), (unsigned long long)rh);
      }
      for (int a = tid + 256; a < na; a += 256) {
        const int k = active[p1 * kKeys + a];
        const int h = hist[p1 * kKeys + k];
        hist[p1 * kKeys + k] = 0;
        store_key(k, p1, atomicAdd(key_counter(k, p1), (unsigned long long)h), h);
      }
    }
    if (tid == 0) n_active[bp] = 0;  // batch b's list is done; pass 1 of batch b + 2 fills it
    if (len > 0) {
      if (lane == 0) ev += (unsigned long long)len;
      pass2(len, rec, bp);
    }
    if (rk >= 0) store_key(rk, p1, rg, rh);
    put_item(snn, wnn);
    __syncthreads();
  }
  if (lane == 0 && ev) atomicAdd(&s_ev, ev);
  __syncthreads();
  if (threadIdx.x == 0 && s_ev) atomicAdd(g.events, s_ev);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
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

// Dynamic shared memory of the queue and bins delivery.
template <bool BINS>
constexpr int deliver_smem_bytes() {
  return kQBatch * kItemEvents * (8 + 2) + (256 + (BINS ? kQBatch * kWin : 0)) * 12;
}

// Applies the queue of arrival step t + 1 to the one-slot accumulator:
// coalesced 16-byte reads of two events, one int32 reduction each.
__global__ void __launch_bounds__(256) drain_kernel(DevNet g, int32_t t_rel) {
  const int64_t t = *g.t_base + t_rel;
  const int32_t x = (int32_t)((t + 1) % g.D);
  const int64_t cnt = (int64_t)min(g.qcnt[x * kQcntStride], (unsigned long long)g.qcap);
  const uint2* q = g.q + (int64_t)x * g.qcap;
  const int64_t np = g.npad;
  int32_t* acc = g.ring + ((t + 1) & 1) * g.nch * np;  // the accumulator of step t + 1
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // eight events per thread and round: four 16-byte loads in flight, then the
  // reductions (an id word of all ones marks no event: ids stay below 2^30 - 1)
  for (int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 8; i0 < cnt; i0 += 8 * stride) {
    uint4 e[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const int64_t i = i0 + 2 * k;
      if (i + 1 < cnt) {
        e[k] = __ldcs(reinterpret_cast<const uint4*>(q + i));
      } else if (i < cnt) {
        const uint2 v = q[i];
        e[k] = make_uint4(v.x, v.y, 0xFFFFFFFFu, 0u);
      } else {
        e[k] = make_uint4(0xFFFFFFFFu, 0u, 0xFFFFFFFFu, 0u);
      }
    }
#pragma unroll
    for (int k = 0; k < 4; k++) {
      if (e[k].x != 0xFFFFFFFFu) atomicAdd(acc + (int64_t)(e[k].x >> 30) * np + (e[k].x & 0x3FFFFFFFu), (int32_t)e[k].y);
      if (e[k].z != 0xFFFFFFFFu) atomicAdd(acc + (int64_t)(e[k].z >> 30) * np + (e[k].z & 0x3FFFFFFFu), (int32_t)e[k].w);
    }
  }
  // the last block to finish empties the queue: every block read the count
  // before its thread 0 counted the block as done
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(g.drain_done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    g.qcnt[x * kQcntStride] = 0;
    *g.drain_done = 0;
  }
}

// Bins mode: sorts the queue of arrival step x = t + t_rel by target region
// into the bins of parity x mod 2, which the neuron update of step x then
// sums in shared memory.  A CTA takes tiles of kBinThreads * kPer events:
//   1. every event gets its rank among the tile's events of its region from a
//      shared-memory histogram;
//   2. one global atomic per region of the tile reserves a contiguous range of
//      that region's bin, and a block scan of the histogram gives each
//      region's offset in the tile;
//   3. the events are placed in shared memory in region order, then written
//      out by consecutive threads, so that a region's run of the tile goes to
//      its bin in coalesced stores (scattered stores of single events from
//      many warps into the same sectors were the kernel's bottleneck).
// A bin that is full sends the rest of its events into the dense spill slot
// of step x (exact int32 adds), as a full queue does.
constexpr int kBinThreads = 1024;

// Exclusive scan of a[0 .. n) into out (in place allowed, n <= 16 * kBinThreads),
// each thread a contiguous chunk; returns the total to every thread.
__device__ __forceinline__ uint32_t bin_block_scan(const uint32_t* a, uint32_t* out, int n, uint32_t* s_warp) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int per = (n + kBinThreads - 1) / kBinThreads;
  const int r0 = tid * per, r1 = min(r0 + per, n);
  uint32_t sum = 0;
  for (int r = r0; r < r1; r++) sum += a[r];
  uint32_t x = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < kBinThreads / 32 ? s_warp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, w, o);
      if (lane >= o) w += y;
    }
    s_warp[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  uint32_t run = (warp ? s_warp[warp - 1] : 0u) + x - sum;
  for (int r = r0; r < r1; r++) {
    const uint32_t v = a[r];
    out[r] = run;
    run += v;
  }
  return s_warp[kBinThreads / 32 - 1];
}

template <bool EV8>
__global__ void __launch_bounds__(kBinThreads, 1) bin_kernel(DevNet g, int32_t t_rel) {
  // events per thread and tile; a 16-bit code leaves room for the rank in
  // the upper half of the event's second word
  constexpr int kPer = EV8 ? 8 : 20;
  constexpr int kTile = kBinThreads * kPer;
  extern __shared__ __align__(16) uint32_t bsm[];
  const int nreg = g.n_reg;
  uint32_t* hist = bsm;                  // [n_reg] events of the tile per region
  uint32_t* base = bsm + nreg;           // [n_reg] start of the tile's range in each bin
  uint32_t* loff = bsm + 2 * nreg;       // [n_reg] start of each region's run in the sorted tile
  uint32_t* sev = bsm + ((3 * nreg + 3) & ~3);  // [kTile] the tile's events in region order (EV8: [kTile][2]), 16-byte aligned
  unsigned short* sreg = reinterpret_cast<unsigned short*>(sev + kTile * (EV8 ? 2 : 1));  // [kTile] their regions
  __shared__ uint32_t s_warp[32];
  const int64_t x = *g.t_base + t_rel;
  const int32_t slot = (int32_t)(x % g.D);
  const int par = (int)(x & 1);
  const int64_t cnt = (int64_t)min(g.qcnt[slot * kQcntStride], (unsigned long long)g.qcap);
  const uint2* q = g.q + (int64_t)slot * g.qcap;
  unsigned long long* bc = g.bcnt + (int64_t)par * nreg * kBcntStride;
  uint32_t* bins = g.bins + (int64_t)par * nreg * g.bcap * (EV8 ? 2 : 1);
  const int64_t bcap = g.bcap;
  const int tid = threadIdx.x;
  for (int r = tid; r < nreg; r += kBinThreads) hist[r] = 0u;
  __syncthreads();
  for (int64_t b0 = (int64_t)blockIdx.x * kTile; b0 < cnt; b0 += (int64_t)gridDim.x * kTile) {
    const int n_tile = (int)min((int64_t)kTile, cnt - b0);
    uint2 e[kPer];
    uint32_t rk[EV8 ? kPer : 1];
#pragma unroll
    for (int u = 0; u < kPer; u++) {
      const int64_t i = b0 + u * kBinThreads + tid;
      e[u] = i < cnt ? __ldcs(q + i) : make_uint2(0xFFFFFFFFu, 0u);  // all-ones id: no event
    }
#pragma unroll
    for (int u = 0; u < kPer; u++) {
      if (e[u].x == 0xFFFFFFFFu) continue;
      const uint32_t k = atomicAdd(&hist[(e[u].x & 0x3FFFFFFFu) >> kRegionShift], 1u);
      if (EV8) rk[u] = k;
      else e[u].y = (e[u].y & 0xFFFFu) | (k << 16);  // k < kTile < 2^16
    }
    __syncthreads();
    // reservations, and each region's offset in the tile; the histogram is
    // cleared for the next tile
    {  // all of this thread's reservations in flight at once (kMaxRegions / kBinThreads per thread at most)
      constexpr int kRegPer = kMaxRegions / kBinThreads;
      unsigned long long got[kRegPer];
#pragma unroll
      for (int q = 0; q < kRegPer; q++) {
        const int r = tid + q * kBinThreads;
        const uint32_t h = r < nreg ? hist[r] : 0u;
        got[q] = h ? atomicAdd(bc + (int64_t)r * kBcntStride, (unsigned long long)h) : 0ull;
      }
#pragma unroll
      for (int q = 0; q < kRegPer; q++) {
        const int r = tid + q * kBinThreads;
        if (r < nreg) base[r] = (uint32_t)min(got[q], (unsigned long long)bcap);
      }
    }
    (void)bin_block_scan(hist, loff, nreg, s_warp);
    __syncthreads();
    for (int r = tid; r < nreg; r += kBinThreads) hist[r] = 0u;
#pragma unroll
    for (int u = 0; u < kPer; u++) {
      if (e[u].x == 0xFFFFFFFFu) continue;
      const uint32_t tgt = e[u].x & 0x3FFFFFFFu, cls = e[u].x >> 30;
      const uint32_t r = tgt >> kRegionShift;
      const uint32_t loc = (tgt & (kRegionNeurons - 1)) | (cls << kRegionShift);
      const uint32_t at = loff[r] + (EV8 ? rk[u] : (e[u].y >> 16));
      if (EV8) reinterpret_cast<uint2*>(sev)[at] = make_uint2(loc, e[u].y);
      else sev[at] = loc | (e[u].y << 16);
      sreg[at] = (unsigned short)r;
    }
    __syncthreads();
    for (int i = tid; i < n_tile; i += kBinThreads) {
      const uint32_t r = sreg[i];
      const int64_t pos = (int64_t)base[r] + (i - (int)loff[r]);
      if (pos < bcap) {
        if (EV8) reinterpret_cast<uint2*>(bins)[(int64_t)r * bcap + pos] = reinterpret_cast<const uint2*>(sev)[i];
        else bins[(int64_t)r * bcap + pos] = sev[i];
      } else {
        const uint32_t loc = EV8 ? reinterpret_cast<const uint2*>(sev)[i].x : (sev[i] & 0xFFFFu);
        const uint32_t code = EV8 ? reinterpret_cast<const uint2*>(sev)[i].y : (sev[i] >> 16);
        const uint32_t cls = (loc >> kRegionShift) & 3u;
        const int64_t tgt = (int64_t)r * kRegionNeurons + (loc & (kRegionNeurons - 1));
        atomicAdd(g.spill + ((int64_t)slot * g.nch + cls) * g.npad + tgt, decode_weight(code, g.wfmt, g.wshift));
        g.spill_dirty[slot] = 1;
      }
    }
    __syncthreads();  // base, loff and the sorted tile are rewritten by the next tile
  }
  // the last block to finish empties the queue: every block read the count
  // before its thread 0 counted the block as done
  __shared__ bool last;
  if (tid == 0) {
    __threadfence();
    last = atomicAdd(g.drain_done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && tid == 0) {
    g.qcnt[slot * kQcntStride] = 0;
    *g.drain_done = 0;
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
  const int64_t t = *g.t_base + t_rel;
  if (v >= g.nv) return;
  const int n_spk = *g.n_spk;
  const int cnt = lower_bound(g.spk, n_spk, g.vstart[v + 1]) - lower_bound(g.spk, n_spk, g.vstart[v]);
  g.vox_spikes[v] += (unsigned long long)cnt;
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

// After a j-only update of step t: its arrivals' spill slot is consumed.
__global__ void spill_clear_kernel(DevNet g, int32_t t_rel) {
  if (g.mode) g.spill_dirty[(*g.t_base + t_rel) % g.D] = 0;
}

__global__ void begin_call_kernel(DevNet g) {
  *g.log_pos = 0;
  *g.call_steps = 0;
  *g.log_trunc = 0;
  g.step_off[0] = 0;
}

// Launch facts of one kernel instance on one device: its SM count, its
// resident CTAs per SM, and (once set) its dynamic shared-memory limit.  The
// function attribute and the occupancy are per device, so a process that
// drives several GPUs sets and queries them once on each.
constexpr int kMaxDevices = 64;
struct DeviceLaunch {
  int sms = 0, per_sm = 0;
};
template <typename Fn>
cudaError_t device_launch(DeviceLaunch (&cache)[kMaxDevices], std::mutex& mu, Fn&& setup, DeviceLaunch* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(mu);
  if (cache[dev].sms == 0) {
    DeviceLaunch d;
    e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = setup(d);
    if (e != cudaSuccess) return e;
    cache[dev] = d;
  }
  *out = cache[dev];
  return cudaSuccess;
}

template <int NCH, int S, bool OU, bool BINS>
cudaError_t launch_update(const DevNet& g, int32_t t_rel, cudaStream_t st, int blocks_per_sm, int32_t upd) {
  using St = Stage<NCH, OU, BINS>;
  static DeviceLaunch cache[kMaxDevices];  // per instance and device
  static std::mutex mu;
  const int smem = (int)St::bytes(S);
  DeviceLaunch dl;
  cudaError_t e0 = device_launch(cache, mu, [&](DeviceLaunch& d) {
    cudaError_t e = cudaFuncSetAttribute(neuron_update_kernel<NCH, S, OU, BINS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int per = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, neuron_update_kernel<NCH, S, OU, BINS>, kUpdateThreads,
                                                      smem);
    d.per_sm = per > 0 ? per : 1;
    return e;
  }, &dl);
  if (e0 != cudaSuccess) return e0;
  const int sms = dl.sms, max_per_sm = dl.per_sm;
  const int per = blocks_per_sm > 0 && blocks_per_sm < max_per_sm ? blocks_per_sm : max_per_sm;
  const int grid = sms * per;  // persistent grid: SMs x resident CTAs
  const int units = BINS ? g.n_reg : g.nblk;  // regions or tiles
  int blocks = grid < units ? grid : units;
  if (BINS && blocks * kMaxRegionsPerCta < units) blocks = (units + kMaxRegionsPerCta - 1) / kMaxRegionsPerCta;
  neuron_update_kernel<NCH, S, OU, BINS><<<blocks, kUpdateThreads, smem, st>>>(g, t_rel, upd);
  return cudaGetLastError();
}

// Stages: 2..4 with two channels, 2..3 with four.
template <bool OU, bool BINS>
cudaError_t launch_update_ou(const DevNet& g, int32_t t_rel, cudaStream_t st, int stages, int blocks_per_sm,
                             int32_t upd) {
  if (g.nch == 2) {
    if (stages == 2) return launch_update<2, 2, OU, BINS>(g, t_rel, st, blocks_per_sm, upd);
    if (stages == 4) return launch_update<2, 4, OU, BINS>(g, t_rel, st, blocks_per_sm, upd);
    return launch_update<2, 3, OU, BINS>(g, t_rel, st, blocks_per_sm, upd);
  }
  if (stages == 3) return launch_update<4, 3, OU, BINS>(g, t_rel, st, blocks_per_sm, upd);
  return launch_update<4, 2, OU, BINS>(g, t_rel, st, blocks_per_sm, upd);
}

// Queue and bins delivery: dynamic shared memory set once per device; the
// grid is at most the CTAs that fit at once (the kernel strides over batches).
template <int W, int C, bool BINS>
cudaError_t launch_deliver_queue(const DevNet& g, int32_t t_rel, int blocks, cudaStream_t st) {
  static DeviceLaunch cache[kMaxDevices];
  static std::mutex mu;
  constexpr int smem = deliver_smem_bytes<BINS>();
  DeviceLaunch dl;
  cudaError_t e = device_launch(cache, mu, [&](DeviceLaunch& d) {
    cudaError_t r = cudaFuncSetAttribute(spike_deliver_queue_kernel<W, C, BINS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (r != cudaSuccess) return r;
    int per = 0;
    r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, spike_deliver_queue_kernel<W, C, BINS>, 256, smem);
    d.per_sm = per > 0 ? per : 1;
    return r;
  }, &dl);
  if (e != cudaSuccess) return e;
  const int most = dl.sms * dl.per_sm;
  spike_deliver_queue_kernel<W, C, BINS><<<blocks < most ? blocks : most, 256, smem, st>>>(g, t_rel);
  return cudaGetLastError();
}

// Run-table delivery: the grid is at most the CTAs that fit at once.
template <int W, int C, bool BINS>
cudaError_t launch_deliver_runs(const DevNet& g, int32_t t_rel, int blocks, cudaStream_t st) {
  static DeviceLaunch cache[kMaxDevices];
  static std::mutex mu;
  DeviceLaunch dl;
  constexpr int smem = (int)RunsSmem<BINS>::kBytes;
  cudaError_t e = device_launch(cache, mu, [&](DeviceLaunch& d) {
    cudaError_t r = cudaFuncSetAttribute(spike_deliver_runs_kernel<W, C, BINS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (r != cudaSuccess) return r;
    int per = 0;
    r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, spike_deliver_runs_kernel<W, C, BINS>, 256, smem);
    d.per_sm = per > 0 ? per : 1;
    return r;
  }, &dl);
  if (e != cudaSuccess) return e;
  const int most = dl.sms * dl.per_sm;
  spike_deliver_runs_kernel<W, C, BINS><<<blocks < most ? blocks : most, 256, smem, st>>>(g, t_rel);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_neuron_update(const DevNet& g, int32_t t_rel, cudaStream_t st, int stages, int blocks_per_sm,
                                 int32_t upd) {
  if (g.mode == kModeBins)
    return g.ou ? launch_update_ou<true, true>(g, t_rel, st, stages, blocks_per_sm, upd)
                : launch_update_ou<false, true>(g, t_rel, st, stages, blocks_per_sm, upd);
  return g.ou ? launch_update_ou<true, false>(g, t_rel, st, stages, blocks_per_sm, upd)
              : launch_update_ou<false, false>(g, t_rel, st, stages, blocks_per_sm, upd);
}

cudaError_t launch_spike_compact(const DevNet& g, int32_t t_rel, cudaStream_t st, int32_t spill_rel) {
  spike_compact_kernel<<<g.ntiles, 256, 0, st>>>(g, t_rel, spill_rel);
  return cudaGetLastError();
}

cudaError_t launch_spill_clear(const DevNet& g, int32_t t_rel, cudaStream_t st) {
  spill_clear_kernel<<<1, 1, 0, st>>>(g, t_rel);
  return cudaGetLastError();
}

cudaError_t launch_spike_deliver(const DevNet& g, int32_t t_rel, int blocks, cudaStream_t st) {
#define DTB_DELIVER(W, C)                                                                         \
  do {                                                                                            \
    if (W != 1 && g.mode && g.runs) {                                                             \
      if (g.mode == kModeBins) return launch_deliver_runs<(W == 1 ? 0 : W), C, true>(g, t_rel, blocks, st); \
      return launch_deliver_runs<(W == 1 ? 0 : W), C, false>(g, t_rel, blocks, st);               \
    }                                                                                             \
    if (g.mode == kModeBins) return launch_deliver_queue<W, C, true>(g, t_rel, blocks, st);      \
    if (g.mode) return launch_deliver_queue<W, C, false>(g, t_rel, blocks, st);                  \
    spike_deliver_kernel<W, C><<<blocks, 256, 0, st>>>(g, t_rel);                                  \
  } while (0)
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

cudaError_t launch_drain(const DevNet& g, int32_t t_rel, int blocks, cudaStream_t st) {
  if (!g.mode) return cudaSuccess;
  drain_kernel<<<blocks, 256, 0, st>>>(g, t_rel);
  return cudaGetLastError();
}

cudaError_t launch_bin(const DevNet& g, int32_t t_rel, cudaStream_t st) {
  if (g.mode != kModeBins) return cudaSuccess;
  static DeviceLaunch cache[kMaxDevices];
  static std::mutex mu;
  // histogram, reservations and offsets per region; the sorted tile (16K
  // one-word or 8K two-word events) and its regions (2 bytes each)
  const int tile_bytes = 20 * kBinThreads * 4 + 20 * kBinThreads * 2;
  const int smem = 4 * ((3 * g.n_reg + 3) & ~3) + tile_bytes;
  DeviceLaunch dl;
  cudaError_t e0 = device_launch(cache, mu, [&](DeviceLaunch& d) {
    const int most = 12 * kMaxRegions + tile_bytes;
    cudaError_t e = cudaFuncSetAttribute(bin_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(bin_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    d.per_sm = 1;
    return e;
  }, &dl);
  if (e0 != cudaSuccess) return e0;
  const int blocks = dl.sms;  // one CTA of kBinThreads per SM
  if (g.ev8) bin_kernel<true><<<blocks, kBinThreads, smem, st>>>(g, t_rel);
  else bin_kernel<false><<<blocks, kBinThreads, smem, st>>>(g, t_rel);
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
