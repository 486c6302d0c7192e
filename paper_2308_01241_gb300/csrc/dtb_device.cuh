// dtb_device.cuh -- device-side layout of one network and the small helpers
// every kernel of the step shares.
//
// HBM layout (struct of arrays, every per-neuron array padded to npad, a
// multiple of 1024, so 128-bit accesses of four neighbours stay aligned):
//   V        float  [npad]             membrane potential
//   j        float  [4][npad]          gating variables AMPA, NMDA, GABAa, GABAb
//   ref      uint8  [npad]             refractory countdown
//   ring     int32  [D][nch][npad]     delayed input accumulators, 2^-16 units
//   flags    uint32 [npad/32]          spike bit per neuron of the current step
//   blk_cnt  int32  [npad/1024]        spikes per 1024-neuron block
//   spk      int32  [npad]             ascending spike ids of the current step
//   row_ptr  int64  [n+1], word uint32 [nnz], w [nnz]   outgoing CSR
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dtb {

constexpr int kNeuronsPerBlock = 1024;  // neuron update: 256 threads x 4 neurons
constexpr int kUpdateThreads = 256;
// neuron update launch modes (see neuron_update_kernel)
constexpr int32_t kUpdFull = 0, kUpdJV = 1, kUpdV = 2, kUpdJ = 3;
constexpr int kCompactBlocksPerTile = 64;  // neuron blocks per compaction CTA
constexpr int kMaxPoisson = 16;
// Delivery work item: up to kItemEvents consecutive synapses of one spiking
// row, so that long rows (heterogeneous out-degree) spread over many warps.
constexpr int kItemEvents = 512;
// Every batch of the delivery reserves queue space with one atomic per arrival
// step on these counters; 128 bytes apart, they spread over L2 slices instead
// of serialising on the three lines that 81 packed counters would share.
// Queue and bin counters are 64-bit, so a reservation can never wrap: a
// position at or beyond the capacity always sends its event to the spill ring.
constexpr int kQcntStride = 16;
// Delivery modes (DTB_DELIVER_* of dtb.h).
constexpr int32_t kModeRing = 0, kModeQueue = 1, kModeBins = 2;
// Bins mode: the neurons fall into regions of kRegionNeurons (kRegionTiles
// update tiles); the events of one arrival step are binned by target region,
// and the neuron update sums a region's bin in shared memory.
constexpr int kRegionShift = 12;
constexpr int kRegionNeurons = 1 << kRegionShift;
constexpr int kRegionTiles = kRegionNeurons / kNeuronsPerBlock;
constexpr int kMaxRegions = 8192;  // the binning kernel's shared-memory histograms (2^25 neurons)
// A bin's count at bcnt[(parity * n_reg + region) * kBcntStride]: one 32-byte
// sector per counter, so that the reservations spread over the L2 slices.
constexpr int kBcntStride = 4;
// Arrival events of one region that the neuron update stages in shared
// memory with one bulk copy (the rest, if any, it reads from the bin directly).
constexpr int kEvBufWords = 7168;
constexpr uint32_t kTagDrive = 1u;
constexpr uint32_t kTagInit = 2u;
constexpr uint32_t kTagOU = 3u;

// Up to kItemEvents consecutive synapses of one spiking neuron's row: the
// synapse index of the first, the first run record of its chunk and the
// chunk's run count (0 when the network keeps no run tables), how many
// synapses, and the source.
struct __align__(16) WorkItem {
  int64_t e0;
  int64_t rp0;
  int32_t len;
  int32_t src;
  int32_t nr;
  int32_t pad;
};

// Run tables of the packed synapse records (queue and bins modes with 16-bit
// weight codes).  Every chunk of kItemEvents synapses of a row is sorted at
// creation by delay, then target; a run is a maximal stretch of one chunk
// whose events wait in one place: the queue of one arrival step (delay d > 1,
// key d) or, for delay 1, the bin of one target region (key kRunRegion |
// region; in the event-queue mode every delay-1 event has key kRunRegion).
// A run record is key | start << 14 | (length - 1) << 23, and each packed
// record carries its run's index within the chunk in bits 16-24 of its
// second word (the weight code stays in bits 0-15).
constexpr uint32_t kRunRegion = 1u << 13;
__host__ __device__ __forceinline__ uint32_t run_key(uint32_t r) { return r & 0x3FFFu; }
__host__ __device__ __forceinline__ int run_start(uint32_t r) { return (int)((r >> 14) & 511u); }
__host__ __device__ __forceinline__ int run_len(uint32_t r) { return (int)(r >> 23) + 1; }

// Per-voxel constants of the Euler map, 80 bytes.
struct __align__(16) VoxConst {
  float kU[4];  // dt * g_u / C
  float dJ[4];  // 1 - dt / tau_u
  float E[4];   // reversal potentials
  float kL, EL, kI, Vth;
  float Vreset;
  int ref_steps;
  float kO;  // dt / C: the OU current's step into V
  int n_first;  // per-tile copy only: neurons of the tile (from its start) in this voxel
};

struct BoldConst {
  float eps, inv_tau_s, inv_tau_f, inv_tau_0, inv_alpha, ln_1mE0, inv_E0, V0, k1, k2, k3, dt_s;
};

struct DevNet {
  int64_t n, npad;
  int32_t nv, nch, D, M;
  int32_t nblk, ntiles;
  int32_t w_ext, wfmt, wshift, coarse_shift;
  uint32_t key0, key1;
  uint32_t T[kMaxPoisson];
  // state
  float* V;
  float* j;
  uint8_t* ref;
  int32_t* ring;
  // constants and lookup tables
  const VoxConst* vc;
  const int32_t* vstart;   // [nv+1]
  const uint16_t* coarse;  // voxel of neuron (c << coarse_shift)
  const uint16_t* blk_vox; // voxel of neuron (b * 1024)
  const VoxConst* tile_vc; // [nblk] constants of the voxel of neuron (b * 1024), n_first set
  const uint8_t* delay;    // [nv][nv]
  const float* inv_nvox;   // [nv] 1 / (n_v * dt_s)
  // synapses
  const int64_t* row_ptr;
  const uint32_t* word;
  const void* w;
  const uint8_t* row_shift;
  const uint8_t* syn_delay;  // [nnz] delay of each synapse, filled once from the voxel-pair table
  // queue and bins modes with 16-bit weight codes: each synapse packed into
  // one 8-byte record (word, weight code | run index << 16), each chunk of a
  // row sorted by delay and target, so that delivery reads a synapse with one
  // load; NULL otherwise (syn_delay is used then)
  const uint2* syn_pack;
  const int64_t* chunk_base;  // [n+1] first chunk of each row (with syn_pack)
  const int64_t* run_ptr;     // [chunks+1] first run of each chunk
  const uint32_t* runs;       // run records
  // per-step scratch
  uint32_t* flags;
  int32_t* blk_cnt;
  int32_t* spk;
  int32_t* n_spk;
  // delivery work items of the current step, ascending by source; blk_items
  // [nblk] per-block counts, n_items their total
  int32_t* blk_items;
  WorkItem* items;
  const uint8_t* nitem;  // [npad] work items of each neuron's row (0 beyond n); used when nitem_ok
  int32_t nitem_ok;      // 0 when some row needs more than 255 items (the update then reads row_ptr)
  int32_t* n_items;
  int64_t* t_base;
  // spike log of the current dtb_step call
  int32_t* log_ids;
  int64_t log_cap;
  int64_t* log_pos;
  int64_t* step_off;
  int32_t* call_steps;
  int32_t* log_trunc;
  // device error word: bit 0 = a bounded wait of the neuron update gave up,
  // bit 1 = an event queue overflowed
  int32_t* err;
  // delivery mode: 0 = dense ring (ring is [D][nch][npad]); 1 = event queues
  // (ring is the one-slot accumulator [nch][npad]; q [D][qcap] entries
  // (target | class << 30, w_acc) waiting for their arrival step, qcnt [D])
  int32_t mode;
  int64_t qcap;
  uint2* q;
  unsigned long long* qcnt;  // queue x's count at qcnt[x * kQcntStride]: one L2 line per counter
  uint32_t* drain_done;  // blocks of the current drain that finished (the last one resets the queue)
  // bins mode (mode 2): queued events carry the synapse's weight code (see
  // weight_code), not its accumulator value.  bins [2][n_reg][bcap] events of
  // one arrival step, by step parity and target region, 1 word each
  // (local target | class << 12 | code << 16) or, with int32 weights, 2 words
  // (local target | class << 12, code); bcnt [2][n_reg][kBcntStride] their counts
  uint32_t* bins;
  unsigned long long* bcnt;
  int64_t bcap;
  int32_t n_reg, ev8;
  // event-queue mode: events that find their queue full are added into this
  // dense ring [D][nch][npad] instead (exact int32 adds), and spill_dirty[x]
  // tells the neuron update of the step congruent to x to consume slot x too
  int32_t* spill;
  int32_t* spill_dirty;
  // counters
  unsigned long long* events;
  unsigned long long* spikes;
  // BOLD
  float* bold;  // [5][nv]: s, f, v, q, y
  unsigned long long* vox_spikes;  // [nv] spikes per voxel since creation / reset
  float* bold_log;
  int32_t bold_every, bold_cap;
  BoldConst bc;
  // Ornstein-Uhlenbeck background current (section III.B), when ou != 0:
  // I <- (ou_d I + ou_c) + ou_s xi, xi an Irwin-Hall(4) normal scaled by ou_xi
  int32_t ou;
  float ou_d, ou_c, ou_s, ou_xi;
  float* Iou;  // [npad]
};

// Philox4x32-10 (Salmon et al. 2011): ten rounds of two 32x32->64 products on
// counter words 0 and 2, high halves mixed into words 1 and 3 with the key,
// key bumped by the Weyl constants after every round.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; r++) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// ---- TMA bulk copies and mbarriers (PTX, sm_90+) ----
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// 1D bulk copy global -> shared, completion counted on bar (16-byte aligned, size % 16 == 0).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// L2 eviction policy for data touched once per step (state streams, synapse
// rows): first to be evicted, so that the accumulators and queues, which see
// scattered reductions and re-reads, keep more of the cache.
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                              uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}
__device__ __forceinline__ void st_hint(float4* p, float4 v, uint64_t policy) {
  asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z),
               "f"(v.w), "l"(policy)
               : "memory");
}
__device__ __forceinline__ void st_hint(uint32_t* p, uint32_t v, uint64_t policy) {
  asm volatile("st.global.L2::cache_hint.b32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(policy) : "memory");
}
__device__ __forceinline__ float4 ld_hint(const float4* p, uint64_t policy) {
  float4 v;
  asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p), "l"(policy));
  return v;
}
__device__ __forceinline__ uint2 ldg_hint(const uint2* p, uint64_t policy) {
  uint2 v;
  asm volatile("ld.global.nc.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;" : "=r"(v.x), "=r"(v.y) : "l"(p), "l"(policy));
  return v;
}
__device__ __forceinline__ uint32_t ldg_hint(const uint32_t* p, uint64_t policy) {
  uint32_t v;
  asm volatile("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(policy));
  return v;
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}
// Waits for phase `phase` of bar for at most max_cycles SM cycles (default
// 2^31, about a second); false when it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase, long long max_cycles = 1ll << 31) {
  if (mbar_try_wait(bar, phase)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, phase))
    if (clock64() - t0 > max_cycles) return false;
  return true;
}

// Bins mode: the stored weight of a synapse as a code that a queued event
// carries, and its accumulator value.  The code is the stored bits (int16,
// int32, bf16) or, for int8, the byte and its total shift (8 + 5 bits), so
// decode_weight(code) equals the weight the other modes add, bit for bit.
template <int WFMT>
__device__ __forceinline__ uint32_t weight_code(const void* w, int64_t e, int shift) {
  if (WFMT == 0) return (uint32_t)(unsigned short)__ldg(reinterpret_cast<const short*>(w) + e);
  if (WFMT == 1) return (uint32_t)__ldg(reinterpret_cast<const int32_t*>(w) + e);
  if (WFMT == 2) return (uint32_t)__ldg(reinterpret_cast<const unsigned short*>(w) + e);
  return (uint32_t)(unsigned char)__ldg(reinterpret_cast<const signed char*>(w) + e) | ((uint32_t)shift << 8);
}
__device__ __forceinline__ int32_t decode_weight(uint32_t code, int32_t wfmt, int32_t wshift) {
  if (wfmt == 0) return (int32_t)(short)(code & 0xFFFFu) * (1 << wshift);
  if (wfmt == 1) return (int32_t)code * (1 << wshift);
  if (wfmt == 2) return __float2int_rn(__fmul_rn(__uint_as_float(code << 16), 65536.0f));
  return (int32_t)(signed char)(code & 0xFFu) * (1 << (code >> 8));
}

// Voxel of neuron i: coarse table entry, then a forward scan of voxel starts.
__device__ __forceinline__ int32_t voxel_of(const DevNet& g, int32_t i) {
  int32_t v = __ldg(g.coarse + (i >> g.coarse_shift));
  while (v + 1 < g.nv && __ldg(g.vstart + v + 1) <= i) v++;
  return v;
}

}  // namespace dtb
