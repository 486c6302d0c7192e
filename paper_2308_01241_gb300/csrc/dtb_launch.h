// dtb_launch.h -- host launchers of the device kernels (internal to libdtb.so).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "dtb_device.cuh"

namespace dtb {

// stages: shared-memory pipeline depth (2..4; 2ch default 3, 4ch default 2);
// blocks_per_sm: resident CTAs per SM of the persistent grid (0 = as many as fit).
cudaError_t launch_neuron_update(const DevNet& g, int32_t t_rel, cudaStream_t st, int stages, int blocks_per_sm,
                                 int32_t upd);
cudaError_t launch_spike_compact(const DevNet& g, int32_t t_rel, cudaStream_t st, int32_t spill_rel);
cudaError_t launch_spill_clear(const DevNet& g, int32_t t_rel, cudaStream_t st);
cudaError_t launch_spike_deliver(const DevNet& g, int32_t t_rel, int blocks, cudaStream_t st);
cudaError_t launch_drain(const DevNet& g, int32_t t_rel, int blocks, cudaStream_t st);
// Bins mode: the queue of arrival step t + t_rel sorted into region bins.
cudaError_t launch_bin(const DevNet& g, int32_t t_rel, cudaStream_t st);
cudaError_t launch_bold_step(const DevNet& g, int32_t t_rel, cudaStream_t st);
cudaError_t launch_advance(const DevNet& g, int32_t k, cudaStream_t st);
cudaError_t launch_begin_call(const DevNet& g, cudaStream_t st);
int deliver_blocks_per_sm();

// setup
cudaError_t launch_init_voltage(const DevNet& g, uint64_t init_seed, cudaStream_t st);
// Validates the CSR (targets < n, classes < nch, rows ascending) and computes
// per-(target, channel) sums of |w_acc| into insum [nch][npad] (zeroed by the
// caller); bad != 0 afterwards on a malformed table, *max_insum = the largest sum.
cudaError_t launch_check_synapses(const DevNet& g, unsigned long long* insum, int* bad,
                                  unsigned long long* max_insum, cudaStream_t st);
cudaError_t launch_ring_sums(const DevNet& g, unsigned long long* sums, cudaStream_t st);
cudaError_t launch_ring_gather(const DevNet& g, const int64_t* idx, int64_t m, int32_t* out, cudaStream_t st);
// Kernel-level spike compaction on caller buffers (standalone.cu).
size_t compact_scratch_bytes(int64_t n);
cudaError_t compact_bits(const uint32_t* bits, int64_t n, int32_t* ids, int32_t* count, void* scratch,
                         cudaStream_t st);
// Event-queue mode: dense ring view <-> queues (x_acc = the accumulator's slot).
cudaError_t launch_queue_to_dense(const DevNet& g, int32_t* dense, int32_t x_acc, cudaStream_t st);
cudaError_t launch_add(int32_t* dst, const int32_t* src, int64_t n, cudaStream_t st);
// Bins mode: adds the bins of step x (parity x mod 2, ring slot x mod D) into
// a dense ring, into per-slot sums [D][nch], and/or into out [m][D][nch] for
// the neurons whose row map [n] gives (-1: not requested); NULL skips a view.
cudaError_t launch_bins_view(const DevNet& g, int64_t x, int32_t* dense, unsigned long long* sums,
                             const int32_t* map, int32_t* out, cudaStream_t st);
cudaError_t launch_dense_to_queue(const DevNet& g, const int32_t* dense, int32_t x_acc, cudaStream_t st);
// Test hook: unused queue and bin entries filled with weight-0 placeholders, counts set to value.
cudaError_t launch_preset_counters(const DevNet& g, unsigned long long value, cudaStream_t st);
cudaError_t launch_queue_sums(const DevNet& g, unsigned long long* sums, int32_t x_acc, cudaStream_t st);
cudaError_t launch_queue_gather(const DevNet& g, const int64_t* idx, int64_t m, int32_t* map, int32_t* out,
                                int32_t x_acc, cudaStream_t st);
// Records msg as the calling thread's dtb_last_error() text; returns code.
int32_t set_last_error(int32_t code, const std::string& msg);
// Fills the per-synapse delay bytes out [nnz] (after the synapse check).
cudaError_t launch_delay_fill(const DevNet& g, uint8_t* out, cudaStream_t st);
// Fills the packed synapse records out [nnz] (queue and bins modes, weight formats
// with 16-bit codes), after the synapse check, each chunk of a row sorted by
// delay and target; counts [chunks] receives each chunk's number of runs
// (g.chunk_base set).
cudaError_t launch_pack_fill(const DevNet& g, uint2* out, int32_t* counts, cudaStream_t st);
// The chunks' run records from the run pointers, and each record's run index.
cudaError_t launch_run_fill(const DevNet& g, uint2* pack, const int64_t* run_ptr, uint32_t* runs, cudaStream_t st);
cudaError_t launch_bounded_wait(long long max_cycles, int32_t arrive, int32_t* status, cudaStream_t st);
cudaError_t launch_item_count(const DevNet& g, uint8_t* out, int32_t* too_long, cudaStream_t st);
cudaError_t launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n, cudaStream_t st);

// Assimilation cycle (assimilate.cu): the device view of an ensemble.
struct EnsDev {
  int32_t C, M;                 // columns, members
  const int32_t* member_voxel;  // [C][M] voxel of each member
  const int32_t* target_voxel;  // [C] observed voxel of each column (or NULL)
  float* theta;                 // [C][M] parameters (log gains)
  const double* g_base;         // [nv][4] base conductances
  const double* cap;            // [nv] membrane capacitance
  double dt;
  int32_t mask;                 // receptors scaled by exp(theta)
  float obs_sd_rel, inflation;
  uint32_t key0, key1;          // Philox key of the observation perturbations
};
// One analysis per column from BOLD sample row `row`, then the members'
// constants and the per-tile copies (tile_vox [nblk]: the voxel whose
// constants tile b copies).
cudaError_t launch_enkf_cycle(const EnsDev& e, const float* bold_log, int32_t nv, int64_t row, const float* obs,
                              uint32_t tr, float* theta_hist, float* hx_hist, float* y_hist, VoxConst* vc,
                              VoxConst* tile_vc, const int32_t* tile_vox, int32_t nblk, cudaStream_t st);
// The members' constants from their current parameters (no analysis).
cudaError_t launch_resample(const EnsDev& e, VoxConst* vc, VoxConst* tile_vc, const int32_t* tile_vox, int32_t nblk,
                            cudaStream_t st);

}  // namespace dtb
