// dtb_api.cu -- the C ABI of libdtb.so (declared in include/dtb.h).
//
// Host-side work: argument validation, per-voxel constants (double, rounded
// once to float), Poisson inversion thresholds, device memory (through the
// caller's allocator hooks when given), the CUDA graph of a chunk of steps,
// and copies in and out.  Every step of the simulation itself runs in the
// kernels of step_kernels.cu.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "dtb.h"
#include "dtb_device.cuh"
#include "dtb_launch.h"

using dtb::DevNet;
using dtb::VoxConst;

namespace {

thread_local std::string g_error;

dtb_status fail(dtb_status code, const std::string& msg) {
  g_error = msg;
  return code;
}

dtb_status cuda_fail(cudaError_t e, const char* where) {
  return fail(DTB_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define DTB_CUDA(call)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

constexpr int kGraphSteps = 32;
constexpr int kTimedKernels = 5;  // update, compaction, delivery, drain or binning, BOLD
// Networks of at most this many 1,024-neuron blocks run the compaction of a
// step beside the neuron update of the next by default: their kernels leave
// most of the GPU idle, and the step is a chain of short launches.  Larger
// networks' updates fill every SM, and the compaction then waits its turn.
constexpr int32_t kBesideMaxBlocks = 4096;
constexpr int kBoldLogCap = 1024;

}  // namespace

struct dtb_net {
  DevNet g{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // side branches of the step sequence: delivery, queue drain and BOLD step
  // (fork and join by events)
  cudaStream_t side[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  dtb_alloc_fn alloc = nullptr;
  dtb_free_fn free_fn = nullptr;
  void* alloc_ctx = nullptr;
  std::vector<void*> owned;
  std::vector<double> vparams;  // [nv][DTB_NP]
  std::vector<int64_t> vstart;
  double dt = 0;
  uint64_t init_seed = 0;
  double ou_mu = 0;          // initial OU current
  int deliver_blocks = 0;
  int update_stages = 3;     // neuron update pipeline depth
  int update_per_sm = 0;     // neuron update CTAs per SM (0 = as many as fit)
  int schedule = -1;         // requested: -1 by size, 0 compaction after the update, 1 beside the next update
  bool beside = false;       // in effect: the compaction of step t runs beside the update of step t + 1
  // the second copy of the spike bits (words) and of the block counts (blocks)
  int64_t flag_par = 0;
  int32_t cnt_par = 0;
  int sms = 1;
  cudaGraphExec_t graph[33] = {};  // graph[k]: a chunk of k body steps (k <= kGraphSteps), built on first use
  int64_t t = 0;           // steps run (mirror of *t_base)
  int64_t call_t0 = 0;     // t at the start of the last dtb_step
  int64_t call_steps = 0;  // steps of the last dtb_step
  int64_t step_off_cap = 0;
  unsigned long long* d_scratch_u64 = nullptr;

  void* dalloc(size_t bytes) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    void* p = nullptr;
    if (alloc) {
      p = alloc(bytes, alloc_ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    if (p) owned.push_back(p);
    return p;
  }
  void dfree(void* p) {
    if (!p) return;
    for (size_t k = 0; k < owned.size(); k++)
      if (owned[k] == p) {
        owned.erase(owned.begin() + (long)k);
        break;
      }
    if (free_fn) free_fn(p, alloc_ctx);
    else cudaFree(p);
  }
  void drop_graphs() {
    for (cudaGraphExec_t& g : graph)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
  }
  ~dtb_net() {
    drop_graphs();
    if (stream) cudaStreamSynchronize(stream);
    for (cudaStream_t s : side)
      if (s) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
      }
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
    for (void* p : owned) {
      if (free_fn) free_fn(p, alloc_ctx);
      else cudaFree(p);
    }
    if (own_stream && stream) cudaStreamDestroy(stream);
  }
};

// An assimilation ensemble over one network (dtb_ensemble_create): its
// columns' member and target voxels, the parameters on the device, and the
// per-tile voxel map that the re-sampled constants are copied along.
struct dtb_ensemble {
  dtb_net* net = nullptr;
  dtb::EnsDev e{};
  int32_t tr_steps = 0;
  uint32_t tr_count = 0;  // TRs analysed so far: the perturbations' counter word
  int32_t* tile_vox = nullptr;
  std::vector<int32_t> member_voxel;  // host copy [C][M]
  std::vector<double> g_base;         // host copy [nv][4]
  std::vector<void*> bufs;            // device buffers from the network's allocator
  ~dtb_ensemble() {
    if (net)
      for (void* p : bufs) net->dfree(p);
  }
};

namespace {

// Constants of the Euler map: each evaluated in double, rounded once to float.
void derive_voxel_consts(const dtb_net* net, std::vector<VoxConst>& out) {
  const int nv = (int)net->vstart.size() - 1;
  out.assign(nv, VoxConst{});
  const double dt = net->dt;
  for (int v = 0; v < nv; v++) {
    const double* P = &net->vparams[(size_t)v * DTB_NP];
    VoxConst& c = out[v];
    for (int u = 0; u < 4; u++) {
      c.kU[u] = (float)((dt * P[DTB_P_G + u]) / P[DTB_P_C]);
      c.dJ[u] = (float)(1.0 - dt / P[DTB_P_TAU + u]);
      c.E[u] = (float)P[DTB_P_E + u];
    }
    c.kL = (float)((dt * P[DTB_P_GL]) / P[DTB_P_C]);
    c.EL = (float)P[DTB_P_EL];
    c.kI = (float)((dt * P[DTB_P_IEXT]) / P[DTB_P_C]);
    c.Vth = (float)P[DTB_P_VTH];
    c.Vreset = (float)P[DTB_P_VRESET];
    c.ref_steps = (int)llround(P[DTB_P_TREF] / dt);
    c.kO = (float)(dt / P[DTB_P_C]);
  }
}

// T_m = floor(2^32 * P(Poisson(lambda) <= m)); the CDF is summed term by term
// in double (p_0 = exp(-lambda), p_m = p_{m-1} * lambda / m); the list stops
// at the first m whose threshold reaches 2^32 - 1.
int poisson_thresholds(double lambda, uint32_t* T, int cap) {
  const double two32 = 4294967296.0;
  if (!(lambda >= 0.0)) return -1;
  double p = exp(-lambda), F = p;
  int M = 0;
  for (int m = 0; m <= 1000; m++) {
    if (m > 0) {
      p = p * lambda / (double)m;
      F = F + p;
    }
    const double x = floor(F * two32);
    if (x >= two32 - 1.0) return M;
    if (M >= cap) return -1;
    T[M++] = (uint32_t)x;
  }
  return -1;
}

dtb_status upload_consts(dtb_net* net) {
  std::vector<VoxConst> vc;
  derive_voxel_consts(net, vc);
  for (const VoxConst& c : vc)
    if (c.ref_steps < 0 || c.ref_steps > 255) return fail(DTB_EINVAL, "refractory steps out of 0..255");
  // per neuron tile: the constants of its first neuron's voxel and how many of
  // its neurons that voxel holds (the neuron update streams this with the tile)
  const DevNet& g = net->g;
  std::vector<VoxConst> tvc((size_t)g.nblk);
  size_t v = 0;
  for (int b = 0; b < g.nblk; b++) {
    const int64_t start = (int64_t)b * dtb::kNeuronsPerBlock;
    while (v + 2 < net->vstart.size() && net->vstart[v + 1] <= start) v++;
    tvc[b] = vc[v];
    tvc[b].n_first = (int)std::min<int64_t>(net->vstart[v + 1] - start, (int64_t)dtb::kNeuronsPerBlock);
  }
  DTB_CUDA(cudaMemcpyAsync((void*)net->g.vc, vc.data(), vc.size() * sizeof(VoxConst), cudaMemcpyHostToDevice,
                           net->stream));
  DTB_CUDA(cudaMemcpyAsync((void*)net->g.tile_vc, tvc.data(), tvc.size() * sizeof(VoxConst),
                           cudaMemcpyHostToDevice, net->stream));
  DTB_CUDA(cudaStreamSynchronize(net->stream));
  return DTB_OK;
}

dtb_status init_state(dtb_net* net) {
  DevNet& g = net->g;
  cudaStream_t st = net->stream;
  DTB_CUDA(cudaMemsetAsync(g.j, 0, sizeof(float) * 4 * g.npad, st));
  DTB_CUDA(cudaMemsetAsync(g.ref, 0, g.npad, st));
  if (g.ring) DTB_CUDA(cudaMemsetAsync(g.ring, 0, sizeof(int32_t) * (size_t)(g.mode ? 2 : g.D) * g.nch * g.npad, st));
  if (g.mode == dtb::kModeBins)
    DTB_CUDA(cudaMemsetAsync(g.bcnt, 0, 8 * dtb::kBcntStride * 2 * (size_t)g.n_reg, st));
  if (g.mode) {
    DTB_CUDA(cudaMemsetAsync(g.qcnt, 0, 8 * dtb::kQcntStride * (size_t)g.D, st));
    DTB_CUDA(cudaMemsetAsync(g.drain_done, 0, 16, st));
    DTB_CUDA(cudaMemsetAsync(g.spill, 0, sizeof(int32_t) * (size_t)g.D * g.nch * g.npad, st));
    DTB_CUDA(cudaMemsetAsync(g.spill_dirty, 0, sizeof(int32_t) * (size_t)g.D, st));
  }
  DTB_CUDA(cudaMemsetAsync(g.t_base, 0, sizeof(int64_t), st));
  DTB_CUDA(cudaMemsetAsync(g.events, 0, sizeof(unsigned long long), st));
  DTB_CUDA(cudaMemsetAsync(g.spikes, 0, sizeof(unsigned long long), st));
  DTB_CUDA(cudaMemsetAsync(g.vox_spikes, 0, 8 * (size_t)g.nv, st));
  DTB_CUDA(dtb::launch_init_voltage(g, net->init_seed, st));
  if (g.ou) {
    std::vector<float> I0((size_t)g.npad, (float)net->ou_mu);
    DTB_CUDA(cudaMemcpyAsync(g.Iou, I0.data(), 4 * (size_t)g.npad, cudaMemcpyHostToDevice, st));
    DTB_CUDA(cudaStreamSynchronize(st));  // I0 leaves scope
  }
  std::vector<float> bold((size_t)5 * g.nv, 0.0f);
  for (int v = 0; v < g.nv; v++) bold[g.nv + v] = bold[2 * g.nv + v] = bold[3 * g.nv + v] = 1.0f;
  DTB_CUDA(cudaMemcpyAsync(g.bold, bold.data(), bold.size() * 4, cudaMemcpyHostToDevice, st));
  DTB_CUDA(cudaStreamSynchronize(st));
  net->t = 0;
  net->call_t0 = 0;
  net->call_steps = 0;
  return DTB_OK;
}

dtb_status ensure_step_off(dtb_net* net, int64_t n_steps) {
  if (n_steps + 1 <= net->step_off_cap) return DTB_OK;
  int64_t cap = net->step_off_cap;
  while (cap < n_steps + 1) cap *= 2;
  void* p = net->dalloc(sizeof(int64_t) * cap);
  if (!p) return fail(DTB_ENOMEM, "step offset buffer");
  DTB_CUDA(cudaStreamSynchronize(net->stream));
  net->dfree(net->g.step_off);
  net->g.step_off = (int64_t*)p;
  net->step_off_cap = cap;
  net->drop_graphs();  // the graphs hold the old pointer
  return DTB_OK;
}

// Steps of a dtb_step call.  The spikes of step t depend on V and j at its
// start only; the arrivals consumed at step t only change j for step t + 1.
// So a call runs
//   head:  V part of step t0 (the stored j is j at its start),
//   body:  for t = t0+1 ..: j part of step t-1, then V part of step t,
//   tail:  j part of the last step,
// and between calls the state is exactly the plain step's.  In the body the
// delivery of step t-1's spikes runs beside the neuron update of step t,
// which does not read its arrivals (they are due at step t + 1 or later).
// Per step, on four streams:
//   s0: update(t) -> compact(t)                      [compact waits deliver(t-1), bold(t-1)]
//   s1: compact(t) -> deliver(t)
//   s2: update(t), deliver(t-1) -> drain of the arrivals at t+1   [queue mode]
//       update(t-1), deliver(t-2) -> binning of the arrivals at t [bins mode]
//   s3: compact(t) -> bold(t)
// and update(t) waits for the drain of the arrivals at t-1 (issued at step
// t-2), or in bins mode for their binning (issued at step t-1).  In bins mode
// delay-1 events go straight into the bins, so the queue of the arrivals at t
// is complete after deliver(t-2); update(t-1) has emptied the bins of that
// parity.  The binning of step t thus runs beside deliver(t-1) and update(t).
// With net->beside (small networks) the compaction moves to s1 as well:
//   s0: update(t)                       [waits deliver(t-2) and the binning or drain above]
//   s1: update(t), bold(t-1) -> compact(t) -> deliver(t)
// so compact(t) runs beside update(t + 1).  The two write different copies of
// the spike bits and block counts (the step's index parity); update(t + 2)
// reuses compact(t)'s copy only after deliver(t), which follows compact(t).
// update(t) still consumes the arrivals at t - 1 after every delivery that
// adds to them: deliver(t-2) for delay 1, the binning or drain for the rest.
// Events are those of this sequence only; work before it is complete.
// tev: NULL, or timing events [k][kTimedKernels][2] recorded right before and
// after each launch on the stream that runs it (kernel index: update,
// compaction, delivery, drain or binning, BOLD); ran[s * kTimedKernels + kk]
// tells which pairs were recorded.
// The network as the update and the compaction of the step with index t_rel
// in a sequence see it: the second copy of the spike bits and block counts
// for odd t_rel.  Consecutive steps alternate; a sequence is joined before the
// next one starts, so a copy is never written while its last step is read.
dtb::DevNet step_view(const dtb_net* net, int32_t t_rel) {
  dtb::DevNet d = net->g;
  if (t_rel & 1) {
    d.flags += net->flag_par;
    d.blk_cnt += net->cnt_par;
    d.blk_items += net->cnt_par;
  }
  return d;
}

dtb_status enqueue_range(dtb_net* net, int32_t k, bool head, cudaEvent_t* tev = nullptr, bool* ran = nullptr) {
  cudaStream_t s0 = net->stream, s1 = net->side[0], s2 = net->side[1], s3 = net->side[2];
  cudaEvent_t evF = net->ev[0], evC = net->ev[1], evB = net->ev[2], evS = net->ev[7];
  cudaEvent_t* evD = net->ev + 3;  // deliver(s), by parity of s
  cudaEvent_t* evR = net->ev + 5;  // drain or binning issued at step s, by parity of s
  const bool q = net->g.mode == dtb::kModeQueue, bins = net->g.mode == dtb::kModeBins;
  auto mark = [&](int32_t s, int kk, int end, cudaStream_t st) -> cudaError_t {
    if (!tev) return cudaSuccess;
    if (ran) ran[s * kTimedKernels + kk] = true;
    return cudaEventRecord(tev[(s * kTimedKernels + kk) * 2 + end], st);
  };
  if (bins && k >= 1) {  // fork of the binning branch: everything before this sequence is done
    DTB_CUDA(cudaEventRecord(evS, s0));
    DTB_CUDA(cudaStreamWaitEvent(s2, evS, 0));
  }
  const bool beside = net->beside;
  for (int32_t s = 0; s < k; s++) {
    const bool first = head && s == 0;
    if (q && s >= 2) DTB_CUDA(cudaStreamWaitEvent(s0, evR[(s - 2) & 1], 0));
    if (bins && s >= 1) DTB_CUDA(cudaStreamWaitEvent(s0, evR[(s - 1) & 1], 0));
    if (beside && s >= 2) DTB_CUDA(cudaStreamWaitEvent(s0, evD[(s - 2) & 1], 0));  // deliver(s-2)
    if (bins) {
      if (s >= 1) DTB_CUDA(cudaStreamWaitEvent(s2, evF, 0));               // update(s-1)
      if (s >= 2) DTB_CUDA(cudaStreamWaitEvent(s2, evD[(s - 2) & 1], 0));  // deliver(s-2)
      DTB_CUDA(mark(s, 3, 0, s2));
      DTB_CUDA(dtb::launch_bin(net->g, s, s2));
      DTB_CUDA(mark(s, 3, 1, s2));
      DTB_CUDA(cudaEventRecord(evR[s & 1], s2));
    }
    DTB_CUDA(mark(s, 0, 0, s0));
    DTB_CUDA(dtb::launch_neuron_update(step_view(net, s), s, s0, net->update_stages, net->update_per_sm,
                                       first ? dtb::kUpdV : dtb::kUpdJV));
    DTB_CUDA(mark(s, 0, 1, s0));
    DTB_CUDA(cudaEventRecord(evF, s0));
    // the compaction: after the update on s0, or beside the next update on s1
    // (there deliver(s-1) precedes it on its own stream)
    cudaStream_t sc = beside ? s1 : s0;
    if (beside) DTB_CUDA(cudaStreamWaitEvent(s1, evF, 0));
    if (s >= 1) {
      if (!beside) DTB_CUDA(cudaStreamWaitEvent(s0, evD[(s - 1) & 1], 0));
      DTB_CUDA(cudaStreamWaitEvent(sc, evB, 0));
    }
    DTB_CUDA(mark(s, 1, 0, sc));
    DTB_CUDA(dtb::launch_spike_compact(step_view(net, s), s, sc, first ? 1 : -1));
    DTB_CUDA(mark(s, 1, 1, sc));
    DTB_CUDA(cudaEventRecord(evC, sc));
    if (!beside) DTB_CUDA(cudaStreamWaitEvent(s1, evC, 0));
    DTB_CUDA(mark(s, 2, 0, s1));
    DTB_CUDA(dtb::launch_spike_deliver(net->g, s, net->deliver_blocks, s1));
    DTB_CUDA(mark(s, 2, 1, s1));
    DTB_CUDA(cudaEventRecord(evD[s & 1], s1));
    if (q) {
      DTB_CUDA(cudaStreamWaitEvent(s2, evF, 0));
      if (s >= 1) DTB_CUDA(cudaStreamWaitEvent(s2, evD[(s - 1) & 1], 0));
      DTB_CUDA(mark(s, 3, 0, s2));
      DTB_CUDA(dtb::launch_drain(net->g, s, net->deliver_blocks, s2));
      DTB_CUDA(mark(s, 3, 1, s2));
      DTB_CUDA(cudaEventRecord(evR[s & 1], s2));
    }
    DTB_CUDA(cudaStreamWaitEvent(s3, evC, 0));
    DTB_CUDA(mark(s, 4, 0, s3));
    DTB_CUDA(dtb::launch_bold_step(net->g, s, s3));
    DTB_CUDA(mark(s, 4, 1, s3));
    DTB_CUDA(cudaEventRecord(evB, s3));
  }
  // join every branch into s0
  if (k >= 1) {
    DTB_CUDA(cudaStreamWaitEvent(s0, evD[(k - 1) & 1], 0));
    DTB_CUDA(cudaStreamWaitEvent(s0, evB, 0));
    if (q) {
      DTB_CUDA(cudaStreamWaitEvent(s0, evR[(k - 1) & 1], 0));
      if (k >= 2) DTB_CUDA(cudaStreamWaitEvent(s0, evR[(k - 2) & 1], 0));
    }
    if (bins) DTB_CUDA(cudaStreamWaitEvent(s0, evR[(k - 1) & 1], 0));
  }
  DTB_CUDA(dtb::launch_advance(net->g, k, s0));
  return DTB_OK;
}

// j part of the last step of a call (t_base has moved past it).
dtb_status enqueue_tail(dtb_net* net) {
  DTB_CUDA(dtb::launch_neuron_update(step_view(net, -1), -1, net->stream, net->update_stages, net->update_per_sm,
                                     dtb::kUpdJ));
  DTB_CUDA(dtb::launch_spill_clear(net->g, -1, net->stream));
  return DTB_OK;
}

// A whole call of n >= 1 steps, the body in graph chunks when it is long.
dtb_status enqueue_call(dtb_net* net, int64_t n, bool use_graph) {
  dtb_status s = enqueue_range(net, 1, true);
  if (s != DTB_OK) return s;
  int64_t left = n - 1;
  while (left > 0) {
    const int32_t c = (int32_t)std::min<int64_t>(left, kGraphSteps);
    if (use_graph && net->graph[c]) {
      DTB_CUDA(cudaGraphLaunch(net->graph[c], net->stream));
    } else {
      s = enqueue_range(net, c, false);
      if (s != DTB_OK) return s;
    }
    left -= c;
  }
  return enqueue_tail(net);
}

// The graph of a chunk of k body steps.
dtb_status build_graph(dtb_net* net, int32_t k) {
  cudaGraph_t graph = nullptr;
  DTB_CUDA(cudaStreamBeginCapture(net->stream, cudaStreamCaptureModeThreadLocal));
  dtb_status st = enqueue_range(net, k, false);
  cudaError_t e = cudaStreamEndCapture(net->stream, &graph);
  if (st != DTB_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&net->graph[k], graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    net->graph[k] = nullptr;
    return cuda_fail(e, "cudaGraphInstantiate");
  }
  return DTB_OK;
}

// The graphs a call of n steps launches (full chunks and the remainder), built
// before any of its work is queued.
dtb_status ensure_graphs(dtb_net* net, int64_t n) {
  if (n < 2) return DTB_OK;
  const int64_t body = n - 1;
  const int32_t rem = (int32_t)(body % kGraphSteps);
  if (body >= kGraphSteps && !net->graph[kGraphSteps]) {
    dtb_status s = build_graph(net, kGraphSteps);
    if (s != DTB_OK) return s;
  }
  if (rem > 0 && !net->graph[rem]) return build_graph(net, rem);
  return DTB_OK;
}

}  // namespace

int32_t dtb::set_last_error(int32_t code, const std::string& msg) { return fail(code, msg); }

namespace {

// The kernels' error word: a bounded wait that gave up (the state of that
// step is incomplete, the call reports DTB_ETIMEOUT and the word is cleared).
dtb_status check_device_error(dtb_net* net) {
  int32_t err = 0;
  DTB_CUDA(cudaMemcpy(&err, net->g.err, 4, cudaMemcpyDeviceToHost));
  if (err == 0) return DTB_OK;
  DTB_CUDA(cudaMemset(net->g.err, 0, 4));
  return fail(DTB_ETIMEOUT, "a bounded wait in the neuron update gave up (TMA copy did not complete)");
}

bool valid_stream(cudaStream_t s) { return s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread; }

// Timing events that are destroyed on every return path.
struct TimingEvents {
  cudaEvent_t e[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int n = 0;
  cudaError_t create(int count) {
    for (n = 0; n < count; n++) {
      const cudaError_t r = cudaEventCreate(&e[n]);
      if (r != cudaSuccess) return r;
    }
    return cudaSuccess;
  }
  ~TimingEvents() {
    for (int k = 0; k < n; k++) cudaEventDestroy(e[k]);
  }
};

// Event-queue mode keeps two accumulator slots by step parity; the view of the
// network whose `ring` is the slot of the arrivals at step t.
DevNet acc_view(const dtb_net* net, int64_t t) {
  DevNet v = net->g;
  if (v.mode) v.ring = net->g.ring + (t & 1) * (int64_t)v.nch * v.npad;
  return v;
}

// The host copy of the conductances follows the members' parameters, so that
// a later re-derivation of the constants (dtb_set_hyperparams of other
// voxels' values is not affected) reproduces what the device wrote.
void ens_mirror(dtb_ensemble* ens, const float* theta) {
  dtb_net* net = ens->net;
  const int mask = ens->e.mask;
  for (size_t k = 0; k < ens->member_voxel.size(); k++) {
    const int32_t v = ens->member_voxel[k];
    const double gain = exp((double)theta[k]);
    for (int u = 0; u < 4; u++)
      if ((mask >> u) & 1) net->vparams[(size_t)v * DTB_NP + DTB_P_G + u] = ens->g_base[(size_t)v * 4 + u] * gain;
  }
}

}  // namespace

extern "C" {

const char* dtb_last_error(void) { return g_error.c_str(); }

dtb_status dtb_create_network(const dtb_network_desc* d, dtb_net** out) {
  if (!out) return fail(DTB_EINVAL, "out is NULL");
  *out = nullptr;
  if (!d) return fail(DTB_EINVAL, "desc is NULL");
  if (d->n_neurons < 1 || d->n_neurons >= (int64_t)1 << 30) return fail(DTB_EINVAL, "n_neurons out of 1..2^30-1");
  if (d->n_voxels < 1 || d->n_voxels > 65535) return fail(DTB_EINVAL, "n_voxels out of 1..65535");
  if (d->n_channels != 2 && d->n_channels != 4) return fail(DTB_EINVAL, "n_channels must be 2 or 4");
  if (!d->voxel_start || !d->voxel_params || !d->delay_vv || !d->row_ptr || !d->syn_word || !d->syn_w)
    return fail(DTB_EINVAL, "a required array is NULL");
  if (!(d->dt > 0.0) || !(d->nu_ext >= 0.0)) return fail(DTB_EINVAL, "dt must be > 0 and nu_ext >= 0");
  if (d->d_max < 1 || d->d_max > 255) return fail(DTB_EINVAL, "d_max out of 1..255");
  if (d->weight_format < 0 || d->weight_format > 3) return fail(DTB_EINVAL, "unknown weight_format");
  if (d->weight_shift < 0 || d->weight_shift > 24) return fail(DTB_EINVAL, "weight_shift out of 0..24");
  if (d->bold_every < 0) return fail(DTB_EINVAL, "bold_every < 0");
  if (d->delivery_mode != DTB_DELIVER_RING && d->delivery_mode != DTB_DELIVER_QUEUE &&
      d->delivery_mode != DTB_DELIVER_BINS)
    return fail(DTB_EINVAL, "unknown delivery_mode");
  if (d->bin_capacity < 0) return fail(DTB_EINVAL, "bin_capacity < 0");
  if (d->event_queue_capacity < 0 || d->event_queue_capacity > ((int64_t)1 << 32) - 64)
    return fail(DTB_EINVAL, "event_queue_capacity out of 0..2^32-64");
  if (d->ou_enable && (!(d->ou_tau > 0.0) || !(d->ou_sigma >= 0.0) || !std::isfinite(d->ou_mu) ||
                       !std::isfinite(d->ou_sigma) || !std::isfinite(d->ou_tau)))
    return fail(DTB_EINVAL, "OU drive needs finite mu, sigma >= 0 and tau > 0");
  const int64_t n = d->n_neurons;
  const int nv = d->n_voxels;
  if (d->voxel_start[0] != 0 || d->voxel_start[nv] != n) return fail(DTB_EINVAL, "voxel_start must run 0..n");
  for (int v = 0; v < nv; v++)
    if (d->voxel_start[v + 1] < d->voxel_start[v]) return fail(DTB_EINVAL, "voxel_start not ascending");
  for (int64_t k = 0; k < (int64_t)nv * nv; k++)
    if (d->delay_vv[k] < 1 || d->delay_vv[k] > d->d_max) return fail(DTB_EINVAL, "delay outside 1..d_max");
  for (int v = 0; v < nv; v++) {
    const double* P = d->voxel_params + (size_t)v * DTB_NP;
    if (!(P[DTB_P_C] > 0.0)) return fail(DTB_EINVAL, "C must be > 0");
    for (int u = 0; u < 4; u++)
      if (!(P[DTB_P_TAU + u] > 0.0)) return fail(DTB_EINVAL, "tau must be > 0");
  }

  dtb_net* net = new dtb_net();
  DevNet& g = net->g;
  net->alloc = d->alloc;
  net->free_fn = d->free;
  net->alloc_ctx = d->alloc_ctx;
  net->dt = d->dt;
  net->init_seed = d->init_seed;
  net->vparams.assign(d->voxel_params, d->voxel_params + (size_t)nv * DTB_NP);
  net->vstart.assign(d->voxel_start, d->voxel_start + nv + 1);
  if (d->stream) {
    net->stream = (cudaStream_t)d->stream;
    if (!valid_stream(net->stream)) {
      delete net;
      return fail(DTB_EINVAL, "stream must not be a default stream (graph capture)");
    }
  } else {
    if (cudaStreamCreateWithFlags(&net->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete net;
      return fail(DTB_ECUDA, "cudaStreamCreate failed");
    }
    net->own_stream = true;
  }
  for (cudaStream_t& s : net->side)
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      delete net;
      return fail(DTB_ECUDA, "cudaStreamCreate failed");
    }
  for (cudaEvent_t& e : net->ev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      delete net;
      return fail(DTB_ECUDA, "cudaEventCreate failed");
    }

  const int64_t npad = (n + dtb::kNeuronsPerBlock - 1) / dtb::kNeuronsPerBlock * dtb::kNeuronsPerBlock;
  g.n = n;
  g.npad = npad;
  g.nv = nv;
  g.nch = d->n_channels;
  g.D = d->d_max + 1;
  g.nblk = (int32_t)(npad / dtb::kNeuronsPerBlock);
  g.ntiles = (g.nblk + dtb::kCompactBlocksPerTile - 1) / dtb::kCompactBlocksPerTile;
  g.w_ext = d->w_ext;
  g.wfmt = d->weight_format;
  g.wshift = d->weight_shift;
  g.key0 = (uint32_t)d->seed;
  g.key1 = (uint32_t)(d->seed >> 32);
  const double lambda = (d->nu_ext * d->dt) / 1000.0;
  g.M = poisson_thresholds(lambda, g.T, dtb::kMaxPoisson);
  if (g.M < 0) {
    delete net;
    return fail(DTB_EINVAL, "drive rate needs more than 16 Poisson thresholds");
  }
  int cs = 0;
  while ((n >> cs) > 8192) cs++;
  g.coarse_shift = cs;

  // lookup tables
  std::vector<int32_t> vs32(nv + 1);
  for (int v = 0; v <= nv; v++) vs32[v] = (int32_t)d->voxel_start[v];
  auto vox_of = [&](int64_t i) {
    int lo = 0, hi = nv - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (d->voxel_start[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
  };
  const int64_t ncoarse = ((n - 1) >> cs) + 1;
  std::vector<uint16_t> coarse(ncoarse), blk_vox(g.nblk);
  for (int64_t c = 0; c < ncoarse; c++) coarse[c] = (uint16_t)vox_of(c << cs);
  for (int b = 0; b < g.nblk; b++) blk_vox[b] = (uint16_t)vox_of(std::min<int64_t>((int64_t)b * 1024, n - 1));
  std::vector<float> inv_nvox(nv);
  const double dt_s = d->dt * 1e-3;
  for (int v = 0; v < nv; v++) {
    const int64_t nn = d->voxel_start[v + 1] - d->voxel_start[v];
    inv_nvox[v] = nn > 0 ? (float)(1.0 / ((double)nn * dt_s)) : 0.0f;
  }
  dtb::BoldConst& bc = g.bc;
  bc.eps = (float)d->bold_eps;
  bc.inv_tau_s = (float)(1.0 / d->bold_tau_s);
  bc.inv_tau_f = (float)(1.0 / d->bold_tau_f);
  bc.inv_tau_0 = (float)(1.0 / d->bold_tau_0);
  bc.inv_alpha = (float)(1.0 / d->bold_alpha);
  bc.ln_1mE0 = (float)log(1.0 - d->bold_E0);
  bc.inv_E0 = (float)(1.0 / d->bold_E0);
  bc.V0 = (float)d->bold_V0;
  bc.k1 = (float)(7.0 * d->bold_E0);
  bc.k2 = 2.0f;
  bc.k3 = (float)(2.0 * d->bold_E0 - 0.2);
  bc.dt_s = (float)dt_s;
  g.bold_every = d->bold_every;
  g.bold_cap = kBoldLogCap;
  g.log_cap = d->spike_log_capacity > 0 ? d->spike_log_capacity : ((int64_t)1 << 25);
  g.mode = d->delivery_mode;
  g.ou = d->ou_enable ? 1 : 0;
  net->ou_mu = d->ou_mu;
  if (g.ou) {
    g.ou_d = (float)(1.0 - d->dt / d->ou_tau);
    g.ou_c = (float)((d->ou_mu * d->dt) / d->ou_tau);
    g.ou_s = (float)(d->ou_sigma * sqrt((2.0 * d->dt) / d->ou_tau));
    g.ou_xi = (float)(1.7320508075688772 / 4294967296.0);  // sqrt(3) * 2^-32
  }
  if (g.mode) {
    int64_t cap = d->event_queue_capacity > 0 ? d->event_queue_capacity : 2 * n;
    cap = std::max<int64_t>(cap, 1024);
    // a multiple of 16 events (the drain reads two events per 16 bytes) and an
    // odd number of 128-byte lines, so that the queues' tails do not all map to
    // the same L2 sets (a power-of-two stride between queues did)
    int64_t qc = (cap + 15) & ~(int64_t)15;
    if (((qc / 16) & 1) == 0) qc += 16;
    g.qcap = qc;
  }
  if (g.mode == dtb::kModeBins) {
    g.n_reg = (g.nblk + dtb::kRegionTiles - 1) / dtb::kRegionTiles;
    if (g.n_reg > dtb::kMaxRegions) {
      delete net;
      return fail(DTB_EINVAL, "bins delivery supports up to 2^25 neurons; use DTB_DELIVER_QUEUE");
    }
    // a region's bin holds four times its share of a full queue (at least
    // 4096, at most the queue)
    int64_t bc = std::max<int64_t>(4 * ((g.qcap + g.n_reg - 1) / g.n_reg), 4096);
    bc = std::min<int64_t>(bc, g.qcap);
    if (d->bin_capacity > 0) bc = d->bin_capacity;
    // a whole, odd number of 128-byte lines per bin (see the queue capacity):
    // 32 events of 4 bytes or 16 of 8 bytes (int32 weights) per line
    g.ev8 = d->weight_format == DTB_W_INT32 ? 1 : 0;
    const int64_t per_line = g.ev8 ? 16 : 32;
    bc = (bc + per_line - 1) / per_line * per_line;
    if (((bc / per_line) & 1) == 0) bc += per_line;
    g.bcap = bc;
  }

  // device memory
  bool ok = true;
  auto A = [&](size_t bytes) {
    void* p = net->dalloc(bytes);
    if (!p) ok = false;
    return p;
  };
  g.V = (float*)A(4 * npad);
  g.j = (float*)A(16 * npad);
  g.ref = (uint8_t*)A(npad);
  if (g.ou) g.Iou = (float*)A(4 * npad);
  if (g.mode != dtb::kModeBins) g.ring = (int32_t*)A((size_t)4 * (g.mode ? 2 : g.D) * g.nch * npad);
  if (g.mode == dtb::kModeBins) {
    g.bins = (uint32_t*)A((size_t)4 * (g.ev8 ? 2 : 1) * 2 * g.n_reg * g.bcap);
    g.bcnt = (unsigned long long*)A((size_t)8 * dtb::kBcntStride * 2 * g.n_reg);
  }
  if (g.mode) {
    g.q = (uint2*)A((size_t)8 * g.D * g.qcap);
    g.qcnt = (unsigned long long*)A((size_t)8 * dtb::kQcntStride * g.D);
    g.drain_done = (uint32_t*)A(16);
    g.spill = (int32_t*)A((size_t)4 * g.D * g.nch * npad);
    g.spill_dirty = (int32_t*)A((size_t)4 * g.D);
  }
  g.vc = (const VoxConst*)A(sizeof(VoxConst) * nv);
  g.vstart = (const int32_t*)A(4 * (nv + 1));
  g.coarse = (const uint16_t*)A(2 * ncoarse);
  g.blk_vox = (const uint16_t*)A(2 * g.nblk);
  g.tile_vc = (const VoxConst*)A(sizeof(VoxConst) * g.nblk);
  g.delay = (const uint8_t*)A((size_t)nv * nv);
  g.inv_nvox = (const float*)A(4 * nv);
  // spike bits and block counts: two copies (the schedule that runs the
  // compaction beside the next update alternates between them)
  net->flag_par = npad / 32;
  net->cnt_par = (g.nblk + 3) & ~3;  // keeps the second copy 16-byte aligned
  g.flags = (uint32_t*)A(2 * (npad / 8));
  g.blk_cnt = (int32_t*)A(8 * (size_t)net->cnt_par);
  g.blk_items = (int32_t*)A(8 * (size_t)net->cnt_par);
  g.n_items = (int32_t*)A(16);
  g.spk = (int32_t*)A(4 * npad);
  g.n_spk = (int32_t*)A(16);
  g.t_base = (int64_t*)A(16);
  g.log_ids = (int32_t*)A(4 * g.log_cap);
  g.log_pos = (int64_t*)A(16);
  g.call_steps = (int32_t*)A(16);
  g.log_trunc = (int32_t*)A(16);
  g.err = (int32_t*)A(16);
  g.events = (unsigned long long*)A(16);
  g.spikes = (unsigned long long*)A(16);
  g.bold = (float*)A(4 * 5 * (size_t)nv);
  g.vox_spikes = (unsigned long long*)A(8 * (size_t)nv);
  g.bold_log = (float*)A(4 * (size_t)kBoldLogCap * nv);
  net->step_off_cap = 1024;
  g.step_off = (int64_t*)A(8 * net->step_off_cap);
  if (!ok) {
    delete net;
    return fail(DTB_ENOMEM, "device allocation failed");
  }
  cudaStream_t st = net->stream;
  auto H2D = [&](const void* dst, const void* src, size_t bytes) {
    return cudaMemcpyAsync((void*)dst, src, bytes, cudaMemcpyHostToDevice, st);
  };
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = H2D(g.vstart, vs32.data(), 4 * (nv + 1));
  if (e == cudaSuccess) e = H2D(g.coarse, coarse.data(), 2 * ncoarse);
  if (e == cudaSuccess) e = H2D(g.blk_vox, blk_vox.data(), 2 * g.nblk);
  if (e == cudaSuccess) e = H2D(g.delay, d->delay_vv, (size_t)nv * nv);
  if (e == cudaSuccess) e = H2D(g.inv_nvox, inv_nvox.data(), 4 * nv);
  if (e == cudaSuccess) e = cudaMemsetAsync(g.V, 0, 4 * npad, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(g.flags, 0, 2 * (npad / 8), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(g.n_spk, 0, 16, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(g.err, 0, 16, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    delete net;
    return cuda_fail(e, "upload of lookup tables");
  }

  // synapses: adopt device arrays or copy host arrays
  int64_t nnz = 0;
  if (d->csr_on_device) {
    e = cudaMemcpy(&nnz, d->row_ptr + n, 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      delete net;
      return cuda_fail(e, "reading row_ptr[n]");
    }
    g.row_ptr = d->row_ptr;
    g.word = d->syn_word;
    g.w = d->syn_w;
    g.row_shift = d->row_shift;
  } else {
    nnz = d->row_ptr[n];
    if (d->row_ptr[0] != 0 || nnz < 0) {
      delete net;
      return fail(DTB_EINVAL, "row_ptr must start at 0 and end at nnz >= 0");
    }
    const size_t wb = d->weight_format == DTB_W_INT32 ? 4 : d->weight_format == DTB_W_INT8 ? 1 : 2;
    void* rp = A(8 * (n + 1));
    void* wd = A(4 * (size_t)nnz);
    void* ww = A(wb * (size_t)nnz);
    void* rs = (d->weight_format == DTB_W_INT8 && d->row_shift) ? A(n) : nullptr;
    if (!ok) {
      delete net;
      return fail(DTB_ENOMEM, "device allocation of the synapse table failed");
    }
    e = H2D(rp, d->row_ptr, 8 * (n + 1));
    if (e == cudaSuccess && nnz) e = H2D(wd, d->syn_word, 4 * (size_t)nnz);
    if (e == cudaSuccess && nnz) e = H2D(ww, d->syn_w, wb * (size_t)nnz);
    if (e == cudaSuccess && rs) e = H2D(rs, d->row_shift, n);
    if (e != cudaSuccess) {
      delete net;
      return cuda_fail(e, "upload of the synapse table");
    }
    g.row_ptr = (const int64_t*)rp;
    g.word = (const uint32_t*)wd;
    g.w = ww;
    g.row_shift = (const uint8_t*)rs;
  }

  // delivery work items: at most one per spike plus one per kItemEvents synapses
  {
    const int64_t cap = n + nnz / dtb::kItemEvents + 1;
    if (cap >= ((int64_t)1 << 31)) {
      delete net;
      return fail(DTB_EINVAL, "too many delivery work items for int32 counts");
    }
    g.items = (dtb::WorkItem*)net->dalloc(sizeof(dtb::WorkItem) * (size_t)cap);
    if (!g.items) {
      delete net;
      return fail(DTB_ENOMEM, "delivery work items");
    }
    if (cudaMemsetAsync(g.n_items, 0, 16, st) != cudaSuccess) {
      delete net;
      return fail(DTB_ECUDA, "memset");
    }
  }

  // validation and overflow bound of the int32 accumulators
  {
    unsigned long long* insum = (unsigned long long*)net->dalloc(8 * (size_t)g.nch * npad);
    void* flagbuf = net->dalloc(64);
    if (!insum || !flagbuf) {
      delete net;
      return fail(DTB_ENOMEM, "scratch of the overflow check");
    }
    int* bad = (int*)flagbuf;
    unsigned long long* mx = (unsigned long long*)((char*)flagbuf + 16);
    e = cudaMemsetAsync(insum, 0, 8 * (size_t)g.nch * npad, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(flagbuf, 0, 64, st);
    if (e == cudaSuccess) e = dtb::launch_check_synapses(g, insum, bad, mx, st);
    int hbad = 0;
    unsigned long long hmx = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hmx, mx, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    net->dfree(insum);
    net->dfree(flagbuf);
    if (e != cudaSuccess) {
      delete net;
      return cuda_fail(e, "synapse check");
    }
    if (hbad) {
      delete net;
      return fail(DTB_EINVAL, (hbad & 1) ? "row_ptr not ascending"
                              : (hbad & 2) ? "synapse target >= n or class >= n_channels"
                                           : "stored weight does not fit int32 after scaling");
    }
    const long double bound = (long double)hmx + (long double)g.M * (long double)(d->w_ext < 0 ? -d->w_ext : d->w_ext);
    if (bound >= 2147483647.0L) {
      delete net;
      return fail(DTB_EOVERFLOW, "sum of |w| into one accumulator plus max drive reaches 2^31");
    }
  }

  // queue and bins modes with 16-bit weight codes: packed synapse records
  // (8 bytes each) instead of the separate delay bytes, each chunk of a row
  // sorted by delay and target, with the chunks' run tables
  if (g.mode != dtb::kModeRing && g.wfmt != DTB_W_INT32 && nnz > 0) {
    // first chunk of every row, from the row pointers
    std::vector<int64_t> rp((size_t)n + 1), cb((size_t)n + 1);
    cudaError_t e2 = cudaMemcpy(rp.data(), g.row_ptr, 8 * ((size_t)n + 1), cudaMemcpyDeviceToHost);
    if (e2 != cudaSuccess) {
      delete net;
      return cuda_fail(e2, "reading row_ptr");
    }
    cb[0] = 0;
    for (int64_t i = 0; i < n; i++) cb[i + 1] = cb[i] + (rp[i + 1] - rp[i] + dtb::kItemEvents - 1) / dtb::kItemEvents;
    const int64_t n_chunks = cb[n];
    rp.clear();
    rp.shrink_to_fit();
    uint2* pk = (uint2*)net->dalloc(8 * (size_t)nnz);
    int64_t* d_cb = (int64_t*)net->dalloc(8 * ((size_t)n + 1));
    int64_t* d_rp = (int64_t*)net->dalloc(8 * ((size_t)n_chunks + 1));
    int32_t* d_cnt = (int32_t*)net->dalloc(4 * (size_t)n_chunks);
    if (!pk || !d_cb || !d_rp || !d_cnt) {
      delete net;
      return fail(DTB_ENOMEM, "packed synapse records and run tables");
    }
    g.chunk_base = d_cb;
    e2 = cudaMemcpyAsync(d_cb, cb.data(), 8 * ((size_t)n + 1), cudaMemcpyHostToDevice, st);
    if (e2 == cudaSuccess) e2 = dtb::launch_pack_fill(g, pk, d_cnt, st);
    std::vector<int32_t> cnt((size_t)n_chunks);
    if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(cnt.data(), d_cnt, 4 * (size_t)n_chunks, cudaMemcpyDeviceToHost, st);
    if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(st);
    if (e2 != cudaSuccess) {
      delete net;
      return cuda_fail(e2, "packed synapse records");
    }
    std::vector<int64_t> run_ptr((size_t)n_chunks + 1);
    run_ptr[0] = 0;
    for (int64_t c = 0; c < n_chunks; c++) run_ptr[c + 1] = run_ptr[c] + cnt[c];
    cnt.clear();
    cnt.shrink_to_fit();
    net->dfree(d_cnt);
    uint32_t* d_runs = (uint32_t*)net->dalloc(4 * (size_t)std::max<int64_t>(run_ptr[n_chunks], 1));
    if (!d_runs) {
      delete net;
      return fail(DTB_ENOMEM, "run tables");
    }
    e2 = cudaMemcpyAsync(d_rp, run_ptr.data(), 8 * ((size_t)n_chunks + 1), cudaMemcpyHostToDevice, st);
    if (e2 == cudaSuccess) e2 = dtb::launch_run_fill(g, pk, d_rp, d_runs, st);
    if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(st);
    if (e2 != cudaSuccess) {
      delete net;
      return cuda_fail(e2, "run tables");
    }
    g.syn_pack = pk;
    g.run_ptr = d_rp;
    g.runs = d_runs;
  } else {  // per-synapse delays (one byte each), read by delivery next to the target word
    uint8_t* sd = (uint8_t*)net->dalloc((size_t)std::max<int64_t>(nnz, 16));
    if (!sd) {
      delete net;
      return fail(DTB_ENOMEM, "per-synapse delays");
    }
    cudaError_t e2 = nnz > 0 ? dtb::launch_delay_fill(g, sd, st) : cudaSuccess;
    if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(st);
    if (e2 != cudaSuccess) {
      delete net;
      return cuda_fail(e2, "per-synapse delays");
    }
    g.syn_delay = sd;
  }

  // work items per neuron (one byte each), streamed with the neuron update's tiles
  {
    uint8_t* ni = (uint8_t*)net->dalloc((size_t)npad);
    if (!ni) {
      delete net;
      return fail(DTB_ENOMEM, "work-item counts");
    }
    g.nitem = ni;
    cudaError_t e2 = cudaMemsetAsync(g.err, 0, 4, st);
    if (e2 == cudaSuccess) e2 = dtb::launch_item_count(g, ni, g.err, st);
    int32_t too_long = 0;
    if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(&too_long, g.err, 4, cudaMemcpyDeviceToHost, st);
    if (e2 == cudaSuccess) e2 = cudaMemsetAsync(g.err, 0, 4, st);
    if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(st);
    if (e2 != cudaSuccess) {
      delete net;
      return cuda_fail(e2, "work-item counts");
    }
    g.nitem_ok = too_long ? 0 : 1;
  }

  dtb_status s = upload_consts(net);
  if (s == DTB_OK) s = init_state(net);
  if (s != DTB_OK) {
    delete net;
    return s;
  }
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  net->deliver_blocks = sms * dtb::deliver_blocks_per_sm();
  net->sms = sms;
  // bins mode: two stages, so that three CTAs (with their arrival sums and
  // staged bins) fit on an SM
  net->update_stages = g.nch == 2 && g.mode != dtb::kModeBins ? 3 : 2;
  net->beside = g.nblk <= kBesideMaxBlocks;
  *out = net;
  return DTB_OK;
}

dtb_status dtb_destroy(dtb_net* net) {
  if (!net) return fail(DTB_EINVAL, "net is NULL");
  delete net;
  return DTB_OK;
}

dtb_status dtb_step(dtb_net* net, int64_t n_steps) {
  if (!net) return fail(DTB_EINVAL, "net is NULL");
  if (n_steps < 0 || n_steps > ((int64_t)1 << 31)) return fail(DTB_EINVAL, "n_steps out of range");
  dtb_status s = ensure_step_off(net, n_steps);
  if (s != DTB_OK) return s;
  s = ensure_graphs(net, n_steps);
  if (s != DTB_OK) return s;
  DTB_CUDA(dtb::launch_begin_call(net->g, net->stream));
  if (n_steps > 0) {
    s = enqueue_call(net, n_steps, true);
    if (s != DTB_OK) return s;
  }
  DTB_CUDA(cudaStreamSynchronize(net->stream));
  net->call_t0 = net->t;
  net->call_steps = n_steps;
  net->t += n_steps;
  return check_device_error(net);
}

dtb_status dtb_step_timed(dtb_net* net, int64_t n_steps, double* ms, int64_t* launches) {
  if (!net || !ms) return fail(DTB_EINVAL, "net or ms is NULL");
  if (n_steps < 0 || n_steps > ((int64_t)1 << 31)) return fail(DTB_EINVAL, "n_steps out of range");
  dtb_status s = ensure_step_off(net, n_steps);
  if (s != DTB_OK) return s;
  double acc[kTimedKernels] = {0, 0, 0, 0, 0};
  int64_t cnt[kTimedKernels] = {0, 0, 0, 0, 0};
  // two sets of events for chunks of kGraphSteps body steps: the host reads
  // one set while the chunk recorded into the other runs, so the device
  // always has the next chunk queued
  constexpr int kPer = kGraphSteps * kTimedKernels * 2;
  struct Set {
    std::vector<cudaEvent_t> ev = std::vector<cudaEvent_t>(kPer, nullptr);
    bool ran[kGraphSteps * kTimedKernels] = {};
    int32_t k = 0;  // steps recorded, 0 = nothing to read
  } sets[2];
  struct Destroy {
    Set* s;
    ~Destroy() {
      for (int q = 0; q < 2; q++)
        for (cudaEvent_t e : s[q].ev)
          if (e) cudaEventDestroy(e);
    }
  } destroy{sets};
  for (Set& st : sets)
    for (cudaEvent_t& e : st.ev) DTB_CUDA(cudaEventCreate(&e));
  auto harvest = [&](Set& st) -> dtb_status {
    for (int32_t q = 0; q < st.k; q++)
      for (int kk = 0; kk < kTimedKernels; kk++) {
        const int at = q * kTimedKernels + kk;
        if (!st.ran[at]) continue;
        DTB_CUDA(cudaEventSynchronize(st.ev[2 * at + 1]));
        float x = 0.0f;
        DTB_CUDA(cudaEventElapsedTime(&x, st.ev[2 * at], st.ev[2 * at + 1]));
        acc[kk] += x;
        cnt[kk] += 1;
        st.ran[at] = false;
      }
    st.k = 0;
    return DTB_OK;
  };
  DTB_CUDA(dtb::launch_begin_call(net->g, net->stream));
  if (n_steps > 0) {
    s = enqueue_range(net, 1, true);  // the first step's V part: not timed
    if (s != DTB_OK) return s;
    int64_t left = n_steps - 1;
    for (int64_t c = 0; left > 0; c++) {
      Set& st = sets[c & 1];
      s = harvest(st);  // the chunk two before this one
      if (s != DTB_OK) return s;
      const int32_t k = (int32_t)std::min<int64_t>(left, kGraphSteps);
      s = enqueue_range(net, k, false, st.ev.data(), st.ran);
      if (s != DTB_OK) return s;
      st.k = k;
      left -= k;
    }
    s = enqueue_tail(net);
    if (s != DTB_OK) return s;
  }
  DTB_CUDA(cudaStreamSynchronize(net->stream));
  for (Set& st : sets) {
    s = harvest(st);
    if (s != DTB_OK) return s;
  }
  for (int kk = 0; kk < kTimedKernels; kk++) {
    ms[kk] = acc[kk];
    if (launches) launches[kk] = cnt[kk];
  }
  net->call_t0 = net->t;
  net->call_steps = n_steps;
  net->t += n_steps;
  return check_device_error(net);
}

dtb_status dtb_get_spikes(dtb_net* net, int64_t* step_offsets, int32_t* ids, int64_t cap, int64_t* n_out) {
  if (!net || !n_out) return fail(DTB_EINVAL, "net or n_out is NULL");
  int64_t pos = 0;
  int32_t trunc = 0;
  DTB_CUDA(cudaMemcpyAsync(&pos, net->g.log_pos, 8, cudaMemcpyDeviceToHost, net->stream));
  DTB_CUDA(cudaMemcpyAsync(&trunc, net->g.log_trunc, 4, cudaMemcpyDeviceToHost, net->stream));
  DTB_CUDA(cudaStreamSynchronize(net->stream));
  *n_out = pos;
  if (step_offsets)
    DTB_CUDA(cudaMemcpyAsync(step_offsets, net->g.step_off, 8 * (net->call_steps + 1), cudaMemcpyDeviceToHost,
                             net->stream));
  if (ids && cap >= pos && pos > 0)
    DTB_CUDA(cudaMemcpyAsync(ids, net->g.log_ids, 4 * pos, cudaMemcpyDeviceToHost, net->stream));
  DTB_CUDA(cudaStreamSynchronize(net->stream));
  if (ids && cap < pos) return fail(DTB_ETRUNC, "ids buffer smaller than *n_out");
  if (trunc) return fail(DTB_ETRUNC, "spike log overflowed during the last dtb_step");
  return DTB_OK;
}

dtb_status dtb_get_bold(dtb_net* net, float* y, float* state) {
  if (!net) return fail(DTB_EINVAL, "net is NULL");
  const int nv = net->g.nv;
  if (state)
    DTB_CUDA(cudaMemcpyAsync(state, net->g.bold, 4 * 4 * (size_t)nv, cudaMemcpyDeviceToHost, net->stream));
  if (y) DTB_CUDA(cudaMemcpyAsync(y, net->g.bold + 4 * nv, 4 * (size_t)nv, cudaMemcpyDeviceToHost, net->stream));
  DTB_CUDA(cudaStreamSynchronize(net->stream));
  return DTB_OK;
}

dtb_status dtb_get_bold_samples(dtb_net* net, float* out, int64_t cap, int64_t* n_samples) {
  if (!net || !n_samples) return fail(DTB_EINVAL, "net or n_samples is NULL");
  const int64_t every = net->g.bold_every;
  if (every <= 0) {
    *n_samples = 0;
    return DTB_OK;
  }
  const int64_t t0 = net->call_t0, t1 = net->call_t0 + net->call_steps;
  int64_t first = t0 / every, last = t1 / every;  // sample indices [first, last)
  if (last - first > net->g.bold_cap) first = last - net->g.bold_cap;
  *n_samples = last - first;
  if (!out) return DTB_OK;
  if (cap < last - first) return fail(DTB_ETRUNC, "out smaller than n_samples");
  const int nv = net->g.nv;
  for (int64_t k = first; k < last; k++)
    DTB_CUDA(cudaMemcpyAsync(out + (k - first) * nv, net->g.bold_log + (k % net->g.bold_cap) * nv, 4 * (size_t)nv,
                             cudaMemcpyDeviceToHost, net->stream));
  DTB_CUDA(cudaStreamSynchronize(net->stream));
  return DTB_OK;
}

dtb_status dtb_get_state(dtb_net* net, float* V, float* j, uint8_t* ref, int32_t* ring, int64_t* t) {
  if (!net) return fail(DTB_EINVAL, "net is NULL");
  const DevNet& g = net->g;
  cudaStream_t st = net->stream;
  const size_t n = (size_t)g.n, np = (size_t)g.npad;
  if (V) DTB_CUDA(cudaMemcpyAsync(V, g.V, 4 * n, cudaMemcpyDeviceToHost, st));
  if (j) DTB_CUDA(cudaMemcpy2DAsync(j, 4 * n, g.j, 4 * np, 4 * n, 4, cudaMemcpyDeviceToHost, st));
  if (ref) DTB_CUDA(cudaMemcpyAsync(ref, g.ref, n, cudaMemcpyDeviceToHost, st));
  if (ring && !g.mode)
    DTB_CUDA(cudaMemcpy2DAsync(ring, 4 * n, g.ring, 4 * np, 4 * n, (size_t)g.D * g.nch, cudaMemcpyDeviceToHost, st));
  if (ring && g.mode) {
    // dense view: the accumulator is slot t mod D, queue x sums into slot x;
    // in bins mode every queue is a slot and the bins of parity t mod 2 hold
    // slot t mod D's delay-1 events
    const size_t bytes = 4 * (size_t)g.D * g.nch * np;
    int32_t* dense = (int32_t*)net->dalloc(bytes);
    if (!dense) return fail(DTB_ENOMEM, "dense ring view");
    const bool bins = g.mode == dtb::kModeBins;
    const int32_t xa = bins ? -1 : (int32_t)(net->t % g.D);
    cudaError_t e = cudaMemcpyAsync(dense, g.spill, bytes, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && !bins)
      e = dtb::launch_add(dense + (size_t)xa * g.nch * np, acc_view(net, net->t).ring, (int64_t)g.nch * np, st);
    if (e == cudaSuccess) e = dtb::launch_queue_to_dense(g, dense, xa, st);
    if (e == cudaSuccess && bins) e = dtb::launch_bins_view(g, net->t, dense, nullptr, nullptr, nullptr, st);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(ring, 4 * n, dense, 4 * np, 4 * n, (size_t)g.D * g.nch, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    net->dfree(dense);
    if (e != cudaSuccess) return cuda_fail(e, "dense ring view");
  }
  DTB_CUDA(cudaStreamSynchronize(st));
  if (t) *t = net->t;
  return DTB_OK;
}

dtb_status dtb_set_state(dtb_net* net, const float* V, const float* j, const uint8_t* ref, const int32_t* ring,
                         int64_t t) {
  if (!net) return fail(DTB_EINVAL, "net is NULL");
  if (t < 0) return fail(DTB_EINVAL, "t < 0");
  const DevNet& g = net->g;
  cudaStream_t st = net->stream;
  const size_t n = (size_t)g.n, np = (size_t)g.npad;
  if (V) DTB_CUDA(cudaMemcpyAsync(g.V, V, 4 * n, cudaMemcpyHostToDevice, st));
  if (j) DTB_CUDA(cudaMemcpy2DAsync(g.j, 4 * np, j, 4 * n, 4 * n, 4, cudaMemcpyHostToDevice, st));
  if (ref) DTB_CUDA(cudaMemcpyAsync(g.ref, ref, n, cudaMemcpyHostToDevice, st));
  if (ring && !g.mode)
    DTB_CUDA(cudaMemcpy2DAsync(g.ring, 4 * np, ring, 4 * n, 4 * n, (size_t)g.D * g.nch, cudaMemcpyHostToDevice, st));
  if (ring && g.mode == dtb::kModeBins) {
    // the whole ring goes into the spill ring, which the neuron update adds
    // in slot by slot; queues and bins start empty
    const size_t bytes = 4 * (size_t)g.D * g.nch * np;
    std::vector<int32_t> dirty((size_t)g.D, 1);
    cudaError_t e = cudaMemsetAsync(g.spill, 0, bytes, st);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(g.spill, 4 * np, ring, 4 * n, 4 * n, (size_t)g.D * g.nch, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(g.spill_dirty, dirty.data(), 4 * (size_t)g.D, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(g.qcnt, 0, 8 * (size_t)dtb::kQcntStride * g.D, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(g.bcnt, 0, 8 * (size_t)dtb::kBcntStride * 2 * g.n_reg, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "dense ring to spill ring");
  } else if (ring && g.mode) {
    // slot t mod D becomes the accumulator, every nonzero entry of the other
    // slots one queued event
    const size_t bytes = 4 * (size_t)g.D * g.nch * np;
    int32_t* dense = (int32_t*)net->dalloc(bytes);
    if (!dense) return fail(DTB_ENOMEM, "dense ring staging");
    const int32_t xa = (int32_t)(t % g.D);
    cudaError_t e = cudaMemsetAsync(dense, 0, bytes, st);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(dense, 4 * np, ring, 4 * n, 4 * n, (size_t)g.D * g.nch, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(g.ring, 0, 4 * (size_t)2 * g.nch * np, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(acc_view(net, t).ring, dense + (size_t)xa * g.nch * np, 4 * (size_t)g.nch * np,
                          cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(g.qcnt, 0, 8 * (size_t)dtb::kQcntStride * g.D, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(g.spill, 0, bytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(g.spill_dirty, 0, 4 * (size_t)g.D, st);
    if (e == cudaSuccess) e = dtb::launch_dense_to_queue(g, dense, xa, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    net->dfree(dense);
    if (e != cudaSuccess) return cuda_fail(e, "dense ring to queues");
  }
  DTB_CUDA(cudaMemcpyAsync(g.t_base, &t, 8, cudaMemcpyHostToDevice, st));
  DTB_CUDA(cudaStreamSynchronize(st));
  net->t = t;
  net->call_steps = 0;
  return DTB_OK;
}

dtb_status dtb_reset(dtb_net* net) {
  if (!net) return fail(DTB_EINVAL, "net is NULL");
  return init_state(net);
}

dtb_status dtb_set_hyperparams(dtb_net* net, const double* g_u) {
  if (!net || !g_u) return fail(DTB_EINVAL, "net or g is NULL");
  const int nv = net->g.nv;
  for (int v = 0; v < nv; v++)
    for (int u = 0; u < 4; u++) {
      if (!(g_u[v * 4 + u] >= 0.0)) return fail(DTB_EINVAL, "conductances must be >= 0");
      net->vparams[(size_t)v * DTB_NP + DTB_P_G + u] = g_u[v * 4 + u];
    }
  return upload_consts(net);
}

dtb_status dtb_get_voxel_spikes(dtb_net* net, int64_t* counts) {
  if (!net || !counts) return fail(DTB_EINVAL, "net or counts is NULL");
  DTB_CUDA(cudaMemcpyAsync(counts, net->g.vox_spikes, 8 * (size_t)net->g.nv, cudaMemcpyDeviceToHost, net->stream));
  DTB_CUDA(cudaStreamSynchronize(net->stream));
  return DTB_OK;
}

dtb_status dtb_counters(dtb_net* net, int64_t* events, int64_t* spikes, int64_t* steps) {
  if (!net) return fail(DTB_EINVAL, "net is NULL");
  unsigned long long ev = 0, sp = 0;
  DTB_CUDA(cudaMemcpyAsync(&ev, net->g.events, 8, cudaMemcpyDeviceToHost, net->stream));
  DTB_CUDA(cudaMemcpyAsync(&sp, net->g.spikes, 8, cudaMemcpyDeviceToHost, net->stream));
  DTB_CUDA(cudaStreamSynchronize(net->stream));
  if (events) *events = (int64_t)ev;
  if (spikes) *spikes = (int64_t)sp;
  if (steps) *steps = net->t;
  return DTB_OK;
}

dtb_status dtb_profile_steps(dtb_net* net, int64_t n_steps, double* ms) {
  if (!net || !ms) return fail(DTB_EINVAL, "net or ms is NULL");
  if (n_steps < 0) return fail(DTB_EINVAL, "n_steps < 0");
  dtb_status s = ensure_step_off(net, n_steps);
  if (s != DTB_OK) return s;
  TimingEvents te;
  DTB_CUDA(te.create(7));
  cudaEvent_t* ev = te.e;
  double acc[5] = {0, 0, 0, 0, 0};
  cudaStream_t st = net->stream;
  DTB_CUDA(dtb::launch_begin_call(net->g, st));
  // bins mode: the binning of step t's arrivals comes first (the update
  // consumes them); its time goes to the drain's entry
  const bool bins = net->g.mode == dtb::kModeBins;
  for (int64_t i = 0; i < n_steps; i++) {
    DTB_CUDA(cudaEventRecord(ev[0], st));
    if (bins) DTB_CUDA(dtb::launch_bin(net->g, 0, st));
    DTB_CUDA(cudaEventRecord(ev[1], st));
    DTB_CUDA(dtb::launch_neuron_update(net->g, 0, st, net->update_stages, net->update_per_sm, dtb::kUpdFull));
    DTB_CUDA(cudaEventRecord(ev[2], st));
    DTB_CUDA(dtb::launch_spike_compact(net->g, 0, st, 0));
    DTB_CUDA(cudaEventRecord(ev[3], st));
    DTB_CUDA(dtb::launch_spike_deliver(net->g, 0, net->deliver_blocks, st));
    DTB_CUDA(cudaEventRecord(ev[4], st));
    if (!bins) DTB_CUDA(dtb::launch_drain(net->g, 0, net->deliver_blocks, st));
    DTB_CUDA(cudaEventRecord(ev[5], st));
    DTB_CUDA(dtb::launch_bold_step(net->g, 0, st));
    DTB_CUDA(cudaEventRecord(ev[6], st));
    DTB_CUDA(dtb::launch_advance(net->g, 1, st));
    DTB_CUDA(cudaEventSynchronize(ev[6]));
    float x[6] = {0, 0, 0, 0, 0, 0};
    for (int k = 0; k < 6; k++) DTB_CUDA(cudaEventElapsedTime(&x[k], ev[k], ev[k + 1]));
    acc[0] += x[1];         // update
    acc[1] += x[2];         // compaction
    acc[2] += x[3];         // delivery
    acc[3] += x[0] + x[4];  // binning or drain
    acc[4] += x[5];         // BOLD
  }
  DTB_CUDA(cudaStreamSynchronize(st));
  for (int k = 0; k < 5; k++) ms[k] = acc[k];
  net->call_t0 = net->t;
  net->call_steps = n_steps;
  net->t += n_steps;
  return check_device_error(net);
}

dtb_status dtb_ring_slot_sums(dtb_net* net, int64_t* sums) {
  if (!net || !sums) return fail(DTB_EINVAL, "net or sums is NULL");
  const size_t pairs = (size_t)net->g.D * net->g.nch;
  unsigned long long* d = (unsigned long long*)net->dalloc(8 * pairs);
  if (!d) return fail(DTB_ENOMEM, "ring sums scratch");
  cudaError_t e = cudaMemsetAsync(d, 0, 8 * pairs, net->stream);
  const int32_t xa = (int32_t)(net->t % net->g.D);
  if (!net->g.mode) {
    if (e == cudaSuccess) e = dtb::launch_ring_sums(net->g, d, net->stream);
  } else {
    const bool bins = net->g.mode == dtb::kModeBins;
    DevNet sp = net->g;   // spilled events, a dense ring
    sp.ring = net->g.spill;
    if (!bins) {
      DevNet one = acc_view(net, net->t);  // the accumulator as a one-slot ring, summed into slot t mod D
      one.D = 1;
      if (e == cudaSuccess) e = dtb::launch_ring_sums(one, d + (size_t)xa * net->g.nch, net->stream);
    }
    if (e == cudaSuccess) e = dtb::launch_ring_sums(sp, d, net->stream);
    if (e == cudaSuccess) e = dtb::launch_queue_sums(net->g, d, bins ? -1 : xa, net->stream);
    if (e == cudaSuccess && bins) e = dtb::launch_bins_view(net->g, net->t, nullptr, d, nullptr, nullptr, net->stream);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(sums, d, 8 * pairs, cudaMemcpyDeviceToHost, net->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(net->stream);
  net->dfree(d);
  if (e != cudaSuccess) return cuda_fail(e, "dtb_ring_slot_sums");
  return DTB_OK;
}

dtb_status dtb_get_ring_at(dtb_net* net, const int64_t* idx, int64_t m, int32_t* out) {
  if (!net || (m > 0 && (!idx || !out)) || m < 0) return fail(DTB_EINVAL, "bad arguments");
  for (int64_t r = 0; r < m; r++)
    if (idx[r] < 0 || idx[r] >= net->g.n) return fail(DTB_EINVAL, "neuron id out of range");
  if (m == 0) return DTB_OK;
  const size_t per = (size_t)net->g.D * net->g.nch;
  int64_t* didx = (int64_t*)net->dalloc(8 * (size_t)m);
  int32_t* dout = (int32_t*)net->dalloc(4 * per * (size_t)m);
  if (!didx || !dout) {
    net->dfree(didx);
    net->dfree(dout);
    return fail(DTB_ENOMEM, "ring gather scratch");
  }
  cudaError_t e = cudaMemcpyAsync(didx, idx, 8 * (size_t)m, cudaMemcpyHostToDevice, net->stream);
  int32_t* map = nullptr;
  if (!net->g.mode) {
    if (e == cudaSuccess) e = dtb::launch_ring_gather(net->g, didx, m, dout, net->stream);
  } else {
    map = (int32_t*)net->dalloc(4 * (size_t)net->g.n);
    if (!map) {
      net->dfree(didx);
      net->dfree(dout);
      return fail(DTB_ENOMEM, "ring gather map");
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(map, 0xFF, 4 * (size_t)net->g.n, net->stream);
    if (e == cudaSuccess)
      e = dtb::launch_queue_gather(acc_view(net, net->t), didx, m, map, dout,
                                   net->g.mode == dtb::kModeBins ? -1 : (int32_t)(net->t % net->g.D), net->stream);
    if (e == cudaSuccess) e = dtb::launch_bins_view(net->g, net->t, nullptr, nullptr, map, dout, net->stream);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, 4 * per * (size_t)m, cudaMemcpyDeviceToHost, net->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(net->stream);
  net->dfree(didx);
  net->dfree(dout);
  net->dfree(map);
  if (e != cudaSuccess) return cuda_fail(e, "dtb_get_ring_at");
  return DTB_OK;
}

dtb_status dtb_autotune(dtb_net* net, int32_t n_steps, int32_t* chosen) {
  if (!net || n_steps < 1) return fail(DTB_EINVAL, "net is NULL or n_steps < 1");
  const int max_del = dtb::deliver_blocks_per_sm();
  struct Cand { int stages, upd, del; };
  std::vector<Cand> cands;
  const int stage_opts[3] = {2, 3, 4};
  for (int s : stage_opts) {
    if (net->g.nch == 4 && s == 4) continue;
    for (int u : {0, 1, 2}) {  // 0: as many as fit (three in bins mode)
      for (int d : {2, 4, 6, 8})
        if (d <= max_del) cands.push_back({s, u, d});
    }
  }
  dtb_status st = ensure_step_off(net, n_steps);
  if (st != DTB_OK) return st;
  TimingEvents te;
  DTB_CUDA(te.create(2));
  cudaEvent_t e0 = te.e[0], e1 = te.e[1];
  double best = 1e30;
  Cand win = {net->update_stages, net->update_per_sm, net->deliver_blocks / std::max(net->sms, 1)};
  for (const Cand& c : cands) {
    net->update_stages = c.stages;
    net->update_per_sm = c.upd;
    net->deliver_blocks = net->sms * c.del;
    DTB_CUDA(dtb::launch_begin_call(net->g, net->stream));
    DTB_CUDA(cudaEventRecord(e0, net->stream));
    st = enqueue_call(net, n_steps, false);
    if (st != DTB_OK) return st;
    DTB_CUDA(cudaEventRecord(e1, net->stream));
    DTB_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    DTB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    net->t += n_steps;
    if (ms < best) {
      best = ms;
      win = c;
    }
  }
  net->update_stages = win.stages;
  net->update_per_sm = win.upd;
  net->deliver_blocks = net->sms * win.del;
  net->drop_graphs();  // launch shapes are baked into the graphs
  net->call_steps = 0;
  if (chosen) {
    chosen[0] = win.stages;
    chosen[1] = win.upd;
    chosen[2] = win.del;
  }
  return check_device_error(net);
}

dtb_status dtb_set_launch_shapes(dtb_net* net, int32_t update_stages, int32_t update_ctas_per_sm,
                                 int32_t deliver_ctas_per_sm) {
  if (!net) return fail(DTB_EINVAL, "net is NULL");
  const int max_stages = net->g.nch == 2 ? 4 : 3;
  if (update_stages < 2 || update_stages > max_stages) return fail(DTB_EINVAL, "update_stages out of range");
  if (update_ctas_per_sm < 0 || update_ctas_per_sm > 2) return fail(DTB_EINVAL, "update_ctas_per_sm out of 0..2");
  if (deliver_ctas_per_sm < 1 || deliver_ctas_per_sm > dtb::deliver_blocks_per_sm())
    return fail(DTB_EINVAL, "deliver_ctas_per_sm out of range");
  net->update_stages = update_stages;
  net->update_per_sm = update_ctas_per_sm;
  net->deliver_blocks = net->sms * deliver_ctas_per_sm;
  net->drop_graphs();  // launch shapes are baked into the graphs
  return DTB_OK;
}

dtb_status dtb_set_schedule(dtb_net* net, int32_t mode) {
  if (!net) return fail(DTB_EINVAL, "net is NULL");
  if (mode < -1 || mode > 1) return fail(DTB_EINVAL, "schedule must be -1, 0 or 1");
  net->schedule = mode;
  net->beside = mode < 0 ? net->g.nblk <= kBesideMaxBlocks : mode == 1;
  net->drop_graphs();  // the schedule is baked into the graphs
  return DTB_OK;
}

dtb_status dtb_get_schedule(dtb_net* net, int32_t* beside) {
  if (!net || !beside) return fail(DTB_EINVAL, "net or beside is NULL");
  *beside = net->beside ? 1 : 0;
  return DTB_OK;
}

dtb_status dtb_get_ou(dtb_net* net, float* I) {
  if (!net || !I) return fail(DTB_EINVAL, "net or I is NULL");
  if (!net->g.ou) return fail(DTB_ESTATE, "the OU drive is off");
  DTB_CUDA(cudaMemcpyAsync(I, net->g.Iou, 4 * (size_t)net->g.n, cudaMemcpyDeviceToHost, net->stream));
  DTB_CUDA(cudaStreamSynchronize(net->stream));
  return DTB_OK;
}

dtb_status dtb_set_ou(dtb_net* net, const float* I) {
  if (!net || !I) return fail(DTB_EINVAL, "net or I is NULL");
  if (!net->g.ou) return fail(DTB_ESTATE, "the OU drive is off");
  DTB_CUDA(cudaMemcpyAsync(net->g.Iou, I, 4 * (size_t)net->g.n, cudaMemcpyHostToDevice, net->stream));
  DTB_CUDA(cudaStreamSynchronize(net->stream));
  return DTB_OK;
}

dtb_status dtb_save_state(dtb_net* net, void* buf, size_t cap, size_t* n_bytes) {
  if (!net || !n_bytes) return fail(DTB_EINVAL, "net or n is NULL");
  const DevNet& g = net->g;
  const size_t n = (size_t)g.n;
  const size_t ringb = 4 * n * (size_t)g.D * g.nch;
  const size_t need = 64 + 4 * n + 16 * n + n + ringb + 20 * (size_t)g.nv + (g.ou ? 4 * n : 0);
  *n_bytes = need;
  if (!buf) return DTB_OK;
  if (cap < need) return fail(DTB_ETRUNC, "checkpoint buffer too small");
  char* p = (char*)buf;
  int64_t hdr[8] = {0x31425444, (int64_t)n, g.nv, g.nch + (g.ou ? 256 : 0), g.D, net->t, 0, 0};
  unsigned long long ev = 0, sp = 0;
  DTB_CUDA(cudaMemcpyAsync(&ev, g.events, 8, cudaMemcpyDeviceToHost, net->stream));
  DTB_CUDA(cudaMemcpyAsync(&sp, g.spikes, 8, cudaMemcpyDeviceToHost, net->stream));
  DTB_CUDA(cudaStreamSynchronize(net->stream));
  hdr[6] = (int64_t)ev;
  hdr[7] = (int64_t)sp;
  memcpy(p, hdr, 64);
  p += 64;
  float* V = (float*)p;
  float* j = V + n;
  uint8_t* ref = (uint8_t*)(j + 4 * n);
  int32_t* ring = (int32_t*)(ref + n);
  float* bold = (float*)((char*)ring + ringb);
  dtb_status s = dtb_get_state(net, V, j, ref, ring, nullptr);
  if (s != DTB_OK) return s;
  DTB_CUDA(cudaMemcpyAsync(bold, g.bold, 20 * (size_t)g.nv, cudaMemcpyDeviceToHost, net->stream));
  if (g.ou) DTB_CUDA(cudaMemcpyAsync(bold + 5 * (size_t)g.nv, g.Iou, 4 * n, cudaMemcpyDeviceToHost, net->stream));
  DTB_CUDA(cudaStreamSynchronize(net->stream));
  return DTB_OK;
}

dtb_status dtb_load_state(dtb_net* net, const void* buf, size_t nbytes) {
  if (!net || !buf) return fail(DTB_EINVAL, "net or buf is NULL");
  const DevNet& g = net->g;
  const size_t n = (size_t)g.n;
  const size_t ringb = 4 * n * (size_t)g.D * g.nch;
  const size_t need = 64 + 4 * n + 16 * n + n + ringb + 20 * (size_t)g.nv + (g.ou ? 4 * n : 0);
  if (nbytes < need) return fail(DTB_EINVAL, "checkpoint too short");
  int64_t hdr[8];
  memcpy(hdr, buf, 64);
  if (hdr[0] != 0x31425444 || hdr[1] != (int64_t)n || hdr[2] != g.nv || hdr[3] != g.nch + (g.ou ? 256 : 0) || hdr[4] != g.D)
    return fail(DTB_EINVAL, "checkpoint does not match this network");
  const char* p = (const char*)buf + 64;
  const float* V = (const float*)p;
  const float* j = V + n;
  const uint8_t* ref = (const uint8_t*)(j + 4 * n);
  const int32_t* ring = (const int32_t*)(ref + n);
  const float* bold = (const float*)((const char*)ring + ringb);
  dtb_status s = dtb_set_state(net, V, j, ref, ring, hdr[5]);
  if (s != DTB_OK) return s;
  const unsigned long long ev = (unsigned long long)hdr[6], sp = (unsigned long long)hdr[7];
  DTB_CUDA(cudaMemcpyAsync(g.bold, bold, 20 * (size_t)g.nv, cudaMemcpyHostToDevice, net->stream));
  if (g.ou) DTB_CUDA(cudaMemcpyAsync(g.Iou, bold + 5 * (size_t)g.nv, 4 * n, cudaMemcpyHostToDevice, net->stream));
  DTB_CUDA(cudaMemcpyAsync(g.events, &ev, 8, cudaMemcpyHostToDevice, net->stream));
  DTB_CUDA(cudaMemcpyAsync(g.spikes, &sp, 8, cudaMemcpyHostToDevice, net->stream));
  DTB_CUDA(cudaStreamSynchronize(net->stream));
  return DTB_OK;
}

dtb_status dtb_ensemble_create(dtb_net* net, const dtb_ensemble_desc* d, dtb_ensemble** out) {
  if (!out) return fail(DTB_EINVAL, "out is NULL");
  *out = nullptr;
  if (!net || !d) return fail(DTB_EINVAL, "net or desc is NULL");
  const int32_t C = d->n_columns, M = d->n_members, nv = net->g.nv;
  if (C < 1 || M < 2) return fail(DTB_EINVAL, "need n_columns >= 1 and n_members >= 2");
  if ((int64_t)C * M > ((int64_t)1 << 28)) return fail(DTB_EINVAL, "n_columns * n_members above 2^28");
  if (!d->member_voxel || !d->theta0 || !d->g_base) return fail(DTB_EINVAL, "member_voxel, theta0 or g_base is NULL");
  if (net->g.bold_every <= 0 || d->tr_steps < 1 || d->tr_steps % net->g.bold_every != 0)
    return fail(DTB_EINVAL, "tr_steps must be a positive multiple of the network's bold_every (> 0)");
  if (!(d->inflation > 0.0f) || !(d->obs_sd_rel >= 0.0f) || !std::isfinite(d->inflation) ||
      !std::isfinite(d->obs_sd_rel))
    return fail(DTB_EINVAL, "need inflation > 0 and obs_sd_rel >= 0");
  if (d->receptor_mask < 0 || d->receptor_mask > 15) return fail(DTB_EINVAL, "receptor_mask out of 0..15");
  const size_t CM = (size_t)C * M;
  std::vector<uint8_t> used((size_t)nv, 0);
  for (size_t k = 0; k < CM; k++) {
    const int32_t v = d->member_voxel[k];
    if (v < 0 || v >= nv) return fail(DTB_EINVAL, "member voxel out of 0..n_voxels-1");
    if (used[v]) return fail(DTB_EINVAL, "a voxel is the member of two columns or twice of one");
    used[v] = 1;
    if (!std::isfinite(d->theta0[k])) return fail(DTB_EINVAL, "theta0 not finite");
  }
  if (d->target_voxel)
    for (int32_t c = 0; c < C; c++)
      if (d->target_voxel[c] < 0 || d->target_voxel[c] >= nv) return fail(DTB_EINVAL, "target voxel out of range");
  for (size_t k = 0; k < (size_t)nv * 4; k++)
    if (!(d->g_base[k] >= 0.0) || !std::isfinite(d->g_base[k])) return fail(DTB_EINVAL, "g_base must be finite, >= 0");

  dtb_ensemble* ens = new dtb_ensemble();
  ens->net = net;
  ens->tr_steps = d->tr_steps;
  ens->member_voxel.assign(d->member_voxel, d->member_voxel + CM);
  ens->g_base.assign(d->g_base, d->g_base + (size_t)nv * 4);
  const DevNet& g = net->g;
  bool ok = true;
  auto A = [&](size_t bytes) {
    void* p = net->dalloc(bytes);
    if (p) ens->bufs.push_back(p);
    else ok = false;
    return p;
  };
  dtb::EnsDev& e = ens->e;
  e.C = C;
  e.M = M;
  e.member_voxel = (const int32_t*)A(4 * CM);
  e.target_voxel = d->target_voxel ? (const int32_t*)A(4 * (size_t)C) : nullptr;
  e.theta = (float*)A(4 * CM);
  e.g_base = (const double*)A(8 * 4 * (size_t)nv);
  e.cap = (const double*)A(8 * (size_t)nv);
  ens->tile_vox = (int32_t*)A(4 * (size_t)g.nblk);
  if (!ok) {
    delete ens;
    return fail(DTB_ENOMEM, "ensemble buffers");
  }
  e.dt = net->dt;
  e.mask = d->receptor_mask ? d->receptor_mask : 3;
  e.obs_sd_rel = d->obs_sd_rel;
  e.inflation = d->inflation;
  e.key0 = (uint32_t)d->seed;
  e.key1 = (uint32_t)(d->seed >> 32);
  std::vector<double> cap((size_t)nv);
  for (int v = 0; v < nv; v++) cap[v] = net->vparams[(size_t)v * DTB_NP + DTB_P_C];
  // the voxel whose constants tile b copies: that of its first neuron (as upload_consts)
  std::vector<int32_t> tv((size_t)g.nblk);
  size_t v = 0;
  for (int b = 0; b < g.nblk; b++) {
    const int64_t start = (int64_t)b * dtb::kNeuronsPerBlock;
    while (v + 2 < net->vstart.size() && net->vstart[v + 1] <= start) v++;
    tv[b] = (int32_t)v;
  }
  cudaStream_t st = net->stream;
  cudaError_t ce = cudaMemcpyAsync((void*)e.member_voxel, d->member_voxel, 4 * CM, cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess && e.target_voxel)
    ce = cudaMemcpyAsync((void*)e.target_voxel, d->target_voxel, 4 * (size_t)C, cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(e.theta, d->theta0, 4 * CM, cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync((void*)e.g_base, d->g_base, 8 * 4 * (size_t)nv, cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync((void*)e.cap, cap.data(), 8 * (size_t)nv, cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(ens->tile_vox, tv.data(), 4 * tv.size(), cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess)
    ce = dtb::launch_resample(e, (VoxConst*)g.vc, (VoxConst*)g.tile_vc, ens->tile_vox, g.nblk, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) {
    delete ens;
    return cuda_fail(ce, "dtb_ensemble_create");
  }
  ens_mirror(ens, d->theta0);
  *out = ens;
  return DTB_OK;
}

dtb_status dtb_ensemble_destroy(dtb_ensemble* ens) {
  if (!ens) return fail(DTB_EINVAL, "ensemble is NULL");
  delete ens;
  return DTB_OK;
}

dtb_status dtb_ensemble_get_theta(dtb_ensemble* ens, float* theta) {
  if (!ens || !theta) return fail(DTB_EINVAL, "ensemble or theta is NULL");
  DTB_CUDA(cudaMemcpyAsync(theta, ens->e.theta, 4 * (size_t)ens->e.C * ens->e.M, cudaMemcpyDeviceToHost,
                           ens->net->stream));
  DTB_CUDA(cudaStreamSynchronize(ens->net->stream));
  return DTB_OK;
}

dtb_status dtb_assimilate(dtb_ensemble* ens, const float* bold_obs, int32_t n_tr, float* theta_hist, float* hx_hist,
                          float* y_hist) {
  if (!ens) return fail(DTB_EINVAL, "ensemble is NULL");
  if (n_tr < 0) return fail(DTB_EINVAL, "n_tr < 0");
  if (!bold_obs && !ens->e.target_voxel) return fail(DTB_EINVAL, "no bold_obs and no target voxels");
  dtb_net* net = ens->net;
  const DevNet& g = net->g;
  if (net->t % g.bold_every != 0) return fail(DTB_ESTATE, "the network's step count is not a multiple of bold_every");
  if (n_tr == 0) return DTB_OK;
  const int32_t C = ens->e.C, M = ens->e.M, T = ens->tr_steps;
  const size_t CM = (size_t)C * M;
  dtb_status s = ensure_step_off(net, T);
  if (s != DTB_OK) return s;
  s = ensure_graphs(net, T);
  if (s != DTB_OK) return s;
  // per-call device buffers: observations and the histories asked for
  struct Tmp {
    dtb_net* net;
    std::vector<void*> p;
    void* get(size_t bytes) {
      void* q = net->dalloc(bytes);
      if (q) p.push_back(q);
      return q;
    }
    ~Tmp() {
      for (void* q : p) net->dfree(q);
    }
  } tmp{net, {}};
  float* d_obs = bold_obs ? (float*)tmp.get(4 * (size_t)n_tr * C) : nullptr;
  float* d_th = theta_hist ? (float*)tmp.get(4 * (size_t)n_tr * CM) : nullptr;
  float* d_hx = hx_hist ? (float*)tmp.get(4 * (size_t)n_tr * CM) : nullptr;
  float* d_y = y_hist ? (float*)tmp.get(4 * (size_t)n_tr * C) : nullptr;
  if ((bold_obs && !d_obs) || (theta_hist && !d_th) || (hx_hist && !d_hx) || (y_hist && !d_y))
    return fail(DTB_ENOMEM, "dtb_assimilate buffers");
  cudaStream_t st = net->stream;
  if (d_obs) DTB_CUDA(cudaMemcpyAsync(d_obs, bold_obs, 4 * (size_t)n_tr * C, cudaMemcpyHostToDevice, st));
  const int64_t t0 = net->t;
  for (int32_t k = 0; k < n_tr; k++) {
    // predict: one TR of the network (the spike log holds the last TR's raster)
    DTB_CUDA(dtb::launch_begin_call(g, st));
    s = enqueue_call(net, T, true);
    if (s != DTB_OK) return s;
    // analysis on the BOLD sample taken after the TR's last step, then re-sampling
    const int64_t t_end = t0 + (int64_t)(k + 1) * T;
    const int64_t row = (t_end / g.bold_every - 1) % g.bold_cap;
    DTB_CUDA(dtb::launch_enkf_cycle(ens->e, g.bold_log, g.nv, row, d_obs ? d_obs + (size_t)k * C : nullptr,
                                    ens->tr_count + (uint32_t)k, d_th ? d_th + (size_t)k * CM : nullptr,
                                    d_hx ? d_hx + (size_t)k * CM : nullptr, d_y ? d_y + (size_t)k * C : nullptr,
                                    (VoxConst*)g.vc, (VoxConst*)g.tile_vc, ens->tile_vox, g.nblk, st));
  }
  if (d_th) DTB_CUDA(cudaMemcpyAsync(theta_hist, d_th, 4 * (size_t)n_tr * CM, cudaMemcpyDeviceToHost, st));
  if (d_hx) DTB_CUDA(cudaMemcpyAsync(hx_hist, d_hx, 4 * (size_t)n_tr * CM, cudaMemcpyDeviceToHost, st));
  if (d_y) DTB_CUDA(cudaMemcpyAsync(y_hist, d_y, 4 * (size_t)n_tr * C, cudaMemcpyDeviceToHost, st));
  std::vector<float> th(CM);
  DTB_CUDA(cudaMemcpyAsync(th.data(), ens->e.theta, 4 * CM, cudaMemcpyDeviceToHost, st));
  DTB_CUDA(cudaStreamSynchronize(st));
  net->call_t0 = t0 + (int64_t)(n_tr - 1) * T;
  net->call_steps = T;
  net->t = t0 + (int64_t)n_tr * T;
  ens->tr_count += (uint32_t)n_tr;
  ens_mirror(ens, th.data());
  return check_device_error(net);
}

dtb_status dtb_spike_compact(const uint32_t* d_bits, int64_t n, int32_t* d_ids, int32_t* d_count, void* stream) {
  if (!d_bits || !d_ids || !d_count) return fail(DTB_EINVAL, "NULL buffer");
  if (n < 1 || n >= ((int64_t)1 << 30)) return fail(DTB_EINVAL, "n out of 1..2^30-1");
  cudaStream_t st = (cudaStream_t)stream;
  void* scratch = nullptr;
  cudaError_t e = cudaMallocAsync(&scratch, dtb::compact_scratch_bytes(n), st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(DTB_ENOMEM, "scratch of dtb_spike_compact");
  }
  e = dtb::compact_bits(d_bits, n, d_ids, d_count, scratch, st);
  cudaError_t e2 = cudaFreeAsync(scratch, st);
  if (e != cudaSuccess) return cuda_fail(e, "dtb_spike_compact");
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFreeAsync");
  return DTB_OK;
}

dtb_status dtb_test_preset_counters(dtb_net* net, uint64_t value) {
  if (!net) return fail(DTB_EINVAL, "net is NULL");
  if (net->g.mode == dtb::kModeRing) return fail(DTB_ESTATE, "the ring mode keeps no event queues");
  const uint64_t cap = (uint64_t)std::max<int64_t>(net->g.qcap, net->g.mode == dtb::kModeBins ? net->g.bcap : 0);
  if (value < cap || value > ((uint64_t)1 << 62)) return fail(DTB_EINVAL, "value out of capacity .. 2^62");
  DTB_CUDA(dtb::launch_preset_counters(net->g, (unsigned long long)value, net->stream));
  DTB_CUDA(cudaStreamSynchronize(net->stream));
  return DTB_OK;
}

dtb_status dtb_bounded_wait_test(int64_t max_cycles, int32_t arrive) {
  if (max_cycles < 1 || max_cycles > ((int64_t)1 << 32)) return fail(DTB_EINVAL, "max_cycles out of 1..2^32");
  int32_t* d = nullptr;
  DTB_CUDA(cudaMalloc(&d, 4));
  int32_t status = -1;
  cudaError_t e = dtb::launch_bounded_wait(max_cycles, arrive ? 1 : 0, d, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(&status, d, 4, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "dtb_bounded_wait_test");
  if (status != 0) return fail(DTB_ETIMEOUT, "the bounded wait gave up");
  return DTB_OK;
}

dtb_status dtb_philox_device(const uint32_t* d_ctr, const uint32_t* d_key, uint32_t* d_out, int64_t n, void* stream) {
  if (n < 0 || (n > 0 && (!d_ctr || !d_key || !d_out))) return fail(DTB_EINVAL, "bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  DTB_CUDA(dtb::launch_philox(d_ctr, d_key, d_out, n, st));
  DTB_CUDA(cudaStreamSynchronize(st));
  return DTB_OK;
}

}  // extern "C"
