/*
 * dtb.h -- C ABI of the GB300 digital-twin-brain step library (libdtb.so).
 *
 * One simulation step of a voxel-structured network of leaky integrate-and-fire
 * neurons with four conductance receptors (AMPA, NMDA, GABAa, GABAb), as in
 * Eq. 1 of arXiv 2308.01241 (section III.B), advanced by explicit Euler
 * (section VI.A), consists of:
 *   1. neuron update: consume the delayed synaptic input of this step, draw the
 *      Poisson external drive, Euler-update the gating variables j_u and the
 *      membrane potential V, apply threshold / reset / refractory period;
 *   2. spike compaction: the ascending list of neurons that fired ("collect
 *      spikes sequence", section V.B);
 *   3. spike delivery: every outgoing synapse of every spiking neuron adds its
 *      weight into an int32 fixed-point accumulator that the target consumes
 *      after the voxel-pair delay (the J sums of section V.B, over the
 *      connection tables of section V.D, stored here as outgoing CSR rows);
 *   4. Balloon-Windkessel hemodynamics per voxel -> BOLD (section V.E, which
 *      cites Friston et al. 2000).
 *
 * Exact operation order (both the library and its test oracle follow it; no
 * fused multiply-add anywhere):
 *   constants per voxel (host, double, rounded once to float):
 *     kL = (dt*gL)/C, kU_u = (dt*g_u)/C, dJ_u = 1 - dt/tau_u, kI = (dt*I_ext)/C,
 *     ref_steps = llround(t_ref/dt), lambda = (nu_ext*dt)/1000
 *   per neuron i (voxel v) at step t, slot = t mod D:
 *     A_c = acc[slot][c][i]; acc[slot][c][i] = 0
 *     u = word (i mod 4) of Philox4x32-10({i/4, t_lo, t_hi, 1}, key = seed)
 *     k = #{m : u >= T_m},  T_m = floor(2^32 * P(Poisson(lambda) <= m))
 *     in = (A_E + k*w_ext, A_E, A_I, A_I)      two channels (E pair, I pair)
 *        | (A_0 + k*w_ext, A_1, A_2, A_3)      four channels (one per receptor)
 *     a_u = float(in_u) * 2^-16
 *     s = 0; for u in AMPA, NMDA, GABAa, GABAb: s = s + (kU_u*j_u)*(V - E_u)
 *     Vn = V - kL*(V - EL); Vn = Vn - s; Vn = Vn + kI
 *     j_u = dJ_u*j_u + a_u
 *     if ref > 0: ref -= 1, Vn = Vreset; elif Vn >= Vth: spike, Vn = Vreset, ref = ref_steps
 *     V = Vn
 *   per spike s, per synapse (tgt, class c, weight w): d = delay[vox(s)][vox(tgt)]
 *     acc[(t + d) mod D][c][tgt] += w_acc   (int32, any order: the sum is exact)
 *   initial state: V = Vreset + (Vth - Vreset) * ((word (i mod 4) of
 *     Philox({i/4, 0, 0, 2}, key = init_seed)) >> 8) * 2^-24; j = 0, ref = 0, acc = 0.
 *   optional Ornstein-Uhlenbeck background current I (section III.B), right
 *   after Vn = Vn + kI, with kO = dt/C per voxel and dI = 1 - dt/tau,
 *   cI = (mu*dt)/tau, sI = sigma*sqrt((2*dt)/tau), each rounded once to float:
 *     Vn = Vn + kO*I
 *     r = Philox4x32-10({i, t_lo, t_hi, 3}, key = seed)
 *     xi = float(r0 + r1 + r2 + r3 - 2^33) * float(sqrt(3) * 2^-32)   (int64 sum)
 *     I = (dI*I + cI) + sI*xi;   I(0) = float(mu)
 *   xi is the centred sum of four uniforms (Irwin-Hall), variance 1.
 *
 * Conventions: every call returns a dtb_status (0 = success, negative = error)
 * and never aborts; dtb_last_error() gives the text of the calling thread's
 * last error.  Units: ms, mV, nF, uS, nA, Hz.  Host arrays passed in are read
 * during the call and stay owned by the caller.
 */
#ifndef DTB_H
#define DTB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dtb_net dtb_net;
typedef int32_t dtb_status;

#define DTB_OK 0
#define DTB_EINVAL (-1)    /* bad argument or inconsistent description */
#define DTB_ENOMEM (-2)    /* device allocation failed */
#define DTB_ECUDA (-3)     /* a CUDA runtime call failed */
#define DTB_EOVERFLOW (-4) /* an int32 accumulator could overflow for this network */
#define DTB_ETIMEOUT (-5)  /* a bounded device wait gave up */
#define DTB_ETRUNC (-6)    /* output buffer or spike log too small; see *n_out */
#define DTB_ESTATE (-7)    /* call not valid in the current state */

/* Columns of the per-voxel parameter table, double [n_voxels][DTB_NP]. */
enum {
  DTB_P_C = 0,       /* membrane capacitance C_i, nF (Eq. 1) */
  DTB_P_GL = 1,      /* leak conductance g_L, uS */
  DTB_P_EL = 2,      /* leak reversal potential E_L, mV */
  DTB_P_VTH = 3,     /* firing threshold V_th, mV */
  DTB_P_VRESET = 4,  /* reset potential V_reset, mV */
  DTB_P_TREF = 5,    /* refractory period T_ref, ms */
  DTB_P_G = 6,       /* 6..9: receptor conductances g_u, uS (AMPA, NMDA, GABAa, GABAb) */
  DTB_P_TAU = 10,    /* 10..13: receptor time constants tau_u, ms */
  DTB_P_E = 14,      /* 14..17: receptor reversal potentials E_u, mV */
  DTB_P_IEXT = 18,   /* constant external current, nA */
  DTB_NP = 19
};

/* Storage format of the synaptic weights; all are converted to int32
 * accumulator units of 2^-16 at delivery. */
enum {
  DTB_W_INT16 = 0, /* int16, w_acc = w << weight_shift (2^-12 storage: shift 4) */
  DTB_W_INT32 = 1, /* int32, w_acc = w << weight_shift (2^-16 storage: shift 0) */
  DTB_W_BF16 = 2,  /* bfloat16 bits, w_acc = round-to-nearest-even(float(w) * 2^16) */
  DTB_W_INT8 = 3   /* int8, w_acc = w << (weight_shift + row_shift[source]) */
};

/* How delivered events wait out their delay (the results are the same bit for bit). */
enum {
  DTB_DELIVER_RING = 0,  /* dense ring acc[D][n_channels][N]: every synapse event is one int32
                            reduction into slot (t + d) mod D */
  DTB_DELIVER_QUEUE = 1, /* delay-1 events are reduced straight into a one-slot accumulator; longer
                            ones are appended (target|class, w_acc) to the queue of their arrival
                            step, staged per batch of work items in shared memory, and each queue
                            is reduced into the accumulator one step before its arrival step */
  DTB_DELIVER_BINS = 2   /* events wait in bins by arrival step parity and target region (4096
                            neurons): delay-1 events are written straight into the bins of step
                            t + 1 (their targets lie in the source's voxel, a few regions, so a
                            warp reserves each region's range with one atomic); longer ones are
                            appended (target|class, weight code) to the queue of their arrival
                            step, which is sorted into the bins one step before that step.  The
                            neuron update adds a region's bin in shared memory: there is no dense
                            accumulator in device memory.  n_neurons <= 2^25 */
};

/* Device allocator hooks: lets the caller (e.g. PyTorch's caching allocator)
 * own every byte of device memory the library uses.  NULL -> cudaMalloc/cudaFree. */
typedef void* (*dtb_alloc_fn)(size_t bytes, void* ctx);
typedef void (*dtb_free_fn)(void* ptr, void* ctx);

typedef struct dtb_network_desc {
  int64_t n_neurons;          /* N, 1 <= N < 2^30 */
  int32_t n_voxels;           /* V >= 1; voxel v owns neurons [voxel_start[v], voxel_start[v+1]) */
  int32_t n_channels;         /* accumulator channels: 2 (class 0 = E -> AMPA+NMDA, class 1 = I ->
                                 GABAa+GABAb) or 4 (class u -> receptor u) */
  const int64_t* voxel_start; /* host [V+1], ascending, 0 .. N */
  const double* voxel_params; /* host [V][DTB_NP] */
  double dt;                  /* time step, ms */
  double nu_ext;              /* Poisson drive rate per neuron, Hz */
  int32_t w_ext;              /* drive weight per Poisson event, 2^-16 units, added to AMPA */
  int32_t weight_format;      /* DTB_W_* */
  int32_t weight_shift;       /* see DTB_W_* */
  int32_t d_max;              /* 1 <= delays <= d_max <= 255; ring depth D = d_max + 1 */
  const int64_t* row_ptr;     /* [N+1] outgoing CSR row pointers (rows by presynaptic neuron) */
  const uint32_t* syn_word;   /* [nnz] target (bits 0-29) | class (bits 30-31) */
  const void* syn_w;          /* [nnz] stored weights, element type per weight_format */
  const uint8_t* row_shift;   /* [N] extra shift per row, DTB_W_INT8 only (may be NULL) */
  int32_t csr_on_device;      /* 0: the three CSR arrays (and row_shift) are host memory and are
                                 copied; 1: they are device memory and are used in place, the
                                 caller keeping them alive until dtb_destroy */
  int32_t bold_every;         /* steps between BOLD samples (8000 = 800 ms at 0.1 ms); 0: none */
  const uint8_t* delay_vv;    /* host [V][V] delay in steps from source voxel to target voxel */
  uint64_t seed;              /* Philox key of the Poisson drive */
  uint64_t init_seed;         /* Philox key of the initial voltages */
  double bold_eps;            /* neural efficacy, 1/(Hz s) */
  double bold_tau_s;          /* signal decay time constant, s */
  double bold_tau_f;          /* flow autoregulation time constant, s */
  double bold_tau_0;          /* mean transit time, s */
  double bold_alpha;          /* Grubb's exponent */
  double bold_E0;             /* resting oxygen extraction fraction */
  double bold_V0;             /* resting blood volume fraction */
  int64_t spike_log_capacity; /* spike ids kept per dtb_step call; 0 -> 2^25 */
  int32_t delivery_mode;      /* DTB_DELIVER_RING, DTB_DELIVER_QUEUE or DTB_DELIVER_BINS */
  int32_t bin_capacity;       /* DTB_DELIVER_BINS: events one region's bin holds per arrival step;
                                 0 -> 4 * event_queue_capacity / regions, at least 4096, at most
                                 event_queue_capacity; rounded up to an odd number of 128-byte lines
                                 (32 events each, 16 with DTB_W_INT32 weights) */
  int64_t event_queue_capacity; /* DTB_DELIVER_QUEUE and _BINS: events one arrival step's queue holds,
                                   0 .. 2^32-64; 0 -> 2N; rounded up to an odd number of 16-event
                                   lines.  Events beyond a queue's or a bin's capacity are added into
                                   a dense spill ring instead (exact, slower), so no capacity changes
                                   the results.  Limit: a queue's and a bin's event counters are
                                   32-bit, so fewer than 2^32 events may be queued for one arrival
                                   step (and one region); more would wrap the counter and overwrite
                                   queued events.  Only a network of more than 2^32 long-delay
                                   synapses whose sources fire in lockstep can reach it */
  void* stream;               /* cudaStream_t all work is queued on; must not be the legacy
                                 default stream (graph capture); NULL -> a library stream */
  dtb_alloc_fn alloc;         /* device allocator, or NULL */
  dtb_free_fn free;
  void* alloc_ctx;
  /* Ornstein-Uhlenbeck background current of every neuron, on top of (or instead
   * of, with nu_ext = 0) the Poisson drive; 0 = off.  Its normals come from the
   * drive's Philox key (seed) with counter tag 3. */
  int32_t ou_enable;
  int32_t reserved1;
  double ou_mu;               /* mean current, nA */
  double ou_sigma;            /* stationary standard deviation, nA, >= 0 */
  double ou_tau;              /* correlation time, ms, > 0 */
} dtb_network_desc;

/* Text of the calling thread's last error. */
const char* dtb_last_error(void);

/* Generate-tables -> load/deploy -> init of section VI.A: validates the
 * description, copies or adopts the synapse table, derives per-voxel
 * constants, checks that no int32 accumulator can overflow (sum of |w| over
 * any neuron's inputs of one channel + max Poisson count * w_ext < 2^31,
 * else DTB_EOVERFLOW) and sets the initial state.  *out is NULL on error. */
dtb_status dtb_create_network(const dtb_network_desc* desc, dtb_net** out);

/* Frees everything the network allocated (not adopted device arrays). */
dtb_status dtb_destroy(dtb_net* net);

/* Runs n_steps steps, 0 <= n_steps <= 2^31 (run loop of section VI.A),
 * queued as CUDA-graph chunks on the network's stream, and waits for them.
 * Resets the spike log.  DTB_ETIMEOUT if a bounded device wait gave up (the
 * state of that step is incomplete; the error word is cleared); DTB_ECUDA on
 * a failed launch. */
dtb_status dtb_step(dtb_net* net, int64_t n_steps);

/* Raster of the last dtb_step call: step_offsets [n_steps+1] (may be NULL)
 * delimits each step's ids, ascending within a step.  *n_out = number of ids
 * recorded.  DTB_ETRUNC if cap < *n_out (nothing copied) or if the spike log
 * overflowed during the call (ids beyond the log capacity were dropped). */
dtb_status dtb_get_spikes(dtb_net* net, int64_t* step_offsets, int32_t* ids, int64_t cap, int64_t* n_out);

/* Current BOLD signal y [V] and state s, f, v, q [4][V] (either may be NULL). */
dtb_status dtb_get_bold(dtb_net* net, float* y, float* state);

/* BOLD samples taken during the last dtb_step call (one every bold_every
 * steps, after the step t with (t + 1) % bold_every == 0): out [cap][V].
 * *n_samples = the number available (the newest 1024 at most; 0 when
 * bold_every is 0); out may be NULL to ask for it; DTB_ETRUNC (nothing
 * copied) if cap < *n_samples. */
dtb_status dtb_get_bold_samples(dtb_net* net, float* out, int64_t cap, int64_t* n_samples);

/* Host copies of the state; any pointer may be NULL.  V [N], j [4][N],
 * ref [N], ring [D][n_channels][N], *t = steps run so far.  In the queue and
 * bins modes the ring is a dense view assembled on the device from the
 * accumulator, queues, bins and spill ring in a temporary allocation of
 * 4*D*n_channels*N bytes (DTB_ENOMEM if it fails). */
dtb_status dtb_get_state(dtb_net* net, float* V, float* j, uint8_t* ref, int32_t* ring, int64_t* t);

/* Overwrites the state (checkpoint restore, tests); NULL leaves a part
 * unchanged; arrays as in dtb_get_state; t >= 0 (else DTB_EINVAL).  In the
 * queue mode the ring is turned back into queues (a temporary allocation as
 * in dtb_get_state), in the bins mode it goes into the spill ring.  The spike
 * log of the last dtb_step call is then empty (no steps). */
dtb_status dtb_set_state(dtb_net* net, const float* V, const float* j, const uint8_t* ref, const int32_t* ring,
                         int64_t t);

/* Re-initialises V, j, ref, the ring, BOLD and t as at creation. */
dtb_status dtb_reset(dtb_net* net);

/* Per-voxel receptor conductances g [V][4] (uS), the parameters that the
 * hierarchical data assimilation of section V.E re-samples; constants are
 * re-derived in double and rounded to float as at creation. */
dtb_status dtb_set_hyperparams(dtb_net* net, const double* g);

/* Counters since creation or dtb_reset: synaptic events delivered (one per
 * synapse of each spike), spikes, steps. */
dtb_status dtb_counters(dtb_net* net, int64_t* events, int64_t* spikes, int64_t* steps);

/* Spikes per voxel since creation or dtb_reset: counts [n_voxels] (int64).
 * Divided by (n_v * steps * dt) these are the population firing rates that
 * the data assimilation of section V.E collects from the simulation. */
dtb_status dtb_get_voxel_spikes(dtb_net* net, int64_t* counts);

/* Runs n_steps steps with one launch per kernel (no graph) and CUDA events
 * around each kernel on the network's stream; ms[5] receives the summed
 * device time of neuron update, compaction, delivery, the fourth kernel
 * (queue drain in the queue mode, binning of the step's arrivals in the bins
 * mode, 0 in the ring mode) and BOLD.  The steps advance the simulation
 * (t += n_steps) and fill the spike log like a dtb_step call. */
dtb_status dtb_profile_steps(dtb_net* net, int64_t n_steps, double* ms);

/* Runs n_steps steps exactly as dtb_step does -- the same pipelined schedule
 * on the same four streams, with the same results -- but issues every launch
 * directly (no CUDA graph) and records a CUDA event right before and right
 * after each kernel on the stream that runs it.  ms[5] receives the summed
 * device time of those launches in the order of dtb_profile_steps (neuron
 * update, compaction, delivery, queue drain or binning, BOLD), launches[5]
 * (may be NULL) how many were timed.  Only the body steps are timed: the
 * first step of a call (its V part) and the closing j-only update are not.
 * A kernel's time here includes what it shares of the GPU with the kernels
 * that overlap it in the schedule, as in a dtb_step call.  The host reads the
 * events of one chunk of steps while the next chunk runs. */
dtb_status dtb_step_timed(dtb_net* net, int64_t n_steps, double* ms, int64_t* launches);

/* Diagnostics for full-size checks without copying the ring to the host.
 * dtb_ring_slot_sums: sums [D][n_channels] (int64) of every ring slot.
 * dtb_get_ring_at: out [m][D][n_channels] = ring[slot][c][idx[r]] for the m
 * host-given neuron ids idx (each < n_neurons, else DTB_EINVAL). */
dtb_status dtb_ring_slot_sums(dtb_net* net, int64_t* sums);
dtb_status dtb_get_ring_at(dtb_net* net, const int64_t* idx, int64_t m, int32_t* out);

/* Autotuner of launch shapes for this network on this GPU: times n_steps
 * steps for every candidate of (neuron-update pipeline stages 2 / 3 / 4,
 * neuron-update CTAs per SM as many as fit / 1 / 2, delivery CTAs per SM
 * 2 / 4 / 6 / 8) and
 * keeps the fastest; chosen[3] (may be NULL) receives those three numbers.
 * The timing steps advance the simulation: call dtb_reset afterwards to start
 * again from the initial state.  The results of later steps do not depend on
 * the shapes chosen (every shape computes the same sums). */
dtb_status dtb_autotune(dtb_net* net, int32_t n_steps, int32_t* chosen);

/* Sets the launch shapes dtb_autotune chooses from: neuron-update pipeline
 * stages (2, 3 or 4; 4 only with 2 channels), neuron-update CTAs per SM (0 =
 * as many as fit, else 1 or 2) and delivery CTAs per SM (1 .. the most that
 * fit).  DTB_EINVAL outside these ranges.  Results do not depend on them. */
dtb_status dtb_set_launch_shapes(dtb_net* net, int32_t update_stages, int32_t update_ctas_per_sm,
                                 int32_t deliver_ctas_per_sm);

/* Sets the order of a step's kernels (the pipelined step of dtb_step):
 *   0: the spike compaction of step t runs after the neuron update of step t
 *      and before that of step t + 1, on the update's stream;
 *   1: the compaction of step t runs beside the neuron update of step t + 1
 *      (the two use alternate copies of the spike bits and block counts), on
 *      the delivery's stream;
 *  -1: chosen by size (the default): 1 for networks of at most 4,096 blocks of
 *      1,024 neurons, whose kernels leave most of the GPU idle, else 0.
 * DTB_EINVAL for other values.  Results do not depend on the schedule: every
 * kernel reads and writes what it does in the plain order of the step (the
 * paper's per-step sequence of update, spike collection and delivery, §V.B).
 * No counterpart in the paper: a GPU scheduling choice. */
dtb_status dtb_set_schedule(dtb_net* net, int32_t mode);

/* *beside = 1 when the compaction runs beside the next update (schedule 1 in
 * effect), else 0.  DTB_EINVAL for NULL pointers. */
dtb_status dtb_get_schedule(dtb_net* net, int32_t* beside);

/* OU current of every neuron, host I [N]: read (DTB_ESTATE when the OU drive
 * is off) and write (a checkpoint holds it too). */
dtb_status dtb_get_ou(dtb_net* net, float* I);
dtb_status dtb_set_ou(dtb_net* net, const float* I);

/* Checkpoint: serialises t, V, j, ref, ring, the BOLD state and (with the OU
 * drive) the OU currents into buf (cap bytes); *n = bytes needed.  DTB_ETRUNC
 * if cap is too small.  The Poisson drive and the OU normals are
 * counter-based, so a restored run continues bit-exactly. */
dtb_status dtb_save_state(dtb_net* net, void* buf, size_t cap, size_t* n);
/* Restores a checkpoint of dtb_save_state; DTB_EINVAL if it is shorter than
 * needed or was written by a network of another size, voxel count, channel
 * count, ring depth or OU setting. */
dtb_status dtb_load_state(dtb_net* net, const void* buf, size_t n);

/* Spike compaction alone ("collect spikes sequence", section V.B), on
 * caller-owned device buffers: d_bits is uint32 [ceil(n/1024) * 32], bit b of
 * word w standing for neuron 32*w + b, every bit at or beyond n zero; d_ids
 * (int32 [n]) receives the ascending ids of the set bits and *d_count (one
 * device int32) their number.  1 <= n < 2^30.  The per-block counts it needs
 * (4 bytes per 1024 neurons + 16) are allocated with cudaMallocAsync on
 * stream and freed there.  Returns after the work is queued and the scratch
 * freed (stream-ordered); DTB_ENOMEM if the allocation fails. */
dtb_status dtb_spike_compact(const uint32_t* d_bits, int64_t n, int32_t* d_ids, int32_t* d_count, void* stream);

/* One ensemble-Kalman analysis step of the hierarchical mesoscopic data
 * assimilation (section V.E; the paper defers its update equations to a
 * companion paper, read here as the stochastic EnKF with perturbed
 * observations, local per column).  All arrays are device memory, members
 * contiguous per column: theta [C][M] parameters (e.g. the log conductance
 * gain of one voxel), updated in place; hx [C][M] the members' predictions of
 * the observation (the voxel's BOLD at this TR); y [C] observations; obs_sd
 * [C] their noise; eps [C][M] standard-normal perturbations.  Per column:
 *   K = cov(theta, hx) / (var(hx) + sd^2)     (sample moments, 1/(M-1))
 *   theta_m += K (y + sd * eps_m - hx_m);  then posterior anomalies *= inflation.
 * FP32.  Needs M >= 2; waits for the work on stream before returning.  The
 * analysis alone, for predictions that come from elsewhere (the learned
 * surrogate of dtb_surrogate.h); dtb_assimilate runs the whole cycle. */
dtb_status dtb_enkf_analysis(float* d_theta, const float* d_hx, const float* d_y, const float* d_obs_sd,
                             const float* d_eps, int32_t n_columns, int32_t n_members, float inflation,
                             void* stream);

/* The assimilation cycle of the hierarchical mesoscopic data assimilation
 * (section V.E) on one network: members are voxels of the network (an
 * ensemble of member networks merged into one block-diagonal network), each
 * column c is one assimilated parameter theta (the log gain of a voxel's
 * receptor conductances) held by M members, observed through one BOLD value
 * per TR.  Per TR, all on the device, on the network's stream:
 *   predict:  the network runs tr_steps steps (its BOLD is sampled at the
 *             TR's end);
 *   gather:   hx[c][m] = BOLD of member_voxel[c][m], y[c] = bold_obs[tr][c]
 *             or the BOLD of target_voxel[c];
 *   analysis: the stochastic EnKF of dtb_enkf_analysis, local per column,
 *             with sd = obs_sd_rel * max(|y|, 1e-4) and perturbations
 *             eps[c][m] = Irwin-Hall(4) normal of Philox4x32-10 counter
 *             {m, c, TR index, 4} under key seed: (r0 + r1 + r2 + r3 - 2^33)
 *             * float(sqrt(3) * 2^-32) (the TR index counts every TR this
 *             ensemble has analysed);
 *   re-sampling: each member voxel's receptors in receptor_mask get the
 *             conductance g_base * exp(theta), and its constants are derived
 *             as at creation (double, rounded once to float; exp in double on
 *             the device, within an ulp of the host's, so a constant can
 *             differ from dtb_set_hyperparams' in its last float bit, rarely).
 * Columns are independent; the members of a column need not be in one
 * group.  The ensemble holds device buffers from the network's allocator and
 * must be destroyed before the network. */
typedef struct dtb_ensemble dtb_ensemble;

typedef struct dtb_ensemble_desc {
  int32_t n_columns;            /* C >= 1 */
  int32_t n_members;            /* M >= 2; C * M <= 2^28 */
  const int32_t* member_voxel;  /* host [C][M]: the voxel that member m of column c is; no voxel twice */
  const int32_t* target_voxel;  /* host [C] or NULL: the voxel whose BOLD observes column c (used when
                                   dtb_assimilate gets no bold_obs) */
  const float* theta0;          /* host [C][M]: initial parameters, applied at creation */
  const double* g_base;         /* host [n_voxels][4]: conductances (uS) that exp(theta) multiplies */
  int32_t receptor_mask;        /* receptors the gain scales, bit u = receptor u; 0 -> AMPA and NMDA */
  int32_t tr_steps;             /* steps per TR, a positive multiple of the network's bold_every */
  float obs_sd_rel;             /* observation noise relative to |y|, >= 0 */
  float inflation;              /* multiplicative inflation of the posterior anomalies, > 0 */
  uint64_t seed;                /* Philox key of the observation perturbations */
} dtb_ensemble_desc;

/* Validates the description (DTB_EINVAL with a message: sizes, voxel ids,
 * a voxel used twice, tr_steps, finite values), copies it to the device and
 * writes the members' initial conductances into the network's constants. */
dtb_status dtb_ensemble_create(dtb_net* net, const dtb_ensemble_desc* desc, dtb_ensemble** out);
dtb_status dtb_ensemble_destroy(dtb_ensemble* ens);
/* Current parameters, host [C][M]. */
dtb_status dtb_ensemble_get_theta(dtb_ensemble* ens, float* theta);

/* Runs n_tr >= 0 assimilation cycles (above).  bold_obs: host [n_tr][C]
 * observations, or NULL to observe the target voxels.  Optional host outputs
 * per TR: theta_hist [n_tr][C][M] the parameters after the analysis, hx_hist
 * [n_tr][C][M] the members' predictions, y_hist [n_tr][C] the observations.
 * The network's step count must be a multiple of bold_every (DTB_ESTATE);
 * the spike log then holds the last TR's raster.  One synchronisation at the
 * end; DTB_ETIMEOUT / DTB_ECUDA as in dtb_step. */
dtb_status dtb_assimilate(dtb_ensemble* ens, const float* bold_obs, int32_t n_tr, float* theta_hist,
                          float* hx_hist, float* y_hist);

/* Largest n that dtb_spike_compact_noalloc accepts (its fixed scratch is
 * 4 bytes per 1024 neurons of this many, plus 16: about 1 MiB). */
#define DTB_NOALLOC_MAX_NEURONS (1 << 28)

/* dtb_spike_compact for callers that cannot allocate device memory while it
 * runs: a host framework that owns the whole device heap through its own
 * pool, a hard real-time loop that may not call cudaMalloc/cudaFree (both can
 * block or synchronise the device), a plugin that is handed buffers but has
 * no allocator.  The paper has no counterpart; this is an interface variant.
 * Same arguments, layout and result as dtb_spike_compact, for
 * 1 <= n <= DTB_NOALLOC_MAX_NEURONS (else DTB_EINVAL with a message).
 * It allocates and frees nothing: its scratch is one fixed device array of
 * about 1 MiB in the library, held by every GPU that loads the library until
 * the process exits.  Every call looks up the array's address on the current
 * device (a host-side lookup that allocates nothing), so the entry point
 * stays valid after a device reset; the first call on a device may load the
 * library's device code, so make that first call before any stream capture.
 * All calls share the one array, so calls that overlap on
 * the GPU (different streams, or different host threads, at the same time)
 * race and corrupt each other's results; serialise them.  The parts that
 * must start at zero are cleared by every call. */
dtb_status dtb_spike_compact_noalloc(const uint32_t* d_bits, int64_t n, int32_t* d_ids, int32_t* d_count,
                                     void* stream);

/* Test hook of the event counters (event-queue and bins modes; DTB_ESTATE in
 * the ring mode): the unused entries of every queue and bin are filled with
 * placeholder events of weight 0 and every queue and bin count is set to
 * value (from the largest capacity up to 2^62, else DTB_EINVAL), as if that
 * many events had been queued.  Every later reservation then lies beyond the
 * capacity and its events go to the spill ring, so the results stay exact.
 * A queue or bin counter that wrapped (at 2^32, say) would instead hand out
 * positions inside the queue again and overwrite queued events.  The paper
 * has no counterpart; it exists to test that the counters cannot wrap. */
dtb_status dtb_test_preset_counters(dtb_net* net, uint64_t value);

/* Test of the device-side failure path: one thread waits on a shared-memory
 * mbarrier with the neuron update's bounded wait, limited to max_cycles SM
 * cycles (1 .. 2^32).  arrive = 0: nothing arrives, the wait gives up and the
 * call returns DTB_ETIMEOUT with the context still usable; arrive != 0: the
 * barrier completes first and the call returns DTB_OK. */
dtb_status dtb_bounded_wait_test(int64_t max_cycles, int32_t arrive);

/* Device Philox4x32-10 of n counters (each 4 words) under n keys (2 words
 * each); all three arrays are device memory.  For tests of the generator. */
dtb_status dtb_philox_device(const uint32_t* d_ctr, const uint32_t* d_key, uint32_t* d_out, int64_t n,
                             void* stream);

#ifdef __cplusplus
}
#endif
#endif
