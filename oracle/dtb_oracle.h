/*
 * dtb_oracle.h -- plain single-threaded C oracle of the digital-twin-brain time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may link or call this library.  The product
 * path (the CUDA library) never does, and the two share no source.
 *
 * The same source is compiled twice: with REAL=float (bit-exact reference for
 * the FP32 GPU path) and with REAL=double (bounds the FP32 one-step error).
 * Exported symbols carry the suffix _f32 / _f64 through ORC_FN().
 *
 * What is computed (paper section III.B, Eq. 1, and section VI.A):
 *   leaky integrate-and-fire neurons, four conductance receptors
 *   (AMPA, NMDA, GABAa, GABAb) with jump-and-decay gating, explicit Euler,
 *   threshold / reset / refractory, Poisson external drive, and exact integer
 *   spike delivery with per-voxel-pair delays.  The Balloon-Windkessel BOLD
 *   model (section V.E, which cites Friston 2000) runs in double in both
 *   builds.
 */
#ifndef DTB_ORACLE_H
#define DTB_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#ifdef REAL
#define ORC_CAT2(a, b) a##b
#define ORC_CAT(a, b) ORC_CAT2(a, b)
#define ORC_FN(name) ORC_CAT(name, ORC_SUFFIX)
#endif

/* column order of the per-voxel parameter table (double [n_vox][ORC_NP]) */
enum {
  ORC_P_C = 0,      /* membrane capacitance, nF */
  ORC_P_GL = 1,     /* leak conductance, uS */
  ORC_P_EL = 2,     /* leak reversal, mV */
  ORC_P_VTH = 3,    /* threshold, mV */
  ORC_P_VRESET = 4, /* reset, mV */
  ORC_P_TREF = 5,   /* refractory period, ms */
  ORC_P_G = 6,      /* 6..9: receptor conductances g_u, uS (AMPA, NMDA, GABAa, GABAb) */
  ORC_P_TAU = 10,   /* 10..13: receptor time constants tau_u, ms */
  ORC_P_E = 14,     /* 14..17: receptor reversal potentials E_u, mV */
  ORC_P_IEXT = 18,  /* constant external current, nA */
  ORC_NP = 19
};

/* weight storage formats of the connection table */
enum { ORC_W_INT16 = 0, ORC_W_INT32 = 1, ORC_W_BF16 = 2, ORC_W_INT8 = 3 };

/* Philox counter tags (counter word 3) */
enum { ORC_TAG_DRIVE = 1u, ORC_TAG_INIT = 2u, ORC_TAG_OU = 3u };

/* Network description, shared by the float and double builds.
 * Connections are given in the paper's pull form (section V.D): for every
 * postsynaptic neuron i a fixed number K of inputs, each with its presynaptic
 * neuron, receptor channel and stored weight. */
typedef struct orc_desc {
  int64_t n;                  /* neurons */
  int32_t n_vox;              /* voxels; voxel v owns neurons [voxel_start[v], voxel_start[v+1]) */
  int32_t n_ch;               /* accumulator channels: 2 (E pair, I pair) or 4 (one per receptor) */
  const int64_t* voxel_start; /* [n_vox + 1] */
  const double* vparams;      /* [n_vox][ORC_NP] */
  double dt;                  /* step, ms */
  double nu_ext;              /* Poisson drive rate per neuron, Hz; lambda = nu_ext * dt / 1000 */
  int32_t w_ext;              /* drive weight per event, accumulator units (2^-16) */
  int32_t K;                  /* in-degree */
  const int32_t* pre;         /* [n][K] presynaptic neuron id */
  const uint8_t* cls;         /* [n][K] channel, < n_ch */
  int32_t wfmt;               /* ORC_W_* */
  const void* w;              /* [n][K] stored weights */
  int32_t wshift;             /* left shift into 2^-16 units (INT16, INT32, INT8) */
  const uint8_t* pre_shift;   /* [n] extra per-presynaptic-neuron shift, INT8 only (else NULL) */
  const uint8_t* delay_vv;    /* [n_vox][n_vox], delay in steps from source voxel to target voxel */
  int32_t d_max;              /* every delay lies in 1..d_max; ring depth D = d_max + 1 */
  uint64_t seed;              /* drive key */
  uint64_t init_seed;         /* initial-voltage key */
  double bold_eps, bold_tau_s, bold_tau_f, bold_tau_0, bold_alpha, bold_E0, bold_V0;
  int64_t index_base;         /* global index of neuron 0 in the Philox counters (a slice of a larger
                                 network computes exactly the slice's draws); 0 for a whole network */
  /* Ornstein-Uhlenbeck background current (section III.B: each neuron receives
   * an uncorrelated OU current); off unless ou_enable.  Per step:
   *   V += (dt/C) * I;  I = ((1 - dt/tau) I + mu dt/tau) + sigma sqrt(2 dt/tau) xi
   * xi = (r0 + r1 + r2 + r3 - 2^33) * sqrt(3) * 2^-32 (Irwin-Hall, four uniforms,
   * unit variance) from Philox({i, t_lo, t_hi, OU}, key = seed); I(0) = mu. */
  int32_t ou_enable;
  double ou_mu, ou_sigma, ou_tau; /* nA, nA, ms */
} orc_desc;

/* Philox4x32-10, the counter-based generator of Salmon et al. (SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Poisson inversion thresholds T[m] = floor(2^32 * P(K <= m)), K ~ Poisson(lambda);
 * returns their count M (k = #{m < M : u >= T[m]}), or -1 if cap is too small. */
int orc_poisson_thresholds(double lambda, uint32_t* T, int cap);

/* Poisson counts k of neurons [i0, i0 + cnt) at step t under drive key seed:
 * k = #{m : u >= T[m]}, u = word (i mod 4) of Philox({i/4, t_lo, t_hi, DRIVE}). */
int orc_drive_counts(uint64_t seed, double lambda, int64_t t, int64_t i0, int64_t cnt, int32_t* k);

/* Pull-form delivery (the weighted spike sums of section V.B over the
 * connection tables of section V.D) for m target neurons: acc [m][n_ch][D]
 * (int64, zeroed by the caller) gets, for every input k of target r that
 * spiked at step t (fired[pre] != 0), its accumulator weight at slot
 * (t + delay(vox(pre), vox(tgt[r]))) mod D.  Returns -1 on bad input. */
int orc_deliver_pull(const orc_desc* d, int64_t m, const int64_t* tgt, const int32_t* pre, const uint8_t* cls,
                     const void* w, const uint8_t* fired, int64_t t, int64_t* acc);

/* One stochastic ensemble-Kalman analysis with perturbed observations,
 * local per column (the hierarchical data assimilation of section V.E,
 * reading: one parameter per voxel, observed by that voxel's BOLD).  Column c
 * holds M members: theta [C][M] (updated in place), hx [C][M] the members'
 * predictions, y [C] the observations, sd [C] their noise, eps [C][M]
 * standard-normal perturbations; lambda inflates the posterior anomalies:
 *   K = cov(theta, hx) / (var(hx) + sd^2)   (sample moments, 1/(M-1))
 *   theta_m += K (y + sd eps_m - hx_m);  theta_m = mean + lambda (theta_m - mean)
 * Double precision.  Returns -1 if M < 2. */
int orc_enkf(double* theta, const double* hx, const double* y, const double* sd, const double* eps, int32_t C,
             int32_t M, double lambda);

/* Balloon-Windkessel parameters (Friston et al. 2000). */
typedef struct orc_bold_params { double eps, tau_s, tau_f, tau_0, alpha, E0, V0; } orc_bold_params;

/* n_steps explicit Euler steps of dt_s seconds at constant voxel rates z [nv]
 * (Hz); state [4][nv] = s, f, v, q is updated in place, y [nv] gets the BOLD. */
void orc_bold_integrate(const orc_bold_params* p, int32_t nv, const double* z, int64_t n_steps, double dt_s,
                        double* state, double* y);

/* ---- per-build entry points (REAL = float -> *_f32, REAL = double -> *_f64) ---- */
#ifdef REAL
typedef struct orc_net orc_net;

/* Builds the network; returns NULL on bad input (orc_error() says why). */
orc_net* ORC_FN(orc_create)(const orc_desc* d);
void ORC_FN(orc_destroy)(orc_net* net);

/* Runs n_steps steps.  Spike ids of each step are appended ascending to ids
 * (capacity ids_cap); step_off[s] .. step_off[s+1] delimit step s of this call.
 * Returns the number of spikes, or -1 on overflow of ids / int32 accumulators. */
int64_t ORC_FN(orc_run)(orc_net* net, int64_t n_steps, int32_t* ids, int64_t ids_cap, int64_t* step_off);

/* State access; any pointer may be NULL.  j is [4][n], ring is [D][n_ch][n]. */
void ORC_FN(orc_get_state)(const orc_net* net, REAL* V, REAL* j, uint8_t* ref, int32_t* ring, int64_t* t);
void ORC_FN(orc_set_state)(orc_net* net, const REAL* V, const REAL* j, const uint8_t* ref, const int32_t* ring, int64_t t);

/* BOLD output y [n_vox] and state s, f, v, q [4][n_vox] (double in both builds). */
void ORC_FN(orc_get_bold)(const orc_net* net, double* y, double* state);

/* OU current of every neuron, I [n] (zeros when the OU drive is off). */
void ORC_FN(orc_get_ou)(const orc_net* net, REAL* I);

/* Replaces the receptor conductances g [n_vox][4] (uS) and re-derives constants. */
void ORC_FN(orc_set_g)(orc_net* net, const double* g);

/* Synaptic events delivered so far (one per synapse of each spiking neuron). */
int64_t ORC_FN(orc_events)(const orc_net* net);
#endif

/* Text of the last error of orc_create / orc_run (this thread). */
const char* orc_error(void);

#ifdef __cplusplus
}
#endif
#endif
