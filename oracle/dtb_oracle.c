/*
 * dtb_oracle.c -- plain, slow, single-threaded C oracle of one simulation step.
 *
 * TEST INFRASTRUCTURE ONLY: linked by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  It shares no
 * source with the CUDA library.
 *
 * Build: cc -O2 -ffp-contract=off -fno-fast-math -DREAL=float  -DORC_SUFFIX=_f32
 *        cc -O2 -ffp-contract=off -fno-fast-math -DREAL=double -DORC_SUFFIX=_f64
 * (no FMA contraction: every multiply and add below is rounded on its own).
 *
 * Parity is pinned by tests/test_oracle_*.py: closed forms of the Euler map,
 * the interspike interval, the gating decay per receptor and class, the
 * relaxation to the conductance-weighted reversal potential under frozen
 * gating, the refractory hold and the >= threshold; the Poisson drive's
 * routing and law; the initial state's law; conservation of delivered
 * weight and hand-worked bf16 / int8 weight values; brute force on 10-neuron
 * nets; the published Philox known answers and cuRAND's Philox; exact
 * Poisson thresholds; the Balloon-Windkessel input, steady state and linear
 * flow response; global-index slices.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "dtb_oracle.h"

typedef REAL real;

static _Thread_local char g_err[256];
static void set_err(const char* msg) { snprintf(g_err, sizeof g_err, "%s", msg); }
const char* orc_error(void) { return g_err; }

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11).  Ten rounds; each round multiplies counter     */
/* words 0 and 2 by the round multipliers, mixes the high halves with words */
/* 1 and 3 and the key, and then bumps the key by the Weyl constants.       */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t MUL0 = 0xD2511F53u, MUL1 = 0xCD9E8D57u;
  const uint32_t WEYL0 = 0x9E3779B9u, WEYL1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; round++) {
    uint64_t p0 = (uint64_t)MUL0 * c0;
    uint64_t p1 = (uint64_t)MUL1 * c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += WEYL0;
    k1 += WEYL1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------ */
/* Poisson drive by inversion.  F(m) = P(K <= m) is summed term by term in  */
/* double (p_0 = exp(-lambda), p_m = p_{m-1} * lambda / m) and the threshold */
/* list stops at the first m whose floor(F(m) * 2^32) reaches 2^32 - 1.     */
/* ------------------------------------------------------------------------ */
int orc_poisson_thresholds(double lambda, uint32_t* T, int cap) {
  const double two32 = 4294967296.0;
  if (!(lambda >= 0.0)) return -1;
  double p = exp(-lambda);
  double F = p;
  int M = 0;
  for (int m = 0;; m++) {
    if (m > 0) {
      p = p * lambda / (double)m;
      F = F + p;
    }
    double x = floor(F * two32);
    if (x >= two32 - 1.0) break;
    if (M >= cap) return -1;
    T[M++] = (uint32_t)x;
    if (m > 1000) return -1;
  }
  return M;
}

/* ------------------------------------------------------------------------ */
/* network                                                                   */
/* ------------------------------------------------------------------------ */
struct orc_net {
  int64_t n;
  int32_t nv, nch, D, M;
  int64_t t;
  int32_t* vox;          /* [n] voxel of each neuron */
  int64_t* vstart;       /* [nv+1] */
  /* per-voxel constants, derived in double and rounded to REAL */
  real *kL, *EL, *kI, *Vth, *Vreset, *kU, *dJ, *E; /* kU, dJ, E are [nv][4] */
  int32_t* ref_steps;
  double* vparams;       /* private copy, [nv][ORC_NP] */
  double dt;
  /* outgoing synapse lists, built here from the pull form */
  int64_t* out_ptr;      /* [n+1] */
  int32_t* out_tgt;
  uint8_t* out_cls;
  int32_t* out_w;        /* accumulator units, 2^-16 */
  uint8_t* out_d;
  /* state */
  int32_t* ring;         /* [D][nch][n] */
  real *V, *j;           /* j is [4][n] */
  uint8_t* ref;
  /* drive */
  uint32_t T[64];
  uint32_t key[2];
  int32_t w_ext;
  int64_t base;          /* global index of neuron 0 */
  int64_t events;
  /* BOLD, double in both builds */
  double *bs, *bf, *bv, *bq, *by;
  double eps, tau_s, tau_f, tau_0, alpha, E0, V0b;
  int32_t* vcount;       /* spikes per voxel in the current step */
  int32_t* spk;          /* [n] spike ids of the current step, ascending */
  /* OU drive */
  int32_t ou;
  real *Iou, *kO;        /* [n] current; [nv] dt / C */
  real ou_d, ou_c, ou_s, ou_xi_scale;
};

static void* xcalloc(size_t n, size_t sz) { return calloc(n ? n : 1, sz); }

/* Per-voxel constants of the Euler map of Eq. 1 (reading: I_sum enters with
 * a minus sign, decay factor 1 - dt/tau):
 *   kL = dt*gL/C, kU_u = dt*g_u/C, dJ_u = 1 - dt/tau_u, kI = dt*I_ext/C,
 * each evaluated in double and rounded once to REAL. */
static void derive_constants(orc_net* net) {
  const double dt = net->dt;
  for (int32_t v = 0; v < net->nv; v++) {
    const double* P = net->vparams + (size_t)v * ORC_NP;
    net->kL[v] = (real)((dt * P[ORC_P_GL]) / P[ORC_P_C]);
    net->EL[v] = (real)P[ORC_P_EL];
    net->kI[v] = (real)((dt * P[ORC_P_IEXT]) / P[ORC_P_C]);
    net->Vth[v] = (real)P[ORC_P_VTH];
    net->Vreset[v] = (real)P[ORC_P_VRESET];
    net->ref_steps[v] = (int32_t)llround(P[ORC_P_TREF] / dt);
    for (int u = 0; u < 4; u++) {
      net->kU[v * 4 + u] = (real)((dt * P[ORC_P_G + u]) / P[ORC_P_C]);
      net->dJ[v * 4 + u] = (real)(1.0 - dt / P[ORC_P_TAU + u]);
      net->E[v * 4 + u] = (real)P[ORC_P_E + u];
    }
  }
}

/* Stored weight -> accumulator units (2^-16).  BF16: the float value times
 * 2^16 rounded to nearest even; integer formats: shifted left. */
static int decode_weight(const orc_desc* d, int64_t idx, int32_t pre, int32_t* out) {
  int64_t w;
  switch (d->wfmt) {
    case ORC_W_INT16: w = (int64_t)((const int16_t*)d->w)[idx] * ((int64_t)1 << d->wshift); break;
    case ORC_W_INT32: w = (int64_t)((const int32_t*)d->w)[idx] * ((int64_t)1 << d->wshift); break;
    case ORC_W_INT8: {
      int s = d->wshift + (d->pre_shift ? d->pre_shift[pre] : 0);
      w = (int64_t)((const int8_t*)d->w)[idx] * ((int64_t)1 << s);
      break;
    }
    case ORC_W_BF16: {
      uint32_t bits = (uint32_t)((const uint16_t*)d->w)[idx] << 16;
      float f;
      memcpy(&f, &bits, 4);
      float x = f * 65536.0f;
      if (!(fabsf(x) < 2147483520.0f)) return -1;
      w = (int64_t)lrintf(x);
      break;
    }
    default: return -1;
  }
  if (w > INT32_MAX || w < INT32_MIN) return -1;
  *out = (int32_t)w;
  return 0;
}

void ORC_FN(orc_destroy)(orc_net* net) {
  if (!net) return;
  free(net->vox); free(net->vstart);
  free(net->kL); free(net->EL); free(net->kI); free(net->Vth); free(net->Vreset);
  free(net->kU); free(net->dJ); free(net->E); free(net->ref_steps); free(net->vparams);
  free(net->out_ptr); free(net->out_tgt); free(net->out_cls); free(net->out_w); free(net->out_d);
  free(net->ring); free(net->V); free(net->j); free(net->ref);
  free(net->bs); free(net->bf); free(net->bv); free(net->bq); free(net->by); free(net->vcount); free(net->spk);
  free(net->Iou); free(net->kO);
  free(net);
}

orc_net* ORC_FN(orc_create)(const orc_desc* d) {
  if (!d || d->n < 0 || d->n_vox < 1 || (d->n_ch != 2 && d->n_ch != 4) || d->K < 0 ||
      d->d_max < 1 || d->d_max > 255 || !(d->dt > 0.0)) {
    set_err("bad sizes");
    return NULL;
  }
  if (d->voxel_start[0] != 0 || d->voxel_start[d->n_vox] != d->n) {
    set_err("voxel_start must run from 0 to n");
    return NULL;
  }
  for (int32_t v = 0; v < d->n_vox; v++)
    if (d->voxel_start[v + 1] < d->voxel_start[v]) { set_err("voxel_start not ascending"); return NULL; }
  orc_net* net = (orc_net*)calloc(1, sizeof(orc_net));
  const int64_t n = d->n;
  const int32_t nv = d->n_vox;
  net->n = n; net->nv = nv; net->nch = d->n_ch; net->D = d->d_max + 1; net->dt = d->dt;
  net->vox = (int32_t*)xcalloc((size_t)n, 4);
  net->vstart = (int64_t*)xcalloc((size_t)nv + 1, 8);
  memcpy(net->vstart, d->voxel_start, ((size_t)nv + 1) * 8);
  for (int32_t v = 0; v < nv; v++)
    for (int64_t i = d->voxel_start[v]; i < d->voxel_start[v + 1]; i++) net->vox[i] = v;
  net->kL = (real*)xcalloc(nv, sizeof(real)); net->EL = (real*)xcalloc(nv, sizeof(real));
  net->kI = (real*)xcalloc(nv, sizeof(real)); net->Vth = (real*)xcalloc(nv, sizeof(real));
  net->Vreset = (real*)xcalloc(nv, sizeof(real));
  net->kU = (real*)xcalloc((size_t)nv * 4, sizeof(real));
  net->dJ = (real*)xcalloc((size_t)nv * 4, sizeof(real));
  net->E = (real*)xcalloc((size_t)nv * 4, sizeof(real));
  net->ref_steps = (int32_t*)xcalloc(nv, 4);
  net->vparams = (double*)xcalloc((size_t)nv * ORC_NP, 8);
  memcpy(net->vparams, d->vparams, (size_t)nv * ORC_NP * 8);
  derive_constants(net);
  for (int32_t v = 0; v < nv; v++)
    if (net->ref_steps[v] < 0 || net->ref_steps[v] > 255) { set_err("refractory steps out of 0..255"); goto fail; }

  /* outgoing lists: count, prefix, fill in (i, k) order */
  const int64_t K = d->K;
  net->out_ptr = (int64_t*)xcalloc((size_t)n + 1, 8);
  for (int64_t i = 0; i < n; i++)
    for (int64_t k = 0; k < K; k++) {
      int32_t p = d->pre[i * K + k];
      if (p < 0 || p >= n) { set_err("presynaptic id out of range"); goto fail; }
      if (d->cls[i * K + k] >= d->n_ch) { set_err("channel out of range"); goto fail; }
      net->out_ptr[p + 1]++;
    }
  for (int64_t i = 0; i < n; i++) net->out_ptr[i + 1] += net->out_ptr[i];
  {
    const int64_t nnz = net->out_ptr[n];
    net->out_tgt = (int32_t*)xcalloc((size_t)nnz, 4);
    net->out_cls = (uint8_t*)xcalloc((size_t)nnz, 1);
    net->out_w = (int32_t*)xcalloc((size_t)nnz, 4);
    net->out_d = (uint8_t*)xcalloc((size_t)nnz, 1);
    int64_t* fill = (int64_t*)xcalloc((size_t)n, 8);
    for (int64_t i = 0; i < n; i++)
      for (int64_t k = 0; k < K; k++) {
        int32_t p = d->pre[i * K + k];
        int64_t e = net->out_ptr[p] + fill[p]++;
        int32_t w;
        if (decode_weight(d, i * K + k, p, &w) != 0) { free(fill); set_err("weight out of range"); goto fail; }
        uint8_t dd = d->delay_vv[(size_t)net->vox[p] * nv + net->vox[i]];
        if (dd < 1 || dd > d->d_max) { free(fill); set_err("delay out of 1..d_max"); goto fail; }
        net->out_tgt[e] = (int32_t)i;
        net->out_cls[e] = d->cls[i * K + k];
        net->out_w[e] = w;
        net->out_d[e] = dd;
      }
    free(fill);
  }

  /* state: V0 = Vreset + (Vth - Vreset) * u, u = (philox word >> 8) * 2^-24 */
  net->ring = (int32_t*)xcalloc((size_t)net->D * net->nch * (size_t)n, 4);
  net->V = (real*)xcalloc((size_t)n, sizeof(real));
  net->j = (real*)xcalloc((size_t)n * 4, sizeof(real));
  net->ref = (uint8_t*)xcalloc((size_t)n, 1);
  net->spk = (int32_t*)xcalloc((size_t)n, 4);
  {
    const uint32_t ikey[2] = {(uint32_t)d->init_seed, (uint32_t)(d->init_seed >> 32)};
    for (int64_t i = 0; i < n; i++) {
      const int64_t gi = i + d->index_base;
      const uint32_t ctr[4] = {(uint32_t)(gi >> 2), 0u, 0u, ORC_TAG_INIT};
      uint32_t r[4];
      orc_philox4x32_10(ctr, ikey, r);
      real u = (real)(r[gi & 3] >> 8) * (real)(1.0 / 16777216.0);
      int32_t v = net->vox[i];
      real span = net->Vth[v] - net->Vreset[v];
      net->V[i] = net->Vreset[v] + span * u;
    }
  }
  /* drive */
  net->M = orc_poisson_thresholds((d->nu_ext * d->dt) / 1000.0, net->T, 64);
  if (net->M < 0) { set_err("bad drive rate"); goto fail; }
  net->key[0] = (uint32_t)d->seed;
  net->key[1] = (uint32_t)(d->seed >> 32);
  net->w_ext = d->w_ext;
  net->base = d->index_base;
  /* OU constants, double rounded once to REAL */
  net->ou = d->ou_enable != 0;
  net->Iou = (real*)xcalloc((size_t)n, sizeof(real));
  net->kO = (real*)xcalloc(nv, sizeof(real));
  if (net->ou) {
    if (!(d->ou_tau > 0.0) || !(d->ou_sigma >= 0.0)) { set_err("OU drive needs tau > 0, sigma >= 0"); goto fail; }
    net->ou_d = (real)(1.0 - d->dt / d->ou_tau);
    net->ou_c = (real)((d->ou_mu * d->dt) / d->ou_tau);
    net->ou_s = (real)(d->ou_sigma * sqrt((2.0 * d->dt) / d->ou_tau));
    net->ou_xi_scale = (real)(1.7320508075688772 / 4294967296.0);
    for (int32_t v = 0; v < nv; v++) net->kO[v] = (real)(d->dt / d->vparams[(size_t)v * ORC_NP + ORC_P_C]);
    for (int64_t i = 0; i < n; i++) net->Iou[i] = (real)d->ou_mu;
  }
  if (net->base < 0 || (net->base & 3) != 0) { set_err("index_base must be a multiple of 4"); goto fail; }
  /* BOLD at rest: s = 0, f = v = q = 1 */
  net->bs = (double*)xcalloc(nv, 8); net->bf = (double*)xcalloc(nv, 8);
  net->bv = (double*)xcalloc(nv, 8); net->bq = (double*)xcalloc(nv, 8);
  net->by = (double*)xcalloc(nv, 8); net->vcount = (int32_t*)xcalloc(nv, 4);
  for (int32_t v = 0; v < nv; v++) { net->bf[v] = 1.0; net->bv[v] = 1.0; net->bq[v] = 1.0; }
  net->eps = d->bold_eps; net->tau_s = d->bold_tau_s; net->tau_f = d->bold_tau_f;
  net->tau_0 = d->bold_tau_0; net->alpha = d->bold_alpha; net->E0 = d->bold_E0; net->V0b = d->bold_V0;
  return net;
fail:
  ORC_FN(orc_destroy)(net);
  return NULL;
}

/* Balloon-Windkessel model of Friston et al. 2000, one explicit Euler step of
 * dt_s seconds driven by the voxel rate z (Hz):
 *   ds/dt = eps*z - s/tau_s - (f - 1)/tau_f
 *   df/dt = s
 *   tau_0 dv/dt = f - v^(1/alpha)
 *   tau_0 dq/dt = f*E(f)/E0 - v^(1/alpha)*q/v,   E(f) = 1 - (1 - E0)^(1/f)
 *   y = V0*(k1*(1 - q) + k2*(1 - q/v) + k3*(1 - v)),  k1 = 7*E0, k2 = 2, k3 = 2*E0 - 0.2
 * All four derivatives are taken at the old state. */
static void bold_euler(const orc_bold_params* p, double* ps, double* pf, double* pv, double* pq, double* py,
                       double z, double dt_s) {
  double s = *ps, f = *pf, vv = *pv, q = *pq;
  double fout = pow(vv, 1.0 / p->alpha);
  double Ef = 1.0 - pow(1.0 - p->E0, 1.0 / f);
  double ds = p->eps * z - s / p->tau_s - (f - 1.0) / p->tau_f;
  double df = s;
  double dv = (f - fout) / p->tau_0;
  double dq = (f * Ef / p->E0 - fout * q / vv) / p->tau_0;
  s = s + dt_s * ds;
  f = f + dt_s * df;
  vv = vv + dt_s * dv;
  q = q + dt_s * dq;
  *ps = s; *pf = f; *pv = vv; *pq = q;
  double k1 = 7.0 * p->E0, k2 = 2.0, k3 = 2.0 * p->E0 - 0.2;
  *py = p->V0 * (k1 * (1.0 - q) + k2 * (1.0 - q / vv) + k3 * (1.0 - vv));
}

void orc_bold_integrate(const orc_bold_params* p, int32_t nv, const double* z, int64_t n_steps, double dt_s,
                        double* state, double* y) {
  for (int64_t t = 0; t < n_steps; t++)
    for (int32_t v = 0; v < nv; v++)
      bold_euler(p, &state[v], &state[nv + v], &state[2 * nv + v], &state[3 * nv + v], &y[v], z[v], dt_s);
}

static void bold_step(orc_net* net, int32_t v, double z, double dt_s) {
  const orc_bold_params p = {net->eps, net->tau_s, net->tau_f, net->tau_0, net->alpha, net->E0, net->V0b};
  bold_euler(&p, &net->bs[v], &net->bf[v], &net->bv[v], &net->bq[v], &net->by[v], z, dt_s);
}

static int32_t voxel_search(const int64_t* vstart, int32_t nv, int64_t i) {
  int32_t lo = 0, hi = nv - 1;
  while (lo < hi) {
    int32_t mid = (lo + hi + 1) / 2;
    if (vstart[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

int orc_deliver_pull(const orc_desc* d, int64_t m, const int64_t* tgt, const int32_t* pre, const uint8_t* cls,
                     const void* w, const uint8_t* fired, int64_t t, int64_t* acc) {
  const int32_t D = d->d_max + 1;
  orc_desc one = *d;
  one.w = w;
  for (int64_t r = 0; r < m; r++) {
    const int32_t vt = voxel_search(d->voxel_start, d->n_vox, tgt[r]);
    for (int32_t k = 0; k < d->K; k++) {
      const int64_t e = r * d->K + k;
      const int32_t p = pre[e];
      if (p < 0 || p >= d->n || cls[e] >= d->n_ch) return -1;
      if (!fired[p]) continue;
      const int32_t vs = voxel_search(d->voxel_start, d->n_vox, p);
      const int32_t dd = d->delay_vv[(int64_t)vs * d->n_vox + vt];
      int32_t wa;
      if (decode_weight(&one, e, p, &wa) != 0) return -1;
      acc[(r * d->n_ch + cls[e]) * D + (t + dd) % D] += wa;
    }
  }
  return 0;
}

int orc_enkf(double* theta, const double* hx, const double* y, const double* sd, const double* eps, int32_t C,
             int32_t M, double lambda) {
  if (M < 2) return -1;
  for (int32_t c = 0; c < C; c++) {
    double* th = theta + (size_t)c * M;
    const double* h = hx + (size_t)c * M;
    const double* e = eps + (size_t)c * M;
    double mt = 0.0, mh = 0.0;
    for (int32_t m = 0; m < M; m++) {
      mt += th[m];
      mh += h[m];
    }
    mt /= M;
    mh /= M;
    double cth = 0.0, chh = 0.0;
    for (int32_t m = 0; m < M; m++) {
      cth += (th[m] - mt) * (h[m] - mh);
      chh += (h[m] - mh) * (h[m] - mh);
    }
    cth /= (M - 1);
    chh /= (M - 1);
    const double K = cth / (chh + sd[c] * sd[c]);
    double ma = 0.0;
    for (int32_t m = 0; m < M; m++) {
      th[m] = th[m] + K * (y[c] + sd[c] * e[m] - h[m]);
      ma += th[m];
    }
    ma /= M;
    for (int32_t m = 0; m < M; m++) th[m] = ma + lambda * (th[m] - ma);
  }
  return 0;
}

/* Poisson count of one neuron-step from its Philox word. */
static int32_t poisson_k(const uint32_t* T, int32_t M, uint32_t u) {
  int32_t k = 0;
  for (int32_t m = 0; m < M; m++) k += (u >= T[m]) ? 1 : 0;
  return k;
}

int orc_drive_counts(uint64_t seed, double lambda, int64_t t, int64_t i0, int64_t cnt, int32_t* k) {
  uint32_t T[64];
  const int M = orc_poisson_thresholds(lambda, T, 64);
  if (M < 0) return -1;
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int64_t i = i0; i < i0 + cnt; i++) {
    const uint32_t ctr[4] = {(uint32_t)(i >> 2), (uint32_t)t, (uint32_t)((uint64_t)t >> 32), ORC_TAG_DRIVE};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    k[i - i0] = poisson_k(T, M, r[i & 3]);
  }
  return 0;
}

int64_t ORC_FN(orc_run)(orc_net* net, int64_t n_steps, int32_t* ids, int64_t ids_cap, int64_t* step_off) {
  const int64_t n = net->n;
  const int32_t nch = net->nch, D = net->D;
  const real SC = (real)(1.0 / 65536.0);
  int64_t n_out = 0;
  if (step_off) step_off[0] = 0;
  for (int64_t s = 0; s < n_steps; s++) {
    const int64_t t = net->t;
    const int64_t slot = t % D;
    int32_t* cur = net->ring + (size_t)slot * nch * (size_t)n;
    int64_t n_spk = 0;
    uint32_t r[4] = {0, 0, 0, 0};
    for (int32_t v = 0; v < net->nv; v++) net->vcount[v] = 0;

    /* 1. neuron update, Eq. 1 by explicit Euler, neurons in ascending order */
    for (int64_t i = 0; i < n; i++) {
      const int32_t v = net->vox[i];
      int32_t A[4] = {0, 0, 0, 0};
      for (int32_t c = 0; c < nch; c++) {
        A[c] = cur[(size_t)c * n + i];
        cur[(size_t)c * n + i] = 0;
      }
      /* Poisson count k from word (gi mod 4) of Philox({gi/4, t_lo, t_hi, DRIVE}), gi = global index */
      const int64_t gi = i + net->base;
      if ((i & 3) == 0) {
        const uint32_t ctr[4] = {(uint32_t)(gi >> 2), (uint32_t)t, (uint32_t)((uint64_t)t >> 32), ORC_TAG_DRIVE};
        orc_philox4x32_10(ctr, net->key, r);
      }
      const int32_t k = poisson_k(net->T, net->M, r[gi & 3]);
      /* arrivals per receptor: E pair -> AMPA, NMDA; I pair -> GABAa, GABAb */
      int64_t in[4];
      if (nch == 2) {
        in[0] = (int64_t)A[0] + (int64_t)k * net->w_ext;
        in[1] = A[0];
        in[2] = A[1];
        in[3] = A[1];
      } else {
        in[0] = (int64_t)A[0] + (int64_t)k * net->w_ext;
        in[1] = A[1];
        in[2] = A[2];
        in[3] = A[3];
      }
      if (in[0] > INT32_MAX || in[0] < INT32_MIN) { set_err("drive overflows int32"); return -1; }
      real a[4];
      for (int u4 = 0; u4 < 4; u4++) a[u4] = (real)(int32_t)in[u4] * SC;

      const real Vold = net->V[i];
      real syn = (real)0;
      for (int u4 = 0; u4 < 4; u4++) {
        real x = Vold - net->E[v * 4 + u4];
        real y = net->kU[v * 4 + u4] * net->j[(size_t)u4 * n + i];
        syn = syn + y * x;
      }
      real Vn = Vold - net->kL[v] * (Vold - net->EL[v]);
      Vn = Vn - syn;
      Vn = Vn + net->kI[v];
      if (net->ou) {
        /* OU current of this step, then its Euler-Maruyama update with an
         * Irwin-Hall normal (sum of the four words of one Philox call) */
        Vn = Vn + net->kO[v] * net->Iou[i];
        const uint32_t oc[4] = {(uint32_t)gi, (uint32_t)t, (uint32_t)((uint64_t)t >> 32), ORC_TAG_OU};
        uint32_t ro[4];
        orc_philox4x32_10(oc, net->key, ro);
        const int64_t S = (int64_t)((uint64_t)ro[0] + ro[1] + ro[2] + ro[3]) - ((int64_t)1 << 33);
        const real xi = (real)S * net->ou_xi_scale;
        const real decayed = net->ou_d * net->Iou[i];
        net->Iou[i] = (decayed + net->ou_c) + net->ou_s * xi;
      }
      for (int u4 = 0; u4 < 4; u4++) {
        real* jj = &net->j[(size_t)u4 * n + i];
        real decayed = net->dJ[v * 4 + u4] * *jj;
        *jj = decayed + a[u4];
      }
      if (net->ref[i] > 0) {
        net->ref[i] = (uint8_t)(net->ref[i] - 1);
        Vn = net->Vreset[v];
      } else if (Vn >= net->Vth[v]) {
        net->spk[n_spk++] = (int32_t)i;
        net->vcount[v]++;
        Vn = net->Vreset[v];
        net->ref[i] = (uint8_t)net->ref_steps[v];
      }
      net->V[i] = Vn;
    }

    /* 2. delivery: every synapse of every neuron that spiked at t adds its
     *    weight to the accumulator read at step t + d */
    for (int64_t e = 0; e < n_spk; e++) {
      const int32_t src = net->spk[e];
      for (int64_t q = net->out_ptr[src]; q < net->out_ptr[src + 1]; q++) {
        const int64_t slot_d = (t + net->out_d[q]) % D;
        int32_t* acc = net->ring + ((size_t)slot_d * nch + net->out_cls[q]) * (size_t)n + net->out_tgt[q];
        int64_t sum = (int64_t)*acc + net->out_w[q];
        if (sum > INT32_MAX || sum < INT32_MIN) { set_err("accumulator overflows int32"); return -1; }
        *acc = (int32_t)sum;
        net->events++;
      }
    }

    /* 3. BOLD from this step's voxel rates */
    const double dt_s = net->dt * 1e-3;
    for (int32_t v = 0; v < net->nv; v++) {
      const int64_t nvox = net->vstart[v + 1] - net->vstart[v];
      double z = nvox > 0 ? (double)net->vcount[v] / ((double)nvox * dt_s) : 0.0;
      bold_step(net, v, z, dt_s);
    }
    if (ids) {
      if (n_out + n_spk > ids_cap) { set_err("spike buffer full"); return -1; }
      memcpy(ids + n_out, net->spk, (size_t)n_spk * 4);
    }
    n_out += n_spk;
    net->t = t + 1;
    if (step_off) step_off[s + 1] = n_out;
  }
  return n_out;
}

void ORC_FN(orc_get_state)(const orc_net* net, real* V, real* j, uint8_t* ref, int32_t* ring, int64_t* t) {
  const size_t n = (size_t)net->n;
  if (V) memcpy(V, net->V, n * sizeof(real));
  if (j) memcpy(j, net->j, 4 * n * sizeof(real));
  if (ref) memcpy(ref, net->ref, n);
  if (ring) memcpy(ring, net->ring, (size_t)net->D * net->nch * n * 4);
  if (t) *t = net->t;
}

void ORC_FN(orc_set_state)(orc_net* net, const real* V, const real* j, const uint8_t* ref, const int32_t* ring, int64_t t) {
  const size_t n = (size_t)net->n;
  if (V) memcpy(net->V, V, n * sizeof(real));
  if (j) memcpy(net->j, j, 4 * n * sizeof(real));
  if (ref) memcpy(net->ref, ref, n);
  if (ring) memcpy(net->ring, ring, (size_t)net->D * net->nch * n * 4);
  net->t = t;
}

void ORC_FN(orc_get_ou)(const orc_net* net, real* I) {
  if (I) memcpy(I, net->Iou, (size_t)net->n * sizeof(real));
}

void ORC_FN(orc_get_bold)(const orc_net* net, double* y, double* state) {
  const size_t nv = (size_t)net->nv;
  if (y) memcpy(y, net->by, nv * 8);
  if (state) {
    memcpy(state, net->bs, nv * 8);
    memcpy(state + nv, net->bf, nv * 8);
    memcpy(state + 2 * nv, net->bv, nv * 8);
    memcpy(state + 3 * nv, net->bq, nv * 8);
  }
}

void ORC_FN(orc_set_g)(orc_net* net, const double* g) {
  for (int32_t v = 0; v < net->nv; v++)
    for (int u = 0; u < 4; u++) net->vparams[(size_t)v * ORC_NP + ORC_P_G + u] = g[v * 4 + u];
  derive_constants(net);
}

int64_t ORC_FN(orc_events)(const orc_net* net) { return net->events; }
