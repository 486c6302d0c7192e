// assimilate.cu -- ensemble-Kalman analysis of the hierarchical data
// assimilation (section V.E): every column (one parameter of one voxel,
// observed by that voxel's BOLD) is updated from its members' statistics.
// The assimilation cycle of dtb_assimilate runs its analysis here too: the
// members' predictions are gathered from the BOLD samples on the device, the
// observation perturbations are drawn on the device, and the updated
// parameters are written straight into the network's per-voxel constants.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "dtb.h"
#include "dtb_device.cuh"
#include "dtb_launch.h"

namespace dtb {
namespace {

constexpr int kEnkfThreads = 128;

__device__ __forceinline__ float block_sum(float x, float* sh) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[w] = x;
  __syncthreads();
  float t = 0.0f;
#pragma unroll
  for (int k = 0; k < kEnkfThreads / 32; k++) t += sh[k];
  return t;
}

// CTA per column c: moments over its M members, gain, perturbed-observation
// update, then inflation of the posterior anomalies.
__global__ void __launch_bounds__(kEnkfThreads) enkf_kernel(float* theta, const float* hx, const float* y,
                                                            const float* sd, const float* eps, int32_t M,
                                                            float lambda) {
  __shared__ float sh[kEnkfThreads / 32];
  const int64_t c = blockIdx.x;
  float* th = theta + c * M;
  const float* h = hx + c * M;
  const float* e = eps + c * M;
  float st = 0.0f, shh = 0.0f;
  for (int m = threadIdx.x; m < M; m += kEnkfThreads) {
    st += th[m];
    shh += h[m];
  }
  const float mt = block_sum(st, sh) / (float)M;
  const float mh = block_sum(shh, sh) / (float)M;
  float cth = 0.0f, chh = 0.0f;
  for (int m = threadIdx.x; m < M; m += kEnkfThreads) {
    const float dt = th[m] - mt, dh = h[m] - mh;
    cth += dt * dh;
    chh += dh * dh;
  }
  cth = block_sum(cth, sh) / (float)(M - 1);
  chh = block_sum(chh, sh) / (float)(M - 1);
  const float s = sd[c];
  const float K = cth / (chh + s * s);
  const float yc = y[c];
  float sa = 0.0f;
  for (int m = threadIdx.x; m < M; m += kEnkfThreads) {
    const float a = th[m] + K * (yc + s * e[m] - h[m]);
    th[m] = a;
    sa += a;
  }
  const float ma = block_sum(sa, sh) / (float)M;
  for (int m = threadIdx.x; m < M; m += kEnkfThreads) th[m] = ma + lambda * (th[m] - ma);
}

// Standard normal of the observation perturbations: the centred sum of the
// four words of one Philox4x32-10 call (Irwin-Hall of order 4, variance 1),
// counter {member, column, TR, 4} under the ensemble's key.
__device__ __forceinline__ float perturbation(uint32_t m, uint32_t c, uint32_t tr, uint32_t k0, uint32_t k1) {
  const uint4 r = philox4x32_10(make_uint4(m, c, tr, 4u), k0, k1);
  const long long S = (long long)((unsigned long long)r.x + r.y + r.z + r.w) - (1LL << 33);
  return __fmul_rn(__ll2float_rn(S), (float)(1.7320508075688772 / 4294967296.0));  // sqrt(3) * 2^-32
}

// Conductance constants of member m of column c from its parameter: the
// receptors in mask get g_base * exp(theta), and kU = (dt * g) / C is
// evaluated in double and rounded once to float, as at creation.
__device__ __forceinline__ void resample_member(const EnsDev& e, int64_t cm, float th, VoxConst* vc) {
  const int32_t v = e.member_voxel[cm];
  const double gain = exp((double)th);
#pragma unroll
  for (int u = 0; u < 4; u++)
    if ((e.mask >> u) & 1) vc[v].kU[u] = (float)((e.dt * (e.g_base[4 * v + u] * gain)) / e.cap[v]);
}

// CTA per column: gather the members' predictions (their voxels' BOLD in
// sample row `row` of the log) and the observation (obs[c], or the target
// voxel's BOLD), then the perturbed-observation analysis of enkf_kernel,
// inflation, the history, and the re-sampled constants.
__global__ void __launch_bounds__(kEnkfThreads) enkf_cycle_kernel(EnsDev e, const float* bold_log, int32_t nv,
                                                                  int64_t row, const float* obs, uint32_t tr,
                                                                  float* theta_hist, float* hx_hist, float* y_hist,
                                                                  VoxConst* vc) {
  __shared__ float sh[kEnkfThreads / 32];
  const int64_t c = blockIdx.x;
  const int32_t M = e.M;
  float* th = e.theta + c * M;
  const int32_t* mv = e.member_voxel + c * M;
  const float* yrow = bold_log + row * nv;
  const float yc = obs ? obs[c] : yrow[e.target_voxel[c]];
  const float s = e.obs_sd_rel * fmaxf(fabsf(yc), 1e-4f);
  float st = 0.0f, shh = 0.0f;
  for (int m = threadIdx.x; m < M; m += kEnkfThreads) {
    st += th[m];
    shh += yrow[mv[m]];
  }
  const float mt = block_sum(st, sh) / (float)M;
  const float mh = block_sum(shh, sh) / (float)M;
  float cth = 0.0f, chh = 0.0f;
  for (int m = threadIdx.x; m < M; m += kEnkfThreads) {
    const float dt = th[m] - mt, dh = yrow[mv[m]] - mh;
    cth += dt * dh;
    chh += dh * dh;
  }
  cth = block_sum(cth, sh) / (float)(M - 1);
  chh = block_sum(chh, sh) / (float)(M - 1);
  const float K = cth / (chh + s * s);
  float sa = 0.0f;
  for (int m = threadIdx.x; m < M; m += kEnkfThreads) {
    const float h = yrow[mv[m]];
    const float a = th[m] + K * (yc + s * perturbation((uint32_t)m, (uint32_t)c, tr, e.key0, e.key1) - h);
    th[m] = a;
    sa += a;
    if (hx_hist) hx_hist[c * M + m] = h;
  }
  const float ma = block_sum(sa, sh) / (float)M;
  for (int m = threadIdx.x; m < M; m += kEnkfThreads) {
    const float a = ma + e.inflation * (th[m] - ma);
    th[m] = a;
    if (theta_hist) theta_hist[c * M + m] = a;
    resample_member(e, c * M + m, a, vc);
  }
  if (threadIdx.x == 0 && y_hist) y_hist[c] = yc;
}

// Constants of every member from its current parameter (no analysis).
__global__ void resample_kernel(EnsDev e, VoxConst* vc) {
  const int64_t n = (int64_t)e.C * e.M;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    resample_member(e, k, e.theta[k], vc);
}

// The per-tile copies of the constants follow their voxel's.
__global__ void tile_consts_kernel(VoxConst* tile_vc, const VoxConst* vc, const int32_t* tile_vox, int32_t nblk) {
  const int32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nblk) return;
  const VoxConst& src = vc[tile_vox[b]];
#pragma unroll
  for (int u = 0; u < 4; u++) tile_vc[b].kU[u] = src.kU[u];
}

}  // namespace
}  // namespace dtb

namespace dtb {

cudaError_t launch_enkf_cycle(const EnsDev& e, const float* bold_log, int32_t nv, int64_t row, const float* obs,
                              uint32_t tr, float* theta_hist, float* hx_hist, float* y_hist, VoxConst* vc,
                              VoxConst* tile_vc, const int32_t* tile_vox, int32_t nblk, cudaStream_t st) {
  enkf_cycle_kernel<<<e.C, kEnkfThreads, 0, st>>>(e, bold_log, nv, row, obs, tr, theta_hist, hx_hist, y_hist, vc);
  tile_consts_kernel<<<(nblk + 255) / 256, 256, 0, st>>>(tile_vc, vc, tile_vox, nblk);
  return cudaGetLastError();
}

cudaError_t launch_resample(const EnsDev& e, VoxConst* vc, VoxConst* tile_vc, const int32_t* tile_vox, int32_t nblk,
                            cudaStream_t st) {
  resample_kernel<<<256, 256, 0, st>>>(e, vc);
  tile_consts_kernel<<<(nblk + 255) / 256, 256, 0, st>>>(tile_vc, vc, tile_vox, nblk);
  return cudaGetLastError();
}

}  // namespace dtb

extern "C" dtb_status dtb_enkf_analysis(float* d_theta, const float* d_hx, const float* d_y, const float* d_obs_sd,
                                     const float* d_eps, int32_t n_columns, int32_t n_members, float inflation,
                                     void* stream) {
  if (!d_theta || !d_hx || !d_y || !d_obs_sd || !d_eps)
    return dtb::set_last_error(DTB_EINVAL, "dtb_enkf_analysis: NULL array");
  if (n_columns < 0 || n_members < 2 || !(inflation > 0.0f))
    return dtb::set_last_error(DTB_EINVAL, "dtb_enkf_analysis: need n_columns >= 0, n_members >= 2, inflation > 0");
  if (n_columns == 0) return DTB_OK;
  dtb::enkf_kernel<<<n_columns, dtb::kEnkfThreads, 0, (cudaStream_t)stream>>>(d_theta, d_hx, d_y, d_obs_sd, d_eps,
                                                                               n_members, inflation);
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return dtb::set_last_error(DTB_ECUDA, std::string("dtb_enkf_analysis: ") + cudaGetErrorString(e));
  return DTB_OK;
}
