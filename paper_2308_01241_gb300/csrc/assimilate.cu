// assimilate.cu -- ensemble-Kalman analysis of the hierarchical data
// assimilation (section V.E): every column (one parameter of one voxel,
// observed by that voxel's BOLD) is updated from its members' statistics.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dtb.h"
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

}  // namespace
}  // namespace dtb

extern "C" dtb_status dtb_assimilate(float* d_theta, const float* d_hx, const float* d_y, const float* d_obs_sd,
                                     const float* d_eps, int32_t n_columns, int32_t n_members, float inflation,
                                     void* stream) {
  if (!d_theta || !d_hx || !d_y || !d_obs_sd || !d_eps)
    return dtb::set_last_error(DTB_EINVAL, "dtb_assimilate: NULL array");
  if (n_columns < 0 || n_members < 2 || !(inflation > 0.0f))
    return dtb::set_last_error(DTB_EINVAL, "dtb_assimilate: need n_columns >= 0, n_members >= 2, inflation > 0");
  if (n_columns == 0) return DTB_OK;
  dtb::enkf_kernel<<<n_columns, dtb::kEnkfThreads, 0, (cudaStream_t)stream>>>(d_theta, d_hx, d_y, d_obs_sd, d_eps,
                                                                               n_members, inflation);
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return dtb::set_last_error(DTB_ECUDA, std::string("dtb_assimilate: ") + cudaGetErrorString(e));
  return DTB_OK;
}
