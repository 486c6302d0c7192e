// mlp.cu -- the learned surrogate's MLP: BF16 tensor-core GEMMs with FP32
// accumulation (mma.sync.m16n8k16), fused bias / GELU epilogues, backward
// pass and Adam, behind the C ABI of include/dtb_surrogate.h.
//
// The layers are 256 wide: every GEMM is a few hundred MFLOP, so the kernels
// are latency-bound and a 64 x 64 register-tiled mma.sync kernel suffices.
// GELU(x) = 0.5 x (1 + erf(x / sqrt 2)) calls erff.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "dtb.h"
#include "dtb_launch.h"
#include "dtb_surrogate.h"

namespace {

typedef __nv_bfloat16 bf16;

constexpr int kT = 64;   // block tile (rows and columns)
constexpr int kBK = 16;  // k step
constexpr int kPad = 8;  // shared-memory row padding (bank spread)

enum { EPI_GELU = 1, EPI_BIAS = 2, EPI_DGELU = 3, EPI_F32 = 4 };

struct Epi {
  const float* bias;  // [N]
  float* z;           // EPI_GELU: pre-activation out [M][N]
  bf16* a;            // EPI_GELU: activation out; EPI_DGELU: gradient out [M][N]
  float* y;           // EPI_BIAS / EPI_F32: fp32 out [M][N]
  const float* zin;   // EPI_DGELU: pre-activation of the layer below [M][N]
};

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C[M][N] = sum_k A(m, k) B(k, n) with A(m, k) = TA ? a[k*lda + m] : a[m*lda + k]
// and B(k, n) = TB ? b[n*ldb + k] : b[k*ldb + n]; out-of-range elements read 0.
// 128 threads = 2 x 2 warps, each 32 x 32 = 2 x 4 mma tiles of 16 x 8.
template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(128) gemm_kernel(const bf16* __restrict__ a, int lda, const bf16* __restrict__ b,
                                                   int ldb, int M, int N, int K, Epi ep) {
  __shared__ __align__(16) bf16 As[kT][kBK + kPad];  // [m][k]
  __shared__ __align__(16) bf16 Bs[kT][kBK + kPad];  // [n][k]
  const int m0 = blockIdx.y * kT, n0 = blockIdx.x * kT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int g = lane >> 2, t = lane & 3;
  const bf16 zero = __float2bfloat16(0.0f);
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; i++)
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
      for (int q = 0; q < 4; q++) acc[i][j][q] = 0.0f;

  for (int k0 = 0; k0 < K; k0 += kBK) {
    for (int idx = threadIdx.x; idx < kT * kBK; idx += 128) {
      int mm, kk;
      if (TA) { kk = idx / kT; mm = idx % kT; } else { mm = idx / kBK; kk = idx % kBK; }
      const int m = m0 + mm, k = k0 + kk;
      As[mm][kk] = (m < M && k < K) ? (TA ? a[(int64_t)k * lda + m] : a[(int64_t)m * lda + k]) : zero;
      int nn, kb;
      if (TB) { nn = idx / kBK; kb = idx % kBK; } else { kb = idx / kT; nn = idx % kT; }
      const int n = n0 + nn, kq = k0 + kb;
      Bs[nn][kb] = (n < N && kq < K) ? (TB ? b[(int64_t)n * ldb + kq] : b[(int64_t)kq * ldb + n]) : zero;
    }
    __syncthreads();
    uint32_t af[2][4], bfr[4][2];
#pragma unroll
    for (int i = 0; i < 2; i++) {
      const int r = wm + i * 16 + g;
      af[i][0] = *reinterpret_cast<const uint32_t*>(&As[r][2 * t]);
      af[i][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][2 * t]);
      af[i][2] = *reinterpret_cast<const uint32_t*>(&As[r][2 * t + 8]);
      af[i][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][2 * t + 8]);
    }
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int c = wn + j * 8 + g;
      bfr[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[c][2 * t]);
      bfr[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[c][2 * t + 8]);
    }
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
      for (int j = 0; j < 4; j++) mma_bf16(acc[i][j], af[i], bfr[j]);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; i++)
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const int m = m0 + wm + i * 16 + g + (q >= 2 ? 8 : 0);
        const int n = n0 + wn + j * 8 + 2 * t + (q & 1);
        if (m >= M || n >= N) continue;
        const int64_t o = (int64_t)m * N + n;
        const float v = acc[i][j][q];
        if (EPI == EPI_GELU) {
          const float z = v + ep.bias[n];
          ep.z[o] = z;
          ep.a[o] = __float2bfloat16(gelu(z));
        } else if (EPI == EPI_BIAS) {
          ep.y[o] = v + ep.bias[n];
        } else if (EPI == EPI_DGELU) {
          ep.a[o] = __float2bfloat16(v * gelu_grad(ep.zin[o]));
        } else {
          ep.y[o] = v;
        }
      }
}

__global__ void to_bf16_kernel(const float* x, bf16* y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16(x[i]);
}

// Mean-squared-error gradient dY = 2 (Y - T) / (B * n_out), stored in bf16 for
// the backward GEMMs; per-block sums of (Y - T)^2 for the loss.
__global__ void mse_grad_kernel(const float* y, const float* tgt, bf16* dy, int64_t n, float scale, float* part) {
  __shared__ float sh[8];
  float s = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float d = y[i] - tgt[i];
    s += d * d;
    dy[i] = __float2bfloat16(2.0f * d * scale);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float tot = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) tot += sh[w];
    part[blockIdx.x] = tot;
  }
}

// db[n] = sum over rows of G[m][n] (bf16 gradient), fp32.
__global__ void colsum_kernel(const bf16* G, int M, int N, float* db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.0f;
  for (int m = 0; m < M; m++) s += __bfloat162float(G[(int64_t)m * N + n]);
  db[n] = s;
}

// Adam (Kingma & Ba 2015) on fp32 master weights; refreshes the bf16 copy.
__global__ void adam_kernel(float* p, bf16* p16, float* m, float* v, const float* gr, int64_t n, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = gr[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float upd = lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    const float np_ = p[i] - upd;
    p[i] = np_;
    if (p16) p16[i] = __float2bfloat16(np_);
  }
}

template <bool TA, bool TB, int EPI>
cudaError_t gemm(const bf16* a, int lda, const bf16* b, int ldb, int M, int N, int K, const Epi& ep, cudaStream_t st) {
  dim3 grid((N + kT - 1) / kT, (M + kT - 1) / kT);
  gemm_kernel<TA, TB, EPI><<<grid, 128, 0, st>>>(a, lda, b, ldb, M, N, K, ep);
  return cudaGetLastError();
}

}  // namespace

struct dtb_mlp {
  int n_in, width, depth, n_out;
  int64_t max_batch;
  int nl;                         // layers = depth + 1
  std::vector<int> din, dout;     // per layer
  std::vector<int64_t> woff, boff;  // offsets in the flat parameter vector
  int64_t n_params = 0;
  float* p = nullptr;             // fp32 master parameters (flat)
  bf16* p16 = nullptr;            // bf16 copy of the weights (same offsets)
  float* m = nullptr;             // Adam moments
  float* v = nullptr;
  float* grad = nullptr;          // fp32 gradients (flat)
  bf16* x16 = nullptr;            // [B][n_in]
  std::vector<bf16*> act;         // act[l]: input of layer l (bf16), l = 1..depth
  std::vector<float*> z;          // z[l]: pre-activation of hidden layer l
  float* y = nullptr;             // [B][n_out]
  bf16* g0 = nullptr;             // gradient ping-pong buffers [B][width]
  bf16* g1 = nullptr;
  bf16* dy = nullptr;             // [B][n_out]
  float* part = nullptr;          // loss partial sums
  int adam_t = 0;
  std::vector<void*> mem;
  void* alloc(size_t bytes) {
    void* q = nullptr;
    if (cudaMalloc(&q, bytes ? bytes : 16) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    mem.push_back(q);
    return q;
  }
  ~dtb_mlp() {
    for (void* q : mem) cudaFree(q);
  }
};

namespace {

dtb_status cuda_err(cudaError_t e, const char* where) {
  return dtb::set_last_error(DTB_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Forward pass over B rows of x16 -> y (fp32), keeping z and activations.
cudaError_t forward(dtb_mlp* n, int64_t B, cudaStream_t st) {
  const bf16* in = n->x16;
  for (int l = 0; l < n->nl; l++) {
    Epi ep{};
    ep.bias = n->p + n->boff[l];
    const bf16* W = n->p16 + n->woff[l];
    cudaError_t e;
    if (l < n->nl - 1) {
      ep.z = n->z[l + 1];
      ep.a = n->act[l + 1];
      e = gemm<false, false, EPI_GELU>(in, n->din[l], W, n->dout[l], (int)B, n->dout[l], n->din[l], ep, st);
      in = n->act[l + 1];
    } else {
      ep.y = n->y;
      e = gemm<false, false, EPI_BIAS>(in, n->din[l], W, n->dout[l], (int)B, n->dout[l], n->din[l], ep, st);
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t stage_input(dtb_mlp* n, const float* d_x, int64_t B, cudaStream_t st) {
  to_bf16_kernel<<<256, 256, 0, st>>>(d_x, n->x16, B * n->n_in);
  return cudaGetLastError();
}

// Loss gradient and backward pass: fills n->grad; *loss_dev partial sums in n->part.
cudaError_t backward(dtb_mlp* n, const float* d_t, int64_t B, cudaStream_t st, int* nparts) {
  const int64_t ny = B * n->n_out;
  const int parts = 256;
  mse_grad_kernel<<<parts, 256, 0, st>>>(n->y, d_t, n->dy, ny, 1.0f / (float)ny, n->part);
  *nparts = parts;
  const bf16* G = n->dy;
  bf16* bufs[2] = {n->g0, n->g1};
  int pb = 0;
  for (int l = n->nl - 1; l >= 0; l--) {
    const bf16* A = l == 0 ? n->x16 : n->act[l];
    Epi ew{};
    ew.y = n->grad + n->woff[l];
    // dW[l] = A^T G : [din][B] x [B][dout]
    cudaError_t e = gemm<true, false, EPI_F32>(A, n->din[l], G, n->dout[l], n->din[l], n->dout[l], (int)B, ew, st);
    if (e != cudaSuccess) return e;
    colsum_kernel<<<(n->dout[l] + 127) / 128, 128, 0, st>>>(G, (int)B, n->dout[l], n->grad + n->boff[l]);
    if (l > 0) {
      // G[l-1] = (G W^T) * gelu'(z[l])
      Epi ed{};
      ed.a = bufs[pb];
      ed.zin = n->z[l];
      e = gemm<false, true, EPI_DGELU>(G, n->dout[l], n->p16 + n->woff[l], n->dout[l], (int)B, n->din[l],
                                        n->dout[l], ed, st);
      if (e != cudaSuccess) return e;
      G = bufs[pb];
      pb ^= 1;
    }
  }
  return cudaGetLastError();
}

}  // namespace

extern "C" {

dtb_status dtb_mlp_create(int32_t n_in, int32_t width, int32_t depth, int32_t n_out, int64_t max_batch,
                          const float* params, dtb_mlp** out) {
  if (!out || !params) return dtb::set_last_error(DTB_EINVAL, "dtb_mlp_create: NULL argument");
  *out = nullptr;
  if (n_in < 1 || width < 1 || depth < 1 || n_out < 1 || max_batch < 1 || max_batch > (1 << 26))
    return dtb::set_last_error(DTB_EINVAL, "dtb_mlp_create: bad sizes");
  dtb_mlp* n = new dtb_mlp();
  n->n_in = n_in; n->width = width; n->depth = depth; n->n_out = n_out; n->max_batch = max_batch;
  n->nl = depth + 1;
  for (int l = 0; l < n->nl; l++) {
    n->din.push_back(l == 0 ? n_in : width);
    n->dout.push_back(l == n->nl - 1 ? n_out : width);
    n->woff.push_back(n->n_params);
    n->n_params += (int64_t)n->din[l] * n->dout[l];
    n->boff.push_back(n->n_params);
    n->n_params += n->dout[l];
  }
  const size_t P = (size_t)n->n_params;
  bool ok = true;
  auto A = [&](size_t bytes) { void* q = n->alloc(bytes); if (!q) ok = false; return q; };
  n->p = (float*)A(4 * P);
  n->p16 = (bf16*)A(2 * P);
  n->m = (float*)A(4 * P);
  n->v = (float*)A(4 * P);
  n->grad = (float*)A(4 * P);
  n->x16 = (bf16*)A(2 * (size_t)max_batch * n_in);
  n->act.assign(n->nl, nullptr);
  n->z.assign(n->nl, nullptr);
  for (int l = 1; l < n->nl; l++) {
    n->act[l] = (bf16*)A(2 * (size_t)max_batch * width);
    n->z[l] = (float*)A(4 * (size_t)max_batch * width);
  }
  n->y = (float*)A(4 * (size_t)max_batch * n_out);
  n->g0 = (bf16*)A(2 * (size_t)max_batch * width);
  n->g1 = (bf16*)A(2 * (size_t)max_batch * width);
  n->dy = (bf16*)A(2 * (size_t)max_batch * n_out);
  n->part = (float*)A(4 * 256);
  if (!ok) {
    delete n;
    return dtb::set_last_error(DTB_ENOMEM, "dtb_mlp_create: device allocation failed");
  }
  cudaError_t e = cudaMemcpy(n->p, params, 4 * P, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(n->m, 0, 4 * P);
  if (e == cudaSuccess) e = cudaMemset(n->v, 0, 4 * P);
  if (e == cudaSuccess) {
    to_bf16_kernel<<<256, 256>>>(n->p, n->p16, (int64_t)P);
    e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) {
    delete n;
    return cuda_err(e, "dtb_mlp_create");
  }
  *out = n;
  return DTB_OK;
}

dtb_status dtb_mlp_destroy(dtb_mlp* n) {
  if (!n) return dtb::set_last_error(DTB_EINVAL, "dtb_mlp_destroy: NULL");
  delete n;
  return DTB_OK;
}

dtb_status dtb_mlp_forward(dtb_mlp* n, const float* d_x, float* d_y, int64_t B, void* stream) {
  if (!n || !d_x || !d_y || B < 1 || B > n->max_batch) return dtb::set_last_error(DTB_EINVAL, "dtb_mlp_forward: NULL argument or batch outside 1..max_batch");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = stage_input(n, d_x, B, st);
  if (e == cudaSuccess) e = forward(n, B, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_y, n->y, 4 * (size_t)B * n->n_out, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? DTB_OK : cuda_err(e, "dtb_mlp_forward");
}

dtb_status dtb_mlp_gradients(dtb_mlp* n, const float* d_x, const float* d_t, int64_t B, float* grads, float* loss,
                             void* stream) {
  if (!n || !d_x || !d_t || B < 1 || B > n->max_batch) return dtb::set_last_error(DTB_EINVAL, "dtb_mlp_gradients: NULL argument or batch outside 1..max_batch");
  cudaStream_t st = (cudaStream_t)stream;
  int parts = 0;
  cudaError_t e = stage_input(n, d_x, B, st);
  if (e == cudaSuccess) e = forward(n, B, st);
  if (e == cudaSuccess) e = backward(n, d_t, B, st, &parts);
  std::vector<float> hp(256);
  if (e == cudaSuccess && loss) e = cudaMemcpyAsync(hp.data(), n->part, 4 * 256, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && grads) e = cudaMemcpyAsync(grads, n->grad, 4 * (size_t)n->n_params, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_err(e, "dtb_mlp_gradients");
  if (loss) {
    double s = 0;
    for (int k = 0; k < parts; k++) s += hp[k];
    *loss = (float)(s / ((double)B * n->n_out));
  }
  return DTB_OK;
}

dtb_status dtb_mlp_train_step(dtb_mlp* n, const float* d_x, const float* d_t, int64_t B, float lr, float* loss,
                              void* stream) {
  dtb_status s = dtb_mlp_gradients(n, d_x, d_t, B, nullptr, loss, stream);
  if (s != DTB_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  n->adam_t++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, (float)n->adam_t), c2 = 1.0f - powf(b2, (float)n->adam_t);
  adam_kernel<<<512, 256, 0, st>>>(n->p, n->p16, n->m, n->v, n->grad, n->n_params, lr, b1, b2, 1e-8f, c1, c2);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  return e == cudaSuccess ? DTB_OK : cuda_err(e, "dtb_mlp_train_step");
}

dtb_status dtb_mlp_get_params(dtb_mlp* n, float* params) {
  if (!n || !params) return dtb::set_last_error(DTB_EINVAL, "dtb_mlp_get_params");
  cudaError_t e = cudaMemcpy(params, n->p, 4 * (size_t)n->n_params, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? DTB_OK : cuda_err(e, "dtb_mlp_get_params");
}

}  // extern "C"
