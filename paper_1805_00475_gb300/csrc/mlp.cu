// The learned edge scorer: a 3-layer perceptron F -> H -> H -> 1 (ReLU),
// fp32 training (forward, backward with the squared-error loss, Adam) and
// bf16 inference, as hand-written CUDA kernels.
//
// Parameter layout (fp32, flat): W1[F][H], b1[H], W2[H][H], b2[H], w3[H], b3.
// A block handles a tile of 32 rows with H = 128 threads; thread t owns hidden
// unit t of both layers.  Activations saved for the backward pass are the
// post-ReLU values h1, h2 ([rows][H] each).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>

#include "tnc_internal.h"

namespace tnc_mlp {

constexpr int F = TNC_MLP_FEATURES;
constexpr int H = TNC_MLP_HIDDEN;
constexpr int kRows = 32;
constexpr int OFF_W1 = 0, OFF_B1 = F * H, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H, OFF_W3 = OFF_B2 + H,
              OFF_B3 = OFF_W3 + H, N_PARAMS = OFF_B3 + 1;
static_assert(N_PARAMS == TNC_MLP_PARAMS, "parameter count");

template <typename WT>
__device__ __forceinline__ float ld(const WT* p, int i);
template <>
__device__ __forceinline__ float ld<float>(const float* p, int i) {
  return p[i];
}
template <>
__device__ __forceinline__ float ld<__nv_bfloat16>(const __nv_bfloat16* p, int i) {
  return __bfloat162float(p[i]);
}

// y[r] = w3 . relu(W2^T relu(W1^T x_r + b1) + b2) + b3; optionally saves h1, h2.
template <typename WT>
__global__ void __launch_bounds__(H) mlp_forward_kernel(const WT* __restrict__ P, const float* __restrict__ X,
                                                        int64_t rows, float* __restrict__ Y, float* __restrict__ h1s,
                                                        float* __restrict__ h2s) {
  __shared__ float xs[kRows][F];
  __shared__ float h1[kRows][H];
  __shared__ float red[kRows][H / 32];
  const int t = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * kRows;
  for (int i = t; i < kRows * F; i += H) {
    const int64_t r = r0 + i / F;
    xs[i / F][i % F] = r < rows ? X[r * F + i % F] : 0.f;
  }
  __syncthreads();
  float w1[F];
#pragma unroll
  for (int f = 0; f < F; f++) w1[f] = ld(P, OFF_W1 + f * H + t);
  const float b1 = ld(P, OFF_B1 + t);
  for (int r = 0; r < kRows; r++) {
    float a = b1;
#pragma unroll
    for (int f = 0; f < F; f++) a = fmaf(xs[r][f], w1[f], a);
    h1[r][t] = fmaxf(a, 0.f);
  }
  __syncthreads();
  float acc[kRows];
  const float b2 = ld(P, OFF_B2 + t);
#pragma unroll
  for (int r = 0; r < kRows; r++) acc[r] = b2;
  for (int j = 0; j < H; j++) {
    const float w = ld(P, OFF_W2 + j * H + t);
#pragma unroll
    for (int r = 0; r < kRows; r++) acc[r] = fmaf(h1[r][j], w, acc[r]);
  }
  const float w3 = ld(P, OFF_W3 + t);
#pragma unroll
  for (int r = 0; r < kRows; r++) {
    const float h2 = fmaxf(acc[r], 0.f);
    if (h2s && r0 + r < rows) h2s[(r0 + r) * H + t] = h2;
    if (h1s && r0 + r < rows) h1s[(r0 + r) * H + t] = h1[r][t];
    float v = h2 * w3;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((t & 31) == 0) red[r][t >> 5] = v;
  }
  __syncthreads();
  if (t < kRows && r0 + t < rows) {
    float s = ld(P, OFF_B3);
#pragma unroll
    for (int w = 0; w < H / 32; w++) s += red[t][w];
    Y[r0 + t] = s;
  }
}

// Backward pass of L = (1/n) sum_r (y_r - t_r)^2 over the n = `rows` rows of
// this call.  Pass 1 (per row): dy, dh2 = dy w3 [h2 > 0], dh1 = W2 dh2 [h1 > 0].
__global__ void __launch_bounds__(H) mlp_backward_rows_kernel(const float* __restrict__ P,
                                                              const float* __restrict__ h1s,
                                                              const float* __restrict__ h2s,
                                                              const float* __restrict__ Y, const float* __restrict__ T,
                                                              int64_t rows, float* __restrict__ dy_out,
                                                              float* __restrict__ dh1s, float* __restrict__ dh2s) {
  __shared__ float dh2[kRows][H];
  __shared__ float dy[kRows];
  const int t = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * kRows;
  if (t < kRows) {
    dy[t] = r0 + t < rows ? 2.f * (Y[r0 + t] - T[r0 + t]) / (float)rows : 0.f;
    if (r0 + t < rows) dy_out[r0 + t] = dy[t];
  }
  __syncthreads();
  const float w3 = P[OFF_W3 + t];
  for (int r = 0; r < kRows; r++) {
    const bool in = r0 + r < rows;
    const float h2 = in ? h2s[(r0 + r) * H + t] : 0.f;
    const float d = h2 > 0.f ? dy[r] * w3 : 0.f;
    dh2[r][t] = d;
    if (in) dh2s[(r0 + r) * H + t] = d;
  }
  __syncthreads();
  // dh1[r][t] = sum_u W2[t][u] dh2[r][u], four passes of 32 columns of W2's row t
  float d1[kRows];
#pragma unroll
  for (int r = 0; r < kRows; r++) d1[r] = 0.f;
  for (int pass = 0; pass < 4; pass++) {
    float w[H / 4];
#pragma unroll
    for (int u = 0; u < H / 4; u++) w[u] = P[OFF_W2 + t * H + pass * (H / 4) + u];
#pragma unroll 4
    for (int r = 0; r < kRows; r++) {
      float s = 0.f;
#pragma unroll
      for (int u = 0; u < H / 4; u++) s = fmaf(dh2[r][pass * (H / 4) + u], w[u], s);
      d1[r] += s;
    }
  }
#pragma unroll
  for (int r = 0; r < kRows; r++) {
    if (r0 + r < rows) {
      const float h1 = h1s[(r0 + r) * H + t];
      dh1s[(r0 + r) * H + t] = h1 > 0.f ? d1[r] : 0.f;
    }
  }
}

// Pass 2 (per parameter, summed over the rows; no atomics, fixed order):
// block j < H:        dW2[j][t] = sum_r h1[r][j] dh2[r][t]
// block H + f (f < F): dW1[f][t] = sum_r x[r][f] dh1[r][t]
// block H + F:        db1[t], db2[t], dw3[t] = sum_r h2[r][t] dy[r], db3
__global__ void __launch_bounds__(H) mlp_backward_params_kernel(const float* __restrict__ X,
                                                                const float* __restrict__ h1s,
                                                                const float* __restrict__ h2s,
                                                                const float* __restrict__ dys,
                                                                const float* __restrict__ dh1s,
                                                                const float* __restrict__ dh2s, int64_t rows,
                                                                float* __restrict__ G) {
  const int t = threadIdx.x;
  const int b = blockIdx.x;
  if (b < H) {
    float g = 0.f;
    for (int64_t r = 0; r < rows; r++) g = fmaf(h1s[r * H + b], dh2s[r * H + t], g);
    G[OFF_W2 + b * H + t] = g;
  } else if (b < H + F) {
    const int f = b - H;
    float g = 0.f;
    for (int64_t r = 0; r < rows; r++) g = fmaf(X[r * F + f], dh1s[r * H + t], g);
    G[OFF_W1 + f * H + t] = g;
  } else {
    float g1 = 0.f, g2 = 0.f, g3 = 0.f, gb3 = 0.f;
    for (int64_t r = 0; r < rows; r++) {
      g1 += dh1s[r * H + t];
      g2 += dh2s[r * H + t];
      g3 = fmaf(h2s[r * H + t], dys[r], g3);
      if (t == 0) gb3 += dys[r];
    }
    G[OFF_B1 + t] = g1;
    G[OFF_B2 + t] = g2;
    G[OFF_W3 + t] = g3;
    if (t == 0) G[OFF_B3] = gb3;
  }
}

__global__ void adam_kernel(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ M,
                            float* __restrict__ V, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float g = G[i];
    const float m = b1 * M[i] + (1.f - b1) * g;
    const float v = b2 * V[i] + (1.f - b2) * g * g;
    M[i] = m;
    V[i] = v;
    P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
  }
}

__global__ void to_bf16_kernel(const float* __restrict__ P, __nv_bfloat16* __restrict__ Q, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) Q[i] = __float2bfloat16(P[i]);
}

// Squared error of a batch, accumulated into loss[0] (sum over rows).
__global__ void sqerr_kernel(const float* __restrict__ Y, const float* __restrict__ T, int64_t rows, float* loss) {
  float s = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += (int64_t)gridDim.x * blockDim.x) {
    const float d = Y[i] - T[i];
    s += d * d;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, s);
}

}  // namespace tnc_mlp

using namespace tnc;

namespace {
#define MLP_TRY(call)                                                                               \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) return set_error(TNC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

unsigned blocks_for(int64_t rows) { return (unsigned)((rows + tnc_mlp::kRows - 1) / tnc_mlp::kRows); }
}  // namespace

namespace tnc {

// Synchronous copy for host code compiled without CUDA headers: dir 0 = host
// to device, 1 = device to host (the stream is synchronised).
void copy_device(void* dst, const void* src, size_t bytes, int dir, void* stream, int* rc) {
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, dir == 0 ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) *rc = set_error(TNC_ERR_CUDA, std::string("copy: ") + cudaGetErrorString(e));
}

int mlp_forward_dev(const float* P, const float* X, int64_t rows, float* Y, float* h1, float* h2, void* stream) {
  if (rows <= 0) return TNC_OK;
  tnc_mlp::mlp_forward_kernel<float><<<blocks_for(rows), tnc_mlp::H, 0, (cudaStream_t)stream>>>(P, X, rows, Y, h1, h2);
  MLP_TRY(cudaGetLastError());
  return TNC_OK;
}

int mlp_forward_bf16_dev(const void* Pb, const float* X, int64_t rows, float* Y, void* stream) {
  if (rows <= 0) return TNC_OK;
  tnc_mlp::mlp_forward_kernel<__nv_bfloat16><<<blocks_for(rows), tnc_mlp::H, 0, (cudaStream_t)stream>>>(
      (const __nv_bfloat16*)Pb, X, rows, Y, nullptr, nullptr);
  MLP_TRY(cudaGetLastError());
  return TNC_OK;
}

}  // namespace tnc

extern "C" {

int tnc_mlp_forward(const float* d_params, const float* d_x, int64_t rows, float* d_y, float* d_h1, float* d_h2,
                    void* cuda_stream) {
  clear_error();
  if (!d_params || !d_x || !d_y || rows < 0) return set_error(TNC_ERR_INVALID, "bad mlp_forward arguments");
  return mlp_forward_dev(d_params, d_x, rows, d_y, d_h1, d_h2, cuda_stream);
}

int tnc_mlp_backward(const float* d_params, const float* d_x, const float* d_h1, const float* d_h2, const float* d_y,
                     const float* d_t, int64_t rows, float* d_scratch, float* d_grads, void* cuda_stream) {
  clear_error();
  if (!d_params || !d_x || !d_h1 || !d_h2 || !d_y || !d_t || !d_scratch || !d_grads || rows < 0)
    return set_error(TNC_ERR_INVALID, "bad mlp_backward arguments");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (rows == 0) {
    MLP_TRY(cudaMemsetAsync(d_grads, 0, (size_t)TNC_MLP_PARAMS * sizeof(float), st));
    return TNC_OK;
  }
  float* dy = d_scratch;
  float* dh1 = dy + rows;
  float* dh2 = dh1 + rows * TNC_MLP_HIDDEN;
  tnc_mlp::mlp_backward_rows_kernel<<<blocks_for(rows), tnc_mlp::H, 0, st>>>(d_params, d_h1, d_h2, d_y, d_t, rows, dy,
                                                                           dh1, dh2);
  tnc_mlp::mlp_backward_params_kernel<<<tnc_mlp::H + tnc_mlp::F + 1, tnc_mlp::H, 0, st>>>(d_x, d_h1, d_h2, dy, dh1, dh2,
                                                                                         rows, d_grads);
  MLP_TRY(cudaGetLastError());
  return TNC_OK;
}

int tnc_mlp_adam(float* d_params, const float* d_grads, float* d_m, float* d_v, int32_t step, float lr,
                 void* cuda_stream) {
  clear_error();
  if (!d_params || !d_grads || !d_m || !d_v || step < 1) return set_error(TNC_ERR_INVALID, "bad mlp_adam arguments");
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)step), c2 = 1.f - std::pow(b2, (float)step);
  tnc_mlp::adam_kernel<<<72, 256, 0, (cudaStream_t)cuda_stream>>>(d_params, d_grads, d_m, d_v, TNC_MLP_PARAMS, lr, b1,
                                                                   b2, 1e-8f, c1, c2);
  MLP_TRY(cudaGetLastError());
  return TNC_OK;
}

int tnc_mlp_to_bf16(const float* d_params, void* d_params_bf16, void* cuda_stream) {
  clear_error();
  if (!d_params || !d_params_bf16) return set_error(TNC_ERR_INVALID, "NULL argument");
  tnc_mlp::to_bf16_kernel<<<72, 256, 0, (cudaStream_t)cuda_stream>>>(d_params, (__nv_bfloat16*)d_params_bf16,
                                                                      TNC_MLP_PARAMS);
  MLP_TRY(cudaGetLastError());
  return TNC_OK;
}

int tnc_mlp_forward_bf16(const void* d_params_bf16, const float* d_x, int64_t rows, float* d_y, void* cuda_stream) {
  clear_error();
  if (!d_params_bf16 || !d_x || !d_y || rows < 0) return set_error(TNC_ERR_INVALID, "bad mlp_forward_bf16 arguments");
  return mlp_forward_bf16_dev(d_params_bf16, d_x, rows, d_y, cuda_stream);
}

size_t tnc_mlp_backward_scratch_floats(int64_t rows) { return rows <= 0 ? 0 : (size_t)rows * (1 + 2 * TNC_MLP_HIDDEN); }

size_t tnc_mlp_train_workspace_bytes(int32_t batch) {
  if (batch <= 0) return 0;
  const size_t b = (size_t)batch;
  // y, h1, h2 and backward scratch (dy, dh1, dh2) for a batch; grads, Adam m and v; loss
  return (b + 2 * b * TNC_MLP_HIDDEN + tnc_mlp_backward_scratch_floats(batch) + 3 * (size_t)TNC_MLP_PARAMS + 64) *
         sizeof(float);
}

// Mini-batch Adam on the squared error.  Epochs walk the rows in the order
// given (the caller shuffles them once); every epoch's mean loss is reported.
int tnc_mlp_train(float* d_params, const float* d_x, const float* d_t, int64_t rows, int32_t epochs, int32_t batch,
                  float lr, void* d_ws, size_t ws_bytes, void* cuda_stream, float* loss_out) {
  clear_error();
  if (!d_params || !d_x || !d_t || rows <= 0 || epochs <= 0 || batch <= 0 || !d_ws)
    return set_error(TNC_ERR_INVALID, "bad mlp_train arguments");
  if (ws_bytes < tnc_mlp_train_workspace_bytes(batch)) return set_error(TNC_ERR_BUFFER, "workspace too small");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  float* y = (float*)d_ws;
  float* h1 = y + batch;
  float* h2 = h1 + (size_t)batch * TNC_MLP_HIDDEN;
  float* scratch = h2 + (size_t)batch * TNC_MLP_HIDDEN;
  float* g = scratch + tnc_mlp_backward_scratch_floats(batch);
  float* m = g + TNC_MLP_PARAMS;
  float* v = m + TNC_MLP_PARAMS;
  float* loss = v + TNC_MLP_PARAMS;
  MLP_TRY(cudaMemsetAsync(m, 0, 2 * (size_t)TNC_MLP_PARAMS * sizeof(float), st));
  int32_t step = 0;
  for (int32_t e = 0; e < epochs; e++) {
    MLP_TRY(cudaMemsetAsync(loss, 0, sizeof(float), st));
    for (int64_t r0 = 0; r0 < rows; r0 += batch) {
      const int64_t nb = std::min<int64_t>(batch, rows - r0);
      const float* xb = d_x + r0 * TNC_MLP_FEATURES;
      const float* tb = d_t + r0;
      int rc = mlp_forward_dev(d_params, xb, nb, y, h1, h2, st);
      if (rc) return rc;
      tnc_mlp::sqerr_kernel<<<std::max<unsigned>(1, (unsigned)std::min<int64_t>((nb + 255) / 256, 64)), 256, 0, st>>>(
          y, tb, nb, loss);
      rc = tnc_mlp_backward(d_params, xb, h1, h2, y, tb, nb, scratch, g, st);
      if (rc) return rc;
      rc = tnc_mlp_adam(d_params, g, m, v, ++step, lr, st);
      if (rc) return rc;
    }
    if (loss_out) {
      float l = 0;
      MLP_TRY(cudaMemcpyAsync(&l, loss, sizeof(float), cudaMemcpyDeviceToHost, st));
      MLP_TRY(cudaStreamSynchronize(st));
      loss_out[e] = l / (float)rows;
    }
  }
  MLP_TRY(cudaStreamSynchronize(st));
  return TNC_OK;
}

}  // extern "C"
