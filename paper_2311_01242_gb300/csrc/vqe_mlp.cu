// Warm-start network kernels: a 3-layer perceptron n_in -> H -> H -> n_out with
// SiLU, BF16 weights and GEMM operands, FP32 accumulation (tensor cores via
// mma.sync m16n8k16 BF16 -> FP32), Adam on FP32 master weights. The network is
// tiny (tens of MFLOP per pass) and latency-bound; every GEMM is one launch of
// 16x8 warp tiles. BF16 rounding happens exactly where the oracle rounds:
// x, h1, h2 (forward), dy, da2, da1 (backward); biases, pre-activations,
// bias gradients and the loss stay FP32.
#include <cstdint>
#include <string>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/vqe.h"
#include "vqe_internal.h"

namespace {

struct MlpDims {
  int B, Bp, I, Ip, H, O, Op;
};

MlpDims mlp_dims(int batch, int n_in, int n_hidden, int n_out) {
  MlpDims d;
  d.B = batch;
  d.Bp = (batch + 15) / 16 * 16;
  d.I = n_in;
  d.Ip = (n_in + 15) / 16 * 16;
  d.H = n_hidden;
  d.O = n_out;
  d.Op = (n_out + 15) / 16 * 16;
  return d;
}

struct ParamOffsets {
  int64_t W1, b1, W2, b2, W3, b3, total;
};

ParamOffsets param_offsets(const MlpDims& d) {
  ParamOffsets p;
  p.W1 = 0;
  p.b1 = p.W1 + int64_t(d.H) * d.Ip;
  p.W2 = p.b1 + d.H;
  p.b2 = p.W2 + int64_t(d.H) * d.H;
  p.W3 = p.b2 + d.H;
  p.b3 = p.W3 + int64_t(d.Op) * d.H;
  p.total = p.b3 + d.Op;
  return p;
}

struct MlpWs {
  __nv_bfloat16 *xb, *h1b, *h2b, *dyb, *da2b, *da1b;
  float *a1, *a2, *y, *dy, *da2, *da1;
  size_t total;
};

size_t al(size_t v) { return (v + 255) & ~size_t(255); }

MlpWs ws_layout(const MlpDims& d, void* base) {
  char* b = static_cast<char*>(base);
  size_t o = 0;
  MlpWs w;
  auto take = [&](size_t bytes) {
    char* p = b ? b + o : nullptr;
    o += al(bytes);
    return p;
  };
  w.xb = reinterpret_cast<__nv_bfloat16*>(take(size_t(d.Bp) * d.Ip * 2));
  w.a1 = reinterpret_cast<float*>(take(size_t(d.Bp) * d.H * 4));
  w.h1b = reinterpret_cast<__nv_bfloat16*>(take(size_t(d.Bp) * d.H * 2));
  w.a2 = reinterpret_cast<float*>(take(size_t(d.Bp) * d.H * 4));
  w.h2b = reinterpret_cast<__nv_bfloat16*>(take(size_t(d.Bp) * d.H * 2));
  w.y = reinterpret_cast<float*>(take(size_t(d.Bp) * d.Op * 4));
  w.dy = reinterpret_cast<float*>(take(size_t(d.Bp) * d.Op * 4));
  w.dyb = reinterpret_cast<__nv_bfloat16*>(take(size_t(d.Bp) * d.Op * 2));
  w.da2 = reinterpret_cast<float*>(take(size_t(d.Bp) * d.H * 4));
  w.da2b = reinterpret_cast<__nv_bfloat16*>(take(size_t(d.Bp) * d.H * 2));
  w.da1 = reinterpret_cast<float*>(take(size_t(d.Bp) * d.H * 4));
  w.da1b = reinterpret_cast<__nv_bfloat16*>(take(size_t(d.Bp) * d.H * 2));
  w.total = o;
  return w;
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return uint32_t(__bfloat16_as_ushort(lo)) | (uint32_t(__bfloat16_as_ushort(hi)) << 16);
}

__device__ __forceinline__ uint32_t ld2(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ float silu_f(float a) { return a / (1.0f + expf(-a)); }
__device__ __forceinline__ float dsilu_f(float a) {
  const float s = 1.0f / (1.0f + expf(-a));
  return s * (1.0f + a * (1.0f - s));
}

// x_b = bf16(x), zero padding to [Bp x Ip]
__global__ void k_cast_x(const float* __restrict__ x, int B, int I, int Bp, int Ip, __nv_bfloat16* __restrict__ xb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Bp * Ip) return;
  const int b = i / Ip, c = i % Ip;
  xb[i] = __float2bfloat16_rn((b < B && c < I) ? x[b * I + c] : 0.0f);
}

// C[b][n] = sum_k A[b][k] W[n][k] + bias[n] for a [Bp x K] BF16 A and [N x K] BF16 W.
// act = 1: pre-activation to pre (FP32) and bf16(silu) to actb; act = 0: C to
// out (row stride ld_out) for rows < rows_valid and cols < cols_valid.
__global__ void k_gemm_fwd(const __nv_bfloat16* __restrict__ A, const __nv_bfloat16* __restrict__ W,
                           const float* __restrict__ bias, int Bp, int K, int N, int act,
                           float* __restrict__ pre, __nv_bfloat16* __restrict__ actb, float* __restrict__ out,
                           int ld_out, int rows_valid, int cols_valid) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, tg = lane & 3;
  const int r0 = blockIdx.y * 16;
  const int n0 = (blockIdx.x * 4 + warp) * 8;
  if (n0 >= N || r0 >= Bp) return;
  float c[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k0 = 0; k0 < K; k0 += 16) {
    uint32_t a[4], b[2];
    a[0] = ld2(A + (r0 + g) * K + k0 + tg * 2);
    a[1] = ld2(A + (r0 + g + 8) * K + k0 + tg * 2);
    a[2] = ld2(A + (r0 + g) * K + k0 + 8 + tg * 2);
    a[3] = ld2(A + (r0 + g + 8) * K + k0 + 8 + tg * 2);
    b[0] = ld2(W + (n0 + g) * K + k0 + tg * 2);
    b[1] = ld2(W + (n0 + g) * K + k0 + 8 + tg * 2);
    mma_bf16(c, a, b);
  }
  const int col = n0 + tg * 2;
  for (int h = 0; h < 2; ++h) {
    const int row = r0 + g + 8 * h;
    for (int j = 0; j < 2; ++j) {
      const float v = c[2 * h + j] + bias[col + j];
      if (act) {
        pre[row * N + col + j] = v;
        actb[row * N + col + j] = __float2bfloat16_rn(silu_f(v));
      } else if (row < rows_valid && col + j < cols_valid) {
        out[row * ld_out + col + j] = v;
      }
    }
  }
}

// dy = 2 (y - t) / (B n_out) on the valid block, 0 on padding; bf16 copy; and
// loss = mean (y - t)^2 by one block (fixed-order strided sums + tree).
__global__ void k_loss_dy(const float* __restrict__ y, const float* __restrict__ t, int B, int O, int Bp, int Op,
                          float* __restrict__ dy, __nv_bfloat16* __restrict__ dyb, float* __restrict__ loss) {
  __shared__ float red[1024];
  const float scale = 2.0f / float(B * O);
  float acc = 0.0f;
  for (int i = threadIdx.x; i < Bp * Op; i += blockDim.x) {
    const int b = i / Op, n = i % Op;
    float d = 0.0f;
    if (b < B && n < O) {
      const float e = y[i] - t[b * O + n];
      acc += e * e;
      d = scale * e;
    }
    dy[i] = d;
    dyb[i] = __float2bfloat16_rn(d);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss[0] = red[0] / float(B * O);
}

// dW[n][k] = sum_b dA[b][n] X[b][k]  (dA: [Bp x N] BF16, X: [Bp x K] BF16)
__global__ void k_gemm_dw(const __nv_bfloat16* __restrict__ dA, const __nv_bfloat16* __restrict__ X, int Bp, int N,
                          int K, float* __restrict__ dW) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, tg = lane & 3;
  const int n0 = blockIdx.y * 16;
  const int k0 = (blockIdx.x * 4 + warp) * 8;
  if (k0 >= K || n0 >= N) return;
  float c[4] = {0.f, 0.f, 0.f, 0.f};
  for (int b0 = 0; b0 < Bp; b0 += 16) {
    uint32_t a[4], b[2];
    const int ba = b0 + tg * 2;
    a[0] = pack2(dA[ba * N + n0 + g], dA[(ba + 1) * N + n0 + g]);
    a[1] = pack2(dA[ba * N + n0 + g + 8], dA[(ba + 1) * N + n0 + g + 8]);
    a[2] = pack2(dA[(ba + 8) * N + n0 + g], dA[(ba + 9) * N + n0 + g]);
    a[3] = pack2(dA[(ba + 8) * N + n0 + g + 8], dA[(ba + 9) * N + n0 + g + 8]);
    b[0] = pack2(X[ba * K + k0 + g], X[(ba + 1) * K + k0 + g]);
    b[1] = pack2(X[(ba + 8) * K + k0 + g], X[(ba + 9) * K + k0 + g]);
    mma_bf16(c, a, b);
  }
  const int col = k0 + tg * 2;
  dW[(n0 + g) * K + col] = c[0];
  dW[(n0 + g) * K + col + 1] = c[1];
  dW[(n0 + g + 8) * K + col] = c[2];
  dW[(n0 + g + 8) * K + col + 1] = c[3];
}

// da_prev[b][k] = (sum_n dA[b][n] W[n][k]) * silu'(a_prev[b][k]); FP32 and BF16 copies.
__global__ void k_gemm_dx(const __nv_bfloat16* __restrict__ dA, const __nv_bfloat16* __restrict__ W, int Bp, int N,
                          int K, const float* __restrict__ a_prev, float* __restrict__ da, __nv_bfloat16* __restrict__ dab) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, tg = lane & 3;
  const int r0 = blockIdx.y * 16;
  const int k0 = (blockIdx.x * 4 + warp) * 8;
  if (k0 >= K || r0 >= Bp) return;
  float c[4] = {0.f, 0.f, 0.f, 0.f};
  for (int m0 = 0; m0 < N; m0 += 16) {
    uint32_t a[4], b[2];
    a[0] = ld2(dA + (r0 + g) * N + m0 + tg * 2);
    a[1] = ld2(dA + (r0 + g + 8) * N + m0 + tg * 2);
    a[2] = ld2(dA + (r0 + g) * N + m0 + 8 + tg * 2);
    a[3] = ld2(dA + (r0 + g + 8) * N + m0 + 8 + tg * 2);
    const int mb = m0 + tg * 2;
    b[0] = pack2(W[mb * K + k0 + g], W[(mb + 1) * K + k0 + g]);
    b[1] = pack2(W[(mb + 8) * K + k0 + g], W[(mb + 9) * K + k0 + g]);
    mma_bf16(c, a, b);
  }
  const int col = k0 + tg * 2;
  for (int h = 0; h < 2; ++h) {
    const int row = r0 + g + 8 * h;
    for (int j = 0; j < 2; ++j) {
      const int idx = row * K + col + j;
      const float v = c[2 * h + j] * dsilu_f(a_prev[idx]);
      da[idx] = v;
      dab[idx] = __float2bfloat16_rn(v);
    }
  }
}

// db[n] = sum over valid rows of d[b][n], in row order.
__global__ void k_bias_grad(const float* __restrict__ d, int B, int N, float* __restrict__ db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.0f;
  for (int b = 0; b < B; ++b) s += d[b * N + n];
  db[n] = s;
}

__global__ void k_adam(int64_t n, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, const int* __restrict__ step, float lr, float beta1, float beta2,
                       float eps, __nv_bfloat16* __restrict__ wb) {
  const int t = *step;
  const float c1 = 1.0f / (1.0f - powf(beta1, float(t)));
  const float c2 = 1.0f / (1.0f - powf(beta2, float(t)));
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const float gi = g[i];
    const float mi = beta1 * m[i] + (1.0f - beta1) * gi;
    const float vi = beta2 * v[i] + (1.0f - beta2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    w[i] = wi;
    wb[i] = __float2bfloat16_rn(wi);
  }
}

__global__ void k_step_inc(int* step) { *step += 1; }

__global__ void k_to_bf16(int64_t n, const float* __restrict__ src, __nv_bfloat16* __restrict__ dst) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    dst[i] = __float2bfloat16_rn(src[i]);
}

int check_dims(int batch, int n_in, int n_hidden, int n_out) {
  if (batch < 1 || batch > (1 << 20) || n_in < 1 || n_in > 4096 || n_out < 1 || n_out > 65536 || n_hidden < 16 ||
      n_hidden > 8192 || n_hidden % 16 != 0)
    return vqe::set_error(VQE_ERR_INVALID_ARG,
                          "MLP dims: batch >= 1, 1 <= n_in <= 4096, n_hidden a multiple of 16 in [16, 8192]");
  return VQE_OK;
}

int cuda_check(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return vqe::set_error(VQE_ERR_CUDA, (std::string(what) + ": " + cudaGetErrorString(e)).c_str());
  return VQE_OK;
}

// forward through the three layers into the workspace; the last layer writes
// to out (row stride ld_out) for the valid rows/cols
void forward_layers(const MlpDims& d, const MlpWs& w, const float* params, const __nv_bfloat16* pb, float* out,
                    int ld_out, int rows_valid, int cols_valid, cudaStream_t s) {
  const ParamOffsets po = param_offsets(d);
  const dim3 blk(128);
  k_gemm_fwd<<<dim3((d.H / 8 + 3) / 4, d.Bp / 16), blk, 0, s>>>(w.xb, pb + po.W1, params + po.b1, d.Bp, d.Ip, d.H, 1,
                                                               w.a1, w.h1b, nullptr, 0, 0, 0);
  k_gemm_fwd<<<dim3((d.H / 8 + 3) / 4, d.Bp / 16), blk, 0, s>>>(w.h1b, pb + po.W2, params + po.b2, d.Bp, d.H, d.H, 1,
                                                               w.a2, w.h2b, nullptr, 0, 0, 0);
  k_gemm_fwd<<<dim3((d.Op / 8 + 3) / 4, d.Bp / 16), blk, 0, s>>>(w.h2b, pb + po.W3, params + po.b3, d.Bp, d.H, d.Op,
                                                                0, nullptr, nullptr, out, ld_out, rows_valid,
                                                                cols_valid);
}

}  // namespace

extern "C" {

int64_t vqe_mlp_param_count(int n_in, int n_hidden, int n_out) {
  if (check_dims(1, n_in, n_hidden, n_out)) return 0;
  return param_offsets(mlp_dims(1, n_in, n_hidden, n_out)).total;
}

size_t vqe_mlp_workspace_bytes(int batch, int n_in, int n_hidden, int n_out) {
  if (check_dims(batch, n_in, n_hidden, n_out)) return 0;
  return ws_layout(mlp_dims(batch, n_in, n_hidden, n_out), nullptr).total;
}

int vqe_mlp_to_bf16(int64_t n, const float* src, uint16_t* dst, vqe_stream_t stream) {
  if (n < 0 || (n > 0 && (!src || !dst))) return vqe::set_error(VQE_ERR_INVALID_ARG, "bad bf16 conversion arguments");
  if (n == 0) return VQE_OK;
  k_to_bf16<<<int((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      n, src, reinterpret_cast<__nv_bfloat16*>(dst));
  return cuda_check("k_to_bf16");
}

int vqe_mlp_forward(int batch, int n_in, int n_hidden, int n_out, const float* x, const float* params,
                    const uint16_t* params_bf16, float* y, void* workspace, size_t workspace_bytes,
                    vqe_stream_t stream_) {
  int rc = check_dims(batch, n_in, n_hidden, n_out);
  if (rc) return rc;
  if (!x || !params || !params_bf16 || !y || !workspace) return vqe::set_error(VQE_ERR_INVALID_ARG, "NULL pointer");
  const MlpDims d = mlp_dims(batch, n_in, n_hidden, n_out);
  const MlpWs w = ws_layout(d, workspace);
  if (workspace_bytes < w.total) return vqe::set_error(VQE_ERR_WORKSPACE, "MLP workspace too small");
  cudaStream_t s = static_cast<cudaStream_t>(stream_);
  k_cast_x<<<(d.Bp * d.Ip + 255) / 256, 256, 0, s>>>(x, d.B, d.I, d.Bp, d.Ip, w.xb);
  forward_layers(d, w, params, reinterpret_cast<const __nv_bfloat16*>(params_bf16), y, d.O, d.B, d.O, s);
  return cuda_check("mlp forward");
}

int vqe_mlp_loss_grad(int batch, int n_in, int n_hidden, int n_out, const float* x, const float* target,
                      const float* params, const uint16_t* params_bf16, float* grads, float* loss,
                      void* workspace, size_t workspace_bytes, vqe_stream_t stream_) {
  int rc = check_dims(batch, n_in, n_hidden, n_out);
  if (rc) return rc;
  if (!x || !target || !params || !params_bf16 || !grads || !loss || !workspace)
    return vqe::set_error(VQE_ERR_INVALID_ARG, "NULL pointer");
  const MlpDims d = mlp_dims(batch, n_in, n_hidden, n_out);
  const MlpWs w = ws_layout(d, workspace);
  if (workspace_bytes < w.total) return vqe::set_error(VQE_ERR_WORKSPACE, "MLP workspace too small");
  cudaStream_t s = static_cast<cudaStream_t>(stream_);
  const ParamOffsets po = param_offsets(d);
  const __nv_bfloat16* pb = reinterpret_cast<const __nv_bfloat16*>(params_bf16);
  k_cast_x<<<(d.Bp * d.Ip + 255) / 256, 256, 0, s>>>(x, d.B, d.I, d.Bp, d.Ip, w.xb);
  forward_layers(d, w, params, pb, w.y, d.Op, d.Bp, d.Op, s);
  k_loss_dy<<<1, 1024, 0, s>>>(w.y, target, d.B, d.O, d.Bp, d.Op, w.dy, w.dyb, loss);
  const dim3 blk(128);
  // layer 3
  k_gemm_dw<<<dim3((d.H / 8 + 3) / 4, d.Op / 16), blk, 0, s>>>(w.dyb, w.h2b, d.Bp, d.Op, d.H,
                                                                                  grads + po.W3);
  k_bias_grad<<<(d.Op + 127) / 128, 128, 0, s>>>(w.dy, d.B, d.Op, grads + po.b3);
  k_gemm_dx<<<dim3((d.H / 8 + 3) / 4, d.Bp / 16), blk, 0, s>>>(w.dyb, pb + po.W3, d.Bp, d.Op, d.H, w.a2, w.da2, w.da2b);
  // layer 2
  k_gemm_dw<<<dim3((d.H / 8 + 3) / 4, d.H / 16), blk, 0, s>>>(w.da2b, w.h1b, d.Bp, d.H, d.H, grads + po.W2);
  k_bias_grad<<<(d.H + 127) / 128, 128, 0, s>>>(w.da2, d.B, d.H, grads + po.b2);
  k_gemm_dx<<<dim3((d.H / 8 + 3) / 4, d.Bp / 16), blk, 0, s>>>(w.da2b, pb + po.W2, d.Bp, d.H, d.H, w.a1, w.da1, w.da1b);
  // layer 1
  k_gemm_dw<<<dim3((d.Ip / 8 + 3) / 4, d.H / 16), blk, 0, s>>>(w.da1b, w.xb, d.Bp, d.H, d.Ip, grads + po.W1);
  k_bias_grad<<<(d.H + 127) / 128, 128, 0, s>>>(w.da1, d.B, d.H, grads + po.b1);
  return cuda_check("mlp loss_grad");
}

int vqe_mlp_adam(int64_t n, float* params, const float* grads, float* m, float* v, int* step_dev, float lr,
                 float beta1, float beta2, float eps, uint16_t* params_bf16, vqe_stream_t stream) {
  if (n < 1 || !params || !grads || !m || !v || !params_bf16 || !step_dev)
    return vqe::set_error(VQE_ERR_INVALID_ARG, "bad Adam arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int blocks = int((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  k_adam<<<blocks, 256, 0, s>>>(n, params, grads, m, v, step_dev, lr, beta1, beta2, eps,
                                reinterpret_cast<__nv_bfloat16*>(params_bf16));
  k_step_inc<<<1, 1, 0, s>>>(step_dev);
  return cuda_check("k_adam");
}

}  // extern "C"
