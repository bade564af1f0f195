// Learned angle proposal (not in the paper): a 272 -> 256 -> 256 -> 256 -> 181 MLP with ReLU hidden
// layers and a sigmoid occupancy output over 1-degree bins, trained with binary cross-entropy on
// logits and Adam. Weights are kept in FP32 (master) and used as BF16 in the tensor-core GEMMs
// (FP32 accumulation). Every product runs through gemm_tc (tcgen05, TMA-fed):
//   forward  A_l = relu(A_{l-1} W_l^T + b_l)          (BF16 row-major and transposed copies)
//            Z   = A_3 W_4^T + b_4                     (FP32 logits)
//   backward dZ_4 = (sigmoid(Z) - Y) / B
//            dW_l = dZ_l^T A_{l-1}  (= dZ_l^T (A_{l-1}^T)^T with both operands K = batch)
//            dA_{l-1} = dZ_l W_l    (= dZ_l (W_l^T)^T with the transposed BF16 weights)
//            dZ_{l-1} = dA_{l-1} * [A_{l-1} > 0]
// Elementwise kernels here: input conversion, loss, ReLU backward (with bias-gradient column
// sums and the transposed BF16 copies), Adam, and the BF16 weight refresh.
#include <cuda_bf16.h>
#include <float.h>

#include "doa_internal.cuh"

namespace doa {

cudaError_t launch_gemm_tc(const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb, int M, int N, int K,
                           int epi, const float *bias, void *D, int ldd, __nv_bfloat16 *DT, int lddt, int *err,
                           cudaStream_t s);

namespace {

constexpr int kIn = DOA_MLP_IN, kHid = DOA_MLP_HIDDEN, kOut = DOA_MLP_OUT;
constexpr int kOutP = (kOut + 7) / 8 * 8;   // BF16 row pitch of 181-wide matrices
constexpr int kDims[5] = {kIn, kHid, kHid, kHid, kOut};

__host__ __device__ inline int pitch8(int n) { return (n + 7) / 8 * 8; }

struct MlpWs {
  __nv_bfloat16 *X0, *X0T, *A[3], *AT[3], *dZ4, *dZ4T, *dZ, *dZT;
  float *Z4, *dA, *loss_acc;
  int *err;
  size_t bytes;
};

MlpWs ws_layout(uint8_t *base, int B) {
  MlpWs w{};
  size_t at = 0;
  auto take = [&](size_t n) {
    uint8_t *p = base ? base + at : nullptr;
    at += (n + 255) / 256 * 256;
    return p;
  };
  w.X0 = reinterpret_cast<__nv_bfloat16 *>(take((size_t)B * kIn * 2));
  w.X0T = reinterpret_cast<__nv_bfloat16 *>(take((size_t)kIn * B * 2));
  for (int l = 0; l < 3; ++l) {
    w.A[l] = reinterpret_cast<__nv_bfloat16 *>(take((size_t)B * kHid * 2));
    w.AT[l] = reinterpret_cast<__nv_bfloat16 *>(take((size_t)kHid * B * 2));
  }
  w.dZ4 = reinterpret_cast<__nv_bfloat16 *>(take((size_t)B * kOutP * 2));
  w.dZ4T = reinterpret_cast<__nv_bfloat16 *>(take((size_t)kOut * B * 2));
  w.dZ = reinterpret_cast<__nv_bfloat16 *>(take((size_t)B * kHid * 2));
  w.dZT = reinterpret_cast<__nv_bfloat16 *>(take((size_t)kHid * B * 2));
  w.Z4 = reinterpret_cast<float *>(take((size_t)B * kOut * 4));
  w.dA = reinterpret_cast<float *>(take((size_t)B * kHid * 4));
  w.loss_acc = reinterpret_cast<float *>(take(4));
  w.err = reinterpret_cast<int *>(take(4));
  w.bytes = at;
  return w;
}

// FP32 features (B x 272) -> BF16 row-major and transposed copies (32 x 32 tiles through smem).
__global__ void input_kernel(const float *X, int B, __nv_bfloat16 *X0, __nv_bfloat16 *X0T) {
  __shared__ float t[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    float v = (r < B && c < kIn) ? X[(size_t)r * kIn + c] : 0.f;
    t[i][threadIdx.x] = v;
    if (r < B && c < kIn) X0[(size_t)r * kIn + c] = __float2bfloat16_rn(v);
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (c < kIn && r < B) X0T[(size_t)c * B + r] = __float2bfloat16_rn(t[threadIdx.x][i]);
  }
}

__global__ void sigmoid_kernel(const float *Z, int n, float *P) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    P[i] = 1.f / (1.f + __expf(-Z[i]));
}

// BCE with logits: loss = mean_b sum_j [max(z,0) - y z + log(1 + e^{-|z|})]; dZ = (sigmoid(z) - y)/B.
// Writes dZ in BF16 row-major (pitch 184, zero padding) and transposed, the bias gradient (column
// sums) and the loss.
__global__ void bce_kernel(const float *Z, const float *Y, int B, __nv_bfloat16 *dZ, __nv_bfloat16 *dZT, float *gb,
                           float *loss) {
  __shared__ float t[32][33];
  __shared__ float colsum[32];
  __shared__ float lsum;
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  if (threadIdx.y == 0) colsum[threadIdx.x] = 0.f;
  if (threadIdx.x == 0 && threadIdx.y == 0) lsum = 0.f;
  __syncthreads();
  const float invB = 1.f / (float)B;
  float lacc = 0.f, cacc = 0.f;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    float g = 0.f;
    if (r < B && c < kOut) {
      const float z = Z[(size_t)r * kOut + c], y = Y[(size_t)r * kOut + c];
      const float sg = 1.f / (1.f + __expf(-z));
      g = (sg - y) * invB;
      lacc += (fmaxf(z, 0.f) - y * z + log1pf(__expf(-fabsf(z)))) * invB;
      cacc += g;
    }
    t[i][threadIdx.x] = g;
    if (r < B && c < kOutP) dZ[(size_t)r * kOutP + c] = __float2bfloat16_rn(g);
  }
  atomicAdd(&colsum[threadIdx.x], cacc);
  atomicAdd(&lsum, lacc);
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (c < kOut && r < B) dZT[(size_t)c * B + r] = __float2bfloat16_rn(t[threadIdx.x][i]);
  }
  if (threadIdx.y == 0 && c0 + threadIdx.x < kOut) atomicAdd(&gb[c0 + threadIdx.x], colsum[threadIdx.x]);
  if (threadIdx.x == 0 && threadIdx.y == 0) atomicAdd(loss, lsum);
}

// dZ = dA * [A > 0] (A is the BF16 activation), BF16 row-major + transposed, bias-gradient sums.
__global__ void relu_back_kernel(const float *dA, const __nv_bfloat16 *A, int B, __nv_bfloat16 *dZ,
                                 __nv_bfloat16 *dZT, float *gb) {
  __shared__ float t[32][33];
  __shared__ float colsum[32];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  if (threadIdx.y == 0) colsum[threadIdx.x] = 0.f;
  __syncthreads();
  float cacc = 0.f;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    float g = 0.f;
    if (r < B) {
      const size_t o = (size_t)r * kHid + c;
      g = __bfloat162float(A[o]) > 0.f ? dA[o] : 0.f;
      dZ[o] = __float2bfloat16_rn(g);
      cacc += g;
    }
    t[i][threadIdx.x] = g;
  }
  atomicAdd(&colsum[threadIdx.x], cacc);
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (r < B) dZT[(size_t)c * B + r] = __float2bfloat16_rn(t[threadIdx.x][i]);
  }
  if (threadIdx.y == 0) atomicAdd(&gb[c0 + threadIdx.x], colsum[threadIdx.x]);
}

struct LayerPtrs {
  float *W, *b, *mW, *vW, *mb, *vb, *gW, *gb;
  __nv_bfloat16 *Wh, *WhT;
  int out, in;
};

// Adam on the FP32 masters, then the BF16 copies (row-major and transposed).
__global__ void adam_kernel(LayerPtrs p, float lr, float b1, float b2, float eps, float c1, float c2, int update) {
  const int nW = p.out * p.in;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nW + p.out; i += gridDim.x * blockDim.x) {
    float *w, *m, *v;
    const float *gp;
    if (i < nW) {
      w = p.W + i; m = p.mW + i; v = p.vW + i; gp = p.gW + i;
    } else {
      w = p.b + (i - nW); m = p.mb + (i - nW); v = p.vb + (i - nW); gp = p.gb + (i - nW);
    }
    if (update) {
      const float g = *gp;
      const float mm = b1 * *m + (1.f - b1) * g;
      const float vv = b2 * *v + (1.f - b2) * g * g;
      *m = mm;
      *v = vv;
      *w -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    }
    if (i < nW) {
      const int r = i / p.in, c = i % p.in;
      const __nv_bfloat16 h = __float2bfloat16_rn(*w);
      p.Wh[(size_t)r * p.in + c] = h;
      p.WhT[(size_t)c * pitch8(p.out) + r] = h;
    }
  }
}

LayerPtrs layer(const doa_mlp *net, int l) {
  LayerPtrs p;
  p.W = net->W[l]; p.b = net->b[l]; p.mW = net->mW[l]; p.vW = net->vW[l];
  p.mb = net->mb[l]; p.vb = net->vb[l]; p.gW = net->gW[l]; p.gb = net->gb[l];
  p.Wh = reinterpret_cast<__nv_bfloat16 *>(net->Wh[l]);
  p.WhT = reinterpret_cast<__nv_bfloat16 *>(net->WhT[l]);
  p.out = kDims[l + 1];
  p.in = kDims[l];
  return p;
}

bool net_ok(const doa_mlp *net, bool train) {
  if (!net) return false;
  for (int l = 0; l < 4; ++l) {
    if (!net->Wh[l] || !net->WhT[l] || !net->b[l]) return false;
    if (train && (!net->W[l] || !net->mW[l] || !net->vW[l] || !net->mb[l] || !net->vb[l] || !net->gW[l] ||
                  !net->gb[l]))
      return false;
  }
  return true;
}

cudaError_t forward(const doa_mlp *net, const float *features, int B, const MlpWs &w, cudaStream_t s) {
  dim3 tb(32, 8);
  input_kernel<<<dim3((kIn + 31) / 32, (B + 31) / 32), tb, 0, s>>>(features, B, w.X0, w.X0T);
  const __nv_bfloat16 *a = w.X0;
  int lda = kIn;
  cudaError_t e;
  for (int l = 0; l < 3; ++l) {
    e = launch_gemm_tc(a, lda, reinterpret_cast<const __nv_bfloat16 *>(net->Wh[l]), kDims[l], B, kHid, kDims[l],
                       2, net->b[l], w.A[l], kHid, w.AT[l], B, w.err, s);
    if (e != cudaSuccess) return e;
    a = w.A[l];
    lda = kHid;
  }
  return launch_gemm_tc(a, kHid, reinterpret_cast<const __nv_bfloat16 *>(net->Wh[3]), kHid, B, kOut, kHid, 1,
                        net->b[3], w.Z4, kOut, nullptr, 0, w.err, s);
}

}  // namespace
}  // namespace doa

using namespace doa;

extern "C" size_t doa_mlp_workspace_bytes(int batch) {
  if (batch < 8 || (batch & 7)) return 0;
  return ws_layout(nullptr, batch).bytes;
}

extern "C" doa_status doa_mlp_refresh(const doa_mlp *net, void *stream) {
  if (!net_ok(net, false)) return DOA_EINVAL;
  for (int l = 0; l < 4; ++l)
    if (!net->W[l]) return DOA_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  for (int l = 0; l < 4; ++l) {
    LayerPtrs p = layer(net, l);
    adam_kernel<<<128, 256, 0, s>>>(p, 0.f, 0.f, 0.f, 0.f, 1.f, 1.f, 0);
  }
  return cudaGetLastError() == cudaSuccess ? DOA_OK : DOA_ECUDA;
}

extern "C" doa_status doa_mlp_forward(const doa_mlp *net, const float *features, int batch, float *probs,
                                      float *logits, void *ws, size_t ws_bytes, void *stream) {
  if (!net_ok(net, false) || !features || batch < 8 || (batch & 7) || !ws) return DOA_EINVAL;
  MlpWs w = ws_layout(static_cast<uint8_t *>(ws), batch);
  if (ws_bytes < w.bytes) return DOA_ENOMEM;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (forward(net, features, batch, w, s) != cudaSuccess) return DOA_ECUDA;
  const int n = batch * kOut;
  if (logits && cudaMemcpyAsync(logits, w.Z4, (size_t)n * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return DOA_ECUDA;
  if (probs) sigmoid_kernel<<<(n + 255) / 256, 256, 0, s>>>(w.Z4, n, probs);
  return cudaGetLastError() == cudaSuccess ? DOA_OK : DOA_ECUDA;
}

extern "C" doa_status doa_mlp_backward(const doa_mlp *net, const float *features, const float *labels, int batch,
                                       float *loss, void *ws, size_t ws_bytes, void *stream) {
  if (!net_ok(net, true) || !features || !labels || batch < 8 || (batch & 7) || !ws) return DOA_EINVAL;
  MlpWs w = ws_layout(static_cast<uint8_t *>(ws), batch);
  if (ws_bytes < w.bytes) return DOA_ENOMEM;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int B = batch;
  for (int l = 0; l < 4; ++l)
    if (cudaMemsetAsync(net->gb[l], 0, (size_t)kDims[l + 1] * 4, s) != cudaSuccess) return DOA_ECUDA;
  if (cudaMemsetAsync(w.loss_acc, 0, 4, s) != cudaSuccess) return DOA_ECUDA;
  if (cudaMemsetAsync(w.dZ4, 0, (size_t)B * kOutP * 2, s) != cudaSuccess) return DOA_ECUDA;
  if (forward(net, features, B, w, s) != cudaSuccess) return DOA_ECUDA;
  dim3 tb(32, 8);
  bce_kernel<<<dim3((kOutP + 31) / 32, (B + 31) / 32), tb, 0, s>>>(w.Z4, labels, B, w.dZ4, w.dZ4T, net->gb[3],
                                                                    w.loss_acc);
  cudaError_t e;
  // layer 4: dW4 = dZ4^T A3, dA3 = dZ4 W4
  e = launch_gemm_tc(w.dZ4T, B, w.AT[2], B, kOut, kHid, B, 0, nullptr, net->gW[3], kHid, nullptr, 0, w.err, s);
  if (e != cudaSuccess) return DOA_ECUDA;
  e = launch_gemm_tc(w.dZ4, kOutP, reinterpret_cast<const __nv_bfloat16 *>(net->WhT[3]), kOutP, B, kHid, kOut, 0,
                     nullptr, w.dA, kHid, nullptr, 0, w.err, s);
  if (e != cudaSuccess) return DOA_ECUDA;
  for (int l = 2; l >= 0; --l) {
    relu_back_kernel<<<dim3(kHid / 32, (B + 31) / 32), tb, 0, s>>>(w.dA, w.A[l], B, w.dZ, w.dZT, net->gb[l]);
    const __nv_bfloat16 *prevT = l == 0 ? w.X0T : w.AT[l - 1];
    e = launch_gemm_tc(w.dZT, B, prevT, B, kHid, kDims[l], B, 0, nullptr, net->gW[l], kDims[l], nullptr, 0, w.err, s);
    if (e != cudaSuccess) return DOA_ECUDA;
    if (l > 0) {
      e = launch_gemm_tc(w.dZ, kHid, reinterpret_cast<const __nv_bfloat16 *>(net->WhT[l]), kHid, B, kHid, kHid, 0,
                         nullptr, w.dA, kHid, nullptr, 0, w.err, s);
      if (e != cudaSuccess) return DOA_ECUDA;
    }
  }
  if (loss && cudaMemcpyAsync(loss, w.loss_acc, 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return DOA_ECUDA;
  return cudaGetLastError() == cudaSuccess ? DOA_OK : DOA_ECUDA;
}

extern "C" doa_status doa_mlp_adam(const doa_mlp *net, float lr, float beta1, float beta2, float eps, int t,
                                   void *stream) {
  if (!net_ok(net, true) || t < 1 || !(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f))
    return DOA_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const float c1 = 1.f - powf(beta1, (float)t), c2 = 1.f - powf(beta2, (float)t);
  for (int l = 0; l < 4; ++l)
    adam_kernel<<<256, 256, 0, s>>>(layer(net, l), lr, beta1, beta2, eps, c1, c2, 1);
  return cudaGetLastError() == cudaSuccess ? DOA_OK : DOA_ECUDA;
}
