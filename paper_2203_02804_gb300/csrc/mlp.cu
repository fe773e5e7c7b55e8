// Kernels of the learned surrogate (include/ttmlp.h): tiled FP32 GEMMs for the
// fully connected layers (weights in FP32 or bfloat16, products accumulated in
// FP32), SiLU and its derivative fused into the epilogues, Adam, MSE and the
// ensemble statistics; and the inference layer on the 5th-generation tensor
// cores (tcgen05.mma kind::f16, bfloat16 operands, FP32 accumulator in TMEM).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "ttmlp.h"
#include "ttprice_tc.cuh"

namespace ttm {

constexpr int kTile = 64;   // output tile (rows and columns)
constexpr int kK = 16;      // k slice staged per step
constexpr int kThreads = 256;  // 16 x 16 threads, 4 x 4 outputs each

__device__ __forceinline__ float silu(float z) { return z / (1.0f + __expf(-z)); }
__device__ __forceinline__ float silu_grad(float z) {
  const float s = 1.0f / (1.0f + __expf(-z));
  return s * (1.0f + z * (1.0f - s));
}

__device__ __forceinline__ float load_w(const float* w, long i) { return w[i]; }
__device__ __forceinline__ float load_w(const __nv_bfloat16* w, long i) { return __bfloat162float(w[i]); }

// C[m][n] = sum_k A(m, k) B(k, n) (+ bias[n]) with strided operands
//   A(m, k) = A[m * sam + k * sak], B(k, n) = B[k * sbk + n * sbn];
// when Aout is set it also receives act(C) (the layer's activation).
template <typename TB>
__global__ void __launch_bounds__(kThreads) gemm_kernel(int M, int N, int K, const float* __restrict__ A, long sam,
                                                       long sak, const TB* __restrict__ B, long sbk, long sbn,
                                                       float* __restrict__ C, long ldc, const float* __restrict__ bias,
                                                       int act, float* __restrict__ Aout) {
  __shared__ float As[kK][kTile + 4];
  __shared__ float Bs[kK][kTile + 4];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * kTile, n0 = blockIdx.x * kTile;
  float acc[4][4] = {};
  // staging order per operand: consecutive threads walk its contiguous index
  // (k when the stride along k is 1, else the row), so the loads coalesce
  const bool a_k_inner = sak == 1, b_k_inner = sbk == 1;
  for (int k0 = 0; k0 < K; k0 += kK) {
    for (int i = threadIdx.x; i < kK * kTile; i += kThreads) {
      const int kk = a_k_inner ? i % kK : i / kTile, mm = a_k_inner ? i / kK : i % kTile;
      const int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < M && k < K) ? A[(long)m * sam + (long)k * sak] : 0.0f;
    }
    for (int i = threadIdx.x; i < kK * kTile; i += kThreads) {
      const int kk = b_k_inner ? i % kK : i / kTile, nn = b_k_inner ? i / kK : i % kTile;
      const int n = n0 + nn, k = k0 + kk;
      Bs[kk][nn] = (n < N && k < K) ? load_w(B, (long)k * sbk + (long)n * sbn) : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty + 16 * i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx + 16 * j;
      if (n >= N) continue;
      float v = acc[i][j];
      if (bias) v += bias[n];
      C[(long)m * ldc + n] = v;
      if (Aout) Aout[(long)m * ldc + n] = act == TT_MLP_SILU ? silu(v) : v;
    }
  }
}

// g = da * act'(z); g may be da itself
__global__ void act_grad_kernel(const float* __restrict__ z, const float* da, float* g, long n, int act) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) g[i] = act == TT_MLP_SILU ? da[i] * silu_grad(z[i]) : da[i];
}

// db[n] = sum over rows of g[:, n] (one thread per column, rows in order)
__global__ void colsum_kernel(const float* __restrict__ g, int rows, int cols, float* __restrict__ db) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.0f;
  for (int r = 0; r < rows; ++r) s += g[(long)r * cols + c];
  db[c] = s;
}

__global__ void mse_kernel(const float* __restrict__ y, const float* __restrict__ t, int n, float* __restrict__ dy,
                           float* __restrict__ loss) {
  __shared__ float part[kThreads];
  float s = 0.0f;
  for (int i = threadIdx.x; i < n; i += kThreads) {
    const float e = y[i] - t[i];
    dy[i] = 2.0f * e / (float)n;
    s += e * e;
  }
  part[threadIdx.x] = s;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = part[0] / (float)n;
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void bf16_kernel(const float* __restrict__ s, __nv_bfloat16* __restrict__ d, long n) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = __float2bfloat16_rn(s[i]);
}

__global__ void ensemble_kernel(const float* __restrict__ p, int members, int n, float* __restrict__ mean,
                                float* __restrict__ spread) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.0f, lo = p[i], hi = p[i];
  for (int e = 0; e < members; ++e) {
    const float v = p[(long)e * n + i];
    s += v;
    lo = fminf(lo, v);
    hi = fmaxf(hi, v);
  }
  mean[i] = s / (float)members;
  spread[i] = hi - lo;
}

__global__ void gather_kernel(const float* __restrict__ src, const int* __restrict__ idx, int rows, int cols,
                              float* __restrict__ dst) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)rows * cols) return;
  const int r = (int)(i / cols), c = (int)(i % cols);
  dst[i] = src[(long)idx[r] * cols + c];
}

// ---------------------------------------------------------------------------
// Tensor-core layer: Y = act(X W^T + b), X [M][K] and W [N][K] bfloat16 (both
// K-major, as stored), 16 <= N <= 256 and K <= 256 multiples of 16.  One CTA of
// four warps takes 128 rows: X's rows and all of W are staged in shared memory
// in the canonical no-swizzle K-major layout (8-row x 16-byte core matrices,
// 128 bytes apart along K, 8-row groups (K/8) 128 bytes apart), one thread
// issues K/16 MMAs of M = 128, N, K = 16 into TMEM and commits them to an
// mbarrier, and each warp reads back its 32 TMEM lanes (rows) to add the bias,
// apply the activation and store FP32 and/or bfloat16 rows.  A completion wait
// that runs out of its bound leaves NaN in the tile's outputs; the wait before
// the tensor memory is freed keeps the full bound.
// ---------------------------------------------------------------------------
constexpr int kTcRows = 128;
constexpr int kTcThreads = 128;

__device__ __forceinline__ uint32_t f16_idesc(int n) {
  // D FP32 (bits 4-5 = 1), A and B bfloat16 (bits 7-9 = 1, 10-12 = 1), both
  // K-major, N >> 3 at bit 17, M >> 4 at bit 24
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// 16-byte chunk c (8 bfloat16 along K) of row r into the K-major layout
__device__ __forceinline__ uint32_t kmaj16(int r, int c, int sbo) { return (r >> 3) * sbo + c * 128 + (r & 7) * 16; }

__global__ void __launch_bounds__(kTcThreads, 1) tc_layer_kernel(const uint16_t* __restrict__ X, int M, int K,
                                                                  const uint16_t* __restrict__ W, const float* bias,
                                                                  int N, int act, float* Yf, uint16_t* Yb) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m0 = blockIdx.x * kTcRows;
  const int sbo = (K / 8) * 128;
  unsigned char* sA = smem;
  unsigned char* sB = smem + (size_t)kTcRows * K * 2;
  uint32_t ncols = 32;
  while ((int)ncols < N) ncols <<= 1;
  if (warp == 0) ttp::tc::tmem_alloc(&tslot, ncols);
  const int kc = K / 8;
  for (int idx = tid; idx < kTcRows * kc; idx += kTcThreads) {
    const int r = idx / kc, c = idx % kc;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (m0 + r < M) v = *reinterpret_cast<const uint4*>(X + (size_t)(m0 + r) * K + c * 8);
    *reinterpret_cast<uint4*>(sA + kmaj16(r, c, sbo)) = v;
  }
  for (int idx = tid; idx < N * kc; idx += kTcThreads) {
    const int r = idx / kc, c = idx % kc;
    *reinterpret_cast<uint4*>(sB + kmaj16(r, c, sbo)) = *reinterpret_cast<const uint4*>(W + (size_t)r * K + c * 8);
  }
  if (tid == 0) ttp::tc::mbar_init(&mbar, 1);
  ttp::tc::fence_async_smem();  // the operands were written by the generic proxy
  ttp::tc::fence_before_sync();
  __syncthreads();
  ttp::tc::fence_after_sync();
  const uint32_t tmem = tslot;
  if (tid == 0) {
    const uint32_t id = f16_idesc(N);
    for (int ks = 0; ks < K / 16; ++ks) {  // K = 16 per instruction: two core matrices, 256 bytes
      const uint64_t a = ttp::tc::smem_desc(ttp::tc::smem_u32(sA) + ks * 256, (uint32_t)sbo);
      const uint64_t b = ttp::tc::smem_desc(ttp::tc::smem_u32(sB) + ks * 256, (uint32_t)sbo);
      mma_f16(tmem, a, b, id, ks > 0 ? 1u : 0u);
    }
    ttp::tc::commit(&mbar);
  }
  const bool done = ttp::tc::mbar_wait(&mbar, 0);
  ttp::tc::fence_after_sync();
  const int row = m0 + 32 * warp + lane;
  for (int c0 = 0; c0 < N; c0 += 8) {
    float v[8];
    ttp::tc::tmem_ld8(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
    ttp::tc::tmem_wait_ld();
    if (row < M) {
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        float z = done ? v[c] + (bias ? bias[c0 + c] : 0.0f) : __int_as_float(0x7fc00000);
        if (act == TT_MLP_SILU) z = silu(z);
        if (Yf) Yf[(size_t)row * N + c0 + c] = z;
        if (Yb) Yb[(size_t)row * N + c0 + c] = __bfloat16_as_ushort(__float2bfloat16_rn(z));
      }
    }
  }
  if (!done) ttp::tc::mbar_wait(&mbar, 0);  // no product in flight when the columns are freed
  ttp::tc::fence_before_sync();
  __syncthreads();
  ttp::tc::fence_after_sync();
  if (warp == 0) ttp::tc::tmem_dealloc(tmem, ncols);
}

template <typename TB>
int gemm(int M, int N, int K, const float* A, long sam, long sak, const TB* B, long sbk, long sbn, float* C,
         long ldc, const float* bias, int act, float* Aout, cudaStream_t st) {
  if (M <= 0 || N <= 0 || K <= 0) return TT_MLP_OK;
  const dim3 grid((N + kTile - 1) / kTile, (M + kTile - 1) / kTile);
  gemm_kernel<TB><<<grid, kThreads, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias, act, Aout);
  return cudaGetLastError() == cudaSuccess ? TT_MLP_OK : TT_MLP_CUDA;
}

inline unsigned blocks(long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace ttm

using namespace ttm;

extern "C" int tt_mlp_forward(const float* x, int batch, int in, const float* w, const float* b, int out, int act,
                              float* z, float* a, void* stream) {
  if (!x || !w || !z || !a || batch < 0 || in < 1 || out < 1) return TT_MLP_INVALID;
  // z[m][n] = sum_k x[m][k] w[n][k] + b[n]
  return gemm<float>(batch, out, in, x, in, 1, w, 1, in, z, out, b, act, a, (cudaStream_t)stream);
}

extern "C" int tt_mlp_forward_bf16(const float* x, int batch, int in, const uint16_t* w_bf16, const float* b,
                                   int out, int act, float* z, float* a, void* stream) {
  if (!x || !w_bf16 || !z || !a || batch < 0 || in < 1 || out < 1) return TT_MLP_INVALID;
  const __nv_bfloat16* w = reinterpret_cast<const __nv_bfloat16*>(w_bf16);
  return gemm<__nv_bfloat16>(batch, out, in, x, in, 1, w, 1, in, z, out, b, act, a, (cudaStream_t)stream);
}

extern "C" int tt_mlp_forward_tc(const uint16_t* x_bf16, int batch, int in, const uint16_t* w_bf16, const float* b,
                                 int out, int act, float* a, uint16_t* a_bf16, void* stream) {
  if (!x_bf16 || !w_bf16 || (!a && !a_bf16) || batch < 0 || in < 16 || in > 256 || in % 16 || out < 16 ||
      out > 256 || out % 16)
    return TT_MLP_INVALID;
  if (batch == 0) return TT_MLP_OK;
  const int smem = (kTcRows + out) * in * 2;
  if (cudaFuncSetAttribute(tc_layer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
    cudaGetLastError();
    return TT_MLP_CUDA;
  }
  tc_layer_kernel<<<(batch + kTcRows - 1) / kTcRows, kTcThreads, smem, (cudaStream_t)stream>>>(
      x_bf16, batch, in, w_bf16, b, out, act, a, a_bf16);
  return cudaGetLastError() == cudaSuccess ? TT_MLP_OK : TT_MLP_CUDA;
}

extern "C" int tt_mlp_backward(const float* x, const float* z, float* da, int batch, int in, const float* w,
                               int out, int act, float* dx, float* dw, float* db, void* stream) {
  if (!x || !z || !da || !w || !dw || !db || batch < 1 || in < 1 || out < 1) return TT_MLP_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  float* g = da;  // dL/dz, written over dL/da
  const long n = (long)batch * out;
  act_grad_kernel<<<blocks(n, 256), 256, 0, st>>>(z, da, g, n, act);
  if (cudaGetLastError() != cudaSuccess) return TT_MLP_CUDA;
  // dw[o][i] = sum_m g[m][o] x[m][i]
  int rc = gemm<float>(out, in, batch, g, 1, out, x, in, 1, dw, in, nullptr, TT_MLP_LINEAR, nullptr, st);
  if (rc != TT_MLP_OK) return rc;
  colsum_kernel<<<blocks(out, 128), 128, 0, st>>>(g, batch, out, db);
  if (cudaGetLastError() != cudaSuccess) return TT_MLP_CUDA;
  // dx[m][i] = sum_o g[m][o] w[o][i]
  if (dx) rc = gemm<float>(batch, in, out, g, out, 1, w, in, 1, dx, in, nullptr, TT_MLP_LINEAR, nullptr, st);
  return rc;
}

extern "C" int tt_mlp_mse(const float* y, const float* t, int n, float* dy, float* loss, void* stream) {
  if (!y || !t || !dy || !loss || n < 1) return TT_MLP_INVALID;
  mse_kernel<<<1, kThreads, 0, (cudaStream_t)stream>>>(y, t, n, dy, loss);
  return cudaGetLastError() == cudaSuccess ? TT_MLP_OK : TT_MLP_CUDA;
}

extern "C" int tt_mlp_adam(float* p, const float* g, float* m, float* v, long long n, float lr, float beta1,
                           float beta2, float eps, int step, void* stream) {
  if (!p || !g || !m || !v || n < 0 || step < 1) return TT_MLP_INVALID;
  const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
  adam_kernel<<<blocks(n, 256), 256, 0, (cudaStream_t)stream>>>(p, g, m, v, n, lr, beta1, beta2, eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? TT_MLP_OK : TT_MLP_CUDA;
}

extern "C" int tt_mlp_to_bf16(const float* src, uint16_t* dst, long long n, void* stream) {
  if (!src || !dst || n < 0) return TT_MLP_INVALID;
  bf16_kernel<<<blocks(n, 256), 256, 0, (cudaStream_t)stream>>>(src, reinterpret_cast<__nv_bfloat16*>(dst), n);
  return cudaGetLastError() == cudaSuccess ? TT_MLP_OK : TT_MLP_CUDA;
}

extern "C" int tt_mlp_ensemble(const float* preds, int members, int n, float* mean, float* spread, void* stream) {
  if (!preds || !mean || !spread || members < 1 || n < 0) return TT_MLP_INVALID;
  if (n == 0) return TT_MLP_OK;
  ensemble_kernel<<<blocks(n, 256), 256, 0, (cudaStream_t)stream>>>(preds, members, n, mean, spread);
  return cudaGetLastError() == cudaSuccess ? TT_MLP_OK : TT_MLP_CUDA;
}

extern "C" int tt_mlp_gather(const float* src, const int* idx, int rows, int cols, float* dst, void* stream) {
  if (!src || !idx || !dst || rows < 0 || cols < 1) return TT_MLP_INVALID;
  if (rows == 0) return TT_MLP_OK;
  gather_kernel<<<blocks((long)rows * cols, 256), 256, 0, (cudaStream_t)stream>>>(src, idx, rows, cols, dst);
  return cudaGetLastError() == cudaSuccess ? TT_MLP_OK : TT_MLP_CUDA;
}
