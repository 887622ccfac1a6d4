// Learned cost surrogate for candidate screening (not in the paper).
//
// An MLP x -> score with x = [theta normalised to [-1, 1] and zero-padded to
// 32 | 16 scene features], `depth` hidden layers Linear + GELU (erf form) of
// width `width`, a scalar linear output, and an affine de-normalisation
// score = mu + sigma * out.  Weights and activations are BF16, products
// accumulate in FP32, the optimiser keeps FP32 master weights (AdamW,
// decoupled decay on weights).  Each CE iteration can then draw a large
// candidate pool, score it, and roll out only the best-scored candidates;
// elites still come from simulated costs only.
//
// Dense layers run on the tensor cores through one tiled GEMM kernel
// (128 x 128 x 32 tiles, 8 warps, mma m16n8k16 BF16 -> FP32) with fused
// epilogues: bias + GELU (forward, also keeping the FP32 pre-activation for
// the backward pass) and GELU' (backward).  Every reduction (loss, bias and
// output-layer gradients, target statistics) runs in a fixed order, so
// training is run-to-run deterministic.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "gelu.cuh"
#include "internal.h"

using namespace cem;

namespace {

typedef __nv_bfloat16 bf16;

int fail(int code, const std::string& m) { return set_last_error(code, m); }

#define SUR_CUDA(call)                                                                                   \
  do {                                                                                                   \
    cudaError_t e_ = (call);                                                                             \
    if (e_ != cudaSuccess)                                                                               \
      return fail(e_ == cudaErrorMemoryAllocation ? CEM_ERR_NO_MEMORY : CEM_ERR_CUDA,                    \
                  std::string(#call ": ") + cudaGetErrorString(e_));                                     \
  } while (0)


// ---------------------------------------------------------------- GEMM
// C[M x N] = op(A)[M x K] * op(B)[K x N] on BF16 tensor cores, FP32 accumulate.
// op(A)(m, k) = a_kmajor ? A[m * lda + k] : A[k * lda + m]
// op(B)(k, n) = b_kmajor ? B[n * ldb + k] : B[k * ldb + n]
constexpr int BM = 128, BN = 128, BK = 32, PADK = 8, GT = 256;

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <int EPI>
__global__ void __launch_bounds__(GT) gemm_bf16_kernel(GemmArgs g) {
  __shared__ __align__(16) bf16 As[BM][BK + PADK];
  __shared__ __align__(16) bf16 Bs[BN][BK + PADK];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = warp >> 2, wn = warp & 3, gq = lane >> 2, tq = lane & 3;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  float acc[4][4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0f;
  const bf16 zero = __float2bfloat16_rn(0.0f);
  const int kbeg = g.kchunk > 0 ? (int)blockIdx.z * g.kchunk : 0;
  const int kend = g.kchunk > 0 ? min(g.K, kbeg + g.kchunk) : g.K;
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll 4
    for (int i = 0; i < BM * BK / GT; ++i) {
      const int e = tid + i * GT;
      const int r = g.a_kmajor ? e / BK : e % BM;
      const int c = g.a_kmajor ? e % BK : e / BM;
      const int m = m0 + r, k = k0 + c;
      bf16 v = zero;
      if (m < g.M && k < kend) v = g.a_kmajor ? g.A[(size_t)m * g.lda + k] : g.A[(size_t)k * g.lda + m];
      As[r][c] = v;
    }
#pragma unroll 4
    for (int i = 0; i < BN * BK / GT; ++i) {
      const int e = tid + i * GT;
      const int r = g.b_kmajor ? e / BK : e % BN;
      const int c = g.b_kmajor ? e % BK : e / BN;
      const int n = n0 + r, k = k0 + c;
      bf16 v = zero;
      if (n < g.N && k < kend) v = g.b_kmajor ? g.B[(size_t)n * g.ldb + k] : g.B[(size_t)k * g.ldb + n];
      Bs[r][c] = v;
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < BK; ks += 16) {
      uint32_t af[4][4], bfr[4][2];
#pragma unroll
      for (int mt = 0; mt < 4; ++mt) {
        const int r = wm * 64 + mt * 16 + gq;
        af[mt][0] = *reinterpret_cast<const uint32_t*>(&As[r][ks + 2 * tq]);
        af[mt][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][ks + 2 * tq]);
        af[mt][2] = *reinterpret_cast<const uint32_t*>(&As[r][ks + 2 * tq + 8]);
        af[mt][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][ks + 2 * tq + 8]);
      }
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int n = wn * 32 + nt * 8 + gq;
        bfr[nt][0] = *reinterpret_cast<const uint32_t*>(&Bs[n][ks + 2 * tq]);
        bfr[nt][1] = *reinterpret_cast<const uint32_t*>(&Bs[n][ks + 2 * tq + 8]);
      }
#pragma unroll
      for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mt][nt], af[mt], bfr[nt]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int mt = 0; mt < 4; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int m = m0 + wm * 64 + mt * 16 + gq + (q >= 2 ? 8 : 0);
        const int n = n0 + wn * 32 + nt * 8 + 2 * tq + (q & 1);
        if (m >= g.M || n >= g.N) continue;
        const float v = acc[mt][nt][q];
        if (EPI == EPI_F32) {
          if (g.part) g.part[((size_t)blockIdx.z * g.M + m) * g.N + n] = v;
          else g.C[(size_t)m * g.ldc + n] = v;
        } else if (EPI == EPI_BIAS_GELU) {
          const float z = v + g.bias[n];
          if (g.C) g.C[(size_t)m * g.ldc + n] = z;
          g.Cb[(size_t)m * g.ldcb + n] = __float2bfloat16_rn(gelu(z));
        } else {
          g.Cb[(size_t)m * g.ldcb + n] = __float2bfloat16_rn(v * gelu_grad(g.zsave[(size_t)m * g.ldz + n]));
        }
      }
}

// C[m, n] = sum over z of part[z][m][n], in z order; with n_real > 0 the
// columns >= n_real are the appended ones column (n_real -> cbias[m]) and padding
__global__ void splitk_sum_kernel(const float* __restrict__ part, int S, int M, int N, float* __restrict__ C, int ldc,
                                  int n_real, float* __restrict__ cbias) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M * N) return;
  const int m = i / N, n = i % N;
  if (n_real > 0 && n > n_real) return;
  float acc = 0.0f;
  for (int z = 0; z < S; ++z) acc += part[(size_t)z * M * N + i];
  if (n_real > 0 && n == n_real) cbias[m] = acc;
  else C[(size_t)m * ldc + n] = acc;
}

// tc: run the product on tcgen05 (csrc/gemm_tc.cu) when its shape allows,
// else on the tiled mma.sync kernel above; status: the tcgen05 path's
// expired-wait flag
template <int EPI>
cudaError_t gemm(const GemmArgs& g, bool tc, int* status, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  const int S = (EPI == EPI_F32 && g.part && g.kchunk > 0) ? (g.K + g.kchunk - 1) / g.kchunk : 1;
  GemmArgs h = g;
  if (S == 1) {  // one chunk: write C directly
    h.kchunk = 0;
    h.part = nullptr;
  }
  cudaError_t e;
  if (tc && gemm_tc_supported(h)) {
    e = gemm_tc(EPI, h, status, st);
  } else if (g.n_real > 0) {
    return cudaErrorInvalidValue;  // the ones column exists on the tcgen05 path only
  } else {
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, S);
    gemm_bf16_kernel<EPI><<<grid, GT, 0, st>>>(h);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess || S == 1 || EPI != EPI_F32) return e;
  splitk_sum_kernel<<<(g.M * g.N + 255) / 256, 256, 0, st>>>(g.part, S, g.M, g.N, g.C, g.ldc, g.n_real, g.cbias);
  return cudaGetLastError();
}

// split of a K-long reduction into at most kMaxSplit chunks of >= 256 rows
// (a multiple of the K tile), so the weight-gradient GEMMs fill the GPU
constexpr int kMaxSplit = 32;
int split_chunk(int K) {
  int S = (K + 255) / 256;
  if (S > kMaxSplit) S = kMaxSplit;
  if (S < 1) S = 1;
  const int c = (K + S - 1) / S;
  return (c + BK - 1) / BK * BK;
}

// -------------------------------------------------------------- small kernels
// out = mu + sigma * (a . w + b) for each row of a [M x W] (one warp per row)
__global__ void output_layer_kernel(const bf16* __restrict__ a, int M, int W, const bf16* __restrict__ w,
                                    const float* __restrict__ b, const float* __restrict__ norm, float* __restrict__ y,
                                    float* __restrict__ raw) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (row >= M) return;
  float s = 0.0f;
  for (int j = lane; j < W; j += 32)
    s = fmaf(__bfloat162float(a[(size_t)row * W + j]), __bfloat162float(w[j]), s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    const float r = s + b[0];
    if (raw) raw[row] = r;
    if (y) y[row] = norm[0] + norm[1] * r;
  }
}

// dy = 2 (raw - (t - mu) / sigma) / B and per-block partial sums of the squared residual
__global__ void loss_kernel(const float* __restrict__ raw, const float* __restrict__ t, const float* __restrict__ norm,
                            int B, float* __restrict__ dy, float* __restrict__ partial) {
  __shared__ float red[256];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float sq = 0.0f;
  if (i < B) {
    const float r = raw[i] - (t[i] - norm[0]) / norm[1];
    dy[i] = 2.0f * r / (float)B;
    sq = r * r;
  }
  red[threadIdx.x] = sq;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// Column sums in two deterministic stages: block (x, z) sums rows
// [64 z, 64 z + 64) of 32 columns (8 row threads per column, rows in a fixed
// interleave, then the 8 partials in order) into part[z][j]; a second pass
// adds part[0..S)[j] the same way (8 interleaved runs, then their sums in
// order).
constexpr int kColRows = 64;  // rows per first-stage block

__global__ void __launch_bounds__(256) colsum_part_kernel(const bf16* __restrict__ X, const float* __restrict__ w,
                                                          int M, int N, float* __restrict__ part) {
  __shared__ float red[8][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + tx, m0 = blockIdx.y * kColRows;
  float acc = 0.0f;
  if (j < N)
#pragma unroll
    for (int r = ty; r < kColRows; r += 8) {
      const int m = m0 + r;
      if (m < M) acc = fmaf(w ? w[m] : 1.0f, __bfloat162float(X[(size_t)m * N + j]), acc);
    }
  red[ty][tx] = acc;
  __syncthreads();
  if (ty == 0 && j < N) {
    float t = 0.0f;
    for (int q = 0; q < 8; ++q) t += red[q][tx];
    part[(size_t)blockIdx.y * N + j] = t;
  }
}

// second stage: 8 row threads per column add partials z = ty, ty + 8, ...
// in order, then the 8 sums are added in order
__global__ void __launch_bounds__(256) colsum_finish_kernel(const float* __restrict__ part, int S, int N,
                                                            float* __restrict__ out) {
  __shared__ float red[8][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + tx;
  float t = 0.0f;
  if (j < N)
    for (int z = ty; z < S; z += 8) t += part[(size_t)z * N + j];
  red[ty][tx] = t;
  __syncthreads();
  if (ty == 0 && j < N) {
    float u = 0.0f;
    for (int q = 0; q < 8; ++q) u += red[q][tx];
    out[j] = u;
  }
}

// out[j] = sum_m w[m] X[m][j] (w = 1 if null) with the two kernels above;
// `part` holds ceil(M / kColRows) x N floats
cudaError_t colsum(const bf16* X, const float* w, int M, int N, float* out, float* part, cudaStream_t st) {
  const int S = (M + kColRows - 1) / kColRows;
  colsum_part_kernel<<<dim3((N + 31) / 32, S), 256, 0, st>>>(X, w, M, N, part);
  colsum_finish_kernel<<<(N + 31) / 32, 256, 0, st>>>(part, S, N, out);
  return cudaGetLastError();
}

// dz[m][j] = dy[m] * w[j] * gelu'(z[m][j]) (the output layer's input gradient)
__global__ void output_backward_kernel(const float* __restrict__ dy, const bf16* __restrict__ w,
                                       const float* __restrict__ z, int M, int W, bf16* __restrict__ dz) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)M * W) return;
  const int m = (int)(i / W), j = (int)(i % W);
  dz[i] = __float2bfloat16_rn(dy[m] * __bfloat162float(w[j]) * gelu_grad(z[i]));
}

// sum of `n` partials (single block, fixed order)
__global__ void finish_sum_kernel(const float* __restrict__ partial, int n, float* __restrict__ out) {
  __shared__ float red[256];
  float s = 0.0f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

// mean and standard deviation of t[M] in FP64 (single block, fixed order):
// norm[0] = mean, norm[1] = std (1 if degenerate)
__global__ void target_stats_kernel(const float* __restrict__ t, int M, float* __restrict__ norm) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < M; i += blockDim.x) s += t[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  const double mean = red[0] / M;
  __syncthreads();
  s = 0.0;
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    const double d = t[i] - mean;
    s += d * d;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double sd = sqrt(red[0] / M);
    norm[0] = (float)mean;
    norm[1] = sd > 1e-12 ? (float)sd : 1.0f;
  }
}

struct Segs {
  int n;
  int off[20], len[20], decay[20];
};

// AdamW on the FP32 master parameters, then refresh their BF16 copies
// adam_t_d: AdamW steps taken before this one (device counter, see step_end_kernel)
// end of a training step: record the batch loss, advance both counters
__global__ void step_end_kernel(int* __restrict__ step_d, long long* __restrict__ adam_t_d,
                                const float* __restrict__ loss_d, float* __restrict__ hist_d) {
  if (hist_d) hist_d[*step_d] = *loss_d;
  *step_d += 1;
  *adam_t_d += 1;
}

__global__ void adamw_kernel(float* __restrict__ p, const float* __restrict__ grad, float* __restrict__ m1,
                             float* __restrict__ m2, bf16* __restrict__ pb, int total, Segs segs, float lr, float b1,
                             float b2, float eps, float wd, const long long* __restrict__ adam_t_d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const float tstep = (float)(*adam_t_d + 1);
  const float c1 = 1.0f - powf(b1, tstep), c2 = 1.0f - powf(b2, tstep);
  int decay = 0;
  for (int s = 0; s < segs.n; ++s)
    if (i >= segs.off[s] && i < segs.off[s] + segs.len[s]) decay = segs.decay[s];
  const float g = grad[i];
  const float a = b1 * m1[i] + (1.0f - b1) * g;
  const float v = b2 * m2[i] + (1.0f - b2) * g * g;
  m1[i] = a;
  m2[i] = v;
  float x = p[i];
  x = x - lr * (decay ? wd : 0.0f) * x - lr * (a / c1) / (sqrtf(v / c2) + eps);
  p[i] = x;
  pb[i] = __float2bfloat16_rn(x);
}

__global__ void to_bf16_kernel(const float* __restrict__ x, size_t n, bf16* __restrict__ y) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = __float2bfloat16_rn(x[i]);
}

// features of N parameter vectors: [clamp(theta) normalised | 0 | scene16]
template <typename TOut>
__global__ void features_kernel(const float* __restrict__ theta, int N, int D, const float* __restrict__ lohi,
                                const float* __restrict__ scene16, TOut* __restrict__ x) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  TOut* o = x + (size_t)n * 48;
  for (int j = 0; j < 48; ++j) {
    float v = 0.0f;
    if (j < D) {
      const float lo = lohi[j], hi = lohi[CEM_MAX_D + j];
      const float t = fminf(fmaxf(theta[(size_t)n * D + j], lo), hi);
      v = hi > lo ? (t - 0.5f * (lo + hi)) / (0.5f * (hi - lo)) : 0.0f;
    } else if (j >= 32) {
      v = scene16[j - 32];
    }
    o[j] = (TOut)v;
  }
}

// minibatch of B rows drawn with replacement (Philox on (step, i)); gathers x and t
// step: the training call's step counter on the device (so one captured
// step replays with a new batch each time)
__global__ void gather_batch_kernel(const bf16* __restrict__ X, const float* __restrict__ t, int M, int in_dim,
                                    int B, uint64_t seed, const int* __restrict__ step_d, bf16* __restrict__ xb,
                                    float* __restrict__ tb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B) return;
  const uint32_t step = (uint32_t)*step_d;
  // one Philox block per row: the first word picks the row
  uint32_t c0 = (uint32_t)i, c1 = step, c2 = 0x5AFEu, c3 = 0u, k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    if (r < 9) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
  }
  const int row = (int)(((uint64_t)c0 * (uint64_t)M) >> 32);
  for (int j = 0; j < in_dim; ++j) xb[(size_t)i * in_dim + j] = X[(size_t)row * in_dim + j];
  tb[i] = t[row];
}

// ---------------------------------------------------------------- top-k
__device__ __forceinline__ uint32_t order_bits(float x) {
  const uint32_t u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ uint64_t score_key(const float* s, int i) {
  float v = s[i];
  if (!isfinite(v)) v = __int_as_float(0x7f800000);
  v = v + 0.0f;
  return ((uint64_t)order_bits(v) << 20) | (uint64_t)i;
}

// indices of the `keep` lowest scores (ties by index), written in ascending
// index order; one CTA of 1024 threads (radix select, then an ordered scan)
__global__ void __launch_bounds__(1024) topk_kernel(const float* __restrict__ score, int N, int keep,
                                                    int32_t* __restrict__ idx) {
  __shared__ uint32_t hist[256];
  __shared__ uint64_t s_prefix, s_mask;
  __shared__ int s_rank;
  __shared__ int warp_tot[32];
  const int tid = threadIdx.x;
  if (tid == 0) {
    s_prefix = 0;
    s_mask = 0;
    s_rank = keep;
  }
  __syncthreads();
  uint64_t kth = ~0ull;
  if (keep < N) {
    int shift = 52;
    while (shift > 0) {
      const int width = shift >= 8 ? 8 : shift;
      shift -= width;
      for (int d = tid; d < 256; d += 1024) hist[d] = 0;
      __syncthreads();
      const uint64_t prefix = s_prefix, mask = s_mask;
      for (int i = tid; i < N; i += 1024) {
        const uint64_t key = score_key(score, i);
        if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & ((1u << width) - 1)], 1u);
      }
      __syncthreads();
      if (tid == 0) {
        uint32_t cum = 0;
        int d = 0;
        for (; d < (1 << width); ++d) {
          if (cum + hist[d] >= (uint32_t)s_rank) break;
          cum += hist[d];
        }
        s_rank -= (int)cum;
        s_prefix |= (uint64_t)d << shift;
        s_mask |= (uint64_t)((1u << width) - 1) << shift;
      }
      __syncthreads();
    }
    kth = s_prefix;
  }
  // ordered compaction: thread tid owns the contiguous range [tid*per, (tid+1)*per)
  const int per = (N + 1023) / 1024;
  const int b = tid * per, e = min(N, b + per);
  int cnt = 0;
  for (int i = b; i < e; ++i) cnt += score_key(score, i) <= kth;
  // exclusive scan of cnt over the block
  int x = cnt;
  const int lane = tid & 31, w = tid >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    int t = warp_tot[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    warp_tot[lane] = t;
  }
  __syncthreads();
  int pos = x - cnt + (w > 0 ? warp_tot[w - 1] : 0);
  for (int i = b; i < e; ++i)
    if (score_key(score, i) <= kth) {
      if (pos < keep) idx[pos] = i;
      ++pos;
    }
}

// the first n_explore pool entries are kept whatever their score (unscreened
// draws from the current distribution): give them the lowest finite score
__global__ void force_keep_kernel(float* __restrict__ score, int n_explore) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_explore) score[i] = -3.402823466e38f;
}

// training target of a simulated sample: log(1 + max(J, 0) + 10 * class),
// which orders samples like the CE key (class first) while costs stay below
// 10, and compresses large costs
__global__ void score_target_kernel(const float* __restrict__ J, const uint8_t* __restrict__ cls, int N,
                                    float* __restrict__ t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float j = J[i];
  t[i] = isfinite(j) ? log1pf(fmaxf(j, 0.0f) + 10.0f * (float)cls[i]) : log1pf(1e6f);
}

__global__ void gather_rows_kernel(const float* __restrict__ src, int n_src, const int32_t* __restrict__ idx, int n,
                                   int D, float* __restrict__ dst) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * D) return;
  const int r = t / D, c = t % D;
  dst[t] = src[(size_t)CEM_DIDX(idx[r], n_src, 9) * D + c];
}

// ---- FP32 debug path (gemm path 3): every input, weight, activation and
// gradient in FP32 and every reduction in ascending index order, one output
// element per thread.  Slow; it exists to check gradients against an exact
// FP64 chain rule without the BF16 rounding of the fast paths.  The sums use
// the compensated dot product Dot2 of Ogita, Rump and Oishi ("Accurate sum
// and dot product", SIAM J. Sci. Comput. 26, 2005): each product's rounding
// error from an FMA, each addition's from TwoSum, both carried in a second
// accumulator, so a sum of thousands of rows is as accurate as if formed in
// twice the working precision and only the elementwise FP32 functions
// (GELU, GELU') limit the result.  Explicit-rounding intrinsics keep the
// compiler from fusing the steps.
struct Dot2 {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float ep = __fmaf_rn(a, b, -p);  // a b = p + ep exactly
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, s);
    const float es = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));  // s + p = t + es exactly
    s = t;
    c = __fadd_rn(c, __fadd_rn(es, ep));
  }
  __device__ __forceinline__ float value() const { return __fadd_rn(s, c); }
};
struct GemmF32 {
  int M, N, K;
  const float* A;
  int lda, a_kmajor;
  const float* B;
  int ldb, b_kmajor;
  float* C;  // EPI_F32: product; EPI_BIAS_GELU: pre-activation z
  int ldc;
  float* Cf;  // EPI_BIAS_GELU: GELU(z); EPI_GELU_BWD: product * GELU'(zsave)
  int ldcf;
  const float* bias;
  const float* zsave;
  int ldz;
};

template <int EPI>
__global__ void __launch_bounds__(256) gemm_f32_kernel(GemmF32 g) {
  __shared__ float As[16][17], Bs[16][17];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m = blockIdx.y * 16 + ty, n = blockIdx.x * 16 + tx;
  Dot2 dot;
  for (int k0 = 0; k0 < g.K; k0 += 16) {
    const int ak = k0 + tx, bk = k0 + ty, bn = blockIdx.x * 16 + tx;
    As[ty][tx] = (m < g.M && ak < g.K) ? (g.a_kmajor ? g.A[(size_t)m * g.lda + ak] : g.A[(size_t)ak * g.lda + m]) : 0.0f;
    Bs[ty][tx] = (bk < g.K && bn < g.N) ? (g.b_kmajor ? g.B[(size_t)bn * g.ldb + bk] : g.B[(size_t)bk * g.ldb + bn])
                                        : 0.0f;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) dot.add(As[ty][kk], Bs[kk][tx]);
    __syncthreads();
  }
  if (m >= g.M || n >= g.N) return;
  const float acc = dot.value();
  if (EPI == EPI_F32) {
    g.C[(size_t)m * g.ldc + n] = acc;
  } else if (EPI == EPI_BIAS_GELU) {
    dot.add(g.bias[n], 1.0f);
    const float z = dot.value();
    g.C[(size_t)m * g.ldc + n] = z;
    g.Cf[(size_t)m * g.ldcf + n] = gelu(z);
  } else {
    g.Cf[(size_t)m * g.ldcf + n] = acc * gelu_grad(g.zsave[(size_t)m * g.ldz + n]);
  }
}

template <int EPI>
cudaError_t gemm_f32(const GemmF32& g, cudaStream_t st) {
  gemm_f32_kernel<EPI><<<dim3((g.N + 15) / 16, (g.M + 15) / 16), 256, 0, st>>>(g);
  return cudaGetLastError();
}

// raw[m] = sum_j a[m][j] w[j] + b (FP32, j ascending)
__global__ void output_layer_f32_kernel(const float* __restrict__ a, int M, int W, const float* __restrict__ w,
                                        const float* __restrict__ b, float* __restrict__ raw) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  Dot2 dot;
  for (int j = 0; j < W; ++j) dot.add(a[(size_t)m * W + j], w[j]);
  dot.add(b[0], 1.0f);
  raw[m] = dot.value();
}

// out[j] = sum_m (w ? w[m] : 1) X[m][j] (FP32, m ascending)
__global__ void colsum_f32_kernel(const float* __restrict__ X, const float* __restrict__ w, int M, int N,
                                  float* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  Dot2 dot;
  for (int m = 0; m < M; ++m) dot.add(w ? w[m] : 1.0f, X[(size_t)m * N + j]);
  out[j] = dot.value();
}

// dz[m][j] = dy[m] w[j] GELU'(z[m][j]) (FP32)
__global__ void output_backward_f32_kernel(const float* __restrict__ dy, const float* __restrict__ w,
                                           const float* __restrict__ z, int M, int W, float* __restrict__ dz) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)M * W) return;
  const int m = (int)(i / W), j = (int)(i % W);
  dz[i] = dy[m] * w[j] * gelu_grad(z[i]);
}

}  // namespace

// ------------------------------------------------------------------ handle
struct cem_surrogate_ctx {
  int in_dim = 48, width = 256, depth = 4, n_layers = 5;
  std::vector<int> w_off, b_off, fan_in, fan_out;  // per layer offsets into the flat parameter vector
  int total = 0;
  float* p = nullptr;   // FP32 master parameters
  bf16* pb = nullptr;   // BF16 copy (same layout)
  float* g = nullptr;   // gradient
  float* m1 = nullptr;  // Adam moments
  float* m2 = nullptr;
  float* norm = nullptr;  // [mu, sigma] of the score
  long long adam_step = 0;
  // activation workspace for up to cap_M rows
  int cap_M = 0;
  bf16* xin = nullptr;
  std::vector<bf16*> act;  // depth buffers [cap_M x width]
  std::vector<float*> pre;  // depth buffers [cap_M x width] (pre-activations)
  bf16* dz_a = nullptr;
  bf16* dz_b = nullptr;
  float* raw = nullptr;
  float* dy = nullptr;
  float* tb = nullptr;
  float* partial = nullptr;
  float* loss_d = nullptr;
  float* splitk = nullptr;   // split-K partials of the weight gradients
  float* colpart = nullptr;  // row-chunk partials of the bias gradients
  // screening workspace
  int cap_pool = 0;
  float* pool_theta = nullptr;
  bf16* pool_x = nullptr;
  float* pool_score = nullptr;
  int32_t* keep_idx = nullptr;
  float* lohi = nullptr;
  float* scene16 = nullptr;
  // fused tcgen05 forward: packed weights (rebuilt when the BF16 weights
  // change), status word of its bounded waits, path selection
  void* tc_pack = nullptr;
  int* tc_status = nullptr;
  int* step_d = nullptr;         // training: step of the current cem_surrogate_train call
  long long* adam_t_d = nullptr;  // training: AdamW steps taken (mirrors adam_step)
  bool tc_pack_valid = false;
  int fwd_path = 0;   // 0 automatic, 1 tiled GEMM, 2 tcgen05
  int gemm_path = 0;  // training GEMMs: 0 automatic (tcgen05 where the shape allows), 1 tiled mma.sync
  int expire_test = 0;
};

namespace {

void sur_free_work(cem_surrogate_ctx* s) {
  cudaFree(s->xin);
  for (auto* a : s->act) cudaFree(a);
  for (auto* a : s->pre) cudaFree(a);
  s->act.clear();
  s->pre.clear();
  cudaFree(s->dz_a);
  cudaFree(s->dz_b);
  cudaFree(s->raw);
  cudaFree(s->dy);
  cudaFree(s->tb);
  cudaFree(s->partial);
  cudaFree(s->loss_d);
  cudaFree(s->splitk);
  cudaFree(s->colpart);
  s->splitk = nullptr;
  s->colpart = nullptr;
  s->xin = nullptr;
  s->dz_a = s->dz_b = nullptr;
  s->raw = s->dy = s->tb = s->partial = s->loss_d = nullptr;
  s->cap_M = 0;
}

int ensure_rows(cem_surrogate_ctx* s, int M) {
  if (M <= s->cap_M) return CEM_OK;
  sur_free_work(s);
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t b) {
    if (e == cudaSuccess) e = dev_malloc(p, b);
  };
  A((void**)&s->xin, sizeof(bf16) * (size_t)M * s->in_dim);
  s->act.assign(s->depth, nullptr);
  s->pre.assign(s->depth, nullptr);
  for (int l = 0; l < s->depth; ++l) {
    A((void**)&s->act[l], sizeof(bf16) * (size_t)M * s->width);
    A((void**)&s->pre[l], sizeof(float) * (size_t)M * s->width);
  }
  A((void**)&s->dz_a, sizeof(bf16) * (size_t)M * s->width);
  A((void**)&s->dz_b, sizeof(bf16) * (size_t)M * s->width);
  A((void**)&s->raw, sizeof(float) * M);
  A((void**)&s->dy, sizeof(float) * M);
  A((void**)&s->tb, sizeof(float) * M);
  A((void**)&s->partial, sizeof(float) * ((M + 255) / 256 + 1));
  A((void**)&s->loss_d, sizeof(float));
  A((void**)&s->splitk, sizeof(float) * (size_t)kMaxSplit * s->width * (std::max(s->width, s->in_dim) + 16));
  A((void**)&s->colpart, sizeof(float) * (size_t)((M + kColRows - 1) / kColRows) * s->width);
  if (e != cudaSuccess) {
    cudaGetLastError();
    sur_free_work(s);
    return fail(CEM_ERR_NO_MEMORY, "surrogate workspace allocation failed");
  }
  s->cap_M = M;
  return CEM_OK;
}

// forward of M rows already in s->xin (BF16); keeps activations for backward
// tc: the dense layers on the tcgen05 GEMM (else the tiled mma.sync kernel)
cudaError_t forward_rows(cem_surrogate_ctx* s, int M, float* y, bool tc, cudaStream_t st) {
  const bf16* a = s->xin;
  int K = s->in_dim;
  for (int l = 0; l < s->depth; ++l) {
    GemmArgs g;
    std::memset(&g, 0, sizeof(g));
    g.M = M;
    g.N = s->width;
    g.K = K;
    g.A = a;
    g.lda = K;
    g.a_kmajor = 1;
    g.B = s->pb + s->w_off[l];
    g.ldb = K;
    g.b_kmajor = 1;
    g.C = s->pre[l];
    g.ldc = s->width;
    g.Cb = s->act[l];
    g.ldcb = s->width;
    g.bias = s->p + s->b_off[l];
    cudaError_t e = gemm<EPI_BIAS_GELU>(g, tc, s->tc_status, st);
    if (e != cudaSuccess) return e;
    a = s->act[l];
    K = s->width;
  }
  const int L = s->depth;
  const int threads = 256;
  output_layer_kernel<<<(M * 32 + threads - 1) / threads, threads, 0, st>>>(
      a, M, s->width, s->pb + s->w_off[L], s->p + s->b_off[L], s->norm, y, s->raw);
  return cudaGetLastError();
}

bool use_tc_gemm(const cem_surrogate_ctx* s) { return s->gemm_path != 1; }

bool use_tc(const cem_surrogate_ctx* s) {
  return s->fwd_path != 1 && mlp_tc_supported(s->in_dim, s->width, s->depth);
}

// scores of M rows, no activations kept: the fused tcgen05 kernel where the
// shape allows, else the tiled GEMM forward.  The rows are BF16 in s->xin,
// or (tcgen05 kernel only) FP32 in xf, which the kernel rounds as it loads.
cudaError_t infer_rows(cem_surrogate_ctx* s, int M, float* y, cudaStream_t st, const float* xf = nullptr) {
  if (!use_tc(s)) return forward_rows(s, M, y, s->fwd_path != 1 && use_tc_gemm(s), st);
  if (!s->tc_pack_valid) {
    MlpTcOffsets off;
    for (int l = 0; l < 4; ++l) off.w[l] = s->w_off[l];
    cudaError_t e = mlp_tc_pack(s->pb, off, s->tc_pack, st);
    if (e != cudaSuccess) return e;
    s->tc_pack_valid = true;
  }
  MlpTcArgs a;
  a.x = s->xin;
  a.xf = xf;
  a.M = M;
  a.wpack = s->tc_pack;
  for (int l = 0; l < 4; ++l) a.bias[l] = s->p + s->b_off[l];
  a.w_out = s->pb + s->w_off[4];
  a.b_out = s->p + s->b_off[4];
  a.norm = s->norm;
  a.y = y;
  a.status = s->tc_status;
  a.expire_test = s->expire_test;
  return mlp_tc_forward(a, st);
}

// gradient of mean((raw - (t - mu)/sigma)^2) for the M rows of the last forward;
// targets in s->tb
cudaError_t backward_rows(cem_surrogate_ctx* s, int M, cudaStream_t st) {
  const int L = s->depth, W = s->width;
  const int blocks = (M + 255) / 256;
  loss_kernel<<<blocks, 256, 0, st>>>(s->raw, s->tb, s->norm, M, s->dy, s->partial);
  finish_sum_kernel<<<1, 256, 0, st>>>(s->partial, blocks, s->loss_d);
  // output layer: dW = dy . a_{L-1}, db = sum dy
  cudaError_t ce = colsum(s->act[L - 1], s->dy, M, W, s->g + s->w_off[L], s->colpart, st);
  if (ce != cudaSuccess) return ce;
  finish_sum_kernel<<<1, 256, 0, st>>>(s->dy, M, s->g + s->b_off[L]);
  // dz of the last hidden layer
  const size_t n = (size_t)M * W;
  output_backward_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s->dy, s->pb + s->w_off[L], s->pre[L - 1], M, W,
                                                                      s->dz_a);
  bf16* dz = s->dz_a;
  bf16* dz_next = s->dz_b;
  for (int l = L - 1; l >= 0; --l) {
    const int K = l == 0 ? s->in_dim : W;
    const bf16* a_in = l == 0 ? s->xin : s->act[l - 1];
    GemmArgs g;  // dW_l [W x K] = dz^T a_in
    std::memset(&g, 0, sizeof(g));
    g.M = W;
    g.N = K;
    g.K = M;
    g.A = dz;
    g.lda = W;
    g.a_kmajor = 0;
    g.B = a_in;
    g.ldb = K;
    g.b_kmajor = 0;
    g.C = s->g + s->w_off[l];
    g.ldc = K;
    g.kchunk = split_chunk(M);
    g.part = s->splitk;
    // on tcgen05 the bias gradient db_l = sum over rows of dz rides along as
    // one more column (a row of ones appended to a_in^T); else a column sum
    GemmArgs ga = g;
    ga.N = K + 16;
    ga.n_real = K;
    ga.cbias = s->g + s->b_off[l];
    cudaError_t e;
    if (use_tc_gemm(s) && gemm_tc_supported(ga)) {
      e = gemm<EPI_F32>(ga, true, s->tc_status, st);
    } else {
      e = gemm<EPI_F32>(g, use_tc_gemm(s), s->tc_status, st);
      if (e == cudaSuccess) e = colsum(dz, nullptr, M, W, s->g + s->b_off[l], s->colpart, st);
    }
    if (e != cudaSuccess) return e;
    if (l > 0) {  // dz_{l-1} = (dz W_l) * gelu'(z_{l-1})
      GemmArgs h;
      std::memset(&h, 0, sizeof(h));
      h.M = M;
      h.N = K;
      h.K = W;
      h.A = dz;
      h.lda = W;
      h.a_kmajor = 1;
      h.B = s->pb + s->w_off[l];
      h.ldb = K;
      h.b_kmajor = 0;
      h.Cb = dz_next;
      h.ldcb = K;
      h.zsave = s->pre[l - 1];
      h.ldz = W;
      e = gemm<EPI_GELU_BWD>(h, use_tc_gemm(s), s->tc_status, st);
      if (e != cudaSuccess) return e;
      bf16* t = dz;
      dz = dz_next;
      dz_next = t;
    }
  }
  return cudaGetLastError();
}

// Gradient of mean((raw - (t - mu)/sigma)^2) over the M rows x_d, t_d in
// FP32 end to end (gemm path 3): FP32 inputs, the FP32 master weights,
// FP32 activations and gradients, the kernels above; the workspace beyond
// the shared row buffers is allocated for the call and freed after it.
int gradient_f32(cem_surrogate_ctx* s, const float* x_d, const float* t_d, int M) {
  int rc = ensure_rows(s, M);
  if (rc != CEM_OK) return rc;
  const int L = s->depth, W = s->width;
  std::vector<float*> act(L, nullptr);
  float* dz = nullptr;
  float* dz_next = nullptr;
  cudaError_t e = cudaSuccess;
  for (auto& a : act)
    if (e == cudaSuccess) e = dev_malloc(&a, sizeof(float) * (size_t)M * W);
  if (e == cudaSuccess) e = dev_malloc(&dz, sizeof(float) * (size_t)M * W);
  if (e == cudaSuccess) e = dev_malloc(&dz_next, sizeof(float) * (size_t)M * W);
  auto release = [&]() {
    for (auto* a : act) cudaFree(a);
    cudaFree(dz);
    cudaFree(dz_next);
  };
  if (e != cudaSuccess) {
    cudaGetLastError();
    release();
    return fail(CEM_ERR_NO_MEMORY, "FP32 gradient workspace allocation failed");
  }
  cudaStream_t st = 0;
  e = cudaMemcpyAsync(s->tb, t_d, sizeof(float) * M, cudaMemcpyDeviceToDevice, st);
  const float* a = x_d;
  int K = s->in_dim;
  for (int l = 0; l < L && e == cudaSuccess; ++l) {
    GemmF32 g;
    std::memset(&g, 0, sizeof(g));
    g.M = M;
    g.N = W;
    g.K = K;
    g.A = a;
    g.lda = K;
    g.a_kmajor = 1;
    g.B = s->p + s->w_off[l];
    g.ldb = K;
    g.b_kmajor = 1;
    g.C = s->pre[l];
    g.ldc = W;
    g.Cf = act[l];
    g.ldcf = W;
    g.bias = s->p + s->b_off[l];
    e = gemm_f32<EPI_BIAS_GELU>(g, st);
    a = act[l];
    K = W;
  }
  const int blocks = (M + 255) / 256;
  if (e == cudaSuccess) {
    output_layer_f32_kernel<<<blocks, 256, 0, st>>>(act[L - 1], M, W, s->p + s->w_off[L], s->p + s->b_off[L],
                                                     s->raw);
    loss_kernel<<<blocks, 256, 0, st>>>(s->raw, s->tb, s->norm, M, s->dy, s->partial);
    finish_sum_kernel<<<1, 256, 0, st>>>(s->partial, blocks, s->loss_d);
    colsum_f32_kernel<<<(W + 255) / 256, 256, 0, st>>>(act[L - 1], s->dy, M, W, s->g + s->w_off[L]);
    colsum_f32_kernel<<<1, 256, 0, st>>>(s->dy, nullptr, M, 1, s->g + s->b_off[L]);
    const size_t n = (size_t)M * W;
    output_backward_f32_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s->dy, s->p + s->w_off[L],
                                                                             s->pre[L - 1], M, W, dz);
    e = cudaGetLastError();
  }
  for (int l = L - 1; l >= 0 && e == cudaSuccess; --l) {
    const int Kl = l == 0 ? s->in_dim : W;
    const float* a_in = l == 0 ? x_d : act[l - 1];
    GemmF32 g;  // dW_l [W x Kl] = dz^T a_in
    std::memset(&g, 0, sizeof(g));
    g.M = W;
    g.N = Kl;
    g.K = M;
    g.A = dz;
    g.lda = W;
    g.a_kmajor = 0;
    g.B = a_in;
    g.ldb = Kl;
    g.b_kmajor = 0;
    g.C = s->g + s->w_off[l];
    g.ldc = Kl;
    e = gemm_f32<EPI_F32>(g, st);
    if (e == cudaSuccess) {
      colsum_f32_kernel<<<(W + 255) / 256, 256, 0, st>>>(dz, nullptr, M, W, s->g + s->b_off[l]);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess && l > 0) {  // dz_{l-1} = (dz W_l) * GELU'(z_{l-1})
      GemmF32 h;
      std::memset(&h, 0, sizeof(h));
      h.M = M;
      h.N = Kl;
      h.K = W;
      h.A = dz;
      h.lda = W;
      h.a_kmajor = 1;
      h.B = s->p + s->w_off[l];
      h.ldb = Kl;
      h.b_kmajor = 0;
      h.Cf = dz_next;
      h.ldcf = Kl;
      h.zsave = s->pre[l - 1];
      h.ldz = W;
      e = gemm_f32<EPI_GELU_BWD>(h, st);
      std::swap(dz, dz_next);
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  release();
  if (e != cudaSuccess) return fail(CEM_ERR_CUDA, std::string("FP32 gradient: ") + cudaGetErrorString(e));
  return CEM_OK;
}

Segs param_segments(const cem_surrogate_ctx* s) {
  Segs sg;
  std::memset(&sg, 0, sizeof(sg));
  for (int l = 0; l < s->n_layers; ++l) {
    sg.off[sg.n] = s->w_off[l];
    sg.len[sg.n] = s->fan_in[l] * s->fan_out[l];
    sg.decay[sg.n++] = 1;
    sg.off[sg.n] = s->b_off[l];
    sg.len[sg.n] = s->fan_out[l];
    sg.decay[sg.n++] = 0;
  }
  return sg;
}

int load_features(cem_surrogate_ctx* s, const float* x_d, int M, cudaStream_t st) {
  int rc = ensure_rows(s, M);
  if (rc != CEM_OK) return rc;
  const size_t n = (size_t)M * s->in_dim;
  to_bf16_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x_d, n, s->xin);
  SUR_CUDA(cudaGetLastError());
  return CEM_OK;
}

bool is_dev(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

int cem_surrogate_create(int in_dim, int width, int depth, uint64_t seed, cem_surrogate_handle* out) {
  set_last_error(CEM_OK, "");
  if (!out) return fail(CEM_ERR_INVALID_ARG, "out handle pointer is NULL");
  *out = nullptr;
  if (in_dim != 48) return fail(CEM_ERR_UNSUPPORTED, "the surrogate input is 48 wide (theta padded to 32 + 16 scene features)");
  if (width < 8 || width > 1024 || width % 8 || depth < 1 || depth > 8)
    return fail(CEM_ERR_UNSUPPORTED, "width in 8..1024 (multiple of 8), depth in 1..8");
  cem_surrogate_ctx* s = new cem_surrogate_ctx();
  s->in_dim = in_dim;
  s->width = width;
  s->depth = depth;
  s->n_layers = depth + 1;
  int o = 0;
  for (int l = 0; l < s->n_layers; ++l) {
    const int fi = l == 0 ? in_dim : width, fo = l == depth ? 1 : width;
    s->fan_in.push_back(fi);
    s->fan_out.push_back(fo);
    s->w_off.push_back(o);
    o += fi * fo;
    s->b_off.push_back(o);
    o += fo;
  }
  s->total = o;
  // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) from a seeded host generator
  std::vector<float> init(o);
  uint64_t st = seed * 6364136223846793005ull + 1442695040888963407ull;
  auto next = [&]() {  // 64-bit LCG, top 24 bits -> [0, 1)
    st = st * 6364136223846793005ull + 1442695040888963407ull;
    return (float)((st >> 40) & 0xFFFFFF) / 16777216.0f;
  };
  for (int l = 0; l < s->n_layers; ++l) {
    const float bound = 1.0f / std::sqrt((float)s->fan_in[l]);
    for (int i = 0; i < s->fan_in[l] * s->fan_out[l] + s->fan_out[l]; ++i)
      init[s->w_off[l] + i] = (2.0f * next() - 1.0f) * bound;
  }
  const float norm0[2] = {0.0f, 1.0f};
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t b) {
    if (e == cudaSuccess) e = dev_malloc(p, b);
  };
  A((void**)&s->p, sizeof(float) * o);
  A((void**)&s->pb, sizeof(bf16) * o);
  A((void**)&s->g, sizeof(float) * o);
  A((void**)&s->m1, sizeof(float) * o);
  A((void**)&s->m2, sizeof(float) * o);
  A((void**)&s->norm, sizeof(float) * 2);
  A((void**)&s->lohi, sizeof(float) * 2 * CEM_MAX_D);
  A((void**)&s->scene16, sizeof(float) * 16);
  if (mlp_tc_supported(in_dim, width, depth)) A(&s->tc_pack, mlp_tc_pack_bytes());
  A((void**)&s->tc_status, sizeof(int));
  A((void**)&s->step_d, sizeof(int));
  A((void**)&s->adam_t_d, sizeof(long long));
  if (e == cudaSuccess) e = cudaMemset(s->tc_status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(s->p, init.data(), sizeof(float) * o, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(s->m1, 0, sizeof(float) * o);
  if (e == cudaSuccess) e = cudaMemset(s->m2, 0, sizeof(float) * o);
  if (e == cudaSuccess) e = cudaMemcpy(s->norm, norm0, sizeof(norm0), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    to_bf16_kernel<<<(o + 255) / 256, 256>>>(s->p, (size_t)o, s->pb);
    e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    cem_surrogate_destroy(s);
    return fail(e == cudaErrorMemoryAllocation ? CEM_ERR_NO_MEMORY : CEM_ERR_CUDA,
                std::string("cem_surrogate_create: ") + cudaGetErrorString(e));
  }
  *out = s;
  return CEM_OK;
}

int cem_surrogate_destroy(cem_surrogate_handle s) {
  if (!s) return CEM_OK;
  cudaDeviceSynchronize();
  sur_free_work(s);
  void* ptrs[] = {s->p, s->pb, s->g, s->m1, s->m2, s->norm, s->lohi, s->scene16,
                  s->pool_theta, s->pool_x, s->pool_score, s->keep_idx, s->tc_pack, s->tc_status,
                  s->step_d, s->adam_t_d};
  for (void* p : ptrs) cudaFree(p);
  delete s;
  return CEM_OK;
}

int cem_surrogate_num_params(cem_surrogate_handle s) { return s ? s->total : 0; }

int cem_surrogate_set_params(cem_surrogate_handle s, const float* params_h, const float* norm_h) {
  if (!s || !params_h) return fail(CEM_ERR_INVALID_ARG, "null argument");
  SUR_CUDA(cudaMemcpy(s->p, params_h, sizeof(float) * s->total, cudaMemcpyHostToDevice));
  if (norm_h) SUR_CUDA(cudaMemcpy(s->norm, norm_h, sizeof(float) * 2, cudaMemcpyHostToDevice));
  to_bf16_kernel<<<(s->total + 255) / 256, 256>>>(s->p, (size_t)s->total, s->pb);
  s->tc_pack_valid = false;
  SUR_CUDA(cudaDeviceSynchronize());
  SUR_CUDA(cudaMemset(s->m1, 0, sizeof(float) * s->total));
  SUR_CUDA(cudaMemset(s->m2, 0, sizeof(float) * s->total));
  s->adam_step = 0;
  return CEM_OK;
}

int cem_surrogate_get_params(cem_surrogate_handle s, float* params_h, float* norm_h) {
  if (!s || !params_h) return fail(CEM_ERR_INVALID_ARG, "null argument");
  SUR_CUDA(cudaMemcpy(params_h, s->p, sizeof(float) * s->total, cudaMemcpyDeviceToHost));
  if (norm_h) SUR_CUDA(cudaMemcpy(norm_h, s->norm, sizeof(float) * 2, cudaMemcpyDeviceToHost));
  return CEM_OK;
}

int cem_surrogate_forward(cem_surrogate_handle s, const float* x_d, int M, float* y_d, void* stream) {
  if (!s) return fail(CEM_ERR_INVALID_ARG, "null handle");
  if (M < 0 || M > (1 << 22)) return fail(CEM_ERR_UNSUPPORTED, "M must be in 0..2^22");
  if (M == 0) return CEM_OK;
  if (!is_dev(x_d) || !is_dev(y_d)) return fail(CEM_ERR_INVALID_ARG, "x and y must be device pointers");
  cudaStream_t st = (cudaStream_t)stream;
  if (use_tc(s) && ((uintptr_t)x_d & 15u) == 0) {  // the fused kernel reads the FP32 rows itself
    SUR_CUDA(infer_rows(s, M, y_d, st, x_d));
    return CEM_OK;
  }
  int rc = load_features(s, x_d, M, st);
  if (rc != CEM_OK) return rc;
  SUR_CUDA(infer_rows(s, M, y_d, st));
  return CEM_OK;
}

int cem_surrogate_set_forward_path(cem_surrogate_handle s, int path) {
  if (!s) return fail(CEM_ERR_INVALID_ARG, "null handle");
  if (path < 0 || path > 2) return fail(CEM_ERR_INVALID_ARG, "path must be 0, 1 or 2");
  if (path == 2 && !mlp_tc_supported(s->in_dim, s->width, s->depth))
    return fail(CEM_ERR_UNSUPPORTED, "the tcgen05 forward needs width 256 and depth 4");
  s->fwd_path = path;
  return CEM_OK;
}

int cem_surrogate_test_expire_wait(cem_surrogate_handle s, int on) {
  if (!s) return fail(CEM_ERR_INVALID_ARG, "null handle");
  s->expire_test = on ? 1 : 0;
  return CEM_OK;
}

int cem_surrogate_forward_path(cem_surrogate_handle s) { return s ? (use_tc(s) ? 2 : 1) : -1; }

int cem_surrogate_set_gemm_path(cem_surrogate_handle s, int path) {
  if (!s) return fail(CEM_ERR_INVALID_ARG, "null handle");
  if (path < 0 || path > 3) return fail(CEM_ERR_INVALID_ARG, "path must be 0, 1, 2 or 3");
  s->gemm_path = path;
  return CEM_OK;
}

int cem_surrogate_gemm_path(cem_surrogate_handle s) {
  return s ? (s->gemm_path == 3 ? 3 : use_tc_gemm(s) ? 2 : 1) : -1;
}

int cem_surrogate_set_adam_state(cem_surrogate_handle s, const float* m1_h, const float* m2_h, long long steps_taken) {
  if (!s || !m1_h || !m2_h) return fail(CEM_ERR_INVALID_ARG, "null argument");
  if (steps_taken < 0) return fail(CEM_ERR_INVALID_ARG, "steps_taken must be >= 0");
  SUR_CUDA(cudaMemcpy(s->m1, m1_h, sizeof(float) * s->total, cudaMemcpyHostToDevice));
  SUR_CUDA(cudaMemcpy(s->m2, m2_h, sizeof(float) * s->total, cudaMemcpyHostToDevice));
  s->adam_step = steps_taken;
  return CEM_OK;
}

int cem_surrogate_get_adam_state(cem_surrogate_handle s, float* m1_h, float* m2_h, long long* steps_taken) {
  if (!s || !m1_h || !m2_h) return fail(CEM_ERR_INVALID_ARG, "null argument");
  SUR_CUDA(cudaDeviceSynchronize());
  SUR_CUDA(cudaMemcpy(m1_h, s->m1, sizeof(float) * s->total, cudaMemcpyDeviceToHost));
  SUR_CUDA(cudaMemcpy(m2_h, s->m2, sizeof(float) * s->total, cudaMemcpyDeviceToHost));
  if (steps_taken) *steps_taken = s->adam_step;
  return CEM_OK;
}

int cem_surrogate_adamw_step(cem_surrogate_handle s, const float* grad_h, float lr, float weight_decay) {
  if (!s || !grad_h) return fail(CEM_ERR_INVALID_ARG, "null argument");
  if (!(lr >= 0.0f) || !(weight_decay >= 0.0f)) return fail(CEM_ERR_INVALID_ARG, "lr and weight decay must be >= 0");
  SUR_CUDA(cudaMemcpy(s->g, grad_h, sizeof(float) * s->total, cudaMemcpyHostToDevice));
  SUR_CUDA(cudaMemcpy(s->adam_t_d, &s->adam_step, sizeof(long long), cudaMemcpyHostToDevice));
  const Segs segs = param_segments(s);
  adamw_kernel<<<(s->total + 255) / 256, 256>>>(s->p, s->g, s->m1, s->m2, s->pb, s->total, segs, lr, 0.9f, 0.999f,
                                                1e-8f, weight_decay, s->adam_t_d);
  SUR_CUDA(cudaGetLastError());
  SUR_CUDA(cudaDeviceSynchronize());
  s->adam_step += 1;
  s->tc_pack_valid = false;
  return CEM_OK;
}

int cem_surrogate_status(cem_surrogate_handle s, int* status_h) {
  if (!s || !status_h) return fail(CEM_ERR_INVALID_ARG, "null argument");
  SUR_CUDA(cudaDeviceSynchronize());
  SUR_CUDA(cudaMemcpy(status_h, s->tc_status, sizeof(int), cudaMemcpyDeviceToHost));
  SUR_CUDA(cudaMemset(s->tc_status, 0, sizeof(int)));
  return CEM_OK;
}

int cem_surrogate_gradient(cem_surrogate_handle s, const float* x_d, const float* t_d, int M, float* grad_h,
                           float* loss_h) {
  if (!s || !grad_h) return fail(CEM_ERR_INVALID_ARG, "null argument");
  if (M < 1 || M > (1 << 22)) return fail(CEM_ERR_UNSUPPORTED, "M must be in 1..2^22");
  if (!is_dev(x_d) || !is_dev(t_d)) return fail(CEM_ERR_INVALID_ARG, "x and t must be device pointers");
  if (s->gemm_path == 3) {
    int rc = gradient_f32(s, x_d, t_d, M);
    if (rc != CEM_OK) return rc;
  } else {
    int rc = load_features(s, x_d, M, 0);
    if (rc != CEM_OK) return rc;
    SUR_CUDA(cudaMemcpy(s->tb, t_d, sizeof(float) * M, cudaMemcpyDeviceToDevice));
    SUR_CUDA(forward_rows(s, M, nullptr, use_tc_gemm(s), 0));
    SUR_CUDA(backward_rows(s, M, 0));
  }
  SUR_CUDA(cudaDeviceSynchronize());
  SUR_CUDA(cudaMemcpy(grad_h, s->g, sizeof(float) * s->total, cudaMemcpyDeviceToHost));
  if (loss_h) {
    float l = 0.0f;
    SUR_CUDA(cudaMemcpy(&l, s->loss_d, sizeof(float), cudaMemcpyDeviceToHost));
    *loss_h = l / M;
  }
  return CEM_OK;
}

int cem_surrogate_train(cem_surrogate_handle s, const float* x_d, const float* t_d, int M, int batch, int steps,
                        float lr, float weight_decay, uint64_t seed, int normalize, float* loss_hist_h) {
  if (!s) return fail(CEM_ERR_INVALID_ARG, "null handle");
  if (M < 1 || batch < 1 || batch > (1 << 20) || steps < 0 || steps > 10000000)
    return fail(CEM_ERR_UNSUPPORTED, "M >= 1, batch in 1..2^20, steps in 0..1e7");
  if (!is_dev(x_d) || !is_dev(t_d)) return fail(CEM_ERR_INVALID_ARG, "x and t must be device pointers");
  // whole data set in BF16 once
  bf16* Xall = nullptr;
  float* hist_d = nullptr;  // per-step losses stay on the device until the end (no per-step sync)
  cudaStream_t st = nullptr;
  if (dev_malloc(&Xall, sizeof(bf16) * (size_t)M * s->in_dim) != cudaSuccess ||
      (loss_hist_h && steps > 0 && dev_malloc(&hist_d, sizeof(float) * (size_t)steps) != cudaSuccess)) {
    cudaGetLastError();
    cudaFree(Xall);
    return fail(CEM_ERR_NO_MEMORY, "training set does not fit");
  }
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(Xall);
    cudaFree(hist_d);
    return fail(CEM_ERR_CUDA, "cem_surrogate_train: stream creation failed");
  }
  cudaDeviceSynchronize();  // earlier work on other streams (parameters, data) is complete
  const size_t n = (size_t)M * s->in_dim;
  to_bf16_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x_d, n, Xall);
  if (normalize) target_stats_kernel<<<1, 256, 0, st>>>(t_d, M, s->norm);
  int rc = ensure_rows(s, batch);
  if (rc != CEM_OK) {
    cudaStreamDestroy(st);
    cudaFree(Xall);
    cudaFree(hist_d);
    return rc;
  }
  const Segs segs = param_segments(s);
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  s->tc_pack_valid = false;  // the BF16 weights change below
  cudaError_t e = cudaMemsetAsync(s->step_d, 0, sizeof(int), st);
  const long long t0 = s->adam_step;
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->adam_t_d, &t0, sizeof(t0), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // t0 is read before this function returns
  // one step: batch -> forward -> backward -> AdamW -> counters; everything
  // that varies between steps is read from the device
  auto enqueue_step = [&]() -> cudaError_t {
    gather_batch_kernel<<<(batch + 255) / 256, 256, 0, st>>>(Xall, t_d, M, s->in_dim, batch, seed, s->step_d,
                                                              s->xin, s->tb);
    cudaError_t r = forward_rows(s, batch, nullptr, use_tc_gemm(s), st);
    if (r == cudaSuccess) r = backward_rows(s, batch, st);
    if (r != cudaSuccess) return r;
    adamw_kernel<<<(s->total + 255) / 256, 256, 0, st>>>(s->p, s->g, s->m1, s->m2, s->pb, s->total, segs, lr, b1, b2,
                                                         eps, weight_decay, s->adam_t_d);
    step_end_kernel<<<1, 1, 0, st>>>(s->step_d, s->adam_t_d, s->loss_d, hist_d);
    return cudaGetLastError();
  };
  // the first step runs directly (it also sets up the kernels), the others
  // replay that step captured as one CUDA graph; direct launches if capture fails
  int done = 0;
  if (e == cudaSuccess && steps > 0) {
    e = enqueue_step();
    done = 1;
  }
  if (e == cudaSuccess && steps > 1) {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const cudaError_t ce = enqueue_step();
      const cudaError_t ee = cudaStreamEndCapture(st, &graph);
      if (ce != cudaSuccess || ee != cudaSuccess || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) exec = nullptr;
    }
    cudaGetLastError();
    if (graph) cudaGraphDestroy(graph);
    for (; done < steps && e == cudaSuccess; ++done) e = exec ? cudaGraphLaunch(exec, st) : enqueue_step();
    if (exec) cudaGraphExecDestroy(exec);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) s->adam_step += steps;
  if (hist_d && e == cudaSuccess) {
    e = cudaMemcpy(loss_hist_h, hist_d, sizeof(float) * (size_t)steps, cudaMemcpyDeviceToHost);
    for (int it = 0; it < steps; ++it) loss_hist_h[it] /= (float)batch;
  }
  cudaStreamDestroy(st);
  cudaFree(Xall);
  cudaFree(hist_d);
  if (e != cudaSuccess) return fail(CEM_ERR_CUDA, std::string("cem_surrogate_train: ") + cudaGetErrorString(e));
  return CEM_OK;
}

int cem_surrogate_features(cem_surrogate_handle s, const float* theta_d, int N, int D, const float* lo_h,
                           const float* hi_h, const float* scene16_h, float* x_d, void* stream) {
  if (!s || D < 1 || D > CEM_MAX_D || N < 0 || !lo_h || !hi_h || !scene16_h)
    return fail(CEM_ERR_INVALID_ARG, "bad feature arguments");
  if (N == 0) return CEM_OK;
  if (!is_dev(theta_d) || !is_dev(x_d)) return fail(CEM_ERR_INVALID_ARG, "theta and x must be device pointers");
  cudaStream_t st = (cudaStream_t)stream;
  float tab[2 * CEM_MAX_D];
  for (int d = 0; d < CEM_MAX_D; ++d) {
    tab[d] = d < D ? lo_h[d] : 0.0f;
    tab[CEM_MAX_D + d] = d < D ? hi_h[d] : 0.0f;
  }
  SUR_CUDA(cudaMemcpyAsync(s->lohi, tab, sizeof(tab), cudaMemcpyHostToDevice, st));
  SUR_CUDA(cudaMemcpyAsync(s->scene16, scene16_h, sizeof(float) * 16, cudaMemcpyHostToDevice, st));
  features_kernel<float><<<(N + 127) / 128, 128, 0, st>>>(theta_d, N, D, s->lohi, s->scene16, x_d);
  SUR_CUDA(cudaGetLastError());
  SUR_CUDA(cudaStreamSynchronize(st));  // the host tables are consumed
  return CEM_OK;
}

}  // extern "C"

namespace {

// screening workspace of a pool of P candidates keeping N
int ensure_pool(cem_surrogate_ctx* s, int P, int N, int D) {
  int rc = ensure_rows(s, P);
  if (rc != CEM_OK) return rc;
  if (P <= s->cap_pool && s->pool_theta) return CEM_OK;
  cudaFree(s->pool_theta);
  cudaFree(s->pool_score);
  cudaFree(s->keep_idx);
  s->pool_theta = nullptr;
  s->pool_score = nullptr;
  s->keep_idx = nullptr;
  cudaError_t e = dev_malloc(&s->pool_theta, sizeof(float) * (size_t)P * CEM_MAX_D);
  if (e == cudaSuccess) e = dev_malloc(&s->pool_score, sizeof(float) * P);
  if (e == cudaSuccess) e = dev_malloc(&s->keep_idx, sizeof(int32_t) * P);
  if (e != cudaSuccess) {
    cudaGetLastError();
    s->cap_pool = 0;
    return fail(CEM_ERR_NO_MEMORY, "screening workspace allocation failed");
  }
  s->cap_pool = P;
  (void)N;
  (void)D;
  return CEM_OK;
}

// pool theta (already sampled, P x D) -> scores -> indices of the N best ->
// theta_keep (N x D), all on `st`; features from the bounds lohi[2 x 18]
// and the scene values scene16[16] (device)
cudaError_t screen_pool_tab(cem_surrogate_ctx* s, int P, int N, int n_explore, int D, const float* lohi,
                            const float* scene16, float* theta_keep, cudaStream_t st) {
  features_kernel<bf16><<<(P + 127) / 128, 128, 0, st>>>(s->pool_theta, P, D, lohi, scene16, s->xin);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = infer_rows(s, P, s->pool_score, st);
  if (e != cudaSuccess) return e;
  if (n_explore > 0) {
    force_keep_kernel<<<(n_explore + 255) / 256, 256, 0, st>>>(s->pool_score, n_explore);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  topk_kernel<<<1, 1024, 0, st>>>(s->pool_score, P, N, s->keep_idx);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  gather_rows_kernel<<<(N * D + 255) / 256, 256, 0, st>>>(s->pool_theta, P, s->keep_idx, N, D, theta_keep);
  return cudaGetLastError();
}

cudaError_t screen_pool(cem_surrogate_ctx* s, int P, int N, int n_explore, int D, float* theta_keep,
                        cudaStream_t st) {
  return screen_pool_tab(s, P, N, n_explore, D, s->lohi, s->scene16, theta_keep, st);
}

int set_tables(cem_surrogate_ctx* s, const cem_skeleton_desc& k, const float* scene16_h, cudaStream_t st) {
  float tab[2 * CEM_MAX_D];
  for (int d = 0; d < CEM_MAX_D; ++d) {
    tab[d] = d < k.D ? k.lo[d] : 0.0f;
    tab[CEM_MAX_D + d] = d < k.D ? k.hi[d] : 0.0f;
  }
  SUR_CUDA(cudaMemcpyAsync(s->lohi, tab, sizeof(tab), cudaMemcpyHostToDevice, st));
  SUR_CUDA(cudaMemcpyAsync(s->scene16, scene16_h, sizeof(float) * 16, cudaMemcpyHostToDevice, st));
  SUR_CUDA(cudaStreamSynchronize(st));
  return CEM_OK;
}

}  // namespace

namespace cem {

#ifdef CEM_DEBUG
CEM_DEBUG_STATUS_ACCESSOR(debug_status_surrogate)
#endif

int surrogate_reserve_pool(cem_surrogate_handle s, int n_pool, int n_keep, int D) {
  if (!s) return fail(CEM_ERR_INVALID_ARG, "null surrogate");
  if (s->in_dim != 48) return fail(CEM_ERR_UNSUPPORTED, "screening needs the 48-feature surrogate input");
  return ensure_pool(s, n_pool, n_keep, D);
}

cudaError_t surrogate_screen_into(cem_surrogate_handle s, const float* mean, const float* chol, uint64_t seed,
                                  const uint32_t* iter_ptr, uint32_t problem, int n_pool, int n_keep, int n_explore,
                                  int D, const float* lohi, const float* scene16, float* theta_keep,
                                  cudaStream_t st) {
  cudaError_t e = launch_sample(mean, chol, seed, iter_ptr, 0, problem, n_pool, D, s->pool_theta, st);
  if (e != cudaSuccess) return e;
  return screen_pool_tab(s, n_pool, n_keep, n_explore, D, lohi, scene16, theta_keep, st);
}

int surrogate_status_word(cem_surrogate_handle s) {
  int v = 0;
  if (!s || cudaMemcpy(&v, s->tc_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
  if (v) cudaMemset(s->tc_status, 0, sizeof(int));
  return v;
}

}  // namespace cem

extern "C" {

int cem_surrogate_screen(cem_handle h, cem_surrogate_handle s, const float* mean_d, const float* chol_d, uint64_t seed,
                         uint32_t iter, uint32_t problem, int n_pool, int n_keep, const float* scene16_h,
                         float* theta_keep_d, int32_t* keep_idx_d, void* stream) {
  set_last_error(CEM_OK, "");
  if (!h || !s || !scene16_h) return fail(CEM_ERR_INVALID_ARG, "null argument");
  if (n_pool < 1 || n_pool > CEM_MAX_N || n_keep < 1 || n_keep > n_pool)
    return fail(CEM_ERR_UNSUPPORTED, "1 <= n_keep <= n_pool <= 2^20");
  if (!is_dev(mean_d) || !is_dev(chol_d) || !is_dev(theta_keep_d) || (keep_idx_d && !is_dev(keep_idx_d)))
    return fail(CEM_ERR_INVALID_ARG, "mean, chol, theta_keep (and keep_idx) must be device pointers");
  const cem_skeleton_desc& k = handle_skeleton(h);
  cudaStream_t st = (cudaStream_t)stream;
  int rc = ensure_pool(s, n_pool, n_keep, k.D);
  if (rc != CEM_OK) return rc;
  rc = set_tables(s, k, scene16_h, st);
  if (rc != CEM_OK) return rc;
  SUR_CUDA(launch_sample(mean_d, chol_d, seed, nullptr, iter, problem, n_pool, k.D, s->pool_theta, st));
  SUR_CUDA(screen_pool(s, n_pool, n_keep, 0, k.D, theta_keep_d, st));
  if (keep_idx_d)
    SUR_CUDA(cudaMemcpyAsync(keep_idx_d, s->keep_idx, sizeof(int32_t) * n_keep, cudaMemcpyDeviceToDevice, st));
  return CEM_OK;
}

}  // extern "C"

namespace {

// the replay ring of cem_solve_screened_ft (features and targets of every
// simulated sample of the run), freed on every way out
struct Replay {
  float* x = nullptr;
  float* t = nullptr;
  ~Replay() {
    cudaFree(x);
    cudaFree(t);
  }
};

// the screened CE loop; ft (may be null): fine-tune the surrogate on the
// run's own simulated samples every ft->every iterations
int solve_screened(cem_handle h, cem_surrogate_handle s, const float* scene16_h, const cem_solve_params* p,
                   int n_pool, int n_explore, const cem_finetune_params* ft, cem_result* out) {
  set_last_error(CEM_OK, "");
  if (!h || !s || !scene16_h || !p || !out) return fail(CEM_ERR_INVALID_ARG, "null argument");
  if (p->N < 1 || n_pool < p->N || n_pool > CEM_MAX_N) return fail(CEM_ERR_UNSUPPORTED, "1 <= N <= n_pool <= 2^20");
  if (n_explore < 0 || n_explore > p->N) return fail(CEM_ERR_INVALID_ARG, "0 <= n_explore <= N");
  if (p->K < 1 || p->K > CEM_MAX_K || p->iters < 1 || p->iters > 100000)
    return fail(CEM_ERR_UNSUPPORTED, "K in 1..4096, iters in 1..1e5");
  const cem_skeleton_desc& k = handle_skeleton(h);
  const int D = k.D, N = p->N;
  Replay rb;
  if (ft) {
    if (ft->every < 0 || ft->steps < 0 || ft->batch < 1 || ft->batch > (1 << 20))
      return fail(CEM_ERR_INVALID_ARG, "fine-tune: every >= 0, steps >= 0, batch in 1..2^20");
    if (ft->capacity < N || ft->capacity % N != 0 || ft->capacity > (1 << 22))
      return fail(CEM_ERR_INVALID_ARG, "fine-tune: capacity a multiple of N, at most 2^22");
    if (s->in_dim != 48) return fail(CEM_ERR_UNSUPPORTED, "fine-tune needs the 48-feature surrogate input");
    if (dev_malloc(&rb.x, sizeof(float) * (size_t)ft->capacity * 48) != cudaSuccess ||
        dev_malloc(&rb.t, sizeof(float) * (size_t)ft->capacity) != cudaSuccess) {
      cudaGetLastError();
      return fail(CEM_ERR_NO_MEMORY, "fine-tune replay buffer does not fit");
    }
  }
  int rc = ensure_pool(s, n_pool, N, D);
  if (rc != CEM_OK) return rc;
  SolveBuffers b;
  rc = handle_solve_buffers(h, N, p->iters, &b);
  if (rc != CEM_OK) return rc;
  cudaStream_t st = b.stream;
  rc = set_tables(s, k, scene16_h, st);
  if (rc != CEM_OK) return rc;
  rc = handle_init_distribution(h, p, &b);
  if (rc != CEM_OK) return rc;
  RefitArgs a;
  std::memset(&a, 0, sizeof(a));
  a.theta = b.theta;
  a.J = b.J;
  a.cls = b.cls;
  a.N = N;
  a.D = D;
  a.K = p->K;
  a.cov_mode = p->cov_mode;
  for (int d = 0; d < D; ++d) {
    a.lo[d] = k.lo[d];
    a.hi[d] = k.hi[d];
  }
  a.mean = b.mean;
  a.cov = b.cov;
  a.chol = b.chol;
  a.k_eff = b.keff;
  a.track = b.track;
  a.hist_J = b.hist_J;
  a.hist_keff = b.hist_keff;
  a.hist_cnt = b.hist_cnt;
  a.status = b.status;
  SUR_CUDA(cudaEventRecord(b.ev0, st));
  for (int j = 0; j < p->iters; ++j) {
    SUR_CUDA(launch_sample(b.mean, b.chol, p->seed, &b.track->iter, 0, p->problem, n_pool, D, s->pool_theta, st));
    SUR_CUDA(screen_pool(s, n_pool, N, n_explore, D, b.theta, st));
    DrArgs dr;
    if (b.dr) {
      dr = *b.dr;
      dr.problem = p->problem;
      dr.iter_ptr = &b.track->iter;
    }
    SUR_CUDA(launch_rollout(b.scene, b.kind, b.theta, N, b.J, b.cls, b.block, b.tpr, b.dr ? &dr : nullptr, st, b.astar));
    if (ft) {  // this iteration's simulated samples (features, score targets) into the ring
      const int pos = (int)(((long long)j * N) % ft->capacity);
      features_kernel<float><<<(N + 127) / 128, 128, 0, st>>>(b.theta, N, D, s->lohi, s->scene16, rb.x + (size_t)pos * 48);
      score_target_kernel<<<(N + 255) / 256, 256, 0, st>>>(b.J, b.cls, N, rb.t + pos);
      SUR_CUDA(cudaGetLastError());
    }
    SUR_CUDA(launch_refit(a, st));
    if (ft && ft->every > 0 && ft->steps > 0 && (j + 1) % ft->every == 0 && j + 1 < p->iters) {
      // fine-tune on every sample simulated so far (the ring's filled part),
      // keeping the target normalisation of the surrogate's training
      const long long seen = (long long)(j + 1) * N;
      const int filled = (int)(seen < ft->capacity ? seen : ft->capacity);
      SUR_CUDA(cudaStreamSynchronize(st));
      rc = cem_surrogate_train(s, rb.x, rb.t, filled, ft->batch < filled ? ft->batch : filled, ft->steps, ft->lr,
                               ft->weight_decay, ft->seed + (uint64_t)j, 0, nullptr);
      if (rc != CEM_OK) return rc;
    }
  }
  SUR_CUDA(cudaEventRecord(b.ev1, st));
  rc = handle_read_result(h, p, &b, out);
  if (rc != CEM_OK) return rc;
  int tc_fail = 0;
  SUR_CUDA(cudaMemcpy(&tc_fail, s->tc_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (tc_fail) {
    cudaMemset(s->tc_status, 0, sizeof(int));
    return fail(CEM_ERR_TIMEOUT, "surrogate forward: a bounded wait on the tensor-core pipeline expired");
  }
  return CEM_OK;
}

}  // namespace

extern "C" {

int cem_solve_screened(cem_handle h, cem_surrogate_handle s, const float* scene16_h, const cem_solve_params* p,
                       int n_pool, int n_explore, cem_result* out) {
  return solve_screened(h, s, scene16_h, p, n_pool, n_explore, nullptr, out);
}

int cem_solve_screened_ft(cem_handle h, cem_surrogate_handle s, const float* scene16_h, const cem_solve_params* p,
                          int n_pool, int n_explore, const cem_finetune_params* ft, cem_result* out) {
  if (!ft) return fail(CEM_ERR_INVALID_ARG, "null fine-tune parameters");
  return solve_screened(h, s, scene16_h, p, n_pool, n_explore, ft, out);
}

}  // extern "C"

extern "C" int cem_surrogate_targets(const float* J_d, const uint8_t* cls_d, int N, float* t_d, void* stream) {
  if (N < 0) return fail(CEM_ERR_INVALID_ARG, "N must be >= 0");
  if (N == 0) return CEM_OK;
  if (!is_dev(J_d) || !is_dev(cls_d) || !is_dev(t_d)) return fail(CEM_ERR_INVALID_ARG, "J, cls and t must be device pointers");
  score_target_kernel<<<(N + 255) / 256, 256, 0, (cudaStream_t)stream>>>(J_d, cls_d, N, t_d);
  SUR_CUDA(cudaGetLastError());
  return CEM_OK;
}
