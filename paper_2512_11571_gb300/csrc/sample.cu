// Sample step of Algorithm 1 (Sec. III-B): draw n_env parameter vectors
// theta ~ N(mean, chol chol^T).
//
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64-bit
// multiplies, a word swap and xors with the round key, the key bumped by the
// Weyl constants between rounds.  Counter (n, c, iter, problem), key = seed;
// call c yields normals 4c..4c+3 of sample n by Box-Muller on word pairs
// with u = (r + 1) 2^-32 in (0, 1].
//
// One thread per sample: the ceil(D/4) Philox calls and the D x D
// triangular product stay in registers; mean and chol are staged in shared
// memory once per block.  The kernel writes N*D*4 bytes and is far from
// any roofline at the CE sizes (N <= 65536); it exists to keep the loop on
// the device.
#include "internal.h"
#include "philox.cuh"

namespace cem {
namespace {

__global__ void __launch_bounds__(256) sample_kernel(const float* __restrict__ mean, const float* __restrict__ chol,
                                                     uint64_t seed, const uint32_t* __restrict__ iter_ptr,
                                                     uint32_t iter, uint32_t problem, int N, int D,
                                                     float* __restrict__ theta) {
  __shared__ float sL[CEM_MAX_D * CEM_MAX_D];
  __shared__ float sm[CEM_MAX_D];
  for (int i = threadIdx.x; i < D * D; i += blockDim.x) sL[i] = chol[i];
  for (int i = threadIdx.x; i < D; i += blockDim.x) sm[i] = mean[i];
  __syncthreads();
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const uint32_t it = iter_ptr ? *iter_ptr : iter;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  float z[20];
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    if (4 * c < D) {
      uint32_t r[4];
      philox4x32_10((uint32_t)n, (uint32_t)c, it, problem, k0, k1, r);
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const float rad = sqrtf(-2.0f * logf(u01(r[2 * p])));
        float sn, cs;
        sincospif(2.0f * u01(r[2 * p + 1]), &sn, &cs);
        z[4 * c + 2 * p] = rad * cs;
        z[4 * c + 2 * p + 1] = rad * sn;
      }
    } else {
#pragma unroll
      for (int p = 0; p < 4; ++p) z[4 * c + p] = 0.0f;
    }
  }
  float* out = theta + (size_t)n * D;
#pragma unroll
  for (int i = 0; i < CEM_MAX_D; ++i) {
    if (i < D) {
      float acc = sm[i];
#pragma unroll
      for (int j = 0; j <= i; ++j) acc = fmaf(sL[i * D + j], z[j], acc);
      out[i] = acc;
    }
  }
}

__global__ void philox_words_kernel(uint64_t seed, uint32_t iter, uint32_t problem, int N, int nc,
                                    uint32_t* __restrict__ words) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * nc) return;
  const int n = t / nc, c = t % nc;
  uint32_t r[4];
  philox4x32_10((uint32_t)n, (uint32_t)c, iter, problem, (uint32_t)seed, (uint32_t)(seed >> 32), r);
  uint32_t* o = words + (size_t)t * 4;
  o[0] = r[0];
  o[1] = r[1];
  o[2] = r[2];
  o[3] = r[3];
}

// Initial distribution of Sec. III-B: uniform inside each parameter's
// region.  Parameter d takes word d of the Philox block (n, d / 4,
// 0xFFFFFFFF, problem); a box parameter is lo + u (hi - lo), an annulus goal
// (dx, dy) of a moveTo is the area-uniform point c + rho (cos, sin)(2 pi u')
// with rho = sqrt(r^2 + u (R^2 - r^2)), less the action's nominal target.
__global__ void __launch_bounds__(128) sample_uniform_kernel(const DevScene* __restrict__ s, uint64_t seed,
                                                             uint32_t problem, int N, int D,
                                                             float* __restrict__ theta) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  float u[20];
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    if (4 * c < D) {
      uint32_t r[4];
      philox4x32_10((uint32_t)n, (uint32_t)c, 0xFFFFFFFFu, problem, k0, k1, r);
#pragma unroll
      for (int p = 0; p < 4; ++p) u[4 * c + p] = u01(r[p]);
    } else {
#pragma unroll
      for (int p = 0; p < 4; ++p) u[4 * c + p] = 0.0f;
    }
  }
  float th[CEM_MAX_D];
#pragma unroll
  for (int d = 0; d < CEM_MAX_D; ++d) th[d] = d < D ? fmaf(u[d], s->hi[d] - s->lo[d], s->lo[d]) : 0.0f;
  for (int a = 0; a < s->n_act; ++a) {
    if (s->act_region[a] != 1) continue;
    const int o = s->act_off[a];
    const float ri = s->act_ring[a][2], ro = s->act_ring[a][3];
    float uo = 0.0f, uo1 = 0.0f;
#pragma unroll
    for (int d = 0; d < CEM_MAX_D - 1; ++d)
      if (d == o) {
        uo = u[d];
        uo1 = u[d + 1];
      }
    const float rho = sqrtf(fmaf(uo, ro * ro - ri * ri, ri * ri));
    float sn, cs;
    sincospif(2.0f * uo1, &sn, &cs);
    const float px = fmaf(rho, cs, s->act_ring[a][0]) - s->act_nom[a][0];
    const float py = fmaf(rho, sn, s->act_ring[a][1]) - s->act_nom[a][1];
#pragma unroll
    for (int d = 0; d < CEM_MAX_D - 1; ++d)
      if (d == o) {
        th[d] = px;
        th[d + 1] = py;
      }
  }
  float* out = theta + (size_t)n * D;
#pragma unroll
  for (int d = 0; d < CEM_MAX_D; ++d)
    if (d < D) out[d] = th[d];
}

// batched sampling: blockIdx.y = problem, samples in x; the same per-sample
// arithmetic as sample_kernel
__global__ void __launch_bounds__(128) sample_batch_kernel(const BatchProblem* __restrict__ probs,
                                                           const float* __restrict__ means,
                                                           const float* __restrict__ chols,
                                                           const Track* __restrict__ tracks,
                                                           float* __restrict__ theta) {
  __shared__ float sL[CEM_MAX_D * CEM_MAX_D];
  __shared__ float sm[CEM_MAX_D];
  const int p = blockIdx.y;
  const BatchProblem pb = probs[p];
  if (!pb.active || (int)(blockIdx.x * blockDim.x) >= pb.N) return;  // inactive, or past this problem
  const int D = pb.D;
  for (int i = threadIdx.x; i < D * D; i += blockDim.x) sL[i] = chols[(size_t)p * CEM_MAX_D * CEM_MAX_D + i];
  for (int i = threadIdx.x; i < D; i += blockDim.x) sm[i] = means[(size_t)p * CEM_MAX_D + i];
  __syncthreads();
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= pb.N) return;
  const uint32_t it = tracks[p].iter;
  const uint32_t k0 = (uint32_t)pb.seed, k1 = (uint32_t)(pb.seed >> 32);
  float z[20];
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    if (4 * c < D) {
      uint32_t r[4];
      philox4x32_10((uint32_t)n, (uint32_t)c, it, pb.problem, k0, k1, r);
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const float rad = sqrtf(-2.0f * logf(u01(r[2 * q])));
        float sn, cs;
        sincospif(2.0f * u01(r[2 * q + 1]), &sn, &cs);
        z[4 * c + 2 * q] = rad * cs;
        z[4 * c + 2 * q + 1] = rad * sn;
      }
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) z[4 * c + q] = 0.0f;
    }
  }
  float* out = theta + pb.theta_off + (size_t)n * D;
#pragma unroll
  for (int i = 0; i < CEM_MAX_D; ++i) {
    if (i < D) {
      float acc = sm[i];
#pragma unroll
      for (int j = 0; j <= i; ++j) acc = fmaf(sL[i * D + j], z[j], acc);
      out[i] = acc;
    }
  }
}

}  // namespace

cudaError_t launch_sample_batch(const BatchProblem* probs_d, int n_problems, int maxN, const float* means,
                                const float* chols, const Track* tracks, float* theta, cudaStream_t st) {
  if (n_problems <= 0 || maxN <= 0) return cudaSuccess;
  const int bs = 128;
  dim3 grid((maxN + bs - 1) / bs, n_problems);
  sample_batch_kernel<<<grid, bs, 0, st>>>(probs_d, means, chols, tracks, theta);
  return cudaGetLastError();
}

cudaError_t launch_sample(const float* mean, const float* chol, uint64_t seed, const uint32_t* iter_ptr,
                          uint32_t iter, uint32_t problem, int N, int D, float* theta, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  const int bs = 128;
  sample_kernel<<<(N + bs - 1) / bs, bs, 0, st>>>(mean, chol, seed, iter_ptr, iter, problem, N, D, theta);
  return cudaGetLastError();
}

cudaError_t launch_sample_uniform(const DevScene* s_d, uint64_t seed, uint32_t problem, int N, int D, float* theta,
                                  cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  const int bs = 128;
  sample_uniform_kernel<<<(N + bs - 1) / bs, bs, 0, st>>>(s_d, seed, problem, N, D, theta);
  return cudaGetLastError();
}

cudaError_t launch_philox_words(uint64_t seed, uint32_t iter, uint32_t problem, int N, int D, uint32_t* words,
                                cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  const int nc = (D + 3) / 4;
  const int total = N * nc, bs = 256;
  philox_words_kernel<<<(total + bs - 1) / bs, bs, 0, st>>>(seed, iter, problem, N, nc, words);
  return cudaGetLastError();
}

}  // namespace cem
