// Update step of Algorithm 1 (Sec. III-B): pick the top-N_e elites and refit
// the sampling distribution to them.
//
// Elite rules of Sec. III-B: samples are ranked by (class, J, index); the
// elites are the K lowest of the best class present among {0: goal reached,
// 1: every action succeeded} -- fewer if fewer exist ("only the n_feasible
// samples are used") -- or, if neither class occurs, of class 2.  The new
// distribution is the maximum-likelihood Gaussian of the elites (the
// KL-minimising CE update of Botev et al.): mean, covariance with 1/K_eff,
// a ridge (1e-4 range)^2; a single elite gets diag((0.05 range)^2)
// ("artificial noise"); the diagonal mode is the independent-normal model of
// Sec. IV-A.
//
// One CTA of 1024 threads per problem.  Selection is an exact MSB-first
// radix select over 52-bit keys (32-bit order-preserving cost bits, 20-bit
// index) with shared-memory histograms, then a bitonic sort of the K_eff
// elites (<= 4096 keys in shared memory; elite rows are read through L2);
// ties are impossible because the index is part of the key.  The keys of
// the first KR * 1024 samples stay in registers across the passes; lanes of
// a warp that fall into the same histogram bin add once (costs are close
// together, so the high bits put most keys in one bin); one warp finds the
// bin that holds the wanted rank (prefix sums over the lanes).  The
// statistics are accumulated in FP64 by groups of four threads per output
// with a fixed reduction order (run-to-run deterministic), and one warp
// factorises the covariance.
#include "internal.h"

namespace cem {
namespace {

constexpr int RT = 1024;
constexpr int KEY_BITS = 52;
constexpr int KR = 4;  // samples per thread whose keys stay in registers (N <= 4096 entirely)
// up to this many elites are staged in shared memory as FP64 rows for the
// statistics (18 parameters: 72 KB); more are read through L2
constexpr int KSTAGE = 512;

__device__ __forceinline__ uint32_t order_bits(float x) {
  const uint32_t u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// class (0..3) and 52-bit key of sample i
__device__ __forceinline__ int classify(const float* __restrict__ J, const uint8_t* __restrict__ cls, int i,
                                        uint64_t& key) {
  float j = J[i];
  int c = cls[i];
  if (c > 3) c = 3;
  if (!isfinite(j)) {
    c = 3;
    j = __int_as_float(0x7f800000);
  }
  j = j + 0.0f;  // -0 -> +0
  key = ((uint64_t)order_bits(j) << 20) | (uint64_t)i;
  return c;
}

__device__ bool cholesky_warp(double* A, int D, int lane) {
  // right-looking, in place, lower triangle; lane i owns row i
  for (int j = 0; j < D; ++j) {
    double d = A[j * D + j];
    const bool ok = d > 0.0;
    if (!__all_sync(0xffffffffu, ok)) return false;
    // one reciprocal square root instead of a square root and a division
    // per row (FP64 is slow on this part; the result is cast to FP32)
    const double r = rsqrt(d);
    const double ljj = d * r;
    __syncwarp();
    if (lane == j) A[j * D + j] = ljj;
    if (lane > j && lane < D) A[lane * D + j] *= r;
    __syncwarp();
    if (lane > j && lane < D)
      for (int k = j + 1; k <= lane; ++k) A[lane * D + k] -= A[lane * D + j] * A[k * D + j];
    __syncwarp();
  }
  return true;
}

__device__ __forceinline__ void refit_body(const RefitArgs& a) {
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ int cnt[4];
  __shared__ uint32_t hist[256];
  __shared__ int s_cstar, s_keff, s_rank, s_n, s_fail;
  __shared__ double s_invk;
  __shared__ uint64_t s_prefix, s_mask;
  __shared__ double s_mean[CEM_MAX_D];
  __shared__ double s_cov[CEM_MAX_D * CEM_MAX_D];
  __shared__ double s_L[CEM_MAX_D * CEM_MAX_D];
  const int tid = threadIdx.x, N = a.N, D = a.D;
  if (tid < 4) cnt[tid] = 0;
  if (tid == 0) s_n = 0;
  __syncthreads();
  // keys and classes of samples tid + r * RT, r < KR (class 4: no sample)
  uint64_t rkey[KR];
  int rcls[KR];
#pragma unroll
  for (int r = 0; r < KR; ++r) {
    const int i = r * RT + tid;
    rcls[r] = 4;
    rkey[r] = 0;
    if (i < N) {
      rcls[r] = classify(a.J, a.cls, i, rkey[r]);
      atomicAdd(&cnt[rcls[r]], 1);
    }
  }
  for (int i = KR * RT + tid; i < N; i += RT) {
    uint64_t key;
    atomicAdd(&cnt[classify(a.J, a.cls, i, key)], 1);
  }
  __syncthreads();
  if (tid == 0) {
    const int cs = cnt[0] > 0 ? 0 : cnt[1] > 0 ? 1 : cnt[2] > 0 ? 2 : -1;
    s_cstar = cs;
    s_keff = cs < 0 ? 0 : min(a.K, cnt[cs]);
    s_invk = s_keff > 0 ? 1.0 / (double)s_keff : 0.0;
    s_rank = s_keff;
    s_prefix = 0;
    s_mask = 0;
  }
  __syncthreads();
  const int cstar = s_cstar, keff = s_keff;
  if (keff > 0) {
    uint64_t kth = ~0ull;
    if (keff < cnt[cstar]) {  // exact radix select of the keff-th smallest key
      int shift = KEY_BITS;
      while (shift > 0) {
        const int width = shift >= 8 ? 8 : shift;
        shift -= width;
        for (int d = tid; d < 256; d += RT) hist[d] = 0;
        __syncthreads();
        const uint64_t prefix = s_prefix, mask = s_mask;
        const uint32_t bmask = (1u << width) - 1;
        // the lanes of a warp with the same bin add once (every lane takes
        // part: the loop bounds are the same for the whole CTA)
        auto count = [&](int c, uint64_t key) {
          const int bin = (c == cstar && (key & mask) == prefix) ? (int)((key >> shift) & bmask) : -1;
          const unsigned same = __match_any_sync(0xffffffffu, bin);
          if (bin >= 0 && (tid & 31) == __ffs(same) - 1) atomicAdd(&hist[bin], (uint32_t)__popc(same));
        };
#pragma unroll
        for (int r = 0; r < KR; ++r)
          if (r * RT < N) count(rcls[r], rkey[r]);
        for (int base = KR * RT; base < N; base += RT) {
          uint64_t key = 0;
          const int c = base + tid < N ? classify(a.J, a.cls, base + tid, key) : 4;
          count(c, key);
        }
        __syncthreads();
        if (tid < 32) {
          // lane l sums bins [l * per, (l + 1) * per); the lane whose range
          // holds the rank-th key walks its bins to the one that holds it
          const int nb = 1 << width, per = (nb + 31) / 32;
          uint32_t loc[8], sum = 0;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int d = tid * per + q;
            loc[q] = (q < per && d < nb) ? hist[d] : 0u;
            sum += loc[q];
          }
          uint32_t incl = sum;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (tid >= o) incl += t;
          }
          const uint32_t rank = (uint32_t)s_rank, excl = incl - sum;
          if (excl < rank && rank <= incl) {
            uint32_t cum = excl;
            int d = tid * per;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              if (q >= per || cum + loc[q] >= rank) break;
              cum += loc[q];
              ++d;
            }
            s_rank = (int)(rank - cum);
            s_prefix |= (uint64_t)d << shift;
            s_mask |= (uint64_t)bmask << shift;
          }
        }
        __syncthreads();
      }
      kth = s_prefix;
    }
    // gather the elites (unordered), then bitonic sort by key
    int P = 1;
    while (P < keff) P <<= 1;
    uint64_t* keys = reinterpret_cast<uint64_t*>(dyn);
    for (int i = tid; i < P; i += RT) keys[i] = ~0ull;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < KR; ++r)
      if (rcls[r] == cstar && rkey[r] <= kth) {
        const int pos = atomicAdd(&s_n, 1);
        if (pos < P) keys[pos] = rkey[r];
      }
    for (int i = KR * RT + tid; i < N; i += RT) {
      uint64_t key;
      if (classify(a.J, a.cls, i, key) == cstar && key <= kth) {
        const int pos = atomicAdd(&s_n, 1);
        if (pos < P) keys[pos] = key;
      }
    }
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = tid; i < P; i += RT) {
          const int ixj = i ^ j;
          if (ixj > i) {
            const uint64_t x = keys[i], y = keys[ixj];
            const bool asc = (i & k) == 0;
            if ((x > y) == asc) {
              keys[i] = y;
              keys[ixj] = x;
            }
          }
        }
        __syncthreads();
      }
    if (a.elite_idx)
      for (int e = tid; e < keff; e += RT) a.elite_idx[e] = (int)(keys[e] & 0xFFFFF);
    // elite e's parameter row (read through L2; the keys stay in shared memory)
    auto eth = [&](int e, int d) -> float { return a.theta[(size_t)CEM_DIDX((int)(keys[e] & 0xFFFFF), a.N, 8) * D + d]; };
    // statistics in FP64: 4 threads per output, fixed reduction order
    const int grp = tid >> 2, part = tid & 3;
    if (keff == 1) {
      if (tid < D) s_mean[tid] = (double)eth(0, tid);
      for (int i = tid; i < D * D; i += RT) {
        const int r = i / D, c = i % D;
        const double w = 0.05 * ((double)a.hi[r] - (double)a.lo[r]);
        s_cov[i] = r == c ? w * w : 0.0;
      }
      __syncthreads();
    } else {
      // keff <= KSTAGE: the elite rows once into shared memory (X[e][d] as
      // FP64), centred after the mean, so each covariance term is one FP64
      // multiply-add on shared operands; the sums run in the same order and
      // give the same values as the L2 path
      const bool staged = keff <= KSTAGE;
      double* X = reinterpret_cast<double*>(dyn + sizeof(uint64_t) * (size_t)P);
      if (staged) {
        for (int q = tid; q < keff * D; q += RT) {
          const int e = q / D;
          X[q] = (double)eth(e, q - e * D);
        }
        __syncthreads();
      }
      double v = 0.0;
      if (grp < D) {
        if (staged)
          for (int e = part; e < keff; e += 4) v += X[e * D + grp];
        else
          for (int e = part; e < keff; e += 4) v += (double)eth(e, grp);
      }
      v += __shfl_down_sync(0xffffffffu, v, 2);
      v += __shfl_down_sync(0xffffffffu, v, 1);
      if (grp < D && part == 0) s_mean[grp] = v * s_invk;
      __syncthreads();
      if (staged) {
        for (int q = tid; q < keff * D; q += RT) X[q] -= s_mean[q % D];
        __syncthreads();
      }
      const int npair = D * (D + 1) / 2;
      int pi = 0, pj = 0;
      if (grp < npair) {  // pair index -> (pi, pj), pi <= pj
        int rem = grp, r = 0;
        while (rem >= D - r) {
          rem -= D - r;
          ++r;
        }
        pi = r;
        pj = r + rem;
      }
      v = 0.0;
      if (grp < npair) {
        if (staged) {
          for (int e = part; e < keff; e += 4) v += X[e * D + pi] * X[e * D + pj];
        } else {
          const double mi = s_mean[pi], mj = s_mean[pj];
          for (int e = part; e < keff; e += 4) v += ((double)eth(e, pi) - mi) * ((double)eth(e, pj) - mj);
        }
      }
      v += __shfl_down_sync(0xffffffffu, v, 2);
      v += __shfl_down_sync(0xffffffffu, v, 1);
      if (grp < npair && part == 0) {
        double c = v * s_invk;
        if (pi == pj) {
          const double w = 1e-4 * ((double)a.hi[pi] - (double)a.lo[pi]);
          c += w * w;
        }
        s_cov[pi * D + pj] = c;
        s_cov[pj * D + pi] = c;
      }
      __syncthreads();
    }
    if (a.cov_mode == CEM_COV_DIAG)
      for (int i = tid; i < D * D; i += RT)
        if (i / D != i % D) s_cov[i] = 0.0;
    __syncthreads();
    if (tid < 32) {
      for (int i = tid; i < D * D; i += 32) s_L[i] = (i % D) <= (i / D) ? s_cov[i] : 0.0;
      __syncwarp();
      bool ok = cholesky_warp(s_L, D, tid);
      if (!ok) {  // fall back to the diagonal
        for (int i = tid; i < D * D; i += 32) {
          const bool dg = i / D == i % D;
          if (!dg) s_cov[i] = 0.0;
          s_L[i] = dg ? s_cov[i] : 0.0;
        }
        __syncwarp();
        ok = cholesky_warp(s_L, D, tid);
      }
      if (tid == 0) s_fail = ok ? 0 : 1;
    }
    __syncthreads();
    if (!s_fail) {
      for (int i = tid; i < D; i += RT) a.mean[i] = (float)s_mean[i];
      for (int i = tid; i < D * D; i += RT) {
        a.cov[i] = (float)s_cov[i];
        a.chol[i] = (i % D) <= (i / D) ? (float)s_L[i] : 0.0f;
      }
    } else if (tid == 0 && a.status) {
      *a.status = CEM_ERR_NOT_PD;
    }
  }
  if (tid == 0) {
    if (a.k_eff) *a.k_eff = keff;
    if (a.track) {
      Track* t = a.track;
      if (keff > 0) {
        const int b = CEM_DIDX((int)(reinterpret_cast<uint64_t*>(dyn)[0] & 0xFFFFF), a.N, 8);
        const float jb = a.J[b];
        if (cstar < t->best_cls || (cstar == t->best_cls && jb < t->best_J)) {
          t->best_cls = cstar;
          t->best_J = jb;
          for (int d = 0; d < D; ++d) t->best_theta[d] = a.theta[(size_t)b * D + d];
        }
      }
      const int h = (int)(t->iter - t->base_iter);
      if (h >= 0 && h < t->hist_len) {
        if (a.hist_J) a.hist_J[h] = t->best_J;
        if (a.hist_keff) a.hist_keff[h] = keff;
        if (a.hist_cnt)
          for (int c = 0; c < 4; ++c) a.hist_cnt[4 * h + c] = cnt[c];
      }
      t->iter += 1;
    }
  }
}

__global__ void __launch_bounds__(RT) refit_kernel(RefitArgs a) { refit_body(a); }

// one CTA per problem of a batch; args[p] describes problem p
__global__ void __launch_bounds__(RT) refit_batch_kernel(const RefitArgs* __restrict__ args) {
  __shared__ RefitArgs a;
  if (threadIdx.x == 0) a = args[blockIdx.x];
  __syncthreads();
  if (a.skip) return;  // an eliminated plan keeps its state
  refit_body(a);
}

}  // namespace

#ifdef CEM_DEBUG
CEM_DEBUG_STATUS_ACCESSOR(debug_status_refit)
#endif

size_t refit_smem_bytes(int K, int D) {
  int P = 1;
  while (P < K) P <<= 1;
  const int ks = K < KSTAGE ? K : KSTAGE;
  return sizeof(uint64_t) * (size_t)P + sizeof(double) * (size_t)(ks > 0 ? ks : 0) * (size_t)(D > 0 ? D : 0);
}

cudaError_t configure_refit() {
  cudaError_t e = cudaFuncSetAttribute(refit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)refit_smem_bytes(CEM_MAX_K, CEM_MAX_D));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(refit_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)refit_smem_bytes(CEM_MAX_K, CEM_MAX_D));
}

cudaError_t launch_refit_batch(const RefitArgs* args_d, int n_problems, int maxK, int maxD, cudaStream_t st) {
  if (n_problems <= 0) return cudaSuccess;
  refit_batch_kernel<<<n_problems, RT, refit_smem_bytes(maxK, maxD), st>>>(args_d);
  return cudaGetLastError();
}

cudaError_t launch_refit(const RefitArgs& a, cudaStream_t st) {
  refit_kernel<<<1, RT, refit_smem_bytes(a.K, a.D), st>>>(a);
  return cudaGetLastError();
}

}  // namespace cem
