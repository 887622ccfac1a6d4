// Dense layers of the surrogate's training step on the 5th-generation tensor
// cores (tcgen05): C = op(A) op(B) with the fused epilogues of the tiled
// path (FP32 / split-K partials, bias + GELU keeping the pre-activation,
// GELU' for the backward pass).
//
// One CTA computes a 128 x TN tile of C (TN <= 64, a multiple of 16) over
// its K range.  Eight warps stage K-slices of 32 into a ring of shared-memory
// buffers with cp.async (16-byte pieces, zero fill outside the operands);
// one thread issues two tcgen05.mma (M = 128, N = TN, K = 16, BF16 x BF16 ->
// FP32) per slice into a TMEM accumulator and commits each slice to the
// mbarrier that frees its buffer; after the last slice each warp drains 32
// columns of its TMEM lane quadrant (one row of C per thread) with
// tcgen05.ld and runs the epilogue.  The small tiles give the batch-sized
// training GEMMs (4096 x 256 x 256) 128 CTAs, so the epilogue math (GELU,
// GELU') spreads over most SMs.
//
// Both operand majors go straight to the tensor core.  A slice of an operand
// with R rows (M or N) is stored as core matrices of 8 x 16 bytes,
// core (r / 8, k / 8) at byte (r / 8 * 4 + k / 8) * 128: K-major sources
// (op(X)(r, k) = X[r * ld + k]) fill a core matrix with 8 rows of 8
// consecutive k, MN-major sources (op(X)(r, k) = X[k * ld + r]) with 8 k of
// 8 consecutive r; the matrix descriptor gives the same strides in both
// cases (128 B between core matrices along K, 512 B along M/N) and the
// instruction descriptor marks each operand's major.  Every global 16-byte
// piece is one contiguous core-matrix row, so a transposed operand costs no
// extra pass.
//
// Waits are bounded (1 s of global time); on expiry the CTA sets *status,
// waits (bounded) for its own MMAs, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "gelu.cuh"
#include "internal.h"

namespace cem {
namespace {

typedef __nv_bfloat16 bf16;

constexpr int TM = 128;      // rows of C per CTA (MMA M)
constexpr int TN_MAX = 64;   // columns of C per CTA (MMA N)
constexpr int KS = 32;       // K per pipeline slice (two K = 16 MMAs)
constexpr int STAGES = 6;
constexpr int THREADS = 256;  // epilogue: warp w drains lane quadrant w % 4, columns 32 (w / 4) ..
constexpr uint32_t A_BYTES = TM * KS * 2;
constexpr uint32_t B_BYTES = TN_MAX * KS * 2;
constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
constexpr uint32_t SM_BAR = STAGES * STAGE_BYTES;        // one mbarrier per stage
constexpr uint32_t SM_TMEM = SM_BAR + STAGES * 8;         // TMEM base from tcgen05.alloc
constexpr uint32_t SM_TOTAL = SM_TMEM + 16;
constexpr uint32_t TMEM_COLS = 64;
constexpr uint64_t kWaitLimitNs = 1000000000ull;
static_assert(TMEM_COLS >= TN_MAX, "accumulator columns");
static_assert(3 * SM_TOTAL <= 227 * 1024, "three CTAs per SM");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// matrix descriptor, no swizzle: start >> 4 (bits 0-13), K-direction core
// stride >> 4 (bits 16-29), M/N-direction core stride >> 4 (bits 32-45),
// version 1 (bits 46-47)
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((512u >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1u << 46;
  return d;
}

// instruction descriptor of kind::f16: D FP32 (bit 4), A and B BF16 (bits
// 7, 10), A / B MN-major (bits 15 / 16), N >> 3 (bits 17-22), M >> 4 (bits 24-28)
__device__ __forceinline__ uint32_t make_idesc(int N, int a_mn, int b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
  uint64_t t0 = 0;
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(phase)
        : "memory");
    if (done) return true;
    const uint64_t t = global_ns();
    if (t0 == 0) t0 = t;
    else if (t - t0 > kWaitLimitNs) return false;
  }
}

// 16 bytes global -> shared, zero-filled when !valid (no byte is read then)
__device__ __forceinline__ void cp16(uint32_t dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}

// 16 bytes into shared memory from registers
__device__ __forceinline__ void st16(uint32_t dst, uint4 v) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(dst), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
               : "memory");
}

// one K-slice [k0, k0 + KS) of an operand with `rows` rows starting at r0
// (extent nrows) into its core-matrix layout at dst; ones_at > 0 (MN-major
// only): rows from ones_at on are not read, row ones_at is 1 and the rest 0
__device__ __forceinline__ void stage_operand(uint32_t dst, const bf16* X, int ld, int kmajor, int r0, int rows,
                                              int nrows, int k0, int kend, int tid, int ones_at = 0) {
  // consecutive threads fill consecutive 16-byte rows of a core matrix
  // (conflict-free shared-memory stores)
  for (int i = tid; i < rows * (KS / 8); i += THREADS) {
    if (kmajor) {  // piece (r, kb): k = k0 + 8 kb .. + 7 of row r
      const int r = i % rows, kb = i / rows;
      const int gr = r0 + r, gk = k0 + kb * 8;
      const bool ok = gr < nrows && gk < kend;
      cp16(dst + (uint32_t)(((r >> 3) * 4 + kb) * 128 + (r & 7) * 16), ok ? X + (size_t)gr * ld + gk : X, ok);
    } else {  // piece (k, g): rows r0 + 8 g .. + 7 at k
      const int k = i % KS, g = i / KS;
      const int gk = k0 + k, gr = r0 + g * 8;
      const uint32_t d = dst + (uint32_t)((g * 4 + (k >> 3)) * 128 + (k & 7) * 16);
      if (ones_at > 0 && gr >= ones_at) {  // BF16 1.0 in the first element of row ones_at
        st16(d, make_uint4(gr == ones_at && gk < kend ? 0x3F80u : 0u, 0u, 0u, 0u));
        continue;
      }
      const bool ok = gk < kend && gr < nrows;
      cp16(d, ok ? X + (size_t)gk * ld + gr : X, ok);
    }
  }
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}

template <int EPI>
__global__ void __launch_bounds__(THREADS) gemm_tc_kernel(const GemmArgs g, int* status) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ volatile int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN_MAX;
  const int tn = g.N - n0 < TN_MAX ? g.N - n0 : TN_MAX;  // a multiple of 16
  const int kbeg = g.kchunk > 0 ? (int)blockIdx.z * g.kchunk : 0;
  const int kend = g.kchunk > 0 ? min(g.K, kbeg + g.kchunk) : g.K;
  const int nk = kend > kbeg ? (kend - kbeg + KS - 1) / KS : 0;
  const uint32_t base = smem_u32(sm), bar0 = base + SM_BAR;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + SM_TMEM);

  if (tid == 0) {
    s_fail = 0;
    for (int s = 0; s < STAGES; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8 * s));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();  // tcgen05.alloc is warp-collective
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = make_idesc(tn, g.a_kmajor ? 0 : 1, g.b_kmajor ? 0 : 1);

  auto load_slice = [&](int kc) {
    const uint32_t sa = base + (uint32_t)(kc % STAGES) * STAGE_BYTES, sb = sa + A_BYTES;
    const int k0 = kbeg + kc * KS;
    stage_operand(sa, g.A, g.lda, g.a_kmajor, m0, TM, g.M, k0, kend, tid);
    stage_operand(sb, g.B, g.ldb, g.b_kmajor, n0, tn, g.N, k0, kend, tid, g.n_real);
  };

  for (int s = 0; s < STAGES - 1; ++s) {
    if (s < nk) load_slice(s);
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  int issued = 0;  // slices whose MMAs were issued (the same in every thread)
  for (int kc = 0; kc < nk; ++kc) {
    const int nxt = kc + STAGES - 1;
    if (nxt < nk) {
      // slice nxt reuses the buffer of slice kc - 1: wait for that slice's MMAs
      if (kc >= 1 && !mbar_wait(bar0 + 8 * ((kc - 1) % STAGES), (uint32_t)((kc - 1) / STAGES) & 1u)) s_fail = 1;
      load_slice(nxt);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group %0;" ::"n"(STAGES - 1) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (s_fail) break;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = base + (uint32_t)(kc % STAGES) * STAGE_BYTES, sb = sa + A_BYTES;
#pragma unroll
      for (int kk = 0; kk < KS; kk += 16) {
        const uint32_t acc = (kc > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(make_desc(sa + (uint32_t)(kk >> 3) * 128u)), "l"(make_desc(sb + (uint32_t)(kk >> 3) * 128u)),
            "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       bar0 + 8 * (kc % STAGES))
                   : "memory");
    }
    issued = kc + 1;
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  // the last issued slice's commit covers every MMA of this CTA
  if (issued > 0 && !mbar_wait(bar0 + 8 * ((issued - 1) % STAGES), (uint32_t)((issued - 1) / STAGES) & 1u))
    s_fail = 2;
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int fail = s_fail;
  if (fail) {
    if (tid == 0) atomicExch(status, fail);
  } else {
    const int quad = warp & 3, cbeg = (warp >> 2) * 32;
    const int m = m0 + quad * 32 + lane;
    const int cend = cbeg + 32 < tn ? cbeg + 32 : tn;
    for (int c = cbeg; c < cend; c += 16) {
      float v[16];
      if (nk > 0) tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c, v);
      else
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = 0.0f;
      if (m >= g.M) continue;
      const int n = n0 + c;
      if (EPI == EPI_F32) {
        if (!g.part && g.n_real > 0 && n >= g.n_real) {  // the ones column: a row sum
          if (n == g.n_real) g.cbias[m] = v[0];
          continue;
        }
        float* dst = g.part ? g.part + ((size_t)blockIdx.z * g.M + m) * g.N + n : g.C + (size_t)m * g.ldc + n;
#pragma unroll
        for (int q = 0; q < 4; ++q)
          reinterpret_cast<float4*>(dst)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      } else if (EPI == EPI_BIAS_GELU) {
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] += g.bias[n + i];
        if (g.C) {
          float* dst = g.C + (size_t)m * g.ldc + n;
#pragma unroll
          for (int q = 0; q < 4; ++q)
            reinterpret_cast<float4*>(dst)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        }
        uint32_t w[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) w[i] = pack_bf16x2(gelu(v[2 * i]), gelu(v[2 * i + 1]));
        uint4* dst = reinterpret_cast<uint4*>(g.Cb + (size_t)m * g.ldcb + n);
        dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
        dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
      } else {
        const float* zs = g.zsave + (size_t)m * g.ldz + n;
        uint32_t w[8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
          w[i] = pack_bf16x2(v[2 * i] * gelu_grad(zs[2 * i]), v[2 * i + 1] * gelu_grad(zs[2 * i + 1]));
        uint4* dst = reinterpret_cast<uint4*>(g.Cb + (size_t)m * g.ldcb + n);
        dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
        dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

bool gemm_tc_supported(const GemmArgs& g) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0) return false;
  if (g.N % 16 != 0) return false;  // MMA N
  // every 16-byte piece lies inside one row of its operand
  if (g.a_kmajor ? (g.K % 8 != 0) : (g.M % 8 != 0)) return false;
  if (g.b_kmajor ? (g.K % 8 != 0) : (g.N % 8 != 0)) return false;
  if (g.lda % 8 != 0 || g.ldb % 8 != 0) return false;
  if (!aligned16(g.A) || !aligned16(g.B)) return false;
  if (g.kchunk > 0 && g.kchunk % KS != 0) return false;
  // the epilogue stores 16 columns as whole vectors
  if (g.C && (g.ldc % 4 != 0 || !aligned16(g.C))) return false;
  if (g.Cb && (g.ldcb % 8 != 0 || !aligned16(g.Cb))) return false;
  if (g.part && !aligned16(g.part)) return false;
  if (g.n_real > 0 && (g.b_kmajor || g.n_real % 16 != 0 || g.N != g.n_real + 16 || !g.cbias)) return false;
  return true;
}

cudaError_t gemm_tc(int epi, const GemmArgs& g, int* status, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  constexpr int kMaxDevices = 64;
  static std::atomic<bool> configured[kMaxDevices][3];  // host threads may race here; the set-up is idempotent
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices || epi < 0 || epi > 2) return cudaErrorInvalidValue;
  if (!configured[dev][epi].load(std::memory_order_acquire)) {
    e = epi == EPI_F32 ? cudaFuncSetAttribute(gemm_tc_kernel<EPI_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)SM_TOTAL)
        : epi == EPI_BIAS_GELU
            ? cudaFuncSetAttribute(gemm_tc_kernel<EPI_BIAS_GELU>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)SM_TOTAL)
            : cudaFuncSetAttribute(gemm_tc_kernel<EPI_GELU_BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)SM_TOTAL);
    if (e != cudaSuccess) return e;
    configured[dev][epi].store(true, std::memory_order_release);
  }
  const int S = (epi == EPI_F32 && g.part && g.kchunk > 0) ? (g.K + g.kchunk - 1) / g.kchunk : 1;
  GemmArgs h = g;
  if (S == 1) {  // one chunk: write C directly
    h.kchunk = 0;
    h.part = nullptr;
  }
  const dim3 grid((g.N + TN_MAX - 1) / TN_MAX, (g.M + TM - 1) / TM, S);
  if (epi == EPI_F32) gemm_tc_kernel<EPI_F32><<<grid, THREADS, SM_TOTAL, st>>>(h, status);
  else if (epi == EPI_BIAS_GELU) gemm_tc_kernel<EPI_BIAS_GELU><<<grid, THREADS, SM_TOTAL, st>>>(h, status);
  else gemm_tc_kernel<EPI_GELU_BWD><<<grid, THREADS, SM_TOTAL, st>>>(h, status);
  return cudaGetLastError();
}

}  // namespace cem
