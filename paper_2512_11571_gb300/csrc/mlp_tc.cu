// Fused surrogate forward on the 5th-generation tensor cores (tcgen05).
//
// One CTA scores 128 candidates through the whole MLP (48 -> 4 x 256 GELU ->
// 1): the activation tile stays in shared memory between layers, each
// layer's weights arrive by bulk TMA copies (cp.async.bulk) from a pre-packed
// global image, one thread issues the tcgen05.mma sequence (M = 128,
// N = 256, K = 16, BF16 x BF16 -> FP32) into a 256-column TMEM accumulator,
// and 8 warps drain TMEM with tcgen05.ld, add the bias, apply GELU and write
// BF16 activations back as the next layer's A operand.  The output layer is a
// dot product fused into the last epilogue.  Rounding points are those of
// the tiled GEMM path: BF16 inputs, weights and activations, FP32
// accumulation, FP32 bias and GELU.  The GELU's erf is the rational
// approximation 7.1.28 of Abramowitz & Stegun (absolute error <= 3e-7, far
// below the BF16 rounding of the activation), evaluated on pairs of
// activations with the packed FP32x2 instructions (fma/mul/add.rn.f32x2:
// two IEEE operations per instruction, half the issue slots of scalar
// code); each warp double-buffers its TMEM loads so the next 32 columns
// are in flight while the current ones are processed; biases and output
// weights are staged in shared memory.
//
// Operands use the canonical K-major layout without swizzling: 8-row x
// 16-byte core matrices stored contiguously (128 B), core matrices adjacent
// along K 128 B apart (leading byte offset), adjacent along M/N K/8 * 128 B
// apart (stride byte offset).  Every wait on an mbarrier is bounded: on
// expiry the CTA records an error code, writes NaN scores for its rows,
// waits (bounded) for its own copies and MMAs in flight, frees its TMEM and
// returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace cem {
namespace {

typedef __nv_bfloat16 bf16;

constexpr int TM = 128;       // rows per CTA (MMA M)
constexpr int WIDTH = 256;    // hidden width (MMA N)
constexpr int IN = 48;        // input features
constexpr int DEPTH = 4;      // hidden layers
constexpr int THREADS = 256;  // 8 warps
constexpr uint64_t kWaitLimitNs = 1000000000ull;  // give up on a pipeline wait after 1 s
constexpr uint32_t kChunk = 16384;  // bytes per bulk copy

// bytes of a [rows x K] BF16 operand
__host__ __device__ constexpr uint32_t operand_bytes(int rows, int K) { return (uint32_t)rows * (uint32_t)K * 2u; }

// byte offset of element (r, k) of a [rows x K] operand in the canonical
// K-major layout (no swizzle): core matrix (r / 8, k / 8), row r % 8 (16 B),
// element k % 8 (2 B)
__host__ __device__ __forceinline__ uint32_t canon_off(int r, int k, int K) {
  return (uint32_t)(r >> 3) * (uint32_t)(K >> 3) * 128u + (uint32_t)(k >> 3) * 128u + (uint32_t)(r & 7) * 16u +
         (uint32_t)(k & 7) * 2u;
}

// packed weight image: W0 [256 x 48], W1..W3 [256 x 256], each canonical
__host__ __device__ constexpr uint32_t w_offset(int l) {
  return l == 0 ? 0u : operand_bytes(WIDTH, IN) + (uint32_t)(l - 1) * operand_bytes(WIDTH, WIDTH);
}
constexpr uint32_t kPackBytes = operand_bytes(WIDTH, IN) + 3u * operand_bytes(WIDTH, WIDTH);

// shared memory plan (bytes)
constexpr uint32_t SM_A = 0;                                     // activations [128 x 256]
constexpr uint32_t SM_W = SM_A + operand_bytes(TM, WIDTH);        // weights [256 x 256]
constexpr uint32_t SM_PART = SM_W + operand_bytes(WIDTH, WIDTH);  // 128 partial dot products
constexpr uint32_t SM_BAR = SM_PART + TM * 4;                     // 2 mbarriers
constexpr uint32_t SM_TMEM = SM_BAR + 16;                         // TMEM base from tcgen05.alloc
constexpr uint32_t SM_TOTAL = SM_TMEM + 16;
static_assert(SM_TOTAL <= 227 * 1024, "shared memory plan exceeds 227 KB");
static_assert(operand_bytes(WIDTH, IN) % 16 == 0 && operand_bytes(WIDTH, WIDTH) % 16 == 0,
              "bulk copies move whole 16-byte units");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// tcgen05 shared-memory matrix descriptor, no swizzle: start address >> 4
// (bits 0-13), leading byte offset >> 4 (bits 16-29), stride byte offset
// >> 4 (bits 32-45), descriptor version 1 (bits 46-47)
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1u << 46;
  return d;
}

// instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, bits 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at
// bits 17-22, M >> 4 at bits 24-28
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// wait for the completion of the phase with parity `phase`; false once
// kWaitLimitNs of global time has passed without it
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

// one thread: copy `bytes` (a multiple of 16) from global to shared through
// the TMA unit in kChunk pieces, completion counted on `bar`
__device__ __forceinline__ void bulk_load(uint32_t dst, const uint8_t* src, uint32_t bytes, uint32_t bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
  for (uint32_t o = 0; o < bytes; o += kChunk) {
    const uint32_t n = bytes - o < kChunk ? bytes - o : kChunk;
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst + o),
        "l"(src + o), "r"(n), "r"(bar)
        : "memory");
  }
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// arrive on `bar` once every tcgen05.mma issued so far by this thread is done
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// issue a load of 32 consecutive FP32 columns of this thread's TMEM lane;
// the registers hold the values only after tmem_wait32 on the same array
__device__ __forceinline__ void tmem_issue32(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

// wait for this thread's TMEM loads; the registers are operands of the wait,
// so the compiler reads none of them before it
__device__ __forceinline__ void tmem_wait32(uint32_t* r) {
  asm volatile(
      "tcgen05.wait::ld.sync.aligned;"
      : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
        "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]),
        "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
        "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
      :
      : "memory");
}

// a pair of FP32 values in one 64-bit register (low, high)
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pk2(float lo, float hi) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void upk2(f32x2 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 ffma2(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f32x2 fmul2(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 fadd2(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// GELU(z) = z Phi(z) of a pair.  With a = |z| and E = erf(a / sqrt 2) =
// 1 - (1 + p(a))^-16 (Abramowitz & Stegun 7.1.28, its coefficients a_i
// scaled by 2^(-i/2) so the polynomial takes a directly), z Phi(z) =
// (z + a E) / 2 for either sign of z, i.e. (z + a) / 2 - (a / 2) (1 + p(a))^-16.
// Overflow of the 16th power to inf gives the exact limit relu(z).
__device__ __forceinline__ f32x2 gelu2(f32x2 z) {
  const f32x2 K1 = pk2(4.986734688e-02f, 4.986734688e-02f), K2 = pk2(2.114100568e-02f, 2.114100568e-02f);
  const f32x2 K3 = pk2(3.277626354e-03f, 3.277626354e-03f), K4 = pk2(3.800357445e-05f, 3.800357445e-05f);
  const f32x2 K5 = pk2(4.889063712e-05f, 4.889063712e-05f), K6 = pk2(5.382974905e-06f, 5.382974905e-06f);
  const f32x2 ONE = pk2(1.0f, 1.0f), HALF = pk2(0.5f, 0.5f);
  const f32x2 a = z & 0x7fffffff7fffffffull;  // |z| of both halves
  f32x2 p = ffma2(a, K6, K5);
  p = ffma2(a, p, K4);
  p = ffma2(a, p, K3);
  p = ffma2(a, p, K2);
  p = ffma2(a, p, K1);
  p = ffma2(a, p, ONE);
  f32x2 q = fmul2(p, p);  // p^16 by four squarings
  q = fmul2(q, q);
  q = fmul2(q, q);
  q = fmul2(q, q);
  float q0, q1;
  upk2(q, q0, q1);
  const f32x2 nr = pk2(-rcp_approx(q0), -rcp_approx(q1));
  const f32x2 ha = fmul2(a, HALF);
  return ffma2(ha, nr, ffma2(z, HALF, ha));
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}

__global__ void __launch_bounds__(THREADS, 1) mlp_forward_tc_kernel(const MlpTcArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ volatile int s_fail;
  __shared__ __align__(16) float sbias[DEPTH * WIDTH];
  __shared__ __align__(16) float swout[WIDTH];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row0 = blockIdx.x * TM;
  const uint32_t sA = smem_u32(sm + SM_A), sW = smem_u32(sm + SM_W);
  const uint32_t bar_w = smem_u32(sm + SM_BAR), bar_mma = bar_w + 8;
  float* part = reinterpret_cast<float*>(sm + SM_PART);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + SM_TMEM);
  const uint8_t* wpack = static_cast<const uint8_t*>(a.wpack);
  const bf16* x = static_cast<const bf16*>(a.x);
  const bf16* w_out = static_cast<const bf16*>(a.w_out);

  if (tid == 0) {
    s_fail = 0;
    mbar_init(bar_w, 1);
    mbar_init(bar_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0) {  // 256 TMEM columns: one FP32 accumulator row per lane
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(WIDTH));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
#pragma unroll
  for (int l = 0; l < DEPTH; ++l)
    for (int i = tid; i < WIDTH; i += THREADS) sbias[l * WIDTH + i] = a.bias[l][i];
  for (int i = tid; i < WIDTH; i += THREADS) swout[i] = __bfloat162float(w_out[i]);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  // (the failure-detection test leaves the barrier without its arrival, so
  // nothing completes it and the first wait runs out with nothing in flight)
  if (tid == 0 && !a.expire_test) bulk_load(sW, wpack + w_offset(0), operand_bytes(WIDTH, IN), bar_w);
  // input tile: 128 rows of 48 BF16 features, 16-byte pieces into the
  // canonical layout; rows past M are zero
  for (int i = tid; i < TM * (IN / 8); i += THREADS) {
    const int r = i / (IN / 8), kb = i % (IN / 8);
    const int m = row0 + r;
    uint4 q = make_uint4(0u, 0u, 0u, 0u);
    if (m < a.M) q = *reinterpret_cast<const uint4*>(x + (size_t)m * IN + kb * 8);
    *reinterpret_cast<uint4*>(sm + SM_A + canon_off(r, kb * 8, IN)) = q;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();

  const uint32_t idesc = make_idesc(TM, WIDTH);
  const int quad = warp & 3, half = warp >> 2;  // TMEM lanes 32 quad.., columns 128 half..
  const int r_local = quad * 32 + lane;
  uint32_t ph_w = 0, ph_mma = 0;
  int pending_w = 1, pending_mma = 0;  // copies / MMAs in flight
  float dot = 0.0f;
  for (int l = 0; l < DEPTH; ++l) {
    const int K = l == 0 ? IN : WIDTH;
    if (!mbar_wait(bar_w, ph_w)) s_fail = 1;
    __syncthreads();
    if (s_fail) break;
    ph_w ^= 1;
    pending_w = 0;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sbo = (uint32_t)(K >> 3) * 128u;
      for (int k0 = 0; k0 < K; k0 += 16) {
        const uint64_t ad = make_desc(sA + (uint32_t)(k0 >> 3) * 128u, 128u, sbo);
        const uint64_t bd = make_desc(sW + (uint32_t)(k0 >> 3) * 128u, 128u, sbo);
        mma_bf16(tmem, ad, bd, idesc, k0 > 0 ? 1u : 0u);
      }
      mma_commit(bar_mma);
    }
    pending_mma = 1;
    if (!mbar_wait(bar_mma, ph_mma)) s_fail = 2;
    __syncthreads();
    if (s_fail) break;
    ph_mma ^= 1;
    pending_mma = 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // the MMAs have finished reading A and W: fetch the next weights now,
    // overlapping the epilogue
    if (l + 1 < DEPTH) {
      if (tid == 0) bulk_load(sW, wpack + w_offset(l + 1), operand_bytes(WIDTH, WIDTH), bar_w);
      pending_w = 1;
    }
    __syncwarp();  // tcgen05.ld is warp-collective: reconverge after thread 0's copy issue
    // epilogue: TMEM -> bias + GELU -> BF16 activations (or the output dot)
    const float* bl = sbias + l * WIDTH;
    // this warp's 128 columns in 4 steps of 32, the next step's TMEM load
    // in flight while the current step is processed
    const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(half * 128);
    uint32_t ra[32], rb[32];
    tmem_issue32(tbase, ra);
    tmem_wait32(ra);
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      uint32_t* cur = (cc & 1) ? rb : ra;
      uint32_t* nxt = (cc & 1) ? ra : rb;
      if (cc + 1 < 4) tmem_issue32(tbase + 32u * (uint32_t)(cc + 1), nxt);
      const int c0 = half * 128 + 32 * cc;
      float v[32];
#pragma unroll
      for (int j = 0; j < 32; j += 2) {
        const float2 b2 = *reinterpret_cast<const float2*>(bl + c0 + j);
        const f32x2 g = gelu2(fadd2(pk2(__uint_as_float(cur[j]), __uint_as_float(cur[j + 1])), pk2(b2.x, b2.y)));
        upk2(g, v[j], v[j + 1]);
      }
      if (l + 1 < DEPTH) {  // packing rounds to BF16 once
#pragma unroll
        for (int kb = 0; kb < 4; ++kb) {
          const uint4 q =
              make_uint4(pack_bf16x2(v[8 * kb], v[8 * kb + 1]), pack_bf16x2(v[8 * kb + 2], v[8 * kb + 3]),
                         pack_bf16x2(v[8 * kb + 4], v[8 * kb + 5]), pack_bf16x2(v[8 * kb + 6], v[8 * kb + 7]));
          *reinterpret_cast<uint4*>(sm + SM_A + canon_off(r_local, c0 + 8 * kb, WIDTH)) = q;
        }
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) dot = fmaf(__bfloat162float(__float2bfloat16_rn(v[j])), swout[c0 + j], dot);
      }
      if (cc + 1 < 4) tmem_wait32(nxt);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
  }
  const int fail = s_fail;
  if (!fail) {
    if (half == 1) part[r_local] = dot;
    __syncthreads();
    if (half == 0) {
      const int m = row0 + r_local;
      if (m < a.M) a.y[m] = a.norm[0] + a.norm[1] * ((dot + part[r_local]) + a.b_out[0]);
    }
  } else {
    // drain what this CTA still has in flight (bounded), report, poison rows
    if (pending_mma) mbar_wait(bar_mma, ph_mma);
    if (pending_w) mbar_wait(bar_w, ph_w);
    if (tid == 0) atomicExch(a.status, fail);
    if (tid < TM && row0 + tid < a.M) a.y[row0 + tid] = __int_as_float(0x7fc00000);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(WIDTH));
}

// W0..W3 (BF16, out x in row-major, at element offsets off.w[l] of the flat
// BF16 parameter vector) -> the canonical packed image
__global__ void pack_weights_kernel(const bf16* __restrict__ pb, MlpTcOffsets off, uint8_t* __restrict__ out) {
  const int l = blockIdx.y;
  const int K = l == 0 ? IN : WIDTH;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= WIDTH * K) return;
  const int n = i / K, k = i % K;
  *reinterpret_cast<bf16*>(out + w_offset(l) + canon_off(n, k, K)) = pb[off.w[l] + i];
}

}  // namespace

bool mlp_tc_supported(int in_dim, int width, int depth) { return in_dim == IN && width == WIDTH && depth == DEPTH; }

size_t mlp_tc_pack_bytes() { return kPackBytes; }

cudaError_t mlp_tc_pack(const void* pb, const MlpTcOffsets& off, void* pack, cudaStream_t st) {
  const dim3 grid((WIDTH * WIDTH + 255) / 256, DEPTH);
  pack_weights_kernel<<<grid, 256, 0, st>>>(static_cast<const bf16*>(pb), off, static_cast<uint8_t*>(pack));
  return cudaGetLastError();
}

cudaError_t mlp_tc_forward(const MlpTcArgs& a, cudaStream_t st) {
  if (a.M <= 0) return cudaSuccess;
  static bool configured = false;
  if (!configured) {
    const cudaError_t e =
        cudaFuncSetAttribute(mlp_forward_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM_TOTAL);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  mlp_forward_tc_kernel<<<(a.M + TM - 1) / TM, THREADS, SM_TOTAL, st>>>(a);
  return cudaGetLastError();
}

}  // namespace cem
