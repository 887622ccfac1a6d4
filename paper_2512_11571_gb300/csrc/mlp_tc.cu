// Fused surrogate forward on the 5th-generation tensor cores (tcgen05).
//
// Scores candidates through the whole MLP (48 -> 4 x 256 GELU -> 1) in one
// persistent launch: one CTA per SM walks over 128-row tiles.  Per CTA, one
// warp issues the weight copies (cp.async.bulk) and the tcgen05.mma sequence
// (M = 128, N = 256, K = 16, BF16 x BF16 -> FP32); 16 epilogue warps drain
// the accumulator with tcgen05.ld, add the bias, apply GELU and write BF16
// activations back into shared memory as the next layer's A operand.
//
// Pipeline.  Two 256-column FP32 accumulators in TMEM serve alternate
// layers, so the next layer's MMAs run while the epilogue still reads the
// current one: the epilogue works in two steps of 32 columns per warp, and
// as soon as every warp has written step c (K-slices c, c + 2, c + 4, c + 6
// of the next layer's A) the MMA warp issues those slices' MMAs.  Hidden
// weights stream through shared memory in 16 KB K-slices: slice j of the
// next layer (or of layer 1 of the next tile) is copied in as soon as the
// MMAs reading slice j of the current layer have finished.  W0 [256 x 48]
// stays resident.  The last layer's epilogue writes no activations, so it
// stages the next tile's input features into the A buffer and the MMA warp
// starts that tile's first layer while the output dot product is finished.
//
// Arithmetic.  Rounding points are those of the tiled GEMM path: BF16
// inputs, weights and activations, FP32 accumulation, FP32 bias and GELU.
// The GELU's erf is the rational approximation 7.1.28 of Abramowitz &
// Stegun (absolute error <= 3e-7, far below the BF16 rounding of the
// activation), evaluated on pairs of activations with the packed FP32x2
// instructions (fma/mul/add.rn.f32x2: two IEEE operations per
// instruction); TMEM loads are double-buffered; biases and output weights
// are staged in shared memory.  The K-slices of a layer accumulate in the
// order the epilogue releases them (0, 2, 4, 6, 1, 3, 5, 7).
//
// Operands use the canonical K-major layout without swizzling: 8-row x
// 16-byte core matrices stored contiguously (128 B), core matrices adjacent
// along K 128 B apart (leading byte offset), adjacent along M/N K/8 * 128 B
// apart (stride byte offset).  Every wait on an mbarrier is bounded: on
// expiry the CTA records an error code, writes NaN scores for all its rows,
// waits (bounded) for its own copies and MMAs in flight, frees its TMEM and
// returns; a flag in shared memory ends the other warps' waits at once.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "internal.h"

namespace cem {
namespace {

typedef __nv_bfloat16 bf16;

constexpr int TM = 128;       // rows per CTA (MMA M)
constexpr int WIDTH = 256;    // hidden width (MMA N)
constexpr int IN = 48;        // input features
constexpr int DEPTH = 4;      // hidden layers
constexpr int KC = 32;        // K per streamed weight slice
constexpr int NCH = WIDTH / KC;  // slices per hidden layer
constexpr int NSTEP = 2;         // epilogue steps per layer (32 columns per warp each)
constexpr int EWARPS = 16;       // epilogue warps: 4 TMEM lane quadrants x 4 column quarters
constexpr int ETHREADS = EWARPS * 32;
constexpr int THREADS = ETHREADS + 32;  // + the MMA warp
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

// packed weight image: W0 [256 x 48] canonical; W1..W3 [256 x 256], scaled
// by 1/2 (see gelu2), each as 8 contiguous K-slices [256 x 32], every slice
// canonical with K = 32
__host__ __device__ constexpr uint32_t w_offset(int l) {
  return l == 0 ? 0u : operand_bytes(WIDTH, IN) + (uint32_t)(l - 1) * operand_bytes(WIDTH, WIDTH);
}
constexpr uint32_t kPackBytes = operand_bytes(WIDTH, IN) + 3u * operand_bytes(WIDTH, WIDTH);
constexpr uint32_t kSliceBytes = operand_bytes(WIDTH, KC);

// shared memory plan (bytes)
constexpr uint32_t SM_A = 0;                                     // activations [128 x 256]
constexpr uint32_t SM_W = SM_A + operand_bytes(TM, WIDTH);        // hidden weights, 8 slices
constexpr uint32_t SM_W0 = SM_W + operand_bytes(WIDTH, WIDTH);    // W0 [256 x 48]
constexpr uint32_t SM_PART = SM_W0 + operand_bytes(WIDTH, IN);    // 3 x 128 partial dot products
constexpr uint32_t SM_BAR = SM_PART + 3 * TM * 4;
// mbarriers: W0 copy, slice copies [8], a step's slices free [2 of 8 used],
// activation steps [2], accumulator ready, drain, next input staged
constexpr int NBAR = 1 + 2 * NCH + NSTEP + 3;
constexpr uint32_t SM_TMEM = SM_BAR + NBAR * 8;                   // TMEM base from tcgen05.alloc
constexpr uint32_t SM_TOTAL = SM_TMEM + 16;
static_assert(SM_TOTAL + (DEPTH + 1) * WIDTH * 4 + 64 <= 227 * 1024, "shared memory plan exceeds 227 KB");
static_assert(operand_bytes(WIDTH, IN) % 16 == 0 && kSliceBytes % 16 == 0, "bulk copies move whole 16-byte units");

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

// mbar_wait that also gives up as soon as *fail is set by another thread
__device__ __forceinline__ bool mbar_wait_or(uint32_t bar, uint32_t phase, volatile int* fail) {
  uint64_t t0 = 0;
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(phase)
        : "memory");
    if (done) return true;
    if (*fail) return false;
    const uint64_t t = global_ns();
    if (t0 == 0) t0 = t;
    else if (t - t0 > kWaitLimitNs) return false;
  }
}

__device__ __forceinline__ void bar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// one thread: one bulk copy of `bytes` (a multiple of 16, at most kChunk)
__device__ __forceinline__ void copy_async(uint32_t dst, const uint8_t* src, uint32_t bytes, uint32_t bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
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

// 2 GELU(z) = 2 z Phi(z) of a pair.  With a = |z| and E = erf(a / sqrt 2) =
// 1 - (1 + p(a))^-16 (Abramowitz & Stegun 7.1.28, its coefficients a_i
// scaled by 2^(-i/2) so the polynomial takes a directly), 2 z Phi(z) =
// z + a E for either sign of z, i.e. (z + a) - a (1 + p(a))^-16.  The factor
// 1/2 of GELU lives in the packed weights of the next layer (and in the
// output weights): scaling by a power of two is exact in BF16 and FP32, so
// every product the tensor core forms is unchanged.  Overflow of the 16th
// power to inf gives the exact limit 2 relu(z).
__device__ __forceinline__ f32x2 gelu2(f32x2 z) {
  const f32x2 K1 = pk2(4.986734688e-02f, 4.986734688e-02f), K2 = pk2(2.114100568e-02f, 2.114100568e-02f);
  const f32x2 K3 = pk2(3.277626354e-03f, 3.277626354e-03f), K4 = pk2(3.800357445e-05f, 3.800357445e-05f);
  const f32x2 K5 = pk2(4.889063712e-05f, 4.889063712e-05f), K6 = pk2(5.382974905e-06f, 5.382974905e-06f);
  const f32x2 ONE = pk2(1.0f, 1.0f);
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
  return ffma2(a, nr, fadd2(z, a));
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
  const uint32_t sA = smem_u32(sm + SM_A), sW = smem_u32(sm + SM_W), sW0 = smem_u32(sm + SM_W0);
  const uint32_t wbar0 = smem_u32(sm + SM_BAR);
  const uint32_t wbar = wbar0 + 8, wfree = wbar + 8 * NCH, abar = wfree + 8 * NCH;
  const uint32_t bar_mma = abar + 8 * NSTEP, bar_drain = bar_mma + 8, xbar = bar_drain + 8;
  const int ntiles = (a.M + TM - 1) / TM;
  float* part = reinterpret_cast<float*>(sm + SM_PART);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + SM_TMEM);
  const uint8_t* wpack = static_cast<const uint8_t*>(a.wpack);
  const bf16* x = static_cast<const bf16*>(a.x);
  const bf16* w_out = static_cast<const bf16*>(a.w_out);

  if (tid == 0) {
    s_fail = 0;
    mbar_init(wbar0, 1);
    for (int j = 0; j < NCH; ++j) {
      mbar_init(wbar + 8 * j, 1);
      mbar_init(wfree + 8 * j, 1);
    }
    for (int c = 0; c < NSTEP; ++c) mbar_init(abar + 8 * c, EWARPS);
    mbar_init(bar_mma, 1);
    mbar_init(bar_drain, 1);
    mbar_init(xbar, EWARPS);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0) {  // two 256-column FP32 accumulators, used by alternate layers
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * WIDTH));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
#pragma unroll
  for (int l = 0; l < DEPTH; ++l)
    for (int i = tid; i < WIDTH; i += THREADS) sbias[l * WIDTH + i] = a.bias[l][i];
  for (int i = tid; i < WIDTH; i += THREADS) swout[i] = 0.5f * __bfloat162float(w_out[i]);  // see gelu2
  for (int i = tid; i < TM * (IN / 8); i += THREADS) {
    const int r = i % TM, kb = i / TM;  // consecutive threads: consecutive rows, conflict-free stores
    const int m = (int)blockIdx.x * TM + r;
    uint4 q = make_uint4(0u, 0u, 0u, 0u);
    if (m < a.M) q = *reinterpret_cast<const uint4*>(x + (size_t)m * IN + kb * 8);
    *reinterpret_cast<uint4*>(sm + SM_A + canon_off(r, kb * 8, IN)) = q;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == EWARPS) {
    // ---- MMA warp: one lane issues the weight copies and the MMAs ----
    if (lane == 0) {
      const uint32_t idesc = make_idesc(TM, WIDTH);
      int fail = 0;
      uint32_t pend_w = 0;  // bit j < NCH: slice j copy not yet waited for; bit NCH: W0
      uint32_t pph = 0;     // bit j: the parity that copy completes
      bool pend_mma = false;
      // (the failure-detection test leaves W0's barrier without its arrival)
      if (!a.expire_test) {
        bulk_load(sW0, wpack + w_offset(0), operand_bytes(WIDTH, IN), wbar0);
        pend_w |= 1u << NCH;
      }
      for (int j = 0; j < NCH; ++j)
        copy_async(sW + j * kSliceBytes, wpack + w_offset(1) + j * kSliceBytes, kSliceBytes, wbar + 8 * j);
      pend_w |= (1u << NCH) - 1u;
      if (!mbar_wait_or(wbar0, 0, &s_fail)) fail = 1;
      else pend_w &= ~(1u << NCH);
      const uint32_t sbo0 = (uint32_t)(IN >> 3) * 128u;
      for (int t = blockIdx.x, it = 0; t < ntiles && !fail; t += gridDim.x, ++it) {
        const bool has_next = t + (int)gridDim.x < ntiles;
        // layer 0: K = 48 from this tile's input (written by the epilogue warps after the first tile)
        if (it > 0 && !mbar_wait_or(xbar, (uint32_t)(it - 1) & 1u, &s_fail)) {
          fail = 5;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        for (int k0 = 0; k0 < IN; k0 += 16)
          mma_bf16(tmem, make_desc(sA + (uint32_t)(k0 >> 3) * 128u, 128u, sbo0),
                   make_desc(sW0 + (uint32_t)(k0 >> 3) * 128u, 128u, sbo0), idesc, k0 > 0 ? 1u : 0u);
        mma_commit(bar_mma);
        pend_mma = true;
        for (int l = 1; l < DEPTH && !fail; ++l) {
          const uint32_t ph = (uint32_t)(it + l - 1) & 1u;  // this layer's slices and activations
          const uint32_t nph = (uint32_t)(it + l) & 1u;     // the refill's completion
          const uint32_t dcol = (uint32_t)(l & 1) * WIDTH;
          const bool refill = l + 1 < DEPTH || has_next;
          const uint8_t* nsrc = wpack + w_offset(l + 1 < DEPTH ? l + 1 : 1);
          for (int cc = 0; cc < NSTEP && !fail; ++cc) {
            // this step's slices first (their copies finished long before), then the activations
            for (int h = 0; h < 4 && !fail; ++h) {
              const int j = NSTEP * h + cc;
              if (!mbar_wait_or(wbar + 8 * j, ph, &s_fail)) fail = 3;
              else pend_w &= ~(1u << j);
            }
            if (fail || !mbar_wait_or(abar + 8 * cc, ph, &s_fail)) {
              fail = 3;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              const int j = NSTEP * h + cc;  // the slice step cc of column quarter h wrote
#pragma unroll
              for (int kk = 0; kk < KC; kk += 16) {
                const uint64_t ad =
                    make_desc(sA + (uint32_t)((j * KC + kk) >> 3) * 128u, 128u, (uint32_t)(WIDTH >> 3) * 128u);
                const uint64_t bd =
                    make_desc(sW + j * kSliceBytes + (uint32_t)(kk >> 3) * 128u, 128u, (uint32_t)(KC >> 3) * 128u);
                mma_bf16(tmem + dcol, ad, bd, idesc, (cc | h | kk) ? 1u : 0u);
              }
            }
            if (refill) mma_commit(wfree + 8 * cc);
            if (cc == NSTEP - 1) mma_commit(bar_mma);
            // the previous step's slices are free: refill them with the next layer's
            if (refill && cc >= 1) {
              if (!mbar_wait_or(wfree + 8 * (cc - 1), ph, &s_fail)) {
                fail = 4;
              } else {
                for (int h = 0; h < 4; ++h) {
                  const int j = NSTEP * h + cc - 1;
                  copy_async(sW + j * kSliceBytes, nsrc + j * kSliceBytes, kSliceBytes, wbar + 8 * j);
                  pend_w |= 1u << j;
                  pph = (pph & ~(1u << j)) | (nph << j);
                }
              }
            }
          }
          if (refill && !fail) {
            if (!mbar_wait_or(wfree + 8 * (NSTEP - 1), ph, &s_fail)) {
              fail = 4;
            } else {
              for (int h = 0; h < 4; ++h) {
                const int j = NSTEP * h + NSTEP - 1;
                copy_async(sW + j * kSliceBytes, nsrc + j * kSliceBytes, kSliceBytes, wbar + 8 * j);
                pend_w |= 1u << j;
                pph = (pph & ~(1u << j)) | (nph << j);
              }
            }
          }
        }
      }
      if (fail) {
        s_fail = fail;
        // drain (bounded): every MMA issued and every copy not yet waited for
        if (pend_mma) {
          mma_commit(bar_drain);
          mbar_wait(bar_drain, 0);
        }
        for (int j = 0; j <= NCH; ++j)
          if (pend_w & (1u << j)) mbar_wait(j == NCH ? wbar0 : wbar + 8 * j, (pph >> j) & 1u);
      }
    }
  } else {
    // ---- epilogue warps: TMEM -> bias + GELU -> BF16 activations, step by step ----
    const int quad = warp & 3, qtr = warp >> 2;  // TMEM lane quadrant, column quarter
    const int r_local = quad * 32 + lane;
    const int tid_e = tid;  // 0 .. ETHREADS - 1
    bool stop = false;  // the same value in every epilogue thread (barrier reduction)
    for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
      const bool has_next = t + (int)gridDim.x < ntiles;
      float dq[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      int l = 0;
      for (; l < DEPTH; ++l) {
        if (!mbar_wait_or(bar_mma, (uint32_t)l & 1u, &s_fail)) {
          if (!s_fail) s_fail = 2;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // the last layer leaves A free: fetch the next tile's input now, store it after the first step
        uint4 xin[2];
        const bool fetch = l + 1 == DEPTH && has_next;
        if (fetch) {
          const int tn = t + (int)gridDim.x;
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int i = tid_e + u * ETHREADS;
            const int m = tn * TM + i % TM;
            xin[u] = m < a.M && i < TM * (IN / 8) ? *reinterpret_cast<const uint4*>(x + (size_t)m * IN + (i / TM) * 8)
                             : make_uint4(0u, 0u, 0u, 0u);
          }
        }
        const float* bl = sbias + l * WIDTH;
        const uint32_t tbase =
            tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(l & 1) * WIDTH + (uint32_t)(qtr * 64);
        uint32_t ra[32], rb[32];
        tmem_issue32(tbase, ra);
        tmem_wait32(ra);
#pragma unroll
        for (int cc = 0; cc < NSTEP; ++cc) {
          uint32_t* cur = (cc & 1) ? rb : ra;
          uint32_t* nxt = (cc & 1) ? ra : rb;
          if (cc + 1 < NSTEP) tmem_issue32(tbase + 32u * (uint32_t)(cc + 1), nxt);
          const int c0 = qtr * 64 + 32 * cc;
          float v[32];
#pragma unroll
          for (int j = 0; j < 32; j += 2) {
            const float2 b2 = *reinterpret_cast<const float2*>(bl + c0 + j);
            const f32x2 g =
                gelu2(fadd2(pk2(__uint_as_float(cur[j]), __uint_as_float(cur[j + 1])), pk2(b2.x, b2.y)));
            upk2(g, v[j], v[j + 1]);
          }
          if (l + 1 < DEPTH) {
#pragma unroll
            for (int kb = 0; kb < 4; ++kb) {
              const uint4 q =
                  make_uint4(pack_bf16x2(v[8 * kb], v[8 * kb + 1]), pack_bf16x2(v[8 * kb + 2], v[8 * kb + 3]),
                             pack_bf16x2(v[8 * kb + 4], v[8 * kb + 5]), pack_bf16x2(v[8 * kb + 6], v[8 * kb + 7]));
              *reinterpret_cast<uint4*>(sm + SM_A + canon_off(r_local, c0 + 8 * kb, WIDTH)) = q;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) bar_arrive(abar + 8 * cc);
            __syncwarp();
          } else {
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
              dq[0] = fmaf(__bfloat162float(__float2bfloat16_rn(v[j])), swout[c0 + j], dq[0]);
              dq[1] = fmaf(__bfloat162float(__float2bfloat16_rn(v[j + 1])), swout[c0 + j + 1], dq[1]);
              dq[2] = fmaf(__bfloat162float(__float2bfloat16_rn(v[j + 2])), swout[c0 + j + 2], dq[2]);
              dq[3] = fmaf(__bfloat162float(__float2bfloat16_rn(v[j + 3])), swout[c0 + j + 3], dq[3]);
            }
            if (cc == 0 && fetch) {
#pragma unroll
              for (int u = 0; u < 2; ++u) {
                const int i = tid_e + u * ETHREADS;
                if (i < TM * (IN / 8))
                  *reinterpret_cast<uint4*>(sm + SM_A + canon_off(i % TM, (i / TM) * 8, IN)) = xin[u];
              }
              asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
              asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
              __syncwarp();
              if (lane == 0) bar_arrive(xbar);
              __syncwarp();
            }
          }
          if (cc + 1 < NSTEP) tmem_wait32(nxt);
        }
        // this layer's TMEM reads precede the arrivals that let a later layer overwrite them
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      }
      const float dot = (dq[0] + dq[1]) + (dq[2] + dq[3]);
      if (qtr > 0) part[(qtr - 1) * TM + r_local] = dot;
      asm volatile("bar.sync 1, %0;" ::"n"(ETHREADS));
      if (qtr == 0 && l == DEPTH) {
        const int m = t * TM + r_local;
        const float sum = (dot + part[r_local]) + (part[TM + r_local] + part[2 * TM + r_local]);
        if (m < a.M) a.y[m] = a.norm[0] + a.norm[1] * (sum + a.b_out[0]);
      }
      // part is rewritten by the next tile; all epilogue threads leave together
      int anyfail;
      asm volatile(
          "{\n .reg .pred q, p;\n setp.ne.s32 q, %1, 0;\n bar.red.or.pred p, 1, %2, q;\n selp.s32 %0, 1, 0, p;\n}\n"
          : "=r"(anyfail)
          : "r"((int)s_fail), "n"(ETHREADS)
          : "memory");
      stop = anyfail != 0;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (s_fail) {
    if (tid == 0) atomicExch(a.status, s_fail);
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x)
      if (tid < TM && t * TM + tid < a.M) a.y[t * TM + tid] = __int_as_float(0x7fc00000);
  }
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * WIDTH));
}

// W0..W3 (BF16, out x in row-major, at element offsets off.w[l] of the flat
// BF16 parameter vector) -> the packed image (W0 canonical, W1..W3 halved and
// in canonical K-slices)
__global__ void pack_weights_kernel(const bf16* __restrict__ pb, MlpTcOffsets off, uint8_t* __restrict__ out) {
  const int l = blockIdx.y;
  const int K = l == 0 ? IN : WIDTH;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= WIDTH * K) return;
  const int n = i / K, k = i % K;
  const uint32_t o = l == 0 ? canon_off(n, k, K) : (uint32_t)(k / KC) * kSliceBytes + canon_off(n, k % KC, KC);
  // layers fed by a GELU output take the factor 1/2 of GELU (exact: a power of two)
  *reinterpret_cast<bf16*>(out + w_offset(l) + o) =
      l == 0 ? pb[off.w[l] + i] : __float2bfloat16_rn(0.5f * __bfloat162float(pb[off.w[l] + i]));
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
  constexpr int kMaxDevices = 64;
  // per device: SM count once its kernel attribute is set (host threads
  // may race to set it; the attribute call is idempotent)
  static std::atomic<int> sms[kMaxDevices];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  int n_sm = sms[dev].load(std::memory_order_acquire);
  if (n_sm == 0) {
    e = cudaFuncSetAttribute(mlp_forward_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM_TOTAL);
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    n_sm = n > 0 ? n : 1;
    sms[dev].store(n_sm, std::memory_order_release);
  }
  const int ntiles = (a.M + TM - 1) / TM;
  mlp_forward_tc_kernel<<<ntiles < n_sm ? ntiles : n_sm, THREADS, SM_TOTAL, st>>>(a);
  return cudaGetLastError();
}

}  // namespace cem
