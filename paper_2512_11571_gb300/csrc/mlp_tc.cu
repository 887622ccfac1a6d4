// Fused surrogate forward on the 5th-generation tensor cores (tcgen05).
//
// Scores candidates through the whole MLP (48 -> 4 x 256 GELU -> 1) in one
// persistent launch: one CTA per SM walks over 128-row tiles, two tiles in
// flight.  Per CTA, one warp streams the hidden weights into shared memory
// (cp.async.bulk), one warp issues the tcgen05.mma sequence (M = 128,
// N = 256, K = 16, BF16 x BF16 -> FP32), and 16 epilogue warps drain a
// tile's 256-column FP32 accumulator in TMEM with tcgen05.ld, apply GELU and
// write BF16 activations back into that tile's shared-memory buffer as the
// next layer's A operand.  Each accumulation starts from the layer's bias:
// while draining, the epilogue stores the next layer's bias (tcgen05.st)
// into the columns it has read, and every MMA accumulates onto it.
//
// Pipeline.  Each tile in flight has its own accumulator (2 x 256 of the 512
// TMEM columns) and its own activation buffer.  The MMA warp and the
// epilogue warps walk the same sequence of (tile, layer) jobs: tile a layer
// l, tile b layer l, tile a layer l + 1, ..., so the epilogue drains one
// tile's accumulator while the tensor core computes the other tile's layer.
// Hidden weights stream through a ring of four 16 KB K-slices in the order
// the MMAs use them (every hidden layer's eight slices, once per tile), each
// slice refilled as soon as the MMAs reading it finish; W0 [256 x 48] stays
// resident.  While a tile's last layer is drained, the next tile's input
// rows are copied into the tile's buffer with cp.async (BF16 rows straight
// into place; FP32 rows into its upper half, rounded to BF16 after the
// drain), so no separate conversion pass reads the features; they were
// asked into L2 two layers earlier.  A tile's score is the sum of four
// column quarters' partial dot products, met per TMEM lane quadrant by a
// 4-warp barrier, the only barrier inside the job loop.
//
// Arithmetic.  Rounding points are those of the tiled GEMM path: BF16
// inputs, weights and activations, FP32 accumulation, FP32 bias and GELU.
// The GELU's erf is the rational approximation 7.1.28 of Abramowitz &
// Stegun (absolute error <= 3e-7, far below the BF16 rounding of the
// activation), evaluated on pairs of activations with the packed FP32x2
// instructions (fma/mul/add.rn.f32x2: two IEEE operations per
// instruction); TMEM loads are double-buffered; biases and output weights
// are staged in shared memory.  The bias enters the FP32 sum first, then the
// K-slices of the layer in order.
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

constexpr int TM = 128;       // rows per tile (MMA M)
constexpr int WIDTH = 256;    // hidden width (MMA N)
constexpr int IN = 48;        // input features
constexpr int DEPTH = 4;      // hidden layers
constexpr int KC = 32;        // K per streamed weight slice
constexpr int NCH = WIDTH / KC;  // slices per hidden layer
constexpr int NSLOT = 4;         // weight slices resident at a time
constexpr int INFLIGHT = 2;      // tiles in flight, each with its own accumulator and buffer
constexpr int EWARPS = 16;       // epilogue warps: 4 TMEM lane quadrants x 4 column quarters
constexpr int ETHREADS = EWARPS * 32;
constexpr int MMA_WARP = EWARPS, LOAD_WARP = EWARPS + 1;
constexpr int THREADS = (EWARPS + 2) * 32;
constexpr int QCOLS = WIDTH / 4;  // columns per epilogue warp
constexpr uint64_t kWaitLimitNs = 1000000000ull;  // give up on a pipeline wait after 1 s
constexpr uint32_t kSuspendNs = 20000;  // a waiting thread sleeps until the phase completes, at most this long
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
constexpr uint32_t SM_A = 0;                                            // activations [128 x 256] per tile in flight
constexpr uint32_t kABytes = operand_bytes(TM, WIDTH);
constexpr uint32_t kXf32Off = 32768;  // FP32 input rows [128 x 48] staged here inside a tile's buffer
constexpr uint32_t SM_W0 = SM_A + INFLIGHT * kABytes;                   // W0 [256 x 48]
constexpr uint32_t SM_W = SM_W0 + operand_bytes(WIDTH, IN);             // weight slice ring
constexpr uint32_t SM_PART = SM_W + NSLOT * kSliceBytes;                // per tile in flight: 4 x 128 partial dots
constexpr uint32_t SM_BAR = SM_PART + INFLIGHT * 4 * TM * 4;
// mbarriers: W0 copy, slot full [4], slot free [4], accumulator ready [2],
// activations (or next input) written [2], drain
constexpr int NBAR = 1 + 2 * NSLOT + 2 * INFLIGHT + 1;
constexpr uint32_t SM_TMEM = SM_BAR + NBAR * 8;                         // TMEM base from tcgen05.alloc
constexpr uint32_t SM_TOTAL = SM_TMEM + 16;
static_assert(SM_TOTAL + (DEPTH + 1) * WIDTH * 4 + 64 <= 227 * 1024, "shared memory plan exceeds 227 KB");
static_assert(operand_bytes(WIDTH, IN) % 16 == 0 && kSliceBytes % 16 == 0, "bulk copies move whole 16-byte units");
static_assert(INFLIGHT * WIDTH <= 512, "one 256-column accumulator per tile in flight");
static_assert(operand_bytes(TM, IN) <= kXf32Off && kXf32Off + TM * IN * 4 <= kABytes,
              "FP32 input rows fit above the BF16 input inside a tile's buffer");

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
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(phase), "r"(kSuspendNs)
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

// mbar_wait that also gives up as soon as *fail is set by another thread,
// or after limit_ns
__device__ __forceinline__ bool mbar_wait_or(uint32_t bar, uint32_t phase, volatile int* fail,
                                             uint64_t limit_ns = kWaitLimitNs) {
  uint64_t t0 = 0;
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(phase), "r"(kSuspendNs)
        : "memory");
    if (done) return true;
    if (*fail) return false;
    const uint64_t t = global_ns();
    if (t0 == 0) t0 = t;
    else if (t - t0 > limit_ns) return false;
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

// store 32 consecutive FP32 columns of this thread's TMEM lane (complete
// after tmem_wait_st)
__device__ __forceinline__ void tmem_store32(uint32_t taddr, const uint32_t* r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]),
      "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]),
      "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// the bias of layer l for this warp's 32 columns c0 .. c0 + 31 into TMEM at
// taddr (every lane: the same values), as the start of the next accumulation
__device__ __forceinline__ void store_bias32(uint32_t taddr, const float* __restrict__ bias_l, int c0) {
  uint32_t r[32];
#pragma unroll
  for (int j = 0; j < 32; j += 4) {
    const float4 b4 = *reinterpret_cast<const float4*>(bias_l + c0 + j);
    r[j] = __float_as_uint(b4.x);
    r[j + 1] = __float_as_uint(b4.y);
    r[j + 2] = __float_as_uint(b4.z);
    r[j + 3] = __float_as_uint(b4.w);
  }
  tmem_store32(taddr, r);
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
  const f32x2 nr = pk2(rcp_approx(-q0), rcp_approx(-q1));  // -1/q: the sign rides on the reciprocal
  return ffma2(a, nr, fadd2(z, a));
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// Input rows of a tile: unit i (0 .. 767) is the 16-byte piece (row i % 128,
// features 8 (i / 128) ..) of the BF16 operand in its canonical K = 48 layout.
constexpr int kUnits = TM * (IN / 8);
constexpr int kUnitsPerThread = (kUnits + ETHREADS - 1) / ETHREADS;

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}

// start copying tile t's input rows into a tile buffer (rows past M read as
// zero): BF16 rows straight into the operand layout, FP32 rows (xf) raw
// into the buffer's upper half
__device__ __forceinline__ void input_copy(uint32_t buf, const MlpTcArgs& a, int t, int tid) {
#pragma unroll
  for (int u = 0; u < kUnitsPerThread; ++u) {
    const int i = tid + u * ETHREADS;
    if (i >= kUnits) break;
    const int r = i % TM, kb = i / TM, m = t * TM + r;
    const bool in = m < a.M;
    const size_t e = (size_t)(in ? m : 0) * IN + (size_t)kb * 8;
    if (a.xf) {
      const uint32_t d = buf + kXf32Off + (uint32_t)(r * IN + kb * 8) * 4u;
      cp_async16(d, a.xf + e, in ? 16u : 0u);
      cp_async16(d + 16u, a.xf + e + 4, in ? 16u : 0u);
    } else {
      cp_async16(buf + canon_off(r, kb * 8, IN), static_cast<const bf16*>(a.x) + e, in ? 16u : 0u);
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// ask L2 for tile t's input rows (they are contiguous: 128 rows of 48 values),
// one 128-byte line per thread, so that the later input_copy finds them there
__device__ __forceinline__ void input_prefetch(const MlpTcArgs& a, int t, int tid) {
  const size_t row0 = (size_t)t * TM, rows = (size_t)min(TM, a.M - t * TM);
  const char* base = a.xf ? reinterpret_cast<const char*>(a.xf + row0 * IN)
                          : reinterpret_cast<const char*>(static_cast<const bf16*>(a.x) + row0 * IN);
  const size_t bytes = rows * IN * (a.xf ? 4 : 2);
  if ((size_t)tid * 128 < bytes) asm volatile("prefetch.global.L2 [%0];" ::"l"(base + (size_t)tid * 128));
}

// once this thread's input_copy has landed (cp.async.wait_all): its FP32
// pieces are rounded to BF16 into the operand layout (the same units the
// same thread copied, so no other thread's copies are read)
__device__ __forceinline__ void input_finish(uint8_t* buf, const MlpTcArgs& a, int tid) {
  if (!a.xf) return;
#pragma unroll
  for (int u = 0; u < kUnitsPerThread; ++u) {
    const int i = tid + u * ETHREADS;
    if (i >= kUnits) break;
    const int r = i % TM, kb = i / TM;
    const float4* f = reinterpret_cast<const float4*>(buf + kXf32Off + (uint32_t)(r * IN + kb * 8) * 4u);
    const float4 lo = f[0], hi = f[1];
    *reinterpret_cast<uint4*>(buf + canon_off(r, kb * 8, IN)) =
        make_uint4(pack_bf16x2(lo.x, lo.y), pack_bf16x2(lo.z, lo.w), pack_bf16x2(hi.x, hi.y), pack_bf16x2(hi.z, hi.w));
  }
}

// the score of row r of tile t from the four column quarters' partial dots (pb[q * 128 + r])
__device__ __forceinline__ void write_score(const MlpTcArgs& a, const float* pb, int t, int r) {
  const int m = t * TM + r;
  if (m < a.M) a.y[m] = a.norm[0] + a.norm[1] * (((pb[r] + pb[TM + r]) + (pb[2 * TM + r] + pb[3 * TM + r])) + a.b_out[0]);
}

__global__ void __launch_bounds__(THREADS, 1) mlp_forward_tc_kernel(const MlpTcArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ volatile int s_fail;
  __shared__ __align__(16) float sbias[DEPTH * WIDTH];
  __shared__ __align__(16) float swout[WIDTH];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t sW0 = smem_u32(sm + SM_W0), sW = smem_u32(sm + SM_W);
  const uint32_t w0bar = smem_u32(sm + SM_BAR);
  const uint32_t fullb = w0bar + 8, freeb = fullb + 8 * NSLOT, accb = freeb + 8 * NSLOT, actb = accb + 8 * INFLIGHT;
  const uint32_t drainb = actb + 8 * INFLIGHT;
  const int ntiles = (a.M + TM - 1) / TM;
  // this CTA's tiles: k = 0 .. n - 1 is tile blockIdx.x + k gridDim.x, held in buffer k % INFLIGHT
  const int n = (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  float* part = reinterpret_cast<float*>(sm + SM_PART);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + SM_TMEM);
  const uint8_t* wpack = static_cast<const uint8_t*>(a.wpack);
  const bf16* w_out = static_cast<const bf16*>(a.w_out);

  if (tid == 0) {
    s_fail = 0;
    mbar_init(w0bar, 1);
    for (int j = 0; j < NSLOT; ++j) {
      mbar_init(fullb + 8 * j, 1);
      mbar_init(freeb + 8 * j, 1);
    }
    for (int b = 0; b < INFLIGHT; ++b) {
      mbar_init(accb + 8 * b, 1);
      mbar_init(actb + 8 * b, EWARPS);
    }
    mbar_init(drainb, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0) {  // one 256-column FP32 accumulator per tile in flight
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(INFLIGHT * WIDTH));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == LOAD_WARP) {
    // ---- weight stream: one lane copies W0, then every hidden layer's slices in MMA order ----
    if (lane == 0) {
      int fail = 0;
      bool w0_pending = false;
      uint32_t issued = 0;  // slices copied so far; slice i goes to slot i % NSLOT
      // (the failure-detection test leaves W0's barrier without its arrival)
      if (!a.expire_test) {
        bulk_load(sW0, wpack + w_offset(0), operand_bytes(WIDTH, IN), w0bar);
        w0_pending = true;
      }
      for (int p = 0; INFLIGHT * p < n && !fail; ++p)
        for (int l = 1; l < DEPTH && !fail; ++l)
          for (int b = 0; b < INFLIGHT && !fail; ++b) {
            if (INFLIGHT * p + b >= n) continue;
            for (int j = 0; j < NCH; ++j) {
              const uint32_t slot = issued % NSLOT, round = issued / NSLOT;
              // the MMA warp's waits are the ones that report (this one only ends the stream)
              if (!mbar_wait_or(freeb + 8 * slot, (round & 1u) ^ 1u, &s_fail, 2 * kWaitLimitNs)) {
                fail = 6;
                break;
              }
              copy_async(sW + slot * kSliceBytes, wpack + w_offset(l) + (uint32_t)j * kSliceBytes, kSliceBytes,
                         fullb + 8 * slot);
              ++issued;
            }
          }
      if (fail && !s_fail) s_fail = fail;
      if (s_fail) {  // every copy this lane issued lands before the CTA lets go of its shared memory (bounded)
        if (w0_pending) mbar_wait(w0bar, 0);
        for (uint32_t i = issued > (uint32_t)NSLOT ? issued - NSLOT : 0u; i < issued; ++i)
          mbar_wait(fullb + 8 * (i % NSLOT), (i / NSLOT) & 1u);
      }
    }
  } else if (warp == MMA_WARP) {
    // ---- MMA issue: one lane, the two tiles in flight alternating layer by layer ----
    if (lane == 0) {
      const uint32_t idesc = make_idesc(TM, WIDTH);
      int fail = 0;
      bool pend = false;
      uint32_t used = 0;                      // slices consumed, in the stream's order (a multiple of NCH)
      uint32_t jobs[INFLIGHT] = {0u, 0u};     // layers issued per buffer: the phase of its barriers
      // descriptors: a step of 8 K-elements (one core matrix, 128 B) adds 8 to the start-address field
      const uint64_t w0d = make_desc(sW0, 128u, (uint32_t)(IN >> 3) * 128u);
      const uint64_t wsd = make_desc(sW, 128u, (uint32_t)(KC >> 3) * 128u);
      static_assert(NCH % NSLOT == 0, "every hidden layer starts at slot 0");
      if (!mbar_wait_or(w0bar, 0, &s_fail)) fail = 1;
      for (int p = 0; INFLIGHT * p < n && !fail; ++p)
        for (int l = 0; l < DEPTH && !fail; ++l)
          for (int b = 0; b < INFLIGHT && !fail; ++b) {
            if (INFLIGHT * p + b >= n) continue;
            // this tile's input (l = 0) or previous layer's activations are written, its accumulator drained
            if (!mbar_wait_or(actb + 8 * b, jobs[b] & 1u, &s_fail)) {
              fail = 3;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sA = smem_u32(sm + SM_A + (uint32_t)b * kABytes);
            const uint32_t d = tmem + (uint32_t)(b * WIDTH);
            if (l == 0) {
              const uint64_t a0 = make_desc(sA, 128u, (uint32_t)(IN >> 3) * 128u);
#pragma unroll
              for (int k0 = 0; k0 < IN; k0 += 16)
                mma_bf16(d, a0 + (uint64_t)(k0 >> 3) * 8u, w0d + (uint64_t)(k0 >> 3) * 8u, idesc, 1u);
            } else {
              const uint64_t a0 = make_desc(sA, 128u, (uint32_t)(WIDTH >> 3) * 128u);
              const uint32_t ph = (used / NSLOT) & 1u;  // the parity of slots 0..3 for slices 0..3
#pragma unroll
              for (int j = 0; j < NCH; ++j) {
                const uint32_t slot = (uint32_t)(j % NSLOT);
                if (!mbar_wait_or(fullb + 8 * slot, ph ^ (uint32_t)((j / NSLOT) & 1), &s_fail)) {
                  fail = 4;
                  break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                for (int kk = 0; kk < KC; kk += 16)
                  mma_bf16(d, a0 + (uint64_t)((j * KC + kk) >> 3) * 8u,
                           wsd + (uint64_t)(slot * (kSliceBytes >> 4)) + (uint64_t)(kk >> 3) * 8u, idesc,
                           1u);
                mma_commit(freeb + 8 * slot);  // the slot refills once these MMAs are done
              }
              used += NCH;
            }
            pend = true;
            if (fail) break;
            mma_commit(accb + 8 * b);
            ++jobs[b];
          }
      if (fail && !s_fail) s_fail = fail;
      if (s_fail && pend) {  // drain (bounded): every MMA issued
        mma_commit(drainb);
        mbar_wait(drainb, 0);
      }
    }
  } else {
    // ---- epilogue: TMEM -> bias + GELU -> BF16 activations, job by job ----
    const int quad = warp & 3, qtr = warp >> 2;  // TMEM lane quadrant (= warp % 4), column quarter
    const int r_local = quad * 32 + lane;
    // the first tiles' inputs start to arrive while the biases are staged
    for (int b = 0; b < INFLIGHT && b < n; ++b)
      input_copy(smem_u32(sm + SM_A + (uint32_t)b * kABytes), a, (int)blockIdx.x + b * (int)gridDim.x, tid);
#pragma unroll
    for (int l = 0; l < DEPTH; ++l)
      for (int i = tid; i < WIDTH; i += ETHREADS) sbias[l * WIDTH + i] = a.bias[l][i];
    for (int i = tid; i < WIDTH; i += ETHREADS) swout[i] = 0.5f * __bfloat162float(w_out[i]);  // see gelu2
    asm volatile("bar.sync 1, %0;" ::"n"(ETHREADS));  // biases and output weights staged
    for (int b = 0; b < INFLIGHT && b < n; ++b)  // the first accumulations start from layer 0's bias
#pragma unroll
      for (int cc = 0; cc < QCOLS / 32; ++cc)
        store_bias32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * WIDTH) + (uint32_t)(qtr * QCOLS + 32 * cc),
                     sbias, qtr * QCOLS + 32 * cc);
    tmem_wait_st();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    asm volatile("cp.async.wait_all;" ::: "memory");
    for (int b = 0; b < INFLIGHT && b < n; ++b) {
      input_finish(sm + SM_A + (uint32_t)b * kABytes, a, tid);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) bar_arrive(actb + 8 * b);
      __syncwarp();
    }
    uint32_t jobs[INFLIGHT] = {0u, 0u};
    bool ok = true;  // this thread's waits all succeeded
    for (int p = 0; INFLIGHT * p < n; ++p)
      for (int l = 0; l < DEPTH; ++l)
        for (int b = 0; b < INFLIGHT; ++b) {
          const int k = INFLIGHT * p + b;
          if (k >= n) continue;
          const uint32_t A = SM_A + (uint32_t)b * kABytes;
          float* pb = part + b * 4 * TM;
          const bool last = l + 1 == DEPTH, next = last && k + INFLIGHT < n;
          // (a thread that saw a failure runs through the remaining jobs without waiting or working,
          // but still takes part in every quadrant barrier)
          bool work = ok && !s_fail;
          if (work && !mbar_wait_or(accb + 8 * b, jobs[b] & 1u, &s_fail, 2 * kWaitLimitNs)) {
            if (!s_fail) s_fail = 2;  // the MMA warp's waits are the ones that report a stalled pipeline first
            ok = work = false;
          }
          ++jobs[b];
          if (work) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (l == 1 && k + INFLIGHT < n) input_prefetch(a, (int)blockIdx.x + (k + INFLIGHT) * (int)gridDim.x, tid);
            // the last layer's MMAs no longer read the buffer: the next tile's input starts to arrive
            if (next) input_copy(smem_u32(sm + A), a, (int)blockIdx.x + (k + INFLIGHT) * (int)gridDim.x, tid);
            const float* bnext = sbias + (last ? 0 : l + 1) * WIDTH;  // layer 0 of the next tile after the last
            const uint32_t tbase =
                tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * WIDTH) + (uint32_t)(qtr * QCOLS);
            f32x2 dq01 = pk2(0.0f, 0.0f), dq23 = pk2(0.0f, 0.0f);
            uint32_t ra[32], rb[32];
            tmem_issue32(tbase, ra);
            tmem_wait32(ra);
#pragma unroll
            for (int cc = 0; cc < QCOLS / 32; ++cc) {
              uint32_t* cur = (cc & 1) ? rb : ra;
              uint32_t* nxt = (cc & 1) ? ra : rb;
              if (cc + 1 < QCOLS / 32) tmem_issue32(tbase + 32u * (uint32_t)(cc + 1), nxt);
              const int c0 = qtr * QCOLS + 32 * cc;
              float v[32];
#pragma unroll
              for (int j = 0; j < 32; j += 2) {
                const f32x2 g = gelu2(pk2(__uint_as_float(cur[j]), __uint_as_float(cur[j + 1])));
                upk2(g, v[j], v[j + 1]);
              }
              if (!last) {
#pragma unroll
                for (int kb = 0; kb < 4; ++kb) {
                  const uint4 q = make_uint4(pack_bf16x2(v[8 * kb], v[8 * kb + 1]),
                                             pack_bf16x2(v[8 * kb + 2], v[8 * kb + 3]),
                                             pack_bf16x2(v[8 * kb + 4], v[8 * kb + 5]),
                                             pack_bf16x2(v[8 * kb + 6], v[8 * kb + 7]));
                  *reinterpret_cast<uint4*>(sm + A + canon_off(r_local, c0 + 8 * kb, WIDTH)) = q;
                }
              } else {
#pragma unroll
                for (int j = 0; j < 32; j += 4) {
                  // the BF16 activation (as the next layer would see it) times the output weight
                  const float4 w4 = *reinterpret_cast<const float4*>(swout + c0 + j);
                  const uint32_t h01 = pack_bf16x2(v[j], v[j + 1]), h23 = pack_bf16x2(v[j + 2], v[j + 3]);
                  dq01 = ffma2(pk2(__uint_as_float(h01 << 16), __uint_as_float(h01 & 0xffff0000u)), pk2(w4.x, w4.y), dq01);
                  dq23 = ffma2(pk2(__uint_as_float(h23 << 16), __uint_as_float(h23 & 0xffff0000u)), pk2(w4.z, w4.w), dq23);
                }
              }
              // these columns now start the next accumulation of this buffer: its bias
              if (!last || next) store_bias32(tbase + 32u * (uint32_t)cc, bnext, c0);
              if (cc + 1 < QCOLS / 32) tmem_wait32(nxt);
            }
            // this layer's TMEM reads and bias stores precede the arrival that lets the next MMAs
            // accumulate
            if (!last || next) tmem_wait_st();
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            if (last) {
              float d0, d1, d2, d3;
              upk2(dq01, d0, d1);
              upk2(dq23, d2, d3);
              pb[qtr * TM + r_local] = (d0 + d1) + (d2 + d3);
              if (next) {  // this thread's pieces of the next input, rounded in place
                asm volatile("cp.async.wait_all;" ::: "memory");
                input_finish(sm + A, a, tid);
              }
            }
            if (!last || next) {
              asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
              __syncwarp();
              if (lane == 0) bar_arrive(actb + 8 * b);
              __syncwarp();
            }
          }
          if (last) {
            // the four column quarters of this lane quadrant (warps quad, quad + 4, ...) meet: the score
            asm volatile("bar.sync %0, %1;" ::"r"(2 + quad), "n"(4 * 32) : "memory");
            if (work && qtr == 0 && !s_fail) write_score(a, pb, (int)blockIdx.x + k * (int)gridDim.x, r_local);
          }
        }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (s_fail) {
    if (tid == 0) atomicExch(a.status, s_fail);
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x)
      if (tid < TM && t * TM + tid < a.M) a.y[t * TM + tid] = __int_as_float(0x7fc00000);
  }
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(INFLIGHT * WIDTH));
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
