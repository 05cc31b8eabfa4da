// FP32 GEMM on the 5th-generation tensor cores (tcgen05) with a three-term
// split: each FP32 operand x = hi + lo, A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi,
// accumulated in FP32 in tensor memory.  Two operand formats: kind::tf32 (hi
// the TF32 truncation of x, lo = x - hi exactly representable: about 21
// significant bits) and kind::f16 with BF16 operands (hi = bf16(x), lo =
// bf16(x - hi): about 16 significant bits).  A and B always share the format.
// One CTA of 128 threads owns a 128 x 64 output tile of one (batch, K-split)
// pair; K advances in chunks of 32 through two shared-memory stages in the
// canonical K-major no-swizzle layout (8-row x 16-byte core matrices), so the
// loads of one chunk overlap the MMAs of the previous one.  One thread issues
// the MMAs and commits them to the stage's mbarrier; every wait is bounded and
// reports through an error flag instead of hanging.
#pragma once
#include <cstdint>

namespace tt {
namespace tc {

constexpr int TM = 128;  // tile rows (MMA M)
constexpr int TN = 64;   // tile columns (MMA N)
constexpr int TK = 32;   // FP32 K per shared-memory stage (4 MMAs of K = 8); BF16 stages hold 2 x TK
constexpr int ROW_BYTES = 128;  // bytes of K per operand row and stage (both formats)
constexpr int THREADS = 128;
// byte sizes of one operand buffer
constexpr int A_BYTES = TM * TK * 4;  // 16 KB
constexpr int B_BYTES = TN * TK * 4;  // 8 KB
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;  // hi and lo of A and B: 48 KB
constexpr int STAGES = 2;
// 8 KB beyond the stages keeps any descriptor walk inside the allocation
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 8 * 1024 + 1024;
constexpr uint32_t TMEM_COLS = 64;
constexpr int EPI_LD = TN + 1;  // padded row of the epilogue staging tile (floats)
static_assert(TM * EPI_LD * 4 <= STAGE_BYTES, "epilogue tile must fit in one stage");

// Canonical K-major layout without swizzle: element (row r, k) of a tile
// with R rows sits in core matrix (r / 8, k / 4) at ((k/4) * (R/8) + r/8) * 128
// bytes, row r % 8 at +16 bytes each, element k % 4 at +4 bytes each.
__host__ __device__ constexpr uint32_t kmajor_offset(int r, int k, int rows) {
  return (uint32_t)((((k >> 2) * (rows >> 3) + (r >> 3)) << 7) + ((r & 7) << 4) + ((k & 3) << 2));
}

// shared-memory matrix descriptor: start, leading-dimension byte offset (between
// core matrices adjacent along K), stride byte offset (adjacent along M/N),
// descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// instruction descriptor of kind::tf32: D F32, A and B TF32, both K-major
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
// instruction descriptor of kind::f16 with BF16 A and B (the same type for
// both operands), D F32, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

constexpr long long WAIT_LIMIT = 1LL << 20;

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
  for (long long it = 0; it < WAIT_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
      :
      : "r"(tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
      :
      : "r"(tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ float tf32_hi(float v) { return __uint_as_float(__float_as_uint(v) & 0xFFFFE000u); }

// BF16 bits of x rounded to nearest even (finite inputs), and back to FP32
__device__ __forceinline__ uint32_t bf16_bits(float x) {
  const uint32_t u = __float_as_uint(x);
  return (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;
}
__device__ __forceinline__ float bf16_val(uint32_t b) { return __uint_as_float(b << 16); }

// Stage an R-row operand tile (rows row0.., K columns k0.. : TK columns in
// FP32, 2 TK in BF16, 128 bytes per row either way) as hi and lo parts.
// Element (r, k) is p[r * ld + k] when KCONTIG, else p[k * ld + r]; rows >=
// nrows and columns >= kend read as zero.  Each thread moves units of one
// 16-byte core-matrix row (four FP32 or eight BF16 consecutive k of one row);
// the unit order puts 8 lanes on one whole core matrix, so the 16-byte shared
// stores do not conflict, and the global reads run along the contiguous index.
template <bool KCONTIG, int R, bool BF16>
__device__ __forceinline__ void stage_operand(const float *__restrict__ p, int ld, int row0, int nrows, int k0,
                                              int kend, uint8_t *hi, uint8_t *lo, int tid) {
  constexpr int EPU = BF16 ? 8 : 4;  // elements per 16-byte unit
#pragma unroll 2
  for (int u = tid; u < R * 8; u += THREADS) {
    int r, kg;
    if (KCONTIG) {
      r = ((u >> 6) << 3) | (u & 7);
      kg = (u >> 3) & 7;
    } else {
      r = u % R;
      kg = u / R;
    }
    const int gr = row0 + r;
    float v[EPU];
#pragma unroll
    for (int i = 0; i < EPU; ++i) {
      const int gk = k0 + EPU * kg + i;
      v[i] = (gr < nrows && gk < kend) ? (KCONTIG ? p[(long long)gr * ld + gk] : p[(long long)gk * ld + gr]) : 0.f;
    }
    const uint32_t off = (uint32_t)(((kg * (R >> 3) + (r >> 3)) << 7) + ((r & 7) << 4));
    if (BF16) {
      uint32_t h[4], l[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const uint32_t h0 = bf16_bits(v[2 * i]), h1 = bf16_bits(v[2 * i + 1]);
        const uint32_t l0 = bf16_bits(v[2 * i] - bf16_val(h0)), l1 = bf16_bits(v[2 * i + 1] - bf16_val(h1));
        h[i] = h0 | (h1 << 16);  // lower k in the lower half-word
        l[i] = l0 | (l1 << 16);
      }
      *reinterpret_cast<uint4 *>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<uint4 *>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
    } else {
      float4 h, l;
      h.x = tf32_hi(v[0]);
      h.y = tf32_hi(v[1]);
      h.z = tf32_hi(v[2]);
      h.w = tf32_hi(v[3]);
      l.x = v[0] - h.x;
      l.y = v[1] - h.y;
      l.z = v[2] - h.z;
      l.w = v[3] - h.w;
      *reinterpret_cast<float4 *>(hi + off) = h;
      *reinterpret_cast<float4 *>(lo + off) = l;
    }
  }
}

// C[z] = alpha op(A[b]) op(B[b]) + beta C[z] over the K range of split q,
// z = blockIdx.z = b * ksplit + q (row-major FP32; op(A) is M x K, op(B) K x N).
// Split q covers K indices [q * kchunk, min(K, (q + 1) * kchunk)).
// lbo / sbo: byte offsets of the operand descriptors (K-adjacent / row-adjacent core matrices).
template <bool TA, bool TB, bool BF16>
__global__ void __launch_bounds__(THREADS) tc_gemm_kernel(int M, int N, int K, int kchunk, int ksplit, float alpha,
                                                          const float *__restrict__ A, int lda, long long sA,
                                                          const float *__restrict__ B, int ldb, long long sB,
                                                          float beta, float *__restrict__ C, int ldc, long long sC,
                                                          uint32_t a_lbo, uint32_t a_sbo, uint32_t b_lbo,
                                                          uint32_t b_sbo, int *__restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t mbar[STAGES];
  __shared__ uint32_t tmem_base_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN, z = blockIdx.z;
  const int bz = z / ksplit, q = z - bz * ksplit;
  A += bz * sA;
  B += bz * sB;
  C += z * sC;
  const int kbeg = q * kchunk, kend = min(K, kbeg + kchunk);
  constexpr int TKE = BF16 ? 2 * TK : TK;  // K elements per stage
  const int nch = kend > kbeg ? (kend - kbeg + TKE - 1) / TKE : 0;
  const uint32_t s_base = (uint32_t)__cvta_generic_to_shared(smem);
  uint32_t mb[STAGES];
#pragma unroll
  for (int s = 0; s < STAGES; ++s) mb[s] = (uint32_t)__cvta_generic_to_shared(&mbar[s]);
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < STAGES; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb[s]) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(&tmem_base_sh)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_sh;
  const uint32_t idesc = BF16 ? idesc_bf16(TM, TN) : idesc_tf32(TM, TN);
  // per stage: commits issued and commit waits completed (uniform over the CTA);
  // a stage has at most one commit outstanding, whose phase parity is waits & 1
  int commits[STAGES] = {0, 0}, waits[STAGES] = {0, 0};
  int ok = 1;
  for (int ch = 0; ch < nch; ++ch) {
    const int s = ch & 1;
    if (commits[s] > waits[s]) {
      // the MMAs of chunk ch - 2 read this stage: wait for them before overwriting it
      const int mine = mbar_wait(mb[s], (uint32_t)(waits[s] & 1)) ? 1 : 0;
      ok = __syncthreads_and(mine);
      if (!ok) break;
      ++waits[s];
    }
    uint8_t *st = smem + s * STAGE_BYTES;
    uint8_t *a_hi = st, *a_lo = st + A_BYTES, *b_hi = st + 2 * A_BYTES, *b_lo = st + 2 * A_BYTES + B_BYTES;
    const int k0 = kbeg + ch * TKE;
    stage_operand<!TA, TM, BF16>(A, lda, m0, M, k0, kend, a_hi, a_lo, tid);
    stage_operand<TB, TN, BF16>(B, ldb, n0, N, k0, kend, b_hi, b_lo, tid);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = s_base + s * STAGE_BYTES, sb = sa + 2 * A_BYTES;
#pragma unroll
      for (int j = 0; j < ROW_BYTES / 32; ++j) {
        // 32 bytes of K per MMA (8 TF32 or 16 BF16): core-matrix columns 2j and 2j + 1
        const uint32_t ao = (uint32_t)(2 * j * (TM / 8)) * 128u, bo = (uint32_t)(2 * j * (TN / 8)) * 128u;
        const uint64_t dah = smem_desc(sa + ao, a_lbo, a_sbo), dal = smem_desc(sa + A_BYTES + ao, a_lbo, a_sbo);
        const uint64_t dbh = smem_desc(sb + bo, b_lbo, b_sbo), dbl = smem_desc(sb + B_BYTES + bo, b_lbo, b_sbo);
        if (BF16) {
          mma_bf16(tmem, dah, dbh, idesc, (ch > 0 || j > 0) ? 1u : 0u);
          mma_bf16(tmem, dah, dbl, idesc, 1u);
          mma_bf16(tmem, dal, dbh, idesc, 1u);
        } else {
          mma_tf32(tmem, dah, dbh, idesc, (ch > 0 || j > 0) ? 1u : 0u);
          mma_tf32(tmem, dah, dbl, idesc, 1u);
          mma_tf32(tmem, dal, dbh, idesc, 1u);
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb[s])
                   : "memory");
    }
    ++commits[s];
  }
  // drain the outstanding commit of each stage (bounded, also after a failed wait)
  int drained = 1;
#pragma unroll
  for (int s = 0; s < STAGES; ++s)
    if (commits[s] > waits[s]) drained &= mbar_wait(mb[s], (uint32_t)(waits[s] & 1)) ? 1 : 0;
  ok = __syncthreads_and(ok & drained);
  if (!ok && tid == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    // accumulator rows -> padded shared tile -> coalesced global rows
    float *stile = reinterpret_cast<float *>(smem);
    const int row = warp * 32 + lane;
    for (int c0 = 0; c0 < TN; c0 += 16) {
      uint32_t r[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
          "%14, %15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 16; ++j) stile[row * EPI_LD + c0 + j] = nch > 0 ? __uint_as_float(r[j]) : 0.f;
    }
    __syncthreads();
    for (int e = tid; e < TM * TN; e += THREADS) {
      const int rr = e / TN, cc = e % TN, gm = m0 + rr, gn = n0 + cc;
      if (gm < M && gn < N) {
        float *cp = C + (long long)gm * ldc + gn;
        const float v = stile[rr * EPI_LD + cc];
        *cp = beta == 0.f ? alpha * v : alpha * v + beta * *cp;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

}  // namespace tc
}  // namespace tt
