// Launcher of the tcgen05 TF32 three-term GEMM (tc_gemm.cuh) used by the
// TT_TF32_SPLIT local solves: same contract as gemm_f32; when the tile grid is
// small, K is split across the CTAs of the same launch and a second kernel
// sums the partial tiles.
#include "common.cuh"
#include "tc_gemm.cuh"

#include <algorithm>
#include <mutex>

namespace tt {

namespace {

__global__ void tc_splitk_reduce(int M, int N, int splitk, int batch, const float *__restrict__ ws, float alpha,
                                 float beta, float *__restrict__ C, int ldc, long long sC) {
  const long long tot = (long long)batch * M * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e / ((long long)M * N));
    const long long r = e % ((long long)M * N);
    const int m = (int)(r / N), n = (int)(r % N);
    float s = 0.f;
    for (int q = 0; q < splitk; ++q) s += ws[((long long)b * splitk + q) * M * N + r];
    float *cp = C + b * sC + (long long)m * ldc + n;
    *cp = beta == 0.f ? alpha * s : alpha * s + beta * *cp;
  }
}

// grid: x over N tiles, y over M tiles, z over (batch, K-split) pairs
template <bool TA, bool TB, bool BF16>
void launch(Ctx *c, int M, int N, int K, int kchunk, int ksplit, float alpha, const float *A, int lda, long long sA,
            const float *B, int ldb, long long sB, float beta, float *C, int ldc, long long sC, int batch) {
  // the dynamic shared-memory opt-in is per device and kernel; set it once for each
  static std::mutex mu;
  static uint64_t done = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (c->device >= 64 || !(done >> c->device & 1)) {
      TT_CHECK_CUDA(cudaFuncSetAttribute(tc::tc_gemm_kernel<TA, TB, BF16>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES));
      if (c->device < 64) done |= 1ull << c->device;
    }
  }
  dim3 grid((N + tc::TN - 1) / tc::TN, (M + tc::TM - 1) / tc::TM, batch * ksplit);
  const uint32_t a_k = (tc::TM / 8) * 128, b_k = (tc::TN / 8) * 128;
  tc::tc_gemm_kernel<TA, TB, BF16><<<grid, tc::THREADS, tc::SMEM_BYTES, c->stream>>>(
      M, N, K, kchunk, ksplit, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, a_k, 128u, b_k, 128u,
      reinterpret_cast<int *>(c->d_scalar + 8));
  c->count();
  TT_CHECK_CUDA(cudaGetLastError());
}

}  // namespace

void gemm_f32_tc(Ctx *c, bool ta, bool tb, int M, int N, int K, float alpha, const float *A, int lda, long long sA,
                 const float *B, int ldb, long long sB, float beta, float *C, int ldc, long long sC, int batch,
                 bool bf16) {
  if (M <= 0 || N <= 0 || batch <= 0 || K <= 0) return;
  TT_REQUIRE(batch <= 65535 && (M + tc::TM - 1) / tc::TM <= 65535, "gemm_f32_tc: grid too large");
  // split K when the tile grid leaves SMs idle and each split keeps >= 2 chunks
  const long long tiles = (long long)((M + tc::TM - 1) / tc::TM) * ((N + tc::TN - 1) / tc::TN) * batch;
  const int tke = bf16 ? 2 * tc::TK : tc::TK;  // K elements per shared-memory stage
  int splitk = 1;
  if (tiles < c->sm_count && K > 4 * tke)
    splitk = (int)std::min<long long>((c->sm_count + tiles - 1) / tiles, (K + 2 * tke - 1) / (2 * tke));
  splitk = std::max(1, std::min({splitk, 32, 65535 / batch}));
  int kchunk = K;
  if (splitk > 1) {
    kchunk = (K + splitk - 1) / splitk;
    kchunk = (kchunk + tke - 1) / tke * tke;
    splitk = (K + kchunk - 1) / kchunk;
  }
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (c->profiling) {
    c->prof_begin(&ev0, &ev1, 2);
    TT_CHECK_CUDA(cudaEventRecord(ev0, c->stream));
  }
  auto go = [&](float *Cp, float al, float be, int ldcp, long long sCp) {
#define TT_TC_GO(TA_, TB_)                                                                                  \
  (bf16 ? launch<TA_, TB_, true>(c, M, N, K, kchunk, splitk, al, A, lda, sA, B, ldb, sB, be, Cp, ldcp, sCp, batch) \
        : launch<TA_, TB_, false>(c, M, N, K, kchunk, splitk, al, A, lda, sA, B, ldb, sB, be, Cp, ldcp, sCp, batch))
    if (ta && tb) TT_TC_GO(true, true);
    else if (ta) TT_TC_GO(true, false);
    else if (tb) TT_TC_GO(false, true);
    else TT_TC_GO(false, false);
#undef TT_TC_GO
  };
  if (splitk == 1) {
    go(C, alpha, beta, ldc, sC);
  } else {
    // partial products land in a workspace laid out [batch][split][M][N], reduced below
    c->ws_tc.ensure(c, ((size_t)batch * splitk * M * N + 1) / 2);
    float *ws = reinterpret_cast<float *>(c->ws_tc.p());
    go(ws, 1.f, 0.f, N, (long long)M * N);
    const long long tot = (long long)batch * M * N;
    const unsigned blocks = (unsigned)std::min<long long>((tot + 255) / 256, 4LL * c->sm_count * 8);
    tc_splitk_reduce<<<blocks, 256, 0, c->stream>>>(M, N, splitk, batch, ws, alpha, beta, C, ldc, sC);
    c->count();
    TT_CHECK_CUDA(cudaGetLastError());
  }
  if (c->profiling) {
    TT_CHECK_CUDA(cudaEventRecord(ev1, c->stream));
    c->gemmtc_flops += 2.0 * M * (double)N * K * batch;
    c->gemmtc_launches += 1;
  }
}

int tc_error_flag(Ctx *c) {
  int v = 0;
  TT_CHECK_CUDA(cudaMemcpyAsync(&v, c->d_scalar + 8, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  c->sync();
  return v;
}

}  // namespace tt
