// Plain FP64 product C = alpha * A * Bt^T + beta * D on CUDA cores (DFMA), the all-FP64 path
// of the density-matrix route.  Same conventions as the sliced kernel: both operands are
// row-major with the contraction index contiguous (B is given as B^T), symmetric mode computes
// tiles on/above the diagonal and mirrors them, Ct receives C^T, D is read as D^T (pass a
// symmetric D).
//
// 64 x 64 output tile per block, 256 threads, 4 x 4 outputs per thread, K staged in
// shared memory 16 at a time.
#include "common.cuh"
#include "gdm_internal.h"

namespace gdm {

namespace {

constexpr int TB = 64;
constexpr int TK = 16;

__global__ void __launch_bounds__(256)
    f64_gemm_kernel(const F64GemmArgs a, int tiles_n) {
  __shared__ double As[TK][TB + 1];
  __shared__ double Bs[TK][TB + 1];
  if (a.skip != nullptr && *a.skip != 0) return;
  int ti, tj;
  const bool sym = (a.mode & kGemmSym) != 0;
  if (sym) {
    int idx = blockIdx.x, i = 0, len = tiles_n;
    while (idx >= len) {
      idx -= len;
      ++i;
      --len;
    }
    ti = i;
    tj = i + idx;
  } else {
    ti = blockIdx.x / tiles_n;
    tj = blockIdx.x % tiles_n;
  }
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  const int row0 = ti * TB, col0 = tj * TB;
  for (int k0 = 0; k0 < a.K; k0 += TK) {
    // load 64 x 16 panels of A and Bt (coalesced along k), store k-major
    for (int e = threadIdx.x; e < TB * TK; e += 256) {
      const int r = e / TK, k = e % TK;
      const int gr = row0 + r, gc = col0 + r, gk = k0 + k;
      As[k][r] = (gr < a.M && gk < a.K) ? a.A[static_cast<int64_t>(gr) * a.lda + gk] : 0.0;
      Bs[k][r] = (gc < a.N && gk < a.K) ? a.Bt[static_cast<int64_t>(gc) * a.ldb + gk] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < TK; ++k) {
      double av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[k][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[k][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
  double alpha = a.alpha, beta = a.beta;
  if (a.coef != nullptr) {
    alpha = a.coef[0];
    beta = a.coef[1];
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gr = row0 + ty * 4 + i;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gc = col0 + tx * 4 + j;
      if (gr >= a.M || gc >= a.N) continue;
      double v = alpha * acc[i][j];
      if (a.D != nullptr) v += beta * a.D[static_cast<int64_t>(gc) * a.ldd + gr];
      if (gr == gc) v += a.diag;
      if (!sym || gr <= gc) a.C[static_cast<int64_t>(gr) * a.ldc + gc] = v;
      if (sym && gr < gc) a.C[static_cast<int64_t>(gc) * a.ldc + gr] = v;
      if (a.Ct != nullptr) a.Ct[static_cast<int64_t>(gc) * a.ldct + gr] = v;
    }
  }
}

}  // namespace

cudaError_t f64_gemm(const F64GemmArgs& a, cudaStream_t stream) {
  if ((a.mode & kGemmSym) && a.M != a.N) return cudaErrorInvalidValue;
  const int tm = (a.M + TB - 1) / TB, tn = (a.N + TB - 1) / TB;
  const int grid = (a.mode & kGemmSym) ? tn * (tn + 1) / 2 : tm * tn;
  if (grid == 0) return cudaSuccess;
  count_launch();
  f64_gemm_kernel<<<grid, 256, 0, stream>>>(a, tn);
  return cudaGetLastError();
}

}  // namespace gdm
