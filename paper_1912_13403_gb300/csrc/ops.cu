// Stateless operations of the C ABI (gdm_op_*): one product, Gershgorin bounds, one TRS4 step.
// They run the same kernels as the solver on caller-owned device buffers; scratch comes from
// the stream-ordered allocator and is released before the call returns.
#include <cmath>
#include <cstddef>
#include <cstring>

#include "../../include/gdm.h"
#include "gdm_internal.h"

using namespace gdm;

namespace {

constexpr int kSplitSlotsOps = 160;  // split-k slots and counted tiles (>= the SM count)

struct Scratch {
  cudaStream_t s;
  void* ptrs[32] = {};
  int n = 0;
  explicit Scratch(cudaStream_t st) : s(st) {}
  template <class T>
  T* get(size_t bytes) {
    void* p = nullptr;
    if (n >= 32 || cudaMallocAsync(&p, bytes, s) != cudaSuccess) return nullptr;
    ptrs[n++] = p;
    return static_cast<T*>(p);
  }
  ~Scratch() {
    for (int i = 0; i < n; ++i) cudaFreeAsync(ptrs[i], s);
    cudaStreamSynchronize(s);
  }
};

bool alloc_slices(Scratch& sc, SliceBuf& b, int rows, int cols) {
  b.rows = rows;
  b.cols = cols;
  b.ld = (cols + 63) / 64 * 64;
  b.rows_alloc = (rows + 127) / 128 * 128;
  b.data = sc.get<__half>(sizeof(__half) * 4 * static_cast<size_t>(b.ld) * b.rows_alloc);
  b.row_scale = sc.get<double>(sizeof(double) * b.rows_alloc);
  return b.data != nullptr && b.row_scale != nullptr;
}

gdm_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return GDM_OK;
  if (e == cudaErrorMemoryAllocation) return GDM_ERR_OOM;
  if (e == cudaErrorInvalidValue) return GDM_ERR_ARG;
  return GDM_ERR_CUDA;
}

#define OPCK(expr)                              \
  do {                                          \
    cudaError_t e_ = (expr);                    \
    if (e_ != cudaSuccess) return cuda_status(e_); \
  } while (0)

// C = A * Bt^T (+ beta D + diag I) through either kernel; slices made on the fly.
cudaError_t run_product(Scratch& sc, const double* A, int64_t lda, const double* Bt, int64_t ldb,
                        double* C, int64_t ldc, int m, int n, int k, int nslice, int max_order,
                        bool sym, const double* D, int64_t ldd, double alpha, double beta,
                        const double* coef, uint32_t* err, int bits = 12) {
  if (nslice == 0) {
    F64GemmArgs a;
    a.M = m;
    a.N = n;
    a.K = k;
    a.mode = sym ? kGemmSym : 0;
    a.A = A;
    a.lda = lda;
    a.Bt = Bt;
    a.ldb = ldb;
    a.C = C;
    a.ldc = ldc;
    a.D = D;
    a.ldd = ldd;
    a.alpha = alpha;
    a.beta = beta;
    a.coef = coef;
    return f64_gemm(a, sc.s);
  }
  SliceBuf sa, sb;
  if (!alloc_slices(sc, sa, m, k) || !alloc_slices(sc, sb, n, k)) return cudaErrorMemoryAllocation;
  cudaError_t e = form_and_slice(A, lda, nullptr, 0, m, k, nullptr, 1, 0, 0, nullptr, 0, &sa,
                                 nslice, nullptr, sc.s, bits);
  if (e != cudaSuccess) return e;
  e = form_and_slice(Bt, ldb, nullptr, 0, n, k, nullptr, 1, 0, 0, nullptr, 0, &sb, nslice,
                     nullptr, sc.s, bits);
  if (e != cudaSuccess) return e;
  SlicedGemmArgs a;
  a.mode = sym ? kGemmSym : 0;
  a.C = C;
  a.ldc = ldc;
  a.D = D;
  a.ldd = ldd;
  a.alpha = alpha;
  a.beta = beta;
  a.coef = coef;
  a.err = err;
  Precision p;
  p.nslice = nslice;
  p.max_order = max_order;
  p.bits = bits;
  // split-k workspace for the last wave of tiles (counters start at zero)
  {
    const size_t tiles = static_cast<size_t>((m + 127) / 128) * ((n + 127) / 128);
    const int slots = static_cast<int>(tiles * 4 < kSplitSlotsOps ? tiles * 4 : kSplitSlotsOps);
    long long* ws = sc.get<long long>(sizeof(long long) * 128 * 128 * slots);
    uint32_t* cnt = sc.get<uint32_t>(sizeof(uint32_t) * kSplitSlotsOps * kEpilogueWarps);
    if (ws != nullptr && cnt != nullptr &&
        cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * kSplitSlotsOps * kEpilogueWarps, sc.s) ==
            cudaSuccess) {
      a.splitk_ws = ws;
      a.splitk_cnt = cnt;
      a.splitk_slots = slots;
      a.splitk_tiles = kSplitSlotsOps;
    }
  }
  e = sliced_gemm(sa, sb, p, a, sc.s);
  if (e != cudaSuccess || !sym) return e;
  return diag_fix(A, lda, Bt, ldb, C, ldc, m, k, alpha, beta, D, ldd, 0.0, coef, sc.s);
}

bool valid_format(int nslice, int max_order) {
  if (nslice == 0) return true;
  return nslice >= 1 && nslice <= 4 && max_order >= 0 && max_order <= 3 &&
         max_order <= 2 * (nslice - 1);
}

}  // namespace

extern "C" {

gdm_status gdm_op_product(const double* A, int64_t lda, const double* Bt, int64_t ldb, double* C,
                          int64_t ldc, int64_t m, int64_t n, int64_t k, int nslice, int max_order,
                          int slice_bits, int symmetric, void* stream) {
  if (slice_bits == 0) slice_bits = 12;
  if (slice_bits < 9 || slice_bits > 12) return GDM_ERR_ARG;
  if (m < 0 || n < 0 || k < 0 || m > (1 << 20) || n > (1 << 20) || k > (1 << 20))
    return GDM_ERR_ARG;
  if (m == 0 || n == 0) return GDM_OK;
  if (A == nullptr || Bt == nullptr || C == nullptr) return GDM_ERR_ARG;
  if (lda < k || ldb < k || ldc < n || !valid_format(nslice, max_order)) return GDM_ERR_ARG;
  if (symmetric && m != n) return GDM_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (k == 0) {
    OPCK(cudaMemset2DAsync(C, sizeof(double) * ldc, 0, sizeof(double) * n, m, s));
    OPCK(cudaStreamSynchronize(s));
    return GDM_OK;
  }
  gdm_status st = GDM_OK;
  {
    Scratch sc(s);
    uint32_t* err = sc.get<uint32_t>(sizeof(uint32_t));
    if (err == nullptr) return GDM_ERR_OOM;
    OPCK(cudaMemsetAsync(err, 0, sizeof(uint32_t), s));
    cudaError_t e = run_product(sc, A, lda, Bt, ldb, C, ldc, static_cast<int>(m),
                                static_cast<int>(n), static_cast<int>(k), nslice, max_order,
                                symmetric != 0, nullptr, 0, 1.0, 0.0, nullptr, err, slice_bits);
    if (e != cudaSuccess) return cuda_status(e);
    uint32_t herr = 0;
    OPCK(cudaMemcpyAsync(&herr, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    OPCK(cudaStreamSynchronize(s));
    if (herr & DEV_ERR_WAIT_TIMEOUT) st = GDM_ERR_TIMEOUT;
  }
  return st;
}

gdm_status gdm_op_gershgorin(const double* A, int64_t lda, int64_t n, double* bounds_host,
                             void* stream) {
  if (A == nullptr || bounds_host == nullptr || n < 1 || lda < n || n > (1 << 20))
    return GDM_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Scratch sc(s);
  double* part = sc.get<double>(sizeof(double) * (2 * ((n + 7) / 8) + 2));
  double* out = sc.get<double>(sizeof(double) * 2);
  if (part == nullptr || out == nullptr) return GDM_ERR_OOM;
  OPCK(gershgorin(A, lda, static_cast<int>(n), part, out, s));
  OPCK(cudaMemcpyAsync(bounds_host, out, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
  OPCK(cudaStreamSynchronize(s));
  return GDM_OK;
}

gdm_status gdm_op_trs4_step(double* X, int64_t ld, int64_t n64, double n_occ, int nslice,
                            int max_order, double* gamma_host, int* branch_host, void* stream) {
  if (X == nullptr || n64 < 1 || ld < n64 || n64 > (1 << 20) || !valid_format(nslice, max_order))
    return GDM_ERR_ARG;
  const int n = static_cast<int>(n64);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Scratch sc(s);
  const size_t mat = sizeof(double) * static_cast<size_t>(ld) * n;
  double* X2 = sc.get<double>(mat);
  double* W = sc.get<double>(mat);
  double* part = sc.get<double>(sizeof(double) * kTraceTerms * ((n + 7) / 8 + 1));
  Trs4State* st = sc.get<Trs4State>(sizeof(Trs4State));
  uint32_t* err = sc.get<uint32_t>(sizeof(uint32_t));
  if (!X2 || !W || !part || !st || !err) return GDM_ERR_OOM;
  OPCK(cudaMemsetAsync(err, 0, sizeof(uint32_t), s));
  Trs4State init;
  memset(&init, 0, sizeof(init));
  init.n_occ = n_occ;
  init.idem = INFINITY;
  OPCK(cudaMemcpyAsync(st, &init, sizeof(init), cudaMemcpyHostToDevice, s));
  OPCK(run_product(sc, X, ld, X, ld, X2, ld, n, n, n, nslice, max_order, true, nullptr, 0, 1.0,
                   0.0, nullptr, err));
  int nb = 0;
  OPCK(trs4_traces(X, X2, ld, n, part, &nb, s));
  OPCK(trs4_control(part, nb, st, -1.0, s));  // tol < 0: never "converged", always step
  Trs4State host;
  OPCK(cudaMemcpyAsync(&host, st, sizeof(host), cudaMemcpyDeviceToHost, s));
  OPCK(cudaStreamSynchronize(s));
  if (!std::isfinite(host.gamma)) return GDM_ERR_NONFINITE;
  const char* base = reinterpret_cast<const char*>(st);
  if (host.branch == 2 || host.branch == 3) {
    // W = g I + (4 - 2g) X + (g - 3) X^2 ; X <- X^2 W   (McWeeny: W = 3I - 2X)
    OPCK(form_and_slice(X, ld, X2, ld, n, n,
                        reinterpret_cast<const double*>(base + offsetof(Trs4State, coefW)), 0, 0,
                        0, W, ld, nullptr, 0, nullptr, s));
    OPCK(run_product(sc, X2, ld, W, ld, X, ld, n, n, n, nslice, max_order, true, nullptr, 0, 1.0,
                     0.0, nullptr, err));
  } else {
    OPCK(form_and_slice(X, ld, X2, ld, n, n,
                        reinterpret_cast<const double*>(base + offsetof(Trs4State, coefX)), 0, 0,
                        0, X, ld, nullptr, 0, nullptr, s));
  }
  OPCK(cudaStreamSynchronize(s));
  if (gamma_host) *gamma_host = host.gamma;
  if (branch_host) *branch_host = host.branch;
  return GDM_OK;
}

}  // extern "C"
