// gdm_op_product_noalloc: the sliced tensor-core product of gdm_op_product without any device
// allocation.  Its FP16 slices, row scales and error word live in one file-scope __device__
// array, so a caller that cannot (or must not) allocate device memory can still use it: for
// example code running while a framework's caching allocator owns nearly all of the GPU's
// memory, code inside a real-time loop that cannot afford an allocation's latency or its
// implicit synchronisation, or code that must not touch the allocator at all.  The caller still
// passes the inputs and the output.
#include <cstring>
#include <mutex>

#include "../../include/gdm.h"
#include "gdm_internal.h"

using namespace gdm;

namespace {

constexpr int kNoAllocMaxDim = 1024;  // m, n and k are each at most this
constexpr int kNoAllocMaxSlices = 4;
constexpr size_t kSliceBytes =
    sizeof(__half) * kNoAllocMaxSlices * static_cast<size_t>(kNoAllocMaxDim) * kNoAllocMaxDim;
constexpr size_t kScaleBytes = sizeof(double) * kNoAllocMaxDim;
constexpr size_t kOffA = 0;
constexpr size_t kOffB = kOffA + kSliceBytes;
constexpr size_t kOffScaleA = kOffB + kSliceBytes;
constexpr size_t kOffScaleB = kOffScaleA + kScaleBytes;
constexpr size_t kOffErr = kOffScaleB + kScaleBytes;
constexpr size_t kScratchBytes = kOffErr + 256;  // 16 MiB + 16 KiB + 256 B

// Held by every GPU that loads this library until the process exits.  Shared by all calls: the
// last call's contents stay behind, and calls that overlap on the GPU race on it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per device.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_scratch_addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

gdm_status to_status(cudaError_t e) {
  if (e == cudaSuccess) return GDM_OK;
  if (e == cudaErrorInvalidValue) return GDM_ERR_ARG;
  return GDM_ERR_CUDA;
}

}  // namespace

extern "C" gdm_status gdm_op_product_noalloc(const double* A, int64_t lda, const double* Bt,
                                             int64_t ldb, double* C, int64_t ldc, int64_t m,
                                             int64_t n, int64_t k, int nslice, int max_order,
                                             int slice_bits, int symmetric, void* stream) {
  if (m < 0 || n < 0 || k < 0) return GDM_ERR_ARG;
  if (m > kNoAllocMaxDim || n > kNoAllocMaxDim || k > kNoAllocMaxDim) return GDM_ERR_ARG;
  if (m == 0 || n == 0) return GDM_OK;
  if (A == nullptr || Bt == nullptr || C == nullptr || lda < k || ldb < k || ldc < n)
    return GDM_ERR_ARG;
  if (symmetric && m != n) return GDM_ERR_ARG;
  if (slice_bits == 0) slice_bits = 12;
  if (slice_bits < 9 || slice_bits > 12) return GDM_ERR_ARG;
  if (nslice != 0 && (nslice < 1 || nslice > kNoAllocMaxSlices || max_order < 0 ||
                      max_order > 3 || max_order > 2 * (nslice - 1)))
    return GDM_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (k == 0) {
    e = cudaMemset2DAsync(C, sizeof(double) * ldc, 0, sizeof(double) * n, m, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return to_status(e);
  }
  if (nslice == 0) {  // the FP64 kernel needs no scratch
    F64GemmArgs a;
    a.M = static_cast<int>(m);
    a.N = static_cast<int>(n);
    a.K = static_cast<int>(k);
    a.mode = symmetric ? kGemmSym : 0;
    a.A = A;
    a.lda = lda;
    a.Bt = Bt;
    a.ldb = ldb;
    a.C = C;
    a.ldc = ldc;
    e = f64_gemm(a, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return to_status(e);
  }

  void* base_v = nullptr;
  e = scratch_address(&base_v);
  if (e != cudaSuccess) return GDM_ERR_CUDA;
  unsigned char* base = static_cast<unsigned char*>(base_v);
  uint32_t* err = reinterpret_cast<uint32_t*>(base + kOffErr);
  e = cudaMemsetAsync(err, 0, sizeof(uint32_t), s);  // the previous call's word is still there
  if (e != cudaSuccess) return to_status(e);

  SliceBuf sa, sb;
  sa.data = reinterpret_cast<__half*>(base + kOffA);
  sa.row_scale = reinterpret_cast<double*>(base + kOffScaleA);
  sa.ld = static_cast<int>((k + 63) / 64 * 64);
  sa.rows_alloc = static_cast<int>((m + 127) / 128 * 128);
  sb.data = reinterpret_cast<__half*>(base + kOffB);
  sb.row_scale = reinterpret_cast<double*>(base + kOffScaleB);
  sb.ld = sa.ld;
  sb.rows_alloc = static_cast<int>((n + 127) / 128 * 128);
  // every row and column the product reads is rewritten below; the TMA boxes read nothing
  // beyond (rows, k), where they fill zeros, so no stale slice of an earlier call is used
  e = form_and_slice(A, lda, nullptr, 0, static_cast<int>(m), static_cast<int>(k), nullptr, 1.0,
                     0.0, 0.0, nullptr, 0, &sa, nslice, nullptr, s, slice_bits);
  if (e == cudaSuccess)
    e = form_and_slice(Bt, ldb, nullptr, 0, static_cast<int>(n), static_cast<int>(k), nullptr,
                       1.0, 0.0, 0.0, nullptr, 0, &sb, nslice, nullptr, s, slice_bits);
  if (e != cudaSuccess) return to_status(e);
  SlicedGemmArgs a;
  a.mode = symmetric ? kGemmSym : 0;
  a.C = C;
  a.ldc = ldc;
  a.err = err;
  Precision p;
  p.nslice = nslice;
  p.max_order = max_order;
  p.bits = slice_bits;
  e = sliced_gemm(sa, sb, p, a, s);
  if (e == cudaSuccess && symmetric)
    e = diag_fix(A, lda, Bt, ldb, C, ldc, static_cast<int>(m), static_cast<int>(k), 1.0, 0.0,
                 nullptr, 0, 0.0, nullptr, s);
  if (e != cudaSuccess) return to_status(e);
  uint32_t herr = 0;
  e = cudaMemcpyAsync(&herr, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return to_status(e);
  if (herr & DEV_ERR_WAIT_TIMEOUT) return GDM_ERR_TIMEOUT;
  return GDM_OK;
}
