// Definition of the solver handle, shared by the handle API (engine.cu) and the batch /
// server runtime (runtime.cu).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/gdm.h"
#include "gdm_internal.h"

namespace gdm {

enum FBuf { F_H, F_S, F_Z, F_ZT, F_X, F_X2, F_XN, F_T, F_U, F_V, F_COUNT };
enum SBuf { SL_S, SL_Z, SL_ZT, SL_A, SL_B, SL_X, SL_X2, SL_W, SL_COUNT };
// Layout of a handle's small[] device scratch (doubles)
enum SmallSlot {
  SM_BOUNDS_S = 0,   // 2
  SM_BOUNDS_H = 2,   // 2
  SM_COEF_A = 4,     // 3
  SM_COEF_B = 8,     // 3
  SM_COEF_X0 = 12,   // 3
  SM_RED = 16,       // 8 reduction outputs
  SM_KCOUNT = 24,    // 1: k stages issued by masked products (as an unsigned 64-bit count)
  SM_GERSH_H = 26,   // 2: Gershgorin bounds of H~
  SM_EST_H = 160,    // 5: estimated bounds of H~, whether used, the raw extreme Ritz values
  SM_EST_S = 168,    // 5: the same for S
  SM_LANCZOS = 32,   // 2 x kMaxLanczos: alpha_k, then beta_k, of the Lanczos recurrence on H~
};
  // lockstep batches: the problem's BatchCtl (batch.cu) from this double on
constexpr int SM_BATCH = 256;

constexpr int kSplitTiles = 160;  // split-k: most tiles split at once (>= the SM count)
constexpr int kSmall = 4096;  // doubles of small device scratch beyond the partials

// Device bytes gdm_init allocates for capacity n (one cudaMalloc).
size_t handle_pool_bytes(int64_t n);

// Solve a handle whose capacity is at least n for a problem of size n with n_occ occupied
// states: the buffers keep the capacity's leading dimension.  Drops S, H and Z.
gdm_status handle_reconfigure(gdm_handle* h, int64_t n, int64_t n_occ);

}  // namespace gdm

struct gdm_handle {
  int device = 0;
  int64_t n = 0, n_occ = 0;
  int64_t n_cap = 0;      // capacity the buffers were allocated for
  int64_t ld = 0;         // leading dimension of every internal n x n buffer
  int rows_alloc = 0;     // rows of slice buffers (multiple of 128)
  cudaStream_t own_stream = nullptr, stream = nullptr;
  gdm_precision prec = GDM_PREC_MIXED;
  int purify = 0;  // gdm_purification
  double trunc_tau = 0.0;          // threshold filtering of the purification (0: off)
  double kstages_dense = 0.0;      // k stages the masked products would issue without masks
  double kstages_issued = 0.0;     // ... and issued (read back after a solve)
  gdm::Precision phase[4] = {{2, 1, 12}, {4, 3, 9}, {4, 3, 9}, {3, 3, 12}};
  // Tr(X - X^2) <= 1e-11 N bounds the eigenvalues' part of ||P - P*||_F / ||P*||_F by
  // 1e-11 sqrt(N): negligible against the route's 1e-6, and the sliced products' idempotency
  // floor (~1e-8 at n = 4096) is then often reached without a step that only confirms it
  double idem_tol = 1e-11, trace_tol = 1e-6;
  bool trace_correct = true;
  double cleanup_tol = -1.0;  // S-metric clean-up above this |Tr(P S) - n_occ| (< 0: never)
  double rescale_tol = 1e-8;  // last-resort rescale above this |Tr(P S) - n_occ|
  int max_ns = 100, max_purif = 200, n_refine = 2;
  int bounds_method = 1;   // gdm_bounds: spectral bounds of H~ for the initial guess
  int lanczos_steps = 24;

  void* pool = nullptr;
  double* f[gdm::F_COUNT] = {};
  gdm::SliceBuf sl[gdm::SL_COUNT];
  double* partials = nullptr;  // 5 n + 64 doubles
  double* lanczos_ws = nullptr;  // 4 * n_cap doubles: the Lanczos recurrence's vectors
  double* small = nullptr;     // kSmall doubles: coefficients, bounds, reductions
  gdm::Trs4State* st_dev = nullptr;
  uint32_t* err_dev = nullptr;
  // split-k of the products' last wave: int64 partial-sum slots and the per-tile counters
  // (kSplitTiles x kEpilogueWarps words right after err_dev, cleared with it)
  long long* split_ws = nullptr;
  uint32_t* split_cnt = nullptr;
  int split_slots = 0;
  double* host_buf = nullptr;  // pinned: kSmall doubles
  gdm::Trs4State* st_host = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;

  bool have_H = false, have_S = false, z_valid = false;
  bool have_P = false;  // F_XN holds the density matrix of the current H and S
  double z_err = 0.0;
  struct HistRow {
    double idem, trace, gamma;
    int branch;
  };
  std::vector<HistRow> hist;  // purification history of the last solve
  // optional timing of the sliced / FP64 product launches (CUDA events on the stream)
  bool profiling = false;
  struct Prof {
    cudaEvent_t a, b;
    double flops;  // issued: tensor-pipe (slice pairs x computed tile area x 2K) or FP64 work
    double alg;    // algorithmic: n^3 for a symmetric product, 2 n^3 for a full one
    int kind;  // 0 sliced, 1 fp64
    int phase;  // gdm_phase of the product
  };
  // totals per kind: 0 sliced, 1 fp64, 2 + p sliced products of phase p
  static constexpr int kProfKinds = 6;
  std::vector<Prof> prof_pending;
  std::vector<cudaEvent_t> ev_pool;
  int64_t prof_launches[kProfKinds] = {};
  double prof_ms[kProfKinds] = {}, prof_flops[kProfKinds] = {}, prof_alg[kProfKinds] = {};
  std::string last_error;
};

