// Internal declarations shared by the .cu files of the density-matrix engine.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gdm {

constexpr int kMaxPairs = 16;
constexpr int kMaxLanczos = 64;  // Lanczos steps at most (the tridiagonal's storage)
constexpr int kEpilogueWarps = 8;   // split-k counters per tile (one per epilogue warp)

// Error word written by kernels (never a trap): bit flags, OR-ed atomically.
enum DeviceError : uint32_t {
  DEV_ERR_WAIT_TIMEOUT = 1u << 0,   // an mbarrier wait ran out of its time limit
  DEV_ERR_BAD_ARG = 1u << 1,        // a kernel saw an argument it cannot handle
  DEV_ERR_NONFINITE = 1u << 2,      // a NaN / Inf reached a reduction
};
constexpr int kGemmSym = 1;  // compute tiles on/above the diagonal, mirror the rest

// A matrix held as FP16 integer slices plus power-of-two row scales (see gemm_sliced.cu):
// row i = row_scale[i] * 2^-11 * sum_s slice_s[i, :] * 2^(-bits * s).
struct SliceBuf {
  __half* data = nullptr;        // [4][rows_alloc][ld]
  double* row_scale = nullptr;   // [rows_alloc]
  int rows = 0, cols = 0;        // logical shape
  int ld = 0;                    // elements per row in memory (multiple of 64)
  int rows_alloc = 0;
  int nslice_valid = 0;          // slices written by the last slicing pass
  int bits = 12;                 // bits per slice after the first (9..12)
  // Optional exact row dot products written by the slicing pass (double-float accurate):
  // row_dot[i] = sum_k y_ik p_ik with p = dot_partner (y itself, or the X2 input of the pass).
  // dot_partner == nullptr: row_dot holds nothing for the current slices.
  double* row_dot = nullptr;     // [rows_alloc] or null (no storage)
  const double* dot_partner = nullptr;
  // optional tile occupancy (ceil(rows/128) x mask_ld words) written by a filtering pass;
  // mask_valid says that it describes the current slices
  uint32_t* tile_mask = nullptr;
  int mask_ld = 0;
  bool mask_valid = false;
};

// Slice count and highest slice-pair order used by a product.
struct Precision {
  int nslice = 3;
  int max_order = 3;
  int bits = 12;   // bits per trailing slice: 12 packs more bits, 9 keeps every order's FP32
                   // accumulator below 2^24 (exact) up to K ~ 8192
};

struct SlicedGemmArgs {
  int M = 0, N = 0, K = 0;
  int mode = 0;                       // kGemmSym
  int num_pairs = 0, nacc = 0, tmem_cols = 0;
  int shift = 12;                     // weight of order o is 2^(-shift * o)
  int8_t pair_s[kMaxPairs] = {}, pair_t[kMaxPairs] = {}, pair_o[kMaxPairs] = {};
  // MMA instructions per 16-wide k step (built from the pairs by build_pairs): A slice, first B
  // slice, N = 256 over B slices t and t+1 (whose orders' accumulators are adjacent), whether
  // it opens its accumulators
  int num_ins = 0;
  int8_t ins_s[kMaxPairs] = {}, ins_t[kMaxPairs] = {}, ins_wide[kMaxPairs] = {},
         ins_open[kMaxPairs] = {};
  const double* row_scale_a = nullptr;
  const double* row_scale_b = nullptr;
  double* C = nullptr;
  int64_t ldc = 0;
  double* Ct = nullptr;               // optional: also write C^T
  int64_t ldct = 0;
  const double* D = nullptr;          // optional addend, read transposed: C_ij += beta D_ji
  int64_t ldd = 0;
  double alpha = 1.0, beta = 0.0;
  double diag = 0.0;                  // added to the diagonal of C
  const double* coef = nullptr;       // optional device {alpha, beta}
  const double* diag_dot = nullptr;   // optional: exact sum_k A_ik Bt_ik replaces C_ii's product
  // optional 128 x 128 tile occupancy of A and Bt (TruncArgs masks, row block x k block):
  // k blocks where either operand's tile is empty are skipped (the first k block always runs,
  // so every accumulator is written); kcount (optional) receives the k stages issued
  const uint32_t* mask_a = nullptr;
  const uint32_t* mask_b = nullptr;
  int mask_ld = 0;
  unsigned long long* kcount = nullptr;
  // k split of the last, partial wave of tiles (sliced_gemm sets split and full_tiles when the
  // caller provides the workspace): splitk_slots slots of 128 x 128 int64 partial sums, and
  // kEpilogueWarps zero-initialised counters per split tile, which the kernel leaves at zero
  int split = 1, full_tiles = 0;
  long long* splitk_ws = nullptr;
  uint32_t* splitk_cnt = nullptr;
  int splitk_slots = 0, splitk_tiles = 0;
  const int* skip = nullptr;          // optional device flag: non-zero -> no-op launch
  uint32_t* err = nullptr;
  int tiles_n = 0, tiles_m = 0;
  // grouped launch (sliced_gemm_grouped): the products of a device table, one after another
  // in the unit order; each entry's own fields describe its product, these only its format
  const struct GroupItem* group = nullptr;
  int ngroup = 0, group_units = 0;
  int unit_begin = 0;                 // grouped: first unit of this product in the launch
};

// One product of a grouped launch: its operands' tensor maps (global memory, aligned as
// CUtensorMap requires) and its arguments (C, leading dimensions, epilogue coefficients, row
// scales, skip flag, M, N, K, tiles, unit_begin); the format fields of `a` are ignored.
struct GroupItem {
  CUtensorMap ta;
  CUtensorMap tb;
  SlicedGemmArgs a;
};

// Number of kernels this library has launched since it was loaded (all threads).
void count_launch(int k = 1);
int64_t launch_count();

int build_pairs(int nslice, int max_order, SlicedGemmArgs* a);
cudaError_t sliced_gemm(const SliceBuf& A, const SliceBuf& Bt, const Precision& prec,
                        SlicedGemmArgs args, cudaStream_t stream);

// Grouped products.  sliced_gemm_group_item fills one table entry for C = alpha A Bt^T (+ ...)
// from the operands' slice buffers and `args` (C, ldc, mode, alpha, ...; skip is the entry's
// own flag); sliced_gemm_grouped then runs every entry of the device table `items` (count
// entries, built with the same format `prec`) in one persistent launch: the CTAs walk the
// 128 x 128 tiles of all products, entries in table order.  Returns cudaErrorInvalidValue for
// operands that do not fit the format.  The k split of the last wave is not used here.
// `bk` is the k extent of the operands' tensor-map boxes: grouped_variant_bk(nslice, variant)
// of the variant the launch will use.  group_assign_units sets each entry's unit_begin (table
// order) and returns the launch's unit count.
cudaError_t sliced_gemm_group_item(const SliceBuf& A, const SliceBuf& Bt, const Precision& prec,
                                   const SlicedGemmArgs& args, GroupItem* item, int bk);
int group_assign_units(GroupItem* items, int count);
cudaError_t sliced_gemm_grouped(const GroupItem* items_dev, int count, int total_units,
                                const Precision& prec, uint32_t* err, cudaStream_t stream,
                                int variant = 0);
// (BK, stages) variants of the grouped kernel for a slice count (the autotuner's choices).
int grouped_variant_count(int nslice);
int grouped_variant_bk(int nslice, int variant);

// K elements per pipeline stage of sliced_gemm for a format with `nslice` slices.
int sliced_gemm_bk(int nslice);

// FP64 product C = alpha * A * Bt^T + beta * D (+ mirror / transposed copy as above).
struct F64GemmArgs {
  int M = 0, N = 0, K = 0;
  int mode = 0;
  const double* A = nullptr;
  int64_t lda = 0;
  const double* Bt = nullptr;
  int64_t ldb = 0;
  double* C = nullptr;
  int64_t ldc = 0;
  double* Ct = nullptr;
  int64_t ldct = 0;
  const double* D = nullptr;
  int64_t ldd = 0;
  double alpha = 1.0, beta = 0.0;
  double diag = 0.0;
  const double* coef = nullptr;
  const int* skip = nullptr;
};
cudaError_t f64_gemm(const F64GemmArgs& a, cudaStream_t stream);

// ---- elementwise / reduction kernels (elementwise.cu) --------------------------------------
// Y = a*X + b*X2 + c*I with (a, b, c) from `coef_dev` (3 doubles) when non-null, else
// (ha, hb, hc).  X2 may be null (then b is ignored).  Writes Y (FP64) when Y != null, and the
// row slices of Y into `out` when out != null and nslice > 0.  dot: 0 none, 1 the row dot
// products sum_k y_ik^2, 2 sum_k y_ik X2_ik, 3 sum_k y_ik X_ik, written to out->row_dot when the buffer has one
// (out->dot_partner then names the partner matrix; otherwise it is reset to null).
enum { kDotNone = 0, kDotSelf = 1, kDotX2 = 2, kDotX = 3 };

// Threshold filtering of the sparse (truncated) purification: values with |y| < tau become zero
// (tau given by the bit pattern of the positive double, compared with the magnitude bits), and
// mask[(row / 128) * mask_ld + col / 128] = 1 marks each 128 x 128 tile that keeps a non-zero
// element.  tau_bits == 0 turns it off.  form_and_slice takes the mask from its output slice
// buffer (tile_mask) and sets mask_valid there; it writes the filtered values in place when Y
// is null.
struct TruncArgs {
  unsigned long long tau_bits = 0;
  uint32_t* mask = nullptr;
  int mask_ld = 0;
};

// purification maps (the values of gdm_purification)
enum { kPurifyTrs4 = 0, kPurifyTrs2 = 1, kPurifyCanonical = 2 };
// Widest row (columns) that form_and_slice forms and slices in one pass (the row stays in
// registers); wider or unaligned rows take two passes, which need Y when the forming is not
// plain and a row dot product is asked for.
constexpr int kFusedMaxCols = 8192;
// zero_pad: the caller guarantees a zero column after the `cols` columns of X, X2 and Y (and
// room for it in the slices): an odd `cols` is then processed as the even cols + 1 by the paired
// one-pass kernels (the engine's buffers keep that column zero).
cudaError_t form_and_slice(const double* X, int64_t ldx, const double* X2, int64_t ldx2,
                           int rows, int cols, const double* coef_dev, double ha, double hb,
                           double hc, double* Y, int64_t ldy, SliceBuf* out, int nslice,
                           const int* skip, cudaStream_t stream, int bits = 12,
                           int dot = kDotNone, const TruncArgs* trunc = nullptr,
                           bool zero_pad = false);
// A[i, col] = 0 for i < rows (the zero column after an odd n).
cudaError_t zero_column(double* A, int64_t lda, int rows, int col, cudaStream_t stream);

// `steps` Lanczos steps on the symmetric n x n matrix A from a fixed start vector (no
// reorthogonalisation): ab_dev[k] = alpha_k and ab_dev[steps + k] = beta_k for k < steps, the
// diagonal and off-diagonal of the tridiagonal whose extreme eigenvalues estimate A's from inside.
// FP32 recurrence (see elementwise.cu); `work` holds >= 2 n doubles (three FP32 vectors and a
// counter); `partials` is unused.  With a32 (n rows of lda32 >= n floats, lda32 even; may be
// null) the first step also writes A truncated to FP32 there and the later steps read that copy.
cudaError_t lanczos(const double* A, int64_t lda, int n, int steps, double* work,
                    double* partials, double* ab_dev, cudaStream_t stream, float* a32 = nullptr,
                    int64_t lda32 = 0);

// Spectral bounds from a Lanczos tridiagonal (small[lanczos_at..]: alpha_0..alpha_{steps-1},
// beta_0..beta_{steps-1}) and Gershgorin's interval (small[gersh_at..+1]): the extreme Ritz values
// by bisection on Sturm counts, widened by 2% of their span and clamped to Gershgorin's
// interval, into small[bounds_at..+1]; small[bounds_at + 2] = 1 when the estimate is used, 0
// when Gershgorin's interval is (a non-finite or degenerate recurrence); small[bounds_at + 3..4]
// the extreme Ritz values themselves (Gershgorin's bounds when there are none).  FP32
// arithmetic (estimates to ~1e-6 of the matrix norm); steps <= kMaxLanczos.
cudaError_t lanczos_bounds(double* small, int steps, int gersh_at, int lanczos_at, int bounds_at,
                           cudaStream_t stream);

// Gershgorin bounds of a symmetric n x n matrix: writes {min_i(a_ii - r_i), max_i(a_ii + r_i)}
// into out_dev[0..1].  `partials` holds >= 2 * ceil(n / 8) doubles.
cudaError_t gershgorin(const double* A, int64_t lda, int n, double* partials, double* out_dev,
                       cudaStream_t stream);

// Per-block partial sums over rows of: Tr X, Tr X2, <X2, X>, ||X2||^2, ||X||^2
// (partials: kTraceTerms doubles per block, `nblocks` returned through *nblocks).
constexpr int kTraceTerms = 5;
// TRS4 trace terms per row (partials: n x kTraceTerms) and the slices of X2 in one pass;
// slice_traces_fits says whether the shapes and alignments allow it.  x_row_dot (may be null):
// ||X_r||^2 per row as X's own slicing pass computed it, taken instead of summing it again.
cudaError_t slice_traces(const double* X2, const double* X, int64_t ld, int n, SliceBuf* out,
                         int nslice, int bits, double* partials, int* nrows, cudaStream_t stream,
                         const int* skip = nullptr, bool zero_pad = false,
                         const double* x_row_dot = nullptr);
bool slice_traces_fits(const double* X2, const double* X, int64_t ld, int n, const SliceBuf* out,
                       int nslice, bool zero_pad = false);
// w->row_dot[i] = <W_i, X2_i> for W = coef[0] X + coef[1] X2 + coef[2] I, from slice_traces'
// per-row terms (so the slicing of W needs no row dot); records X2 as w's dot partner.
cudaError_t w_row_dots(const double* partials, int n, const double* coef_dev, SliceBuf* w,
                       const double* X2, cudaStream_t stream);
cudaError_t trs4_traces(const double* X, const double* X2, int64_t ld, int n, double* partials,
                        int* nblocks, cudaStream_t stream, const int* skip = nullptr);

// (skip: a non-zero flag makes the launch a no-op, for the problems of a lockstep batch that
// have finished.)
// Deterministic partial dot products of sum_ij A_ij B_ij (B null -> A_ij^2), with an optional
// -1 on the diagonal of A first when `minus_identity` (||A - I||^2): one partial per row (rows of
// at most kFusedMaxCols columns), else one per block of rows; *nblocks gives the count, and
// partials must hold `rows` doubles.
cudaError_t dot_partials(const double* A, int64_t lda, const double* B, int64_t ldb, int rows,
                         int cols, int minus_identity, double* partials, int* nblocks,
                         cudaStream_t stream, const int* skip = nullptr, bool zero_pad = false);
cudaError_t reduce_partials(const double* partials, int nblocks, int nterms, double* out_dev,
                            cudaStream_t stream);

// TRS4 controller state (device, one per solve).
struct Trs4State {
  double n_occ;
  double t[kTraceTerms];  // reduced traces of this iteration
  double gamma;
  double idem;            // Tr(X - X^2) = t1 - ||X||^2
  double idem_prev;
  double trG;
  double coefW[3];        // W = a X + b X2 + c I; X_next = X2 W
  double coefX[3];        // X_next = a X + b X2 for the branches without a product
  double gemm_coef[2];    // (1, 0): alpha and beta of the X2 W product (no addend)
  int method;             // kPurify*
  int branch;             // 0: 2X - X2, 1: X2, 2: X2 W (TRS4 F + gamma G), 3: McWeeny X2 (3I - 2X),
                          // 4: X W (canonical)
  int skip_gemm;          // 1 unless branch 2 or 3
  int skip_form_x;        // 1 when branch 2 or 3
  int stop;               // 1: converged (X is final), 2: stalled, 3: non-finite, 4: cap
  int iter;
  int stall;
  // lockstep batches (zero in a single solve, which leaves the loop at the first stop):
  int done;               // set at the first stop; later controls change nothing
  int final_buf;          // 0: the final iterate is in the iteration's even buffer, 1: odd
  double final_idem;
  int max_iter;           // > 0: stop with 4 once iter reaches it
  int check_trace;        // 1: a trace outside [-0.5, n + 0.5] stops with 3 and sets failed
  int failed;
  double n;               // matrix size (for check_trace)
  int floor_rule;         // 1: also stop once a quadratic step lands at the rounding floor
};
cudaError_t trs4_control(const double* partials, int nblocks, Trs4State* st, double tol_idem,
                         cudaStream_t stream);

// Coefficients {a, 0, c} of the canonical initial guess X0 = a H~ + c I from the bounds and
// the trace of H~ (read from its diagonal).
cudaError_t canonical_x0_coefficients(const double* bounds_dev, const double* Ht, int64_t ld, int n,
                                      double n_occ, double* coef_dev, cudaStream_t stream);

// Set the bounds-dependent coefficients of the initial guess
// X0 = (eps_max I - H~)/(eps_max - eps_min): coef = {-1/(hi-lo), 0, hi/(hi-lo)}.
cudaError_t x0_coefficients(const double* bounds_dev, double* coef_dev, cudaStream_t stream);
// coef = {s, 0, 0} with s = 1 / bound[1] (Y_0 = S / c) or s = 1 / sqrt(bound[1]).
cudaError_t scale_coefficients(const double* bounds_dev, int inv_sqrt, double* coef_dev,
                               cudaStream_t stream);

// Diagonal of a square product recomputed from the FP64 operands (FP32 double-float dot
// products, ~2^-48 relative): C_ii = alpha <A_i, Bt_i> + beta D_ii + diag ((alpha, beta) from
// coef when non-null).  Run after the sliced product (see elementwise.cu).
cudaError_t diag_fix(const double* A, int64_t lda, const double* Bt, int64_t ldb, double* C,
                     int64_t ldc, int n, int K, double alpha, double beta, const double* D,
                     int64_t ldd, double diag, const double* coef, cudaStream_t stream,
                     const int* skip = nullptr);

// X <- X * target / Tr X (trace in FP64); fix_out (device, 2 doubles) = {target/Tr X - 1,
// target/Tr X}.
cudaError_t trace_scale(double* X, int64_t ld, int n, double target, double* fix_out,
                        cudaStream_t stream);

// Symmetrise in place: A <- (A + A^T) / 2.
cudaError_t symmetrise(double* A, int64_t lda, int n, cudaStream_t stream);

// Copy rows x cols into a dense-ld destination (device-to-device, strided).
cudaError_t set_identity(double* A, int64_t lda, int n, cudaStream_t stream);
// Whether dot_partials(A, lda, v, 0, n, n, 0, y, ...) is the matrix-vector product y = A v in
// double-float (one block per row, the vector read as every row of B): n even, at most
// kFusedMaxCols, lda even, A and v 16-byte aligned.
bool matvec_rows_fit(const double* A, int64_t lda, int n, const double* v);
// v[j] = +-1 (j < n) from an integer hash of (j, seed).
cudaError_t fill_rademacher(double* v, int n, unsigned seed, cudaStream_t stream);

}  // namespace gdm
