// Handle, solve plan and C ABI of the density-matrix engine (include/gdm.h).
//
// Solve plan for one (H, S) pair, all on the handle's stream:
//   1. Z with Z^T S Z = I (cached per geometry, Sec. 2.7 "reinit"):
//        coupled Newton-Schulz for S^{-1/2}: c = Gershgorin bound of S, Y_0 = S/c, Z_0 = I,
//        M = Y_k Z_k,  Y_{k+1} = (3 Y_k - M Y_k)/2,  Z_{k+1} = (3 Z_k - M^T Z_k)/2
//        (the same iteration as T = (3I - Z Y)/2, Y <- Y T, Z <- T Z, written so that every
//        product has a symmetric right factor and the two updates are symmetric products);
//        Z_0' = Z_k / sqrt(c); then Z <- Z (I - delta/2 + 3 delta^2/8), delta = Z^T S Z - I,
//        which drives Z^T S Z to I without needing Z = S^{-1/2} exactly.
//   2. H~ = Z^T H Z                                          (Sec. 2.2.2, Eq. ntpoly_lowdin)
//   3. X_0 = (eps_max I - H~)/(eps_max - eps_min), Gershgorin eps  (Eq. ntpoly_scale_hamiltonian)
//   4. TRS4 purification X <- f(X)                           (Eq. ntpoly_purification; Table 1)
//   5. P = Z X Z^T, Tr(P S), Tr(P H)                          (Sec. 4, back-transform)
// Products run through the sliced tensor-core kernel (mixed precision) or the FP64 kernel.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "../../include/gdm.h"
#include "gdm_internal.h"
#include "handle.h"

using namespace gdm;

namespace {


gdm_status set_err(gdm_handle* h, gdm_status st, const char* fmt, ...) {
  if (h != nullptr) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    h->last_error = buf;
  }
  return st;
}

#define CK(expr)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (expr);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return set_err(h, GDM_ERR_CUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));   \
  } while (0)

struct Op {
  double* f;
  SliceBuf* sl;
};

bool mixed(const gdm_handle* h) { return h->prec == GDM_PREC_MIXED; }

// A phase runs on the sliced tensor-core kernel unless the handle is in FP64 mode or the
// phase's slice count is 0 (that phase then uses the FP64 kernel).
bool sliced(const gdm_handle* h, int ph) { return mixed(h) && h->phase[ph].nslice > 0; }

// device address of a field of the device-resident controller state
const double* st_field(const gdm_handle* h, size_t offset) {
  return reinterpret_cast<const double*>(reinterpret_cast<const char*>(h->st_dev) + offset);
}

int slices_for(const gdm_handle* h, int ph) { return sliced(h, ph) ? h->phase[ph].nslice : 0; }

cudaEvent_t pool_event(gdm_handle* h) {
  if (!h->ev_pool.empty()) {
    cudaEvent_t e = h->ev_pool.back();
    h->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Fold the recorded launch timings into the totals (the stream must be idle).
void collect_profile(gdm_handle* h) {
  for (auto& p : h->prof_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      h->prof_ms[p.kind] += ms;
      h->prof_flops[p.kind] += p.flops;
      h->prof_alg[p.kind] += p.alg;
      h->prof_launches[p.kind] += 1;
      if (p.kind == 0) {
        h->prof_ms[2 + p.phase] += ms;
        h->prof_flops[2 + p.phase] += p.flops;
        h->prof_alg[2 + p.phase] += p.alg;
        h->prof_launches[2 + p.phase] += 1;
      }
    }
    h->ev_pool.push_back(p.a);
    h->ev_pool.push_back(p.b);
  }
  h->prof_pending.clear();
}

// The device error word and the split-k counters (an aborted launch can leave a counter set).
cudaError_t clear_device_flags(gdm_handle* h, cudaStream_t s) {
  return cudaMemsetAsync(h->err_dev, 0,
                         sizeof(uint32_t) * (1 + static_cast<size_t>(kSplitTiles) * kEpilogueWarps),
                         s);
}

// Algorithmic work of one n x n x n product: n^3 when only the upper triangle of a symmetric
// result is formed, 2 n^3 otherwise (the count the roofline of the route is quoted in).
double alg_flops(const gdm_handle* h, bool sym) {
  const double n = static_cast<double>(h->n);
  return (sym ? 1.0 : 2.0) * n * n * n;
}

// Tensor-pipe work of one sliced launch: slice pairs x computed tile area x 2 K
double sliced_flops(const gdm_handle* h, const Precision& pr, bool sym) {
  const double n = static_cast<double>(h->n);
  const double t = std::ceil(n / 128.0);
  const double tiles = sym ? t * (t + 1) / 2 : t * t;
  SlicedGemmArgs tmp;
  const int pairs = build_pairs(pr.nslice, pr.max_order, &tmp);
  return pairs * tiles * 128.0 * 128.0 * 2.0 * n;
}

// C = alpha * A * Bt^T + beta * D + diag * I (sym: C symmetric, upper tiles + mirror)
// exact_diag: recompute the diagonal from the FP64 operands.  Needed where the two factors
// have (nearly) parallel rows (X X, X^2 W, delta delta): there the residual-slice terms of the
// diagonal add up with one sign and the FP32 accumulators' truncation biases them.
// fmt: a format other than the phase's for this product (its slice width must be the
// operands'; it may read only their leading slices), e.g. a short format for a small term.
cudaError_t product(gdm_handle* h, Op A, Op Bt, double* C, double* Ct, const double* D,
                    double alpha, double beta, double diag, bool sym, int ph,
                    const double* coef = nullptr, bool exact_diag = false,
                    const Precision* fmt = nullptr) {
  const int n = static_cast<int>(h->n);
  if (sliced(h, ph)) {
    const Precision& pr = fmt != nullptr ? *fmt : h->phase[ph];
    SlicedGemmArgs a;
    a.mode = sym ? kGemmSym : 0;
    a.C = C;
    a.ldc = h->ld;
    a.Ct = Ct;
    a.ldct = h->ld;
    a.D = D;
    a.ldd = h->ld;
    a.alpha = alpha;
    a.beta = beta;
    a.diag = diag;
    a.coef = coef;
    a.err = h->err_dev;
    a.splitk_ws = h->split_ws;
    a.splitk_cnt = h->split_cnt;
    a.splitk_slots = h->split_slots;
    a.splitk_tiles = kSplitTiles;
    // truncated purification: skip the k blocks where an operand tile is empty
    if (ph == GDM_PHASE_PURIFY && h->trunc_tau > 0.0 && A.sl->mask_valid && Bt.sl->mask_valid) {
      a.mask_a = A.sl->tile_mask;
      a.mask_b = Bt.sl->tile_mask;
      a.mask_ld = A.sl->mask_ld;
      a.kcount = reinterpret_cast<unsigned long long*>(h->small + SM_KCOUNT);
      const double t = std::ceil(static_cast<double>(n) / 128.0);
      const double nk = std::ceil(static_cast<double>(n) /
                                  static_cast<double>(sliced_gemm_bk(pr.nslice)));
      h->kstages_dense += (sym ? t * (t + 1) / 2 : t * t) * nk;
    }
    // exact diagonal from the row dot products of the right operand's slicing pass, when that
    // pass paired its rows with the left operand (X X, X^2 W, delta delta)
    if (exact_diag && Bt.sl->row_dot != nullptr && Bt.sl->dot_partner == A.f)
      a.diag_dot = Bt.sl->row_dot;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (h->profiling) {
      e0 = pool_event(h);
      e1 = pool_event(h);
      cudaEventRecord(e0, h->stream);
    }
    cudaError_t e = sliced_gemm(*A.sl, *Bt.sl, pr, a, h->stream);
    if (e != cudaSuccess) return e;
    if (h->profiling) {
      cudaEventRecord(e1, h->stream);
      h->prof_pending.push_back({e0, e1, sliced_flops(h, pr, sym), alg_flops(h, sym), 0, ph});
    }
    if (!exact_diag || a.diag_dot != nullptr) return cudaSuccess;
    e = diag_fix(A.f, h->ld, Bt.f, h->ld, C, h->ld, n, n, alpha, beta, D, h->ld, diag, coef,
                 h->stream);
    if (e != cudaSuccess || Ct == nullptr) return e;
    return diag_fix(A.f, h->ld, Bt.f, h->ld, Ct, h->ld, n, n, alpha, beta, D, h->ld, diag, coef,
                    h->stream);
  }
  F64GemmArgs a;
  a.M = n;
  a.N = n;
  a.K = n;
  a.mode = sym ? kGemmSym : 0;
  a.A = A.f;
  a.lda = h->ld;
  a.Bt = Bt.f;
  a.ldb = h->ld;
  a.C = C;
  a.ldc = h->ld;
  a.Ct = Ct;
  a.ldct = h->ld;
  a.D = D;
  a.ldd = h->ld;
  a.alpha = alpha;
  a.beta = beta;
  a.diag = diag;
  a.coef = coef;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (h->profiling) {
    e0 = pool_event(h);
    e1 = pool_event(h);
    cudaEventRecord(e0, h->stream);
  }
  cudaError_t e = f64_gemm(a, h->stream);
  if (h->profiling && e == cudaSuccess) {
    cudaEventRecord(e1, h->stream);
    const double nn = static_cast<double>(n);
    const double t = std::ceil(nn / 64.0);
    h->prof_pending.push_back(
        {e0, e1, (sym ? t * (t + 1) / 2 : t * t) * 64.0 * 64.0 * 2.0 * nn, alg_flops(h, sym), 1, ph});
  }
  return e;
}

// Slice `src` (FP64) into `dst` in the format of phase `ph` (no-op when that phase is FP64).
// Threshold filtering for the purification's operands when truncation is on (else null).
const TruncArgs* purify_trunc(const gdm_handle* h, TruncArgs* tmp) {
  if (!(h->trunc_tau > 0.0)) return nullptr;
  double t = h->trunc_tau;
  std::memcpy(&tmp->tau_bits, &t, sizeof(t));
  return tmp;
}

cudaError_t slice(gdm_handle* h, const double* src, SliceBuf* dst, int ph, int dot = kDotNone,
                  const TruncArgs* trunc = nullptr) {
  const int n = static_cast<int>(h->n);
  if (!sliced(h, ph)) {
    if (trunc == nullptr) return cudaSuccess;
    // FP64 products: filter the matrix in place (no slices)
    return form_and_slice(src, h->ld, nullptr, 0, n, n, nullptr, 1.0, 0.0, 0.0, nullptr, 0,
                          nullptr, 0, nullptr, h->stream, 12, kDotNone, trunc, true);
  }
  return form_and_slice(src, h->ld, nullptr, 0, n, n, nullptr, 1.0, 0.0, 0.0, nullptr, 0, dst,
                        h->phase[ph].nslice, nullptr, h->stream, h->phase[ph].bits, dot, trunc,
                        true);
}

int bits_for(const gdm_handle* h, int ph) { return h->phase[ph].bits; }

// Synchronous scalar read-back of small[SM_RED + k] for k < count.
gdm_status read_small(gdm_handle* h, int offset, int count, double* out) {
  CK(cudaMemcpyAsync(h->host_buf, h->small + offset, sizeof(double) * count,
                     cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  for (int i = 0; i < count; ++i) out[i] = h->host_buf[i];
  return GDM_OK;
}

// sum_ij (A - I)_ij^2 (minus_identity) or sum_ij A_ij B_ij into *out (synchronous)
gdm_status dot(gdm_handle* h, const double* A, const double* B, int minus_identity,
               double* out) {
  const int n = static_cast<int>(h->n);
  int nb = 0;
  CK(dot_partials(A, h->ld, B, h->ld, n, n, minus_identity, h->partials, &nb, h->stream,
                  nullptr, true));
  CK(reduce_partials(h->partials, nb, 1, h->small + SM_RED, h->stream));
  return read_small(h, SM_RED, 1, out);
}

gdm_status check_device_error(gdm_handle* h) {
  uint32_t e = 0;
  CK(cudaMemcpyAsync(&e, h->err_dev, sizeof(uint32_t), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (e & DEV_ERR_WAIT_TIMEOUT)
    return set_err(h, GDM_ERR_TIMEOUT, "a kernel wait ran out of time (device error 0x%x)", e);
  if (e != 0) return set_err(h, GDM_ERR_CUDA, "device error word 0x%x", e);
  return GDM_OK;
}

// ------------------------------------------------------------------------------------------
// step 1: Z with Z^T S Z = I
// ------------------------------------------------------------------------------------------
constexpr int kLanczosS = 16;  // Lanczos steps on S for its spectral estimates
constexpr double kNsHandoff = 0.005;  // ||I - M||_F at which Newton-Schulz hands over

// ||Z^T S Z - I||_F of the refined Z from two Rademacher probes v: E ||(Z^T S Z - I) v||^2 =
// ||Z^T S Z - I||_F^2, and each probe costs three double-float matrix-vector products
// (u = Z v, w = S u, t = Z^T w, reading Z^T from its explicit copy) and an FP64 difference
// t - v, where forming Z^T S Z itself takes two full-precision products.  Scratch: four rows of
// F_U (the refinement's delta, no longer needed).  *done = false (nothing run) when the rows do
// not fit the one-block-per-row products; the caller then measures.
gdm_status probe_z_err(gdm_handle* h, const double* Z, const double* Zt, double* z_err,
                       bool* done) {
  *done = false;
  const int n = static_cast<int>(h->n);
  const int64_t ld = h->ld;
  cudaStream_t s = h->stream;
  const double* S = h->f[F_S];
  double* v = h->f[F_U];
  double *u = v + ld, *w = v + 2 * ld, *t = v + 3 * ld;
  if (n < 4 || !matvec_rows_fit(Z, ld, n, v) || !matvec_rows_fit(Zt, ld, n, v) ||
      !matvec_rows_fit(S, ld, n, v))
    return GDM_OK;
  constexpr int kProbes = 2;
  for (int p = 0; p < kProbes; ++p) {
    int nb = 0;
    CK(fill_rademacher(v, n, 0x51u + static_cast<unsigned>(p), s));
    CK(dot_partials(Z, ld, v, 0, n, n, 0, u, &nb, s));
    CK(dot_partials(S, ld, u, 0, n, n, 0, w, &nb, s));
    CK(dot_partials(Zt, ld, w, 0, n, n, 0, t, &nb, s));
    CK(form_and_slice(t, ld, v, ld, 1, n, nullptr, 1.0, -1.0, 0.0, t, ld, nullptr, 0, nullptr, s));
    CK(dot_partials(t, ld, nullptr, 0, 1, n, 0, h->partials + p, &nb, s));  // ||t - v||^2
  }
  CK(reduce_partials(h->partials, kProbes, 1, h->small + SM_RED, s));
  double sum = 0.0;
  const gdm_status st = read_small(h, SM_RED, 1, &sum);
  if (st != GDM_OK) return st;
  *z_err = std::sqrt(sum / kProbes);
  *done = true;
  return GDM_OK;
}

// Whether a refinement step taken from ||delta||_F = before, which measured `after`, reached
// the rounding floor (the third-order prediction (5/8) before^3 is at or below what is left).
bool refine_at_floor(double before, double after) {
  return std::isfinite(before) && 0.625 * before * before * before <= after;
}

// The Newton-Schulz eigenvalue map g(x) = x (3 - x)^2 / 4 and the scale of step `it` for a
// smallest eigenvalue l of M: the first step is plain (it brings every eigenvalue into (0, 1]),
// later ones take alpha = 3 / (1 + sqrt(l) + l) (capped at 2.9) until l passes 0.3.
double ns_g(double x) { return x * (3.0 - x) * (3.0 - x) * 0.25; }
double ns_alpha(int it, double l) {
  if (it == 0 || !(l > 0.0) || l >= 0.3) return 1.0;
  const double r = std::sqrt(l);
  return std::min(2.9, 3.0 / (1.0 + r + l));
}
gdm_status compute_z(gdm_handle* h, gdm_info* info) {
  const int n = static_cast<int>(h->n);
  const int64_t ld = h->ld;
  cudaStream_t s = h->stream;
  const int ns_sl = slices_for(h, GDM_PHASE_NEWTON_SCHULZ);
  const int ref_sl = slices_for(h, GDM_PHASE_REFINE);
  double* S = h->f[F_S];
  double* bounds = h->small + SM_BOUNDS_S;
  double* coef_inv = h->small + SM_COEF_A;
  double* coef_isqrt = h->small + SM_COEF_B;

  // Gershgorin's interval of S and the extreme Ritz values of a short Lanczos recurrence
  // (estimates of lambda_max and lambda_min of S from inside the spectrum)
  CK(gershgorin(S, ld, n, h->partials, bounds, s));
  const int lzs = std::min(kLanczosS, n);
  // the FP32 copy of S for the recurrence's later steps lives in M's buffer (unused until the
  // Newton-Schulz iteration)
  CK(lanczos(S, ld, n, lzs, h->lanczos_ws, h->partials, h->small + SM_LANCZOS, s,
             reinterpret_cast<float*>(h->f[F_T]), ld));
  CK(lanczos_bounds(h->small, lzs, SM_BOUNDS_S, SM_LANCZOS, SM_EST_S, s));
  double smv[SM_EST_S + 5];
  gdm_status st = read_small(h, 0, SM_EST_S + 5, smv);
  if (st != GDM_OK) return st;
  const double bnd[2] = {smv[SM_BOUNDS_S], smv[SM_BOUNDS_S + 1]};
  if (!std::isfinite(bnd[0]) || !std::isfinite(bnd[1]))
    return set_err(h, GDM_ERR_NONFINITE, "overlap matrix has non-finite entries");
  if (bnd[1] <= 0.0) return set_err(h, GDM_ERR_NOT_SPD, "overlap Gershgorin bound <= 0");
  const double ritz_min = smv[SM_EST_S + 3], ritz_max = smv[SM_EST_S + 4];

  double *Y = h->f[F_X], *Z = h->f[F_XN], *M = h->f[F_T], *Mt = h->f[F_U];
  double *Yn = h->f[F_X2], *Zn = h->f[F_V];
  SliceBuf *sY = &h->sl[SL_X], *sZ = &h->sl[SL_Z], *sM = &h->sl[SL_A], *sMt = &h->sl[SL_B];
  const double rn = std::sqrt(static_cast<double>(n));
  const double ns_handoff = (mixed(h) && h->n_refine >= 1) ? kNsHandoff : 0.0;
  double prev = INFINITY, res = INFINITY;
  int it = 0;
  bool converged = false;
  // The iteration converges for every scale c with lambda_max(S)/c < 3, and the number of
  // steps grows with c/lambda_min(S).  Gershgorin's bound can exceed lambda_max many times over
  // for a dense S, so the first attempt uses 1.05 x the largest Ritz value (never above
  // Gershgorin); if that attempt diverges, the second uses Gershgorin's guaranteed bound.
  // Scaled steps.  Each eigenvalue m of M = Y Z (in (0, 1] after one plain step) maps to
  // g(alpha m), g(x) = x (3 - x)^2 / 4, when T = sqrt(alpha) (3I - alpha M)/2 (alpha = 1 is the
  // plain step).  With the smallest eigenvalue at l, alpha = 3 / (1 + r + r^2), r = sqrt(l),
  // solves g(alpha l) = g(alpha), so the whole interval [l, 1] lands in [g(alpha l), 1]: the
  // lower end grows ~6.5-fold per step instead of 2.25-fold (cond(S) = 1e3: 11 -> 8 steps).
  // l comes from the smallest Ritz value, which lies above lambda_min, so alpha errs on the
  // small side; every alpha in [1, 3) keeps all eigenvalues in (0, 1], so the iteration
  // converges whatever l is.
  for (int attempt = 0; attempt < 2; ++attempt) {
    const double c = (attempt == 0 && ritz_max > 0.0 && std::isfinite(ritz_max))
                         ? std::min(bnd[1], 1.05 * ritz_max) : bnd[1];
    double lsc = (ritz_min > 0.0 && std::isfinite(ritz_min)) ? std::min(1.0, ritz_min / c) : 1.0;
    h->host_buf[0] = bnd[0];
    h->host_buf[1] = c;
    CK(cudaMemcpyAsync(bounds, h->host_buf, 2 * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(scale_coefficients(bounds, 0, coef_inv, s));
    CK(scale_coefficients(bounds, 1, coef_isqrt, s));
    CK(form_and_slice(S, ld, nullptr, 0, n, n, coef_inv, 0, 0, 0, Y, ld, ns_sl > 0 ? sY : nullptr,
                      ns_sl, nullptr, s, bits_for(h, GDM_PHASE_NEWTON_SCHULZ), kDotNone, nullptr, true));
    CK(set_identity(Z, ld, n, s));
    CK(slice(h, Z, sZ, GDM_PHASE_NEWTON_SCHULZ));
    prev = INFINITY;
    res = INFINITY;
    converged = false;
    bool diverged = false;
    for (it = 0; it < h->max_ns; ++it) {
      // M = Y Z in full, with M^T: Y and Z commute only up to rounding, and making M symmetric
      // (one T for both updates) let that error grow until the iteration diverged for
      // cond(S) = 1e3 (measured)
      CK(product(h, {Y, sY}, {Z, sZ}, M, Mt, nullptr, 1.0, 0.0, 0.0, false,
                 GDM_PHASE_NEWTON_SCHULZ));
      double r2 = 0.0;
      st = dot(h, M, nullptr, 1, &r2);
      if (st != GDM_OK) return st;
      res = std::sqrt(r2);
      if (!std::isfinite(res) || res > 1e6 * rn) {
        if (attempt == 0) {
          diverged = true;
          break;
        }
        return set_err(h, GDM_ERR_NOT_SPD,
                       "Newton-Schulz for S^-1/2 diverged (residual %g): S not positive definite",
                       res);
      }
      // Hand over to the refinement once ||I - M||_F <= 0.005: one third-order refinement step
      // then takes Z^T S Z - I to about (5/8) 0.005^3 = 7.8e-8, at the products' rounding floor.
      // A refinement step (four 4-slice products) costs about five Newton-Schulz steps (three
      // 2-slice products), so the last quadratic Newton-Schulz step from ~0.05 is the cheaper way
      // down to 0.005 than a second refinement step.
      if (res <= ns_handoff || res <= 1e-13 * rn || (res < 1e-2 * rn && res > 0.5 * prev)) {
        converged = true;
        break;
      }
      prev = res;
      // T = sqrt(alpha) (3I - alpha M)/2 and T^T, formed in place while slicing, so that
      // Y <- T Y and Z <- T^T Z are plain products (no addend in the epilogue)
      const double alpha = ns_alpha(it, lsc);
      lsc = ns_g(alpha * lsc);
      const double ta = -0.5 * alpha * std::sqrt(alpha), tc = 1.5 * std::sqrt(alpha);
      CK(form_and_slice(M, ld, nullptr, 0, n, n, nullptr, ta, 0.0, tc, M, ld,
                        ns_sl > 0 ? sM : nullptr, ns_sl, nullptr, s,
                        bits_for(h, GDM_PHASE_NEWTON_SCHULZ), kDotNone, nullptr, true));
      CK(form_and_slice(Mt, ld, nullptr, 0, n, n, nullptr, ta, 0.0, tc, Mt, ld,
                        ns_sl > 0 ? sMt : nullptr, ns_sl, nullptr, s,
                        bits_for(h, GDM_PHASE_NEWTON_SCHULZ), kDotNone, nullptr, true));
      CK(product(h, {M, sM}, {Y, sY}, Yn, nullptr, nullptr, 1.0, 0.0, 0.0, true,
                 GDM_PHASE_NEWTON_SCHULZ));
      CK(product(h, {Mt, sMt}, {Z, sZ}, Zn, nullptr, nullptr, 1.0, 0.0, 0.0, true,
                 GDM_PHASE_NEWTON_SCHULZ));
      std::swap(Y, Yn);
      std::swap(Z, Zn);
      CK(slice(h, Y, sY, GDM_PHASE_NEWTON_SCHULZ));
      CK(slice(h, Z, sZ, GDM_PHASE_NEWTON_SCHULZ));
    }
    if (!diverged) break;
  }
  if (info) info->ns_iters = it;
  (void)converged;  // a capped run is still refined below; z_err reports the outcome

  // Z_0 = Z_k / sqrt(c), symmetric: its transpose is itself
  double* Zc = h->f[F_Z];
  CK(form_and_slice(Z, ld, nullptr, 0, n, n, coef_isqrt, 0, 0, 0, Zc, ld,
                    ref_sl > 0 ? &h->sl[SL_Z] : nullptr, ref_sl, nullptr, s,
                    bits_for(h, GDM_PHASE_REFINE), kDotNone, nullptr, true));
  CK(slice(h, S, &h->sl[SL_S], GDM_PHASE_REFINE));
  Op zc = {Zc, &h->sl[SL_Z]};
  Op zct = zc;
  const int nref = mixed(h) ? h->n_refine : 1;
  double derr = 0.0, derr_prev = INFINITY;
  for (int r = 0; r <= nref; ++r) {
    double* T = h->f[F_T];
    double* Dl = h->f[F_U];
    double* F = h->f[F_V];
    if (r == nref && r > 0) {
      // after the last step only the report remains: estimate it from probes where they fit
      bool probed = false;
      st = probe_z_err(h, zc.f, zct.f, &derr, &probed);
      if (st != GDM_OK) return st;
      if (probed) {
        if (!std::isfinite(derr)) return set_err(h, GDM_ERR_NONFINITE, "non-finite Z^T S Z");
        break;
      }
    } else if (r > 0 && 0.625 * derr_prev * derr_prev < 1e-4) {
      // The step from derr_prev < 0.0126 predicts (5/8) derr_prev^3 < 1e-4 derr_prev: it most
      // likely landed on the rounding floor.  The probes decide that at a fraction of the cost
      // of forming delta; only if they see the step still converging is delta formed for the
      // next one.  A wrong call (the estimate at or above the prediction while the true
      // ||delta||_F is below it) stops with ||delta||_F under the prediction, at most
      // (5/8) 0.0126^3 = 1.3e-6.
      double est = 0.0;
      bool probed = false;
      st = probe_z_err(h, zc.f, zct.f, &est, &probed);
      if (st != GDM_OK) return st;
      if (probed && std::isfinite(est) && refine_at_floor(derr_prev, est)) {
        derr = est;
        break;
      }
    }
    // Exact diagonals (recomputed from the FP64 operands) for T, delta and Z F: when S is
    // close to I the two factors of each have nearly parallel rows, the truncating FP32
    // accumulators bias every diagonal entry the same way, and the refinement would then drive
    // the computed delta to zero while the true Z^T S Z - I keeps that bias on its diagonal -
    // an electron-count error of about bias x n_occ (measured 3.8e-5 at n = 8192).
    CK(product(h, zct, {S, &h->sl[SL_S]}, T, nullptr, nullptr, 1.0, 0.0, 0.0, false,
               GDM_PHASE_REFINE, nullptr, true));                    // T = Z^T S
    CK(slice(h, T, &h->sl[SL_A], GDM_PHASE_REFINE));
    CK(product(h, {T, &h->sl[SL_A]}, zct, Dl, nullptr, nullptr, 1.0, 0.0, -1.0, true,
               GDM_PHASE_REFINE, nullptr, true));                    // delta = Z^T S Z - I
    double d2 = 0.0;
    st = dot(h, Dl, nullptr, 0, &d2);
    if (st != GDM_OK) return st;
    derr = std::sqrt(d2);
    if (!std::isfinite(derr)) return set_err(h, GDM_ERR_NONFINITE, "non-finite Z^T S Z");
    if (r == nref || derr == 0.0) break;
    // The step is third order: with F = I - delta/2 + 3 delta^2/8 (delta symmetric, so F
    // commutes with it), delta' = (I + delta) F^2 - I = (5/8) delta^3 - (15/64) delta^4 +
    // (9/64) delta^5, so ||delta'||_F <= (5/8) ||delta||_F^3 to leading order.  When the
    // delta measured after a step is at or above that prediction, it is the rounding floor that
    // the sliced products leave in Z^T S Z, and another step cannot lower it.
    if (refine_at_floor(derr_prev, derr)) break;
    derr_prev = derr;
    // The update as Z <- Z + Z G with G = F - I = -delta/2 + 3 delta^2/8: both products have a
    // small factor (||delta|| <= ~0.005 after the hand-over), so they read only the leading
    // slices of their operands - delta^2 two (20 bits with the 9-bit format), Z G three
    // (29 bits) - and Z itself is added exactly in FP64 by the epilogue.  Their rounding then
    // stays far below the step's remainder (5/8) delta^3.  delta^2 keeps the exact diagonal
    // (delta's rows are parallel to themselves); Z G needs none (Z's rows are not parallel to
    // G's, and Z's own diagonal is added in FP64).
    const Precision& rp = h->phase[GDM_PHASE_REFINE];
    const int sq_ns = std::min(rp.nslice, 2), zg_ns = std::min(rp.nslice, 3);
    const Precision sq_fmt{sq_ns, std::min(1, 2 * (sq_ns - 1)), rp.bits};
    const Precision zg_fmt{zg_ns, std::min(2, 2 * (zg_ns - 1)), rp.bits};
    CK(slice(h, Dl, &h->sl[SL_B], GDM_PHASE_REFINE, kDotSelf));
    CK(product(h, {Dl, &h->sl[SL_B]}, {Dl, &h->sl[SL_B]}, F, nullptr, Dl, 0.375, -0.5, 0.0, true,
               GDM_PHASE_REFINE, nullptr, true, &sq_fmt));           // G = -d/2 + 3d^2/8
    CK(slice(h, F, &h->sl[SL_A], GDM_PHASE_REFINE));
    double* Znew = h->f[F_X];
    double* Zt_new = h->f[F_X2];
    // Z + Z G: the addend is read transposed, so Z enters through Z^T
    CK(product(h, zc, {F, &h->sl[SL_A]}, Znew, Zt_new, zct.f, 1.0, 1.0, 0.0, false,
               GDM_PHASE_REFINE, nullptr, false, &zg_fmt));          // Z <- Z (I + G)
    std::swap(h->f[F_Z], h->f[F_X]);
    std::swap(h->f[F_ZT], h->f[F_X2]);
    CK(slice(h, h->f[F_Z], &h->sl[SL_Z], GDM_PHASE_REFINE));
    CK(slice(h, h->f[F_ZT], &h->sl[SL_ZT], GDM_PHASE_REFINE));
    zc = {h->f[F_Z], &h->sl[SL_Z]};
    zct = {h->f[F_ZT], &h->sl[SL_ZT]};
    if (info) info->refine_iters = r + 1;
  }
  if (zct.f == zc.f) {
    // no refinement step ran: Z is symmetric, keep an explicit transpose for the later steps
    CK(cudaMemcpyAsync(h->f[F_ZT], h->f[F_Z], sizeof(double) * ld * n, cudaMemcpyDeviceToDevice,
                       s));
  }
  // Z and Z^T in the format of the transform phase, which uses them from here on
  CK(slice(h, h->f[F_Z], &h->sl[SL_Z], GDM_PHASE_TRANSFORM));
  CK(slice(h, h->f[F_ZT], &h->sl[SL_ZT], GDM_PHASE_TRANSFORM));
  h->z_err = derr;
  h->z_valid = true;
  return GDM_OK;
}

// ------------------------------------------------------------------------------------------
// S-metric clean-up of the back-transformed density matrix
// ------------------------------------------------------------------------------------------
// McWeeny's map in the S metric, P' = 3 P S P - 2 P S P S P (the paper's conditions P S P = P,
// Tr(P S) = n_occ, Eq. density_matrix_conditions, read in the non-orthogonal basis).  With
// D = P S P - P it is P' = P S P - 2 D S P: two products of the transform's accuracy give P S
// and P S P, and the product with the small D needs only the Newton-Schulz format.  When
// P = Z X Z^T with X a projector and Z^T S Z = I + delta, Tr(P' S) - n_occ is O(delta^2)
// instead of O(delta).  *s_idem = ||P S P - P||_F of the matrix it was given.  Writes the
// result into F_XN (swapped with F_V).
gdm_status metric_cleanup(gdm_handle* h, double* s_idem) {
  const int n = static_cast<int>(h->n);
  const int64_t ld = h->ld;
  cudaStream_t s = h->stream;
  double* P = h->f[F_XN];
  double* S = h->f[F_S];
  double* T = h->f[F_T];    // P S
  double* PSP = h->f[F_U];
  double* D = h->f[F_X2];
  double* Pn = h->f[F_V];
  const int ns_sl = slices_for(h, GDM_PHASE_NEWTON_SCHULZ);
  CK(slice(h, P, &h->sl[SL_B], GDM_PHASE_TRANSFORM));
  // S's slices from the refinement serve when that phase used the transform's format
  Op s_op = {S, &h->sl[SL_S]};
  const Precision& pr = h->phase[GDM_PHASE_REFINE];
  const Precision& pt = h->phase[GDM_PHASE_TRANSFORM];
  if (sliced(h, GDM_PHASE_TRANSFORM) &&
      !(sliced(h, GDM_PHASE_REFINE) && pr.nslice == pt.nslice && pr.bits == pt.bits &&
        h->sl[SL_S].nslice_valid >= pt.nslice && h->sl[SL_S].bits == pt.bits)) {
    CK(slice(h, S, &h->sl[SL_X], GDM_PHASE_TRANSFORM));
    s_op = {S, &h->sl[SL_X]};
  }
  CK(product(h, {P, &h->sl[SL_B]}, s_op, T, nullptr, nullptr, 1.0, 0.0, 0.0, false,
             GDM_PHASE_TRANSFORM, nullptr, true));                   // T = P S
  CK(slice(h, T, &h->sl[SL_A], GDM_PHASE_TRANSFORM));
  CK(product(h, {T, &h->sl[SL_A]}, {P, &h->sl[SL_B]}, PSP, nullptr, nullptr, 1.0, 0.0, 0.0, true,
             GDM_PHASE_TRANSFORM, nullptr, true));                   // P S P (symmetric)
  CK(form_and_slice(PSP, ld, P, ld, n, n, nullptr, 1.0, -1.0, 0.0, D, ld,
                    ns_sl > 0 ? &h->sl[SL_X2] : nullptr, ns_sl, nullptr, s,
                    bits_for(h, GDM_PHASE_NEWTON_SCHULZ), kDotNone, nullptr, true));          // D = P S P - P
  double d2 = 0.0;
  gdm_status st = dot(h, D, nullptr, 0, &d2);
  if (st != GDM_OK) return st;
  *s_idem = std::sqrt(d2);
  CK(slice(h, T, &h->sl[SL_W], GDM_PHASE_NEWTON_SCHULZ));
  // P' = P S P - 2 D (P S)^T = P S P - 2 D S P, symmetric (D S P = P S P S P - P S P)
  CK(product(h, {D, &h->sl[SL_X2]}, {T, &h->sl[SL_W]}, Pn, nullptr, PSP, -2.0, 1.0, 0.0, true,
             GDM_PHASE_NEWTON_SCHULZ));
  std::swap(h->f[F_XN], h->f[F_V]);
  return GDM_OK;
}

// ------------------------------------------------------------------------------------------
// steps 2-5
// ------------------------------------------------------------------------------------------
gdm_status solve_core(gdm_handle* h, gdm_info* info, double* energy_out) {
  const int n = static_cast<int>(h->n);
  const int64_t ld = h->ld;
  cudaStream_t s = h->stream;
  gdm_status st;
  CK(clear_device_flags(h, s));
  if (!h->z_valid) {
    st = compute_z(h, info);
    if (st != GDM_OK) return st;
  }
  if (info) info->z_err = h->z_err;
  const int tr_sl = slices_for(h, GDM_PHASE_TRANSFORM);
  const int pu_sl = slices_for(h, GDM_PHASE_PURIFY);
  Op Z = {h->f[F_Z], &h->sl[SL_Z]}, Zt = {h->f[F_ZT], &h->sl[SL_ZT]};
  double* H = h->f[F_H];

  // H~ = Z^T H Z
  CK(slice(h, H, &h->sl[SL_A], GDM_PHASE_TRANSFORM));
  CK(product(h, Zt, {H, &h->sl[SL_A]}, h->f[F_T], nullptr, nullptr, 1.0, 0.0, 0.0, false,
             GDM_PHASE_TRANSFORM));
  CK(slice(h, h->f[F_T], &h->sl[SL_B], GDM_PHASE_TRANSFORM));
  double* Ht = h->f[F_U];
  CK(product(h, {h->f[F_T], &h->sl[SL_B]}, Zt, Ht, nullptr, nullptr, 1.0, 0.0, 0.0, true,
             GDM_PHASE_TRANSFORM));

  // Spectral bounds of H~ (Eq. ntpoly_scale_hamiltonian takes them "estimated"): Gershgorin's
  // discs always enclose the spectrum but, for a dense H~, span it many times over, and the
  // initial guess then squeezes the gap at n_occ by that factor - more purification steps, and
  // every product's rounding is amplified by the inverse of that gap when it turns the occupied
  // subspace.  The extreme Ritz values of a short Lanczos recurrence estimate the spectrum from
  // inside; widened by 2% of their span (a margin that covers the Ritz values' distance from
  // the extremes for smooth spectra many times over) and clamped to Gershgorin's interval, they
  // give the bounds.  The purification tolerates eigenvalues a little outside [0, 1]
  // (x = 1 + d maps to 1 + (gamma - 4) d^2, x = -d to gamma d^2 - 4 d^3); if it still fails, it
  // restarts from Gershgorin's bounds.
  CK(gershgorin(Ht, ld, n, h->partials, h->small + SM_GERSH_H, s));
  const int lz = (h->bounds_method == GDM_BOUNDS_LANCZOS)
                     ? static_cast<int>(std::min<int64_t>(h->lanczos_steps, n)) : 0;
  if (lz > 0) {
    // T = Z^T H is consumed: its buffer takes the FP32 copy of H~
    CK(lanczos(Ht, ld, n, lz, h->lanczos_ws, h->partials, h->small + SM_LANCZOS, s,
               reinterpret_cast<float*>(h->f[F_T]), ld));
    CK(lanczos_bounds(h->small, lz, SM_GERSH_H, SM_LANCZOS, SM_EST_H, s));
  }
  double sm[SM_EST_H + 3];
  st = read_small(h, 0, SM_EST_H + 3, sm);
  if (st != GDM_OK) return st;
  const double g_lo = sm[SM_GERSH_H], g_hi = sm[SM_GERSH_H + 1];
  if (!std::isfinite(g_lo) || !std::isfinite(g_hi))
    return set_err(h, GDM_ERR_NONFINITE, "non-finite orthogonalised Hamiltonian");
  if (!(g_hi > g_lo)) return set_err(h, GDM_ERR_NO_GAP, "degenerate spectrum bounds");
  const bool use_lanczos = lz > 0 && sm[SM_EST_H + 2] != 0.0;
  const double l_lo = use_lanczos ? sm[SM_EST_H] : g_lo;
  const double l_hi = use_lanczos ? sm[SM_EST_H + 1] : g_hi;
  double* X = h->f[F_X];
  double* X2 = h->f[F_X2];
  double* Xn = h->f[F_XN];
  // truncated purification (gdm_set_truncation): every matrix entering a product is filtered
  TruncArgs trunc_args;
  const TruncArgs* tr = purify_trunc(h, &trunc_args);
  const double tol_abs = h->idem_tol * static_cast<double>(h->n_occ);
  double last_idem = INFINITY;
  int it = 0;
  int stop = 4;
  double* W = h->f[F_V];
  for (int attempt = use_lanczos ? 0 : 1; attempt < 2; ++attempt) {
  const double bh[2] = {attempt == 0 ? l_lo : g_lo, attempt == 0 ? l_hi : g_hi};
  h->host_buf[0] = bh[0];
  h->host_buf[1] = bh[1];
  CK(cudaMemcpyAsync(h->small + SM_BOUNDS_H, h->host_buf, 2 * sizeof(double),
                     cudaMemcpyHostToDevice, s));
  if (info) {
    info->eps_min = bh[0];
    info->eps_max = bh[1];
    info->bounds_restart = attempt == 1 && use_lanczos ? 1 : 0;
  }
  if (h->purify == kPurifyCanonical)
    CK(canonical_x0_coefficients(h->small + SM_BOUNDS_H, Ht, ld, n,
                                 static_cast<double>(h->n_occ), h->small + SM_COEF_X0, s));
  else
    CK(x0_coefficients(h->small + SM_BOUNDS_H, h->small + SM_COEF_X0, s));
  h->kstages_dense = 0.0;
  h->kstages_issued = 0.0;
  if (tr != nullptr)
    CK(cudaMemsetAsync(h->small + SM_KCOUNT, 0, sizeof(unsigned long long), s));
  CK(form_and_slice(Ht, ld, nullptr, 0, n, n, h->small + SM_COEF_X0, 0, 0, 0, X, ld,
                    pu_sl > 0 ? &h->sl[SL_X] : nullptr, pu_sl, nullptr, s,
                    bits_for(h, GDM_PHASE_PURIFY), kDotSelf, tr, true));

  // TRS4
  Trs4State init;
  memset(&init, 0, sizeof(init));
  init.n_occ = static_cast<double>(h->n_occ);
  init.method = h->purify;
  init.idem = INFINITY;
  init.floor_rule = (tr == nullptr) ? 1 : 0;  // a filtered route has its own, higher floor
  CK(cudaMemcpyAsync(h->st_dev, &init, sizeof(init), cudaMemcpyHostToDevice, s));
  h->hist.clear();
  last_idem = INFINITY;
  stop = 4;
  bool failed = false;
  for (it = 0; it < h->max_purif; ++it) {
    CK(product(h, {X, &h->sl[SL_X]}, {X, &h->sl[SL_X]}, X2, nullptr, nullptr, 1.0, 0.0, 0.0, true,
               GDM_PHASE_PURIFY, nullptr, true));
    // with truncation X^2 is filtered (and sliced) before its traces are taken; without it the
    // traces and X^2's slices come from one pass over X and X^2
    int nb = 0;
    bool x2_sliced = false, row_terms = false;
    if (tr != nullptr) {
      CK(slice(h, X2, &h->sl[SL_X2], GDM_PHASE_PURIFY, kDotNone, tr));
      x2_sliced = true;
    } else if (pu_sl > 0 && slice_traces_fits(X2, X, ld, n, &h->sl[SL_X2], pu_sl, true)) {
      // X's slicing pass left ||X_r||^2 in its row dots (self dots of X)
      const SliceBuf& sx = h->sl[SL_X];
      const double* x_dots = (sx.row_dot != nullptr && sx.dot_partner == X) ? sx.row_dot : nullptr;
      CK(slice_traces(X2, X, ld, n, &h->sl[SL_X2], pu_sl, bits_for(h, GDM_PHASE_PURIFY),
                      h->partials, &nb, s, nullptr, true, x_dots));
      x2_sliced = true;
      row_terms = true;
    }
    if (nb == 0) CK(trs4_traces(X, X2, ld, n, h->partials, &nb, s));
    CK(trs4_control(h->partials, nb, h->st_dev, tol_abs, s));
    CK(cudaMemcpyAsync(h->st_host, h->st_dev, sizeof(Trs4State), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const Trs4State& t = *h->st_host;
    h->hist.push_back({t.idem, t.t[0], t.gamma, t.stop != 0 ? -1 : t.branch});
    // a trace outside [0, n] means eigenvalues far outside [0, 1]: the bounds did not enclose
    // the spectrum (only estimated bounds can do that)
    if (attempt == 0 && (t.stop == 3 || !(t.t[0] > -0.5 && t.t[0] < static_cast<double>(n) + 0.5))) {
      failed = true;
      break;
    }
    if (t.stop != 0) {
      stop = t.stop;
      // at the arithmetic's floor a further step only adds rounding: if this iterate is worse
      // than the previous one, return to the previous one (still in Xn)
      if (stop == 2 && it > 0 && std::fabs(t.idem) > std::fabs(t.idem_prev)) {
        std::swap(X, Xn);
        h->hist.back().branch = -2;
        last_idem = t.idem_prev;
      } else {
        last_idem = t.idem;
      }
      break;
    }
    last_idem = t.idem;
    if (t.branch == 4) {  // canonical: X <- X W, W = a X + b X^2 + c I (X's slices are current)
      CK(form_and_slice(X, ld, X2, ld, n, n, st_field(h, offsetof(Trs4State, coefW)), 0, 0, 0,
                        W, ld, pu_sl > 0 ? &h->sl[SL_W] : nullptr, pu_sl, nullptr, s,
                        bits_for(h, GDM_PHASE_PURIFY), kDotX, tr, true));
      CK(product(h, {X, &h->sl[SL_X]}, {W, &h->sl[SL_W]}, Xn, nullptr, nullptr, 1.0, 0.0, 0.0,
                 tr == nullptr, GDM_PHASE_PURIFY, nullptr, true));
      if (tr != nullptr) CK(symmetrise(Xn, ld, n, s));
      CK(slice(h, Xn, &h->sl[SL_X], GDM_PHASE_PURIFY, kDotSelf, tr));
    } else if (t.branch == 2 || t.branch == 3) {  // a product: F + gamma G, or McWeeny
      if (!x2_sliced) CK(slice(h, X2, &h->sl[SL_X2], GDM_PHASE_PURIFY));
      // W itself is needed only with filtering or FP64 products (the sliced product takes its
      // diagonal from the row dot products with X^2)
      const bool need_w = tr != nullptr || pu_sl == 0 || n + (n & 1) > kFusedMaxCols;
      // W's row dot products with X^2 follow from the per-row trace terms when slice_traces
      // produced them (no filtering): a <X_i, X2_i> + b ||X2_i||^2 + c (X2)_ii
      const bool dots_from_traces = row_terms;
      const double* coefW = st_field(h, offsetof(Trs4State, coefW));
      CK(form_and_slice(X, ld, X2, ld, n, n, coefW, 0, 0, 0, need_w ? W : nullptr, ld,
                        pu_sl > 0 ? &h->sl[SL_W] : nullptr, pu_sl, nullptr, s,
                        bits_for(h, GDM_PHASE_PURIFY), dots_from_traces ? kDotNone : kDotX2, tr, true));
      if (dots_from_traces) CK(w_row_dots(h->partials, n, coefW, &h->sl[SL_W], X2, s));
      // with filtering X^2 and W no longer commute: the full product is symmetrised
      CK(product(h, {X2, &h->sl[SL_X2]}, {W, &h->sl[SL_W]}, Xn, nullptr, nullptr, 1.0, 0.0, 0.0,
                 tr == nullptr, GDM_PHASE_PURIFY, nullptr, true));
      if (tr != nullptr) CK(symmetrise(Xn, ld, n, s));
      CK(slice(h, Xn, &h->sl[SL_X], GDM_PHASE_PURIFY, kDotSelf, tr));
    } else {
      CK(form_and_slice(X, ld, X2, ld, n, n, st_field(h, offsetof(Trs4State, coefX)), 0, 0, 0,
                        Xn, ld, pu_sl > 0 ? &h->sl[SL_X] : nullptr, pu_sl, nullptr, s,
                        bits_for(h, GDM_PHASE_PURIFY), kDotSelf, tr, true));
    }
    std::swap(X, Xn);
  }
  if (attempt == 0 && failed) continue;  // again from Gershgorin's bounds
  break;
  }
  h->f[F_X] = X;
  h->f[F_XN] = Xn;
  if (info) {
    info->purif_iters = it;
    info->stop_reason = stop;
    info->idem_err = last_idem;
    info->kstage_fraction = 1.0;
  }
  if (tr != nullptr && h->kstages_dense > 0.0) {
    unsigned long long issued = 0;
    CK(cudaMemcpyAsync(&issued, h->small + SM_KCOUNT, sizeof(issued), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    h->kstages_issued = static_cast<double>(issued);
    if (info) info->kstage_fraction = h->kstages_issued / h->kstages_dense;
  }
  if (stop == 3) return set_err(h, GDM_ERR_NONFINITE, "non-finite traces during purification");

  // Final trace reset (zeroth order): X <- X * N / Tr X.  TRS4 keeps Tr X = N through its
  // gamma steps; the McWeeny endgame does not, and the rounding of the products leaves Tr X off
  // by about the idempotency floor.  The scale factor differs from 1 by that relative amount,
  // so idempotency and the subspace are unchanged to that order.
  {
    CK(trace_scale(X, ld, n, static_cast<double>(h->n_occ), h->small + SM_RED + 4, s));
    double fix = 0.0;
    st = read_small(h, SM_RED + 4, 1, &fix);
    if (st != GDM_OK) return st;
    if (info) info->trace_fix = fix;
  }

  // P = Z X Z^T  (X re-sliced in the transform format)
  CK(slice(h, X, &h->sl[SL_X], GDM_PHASE_TRANSFORM));
  CK(product(h, Z, {X, &h->sl[SL_X]}, h->f[F_T], nullptr, nullptr, 1.0, 0.0, 0.0, false,
             GDM_PHASE_TRANSFORM));
  CK(slice(h, h->f[F_T], &h->sl[SL_A], GDM_PHASE_TRANSFORM));
  double* P = h->f[F_XN];
  // exact diagonal: it carries the electron count Tr(P S) when S is close to I
  CK(product(h, {h->f[F_T], &h->sl[SL_A]}, Z, P, nullptr, nullptr, 1.0, 0.0, 0.0, true,
             GDM_PHASE_TRANSFORM, nullptr, true));
  // Electron count in the S metric.  What can leave it off is Z^T S Z - I (the accuracy to
  // which the products resolve the overlap) and the products of the back-transform: P = Z X Z^T
  // is then a projector in a slightly different metric.  With the exact diagonals above, the
  // count is within a few 1e-9 for well-conditioned overlaps (measured at n = 4362 and 8192)
  // and about 1e-7 at cond(S) = 1e3, n = 4096, where the 38-bit products' resolution of
  // Z^T S Z is the floor.  The optional S-metric McWeeny step restores P S P = P; the scalar
  // rescale P <- P N / Tr(P S) is the last resort above 1e-8 and is reported when it fires.
  double trps = 0.0, e = 0.0;
  st = dot(h, P, h->f[F_S], 0, &trps);
  if (st != GDM_OK) return st;
  const double N = static_cast<double>(h->n_occ);
  if (info) {
    info->trace_err_raw = std::fabs(trps - N);
    info->s_idem_err = -1.0;
    info->metric_cleanup = 0;
    info->trace_rescaled = 0;
  }
  if (h->cleanup_tol >= 0.0 && std::isfinite(trps) && std::fabs(trps - N) > h->cleanup_tol) {
    double s_idem = 0.0;
    st = metric_cleanup(h, &s_idem);
    if (st != GDM_OK) return st;
    P = h->f[F_XN];
    st = dot(h, P, h->f[F_S], 0, &trps);
    if (st != GDM_OK) return st;
    if (info) {
      info->s_idem_err = s_idem;
      info->metric_cleanup = 1;
    }
  }
  if (h->trace_correct && std::isfinite(trps) && trps > 0.0 &&
      std::fabs(trps - N) > h->rescale_tol) {
    CK(form_and_slice(P, ld, nullptr, 0, n, n, nullptr, N / trps, 0.0, 0.0, P, ld, nullptr, 0,
                      nullptr, s, 12, kDotNone, nullptr, true));
    st = dot(h, P, h->f[F_S], 0, &trps);
    if (st != GDM_OK) return st;
    if (info) info->trace_rescaled = 1;
  }
  st = dot(h, P, H, 0, &e);
  if (st != GDM_OK) return st;
  st = check_device_error(h);
  if (st != GDM_OK) return st;
  if (info) {
    info->trace_err = std::fabs(trps - static_cast<double>(h->n_occ));
    info->energy = e;
  }
  if (energy_out) *energy_out = e;
  if (!std::isfinite(e) || !std::isfinite(trps))
    return set_err(h, GDM_ERR_NONFINITE, "non-finite outputs");
  if (stop == 4) return set_err(h, GDM_ERR_NOT_CONVERGED, "purification reached the iteration cap");
  if (h->trace_tol > 0 && std::fabs(trps - static_cast<double>(h->n_occ)) > h->trace_tol)
    return set_err(h, GDM_ERR_NOT_CONVERGED, "|Tr(PS) - N| = %g above tolerance",
                   std::fabs(trps - static_cast<double>(h->n_occ)));
  return GDM_OK;
}

gdm_status ingest(gdm_handle* h, const double* src, int64_t ld_src, gdm_mem mem, double* dst) {
  if (src == nullptr) return set_err(h, GDM_ERR_ARG, "null matrix pointer");
  if (ld_src < h->n) return set_err(h, GDM_ERR_ARG, "leading dimension %lld < n",
                                     static_cast<long long>(ld_src));
  if (mem != GDM_MEM_HOST && mem != GDM_MEM_DEVICE) return set_err(h, GDM_ERR_ARG, "bad mem kind");
  CK(cudaSetDevice(h->device));
  const size_t w = sizeof(double) * static_cast<size_t>(h->n);
  CK(cudaMemcpy2DAsync(dst, sizeof(double) * h->ld, src, sizeof(double) * ld_src, w,
                       static_cast<size_t>(h->n),
                       mem == GDM_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                       h->stream));
  CK(symmetrise(dst, h->ld, static_cast<int>(h->n), h->stream));
  double s2 = 0.0;
  gdm_status st = dot(h, dst, nullptr, 0, &s2);
  if (st != GDM_OK) return st;
  if (!std::isfinite(s2)) return set_err(h, GDM_ERR_NONFINITE, "input matrix has NaN/Inf");
  return GDM_OK;
}

void free_all(gdm_handle* h) {
  for (auto& p : h->prof_pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  h->prof_pending.clear();
  for (auto e : h->ev_pool) cudaEventDestroy(e);
  h->ev_pool.clear();
  if (h->pool) cudaFree(h->pool);
  if (h->host_buf) cudaFreeHost(h->host_buf);
  if (h->st_host) cudaFreeHost(h->st_host);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
  h->pool = nullptr;
}

}  // namespace

namespace {

// Byte layout of a handle's single device allocation for capacity n.
struct PoolLayout {
  size_t fbytes, sdata, sscale, pbytes, lbytes, small_bytes, st_bytes, flag_bytes, split_slots,
      split_bytes, total;
  explicit PoolLayout(int64_t n) {
    auto up = [](size_t x) { return (x + 1023) / 1024 * 1024; };
    const size_t ld = static_cast<size_t>((n + 63) / 64 * 64);
    const size_t rows_alloc = static_cast<size_t>((n + 127) / 128 * 128);
    const size_t tiles = rows_alloc / 128;
    fbytes = up(sizeof(double) * ld * static_cast<size_t>(n));
    sdata = up(sizeof(__half) * 4 * ld * rows_alloc);
    // row scales, row dot products, then the 128 x 128 tile occupancy words
    sscale = up(2 * sizeof(double) * rows_alloc + sizeof(uint32_t) * tiles * tiles);
    pbytes = up(sizeof(double) * (kTraceTerms * static_cast<size_t>(n) + 64));
    // the Lanczos recurrence's vectors (x as two float halves, y, v, v_prev); kept out of the
    // n x n buffers, whose column n must stay zero
    lbytes = up(sizeof(double) * 4 * static_cast<size_t>(n));
    small_bytes = up(sizeof(double) * kSmall);
    st_bytes = up(sizeof(Trs4State));
    // the device error word, then the split-k counters
    flag_bytes = up(sizeof(uint32_t) * (1 + static_cast<size_t>(kSplitTiles) * kEpilogueWarps));
    // split-k partial sums: a part per SM at most, and never more than 4 per tile
    split_slots = std::min<size_t>(kSplitTiles, 4 * tiles * tiles);
    split_bytes = up(sizeof(long long) * 128 * 128 * split_slots);
    total = F_COUNT * fbytes + SL_COUNT * (sdata + sscale) + pbytes + lbytes + small_bytes +
            st_bytes + flag_bytes + split_bytes;
  }
};

}  // namespace

namespace gdm {

size_t handle_pool_bytes(int64_t n) { return PoolLayout(n).total; }

gdm_status handle_reconfigure(gdm_handle* h, int64_t n, int64_t n_occ) {
  if (h == nullptr) return GDM_ERR_ARG;
  if (n < 1 || n > h->n_cap || n_occ <= 0 || n_occ >= n)
    return set_err(h, GDM_ERR_ARG, "problem n=%lld, n_occ=%lld does not fit capacity %lld",
                   static_cast<long long>(n), static_cast<long long>(n_occ),
                   static_cast<long long>(h->n_cap));
  h->n = n;
  h->n_occ = n_occ;
  // the column after the n columns of every buffer must be zero (the paired kernels read it
  // for an odd n); a larger earlier problem left data there
  if (n < h->ld)
    for (int i = 0; i < F_COUNT; ++i)
      if (zero_column(h->f[i], h->ld, static_cast<int>(n), static_cast<int>(n), h->stream) !=
          cudaSuccess)
        return set_err(h, GDM_ERR_CUDA, "zeroing the padding column failed");
  h->have_H = false;
  h->have_S = false;
  h->have_P = false;
  h->z_valid = false;
  for (int i = 0; i < SL_COUNT; ++i) {
    h->sl[i].rows = static_cast<int>(n);
    h->sl[i].cols = static_cast<int>(n);
    h->sl[i].nslice_valid = 0;
    h->sl[i].dot_partner = nullptr;
    h->sl[i].mask_valid = false;
  }
  return GDM_OK;
}

}  // namespace gdm

// ==========================================================================================
// C ABI
// ==========================================================================================
extern "C" {

const char* gdm_status_string(gdm_status s) {
  switch (s) {
    case GDM_OK: return "GDM_OK";
    case GDM_ERR_ARG: return "GDM_ERR_ARG";
    case GDM_ERR_STATE: return "GDM_ERR_STATE";
    case GDM_ERR_NOT_SPD: return "GDM_ERR_NOT_SPD";
    case GDM_ERR_NONFINITE: return "GDM_ERR_NONFINITE";
    case GDM_ERR_NO_GAP: return "GDM_ERR_NO_GAP";
    case GDM_ERR_NOT_CONVERGED: return "GDM_ERR_NOT_CONVERGED";
    case GDM_ERR_OOM: return "GDM_ERR_OOM";
    case GDM_ERR_BUDGET: return "GDM_ERR_BUDGET";
    case GDM_ERR_TIMEOUT: return "GDM_ERR_TIMEOUT";
    case GDM_ERR_CUDA: return "GDM_ERR_CUDA";
  }
  return "GDM_UNKNOWN_STATUS";
}

const char* gdm_last_error(const gdm_handle* h) {
  if (h == nullptr) return "null handle";
  return h->last_error.c_str();
}

gdm_status gdm_init(gdm_handle** out, int64_t n_basis, int64_t n_occ, int device) {
  if (out == nullptr) return GDM_ERR_ARG;
  *out = nullptr;
  if (n_basis < 1 || n_basis > (1 << 16) || n_occ <= 0 || n_occ >= n_basis) return GDM_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return GDM_ERR_ARG;
  gdm_handle* h = new gdm_handle();
  h->device = device;
  h->n = n_basis;
  h->n_cap = n_basis;
  h->n_occ = n_occ;
  h->ld = (n_basis + 63) / 64 * 64;
  h->rows_alloc = static_cast<int>((n_basis + 127) / 128 * 128);
  if (cudaSetDevice(device) != cudaSuccess) {
    delete h;
    return GDM_ERR_CUDA;
  }
  PoolLayout L(n_basis);
  if (cudaMalloc(&h->pool, L.total) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return GDM_ERR_OOM;
  }
  uint8_t* p = static_cast<uint8_t*>(h->pool);
  for (int i = 0; i < F_COUNT; ++i) {
    h->f[i] = reinterpret_cast<double*>(p);
    p += L.fbytes;
  }
  for (int i = 0; i < SL_COUNT; ++i) {
    h->sl[i].data = reinterpret_cast<__half*>(p);
    p += L.sdata;
    h->sl[i].row_scale = reinterpret_cast<double*>(p);
    h->sl[i].row_dot = h->sl[i].row_scale + h->rows_alloc;
    h->sl[i].tile_mask = reinterpret_cast<uint32_t*>(h->sl[i].row_dot + h->rows_alloc);
    h->sl[i].mask_ld = h->rows_alloc / 128;
    p += L.sscale;
    h->sl[i].ld = static_cast<int>(h->ld);
    h->sl[i].rows_alloc = h->rows_alloc;
    h->sl[i].rows = static_cast<int>(n_basis);
    h->sl[i].cols = static_cast<int>(n_basis);
  }
  h->partials = reinterpret_cast<double*>(p);
  p += L.pbytes;
  h->lanczos_ws = reinterpret_cast<double*>(p);
  p += L.lbytes;
  h->small = reinterpret_cast<double*>(p);
  p += L.small_bytes;
  h->st_dev = reinterpret_cast<Trs4State*>(p);
  p += L.st_bytes;
  h->err_dev = reinterpret_cast<uint32_t*>(p);
  h->split_cnt = h->err_dev + 1;
  p += L.flag_bytes;
  h->split_ws = reinterpret_cast<long long*>(p);
  h->split_slots = static_cast<int>(L.split_slots);
  if (cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMallocHost(&h->host_buf, sizeof(double) * kSmall) != cudaSuccess ||
      cudaMallocHost(&h->st_host, sizeof(Trs4State)) != cudaSuccess ||
      cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess) {
    cudaGetLastError();
    free_all(h);
    delete h;
    return GDM_ERR_CUDA;
  }
  h->stream = h->own_stream;
  if (cudaMemsetAsync(h->pool, 0, L.total, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess) {
    free_all(h);
    delete h;
    return GDM_ERR_CUDA;
  }
  *out = h;
  return GDM_OK;
}

static_assert(GDM_PURIFY_TRS4 == kPurifyTrs4 && GDM_PURIFY_TRS2 == kPurifyTrs2 &&
                  GDM_PURIFY_CANONICAL == kPurifyCanonical,
              "purification codes");

gdm_status gdm_set_purification(gdm_handle* h, gdm_purification method) {
  if (h == nullptr) return GDM_ERR_ARG;
  if (method != GDM_PURIFY_TRS4 && method != GDM_PURIFY_TRS2 && method != GDM_PURIFY_CANONICAL)
    return set_err(h, GDM_ERR_ARG, "unknown purification method %d", static_cast<int>(method));
  h->purify = static_cast<int>(method);
  return GDM_OK;
}

gdm_status gdm_set_bounds(gdm_handle* h, gdm_bounds method, int lanczos_steps) {
  if (h == nullptr) return GDM_ERR_ARG;
  if (method != GDM_BOUNDS_GERSHGORIN && method != GDM_BOUNDS_LANCZOS)
    return set_err(h, GDM_ERR_ARG, "unknown bounds method %d", static_cast<int>(method));
  if (lanczos_steps < 0 || lanczos_steps > kMaxLanczos)
    return set_err(h, GDM_ERR_ARG, "lanczos_steps must be 0..%d", kMaxLanczos);
  h->bounds_method = static_cast<int>(method);
  if (lanczos_steps > 0) h->lanczos_steps = lanczos_steps;
  return GDM_OK;
}

gdm_status gdm_set_truncation(gdm_handle* h, double threshold) {
  if (h == nullptr) return GDM_ERR_ARG;
  if (!(threshold >= 0.0) || !std::isfinite(threshold))
    return set_err(h, GDM_ERR_ARG, "truncation threshold must be finite and >= 0");
  h->trunc_tau = threshold;
  return GDM_OK;
}

gdm_status gdm_set_precision(gdm_handle* h, gdm_precision prec) {
  if (h == nullptr) return GDM_ERR_ARG;
  if (prec != GDM_PREC_FP64 && prec != GDM_PREC_MIXED)
    return set_err(h, GDM_ERR_ARG, "unknown precision %d", static_cast<int>(prec));
  if (prec != h->prec) h->z_valid = false;
  h->prec = prec;
  return GDM_OK;
}

gdm_status gdm_set_slices(gdm_handle* h, gdm_phase phase, int nslice, int max_order,
                          int slice_bits) {
  if (h == nullptr) return GDM_ERR_ARG;
  if (phase < GDM_PHASE_NEWTON_SCHULZ || phase > GDM_PHASE_PURIFY)
    return set_err(h, GDM_ERR_ARG, "unknown phase %d", static_cast<int>(phase));
  const bool fp64 = (nslice == 0 && max_order == 0);
  if (!fp64 && (nslice < 1 || nslice > 4 || max_order < 0 || max_order > 3 ||
                max_order > 2 * (nslice - 1)))
    return set_err(h, GDM_ERR_ARG, "invalid slice format (%d, %d)", nslice, max_order);
  if (slice_bits == 0) slice_bits = 12;
  if (slice_bits < 9 || slice_bits > 12)
    return set_err(h, GDM_ERR_ARG, "slice_bits must be 9..12 (or 0 for 12)");
  h->phase[phase] = {nslice, max_order, slice_bits};
  if (phase == GDM_PHASE_NEWTON_SCHULZ || phase == GDM_PHASE_REFINE) h->z_valid = false;
  return GDM_OK;
}

gdm_status gdm_set_tolerance(gdm_handle* h, double idem_tol, double trace_tol) {
  if (h == nullptr) return GDM_ERR_ARG;
  if (!(idem_tol >= 0.0) || !(trace_tol >= 0.0))
    return set_err(h, GDM_ERR_ARG, "tolerances must be >= 0");
  h->idem_tol = idem_tol;
  h->trace_tol = trace_tol;
  return GDM_OK;
}

gdm_status gdm_set_profiling(gdm_handle* h, int enable) {
  if (h == nullptr) return GDM_ERR_ARG;
  h->profiling = (enable != 0);
  return GDM_OK;
}

gdm_status gdm_get_profile_ex(gdm_handle* h, int kind, int64_t* launches, double* ms,
                              double* flops, double* alg_flops_out, int reset) {
  if (h == nullptr || kind < 0 || kind >= gdm_handle::kProfKinds) return GDM_ERR_ARG;
  if (launches) *launches = h->prof_launches[kind];
  if (ms) *ms = h->prof_ms[kind];
  if (flops) *flops = h->prof_flops[kind];
  if (alg_flops_out) *alg_flops_out = h->prof_alg[kind];
  if (reset) {
    h->prof_launches[kind] = 0;
    h->prof_ms[kind] = 0.0;
    h->prof_flops[kind] = 0.0;
    h->prof_alg[kind] = 0.0;
  }
  return GDM_OK;
}

gdm_status gdm_get_profile(gdm_handle* h, int kind, int64_t* launches, double* ms,
                           double* flops, int reset) {
  return gdm_get_profile_ex(h, kind, launches, ms, flops, nullptr, reset);
}

int64_t gdm_launch_count(void) { return launch_count(); }

gdm_status gdm_set_metric_cleanup(gdm_handle* h, double threshold) {
  if (h == nullptr) return GDM_ERR_ARG;
  if (std::isnan(threshold)) return set_err(h, GDM_ERR_ARG, "threshold is NaN");
  h->cleanup_tol = threshold;
  return GDM_OK;
}

gdm_status gdm_set_trace_correction(gdm_handle* h, int enable) {
  if (h == nullptr) return GDM_ERR_ARG;
  h->trace_correct = (enable != 0);
  return GDM_OK;
}

gdm_status gdm_set_max_iter(gdm_handle* h, int ns_max, int purif_max) {
  if (h == nullptr) return GDM_ERR_ARG;
  if (ns_max < 0 || purif_max < 0) return set_err(h, GDM_ERR_ARG, "negative iteration cap");
  if (ns_max > 0) h->max_ns = ns_max;
  if (purif_max > 0) h->max_purif = purif_max;
  return GDM_OK;
}

gdm_status gdm_set_stream(gdm_handle* h, void* stream) {
  if (h == nullptr) return GDM_ERR_ARG;
  h->stream = (stream != nullptr) ? static_cast<cudaStream_t>(stream) : h->own_stream;
  return GDM_OK;
}

gdm_status gdm_set_overlap(gdm_handle* h, const double* S, int64_t ld, gdm_mem mem) {
  if (h == nullptr) return GDM_ERR_ARG;
  h->have_S = false;
  h->have_P = false;
  h->z_valid = false;
  gdm_status st = ingest(h, S, ld, mem, h->f[F_S]);
  if (st == GDM_OK) h->have_S = true;
  return st;
}

gdm_status gdm_set_hamiltonian(gdm_handle* h, const double* H, int64_t ld, gdm_mem mem) {
  if (h == nullptr) return GDM_ERR_ARG;
  h->have_H = false;
  h->have_P = false;
  gdm_status st = ingest(h, H, ld, mem, h->f[F_H]);
  if (st == GDM_OK) h->have_H = true;
  return st;
}

gdm_status gdm_solve_dm(gdm_handle* h, double* P, int64_t ld, gdm_mem mem, double* energy,
                        gdm_info* info) {
  if (h == nullptr) return GDM_ERR_ARG;
  if (!h->have_H || !h->have_S)
    return set_err(h, GDM_ERR_STATE, "set the Hamiltonian and the overlap before solving");
  if (P != nullptr && ld < h->n) return set_err(h, GDM_ERR_ARG, "leading dimension < n");
  if (mem != GDM_MEM_HOST && mem != GDM_MEM_DEVICE) return set_err(h, GDM_ERR_ARG, "bad mem kind");
  CK(cudaSetDevice(h->device));
  gdm_info local;
  memset(&local, 0, sizeof(local));
  CK(cudaEventRecord(h->ev0, h->stream));
  h->have_P = false;
  gdm_status st = solve_core(h, &local, energy);
  CK(cudaEventRecord(h->ev1, h->stream));
  h->have_P = (st == GDM_OK || st == GDM_ERR_NOT_CONVERGED);
  if (P != nullptr && (st == GDM_OK || st == GDM_ERR_NOT_CONVERGED)) {
    CK(cudaMemcpy2DAsync(P, sizeof(double) * ld, h->f[F_XN], sizeof(double) * h->ld,
                         sizeof(double) * h->n, static_cast<size_t>(h->n),
                         mem == GDM_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                         h->stream));
  }
  CK(cudaStreamSynchronize(h->stream));
  collect_profile(h);
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, h->ev0, h->ev1) == cudaSuccess) local.ms_total = ms;
  if (info) *info = local;
  return st;
}

gdm_status gdm_get_edm(gdm_handle* h, double* Q, int64_t ld, gdm_mem mem) {
  if (h == nullptr) return GDM_ERR_ARG;
  if (!h->have_P || !h->have_H)
    return set_err(h, GDM_ERR_STATE, "no density matrix: solve before asking for the EDM");
  if (Q == nullptr) return set_err(h, GDM_ERR_ARG, "null output pointer");
  if (ld < h->n) return set_err(h, GDM_ERR_ARG, "leading dimension < n");
  if (mem != GDM_MEM_HOST && mem != GDM_MEM_DEVICE) return set_err(h, GDM_ERR_ARG, "bad mem kind");
  CK(cudaSetDevice(h->device));
  cudaStream_t s = h->stream;
  CK(clear_device_flags(h, s));
  // Q = P H P: T = P H (H symmetric, so it is its own transposed operand), then Q = T P^T with
  // P symmetric; both products run in the transform phase's format.
  double* P = h->f[F_XN];
  double* H = h->f[F_H];
  double* T = h->f[F_T];
  double* Qd = h->f[F_V];
  CK(slice(h, P, &h->sl[SL_A], GDM_PHASE_TRANSFORM));
  CK(slice(h, H, &h->sl[SL_B], GDM_PHASE_TRANSFORM));
  CK(product(h, {P, &h->sl[SL_A]}, {H, &h->sl[SL_B]}, T, nullptr, nullptr, 1.0, 0.0, 0.0, false,
             GDM_PHASE_TRANSFORM));
  CK(slice(h, T, &h->sl[SL_X], GDM_PHASE_TRANSFORM));
  CK(product(h, {T, &h->sl[SL_X]}, {P, &h->sl[SL_A]}, Qd, nullptr, nullptr, 1.0, 0.0, 0.0, true,
             GDM_PHASE_TRANSFORM, nullptr, true));
  CK(cudaMemcpy2DAsync(Q, sizeof(double) * ld, Qd, sizeof(double) * h->ld,
                       sizeof(double) * h->n, static_cast<size_t>(h->n),
                       mem == GDM_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  collect_profile(h);
  return check_device_error(h);
}

gdm_status gdm_extrapolate_dm(gdm_handle* h, const double* S_new, int64_t lds, gdm_mem mem_s,
                              double* P, int64_t ldp, gdm_mem mem_p) {
  if (h == nullptr) return GDM_ERR_ARG;
  if (!h->have_P) return set_err(h, GDM_ERR_STATE, "no density matrix to extrapolate: solve first");
  if (P == nullptr) return set_err(h, GDM_ERR_ARG, "null output pointer");
  if (ldp < h->n) return set_err(h, GDM_ERR_ARG, "leading dimension < n");
  if (mem_p != GDM_MEM_HOST && mem_p != GDM_MEM_DEVICE)
    return set_err(h, GDM_ERR_ARG, "bad mem kind");
  CK(cudaSetDevice(h->device));
  cudaStream_t s = h->stream;
  const int64_t ld = h->ld;
  CK(clear_device_flags(h, s));
  // X0 = Z0^{-1} P0 Z0^{-T}, the last solve's projector in the orthogonal basis, is still in
  // F_X; keep it in F_H (the Hamiltonian belongs to the old geometry and is dropped)
  CK(cudaMemcpyAsync(h->f[F_H], h->f[F_X], sizeof(double) * ld * h->n, cudaMemcpyDeviceToDevice,
                     s));
  h->have_H = false;
  h->have_P = false;
  h->have_S = false;
  h->z_valid = false;
  gdm_status st = ingest(h, S_new, lds, mem_s, h->f[F_S]);
  if (st != GDM_OK) return st;
  h->have_S = true;
  st = compute_z(h, nullptr);  // Z1 for the new overlap, cached for the next solve
  if (st != GDM_OK) return st;
  // P1 = Z1 X0 Z1^T (the back-transform of the solve, applied to X0)
  double* X0 = h->f[F_H];
  Op Z = {h->f[F_Z], &h->sl[SL_Z]};
  CK(slice(h, X0, &h->sl[SL_X], GDM_PHASE_TRANSFORM));
  CK(product(h, Z, {X0, &h->sl[SL_X]}, h->f[F_T], nullptr, nullptr, 1.0, 0.0, 0.0, false,
             GDM_PHASE_TRANSFORM));
  CK(slice(h, h->f[F_T], &h->sl[SL_A], GDM_PHASE_TRANSFORM));
  double* P1 = h->f[F_XN];
  CK(product(h, {h->f[F_T], &h->sl[SL_A]}, Z, P1, nullptr, nullptr, 1.0, 0.0, 0.0, true,
             GDM_PHASE_TRANSFORM, nullptr, true));
  CK(cudaMemcpy2DAsync(P, sizeof(double) * ldp, P1, sizeof(double) * ld, sizeof(double) * h->n,
                       static_cast<size_t>(h->n),
                       mem_p == GDM_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                       s));
  CK(cudaStreamSynchronize(s));
  collect_profile(h);
  return check_device_error(h);
}

int gdm_get_history(const gdm_handle* h, int max_rows, double* idem, double* trace, double* gamma,
                    int* branch) {
  if (h == nullptr) return 0;
  const int n = static_cast<int>(h->hist.size());
  const int m = n < max_rows ? n : max_rows;
  for (int i = 0; i < m; ++i) {
    if (idem) idem[i] = h->hist[i].idem;
    if (trace) trace[i] = h->hist[i].trace;
    if (gamma) gamma[i] = h->hist[i].gamma;
    if (branch) branch[i] = h->hist[i].branch;
  }
  return n;
}

gdm_status gdm_reinit(gdm_handle* h) {
  if (h == nullptr) return GDM_ERR_ARG;
  h->have_H = false;
  h->have_S = false;
  h->have_P = false;
  h->z_valid = false;
  return GDM_OK;
}

gdm_status gdm_finalize(gdm_handle* h) {
  if (h == nullptr) return GDM_OK;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  free_all(h);
  delete h;
  return GDM_OK;
}

}  // extern "C"
