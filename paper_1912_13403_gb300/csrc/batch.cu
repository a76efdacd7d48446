// Lockstep batches: many independent problems (the paper's spin / k-point "unit tasks", Sec. 2.4,
// solved fully in parallel) advance together through the route, and every matrix product step
// of all problems is ONE persistent grouped launch of the sliced tensor-core kernel over a device
// table of products (gemm_sliced.cu, sliced_gemm_grouped): the CTAs walk the 128 x 128 tiles of
// every problem's product, so small problems (10-300 tiles each) fill the 152 SMs together.
//
// Control lives on the device.  Each problem keeps its own flags (BatchCtl, Trs4State) that its
// control kernels set from its reductions - Newton-Schulz converged or diverged, refinement
// done, the TRS4 branch, stop - and every kernel that could overwrite a finished problem's
// result reads a skip flag.  The phases are captured once per batch shape as CUDA graphs:
//   pre   S's bounds (Gershgorin, Lanczos), the scale c, Y_0 = S / c, Z_0 = I, slices
//   ns    two unrolled Newton-Schulz iterations (buffers alternate by iteration parity)
//   rf    the Z refinement (unrolled: three evaluations of Z^T S Z - I, two updates), H~,
//         spectral bounds (Gershgorin + Lanczos + bisection on the device), X_0
//   pu    two unrolled TRS4 iterations
//   post  the final iterate's buffer, trace reset, back-transform, count, energy
// The host replays ns and pu until every problem's flag says done, reading the flags once per
// two replays (four iterations): no host synchronisation per iteration.  A problem that fails in
// the lockstep (Newton-Schulz diverged, estimated bounds too tight, iteration cap) is solved again
// alone by the single-problem engine afterwards.
//
// The grouped kernel's (k tile, stage count) variant for each slice format is chosen by timing
// the variants on the batch's own largest product (autotune), and remembered in a small JSON file
// keyed by GPU name, slice format and the launch's size class.
#include <sys/stat.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/gdm.h"
#include "gdm_internal.h"
#include "handle.h"

namespace gdm {

// Per-problem control state of a lockstep batch (device, in the handle's small[] at SM_BATCH).
struct BatchCtl {
  int ns_off;      // Newton-Schulz finished: skip its work
  int ns_iters;
  int ns_parity;   // parity of the iteration whose Y, Z are final
  int ns_failed;   // diverged
  int rf_off;      // refinement finished
  int rf_final;    // evaluation (0, 1, 2) whose Z is final
  int rf_steps;    // refinement updates taken
  int rf_failed;
  int rescaled;    // the last-resort count rescale fired
  int pad_;
  double ns_prev, rf_prev, rf_derr, count_raw, factor;
  double ns_l;       // lower end of M's spectrum for the scaled Newton-Schulz steps
  double ns_coef[3]; // T = coef[0] M + coef[2] I of this step
};
static_assert(sizeof(BatchCtl) <= 512, "BatchCtl fits the small[] tail");

namespace {

constexpr int kSideStreams = 16;
constexpr int kNref = 2;         // refinement updates at most (as the single engine)
constexpr int kLanczosSteps = 24;
constexpr int kLanczosS = 16;  // as the single engine (engine.cu)

__global__ void batch_init_kernel(BatchCtl* c, Trs4State* st, double n_occ, int n, int max_purif) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  memset(c, 0, sizeof(BatchCtl));
  c->ns_prev = INFINITY;
  c->rf_prev = INFINITY;
  memset(st, 0, sizeof(Trs4State));
  st->n_occ = n_occ;
  st->method = kPurifyTrs4;
  st->idem = INFINITY;
  st->max_iter = max_purif;
  st->check_trace = 1;
  st->floor_rule = 1;
  st->n = static_cast<double>(n);
}

// The single engine's Newton-Schulz eigenvalue map and step scale (engine.cu, compute_z).
__device__ double ns_g_dev(double x) { return x * (3.0 - x) * (3.0 - x) * 0.25; }
__device__ double ns_alpha_dev(int it, double l) {
  if (it == 0 || !(l > 0.0) || l >= 0.3) return 1.0;
  const double r = sqrt(l);
  return fmin(2.9, 3.0 / (1.0 + r + l));
}

// The scale c of S (1.05 x the largest Ritz value, at most Gershgorin's bound) into
// small[SM_BOUNDS_S + 1], and the lower end l = smallest Ritz value / c of the first step.
__global__ void ns_init_kernel(double* small, BatchCtl* c) {
  const double g_hi = small[SM_BOUNDS_S + 1];
  const double rmin = small[SM_EST_S + 3], rmax = small[SM_EST_S + 4];
  const double sc = (rmax > 0.0 && isfinite(rmax)) ? fmin(g_hi, 1.05 * rmax) : g_hi;
  small[SM_BOUNDS_S + 1] = sc;
  c->ns_l = (rmin > 0.0 && isfinite(rmin)) ? fmin(1.0, rmin / sc) : 1.0;
}

// After M = Y Z and ||I - M||_F^2 in *red: the single engine's stopping rules (hand over at
// ||I - M||_F <= handoff, the rounding floor, or a stall below 1e-2 sqrt n; divergence), then
// the coefficients of this step's T = sqrt(alpha) (3I - alpha M)/2.
__global__ void ns_control_kernel(BatchCtl* c, const double* red, double rn, double handoff,
                                  int parity, int max_ns) {
  if (c->ns_off) return;
  const double res = sqrt(*red);
  if (!isfinite(res) || res > 1e6 * rn) {
    c->ns_failed = 1;
    c->ns_off = 1;
    c->ns_parity = parity;
    return;
  }
  if (res <= handoff || res <= 1e-13 * rn || (res < 1e-2 * rn && res > 0.5 * c->ns_prev) ||
      c->ns_iters >= max_ns) {
    c->ns_off = 1;
    c->ns_parity = parity;
    return;
  }
  c->ns_prev = res;
  const double alpha = ns_alpha_dev(c->ns_iters, c->ns_l);
  c->ns_l = ns_g_dev(alpha * c->ns_l);
  c->ns_coef[0] = -0.5 * alpha * sqrt(alpha);
  c->ns_coef[1] = 0.0;
  c->ns_coef[2] = 1.5 * sqrt(alpha);
  c->ns_iters += 1;
}

// After delta = Z_r^T S Z_r - I and ||delta||_F^2 in *red, at evaluation r.
__global__ void rf_control_kernel(BatchCtl* c, const double* red, int r, int nref) {
  if (c->rf_off) return;
  const double derr = sqrt(*red);
  c->rf_derr = derr;
  if (!isfinite(derr)) {
    c->rf_failed = 1;
    c->rf_off = 1;
    c->rf_final = r;
    return;
  }
  // (the single engine's rules: the last evaluation, delta = 0, or the rounding floor reached,
  // i.e. the third-order prediction (5/8) prev^3 at or below what was measured)
  if (r == nref || derr == 0.0 ||
      (isfinite(c->rf_prev) && 0.625 * c->rf_prev * c->rf_prev * c->rf_prev <= derr)) {
    c->rf_off = 1;
    c->rf_final = r;
    return;
  }
  c->rf_prev = derr;
  c->rf_steps = r + 1;
}

// dst <- src (n x n, leading dimension ld) when *flag == want.
__global__ void copy_if_kernel(double* dst, const double* src, int64_t ld, int n, const int* flag,
                               int want) {
  if (*flag != want) return;
  const int row = blockIdx.x;
  for (int j = threadIdx.x; j < n; j += blockDim.x) dst[row * ld + j] = src[row * ld + j];
}

// The count Tr(P S) in *count: factor = n_occ / count when it is off by more than tol (the
// last-resort rescale), else 1.
__global__ void count_factor_kernel(BatchCtl* c, const double* count, double n_occ, double tol) {
  const double t = *count;
  c->count_raw = t;
  const bool fix = isfinite(t) && t > 0.0 && fabs(t - n_occ) > tol;
  c->factor = fix ? n_occ / t : 1.0;
  c->rescaled = fix ? 1 : 0;
}

__global__ void scale_if_kernel(double* P, int64_t ld, int n, const BatchCtl* c) {
  if (!c->rescaled) return;
  const double f = c->factor;
  const int row = blockIdx.x;
  for (int j = threadIdx.x; j < n; j += blockDim.x) P[row * ld + j] *= f;
}

// out[i] = *flags[i]: the host reads every problem's flag with one copy.
__global__ void gather_flags_kernel(const int* const* flags, int count, int* out) {
  for (int i = threadIdx.x; i < count; i += blockDim.x) out[i] = *flags[i];
}

// ------------------------------------------------------------------------------------------
// autotune cache: {"<gpu>|s<nslice>|u<size class>": variant, ...}
// ------------------------------------------------------------------------------------------
std::map<std::string, int> g_tune;
bool g_tune_loaded = false;

std::string tune_path() {
  const char* p = getenv("GDM_AUTOTUNE_CACHE");
  if (p != nullptr && p[0] != 0) return p;
  const char* home = getenv("HOME");
  return std::string(home ? home : "/tmp") + "/.cache/gdm_autotune.json";
}

void tune_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  FILE* f = fopen(tune_path().c_str(), "r");
  if (f == nullptr) return;
  std::string text;
  char buf[4096];
  size_t got;
  while ((got = fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, got);
  fclose(f);
  size_t pos = 0;
  while ((pos = text.find('"', pos)) != std::string::npos) {
    const size_t end = text.find('"', pos + 1);
    if (end == std::string::npos) break;
    const std::string key = text.substr(pos + 1, end - pos - 1);
    const size_t colon = text.find(':', end);
    if (colon == std::string::npos) break;
    g_tune[key] = atoi(text.c_str() + colon + 1);
    pos = colon + 1;
  }
}

void tune_store() {
  const std::string path = tune_path();
  const size_t slash = path.rfind('/');
  if (slash != std::string::npos) mkdir(path.substr(0, slash).c_str(), 0755);  // may exist
  FILE* f = fopen(path.c_str(), "w");
  if (f == nullptr) return;  // no writable cache: the choices stay in memory
  fprintf(f, "{");
  bool first = true;
  for (const auto& kv : g_tune) {
    fprintf(f, "%s\n  \"%s\": %d", first ? "" : ",", kv.first.c_str(), kv.second);
    first = false;
  }
  fprintf(f, "\n}\n");
  fclose(f);
}

std::string gpu_name(int device) {
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return "unknown";
  std::string s = prop.name;
  for (char& ch : s)
    if (ch == '"' || ch == '|') ch = '_';
  return s;
}

// ------------------------------------------------------------------------------------------
// the executor
// ------------------------------------------------------------------------------------------
struct Site {
  Precision prec;
  int units = 0;
  GroupItem* dev[2] = {nullptr, nullptr};  // the table for each (k tile, stages) variant
  std::vector<GroupItem> host[2];
};

struct BatchExec {
  int device = 0;
  std::vector<int64_t> n, nocc;
  std::vector<gdm_handle*> h;
  cudaStream_t main = nullptr;
  cudaStream_t side[kSideStreams] = {};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[kSideStreams] = {};
  std::vector<Site> sites;
  int site_cursor = 0;
  bool planning = false;
  int variant[5] = {0, 0, 0, 0, 0};
  uint32_t* err_dev = nullptr;
  const int** ns_flags_dev = nullptr;
  const int** pu_flags_dev = nullptr;
  int* flags_dev = nullptr;
  int* flags_host = nullptr;
  cudaGraphExec_t g[5] = {};
  int g_kernels[5] = {};  // kernel nodes of each graph (the library's launch count per replay)
  cudaError_t first_error = cudaSuccess;
  std::string error;

  ~BatchExec() {
    if (main) cudaStreamSynchronize(main);
    for (auto& e : g)
      if (e) cudaGraphExecDestroy(e);
    for (auto& s : sites)
      for (auto& d : s.dev)
        if (d) cudaFree(d);
    if (err_dev) cudaFree(err_dev);
    if (ns_flags_dev) cudaFree(ns_flags_dev);
    if (pu_flags_dev) cudaFree(pu_flags_dev);
    if (flags_dev) cudaFree(flags_dev);
    if (flags_host) cudaFreeHost(flags_host);
    if (ev_fork) cudaEventDestroy(ev_fork);
    for (auto& e : ev_join)
      if (e) cudaEventDestroy(e);
    for (auto& s : side)
      if (s) cudaStreamDestroy(s);
    if (main) cudaStreamDestroy(main);
    for (auto* x : h) gdm_finalize(x);
  }

  void note(cudaError_t e, const char* what) {
    if (e != cudaSuccess && first_error == cudaSuccess) {
      first_error = e;
      error = std::string(what) + ": " + cudaGetErrorString(e);
    }
  }

  int count() const { return static_cast<int>(h.size()); }
  // Whether problem p's slicing passes write the exact row dot products (the one-pass kernels,
  // over the zero column after an odd n, up to kFusedMaxCols); otherwise its exact diagonals are recomputed after the
  // grouped product, as the single engine does when a slicing pass had no dot partner.
  bool rowdots(int p) const { return h[p]->n + (h[p]->n & 1) <= kFusedMaxCols; }
  BatchCtl* ctl(int p) const { return reinterpret_cast<BatchCtl*>(h[p]->small + SM_BATCH); }

  // per-problem work of a phase on the side streams, joined back into the main stream
  template <class F>
  void per_problem(F&& fn) {
    if (planning) return;
    note(cudaEventRecord(ev_fork, main), "record fork");
    for (int i = 0; i < kSideStreams; ++i) note(cudaStreamWaitEvent(side[i], ev_fork, 0), "wait fork");
    for (int p = 0; p < count(); ++p) note(fn(p, side[p % kSideStreams]), "per-problem kernel");
    for (int i = 0; i < kSideStreams; ++i) {
      note(cudaEventRecord(ev_join[i], side[i]), "record join");
      note(cudaStreamWaitEvent(main, ev_join[i], 0), "wait join");
    }
  }

  // One grouped launch: in the planning pass, the table entry of every problem (operands, output
  // and epilogue as `make(p, args)` describes them, for each variant's k tile); in the capture
  // pass, the launch of the chosen variant's table.
  template <class F>
  void grouped(int ph, F&& make, const Precision* fmt = nullptr) {
    const int idx = site_cursor++;
    if (planning) {
      Site s;
      s.prec = fmt != nullptr ? *fmt : h[0]->phase[ph];
      for (int v = 0; v < grouped_variant_count(s.prec.nslice); ++v) {
        const int bk = grouped_variant_bk(s.prec.nslice, v);
        s.host[v].resize(count());
        for (int p = 0; p < count(); ++p) {
          const SliceBuf* A = nullptr;
          const SliceBuf* Bt = nullptr;
          SlicedGemmArgs a;
          make(p, a, A, Bt);
          SliceBuf sa = *A, sb = *Bt;  // the slices exist once the batch runs: describe them
          sa.bits = sb.bits = s.prec.bits;
          note(sliced_gemm_group_item(sa, sb, s.prec, a, &s.host[v][p], bk), "group item");
        }
        s.units = group_assign_units(s.host[v].data(), count());
      }
      sites.push_back(std::move(s));
      return;
    }
    Site& s = sites[idx];
    const int v = variant[s.prec.nslice] < grouped_variant_count(s.prec.nslice)
                      ? variant[s.prec.nslice] : 0;
    note(sliced_gemm_grouped(s.dev[v], count(), s.units, s.prec, err_dev, main, v),
         "grouped product");
  }

  // slicing/forming of problem p on stream st in the format of phase ph
  cudaError_t fas(int p, cudaStream_t st, const double* X, const double* X2, const double* coef,
                  double ha, double hb, double hc, double* Y, SliceBuf* out, int ph,
                  const int* skip, int dot = kDotNone) {
    gdm_handle* q = h[p];
    const int n = static_cast<int>(q->n);
    return form_and_slice(X, q->ld, X2, q->ld, n, n, coef, ha, hb, hc, Y, q->ld, out,
                          out ? q->phase[ph].nslice : 0, skip, st, q->phase[ph].bits, dot,
                          nullptr, true);
  }

  // ---- the phases ----------------------------------------------------------------------------
  void phase_pre() {
    per_problem([&](int p, cudaStream_t st) -> cudaError_t {
      gdm_handle* q = h[p];
      const int n = static_cast<int>(q->n);
      cudaError_t e;
      batch_init_kernel<<<1, 1, 0, st>>>(ctl(p), q->st_dev, static_cast<double>(q->n_occ), n,
                                         q->max_purif);
      count_launch();
      double* bounds = q->small + SM_BOUNDS_S;
      if ((e = gershgorin(q->f[F_S], q->ld, n, q->partials, bounds, st)) != cudaSuccess) return e;
      const int lzs = std::min(kLanczosS, n);
      if ((e = lanczos(q->f[F_S], q->ld, n, lzs, q->lanczos_ws, q->partials, q->small + SM_LANCZOS,
                       st)) != cudaSuccess)
        return e;
      if ((e = lanczos_bounds(q->small, lzs, SM_BOUNDS_S, SM_LANCZOS, SM_EST_S, st)) !=
          cudaSuccess)
        return e;
      ns_init_kernel<<<1, 1, 0, st>>>(q->small, ctl(p));
      count_launch();
      if ((e = scale_coefficients(bounds, 0, q->small + SM_COEF_A, st)) != cudaSuccess) return e;
      if ((e = scale_coefficients(bounds, 1, q->small + SM_COEF_B, st)) != cudaSuccess) return e;
      if ((e = fas(p, st, q->f[F_S], nullptr, q->small + SM_COEF_A, 0, 0, 0, q->f[F_X],
                   &q->sl[SL_X], GDM_PHASE_NEWTON_SCHULZ, nullptr)) != cudaSuccess)
        return e;
      if ((e = set_identity(q->f[F_XN], q->ld, n, st)) != cudaSuccess) return e;
      return fas(p, st, q->f[F_XN], nullptr, nullptr, 1.0, 0, 0, nullptr, &q->sl[SL_Z],
                 GDM_PHASE_NEWTON_SCHULZ, nullptr);
    });
  }

  // Newton-Schulz iteration of parity `par`: (Y, Z) in (X, XN) for even, (X2, V) for odd.
  void phase_ns_iteration(int par) {
    const int Yb = par ? F_X2 : F_X, Zb = par ? F_V : F_XN;
    const int Ynb = par ? F_X : F_X2, Znb = par ? F_XN : F_V;
    grouped(GDM_PHASE_NEWTON_SCHULZ, [&](int p, SlicedGemmArgs& a, const SliceBuf*& A,
                                         const SliceBuf*& B) {
      gdm_handle* q = h[p];
      A = &q->sl[SL_X];
      B = &q->sl[SL_Z];
      a.C = q->f[F_T];
      a.ldc = q->ld;
      a.Ct = q->f[F_U];
      a.ldct = q->ld;
      a.skip = &ctl(p)->ns_off;
    });
    per_problem([&](int p, cudaStream_t st) -> cudaError_t {
      gdm_handle* q = h[p];
      const int n = static_cast<int>(q->n);
      int nb = 0;
      cudaError_t e = dot_partials(q->f[F_T], q->ld, nullptr, q->ld, n, n, 1, q->partials, &nb, st,
                                   &ctl(p)->ns_off, true);
      if (e != cudaSuccess) return e;
      if ((e = reduce_partials(q->partials, nb, 1, q->small + SM_RED, st)) != cudaSuccess) return e;
      const double handoff = (q->n_refine >= 1) ? 0.005 : 0.0;  // as the single engine
      ns_control_kernel<<<1, 1, 0, st>>>(ctl(p), q->small + SM_RED, std::sqrt(double(n)), handoff,
                                         par, q->max_ns);
      count_launch();
      const int* skip = &ctl(p)->ns_off;
      const double* coef = &ctl(p)->ns_coef[0];
      if ((e = fas(p, st, q->f[F_T], nullptr, coef, 0, 0, 0, q->f[F_T], &q->sl[SL_A],
                   GDM_PHASE_NEWTON_SCHULZ, skip)) != cudaSuccess)
        return e;
      return fas(p, st, q->f[F_U], nullptr, coef, 0, 0, 0, q->f[F_U], &q->sl[SL_B],
                 GDM_PHASE_NEWTON_SCHULZ, skip);
    });
    grouped(GDM_PHASE_NEWTON_SCHULZ, [&](int p, SlicedGemmArgs& a, const SliceBuf*& A,
                                         const SliceBuf*& B) {
      gdm_handle* q = h[p];
      A = &q->sl[SL_A];
      B = &q->sl[SL_X];
      a.mode = kGemmSym;
      a.C = q->f[Ynb];
      a.ldc = q->ld;
      a.skip = &ctl(p)->ns_off;
    });
    grouped(GDM_PHASE_NEWTON_SCHULZ, [&](int p, SlicedGemmArgs& a, const SliceBuf*& A,
                                         const SliceBuf*& B) {
      gdm_handle* q = h[p];
      A = &q->sl[SL_B];
      B = &q->sl[SL_Z];
      a.mode = kGemmSym;
      a.C = q->f[Znb];
      a.ldc = q->ld;
      a.skip = &ctl(p)->ns_off;
    });
    per_problem([&](int p, cudaStream_t st) -> cudaError_t {
      gdm_handle* q = h[p];
      const int* skip = &ctl(p)->ns_off;
      cudaError_t e = fas(p, st, q->f[Ynb], nullptr, nullptr, 1.0, 0, 0, nullptr, &q->sl[SL_X],
                          GDM_PHASE_NEWTON_SCHULZ, skip);
      if (e != cudaSuccess) return e;
      return fas(p, st, q->f[Znb], nullptr, nullptr, 1.0, 0, 0, nullptr, &q->sl[SL_Z],
                 GDM_PHASE_NEWTON_SCHULZ, skip);
    });
    (void)Yb;
    (void)Zb;
  }

  // Evaluation r of the refinement on Z_r (FP64 zf / zt, slices zs / zts), then (r < kNref)
  // the update Z_{r+1} = Z_r F into (nz, nzt).
  void refine_step(int r, int zf, int ztf, int nzf, int nztf) {
    (void)zf;  // Z_r enters through its slices and, transposed, through ztf
    // T = Z^T S (exact diagonal), delta = T Z - I (exact diagonal)
    const int zs = (r == 0) ? SL_Z : SL_ZT;  // Z^T's slices (Z_0 is symmetric)
    grouped(GDM_PHASE_REFINE, [&](int p, SlicedGemmArgs& a, const SliceBuf*& A,
                                  const SliceBuf*& B) {
      gdm_handle* q = h[p];
      A = &q->sl[zs];
      B = &q->sl[SL_S];
      a.C = q->f[F_T];
      a.ldc = q->ld;
      a.skip = &ctl(p)->rf_off;
    });
    per_problem([&](int p, cudaStream_t st) -> cudaError_t {
      gdm_handle* q = h[p];
      const int n = static_cast<int>(q->n);
      cudaError_t e = diag_fix(q->f[ztf], q->ld, q->f[F_S], q->ld, q->f[F_T], q->ld, n, n, 1.0,
                               0.0, nullptr, 0, 0.0, nullptr, st, &ctl(p)->rf_off);
      if (e != cudaSuccess) return e;
      return fas(p, st, q->f[F_T], nullptr, nullptr, 1.0, 0, 0, nullptr, &q->sl[SL_A],
                 GDM_PHASE_REFINE, &ctl(p)->rf_off);
    });
    grouped(GDM_PHASE_REFINE, [&](int p, SlicedGemmArgs& a, const SliceBuf*& A,
                                  const SliceBuf*& B) {
      gdm_handle* q = h[p];
      A = &q->sl[SL_A];
      B = &q->sl[zs];
      a.mode = kGemmSym;
      a.diag = -1.0;
      a.C = q->f[F_U];
      a.ldc = q->ld;
      a.skip = &ctl(p)->rf_off;
    });
    per_problem([&](int p, cudaStream_t st) -> cudaError_t {
      gdm_handle* q = h[p];
      const int n = static_cast<int>(q->n);
      cudaError_t e = diag_fix(q->f[F_T], q->ld, q->f[ztf], q->ld, q->f[F_U], q->ld, n, n, 1.0,
                               0.0, nullptr, 0, -1.0, nullptr, st, &ctl(p)->rf_off);
      if (e != cudaSuccess) return e;
      int nb = 0;
      if ((e = dot_partials(q->f[F_U], q->ld, nullptr, q->ld, n, n, 0, q->partials, &nb, st,
                            &ctl(p)->rf_off, true)) != cudaSuccess)
        return e;
      if ((e = reduce_partials(q->partials, nb, 1, q->small + SM_RED, st)) != cudaSuccess) return e;
      rf_control_kernel<<<1, 1, 0, st>>>(ctl(p), q->small + SM_RED, r, kNref);
      count_launch();
      if (r == kNref) return cudaSuccess;
      // delta's slices with its row dot products (the F product's exact diagonal)
      return fas(p, st, q->f[F_U], nullptr, nullptr, 1.0, 0, 0, nullptr, &q->sl[SL_B],
                 GDM_PHASE_REFINE, &ctl(p)->rf_off, kDotSelf);
    });
    if (r == kNref) return;
    // the update as Z + Z G, G = -delta/2 + 3 delta^2/8, with the single engine's short
    // formats for the two products with a small factor (engine.cu, compute_z)
    const Precision& rp = h[0]->phase[GDM_PHASE_REFINE];
    const int sq_ns = std::min(rp.nslice, 2), zg_ns = std::min(rp.nslice, 3);
    const Precision sq_fmt{sq_ns, std::min(1, 2 * (sq_ns - 1)), rp.bits};
    const Precision zg_fmt{zg_ns, std::min(2, 2 * (zg_ns - 1)), rp.bits};
    grouped(GDM_PHASE_REFINE, [&](int p, SlicedGemmArgs& a, const SliceBuf*& A,
                                  const SliceBuf*& B) {
      gdm_handle* q = h[p];
      A = &q->sl[SL_B];
      B = &q->sl[SL_B];
      a.mode = kGemmSym;
      a.C = q->f[F_V];
      a.ldc = q->ld;
      a.D = q->f[F_U];
      a.ldd = q->ld;
      a.alpha = 0.375;
      a.beta = -0.5;
      a.diag = 0.0;
      a.diag_dot = rowdots(p) ? q->sl[SL_B].row_dot : nullptr;
      a.skip = &ctl(p)->rf_off;
    }, &sq_fmt);
    per_problem([&](int p, cudaStream_t st) -> cudaError_t {
      gdm_handle* q = h[p];
      const int n = static_cast<int>(q->n);
      if (!rowdots(p)) {
        cudaError_t e = diag_fix(q->f[F_U], q->ld, q->f[F_U], q->ld, q->f[F_V], q->ld, n, n, 0.375,
                                 -0.5, q->f[F_U], q->ld, 0.0, nullptr, st, &ctl(p)->rf_off);
        if (e != cudaSuccess) return e;
      }
      return fas(p, st, q->f[F_V], nullptr, nullptr, 1.0, 0, 0, nullptr, &q->sl[SL_A],
                 GDM_PHASE_REFINE, &ctl(p)->rf_off);
    });
    grouped(GDM_PHASE_REFINE, [&](int p, SlicedGemmArgs& a, const SliceBuf*& A,
                                  const SliceBuf*& B) {
      gdm_handle* q = h[p];
      A = &q->sl[SL_Z];
      B = &q->sl[SL_A];
      a.C = q->f[nzf];
      a.ldc = q->ld;
      a.Ct = q->f[nztf];
      a.ldct = q->ld;
      a.D = q->f[ztf];  // read transposed: Z itself
      a.ldd = q->ld;
      a.beta = 1.0;
      a.skip = &ctl(p)->rf_off;
    }, &zg_fmt);
    per_problem([&](int p, cudaStream_t st) -> cudaError_t {
      gdm_handle* q = h[p];
      const int* skip = &ctl(p)->rf_off;
      cudaError_t e;
      if ((e = fas(p, st, q->f[nzf], nullptr, nullptr, 1.0, 0, 0, nullptr, &q->sl[SL_Z],
                   GDM_PHASE_REFINE, skip)) != cudaSuccess)
        return e;
      return fas(p, st, q->f[nztf], nullptr, nullptr, 1.0, 0, 0, nullptr, &q->sl[SL_ZT],
                 GDM_PHASE_REFINE, skip);
    });
  }

  void phase_rf() {
    // Z_0' = Z_k / sqrt(c) from the buffer of the final Newton-Schulz parity; S's slices
    per_problem([&](int p, cudaStream_t st) -> cudaError_t {
      gdm_handle* q = h[p];
      const int n = static_cast<int>(q->n);
      copy_if_kernel<<<n, 256, 0, st>>>(q->f[F_XN], q->f[F_V], q->ld, n, &ctl(p)->ns_parity, 1);
      count_launch();
      cudaError_t e = fas(p, st, q->f[F_XN], nullptr, q->small + SM_COEF_B, 0, 0, 0, q->f[F_Z],
                          &q->sl[SL_Z], GDM_PHASE_REFINE, nullptr);
      if (e != cudaSuccess) return e;
      return fas(p, st, q->f[F_S], nullptr, nullptr, 1.0, 0, 0, nullptr, &q->sl[SL_S],
                 GDM_PHASE_REFINE, nullptr);
    });
    // evaluations on Z_0 (Z, Z), Z_1 (X, X2), Z_2 (Z, ZT); updates into the other pair
    refine_step(0, F_Z, F_Z, F_X, F_X2);
    refine_step(1, F_X, F_X2, F_Z, F_ZT);
    refine_step(2, F_Z, F_ZT, F_X, F_X2);
    // the final Z into (Z, ZT), then Z and Z^T in the transform's format; H's slices
    per_problem([&](int p, cudaStream_t st) -> cudaError_t {
      gdm_handle* q = h[p];
      const int n = static_cast<int>(q->n);
      const int* fin = &ctl(p)->rf_final;
      copy_if_kernel<<<n, 256, 0, st>>>(q->f[F_ZT], q->f[F_Z], q->ld, n, fin, 0);
      copy_if_kernel<<<n, 256, 0, st>>>(q->f[F_Z], q->f[F_X], q->ld, n, fin, 1);
      copy_if_kernel<<<n, 256, 0, st>>>(q->f[F_ZT], q->f[F_X2], q->ld, n, fin, 1);
      count_launch(3);
      cudaError_t e = fas(p, st, q->f[F_Z], nullptr, nullptr, 1.0, 0, 0, nullptr, &q->sl[SL_Z],
                          GDM_PHASE_TRANSFORM, nullptr);
      if (e != cudaSuccess) return e;
      if ((e = fas(p, st, q->f[F_ZT], nullptr, nullptr, 1.0, 0, 0, nullptr, &q->sl[SL_ZT],
                   GDM_PHASE_TRANSFORM, nullptr)) != cudaSuccess)
        return e;
      return fas(p, st, q->f[F_H], nullptr, nullptr, 1.0, 0, 0, nullptr, &q->sl[SL_A],
                 GDM_PHASE_TRANSFORM, nullptr);
    });
    // H~ = Z^T H Z
    grouped(GDM_PHASE_TRANSFORM, [&](int p, SlicedGemmArgs& a, const SliceBuf*& A,
                                     const SliceBuf*& B) {
      gdm_handle* q = h[p];
      A = &q->sl[SL_ZT];
      B = &q->sl[SL_A];
      a.C = q->f[F_T];
      a.ldc = q->ld;
    });
    per_problem([&](int p, cudaStream_t st) -> cudaError_t {
      gdm_handle* q = h[p];
      return fas(p, st, q->f[F_T], nullptr, nullptr, 1.0, 0, 0, nullptr, &q->sl[SL_B],
                 GDM_PHASE_TRANSFORM, nullptr);
    });
    grouped(GDM_PHASE_TRANSFORM, [&](int p, SlicedGemmArgs& a, const SliceBuf*& A,
                                     const SliceBuf*& B) {
      gdm_handle* q = h[p];
      A = &q->sl[SL_B];
      B = &q->sl[SL_ZT];
      a.mode = kGemmSym;
      a.C = q->f[F_U];
      a.ldc = q->ld;
    });
    // spectral bounds of H~ and X_0 (with its slices and row dots)
    per_problem([&](int p, cudaStream_t st) -> cudaError_t {
      gdm_handle* q = h[p];
      const int n = static_cast<int>(q->n);
      const int lz = std::min(kLanczosSteps, n);
      cudaError_t e = gershgorin(q->f[F_U], q->ld, n, q->partials, q->small + SM_GERSH_H, st);
      if (e != cudaSuccess) return e;
      if ((e = lanczos(q->f[F_U], q->ld, n, lz, q->lanczos_ws, q->partials, q->small + SM_LANCZOS,
                       st)) != cudaSuccess)
        return e;
      if ((e = lanczos_bounds(q->small, lz, SM_GERSH_H, SM_LANCZOS, SM_EST_H, st)) !=
          cudaSuccess)
        return e;
      if ((e = x0_coefficients(q->small + SM_EST_H, q->small + SM_COEF_X0, st)) != cudaSuccess)
        return e;
      return fas(p, st, q->f[F_U], nullptr, q->small + SM_COEF_X0, 0, 0, 0, q->f[F_X],
                 &q->sl[SL_X], GDM_PHASE_PURIFY, nullptr, kDotSelf);
    });
  }

  // TRS4 iteration of parity `par`: X in X (even) or XN (odd), the next iterate in the other.
  void phase_pu_iteration(int par) {
    const int Xb = par ? F_XN : F_X, Xnb = par ? F_X : F_XN;
    grouped(GDM_PHASE_PURIFY, [&](int p, SlicedGemmArgs& a, const SliceBuf*& A,
                                  const SliceBuf*& B) {
      gdm_handle* q = h[p];
      A = &q->sl[SL_X];
      B = &q->sl[SL_X];
      a.mode = kGemmSym;
      a.C = q->f[F_X2];
      a.ldc = q->ld;
      // X's slicing paired its rows with themselves
      a.diag_dot = rowdots(p) ? q->sl[SL_X].row_dot : nullptr;
      a.skip = &q->st_dev->done;
    });
    per_problem([&](int p, cudaStream_t st) -> cudaError_t {
      gdm_handle* q = h[p];
      const int n = static_cast<int>(q->n);
      const int nsl = q->phase[GDM_PHASE_PURIFY].nslice, bits = q->phase[GDM_PHASE_PURIFY].bits;
      double* X = q->f[Xb];
      double* X2 = q->f[F_X2];
      const int* done = &q->st_dev->done;
      int nb = 0;
      cudaError_t e;
      if (!rowdots(p) &&
          (e = diag_fix(X, q->ld, X, q->ld, X2, q->ld, n, n, 1.0, 0.0, nullptr, 0, 0.0, nullptr,
                        st, done)) != cudaSuccess)
        return e;
      const bool fused = rowdots(p) && slice_traces_fits(X2, X, q->ld, n, &q->sl[SL_X2], nsl, true);
      if (fused)
        e = slice_traces(X2, X, q->ld, n, &q->sl[SL_X2], nsl, bits, q->partials, &nb, st, done,
                         true);
      else e = trs4_traces(X, X2, q->ld, n, q->partials, &nb, st, done);
      if (e != cudaSuccess) return e;
      if ((e = trs4_control(q->partials, nb, q->st_dev, q->idem_tol * double(q->n_occ), st)) !=
          cudaSuccess)
        return e;
      const int* skip_gemm = &q->st_dev->skip_gemm;
      const double* coefW = &q->st_dev->coefW[0];
      if (!fused &&
          (e = fas(p, st, X2, nullptr, nullptr, 1.0, 0, 0, nullptr, &q->sl[SL_X2],
                   GDM_PHASE_PURIFY, skip_gemm)) != cudaSuccess)
        return e;
      if ((e = fas(p, st, X, X2, coefW, 0, 0, 0, fused ? nullptr : q->f[F_V], &q->sl[SL_W],
                   GDM_PHASE_PURIFY, skip_gemm, fused ? kDotNone : kDotX2)) != cudaSuccess)
        return e;
      if (fused) return w_row_dots(q->partials, n, coefW, &q->sl[SL_W], X2, st);
      return cudaSuccess;
    });
    grouped(GDM_PHASE_PURIFY, [&](int p, SlicedGemmArgs& a, const SliceBuf*& A,
                                  const SliceBuf*& B) {
      gdm_handle* q = h[p];
      A = &q->sl[SL_X2];
      B = &q->sl[SL_W];
      a.mode = kGemmSym;
      a.C = q->f[Xnb];
      a.ldc = q->ld;
      a.diag_dot = rowdots(p) ? q->sl[SL_W].row_dot : nullptr;  // W's row dots with X^2
      a.skip = &q->st_dev->skip_gemm;
    });
    per_problem([&](int p, cudaStream_t st) -> cudaError_t {
      gdm_handle* q = h[p];
      const int n = static_cast<int>(q->n);
      cudaError_t e;
      // without row dots, W was written out (the unfused slicing) and the diagonal is recomputed
      if (!rowdots(p) &&
          (e = diag_fix(q->f[F_X2], q->ld, q->f[F_V], q->ld, q->f[Xnb], q->ld, n, n, 1.0, 0.0,
                        nullptr, 0, 0.0, nullptr, st, &q->st_dev->skip_gemm)) != cudaSuccess)
        return e;
      e = fas(p, st, q->f[Xnb], nullptr, nullptr, 1.0, 0, 0, nullptr, &q->sl[SL_X],
              GDM_PHASE_PURIFY, &q->st_dev->skip_gemm, kDotSelf);
      if (e != cudaSuccess) return e;
      return fas(p, st, q->f[Xb], q->f[F_X2], &q->st_dev->coefX[0], 0, 0, 0, q->f[Xnb],
                 &q->sl[SL_X], GDM_PHASE_PURIFY, &q->st_dev->skip_form_x, kDotSelf);
    });
  }

  void phase_post() {
    per_problem([&](int p, cudaStream_t st) -> cudaError_t {
      gdm_handle* q = h[p];
      const int n = static_cast<int>(q->n);
      copy_if_kernel<<<n, 256, 0, st>>>(q->f[F_X], q->f[F_XN], q->ld, n, &q->st_dev->final_buf, 1);
      count_launch();
      cudaError_t e = trace_scale(q->f[F_X], q->ld, n, double(q->n_occ), q->small + SM_RED + 4, st);
      if (e != cudaSuccess) return e;
      return fas(p, st, q->f[F_X], nullptr, nullptr, 1.0, 0, 0, nullptr, &q->sl[SL_X],
                 GDM_PHASE_TRANSFORM, nullptr);
    });
    grouped(GDM_PHASE_TRANSFORM, [&](int p, SlicedGemmArgs& a, const SliceBuf*& A,
                                     const SliceBuf*& B) {
      gdm_handle* q = h[p];
      A = &q->sl[SL_Z];
      B = &q->sl[SL_X];
      a.C = q->f[F_T];
      a.ldc = q->ld;
    });
    per_problem([&](int p, cudaStream_t st) -> cudaError_t {
      gdm_handle* q = h[p];
      return fas(p, st, q->f[F_T], nullptr, nullptr, 1.0, 0, 0, nullptr, &q->sl[SL_A],
                 GDM_PHASE_TRANSFORM, nullptr);
    });
    grouped(GDM_PHASE_TRANSFORM, [&](int p, SlicedGemmArgs& a, const SliceBuf*& A,
                                     const SliceBuf*& B) {
      gdm_handle* q = h[p];
      A = &q->sl[SL_A];
      B = &q->sl[SL_Z];
      a.mode = kGemmSym;
      a.C = q->f[F_XN];
      a.ldc = q->ld;
    });
    per_problem([&](int p, cudaStream_t st) -> cudaError_t {
      gdm_handle* q = h[p];
      const int n = static_cast<int>(q->n);
      double* P = q->f[F_XN];
      // exact diagonal (it carries the count when S is close to I), count, rescale, count, energy
      cudaError_t e = diag_fix(q->f[F_T], q->ld, q->f[F_Z], q->ld, P, q->ld, n, n, 1.0, 0.0,
                               nullptr, 0, 0.0, nullptr, st);
      if (e != cudaSuccess) return e;
      int nb = 0;
      if ((e = dot_partials(P, q->ld, q->f[F_S], q->ld, n, n, 0, q->partials, &nb, st, nullptr,
                            true)) !=
          cudaSuccess)
        return e;
      if ((e = reduce_partials(q->partials, nb, 1, q->small + SM_RED, st)) != cudaSuccess) return e;
      count_factor_kernel<<<1, 1, 0, st>>>(ctl(p), q->small + SM_RED, double(q->n_occ),
                                           q->trace_correct ? q->rescale_tol : INFINITY);
      scale_if_kernel<<<n, 256, 0, st>>>(P, q->ld, n, ctl(p));
      count_launch(2);
      if ((e = dot_partials(P, q->ld, q->f[F_S], q->ld, n, n, 0, q->partials, &nb, st, nullptr,
                            true)) !=
          cudaSuccess)
        return e;
      if ((e = reduce_partials(q->partials, nb, 1, q->small + SM_RED + 1, st)) != cudaSuccess)
        return e;
      if ((e = dot_partials(P, q->ld, q->f[F_H], q->ld, n, n, 0, q->partials, &nb, st, nullptr,
                            true)) !=
          cudaSuccess)
        return e;
      return reduce_partials(q->partials, nb, 1, q->small + SM_RED + 2, st);
    });
  }

  // ---- construction ----------------------------------------------------------------------
  // The phases in order; `which` < 0 plans every phase, else captures phase `which`.
  void record(int which) {
    site_cursor = 0;
    if (which < 0 || which == 0) phase_pre();
    else site_cursor += 0;
    if (which < 0 || which == 1) {
      phase_ns_iteration(0);
      phase_ns_iteration(1);
    } else {
      site_cursor += 6;
    }
    if (which < 0 || which == 2) phase_rf();
    else site_cursor += 10 + 2;
    if (which < 0 || which == 3) {
      phase_pu_iteration(0);
      phase_pu_iteration(1);
    } else {
      site_cursor += 4;
    }
    if (which < 0 || which == 4) phase_post();
  }

  cudaError_t capture(int which) {
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(main, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return e;
    const int64_t launches0 = launch_count();
    record(which);
    count_launch(-static_cast<int>(launch_count() - launches0));  // nothing ran yet
    e = cudaStreamEndCapture(main, &graph);
    if (e != cudaSuccess) return e;
    if (first_error != cudaSuccess) {
      cudaGraphDestroy(graph);
      return first_error;
    }
    size_t nodes = 0;
    if (cudaGraphGetNodes(graph, nullptr, &nodes) == cudaSuccess && nodes > 0) {
      std::vector<cudaGraphNode_t> list(nodes);
      cudaGraphGetNodes(graph, list.data(), &nodes);
      int kernels = 0;
      for (auto nd : list) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
      }
      g_kernels[which] = kernels;
    }
    e = cudaGraphInstantiate(&g[which], graph, 0);
    cudaGraphDestroy(graph);
    return e;
  }

  // Time the grouped variants of each slice format on its largest site; remember the choice.
  void autotune() {
    tune_load();
    const std::string gpu = gpu_name(device);
    for (int ns = 1; ns <= 4; ++ns) {
      int best_site = -1;
      for (size_t i = 0; i < sites.size(); ++i)
        if (sites[i].prec.nslice == ns && (best_site < 0 || sites[i].units > sites[best_site].units))
          best_site = static_cast<int>(i);
      if (best_site < 0) continue;
      Site& s = sites[best_site];
      int cls = 0;
      while ((1 << (cls + 1)) <= s.units) ++cls;
      char key[256];
      snprintf(key, sizeof(key), "%s|s%d|u%d", gpu.c_str(), ns, cls);
      auto it = g_tune.find(key);
      if (it != g_tune.end()) {
        variant[ns] = it->second;
        continue;
      }
      const int nv = grouped_variant_count(ns);
      double best_ms = INFINITY;
      int best = 0;
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      for (int v = 0; v < nv; ++v) {
        float ms_min = INFINITY;
        for (int rep = 0; rep < 3; ++rep) {
          cudaEventRecord(e0, main);
          note(sliced_gemm_grouped(s.dev[v], count(), s.units, s.prec, err_dev, main, v),
               "autotune launch");
          cudaEventRecord(e1, main);
          cudaEventSynchronize(e1);
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (rep > 0) ms_min = std::min(ms_min, ms);
        }
        if (ms_min < best_ms) {
          best_ms = ms_min;
          best = v;
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      variant[ns] = best;
      g_tune[key] = best;
      tune_store();
    }
  }

  gdm_status build(int dev, const std::vector<int64_t>& nn, const std::vector<int64_t>& occ) {
    device = dev;
    n = nn;
    nocc = occ;
    for (size_t p = 0; p < nn.size(); ++p) {
      gdm_handle* q = nullptr;
      gdm_status st = gdm_init(&q, nn[p], occ[p], dev);
      if (st != GDM_OK) return st;
      h.push_back(q);
    }
    if (cudaStreamCreateWithFlags(&main, cudaStreamNonBlocking) != cudaSuccess) return GDM_ERR_CUDA;
    for (auto& s : side)
      if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return GDM_ERR_CUDA;
    if (cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming) != cudaSuccess) return GDM_ERR_CUDA;
    for (auto& e : ev_join)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return GDM_ERR_CUDA;
    const int cnt = count();
    if (cudaMalloc(&err_dev, 256) != cudaSuccess ||
        cudaMalloc(&ns_flags_dev, sizeof(int*) * cnt) != cudaSuccess ||
        cudaMalloc(&pu_flags_dev, sizeof(int*) * cnt) != cudaSuccess ||
        cudaMalloc(&flags_dev, sizeof(int) * cnt) != cudaSuccess ||
        cudaMallocHost(&flags_host, sizeof(int) * cnt) != cudaSuccess)
      return GDM_ERR_OOM;
    cudaMemset(err_dev, 0, 256);
    std::vector<const int*> nsf(cnt), puf(cnt);
    for (int p = 0; p < cnt; ++p) {
      nsf[p] = &ctl(p)->ns_off;
      puf[p] = &h[p]->st_dev->done;
    }
    cudaMemcpy(ns_flags_dev, nsf.data(), sizeof(int*) * cnt, cudaMemcpyHostToDevice);
    cudaMemcpy(pu_flags_dev, puf.data(), sizeof(int*) * cnt, cudaMemcpyHostToDevice);
    // plan: the grouped tables of every launch site, uploaded once
    planning = true;
    record(-1);
    planning = false;
    if (first_error != cudaSuccess) return GDM_ERR_CUDA;
    for (auto& s : sites)
      for (int v = 0; v < 2; ++v) {
        if (s.host[v].empty()) continue;
        if (cudaMalloc(&s.dev[v], sizeof(GroupItem) * cnt) != cudaSuccess) return GDM_ERR_OOM;
        cudaMemcpy(s.dev[v], s.host[v].data(), sizeof(GroupItem) * cnt, cudaMemcpyHostToDevice);
      }
    autotune();
    cudaStreamSynchronize(main);
    for (int k = 0; k < 5; ++k)
      if (capture(k) != cudaSuccess) return GDM_ERR_CUDA;
    return first_error == cudaSuccess ? GDM_OK : GDM_ERR_CUDA;
  }

  cudaError_t launch_graph(int k) {
    count_launch(g_kernels[k]);
    return cudaGraphLaunch(g[k], main);
  }

  // Replay graph `k` two at a time until every flag in `flags` is set (at most `cap` replays).
  cudaError_t loop(int k, const int** flags, int cap, int* replays) {
    *replays = 0;
    while (*replays < cap) {
      for (int r = 0; r < 2 && *replays < cap; ++r, ++*replays) {
        cudaError_t e = launch_graph(k);
        if (e != cudaSuccess) return e;
      }
      gather_flags_kernel<<<1, 256, 0, main>>>(flags, count(), flags_dev);
      count_launch();
      cudaError_t e = cudaMemcpyAsync(flags_host, flags_dev, sizeof(int) * count(),
                                      cudaMemcpyDeviceToHost, main);
      if (e != cudaSuccess) return e;
      if ((e = cudaStreamSynchronize(main)) != cudaSuccess) return e;
      bool all = true;
      for (int p = 0; p < count(); ++p) all = all && flags_host[p] != 0;
      if (all) break;
    }
    return cudaSuccess;
  }
};

// The executor of the last batch shape (its handles, tables and graphs), reused while the
// shapes repeat.  Never destroyed at process exit (the CUDA runtime may be gone by then); the
// driver frees the memory with the process, gdm_batch_release frees it earlier.
std::mutex g_exec_mutex;
BatchExec* g_exec = nullptr;

// Same device and the same problem sizes as the cached executor?
bool same_shape(const BatchExec* x, int device, const gdm_problem* pr, int count) {
  if (x == nullptr || x->device != device || x->count() != count) return false;
  for (int i = 0; i < count; ++i)
    if (x->n[i] != pr[i].n_basis || x->nocc[i] != pr[i].n_occ) return false;
  return true;
}

}  // namespace

// Solve `count` problems as one lockstep batch; the results of problems that fail in the lockstep
// are marked for a solo solve (results[i].status = GDM_ERR_STATE and *resolve[i] = 1).
gdm_status batch_solve_grouped(const gdm_problem* pr, int count, gdm_result* res, int device,
                               std::vector<int>* resolve) {
  std::lock_guard<std::mutex> lock(g_exec_mutex);
  if (cudaSetDevice(device) != cudaSuccess) return GDM_ERR_CUDA;
  if (!same_shape(g_exec, device, pr, count)) {
    delete g_exec;
    g_exec = nullptr;
    std::unique_ptr<BatchExec> x(new BatchExec());
    std::vector<int64_t> nn(count), occ(count);
    for (int i = 0; i < count; ++i) {
      nn[i] = pr[i].n_basis;
      occ[i] = pr[i].n_occ;
    }
    gdm_status st = x->build(device, nn, occ);
    if (st != GDM_OK) return st;
    g_exec = x.release();
  }
  BatchExec& x = *g_exec;
  const double t0 = std::chrono::duration<double>(
      std::chrono::steady_clock::now().time_since_epoch()).count();
  cudaStream_t s = x.main;
  // ingest (outside the graphs: the caller's buffers differ from call to call)
  for (int p = 0; p < count; ++p) {
    gdm_handle* q = x.h[p];
    const size_t w = sizeof(double) * static_cast<size_t>(q->n);
    const cudaMemcpyKind kind =
        pr[p].mem == GDM_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (cudaMemcpy2DAsync(q->f[F_H], sizeof(double) * q->ld, pr[p].H, sizeof(double) * pr[p].ldh,
                          w, q->n, kind, s) != cudaSuccess ||
        cudaMemcpy2DAsync(q->f[F_S], sizeof(double) * q->ld, pr[p].S, sizeof(double) * pr[p].lds,
                          w, q->n, kind, s) != cudaSuccess ||
        symmetrise(q->f[F_H], q->ld, static_cast<int>(q->n), s) != cudaSuccess ||
        symmetrise(q->f[F_S], q->ld, static_cast<int>(q->n), s) != cudaSuccess)
      return GDM_ERR_CUDA;
  }
  cudaMemsetAsync(x.err_dev, 0, sizeof(uint32_t), s);
  int replays_ns = 0, replays_pu = 0;
  int max_ns = 0, max_pu = 0;
  for (auto* q : x.h) {
    max_ns = std::max(max_ns, q->max_ns);
    max_pu = std::max(max_pu, q->max_purif);
  }
  // GDM_BATCH_VERBOSE=1 prints each phase's device time and the replays to stderr
  const bool verbose = getenv("GDM_BATCH_VERBOSE") != nullptr;
  cudaEvent_t ev[6] = {};
  if (verbose)
    for (auto& v : ev) cudaEventCreate(&v);
  if (verbose) cudaEventRecord(ev[0], s);
  cudaError_t e = x.launch_graph(0);
  if (verbose) cudaEventRecord(ev[1], s);
  if (e == cudaSuccess) e = x.loop(1, x.ns_flags_dev, max_ns / 2 + 2, &replays_ns);
  if (verbose) cudaEventRecord(ev[2], s);
  if (e == cudaSuccess) e = x.launch_graph(2);
  if (verbose) cudaEventRecord(ev[3], s);
  if (e == cudaSuccess) e = x.loop(3, x.pu_flags_dev, max_pu / 2 + 2, &replays_pu);
  if (verbose) cudaEventRecord(ev[4], s);
  if (e == cudaSuccess) e = x.launch_graph(4);
  if (verbose) {
    cudaEventRecord(ev[5], s);
    cudaEventSynchronize(ev[5]);
    float ms[5] = {};
    for (int k = 0; k < 5; ++k) cudaEventElapsedTime(&ms[k], ev[k], ev[k + 1]);
    fprintf(stderr,
            "[gdm batch] %d problems: pre %.2f ms, newton-schulz %.2f ms (%d replays of %d "
            "kernels), refine+transform+bounds %.2f ms, purification %.2f ms (%d replays of %d "
            "kernels), post %.2f ms; grouped variants s2:%d s3:%d s4:%d\n",
            count, ms[0], ms[1], replays_ns, x.g_kernels[1], ms[2], ms[3], replays_pu,
            x.g_kernels[3], ms[4], x.variant[2], x.variant[3], x.variant[4]);
    for (auto& v : ev) cudaEventDestroy(v);
  }
  // results: each problem's small[] and controller state, P to the caller
  for (int p = 0; p < count && e == cudaSuccess; ++p) {
    gdm_handle* q = x.h[p];
    e = cudaMemcpyAsync(q->host_buf, q->small, sizeof(double) * (SM_BATCH + 64),
                        cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(q->st_host, q->st_dev, sizeof(Trs4State), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && pr[p].P != nullptr)
      e = cudaMemcpy2DAsync(pr[p].P, sizeof(double) * pr[p].ldp, q->f[F_XN],
                            sizeof(double) * q->ld, sizeof(double) * q->n, q->n,
                            pr[p].p_mem == GDM_MEM_HOST ? cudaMemcpyDeviceToHost
                                                        : cudaMemcpyDeviceToDevice,
                            s);
  }
  uint32_t herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, x.err_dev, sizeof(herr), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    delete g_exec;
    g_exec = nullptr;
    return GDM_ERR_CUDA;
  }
  if (herr & DEV_ERR_WAIT_TIMEOUT) return GDM_ERR_TIMEOUT;
  const double t1 = std::chrono::duration<double>(
      std::chrono::steady_clock::now().time_since_epoch()).count();
  resolve->assign(count, 0);
  for (int p = 0; p < count; ++p) {
    gdm_handle* q = x.h[p];
    const double* sm = q->host_buf;
    const BatchCtl* c = reinterpret_cast<const BatchCtl*>(sm + SM_BATCH);
    const Trs4State& t = *q->st_host;
    gdm_result& r = res[p];
    memset(&r, 0, sizeof(r));
    const double N = static_cast<double>(q->n_occ);
    r.info.ns_iters = c->ns_iters;
    r.info.refine_iters = c->rf_steps;
    r.info.purif_iters = t.stop != 0 ? t.iter - 1 : t.iter;  // steps taken (the stop takes none)
    r.info.stop_reason = t.stop;
    r.info.idem_err = t.final_idem;
    r.info.z_err = c->rf_derr;
    r.info.trace_err_raw = std::fabs(c->count_raw - N);
    r.info.trace_err = std::fabs(sm[SM_RED + 1] - N);
    r.info.energy = sm[SM_RED + 2];
    r.info.eps_min = sm[SM_EST_H];
    r.info.eps_max = sm[SM_EST_H + 1];
    r.info.trace_fix = sm[SM_RED + 4];
    r.info.kstage_fraction = 1.0;
    r.info.trace_rescaled = c->rescaled;
    r.info.s_idem_err = -1.0;
    r.info.ms_total = (t1 - t0) * 1e3;
    r.energy = r.info.energy;
    r.latency_ms = (t1 - t0) * 1e3;
    const bool ok = !c->ns_failed && !c->rf_failed && !t.failed && t.stop != 3 && t.stop != 4 &&
                    std::isfinite(r.energy) && r.info.trace_err <= q->trace_tol;
    r.status = ok ? GDM_OK : GDM_ERR_STATE;
    (*resolve)[p] = ok ? 0 : 1;
    if (!ok && getenv("GDM_BATCH_VERBOSE") != nullptr)
      fprintf(stderr,
              "[gdm batch] problem %d (n=%lld) solved again alone: ns_failed %d rf_failed %d "
              "trs4 stop %d failed %d iter %d, energy %g, count error %g\n",
              p, static_cast<long long>(q->n), c->ns_failed, c->rf_failed, t.stop, t.failed,
              t.iter, r.energy, r.info.trace_err);
  }
  (void)replays_ns;
  (void)replays_pu;
  return GDM_OK;
}

// Release the cached batch executor (its handles and graphs).
void batch_release() {
  std::lock_guard<std::mutex> lock(g_exec_mutex);
  delete g_exec;
  g_exec = nullptr;
}

}  // namespace gdm
