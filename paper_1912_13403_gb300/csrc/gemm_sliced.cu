// Sliced-FP16 tensor-core product C = alpha * A * B + beta * D on sm_103a (tcgen05 + TMEM + TMA).
//
// Every matrix product of the density-matrix route (the Loewdin transform H~ = S^{-1/2} H
// S^{-1/2}, Sec. 2.2.2 Eq. ntpoly_lowdin; the purification steps P_{n+1} = f(P_n), Eq.
// ntpoly_purification; the back-transform) goes through this kernel.
//
// Number format.  Each operand row i is stored as up to four FP16 "slices" holding integers:
//     a_ik = sigma_i * 2^-11 * sum_s m_s[i,k] * 2^(-b s),   |m_s| <= 2048,
// where sigma_i is a power of two >= ||a_i||_2, so that ||m_0[i,:]||_2 <= 2^11 (+ rounding), and
// b (9..12) is the width of the trailing slices.  The product of two slices is accumulated by
// the tensor core in FP32.  Slice pairs of the same order o = s + t share one TMEM accumulator;
// order 0 stays below 2^23 in magnitude for every partial sum (Cauchy-Schwarz on the row
// norms), so it is exact; the higher orders are integers too and are exact while their partial
// sums stay below 2^24 (with b = 9 that holds for the random-walk sums of residual slices up to
// K ~ 8192; with b = 12 the order-2 sum rounds at a relative weight of about 2^-46).  The
// epilogue combines
//     C_ij = alpha * sigma_i sigma_j 2^-22 * sum_o 2^(-b o) acc_o[i,j] + beta * D_ij
// in FP64.  The operand B is given as the row slices of B^T (for the symmetric right operands
// of this route that is B itself).
//
// Kernel shape: persistent, one CTA per SM, each CTA walks the 128x128 output tiles
// blockIdx.x, blockIdx.x + gridDim.x, ...  The slice pairs of one 16-wide k step go out as few,
// wide MMAs: A slice s times two adjacent B slices is one M = 128, N = 256 instruction (the two
// B panels are adjacent in shared memory and the two orders' accumulators are adjacent in
// TMEM), which cuts the instructions per k step (3 slices: 8 pair MMAs become 5) and the
// shared-memory reads of A.  12 warps.  Warp 0: TMA producer (a 3-D box loads all slices of a
// 128 x BK panel at once, BK = 64 for up to 3 slices); its stage ring runs on across tiles, so
// the next tile's operands stream in while the current tile's epilogue runs.  Warp 1: TMEM
// allocator and the single MMA-issuing thread.  Warps 4-11: epilogue, two warps per TMEM lane
// quarter (32*(warp%4) ...), each covering 64 of the 128 columns; a warp reads all of its
// accumulator columns into int64 registers first and releases TMEM, so that the conversion and
// the stores overlap the next tile's MMAs.  Formats with at most two orders keep two
// accumulator sets in TMEM (the MMAs never wait for the epilogue); the tiles of the last,
// partial wave are split along k (sliced_gemm).  Symmetric mode computes only tiles
// on or above the diagonal and writes the mirror image.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "gdm_internal.h"

namespace gdm {

namespace {

constexpr int kBM = 128;
constexpr int kBN = 128;
// 12 warps: warpgroup 0 = TMA producer (warp 0), MMA issuer (warp 1) and two idle warps;
// warpgroups 1-2 = the 8 epilogue warps.  Launched with 168 registers a thread, the control
// warpgroup gives registers to the epilogue (4 x 32 x 104 + 8 x 32 x 200 = 384 x 168), which
// then holds a whole 32 x 64 accumulator block as int64 without spilling.
constexpr int kThreads = 384;
constexpr int kEpiWarps = kEpilogueWarps;
constexpr int kEpiWarp0 = 4;
constexpr int kLaunchRegs = 168;
constexpr int kCtrlRegs = 104;
constexpr int kEpiRegs = 200;
static_assert(4 * 32 * kCtrlRegs + kEpiWarps * 32 * kEpiRegs == kThreads * kLaunchRegs,
              "register split must equal the launch allocation");
static_assert(kLaunchRegs * kThreads <= 65536, "launch registers");
constexpr int kStageCols = 8;  // epilogue staging: 32 rows x 8 columns per warp
constexpr int kPairsUsed = 10;  // most slice pairs of a format (4 slices, orders 0..3)

template <int NSLICE, int BK, int STAGES>
struct GemmCfg {
  static constexpr uint32_t kTileBytes = kBM * BK * 2;                // one slice panel
  static constexpr uint32_t kStageBytes = 2u * NSLICE * kTileBytes;   // A and B panels
  static constexpr uint32_t kStagingBytes = kEpiWarps * 32 * (kStageCols + 1) * 8;
  static constexpr uint32_t kSmemBytes = STAGES * kStageBytes + kStagingBytes + 1024;
  static_assert(BK == 64 || BK == 32, "BK must be 64 (128B swizzle) or 32 (64B swizzle)");
  static_assert(kSmemBytes <= 227 * 1024, "shared memory budget");
};

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, int bk) {
  // K-major, swizzle width = one row of the panel (bk * 2 bytes), 8-row groups contiguous.
  const uint32_t sbo = 8u * bk * 2u;
  const uint64_t layout = (bk == 64) ? 2ull : 4ull;  // SWIZZLE_128B : SWIZZLE_64B
  uint64_t d = 0;
  d |= static_cast<uint64_t>((addr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>(1u) << 16;
  d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
  d |= static_cast<uint64_t>(1u) << 46;
  d |= layout << 61;
  return d;
}

// Upper-triangle tile index -> (ti, tj) with ti <= tj, row-major over the triangle.
__device__ __forceinline__ void upper_tile(int idx, int nt, int& ti, int& tj) {
  int i = 0;
  int row_len = nt;
  while (idx >= row_len) {
    idx -= row_len;
    ++i;
    --row_len;
  }
  ti = i;
  tj = i + idx;
}

// ---- epilogue arithmetic without FP64 instructions ----------------------------------------
// Every accumulator holds an integer value: products of integer slices, summed in FP32 (exact
// below 2^24, and FP32 values at or above 2^24 are integers too).

// int64 value of an integer-valued FP32 with |v| < 2^44, in eight FP32 / integer instructions:
// v = H 2^22 + L with H = round(v / 2^22) and |L| <= 2^21, both read off the bit pattern of a
// sum with a bias 1.5 * 2^(23 + k), which rounds to a multiple of 2^k (all steps exact).
__device__ __forceinline__ long long f32_int_exact(uint32_t bits) {
  const float v = __uint_as_float(bits);
  const float kBigBias = 52776558133248.0f;  // 1.5 * 2^45: multiples of 2^22
  const float kBias = 12582912.0f;           // 1.5 * 2^23: multiples of 1
  const float hb = v + kBigBias;
  const int H = __float_as_int(hb) - 0x56400000;
  const float l = v - (hb - kBigBias);
  const int L = __float_as_int(l + kBias) - 0x4B400000;
  return static_cast<long long>(H) * 4194304LL + L;
}

// finiteness from the bit pattern (integer compare, no FP64 instruction)
__device__ __forceinline__ bool finite_bits(double s) {
  return ((static_cast<unsigned long long>(__double_as_longlong(s)) >> 52) & 0x7FF) != 0x7FF;
}

// alpha = +-2^k exactly?  (then scaling is an exponent shift)
__device__ __forceinline__ bool pow2_scalar(double a, int& k, bool& neg) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(a));
  const int E = static_cast<int>((b >> 52) & 0x7FF);
  if (E == 0 || E == 0x7FF || (b & ((1ULL << 52) - 1)) != 0) return false;
  k = E - 1023;
  neg = (b >> 63) != 0;
  return true;
}

// exponent of a power-of-two double (the row scales)
__device__ __forceinline__ int pow2_exponent(double s) {
  return static_cast<int>((static_cast<unsigned long long>(__double_as_longlong(s)) >> 52) &
                          0x7FF) - 1023;
}

// T * 2^ex as a double, rounded to nearest even, built from integer operations (|T| < 2^63;
// results below the normal range flush to 0).
__device__ __forceinline__ double scaled_int_to_double(long long T, int ex) {
  if (T == 0) return 0.0;
  const unsigned long long sign = (T < 0) ? (1ULL << 63) : 0ULL;
  unsigned long long u = (T < 0) ? static_cast<unsigned long long>(-T)
                                 : static_cast<unsigned long long>(T);
  const int msb = 63 - __clzll(u);
  int e = msb + ex;
  unsigned long long mant;
  if (msb > 52) {
    const int r = msb - 52;
    mant = u >> r;
    const unsigned long long rem = u & ((1ULL << r) - 1);
    const unsigned long long half = 1ULL << (r - 1);
    if (rem > half || (rem == half && (mant & 1ULL))) ++mant;
    if (mant == (1ULL << 53)) {
      mant >>= 1;
      ++e;
    }
  } else {
    mant = u << (52 - msb);
  }
  if (e + 1023 <= 0) return 0.0;
  return __longlong_as_double(static_cast<long long>(
      sign | (static_cast<unsigned long long>(e + 1023) << 52) | (mant & ((1ULL << 52) - 1))));
}

// Out-of-line FP64 steps of the epilogue (see the call sites).
__device__ __noinline__ double fp64_scale(double v, double a) { return v * a; }
__device__ __noinline__ double fp64_axpy(double a, double x, double y) { return fma(a, x, y); }
// C_ii from the exact row dot product of the slicing pass when there is one: the FP32
// accumulation truncates, and on the diagonal of a product of (nearly) parallel rows its
// residual-slice terms form a positive sum whose truncation biases C_ii; plus the diagonal shift.
__device__ __noinline__ double diagonal_value(double v, const double* diag_dot, double shift,
                                              int i, double alpha) {
  if (diag_dot != nullptr) v = alpha * diag_dot[i];
  return v + shift;
}

// Does the k stage kb of tile (ti, tj) contribute?  Only with tile masks: the first 128-wide
// k block always runs (so that every accumulator is written), the others when both operand
// tiles hold a non-zero element.
__device__ __forceinline__ bool kstage_active(const uint32_t* mask_a, const uint32_t* mask_b,
                                              int mask_ld, int ti, int tj, int kb, int bk) {
  if (mask_a == nullptr) return true;
  const int k128 = (kb * bk) >> 7;
  if (k128 == 0) return true;
  return __ldg(mask_a + ti * mask_ld + k128) != 0u && __ldg(mask_b + tj * mask_ld + k128) != 0u;
}

// Work unit u of the launch -> output tile, k-block range and split part (-1: whole tile).
// The tiles of the last, partial wave are split along k into args.split parts, so that every
// CTA runs the same number of whole tiles plus at most one part (see sliced_gemm).
__device__ __forceinline__ void unit_of(int u, const SlicedGemmArgs& a, int nk, int& tile,
                                        int& kb0, int& kb1, int& part) {
  if (a.split <= 1 || u < a.full_tiles) {
    tile = u;
    kb0 = 0;
    kb1 = nk;
    part = -1;
    return;
  }
  const int v = u - a.full_tiles;
  tile = a.full_tiles + v / a.split;
  part = v % a.split;
  kb0 = part * nk / a.split;
  kb1 = (part + 1) * nk / a.split;
}

// One work unit of a launch, decoded the same way by the producer, the MMA issuer and the
// epilogue: the output tile, its k-block range and split part (-1: whole tile), the product it
// belongs to (its arguments and operand maps) and whether that product is skipped.
struct Unit {
  int ti, tj, kb0, kb1, part, tile;
  const SlicedGemmArgs* ep;
  const CUtensorMap* ma;
  const CUtensorMap* mb;
  bool skip;
};

template <bool GROUPED, int BK>
__device__ __forceinline__ void decode_unit(int u, const SlicedGemmArgs& args, int nk,
                                            const CUtensorMap* tmA, const CUtensorMap* tmB,
                                            Unit& w) {
  if constexpr (GROUPED) {
    // the last table entry whose first unit is <= u (entries in unit order)
    int lo = 0, hi = args.ngroup - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (args.group[mid].a.unit_begin <= u) lo = mid; else hi = mid - 1;
    }
    const GroupItem& it = args.group[lo];
    w.ep = &it.a;
    w.ma = &it.ta;
    w.mb = &it.tb;
    w.skip = it.a.skip != nullptr && *it.a.skip != 0;
    const int t = u - it.a.unit_begin;
    if (it.a.mode & kGemmSym) upper_tile(t, it.a.tiles_n, w.ti, w.tj);
    else { w.ti = t / it.a.tiles_n; w.tj = t % it.a.tiles_n; }
    w.kb0 = 0;
    w.kb1 = (it.a.K + BK - 1) / BK;
    w.part = -1;
    w.tile = t;
  } else {
    unit_of(u, args, nk, w.tile, w.kb0, w.kb1, w.part);
    if (args.mode & kGemmSym) upper_tile(w.tile, args.tiles_n, w.ti, w.tj);
    else { w.ti = w.tile / args.tiles_n; w.tj = w.tile % args.tiles_n; }
    w.ep = &args;
    w.ma = tmA;
    w.mb = tmB;
    w.skip = false;
  }
}

template <int NSLICE, int BK, int STAGES, bool GROUPED>
__global__ void __launch_bounds__(kThreads, 1)
    sliced_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                       const __grid_constant__ CUtensorMap tmB, const SlicedGemmArgs args) {
  using Cfg = GemmCfg<NSLICE, BK, STAGES>;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ __align__(8) uint64_t acc_full_bar[2];
  __shared__ __align__(8) uint64_t acc_empty_bar[2];
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_flag;

  // uniform: same word for all threads (a grouped launch skips per product instead)
  if (!GROUPED && args.skip != nullptr && *args.skip != 0) return;

  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  double* staging_all = reinterpret_cast<double*>(smem + STAGES * Cfg::kStageBytes);

  int nunits;
  if constexpr (GROUPED) {
    nunits = args.group_units;
  } else {
    const int tn = args.tiles_n;
    const int ntiles = (args.mode & kGemmSym) ? tn * (tn + 1) / 2 : args.tiles_m * tn;
    nunits = args.split > 1 ? args.full_tiles + (ntiles - args.full_tiles) * args.split : ntiles;
  }
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t ncols = static_cast<uint32_t>(args.tmem_cols);
  // two accumulator sets when a set takes at most half of TMEM (at most 2 orders): the MMAs of
  // the next tile then run while the epilogue drains this one
  const int nbuf = (args.nacc * kBN * 2 <= args.tmem_cols) ? 2 : 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full_bar[b], 1);
      mbar_init(&acc_empty_bar[b], kEpiWarps);
    }
    abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(&tmem_base_sh, ncols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base_sh;
  const int nk = (args.K + BK - 1) / BK;
  if (warp < kEpiWarp0) {
    // ---------------- control warpgroup: producer, MMA issuer, two idle warps ----------------
    setmaxnreg_dec<kCtrlRegs>();
  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer: one stage ring across all tiles of this CTA -----------
      if constexpr (!GROUPED) {
        tma_prefetch_desc(&tmA);
        tma_prefetch_desc(&tmB);
      }
      int it = 0;
      bool stop = false;
      for (int u = blockIdx.x; u < nunits && !stop; u += gridDim.x) {
        Unit w;
        decode_unit<GROUPED, BK>(u, args, nk, &tmA, &tmB, w);
        if (w.skip) continue;
        const int ti = w.ti, tj = w.tj;
        for (int kb = w.kb0; kb < w.kb1; ++kb) {
          if (!kstage_active(args.mask_a, args.mask_b, args.mask_ld, ti, tj, kb, BK)) continue;
          const int s = it % STAGES;
          const uint32_t ph = (it / STAGES) & 1u;
          if (!mbar_wait_bounded(&empty_bar[s], ph ^ 1u, args.err, &abort_flag)) {
            stop = true;
            break;
          }
          mbar_arrive_expect_tx(&full_bar[s], Cfg::kStageBytes);
          uint8_t* st = smem + s * Cfg::kStageBytes;
          tma_load_3d(st, w.ma, &full_bar[s], kb * BK, ti * kBM, 0);
          tma_load_3d(st + NSLICE * Cfg::kTileBytes, w.mb, &full_bar[s], kb * BK, tj * kBN, 0);
          ++it;
        }
      }
      if (stop) {
        // let copies already in flight land before the CTA can exit
        for (int j = (it > STAGES ? it - STAGES : 0); j < it; ++j)
          mbar_wait_bounded(&full_bar[j % STAGES], (j / STAGES) & 1u, nullptr, nullptr,
                            100000000ull);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer (one thread) ----------------
      // Everything but the stage base is fixed per launch: per-instruction descriptor offsets
      // (16-byte units), accumulator columns, instruction descriptors (N = 128 or 256) and
      // whether the instruction opens its accumulators; the unrolled issue loop is then two adds
      // per MMA.
      const uint32_t idesc_n[2] = {idesc_f16_f32(kBM, kBN), idesc_f16_f32(kBM, 2 * kBN)};
      const uint64_t desc_fixed = smem_desc(0u, BK);
      uint32_t offa[kPairsUsed], offb[kPairsUsed], dcol[kPairsUsed], opens[kPairsUsed],
          idsc[kPairsUsed];
      const int ni = args.num_ins;
#pragma unroll
      for (int p = 0; p < kPairsUsed; ++p) {
        const int pp = p < ni ? p : 0;
        offa[p] = (static_cast<uint32_t>(args.ins_s[pp]) * Cfg::kTileBytes) >> 4;
        offb[p] = (static_cast<uint32_t>(args.ins_t[pp]) * Cfg::kTileBytes) >> 4;
        dcol[p] = static_cast<uint32_t>((args.ins_s[pp] + args.ins_t[pp]) * kBN);
        opens[p] = static_cast<uint32_t>(args.ins_open[pp]);
        idsc[p] = idesc_n[args.ins_wide[pp] ? 1 : 0];
      }
      int it = 0, tcount = 0;
      unsigned long long issued = 0;
      bool stop = false;
      // tcount counts the units this CTA computes (skipped ones take no accumulator set)
      for (int u = blockIdx.x; u < nunits && !stop; u += gridDim.x) {
        Unit w;
        decode_unit<GROUPED, BK>(u, args, nk, &tmA, &tmB, w);
        if (w.skip) continue;
        const int buf = tcount % nbuf, use = tcount / nbuf;
        ++tcount;
        if (use > 0 &&
            !mbar_wait_bounded(&acc_empty_bar[buf], (use - 1) & 1u, args.err, &abort_flag)) {
          stop = true;
          break;
        }
        tc_fence_after();
        const uint32_t tacc = tbase + static_cast<uint32_t>(buf * args.nacc * kBN);
        const int ti = w.ti, tj = w.tj, kb0 = w.kb0, kb1 = w.kb1;
        for (int kb = kb0; kb < kb1; ++kb) {
          if (!kstage_active(args.mask_a, args.mask_b, args.mask_ld, ti, tj, kb, BK)) continue;
          const int s = it % STAGES;
          const uint32_t ph = (it / STAGES) & 1u;
          if (!mbar_wait_bounded(&full_bar[s], ph, args.err, &abort_flag)) {
            stop = true;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(smem + s * Cfg::kStageBytes);
          const uint64_t ad0 = desc_fixed | static_cast<uint64_t>((a0 >> 4) & 0x3FFFu);
          const uint64_t bd0 =
              desc_fixed | static_cast<uint64_t>(((a0 + NSLICE * Cfg::kTileBytes) >> 4) & 0x3FFFu);
          // instruction outer, k step inner: consecutive MMAs read adjacent 32-byte columns of
          // the same 128-byte operand rows (measured: the k-step-outer order runs 2.5x slower)
#pragma unroll
          for (int p = 0; p < kPairsUsed; ++p) {
            if (p < ni) {
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk) {
                const uint32_t acc = (kb > kb0 || kk > 0 || opens[p] == 0u) ? 1u : 0u;
                umma_f16(tacc + dcol[p], ad0 + offa[p] + 2u * kk, bd0 + offb[p] + 2u * kk,
                         idsc[p], acc);
              }
            }
          }
          umma_commit(&empty_bar[s]);  // stage reusable once these MMAs have read it
          ++it;
          ++issued;
        }
        umma_commit(&acc_full_bar[buf]);  // accumulators of this tile final (also on abort)
      }
      if (args.kcount != nullptr) atomicAdd(args.kcount, issued);
    }
  }
  } else {
    setmaxnreg_inc<kEpiRegs>();
    // ---------------- epilogue (warps 4..11) ----------------
    const int q = warp & 3;          // TMEM lane quarter this warp may access
    const int ew = warp - kEpiWarp0;
    const int half = ew >> 2;        // which 64 of the 128 columns
    double* stage = staging_all + ew * (32 * (kStageCols + 1));
    int tcount = 0;
    for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
      Unit w;
      decode_unit<GROUPED, BK>(u, args, nk, &tmA, &tmB, w);
      if (w.skip) continue;
      const SlicedGemmArgs& ep = *w.ep;  // this unit's product (args itself for one product)
      const int ti = w.ti, tj = w.tj, part = w.part, tile = w.tile;
      const bool sym = (ep.mode & kGemmSym) != 0;
      double alpha = ep.alpha, beta = ep.beta;
      if (ep.coef != nullptr) {
        alpha = ep.coef[0];
        beta = ep.coef[1];
      }
      int alpha_k = 0;
      bool alpha_neg = false;
      const bool pow2_alpha = pow2_scalar(alpha, alpha_k, alpha_neg);
      const int buf = tcount % nbuf, use = tcount / nbuf;
      ++tcount;
      const bool ok = mbar_wait_bounded(&acc_full_bar[buf], use & 1u, args.err, &abort_flag);
      const uint32_t tacc = tbase + static_cast<uint32_t>(buf * args.nacc * kBN);
      tc_fence_after();
      if (!ok || abort_flag) break;
      const bool diag_tile = (ti == tj);
      const int r0 = ti * kBM + q * 32;
      const int grow = r0 + lane;
      const double sa = (grow < ep.M) ? ep.row_scale_a[grow] : 0.0;
      const bool sa_ok = finite_bits(sa);
      const int ex_base = pow2_exponent(sa) - 22 - args.shift * (args.nacc - 1) +
                          (pow2_alpha ? alpha_k : 0);
      // finished integer sums T (row grow, 32 columns from ccol) -> C (and mirror / C^T)
      // (a loop over groups of 8 columns, not unrolled, with T shifted down by 8 after each
      // group: one copy of the per-element code, small enough for the instruction cache;
      // destroys T)
      auto store_chunk = [&](int ccol, long long (&T)[32]) {
        const int c0 = tj * kBN + ccol;
#pragma unroll 1
        for (int sc = 0; sc < 32 / kStageCols; ++sc) {
          // thread = row: finished values; mirror / transposed writes are coalesced here
#pragma unroll
          for (int jj = 0; jj < kStageCols; ++jj) {
            const int j = jj;
            const int gcol = c0 + sc * kStageCols + jj;
            double val = 0.0;
            if (grow < ep.M && gcol < ep.N) {
              const double sb = ep.row_scale_b[gcol];
              if (sa_ok && finite_bits(sb)) {
                const long long tv = (pow2_alpha && alpha_neg) ? -T[j] : T[j];
                val = scaled_int_to_double(tv, ex_base + pow2_exponent(sb));
                if (!pow2_alpha) val = fp64_scale(val, alpha);
              } else {
                // a NaN / Inf row scale marks a non-finite input row; bit-level propagation
                val = finite_bits(sa) ? sb : sa;
              }
              // FP64 arithmetic only where it is needed, in out-of-line calls behind uniform or
              // per-element tests (GB300 issues FP64 at about 1/64 of the FP32 rate, and an
              // if-converted FP64 instruction would run for every element)
              if (diag_tile && grow == gcol)
                val = diagonal_value(val, ep.diag_dot, ep.diag, grow, alpha);
              if (ep.D != nullptr)
                val = fp64_axpy(beta, ep.D[static_cast<int64_t>(gcol) * ep.ldd + grow], val);
              if (sym && grow < gcol) ep.C[static_cast<int64_t>(gcol) * ep.ldc + grow] = val;
              if (ep.Ct != nullptr) ep.Ct[static_cast<int64_t>(gcol) * ep.ldct + grow] = val;
            }
            stage[lane * (kStageCols + 1) + jj] = val;
          }
          __syncwarp();
          // 4 rows x 8 columns per store instruction: 64-byte row segments
          const int cc = lane % kStageCols;
          const int gcol = c0 + sc * kStageCols + cc;
#pragma unroll
          for (int rr = lane / kStageCols; rr < 32; rr += 32 / kStageCols) {
            const int row = r0 + rr;
            if (row < ep.M && gcol < ep.N && (!sym || row <= gcol))
              ep.C[static_cast<int64_t>(row) * ep.ldc + gcol] =
                  stage[rr * (kStageCols + 1) + cc];
          }
          __syncwarp();
#pragma unroll
          for (int j = 0; j < 32 - kStageCols; ++j) T[j] = T[j + kStageCols];
        }
      };
      // a split part leaves its sums in its workspace slot, column-major in the tile
      // (coalesced: lane = row); the last part to finish adds them up and stores the tile
      long long* wsp = nullptr;
      if (part >= 0)
        wsp = args.splitk_ws +
              (static_cast<int64_t>(tile - args.full_tiles) * args.split + part) * (kBM * kBN) +
              q * 32 + lane;
      // Every TMEM read of this warp first (its 64 columns, 16 per load, Horner in 2^shift with
      // order 0 first), then the accumulators are released, then the conversion and the stores
      // run while the MMAs of the next tile proceed.
      long long T0[32], T1[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        T0[j] = 0;
        T1[j] = 0;
      }
      const uint32_t trow = tacc + (static_cast<uint32_t>(q * 32) << 16) +
                            static_cast<uint32_t>(half * 64);
      for (int o = 0; o < args.nacc; ++o) {
        const uint32_t tcol = trow + static_cast<uint32_t>(o * kBN);
        uint32_t r[16];
        tmem_ld_32x32b_x16(tcol, r);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j) T0[j] = (T0[j] << args.shift) + f32_int_exact(r[j]);
        tmem_ld_32x32b_x16(tcol + 16u, r);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j) T0[16 + j] = (T0[16 + j] << args.shift) + f32_int_exact(r[j]);
        tmem_ld_32x32b_x16(tcol + 32u, r);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j) T1[j] = (T1[j] << args.shift) + f32_int_exact(r[j]);
        tmem_ld_32x32b_x16(tcol + 48u, r);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j) T1[16 + j] = (T1[16 + j] << args.shift) + f32_int_exact(r[j]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty_bar[buf]);
      if (wsp != nullptr) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          wsp[(half * 64 + j) * kBM] = T0[j];
          wsp[(half * 64 + 32 + j) * kBM] = T1[j];
        }
      } else {
        // one copy of the store code in the instruction stream
#pragma unroll 1
        for (int c = 0; c < 2; ++c) {
          store_chunk(half * 64 + 32 * c, T0);
          if (c == 0) {
#pragma unroll
            for (int j = 0; j < 32; ++j) T0[j] = T1[j];
          }
        }
      }
      if (wsp != nullptr) {
        // publish this part's sums, then count it in; no CTA ever waits for another
        __threadfence();
        __syncwarp();
        uint32_t* cnt = args.splitk_cnt + (tile - args.full_tiles) * kEpiWarps + ew;
        unsigned prev = 0u;
        if (lane == 0) prev = atomicAdd(cnt, 1u);
        prev = __shfl_sync(0xffffffffu, prev, 0);
        if (prev + 1u == static_cast<unsigned>(args.split)) {
          if (lane == 0) *cnt = 0u;  // every part has counted in: ready for the next launch
          __threadfence();
          const long long* wst =
              args.splitk_ws +
              static_cast<int64_t>(tile - args.full_tiles) * args.split * (kBM * kBN) + q * 32 +
              lane;
          for (int c = 0; c < 2; ++c) {
            const int ccol = half * 64 + c * 32;
            long long T[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) T[j] = 0;
            for (int pp = 0; pp < args.split; ++pp) {
#pragma unroll
              for (int j = 0; j < 32; ++j)
                T[j] += __ldcg(wst + static_cast<int64_t>(pp) * (kBM * kBN) + (ccol + j) * kBM);
            }
            store_chunk(ccol, T);
          }
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tbase, ncols);
  }
}

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// SMs of the current device (one persistent CTA each)
int device_sms() {
  int dev = 0;
  cudaGetDevice(&dev);
  static int cache[64] = {};
  if (dev < 0 || dev >= 64) dev = 0;
  if (cache[dev] == 0) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cache[dev] = n > 0 ? n : 148;
  }
  return cache[dev];
}

// 3-D map over slices: dims (K, rows, nslice), box (bk, 128, nslice), FP16, swizzle = bk*2 B.
bool make_slice_map(CUtensorMap* map, const SliceBuf& sb, int bk, int nslice) {
  EncodeTiledFn enc = get_encode_fn();
  if (!enc) return false;
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(sb.cols), static_cast<cuuint64_t>(sb.rows),
                        static_cast<cuuint64_t>(nslice)};
  cuuint64_t strides[2] = {static_cast<cuuint64_t>(sb.ld) * 2,
                           static_cast<cuuint64_t>(sb.ld) * sb.rows_alloc * 2};
  cuuint32_t box[3] = {static_cast<cuuint32_t>(bk), 128u, static_cast<cuuint32_t>(nslice)};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, const_cast<__half*>(sb.data), dims,
                   strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int NSLICE, int BK, int STAGES, bool GROUPED = false>
cudaError_t launch_cfg(const CUtensorMap& ta, const CUtensorMap& tb, const SlicedGemmArgs& a,
                       int grid, cudaStream_t stream) {
  using Cfg = GemmCfg<NSLICE, BK, STAGES>;
  auto kern = sliced_gemm_kernel<NSLICE, BK, STAGES, GROUPED>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(Cfg::kSmemBytes));
  if (e != cudaSuccess) return e;
  // the register split inside the kernel assumes exactly kLaunchRegs registers a thread at launch
  static const int regs = [&] {
    cudaFuncAttributes fa;
    return cudaFuncGetAttributes(&fa, kern) == cudaSuccess ? fa.numRegs : -1;
  }();
  if (regs != kLaunchRegs) return cudaErrorInvalidConfiguration;
  count_launch();
  const int sms = device_sms();
  const int blocks = grid < sms ? grid : sms;
  kern<<<blocks, kThreads, Cfg::kSmemBytes, stream>>>(ta, tb, a);
  return cudaGetLastError();
}

}  // namespace

namespace {
std::atomic<int64_t> g_launches{0};
}
void count_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

// Pair list for `nslice` slices and highest order `max_order`: all (s, t) with s, t < nslice
// and s + t <= max_order, ordered by order.
int build_pairs(int nslice, int max_order, SlicedGemmArgs* a) {
  int np = 0;
  for (int o = 0; o <= max_order; ++o)
    for (int s = 0; s <= o; ++s) {
      const int t = o - s;
      if (s < nslice && t < nslice && np < kMaxPairs) {
        a->pair_s[np] = static_cast<int8_t>(s);
        a->pair_t[np] = static_cast<int8_t>(t);
        a->pair_o[np] = static_cast<int8_t>(o);
        ++np;
      }
    }
  a->num_pairs = np;
  // MMA instructions: for each A slice s, the B slices t = 0, 1, ... in twos where both pairs
  // exist (one N = 256 MMA over B slices t and t+1, which are adjacent 128-row panels in shared
  // memory, into the adjacent accumulators of orders s+t and s+t+1), else one N = 128 MMA; a
  // two-slice MMA that would open one accumulator and add into the other is split.
  int ni = 0;
  uint32_t opened = 0;
  for (int s = 0; s < nslice; ++s) {
    for (int t = 0; t < nslice && s + t <= max_order && ni < kMaxPairs;) {
      const int o = s + t;
      bool wide = t + 1 < nslice && o + 1 <= max_order;
      if (wide && ((opened >> o) & 1u) != ((opened >> (o + 1)) & 1u)) wide = false;
      a->ins_s[ni] = static_cast<int8_t>(s);
      a->ins_t[ni] = static_cast<int8_t>(t);
      a->ins_wide[ni] = wide ? 1 : 0;
      a->ins_open[ni] = ((opened >> o) & 1u) ? 0 : 1;
      opened |= (wide ? 3u : 1u) << o;
      ++ni;
      t += wide ? 2 : 1;
    }
  }
  a->num_ins = ni;
  a->nacc = max_order + 1;
  a->tmem_cols = 512;  // at most 2 orders: two accumulator sets (double buffering)
  return np;
}

int sliced_gemm_bk(int nslice) { return (nslice >= 4) ? 32 : 64; }

cudaError_t sliced_gemm(const SliceBuf& A, const SliceBuf& B, const Precision& prec,
                        SlicedGemmArgs args, cudaStream_t stream) {
  const int nslice = prec.nslice;
  if (nslice < 1 || nslice > 4 || prec.max_order < 0 || prec.max_order > 3 ||
      prec.max_order > 2 * (nslice - 1))
    return cudaErrorInvalidValue;
  if (A.nslice_valid < nslice || B.nslice_valid < nslice) return cudaErrorInvalidValue;
  if ((nslice > 1 && (A.bits != prec.bits || B.bits != prec.bits))) return cudaErrorInvalidValue;
  args.shift = prec.bits;
  if (A.cols != B.cols) return cudaErrorInvalidValue;  // contraction length
  if (build_pairs(nslice, prec.max_order, &args) > kPairsUsed) return cudaErrorInvalidValue;
  args.M = A.rows;
  args.N = B.rows;
  args.K = A.cols;
  args.row_scale_a = A.row_scale;
  args.row_scale_b = B.row_scale;
  if ((args.mode & kGemmSym) && args.M != args.N) return cudaErrorInvalidValue;
  const int tm = (args.M + kBM - 1) / kBM;
  const int tn = (args.N + kBN - 1) / kBN;
  args.tiles_n = tn;
  args.tiles_m = tm;
  const int ntiles = (args.mode & kGemmSym) ? tn * (tn + 1) / 2 : tm * tn;
  if (ntiles == 0) return cudaSuccess;
  const int bk = sliced_gemm_bk(nslice);

  // k split of the last wave: with W whole waves of tiles over the SMs and `tail` tiles left,
  // the tail tiles run as `split` k-parts each (tail x split <= SMs), so the launch takes
  // W + 1/split tile times instead of W + 1 (n = 4096, symmetric: 528 tiles = 3 x 152 + 72,
  // split 2).  Not with tile masks (a part could skip all of its k blocks).
  args.split = 1;
  args.full_tiles = ntiles;
  const int sms = device_sms();
  const int nk = (args.K + bk - 1) / bk;
  if (args.splitk_ws != nullptr && args.splitk_cnt != nullptr &&
      args.mask_a == nullptr && args.mask_b == nullptr) {
    const int tail = ntiles % sms;
    int sp = tail > 0 ? sms / tail : 1;
    if (sp > 4) sp = 4;
    if (sp > nk) sp = nk;
    if (sp >= 2 && tail * sp <= args.splitk_slots && tail <= args.splitk_tiles) {
      args.split = sp;
      args.full_tiles = ntiles - tail;
    }
  }
  const int grid = args.split > 1 ? args.full_tiles + (ntiles - args.full_tiles) * args.split
                                  : ntiles;

  // 128-byte TMA lines (BK = 64) wherever two stages fit: the TMA's cost per stage grows with
  // its line count (~1.5 cycles per line) as much as with its bytes, so longer lines beat a
  // deeper ring (measured: 3 slices with BK = 64 and 2 stages run 13-17% faster than with
  // BK = 32 and 4 stages).  Four slices need BK = 32 to fit two or more stages.
  CUtensorMap ta, tb;
  if (!make_slice_map(&ta, A, bk, nslice) || !make_slice_map(&tb, B, bk, nslice))
    return cudaErrorInvalidValue;
  switch (nslice) {
    case 1: return launch_cfg<1, 64, 6>(ta, tb, args, grid, stream);
    case 2: return launch_cfg<2, 64, 3>(ta, tb, args, grid, stream);
    case 3: return launch_cfg<3, 64, 2>(ta, tb, args, grid, stream);
    default: return launch_cfg<4, 32, 3>(ta, tb, args, grid, stream);
  }
}

}  // namespace gdm

// ------------------------------------------------------------------------------------------
// grouped launches
// ------------------------------------------------------------------------------------------
namespace gdm {

namespace {
// (BK, stages) variants of the grouped kernel per slice count; variant 0 is the single
// product's configuration.  All fit the shared-memory budget (GemmCfg's static_assert).
struct GroupVariant {
  int bk, stages;
};
constexpr GroupVariant kGroupVariants[5][2] = {
    {{64, 6}, {64, 6}}, {{64, 6}, {64, 6}}, {{64, 3}, {32, 6}}, {{64, 2}, {32, 4}}, {{32, 3}, {32, 2}}};
}  // namespace

int grouped_variant_count(int nslice) { return (nslice >= 2 && nslice <= 4) ? 2 : 1; }

int grouped_variant_bk(int nslice, int variant) {
  if (nslice < 1 || nslice > 4) return 0;
  if (variant < 0 || variant >= grouped_variant_count(nslice)) variant = 0;
  return kGroupVariants[nslice][variant].bk;
}

cudaError_t sliced_gemm_group_item(const SliceBuf& A, const SliceBuf& Bt, const Precision& prec,
                                   const SlicedGemmArgs& args, GroupItem* item, int bk) {
  const int nslice = prec.nslice;
  if (nslice < 1 || nslice > 4) return cudaErrorInvalidValue;
  if (A.cols != Bt.cols) return cudaErrorInvalidValue;
  if (nslice > 1 && (A.bits != prec.bits || Bt.bits != prec.bits)) return cudaErrorInvalidValue;
  if ((args.mode & kGemmSym) && A.rows != Bt.rows) return cudaErrorInvalidValue;
  if (args.mask_a != nullptr || args.mask_b != nullptr) return cudaErrorInvalidValue;
  memset(item, 0, sizeof(*item));
  item->a = args;
  item->a.M = A.rows;
  item->a.N = Bt.rows;
  item->a.K = A.cols;
  item->a.row_scale_a = A.row_scale;
  item->a.row_scale_b = Bt.row_scale;
  item->a.tiles_m = (A.rows + kBM - 1) / kBM;
  item->a.tiles_n = (Bt.rows + kBN - 1) / kBN;
  item->a.split = 1;
  item->a.group = nullptr;
  if (!make_slice_map(&item->ta, A, bk, nslice) || !make_slice_map(&item->tb, Bt, bk, nslice))
    return cudaErrorInvalidValue;
  return cudaSuccess;
}

int group_assign_units(GroupItem* items, int count) {
  int u = 0;
  for (int i = 0; i < count; ++i) {
    const SlicedGemmArgs& a = items[i].a;
    items[i].a.unit_begin = u;
    u += (a.mode & kGemmSym) ? a.tiles_n * (a.tiles_n + 1) / 2 : a.tiles_m * a.tiles_n;
  }
  return u;
}

cudaError_t sliced_gemm_grouped(const GroupItem* items_dev, int count, int total_units,
                                const Precision& prec, uint32_t* err, cudaStream_t stream,
                                int variant) {
  const int nslice = prec.nslice;
  if (nslice < 1 || nslice > 4 || prec.max_order < 0 || prec.max_order > 3 ||
      prec.max_order > 2 * (nslice - 1))
    return cudaErrorInvalidValue;
  if (count <= 0 || total_units <= 0) return cudaSuccess;
  SlicedGemmArgs a;
  if (build_pairs(nslice, prec.max_order, &a) > kPairsUsed) return cudaErrorInvalidValue;
  a.shift = prec.bits;
  a.err = err;
  a.group = items_dev;
  a.ngroup = count;
  a.group_units = total_units;
  CUtensorMap unused;
  memset(&unused, 0, sizeof(unused));
  if (variant < 0 || variant >= grouped_variant_count(nslice)) variant = 0;
  switch (nslice * 10 + variant) {
    case 10: return launch_cfg<1, 64, 6, true>(unused, unused, a, total_units, stream);
    case 20: return launch_cfg<2, 64, 3, true>(unused, unused, a, total_units, stream);
    case 21: return launch_cfg<2, 32, 6, true>(unused, unused, a, total_units, stream);
    case 30: return launch_cfg<3, 64, 2, true>(unused, unused, a, total_units, stream);
    case 31: return launch_cfg<3, 32, 4, true>(unused, unused, a, total_units, stream);
    case 40: return launch_cfg<4, 32, 3, true>(unused, unused, a, total_units, stream);
    default: return launch_cfg<4, 32, 2, true>(unused, unused, a, total_units, stream);
  }
}

}  // namespace gdm
