// Internal definitions shared by the sm_103a kernels of the Nystrom LS-SVM ODE solver.
// (Product code: none of this is used by, or uses, the CPU oracle.)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "nys.h"

namespace nys {

// Index checks of the debug build (compiled with NYS_DEBUG_CHECKS, see
// build.build(debug=True)): NYS_IDX_OK(cond) is the condition there and the
// constant true otherwise, so the release kernels carry no check.  A failed
// check skips its access and is reported per instance as NYS_EBOUNDS (the
// assembly through its error word, value kErrBounds; the setup through
// m_eff = kMeffBounds).
#ifdef NYS_DEBUG_CHECKS
#define NYS_IDX_OK(cond) (cond)
#else
#define NYS_IDX_OK(cond) true
#endif
constexpr int kErrBounds = 3;
// Largest estimated error, relative to the solution (omega, b), that the mixed
// path's last refinement pass may leave
constexpr double kRefineTrust = 1e-4;
// Default refinement: an instance whose estimated error after the base passes is
// above kRefineAgain (relative to (omega, b)) takes one more pass; the others
// skip it
constexpr double kRefineAgain = 1e-8;
constexpr int kMeffBounds = -2;


constexpr int kMMax = NYS_M_MAX_MIXED;    // landmarks, shared-memory kernels
constexpr int kMLarge = NYS_M_MAX;        // landmarks, global-workspace kernels (FP64)
constexpr int kNtRowState = 5;            // Newton row state: Fy, d, f_y, f_u + delta, e f_yu
constexpr int kM1Max = kMMax + 1;         // (omega, b)
constexpr int kM2Max = kMMax + 2;         // augmented row [kappa; -f_p; r]
constexpr int kMPMax = 120;               // kM2Max rounded up to a multiple of 8

struct ff { float hi, lo; };

// Constants of an instance in float-float (computed once on the host), so that
// the per-row work of the FP32 kernels needs no FP64 arithmetic or conversion.
struct RowConst {
  ff A0, A1, A2, w1;   // constant-coefficient operator (kind LIN)
  ff is, is2;          // 1/sigma, 1/sigma^2
  ff th0, dth;         // r(t_i) = c sin(th0 + i dth)
  float c;
};

// Device descriptor of one ODE instance (built on the host by nys_setup).
struct Inst {
  int32_t p, n, m, kind;
  int32_t lset;        // landmark set (shared Nystrom factor)
  int32_t slot_count;  // assembly row-pass partial slots of this instance
  int64_t slot_begin;  // first slot (slots of an instance are contiguous)
  int64_t rslot_begin; // refinement row-pass slots (own work list, larger chunks)
  int32_t rslot_count;
  int32_t bc;          // nys_conditions: 1 = boundary values y(t_1), y(t_n), rows 2..n-1
  int64_t lm_off;      // landmark grid indices (int32) in lm_idx[]
  int64_t tab_off;     // kind TABLE: (p+1) x n doubles in tab[]; else -1
  int64_t y_off;       // Newton: auxiliary y_i (n-1 doubles) in yaux[]
  double t0, h;        // t_i (0-based i) = t0 + i h
  double sigma, gamma;
  double v[4];         // condition values (p of them)
  double c[8];
  // derived constants (host-computed in FP64)
  double hs;           // h / sigma
  double th0, dth;     // LIN: omega*t0 + phi0 and omega*h, both reduced mod 2 pi
  RowConst rk;         // float-float operator constants (row_const, set by the host)
};

// A landmark set: m indices on a grid of n points with spacing h, kernel width
// sigma.  Slot b of the set array belongs to instance b; it is active when b is
// the first instance with this set (the others point to it through Inst::lset).
struct Lset {
  int32_t m, m_eff;    // m_eff written by the setup kernel
  int32_t n, K;        // K: largest tabulated lag, exp(-(K h/sigma)^2) < 1e-34
  int32_t active;
  int32_t omode;       // 1: ill-conditioned landmark kernel (smallest kept eigenvalue
                       // < kOmegaCond * largest; FP64 contexts: span beyond
                       // kKernelSpan / sqrt(n)): row passes project every row
                       // through W (omega coordinates) instead of accumulating in
                       // kernel coordinates, which would lose precision there
  int64_t lm_off;
  int64_t w_off;       // W: m x m doubles (rows k < m_eff used), row-major
  int64_t lag_off;     // lag tables (floats): 6 per lag k = 0..K, see k_setup_lag
  double hs;           // h / sigma
};
// Band of the FP32 assembly Grams: a window keeps the landmarks with
// ((t_i - s_j)/sigma)^2 <= kAsmBandU for one of its rows (exp(-16) < 2^-23,
// FP32's rounding: these Grams only precondition the FP64-accurate refinement).
constexpr double kAsmBandU = 16.0;
__host__ __device__ __forceinline__ int asm_band_lag(double hs, int n) {
  return (int)fmin(ceil(sqrt(kAsmBandU) / hs), (double)n);
}
// CUDA-core band assembly (k_assemble_band): landmark columns per window, kappa
// table capacity per warp (floats: 2 (Kb + W - 1) + 1 lags and W zeros), unit
// Gram columns (unit landmarks + 2).
constexpr int kBandLm = 14;
constexpr int kBandTabCap = 4096;
constexpr int kBandUnitCols = 48;
// Band refinement pass (k_refine_band): its residuals keep the landmarks with
// u = ((t_i - s_j)/sigma)^2 <= kRefBandU of a row (exp(-32) < 2^-46 relative
// to the kernel's peak: 2^22 below the FP32 factor's rounding, which the
// refinement removes, and 2^26 below the MIXED path's error bar); landmark
// columns per window, float-float kappa table capacity per CTA
// (2 (K + W - 1) + 1 lags and W zeros), longest window.
constexpr double kRefBandU = 32.0;
__host__ __device__ __forceinline__ int refine_band_lag(double hs, int n) {
  return (int)fmin(ceil(sqrt(kRefBandU) / hs), (double)(n - 1));
}
constexpr int kRbLm = 16;
constexpr int kRbTabCap = 8192;
constexpr int kRbMaxW = 512;
// warps per CTA of k_refine_band (two CTAs per SM)
constexpr int kRbWarps = 8;

// Largest lag whose kernel value is kept: (K hs)^2 <= kLagU.
constexpr double kLagU = 80.0;
constexpr double kOmegaCond = 1e-7;
// FP64 contexts: the kernel-coordinate Gram W G W^T rounds to about
// cond u sqrt(n) relative (cond = lambda_max / lambda_min of the kept
// eigenvalues, u = 2^-53, n rows); a set uses it only while that stays below
// 1e-11 (cond sqrt(n) <= 1e-11 / u), otherwise omega coordinates, whose
// per-row projection rounds like the definition's own phi = W k.
constexpr double kKernelSpan = 1e-11 * 9007199254740992.0;

// One unit of a row pass: rows i in [r0, r1) (0-based grid index, 1 <= i <= n-1).
struct Work {
  int32_t inst, r0, r1, slot;
  int32_t e0, e1;      // FP64 assembly: packed Gram entries [e0, e1) of the rows
                       // (one part of a Gram too large for one item), else 0, max
};

// Instances with m > kMMax (FP64, linear): their landmark sets are factored and
// their KKT systems solved in a global workspace (one area of `stride` doubles per
// listed instance, shared by the setup and the solve, which run one after the
// other), their Gram is assembled in entry parts and its row-chunk partials are
// summed by a separate many-CTA pass.
struct BigSet {
  const int32_t* ids = nullptr;   // device: the instances (== their landmark-set slots)
  int n = 0;
  double* ws = nullptr;           // device workspace, n x stride doubles
  int64_t stride = 0;
};
// FP64 assembly accumulators per thread for Grams of more than kMMax + 2 columns
// (the entries of one work item: kAsm64BigK x its 256 threads)
constexpr int kAsm64BigK = 26;
constexpr int kAsm64Span = kAsm64BigK * 256;

// Per-instance solve storage offsets (element offsets in the typed arenas).
struct SolveSlots {
  int64_t fac;   // factor arena (T): V[2][M1] R[2][2] H1[2][M1] L[N2][N2]
  int64_t x;     // FP64: x = (omega (m_eff), b), lambda (2)  -- stride xs
  int64_t z;     // FP64: z = W^T omega (m), b               -- kernel coordinates
  int64_t cw;    // FP64: C_omega (2 x M1) constraint rows in omega coordinates
};

// ---------------------------------------------------------------------------
// float-float helpers (Dekker / Knuth two-sum and FMA-based two-product)
// ---------------------------------------------------------------------------

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = ff_two_sum(a.hi, b.hi);
  float lo = s.lo + a.lo + b.lo;
  float hi = s.hi + lo;
  return {hi, lo - (hi - s.hi)};
}
// a (float, exact) times b (ff), added to acc (ff)
__device__ __forceinline__ ff ff_fma_f(float a, ff b, ff acc) {
  float p = a * b.hi;
  float pe = fmaf(a, b.hi, -p);
  pe = fmaf(a, b.lo, pe);
  ff s = ff_two_sum(acc.hi, p);
  float lo = s.lo + pe + acc.lo;
  float hi = s.hi + lo;
  return {hi, lo - (hi - s.hi)};
}
__device__ __forceinline__ ff ff_mul_ff(ff a, ff b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const float hi = p + e;
  return {hi, e - (hi - p)};
}
__host__ __device__ __forceinline__ ff ff_from_double(double x) {
  float hi = (float)x;
  return {hi, (float)(x - (double)hi)};
}
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// ---------------------------------------------------------------------------
// exp(-u) for u >= 0 in FP32 with an extra-precise argument (u_hi + u_lo).
// Cody-Waite range reduction u*log2(e) = n + f with ln2 split in two parts,
// exp(-r) on |r| <= ln2/2 by its Taylor polynomial to degree 7 (truncation
// error < 1.2e-8 relative), scaling by 2^n through the exponent field.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float exp_neg_accurate(float u_hi, float u_lo) {
  const float kLog2e = 1.44269504088896341f;
  const float kLn2Hi = 0.693145751953125f;        // 12 significant bits: n * kLn2Hi exact
  const float kLn2Lo = 1.42860682030941723e-06f;  // ln 2 - kLn2Hi
  if (u_hi > 103.0f) return 0.0f;                 // below the smallest subnormal
  float nf = rintf(u_hi * kLog2e);
  float r = fmaf(-nf, kLn2Hi, u_hi);
  r = fmaf(-nf, kLn2Lo, r);
  r = r + u_lo;                                   // exp(-u) = 2^-n exp(-r)
  float x = -r;
  // Horner form of sum_{k=0..7} x^k / k!
  float q = 1.0f / 5040.0f;
  q = fmaf(q, x, 1.0f / 720.0f);
  q = fmaf(q, x, 1.0f / 120.0f);
  q = fmaf(q, x, 1.0f / 24.0f);
  q = fmaf(q, x, 1.0f / 6.0f);
  q = fmaf(q, x, 0.5f);
  q = fmaf(q, x, 1.0f);
  q = fmaf(q, x, 1.0f);
  // times 2^-n; n in [0, 149]: split the scale to stay in the normal range
  int n = (int)nf;
  int n1 = n >> 1, n2 = n - n1;
  float s1 = __int_as_float((127 - n1) << 23);
  float s2 = __int_as_float((127 - n2) << 23);
  return (q * s1) * s2;
}

// Fast exp(-u) on the MUFU unit (approximate; used where the refinement
// corrects the result).
__device__ __forceinline__ float exp_neg_fast(float u) {
  return exp2f(-u * 1.44269504088896341f);
}

// ---------------------------------------------------------------------------
// Per-row ODE operator coefficients.  For row i:
//   kappa_j = k^(p) - sum_k f_k k^(p-k) = e_j (A0 + A1 x_j + A2 u_j),
//   x_j = (t_i - s_j)/sigma, u_j = x_j^2, e_j = exp(-u_j),
// because k' = -2 x/sigma e and k'' = (4u - 2)/sigma^2 e (Section 3).
//   p = 2: A0 = -f_2 - 2/sigma^2, A1 = 2 f_1/sigma, A2 = 4/sigma^2
//   p = 1: A0 = -f_1,             A1 = -2/sigma,   A2 = 0
// w1 = -f_p(t_i) (coefficient of b), rr = r(t_i).
// ---------------------------------------------------------------------------
struct RowCoef { double A0, A1, A2, w1, rr; };

__device__ __forceinline__ void coef_f(const Inst& I, const double* tab, int i, double& f1,
                                       double& f2, double& rr) {
  if (I.kind == NYS_COEF_TABLE) {
    const double* T = tab + I.tab_off;
    f1 = T[i];
    f2 = (I.p == 2) ? T[(int64_t)I.n + i] : 0.0;
    rr = T[(int64_t)I.p * I.n + i];
  } else {  // LIN: f_k = -a_k, r = c sin(omega t + phi0)
    f1 = -I.c[0];
    f2 = (I.p == 2) ? -I.c[1] : 0.0;
    rr = 0.0;  // filled by the caller's own sine evaluation
  }
}

__host__ __device__ __forceinline__ RowCoef row_coef_from_f(const Inst& I, double f1, double f2, double rr) {
  RowCoef R;
  const double is = 1.0 / I.sigma, is2 = is * is;
  if (I.p == 2) {
    R.A0 = -f2 - 2.0 * is2;
    R.A1 = 2.0 * f1 * is;
    R.A2 = 4.0 * is2;
    R.w1 = -f2;
  } else {
    R.A0 = -f1;
    R.A1 = -2.0 * is;
    R.A2 = 0.0;
    R.w1 = -f1;
  }
  R.rr = rr;
  return R;
}

// r(t_i) = c sin(theta_i), theta_i = th0 + i dth (LIN kind), in FP64.
__device__ __forceinline__ double lin_rhs_f64(const Inst& I, int i) {
  double t = I.t0 + (double)i * I.h;
  return I.c[2] * sin(I.c[3] * t + I.c[4]);
}

// Operator coefficients of row i for the FP64 row pass, any order p <= 4:
//   kappa_j(t_i) = exp(-x^2) (A0 + A1 x + A2 x^2 + A3 x^3 + A4 x^4),  x = (t_i - s_j)/sigma,
// from the kernel's t-derivatives k^(l) = (-1/sigma)^l H_l(x) exp(-x^2) (physicists'
// Hermite: H1 = 2x, H2 = 4x^2 - 2, H3 = 8x^3 - 12x, H4 = 16x^4 - 48x^2 + 12) and
// kappa = k^(p) - sum_{k=1..p} f_k k^(p-k) (Section 3.1); w1 = -f_p multiplies b.
struct RowCoef4 { double A[5], w1, rr; };

__device__ __forceinline__ RowCoef4 row_coef_f64(const Inst& I, const double* tab, int i) {
  double f[4] = {0.0, 0.0, 0.0, 0.0};
  RowCoef4 R;
  const int p = I.p;
  if (I.kind == NYS_COEF_TABLE) {
    const double* T = tab + I.tab_off;
    for (int k = 0; k < p; ++k) f[k] = T[(int64_t)k * I.n + i];
    R.rr = T[(int64_t)p * I.n + i];
  } else {  // LIN (p <= 2): f_k = -a_k, r = c sin(omega t + phi0)
    f[0] = -I.c[0];
    if (p == 2) f[1] = -I.c[1];
    R.rr = lin_rhs_f64(I, i);
  }
  double g[5] = {0.0, 0.0, 0.0, 0.0, 0.0};   // g_l = c_l (-1/sigma)^l, c_p = 1, c_{p-k} = -f_k
  const double ms = -1.0 / I.sigma;
  double pw = 1.0;
  for (int l = 0; l <= p; ++l) {
    g[l] = ((l == p) ? 1.0 : -f[p - l - 1]) * pw;
    pw *= ms;
  }
  R.A[0] = g[0] - 2.0 * g[2] + 12.0 * g[4];
  R.A[1] = 2.0 * g[1] - 12.0 * g[3];
  R.A[2] = 4.0 * g[2] - 48.0 * g[4];
  R.A[3] = 8.0 * g[3];
  R.A[4] = 16.0 * g[4];
  R.w1 = -f[p - 1];
  return R;
}

__host__ __device__ __forceinline__ RowConst row_const(const Inst& I) {
  RowConst K;
  double f1 = -I.c[0], f2 = (I.p == 2) ? -I.c[1] : 0.0, rr = 0.0;
  const RowCoef R = row_coef_from_f(I, f1, f2, rr);
  K.A0 = ff_from_double(R.A0);
  K.A1 = ff_from_double(R.A1);
  K.A2 = ff_from_double(R.A2);
  K.w1 = ff_from_double(R.w1);
  K.is = ff_from_double(1.0 / I.sigma);
  K.is2 = ff_from_double(1.0 / (I.sigma * I.sigma));
  K.th0 = ff_from_double(I.th0);
  K.dth = ff_from_double(I.dth);
  K.c = (float)I.c[2];
  return K;
}

// c sin(theta_i) in FP32 with a float-float argument: theta_i = th0 + i dth
// with th0 and dth reduced mod 2 pi on the host, the product i dth split exactly
// by FMA and the sum reduced again (Cody-Waite with 2 pi in two parts); about
// one FP32 ulp.
__device__ __forceinline__ float lin_rhs_ff(const RowConst& K, int i) {
  const float k2PiHi = 6.28318548202514648f;
  const float k2PiLo = -1.74845553e-07f;
  const float fi = (float)i;
  const float p = fi * K.dth.hi;
  float pe = fmaf(fi, K.dth.hi, -p);
  pe = fmaf(fi, K.dth.lo, pe);
  const ff th = ff_add(K.th0, ff{p, pe});
  const float k = rintf(th.hi * 0.159154943091895336f);
  const float a = fmaf(-k, k2PiHi, th.hi);
  const float b = fmaf(-k, k2PiLo, th.lo);
  const ff r = ff_two_sum(a, b);
  float s, cth;
  sincosf(r.hi, &s, &cth);
  return K.c * fmaf(cth, r.lo, s);
}

// sin and cos of theta_i = th0 + i dth (LIN right-hand side), argument in
// float-float and reduced mod 2 pi as in lin_rhs_ff
__device__ __forceinline__ void lin_sincos(const RowConst& K, int i, float& s, float& c) {
  const float k2PiHi = 6.28318548202514648f;
  const float k2PiLo = -1.74845553e-07f;
  const float fi = (float)i;
  const float p = fi * K.dth.hi;
  float pe = fmaf(fi, K.dth.hi, -p);
  pe = fmaf(fi, K.dth.lo, pe);
  const ff th = ff_add(K.th0, ff{p, pe});
  const float k = rintf(th.hi * 0.159154943091895336f);
  const float a = fmaf(-k, k2PiHi, th.hi);
  const float b = fmaf(-k, k2PiLo, th.lo);
  const ff r = ff_two_sum(a, b);
  float sn, cs;
  sincosf(r.hi, &sn, &cs);
  s = fmaf(cs, r.lo, sn);
  c = fmaf(-sn, r.lo, cs);
}

// Operator coefficients of row i in float-float (TABLE kind reads the FP64
// table and converts; LIN uses the constants).  Returns A0, A1, A2, w1, r.
__device__ __forceinline__ void row_coef_ff(const Inst& I, const RowConst& K,
                                            const double* __restrict__ tab, int i, ff* out) {
  if (I.kind == NYS_COEF_TABLE) {
    const double* T = tab + I.tab_off;
    const ff f1 = ff_from_double(T[i]);
    const ff f2 = (I.p == 2) ? ff_from_double(T[(int64_t)I.n + i]) : ff{0.f, 0.f};
    const ff rr = ff_from_double(T[(int64_t)I.p * I.n + i]);
    if (I.p == 2) {
      out[0] = ff_add(ff{-f2.hi, -f2.lo}, ff{-2.f * K.is2.hi, -2.f * K.is2.lo});
      const ff t = ff_mul_ff(f1, K.is);
      out[1] = ff{2.f * t.hi, 2.f * t.lo};
      out[2] = ff{4.f * K.is2.hi, 4.f * K.is2.lo};
      out[3] = ff{-f2.hi, -f2.lo};
    } else {
      out[0] = ff{-f1.hi, -f1.lo};
      out[1] = ff{-2.f * K.is.hi, -2.f * K.is.lo};
      out[2] = ff{0.f, 0.f};
      out[3] = ff{-f1.hi, -f1.lo};
    }
    out[4] = rr;
  } else {
    out[0] = K.A0; out[1] = K.A1; out[2] = K.A2; out[3] = K.w1;
    out[4] = ff{lin_rhs_ff(K, i), 0.f};
  }
}

__host__ __device__ __forceinline__ int round_up(int x, int a) { return (x + a - 1) / a * a; }

}  // namespace nys
