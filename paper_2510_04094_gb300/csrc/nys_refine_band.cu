// Refinement row pass of the mixed path (Section 3.1's system, residuals from
// the definition of the problem) for kind LIN on narrow landmark windows.
//
// For the rows i of a work unit and z~ = (W^T omega, b) of the last solve:
//     s_i = r_i - sum_j kappa_ij z~_j - w1 z~_b,   acc_j = sum_i kappa_ij s_i,
//     acc_b = w1 sum_i s_i,
// with kappa_ij = kappa(i - idx_j) over the landmarks within the band
// u = ((t_i - s_j)/sigma)^2 <= kRefBandU (kernel values below 2^-46 of the
// peak dropped; k_refine_rows keeps u <= kLagU) and float-float arithmetic
// throughout, as in k_refine_rows; the unit's slot receives acc (m + 1
// doubles).
//
// A CTA (kRbWarps = 8 warps) takes one unit at a time:
//   * it folds kappa(lag), lag = -Kt..Kt (Kt = K + W - 1), into a float-float
//     table in shared memory, followed by W zeros, and loads z~;
//   * warp w takes windows w, w + 8, ... of W rows; lane l takes rows
//     row0 + l + 32 q.  A window sees at most kRbLm landmarks (the host's
//     plan): their z~ stay in registers; a first pass over the window's rows
//     forms s_i, a second adds kappa_ij s_i into per-lane accumulators;
//   * a float-float reduce-scatter over the warp leaves lane j with window
//     column j's sum (lane kRbLm with sum_i s_i), which it adds into the
//     warp's unit accumulator; after the unit the eight warps' accumulators
//     are added in a fixed order and stored.
// A window that breaks the plan (more landmarks than planned, a table larger
// than its space: a stale plan) sets the instance's status to NYS_ESTATE.
#include "nys_internal.cuh"

namespace nys {

constexpr int kRbThreads = 32 * kRbWarps;
constexpr int kRbSmemBytes =
    kRbTabCap * 8 + kM1Max * 8 + kRbWarps * kM1Max * 8 + kMMax * 4 + kRbWarps * kRbMaxW * 8;
static_assert((kRbTabCap * 8 + kM1Max * 8 + kRbWarps * kM1Max * 8 + kMMax * 4) % 8 == 0, "scratch alignment");
static_assert(kRbLm + 1 <= 32, "one reduced column per lane");
static_assert(kRbLm % 2 == 0, "columns in packed pairs");
static_assert(2 * (kRbSmemBytes + 1024) <= 228 * 1024, "two CTAs per SM");

size_t refine_band_smem_bytes() { return (size_t)kRbSmemBytes; }

// acc += a * b (float-float; exact leading product, TwoSum on the high parts,
// the rest gathered in the low part)
__device__ __forceinline__ void rb_fma(ff& acc, ff a, ff b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const float s = acc.hi + p;
  const float bb = s - acc.hi;
  const float err = (acc.hi - (s - bb)) + (p - bb);
  acc.hi = s;
  acc.lo += err + e;
}

__device__ __forceinline__ ff rb_norm(ff a) {
  const float hi = a.hi + a.lo;
  return {hi, a.lo - (hi - a.hi)};
}

// Two independent float-float multiply-adds in the packed FP32 pipe
// instructions (f32x2: one issue slot for both lanes of the pair, the same
// IEEE operations per element as rb_fma): acc.k += a.k * b.k, k = x, y.
struct ff2 { float2 hi, lo; };
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ void rb_fma2(ff2& acc, const ff2& a, const ff2& b) {
  const float2 p = __fmul2_rn(a.hi, b.hi);
  float2 e = __ffma2_rn(a.hi, b.hi, neg2(p));
  e = __ffma2_rn(a.hi, b.lo, e);
  e = __ffma2_rn(a.lo, b.hi, e);
  const float2 sm = __fadd2_rn(acc.hi, p);
  const float2 bb = __fadd2_rn(sm, neg2(acc.hi));
  const float2 err = __fadd2_rn(__fadd2_rn(acc.hi, neg2(__fadd2_rn(sm, neg2(bb)))),
                                __fadd2_rn(p, neg2(bb)));
  acc.hi = sm;
  acc.lo = __fadd2_rn(acc.lo, __fadd2_rn(err, e));
}

// One window (R = W / 32 rows per lane), in two passes over its rows so that
// few registers are live (four warps per scheduler hide the latencies):
//   1. s_i = r_i - sum_j kappa_ij z~_j - w1 z~_b (two interleaved chains), kept
//      in the warp's scratch (rows past r1 get s = 0);
//   2. acc_j += kappa_ij s_i (columns j, j+1 in packed instructions),
//      sum_s += s_i.
// Table loads are conflict-free: the lanes read consecutive lags.
__device__ __forceinline__ void rb_window(ff2* acc, ff& sum_s, const float2* __restrict__ tab,
                                          const int* base, const ff2* zr, ff w1zb,
                                          const RowConst& RK, int row0, int r1, int R, int lane,
                                          float2* scr) {
#pragma unroll 2
  for (int q = 0; q < R; ++q) {
    const int i = row0 + lane + 32 * q;
    ff sp0 = {0.f, 0.f}, sp1 = {0.f, 0.f};
#pragma unroll
    for (int j = 0; j < kRbLm; j += 2) {
      const float2 k0 = tab[base[j] + lane + 32 * q];
      const float2 k1 = tab[base[j + 1] + lane + 32 * q];
      rb_fma(sp0, ff{k0.x, k0.y}, ff{zr[j >> 1].hi.x, zr[j >> 1].lo.x});
      rb_fma(sp1, ff{k1.x, k1.y}, ff{zr[j >> 1].hi.y, zr[j >> 1].lo.y});
    }
    const ff spv = ff_add(ff_add(rb_norm(sp0), rb_norm(sp1)), w1zb);
    ff sv = {0.f, 0.f};
    if (i < r1) sv = ff_add(ff{lin_rhs_ff(RK, i), 0.f}, ff{-spv.hi, -spv.lo});
    scr[32 * q + lane] = make_float2(sv.hi, sv.lo);
    sum_s = ff_add(sum_s, sv);
  }
#pragma unroll 2
  for (int q = 0; q < R; ++q) {
    const float2 s2 = scr[32 * q + lane];
    const ff2 sv = {make_float2(s2.x, s2.x), make_float2(s2.y, s2.y)};
#pragma unroll
    for (int j = 0; j < kRbLm; j += 2) {
      const float2 k0 = tab[base[j] + lane + 32 * q];
      const float2 k1 = tab[base[j + 1] + lane + 32 * q];
      rb_fma2(acc[j >> 1], ff2{make_float2(k0.x, k1.x), make_float2(k0.y, k1.y)}, sv);
    }
  }
}

// Float-float reduce-scatter of 32 values over the warp: afterwards lane l
// holds the warp sum of value l.
template <int H>
__device__ __forceinline__ void rb_rs_level(ff* v, int lane) {
  const bool up = (lane & H) != 0;
#pragma unroll
  for (int p = 0; p < H; ++p) {
    const ff lo = v[p], hi = v[p + H];
    const ff send = up ? lo : hi;
    const ff keep = up ? hi : lo;
    const ff got = {__shfl_xor_sync(0xffffffffu, send.hi, H), __shfl_xor_sync(0xffffffffu, send.lo, H)};
    v[p] = ff_add(keep, got);
  }
}

__global__ void __launch_bounds__(kRbThreads, 2)
k_refine_band(const Inst* __restrict__ insts, const Lset* __restrict__ lsets,
              const float* __restrict__ lag, const Work* __restrict__ work, int nwork,
              int* __restrict__ counter, const int32_t* __restrict__ lm_idx,
              const double* __restrict__ zs, int ZS, double* __restrict__ part,
              const int64_t* __restrict__ slot_off, int32_t* __restrict__ st_all,
              const int32_t* __restrict__ skip_in) {
  extern __shared__ __align__(16) unsigned char rb_raw[];
  float2* tab = reinterpret_cast<float2*>(rb_raw);                // [kRbTabCap]
  float2* zsh = tab + kRbTabCap;                                  // [kM1Max] z~ (float-float)
  float2* uacc = zsh + kM1Max;                                    // [kRbWarps][kM1Max]
  int* sidx = reinterpret_cast<int*>(uacc + kRbWarps * kM1Max);   // [kMMax]
  float2* scr = reinterpret_cast<float2*>(sidx + kMMax) + (threadIdx.x >> 5) * kRbMaxW;   // s_i of a window
  __shared__ int s_item, s_bad, s_dbad;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (;;) {
    if (tid == 0) { s_item = atomicAdd(counter, 1); s_bad = 0; s_dbad = 0; }
    __syncthreads();
    const int w = s_item;
    if (w >= nwork) break;
    const Work wk = work[w];
    const Inst& I = insts[wk.inst];
    const Lset& L = lsets[I.lset];
    const int m = I.m, K = min(refine_band_lag(I.hs, I.n), L.K), W = wk.e0, R = W >> 5;
    const int r0 = wk.r0, r1 = wk.r1;
    const int Kt = K + W - 1, ntab = 2 * Kt + 1;
    // instances that failed, or that an adaptive pass leaves out (skip_in)
    const bool skip = (st_all[wk.inst] != NYS_OK) || (skip_in && skip_in[wk.inst]);
    const bool fits = ntab + W <= kRbTabCap && W >= 32 && W <= kRbMaxW && (W & (W - 1)) == 0 &&
                      m <= kMMax;
    if (!skip && fits) {
      for (int j = tid; j < m; j += kRbThreads) sidx[j] = lm_idx[I.lm_off + j];
      for (int j = tid; j <= m; j += kRbThreads) {
        const ff z = ff_from_double(zs[(int64_t)wk.inst * ZS + j]);
        zsh[j] = make_float2(z.hi, z.lo);
      }
      for (int e = tid; e < kRbWarps * kM1Max; e += kRbThreads) uacc[e] = make_float2(0.f, 0.f);
      // kappa(+a), kappa(-a) = e(a) +- A1 b1(a), e(a) = A0 b0(a) + A2 b2(a), in
      // float-float from the lag tables (zero beyond lag K)
      const float* __restrict__ T = lag + L.lag_off;
      const ff A0 = I.rk.A0, A1 = I.rk.A1, A2 = I.rk.A2;
      for (int a0 = 0; a0 <= Kt; a0 += 2 * kRbThreads) {
        float t6[2][6];   // two lags per thread in flight
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int a = a0 + tid + k * kRbThreads;
#pragma unroll
          for (int c = 0; c < 6; ++c) t6[k][c] = (a <= K) ? __ldg(T + 6 * a + c) : 0.f;
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int a = a0 + tid + k * kRbThreads;
          if (a <= Kt) {
            const ff ev = ff_add(ff_mul_ff(A0, ff{t6[k][0], t6[k][1]}),
                                 ff_mul_ff(A2, ff{t6[k][4], t6[k][5]}));
            const ff od = ff_mul_ff(A1, ff{t6[k][2], t6[k][3]});
            const ff kp = ff_add(ev, od), km = ff_add(ev, ff{-od.hi, -od.lo});
            tab[Kt + a] = make_float2(kp.hi, kp.lo);
            tab[Kt - a] = make_float2(km.hi, km.lo);
          }
        }
      }
      for (int e = ntab + tid; e < ntab + W; e += kRbThreads) tab[e] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    if (!skip && fits) {
      const RowConst RK = I.rk;
      const float2 zb2 = zsh[m];
      const ff w1zb = ff_mul_ff(RK.w1, ff{zb2.x, zb2.y});
      float2* ua = uacc + warp * kM1Max;
      int wlo = 0, whi = 0;
      for (int row0 = r0 + warp * W; row0 < r1; row0 += kRbWarps * W) {
        // landmarks with idx in [row0 - K, row0 + W - 1 + K]
        while (wlo < m && sidx[wlo] < row0 - K) ++wlo;
        if (whi < wlo) whi = wlo;
        while (whi < m && sidx[whi] <= row0 + W - 1 + K) ++whi;
        const int A = whi - wlo;
        if (A > kRbLm) {
          if (lane == 0) s_bad = 1;
          break;
        }
        int base[kRbLm];
        ff2 zr[kRbLm / 2], acc[kRbLm / 2];
        bool tab_ok = true;   // every table read inside the CTA's table (debug builds)
#pragma unroll
        for (int j = 0; j < kRbLm; j += 2) {
          float2 z[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const bool in = j + h < A;
            base[j + h] = in ? Kt + row0 - sidx[wlo + j + h] : ntab;
            tab_ok = tab_ok && NYS_IDX_OK(base[j + h] >= 0 && base[j + h] + W <= kRbTabCap);
            z[h] = in ? zsh[wlo + j + h] : make_float2(0.f, 0.f);
          }
          zr[j >> 1] = ff2{make_float2(z[0].x, z[1].x), make_float2(z[0].y, z[1].y)};
          acc[j >> 1] = ff2{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        }
        if (!tab_ok) {
          if (lane == 0) s_dbad = 1;
          break;
        }
        ff sum_s = {0.f, 0.f};
        rb_window(acc, sum_s, tab, base, zr, w1zb, RK, row0, r1, R, lane, scr);
        // 32 values: the window columns, sum_s, zero padding; lane l ends with value l
        ff v[32];
#pragma unroll
        for (int j = 0; j < 32; ++j)
          v[j] = (j < kRbLm) ? rb_norm((j & 1) ? ff{acc[j >> 1].hi.y, acc[j >> 1].lo.y}
                                               : ff{acc[j >> 1].hi.x, acc[j >> 1].lo.x})
                             : (j == kRbLm ? rb_norm(sum_s) : ff{0.f, 0.f});
        rb_rs_level<16>(v, lane);
        rb_rs_level<8>(v, lane);
        rb_rs_level<4>(v, lane);
        rb_rs_level<2>(v, lane);
        rb_rs_level<1>(v, lane);
        const int col = (lane < A) ? wlo + lane : (lane == kRbLm ? m : -1);
        if (col >= 0 && NYS_IDX_OK(col <= m)) {
          ff add = v[0];
          if (lane == kRbLm) add = ff_mul_ff(RK.w1, add);     // acc_b = w1 sum_i s_i
          const float2 cur = ua[col];
          const ff t = ff_add(ff{cur.x, cur.y}, add);
          ua[col] = make_float2(t.hi, t.lo);
        }
        __syncwarp();
      }
    }
    __syncthreads();
    if (tid == 0 && !skip && (!fits || s_bad)) st_all[wk.inst] = NYS_ESTATE;
    if (tid == 0 && !skip && s_dbad) st_all[wk.inst] = NYS_EBOUNDS;
    double* out = part + slot_off[wk.slot];
    for (int j = tid; j <= m; j += kRbThreads) {
      double v = 0.0;
      if (!skip && fits) {
        ff t = {0.f, 0.f};
        for (int q = 0; q < kRbWarps; ++q) {
          const float2 u = uacc[q * kM1Max + j];
          t = ff_add(t, ff{u.x, u.y});
        }
        v = (double)t.hi + (double)t.lo;
      }
      out[j] = v;
    }
    __syncthreads();
  }
}

cudaError_t launch_refine_band(const Inst* insts, const Lset* lsets, const float* lag,
                               const Work* work, int nwork, int* counter, const int32_t* lm,
                               const double* zs, int ZS, double* part, const int64_t* slot_off,
                               int32_t* st, const int32_t* skip_in, int num_sms, cudaStream_t s) {
  if (nwork <= 0) return cudaSuccess;
  const size_t sm = refine_band_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(k_refine_band, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm);
  if (e != cudaSuccess) return e;
  const int grid = min(nwork, 2 * num_sms);
  k_refine_band<<<grid, kRbThreads, sm, s>>>(insts, lsets, lag, work, nwork, counter, lm, zs, ZS,
                                             part, slot_off, st, skip_in);
  return cudaGetLastError();
}

}  // namespace nys
