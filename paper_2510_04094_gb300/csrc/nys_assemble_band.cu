// Fused assembly of Lemma 1's Gram (Section 3.1) on the CUDA cores for narrow
// landmark windows, mixed path (kind LIN).
//
// G = sum_i psi_i psi_i^T over the collocation rows of a work unit, psi_i =
// [kappa_i (landmark window); -f_p(t_i); r(t_i)].  The RBF kernel is negligible
// beyond the band u = ((t_i - s_j)/sigma)^2 <= kAsmBandU, so the rows of a short
// window of W consecutive rows only see the landmarks within Kb grid steps of
// it.  When every window of an instance sees at most kBandLm landmarks (the
// host's band plan), psi has at most 16 nonzero columns per window and the
// Gram of a window is a 16 x 16 contraction over W rows: 136 FP32 products
// per row, which the CUDA cores do faster than the tensor cores can take them
// in the block-diagonal packing a 16-wide window needs.
//
// One warp per work unit (persistent grid, atomic queue of units):
//   * it folds kappa(lag) = A0 b0 + A1 b1 + A2 b2 for the lags -Kt..Kt the
//     unit's windows meet (the landmark set's lag tables, k_setup_lag) into a
//     table in its shared memory, followed by W zeros;
//   * lane l takes rows row0 + l + 32 q (q < W / 32) of each window: features
//     from the table (one conflict-free load per landmark column, the 32 lanes
//     reading consecutive lags), -f_p, and r(t_i) = c sin(theta_i) (exact
//     float-float argument every 64 rows per lane, rotations by 32 rows in
//     between); its 136 products accumulate in FP32 registers (packed pairs);
//   * after the window a butterfly reduce-scatter over the warp (shuffles) sums
//     the 32 lanes' accumulators, leaving each lane at most 5 distinct entries,
//     which it adds into the unit's Gram in shared memory in compensated FP32
//     (two-sum, so the unit sum is exact to about 2^-44 relative);
//   * after the unit's last window the warp stores the unit Gram to the unit's
//     slot: [first landmark, landmark count, packed upper Gram] (doubles), the
//     format of the tensor-core kernel, read by k_solve.
// Column layout of a window: slots 0..13 landmarks (slots past the window's
// landmark count read the zero block of the table), slot 14 = -f_p, slot 15 =
// r.  The per-row accumulation depth is W / 32 <= 16 products per lane before
// the exact-order reduction, well inside FP32's accuracy for a preconditioner
// Gram that the FP64-accurate refinement corrects.
//
// A window or unit that breaks the plan (more landmarks than planned, a table
// larger than its space) is skipped and recorded in the error word (value 2);
// the solve then reports NYS_ESTATE for every instance.  The host re-plans when
// nys_update changes sigma, so this only guards against a stale plan.
#include "nys_internal.cuh"

namespace nys {

constexpr int kBandWarps = 8;
constexpr int kBandThreads = 32 * kBandWarps;
constexpr int kBandSlots = kBandLm + 2;        // window columns
constexpr int kBandEnt = kBandSlots * (kBandSlots + 1) / 2;   // 136 accumulators
constexpr int kBandOut = 5;                    // entries per lane after the reduce-scatter
constexpr int kBandGuCols = kBandUnitCols;     // unit Gram columns, at most
constexpr int kBandGuEnt = kBandGuCols * (kBandGuCols + 1) / 2;
constexpr int kBandWarpBytes = kBandTabCap * 4 + kBandGuEnt * 8 + kBandGuCols * 4;
static_assert(kBandWarpBytes % 16 == 0, "warp area alignment");
static_assert(kBandWarps * kBandWarpBytes <= 227 * 1024, "shared memory of one CTA");
static_assert(kBandSlots == 16 && kBandLm % 2 == 0, "the accumulator pairing of BandAcc");

size_t asm_band_smem_bytes() { return (size_t)kBandWarps * kBandWarpBytes; }

// g += x in compensated FP32 (error-free two-sum into g.x, rounding errors
// collected in g.y)
__device__ __forceinline__ void band_acc(float2* p, float x) {
  float2 g = *p;
  const float s = __fadd_rn(g.x, x);
  const float z = __fsub_rn(s, g.x);
  g.y = __fadd_rn(g.y, __fadd_rn(__fsub_rn(g.x, __fsub_rn(s, z)), __fsub_rn(x, z)));
  g.x = s;
  *p = g;
}

// One level of the butterfly reduce-scatter: the lane keeps half of its N
// entries (the upper half when its `mask` bit is set), sends the other half
// to the lane `mask` away and adds what it receives.
template <int N, int MASK>
__device__ __forceinline__ void band_rs_level(float* v, int lane) {
  constexpr int H = (N + 1) / 2;
  const bool up = (lane & MASK) != 0;
#pragma unroll
  for (int p = 0; p < H; ++p) {
    const float lo = v[p];
    const float hi = (p + H < N) ? v[p + H] : 0.f;
    const float send = up ? lo : hi;
    const float keep = up ? hi : lo;
    v[p] = keep + __shfl_xor_sync(0xffffffffu, send, MASK);
  }
}

// The 136 accumulators of a window in registers: row j of the upper triangle
// (columns l >= j) as pairs (l, l+1) for even l, which the packed FP32
// instructions update two at a time, and for odd j the single (j, j) first.
// pr[] and sg[] hold the entries in the packed row-major order below.
struct BandAcc {
  float2 pr[64];
  float sg[8];
};
// flat packed row-major index of (j, l) -> position in BandAcc (compile-time)
__host__ __device__ constexpr int band_flat(int j, int l) { return j * kBandSlots - j * (j - 1) / 2 + (l - j); }

// Products of one row's features (fp[c] = (f[2c], f[2c+1])) into the accumulators
__device__ __forceinline__ void band_row(BandAcc& A, const float2* fp) {
  int q = 0;
#pragma unroll
  for (int j = 0; j < kBandSlots; ++j) {
    const float fj = (j & 1) ? fp[j >> 1].y : fp[j >> 1].x;
    if (j & 1) A.sg[j >> 1] = fmaf(fj, fj, A.sg[j >> 1]);
    const float2 fjj = make_float2(fj, fj);
#pragma unroll
    for (int l = (j + 1) & ~1; l < kBandSlots; l += 2, ++q) A.pr[q] = __ffma2_rn(fjj, fp[l >> 1], A.pr[q]);
  }
}

// The accumulators in the packed row-major order (a register renaming)
__device__ __forceinline__ void band_flatten(const BandAcc& A, float* v) {
  int q = 0;
#pragma unroll
  for (int j = 0; j < kBandSlots; ++j) {
    if (j & 1) v[band_flat(j, j)] = A.sg[j >> 1];
#pragma unroll
    for (int l = (j + 1) & ~1; l < kBandSlots; l += 2, ++q) {
      v[band_flat(j, l)] = A.pr[q].x;
      v[band_flat(j, l + 1)] = A.pr[q].y;
    }
  }
}

// theta advances by 32 dth to the lane's next row
__device__ __forceinline__ void band_rotate(float& sn, float& cs, float C32, float S32) {
  const float s2 = fmaf(sn, C32, cs * S32);
  cs = fmaf(cs, C32, -sn * S32);
  sn = s2;
}

// Rows of one full window: lane l takes rows row0 + l + 32 q, q < R (R known
// at compile time: the table loads use immediate offsets and can be issued
// ahead of the previous row's products).
template <int R>
__device__ __forceinline__ void band_window_full(BandAcc& acc, const float* __restrict__ tl,
                                                 const int* base, int lane, float w1, float cr,
                                                 float& sn, float& cs, float C32, float S32) {
  const float* p[kBandLm];
#pragma unroll
  for (int j = 0; j < kBandLm; ++j) p[j] = tl + base[j] + lane;
#pragma unroll
  for (int q = 0; q < R; ++q) {
    float2 fp[kBandSlots / 2];
#pragma unroll
    for (int j = 0; j < kBandLm; j += 2) fp[j >> 1] = make_float2(p[j][32 * q], p[j + 1][32 * q]);
    fp[kBandLm >> 1] = make_float2(w1, cr * sn);
    band_row(acc, fp);
    band_rotate(sn, cs, C32, S32);
  }
}

// The last window of a unit, which runs past its last row r1: rows >= r1
// contribute nothing.
__device__ __forceinline__ void band_window_tail(BandAcc& acc, const float* __restrict__ tl,
                                              const int* base, int R, int lane, int row0, int r1,
                                              float w1, float cr, float& sn, float& cs, float C32,
                                              float S32) {
  for (int q = 0; q < R; ++q) {
    const int o = lane + 32 * q;
    const bool ok = row0 + o < r1;
    float2 fp[kBandSlots / 2];
#pragma unroll
    for (int j = 0; j < kBandLm; j += 2)
      fp[j >> 1] = ok ? make_float2(tl[base[j] + o], tl[base[j + 1] + o]) : make_float2(0.f, 0.f);
    fp[kBandLm >> 1] = ok ? make_float2(w1, cr * sn) : make_float2(0.f, 0.f);
    band_row(acc, fp);
    band_rotate(sn, cs, C32, S32);
  }
}

__global__ void __launch_bounds__(kBandThreads, 1)
k_assemble_band(const Inst* __restrict__ insts, const Lset* __restrict__ lsets,
                const float* __restrict__ lag, const Work* __restrict__ work, int nwork,
                int* __restrict__ counter, const int32_t* __restrict__ lm_idx,
                double* __restrict__ part, const int64_t* __restrict__ slot_off,
                int32_t* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char band_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* wa = band_raw + (size_t)warp * kBandWarpBytes;
  float* tab = reinterpret_cast<float*>(wa);                               // [kBandTabCap]
  float2* Gu = reinterpret_cast<float2*>(wa + kBandTabCap * 4);            // [kBandGuEnt]
  int* uidx = reinterpret_cast<int*>(wa + kBandTabCap * 4 + kBandGuEnt * 8);   // [kBandGuCols]

  // the entries this lane holds after the reduce-scatter: e = off + p, and
  // their window columns (j, l), j <= l, packed row-major over 16 columns
  // (the halves kept at the five levels are 68, 34, 17, 9 and 5 entries; a lane
  // that took the upper half of an odd count holds one zero pad, which it skips:
  // the real entry of that position belongs to another lane)
  const int b0 = lane & 1, b1 = (lane >> 1) & 1;
  const int off = ((lane >> 4) & 1) * 68 + ((lane >> 3) & 1) * 34 + ((lane >> 2) & 1) * 17 +
                  b1 * 9 + b0 * 5;
  const int nreal = b0 ? (b1 ? 3 : 4) : 5;
  int oj[kBandOut], ol[kBandOut];
#pragma unroll
  for (int p = 0; p < kBandOut; ++p) {
    oj[p] = -1;
    ol[p] = -1;
    if (p < nreal) {
      int j = 0, rem = off + p;
      while (rem >= kBandSlots - j) { rem -= kBandSlots - j; ++j; }
      oj[p] = j;
      ol[p] = j + rem;
    }
  }

  for (;;) {
    int w = 0;
    if (lane == 0) w = atomicAdd(counter, 1);
    w = __shfl_sync(0xffffffffu, w, 0);
    if (w >= nwork) break;
    const Work wk = work[w];
    const Inst& I = insts[wk.inst];
    const Lset& LS = lsets[I.lset];
    const int n = I.n, m = I.m, W = wk.e0, R = W >> 5;
    const int r0 = wk.r0, r1 = wk.r1;
    const int Kb = asm_band_lag(I.hs, n);
    const int Kt = Kb + W - 1, Kset = LS.K;
    const int ntab = 2 * Kt + 1;
    const int* idx = lm_idx + I.lm_off;
    // unit window: landmarks with idx in [r0 - Kb, r1 - 1 + Kb]
    int a = 0, b = m;
    while (a < b) { const int c = (a + b) >> 1; if (idx[c] < r0 - Kb) a = c + 1; else b = c; }
    const int jlo_u = a;
    b = m;
    while (a < b) { const int c = (a + b) >> 1; if (idx[c] <= r1 - 1 + Kb) a = c + 1; else b = c; }
    const int Au = a - jlo_u, M2u = Au + 2, Eu = M2u * (M2u + 1) / 2;
    if (M2u > kBandGuCols || ntab + W > kBandTabCap ||
        (W != 32 && W != 64 && W != 128 && W != 256 && W != 512)) {
      if (lane == 0) atomicExch(err, 2);
      continue;
    }
    __syncwarp();   // the previous unit's reads of tab / Gu / uidx are done
    for (int j = lane; j < Au; j += 32) uidx[j] = idx[jlo_u + j];
    for (int e = lane; e < Eu; e += 32) Gu[e] = make_float2(0.f, 0.f);
    {
      // kappa(+a) and kappa(-a) from one read of b0, b1, b2 at lag a (b1 odd);
      // four lags per lane in flight
      const float A0 = I.rk.A0.hi, A1 = I.rk.A1.hi, A2 = I.rk.A2.hi;
      const float* __restrict__ T = lag + LS.lag_off;
      const int amax = min(Kt, Kset);
      for (int a0 = 0; a0 <= Kt; a0 += 128) {
        float t0[4], t1[4], t2[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int a = a0 + lane + 32 * k;
          const bool in = a <= amax;
          t0[k] = in ? __ldg(T + 6 * a) : 0.f;
          t1[k] = in ? __ldg(T + 6 * a + 2) : 0.f;
          t2[k] = in ? __ldg(T + 6 * a + 4) : 0.f;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int a = a0 + lane + 32 * k;
          if (a <= Kt) {
            const float ev = fmaf(A2, t2[k], A0 * t0[k]);
            tab[Kt + a] = fmaf(A1, t1[k], ev);
            tab[Kt - a] = fmaf(-A1, t1[k], ev);
          }
        }
      }
      for (int e = ntab + lane; e < ntab + W; e += 32) tab[e] = 0.f;   // zero block
    }
    const RowConst RK = I.rk;                          // in registers for the unit
    const float w1 = RK.w1.hi, cr = RK.c;
    float C32, S32;
    {
      const double be = remainder(32.0 * I.dth, 6.283185307179586476925286766559);
      sincosf((float)be, &S32, &C32);
    }
    __syncwarp();
    bool bad = false, dbad = false;
    int wlo = 0, whi = 0;                              // unit landmarks [wlo, whi) of the window
    float sn = 0.f, cs = 1.f;                          // sin, cos of theta at the lane's next row
    for (int row0 = r0, win = 0; row0 < r1; row0 += W, ++win) {
      while (wlo < Au && uidx[wlo] < row0 - Kb) ++wlo;
      if (whi < wlo) whi = wlo;
      while (whi < Au && uidx[whi] <= row0 + W - 1 + Kb) ++whi;
      const int A = whi - wlo;
      if (A > kBandLm) { bad = true; break; }
      // table position of lane 0's first row per column: kappa(i - s_j) sits at
      // Kt + i - idx_j; empty columns read the zero block at ntab
      int base[kBandLm];
      bool tab_ok = true;   // every table read inside the warp's table (debug builds)
#pragma unroll
      for (int j = 0; j < kBandLm; ++j) {
        base[j] = (j < A) ? Kt + row0 - uidx[wlo + j] : ntab;
        tab_ok = tab_ok && NYS_IDX_OK(base[j] >= 0 && base[j] + W <= kBandTabCap);
      }
      if (!tab_ok) { dbad = true; break; }
      // exact argument every 64 rows per lane (every 8 windows below 256
      // rows), rotations by 32 dth in between (a rotation adds about one FP32
      // rounding to sin and cos)
      if (win % (R >= 8 ? 64 / R : 8) == 0) lin_sincos(RK, row0 + lane, sn, cs);
      BandAcc bacc;
#pragma unroll
      for (int q = 0; q < 64; ++q) bacc.pr[q] = make_float2(0.f, 0.f);
#pragma unroll
      for (int q = 0; q < 8; ++q) bacc.sg[q] = 0.f;
      if (row0 + W <= r1) {
        switch (R) {
          case 16: band_window_full<16>(bacc, tab, base, lane, w1, cr, sn, cs, C32, S32); break;
          case 8: band_window_full<8>(bacc, tab, base, lane, w1, cr, sn, cs, C32, S32); break;
          case 4: band_window_full<4>(bacc, tab, base, lane, w1, cr, sn, cs, C32, S32); break;
          case 2: band_window_full<2>(bacc, tab, base, lane, w1, cr, sn, cs, C32, S32); break;
          default: band_window_full<1>(bacc, tab, base, lane, w1, cr, sn, cs, C32, S32); break;
        }
      } else {
        band_window_tail(bacc, tab, base, R, lane, row0, r1, w1, cr, sn, cs, C32, S32);
      }
      float acc[kBandEnt];
      band_flatten(bacc, acc);
      // reduce-scatter: 136 -> 68 -> 34 -> 17 -> 9 -> 5 entries per lane
      band_rs_level<136, 16>(acc, lane);
      band_rs_level<68, 8>(acc, lane);
      band_rs_level<34, 4>(acc, lane);
      band_rs_level<17, 2>(acc, lane);
      band_rs_level<9, 1>(acc, lane);
      // unit coordinates: landmark slot j < A -> (wlo + j), -f_p -> Au, r -> Au + 1
#pragma unroll
      for (int p = 0; p < kBandOut; ++p) {
        const int j = oj[p], l = ol[p];
        if (j < 0) continue;
        const int ju = (j < kBandLm) ? ((j < A) ? wlo + j : -1) : Au + (j - kBandLm);
        const int lu = (l < kBandLm) ? ((l < A) ? wlo + l : -1) : Au + (l - kBandLm);
        if (ju < 0 || lu < 0) continue;
        if (!NYS_IDX_OK(ju <= lu && lu < M2u)) { dbad = true; continue; }
        band_acc(&Gu[ju * M2u - ju * (ju - 1) / 2 + (lu - ju)], acc[p]);
      }
      __syncwarp();   // Gu entries move between lanes from one window to the next
    }
    dbad = __any_sync(0xffffffffu, dbad);
    if (dbad) {
      if (lane == 0) atomicExch(err, kErrBounds);
      continue;
    }
    if (bad) {
      if (lane == 0) atomicExch(err, 2);
      continue;
    }
    double* out = part + slot_off[wk.slot];
    if (lane == 0) { out[0] = (double)jlo_u; out[1] = (double)Au; }
    // the solve adds the unit Grams in FP32: one rounding of the compensated pair
    for (int e = lane; e < Eu; e += 32) {
      const float2 g = Gu[e];
      out[2 + e] = (double)(g.x + g.y);
    }
  }
}

cudaError_t launch_assemble_band(const Inst* insts, const Lset* lsets, const float* lag,
                                 const Work* work, int nwork, int* counter, const int32_t* lm,
                                 double* part, const int64_t* slot_off, int32_t* err, int num_sms,
                                 cudaStream_t st) {
  const size_t sm = asm_band_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(k_assemble_band, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm);
  if (e != cudaSuccess) return e;
  int grid = (nwork + kBandWarps - 1) / kBandWarps;
  if (grid > num_sms) grid = num_sms;
  if (grid < 1) return cudaSuccess;
  k_assemble_band<<<grid, kBandThreads, sm, st>>>(insts, lsets, lag, work, nwork, counter, lm, part,
                                                  slot_off, err);
  return cudaGetLastError();
}

}  // namespace nys
