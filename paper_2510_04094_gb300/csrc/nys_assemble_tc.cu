// Fused assembly of Lemma 1's Gram (Section 3.1) on the tensor cores, mixed path.
//
// A work unit (instance, range of collocation rows) needs
// G = sum_i psi_i psi_i^T of the augmented rows psi_i = [kappa_i (landmark
// window); -f_p(t_i); r(t_i)]: a dense contraction over the rows, run as tcgen05
// MMAs (kind::tf32) with FP32 accumulators in tensor memory.  The unit is cut
// into sub-chunks, each with the narrow landmark window its rows see; a
// sub-chunk's Gram is added, in FP64, into the unit's Gram in shared memory,
// which is stored to the unit's slot after its last sub-chunk (slot format
// [first landmark, landmark count, packed upper Gram], read by k_solve).
//
// Precision.  Features are split into TF32 parts hi = rn_tf32(psi) and
// lo = rn_tf32(psi - hi); the Gram takes hi hi^T + hi lo^T + lo hi^T + lo lo^T,
// i.e. the products of psi to about FP32 accuracy.  The tensor core's FP32
// accumulation loses accuracy with the number of MMAs accumulated into one
// entry (measured: 16 MMA steps per entry left 4x the error of 4 steps), so a
// sub-chunk is cut short enough that no accumulator entry takes more than
// kTcMmaSteps MMA steps before the epilogue moves it into FP64.  This Gram only
// feeds the FP32 factor that the FP64-accurate refinement then corrects, so a
// window keeps the landmarks with exp(-u) >= e^-24 for one of its rows
// (u = ((t_i - s_j)/sigma)^2 <= kAsmBandU): the dropped values are below 2^-34
// of the kernel's peak, under the FP32 accumulation's own rounding.  The
// residual passes keep the FP64 band (u <= 80).
//
// Operand tile (one pipeline stage): 128 operand rows x 32 K positions of
// TF32, K-major, 128-byte swizzle (16 KB).  With a window of M2 = A + 2
// columns, slots are grouped in blocks of Bs = 16, 32 or 64 >= M2:
//   operand row rho = Bs (2 r + h) + j: row set r (R = 64 / Bs of them),
//   h = 0 (hi) or 1 (lo), slot j; K position k of row set r = collocation row
//   32 r + k of the stage.
// One 128 x 128 x 8 MMA with A = B = the tile adds, for each row set, the four
// hi/lo products of 8 rows to its diagonal 2Bs x 2Bs block of the accumulator
// (the off-diagonal blocks mix row sets and are not read): 32 rows per MMA at
// Bs = 16.  Windows of more than 64 columns (Bs = 128) put each slot on one
// operand row and the K positions as [hi rows 0-7 | lo 0-7 | hi 8-15 | lo 8-15]:
// three MMAs (hi.hi, hi.lo, lo.hi) per 8 rows accumulate G itself.
//
// Features.  On the uniform grid a landmark is a grid point, so a feature
// depends on the lag t_i - s_j = (i - idx_j) h only.  For constant
// coefficients (kind LIN) the producers fold kappa(lag) = A0 b0 + A1 b1 + A2 b2
// from the landmark set's lag tables (k_setup_lag) once per work unit into a
// table in shared memory, already split into hi/lo.  Every lane of a producer
// unit then reads its value from one shared-memory source per sub-chunk -- the
// table at its lag, the sub-chunk's split r(t_i), the -f_p cell or a zero cell
// -- advancing by a fixed stride per stage: one 8-byte load and two stores per
// operand pair, no branches.  Tabulated coefficients (kind TABLE), or a table
// larger than shared memory allows, evaluate each feature (FP32, MUFU
// exponential).
//
// Warp roles (persistent CTA per SM, all hand-offs through mbarriers):
//   * four setup warps take work units from the queue and prepare sub-chunks
//     into a ring of kTcSub buffers: window (advanced along the unit),
//     landmark indices, the split r(t_i) (and the row coefficients of kind
//     TABLE);
//   * kTcProducers producer warps write the operand tiles of a ring of
//     kTcStages stages: 64 warp-wide units per stage, one value per lane (hi and
//     lo stores fill 4 K positions x 8 operand rows, conflict-free);
//   * one issuer thread issues the MMAs of a sub-chunk into its accumulator
//     (one of kTcSub sets of 128 tensor-memory columns) and commits;
//   * four epilogue warps read a finished accumulator (tcgen05.ld), add the
//     hi/lo blocks and row sets, and add the sub-chunk Gram into the unit's
//     FP64 Gram; after the unit's last sub-chunk they store it.
// Every wait is bounded (wait_iter polls of <= 1 us each).  A role group that
// shares named barriers takes each go/stop decision collectively (one thread
// waits and publishes the outcome), so no warp leaves a barrier group alone.
// On timeout the kernel records an error word (reported as NYS_ETIMEOUT by the
// solve), lets its MMAs drain (bounded), frees its tensor memory and returns.
#include <algorithm>

#include "nys_internal.cuh"
#include "nys_tc.cuh"

namespace nys {

constexpr int kTcProducers = 8;                        // producer warps 0..7
constexpr int kTcProdThreads = 32 * kTcProducers;
constexpr int kTcIssuerWarp = kTcProducers;            // warp 8
constexpr int kTcEpiWarp0 = kTcProducers + 1;          // warps 9..12
constexpr int kTcSetupWarp0 = kTcProducers + 5;        // warps 13..16
constexpr int kTcSetupThreads = 128;
constexpr int kTcThreads = 32 * (kTcProducers + 5) + kTcSetupThreads;
constexpr int kTcStages = 5;
constexpr int kTcTileBytes = 16384;      // 128 operand rows x 32 K positions (TF32)
constexpr int kTcStageArea = kTcStages * kTcTileBytes;
constexpr int kTcSub = 4;                // sub-chunk ring = tensor-memory accumulator sets
constexpr int kTcSubRows = 256;          // longest sub-chunk
constexpr int kTcUnitsPerStage = 64;     // warp-wide units of a stage (one value per lane)
constexpr int kTcUnitsPerWarp = kTcUnitsPerStage / kTcProducers;
constexpr int kTcSLd = 65;               // epilogue staging stride (Bs <= 64, padded)
constexpr int kTcSBytes = 128 * kTcSLd * 4;
constexpr int kTcGuMax = (kMMax + 2) * (kMMax + 3) / 2;   // unit Gram entries (float2 each)
constexpr int kTcLmCap = 128;            // landmark indices per sub-chunk buffer
constexpr int kTcTabCap = 4096;          // kappa(lag) table entries (hi, lo)
constexpr uint32_t kTcSetCols = 128;
constexpr uint32_t kTcCols = kTcSub * kTcSetCols;   // the whole tensor memory of the SM
constexpr int kTcMmaSteps = 8;           // MMA steps per accumulator entry, at most
constexpr int kTcDrainIter = 1 << 22;    // final wait for the MMAs in flight
static_assert(kTcUnitsPerStage % kTcProducers == 0 && kTcProducers == 8,
              "the unit decoding below assumes 8 producer warps");

// dynamic shared memory layout (byte offsets from the 1024-aligned base)
constexpr int kTcOffS = kTcStageArea;                            // float  [128][kTcSLd]
constexpr int kTcOffTab = kTcOffS + kTcSBytes;                   // float2 [kTcTabCap]
constexpr int kTcOffGu = kTcOffTab + kTcTabCap * 8;              // float2 [kTcGuMax]
constexpr int kTcOffRs = kTcOffGu + (kTcGuMax * 8 + 15) / 16 * 16;   // float2 [kTcSub][kTcSubRows]
constexpr int kTcOffCo = kTcOffRs + kTcSub * kTcSubRows * 8;     // float4 [kTcSub][kTcSubRows]
constexpr int kTcOffLm = kTcOffCo + kTcSub * kTcSubRows * 16;    // int    [kTcSub][kTcLmCap]
constexpr int kTcOffCell = kTcOffLm + kTcSub * kTcLmCap * 4;     // float2 [kTcSub][2]: -f_p, 0
constexpr int kTcSmemUsed = kTcOffCell + kTcSub * 16;
static_assert(kTcOffTab % 8 == 0 && kTcOffGu % 8 == 0 && kTcOffRs % 8 == 0 && kTcOffCo % 16 == 0 &&
              kTcOffCell % 8 == 0, "alignment");
static_assert(kTcSmemUsed + 1024 + 2048 <= 227 * 1024, "shared memory of one CTA");

size_t asm_tc_smem_bytes() { return (size_t)kTcSmemUsed + 1024; }

// One sub-chunk (nst < 0: no more work).
struct TcSub {
  int nst;         // pipeline stages of the sub-chunk
  int Bs, N;       // slot block; MMA N (128, or M2 rounded up to 16 when Bs = 128)
  int A, M2;       // window landmarks, Gram columns (A + 2)
  int r0, nrows;   // first collocation row (0-based grid index), row count
  int joff;        // window start - unit window start
  int Au, jlo_u;   // unit window
  int first, last; // first / last sub-chunk of its unit
  int mode;        // 0: kappa table (kind LIN); 1: features evaluated, LIN; 2: kind TABLE
  int Kt;          // table: lags -Kt..Kt at entries 0..2Kt
  int Kset;        // lag tables of the landmark set cover lags 0..Kset
  int unit;        // work unit whose constants (below) the buffer holds
  int64_t slot_off, lag_off;
  float hsc, LA0, LB1, LB2, w1;    // evaluated features: scaled operator constants
  float A0, A1, A2;                // table: operator constants
};

__device__ __forceinline__ void bar_named(int id, int count) {
  asm volatile("bar.sync %0, %1;" :: "r"(id), "r"(count) : "memory");
}

// round to nearest TF32 (ties away from zero): the low 13 mantissa bits cleared
__device__ __forceinline__ float rn_tf32(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}
__device__ __forceinline__ float2 split_tf32(float v) {
  const float h = rn_tf32(v);
  return make_float2(h, rn_tf32(v - h));
}

// warp-uniform bounded wait: lane 0 polls (acquire), the warp barrier orders the
// other lanes' later accesses after it
__device__ __forceinline__ bool warp_wait(uint32_t mbar, uint32_t parity, int iters) {
  int ok = 0;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait_bounded(mbar, parity, iters) ? 1 : 0;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  __syncwarp();
  return ok != 0;
}

// The producer warps meet (bounded): each warp's accesses so far happen before
// every producer warp's accesses after it.  ph: this warp's count of meetings.
__device__ __forceinline__ bool prod_meet(uint64_t* bar, uint32_t& ph, int iters) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive(smem_u32(bar));
  const bool ok = warp_wait(smem_u32(bar), ph & 1u, iters);
  ++ph;
  return ok;
}

// landmark window of rows [r0, r1): indices j with |i - idx_j| <= K for a row i
__device__ __forceinline__ void lm_window(const int* idx, int m, int r0, int r1, int K, int& jlo,
                                          int& A) {
  int a = 0, b = m;
  while (a < b) { const int c = (a + b) >> 1; if (idx[c] < r0 - K) a = c + 1; else b = c; }
  jlo = a;
  b = m;
  while (a < b) { const int c = (a + b) >> 1; if (idx[c] <= r1 - 1 + K) a = c + 1; else b = c; }
  A = a - jlo;
}

// g += x in compensated FP32: g.x + g.y carries the running sum, g.y the
// rounding errors of the additions into g.x (error-free two-sum)
__device__ __forceinline__ void acc_comp(float2* p, float x) {
  float2 g = *p;
  const float s = __fadd_rn(g.x, x);
  const float z = __fsub_rn(s, g.x);
  g.y = __fadd_rn(g.y, __fadd_rn(__fsub_rn(g.x, __fsub_rn(s, z)), __fsub_rn(x, z)));
  g.x = s;
  *p = g;
}

__device__ __forceinline__ int slot_block(int M2) {
  return (M2 <= 16) ? 16 : (M2 <= 32 ? 32 : (M2 <= 64 ? 64 : 128));
}

// Operand offsets of unit k of producer warp `warp`: the row t0 of the stage,
// the slot j and the byte offsets of the lane's hi and lo words.
template <int BS>
__device__ __forceinline__ void unit_layout(int warp, int k, int lane, int& t0, int& j,
                                            uint32_t& oh, uint32_t& ol) {
  if (BS <= 64) {
    // u = warp + 8 k: row set r = u / BS, slot j = u % BS (warp-uniform); lane =
    // K position, so a store fills one whole 128-byte operand row
    const int u = warp + 8 * k;
    const int r = u / BS;
    j = u % BS;
    t0 = 32 * r + lane;
    const int rho = 2 * r * BS + j;                    // hi row; lo row rho + BS
    oh = ((uint32_t)(rho >> 3) << 10) + ((uint32_t)(rho & 7) << 7) +
         ((uint32_t)(((lane >> 2) ^ rho) & 7) << 4) + ((uint32_t)(lane & 3) << 2);
    ol = oh + (uint32_t)BS * 128u;                     // same row of its 8-row atom
  } else {
    // u = warp + 8 k: slot group g = u >> 2, row quad c = u & 3
    const int j8 = lane >> 2, w4 = lane & 3;
    const int u = warp + 8 * k;
    const int g = u >> 2, c = u & 3;
    const int qh = 4 * (c >> 1) + (c & 1), ql = qh + 2;
    t0 = 4 * c + w4;
    j = 8 * g + j8;
    oh = ((uint32_t)g << 10) + (j8 << 7) + (((qh ^ j8) & 7) << 4) + (w4 << 2);
    ol = ((uint32_t)g << 10) + (j8 << 7) + (((ql ^ j8) & 7) << 4) + (w4 << 2);
  }
}

// Producer work of one sub-chunk with slot block BS.  Per lane and unit one
// shared-memory source (kappa table at the lane's lag, split r(t_i), the -f_p
// cell or the zero cell) and its advance per stage; per stage the eight values
// are loaded first, then stored (the compiler cannot move loads past stores to
// the same array).
template <int BS>
__device__ __forceinline__ void produce_sub(const TcSub& M, int b, unsigned char* sm, int& gs,
                                            int warp, int lane, int wait_iter, uint64_t* s_full,
                                            uint64_t* s_empty, bool& late) {
  constexpr int SR = (BS <= 64) ? 2048 / BS : 16;      // rows per stage
  const int A = M.A, nrows = M.nrows, nst = M.nst, mode = M.mode;
  const int* lmb = reinterpret_cast<const int*>(sm + kTcOffLm) + b * kTcLmCap;
  uint32_t src[kTcUnitsPerWarp], step[kTcUnitsPerWarp], oh[kTcUnitsPerWarp], ol[kTcUnitsPerWarp];
  int t0s[kTcUnitsPerWarp], js[kTcUnitsPerWarp], dj[kTcUnitsPerWarp];
#pragma unroll
  for (int k = 0; k < kTcUnitsPerWarp; ++k) {
    unit_layout<BS>(warp, k, lane, t0s[k], js[k], oh[k], ol[k]);
    dj[k] = lmb[min(js[k], kTcLmCap - 1)];              // landmark index (used when j < A)
  }
  const uint32_t cell = kTcOffCell + 16u * b;          // [-f_p hi/lo, zero]
  const int lag_base = M.Kt + M.r0;
#pragma unroll
  for (int k = 0; k < kTcUnitsPerWarp; ++k) {
    const int j = js[k];
    if (j < A) {         // landmark: kappa(lag), lag = t_i - s_j in grid steps
      src[k] = kTcOffTab + 8u * (uint32_t)(lag_base + t0s[k] - dj[k]);
      step[k] = 8u * SR;
    } else if (j == A + 1) {                            // r(t_i)
      src[k] = kTcOffRs + 8u * (uint32_t)(b * kTcSubRows + t0s[k]);
      step[k] = 8u * SR;
    } else {                                            // -f_p, or zero padding
      src[k] = cell + (j == A ? 0u : 8u);
      step[k] = 0u;
    }
  }
  for (int k = 0; k < nst; ++k, ++gs) {
    const int st = gs % kTcStages;
    if (gs >= kTcStages && !late)   // the MMAs that read this stage must be done
      late = !warp_wait(smem_u32(&s_empty[st]), (uint32_t)(((gs / kTcStages) - 1) & 1), wait_iter);
    if (!late) {
      unsigned char* tile = sm + st * kTcTileBytes;
      float2 v[kTcUnitsPerWarp];
      if (mode == 0) {
#pragma unroll
        for (int q = 0; q < kTcUnitsPerWarp; ++q)
          v[q] = *reinterpret_cast<const float2*>(sm + src[q] + (uint32_t)k * step[q]);
      } else {
        // evaluated features: exp(-x^2) = 2^(-y^2), y = x sqrt(log2 e)
        const float4* co = reinterpret_cast<const float4*>(sm + kTcOffCo) + b * kTcSubRows;
        const float ic1 = 0.832554611157698f, ic2 = 0.693147180559945f;
#pragma unroll
        for (int q = 0; q < kTcUnitsPerWarp; ++q) {
          const int tc = max(0, min(t0s[q] + k * SR, nrows - 1));
          if (js[q] < A) {
            float A0 = M.LA0, B1 = M.LB1, B2 = M.LB2;
            if (mode == 2) {
              const float4 c4 = co[tc];
              A0 = c4.x; B1 = c4.y * ic1; B2 = -c4.z * ic2;
            }
            const float y = (float)(M.r0 + t0s[q] + k * SR - dj[q]) * M.hsc;
            const float nu = -y * y;
            v[q] = split_tf32(ex2_approx(nu) * fmaf(B2, nu, fmaf(B1, y, A0)));
          } else if (js[q] == A && mode == 2) {
            v[q] = split_tf32(co[tc].w);
          } else {
            v[q] = *reinterpret_cast<const float2*>(sm + src[q] + (uint32_t)k * step[q]);
          }
        }
      }
      if ((k + 1) * SR > nrows) {                       // rows past the end in this stage
#pragma unroll
        for (int q = 0; q < kTcUnitsPerWarp; ++q)
          if (t0s[q] + k * SR >= nrows) v[q] = make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int q = 0; q < kTcUnitsPerWarp; ++q) {
        *reinterpret_cast<float*>(tile + oh[q]) = v[q].x;
        *reinterpret_cast<float*>(tile + ol[q]) = v[q].y;
      }
    }
    fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0) mbar_arrive(smem_u32(&s_full[st]));
  }
}

__global__ void __launch_bounds__(kTcThreads, 1)
k_assemble_tc(const Inst* __restrict__ insts, const Lset* __restrict__ lsets,
              const float* __restrict__ lag, const Work* __restrict__ work, int nwork,
              int* __restrict__ counter, const int32_t* __restrict__ lm_idx,
              const double* __restrict__ ctab, double* __restrict__ part,
              const int64_t* __restrict__ slot_off, int32_t* __restrict__ err, int wait_iter) {
  extern __shared__ unsigned char tc_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(tc_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  float* S = reinterpret_cast<float*>(sm + kTcOffS);
  float2* tab = reinterpret_cast<float2*>(sm + kTcOffTab);
  float2* Gu = reinterpret_cast<float2*>(sm + kTcOffGu);   // unit Gram, compensated FP32
  float2* s_rs = reinterpret_cast<float2*>(sm + kTcOffRs);  // [kTcSub][kTcSubRows]
  float4* s_co = reinterpret_cast<float4*>(sm + kTcOffCo);  // [kTcSub][kTcSubRows]
  int* s_lm = reinterpret_cast<int*>(sm + kTcOffLm);        // [kTcSub][kTcLmCap]
  float2* s_cell = reinterpret_cast<float2*>(sm + kTcOffCell);   // [kTcSub][2]
  __shared__ __align__(8) uint64_t s_full[kTcStages], s_empty[kTcStages];
  __shared__ __align__(8) uint64_t s_ready[kTcSub], s_used[kTcSub], s_accf[kTcSub], s_afree[kTcSub];
  __shared__ __align__(8) uint64_t s_drain, s_pbar;
  __shared__ TcSub s_meta[kTcSub];
  __shared__ int s_uidx[kMMax];            // landmark indices of the setup warps' unit
  __shared__ uint32_t s_tmem;
  __shared__ int s_w, s_abort, s_eok[kTcSub], s_sok[kTcSub];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) tmem_alloc(smem_u32(&s_tmem), kTcCols);
  if (tid == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(smem_u32(&s_full[s]), kTcProducers);
      mbar_init(smem_u32(&s_empty[s]), 1);
    }
    for (int b = 0; b < kTcSub; ++b) {
      mbar_init(smem_u32(&s_ready[b]), kTcSetupThreads);
      mbar_init(smem_u32(&s_used[b]), kTcProducers + 1 + 4);   // producers, issuer, epilogue warps
      mbar_init(smem_u32(&s_accf[b]), 1);
      mbar_init(smem_u32(&s_afree[b]), 1);
    }
    mbar_init(smem_u32(&s_drain), 1);
    mbar_init(smem_u32(&s_pbar), kTcProducers);
    for (int b = 0; b < kTcSub; ++b) s_meta[b].unit = -1;
    mbar_fence_init();
    s_abort = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  if (warp < kTcProducers) {
    // =========================== producers ===========================
    int gs = 0;                                        // stages produced so far
    uint32_t pph = 0;                                  // meetings at s_pbar
    bool late = false;
    for (int s = 0;; ++s) {
      const int b = s % kTcSub;
      // each warp waits for the sub-chunk on its own; they meet only around a
      // kappa table rebuild (bounded mbarrier waits: a warp that gives up
      // cannot hold the others)
      late = !warp_wait(smem_u32(&s_ready[b]), (uint32_t)((s / kTcSub) & 1), wait_iter) ||
             *(volatile int*)&s_abort;
      if (late) break;
      const TcSub M = s_meta[b];
      if (M.nst < 0) break;
      if (M.first && M.mode == 0) {
        // kappa(lag), lag = -Kt..Kt, of this unit, once every producer is past
        // the previous unit's stages: A0 b0 + A1 b1 + A2 b2 from the landmark
        // set's lag tables (zero beyond lag Kset), split into hi/lo
        if (!prod_meet(&s_pbar, pph, wait_iter)) { late = true; break; }
        const float* T = lag + M.lag_off;
        for (int e = tid; e <= 2 * M.Kt; e += kTcProdThreads) {
          const int lg = e - M.Kt, a = lg < 0 ? -lg : lg;
          float v = 0.f;
          if (a <= M.Kset) {
            const float b1 = lg < 0 ? -T[6 * a + 2] : T[6 * a + 2];
            v = fmaf(M.A2, T[6 * a + 4], fmaf(M.A1, b1, M.A0 * T[6 * a]));
          }
          tab[e] = split_tf32(v);
        }
        if (!prod_meet(&s_pbar, pph, wait_iter)) { late = true; break; }
      }
      switch (M.Bs) {
        case 16: produce_sub<16>(M, b, sm, gs, warp, lane, wait_iter, s_full, s_empty, late); break;
        case 32: produce_sub<32>(M, b, sm, gs, warp, lane, wait_iter, s_full, s_empty, late); break;
        case 64: produce_sub<64>(M, b, sm, gs, warp, lane, wait_iter, s_full, s_empty, late); break;
        default: produce_sub<128>(M, b, sm, gs, warp, lane, wait_iter, s_full, s_empty, late); break;
      }
      __syncwarp();
      if (lane == 0 && !late) mbar_arrive(smem_u32(&s_used[b]));   // buffer b may be refilled
      if (late) break;
    }
    if (late && lane == 0) atomicExch(&s_abort, 1);
  } else if (warp >= kTcSetupWarp0) {
    // ============================== setup ==============================
    const int st = tid - 32 * kTcSetupWarp0;           // 0..127
    int w = -1;                                        // current unit
    int row = 0, ur0 = 0, r1 = 0, m = 0, Kb = 0, jlo_u = 0, Au = 0, mode = 0, Kt = 0;
    int wlo = 0, whi = 0;                              // window of the last sub-chunk
    int64_t uslot = 0;
    float cb = 1.f, sb = 0.f;                          // rotation of the sine by 128 rows
    Inst I;
    Lset LS;
    for (int s = 0;; ++s) {
      const int b = s % kTcSub;
      if (s >= kTcSub) {   // every consumer of sub-chunk s - kTcSub is done with buffer b
        if (st == 0)
          s_sok[b] = mbar_wait_bounded(smem_u32(&s_used[b]), (uint32_t)(((s / kTcSub) - 1) & 1), wait_iter) ? 1 : 0;
        bar_named(3, kTcSetupThreads);
        if (!s_sok[b]) { if (st == 0) atomicExch(&s_abort, 1); break; }
      }
      if (w < 0 || row >= r1) {                        // next work unit
        if (st == 0) s_w = *(volatile int*)&s_abort ? nwork : atomicAdd(counter, 1);
        bar_named(3, kTcSetupThreads);
        w = s_w;
        bar_named(3, kTcSetupThreads);                 // every thread has read s_w
        if (w >= nwork) {                              // sentinel for the consumers
          if (st == 0) s_meta[b].nst = -1;
          mbar_arrive(smem_u32(&s_ready[b]));
          break;
        }
        const Work wk = work[w];
        I = insts[wk.inst];
        LS = lsets[I.lset];
        m = I.m;
        row = ur0 = wk.r0;
        r1 = wk.r1;
        uslot = slot_off[wk.slot];
        // band of the sub-chunk windows: u = (k h / sigma)^2 <= kAsmBandU
        Kb = asm_band_lag(I.hs, I.n);
        Kt = Kb + kTcSubRows - 1;
        mode = (I.kind == NYS_COEF_LIN) ? ((2 * Kt + 1 <= kTcTabCap && lag != nullptr) ? 0 : 1) : 2;
        if (I.kind == NYS_COEF_LIN) {
          // sin and cos of 128 dth (dth reduced mod 2 pi on the host)
          const double be = remainder(128.0 * I.dth, 6.283185307179586476925286766559);
          sincosf((float)be, &sb, &cb);
        }
        for (int j = st; j < m; j += kTcSetupThreads) s_uidx[j] = lm_idx[I.lm_off + j];
        bar_named(3, kTcSetupThreads);
        lm_window(s_uidx, m, row, r1, Kb, jlo_u, Au);
        wlo = whi = jlo_u;
      }
      // window of rows [row, row + n_sub), advanced from the previous one (rows
      // only move forward inside a unit)
      int n_sub = min(kTcSubRows, r1 - row);
      while (wlo < m && s_uidx[wlo] < row - Kb) ++wlo;
      if (whi < wlo) whi = wlo;
      while (whi < m && s_uidx[whi] <= row + n_sub - 1 + Kb) ++whi;
      int jlo = wlo, A = whi - wlo;
      int Bs = slot_block(A + 2);
      // at most kTcMmaSteps MMA steps per accumulator entry
      const int cap = (Bs <= 64) ? kTcMmaSteps * 512 / Bs : 32;
      if (n_sub > cap) {
        n_sub = cap;
        lm_window(s_uidx, m, row, row + n_sub, Kb, jlo, A);
        Bs = slot_block(A + 2);
        // the running window is the exact one of the rows actually taken: the
        // kappa table covers the lags of window landmarks only
        wlo = jlo;
        whi = jlo + A;
      }
      const int M2 = A + 2;
      const int SR = (Bs <= 64) ? 2048 / Bs : 16;
      const RowConst RK = I.rk;
      for (int j = st; j < A; j += kTcSetupThreads) s_lm[b * kTcLmCap + j] = s_uidx[jlo + j];
      if (I.kind == NYS_COEF_LIN) {
        // r(t_i) = c sin(theta_i): one sine per thread, then a rotation by 128 rows
        if (st < n_sub) {
          float sn, cs;
          lin_sincos(RK, row + st, sn, cs);
          s_rs[b * kTcSubRows + st] = split_tf32(RK.c * sn);
          if (st + 128 < n_sub) s_rs[b * kTcSubRows + st + 128] = split_tf32(RK.c * fmaf(sn, cb, cs * sb));
        }
      } else {
        for (int t = st; t < n_sub; t += kTcSetupThreads) {
          ff c5[5];
          row_coef_ff(I, RK, ctab, row + t, c5);
          s_rs[b * kTcSubRows + t] = split_tf32(c5[4].hi);
          s_co[b * kTcSubRows + t] = make_float4(c5[0].hi, c5[1].hi, c5[2].hi, c5[3].hi);
        }
      }
      if (st == 0) {
        TcSub& M = s_meta[b];
        M.nst = (n_sub + SR - 1) / SR;
        M.Bs = Bs;
        M.N = (Bs <= 64) ? 128 : round_up(M2, 16);
        M.A = A;
        M.M2 = M2;
        M.r0 = row;
        M.nrows = n_sub;
        M.joff = jlo - jlo_u;
        M.first = (row == ur0) ? 1 : 0;
        M.last = (row + n_sub >= r1) ? 1 : 0;
        if (M.unit != w) {                             // the unit's constants
          M.unit = w;
          M.Au = Au;
          M.jlo_u = jlo_u;
          M.mode = mode;
          M.Kt = Kt;
          M.Kset = LS.K;
          M.slot_off = uslot;
          M.lag_off = LS.lag_off;
          M.hsc = (float)I.hs * 1.20112240878645f;
          M.LA0 = RK.A0.hi;
          M.LB1 = RK.A1.hi * 0.832554611157698f;
          M.LB2 = -RK.A2.hi * 0.693147180559945f;
          M.w1 = RK.w1.hi;
          M.A0 = RK.A0.hi;
          M.A1 = RK.A1.hi;
          M.A2 = RK.A2.hi;
          s_cell[2 * b] = split_tf32(RK.w1.hi);
          s_cell[2 * b + 1] = make_float2(0.f, 0.f);
        }
      }
      row += n_sub;
      mbar_arrive(smem_u32(&s_ready[b]));              // each thread: its writes are done
    }
  } else if (warp == kTcIssuerWarp) {
    // ============================= issuer =============================
    if (lane == 0) {
      int gs = 0;
      for (int s = 0;; ++s) {
        const int b = s % kTcSub;
        if (!mbar_wait_bounded(smem_u32(&s_ready[b]), (uint32_t)((s / kTcSub) & 1), wait_iter)) {
          atomicExch(&s_abort, 1);
          break;
        }
        const int nst = s_meta[b].nst, Bs = s_meta[b].Bs, N = s_meta[b].N;
        mbar_arrive(smem_u32(&s_used[b]));
        if (nst < 0) break;
        if (s >= kTcSub &&   // the epilogue has read this accumulator set
            !mbar_wait_bounded(smem_u32(&s_afree[b]), (uint32_t)(((s / kTcSub) - 1) & 1), wait_iter)) {
          atomicExch(&s_abort, 1);
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)b * kTcSetCols;
        const uint32_t idesc = tc_idesc_tf32(128, N);
        bool late = false;
        uint32_t acc = 0;
        for (int k = 0; k < nst; ++k, ++gs) {
          const int st = gs % kTcStages;
          if (!mbar_wait_bounded(smem_u32(&s_full[st]), (uint32_t)((gs / kTcStages) & 1), wait_iter)) {
            late = true;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(sm + st * kTcTileBytes);
          if (Bs <= 64) {
#pragma unroll
            for (int t = 0; t < 4; ++t) {              // 4 K steps of 8 positions
              const uint64_t da = tc_desc_sw128(a0 + 32u * t);
              tc_mma_tf32(d, da, da, idesc, acc);
              acc = 1;
            }
          } else {
#pragma unroll
            for (int gg = 0; gg < 2; ++gg) {           // rows 8 gg .. 8 gg + 7
              const uint64_t dh = tc_desc_sw128(a0 + 64u * gg);
              const uint64_t dl = tc_desc_sw128(a0 + 64u * gg + 32u);
              tc_mma_tf32(d, dh, dh, idesc, acc);
              acc = 1;
              tc_mma_tf32(d, dh, dl, idesc, 1u);
              tc_mma_tf32(d, dl, dh, idesc, 1u);
            }
          }
          tc_commit(smem_u32(&s_empty[st]));
        }
        if (late) { atomicExch(&s_abort, 1); break; }
        tc_commit(smem_u32(&s_accf[b]));
      }
      // every MMA issued by this thread has completed once this commit arrives
      tc_commit(smem_u32(&s_drain));
      mbar_wait_bounded(smem_u32(&s_drain), 0, kTcDrainIter);
    }
  } else {
    // ============================ epilogue (4 warps) ============================
    const int et = tid - 32 * kTcEpiWarp0;             // 0..127
    const int quad = warp & 3;                         // tensor-memory lane quarter
    const int rho = 32 * quad + lane;                  // operand row of this thread
    for (int s = 0;; ++s) {
      const int b = s % kTcSub;
      const uint32_t par = (uint32_t)((s / kTcSub) & 1);
      // one thread waits for the sub-chunk (its description, then its
      // accumulator) and publishes the outcome, so that the four warps take the
      // same path through their named barriers
      if (et == 0) {
        int ok = mbar_wait_bounded(smem_u32(&s_ready[b]), par, wait_iter) ? 1 : 0;
        if (ok && s_meta[b].nst >= 0)
          ok = mbar_wait_bounded(smem_u32(&s_accf[b]), par, wait_iter) ? 1 : 0;
        s_eok[b] = ok;
      }
      bar_named(2, 128);
      if (!s_eok[b]) { if (et == 0) atomicExch(&s_abort, 1); break; }
      const int nst = s_meta[b].nst;
      const int Bs = s_meta[b].Bs, A = s_meta[b].A, M2 = s_meta[b].M2;
      const int joff = s_meta[b].joff, Au = s_meta[b].Au;
      const int first = s_meta[b].first, last = s_meta[b].last, jlo_u = s_meta[b].jlo_u;
      const int64_t so = s_meta[b].slot_off;
      const int Nc = s_meta[b].N;
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&s_used[b]));   // this warp has read the description
      if (nst < 0) break;
      const int M2u = Au + 2, Eu = M2u * (M2u + 1) / 2;
      tc_fence_after();
      const uint32_t lanebase = tmem + (uint32_t)b * kTcSetCols + ((uint32_t)(32 * quad) << 16);
      if (Bs <= 64) {
        // lane rho = Bs (2 r + h) + j reads its row set's block: columns
        // 2 Bs r + l (hi) and 2 Bs r + Bs + l (lo), l < Bs
        const int r = rho / (2 * Bs);
        const uint32_t c0 = (uint32_t)(2 * Bs * r);
        for (int l0 = 0; l0 < Bs; l0 += 16) {
          uint32_t vh[16], vl[16];
          tmem_ld16_nowait(lanebase + c0 + (uint32_t)l0, vh);
          tmem_ld16_nowait(lanebase + c0 + (uint32_t)(Bs + l0), vl);
          tmem_wait_ld();
#pragma unroll
          for (int t = 0; t < 16; ++t)
            S[rho * kTcSLd + l0 + t] = __uint_as_float(vh[t]) + __uint_as_float(vl[t]);
        }
        if (first)
          for (int e = et; e < Eu; e += 128) Gu[e] = make_float2(0.f, 0.f);
        tc_fence_before();
        bar_named(2, 128);                             // accumulator read, S complete, Gu clear
        if (et == 0) mbar_arrive(smem_u32(&s_afree[b]));
        const int nq = 128 / Bs;                       // operand rows per slot (row sets x hi/lo)
        const int lb = (Bs == 16) ? 4 : (Bs == 32 ? 5 : 6);
        for (int e = et; e < Bs * Bs; e += 128) {
          const int j = e >> lb, l = e & (Bs - 1);
          if (l >= j && l < M2) {
            float sum = 0.f;
            for (int q = 0; q < nq; ++q) sum += S[(q * Bs + j) * kTcSLd + l];
            const int ju = (j < A) ? j + joff : Au + (j - A);
            const int lu = (l < A) ? l + joff : Au + (l - A);
            acc_comp(&Gu[ju * M2u - ju * (ju - 1) / 2 + (lu - ju)], sum);
          }
        }
      } else {
        if (first) {
          for (int e = et; e < Eu; e += 128) Gu[e] = make_float2(0.f, 0.f);
          bar_named(2, 128);
        }
        // lane rho = slot j holds row j of the sub-chunk Gram itself
        const int j = rho;
        for (int l0 = 0; l0 < Nc; l0 += 16) {
          uint32_t v[16];
          tmem_ld16_nowait(lanebase + (uint32_t)l0, v);
          tmem_wait_ld();
          if (j < M2) {
            const int ju = (j < A) ? j + joff : Au + (j - A);
#pragma unroll
            for (int t = 0; t < 16; ++t) {
              const int l = l0 + t;
              if (l >= j && l < M2) {
                const int lu = (l < A) ? l + joff : Au + (l - A);
                acc_comp(&Gu[ju * M2u - ju * (ju - 1) / 2 + (lu - ju)], __uint_as_float(v[t]));
              }
            }
          }
        }
        tc_fence_before();
        bar_named(2, 128);
        if (et == 0) mbar_arrive(smem_u32(&s_afree[b]));
      }
      bar_named(2, 128);                               // Gu updated, S free
      if (last) {
        // slot: [first landmark, landmark count, packed upper Gram of the unit]
        double* out = part + so;
        if (et == 0) { out[0] = (double)jlo_u; out[1] = (double)Au; }
        for (int e = et; e < Eu; e += 128) {
          const float2 g = Gu[e];
          out[2 + e] = (double)g.x + (double)g.y;
        }
        bar_named(2, 128);                             // Gu may be cleared for the next unit
      }
    }
  }

  if (tid == 0 && s_abort) atomicExch(err, 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, kTcCols);
}

cudaError_t launch_assemble_tc(const Inst* insts, const Lset* lsets, const float* lag,
                               const Work* work, int nwork, int* counter, const int32_t* lm,
                               const double* tab, double* part, const int64_t* slot_off,
                               int32_t* err, int num_sms, int wait_iter, cudaStream_t st) {
  const size_t sm = asm_tc_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(k_assemble_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm);
  if (e != cudaSuccess) return e;
  const int grid = nwork < num_sms ? nwork : num_sms;
  if (grid < 1) return cudaSuccess;
  k_assemble_tc<<<grid, kTcThreads, sm, st>>>(insts, lsets, lag, work, nwork, counter, lm, tab, part,
                                              slot_off, err, wait_iter);
  return cudaGetLastError();
}

// Rows per work unit of the tensor-core kernel: long ranges (a unit's Gram stays
// in shared memory across its sub-chunks, and its kappa table is built once),
// split enough to give every SM several units.
int64_t asm_tc_unit_rows(int64_t total_rows, int batch, int num_sms) {
  const int64_t target = std::max<int64_t>(batch, 4LL * num_sms);
  return std::max<int64_t>(kTcSubRows, (total_rows + target - 1) / target);
}

}  // namespace nys
