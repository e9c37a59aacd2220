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
// (u = ((t_i - s_j)/sigma)^2 <= kTcBandU): the dropped values are below 2^-34
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
// table in shared memory, already split into hi/lo; a feature is then one
// table read.  Tabulated coefficients (kind TABLE), or a table larger than
// shared memory allows, evaluate each feature (FP32, MUFU exponential).
//
// Warp roles (persistent CTA per SM, all hand-offs through mbarriers):
//   * two setup warps take work units from the queue and prepare sub-chunks
//     into a ring of kTcSub buffers: window, landmark indices, r(t_i) of the
//     rows (and the row coefficients of kind TABLE);
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

constexpr int kTcProducers = 16;                       // producer warps 0..15
constexpr int kTcProdThreads = 32 * kTcProducers;
constexpr int kTcIssuerWarp = kTcProducers;            // warp 16
constexpr int kTcEpiWarp0 = kTcProducers + 1;          // warps 17..20
constexpr int kTcSetupWarp0 = kTcProducers + 5;        // warps 21, 22
constexpr int kTcSetupThreads = 64;
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
constexpr int kTcGuMax = (kMMax + 2) * (kMMax + 3) / 2;   // unit Gram entries (FP64)
constexpr int kTcLmCap = 128;            // landmark indices per sub-chunk buffer
constexpr int kTcTabCap = 4096;          // kappa(lag) table entries (hi, lo)
constexpr uint32_t kTcSetCols = 128;
constexpr uint32_t kTcCols = kTcSub * kTcSetCols;   // the whole tensor memory of the SM
constexpr double kTcBandU = 24.0;
constexpr int kTcMmaSteps = 8;           // MMA steps per accumulator entry, at most
constexpr int kTcDrainIter = 1 << 22;    // final wait for the MMAs in flight
static_assert(kTcUnitsPerStage % kTcProducers == 0, "units split evenly over producers");

// dynamic shared memory layout (offsets from the 1024-aligned base)
constexpr int kTcOffS = kTcStageArea;
constexpr int kTcOffTab = kTcOffS + kTcSBytes;                   // float2
constexpr int kTcOffCo = kTcOffTab + kTcTabCap * 8;              // float4
constexpr int kTcOffGu = kTcOffCo + kTcSub * kTcSubRows * 16;    // double
constexpr int kTcOffR = kTcOffGu + kTcGuMax * 8;
constexpr int kTcOffLm = kTcOffR + kTcSub * kTcSubRows * 4;
constexpr int kTcSmemUsed = kTcOffLm + kTcSub * kTcLmCap * 4;
static_assert(kTcOffTab % 8 == 0 && kTcOffCo % 16 == 0 && kTcOffGu % 8 == 0, "alignment");
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

// warp-uniform bounded wait (lane 0 polls)
__device__ __forceinline__ bool warp_wait(uint32_t mbar, uint32_t parity, int iters) {
  int ok = 0;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait_bounded(mbar, parity, iters) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
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

// Producer work of one sub-chunk with slot block BS: per warp, kTcUnitsPerWarp
// units per stage.  Operand offsets depend on BS only; the feature of a lane is
// a table read (mode 0) or evaluated (modes 1, 2).
template <int BS>
__device__ __forceinline__ void produce_sub(const TcSub& M, unsigned char* sm, const float2* tab,
                                            const float* rr, const float4* co, const int* lmb,
                                            int& gs, int warp, int lane, int wait_iter,
                                            uint64_t* s_full, uint64_t* s_empty, bool& late) {
  constexpr int SR = (BS <= 64) ? 2048 / BS : 16;      // rows per stage
  constexpr uint32_t kLoOff = (BS <= 64) ? (uint32_t)BS * 128u : 0u;
  const int j8 = lane >> 2, w4 = lane & 3;
  const int A = M.A, nrows = M.nrows, mode = M.mode;
  int u_t0[kTcUnitsPerWarp], u_kind[kTcUnitsPerWarp], u_ti[kTcUnitsPerWarp], u_step[kTcUnitsPerWarp];
  uint32_t u_oh[kTcUnitsPerWarp], u_ol[kTcUnitsPerWarp];
  bool u_plain[kTcUnitsPerWarp];
#pragma unroll
  for (int k = 0; k < kTcUnitsPerWarp; ++k) {
    const int u = warp + k * kTcProducers;
    int t0, j;
    uint32_t oh, ol;
    if (BS <= 64) {
      constexpr int ng = BS >> 3;
      const int q = u & 7, rg = u >> 3;
      const int g = rg % ng, r = rg / ng;
      t0 = 32 * r + 4 * q + w4;
      j = 8 * g + j8;
      oh = ((uint32_t)(((2 * r * BS) >> 3) + g) << 10) + (j8 << 7) + (((q ^ j8) & 7) << 4) + (w4 << 2);
      ol = oh + kLoOff;
    } else {
      const int g = u >> 2, c = u & 3;
      const int qh = 4 * (c >> 1) + (c & 1), ql = qh + 2;
      t0 = 4 * c + w4;
      j = 8 * g + j8;
      oh = ((uint32_t)g << 10) + (j8 << 7) + (((qh ^ j8) & 7) << 4) + (w4 << 2);
      ol = ((uint32_t)g << 10) + (j8 << 7) + (((ql ^ j8) & 7) << 4) + (w4 << 2);
    }
    u_t0[k] = t0;
    u_oh[k] = oh;
    u_ol[k] = ol;
    const int kd = (j < A) ? 0 : (j == A ? 1 : (j == A + 1 ? 2 : 3));
    u_kind[k] = kd;
    const int lag0 = M.r0 + t0 - lmb[max(0, min(j, A - 1))];   // t_i - s_j in grid steps
    // table index of stage 0 and its advance per stage (other slots: the centre)
    u_ti[k] = (kd == 0) ? lag0 : 0;
    u_step[k] = (kd == 0) ? SR : 0;
    // a unit whose 8 slots are all landmarks needs no per-lane selection
    u_plain[k] = (8 * ((j - j8) >> 3) + 7 < A);
  }
  const bool full = (nrows == M.nst * SR);               // no rows past the end
  const float w1h = rn_tf32(M.w1), w1l = rn_tf32(M.w1 - w1h);
  // evaluated features: sqrt(log2 e) scalings of the operator constants
  const float ic1 = 0.832554611157698f, ic2 = 0.693147180559945f;
  for (int k = 0; k < M.nst; ++k, ++gs) {
    const int st = gs % kTcStages;
    if (gs >= kTcStages && !late)   // the MMAs that read this stage must be done
      late = !warp_wait(smem_u32(&s_empty[st]), (uint32_t)(((gs / kTcStages) - 1) & 1), wait_iter);
    if (!late) {
      unsigned char* tile = sm + st * kTcTileBytes;
#pragma unroll
      for (int q = 0; q < kTcUnitsPerWarp; ++q) {
        const int t = u_t0[q] + k * SR;                  // row of the sub-chunk
        float hv, lv;
        if (mode == 0) {
          const float2 kv = tab[M.Kt + u_ti[q] + k * u_step[q]];
          hv = kv.x;
          lv = kv.y;
        } else {
          const int tc = max(0, min(t, nrows - 1));
          float A0 = M.LA0, B1 = M.LB1, B2 = M.LB2;
          if (mode == 2) {
            const float4 c4 = co[tc];
            A0 = c4.x; B1 = c4.y * ic1; B2 = -c4.z * ic2;
          }
          // exp(-x^2) = 2^(-y^2), y = x sqrt(log2 e), x = (t_i - s_j) / sigma
          const float y = (float)(u_ti[q] + k * u_step[q]) * M.hsc;
          const float nu = -y * y;
          const float v = ex2_approx(nu) * fmaf(B2, nu, fmaf(B1, y, A0));
          hv = rn_tf32(v);
          lv = rn_tf32(v - hv);
        }
        if (!u_plain[q]) {                               // warp-uniform
          const int kd = u_kind[q];
          if (kd != 0) {
            const int tc = max(0, min(t, nrows - 1));
            float sv = 0.f;
            if (kd == 1) sv = (mode == 2) ? co[tc].w : M.w1;
            else if (kd == 2) sv = rr[tc];
            if (kd == 1 && mode != 2) { hv = w1h; lv = w1l; }
            else { hv = rn_tf32(sv); lv = rn_tf32(sv - hv); }
          }
        }
        if (!full && t >= nrows) { hv = 0.f; lv = 0.f; }
        unsigned char* p = tile + u_oh[q];
        *reinterpret_cast<float*>(p) = hv;
        if (BS <= 64) *reinterpret_cast<float*>(p + kLoOff) = lv;
        else *reinterpret_cast<float*>(tile + u_ol[q]) = lv;
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
  double* Gu = reinterpret_cast<double*>(sm + kTcOffGu);
  float* s_r = reinterpret_cast<float*>(sm + kTcOffR);      // [kTcSub][kTcSubRows]
  float4* s_co = reinterpret_cast<float4*>(sm + kTcOffCo);  // [kTcSub][kTcSubRows]
  int* s_lm = reinterpret_cast<int*>(sm + kTcOffLm);        // [kTcSub][kTcLmCap]
  __shared__ __align__(8) uint64_t s_full[kTcStages], s_empty[kTcStages];
  __shared__ __align__(8) uint64_t s_ready[kTcSub], s_used[kTcSub], s_accf[kTcSub], s_afree[kTcSub];
  __shared__ __align__(8) uint64_t s_drain;
  __shared__ TcSub s_meta[kTcSub];
  __shared__ int s_uidx[kMMax];            // landmark indices of the setup warps' unit
  __shared__ uint32_t s_tmem;
  __shared__ int s_w, s_abort, s_eok, s_sok, s_pok[kTcSub];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) tmem_alloc(smem_u32(&s_tmem), kTcCols);
  if (tid == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(smem_u32(&s_full[s]), kTcProducers);
      mbar_init(smem_u32(&s_empty[s]), 1);
    }
    for (int b = 0; b < kTcSub; ++b) {
      mbar_init(smem_u32(&s_ready[b]), kTcSetupThreads);
      mbar_init(smem_u32(&s_used[b]), kTcProducers + 2);   // producers, issuer, epilogue
      mbar_init(smem_u32(&s_accf[b]), 1);
      mbar_init(smem_u32(&s_afree[b]), 1);
    }
    mbar_init(smem_u32(&s_drain), 1);
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
    bool late = false;
    for (int s = 0;; ++s) {
      const int b = s % kTcSub;
      // one thread waits for the sub-chunk and publishes the outcome (named
      // barrier 1 holds the whole producer group)
      if (tid == 0)
        s_pok[b] = (!*(volatile int*)&s_abort &&
                    mbar_wait_bounded(smem_u32(&s_ready[b]), (uint32_t)((s / kTcSub) & 1), wait_iter)) ? 1 : 0;
      bar_named(1, kTcProdThreads);
      if (!s_pok[b]) { if (tid == 0) atomicExch(&s_abort, 1); break; }
      const TcSub M = s_meta[b];
      if (M.nst < 0) break;
      if (M.first && M.mode == 0) {
        // kappa(lag), lag = -Kt..Kt, of this unit: every producer is past the
        // previous unit's stages (barrier above); A0 b0 + A1 b1 + A2 b2 from the
        // landmark set's lag tables (zero beyond lag Kset), split into hi/lo
        const float* T = lag + M.lag_off;
        for (int e = tid; e <= 2 * M.Kt; e += kTcProdThreads) {
          const int lg = e - M.Kt, a = lg < 0 ? -lg : lg;
          float v = 0.f;
          if (a <= M.Kset) {
            const float b1 = lg < 0 ? -T[6 * a + 2] : T[6 * a + 2];
            v = fmaf(M.A2, T[6 * a + 4], fmaf(M.A1, b1, M.A0 * T[6 * a]));
          }
          const float h = rn_tf32(v);
          tab[e] = make_float2(h, rn_tf32(v - h));
        }
        bar_named(1, kTcProdThreads);
      }
      const float* rr = s_r + b * kTcSubRows;
      const float4* co = s_co + b * kTcSubRows;
      const int* lmb = s_lm + b * kTcLmCap;
      switch (M.Bs) {
        case 16: produce_sub<16>(M, sm, tab, rr, co, lmb, gs, warp, lane, wait_iter, s_full, s_empty, late); break;
        case 32: produce_sub<32>(M, sm, tab, rr, co, lmb, gs, warp, lane, wait_iter, s_full, s_empty, late); break;
        case 64: produce_sub<64>(M, sm, tab, rr, co, lmb, gs, warp, lane, wait_iter, s_full, s_empty, late); break;
        default: produce_sub<128>(M, sm, tab, rr, co, lmb, gs, warp, lane, wait_iter, s_full, s_empty, late); break;
      }
      __syncwarp();
      if (lane == 0) {
        if (late) atomicExch(&s_abort, 1);
        mbar_arrive(smem_u32(&s_used[b]));             // sub-chunk buffer b may be refilled
      }
    }
  } else if (warp >= kTcSetupWarp0) {
    // ============================== setup ==============================
    const int st = tid - 32 * kTcSetupWarp0;           // 0..63
    int w = -1;                                        // current unit
    int row = 0, ur0 = 0, r1 = 0, m = 0, Kb = 0, jlo_u = 0, Au = 0, mode = 0, Kt = 0;
    int64_t uslot = 0;
    float cb = 1.f, sb = 0.f;                          // rotation of the sine by 64 rows
    Inst I;
    Lset LS;
    for (int s = 0;; ++s) {
      const int b = s % kTcSub;
      if (s >= kTcSub) {   // every consumer of sub-chunk s - kTcSub is done with buffer b
        if (st == 0)
          s_sok = mbar_wait_bounded(smem_u32(&s_used[b]), (uint32_t)(((s / kTcSub) - 1) & 1), wait_iter) ? 1 : 0;
        bar_named(3, kTcSetupThreads);
        const int ok = s_sok;
        bar_named(3, kTcSetupThreads);
        if (!ok) { if (st == 0) atomicExch(&s_abort, 1); break; }
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
        // band of the sub-chunk windows: u = (k h / sigma)^2 <= kTcBandU
        Kb = (int)fmin(ceil(sqrt(kTcBandU) / I.hs), (double)I.n);
        Kt = Kb + kTcSubRows - 1;
        mode = (I.kind == NYS_COEF_LIN) ? ((2 * Kt + 1 <= kTcTabCap && lag != nullptr) ? 0 : 1) : 2;
        if (I.kind == NYS_COEF_LIN) {
          // sin and cos of 64 dth (dth reduced mod 2 pi on the host)
          const double be = remainder(64.0 * I.dth, 6.283185307179586476925286766559);
          sincosf((float)be, &sb, &cb);
        }
        for (int j = st; j < m; j += kTcSetupThreads) s_uidx[j] = lm_idx[I.lm_off + j];
        bar_named(3, kTcSetupThreads);
        lm_window(s_uidx, m, row, r1, Kb, jlo_u, Au);
      }
      // sub-chunk length: at most kTcMmaSteps MMA steps per accumulator entry
      int n_sub = min(kTcSubRows, r1 - row);
      int jlo, A;
      lm_window(s_uidx, m, row, row + n_sub, Kb, jlo, A);
      int Bs = (A + 2 <= 16) ? 16 : (A + 2 <= 32 ? 32 : (A + 2 <= 64 ? 64 : 128));
      const int cap = (Bs <= 64) ? kTcMmaSteps * 512 / Bs : 32;
      if (n_sub > cap) {
        n_sub = cap;
        lm_window(s_uidx, m, row, row + n_sub, Kb, jlo, A);
        Bs = (A + 2 <= 16) ? 16 : (A + 2 <= 32 ? 32 : (A + 2 <= 64 ? 64 : 128));
      }
      const int M2 = A + 2;
      const int SR = (Bs <= 64) ? 2048 / Bs : 16;
      const RowConst RK = I.rk;
      for (int j = st; j < A; j += kTcSetupThreads) s_lm[b * kTcLmCap + j] = s_uidx[jlo + j];
      if (I.kind == NYS_COEF_LIN) {
        // r(t_i) = c sin(theta_i): one sine per thread, then rotations by 64 rows
        if (st < n_sub) {
          float sn, cs;
          lin_sincos(RK, row + st, sn, cs);
          for (int t = st; t < n_sub; t += kTcSetupThreads) {
            s_r[b * kTcSubRows + t] = RK.c * sn;
            const float s2 = fmaf(sn, cb, cs * sb);
            cs = fmaf(cs, cb, -sn * sb);
            sn = s2;
          }
        }
      } else {
        for (int t = st; t < n_sub; t += kTcSetupThreads) {
          ff c5[5];
          row_coef_ff(I, RK, ctab, row + t, c5);
          s_r[b * kTcSubRows + t] = c5[4].hi;
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
        M.Au = Au;
        M.jlo_u = jlo_u;
        M.first = (row == ur0) ? 1 : 0;
        M.last = (row + n_sub >= r1) ? 1 : 0;
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
      // one thread waits (bounded) and publishes the outcome, so that the four
      // warps take the same path through their named barriers
      if (et == 0) s_eok = mbar_wait_bounded(smem_u32(&s_ready[b]), (uint32_t)((s / kTcSub) & 1), wait_iter) ? 1 : 0;
      bar_named(2, 128);
      const bool okm = s_eok != 0;
      const TcSub M = s_meta[b];
      bar_named(2, 128);                               // all four warps have read the meta
      if (et == 0) mbar_arrive(smem_u32(&s_used[b]));
      if (!okm) { if (et == 0) atomicExch(&s_abort, 1); break; }
      if (M.nst < 0) break;
      const int M2u = M.Au + 2, Eu = M2u * (M2u + 1) / 2;
      if (M.first) {
        for (int e = et; e < Eu; e += 128) Gu[e] = 0.0;
        bar_named(2, 128);
      }
      if (et == 0) s_eok = mbar_wait_bounded(smem_u32(&s_accf[b]), (uint32_t)((s / kTcSub) & 1), wait_iter) ? 1 : 0;
      bar_named(2, 128);
      if (s_eok == 0) { if (et == 0) atomicExch(&s_abort, 1); break; }
      tc_fence_after();
      const uint32_t lanebase = tmem + (uint32_t)b * kTcSetCols + ((uint32_t)(32 * quad) << 16);
      const int Bs = M.Bs, A = M.A, M2 = M.M2;
      // sub-chunk column c -> unit column (landmarks shift by joff; -f_p, r last)
      const int joff = M.joff, Au = M.Au;
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
        tc_fence_before();
        bar_named(2, 128);                             // accumulator read, S complete
        if (et == 0) mbar_arrive(smem_u32(&s_afree[b]));
        const int nq = 128 / Bs;                       // operand rows per slot (row sets x hi/lo)
        const float invM2 = 1.0f / (float)M2;
        for (int e = et; e < M2 * M2; e += 128) {
          const int j = (int)(((float)e + 0.5f) * invM2);
          const int l = e - j * M2;
          if (l >= j) {
            float sum = 0.f;
            for (int q = 0; q < nq; ++q) sum += S[(q * Bs + j) * kTcSLd + l];
            const int ju = (j < A) ? j + joff : Au + (j - A);
            const int lu = (l < A) ? l + joff : Au + (l - A);
            Gu[ju * M2u - ju * (ju - 1) / 2 + (lu - ju)] += (double)sum;
          }
        }
      } else {
        // lane rho = slot j holds row j of the sub-chunk Gram itself
        const int j = rho;
        for (int l0 = 0; l0 < M.N; l0 += 16) {
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
                Gu[ju * M2u - ju * (ju - 1) / 2 + (lu - ju)] += (double)__uint_as_float(v[t]);
              }
            }
          }
        }
        tc_fence_before();
        bar_named(2, 128);
        if (et == 0) mbar_arrive(smem_u32(&s_afree[b]));
      }
      bar_named(2, 128);                               // Gu updated, S free
      if (M.last) {
        // slot: [first landmark, landmark count, packed upper Gram of the unit]
        double* out = part + M.slot_off;
        if (et == 0) { out[0] = (double)M.jlo_u; out[1] = (double)Au; }
        for (int e = et; e < Eu; e += 128) out[2 + e] = Gu[e];
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
