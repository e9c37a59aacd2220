// Fused assembly of Lemma 1's Gram (Section 3.1) on the tensor cores, mixed path.
//
// A work item (instance, chunk of <= 1024 consecutive collocation rows) needs
// G = sum_i psi_i psi_i^T of the augmented rows psi_i = [kappa_i (window of A
// landmarks); -f_p(t_i); r(t_i)], M2 = A + 2 columns: a dense contraction over
// the rows, run as tcgen05 MMAs (kind::tf32) with accumulators in tensor memory.
//
// Operands.  Features are split into TF32 parts hi = tf32(psi), lo = psi - hi
// and G accumulates hi hi^T + hi lo^T + lo hi^T (the dropped lo lo^T term is
// 2^-22 relative), so the products carry ~22 bits and D stays symmetric.  The
// operand tile is 128 rows x 32 K positions, K-major with the 128-byte swizzle.
// Block-diagonal packing: the 128 operand rows hold P = 128 / Bs blocks of
// Bs >= M2 slots; block p carries rows 32 p .. 32 p + 31 of the stage on the
// same 32 K positions, so one 128 x 128 x 8 MMA adds the Gram of P x 8 rows
// to its diagonal blocks (the off-diagonal blocks mix rows and are not read).
//
// Warp roles (persistent CTA per SM, all hand-offs through mbarriers):
//   * two setup warps prepare the next work item while the current one is
//     produced: fetch it, load its landmarks, evaluate r(t_i) of its rows,
//     find its landmark window; item data double-buffered;
//   * 20 producer warps evaluate features (FP32, MUFU exponential) straight
//     into the operand layout (one warp store fills one 8-slot x 4-row core
//     matrix, conflict-free; a warp takes half of the K chunks of one 8-slot
//     group per unit) and arrive on the stage's "full" barrier; four stage
//     buffers;
//   * one issuer warp waits for "full", issues the MMAs (two accumulators per
//     item, alternating) and commits to the stage's "empty" barrier and, after
//     the item's last stage, to the accumulator barrier;
//   * four epilogue warps read the accumulators from tensor memory, add the
//     diagonal blocks and store the packed upper triangle as doubles in the
//     slot format of the CUDA-core kernel ([jlo, A, upper Gram]).
// Items alternate between two tensor-memory accumulator sets and two metadata
// slots, so the epilogue and the MMA tail of one item overlap the production
// of the next.  Every wait is bounded; on timeout the kernel records an error
// word (reported as NYS_ETIMEOUT by the solve), lets its MMAs drain (bounded),
// frees its tensor memory and returns.
#include "nys_internal.cuh"
#include "nys_tc.cuh"

namespace nys {

constexpr int kTcProducers = 20;                       // producer warps 0..19
constexpr int kTcIssuerWarp = kTcProducers;            // warp 20
constexpr int kTcEpiWarp0 = kTcProducers + 1;          // warps 21..24
constexpr int kTcSetupWarp0 = kTcProducers + 5;        // warps 25, 26
constexpr int kTcSetupThreads = 64;
constexpr int kTcThreads = 32 * (kTcProducers + 5) + kTcSetupThreads;
constexpr int kTcStages = 4;
constexpr int kTcTileBytes = 16384;      // 128 operand rows x 32 K positions (TF32)
constexpr int kTcStageBytes = 2 * kTcTileBytes;   // hi + lo
constexpr int kTcStageArea = kTcStages * kTcStageBytes;
constexpr int kTcSBytes = 128 * 129 * 4; // epilogue staging: P blocks of Bs x (Bs + 1)
constexpr int kTcMaxRows = 1024;         // rows of a work item (the host keeps items this size)
constexpr int kTcWaitIter = 1 << 22;     // try_wait polls (<= 1 us each) before giving up
constexpr int kTcAcc = 2;                // accumulators per item (alternating MMAs)
constexpr uint32_t kTcAccCols = 128;     // columns per accumulator (N <= 128)
constexpr uint32_t kTcSetCols = kTcAcc * kTcAccCols;
constexpr uint32_t kTcCols = 2 * kTcSetCols;   // two sets: the whole tensor memory of the SM

size_t asm_tc_smem_bytes() { return (size_t)kTcStageArea + kTcSBytes + 1024; }

struct TcItem {          // metadata of a work item for the issuer and the epilogue
  int w, slot, jlo, A, M2, P, Bs, N, nst;
};

struct TcProd {          // what the producers need of a work item (nst < 0: no more items)
  int r0, nrows, m, jlo, A, P, Bs, SR, Gf, nst, lin;
  float hsc, LA0, LB1, LB2, w1;
};

__device__ __forceinline__ void bar_named(int id, int count) {
  asm volatile("bar.sync %0, %1;" :: "r"(id), "r"(count) : "memory");
}

__global__ void __launch_bounds__(kTcThreads, 1)
k_assemble_tc(const Inst* __restrict__ insts, const Lset* __restrict__ lsets,
              const Work* __restrict__ work, int nwork, int* __restrict__ counter,
              const int32_t* __restrict__ lm_idx, const double* __restrict__ tab,
              double* __restrict__ part, const int64_t* __restrict__ slot_off,
              int32_t* __restrict__ err) {
  extern __shared__ unsigned char tc_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(tc_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  float* S = reinterpret_cast<float*>(sm + kTcStageArea);
  __shared__ __align__(8) uint64_t s_full[kTcStages], s_empty[kTcStages];
  __shared__ __align__(8) uint64_t s_mfull[2], s_mfree[2], s_accf[2], s_afree[2], s_drain;
  __shared__ __align__(8) uint64_t s_sfull[2], s_sempty[2];
  __shared__ TcItem s_meta[2];
  __shared__ TcProd s_pm[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_w, s_abort, s_eok, s_sok;
  __shared__ int s_idx[2][kMMax];
  __shared__ float s_r[2][kTcMaxRows];   // r(t_i) of the rows of the item
  __shared__ float4 s_co[kTcMaxRows];    // kind TABLE: (A0, A1, A2, w1) of every row
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) tmem_alloc(smem_u32(&s_tmem), kTcCols);
  if (tid == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(smem_u32(&s_full[s]), kTcProducers);
      mbar_init(smem_u32(&s_empty[s]), 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(smem_u32(&s_mfull[s]), 1);
      mbar_init(smem_u32(&s_mfree[s]), 2);
      mbar_init(smem_u32(&s_accf[s]), 1);
      mbar_init(smem_u32(&s_afree[s]), 1);
    }
    mbar_init(smem_u32(&s_drain), 1);
    for (int s = 0; s < 2; ++s) {
      mbar_init(smem_u32(&s_sfull[s]), kTcSetupThreads);
      mbar_init(smem_u32(&s_sempty[s]), kTcProducers);
    }
    mbar_fence_init();
    s_abort = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  if (warp < kTcProducers) {
    // =========================== producers ===========================
    // mbarrier phase parities and buffer states as bit masks (bit = buffer),
    // kept in registers
    uint32_t ph_empty = 0, ph_sfull = 0, used = 0;
    int gs = 0;                                        // stages produced so far
    for (int it = 0;; ++it) {
      const int rs = it & 1;
      // the setup warps have prepared this item in buffer rs
      if (!mbar_wait_bounded(smem_u32(&s_sfull[rs]), (ph_sfull >> rs) & 1u, kTcWaitIter)) {
        atomicExch(&s_abort, 1);
        break;
      }
      ph_sfull ^= 1u << rs;
      const TcProd Pm = s_pm[rs];
      if (Pm.nst < 0) break;
      const int* idx = s_idx[rs];
      const float* rr = s_r[rs];
      const int m = Pm.m, nrows = Pm.nrows, jlo = Pm.jlo, A = Pm.A, P = Pm.P, Bs = Pm.Bs;
      const int SR = Pm.SR, Gf = Pm.Gf, nst = Pm.nst;
      const bool lin = Pm.lin != 0;
      // This warp's units (block p, 8-slot group g, K half qh) are the same in
      // every stage of the item: at most two, since 2 P Gf <= 32 < 2 x 20.
      // lane -> (slot j8, K position w4)
      static_assert(2 * kTcProducers >= 32, "two units per producer warp cover a stage");
      const float invGf = 1.0f / (float)Gf;
      const float hsc = Pm.hsc;                        // h / sigma * sqrt(log2 e)
      const int tmax = min(nrows, kTcMaxRows) - 1;
      const int j8 = lane >> 2, w4 = lane & 3;
      // Balance: the units of the last 8-slot group of each block (2 P of them;
      // the group with the -f_p / r columns, whose lanes take several paths) are
      // the slowest.  Units are listed with those first, and the warps that get a
      // single unit (when there are more units than warps) take the head of the
      // list, the others two each from the rest.
      const int nunits = 2 * P * Gf;
      const int ndbl = max(0, nunits - kTcProducers);       // warps with two units
      const int nsgl = kTcProducers - ndbl;
      int u_kind[2], u_t0[2], u_lag[2], u_off[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        int li = -1;                                     // index in the unit list
        if (warp < nsgl) li = (u == 0 && warp < nunits) ? warp : -1;
        else li = nsgl + 2 * (warp - nsgl) + u;
        u_kind[u] = -1;
        u_t0[u] = u_lag[u] = u_off[u] = 0;
        if (li >= 0 && li < nunits) {
          int pb, g, qh;
          if (li < 2 * P) {                              // last group of block li / 2
            pb = li >> 1; qh = li & 1; g = Gf - 1;
          } else {                                       // groups 0 .. Gf - 2
            const int l2 = li - 2 * P, pg = l2 >> 1;
            qh = l2 & 1;
            pb = (int)(((float)pg + 0.5f) / (float)(Gf - 1));
            g = pg - pb * (Gf - 1);
          }
          const int j = (g << 3) + j8;               // local column of this lane
          const int idxj = idx[min(jlo + j, m - 1)];
          u_kind[u] = (j < A) ? 0 : (j == A ? 1 : (j == A + 1 ? 2 : 3));
          u_t0[u] = 32 * pb + w4 + 16 * qh;            // item row of the first chunk (stage 0)
          u_lag[u] = Pm.r0 + u_t0[u] - idxj;           // its lag t_i - s_j in grid steps
          // operand row of (pb, g, j8), K word w4, and the K-half's swizzle bit
          u_off[u] = ((((pb * Bs) >> 3) + g) << 10) + (j8 << 7) + (w4 << 2) +
                     (((qh ^ (j8 >> 2)) & 1) << 6);
        }
      }
      int xq[4];   // 128-byte swizzle of K chunk q + 4 qh: ((q + 4 qh) ^ j8) & 7
#pragma unroll
      for (int q = 0; q < 4; ++q) xq[q] = (q ^ (j8 & 3)) << 4;
      // A0 + A1 x + A2 x^2 = A0 + (A1 / c) y + (A2 / c^2) y^2, y = c x, c = sqrt(log2 e)
      const float ic1 = 0.832554611157698f, ic2 = 0.693147180559945f;
      const float LA0 = Pm.LA0, LB1 = Pm.LB1, LB2 = Pm.LB2, w1 = Pm.w1;
      bool late = false;
      for (int k = 0; k < nst; ++k, ++gs) {
        const int s = gs & (kTcStages - 1);
        if ((used >> s) & 1u) {  // the MMAs that read this buffer must be done
          late = late || !mbar_wait_bounded(smem_u32(&s_empty[s]), (ph_empty >> s) & 1u, kTcWaitIter);
          ph_empty ^= 1u << s;
        }
        used |= 1u << s;
        unsigned char* hi = sm + s * kTcStageBytes;
        if (!late) {
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int kind = u_kind[u];
            if (kind < 0) continue;                    // warp-uniform
            const int t0 = k * SR + u_t0[u];           // item row of this lane's first chunk
            // the 4 K chunks of this lane are independent: evaluate all, then store
            float vv[4];
            if (kind == 0) {
              // y = x sqrt(log2 e), x = (t_i - s_j) / sigma at the rows t0 + 4q (one
              // FMA per chunk); exp(-x^2) = 2^(-y^2)
              const float y0 = (float)(u_lag[u] + k * SR) * hsc;
              const float dy = 4.f * hsc;
              float A0 = LA0, B1 = LB1, B2 = LB2;
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                if (!lin) {
                  const float4 co = s_co[min(t0 + 4 * q, tmax)];
                  A0 = co.x; B1 = co.y * ic1; B2 = -co.z * ic2;
                }
                const float y = fmaf((float)q, dy, y0);
                const float nu = -y * y;                 // -y^2
                vv[q] = ex2_approx(nu) * fmaf(B2, nu, fmaf(B1, y, A0));
              }
            } else {
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const int tc = min(t0 + 4 * q, tmax);
                vv[q] = (kind == 1) ? (lin ? w1 : s_co[tc].w) : (kind == 2 ? rr[tc] : 0.f);
              }
            }
            if (t0 + 12 >= nrows) {                    // rows past the end of the item
#pragma unroll
              for (int q = 0; q < 4; ++q)
                if (t0 + 4 * q >= nrows) vv[q] = 0.f;
            }
            unsigned char* hrow = hi + u_off[u];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              // TF32 part by truncation (the low part v - hi is exact either way)
              const float h = __uint_as_float(__float_as_uint(vv[q]) & 0xFFFFE000u);
              float* dst = reinterpret_cast<float*>(hrow + xq[q]);
              dst[0] = h;
              dst[kTcTileBytes / 4] = vv[q] - h;
            }
          }
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&s_full[s]));
      }
      if (late && lane == 0) atomicExch(&s_abort, 1);
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&s_sempty[rs]));   // buffer rs may be refilled
    }
  } else if (warp >= kTcSetupWarp0) {
    // ============================== setup ==============================
    // Prepares item it + 1 while the producers fill the stages of item it:
    // fetches the work item, loads its landmarks, evaluates r(t_i) (and the
    // row coefficients of kind TABLE), finds the landmark window and publishes
    // the metadata to the producers (buffer it % 2) and to the issuer and the
    // epilogue (slot it % 2).
    const int st = tid - 32 * kTcSetupWarp0;           // 0..63
    uint32_t ph_sempty = 0, ph_mfree = 0, waited = 0;   // bit masks (bit = buffer)
    for (int it = 0;; ++it) {
      const int rs = it & 1;
      // buffer rs held item it - 2: the producers must be done with it
      if (it >= 2 && !((waited >> rs) & 1u)) {
        if (st == 0) s_sok = mbar_wait_bounded(smem_u32(&s_sempty[rs]), (ph_sempty >> rs) & 1u, kTcWaitIter) ? 1 : 0;
        ph_sempty ^= 1u << rs;
        bar_named(3, kTcSetupThreads);
        if (!s_sok) atomicExch(&s_abort, 1);
      }
      waited &= ~(1u << rs);
      if (st == 0) s_w = s_abort ? nwork : atomicAdd(counter, 1);
      bar_named(3, kTcSetupThreads);
      const int w = s_w;
      bar_named(3, kTcSetupThreads);                   // every thread has read s_w
      if (w >= nwork) {   // sentinels for the producers, the issuer and the epilogue
        if (st == 0) {
          s_pm[rs].nst = -1;
          bool ok = true;
          if (it >= 2) ok = mbar_wait_bounded(smem_u32(&s_mfree[rs]), (ph_mfree >> rs) & 1u, kTcWaitIter);
          if (!ok) atomicExch(&s_abort, 1);
          s_meta[rs].nst = -1;
          mbar_arrive(smem_u32(&s_mfull[rs]));
        }
        mbar_arrive(smem_u32(&s_sfull[rs]));
        break;
      }
      const Work wk = work[w];
      const Inst& I = insts[wk.inst];
      const int m = I.m;
      const int nrows = wk.r1 - wk.r0;
      const bool lin = (I.kind == NYS_COEF_LIN);
      const RowConst RK = I.rk;
      for (int j = st; j < m; j += kTcSetupThreads) s_idx[rs][j] = lm_idx[I.lm_off + j];
      if (!lin && it >= 1) {
        // s_co has one buffer: the producers must be done with item it - 1
        if (st == 0) s_sok = mbar_wait_bounded(smem_u32(&s_sempty[rs ^ 1]), ((ph_sempty >> (rs ^ 1)) & 1u), kTcWaitIter) ? 1 : 0;
        ph_sempty ^= 1u << (rs ^ 1);
        waited |= 1u << (rs ^ 1);
        bar_named(3, kTcSetupThreads);
        if (!s_sok) atomicExch(&s_abort, 1);
      }
      for (int t = st; t < nrows && t < kTcMaxRows; t += kTcSetupThreads) {
        const int i = wk.r0 + t;
        if (lin) {
          s_r[rs][t] = lin_rhs_ff(RK, i);
        } else {
          ff c5[5];
          row_coef_ff(I, RK, tab, i, c5);
          s_r[rs][t] = c5[4].hi;
          s_co[t] = make_float4(c5[0].hi, c5[1].hi, c5[2].hi, c5[3].hi);
        }
      }
      bar_named(3, kTcSetupThreads);                   // s_idx of this item complete
      if (st == 0) {
        // landmark window of the chunk: |i - idx_j| <= K for some row i in [r0, r1)
        const int* idx = s_idx[rs];
        const int Kl = lsets[I.lset].K;
        int a = 0, b = m;
        while (a < b) { const int c = (a + b) >> 1; if (idx[c] < wk.r0 - Kl) a = c + 1; else b = c; }
        const int jlo = a;
        b = m;
        while (a < b) { const int c = (a + b) >> 1; if (idx[c] <= wk.r1 - 1 + Kl) a = c + 1; else b = c; }
        const int A = a - jlo;
        const int M2 = A + 2;
        const int P = (M2 <= 32) ? 4 : (M2 <= 64 ? 2 : 1);
        const int Bs = 128 / P;
        const int SR = 32 * P;                          // rows per stage
        const int nst = (nrows <= kTcMaxRows) ? (nrows + SR - 1) / SR : 0;
        bool ok = true;
        if (it >= 2) ok = mbar_wait_bounded(smem_u32(&s_mfree[rs]), (ph_mfree >> rs) & 1u, kTcWaitIter);
        if (it >= 2) ph_mfree ^= 1u << rs;
        if (!ok || nrows > kTcMaxRows) atomicExch(&s_abort, 1);
        TcItem& M = s_meta[rs];
        M.w = w; M.slot = wk.slot; M.jlo = jlo; M.A = A; M.M2 = M2; M.P = P; M.Bs = Bs;
        M.N = (P > 1) ? 128 : round_up(M2, 16);
        M.nst = ok ? nst : 0;
        mbar_arrive(smem_u32(&s_mfull[rs]));
        TcProd& Q = s_pm[rs];
        Q.r0 = wk.r0; Q.nrows = nrows; Q.m = m; Q.jlo = jlo; Q.A = A; Q.P = P; Q.Bs = Bs;
        Q.SR = SR; Q.Gf = (M2 + 7) >> 3;               // 8-slot groups written per block
        Q.nst = ok ? nst : 0;
        Q.lin = lin ? 1 : 0;
        Q.hsc = (float)I.hs * 1.20112240878645f;
        Q.LA0 = RK.A0.hi;
        Q.LB1 = RK.A1.hi * 0.832554611157698f;
        Q.LB2 = -RK.A2.hi * 0.693147180559945f;
        Q.w1 = RK.w1.hi;
      }
      mbar_arrive(smem_u32(&s_sfull[rs]));             // each thread: its writes are done
    }
  } else if (warp == kTcIssuerWarp) {
    // ============================= issuer =============================
    if (lane == 0) {
      uint32_t ph_full = 0, ph_mfull = 0, ph_afree = 0;   // bit masks (bit = buffer)
      int gs = 0;
      uint32_t ncommit_acc = 0;   // commits to the accumulator barriers
      for (int it = 0;; ++it) {
        const int rs = it & 1;
        if (!mbar_wait_bounded(smem_u32(&s_mfull[rs]), (ph_mfull >> rs) & 1u, kTcWaitIter)) {
          atomicExch(&s_abort, 1);
          break;
        }
        ph_mfull ^= 1u << rs;
        const TcItem M = s_meta[rs];
        mbar_arrive(smem_u32(&s_mfree[rs]));
        if (M.nst < 0) break;
        if (M.nst == 0) { atomicExch(&s_abort, 1); break; }   // producers gave up
        if (it >= 2) {   // the epilogue of item it - 2 has read this accumulator set
          const bool ok = mbar_wait_bounded(smem_u32(&s_afree[rs]), (ph_afree >> rs) & 1u, kTcWaitIter);
          ph_afree ^= 1u << rs;
          if (!ok) { atomicExch(&s_abort, 1); break; }
        }
        tc_fence_after();
        const uint32_t idesc = tc_idesc_tf32(128, M.N);
        const uint32_t dset = tmem + (uint32_t)rs * kTcSetCols;
        bool late = false;
        uint32_t started = 0;
        int rot = 0;
        for (int k = 0; k < M.nst; ++k, ++gs) {
          const int s = gs & (kTcStages - 1);
          if (!mbar_wait_bounded(smem_u32(&s_full[s]), (ph_full >> s) & 1u, kTcWaitIter)) { late = true; break; }
          ph_full ^= 1u << s;
          tc_fence_after();
          const uint32_t ha = smem_u32(sm + s * kTcStageBytes);
          const uint32_t la = ha + (uint32_t)kTcTileBytes;
          for (int t = 0; t < 4; ++t) {                // 4 K steps of 8 positions
            const uint64_t dh = tc_desc_sw128(ha + 32u * t);
            const uint64_t dl = tc_desc_sw128(la + 32u * t);
            const uint64_t da[3] = {dh, dh, dl}, db[3] = {dh, dl, dh};
#pragma unroll
            for (int q3 = 0; q3 < 3; ++q3) {
              tc_mma_tf32(dset + (uint32_t)rot * kTcAccCols, da[q3], db[q3], idesc,
                          (started >> rot) & 1u);
              started |= 1u << rot;
              rot ^= 1;
            }
          }
          tc_commit(smem_u32(&s_empty[s]));
        }
        if (late) { atomicExch(&s_abort, 1); break; }
        tc_commit(smem_u32(&s_accf[rs]));
        ++ncommit_acc;
      }
      // every MMA issued by this thread has completed once this commit arrives
      tc_commit(smem_u32(&s_drain));
      mbar_wait_bounded(smem_u32(&s_drain), 0, kTcWaitIter);
      (void)ncommit_acc;
    }
  } else {
    // ============================ epilogue (warps 21..24) ============================
    const int et = tid - 32 * kTcEpiWarp0;             // 0..127
    const int quad = warp & 3;                         // tensor-memory lane quarter
    uint32_t ph_mfull = 0, ph_accf = 0;   // bit masks (bit = buffer)
    for (int it = 0;; ++it) {
      const int rs = it & 1;
      // one thread waits (bounded) and publishes the outcome, so that the four
      // warps take the same path through their named barriers
      if (et == 0) s_eok = mbar_wait_bounded(smem_u32(&s_mfull[rs]), (ph_mfull >> rs) & 1u, kTcWaitIter) ? 1 : 0;
      ph_mfull ^= 1u << rs;
      bar_named(2, 128);
      const bool okm = s_eok != 0;
      const TcItem M = s_meta[rs];
      bar_named(2, 128);                               // all four warps have read the slot
      if (et == 0) mbar_arrive(smem_u32(&s_mfree[rs]));
      if (!okm) { if (et == 0) atomicExch(&s_abort, 1); break; }
      if (M.nst < 0) break;
      if (M.nst == 0) {   // an aborted item: no accumulator commit follows
        if (et == 0) { atomicExch(&s_abort, 1); mbar_arrive(smem_u32(&s_afree[rs])); }
        continue;
      }
      if (et == 0) s_eok = mbar_wait_bounded(smem_u32(&s_accf[rs]), (ph_accf >> rs) & 1u, kTcWaitIter) ? 1 : 0;
      ph_accf ^= 1u << rs;
      bar_named(2, 128);
      const bool oka = s_eok != 0;
      tc_fence_after();
      const int P = M.P, Bs = M.Bs, M2 = M.M2;
      const int ldS = Bs + 1;                          // padded: conflict-free row stores
      const int p = (32 * quad) / Bs;                  // block of this lane quarter
      const int j = 32 * quad + lane - p * Bs;         // row within the block
      const uint32_t lanebase = tmem + (uint32_t)rs * kTcSetCols + ((uint32_t)(32 * quad) << 16);
      const int ncol = min(Bs, round_up(M2, 16));
      if (oka) {
        for (int c0 = 0; c0 < ncol; c0 += 16) {
          const uint32_t col = (uint32_t)(p * Bs + c0);
          uint32_t r[kTcAcc][16];
#pragma unroll
          for (int a = 0; a < kTcAcc; ++a) tmem_ld16_nowait(lanebase + (uint32_t)a * kTcAccCols + col, r[a]);
          tmem_wait_ld();
          if (j < M2) {
#pragma unroll
            for (int t = 0; t < 16; ++t) {
              float v = 0.f;
#pragma unroll
              for (int a = 0; a < kTcAcc; ++a) v += __uint_as_float(r[a][t]);
              if (c0 + t < M2) S[(p * Bs + j) * ldS + c0 + t] = v;
            }
          }
        }
      }
      tc_fence_before();
      bar_named(2, 128);                               // accumulators read, S complete
      if (et == 0) mbar_arrive(smem_u32(&s_afree[rs]));
      if (!oka) { if (et == 0) atomicExch(&s_abort, 1); break; }
      // slot: [first landmark, landmark count, packed upper local Gram]
      double* out = part + slot_off[M.slot];
      if (et == 0) { out[0] = (double)M.jlo; out[1] = (double)M.A; }
      const float invM2 = 1.0f / (float)M2;
      for (int e = et; e < M2 * M2; e += 128) {
        const int rr = (int)(((float)e + 0.5f) * invM2);
        const int l = e - rr * M2;
        if (l >= rr) {
          float sum = 0.f;
          for (int pp = 0; pp < P; ++pp) sum += S[(pp * Bs + rr) * ldS + l];
          out[2 + rr * M2 - rr * (rr - 1) / 2 - rr + l] = (double)sum;
        }
      }
      bar_named(2, 128);                               // S is free for the next item
    }
  }

  if (tid == 0 && s_abort) atomicExch(err, 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, kTcCols);
}

cudaError_t launch_assemble_tc(const Inst* insts, const Lset* lsets, const Work* work, int nwork,
                               int* counter, const int32_t* lm, const double* tab, double* part,
                               const int64_t* slot_off, int32_t* err, int num_sms,
                               cudaStream_t st) {
  const size_t sm = asm_tc_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(k_assemble_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm);
  if (e != cudaSuccess) return e;
  const int grid = nwork < num_sms ? nwork : num_sms;
  if (grid < 1) return cudaSuccess;
  k_assemble_tc<<<grid, kTcThreads, sm, st>>>(insts, lsets, work, nwork, counter, lm, tab, part,
                                              slot_off, err);
  return cudaGetLastError();
}

}  // namespace nys
