// Fused assembly of Lemma 1's Gram (Section 3.1) on the tensor cores, mixed path.
//
// A work item (instance, chunk of consecutive collocation rows) needs the Gram
// G = sum_i psi_i psi_i^T of the augmented rows psi_i = [kappa_i (window of A
// landmarks); -f_p(t_i); r(t_i)], M2 = A + 2 columns.  This is a dense
// contraction over the rows, so it runs as tcgen05 MMAs with the accumulator
// in tensor memory.  Warp roles:
//   * 16 producer warps evaluate the features (FP32, MUFU exponential) of a
//     stage of KT rows and store them straight into the operand layout of the
//     MMA (K-major, 128-byte swizzle: one warp store fills one 8-feature x
//     4-row core matrix, conflict-free), split into TF32 parts hi = tf32(psi)
//     and lo = psi - hi; each warp then arrives on the stage's "full" mbarrier;
//   * one issuer warp waits for "full", issues per 8-row K step
//     D += hi hi^T + hi lo^T + lo hi^T (three kind::tf32 MMAs; the dropped
//     lo lo^T term is 2^-22 relative, so the products carry ~22 bits and D
//     stays symmetric) and commits to the stage's "empty" mbarrier, which the
//     producers wait on before they overwrite the buffer (two stages).  The
//     MMAs of a tile this small are latency-bound when chained on one
//     accumulator, so they rotate over four accumulators, summed at the end;
//   * after the last stage the issuer commits to an accumulator barrier;
//     producer warps 0-3 then read D from tensor memory and store the packed
//     upper triangle of the local Gram as doubles, in the slot format of the
//     CUDA-core kernel ([jlo, A, upper Gram]).
// M = 64 when M2 <= 64 (row r of D in lane 32 (r / 16) + r % 16), else 128
// (row r in lane r).  The remaining error of the FP32 features and the TF32
// split is removed by the FP64-accurate refinement of the mixed path.
// Every mbarrier wait is bounded; on timeout the kernel records an error word
// (read by the solve, which reports NYS_ETIMEOUT), drains its MMAs (bounded),
// frees its tensor memory and returns.
#include "nys_internal.cuh"
#include "nys_tc.cuh"

namespace nys {

constexpr int kTcProducers = 20;                       // producer warps
constexpr int kTcThreads = 32 * (kTcProducers + 1);    // + one MMA-issuer warp
constexpr int kTcStages = 4;
constexpr int kTcTileBytes = 16384;      // 128 operand rows x 32 K positions (TF32)
constexpr int kTcStageBytes = 2 * kTcTileBytes;   // hi + lo
constexpr int kTcMaxRows = 1024;         // rows of a work item with a tabulated r(t_i)
constexpr int kTcWaitIter = 1 << 22;     // try_wait polls before giving up (seconds)
constexpr int kTcAcc = 4;                // independent accumulators (MMA chains)
constexpr uint32_t kTcAccCols = 128;     // columns per accumulator (N <= 128)
constexpr uint32_t kTcCols = kTcAcc * kTcAccCols;   // the whole tensor memory of the SM

size_t asm_tc_smem_bytes() { return (size_t)kTcStages * kTcStageBytes + 1024; }

__global__ void __launch_bounds__(kTcThreads, 1)
k_assemble_tc(const Inst* __restrict__ insts, const Lset* __restrict__ lsets,
              const Work* __restrict__ work, int nwork, int* __restrict__ counter,
              const int32_t* __restrict__ lm_idx, const double* __restrict__ tab,
              double* __restrict__ part, const int64_t* __restrict__ slot_off,
              int32_t* __restrict__ err) {
  extern __shared__ unsigned char tc_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(tc_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  __shared__ __align__(8) uint64_t s_full[kTcStages], s_empty[kTcStages], s_accf;
  __shared__ uint32_t s_tmem;
  __shared__ int s_item, s_abort;
  __shared__ int s_idx[kMMax];
  __shared__ float s_r[kTcMaxRows];   // r(t_i) of the rows of the work item
  __shared__ float4 s_co[kTcMaxRows]; // kind TABLE: (A0, A1, A2, w1) of every row
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool issuer = (warp == kTcProducers);

  if (warp == 0) tmem_alloc(smem_u32(&s_tmem), kTcCols);
  if (tid == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(smem_u32(&s_full[s]), kTcProducers);
      mbar_init(smem_u32(&s_empty[s]), 1);
    }
    mbar_init(smem_u32(&s_accf), 1);
    mbar_fence_init();
    s_abort = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  // phase bits (uniform within each role)
  uint32_t ph_full[kTcStages], ph_empty[kTcStages], ph_acc = 0;
  uint32_t nacc = 0;   // issuer: commits to the accumulator barrier so far
  bool used[kTcStages];
#pragma unroll
  for (int s = 0; s < kTcStages; ++s) { ph_full[s] = 0; ph_empty[s] = 0; used[s] = false; }

  for (;;) {
    if (tid == 0) s_item = atomicAdd(counter, 1);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const int w = s_item;
    if (w >= nwork || s_abort) break;
    const Work wk = work[w];
    const Inst I = insts[wk.inst];
    const int m = I.m;
    const int nrows = wk.r1 - wk.r0;
    const bool lin = (I.kind == NYS_COEF_LIN);
    const RowConst RK = I.rk;
    for (int j = tid; j < m; j += kTcThreads) s_idx[j] = lm_idx[I.lm_off + j];
    // per-row right-hand side (and, kind TABLE, operator coefficients), once per row
    // (the work list keeps the rows of a tensor-core work item <= kTcMaxRows)
    for (int t = tid; t < nrows && t < kTcMaxRows; t += kTcThreads) {
      const int i = wk.r0 + t;
      if (lin) {
        s_r[t] = lin_rhs_ff(RK, i);
      } else {
        ff c5[5];
        row_coef_ff(I, RK, tab, i, c5);
        s_r[t] = c5[4].hi;
        s_co[t] = make_float4(c5[0].hi, c5[1].hi, c5[2].hi, c5[3].hi);
      }
    }
    __syncthreads();
    // landmark window of the chunk: |i - idx_j| <= K for some row i in [r0, r1)
    const int Kl = lsets[I.lset].K;
    int jlo, A;
    {
      int a = 0, b = m;
      while (a < b) { const int c = (a + b) >> 1; if (s_idx[c] < wk.r0 - Kl) a = c + 1; else b = c; }
      jlo = a;
      b = m;
      while (a < b) { const int c = (a + b) >> 1; if (s_idx[c] <= wk.r1 - 1 + Kl) a = c + 1; else b = c; }
      A = a - jlo;
    }
    const int M2 = A + 2;
    // Block-diagonal packing: the 128 operand rows hold P = 128 / Bs blocks of
    // Bs >= M2 feature slots; block p carries rows 32 p .. 32 p + 31 of the
    // stage on the same 32 K positions, so one 128 x 128 x 8 MMA accumulates
    // the Gram of 4 x 8 rows (P = 4) in its diagonal blocks D[p][p]; the
    // off-diagonal blocks mix different rows and are never read.
    const int P = (M2 <= 32) ? 4 : (M2 <= 64 ? 2 : 1);
    const int Bs = 128 / P;
    const int N = (P > 1) ? 128 : round_up(M2, 16);
    const int SR = 32 * P;                            // rows per stage
    const int Gf = (M2 + 7) >> 3;                     // 8-slot groups written per block
    const float invGf = 1.0f / (float)Gf;
    const int nst = (nrows <= kTcMaxRows) ? (nrows + SR - 1) / SR : 0;
    if (nrows > kTcMaxRows && tid == 0) atomicExch(&s_abort, 1);
    const float hs = (float)I.hs;
    const int tmax = min(nrows, kTcMaxRows) - 1;

    if (!issuer) {
      // ---------------- producers ----------------
      bool late = false;
      for (int k = 0; k < nst && !late; ++k) {
        const int s = k & (kTcStages - 1);
        if (used[s]) {  // the MMAs that read this buffer must be done
          late = !mbar_wait_bounded(smem_u32(&s_empty[s]), ph_empty[s], kTcWaitIter);
          ph_empty[s] ^= 1u;
        }
        used[s] = true;
        if (late) break;
        unsigned char* hi = sm + s * kTcStageBytes;
        const int j8 = lane >> 2, w4 = lane & 3;
        // warp -> (block p, 8-slot group g) pairs; lane -> (slot j8, K position w4)
        for (int pg = warp; pg < P * Gf; pg += kTcProducers) {
          const int p = (int)(((float)pg + 0.5f) * invGf);
          const int g = pg - p * Gf;
          const int j = (g << 3) + j8;                 // local column of this lane
          const int idxj = s_idx[min(jlo + j, m - 1)];
          const int kind = (j < A) ? 0 : (j == A ? 1 : (j == A + 1 ? 2 : 3));
          const int t0 = k * SR + 32 * p + w4;          // row (item-relative) for q = 0
          unsigned char* hrow = hi + ((((p * Bs) >> 3) + g) << 10) + (j8 << 7) + (w4 << 2);
          unsigned char* lrow = hrow + kTcTileBytes;
          // the 8 K chunks of this lane are independent: evaluate all, then store
          float vv[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) {                // 4-row K chunks
            const int t = t0 + 4 * q;
            const float x = (float)(wk.r0 + t - idxj) * hs;
            const float u = x * x;
            const int tc = min(t, tmax);
            float A0 = RK.A0.hi, A1 = RK.A1.hi, A2 = RK.A2.hi, w1 = RK.w1.hi;
            if (!lin) {
              const float4 co = s_co[tc];
              A0 = co.x; A1 = co.y; A2 = co.z; w1 = co.w;
            }
            float v = exp_neg_fast(u) * fmaf(A2, u, fmaf(A1, x, A0));
            if (kind != 0) v = (kind == 1) ? w1 : (kind == 2 ? s_r[tc] : 0.f);
            vv[q] = (t < nrows) ? v : 0.f;
          }
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float h = to_tf32(vv[q]);
            const int ch = ((q ^ j8) & 7) << 4;        // 128-byte swizzle
            *reinterpret_cast<float*>(hrow + ch) = h;
            *reinterpret_cast<float*>(lrow + ch) = vv[q] - h;
          }
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&s_full[s]));
      }
      if (late && lane == 0) atomicExch(&s_abort, 1);
      // ---------------- epilogue (warps 0-3) ----------------
      if (warp < 4) {
        bool ok = !late && mbar_wait_bounded(smem_u32(&s_accf), ph_acc, kTcWaitIter);
        tc_fence_after();
        if (!ok) {
          if (lane == 0) atomicExch(&s_abort, 1);
        } else {
          // warp w holds TMEM lanes 32 w .. 32 w + 31 = rows of block p = 32 w / Bs;
          // stage its diagonal block (summed over the accumulators) in shared
          // memory: S[p][j][l], Bs x Bs per block (the stage buffers are idle)
          float* S = reinterpret_cast<float*>(sm);
          const int p = (32 * warp) / Bs;
          const int j = 32 * warp + lane - p * Bs;     // row within the block
          const int ncol = min(Bs, round_up(M2, 16));
          const uint32_t lanebase = tmem + ((uint32_t)(32 * warp) << 16);
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
                if (c0 + t < M2) S[(p * Bs + j) * Bs + c0 + t] = v;
              }
            }
          }
          asm volatile("bar.sync 1, 128;" ::: "memory");   // the four epilogue warps
          // slot: [first landmark, landmark count, packed upper local Gram];
          // (r, l) over the square, one entry per thread and step
          double* out = part + slot_off[wk.slot];
          if (tid == 0) { out[0] = (double)jlo; out[1] = (double)A; }
          const float invM2 = 1.0f / (float)M2;
          for (int e = tid; e < M2 * M2; e += 128) {
            const int r = (int)(((float)e + 0.5f) * invM2);
            const int l = e - r * M2;
            if (l >= r) {
              float sum = 0.f;
              for (int pp = 0; pp < P; ++pp) sum += S[(pp * Bs + r) * Bs + l];
              out[2 + r * M2 - r * (r - 1) / 2 - r + l] = (double)sum;
            }
          }
        }
      }
      ph_acc ^= 1u;
    } else if (lane == 0) {
      // ---------------- MMA issuer ----------------
      const uint32_t idesc = tc_idesc_tf32(128, N);
      bool late = false;
      uint32_t started = 0;   // accumulators written in this item
      int rot = 0;
      for (int k = 0; k < nst; ++k) {
        const int s = k & (kTcStages - 1);
        if (!mbar_wait_bounded(smem_u32(&s_full[s]), ph_full[s], kTcWaitIter)) { late = true; break; }
        ph_full[s] ^= 1u;
        tc_fence_after();
        const uint32_t ha = smem_u32(sm + s * kTcStageBytes);
        const uint32_t la = ha + (uint32_t)kTcTileBytes;
        for (int t = 0; t < 4; ++t) {                  // 4 K steps of 8 positions
          const uint64_t dh = tc_desc_sw128(ha + 32u * t);
          const uint64_t dl = tc_desc_sw128(la + 32u * t);
          const uint64_t da[3] = {dh, dh, dl}, db[3] = {dh, dl, dh};
#pragma unroll
          for (int q3 = 0; q3 < 3; ++q3) {
            const uint32_t d = tmem + (uint32_t)rot * kTcAccCols;
            tc_mma_tf32(d, da[q3], db[q3], idesc, (started >> rot) & 1u);
            started |= 1u << rot;
            rot = (rot + 1) & (kTcAcc - 1);
          }
        }
        tc_commit(smem_u32(&s_empty[s]));
      }
      if (late) {
        atomicExch(&s_abort, 1);
      } else {
        tc_commit(smem_u32(&s_accf));
        ++nacc;
      }
    }
  }

  if (s_abort && tid == 0) atomicExch(err, 1);
  // drain: MMAs still in flight finish before the tensor memory is released
  if (issuer && lane == 0) {
    tc_commit(smem_u32(&s_accf));
    mbar_wait_bounded(smem_u32(&s_accf), nacc & 1u, kTcWaitIter);
  }
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
