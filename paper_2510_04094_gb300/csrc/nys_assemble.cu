// Fused row pass of Lemma 1 (Section 3.1): for each collocation row i = 2..n,
// evaluate the RBF kernel and its t-derivatives against the m landmarks, apply
// the ODE operator, and accumulate the Gram of the augmented row
//     psi_i = [kappa_i (m); -f_p(t_i); r(t_i)],
//     kappa_i = k^(p)(t_i) - sum_k f_k(t_i) k^(p-k)(t_i),
// so that   G = sum psi psi^T  holds  sum kappa kappa^T, sum kappa (-f_p),
// sum f_p^2 and the right-hand sides sum kappa r, sum (-f_p) r.
// The Nystrom projection W is linear, so A^T A of Lemma 1 is B G B^T with
// B = blkdiag(W, 1); it is applied once per instance in the solve kernel
// instead of once per row, and no n x m feature matrix is ever stored.
//
// Work is a list of (instance, row range) items taken from an atomic queue by
// a persistent grid; each item writes its packed upper-triangular partial Gram
// (M2 (M2+1)/2 doubles, M2 = m + 2) to its own slot.  A Gram of more than
// kMMax + 2 columns is split into parts (packed entries [e0, e1), at most
// kAsm64Span each), one work item per part of a row range, all writing their own
// entries of the range's slot; k_gram_reduce then sums the slots of each such
// instance over many CTAs.
#include "nys_internal.cuh"

namespace nys {

// ---------------------------------------------------------------------------
// FP64 variant: one accumulator set per thread over packed Gram entries.
// ---------------------------------------------------------------------------
constexpr int kAsm64Threads = 256;
constexpr int kAsm64Rows = 32;

// Omega mode (landmark sets flagged ill-conditioned by the setup): the tile of
// kernel-coordinate rows is projected through W (psi_w = psi_k W^T, one m x m_eff
// product per row, as the feature map phi = W k of eq32 prescribes) and the
// Gram is accumulated over (m_eff + 2) omega-coordinate columns; the slot header
// then reads [-1, m_eff].
template <int KMAX>
__global__ void __launch_bounds__(kAsm64Threads)
k_assemble_f64(const Inst* __restrict__ insts, const Lset* __restrict__ lsets,
               const double* __restrict__ W_all, const Work* __restrict__ work, int nwork,
               int* __restrict__ counter, const int32_t* __restrict__ lm_idx,
               const double* __restrict__ tab, double* __restrict__ part,
               const int64_t* __restrict__ slot_off) {
  extern __shared__ double sm64[];
  __shared__ int s_item;
  __shared__ int s_idx[kMLarge];
  __shared__ double s_rc[kAsm64Rows][7];   // A0..A4, w1, r
  __shared__ unsigned char s_pair[2 * KMAX * kAsm64Threads];   // (j, l) of the item's entries
  static_assert(kMLarge + 2 <= 255, "Gram column index must fit a byte");
  const int tid = threadIdx.x;
  int cached_m2 = -1, cached_e0 = -1;

  for (;;) {
    if (tid == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int w = s_item;
    if (w >= nwork) break;
    const Work wk = work[w];
    const Inst I = insts[wk.inst];
    const int m = I.m, ld = m + 3;
    int omode = 0, me = m;
    if (lsets != nullptr) {
      const Lset L = lsets[I.lset];
      omode = L.omode;
      me = L.m_eff;
    }
    const double* W = (lsets != nullptr) ? W_all + lsets[I.lset].w_off : nullptr;
    const int D = omode ? me : m;          // feature columns of the Gram
    const int M2 = D + 2;
    const int Efull = M2 * (M2 + 1) / 2;
    // this item's packed entries [e0, e0 + E) (the host keeps e1 - e0 <= KMAX x threads)
    const int e0 = wk.e0;
    const int E = min(max(0, min(Efull, wk.e1) - e0), KMAX * kAsm64Threads);
    for (int j = tid; j < m; j += kAsm64Threads) s_idx[j] = lm_idx[I.lm_off + j];
    if (M2 != cached_m2 || e0 != cached_e0) {
      __syncthreads();
      // packed row j starts at S(j) = j M2 - j (j - 1) / 2: invert, then correct
      for (int e = tid; e < E; e += kAsm64Threads) {
        const int g = e0 + e;
        const double b2 = 2.0 * M2 + 1.0;
        int j = (int)((b2 - sqrt(b2 * b2 - 8.0 * g)) * 0.5);
        j = max(0, min(j, M2 - 1));
        while (j > 0 && j * M2 - j * (j - 1) / 2 > g) --j;
        while (j + 1 < M2 && (j + 1) * M2 - (j + 1) * j / 2 <= g) ++j;
        const int rem = g - (j * M2 - j * (j - 1) / 2);
        s_pair[2 * e] = (unsigned char)j;
        s_pair[2 * e + 1] = (unsigned char)(j + rem);
      }
      cached_m2 = M2;
      cached_e0 = e0;
    }
    double acc[KMAX];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) acc[k] = 0.0;
    __syncthreads();

    double* psi = sm64;
    for (int base = wk.r0; base < wk.r1; base += kAsm64Rows) {
      if (tid < kAsm64Rows) {
        const int i = base + tid;
        if (i < wk.r1) {
          const RowCoef4 R = row_coef_f64(I, tab, i);
#pragma unroll
          for (int q = 0; q < 5; ++q) s_rc[tid][q] = R.A[q];
          s_rc[tid][5] = R.w1;
          s_rc[tid][6] = R.rr;
        }
      }
      __syncthreads();
      for (int e = tid; e < kAsm64Rows * (m + 2); e += kAsm64Threads) {
        const int r = e / (m + 2), j = e - r * (m + 2);
        const int i = base + r;
        double val = 0.0;
        if (i < wk.r1) {
          if (j < m) {
            const double x = (double)(i - s_idx[j]) * I.hs;
            const double* A = s_rc[r];
            val = exp(-x * x) * fma(x, fma(x, fma(x, fma(x, A[4], A[3]), A[2]), A[1]), A[0]);
          } else {
            val = s_rc[r][5 + (j - m)];
          }
        }
        psi[r * ld + j] = val;
      }
      __syncthreads();
      if (omode) {  // project the kernel-coordinate rows: psi_w[r][k] = sum_j W[k][j] psi[r][j]
        // (only the columns k >= the item's first Gram row are read)
        double* pw = psi + kAsm64Rows * ld;
        const int k0 = (E > 0) ? s_pair[0] : M2, nk = M2 - k0;
        for (int e = tid; e < kAsm64Rows * nk; e += kAsm64Threads) {
          const int r = e / nk, k = k0 + (e - r * nk);
          double v;
          if (k < me) {
            v = 0.0;
            for (int j = 0; j < m; ++j) v = fma(W[k * m + j], psi[r * ld + j], v);
          } else {
            v = psi[r * ld + m + (k - me)];
          }
          pw[r * ld + k] = v;
        }
        __syncthreads();
      }
      const int rows = min(kAsm64Rows, wk.r1 - base);
      const double* pg = omode ? psi + kAsm64Rows * ld : psi;
#pragma unroll
      for (int k = 0; k < KMAX; ++k) {
        const int e = tid + k * kAsm64Threads;
        if (e < E) {
          const int j = s_pair[2 * e], l = s_pair[2 * e + 1];
          double a = acc[k];
          for (int r = 0; r < rows; ++r) a = fma(pg[r * ld + j], pg[r * ld + l], a);
          acc[k] = a;
        }
      }
      __syncthreads();
    }
    // slot layout: [first landmark, landmark count, packed upper Gram]
    double* out = part + slot_off[wk.slot];
    if (tid == 0 && e0 == 0) { out[0] = omode ? -1.0 : 0.0; out[1] = (double)D; }
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
      const int e = tid + k * kAsm64Threads;
      if (e < E) out[2 + e0 + e] = acc[k];
    }
  }
}

// ---------------------------------------------------------------------------
// FP32 variant (mixed-precision path).  The Gram is tiled in 8 x 8 register
// blocks of the upper triangle (U = NB (NB+1)/2 blocks, NB = MP/8); S row
// slices of U threads each split the rows of a tile, every thread running a
// plain FP32 FMA accumulation of its 64 entries over its rows (operands for
// the next row are loaded while the current row's 64 FMAs issue).  The S slice
// sums are added at the end of the work item and stored as doubles.  The
// accumulation error is removed later by FP64-accurate refinement.
// Features are evaluated per entry with the MUFU exponential (measured faster
// here than filling the tile from a lag table in shared memory, whose lookups
// across landmark columns conflict in the banks).
// Band structure: kappa_ij vanishes (exp(-u) < 2e-35, u > 80) once |i - idx_j|
// exceeds the landmark set's lag K, so a work item of consecutive rows only
// needs the landmarks idx_j in [r0 - K, r1 - 1 + K]: it accumulates the local
// Gram of that window (plus the -f_p and r columns) and records where the
// window starts; the solve kernel adds the local Grams into the full one.
// ---------------------------------------------------------------------------
constexpr int kAsm32Threads = 384;
constexpr int kAsm32Rows = 256;
constexpr int kPadF = 4;          // row padding of the psi tile (floats)

__global__ void __launch_bounds__(kAsm32Threads, 1)
k_assemble_f32(const Inst* __restrict__ insts, const Lset* __restrict__ lsets,
               const float* __restrict__ lag, const Work* __restrict__ work, int nwork,
               int* __restrict__ counter, const int32_t* __restrict__ lm_idx,
               const double* __restrict__ tab, double* __restrict__ part,
               const int64_t* __restrict__ slot_off, int tile_floats, int k_cap) {
  extern __shared__ __align__(16) float sm32[];
  __shared__ int s_item;
  __shared__ int s_idx[kMMax];
  __shared__ float s_rc[kAsm32Rows][5];
  const int tid = threadIdx.x;
  float* psi = sm32;
  (void)lsets; (void)lag; (void)tile_floats; (void)k_cap;

  for (;;) {
    if (tid == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int w = s_item;
    if (w >= nwork) break;
    const Work wk = work[w];
    const Inst I = insts[wk.inst];
    const int m = I.m;
    for (int j = tid; j < m; j += kAsm32Threads) s_idx[j] = lm_idx[I.lm_off + j];
    __syncthreads();
    // landmark window of this row range
    int jlo = 0, A = m;
    if (lsets != nullptr) {
      const int Kl = lsets[I.lset].K;
      int a = 0, b = m;
      while (a < b) { const int c = (a + b) >> 1; if (s_idx[c] < wk.r0 - Kl) a = c + 1; else b = c; }
      jlo = a;
      b = m;
      while (a < b) { const int c = (a + b) >> 1; if (s_idx[c] <= wk.r1 - 1 + Kl) a = c + 1; else b = c; }
      A = a - jlo;
    }
    const int M2 = A + 2;
    const int MP = round_up(M2, 8), NB = MP / 8, U = NB * (NB + 1) / 2;
    const int S = max(1, kAsm32Threads / U);
    const int ld = MP + kPadF;
    const RowConst RK = I.rk;

    // this thread's block (bj <= bl) and slice
    const bool active = tid < U * S;
    const int slice = tid / U, u = tid - slice * U;
    int bj = 0, bl = 0;
    {
      int rem = u;
      while (rem >= NB - bj) { rem -= NB - bj; ++bj; }
      bl = bj + rem;
    }
    // feature-phase mapping: column fj, rows fr0 + k*RS
    const int RS = kAsm32Threads / MP;
    const int fj = tid % MP, fr0 = tid / MP;
    const float hs = (float)I.hs;

    float acc[64];
#pragma unroll
    for (int k = 0; k < 64; ++k) acc[k] = 0.f;
    __syncthreads();
    const int sidx = (fj < A) ? s_idx[jlo + fj] : 0;

    for (int base = wk.r0; base < wk.r1; base += kAsm32Rows) {
      const int rows = min(kAsm32Rows, wk.r1 - base);
      // per-row quantities, one row per thread (r(t_i) needs a sine per row)
      if (tid < rows) {
        ff c5[5];
        row_coef_ff(I, RK, tab, base + tid, c5);
#pragma unroll
        for (int q = 0; q < 5; ++q) s_rc[tid][q] = c5[q].hi;
      }
      __syncthreads();
      if (fr0 < RS) {
        for (int r = fr0; r < kAsm32Rows; r += RS) {
          const int i = base + r;
          float val = 0.f;
          if (r < rows && fj < M2) {
            if (fj < A) {
              const float x = (float)(i - sidx) * hs;
              const float uu = x * x;
              val = exp_neg_fast(uu) * fmaf(s_rc[r][2], uu, fmaf(s_rc[r][1], x, s_rc[r][0]));
            } else {
              val = s_rc[r][3 + (fj - A)];
            }
          }
          psi[r * ld + fj] = val;
        }
      }
      __syncthreads();
      if (active && slice < rows) {
        const float* pa = psi + 8 * bj;
        const float* pb = psi + 8 * bl;
        int r = slice;
        float4 a0 = *reinterpret_cast<const float4*>(pa + r * ld);
        float4 a1 = *reinterpret_cast<const float4*>(pa + r * ld + 4);
        float4 b0 = *reinterpret_cast<const float4*>(pb + r * ld);
        float4 b1 = *reinterpret_cast<const float4*>(pb + r * ld + 4);
        for (;;) {
          const int rn = r + S;
          const bool more = rn < rows;
          float4 na0, na1, nb0, nb1;
          if (more) {
            na0 = *reinterpret_cast<const float4*>(pa + rn * ld);
            na1 = *reinterpret_cast<const float4*>(pa + rn * ld + 4);
            nb0 = *reinterpret_cast<const float4*>(pb + rn * ld);
            nb1 = *reinterpret_cast<const float4*>(pb + rn * ld + 4);
          }
          const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
          const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
          for (int x = 0; x < 8; ++x)
#pragma unroll
            for (int y = 0; y < 8; ++y) acc[x * 8 + y] = fmaf(av[x], bv[y], acc[x * 8 + y]);
          if (!more) break;
          a0 = na0; a1 = na1; b0 = nb0; b1 = nb1;
          r = rn;
        }
      }
      __syncthreads();
    }
    // add the S slice sums (FP32) and store the packed upper triangle as doubles
    // entry k of every thread's block at red[k * SU + thread]: consecutive threads
    // store to consecutive words (no bank conflicts)
    float* red = sm32;  // 64 * S * U floats <= 64 * 384 (the tile and table are dead)
    const int SU = S * U;
    if (active) {
#pragma unroll
      for (int k = 0; k < 64; ++k) red[k * SU + slice * U + u] = acc[k];
    }
    __syncthreads();
    // slot layout: [first landmark, landmark count, packed upper local Gram]
    const int E = M2 * (M2 + 1) / 2;
    double* out = part + slot_off[wk.slot];
    if (tid == 0) { out[0] = (double)jlo; out[1] = (double)A; }
    for (int e = tid; e < E; e += kAsm32Threads) {
      int j = 0, rem = e;
      while (rem >= M2 - j) { rem -= M2 - j; ++j; }
      const int l = j + rem;
      const int cb = j >> 3, lb = l >> 3;
      const int ub = cb * NB - cb * (cb - 1) / 2 + (lb - cb);
      const int k = (j & 7) * 8 + (l & 7);
      float sum = 0.f;
      for (int q = 0; q < S; ++q) sum += red[k * SU + q * U + ub];
      out[2 + e] = (double)sum;
    }
    __syncthreads();
  }
}

static int asm32_tile_floats(int m_max) {
  return kAsm32Rows * (round_up(m_max + 2, 8) + kPadF);
}

size_t asm_smem_bytes(bool fp32, int m_max, int k_cap) {
  const int M2 = m_max + 2;
  if (fp32) {
    const size_t tile = sizeof(float) * ((size_t)asm32_tile_floats(m_max) + 2 * (size_t)k_cap + 1);
    const size_t red = sizeof(float) * (size_t)kAsm32Threads * 64;
    return tile > red ? tile : red;
  }
  return sizeof(double) * 2 * (size_t)kAsm64Rows * (M2 + 1);
}

cudaError_t launch_assemble_tc(const Inst* insts, const Lset* lsets, const float* lag,
                               const Work* work, int nwork, int* counter, const int32_t* lm,
                               const double* tab, double* part, const int64_t* slot_off,
                               int32_t* err, int num_sms, int wait_iter, cudaStream_t st);
cudaError_t launch_assemble_band(const Inst* insts, const Lset* lsets, const float* lag,
                                 const Work* work, int nwork, int* counter, const int32_t* lm,
                                 double* part, const int64_t* slot_off, int32_t* err, int num_sms,
                                 cudaStream_t st);

// Sum of the row-chunk partial Grams of each listed instance (Grams of more than
// kMMax + 2 columns), into its first slot: a thread per packed entry, the slots
// added in their fixed order, so the result does not depend on the grid.
__global__ void __launch_bounds__(256)
k_gram_reduce(const Inst* __restrict__ insts, BigSet big, double* __restrict__ part,
              const int64_t* __restrict__ slot_off) {
  for (int bi = blockIdx.y; bi < big.n; bi += gridDim.y) {
    const Inst I = insts[big.ids[bi]];
    if (I.slot_count <= 1) continue;
    double* P0 = part + slot_off[I.slot_begin];
    const int D = (int)P0[1], M2 = D + 2, E = M2 * (M2 + 1) / 2;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
      double s = P0[2 + e];
      for (int q = 1; q < I.slot_count; ++q) s += part[slot_off[I.slot_begin + q] + 2 + e];
      P0[2 + e] = s;
    }
  }
}

template <int K>
static cudaError_t launch64(const Inst* insts, const Lset* lsets, const double* W,
                            const Work* work, int nwork, int* counter, const int32_t* lm,
                            const double* tab, double* part, const int64_t* slot_off, size_t sm,
                            int grid, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_assemble_f64<K>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_assemble_f64<K><<<grid, kAsm64Threads, sm, st>>>(insts, lsets, W, work, nwork, counter, lm,
                                                     tab, part, slot_off);
  return cudaGetLastError();
}

cudaError_t launch_assemble(bool fp32, const Inst* insts, const Lset* lsets, const float* lag,
                            const double* W, const Work* work, int nwork, int* counter,
                            const int32_t* lm, const double* tab, double* part,
                            const int64_t* slot_off, int m_max, int k_max, int num_sms,
                            cudaStream_t st, int asm_kind, int32_t* err, BigSet big,
                            int tc_wait, int nband) {
  // counter[0]: queue of the tensor-core / CUDA-core / FP64 kernel; counter[1]:
  // queue of the band kernel (the first nband work items)
  const bool band = fp32 && asm_kind == NYS_ASM_AUTO && err != nullptr && nband > 0;
  cudaError_t e = cudaMemsetAsync(counter, 0, (band ? 2 : 1) * sizeof(int), st);
  if (e != cudaSuccess) return e;
  if (err != nullptr) {  // error word read by the solve (NYS_ETIMEOUT / NYS_ESTATE)
    e = cudaMemsetAsync(err, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
  }
  if (fp32 && (asm_kind == NYS_ASM_AUTO || asm_kind == NYS_ASM_TC) && err != nullptr) {
    // band units on the CUDA cores, the rest on the tensor cores
    if (band) {
      e = launch_assemble_band(insts, lsets, lag, work, nband, counter + 1, lm, part, slot_off, err,
                               num_sms, st);
      if (e != cudaSuccess || nband >= nwork) return e;
    }
    return launch_assemble_tc(insts, lsets, lag, work + (band ? nband : 0), nwork - (band ? nband : 0),
                              counter, lm, tab, part, slot_off, err, num_sms,
                              tc_wait < 0 ? (1 << 22) : tc_wait, st);
  }
  // k_cap: capacity of the shared-memory kappa table, fixed at launch (an update
  // that lengthens the lag tables makes those instances use computed features)
  const int k_cap = 0;  // features are computed, no table in shared memory
  const size_t sm = asm_smem_bytes(fp32, m_max, k_cap);
  if (fp32) {
    e = cudaFuncSetAttribute(k_assemble_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int grid = min(nwork, num_sms);
    k_assemble_f32<<<grid, kAsm32Threads, sm, st>>>(insts, lsets, lag, work, nwork, counter, lm, tab,
                                                    part, slot_off, asm32_tile_floats(m_max), k_cap);
    return cudaGetLastError();
  }
  const int M2 = m_max + 2, E = M2 * (M2 + 1) / 2;
  const int kneed = (E + kAsm64Threads - 1) / kAsm64Threads;
  const int grid = min(nwork, num_sms * 2);
#define A64 insts, lsets, W, work, nwork, counter, lm, tab, part, slot_off, sm, grid, st
  if (kneed <= 4) e = launch64<4>(A64);
  else if (kneed <= 8) e = launch64<8>(A64);
  else if (kneed <= 14) e = launch64<14>(A64);
  else if (kneed <= 20) e = launch64<20>(A64);
  else e = launch64<kAsm64BigK>(A64);   // above kMMax the host splits Grams into parts
#undef A64
  if (e != cudaSuccess || big.n == 0) return e;
  // many CTAs per instance: the slots of a single long instance are summed at
  // HBM speed instead of by its one solve CTA
  const int EB = (kMLarge + 2) * (kMLarge + 3) / 2;
  k_gram_reduce<<<dim3(std::max(1, std::min((EB + 255) / 256, 4 * num_sms / std::max(1, big.n))),
                       std::min(big.n, 65535)), 256, 0, st>>>(insts, big, part, slot_off);
  return cudaGetLastError();
}

}  // namespace nys
