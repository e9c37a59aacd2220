// Per-instance solve of Lemma 1's system (Section 3.1) and, for the mixed
// path, residual refinement.
//
// Lemma 1 as a constrained least-squares problem in (omega, b):
//     [ H  C^T ] [x     ]   [g]     H = D + gamma B G_kk B^T  (D = diag(1_m, 0))
//     [ C  0   ] [lambda] = [v],    g = gamma B g_k,  B = blkdiag(W, 1)
// with G_kk, g_k the kernel-coordinate sums of the fused row pass and C the p
// condition rows, e.g. [phi(t_1) 1; phi'(t_1) 0] for second-order initial
// values (Lemma 1 sign convention: H x + C^T lambda = g).  Solved by the
// null-space method: Householder reflectors Q with Q^T C^T = [R; 0] (p <= 4),
// y = Q^T x, y_1 = R^{-T} v, Cholesky of the projected block H'_22 for y_2,
// lambda from the first p rows.
// The KKT matrix itself mixes scales gamma n |kappa|^2 and 1 (cond ~ 1e27);
// the projected block has the conditioning of the fit (~1e2-1e4 here).
//
// T = double: the plain FP64 path.  T = float: the factor of the mixed path;
// its error is removed by refinement passes whose residuals are computed
// from the definition of the problem with FP64-accurate features.
#include "nys_cta.cuh"

namespace nys {

constexpr int kSolveThreads = 128;
constexpr int kSolveThreadsBig = 512;   // global-workspace solves (m > kMMax)

int64_t fac_elems(int m_max) { return fac_elems_inline(m_max); }

// ---------------------------------------------------------------------------
// K3: form H, g, C; factor; solve.  One CTA per instance.
// Shared memory (m <= kMMax) or the instance's global area (m > kMMax):
// G (m+1) x (m+2) [T], H M1 x M1 [T], Y-block 8 x m [T], vectors.
// ---------------------------------------------------------------------------
// MM = kMMax: one CTA per instance, matrices in shared memory; instances with
// more landmarks are left to MM = kMLarge: one CTA per listed instance, the same
// steps on its own global (L2-resident) area, whose row chunks k_gram_reduce has
// already summed into the first slot.
// (FP32, shared memory: seven CTAs of 128 threads per SM)
template <typename T, int MM>
__global__ void __launch_bounds__(MM > kMMax ? kSolveThreadsBig : kSolveThreads,
                                  (MM <= kMMax && sizeof(T) == sizeof(float)) ? 7 : 1)
k_solve(const Inst* __restrict__ insts, const Lset* __restrict__ lsets,
        const double* __restrict__ W_all, const T* __restrict__ Wt_all,
        const double* __restrict__ part,
        const int64_t* __restrict__ slot_off, const int32_t* __restrict__ lm_idx,
        T* __restrict__ fac_all, int64_t facs, double* __restrict__ xs, double* __restrict__ zs,
        double* __restrict__ cws, int XS, int ZS, int M1S, const int32_t* __restrict__ st_init,
        int32_t* __restrict__ st_all, double gamma_scale, const int32_t* __restrict__ asm_err,
        BigSet big, const double* __restrict__ crow) {
  constexpr bool kBig = MM > kMMax;
  const int b = kBig ? big.ids[blockIdx.x] : blockIdx.x;
  const Inst I = insts[b];
  if (!kBig && I.m > kMMax) return;   // solved by the global-workspace variant
  const Lset LS = lsets[I.lset];
  // omega mode (ill-conditioned landmark kernel): the row pass projected each
  // row through W, so the slots hold the Gram in omega coordinates.  The FP32
  // factor is too coarse there; the mixed path reports NYS_EPRECISION.
  const bool om = (LS.omode != 0);
  // more conditions than unknowns (m_eff + 1 < p after truncation): no solution
  const int st0 = (st_init[b] != NYS_OK) ? st_init[b]
                  : (om && (sizeof(T) == sizeof(float) || asm_err != nullptr)) ? NYS_EPRECISION
                  : (asm_err != nullptr && *asm_err == 2) ? NYS_ESTATE   // stale band plan
                  : (asm_err != nullptr && *asm_err == kErrBounds) ? NYS_EBOUNDS
                  : (asm_err != nullptr && *asm_err != 0) ? NYS_ETIMEOUT
                  : (LS.m_eff == kMeffBounds) ? NYS_EBOUNDS
                  : (LS.m_eff + 1 < I.p) ? NYS_ENOTSPD : NYS_OK;
  if (st0 != NYS_OK) {  // no solution: zero x and z, report the status
    for (int k = threadIdx.x; k < XS; k += blockDim.x) xs[(int64_t)b * XS + k] = 0.0;
    for (int k = threadIdx.x; k < ZS; k += blockDim.x) zs[(int64_t)b * ZS + k] = 0.0;
    if (threadIdx.x == 0) st_all[b] = st0;
    return;
  }
  const int m = I.m, p = I.p, me = LS.m_eff;
  const int M1 = me + 1, N2 = M1 - p;
  const int Dg = om ? me : m;          // feature columns of the accumulated Gram
  const int ldg = Dg + 2, ldh = M1;
  const double* W = W_all + LS.w_off;  // m x m, rows < me
  const T* Wt = Wt_all + LS.w_off;     // same in T
  const double gamma = I.gamma * gamma_scale;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* Gs = kBig ? reinterpret_cast<T*>(big.ws + (int64_t)blockIdx.x * big.stride)
               : reinterpret_cast<T*>(smraw);             // (Dg+1) x (Dg+2), room for (m+1) x (m+2)
  T* Hs = Gs + (m + 1) * (m + 2);                    // M1 x M1
  T* Yb = Hs + M1 * ldh;                             // 8 x m
  T* vec = Yb + 8 * m;                               // misc vectors
  T* g = vec;                                        // M1
  T* hb = g + M1;                                    // me
  T* Vh = hb + M1;                                   // p x M1 Householder (p <= 4)
  T* w = Vh + 4 * M1;                                // M1 scratch
  T* y = w + M1;                                     // M1
  T* red = y + M1;                                   // 40
  // condition rows in omega coordinates (4 x (m+1)) and their kernel-coordinate
  // forms (4 x m), FP64, 16-byte aligned after the T area
  double* s_c = reinterpret_cast<double*>(
      (reinterpret_cast<uintptr_t>(red + 40) + 15) & ~static_cast<uintptr_t>(15));
  double* s_e = s_c + 4 * (m + 1);
  __shared__ int s_flag;
  __shared__ T s_beta[4], s_Rm[4][4];               // reflector scales, R (upper, p x p)

  // 1. add the partial Grams of the row chunks into G (symmetric, full).  A slot
  //    holds [first column jlo (-1: omega coordinates, all me columns), count A,
  //    packed upper Gram over the local columns (features jlo..jlo+A-1, then
  //    -f_p, then r)]; slots are added one after the other, so the sum order is
  //    fixed.
  for (int e = threadIdx.x; e < (Dg + 1) * ldg; e += blockDim.x) Gs[e] = T(0);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  bool dbg_bad = false;   // a slot whose column range leaves G (debug builds)
  for (int q = 0; q < (kBig ? 1 : I.slot_count); ++q) {
    const double* P = part + slot_off[I.slot_begin + q];
    const int jlo = (int)P[0] < 0 ? 0 : (int)P[0], A = (int)P[1], M2l = A + 2;
    if (!NYS_IDX_OK(A >= 0 && jlo + A <= Dg)) {
      dbg_bad = true;
      continue;
    }
    // a warp per packed row a (local columns bb >= a start at a M2l - a (a-1) / 2);
    // row A + 1 holds only the (r, r) entry, which is not needed
    for (int a = warp; a <= A; a += nw) {
      const int j = (a < A) ? jlo + a : Dg;
      const double* Pa = P + 2 + a * M2l - a * (a - 1) / 2 - a;
      for (int bb = a + lane; bb < M2l; bb += 32) {
        const int l = (bb < A) ? jlo + bb : Dg + (bb - A);
        const T v = (T)Pa[bb];
        Gs[j * ldg + l] += v;
        if (l <= Dg && l != j) Gs[l * ldg + j] += v;
      }
    }
    __syncthreads();
  }
  if (om) {
    // 2-3 in omega coordinates: H = D + gamma G, g = gamma G[:, r]
    for (int e = threadIdx.x; e < M1 * M1; e += blockDim.x) {
      const int k = e / M1, l = e - k * M1;
      Hs[k * ldh + l] = (T)gamma * Gs[k * ldg + l] + ((k == l && k < me) ? T(1) : T(0));
    }
    for (int k = threadIdx.x; k < M1; k += blockDim.x) g[k] = (T)gamma * Gs[k * ldg + me + 1];
    __syncthreads();
  } else {
    // 2. small pieces: H_wb = W G_kb, g_w = W g_k, H_bb, g_b
    for (int k = threadIdx.x; k < me; k += blockDim.x) {
      T s1 = 0, s2 = 0;
      for (int j = 0; j < m; ++j) {
        const T wkj = Wt[k * m + j];
        s1 += wkj * Gs[j * ldg + m];
        s2 += wkj * Gs[j * ldg + m + 1];
      }
      hb[k] = s1;
      g[k] = (T)gamma * s2;
    }
    if (threadIdx.x == 0) g[me] = (T)gamma * Gs[m * ldg + m + 1];
    __syncthreads();
    // 3. H_ww = gamma W G_kk W^T + I.  Y = W G_kk (odd row stride ldy) goes to
    //    the H area and the 8-row block after it when it fits; as G is
    //    symmetric, H_kl = sum_j W_kj Y_lj, so both products read a row of W
    //    that is the same for the whole warp (broadcast) and G or Y with unit
    //    or odd stride.  H is then written over G, which is no longer needed.
    //    Otherwise (many eigenpairs dropped) in blocks of 8 rows of Y.
    const T gbb = Gs[m * ldg + m];
    const int ldy = (m + 1) | 1;
    if (sizeof(T) == sizeof(float) && me * ldy <= M1 * ldh + 8 * m) {
      // FP32 factors: 4 x 4 register tiles (a tile reads 4 W and 4 G / Y values
      // per 16 multiply-adds)
      T* Ys = Hs;
      const int tk = (me + 3) >> 2, tl = (m + 3) >> 2;
      for (int e = threadIdx.x; e < tk * tl; e += blockDim.x) {
        const int k0 = 4 * (e / tl), l0 = 4 * (e - (e / tl) * tl);
        const T* wr[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) wr[a] = Wt + min(k0 + a, me - 1) * m;
        T acc[4][4] = {};
        for (int j = 0; j < m; ++j) {
          T w[4], gv[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) w[a] = wr[a][j];
#pragma unroll
          for (int c = 0; c < 4; ++c) gv[c] = Gs[j * ldg + min(l0 + c, m - 1)];
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][c] += w[a] * gv[c];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < 4; ++c)
            if (k0 + a < me && l0 + c < m) Ys[(k0 + a) * ldy + l0 + c] = acc[a][c];
      }
      __syncthreads();
      Hs = Gs;
      const int th = (me + 3) >> 2;
      for (int e = threadIdx.x; e < th * th; e += blockDim.x) {
        const int k0 = 4 * (e / th), l0 = 4 * (e - (e / th) * th);
        const T* wr[4];
        const T* yr[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          wr[a] = Wt + min(k0 + a, me - 1) * m;
          yr[a] = Ys + min(l0 + a, me - 1) * ldy;
        }
        T acc[4][4] = {};
        for (int j = 0; j < m; ++j) {
          T w[4], y[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) { w[a] = wr[a][j]; y[a] = yr[a][j]; }
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][c] += w[a] * y[c];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int k = k0 + a, l = l0 + c;
            if (k < me && l < me) Hs[k * ldh + l] = (T)gamma * acc[a][c] + (k == l ? T(1) : T(0));
          }
      }
    } else if (me * ldy <= M1 * ldh + 8 * m) {
      // each thread: rows k, k + 1 of one column (two independent sums per load)
      T* Ys = Hs;
      const int kp = (me + 1) >> 1;
      for (int e = threadIdx.x; e < kp * m; e += blockDim.x) {
        const int k = 2 * (e / m), l = e - (e / m) * m;
        const bool two = k + 1 < me;
        const T* w0 = Wt + k * m;
        const T* w1 = two ? w0 + m : w0;
        T s0 = 0, s1 = 0;
        for (int j = 0; j < m; ++j) {
          const T g = Gs[j * ldg + l];
          s0 += w0[j] * g;
          s1 += w1[j] * g;
        }
        Ys[k * ldy + l] = s0;
        if (two) Ys[(k + 1) * ldy + l] = s1;
      }
      __syncthreads();
      Hs = Gs;
      for (int e = threadIdx.x; e < kp * me; e += blockDim.x) {
        const int k = 2 * (e / me), l = e - (e / me) * me;
        const bool two = k + 1 < me;
        const T* w0 = Wt + k * m;
        const T* w1 = two ? w0 + m : w0;
        const T* yl = Ys + l * ldy;
        T s0 = 0, s1 = 0;
        for (int j = 0; j < m; ++j) {
          const T y = yl[j];
          s0 += w0[j] * y;
          s1 += w1[j] * y;
        }
        Hs[k * ldh + l] = (T)gamma * s0 + (k == l ? T(1) : T(0));
        if (two) Hs[(k + 1) * ldh + l] = (T)gamma * s1 + (k + 1 == l ? T(1) : T(0));
      }
    } else {
      for (int k0 = 0; k0 < me; k0 += 8) {
        const int kb = min(8, me - k0);
        for (int e = threadIdx.x; e < kb * m; e += blockDim.x) {
          const int kk = e / m, l = e - kk * m;
          T s = 0;
          for (int j = 0; j < m; ++j) s += Wt[(k0 + kk) * m + j] * Gs[j * ldg + l];
          Yb[kk * m + l] = s;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < kb * me; e += blockDim.x) {
          const int kk = e / me, l = e - kk * me;
          T s = 0;
          for (int j = 0; j < m; ++j) s += Yb[kk * m + j] * Wt[l * m + j];
          Hs[(k0 + kk) * ldh + l] = (T)gamma * s + ((k0 + kk) == l ? T(1) : T(0));
        }
        __syncthreads();
      }
    }
    for (int k = threadIdx.x; k < me; k += blockDim.x) {
      Hs[k * ldh + me] = (T)gamma * hb[k];
      Hs[me * ldh + k] = (T)gamma * hb[k];
    }
    if (threadIdx.x == 0) Hs[me * ldh + me] = (T)gamma * gbb;
  }
  // 4. condition rows in omega coordinates (FP64), c_r = [W k^(d_r)(tau_r); [d_r == 0]]:
  //    initial values (Lemma 1) tau_r = t_1, d_r = r; boundary values (Appendix A.4)
  //    t_1 then t_n, d_r = 0 for p = 2, and d_r = 0, 1 at each end for p = 4
  //    (Problem 16).  k^(d)(tau) = (-1/sigma)^d H_d(x) exp(-x^2), x = (tau - s_j)/sigma.
  const bool bvp = (I.bc == NYS_BC_BVP);
  const int hp = bvp ? p / 2 : p;                       // conditions at t_1
  // the set's rows (k_setup_crow) when this instance has the set's sigma: the
  // same numbers this block would form
  const bool use_crow = (crow != nullptr) && (I.sigma == insts[I.lset].sigma);
  if (use_crow) {
    const double* E = crow + (int64_t)I.lset * 8 * (XS - 3);
    for (int k = threadIdx.x; k < M1; k += blockDim.x) {
      double sr[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        if (r < p) {
          const int at_n = (r >= hp), d = at_n ? r - hp : r;
          sr[r] = (k < me) ? E[(4 * at_n + d) * (XS - 3) + k] : (d == 0 ? 1.0 : 0.0);
          s_c[r * (m + 1) + k] = sr[r];
        }
      }
      cws[(int64_t)b * 2 * M1S + k] = sr[0];
      cws[(int64_t)b * 2 * M1S + M1S + k] = sr[1];
    }
  }
  for (int e = threadIdx.x; e < (use_crow ? 0 : p * m); e += blockDim.x) {
    const int r = e / m, j = e - r * m;
    const int at_n = (r >= hp), d = at_n ? r - hp : r;
    const double x = (double)((at_n ? I.n - 1 : 0) - lm_idx[I.lm_off + j]) * I.hs;
    const double x2 = x * x;
    double H;                                           // physicists' Hermite H_d(x)
    if (d == 0) H = 1.0;
    else if (d == 1) H = 2.0 * x;
    else if (d == 2) H = 4.0 * x2 - 2.0;
    else H = (8.0 * x2 - 12.0) * x;
    double sc = 1.0;                                    // (-1/sigma)^d
    for (int q = 0; q < d; ++q) sc *= -1.0 / I.sigma;
    s_e[r * m + j] = sc * H * exp(-x2);
  }
  __syncthreads();
  for (int k = warp; k < (use_crow ? 0 : M1); k += nw) {   // a warp per row of W (coalesced)
    double sr[4] = {0.0, 0.0, 0.0, 0.0};
    if (k < me) {
      for (int j = lane; j < m; j += 32) {
        const double wkj = W[k * m + j];
#pragma unroll
        for (int r = 0; r < 4; ++r)
          if (r < p) sr[r] += wkj * s_e[r * m + j];
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
        for (int o = 16; o > 0; o >>= 1) sr[r] += __shfl_xor_sync(0xffffffffu, sr[r], o);
    } else {
#pragma unroll
      for (int r = 0; r < 4; ++r) sr[r] = (r < p && (r == 0 || r == hp)) ? 1.0 : 0.0;
    }
    if (lane == 0) {
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (r < p) s_c[r * (m + 1) + k] = sr[r];
      // rows 0, 1 for the refinement and gradient passes (orders <= 2)
      cws[(int64_t)b * 2 * M1S + k] = sr[0];
      cws[(int64_t)b * 2 * M1S + M1S + k] = sr[1];
    }
  }
  __syncthreads();
  // 5. Householder QR of C^T (M1 x p): column k (in the 8-row block buffer, free
  //    now) takes the reflectors 0..k-1, gives R[0..k-1][k], then its reflector
  T* cr = Yb;                                           // p x M1
  for (int e = threadIdx.x; e < p * M1; e += blockDim.x) {
    const int k = e / M1, i = e - k * M1;
    cr[e] = (T)s_c[k * (m + 1) + i];
    Vh[e] = T(0);
  }
  __syncthreads();
  for (int k = 0; k < p; ++k) {
    for (int j = 0; j < k; ++j) apply_house_vec(cr + k * M1, M1, Vh + j * M1, s_beta[j], red);
    if (threadIdx.x == 0)
      for (int j = 0; j < k; ++j) s_Rm[j][k] = cr[k * M1 + j];
    const T rkk = house(cr + k * M1 + k, Vh + k * M1 + k, M1 - k, &s_beta[k], red);
    if (threadIdx.x == 0) s_Rm[k][k] = rkk;
    __syncthreads();
  }
  // 6. H' = Q^T H Q, g' = Q^T g
  // (reflector k has zeros in its first k entries; apply it to the full matrix
  //  so the off-diagonal rows/columns are transformed too)
  for (int k = 0; k < p; ++k) {
    apply_house_sym(Hs, ldh, M1, Vh + k * M1, s_beta[k], w, red);
    apply_house_vec(g, M1, Vh + k * M1, s_beta[k], red);
  }
  // the stored factor (orders <= 2: refinement and gradient): the first p rows of
  // H', the reflectors and R
  T* facb = fac_all + (int64_t)b * facs;
  FacView<T> F = fac_view(facb, M1);
  if (p <= 2) {
    for (int e = threadIdx.x; e < p * M1; e += blockDim.x) {
      const int k = e / M1, j = e - k * M1;
      F.H1[k * M1 + j] = Hs[k * ldh + j];
      F.V[k * M1 + j] = Vh[k * M1 + j];
    }
    if (threadIdx.x < 2) F.beta[threadIdx.x] = (threadIdx.x < p) ? s_beta[threadIdx.x] : T(0);
    if (threadIdx.x == 0) {
      F.R[0] = s_Rm[0][0];
      F.R[1] = (p == 2) ? s_Rm[0][1] : T(0);
      F.R[2] = (p == 2) ? s_Rm[1][1] : T(0);
    }
  }
  // 7. y1 = R^{-T} v ; rhs2 = g'[p:] - H'[p:, :p] y1
  if (threadIdx.x == 0) {
    T yk[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (k < p) {
        T sv = (T)I.v[k];
#pragma unroll
        for (int j = 0; j < k; ++j) sv -= s_Rm[j][k] * yk[j];
        yk[k] = sv / s_Rm[k][k];
        y[k] = yk[k];
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < N2; i += blockDim.x) {
    T s = g[p + i];
    for (int k = 0; k < p; ++k) s -= Hs[(p + i) * ldh + k] * y[k];
    y[p + i] = s;
  }
  __syncthreads();
  // 8. Cholesky of H'_22 and solve (rows 0..p-1 of H' stay as they are)
  T* A22 = Hs + p * ldh + p;
  const bool ok = block_cholesky(A22, ldh, N2, &s_flag);
  cta_chol_solve(A22, ldh, N2, y + p);
  if (p <= 2) {
    for (int e = threadIdx.x; e < N2 * N2; e += blockDim.x) {
      const int i = e / N2, j = e - i * N2;
      F.L[i * N2 + j] = (j <= i) ? A22[i * ldh + j] : T(0);
    }
  }
  // 9. lambda = R^{-1}(g'[:p] - H'[:p, :] y)
  // (loops over the fixed bound 4 keep qk and lam in registers)
  T qk[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) qk[k] = (k < p) ? cta_dot(Hs + k * ldh, y, M1, red) : T(0);
  double lam[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int k = 3; k >= 0; --k) {
    if (k < p) {
      T sv = g[k] - qk[k];
#pragma unroll
      for (int j = k + 1; j < 4; ++j)
        if (j < p) sv -= s_Rm[k][j] * (T)lam[j];
      lam[k] = (double)(sv / s_Rm[k][k]);
    }
  }
  const double lam0 = lam[0], lam1 = lam[1];
  // 10. x = Q y
  for (int k = p - 1; k >= 0; --k) apply_house_vec(y, M1, Vh + k * M1, s_beta[k], red);
  double* xb = xs + (int64_t)b * XS;
  for (int k = threadIdx.x; k < XS; k += blockDim.x) {
    double val = 0.0;
    if (k < me) val = (double)y[k];
    else if (k == XS - 3) val = (double)y[me];
    else if (k == XS - 2) val = lam0;                 // the first two multipliers
    else if (k == XS - 1) val = (p >= 2) ? lam1 : 0.0;
    xb[k] = val;
  }
  __syncthreads();
  // 11. kernel coordinates z = W^T omega, b
  double* zb = zs + (int64_t)b * ZS;
  for (int j = threadIdx.x; j <= m; j += blockDim.x) {
    double s = 0.0;
    if (j < m) {
      for (int k = 0; k < me; ++k) s += W[k * m + j] * xb[k];
    } else {
      s = xb[XS - 3];
    }
    zb[j] = s;
  }
  if (threadIdx.x == 0) {
    int st = ok ? NYS_OK : NYS_ENOTSPD;
    bool fin = isfinite((double)y[me]);
#pragma unroll
    for (int k = 0; k < 4; ++k) fin = fin && (k >= p || isfinite(lam[k]));
    if (ok && !fin) st = NYS_ENONFINITE;
    if (dbg_bad) st = NYS_EBOUNDS;
    st_all[b] = st;
  }
}

size_t solve_smem_bytes(bool fp32, int m_max) {
  const int m = m_max, M1 = m + 1;
  const size_t es = fp32 ? sizeof(float) : sizeof(double);
  return es * ((size_t)(m + 1) * (m + 2) + (size_t)M1 * M1 + 8 * m + 8 * M1 + 40) + 16 +
         sizeof(double) * (4 * (size_t)(m + 1) + 4 * (size_t)m);
}

size_t solve_ws_doubles() { return solve_smem_bytes(false, kMLarge) / sizeof(double) + 1; }

// ---------------------------------------------------------------------------
// K4a: refinement row pass (mixed path).  For each row the residual
//     s_i = r_i - kappa~_i^T z~,   z~ = (W^T omega, b)   (kernel coordinates)
// with FP64-accurate features, in float-float, then acc_j += kappa~_ij s_i.
// Features come from the landmark set's lag tables (k_setup_lag): kappa_ij =
// A0 b0(k) + A1 b1(k) + A2 b2(k), k = i - idx_j.  For constant coefficients
// (kind LIN) the combination is folded once per work item into a kappa(k)
// table in shared memory; otherwise (kind TABLE, or a table too large for
// shared memory) it is formed per entry from the global tables.
// ---------------------------------------------------------------------------
constexpr int kRefThreads = 256;
constexpr int kRefRows = 256;
constexpr int kRefLagMax = 10000;   // largest K of the shared-memory kappa table
constexpr int kRefPad = 32;         // zero entries on each side of the kappa table
static_assert(kRefRows == kRefThreads, "the residual pass maps one row to each thread");

__device__ __forceinline__ ff ff_mul(ff a, ff b) { return ff_mul_ff(a, b); }

// kappa of lag k from the global lag tables and float-float coefficients
__device__ __forceinline__ ff kappa_lag(const float* __restrict__ T, int K, int k, ff A0, ff A1,
                                        ff A2) {
  const int a = k < 0 ? -k : k;
  if (a > K) return {0.f, 0.f};
  const float* t = T + 6 * a;
  ff b1 = {t[2], t[3]};
  if (k < 0) { b1.hi = -b1.hi; b1.lo = -b1.lo; }
  ff r = ff_mul(A0, ff{t[0], t[1]});
  r = ff_add(r, ff_mul(A1, b1));
  r = ff_add(r, ff_mul(A2, ff{t[4], t[5]}));
  return r;
}

// acc += a * b for float-float a, b: exact leading product by FMA, TwoSum on
// the high parts, everything else gathered in the low part (renormalised by
// the caller at the end).
__device__ __forceinline__ void ff_acc_mul(ff& acc, ff a, ff b) {
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
__device__ __forceinline__ ff ff_norm(ff a) {
  const float hi = a.hi + a.lo;
  return {hi, a.lo - (hi - a.hi)};
}

constexpr int kRefWarps = kRefThreads / 32;

// four CTAs per SM (64 registers): occupancy hides the latency of the
// float-float chains better than the registers saved would
__global__ void __launch_bounds__(kRefThreads, 4)
k_refine_rows(const Inst* __restrict__ insts, const Lset* __restrict__ lsets,
              const float* __restrict__ lag, const Work* __restrict__ work, int nwork,
              int* __restrict__ counter, const int32_t* __restrict__ lm_idx,
              const double* __restrict__ tab, const double* __restrict__ zs, int ZS,
              double* __restrict__ part, const int64_t* __restrict__ slot_off,
              const int32_t* __restrict__ st_all, const int32_t* __restrict__ skip_in, int k_cap) {
  // k_cap: capacity of the shared-memory kappa table (fixed at launch, so a
  // graph captured earlier stays safe when an update lengthens the tables)
  extern __shared__ __align__(16) float2 smr[];
  __shared__ int s_item;
  __shared__ int s_idx[kMMax];
  __shared__ float4 s_zj[kM1Max];   // per column: z~ hi, lo, landmark index (bits), -
  __shared__ float2 s_s[kRefRows];  // residuals (float-float)
  __shared__ float2 s_acc[kM1Max];  // column sums of the item (float-float)
  __shared__ float s_rc[kRefRows * 10];  // per row: A0 A1 A2 w1 r, each as hi/lo
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int wi = s_item;
    if (wi >= nwork) break;
    const Work wk = work[wi];
    const Inst I = insts[wk.inst];
    const Lset L = lsets[I.lset];
    const float* T = lag + L.lag_off;
    const int m = I.m, K = L.K;
    const bool folded = (I.kind == NYS_COEF_LIN) && (K <= k_cap);
    float2* kk = smr;   // kappa(t - K - kRefPad), t = 0..2K + 2 kRefPad, float-float
    for (int j = tid; j < m; j += kRefThreads) s_idx[j] = lm_idx[I.lm_off + j];
    for (int j = tid; j <= m; j += kRefThreads) {
      const ff z = ff_from_double(zs[(int64_t)wk.inst * ZS + j]);
      s_zj[j] = make_float4(z.hi, z.lo, __int_as_float(j < m ? lm_idx[I.lm_off + j] : 0), 0.f);
    }
    // instances that failed, or that an adaptive pass leaves out (skip_in)
    const bool skip = (st_all[wk.inst] != NYS_OK) || (skip_in && skip_in[wk.inst]);
    const RowConst RK = I.rk;
    if (folded && !skip) {  // constant operator: kappa(k) for k = -K..K
      // (zero beyond lag K, so the padding holds zeros)
      for (int t = tid; t <= 2 * (K + kRefPad); t += kRefThreads) {
        const ff kv = kappa_lag(T, K, t - K - kRefPad, RK.A0, RK.A1, RK.A2);
        kk[t] = make_float2(kv.hi, kv.lo);
      }
    }
    // The sums acc_j = sum_i kappa~_ij s_i cancel almost completely at the
    // solution (the residual is orthogonal to the features up to the
    // regularisation), so they are accumulated in float-float.  Warp w owns
    // columns j = w, w + 8, ...; its lanes walk the rows of a chunk, then the
    // warp adds its lane sums into s_acc[j].
    for (int j = tid; j <= m; j += kRefThreads) s_acc[j] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int base = wk.r0; base < wk.r1 && !skip; base += kRefRows) {
      const int rows = min(kRefRows, wk.r1 - base);
      // per-row coefficients (float-float)
      for (int r = tid; r < rows; r += kRefThreads) {
        ff c5[5];
        row_coef_ff(I, RK, tab, base + r, c5);
        float* rc = s_rc + r * 10;
#pragma unroll
        for (int q = 0; q < 5; ++q) { rc[2 * q] = c5[q].hi; rc[2 * q + 1] = c5[q].lo; }
      }
      __syncthreads();
      // residual of each row, one row per thread: s = r - kappa~^T z~.  kappa
      // vanishes beyond lag K; a warp walks the landmarks within lag K of any
      // of its 32 rows (one range for all lanes), so a lane's lag stays within
      // K + 31 and its table index inside the zero padding.
      if (warp * 32 < rows) {
        const int ia = base + warp * 32, ib = base + min(rows, warp * 32 + 32) - 1;
        int a = 0, b = m;             // first j with idx_j >= ia - K
        while (a < b) { const int c = (a + b) >> 1; if (s_idx[c] < ia - K) a = c + 1; else b = c; }
        const int jlo = a;
        b = m;                        // first j with idx_j > ib + K
        while (a < b) { const int c = (a + b) >> 1; if (s_idx[c] <= ib + K) a = c + 1; else b = c; }
        const int jhi = a;
        const int r = tid;
        if (r < rows) {
          const int i = base + r;
          const float* rc = s_rc + r * 10;
          ff sp = {0.f, 0.f};   // sum of kappa~ z~ (subtracted at the end)
          if (folded) {
            // two interleaved accumulators: independent dependency chains
            const int iK = i + K + kRefPad;
            ff sp1 = {0.f, 0.f};
            int j = jlo;
            for (; j + 1 < jhi; j += 2) {
              const float4 z0 = s_zj[j], z1 = s_zj[j + 1];
              const float2 k0 = kk[iK - __float_as_int(z0.z)], k1 = kk[iK - __float_as_int(z1.z)];
              ff_acc_mul(sp, ff{k0.x, k0.y}, ff{z0.x, z0.y});
              ff_acc_mul(sp1, ff{k1.x, k1.y}, ff{z1.x, z1.y});
            }
            if (j < jhi) {
              const float4 z0 = s_zj[j];
              const float2 k0 = kk[iK - __float_as_int(z0.z)];
              ff_acc_mul(sp, ff{k0.x, k0.y}, ff{z0.x, z0.y});
            }
            sp = ff_add(ff_norm(sp), ff_norm(sp1));
          } else {
            const ff A0 = {rc[0], rc[1]}, A1 = {rc[2], rc[3]}, A2 = {rc[4], rc[5]};
            for (int j = jlo; j < jhi; ++j) {
              const float4 zj = s_zj[j];
              ff_acc_mul(sp, kappa_lag(T, K, i - __float_as_int(zj.z), A0, A1, A2), ff{zj.x, zj.y});
            }
          }
          const float4 zb = s_zj[m];
          ff_acc_mul(sp, ff{rc[6], rc[7]}, ff{zb.x, zb.y});
          sp = ff_norm(sp);
          const ff sres = ff_add(ff{rc[8], rc[9]}, ff{-sp.hi, -sp.lo});
          s_s[r] = make_float2(sres.hi, sres.lo);
        }
      }
      __syncthreads();
      // acc_j += kappa~_ij s_i: lanes over rows (conflict-free table reads), one
      // column at a time (a compact loop: the column count varies per chunk)
#pragma unroll 1
      for (int j = warp; j <= m; j += kRefWarps) {
        int rlo = 0, rhi = rows, toff = 0, cj = 0;
        if (j < m) {
          // rows within lag K of landmark j: table index r + toff in the table
          cj = s_idx[j];
          rlo = max(0, cj - K - base);
          rhi = min(rows, cj + K + 1 - base);
          toff = base - cj + K + kRefPad;
        }
        if (rlo >= rhi) continue;                        // warp-uniform
        ff a = {0.f, 0.f};
        if (j == m) {          // the b column: every row
          for (int r = lane; r < rows; r += 32) {
            const float* rc = s_rc + r * 10;
            const float2 sv = s_s[r];
            ff_acc_mul(a, ff{rc[6], rc[7]}, ff{sv.x, sv.y});
          }
        } else if (folded) {
          for (int r = rlo + lane; r < rhi; r += 32) {
            const float2 kv = kk[r + toff], sv = s_s[r];
            ff_acc_mul(a, ff{kv.x, kv.y}, ff{sv.x, sv.y});
          }
        } else {
          for (int r = rlo + lane; r < rhi; r += 32) {
            const float* rc = s_rc + r * 10;
            const ff kv = kappa_lag(T, K, base + r - cj, ff{rc[0], rc[1]}, ff{rc[2], rc[3]},
                                    ff{rc[4], rc[5]});
            const float2 sv = s_s[r];
            ff_acc_mul(a, kv, ff{sv.x, sv.y});
          }
        }
        a = ff_norm(a);
        for (int o = 16; o > 0; o >>= 1) {
          const ff bb = {__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
          a = ff_add(a, bb);
        }
        if (lane == 0) {                                 // column j belongs to this warp
          const float2 cur = s_acc[j];
          const ff t = ff_add(ff{cur.x, cur.y}, a);
          s_acc[j] = make_float2(t.hi, t.lo);
        }
      }
      __syncthreads();
    }
    // write the partial (M1 doubles)
    double* out = part + slot_off[wk.slot];
    for (int j = tid; j <= m; j += kRefThreads) {
      const float2 a = s_acc[j];
      out[j] = skip ? 0.0 : (double)a.x + (double)a.y;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// K4b: refinement update per instance (FP64 residual equations, T factor):
//   h = gamma B acc - D x - C^T lambda,  c = v - C x,  [dx; dl] = K~^{-1} [h; c]
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kSolveThreads)
k_refine_update(const Inst* __restrict__ insts, const Lset* __restrict__ lsets,
                const double* __restrict__ W_all, const double* __restrict__ part,
                const int64_t* __restrict__ slot_off, const T* __restrict__ fac_all, int64_t facs,
                double* __restrict__ xs, double* __restrict__ zs, const double* __restrict__ cws,
                int XS, int ZS, int M1S, int32_t* __restrict__ st_all, double gamma_scale,
                double* __restrict__ rcorr, int pass, int last,
                const int32_t* __restrict__ skip_in, int32_t* __restrict__ skip_out) {
  const int b = blockIdx.x;
  if (st_all[b] != NYS_OK || (skip_in && skip_in[b])) return;
  const Inst& I = insts[b];   // a reference: I.v[tid] would copy the struct to local memory
  const Lset LS = lsets[I.lset];
  const int m = I.m, p = I.p, me = LS.m_eff, M1 = me + 1;
  const double* W = W_all + LS.w_off;
  const double gamma = I.gamma * gamma_scale;
  __shared__ double acc[kM1Max + 1];
  __shared__ T h[kM1Max + 1], dx[kM1Max + 1], red[40];
  __shared__ T cr[2], dl[2];
  __shared__ double xsh[kM1Max + 3];   // x = (omega, b, lambda)
  double* xb = xs + (int64_t)b * XS;
  // the previous pass's relative correction, read early (used at the end)
  const double prev_d = (threadIdx.x == 0 && pass > 0) ? rcorr[b] : 0.0;
  const double* C0 = cws + (int64_t)b * 2 * M1S;
  const double* C1 = C0 + M1S;
  // the stored factor L into shared memory first: its loads overlap the rest
  const FacView<T> F = fac_view(const_cast<T*>(fac_all) + (int64_t)b * facs, M1);
  extern __shared__ __align__(16) unsigned char upd_raw[];   // the factor L, N2 x N2
  T* Ls = reinterpret_cast<T*>(upd_raw);
  {
    const int ne = (M1 - p) * (M1 - p);
    unsigned dyn = 0;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    if (!NYS_IDX_OK((size_t)ne * sizeof(T) <= dyn)) {
      if (threadIdx.x == 0) st_all[b] = NYS_EBOUNDS;
      return;
    }
#pragma unroll 4
    for (int e = threadIdx.x; e < ne; e += blockDim.x) Ls[e] = F.L[e];
  }
  for (int j = threadIdx.x; j < XS; j += blockDim.x) xsh[j] = xb[j];
  for (int j = threadIdx.x; j <= m; j += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < I.rslot_count; ++q) s += part[slot_off[I.rslot_begin + q] + j];
    acc[j] = s;
  }
  __syncthreads();
  const double lam0 = xsh[XS - 2], lam1 = (p == 2) ? xsh[XS - 1] : 0.0;
  for (int k = threadIdx.x; k < M1; k += blockDim.x) {
    double s;
    if (k < me) {
      // two interleaved partial sums (the DFMA chain halved)
      double s0 = 0.0, s1 = 0.0;
      const double* wk = W + k * m;
      int j = 0;
#pragma unroll 4
      for (; j + 1 < m; j += 2) {
        s0 += wk[j] * acc[j];
        s1 += wk[j + 1] * acc[j + 1];
      }
      if (j < m) s0 += wk[j] * acc[j];
      s = gamma * (s0 + s1) - xsh[k];
    } else {
      s = gamma * acc[m];
    }
    s -= C0[k] * lam0;
    if (p == 2) s -= C1[k] * lam1;
    h[k] = (T)s;
  }
  if (threadIdx.x < p) {
    const double* Ck = threadIdx.x == 0 ? C0 : C1;
    double s = I.v[threadIdx.x];
    for (int k = 0; k < me; ++k) s -= Ck[k] * xsh[k];
    s -= Ck[me] * xsh[XS - 3];
    cr[threadIdx.x] = (T)s;
  }
  __syncthreads();
  kkt_apply(F, M1, p, h, cr, dx, dl, red, Ls, true);
  // largest correction (FP32) and solution entry (high word of |x|: the exponent
  // and 20 mantissa bits, an integer max) over (omega, b), for the trust check
  float dmax = 0.f;
  int xhi = 0;
  for (int k = threadIdx.x; k < M1; k += blockDim.x) {
    const int slot = (k < me) ? k : XS - 3;
    const double v = xsh[slot] + (double)dx[k];
    xsh[slot] = v;
    xb[slot] = v;
    dmax = fmaxf(dmax, fabsf((float)dx[k]));
    xhi = max(xhi, __double2hiint(v) & 0x7fffffff);
  }
  for (int o = 16; o > 0; o >>= 1) {
    dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    xhi = max(xhi, __shfl_xor_sync(0xffffffffu, xhi, o));
  }
  __shared__ float s_dx[kSolveThreads / 32];
  __shared__ int s_xh[kSolveThreads / 32];
  if ((threadIdx.x & 31) == 0) {
    s_dx[threadIdx.x >> 5] = dmax;
    s_xh[threadIdx.x >> 5] = xhi;
  }
  if (threadIdx.x == 0) {
    xsh[XS - 2] += (double)dl[0];
    xb[XS - 2] = xsh[XS - 2];
    if (p == 2) {
      xsh[XS - 1] += (double)dl[1];
      xb[XS - 1] = xsh[XS - 1];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // Refinement trust.  d = max|dx| / max|x| over (omega, b) is this pass's
    // relative correction.  A pass contracts the error by a factor rho that is
    // about the relative error of the FP32 solve itself, i.e. the first pass's d,
    // and, once two passes ran, the ratio of the last two corrections; the error
    // left after the last pass is then about rho * d.  Above kRefineTrust the
    // factor is too coarse (an ill-conditioned landmark kernel through the FP32
    // Gram, e.g.; rho >= 1 means the passes diverge) and the instance reports
    // NYS_EPRECISION instead of a solution that does not converge.
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      dmax = fmaxf(dmax, s_dx[w]);
      xhi = max(xhi, s_xh[w]);
    }
    const double xmax = __hiloint2double(xhi, 0);
    const double d = dmax > 0.f ? (double)dmax / xmax : 0.0;   // NaN / inf when x is 0 or not finite
    const double rho = pass == 0 ? d : (prev_d > 0.0 ? d / prev_d : (d > 0.0 ? 1.0 : 0.0));
    rcorr[b] = d;
    if (last && !(rho * d <= kRefineTrust)) st_all[b] = NYS_EPRECISION;
    // the adaptive pass that follows: only instances still above kRefineAgain
    if (skip_out) skip_out[b] = (rho * d <= kRefineAgain) ? 1 : 0;
  }
  double* zb = zs + (int64_t)b * ZS;
  for (int j = threadIdx.x; j <= m; j += blockDim.x) {
    double s = 0.0;
    if (j < m) {
      double s0 = 0.0, s1 = 0.0;
      int k = 0;
#pragma unroll 4
      for (; k + 1 < me; k += 2) {
        s0 += W[k * m + j] * xsh[k];
        s1 += W[(k + 1) * m + j] * xsh[k + 1];
      }
      if (k < me) s0 += W[k * m + j] * xsh[k];
      s = s0 + s1;
    } else {
      s = xsh[XS - 3];
    }
    zb[j] = s;
  }
  if (threadIdx.x == 0) {
    if (!isfinite(xb[XS - 3]) || !isfinite(xb[XS - 2])) st_all[b] = NYS_ENONFINITE;
  }
}

// ---------------------------------------------------------------------------
// Newton step for Lemma 2 (Eq. 3.2.1), one CTA per instance, FP64.  Reads the
// partials of k_newton_pass (reduced Gram G and vectors v, u in kernel
// coordinates, sum Fy^2, small-pivot count) and
//   grad_x L = D x + C^T lambda + B u,   |F|^2 = |grad_x L|^2 + sum Fy^2 + |C x - v|^2,
// applies the stopping rule (|dx_prev| <= tol (1 + |x|) and |F| <= tol max(1, |F0|),
// x = (omega, b)) and the iteration cap, falls back to Gauss-Newton (re-pass,
// mode 1) when a pivot d_i <= 1e-12 gamma or the projected reduced Hessian is
// not positive definite, and otherwise solves
//   [D + B G B^T, C^T; C, 0] [dx; dlambda] = [-(D x + C^T lambda + B v); v - C x]
// by the null-space Cholesky method and updates x, lambda, z = B^T x, dz = B^T dx.
// flags[0]: some instance took a step; flags[1]: some instance needs a re-pass.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSolveThreads)
k_newton_step(const Inst* __restrict__ insts, const Lset* __restrict__ lsets,
              const double* __restrict__ W_all, const double* __restrict__ part,
              const int64_t* __restrict__ slot_off, const int32_t* __restrict__ lm_idx,
              double* __restrict__ xs, double* __restrict__ zs, double* __restrict__ dzs,
              double* __restrict__ cws, int XS, int ZS, int M1S, int32_t* __restrict__ st_all,
              int32_t* __restrict__ active, int32_t* __restrict__ iters, double* __restrict__ nrm,
              int max_iter, double tol, int32_t* __restrict__ flags, int mode,
              int32_t* __restrict__ live) {
  const int b = blockIdx.x;
  if (*live == 0) return;   // every instance has stopped
  const int act = active[b];
  if (act == 0 || (mode == 1 && act != 2)) return;
  const Inst I = insts[b];
  const Lset LS = lsets[I.lset];
  const int m = I.m, p = I.p, me = LS.m_eff;
  // omega mode: the row pass accumulated G, v, u in omega coordinates (D = me)
  const bool om = (LS.omode != 0);
  const int D = om ? me : m;
  const int M1 = me + 1, M1k = D + 1, N2 = M1 - p;
  const int ldg = D + 2, ldh = M1;
  const int E1 = M1k * (M1k + 1) / 2;
  const double* W = W_all + LS.w_off;
  extern __shared__ __align__(16) unsigned char smraw_nt[];
  double* Gs = reinterpret_cast<double*>(smraw_nt);   // (D+1) x (D+2): G | v
  double* Hs = Gs + (m + 1) * (m + 2);                 // M1 x M1
  double* Yb = Hs + M1 * ldh;                          // 8 x m
  double* g = Yb + 8 * m;                              // M1
  double* hb = g + M1;
  double* Vh = hb + M1;                                // 2 x M1
  double* c2 = Vh + 2 * M1;
  double* w = c2 + M1;
  double* y = w + M1;
  double* red = y + M1;                                // 40
  __shared__ double s_u[kM1Max], s_gx[kM1Max + 1];
  __shared__ double s_c[2][kM1Max];
  __shared__ double s_sc[4];   // sum Fy^2, small count, |h|^2, |x|^2
  __shared__ double s_beta[2], s_R[4];
  __shared__ int s_flag;
  double* xb = xs + (int64_t)b * XS;

  // 1. partial sums in slot order
  for (int e = threadIdx.x; e < (D + 1) * ldg; e += blockDim.x) Gs[e] = 0.0;
  if (threadIdx.x < 4) s_sc[threadIdx.x] = 0.0;
  __syncthreads();
  for (int q = 0; q < I.slot_count; ++q) {
    const double* P = part + slot_off[I.slot_begin + q];
    for (int e = threadIdx.x; e < E1; e += blockDim.x) {
      int j = 0, rem = e;
      while (rem >= M1k - j) { rem -= M1k - j; ++j; }
      const int l = j + rem;
      Gs[j * ldg + l] += P[e];
      if (l != j) Gs[l * ldg + j] += P[e];
    }
    for (int j = threadIdx.x; j <= D; j += blockDim.x) {
      Gs[j * ldg + D + 1] += P[E1 + j];
      s_u[j] = (q == 0 ? 0.0 : s_u[j]) + P[E1 + M1k + j];
    }
    if (threadIdx.x == 0) {
      s_sc[0] += P[E1 + 2 * M1k];
      s_sc[1] += P[E1 + 2 * M1k + 1];
    }
    __syncthreads();
  }
  // 2. condition rows in omega coordinates (initial values: [W k(t_1); 1],
  //    [W k'(t_1); 0]; boundary values, Appendix A.4: [W k(t_1); 1], [W k(t_n); 1]),
  //    grad_x L, |F|
  __shared__ double s_e[2][kMMax];
  const bool bvp = (I.bc == NYS_BC_BVP);
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    const double x = (double)(0 - lm_idx[I.lm_off + j]) * I.hs;
    const double e = exp(-x * x);
    s_e[0][j] = e;
    if (bvp) {
      const double xn = (double)(I.n - 1 - lm_idx[I.lm_off + j]) * I.hs;
      s_e[1][j] = exp(-xn * xn);
    } else {
      s_e[1][j] = (-2.0 * x / I.sigma) * e;
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < M1; k += blockDim.x) {
    double s0 = 0.0, s1 = 0.0;
    if (k < me) {
      for (int j = 0; j < m; ++j) {
        s0 += W[k * m + j] * s_e[0][j];
        s1 += W[k * m + j] * s_e[1][j];
      }
    } else {
      s0 = 1.0;
      s1 = bvp ? 1.0 : 0.0;
    }
    s_c[0][k] = s0;
    s_c[1][k] = s1;
    cws[(int64_t)b * 2 * M1S + k] = s0;
    cws[(int64_t)b * 2 * M1S + M1S + k] = s1;
  }
  __syncthreads();
  const double lam0 = xb[XS - 2], lam1 = (p == 2) ? xb[XS - 1] : 0.0;
  for (int k = threadIdx.x; k < M1; k += blockDim.x) {
    double s;
    if (k < me) {
      s = xb[k];
      if (om) s += s_u[k];
      else
        for (int j = 0; j < m; ++j) s += W[k * m + j] * s_u[j];
    } else {
      s = s_u[D];
    }
    s += s_c[0][k] * lam0 + s_c[1][k] * lam1;
    s_gx[k] = s;
  }
  if (threadIdx.x < 2 && threadIdx.x < p) {
    const int kk = threadIdx.x;
    double h = -I.v[kk];
    for (int k = 0; k < me; ++k) h += s_c[kk][k] * xb[k];
    h += s_c[kk][me] * xb[XS - 3];
    atomicAdd(&s_sc[2], h * h);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double gx2 = 0.0, x2 = 0.0;
    for (int k = 0; k < M1; ++k) gx2 += s_gx[k] * s_gx[k];
    for (int k = 0; k < me; ++k) x2 += xb[k] * xb[k];
    x2 += xb[XS - 3] * xb[XS - 3];
    s_sc[3] = x2;
    s_gx[M1] = sqrt(gx2 + s_sc[0] + s_sc[2]);   // |F|
  }
  __syncthreads();
  if (mode == 2) {   // warm start: |F| at the default start, the stopping test's scale
    if (threadIdx.x == 0) {
      nrm[(int64_t)b * 4] = s_gx[M1];
      nrm[(int64_t)b * 4 + 2] = 1.0;
    }
    return;
  }
  if (mode == 0) {
    const int it = iters[b];
    const double nF = s_gx[M1];
    if (threadIdx.x == 0) {
      int decision = 0;   // 0: step, 1: converged, 2: cap, 3: re-pass
      if (it == 0 && nrm[(int64_t)b * 4 + 2] == 0.0) nrm[(int64_t)b * 4] = nF;
      const double F0 = nrm[(int64_t)b * 4];
      if (it > 0 && nrm[(int64_t)b * 4 + 1] <= tol * (1.0 + sqrt(s_sc[3])) && nF <= tol * fmax(1.0, F0))
        decision = 1;
      else if (it >= max_iter)
        decision = 2;
      else if (s_sc[1] > 0.0)
        decision = 3;
      if (decision == 1) { active[b] = 0; st_all[b] = NYS_OK; atomicSub(live, 1); }
      if (decision == 2) { active[b] = 0; st_all[b] = NYS_ENOCONV; atomicSub(live, 1); }
      if (decision == 3) { active[b] = 2; atomicOr(&flags[1], 1); }
      s_flag = decision;
    }
    __syncthreads();
    if (s_flag != 0) return;
  }
  // 3. H = D + B G B^T, rhs = -(D x + C^T lambda + B v)  (B = I in omega mode)
  if (om) {
    for (int e = threadIdx.x; e < M1 * M1; e += blockDim.x) {
      const int k = e / M1, l = e - k * M1;
      Hs[k * ldh + l] = Gs[k * ldg + l] + ((k == l && k < me) ? 1.0 : 0.0);
    }
    for (int k = threadIdx.x; k < me; k += blockDim.x)
      g[k] = -(xb[k] + Gs[k * ldg + D + 1] + s_c[0][k] * lam0 + s_c[1][k] * lam1);
    if (threadIdx.x == 0) g[me] = -(Gs[D * ldg + D + 1] + s_c[0][me] * lam0 + s_c[1][me] * lam1);
    __syncthreads();
  } else {
    for (int k = threadIdx.x; k < me; k += blockDim.x) {
      double s1 = 0.0, s2 = 0.0;
      for (int j = 0; j < m; ++j) {
        s1 += W[k * m + j] * Gs[j * ldg + m];
        s2 += W[k * m + j] * Gs[j * ldg + m + 1];
      }
      hb[k] = s1;
      g[k] = -(xb[k] + s2 + s_c[0][k] * lam0 + s_c[1][k] * lam1);
    }
    if (threadIdx.x == 0) g[me] = -(Gs[m * ldg + m + 1] + s_c[0][me] * lam0 + s_c[1][me] * lam1);
    __syncthreads();
    for (int k0 = 0; k0 < me; k0 += 8) {
      const int kb = min(8, me - k0);
      for (int e = threadIdx.x; e < kb * m; e += blockDim.x) {
        const int kk = e / m, l = e - kk * m;
        double s = 0.0;
        for (int j = 0; j < m; ++j) s += W[(k0 + kk) * m + j] * Gs[j * ldg + l];
        Yb[kk * m + l] = s;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < kb * me; e += blockDim.x) {
        const int kk = e / me, l = e - kk * me;
        double s = 0.0;
        for (int j = 0; j < m; ++j) s += Yb[kk * m + j] * W[l * m + j];
        Hs[(k0 + kk) * ldh + l] = s + ((k0 + kk) == l ? 1.0 : 0.0);
      }
      __syncthreads();
    }
    for (int k = threadIdx.x; k < me; k += blockDim.x) {
      Hs[k * ldh + me] = hb[k];
      Hs[me * ldh + k] = hb[k];
    }
    if (threadIdx.x == 0) Hs[me * ldh + me] = Gs[m * ldg + m];
  }
  // Householder reflectors of C^T
  for (int k = threadIdx.x; k < M1; k += blockDim.x) {
    w[k] = s_c[0][k];
    c2[k] = s_c[1][k];
  }
  __syncthreads();
  {
    const double r00 = house(w, Vh, M1, &s_beta[0], red);
    if (threadIdx.x == 0) s_R[0] = r00;
    __syncthreads();
    if (p == 2) {
      apply_house_vec(c2, M1, Vh, s_beta[0], red);
      if (threadIdx.x == 0) s_R[1] = c2[0];
      for (int k = threadIdx.x; k < M1; k += blockDim.x) Vh[M1 + k] = 0.0;
      __syncthreads();
      const double r11 = house(c2 + 1, Vh + M1 + 1, M1 - 1, &s_beta[1], red);
      if (threadIdx.x == 0) s_R[2] = r11;
      __syncthreads();
    }
  }
  for (int k = 0; k < p; ++k) {
    apply_house_sym(Hs, ldh, M1, Vh + k * M1, s_beta[k], w, red);
    apply_house_vec(g, M1, Vh + k * M1, s_beta[k], red);
  }
  // y1 = R^{-T} (v - C x)
  if (threadIdx.x == 0) {
    double h0 = I.v[0], h1 = (p == 2) ? I.v[1] : 0.0;
    for (int k = 0; k < me; ++k) { h0 -= s_c[0][k] * xb[k]; h1 -= s_c[1][k] * xb[k]; }
    h0 -= s_c[0][me] * xb[XS - 3];
    h1 -= s_c[1][me] * xb[XS - 3];
    y[0] = h0 / s_R[0];
    if (p == 2) y[1] = (h1 - s_R[1] * y[0]) / s_R[2];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < N2; i += blockDim.x) {
    double sv = g[p + i];
    for (int k = 0; k < p; ++k) sv -= Hs[(p + i) * ldh + k] * y[k];
    y[p + i] = sv;
  }
  __syncthreads();
  // keep the first p rows of H' for lambda before the factorisation
  for (int e = threadIdx.x; e < p * M1; e += blockDim.x) Yb[e] = Hs[(e / M1) * ldh + (e % M1)];
  double* A22 = Hs + p * ldh + p;
  const bool ok = block_cholesky(A22, ldh, N2, &s_flag);
  if (!ok) {
    if (threadIdx.x == 0) {
      if (mode == 0) { active[b] = 2; atomicOr(&flags[1], 1); }
      else { active[b] = 0; st_all[b] = NYS_ENOTSPD; atomicSub(live, 1); }
    }
    return;
  }
  cta_chol_solve(A22, ldh, N2, y + p);
  const double q0 = cta_dot(Yb, y, M1, red);
  const double q1 = (p == 2) ? cta_dot(Yb + M1, y, M1, red) : 0.0;
  double dl0 = 0.0, dl1 = 0.0;
  if (p == 2) {
    dl1 = (g[1] - q1) / s_R[2];
    dl0 = (g[0] - q0 - s_R[1] * dl1) / s_R[0];
  } else {
    dl0 = (g[0] - q0) / s_R[0];
  }
  for (int k = p - 1; k >= 0; --k) apply_house_vec(y, M1, Vh + k * M1, s_beta[k], red);
  // 4. update x, lambda; dz = B^T dx, z = B^T x
  for (int k = threadIdx.x; k < M1; k += blockDim.x) {
    const int slot = (k < me) ? k : XS - 3;
    xb[slot] += y[k];
  }
  if (threadIdx.x == 0) {
    xb[XS - 2] += dl0;
    if (p == 2) xb[XS - 1] += dl1;
    double d2 = 0.0;
    for (int k = 0; k < M1; ++k) d2 += y[k] * y[k];
    nrm[(int64_t)b * 4 + 1] = sqrt(d2);
    iters[b] += 1;
    active[b] = 1;
    atomicOr(&flags[0], 1);
  }
  __syncthreads();
  double* zb = zs + (int64_t)b * ZS;
  double* dzb = dzs + (int64_t)b * ZS;
  for (int j = threadIdx.x; j <= m; j += blockDim.x) {
    double s = 0.0, ds = 0.0;
    if (j < m) {
      for (int k = 0; k < me; ++k) { s += W[k * m + j] * xb[k]; ds += W[k * m + j] * y[k]; }
    } else {
      s = xb[XS - 3];
      ds = y[me];
    }
    zb[j] = s;
    if (!om) dzb[j] = ds;
  }
  // omega mode: the row pass reads the step in omega coordinates, b last
  if (om)
    for (int k = threadIdx.x; k < M1; k += blockDim.x) dzb[k] = y[k];
}

cudaError_t launch_newton_step(const Inst* insts, const Lset* lsets, const double* W,
                               const double* part, const int64_t* slot_off, const int32_t* lm,
                               double* xs, double* zs, double* dzs, double* cws, int XS, int ZS,
                               int M1S, int32_t* st, int32_t* active, int32_t* iters, double* nrm,
                               int max_iter, double tol, int32_t* flags, int mode, int batch,
                               int m_max, cudaStream_t s, int32_t* live) {
  const size_t sm = solve_smem_bytes(false, m_max);
  cudaError_t e = cudaFuncSetAttribute(k_newton_step, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm);
  if (e != cudaSuccess) return e;
  k_newton_step<<<batch, kSolveThreads, sm, s>>>(insts, lsets, W, part, slot_off, lm, xs, zs, dzs,
                                                  cws, XS, ZS, M1S, st, active, iters, nrm,
                                                  max_iter, tol, flags, mode, live);
  return cudaGetLastError();
}

size_t refine_smem_bytes(int k_max) {
  const int K = k_max < kRefLagMax ? k_max : kRefLagMax;
  const size_t table = sizeof(float) * 2 * (size_t)(2 * (K + kRefPad) + 1);
  const size_t red = sizeof(float) * (size_t)kRefThreads * 2 + 64;
  return table > red ? table : red;
}

// ---- launchers --------------------------------------------------------------

cudaError_t launch_solve(bool fp32, const Inst* insts, const Lset* lsets, const double* W,
                         const float* W32, const double* part, const int64_t* slot_off, const int32_t* lm,
                         void* fac, int64_t facs, double* xs, double* zs, double* cws, int XS,
                         int ZS, int M1S, const int32_t* st_init, int32_t* st, double gamma_scale,
                         int batch, int m_max, cudaStream_t s, const int32_t* asm_err,
                         BigSet big, const double* crow, bool fac64) {
  // the factor's type: FP32 for NYS_MIXED, FP64 otherwise (a MIXED context with
  // an FP64 factor passes fp32 with fac64; its asm_err marks it as mixed)
  if (fac64) fp32 = false;
  const size_t sm = solve_smem_bytes(fp32, m_max < kMMax ? m_max : kMMax);
  cudaError_t e;
  if (fp32) {
    e = cudaFuncSetAttribute(k_solve<float, kMMax>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sm);
    if (e != cudaSuccess) return e;
    k_solve<float, kMMax><<<batch, kSolveThreads, sm, s>>>(insts, lsets, W, W32, part, slot_off, lm,
                                                            (float*)fac, facs, xs, zs, cws, XS, ZS,
                                                            M1S, st_init, st, gamma_scale, asm_err,
                                                            BigSet(), crow);
  } else {
    e = cudaFuncSetAttribute(k_solve<double, kMMax>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sm);
    if (e != cudaSuccess) return e;
    k_solve<double, kMMax><<<batch, kSolveThreads, sm, s>>>(insts, lsets, W, W, part, slot_off, lm,
                                                             (double*)fac, facs, xs, zs, cws, XS,
                                                             ZS, M1S, st_init, st, gamma_scale,
                                                             asm_err, BigSet(), crow);
    if (big.n > 0 && (e = cudaGetLastError()) == cudaSuccess)
      k_solve<double, kMLarge><<<big.n, kSolveThreadsBig, 0, s>>>(
          insts, lsets, W, W, part, slot_off, lm, (double*)fac, facs, xs, zs, cws, XS, ZS, M1S,
          st_init, st, gamma_scale, asm_err, big, crow);
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_refine_band(const Inst* insts, const Lset* lsets, const float* lag,
                               const Work* work, int nwork, int* counter, const int32_t* lm,
                               const double* zs, int ZS, double* part, const int64_t* slot_off,
                               int32_t* st, const int32_t* skip_in, int num_sms, cudaStream_t s);

cudaError_t launch_refine(const Inst* insts, const Lset* lsets, const double* W, const float* lag,
                          const Work* work, int nwork, int* counter, const int32_t* lm,
                          const double* tab, double* part, const int64_t* slot_off,
                          const void* fac, int64_t facs, double* xs, double* zs, const double* cws,
                          int XS, int ZS, int M1S, int32_t* st, double gamma_scale, int batch,
                          int m_max, int k_max, int num_sms, cudaStream_t s, int nrband,
                          bool fac64, double* rcorr, int pass, bool last, const int32_t* skip_in,
                          int32_t* skip_out) {
  // the first nrband items: k_refine_band (queue counter[1]); the rest k_refine_rows
  cudaError_t e = cudaMemsetAsync(counter, 0, (nrband > 0 ? 2 : 1) * sizeof(int), s);
  if (e != cudaSuccess) return e;
  if (nrband > 0) {
    e = launch_refine_band(insts, lsets, lag, work, nrband, counter + 1, lm, zs, ZS, part, slot_off,
                           st, skip_in, num_sms, s);
    if (e != cudaSuccess) return e;
    work += nrband;
    nwork -= nrband;
  }
  const int k_cap = k_max < kRefLagMax ? k_max : kRefLagMax;
  const size_t sm = refine_smem_bytes(k_cap);
  e = cudaFuncSetAttribute(k_refine_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  // as many co-resident CTAs as registers and shared memory allow
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_refine_rows, kRefThreads, sm);
  const int grid = min(nwork, num_sms * max(1, per_sm));
  if (grid > 0) {
    k_refine_rows<<<grid, kRefThreads, sm, s>>>(insts, lsets, lag, work, nwork, counter, lm, tab, zs,
                                                 ZS, part, slot_off, st, skip_in, k_cap);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // x is staged in kM1Max + 3 doubles of shared memory (mixed contexts: m_max <= kMMax)
  if (XS > kM1Max + 3) return cudaErrorInvalidValue;
  // shared memory for the factor L (N2 = m_eff + 1 - p <= m_max)
  const size_t lsm = (size_t)m_max * m_max * (fac64 ? sizeof(double) : sizeof(float));
  if (fac64) {
    e = cudaFuncSetAttribute(k_refine_update<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)lsm);
    if (e != cudaSuccess) return e;
    k_refine_update<double><<<batch, kSolveThreads, lsm, s>>>(insts, lsets, W, part, slot_off,
                                                               (const double*)fac, facs, xs, zs,
                                                               cws, XS, ZS, M1S, st, gamma_scale,
                                                               rcorr, pass, last ? 1 : 0, skip_in,
                                                              skip_out);
  } else {
    e = cudaFuncSetAttribute(k_refine_update<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)lsm);
    if (e != cudaSuccess) return e;
    k_refine_update<float><<<batch, kSolveThreads, lsm, s>>>(insts, lsets, W, part, slot_off,
                                                              (const float*)fac, facs, xs, zs, cws,
                                                              XS, ZS, M1S, st, gamma_scale,
                                                              rcorr, pass, last ? 1 : 0, skip_in,
                                                              skip_out);
  }
  return cudaGetLastError();
}

}  // namespace nys
