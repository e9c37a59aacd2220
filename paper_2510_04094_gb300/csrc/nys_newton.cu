// Newton's method for nonlinear ODEs (Lemma 2, Section 3.2; Eq. 2.2; Eq. 3.2.1).
//
// Family: y^(p) = f(t, y, u), u = y^(p-1) = omega^T phi^(p-1)(t_i) (plus b for p = 1),
//   f = P(y) - delta u + beta u^2 / y [p = 2 for delta, beta] + g cos(omega t),
// P(y) = c0 + c1 y + c2 y^2 + c3 y^3 (beta: Problem 15 of Appendix A.6).
// Lagrangian (Appendix A.5):
//   L = 1/2 |omega|^2 + gamma/2 sum e_i^2 + gamma/2 sum xi_i^2 + sum_k lambda_k h_k,
//   e_i = omega^T q_i - P(y_i) - rho_i,   q_i = phi^(p)(t_i) + delta phi^(p-1)(t_i),
//   xi_i = y_i - omega^T phi(t_i) - b,    rho_i = g cos(omega t_i).
// The Jacobian of grad L has a diagonal y-block d_i = gamma (P'^2 - e_i P'' + 1)
// (Gauss-Newton: without the e_i P'' term), so each y_i is eliminated exactly,
// row by row: with qt = [q; 0], st = [phi; 1] (in kernel coordinates, q = W kq),
//   S   = D + sum_i [qt st] M_i [qt st]^T,   M_i = gamma I - (gamma^2/d_i) [P'; 1][P'; 1]^T
//   rhs = -grad_x L - sum_i (Fy_i / d_i) gamma (P' qt + st),   Fy_i = dL/dy_i
//   [S C^T; C 0] [dx; dlambda] = [rhs; -h],   dy_i = -(Fy_i - gamma (P' qt + st)^T dx) / d_i.
// These are the iterates of the dense (m+n+p) Newton system, at O(n m^2) per step.
// With beta != 0, f is nonlinear in u: q_i = phi'' + (delta - f_u) phi' follows the
// iterate (f_u = -delta + 2 beta u / y), and the Hessian gains - e f_uu pt pt^T and
// - e f_yu pt with pt = [phi'; 0]: each row adds the Gram of [qt st pt] with a
// symmetric 3 x 3 weight (Gauss-Newton drops the e-terms), two more shared tiles.
// Omega mode (landmark kernel with lambda_min < 1e-7 lambda_max): the rows are
// projected through W (qt, st in omega coordinates) before the Gram, since the
// kernel-coordinate Gram W G W^T loses the digits that cond(W)^2 costs.
//
// This file: initialisation and the fused FP64 row pass.  The per-instance
// step (stopping test, Gauss-Newton fallback, null-space Cholesky solve) is in
// nys_solve.cu (k_newton_step).
#include "nys_internal.cuh"

namespace nys {

constexpr int kNtThreads = 256;
constexpr int kNtRows = 32;

// x0: omega = 0, b = v_1, lambda = 0; y_i = v_1.  live counts the running
// instances (the caller zeroes it first); every later Newton kernel returns at
// once when it is 0.
__global__ void k_newton_init(const Inst* __restrict__ insts, double* __restrict__ xs,
                              double* __restrict__ zs, double* __restrict__ dzs,
                              double* __restrict__ yaux, double* __restrict__ nrm,
                              int32_t* __restrict__ iters, int32_t* __restrict__ active,
                              int32_t* __restrict__ st, const int32_t* __restrict__ st_init,
                              int XS, int ZS, int32_t* __restrict__ live) {
  const int b = blockIdx.x;
  const Inst I = insts[b];
  for (int k = threadIdx.x; k < XS; k += blockDim.x) xs[(int64_t)b * XS + k] = (k == XS - 3) ? I.v[0] : 0.0;
  for (int j = threadIdx.x; j < ZS; j += blockDim.x) {
    zs[(int64_t)b * ZS + j] = (j == I.m) ? I.v[0] : 0.0;
    dzs[(int64_t)b * ZS + j] = 0.0;
  }
  for (int r = threadIdx.x; r < I.n - 1; r += blockDim.x) yaux[I.y_off + r] = I.v[0];
  if (threadIdx.x < 4) nrm[(int64_t)b * 4 + threadIdx.x] = 0.0;
  if (threadIdx.x == 0) {
    iters[b] = 0;
    st[b] = st_init[b];
    active[b] = (st_init[b] == NYS_OK) ? 1 : 0;
    if (st_init[b] == NYS_OK) atomicAdd(live, 1);
  }
}

// Warm start from the caller's buffer [x (x_out's layout) | y (y_aux_out's
// layout)]: x = (omega, b, lambda), its kernel coordinates z = (W^T omega, b),
// and the auxiliary unknowns y_i of Lemma 2 (at a solution they differ from the
// fit y^(t_i) by xi_i, which need not be small: e_i and xi_i carry the same
// weight gamma).
__global__ void k_newton_warm(const Inst* __restrict__ insts, const Lset* __restrict__ lsets,
                              const double* __restrict__ W_all, const double* __restrict__ warm,
                              double* __restrict__ xs, double* __restrict__ zs,
                              double* __restrict__ yaux, const int32_t* __restrict__ st_init,
                              int XS, int ZS, int batch) {
  const int b = blockIdx.x;
  if (st_init[b] != NYS_OK) return;
  const Inst I = insts[b];
  const Lset L = lsets[I.lset];
  const int m = I.m, me = L.m_eff;
  const double* W = W_all + L.w_off;
  __shared__ double s_x[kMMax + 3];
  for (int k = threadIdx.x; k < XS; k += blockDim.x) {
    const double v = warm[(int64_t)b * XS + k];
    s_x[k] = (k < me || k >= XS - 3) ? v : 0.0;   // omega beyond m_eff is zero
    xs[(int64_t)b * XS + k] = s_x[k];
  }
  __syncthreads();
  for (int j = threadIdx.x; j <= m; j += blockDim.x) {
    double z = s_x[XS - 3];
    if (j < m) {
      z = 0.0;
      for (int k = 0; k < me; ++k) z += W[k * m + j] * s_x[k];
    }
    zs[(int64_t)b * ZS + j] = z;
  }
  const double* wy = warm + (int64_t)batch * XS + I.y_off;
  for (int r = threadIdx.x; r < I.n - 1; r += blockDim.x) yaux[I.y_off + r] = wy[r];
}

// Partial-slot layout of one work item (doubles):
//   [0, E1)            packed upper reduced Gram over (m+1) kernel coordinates
//   [E1, E1+M1)        v = sum (c_q qt + c_s st)      (right-hand side part)
//   [E1+M1, E1+2M1)    u = sum (gamma e qt - gamma xi st)   (grad_x L part)
//   E1+2M1             sum Fy_i^2
//   E1+2M1+1           number of rows with d_i <= 1e-12 gamma (full Newton only)
//
// mode 0: every running instance, full Newton d_i, and (apply_dy) the y-update of
//         the previous step first;  mode 1: instances flagged for a Gauss-Newton
//         re-pass (active == 2), Gauss-Newton d_i, no y-update.
template <int KMAX>
__global__ void __launch_bounds__(kNtThreads)
k_newton_pass(const Inst* __restrict__ insts, const Lset* __restrict__ lsets,
              const double* __restrict__ W_all, const Work* __restrict__ work, int nwork,
              int* __restrict__ counter, const int32_t* __restrict__ lm_idx,
              const double* __restrict__ xs, int XS,
              const double* __restrict__ zs, const double* __restrict__ dzs, int ZS,
              double* __restrict__ yaux, double* __restrict__ rowstate,
              double* __restrict__ part, const int64_t* __restrict__ slot_off,
              const int32_t* __restrict__ active, int mode, int apply_dy, int tiles,
              const int32_t* __restrict__ live) {
  if (*live == 0) return;   // every instance has stopped (the same value for all threads)
  extern __shared__ double smn[];
  __shared__ int s_item;
  __shared__ int s_idx[kMMax];
  __shared__ unsigned char s_pair[2 * kM1Max * (kM1Max + 1) / 2];
  __shared__ double s_z[kM1Max], s_dz[kM1Max];
  __shared__ double s_c[kNtRows][4];   // c_q, c_s, gamma e, -gamma xi
  __shared__ double s_m[kNtRows][8];   // beta rows: M_qq M_qs M_qp M_ss M_sp M_pp, c_p, f_u + delta
  __shared__ double s_red[kNtThreads / 32][2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int cached_m1 = -1;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int w = s_item;
    if (w >= nwork) break;
    const Work wk = work[w];
    const int act = active[wk.inst];
    if ((mode == 0 && act == 0) || (mode == 1 && act != 2)) {
      __syncthreads();
      continue;
    }
    const Inst I = insts[wk.inst];
    const Lset L = lsets[I.lset];
    const int om = L.omode;
    const double* W = W_all + L.w_off;
    // D feature columns: m kernel coordinates, or m_eff omega coordinates
    const int m = I.m, D = om ? L.m_eff : m, M1 = D + 1, ld = m + 2;
    const int E1 = M1 * (M1 + 1) / 2;
    const double gam = I.gamma, sig = I.sigma, is = 1.0 / sig, is2 = is * is;
    const double c0 = I.c[0], c1 = I.c[1], c2 = I.c[2], c3 = I.c[3];
    const double delta = (I.p == 2) ? I.c[4] : 0.0, gf = I.c[5], wf = I.c[6];
    const double beta = (I.p == 2) ? I.c[7] : 0.0;
    const bool nlu = (beta != 0.0) && (tiles >= 6);   // warp-uniform
    for (int j = tid; j < m; j += kNtThreads) s_idx[j] = lm_idx[I.lm_off + j];
    for (int j = tid; j <= D; j += kNtThreads) {
      // current iterate and last step in the frame of the Gram (dzs holds the
      // step in that frame; omega mode reads (omega, b) from x)
      s_z[j] = om ? xs[(int64_t)wk.inst * XS + (j < D ? j : XS - 3)] : zs[(int64_t)wk.inst * ZS + j];
      s_dz[j] = dzs[(int64_t)wk.inst * ZS + j];
    }
    if (M1 != cached_m1) {
      for (int e = tid; e < E1; e += kNtThreads) {
        int j = 0, rem = e;
        while (rem >= M1 - j) { rem -= M1 - j; ++j; }
        s_pair[2 * e] = (unsigned char)j;
        s_pair[2 * e + 1] = (unsigned char)(j + rem);
      }
      cached_m1 = M1;
    }
    double acc[KMAX];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) acc[k] = 0.0;
    double vacc = 0.0, uacc = 0.0, fy2 = 0.0;
    int nsmall = 0;
    double* tk0 = smn;                   // kNtRows x ld each
    double* tk1 = tk0 + kNtRows * ld;
    double* tk2 = tk1 + kNtRows * ld;
    double* tk3 = tk2 + kNtRows * ld;
    double* tk4 = tk3 + kNtRows * ld;    // beta rows only (tiles == 6)
    double* tk5 = tk4 + kNtRows * ld;
    // qt, st (pt): the rows in the frame of the Gram; ta = M11 qt + M12 st (+ M13 pt),
    // tb = M12 qt + M22 st (+ M23 pt), tc = M13 qt + M23 st + M33 pt
    double* tq = om ? tk2 : tk0;
    double* ts = om ? tk3 : tk1;
    double* ta = om ? tk0 : tk2;
    double* tb = om ? tk1 : tk3;
    double* tp = om ? tk5 : tk4;
    double* tc = om ? tk4 : tk5;
    __syncthreads();
    for (int base = wk.r0; base < wk.r1; base += kNtRows) {
      const int rows = min(kNtRows, wk.r1 - base);
      // features of the tile in kernel coordinates (FP64), into tk0 / tk1
      for (int e = tid; e < kNtRows * (m + 1); e += kNtThreads) {
        const int r = e / (m + 1), j = e - r * (m + 1);
        double q = 0.0, s = 0.0, pv = 0.0;
        if (r < rows) {
          if (j < m) {
            const double x = (double)(base + r - s_idx[j]) * I.hs;
            const double u = x * x;
            const double ex = exp(-u);
            const double k1 = -2.0 * x * is * ex;
            if (I.p == 2) q = (4.0 * u - 2.0) * is2 * ex + delta * k1;
            else q = k1;
            s = ex;
            pv = k1;
          } else {
            q = 0.0;
            s = 1.0;
          }
        }
        tk0[r * ld + j] = q;
        tk1[r * ld + j] = s;
        if (nlu) tk4[r * ld + j] = pv;
      }
      __syncthreads();
      if (om) {  // omega coordinates: [W kq; 0], [W k; 1]
        for (int e = tid; e < kNtRows * M1; e += kNtThreads) {
          const int r = e / M1, k = e - r * M1;
          double q = 0.0, s = 1.0;
          if (k < D) {
            s = 0.0;
            for (int j = 0; j < m; ++j) {
              q = fma(W[k * m + j], tk0[r * ld + j], q);
              s = fma(W[k * m + j], tk1[r * ld + j], s);
            }
          }
          tq[r * ld + k] = q;
          ts[r * ld + k] = s;
          if (nlu) {
            double pv = 0.0;
            if (k < D)
              for (int j = 0; j < m; ++j) pv = fma(W[k * m + j], tk4[r * ld + j], pv);
            tp[r * ld + k] = pv;
          }
        }
        __syncthreads();
      }
      // per-row scalars: one warp per row, lanes over landmarks
      for (int r = warp; r < rows; r += kNtThreads / 32) {
        double Q = 0.0, Ph = 0.0, Qd = 0.0, Sd = 0.0, U = 0.0, Pd = 0.0;
        for (int j = lane; j <= D; j += 32) {
          const double qv = tq[r * ld + j], sv = ts[r * ld + j];
          Q = fma(qv, s_z[j], Q);
          Ph = fma(sv, s_z[j], Ph);
          Qd = fma(qv, s_dz[j], Qd);
          Sd = fma(sv, s_dz[j], Sd);
          if (nlu) {
            const double pv = tp[r * ld + j];
            U = fma(pv, s_z[j], U);
            Pd = fma(pv, s_dz[j], Pd);
          }
        }
        for (int o = 16; o > 0; o >>= 1) {
          Q += __shfl_xor_sync(0xffffffffu, Q, o);
          Ph += __shfl_xor_sync(0xffffffffu, Ph, o);
          Qd += __shfl_xor_sync(0xffffffffu, Qd, o);
          Sd += __shfl_xor_sync(0xffffffffu, Sd, o);
          if (nlu) {
            U += __shfl_xor_sync(0xffffffffu, U, o);
            Pd += __shfl_xor_sync(0xffffffffu, Pd, o);
          }
        }
        if (lane == 0) {
          const int i = base + r;
          const int64_t yo = I.y_off + (i - 1);
          double y = yaux[yo];
          double* rs = rowstate + kNtRowState * yo;
          if (mode == 0 && apply_dy) {   // y-update of the previous step
            // (its q was qt - h_u pt with the previous h_u; e f_yu weights pt)
            const double Qp = nlu ? Qd - rs[3] * Pd : Qd;
            const double wd = rs[2] * Qp + Sd + (nlu ? rs[4] * Pd : 0.0);
            y += -(rs[0] - gam * wd) / rs[1];
            yaux[yo] = y;
          }
          const double P = c0 + y * (c1 + y * (c2 + y * c3));
          const double rho = gf * cos(wf * (I.t0 + (double)i * I.h));
          double fy = c1 + y * (2.0 * c2 + 3.0 * c3 * y);   // f_y
          double fyy = 2.0 * c2 + 6.0 * c3 * y;               // f_yy
          double e = Q - P - rho;                             // Q = (phi'' + delta phi')^T x
          double hu = 0.0, cyu = 0.0, cu = 0.0;
          if (nlu) {   // beta u^2 / y
            const double iy = 1.0 / y, bu = beta * U * iy;
            e -= bu * U;
            fy -= bu * U * iy;
            fyy += 2.0 * bu * U * iy * iy;
            hu = 2.0 * bu;                                    // f_u + delta
            cyu = e * (-2.0 * bu * iy);                       // e f_yu
            cu = e * (2.0 * beta * iy);                       // e f_uu
          }
          const double xi = y - Ph;
          const double Fy = -gam * e * fy + gam * xi;
          const double dfull = gam * (fy * fy - e * fyy + 1.0);
          if (mode == 0 && !(dfull > 1e-12 * gam)) ++nsmall;
          const double d = (mode == 0) ? dfull : gam * (fy * fy + 1.0);
          if (mode != 0) { cyu = 0.0; cu = 0.0; }             // Gauss-Newton
          rs[0] = Fy;
          rs[1] = d;
          rs[2] = fy;
          rs[3] = hu;
          rs[4] = cyu;
          fy2 = fma(Fy, Fy, fy2);
          const double g2d = gam * gam / d;
          // M = diag(gamma, gamma, -gamma e f_uu) - (gamma^2/d) w w^T, w = [f_y 1 e f_yu]
          s_c[r][0] = gam * e + gam * fy * Fy / d;   // c_q
          s_c[r][1] = -gam * xi + gam * Fy / d;      // c_s
          s_c[r][2] = gam * e;
          s_c[r][3] = -gam * xi;
          const double M11 = gam - g2d * fy * fy, M12 = -g2d * fy, M22 = gam - g2d;
          if (nlu) {
            s_m[r][0] = M11;
            s_m[r][1] = M12;
            s_m[r][2] = -g2d * fy * cyu;             // M13
            s_m[r][3] = M22;
            s_m[r][4] = -g2d * cyu;                  // M23
            s_m[r][5] = -gam * cu - g2d * cyu * cyu; // M33
            s_m[r][6] = gam * cyu * Fy / d;          // c_p
            s_m[r][7] = hu;
          } else {
            // stash M in the first two slots of the a/b rows (overwritten below)
            ta[r * ld + M1] = M11;
            tb[r * ld + M1] = M22;
            ts[r * ld + M1] = M12;
          }
        }
      }
      __syncthreads();
      if (nlu) {
        // the row's d e / d x: qt - h_u pt, then the three combinations
        for (int e = tid; e < rows * M1; e += kNtThreads) {
          const int r = e / M1, j = e - r * M1;
          const double pv = tp[r * ld + j], sv = ts[r * ld + j];
          const double qv = tq[r * ld + j] - s_m[r][7] * pv;
          tq[r * ld + j] = qv;
          ta[r * ld + j] = s_m[r][0] * qv + s_m[r][1] * sv + s_m[r][2] * pv;
          tb[r * ld + j] = s_m[r][1] * qv + s_m[r][3] * sv + s_m[r][4] * pv;
          tc[r * ld + j] = s_m[r][2] * qv + s_m[r][4] * sv + s_m[r][5] * pv;
        }
      } else {
        for (int e = tid; e < rows * M1; e += kNtThreads) {
          const int r = e / M1, j = e - r * M1;
          const double M11 = ta[r * ld + M1], M22 = tb[r * ld + M1], M12 = ts[r * ld + M1];
          const double q = tq[r * ld + j], s = ts[r * ld + j];
          ta[r * ld + j] = M11 * q + M12 * s;
          tb[r * ld + j] = M12 * q + M22 * s;
        }
      }
      __syncthreads();
      // reduced Gram: G_jl += a_j qt_l + b_j st_l
#pragma unroll
      for (int k = 0; k < KMAX; ++k) {
        const int e = tid + k * kNtThreads;
        if (e < E1) {
          const int j = s_pair[2 * e], l = s_pair[2 * e + 1];
          double a = acc[k];
          if (nlu) {
            for (int r = 0; r < rows; ++r) {
              a = fma(ta[r * ld + j], tq[r * ld + l], a);
              a = fma(tb[r * ld + j], ts[r * ld + l], a);
              a = fma(tc[r * ld + j], tp[r * ld + l], a);
            }
          } else {
            for (int r = 0; r < rows; ++r) {
              a = fma(ta[r * ld + j], tq[r * ld + l], a);
              a = fma(tb[r * ld + j], ts[r * ld + l], a);
            }
          }
          acc[k] = a;
        }
      }
      if (tid < M1) {
        for (int r = 0; r < rows; ++r) {
          vacc = fma(s_c[r][0], tq[r * ld + tid], fma(s_c[r][1], ts[r * ld + tid], vacc));
          uacc = fma(s_c[r][2], tq[r * ld + tid], fma(s_c[r][3], ts[r * ld + tid], uacc));
          if (nlu) vacc = fma(s_m[r][6], tp[r * ld + tid], vacc);
        }
      }
      __syncthreads();
    }
    // write the partial
    double* out = part + slot_off[wk.slot];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
      const int e = tid + k * kNtThreads;
      if (e < E1) out[e] = acc[k];
    }
    if (tid < M1) {
      out[E1 + tid] = vacc;
      out[E1 + M1 + tid] = uacc;
    }
    // block sums of Fy^2 and of the small-pivot count (only lane 0 of each warp holds values)
    for (int o = 16; o > 0; o >>= 1) {
      fy2 += __shfl_xor_sync(0xffffffffu, fy2, o);
      nsmall += __shfl_xor_sync(0xffffffffu, nsmall, o);
    }
    if (lane == 0) { s_red[warp][0] = fy2; s_red[warp][1] = (double)nsmall; }
    __syncthreads();
    if (tid == 0) {
      double f = 0.0, c = 0.0;
      for (int q = 0; q < kNtThreads / 32; ++q) { f += s_red[q][0]; c += s_red[q][1]; }
      out[E1 + 2 * M1] = f;
      out[E1 + 2 * M1 + 1] = c;
    }
    __syncthreads();
  }
}

// tiles: 4, or 6 when some instance has a beta u^2 / y term
size_t newton_pass_smem(int m_max, int tiles) {
  return sizeof(double) * (size_t)tiles * kNtRows * (m_max + 2);
}

template <int K>
static cudaError_t launch_pass_k(const Inst* insts, const Lset* lsets, const double* W,
                                 const Work* work, int nwork, int* counter, const int32_t* lm,
                                 const double* xs, int XS, const double* zs, const double* dzs, int ZS,
                                 double* yaux, double* rowstate, double* part,
                                 const int64_t* slot_off, const int32_t* active, int mode,
                                 int apply_dy, int m_max, int tiles, int num_sms, cudaStream_t s,
                                 const int32_t* live) {
  const size_t sm = newton_pass_smem(m_max, tiles);
  cudaError_t e = cudaFuncSetAttribute(k_newton_pass<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm);
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_newton_pass<K>, kNtThreads, sm);
  const int grid = min(nwork, num_sms * max(1, per_sm));
  k_newton_pass<K><<<grid, kNtThreads, sm, s>>>(insts, lsets, W, work, nwork, counter, lm, xs, XS,
                                                  zs, dzs, ZS, yaux,
                                                  rowstate, part, slot_off, active, mode, apply_dy,
                                                  tiles, live);
  return cudaGetLastError();
}

cudaError_t launch_newton_pass(const Inst* insts, const Lset* lsets, const double* W,
                               const Work* work, int nwork, int* counter, const int32_t* lm,
                               const double* xs, int XS, const double* zs, const double* dzs, int ZS,
                               double* yaux, double* rowstate, double* part,
                               const int64_t* slot_off, const int32_t* active, int mode,
                               int apply_dy, int m_max, int tiles, int num_sms, cudaStream_t s,
                               const int32_t* live) {
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  const int M1 = m_max + 1, E1 = M1 * (M1 + 1) / 2;
  const int kneed = (E1 + kNtThreads - 1) / kNtThreads;
#define NT_ARGS insts, lsets, W, work, nwork, counter, lm, xs, XS, zs, dzs, ZS, yaux, rowstate, part, slot_off, active, \
                mode, apply_dy, m_max, tiles, num_sms, s, live
  if (kneed <= 4) return launch_pass_k<4>(NT_ARGS);
  if (kneed <= 8) return launch_pass_k<8>(NT_ARGS);
  if (kneed <= 14) return launch_pass_k<14>(NT_ARGS);
  if (kneed <= 20) return launch_pass_k<20>(NT_ARGS);
  return launch_pass_k<26>(NT_ARGS);
#undef NT_ARGS
}

// warm == nullptr: the default start (and live counted from 0);
// warm != nullptr: only x, z, y replaced by the warm start (nrm, iters kept)
cudaError_t launch_newton_init(const Inst* insts, const Lset* lsets, const double* W,
                               const int32_t* lm, const double* warm, double* xs, double* zs,
                               double* dzs, double* yaux, double* nrm, int32_t* iters,
                               int32_t* active, int32_t* st, const int32_t* st_init, int XS, int ZS,
                               int batch, int32_t* live, cudaStream_t s) {
  if (warm != nullptr) {
    k_newton_warm<<<batch, 256, 0, s>>>(insts, lsets, W, warm, xs, zs, yaux, st_init, XS, ZS, batch);
    return cudaGetLastError();
  }
  cudaError_t e = cudaMemsetAsync(live, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  k_newton_init<<<batch, 256, 0, s>>>(insts, xs, zs, dzs, yaux, nrm, iters, active, st, st_init, XS,
                                      ZS, live);
  return cudaGetLastError();
}

}  // namespace nys
