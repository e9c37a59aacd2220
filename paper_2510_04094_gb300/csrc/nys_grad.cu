// Adjoint gradient of a loss on the fitted solution with respect to the
// problem parameters theta = (a_1, a_2, c, omega, y0, y0', sigma) of
//     y^(p) + a_1 y^(p-1) [+ a_2 y] = c sin(omega t + phi0),  y(t_1) = y0 [, y'(t_1) = y0'],
// for the Nystrom LS-SVM solution of Lemma 1 (Section 3.1).  Parameter
// estimation is the use the paper cites for LS-SVM ODE solvers (Introduction);
// it prints no gradient, so this is the implicit-function derivative of
// Lemma 1's system written out:
//
//   F(x, lambda; theta) = [D x + gamma sum_i a~_i (a~_i^T x - r_i) + C^T lambda ; C x - v] = 0
//   K mu = d loss / d(x, lambda)       (K = Lemma 1's matrix, symmetric)
//   d loss / d theta = explicit part - mu^T dF/dtheta.
//
// In kernel coordinates z = (alpha, b), alpha = W^T omega, the problem is
// min 1/2 alpha^T Omega alpha + gamma/2 sum_i (kappa~_i^T z - r_i)^2 with the
// initial-condition rows E z = v; the adjoint in these coordinates is
// mu~ = (W^T mu_omega, mu_b) with the same mu_lambda.  Every parameter except
// sigma enters only through kappa~_i, r_i or v, so the row terms are O(m)
// contractions of kernel rows with alpha and mu~.  sigma also enters Omega,
// E and the model at the observation times; in kernel coordinates no
// eigenvector derivative is needed, which is exact when every eigenpair of
// Omega is kept (m_eff = m).  With truncated landmark kernels the sigma entry
// is NaN.
//
// Kernels: k_grad_adjoint (per instance: right-hand side at the observation
// times, adjoint solve with the stored FP64 factor, instance-level sigma
// terms), k_grad_rows (persistent row pass over the balanced work list,
// five row sums per work item), k_grad_final (slot sums in fixed order).
#include "nys_cta.cuh"

namespace nys {

constexpr int kGradThreads = 256;
constexpr int kGradRowThreads = 256;
constexpr int kGradSums = 5;   // S_a, S_b, S_c, S_omega, S_sigma

// RBF derivatives at x = (t - s) / sigma, e = exp(-x^2):
//   k = e, k' = -2x/sigma e, k'' = (4x^2 - 2)/sigma^2 e,
//   dk/dsigma = 2x^2/sigma e, dk'/dsigma = 4x(1 - x^2)/sigma^2 e,
//   dk''/dsigma = (8x^4 - 20x^2 + 4)/sigma^3 e.
__device__ __forceinline__ double dsig_k0(double x, double e, double is) { return 2.0 * x * x * is * e; }
__device__ __forceinline__ double dsig_k1(double x, double e, double is) {
  return 4.0 * x * (1.0 - x * x) * is * is * e;
}

// adj layout per instance (stride AS doubles): mu~ (ZS: alpha part, b at index m),
// then [valid, g_a, g_b, g_c, g_omega, g_y0, g_y0', g_sigma] (instance-level parts).
__global__ void __launch_bounds__(kGradThreads)
k_grad_adjoint(const Inst* __restrict__ insts, const Lset* __restrict__ lsets,
               const double* __restrict__ W_all, const double* __restrict__ fac_all, int64_t facs,
               const double* __restrict__ xs, const double* __restrict__ zs,
               const int32_t* __restrict__ lm_idx, int XS, int ZS, const int32_t* __restrict__ st,
               const double* __restrict__ obs_t, const int64_t* __restrict__ obs_off,
               const double* __restrict__ dl_dy, double* __restrict__ adj, int AS) {
  const int b = blockIdx.x;
  const Inst I = insts[b];
  const Lset LS = lsets[I.lset];
  double* ab = adj + (int64_t)b * AS;
  const bool valid = (st[b] == NYS_OK) && (I.kind == NYS_COEF_LIN);
  if (!valid) {
    for (int k = threadIdx.x; k < AS; k += blockDim.x) ab[k] = 0.0;
    return;
  }
  const int m = I.m, p = I.p, me = LS.m_eff, M1 = me + 1;
  const double* W = W_all + LS.w_off;
  const double is = 1.0 / I.sigma;
  __shared__ double s_s[kMMax], s_al[kMMax], s_hk[kM1Max];
  __shared__ double s_h[kM1Max], s_mx[kM1Max], s_mu[kM1Max];
  __shared__ double s_ml[2], s_cr[2], red[40];
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    s_s[j] = I.t0 + (double)lm_idx[I.lm_off + j] * I.h;
    s_al[j] = zs[(int64_t)b * ZS + j];
  }
  if (threadIdx.x < 2) s_cr[threadIdx.x] = 0.0;
  __syncthreads();
  const int64_t q0 = obs_off[b], q1 = obs_off[b + 1];
  // 1. d loss / dz: h_k[j] = sum_q u_q k(tau_q, s_j), h_k[m] = sum_q u_q
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    double s = 0.0;
    for (int64_t q = q0; q < q1; ++q) {
      const double x = (obs_t[q] - s_s[j]) * is;
      s = fma(dl_dy[q], exp(-x * x), s);
    }
    s_hk[j] = s;
  }
  // explicit sigma term: sum_q u_q alpha^T dk(tau_q)/dsigma; and sum_q u_q
  double ex = 0.0, su = 0.0;
  for (int64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < m; ++j) {
      const double x = (obs_t[q] - s_s[j]) * is;
      s = fma(s_al[j], dsig_k0(x, exp(-x * x), is), s);
    }
    ex = fma(dl_dy[q], s, ex);
    su += dl_dy[q];
  }
  {
    __shared__ double s_two[kGradThreads / 32][2];
    for (int o = 16; o > 0; o >>= 1) {
      ex += __shfl_xor_sync(0xffffffffu, ex, o);
      su += __shfl_xor_sync(0xffffffffu, su, o);
    }
    if ((threadIdx.x & 31) == 0) { s_two[threadIdx.x >> 5][0] = ex; s_two[threadIdx.x >> 5][1] = su; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0, c = 0.0;
      for (int w = 0; w < kGradThreads / 32; ++w) { a += s_two[w][0]; c += s_two[w][1]; }
      red[34] = a;
      s_hk[m] = c;
    }
    __syncthreads();
  }
  const double expl_sigma = red[34];
  __syncthreads();
  // 2. omega coordinates: h = B h_k, B = blkdiag(W, 1)
  for (int k = threadIdx.x; k < M1; k += blockDim.x) {
    double s = 0.0;
    if (k < me) {
      for (int j = 0; j < m; ++j) s = fma(W[k * m + j], s_hk[j], s);
    } else {
      s = s_hk[m];
    }
    s_h[k] = s;
  }
  __syncthreads();
  // 3. K mu = [h; 0] with the stored factor
  const FacView<double> F = fac_view(const_cast<double*>(fac_all) + (int64_t)b * facs, M1);
  kkt_apply(F, M1, p, s_h, s_cr, s_mx, s_ml, red);
  // 4. mu~ = (W^T mu_omega, mu_b)
  for (int j = threadIdx.x; j <= m; j += blockDim.x) {
    double s = 0.0;
    if (j < m) {
      for (int k = 0; k < me; ++k) s = fma(W[k * m + j], s_mx[k], s);
    } else {
      s = s_mx[me];
    }
    s_mu[j] = s;
    ab[j] = s;
  }
  __syncthreads();
  // 5. instance-level sigma terms: - mu~^T dOmega/dsigma alpha
  //    - lambda^T dE/dsigma mu~ - mu_lambda^T dE/dsigma z
  double acc = 0.0;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int j = e / m, l = e - j * m;
    const double x = (s_s[j] - s_s[l]) * is;
    acc = fma(s_mu[j] * s_al[l], dsig_k0(x, exp(-x * x), is), acc);
  }
  const double lam0 = xs[(int64_t)b * XS + XS - 2], lam1 = (p == 2) ? xs[(int64_t)b * XS + XS - 1] : 0.0;
  double e0mu = 0.0, e0al = 0.0, e1mu = 0.0, e1al = 0.0;   // dE/dsigma rows against mu~, alpha
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    const double x = (I.t0 - s_s[j]) * is;
    const double ee = exp(-x * x);
    const double d0 = dsig_k0(x, ee, is), d1 = dsig_k1(x, ee, is);
    e0mu = fma(d0, s_mu[j], e0mu);
    e0al = fma(d0, s_al[j], e0al);
    e1mu = fma(d1, s_mu[j], e1mu);
    e1al = fma(d1, s_al[j], e1al);
  }
  const double t_om = cta_sum(acc, red);
  const double t_e0mu = cta_sum(e0mu, red), t_e0al = cta_sum(e0al, red);
  const double t_e1mu = cta_sum(e1mu, red), t_e1al = cta_sum(e1al, red);
  if (threadIdx.x == 0) {
    double gs = expl_sigma - t_om - lam0 * t_e0mu - s_ml[0] * t_e0al;
    if (p == 2) gs -= lam1 * t_e1mu + s_ml[1] * t_e1al;
    if (me < m) gs = __longlong_as_double(0x7ff8000000000000LL);  // truncated: not available
    double* g = ab + ZS;
    g[0] = 1.0;                      // valid
    g[1] = 0.0; g[2] = 0.0; g[3] = 0.0; g[4] = 0.0;
    g[5] = s_ml[0];                  // d loss / d y0 = mu_lambda_1
    g[6] = (p == 2) ? s_ml[1] : 0.0; // d loss / d y0'
    g[7] = gs;
  }
}

// Row pass: for each row i (t_i, kappa~_i, r_i) of a work item
//   e_i = kappa~_i^T z - r_i,  d_i = kappa~_i^T mu~
//   S_a += (dk_a^T mu~) e_i + d_i (dk_a^T z),  dk_a = d kappa~_i / d a_1
//   S_b += same for a_2 (p = 2),  S_c += d_i sin(th_i),  S_omega += d_i c t_i cos(th_i)
//   S_sigma += (dkappa/dsigma^T mu~) e_i + d_i (dkappa/dsigma^T alpha)
// Landmarks beyond the set's lag K (kernel value < 1e-34) are skipped.
__global__ void __launch_bounds__(kGradRowThreads)
k_grad_rows(const Inst* __restrict__ insts, const Lset* __restrict__ lsets,
            const Work* __restrict__ work, int nwork, int* __restrict__ counter,
            const int32_t* __restrict__ lm_idx, const double* __restrict__ zs, int ZS,
            const double* __restrict__ adj, int AS, double* __restrict__ part,
            const int64_t* __restrict__ slot_off) {
  __shared__ int s_item;
  __shared__ int s_idx[kMMax];
  __shared__ double s_al[kMMax], s_mu[kMMax];
  __shared__ double s_red[kGradRowThreads / 32][kGradSums];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int w = s_item;
    if (w >= nwork) break;
    const Work wk = work[w];
    const Inst I = insts[wk.inst];
    const double* ab = adj + (int64_t)wk.inst * AS;
    if (ab[ZS] == 0.0) {   // invalid instance: nothing to add
      __syncthreads();
      continue;
    }
    const int m = I.m, p = I.p, K = lsets[I.lset].K;
    for (int j = tid; j < m; j += kGradRowThreads) {
      s_idx[j] = lm_idx[I.lm_off + j];
      s_al[j] = zs[(int64_t)wk.inst * ZS + j];
      s_mu[j] = ab[j];
    }
    __syncthreads();
    const double zb = zs[(int64_t)wk.inst * ZS + m], mub = ab[m];
    const double is = 1.0 / I.sigma, is2 = is * is;
    const double a1 = I.c[0], a2 = (p == 2) ? I.c[1] : 0.0, ap = (p == 2) ? a2 : a1;
    const double cc = I.c[2], om = I.c[3], ph = I.c[4];
    double S[kGradSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int i = wk.r0 + tid; i < wk.r1; i += kGradRowThreads) {
      // landmark window [jlo, jhi): |i - idx_j| <= K
      int lo = 0, hi = m;
      while (lo < hi) { const int md = (lo + hi) >> 1; if (s_idx[md] < i - K) lo = md + 1; else hi = md; }
      const int jlo = lo;
      hi = m;
      while (lo < hi) { const int md = (lo + hi) >> 1; if (s_idx[md] <= i + K) lo = md + 1; else hi = md; }
      const int jhi = lo;
      double ka = 0.0, km = 0.0;      // kappa . alpha, kappa . mu~
      double da = 0.0, dm = 0.0;      // (d kappa / d a_1) . alpha, . mu~
      double ba = 0.0, bm = 0.0;      // k . alpha, k . mu~  (d kappa / d a_2 for p = 2)
      double sa = 0.0, sm = 0.0;      // (d kappa / d sigma) . alpha, . mu~
      for (int j = jlo; j < jhi; ++j) {
        const double x = (double)(i - s_idx[j]) * I.hs;
        const double u = x * x;
        const double e = exp(-u);
        const double k0 = e;
        const double k1 = -2.0 * x * is * e;
        const double d0 = 2.0 * u * is * e;
        const double d1 = 4.0 * x * (1.0 - u) * is2 * e;
        double kap, dk_a, dsk;
        if (p == 2) {
          const double k2 = (4.0 * u - 2.0) * is2 * e;
          const double d2 = (8.0 * u * u - 20.0 * u + 4.0) * is2 * is * e;
          kap = k2 + a1 * k1 + a2 * k0;
          dk_a = k1;
          dsk = d2 + a1 * d1 + a2 * d0;
        } else {
          kap = k1 + a1 * k0;
          dk_a = k0;
          dsk = d1 + a1 * d0;
        }
        const double al = s_al[j], mu = s_mu[j];
        ka = fma(kap, al, ka);
        km = fma(kap, mu, km);
        da = fma(dk_a, al, da);
        dm = fma(dk_a, mu, dm);
        ba = fma(k0, al, ba);
        bm = fma(k0, mu, bm);
        sa = fma(dsk, al, sa);
        sm = fma(dsk, mu, sm);
      }
      const double t = I.t0 + (double)i * I.h;
      double sn, cs;
      sincos(om * t + ph, &sn, &cs);
      const double ei = ka + ap * zb - cc * sn;
      const double di = km + ap * mub;
      if (p == 2) {
        S[0] = fma(dm, ei, fma(di, da, S[0]));
        S[1] = fma(bm + mub, ei, fma(di, ba + zb, S[1]));
      } else {
        S[0] = fma(dm + mub, ei, fma(di, da + zb, S[0]));
      }
      S[2] = fma(di, sn, S[2]);
      S[3] = fma(di, cc * t * cs, S[3]);
      S[4] = fma(sm, ei, fma(di, sa, S[4]));
    }
#pragma unroll
    for (int k = 0; k < kGradSums; ++k)
      for (int o = 16; o > 0; o >>= 1) S[k] += __shfl_xor_sync(0xffffffffu, S[k], o);
    if (lane == 0)
      for (int k = 0; k < kGradSums; ++k) s_red[warp][k] = S[k];
    __syncthreads();
    if (tid < kGradSums) {
      double s = 0.0;
      for (int q = 0; q < kGradRowThreads / 32; ++q) s += s_red[q][tid];
      part[slot_off[wk.slot] + tid] = s;
    }
    __syncthreads();
  }
}

// grad = [-g S_a, -g S_b, g S_c, g S_omega, mu_l1, mu_l2, sigma terms - g S_sigma]
__global__ void k_grad_final(const Inst* __restrict__ insts, const double* __restrict__ adj, int AS,
                             int ZS, const double* __restrict__ part,
                             const int64_t* __restrict__ slot_off, double* __restrict__ grad_out,
                             int batch, double gamma_scale) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  const Inst I = insts[b];
  const double* g = adj + (int64_t)b * AS + ZS;
  double* out = grad_out + (int64_t)b * 7;
  if (g[0] == 0.0) {
    for (int k = 0; k < 7; ++k) out[k] = __longlong_as_double(0x7ff8000000000000LL);
    return;
  }
  double S[kGradSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int q = 0; q < I.rslot_count; ++q) {
    const double* P = part + slot_off[I.rslot_begin + q];
    for (int k = 0; k < kGradSums; ++k) S[k] += P[k];
  }
  const double gam = I.gamma * gamma_scale;
  out[0] = -gam * S[0];
  out[1] = (I.p == 2) ? -gam * S[1] : 0.0;
  out[2] = gam * S[2];
  out[3] = gam * S[3];
  out[4] = g[5];
  out[5] = g[6];
  out[6] = g[7] - gam * S[4];
}

size_t grad_adj_stride(int ZS) { return (size_t)ZS + 8; }

cudaError_t launch_grad(const Inst* insts, const Lset* lsets, const double* W, const double* fac,
                        int64_t facs, const double* xs, const double* zs, const int32_t* lm, int XS,
                        int ZS, const int32_t* st, const double* obs_t, const int64_t* obs_off,
                        const double* dl_dy, double* adj, const Work* rwork, int nrwork,
                        int* counter, double* part, const int64_t* slot_off, double* grad_out,
                        double gamma_scale, int batch, int num_sms, cudaStream_t s) {
  const int AS = (int)grad_adj_stride(ZS);
  k_grad_adjoint<<<batch, kGradThreads, 0, s>>>(insts, lsets, W, fac, facs, xs, zs, lm, XS, ZS, st,
                                                obs_t, obs_off, dl_dy, adj, AS);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grad_rows, kGradRowThreads, 0);
  const int grid = min(nrwork, num_sms * max(1, per_sm));
  k_grad_rows<<<grid, kGradRowThreads, 0, s>>>(insts, lsets, rwork, nrwork, counter, lm, zs, ZS, adj,
                                               AS, part, slot_off);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_grad_final<<<(batch + 127) / 128, 128, 0, s>>>(insts, adj, AS, ZS, part, slot_off, grad_out,
                                                   batch, gamma_scale);
  return cudaGetLastError();
}

}  // namespace nys
