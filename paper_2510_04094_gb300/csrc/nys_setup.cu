// Nystrom setup (Appendix A.3 and the feature map eq32): landmark kernel Omega_mm,
// symmetric eigendecomposition in FP64, feature factor W = Lambda^{-1/2} U^T
// with eigenpairs below tau * lambda_max dropped.
//
// One CTA per distinct landmark set.  Eigensolver: parallel cyclic Jacobi
// (Golub & Van Loan, Matrix Computations, Sec. 8.5) with the round-robin
// ("chess tournament") ordering, so the m/2 rotations of a round touch
// disjoint row/column pairs and run concurrently.  A and the rotation
// accumulator V live in shared memory (2 m (m+1) doubles, <= 203 KB for
// m <= kMMax); larger landmark sets use a global (L2-resident) area instead.
#include "nys_internal.cuh"

namespace nys {

constexpr int kMaxSweeps = 40;

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) red[0] = s;
  }
  __syncthreads();
  s = red[0];
  __syncthreads();
  return s;
}

__device__ __forceinline__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
    if (threadIdx.x == 0) red[0] = s;
  }
  __syncthreads();
  s = red[0];
  __syncthreads();
  return s;
}

// Parallel cyclic Jacobi sweeps on the symmetric m x m matrix A (ld), rotations
// accumulated in V.  Round-robin ("chess tournament") pairing of N = m rounded
// up to even players: in round r player 0 stays, the others sit at
// 1 + ((k - 1 - r) mod (N - 1)); pair k = (slot k, slot N-1-k); index m, if
// present, sits out (identity rotation).  Each round: one thread per pair
// computes the pair's rotation (symmetric Schur decomposition) from the
// round's starting entries; after a barrier the CTA applies A <- J^T A J to
// whole 2x2 blocks (row pair a, column pair b: the column rotation, then the
// row rotation, as two sequential one-sided passes would) and V <- V J to row
// segments, all independent.  Stops when off(A)^2 <=
// tol tot(A)^2, or (stall > 0) once off(A)^2 <= stall tot(A)^2 and a sweep no
// longer shrinks it fourfold: the rounding floor of the working precision.
__device__ __forceinline__ int rr_pos(int k, int r, int N) {
  if (k == 0) return 0;
  int t = (k - 1 - r) % (N - 1);
  if (t < 0) t += N - 1;
  return 1 + t;
}

template <typename T, int kJW>   // kJW: warps of the CTA
__device__ void jacobi_sweeps(T* A, T* V, int ld, int m, int N, T* cs, int* pq, double* red,
                              double tol, int max_sweeps, double stall) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int half = N / 2;
  constexpr int kJB = sizeof(T) == 4 ? 4 : 2;   // row pairs whose loads are batched
  double prev = 1e300;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int j = warp; j < m; j += nw)
      for (int l = lane; l < m; l += 32) {
        const double a = (double)A[j * ld + l];
        tot += a * a;
        if (j != l) off += a * a;
      }
    off = block_sum(off, red);
    tot = block_sum(tot, red);
    if (off <= tol * tot) break;
    if (stall > 0.0 && off <= stall * tot && off > 0.25 * prev) break;
    prev = off;
    for (int round = 0; round < N - 1; ++round) {
      for (int k = tid; k < half; k += nt) {
        int p = rr_pos(k, round, N), q = rr_pos(N - 1 - k, round, N);
        if (p > q) { const int t = p; p = q; q = t; }
        T c = T(1), sn = T(0);
        if (q < m) {
          const T apq = A[p * ld + q];
          if (fabs(apq) > T(1e-30)) {
            const T tau_ = (A[q * ld + q] - A[p * ld + p]) / (T(2) * apq);
            const T t = (tau_ >= T(0) ? T(1) : T(-1)) / (fabs(tau_) + sqrt(T(1) + tau_ * tau_));
            c = T(1) / sqrt(T(1) + t * t);
            sn = t * c;
          }
        }
        cs[k] = c;
        cs[half + k] = sn;
        pq[k] = p;
        pq[half + k] = q;
      }
      __syncthreads();
      // lane <-> column pair b (its rotation read once per round); warp <-> row
      // pairs a and rows i of V; a thread's loads all precede its stores
      for (int b = lane; b < half; b += 32) {
        const int p2 = pq[b], q2 = pq[half + b];
        const T c2 = cs[b], s2 = cs[half + b];
        const bool h2 = q2 < m;
        for (int a0 = warp; a0 < half; a0 += kJB * kJW) {
        T x[kJB][4];
#pragma unroll
        for (int j = 0; j < kJB; ++j) {
          const int a = a0 + j * kJW;
          if (a < half) {
            const int p1 = pq[a], q1 = pq[half + a];
            const bool h1 = q1 < m;
            x[j][0] = A[p1 * ld + p2];
            x[j][1] = h2 ? A[p1 * ld + q2] : T(0);
            x[j][2] = h1 ? A[q1 * ld + p2] : T(0);
            x[j][3] = (h1 && h2) ? A[q1 * ld + q2] : T(0);
          }
        }
#pragma unroll
        for (int j = 0; j < kJB; ++j) {
          const int a = a0 + j * kJW;
          if (a < half) {
            const int p1 = pq[a], q1 = pq[half + a];
            const T c1 = cs[a], s1 = cs[half + a];
            const bool h1 = q1 < m;
            const T y00 = c2 * x[j][0] - s2 * x[j][1], y01 = s2 * x[j][0] + c2 * x[j][1];
            const T y10 = c2 * x[j][2] - s2 * x[j][3], y11 = s2 * x[j][2] + c2 * x[j][3];
            A[p1 * ld + p2] = c1 * y00 - s1 * y10;
            if (h2) A[p1 * ld + q2] = c1 * y01 - s1 * y11;
            if (h1) A[q1 * ld + p2] = s1 * y00 + c1 * y10;
            if (h1 && h2) A[q1 * ld + q2] = s1 * y01 + c1 * y11;
          }
        }
        }
        if (h2) {
          for (int i0 = warp; i0 < m; i0 += 4 * kJW) {
            T vp[4], vq[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int i = i0 + u * kJW;
              if (i < m) { vp[u] = V[i * ld + p2]; vq[u] = V[i * ld + q2]; }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int i = i0 + u * kJW;
              if (i < m) {
                V[i * ld + p2] = c2 * vp[u] - s2 * vq[u];
                V[i * ld + q2] = s2 * vp[u] + c2 * vq[u];
              }
            }
          }
        }
      }
      __syncthreads();
    }
  }
}

// perm[0..m) = indices of the diagonal entries of A in descending order (ties by
// index), one rank per thread
template <typename T>
__device__ void sort_desc(const T* A, int ld, int m, int* perm) {
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    const T d = A[k * ld + k];
    int r = 0;
    for (int j = 0; j < m; ++j) {
      const T e = A[j * ld + j];
      r += (e > d) || (e == d && j < k);
    }
    perm[r] = k;
  }
  __syncthreads();
}

// NT threads per CTA: 256 for the small landmark counts (several CTAs per SM),
// 512 / 1024 for the large ones, whose shared memory leaves room for 2 / 1 CTAs.
// kG: landmark counts above kMMax, whose matrices do not fit in shared memory,
// work in a global (L2-resident) area of their own, one CTA per listed set.
template <int NT, bool kG>
__global__ void __launch_bounds__(NT, NT == 256 ? 4 : (NT == 512 ? 2 : 1))
k_setup_eig(Lset* lsets, const int32_t* __restrict__ lm_idx, double* __restrict__ W_all,
            float* __restrict__ W32_all, double* __restrict__ lam_all, double tau, int allow_chol,
            int m_lo, int m_hi, BigSet big) {
  // the grid covers every slot; inactive slots (instances that share another
  // instance's set) return at once, so a captured graph stays valid when an
  // update changes which instances share
  const int L = kG ? big.ids[blockIdx.x] : blockIdx.x;
  const Lset S = lsets[L];
  // one launch per landmark-count class (m_lo, m_hi], each with shared memory
  // for its own largest m
  if (!S.active || S.m <= m_lo || S.m > m_hi) return;
  const int m = S.m;
  const int N = m + (m & 1);  // even player count; index m (if present) is a bye
  const int ld = m + 1;
  extern __shared__ double smem_eig[];
  double* sm = kG ? big.ws + (int64_t)blockIdx.x * big.stride : smem_eig;
  double* A = sm;
  double* V = A + m * ld;
  double* cs = V + m * ld;                 // N/2 cosines then N/2 sines
  double* red = cs + N;                    // 32
  int* pos = reinterpret_cast<int*>(red + 32);   // N: the round's pairs (p then q)
  int* perm = pos + N;                     // m
  int* idx = perm + m;                     // m
  const int tid = threadIdx.x, nt = blockDim.x;

  for (int j = tid; j < m; j += nt) idx[j] = lm_idx[S.lm_off + j];
  __syncthreads();
  double* Wl = W_all + S.w_off;
  float* W32l = W32_all + S.w_off;

  // Cholesky route.  Any W with W^T W = Omega^-1 gives the same features up to
  // an orthogonal map of omega-space, hence the same fit (Appendix A.3's factor
  // Lambda^-1/2 U^T is one such W).  With Omega = L L^T, W = L^-1 costs m^3/3
  // + m^3/3 FP64 flops instead of a Jacobi eigendecomposition's ~10 sweeps.
  // It is used when the bound cond(Omega) <= |Omega|_inf |W|_F^2 certifies
  // that nothing would be truncated and that the kernel-coordinate Gram keeps
  // its precision (cond(Omega) sqrt(n) <= kKernelSpan).  Only for
  // FP64 solves (allow_chol): L^-1 has large alternating entries, and the FP32
  // factor of the mixed path built from it refines about ten times slower
  // than one built from the nearly orthogonal rows of Lambda^-1/2 U^T.
  if (allow_chol) {
    for (int e = tid; e < m * m; e += nt) {
      const int j = e / m, l = e % m;
      const double d = (double)(idx[j] - idx[l]) * S.hs;
      V[j * ld + l] = exp(-d * d);
    }
    __shared__ int s_bad;
    if (tid == 0) s_bad = 0;
    __syncthreads();
    // |Omega|_2 <= |Omega|_inf (largest row sum; the entries are positive)
    double rmax = 0.0;
    for (int j = tid; j < m; j += nt) {
      double rs = 0.0;
      for (int l = 0; l < m; ++l) rs += V[j * ld + l];
      rmax = fmax(rmax, rs);
    }
    rmax = block_max(rmax, red);
    for (int k = 0; k < m; ++k) {   // lower Cholesky of Omega in V
      if (tid == 0) {
        const double d = V[k * ld + k];
        if (!(d > 0.0)) { s_bad = 1; V[k * ld + k] = 1.0; }
        else V[k * ld + k] = sqrt(d);
      }
      __syncthreads();
      const double lkk = V[k * ld + k];
      for (int i = k + 1 + tid; i < m; i += nt) V[i * ld + k] /= lkk;
      __syncthreads();
      const int R = m - k - 1;
      for (int e = tid; e < R * R; e += nt) {
        const int i = k + 1 + e / R, j = k + 1 + e % R;
        if (j <= i) V[i * ld + j] -= V[i * ld + k] * V[j * ld + k];
      }
      __syncthreads();
    }
    // W = L^-1 into A (lower triangular), one column per thread: L w = e_c
    for (int c = tid; c < m; c += nt) {
      for (int i = 0; i < c; ++i) A[i * ld + c] = 0.0;
      for (int i = c; i < m; ++i) {
        double sv = (i == c) ? 1.0 : 0.0;
        for (int k2 = c; k2 < i; ++k2) sv -= V[i * ld + k2] * A[k2 * ld + c];
        A[i * ld + c] = sv / V[i * ld + i];
      }
    }
    __syncthreads();
    {
      double f2 = 0.0;
      for (int e = tid; e < m * m; e += nt) {
        const double w = A[(e / m) * ld + (e % m)];
        f2 += w * w;
      }
      f2 = block_sum(f2, red);
      // cond(Omega) <= |Omega|_inf |Omega^-1|_2 <= rmax |W|_F^2 certifies that the
      // kernel-coordinate Gram stays within its FP64 budget (kKernelSpan)
      const bool chol_ok = allow_chol && (s_bad == 0) && isfinite(f2) &&
                           (rmax * f2 * sqrt((double)S.n) <= kKernelSpan);
      if (chol_ok) {
        for (int e = tid; e < m * m; e += nt) {
          const double w = A[(e / m) * ld + (e % m)];
          Wl[e] = w;
          W32l[e] = (float)w;
        }
        for (int k = tid; k < m; k += nt) {
          const double l = V[k * ld + k];
          lam_all[(int64_t)L * kMLarge + k] = l * l;   // Cholesky pivots (informational)
        }
        if (tid == 0) {
          lsets[L].m_eff = m;
          lsets[L].omode = 0;
        }
        return;
      }
    }
  }
  // FP32 route (mixed contexts): Jacobi sweeps in FP32 (64x the FP64 rate), then
  // one FP64 correction that makes W an exact whitening again: with W0 from the
  // FP32 eigenpairs, M = W0 Omega W0^T = I + E and W = (I - E/2) W0 satisfies
  // W^T W = Omega^-1 up to O(E^2); its rows stay nearly orthogonal, which the
  // FP32 factor of the mixed path needs.  Used when lambda_min > 1e-5 lambda_max
  // (nothing truncated) and |E| <= 1e-5; otherwise the FP64 Jacobi below.
  if (!allow_chol) {
    for (int e = tid; e < m * m; e += nt) {
      const int j = e / m, l = e % m;
      const double d = (double)(idx[j] - idx[l]) * S.hs;
      A[j * ld + l] = exp(-d * d);
    }
    float* Af = reinterpret_cast<float*>(V);   // two m x ld float matrices in V's space
    float* Vf = Af + m * ld;
    __syncthreads();
    for (int e = tid; e < m * m; e += nt) {
      const int j = e / m, l = e % m;
      Af[j * ld + l] = (float)A[j * ld + l];
      Vf[j * ld + l] = (j == l) ? 1.f : 0.f;
    }
    __syncthreads();
    // FP32 sweeps reach off(A)^2 ~ 1e-13 tot(A)^2; the correction below absorbs the rest
    jacobi_sweeps<float, NT / 32>(Af, Vf, ld, m, N, reinterpret_cast<float*>(cs), pos, red, 1e-13,
                                  kMaxSweeps, 1e-9);
    sort_desc(Af, ld, m, perm);
    if (tid == 0) {
      const double lmax = Af[perm[0] * ld + perm[0]], lmin = Af[perm[m - 1] * ld + perm[m - 1]];
      red[0] = (lmin > 1e-5 * lmax && lmin > 0.0) ? 1.0 : 0.0;
    }
    __syncthreads();
    const bool well = red[0] != 0.0;
    __syncthreads();
    if (well) {
      // W0 = Lambda^-1/2 U^T (descending), straight to the output (one square
      // root and reciprocal per eigenvalue, in the free cosine area)
      double* rsq = cs;
      for (int k = tid; k < m; k += nt) rsq[k] = 1.0 / sqrt((double)Af[perm[k] * ld + perm[k]]);
      __syncthreads();
      for (int e = tid; e < m * m; e += nt) {
        const int k = e / m, j = e % m;
        const int c = perm[k];
        Wl[e] = (double)Vf[j * ld + c] * rsq[k];
      }
      for (int k = tid; k < m; k += nt) lam_all[(int64_t)L * kMLarge + k] = (double)Af[perm[k] * ld + perm[k]];
      __syncthreads();
      double* Tm = V;                           // T = W0 Omega (the FP32 matrices are done)
      for (int e = tid; e < m * m; e += nt) {
        const int k = e / m, j = e % m;
        double sv = 0.0;
        for (int i = 0; i < m; ++i) sv += Wl[k * m + i] * A[i * ld + j];
        Tm[k * ld + j] = sv;
      }
      __syncthreads();
      for (int e = tid; e < m * m; e += nt) {   // E = T W0^T - I, into A
        const int k = e / m, l = e % m;
        double sv = 0.0;
        for (int j = 0; j < m; ++j) sv += Tm[k * ld + j] * Wl[l * m + j];
        A[k * ld + l] = sv - (k == l ? 1.0 : 0.0);
      }
      __syncthreads();
      double emax = 0.0;
      for (int e = tid; e < m * m; e += nt) emax = fmax(emax, fabs(A[(e / m) * ld + (e % m)]));
      emax = block_max(emax, red);
      if (emax <= 1e-5) {
        for (int e = tid; e < m * m; e += nt) {   // W = W0 - E W0 / 2, into V
          const int k = e / m, j = e % m;
          double sv = 0.0;
          for (int l = 0; l < m; ++l) sv += A[k * ld + l] * Wl[l * m + j];
          Tm[k * ld + j] = Wl[k * m + j] - 0.5 * sv;
        }
        __syncthreads();
        for (int e = tid; e < m * m; e += nt) {
          const double w = Tm[(e / m) * ld + (e % m)];
          Wl[e] = w;
          W32l[e] = (float)w;
        }
        if (tid == 0) {
          lsets[L].m_eff = m;
          lsets[L].omode = 0;
        }
        return;
      }
    }
  }
  // FP64 Jacobi route: the landmark kernel again, V = I
  for (int e = tid; e < m * m; e += nt) {
    const int j = e / m, l = e % m;
    const double d = (double)(idx[j] - idx[l]) * S.hs;
    A[j * ld + l] = exp(-d * d);
    V[j * ld + l] = (j == l) ? 1.0 : 0.0;
  }
  __syncthreads();
  jacobi_sweeps<double, NT / 32>(A, V, ld, m, N, cs, pos, red, 1e-30, kMaxSweeps, 0.0);

  // sort eigenvalues descending, keep lambda > tau * lambda_max
  sort_desc(A, ld, m, perm);
  if (tid == 0) {
    const double lmax = A[perm[0] * ld + perm[0]];
    int me = 0;
    while (me < m && A[perm[me] * ld + perm[me]] > tau * lmax) ++me;
    lsets[L].m_eff = me;
    const double lmin = A[perm[me - 1] * ld + perm[me - 1]];
    // omega coordinates: a span beyond what the FP32 factor or (FP64 contexts,
    // allow_chol) the FP64 kernel-coordinate Gram can carry, see kKernelSpan
    lsets[L].omode = (lmin < kOmegaCond * lmax ||
                      (allow_chol && lmax > lmin * (kKernelSpan / sqrt((double)S.n)))) ? 1 : 0;
    red[0] = (double)me;
  }
  __syncthreads();
  const int me = (int)red[0];
  for (int e = tid; e < m * m; e += nt) {
    const int k = e / m, j = e % m;
    double w = 0.0;
    if (k < me) {
      const int c = perm[k];
      w = V[j * ld + c] / sqrt(A[c * ld + c]);
    }
    Wl[e] = w;
    W32l[e] = (float)w;
  }
  for (int k = tid; k < m; k += nt) lam_all[(int64_t)L * kMLarge + k] = A[perm[k] * ld + perm[k]];
}

// Lag tables of a landmark set on its uniform grid.  Every feature value of
// Section 3 depends on t_i - s_j = k h only (landmarks are grid points), so for
// k = 0..K the setup stores, in FP64 rounded to float-float,
//     b0(k) = e,  b1(k) = x e,  b2(k) = u e,   x = k h/sigma, u = x^2, e = exp(-u)
// (b0, b2 even and b1 odd in k).  kappa of any row is A0 b0 + A1 b1 + A2 b2.
__global__ void __launch_bounds__(256)
k_setup_lag(const Lset* __restrict__ lsets, float* __restrict__ lag) {
  const Lset S = lsets[blockIdx.x];
  if (!S.active) return;
  float* T = lag + S.lag_off;
  for (int k = blockIdx.y * blockDim.x + threadIdx.x; k <= S.K; k += gridDim.y * blockDim.x) {
    const double x = (double)k * S.hs;
    const double u = x * x;
    const double e = exp(-u);
    const double b[3] = {e, x * e, u * e};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float hi = (float)b[q];
      T[6 * k + 2 * q] = hi;
      T[6 * k + 2 * q + 1] = (float)(b[q] - (double)hi);
    }
  }
}

size_t setup_smem_bytes(int m) {
  const int N = m + (m & 1);
  return sizeof(double) * (2 * (size_t)m * (m + 1) + N + 32) + sizeof(int) * (N + 2 * m);
}

// The lag tables feed the row passes; the eigendecomposition only the solve.
cudaError_t launch_lag(const Lset* lsets, int capacity, float* lag, cudaStream_t st) {
  if (capacity == 0 || lag == nullptr) return cudaSuccess;
  k_setup_lag<<<dim3(capacity, 8), 256, 0, st>>>(lsets, lag);
  return cudaGetLastError();
}

// m_bounds: increasing class bounds of the landmark counts present (nclass of
// them, the last >= every m); nclass == 0: one class up to m_max.
template <int NT>
static cudaError_t launch_eig_class(Lset* lsets, int capacity, const int32_t* lm_idx, double* W,
                                    float* W32, double* lam, double tau, int allow_chol, int lo,
                                    int hi, cudaStream_t st) {
  const size_t sm = setup_smem_bytes(hi);
  cudaError_t e = cudaFuncSetAttribute(k_setup_eig<NT, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_setup_eig<NT, false><<<capacity, NT, sm, st>>>(lsets, lm_idx, W, W32, lam, tau, allow_chol, lo,
                                                   hi, BigSet());
  return cudaGetLastError();
}

size_t setup_ws_doubles() { return setup_smem_bytes(kMLarge) / sizeof(double) + 1; }

static cudaError_t launch_eig_sets(Lset* lsets, int capacity, const int32_t* lm_idx, double* W,
                                   float* W32, double* lam, double tau, int m_max, cudaStream_t st,
                                   int allow_chol, const int* m_bounds, int nclass, BigSet big,
                                   int few_sets);

// Condition rows of every active landmark set in omega coordinates (FP64), at
// the kernel width sigma of the set's first instance (Lemma 1's C, Appendix A.4):
//     E[e][d][k] = sum_j W_kj (-1/sigma)^d H_d(x_j) exp(-x_j^2),  x_j = (tau_e - idx_j) h/sigma,
// tau_0 = 0 (t_1), tau_1 = n - 1 (t_n), d = 0..3 (physicists' Hermite H_d),
// rows k < m_eff (zero from m_eff on), summed as the solve would (a warp per
// row, lanes over j, then a butterfly), so that the solve of every instance with
// this set and sigma reads them instead of forming its own.
__global__ void __launch_bounds__(128)
k_setup_crow(const Inst* __restrict__ insts, const Lset* __restrict__ lsets,
             const int32_t* __restrict__ lm_idx, const double* __restrict__ W_all,
             double* __restrict__ crow, int CS) {
  const Lset L = lsets[blockIdx.x];
  if (!L.active) return;
  __shared__ double s_e[8][kMLarge];
  const int m = L.m, me = L.m_eff;
  const double sigma = insts[blockIdx.x].sigma;
  for (int e = threadIdx.x; e < 8 * m; e += blockDim.x) {
    const int q = e / m, j = e - q * m, end = q >> 2, d = q & 3;
    const double x = (double)((end ? L.n - 1 : 0) - lm_idx[L.lm_off + j]) * L.hs;
    const double x2 = x * x;
    double H;
    if (d == 0) H = 1.0;
    else if (d == 1) H = 2.0 * x;
    else if (d == 2) H = 4.0 * x2 - 2.0;
    else H = (8.0 * x2 - 12.0) * x;
    double sc = 1.0;
    for (int r = 0; r < d; ++r) sc *= -1.0 / sigma;
    s_e[q][j] = sc * H * exp(-x2);
  }
  __syncthreads();
  const double* W = W_all + L.w_off;
  double* E = crow + (int64_t)blockIdx.x * 8 * CS;
  const int lane = threadIdx.x & 31;
  for (int k = threadIdx.x >> 5; k < m; k += blockDim.x >> 5) {
    double sr[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (k < me) {
      for (int j = lane; j < m; j += 32) {
        const double w = W[(int64_t)k * m + j];
#pragma unroll
        for (int q = 0; q < 8; ++q) sr[q] += w * s_e[q][j];
      }
#pragma unroll
      for (int q = 0; q < 8; ++q)
        for (int o = 16; o > 0; o >>= 1) sr[q] += __shfl_xor_sync(0xffffffffu, sr[q], o);
    }
    if (lane < 8) {
      double v = sr[0];
#pragma unroll
      for (int q = 1; q < 8; ++q) if (lane == q) v = sr[q];
      E[lane * CS + k] = v;
    }
  }
}

cudaError_t launch_eig(Lset* lsets, int capacity, const int32_t* lm_idx, double* W, float* W32,
                       double* lam, double tau, int m_max, cudaStream_t st, int allow_chol,
                       const int* m_bounds, int nclass, BigSet big, double* crow,
                       const Inst* insts, int few_sets) {
  if (capacity == 0) return cudaSuccess;
  cudaError_t ec = launch_eig_sets(lsets, capacity, lm_idx, W, W32, lam, tau, m_max, st, allow_chol,
                                   m_bounds, nclass, big, few_sets);
  if (ec != cudaSuccess || crow == nullptr || insts == nullptr) return ec;
  k_setup_crow<<<capacity, 128, 0, st>>>(insts, lsets, lm_idx, W, crow, m_max);
  return cudaGetLastError();
}

static cudaError_t launch_eig_sets(Lset* lsets, int capacity, const int32_t* lm_idx, double* W,
                                   float* W32, double* lam, double tau, int m_max, cudaStream_t st,
                                   int allow_chol, const int* m_bounds, int nclass, BigSet big,
                                   int few_sets) {
  int lo = 0;
  for (int k = 0; k < (nclass > 0 ? nclass : 1) && lo < kMMax; ++k) {
    const int hi = std::min((nclass > 0) ? m_bounds[k] : m_max, kMMax);
    if (hi <= lo) continue;
    // threads per CTA from the class's shared memory: one CTA per SM above
    // ~113 KB, two above ~75 KB (of the SM's 228 KB)
    const size_t sm = setup_smem_bytes(hi);
    cudaError_t e;
    // few sets (no more than SMs): wider CTAs shorten each set's Jacobi rounds
    // (measured: a single m = 50 set, FP32 route, 512 threads 0.06 ms faster than 256)
    if (few_sets && !allow_chol && sm <= 113 * 1024)
      e = launch_eig_class<512>(lsets, capacity, lm_idx, W, W32, lam, tau, allow_chol, lo, hi, st);
    else if (sm > 113 * 1024)
      e = launch_eig_class<1024>(lsets, capacity, lm_idx, W, W32, lam, tau, allow_chol, lo, hi, st);
    else if (sm > 75 * 1024)
      e = launch_eig_class<512>(lsets, capacity, lm_idx, W, W32, lam, tau, allow_chol, lo, hi, st);
    else
      e = launch_eig_class<256>(lsets, capacity, lm_idx, W, W32, lam, tau, allow_chol, lo, hi, st);
    if (e != cudaSuccess) return e;
    lo = hi;
  }
  if (big.n > 0) {   // landmark counts above kMMax: global workspace
    k_setup_eig<1024, true><<<big.n, 1024, 0, st>>>(lsets, lm_idx, W, W32, lam, tau, allow_chol,
                                                     kMMax, kMLarge, big);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_setup(Lset* lsets, int capacity, const int32_t* lm_idx, double* W, float* W32,
                         double* lam, float* lag, double tau, int m_max, cudaStream_t st,
                         int allow_chol, const int* m_bounds, int nclass, BigSet big, double* crow,
                         const Inst* insts, int few_sets) {
  cudaError_t e = launch_lag(lsets, capacity, lag, st);
  if (e != cudaSuccess) return e;
  return launch_eig(lsets, capacity, lm_idx, W, W32, lam, tau, m_max, st, allow_chol, m_bounds,
                    nclass, big, crow, insts, few_sets);
}

}  // namespace nys
