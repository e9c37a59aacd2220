// Block-level (one CTA) dense linear algebra used by the per-instance solve
// kernels: reductions, Householder reflectors, Cholesky, triangular solves and
// the null-space KKT solve with a stored factor.
#pragma once
#include "nys_internal.cuh"

namespace nys {

template <typename T>
struct FacView {  // factor storage of one instance in the T arena
  T* V;    // 2 x M1 Householder vectors
  T* beta; // 2
  T* R;    // 4: R00, R01, R11
  T* H1;   // 2 x M1: first p rows of Q^T H Q
  T* L;    // N2 x N2 lower Cholesky factor (row-major, ld N2)
};
template <typename T>
__device__ __forceinline__ FacView<T> fac_view(T* base, int M1) {
  FacView<T> f;
  f.V = base;
  f.beta = base + 2 * M1;
  f.R = f.beta + 2;
  f.H1 = f.R + 4;
  f.L = f.H1 + 2 * M1;
  return f;
}
inline int64_t fac_elems_inline(int m_max) {
  const int M1 = m_max + 1;
  return 2 * M1 + 2 + 4 + 2 * M1 + (int64_t)M1 * M1;
}

// ---- CTA helpers -----------------------------------------------------------
template <typename T>
__device__ T cta_dot(const T* a, const T* b, int n, T* red) {
  T s = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += a[i] * b[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    T t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    red[32] = t;
  }
  __syncthreads();
  const T r = red[32];
  __syncthreads();
  return r;
}

// Sum over the block of one value per thread (every thread gets the sum).
template <typename T>
__device__ T cta_sum(T s, T* red) {
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    T t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    red[32] = t;
  }
  __syncthreads();
  const T r = red[32];
  __syncthreads();
  return r;
}

// Householder vector of x[0..n): v with v[0] = x0 + sign(x0)|x|, beta = 2/(v^T v),
// (I - beta v v^T) x = -sign(x0)|x| e_0.  Returns the diagonal value.
template <typename T>
__device__ T house(const T* x, T* v, int n, T* beta, T* red) {
  const T nrm2 = cta_dot(x, x, n, red);
  const T nrm = sqrt(nrm2);
  const T x0 = x[0];
  const T sg = (x0 >= T(0)) ? T(1) : T(-1);
  for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = (i == 0) ? x0 + sg * nrm : x[i];
  __syncthreads();
  const T vv = nrm2 + T(2) * sg * nrm * x0 + nrm2;  // |v|^2 = 2|x|^2 + 2|x0||x|
  if (threadIdx.x == 0) *beta = (vv > T(0)) ? T(2) / vv : T(0);
  __syncthreads();
  return -sg * nrm;
}

// A <- (I - b v v^T) A (I - b v v^T) for symmetric A (n x n, ld), w scratch n.
template <typename T>
__device__ void apply_house_sym(T* A, int ld, int n, const T* v, T b, T* w, T* red) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    T s = 0;
    for (int j = 0; j < n; ++j) s += A[i * ld + j] * v[j];
    w[i] = b * s;
  }
  __syncthreads();
  const T k = T(0.5) * b * cta_dot(v, w, n, red);
  for (int i = threadIdx.x; i < n; i += blockDim.x) w[i] -= k * v[i];
  __syncthreads();
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e - (e / n) * n;
    A[i * ld + j] -= v[i] * w[j] + w[i] * v[j];
  }
  __syncthreads();
}

// x <- (I - b v v^T) x
template <typename T>
__device__ void apply_house_vec(T* x, int n, const T* v, T b, T* red) {
  const T s = b * cta_dot(v, x, n, red);
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] -= s * v[i];
  __syncthreads();
}

// In-place lower Cholesky of A (n x n, ld).  Returns false on a non-positive
// pivot (which is replaced by 1).  One barrier per column: every thread takes
// the pivot of column k, the trailing update (a warp per row) scales the
// column entries it reads on the fly, and column k itself is scaled after the
// barrier, while the next update no longer reads it.
template <typename T>
__device__ bool cta_cholesky(T* A, int ld, int n, int* flag) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  bool bad = false;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    T d = A[k * ld + k];
    if (!(d > T(0))) { bad = true; d = T(1); }
    const T lkk = sqrt(d), inv = T(1) / lkk;
    for (int i = k + 1 + warp; i < n; i += nw) {
      const T lik = A[i * ld + k] * inv;
      for (int j = k + 1 + lane; j <= i; j += 32) A[i * ld + j] -= lik * (A[j * ld + k] * inv);
    }
    __syncthreads();
    if (threadIdx.x == 0) A[k * ld + k] = lkk;
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) A[i * ld + k] *= inv;
  }
  __syncthreads();
  if (threadIdx.x == 0) *flag = bad ? 1 : 0;
  return !bad;
}

// In-place lower Cholesky of A (n x n, ld) by the calling warp alone (warp
// barriers only, for small n where block barriers would dominate): lane l
// owns rows l, l + 32, ...; per column k every lane scales its entries of
// column k, then subtracts L_ik L_jk from its rows' trailing entries (column k
// is read by all lanes at the same j: broadcast).  Returns false on a
// non-positive pivot (replaced by 1).
template <typename T>
__device__ bool warp_cholesky(T* A, int ld, int n) {
  const int lane = threadIdx.x & 31;
  bool bad = false;
  for (int k = 0; k < n; ++k) {
    T d = A[k * ld + k];
    if (!(d > T(0))) { bad = true; d = T(1); }
    const T lkk = sqrt(d), inv = T(1) / lkk;
    for (int i = k + 1 + lane; i < n; i += 32) A[i * ld + k] *= inv;
    __syncwarp();
    if (lane == 0) A[k * ld + k] = lkk;
    for (int i = k + 1 + lane; i < n; i += 32) {
      const T lik = A[i * ld + k];
      T* ai = A + i * ld;
      for (int j = k + 1; j <= i; ++j) ai[j] -= lik * A[j * ld + k];
    }
    __syncwarp();
  }
  return !bad;
}

// In-place lower Cholesky of A (n x n, ld), right-looking by panels of 4
// columns: warp 0 factors the panel (pivots, scaling, the panel's own
// updates, warp barriers only), then the whole block subtracts the panel's
// rank-4 product from the trailing lower triangle (a warp per row, lanes over
// columns).  Two block barriers per panel instead of one per column, and each
// trailing entry is read and written once per panel.  Returns false on a
// non-positive pivot (replaced by 1); every thread gets the outcome.
template <typename T>
__device__ bool cta_cholesky_panel(T* A, int ld, int n, int* flag) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  for (int k0 = 0; k0 < n; k0 += 4) {
    const int kb = min(4, n - k0), k1 = k0 + kb;
    if (warp == 0) {
      for (int c = k0; c < k1; ++c) {
        T d = A[c * ld + c];
        if (!(d > T(0))) {
          if (lane == 0) s_bad = 1;
          d = T(1);
        }
        const T lkk = sqrt(d), inv = T(1) / lkk;
        for (int i = c + 1 + lane; i < n; i += 32) A[i * ld + c] *= inv;
        __syncwarp();
        if (lane == 0) A[c * ld + c] = lkk;
        for (int i = c + 1 + lane; i < n; i += 32) {
          const T lic = A[i * ld + c];
          for (int j = c + 1; j < k1 && j <= i; ++j) A[i * ld + j] -= lic * A[j * ld + c];
        }
        __syncwarp();
      }
    }
    __syncthreads();
    for (int i = k1 + warp; i < n; i += nw) {
      T li[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) li[c] = (c < kb) ? A[i * ld + k0 + c] : T(0);
      for (int j = k1 + lane; j <= i; j += 32) {
        T sv = T(0);
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (c < kb) sv += li[c] * A[j * ld + k0 + c];
        A[i * ld + j] -= sv;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *flag = s_bad;
  __syncthreads();
  return *flag == 0;
}

// Cholesky by the whole block: FP32 by panels (cta_cholesky_panel); FP64 one
// warp for n <= kWarpCholMax (warp barriers only), else cta_cholesky.  Every
// thread gets the outcome.  Measured on the metric batch (n = 49, seven solve
// CTAs per SM) the column-by-column block version beat the one-warp version, so
// the warp version is off (kWarpCholMax = 0).
constexpr int kWarpCholMax = 0;
template <typename T>
__device__ bool block_cholesky(T* A, int ld, int n, int* flag) {
  // FP32 factors (MIXED): the panel version; FP64 keeps the column-by-column
  // order of its results
  if (sizeof(T) == sizeof(float)) return cta_cholesky_panel(A, ld, n, flag);
  if (n > kWarpCholMax) return cta_cholesky(A, ld, n, flag);
  __syncthreads();
  if (threadIdx.x < 32) {
    const bool ok = warp_cholesky(A, ld, n);
    if (threadIdx.x == 0) *flag = ok ? 0 : 1;
  }
  __syncthreads();
  return *flag == 0;
}

// Solve L L^T y = b in place by the calling warp (L lower, n x n, ld).  FP32:
// the reciprocals of the diagonal first (all lanes at once), then the two
// substitutions with one multiply per step on the critical path.  FP64 divides
// (the correctly rounded quotients keep the FP64 path's results unchanged on
// ill-conditioned systems).
template <typename T>
__device__ void warp_chol_solve(const T* L, int ld, int n, T* b) {
  const int lane = threadIdx.x & 31;
  if (sizeof(T) == sizeof(double)) {
    for (int k = 0; k < n; ++k) {
      const T yk = b[k] / L[k * ld + k];
      __syncwarp();
      for (int i = k + 1 + lane; i < n; i += 32) b[i] -= L[i * ld + k] * yk;
      if (lane == 0) b[k] = yk;
      __syncwarp();
    }
    for (int k = n - 1; k >= 0; --k) {
      const T yk = b[k] / L[k * ld + k];
      __syncwarp();
      for (int i = lane; i < k; i += 32) b[i] -= L[k * ld + i] * yk;
      if (lane == 0) b[k] = yk;
      __syncwarp();
    }
    return;
  }
  if (n > 128) {
    for (int k = 0; k < n; ++k) {
      const T yk = b[k] / L[k * ld + k];
      __syncwarp();
      for (int i = k + 1 + lane; i < n; i += 32) b[i] -= L[i * ld + k] * yk;
      if (lane == 0) b[k] = yk;
      __syncwarp();
    }
    for (int k = n - 1; k >= 0; --k) {
      const T yk = b[k] / L[k * ld + k];
      __syncwarp();
      for (int i = lane; i < k; i += 32) b[i] -= L[k * ld + i] * yk;
      if (lane == 0) b[k] = yk;
      __syncwarp();
    }
    return;
  }
  // b and the reciprocal diagonal in registers (lane: rows lane + 32 r); per
  // step one shuffle and one multiply on the critical path, the L loads off it
  T bv[4], rd[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = lane + 32 * r;
    bv[r] = (i < n) ? b[i] : T(0);
    rd[r] = (i < n) ? T(1) / L[i * ld + i] : T(0);
  }
  // L y = b
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int kn = min(32, n - 32 * c);
#pragma unroll 4
    for (int kk = 0; kk < kn; ++kk) {
      const int k = 32 * c + kk;
      const T yk = __shfl_sync(0xffffffffu, bv[c], kk) * __shfl_sync(0xffffffffu, rd[c], kk);
#pragma unroll
      for (int r = c; r < 4; ++r) {
        const int i = lane + 32 * r;
        if (i > k && i < n) bv[r] -= L[i * ld + k] * yk;
      }
      if (lane == kk) bv[c] = yk;
    }
  }
  // L^T x = y
#pragma unroll
  for (int c = 3; c >= 0; --c) {
    const int kn = min(32, n - 32 * c);
#pragma unroll 4
    for (int kk = kn - 1; kk >= 0; --kk) {
      const int k = 32 * c + kk;
      const T xk = __shfl_sync(0xffffffffu, bv[c], kk) * __shfl_sync(0xffffffffu, rd[c], kk);
#pragma unroll
      for (int r = 0; r <= c; ++r) {
        const int i = lane + 32 * r;
        if (i < k) bv[r] -= L[k * ld + i] * xk;
      }
      if (lane == kk) bv[c] = xk;
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = lane + 32 * r;
    if (i < n) b[i] = bv[r];
  }
  __syncwarp();
}

// Solve L L^T y = b in place (b overwritten), L lower (n x n, ld).  One warp
// runs both substitutions (warp barriers only); the block waits for it.
template <typename T>
__device__ void cta_chol_solve(const T* L, int ld, int n, T* b) {
  __syncthreads();
  if (threadIdx.x < 32) warp_chol_solve(L, ld, n, b);
  __syncthreads();
}

// Apply the stored factor: given residuals (h: M1, cr: p) return the KKT
// solution (dx: M1, dl: p) of [H C^T; C 0][dx; dl] = [h; cr].  All arrays in
// shared memory; h is overwritten.
// Ls (or nullptr): shared memory for a copy of the N2 x N2 factor L, which the
// substitutions then read there instead of in the global arena; copied here
// unless the caller has staged it (Ls_ready; ordered by the barriers below).
template <typename T>
__device__ void kkt_apply(const FacView<T>& F, int M1, int p, T* h, const T* cr, T* dx, T* dl,
                          T* red, T* Ls = nullptr, bool Ls_ready = false) {
  const T* Lf = F.L;
  if (Ls != nullptr) {
    if (!Ls_ready) {
      const int ne = (M1 - p) * (M1 - p);
      for (int e = threadIdx.x; e < ne; e += blockDim.x) Ls[e] = F.L[e];
    }
    Lf = Ls;
  }
  // h' = Q^T h = H_p .. H_1 h
  for (int k = 0; k < p; ++k) apply_house_vec(h, M1, F.V + k * M1, F.beta[k], red);
  // y1 = R^{-T} cr
  __shared__ T y1s[2];
  if (threadIdx.x == 0) {
    y1s[0] = cr[0] / F.R[0];
    if (p == 2) y1s[1] = (cr[1] - F.R[1] * y1s[0]) / F.R[2];
  }
  __syncthreads();
  const int N2 = M1 - p;
  // rhs2 = h'[p:] - H'[p:, :p] y1   (H'[p:, :p] = H1[:, p:]^T)
  for (int i = threadIdx.x; i < N2; i += blockDim.x) {
    T s = h[p + i];
    for (int k = 0; k < p; ++k) s -= F.H1[k * M1 + p + i] * y1s[k];
    dx[p + i] = s;
  }
  __syncthreads();
  cta_chol_solve(Lf, N2, N2, dx + p);
  // lambda: R lam = h'[:p] - H'[:p, :] y
  if (threadIdx.x < 2 && threadIdx.x < p) dx[threadIdx.x] = y1s[threadIdx.x];
  __syncthreads();
  T r0 = cta_dot(F.H1, dx, M1, red);
  T r1 = (p == 2) ? cta_dot(F.H1 + M1, dx, M1, red) : T(0);
  if (threadIdx.x == 0) {
    r0 = h[0] - r0;
    r1 = (p == 2) ? h[1] - r1 : T(0);
    if (p == 2) {
      dl[1] = r1 / F.R[2];
      dl[0] = (r0 - F.R[1] * dl[1]) / F.R[0];
    } else {
      dl[0] = r0 / F.R[0];
    }
  }
  __syncthreads();
  // dx = Q y = H_1 .. H_p y
  for (int k = p - 1; k >= 0; --k) apply_house_vec(dx, M1, F.V + k * M1, F.beta[k], red);
}

}  // namespace nys
