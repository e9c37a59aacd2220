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
  int t = k - 1 - r;   // 0 <= k - 1, r < N - 1
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

// ---- FP32 route eigensolver --------------------------------------------------
// Rotation annihilating apq of the symmetric block [[app, apq], [apq, aqq]]
// (Golub & Van Loan's symmetric Schur step): tau = (aqq - app) / (2 apq),
// t = sign(tau) / (|tau| + sqrt(1 + tau^2)) (t -> 0 once tau^2 overflows),
// c = 1 / sqrt(1 + t^2), s = t c.  The two divisions are the approximate ones
// (a small error in t only perturbs the angle); c is the approximate reciprocal
// square root refined by one Newton-Raphson step, so that c^2 + s^2 = 1 to
// FP32 rounding, which keeps the accumulated V orthogonal.
__device__ __forceinline__ void f32_rotation(float app, float aqq, float apq, float& c, float& s) {
  c = 1.f;
  s = 0.f;
  if (fabsf(apq) > 1e-30f) {
    const float tau = __fdividef(aqq - app, 2.f * apq);
    const float t = __fdividef(copysignf(1.f, tau), fabsf(tau) + sqrtf(fmaf(tau, tau, 1.f)));
    if (t != 0.f) {
      const float x = fmaf(t, t, 1.f);
      const float y = rsqrtf(x);
      c = y * fmaf(-0.5f * x * y, y, 1.5f);
      s = t * c;
    }
  }
}

// (sh, sl) += u (w.x + w.y): the product u w.x split exactly (FMA), summed by
// Knuth's two-sum, the low parts gathered in sl (float-float accumulation)
__device__ __forceinline__ void ff_fma(float& sh, float& sl, float u, float2 w) {
  const float p = u * w.x;
  const float pe = fmaf(u, w.x, -p);
  const float t = sh + p;
  const float z = t - sh;
  const float err = (sh - (t - z)) + (p - z);
  sh = t;
  sl = fmaf(u, w.y, sl + (err + pe));
}

__device__ __forceinline__ int upk(int i, int j, int ld) { return min(i, j) * ld + max(i, j); }

// Rotates the 2x2 block of rows (r1, r2) and columns (c1, c2) of A (packed
// upper addresses e0..e3 of (r1,c1), (r1,c2), (r2,c1), (r2,c2)): the column
// rotation (c2, s2), then the row rotation (c1, s1).
__device__ __forceinline__ void f32_block(float* A, int e0, int e1, int e2, int e3, float c1,
                                          float s1, float c2, float s2) {
  const float x0 = A[e0], x1 = A[e1], x2 = A[e2], x3 = A[e3];
  const float y00 = c2 * x0 - s2 * x1, y01 = s2 * x0 + c2 * x1;
  const float y10 = c2 * x2 - s2 * x3, y11 = s2 * x2 + c2 * x3;
  A[e0] = c1 * y00 - s1 * y10;
  A[e1] = c1 * y01 - s1 * y11;
  A[e2] = s1 * y00 + c1 * y10;
  A[e3] = s1 * y01 + c1 * y11;
}

// Parallel cyclic Jacobi in FP32 on one CTA of NW warps (the same tournament
// ordering as jacobi_sweeps).  A: the even-padded N x N matrix in shared
// memory, only its upper triangle stored and updated (entry (i, j) at
// min(i,j) ldf + max(i,j)); the bye player of an odd m is a zero row and
// column.  A round: warp 0 computes the rotations of the pairs into
// prm[b] = (p | swapped << 16, q, c, s) (p < q the pair's players, swapped:
// slot b holds q); a barrier; the upper 2x2 blocks (a, b), a < b, are rotated
// by the warp of row pair a, folded with row pair half-1-a so that each lane
// has one block, and the diagonal blocks by the last warp; a second barrier.
// The accumulated rotations V live in registers: lane b holds the tournament
// slots (b, N-1-b) of the rows w + NW u of warp w.  After each round the
// players move one slot (k -> k+1 over 1..N-1, slot 0 fixed), two shuffles per
// register row, so every lane keeps rotating its own pair of slots; after a
// whole sweep each player is back in its own slot and V (m rows, ldf) is
// written to Vout in player order.  Stopping rule as jacobi_sweeps.  Returns 1;
// 0 (nothing done) when N > NW U (not enough register rows); -1 when an index
// check of a debug build failed.
template <int NW, int HB, int U>
__device__ int jacobi_f32(float* A, float* Vout, int ldf, int m, float4* prm, float* red,
                          double tol, int max_sweeps, double stall) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int N = m + (m & 1), half = N >> 1, nfold = (half + 1) >> 1;
  if (N > NW * U || half > 32 * HB) return 0;
  __shared__ int s_jbad;
  if (threadIdx.x == 0) s_jbad = 0;
  float vf[U][HB], vs[U][HB];
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int hb = 0; hb < HB; ++hb) {
      const int i = warp + NW * u, b = lane + 32 * hb;
      vf[u][hb] = (i == b) ? 1.f : 0.f;
      vs[u][hb] = (i == N - 1 - b) ? 1.f : 0.f;
    }
  double prev = 1e300;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    float off = 0.f, dg = 0.f;
    for (int j = warp; j < m; j += NW)
      for (int l = j + lane; l < m; l += 32) {
        const float a = A[j * ldf + l];
        if (l == j) dg = fmaf(a, a, dg);
        else off = fmaf(a, a, off);
      }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      dg += __shfl_xor_sync(0xffffffffu, dg, o);
    }
    if (lane == 0) { red[warp] = off; red[NW + warp] = dg; }
    __syncthreads();
    off = 0.f;
    dg = 0.f;
#pragma unroll
    for (int w = 0; w < NW; ++w) { off += red[w]; dg += red[NW + w]; }
    __syncthreads();
    off *= 2.f;
    const double offd = off, totd = (double)off + (double)dg;
    if (offd <= tol * totd) break;
    if (stall > 0.0 && offd <= stall * totd && offd > 0.25 * prev) break;
    prev = offd;
    for (int r = 0; r < N - 1; ++r) {
      if (warp == 0) {
#pragma unroll
        for (int hb = 0; hb < HB; ++hb) {
          const int b = lane + 32 * hb;
          if (b < half) {
            const int f = rr_pos(b, r, N), g = rr_pos(N - 1 - b, r, N);
            const int p = min(f, g), q = max(f, g);
            float c, sn;
            f32_rotation(A[p * ldf + p], A[q * ldf + q], A[p * ldf + q], c, sn);
            prm[b] = make_float4(__int_as_float(p | (f > g ? 0x10000 : 0)), __int_as_float(q), c, sn);
          }
        }
      }
      __syncthreads();
      int pp[HB], qq[HB];
      float cc[HB], ss[HB], se[HB];
#pragma unroll
      for (int hb = 0; hb < HB; ++hb) {
        const float4 P = prm[min(lane + 32 * hb, half - 1)];
        const int pe = __float_as_int(P.x);
        pp[hb] = pe & 0xffff;
        qq[hb] = __float_as_int(P.y);
        cc[hb] = P.z;
        ss[hb] = P.w;
        se[hb] = (pe & 0x10000) ? -P.w : P.w;   // the sine in slot order
      }
      // off-diagonal upper blocks: lane b takes (a, b) for b > a, else
      // (half-1-a, half-1-b) (none for the middle row pair of an odd half)
      for (int a = warp; a < nfold; a += NW) {
        const int a2 = half - 1 - a;
        const float4 PA = prm[a], PB = prm[a2];
#pragma unroll
        for (int hb = 0; hb < HB; ++hb) {
          const int b = lane + 32 * hb;
          const bool up = b > a;
          const bool ok = b < half && (up || (b < a && a2 != a));
          const float4 PC = prm[up ? min(b, half - 1) : half - 1 - b];
          const float4 PR = up ? PA : PB;
          const int r1 = __float_as_int(PR.x) & 0xffff, r2 = __float_as_int(PR.y);
          const int c1 = __float_as_int(PC.x) & 0xffff, c2 = __float_as_int(PC.y);
          if (ok && !NYS_IDX_OK(r1 < r2 && r2 < N && c1 < c2 && c2 < N)) s_jbad = 1;
          else if (ok)
            f32_block(A, upk(r1, c1, ldf), upk(r1, c2, ldf), upk(r2, c1, ldf), upk(r2, c2, ldf),
                      PR.z, PR.w, PC.z, PC.w);
        }
      }
      // diagonal blocks (p, q) x (p, q): the same two-sided rotation; (q, p)
      // is the stored (p, q)
      if (warp == NW - 1) {
#pragma unroll
        for (int hb = 0; hb < HB; ++hb) {
          if (lane + 32 * hb < half) {
            const int ep = pp[hb] * ldf + pp[hb], eq = qq[hb] * ldf + qq[hb];
            const int e = pp[hb] * ldf + qq[hb];
            const float c = cc[hb], sn = ss[hb];
            const float x0 = A[ep], x1 = A[e], x3 = A[eq];
            const float y00 = c * x0 - sn * x1, y01 = sn * x0 + c * x1;
            const float y10 = c * x1 - sn * x3, y11 = sn * x1 + c * x3;
            A[ep] = c * y00 - sn * y10;
            A[e] = c * y01 - sn * y11;
            A[eq] = sn * y01 + c * y11;
          }
        }
      }
      // V <- V J (lanes past the pairs rotate copies of the last pair's slots,
      // never read), then the slot shift: first(b) <- first(b-1), first(1) <-
      // second(0), first(0) stays; second(b) <- second(b+1), second(half-1) <-
      // first(half-1)
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int hb = 0; hb < HB; ++hb) {
          const float f = vf[u][hb], g = vs[u][hb];
          vf[u][hb] = cc[hb] * f - se[hb] * g;
          vs[u][hb] = se[hb] * f + cc[hb] * g;
        }
      const int src_up = (lane + 31) & 31, src_dn = (lane + 1) & 31;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (HB == 1) {
          const float x = lane == 0 ? vs[u][0] : vf[u][0];
          const float up = __shfl_sync(0xffffffffu, x, src_up);
          const float dn = __shfl_sync(0xffffffffu, vs[u][0], src_dn);
          const float nf = lane == 0 ? vf[u][0] : up;
          const float ns = lane == half - 1 ? vf[u][0] : dn;
          vf[u][0] = nf;
          vs[u][0] = ns;
        } else {
          const float x0 = lane == 0 ? vs[u][0] : vf[u][0];
          const float r0 = __shfl_sync(0xffffffffu, x0, src_up);
          const float r1 = __shfl_sync(0xffffffffu, vf[u][HB - 1], src_up);
          const float d0 = __shfl_sync(0xffffffffu, vs[u][0], src_dn);
          const float d1 = __shfl_sync(0xffffffffu, vs[u][HB - 1], src_dn);
          const float nf0 = lane == 0 ? vf[u][0] : r0;
          const float nf1 = lane == 0 ? r0 : r1;
          float ns0 = lane == 31 ? d1 : d0;
          float ns1 = d1;
          if (lane == half - 1) ns0 = vf[u][0];
          if (lane + 32 == half - 1) ns1 = vf[u][HB - 1];
          vf[u][0] = nf0;
          vf[u][HB - 1] = nf1;
          vs[u][0] = ns0;
          vs[u][HB - 1] = ns1;
        }
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int hb = 0; hb < HB; ++hb) {
      const int i = warp + NW * u, b = lane + 32 * hb;
      if (i < m && b < half) {
        if (b < m) Vout[i * ldf + b] = vf[u][hb];
        if (N - 1 - b < m) Vout[i * ldf + N - 1 - b] = vs[u][hb];
      }
    }
  __syncthreads();
  return s_jbad ? -1 : 1;
}

// doubles of k_setup_eig's V area: m (m+1), or (N + m)(N + 1) floats for odd m
__host__ __device__ constexpr int eig_v_doubles(int m) { return m * (m + 1) + 2 * m + 2; }

// register rows of jacobi_f32 per warp for the CTA widths of k_setup_eig: the
// widths' FP32-route landmark classes (256: m <= 64, 512: m <= 83, 1024:
// m <= kMMax) bound N
template <int NT, int HB>
__host__ __device__ constexpr int f32_vrows() {
  return HB == 1 ? 64 / (NT / 32) : (NT == 512 ? 6 : 4);
}

// NT threads per CTA: 256 for the small landmark counts (several CTAs per SM),
// 512 / 1024 for the large ones, whose shared memory leaves room for 2 / 1 CTAs.
// kG: landmark counts above kMMax, whose matrices do not fit in shared memory,
// work in a global (L2-resident) area of their own, one CTA per listed set.
template <int NT, bool kG>
__global__ void __launch_bounds__(NT, NT == 256 ? 4 : (NT == 512 ? 2 : 1))
k_setup_eig(Lset* lsets, const int32_t* __restrict__ lm_idx, double* __restrict__ W_all,
            float* __restrict__ W32_all, double* __restrict__ lam_all, double tau, int allow_chol,
            int m_lo, int m_hi, BigSet big, const float* __restrict__ lag, int fb_only) {
  // the grid covers every slot; inactive slots (instances that share another
  // instance's set) return at once, so a captured graph stays valid when an
  // update changes which instances share
  const int L = kG ? big.ids[blockIdx.x] : blockIdx.x;
  const Lset S = lsets[L];
  // one launch per landmark-count class (m_lo, m_hi], each with shared memory
  // for its own largest m; fb_only: only the sets that k_setup_eig_f32 handed
  // over (m_eff = -1), by the FP64 Jacobi route
  if (!S.active || S.m <= m_lo || S.m > m_hi) return;
  if (fb_only && S.m_eff != -1) return;
  const int m = S.m;
  const int N = m + (m & 1);  // even player count; index m (if present) is a bye
  const int ld = m + 1;
  extern __shared__ __align__(16) double smem_eig[];
  double* sm = kG ? big.ws + (int64_t)blockIdx.x * big.stride : smem_eig;
  double* A = sm;
  double* V = A + m * ld;
  // V's area holds m x ld doubles, or the FP32 route's two N x (N+1) and
  // m x (N+1) float matrices (even size: cs stays 16-byte aligned)
  double* cs = V + eig_v_doubles(m);       // N/2 cosines then N/2 sines
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
  // FP32 route (mixed contexts): Jacobi sweeps in FP32 (jacobi_f32), then one
  // correction that makes W an exact whitening again: with W0 = D U^T from the
  // FP32 eigenpairs (D = Lambda^-1/2), M = W0 Omega W0^T = I + E and
  // W = (I - E/2) W0 satisfies W^T W = Omega^-1 up to O(E^2); its rows stay
  // nearly orthogonal, which the FP32 factor of the mixed path needs.  The
  // products U^T Omega U run in float-float on the FP32 pipe (Omega's entries
  // are the lag table's float-float b0, exact FP64 kernel values to 2^-48);
  // the diagonal of E in FP64; E's off-diagonal entries (of size ~1e-6) and
  // the correction E W0 in FP32, whose relative error leaves W exact to ~1e-13.
  // Used when lambda_min > 1e-5 lambda_max (nothing truncated) and |E| <= 1e-5;
  // otherwise the FP64 Jacobi below.
  if (!kG && !allow_chol && !fb_only) {
    const int ldf = N + 1;
    float2* Om = reinterpret_cast<float2*>(A);   // Omega, then T: m x ld float-float
    float* Af = reinterpret_cast<float*>(V);     // N x ldf, upper triangle; then G
    float* Vf = Af + N * ldf;                    // m x ldf
    const float* lagS = lag != nullptr ? lag + S.lag_off : nullptr;
    for (int e = tid; e < m * m; e += nt) {
      const int j = e / m, l = e % m;
      const int k = abs(idx[j] - idx[l]);
      float2 w = make_float2(0.f, 0.f);
      if (lagS != nullptr) {
        if (k <= S.K) w = make_float2(lagS[6 * k], lagS[6 * k + 1]);
      } else {
        const double d = (double)k * S.hs, x = exp(-d * d);
        w.x = (float)x;
        w.y = (float)(x - (double)w.x);
      }
      Om[j * ld + l] = w;
      if (j <= l) Af[j * ldf + l] = w.x;
    }
    if (N > m)
      for (int i = tid; i < N; i += nt) Af[i * ldf + m] = 0.f;
    __syncthreads();
    float4* prm = reinterpret_cast<float4*>(cs);
    float* redf = reinterpret_cast<float*>(red);
    // FP32 sweeps reach off(A)^2 ~ 1e-13 tot(A)^2; the correction absorbs the rest
    // two slot pairs per lane (N > 64) only on the 512- and 1024-thread CTAs
    // (the launcher sends the FP32 route's classes above m = 64 there)
    int jr = 0;
    if (N <= 64)
      jr = jacobi_f32<NT / 32, 1, f32_vrows<NT, 1>()>(Af, Vf, ldf, m, prm, redf, 1e-13,
                                                      kMaxSweeps, 1e-9);
    else if constexpr (NT >= 512)
      jr = jacobi_f32<NT / 32, 2, f32_vrows<NT, 2>()>(Af, Vf, ldf, m, prm, redf, 1e-13,
                                                      kMaxSweeps, 1e-9);
    if (jr < 0) {
      if (tid == 0) lsets[L].m_eff = kMeffBounds;
      return;
    }
    if (jr > 0) {
      sort_desc(Af, ldf, m, perm);
      if (tid == 0) {
        const double lmax = Af[perm[0] * ldf + perm[0]];
        const double lmin = Af[perm[m - 1] * ldf + perm[m - 1]];
        red[0] = (lmin > 1e-5 * lmax && lmin > 0.0) ? 1.0 : 0.0;
      }
      __syncthreads();
      const bool well = red[0] != 0.0;
      __syncthreads();
      if (well) {
        // D as float-float (hi, lo) in the rotation area
        float2* rsq = reinterpret_cast<float2*>(cs);
        for (int k = tid; k < m; k += nt) {
          const double l = Af[perm[k] * ldf + perm[k]];
          const double r = 1.0 / sqrt(l);
          const float h = (float)r;
          rsq[k] = make_float2(h, (float)(r - (double)h));
          lam_all[(int64_t)L * kMLarge + k] = l;
        }
        __syncthreads();
        // T = U^T Omega (U_ik = Vf[i][perm[k]]): float-float, by column blocks
        // of Omega, each overwritten by the same columns of T
        constexpr int kTE = 8;
        const int cw = max(1, (kTE * nt) / m);
        for (int j0 = 0; j0 < m; j0 += cw) {
          const int jn = min(cw, m - j0);
          float2 acc[kTE];
#pragma unroll
          for (int q = 0; q < kTE; ++q) {
            const int e = tid + q * nt;
            float sh = 0.f, sl = 0.f;
            if (e < m * jn) {
              const int k = e / jn, j = j0 + e % jn;
              const int c = perm[k];
              for (int i = 0; i < m; ++i) ff_fma(sh, sl, Vf[i * ldf + c], Om[i * ld + j]);
            }
            acc[q] = make_float2(sh, sl);
          }
          __syncthreads();
#pragma unroll
          for (int q = 0; q < kTE; ++q) {
            const int e = tid + q * nt;
            if (e < m * jn) {
              const float h = acc[q].x + acc[q].y;
              Om[(e / jn) * ld + j0 + e % jn] = make_float2(h, acc[q].y - (h - acc[q].x));
            }
          }
          __syncthreads();
        }
        // M = T U, E = D M D - I; G[k][perm[l]] = E_kl D_l (FP32) over Af
        float* G = Af;
        float emax = 0.f;
        for (int e = tid; e < m * m; e += nt) {
          const int k = e / m, l = e % m;
          const int c = perm[l];
          float sh = 0.f, sl = 0.f;
          for (int j = 0; j < m; ++j) ff_fma(sh, sl, Vf[j * ldf + c], Om[k * ld + j]);
          float E;
          if (k == l) {
            const double r = (double)rsq[k].x + (double)rsq[k].y;
            E = (float)(((double)sh + (double)sl) * r * r - 1.0);
          } else {
            E = (sh + sl) * rsq[k].x * rsq[l].x;
          }
          emax = fmaxf(emax, fabsf(E));
          G[k * m + c] = E * rsq[l].x;
        }
        emax = (float)block_max((double)emax, red);
        if (emax <= 1e-5f) {
          // W = W0 - (E W0) / 2, W0_kj = D_k U_jk (D_k U_jk as an exact
          // float-float product)
          for (int e = tid; e < m * m; e += nt) {
            const int k = e / m, j = e % m;
            float corr = 0.f;
            for (int c = 0; c < m; ++c) corr = fmaf(G[k * m + c], Vf[j * ldf + c], corr);
            const float u = Vf[j * ldf + perm[k]];
            const float2 r = rsq[k];
            const float ph = r.x * u;
            const float pl = fmaf(r.x, u, -ph) + r.y * u - 0.5f * corr;
            const double w = (double)ph + (double)pl;
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
    __syncthreads();
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

// MIXED route for the large landmark counts on a compact shared-memory area
// (two CTAs per SM where the FP64 fallback's area would hold one): Omega's
// upper triangle and V as in k_setup_eig's FP32 route, Omega's float-float
// entries read from the lag table by column blocks, T = U^T Omega kept in the
// set's W area (global, L2-resident; W overwrites it at the end) and read back
// by row blocks.  Sets the route cannot take (nothing truncated: lambda_min >
// 1e-5 lambda_max, |E| <= 1e-5; the lag table present) get m_eff = -1 and are
// factored by k_setup_eig's FP64 route in a second launch (fb_only).
constexpr int kF32Blk = 8;   // columns of Omega / rows of T staged per block
constexpr int kF32cThreads = 256;
__host__ __device__ inline size_t f32c_smem_bytes(int m) {
  const int N = m + (m & 1);
  return 4 * (size_t)(N + m) * (N + 1) + 16 + 8 * (size_t)kF32Blk * m + 16 + 8 * (size_t)(N + 32) +
         4 * (size_t)(2 * m);
}

template <int NT>
__global__ void __launch_bounds__(NT, 2)
k_setup_eig_f32(Lset* lsets, const int32_t* __restrict__ lm_idx, double* __restrict__ W_all,
                float* __restrict__ W32_all, double* __restrict__ lam_all, int m_lo, int m_hi,
                const float* __restrict__ lag) {
  const int L = blockIdx.x;
  const Lset S = lsets[L];
  if (!S.active || S.m <= m_lo || S.m > m_hi) return;
  const int m = S.m, N = m + (m & 1), ldf = N + 1, tid = threadIdx.x, nt = blockDim.x;
  extern __shared__ __align__(16) unsigned char f32c_raw[];
  float* Af = reinterpret_cast<float*>(f32c_raw);   // N x ldf, upper triangle; then G (m x m)
  float* Vf = Af + N * ldf;                          // m x ldf
  // (N + m)(N + 1) floats end on a 4-byte boundary for odd m: align the float2 scratch
  float2* scr = reinterpret_cast<float2*>(
      (reinterpret_cast<uintptr_t>(Vf + m * ldf) + 15) & ~static_cast<uintptr_t>(15));   // kF32Blk x m
  double* cs = reinterpret_cast<double*>(
      (reinterpret_cast<uintptr_t>(scr + kF32Blk * m) + 15) & ~static_cast<uintptr_t>(15));
  double* red = cs + N;
  int* perm = reinterpret_cast<int*>(red + 32);
  int* idx = perm + m;
  for (int j = tid; j < m; j += nt) idx[j] = lm_idx[S.lm_off + j];
  __syncthreads();
  double* Wl = W_all + S.w_off;
  float* W32l = W32_all + S.w_off;
  const float* lagS = lag + S.lag_off;
  auto omega = [&](int j, int l) -> float2 {
    const int k = abs(idx[j] - idx[l]);
    return k <= S.K ? make_float2(lagS[6 * k], lagS[6 * k + 1]) : make_float2(0.f, 0.f);
  };
  bool done = false;
  if (lag != nullptr) {
    for (int e = tid; e < m * m; e += nt) {
      const int j = e / m, l = e % m;
      if (j <= l) Af[j * ldf + l] = omega(j, l).x;
    }
    if (N > m)
      for (int i = tid; i < N; i += nt) Af[i * ldf + m] = 0.f;
    __syncthreads();
    float4* prm = reinterpret_cast<float4*>(cs);
    float* redf = reinterpret_cast<float*>(red);
    int jr = 0;
    if (N <= 64)
      jr = jacobi_f32<NT / 32, 1, (64 + NT / 32 - 1) / (NT / 32)>(Af, Vf, ldf, m, prm, redf,
                                                                  1e-13, kMaxSweeps, 1e-9);
    else
      jr = jacobi_f32<NT / 32, 2, (kMMax + (kMMax & 1) + NT / 32 - 1) / (NT / 32)>(
          Af, Vf, ldf, m, prm, redf, 1e-13, kMaxSweeps, 1e-9);
    if (jr < 0) {
      if (tid == 0) lsets[L].m_eff = kMeffBounds;
      return;
    }
    if (jr > 0) {
      sort_desc(Af, ldf, m, perm);
      if (tid == 0) {
        const double lmax = Af[perm[0] * ldf + perm[0]];
        const double lmin = Af[perm[m - 1] * ldf + perm[m - 1]];
        red[0] = (lmin > 1e-5 * lmax && lmin > 0.0) ? 1.0 : 0.0;
      }
      __syncthreads();
      const bool well = red[0] != 0.0;
      __syncthreads();
      if (well) {
        float2* rsq = reinterpret_cast<float2*>(cs);
        for (int k = tid; k < m; k += nt) {
          const double l = Af[perm[k] * ldf + perm[k]];
          const double r = 1.0 / sqrt(l);
          const float h = (float)r;
          rsq[k] = make_float2(h, (float)(r - (double)h));
          lam_all[(int64_t)L * kMLarge + k] = l;
        }
        __syncthreads();
        // T = U^T Omega in float-float, by blocks of Omega's columns staged from
        // the lag table, into the W area (m x m float2)
        float2* Tg = reinterpret_cast<float2*>(Wl);
        for (int j0 = 0; j0 < m; j0 += kF32Blk) {
          const int jn = min(kF32Blk, m - j0);
          for (int e = tid; e < m * jn; e += nt) scr[e] = omega(e / jn, j0 + e % jn);
          __syncthreads();
          for (int e = tid; e < m * jn; e += nt) {
            const int k = e / jn, jj = e % jn;
            const int c = perm[k];
            float sh = 0.f, sl = 0.f;
            for (int i = 0; i < m; ++i) ff_fma(sh, sl, Vf[i * ldf + c], scr[i * jn + jj]);
            const float h = sh + sl;
            Tg[k * m + j0 + jj] = make_float2(h, sl - (h - sh));
          }
          __syncthreads();
        }
        // M = T U by blocks of T's rows, E = D M D - I; G[k][perm[l]] = E_kl D_l
        float* G = Af;
        float emax = 0.f;
        for (int k0 = 0; k0 < m; k0 += kF32Blk) {
          const int kn = min(kF32Blk, m - k0);
          for (int e = tid; e < kn * m; e += nt) scr[e] = Tg[k0 * m + e];
          __syncthreads();
          for (int e = tid; e < kn * m; e += nt) {
            const int kk = e / m, l = e % m, k = k0 + kk;
            const int c = perm[l];
            float sh = 0.f, sl = 0.f;
            for (int j = 0; j < m; ++j) ff_fma(sh, sl, Vf[j * ldf + c], scr[kk * m + j]);
            float E;
            if (k == l) {
              const double r = (double)rsq[k].x + (double)rsq[k].y;
              E = (float)(((double)sh + (double)sl) * r * r - 1.0);
            } else {
              E = (sh + sl) * rsq[k].x * rsq[l].x;
            }
            emax = fmaxf(emax, fabsf(E));
            G[k * m + c] = E * rsq[l].x;
          }
          __syncthreads();
        }
        emax = (float)block_max((double)emax, red);
        if (emax <= 1e-5f) {
          for (int e = tid; e < m * m; e += nt) {
            const int k = e / m, j = e % m;
            float corr = 0.f;
            for (int c = 0; c < m; ++c) corr = fmaf(G[k * m + c], Vf[j * ldf + c], corr);
            const float u = Vf[j * ldf + perm[k]];
            const float2 r = rsq[k];
            const float ph = r.x * u;
            const float pl = fmaf(r.x, u, -ph) + r.y * u - 0.5f * corr;
            const double w = (double)ph + (double)pl;
            Wl[e] = w;
            W32l[e] = (float)w;
          }
          done = true;
        }
      }
    }
  }
  if (tid == 0) {
    lsets[L].m_eff = done ? m : -1;
    if (done) lsets[L].omode = 0;
  }
}

size_t setup_smem_bytes(int m) {
  const int N = m + (m & 1);
  return sizeof(double) * ((size_t)m * (m + 1) + eig_v_doubles(m) + N + 32) +
         sizeof(int) * (N + 2 * m);
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
                                    int hi, cudaStream_t st, const float* lag, int fb_only = 0) {
  const size_t sm = setup_smem_bytes(hi);
  cudaError_t e = cudaFuncSetAttribute(k_setup_eig<NT, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_setup_eig<NT, false><<<capacity, NT, sm, st>>>(lsets, lm_idx, W, W32, lam, tau, allow_chol, lo,
                                                   hi, BigSet(), lag, fb_only);
  return cudaGetLastError();
}

size_t setup_ws_doubles() { return setup_smem_bytes(kMLarge) / sizeof(double) + 1; }

static cudaError_t launch_eig_sets(Lset* lsets, int capacity, const int32_t* lm_idx, double* W,
                                   float* W32, double* lam, double tau, int m_max, cudaStream_t st,
                                   int allow_chol, const int* m_bounds, int nclass, BigSet big,
                                   int few_sets, const float* lag);

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
                       const Inst* insts, int few_sets, const float* lag) {
  if (capacity == 0) return cudaSuccess;
  cudaError_t ec = launch_eig_sets(lsets, capacity, lm_idx, W, W32, lam, tau, m_max, st, allow_chol,
                                   m_bounds, nclass, big, few_sets, lag);
  if (ec != cudaSuccess || crow == nullptr || insts == nullptr) return ec;
  k_setup_crow<<<capacity, 128, 0, st>>>(insts, lsets, lm_idx, W, crow, m_max);
  return cudaGetLastError();
}

static cudaError_t launch_eig_sets(Lset* lsets, int capacity, const int32_t* lm_idx, double* W,
                                   float* W32, double* lam, double tau, int m_max, cudaStream_t st,
                                   int allow_chol, const int* m_bounds, int nclass, BigSet big,
                                   int few_sets, const float* lag) {
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
    if (!allow_chol && lag != nullptr && sm > 113 * 1024 && f32c_smem_bytes(hi) <= 113 * 1024) {
      // MIXED, large m: the compact FP32 route two CTAs per SM, then the FP64
      // route for the sets it hands over (m_eff = -1; none when it succeeds)
      const size_t sc = f32c_smem_bytes(hi);
      e = cudaFuncSetAttribute(k_setup_eig_f32<kF32cThreads>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sc);
      if (e == cudaSuccess) {
        k_setup_eig_f32<kF32cThreads><<<capacity, kF32cThreads, sc, st>>>(lsets, lm_idx, W, W32, lam,
                                                                          lo, hi, lag);
        e = cudaGetLastError();
      }
      if (e == cudaSuccess)
        e = launch_eig_class<1024>(lsets, capacity, lm_idx, W, W32, lam, tau, allow_chol, lo, hi,
                                   st, lag, 1);
    } else if (few_sets && !allow_chol && sm <= 113 * 1024)
      e = launch_eig_class<512>(lsets, capacity, lm_idx, W, W32, lam, tau, allow_chol, lo, hi, st, lag);
    else if (sm > 113 * 1024)
      e = launch_eig_class<1024>(lsets, capacity, lm_idx, W, W32, lam, tau, allow_chol, lo, hi, st, lag);
    else if (sm > 75 * 1024 || (!allow_chol && hi > 64))
      e = launch_eig_class<512>(lsets, capacity, lm_idx, W, W32, lam, tau, allow_chol, lo, hi, st, lag);
    else
      e = launch_eig_class<256>(lsets, capacity, lm_idx, W, W32, lam, tau, allow_chol, lo, hi, st, lag);
    if (e != cudaSuccess) return e;
    lo = hi;
  }
  if (big.n > 0) {   // landmark counts above kMMax: global workspace
    k_setup_eig<1024, true><<<big.n, 1024, 0, st>>>(lsets, lm_idx, W, W32, lam, tau, allow_chol,
                                                     kMMax, kMLarge, big, nullptr, 0);
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
                    nclass, big, crow, insts, few_sets, lag);
}

}  // namespace nys
