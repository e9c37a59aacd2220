// Model evaluation y^(d)(t) = omega^T phi^(d)(t) + b [d == 0] (Section 3), done in
// kernel coordinates: omega^T W k^(d)(t) = z^T k^(d)(t) with z = W^T omega.
#include "nys_internal.cuh"

namespace nys {

__global__ void __launch_bounds__(128)
k_eval(const Inst* __restrict__ insts, const double* __restrict__ zs, int ZS,
       const int32_t* __restrict__ lm_idx, const double* __restrict__ tq,
       const int64_t* __restrict__ tq_off, int deriv, double* __restrict__ yq) {
  const int b = blockIdx.x;
  const Inst I = insts[b];
  const int m = I.m;
  __shared__ double s_z[kMLarge + 1];
  __shared__ double s_s[kMLarge];
  for (int j = threadIdx.x; j <= m; j += blockDim.x) s_z[j] = zs[(int64_t)b * ZS + j];
  for (int j = threadIdx.x; j < m; j += blockDim.x) s_s[j] = I.t0 + (double)lm_idx[I.lm_off + j] * I.h;
  __syncthreads();
  const double is = 1.0 / I.sigma;
  for (int64_t q = tq_off[b] + threadIdx.x; q < tq_off[b + 1]; q += blockDim.x) {
    const double t = tq[q];
    double acc = (deriv == 0) ? s_z[m] : 0.0;
    for (int j = 0; j < m; ++j) {
      const double x = (t - s_s[j]) * is;
      const double e = exp(-x * x);
      double k;
      if (deriv == 0) k = e;
      else if (deriv == 1) k = -2.0 * x * is * e;
      else k = (4.0 * x * x - 2.0) * is * is * e;
      acc = fma(s_z[j], k, acc);
    }
    yq[q] = acc;
  }
}

cudaError_t launch_eval(const Inst* insts, const double* zs, int ZS, const int32_t* lm,
                        const double* tq, const int64_t* tq_off, int deriv, double* yq, int batch,
                        cudaStream_t s) {
  k_eval<<<batch, 128, 0, s>>>(insts, zs, ZS, lm, tq, tq_off, deriv, yq);
  return cudaGetLastError();
}

}  // namespace nys
