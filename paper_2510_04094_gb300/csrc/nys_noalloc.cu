// Allocation-free FP64 solve of a small batch of linear instances.
//
// For callers that cannot call cudaMalloc: processes whose device memory is
// reserved up front by another allocator (a framework's caching pool, a
// fixed-budget server), or latency-critical code where a device allocation
// (which may synchronise the device) is not acceptable.  The computation is
// the one of nys_setup + nys_assemble + nys_solve with precision FP64: the same
// Nystrom setup, fused row-pass and solve kernels, but every workspace --
// descriptors, the Nystrom factor, the per-chunk partial Gram sums of the row
// pass (its scratch), the factorisation -- is carved out of one file-scope
// static device array of NYS_NOALLOC_SCRATCH_BYTES bytes.  Every GPU that
// loads the library holds that array until the process exits.
//
// Sharing: all calls on a device use the same array and it keeps the last
// call's contents; what must start at zero (the row-pass work counter) is
// cleared by each call.  Calls whose GPU work overlaps (two streams, or two
// host threads) race on the array: serialise them.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "nys_internal.cuh"

namespace nys {
cudaError_t launch_setup(Lset* lsets, int capacity, const int32_t* lm_idx, double* W, float* W32,
                         double* lam, float* lag, double tau, int m_max, cudaStream_t st,
                         int allow_chol, const int* m_bounds, int nclass,
                         BigSet big = BigSet(), double* crow = nullptr,
                         const Inst* insts = nullptr, int few_sets = 0);
cudaError_t launch_assemble(bool fp32, const Inst* insts, const Lset* lsets, const float* lag,
                            const double* W, const Work* work, int nwork, int* counter,
                            const int32_t* lm, const double* tab, double* part,
                            const int64_t* slot_off, int m_max, int k_max, int num_sms,
                            cudaStream_t st, int asm_kind, int32_t* err,
                            BigSet big = BigSet(), int tc_wait = -1, int nband = 0);
cudaError_t launch_solve(bool fp32, const Inst* insts, const Lset* lsets, const double* W,
                         const float* W32, const double* part, const int64_t* slot_off,
                         const int32_t* lm, void* fac, int64_t facs, double* xs, double* zs,
                         double* cws, int XS, int ZS, int M1S, const int32_t* st_init,
                         int32_t* st, double gamma_scale, int batch, int m_max, cudaStream_t s,
                         const int32_t* asm_err, BigSet big = BigSet(), const double* crow = nullptr,
                         bool fac64 = false);
int64_t fac_elems(int m_max);
int32_t set_last_error(int32_t code, const char* msg);  // nys_api.cu: feeds nys_last_error()
}  // namespace nys

using namespace nys;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NYS_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
constexpr int kChunks = NYS_NOALLOC_MAX_CHUNKS;
std::mutex g_mu;
void* g_base[kMaxDevices];
int g_sms[kMaxDevices];

int32_t err(int32_t code, const char* msg) { return set_last_error(code, msg); }

// Device address of the static array (host code cannot use the symbol itself).
// Looked up once per device, with that device current.
int32_t scratch_base(void** base, int* sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return err(NYS_ECUDA, "nys_solve_noalloc: no current CUDA device");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_base[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return err(NYS_ECUDA, "nys_solve_noalloc: cudaGetSymbolAddress failed");
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return err(NYS_ECUDA, "nys_solve_noalloc: device query failed");
    g_base[dev] = p;
    g_sms[dev] = n;
  }
  *base = g_base[dev];
  *sms = g_sms[dev];
  return NYS_OK;
}

size_t carve(size_t& off, size_t bytes) {
  const size_t at = (off + 255) & ~size_t(255);
  off = at + bytes;
  return at;
}
}  // namespace

extern "C" int32_t nys_solve_noalloc(const nys_instance* q, int32_t batch, double* x_out,
                                     int32_t* status_out, void* stream) {
  if (!q || !x_out || !status_out) return err(NYS_EINVAL, "nys_solve_noalloc: NULL argument");
  if (batch < 1 || batch > NYS_NOALLOC_MAX_BATCH)
    return err(NYS_EINVAL, "nys_solve_noalloc: batch must be in [1, NYS_NOALLOC_MAX_BATCH]");
  int m_max = 2;
  for (int b = 0; b < batch; ++b) {
    const nys_instance& s = q[b];
    if (s.kind != NYS_COEF_LIN) return err(NYS_EINVAL, "nys_solve_noalloc: kind must be NYS_COEF_LIN");
    if (s.p != 1 && s.p != 2) return err(NYS_EINVAL, "nys_solve_noalloc: p must be 1 or 2");
    if (s.m < 2 || s.m > NYS_NOALLOC_MAX_M || s.n < 3 || s.m > s.n || s.n > NYS_NOALLOC_MAX_N)
      return err(NYS_EINVAL, "nys_solve_noalloc: need 2 <= m <= min(n, NYS_NOALLOC_MAX_M), "
                             "3 <= n <= NYS_NOALLOC_MAX_N");
    if (!(s.t1 > s.t0) || !(s.sigma > 0) || !(s.gamma > 0))
      return err(NYS_EINVAL, "nys_solve_noalloc: need t1 > t0, sigma > 0, gamma > 0");
    if ((s.bc != NYS_BC_IVP && s.bc != NYS_BC_BVP) || s.reserved != 0 || (s.bc == NYS_BC_BVP && s.p != 2))
      return err(NYS_EINVAL, "nys_solve_noalloc: bc must be NYS_BC_IVP, or NYS_BC_BVP with p = 2");
    if (s.m > m_max) m_max = s.m;
  }
  void* base = nullptr;
  int sms = 0;
  int32_t r = scratch_base(&base, &sms);
  if (r != NYS_OK) return r;
  cudaStream_t st = (cudaStream_t)stream;

  // host descriptors on the stack (nothing is allocated)
  Inst inst[NYS_NOALLOC_MAX_BATCH];
  Lset lset[NYS_NOALLOC_MAX_BATCH];
  int32_t lm[NYS_NOALLOC_MAX_BATCH * NYS_NOALLOC_MAX_M];
  Work work[NYS_NOALLOC_MAX_BATCH * kChunks];
  int64_t soff[NYS_NOALLOC_MAX_BATCH * kChunks];
  int32_t stinit[NYS_NOALLOC_MAX_BATCH + 1];
  int nwork = 0, nl = 0;
  int64_t poff = 0;
  for (int b = 0; b < batch; ++b) {
    const nys_instance& s = q[b];
    Inst& I = inst[b];
    I = Inst{};
    I.p = s.p; I.n = s.n; I.m = s.m; I.kind = s.kind;
    I.bc = s.bc;
    I.lm_off = (int64_t)b * NYS_NOALLOC_MAX_M;
    I.tab_off = -1;
    I.t0 = s.t0;
    I.h = (s.t1 - s.t0) / (double)(s.n - 1);
    I.sigma = s.sigma;
    I.gamma = s.gamma;
    I.v[0] = s.v[0];
    I.v[1] = (s.p == 2) ? s.v[1] : 0.0;
    I.v[2] = I.v[3] = 0.0;
    bool fin = std::isfinite(s.v[0]) && std::isfinite(I.v[1]);
    for (int k = 0; k < 8; ++k) {
      I.c[k] = s.c[k];
      fin = fin && std::isfinite(s.c[k]);
    }
    if (s.p == 1) I.c[1] = 0.0;
    I.hs = I.h / s.sigma;
    const double tp = 6.283185307179586476925286766559;
    I.th0 = std::remainder(s.c[3] * s.t0 + s.c[4], tp);
    I.dth = std::remainder(s.c[3] * I.h, tp);
    stinit[b] = fin ? NYS_OK : NYS_ENONFINITE;
    int32_t* li = lm + I.lm_off;
    for (int j = 0; j < s.m; ++j) {
      li[j] = s.landmarks ? s.landmarks[j]
                          : (int32_t)(((int64_t)j * (s.n - 1) + (s.m - 1) / 2) / (s.m - 1));
      if (li[j] < 0 || li[j] >= s.n || (j > 0 && li[j] <= li[j - 1]))
        return err(NYS_EINVAL, "nys_solve_noalloc: landmarks must be increasing indices in [0, n)");
    }
    // one Nystrom factor per instance (no de-duplication here)
    Lset& L = lset[nl];
    L = Lset{};
    L.m = s.m;
    L.m_eff = s.m;
    L.n = s.n;
    L.active = 1;   // no lag tables on this path (FP64 features are computed directly)
    L.lm_off = I.lm_off;
    L.w_off = (int64_t)nl * m_max * m_max;
    L.hs = I.hs;
    I.lset = nl++;
    const int nrows = s.n - 1 - (s.bc == NYS_BC_BVP ? 1 : 0);   // rows 2..n (2..n-1)
    const int chunks = nrows < 64 * kChunks ? 1 : kChunks;
    const int64_t E = (int64_t)(s.m + 2) * (s.m + 3) / 2 + 2;   // + [first landmark, count]
    I.slot_begin = nwork;
    I.slot_count = chunks;
    for (int k = 0; k < chunks; ++k) {
      Work& w = work[nwork];
      w.inst = b;
      w.r0 = 1 + (int)((int64_t)nrows * k / chunks);
      w.r1 = 1 + (int)((int64_t)nrows * (k + 1) / chunks);
      w.slot = nwork;
      w.e0 = 0;
      w.e1 = INT32_MAX;
      soff[nwork++] = poff;
      poff += E;
    }
  }
  stinit[batch] = nl;
  const int XS = m_max + 3, ZS = m_max + 1, M1S = m_max + 1;
  const int64_t facs = fac_elems(m_max);

  // carve the static array
  size_t off = 0;
  unsigned char* B = static_cast<unsigned char*>(base);
  const size_t o_inst = carve(off, sizeof(Inst) * batch);
  const size_t o_lset = carve(off, sizeof(Lset) * nl);
  const size_t o_lm = carve(off, sizeof(int32_t) * batch * NYS_NOALLOC_MAX_M);
  const size_t o_work = carve(off, sizeof(Work) * nwork);
  const size_t o_soff = carve(off, sizeof(int64_t) * nwork);
  const size_t o_st = carve(off, sizeof(int32_t) * (batch + 1));
  const size_t o_cnt = carve(off, sizeof(int32_t));
  const size_t o_part = carve(off, sizeof(double) * poff);
  const size_t o_W = carve(off, sizeof(double) * nl * m_max * m_max);
  const size_t o_W32 = carve(off, sizeof(float) * nl * m_max * m_max);
  const size_t o_lam = carve(off, sizeof(double) * nl * NYS_M_MAX);
  const size_t o_fac = carve(off, sizeof(double) * batch * facs);
  const size_t o_zs = carve(off, sizeof(double) * batch * ZS);
  const size_t o_cws = carve(off, sizeof(double) * batch * 2 * M1S);
  if (off > (size_t)NYS_NOALLOC_SCRATCH_BYTES)
    return err(NYS_EINVAL, "nys_solve_noalloc: workspace exceeds NYS_NOALLOC_SCRATCH_BYTES");

#define NA_CK(call)                                                               \
  do {                                                                            \
    if ((call) != cudaSuccess) return err(NYS_ECUDA, "nys_solve_noalloc: " #call); \
  } while (0)
  // descriptors: host stack -> static array (pageable source, staged before return)
  NA_CK(cudaMemcpyAsync(B + o_inst, inst, sizeof(Inst) * batch, cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(B + o_lset, lset, sizeof(Lset) * nl, cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(B + o_lm, lm, sizeof(int32_t) * batch * NYS_NOALLOC_MAX_M,
                        cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(B + o_work, work, sizeof(Work) * nwork, cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(B + o_soff, soff, sizeof(int64_t) * nwork, cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(B + o_st, stinit, sizeof(int32_t) * (batch + 1), cudaMemcpyHostToDevice, st));
  // pageable sources may still be read by an in-flight copy after return: wait
  NA_CK(cudaStreamSynchronize(st));
  Inst* d_inst = reinterpret_cast<Inst*>(B + o_inst);
  Lset* d_lset = reinterpret_cast<Lset*>(B + o_lset);
  const int32_t* d_lm = reinterpret_cast<const int32_t*>(B + o_lm);
  const int32_t* d_stinit = reinterpret_cast<const int32_t*>(B + o_st);
  NA_CK(launch_setup(d_lset, nl, d_lm, reinterpret_cast<double*>(B + o_W),
                     reinterpret_cast<float*>(B + o_W32), reinterpret_cast<double*>(B + o_lam),
                     nullptr, 1e-12, m_max, st, 1, nullptr, 0));
  // the work counter is cleared inside launch_assemble before the kernel
  NA_CK(launch_assemble(false, d_inst, d_lset, nullptr, reinterpret_cast<const double*>(B + o_W),
                        reinterpret_cast<const Work*>(B + o_work),
                        nwork, reinterpret_cast<int*>(B + o_cnt), d_lm, nullptr,
                        reinterpret_cast<double*>(B + o_part),
                        reinterpret_cast<const int64_t*>(B + o_soff), m_max, 0, sms, st, 1,
                        nullptr));
  NA_CK(launch_solve(false, d_inst, d_lset, reinterpret_cast<const double*>(B + o_W),
                     reinterpret_cast<const float*>(B + o_W32),
                     reinterpret_cast<const double*>(B + o_part),
                     reinterpret_cast<const int64_t*>(B + o_soff), d_lm, B + o_fac, facs, x_out,
                     reinterpret_cast<double*>(B + o_zs), reinterpret_cast<double*>(B + o_cws), XS,
                     ZS, M1S, d_stinit, status_out, 1.0, batch, m_max, st, nullptr));
#undef NA_CK
  return NYS_OK;
}
