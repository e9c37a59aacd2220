// Host side of the C ABI declared in include/nys.h: argument validation,
// descriptor packing, landmark-set de-duplication, row-pass work lists,
// device workspaces, kernel launches and CUDA-graph capture.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "nys_internal.cuh"

namespace nys {
// kernel launchers (defined in the other translation units)
cudaError_t launch_setup(Lset* lsets, int capacity, const int32_t* lm_idx, double* W, float* W32,
                         double* lam, float* lag, double tau, int m_max, cudaStream_t st,
                         int allow_chol, const int* m_bounds, int nclass,
                         BigSet big = BigSet(), double* crow = nullptr,
                         const Inst* insts = nullptr, int few_sets = 0);
cudaError_t launch_lag(const Lset* lsets, int capacity, float* lag, cudaStream_t st);
cudaError_t launch_eig(Lset* lsets, int capacity, const int32_t* lm_idx, double* W, float* W32,
                       double* lam, double tau, int m_max, cudaStream_t st, int allow_chol,
                       const int* m_bounds, int nclass, BigSet big = BigSet(), double* crow = nullptr,
                       const Inst* insts = nullptr, int few_sets = 0, const float* lag = nullptr);
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
cudaError_t launch_refine(const Inst* insts, const Lset* lsets, const double* W, const float* lag,
                          const Work* work, int nwork, int* counter, const int32_t* lm,
                          const double* tab,
                          double* part, const int64_t* slot_off, const void* fac, int64_t facs,
                          double* xs, double* zs, const double* cws, int XS, int ZS, int M1S,
                          int32_t* st, double gamma_scale, int batch, int m_max, int k_max,
                          int num_sms, cudaStream_t s, int nrband, bool fac64, double* rcorr,
                          int pass, bool last, const int32_t* skip_in, int32_t* skip_out);
cudaError_t launch_eval(const Inst* insts, const double* zs, int ZS, const int32_t* lm,
                        const double* tq, const int64_t* tq_off, int deriv, double* yq, int batch,
                        cudaStream_t s);

int64_t fac_elems(int m_max);
int64_t asm_tc_unit_rows(int64_t total_rows, int batch, int num_sms);
size_t setup_ws_doubles();
size_t solve_ws_doubles();
size_t grad_adj_stride(int ZS);
cudaError_t launch_grad(const Inst* insts, const Lset* lsets, const double* W, const double* fac,
                        int64_t facs, const double* xs, const double* zs, const int32_t* lm, int XS,
                        int ZS, const int32_t* st, const double* obs_t, const int64_t* obs_off,
                        const double* dl_dy, double* adj, const Work* rwork, int nrwork,
                        int* counter, double* part, const int64_t* slot_off, double* grad_out,
                        double gamma_scale, int batch, int num_sms, cudaStream_t s);
cudaError_t launch_newton_init(const Inst* insts, const Lset* lsets, const double* W,
                               const int32_t* lm, const double* warm, double* xs, double* zs,
                               double* dzs, double* yaux, double* nrm, int32_t* iters,
                               int32_t* active, int32_t* st, const int32_t* st_init, int XS, int ZS,
                               int batch, int32_t* live, cudaStream_t s);
cudaError_t launch_newton_pass(const Inst* insts, const Lset* lsets, const double* W,
                               const Work* work, int nwork, int* counter, const int32_t* lm,
                               const double* xs, int XS, const double* zs, const double* dzs, int ZS,
                               double* yaux, double* rowstate, double* part,
                               const int64_t* slot_off, const int32_t* active, int mode,
                               int apply_dy, int m_max, int tiles, int num_sms, cudaStream_t s,
                               const int32_t* live);
cudaError_t launch_newton_step(const Inst* insts, const Lset* lsets, const double* W,
                               const double* part, const int64_t* slot_off, const int32_t* lm,
                               double* xs, double* zs, double* dzs, double* cws, int XS, int ZS,
                               int M1S, int32_t* st, int32_t* active, int32_t* iters, double* nrm,
                               int max_iter, double tol, int32_t* flags, int mode, int batch,
                               int m_max, cudaStream_t s, int32_t* live);
}  // namespace nys

using namespace nys;

// ---------------------------------------------------------------------------
static thread_local std::string g_err;
static int32_t fail(int32_t code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}
namespace nys {
// lets other translation units report through nys_last_error()
int32_t set_last_error(int32_t code, const char* msg) {
  g_err = msg;
  return code;
}
}  // namespace nys

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(NYS_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),     \
                  __FILE__, __LINE__);                                                   \
  } while (0)

template <typename T>
struct DBuf {  // owning device buffer
  T* p = nullptr;
  size_t n = 0;
  cudaError_t alloc(size_t count) {
    n = count;
    if (count == 0) return cudaSuccess;
    return cudaMalloc(reinterpret_cast<void**>(&p), count * sizeof(T));
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() { release(); }   // every buffer of a context goes with it
};

struct GraphKey {
  double* x;
  int32_t* st;
  cudaGraphExec_t exec;
};

// a captured nys_newton: its arguments and the graph
struct NewtonGraph {
  int32_t max_iter;
  double tol;
  const double* warm;
  double *x, *y;
  int32_t *it, *st;
  cudaGraphExec_t exec;
};

struct nys_ctx {
  int batch = 0, m_max = 0, p_max = 0, num_sms = 0, nwork = 0, nrwork = 0, nlset = 0;
  int XS = 0, ZS = 0, M1S = 0;
  int64_t facs = 0;
  nys_options opt{};
  bool fp32 = false;           // FP32 assembly (NYS_MIXED, NYS_MIXED_F64F)
  bool fac64 = false;          // NYS_MIXED_F64F: FP64 H and Cholesky factor
  bool any_nl = false, any_lin = false;
  int nt_tiles = 4;            // shared tiles of the Newton row pass (6 with a beta term)
  bool solved = false, assembled = false;
  std::vector<nys_instance> shape;        // p, n, m, kind per instance (for update checks)
  std::vector<uint8_t> lm_dflt;           // 1: instance b's landmarks are default_landmarks(n, m)
  std::vector<int32_t> h_lm;               // landmark indices (host)
  std::vector<int64_t> h_lm_off;
  std::vector<Inst> h_inst;
  std::vector<Lset> h_lset;
  std::vector<int32_t> h_stinit;
  std::vector<double> h_tab;
  std::vector<int64_t> h_lagcap;           // lag-table offset of slot b (floats)
  int64_t total_rows = 0;
  int64_t lag_floats = 0;
  int64_t rpi = 0;                // rows per work item of the CUDA-core / FP64 row passes
  int64_t tc_rpi = 0;             // rows per work unit of the tensor-core assembly
  int64_t asm_rows = 0;           // rows per item of the assembly work list in use
  int tc_wait = -1;               // polls per bounded wait of the tensor-core kernel (-1: default)
  int asm_slots = 0;              // assembly slot region (capacity) in slot_off / part
  int64_t asm_elems = 0;          // its doubles in part
  int nband = 0;                  // leading items of the work list for the band kernel
  std::vector<Work> h_rwork;      // refinement work list as built at setup (cost order)
  std::vector<int> rband_w;       // refinement band plan per instance: window rows (0: k_refine_rows)
  int nrband = 0;                 // leading items of the refinement list for k_refine_band
  std::vector<int> band_w;        // band plan per instance: window rows (0: tensor cores), unit
  std::vector<int> band_u;        // rows (the layout uses it unless the slot region is too small)
  bool tune_pending = false;      // NYS_ASM_TUNE: choose kernel and item size at first use
  std::vector<int> eig_bounds;    // landmark-count classes of the setup launches
  int k_max = 0;                  // largest lag-table length of the current sets
  // device
  DBuf<Inst> inst;
  DBuf<Lset> lset;
  DBuf<int32_t> lm;
  DBuf<double> tab;
  DBuf<Work> work, rwork;
  DBuf<int64_t> slot_off;   // assembly slots first, then refinement slots
  DBuf<double> part;
  DBuf<double> W;
  DBuf<float> W32;
  DBuf<float> lag;
  DBuf<double> lam;
  DBuf<double> crow;        // condition rows per landmark set (k_setup_crow): batch x 8 x m_max
  DBuf<unsigned char> fac;
  // instances with m > kMMax: ids and their global factor / solve workspace
  DBuf<int32_t> big_ids;
  DBuf<double> big_ws;
  int nbig = 0;
  int64_t big_stride = 0;
  BigSet bigset() const {
    BigSet g;
    g.ids = big_ids.p;
    g.n = nbig;
    g.ws = big_ws.p;
    g.stride = big_stride;
    return g;
  }
  DBuf<double> xs, zs, dzs, cws;
  DBuf<double> rcorr;       // MIXED: each instance's last relative refinement correction
  DBuf<int32_t> rskip;      // MIXED, default refinement: 1 = the instance skips the adaptive pass
  int refine_adapt = 0;     // default refinement: one adaptive pass after opt.refine_steps
  DBuf<int32_t> st, stinit, counter, err;
  // Newton state
  DBuf<double> yaux, rowstate, nrm;
  DBuf<int64_t> row_off;
  DBuf<int32_t> active, iters, any_active, live;
  // gradient scratch
  DBuf<double> adj;
  // pinned staging for descriptor uploads
  Inst* pin_inst = nullptr;
  Lset* pin_lset = nullptr;
  int32_t* pin_st = nullptr;   // batch + 1 entries: statuses, then the set count
  int32_t* pin_flag = nullptr;
  cudaEvent_t staged = nullptr;
  std::vector<GraphKey> graphs;
  std::vector<NewtonGraph> ngraphs;
  bool factor_stale = true;
  bool join_pending = false;     // factor running on the side stream
  int64_t upload_bytes = 0;
  cudaStream_t side = nullptr;   // runs the Nystrom setup beside the row pass
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

static bool finite_all(const double* a, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

static double mod2pi(double x) {
  const double tp = 6.283185307179586476925286766559;
  double r = std::fmod(x, tp);
  if (r > M_PI) r -= tp;
  if (r < -M_PI) r += tp;
  return r;
}

// Validate one instance.  Returns NYS_OK, NYS_EINVAL (message set) or
// NYS_ENONFINITE (non-finite coefficient data: the instance is skipped).
static int32_t check_instance(const nys_instance& q, int b) {
  if (q.p < 1 || q.p > 4) return fail(NYS_EINVAL, "instance %d: p must be in 1..4 (got %d)", b, q.p);
  if (q.p > 2 && q.kind != NYS_COEF_TABLE)
    return fail(NYS_EINVAL, "instance %d: orders 3 and 4 need kind NYS_COEF_TABLE", b);
  if (q.n < 3 || q.n > (1 << 24)) return fail(NYS_EINVAL, "instance %d: n must be in [3, 2^24] (got %d)", b, q.n);
  if (q.m < 2 || q.m > NYS_M_MAX || q.m > q.n)
    return fail(NYS_EINVAL, "instance %d: m must be in [2, min(n, %d)] (got %d)", b, NYS_M_MAX, q.m);
  if (q.kind < 0 || q.kind > 2) return fail(NYS_EINVAL, "instance %d: unknown kind %d", b, q.kind);
  if (!(std::isfinite(q.t0) && std::isfinite(q.t1) && q.t1 > q.t0))
    return fail(NYS_EINVAL, "instance %d: need finite t0 < t1", b);
  if (!(std::isfinite(q.sigma) && q.sigma > 0)) return fail(NYS_EINVAL, "instance %d: sigma must be > 0", b);
  if (!(std::isfinite(q.gamma) && q.gamma > 0)) return fail(NYS_EINVAL, "instance %d: gamma must be > 0", b);
  if (q.kind == NYS_COEF_POLY_NL && q.p == 1 && (q.c[4] != 0.0 || q.c[7] != 0.0))
    return fail(NYS_EINVAL, "instance %d: the delta y' and beta y'^2 / y terms need p = 2", b);
  if (q.kind == NYS_COEF_TABLE && q.coef_table == nullptr)
    return fail(NYS_EINVAL, "instance %d: kind TABLE needs coef_table", b);
  if (q.bc != NYS_BC_IVP && q.bc != NYS_BC_BVP)
    return fail(NYS_EINVAL, "instance %d: bc must be NYS_BC_IVP or NYS_BC_BVP (got %d)", b, q.bc);
  if (q.reserved != 0) return fail(NYS_EINVAL, "instance %d: reserved must be 0", b);
  if (q.bc == NYS_BC_BVP && q.p != 2 && q.p != 4)
    return fail(NYS_EINVAL, "instance %d: boundary values need order 2 or 4", b);
  if (q.landmarks) {
    for (int j = 0; j < q.m; ++j) {
      if (q.landmarks[j] < 0 || q.landmarks[j] >= q.n || (j > 0 && q.landmarks[j] <= q.landmarks[j - 1]))
        return fail(NYS_EINVAL, "instance %d: landmarks must be increasing indices in [0, n)", b);
    }
  }
  bool fin = finite_all(q.v, q.p) && finite_all(q.c, 8);
  if (q.kind == NYS_COEF_TABLE) fin = fin && finite_all(q.coef_table, (q.p + 1) * q.n);
  return fin ? NYS_OK : NYS_ENONFINITE;
}

// collocation rows of an instance: i = 2..n (initial values) or 2..n-1
// (boundary values); 0-based row indices 1 .. collocation_rows(q)
static int collocation_rows(const nys_instance& q) {
  return q.n - 1 - (q.bc == NYS_BC_BVP ? 1 : 0);
}

static void default_landmarks(int n, int m, int32_t* out) {
  for (int j = 0; j < m; ++j)
    out[j] = (int32_t)(((int64_t)j * (n - 1) + (m - 1) / 2) / (m - 1));
}

// Instance fields that an update may change; the landmark-set fields (lset,
// lm_off) and the work-list fields of h_inst are kept.
static void fill_inst(nys_ctx* c, const nys_instance& s, Inst& I) {
  I.t0 = s.t0;
  I.h = (s.t1 - s.t0) / (double)(s.n - 1);
  I.sigma = s.sigma;
  // eq32's sqrt(m) feature scale is the same problem with gamma -> m gamma
  I.gamma = c->opt.scale_sqrt_m ? s.gamma * s.m : s.gamma;
  for (int k = 0; k < 4; ++k) I.v[k] = (k < s.p) ? s.v[k] : 0.0;
  for (int k = 0; k < 8; ++k) I.c[k] = s.c[k];
  if (s.p == 1 && s.kind == NYS_COEF_LIN) I.c[1] = 0.0;
  I.hs = I.h / s.sigma;
  I.th0 = mod2pi(s.c[3] * s.t0 + s.c[4]);
  I.dth = mod2pi(s.c[3] * I.h);
  I.rk = row_const(I);
  I.tab_off = -1;
  if (s.kind == NYS_COEF_TABLE) {
    I.tab_off = (int64_t)c->h_tab.size();
    c->h_tab.insert(c->h_tab.end(), s.coef_table, s.coef_table + (size_t)(s.p + 1) * s.n);
  }
}

static int32_t repack_same_sets(nys_ctx* c, const nys_instance* q);
static int32_t pack_all(nys_ctx* c, const nys_instance* q, bool first);

// Fill h_inst / h_lset / h_stinit / h_tab from the instance array (host only).
// An update (first = false) keeps p, n, m, kind, bc and the landmarks; when no
// instance's h / sigma changed either, the landmark sets and their sharing are
// those of the previous call and are kept as they are (no key map rebuilt).
static int32_t pack(nys_ctx* c, const nys_instance* q, bool first, bool* same_out = nullptr) {
  const int B = c->batch;
  if (same_out) *same_out = false;
  if (!first) {
    bool same_sets = ((int)c->h_inst.size() == B);
    for (int b = 0; b < B && same_sets; ++b) {
      const nys_instance& s = q[b];
      const double h = (s.t1 - s.t0) / (double)(s.n - 1);
      same_sets = (h / s.sigma == c->h_inst[b].hs);
    }
    if (same_sets) {
      if (same_out) *same_out = true;
      return repack_same_sets(c, q);
    }
  }
  // an update keeps the work-list fields of the descriptors (and all of them
  // when it fails)
  std::vector<Inst> keep;
  if (!first) keep = c->h_inst;
  int32_t r = pack_all(c, q, first);
  if (!first) {
    if (r != NYS_OK) {
      c->h_inst = keep;
      return r;
    }
    for (int b = 0; b < B; ++b) {
      c->h_inst[b].slot_begin = keep[b].slot_begin;
      c->h_inst[b].slot_count = keep[b].slot_count;
      c->h_inst[b].rslot_begin = keep[b].rslot_begin;
      c->h_inst[b].rslot_count = keep[b].rslot_count;
      c->h_inst[b].y_off = keep[b].y_off;
    }
  }
  return r;
}

static int32_t pack_all(nys_ctx* c, const nys_instance* q, bool first) {
  const int B = c->batch;
  c->h_inst.assign(B, Inst{});
  c->h_stinit.assign(B, NYS_OK);
  if (first) {
    c->h_lm.clear();
    c->h_lm_off.assign(B, 0);
    c->lm_dflt.assign(B, 0);
  }
  c->h_tab.clear();
  std::map<std::vector<int64_t>, int> keys;
  c->h_lset.clear();
  c->nlset = 0;
  c->k_max = 0;
  for (int b = 0; b < B; ++b) {
    const nys_instance& s = q[b];
    int32_t r = check_instance(s, b);
    if (r == NYS_EINVAL) return r;
    if (!first) {
      const nys_instance& o = c->shape[b];
      if (o.p != s.p || o.n != s.n || o.m != s.m || o.kind != s.kind || o.bc != s.bc)
        return fail(NYS_EINVAL, "nys_update: instance %d changed p, n, m, kind or bc", b);
    }
    std::vector<int32_t> lm(s.m);
    if (s.landmarks) std::memcpy(lm.data(), s.landmarks, sizeof(int32_t) * s.m);
    else default_landmarks(s.n, s.m, lm.data());
    if (first) {
      c->h_lm_off[b] = (int64_t)c->h_lm.size();
      c->h_lm.insert(c->h_lm.end(), lm.begin(), lm.end());
      bool dflt = true;
      for (int j = 0; j < s.m && dflt; ++j)
        dflt = lm[j] == (int32_t)(((int64_t)j * (s.n - 1) + (s.m - 1) / 2) / (s.m - 1));
      c->lm_dflt[b] = dflt ? 1 : 0;
    } else {
      if (std::memcmp(lm.data(), c->h_lm.data() + c->h_lm_off[b], sizeof(int32_t) * s.m) != 0)
        return fail(NYS_EINVAL, "nys_update: instance %d changed its landmarks", b);
    }
    Inst& I = c->h_inst[b];
    I.p = s.p; I.n = s.n; I.m = s.m; I.kind = s.kind;
    I.bc = s.bc;
    I.lm_off = c->h_lm_off[b];
    fill_inst(c, s, I);
    c->h_stinit[b] = r;
    // landmark-set key: n, m, indices, bits of h/sigma.  Slot b is the set of
    // instance b; only the first instance with a given key is active.
    std::vector<int64_t> key(lm.begin(), lm.end());
    int64_t hbits;
    std::memcpy(&hbits, &I.hs, sizeof hbits);
    key.push_back(hbits);
    key.push_back(s.m);
    key.push_back(s.n);
    Lset L{};
    L.m = s.m;
    L.m_eff = s.m;
    L.n = s.n;
    L.K = (int)std::min<double>(s.n - 1, std::ceil(std::sqrt(kLagU) / I.hs));
    L.lm_off = I.lm_off;
    L.w_off = (int64_t)b * c->m_max * c->m_max;
    L.lag_off = c->h_lagcap[b];
    L.hs = I.hs;
    auto it = keys.find(key);
    if (it == keys.end()) {
      keys.emplace(std::move(key), b);
      L.active = 1;
      I.lset = b;
      ++c->nlset;
    } else {
      L.active = 0;
      I.lset = it->second;
    }
    c->h_lset.push_back(L);
    c->k_max = std::max(c->k_max, L.K);
  }
  return NYS_OK;
}

// nys_update with unchanged landmark sets: validate, refresh the per-instance
// fields in place.
static int32_t repack_same_sets(nys_ctx* c, const nys_instance* q) {
  const int B = c->batch;
  for (int b = 0; b < B; ++b) {
    const nys_instance& s = q[b];
    const nys_instance& o = c->shape[b];
    if (o.p != s.p || o.n != s.n || o.m != s.m || o.kind != s.kind || o.bc != s.bc)
      return fail(NYS_EINVAL, "nys_update: instance %d changed p, n, m, kind or bc", b);
    // default landmarks of an unchanged (n, m) over stored defaults: equal by construction
    if (!s.landmarks && c->lm_dflt[b]) continue;
    int32_t dflt[NYS_M_MAX];
    const int32_t* lm = s.landmarks;
    if (!lm) {
      default_landmarks(s.n, s.m, dflt);
      lm = dflt;
    }
    if (std::memcmp(lm, c->h_lm.data() + c->h_lm_off[b], sizeof(int32_t) * s.m) != 0)
      return fail(NYS_EINVAL, "nys_update: instance %d changed its landmarks", b);
  }
  std::vector<int32_t> st(B);
  for (int b = 0; b < B; ++b) {
    st[b] = check_instance(q[b], b);
    if (st[b] == NYS_EINVAL) return st[b];
  }
  c->h_tab.clear();
  for (int b = 0; b < B; ++b) {
    fill_inst(c, q[b], c->h_inst[b]);
    c->h_stinit[b] = st[b];
  }
  return NYS_OK;
}

static cudaError_t enqueue_factor(nys_ctx* c, cudaStream_t s) {
  return launch_setup(c->lset.p, c->batch, c->lm.p, c->W.p, c->W32.p, c->lam.p, c->lag.p,
                      c->opt.eig_tau > 0 ? c->opt.eig_tau : 1e-12, c->m_max, s, c->fp32 ? 0 : 1,
                      c->eig_bounds.data(), (int)c->eig_bounds.size(), c->bigset(), c->crow.p,
                      c->inst.p, c->nlset <= c->num_sms ? 1 : 0);
}

// The lag tables (read by the row passes) go on the caller's stream; the
// eigendecomposition is forked onto the side stream: the row pass works in
// kernel coordinates and does not need W, so the two overlap; the solve joins.
static cudaError_t fork_factor(nys_ctx* c, cudaStream_t s) {
  cudaError_t e = launch_lag(c->lset.p, c->batch, c->lag.p, s);
  if (e == cudaSuccess) e = cudaEventRecord(c->ev_fork, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->side, c->ev_fork, 0);
  if (e == cudaSuccess)
    e = launch_eig(c->lset.p, c->batch, c->lm.p, c->W.p, c->W32.p, c->lam.p,
                   c->opt.eig_tau > 0 ? c->opt.eig_tau : 1e-12, c->m_max, c->side,
                   c->fp32 ? 0 : 1, c->eig_bounds.data(), (int)c->eig_bounds.size(), c->bigset(),
                   c->crow.p, c->inst.p, c->nlset <= c->num_sms ? 1 : 0, c->lag.p);
  if (e == cudaSuccess) e = cudaEventRecord(c->ev_join, c->side);
  return e;
}

// upload_lset = false keeps the device landmark-set descriptors, whose m_eff and
// omode the factor kernel wrote (an update that keeps every landmark set).
// factor_now runs the factor on the caller's stream before anything else: a row
// pass needs the final omode of its set (omega-mode sets project each row through
// W), so descriptors uploaded with the host's initial omode must not meet a row
// pass that overlaps a forked factor.
static int32_t upload_and_setup(nys_ctx* c, cudaStream_t s, bool factor_now, bool upload_lset = true) {
  // reuse of the pinned staging buffers: wait for the previous upload
  CK(cudaEventSynchronize(c->staged));
  std::memcpy(c->pin_inst, c->h_inst.data(), sizeof(Inst) * c->batch);
  if (upload_lset) std::memcpy(c->pin_lset, c->h_lset.data(), sizeof(Lset) * c->batch);
  std::memcpy(c->pin_st, c->h_stinit.data(), sizeof(int32_t) * c->batch);

  CK(cudaMemcpyAsync(c->inst.p, c->pin_inst, sizeof(Inst) * c->batch, cudaMemcpyHostToDevice, s));
  if (upload_lset)
    CK(cudaMemcpyAsync(c->lset.p, c->pin_lset, sizeof(Lset) * c->batch, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c->stinit.p, c->pin_st, sizeof(int32_t) * c->batch, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c->st.p, c->pin_st, sizeof(int32_t) * c->batch, cudaMemcpyHostToDevice, s));

  if (!c->h_tab.empty())
    CK(cudaMemcpyAsync(c->tab.p, c->h_tab.data(), sizeof(double) * c->h_tab.size(),
                       cudaMemcpyHostToDevice, s));
  CK(cudaEventRecord(c->staged, s));
  if (!c->h_tab.empty()) CK(cudaStreamSynchronize(s));  // pageable source
  c->upload_bytes = (int64_t)(sizeof(Inst) * c->batch + (upload_lset ? sizeof(Lset) * c->batch : 0) +
                              2 * sizeof(int32_t) * c->batch + sizeof(double) * c->h_tab.size());
  c->factor_stale = true;
  if (factor_now) {
    CK(enqueue_factor(c, s));
    c->factor_stale = false;
  }
  c->assembled = false;
  c->solved = false;
  return NYS_OK;
}

extern "C" {

const char* nys_last_error(void) { return g_err.c_str(); }

const char* nys_status_str(int32_t s) {
  switch (s) {
    case NYS_OK: return "ok";
    case NYS_EINVAL: return "invalid argument";
    case NYS_ENOMEM: return "out of memory";
    case NYS_ECUDA: return "CUDA error";
    case NYS_ENOTSPD: return "projected Hessian not positive definite";
    case NYS_ENOCONV: return "Newton iteration cap reached";
    case NYS_ENONFINITE: return "non-finite input or result";
    case NYS_ETIMEOUT: return "device wait timed out";
    case NYS_EPRECISION: return "landmark kernel too ill-conditioned for the mixed path";
    case NYS_ESTATE: return "call out of order";
    case NYS_EBOUNDS: return "index check failed (debug build)";
    default: return "unknown status";
  }
}

void nys_destroy(nys_ctx* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
  for (auto& g : c->ngraphs) cudaGraphExecDestroy(g.exec);
  c->inst.release(); c->lset.release(); c->lm.release(); c->tab.release(); c->work.release(); c->rwork.release();
  c->slot_off.release(); c->part.release(); c->W.release(); c->W32.release(); c->lam.release();
  c->fac.release(); c->lag.release(); c->xs.release(); c->zs.release(); c->dzs.release(); c->cws.release();
  c->st.release(); c->stinit.release(); c->counter.release(); c->yaux.release(); c->rowstate.release();
  c->nrm.release(); c->row_off.release(); c->active.release(); c->iters.release(); c->live.release();
  c->any_active.release(); c->adj.release();
  if (c->pin_inst) cudaFreeHost(c->pin_inst);
  if (c->pin_lset) cudaFreeHost(c->pin_lset);
  if (c->pin_st) cudaFreeHost(c->pin_st);
  if (c->pin_flag) cudaFreeHost(c->pin_flag);
  if (c->staged) cudaEventDestroy(c->staged);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->side) cudaStreamDestroy(c->side);
  delete c;
}

// Most landmarks (sorted grid indices) within any len consecutive grid points.
static int lm_span_count(const int32_t* idx, int m, int64_t len) {
  int best = 0;
  for (int a = 0, z = 0; a < m; ++a) {
    if (z < a) z = a;
    while (z < m && idx[z] <= idx[a] + len - 1) ++z;
    best = std::max(best, z - a);
  }
  return best;
}

// Band plan of instance b for k_assemble_band (kind LIN): the longest window W
// (512, 256, 128, 64 or 32 rows) whose rows see at most kBandLm landmarks within the
// band lag Kb, with its kappa table (2 (Kb + W - 1) + 1 lags and W zeros) in
// kBandTabCap floats; then unit rows U, a multiple of W of at most
// max(W, target) rows, whose landmarks + 2 fit kBandUnitCols.  W = 0: the
// instance goes to the tensor-core kernel.
static void band_plan(const nys_ctx* c, int b, int64_t target, int& W, int& U) {
  W = U = 0;
  const Inst& I = c->h_inst[b];
  if (I.kind != NYS_COEF_LIN || I.m > kMMax) return;
  const int32_t* idx = c->h_lm.data() + c->h_lm_off[b];
  const int Kb = asm_band_lag(I.hs, I.n);
  for (int w = 512; w >= 32; w /= 2) {
    if (2LL * (Kb + w - 1) + 1 + w <= kBandTabCap && lm_span_count(idx, I.m, w + 2LL * Kb) <= kBandLm) {
      W = w;
      break;
    }
  }
  if (W == 0) return;
  const int64_t cap = std::max<int64_t>(W, std::min<int64_t>(target, 8192) / W * W);
  U = W;
  for (int64_t u = 2LL * W; u <= cap; u += W) {
    if (lm_span_count(idx, I.m, u + 2LL * Kb) + 2 > kBandUnitCols) break;
    U = (int)u;
  }
}

// Refinement band plan of instance b for k_refine_band (mixed path, kind LIN):
// a window W (512 down to 32 rows) whose rows see at most kRbLm landmarks within
// its band lag K (u <= kRefBandU), with its float-float kappa table
// (2 (K + W - 1) + 1 lags and W zeros) in kRbTabCap entries; 0: k_refine_rows.
static int refine_band_plan(const nys_ctx* c, int b, int64_t unit_rows) {
  const Inst& I = c->h_inst[b];
  if (!c->fp32 || I.kind != NYS_COEF_LIN || I.m > kMMax) return 0;
  const int K = std::min(refine_band_lag(I.hs, I.n), c->h_lset[b].K);
  const int32_t* idx = c->h_lm.data() + c->h_lm_off[b];
  // among the feasible windows, the one with the shortest unit time: its
  // kRbWarps warps take ceil(windows / kRbWarps) windows each, a window costing
  // W / 32 rows per lane plus its reduction (about one row's worth)
  int best = 0;
  double best_t = 0.0;
  for (int w = kRbMaxW; w >= 32; w /= 2) {
    if (2LL * (K + w - 1) + 1 + w > kRbTabCap || lm_span_count(idx, I.m, w + 2LL * K) > kRbLm)
      continue;
    const int64_t nwin = (std::max<int64_t>(1, unit_rows) + w - 1) / w;
    const double t = (double)((nwin + kRbWarps - 1) / kRbWarps) * (w / 32 + 1);
    if (best == 0 || t < best_t) { best = w; best_t = t; }
  }
  return best;
}

// Refinement work list in use: the setup's list with the items of planned
// instances first (window rows in Work::e0).  Returns whether the plan changed.
static bool refine_layout(nys_ctx* c, std::vector<Work>& out) {
  std::vector<int> wr(c->batch);
  std::vector<int64_t> urows(c->batch, 0);       // longest refinement item per instance
  for (const Work& w : c->h_rwork) urows[w.inst] = std::max<int64_t>(urows[w.inst], w.r1 - w.r0);
  for (int b = 0; b < c->batch; ++b) wr[b] = refine_band_plan(c, b, urows[b]);
  const bool changed = (wr != c->rband_w);
  c->rband_w = wr;
  out.clear();
  for (const Work& w : c->h_rwork)
    if (wr[w.inst]) { Work x = w; x.e0 = wr[w.inst]; x.e1 = 0; out.push_back(x); }
  c->nrband = (int)out.size();
  for (const Work& w : c->h_rwork)
    if (!wr[w.inst]) out.push_back(w);
  return changed;
}

// Band unit length aimed at: about 4 units per warp of the band kernel's
// persistent grid (8 warps per SM).
static int64_t band_target(const nys_ctx* c) {
  return std::max<int64_t>(256, c->total_rows / (32LL * c->num_sms));
}

// Assembly work list: the rows of every instance in chunks of at most rpi rows,
// sorted by cost (rows x (m+2)^2, longest first, for the persistent grid); slot
// offsets into `part` from 0.  Sets the instances' assembly slot ranges.  With
// `band`, instances with a band plan are cut into its units instead (window
// rows in Work::e0) and listed first; *nband receives their count.
static int64_t asm_layout(nys_ctx* c, int64_t rpi, std::vector<Work>& wl, std::vector<int64_t>& soff,
                          bool band = false, int* nband = nullptr) {
  wl.clear();
  soff.clear();
  int64_t poff = 0;
  int slot = 0;
  std::vector<Work> bl;
  if (band) {
    c->band_w.assign(c->batch, 0);
    c->band_u.assign(c->batch, 0);
  }
  const int64_t target = band_target(c);
  for (int b = 0; b < c->batch; ++b) {
    const int nrows = collocation_rows(c->shape[b]);
    const int M2 = c->shape[b].m + 2;
    // a Gram of more than kMMax + 2 columns: parts of at most kAsm64Span packed
    // entries per work item, and chunks of at least 512 rows (the slots of
    // these instances are summed by a separate pass)
    const bool bigm = c->shape[b].m > kMMax;
    const int64_t Elin = (int64_t)M2 * (M2 + 1) / 2;
    const int parts = bigm ? (int)((Elin + kAsm64Span - 1) / kAsm64Span) : 1;
    int bw = 0, bu = 0;
    if (band) {
      band_plan(c, b, target, bw, bu);
      c->band_w[b] = bw;
      c->band_u[b] = bu;
    }
    const int64_t rpb = bw ? bu : (bigm ? std::max<int64_t>(rpi, 512) : rpi);
    const int chunks = (int)std::max<int64_t>(1, (nrows + rpb - 1) / rpb);
    // band units: equal shares rounded up to whole windows
    const int64_t ubw = bw ? ((nrows + chunks - 1) / chunks + bw - 1) / bw * bw : 0;
    // linear: [first landmark, count] + packed Gram over m + 2 columns;
    // Newton: packed Gram over m + 1 columns, two (m+1)-vectors, two scalars
    const int64_t E = std::max<int64_t>((int64_t)M2 * (M2 + 1) / 2 + 2,
                                        (int64_t)(M2 - 1) * M2 / 2 + 2 * (M2 - 1) + 2);
    c->h_inst[b].slot_begin = slot;
    c->h_inst[b].slot_count = chunks;
    for (int k = 0; k < chunks; ++k) {
      for (int pt = 0; pt < parts; ++pt) {
        Work w;
        w.inst = b;
        if (bw) {
          w.r0 = 1 + (int)std::min<int64_t>(nrows, ubw * k);
          w.r1 = 1 + (int)std::min<int64_t>(nrows, ubw * (k + 1));
          w.e0 = bw;
          w.e1 = 0;
        } else {
          w.r0 = 1 + (int)((int64_t)nrows * k / chunks);
          w.r1 = 1 + (int)((int64_t)nrows * (k + 1) / chunks);
          w.e0 = bigm ? (int)(Elin * pt / parts) : 0;
          w.e1 = bigm ? (int)(Elin * (pt + 1) / parts) : INT32_MAX;
        }
        w.slot = slot;
        (bw ? bl : wl).push_back(w);
      }
      ++slot;
      soff.push_back(poff);
      poff += E;
    }
  }
  const std::vector<nys_instance>& q = c->shape;
  auto cost = [&](const Work& a) {
    const double M2 = q[a.inst].m + 2;
    const double ent = std::min(M2 * (M2 + 1) / 2, (double)a.e1) - a.e0;
    return (double)(a.r1 - a.r0) * ent;
  };
  std::stable_sort(wl.begin(), wl.end(), [&](const Work& a, const Work& b2) {
    return cost(a) > cost(b2);
  });
  std::stable_sort(bl.begin(), bl.end(), [&](const Work& a, const Work& b2) {
    return a.r1 - a.r0 > b2.r1 - b2.r0;
  });
  if (nband) *nband = (int)bl.size();
  wl.insert(wl.begin(), bl.begin(), bl.end());
  return poff;
}

int32_t nys_setup(nys_ctx** out, const nys_instance* q, int32_t batch, const nys_options* opt,
                  void* stream) {
  if (!out) return fail(NYS_EINVAL, "nys_setup: out is NULL");
  *out = nullptr;
  if (!q || batch < 1) return fail(NYS_EINVAL, "nys_setup: need batch >= 1 instances");
  nys_ctx* c = new nys_ctx();
  c->batch = batch;
  if (opt) c->opt = *opt;
  else { c->opt.precision = NYS_FP64; c->opt.refine_steps = -1; }
  if (c->opt.precision != NYS_FP64 && c->opt.precision != NYS_MIXED &&
      c->opt.precision != NYS_MIXED_F64F) {
    delete c;
    return fail(NYS_EINVAL, "nys_setup: unknown precision %d", c->opt.precision);
  }
  if (c->opt.assembly != NYS_ASM_AUTO && c->opt.assembly != NYS_ASM_SIMT &&
      c->opt.assembly != NYS_ASM_TUNE && c->opt.assembly != NYS_ASM_TC) {
    const int a = c->opt.assembly;
    delete c;
    return fail(NYS_EINVAL, "nys_setup: unknown assembly kernel %d", a);
  }
  // default refinement: one pass for every instance (two when the batch holds
  // boundary value instances, whose FP32 factor contracts the error more
  // slowly), then an adaptive pass for the instances whose estimated error is
  // still above kRefineAgain: a landmark kernel near the conditioning limit
  // (sigma about one landmark spacing at m = 64..100, n up to 2e4) can leave a
  // few 1e-6 after one pass
  if (c->opt.refine_steps < 0) {
    bool any_bvp = false;
    for (int b = 0; b < batch; ++b) any_bvp = any_bvp || (q[b].bc == NYS_BC_BVP);
    c->opt.refine_steps = any_bvp ? 2 : 1;
    c->refine_adapt = 1;
  }
  if (c->opt.refine_steps > 8) { delete c; return fail(NYS_EINVAL, "nys_setup: refine_steps > 8"); }
  c->fp32 = (c->opt.precision == NYS_MIXED || c->opt.precision == NYS_MIXED_F64F);
  c->fac64 = (c->opt.precision == NYS_MIXED_F64F);
  for (int b = 0; b < batch && c->fp32; ++b)
    if (q[b].p > 2) {
      delete c;
      return fail(NYS_EINVAL, "instance %d: orders 3 and 4 need precision NYS_FP64", b);
    }
  for (int b = 0; b < batch; ++b) {
    if (q[b].m <= NYS_M_MAX_MIXED || q[b].m > NYS_M_MAX) continue;
    const char* why = c->fp32 ? "precision NYS_FP64"
                      : (q[b].kind == NYS_COEF_POLY_NL) ? "a linear kind (Newton takes m <= NYS_M_MAX_MIXED)"
                      : nullptr;
    if (why) {
      delete c;
      return fail(NYS_EINVAL, "instance %d: m > %d needs %s", b, NYS_M_MAX_MIXED, why);
    }
  }
  for (int b = 0; b < batch; ++b) {
    c->m_max = std::max(c->m_max, std::max(2, q[b].m));
    c->p_max = std::max(c->p_max, q[b].p);
  }
  c->m_max = std::min(c->m_max, NYS_M_MAX);
  {  // setup launch classes: the distinct m values, or 16-wide buckets when many
    std::vector<int> ms;
    for (int b = 0; b < batch; ++b) ms.push_back(std::min(std::max(2, q[b].m), NYS_M_MAX));
    std::sort(ms.begin(), ms.end());
    ms.erase(std::unique(ms.begin(), ms.end()), ms.end());
    if (ms.size() > 6) {
      for (int& v : ms) v = std::min(NYS_M_MAX, (v + 15) / 16 * 16);
      ms.erase(std::unique(ms.begin(), ms.end()), ms.end());
    }
    c->eig_bounds = ms;
  }
  c->shape.assign(q, q + batch);
  c->h_lagcap.assign(batch, 0);
  {
    int64_t o = 0;
    for (int b = 0; b < batch; ++b) {
      c->h_lagcap[b] = o;
      o += 6LL * std::max(3, q[b].n);
    }
    c->lag_floats = o;
  }
  for (auto& s : c->shape) { s.landmarks = nullptr; s.coef_table = nullptr; }
  int32_t r = pack(c, q, true);
  if (r != NYS_OK) { delete c; return r; }
  for (int b = 0; b < batch; ++b) {
    if (q[b].kind == NYS_COEF_POLY_NL) c->any_nl = true;
    else c->any_lin = true;
    // a beta u^2 / y term needs the Newton row pass's two extra tiles
    if (q[b].kind == NYS_COEF_POLY_NL && q[b].p == 2 && q[b].c[7] != 0.0) c->nt_tiles = 6;
  }
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (ce != cudaSuccess) { delete c; return fail(NYS_ECUDA, "no CUDA device: %s", cudaGetErrorString(ce)); }
  cudaStream_t s = (cudaStream_t)stream;

  // row-pass work list: split instances so that there are >= 4 items per SM
  int64_t total_rows = 0;
  for (int b = 0; b < batch; ++b) total_rows += collocation_rows(q[b]);
  c->total_rows = total_rows;
  const int64_t target = std::max<int64_t>(batch, 4LL * c->num_sms);
  int64_t rpi = std::max<int64_t>(64, (total_rows + target - 1) / target);
  // FP32 row pass: chunks of at most 1024 rows, whose landmark windows are narrow
  if (c->fp32) rpi = std::min<int64_t>(rpi, 1024);
  c->rpi = rpi;
  // tensor-core assembly: long work units (each cut into narrow sub-chunks in the kernel)
  c->tc_rpi = asm_tc_unit_rows(total_rows, batch, c->num_sms);
  c->tune_pending = c->fp32 && c->opt.assembly == NYS_ASM_TUNE;
  if (c->opt.assembly == NYS_ASM_TUNE && !c->fp32) c->opt.assembly = NYS_ASM_AUTO;
  const bool hyb = c->fp32 && (c->opt.assembly == NYS_ASM_AUTO || c->tune_pending);
  const bool tcu = hyb || (c->fp32 && c->opt.assembly == NYS_ASM_TC);
  // the assembly slot region holds the largest layout this context may use:
  // band units + tensor-core units (the layout in use, built last), the
  // tensor-core units alone (used when a re-plan outgrows the region) and, with
  // the tuner pending, the CUDA-core kernel's 512-row items
  std::vector<Work> wl;
  std::vector<int64_t> soff;
  int64_t asm_elems = 0;
  size_t asm_work_cap = 0, asm_slots = 0;
  auto account = [&](int64_t el) {
    asm_elems = std::max(asm_elems, el);
    asm_work_cap = std::max(asm_work_cap, wl.size());
    asm_slots = std::max(asm_slots, soff.size());
  };
  if (c->tune_pending) account(asm_layout(c, std::min<int64_t>(rpi, 512), wl, soff));
  if (hyb) account(asm_layout(c, c->tc_rpi, wl, soff));
  account(asm_layout(c, tcu ? c->tc_rpi : rpi, wl, soff, hyb, &c->nband));
  soff.resize(asm_slots, 0);
  c->asm_slots = (int)asm_slots;
  c->asm_elems = asm_elems;
  c->asm_rows = tcu ? c->tc_rpi : rpi;
  int64_t poff = asm_elems;
  int slot = c->asm_slots;
  // refinement work list: balance rule only (its per-item setup, a lag table
  // per instance, favours long chunks); slots of M1 doubles after the others
  std::vector<Work> rwl;
  {
    const int64_t rpr = std::max<int64_t>(64, (total_rows + target - 1) / target);
    for (int b = 0; b < batch; ++b) {
      const int nrows = collocation_rows(q[b]);
      const int chunks = (int)std::max<int64_t>(1, (nrows + rpr - 1) / rpr);
      c->h_inst[b].rslot_begin = slot;
      c->h_inst[b].rslot_count = chunks;
      for (int k = 0; k < chunks; ++k) {
        Work w;
        w.inst = b;
        w.r0 = 1 + (int)((int64_t)nrows * k / chunks);
        w.r1 = 1 + (int)((int64_t)nrows * (k + 1) / chunks);
        w.slot = slot++;
        w.e0 = 0;
        w.e1 = INT32_MAX;
        rwl.push_back(w);
        soff.push_back(poff);
        poff += std::max(q[b].m + 1, 8);   // refinement: m + 1; gradient: 5
      }
    }
  }
  auto by_cost = [&](const Work& a, const Work& b2) {
    const double ca = (double)(a.r1 - a.r0) * (q[a.inst].m + 2) * (q[a.inst].m + 2);
    const double cb = (double)(b2.r1 - b2.r0) * (q[b2.inst].m + 2) * (q[b2.inst].m + 2);
    return ca > cb;
  };
  std::stable_sort(rwl.begin(), rwl.end(), by_cost);
  c->h_rwork = rwl;
  refine_layout(c, rwl);
  c->nwork = (int)wl.size();
  c->nrwork = (int)rwl.size();
  c->XS = c->m_max + 3;
  c->ZS = c->m_max + 1;
  c->M1S = c->m_max + 1;
  c->facs = fac_elems(c->m_max);
  const size_t es = (c->fp32 && !c->fac64) ? sizeof(float) : sizeof(double);
  // Newton row offsets
  std::vector<int64_t> roff(batch);
  int64_t ytot = 0;
  for (int b = 0; b < batch; ++b) {
    c->h_inst[b].y_off = ytot;
    roff[b] = ytot;
    ytot += q[b].n - 1;
  }

  cudaError_t e = cudaSuccess;
  auto A = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
  A(c->inst.alloc(batch));
  A(c->lset.alloc(batch));
  A(c->lm.alloc(c->h_lm.size()));
  A(c->tab.alloc(std::max<size_t>(1, c->h_tab.size())));
  A(c->work.alloc(std::max(asm_work_cap, wl.size())));
  A(c->rwork.alloc(rwl.size()));
  A(c->slot_off.alloc(soff.size()));
  A(c->part.alloc((size_t)poff));
  A(c->W.alloc((size_t)batch * c->m_max * c->m_max));
  A(c->W32.alloc((size_t)batch * c->m_max * c->m_max));
  if (c->fp32) A(c->lag.alloc((size_t)c->lag_floats));
  A(c->lam.alloc((size_t)batch * NYS_M_MAX));
  A(c->crow.alloc((size_t)batch * 8 * c->m_max));
  A(c->fac.alloc((size_t)batch * c->facs * (c->any_nl ? sizeof(double) : es)));
  {
    std::vector<int32_t> ids;
    for (int b = 0; b < batch; ++b)
      if (q[b].m > kMMax) ids.push_back(b);
    c->nbig = (int)ids.size();
    if (c->nbig > 0) {
      c->big_stride = (int64_t)std::max(setup_ws_doubles(), solve_ws_doubles());
      c->big_stride = (c->big_stride + 31) / 32 * 32;
      A(c->big_ids.alloc(ids.size()));
      A(c->big_ws.alloc((size_t)c->nbig * c->big_stride));
      if (e == cudaSuccess)
        A(cudaMemcpy(c->big_ids.p, ids.data(), sizeof(int32_t) * ids.size(), cudaMemcpyHostToDevice));
    }
  }
  A(c->xs.alloc((size_t)batch * c->XS));
  A(c->zs.alloc((size_t)batch * c->ZS));
  A(c->dzs.alloc((size_t)batch * c->ZS));
  A(c->cws.alloc((size_t)batch * 2 * c->M1S));
  if (c->fp32) A(c->rcorr.alloc(batch));
  if (c->fp32) A(c->rskip.alloc(batch));
  if (c->any_lin && !c->fp32) A(c->adj.alloc((size_t)batch * grad_adj_stride(c->ZS)));
  A(c->st.alloc(batch));
  A(c->stinit.alloc(batch));
  A(c->counter.alloc(2));
  A(c->err.alloc(1));
  if (c->any_nl) {
    A(c->yaux.alloc((size_t)ytot));
    A(c->rowstate.alloc((size_t)ytot * kNtRowState));
    A(c->row_off.alloc(batch));
    A(c->nrm.alloc((size_t)batch * 4));
    A(c->active.alloc(batch));
    A(c->iters.alloc(batch));
    A(c->any_active.alloc(2));
    A(c->live.alloc(1));
  }
  A(cudaMallocHost(reinterpret_cast<void**>(&c->pin_inst), sizeof(Inst) * batch));
  A(cudaMallocHost(reinterpret_cast<void**>(&c->pin_lset), sizeof(Lset) * batch));
  A(cudaMallocHost(reinterpret_cast<void**>(&c->pin_st), sizeof(int32_t) * (batch + 1)));
  A(cudaMallocHost(reinterpret_cast<void**>(&c->pin_flag), 2 * sizeof(int32_t)));
  A(cudaEventCreateWithFlags(&c->staged, cudaEventDisableTiming));
  A(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
  A(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
  A(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
  if (e != cudaSuccess) {
    const bool oom = (e == cudaErrorMemoryAllocation);
    nys_destroy(c);
    return fail(oom ? NYS_ENOMEM : NYS_ECUDA, "nys_setup: allocation failed: %s", cudaGetErrorString(e));
  }
  // one-time uploads (pageable sources: synchronous with respect to the host)
  A(cudaMemcpyAsync(c->lm.p, c->h_lm.data(), sizeof(int32_t) * c->h_lm.size(), cudaMemcpyHostToDevice, s));
  A(cudaMemcpyAsync(c->work.p, wl.data(), sizeof(Work) * wl.size(), cudaMemcpyHostToDevice, s));
  A(cudaMemcpyAsync(c->rwork.p, rwl.data(), sizeof(Work) * rwl.size(), cudaMemcpyHostToDevice, s));
  A(cudaMemcpyAsync(c->slot_off.p, soff.data(), sizeof(int64_t) * soff.size(), cudaMemcpyHostToDevice, s));
  if (c->any_nl) A(cudaMemcpyAsync(c->row_off.p, roff.data(), sizeof(int64_t) * batch, cudaMemcpyHostToDevice, s));
  A(cudaStreamSynchronize(s));
  if (e != cudaSuccess) {
    nys_destroy(c);
    return fail(NYS_ECUDA, "nys_setup: upload failed: %s", cudaGetErrorString(e));
  }
  r = upload_and_setup(c, s, true);
  if (r != NYS_OK) { nys_destroy(c); return r; }
  *out = c;
  return NYS_OK;
}

static int32_t set_asm_layout(nys_ctx* c, int64_t rpi, cudaStream_t s, bool band);

// After a sigma change: rebuild the assembly and refinement work lists if an
// instance's band plan changed (captured graphs hold the old lists' lengths).
static int32_t replan_band(nys_ctx* c, cudaStream_t s) {
  if (!c->fp32) return NYS_OK;
  {
    // refinement list: same items, planned ones first
    std::vector<Work> rwl;
    if (refine_layout(c, rwl)) {
      CK(cudaDeviceSynchronize());
      for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
      c->graphs.clear();
      CK(cudaMemcpy(c->rwork.p, rwl.data(), sizeof(Work) * rwl.size(), cudaMemcpyHostToDevice));
    }
  }
  if (c->opt.assembly != NYS_ASM_AUTO || c->tune_pending) return NYS_OK;
  bool same = ((int)c->band_w.size() == c->batch);
  const int64_t target = band_target(c);
  for (int b = 0; b < c->batch && same; ++b) {
    int w = 0, u = 0;
    band_plan(c, b, target, w, u);
    same = (w == c->band_w[b] && u == c->band_u[b]);
  }
  if (same) return NYS_OK;
  CK(cudaDeviceSynchronize());
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
  return set_asm_layout(c, c->tc_rpi, s, true);
}

int32_t nys_update(nys_ctx* c, const nys_instance* q, void* stream) {
  if (!c || !q) return fail(NYS_EINVAL, "nys_update: NULL argument");
  bool same_sets = false;
  int32_t r = pack(c, q, false, &same_sets);
  if (r != NYS_OK) return r;
  if (!same_sets) {
    r = replan_band(c, (cudaStream_t)stream);
    if (r != NYS_OK) return r;
  }
  // same landmark sets: the device descriptors (and the factor's m_eff, omode)
  // stay valid; otherwise new ones, factored before the next row pass
  return upload_and_setup(c, (cudaStream_t)stream, !same_sets, !same_sets);
}

// ---- assembly autotuner ------------------------------------------------------
// Rebuild the assembly work list for chunks of rpi rows (within the slot region
// sized at setup) and upload it with the instances' slot ranges.
static int32_t set_asm_layout(nys_ctx* c, int64_t rpi, cudaStream_t s, bool band) {
  std::vector<Work> wl;
  std::vector<int64_t> soff;
  int nb = 0;
  int64_t el = asm_layout(c, rpi, wl, soff, band, &nb);
  if (band && ((int)soff.size() > c->asm_slots || el > c->asm_elems)) {
    // tensor-core units only (sized into the region at setup); band_w / band_u
    // keep the plan, so an unchanged plan is not laid out again
    const std::vector<int> w0 = c->band_w, u0 = c->band_u;
    el = asm_layout(c, rpi, wl, soff, false, &nb);
    c->band_w = w0;
    c->band_u = u0;
  }
  if ((int)soff.size() > c->asm_slots || el > c->asm_elems)
    return fail(NYS_ESTATE, "assembly layout exceeds its slot region");
  CK(cudaStreamSynchronize(s));
  CK(cudaMemcpy(c->work.p, wl.data(), sizeof(Work) * wl.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c->slot_off.p, soff.data(), sizeof(int64_t) * soff.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c->inst.p, c->h_inst.data(), sizeof(Inst) * c->batch, cudaMemcpyHostToDevice));
  c->nwork = (int)wl.size();
  c->nband = nb;
  c->asm_rows = rpi;
  return NYS_OK;
}

// Time every (kernel, rows per item) candidate on this batch -- band units plus
// tensor-core units, tensor-core units alone, the older CUDA-core kernel with
// 512- and 1024-row items -- one warm-up and three timed launches each; keep
// the fastest.  Runs once, outside any graph.
static int32_t tune_assembly(nys_ctx* c, cudaStream_t s) {
  c->tune_pending = false;
  if (c->factor_stale) {
    CK(enqueue_factor(c, s));
    c->factor_stale = false;
  }
  if (c->join_pending) {
    CK(cudaStreamWaitEvent(s, c->ev_join, 0));
    c->join_pending = false;
  }
  struct Cand { int kind; int64_t rows; };
  // NYS_ASM_AUTO: band units (CUDA cores) where the plan allows, tensor-core units elsewhere
  const Cand cand[4] = {{NYS_ASM_AUTO, c->tc_rpi}, {NYS_ASM_TC, c->tc_rpi},
                        {NYS_ASM_SIMT, std::min<int64_t>(c->rpi, 512)}, {NYS_ASM_SIMT, c->rpi}};
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_k = 0;
  for (int k = 0; k < 4; ++k) {
    if (k == 3 && cand[3].rows == cand[2].rows) continue;
    if (k == 1 && c->nband == 0) continue;   // no band units: the same as candidate 0
    int32_t r = set_asm_layout(c, cand[k].rows, s, cand[k].kind == NYS_ASM_AUTO);
    if (r != NYS_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return r; }
    float tot = 0.f;
    for (int rep = 0; rep < 4; ++rep) {
      CK(cudaEventRecord(e0, s));
      CK(launch_assemble(c->fp32, c->inst.p, c->lset.p, c->lag.p, c->W.p, c->work.p, c->nwork,
                         c->counter.p, c->lm.p, c->tab.p, c->part.p, c->slot_off.p, c->m_max,
                         c->k_max, c->num_sms, s, cand[k].kind, c->err.p, c->bigset(), c->tc_wait, c->nband));
      CK(cudaEventRecord(e1, s));
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (rep > 0) tot += ms;
    }
    if (tot < best) { best = tot; best_k = k; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->opt.assembly = cand[best_k].kind;
  return set_asm_layout(c, cand[best_k].rows, s, cand[best_k].kind == NYS_ASM_AUTO);
}

int32_t nys_assembly_config(nys_ctx* c, void* stream, int32_t* kernel_out, int32_t* rows_out) {
  if (!c) return fail(NYS_EINVAL, "nys_assembly_config: NULL context");
  if (c->tune_pending) {
    const int32_t r = tune_assembly(c, (cudaStream_t)stream);
    if (r != NYS_OK) return r;
  }
  if (kernel_out) *kernel_out = c->opt.assembly;
  if (rows_out) *rows_out = (int32_t)c->asm_rows;
  return NYS_OK;
}

int32_t nys_assembly_items(const nys_ctx* c, int32_t* band_items, int32_t* other_items) {
  if (!c || !band_items || !other_items) return fail(NYS_EINVAL, "nys_assembly_items: NULL argument");
  const bool band = c->fp32 && c->opt.assembly == NYS_ASM_AUTO;
  *band_items = band ? c->nband : 0;
  *other_items = c->nwork - *band_items;
  return NYS_OK;
}

int32_t nys_assemble(nys_ctx* c, void* stream) {
  if (!c) return fail(NYS_EINVAL, "nys_assemble: NULL context");
  if (c->any_nl) return fail(NYS_EINVAL, "nys_assemble: the batch holds nonlinear instances (use nys_newton)");
  if (c->tune_pending) {
    const int32_t r = tune_assembly(c, (cudaStream_t)stream);
    if (r != NYS_OK) return r;
  }
  if (c->factor_stale) {
    CK(fork_factor(c, (cudaStream_t)stream));
    c->factor_stale = false;
    c->join_pending = true;
  }
  CK(launch_assemble(c->fp32, c->inst.p, c->lset.p, c->lag.p, c->W.p, c->work.p,
                     c->nwork, c->counter.p, c->lm.p, c->tab.p, c->part.p, c->slot_off.p, c->m_max,
                     c->k_max, c->num_sms, (cudaStream_t)stream, c->opt.assembly, c->err.p,
                     c->bigset(), c->tc_wait, c->nband));
  c->assembled = true;
  return NYS_OK;
}

static int32_t solve_impl(nys_ctx* c, cudaStream_t s, double* x_out, int32_t* status_out) {
  const double gscale = 1.0;
  CK(launch_solve(c->fp32, c->inst.p, c->lset.p, c->W.p, c->W32.p, c->part.p, c->slot_off.p,
                  c->lm.p, c->fac.p, c->facs, c->xs.p, c->zs.p, c->cws.p, c->XS, c->ZS, c->M1S,
                  c->stinit.p, c->st.p, gscale, c->batch, c->m_max, s,
                  c->fp32 ? c->err.p : nullptr, c->bigset(), c->crow.p, c->fac64));
  if (c->fp32) {
    // the base passes, then (default refinement) the adaptive pass, which the
    // instances marked by the pass before it skip
    const int passes = c->opt.refine_steps + c->refine_adapt;
    for (int k = 0; k < passes; ++k) {
      const bool adaptive = c->refine_adapt && k == passes - 1;
      const bool decides = c->refine_adapt && k == passes - 2;
      CK(launch_refine(c->inst.p, c->lset.p, c->W.p, c->lag.p, c->rwork.p, c->nrwork, c->counter.p,
                       c->lm.p, c->tab.p, c->part.p, c->slot_off.p, c->fac.p, c->facs, c->xs.p, c->zs.p,
                       c->cws.p, c->XS, c->ZS, c->M1S, c->st.p, gscale, c->batch, c->m_max,
                       c->k_max, c->num_sms, s, c->nrband, c->fac64, c->rcorr.p, k, k == passes - 1,
                       adaptive ? c->rskip.p : nullptr, decides ? c->rskip.p : nullptr));
    }
  }
  if (x_out)
    CK(cudaMemcpyAsync(x_out, c->xs.p, sizeof(double) * c->batch * c->XS, cudaMemcpyDeviceToDevice, s));
  if (status_out)
    CK(cudaMemcpyAsync(status_out, c->st.p, sizeof(int32_t) * c->batch, cudaMemcpyDeviceToDevice, s));
  return NYS_OK;
}

int32_t nys_solve(nys_ctx* c, void* stream, double* x_out, int32_t* status_out) {
  if (!c) return fail(NYS_EINVAL, "nys_solve: NULL context");
  if (!c->assembled) return fail(NYS_ESTATE, "nys_solve: call nys_assemble first");
  if (c->join_pending) {
    CK(cudaStreamWaitEvent((cudaStream_t)stream, c->ev_join, 0));
    c->join_pending = false;
  }
  int32_t r = solve_impl(c, (cudaStream_t)stream, x_out, status_out);
  if (r == NYS_OK) c->solved = true;
  return r;
}

int32_t nys_run(nys_ctx* c, void* stream, double* x_out, int32_t* status_out) {
  if (!c) return fail(NYS_EINVAL, "nys_run: NULL context");
  if (c->any_nl) return fail(NYS_EINVAL, "nys_run: the batch holds nonlinear instances");
  cudaStream_t s = (cudaStream_t)stream;
  if (c->tune_pending) {
    const int32_t r = tune_assembly(c, s);
    if (r != NYS_OK) return r;
  }
  cudaGraphExec_t exec = nullptr;
  for (auto& g : c->graphs)
    if (g.x == x_out && g.st == status_out) exec = g.exec;
  if (!exec) {
    // capture on a private stream so the legacy default stream can be used by callers
    cudaStream_t cs;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { cudaStreamDestroy(cs); CK(e); }
    int32_t r = NYS_OK;
    {
      cudaError_t e2 = fork_factor(c, cs);
      if (e2 == cudaSuccess)
        e2 = launch_assemble(c->fp32, c->inst.p, c->lset.p, c->lag.p, c->W.p,
                             c->work.p, c->nwork, c->counter.p, c->lm.p, c->tab.p, c->part.p,
                             c->slot_off.p, c->m_max, c->k_max, c->num_sms, cs, c->opt.assembly,
                             c->err.p, c->bigset(), c->tc_wait, c->nband);
      if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(cs, c->ev_join, 0);
      if (e2 != cudaSuccess) r = fail(NYS_ECUDA, "capture: assemble: %s", cudaGetErrorString(e2));
      if (r == NYS_OK) r = solve_impl(c, cs, x_out, status_out);
    }
    e = cudaStreamEndCapture(cs, &graph);
    cudaStreamDestroy(cs);
    if (r != NYS_OK) { if (e == cudaSuccess) cudaGraphDestroy(graph); return r; }
    CK(e);
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(e);
    c->graphs.push_back({x_out, status_out, exec});
  }
  if (c->join_pending) {  // a setup forked by an earlier nys_assemble
    CK(cudaStreamWaitEvent(s, c->ev_join, 0));
    c->join_pending = false;
  }
  CK(cudaGraphLaunch(exec, s));
  c->assembled = c->solved = true;
  c->factor_stale = false;
  return NYS_OK;
}

int32_t nys_set_wait_limit(nys_ctx* c, int32_t polls) {
  if (!c) return fail(NYS_EINVAL, "nys_set_wait_limit: NULL context");
  c->tc_wait = polls < 0 ? -1 : polls;
  // captured graphs hold the old limit among their kernel arguments
  cudaDeviceSynchronize();
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
  return NYS_OK;
}

int64_t nys_upload_bytes(const nys_ctx* c) { return c ? c->upload_bytes : 0; }

int32_t nys_x_stride(const nys_ctx* c) { return c ? c->XS : 0; }

int32_t nys_m_eff(nys_ctx* c, void* stream, int32_t* out) {
  if (!c || !out) return fail(NYS_EINVAL, "nys_m_eff: NULL argument");
  std::vector<Lset> L(c->batch);
  CK(cudaMemcpyAsync(L.data(), c->lset.p, sizeof(Lset) * c->batch, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  for (int b = 0; b < c->batch; ++b) out[b] = L[c->h_inst[b].lset].m_eff;
  return NYS_OK;
}

int32_t nys_eval(nys_ctx* c, void* stream, const double* tq, const int64_t* tq_off, int32_t deriv,
                 double* yq_out) {
  if (!c || !tq || !tq_off || !yq_out) return fail(NYS_EINVAL, "nys_eval: NULL argument");
  if (deriv < 0 || deriv > 2) return fail(NYS_EINVAL, "nys_eval: deriv must be 0, 1 or 2");
  if (!c->solved) return fail(NYS_ESTATE, "nys_eval: no solution yet");
  CK(launch_eval(c->inst.p, c->zs.p, c->ZS, c->lm.p, tq, tq_off, deriv, yq_out, c->batch,
                 (cudaStream_t)stream));
  return NYS_OK;
}

// The Newton iteration enqueued as a fixed sequence: for each of max_iter + 1
// rounds a full-Newton row pass and step, then a Gauss-Newton re-pass and step
// that only the instances flagged by the first step take.  Instances that stop
// leave the row passes; once none is running every kernel returns at once
// (device counter), so no round needs a host decision.
static int32_t newton_enqueue(nys_ctx* c, cudaStream_t s, int32_t max_iter, double tol,
                              const double* warm, double* x_out, double* y_aux_out,
                              int32_t* iters_out, int32_t* status_out) {
  int32_t* flags = c->any_active.p;   // [stepped, needs re-pass] (informational)
  CK(launch_newton_init(c->inst.p, c->lset.p, c->W.p, c->lm.p, nullptr, c->xs.p, c->zs.p, c->dzs.p,
                        c->yaux.p, c->nrm.p, c->iters.p, c->active.p, c->st.p, c->stinit.p, c->XS,
                        c->ZS, c->batch, c->live.p, s));
  if (warm) {
    // the stopping test's scale |F0| is taken at the default start, so that a
    // warm start stops by the same rule as a cold one; then x, z, y from warm
    CK(launch_newton_pass(c->inst.p, c->lset.p, c->W.p, c->work.p, c->nwork, c->counter.p, c->lm.p,
                          c->xs.p, c->XS, c->zs.p, c->dzs.p, c->ZS, c->yaux.p, c->rowstate.p,
                          c->part.p, c->slot_off.p, c->active.p, 0, 0, c->m_max, c->nt_tiles,
                          c->num_sms, s, c->live.p));
    CK(launch_newton_step(c->inst.p, c->lset.p, c->W.p, c->part.p, c->slot_off.p, c->lm.p, c->xs.p,
                          c->zs.p, c->dzs.p, c->cws.p, c->XS, c->ZS, c->M1S, c->st.p, c->active.p,
                          c->iters.p, c->nrm.p, max_iter, tol, flags, 2, c->batch, c->m_max, s,
                          c->live.p));
    CK(launch_newton_init(c->inst.p, c->lset.p, c->W.p, c->lm.p, warm, c->xs.p, c->zs.p, c->dzs.p,
                          c->yaux.p, nullptr, c->iters.p, c->active.p, c->st.p, c->stinit.p, c->XS,
                          c->ZS, c->batch, c->live.p, s));
  }
  for (int k = 0; k <= max_iter; ++k) {
    CK(cudaMemsetAsync(flags, 0, 2 * sizeof(int32_t), s));
    for (int mode = 0; mode < 2; ++mode) {
      CK(launch_newton_pass(c->inst.p, c->lset.p, c->W.p, c->work.p, c->nwork, c->counter.p,
                            c->lm.p, c->xs.p, c->XS, c->zs.p, c->dzs.p, c->ZS, c->yaux.p,
                            c->rowstate.p, c->part.p, c->slot_off.p, c->active.p, mode,
                            (mode == 0 && k > 0) ? 1 : 0, c->m_max, c->nt_tiles, c->num_sms, s,
                            c->live.p));
      CK(launch_newton_step(c->inst.p, c->lset.p, c->W.p, c->part.p, c->slot_off.p, c->lm.p,
                            c->xs.p, c->zs.p, c->dzs.p, c->cws.p, c->XS, c->ZS, c->M1S, c->st.p,
                            c->active.p, c->iters.p, c->nrm.p, max_iter, tol, flags, mode,
                            c->batch, c->m_max, s, c->live.p));
    }
  }
  if (x_out)
    CK(cudaMemcpyAsync(x_out, c->xs.p, sizeof(double) * c->batch * c->XS, cudaMemcpyDeviceToDevice, s));
  if (status_out)
    CK(cudaMemcpyAsync(status_out, c->st.p, sizeof(int32_t) * c->batch, cudaMemcpyDeviceToDevice, s));
  if (iters_out)
    CK(cudaMemcpyAsync(iters_out, c->iters.p, sizeof(int32_t) * c->batch, cudaMemcpyDeviceToDevice, s));
  if (y_aux_out)
    CK(cudaMemcpyAsync(y_aux_out, c->yaux.p, sizeof(double) * c->yaux.n, cudaMemcpyDeviceToDevice, s));
  return NYS_OK;
}

int32_t nys_newton(nys_ctx* c, void* stream, int32_t max_iter, double tol, const double* warm,
                   double* x_out, double* y_aux_out, int32_t* iters_out, int32_t* status_out) {
  if (!c) return fail(NYS_EINVAL, "nys_newton: NULL context");
  if (!c->any_nl || c->any_lin)
    return fail(NYS_EINVAL, "nys_newton: every instance must be of kind NYS_COEF_POLY_NL");
  if (max_iter < 0 || max_iter > 1000) return fail(NYS_EINVAL, "nys_newton: max_iter must be in [0, 1000]");
  if (!(tol > 0)) return fail(NYS_EINVAL, "nys_newton: tol must be > 0");
  cudaStream_t s = (cudaStream_t)stream;
  if (c->factor_stale) {
    CK(enqueue_factor(c, s));
    c->factor_stale = false;
  }
  if (c->join_pending) {
    CK(cudaStreamWaitEvent(s, c->ev_join, 0));
    c->join_pending = false;
  }
  cudaGraphExec_t exec = nullptr;
  for (auto& g : c->ngraphs)
    if (g.max_iter == max_iter && g.tol == tol && g.warm == warm && g.x == x_out &&
        g.y == y_aux_out && g.it == iters_out && g.st == status_out)
      exec = g.exec;
  if (!exec) {
    // capture on a private stream so the legacy default stream can be used by callers
    cudaStream_t cs;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { cudaStreamDestroy(cs); CK(e); }
    const int32_t r = newton_enqueue(c, cs, max_iter, tol, warm, x_out, y_aux_out, iters_out,
                                     status_out);
    e = cudaStreamEndCapture(cs, &graph);
    cudaStreamDestroy(cs);
    if (r != NYS_OK) { if (e == cudaSuccess) cudaGraphDestroy(graph); return r; }
    CK(e);
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(e);
    c->ngraphs.push_back({max_iter, tol, warm, x_out, y_aux_out, iters_out, status_out, exec});
  }
  CK(cudaGraphLaunch(exec, s));
  c->solved = true;
  return NYS_OK;
}

int32_t nys_grad(nys_ctx* c, void* stream, const double* obs_t, const int64_t* obs_off,
                 const double* dl_dy, double* grad_out) {
  if (!c || !obs_t || !obs_off || !dl_dy || !grad_out) return fail(NYS_EINVAL, "nys_grad: NULL argument");
  if (c->any_nl) return fail(NYS_EINVAL, "nys_grad: defined for linear (NYS_COEF_LIN) batches");
  for (int b = 0; b < c->batch; ++b) {
    if (c->shape[b].bc != NYS_BC_IVP) return fail(NYS_EINVAL, "nys_grad: initial value problems only");
    if (c->shape[b].p > 2) return fail(NYS_EINVAL, "nys_grad: orders 1 and 2 only");
  }
  if (c->fp32) return fail(NYS_ESTATE, "nys_grad: needs a context created with precision NYS_FP64");
  if (c->nbig > 0) return fail(NYS_EINVAL, "nys_grad: m <= %d only", NYS_M_MAX_MIXED);
  if (!c->solved) return fail(NYS_ESTATE, "nys_grad: no solution yet");
  CK(launch_grad(c->inst.p, c->lset.p, c->W.p, (const double*)c->fac.p, c->facs, c->xs.p, c->zs.p,
                 c->lm.p, c->XS, c->ZS, c->st.p, obs_t, obs_off, dl_dy, c->adj.p, c->rwork.p,
                 c->nrwork, c->counter.p, c->part.p, c->slot_off.p, grad_out, 1.0, c->batch,
                 c->num_sms, (cudaStream_t)stream));
  return NYS_OK;
}

}  // extern "C"
