// libfctn C ABI: handle state, the PAM sweep driver (Algorithms 1 and 2) and
// the data movement around it.  Every arithmetic step runs in the kernels of
// kernels_*.cu; this file plans index maps, owns device memory and orders
// launches on the handle's stream.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "fctn_internal.cuh"

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) return fail(FCTN_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// ---- labelled views (FCTN format bookkeeping) ------------------------------
struct Lab {
  int kind, a, b;  // kind 0: physical mode a; kind 1: bond (a, b), a < b
  bool operator==(const Lab& o) const { return kind == o.kind && a == o.a && b == o.b; }
};
Lab mode_lab(int t) { return Lab{0, t, -1}; }
Lab bond_lab(int x, int y) { return Lab{1, x < y ? x : y, x < y ? y : x}; }

struct View {
  int n = 0;
  Lab lab[FCTN_MAXD];
  int64_t ext[FCTN_MAXD];
  int64_t str[FCTN_MAXD];
  int find(const Lab& l) const {
    for (int i = 0; i < n; ++i)
      if (lab[i] == l) return i;
    return -1;
  }
  int64_t size() const {
    int64_t s = 1;
    for (int i = 0; i < n; ++i) s *= ext[i];
    return s;
  }
};

View dense_view(int n, const Lab* labs, const int64_t* ext) {
  View v;
  v.n = n;
  int64_t st = 1;
  for (int i = n - 1; i >= 0; --i) {
    v.lab[i] = labs[i];
    v.ext[i] = ext[i];
    v.str[i] = st;
    st *= ext[i];
  }
  return v;
}

// One table-driven contraction (kernels_sgemm.cu) of a plan: its shape, the
// offset (in ints) of its six tables in the handle's table buffer, and whether
// the operands are passed swapped (so that C's innermost index runs along n).
struct SgPlanH {
  SgShape sh{};
  size_t tab = 0;
  bool swap = false;
  bool tcok = false;       // served by the tensor-core contraction while the route's products are TF32
  bool round_out = false;  // there its output is an operand of the next tensor-core step: rounded to TF32
  TccShape tcs{};
};

// Head-mode association of a sweep (order 1, ..., N; head = mode 1, index 0
// here).  M_0, the merged tensor of every factor but the head, serves three
// products: the head's right-hand side X_(0) M_0^T, the reconstruction
// F = A_(0) M_0 of the X update (the merged tensor that Algorithm 2 keeps for
// the X update, here the head's), and, through Z = X_(0)^T A_(0), the
// right-hand sides of all other factors: X_(k) M_k^T is Z contracted with the
// factors t != 0, k (the same products, associated differently).  The
// Gram M_k M_k^T of every factor is the contraction of the factor Grams
// H_t = A_(t)^T A_(t), t != k, over their shared bond pairs.
struct HeadRoute {
  bool on = false;
  int64_t s0 = 0, P0 = 0;
  SgPlanH m0[FCTN_MAX_ORDER];  // chain building M_0 from factors m0fac[0], m0fac[1], ... (nm0 steps)
  int m0fac[FCTN_MAX_ORDER] = {};
  int nm0 = 0;
  SgPlanH y0, z;               // Y_0 raw = X_(0) M_0^T, Z = X_(0)^T A_(0)
  SgPlanH ys[FCTN_MAX_ORDER][FCTN_MAX_ORDER];  // per k >= 1: Z (x) A_t for t in yfac[k]
  int yfac[FCTN_MAX_ORDER][FCTN_MAX_ORDER] = {};
  int nys[FCTN_MAX_ORDER] = {};
  int yshare[FCTN_MAX_ORDER] = {};  // leading steps of ys[k] whose result factor k-1's chain left in U
  SgPlanH hg[FCTN_MAX_ORDER];  // H_t
  SgPlanH env[FCTN_MAX_ORDER][FCTN_MAX_ORDER];  // per k: chain of H_t, t != k, in the order efac[k]
  int efac[FCTN_MAX_ORDER][FCTN_MAX_ORDER] = {};
  int nenv[FCTN_MAX_ORDER] = {};
  int eshare[FCTN_MAX_ORDER] = {};  // leading steps of env[k] whose result factor k-1's chain left in E
  int64_t u_elems = 0, e_elems = 0, part_main = 0, part_side = 0;
  float *M0 = nullptr, *Zb = nullptr, *U[2] = {nullptr, nullptr}, *E[2] = {nullptr, nullptr};
  float* H[FCTN_MAX_ORDER] = {};
  float *Yraw = nullptr, *pm = nullptr, *ps = nullptr;
  int* tabs = nullptr;
  bool m0_valid = false;
  bool hvalid[FCTN_MAX_ORDER] = {};
  // tensor-core products (TF32 / BF16): Y_0 = X M_0^T, Z = X^T A_0 and
  // F^T = M_0^T A_0^T with the X update, on TMA-fed tcgen05 GEMMs
  bool tc = false, bf16 = false;
  bool fp32_now = false;           // the CUDA-core FP32 products serve (finish_fp32_at reached)
  double prev_rel = 0.0;           // lowest rel_change so far and the sweeps since it fell
  int stall = 0;
  bool xt_valid = false;           // XT (and the BF16 copy of X) hold the present X
  int64_t ldt = 0, ld0 = 0;        // leading dimensions of XT / A0T (I_0) and of M0T / A0p (s_0 padded)
  TgArgs ty{}, tz{}, tf{};         // shapes of the three GEMMs
  alignas(64) unsigned char maps[6][128];  // tensor maps: Y (A, B), Z (A, B), F (A, B)
  void *M0T = nullptr, *XT = nullptr, *A0T = nullptr, *A0p = nullptr;  // operand copies (FP32 or BF16)
  void *Xb = nullptr, *M0b = nullptr;  // BF16 copies of X and M_0
  float* tpart = nullptr;              // K-split partials of Y_0
};

}  // namespace

struct fctn_handle {
  fctn_params p;
  int N = 0;
  int64_t I[FCTN_MAX_ORDER] = {}, s[FCTN_MAX_ORDER] = {}, Pk[FCTN_MAX_ORDER] = {};
  int64_t P = 0;
  int R[FCTN_MAX_ORDER][FCTN_MAX_ORDER] = {};
  cudaStream_t st = nullptr;
  bool f64 = true;
  size_t esz = 8;
  // device state
  void* X = nullptr;
  uint32_t* bits = nullptr;
  double* A64[FCTN_MAX_ORDER] = {};
  void* Ac[FCTN_MAX_ORDER] = {};
  double* Q64[FCTN_MAX_ORDER] = {};
  float* Q32[FCTN_MAX_ORDER] = {};
  double* QT64[FCTN_MAX_ORDER] = {};  // Q^T (rows = eigenvectors), for the forward solve
  float* QT32[FCTN_MAX_ORDER] = {};
  double* Lam[FCTN_MAX_ORDER] = {};
  void* M = nullptr;              // merged tensor of the factor updated last (Algorithm 2 reuse)
  bool mat[FCTN_MAX_ORDER] = {};  // M_k is small enough to keep for the X update
  PairPlan pp[FCTN_MAX_ORDER];    // pair form of every M_k
  TcPlan tp[FCTN_MAX_ORDER];      // tensor-core Gram plan (TF32 / BF16)
  FactGram fg[FCTN_MAX_ORDER];    // Gram from the operand Grams (when cheaper)
  void* hbuf = nullptr;           // HL, HR of FactGram
  double* qwork = nullptr;        // fctn_quality partial sums (allocated on first use)
  size_t qwork_n = 0;
  // FactGram runs on a second stream, forked from and joined to `st`, so that
  // it overlaps the right-hand-side kernel (a parallel branch of the graph)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool tc = false;
  int* tabs = nullptr;            // device index tables of the pair forms
  void* ones = nullptr;           // the constant 1 (second operand when N = 2)
  void* Lbuf = nullptr;           // chain intermediate (no pair cache, N >= 4)
  void* T[2] = {nullptr, nullptr};
  int Tver[2][FCTN_MAX_ORDER] = {};  // versions of the members of each half when T was built
  bool Tvalid[2] = {false, false};
  void* chain[2] = {nullptr, nullptr};
  void* part = nullptr;
  double *Gd = nullptr, *Yd = nullptr, *Rd = nullptr, *Aprev = nullptr;
  void *Gs = nullptr, *Ys = nullptr, *C = nullptr, *Phi = nullptr, *W1 = nullptr, *Z = nullptr, *W2 = nullptr,
       *Rs = nullptr, *gwork = nullptr;
  int* status = nullptr;
  int* eig_used = nullptr;
  int eig_cap = 60;  // Jacobi sweep cap per eigendecomposition (fctn_params.eig_max_sweeps)
  float* eig_rec = nullptr;  // rotation blocks of the large FP32 eigensolver (128 < s <= 224)
  bool chol[FCTN_MAX_ORDER] = {};  // factor k solved by shifted Cholesky (FCTN_SOLVE_CHOL)
  float *cholL = nullptr, *cholD = nullptr;  // its packed factors and diagonal-block inverses
  float *cholRt = nullptr, *Alo = nullptr;   // Q^T R, and the low half of the double-float factor
  void* Ck[FCTN_MAX_ORDER] = {};
  bool cvalid[FCTN_MAX_ORDER] = {};
  double lam_min[FCTN_MAX_ORDER] = {};
  double *red = nullptr, *traces = nullptr, *stats = nullptr;
  void* stage = nullptr;
  uint8_t* stage_mask = nullptr;
  size_t stage_bytes = 0;
  // bookkeeping
  int64_t t = 0;
  int ver[FCTN_MAX_ORDER] = {};
  bool data_set = false, factors_set = false;
  int64_t launches = 0;
  std::vector<void*> allocs;
  // CUDA graphs: one executable graph per sweep signature; `dry` replays the
  // host bookkeeping of a sweep without launching (the graph does the work)
  bool use_graphs = true;
  bool dry = false;
  bool own_stream = false;
  struct GraphEnt {
    uint64_t key;
    cudaGraphExec_t exec;
  };
  std::vector<GraphEnt> graphs;
  // profiling: CUDA events around every launch of one kernel class
  int prof_class = -1;
  std::vector<cudaEvent_t> prof_ev;  // pairs
  size_t prof_used = 0;
  int64_t prof_launches = 0;
  double prof_ms = 0.0, prof_bytes = 0.0, prof_flops = 0.0;
  double cls_bytes = 0.0, cls_flops = 0.0;  // algorithmic counts of the class, since fctn_profile()
  int64_t cls_launches = 0;
  HeadRoute hr;  // head-mode association (FP32 / TF32 / BF16 with reuse and the plain order)
};

namespace {

int rank_of(const fctn_handle* h, int a, int b) { return h->R[a < b ? a : b][a < b ? b : a]; }

// Factor t, unfolded (I_t x s_t): labels [mode t, bonds (t,u) for u != t ascending].
View factor_view(const fctn_handle* h, int t) {
  Lab labs[FCTN_MAXD];
  int64_t ext[FCTN_MAXD];
  int n = 0;
  labs[n] = mode_lab(t);
  ext[n++] = h->I[t];
  for (int u = 0; u < h->N; ++u)
    if (u != t) {
      labs[n] = bond_lab(t, u);
      ext[n++] = rank_of(h, t, u);
    }
  return dense_view(n, labs, ext);
}

// Factor t in its FCTN (D1) layout: mode t at position t.
View factor_d1_view(const fctn_handle* h, int t) {
  Lab labs[FCTN_MAXD];
  int64_t ext[FCTN_MAXD];
  for (int u = 0; u < h->N; ++u) {
    labs[u] = (u == t) ? mode_lab(t) : bond_lab(t, u);
    ext[u] = (u == t) ? h->I[t] : rank_of(h, t, u);
  }
  return dense_view(h->N, labs, ext);
}

int make_plan(const View& A, const View* B, const Lab* out, int nout, ContractPlan* p, View* outv) {
  memset(p, 0, sizeof *p);
  if (nout > FCTN_MAXD) return fail(FCTN_E_UNSUPPORTED, "contraction output has %d indices (max %d)", nout, FCTN_MAXD);
  int64_t ext[FCTN_MAXD];
  for (int i = 0; i < nout; ++i) {
    int ia = A.find(out[i]);
    int ib = B ? B->find(out[i]) : -1;
    if (ia < 0 && ib < 0) return fail(FCTN_E_ARG, "output index not found in the operands");
    ext[i] = ia >= 0 ? A.ext[ia] : B->ext[ib];
    p->out_ext[i] = ext[i];
    p->a_str[i] = ia >= 0 ? A.str[ia] : 0;
    p->b_str[i] = ib >= 0 ? B->str[ib] : 0;
  }
  p->nout = nout;
  p->con_size = 1;
  if (B) {
    for (int i = 0; i < A.n; ++i) {
      bool in_out = false;
      for (int j = 0; j < nout; ++j) in_out |= (out[j] == A.lab[i]);
      if (in_out) continue;
      int ib = B->find(A.lab[i]);
      if (ib < 0) return fail(FCTN_E_ARG, "free index of A missing from the output");
      if (p->ncon >= FCTN_MAXC) return fail(FCTN_E_UNSUPPORTED, "too many contracted indices");
      p->con_ext[p->ncon] = A.ext[i];
      p->ca_str[p->ncon] = A.str[i];
      p->cb_str[p->ncon] = B->str[ib];
      p->con_size *= A.ext[i];
      p->ncon++;
    }
  }
  if (p->con_size > FCTN_CON_TABLE)
    return fail(FCTN_E_UNSUPPORTED, "contraction length %lld exceeds %d", (long long)p->con_size, FCTN_CON_TABLE);
  *outv = dense_view(nout, out, ext);
  p->out_size = outv->size();
  return FCTN_OK;
}

// Labels of A x B when the result keeps every unshared index (A's first);
// -1 (nothing written past out[FCTN_MAXD - 1]) if they would be more than FCTN_MAXD.
int joint_order(const View& A, const View& B, Lab* out) {
  int n = 0;
  for (int i = 0; i < A.n; ++i)
    if (B.find(A.lab[i]) < 0) {
      if (n >= FCTN_MAXD) return -1;
      out[n++] = A.lab[i];
    }
  for (int i = 0; i < B.n; ++i)
    if (A.find(B.lab[i]) < 0) {
      if (n >= FCTN_MAXD) return -1;
      out[n++] = B.lab[i];
    }
  return n;
}

// Profiling hooks around one launch of kernel class `cls` with algorithmic
// byte / flop counts (bytes, flops).
int prof_pre(fctn_handle* h, int cls, double bytes, double flops) {
  if (h->prof_class != cls) return FCTN_OK;
  h->cls_launches++;
  h->cls_bytes += bytes;
  h->cls_flops += flops;
  if (h->prof_used + 2 > h->prof_ev.size()) {
    for (int i = 0; i < 64; ++i) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      h->prof_ev.push_back(e);
    }
  }
  CK(cudaEventRecord(h->prof_ev[h->prof_used], h->st));
  return FCTN_OK;
}
int prof_post(fctn_handle* h, int cls) {
  if (h->prof_class != cls) return FCTN_OK;
  CK(cudaEventRecord(h->prof_ev[h->prof_used + 1], h->st));
  h->prof_used += 2;
  return FCTN_OK;
}

// LAUNCH(cls, bytes, flops, stmt): skip in dry mode, count, profile, check.
#define LAUNCH(cls, bytes, flops, stmt)                  \
  do {                                                    \
    if (h->dry) {                                         \
      h->launches++; /* replayed from the sweep graph */  \
    } else {                                              \
      int prc_ = prof_pre(h, (cls), (bytes), (flops));    \
      if (prc_) return prc_;                              \
      stmt;                                               \
      h->launches++;                                      \
      CK(cudaGetLastError());                             \
      prc_ = prof_post(h, (cls));                         \
      if (prc_) return prc_;                              \
    }                                                     \
  } while (0)
// The same for a launcher that issues n kernels on `strm` (outside the profiler).
#define LAUNCH_ON(n, stmt)                                \
  do {                                                    \
    if (!h->dry) {                                        \
      stmt;                                               \
      CK(cudaGetLastError());                             \
    }                                                     \
    h->launches += (n);                                   \
  } while (0)
#define LCHK()                  \
  do {                          \
    h->launches++;              \
    CK(cudaGetLastError());     \
  } while (0)

int launch_plan(fctn_handle* h, const void* A, const void* B, void* out, const ContractPlan& p) {
  const double bytes = (double)p.out_size * h->esz;
  const double flops = B ? 2.0 * (double)p.out_size * (double)p.con_size : 0.0;
  if (h->f64)
    LAUNCH(FCTN_KC_MERGED, bytes, flops,
           launch_contract_f64((const double*)A, (const double*)B, (double*)out, p, h->st));
  else
    LAUNCH(FCTN_KC_MERGED, bytes, flops,
           launch_contract_f32((const float*)A, (const float*)B, (float*)out, p, h->st));
  return FCTN_OK;
}

// Contract the factors `ids` (in this order) from scratch; the last step
// writes `dst` in the label order `final_order` (Algorithm 1's sequence).
int run_chain(fctn_handle* h, const int* ids, int nids, const Lab* final_order, int nfinal, void* dst) {
  View cur = factor_view(h, ids[0]);
  const void* curp = h->Ac[ids[0]];
  if (nids == 1) {
    ContractPlan p;
    View ov;
    int rc = make_plan(cur, nullptr, final_order, nfinal, &p, &ov);
    if (rc) return rc;
    return launch_plan(h, curp, nullptr, dst, p);
  }
  for (int i = 1; i < nids; ++i) {
    View nx = factor_view(h, ids[i]);
    Lab ord[FCTN_MAXD];
    int n;
    const bool last = (i == nids - 1);
    if (last) {
      n = nfinal;
      memcpy(ord, final_order, sizeof(Lab) * nfinal);
    } else {
      n = joint_order(cur, nx, ord);
      if (n < 0) return fail(FCTN_E_UNSUPPORTED, "chain intermediate has more than %d indices", FCTN_MAXD);
    }
    ContractPlan p;
    View ov;
    int rc = make_plan(cur, &nx, ord, n, &p, &ov);
    if (rc) return rc;
    void* o = last ? dst : h->chain[i % 2];
    rc = launch_plan(h, curp, h->Ac[ids[i]], o, p);
    if (rc) return rc;
    cur = ov;
    curp = o;
  }
  return FCTN_OK;
}

// Halves of the modes whose intermediates are shared (Algorithm 2; for
// N = 4 the pairs (1,2) and (3,4); for N >= 5 the generalisation of Table 2's
// reuse): half 0 = modes 0 .. N/2 - 1, half 1 = the rest.  Every M_k of one
// half contracts the other half's intermediate with its own half's other
// factors.
int half_lo(const fctn_handle* h, int q) { return q == 0 ? 0 : h->N / 2; }
int half_hi(const fctn_handle* h, int q) { return q == 0 ? h->N / 2 : h->N; }
int half_of(const fctn_handle* h, int k) { return k < h->N / 2 ? 0 : 1; }

// The members of k's own half except k; returns their count.
int own_others(const fctn_handle* h, int k, int* ids) {
  const int q = half_of(h, k);
  int n = 0;
  for (int u = half_lo(h, q); u < half_hi(h, q); ++u)
    if (u != k) ids[n++] = u;
  return n;
}

// Intermediate of half q: its modes ascending, then for every member u
// (ascending) its bonds (u, v) to the other half, v ascending.
View half_out_view(const fctn_handle* h, int q, Lab* ord, int* n) {
  int m = 0;
  const int lo = half_lo(h, q), hi = half_hi(h, q);
  for (int u = lo; u < hi; ++u) ord[m++] = mode_lab(u);
  for (int u = lo; u < hi; ++u)
    for (int v = 0; v < h->N; ++v)
      if (v < lo || v >= hi) ord[m++] = bond_lab(u, v);
  *n = m;
  int64_t ext[FCTN_MAXD];
  for (int i = 0; i < m; ++i) ext[i] = ord[i].kind == 0 ? h->I[ord[i].a] : rank_of(h, ord[i].a, ord[i].b);
  return dense_view(m, ord, ext);
}
bool reuse_pairs(const fctn_handle* h) { return h->p.reuse && h->N >= 4; }

// The cached intermediate of half q is current (built from the members' present versions).
bool half_valid(const fctn_handle* h, int q) {
  if (!h->Tvalid[q]) return false;
  for (int u = half_lo(h, q); u < half_hi(h, q); ++u)
    if (h->Tver[q][u - half_lo(h, q)] != h->ver[u]) return false;
  return true;
}

// Sizes of every intermediate of the chains (for allocation).
int64_t chain_need(const fctn_handle* h) {
  int64_t need = 0;
  bool too_many = false;
  auto sim = [&](const int* ids, int nids) {
    View cur = factor_view(h, ids[0]);
    for (int i = 1; i < nids - 1; ++i) {
      View nx = factor_view(h, ids[i]);
      Lab ord[FCTN_MAXD];
      int n = joint_order(cur, nx, ord);
      if (n < 0) {
        too_many = true;
        return;
      }
      int64_t ext[FCTN_MAXD];
      for (int j = 0; j < n; ++j) {
        int ia = cur.find(ord[j]);
        ext[j] = ia >= 0 ? cur.ext[ia] : nx.ext[nx.find(ord[j])];
      }
      cur = dense_view(n, ord, ext);
      if (cur.size() > need) need = cur.size();
    }
  };
  int ids[FCTN_MAX_ORDER];
  for (int k = 0; k < h->N; ++k) {
    int c = 0;
    for (int t = 0; t < h->N; ++t)
      if (t != k) ids[c++] = t;
    sim(ids, c);
  }
  for (int t = 0; t < h->N; ++t) ids[t] = t;
  sim(ids, h->N);
  if (reuse_pairs(h)) {  // half intermediates and the own-half chains
    for (int q = 0; q < 2; ++q) {
      int m = 0;
      for (int u = half_lo(h, q); u < half_hi(h, q); ++u) ids[m++] = u;
      sim(ids, m);
    }
    for (int k = 0; k < h->N; ++k) sim(ids, own_others(h, k, ids));
  }
  return too_many ? -1 : need;
}

// Pair intermediates of Algorithm 2 (N = 4): index 0 = (A_1, A_2), 1 = (A_3, A_4).
int64_t view_row(const View& v) {
  int64_t r = 1;
  for (int i = 0; i < v.n; ++i)
    if (v.lab[i].kind == 1) r *= v.ext[i];
  return r;
}

// Others of k except the last one (contracted in ascending order into L when
// there is no pair cache); *last_other gets the remaining one (operand R).
void chain_ids(const fctn_handle* h, int k, int* ids, int* n, int* last_other) {
  int c = 0, lo = -1;
  for (int t = 0; t < h->N; ++t)
    if (t != k) { ids[c++] = t; lo = t; }
  *n = c - 1;
  *last_other = lo;
}

// View of the chain product of `ids`: physical modes first (ascending), then bonds.
View chain_result_view(const fctn_handle* h, const int* ids, int nids, Lab* ord, int* nord) {
  View cur = factor_view(h, ids[0]);
  for (int i = 1; i < nids; ++i) {
    View nx = factor_view(h, ids[i]);
    Lab o[FCTN_MAXD];
    int n = joint_order(cur, nx, o);
    if (n < 0) n = 0;  // unreachable: check_params bounds every chain by FCTN_MAXD labels
    int64_t ext[FCTN_MAXD];
    for (int q = 0; q < n; ++q) {
      int ia = cur.find(o[q]);
      ext[q] = ia >= 0 ? cur.ext[ia] : nx.ext[nx.find(o[q])];
    }
    cur = dense_view(n, o, ext);
  }
  Lab o2[FCTN_MAXD];
  int64_t e2[FCTN_MAXD];
  int m = 0;
  for (int t = 0; t < h->N; ++t) {
    int i = cur.find(mode_lab(t));
    if (i >= 0) { o2[m] = cur.lab[i]; e2[m++] = cur.ext[i]; }
  }
  for (int i = 0; i < cur.n; ++i)
    if (cur.lab[i].kind == 1) { o2[m] = cur.lab[i]; e2[m++] = cur.ext[i]; }
  memcpy(ord, o2, sizeof(Lab) * m);
  *nord = m;
  return dense_view(m, o2, e2);
}

// Operand views of M_k's pair form (L x R).
void pair_operands(const fctn_handle* h, int k, View* L, View* R) {
  const int N = h->N;
  if (N == 2) {
    *L = factor_view(h, 1 - k);
    R->n = 0;
    return;
  }
  if (N == 3) {
    int a = -1, b = -1;
    for (int t = 0; t < 3; ++t)
      if (t != k) { if (a < 0) a = t; else b = t; }
    *L = factor_view(h, a);
    *R = factor_view(h, b);
    return;
  }
  if (reuse_pairs(h)) {
    const int o = 1 - half_of(h, k);
    int ids[FCTN_MAX_ORDER];
    const int n = own_others(h, k, ids);
    Lab ord[FCTN_MAXD];
    int no;
    *R = half_out_view(h, o, ord, &no);
    *L = n == 1 ? factor_view(h, ids[0]) : chain_result_view(h, ids, n, ord, &no);
    return;
  }
  int ids[FCTN_MAX_ORDER], n, lo;
  chain_ids(h, k, ids, &n, &lo);
  Lab ord[FCTN_MAXD];
  int no;
  *L = chain_result_view(h, ids, n, ord, &no);
  *R = factor_view(h, lo);
}

// Index tables of M_k = L x R in the canonical order (bonds (k,t), modes t).
int plan_pair(const fctn_handle* h, int k, const View& L, const View& R, PairPlan* pp, std::vector<int>* tab) {
  memset(pp, 0, sizeof *pp);
  const int N = h->N;
  const int64_t s = h->s[k];
  int nsg = 0;
  int64_t sext[FCTN_MAX_ORDER], slstr[FCTN_MAX_ORDER], srstr[FCTN_MAX_ORDER];
  for (int t = 0; t < N; ++t) {
    if (t == k) continue;
    Lab b = bond_lab(k, t);
    int il = L.find(b), ir = R.find(b);
    if ((il >= 0) == (ir >= 0)) return fail(FCTN_E_STATE, "bond (%d,%d) must belong to exactly one operand", k, t);
    sext[nsg] = rank_of(h, k, t);
    slstr[nsg] = il >= 0 ? L.str[il] : 0;
    srstr[nsg] = ir >= 0 ? R.str[ir] : 0;
    nsg++;
  }
  pp->nd = 0;
  for (int t = 0; t < N; ++t) {
    if (t == k) continue;
    Lab m = mode_lab(t);
    int il = L.find(m), ir = R.find(m);
    if ((il >= 0) == (ir >= 0)) return fail(FCTN_E_STATE, "mode %d must belong to exactly one operand", t);
    pp->ext[pp->nd] = h->I[t];
    pp->lstr[pp->nd] = il >= 0 ? L.str[il] : 0;
    pp->rstr[pp->nd] = ir >= 0 ? R.str[ir] : 0;
    pp->nd++;
  }
  int nk = 0;
  int64_t kext[FCTN_MAXD], klstr[FCTN_MAXD], krstr[FCTN_MAXD];
  int64_t K = 1;
  for (int i = 0; i < L.n; ++i) {
    if (L.lab[i].kind != 1) continue;
    int ir = R.find(L.lab[i]);
    if (ir < 0) {
      if (!(L.lab[i].a == k || L.lab[i].b == k)) return fail(FCTN_E_STATE, "dangling bond in the left operand");
      continue;
    }
    kext[nk] = L.ext[i];
    klstr[nk] = L.str[i];
    krstr[nk] = R.str[ir];
    K *= L.ext[i];
    nk++;
  }
  if (K > 4096) return fail(FCTN_E_UNSUPPORTED, "pair contraction length %lld too large", (long long)K);
  pp->K = (int)K;
  pp->Ljs = (int)view_row(L);
  pp->Rjs = R.n ? (int)view_row(R) : 1;
  tab->assign((size_t)(2 * s + 2 * K), 0);
  for (int64_t sg = 0; sg < s; ++sg) {
    int64_t r = sg, lo = 0, ro = 0;
    for (int d = nsg - 1; d >= 0; --d) {
      int64_t dig = r % sext[d];
      r /= sext[d];
      lo += dig * slstr[d];
      ro += dig * srstr[d];
    }
    (*tab)[sg] = (int)lo;
    (*tab)[s + sg] = (int)ro;
  }
  for (int64_t q = 0; q < K; ++q) {
    int64_t r = q, lo = 0, ro = 0;
    for (int d = nk - 1; d >= 0; --d) {
      int64_t dig = r % kext[d];
      r /= kext[d];
      lo += dig * klstr[d];
      ro += dig * krstr[d];
    }
    (*tab)[2 * s + q] = (int)lo;
    (*tab)[2 * s + K + q] = (int)ro;
  }
  return FCTN_OK;
}

// Make M_k's pair operands current (pair cache / chain intermediate) and
// return their device pointers.
int prepare_pair(fctn_handle* h, int k, const void** L, const void** R) {
  const int N = h->N;
  if (N == 2) {
    *L = h->Ac[1 - k];
    *R = h->ones;
    return FCTN_OK;
  }
  if (N == 3) {
    int a = -1, b = -1;
    for (int t = 0; t < 3; ++t)
      if (t != k) { if (a < 0) a = t; else b = t; }
    *L = h->Ac[a];
    *R = h->Ac[b];
    return FCTN_OK;
  }
  if (reuse_pairs(h)) {
    const int o = 1 - half_of(h, k);
    if (!half_valid(h, o)) {
      Lab ord[FCTN_MAXD];
      int n;
      half_out_view(h, o, ord, &n);
      int ids[FCTN_MAX_ORDER], m = 0;
      for (int u = half_lo(h, o); u < half_hi(h, o); ++u) ids[m++] = u;
      int rc = run_chain(h, ids, m, ord, n, h->T[o]);
      if (rc) return rc;
      h->Tvalid[o] = true;
      for (int u = half_lo(h, o); u < half_hi(h, o); ++u) h->Tver[o][u - half_lo(h, o)] = h->ver[u];
    }
    int ids[FCTN_MAX_ORDER];
    const int n = own_others(h, k, ids);
    if (n == 1) {
      *L = h->Ac[ids[0]];
    } else {
      Lab ord[FCTN_MAXD];
      int no;
      chain_result_view(h, ids, n, ord, &no);
      int rc = run_chain(h, ids, n, ord, no, h->Lbuf);
      if (rc) return rc;
      *L = h->Lbuf;
    }
    *R = h->T[o];
    return FCTN_OK;
  }
  int ids[FCTN_MAX_ORDER], n, lo;
  chain_ids(h, k, ids, &n, &lo);
  Lab ord[FCTN_MAXD];
  int no;
  chain_result_view(h, ids, n, ord, &no);
  int rc = run_chain(h, ids, n, ord, no, h->Lbuf);
  if (rc) return rc;
  *L = h->Lbuf;
  *R = h->Ac[lo];
  return FCTN_OK;
}

GramPlan gram_plan(const fctn_handle* h, int k) {
  GramPlan g;
  g.s = h->s[k];
  g.I = h->I[k];
  g.Pk = h->Pk[k];
  int64_t pre = 1, post = 1;
  for (int t = 0; t < k; ++t) pre *= h->I[t];
  for (int t = k + 1; t < h->N; ++t) post *= h->I[t];
  g.xv = ModeView{pre, h->I[k], post};
  g.gcols = h->fg[k].use ? 0 : g.s;
  g.ncols = g.gcols + g.I;
  g.tiles_r = (int)((g.s + 63) / 64);
  g.tiles_c = (int)((g.ncols + 63) / 64);
  int64_t ctas_per_split = g.tiles_r * g.tiles_c;
  if (h->tc) ctas_per_split = h->tp[k].n_groups > 0 ? h->tp[k].n_groups : 1;
  // CTAs of the right-hand-side kernel: the tuned budget, else about 2 per
  // SM, or 96 with the factored Gram (whose eigensolver runs beside it on
  // the side branch), so that SMs stay free for that branch
  const int64_t ctas = h->p.rhs_ctas > 0 ? h->p.rhs_ctas : (h->fg[k].use ? 96 : 2 * 152);
  int64_t target = (ctas + ctas_per_split - 1) / ctas_per_split;
  // tensor-core path: at least two 32-column chunks per CTA, so the per-split
  // partial (s x (s + I) floats) stays small against the columns it consumes
  int64_t maxsplit = h->tc ? (g.Pk + 63) / 64 : (g.Pk + 31) / 32;
  int64_t ks = target < maxsplit ? target : maxsplit;
  if (ks < 1) ks = 1;
  int64_t chunk = (g.Pk + ks - 1) / ks;
  chunk = (chunk + 31) / 32 * 32;
  g.kchunk = chunk;
  g.ksplit = (int)((g.Pk + chunk - 1) / chunk);
  return g;
}

int check_params(const fctn_params* p) {
  if (!p) return fail(FCTN_E_ARG, "params is NULL");
  if (p->order < 2 || p->order > FCTN_MAX_ORDER) return fail(FCTN_E_ARG, "order %d outside [2, %d]", p->order, FCTN_MAX_ORDER);
  if (p->precision < FCTN_FP64 || p->precision > FCTN_BF16) return fail(FCTN_E_ARG, "unknown precision %d", p->precision);
  if (p->order_policy != FCTN_ORDER_PLAIN && p->order_policy != FCTN_ORDER_ALTERNATE)
    return fail(FCTN_E_ARG, "unknown order policy %d", p->order_policy);
  if (p->laplacian_sign != FCTN_LAPLACIAN_PSD && p->laplacian_sign != FCTN_LAPLACIAN_PRINTED)
    return fail(FCTN_E_ARG, "unknown laplacian sign %d", p->laplacian_sign);
  if (p->gram_mode < FCTN_GRAM_AUTO || p->gram_mode > FCTN_GRAM_FACTORED)
    return fail(FCTN_E_ARG, "unknown gram mode %d", p->gram_mode);
  if (p->refine_steps < 0 || p->refine_steps > 8) return fail(FCTN_E_ARG, "refine_steps %d outside [0, 8]", p->refine_steps);
  if (p->rhs_ctas < 0 || p->rhs_ctas > 16 * 152) return fail(FCTN_E_ARG, "rhs_ctas %d outside [0, 2432]", p->rhs_ctas);
  if (p->eig_max_sweeps < 0 || p->eig_max_sweeps > 1000)
    return fail(FCTN_E_ARG, "eig_max_sweeps %d outside [0, 1000]", p->eig_max_sweeps);
  if (!(p->eig_tol >= 0.0 && p->eig_tol < 1.0)) return fail(FCTN_E_ARG, "eig_tol must lie in [0, 1)");
  if (!(p->finish_fp32_at >= 0.0)) return fail(FCTN_E_ARG, "finish_fp32_at must be >= 0");
  if (p->tile_code < 0 || p->tile_code > 255) return fail(FCTN_E_ARG, "tile_code %d outside [0, 255]", p->tile_code);
  if (p->solve_method < FCTN_SOLVE_AUTO || p->solve_method > FCTN_SOLVE_CHOL)
    return fail(FCTN_E_ARG, "unknown solve method %d", p->solve_method);
  if (!(p->rho > 0)) return fail(FCTN_E_ARG, "rho must be > 0");
  for (int k = 0; k < p->order; ++k) {
    if (p->dims[k] < 1 || p->dims[k] > (1 << 24)) return fail(FCTN_E_ARG, "dims[%d] = %lld out of range", k, (long long)p->dims[k]);
    if (!(p->lambda[k] >= 0) || !(p->delta[k] >= 0)) return fail(FCTN_E_ARG, "lambda/delta[%d] must be >= 0", k);
    for (int t = k + 1; t < p->order; ++t)
      if (p->ranks[k][t] < 1 || p->ranks[k][t] > 64) return fail(FCTN_E_ARG, "rank R[%d][%d] = %d out of range", k, t, p->ranks[k][t]);
  }
  if (p->solve_method == FCTN_SOLVE_CHOL) {
    if (p->precision == FCTN_FP64) return fail(FCTN_E_UNSUPPORTED, "the Cholesky solve is FP32 (precision FP64 given)");
    for (int k = 0; k < p->order; ++k) {
      int64_t sk = 1;
      for (int t = 0; t < p->order; ++t)
        if (t != k) sk *= p->ranks[k < t ? k : t][k < t ? t : k];
      if (!chol_supported((int)(sk > (1 << 20) ? (1 << 20) : sk)))
        return fail(FCTN_E_UNSUPPORTED, "the Cholesky solve needs s_k <= 256 (s_%d = %lld)", k, (long long)sk);
    }
  }
  // every chain intermediate of m factors has m (N - m + 1) labels at most
  for (int m = 1; m <= p->order; ++m)
    if (m * (p->order - m + 1) > FCTN_MAXD)
      return fail(FCTN_E_UNSUPPORTED, "order %d: chain intermediates exceed %d indices", p->order, FCTN_MAXD);
  return FCTN_OK;
}

void fill_shapes(fctn_handle* h, const fctn_params* p) {
  h->p = *p;
  h->N = p->order;
  h->P = 1;
  for (int k = 0; k < h->N; ++k) {
    h->I[k] = p->dims[k];
    h->P *= p->dims[k];
    for (int t = k + 1; t < h->N; ++t) h->R[k][t] = h->R[t][k] = p->ranks[k][t];
  }
  for (int k = 0; k < h->N; ++k) {
    h->Pk[k] = h->P / h->I[k];
    int64_t s = 1;
    for (int t = 0; t < h->N; ++t)
      if (t != k) s *= h->R[k][t];
    h->s[k] = s;
  }
  h->f64 = (p->precision == FCTN_FP64);
  h->esz = h->f64 ? 8 : 4;
  h->tc = (p->precision == FCTN_TF32 || p->precision == FCTN_BF16);
  h->eig_cap = p->eig_max_sweeps > 0 ? p->eig_max_sweeps : 60;
  for (int k = 0; k < h->N; ++k)
    h->chol[k] = !h->f64 && p->solve_method != FCTN_SOLVE_EIG && chol_supported((int)h->s[k]);
}

// Floats of the shared Cholesky buffers (factors, diagonal-block inverses).
void chol_floats(const fctn_handle* h, size_t* nl, size_t* nd) {
  *nl = 0;
  *nd = 0;
  for (int k = 0; k < h->N; ++k)
    if (h->chol[k]) {
      *nl = std::max(*nl, chol_factor_floats((int)h->I[k], (int)h->s[k]));
      *nd = std::max(*nd, chol_dinv_floats((int)h->I[k], (int)h->s[k]));
    }
}

struct Sizes {
  int64_t M, chain, T[2], part, Is, ss, maxI, maxs, maxfac, red_blocks, lbuf, hbuf;
};

// M_k is kept for the X update (Algorithm 2) when it takes at most 64 MB:
// it then stays in L2 between its write and its read.  Larger merged tensors
// are formed again on chip by the X update instead of a round trip through HBM.
bool materialise_ok(const fctn_handle* h, int k) { return (double)h->s[k] * h->Pk[k] * h->esz <= 64.0 * 1024 * 1024; }

int64_t lbuf_need(const fctn_handle* h) {
  if (h->N < 4) return 0;
  int64_t need = 0;
  if (reuse_pairs(h)) {  // the own-half chains of M_k (more than one other member: N >= 5)
    for (int k = 0; k < h->N; ++k) {
      int ids[FCTN_MAX_ORDER];
      const int n = own_others(h, k, ids);
      if (n < 2) continue;
      Lab ord[FCTN_MAXD];
      int no;
      int64_t sz = chain_result_view(h, ids, n, ord, &no).size();
      if (sz > need) need = sz;
    }
    return need;
  }
  for (int k = 0; k < h->N; ++k) {
    int ids[FCTN_MAX_ORDER], n, lo;
    chain_ids(h, k, ids, &n, &lo);
    Lab ord[FCTN_MAXD];
    int no;
    int64_t sz = chain_result_view(h, ids, n, ord, &no).size();
    if (sz > need) need = sz;
  }
  return need;
}

// Host-only planning of every factor's pair form (and its index tables) and,
// for the tensor-core precisions, of the tcgen05 Gram kernel.
// Factored Gram of M_k (FactGram) from its pair plan: rows sigma split into
// the distinct L and R row offsets, the F_L / F_R row offsets and column
// offsets.  FCTN_GRAM_AUTO uses it outside FP64 when its multiply-adds,
// (nL K)^2 JL + (nR K)^2 JR + s^2 K^2, are fewer than the s^2 P_k of the
// direct Gram (by 8x against the tensor-core Gram, whose multiply-adds run at
// a higher rate).
void plan_fact(const fctn_handle* h, int k, const PairPlan& pp, const std::vector<int>& tab, FactGram* f,
               std::vector<int>* ftab) {
  memset(f, 0, sizeof *f);
  ftab->clear();
  const int s = (int)h->s[k], K = pp.K;
  std::vector<int> uL, uR, a(s), b(s);
  for (int sg = 0; sg < s; ++sg) {
    const int lo = tab[sg], ro = tab[s + sg];
    int ia = -1, ib = -1;
    for (int i = 0; i < (int)uL.size(); ++i)
      if (uL[i] == lo) ia = i;
    if (ia < 0) { ia = (int)uL.size(); uL.push_back(lo); }
    for (int i = 0; i < (int)uR.size(); ++i)
      if (uR[i] == ro) ib = i;
    if (ib < 0) { ib = (int)uR.size(); uR.push_back(ro); }
    a[sg] = ia;
    b[sg] = ib;
  }
  const int nL = (int)uL.size(), nR = (int)uR.size();
  if ((int64_t)nL * nR != s) return;
  // the column digits held by each operand
  int64_t JL = 1, JR = 1;
  int ndl = 0, ndr = 0;
  int64_t el[FCTN_MAX_ORDER], sl[FCTN_MAX_ORDER], er[FCTN_MAX_ORDER], sr[FCTN_MAX_ORDER];
  for (int d = 0; d < pp.nd; ++d) {
    if (pp.lstr[d] != 0) { el[ndl] = pp.ext[d]; sl[ndl++] = pp.lstr[d]; JL *= pp.ext[d]; }
    else { er[ndr] = pp.ext[d]; sr[ndr++] = pp.rstr[d]; JR *= pp.ext[d]; }
  }
  const int64_t rl = (int64_t)nL * K, rr = (int64_t)nR * K;
  if (rl > 4096 || rr > 4096 || JL > (1 << 24) || JR > (1 << 24)) return;
  const double fact = (double)rl * rl * JL + (double)rr * rr * JR + (double)s * s * K * K;
  const double direct = (double)s * s * h->Pk[k];
  if (h->p.gram_mode == FCTN_GRAM_DIRECT) return;
  if (h->p.gram_mode == FCTN_GRAM_AUTO && (h->f64 || fact * (h->tc ? 8.0 : 1.0) >= direct)) return;
  f->use = 1;
  f->nL = nL;
  f->nR = nR;
  f->K = K;
  f->rl = (int)rl;
  f->rr = (int)rr;
  f->JL = (int)JL;
  f->JR = (int)JR;
  const int* lk = tab.data() + 2 * s;
  const int* rk = lk + K;
  for (int i = 0; i < nL; ++i)
    for (int q = 0; q < K; ++q) ftab->push_back(uL[i] + lk[q]);
  for (int i = 0; i < nR; ++i)
    for (int q = 0; q < K; ++q) ftab->push_back(uR[i] + rk[q]);
  ftab->insert(ftab->end(), a.begin(), a.end());
  ftab->insert(ftab->end(), b.begin(), b.end());
  auto cols = [&](int nd, const int64_t* ext, const int64_t* str, int64_t J) {
    for (int64_t j = 0; j < J; ++j) {
      int64_t r = j, o = 0;
      for (int d = nd - 1; d >= 0; --d) {
        o += (r % ext[d]) * str[d];
        r /= ext[d];
      }
      ftab->push_back((int)o);
    }
  };
  cols(ndl, el, sl, JL);
  cols(ndr, er, sr, JR);
}

int plan_all(fctn_handle* h, std::vector<int>* all, size_t* offs) {
  if (chain_need(h) < 0) return fail(FCTN_E_UNSUPPORTED, "a chain intermediate has more than %d indices", FCTN_MAXD);
  for (int k = 0; k < h->N; ++k) {
    View L, R;
    pair_operands(h, k, &L, &R);
    std::vector<int> tab;
    int rc = plan_pair(h, k, L, R, &h->pp[k], &tab);
    if (rc) return rc;
    if (offs) offs[k] = all->size();
    all->insert(all->end(), tab.begin(), tab.end());
    std::vector<int> ftab;
    plan_fact(h, k, h->pp[k], tab, &h->fg[k], &ftab);
    if (offs) offs[FCTN_MAX_ORDER + k] = all->size();
    all->insert(all->end(), ftab.begin(), ftab.end());
    h->mat[k] = h->p.reuse && materialise_ok(h, k) && !h->hr.on;
    if (h->tc && !h->hr.on) {
      h->tp[k].n_groups = 0;
      GramPlan g = gram_plan(h, k);
      rc = tc_plan(h->pp[k], g, h->p.precision, &h->tp[k]);
      if (rc) return fail(rc, "tensor-core Gram kernel does not cover factor %d (s_k = %lld)", k, (long long)h->s[k]);
    }
  }
  return FCTN_OK;
}

// ---- head-mode association: planning ---------------------------------------
// Second copy of a bond in a Gram H_t = A_(t)^T A_(t) (kind 2).
Lab pbond_lab(int x, int y) { return Lab{2, x < y ? x : y, x < y ? y : x}; }

// Mixed-radix offsets: for every index e over the digits (last fastest),
// o1[e] = sum digit * s1, o2[e] = sum digit * s2.
void radix_offsets(int nd, const int64_t* ext, const int64_t* s1, const int64_t* s2, int* o1, int* o2) {
  int64_t total = 1;
  for (int d = 0; d < nd; ++d) total *= ext[d];
  for (int64_t e = 0; e < total; ++e) {
    int64_t r = e, a = 0, b = 0;
    for (int d = nd - 1; d >= 0; --d) {
      const int64_t dig = r % ext[d];
      r /= ext[d];
      a += dig * s1[d];
      b += dig * s2[d];
    }
    o1[e] = (int)a;
    o2[e] = (int)b;
  }
}

int64_t max_offset(const View& v) {
  int64_t o = 0;
  for (int i = 0; i < v.n; ++i) o += (v.ext[i] - 1) * v.str[i];
  return o;
}

// Plan C = A (x) B (every shared label contracted) with C laid out as `C`.
// The operand that holds C's innermost label plays B, so that consecutive
// columns n are consecutive in C; except for small outputs with one side
// under 64 (the chains' 36-wide bond pairs), where the wide side plays M so
// that the narrow one pads a 64-column tile rather than a 128-row one.
int sg_plan(const View& A0, const View& B0, const View& C, SgPlanH* out, std::vector<int>* tabs, int split = 0) {
  bool swap = C.n > 0 && A0.find(C.lab[C.n - 1]) >= 0;
  {
    int64_t ma0 = 1, nb0 = 1;
    for (int i = 0; i < C.n; ++i) (A0.find(C.lab[i]) >= 0 ? ma0 : nb0) *= C.ext[i];
    if (ma0 * nb0 <= ((int64_t)1 << 22) && (ma0 < 64 || nb0 < 64) && ma0 != nb0) swap = ma0 < nb0;
  }
  const View& A = swap ? B0 : A0;
  const View& B = swap ? A0 : B0;
  int64_t mext[FCTN_MAXD], ma[FCTN_MAXD], mc[FCTN_MAXD], next[FCTN_MAXD], nb[FCTN_MAXD], nc[FCTN_MAXD];
  int64_t kext[FCTN_MAXD], ka[FCTN_MAXD], kbs[FCTN_MAXD];
  int nm = 0, nn = 0, nk = 0;
  int64_t M = 1, Nn = 1, K = 1;
  for (int i = 0; i < C.n; ++i) {
    const int ia = A.find(C.lab[i]), ib = B.find(C.lab[i]);
    if ((ia >= 0) == (ib >= 0)) return fail(FCTN_E_STATE, "contraction plan: output index in both or neither operand");
    if (ia >= 0) {
      mext[nm] = C.ext[i], ma[nm] = A.str[ia], mc[nm++] = C.str[i];
      M *= C.ext[i];
    } else {
      next[nn] = C.ext[i], nb[nn] = B.str[ib], nc[nn++] = C.str[i];
      Nn *= C.ext[i];
    }
  }
  for (int i = 0; i < A.n; ++i) {
    if (C.find(A.lab[i]) >= 0) continue;
    const int ib = B.find(A.lab[i]);
    if (ib < 0) return fail(FCTN_E_STATE, "contraction plan: free index missing from the output");
    kext[nk] = A.ext[i], ka[nk] = A.str[i], kbs[nk++] = B.str[ib];
    K *= A.ext[i];
  }
  for (int i = 0; i < B.n; ++i)
    if (C.find(B.lab[i]) < 0 && A.find(B.lab[i]) < 0)
      return fail(FCTN_E_STATE, "contraction plan: free index missing from the output");
  const int64_t lim = (int64_t)1 << 31;
  if (M >= lim || Nn >= lim || K >= lim || max_offset(A) >= lim || max_offset(B) >= lim || max_offset(C) >= lim)
    return fail(FCTN_E_UNSUPPORTED, "contraction plan: a tensor of the sweep exceeds 2^31 elements");
  out->swap = swap;
  out->tab = tabs->size();
  tabs->resize(out->tab + (size_t)(2 * M + 2 * Nn + 2 * K));
  int* am = tabs->data() + out->tab;
  int* cm = am + M;
  int* bn = cm + M;
  int* cn = bn + Nn;
  int* ak = cn + Nn;
  int* bk = ak + K;
  radix_offsets(nm, mext, ma, mc, am, cm);
  radix_offsets(nn, next, nb, nc, bn, cn);
  radix_offsets(nk, kext, ka, kbs, ak, bk);
  sg_shape((int)M, (int)Nn, (int)K, &out->sh, split);
  // loader lanes: along k when A's (B's) innermost contracted digit is
  // contiguous, else along m (n) when that digit is
  out->sh.a_mfast = (nk == 0 || ka[nk - 1] != 1) && nm > 0 && ma[nm - 1] == 1;
  out->sh.b_nfast = (nk == 0 || kbs[nk - 1] != 1) && nn > 0 && nb[nn - 1] == 1;
  return FCTN_OK;
}

View x_view(const fctn_handle* h) {
  Lab l[FCTN_MAXD];
  int64_t e[FCTN_MAXD];
  for (int t = 0; t < h->N; ++t) l[t] = mode_lab(t), e[t] = h->I[t];
  return dense_view(h->N, l, e);
}
// M_0 (s_0 x P_0): bonds (0, t) ascending, then modes 1 .. N-1.
View m0_view(const fctn_handle* h) {
  Lab l[FCTN_MAXD];
  int64_t e[FCTN_MAXD];
  int n = 0;
  for (int t = 1; t < h->N; ++t) l[n] = bond_lab(0, t), e[n++] = rank_of(h, 0, t);
  for (int t = 1; t < h->N; ++t) l[n] = mode_lab(t), e[n++] = h->I[t];
  return dense_view(n, l, e);
}
// Z = X_(0)^T A_(0) (P_0 x s_0): modes 1 .. N-1, then bonds (0, t).
View z_view(const fctn_handle* h) {
  Lab l[FCTN_MAXD];
  int64_t e[FCTN_MAXD];
  int n = 0;
  for (int t = 1; t < h->N; ++t) l[n] = mode_lab(t), e[n++] = h->I[t];
  for (int t = 1; t < h->N; ++t) l[n] = bond_lab(0, t), e[n++] = rank_of(h, 0, t);
  return dense_view(n, l, e);
}
// Gram of factor t's bonds (s_t x s_t): bonds (t, u) ascending, then their second copies.
View hgram_view(const fctn_handle* h, int t) {
  Lab l[FCTN_MAXD];
  int64_t e[FCTN_MAXD];
  int n = 0;
  for (int u = 0; u < h->N; ++u)
    if (u != t) l[n] = bond_lab(t, u), e[n++] = rank_of(h, t, u);
  for (int u = 0; u < h->N; ++u)
    if (u != t) l[n] = pbond_lab(t, u), e[n++] = rank_of(h, t, u);
  return dense_view(n, l, e);
}
// Factor t with its bonds relabelled as second copies.
View factor_primed_view(const fctn_handle* h, int t) {
  View v = factor_view(h, t);
  for (int i = 0; i < v.n; ++i)
    if (v.lab[i].kind == 1) v.lab[i].kind = 2;
  return v;
}
View joint_view(const View& a, const View& b, int* rc) {
  Lab o[FCTN_MAXD];
  int64_t e[FCTN_MAXD];
  const int n = joint_order(a, b, o);
  if (n < 0) {
    *rc = FCTN_E_UNSUPPORTED;
    return View{};
  }
  for (int q = 0; q < n; ++q) {
    const int ia = a.find(o[q]);
    e[q] = ia >= 0 ? a.ext[ia] : b.ext[b.find(o[q])];
  }
  return dense_view(n, o, e);
}

// Decide and plan the head-mode association (FP32 / TF32 / BF16 with reuse,
// the plain order (N = 3 has only one order), N >= 3); the old route stays in
// place otherwise.  Intermediates larger than 2^28 elements turn it off.
int plan_route(fctn_handle* h, std::vector<int>* tabs) {
  HeadRoute& r = h->hr;
  r = HeadRoute{};
  const int N = h->N;
  r.on = !h->f64 && h->p.reuse && N >= 3 && (h->p.order_policy == FCTN_ORDER_PLAIN || N == 3);
  if (!r.on) return FCTN_OK;
  r.s0 = h->s[0];
  r.P0 = h->Pk[0];
  int rc = FCTN_OK;
  std::vector<int> t0;  // tables of this plan (appended at the end, or dropped)
  // tile code (fctn_autotune_tiles): K-split target of the table-driven
  // contractions (CUDA-core and tensor-core)
  static const int kSgSplit[4] = {0, 152, 4 * 152, 1};
  const int sgs = kSgSplit[(h->p.tile_code >> 5) & 3];
  auto track = [](int64_t* mx, int64_t v) { *mx = v > *mx ? v : *mx; };
  // M_0: factors 1 .. N-1, greedily in the order that keeps the chain
  // intermediates smallest (the pair with the smallest joint tensor first:
  // for 256x256x31x8, A_(2) (x) A_(3) is 1.3 MB where A_(1) (x) A_(2) is 41 MB)
  {
    int order[FCTN_MAX_ORDER], n = 0;
    bool used[FCTN_MAX_ORDER] = {};
    int64_t best = -1;
    for (int a = 1; a < N; ++a)
      for (int b = a + 1; b < N; ++b) {
        int rcj = FCTN_OK;
        const int64_t sz = N == 3 ? 0 : joint_view(factor_view(h, a), factor_view(h, b), &rcj).size();
        if (rcj == FCTN_OK && (best < 0 || sz < best)) {
          best = sz;
          order[0] = a;
          order[1] = b;
        }
      }
    used[order[0]] = used[order[1]] = true;
    n = 2;
    View cur = joint_view(factor_view(h, order[0]), factor_view(h, order[1]), &rc);
    if (rc) return fail(rc, "head route: chain intermediate has too many indices");
    while (n < N - 1) {
      int pick = -1;
      int64_t bs = -1;
      for (int t = 1; t < N; ++t) {
        if (used[t]) continue;
        int rcj = FCTN_OK;
        const int64_t sz = joint_view(cur, factor_view(h, t), &rcj).size();
        if (rcj == FCTN_OK && (bs < 0 || sz < bs)) bs = sz, pick = t;
      }
      if (pick < 0) return fail(FCTN_E_UNSUPPORTED, "head route: chain intermediate has too many indices");
      used[pick] = true;
      order[n++] = pick;
      cur = joint_view(cur, factor_view(h, pick), &rc);
    }
    for (int i = 0; i < N - 1; ++i) r.m0fac[i] = order[i];
    cur = factor_view(h, order[0]);
    for (int i = 1; i < N - 1; ++i) {
      View nx = factor_view(h, order[i]);
      View o = (i == N - 2) ? m0_view(h) : joint_view(cur, nx, &rc);
      if (rc) return fail(rc, "head route: chain intermediate has too many indices");
      if (i < N - 2) track(&r.u_elems, o.size());
      if ((rc = sg_plan(cur, nx, o, &r.m0[r.nm0], &t0, sgs))) return rc;
      track(&r.part_main, (int64_t)sg_part_elems(r.m0[r.nm0].sh));
      r.nm0++;
      cur = o;
    }
  }
  if ((rc = sg_plan(x_view(h), m0_view(h), factor_view(h, 0), &r.y0, &t0, sgs))) return rc;
  if ((rc = sg_plan(x_view(h), factor_view(h, 0), z_view(h), &r.z, &t0, sgs))) return rc;
  track(&r.part_main, (int64_t)sg_part_elems(r.y0.sh));
  track(&r.part_main, (int64_t)sg_part_elems(r.z.sh));
  // right-hand sides of k >= 1: Z contracted with the factors t != 0, k,
  // the largest mode first (it shrinks the intermediate most)
  for (int k = 1; k < N; ++k) {
    int ids[FCTN_MAX_ORDER], n = 0;
    for (int t = 1; t < N; ++t)
      if (t != k) ids[n++] = t;
    for (int a = 0; a < n; ++a)
      for (int b = a + 1; b < n; ++b)
        if (h->I[ids[b]] > h->I[ids[a]]) std::swap(ids[a], ids[b]);
    View cur = z_view(h);
    for (int q = 0; q < n; ++q) {
      View nx = factor_view(h, ids[q]);
      View o = (q == n - 1) ? factor_view(h, k) : joint_view(cur, nx, &rc);
      if (rc) return fail(rc, "head route: chain intermediate has too many indices");
      if (q < n - 1) track(&r.u_elems, o.size());
      if ((rc = sg_plan(cur, nx, o, &r.ys[k][q], &t0, sgs))) return rc;
      track(&r.part_main, (int64_t)sg_part_elems(r.ys[k][q].sh));
      r.yfac[k][q] = ids[q];
      cur = o;
    }
    r.nys[k] = n;
  }
  // Leading steps shared with factor k-1's chain: the same factors in the
  // same order give the same intermediate (Z and those factors do not change
  // between the two right-hand sides, since neither k-1 nor k is among
  // them); shared when the intermediate is still in its U buffer, i.e. when
  // only the final step of k-1's chain follows it.  With N = 4 the first
  // step Z (x) A_(1) of factors 2 and 3 is formed once.
  for (int k = 2; k < N; ++k) {
    int L = 0;
    while (L < r.nys[k] - 1 && L < r.nys[k - 1] - 1 && r.yfac[k][L] == r.yfac[k - 1][L]) ++L;
    r.yshare[k] = (L > 0 && r.nys[k - 1] == L + 1) ? L : 0;
  }
  // factor Grams and, per k, their chain over t != k (ascending)
  for (int t = 0; t < N; ++t) {
    if ((rc = sg_plan(factor_view(h, t), factor_primed_view(h, t), hgram_view(h, t), &r.hg[t], &t0, sgs))) return rc;
    track(&r.part_side, (int64_t)sg_part_elems(r.hg[t].sh));
  }
  // Chain order: for the pair {k, k ^ 1} (N >= 4) the factors other than
  // both come first (ascending) and the partner last, so that the two
  // chains share everything but their last step: those Grams do not change
  // between the two factor updates, and the odd member reuses the even
  // member's intermediate (still in its E buffer: only the final step,
  // which writes G, follows it).  Otherwise ascending.
  for (int k = 0; k < N; ++k) {
    int ids[FCTN_MAX_ORDER], n = 0;
    const int pk = k ^ 1;
    const bool paired = N >= 4 && pk < N;
    for (int t = 0; t < N; ++t)
      if (t != k && !(paired && t == pk)) ids[n++] = t;
    if (paired) ids[n++] = pk;
    for (int i = 0; i < n; ++i) r.efac[k][i] = ids[i];
    r.eshare[k] = (paired && (k & 1)) ? n - 2 : 0;
    View cur = hgram_view(h, ids[0]);
    for (int q = 1; q < n; ++q) {
      View nx = hgram_view(h, ids[q]);
      View o = (q == n - 1) ? hgram_view(h, k) : joint_view(cur, nx, &rc);
      if (rc) return fail(rc, "head route: Gram chain intermediate has too many indices");
      if (q < n - 1) track(&r.e_elems, o.size());
      if ((rc = sg_plan(cur, nx, o, &r.env[k][q - 1], &t0, sgs))) return rc;
      track(&r.part_side, (int64_t)sg_part_elems(r.env[k][q - 1].sh));
      cur = o;
    }
    r.nenv[k] = n - 1;
  }
  const int64_t cap = (int64_t)1 << 28;
  if (r.u_elems > cap || r.e_elems > cap || r.part_main > cap || r.part_side > cap) {
    r = HeadRoute{};
    return FCTN_OK;
  }
  // tensor-core products: every operand row a multiple of 16 bytes (TMA)
  if (h->tc && !(h->p.tile_code & 1)) {  // tile code bit 0: CUDA-core products instead
    const int elem = h->p.precision == FCTN_BF16 ? 2 : 4, al = 16 / elem;
    static const int kTySplit[4] = {2 * 152, 152, 4 * 152, 76};
    static const int kTyStages[4] = {0, 2, 4, 6};
    const int64_t I0 = h->I[0];
    if (r.P0 % al == 0 && I0 % al == 0 && r.P0 < ((int64_t)1 << 31)) {
      r.tc = true;
      r.bf16 = elem == 2;
      r.ldt = I0;
      r.ld0 = (r.s0 + al - 1) / al * al;
      tg_shape((int)I0, (int)r.s0, (int)r.P0, elem, kTySplit[(h->p.tile_code >> 3) & 3], &r.ty);
      if (kTyStages[(h->p.tile_code >> 1) & 3]) {
        r.ty.S = kTyStages[(h->p.tile_code >> 1) & 3];
        while (r.ty.S > 2 && tg_smem_bytes(r.ty.BN, r.ty.S) > 200 * 1024) --r.ty.S;
      }
      tg_shape((int)r.P0, (int)r.s0, (int)I0, elem, 0, &r.tz);
      tg_shape((int)r.P0, (int)I0, (int)r.s0, 4, 0, &r.tf);  // the reconstruction stays TF32 (see route_build_m0)
      r.ty.mode = TG_PARTIAL;
      r.tz.mode = TG_STORE;
      r.tf.mode = TG_XUPDATE;
      // The M_0 chain and the right-hand-side chains from Z on the tensor
      // cores too (the Gram chains stay FP32: the conditioning of Eq. 5
      // rests on them).  Their operands arrive rounded to TF32 from their
      // producers (Z from its GEMM, the chain intermediates from the
      // previous step) except the factors, which the kernel rounds as it
      // stages them.
      auto tcplan = [&](SgPlanH& q, bool a0_factor, bool round_out) {
        tcc_shape(q.sh, sgs, &q.tcs);
        q.tcs.round_a = q.swap ? 1 : (a0_factor ? 1 : 0);
        q.tcs.round_b = q.swap ? (a0_factor ? 1 : 0) : 1;
        q.tcok = true;
        q.round_out = round_out;
        track(&r.part_main, (int64_t)tcc_part_elems(q.tcs));
      };
      for (int i = 0; i < r.nm0; ++i) tcplan(r.m0[i], i == 0, i < r.nm0 - 1);
      for (int k = 1; k < N; ++k)
        for (int q = 0; q < r.nys[k]; ++q) tcplan(r.ys[k][q], false, q < r.nys[k] - 1);
      r.tz.round_tf32 = 1;  // Z: an operand of the right-hand-side chains
      if (r.part_main > cap) {
        r = HeadRoute{};
        return FCTN_OK;
      }
    }
  }
  // table offsets are relative to this plan's block, which starts at tabs->size()
  const size_t base = tabs->size();
  auto rebase = [&](SgPlanH& q) { q.tab += base; };
  for (int i = 0; i < r.nm0; ++i) rebase(r.m0[i]);
  rebase(r.y0);
  rebase(r.z);
  for (int k = 1; k < N; ++k)
    for (int q = 0; q < r.nys[k]; ++q) rebase(r.ys[k][q]);
  for (int t = 0; t < N; ++t) rebase(r.hg[t]);
  for (int k = 0; k < N; ++k)
    for (int q = 0; q < r.nenv[k]; ++q) rebase(r.env[k][q]);
  tabs->insert(tabs->end(), t0.begin(), t0.end());
  return FCTN_OK;
}

Sizes sizes_of(const fctn_handle* h) {
  Sizes z{};
  for (int k = 0; k < h->N; ++k) {
    if (h->p.reuse && materialise_ok(h, k) && h->s[k] * h->Pk[k] > z.M) z.M = h->s[k] * h->Pk[k];
    GramPlan g = gram_plan(h, k);
    if (g.ksplit * g.s * g.ncols > z.part) z.part = g.ksplit * g.s * g.ncols;
    if (h->I[k] * h->s[k] > z.Is) z.Is = h->I[k] * h->s[k];
    if (h->s[k] * h->s[k] > z.ss) z.ss = h->s[k] * h->s[k];
    if (h->I[k] > z.maxI) z.maxI = h->I[k];
    if (h->s[k] > z.maxs) z.maxs = h->s[k];
    int64_t b = xupdate_blocks(g);
    if (b > z.red_blocks) z.red_blocks = b;
    if (h->fg[k].use) {
      int64_t hb = (int64_t)h->fg[k].rl * h->fg[k].rl + (int64_t)h->fg[k].rr * h->fg[k].rr;
      if (hb > z.hbuf) z.hbuf = hb;
    }
  }
  z.maxfac = z.Is;
  z.chain = chain_need(h);
  z.lbuf = lbuf_need(h);
  if (h->hr.on) {  // the head-mode route has buffers of its own (route_bytes); the
    // chain buffers stay for fctn_contract
    z.M = z.part = z.hbuf = z.lbuf = 0;
    return z;
  }
  if (reuse_pairs(h)) {
    for (int q = 0; q < 2; ++q) {
      Lab ord[FCTN_MAXD];
      int n;
      z.T[q] = half_out_view(h, q, ord, &n).size();
    }
  }
  return z;
}

void release_side(fctn_handle* h) {
  if (h->side) cudaStreamSynchronize(h->side);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->side) cudaStreamDestroy(h->side);
  h->side = nullptr;
  h->ev_fork = h->ev_join = nullptr;
}

// Device bytes of the head-mode route's own buffers.
size_t route_bytes(const fctn_handle* h, size_t tab_ints) {
  const HeadRoute& r = h->hr;
  if (!r.on) return 0;
  size_t b = 2 * (size_t)r.s0 * r.P0 * 4;            // M_0, Z
  b += 2 * (size_t)r.u_elems * 4 + 2 * (size_t)r.e_elems * 4;
  b += ((size_t)r.part_main + (size_t)r.part_side) * 4;
  int64_t Is = 0;
  for (int k = 0; k < h->N; ++k) {
    b += (size_t)h->s[k] * h->s[k] * 4;                // H_k
    Is = h->I[k] * h->s[k] > Is ? h->I[k] * h->s[k] : Is;
  }
  b += (size_t)Is * 4 + tab_ints * sizeof(int);
  if (r.tc) {
    const size_t e = r.bf16 ? 2 : 4;
    const int64_t I0 = h->I[0];
    b += ((size_t)r.P0 * r.ldt + (size_t)r.s0 * r.ldt) * e + ((size_t)r.P0 * r.ld0 + (size_t)I0 * r.ld0) * 4;
    if (r.bf16) b += ((size_t)h->P + (size_t)r.s0 * r.P0) * 2;
    b += (size_t)r.ty.ksplit * I0 * r.s0 * 4;
  }
  return b;
}

size_t footprint(const fctn_handle* h) {
  Sizes z = sizes_of(h);
  size_t e = h->esz, b = 0;
  b += h->P * e + ((h->P + 31) / 32) * 4;                 // X, mask bits
  b += z.M * e + 2 * z.chain * e + z.lbuf * e + (z.T[0] + z.T[1]) * e;  // merged, chain, pairs
  b += z.part * e;                                        // split-K partials
  b += z.hbuf * e;                                        // operand Grams
  for (int k = 0; k < h->N; ++k) {
    b += h->I[k] * h->s[k] * (8 + e);                     // factors (FP64 master + compute copy)
    b += h->I[k] * h->I[k] * 24 + h->I[k] * 8;            // L_k basis and its transpose
  }
  b += 4 * z.Is * 8 + z.ss * 8;                           // Gd, Yd, Rd, previous factor
  size_t se = h->f64 ? 8 : 4;
  b += (2 * z.ss + z.maxs + 5 * z.Is) * se + 4 * z.ss * se;  // solve buffers + eigensolver work
  if (!h->f64) {
    size_t rec = 0;
    for (int k = 0; k < h->N; ++k) rec = std::max(rec, eig_record_floats((int)h->s[k]));
    b += rec * 4;  // rotation record of the large eigensolver
  }
  for (int k = 0; k < h->N; ++k) b += h->s[k] * h->s[k] * se;  // warm-start eigenvectors
  size_t nl, nd;
  chol_floats(h, &nl, &nd);
  b += (nl + nd) * 4;  // Cholesky factors
  if (nl) b += 2 * z.Is * 4;  // Q^T R and the double-float split of the factor
  b += (z.red_blocks * 3 + h->N * 32 + 8) * 8 + 16;
  int64_t stage = h->P > z.maxfac ? h->P : z.maxfac;
  b += stage * e + h->P;                                  // staging
  return b;
}

int dalloc(fctn_handle* h, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(FCTN_E_OOM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
  }
  h->allocs.push_back(*p);
  return FCTN_OK;
}

void free_all(fctn_handle* h) {
  for (void* p : h->allocs) cudaFree(p);
  h->allocs.clear();
}

int copy_in(fctn_handle* h, void* dst, const void* src, size_t bytes, int where) {
  if (where != FCTN_HOST && where != FCTN_DEVICE) return fail(FCTN_E_ARG, "where must be FCTN_HOST or FCTN_DEVICE");
  CK(cudaMemcpyAsync(dst, src, bytes, where == FCTN_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, h->st));
  return FCTN_OK;
}

int copy_out(fctn_handle* h, void* dst, const void* src, size_t bytes, int where) {
  if (where != FCTN_HOST && where != FCTN_DEVICE) return fail(FCTN_E_ARG, "where must be FCTN_HOST or FCTN_DEVICE");
  CK(cudaMemcpyAsync(dst, src, bytes, where == FCTN_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->st));
  if (where == FCTN_HOST) CK(cudaStreamSynchronize(h->st));
  return FCTN_OK;
}


// The trace terms of Eq. 2 for every factor (one launch on stream st).
void launch_traces(fctn_handle* h, cudaStream_t st) {
  const double sgn = h->p.laplacian_sign == FCTN_LAPLACIAN_PRINTED ? -1.0 : 1.0;
  TraceArgs a{};
  for (int k = 0; k < h->N; ++k) {
    a.A[k] = h->A64[k];
    a.I[k] = h->I[k];
    a.s[k] = h->s[k];
    a.c0[k] = sgn * (2.0 + h->p.delta[k]);
    a.c1[k] = -sgn;
    a.lam[k] = h->p.lambda[k];
  }
  launch_trace_all(a, h->N, h->traces, st);
}

// Rotation threshold of the FP32 Gram eigensolver: the caller's, else one
// matched to the FP64 refinement of the solve, which removes what the
// eigenbasis leaves: two refinement steps tolerate off-diagonal ratios of
// 2e-4 (one Jacobi sweep from a warm start), one step 2e-5; without
// refinement the kernels' own sqrt(s) FLT_EPSILON (0 here).
double eig_tol_eff(const fctn_handle* h) {
  if (h->p.eig_tol > 0.0) return h->p.eig_tol;
  if (h->f64) return 0.0;
  return h->p.refine_steps >= 2 ? 2e-4 : h->p.refine_steps == 1 ? 2e-5 : 0.0;
}

// Factorization step of the FP32 solve of factor k on stream st: the shifted
// Cholesky factors of G + (lam mu_j + rho) I, or the eigendecomposition of G
// (Eq. 7) warm-started from the previous sweep's eigenbasis.
void prep_f32(fctn_handle* h, int k, cudaStream_t st) {
  const int I = (int)h->I[k], s = (int)h->s[k];
  const double sgn = h->p.laplacian_sign == FCTN_LAPLACIAN_PRINTED ? -1.0 : 1.0;
  if (h->chol[k]) {
    launch_chol_factor((const float*)h->Gs, I, s, h->p.lambda[k], sgn * (2.0 + h->p.delta[k]), -sgn, h->p.rho,
                       h->cholL, h->cholD, h->status, st);
    return;
  }
  launch_eig_f32((const float*)h->Gs, (float*)h->Ck[k], (float*)h->Phi, (float*)h->gwork, s, h->cvalid[k] ? 1 : 0,
                 h->eig_cap, h->lam_min[k] + h->p.rho, h->status, h->eig_used + k, st, h->eig_rec, eig_tol_eff(h));
}
int prep_f32_launches(const fctn_handle* h, int k) {
  return h->chol[k] ? 1 : eig_launches((int)h->s[k], h->cvalid[k] ? 1 : 0, h->eig_rec != nullptr);
}
// Solve of Eq. 5 for factor k through the shifted Cholesky factors, then
// refine_steps passes on the residual of Eq. 5 (summed in double-float):
// Q^T Y, substitution, A = Q W; R, Q^T R, substitution, A += Q W.
int chol_solve(fctn_handle* h, int k, bool rt_done = false) {
  const int I = (int)h->I[k], s = (int)h->s[k];
  const double lam = h->p.lambda[k], rho = h->p.rho;
  const double sgn = h->p.laplacian_sign == FCTN_LAPLACIAN_PRINTED ? -1.0 : 1.0;
  const double c0 = sgn * (2.0 + h->p.delta[k]), c1 = -sgn;
  float* W = (float*)h->Z;
  float* Ac = (float*)h->Ac[k];
  const double ge = 2.0 * (double)I * I * s, sub = 2.0 * (double)I * s * s;
  // the solve's chain runs after the join with the factorization branch, so
  // its kernels may launch programmatically (nothing else needs the SMs)
  PdlScope pdl(h->hr.on && (h->p.tile_code & 128));
  if (!rt_done)  // Q^T Y (the head route forms it before joining the factorization branch)
    LAUNCH(FCTN_KC_SOLVE, 0.0, ge,
           launch_basis_gemm(0, h->QT32[k], (const float*)h->Ys, I, s, h->cholRt, nullptr, nullptr, nullptr, h->st));
  LAUNCH(FCTN_KC_SUBST, 0.0, sub, launch_chol_subst(h->cholRt, I, s, h->cholL, h->cholD, W, h->status, h->st));
  LAUNCH(FCTN_KC_SOLVE, 0.0, ge, launch_basis_gemm(1, h->Q32[k], W, I, s, nullptr, h->A64[k], Ac, h->Alo, h->st));
  for (int r = 0; r < h->p.refine_steps; ++r) {
    LAUNCH(FCTN_KC_RESID, 0.0, sub,
           launch_resid_df(h->Yd, h->A64[k], Ac, h->Alo, (const float*)h->Gs, I, s, lam, rho, c0, c1, (float*)h->Rs,
                           h->st));
    LAUNCH(FCTN_KC_SOLVE, 0.0, ge,
           launch_basis_gemm(0, h->QT32[k], (const float*)h->Rs, I, s, h->cholRt, nullptr, nullptr, nullptr, h->st));
    LAUNCH(FCTN_KC_SUBST, 0.0, sub, launch_chol_subst(h->cholRt, I, s, h->cholL, h->cholD, W, h->status, h->st));
    LAUNCH(FCTN_KC_SOLVE, 0.0, ge, launch_basis_gemm(2, h->Q32[k], W, I, s, nullptr, h->A64[k], Ac, h->Alo, h->st));
  }
  return FCTN_OK;
}

// Forward half of the FP32 Eq. 8 solve of factor k: W from the right-hand side R.
void fwd_f32(fctn_handle* h, int k, const float* R, float* W) {
  const int I = (int)h->I[k], s = (int)h->s[k];
  launch_solve_fwd_f32(h->QT32[k], R, (const float*)h->Ck[k], h->Lam[k], (const float*)h->Phi, h->p.lambda[k],
                       h->p.rho, I, s, W, h->status, h->st);
}

// Eqs. 5-9 for factor k; M_k is formed on chip from its pair operands L, R
// (and written to Mout when that is non-null).
int update_factor(fctn_handle* h, int k, const void* L, const void* R, void* Mout) {
  GramPlan g = gram_plan(h, k);
  const int I = (int)h->I[k], s = (int)h->s[k];
  const double lam = h->p.lambda[k], rho = h->p.rho;
  const double sgn = h->p.laplacian_sign == FCTN_LAPLACIAN_PRINTED ? -1.0 : 1.0;
  const double c0 = sgn * (2.0 + h->p.delta[k]), c1 = -sgn;
  const double tmin = h->lam_min[k] + rho;  // min_i lam Lambda_i + rho; T > 0 needs Phi_min + tmin > 0
  const int warm = h->cvalid[k] ? 1 : 0;
  const double e = (double)h->esz;
  const double part_elems = (double)g.ksplit * g.s * g.ncols;
  // algorithmic traffic / work of each step
  const double gram_bytes = (double)h->P * e + part_elems * e + (Mout ? (double)g.s * g.Pk * e : 0.0);
  const double gram_flops = 2.0 * (double)g.s * (double)g.ncols * (double)g.Pk;
  const FactGram& fg = h->fg[k];
  const double fact_flops = fg.use ? 2.0 * ((double)fg.rl * fg.rl * fg.JL + (double)fg.rr * fg.rr * fg.JR +
                                            (double)s * s * fg.K * fg.K)
                                   : 0.0;
  const double red_bytes = part_elems * e + (double)g.s * g.ncols * 8.0 * 2;
  const double fwd_flops = 2.0 * ((double)I * I * s + 2.0 * (double)I * s * s);  // Q^T R, then C and C^T
  const double bwd_flops = 2.0 * (double)I * I * s;                              // Q W
  const double resid_flops = 2.0 * (double)I * s * s;
  const bool extrap = h->p.extrap_alpha != 0.0;
  if (extrap && !h->dry)
    CK(cudaMemcpyAsync(h->Aprev, h->A64[k], (size_t)I * s * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  // FactGram and the eigendecomposition of its Gram (which does not depend
  // on X) on the side stream, overlapping the right-hand-side kernel and its
  // reduction; the solve joins both.  The per-class profiler times launches
  // on `st` one by one, so it runs them there.
  const bool fork = fg.use && h->side && h->prof_class < 0;
  cudaStream_t fst = fork ? h->side : h->st;
  void* HL = h->hbuf;
  void* HR = (char*)h->hbuf + (size_t)fg.rl * fg.rl * h->esz;
  if (fork && !h->dry) {
    CK(cudaEventRecord(h->ev_fork, h->st));
    CK(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
  }
  if (fg.use) {
    if (fork) {
      if (h->f64) {
        LAUNCH_ON(3, launch_fact_gram_f64(fg, (const double*)L, (const double*)R, (double*)HL, (double*)HR, s, h->Gd,
                                          fst));
        LAUNCH_ON(1, launch_eig_f64(h->Gd, (double*)h->Ck[k], (double*)h->Phi, (double*)h->gwork, s, warm, h->eig_cap, tmin,
                                    h->status, h->eig_used + k, fst));
      } else {
        LAUNCH_ON(3, launch_fact_gram_f32(fg, (const float*)L, (const float*)R, (float*)HL, (float*)HR, s, h->Gd,
                                          (float*)h->Gs, fst));
        LAUNCH_ON(prep_f32_launches(h, k), prep_f32(h, k, fst));
      }
      if (!h->dry) CK(cudaEventRecord(h->ev_join, h->side));
    } else if (h->f64) {
      LAUNCH(FCTN_KC_GRAM, 0.0, fact_flops,
             launch_fact_gram_f64(fg, (const double*)L, (const double*)R, (double*)HL, (double*)HR, s, h->Gd, fst));
      h->launches += 2;
    } else {
      LAUNCH(FCTN_KC_GRAM, 0.0, fact_flops,
             launch_fact_gram_f32(fg, (const float*)L, (const float*)R, (float*)HL, (float*)HR, s, h->Gd,
                                  (float*)h->Gs, fst));
      h->launches += 2;
    }
  }
  if (h->f64) {
    double *Ck = (double*)h->Ck[k], *Phi = (double*)h->Phi, *Z = (double*)h->Z;
    LAUNCH(FCTN_KC_GRAM, gram_bytes, gram_flops,
           launch_gram_fused_f64(h->pp[k], (const double*)L, (const double*)R, (const double*)h->X,
                                 (double*)h->part, g, (double*)Mout, h->st));
    LAUNCH(FCTN_KC_REDUCE, red_bytes, part_elems,
           launch_reduce_gram_rhs_f64((const double*)h->part, g, h->A64[k], rho, h->Gd, h->Yd, h->st));
    if (fork && !h->dry) CK(cudaStreamWaitEvent(h->st, h->ev_join, 0));
    if (!fork)
      LAUNCH(FCTN_KC_EIG, 0.0, 0.0,
             launch_eig_f64(h->Gd, Ck, Phi, (double*)h->gwork, s, warm, h->eig_cap, tmin, h->status, h->eig_used + k, h->st));
    // Eq. 8, then refinement passes on the FP64 residual of Eq. 5 (the
    // first residual is fused into the first backward pass)
    const int nref = h->p.refine_steps;
    LAUNCH(FCTN_KC_SOLVE, 0.0, fwd_flops,
           launch_solve_fwd_f64(h->QT64[k], h->Yd, Ck, h->Lam[k], Phi, lam, rho, I, s, Z, h->status, h->st));
    LAUNCH(FCTN_KC_SOLVE, 0.0, bwd_flops + (nref > 0 ? resid_flops : 0.0),
           launch_solve_bwd_f64(h->Q64[k], Z, I, s, 0, h->A64[k], (double*)h->Ac[k], h->Yd, h->Gd, lam, rho, c0, c1,
                                nref > 0 ? h->Rd : nullptr, h->status, h->st));
    for (int r = 0; r < nref; ++r) {
      if (r > 0)
        LAUNCH(FCTN_KC_SOLVE, 0.0, resid_flops,
               launch_resid_f64(h->Yd, h->A64[k], h->Gd, I, s, lam, rho, c0, c1, h->Rd, h->st));
      LAUNCH(FCTN_KC_SOLVE, 0.0, fwd_flops,
             launch_solve_fwd_f64(h->QT64[k], h->Rd, Ck, h->Lam[k], Phi, lam, rho, I, s, Z, h->status, h->st));
      LAUNCH(FCTN_KC_SOLVE, 0.0, bwd_flops,
             launch_solve_bwd_f64(h->Q64[k], Z, I, s, 1, h->A64[k], (double*)h->Ac[k], nullptr, nullptr, lam, rho, c0,
                                  c1, nullptr, h->status, h->st));
    }
  } else {
    float *Ck = (float*)h->Ck[k], *Phi = (float*)h->Phi, *Z = (float*)h->Z;
    if (h->tc) {
      LAUNCH(FCTN_KC_GRAM, gram_bytes, gram_flops,
             launch_gram_tc(h->pp[k], (const float*)L, (const float*)R, (const float*)h->X, (float*)h->part, g,
                            h->tp[k], h->p.precision, (float*)Mout, h->status, h->st));
    } else {
      LAUNCH(FCTN_KC_GRAM, gram_bytes, gram_flops,
             launch_gram_fused_f32(h->pp[k], (const float*)L, (const float*)R, (const float*)h->X,
                                   (float*)h->part, g, (float*)Mout, h->st));
    }
    LAUNCH(FCTN_KC_REDUCE, red_bytes, part_elems,
           launch_reduce_gram_rhs_f32((const float*)h->part, g, h->A64[k], rho, h->Gd, h->Yd, (float*)h->Gs,
                                      (float*)h->Ys, h->st));
    if (fork && !h->dry) CK(cudaStreamWaitEvent(h->st, h->ev_join, 0));
    if (!fork) {
      LAUNCH(FCTN_KC_EIG, 0.0, 0.0, prep_f32(h, k, h->st));
      h->launches += prep_f32_launches(h, k) - 1;
    }
    const int nref = h->p.refine_steps;
    if (h->chol[k]) {
      int rc = chol_solve(h, k);
      if (rc) return rc;
    } else {
      LAUNCH(FCTN_KC_SOLVE, 0.0, fwd_flops, fwd_f32(h, k, (const float*)h->Ys, Z));
      LAUNCH(FCTN_KC_SOLVE, 0.0, bwd_flops + (nref > 0 ? resid_flops : 0.0),
             launch_solve_bwd_f32(h->Q32[k], Z, I, s, 0, h->A64[k], (float*)h->Ac[k], h->Yd, h->Gd, lam, rho, c0, c1,
                                  nref > 0 ? (float*)h->Rs : nullptr, h->status, h->st));
      for (int r = 0; r < nref; ++r) {
        if (r > 0)
          LAUNCH(FCTN_KC_SOLVE, 0.0, resid_flops,
                 launch_resid_f32(h->Yd, h->A64[k], h->Gd, I, s, lam, rho, c0, c1, (float*)h->Rs, h->st));
        LAUNCH(FCTN_KC_SOLVE, 0.0, fwd_flops, fwd_f32(h, k, (const float*)h->Rs, Z));
        LAUNCH(FCTN_KC_SOLVE, 0.0, bwd_flops,
               launch_solve_bwd_f32(h->Q32[k], Z, I, s, 1, h->A64[k], (float*)h->Ac[k], nullptr, nullptr, lam, rho,
                                    c0, c1, nullptr, h->status, h->st));
      }
    }
  }
  if (extrap) {
    if (h->f64)
      LAUNCH(FCTN_KC_SOLVE, 0.0, 0.0,
             launch_extrap_f64(h->A64[k], h->Aprev, h->p.extrap_alpha, h->p.extrap_beta, (double*)h->Ac[k],
                               (int64_t)I * s, h->st));
    else
      LAUNCH(FCTN_KC_SOLVE, 0.0, 0.0,
             launch_extrap_f32(h->A64[k], h->Aprev, h->p.extrap_alpha, h->p.extrap_beta, (float*)h->Ac[k],
                               (int64_t)I * s, h->st));
  }
  h->cvalid[k] = true;
  h->ver[k]++;
  return FCTN_OK;
}

// ---- head-mode association: one sweep ----------------------------------------
SgTabs sg_tabs(const fctn_handle* h, const SgPlanH& q) {
  const int* b = h->hr.tabs + q.tab;
  const int M = q.sh.M, N = q.sh.N;
  return SgTabs{b, b + M, b + 2 * M, b + 2 * M + N, b + 2 * M + 2 * N, b + 2 * M + 2 * N + q.sh.K};
}

// C = A (x) B by plan q on stream st (operands passed swapped when the plan says so).
// The tensor-core contraction serves a plan that has one while the route's
// products are TF32 / BF16 (not after the switch to FP32 products).
bool sg_on_tc(const fctn_handle* h, const SgPlanH& q) { return q.tcok && h->hr.tc && !h->hr.fp32_now; }
void run_sg(const fctn_handle* h, const SgPlanH& q, const float* A, const float* B, float* C, float* part,
            cudaStream_t st) {
  if (sg_on_tc(h, q)) {
    TccShape ts = q.tcs;
    ts.sh.round_tf32 = q.sh.round_tf32 || q.round_out;
    launch_tcc(ts, sg_tabs(h, q), q.swap ? B : A, q.swap ? A : B, C, part, h->status, st);
    return;
  }
  launch_sgemm(q.sh, sg_tabs(h, q), q.swap ? B : A, q.swap ? A : B, C, part, st);
}
double sg_flops(const SgPlanH& q) { return 2.0 * (double)q.sh.M * q.sh.N * q.sh.K; }
// algorithmic bytes of a contraction: every operand element read once, C written once (FP32)
double sg_bytes(const SgPlanH& q) {
  return 4.0 * ((double)q.sh.M * q.sh.K + (double)q.sh.N * q.sh.K + (double)q.sh.M * q.sh.N);
}
int sg_launches(const fctn_handle* h, const SgPlanH& q) {
  if (sg_on_tc(h, q)) return tcc_launches(q.tcs);
  return q.sh.ksplit > 1 ? 2 : 1;
}

// M_0 from the present factors 1 .. N-1 (the planned chain order).
int route_build_m0(fctn_handle* h) {
  HeadRoute& r = h->hr;
  const float* cur = (const float*)h->Ac[r.m0fac[0]];
  const bool tf32_ops = r.tc && !r.fp32_now && !r.bf16;  // M_0 is then a TF32 operand: rounded as it is written
  for (int i = 0; i < r.nm0; ++i) {
    float* o = (i == r.nm0 - 1) ? r.M0 : r.U[i % 2];
    SgPlanH q = r.m0[i];
    q.sh.round_tf32 = (i == r.nm0 - 1 && tf32_ops) ? 1 : 0;
    LAUNCH(FCTN_KC_MERGED, sg_bytes(q), sg_flops(q),
           run_sg(h, q, cur, (const float*)h->Ac[r.m0fac[i + 1]], o, r.pm, h->st));
    h->launches += sg_launches(h, q) - 1;
    cur = o;
  }
  if (r.tc && !r.fp32_now) {
    // tensor-core operands: M_0 (Y_0's B: TF32-rounded, or BF16) and M_0^T
    // (F^T's A, TF32-rounded in both precisions: the reconstruction of Eq. 10
    // sets the completed entries directly, and BF16 operands there moved the
    // final PSNR by 0.11 dB on 48 x 40 x 9, beyond the 0.05 dB target)
    const double mb = (double)r.s0 * r.P0 * 4.0;
    if (r.bf16) {
      LAUNCH(FCTN_KC_MERGED, mb, 0.0,
             launch_copy_bf16(r.M0, r.s0, r.P0, r.P0, (__nv_bfloat16*)r.M0b, r.P0, h->st));
      LAUNCH(FCTN_KC_MERGED, mb, 0.0, launch_transpose_f32(r.M0, r.s0, r.P0, r.P0, (float*)r.M0T, r.ld0, 1, h->st));
    } else {  // M_0 already rounded by its contraction
      LAUNCH(FCTN_KC_MERGED, mb, 0.0, launch_transpose_f32(r.M0, r.s0, r.P0, r.P0, (float*)r.M0T, r.ld0, 0, h->st));
    }
  }
  r.m0_valid = true;
  return FCTN_OK;
}

// Tensor-core copies of A_(0): A_0^T (Z's B operand) and A_0 padded to ld0
// (F^T's B operand).
int route_a0_copies(fctn_handle* h) {
  HeadRoute& r = h->hr;
  const int64_t I0 = h->I[0];
  const float* A = (const float*)h->Ac[0];
  if (r.bf16) {
    LAUNCH(FCTN_KC_MISC, 0.0, 0.0, launch_transpose_bf16(A, I0, r.s0, r.s0, (__nv_bfloat16*)r.A0T, r.ldt, h->st));
    LAUNCH(FCTN_KC_MISC, 0.0, 0.0, launch_copy_f32(A, I0, r.s0, r.s0, (float*)r.A0p, r.ld0, 1, h->st));
  } else {
    LAUNCH(FCTN_KC_MISC, 0.0, 0.0, launch_transpose_f32(A, I0, r.s0, r.s0, (float*)r.A0T, r.ldt, 1, h->st));
    LAUNCH(FCTN_KC_MISC, 0.0, 0.0, launch_copy_f32(A, I0, r.s0, r.s0, (float*)r.A0p, r.ld0, 1, h->st));
  }
  return FCTN_OK;
}

// Eq. 8 solve with its FP64 refinement for factor k (FP32 operands), the
// eigendecomposition first unless it already ran on the side stream.
int route_solve(fctn_handle* h, int k, bool eig_done, bool rt_done) {
  const int I = (int)h->I[k], s = (int)h->s[k];
  const double lam = h->p.lambda[k], rho = h->p.rho;
  const double sgn = h->p.laplacian_sign == FCTN_LAPLACIAN_PRINTED ? -1.0 : 1.0;
  const double c0 = sgn * (2.0 + h->p.delta[k]), c1 = -sgn;
  const double tmin = h->lam_min[k] + rho;
  const int warm = h->cvalid[k] ? 1 : 0;
  const double fwd_flops = 2.0 * ((double)I * I * s + 2.0 * (double)I * s * s);
  const double bwd_flops = 2.0 * (double)I * I * s;
  const double resid_flops = 2.0 * (double)I * s * s;
  float *Ck = (float*)h->Ck[k], *Phi = (float*)h->Phi, *Z = (float*)h->Z;
  if (!eig_done && h->chol[k]) {
    LAUNCH(FCTN_KC_EIG, 0.0, (double)chol_groups(I) * s * s * s / 3.0, prep_f32(h, k, h->st));
  } else if (!eig_done && eig_is_big(s)) {  // the two stages timed apart
    const double ss = (double)s * s;
    if (warm) {
      LAUNCH(FCTN_KC_EIGAUX, 0.0, 8.0 * ss * s,
             launch_eig_big_prep((const float*)h->Gs, Ck, (float*)h->gwork, s, h->st));
      h->launches += eig_big_prep_launches() - 1;
    }
    LAUNCH(FCTN_KC_EIG, 0.0, 0.0,
           launch_eig_big_jacobi((const float*)h->Gs, Ck, Phi, (float*)h->gwork, s, warm, h->eig_cap, tmin,
                                 eig_tol_eff(h), h->status, h->eig_used + k, h->st));
  } else if (!eig_done) {
    LAUNCH(FCTN_KC_EIG, 0.0, 0.0,
           launch_eig_f32((const float*)h->Gs, Ck, Phi, (float*)h->gwork, s, warm, h->eig_cap, tmin, h->status,
                          h->eig_used + k, h->st, h->eig_rec, eig_tol_eff(h)));
    h->launches += eig_launches(s, warm, h->eig_rec != nullptr) - 1;
  }
  const int nref = h->p.refine_steps;
  if (h->chol[k]) {
    int rc = chol_solve(h, k, rt_done);
    if (rc) return rc;
  } else {
    LAUNCH(FCTN_KC_SOLVE, 0.0, fwd_flops, fwd_f32(h, k, (const float*)h->Ys, Z));
    LAUNCH(FCTN_KC_SOLVE, 0.0, bwd_flops + (nref > 0 ? resid_flops : 0.0),
           launch_solve_bwd_f32(h->Q32[k], Z, I, s, 0, h->A64[k], (float*)h->Ac[k], h->Yd, h->Gd, lam, rho, c0, c1,
                                nref > 0 ? (float*)h->Rs : nullptr, h->status, h->st));
    for (int r = 0; r < nref; ++r) {
      if (r > 0)
        LAUNCH(FCTN_KC_SOLVE, 0.0, resid_flops,
               launch_resid_f32(h->Yd, h->A64[k], h->Gd, I, s, lam, rho, c0, c1, (float*)h->Rs, h->st));
      LAUNCH(FCTN_KC_SOLVE, 0.0, fwd_flops, fwd_f32(h, k, (const float*)h->Rs, Z));
      LAUNCH(FCTN_KC_SOLVE, 0.0, bwd_flops,
             launch_solve_bwd_f32(h->Q32[k], Z, I, s, 1, h->A64[k], (float*)h->Ac[k], nullptr, nullptr, lam, rho, c0,
                                  c1, nullptr, h->status, h->st));
    }
  }
  if (h->p.extrap_alpha != 0.0)
    LAUNCH(FCTN_KC_SOLVE, 0.0, 0.0,
           launch_extrap_f32(h->A64[k], h->Aprev, h->p.extrap_alpha, h->p.extrap_beta, (float*)h->Ac[k],
                             (int64_t)I * s, h->st));
  h->cvalid[k] = true;
  h->ver[k]++;
  return FCTN_OK;
}

// One sweep in the order 1, ..., N (Algorithm 1's order) by the head-mode
// association; the Gram chain and the eigendecomposition of factor k run on
// the side stream beside its right-hand side.
int route_sweep(fctn_handle* h) {
  HeadRoute& r = h->hr;
  const int N = h->N;
  const bool fork = h->side && h->prof_class < 0;
  const double rho = h->p.rho;
  const float* X = (const float*)h->X;
  for (int t = 0; t < N; ++t)
    if (!r.hvalid[t]) {
      LAUNCH(FCTN_KC_ENV, 0.0, sg_flops(r.hg[t]),
             launch_gram_at((const float*)h->Ac[t], (int)h->I[t], (int)h->s[t], r.H[t], h->st));
      r.hvalid[t] = true;
    }
  int rc;
  if (!r.m0_valid && (rc = route_build_m0(h))) return rc;
  const bool tcp = r.tc && !r.fp32_now;  // tensor-core products this sweep
  if (tcp && !r.xt_valid) {  // X^T (and the BF16 X) of the present X, after fctn_set_data
    const int64_t I0 = h->I[0];
    if (r.bf16) {
      LAUNCH(FCTN_KC_MISC, 0.0, 0.0,
             launch_transpose_bf16(X, I0, r.P0, r.P0, (__nv_bfloat16*)r.XT, r.ldt, h->st));
      LAUNCH(FCTN_KC_MISC, 0.0, 0.0, launch_copy_bf16(X, I0, r.P0, r.P0, (__nv_bfloat16*)r.Xb, r.P0, h->st));
    } else {
      LAUNCH(FCTN_KC_MISC, 0.0, 0.0, launch_transpose_f32(X, I0, r.P0, r.P0, (float*)r.XT, r.ldt, 1, h->st));
    }
    r.xt_valid = true;
  }
  for (int k = 0; k < N; ++k) {
    const int I = (int)h->I[k], s = (int)h->s[k];
    const int warm = h->cvalid[k] ? 1 : 0;
    const double tmin = h->lam_min[k] + rho;
    if (h->p.extrap_alpha != 0.0 && !h->dry)
      CK(cudaMemcpyAsync(h->Aprev, h->A64[k], (size_t)I * s * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    // Gram of M_k: chain of the factor Grams H_t, t != k (side stream)
    cudaStream_t gs = fork ? h->side : h->st;
    if (fork && !h->dry) {
      CK(cudaEventRecord(h->ev_fork, h->st));
      CK(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
    }
    {
      const int* ids = r.efac[k];
      const int q0 = r.eshare[k];  // steps already formed for the partner factor
      const float* cur = q0 > 0 ? r.E[(q0 - 1) % 2] : r.H[ids[0]];
      for (int q = q0; q < r.nenv[k]; ++q) {
        float* o = (q == r.nenv[k] - 1) ? (float*)h->Gs : r.E[q % 2];
        const SgPlanH& pl = r.env[k][q];
        if (fork) {
          LAUNCH_ON(sg_launches(h, pl), run_sg(h, pl, cur, r.H[ids[q + 1]], o, r.ps, gs));
        } else {
          LAUNCH(FCTN_KC_ENV, 0.0, sg_flops(pl), run_sg(h, pl, cur, r.H[ids[q + 1]], o, r.ps, gs));
          h->launches += sg_launches(h, pl) - 1;
        }
        cur = o;
      }
      if (fork) {
        LAUNCH_ON(1, launch_finish_gram((float*)h->Gs, h->Gd, s, gs));
        LAUNCH_ON(prep_f32_launches(h, k), prep_f32(h, k, gs));
        if (!h->dry) CK(cudaEventRecord(h->ev_join, h->side));
      } else {
        LAUNCH(FCTN_KC_ENV, 0.0, 0.0, launch_finish_gram((float*)h->Gs, h->Gd, s, gs));
      }
    }
    // right-hand side X_(k) M_k^T (main stream)
    if (k == 0 && tcp) {
      TgArgs a = r.ty;
      a.out = r.tpart;
      a.status = h->status;
      const double e = r.bf16 ? 2.0 : 4.0;
      LAUNCH(FCTN_KC_GRAM, ((double)h->P + (double)r.s0 * r.P0) * e, 2.0 * (double)h->I[0] * r.s0 * r.P0,
             launch_tg_gemm(r.maps[0], r.maps[1], a, r.bf16, h->st));
      LAUNCH(FCTN_KC_REDUCE, 0.0, 0.0,
             launch_tg_reduce(r.tpart, a.ksplit, (int64_t)h->I[0] * r.s0, r.Yraw, h->st));
    } else if (k == 0) {
      LAUNCH(FCTN_KC_GRAM, (double)h->P * 4.0, sg_flops(r.y0), run_sg(h, r.y0, X, r.M0, r.Yraw, r.pm, h->st));
      h->launches += sg_launches(h, r.y0) - 1;
    } else {
      const int q0 = r.yshare[k];
      const float* cur = q0 > 0 ? r.U[(q0 - 1) % 2] : r.Zb;
      for (int q = q0; q < r.nys[k]; ++q) {
        float* o = (q == r.nys[k] - 1) ? r.Yraw : r.U[q % 2];
        const SgPlanH& pl = r.ys[k][q];
        LAUNCH(FCTN_KC_RHS2, sg_bytes(pl), sg_flops(pl),
               run_sg(h, pl, cur, (const float*)h->Ac[r.yfac[k][q]], o, r.pm, h->st));
        h->launches += sg_launches(h, pl) - 1;
        cur = o;
      }
    }
    LAUNCH(FCTN_KC_REDUCE, 0.0, 0.0,
           launch_finish_rhs(r.Yraw, h->A64[k], rho, h->Yd, (float*)h->Ys, (int64_t)I * s, h->st));
    // Q^T Y of the Cholesky solve does not need the factorization: formed
    // here, beside the factorization branch, before the join
    if (h->chol[k])
      LAUNCH(FCTN_KC_SOLVE, 0.0, 2.0 * (double)I * I * s,
             launch_basis_gemm(0, h->QT32[k], (const float*)h->Ys, I, s, h->cholRt, nullptr, nullptr, nullptr, h->st));
    if (fork && !h->dry) CK(cudaStreamWaitEvent(h->st, h->ev_join, 0));
    if ((rc = route_solve(h, k, fork, h->chol[k]))) return rc;
    // Gram of the new factor for the later Gram chains
    LAUNCH(FCTN_KC_ENV, 0.0, sg_flops(r.hg[k]),
           launch_gram_at((const float*)h->Ac[k], (int)h->I[k], (int)h->s[k], r.H[k], h->st));
    if (k == 0 && tcp) {  // Z = X_(0)^T A_(0) with the new head factor (tensor cores)
      if ((rc = route_a0_copies(h))) return rc;
      TgArgs a = r.tz;
      a.out = r.Zb;
      a.ldo = r.s0;
      a.status = h->status;
      const double e = r.bf16 ? 2.0 : 4.0;
      LAUNCH(FCTN_KC_GRAM, (double)h->P * e + (double)r.s0 * r.P0 * 4.0, 2.0 * (double)h->I[0] * r.s0 * r.P0,
             launch_tg_gemm(r.maps[2], r.maps[3], a, r.bf16, h->st));
    } else if (k == 0) {  // Z = X_(0)^T A_(0) with the new head factor
      LAUNCH(FCTN_KC_GRAM, (double)h->P * 4.0, sg_flops(r.z),
             run_sg(h, r.z, X, (const float*)h->Ac[0], r.Zb, r.pm, h->st));
      h->launches += sg_launches(h, r.z) - 1;
    }
  }
  // the trace terms of Eq. 2 need only the new factors: on the side stream,
  // beside M_0 and the X update
  if (fork) {
    if (!h->dry) {
      CK(cudaEventRecord(h->ev_fork, h->st));
      CK(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
    }
    LAUNCH_ON(1, launch_traces(h, h->side));
    if (!h->dry) CK(cudaEventRecord(h->ev_join, h->side));
  }
  // M_0 of the new factors 1 .. N-1, then Eq. 10 with F = A_(0) M_0
  if ((rc = route_build_m0(h))) return rc;
  GramPlan g = gram_plan(h, 0);
  int nred = xupdate_blocks(g);
  if (tcp) {  // F^T = M_0^T A_(0)^T with Eq. 10 in the epilogue (tensor cores)
    TgArgs a = r.tf;
    a.X = (float*)h->X;
    a.bits = h->bits;
    a.P0 = r.P0;
    a.rho = rho;
    a.XT = r.bf16 ? nullptr : (float*)r.XT;
    a.XTb = r.bf16 ? (__nv_bfloat16*)r.XT : nullptr;
    a.Xb = r.bf16 ? (__nv_bfloat16*)r.Xb : nullptr;
    a.ldt = r.ldt;
    a.round_tf32 = 1;
    a.red = h->red;
    a.status = h->status;
    const double e = r.bf16 ? 2.0 : 4.0;
    // X read and written, X^T written (and the BF16 X), mask bits, M_0^T read
    const double xb = (double)h->P * (8.0 + e + (r.bf16 ? 2.0 : 0.0)) + (double)h->P / 8.0 + (double)r.s0 * r.P0 * 4.0;
    LAUNCH(FCTN_KC_XUPDATE, xb, 2.0 * (double)h->P * r.s0, launch_tg_gemm(r.maps[4], r.maps[5], a, 0, h->st));
    nred = (int)(((r.P0 + 127) / 128) * ((h->I[0] + a.BN - 1) / a.BN));
  } else {
    const double xb = 2.0 * (double)h->P * 4.0 + (double)r.s0 * r.P0 * 4.0 + (double)h->P / 8.0;
    LAUNCH(FCTN_KC_XUPDATE, xb, 2.0 * (double)h->P * r.s0,
           launch_xupdate_f32((const float*)h->Ac[0], r.M0, (float*)h->X, h->bits, rho, g, h->red, h->st));
    r.xt_valid = false;  // X moved without its transposed copy
  }
  if (fork) {
    if (!h->dry) CK(cudaStreamWaitEvent(h->st, h->ev_join, 0));
  } else {
    LAUNCH(FCTN_KC_MISC, 0.0, 0.0, launch_traces(h, h->st));
  }
  LAUNCH(FCTN_KC_MISC, 0.0, 0.0, launch_finalize(h->red, nred, h->traces, h->N, h->stats, h->st));
  h->t++;
  return FCTN_OK;
}

void sweep_order(const fctn_handle* h, int64_t t_next, int* order) {
  if (h->p.order_policy == FCTN_ORDER_ALTERNATE && h->N >= 4 && t_next % 2 == 0) {
    int m = 0;  // second half first: the first half's intermediate is still valid
    for (int u = half_lo(h, 1); u < half_hi(h, 1); ++u) order[m++] = u;
    for (int u = half_lo(h, 0); u < half_hi(h, 0); ++u) order[m++] = u;
    return;
  }
  for (int k = 0; k < h->N; ++k) order[k] = k;
}

// One sweep: every factor update in the current order, then the X update.
int sweep_body(fctn_handle* h) {
  if (h->hr.on) return route_sweep(h);
  int order[FCTN_MAX_ORDER];
  sweep_order(h, h->t + 1, order);
  const int last = order[h->N - 1];
  int rc;
  const void *L = nullptr, *R = nullptr;
  for (int i = 0; i < h->N; ++i) {
    const int k = order[i];
    if ((rc = prepare_pair(h, k, &L, &R))) return rc;
    // Algorithm 2: keep M'_last (every other factor is already new when the
    // last factor is updated) for the X update, if it is small enough
    void* Mout = (h->p.reuse && k == last && h->mat[k]) ? h->M : nullptr;
    if ((rc = update_factor(h, k, L, R, Mout))) return rc;
  }
  // Eq. 10 with F = FCTN(A^{t+1}) = A_last(last) M'_last, fused with the stop-test sums
  GramPlan g = gram_plan(h, last);
  const double e = (double)h->esz;
  const double xf = 2.0 * (double)g.I * g.s * g.Pk;
  if (h->p.reuse && h->mat[last]) {
    const double xb = 2.0 * (double)h->P * e + (double)g.s * g.Pk * e + (double)h->P / 8.0;
    if (h->f64)
      LAUNCH(FCTN_KC_XUPDATE, xb, xf,
             launch_xupdate_f64((const double*)h->Ac[last], (const double*)h->M, (double*)h->X, h->bits, h->p.rho,
                                g, h->red, h->st));
    else
      LAUNCH(FCTN_KC_XUPDATE, xb, xf,
             launch_xupdate_f32((const float*)h->Ac[last], (const float*)h->M, (float*)h->X, h->bits, h->p.rho, g,
                                h->red, h->st));
  } else {
    // Algorithm 1 (FCTN from scratch), or a merged tensor too large to keep:
    // the pair operands are made current and M'_last is formed on chip
    if (!h->p.reuse && (rc = prepare_pair(h, last, &L, &R))) return rc;
    const double xb = 2.0 * (double)h->P * e + (double)h->P / 8.0;
    if (h->f64)
      LAUNCH(FCTN_KC_XUPDATE, xb, xf,
             launch_xupdate_fused_f64(h->pp[last], (const double*)L, (const double*)R, (const double*)h->Ac[last],
                                      (double*)h->X, h->bits, h->p.rho, g, h->red, h->st));
    else
      LAUNCH(FCTN_KC_XUPDATE, xb, xf,
             launch_xupdate_fused_f32(h->pp[last], (const float*)L, (const float*)R, (const float*)h->Ac[last],
                                      (float*)h->X, h->bits, h->p.rho, g, h->red, h->st));
  }
  LAUNCH(FCTN_KC_MISC, 0.0, 0.0, launch_traces(h, h->st));
  LAUNCH(FCTN_KC_MISC, 0.0, 0.0, launch_finalize(h->red, xupdate_blocks(g), h->traces, h->N, h->stats, h->st));
  h->t++;
  return FCTN_OK;
}

// Everything that decides which kernels a sweep launches (with which
// arguments) and is not fixed by the handle: the order parity, the warm-start
// state of every factor and the validity of the cached pair intermediates.
uint64_t sweep_key(const fctn_handle* h) {
  // the order parity matters only to the alternating order of the merged-tensor route
  const bool par = h->p.order_policy == FCTN_ORDER_ALTERNATE && h->N >= 4 && !h->hr.on;
  uint64_t key = par ? (uint64_t)((h->t + 1) % 2) : 0u;
  for (int k = 0; k < h->N; ++k) key |= (uint64_t)(h->cvalid[k] ? 1 : 0) << (1 + k);
  for (int q = 0; q < 2; ++q) {
    bool v = reuse_pairs(h) && half_valid(h, q);
    key |= (uint64_t)(v ? 1 : 0) << (12 + q);
  }
  if (h->hr.on) {
    key |= (uint64_t)(h->hr.m0_valid ? 1 : 0) << 14;
    key |= (uint64_t)(h->hr.xt_valid ? 1 : 0) << 24;
    key |= (uint64_t)(h->hr.fp32_now ? 1 : 0) << 25;
    for (int k = 0; k < h->N; ++k) key |= (uint64_t)(h->hr.hvalid[k] ? 1 : 0) << (15 + k);
  }
  return key;
}

int one_sweep(fctn_handle* h) {
  // profiling times launches one by one, so it runs the sweep eagerly
  if (!h->use_graphs || h->prof_class >= 0) return sweep_body(h);
  const uint64_t key = sweep_key(h);
  for (auto& g : h->graphs) {
    if (g.key == key) {
      h->dry = true;
      int rc = sweep_body(h);
      h->dry = false;
      if (rc) return rc;
      CK(cudaGraphLaunch(g.exec, h->st));
      return FCTN_OK;
    }
  }
  // capture this signature once, then launch it
  const int64_t t0 = h->t;
  int ver0[FCTN_MAX_ORDER];
  memcpy(ver0, h->ver, sizeof ver0);
  CK(cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal));
  int rc = sweep_body(h);
  cudaGraph_t graph = nullptr;
  cudaError_t ce = cudaStreamEndCapture(h->st, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (ce != cudaSuccess) return fail(FCTN_E_CUDA, "graph capture: %s", cudaGetErrorString(ce));
  cudaGraphExec_t exec = nullptr;
  ce = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) return fail(FCTN_E_CUDA, "graph instantiate: %s", cudaGetErrorString(ce));
  h->graphs.push_back({key, exec});
  (void)t0;
  (void)ver0;
  CK(cudaGraphLaunch(exec, h->st));
  return FCTN_OK;
}

int read_stats(fctn_handle* h, fctn_stats* out) {
  double st[4];
  int status = 0;
  int used[FCTN_MAX_ORDER] = {};
  CK(cudaMemcpyAsync(st, h->stats, sizeof st, cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(&status, h->status, sizeof status, cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(used, h->eig_used, sizeof(int) * h->N, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  int umax = 0, capped = 0;
  for (int k = 0; k < h->N; ++k) {
    const int u = used[k] < 0 ? -used[k] : used[k];  // negative: stopped at the sweep cap
    umax = u > umax ? u : umax;
    capped += used[k] < 0 ? 1 : 0;
  }
  if (out) {
    out->t = h->t;
    out->rel_change = st[0];
    out->objective = st[1];
    out->data_term = st[2];
    out->converged = 0;
    out->status = status;
    out->eig_sweeps = umax;
    out->eig_capped = capped;
  }
  if (status == FCTN_E_SINGULAR) return fail(FCTN_E_SINGULAR, "min T <= 0: the Sylvester system of Eq. 5 is not positive definite");
  if (status == FCTN_E_TIMEOUT)
    return fail(FCTN_E_TIMEOUT, "a bounded device wait gave up (a tensor-core pipeline or bulk-copy barrier of a "
                                "sweep kernel); the sweep's results are not valid");
  if (st[3] != 0.0) {
    if (out) out->status = FCTN_E_NONFINITE;
    return fail(FCTN_E_NONFINITE, "non-finite value in the stop-test reductions");
  }
  return FCTN_OK;
}

}  // namespace

int fctn_internal_fail(int code, const char* msg) { return fail(code, "%s", msg); }

int fctn_internal_sweep_async(fctn_handle* h, double* pinned) {
  if (!h->data_set || !h->factors_set) return fail(FCTN_E_STATE, "set data and factors before sweeping");
  int rc = one_sweep(h);
  if (rc) return rc;
  CK(cudaMemcpyAsync(pinned, h->stats, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(pinned + 4, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  pinned[5] = (double)h->t;
  return FCTN_OK;
}

cudaStream_t fctn_internal_stream(fctn_handle* h) { return h->st; }

int fctn_internal_sweep_eager(fctn_handle* h, double* pinned) {
  if (!h->data_set || !h->factors_set) return fail(FCTN_E_STATE, "set data and factors before sweeping");
  int rc = sweep_body(h);
  if (rc) return rc;
  CK(cudaMemcpyAsync(pinned, h->stats, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(pinned + 4, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  pinned[5] = (double)h->t;
  return FCTN_OK;
}

int fctn_internal_sweep_dry(fctn_handle* h, double* pinned) {
  h->dry = true;
  int rc = sweep_body(h);
  h->dry = false;
  if (rc) return rc;
  pinned[5] = (double)h->t;
  return FCTN_OK;
}

uint64_t fctn_internal_sweep_key(fctn_handle* h) { return sweep_key(h); }

void fctn_internal_after_sweep(fctn_handle* h, double rel_change) {
  HeadRoute& r = h->hr;
  if (!r.tc || r.fp32_now || !(h->p.finish_fp32_at > 0.0)) return;
  // the change stalls at the tensor-core products' rounding floor, where it
  // fluctuates: ten sweeps without a new low (1 % below the lowest so far)
  // also turn to FP32
  if (r.prev_rel <= 0.0 || rel_change < 0.99 * r.prev_rel) {
    r.prev_rel = rel_change;
    r.stall = 0;
  } else {
    r.stall++;
  }
  if (rel_change <= h->p.finish_fp32_at || r.stall >= 10) r.fp32_now = true;
}

extern "C" {

size_t fctn_last_error(char* buf, size_t n) {
  if (buf && n) {
    size_t c = g_err.size() < n - 1 ? g_err.size() : n - 1;
    memcpy(buf, g_err.data(), c);
    buf[c] = 0;
  }
  return g_err.size();
}

const char* fctn_version(void) { return "libfctn 0.1 (sm_103a)"; }

int fctn_footprint_bytes(const fctn_params* p, size_t* out) {
  int rc = check_params(p);
  if (rc) return rc;
  if (!out) return fail(FCTN_E_ARG, "out is NULL");
  fctn_handle tmp;
  fill_shapes(&tmp, p);
  std::vector<int> tabs, rtabs;
  if ((rc = plan_route(&tmp, &rtabs))) return rc;
  if ((rc = plan_all(&tmp, &tabs, nullptr))) return rc;
  *out = footprint(&tmp) + tabs.size() * sizeof(int) + route_bytes(&tmp, rtabs.size());
  return FCTN_OK;
}

int fctn_create(const fctn_params* p, void* stream, fctn_handle** out) {
  int rc = check_params(p);
  if (rc) return rc;
  if (!out) return fail(FCTN_E_ARG, "out is NULL");
  fctn_handle* h = new fctn_handle();
  fill_shapes(h, p);
  h->st = (cudaStream_t)stream;
  if (!h->st) {
    // a private blocking stream (ordered with the legacy default stream) so that
    // sweeps can be captured as CUDA graphs
    cudaError_t se = cudaStreamCreate(&h->st);
    if (se != cudaSuccess) {
      delete h;
      return fail(FCTN_E_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(se));
    }
    h->own_stream = true;
  }
  std::vector<int> all_tabs, route_tabs;
  size_t tab_offs[2 * FCTN_MAX_ORDER];  // pair tables, then FactGram tables
  if ((rc = plan_route(h, &route_tabs)) || (rc = plan_all(h, &all_tabs, tab_offs))) {
    if (h->own_stream) cudaStreamDestroy(h->st);
    delete h;
    return rc;
  }
  Sizes z = sizes_of(h);
  const size_t e = h->esz, se = h->f64 ? 8 : 4;
#define A_(ptr, bytes)                                      \
  do {                                                      \
    if ((rc = dalloc(h, (void**)&(ptr), (bytes)))) {        \
      free_all(h);                                          \
      if (h->own_stream) cudaStreamDestroy(h->st);          \
      delete h;                                             \
      return rc;                                            \
    }                                                       \
  } while (0)
  A_(h->X, h->P * e);
  A_(h->bits, ((h->P + 31) / 32) * 4);
  if (z.M) A_(h->M, z.M * e);
  if (z.lbuf) A_(h->Lbuf, z.lbuf * e);
  A_(h->ones, 16);
  if (z.chain) { A_(h->chain[0], z.chain * e); A_(h->chain[1], z.chain * e); }
  if (reuse_pairs(h)) { A_(h->T[0], z.T[0] * e); A_(h->T[1], z.T[1] * e); }
  A_(h->part, z.part * e);
  if (z.hbuf) A_(h->hbuf, z.hbuf * e);
  for (int k = 0; k < h->N; ++k) {
    A_(h->A64[k], h->I[k] * h->s[k] * 8);
    A_(h->Ac[k], h->I[k] * h->s[k] * e);
    A_(h->Q64[k], h->I[k] * h->I[k] * 8);
    A_(h->Q32[k], h->I[k] * h->I[k] * 4);
    A_(h->QT64[k], h->I[k] * h->I[k] * 8);
    A_(h->QT32[k], h->I[k] * h->I[k] * 4);
    A_(h->Lam[k], h->I[k] * 8);
  }
  A_(h->Gd, z.ss * 8);
  A_(h->Yd, z.Is * 8);
  A_(h->Rd, z.Is * 8);
  A_(h->Aprev, z.Is * 8);
  A_(h->Gs, z.ss * se);
  A_(h->Ys, z.Is * se);
  A_(h->C, z.ss * se);
  A_(h->Phi, z.maxs * se);
  A_(h->W1, z.Is * se);
  A_(h->Z, z.Is * se);
  A_(h->W2, z.Is * se);
  A_(h->Rs, z.Is * 4);
  A_(h->gwork, 4 * z.ss * se);
  if (!h->f64) {
    size_t rec = 0;
    for (int k = 0; k < h->N; ++k) rec = std::max(rec, eig_record_floats((int)h->s[k]));
    if (rec) A_(h->eig_rec, rec * 4);
  }
  {
    size_t nl, nd;
    chol_floats(h, &nl, &nd);
    if (nl) {
      A_(h->cholL, nl * 4);
      A_(h->cholD, nd * 4);
      A_(h->cholRt, z.Is * 4);
      A_(h->Alo, z.Is * 4);
    }
  }
  A_(h->status, 16);
  A_(h->eig_used, FCTN_MAX_ORDER * sizeof(int));
  for (int k = 0; k < h->N; ++k) A_(h->Ck[k], h->s[k] * h->s[k] * se);
  A_(h->red, z.red_blocks * 3 * 8);
  A_(h->traces, h->N * 32 * 8);
  A_(h->stats, 8 * 8);
  h->stage_bytes = (size_t)(h->P > z.maxfac ? h->P : z.maxfac) * e;
  A_(h->stage, h->stage_bytes);
  A_(h->stage_mask, h->P);
  if (h->hr.on) {
    HeadRoute& r = h->hr;
    A_(r.M0, (size_t)r.s0 * r.P0 * 4);
    A_(r.Zb, (size_t)r.s0 * r.P0 * 4);
    A_(r.U[0], (size_t)r.u_elems * 4);
    A_(r.U[1], (size_t)r.u_elems * 4);
    A_(r.E[0], (size_t)r.e_elems * 4);
    A_(r.E[1], (size_t)r.e_elems * 4);
    A_(r.pm, (size_t)r.part_main * 4);
    A_(r.ps, (size_t)r.part_side * 4);
    for (int k = 0; k < h->N; ++k) A_(r.H[k], (size_t)h->s[k] * h->s[k] * 4);
    A_(r.Yraw, (size_t)z.Is * 4);
    A_(r.tabs, route_tabs.size() * sizeof(int));
    if (r.tc) {
      const size_t el = r.bf16 ? 2 : 4;
      const int64_t I0 = h->I[0];
      A_(r.M0T, (size_t)r.P0 * r.ld0 * 4);
      A_(r.XT, (size_t)r.P0 * r.ldt * el);
      A_(r.A0T, (size_t)r.s0 * r.ldt * el);
      A_(r.A0p, (size_t)I0 * r.ld0 * 4);
      if (r.bf16) {
        A_(r.Xb, (size_t)h->P * 2);
        A_(r.M0b, (size_t)r.s0 * r.P0 * 2);
      }
      A_(r.tpart, (size_t)r.ty.ksplit * I0 * r.s0 * 4);
      const int e = (int)el;
      int mrc = tg_make_map(r.maps[0], r.bf16 ? r.Xb : h->X, I0, r.P0, r.P0, e, 128);
      if (!mrc) mrc = tg_make_map(r.maps[1], r.bf16 ? r.M0b : (void*)r.M0, r.s0, r.P0, r.P0, e, r.ty.BN);
      if (!mrc) mrc = tg_make_map(r.maps[2], r.XT, r.P0, I0, r.ldt, e, 128);
      if (!mrc) mrc = tg_make_map(r.maps[3], r.A0T, r.s0, I0, r.ldt, e, r.tz.BN);
      if (!mrc) mrc = tg_make_map(r.maps[4], r.M0T, r.P0, r.s0, r.ld0, 4, 128);
      if (!mrc) mrc = tg_make_map(r.maps[5], r.A0p, I0, r.s0, r.ld0, 4, r.tf.BN);
      if (mrc) r.tc = false;  // no tensor maps here: the CUDA-core products serve instead
    }
    cudaError_t ce = cudaMemcpy(r.tabs, route_tabs.data(), route_tabs.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) {
      free_all(h);
      if (h->own_stream) cudaStreamDestroy(h->st);
      delete h;
      return fail(FCTN_E_CUDA, "fctn_create: %s", cudaGetErrorString(ce));
    }
  }
  {
    // index tables of the pair forms
    std::vector<int>& all = all_tabs;
    size_t* offs = tab_offs;
    A_(h->tabs, all.size() * sizeof(int));
    for (int k = 0; k < h->N; ++k) {
      h->pp[k].tab = h->tabs + offs[k];
      h->fg[k].tab = h->tabs + offs[FCTN_MAX_ORDER + k];
    }
    cudaError_t ce = cudaMemcpy(h->tabs, all.data(), all.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) {
      if (h->f64) {
        double one = 1.0;
        ce = cudaMemcpy(h->ones, &one, sizeof one, cudaMemcpyHostToDevice);
      } else {
        float one = 1.0f;
        ce = cudaMemcpy(h->ones, &one, sizeof one, cudaMemcpyHostToDevice);
      }
    }
    if (ce != cudaSuccess) {
      free_all(h);
      if (h->own_stream) cudaStreamDestroy(h->st);
      delete h;
      return fail(FCTN_E_CUDA, "fctn_create: %s", cudaGetErrorString(ce));
    }
  }
#undef A_
  bool any_fact = h->hr.on;  // the route's Gram chains run on the side stream too
  for (int k = 0; k < h->N; ++k) any_fact = any_fact || h->fg[k].use;
  if (any_fact) {
    cudaError_t ce = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
    if (ce != cudaSuccess) {
      release_side(h);
      free_all(h);
      if (h->own_stream) cudaStreamDestroy(h->st);
      delete h;
      return fail(FCTN_E_CUDA, "fctn_create: %s", cudaGetErrorString(ce));
    }
  }
  for (int k = 0; k < h->N; ++k) {
    // min_i lambda_k Lambda_i over the closed-form spectrum of L_k
    const double sg = p->laplacian_sign == FCTN_LAPLACIAN_PRINTED ? -1.0 : 1.0;
    double mn = 1e300;
    for (int64_t j = 0; j < h->I[k]; ++j) {
      double mu = sg * (2.0 + p->delta[k] - 2.0 * cos(2.0 * M_PI * (double)j / (double)h->I[k]));
      double v = p->lambda[k] * mu;
      if (v < mn) mn = v;
    }
    h->lam_min[k] = mn;
    launch_laplacian_basis(h->I[k], p->delta[k], p->laplacian_sign, h->Q64[k], h->Q32[k], h->QT64[k], h->QT32[k],
                           h->Lam[k], h->st);
    h->launches++;
  }
  cudaError_t ce = cudaMemsetAsync(h->status, 0, 16, h->st);
  if (ce == cudaSuccess) ce = cudaGetLastError();
  if (ce != cudaSuccess) {
    free_all(h);
    delete h;
    return fail(FCTN_E_CUDA, "fctn_create: %s", cudaGetErrorString(ce));
  }
  *out = h;
  return FCTN_OK;
}

int fctn_set_data(fctn_handle* h, const void* Y, const uint8_t* mask, int where) {
  if (!h || !Y || !mask) return fail(FCTN_E_ARG, "NULL argument");
  int rc;
  const void* ysrc = Y;
  const uint8_t* msrc = mask;
  if (where == FCTN_HOST) {
    if ((rc = copy_in(h, h->stage, Y, h->P * h->esz, where))) return rc;
    if ((rc = copy_in(h, h->stage_mask, mask, h->P, where))) return rc;
    ysrc = h->stage;
    msrc = h->stage_mask;
  } else if (where != FCTN_DEVICE) {
    return fail(FCTN_E_ARG, "where must be FCTN_HOST or FCTN_DEVICE");
  }
  if (h->f64)
    launch_init_x_mask_f64((const double*)ysrc, msrc, (double*)h->X, h->bits, h->P, h->st);
  else
    launch_init_x_mask_f32((const float*)ysrc, msrc, (float*)h->X, h->bits, h->P, h->st);
  LCHK();
  h->data_set = true;
  h->t = 0;
  h->Tvalid[0] = h->Tvalid[1] = false;
  for (int k = 0; k < h->N; ++k) h->cvalid[k] = false;
  h->hr.xt_valid = false;
  h->hr.fp32_now = false;
  h->hr.prev_rel = 0.0;
  h->hr.stall = 0;
  return FCTN_OK;
}

// New entries of a factor under rank growth: scale (2u - 1) with u the
// (c + 1)-th output of SplitMix64 (Steele, Lea & Flood 2014) seeded with
// `seed`, c = k 2^40 + idx (idx: row-major index in factor k's new FCTN
// shape), mapped to [0, 1) by its top 53 bits.
static double growth_noise(uint64_t seed, int k, uint64_t idx, double scale) {
  uint64_t z = seed + ((((uint64_t)k) << 40) + idx + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z ^= z >> 31;
  const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
  return scale * (2.0 * u - 1.0);
}

int fctn_grow_ranks(fctn_handle* h, const int32_t ranks[FCTN_MAX_ORDER][FCTN_MAX_ORDER], double scale,
                    uint64_t seed) {
  if (!h || !ranks) return fail(FCTN_E_ARG, "NULL argument");
  if (!h->data_set || !h->factors_set) return fail(FCTN_E_STATE, "data and factors must be set");
  const int N = h->N;
  fctn_params p2 = h->p;
  bool grow = false;
  for (int a = 0; a < N; ++a)
    for (int b = a + 1; b < N; ++b) {
      if (ranks[a][b] < h->R[a][b]) return fail(FCTN_E_ARG, "rank (%d,%d) would shrink", a, b);
      grow = grow || ranks[a][b] > h->R[a][b];
      p2.ranks[a][b] = ranks[a][b];
    }
  if (!grow) return FCTN_OK;
  int rc = check_params(&p2);
  if (rc) return rc;
  // current factors, FP64 master, in the FCTN layout
  std::vector<std::vector<double>> old(N);
  for (int k = 0; k < N; ++k) {
    const size_t n = (size_t)(h->I[k] * h->s[k]);
    View src = factor_view(h, k), dst = factor_d1_view(h, k);
    ContractPlan pl;
    View ov;
    if ((rc = make_plan(src, nullptr, dst.lab, dst.n, &pl, &ov))) return rc;
    launch_contract_f64(h->A64[k], nullptr, h->Aprev, pl, h->st);
    h->launches++;
    CK(cudaGetLastError());
    old[k].resize(n);
    CK(cudaMemcpyAsync(old[k].data(), h->Aprev, n * 8, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
  }
  fctn_handle* h2 = nullptr;
  if ((rc = fctn_create(&p2, (void*)h->st, &h2))) return rc;
  // the completed tensor, mask and sweep count carry over
  cudaError_t ce = cudaMemcpyAsync(h2->X, h->X, (size_t)h->P * h->esz, cudaMemcpyDeviceToDevice, h->st);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(h2->bits, h->bits, (size_t)((h->P + 31) / 32) * 4, cudaMemcpyDeviceToDevice, h->st);
  if (ce != cudaSuccess) {
    fctn_destroy(h2);
    return fail(FCTN_E_CUDA, "fctn_grow_ranks: %s", cudaGetErrorString(ce));
  }
  h2->data_set = true;
  // factors padded along the grown bonds
  std::vector<std::vector<unsigned char>> nf(N);
  std::vector<const void*> ptrs(N);
  for (int k = 0; k < N; ++k) {
    int64_t oe[FCTN_MAX_ORDER], ne[FCTN_MAX_ORDER];
    for (int t = 0; t < N; ++t) {
      oe[t] = t == k ? h->I[k] : h->R[t < k ? t : k][t < k ? k : t];
      ne[t] = t == k ? h->I[k] : h2->R[t < k ? t : k][t < k ? k : t];
    }
    const size_t n = (size_t)(h2->I[k] * h2->s[k]);
    nf[k].resize(n * h2->esz);
    int64_t d[FCTN_MAX_ORDER] = {};
    for (size_t e = 0; e < n; ++e) {
      // multi-index of e (row-major over ne), old flat index if inside
      int64_t r = (int64_t)e, of = 0, ost = 1;
      bool inside = true;
      for (int t = N - 1; t >= 0; --t) {
        d[t] = r % ne[t];
        r /= ne[t];
      }
      for (int t = N - 1; t >= 0; --t) {
        inside = inside && d[t] < oe[t];
        of += d[t] * ost;
        ost *= oe[t];
      }
      const double v = inside ? old[k][(size_t)of] : growth_noise(seed, k, (uint64_t)e, scale);
      if (h2->f64)
        ((double*)nf[k].data())[e] = v;
      else
        ((float*)nf[k].data())[e] = (float)v;
    }
    ptrs[k] = nf[k].data();
  }
  if ((rc = fctn_set_factors(h2, ptrs.data(), FCTN_HOST))) {
    fctn_destroy(h2);
    return rc;
  }
  h2->t = h->t;  // after fctn_set_factors, which starts a new run at t = 0
  CK(cudaStreamSynchronize(h->st));
  // h takes the new state; h2 takes the old one (and not the stream) and goes
  std::swap(*h, *h2);
  std::swap(h->own_stream, h2->own_stream);
  h->launches += h2->launches;
  return fctn_destroy(h2);
}

int fctn_autotune(const fctn_params* p, const void* Y, const uint8_t* mask, const void* const* factors, int where,
                  const int32_t* cand, int ncand, int sweeps, void* cuda_stream, int32_t* best, double* ms_out) {
  static const int32_t builtin[6] = {96, 120, 152, 192, 228, 304};
  if (!p || !Y || !mask || !factors || !best) return fail(FCTN_E_ARG, "NULL argument");
  if (sweeps < 1 || sweeps > 1000) return fail(FCTN_E_ARG, "sweeps %d outside [1, 1000]", sweeps);
  if (!cand) {
    cand = builtin;
    ncand = 6;
  }
  if (ncand < 1 || ncand > 64) return fail(FCTN_E_ARG, "ncand %d outside [1, 64]", ncand);
  for (int i = 0; i < ncand; ++i)
    if (cand[i] < 0 || cand[i] > 16 * 152) return fail(FCTN_E_ARG, "candidate %d outside [0, 2432]", cand[i]);
  int rc = check_params(p);
  if (rc) return rc;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(FCTN_E_CUDA, "fctn_autotune: cudaEventCreate failed");
  }
  double best_ms = 0.0;
  for (int i = 0; i < ncand && rc == FCTN_OK; ++i) {
    fctn_params q = *p;
    q.rhs_ctas = cand[i];
    fctn_handle* h = nullptr;
    if ((rc = fctn_create(&q, cuda_stream, &h))) break;
    fctn_stats st{};
    float ms = 0.f;
    if (!(rc = fctn_set_data(h, Y, mask, where)) && !(rc = fctn_set_factors(h, factors, where)) &&
        !(rc = fctn_pam_sweep(h, 2 * sweeps, nullptr))) {
      cudaError_t ce = cudaEventRecord(e0, h->st);
      if (ce == cudaSuccess) rc = fctn_pam_sweep(h, sweeps, nullptr);
      if (ce == cudaSuccess && !rc) ce = cudaEventRecord(e1, h->st);
      if (ce == cudaSuccess && !rc) ce = cudaEventSynchronize(e1);
      if (ce == cudaSuccess && !rc) ce = cudaEventElapsedTime(&ms, e0, e1);
      if (ce != cudaSuccess) rc = fail(FCTN_E_CUDA, "fctn_autotune: %s", cudaGetErrorString(ce));
      if (!rc && !(rc = fctn_pam_sweep(h, 0, &st)) && st.status != FCTN_OK)
        rc = fail(st.status, "fctn_autotune: probe sweep failed with status %d", st.status);
    }
    const int drc = fctn_destroy(h);
    if (!rc) rc = drc;
    if (rc) break;
    const double per = (double)ms / sweeps;
    if (ms_out) ms_out[i] = per;
    if (i == 0 || per < best_ms) {
      best_ms = per;
      *best = cand[i];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

int fctn_autotune_tiles(const fctn_params* p, const void* Y, const uint8_t* mask, const void* const* factors,
                        int where, const int32_t* cand, int ncand, int sweeps, void* cuda_stream, int32_t* best,
                        double* ms_out) {
  // the built-in rule; CUDA-core products; 2 / 4 pipeline stages; K split of
  // X_(1) M_1^T over 152 / 608 CTAs; K split of the table-driven contractions
  // over 152 / 608 CTAs / none; programmatic dependent launches in the solve
  // chain, alone and with the two K splits over 152 CTAs
  static const int32_t builtin[12] = {0, 1, 2, 4, 8, 16, 32, 64, 96, 128, 136, 160};
  if (!p || !Y || !mask || !factors || !best) return fail(FCTN_E_ARG, "NULL argument");
  if (sweeps < 1 || sweeps > 1000) return fail(FCTN_E_ARG, "sweeps %d outside [1, 1000]", sweeps);
  if (!cand) {
    cand = builtin;
    ncand = 12;
  }
  if (ncand < 1 || ncand > 64) return fail(FCTN_E_ARG, "ncand %d outside [1, 64]", ncand);
  for (int i = 0; i < ncand; ++i)
    if (cand[i] < 0 || cand[i] > 255) return fail(FCTN_E_ARG, "candidate %d outside [0, 255]", cand[i]);
  int rc = check_params(p);
  if (rc) return rc;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(FCTN_E_CUDA, "fctn_autotune_tiles: cudaEventCreate failed");
  }
  double best_ms = 0.0;
  for (int i = 0; i < ncand && rc == FCTN_OK; ++i) {
    fctn_params q = *p;
    q.tile_code = cand[i];
    fctn_handle* h = nullptr;
    if ((rc = fctn_create(&q, cuda_stream, &h))) break;
    fctn_stats st{};
    float ms = 0.f;
    if (!(rc = fctn_set_data(h, Y, mask, where)) && !(rc = fctn_set_factors(h, factors, where)) &&
        !(rc = fctn_pam_sweep(h, 2 * sweeps, nullptr))) {
      cudaError_t ce = cudaEventRecord(e0, h->st);
      if (ce == cudaSuccess) rc = fctn_pam_sweep(h, sweeps, nullptr);
      if (ce == cudaSuccess && !rc) ce = cudaEventRecord(e1, h->st);
      if (ce == cudaSuccess && !rc) ce = cudaEventSynchronize(e1);
      if (ce == cudaSuccess && !rc) ce = cudaEventElapsedTime(&ms, e0, e1);
      if (ce != cudaSuccess) rc = fail(FCTN_E_CUDA, "fctn_autotune_tiles: %s", cudaGetErrorString(ce));
      if (!rc && !(rc = fctn_pam_sweep(h, 0, &st)) && st.status != FCTN_OK)
        rc = fail(st.status, "fctn_autotune_tiles: probe sweep failed with status %d", st.status);
    }
    const int drc = fctn_destroy(h);
    if (!rc) rc = drc;
    if (rc) break;
    const double per = (double)ms / sweeps;
    if (ms_out) ms_out[i] = per;
    if (i == 0 || per < best_ms) {
      best_ms = per;
      *best = cand[i];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

int fctn_quality(fctn_handle* h, const void* truth, int where, double* psnr, double* ssim) {
  if (!h || !truth) return fail(FCTN_E_ARG, "NULL argument");
  if (!h->data_set) return fail(FCTN_E_STATE, "no data set");
  if (where != FCTN_HOST && where != FCTN_DEVICE) return fail(FCTN_E_ARG, "where must be FCTN_HOST or FCTN_DEVICE");
  int rc;
  const void* tsrc = truth;
  if (where == FCTN_HOST) {
    if ((rc = copy_in(h, h->stage, truth, h->P * h->esz, where))) return rc;
    tsrc = h->stage;
  }
  const int64_t rows = h->N >= 2 ? h->I[0] * h->I[1] : h->I[0];
  const int64_t ncol = h->P / rows;
  const int nblocks = 152;
  const size_t need = quality_work_doubles(ncol, nblocks) + 2;
  if (h->qwork_n < need) {
    void* p = nullptr;
    if ((rc = dalloc(h, &p, need * sizeof(double)))) return rc;
    h->qwork = (double*)p;
    h->qwork_n = need;
  }
  double* out = h->qwork + need - 2;
  if (h->f64)
    launch_quality_f64((const double*)h->X, (const double*)tsrc, rows, ncol, 1e-4, 9e-4, h->qwork, nblocks, out,
                       h->st);
  else
    launch_quality_f32((const float*)h->X, (const float*)tsrc, rows, ncol, 1e-4, 9e-4, h->qwork, nblocks, out,
                       h->st);
  h->launches += 2;
  CK(cudaGetLastError());
  double v[2];
  CK(cudaMemcpyAsync(v, out, sizeof v, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (psnr) *psnr = v[0];
  if (ssim) *ssim = v[1];
  return FCTN_OK;
}

int fctn_set_factors(fctn_handle* h, const void* const* factors, int where) {
  if (!h || !factors) return fail(FCTN_E_ARG, "NULL argument");
  int rc;
  for (int k = 0; k < h->N; ++k) {
    if (!factors[k]) return fail(FCTN_E_ARG, "factor %d is NULL", k);
    const size_t n = (size_t)(h->I[k] * h->s[k]);
    if ((rc = copy_in(h, h->stage, factors[k], n * h->esz, where))) return rc;
    View src = factor_d1_view(h, k), dst = factor_view(h, k);
    ContractPlan pl;
    View ov;
    if ((rc = make_plan(src, nullptr, dst.lab, dst.n, &pl, &ov))) return rc;
    if ((rc = launch_plan(h, h->stage, nullptr, h->Ac[k], pl))) return rc;
    if (h->f64) {
      CK(cudaMemcpyAsync(h->A64[k], h->Ac[k], n * 8, cudaMemcpyDeviceToDevice, h->st));
    } else {
      launch_convert_f32_to_f64((const float*)h->Ac[k], h->A64[k], (int64_t)n, h->st);
      LCHK();
    }
    h->ver[k] = 0;
  }
  h->factors_set = true;
  h->t = 0;
  h->Tvalid[0] = h->Tvalid[1] = false;
  for (int k = 0; k < h->N; ++k) h->cvalid[k] = false;
  h->hr.m0_valid = false;
  for (int k = 0; k < h->N; ++k) h->hr.hvalid[k] = false;
  h->hr.fp32_now = false;
  h->hr.prev_rel = 0.0;
  h->hr.stall = 0;
  return FCTN_OK;
}

int fctn_contract(fctn_handle* h, void* out, int where) {
  if (!h || !out) return fail(FCTN_E_ARG, "NULL argument");
  if (!h->factors_set) return fail(FCTN_E_STATE, "factors not set");
  Lab fin[FCTN_MAXD];
  int ids[FCTN_MAX_ORDER];
  for (int t = 0; t < h->N; ++t) {
    fin[t] = mode_lab(t);
    ids[t] = t;
  }
  void* dst = where == FCTN_DEVICE ? out : h->stage;
  int rc = run_chain(h, ids, h->N, fin, h->N, dst);
  if (rc) return rc;
  if (where == FCTN_HOST) return copy_out(h, out, h->stage, h->P * h->esz, where);
  if (where != FCTN_DEVICE) return fail(FCTN_E_ARG, "where must be FCTN_HOST or FCTN_DEVICE");
  return FCTN_OK;
}

int fctn_pam_sweep(fctn_handle* h, int nsweeps, fctn_stats* stats) {
  if (!h) return fail(FCTN_E_ARG, "NULL handle");
  if (nsweeps < 0) return fail(FCTN_E_ARG, "nsweeps < 0");
  if (!h->data_set || !h->factors_set) return fail(FCTN_E_STATE, "set data and factors before sweeping");
  for (int i = 0; i < nsweeps; ++i) {
    int rc = one_sweep(h);
    if (rc) return rc;
  }
  if (stats) return read_stats(h, stats);
  return FCTN_OK;
}

int fctn_complete(fctn_handle* h, double tol, int max_sweeps, void* out_X, int where, fctn_stats* stats) {
  if (!h) return fail(FCTN_E_ARG, "NULL handle");
  if (!h->data_set || !h->factors_set) return fail(FCTN_E_STATE, "set data and factors before sweeping");
  fctn_stats st{};
  int converged = 0;
  int rc = FCTN_OK;
  do {
    if ((rc = one_sweep(h))) break;
    if ((rc = read_stats(h, &st))) break;
    if (tol > 0 && st.rel_change <= tol) converged = 1;
    fctn_internal_after_sweep(h, st.rel_change);
  } while (!converged && h->t < max_sweeps);
  st.converged = converged;
  st.status = rc;
  st.t = h->t;
  if (stats) *stats = st;
  if (rc) return rc;
  if (out_X) return copy_out(h, out_X, h->X, h->P * h->esz, where);
  return FCTN_OK;
}

int fctn_get_factor(fctn_handle* h, int k, void* out, int where) {
  if (!h || !out) return fail(FCTN_E_ARG, "NULL argument");
  if (k < 0 || k >= h->N) return fail(FCTN_E_ARG, "factor index %d out of range", k);
  if (!h->factors_set) return fail(FCTN_E_STATE, "factors not set");
  const size_t n = (size_t)(h->I[k] * h->s[k]);
  int rc;
  // FP64 master -> compute precision -> FCTN layout
  void* tmp = h->W1;  // I_k x s_k scratch in solve precision (same width as compute here)
  if (h->f64) {
    CK(cudaMemcpyAsync(tmp, h->A64[k], n * 8, cudaMemcpyDeviceToDevice, h->st));
  } else {
    launch_convert_f64_to_f32(h->A64[k], (float*)tmp, (int64_t)n, h->st);
    LCHK();
  }
  View src = factor_view(h, k), dst = factor_d1_view(h, k);
  ContractPlan pl;
  View ov;
  if ((rc = make_plan(src, nullptr, dst.lab, dst.n, &pl, &ov))) return rc;
  void* d = where == FCTN_DEVICE ? out : h->stage;
  if ((rc = launch_plan(h, tmp, nullptr, d, pl))) return rc;
  if (where == FCTN_HOST) return copy_out(h, out, h->stage, n * h->esz, where);
  return FCTN_OK;
}

int fctn_get_X(fctn_handle* h, void* out, int where) {
  if (!h || !out) return fail(FCTN_E_ARG, "NULL argument");
  if (!h->data_set) return fail(FCTN_E_STATE, "data not set");
  return copy_out(h, out, h->X, h->P * h->esz, where);
}

int fctn_sync(fctn_handle* h) {
  if (!h) return fail(FCTN_E_ARG, "NULL handle");
  CK(cudaStreamSynchronize(h->st));
  return FCTN_OK;
}

int fctn_launch_count(fctn_handle* h, int64_t* out) {
  if (!h || !out) return fail(FCTN_E_ARG, "NULL argument");
  *out = h->launches;
  return FCTN_OK;
}

int fctn_set_graphs(fctn_handle* h, int enable) {
  if (!h) return fail(FCTN_E_ARG, "NULL handle");
  h->use_graphs = enable != 0;
  return FCTN_OK;
}

int fctn_profile(fctn_handle* h, int kernel_class) {
  if (!h) return fail(FCTN_E_ARG, "NULL handle");
  if (kernel_class < -1 || kernel_class >= FCTN_KC_COUNT) return fail(FCTN_E_ARG, "unknown kernel class %d", kernel_class);
  CK(cudaStreamSynchronize(h->st));
  h->prof_class = kernel_class;
  h->prof_used = 0;
  h->prof_ms = h->prof_bytes = h->prof_flops = 0.0;
  h->cls_bytes = h->cls_flops = 0.0;
  h->cls_launches = 0;
  return FCTN_OK;
}

int fctn_profile_read(fctn_handle* h, int64_t* launches, double* ms, double* alg_bytes, double* alg_flops) {
  if (!h) return fail(FCTN_E_ARG, "NULL handle");
  CK(cudaStreamSynchronize(h->st));
  for (size_t i = 0; i + 1 < h->prof_used; i += 2) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, h->prof_ev[i], h->prof_ev[i + 1]));
    h->prof_ms += t;
  }
  h->prof_used = 0;
  if (launches) *launches = h->cls_launches;
  if (ms) *ms = h->prof_ms;
  if (alg_bytes) *alg_bytes = h->cls_bytes;
  if (alg_flops) *alg_flops = h->cls_flops;
  return FCTN_OK;
}

int fctn_destroy(fctn_handle* h) {
  if (!h) return FCTN_OK;
  cudaStreamSynchronize(h->st);
  for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
  for (auto e : h->prof_ev) cudaEventDestroy(e);
  release_side(h);
  free_all(h);
  if (h->own_stream) cudaStreamDestroy(h->st);
  delete h;
  return FCTN_OK;
}

}  // extern "C"
