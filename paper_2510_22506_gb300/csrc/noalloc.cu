// fctn_contract_noalloc: the FCTN contraction without any device allocation.
//
// The two intermediates of the ascending contraction chain live in one
// file-scope device array (FCTN_NOALLOC_SCRATCH_BYTES, split in two halves).
// Host code cannot use the array's name as a device address: every call asks
// for its address with cudaGetSymbolAddress, with the caller's device
// current, and passes that address to the kernels.  The lookup is repeated
// per call (it is cheap next to the launches) so that a device reset or a new
// primary context, which can move the array, never leaves a stale address.
#include <cstring>

#include "fctn_internal.cuh"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[FCTN_NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array on the current device.
int scratch_address(void** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();  // the failed lookup is reported here, not by a later call
    return fctn_internal_fail(FCTN_E_CUDA, "cudaGetSymbolAddress of the scratch array failed");
  }
  *out = p;
  return FCTN_OK;
}

// Labels: mode t -> (0, t); bond (a, b), a < b -> (1, a * 8 + b).
struct NLab {
  int kind, id;
  bool operator==(const NLab& o) const { return kind == o.kind && id == o.id; }
};

struct NView {
  int n = 0;
  NLab lab[FCTN_MAXD];
  int64_t ext[FCTN_MAXD], str[FCTN_MAXD];
  int find(const NLab& l) const {
    for (int i = 0; i < n; ++i)
      if (lab[i] == l) return i;
    return -1;
  }
  int64_t size() const {
    int64_t s = 1;
    for (int i = 0; i < n; ++i) s *= ext[i];
    return s;
  }
  void dense() {
    int64_t st = 1;
    for (int i = n - 1; i >= 0; --i) {
      str[i] = st;
      st *= ext[i];
    }
  }
};

NLab bond(int a, int b) { return NLab{1, (a < b ? a : b) * 8 + (a < b ? b : a)}; }

// Factor k in its FCTN shape: position t holds mode k (t == k) or bond (k, t).
NView factor_view(int N, const int64_t* dims, const int32_t* R, int k) {
  NView v;
  v.n = N;
  for (int t = 0; t < N; ++t) {
    if (t == k) {
      v.lab[t] = NLab{0, k};
      v.ext[t] = dims[k];
    } else {
      v.lab[t] = bond(k, t);
      v.ext[t] = R[(k < t ? k : t) * N + (k < t ? t : k)];
    }
  }
  v.dense();
  return v;
}

int plan(const NView& A, const NView& B, const NLab* out, int nout, ContractPlan* p, NView* ov) {
  memset(p, 0, sizeof *p);
  ov->n = nout;
  for (int i = 0; i < nout; ++i) {
    int ia = A.find(out[i]), ib = B.find(out[i]);
    ov->lab[i] = out[i];
    ov->ext[i] = ia >= 0 ? A.ext[ia] : B.ext[ib];
    p->out_ext[i] = ov->ext[i];
    p->a_str[i] = ia >= 0 ? A.str[ia] : 0;
    p->b_str[i] = ib >= 0 ? B.str[ib] : 0;
  }
  p->nout = nout;
  p->con_size = 1;
  for (int i = 0; i < A.n; ++i) {
    bool in_out = false;
    for (int j = 0; j < nout; ++j) in_out |= (out[j] == A.lab[i]);
    if (in_out) continue;
    int ib = B.find(A.lab[i]);
    if (ib < 0 || p->ncon >= FCTN_MAXC) return fctn_internal_fail(FCTN_E_ARG, "inconsistent FCTN ranks");
    p->con_ext[p->ncon] = A.ext[i];
    p->ca_str[p->ncon] = A.str[i];
    p->cb_str[p->ncon] = B.str[ib];
    p->con_size *= A.ext[i];
    p->ncon++;
  }
  if (p->con_size > FCTN_CON_TABLE) return fctn_internal_fail(FCTN_E_UNSUPPORTED, "contraction length too large");
  ov->dense();
  p->out_size = ov->size();
  return FCTN_OK;
}

}  // namespace

extern "C" int fctn_contract_noalloc(int order, const int64_t* dims, const int32_t* ranks, int precision,
                                     const void* const* factors, void* out, void* cuda_stream) {
  if (order < 2 || order > FCTN_MAX_ORDER || !dims || !ranks || !factors || !out)
    return fctn_internal_fail(FCTN_E_ARG, "fctn_contract_noalloc: bad order or NULL argument");
  if (precision != FCTN_FP64 && precision != FCTN_FP32)
    return fctn_internal_fail(FCTN_E_ARG, "fctn_contract_noalloc: precision must be FCTN_FP64 or FCTN_FP32");
  const int N = order;
  for (int k = 0; k < N; ++k) {
    if (dims[k] < 1 || !factors[k]) return fctn_internal_fail(FCTN_E_ARG, "fctn_contract_noalloc: bad size or factor");
    for (int t = k + 1; t < N; ++t)
      if (ranks[k * N + t] < 1) return fctn_internal_fail(FCTN_E_ARG, "fctn_contract_noalloc: ranks must be >= 1");
  }
  const size_t esz = precision == FCTN_FP64 ? 8 : 4;
  const size_t half = (size_t)FCTN_NOALLOC_SCRATCH_BYTES / 2;
  // plan the chain and check every intermediate against the scratch limit
  ContractPlan plans[FCTN_MAX_ORDER];
  NView cur = factor_view(N, dims, ranks, 0);
  for (int i = 1; i < N; ++i) {
    NView nx = factor_view(N, dims, ranks, i);
    NLab ord[FCTN_MAXD];
    int n = 0;
    bool too_many = false;
    auto push = [&](const NLab& l) {
      if (n >= FCTN_MAXD) too_many = true;
      else ord[n++] = l;
    };
    if (i == N - 1) {
      for (int t = 0; t < N; ++t) push(NLab{0, t});
    } else {
      for (int q = 0; q < cur.n; ++q)
        if (nx.find(cur.lab[q]) < 0) push(cur.lab[q]);
      for (int q = 0; q < nx.n; ++q)
        if (cur.find(nx.lab[q]) < 0) push(nx.lab[q]);
    }
    if (too_many) return fctn_internal_fail(FCTN_E_UNSUPPORTED, "fctn_contract_noalloc: too many indices");
    NView ov;
    int rc = plan(cur, nx, ord, n, &plans[i], &ov);
    if (rc) return rc;
    if (i < N - 1 && (size_t)ov.size() * esz > half)
      return fctn_internal_fail(FCTN_E_ARG,
                                "fctn_contract_noalloc: an intermediate exceeds the scratch limit "
                                "(FCTN_NOALLOC_SCRATCH_BYTES / 2 per intermediate)");
    cur = ov;
  }
  // an error left pending by earlier, unrelated work on this thread would be
  // read back after the first launch below and abort the chain half-way; it
  // is reported (and cleared) here instead, before anything is queued
  cudaError_t pending = cudaGetLastError();
  if (pending != cudaSuccess)
    return fctn_internal_fail(FCTN_E_CUDA, "fctn_contract_noalloc: a CUDA error was pending before the call");
  void* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  unsigned char* halves[2] = {(unsigned char*)scratch, (unsigned char*)scratch + half};
  const void* src = factors[0];
  for (int i = 1; i < N; ++i) {
    void* dst = (i == N - 1) ? out : (void*)halves[i % 2];
    if (precision == FCTN_FP64)
      launch_contract_f64((const double*)src, (const double*)factors[i], (double*)dst, plans[i], st);
    else
      launch_contract_f32((const float*)src, (const float*)factors[i], (float*)dst, plans[i], st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fctn_internal_fail(FCTN_E_CUDA, cudaGetErrorString(e));
    src = dst;
  }
  return FCTN_OK;
}
