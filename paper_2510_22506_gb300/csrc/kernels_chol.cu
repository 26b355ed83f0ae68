// Shifted-Cholesky solve of the factor subproblem (Eq. 5, Eq. 6).
//
// With the real orthonormal eigenbasis Q of the circulant L_k (L_k = Q diag(mu)
// Q^T, mu_j = c0 + 2 c1 cos(2 pi j / I) for the stencil (c1, c0, c1)), Eq. 5
//   A (G + rho I) + lam L_k A = Y
// becomes, for W = Q^T A, one symmetric positive definite system per row:
//   W_i (G + c_i I) = (Q^T Y)_i,   c_i = lam mu_i + rho
// (Eq. 6 is block diagonal in this basis).  This gives the same unique
// solution as Eq. 8 without the eigendecomposition of G.  The cos and sin
// columns of one frequency j share mu_j, so the I rows need floor(I / 2) + 1
// factorizations ("groups"): group 0 is column 0; group j is columns 2j - 1
// and 2j; for even I, group I / 2 is column I - 1.
//
// Packed panel layout of a factor (s <= 256, padded to sp = 32 np): panel q
// holds rows [32 q, sp) of columns [32 q, 32 q + 32), column-major, element
// (r, 32 q + c) at poff(q) + c (sp - 32 q) + (r - 32 q).  The padding is the
// identity, so it factors to itself and leaves the solution unchanged.
//
// k_chol_factor: one CTA per group: G + c_j I (FP32) in shared memory,
// right-looking blocked Cholesky G + c_j I = L L^T over the panels (the 32 x 32
// diagonal block by one warp in registers, the rows below by one thread each,
// the trailing update in 4 x 8 register tiles of 32 x 32 blocks); writes L and
// the inverses of its diagonal blocks.  A pivot that is not positive means
// that G + c_j I is not positive definite (some T_ij of Eq. 8 <= 0): status
// FCTN_E_SINGULAR, as for the eigen route.
// k_chol_solve: one CTA per group: b = (Q^T R) for the group's rows, R
// streamed through shared memory by bulk copies, then L z = b and L^T w = z
// panel by panel (diagonal blocks through their inverses), w into W.
#include "fctn_internal.cuh"

namespace {

constexpr int CH_NT = 256;
constexpr int CH_MAXS = 256;
constexpr unsigned CH_FULL = 0xffffffffu;

__host__ __device__ inline int ch_npan(int s) { return (s + 31) / 32; }
__host__ __device__ inline int ch_poff(int q, int sp) { return 32 * q * sp - 512 * q * (q - 1); }
__host__ __device__ inline int ch_pack(int s) {
  const int n = ch_npan(s);
  return ch_poff(n, 32 * n);
}

// Rows (basis columns) of group g; returns their number (1 or 2).
__device__ inline int ch_rows(int g, int I, int* r) {
  if (g == 0) {
    r[0] = 0;
    return 1;
  }
  if (2 * g == I) {
    r[0] = I - 1;
    return 1;
  }
  r[0] = 2 * g - 1;
  r[1] = 2 * g;
  return 2;
}

__device__ __forceinline__ unsigned ch_su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__global__ void __launch_bounds__(CH_NT) k_chol_factor(const float* __restrict__ G, int s, int I, double lam,
                                                       double c0, double c1, double rho, float* __restrict__ Lout,
                                                       float* __restrict__ Dout, int* status) {
  extern __shared__ __align__(16) float P[];
  __shared__ float rdiag[32];
  __shared__ int bad;
  const int g = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int np = ch_npan(s), sp = 32 * np;
  const float shift = (float)(lam * (c0 + 2.0 * c1 * cospi(2.0 * (double)g / (double)I)) + rho);
  if (tid == 0) bad = 0;
  // G + c I into the panels; G is symmetric, so element (r, col) is read as
  // G[col][r], consecutive threads on consecutive r
  for (int q = 0; q < np; ++q) {
    const int nr = sp - 32 * q;
    float* Pq = P + ch_poff(q, sp);
    for (int e = tid; e < 32 * nr; e += CH_NT) {
      const int c = e / nr, rl = e - c * nr;
      const int r = 32 * q + rl, col = 32 * q + c;
      float v = (r == col) ? 1.0f : 0.0f;
      if (r < s && col < s) v = G[(size_t)col * s + r] + (r == col ? shift : 0.0f);
      Pq[e] = v;
    }
  }
  __syncthreads();
  for (int p = 0; p < np; ++p) {
    const int nr = sp - 32 * p;
    float* Pp = P + ch_poff(p, sp);
    // 1. diagonal block: lane r holds row r; column j is scaled by
    //    1 / sqrt(pivot), then the rank-1 update of the columns right of it
    if (warp == 0) {
      float d[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) d[c] = Pp[c * nr + lane];
      bool ok = true;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        float piv = __shfl_sync(CH_FULL, d[j], j);
        if (!(piv > 0.0f)) {
          ok = false;
          piv = 1.0f;
        }
        const float rs = rsqrtf(piv);
        d[j] = (lane == j) ? piv * rs : d[j] * rs;
#pragma unroll
        for (int c = j + 1; c < 32; ++c) d[c] = fmaf(-d[j], __shfl_sync(CH_FULL, d[j], c), d[c]);
        if (lane == 0) rdiag[j] = rs;
      }
#pragma unroll
      for (int c = 0; c < 32; ++c)
        if (c <= lane) Pp[c * nr + lane] = d[c];
      if (!ok && lane == 0) bad = 1;
    }
    __syncthreads();
    // 2. rows below the block: x L_pp^T = a, one row per thread
    for (int t = tid; t < nr - 32; t += CH_NT) {
      const int rl = 32 + t;
      float x[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) x[c] = Pp[c * nr + rl];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        x[j] *= rdiag[j];
#pragma unroll
        for (int k = j + 1; k < 32; ++k) x[k] = fmaf(-x[j], Pp[j * nr + k], x[k]);
      }
#pragma unroll
      for (int c = 0; c < 32; ++c) Pp[c * nr + rl] = x[c];
    }
    __syncthreads();
    // 3. trailing update: block (rb, q), p < q <= rb < np, of panel q minus
    //    L[rb rows, panel p] L[q rows, panel p]^T; one warp per block
    const int nt = np - 1 - p, ntile = nt * (nt + 1) / 2;
    const int r0 = (lane & 7) * 4, cb = (lane >> 3) * 8;
    for (int ti = warp; ti < ntile; ti += CH_NT / 32) {
      int q = p + 1, rem = ti;
      while (rem >= np - q) {
        rem -= np - q;
        ++q;
      }
      const int rb = q + rem;
      const float* Ap = Pp + (32 * rb - 32 * p) + r0;
      const float* Bp = Pp + (32 * q - 32 * p) + cb;
      float acc[4][8];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
#pragma unroll 4
      for (int k = 0; k < 32; ++k) {
        const float4 a = *reinterpret_cast<const float4*>(Ap + k * nr);
        const float4 b0 = *reinterpret_cast<const float4*>(Bp + k * nr);
        const float4 b1 = *reinterpret_cast<const float4*>(Bp + k * nr + 4);
        const float av[4] = {a.x, a.y, a.z, a.w};
        const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
      }
      const int nq = sp - 32 * q;
      float* Cq = P + ch_poff(q, sp) + (32 * rb - 32 * q) + r0;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float4* o = reinterpret_cast<float4*>(Cq + (cb + j) * nq);
        float4 v = *o;
        v.x -= acc[0][j];
        v.y -= acc[1][j];
        v.z -= acc[2][j];
        v.w -= acc[3][j];
        *o = v;
      }
    }
    __syncthreads();
  }
  // L (packed) to global memory
  const int tot = ch_pack(s);
  float* Lg = Lout + (size_t)g * tot;
  for (int e = tid * 4; e < tot; e += CH_NT * 4)
    *reinterpret_cast<float4*>(Lg + e) = *reinterpret_cast<const float4*>(P + e);
  // inverses of the diagonal blocks, row-major: lane c forms column c of
  // L_pp^{-1} by forward substitution on e_c
  for (int p = warp; p < np; p += CH_NT / 32) {
    const int nr = sp - 32 * p;
    const float* Pp = P + ch_poff(p, sp);
    float y[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) y[k] = (k == lane) ? 1.0f : 0.0f;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      y[j] *= __frcp_rn(Pp[j * nr + j]);
#pragma unroll
      for (int k = j + 1; k < 32; ++k) y[k] = fmaf(-Pp[j * nr + k], y[j], y[k]);
    }
    float* Dg = Dout + ((size_t)g * np + p) * 1024;
#pragma unroll
    for (int k = 0; k < 32; ++k) Dg[k * 32 + lane] = y[k];
  }
  if (tid == 0 && bad) atomicCAS(status, FCTN_OK, FCTN_E_SINGULAR);
}

// Shared-memory layout of k_chol_solve (byte offsets, 16-byte aligned).
struct ChSolveLayout {
  size_t l, rs, ds, b, qs, red, total;
  int NC;
};
__host__ __device__ inline size_t ch_al16(size_t b) { return (b + 15) & ~(size_t)15; }
__host__ __device__ inline ChSolveLayout ch_solve_layout(int I, int s) {
  ChSolveLayout o;
  const int np = ch_npan(s), sp = 32 * np;
  const size_t fixed = (size_t)ch_pack(s) * 4 + (size_t)np * 32 * 33 * 4 + 2 * (size_t)sp * 4 + 64 * 4 + 256;
  const size_t budget = 216 * 1024;
  long nc = budget > fixed ? (long)((budget - fixed) / (2 * 4 * (size_t)s + 16)) : 4;
  nc = nc > 32 ? 32 : nc;
  nc = nc < 4 ? 4 : (nc & ~3L);
  if (nc > I) nc = I;
  // the partial sums of the column groups reuse the staging buffers
  const int KS = s >= CH_NT ? 1 : CH_NT / s;
  const long need = (KS * 2 * (long)s + 2 * (long)s - 1) / (2 * (long)s);
  if (nc < need) nc = need;
  o.NC = (int)nc;
  o.l = 0;
  o.rs = ch_al16(o.l + (size_t)ch_pack(s) * 4);
  o.ds = ch_al16(o.rs + 2 * (size_t)o.NC * s * 4);
  o.b = ch_al16(o.ds + (size_t)np * 32 * 33 * 4);
  o.qs = ch_al16(o.b + 2 * (size_t)sp * 4);
  o.red = ch_al16(o.qs + 4 * (size_t)o.NC * 4);
  o.total = ch_al16(o.red + 64 * 4);
  return o;
}

__device__ __forceinline__ bool ch_wait(uint64_t* bar, unsigned phase) {
  for (long long it = 0; it < (1ll << 26); ++it) {
    unsigned r;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(r)
        : "r"(ch_su32(bar)), "r"(phase));
    if (r) return true;
  }
  return false;
}

__device__ __forceinline__ void ch_bulk(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(ch_su32(bar)), "r"(bytes));
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(ch_su32(dst)),
      "l"(src), "r"(bytes), "r"(ch_su32(bar))
      : "memory");
}

__global__ void __launch_bounds__(CH_NT) k_chol_solve(const float* __restrict__ QT, const float* __restrict__ R,
                                                      int I, int s, const float* __restrict__ Lp,
                                                      const float* __restrict__ Dinv, float* __restrict__ W,
                                                      int* status) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ __align__(8) uint64_t bars[3];
  const ChSolveLayout Ly = ch_solve_layout(I, s);
  float* Ls = (float*)(sm + Ly.l);
  float* Rs = (float*)(sm + Ly.rs);
  float* Ds = (float*)(sm + Ly.ds);
  float* bv = (float*)(sm + Ly.b);
  float* qs = (float*)(sm + Ly.qs);
  float* red = (float*)(sm + Ly.red);
  const int NC = Ly.NC;
  const int g = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int rows[2] = {0, 0};
  const int nrw = ch_rows(g, I, rows);
  const int np = ch_npan(s), sp = 32 * np, tot = ch_pack(s);
  const float* Lg = Lp + (size_t)g * tot;
  const bool bulkL = ((uintptr_t)Lg % 16) == 0;
  const bool bulkR = ((uintptr_t)R % 16) == 0 && (s % 4) == 0;
  if (tid == 0) {
    for (int i = 0; i < 3; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(ch_su32(&bars[i])));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
  }
  __syncthreads();
  if (tid == 0 && bulkL) ch_bulk(Ls, Lg, (unsigned)tot * 4u, &bars[0]);
  if (!bulkL)
    for (int e = tid; e < tot; e += CH_NT) Ls[e] = Lg[e];
  for (int e = tid; e < np * 1024; e += CH_NT) {
    const int p = e >> 10, w = e & 1023;
    Ds[p * 1056 + (w >> 5) * 33 + (w & 31)] = Dinv[(size_t)g * np * 1024 + e];
  }
  // b = (Q^T R)[rows]: thread (kq, j) sums rows m = kq, kq + KS, ... of each chunk
  const int KS = s >= CH_NT ? 1 : CH_NT / s;
  const int j = tid % s, kq = tid / s;
  const bool act = kq < KS && j < s;
  float acc0 = 0.0f, acc1 = 0.0f;
  const int nch = (I + NC - 1) / NC;
  unsigned ph[2] = {0u, 0u};
  bool ok = true;
  if (bulkR && tid == 0) ch_bulk(Rs, R, (unsigned)(min(NC, I) * s * 4), &bars[1]);
  for (int c = 0; c < nch; ++c) {
    const int n0 = c * NC, nc = min(NC, I - n0);
    float* buf = Rs + (size_t)(c & 1) * NC * s;
    float* qb = qs + (c & 1) * 2 * NC;
    if (bulkR && tid == 0 && c + 1 < nch) {
      const int n1 = n0 + NC, nc1 = min(NC, I - n1);
      ch_bulk(Rs + (size_t)((c + 1) & 1) * NC * s, R + (size_t)n1 * s, (unsigned)(nc1 * s * 4), &bars[1 + ((c + 1) & 1)]);
    }
    for (int e = tid; e < nrw * nc; e += CH_NT) {
      const int t = e / nc, m = e - t * nc;
      qb[t * NC + m] = QT[(size_t)rows[t] * I + n0 + m];
    }
    if (bulkR) {
      ok = ch_wait(&bars[1 + (c & 1)], ph[c & 1]) && ok;
      ph[c & 1] ^= 1u;
    } else {
      for (int e = tid; e < nc * s; e += CH_NT) buf[e] = R[(size_t)n0 * s + e];
    }
    __syncthreads();
    if (act) {
      if (nrw == 2) {
        for (int m = kq; m < nc; m += KS) {
          const float x = buf[m * s + j];
          acc0 = fmaf(qb[m], x, acc0);
          acc1 = fmaf(qb[NC + m], x, acc1);
        }
      } else {
        for (int m = kq; m < nc; m += KS) acc0 = fmaf(qb[m], buf[m * s + j], acc0);
      }
    }
    __syncthreads();
  }
  // combine the column groups' partial sums in group order (staging buffers are free now)
  if (act) {
    Rs[(kq * 2 + 0) * s + j] = acc0;
    Rs[(kq * 2 + 1) * s + j] = acc1;
  }
  __syncthreads();
  for (int e = tid; e < 2 * sp; e += CH_NT) {
    const int t = e / sp, jj = e - t * sp;
    float v = 0.0f;
    if (jj < s && t < nrw)
      for (int q = 0; q < KS; ++q) v += Rs[(q * 2 + t) * s + jj];
    bv[e] = v;
  }
  if (bulkL) ok = ch_wait(&bars[0], 0) && ok;
  if (!ok) atomicCAS(status, FCTN_OK, FCTN_E_TIMEOUT);
  __syncthreads();
  // L z = b
  for (int p = 0; p < np; ++p) {
    const int nr = sp - 32 * p;
    const float* Lq = Ls + ch_poff(p, sp);
    const float* D = Ds + p * 1056;
    if (warp == 0) {
      float z[2];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        float a = 0.0f;
        if (t < nrw)
#pragma unroll 8
          for (int k = 0; k < 32; ++k) a = fmaf(D[lane * 33 + k], bv[t * sp + 32 * p + k], a);
        z[t] = a;
      }
      __syncwarp();
#pragma unroll
      for (int t = 0; t < 2; ++t)
        if (t < nrw) bv[t * sp + 32 * p + lane] = z[t];
    }
    __syncthreads();
    for (int i = tid; i < nr - 32; i += CH_NT) {
      const int rl = 32 + i;
      float a0 = 0.0f, a1 = 0.0f;
#pragma unroll 8
      for (int k = 0; k < 32; ++k) {
        const float l = Lq[k * nr + rl];
        a0 = fmaf(l, bv[32 * p + k], a0);
        a1 = fmaf(l, bv[sp + 32 * p + k], a1);
      }
      bv[32 * p + rl] -= a0;
      bv[sp + 32 * p + rl] -= a1;
    }
    __syncthreads();
  }
  // L^T w = z
  for (int p = np - 1; p >= 0; --p) {
    const int nr = sp - 32 * p;
    const float* Lq = Ls + ch_poff(p, sp);
    const float* D = Ds + p * 1056;
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const int c = warp * 4 + cc;
      float a0 = 0.0f, a1 = 0.0f;
      for (int rl = 32 + lane; rl < nr; rl += 32) {
        const float l = Lq[c * nr + rl];
        a0 = fmaf(l, bv[32 * p + rl], a0);
        a1 = fmaf(l, bv[sp + 32 * p + rl], a1);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(CH_FULL, a0, o);
        a1 += __shfl_xor_sync(CH_FULL, a1, o);
      }
      if (lane == 0) {
        red[c] = a0;
        red[32 + c] = a1;
      }
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        if (t >= nrw) break;
        const float y = bv[t * sp + 32 * p + lane] - red[t * 32 + lane];
        float a = 0.0f;
#pragma unroll
        for (int k = 0; k < 32; ++k) a = fmaf(D[k * 33 + lane], __shfl_sync(CH_FULL, y, k), a);
        bv[t * sp + 32 * p + lane] = a;
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < nrw * s; e += CH_NT) {
    const int t = e / s, jj = e - t * s;
    W[(size_t)rows[t] * s + jj] = bv[t * sp + jj];
  }
}

}  // namespace

int chol_groups(int I) { return I / 2 + 1; }
bool chol_supported(int s) { return s >= 1 && s <= CH_MAXS; }
size_t chol_factor_floats(int I, int s) { return (size_t)chol_groups(I) * ch_pack(s); }
size_t chol_dinv_floats(int I, int s) { return (size_t)chol_groups(I) * ch_npan(s) * 1024; }

void launch_chol_factor(const float* G, int I, int s, double lam, double c0, double c1, double rho, float* L,
                        float* Dinv, int* status, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_chol_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  const size_t bytes = (size_t)ch_pack(s) * 4;
  k_chol_factor<<<chol_groups(I), CH_NT, bytes, st>>>(G, s, I, lam, c0, c1, rho, L, Dinv, status);
}

void launch_chol_solve(const float* QT, const float* R, int I, int s, const float* L, const float* Dinv, float* W,
                       int* status, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_chol_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    attr = true;
  }
  const ChSolveLayout Ly = ch_solve_layout(I, s);
  k_chol_solve<<<chol_groups(I), CH_NT, Ly.total, st>>>(QT, R, I, s, L, Dinv, W, status);
}
