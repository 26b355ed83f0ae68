// Merged tensor formed on chip, fused into its two consumers (CUDA-core path).
//
// Every merged tensor the sweep needs is the contraction of two operands,
// M_k[sigma, j] = sum_kappa L[row_L(j), lo(sigma) + lk(kappa)] * R[row_R(j), ro(sigma) + rk(kappa)]
// (Property 1; N = 3: L = A_a, R = A_b; N = 4 with reuse: L = A_b, R = the
// cached pair intermediate T_cd of Algorithm 2; N = 2: R is the constant 1).
// A chunk of columns j is formed into shared memory and consumed at once:
//   gram_fused:    D = M_k [M_k ; X_(k)]^T partials (Gram and right-hand side
//                  of Eq. 5), optionally writing M_k out (the merged tensor
//                  of the factor updated last, reused by the X update).
//   xupdate_fused: F = A_k(k) M_k and the masked proximal update of Eq. 10.
#include "fctn_internal.cuh"
#include <algorithm>

#include "fctn_tile.cuh"

namespace {

constexpr int NT = 256;

// Leading dimension of the formed tile: all 64-row output tiles, plus 4
// (a multiple of 4, so rows start 16-byte aligned).
__host__ __device__ __forceinline__ int gram_ldm(const GramPlan& g) { return g.tiles_r * 64 + 4; }

__device__ __forceinline__ int64_t xaddr(const ModeView& v, int64_t i, int64_t j) {
  uint32_t jj = (uint32_t)j, post = (uint32_t)v.post;
  uint32_t a = jj / post, b = jj - a * post;
  return ((int64_t)a * v.I + i) * v.post + b;
}

// Form Ms[jj * ldm + sigma] for jj in [0, nb) of columns starting at j0
// (nb <= 32; columns at or beyond Pk are zero).  The distinct L / R rows of
// the columns are staged once each (Ls, Rs), with the per-column slots and row
// offsets in lsl/rsl and cl/cr.  Tables lo, ro, lk, rk in shared memory.
template <typename T>
__device__ __forceinline__ void form_tile(const PairPlan& p, const T* __restrict__ L, const T* __restrict__ R,
                                          int64_t j0, int nb, int64_t Pk, T* Ls, T* Rs, int64_t* cl, int64_t* cr,
                                          int* lsl, int* rsl, int* cnt, const int* lo, const int* ro, const int* lk,
                                          const int* rk, int s, T* Ms, int ldm) {
  const int tid = threadIdx.x;
  if (tid < 32) fctn_tile::chunk_slots(p, j0, nb, Pk, lsl, rsl, cl, cr, cnt);
  __syncthreads();
  for (int e = tid; e < cnt[0] * p.Ljs; e += NT) {
    int q = e / p.Ljs, c = e - q * p.Ljs;
    Ls[e] = L[cl[q] + c];
  }
  for (int e = tid; e < cnt[1] * p.Rjs; e += NT) {
    int q = e / p.Rjs, c = e - q * p.Rjs;
    Rs[e] = R[cr[q] + c];
  }
  __syncthreads();
  for (int e = tid; e < nb * s; e += NT) {
    int jj = e / s, sg = e - jj * s;
    T acc = 0;
    if (j0 + jj < Pk) {
      const T* l = Ls + lsl[jj] * p.Ljs + lo[sg];
      const T* r = Rs + rsl[jj] * p.Rjs + ro[sg];
      for (int q = 0; q < p.K; ++q) acc = fma(l[lk[q]], r[rk[q]], acc);
    }
    Ms[jj * ldm + sg] = acc;
  }
  __syncthreads();
}

__device__ __forceinline__ void load4(const float* p, float* v) {
  float4 t = *(const float4*)p;
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void load4(const double* p, double* v) {
  double2 t0 = *(const double2*)p, t1 = *(const double2*)(p + 2);
  v[0] = t0.x; v[1] = t0.y; v[2] = t1.x; v[3] = t1.y;
}

// Asynchronous global -> shared copy of one element (zero-filled when !valid).
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(T) == 4) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0));
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 8 : 0));
  }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Gram + right-hand side partials with M_k formed on chip.  Two-stage
// pipeline over chunks of BK columns: the slabs of L and R rows and the X
// rows of chunk c+1 are copied asynchronously while chunk c is formed and
// consumed.
template <typename T>
__global__ void __launch_bounds__(NT) k_gram_fused(PairPlan p, const T* __restrict__ L, const T* __restrict__ R,
                                                   const T* __restrict__ X, T* __restrict__ part, GramPlan g, int BK,
                                                   T* __restrict__ Mout) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int s = (int)g.s;
  const int ldm = gram_ldm(g);  // rows of the formed tile, padded to the 64-row tiles (zero beyond s)
  int* lo = (int*)sm;
  int* ro = lo + s;
  int* lk = ro + s;
  int* rk = lk + p.K;
  int64_t* cl = (int64_t*)(((uintptr_t)(rk + p.K) + 15) & ~(uintptr_t)15);  // [2][BK]
  int64_t* cr = cl + 2 * BK;                                                  // [2][BK]
  T* Ms = (T*)(cr + 2 * BK);                    // BK x ldm, Ms[kk*ldm + sigma] (16-byte aligned)
  T* Xs = Ms + (size_t)BK * ldm;                // [2][BK * 64]
  T* Ls = Xs + (size_t)2 * BK * 64;             // [2][BK * Ljs]
  T* Rs = Ls + (size_t)2 * BK * p.Ljs;          // [2][BK * Rjs]
  __shared__ int lsl[2][32], rsl[2][32], cnt[2][2];  // per stage: row slots of the columns, distinct-row counts
  __shared__ int64_t xcol[2][32];                    // per stage: offset of X_(k)[0, j] (-1 past the chunk)
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  for (int e = tid; e < s; e += NT) {
    lo[e] = p.tab[e];
    ro[e] = p.tab[s + e];
  }
  for (int e = tid; e < p.K; e += NT) {
    lk[e] = p.tab[2 * s + e];
    rk[e] = p.tab[2 * s + p.K + e];
  }
  const int64_t r0 = (int64_t)blockIdx.y * 64, c0 = (int64_t)blockIdx.x * 64;
  const int64_t kb = (int64_t)blockIdx.z * g.kchunk;
  const int64_t ke = min(kb + g.kchunk, g.Pk);
  const bool write_m = Mout != nullptr && blockIdx.x == 0 && blockIdx.y == 0;
  const bool has_x = c0 + 64 > g.gcols;
  const int nchunk = (int)((ke - kb + BK - 1) / BK);
  // steps of (row, column) when a flat index advances by NT
  const int dqL = NT / p.Ljs, dcL = NT % p.Ljs, dqR = NT / p.Rjs, dcR = NT % p.Rjs;
  const int dqS = NT / s, dcS = NT % s;

  // decode the columns of chunk c into buffer b (then a barrier), and issue its copies
  auto issue = [&](int c, int b) {
    const int64_t k0 = kb + (int64_t)c * BK;
    if (tid < 32) {
      fctn_tile::chunk_slots(p, k0, BK, ke, lsl[b], rsl[b], cl + b * BK, cr + b * BK, cnt[b]);
      if (has_x && g.xv.post != 1 && tid < BK) {  // j = a * post + b'  ->  a * I * post + b'
        const int64_t j = k0 + tid;
        const uint32_t post = (uint32_t)g.xv.post, jj = (uint32_t)j;
        const uint32_t a = jj / post;
        xcol[b][tid] = j < ke ? ((int64_t)a * g.xv.I) * g.xv.post + (jj - a * post) : -1;
      }
    }
    __syncthreads();
    T* ls = Ls + (size_t)b * BK * p.Ljs;
    T* rs = Rs + (size_t)b * BK * p.Rjs;
    {
      int q = tid / p.Ljs, c_ = tid - q * p.Ljs;
      for (int e = tid; e < cnt[b][0] * p.Ljs; e += NT) {
        cp_async_elem(ls + e, L + cl[b * BK + q] + c_, true);
        q += dqL;
        c_ += dcL;
        if (c_ >= p.Ljs) { c_ -= p.Ljs; ++q; }
      }
    }
    {
      int q = tid / p.Rjs, c_ = tid - q * p.Rjs;
      for (int e = tid; e < cnt[b][1] * p.Rjs; e += NT) {
        cp_async_elem(rs + e, R + cr[b * BK + q] + c_, true);
        q += dqR;
        c_ += dcR;
        if (c_ >= p.Rjs) { c_ -= p.Rjs; ++q; }
      }
    }
    if (has_x) {
      T* xs = Xs + (size_t)b * BK * 64;
      if (g.xv.post == 1) {
        for (int e = tid; e < 64 * BK; e += NT) {
          int cc = e % 64, kk = e / 64;
          int64_t col = c0 + cc, j = k0 + kk;
          bool v = col >= g.gcols && col < g.ncols && j < ke;
          cp_async_elem(xs + kk * 64 + cc, v ? X + j * g.xv.I + (col - g.gcols) : X, v);
        }
      } else {
        // a warp takes 32 consecutive rows of one column: conflict-free in
        // shared memory; element (cc, kk) at xcol[kk] + row * post
        const int cc = tid % 64;
        const int64_t col = c0 + cc;
        const bool vc = col >= g.gcols && col < g.ncols;
        const int64_t roff = (col - g.gcols) * g.xv.post;
        for (int kk = tid / 64; kk < BK; kk += NT / 64) {
          const int64_t xc = xcol[b][kk];
          const bool v = vc && xc >= 0;
          cp_async_elem(xs + kk * 64 + cc, v ? X + xc + roff : X, v);
        }
      }
    }
    cp_async_commit();
  };

  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0;
  for (int e = tid; e < BK * ldm; e += NT) Ms[e] = 0;  // rows >= s stay zero
  __syncthreads();
  if (nchunk > 0) issue(0, 0);
  for (int c = 0; c < nchunk; ++c) {
    const int b = c & 1;
    const int64_t k0 = kb + (int64_t)c * BK;
    const int nb = (int)min((int64_t)BK, ke - k0);
    if (c + 1 < nchunk) {
      issue(c + 1, b ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    // form the M_k tile of this chunk
    {
      const T* ls = Ls + (size_t)b * BK * p.Ljs;
      const T* rs = Rs + (size_t)b * BK * p.Rjs;
      int jj = tid / s, sg = tid - jj * s;
      for (int e = tid; e < BK * s; e += NT) {
        T a = 0;
        if (k0 + jj < ke) {
          const T* l = ls + lsl[b][jj] * p.Ljs + lo[sg];
          const T* r = rs + rsl[b][jj] * p.Rjs + ro[sg];
          for (int q = 0; q < p.K; ++q) a = fma(l[lk[q]], r[rk[q]], a);
        }
        Ms[jj * ldm + sg] = a;
        jj += dqS;
        sg += dcS;
        if (sg >= s) { sg -= s; ++jj; }
      }
    }
    __syncthreads();
    if (write_m) {
      for (int e = tid; e < s * nb; e += NT) {
        int sg = e / nb, jj = e - sg * nb;
        Mout[(int64_t)sg * g.Pk + k0 + jj] = Ms[jj * ldm + sg];
      }
    }
    const T* xs = Xs + (size_t)b * BK * 64;
    const T* ap = Ms + r0 + ty * 4;  // rows >= s are zero in Ms
    if (c0 + 64 <= g.gcols || c0 >= g.gcols) {
      // the 64 columns of this tile are all Gram columns (from Ms) or all X rows (from xs)
      const T* bp = (c0 + 64 <= g.gcols) ? Ms + c0 + tx * 4 : xs + tx * 4;
      const int bstr = (c0 + 64 <= g.gcols) ? ldm : 64;
#pragma unroll 4
      for (int kk = 0; kk < nb; ++kk) {
        T av[4], bv[4];
        load4(ap + kk * ldm, av);
        load4(bp + kk * bstr, bv);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b2 = 0; b2 < 4; ++b2) acc[a][b2] = fma(av[a], bv[b2], acc[a][b2]);
      }
    } else {
      for (int kk = 0; kk < nb; ++kk) {
        T av[4], bv[4];
        load4(ap + kk * ldm, av);
#pragma unroll
        for (int b2 = 0; b2 < 4; ++b2) {
          int64_t col = c0 + tx * 4 + b2;
          bv[b2] = col < g.gcols ? Ms[kk * ldm + col] : xs[kk * 64 + tx * 4 + b2];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b2 = 0; b2 < 4; ++b2) acc[a][b2] = fma(av[a], bv[b2], acc[a][b2]);
      }
    }
    __syncthreads();
  }
  T* P = part + (int64_t)blockIdx.z * g.s * g.ncols;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    int64_t row = r0 + ty * 4 + a;
    if (row >= g.s) continue;
#pragma unroll
    for (int b2 = 0; b2 < 4; ++b2) {
      int64_t col = c0 + tx * 4 + b2;
      if (col < g.ncols) P[row * g.ncols + col] = acc[a][b2];
    }
  }
}

// F = A_(k) M_k over a 64 (rows i) x 64 (columns j) tile, M_k formed on chip
// in column sub-chunks of CB, then Eq. 10 and the stop-test partial sums.
template <typename T>
__global__ void __launch_bounds__(NT) k_xupdate_fused(PairPlan p, const T* __restrict__ L, const T* __restrict__ R,
                                                      const T* __restrict__ Ak, T* __restrict__ X,
                                                      const uint32_t* __restrict__ bits, double rho, GramPlan g,
                                                      int CB, double* __restrict__ red) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int s = (int)g.s;
  const int ldm = s + 1;
  int* lo = (int*)sm;
  int* ro = lo + s;
  int* lk = ro + s;
  int* rk = lk + p.K;
  int64_t* cl = (int64_t*)(((uintptr_t)(rk + p.K) + 15) & ~(uintptr_t)15);
  int64_t* cr = cl + CB;
  T* Ls = (T*)(cr + CB);
  T* Rs = Ls + (size_t)CB * p.Ljs;
  T* Ms = Rs + (size_t)CB * p.Rjs;     // 64 x ldm (column jj, row sigma)
  T* As = Ms + (size_t)64 * ldm;       // 64 x s  (row i, sigma)
  __shared__ double sred[3][NT / 32];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  for (int e = tid; e < s; e += NT) {
    lo[e] = p.tab[e];
    ro[e] = p.tab[s + e];
  }
  for (int e = tid; e < p.K; e += NT) {
    lk[e] = p.tab[2 * s + e];
    rk[e] = p.tab[2 * s + p.K + e];
  }
  const int64_t i0 = (int64_t)blockIdx.y * 64, j0 = (int64_t)blockIdx.x * 64;
  for (int e = tid; e < 64 * s; e += NT) {
    int r = e / s, sg = e - r * s;
    As[e] = (i0 + r < g.I) ? Ak[(i0 + r) * g.s + sg] : (T)0;
  }
  __syncthreads();
  __shared__ int lsl[32], rsl[32], cnt[2];
  for (int c = 0; c < 64; c += CB)
    form_tile<T>(p, L, R, j0 + c, CB, g.Pk, Ls, Rs, cl, cr, lsl, rsl, cnt, lo, ro, lk, rk, s, Ms + (size_t)c * ldm,
                 ldm);
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0;
  for (int sg = 0; sg < s; ++sg) {
    T av[4], bv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) av[a] = As[(ty * 4 + a) * s + sg];
#pragma unroll
    for (int b = 0; b < 4; ++b) bv[b] = Ms[(tx * 4 + b) * ldm + sg];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
  }
  T d2 = 0, x2 = 0, r2 = 0;
  __syncthreads();  // Ms and As are consumed: the F tile reuses Ms
  fctn_tile::xupdate_tile<T>(acc, Ms, i0, j0, g, X, bits, rho, d2, x2, r2);
  double v[3] = {(double)d2, (double)x2, (double)r2};
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    double t = v[q];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((tid & 31) == 0) sred[q][tid >> 5] = t;
  }
  __syncthreads();
  if (tid < 3) {
    double t = 0.0;
    for (int w = 0; w < NT / 32; ++w) t += sred[tid][w];
    int64_t blk = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    red[blk * 3 + tid] = t;
  }
}

size_t head_bytes(const PairPlan& p, int s, int nb) {
  size_t b = (size_t)(2 * s + 2 * p.K) * 4;
  b = (b + 15) & ~(size_t)15;
  return b + 2 * (size_t)nb * 8;
}

}  // namespace

size_t gram_fused_smem(const PairPlan& p, int s, int bk, int elem) {
  // tables, 2 x column offsets, formed tile, 2 x (X rows, L slab, R slab)
  const int ldm = ((s + 63) / 64) * 64 + 4;
  return head_bytes(p, s, 2 * bk) + (size_t)bk * (2 * (p.Ljs + p.Rjs + 64) + ldm) * elem;
}

int gram_fused_bk(const PairPlan& p, int s, int elem) {
  for (int bk = 32; bk >= 4; bk /= 2)
    if (gram_fused_smem(p, s, bk, elem) <= 110 * 1024) return bk;
  return 4;
}

int xupdate_fused_cb(const PairPlan& p, int s, int elem) {
  for (int cb = 32; cb >= 1; cb /= 2) {
    size_t b = head_bytes(p, s, cb) + ((size_t)cb * (p.Ljs + p.Rjs) + 64 * std::max((size_t)(2 * s + 1), (size_t)65)) * elem;
    if (b <= 200 * 1024) return cb;
  }
  return 1;
}

size_t xupdate_fused_smem(const PairPlan& p, int s, int cb, int elem) {
  // Ms (64 x (s+1)) and As (64 x s); afterwards the F tile (64 x 65) in their place
  return head_bytes(p, s, cb) + ((size_t)cb * (p.Ljs + p.Rjs) + 64 * std::max((size_t)(2 * s + 1), (size_t)65)) * elem;
}

template <typename T>
static void gram_fused(const PairPlan& p, const T* L, const T* R, const T* X, T* part, const GramPlan& g, T* Mout,
                       cudaStream_t st) {
  const int bk = gram_fused_bk(p, (int)g.s, sizeof(T));
  const size_t sb = gram_fused_smem(p, (int)g.s, bk, sizeof(T));
  cudaFuncSetAttribute(k_gram_fused<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  dim3 grid(g.tiles_c, g.tiles_r, g.ksplit);
  k_gram_fused<T><<<grid, NT, sb, st>>>(p, L, R, X, part, g, bk, Mout);
}

template <typename T>
static void xupdate_fused(const PairPlan& p, const T* L, const T* R, const T* Ak, T* X, const uint32_t* bits,
                          double rho, const GramPlan& g, double* red, cudaStream_t st) {
  const int cb = xupdate_fused_cb(p, (int)g.s, sizeof(T));
  const size_t sb = xupdate_fused_smem(p, (int)g.s, cb, sizeof(T));
  cudaFuncSetAttribute(k_xupdate_fused<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  dim3 grid((unsigned)((g.Pk + 63) / 64), (unsigned)((g.I + 63) / 64));
  k_xupdate_fused<T><<<grid, NT, sb, st>>>(p, L, R, Ak, X, bits, rho, g, cb, red);
}

void launch_gram_fused_f32(const PairPlan& p, const float* L, const float* R, const float* X, float* part,
                           const GramPlan& g, float* Mout, cudaStream_t st) {
  gram_fused<float>(p, L, R, X, part, g, Mout, st);
}
void launch_gram_fused_f64(const PairPlan& p, const double* L, const double* R, const double* X, double* part,
                           const GramPlan& g, double* Mout, cudaStream_t st) {
  gram_fused<double>(p, L, R, X, part, g, Mout, st);
}
void launch_xupdate_fused_f32(const PairPlan& p, const float* L, const float* R, const float* Ak, float* X,
                              const uint32_t* bits, double rho, const GramPlan& g, double* red, cudaStream_t st) {
  xupdate_fused<float>(p, L, R, Ak, X, bits, rho, g, red, st);
}
void launch_xupdate_fused_f64(const PairPlan& p, const double* L, const double* R, const double* Ak, double* X,
                              const uint32_t* bits, double rho, const GramPlan& g, double* red, cudaStream_t st) {
  xupdate_fused<double>(p, L, R, Ak, X, bits, rho, g, red, st);
}
