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
// the trailing update in 4 x 8 register tiles of 32 x 32 blocks, with the
// next diagonal block factored beside it); writes L and the inverses of its
// diagonal blocks.  A pivot that is not positive means
// that G + c_j I is not positive definite (some T_ij of Eq. 8 <= 0): status
// FCTN_E_SINGULAR, as for the eigen route.
// The solve around the factors (one refinement step shown):
//   R~ = Q^T Y (k_bgemm), W = rows of R~ through L L^T (k_chol_subst),
//   A = Q W (k_bgemm, FP64 master with its double-float split),
//   R = Y - lam L A - rho A - A G (k_resid_df), then R~ = Q^T R, the
//   substitution again and A += Q W.
#include <cuda.h>

#include <cstring>

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

// Bounded wait: tries of up to 256 ns each (the thread sleeps until the
// phase completes or the time runs out), about 1 s in all.
__device__ __forceinline__ bool ch_wait(uint64_t* bar, unsigned phase) {
  for (long long it = 0; it < (1ll << 22); ++it) {
    unsigned r;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(r)
        : "r"(ch_su32(bar)), "r"(phase), "r"(256u));
    if (r) return true;
  }
  return false;
}

__device__ __forceinline__ void ch_expect(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(ch_su32(bar)), "r"(bytes));
}
// Bulk copy that completes on `bar` (whose expected bytes were set beforehand).
__device__ __forceinline__ void ch_copy(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(ch_su32(dst)),
      "l"(src), "r"(bytes), "r"(ch_su32(bar))
      : "memory");
}
__device__ __forceinline__ void ch_bar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(ch_su32(bar)));
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
}

// Diagonal-block inverses are stored with a row stride of 33 floats (the
// layout the solve kernel reads without bank conflicts in both orientations).
constexpr int CH_DSTR = 33, CH_DBLK = 32 * CH_DSTR;

// Tensor maps of G for the panels: map q loads rows 32 q .. 32 q + 31 of G
// (columns of panel q) and columns 32 q .. sp - 1 (its rows) as one dense
// 32 x (sp - 32 q) box, which is the panel's column-major layout; outside G
// the box reads zero.
struct ChMaps {
  CUtensorMap m[CH_MAXS / 32];
  int on;
};


// Diagonal block of panel p, by one warp: lane r holds row r; column j is
// scaled by 1 / sqrt(pivot), then the rank-1 update of the columns right of
// it; rdiag[j] = 1 / l_jj.  Not inlined: it keeps its registers apart from
// the trailing update it runs beside.
__device__ __noinline__ void ch_factor_diag(float* __restrict__ P, int p, int sp, int s, float shift,
                                            float* __restrict__ rdiag, int* bad) {
  const int lane = threadIdx.x & 31;
  const int nr = sp - 32 * p;
  float* Pp = P + ch_poff(p, sp);
  float d[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    d[c] = Pp[c * nr + lane];
    if (c == lane && 32 * p + c < s) d[c] += shift;  // G + c I
  }
  bool ok = true;
  // Column j's pivot and 1 / sqrt(pivot) are formed as soon as column j - 1
  // has updated it, ahead of the rest of column j - 1's update, so that the
  // chain from pivot to pivot is not queued behind those shuffles.
  auto pivot = [&](float v, float& piv, float& rs) {
    piv = v;
    if (!(piv > 0.0f)) {
      ok = false;
      piv = 1.0f;
    }
    rs = rsqrtf(piv);
  };
  float piv, rs;
  pivot(__shfl_sync(CH_FULL, d[0], 0), piv, rs);
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    d[j] = (lane == j) ? piv * rs : d[j] * rs;
    if (lane == 0) rdiag[j] = rs;
    float npiv = 1.0f, nrs = 1.0f;
    if (j + 1 < 32) {
      d[j + 1] = fmaf(-d[j], __shfl_sync(CH_FULL, d[j], j + 1), d[j + 1]);
      pivot(__shfl_sync(CH_FULL, d[j + 1], j + 1), npiv, nrs);
    }
#pragma unroll
    for (int c = j + 2; c < 32; ++c) d[c] = fmaf(-d[j], __shfl_sync(CH_FULL, d[j], c), d[c]);
    piv = npiv;
    rs = nrs;
  }
#pragma unroll
  for (int c = 0; c < 32; ++c)
    if (c <= lane) Pp[c * nr + lane] = d[c];
  if (!ok && lane == 0) *bad = 1;
}

// Rows 8 w .. 8 w + 7 of the next diagonal block (block (p + 1, p + 1), all
// 32 columns) minus their trailing update from panel p: the four warps
// w = 0..3, one per SM sub-partition, update that block together before
// warp 0 factors it.
__device__ __forceinline__ void ch_syrk_diag_rows(float* __restrict__ P, int p, int sp, int w) {
  const int lane = threadIdx.x & 31;
  const int nr = sp - 32 * p, nq = nr - 32;
  const float* Pp = P + ch_poff(p, sp);
  const int r = 8 * w + (lane & 7), cb = (lane >> 3) * 8;
  const float* Ap = Pp + 32 + r;
  const float* Bp = Pp + 32 + cb;
  float acc[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) acc[j] = 0.0f;
#pragma unroll 8
  for (int k = 0; k < 32; ++k) {
    const float a = Ap[k * nr];
    const float4 b0 = *reinterpret_cast<const float4*>(Bp + k * nr);
    const float4 b1 = *reinterpret_cast<const float4*>(Bp + k * nr + 4);
    const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = fmaf(a, bv[j], acc[j]);
  }
  float* Cq = P + ch_poff(p + 1, sp) + r;
#pragma unroll
  for (int j = 0; j < 8; ++j) Cq[(cb + j) * nq] -= acc[j];
}

// Trailing-update tile ti of panel p (one warp): block (rb, q), p < q <= rb <
// np, of panel q minus L[rb rows, panel p] L[q rows, panel p]^T.
__device__ __forceinline__ void ch_syrk_tile(float* __restrict__ P, int p, int sp, int np, int ti) {
  const int lane = threadIdx.x & 31;
  const int nr = sp - 32 * p;
  const float* Pp = P + ch_poff(p, sp);
  const int r0 = (lane & 7) * 4, cb = (lane >> 3) * 8;
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

__global__ void __launch_bounds__(CH_NT) k_chol_factor(const float* __restrict__ G, int s, int I, double lam,
                                                       double c0, double c1, double rho, float* __restrict__ Lout,
                                                       float* __restrict__ Dout, int* status,
                                                       const __grid_constant__ ChMaps maps) {
  pdl_prologue();
  // TMA boxes need a 128-byte aligned destination: checked below, the
  // scalar path is taken otherwise
  extern __shared__ __align__(128) float P[];
  __shared__ float rdiag[32];
  __shared__ int bad;
  const int g = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int np = ch_npan(s), sp = 32 * np;
  // the shift c_g = lam mu_g + rho (Eq. 6), computed in FP64 by one thread
  // (FP64 is scarce on this GPU) and read by all after the loads
  __shared__ float shift_s;
  // G into the panels.  G is symmetric, so column col of panel q (rows
  // 32 q .. s - 1) is the row segment G[col][32 q .. s).  With tensor maps
  // (s % 4 == 0): one TMA box per panel (zero outside G), then the identity
  // on the padded diagonal; otherwise scalar loads.  The shift c is added to
  // the pivots in step 1.
  __shared__ __align__(8) uint64_t gbar;
  if (tid == 0) bad = 0;
  if (tid == 32) shift_s = (float)(lam * (c0 + 2.0 * c1 * cospi(2.0 * (double)g / (double)I)) + rho);
  if (maps.on && (ch_su32(P) & 127u) == 0) {
    if (tid == 0) {
      ch_bar_init(&gbar);
      ch_expect(&gbar, (unsigned)ch_pack(s) * 4u);
      for (int q = 0; q < np; ++q)
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
            "[%4];\n" ::"r"(ch_su32(P + ch_poff(q, sp))),
            "l"((uint64_t)&maps.m[q]), "r"(32 * q), "r"(32 * q), "r"(ch_su32(&gbar))
            : "memory");
    }
    __syncthreads();
    if (!ch_wait(&gbar, 0) && tid == 0) atomicCAS(status, FCTN_OK, FCTN_E_TIMEOUT);
    __syncthreads();
    if (tid < sp - s) {  // padded columns: identity on the diagonal
      const int col = s + tid, q = col >> 5;
      P[ch_poff(q, sp) + (col & 31) * (sp - 32 * q) + (col - 32 * q)] = 1.0f;
    }
  } else {
    for (int col = warp; col < sp; col += CH_NT / 32) {
      const int q = col >> 5, nr = sp - 32 * q;
      float* dst = P + ch_poff(q, sp) + (col & 31) * nr - 32 * q;  // dst[r] = element (r, col)
      for (int r = 32 * q + lane; r < sp; r += 32)
        dst[r] = (col < s && r < s) ? G[(size_t)col * s + r] : (r == col ? 1.0f : 0.0f);
    }
  }
  __syncthreads();
  const float shift = shift_s;
  if (warp == 0) ch_factor_diag(P, 0, sp, s, shift, rdiag, &bad);
  __syncthreads();
  for (int p = 0; p < np; ++p) {
    const int nr = sp - 32 * p;
    float* Pp = P + ch_poff(p, sp);
    // 2. rows below the block: x L_pp^T = a, one row per thread of warps
    //    1..7; warp 0 meanwhile forms the block's inverse for the solve
    if (warp == 0) {
      float y[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) y[k] = (k == lane) ? 1.0f : 0.0f;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        y[j] *= rdiag[j];
#pragma unroll
        for (int kb = (j + 1) / 4; kb < 8; ++kb) {  // column j of L_pp below the diagonal, 16 bytes at a time
          const float4 l = *reinterpret_cast<const float4*>(Pp + j * nr + 4 * kb);
          const float lv[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
          for (int i = 0; i < 4; ++i)
            if (4 * kb + i > j) y[4 * kb + i] = fmaf(-lv[i], y[j], y[4 * kb + i]);
        }
      }
      float* Dg = Dout + ((size_t)g * np + p) * CH_DBLK;
#pragma unroll
      for (int k = 0; k < 32; ++k) Dg[k * CH_DSTR + lane] = y[k];
      Dg[lane * CH_DSTR + 32] = 0.0f;
    }
    for (int t = tid - 32; t >= 0 && t < nr - 32; t += CH_NT - 32) {
      const int rl = 32 + t;
      float x[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) x[c] = Pp[c * nr + rl];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        x[j] *= rdiag[j];
#pragma unroll
        for (int kb = (j + 1) / 4; kb < 8; ++kb) {
          const float4 l = *reinterpret_cast<const float4*>(Pp + j * nr + 4 * kb);
          const float lv[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
          for (int i = 0; i < 4; ++i)
            if (4 * kb + i > j) x[4 * kb + i] = fmaf(-x[j], lv[i], x[4 * kb + i]);
        }
      }
#pragma unroll
      for (int c = 0; c < 32; ++c) Pp[c * nr + rl] = x[c];
    }
    __syncthreads();
    // panel p is final: to global memory (the stores overlap the update below)
    {
      float* Lg = Lout + (size_t)g * ch_pack(s) + ch_poff(p, sp);
      for (int e = tid * 4; e < 32 * nr; e += CH_NT * 4)
        *reinterpret_cast<float4*>(Lg + e) = *reinterpret_cast<const float4*>(Pp + e);
    }
    // 3. trailing update with look-ahead: warps 0-3 (one per SM
    //    sub-partition) update the next diagonal block (tile 0), 8 rows
    //    each, and warp 0 factors it as soon as the four are done (named
    //    barrier 1: warps 1-3 arrive without waiting); warps 1-7 update the
    //    remaining blocks
    const int nt = np - 1 - p, ntile = nt * (nt + 1) / 2;
    if (ntile > 0) {
      if (warp < 4) {
        ch_syrk_diag_rows(P, p, sp, warp);
        if (warp == 0) {
          asm volatile("bar.sync 1, 128;\n" ::: "memory");
          ch_factor_diag(P, p + 1, sp, s, shift, rdiag, &bad);
        } else {
          asm volatile("bar.arrive 1, 128;\n" ::: "memory");
        }
      }
      if (warp != 0)
        for (int ti = warp; ti < ntile; ti += CH_NT / 32 - 1) ch_syrk_tile(P, p, sp, np, ti);
    }
    __syncthreads();
  }
  if (tid == 0 && bad) atomicCAS(status, FCTN_OK, FCTN_E_SINGULAR);
}

// k_chol_subst: one CTA per group: L z = b and L^T w = z for the group's
// rows b of R~ = Q^T R, panel by panel: the diagonal block through its
// inverse (one warp), the rest of the panel by the other threads.  L and the
// block inverses arrive by bulk copies; w is written to the rows of W.
__host__ __device__ inline size_t ch_subst_bytes(int s) {
  const int np = ch_npan(s);
  return (size_t)ch_pack(s) * 4 + (size_t)np * CH_DBLK * 4 + 2 * 32 * (size_t)np * 4;
}

__global__ void __launch_bounds__(CH_NT) k_chol_subst(const float* __restrict__ Rt, int I, int s,
                                                      const float* __restrict__ Lp, const float* __restrict__ Dinv,
                                                      float* __restrict__ W, int* status) {
  pdl_prologue();
  extern __shared__ __align__(16) float smf[];
  __shared__ __align__(8) uint64_t bar;
  const int g = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int rows[2] = {0, 0};
  const int nrw = ch_rows(g, I, rows);
  const int np = ch_npan(s), sp = 32 * np, tot = ch_pack(s);
  float* Ls = smf;
  float* Ds = Ls + tot;
  float* bv = Ds + np * CH_DBLK;
  const float* Lg = Lp + (size_t)g * tot;
  const float* Dg = Dinv + (size_t)g * np * CH_DBLK;
  const bool bulk = ((uintptr_t)Lg % 16) == 0 && ((uintptr_t)Dg % 16) == 0;
  if (tid == 0 && bulk) {
    ch_bar_init(&bar);
    ch_expect(&bar, (unsigned)(tot + np * CH_DBLK) * 4u);
    ch_copy(Ls, Lg, (unsigned)tot * 4u, &bar);
    ch_copy(Ds, Dg, (unsigned)(np * CH_DBLK) * 4u, &bar);
  }
  if (!bulk) {
    for (int e = tid; e < tot; e += CH_NT) Ls[e] = Lg[e];
    for (int e = tid; e < np * CH_DBLK; e += CH_NT) Ds[e] = Dg[e];
  }
  for (int e = tid; e < 2 * sp; e += CH_NT) {
    const int t = e / sp, j = e - t * sp;
    bv[e] = (t < nrw && j < s) ? Rt[(size_t)rows[t] * s + j] : 0.0f;
  }
  __syncthreads();  // the barrier's initialisation is visible before anyone waits on it
  if (bulk && !ch_wait(&bar, 0) && tid == 0) atomicCAS(status, FCTN_OK, FCTN_E_TIMEOUT);
  __syncthreads();
  // L z = b
  for (int p = 0; p < np; ++p) {
    const int nr = sp - 32 * p;
    const float* Lq = Ls + ch_poff(p, sp);
    const float* D = Ds + p * CH_DBLK;
    if (warp == 0) {
      float z0 = 0.0f, z1 = 0.0f;
#pragma unroll 8
      for (int k = 0; k < 32; ++k) {
        const float d = D[lane * CH_DSTR + k];
        z0 = fmaf(d, bv[32 * p + k], z0);
        z1 = fmaf(d, bv[sp + 32 * p + k], z1);
      }
      __syncwarp();
      bv[32 * p + lane] = z0;
      bv[sp + 32 * p + lane] = z1;
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
  // L^T w = z, right-looking: w_p from the diagonal block's inverse, then
  // its contribution removed from every earlier z (one thread per column)
  for (int p = np - 1; p >= 0; --p) {
    const float* D = Ds + p * CH_DBLK;
    if (warp == 0) {
      const float y0 = bv[32 * p + lane], y1 = bv[sp + 32 * p + lane];
      float w0 = 0.0f, w1 = 0.0f;
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        const float d = D[k * CH_DSTR + lane];
        w0 = fmaf(d, __shfl_sync(CH_FULL, y0, k), w0);
        w1 = fmaf(d, __shfl_sync(CH_FULL, y1, k), w1);
      }
      bv[32 * p + lane] = w0;
      bv[sp + 32 * p + lane] = w1;
    }
    __syncthreads();
    for (int c = tid; c < 32 * p; c += CH_NT) {
      const int q = c >> 5, nrq = sp - 32 * q;
      const float* Lc = Ls + ch_poff(q, sp) + (c & 31) * nrq + 32 * (p - q);  // Lc[i] = L[32 p + i][c]
      float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
      for (int i4 = 0; i4 < 8; ++i4) {
        const float4 l = *reinterpret_cast<const float4*>(Lc + 4 * i4);
        const float lv[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          a0 = fmaf(lv[u], bv[32 * p + 4 * i4 + u], a0);
          a1 = fmaf(lv[u], bv[sp + 32 * p + 4 * i4 + u], a1);
        }
      }
      bv[c] -= a0;
      bv[sp + c] -= a1;
    }
    __syncthreads();
  }
  for (int e = tid; e < nrw * s; e += CH_NT) {
    const int t = e / s, j = e - t * s;
    W[(size_t)rows[t] * s + j] = bv[t * sp + j];
  }
}

// ---- products with the L_k basis and the residual of Eq. 5 -----------------
// C (M x N) = A (M x K) B (K x N), row-major FP32 operands, one 32 x 32 tile
// of C per CTA of 256 threads (thread (ty, tx) owns rows ty, ty + 16 and
// columns tx, tx + 16); K in chunks of 64 staged through shared memory, the
// next chunk's loads in flight while the current chunk is multiplied.
// Epilogues: BG_STORE out32 = C; BG_SET A64 = C; BG_ADD A64 += C; with
// BG_SET / BG_ADD also Ac = hi(A64) = float(A64) and Alo = float(A64 - hi),
// the double-float split that the residual kernel reads.
enum { BG_STORE = 0, BG_SET = 1, BG_ADD = 2 };
constexpr int BG_KC = 64;

template <int MODE>
__global__ void __launch_bounds__(256) k_bgemm(const float* __restrict__ A, const float* __restrict__ B, int M, int N,
                                               int K, float* __restrict__ out32, double* __restrict__ A64,
                                               float* __restrict__ Ac, float* __restrict__ Alo) {
  pdl_prologue();
  __shared__ float As[32][BG_KC + 1];
  __shared__ float Bs[BG_KC][33];
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int m0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
  float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  float ra[8], rb[8];
  auto load = [&](int k0) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = tid + u * 256;
      const int am = e >> 6, ak = e & 63;  // A: 32 rows x 64 k
      const int bk = e >> 5, bn = e & 31;  // B: 64 k x 32 columns
      ra[u] = (m0 + am < M && k0 + ak < K) ? A[(size_t)(m0 + am) * K + k0 + ak] : 0.0f;
      rb[u] = (k0 + bk < K && n0 + bn < N) ? B[(size_t)(k0 + bk) * N + n0 + bn] : 0.0f;
    }
  };
  load(0);
  for (int k0 = 0; k0 < K; k0 += BG_KC) {
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = tid + u * 256;
      As[e >> 6][e & 63] = ra[u];
      Bs[e >> 5][e & 31] = rb[u];
    }
    __syncthreads();
    if (k0 + BG_KC < K) load(k0 + BG_KC);
#pragma unroll 16
    for (int k = 0; k < BG_KC; ++k) {
      const float a0 = As[ty][k], a1 = As[ty + 16][k];
      const float b0 = Bs[k][tx], b1 = Bs[k][tx + 16];
      acc[0][0] = fmaf(a0, b0, acc[0][0]);
      acc[0][1] = fmaf(a0, b1, acc[0][1]);
      acc[1][0] = fmaf(a1, b0, acc[1][0]);
      acc[1][1] = fmaf(a1, b1, acc[1][1]);
    }
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int m = m0 + ty + 16 * a, n = n0 + tx + 16 * b;
      if (m >= M || n >= N) continue;
      const size_t o = (size_t)m * N + n;
      if (MODE == BG_STORE) {
        out32[o] = acc[a][b];
      } else {
        const double v = MODE == BG_SET ? (double)acc[a][b] : A64[o] + (double)acc[a][b];
        A64[o] = v;
        const float hi = (float)v;
        Ac[o] = hi;
        Alo[o] = (float)(v - (double)hi);
      }
    }
}

// R = Y - lam L A - rho A - A G (Eq. 5) on a 16 x 32 tile (rows i0.., columns
// j0..), stored as FP32: the right-hand side of the refinement solve.  A is
// the double-float pair (Ac, Alo) of the FP64 factor; the products A G are
// exact FP32 products (fma gives each rounding error) summed with
// Neumaier's compensation, so the sum carries about twice the FP32
// precision (FP64 arithmetic runs at 1/64 of the FP32 rate on this GPU);
// Y, the stencil of L and the final difference are FP64.
__device__ __forceinline__ void ch_acopy4(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(ch_su32(dst)), "l"(src) : "memory");
}

// The same product with all of K (<= BG_KS16) staged at once by 16-byte
// asynchronous copies (A rows and B rows of the tile are contiguous when
// K % 4 == 0 and N % 4 == 0), then multiplied from shared memory.
constexpr int BG_KS16 = 256;
constexpr int BG_AST = BG_KS16 + 4, BG_BST = 36;  // row strides (16-byte rows)
__host__ __device__ inline size_t bg16_smem_bytes() { return ((size_t)32 * BG_AST + (size_t)BG_KS16 * BG_BST) * 4; }

__device__ __forceinline__ void ch_acopy16(float* dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(ch_su32(dst)), "l"(src) : "memory");
}

template <int MODE>
__global__ void __launch_bounds__(256) k_bgemm16(const float* __restrict__ A, const float* __restrict__ B, int M,
                                                 int N, int K, float* __restrict__ out32, double* __restrict__ A64,
                                                 float* __restrict__ Ac, float* __restrict__ Alo) {
  pdl_prologue();
  extern __shared__ __align__(16) float b16[];
  float* As = b16;                  // [32][BG_AST]: As[m][k] = A[m0 + m][k]
  float* Bs = b16 + 32 * BG_AST;    // [K][BG_BST]:  Bs[k][n] = B[k][n0 + n]
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int m0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
  const int K4 = K / 4;
  for (int e = tid; e < 32 * K4; e += 256) {
    const int m = e / K4, k4 = e - m * K4;
    float* dst = As + m * BG_AST + 4 * k4;
    if (m0 + m < M)
      ch_acopy16(dst, A + (size_t)(m0 + m) * K + 4 * k4);
    else
      *reinterpret_cast<float4*>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  for (int e = tid; e < K * 8; e += 256) {
    const int k = e >> 3, n4 = e & 7;
    float* dst = Bs + k * BG_BST + 4 * n4;
    if (n0 + 4 * n4 + 3 < N)
      ch_acopy16(dst, B + (size_t)k * N + n0 + 4 * n4);
    else
      for (int u = 0; u < 4; ++u) dst[u] = n0 + 4 * n4 + u < N ? B[(size_t)k * N + n0 + 4 * n4 + u] : 0.0f;
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  const float* a0p = As + ty * BG_AST;
  const float* a1p = As + (ty + 16) * BG_AST;
#pragma unroll 8
  for (int k = 0; k < K; ++k) {
    const float a0 = a0p[k], a1 = a1p[k];
    const float b0 = Bs[k * BG_BST + tx], b1 = Bs[k * BG_BST + tx + 16];
    acc[0][0] = fmaf(a0, b0, acc[0][0]);
    acc[0][1] = fmaf(a0, b1, acc[0][1]);
    acc[1][0] = fmaf(a1, b0, acc[1][0]);
    acc[1][1] = fmaf(a1, b1, acc[1][1]);
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int m = m0 + ty + 16 * a, n = n0 + tx + 16 * b;
      if (m >= M || n >= N) continue;
      const size_t o = (size_t)m * N + n;
      if (MODE == BG_STORE) {
        out32[o] = acc[a][b];
      } else {
        const double v = MODE == BG_SET ? (double)acc[a][b] : A64[o] + (double)acc[a][b];
        A64[o] = v;
        const float hi = (float)v;
        Ac[o] = hi;
        Alo[o] = (float)(v - (double)hi);
      }
    }
}

// H = A^T A for A (I x s, row-major FP32): the factor Gram H_t = A_(t)^T A_(t)
// of the Gram chains.  One 32 x 32 tile of H per CTA for tiles (ta <= tb)
// only, each written to both triangles; K = I in chunks of 64 as in k_bgemm.
__global__ void __launch_bounds__(256) k_gram_at(const float* __restrict__ A, int I, int s, float* __restrict__ H) {
  pdl_prologue();
  __shared__ float As[BG_KC][33];
  __shared__ float Bs[BG_KC][33];
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int nt = (s + 31) / 32;
  int t = blockIdx.x, ta = 0;
  while (t >= nt - ta) {
    t -= nt - ta;
    ++ta;
  }
  const int a0 = 32 * ta, b0 = 32 * (ta + t);
  float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  float ra[8], rb[8];
  auto load = [&](int k0) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = tid + u * 256, k = e >> 5, c = e & 31;
      const bool kin = k0 + k < I;
      ra[u] = (kin && a0 + c < s) ? A[(size_t)(k0 + k) * s + a0 + c] : 0.0f;
      rb[u] = (kin && b0 + c < s) ? A[(size_t)(k0 + k) * s + b0 + c] : 0.0f;
    }
  };
  load(0);
  for (int k0 = 0; k0 < I; k0 += BG_KC) {
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = tid + u * 256;
      As[e >> 5][e & 31] = ra[u];
      Bs[e >> 5][e & 31] = rb[u];
    }
    __syncthreads();
    if (k0 + BG_KC < I) load(k0 + BG_KC);
#pragma unroll 16
    for (int k = 0; k < BG_KC; ++k) {
      const float x0 = As[k][ty], x1 = As[k][ty + 16];
      const float y0 = Bs[k][tx], y1 = Bs[k][tx + 16];
      acc[0][0] = fmaf(x0, y0, acc[0][0]);
      acc[0][1] = fmaf(x0, y1, acc[0][1]);
      acc[1][0] = fmaf(x1, y0, acc[1][0]);
      acc[1][1] = fmaf(x1, y1, acc[1][1]);
    }
  }
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int a = a0 + ty + 16 * u, b = b0 + tx + 16 * v;
      if (a >= s || b >= s) continue;
      H[(size_t)a * s + b] = acc[u][v];
      H[(size_t)b * s + a] = acc[u][v];
    }
}

// k_gram_at with all of K = I (<= BG_KS16) staged at once by 16-byte
// asynchronous copies (s % 4 == 0): tile columns a0.., b0.. of every row.
__global__ void __launch_bounds__(256) k_gram_at16(const float* __restrict__ A, int I, int s, float* __restrict__ H) {
  pdl_prologue();
  extern __shared__ __align__(16) float g16[];
  float* As = g16;                 // [I][BG_BST]: As[k][c] = A[k][a0 + c]
  float* Bs = g16 + BG_KS16 * BG_BST;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int nt = (s + 31) / 32;
  int t = blockIdx.x, ta = 0;
  while (t >= nt - ta) {
    t -= nt - ta;
    ++ta;
  }
  const int a0 = 32 * ta, b0 = 32 * (ta + t);
  for (int e = tid; e < I * 16; e += 256) {
    const int k = e >> 4, h = (e >> 3) & 1, c4 = e & 7;  // h: 0 the a-tile, 1 the b-tile
    const int col0 = (h ? b0 : a0) + 4 * c4;
    float* dst = (h ? Bs : As) + k * BG_BST + 4 * c4;
    if (col0 + 3 < s)
      ch_acopy16(dst, A + (size_t)k * s + col0);
    else
      for (int u = 0; u < 4; ++u) dst[u] = col0 + u < s ? A[(size_t)k * s + col0 + u] : 0.0f;
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll 8
  for (int k = 0; k < I; ++k) {
    const float x0 = As[k * BG_BST + ty], x1 = As[k * BG_BST + ty + 16];
    const float y0 = Bs[k * BG_BST + tx], y1 = Bs[k * BG_BST + tx + 16];
    acc[0][0] = fmaf(x0, y0, acc[0][0]);
    acc[0][1] = fmaf(x0, y1, acc[0][1]);
    acc[1][0] = fmaf(x1, y0, acc[1][0]);
    acc[1][1] = fmaf(x1, y1, acc[1][1]);
  }
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int a = a0 + ty + 16 * u, b = b0 + tx + 16 * v;
      if (a >= s || b >= s) continue;
      H[(size_t)a * s + b] = acc[u][v];
      H[(size_t)b * s + a] = acc[u][v];
    }
}

constexpr int RD_ROWS = 8;

__device__ __forceinline__ void df_add(float& s, float& c, float p) {
  const float t = s + p;
  c += fabsf(s) >= fabsf(p) ? (s - t) + p : (p - t) + s;
  s = t;
}

// One output per thread (row r = tid / 32 of the tile, column tid % 32); the
// even and odd terms of the sum go to two independent compensated chains.
__global__ void __launch_bounds__(256) k_resid_df(const double* __restrict__ Yd, const double* __restrict__ A64,
                                                  const float* __restrict__ Ac, const float* __restrict__ Alo,
                                                  const float* __restrict__ G, int I, int s, double lam, double rho,
                                                  double c0, double c1, float* __restrict__ R) {
  pdl_prologue();
  extern __shared__ __align__(16) float rsm[];
  float* Ah = rsm;                    // [RD_ROWS][s]
  float* Al = Ah + RD_ROWS * s;       // [RD_ROWS][s]
  float* Gt = Al + RD_ROWS * s;       // [s][33]: columns j0 .. j0 + 31 of G
  const int tid = threadIdx.x, r = tid >> 5, cx = tid & 31;
  const int i0 = blockIdx.y * RD_ROWS, j0 = blockIdx.x * 32;
  // operands staged by 4-byte asynchronous copies, all in flight at once
  // (zeros written directly outside the matrices)
  for (int e = tid; e < RD_ROWS * s; e += 256) {
    const int rr = e / s, q = e - rr * s;
    if (i0 + rr < I) {
      ch_acopy4(Ah + e, Ac + (size_t)(i0 + rr) * s + q);
      ch_acopy4(Al + e, Alo + (size_t)(i0 + rr) * s + q);
    } else {
      Ah[e] = 0.0f;
      Al[e] = 0.0f;
    }
  }
  for (int e = tid; e < s * 32; e += 256) {
    const int q = e >> 5, c = e & 31;
    if (j0 + c < s)
      ch_acopy4(Gt + q * 33 + c, G + (size_t)q * s + j0 + c);
    else
      Gt[q * 33 + c] = 0.0f;
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  float sa = 0.f, ka = 0.f, sb = 0.f, kb = 0.f;
  const float* ah = Ah + r * s;
  const float* al = Al + r * s;
  int q = 0;
  for (; q + 1 < s; q += 2) {
    const float h0 = ah[q], l0 = al[q], g0 = Gt[q * 33 + cx];
    const float h1 = ah[q + 1], l1 = al[q + 1], g1 = Gt[(q + 1) * 33 + cx];
    const float p0 = h0 * g0, p1 = h1 * g1;
    ka += fmaf(h0, g0, -p0);
    kb += fmaf(h1, g1, -p1);
    ka = fmaf(l0, g0, ka);
    kb = fmaf(l1, g1, kb);
    df_add(sa, ka, p0);
    df_add(sb, kb, p1);
  }
  if (q < s) {
    const float h0 = ah[q], l0 = al[q], g0 = Gt[q * 33 + cx];
    const float p0 = h0 * g0;
    ka += fmaf(h0, g0, -p0);
    ka = fmaf(l0, g0, ka);
    df_add(sa, ka, p0);
  }
  const int i = i0 + r, j = j0 + cx;
  if (i >= I || j >= s) return;
  const int im = (i - 1 + I) % I, ip = (i + 1) % I;
  const double ag = ((double)sa + (double)sb) + ((double)ka + (double)kb);
  const double a = A64[(size_t)i * s + j];
  const double la = c0 * a + c1 * (A64[(size_t)im * s + j] + A64[(size_t)ip * s + j]);
  R[(size_t)i * s + j] = (float)(Yd[(size_t)i * s + j] - lam * la - rho * a - ag);
}

}  // namespace

int chol_groups(int I) { return I / 2 + 1; }
bool chol_supported(int s) { return s >= 1 && s <= CH_MAXS; }
size_t chol_factor_floats(int I, int s) { return (size_t)chol_groups(I) * ch_pack(s); }
size_t chol_dinv_floats(int I, int s) { return (size_t)chol_groups(I) * ch_npan(s) * CH_DBLK; }

void launch_chol_factor(const float* G, int I, int s, double lam, double c0, double c1, double rho, float* L,
                        float* Dinv, int* status, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_chol_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  const size_t bytes = (size_t)ch_pack(s) * 4;
  ChMaps maps;
  memset(&maps, 0, sizeof(maps));
  maps.on = (s % 4) == 0 ? 1 : 0;
  const int np = ch_npan(s), sp = 32 * np;
  for (int q = 0; q < np && maps.on; ++q)
    if (tma_map_f32(&maps.m[q], G, s, s, s, sp - 32 * q, 32) != FCTN_OK) maps.on = 0;
  launch_pdl(k_chol_factor, chol_groups(I), dim3(CH_NT), bytes, st, G, s, I, lam, c0, c1, rho, L, Dinv, status, maps);
}

void launch_chol_subst(const float* Rt, int I, int s, const float* L, const float* Dinv, float* W, int* status,
                       cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_chol_subst, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  launch_pdl(k_chol_subst, chol_groups(I), dim3(CH_NT), ch_subst_bytes(s), st, Rt, I, s, L, Dinv, W, status);
}

void launch_basis_gemm(int mode, const float* Qm, const float* B, int I, int s, float* out32, double* A64, float* Ac,
                       float* Alo, cudaStream_t st) {
  dim3 grid((unsigned)((s + 31) / 32), (unsigned)((I + 31) / 32));
  const bool v16 = I % 4 == 0 && s % 4 == 0 && I <= BG_KS16 && ((uintptr_t)Qm & 15) == 0 && ((uintptr_t)B & 15) == 0;
  if (v16) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_bgemm16<BG_STORE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bg16_smem_bytes());
      cudaFuncSetAttribute(k_bgemm16<BG_SET>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bg16_smem_bytes());
      cudaFuncSetAttribute(k_bgemm16<BG_ADD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bg16_smem_bytes());
      attr = true;
    }
    const size_t sm = bg16_smem_bytes();
    if (mode == BG_STORE)
      launch_pdl(k_bgemm16<BG_STORE>, grid, dim3(256), sm, st, Qm, B, I, s, I, out32, A64, Ac, Alo);
    else if (mode == BG_SET)
      launch_pdl(k_bgemm16<BG_SET>, grid, dim3(256), sm, st, Qm, B, I, s, I, out32, A64, Ac, Alo);
    else
      launch_pdl(k_bgemm16<BG_ADD>, grid, dim3(256), sm, st, Qm, B, I, s, I, out32, A64, Ac, Alo);
    return;
  }
  if (mode == BG_STORE)
    launch_pdl(k_bgemm<BG_STORE>, grid, dim3(256), 0, st, Qm, B, I, s, I, out32, A64, Ac, Alo);
  else if (mode == BG_SET)
    launch_pdl(k_bgemm<BG_SET>, grid, dim3(256), 0, st, Qm, B, I, s, I, out32, A64, Ac, Alo);
  else
    launch_pdl(k_bgemm<BG_ADD>, grid, dim3(256), 0, st, Qm, B, I, s, I, out32, A64, Ac, Alo);
}

void launch_gram_at(const float* A, int I, int s, float* H, cudaStream_t st) {
  const int nt = (s + 31) / 32;
  if (s % 4 == 0 && I <= BG_KS16 && ((uintptr_t)A & 15) == 0) {
    static bool attr = false;
    const size_t sm = (size_t)2 * BG_KS16 * BG_BST * 4;
    if (!attr) {
      cudaFuncSetAttribute(k_gram_at16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      attr = true;
    }
    launch_pdl(k_gram_at16, nt * (nt + 1) / 2, dim3(256), sm, st, A, I, s, H);
    return;
  }
  launch_pdl(k_gram_at, nt * (nt + 1) / 2, dim3(256), 0, st, A, I, s, H);
}

void launch_resid_df(const double* Yd, const double* A64, const float* Ac, const float* Alo, const float* G, int I,
                     int s, double lam, double rho, double c0, double c1, float* R, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_resid_df, cudaFuncAttributeMaxDynamicSharedMemorySize, 120 * 1024);
    attr = true;
  }
  const size_t bytes = ((size_t)2 * RD_ROWS * s + (size_t)s * 33) * 4;
  dim3 grid((unsigned)((s + 31) / 32), (unsigned)((I + RD_ROWS - 1) / RD_ROWS));
  launch_pdl(k_resid_df, grid, dim3(256), bytes, st, Yd, A64, Ac, Alo, G, I, s, lam, rho, c0, c1, R);
}
