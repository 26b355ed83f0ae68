// Factor solve of Eqs. 5-8: the symmetric eigendecomposition of the Gram
// (block-ordered two-sided Jacobi for FP32 Grams up to 128 x 128, one-sided
// Jacobi otherwise), the eigen-route solve with its FP64 refinement, and the
// reductions of the objective (Eq. 2) and the stop test.
#include <float.h>

#include <algorithm>

#include "fctn_internal.cuh"
#include "fctn_jacobi.cuh"

namespace {
using namespace fctn_jacobi;

// ------------------------------------------------------- eigensolver ----
template <typename T> struct Eps;
template <> struct Eps<float> { static __device__ float v() { return FLT_EPSILON; } };
template <> struct Eps<double> { static __device__ double v() { return DBL_EPSILON; } };

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Symmetric eigendecomposition G = C Phi C^T (Eq. 7) by one-sided Jacobi
// (Hestenes 1958): the columns a_j of A = G V are made mutually orthogonal by
// plane rotations applied to A and V alike, so A = G V stays invariant and,
// at convergence, the columns of V are eigenvectors of the symmetric G and
// Phi_j = v_j^T G v_j = v_j . a_j.  Pairs follow the round-robin schedule
// (m/2 disjoint pairs per round, m-1 rounds per sweep); a group of 8 lanes
// owns one pair; a pair only touches its own two rows of A^T and V^T, so one
// barrier per round suffices.  A pair is skipped once
// (a_p . a_q)^2 <= tol^2 |a_p|^2 |a_q|^2 + floor^2 with tol = sqrt(s) eps and
// floor = eps^2 ||G||_F^2 / s.
// Warm start: V0 (the previous sweep's C for the same factor) is first
// re-orthonormalised by one Newton-Schulz step V0 (3I - V0^T V0)/2.
// Also checks min_j Phi_j + tmin > 0 (T of Eq. 8 positive) -> FCTN_E_SINGULAR.
// The sweep limit is not an error: *sweeps_used is then -max_sweeps (the
// sign tells the host that the stop test did not hold).
constexpr int EG = 16;  // lanes per pair

// Sum over the EG lanes of one group.  The mask names only this group's lanes:
// other groups of the same warp may be skipping a pair or have left the loop.
template <typename T>
__device__ __forceinline__ T group_sum(T v) {
  const unsigned mask = (EG == 32) ? 0xffffffffu : (((1u << EG) - 1u) << (EG * ((threadIdx.x & 31) / EG)));
#pragma unroll
  for (int o = EG / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
  return v;
}

// Rotation (cos, sin) that zeroes a_p . a_q: t = sgn(zeta) / (|zeta| + sqrt(1 + zeta^2)),
// zeta = (|a_q|^2 - |a_p|^2) / (2 a_p . a_q).  In FP32 the angle uses fast
// approximations (an inexact angle only leaves the pair slightly less
// orthogonal), while c = 1/sqrt(1 + t^2) gets a Newton step so that the
// rotation stays orthogonal to working precision.
__device__ __forceinline__ void rot_cs(float al, float be, float ga, float& cs, float& sn, float& t) {
  float zeta = __fdividef(be - al, 2.f * ga);
  float w = fmaf(zeta, zeta, 1.f);
  float sq = w * rsqrtf(w);
  t = __fdividef(zeta >= 0.f ? 1.f : -1.f, fabsf(zeta) + sq);
  float x = fmaf(t, t, 1.f);
  float y = rsqrtf(x);
  cs = y * fmaf(-0.5f * x * y, y, 1.5f);  // one Newton step: c^2 (1 + t^2) = 1 to about an ulp
  sn = cs * t;
}
__device__ __forceinline__ void rot_cs(float al, float be, float ga, float& cs, float& sn) {
  float t;
  rot_cs(al, be, ga, cs, sn, t);
}
__device__ __forceinline__ void rot_cs(double al, double be, double ga, double& cs, double& sn) {
  double zeta = (be - al) / (2.0 * ga);
  double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  cs = 1.0 / sqrt(1.0 + t * t);
  sn = cs * t;
}

// A_SM / V_SM: A^T / V^T live in shared memory (compile-time, so that the
// accesses compile to shared-memory loads rather than generic ones).
template <typename T, bool A_SM, bool V_SM>
__global__ void __launch_bounds__(1024) k_eig1(const T* __restrict__ G, T* __restrict__ Cio, T* __restrict__ Phi,
                                               T* __restrict__ gwork, int s, int warm, int max_sweeps, double tmin,
                                               int* status, int* sweeps_used) {
  extern __shared__ __align__(16) unsigned char sm[];
  constexpr bool a_smem = A_SM, v_smem = V_SM;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
  const int grp = tid / EG, gl = tid % EG, ngrp = nt / EG;
  const int m = s + (s & 1), npair = m / 2;
  const int64_t ss = (int64_t)s * s;
  T* At;  // row j = a_j
  T* Vt;  // row j = v_j
  if constexpr (a_smem) At = (T*)sm; else At = gwork;
  if constexpr (v_smem) Vt = (T*)sm + (a_smem ? ss : 0); else Vt = gwork + ss;
  T* S = gwork + 2 * ss;                                 // s x s scratch (global)
  __shared__ T red[32];
  __shared__ int rotated;
  // ---- V0 and A = G V0
  if (warm) {
    for (int64_t e = tid; e < ss; e += nt) {             // At <- V0^T (row j = v0_j)
      int r = (int)(e / s), j = (int)(e % s);
      At[(int64_t)j * s + r] = Cio[e];
    }
    __syncthreads();
    for (int64_t e = tid; e < ss; e += nt) {             // S = V0^T V0 (from V0 in global: no bank conflicts)
      int a = (int)(e / s), b = (int)(e % s);
      T acc = 0;
      for (int r = 0; r < s; ++r) acc = fma(Cio[(int64_t)r * s + a], Cio[(int64_t)r * s + b], acc);
      S[e] = acc;
    }
    __syncthreads();
    for (int64_t e = tid; e < ss; e += nt) {             // Vt[j][r] = 1.5 v0_j[r] - 0.5 sum_q S[j][q] v0_q[r]
      int j = (int)(e / s), r = (int)(e % s);
      T acc = 0;
      for (int q = 0; q < s; ++q) acc = fma(S[(int64_t)j * s + q], At[(int64_t)q * s + r], acc);
      Vt[e] = (T)1.5 * At[e] - (T)0.5 * acc;
    }
  } else {
    for (int64_t e = tid; e < ss; e += nt) Vt[e] = (e / s == e % s) ? (T)1 : (T)0;
  }
  __syncthreads();
  for (int64_t e = tid; e < ss; e += nt) {               // At[j][c] = sum_r G[r][c] v_j[r]   (G symmetric)
    int j = (int)(e / s), c = (int)(e % s);
    T acc = 0;
    for (int r = 0; r < s; ++r) acc = fma(G[(int64_t)r * s + c], Vt[(int64_t)j * s + r], acc);
    At[e] = acc;
  }
  T fr = 0;
  for (int64_t e = tid; e < ss; e += nt) fr = fma(G[e], G[e], fr);
  fr = warp_sum(fr);
  if (lane == 0) red[tid >> 5] = fr;
  __syncthreads();
  if (tid == 0) {
    T t = 0;
    for (int w = 0; w < nt / 32; ++w) t += red[w];
    red[0] = t;
  }
  __syncthreads();
  const T eps = Eps<T>::v();
  const T tol = sqrt((T)(s > 1 ? s : 1)) * eps;
  // float4 rows: FP32, s a multiple of 4, rows 16-byte aligned (shared or
  // cudaMalloc'ed work, row stride s * 4 bytes)
  const bool vec4 = (sizeof(T) == 4) && (s % 4 == 0) && (s <= 16 * EG);  // at most 4 float4 per lane per row
  const int s4 = s / 4;
  const T floor_abs = eps * eps * red[0] / (T)(s > 0 ? s : 1);
  const T tol2 = tol * tol, floor2 = floor_abs * floor_abs;
  int sweep = 0;
  bool converged = (s <= 1);
  __shared__ float mu_max;  // largest (a_p.a_q)^2 / (|a_p|^2 |a_q|^2) rotated in this sweep
  for (; sweep < max_sweeps && !converged; ++sweep) {
    if (tid == 0) {
      rotated = 0;
      mu_max = 0.f;
    }
    __syncthreads();
    int any = 0;
    float mu_mine = 0.f;
    for (int round = 0; round < m - 1; ++round) {
      for (int idx = grp; idx < npair; idx += ngrp) {
        int p, q;
        if (idx == 0) { p = m - 1; q = round; }
        else { p = round + idx; if (p >= m - 1) p -= m - 1; q = round - idx; if (q < 0) q += m - 1; }
        if (p > q) { int t_ = p; p = q; q = t_; }
        if (q >= s) continue;
        T* ap = At + (int64_t)p * s;
        T* aq = At + (int64_t)q * s;
        T* vp = Vt + (int64_t)p * s;
        T* vq = Vt + (int64_t)q * s;
        T al = 0, be = 0, ga = 0;
        // rows of A kept in registers between the dot products and the rotation
        float4 xr[4], yr[4];
        if (vec4) {
          const float4* p4 = (const float4*)ap;
          const float4* q4 = (const float4*)aq;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int c = gl + u * EG;
            if (c < s4) {
              float4 x = p4[c], y = q4[c];
              xr[u] = x;
              yr[u] = y;
              al = fma(x.x, x.x, fma(x.y, x.y, fma(x.z, x.z, fma(x.w, x.w, al))));
              be = fma(y.x, y.x, fma(y.y, y.y, fma(y.z, y.z, fma(y.w, y.w, be))));
              ga = fma(x.x, y.x, fma(x.y, y.y, fma(x.z, y.z, fma(x.w, y.w, ga))));
            }
          }
        } else {
          for (int c = gl; c < s; c += EG) {
            T x = ap[c], y = aq[c];
            al = fma(x, x, al);
            be = fma(y, y, be);
            ga = fma(x, y, ga);
          }
        }
        al = group_sum(al);
        be = group_sum(be);
        ga = group_sum(ga);
        // rotate iff ga^2 > tol^2 al be + floor^2 (products only)
        const T ab = al * be, g2 = ga * ga;
        if (!(g2 > tol2 * ab + floor2)) continue;
        any = 1;
        mu_mine = fmaxf(mu_mine, (float)g2 * __frcp_rn((float)ab));  // squared ratio (ab > 0 here)
        T cs, sn;
        rot_cs(al, be, ga, cs, sn);
        if (vec4) {
          float4* p4 = (float4*)ap;
          float4* q4 = (float4*)aq;
          float4* u4 = (float4*)vp;
          float4* w4 = (float4*)vq;
#pragma unroll
          for (int uu = 0; uu < 4; ++uu) {
            const int c = gl + uu * EG;
            if (c >= s4) continue;
            float4 x = xr[uu], y = yr[uu], u = u4[c], w = w4[c];
            p4[c] = make_float4(cs * x.x - sn * y.x, cs * x.y - sn * y.y, cs * x.z - sn * y.z, cs * x.w - sn * y.w);
            q4[c] = make_float4(sn * x.x + cs * y.x, sn * x.y + cs * y.y, sn * x.z + cs * y.z, sn * x.w + cs * y.w);
            u4[c] = make_float4(cs * u.x - sn * w.x, cs * u.y - sn * w.y, cs * u.z - sn * w.z, cs * u.w - sn * w.w);
            w4[c] = make_float4(sn * u.x + cs * w.x, sn * u.y + cs * w.y, sn * u.z + cs * w.z, sn * u.w + cs * w.w);
          }
        } else {
          for (int c = gl; c < s; c += EG) {
            T x = ap[c], y = aq[c];
            ap[c] = cs * x - sn * y;
            aq[c] = sn * x + cs * y;
            T u = vp[c], w = vq[c];
            vp[c] = cs * u - sn * w;
            vq[c] = sn * u + cs * w;
          }
        }
      }
      __syncthreads();
    }
    if (any) {
      rotated = 1;
      atomicMax((int*)&mu_max, __float_as_int(mu_mine));  // non-negative floats order as ints
    }
    __syncthreads();
    // cyclic Jacobi converges quadratically: after a sweep whose largest
    // rotated off-term was below sqrt(tol), the next sweep would rotate
    // nothing above tol
    converged = (rotated == 0) || (mu_max < (float)tol);  // mu^2 < tol  <=>  mu < sqrt(tol)
    __syncthreads();
  }
  // Phi_j = v_j . a_j ; C[r][j] = Vt[j][r]
  for (int j = grp; j < s; j += ngrp) {
    T acc = 0;
    for (int c = gl; c < s; c += EG) acc = fma(Vt[(int64_t)j * s + c], At[(int64_t)j * s + c], acc);
    acc = group_sum(acc);
    if (gl == 0) Phi[j] = acc;
  }
  for (int64_t e = tid; e < ss; e += nt) {
    int r = (int)(e / s), j = (int)(e % s);
    Cio[e] = Vt[(int64_t)j * s + r];
  }
  __syncthreads();
  if (tid == 0) {
    T mn = Phi[0];
    for (int j = 1; j < s; ++j) mn = fmin(mn, Phi[j]);
    if (!((double)mn + tmin > 0.0)) atomicCAS(status, FCTN_OK, FCTN_E_SINGULAR);
    // not converged within max_sweeps: the eigenbasis is still orthogonal to
    // working precision; the refinement pass of the solve absorbs the rest.
    // The cap is reported (-max_sweeps) rather than failing.
    if (sweeps_used) *sweeps_used = converged ? sweep : -max_sweeps;
  }
}

// ---------------------------------------- two-sided Jacobi, FP32, s <= 128 ----
// The same decomposition G = C Phi C^T (Eq. 7) by the classical two-sided
// cyclic Jacobi method on B = V^T G V (Jacobi 1846; parallel orderings as in
// Golub & Van Loan, Sec. 8.5): each rotation J(p, q) zeroes B_pq,
// B <- J^T B J, V <- V J; at convergence Phi = diag(B), C = V.
// Warm start: V = V0 (3I - V0^T V0)/2 (one Newton-Schulz step on the previous
// sweep's C), B = V^T (G V).  The index set is padded to m = s rounded up to
// 8 (the padding rows and columns of B are zero and never rotate).

// out[i][j] = ca * sum_k op(X)[i][k] Y[k][j] (+ cb * Add[i][j]) for i, j < m,
// op(X) = X or X^T; m % 4 == 0; X, Y rows 16-byte aligned with strides that
// are multiples of 4.  Each thread owns a 4 x 4 tile; the Y rows are read as
// float4 (a warp reads consecutive words), X as a float4 of row k (TN) or as
// four words of column k (NN), shared by the threads of the same tile row.
template <bool TN>
__device__ __forceinline__ void sm_mm(float* __restrict__ out, int so, const float* __restrict__ X, int sx,
                                      const float* __restrict__ Y, int sy, int m, float ca,
                                      const float* __restrict__ Add, int sa, float cb) {
  const int mq = m / 4, ntile = mq * mq;
  for (int t = threadIdx.x; t < ntile; t += blockDim.x) {
    const int i0 = (t / mq) * 4, j0 = (t % mq) * 4;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
#pragma unroll 4
    for (int k = 0; k < m; ++k) {
      float x[4];
      if (TN) {
        const float4 xv = *(const float4*)(X + k * sx + i0);
        x[0] = xv.x;
        x[1] = xv.y;
        x[2] = xv.z;
        x[3] = xv.w;
      } else {
#pragma unroll
        for (int a = 0; a < 4; ++a) x[a] = X[(i0 + a) * sx + k];
      }
      const float4 yv = *(const float4*)(Y + k * sy + j0);
      const float y[4] = {yv.x, yv.y, yv.z, yv.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(x[a], y[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        float v = ca * acc[a][b];
        if (Add) v = fmaf(cb, Add[(i0 + a) * sa + j0 + b], v);
        out[(i0 + a) * so + j0 + b] = v;
      }
  }
}

// dst[r][j] (stride sd) <- src[r s + j] for r, j < m, zero outside s x s;
// warp w takes rows w, w + warps, ... (at most 8: the eigensolver launches at
// least m / 8 warps) and lane l columns l, l + 32, ... (m <= 128), with all of
// a thread's loads (two batches of 16) in flight before its stores.  Returns the thread's sum of
// squares of what it loaded.
__device__ __forceinline__ float ej_load(float* __restrict__ dst, int sd, const float* __restrict__ src, int s,
                                         int m) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  float ss = 0.f;
#pragma unroll
  for (int h = 0; h < 2; ++h) {  // two batches of 16 loads
    float v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int r = warp + (h * 4 + (u >> 2)) * nwarp, j = lane + (u & 3) * 32;
      v[u] = (r < s && j < s) ? src[r * s + j] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int r = warp + (h * 4 + (u >> 2)) * nwarp, j = lane + (u & 3) * 32;
      if (r < m && j < m) dst[r * sd + j] = v[u];
      ss = fmaf(v[u], v[u], ss);
    }
  }
  return ss;
}

// out = X^T Y for a product known to be symmetric (m % 4 == 0, layouts as
// sm_mm<true>): only the 4 x 4 tiles on and above the diagonal are formed,
// and each is written to both triangles, so out is exactly symmetric.
__device__ __forceinline__ void sm_mm_sym(float* __restrict__ out, int so, const float* __restrict__ X, int sx,
                                          const float* __restrict__ Y, int sy, int m) {
  const int mq = m / 4, ntile = mq * (mq + 1) / 2;
  for (int t = threadIdx.x; t < ntile; t += blockDim.x) {
    int ti = 0, b = t;
    while (b >= mq - ti) {
      b -= mq - ti;
      ++ti;
    }
    const int i0 = ti * 4, j0 = (ti + b) * 4;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][c] = 0.f;
#pragma unroll 4
    for (int k = 0; k < m; ++k) {
      const float4 xv = *(const float4*)(X + k * sx + i0);
      const float4 yv = *(const float4*)(Y + k * sy + j0);
      const float x[4] = {xv.x, xv.y, xv.z, xv.w}, y[4] = {yv.x, yv.y, yv.z, yv.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = fmaf(x[a], y[c], acc[a][c]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (b != 0 || a <= c) {
          out[(i0 + a) * so + j0 + c] = acc[a][c];
          out[(j0 + c) * so + i0 + a] = acc[a][c];
        }
  }
}

// Block-ordered two-sided Jacobi (FP32, s <= EIG3_MAX), one CTA: cyclic
// Jacobi sweeps whose pairs are ordered so that one parallel step
// touches only the index sets of disjoint 8 x 8 subproblems.  The m indices
// form nb = m / 4 blocks of four; outer round r pairs block P with block Q by
// the round-robin schedule, and half a warp rotates the submatrix B[S, S] of
// such a pair (S = P u Q, local indices 0-3 and 4-7) in four rounds of cross pairs
// (i, 4 + (i xor t)), preceded in the first outer round of a sweep by three
// rounds of pairs within a block, accumulating the product U of its
// rotations.  Every pair (p, q) is thus rotated once per sweep, as in a
// scalar cyclic sweep, and the rotation of a pair sees the same B_pp, B_qq,
// B_pq as it would there (rotations of other subproblems touch other rows
// and columns).  The CTA then applies J = diag(U) over the subproblems by
// 8 x 8 products held in registers: B <- J^T B and V^T <- J^T V^T (rows,
// 8 x 4 tiles), then B <- B J (columns, 4 x 8 tiles), the diagonal
// superblocks taking the rotated submatrix.  Inner rounds cost warp
// synchronisations only (a warp runs two subproblems in lockstep, so that
// fewer warps contend for issue slots); an outer round costs three block
// barriers.
// Rotation test and stop test: rotate iff B_pq^2 > tol^2 (|B_pp| + t)
// (|B_qq| + t) + floor^2 (tol = sqrt(s) eps, floor = eps ||G||_F / sqrt(s),
// t = max(tmin, 0), the smallest shift of Eq. 8: see k_eig4); stop after a
// sweep whose largest rotated ratio was below tol (quadratic convergence: the
// next sweep would rotate nothing), or before a sweep in which no pair would
// rotate (one scan of the upper triangle).
constexpr int EIG3_MAX = 128;
constexpr int EIGC_MIN = 64, EIGC_MAX = 256;  // FP32 Grams with EIGC_MIN < s <= EIGC_MAX: cluster Jacobi
constexpr int EJ_NT = 512;   // most threads
constexpr int EJ_TPT = 2;    // row tasks per thread: 128 * 128 / 16 <= 2 * 512

// Rotation of a pair from its 2 x 2 block [a g; g b] without a branch:
// t = sgn(d) 2g / (|d| + hypot(d, 2g)), d = b - a (the smaller root of
// t^2 + 2 zeta t - 1 = 0, zeta = d / 2g), c = 1 / sqrt(1 + t^2) with one
// Newton step (so that c^2 + sn^2 = 1 to about an ulp), sn = c t.  Returns
// g^2 / |a b| if the pair rotates, else -1 with c = 1, sn = t = 0.
__device__ __forceinline__ float ej_rot(float a, float b, float g, float tol2, float floor2, float& c, float& sn,
                                        float& t) {
  const float ab = fabsf(a * b), g2 = g * g;
  const bool rot = g2 > tol2 * ab + floor2;
  const float d = b - a, tg = 2.f * g;
  const float h = fmaf(d, d, tg * tg);
  const float hy = h * rsqrtf(h);
  const float tt = __fdividef(d >= 0.f ? tg : -tg, fabsf(d) + hy);
  const float x = fmaf(tt, tt, 1.f);
  const float y = rsqrtf(x);
  const float cc = y * fmaf(-0.5f * x * y, y, 1.5f);
  c = rot ? cc : 1.f;
  sn = rot ? cc * tt : 0.f;
  t = rot ? tt : 0.f;
  return rot ? __fdividef(g2, fmaxf(ab, FLT_MIN)) : -1.f;
}

// One inner round of a half warp on its subproblem (S, U in shared memory),
// the same instructions on every lane.  Lane L of the half updates the
// 2 x 2 block (L >> 2, L & 3) of the grid of this round's four pairs (rows
// rotated by the first pair, columns by the second; a diagonal block keeps
// the exact Jacobi update with zeroed off-diagonal) and rotates rows L >> 2
// and 4 + (L >> 2) of U by pair L & 3; lanes 0, 5, 10, 15 count their pair's
// rotation.  The two halves of a warp run two subproblems in lockstep.
template <bool W, int T>
__device__ __forceinline__ void ej_round(float* __restrict__ Sw, float* __restrict__ Uw, int hl, float tol2,
                                         float floor2, unsigned& cnt, float& cmu) {
  const int k = hl >> 2, l = hl & 3;
  int pk, qk, pl, ql;
  ej_pair(W, T, k, pk, qk);
  ej_pair(W, T, l, pl, ql);
  const float ak = Sw[pk * 9], bk = Sw[qk * 9], gk = Sw[pk * 8 + qk];
  const float al = Sw[pl * 9], bl = Sw[ql * 9], gl = Sw[pl * 8 + ql];
  const float x00 = Sw[pk * 8 + pl], x01 = Sw[pk * 8 + ql];
  const float x10 = Sw[qk * 8 + pl], x11 = Sw[qk * 8 + ql];
  const float u00 = Uw[k * 8 + pl], u01 = Uw[k * 8 + ql];
  const float u10 = Uw[(k + 4) * 8 + pl], u11 = Uw[(k + 4) * 8 + ql];
  __syncwarp();  // every read of this round before any write
  float ck, sk, tk, cl, sl, tl;
  const float mu = ej_rot(ak, bk, gk, tol2, floor2, ck, sk, tk);
  ej_rot(al, bl, gl, tol2, floor2, cl, sl, tl);
  const float y00 = ck * x00 - sk * x10, y01 = ck * x01 - sk * x11;
  const float y10 = sk * x00 + ck * x10, y11 = sk * x01 + ck * x11;
  float z00 = cl * y00 - sl * y01, z01 = sl * y00 + cl * y01;
  float z10 = cl * y10 - sl * y11, z11 = sl * y10 + cl * y11;
  const bool dg = (k == l) && mu >= 0.f;
  if (dg) {
    z00 = fmaf(-tk, gk, ak);
    z11 = fmaf(tk, gk, bk);
    z01 = 0.f;
    z10 = 0.f;
    ++cnt;
    cmu = fmaxf(cmu, mu);
  }
  Sw[pk * 8 + pl] = z00;
  Sw[pk * 8 + ql] = z01;
  Sw[qk * 8 + pl] = z10;
  Sw[qk * 8 + ql] = z11;
  Uw[k * 8 + pl] = cl * u00 - sl * u01;
  Uw[k * 8 + ql] = sl * u00 + cl * u01;
  Uw[(k + 4) * 8 + pl] = cl * u10 - sl * u11;
  Uw[(k + 4) * 8 + ql] = sl * u10 + cl * u11;
  __syncwarp();
}

__global__ void __launch_bounds__(EJ_NT) k_eig3(const float* __restrict__ G, float* __restrict__ Cio,
                                                float* __restrict__ Phi, int s, int warm, int max_sweeps,
                                                double tmin, double tol_in, int* status, int* sweeps_used) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int m = (s + 7) & ~7, sp = m + 4, nb = m / 4, nsub = m / 8, nsub2 = (nsub + 1) / 2;
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31, nwarp = nt >> 5;
  float* X1 = (float*)sm;
  float* X2 = X1 + m * sp;
  float* X3 = X2 + m * sp;  // warm-start scratch
  float* SC = X3 + m * sp;  // the subproblems and a spare slot
  __shared__ float red[32];
  __shared__ unsigned wrot[32], wmu[32];  // per subproblem warp: rotations and largest ratio of a sweep
  __shared__ int pq[16];                  // per subproblem: blocks P | Q << 16
  // B in X1, V^T in X2 (both stride sp); element loops run a warp per row
  // and a lane per column
  if (warm) {
    ej_load(X1, sp, Cio, s, m);  // X1 <- V0 (row r, column j)
    __syncthreads();
    sm_mm_sym(X2, sp, X1, sp, X1, sp, m);  // S = V0^T V0
    __syncthreads();
    sm_mm<false>(X3, sp, X1, sp, X2, sp, m, -0.5f, X1, sp, 1.5f);  // V = 1.5 V0 - 0.5 V0 S
    __syncthreads();
  }
  float fr = ej_load(X1, sp, G, s, m);  // X1 <- G; ||G||_F
  if (!warm)
    for (int r = warp; r < m; r += nwarp)
      for (int j = lane; j < m; j += 32) X2[r * sp + j] = (r == j) ? 1.f : 0.f;
  fr = warp_sum(fr);
  if (lane == 0) red[warp] = fr;
  __syncthreads();
  if (warm) {
    sm_mm<true>(X2, sp, X1, sp, X3, sp, m, 1.f, nullptr, 0, 0.f);  // W = G V = G^T V (G symmetric)
    __syncthreads();
    sm_mm_sym(X1, sp, X3, sp, X2, sp, m);  // B = V^T W, exactly symmetric
    __syncthreads();
    for (int r = warp; r < m; r += nwarp)  // V^T
      for (int j = lane; j < m; j += 32) X2[j * sp + r] = X3[r * sp + j];
  } else {
    for (int r = warp; r < m; r += nwarp)  // symmetrise B = G
      for (int j = lane; j < m; j += 32)
        if (r < j) {
          const float v = 0.5f * (X1[r * sp + j] + X1[j * sp + r]);
          X1[r * sp + j] = v;
          X1[j * sp + r] = v;
        }
  }
  if (tid == 0) {
    float t = 0.f;
    for (int w = 0; w < nwarp; ++w) t += red[w];
    red[0] = sqrtf(t);
  }
  __syncthreads();
  const float eps = FLT_EPSILON;
  const float tol = tol_in > 0.0 ? (float)tol_in : sqrtf((float)(s > 1 ? s : 1)) * eps;
  const float tol2 = tol * tol;
  const float floor_abs = eps * red[0] * rsqrtf((float)(s > 0 ? s : 1));
  const float floor2 = floor_abs * floor_abs;
  float* B = X1;
  float* Vt = X2;
  // This thread's row tasks (subproblem a, column quad cq; on V^T if v) and
  // column task (subproblem b, row quad rq), fixed for the whole call; a
  // quarter warp shares a and takes consecutive quads, resp. shares rq and
  // takes eight subproblems.
  const int nq = m / 4, nr1 = nsub * nq;
  int rt[EJ_TPT];
#pragma unroll
  for (int i = 0; i < EJ_TPT; ++i) {
    const int t1 = tid + i * nt;
    if (t1 < 2 * nr1) {
      const int v = t1 >= nr1, tt = v ? t1 - nr1 : t1;
      rt[i] = (tt / nq) | (tt % nq) << 8 | v << 16;
    } else {
      rt[i] = -1;
    }
  }
  const int ctk = tid < nr1 ? (tid % nsub) | (tid / nsub) << 8 : -1;
  unsigned cnt = 0;  // rotations and largest ratio of this lane's pair in the current sweep
  float cmu = 0.f;
  int sweep = 0;
  bool converged = (s <= 1);
  const float tsh = tmin > 0.0 ? (float)tmin : 0.f;
  __shared__ int any_rot;
  for (; sweep < max_sweeps && !converged; ++sweep) {
    // a sweep in which no pair would pass the rotation test changes nothing:
    // scan the upper triangle once and stop without running it
    if (tid == 0) any_rot = 0;
    __syncthreads();
    {
      bool want = false;
      for (int e = tid; e < s * s && !want; e += nt) {
        const int p = e / s, q = e - p * s;
        if (q <= p) continue;
        const float a = B[p * sp + p], b = B[q * sp + q], g = B[p * sp + q];
        want = g * g > tol2 * (fabsf(a) + tsh) * (fabsf(b) + tsh) + floor2;
      }
      if (__any_sync(0xffffffffu, want) && lane == 0) any_rot = 1;
    }
    __syncthreads();
    if (!any_rot) {
      converged = true;
      break;
    }
    for (int r = 0; r < nb - 1; ++r) {
      for (int sw = warp; sw < nsub2; sw += nwarp) {
        const int sub = 2 * sw + (lane >> 4), hl = lane & 15;
        const bool real = sub < nsub;  // else the spare slot, which never rotates
        float* Sw = SC + (real ? sub : nsub) * EJ_SUB;
        float* Uw = Sw + 64;
        int P = 0, Q = 0;
        if (real) {
          round_pair(nb, r, sub, P, Q);
          if (hl == 0) pq[sub] = P | Q << 16;
        }
        for (int e = hl; e < 64; e += 16) {
          const int i = e >> 3, j = e & 7;
          const int gi = i < 4 ? 4 * P + i : 4 * Q + i - 4, gj = j < 4 ? 4 * P + j : 4 * Q + j - 4;
          Sw[e] = real ? B[gi * sp + gj] : 0.f;
          Uw[e] = (i == j) ? 1.f : 0.f;
        }
        __syncwarp();
        if (r == 0) {
          ej4_round<true, 0>(Sw, Uw, hl, tol2, floor2, tsh, cnt, cmu);
          ej4_round<true, 1>(Sw, Uw, hl, tol2, floor2, tsh, cnt, cmu);
          ej4_round<true, 2>(Sw, Uw, hl, tol2, floor2, tsh, cnt, cmu);
        }
        ej4_round<false, 0>(Sw, Uw, hl, tol2, floor2, tsh, cnt, cmu);
        ej4_round<false, 1>(Sw, Uw, hl, tol2, floor2, tsh, cnt, cmu);
        ej4_round<false, 2>(Sw, Uw, hl, tol2, floor2, tsh, cnt, cmu);
        ej4_round<false, 3>(Sw, Uw, hl, tol2, floor2, tsh, cnt, cmu);
      }
      if (r == nb - 2 && warp < nsub2) {  // this sweep's totals per warp
        const unsigned cn = __reduce_add_sync(0xffffffffu, cnt);
        const unsigned mx = __reduce_max_sync(0xffffffffu, __float_as_uint(cmu));  // cmu >= 0
        if (lane == 0) {
          wrot[warp] = cn;
          wmu[warp] = mx;
        }
        cnt = 0;
        cmu = 0.f;
      }
      __syncthreads();
      // rows: B[S_a, quad] <- U_a^T B[S_a, quad] outside S_a's own columns,
      // and V^T[S_a, quad] <- U_a^T V^T[S_a, quad]
#pragma unroll
      for (int i = 0; i < EJ_TPT; ++i) {
        if (rt[i] < 0) break;
        const int a = rt[i] & 0xff, cq = (rt[i] >> 8) & 0xff;
        const bool isv = rt[i] >> 16;
        const int P = pq[a] & 0xffff, Q = pq[a] >> 16;
        if (!isv && (cq == P || cq == Q)) continue;
        float* Mx = (isv ? Vt : B) + 4 * cq;
        const float* Ua = SC + a * EJ_SUB + 64;
        float acc[8][4];
#pragma unroll
        for (int o = 0; o < 8; ++o) acc[o][0] = acc[o][1] = acc[o][2] = acc[o][3] = 0.f;
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const float4 x = *(const float4*)(Mx + (kk < 4 ? 4 * P + kk : 4 * Q + kk - 4) * sp);
          const float4 ua = *(const float4*)(Ua + kk * 8), ub = *(const float4*)(Ua + kk * 8 + 4);
          const float u[8] = {ua.x, ua.y, ua.z, ua.w, ub.x, ub.y, ub.z, ub.w};
#pragma unroll
          for (int o = 0; o < 8; ++o) {
            acc[o][0] = fmaf(u[o], x.x, acc[o][0]);
            acc[o][1] = fmaf(u[o], x.y, acc[o][1]);
            acc[o][2] = fmaf(u[o], x.z, acc[o][2]);
            acc[o][3] = fmaf(u[o], x.w, acc[o][3]);
          }
        }
#pragma unroll
        for (int o = 0; o < 8; ++o)
          *(float4*)(Mx + (o < 4 ? 4 * P + o : 4 * Q + o - 4) * sp) =
              make_float4(acc[o][0], acc[o][1], acc[o][2], acc[o][3]);
      }
      __syncthreads();
      // columns: B[quad, S_b] <- B[quad, S_b] U_b; the subproblem's own
      // superblock from its warp
      if (ctk >= 0) {
        const int b = ctk & 0xff, rq = ctk >> 8;
        const int P = pq[b] & 0xffff, Q = pq[b] >> 16;
        const float* Sb = SC + b * EJ_SUB;
        float* row0 = B + 4 * rq * sp;
        if (rq == P || rq == Q) {
          const int l0 = rq == P ? 0 : 4;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            *(float4*)(row0 + i * sp + 4 * P) = *(const float4*)(Sb + (l0 + i) * 8);
            *(float4*)(row0 + i * sp + 4 * Q) = *(const float4*)(Sb + (l0 + i) * 8 + 4);
          }
        } else {
          float w[4][8];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float4 w0 = *(const float4*)(row0 + i * sp + 4 * P), w1 = *(const float4*)(row0 + i * sp + 4 * Q);
            w[i][0] = w0.x;
            w[i][1] = w0.y;
            w[i][2] = w0.z;
            w[i][3] = w0.w;
            w[i][4] = w1.x;
            w[i][5] = w1.y;
            w[i][6] = w1.z;
            w[i][7] = w1.w;
          }
          const float* Ub = Sb + 64;
          float o[4][8];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) o[i][j] = 0.f;
#pragma unroll
          for (int kk = 0; kk < 8; ++kk) {
            const float4 ua = *(const float4*)(Ub + kk * 8), uc = *(const float4*)(Ub + kk * 8 + 4);
            const float u[8] = {ua.x, ua.y, ua.z, ua.w, uc.x, uc.y, uc.z, uc.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
              for (int j = 0; j < 8; ++j) o[i][j] = fmaf(w[i][kk], u[j], o[i][j]);
          }
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            *(float4*)(row0 + i * sp + 4 * P) = make_float4(o[i][0], o[i][1], o[i][2], o[i][3]);
            *(float4*)(row0 + i * sp + 4 * Q) = make_float4(o[i][4], o[i][5], o[i][6], o[i][7]);
          }
        }
      }
      __syncthreads();
    }
    unsigned cn = 0, mx = 0;
    for (int w = 0; w < min(nsub2, nwarp); ++w) {
      cn += wrot[w];
      mx = max(mx, wmu[w]);
    }
    converged = (cn == 0) || (__uint_as_float(mx) < tol);
  }
  for (int j = tid; j < s; j += nt) Phi[j] = B[j * sp + j];
  for (int r = warp; r < s; r += nwarp)  // C[r][j] = V[r][j] = V^T[j][r]
    for (int j = lane; j < s; j += 32) Cio[r * s + j] = Vt[j * sp + r];
  __syncthreads();
  if (tid == 0) {
    float mn = Phi[0];
    for (int j = 1; j < s; ++j) mn = fminf(mn, Phi[j]);
    if (!((double)mn + tmin > 0.0)) atomicCAS(status, FCTN_OK, FCTN_E_SINGULAR);
    if (sweeps_used) *sweeps_used = converged ? sweep : -max_sweeps;
  }
}

// ------------------------------ block-ordered Jacobi, FP32, 128 < s <= 224 ----
// The method of k_eig3 for Grams whose B and V^T do not fit on one SM
// together.  B = V^T G V alone stays in shared memory (224 x 228 floats at
// most); the warm-start products (one Newton-Schulz step V = V0 (3I -
// V0^T V0) / 2, then B = V^T (G V)) run before it as multi-CTA products
// (k_mm_small), and the rotation blocks U of every outer round are recorded
// in global memory instead of being applied to V^T on chip.  k_eig_apply then
// forms C = V J_1 J_2 ... row by row over many CTAs: a row of V meets every
// round's 8 x 8 blocks in order, independently of the other rows.
// Rotation test: rotate iff B_pq^2 > tol^2 (|B_pp| + t)(|B_qq| + t) + floor^2
// with t = max(tmin, 0), the smallest shift lambda Lambda_i + rho of Eq. 8:
// the solve divides by Phi_j + lambda Lambda_i + rho, so an off-diagonal B_pq
// perturbs it by B_pq / sqrt((Phi_p + t)(Phi_q + t)) at most, and pairs of
// eigenvalues far below the shift need no more accuracy than that.
constexpr int EIG4_MAX = 224;
constexpr int EJ4_NT = 512;          // 128 registers a thread: the 8 x 4 / 4 x 8 tiles stay unspilled
constexpr int EJ4_TPT = 4;           // row / column tasks per thread: (224 / 8) (224 / 4) <= 4 * 512
constexpr int EIG4_REC_SWEEPS = 16;  // sweeps whose rotation blocks fit the record

// C = ca op(A) Bm + cb D for s x s row-major matrices (op(A) = A or A^T),
// one 32 x 32 tile per CTA of 256 threads (2 x 2 outputs each).
template <bool TA>
__global__ void __launch_bounds__(256) k_mm_small(const float* __restrict__ A, const float* __restrict__ Bm,
                                                  const float* __restrict__ D, float* __restrict__ C, int s, float ca,
                                                  float cb) {
  __shared__ float As[32][33], Bs[32][33];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  for (int k0 = 0; k0 < s; k0 += 32) {
    for (int e = threadIdx.x; e < 1024; e += 256) {
      const int r = e >> 5, c = e & 31;
      // As[r][c] = op(A)[i0 + r][k0 + c]
      const int ai = i0 + r, ak = k0 + c;
      float av = 0.f;
      if (ai < s && ak < s) av = TA ? A[(int64_t)ak * s + ai] : A[(int64_t)ai * s + ak];
      As[r][c] = av;
      const int bk = k0 + r, bj = j0 + c;
      Bs[r][c] = (bk < s && bj < s) ? Bm[(int64_t)bk * s + bj] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const float a0 = As[ty * 2][k], a1 = As[ty * 2 + 1][k];
      const float b0 = Bs[k][tx * 2], b1 = Bs[k][tx * 2 + 1];
      acc[0][0] = fmaf(a0, b0, acc[0][0]);
      acc[0][1] = fmaf(a0, b1, acc[0][1]);
      acc[1][0] = fmaf(a1, b0, acc[1][0]);
      acc[1][1] = fmaf(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int i = i0 + ty * 2 + a, j = j0 + tx * 2 + b;
      if (i < s && j < s) {
        float v = ca * acc[a][b];
        if (D) v = fmaf(cb, D[(int64_t)i * s + j], v);
        C[(int64_t)i * s + j] = v;
      }
    }
}

// Jacobi sweeps on B (s x s in global memory, from the warm-start products
// or G itself).  Records, for outer round n (counted over all sweeps), the
// blocks U of the subproblems that rotated (entries RoundStart[n] ..
// RoundStart[n + 1] - 1 of Urec, 64 floats each, and of PQrec, their block
// pair); a subproblem without rotations has U = I and is neither recorded
// nor applied to B.  *nrounds gets the number of rounds.
__global__ void __launch_bounds__(EJ4_NT) k_eig4(const float* __restrict__ Bin, float* __restrict__ Phi, int s,
                                                 int max_sweeps, double tmin, float* __restrict__ Urec,
                                                 int* __restrict__ PQrec, int* __restrict__ RoundStart,
                                                 int* __restrict__ nrounds, int* status, int* sweeps_used) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int m = (s + 7) & ~7, sp = m + 4, nb = m / 4, nsub = m / 8, nsub2 = (nsub + 1) / 2;
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31, nwarp = nt >> 5;
  float* B = (float*)sm;
  float* SC = B + m * sp;
  __shared__ float red[32];
  __shared__ unsigned wrot[32], wmu[32];
  __shared__ int pq[32];
  __shared__ int rotf[32];   // subproblem rotated in this outer round
  __shared__ int slot[32];   // its entry in the record, or -1
  __shared__ int nrec_s;     // entries recorded so far
  float fr = 0.f;
  if (tid == 0) nrec_s = 0;
  for (int r = warp; r < m; r += nwarp)
    for (int j = lane; j < m; j += 32) {
      float v = 0.f;
      if (r < s && j < s) v = 0.5f * (Bin[(int64_t)r * s + j] + Bin[(int64_t)j * s + r]);
      B[r * sp + j] = v;
      fr = fmaf(v, v, fr);
    }
  fr = warp_sum(fr);
  if (lane == 0) red[warp] = fr;
  __syncthreads();
  if (tid == 0) {
    float t = 0.f;
    for (int w = 0; w < nwarp; ++w) t += red[w];
    red[0] = sqrtf(t);
  }
  __syncthreads();
  const float eps = FLT_EPSILON;
  const float tol = sqrtf((float)(s > 1 ? s : 1)) * eps;
  const float tol2 = tol * tol;
  const float floor_abs = eps * red[0] * rsqrtf((float)(s > 0 ? s : 1));
  const float floor2 = floor_abs * floor_abs;
  const float tsh = tmin > 0.0 ? (float)tmin : 0.f;
  const int nq = m / 4, nr1 = nsub * nq;
  int rt[EJ4_TPT], ct[EJ4_TPT];
#pragma unroll
  for (int i = 0; i < EJ4_TPT; ++i) {
    const int t1 = tid + i * nt;
    rt[i] = t1 < nr1 ? (t1 / nq) | (t1 % nq) << 8 : -1;
    ct[i] = t1 < nr1 ? (t1 % nsub) | (t1 / nsub) << 8 : -1;
  }
  unsigned cnt = 0;
  float cmu = 0.f;
  int sweep = 0, nround = 0;
  bool converged = (s <= 1);
  const int sweep_cap = max_sweeps < EIG4_REC_SWEEPS ? max_sweeps : EIG4_REC_SWEEPS;
  __shared__ int any_rot;
  for (; sweep < sweep_cap && !converged; ++sweep) {
    // a sweep in which no pair would pass the rotation test changes nothing:
    // scan the upper triangle once and stop without running it
    if (tid == 0) any_rot = 0;
    __syncthreads();
    {
      bool want = false;
      for (int e = tid; e < s * s && !want; e += nt) {
        const int p = e / s, q = e - p * s;
        if (q <= p) continue;
        const float a = B[p * sp + p], b = B[q * sp + q], g = B[p * sp + q];
        want = g * g > tol2 * (fabsf(a) + tsh) * (fabsf(b) + tsh) + floor2;
      }
      if (__any_sync(0xffffffffu, want) && lane == 0) any_rot = 1;
    }
    __syncthreads();
    if (!any_rot) {
      converged = true;
      break;
    }
    for (int r = 0; r < nb - 1; ++r, ++nround) {
      for (int sw = warp; sw < nsub2; sw += nwarp) {
        const int sub = 2 * sw + (lane >> 4), hl = lane & 15;
        const bool real = sub < nsub;
        float* Sw = SC + (real ? sub : nsub) * EJ_SUB;
        float* Uw = Sw + 64;
        int P = 0, Q = 0;
        if (real) {
          round_pair(nb, r, sub, P, Q);
          if (hl == 0) pq[sub] = P | Q << 16;
        }
        for (int e = hl; e < 64; e += 16) {
          const int i = e >> 3, j = e & 7;
          const int gi = i < 4 ? 4 * P + i : 4 * Q + i - 4, gj = j < 4 ? 4 * P + j : 4 * Q + j - 4;
          Sw[e] = real ? B[gi * sp + gj] : 0.f;
          Uw[e] = (i == j) ? 1.f : 0.f;
        }
        __syncwarp();
        const unsigned cnt0 = cnt;
        if (r == 0) {
          ej4_round<true, 0>(Sw, Uw, hl, tol2, floor2, tsh, cnt, cmu);
          ej4_round<true, 1>(Sw, Uw, hl, tol2, floor2, tsh, cnt, cmu);
          ej4_round<true, 2>(Sw, Uw, hl, tol2, floor2, tsh, cnt, cmu);
        }
        ej4_round<false, 0>(Sw, Uw, hl, tol2, floor2, tsh, cnt, cmu);
        ej4_round<false, 1>(Sw, Uw, hl, tol2, floor2, tsh, cnt, cmu);
        ej4_round<false, 2>(Sw, Uw, hl, tol2, floor2, tsh, cnt, cmu);
        ej4_round<false, 3>(Sw, Uw, hl, tol2, floor2, tsh, cnt, cmu);
        const unsigned any = __ballot_sync(0xffffffffu, cnt != cnt0);
        if (real && hl == 0) rotf[sub] = ((any >> (lane & 16)) & 0xffffu) != 0u;
      }
      if (r == nb - 2 && warp < nsub2) {
        const unsigned cn = __reduce_add_sync(0xffffffffu, cnt);
        const unsigned mx = __reduce_max_sync(0xffffffffu, __float_as_uint(cmu));
        if (lane == 0) {
          wrot[warp] = cn;
          wmu[warp] = mx;
        }
        cnt = 0;
        cmu = 0.f;
      }
      __syncthreads();
      // record the blocks of the subproblems that rotated (k_eig_apply);
      // round n's entries start at RoundStart[n]
      if (warp == 0) {
        const bool f = lane < nsub && rotf[lane];
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        const int base = nrec_s;
        if (lane < nsub) slot[lane] = f ? base + __popc(bal & ((1u << lane) - 1u)) : -1;
        if (lane == 0) {
          RoundStart[nround] = base;
          RoundStart[nround + 1] = base + __popc(bal);
        }
        __syncwarp();
        if (lane == 0) nrec_s = base + __popc(bal);
      }
      __syncthreads();
      for (int e = tid; e < nsub * 64; e += nt) {
        const int a = e >> 6, q = slot[a];
        if (q >= 0) Urec[(int64_t)q * 64 + (e & 63)] = SC[a * EJ_SUB + 64 + (e & 63)];
      }
      for (int a = tid; a < nsub; a += nt)
        if (slot[a] >= 0) PQrec[slot[a]] = pq[a];
      // rows: B[S_a, quad] <- U_a^T B[S_a, quad] outside S_a's own columns
#pragma unroll
      for (int i = 0; i < EJ4_TPT; ++i) {
        if (rt[i] < 0) break;
        const int a = rt[i] & 0xff, cq = rt[i] >> 8;
        const int P = pq[a] & 0xffff, Q = pq[a] >> 16;
        if (cq == P || cq == Q || !rotf[a]) continue;  // U_a = I: nothing to apply
        float* Mx = B + 4 * cq;
        const float* Ua = SC + a * EJ_SUB + 64;
        float acc[8][4];
#pragma unroll
        for (int o = 0; o < 8; ++o) acc[o][0] = acc[o][1] = acc[o][2] = acc[o][3] = 0.f;
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const float4 x = *(const float4*)(Mx + (kk < 4 ? 4 * P + kk : 4 * Q + kk - 4) * sp);
          const float4 ua = *(const float4*)(Ua + kk * 8), ub = *(const float4*)(Ua + kk * 8 + 4);
          const float u[8] = {ua.x, ua.y, ua.z, ua.w, ub.x, ub.y, ub.z, ub.w};
#pragma unroll
          for (int o = 0; o < 8; ++o) {
            acc[o][0] = fmaf(u[o], x.x, acc[o][0]);
            acc[o][1] = fmaf(u[o], x.y, acc[o][1]);
            acc[o][2] = fmaf(u[o], x.z, acc[o][2]);
            acc[o][3] = fmaf(u[o], x.w, acc[o][3]);
          }
        }
#pragma unroll
        for (int o = 0; o < 8; ++o)
          *(float4*)(Mx + (o < 4 ? 4 * P + o : 4 * Q + o - 4) * sp) =
              make_float4(acc[o][0], acc[o][1], acc[o][2], acc[o][3]);
      }
      __syncthreads();
      // columns: B[quad, S_b] <- B[quad, S_b] U_b; the superblock from its warp
#pragma unroll
      for (int i = 0; i < EJ4_TPT; ++i) {
        if (ct[i] < 0) break;
        const int b = ct[i] & 0xff, rq = ct[i] >> 8;
        if (!rotf[b]) continue;  // U_b = I and the superblock is unchanged
        const int P = pq[b] & 0xffff, Q = pq[b] >> 16;
        const float* Sb = SC + b * EJ_SUB;
        float* row0 = B + 4 * rq * sp;
        if (rq == P || rq == Q) {
          const int l0 = rq == P ? 0 : 4;
#pragma unroll
          for (int ii = 0; ii < 4; ++ii) {
            *(float4*)(row0 + ii * sp + 4 * P) = *(const float4*)(Sb + (l0 + ii) * 8);
            *(float4*)(row0 + ii * sp + 4 * Q) = *(const float4*)(Sb + (l0 + ii) * 8 + 4);
          }
        } else {
          float w[4][8];
#pragma unroll
          for (int ii = 0; ii < 4; ++ii) {
            const float4 w0 = *(const float4*)(row0 + ii * sp + 4 * P), w1 = *(const float4*)(row0 + ii * sp + 4 * Q);
            w[ii][0] = w0.x;
            w[ii][1] = w0.y;
            w[ii][2] = w0.z;
            w[ii][3] = w0.w;
            w[ii][4] = w1.x;
            w[ii][5] = w1.y;
            w[ii][6] = w1.z;
            w[ii][7] = w1.w;
          }
          const float* Ub = Sb + 64;
          float o[4][8];
#pragma unroll
          for (int ii = 0; ii < 4; ++ii)
#pragma unroll
            for (int j = 0; j < 8; ++j) o[ii][j] = 0.f;
#pragma unroll
          for (int kk = 0; kk < 8; ++kk) {
            const float4 ua = *(const float4*)(Ub + kk * 8), uc = *(const float4*)(Ub + kk * 8 + 4);
            const float u[8] = {ua.x, ua.y, ua.z, ua.w, uc.x, uc.y, uc.z, uc.w};
#pragma unroll
            for (int ii = 0; ii < 4; ++ii)
#pragma unroll
              for (int j = 0; j < 8; ++j) o[ii][j] = fmaf(w[ii][kk], u[j], o[ii][j]);
          }
#pragma unroll
          for (int ii = 0; ii < 4; ++ii) {
            *(float4*)(row0 + ii * sp + 4 * P) = make_float4(o[ii][0], o[ii][1], o[ii][2], o[ii][3]);
            *(float4*)(row0 + ii * sp + 4 * Q) = make_float4(o[ii][4], o[ii][5], o[ii][6], o[ii][7]);
          }
        }
      }
      __syncthreads();
    }
    unsigned cn = 0, mx = 0;
    for (int w = 0; w < min(nsub2, nwarp); ++w) {
      cn += wrot[w];
      mx = max(mx, wmu[w]);
    }
    converged = (cn == 0) || (__uint_as_float(mx) < tol);
  }
  for (int j = tid; j < s; j += nt) Phi[j] = B[j * sp + j];
  __syncthreads();
  if (tid == 0) {
    float mn = Phi[0];
    for (int j = 1; j < s; ++j) mn = fminf(mn, Phi[j]);
    if (!((double)mn + tmin > 0.0)) atomicCAS(status, FCTN_OK, FCTN_E_SINGULAR);
    *nrounds = nround;
    if (sweeps_used) *sweeps_used = converged ? sweep : -sweep;
  }
}

// C = V J_1 J_2 ... J_n (n = *nrounds): row r of V (or of I when V is null)
// meets every recorded round's blocks in order.  A warp holds one row in
// shared memory and its lanes take the round's recorded blocks; the CTA
// stages each round's blocks once for its eight rows, the next round's
// blocks loaded into registers while the current round is applied.
__global__ void __launch_bounds__(256) k_eig_apply(const float* __restrict__ V, const float* __restrict__ Urec,
                                                   const int* __restrict__ PQrec, const int* __restrict__ RoundStart,
                                                   const int* __restrict__ nrounds, float* __restrict__ C, int s) {
  constexpr int MAXB = EIG4_MAX / 8;
  __shared__ float row[8][EIG4_MAX + 4];
  __shared__ float Us[2][MAXB][65];  // stride 65: lanes on different blocks hit different banks
  __shared__ int pqs[2][MAXB];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m = (s + 7) & ~7;
  const int r = blockIdx.x * 8 + warp;
  for (int j = lane; j < m; j += 32)
    row[warp][j] = (r < s && j < s) ? (V ? V[(int64_t)r * s + j] : (j == r ? 1.f : 0.f)) : 0.f;
  const int n = *nrounds;
  // register staging of one round: up to MAXB * 64 floats over 256 threads
  constexpr int PER = (MAXB * 64 + 255) / 256;
  float stage[PER];
  int sp_cnt = 0, sp_pq = 0;
  auto fetch = [&](int q) {
    const int b = RoundStart[q], cnt = RoundStart[q + 1] - b;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int e = threadIdx.x + 256 * i;
      stage[i] = e < cnt * 64 ? Urec[(int64_t)b * 64 + e] : 0.f;
    }
    sp_cnt = cnt;
    sp_pq = threadIdx.x < cnt ? PQrec[b + threadIdx.x] : 0;
  };
  if (n > 0) fetch(0);
  for (int q = 0; q < n; ++q) {
    const int buf = q & 1, cnt = sp_cnt;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int e = threadIdx.x + 256 * i;
      if (e < cnt * 64) Us[buf][e >> 6][e & 63] = stage[i];
    }
    if (threadIdx.x < cnt) pqs[buf][threadIdx.x] = sp_pq;
    __syncthreads();
    if (q + 1 < n) fetch(q + 1);  // in flight while this round is applied
    for (int a = lane; a < cnt; a += 32) {
      const int P = pqs[buf][a] & 0xffff, Q = pqs[buf][a] >> 16;
      float x[8], y[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) x[i] = row[warp][i < 4 ? 4 * P + i : 4 * Q + i - 4];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float acc = 0.f;
#pragma unroll
        for (int i = 0; i < 8; ++i) acc = fmaf(x[i], Us[buf][a][i * 8 + j], acc);
        y[j] = acc;
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) row[warp][j < 4 ? 4 * P + j : 4 * Q + j - 4] = y[j];
    }
    __syncwarp();
  }
  if (r < s)
    for (int j = lane; j < s; j += 32) C[(int64_t)r * s + j] = row[warp][j];
}

// X = I + first-order eigenvector correction of a nearly diagonal symmetric B:
// X_pq = B_pq / (B_qq - B_pp) for p != q when the gap exceeds 8 |B_pq|, else
// 0.  V X holds columns v_q + sum_p X_pq v_p, which after re-orthonormalising
// leave off-diagonal entries of order B_pq^2 / gap; close pairs are left to
// Jacobi.  X is antisymmetric off the diagonal, so (V X)^T (V X) = I + X^T X;
// when ||X||_F > 1/4 the step is dropped (X = I), since one Newton-Schulz
// step then no longer restores orthonormality to working precision.  One CTA.
__global__ void __launch_bounds__(1024) k_first_order(const float* __restrict__ B, float* __restrict__ X, int s) {
  __shared__ float red[32];
  const int64_t n = (int64_t)s * s;
  float ss = 0.f;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
    const int p = (int)(e / s), q = (int)(e - (int64_t)p * s);
    float v = 1.f;
    if (p != q) {
      const float bpq = 0.5f * (B[e] + B[(int64_t)q * s + p]);
      const float gap = B[(int64_t)q * s + q] - B[(int64_t)p * s + p];
      v = fabsf(gap) > 8.f * fabsf(bpq) ? bpq / gap : 0.f;
      ss = fmaf(v, v, ss);
    }
    X[e] = v;
  }
  ss = warp_sum(ss);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x < 32) {
    float t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    t = warp_sum(t);
    if (threadIdx.x == 0) red[0] = t;
  }
  __syncthreads();
  if (red[0] > 1.f / 16.f)
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
      const int p = (int)(e / s), q = (int)(e - (int64_t)p * s);
      X[e] = p == q ? 1.f : 0.f;
    }
}

size_t eig4_smem(int s) {
  const int m = (s + 7) & ~7, sp = m + 4;
  return (size_t)(m * sp + (m / 8 + 1) * EJ_SUB) * sizeof(float);
}

size_t eig3_smem(int s) {
  const int m = (s + 7) & ~7, sp = m + 4;
  return (size_t)(3 * m * sp + (m / 8 + 1) * EJ_SUB) * sizeof(float);
}


struct EigCfg {
  int a_smem, v_smem;
  size_t bytes;
};

EigCfg eig_cfg(int s, int elem) {
  const size_t lim = 220 * 1024;
  const size_t mat = (size_t)s * s * elem;
  if (2 * mat <= lim) return {1, 1, 2 * mat};
  if (mat <= lim) return {1, 0, mat};
  return {0, 0, 0};
}

// FP32 Grams with 128 < s <= 224: warm-start products (4 multi-CTA launches),
// k_eig4, k_eig_apply.  work: 4 s^2 floats; rec: eig_record_floats(s) floats.
struct BigRec {
  float* Urec;
  int *PQrec, *RoundStart, *nr;
};
BigRec big_rec(float* rec, int s) {
  const int m = (s + 7) & ~7, nsub = m / 8, rounds = EIG4_REC_SWEEPS * (m / 4 - 1);
  BigRec b;
  b.Urec = rec;
  b.PQrec = (int*)(rec + (int64_t)rounds * nsub * 64);
  b.RoundStart = b.PQrec + rounds * nsub;
  b.nr = b.RoundStart + rounds + 1;
  return b;
}

}  // namespace

// Warm-start products of the large eigensolver (work: W, V, T, B of s^2 each).
void launch_eig_big_prep(const float* G, const float* C, float* work, int s, cudaStream_t st) {
  const int64_t ss = (int64_t)s * s;
  float *W = work, *V = work + ss, *T = work + 2 * ss, *B = work + 3 * ss;
  const dim3 g2((s + 31) / 32, (s + 31) / 32);
  k_mm_small<true><<<g2, 256, 0, st>>>(C, C, nullptr, W, s, 1.f, 0.f);    // W = V0^T V0
  k_mm_small<false><<<g2, 256, 0, st>>>(C, W, C, V, s, -0.5f, 1.5f);      // V = 1.5 V0 - 0.5 V0 W
  k_mm_small<false><<<g2, 256, 0, st>>>(G, V, nullptr, T, s, 1.f, 0.f);   // T = G V
  k_mm_small<true><<<g2, 256, 0, st>>>(V, T, nullptr, B, s, 1.f, 0.f);    // B = V^T T
}
int eig_big_prep_launches() { return 4; }

// The Jacobi sweeps on one cluster of 8 CTAs (kernels_eigc.cu): B from the
// warm-start products (V among them), or G and the identity cold.
void launch_eig_big_jacobi(const float* G, float* C, float* Phi, float* work, int s, int warm, int max_sweeps,
                           double tmin, double tol, int* status, int* used, cudaStream_t st) {
  const int64_t ss = (int64_t)s * s;
  launch_eigc(warm ? work + 3 * ss : G, warm ? work + ss : nullptr, Phi, C, s, max_sweeps, tmin, tol, status, used,
              st);
}

bool eig_is_big(int s) { return s > EIGC_MIN && s <= EIGC_MAX; }

namespace {

void eig_big(const float* G, float* C, float* Phi, float* work, int s, int warm, int max_sweeps, double tmin,
             double tol, int* status, int* used, cudaStream_t st) {
  if (warm) launch_eig_big_prep(G, C, work, s, st);
  launch_eig_big_jacobi(G, C, Phi, work, s, warm, max_sweeps, tmin, tol, status, used, st);
}

template <typename T>
void eig(const T* G, T* C, T* Phi, T* work, int s, int warm, int max_sweeps, double tmin, int* status, int* used,
         cudaStream_t st, double tol = 0.0) {
  if (sizeof(T) == 4 && s <= EIG3_MAX) {
    const int m = (s + 7) & ~7, nsub = m / 8;
    // one warp per subproblem; one thread per row task up to EJ_NT
    const int threads = std::min(EJ_NT, std::max({64, 32 * nsub, ((m * m / 16 + 31) / 32) * 32}));
    const size_t bytes = eig3_smem(s);
    static bool attr3 = false;
    if (!attr3) {
      cudaFuncSetAttribute(k_eig3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)eig3_smem(EIG3_MAX));
      attr3 = true;
    }
    k_eig3<<<1, threads, bytes, st>>>((const float*)G, (float*)C, (float*)Phi, s, warm, max_sweeps, tmin, tol, status,
                                       used);
    return;
  }
  EigCfg cfg = eig_cfg(s, (int)sizeof(T));
  int npair = (s + (s & 1)) / 2;
  int threads = ((npair * EG + 31) / 32) * 32;
  if (threads < 64) threads = 64;
  if (threads > 1024) threads = 1024;
  static bool attr_set[2] = {false, false};
  if (!attr_set[sizeof(T) == 8]) {
    cudaFuncSetAttribute(k_eig1<T, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    cudaFuncSetAttribute(k_eig1<T, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    attr_set[sizeof(T) == 8] = true;
  }
  if (cfg.a_smem && cfg.v_smem)
    k_eig1<T, true, true><<<1, threads, cfg.bytes, st>>>(G, C, Phi, work, s, warm, max_sweeps, tmin, status, used);
  else if (cfg.a_smem)
    k_eig1<T, true, false><<<1, threads, cfg.bytes, st>>>(G, C, Phi, work, s, warm, max_sweeps, tmin, status, used);
  else
    k_eig1<T, false, false><<<1, threads, cfg.bytes, st>>>(G, C, Phi, work, s, warm, max_sweeps, tmin, status, used);
}

// ------------------------------------------------------------- solve ----
// Eq. 8 with the eigenbasis Q of L_k (I x I row-major, column i =
// eigenvector i; QT = Q^T) and the eigenvectors C of the Gram (s x s,
// column j), in two kernels over blocks of TI factor rows:
//   k_solve_fwd:  P = Q^T R, Z = (P C) / (lam Lambda_i + Phi_j + rho), W = Z C^T
//   k_solve_bwd:  A = Q W into the FP64 master (stored or added) and the
//                 compute copy, optionally with the FP64 residual of Eq. 5.
// The operand that every block needs whole (R or W, I x s) is staged in
// shared memory in chunks of NC rows by the bulk-copy engine; the sum over
// the I rows is split over KS thread groups and combined in a fixed order.
constexpr int SOLVE_NT = 512;

// One bulk copy global -> shared by the TMA engine (cp.async.bulk), completed
// on an mbarrier by transaction bytes; thread 0 issues, every thread waits
// (bounded: on expiry *status gets FCTN_E_TIMEOUT and the caller's loop
// continues with whatever landed).  Needs 16-byte aligned addresses and a
// size that is a multiple of 16.
__device__ __forceinline__ unsigned su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, uint64_t* bar, unsigned phase,
                                          int* status) {
  if (threadIdx.x == 0) {
    // order the block's earlier generic-proxy accesses of dst before the async-proxy write
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(su32(bar)), "r"(bytes));
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(su32(dst)),
        "l"(src), "r"(bytes), "r"(su32(bar))
        : "memory");
  }
  bool ok = false;
  for (long long it = 0; it < (1ll << 26) && !ok; ++it) {
    unsigned r;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(r)
        : "r"(su32(bar)), "r"(phase));
    ok = r != 0;
  }
  if (!ok && threadIdx.x == 0) atomicCAS(status, FCTN_OK, FCTN_E_TIMEOUT);
}

__device__ __forceinline__ bool aligned16(const void* p, size_t bytes) {
  return ((uintptr_t)p % 16 == 0) && (bytes % 16 == 0);
}

// Copy n contiguous elements global -> shared with several loads in flight.
template <typename T>
__device__ __forceinline__ void stage(T* __restrict__ dst, const T* __restrict__ src, int n) {
  const int tid = threadIdx.x, nt = blockDim.x;
  int e = tid;
  for (; e + 3 * nt < n; e += 4 * nt) {
    T a = src[e], b = src[e + nt], c = src[e + 2 * nt], d = src[e + 3 * nt];
    dst[e] = a;
    dst[e + nt] = b;
    dst[e + 2 * nt] = c;
    dst[e + 3 * nt] = d;
  }
  for (; e < n; e += nt) dst[e] = src[e];
}

// Offsets into dynamic shared memory, 16-byte aligned.
__host__ __device__ inline size_t al16(size_t b) { return (b + 15) & ~(size_t)15; }

template <typename T>
struct FwdLayout {
  size_t rs, qs, part, ps, cs, total;
};
template <typename T>
__host__ __device__ inline FwdLayout<T> fwd_layout(int I, int s, int NC, int TI, int KS, int stageC) {
  FwdLayout<T> L;
  L.rs = 0;
  L.qs = al16(L.rs + (size_t)NC * s * sizeof(T));
  L.part = al16(L.qs + (size_t)TI * I * sizeof(T));
  L.ps = al16(L.part + (size_t)KS * TI * s * sizeof(T));
  L.cs = al16(L.ps + (size_t)TI * s * sizeof(T));
  L.total = al16(L.cs + (stageC ? (size_t)s * (s + 1) * sizeof(T) : 0));
  return L;
}

template <typename T>
struct BwdLayout {
  size_t ws, ad, qs, part, total;
};
template <typename T>
__host__ __device__ inline BwdLayout<T> bwd_layout(int I, int s, int NC, int NR, int KS) {
  BwdLayout<T> L;
  L.ws = 0;
  L.ad = al16(L.ws + (size_t)NC * s * sizeof(T));
  L.qs = al16(L.ad + (size_t)NR * s * sizeof(double));
  L.part = al16(L.qs + (size_t)NR * I * sizeof(T));
  L.total = al16(L.part + (size_t)KS * NR * s * sizeof(T));
  return L;
}

// Stage rows [n0, n0 + nc) of an I x s operand into shared memory: one bulk
// copy when aligned, else plain loads.
template <typename T>
__device__ __forceinline__ void stage_rows(T* dst, const T* src_base, int n0, int nc, int s, uint64_t* bar,
                                           unsigned& phase, int* status) {
  const T* src = src_base + (int64_t)n0 * s;
  const size_t bytes = (size_t)nc * s * sizeof(T);
  if (aligned16(src, bytes) && bytes > 0) {
    bulk_copy(dst, src, (unsigned)bytes, bar, phase, status);
    phase ^= 1u;
  } else {
    stage(dst, src, nc * s);
  }
}

// Partial sums over the rows n = kq, kq + KS, ... of a staged chunk for the
// NR block rows: acc[t] += Qs[t][n0 + n] * Xs[n][j].
template <typename T, int NRMAX>
__device__ __forceinline__ void chunk_product(const T* __restrict__ Qs, int I, const T* __restrict__ Xs, int s,
                                              int n0, int nc, int j, int kq, int KS, int nr, T* acc) {
  int n = kq;
  for (; n + KS < nc; n += 2 * KS) {
    const T x0 = Xs[n * s + j], x1 = Xs[(n + KS) * s + j];
#pragma unroll
    for (int t = 0; t < NRMAX; ++t)
      if (t < nr) acc[t] = fma(Qs[t * I + n0 + n + KS], x1, fma(Qs[t * I + n0 + n], x0, acc[t]));
  }
  if (n < nc) {
    const T x0 = Xs[n * s + j];
#pragma unroll
    for (int t = 0; t < NRMAX; ++t)
      if (t < nr) acc[t] = fma(Qs[t * I + n0 + n], x0, acc[t]);
  }
}

// Forward half of Eq. 8 for factor rows [i0, i0 + TI):
//   P = (Q^T R)[rows], Z = (P C) / (lam Lambda_i + Phi_j + rho), W = Z C^T.
template <typename T, int TI>
__global__ void __launch_bounds__(SOLVE_NT) k_solve_fwd(const T* __restrict__ QT, const T* __restrict__ Rm,
                                                        const T* __restrict__ C, const double* __restrict__ LamL,
                                                        const T* __restrict__ Phi, double lam, double rho, int I,
                                                        int s, int NC, int KS, int stageC, T* __restrict__ W,
                                                        int* status) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ __align__(8) uint64_t bar;
  const FwdLayout<T> L = fwd_layout<T>(I, s, NC, TI, KS, stageC);
  T* Rs = (T*)(sm + L.rs);
  T* Qs = (T*)(sm + L.qs);
  T* part = (T*)(sm + L.part);
  T* Ps = (T*)(sm + L.ps);
  T* Cs = (T*)(sm + L.cs);
  const int tid = threadIdx.x, nt = blockDim.x, i0 = blockIdx.x * TI;
  const int nv = min(TI, I - i0);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
  }
  for (int e = tid; e < TI * I; e += nt) {  // rows of Q^T = columns of Q
    const int r = e / I, n = e % I;
    Qs[e] = r < nv ? QT[(int64_t)(i0 + r) * I + n] : (T)0;
  }
  const int cst = stageC ? s + 1 : s;
  const T* Cp = stageC ? Cs : C;
  if (stageC)
    for (int e = tid; e < s * s; e += nt) Cs[(e / s) * cst + e % s] = C[e];
  // column j of P in thread j mod cols (KS = threads / cols groups split
  // the rows); more than one column group only when s exceeds the threads
  const int cols = min(s, nt), jl = tid % cols, kq = tid / cols;
  const bool act = kq < KS;
  unsigned phase = 0;
  for (int jb = 0; jb < s; jb += cols) {
    const int j = jb + jl;
    T acc[TI];
#pragma unroll
    for (int t = 0; t < TI; ++t) acc[t] = 0;
    for (int n0 = 0; n0 < I; n0 += NC) {
      const int nc = min(NC, I - n0);
      __syncthreads();  // previous chunk consumed; on the first pass, Qs and the barrier init visible
      stage_rows(Rs, Rm, n0, nc, s, &bar, phase, status);
      __syncthreads();
      if (act && j < s) chunk_product<T, TI>(Qs, I, Rs, s, n0, nc, j, kq, KS, TI, acc);
    }
    if (act && j < s)
#pragma unroll
      for (int t = 0; t < TI; ++t) part[(kq * TI + t) * s + j] = acc[t];
  }
  __syncthreads();
  for (int e = tid; e < TI * s; e += nt) {  // fixed-order combine of the KS partial sums
    T v = 0;
    for (int q = 0; q < KS; ++q) v += part[q * TI * s + e];
    Ps[e] = v;
  }
  __syncthreads();
  for (int e = tid; e < TI * s; e += nt) {  // Z = (P C) / T  (into part)
    const int r = e / s, jj = e % s;
    T a0 = 0, a1 = 0;
    int q = 0;
    for (; q + 1 < s; q += 2) {
      a0 = fma(Ps[r * s + q], Cp[q * cst + jj], a0);
      a1 = fma(Ps[r * s + q + 1], Cp[(q + 1) * cst + jj], a1);
    }
    if (q < s) a0 = fma(Ps[r * s + q], Cp[q * cst + jj], a0);
    const double tt = r < nv ? lam * LamL[i0 + r] + (double)Phi[jj] + rho : 1.0;
    part[e] = (T)((double)(a0 + a1) / tt);
  }
  __syncthreads();
  for (int e = tid; e < nv * s; e += nt) {  // W = Z C^T
    const int r = e / s, jj = e % s;
    T a0 = 0, a1 = 0;
    int q = 0;
    for (; q + 1 < s; q += 2) {
      a0 = fma(part[r * s + q], Cp[jj * cst + q], a0);
      a1 = fma(part[r * s + q + 1], Cp[jj * cst + q + 1], a1);
    }
    if (q < s) a0 = fma(part[r * s + q], Cp[jj * cst + q], a0);
    W[(int64_t)(i0 + r) * s + jj] = a0 + a1;
  }
}

// Backward half of Eq. 8 for factor rows [i0, i0 + TI): A = (Q W)[rows],
// stored to (accumulate = 0) or added to (accumulate = 1) the FP64 master,
// and to the compute copy.  With Rout (accumulate = 0 only), also the FP64
// residual of Eq. 5 for these rows, R = Y - lam L A - rho A - A G; the block
// then also forms A for the cyclic neighbour rows i0 - 1 and i0 + nv (slot
// t holds row (i0 - 1 + t) mod I), with the same arithmetic as the blocks
// that own them.
template <typename T, typename Tc, int TI>
__global__ void __launch_bounds__(SOLVE_NT) k_solve_bwd(const T* __restrict__ Q, const T* __restrict__ Wm, int I,
                                                        int s, int NC, int KS, int accumulate,
                                                        double* __restrict__ A64, Tc* __restrict__ Ac,
                                                        const double* __restrict__ Yd,
                                                        const double* __restrict__ Gd, double lam, double rho,
                                                        double c0, double c1, T* __restrict__ Rout, int* status) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ __align__(8) uint64_t bar;
  constexpr int NRMAX = TI + 2;
  const BwdLayout<T> L = bwd_layout<T>(I, s, NC, NRMAX, KS);
  T* Ws = (T*)(sm + L.ws);
  double* Ad = (double*)(sm + L.ad);
  T* Qs = (T*)(sm + L.qs);
  T* part = (T*)(sm + L.part);
  const int tid = threadIdx.x, nt = blockDim.x, i0 = blockIdx.x * TI;
  const int nv = min(TI, I - i0);
  const bool res = Rout != nullptr;
  const int nr = res ? nv + 2 : nv, off = res ? 1 : 0;  // slot t <-> row (i0 - off + t) mod I
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
  }
  for (int e = tid; e < nr * I; e += nt) {
    const int t = e / I, n = e % I;
    const int row = (i0 - off + t + I) % I;
    Qs[e] = Q[(int64_t)row * I + n];
  }
  const int cols = min(s, nt), jl = tid % cols, kq = tid / cols;  // as in k_solve_fwd
  const bool act = kq < KS;
  unsigned phase = 0;
  for (int jb = 0; jb < s; jb += cols) {
    const int j = jb + jl;
    T acc[NRMAX];
#pragma unroll
    for (int t = 0; t < NRMAX; ++t) acc[t] = 0;
    for (int n0 = 0; n0 < I; n0 += NC) {
      const int nc = min(NC, I - n0);
      __syncthreads();
      stage_rows(Ws, Wm, n0, nc, s, &bar, phase, status);
      __syncthreads();
      if (act && j < s) chunk_product<T, NRMAX>(Qs, I, Ws, s, n0, nc, j, kq, KS, nr, acc);
    }
    if (act && j < s)
#pragma unroll
      for (int t = 0; t < NRMAX; ++t)
        if (t < nr) part[(kq * NRMAX + t) * s + j] = acc[t];
  }
  __syncthreads();
  for (int e = tid; e < nr * s; e += nt) {
    const int t = e / s, jj = e % s;
    T v = 0;
    for (int q = 0; q < KS; ++q) v += part[(q * NRMAX + t) * s + jj];
    const int row = (i0 - off + t + I) % I;
    const int64_t o = (int64_t)row * s + jj;
    const double a = accumulate ? A64[o] + (double)v : (double)v;
    Ad[e] = a;
    if (t >= off && t < off + nv) {
      A64[o] = a;
      Ac[o] = (Tc)a;
    }
  }
  if (!res) return;
  __syncthreads();
  if (s <= nt && nv * KS * s * (int)sizeof(double) <= KS * NRMAX * s * (int)sizeof(T)) {
    // (A G)[r][jj] split over the KS thread groups (q = g, g + KS, ...), the
    // partial sums combined in group order; G staged in shared memory (in
    // the W staging area, free now) when it fits there
    const bool gsm = (size_t)s * s * sizeof(double) <= L.ad - L.ws;
    double* Gs = (double*)(sm + L.ws);
    if (gsm) {
      for (int e = tid; e < s * s; e += nt) Gs[e] = Gd[e];
      __syncthreads();
    }
    const double* Gp = gsm ? Gs : Gd;
    double* pr = (double*)(sm + L.part);  // [KS][nv][s]
    const int jj = tid % s, g = tid / s;
    if (g < KS)
      for (int r = 0; r < nv; ++r) {
        const int t = r + 1;
        double acc = 0.0;
        for (int q = g; q < s; q += KS) acc = fma(Ad[t * s + q], Gp[(int64_t)q * s + jj], acc);
        pr[(g * nv + r) * s + jj] = acc;
      }
    __syncthreads();
    for (int e = tid; e < nv * s; e += nt) {
      const int r = e / s, jc = e % s, t = r + 1;
      const int64_t o = (int64_t)(i0 + r) * s + jc;
      double ag = 0.0;
      for (int gg = 0; gg < KS; ++gg) ag += pr[(gg * nv + r) * s + jc];
      const double a = Ad[t * s + jc];
      const double la = c0 * a + c1 * (Ad[(t - 1) * s + jc] + Ad[(t + 1) * s + jc]);
      Rout[o] = (T)(Yd[o] - lam * la - rho * a - ag);
    }
    return;
  }
  for (int e = tid; e < nv * s; e += nt) {  // s above the block: one thread per output
    const int r = e / s, jj = e % s, t = r + 1;
    const int64_t o = (int64_t)(i0 + r) * s + jj;
    double g0 = 0.0, g1 = 0.0;
    int q = 0;
    for (; q + 1 < s; q += 2) {
      g0 = fma(Ad[t * s + q], Gd[(int64_t)q * s + jj], g0);
      g1 = fma(Ad[t * s + q + 1], Gd[(int64_t)(q + 1) * s + jj], g1);
    }
    if (q < s) g0 = fma(Ad[t * s + q], Gd[(int64_t)q * s + jj], g0);
    const double a = Ad[t * s + jj];
    const double la = c0 * a + c1 * (Ad[(t - 1) * s + jj] + Ad[(t + 1) * s + jj]);
    Rout[o] = (T)(Yd[o] - lam * la - rho * a - (g0 + g1));
  }
}

template <typename T>
struct SolveCfg {
  int TI, KS, NC, stageC;
  size_t bytes;
};

// Row-block size, K split and chunk of staged rows for the two solve kernels.
template <typename T>
SolveCfg<T> solve_cfg(int I, int s, bool bwd, bool res) {
  SolveCfg<T> c;
  c.TI = 1;  // one factor row per CTA: measured faster than two; more CTAs outweigh the extra halo rows
  c.KS = std::max(1, SOLVE_NT / s);
  c.stageC = (!bwd && (size_t)s * (s + 1) * sizeof(T) <= 40 * 1024) ? 1 : 0;
  const size_t budget = 160 * 1024;
  size_t fixed = bwd ? bwd_layout<T>(I, s, 0, c.TI + 2, c.KS).total : fwd_layout<T>(I, s, 0, c.TI, c.KS, c.stageC).total;
  const size_t per = (size_t)s * sizeof(T);
  long nc = budget > fixed + 32 ? (long)((budget - fixed - 32) / per) : 1;
  nc = std::max(1L, std::min<long>(nc, I));
  c.NC = (int)nc;
  c.bytes = bwd ? bwd_layout<T>(I, s, c.NC, c.TI + 2, c.KS).total : fwd_layout<T>(I, s, c.NC, c.TI, c.KS, c.stageC).total;
  (void)res;
  return c;
}

template <typename T>
void solve_fwd(const T* QT, const T* R, const T* C, const double* LamL, const T* Phi, double lam, double rho, int I,
               int s, T* W, int* status, cudaStream_t st) {
  SolveCfg<T> c = solve_cfg<T>(I, s, false, false);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_solve_fwd<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  const int grid = (I + c.TI - 1) / c.TI;
  k_solve_fwd<T, 1><<<grid, SOLVE_NT, c.bytes, st>>>(QT, R, C, LamL, Phi, lam, rho, I, s, c.NC, c.KS, c.stageC, W,
                                                      status);
}

template <typename T, typename Tc>
void solve_bwd(const T* Q, const T* W, int I, int s, int accumulate, double* A64, Tc* Ac, const double* Yd,
               const double* Gd, double lam, double rho, double c0, double c1, T* Rout, int* status,
               cudaStream_t st) {
  SolveCfg<T> c = solve_cfg<T>(I, s, true, Rout != nullptr);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_solve_bwd<T, Tc, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  const int grid = (I + c.TI - 1) / c.TI;
  k_solve_bwd<T, Tc, 1><<<grid, SOLVE_NT, c.bytes, st>>>(Q, W, I, s, c.NC, c.KS, accumulate, A64, Ac, Yd, Gd, lam,
                                                          rho, c0, c1, Rout, status);
}

// FP64 residual of Eq. 5, one CTA per row: R = Y - lam L A - rho A - A G.
template <typename Tout>
__global__ void __launch_bounds__(128) k_resid(const double* __restrict__ Y, const double* __restrict__ A,
                                               const double* __restrict__ G, int I, int s, double lam, double rho,
                                               double c0, double c1, Tout* __restrict__ R) {
  const int i = blockIdx.x;
  const int ip = (i + 1) % I, im = (i - 1 + I) % I;
  for (int j = threadIdx.x; j < s; j += blockDim.x) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int q = 0;
    for (; q + 3 < s; q += 4) {
      a0 = fma(A[(int64_t)i * s + q], G[(int64_t)q * s + j], a0);
      a1 = fma(A[(int64_t)i * s + q + 1], G[(int64_t)(q + 1) * s + j], a1);
      a2 = fma(A[(int64_t)i * s + q + 2], G[(int64_t)(q + 2) * s + j], a2);
      a3 = fma(A[(int64_t)i * s + q + 3], G[(int64_t)(q + 3) * s + j], a3);
    }
    for (; q < s; ++q) a0 = fma(A[(int64_t)i * s + q], G[(int64_t)q * s + j], a0);
    double acc = (a0 + a1) + (a2 + a3);
    int64_t o = (int64_t)i * s + j;
    double a = A[o];
    double la = c0 * a + c1 * (A[(int64_t)ip * s + j] + A[(int64_t)im * s + j]);
    R[o] = (Tout)(Y[o] - lam * la - rho * a - acc);
  }
}

// Asymmetric extrapolation (Sec. 4.3): A <- A + alpha (A - beta A_old), FP64
// master and compute copy.
template <typename Tc>
__global__ void k_extrap(double* __restrict__ A, const double* __restrict__ Aold, double alpha, double beta,
                         Tc* __restrict__ Ac, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double a = A[e];
    a += alpha * (a - beta * Aold[e]);
    A[e] = a;
    Ac[e] = (Tc)a;
  }
}

// lam/2 * tr(A^T L A) partial sums; L is the cyclic stencil (c0 on the
// diagonal, c1 on both neighbours, coinciding entries summed).
constexpr int TRACE_BLOCKS = 32;

// The trace terms of every factor in one launch: block (b, k) sums rows
// b, b + TRACE_BLOCKS, ... of factor k (threads over the columns).
__global__ void k_trace_all(TraceArgs a, double* __restrict__ out) {
  pdl_prologue();
  __shared__ double red[32];
  const int k = blockIdx.y;
  const double* A = a.A[k];
  const int64_t I = a.I[k], s = a.s[k];
  double acc = 0.0;
  for (int64_t i = blockIdx.x; i < I; i += gridDim.x) {
    const int64_t ip = (i + 1) % I, im = (i - 1 + I) % I;
    for (int64_t j = threadIdx.x; j < s; j += blockDim.x) {
      const double v = A[i * s + j];
      acc += v * (a.c0[k] * v + a.c1[k] * (A[ip * s + j] + A[im * s + j]));
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[k * gridDim.x + blockIdx.x] = 0.5 * a.lam[k] * t;
  }
}

__global__ void k_finalize(const double* __restrict__ red, int nblocks, const double* __restrict__ traces, int N,
                           double* __restrict__ stats) {
  pdl_prologue();
  __shared__ double sh[3][256];
  double v[3] = {0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    v[0] += red[b * 3 + 0];
    v[1] += red[b * 3 + 1];
    v[2] += red[b * 3 + 2];
  }
  for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] = v[q];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double tr = 0.0;
    for (int i = 0; i < N * TRACE_BLOCKS; ++i) tr += traces[i];
    double d2 = sh[0][0], x2 = sh[1][0], r2 = sh[2][0];
    stats[0] = sqrt(d2) / sqrt(x2);
    stats[2] = 0.5 * r2;
    stats[1] = 0.5 * r2 + tr;
    stats[3] = (isfinite(d2) && isfinite(x2) && isfinite(r2) && isfinite(tr) && isfinite(stats[0])) ? 0.0 : 1.0;
  }
}

}  // namespace

void launch_eig_f32(const float* G, float* C, float* Phi, float* work, int s, int warm, int max_sweeps,
                    double tmin, int* status, int* used, cudaStream_t st, float* rec, double tol) {
  (void)rec;
  if (eig_is_big(s)) {
    eig_big(G, C, Phi, work, s, warm, max_sweeps, tmin, tol, status, used, st);
    return;
  }
  eig<float>(G, C, Phi, work, s, warm, max_sweeps, tmin, status, used, st, tol);
}

size_t eig_record_floats(int s) {
  if (eig_is_big(s) || s <= EIG3_MAX || s > EIG4_MAX) return 0;  // the cluster Jacobi keeps V on chip
  const int m = (s + 7) & ~7, nsub = m / 8, rounds = EIG4_REC_SWEEPS * (m / 4 - 1);
  return (size_t)rounds * nsub * 64 + (size_t)rounds * nsub + rounds + 18;  // blocks, pairs, round starts, count
}
int eig_launches(int s, int warm, int recorded) {
  (void)recorded;
  if (eig_is_big(s)) return warm ? 5 : 1;  // warm-start products (4), cluster Jacobi
  return 1;
}
void launch_eig_f64(const double* G, double* C, double* Phi, double* work, int s, int warm, int max_sweeps,
                    double tmin, int* status, int* used, cudaStream_t st) {
  eig<double>(G, C, Phi, work, s, warm, max_sweeps, tmin, status, used, st);
}
void launch_solve_fwd_f32(const float* QT, const float* R, const float* C, const double* LamL, const float* Phi,
                          double lam, double rho, int I, int s, float* W, int* status, cudaStream_t st) {
  solve_fwd<float>(QT, R, C, LamL, Phi, lam, rho, I, s, W, status, st);
}
void launch_solve_fwd_f64(const double* QT, const double* R, const double* C, const double* LamL, const double* Phi,
                          double lam, double rho, int I, int s, double* W, int* status, cudaStream_t st) {
  solve_fwd<double>(QT, R, C, LamL, Phi, lam, rho, I, s, W, status, st);
}
void launch_solve_bwd_f32(const float* Q, const float* W, int I, int s, int accumulate, double* A64, float* Ac,
                          const double* Yd, const double* Gd, double lam, double rho, double c0, double c1, float* Rout,
                          int* status, cudaStream_t st) {
  solve_bwd<float, float>(Q, W, I, s, accumulate, A64, Ac, Yd, Gd, lam, rho, c0, c1, Rout, status, st);
}
void launch_solve_bwd_f64(const double* Q, const double* W, int I, int s, int accumulate, double* A64, double* Ac,
                          const double* Yd, const double* Gd, double lam, double rho, double c0, double c1,
                          double* Rout, int* status, cudaStream_t st) {
  solve_bwd<double, double>(Q, W, I, s, accumulate, A64, Ac, Yd, Gd, lam, rho, c0, c1, Rout, status, st);
}
void launch_resid_f32(const double* Y, const double* A, const double* G, int I, int s, double lam, double rho,
                      double c0, double c1, float* R, cudaStream_t st) {
  k_resid<float><<<I, 128, 0, st>>>(Y, A, G, I, s, lam, rho, c0, c1, R);
}
void launch_resid_f64(const double* Y, const double* A, const double* G, int I, int s, double lam, double rho,
                      double c0, double c1, double* R, cudaStream_t st) {
  k_resid<double><<<I, 128, 0, st>>>(Y, A, G, I, s, lam, rho, c0, c1, R);
}
void launch_trace_all(const TraceArgs& a, int N, double* out, cudaStream_t st) {
  launch_pdl(k_trace_all, dim3(TRACE_BLOCKS, (unsigned)N), dim3(256), 0, st, a, out);
}
void launch_finalize(const double* red, int nblocks, const double* traces, int N, double* stats, cudaStream_t st) {
  launch_pdl(k_finalize, dim3(1), dim3(256), 0, st, red, nblocks, traces, N, stats);
}

void launch_extrap_f32(double* A, const double* Aold, double alpha, double beta, float* Ac, int64_t n,
                       cudaStream_t st) {
  k_extrap<float><<<(unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024), 256, 0, st>>>(A, Aold, alpha, beta,
                                                                                            Ac, n);
}
void launch_extrap_f64(double* A, const double* Aold, double alpha, double beta, double* Ac, int64_t n,
                       cudaStream_t st) {
  k_extrap<double><<<(unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024), 256, 0, st>>>(A, Aold, alpha,
                                                                                             beta, Ac, n);
}
