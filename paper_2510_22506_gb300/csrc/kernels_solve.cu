// Factor solve of Eqs. 5-8: the symmetric eigendecomposition of the Gram
// (one-sided Jacobi), the eigen-route solve with its FP64 refinement, and the
// reductions of the objective (Eq. 2) and the stop test.
#include <float.h>

#include "fctn_internal.cuh"

namespace {

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
// The sweep limit is not an error: *sweeps_used then equals max_sweeps.
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
__device__ __forceinline__ void rot_cs(float al, float be, float ga, float& cs, float& sn) {
  float zeta = __fdividef(be - al, 2.f * ga);
  float w = fmaf(zeta, zeta, 1.f);
  float sq = w * rsqrtf(w);
  float t = __fdividef(zeta >= 0.f ? 1.f : -1.f, fabsf(zeta) + sq);
  float x = fmaf(t, t, 1.f);
  float y = rsqrtf(x);
  cs = y * fmaf(-0.5f * x * y, y, 1.5f);  // one Newton step: c^2 (1 + t^2) = 1 to about an ulp
  sn = cs * t;
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
    // The sweep count is reported (== max_sweeps) rather than failing.
    if (sweeps_used) *sweeps_used = converged ? sweep : max_sweeps;
  }
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

template <typename T>
void eig(const T* G, T* C, T* Phi, T* work, int s, int warm, int max_sweeps, double tmin, int* status, int* used,
         cudaStream_t st) {
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
// Eq. 8 in two row-block kernels (Q: real eigenbasis of L_k, I x I row-major,
// column i = eigenvector i; C: eigenvectors of G, s x s, column j):
//   solve_a:  Z[i,:] = ((Q^T R)[i,:] C) / (lam Lambda_i + Phi_j + rho)
//   solve_b:  A[i,:] = (Q[i,:] Z) C^T, written to the FP64 master (or added
//             to it, for a refinement pass) and to the compute copy.
constexpr int SB = 8;  // rows per CTA

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

// Row chunks of R (NC x s) and the matching slice of Q are staged in shared
// memory; each thread owns fixed entries of the SB x s block, accumulated over
// the chunks in a fixed order.
template <typename T>
__global__ void __launch_bounds__(256) k_solve_a(const T* __restrict__ Q, const T* __restrict__ Rm,
                                                 const T* __restrict__ C, const double* __restrict__ LamL,
                                                 const T* __restrict__ Phi, double lam, double rho, int I, int s,
                                                 int NC, T* __restrict__ Z, int* status) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ __align__(8) uint64_t bar;
  T* Rs = (T*)sm;                  // NC x s (first: 16-byte aligned for the bulk copy)
  T* W = Rs + (size_t)NC * s;      // SB x s
  T* Qs = W + (size_t)SB * s;      // NC x SB  (Qs[n][r] = Q[n0 + n][i0 + r])
  const int i0 = blockIdx.x * SB;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
  }
  for (int e = tid; e < SB * s; e += nt) W[e] = 0;
  unsigned phase = 0;
  for (int n0 = 0; n0 < I; n0 += NC) {
    const int nc = min(NC, I - n0);
    __syncthreads();
    const T* src = Rm + (int64_t)n0 * s;
    const size_t bytes = (size_t)nc * s * sizeof(T);
    if (aligned16(src, bytes)) {
      bulk_copy(Rs, src, (unsigned)bytes, &bar, phase, status);
      phase ^= 1u;
    } else {
      stage(Rs, src, nc * s);
    }
    for (int e = tid; e < nc * SB; e += nt) {
      int n = e / SB, r = e % SB;
      Qs[e] = (i0 + r < I) ? Q[(int64_t)(n0 + n) * I + i0 + r] : (T)0;
    }
    __syncthreads();
    for (int e = tid; e < SB * s; e += nt) {
      int r = e / s, j = e % s;
      T a0 = 0, a1 = 0;
      int n = 0;
      for (; n + 1 < nc; n += 2) {
        a0 = fma(Qs[n * SB + r], Rs[n * s + j], a0);
        a1 = fma(Qs[(n + 1) * SB + r], Rs[(n + 1) * s + j], a1);
      }
      if (n < nc) a0 = fma(Qs[n * SB + r], Rs[n * s + j], a0);
      W[e] += a0 + a1;
    }
  }
  __syncthreads();
  for (int e = tid; e < SB * s; e += nt) {
    int r = e / s, j = e % s;
    int i = i0 + r;
    if (i >= I) continue;
    T a0 = 0, a1 = 0;
    int q = 0;
    for (; q + 1 < s; q += 2) {
      a0 = fma(W[r * s + q], C[(int64_t)q * s + j], a0);
      a1 = fma(W[r * s + q + 1], C[(int64_t)(q + 1) * s + j], a1);
    }
    if (q < s) a0 = fma(W[r * s + q], C[(int64_t)q * s + j], a0);
    double t = lam * LamL[i] + (double)Phi[j] + rho;
    Z[(int64_t)i * s + j] = (T)((double)(a0 + a1) / t);
  }
}

template <typename T, typename Tc>
__global__ void __launch_bounds__(256) k_solve_b(const T* __restrict__ Q, const T* __restrict__ Z,
                                                 const T* __restrict__ C, int I, int s, int NC, int accumulate,
                                                 double* __restrict__ A64, Tc* __restrict__ Ac, int* status) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ __align__(8) uint64_t bar;
  T* Zs = (T*)sm;                  // NC x s (first: 16-byte aligned for the bulk copy)
  T* U = Zs + (size_t)NC * s;      // SB x s
  T* Qs = U + (size_t)SB * s;      // SB x NC (Qs[r][n] = Q[i0 + r][n0 + n])
  const int i0 = blockIdx.x * SB;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
  }
  for (int e = tid; e < SB * s; e += nt) U[e] = 0;
  unsigned phase = 0;
  for (int n0 = 0; n0 < I; n0 += NC) {
    const int nc = min(NC, I - n0);
    __syncthreads();
    const T* src = Z + (int64_t)n0 * s;
    const size_t bytes = (size_t)nc * s * sizeof(T);
    if (aligned16(src, bytes)) {
      bulk_copy(Zs, src, (unsigned)bytes, &bar, phase, status);
      phase ^= 1u;
    } else {
      stage(Zs, src, nc * s);
    }
    for (int e = tid; e < SB * nc; e += nt) {
      int r = e / nc, n = e % nc;
      Qs[r * NC + n] = (i0 + r < I) ? Q[(int64_t)(i0 + r) * I + n0 + n] : (T)0;
    }
    __syncthreads();
    for (int e = tid; e < SB * s; e += nt) {
      int r = e / s, j = e % s;
      T a0 = 0, a1 = 0;
      int n = 0;
      for (; n + 1 < nc; n += 2) {
        a0 = fma(Qs[r * NC + n], Zs[n * s + j], a0);
        a1 = fma(Qs[r * NC + n + 1], Zs[(n + 1) * s + j], a1);
      }
      if (n < nc) a0 = fma(Qs[r * NC + n], Zs[n * s + j], a0);
      U[e] += a0 + a1;
    }
  }
  __syncthreads();
  for (int e = tid; e < SB * s; e += nt) {
    int r = e / s, j = e % s;
    int i = i0 + r;
    if (i >= I) continue;
    T a0 = 0, a1 = 0;
    int q = 0;
    for (; q + 1 < s; q += 2) {
      a0 = fma(U[r * s + q], C[(int64_t)j * s + q], a0);
      a1 = fma(U[r * s + q + 1], C[(int64_t)j * s + q + 1], a1);
    }
    if (q < s) a0 = fma(U[r * s + q], C[(int64_t)j * s + q], a0);
    int64_t o = (int64_t)i * s + j;
    double v = accumulate ? A64[o] + (double)(a0 + a1) : (double)(a0 + a1);
    A64[o] = v;
    Ac[o] = (Tc)v;
  }
}

// rows of R / Z staged per chunk so that the staging fits in ~96 KB
int solve_chunk(int I, int s, int elem) {
  size_t budget = 96 * 1024 / elem;
  size_t fixed = (size_t)SB * s;
  size_t per = (size_t)s + SB;
  int nc = (int)((budget > fixed ? budget - fixed : per) / per);
  if (nc < 1) nc = 1;
  return nc < I ? nc : I;
}

size_t solve_smem(int I, int s, int NC, int elem) { return ((size_t)SB * s + (size_t)NC * s + (size_t)NC * SB) * elem; }

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
__global__ void k_trace(const double* __restrict__ A, int64_t I, int64_t s, double c0, double c1, double lam,
                        double* __restrict__ out) {
  __shared__ double red[32];
  double acc = 0.0;
  const int64_t n = I * s;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / s, j = e % s;
    int64_t ip = (i + 1) % I, im = (i - 1 + I) % I;
    double a = A[e];
    acc += a * (c0 * a + c1 * (A[ip * s + j] + A[im * s + j]));
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[blockIdx.x] = 0.5 * lam * t;
  }
}

constexpr int TRACE_BLOCKS = 32;

__global__ void k_finalize(const double* __restrict__ red, int nblocks, const double* __restrict__ traces, int N,
                           double* __restrict__ stats) {
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
                    double tmin, int* status, int* used, cudaStream_t st) {
  eig<float>(G, C, Phi, work, s, warm, max_sweeps, tmin, status, used, st);
}
void launch_eig_f64(const double* G, double* C, double* Phi, double* work, int s, int warm, int max_sweeps,
                    double tmin, int* status, int* used, cudaStream_t st) {
  eig<double>(G, C, Phi, work, s, warm, max_sweeps, tmin, status, used, st);
}
void launch_solve_a_f32(const float* Q, const float* R, const float* C, const double* LamL, const float* Phi,
                        double lam, double rho, int I, int s, float* Z, int* status, cudaStream_t st) {
  int nc = solve_chunk(I, s, sizeof(float));
  size_t sb = solve_smem(I, s, nc, sizeof(float));
  if (sb > 48 * 1024) cudaFuncSetAttribute(k_solve_a<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb);
  k_solve_a<float><<<(I + SB - 1) / SB, 256, sb, st>>>(Q, R, C, LamL, Phi, lam, rho, I, s, nc, Z, status);
}
void launch_solve_a_f64(const double* Q, const double* R, const double* C, const double* LamL, const double* Phi,
                        double lam, double rho, int I, int s, double* Z, int* status, cudaStream_t st) {
  int nc = solve_chunk(I, s, sizeof(double));
  size_t sb = solve_smem(I, s, nc, sizeof(double));
  if (sb > 48 * 1024) cudaFuncSetAttribute(k_solve_a<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb);
  k_solve_a<double><<<(I + SB - 1) / SB, 256, sb, st>>>(Q, R, C, LamL, Phi, lam, rho, I, s, nc, Z, status);
}
void launch_solve_b_f32(const float* Q, const float* Z, const float* C, int I, int s, int accumulate, double* A64,
                        float* Ac, int* status, cudaStream_t st) {
  int nc = solve_chunk(I, s, sizeof(float));
  size_t sb = solve_smem(I, s, nc, sizeof(float));
  if (sb > 48 * 1024)
    cudaFuncSetAttribute(k_solve_b<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb);
  k_solve_b<float, float><<<(I + SB - 1) / SB, 256, sb, st>>>(Q, Z, C, I, s, nc, accumulate, A64, Ac, status);
}
void launch_solve_b_f64(const double* Q, const double* Z, const double* C, int I, int s, int accumulate, double* A64,
                        double* Ac, int* status, cudaStream_t st) {
  int nc = solve_chunk(I, s, sizeof(double));
  size_t sb = solve_smem(I, s, nc, sizeof(double));
  if (sb > 48 * 1024)
    cudaFuncSetAttribute(k_solve_b<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb);
  k_solve_b<double, double><<<(I + SB - 1) / SB, 256, sb, st>>>(Q, Z, C, I, s, nc, accumulate, A64, Ac, status);
}
void launch_resid_f32(const double* Y, const double* A, const double* G, int I, int s, double lam, double rho,
                      double c0, double c1, float* R, cudaStream_t st) {
  k_resid<float><<<I, 128, 0, st>>>(Y, A, G, I, s, lam, rho, c0, c1, R);
}
void launch_resid_f64(const double* Y, const double* A, const double* G, int I, int s, double lam, double rho,
                      double c0, double c1, double* R, cudaStream_t st) {
  k_resid<double><<<I, 128, 0, st>>>(Y, A, G, I, s, lam, rho, c0, c1, R);
}
void launch_trace_term(const double* A, int64_t I, int64_t s, double c0, double c1, double lam, double* out,
                       cudaStream_t st) {
  k_trace<<<TRACE_BLOCKS, 256, 0, st>>>(A, I, s, c0, c1, lam, out);
}
void launch_finalize(const double* red, int nblocks, const double* traces, int N, double* stats, cudaStream_t st) {
  k_finalize<<<1, 256, 0, st>>>(red, nblocks, traces, N, stats);
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
