// Device helpers of the block-ordered Jacobi eigensolvers (kernels_solve.cu,
// kernels_eigc.cu): the round-robin pair schedule, the pairs of the inner
// rounds of one 8 x 8 subproblem, and one inner round with the rotation test
// relative to the shifted diagonal of Eq. 8.
#pragma once

#include <cfloat>

namespace fctn_jacobi {

constexpr int EJ_SUB = 132;  // floats per subproblem: S (8 x 8), U (8 x 8), 4 against bank conflicts

// Pair idx of round `round` of the round-robin schedule over m indices.
__device__ __forceinline__ void round_pair(int m, int round, int idx, int& p, int& q) {
  if (idx == 0) {
    p = m - 1;
    q = round;
  } else {
    p = round + idx;
    if (p >= m - 1) p -= m - 1;
    q = round - idx;
    if (q < 0) q += m - 1;
  }
  if (p > q) {
    int t = p;
    p = q;
    q = t;
  }
}

// Pair k (0-3) of inner round t: within-block rounds t = 0-2 pair (0,1)(2,3),
// (0,2)(1,3), (0,3)(1,2) inside block P (k = 0, 1) and block Q (k = 2, 3);
// cross rounds pair (k, 4 + (k xor t)).
__device__ __forceinline__ void ej_pair(bool within, int t, int k, int& p, int& q) {
  if (within) {
    constexpr unsigned code = 4u | 14u << 4 | 8u << 8 | 13u << 12 | 12u << 16 | 9u << 20;  // a | b << 2 per (t, k & 1)
    const unsigned v = (code >> ((t * 2 + (k & 1)) * 4)) & 15u;
    const int base = (k & 2) << 1;
    p = base + (int)(v & 3u);
    q = base + (int)(v >> 2);
  } else {
    p = k;
    q = 4 + (k ^ t);
  }
}

// Rotation test relative to the shifted diagonal (see k_eig4): rotate iff
// B_pq^2 > tol^2 (|B_pp| + t)(|B_qq| + t) + floor^2, t = max(tmin, 0).
__device__ __forceinline__ float ej_rot_shift(float a, float b, float g, float tol2, float floor2, float tsh,
                                              float& c, float& sn, float& t) {
  const float ab = (fabsf(a) + tsh) * (fabsf(b) + tsh), g2 = g * g;
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

// ej_round with the shifted rotation test (see k_eig4).
template <bool W, int T>
__device__ __forceinline__ void ej4_round(float* __restrict__ Sw, float* __restrict__ Uw, int hl, float tol2,
                                          float floor2, float tsh, unsigned& cnt, float& cmu) {
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
  __syncwarp();
  float ck, sk, tk, cl, sl, tl;
  const float mu = ej_rot_shift(ak, bk, gk, tol2, floor2, tsh, ck, sk, tk);
  ej_rot_shift(al, bl, gl, tol2, floor2, tsh, cl, sl, tl);
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


}  // namespace fctn_jacobi
