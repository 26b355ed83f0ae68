// Device helpers shared by the kernels that form tiles of a merged tensor M_k
// from its pair operands (see PairPlan): column decoding and the
// de-duplication of the operand rows that a chunk of columns needs.
#pragma once

#include "fctn_internal.cuh"

namespace fctn_tile {

__device__ __forceinline__ void decode_col(const PairPlan& p, int64_t j, int64_t& lo, int64_t& ro) {
  lo = 0;
  ro = 0;
  for (int d = p.nd - 1; d >= 0; --d) {
    int64_t e = p.ext[d];
    int64_t dig = j % e;
    j /= e;
    lo += dig * p.lstr[d];
    ro += dig * p.rstr[d];
  }
}

// Row slots of one chunk of nb <= 32 columns starting at j0 (columns at or
// beyond `end` get offset 0 and are zero-filled by the caller).  Executed by
// one full warp.  Writes, per column jj, the slot of its L row and of its R
// row (lsl[jj], rsl[jj]); per slot, the element offset of the row in L / R
// (lrow, rrow); and the slot counts (cnt[0] = L rows, cnt[1] = R rows).
// Consecutive columns often share a row (when the other operand's modes vary
// fastest), so a chunk stages each distinct row once.
__device__ __forceinline__ void chunk_slots(const PairPlan& p, int64_t j0, int nb, int64_t end, int* lsl, int* rsl,
                                            int64_t* lrow, int64_t* rrow, int* cnt) {
  const int lane = threadIdx.x & 31;
  int64_t lo = 0, ro = 0;
  const bool live = lane < nb;
  if (live && j0 + lane < end) decode_col(p, j0 + lane, lo, ro);
  // first lane with the same offset
  int fl = lane, fr = lane;
  for (int q = 0; q < 32; ++q) {
    int64_t ol = __shfl_sync(0xffffffffu, lo, q);
    int64_t orr = __shfl_sync(0xffffffffu, ro, q);
    if (q < lane && q < nb) {
      if (fl == lane && ol == lo) fl = q;
      if (fr == lane && orr == ro) fr = q;
    }
  }
  const unsigned firstL = __ballot_sync(0xffffffffu, live && fl == lane);
  const unsigned firstR = __ballot_sync(0xffffffffu, live && fr == lane);
  const unsigned below = (1u << lane) - 1u;
  const int my_l = __popc(firstL & below), my_r = __popc(firstR & below);
  const int sl = __shfl_sync(0xffffffffu, my_l, fl);
  const int sr = __shfl_sync(0xffffffffu, my_r, fr);
  if (live) {
    lsl[lane] = sl;
    rsl[lane] = sr;
    if (fl == lane) lrow[my_l] = lo;
    if (fr == lane) rrow[my_r] = ro;
  }
  if (lane == 0) {
    cnt[0] = __popc(firstL);
    cnt[1] = __popc(firstR);
  }
}

}  // namespace fctn_tile

namespace fctn_tile {

// Offset of X_(k)[i, j] in the row-major tensor (view (pre, I, post), j = a * post + b).
__device__ __forceinline__ int64_t x_offset(const ModeView& v, int64_t i, int64_t j) {
  const uint32_t jj = (uint32_t)j, post = (uint32_t)v.post;
  const uint32_t a = jj / post, b = jj - a * post;
  return ((int64_t)a * v.I + i) * v.post + b;
}

// Eq. 10 on one 64 x 64 tile (rows i0.., columns j0.. of X_(k)) of
// F = A_(k) M_k held as acc[4][4] by thread (ty, tx) = (tid / 16, tid % 16)
// of a 256-thread block.  F goes through shared memory (Fs: 64 x 65) so that
// X and the mask are read and written in memory order: runs along i when the
// mode is the fastest one (post == 1: X_(k)[i, j] at j I + i), along j
// otherwise.  Adds the thread's parts of ||Xnew - Xold||^2, ||Xold||^2 and
// ||Xnew - F||^2 to d2, x2, r2.  Ends with the block synchronised.
template <typename T>
__device__ __forceinline__ void xupdate_tile(const T (&acc)[4][4], T* Fs, int64_t i0, int64_t j0, const GramPlan& g,
                                             T* __restrict__ X, const uint32_t* __restrict__ bits, double rho,
                                             T& d2, T& x2, T& r2) {
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16, nt = blockDim.x;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) Fs[(ty * 4 + a) * 65 + tx * 4 + b] = acc[a][b];
  __syncthreads();
  const int ni = (int)min((int64_t)64, g.I - i0), nj = (int)min((int64_t)64, g.Pk - j0);
  const T r = (T)rho, inv = (T)(1.0 / (1.0 + rho));
  auto upd = [&](int64_t e, T f) {
    const T xo = X[e];
    const bool obs = (bits[e >> 5] >> (e & 31)) & 1u;
    const T xn = obs ? xo : (f + r * xo) * inv;
    X[e] = xn;
    const T d = xn - xo, q = xn - f;
    d2 = fma(d, d, d2);
    x2 = fma(xo, xo, x2);
    r2 = fma(q, q, r2);
  };
  if (ni > 0 && nj > 0) {
    if (g.xv.post == 1) {
      for (int e = tid; e < ni * nj; e += nt) {
        const int jj = e / ni, ii = e - jj * ni;
        upd((j0 + jj) * g.xv.I + i0 + ii, Fs[ii * 65 + jj]);
      }
    } else {
      for (int e = tid; e < ni * nj; e += nt) {
        const int ii = e / nj, jj = e - ii * nj;
        upd(x_offset(g.xv, i0 + ii, j0 + jj), Fs[ii * 65 + jj]);
      }
    }
  }
  __syncthreads();
}

}  // namespace fctn_tile
