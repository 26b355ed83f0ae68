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
