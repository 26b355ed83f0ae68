// Tensor-core (tcgen05 / TMEM) Gram + right-hand side of Eq. 5 for the TF32
// and BF16 precisions, with M_k formed on chip.
//
// Per K-chunk of BK columns j of M_k the CTA
//   1. copies the L / R rows of the chunk's pair operands (cp.async),
//   2. forms the M_k tile (CUDA cores, FP32) and writes it, rounded to the
//      operand type (TF32; or BF16 split into hi + lo parts), into a K-major
//      shared-memory operand (no swizzle: 8-row x 16-byte core matrices,
//      K-adjacent core matrices 128 B apart),
//   3. writes the chunk's X_(k) rows into a second operand,
//   4. has one thread issue tcgen05.mma: D_b (TMEM, FP32) += M_b [M ; X]^T for
//      each 128-row block b of M_k, then tcgen05.commit to the buffer's
//      mbarrier.
// Operand buffers are double-buffered: forming chunk c+1 overlaps the MMAs of
// chunk c.  At the end the accumulators are read with tcgen05.ld and written
// as this split's partial of D = M [M ; X_(k)]^T (same layout as the CUDA-core
// path, reduced by k_reduce_gram_rhs in a fixed order).
//
// Every mbarrier wait is bounded; on expiry the kernel records
// FCTN_E_TIMEOUT, waits (bounded) for its MMAs, frees its TMEM and returns.
#include <cuda_bf16.h>

#include <cstring>

#include "fctn_internal.cuh"
#include "fctn_tile.cuh"

namespace {

constexpr int TC_THREADS = 512;  // 16 warps; TMEM lane quarter = warp % 4
constexpr long long kSpinLimit = 1ll << 26;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }


__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(valid ? 4 : 0));
}

// ---- operand element types ------------------------------------------------
// TF32: one operand per value (rounded to nearest TF32).
struct OpTF32 {
  static constexpr int kc = 4;        // elements per 16-byte core-matrix row
  static constexpr uint32_t fmt = 2;  // TF32
  static constexpr bool split = false;
  __device__ static __forceinline__ void put(unsigned char* base, uint32_t off, uint32_t, float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    *(uint32_t*)(base + off) = r;
  }
};
// BF16: every value is split as v = hi + lo with hi = bf16(v), lo = bf16(v - hi);
// the hi part is stored at `off`, the lo part `lo_off` bytes further, and a
// product x.y is computed as hi.hi + hi.lo + lo.hi (three MMAs), which keeps
// about 16 significant bits of every operand while the MMAs run in BF16.
struct OpBF16 {
  static constexpr int kc = 8;
  static constexpr uint32_t fmt = 1;  // BF16
  static constexpr bool split = true;
  __device__ static __forceinline__ void put(unsigned char* base, uint32_t off, uint32_t lo_off, float v) {
    __nv_bfloat16 hi = __float2bfloat16_rn(v);
    *(__nv_bfloat16*)(base + off) = hi;
    *(__nv_bfloat16*)(base + off + lo_off) = __float2bfloat16_rn(v - __bfloat162float(hi));
  }
};

// Byte offset of element (row r, k) in a K-major no-swizzle operand with
// BK columns: core matrix (r/8, k/kc), 8 rows of 16 bytes each.
template <class Op>
__device__ __forceinline__ uint32_t op_off(int r, int k, int BK) {
  const uint32_t sbo = (uint32_t)(BK / Op::kc) * 128u;
  return (uint32_t)(r >> 3) * sbo + (uint32_t)(k / Op::kc) * 128u + (uint32_t)(r & 7) * 16u +
         (uint32_t)(k % Op::kc) * (16u / Op::kc);
}

// Element e of an operand with BK columns taken in core-matrix order: core
// matrix e / (8 kc) (row block, column block; lg_nkc = log2(BK / kc)), then its
// 8 rows x kc columns row-major, so that consecutive e are consecutive bytes
// (a warp's stores hit distinct banks).
template <class Op>
__device__ __forceinline__ void cm_rc(int e, int lg_nkc, int& r, int& k) {
  constexpr int per = 8 * Op::kc;
  const int cm = e / per, w = e - cm * per;
  r = ((cm >> lg_nkc) << 3) + w / Op::kc;
  k = (cm & ((1 << lg_nkc) - 1)) * Op::kc + w % Op::kc;
}

// tcgen05 shared-memory matrix descriptor (no swizzle, version 1).
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version
  return d;                // base offset 0, layout: no swizzle
}

// Instruction descriptor: dense, D = F32, A = B = fmt, both K-major, N, M = 128.
__device__ __forceinline__ uint32_t make_idesc(uint32_t fmt, int N) {
  uint32_t d = 0;
  d |= 1u << 4;                          // D format F32
  d |= fmt << 7;                         // A format
  d |= fmt << 10;                        // B format
  d |= (uint32_t)(N >> 3) << 17;         // N / 8
  d |= (uint32_t)(128 >> 4) << 24;       // M / 16
  return d;
}

template <class Op>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int accumulate);

template <>
__device__ __forceinline__ void mma<OpTF32>(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            int accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
template <>
__device__ __forceinline__ void mma<OpBF16>(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            int accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
}

// Bounded wait for the phase with the given parity; false on expiry.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  const unsigned a = smem_u32(bar);
  for (long long it = 0; it < kSpinLimit; ++it) {
    unsigned ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity));
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar)));
}

template <class Op>
__global__ void __launch_bounds__(TC_THREADS) k_gram_tc(PairPlan p, const float* __restrict__ L,
                                                        const float* __restrict__ R, const float* __restrict__ X,
                                                        float* __restrict__ part, GramPlan g, TcPlan tp,
                                                        float* __restrict__ Mout, int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int s = (int)g.s;
  const int BK = tp.BK;
  const TcGroup grp = tp.groups[blockIdx.x];
  // split operands (BF16): the lo parts fill the second half of each buffer
  const uint32_t a_lo = Op::split ? tp.a_bytes / 2 : 0, x_lo = Op::split ? tp.x_bytes / 2 : 0;
  // ---- shared memory carve-up
  unsigned char* A_buf[2];
  unsigned char* X_buf[2];
  A_buf[0] = sm;
  A_buf[1] = A_buf[0] + tp.a_bytes;
  X_buf[0] = A_buf[1] + tp.a_bytes;
  X_buf[1] = X_buf[0] + tp.x_bytes;
  float* Ls = (float*)(X_buf[1] + tp.x_bytes);
  float* Rs = Ls + (size_t)BK * p.Ljs;
  int* lo = (int*)(Rs + (size_t)BK * p.Rjs);
  int* ro = lo + s;
  int* lk = ro + s;
  int* rk = lk + p.K;
  int64_t* cl = (int64_t*)(((uintptr_t)(rk + p.K) + 15) & ~(uintptr_t)15);
  int64_t* cr = cl + BK;
  uint64_t* bars = (uint64_t*)(cr + BK);  // 2 mbarriers
  uint32_t* tmem_slot = (uint32_t*)(bars + 2);
  __shared__ int abort_flag;
  __shared__ int lsl[32], rsl[32], cnt[2];  // row slot of every column, distinct-row counts
  __shared__ int64_t xcol[32];              // offset of X_(k)[0, j] of every column (-1 past the chunk)
  const int lg_nkc = __ffs(BK / Op::kc) - 1;

  for (int e = tid; e < s; e += TC_THREADS) {
    lo[e] = p.tab[e];
    ro[e] = p.tab[s + e];
  }
  for (int e = tid; e < p.K; e += TC_THREADS) {
    lk[e] = p.tab[2 * s + e];
    rk[e] = p.tab[2 * s + p.K + e];
  }
  // zero the padding rows of both operands once (rows >= s of M_k, rows
  // >= valid X rows); every other element is rewritten for every chunk
  {
    const uint32_t row_bytes = (uint32_t)BK * (16u / Op::kc);  // one row: BK elements
    const int a_rows = tp.n_mb * 128, a_pad0 = s & ~7;             // core-matrix rows from s/8*8
    for (int b = 0; b < 2; ++b) {
      for (int e = tid; e < (a_rows - a_pad0) * BK; e += TC_THREADS) {
        int r = a_pad0 + e / BK, k = e % BK;
        if (r >= s) Op::put(A_buf[b], op_off<Op>(r, k, BK), a_lo, 0.f);
      }
      const int xvalid = (int)min((int64_t)grp.xw, g.I - grp.xi0);
      for (int e = tid; e < grp.xw * BK; e += TC_THREADS) {
        int r = e / BK, k = e % BK;
        if (r >= xvalid) Op::put(X_buf[b], op_off<Op>(r, k, BK), x_lo, 0.f);
      }
    }
    (void)row_bytes;
  }
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(tp.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
  const uint32_t tmem = *tmem_slot;

  const int64_t kb = (int64_t)blockIdx.z * g.kchunk;
  const int64_t ke = min(kb + g.kchunk, g.Pk);
  const int nchunk = (int)((ke - kb + BK - 1) / BK);
  const int mrows = tp.n_mb * 128;  // rows of the M_k operand (zero beyond s)
  unsigned uses[2] = {0u, 0u};
  const uint32_t lbo = 128u, sbo = (uint32_t)(BK / Op::kc) * 128u;
  constexpr int KSTEP = (Op::kc == 4) ? 8 : 16;  // K per MMA instruction

  for (int c = 0; c < nchunk; ++c) {
    const int b = c & 1;
    const int64_t k0 = kb + (int64_t)c * BK;
    // buffer b is free once the MMAs of chunk c-2 completed
    if (uses[b] > 0) {
      bool ok = true;
      if (tid == 0) ok = mbar_wait(&bars[b], (uses[b] - 1) & 1u);
      if (tid == 0 && !ok) abort_flag = 1;
      __syncthreads();
      if (abort_flag) break;
    }
    // 1. the distinct L and R rows of the chunk's columns
    if (warp == 0) {
      fctn_tile::chunk_slots(p, k0, BK, ke, lsl, rsl, cl, cr, cnt);
      if (lane < BK) {  // j = a * post + b'  ->  a * I * post + b'
        const int64_t j = k0 + lane;
        const uint32_t post = (uint32_t)g.xv.post, jj = (uint32_t)j;
        const uint32_t a = jj / post;
        xcol[lane] = j < ke ? ((int64_t)a * g.xv.I) * g.xv.post + (jj - a * post) : -1;
      }
    }
    __syncthreads();
    for (int e = tid; e < cnt[0] * p.Ljs; e += TC_THREADS) {
      int q = e / p.Ljs, c_ = e - q * p.Ljs;
      cp_async4(Ls + e, L + cl[q] + c_, true);
    }
    for (int e = tid; e < cnt[1] * p.Rjs; e += TC_THREADS) {
      int q = e / p.Rjs, c_ = e - q * p.Rjs;
      cp_async4(Rs + e, R + cr[q] + c_, true);
    }
    asm volatile("cp.async.commit_group;\n" ::);
    // 3. X rows of this group into the X operand (overlaps the slab copies),
    //    in core-matrix order; rows >= xvalid stay zero
    if (grp.xw > 0) {
      unsigned char* xb = X_buf[b];
      const int xvalid = (int)min((int64_t)grp.xw, g.I - grp.xi0);
      const int rows8 = (xvalid + 7) & ~7;
      for (int e = tid; e < rows8 * BK; e += TC_THREADS) {
        int r, kk;
        cm_rc<Op>(e, lg_nkc, r, kk);
        if (r >= xvalid) continue;
        const int64_t xc = xcol[kk];
        const float v = xc >= 0 ? __ldg(X + xc + (int64_t)(grp.xi0 + r) * g.xv.post) : 0.f;
        Op::put(xb, op_off<Op>(r, kk, BK), x_lo, v);
      }
    }
    asm volatile("cp.async.wait_group 0;\n" ::);
    __syncthreads();
    // 2. M_k tile (FP32 on the CUDA cores) into the A operand; group 0 also
    //    writes it out (FP32) when M_k is kept for the X update
    {
      unsigned char* ab = A_buf[b];
      const bool wm = Mout != nullptr && blockIdx.x == 0;
      const int rows8 = (s + 7) & ~7;
      for (int e = tid; e < rows8 * BK; e += TC_THREADS) {  // core-matrix order
        int sg, jj;
        cm_rc<Op>(e, lg_nkc, sg, jj);
        if (sg >= s) continue;
        const float* l = Ls + lsl[jj] * p.Ljs + lo[sg];
        const float* r = Rs + rsl[jj] * p.Rjs + ro[sg];
        float a = 0.f;
        if (k0 + jj < ke)
          for (int q = 0; q < p.K; ++q) a = fmaf(l[lk[q]], r[rk[q]], a);
        Op::put(ab, op_off<Op>(sg, jj, BK), a_lo, a);
        if (wm && k0 + jj < ke) Mout[(int64_t)sg * g.Pk + k0 + jj] = a;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::);
    __syncthreads();
    // 4. MMAs of this chunk (one thread)
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
      const uint32_t abase = smem_u32(A_buf[b]);
      const uint32_t xbase = smem_u32(X_buf[b]);
      for (int mb = 0; mb < tp.n_mb; ++mb) {
        const uint32_t a_blk = abase + (uint32_t)(mb * 16) * sbo;  // 128 rows = 16 core-matrix rows
        const uint32_t dcol = (uint32_t)(mb * grp.width);
        for (int ks = 0; ks < BK / KSTEP; ++ks) {
          const uint32_t koff = (uint32_t)(ks * (KSTEP / Op::kc)) * lbo;
          const uint64_t ad = make_desc(a_blk + koff, lbo, sbo);
          const int acc = (c > 0 || ks > 0) ? 1 : 0;
          if (grp.mw > 0) {  // M part of B: rows 0..mw of the same operand
            const uint64_t bd = make_desc(abase + koff, lbo, sbo);
            const uint32_t id = make_idesc(Op::fmt, grp.mw);
            mma<Op>(tmem + dcol, ad, bd, id, acc);
            if (Op::split) {
              mma<Op>(tmem + dcol, ad, make_desc(abase + a_lo + koff, lbo, sbo), id, 1);   // hi . lo
              mma<Op>(tmem + dcol, make_desc(a_blk + a_lo + koff, lbo, sbo), bd, id, 1);   // lo . hi
            }
          }
          if (grp.xw > 0) {
            const uint64_t bd = make_desc(xbase + koff, lbo, sbo);
            const uint32_t id = make_idesc(Op::fmt, grp.xw);
            mma<Op>(tmem + dcol + (uint32_t)grp.mw, ad, bd, id, acc);
            if (Op::split) {
              mma<Op>(tmem + dcol + (uint32_t)grp.mw, ad, make_desc(xbase + x_lo + koff, lbo, sbo), id, 1);
              mma<Op>(tmem + dcol + (uint32_t)grp.mw, make_desc(a_blk + a_lo + koff, lbo, sbo), bd, id, 1);
            }
          }
        }
      }
      mma_commit(&bars[b]);
    }
    uses[b]++;
    (void)mrows;
  }
  // ---- wait for the last MMAs (both buffers), then read the accumulators
  bool ok = !abort_flag;
  if (tid == 0) {
    for (int b = 0; b < 2; ++b)
      if (uses[b] > 0 && !mbar_wait(&bars[b], (uses[b] - 1) & 1u)) ok = false;
    if (!ok) atomicCAS(status, FCTN_OK, FCTN_E_TIMEOUT);
    abort_flag = ok ? 0 : 1;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
  if (!abort_flag && nchunk > 0) {
    float* P = part + (int64_t)blockIdx.z * g.s * g.ncols;
    // a warp reads the TMEM lanes of its quarter (warp % 4); the warps of a
    // quarter take turns over the groups of 8 columns
    const int wq = warp & 3, wh = warp >> 2, nwh = TC_THREADS / 128;
    for (int mb = 0; mb < tp.n_mb; ++mb) {
      const int row = mb * 128 + wq * 32 + lane;  // TMEM lane = row within the block
      for (int c0 = wh * 8; c0 < grp.width; c0 += 8 * nwh) {
        uint32_t v[8];
        const uint32_t taddr = tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)(mb * grp.width + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
        if (row < s) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int cc = c0 + q;
            int64_t col;
            if (cc < grp.mw) col = cc;                       // Gram column
            else col = g.gcols + grp.xi0 + (cc - grp.mw);      // right-hand-side column
            bool valid = (cc < grp.mw) ? (cc < s) : (grp.xi0 + (cc - grp.mw) < g.I);
            if (valid) P[(int64_t)row * g.ncols + col] = __uint_as_float(v[q]);
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tp.tmem_cols));
}

}  // namespace

// Host planning: groups of output columns per CTA so that every group fits
// 512 TMEM columns (n_mb blocks of 128 rows x group width).
int tc_plan(const PairPlan& p, const GramPlan& g, int precision, TcPlan* tp) {
  memset(tp, 0, sizeof *tp);
  const int s = (int)g.s, I = (int)g.I;
  if (s > 256) return FCTN_E_UNSUPPORTED;
  tp->n_mb = (s + 127) / 128;
  const int mw = g.gcols > 0 ? (s + 15) / 16 * 16 : 0;  // no Gram columns when the Gram is factored
  const int xw_all = (I + 15) / 16 * 16;
  int ng = 0;
  if (tp->n_mb * (mw + xw_all) <= 512 && mw + xw_all <= 512) {
    // M part and all X rows in one group (two MMAs of N <= 256 each)
    if (mw <= 256 && xw_all <= 256) {
      tp->groups[ng++] = TcGroup{mw, 0, xw_all, mw + xw_all};
    }
  }
  if (ng == 0) {
    if (mw > 0) tp->groups[ng++] = TcGroup{mw, 0, 0, mw};
    for (int x0 = 0; x0 < I; x0 += 256) {
      int w = I - x0 < 256 ? (I - x0 + 15) / 16 * 16 : 256;
      if (ng >= TC_MAX_GROUPS) return FCTN_E_UNSUPPORTED;
      tp->groups[ng++] = TcGroup{0, x0, w, w};
    }
  }
  tp->n_groups = ng;
  int maxw = 0;
  for (int i = 0; i < ng; ++i) maxw = tp->groups[i].width > maxw ? tp->groups[i].width : maxw;
  int need = tp->n_mb * maxw, cols = 32;
  while (cols < need) cols <<= 1;
  if (cols > 512) return FCTN_E_UNSUPPORTED;
  tp->tmem_cols = cols;
  const int esz = 4;  // TF32: 4-byte values; BF16: hi + lo parts of 2 bytes each
  // columns per chunk: operands (double-buffered) + slabs within ~200 KB
  int maxx = 0;
  for (int i = 0; i < ng; ++i) maxx = tp->groups[i].xw > maxx ? tp->groups[i].xw : maxx;
  for (int bk = 32; bk >= 16; bk /= 2) {
    size_t a = (size_t)tp->n_mb * 128 * bk * esz, x = (size_t)(maxx > 0 ? maxx : 16) * bk * esz;
    size_t slabs = (size_t)bk * (p.Ljs + p.Rjs) * 4;
    size_t tabs = (size_t)(2 * s + 2 * p.K) * 4 + 16 + 2 * (size_t)bk * 8 + 64;
    size_t total = 2 * a + 2 * x + slabs + tabs;
    tp->BK = bk;
    tp->a_bytes = (uint32_t)a;
    tp->x_bytes = (uint32_t)x;
    tp->smem = total;
    if (total <= 200 * 1024) return FCTN_OK;
  }
  return tp->smem <= 200 * 1024 ? FCTN_OK : FCTN_E_UNSUPPORTED;
}

void launch_gram_tc(const PairPlan& p, const float* L, const float* R, const float* X, float* part,
                    const GramPlan& g, const TcPlan& tp, int precision, float* Mout, int* status, cudaStream_t st) {
  dim3 grid(tp.n_groups, 1, g.ksplit);
  // The shared-memory limit is set once to the most any plan asks for (tc_plan
  // keeps tp.smem <= 200 KB), not to this launch's size: a launch recorded in
  // a graph with a larger size than a later launch set the limit to would no
  // longer fit the function's limit when it is launched on its own (as a
  // profiler replaying graph nodes one by one does).
  static bool attr[2] = {false, false};
  if (precision == FCTN_BF16) {
    if (!attr[1]) {
      cudaFuncSetAttribute(k_gram_tc<OpBF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      attr[1] = true;
    }
    k_gram_tc<OpBF16><<<grid, TC_THREADS, tp.smem, st>>>(p, L, R, X, part, g, tp, Mout, status);
  } else {
    if (!attr[0]) {
      cudaFuncSetAttribute(k_gram_tc<OpTF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      attr[0] = true;
    }
    k_gram_tc<OpTF32><<<grid, TC_THREADS, tp.smem, st>>>(p, L, R, X, part, g, tp, Mout, status);
  }
}
