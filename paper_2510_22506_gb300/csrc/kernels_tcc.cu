// Gather-fed tcgen05 contraction (TF32): the table-driven contraction of
// k_sgemm,
//   C[cm[m] + cn[n]] = sum_k A[am[m] + ak[k]] * B[bn[n] + bk[k]],
// with the product on the tensor cores.  It serves the contractions of the
// head-mode association whose operands are strided views of labelled tensors
// (the M_0 chain and the right-hand-side chains from Z, Definition 3) in the
// tensor-core precisions; the Gram chains stay on k_sgemm in FP32.
//
// One CTA computes a 128 x BN tile of C over one K range.  Warps 0-7 gather
// each 32-wide K chunk of A (128 x 32) and B (BN x 32) with 4-byte
// asynchronous copies into a ring of S shared-memory stages laid out in the
// canonical K-major form of tcgen05 without swizzle (core matrices of 8 rows
// x 16 bytes; K-adjacent core matrices 128 bytes apart, 8-row groups 1024
// bytes apart).  Every copy instruction of a warp fills one whole core
// matrix, so its shared-memory writes are free of bank conflicts.  Two
// chunks later the gatherers round their elements of a chunk in place to the
// nearest TF32 value (the tensor cores would otherwise truncate), unless the
// operand's producer rounded it already, and release the stage to warp 8,
// one lane of which issues the MMAs (M = 128, N = BN, K = 8 each) and
// commits the stage back.  Warps 0-7 then read the accumulator (tcgen05.ld;
// warp w holds TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31) and store C through
// the tables, or this split's dense partial tile, which k_sg_reduce adds in
// split order.
//
// Every mbarrier wait is bounded: on expiry the CTA records FCTN_E_TIMEOUT,
// the other roles stop, the copies and MMAs already issued are waited for and
// the TMEM is freed before the CTA exits.
#include "fctn_internal.cuh"

namespace {

constexpr int TCC_GATHER = 256;                // warps 0-7: gather, then the epilogue
constexpr int TCC_THREADS = TCC_GATHER + 32;  // warp 8: TMEM and the MMAs
constexpr int TCC_BK = 32;                     // K elements per stage
constexpr int TCC_MAXS = 8;
constexpr long long kTccSpin = 1ll << 22;  // tries of up to 256 ns each (about 1 s)

__device__ __forceinline__ uint32_t tcc_s32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tcc_copy(uint32_t dst, const float* src, int nbytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(src), "r"(nbytes) : "memory");
}

__device__ __forceinline__ bool tcc_wait(uint64_t* bar, uint32_t par, volatile int* abort) {
  const uint32_t a = tcc_s32(bar);
  for (long long it = 0; it < kTccSpin; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(par), "r"(256u)
        : "memory");
    if (ok) return true;
    if (abort && *abort) return false;
  }
  return false;
}

// K-major, no swizzle, 32 K elements per row: version-1 descriptor with the
// K-adjacent core matrices 128 bytes apart (leading byte offset) and the
// 8-row groups 1024 bytes apart (stride byte offset).
__device__ __forceinline__ uint64_t tcc_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)(128u >> 4) << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

__global__ void __launch_bounds__(TCC_THREADS) k_tcc(SgShape sh, SgTabs t, const float* __restrict__ A,
                                                     const float* __restrict__ B, float* __restrict__ C,
                                                     float* __restrict__ part, int BN, int S, int round_a,
                                                     int round_b, int* __restrict__ status) {
  pdl_prologue();
  extern __shared__ __align__(128) unsigned char tsm[];
  __shared__ __align__(8) uint64_t full[TCC_MAXS], empty[TCC_MAXS], accf;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t a_bytes = 128u * TCC_BK * 4u, b_bytes = (uint32_t)BN * TCC_BK * 4u, st_bytes = a_bytes + b_bytes;
  const int m0 = blockIdx.x * 128, n0 = blockIdx.y * BN;
  const int kb = blockIdx.z * sh.kchunk, ke = min(kb + sh.kchunk, sh.K);
  const int kn = ke > kb ? ke - kb : 0;
  const int nk = (kn + TCC_BK - 1) / TCC_BK;
  int* am_s = (int*)(tsm + (size_t)S * st_bytes);
  int* cm_s = am_s + 128;
  int* bn_s = cm_s + 128;
  int* cn_s = bn_s + BN;
  int* run_s = cn_s + BN;  // per 4 columns: their outputs are 4 consecutive, 16-byte aligned offsets
  int* ak_s = run_s + BN / 4;
  int* bk_s = ak_s + sh.kchunk;
  // rows beyond M (columns beyond N) stage a copy of row 0: D rows (columns)
  // depend on their own A rows (B rows) only, and these are not stored
  for (int i = tid; i < 128; i += TCC_THREADS) {
    const bool v = m0 + i < sh.M;
    am_s[i] = v ? t.am[m0 + i] : t.am[0];
    cm_s[i] = v ? t.cm[m0 + i] : 0;
  }
  for (int i = tid; i < BN; i += TCC_THREADS) {
    const bool v = n0 + i < sh.N;
    bn_s[i] = v ? t.bn[n0 + i] : t.bn[0];
    cn_s[i] = v ? t.cn[n0 + i] : -1;
  }
  for (int i = tid; i < kn; i += TCC_THREADS) {
    ak_s[i] = t.ak[kb + i];
    bk_s[i] = t.bk[kb + i];
  }
  uint32_t ncols = 32;
  while ((int)ncols < BN) ncols <<= 1;
  if (tid == 0) {
    for (int i = 0; i < S; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(tcc_s32(&full[i])), "r"(TCC_GATHER));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(tcc_s32(&empty[i])), "r"(1));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(tcc_s32(&accf)), "r"(1));
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == TCC_GATHER / 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(tcc_s32(&tmem_slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  for (int j = tid; j < BN / 4; j += TCC_THREADS) {
    const int c = cn_s[4 * j];
    run_s[j] = c >= 0 && (c & 3) == 0 && cn_s[4 * j + 1] == c + 1 && cn_s[4 * j + 2] == c + 2 &&
               cn_s[4 * j + 3] == c + 3;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t sbase = tcc_s32(tsm);

  if (warp < TCC_GATHER / 32) {
    // This thread's element of every core matrix it fills: warp w fills the
    // K groups w % 4 and w % 4 + 4 (K columns 4 (w % 4) + kk and
    // 16 + 4 (w % 4) + kk) of the row groups g = 2 j + w / 4 (rows 8 g + rr).
    // A lane's (rr, kk) runs along the rows (8 rows x 4 K per instruction)
    // when the row digit is contiguous in memory, else along K (4 K x 8
    // rows).  The row pointers stay in registers for the whole K range.
    const int wk = warp & 3, wg = warp >> 2;
    const int rrA = sh.a_mfast ? (lane & 7) : (lane >> 2), kkA = sh.a_mfast ? (lane >> 3) : (lane & 3);
    const int rrB = sh.b_nfast ? (lane & 7) : (lane >> 2), kkB = sh.b_nfast ? (lane >> 3) : (lane & 3);
    const int rgB = BN >> 3;  // row groups of B (at most 16)
    const float* ap[8];
    const float* bp[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int g = 2 * j + wg;
      ap[j] = A + am_s[8 * g + rrA];
      bp[j] = B + (g < rgB ? bn_s[8 * g + rrB] : 0);
    }
    const uint32_t dA = (uint32_t)wg * 1024u + (uint32_t)wk * 128u + (uint32_t)rrA * 16u + (uint32_t)kkA * 4u;
    const uint32_t dB =
        a_bytes + (uint32_t)wg * 1024u + (uint32_t)wk * 128u + (uint32_t)rrB * 16u + (uint32_t)kkB * 4u;
    // ---- gather chunk c into stage c % S
    auto gather = [&](int c) {
      const uint32_t st0 = sbase + (uint32_t)(c % S) * st_bytes;
      const int kc = c * TCC_BK + 4 * wk;
#pragma unroll
      for (int h2 = 0; h2 < 2; ++h2) {
        // K beyond the range reads nothing and stages zeros
        const int ka = kc + 16 * h2 + kkA, kq = kc + 16 * h2 + kkB;
        const bool va = ka < kn, vb = kq < kn;
        const int oa = va ? ak_s[ka] : 0, ob = vb ? bk_s[kq] : 0;
        const int sa = va ? 4 : 0, sb = vb ? 4 : 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) tcc_copy(st0 + dA + 2048u * j + 512u * h2, ap[j] + oa, sa);
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (2 * j + wg < rgB) tcc_copy(st0 + dB + 2048u * j + 512u * h2, bp[j] + ob, sb);
      }
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    // ---- round this thread's elements of chunk c to TF32 where the operand
    // is not rounded already, and release the stage to the MMA warp
    auto rnd = [](unsigned char* p) {
      uint32_t u;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(*(float*)p));
      *(uint32_t*)p = u;
    };
    auto release = [&](int c) {
      unsigned char* st0 = tsm + (size_t)(c % S) * st_bytes;
      if (round_a)
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2)
#pragma unroll
          for (int j = 0; j < 8; ++j) rnd(st0 + dA + 2048u * j + 512u * h2);
      if (round_b)
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2)
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (2 * j + wg < rgB) rnd(st0 + dB + 2048u * j + 512u * h2);
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(tcc_s32(&full[c % S])) : "memory");
    };
    int issued = 0, released = 0;
    for (int c = 0; c < nk; ++c) {
      // stage c % S is free once the MMAs of chunk c - S are done
      if (c >= S && !tcc_wait(&empty[c % S], (uint32_t)((c / S - 1) & 1), &abort_flag)) {
        abort_flag = 1;
        break;
      }
      gather(c);
      ++issued;
      if (c >= 2) {  // chunk c - 2 has landed
        asm volatile("cp.async.wait_group 2;\n" ::: "memory");
        release(c - 2);
        ++released;
      }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");  // every copy lands before the stage is used or the CTA exits
    if (!abort_flag)
      for (; released < issued; ++released) release(released);
    // ---- epilogue: warp w reads TMEM lane quarter w % 4, the 16-column
    // blocks w / 4, w / 4 + 2, ...
    bool ok = nk == 0 || tcc_wait(&accf, 0u, &abort_flag);
    ok = __all_sync(0xffffffffu, ok);
    if (!ok) abort_flag = 1;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (ok) {
      const int rl = 32 * wk + lane, row = m0 + rl;
      const bool row_al = ((((uintptr_t)C) >> 2) + (uintptr_t)cm_s[rl]) % 4 == 0;  // C + cm 16-byte aligned
      for (int c0 = 16 * wg; c0 < BN; c0 += 32) {
        uint32_t v[16];
        const uint32_t taddr = tmem + ((uint32_t)(32 * wk) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        if (row >= sh.M) continue;
        float f[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          f[j] = nk > 0 ? __uint_as_float(v[j]) : 0.f;
          if (sh.ksplit == 1 && sh.round_tf32) {
            uint32_t x;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(x) : "f"(f[j]));
            f[j] = __uint_as_float(x);
          }
        }
        if (sh.ksplit == 1) {
          float* o = C + cm_s[rl];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int j = c0 + 4 * u;
            if (row_al && run_s[j >> 2]) {
              *reinterpret_cast<float4*>(o + cn_s[j]) = make_float4(f[4 * u], f[4 * u + 1], f[4 * u + 2], f[4 * u + 3]);
            } else {
#pragma unroll
              for (int q = 0; q < 4; ++q)
                if (cn_s[j + q] >= 0) o[cn_s[j + q]] = f[4 * u + q];
            }
          }
        } else {
          float* o = part + ((int64_t)blockIdx.z * sh.M + row) * sh.N + n0 + c0;
          if (n0 + c0 + 16 <= sh.N && (((uintptr_t)o) & 15) == 0) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
              *reinterpret_cast<float4*>(o + 4 * u) = make_float4(f[4 * u], f[4 * u + 1], f[4 * u + 2], f[4 * u + 3]);
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (n0 + c0 + j < sh.N) o[j] = f[j];
          }
        }
      }
    }
  } else if (lane == 0) {
    // ---- MMA issuer: D (TMEM, FP32) += A_chunk B_chunk^T
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) | ((128u >> 4) << 24);
    for (int c = 0; c < nk; ++c) {
      const int st = c % S;
      if (!tcc_wait(&full[st], (uint32_t)((c / S) & 1), &abort_flag)) {
        abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t sa = sbase + (uint32_t)st * st_bytes, sb = sa + a_bytes;
      const int kv = min(TCC_BK, kn - c * TCC_BK);
      const int nks = (kv + 7) >> 3;  // K steps holding data (the rest of the chunk is zero)
      for (int ks = 0; ks < nks; ++ks) {
        const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(tcc_desc(sa + 256u * ks)), "l"(tcc_desc(sb + 256u * ks)), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       tcc_s32(&empty[st]))
                   : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     tcc_s32(&accf))
                 : "memory");
    // the accumulator is not released before the MMAs issued above are done
    tcc_wait(&accf, 0u, nullptr);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (tid == 0 && abort_flag) atomicCAS(status, FCTN_OK, FCTN_E_TIMEOUT);
  if (warp == TCC_GATHER / 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols));
}

size_t tcc_smem(int BN, int S, int kchunk) {
  return (size_t)S * (128 + BN) * TCC_BK * 4 + (size_t)(256 + 2 * BN + BN / 4 + 2 * kchunk) * 4;
}

}  // namespace

// N per CTA: N rounded up to 16, at most 128; K split when the tiles alone
// leave most SMs idle and K is long (about split_ctas CTAs, 0 = two per SM);
// as many stages (3 to 8) as the chunks of a split need while two CTAs still
// share an SM (110 KB each), so that one CTA's epilogue overlaps the other's
// copies.
void tcc_shape(const SgShape& sg, int split_ctas, TccShape* ts) {
  ts->sh = sg;
  // a large output whose contiguous digit is a column digit (the k_sgemm
  // orientation) is computed transposed, so that the 32 lanes of a warp,
  // which hold 32 rows of the tile, store 32 consecutive elements
  ts->flip = sg.M >= 128 && sg.N >= 128 && (int64_t)sg.M * sg.N >= ((int64_t)1 << 22);
  if (ts->flip) {
    ts->sh.M = sg.N;
    ts->sh.N = sg.M;
    ts->sh.a_mfast = sg.b_nfast;
    ts->sh.b_nfast = sg.a_mfast;
  }
  const int M = ts->sh.M, N = ts->sh.N, K = ts->sh.K;
  ts->BN = N >= 128 ? 128 : (N + 15) / 16 * 16;
  if (ts->BN < 16) ts->BN = 16;
  const int tiles = ((M + 127) / 128) * ((N + ts->BN - 1) / ts->BN);
  const int chunks = (K + TCC_BK - 1) / TCC_BK;
  const int target = split_ctas > 0 ? split_ctas : 2 * 152;
  int ks = 1;
  if (tiles < target && chunks >= 8) {
    ks = (target + tiles - 1) / tiles;
    const int maxks = chunks / 4;
    ks = ks < maxks ? ks : maxks;
    if (ks < 1) ks = 1;
  }
  const int per = chunks > 0 ? (chunks + ks - 1) / ks : 1;
  ts->sh.kchunk = per * TCC_BK;
  ts->sh.ksplit = K > 0 ? (K + ts->sh.kchunk - 1) / ts->sh.kchunk : 1;
  int S = per < 3 ? 3 : (per > TCC_MAXS ? TCC_MAXS : per);
  while (S > 3 && tcc_smem(ts->BN, S, ts->sh.kchunk) > 110 * 1024) --S;
  ts->S = S;
  ts->round_a = ts->round_b = 1;
}

size_t tcc_part_elems(const TccShape& ts) {
  return ts.sh.ksplit > 1 ? (size_t)ts.sh.ksplit * ts.sh.M * ts.sh.N : 0;
}

int tcc_launches(const TccShape& ts) { return ts.sh.ksplit > 1 ? 2 : 1; }

void launch_tcc(const TccShape& ts, const SgTabs& t, const float* A, const float* B, float* C, float* part,
                int* status, cudaStream_t st) {
  const SgShape& sh = ts.sh;
  if (sh.M <= 0 || sh.N <= 0) return;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_tcc, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
    attr = true;
  }
  const dim3 grid((sh.M + 127) / 128, (sh.N + ts.BN - 1) / ts.BN, sh.ksplit);
  const SgTabs u = ts.flip ? SgTabs{t.bn, t.cn, t.am, t.cm, t.bk, t.ak} : t;
  const float* a = ts.flip ? B : A;
  const float* b = ts.flip ? A : B;
  launch_pdl(k_tcc, grid, dim3(TCC_THREADS), tcc_smem(ts.BN, ts.S, sh.kchunk), st, sh, u, a, b, C, part, ts.BN,
             ts.S, ts.flip ? ts.round_b : ts.round_a, ts.flip ? ts.round_a : ts.round_b, status);
  if (sh.ksplit > 1) launch_sg_reduce(sh, u, part, C, st);
}
