// TMA-fed tcgen05 GEMM for the large products of the head-mode association:
//   Y_1 raw = X_(1) M_1^T   (split over K = P_1, partial tiles reduced in order)
//   Z       = X_(1)^T A_(1) (stored)
//   F^T     = M_1^T A_(1)^T (the X update of Eq. 10 fused into the epilogue)
// D[M x N] = A[M x K] B[N x K]^T with both operands K-major in global memory.
//
// One CTA computes one 128 x BN tile of D over one K range with three warp
// roles: warp 0 (one lane) issues the TMA copies of the A and B tiles of each
// 128-byte K chunk into a ring of S shared-memory stages (128-byte swizzle,
// the canonical K-major layout of tcgen05), warp 1 (one lane) issues the
// tcgen05.mma instructions (M = 128, N = BN, accumulator in TMEM) and commits
// each stage back to the producer, warps 2-5 read the accumulator with
// tcgen05.ld (each warp its 32-lane quarter of TMEM) and run the epilogue.
// Every mbarrier wait is bounded: on expiry the CTA records FCTN_E_TIMEOUT,
// the other roles stop, the copies and MMAs already issued are waited for
// (bounded again) and the TMEM is freed before the CTA exits.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cstring>

#include "fctn_internal.cuh"

namespace {

constexpr int TG_THREADS = 192;
constexpr long long kTgSpin = 1ll << 22;  // tries of up to 256 ns each (about 1 s)

__device__ __forceinline__ uint32_t s32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mb_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(s32(bar)), "r"(count));
}

// true once the phase with parity `par` has completed; false after the
// iteration limit or when another role raised *abort.
__device__ __forceinline__ bool mb_wait(uint64_t* bar, uint32_t par, volatile int* abort) {
  const uint32_t a = s32(bar);
  for (long long it = 0; it < kTgSpin; ++it) {
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

__device__ __forceinline__ void mb_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(s32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          s32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(s32(bar))
      : "memory");
}

// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzle:
// rows of 128 bytes, 8-row groups 1024 bytes apart (SBO), version 1, layout
// SWIZZLE_128B; the leading byte offset is not used by this layout.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor: D = F32, A = B = fmt (TF32 = 2 under kind::tf32,
// BF16 = 1 under kind::f16), both K-major, N, M = 128.
__device__ __forceinline__ uint32_t tg_idesc(uint32_t fmt, int N) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

struct TgTF32 {
  static constexpr uint32_t fmt = 2;
  __device__ static __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc));
  }
};
struct TgBF16 {
  static constexpr uint32_t fmt = 1;
  __device__ static __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc));
  }
};

__device__ __forceinline__ void mma_commit_to(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(s32(bar))
               : "memory");
}

__device__ __forceinline__ float tf32_round(float v) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(v));
  return __uint_as_float(u);
}

}  // namespace

namespace {

template <class Op>
__global__ void __launch_bounds__(TG_THREADS) k_tg_gemm(const __grid_constant__ CUtensorMap mapA,
                                                           const __grid_constant__ CUtensorMap mapB, TgArgs a) {
  pdl_prologue();
  extern __shared__ unsigned char smraw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  constexpr int MAXS = 8;
  __shared__ __align__(8) uint64_t full[MAXS], empty[MAXS], accf;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  __shared__ double sred[3][4];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int S = a.S, BN = a.BN;
  const uint32_t a_bytes = 128u * 128u, b_bytes = (uint32_t)BN * 128u, st_bytes = a_bytes + b_bytes;
  const int m0 = blockIdx.x * 128, n0 = blockIdx.y * BN;
  const int kb0 = blockIdx.z * a.kchunk;
  const int kend = min(a.K, kb0 + a.kchunk);
  constexpr int CH = 128;                       // bytes of K per stage
  const int kel = CH / (int)(Op::fmt == 2 ? 4 : 2);  // K elements per stage
  const int nk = kend > kb0 ? (kend - kb0 + kel - 1) / kel : 0;
  uint32_t ncols = 32;
  while ((int)ncols < BN) ncols <<= 1;

  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mb_init(&full[i], 1);
      mb_init(&empty[i], 1);
    }
    mb_init(&accf, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(s32(&tmem_slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- producer: TMA copies of A (128 x kel) and B (BN x kel) per stage
    int issued = 0;
    for (int kb = 0; kb < nk; ++kb) {
      const int st = kb % S;
      if (kb >= S && !mb_wait(&empty[st], (uint32_t)((kb / S - 1) & 1), &abort_flag)) {
        abort_flag = 1;
        break;
      }
      unsigned char* sa = sm + (size_t)st * st_bytes;
      mb_expect_tx(&full[st], st_bytes);
      const int kx = kb0 + kb * kel;
      tma_load_2d(sa, &mapA, kx, m0, &full[st]);
      tma_load_2d(sa + a_bytes, &mapB, kx, n0, &full[st]);
      ++issued;
    }
    // copies in flight land before the CTA may exit
    for (int kb = issued - S > 0 ? issued - S : 0; kb < issued; ++kb)
      mb_wait(&full[kb % S], (uint32_t)((kb / S) & 1), nullptr);
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    const uint32_t idesc = tg_idesc(Op::fmt, BN);
    for (int kb = 0; kb < nk; ++kb) {
      const int st = kb % S;
      if (!mb_wait(&full[st], (uint32_t)((kb / S) & 1), &abort_flag)) {
        abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t sa = s32(sm + (size_t)st * st_bytes), sb = sa + a_bytes;
#pragma unroll
      for (int ks = 0; ks < 4; ++ks)  // 32 bytes of K per instruction
        Op::mma(tmem, sw128_desc(sa + 32u * ks), sw128_desc(sb + 32u * ks), idesc, (kb > 0 || ks > 0) ? 1u : 0u);
      mma_commit_to(&empty[st]);
    }
    mma_commit_to(&accf);  // completes once every MMA issued above is done
    // the accumulator is not released (TMEM dealloc) before the MMAs finish,
    // even after an abort
    mb_wait(&accf, 0u, nullptr);
  } else if (warp >= 2) {
    // ---- epilogue: TMEM lane quarter (warp % 4) = rows 32 q .. 32 q + 31
    const int q = warp & 3;
    const int row = m0 + 32 * q + lane;
    const int rowc = row < a.M ? row : a.M - 1;  // clamped: loads stay in bounds, stores are skipped
    float d2 = 0.f, x2 = 0.f, r2 = 0.f;  // per-thread sums in FP32, combined in FP64 below
    // Eq. 10 epilogue: X_(1)[i, j] and its mask word for the 16 columns of
    // the next TMEM block are loaded before this block's stores, so that a
    // block's loads are in flight together and overlap the previous block
    float xp[16];
    uint32_t bp[16];
    auto xload = [&](int c0) {
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) {
        const int i = min(n0 + c0 + jj, a.N - 1);
        const int64_t e = (int64_t)i * a.P0 + rowc;
        xp[jj] = a.X[e];
        bp[jj] = a.bits[e >> 5];
      }
    };
    if (a.mode == TG_XUPDATE) xload(0);  // independent of the accumulator: overlaps the MMAs
    const bool ok = nk == 0 || mb_wait(&accf, 0u, &abort_flag);
    if (!ok) abort_flag = 1;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (ok) {
      for (int c0 = 0; c0 < BN; c0 += 16) {
        float xo[16];
        uint32_t bw[16];
        if (a.mode == TG_XUPDATE) {
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            xo[jj] = xp[jj];
            bw[jj] = bp[jj];
          }
          if (c0 + 16 < BN) xload(c0 + 16);
        }
        uint32_t v[16];
        const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        if (row >= a.M) continue;
        if (a.mode == TG_PARTIAL || a.mode == TG_STORE) {
          // 16 consecutive columns of this lane's row: four 16-byte stores
          // when they are whole and aligned, else element by element
          float* o = a.mode == TG_PARTIAL ? a.out + ((int64_t)blockIdx.z * a.M + row) * a.N + n0 + c0
                                          : a.out + (int64_t)row * a.ldo + n0 + c0;
          float f[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            f[j] = nk > 0 ? __uint_as_float(v[j]) : 0.f;
            if (a.mode == TG_STORE && a.round_tf32) f[j] = tf32_round(f[j]);
          }
          if (n0 + c0 + 16 <= a.N && ((uintptr_t)o & 15) == 0) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
              *reinterpret_cast<float4*>(o + 4 * u) = make_float4(f[4 * u], f[4 * u + 1], f[4 * u + 2], f[4 * u + 3]);
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (n0 + c0 + j < a.N) o[j] = f[j];
          }
        } else {
          // F^T[j, i]: Eq. 10 on X_(1)[i, j] (row j = this lane, i = column)
          const float r = (float)a.rho, inv = (float)(1.0 / (1.0 + a.rho));
          float xt[16];
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            const int i = n0 + c0 + jj;
            const float f = nk > 0 ? __uint_as_float(v[jj]) : 0.f;
            const int64_t e = (int64_t)i * a.P0 + row;
            const bool obs = (bw[jj] >> (e & 31)) & 1u;
            const float xn = obs ? xo[jj] : (f + r * xo[jj]) * inv;
            xt[jj] = xn;
            if (i >= a.N) continue;
            a.X[e] = xn;
            if (a.Xb) a.Xb[e] = __float2bfloat16_rn(xn);
            const float d = xn - xo[jj], qq = xn - f;
            d2 = fmaf(d, d, d2);
            x2 = fmaf(xo[jj], xo[jj], x2);
            r2 = fmaf(qq, qq, r2);
          }
          if (a.XT) {  // 16 consecutive columns of row j: four 16-byte stores when the row is whole
            float* o = a.XT + (int64_t)row * a.ldt + n0 + c0;
            if (a.round_tf32)
#pragma unroll
              for (int jj = 0; jj < 16; ++jj) xt[jj] = tf32_round(xt[jj]);
            if (n0 + c0 + 16 <= a.N) {
#pragma unroll
              for (int u = 0; u < 4; ++u)
                *(float4*)(o + 4 * u) = make_float4(xt[4 * u], xt[4 * u + 1], xt[4 * u + 2], xt[4 * u + 3]);
            } else {
              for (int jj = 0; jj < 16; ++jj)
                if (n0 + c0 + jj < a.N) o[jj] = xt[jj];
            }
          }
          if (a.XTb) {
            __nv_bfloat16* o = a.XTb + (int64_t)row * a.ldt + n0 + c0;
#pragma unroll
            for (int jj = 0; jj < 16; ++jj)
              if (n0 + c0 + jj < a.N) o[jj] = __float2bfloat16_rn(xt[jj]);
          }
        }
      }
    }
    if (a.mode == TG_XUPDATE) {
      double t[3] = {(double)d2, (double)x2, (double)r2};
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        for (int o = 16; o > 0; o >>= 1) t[u] += __shfl_xor_sync(0xffffffffu, t[u], o);
        if (lane == 0) sred[u][warp - 2] = t[u];
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) {
    if (abort_flag) atomicCAS(a.status, FCTN_OK, FCTN_E_TIMEOUT);
    if (a.mode == TG_XUPDATE) {
      const int64_t blk = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
      for (int u = 0; u < 3; ++u) a.red[blk * 3 + u] = sred[u][0] + sred[u][1] + sred[u][2] + sred[u][3];
    }
  }
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols));
}

// Sum of the K-split partials of a TG_PARTIAL launch (split order, compensated):
// out[row * N + col] = sum_z part[z][row][col].
__global__ void k_tg_reduce(const float* __restrict__ part, int ksplit, int64_t MN, float* __restrict__ out) {
  pdl_prologue();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < MN; e += (int64_t)gridDim.x * blockDim.x) {
    out[e] = split_sum(part, ksplit, MN, e);
  }
}

}  // namespace

// ---- host -------------------------------------------------------------------
namespace {

typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static EncodeTiled fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiled)p;
    else
      cudaGetLastError();
  }
  return fn;
}

}  // namespace

int tg_make_map(void* map, const void* base, int64_t rows, int64_t cols, int64_t ld, int elem, int box_rows) {
  EncodeTiled fn = encode_fn();
  if (!fn) return FCTN_E_CUDA;
  if (((uintptr_t)base & 15) || (ld * elem) % 16 || box_rows < 1 || box_rows > 256) return FCTN_E_UNSUPPORTED;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(ld * elem)};
  const cuuint32_t box[2] = {(cuuint32_t)(128 / elem), (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  CUresult r = fn((CUtensorMap*)map, elem == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                  (void*)base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? FCTN_OK : FCTN_E_UNSUPPORTED;
}

// Row-major FP32 matrix (rows x cols, leading dimension ld) with an
// unswizzled box of box_rows x box_cols (dense in shared memory, inner
// dimension box_cols); elements outside the matrix load as zero.
int tma_map_f32(void* map, const float* base, int64_t rows, int64_t cols, int64_t ld, int box_cols, int box_rows) {
  EncodeTiled fn = encode_fn();
  if (!fn) return FCTN_E_CUDA;
  if (((uintptr_t)base & 15) || (ld * 4) % 16 || box_rows < 1 || box_rows > 256 || box_cols < 4 || box_cols > 256 ||
      (box_cols * 4) % 16)
    return FCTN_E_UNSUPPORTED;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(ld * 4)};
  const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  CUresult r = fn((CUtensorMap*)map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? FCTN_OK : FCTN_E_UNSUPPORTED;
}

size_t tg_smem_bytes(int BN, int S) { return (size_t)S * (128 * 128 + (size_t)BN * 128) + 1024; }

// BN: N rounded up to 16 (one column tile when N <= 256, else tiles of 256);
// S: as many stages as fit 200 KB (at most 8; the launch allows 202 KB, the
// extra for aligning the ring to 1024 bytes); K split so that about
// want_ctas CTAs run, each with at least 4 chunks.
void tg_shape(int M, int N, int K, int elem, int want_ctas, TgArgs* a) {
  a->M = M;
  a->N = N;
  a->K = K;
  a->BN = N <= 256 ? (N + 15) / 16 * 16 : 256;
  const int kel = 128 / elem;
  const int chunks = (K + kel - 1) / kel;
  // a long K loop gets a deep ring; a short one (K <= 8 chunks) two stages,
  // so that two CTAs (and their epilogues) share an SM
  int S = chunks > 8 ? 8 : 2;
  while (S > 2 && tg_smem_bytes(a->BN, S) > 200 * 1024) --S;
  a->S = S;
  const int tiles = ((M + 127) / 128) * ((N + a->BN - 1) / a->BN);
  int ks = tiles >= want_ctas ? 1 : (want_ctas + tiles - 1) / tiles;
  const int maxks = chunks / 4 > 0 ? chunks / 4 : 1;
  ks = ks < maxks ? ks : maxks;
  int per = (chunks + ks - 1) / ks;
  a->kchunk = per * kel;
  a->ksplit = (K + a->kchunk - 1) / a->kchunk;
  if (a->ksplit < 1) a->ksplit = 1;
}

void launch_tg_gemm(const void* mapA, const void* mapB, const TgArgs& a, int bf16, cudaStream_t st) {
  const dim3 grid((a.M + 127) / 128, (a.N + a.BN - 1) / a.BN, a.ksplit);
  const size_t smem = tg_smem_bytes(a.BN, a.S);
  static bool attr[2] = {false, false};
  if (bf16) {
    if (!attr[1]) {
      cudaFuncSetAttribute(k_tg_gemm<TgBF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 202 * 1024);
      attr[1] = true;
    }
    launch_pdl(k_tg_gemm<TgBF16>, grid, dim3(TG_THREADS), smem, st, *(const CUtensorMap*)mapA, *(const CUtensorMap*)mapB, a);
  } else {
    if (!attr[0]) {
      cudaFuncSetAttribute(k_tg_gemm<TgTF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 202 * 1024);
      attr[0] = true;
    }
    launch_pdl(k_tg_gemm<TgTF32>, grid, dim3(TG_THREADS), smem, st, *(const CUtensorMap*)mapA, *(const CUtensorMap*)mapB, a);
  }
}

void launch_tg_reduce(const float* part, int ksplit, int64_t MN, float* out, cudaStream_t st) {
  int64_t b = (MN + 255) / 256;
  launch_pdl(k_tg_reduce, dim3((unsigned)(b < 608 ? (b < 1 ? 1 : b) : 608)), dim3(256), 0, st, part, ksplit, MN, out);
}
