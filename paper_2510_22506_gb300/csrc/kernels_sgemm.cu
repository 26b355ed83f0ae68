// Table-driven FP32 contraction on the CUDA cores, and the small kernels of
// the head-mode association of a sweep.
//
// A binary contraction of two labelled tensors (Definition 3) becomes a GEMM
// once its free indices are split into the row digits m (held by A), the
// column digits n (held by B) and the contracted digits k (held by both):
//   C[cm[m] + cn[n]] = sum_k A[am[m] + ak[k]] * B[bn[n] + bk[k]].
// The six offset tables are built once per plan on the host, so any strided
// layout of A, B and C is served by one kernel without mixed-radix decoding
// per element.  The CTA tile is 128 x 64 with K chunks of 16 staged through
// shared memory (the next chunk is loaded into registers while the current
// one is multiplied), 8 x 4 outputs per thread.  With a K split the CTAs of
// one tile write dense partials that k_sg_reduce adds in split order.
#include <cstring>

#include "fctn_internal.cuh"

thread_local bool g_pdl = false;  // see launch_pdl

namespace {

constexpr int SG_BM = 128, SG_BN = 64, SG_BK = 16, SG_THREADS = 256;

__device__ __forceinline__ float sg_tf32(float v) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(v));
  return __uint_as_float(u);
}

// 4-byte asynchronous copy global -> shared; nbytes = 0 writes a zero
// (the source is then not read).
__device__ __forceinline__ void sg_acopy(float* dst, const float* src, int nbytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(nbytes)
               : "memory");
}

constexpr int SG_ST = 3;  // pipeline stages of the operand tiles

__global__ void __launch_bounds__(SG_THREADS) k_sgemm(SgShape sh, SgTabs t, const float* __restrict__ A,
                                                      const float* __restrict__ B, float* __restrict__ C,
                                                      float* __restrict__ part) {
  pdl_prologue();
  __shared__ __align__(16) float As[SG_ST][SG_BK][SG_BM + 4];
  __shared__ __align__(16) float Bs[SG_ST][SG_BK][SG_BN + 4];
  __shared__ int am_s[SG_BM], bn_s[SG_BN];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.x * SG_BM, n0 = blockIdx.y * SG_BN;
  const int kb = blockIdx.z * sh.kchunk, ke = min(kb + sh.kchunk, sh.K);
  for (int i = tid; i < SG_BM; i += SG_THREADS) am_s[i] = (m0 + i < sh.M) ? t.am[m0 + i] : -1;
  for (int i = tid; i < SG_BN; i += SG_THREADS) bn_s[i] = (n0 + i < sh.N) ? t.bn[n0 + i] : -1;
  __syncthreads();
  // loader mappings: consecutive lanes take consecutive k (the contracted
  // digit is innermost in the operand) or consecutive rows m / columns n
  // (the row / column digit is innermost), whichever reads memory in order.
  // The tiles of step k0 go to stage buf by asynchronous copies (zeros
  // outside the operands), SG_ST - 1 steps ahead of the multiply.
  auto issue = [&](int k0, int buf) {
    if (sh.a_mfast) {  // A: m = tid % 128, k = tid / 128 + 2 i
      const int a = am_s[tid & 127];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int kk = (tid >> 7) + 2 * i, k = k0 + kk;
        const bool v = k < ke && a >= 0;
        sg_acopy(&As[buf][kk][tid & 127], v ? A + (int64_t)a + t.ak[k] : A, v ? 4 : 0);
      }
    } else {  // A: k = tid % 16, m = tid / 16 + 16 i
      const int kk = tid & 15, k = k0 + kk;
      const bool kv = k < ke;
      const int ao = kv ? t.ak[k] : 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int mm = (tid >> 4) + 16 * i, a = am_s[mm];
        const bool v = kv && a >= 0;
        sg_acopy(&As[buf][kk][mm], v ? A + (int64_t)a + ao : A, v ? 4 : 0);
      }
    }
    if (sh.b_nfast) {  // B: n = tid % 64, k = tid / 64 + 4 i
      const int b = bn_s[tid & 63];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int kk = (tid >> 6) + 4 * i, k = k0 + kk;
        const bool v = k < ke && b >= 0;
        sg_acopy(&Bs[buf][kk][tid & 63], v ? B + (int64_t)b + t.bk[k] : B, v ? 4 : 0);
      }
    } else {  // B: k = tid % 16, n = tid / 16 + 16 i
      const int kk = tid & 15, k = k0 + kk;
      const bool kv = k < ke;
      const int bo = kv ? t.bk[k] : 0;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int nn = (tid >> 4) + 16 * i, b = bn_s[nn];
        const bool v = kv && b >= 0;
        sg_acopy(&Bs[buf][kk][nn], v ? B + (int64_t)b + bo : B, v ? 4 : 0);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  const int nsteps = ke > kb ? (ke - kb + SG_BK - 1) / SG_BK : 0;
  // prologue: stages 0 .. SG_ST - 2 (empty groups keep the wait counts uniform)
#pragma unroll
  for (int st = 0; st < SG_ST - 1; ++st) {
    if (st < nsteps)
      issue(kb + st * SG_BK, st);
    else
      asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  for (int i = 0; i < nsteps; ++i) {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(SG_ST - 2) : "memory");
    __syncthreads();  // stage i visible to all; stage (i - 1) % SG_ST free for reuse
    if (i + SG_ST - 1 < nsteps)
      issue(kb + (i + SG_ST - 1) * SG_BK, (i + SG_ST - 1) % SG_ST);
    else
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    const int buf = i % SG_ST;
#pragma unroll
    for (int kk = 0; kk < SG_BK; ++kk) {
      const float4 a0 = *(const float4*)&As[buf][kk][ty * 4];
      const float4 a1 = *(const float4*)&As[buf][kk][64 + ty * 4];
      const float4 b = *(const float4*)&Bs[buf][kk][tx * 4];
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int ii = 0; ii < 8; ++ii)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[ii][j] = fmaf(av[ii], bv[j], acc[ii][j]);
    }
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  // this thread's four columns: one 16-byte store per row when they are
  // consecutive in the output (and aligned), else element by element
  const int nb = n0 + tx * 4;
  int cn4[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) cn4[j] = (nb + j < sh.N) ? t.cn[nb + j] : -1;
  const bool run4 = sh.ksplit == 1 && nb + 3 < sh.N && cn4[1] == cn4[0] + 1 && cn4[2] == cn4[0] + 2 &&
                    cn4[3] == cn4[0] + 3;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int mm = (i < 4) ? ty * 4 + i : 64 + ty * 4 + (i - 4);
    const int m = m0 + mm;
    if (m >= sh.M) continue;
    float v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = sh.round_tf32 ? sg_tf32(acc[i][j]) : acc[i][j];
    if (sh.ksplit == 1) {
      float* o = C + (int64_t)t.cm[m];
      if (run4 && (((uintptr_t)(o + cn4[0])) & 15) == 0) {
        *reinterpret_cast<float4*>(o + cn4[0]) = make_float4(v[0], v[1], v[2], v[3]);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (cn4[j] >= 0) o[cn4[j]] = v[j];
      }
    } else {
      float* o = part + ((int64_t)blockIdx.z * sh.M + m) * sh.N + nb;
      if (nb + 3 < sh.N && (((uintptr_t)o) & 15) == 0) {
        *reinterpret_cast<float4*>(o) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (nb + j < sh.N) o[j] = acc[i][j];
      }
    }
  }
}

// C[cm[m] + cn[n]] = sum over the K split (in split order, compensated) of the partials.
__global__ void k_sg_reduce(SgShape sh, SgTabs t, const float* __restrict__ part, float* __restrict__ C) {
  pdl_prologue();
  const int64_t MN = (int64_t)sh.M * sh.N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < MN; e += (int64_t)gridDim.x * blockDim.x) {
    const float s = split_sum(part, sh.ksplit, MN, e);
    const int m = (int)(e / sh.N), n = (int)(e - (int64_t)m * sh.N);
    C[(int64_t)t.cm[m] + t.cn[n]] = sh.round_tf32 ? sg_tf32(s) : s;
  }
}

// Yd = Yraw + rho * A_old (Eq. 5 right-hand side), Ys = float(Yd); n = I s.
__global__ void k_finish_rhs(const float* __restrict__ Yraw, const double* __restrict__ Aold, double rho,
                             double* __restrict__ Yd, float* __restrict__ Ys, int64_t n) {
  pdl_prologue();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double y = (double)Yraw[e] + rho * Aold[e];
    Yd[e] = y;
    Ys[e] = (float)y;
  }
}

// Gd = double(Gs), symmetrised ((G + G^T) / 2 in FP32 first, so that Gs and
// Gd hold the same symmetric matrix); s x s.
__global__ void k_finish_gram(float* __restrict__ Gs, double* __restrict__ Gd, int s) {
  pdl_prologue();
  const int64_t n = (int64_t)s * s;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / s), j = (int)(e - (int64_t)i * s);
    if (j < i) continue;
    const float v = 0.5f * (Gs[(int64_t)i * s + j] + Gs[(int64_t)j * s + i]);
    Gs[(int64_t)i * s + j] = v;
    Gs[(int64_t)j * s + i] = v;
    Gd[(int64_t)i * s + j] = v;
    Gd[(int64_t)j * s + i] = v;
  }
}

// dst[c * ldd + r] = round(src[r * lds + c]) for r < rows, c < cols (dst
// entries r >= rows of a padded leading dimension are not written).
// Rounding: 0 = none, 1 = to nearest TF32 (kept in FP32 storage).
__global__ void k_transpose_round(const float* __restrict__ src, int64_t rows, int64_t cols, int64_t lds,
                                  float* __restrict__ dst, int64_t ldd, int round) {
  pdl_prologue();
  __shared__ float tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t r = r0 + i, c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < rows && c < cols) ? src[r * lds + c] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t c = c0 + i, r = r0 + threadIdx.x;
    if (c < cols && r < rows) {
      float v = tile[threadIdx.x][i];
      if (round) {
        uint32_t u;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(v));
        v = __uint_as_float(u);
      }
      dst[c * ldd + r] = v;
    }
  }
}

// dst[r * ldd + c] = round(src[r * lds + c]) (a padded, optionally rounded copy).
__global__ void k_copy_round(const float* __restrict__ src, int64_t rows, int64_t cols, int64_t lds,
                             float* __restrict__ dst, int64_t ldd, int round) {
  pdl_prologue();
  const int64_t n = rows * ldd;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / ldd, c = e - r * ldd;
    float v = c < cols ? src[r * lds + c] : 0.f;
    if (round) {
      uint32_t u;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(v));
      v = __uint_as_float(u);
    }
    dst[e] = v;
  }
}

// BF16 copies of the same two kinds (operands of the BF16 tensor-core GEMMs).
__global__ void k_transpose_bf16(const float* __restrict__ src, int64_t rows, int64_t cols, int64_t lds,
                                 __nv_bfloat16* __restrict__ dst, int64_t ldd) {
  pdl_prologue();
  __shared__ float tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t r = r0 + i, c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < rows && c < cols) ? src[r * lds + c] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t c = c0 + i, r = r0 + threadIdx.x;
    if (c < cols && r < rows) dst[c * ldd + r] = __float2bfloat16_rn(tile[threadIdx.x][i]);
  }
}

__global__ void k_copy_bf16(const float* __restrict__ src, int64_t rows, int64_t cols, int64_t lds,
                            __nv_bfloat16* __restrict__ dst, int64_t ldd) {
  pdl_prologue();
  const int64_t n = rows * ldd;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / ldd, c = e - r * ldd;
    dst[e] = __float2bfloat16_rn(c < cols ? src[r * lds + c] : 0.f);
  }
}

int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  return (int)(b < 4 * 152 ? (b < 1 ? 1 : b) : 4 * 152);
}

}  // namespace

void sg_shape(int M, int N, int K, SgShape* sh, int split_ctas) {
  sh->a_mfast = sh->b_nfast = 0;
  sh->round_tf32 = 0;
  sh->M = M;
  sh->N = N;
  sh->K = K;
  const int tiles = ((M + SG_BM - 1) / SG_BM) * ((N + SG_BN - 1) / SG_BN);
  int ks = 1;
  // split K when the tiles alone would leave most SMs idle and K is long:
  // about split_ctas CTAs in all (0 = two per SM, 1 = no split)
  const int target = split_ctas > 0 ? split_ctas : 2 * 152;
  if (tiles < target && K >= 8 * SG_BK) {
    ks = (target + tiles - 1) / tiles;
    const int maxks = K / (4 * SG_BK);
    ks = ks < maxks ? ks : maxks;
    if (ks < 1) ks = 1;
  }
  int chunk = (K + ks - 1) / ks;
  chunk = (chunk + SG_BK - 1) / SG_BK * SG_BK;
  sh->kchunk = chunk > 0 ? chunk : SG_BK;
  sh->ksplit = K > 0 ? (K + sh->kchunk - 1) / sh->kchunk : 1;
}

size_t sg_part_elems(const SgShape& sh) { return sh.ksplit > 1 ? (size_t)sh.ksplit * sh.M * sh.N : 0; }

void launch_sgemm(const SgShape& sh, const SgTabs& t, const float* A, const float* B, float* C, float* part,
                  cudaStream_t st) {
  if (sh.M <= 0 || sh.N <= 0) return;
  dim3 grid((sh.M + SG_BM - 1) / SG_BM, (sh.N + SG_BN - 1) / SG_BN, sh.ksplit);
  launch_pdl(k_sgemm, grid, dim3(SG_THREADS), 0, st, sh, t, A, B, C, part);
  if (sh.ksplit > 1) {
    const int64_t mn = (int64_t)sh.M * sh.N;
    launch_pdl(k_sg_reduce, grid_for(mn, 256), dim3(256), 0, st, sh, t, part, C);
  }
}

void launch_sg_reduce(const SgShape& sh, const SgTabs& t, const float* part, float* C, cudaStream_t st) {
  launch_pdl(k_sg_reduce, grid_for((int64_t)sh.M * sh.N, 256), dim3(256), 0, st, sh, t, part, C);
}

void launch_finish_rhs(const float* Yraw, const double* Aold, double rho, double* Yd, float* Ys, int64_t n,
                       cudaStream_t st) {
  launch_pdl(k_finish_rhs, grid_for(n, 256), dim3(256), 0, st, Yraw, Aold, rho, Yd, Ys, n);
}

void launch_finish_gram(float* Gs, double* Gd, int s, cudaStream_t st) {
  launch_pdl(k_finish_gram, grid_for((int64_t)s * s, 256), dim3(256), 0, st, Gs, Gd, s);
}

void launch_transpose_f32(const float* src, int64_t rows, int64_t cols, int64_t lds, float* dst, int64_t ldd,
                          int round_tf32, cudaStream_t st) {
  dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
  launch_pdl(k_transpose_round, grid, dim3(32, 8), 0, st, src, rows, cols, lds, dst, ldd, round_tf32);
}

void launch_copy_f32(const float* src, int64_t rows, int64_t cols, int64_t lds, float* dst, int64_t ldd,
                     int round_tf32, cudaStream_t st) {
  launch_pdl(k_copy_round, grid_for(rows * ldd, 256), dim3(256), 0, st, src, rows, cols, lds, dst, ldd, round_tf32);
}

void launch_transpose_bf16(const float* src, int64_t rows, int64_t cols, int64_t lds, __nv_bfloat16* dst,
                           int64_t ldd, cudaStream_t st) {
  dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
  launch_pdl(k_transpose_bf16, grid, dim3(32, 8), 0, st, src, rows, cols, lds, dst, ldd);
}

void launch_copy_bf16(const float* src, int64_t rows, int64_t cols, int64_t lds, __nv_bfloat16* dst, int64_t ldd,
                      cudaStream_t st) {
  launch_pdl(k_copy_bf16, grid_for(rows * ldd, 256), dim3(256), 0, st, src, rows, cols, lds, dst, ldd);
}
