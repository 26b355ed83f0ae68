// Reduction of the split-K Gram / right-hand-side partials of Eq. 5, and the
// X update of Eq. 10 from a materialised merged tensor (CUDA-core path).
//
// reduce:   every chunk of columns of M_k wrote its own partial of
//           D = M_k [M_k ; X_(k)]^T; they are summed in a fixed order
//           (deterministic: a rerun gives identical bytes).
// xupdate:  F = A_k(k) M_k (the reuse path of Algorithm 2, where M_k is the
//           merged tensor of the factor updated last, kept from its update)
//           fused with the masked proximal update of Eq. 10 and the
//           stop-test reductions.
#include <cooperative_groups.h>

#include "fctn_internal.cuh"
#include "fctn_tile.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int TM = 64, TN = 64, TK = 32, NT = 256;

__device__ __forceinline__ int64_t xaddr(const ModeView& v, int64_t i, int64_t j) {
  // j < 2^32 always (P_k = P / I_k with P < 2^40 and I_k >= 1 is checked on the host)
  uint32_t jj = (uint32_t)j, post = (uint32_t)v.post;
  uint32_t a = jj / post, b = jj - a * post;
  return ((int64_t)a * v.I + i) * v.post + b;
}

template <typename T>
__global__ void k_reduce_gram_rhs(const T* __restrict__ part, GramPlan g, const double* __restrict__ A_old,
                                  double rho, double* __restrict__ Gd, double* __restrict__ Yd,
                                  float* __restrict__ Gs, float* __restrict__ Ys) {
  const int64_t total = g.s * g.ncols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    // fixed-order compensated (Kahan) sum in the partials' precision
    T sum = 0, comp = 0;
    for (int z = 0; z < g.ksplit; ++z) {
      T y = part[(int64_t)z * total + e] - comp;
      T t = sum + y;
      comp = (t - sum) - y;
      sum = t;
    }
    double acc = (double)sum;
    int64_t row = e / g.ncols, col = e % g.ncols;
    if (col < g.gcols) {
      Gd[row * g.s + col] = acc;
      if (Gs) Gs[row * g.s + col] = (float)acc;
    } else {
      int64_t i = col - g.gcols;
      double y = acc + rho * A_old[i * g.s + row];
      Yd[i * g.s + row] = y;
      if (Ys) Ys[i * g.s + row] = (float)y;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(NT) k_xupdate(const T* __restrict__ Ak, const T* __restrict__ M,
                                                T* __restrict__ X, const uint32_t* __restrict__ bits, double rho,
                                                GramPlan g, double* __restrict__ red) {
  // As, Bs for the product; afterwards the F tile (64 x 65) in their place
  constexpr int kAB = 2 * TK * (TM + 4), kF = 64 * 65;
  __shared__ __align__(16) T sbuf[kAB > kF ? kAB : kF];
  T(*As)[TM + 4] = reinterpret_cast<T(*)[TM + 4]>(sbuf);
  T(*Bs)[TN + 4] = reinterpret_cast<T(*)[TN + 4]>(sbuf + TK * (TM + 4));
  __shared__ double sred[3][NT / 32];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int64_t i0 = (int64_t)blockIdx.y * TM;
  const int64_t j0 = (int64_t)blockIdx.x * TN;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0;
  for (int64_t k0 = 0; k0 < g.s; k0 += TK) {
    for (int e = tid; e < TM * TK; e += NT) {
      int r = e / TK, kk = e % TK;
      int64_t i = i0 + r, sg = k0 + kk;
      As[kk][r] = (i < g.I && sg < g.s) ? Ak[i * g.s + sg] : (T)0;
    }
    for (int e = tid; e < TN * TK; e += NT) {
      int c = e % TN, kk = e / TN;
      int64_t j = j0 + c, sg = k0 + kk;
      Bs[kk][c] = (j < g.Pk && sg < g.s) ? M[sg * g.Pk + j] : (T)0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < TK; ++kk) {
      T av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[kk][ty * 4 + a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx * 4 + b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
  T d2 = 0, x2 = 0, r2 = 0;
  fctn_tile::xupdate_tile<T>(acc, sbuf, i0, j0, g, X, bits, rho, d2, x2, r2);
  double v[3] = {(double)d2, (double)x2, (double)r2};
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    double t = v[q];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((tid & 31) == 0) sred[q][tid >> 5] = t;
  }
  __syncthreads();
  if (tid < 3) {
    double t = 0.0;
    for (int w = 0; w < NT / 32; ++w) t += sred[tid][w];
    int64_t blk = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    red[blk * 3 + tid] = t;
  }
}

unsigned rgrid(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > 152 * 4) b = 152 * 4;
  return (unsigned)b;
}


// ---- Gram of M_k from the Grams of its pair operands (FactGram) -------------
// H = F F^T, F[r][j] = Src[col[j] + roff[r]] (r < rows, j < J), for both
// operands in one launch: one cluster of OG_SPLIT CTAs per 64 x 64 tile of H
// (the tiles of HL, then those of HR).  CTA q of a cluster sums its share of
// the columns j in chunks of 32 gathered into shared memory (the next chunk's
// gathers in flight while the current one is consumed); the cluster then adds
// the OG_SPLIT partial tiles through distributed shared memory, CTA q
// reducing rows 8q..8q+7 of the tile in rank order (a fixed summation order).
constexpr int OG_SPLIT = 8;

template <typename T>
__global__ void __cluster_dims__(OG_SPLIT, 1, 1) __launch_bounds__(256)
    k_op_gram(const T* __restrict__ SrcL, const int* __restrict__ roffL, const int* __restrict__ colL, int rowsL,
              int JL, T* __restrict__ HL, const T* __restrict__ SrcR, const int* __restrict__ roffR,
              const int* __restrict__ colR, int rowsR, int JR, T* __restrict__ HR) {
  constexpr int BJ = 32;
  __shared__ __align__(16) T Fs[2 * BJ * 64];  // the two gathered chunks, then the partial tile
  T* Fa = Fs;
  T* Fb = Fs + BJ * 64;
  cg::cluster_group cluster = cg::this_cluster();
  const int q = (int)cluster.block_rank();
  const int tile = blockIdx.x / OG_SPLIT;
  const int txL = (rowsL + 63) / 64, ntL = txL * txL;
  const bool isL = tile < ntL;
  const T* Src = isL ? SrcL : SrcR;
  const int* roff = isL ? roffL : roffR;
  const int* col = isL ? colL : colR;
  const int rows = isL ? rowsL : rowsR, J = isL ? JL : JR;
  T* H = isL ? HL : HR;
  const int tx_ = (rows + 63) / 64, t = isL ? tile : tile - ntL;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int r0 = (t / tx_) * 64, c0 = (t % tx_) * 64;
  const int per = (J + OG_SPLIT - 1) / OG_SPLIT, jb = min(J, q * per), je = min(J, jb + per);
  const int rr = tid % 64, jq = tid / 64;  // gathers rows r0 + rr and c0 + rr at columns j0 + jq + 4u
  const int oa = r0 + rr < rows ? roff[r0 + rr] : -1;
  const int ob = c0 + rr < rows ? roff[c0 + rr] : -1;
  T va[8], vb[8];
  auto gather = [&](int j0) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int j = j0 + jq + 4 * u;
      const int o = j < je ? col[j] : -1;
      va[u] = (o >= 0 && oa >= 0) ? Src[(int64_t)o + oa] : (T)0;
      vb[u] = (o >= 0 && ob >= 0) ? Src[(int64_t)o + ob] : (T)0;
    }
  };
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0;
  if (jb < je) gather(jb);
  for (int j0 = jb; j0 < je; j0 += BJ) {
    __syncthreads();  // the previous chunk is consumed
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      Fa[(jq + 4 * u) * 64 + rr] = va[u];
      Fb[(jq + 4 * u) * 64 + rr] = vb[u];
    }
    __syncthreads();
    if (j0 + BJ < je) gather(j0 + BJ);
    const int nb = min(BJ, je - j0);
    for (int jj = 0; jj < nb; ++jj) {
      T av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        av[a] = Fa[jj * 64 + ty * 4 + a];
        bv[a] = Fb[jj * 64 + tx * 4 + a];
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
  }
  __syncthreads();  // the last chunk is consumed: Fs takes the partial tile
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) Fs[(ty * 4 + a) * 64 + tx * 4 + b] = acc[a][b];
  cluster.sync();
  for (int e = tid; e < 8 * 64; e += blockDim.x) {
    const int rl = 8 * q + e / 64, c = e % 64;
    T v = 0;
    for (int rk = 0; rk < OG_SPLIT; ++rk) v += cluster.map_shared_rank(Fs, rk)[rl * 64 + c];
    const int r = r0 + rl, cc = c0 + c;
    if (r < rows && cc < rows) H[(int64_t)r * rows + cc] = v;
  }
  cluster.sync();  // every partial tile stays in place until the cluster has read it
}

// G[sigma, sigma'] = sum_{kappa, kappa'} HL[a K + kappa, a' K + kappa'] HR[b K + kappa, b' K + kappa']
// with a = a_of[sigma], b = b_of[sigma] (FactGram); into Gd (FP64) and Gs.
template <typename T>
__global__ void k_gram_combine(const T* __restrict__ HL, const T* __restrict__ HR, const int* __restrict__ a_of,
                               const int* __restrict__ b_of, int s, int K, int rl, int rr, double* __restrict__ Gd,
                               float* __restrict__ Gs) {
  const int64_t total = (int64_t)s * s;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int sg = (int)(e / s), sg2 = (int)(e % s);
    const T* hl = HL + (int64_t)a_of[sg] * K * rl + (int64_t)a_of[sg2] * K;
    const T* hr = HR + (int64_t)b_of[sg] * K * rr + (int64_t)b_of[sg2] * K;
    T acc = 0;
    for (int q = 0; q < K; ++q)
      for (int q2 = 0; q2 < K; ++q2) acc = fma(hl[(int64_t)q * rl + q2], hr[(int64_t)q * rr + q2], acc);
    Gd[e] = (double)acc;
    if (Gs) Gs[e] = (float)acc;
  }
}

template <typename T>
void fact_gram(const FactGram& f, const T* L, const T* R, T* HL, T* HR, int s, double* Gd, float* Gs,
               cudaStream_t st) {
  const int* offL = f.tab;
  const int* offR = offL + f.rl;
  const int* a_of = offR + f.rr;
  const int* b_of = a_of + s;
  const int* colL = b_of + s;
  const int* colR = colL + f.JL;
  const int tl = (f.rl + 63) / 64, tr = (f.rr + 63) / 64;
  k_op_gram<T><<<(tl * tl + tr * tr) * OG_SPLIT, 256, 0, st>>>(L, offL, colL, f.rl, f.JL, HL, R, offR, colR, f.rr,
                                                                f.JR, HR);
  k_gram_combine<T><<<rgrid((int64_t)s * s), 256, 0, st>>>(HL, HR, a_of, b_of, s, f.K, f.rl, f.rr, Gd, Gs);
}

}  // namespace

void launch_reduce_gram_rhs_f32(const float* partials, const GramPlan& g, const double* A_old, double rho,
                                double* Gd, double* Yd, float* Gs, float* Ys, cudaStream_t s) {
  k_reduce_gram_rhs<float><<<rgrid(g.s * g.ncols), 256, 0, s>>>(partials, g, A_old, rho, Gd, Yd, Gs, Ys);
}
void launch_reduce_gram_rhs_f64(const double* partials, const GramPlan& g, const double* A_old, double rho,
                                double* Gd, double* Yd, cudaStream_t s) {
  k_reduce_gram_rhs<double><<<rgrid(g.s * g.ncols), 256, 0, s>>>(partials, g, A_old, rho, Gd, Yd, nullptr, nullptr);
}
int xupdate_blocks(const GramPlan& g) {
  return (int)(((g.Pk + TN - 1) / TN) * ((g.I + TM - 1) / TM));
}
void launch_xupdate_f32(const float* Ak, const float* M, float* X, const uint32_t* bits, double rho,
                        const GramPlan& g, double* red, cudaStream_t s) {
  dim3 grid((unsigned)((g.Pk + TN - 1) / TN), (unsigned)((g.I + TM - 1) / TM));
  k_xupdate<float><<<grid, NT, 0, s>>>(Ak, M, X, bits, rho, g, red);
}
void launch_xupdate_f64(const double* Ak, const double* M, double* X, const uint32_t* bits, double rho,
                        const GramPlan& g, double* red, cudaStream_t s) {
  dim3 grid((unsigned)((g.Pk + TN - 1) / TN), (unsigned)((g.I + TM - 1) / TM));
  k_xupdate<double><<<grid, NT, 0, s>>>(Ak, M, X, bits, rho, g, red);
}

void launch_fact_gram_f32(const FactGram& f, const float* L, const float* R, float* HL, float* HR, int s, double* Gd,
                          float* Gs, cudaStream_t st) {
  fact_gram<float>(f, L, R, HL, HR, s, Gd, Gs, st);
}
void launch_fact_gram_f64(const FactGram& f, const double* L, const double* R, double* HL, double* HR, int s,
                          double* Gd, cudaStream_t st) {
  fact_gram<double>(f, L, R, HL, HR, s, Gd, nullptr, st);
}
