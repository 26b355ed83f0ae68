// Cluster-parallel block-ordered Jacobi for the FP32 Gram eigendecomposition
// (Eq. 7): the method of k_eig3 / k_eig4 spread over a thread-block cluster
// of CL (4 to 8) CTAs.
//
// The index set is padded to m = 8 CL T and split into nb = m / 4 blocks;
// every outer round pairs the blocks by the round-robin schedule into
// nsub = nb / 2 subproblems ("tables"), T per CTA.  A CTA
// keeps the rows of B = V^T G V and of V^T for the blocks at its tables, over
// all m columns.  Per round:
//   1. each CTA rotates its tables' 8 x 8 subproblems (half a warp each, the
//      inner rounds of k_eig3) and stores their rotation blocks U into every
//      CTA's table list through distributed shared memory;
//   2. cluster barrier;
//   3. row update of its own rows (B and V^T): rows S_a <- U_a^T rows S_a;
//   4. column update of its own rows for every subproblem b: columns S_b <-
//      columns S_b U_b, the 8 x 8 superblocks of its own tables taken from the
//      rotated subproblems; the result is written straight into the row
//      slots of the CTA that holds the block in the next round (its own or a
//      neighbour's, through distributed shared memory), together with the
//      block's V^T rows;
//   5. cluster barrier; the slot buffers swap.
// B and V^T never leave the cluster between the warm-start products and the
// result.  Rotation and stop tests are those of k_eig4 (relative to the
// shifted diagonal); a sweep starts only if some pair would rotate.
#include <cooperative_groups.h>

#include <cstring>

#include "fctn_internal.cuh"
#include "fctn_jacobi.cuh"

namespace cg = cooperative_groups;
using namespace fctn_jacobi;

namespace {

constexpr int EC_MAXCL = 8;  // CTAs per cluster at most (portable cluster size)
constexpr int EC_NT = 256;   // threads per CTA
constexpr int EC_MAXM = 256;
constexpr int EC_UP = 68;    // floats per published block: U (64), rotated flag, pad

// m = 8 CL T >= s (CL CTAs, T tables each): the cluster size with the least
// padding (ties: the larger cluster), so that the rounds m / 4 - 1 of a sweep
// are as few as the index set allows: s = 216 -> 7 x 4 tables, m = 224.
struct EcDims {
  int CL, m, nb, nsub, T, rows, sp;
};
__host__ __device__ inline EcDims ec_dims(int s) {
  const int need = (s + 7) / 8;  // tables
  EcDims d{};
  int best = 1 << 30;
  for (int cl = EC_MAXCL; cl >= 4; --cl) {
    const int t = (need + cl - 1) / cl, m = 8 * cl * t;
    if (m < best) {
      best = m;
      d.CL = cl;
      d.T = t;
    }
  }
  d.m = 8 * d.CL * d.T;
  d.nb = d.m / 4;
  d.nsub = d.nb / 2;
  d.rows = 8 * d.T;
  d.sp = d.m + 4;
  return d;
}
__host__ __device__ inline size_t ec_smem_floats(int s) {
  const EcDims d = ec_dims(s);
  return (size_t)4 * d.rows * d.sp          // B and V^T, two slot buffers each
         + (size_t)d.nsub * EC_UP            // blocks of every table (pushed by their CTAs)
         + (size_t)(d.T + 1) * EJ_SUB;       // subproblems (and a spare slot)
}

__global__ void __launch_bounds__(EC_NT)
    k_eigc(const float* __restrict__ Bin, const float* __restrict__ Vin, float* __restrict__ Phi,
           float* __restrict__ C, int s, int max_sweeps, double tmin, double tol_in, int* status,
           int* sweeps_used) {
  cg::cluster_group cluster = cg::this_cluster();
  const int cr = (int)cluster.block_rank();
  const EcDims D = ec_dims(s);
  const int m = D.m, nb = D.nb, nsub = D.nsub, T = D.T, sp = D.sp, rows = D.rows, CL = D.CL;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarp = EC_NT >> 5;
  extern __shared__ __align__(16) float esm[];
  float* Bb[2] = {esm, esm + rows * sp};
  float* Vb[2] = {esm + 2 * rows * sp, esm + 3 * rows * sp};
  float* Uall = esm + 4 * rows * sp;
  float* SC = Uall + nsub * EC_UP;
  // the round-robin schedule of a sweep, once: blocks of every table per
  // round (P | Q << 16) and table * 2 + half of every block in the round after
  __shared__ int pq_tab[EC_MAXM / 4 - 1][EC_MAXM / 8];
  __shared__ int wn_tab[EC_MAXM / 4 - 1][EC_MAXM / 4];
  __shared__ float dpub[EC_MAXM / 8 * 8];  // published: diagonal of the own rows
  __shared__ float diag[EC_MAXM];          // gathered diagonal of B
  __shared__ float pub_fr;                 // published: share of ||B||_F^2
  __shared__ unsigned pub_cnt, pub_mx;     // published: rotations and largest ratio of a sweep
  __shared__ int pub_scan;                 // published: some own pair would rotate
  __shared__ float red[EC_NT / 32];
  __shared__ float gnorm;
  __shared__ int g_any;
  __shared__ unsigned g_cnt, g_mx;

  for (int e = tid; e < (nb - 1) * nsub; e += EC_NT) {
    const int rr = e / nsub, a = e - rr * nsub;
    int P, Q;
    round_pair(nb, rr, a, P, Q);
    pq_tab[rr][a] = P | Q << 16;
    const int rp = rr == 0 ? nb - 2 : rr - 1;  // round rr follows round rp
    wn_tab[rp][P] = 2 * a;
    wn_tab[rp][Q] = 2 * a + 1;
  }
  // ---- initial rows (round 0 of the first sweep)
  float fr = 0.f;
  for (int lr = warp; lr < rows; lr += nwarp) {
    const int a = cr * T + lr / 8, i = lr % 8;
    int P, Q;
    round_pair(nb, 0, a, P, Q);
    const int g = i < 4 ? 4 * P + i : 4 * Q + i - 4;  // global row
    for (int j = lane; j < m; j += 32) {
      float b = 0.f, v;
      if (g < s && j < s) b = 0.5f * (Bin[(int64_t)g * s + j] + Bin[(int64_t)j * s + g]);
      if (Vin) v = (g < s && j < s) ? Vin[(int64_t)j * s + g] : (g == j ? 1.f : 0.f);  // V^T[g][j] = V[j][g]
      else v = g == j ? 1.f : 0.f;
      Bb[0][lr * sp + j] = b;
      Vb[0][lr * sp + j] = v;
      fr = fmaf(b, b, fr);
    }
  }
  for (int o = 16; o > 0; o >>= 1) fr += __shfl_xor_sync(0xffffffffu, fr, o);
  if (lane == 0) red[warp] = fr;
  __syncthreads();
  if (tid == 0) {
    float t = 0.f;
    for (int w = 0; w < nwarp; ++w) t += red[w];
    pub_fr = t;
  }
  cluster.sync();
  if (tid == 0) {
    float t = 0.f;
    for (int q = 0; q < CL; ++q) t += *cluster.map_shared_rank(&pub_fr, q);
    gnorm = sqrtf(t);
  }
  __syncthreads();
  const float eps = FLT_EPSILON;
  const float tol = tol_in > 0.0 ? (float)tol_in : sqrtf((float)(s > 1 ? s : 1)) * eps, tol2 = tol * tol;
  const float floor_abs = eps * gnorm * rsqrtf((float)(s > 0 ? s : 1)), floor2 = floor_abs * floor_abs;
  const float tsh = tmin > 0.0 ? (float)tmin : 0.f;

  int cur = 0, sweep = 0, r = 0;
  bool converged = s <= 1;
  unsigned cnt = 0;
  float cmu = 0.f;
  const int nsw = (T + 1) / 2;  // warps with subproblems (two per warp)
  for (; sweep < max_sweeps && !converged; ++sweep) {
    // ---- scan: would any pair pass the rotation test?  (layout of round 0)
    for (int lr = tid; lr < rows; lr += EC_NT) {
      const int a = cr * T + lr / 8, i = lr % 8;
      int P, Q;
      round_pair(nb, 0, a, P, Q);
      const int g = i < 4 ? 4 * P + i : 4 * Q + i - 4;
      dpub[lr] = Bb[cur][lr * sp + g];
    }
    if (tid == 0) pub_scan = 0;
    cluster.sync();  // (A) diagonals published
    for (int e = tid; e < CL * rows; e += EC_NT) {
      const int q = e / rows, lr = e - q * rows;
      const int a = q * T + lr / 8, i = lr % 8;
      int P, Q;
      round_pair(nb, 0, a, P, Q);
      diag[i < 4 ? 4 * P + i : 4 * Q + i - 4] = cluster.map_shared_rank(dpub, q)[lr];
    }
    __syncthreads();
    {
      bool want = false;
      for (int e = tid; e < rows * m && !want; e += EC_NT) {
        const int lr = e / m, j = e - lr * m;
        const int a = cr * T + lr / 8, i = lr % 8;
        int P, Q;
        round_pair(nb, 0, a, P, Q);
        const int g = i < 4 ? 4 * P + i : 4 * Q + i - 4;
        if (j <= g || j >= s || g >= s) continue;
        const float b = Bb[cur][lr * sp + j];
        want = b * b > tol2 * (fabsf(diag[g]) + tsh) * (fabsf(diag[j]) + tsh) + floor2;
      }
      if (__any_sync(0xffffffffu, want) && lane == 0) atomicOr(&pub_scan, 1);
    }
    cluster.sync();  // (B) scan flags published
    if (tid == 0) {
      int any = 0;
      for (int q = 0; q < CL; ++q) any |= *cluster.map_shared_rank(&pub_scan, q);
      g_any = any;
      pub_cnt = 0u;  // nobody reads these until the end of the sweep
      pub_mx = 0u;
    }
    __syncthreads();
    const bool any_rot = g_any != 0;
    cluster.sync();  // (C) every flag read before the next sweep writes it
    if (!any_rot) {
      converged = true;
      break;
    }
    cnt = 0;
    cmu = 0.f;
    for (r = 0; r < nb - 1; ++r) {
      // ---- 1. subproblems of this CTA's tables
      const int* pq = pq_tab[r];
      const int* where_nxt = wn_tab[r];
      for (int sw = warp; sw < nsw; sw += nwarp) {
        const int al = 2 * sw + (lane >> 4), hl = lane & 15;
        const bool real = al < T;
        float* Sw = SC + (real ? al : T) * EJ_SUB;
        float* Uw = Sw + 64;
        int P = 0, Q = 0;
        if (real) {
          P = pq[cr * T + al] & 0xffff;
          Q = pq[cr * T + al] >> 16;
        }
        for (int e = hl; e < 64; e += 16) {
          const int i = e >> 3, j = e & 7;
          const int gj = j < 4 ? 4 * P + j : 4 * Q + j - 4;
          Sw[e] = real ? Bb[cur][(al * 8 + i) * sp + gj] : 0.f;
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
        if (real) {
          // push the block (and its rotated flag) into every CTA's copy of
          // the table list: remote stores do not wait for a round trip
          const int a = cr * T + al;
          const float4 u4 = *(const float4*)(Uw + 4 * hl);
          const float fl = ((any >> (lane & 16)) & 0xffffu) ? 1.f : 0.f;
#pragma unroll
          for (int q = 0; q < CL; ++q) {
            float* dst = cluster.map_shared_rank(Uall, q) + a * EC_UP;
            *(float4*)(dst + 4 * hl) = u4;
            if (hl == 0) dst[64] = fl;
          }
        }
      }
      cluster.sync();  // (#1) every table's block is in every CTA
      // ---- 3. row update of the own rows (B outside the own superblocks, V^T whole)
      for (int t = tid; t < 2 * T * (m / 4); t += EC_NT) {
        const int isv = t >= T * (m / 4), tt = isv ? t - T * (m / 4) : t;
        const int al = tt / (m / 4), cq = tt - al * (m / 4);
        const int a = cr * T + al;
        if (Uall[a * EC_UP + 64] == 0.f) continue;  // U_a = I
        const int P = pq[a] & 0xffff, Q = pq[a] >> 16;
        if (!isv && (cq == P || cq == Q)) continue;
        float* Mx = (isv ? Vb[cur] : Bb[cur]) + al * 8 * sp + 4 * cq;
        const float* Ua = Uall + a * EC_UP;
        float acc[8][4];
#pragma unroll
        for (int o = 0; o < 8; ++o) acc[o][0] = acc[o][1] = acc[o][2] = acc[o][3] = 0.f;
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const float4 x = *(const float4*)(Mx + kk * sp);
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
        for (int o = 0; o < 8; ++o) *(float4*)(Mx + o * sp) = make_float4(acc[o][0], acc[o][1], acc[o][2], acc[o][3]);
      }
      __syncthreads();
      // ---- 4. column update of the own rows into the next round's slots
      const int nxt = cur ^ 1;
      for (int t = tid; t < 2 * T * nsub; t += EC_NT) {
        const int rq = t / nsub, b = t - rq * nsub;  // own row quad, column table
        const int al = rq / 2, half = rq & 1;
        const int a = cr * T + al;
        const int Pa = pq[a] & 0xffff, Qa = pq[a] >> 16;
        const int blk = half ? Qa : Pa;                 // the block these four rows belong to
        const int wn = where_nxt[blk], ta = wn >> 1, th = wn & 1;
        float* dst = cluster.map_shared_rank(Bb[nxt], ta / T) + ((ta % T) * 8 + th * 4) * sp;
        const float* src = Bb[cur] + (al * 8 + half * 4) * sp;
        const int P = pq[b] & 0xffff, Q = pq[b] >> 16;
        if (b == a) {  // own superblock: the rotated subproblem
          const float* Sb = SC + al * EJ_SUB + half * 32;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            *(float4*)(dst + i * sp + 4 * P) = *(const float4*)(Sb + i * 8);
            *(float4*)(dst + i * sp + 4 * Q) = *(const float4*)(Sb + i * 8 + 4);
          }
        } else if (Uall[b * EC_UP + 64] == 0.f) {  // U_b = I: the rows move unchanged
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            *(float4*)(dst + i * sp + 4 * P) = *(const float4*)(src + i * sp + 4 * P);
            *(float4*)(dst + i * sp + 4 * Q) = *(const float4*)(src + i * sp + 4 * Q);
          }
        } else {
          const float* Ub = Uall + b * EC_UP;
          float u[64];
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const float4 t4 = *(const float4*)(Ub + 4 * e);
            u[4 * e] = t4.x, u[4 * e + 1] = t4.y, u[4 * e + 2] = t4.z, u[4 * e + 3] = t4.w;
          }
#pragma unroll
          for (int i = 0; i < 4; ++i) {  // one row at a time: out_j = sum_k w_k U[k][j]
            const float4 w0 = *(const float4*)(src + i * sp + 4 * P), w1 = *(const float4*)(src + i * sp + 4 * Q);
            const float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
            float o[8];
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
              float acc = 0.f;
#pragma unroll
              for (int kk = 0; kk < 8; ++kk) acc = fmaf(w[kk], u[kk * 8 + jj], acc);
              o[jj] = acc;
            }
            *(float4*)(dst + i * sp + 4 * P) = make_float4(o[0], o[1], o[2], o[3]);
            *(float4*)(dst + i * sp + 4 * Q) = make_float4(o[4], o[5], o[6], o[7]);
          }
        }
      }
      // V^T rows move with their block
      for (int t = tid; t < 2 * T * (m / 4); t += EC_NT) {
        const int rq = t / (m / 4), cq = t - rq * (m / 4);
        const int al = rq / 2, half = rq & 1;
        const int a = cr * T + al;
        const int blk = half ? (pq[a] >> 16) : (pq[a] & 0xffff);
        const int wn = where_nxt[blk], ta = wn >> 1, th = wn & 1;
        float* dst = cluster.map_shared_rank(Vb[nxt], ta / T) + ((ta % T) * 8 + th * 4) * sp + 4 * cq;
        const float* src = Vb[cur] + (al * 8 + half * 4) * sp + 4 * cq;
#pragma unroll
        for (int i = 0; i < 4; ++i) *(float4*)(dst + i * sp) = *(const float4*)(src + i * sp);
      }
      cluster.sync();  // (#2) the next round's rows are in place everywhere
      cur = nxt;
    }
    // ---- end of a sweep: rotations and largest ratio over the cluster
    if (warp < nsw) {
      const unsigned cn = __reduce_add_sync(0xffffffffu, cnt);
      const unsigned mx = __reduce_max_sync(0xffffffffu, __float_as_uint(cmu));  // cmu >= 0
      if (lane == 0) {
        atomicAdd(&pub_cnt, cn);
        atomicMax(&pub_mx, mx);
      }
    }
    cluster.sync();  // (D) sweep totals published
    if (tid == 0) {
      unsigned c = 0u, mx = 0u;
      for (int q = 0; q < CL; ++q) {
        c += *cluster.map_shared_rank(&pub_cnt, q);
        mx = max(mx, *cluster.map_shared_rank(&pub_mx, q));
      }
      g_cnt = c;
      g_mx = mx;
    }
    __syncthreads();
    converged = (g_cnt == 0u) || (__uint_as_float(g_mx) < tol);
    cluster.sync();  // (E) totals read everywhere before the next sweep resets them
  }
  // ---- results: eigenvalues (diagonal of B) and C = V (C[g][j] = V^T[j][g])
  float mn = 3.4e38f;
  for (int lr = warp; lr < rows; lr += nwarp) {
    const int a = cr * T + lr / 8, i = lr % 8;
    int P, Q;
    round_pair(nb, 0, a, P, Q);
    const int j = i < 4 ? 4 * P + i : 4 * Q + i - 4;  // global index of this row (round 0 layout)
    if (j >= s) continue;
    if (lane == 0) {
      const float ph = Bb[cur][lr * sp + j];
      Phi[j] = ph;
      mn = fminf(mn, ph);
    }
    for (int g = lane; g < s; g += 32) C[(int64_t)g * s + j] = Vb[cur][lr * sp + g];
  }
  if (lane == 0) red[warp] = mn;
  __syncthreads();
  if (tid == 0) {
    float t = red[0];
    for (int w = 1; w < nwarp; ++w) t = fminf(t, red[w]);
    if (!((double)t + tmin > 0.0)) atomicCAS(status, FCTN_OK, FCTN_E_SINGULAR);
    if (cr == 0 && sweeps_used) *sweeps_used = converged ? sweep : -sweep;
  }
}

}  // namespace

size_t eigc_smem_bytes(int s) { return ec_smem_floats(s) * sizeof(float); }

void launch_eigc(const float* Bin, const float* Vin, float* Phi, float* C, int s, int max_sweeps, double tmin,
                 double tol, int* status, int* used, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_eigc, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  const EcDims d = ec_dims(s);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(d.CL, 1, 1);
  cfg.blockDim = dim3(EC_NT, 1, 1);
  cfg.dynamicSmemBytes = eigc_smem_bytes(s);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = d.CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_eigc, Bin, Vin, Phi, C, s, max_sweeps, tmin, tol, status, used);
}
