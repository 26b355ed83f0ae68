// Generic tensor contraction / permutation, L_k eigenbasis, input staging.
//
// k_contract evaluates one contraction of Definition 3 (or a transposition,
// Definition 1, when B is null) through a mixed-radix index plan.  It forms
// the pair intermediates and merged tensors M_k of Algorithms 1/2 and the
// full FCTN contraction of the FCTN format.
#include "fctn_internal.cuh"

namespace {

// Offsets of the contracted index q into A and B, in shared memory.
template <typename T>
__device__ __forceinline__ void con_table(const ContractPlan& p, int32_t* offA, int32_t* offB) {
  for (int64_t q = threadIdx.x; q < p.con_size; q += blockDim.x) {
    int64_t r = q, oa = 0, ob = 0;
    for (int d = p.ncon - 1; d >= 0; --d) {
      int64_t e = p.con_ext[d];
      int64_t dig = r % e;
      r /= e;
      oa += dig * p.ca_str[d];
      ob += dig * p.cb_str[d];
    }
    offA[q] = (int32_t)oa;
    offB[q] = (int32_t)ob;
  }
  __syncthreads();
}

// One warp per run of the innermost output digit: the outer digits are
// decoded once per run, lanes walk the innermost digit (coalesced stores).
template <typename T>
__global__ void __launch_bounds__(256) k_contract_rows(const T* __restrict__ A, const T* __restrict__ B,
                                                       T* __restrict__ out, ContractPlan p) {
  __shared__ int32_t offA[FCTN_CON_TABLE];
  __shared__ int32_t offB[FCTN_CON_TABLE];
  if (B) con_table<T>(p, offA, offB);
  const int lane = threadIdx.x & 31;
  const int last = p.nout - 1;
  const int64_t E = p.out_ext[last];
  const int64_t sa = p.a_str[last], sb = p.b_str[last];
  const int64_t rows = p.out_size / E;
  const int64_t K = p.con_size;
  const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); r < rows; r += wstride) {
    int64_t rr = r, ao = 0, bo = 0;
    for (int d = last - 1; d >= 0; --d) {
      int64_t e = p.out_ext[d];
      int64_t dig = rr % e;
      rr /= e;
      ao += dig * p.a_str[d];
      bo += dig * p.b_str[d];
    }
    T* o = out + r * E;
    for (int64_t e = lane; e < E; e += 32) {
      const T* a = A + ao + e * sa;
      if (B == nullptr) {
        o[e] = a[0];
      } else {
        const T* b = B + bo + e * sb;
        T acc = 0;
        for (int64_t q = 0; q < K; ++q) acc = fma(a[offA[q]], b[offB[q]], acc);
        o[e] = acc;
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_contract(const T* __restrict__ A, const T* __restrict__ B,
                                                  T* __restrict__ out, ContractPlan p) {
  __shared__ int32_t offA[FCTN_CON_TABLE];
  __shared__ int32_t offB[FCTN_CON_TABLE];
  if (B) con_table<T>(p, offA, offB);
  const int64_t K = p.con_size;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < p.out_size; o += stride) {
    int64_t r = o, ao = 0, bo = 0;
    for (int d = p.nout - 1; d >= 0; --d) {
      int64_t e = p.out_ext[d];
      int64_t dig = r % e;
      r /= e;
      ao += dig * p.a_str[d];
      bo += dig * p.b_str[d];
    }
    if (B == nullptr) {
      out[o] = A[ao];
    } else {
      T acc = 0;
      const T* a = A + ao;
      const T* b = B + bo;
      for (int64_t q = 0; q < K; ++q) acc = fma(a[offA[q]], b[offB[q]], acc);
      out[o] = acc;
    }
  }
}

template <typename T>
void contract(const T* A, const T* B, T* out, const ContractPlan& p, cudaStream_t s) {
  if (p.out_size == 0) return;
  const int64_t E = p.out_ext[p.nout - 1];
  if (E >= 16) {
    int64_t rows = p.out_size / E;
    int64_t blocks = (rows + 7) / 8;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_contract_rows<T><<<(unsigned)blocks, 256, 0, s>>>(A, B, out, p);
  } else {
    int64_t blocks = (p.out_size + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_contract<T><<<(unsigned)blocks, 256, 0, s>>>(A, B, out, p);
  }
}

// Real orthonormal eigenbasis of the symmetric circulant L_k (Eq. 7 with the
// DFT replaced by its real cos/sin form).  Column 0: constant; columns
// (2j-1, 2j): cos / sin of frequency j; for even I the last column is the
// alternating vector.  Eigenvalue of frequency j: sgn*(2 + delta - 2cos(2 pi j/I)),
// which also covers I <= 2 where the stencil entries add up.
__global__ void k_laplacian_basis(int64_t I, double delta, int sign, double* Q, float* Qf, double* QT, float* QTf,
                                  double* Lam) {
  const double sgn = sign == FCTN_LAPLACIAN_PRINTED ? -1.0 : 1.0;
  const int64_t total = I * I;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t n = e / I, col = e % I;
    double v;
    if (col == 0) {
      v = rsqrt((double)I);
    } else if ((I % 2 == 0) && col == I - 1) {
      v = (n % 2 == 0 ? 1.0 : -1.0) * rsqrt((double)I);
    } else {
      int64_t j = (col + 1) / 2;
      int64_t m = (j * n) % I;
      double arg = 2.0 * (double)m / (double)I;
      v = sqrt(2.0 / (double)I) * ((col % 2 == 1) ? cospi(arg) : sinpi(arg));
    }
    Q[e] = v;
    if (Qf) Qf[e] = (float)v;
    if (QT) QT[col * I + n] = v;
    if (QTf) QTf[col * I + n] = (float)v;
    if (n == 0) {
      int64_t j = (col == 0) ? 0 : ((I % 2 == 0 && col == I - 1) ? I / 2 : (col + 1) / 2);
      Lam[col] = sgn * (2.0 + delta - 2.0 * cospi(2.0 * (double)j / (double)I));
    }
  }
}

template <typename T>
__global__ void k_init_x_mask(const T* __restrict__ Y, const uint8_t* __restrict__ mask, T* __restrict__ X,
                              uint32_t* __restrict__ bits, int64_t n) {
  // one warp per 32 consecutive elements -> one mask word
  const int64_t nw = (n + 31) / 32;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = warp; w < nw; w += nwarps) {
    int64_t e = w * 32 + lane;
    bool obs = false;
    if (e < n) {
      obs = mask[e] != 0;
      X[e] = obs ? Y[e] : (T)0;
    }
    uint32_t b = __ballot_sync(0xffffffffu, obs);
    if (lane == 0) bits[w] = b;
  }
}

template <typename A, typename B>
__global__ void k_convert(const A* __restrict__ in, B* __restrict__ out, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (B)in[e];
}

unsigned grid_for(int64_t n, int per = 256) {
  int64_t b = (n + per - 1) / per;
  if (b < 1) b = 1;
  if (b > 152 * 8) b = 152 * 8;
  return (unsigned)b;
}

}  // namespace

void launch_contract_f32(const float* A, const float* B, float* out, const ContractPlan& p, cudaStream_t s) {
  contract<float>(A, B, out, p, s);
}
void launch_contract_f64(const double* A, const double* B, double* out, const ContractPlan& p, cudaStream_t s) {
  contract<double>(A, B, out, p, s);
}
void launch_laplacian_basis(int64_t I, double delta, int sign, double* Q, float* Qf, double* QT, float* QTf, double* Lam,
                            cudaStream_t s) {
  k_laplacian_basis<<<grid_for(I * I), 256, 0, s>>>(I, delta, sign, Q, Qf, QT, QTf, Lam);
}
void launch_init_x_mask_f32(const float* Y, const uint8_t* mask, float* X, uint32_t* bits, int64_t n,
                            cudaStream_t s) {
  k_init_x_mask<float><<<grid_for(n), 256, 0, s>>>(Y, mask, X, bits, n);
}
void launch_init_x_mask_f64(const double* Y, const uint8_t* mask, double* X, uint32_t* bits, int64_t n,
                            cudaStream_t s) {
  k_init_x_mask<double><<<grid_for(n), 256, 0, s>>>(Y, mask, X, bits, n);
}
void launch_convert_f64_to_f32(const double* in, float* out, int64_t n, cudaStream_t s) {
  k_convert<double, float><<<grid_for(n), 256, 0, s>>>(in, out, n);
}
void launch_convert_f32_to_f64(const float* in, double* out, int64_t n, cudaStream_t s) {
  k_convert<float, double><<<grid_for(n), 256, 0, s>>>(in, out, n);
}
