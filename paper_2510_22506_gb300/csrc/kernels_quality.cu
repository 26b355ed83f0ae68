// Quality of a completed tensor against the ground truth (Sec. 4): PSNR and
// SSIM of every slice spanned by modes 1-2, averaged over the remaining
// indices.  The tensor is row-major (I_1, I_2, rest), so the slice index t is
// the position within a row of the (I_1 I_2) x T view.  Per-slice sums are
// accumulated in FP64 in a fixed order (blocks of rows, then blocks in order).
#include "fctn_internal.cuh"

namespace {

constexpr int QNT = 256;
constexpr int QS = 6;  // sums per slice: x, y, x^2, y^2, xy, (x - y)^2

// Block b: rows [b*rows_per, (b+1)*rows_per); thread (t, g) sums rows g, g+G,
// ... of column t; the G partials of a column are combined in order.
template <typename T>
__global__ void __launch_bounds__(QNT) k_slice_sums(const T* __restrict__ X, const T* __restrict__ Y, int64_t rows,
                                                    int64_t ncol, int64_t rows_per, double* __restrict__ part) {
  extern __shared__ double sh[];  // [G][ncol_chunk][QS]
  const int64_t r0 = (int64_t)blockIdx.x * rows_per;
  const int64_t r1 = min(rows, r0 + rows_per);
  const int G = ncol >= QNT ? 1 : QNT / (int)ncol;
  for (int64_t t0 = 0; t0 < ncol; t0 += QNT) {
    const int64_t nc = min((int64_t)QNT, ncol - t0);
    const int tc = threadIdx.x % (int)nc, g = threadIdx.x / (int)nc;
    double s[QS] = {0, 0, 0, 0, 0, 0};
    if (g < G && threadIdx.x < nc * G) {
      for (int64_t r = r0 + g; r < r1; r += G) {
        const double x = (double)X[r * ncol + t0 + tc], y = (double)Y[r * ncol + t0 + tc];
        const double d = x - y;
        s[0] += x;
        s[1] += y;
        s[2] = fma(x, x, s[2]);
        s[3] = fma(y, y, s[3]);
        s[4] = fma(x, y, s[4]);
        s[5] = fma(d, d, s[5]);
      }
      for (int q = 0; q < QS; ++q) sh[((int64_t)g * nc + tc) * QS + q] = s[q];
    }
    __syncthreads();
    if (threadIdx.x < nc) {
      double a[QS] = {0, 0, 0, 0, 0, 0};
      for (int gg = 0; gg < G; ++gg)
        for (int q = 0; q < QS; ++q) a[q] += sh[((int64_t)gg * nc + threadIdx.x) * QS + q];
      for (int q = 0; q < QS; ++q) part[((int64_t)blockIdx.x * ncol + t0 + threadIdx.x) * QS + q] = a[q];
    }
    __syncthreads();
  }
}

// One thread per slice: sums over the blocks in order, then the slice's PSNR
// (Max = 1, MSE floored at 1e-12) and SSIM; thread 0 then averages.
__global__ void k_slice_quality(const double* __restrict__ part, int nblocks, int64_t ncol, int64_t n, double c1,
                                double c2, double* __restrict__ per, double* __restrict__ out) {
  for (int64_t t = threadIdx.x; t < ncol; t += blockDim.x) {
    double a[QS] = {0, 0, 0, 0, 0, 0};
    for (int b = 0; b < nblocks; ++b)
      for (int q = 0; q < QS; ++q) a[q] += part[((int64_t)b * ncol + t) * QS + q];
    const double dn = (double)n;
    const double mx = a[0] / dn, my = a[1] / dn;
    const double den = n > 1 ? dn - 1.0 : 1.0;
    const double vx = (a[2] - dn * mx * mx) / den, vy = (a[3] - dn * my * my) / den;
    const double cxy = (a[4] - dn * mx * my) / den;
    const double ssim = ((2.0 * mx * my + c1) * (2.0 * cxy + c2)) / ((mx * mx + my * my + c1) * (vx + vy + c2));
    const double mse = a[5] / dn;
    per[2 * t] = 10.0 * log10(1.0 / fmax(mse, 1e-12));
    per[2 * t + 1] = ssim;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ps = 0.0, ss = 0.0;
    for (int64_t t = 0; t < ncol; ++t) {
      ps += per[2 * t];
      ss += per[2 * t + 1];
    }
    out[0] = ps / (double)ncol;
    out[1] = ss / (double)ncol;
  }
}

template <typename T>
void quality(const T* X, const T* Y, int64_t rows, int64_t ncol, double c1, double c2, double* work, int nblocks,
             double* out, cudaStream_t st) {
  const int64_t rows_per = (rows + nblocks - 1) / nblocks;
  const int nb = (int)((rows + rows_per - 1) / rows_per);
  const int64_t nc = ncol < QNT ? ncol : QNT;
  const int G = ncol >= QNT ? 1 : QNT / (int)ncol;
  const size_t smem = (size_t)G * nc * QS * sizeof(double);
  k_slice_sums<T><<<nb, QNT, smem, st>>>(X, Y, rows, ncol, rows_per, work);
  double* per = work + (size_t)nb * ncol * QS;
  k_slice_quality<<<1, 256, 0, st>>>(work, nb, ncol, rows, c1, c2, per, out);
}

}  // namespace

size_t quality_work_doubles(int64_t ncol, int nblocks) { return (size_t)nblocks * ncol * QS + 2 * (size_t)ncol; }

void launch_quality_f32(const float* X, const float* Y, int64_t rows, int64_t ncol, double c1, double c2,
                        double* work, int nblocks, double* out, cudaStream_t st) {
  quality<float>(X, Y, rows, ncol, c1, c2, work, nblocks, out, st);
}
void launch_quality_f64(const double* X, const double* Y, int64_t rows, int64_t ncol, double c1, double c2,
                        double* work, int nblocks, double* out, cudaStream_t st) {
  quality<double>(X, Y, rows, ncol, c1, c2, work, nblocks, out, st);
}
