// Subspace kernels of the ground-state iteration (tdks_ground_state): overlaps of two sets of
// orbitals and linear combinations of a set with a small matrix, per k-point.  Orbitals are
// [nk][norb][npts] complex (FP32 or FP64); matrices [nk][norb][norb] double2; sums in FP64.
#include <cuda_runtime.h>

#include "tdks_internal.h"

namespace tdks {

namespace {

constexpr int kGramThreads = 256;

// out[k][i][j] = dV sum_r conj(A[k][i][r]) B[k][j][r].  One CTA per (i, j, k), fixed-order tree.
template <typename T>
__global__ void __launch_bounds__(kGramThreads) k_gram(const typename Cplx<T>::type* __restrict__ A,
                                                      const typename Cplx<T>::type* __restrict__ B, int norb,
                                                      int npts, double dV, double2* __restrict__ out) {
  __shared__ double red[2 * kGramThreads];
  const int i = blockIdx.x / norb, j = blockIdx.x - i * norb, k = blockIdx.y;
  const auto* a = A + ((size_t)k * norb + i) * npts;
  const auto* b = B + ((size_t)k * norb + j) * npts;
  double re = 0.0, im = 0.0;
  for (int r = threadIdx.x; r < npts; r += blockDim.x) {
    const double ax = a[r].x, ay = a[r].y, bx = b[r].x, by = b[r].y;
    re += ax * bx + ay * by;
    im += ax * by - ay * bx;
  }
  red[threadIdx.x] = re;
  red[kGramThreads + threadIdx.x] = im;
  __syncthreads();
  for (int o = kGramThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[threadIdx.x] += red[threadIdx.x + o];
      red[kGramThreads + threadIdx.x] += red[kGramThreads + threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[((size_t)k * norb + i) * norb + j] = double2{red[0] * dV, red[kGramThreads] * dV};
}

// out[k][j][r] = a V[k][j][r] + c0 U[k][j][r] + b sum_i U[k][i][r] M[k][i][j]   (V may be NULL when a = 0).
// One thread per (grid point, k); the point's values of all orbitals of U are read once per j.
template <typename T>
__global__ void k_basis(const typename Cplx<T>::type* __restrict__ U, const typename Cplx<T>::type* __restrict__ V,
                        const double2* __restrict__ M, int norb, int npts, double a, double c0, double b,
                        typename Cplx<T>::type* __restrict__ out) {
  using C = typename Cplx<T>::type;
  const int k = blockIdx.y;
  const C* u = U + (size_t)k * norb * npts;
  const double2* m = M + (size_t)k * norb * norb;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < npts; r += gridDim.x * blockDim.x) {
    for (int j = 0; j < norb; ++j) {
      double sx = 0.0, sy = 0.0;
      for (int i = 0; i < norb; ++i) {
        const C ui = u[(size_t)i * npts + r];
        const double2 mij = m[i * norb + j];
        sx += (double)ui.x * mij.x - (double)ui.y * mij.y;
        sy += (double)ui.x * mij.y + (double)ui.y * mij.x;
      }
      const C uj = u[(size_t)j * npts + r];
      double ox = c0 * (double)uj.x + b * sx, oy = c0 * (double)uj.y + b * sy;
      if (a != 0.0) {
        const C vj = V[((size_t)k * norb + j) * npts + r];
        ox += a * (double)vj.x;
        oy += a * (double)vj.y;
      }
      out[((size_t)k * norb + j) * npts + r] = C{(T)ox, (T)oy};
    }
  }
}

// out = a A + b B + g C, elementwise over n complex values (C unread when g = 0): one step of the
// Chebyshev filter's three-term recurrence
template <typename T>
__global__ void k_lincomb3(const typename Cplx<T>::type* __restrict__ A, const typename Cplx<T>::type* __restrict__ B,
                           const typename Cplx<T>::type* __restrict__ Cv, double a, double b, double g, long long n,
                           typename Cplx<T>::type* __restrict__ out) {
  using C = typename Cplx<T>::type;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const C x = A[i], y = B[i];
    double re = a * (double)x.x + b * (double)y.x, im = a * (double)x.y + b * (double)y.y;
    if (g != 0.0) {
      const C z = Cv[i];
      re += g * (double)z.x;
      im += g * (double)z.y;
    }
    out[i] = C{(T)re, (T)im};
  }
}

// vin <- vin + mix (vout - vin); vout <- vin (the mixed potential becomes the current V_Hxc)
__global__ void k_mix_potential(double* __restrict__ vin, double* __restrict__ vout, long long n, double mix) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = vin[i] + mix * (vout[i] - vin[i]);
    vin[i] = v;
    vout[i] = v;
  }
}

}  // namespace

template <typename T>
cudaError_t launch_gram(const typename Cplx<T>::type* A, const typename Cplx<T>::type* B, int nk, int norb, int npts,
                        double dV, double2* out, cudaStream_t s) {
  k_gram<T><<<dim3(norb * norb, nk), kGramThreads, 0, s>>>(A, B, norb, npts, dV, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_basis(const typename Cplx<T>::type* U, const typename Cplx<T>::type* V, const double2* M, int nk,
                         int norb, int npts, double a, double c0, double b, typename Cplx<T>::type* out,
                         cudaStream_t s) {
  int bx = (npts + 255) / 256;
  if (bx > 152 * 8) bx = 152 * 8;
  k_basis<T><<<dim3(bx, nk), 256, 0, s>>>(U, V, M, norb, npts, a, c0, b, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_lincomb3(const typename Cplx<T>::type* A, const typename Cplx<T>::type* B,
                            const typename Cplx<T>::type* Cv, double a, double b, double g, long long n,
                            typename Cplx<T>::type* out, cudaStream_t s) {
  long long bl = (n + 255) / 256;
  if (bl > 152 * 16) bl = 152 * 16;
  k_lincomb3<T><<<(int)(bl < 1 ? 1 : bl), 256, 0, s>>>(A, B, Cv, a, b, g, n, out);
  return cudaGetLastError();
}
template cudaError_t launch_lincomb3<float>(const float2*, const float2*, const float2*, double, double, double,
                                            long long, float2*, cudaStream_t);
template cudaError_t launch_lincomb3<double>(const double2*, const double2*, const double2*, double, double, double,
                                             long long, double2*, cudaStream_t);

cudaError_t launch_mix_potential(double* vin, double* vout, long long n, double mix, cudaStream_t s) {
  long long b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  k_mix_potential<<<(int)b, 256, 0, s>>>(vin, vout, n, mix);
  return cudaGetLastError();
}

template cudaError_t launch_gram<float>(const float2*, const float2*, int, int, int, double, double2*, cudaStream_t);
template cudaError_t launch_gram<double>(const double2*, const double2*, int, int, int, double, double2*, cudaStream_t);
template cudaError_t launch_basis<float>(const float2*, const float2*, const double2*, int, int, int, double, double,
                                         double, float2*, cudaStream_t);
template cudaError_t launch_basis<double>(const double2*, const double2*, const double2*, int, int, int, double, double,
                                          double, double2*, cudaStream_t);

}  // namespace tdks
