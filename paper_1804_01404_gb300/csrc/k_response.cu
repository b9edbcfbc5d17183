// Response analysis of a finished run, on the GPU: masked Fourier transforms of the time series
// that the step observables give.
//   * Eq. (distribution): the oscillator-strength distribution df/dE from the induced dipole after
//     an impulsive kick of strength kappa;
//   * Eq. (sigma_ft): the conductivity sigma(w) = -(c / A0) int_0^T e^{iwt} f(t/T) I(t) dt from the
//     current after a vector-potential step A0 (here given as A'0 = A0 / c, the unit of the
//     library's fields, so c / A0 = 1 / A'0), and eps(w) = 1 + 4 pi i sigma(w) / w; optionally
//     with the mean current removed first (Sec. 4.1 example: sigma(0) = 0 for a gapped material).
// Both use the cubic mask f(x) = 1 - 3x^2 + 2x^3 and the samples t_i = i dt, i = 0..n-1, T = t_{n-1},
// summed with weight dt.
//   * Sec. 4.1: the work done by the field per unit volume, W(t) = int_0^t I(t').E(t') dt' (the
//     electronic excitation energy per volume when the xc potential derives from an energy
//     functional), as a cumulative trapezoid sum.
//   * Sec. 2.1 ground-state outputs: the density of states of a set of orbital energies, Gaussian
//     broadened.
// FP64 throughout.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "../../include/tdks.h"
#include "tdks_internal.h"

namespace tdks {

namespace {

constexpr int kFtThreads = 256;
constexpr double kPiR = 3.14159265358979323846;

__device__ __forceinline__ double mask(double u) { return 1.0 - 3.0 * u * u + 2.0 * u * u * u; }

// Sum of a pair over the CTA (fixed order); the result is valid in thread 0.
__device__ __forceinline__ void block_sum2(double& a, double& b, double* red) {
  red[threadIdx.x] = a;
  red[kFtThreads + threadIdx.x] = b;
  __syncthreads();
  for (int o = kFtThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[threadIdx.x] += red[threadIdx.x + o];
      red[kFtThreads + threadIdx.x] += red[kFtThreads + threadIdx.x + o];
    }
    __syncthreads();
  }
  a = red[0];
  b = red[kFtThreads];
}

// xbar = sum_i f(t_i/T) x_i / sum_i f(t_i/T): the mask-weighted mean, the one whose removal makes the
// masked transform vanish at w = 0.  One CTA.
__global__ void __launch_bounds__(kFtThreads) k_masked_mean(const double* __restrict__ x, int n, double* xbar) {
  __shared__ double red[2 * kFtThreads];
  const double T = (n - 1);
  double s = 0.0, w = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double f = mask(n > 1 ? i / T : 0.0);
    s += f * x[i];
    w += f;
  }
  block_sum2(s, w, red);
  if (threadIdx.x == 0) *xbar = (w != 0.0) ? s / w : 0.0;
}

// F(w_j) = dt sum_i f(t_i/T) (x_i - xbar) exp(i w_j t_i).  One CTA per frequency; thread k sums a
// contiguous chunk of samples, starting from an exact phase factor and rotating it by exp(i w dt)
// from sample to sample (at most n / 256 rotations, so the recurrence error stays near the
// rounding of one product); the chunk sums are added in a fixed-order tree.
__global__ void __launch_bounds__(kFtThreads) k_masked_ft(const double* __restrict__ x, int n, double dt,
                                                         const double* __restrict__ xbar,
                                                         const double* __restrict__ w, double2* __restrict__ F) {
  __shared__ double red[2 * kFtThreads];
  const double om = w[blockIdx.x];
  const double mean = xbar ? *xbar : 0.0;
  const int chunk = (n + kFtThreads - 1) / kFtThreads;
  const int i0 = threadIdx.x * chunk, i1 = min(n, i0 + chunk);
  double re = 0.0, im = 0.0;
  if (i0 < i1) {
    double s, c, rs, rc;
    sincos(om * (i0 * dt), &s, &c);
    sincos(om * dt, &rs, &rc);
    for (int i = i0; i < i1; ++i) {
      const double v = mask(n > 1 ? (double)i / (n - 1) : 0.0) * (x[i] - mean);
      re += v * c;
      im += v * s;
      const double c2 = c * rc - s * rs;
      s = s * rc + c * rs;
      c = c2;
    }
  }
  block_sum2(re, im, red);
  if (threadIdx.x == 0) F[blockIdx.x] = double2{re * dt, im * dt};
}

// kind 0: out[j] = -(2 w_j / (pi kappa)) Im F_j                      (df/dE, Eq. distribution)
// kind 1: out[2j..] = sigma_j = -F_j / A'0; eps[2j..] = 1 + 4 pi i sigma_j / w_j   (Eq. sigma_ft)
__global__ void k_response_finish(const double2* __restrict__ F, const double* __restrict__ w, int nw, int kind,
                                  double scale, double* __restrict__ out, double* __restrict__ eps) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nw) return;
  const double2 f = F[j];
  if (kind == 0) {
    out[j] = -(2.0 * w[j] / (kPiR * scale)) * f.y;
    return;
  }
  const double sr = -f.x / scale, si = -f.y / scale;
  out[2 * j] = sr;
  out[2 * j + 1] = si;
  if (eps) {
    eps[2 * j] = 1.0 - 4.0 * kPiR * si / w[j];
    eps[2 * j + 1] = 4.0 * kPiR * sr / w[j];
  }
}

// W[0] = 0, W[i] = W[i-1] + dt/2 (g[i-1] + g[i]), g[i] = I[i].E[i] (3-vectors).  One CTA: thread k
// owns a contiguous chunk of increments, the chunk totals are scanned in shared memory (fixed
// order), and each thread then writes its chunk's running sums.
constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads) k_work(const double* __restrict__ I, const double* __restrict__ E,
                                                       int n, double dt, double* __restrict__ W) {
  __shared__ double tot[kScanThreads];
  auto g = [&](int i) { return I[3 * i] * E[3 * i] + I[3 * i + 1] * E[3 * i + 1] + I[3 * i + 2] * E[3 * i + 2]; };
  const int m = n - 1;                                  // increments 1..n-1
  const int chunk = (m + kScanThreads - 1) / kScanThreads;
  const int i0 = 1 + threadIdx.x * chunk, i1 = min(n, i0 + chunk);
  double s = 0.0;
  for (int i = i0; i < i1; ++i) s += 0.5 * dt * (g(i - 1) + g(i));
  tot[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < kScanThreads; o <<= 1) {          // inclusive scan (Hillis-Steele)
    const double add = threadIdx.x >= o ? tot[threadIdx.x - o] : 0.0;
    __syncthreads();
    tot[threadIdx.x] += add;
    __syncthreads();
  }
  double run = threadIdx.x > 0 ? tot[threadIdx.x - 1] : 0.0;
  if (threadIdx.x == 0) W[0] = 0.0;
  for (int i = i0; i < i1; ++i) {
    run += 0.5 * dt * (g(i - 1) + g(i));
    W[i] = run;
  }
}

// D(E_j) = sum_k w_k sum_n 2 g(E_j - e_nk), g the normalised Gaussian of width sigma; one thread per
// energy, levels in fixed order.
__global__ void k_dos(const double* __restrict__ eps, int nk, int norb, const double* __restrict__ kw,
                      const double* __restrict__ E, int nE, double sigma, double* __restrict__ D) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nE) return;
  const double e = E[j], inv = 1.0 / sigma, norm = 2.0 * inv / sqrt(2.0 * 3.14159265358979323846);
  double acc = 0.0;
  for (int k = 0; k < nk; ++k) {
    double sk = 0.0;
    for (int n = 0; n < norb; ++n) {
      const double x = (e - eps[k * norb + n]) * inv;
      sk += exp(-0.5 * x * x);
    }
    acc += kw[k] * sk;
  }
  D[j] = norm * acc;
}

tdks_status rfail(tdks_status s, const char* msg) {
  set_last_error(msg);
  return s;
}

// Host arrays in and out; device scratch for one call (synchronous on the stream).
tdks_status masked_response(const double* x, int nt, double dt, const double* w, int nw, int subtract_mean,
                            int kind, double scale, double* out, double* eps, void* stream) {
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t bx = sizeof(double) * (size_t)nt, bw = sizeof(double) * (size_t)nw;
  const size_t bout = sizeof(double) * (size_t)nw * (kind == 0 ? 1 : 2);
  double *dx = nullptr, *dw = nullptr, *dmean = nullptr, *dout = nullptr, *deps = nullptr;
  double2* dF = nullptr;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  chk(cudaMalloc(&dx, bx));
  chk(cudaMalloc(&dw, bw));
  chk(cudaMalloc(&dmean, sizeof(double)));
  chk(cudaMalloc(&dF, sizeof(double2) * (size_t)nw));
  chk(cudaMalloc(&dout, bout));
  if (eps) chk(cudaMalloc(&deps, bout));
  if (e == cudaSuccess) {
    chk(cudaMemcpyAsync(dx, x, bx, cudaMemcpyHostToDevice, s));
    chk(cudaMemcpyAsync(dw, w, bw, cudaMemcpyHostToDevice, s));
  }
  if (e == cudaSuccess) {
    if (subtract_mean) {
      k_masked_mean<<<1, kFtThreads, 0, s>>>(dx, nt, dmean);
      chk(cudaGetLastError());
    }
    k_masked_ft<<<nw, kFtThreads, 0, s>>>(dx, nt, dt, subtract_mean ? dmean : nullptr, dw, dF);
    chk(cudaGetLastError());
    k_response_finish<<<(nw + 127) / 128, 128, 0, s>>>(dF, dw, nw, kind, scale, dout, deps);
    chk(cudaGetLastError());
  }
  if (e == cudaSuccess) chk(cudaMemcpyAsync(out, dout, bout, cudaMemcpyDeviceToHost, s));
  if (e == cudaSuccess && eps) chk(cudaMemcpyAsync(eps, deps, bout, cudaMemcpyDeviceToHost, s));
  if (e == cudaSuccess) chk(cudaStreamSynchronize(s));
  cudaFree(dx);
  cudaFree(dw);
  cudaFree(dmean);
  cudaFree(dF);
  cudaFree(dout);
  cudaFree(deps);
  if (e != cudaSuccess) return rfail(e == cudaErrorMemoryAllocation ? TDKS_ENOMEM : TDKS_ECUDA,
                                     (std::string("response analysis: ") + cudaGetErrorString(e)).c_str());
  return TDKS_OK;
}

tdks_status check_series(const double* x, int nt, double dt, const double* w, int nw, const double* out) {
  if (!x || !w || !out) return rfail(TDKS_EINVAL, "response analysis: null array");
  if (nt < 2) return rfail(TDKS_EINVAL, "response analysis: need at least two samples");
  if (nw < 1 || nw > (1 << 24)) return rfail(TDKS_EINVAL, "response analysis: frequency count outside 1..2^24");
  if (!(dt > 0.0) || !std::isfinite(dt)) return rfail(TDKS_EINVAL, "response analysis: dt must be positive");
  return TDKS_OK;
}

}  // namespace

}  // namespace tdks

using tdks::check_series;
using tdks::k_dos;
using tdks::k_work;
using tdks::masked_response;
using tdks::rfail;

extern "C" tdks_status tdks_oscillator_strength(const double* d, int nt, double dt, double kappa, const double* E,
                                                int nE, double* dfdE, void* stream) {
  tdks_status st = check_series(d, nt, dt, E, nE, dfdE);
  if (st != TDKS_OK) return st;
  if (!(kappa != 0.0) || !std::isfinite(kappa)) return rfail(TDKS_EINVAL, "tdks_oscillator_strength: kappa must be nonzero");
  return masked_response(d, nt, dt, E, nE, 0, 0, kappa, dfdE, nullptr, stream);
}

extern "C" tdks_status tdks_conductivity(const double* I, int nt, double dt, double Ap0, const double* w, int nw,
                                         int subtract_mean, double* sigma, double* eps, void* stream) {
  tdks_status st = check_series(I, nt, dt, w, nw, sigma);
  if (st != TDKS_OK) return st;
  if (!(Ap0 != 0.0) || !std::isfinite(Ap0)) return rfail(TDKS_EINVAL, "tdks_conductivity: Ap0 must be nonzero");
  if (eps)
    for (int j = 0; j < nw; ++j)
      if (!(w[j] > 0.0)) return rfail(TDKS_EINVAL, "tdks_conductivity: eps needs every frequency > 0");
  return masked_response(I, nt, dt, w, nw, subtract_mean ? 1 : 0, 1, Ap0, sigma, eps, stream);
}

extern "C" tdks_status tdks_work(const double* I, const double* E, int nt, double dt, double* W, void* stream) {
  if (!I || !E || !W) return rfail(TDKS_EINVAL, "tdks_work: null array");
  if (nt < 1 || nt > (1 << 26)) return rfail(TDKS_EINVAL, "tdks_work: nt outside 1..2^26");
  if (!(dt > 0.0) || !std::isfinite(dt)) return rfail(TDKS_EINVAL, "tdks_work: dt must be positive");
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t b3 = sizeof(double) * 3 * (size_t)nt, b1 = sizeof(double) * (size_t)nt;
  double *dI = nullptr, *dE = nullptr, *dW = nullptr;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  chk(cudaMalloc(&dI, b3));
  chk(cudaMalloc(&dE, b3));
  chk(cudaMalloc(&dW, b1));
  if (e == cudaSuccess) {
    chk(cudaMemcpyAsync(dI, I, b3, cudaMemcpyHostToDevice, s));
    chk(cudaMemcpyAsync(dE, E, b3, cudaMemcpyHostToDevice, s));
  }
  if (e == cudaSuccess) {
    k_work<<<1, tdks::kScanThreads, 0, s>>>(dI, dE, nt, dt, dW);
    chk(cudaGetLastError());
  }
  if (e == cudaSuccess) chk(cudaMemcpyAsync(W, dW, b1, cudaMemcpyDeviceToHost, s));
  if (e == cudaSuccess) chk(cudaStreamSynchronize(s));
  cudaFree(dI);
  cudaFree(dE);
  cudaFree(dW);
  if (e != cudaSuccess) return rfail(e == cudaErrorMemoryAllocation ? TDKS_ENOMEM : TDKS_ECUDA,
                                     (std::string("tdks_work: ") + cudaGetErrorString(e)).c_str());
  return TDKS_OK;
}

extern "C" tdks_status tdks_dos(const double* eps, int nk, int norb, const double* kw, const double* E, int nE,
                                double sigma, double* dos, void* stream) {
  if (!eps || !kw || !E || !dos) return rfail(TDKS_EINVAL, "tdks_dos: null array");
  if (nk < 1 || norb < 1 || (long long)nk * norb > (1LL << 24)) return rfail(TDKS_EINVAL, "tdks_dos: nk * norb outside 1..2^24");
  if (nE < 1 || nE > (1 << 24)) return rfail(TDKS_EINVAL, "tdks_dos: nE outside 1..2^24");
  if (!(sigma > 0.0) || !std::isfinite(sigma)) return rfail(TDKS_EINVAL, "tdks_dos: sigma must be positive");
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t be = sizeof(double) * (size_t)nk * norb, bk = sizeof(double) * (size_t)nk, bE = sizeof(double) * (size_t)nE;
  double *de = nullptr, *dk = nullptr, *dE = nullptr, *dD = nullptr;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  chk(cudaMalloc(&de, be));
  chk(cudaMalloc(&dk, bk));
  chk(cudaMalloc(&dE, bE));
  chk(cudaMalloc(&dD, bE));
  if (e == cudaSuccess) {
    chk(cudaMemcpyAsync(de, eps, be, cudaMemcpyHostToDevice, s));
    chk(cudaMemcpyAsync(dk, kw, bk, cudaMemcpyHostToDevice, s));
    chk(cudaMemcpyAsync(dE, E, bE, cudaMemcpyHostToDevice, s));
  }
  if (e == cudaSuccess) {
    k_dos<<<(nE + 255) / 256, 256, 0, s>>>(de, nk, norb, dk, dE, nE, sigma, dD);
    chk(cudaGetLastError());
  }
  if (e == cudaSuccess) chk(cudaMemcpyAsync(dos, dD, bE, cudaMemcpyDeviceToHost, s));
  if (e == cudaSuccess) chk(cudaStreamSynchronize(s));
  cudaFree(de);
  cudaFree(dk);
  cudaFree(dE);
  cudaFree(dD);
  if (e != cudaSuccess) return rfail(e == cudaErrorMemoryAllocation ? TDKS_ENOMEM : TDKS_ECUDA,
                                     (std::string("tdks_dos: ") + cudaGetErrorString(e)).c_str());
  return TDKS_OK;
}
