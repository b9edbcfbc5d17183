// TB-mBJ exchange potential (xc = 3; Sec. 4.1 names the Becke-Johnson potential and its
// Tran-Blaha variant as options besides the LDA).  Published forms, per spin channel of the
// spin-unpolarised system (rho_s = rho/2, t_s = tau~/2):
//   D   = 2 t_s - |grad rho_s|^2 / (4 rho_s)              (curvature of the Fermi hole)
//   Q   = (lap rho_s - 2 gamma D) / 6,  gamma = 0.8
//   x   : x exp(-2x/3) / (x - 2) = (2/3) pi^(2/3) rho_s^(5/3) / Q      (Becke-Roussel hole)
//   b   = (x^3 exp(-x) / (8 pi rho_s))^(1/3)
//   v_BR = -(1/b) (1 - exp(-x) - x exp(-x) / 2)
//   v_x = c v_BR + (3c - 2) (1/pi) sqrt(5/12) sqrt(2 t_s / rho_s)
//   c   = alpha + beta sqrt(g), g = (1/Omega) int |grad rho| / rho,  alpha = -0.012, beta = 1.023
// tau~ = tau - |j|^2 / (2 rho) is the kinetic energy density of the time-dependent orbitals with
// the current's share removed (unchanged by a uniform A'), tau = sum_k w_k sum_n |(D1 + i k) u|^2,
// j = sum_k w_k sum_n 2 Im(conj(u) (D1 + i k) u).  Derivatives are the 8th-order central
// differences of the orbital stencil (periodic wrap, or zero outside an isolated box).  Points with
// rho <= 1e-10 get no mBJ potential.
//
// Three launches: k_tau (partial sums of rho, tau, j over chunks of orbitals, one thread per grid
// point; k_tau_pair: one thread per two x-adjacent points of FP32 grids with an even nx), k_mbj_g (the cell average g and c, one grid_sum; skipped when c is fixed) and k_mbj_x
// (folds the chunks, differentiates rho, solves the Becke-Roussel equation and adds v_x to V).
#include <cuda_runtime.h>

#include "grid_sum.cuh"
#include "tdks_internal.h"

namespace tdks {

namespace {

constexpr int kMbjThreads = 128;          // k_tau, k_mbj_g
constexpr int kBrThreads = 64;            // k_mbj_x: FP64-bound per SM, so spread over as many SMs as possible
constexpr double kPi = 3.14159265358979323846;
constexpr double kRhoMin = 1e-10;
constexpr double kGamma = 0.8, kAlpha = -0.012, kBeta = 1.023;

struct Fd {   // the stencil's difference coefficients (kFD1, kFD2), passed by value
  double d1[4], d2[5];
};

template <typename T>
struct D1h {  // first-derivative coefficients FD1[m] / h_a in the orbitals' precision, formed on the host
  T c[3][4];
};

struct Nbr {   // linear indices of the 4 neighbours per side along each axis (-1: outside the box)
  int p[3][4], m[3][4];
};

__device__ __forceinline__ Nbr neighbours(int ix, int iy, int iz, int nx, int ny, int nz, int periodic) {
  Nbr b;
  const int n[3] = {nx, ny, nz}, i[3] = {ix, iy, iz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int m = 1; m <= 4; ++m) {
      int jp = i[a] + m, jm = i[a] - m;
      bool op = true, om = true;
      if (periodic) {
        jp = jp >= n[a] ? jp - n[a] : jp;       // n >= 4: one wrap suffices
        jm = jm < 0 ? jm + n[a] : jm;
      } else {
        op = jp < n[a];
        om = jm >= 0;
      }
      int cp[3] = {ix, iy, iz}, cm[3] = {ix, iy, iz};
      cp[a] = jp;
      cm[a] = jm;
      b.p[a][m - 1] = op ? (cp[2] * ny + cp[1]) * nx + cp[0] : -1;
      b.m[a][m - 1] = om ? (cm[2] * ny + cm[1]) * nx + cm[0] : -1;
    }
  }
  return b;
}

template <typename V>
__device__ __forceinline__ V ld_or_zero(const V* f, int i) {
  return i >= 0 ? f[i] : V{};
}

// part[(chunk * 5 + c) * npts + p], c = rho, tau, j_x, j_y, j_z, over the orbitals of one chunk.
template <typename T>
__global__ void __launch_bounds__(kMbjThreads) k_tau(const typename Cplx<T>::type* __restrict__ u, int nk, int norb,
                                                    int nx, int ny, int nz, int periodic,
                                                    const double* __restrict__ kpts, const double* __restrict__ kw,
                                                    D1h<T> d1, int ochunk, double* __restrict__ part) {
  using C = typename Cplx<T>::type;
  const int npts = nx * ny * nz;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npts) return;
  const int ix = p % nx, iy = (p / nx) % ny, iz = p / (nx * ny);
  const Nbr nb = neighbours(ix, iy, iz, nx, ny, nz, periodic);
  const int o0 = blockIdx.y * ochunk, o1 = min(o0 + ochunk, nk * norb);
  T acc[5] = {0, 0, 0, 0, 0};
  // the orbitals of one k at a time: unweighted sums over them, weighted once per k (the weight and
  // wave vector are converted once per k -- FP64 -> FP32 conversions run on the slow FP64 pipe), and
  // a branch-free inner loop whose loads the compiler can overlap across orbitals
  for (int o = o0; o < o1;) {
    const int k = o / norb;
    const int oe = min(o1, (k + 1) * norb);
    const T q[3] = {(T)kpts[3 * k], (T)kpts[3 * k + 1], (T)kpts[3 * k + 2]};
    T sk[5] = {0, 0, 0, 0, 0};
#pragma unroll 2
    for (; o < oe; ++o) {
      const C* f = u + (size_t)o * npts;
      const C c0 = f[p];
      sk[0] += c0.x * c0.x + c0.y * c0.y;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        C g = C{-q[a] * c0.y, q[a] * c0.x};                             // i q u
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const C fp = ld_or_zero(f, nb.p[a][m]), fm = ld_or_zero(f, nb.m[a][m]);
          g.x += d1.c[a][m] * (fp.x - fm.x);
          g.y += d1.c[a][m] * (fp.y - fm.y);
        }
        sk[1] += g.x * g.x + g.y * g.y;
        sk[2 + a] += c0.x * g.y - c0.y * g.x;                           // Im(conj(u) g)
      }
    }
    const T w = (T)(2.0 * kw[k]);
    acc[0] += w * sk[0];
    acc[1] += T(0.5) * w * sk[1];
#pragma unroll
    for (int c = 2; c < 5; ++c) acc[c] += w * sk[c];
  }
#pragma unroll
  for (int c = 0; c < 5; ++c) part[((size_t)blockIdx.y * 5 + c) * npts + p] = (double)acc[c];
}

// k_tau for FP32 grids with an even nx: a thread takes two x-adjacent points (x even).  The orbital
// values of a point pair are one 16-byte load, so the values the two points need -- their centres,
// x +- 1..4 of both, and y +- 1..4 and z +- 1..4 of the pair -- are 21 loads instead of 50.  With an
// even nx a neighbour pair is wholly inside or wholly outside an isolated box.  Same sums as k_tau.
__device__ __forceinline__ float4 ld4_or_zero(const float2* f, int i) {
  return i >= 0 ? __ldg(reinterpret_cast<const float4*>(f + i)) : make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void __launch_bounds__(kMbjThreads) k_tau_pair(const float2* __restrict__ u, int nk, int norb, int nx,
                                                         int ny, int nz, int periodic,
                                                         const double* __restrict__ kpts,
                                                         const double* __restrict__ kw, D1h<float> d1, int ochunk,
                                                         double* __restrict__ part) {
  const int npts = nx * ny * nz, nxh = nx / 2;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= npts / 2) return;
  const int ix = 2 * (t % nxh), iy = (t / nxh) % ny, iz = t / (nxh * ny);
  const int p = (iz * ny + iy) * nx + ix;
  int ox[4], oy[8], oz[8];                         // neighbour pairs (-1: outside the box)
  const int dxs[4] = {-4, -2, 2, 4};
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    int jx = ix + dxs[j];
    bool in = true;
    if (periodic) jx = jx < 0 ? jx + nx : (jx >= nx ? jx - nx : jx);
    else in = jx >= 0 && jx < nx;
    ox[j] = in ? (iz * ny + iy) * nx + jx : -1;
  }
#pragma unroll
  for (int m = 1; m <= 4; ++m) {
#pragma unroll
    for (int sgn = 0; sgn < 2; ++sgn) {
      int jy = sgn == 0 ? iy + m : iy - m, jz = sgn == 0 ? iz + m : iz - m;
      bool iny = true, inz = true;
      if (periodic) {
        jy = jy < 0 ? jy + ny : (jy >= ny ? jy - ny : jy);
        jz = jz < 0 ? jz + nz : (jz >= nz ? jz - nz : jz);
      } else {
        iny = jy >= 0 && jy < ny;
        inz = jz >= 0 && jz < nz;
      }
      oy[2 * (m - 1) + sgn] = iny ? (iz * ny + jy) * nx + ix : -1;
      oz[2 * (m - 1) + sgn] = inz ? (jz * ny + iy) * nx + ix : -1;
    }
  }
  const int o0 = blockIdx.y * ochunk, o1 = min(o0 + ochunk, nk * norb);
  float acc[2][5] = {{0, 0, 0, 0, 0}, {0, 0, 0, 0, 0}};
  for (int o = o0; o < o1;) {
    const int k = o / norb;
    const int oe = min(o1, (k + 1) * norb);
    const float q[3] = {(float)kpts[3 * k], (float)kpts[3 * k + 1], (float)kpts[3 * k + 2]};
    float sk[2][5] = {{0, 0, 0, 0, 0}, {0, 0, 0, 0, 0}};
#pragma unroll 1
    for (; o < oe; ++o) {
      const float2* f = u + (size_t)o * npts;
      const float4 c = __ldg(reinterpret_cast<const float4*>(f + p));
      float4 X[4], Y[8], Z[8];
#pragma unroll
      for (int j = 0; j < 4; ++j) X[j] = ld4_or_zero(f, ox[j]);
#pragma unroll
      for (int j = 0; j < 8; ++j) { Y[j] = ld4_or_zero(f, oy[j]); Z[j] = ld4_or_zero(f, oz[j]); }
      // x +- m of point A (x) and B (x + 1), m = 1..4
      const float2 lo_c = make_float2(c.x, c.y), hi_c = make_float2(c.z, c.w);
      auto lo = [](float4 v) { return make_float2(v.x, v.y); };
      auto hi = [](float4 v) { return make_float2(v.z, v.w); };
      const float2 axp[4] = {hi_c, lo(X[2]), hi(X[2]), lo(X[3])}, axm[4] = {hi(X[1]), lo(X[1]), hi(X[0]), lo(X[0])};
      const float2 bxp[4] = {lo(X[2]), hi(X[2]), lo(X[3]), hi(X[3])}, bxm[4] = {lo_c, hi(X[1]), lo(X[1]), hi(X[0])};
#pragma unroll
      for (int pt = 0; pt < 2; ++pt) {
        const float2 c0 = pt == 0 ? lo_c : hi_c;
        sk[pt][0] += c0.x * c0.x + c0.y * c0.y;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          float2 g = make_float2(-q[a] * c0.y, q[a] * c0.x);            // i q u
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            float2 fp, fm;
            if (a == 0) { fp = pt == 0 ? axp[m] : bxp[m]; fm = pt == 0 ? axm[m] : bxm[m]; }
            else if (a == 1) { fp = pt == 0 ? lo(Y[2 * m]) : hi(Y[2 * m]); fm = pt == 0 ? lo(Y[2 * m + 1]) : hi(Y[2 * m + 1]); }
            else { fp = pt == 0 ? lo(Z[2 * m]) : hi(Z[2 * m]); fm = pt == 0 ? lo(Z[2 * m + 1]) : hi(Z[2 * m + 1]); }
            g.x += d1.c[a][m] * (fp.x - fm.x);
            g.y += d1.c[a][m] * (fp.y - fm.y);
          }
          sk[pt][1] += g.x * g.x + g.y * g.y;
          sk[pt][2 + a] += c0.x * g.y - c0.y * g.x;                    // Im(conj(u) g)
        }
      }
    }
    const float w = (float)(2.0 * kw[k]);
#pragma unroll
    for (int pt = 0; pt < 2; ++pt) {
      acc[pt][0] += w * sk[pt][0];
      acc[pt][1] += 0.5f * w * sk[pt][1];
#pragma unroll
      for (int cc = 2; cc < 5; ++cc) acc[pt][cc] += w * sk[pt][cc];
    }
  }
#pragma unroll
  for (int cc = 0; cc < 5; ++cc) {
    part[((size_t)blockIdx.y * 5 + cc) * npts + p] = (double)acc[0][cc];
    part[((size_t)blockIdx.y * 5 + cc) * npts + p + 1] = (double)acc[1][cc];
  }
}

// |grad rho|^2 and lap rho at p by the 8th-order differences
__device__ __forceinline__ void rho_derivs(const double* __restrict__ rho, const Nbr& nb, double r0,
                                           const double h[3], const Fd& fd, double* g2, double* lap) {
  double gg = 0.0, ll = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double d = 0.0, s = fd.d2[0] * r0;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const double fp = ld_or_zero(rho, nb.p[a][m]), fm = ld_or_zero(rho, nb.m[a][m]);
      d += fd.d1[m] * (fp - fm);
      s += fd.d2[m + 1] * (fp + fm);
    }
    d /= h[a];
    gg += d * d;
    ll += s / (h[a] * h[a]);
  }
  *g2 = gg;
  *lap = ll;
}

// c = alpha + beta sqrt(g) from the density (written by the last CTA)
__global__ void __launch_bounds__(kMbjThreads) k_mbj_g(const double* __restrict__ rho, int nx, int ny, int nz,
                                                      int periodic, double hx, double hy, double hz, Fd fd,
                                                      double* partials, unsigned* ticket, double* c_out) {
  __shared__ double tot[1];
  const int npts = nx * ny * nz;
  const double h[3] = {hx, hy, hz};
  double v[1] = {0.0};
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npts; p += gridDim.x * blockDim.x) {
    const double r0 = rho[p];
    if (r0 > kRhoMin) {
      const Nbr nb = neighbours(p % nx, (p / nx) % ny, p / (nx * ny), nx, ny, nz, periodic);
      double g2, lap;
      rho_derivs(rho, nb, r0, h, fd, &g2, &lap);
      v[0] += sqrt(g2) / r0;
    }
  }
  if (grid_sum<1>(v, partials, ticket, tot) && threadIdx.x == 0) *c_out = kAlpha + kBeta * sqrt(tot[0] / npts);
}

// H(x) = x exp(-2x/3) - y (x - 2): the Becke-Roussel equation times (x - 2), one root per branch
__device__ __forceinline__ double br_h(double x, double y) { return x * exp(-2.0 * x / 3.0) - y * (x - 2.0); }

__device__ __forceinline__ float br_hf(float x, float y) { return x * __expf(-2.0f * x / 3.0f) - y * (x - 2.0f); }

// Root x of x exp(-2x/3)/(x-2) = y: y < 0 in (0, 2) (H(0) = 2y < 0 < H(2)), y > 0 in (2, hi)
// (H(2) > 0 > H(hi)).  The bracket is narrowed by bisection in FP32 (26 steps; FP64 arithmetic runs
// at a small fraction of the FP32 rate on this GPU) and widened by a relative 1e-5 to cover the
// FP32 rounding of H; FP64 Newton steps kept inside it then reach full precision.  Where y is
// outside the FP32 range, or the widened bracket does not keep the signs of H, the bisection runs
// in FP64 (34 steps) on the whole branch.
__device__ double br_root(double y) {
  double neg = 0.0, pos = 0.0;        // H(neg) < 0 < H(pos)
  bool have = false;
  const double ay = fabs(y);
  if (ay > 1e-30 && ay < 1e30) {
    const float yf = (float)y;
    float nf, pf;
    if (yf < 0.0f) {
      nf = 0.0f;
      pf = 2.0f;
    } else {
      pf = 2.0f;
      nf = 4.0f;
      while (br_hf(nf, yf) > 0.0f && nf < 256.0f) nf *= 2.0f;   // y > 1e-30: the root is below 160
    }
    for (int it = 0; it < 26; ++it) {
      const float mid = 0.5f * (nf + pf);
      if (br_hf(mid, yf) < 0.0f) nf = mid; else pf = mid;
    }
    const double a = fmin((double)nf, (double)pf), b = fmax((double)nf, (double)pf);
    const double pad = 1e-5 * b;
    neg = y < 0.0 ? fmax(a - pad, 0.0) : b + pad;
    pos = y < 0.0 ? fmin(b + pad, 2.0) : fmax(a - pad, 2.0);
    have = br_h(neg, y) < 0.0 && br_h(pos, y) > 0.0;
  }
  if (!have) {
    if (y < 0.0) {
      neg = 0.0;
      pos = 2.0;
    } else {
      pos = 2.0;
      neg = 4.0;
      while (br_h(neg, y) > 0.0 && neg < 4096.0) neg *= 2.0;   // exp(-2x/3) underflows long before 4096
    }
    for (int it = 0; it < 34; ++it) {
      const double mid = 0.5 * (neg + pos);
      if (br_h(mid, y) < 0.0) neg = mid; else pos = mid;
    }
  }
  double x = 0.5 * (neg + pos);
  const double lo = fmin(neg, pos), hi = fmax(neg, pos);
  for (int it = 0; it < 5; ++it) {   // Newton, kept inside [lo, hi] (the root may sit at an end, x = 2)
    const double e = exp(-2.0 * x / 3.0);
    const double f = x * e - y * (x - 2.0), df = e * (1.0 - 2.0 * x / 3.0) - y;
    if (df == 0.0) break;
    const double xn = x - f / df;
    if (!(xn >= lo && xn <= hi)) break;
    x = xn;
  }
  return x;
}

// V[p] += v_x^mBJ(rho, grad rho, lap rho, tau~) with c = c_fixed (> 0) or *c_dev
__global__ void __launch_bounds__(kBrThreads) k_mbj_x(const double* __restrict__ rho, const double* __restrict__ part,
                                                      int nchunk, int nx, int ny, int nz, int periodic, double hx,
                                                      double hy, double hz, Fd fd, double c_fixed,
                                                      const double* __restrict__ c_dev, double* __restrict__ V) {
  const int npts = nx * ny * nz;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npts) return;
  const double r0 = rho[p];
  if (!(r0 > kRhoMin)) return;
  const double h[3] = {hx, hy, hz};
  // tau~ from the orbitals' chunks (their own rho for the current's share), chunks in order
  double s[5] = {0, 0, 0, 0, 0};
  for (int ch = 0; ch < nchunk; ++ch)
#pragma unroll
    for (int c = 0; c < 5; ++c) s[c] += part[((size_t)ch * 5 + c) * npts + p];
  double tt = 0.0;
  if (s[0] > 0.0) tt = fmax(s[1] - (s[2] * s[2] + s[3] * s[3] + s[4] * s[4]) / (2.0 * s[0]), 0.0);
  const Nbr nb = neighbours(p % nx, (p / nx) % ny, p / (nx * ny), nx, ny, nz, periodic);
  double g2, lap;
  rho_derivs(rho, nb, r0, h, fd, &g2, &lap);
  const double c = c_fixed > 0.0 ? c_fixed : *c_dev;
  const double rs = 0.5 * r0, ts = 0.5 * tt, gs2 = 0.25 * g2;
  const double D = 2.0 * ts - gs2 / (4.0 * rs);
  const double Q = (0.5 * lap - 2.0 * kGamma * D) / 6.0;
  const double K = (2.0 / 3.0) * cbrt(kPi * kPi) * rs * cbrt(rs * rs);     // (2/3) pi^(2/3) rho_s^(5/3)
  const double x = Q != 0.0 ? br_root(K / Q) : 2.0;
  const double ex = exp(-x);
  const double b = cbrt(x * x * x * ex / (8.0 * kPi * rs));
  const double vbr = -(1.0 - ex - 0.5 * x * ex) / b;
  V[p] += c * vbr + (3.0 * c - 2.0) / kPi * sqrt(5.0 / 12.0) * sqrt(2.0 * ts / rs);
}

}  // namespace

// chunks of orbitals for k_tau: one wave of about 8 CTAs of points x chunks per SM (the register
// limit of the FP32 kernel, 64 registers x 128 threads)
int mbj_chunks(long long npts, int norb_tot) {
  const long long bx = (npts + kMbjThreads - 1) / kMbjThreads;
  long long ch = (152LL * 8) / bx;
  if (ch > norb_tot) ch = norb_tot;
  return ch < 1 ? 1 : (int)ch;
}

template <typename T>
cudaError_t launch_mbj(const typename Cplx<T>::type* u, int nk, int norb, const int n[3], int periodic,
                       const double h[3], const double* kpts, const double* kw, const double* rho, double c_fixed,
                       double* part, int nchunk, double* partials, unsigned* ticket, double* c_dev, double* V,
                       cudaStream_t s, int* nlaunch) {
  const int npts = n[0] * n[1] * n[2];
  const int norb_tot = nk * norb;
  const int ochunk = (norb_tot + nchunk - 1) / nchunk;
  const int bx = (npts + kMbjThreads - 1) / kMbjThreads;
  Fd fd;
  for (int m = 0; m < 4; ++m) fd.d1[m] = kFD1[m];
  for (int m = 0; m < 5; ++m) fd.d2[m] = kFD2[m];
  D1h<T> d1;
  for (int a = 0; a < 3; ++a)
    for (int m = 0; m < 4; ++m) d1.c[a][m] = (T)(kFD1[m] / h[a]);
  if constexpr (sizeof(T) == 4) {
    if (n[0] % 2 == 0) {
      const int bx2 = (npts / 2 + kMbjThreads - 1) / kMbjThreads;
      k_tau_pair<<<dim3(bx2, nchunk), kMbjThreads, 0, s>>>(u, nk, norb, n[0], n[1], n[2], periodic, kpts, kw, d1,
                                                          ochunk, part);
    } else {
      k_tau<T><<<dim3(bx, nchunk), kMbjThreads, 0, s>>>(u, nk, norb, n[0], n[1], n[2], periodic, kpts, kw, d1, ochunk,
                                                        part);
    }
  } else {
    k_tau<T><<<dim3(bx, nchunk), kMbjThreads, 0, s>>>(u, nk, norb, n[0], n[1], n[2], periodic, kpts, kw, d1, ochunk,
                                                      part);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int nl = 2;
  if (!(c_fixed > 0.0)) {
    k_mbj_g<<<grid_sum_blocks(npts, kMbjThreads), kMbjThreads, 0, s>>>(rho, n[0], n[1], n[2], periodic, h[0], h[1],
                                                                      h[2], fd, partials, ticket, c_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    nl = 3;
  }
  k_mbj_x<<<(npts + kBrThreads - 1) / kBrThreads, kBrThreads, 0, s>>>(rho, part, nchunk, n[0], n[1], n[2], periodic,
                                                                    h[0], h[1], h[2], fd, c_fixed, c_dev, V);
  if (nlaunch) *nlaunch = nl;
  return cudaGetLastError();
}

template cudaError_t launch_mbj<float>(const float2*, int, int, const int*, int, const double*, const double*,
                                       const double*, const double*, double, double*, int, double*, unsigned*, double*,
                                       double*, cudaStream_t, int*);
template cudaError_t launch_mbj<double>(const double2*, int, int, const int*, int, const double*, const double*,
                                        const double*, const double*, double, double*, int, double*, unsigned*,
                                        double*, double*, cudaStream_t, int*);

}  // namespace tdks
