// Grid kernels in FP64: FFT Poisson solve (periodic and zero-padded isolated), LDA (lda.cuh),
// potential combination, density, dipole and current reductions, kick, local potential.
//
// FFT: batched 1D Stockham transforms in shared memory, one launch per axis, mixed radix
// (4, 2, 3, 5, ...).  A CTA loads LB lines of the 3D array into shared memory -- for the y and z
// axes the LB lines are consecutive in x, so every global access is coalesced -- runs all radix
// stages there, and writes the lines back in natural order.  Periodic boxes whose xy-plane fits in
// shared memory take the x and y passes in one launch per direction (k_fft_planes: one CTA per
// plane; for a single cell k_fft_planes_cluster splits each plane over a thread-block cluster and
// transforms output by output, since its FP64 work would otherwise sit on a few SMs).
#include <cstring>

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "ff.cuh"
#include "grid_sum.cuh"
#include "lda.cuh"
#include "pdl.cuh"
#include "tdks_internal.h"

namespace tdks {

namespace {

constexpr int kFftThreads = 256;
constexpr int kMaxRadices = 16;
constexpr size_t kPlaneSmemLimit = 160 * 1024;   // xy-plane kernels: twiddles + two plane buffers
// the cluster-split plane kernels ask for at least this much shared memory, so that no two of their
// CTAs share an SM (and its FP64 pipes)
constexpr size_t kPlaneClusterMinSmem = 116 * 1024;

struct FftPlanArgs {
  int nrad;
  int rad[kMaxRadices];
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return double2{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

// twiddle exp(dir * 2 pi i t / n) from the table tw[t] = exp(-2 pi i t / n)
__device__ __forceinline__ double2 twd(const double2* tw, int t, int n, int dir) {
  double2 w = tw[t % n];
  if (dir > 0) w.y = -w.y;
  return w;
}

// One radix-R step of a Stockham transform: inputs src[jb + r n/R] times the stage twiddles
// exp(dir 2 pi i r k / (Ns R)), then an R-point DFT with exp(dir 2 pi i r m / R), outputs to
// dst[(jb / Ns) Ns R + k + m Ns].  The small DFTs of R = 2, 3, 4, 5 are written out in their
// standard split forms (sums and differences of conjugate pairs), so a radix-4 step costs three
// complex products and a radix-5 step four instead of R^2.
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return double2{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return double2{a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ double2 cscale(double s, double2 a) { return double2{s * a.x, s * a.y}; }
// dir * i * a
__device__ __forceinline__ double2 cmul_di(int dir, double2 a) {
  return dir > 0 ? double2{-a.y, a.x} : double2{a.y, -a.x};
}

template <int R>
__device__ __forceinline__ void butterfly(const double2* __restrict__ src, double2* __restrict__ dst,
                                          int n, int Ns, int jb, const double2* tw, int dir) {
  const int nr = n / R;
  const int k = jb % Ns;
  const int tstep = n / (Ns * R);                 // r k tstep < n: no reduction needed
  double2 v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    double2 x = src[jb + r * nr];
    if (r > 0 && k > 0) {
      double2 w = tw[r * k * tstep];
      if (dir > 0) w.y = -w.y;
      x = cmul(x, w);
    }
    v[r] = x;
  }
  const int base = (jb / Ns) * Ns * R + k;
  if (R == 2) {
    dst[base] = cadd(v[0], v[1]);
    dst[base + Ns] = csub(v[0], v[1]);
  } else if (R == 3) {
    constexpr double h3 = 0.86602540378443864676;  // sin(2 pi / 3)
    const double2 t = cadd(v[1], v[2]);
    const double2 sm = csub(v[0], cscale(0.5, t));
    const double2 d = cmul_di(dir, cscale(h3, csub(v[1], v[2])));
    dst[base] = cadd(v[0], t);
    dst[base + Ns] = cadd(sm, d);
    dst[base + 2 * Ns] = csub(sm, d);
  } else if (R == 4) {
    const double2 a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
    const double2 c = cadd(v[1], v[3]), d = cmul_di(dir, csub(v[1], v[3]));
    dst[base] = cadd(a, c);
    dst[base + Ns] = cadd(b, d);
    dst[base + 2 * Ns] = csub(a, c);
    dst[base + 3 * Ns] = csub(b, d);
  } else {                                          // R == 5
    constexpr double c1 = 0.30901699437494742410, c2 = -0.80901699437494742410;   // cos(2 pi/5), cos(4 pi/5)
    constexpr double s1 = 0.95105651629515357212, s2 = 0.58778525229247312917;    // sin(2 pi/5), sin(4 pi/5)
    const double2 a1 = cadd(v[1], v[4]), a2 = cadd(v[2], v[3]);
    const double2 b1 = csub(v[1], v[4]), b2 = csub(v[2], v[3]);
    const double2 t1 = cadd(v[0], cadd(cscale(c1, a1), cscale(c2, a2)));
    const double2 t2 = cadd(v[0], cadd(cscale(c2, a1), cscale(c1, a2)));
    const double2 u1 = cmul_di(dir, cadd(cscale(s1, b1), cscale(s2, b2)));
    const double2 u2 = cmul_di(dir, csub(cscale(s2, b1), cscale(s1, b2)));
    dst[base] = cadd(v[0], cadd(a1, a2));
    dst[base + Ns] = cadd(t1, u1);
    dst[base + 4 * Ns] = csub(t1, u1);
    dst[base + 2 * Ns] = cadd(t2, u2);
    dst[base + 3 * Ns] = csub(t2, u2);
  }
}

__device__ void butterfly_generic(const double2* __restrict__ src, double2* __restrict__ dst, int n,
                                  int R, int Ns, int jb, const double2* tw, int dir) {
  const int nr = n / R;
  const int k = jb % Ns;
  const int tstep = n / (Ns * R);
  const int base = (jb / Ns) * Ns * R + k;
  for (int m = 0; m < R; ++m) {
    double2 y = {0.0, 0.0};
    for (int r = 0; r < R; ++r) {
      double2 x = src[jb + r * nr];
      if (r > 0) x = cmul(x, twd(tw, r * k * tstep, n, dir));
      const double2 w = twd(tw, r * m * nr, n, dir);
      y.x += x.x * w.x - x.y * w.y;
      y.y += x.x * w.y + x.y * w.x;
    }
    dst[base + m * Ns] = y;
  }
}

// Transforms nl lines of length n stored one after another in src (Stockham, ping-ponging between
// src and dst); on return src holds the result.  All threads of the CTA take part.
__device__ __forceinline__ void stockham_lines(double2*& src, double2*& dst, int n, int nl, const double2* tw,
                                               const FftPlanArgs& plan, int dir) {
  int Ns = 1;
  for (int s = 0; s < plan.nrad; ++s) {
    const int R = plan.rad[s];
    const int nb = n / R;
    for (int b = threadIdx.x; b < nl * nb; b += blockDim.x) {
      const int j = b / nb, jb = b - j * nb;
      const double2* sl = src + j * n;
      double2* dl = dst + j * n;
      switch (R) {
        case 2: butterfly<2>(sl, dl, n, Ns, jb, tw, dir); break;
        case 3: butterfly<3>(sl, dl, n, Ns, jb, tw, dir); break;
        case 4: butterfly<4>(sl, dl, n, Ns, jb, tw, dir); break;
        case 5: butterfly<5>(sl, dl, n, Ns, jb, tw, dir); break;
        default: butterfly_generic(sl, dl, n, R, Ns, jb, tw, dir); break;
      }
    }
    __syncthreads();
    double2* t = src; src = dst; dst = t;
    Ns *= R;
  }
}

// The same transform computed output by output, for kernels whose lines are few: an FP64
// instruction occupies its SM sub-partition for the same time whether one lane or all 32 are active,
// and one warp's FP64 instructions do not overlap, so a stage costs about the longest chain of FP64
// instructions any thread runs.  A butterfly per thread runs the whole radix-R DFT (a radix-5 step
// with its twiddles: about 50 FP64 instructions); here thread t forms element q of line t / n alone,
//   dst[q] = sum_r src[jb + r n/R] exp(dir 2 pi i r (k tstep + m n/R) / n),
// with q = g Ns R + m Ns + k, jb = g Ns + k, tstep = n / (Ns R) (the stage twiddle and the R-point
// DFT factor merge into one table entry): 4 (R - 1) FMAs, or 2 (R - 1) adds where the factors are
// +-1, +-i (the first stage of radix 2 or 4).  Threads read src and write dst; the caller
// synchronises between stages.
__device__ __forceinline__ void stage_out(const double2* __restrict__ src, double2* __restrict__ dst, int n,
                                          int nl, int R, int Ns, const double2* __restrict__ tw, int dir) {
  const int nr = n / R, span = Ns * R, tstep = n / span;
  for (int t = threadIdx.x; t < nl * n; t += blockDim.x) {
    const int j = t / n, q = t - j * n;
    const int g = q / span, rem = q - g * span;
    const int m = rem / Ns, k = rem - m * Ns;
    const double2* sl = src + j * n + g * Ns + k;
    double2 acc = sl[0];
    if (Ns == 1 && (R == 2 || R == 4)) {
      // factor (-dir i)^(r m) for R = 4, (-1)^(r m) for R = 2: x (-i)^p = (b, -a), (-a, -b), (-b, a)
      for (int r = 1; r < R; ++r) {
        const double2 x = sl[r * nr];
        int p = (R == 4 ? r * m : 2 * r * m) & 3;
        if (dir > 0) p = (4 - p) & 3;
        const double re = (p & 1) ? x.y : x.x, im = (p & 1) ? x.x : x.y;
        acc.x = fma(p < 2 ? 1.0 : -1.0, re, acc.x);
        acc.y = fma((p == 0 || p == 3) ? 1.0 : -1.0, im, acc.y);
      }
    } else {
      const int step = k * tstep + m * nr;             // < n, so (r step) mod n by one wrap per r
      int ti = 0;
      for (int r = 1; r < R; ++r) {
        const double2 x = sl[r * nr];
        ti += step;
        ti -= ti >= n ? n : 0;
        double2 w = tw[ti];
        if (dir > 0) w.y = -w.y;
        acc.x = fma(x.x, w.x, acc.x);
        acc.x = fma(-x.y, w.y, acc.x);
        acc.y = fma(x.x, w.y, acc.y);
        acc.y = fma(x.y, w.x, acc.y);
      }
    }
    dst[t] = acc;
  }
}

// All stages of stage_out over nl lines (ping-pong between src and dst; on return src holds the
// result).
__device__ __forceinline__ void lines_out(double2*& src, double2*& dst, int n, int nl, const double2* tw,
                                          const FftPlanArgs& plan, int dir) {
  int Ns = 1;
  for (int s = 0; s < plan.nrad; ++s) {
    stage_out(src, dst, n, nl, plan.rad[s], Ns, tw, dir);
    __syncthreads();
    double2* t = src; src = dst; dst = t;
    Ns *= plan.rad[s];
  }
}

// stage_out with the line length, radix and stage span known at compile time (the index divisions
// become multiplications); the same arithmetic.
template <int N, int R, int NS>
__device__ __forceinline__ void stage_out_c(const double2* __restrict__ src, double2* __restrict__ dst, int nl,
                                            const double2* __restrict__ tw, int dir) {
  constexpr int nr = N / R, span = NS * R, tstep = N / span;
  for (int t = threadIdx.x; t < nl * N; t += blockDim.x) {
    const int j = t / N, q = t - j * N;
    const int g = q / span, rem = q - g * span;
    const int m = rem / NS, k = rem - m * NS;
    const double2* sl = src + j * N + g * NS + k;
    double2 acc = sl[0];
    if constexpr (NS == 1 && (R == 2 || R == 4)) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const double2 x = sl[r * nr];
        int p = (R == 4 ? r * m : 2 * r * m) & 3;
        if (dir > 0) p = (4 - p) & 3;
        const double re = (p & 1) ? x.y : x.x, im = (p & 1) ? x.x : x.y;
        acc.x = fma(p < 2 ? 1.0 : -1.0, re, acc.x);
        acc.y = fma((p == 0 || p == 3) ? 1.0 : -1.0, im, acc.y);
      }
    } else {
      const int step = k * tstep + m * nr;
      int ti = 0;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const double2 x = sl[r * nr];
        ti += step;
        ti -= ti >= N ? N : 0;
        double2 w = tw[ti];
        if (dir > 0) w.y = -w.y;
        acc.x = fma(x.x, w.x, acc.x);
        acc.x = fma(-x.y, w.y, acc.x);
        acc.y = fma(x.x, w.y, acc.y);
        acc.y = fma(x.y, w.x, acc.y);
      }
    }
    dst[t] = acc;
  }
}

// Lines of a compiled length N (N > 0: 16 = 4 x 4, 20 = 4 x 5, the radix plans of fft_radices) or
// of the runtime length n and plan (N = 0).
template <int N>
__device__ __forceinline__ void lines_any(double2*& src, double2*& dst, int n, int nl, const double2* tw,
                                          const FftPlanArgs& plan, int dir) {
  if constexpr (N == 0) {
    lines_out(src, dst, n, nl, tw, plan, dir);
  } else {
    static_assert(N == 16 || N == 20, "compiled line lengths: 16 and 20");
    stage_out_c<N, 4, 1>(src, dst, nl, tw, dir);
    __syncthreads();
    { double2* t = src; src = dst; dst = t; }
    stage_out_c<N, N / 4, 4>(src, dst, nl, tw, dir);
    __syncthreads();
    { double2* t = src; src = dst; dst = t; }
  }
}

// Optional work fused into a line pass, so the Hartree + exchange solve takes five launches:
//   load_real  (x pass, forward): lines are read from a real array [n2*batch][n1][n0], zero padded
//              to the transform box, instead of from `data` (replaces a packing kernel);
//   spectral   (z pass): after the forward transform each value is multiplied by the Poisson
//              factor of its wave vector (periodic: 4 pi / G^2 / N, G = 0 dropped, from the table
//              ghat when one is given, else computed; isolated: the Hockney spectrum ghat times
//              gscale) and the line is transformed back in place;
//   store_epi  (x pass, inverse): instead of writing the line back, the inside points n0 x n1 x n2
//              get vhxc = Re(value) + V_xc(rho) (lda.cuh: xc = 1 exchange, 2 exchange + correlation).
__device__ __forceinline__ double freq(int m, int n) { return (m <= (n - 1) / 2) ? m : m - n; }

//   zero_from  (forward y and z passes of a padded box): elements e >= zero_from of every line are
//              taken as zero instead of read (that part of the box was never written).
struct FftHooks {
  int load_real;
  int zero_from;
  const double* rsrc;
  int n0, n1, n2;                 // unpadded extent of rsrc / vhxc (n2 per cell)
  int spectral;                   // 0 none, 1 periodic, 2 Hockney
  double L[3];
  double inv_n;
  const double* ghat;
  double gscale;
  int store_epi;
  double* vhxc;
  const double* rho;
  int xc;
  int store_lim;                  // > 0: store only elements e < store_lim of each line
  int herm;                       // 1: elements e > n/2 are conj(element n - e) (a real line's spectrum)
};

// data: 3D array [dims2][dims1][dims0]; transform lines along one axis.  Line l starts at
// (l % cnt_lo) * s_lo + (l / cnt_lo) * s_hi (the two other coordinates), elements estride apart; with
// cnt_mid > 0 the second coordinate h = l / cnt_lo is split further, (h % cnt_mid) * s_hi +
// (h / cnt_mid) * s_cell (the z lines of the x frequencies kx < xh of every cell of a batch).
__global__ void __launch_bounds__(kFftThreads) k_fft_lines(double2* data, int n, int nlines, int LB,
                                                          long long cnt_lo, long long s_lo, long long s_hi,
                                                          long long cnt_mid, long long s_cell,
                                                          long long estride, int xaxis,
                                                          const double2* __restrict__ tw_g,
                                                          FftPlanArgs plan, int dir, int m0, int m1, int m2,
                                                          FftHooks hk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* tw = reinterpret_cast<double2*>(smem_raw);
  double2* b0 = tw + n;
  double2* b1 = b0 + (size_t)LB * n;
  const int l0 = blockIdx.x * LB;
  const int nl = min(LB, nlines - l0);
  for (int t = threadIdx.x; t < n; t += blockDim.x) tw[t] = tw_g[t];
  const int tot = nl * n;
  auto line_start = [&](long long l) -> long long {
    const long long h = l / cnt_lo;
    if (cnt_mid > 0) return (l % cnt_lo) * s_lo + (h % cnt_mid) * s_hi + (h / cnt_mid) * s_cell;
    return (l % cnt_lo) * s_lo + h * s_hi;
  };
  // grid coordinates (x, y, z within the box, cell) of element e of local line j
  auto coords3 = [&](int j, int e, int& x, int& y, int& z) {
    const long long start = line_start(l0 + j) + e * estride;
    x = (int)(start % m0);
    const long long r = start / m0;
    y = (int)(r % m1);
    z = (int)(r / m1);                            // includes the cell: z + cell * m2
  };
  for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
    int j, e;
    if (xaxis) { j = idx / n; e = idx - j * n; } else { e = idx / nl; j = idx - e * nl; }
    const long long start = line_start(l0 + j);
    if (hk.load_real) {
      int x, y, z;
      coords3(j, e, x, y, z);
      const int cell = z / m2, zc = z - cell * m2;
      double v = 0.0;
      if (x < hk.n0 && y < hk.n1 && zc < hk.n2)
        v = hk.rsrc[(((long long)cell * hk.n2 + zc) * hk.n1 + y) * hk.n0 + x];
      b0[j * n + e] = double2{v, 0.0};
    } else if (hk.zero_from > 0 && e >= hk.zero_from) {
      b0[j * n + e] = double2{0.0, 0.0};
    } else if (hk.herm && e > n / 2) {
      const double2 c = data[start + (long long)(n - e) * estride];
      b0[j * n + e] = double2{c.x, -c.y};
    } else {
      b0[j * n + e] = data[start + e * estride];
    }
  }
  __syncthreads();
  double2* src = b0;
  double2* dst = b1;
  stockham_lines(src, dst, n, nl, tw, plan, dir);
  if (hk.spectral) {
    const int cellsz = m0 * m1 * m2;
    for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
      const int j = idx / n, e = idx - j * n;
      double f;
      if (hk.ghat) {   // table of one box: offset of the element within its cell (sizes < 2^31)
        const int off = (int)(line_start(l0 + j) + e * estride);
        f = hk.ghat[off % cellsz];
        if (hk.spectral == 2) f *= hk.gscale;
      } else {
        int x, y, z;
        coords3(j, e, x, y, z);
        const int zc = z % m2;
        const double gx = 2.0 * kPi * freq(x, m0) / hk.L[0], gy = 2.0 * kPi * freq(y, m1) / hk.L[1],
                     gz = 2.0 * kPi * freq(zc, m2) / hk.L[2];
        const double g2 = gx * gx + gy * gy + gz * gz;
        f = (g2 == 0.0) ? 0.0 : 4.0 * kPi / g2 * hk.inv_n;
      }
      const double2 v = src[idx];
      src[idx] = double2{v.x * f, v.y * f};
    }
    __syncthreads();
    stockham_lines(src, dst, n, nl, tw, plan, -dir);
  }
  for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
    int j, e;
    if (xaxis) { j = idx / n; e = idx - j * n; } else { e = idx / nl; j = idx - e * nl; }
    if (hk.store_epi) {
      int x, y, z;
      coords3(j, e, x, y, z);
      const int cell = z / m2, zc = z - cell * m2;
      if (x < hk.n0 && y < hk.n1 && zc < hk.n2) {
        const long long o = (((long long)cell * hk.n2 + zc) * hk.n1 + y) * hk.n0 + x;
        double v = src[j * n + e].x;
        v += lda_vxc(hk.rho[o], hk.xc);
        hk.vhxc[o] = v;
      }
    } else if (hk.store_lim <= 0 || e < hk.store_lim) {
      data[line_start(l0 + j) + e * estride] = src[j * n + e];
    }
  }
}

// Periodic boxes whose xy-plane fits in shared memory: the x and y passes of the Hartree solve run
// in one launch, one CTA per (z plane, cell), with the plane transposed in shared memory between
// the two line sets.  xh < m0: only the x frequencies kx < xh (kx <= m0/2) go through the y (and z)
// passes: the density is real and the Poisson factor real and even, so after the inverse z and y
// passes every x line satisfies X(m0 - kx) = conj(X(kx)), and the inverse x pass rebuilds the rest.
// Forward (FWD): the real density plane rho[cell][z] is transformed along x, then y, and written to
// data.  Inverse: the plane of data is transformed back along y, then x, and
// the epilogue writes vhxc = Re(value) + V_xc(rho) (lda.cuh).  Twiddle tables tw0
// (length m0) and tw1 (length m1); shared memory: m0 + m1 twiddles and two m0 m1 buffers.
template <bool FWD>
__global__ void __launch_bounds__(kFftThreads) k_fft_planes(double2* data, int m0, int m1, int m2,
                                                            const double2* __restrict__ tw0_g,
                                                            const double2* __restrict__ tw1_g,
                                                            FftPlanArgs plan0, FftPlanArgs plan1,
                                                            const double* __restrict__ rho, int xc,
                                                            double* __restrict__ vhxc, int xh) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int np = m0 * m1;
  double2* tw0 = reinterpret_cast<double2*>(smem_raw);
  double2* tw1 = tw0 + m0;
  double2* b0 = tw1 + m1;
  double2* b1 = b0 + np;
  for (int t = threadIdx.x; t < m0; t += blockDim.x) tw0[t] = tw0_g[t];
  for (int t = threadIdx.x; t < m1; t += blockDim.x) tw1[t] = tw1_g[t];
  const long long plane = (long long)blockIdx.x * np;   // blockIdx.x = cell * m2 + z
  double2* src = b0;
  double2* dst = b1;
  if (FWD) {
    for (int i = threadIdx.x; i < np; i += blockDim.x) b0[i] = double2{rho[plane + i], 0.0};   // [y][x]
    __syncthreads();
    stockham_lines(src, dst, m0, m1, tw0, plan0, -1);                 // x lines
    for (int i = threadIdx.x; i < xh * m1; i += blockDim.x) {         // [y][x] -> [x][y], x < xh
      const int x = i / m1, y = i - x * m1;
      dst[x * m1 + y] = src[y * m0 + x];
    }
    __syncthreads();
    { double2* t = src; src = dst; dst = t; }
    stockham_lines(src, dst, m1, xh, tw1, plan1, -1);                 // y lines
    for (int i = threadIdx.x; i < xh * m1; i += blockDim.x) {         // [x][y] -> global [y][x]
      const int y = i / xh, x = i - y * xh;
      data[plane + (long long)y * m0 + x] = src[x * m1 + y];
    }
  } else {
    for (int i = threadIdx.x; i < xh * m1; i += blockDim.x) {         // global [y][x] -> [x][y], x < xh
      const int y = i / xh, x = i - y * xh;
      b0[x * m1 + y] = data[plane + (long long)y * m0 + x];
    }
    __syncthreads();
    stockham_lines(src, dst, m1, xh, tw1, plan1, +1);                 // y lines
    for (int i = threadIdx.x; i < np; i += blockDim.x) {              // [x][y] -> [y][x]
      const int y = i / m0, x = i - y * m0;
      if (x < xh) {
        dst[i] = src[x * m1 + y];
      } else {                                                        // X(m0 - kx) = conj(X(kx))
        const double2 c = src[(m0 - x) * m1 + y];
        dst[i] = double2{c.x, -c.y};
      }
    }
    __syncthreads();
    { double2* t = src; src = dst; dst = t; }
    stockham_lines(src, dst, m0, m1, tw0, plan0, +1);                 // x lines
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
      double v = src[i].x;
      v += lda_vxc(rho[plane + i], xc);
      vhxc[plane + i] = v;
    }
  }
}

// The same two passes for one periodic cell, each z plane split over a thread-block cluster of CL
// CTAs so that the FP64 butterflies of a plane run on CL SMs (the FP64 pipes of the few SMs of one
// CTA per plane are the limit otherwise).  CTA r of a cluster owns the rows y in [r m1 / CL,
// (r+1) m1 / CL) for the x pass and the columns kx in [r xh / CL, (r+1) xh / CL) for the y pass; the
// transpose between the passes writes each value into the shared memory of the CTA that owns it
// (distributed shared memory), then the cluster barrier.  The lines are transformed output by output
// (lines_out), one thread per element.  Forward: rows of the density -> x spectra
// -> columns kx < xh -> y spectra -> data.  Inverse: columns of data -> y inverse -> rows, with
// X(m0 - kx) = conj(X(kx)) filling kx >= xh -> x inverse -> vhxc = Re + vhxc (V_xc(rho), written by the
// z pass launch; V_H alone for xc = 0).  Shared memory:
// m0 + m1 twiddles, two row buffers of rmax x m0 and two column buffers of cmax x m1.  N > 0: a cube
// of edge N (16 or 20) compiled in.
template <bool FWD, int N>
__global__ void __launch_bounds__(kFftThreads) k_fft_planes_cluster(double2* data, int m0_, int m1_, int xh_,
                                                                    const double2* __restrict__ tw0_g,
                                                                    const double2* __restrict__ tw1_g,
                                                                    FftPlanArgs plan0, FftPlanArgs plan1,
                                                                    const double* __restrict__ rho, int xc,
                                                                    double* __restrict__ vhxc, int rmax, int cmax,
                                                                    const double* __restrict__ vpred, double* partials,
                                                                    unsigned* ticket, double* res, int decide, double thr,
                                                                    double* __restrict__ vnext, double* fb,
                                                                    cudaGraphConditionalHandle handle) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int m0 = N > 0 ? N : m0_, m1 = N > 0 ? N : m1_, xh = N > 0 ? N / 2 + 1 : xh_;
  const int CL = (int)cluster.num_blocks();
  const int r = (int)cluster.block_rank();
  __shared__ int rb[9], cb[9];                      // first row / column of each rank (CL <= 8)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* tw0 = reinterpret_cast<double2*>(smem_raw);
  double2* tw1 = tw0 + m0;
  double2* rowA = tw1 + m1;
  double2* rowB = rowA + (size_t)rmax * m0;
  double2* colA = rowB + (size_t)rmax * m0;
  double2* colB = colA + (size_t)cmax * m1;
  // every CTA of the cluster must be running before any writes into its shared memory: arrive here,
  // wait just before the first remote store
  asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
  pdl_trigger();
  for (int t = threadIdx.x; t < m0; t += blockDim.x) tw0[t] = tw0_g[t];     // tables fixed at set-up
  for (int t = threadIdx.x; t < m1; t += blockDim.x) tw1[t] = tw1_g[t];
  if (threadIdx.x <= (unsigned)CL) {
    rb[threadIdx.x] = (int)threadIdx.x * m1 / CL;
    cb[threadIdx.x] = (int)threadIdx.x * xh / CL;
  }
  pdl_wait();                                                                 // the kernel before
  const int y0 = r * m1 / CL, ny = (r + 1) * m1 / CL - y0;
  const int x0 = r * xh / CL, nc = (r + 1) * xh / CL - x0;
  const long long plane = (long long)(blockIdx.x / CL) * m0 * m1;
  if (FWD) {
    for (int i = threadIdx.x; i < ny * m0; i += blockDim.x)
      rowA[i] = double2{rho[plane + (long long)y0 * m0 + i], 0.0};
    __syncthreads();
    double2* src = rowA;
    double2* dst = rowB;
    lines_any<N>(src, dst, m0, ny, tw0, plan0, -1);                 // x lines of the own rows
    asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
    for (int i = threadIdx.x; i < ny * xh; i += blockDim.x) {        // row spectra -> column owners
      const int yy = i / xh, kx = i - yy * xh;
      int o = 0;
      while (o + 1 < CL && cb[o + 1] <= kx) ++o;
      double2* col = cluster.map_shared_rank(colA, o);
      col[(kx - cb[o]) * m1 + y0 + yy] = src[yy * m0 + kx];
    }
    cluster.sync();
    src = colA;
    dst = colB;
    lines_any<N>(src, dst, m1, nc, tw1, plan1, -1);                 // y lines of the own columns
    for (int i = threadIdx.x; i < m1 * nc; i += blockDim.x) {
      const int y = i / nc, c = i - y * nc;
      data[plane + (long long)y * m0 + x0 + c] = src[c * m1 + y];
    }
  } else {
    for (int i = threadIdx.x; i < m1 * nc; i += blockDim.x) {
      const int y = i / nc, c = i - y * nc;
      colA[c * m1 + y] = data[plane + (long long)y * m0 + x0 + c];
    }
    __syncthreads();
    double2* src = colA;
    double2* dst = colB;
    lines_any<N>(src, dst, m1, nc, tw1, plan1, +1);                 // y lines of the own columns
    asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
    for (int i = threadIdx.x; i < nc * m1; i += blockDim.x) {        // -> row owners, with the mirror
      const int c = i / m1, y = i - c * m1, kx = x0 + c;
      int o = 0;
      while (o + 1 < CL && rb[o + 1] <= y) ++o;
      double2* row = cluster.map_shared_rank(rowA, o) + (size_t)(y - rb[o]) * m0;
      const double2 v = src[c * m1 + y];
      row[kx] = v;
      if (kx >= 1 && m0 - kx >= xh) row[m0 - kx] = double2{v.x, -v.y};
    }
    cluster.sync();
    src = rowA;
    dst = rowB;
    lines_any<N>(src, dst, m0, ny, tw0, plan0, +1);                 // x lines of the own rows
    double acc[2] = {0.0, 0.0};                                  // misfit sums (vpred given)
    for (int i = threadIdx.x; i < ny * m0; i += blockDim.x) {   // V_xc from the z pass launch
      const long long o = plane + (long long)y0 * m0 + i;
      const double v = xc > 0 ? src[i].x + vhxc[o] : src[i].x;
      vhxc[o] = v;
      if (decide) vnext[o] = v;
      if (vpred) {
        const double d = v - vpred[o];
        acc[0] += d * d;
        acc[1] += v * v;
      }
    }
    if (vpred) {                                                 // the same for every CTA
      __shared__ double tot[2];
      if (grid_sum<2>(acc, partials, ticket, tot) && threadIdx.x == 0) {
        const double r = sqrt(tot[0] / fmax(tot[1], 1e-300));
        *res = r;
        if (decide) {                                            // as k_decide
          const bool ok = (r <= thr) && (r == r) && (r < 1e300);
          if (!ok) *fb += 1.0;
          cudaGraphSetConditional(handle, ok ? 0u : 1u);
        }
      }
    }
  }
}

// The z pass of one periodic cell after the cluster plane kernels: the z lines of the x frequencies
// kx < xh (all y), LZ lines per CTA, forward, times the Poisson factor pfac of the element, inverse,
// in place; output by output (lines_out), one thread per element.  The CTAs past the z lines form
// V_xc(rho) of every point into vxc (xc > 0), which the inverse plane kernel adds to V_H: the
// exchange-correlation chains run beside the z transforms instead of after the last one.
template <int N>
__global__ void __launch_bounds__(kFftThreads) k_fft_zcol(double2* data, int m0_, int m1_, int m2_, int xh_, int LZ,
                                                         const double2* __restrict__ tw_g, FftPlanArgs plan,
                                                         const double* __restrict__ pfac,
                                                         const double* __restrict__ rho, int xc,
                                                         double* __restrict__ vxc) {
  const int m0 = N > 0 ? N : m0_, m1 = N > 0 ? N : m1_, m2 = N > 0 ? N : m2_, xh = N > 0 ? N / 2 + 1 : xh_;
  pdl_trigger();
  pdl_wait();
  const int nzb = (xh * m1 + LZ - 1) / LZ;
  if ((int)blockIdx.x >= nzb) {
    const int npts = m0 * m1 * m2;
    for (int p = (blockIdx.x - nzb) * blockDim.x + threadIdx.x; p < npts; p += (gridDim.x - nzb) * blockDim.x)
      vxc[p] = lda_vxc(rho[p], xc);
    return;
  }
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* tw = reinterpret_cast<double2*>(smem_raw);
  double2* b0 = tw + m2;
  double2* b1 = b0 + (size_t)LZ * m2;
  for (int t = threadIdx.x; t < m2; t += blockDim.x) tw[t] = tw_g[t];
  const int nlines = xh * m1, l0 = blockIdx.x * LZ;
  const int nl = min(LZ, nlines - l0);
  const int d01 = m0 * m1;
  for (int t = threadIdx.x; t < nl * m2; t += blockDim.x) {   // element e of line j, consecutive lines in x
    const int e = t / nl, j = t - e * nl, l = l0 + j;
    const int y = l / xh, x = l - y * xh;
    b0[j * m2 + e] = data[x + y * m0 + e * d01];
  }
  __syncthreads();
  double2* src = b0;
  double2* dst = b1;
  lines_any<N>(src, dst, m2, nl, tw, plan, -1);
  for (int t = threadIdx.x; t < nl * m2; t += blockDim.x) {
    const int j = t / m2, e = t - j * m2, l = l0 + j;
    const int y = l / xh, x = l - y * xh;
    const double f = pfac[x + y * m0 + e * d01];
    src[t] = double2{src[t].x * f, src[t].y * f};
  }
  __syncthreads();
  lines_any<N>(src, dst, m2, nl, tw, plan, +1);
  for (int t = threadIdx.x; t < nl * m2; t += blockDim.x) {
    const int e = t / nl, j = t - e * nl, l = l0 + j;
    const int y = l / xh, x = l - y * xh;
    data[x + y * m0 + e * d01] = src[j * m2 + e];
  }
}

// The periodic Poisson factor of every wave vector of one box: 4 pi / G^2 * inv_n, 0 at G = 0
// (the same arithmetic as the computed form of the spectral hook).
__global__ void k_poisson_table(double* __restrict__ t, int m0, int m1, int m2, double L0, double L1, double L2,
                                double inv_n) {
  const int total = m0 * m1 * m2;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int x = i % m0, y = (i / m0) % m1, z = i / (m0 * m1);
    const double gx = 2.0 * kPi * freq(x, m0) / L0, gy = 2.0 * kPi * freq(y, m1) / L1,
                 gz = 2.0 * kPi * freq(z, m2) / L2;
    const double g2 = gx * gx + gy * gy + gz * gz;
    t[i] = (g2 == 0.0) ? 0.0 : 4.0 * kPi / g2 * inv_n;
  }
}

__global__ void k_pack_real(const double* __restrict__ src, int nx, int ny, int nz,
                            double2* __restrict__ dst, int mx, int my, int mz) {
  const long long total = (long long)mx * my * mz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % mx);
    const long long r = i / mx;
    const int y = (int)(r % my), z = (int)(r / my);
    double v = 0.0;
    if (x < nx && y < ny && z < nz) v = src[((long long)z * ny + y) * nx + x];
    dst[i] = double2{v, 0.0};
  }
}

__global__ void k_poisson_periodic(double2* data, int nx, int ny, int nz, double Lx, double Ly,
                                   double Lz, int batch) {
  const long long cellsz = (long long)nx * ny * nz;
  const long long total = cellsz * batch;
  const double inv_n = 1.0 / (double)cellsz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long j = i % cellsz;
    const int x = (int)(j % nx);
    const long long r = j / nx;
    const int y = (int)(r % ny), z = (int)(r / ny);
    const double gx = 2.0 * kPi * freq(x, nx) / Lx, gy = 2.0 * kPi * freq(y, ny) / Ly,
                 gz = 2.0 * kPi * freq(z, nz) / Lz;
    const double g2 = gx * gx + gy * gy + gz * gz;
    const double f = (g2 == 0.0) ? 0.0 : 4.0 * kPi / g2 * inv_n;
    double2 v = data[i];
    data[i] = double2{v.x * f, v.y * f};
  }
}

__global__ void k_scale_by_real(double2* data, const double* __restrict__ g, double scale,
                                long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const double f = g[i] * scale;
    double2 v = data[i];
    data[i] = double2{v.x * f, v.y * f};
  }
}

__global__ void k_hxc_epilogue(const double2* __restrict__ fft, int mx, int my,
                               const double* __restrict__ rho, int nx, int ny, int nz,
                               double scale_h, int hartree, int xc, double* __restrict__ vhxc) {
  const long long total = (long long)nx * ny * nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx);
    const long long r = i / nx;
    const int y = (int)(r % ny), z = (int)(r / ny);
    double v = 0.0;
    if (hartree) v += scale_h * fft[((long long)z * my + y) * mx + x].x;
    v += lda_vxc(rho[i], xc);
    vhxc[i] = v;
  }
}

__global__ void k_combine(const double* __restrict__ vloc, const double* __restrict__ v1, double a,
                          const double* __restrict__ v2, double b, double* __restrict__ o64,
                          float* __restrict__ o32, int npts, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double v = vloc[i % npts];
    if (v1) v += a * v1[i];
    if (v2) v += b * v2[i];
    if (o64) o64[i] = v;
    if (o32) o32[i] = (float)v;
  }
}

template <typename C>
__global__ void k_density(const C* __restrict__ psi, int nk, int norb, int npts,
                          const double* __restrict__ kw, double* __restrict__ rho) {
  using R = decltype(C{}.x);
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npts; p += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int k = 0; k < nk; ++k) {
      R s = 0;                        // per-k partial in the orbital precision
      for (int n = 0; n < norb; ++n) {
        const C u = psi[((size_t)k * norb + n) * npts + p];
        s += u.x * u.x + u.y * u.y;
      }
      acc += 2.0 * kw[k] * (double)s;
    }
    rho[p] = acc;
  }
}

__device__ __forceinline__ double coord(int j, int n, double h, int periodic) {
  return periodic ? j * h : (j - 0.5 * (n - 1)) * h;
}

template <typename C>
__global__ void k_kick(C* psi, long long norb_tot, int nx, int ny, int nz, double hx, double hy,
                       double hz, int periodic, double kx, double ky, double kz) {
  const long long npts = (long long)nx * ny * nz;
  const long long total = npts * norb_tot;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long p = i % npts;
    const int x = (int)(p % nx);
    const long long r = p / nx;
    const int y = (int)(r % ny), z = (int)(r / ny);
    const double arg = kx * coord(x, nx, hx, periodic) + ky * coord(y, ny, hy, periodic) +
                       kz * coord(z, nz, hz, periodic);
    double s, c;
    sincos(arg, &s, &c);
    C u = psi[i];
    const double re = u.x * c - u.y * s, im = u.x * s + u.y * c;
    psi[i] = C{(decltype(u.x))re, (decltype(u.x))im};
  }
}

__global__ void k_vloc_isolated(double* v, int nx, int ny, int nz, double hx, double hy, double hz,
                                const double* __restrict__ atoms, int natom) {
  const long long total = (long long)nx * ny * nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx);
    const long long r = i / nx;
    const int y = (int)(r % ny), z = (int)(r / ny);
    const double px = coord(x, nx, hx, 0), py = coord(y, ny, hy, 0), pz = coord(z, nz, hz, 0);
    double acc = 0.0;
    for (int a = 0; a < natom; ++a) {
      const double dx = px - atoms[5 * a], dy = py - atoms[5 * a + 1], dz = pz - atoms[5 * a + 2];
      const double Z = atoms[5 * a + 3], sg = atoms[5 * a + 4];
      const double d = sqrt(dx * dx + dy * dy + dz * dz);
      acc += (d == 0.0) ? -2.0 * Z / (sg * sqrt(kPi)) : -Z * erf(d / sg) / d;
    }
    v[i] = acc;
  }
}

__global__ void k_hockney(double2* g, int mx, int my, int mz, int nx, int ny, int nz, double hx,
                          double hy, double hz, double g0) {
  const long long total = (long long)mx * my * mz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % mx);
    const long long r = i / mx;
    const int y = (int)(r % my), z = (int)(r / my);
    const double dx = ((x <= nx) ? x : mx - x) * hx;
    const double dy = ((y <= ny) ? y : my - y) * hy;
    const double dz = ((z <= nz) ? z : mz - z) * hz;
    const double d = sqrt(dx * dx + dy * dy + dz * dz);
    g[i] = double2{(i == 0) ? g0 : 1.0 / d, 0.0};
  }
}

__global__ void k_real_part(const double2* __restrict__ s, double* __restrict__ d, long long n,
                            double scale) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    d[i] = s[i].x * scale;
}

__global__ void k_f32(const double* __restrict__ s, float* __restrict__ d, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    d[i] = (float)s[i];
}

constexpr int kRedThreads = 256;

// d_mu = -sum r_mu (rho - rho0) dV and N = sum rho dV, summed over all CTAs by grid_sum;
// out[3..5] = d, out[6] = N.
__global__ void __launch_bounds__(kRedThreads) k_dipole(
    const double* __restrict__ rho, const double* __restrict__ rho0, int nx, int ny, int nz,
    double hx, double hy, double hz, int periodic, double* partials, unsigned* ticket, double* out) {
  __shared__ double tot[4];
  double acc[4] = {0, 0, 0, 0};
  const long long total = (long long)nx * ny * nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx);
    const long long r = i / nx;
    const int y = (int)(r % ny), z = (int)(r / ny);
    const double dr = rho[i] - rho0[i];
    acc[0] += coord(x, nx, hx, periodic) * dr;
    acc[1] += coord(y, ny, hy, periodic) * dr;
    acc[2] += coord(z, nz, hz, periodic) * dr;
    acc[3] += rho[i];
  }
  if (!grid_sum<4>(acc, partials, ticket, tot)) return;
  if (threadIdx.x < 4) {
    const double dV = hx * hy * hz;
    out[3 + threadIdx.x] = (threadIdx.x < 3) ? -tot[threadIdx.x] * dV : tot[threadIdx.x] * dV;
  }
}

// J_d = -(1/Omega) sum_k w_k sum_n 2 (jloc_d + jnl_d): one block, fixed-order tree reduction.
__global__ void __launch_bounds__(256) k_reduce_current(const double* __restrict__ obs, int nk, int norb,
                                                        const double* __restrict__ kw, double inv_omega,
                                                        int periodic, double* out) {
  __shared__ double red[3][256];
  double acc[3] = {0, 0, 0};
  const int tot = nk * norb;
  const double* ob = obs + (size_t)blockIdx.x * tot * 8;   // this block's cell
  out += blockIdx.x * 8;
  if (periodic)
#pragma unroll 4
    for (int o = threadIdx.x; o < tot; o += blockDim.x) {   // unrolled: the loads of 4 orbitals in flight
      const double w = 2.0 * kw[o / norb];
      for (int d = 0; d < 3; ++d) acc[d] += w * (ob[(size_t)o * 8 + 1 + d] + ob[(size_t)o * 8 + 4 + d]);
    }
  for (int d = 0; d < 3; ++d) red[d][threadIdx.x] = acc[d];
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h)
      for (int d = 0; d < 3; ++d) red[d][threadIdx.x] += red[d][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x < 3) out[threadIdx.x] = -red[threadIdx.x][0] * inv_omega;
}

template <typename C>
__global__ void __launch_bounds__(256) k_orbital_dots(const C* __restrict__ u, const C* __restrict__ hu,
                                                      int npts, double dV, double* out) {
  __shared__ double red[2][256];
  const int o = blockIdx.x;
  const C* a = u + (size_t)o * npts;
  const C* b = hu ? hu + (size_t)o * npts : nullptr;
  double n = 0, e = 0;
  for (int p = threadIdx.x; p < npts; p += blockDim.x) {
    const C x = a[p];
    n += (double)x.x * x.x + (double)x.y * x.y;
    if (b) { const C y = b[p]; e += (double)x.x * y.x + (double)x.y * y.y; }
  }
  red[0][threadIdx.x] = n;
  red[1][threadIdx.x] = e;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) { red[0][threadIdx.x] += red[0][threadIdx.x + h]; red[1][threadIdx.x] += red[1][threadIdx.x + h]; }
    __syncthreads();
  }
  if (threadIdx.x < 8) {
    double v = 0;
    if (threadIdx.x == 0) v = red[0][0] * dV;
    if (threadIdx.x == 7) v = red[1][0] * dV;
    out[(size_t)o * 8 + threadIdx.x] = v;
  }
}

// rho[cell][p] = sum_k w_k rho32[cell][k][p].  Eight lanes share a point, each summing every eighth
// k in float-float (ff.cuh) with the weights as float pairs (split once at set-up), four loads in
// flight before their sums (the partials were just written: L2 latency), then the lanes add their
// sums by shuffles; one FP64 conversion per point.  32-bit indices (the host checks the size).
constexpr int kFoldLanes = 8;
__global__ void __launch_bounds__(256) k_fold_density(const float* __restrict__ r32, int nk, int npts,
                                                      const float* __restrict__ wsplit, double* __restrict__ rho,
                                                      long long n) {
  pdl_trigger();                                    // the Hartree solve may be scheduled (pdl.cuh)
  const int total = (int)n * kFoldLanes;
  for (int t0 = blockIdx.x * blockDim.x; t0 < total; t0 += gridDim.x * blockDim.x) {
    const int t = t0 + threadIdx.x;                 // every lane of the warp runs the iteration
    const bool act = t < total;
    const int i = act ? t / kFoldLanes : 0;
    const int part = t % kFoldLanes;
    FF acc{0.f, 0.f};
    if (act) {
      const int cell = i / npts, p = i - cell * npts;
      const float* base = r32 + cell * nk * npts + p;
      int k = part;
      for (; k + 3 * kFoldLanes < nk; k += 4 * kFoldLanes) {
        float x[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) x[j] = base[(k + j * kFoldLanes) * npts];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int kk = k + j * kFoldLanes;
          acc = ff_add(acc, ff_mul(__ldg(wsplit + 2 * kk), __ldg(wsplit + 2 * kk + 1), x[j]));
        }
      }
      for (; k < nk; k += kFoldLanes)
        acc = ff_add(acc, ff_mul(__ldg(wsplit + 2 * k), __ldg(wsplit + 2 * k + 1), base[k * npts]));
    }
#pragma unroll
    for (int o = 1; o < kFoldLanes; o <<= 1) acc = ff_add(acc, ff_shfl_xor(acc, o));
    if (act && part == 0) rho[i] = ff_to_double(acc);
  }
}

int grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

cudaError_t launch_fft_axis_hooked(double2* data, const int dims[3], int axis, int dir, const double2* tw,
                                   const int* radices, int nrad, cudaStream_t s, int batch, int lim_lo,
                                   int lim_hi, const void* hooks, int zx_lim = 0);

cudaError_t launch_fft_axis(double2* data, const int dims[3], int axis, int dir, const double2* tw,
                            const int* radices, int nrad, cudaStream_t s, int batch, int lim_lo, int lim_hi) {
  FftHooks hk;
  std::memset(&hk, 0, sizeof(hk));
  return launch_fft_axis_hooked(data, dims, axis, dir, tw, radices, nrad, s, batch, lim_lo, lim_hi, &hk);
}

// zx_lim > 0 (z axis): only the z lines of x < zx_lim, every y (and every cell of a batch).
cudaError_t launch_fft_axis_hooked(double2* data, const int dims[3], int axis, int dir, const double2* tw,
                                   const int* radices, int nrad, cudaStream_t s, int batch, int lim_lo,
                                   int lim_hi, const void* hooks, int zx_lim) {
  const FftHooks& hk = *static_cast<const FftHooks*>(hooks);
  const int n = dims[axis];
  if (nrad > kMaxRadices) return cudaErrorInvalidValue;
  FftPlanArgs plan;
  plan.nrad = nrad;
  for (int i = 0; i < nrad; ++i) plan.rad[i] = radices[i];
  // the two other coordinates of a line: lo (faster) and hi; hi of the last axis runs over the batch
  long long cnt_lo, cnt_hi, s_lo, s_hi, estride, cnt_mid = 0, s_cell = 0;
  const long long d01 = (long long)dims[0] * dims[1];
  if (axis == 0) { cnt_lo = dims[1]; cnt_hi = (long long)dims[2] * batch; s_lo = dims[0]; s_hi = d01; estride = 1; }
  else if (axis == 1) { cnt_lo = dims[0]; cnt_hi = (long long)dims[2] * batch; s_lo = 1; s_hi = d01; estride = dims[0]; }
  else if (zx_lim > 0 && batch == 1) { cnt_lo = zx_lim; cnt_hi = dims[1]; s_lo = 1; s_hi = dims[0]; estride = d01; }
  else if (zx_lim > 0) {                 // x < zx_lim, every y, every cell
    cnt_lo = zx_lim; cnt_hi = (long long)dims[1] * batch; s_lo = 1; s_hi = dims[0];
    cnt_mid = dims[1]; s_cell = d01 * dims[2]; estride = d01;
  }
  else { cnt_lo = d01; cnt_hi = batch; s_lo = 1; s_hi = d01 * dims[2]; estride = d01; }
  // pruned transforms: only the lines with lo < lim_lo and hi < lim_hi (a zero-padded input, or
  // an output of which only a corner is used)
  const long long use_lo = (lim_lo > 0 && lim_lo < cnt_lo) ? lim_lo : cnt_lo;
  const long long use_hi = (lim_hi > 0 && lim_hi < cnt_hi) ? lim_hi : cnt_hi;
  const int nlines = (int)(use_lo * use_hi);
  // lines per CTA: at most 16 and what 96 KB of shared memory holds, and few enough that the
  // lines spread over all SMs (two CTAs per SM), since each SM's FP64 rate bounds its share
  int LB = 16;
  while (LB > 1 && (size_t)(2 * LB + 1) * n * sizeof(double2) > 96 * 1024) LB /= 2;
  while (LB > 1 && nlines / LB < 2 * 152) LB /= 2;
  const size_t smem = (size_t)(2 * LB + 1) * n * sizeof(double2);
  cudaError_t e = cudaFuncSetAttribute(k_fft_lines, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = (nlines + LB - 1) / LB;
  k_fft_lines<<<grid, kFftThreads, smem, s>>>(data, n, nlines, LB, use_lo, s_lo, s_hi, cnt_mid, s_cell, estride,
                                              axis == 0 ? 1 : 0, tw, plan, dir, dims[0], dims[1], dims[2], hk);
  return cudaGetLastError();
}

namespace {

size_t plane_cluster_smem(const int m[3], int cl) {
  const int xh = m[0] / 2 + 1;
  const int rmax = (m[1] + cl - 1) / cl, cmax = (xh + cl - 1) / cl;
  const size_t need = ((size_t)m[0] + m[1] + 2 * (size_t)rmax * m[0] + 2 * (size_t)cmax * m[1]) * sizeof(double2);
  return need > kPlaneClusterMinSmem ? need : kPlaneClusterMinSmem;
}

}  // namespace

int hartree_plane_cluster(const int m[3], int batch, int periodic) {
  const size_t plane_smem = ((size_t)m[0] + m[1] + 2 * (size_t)m[0] * m[1]) * sizeof(double2);
  if (!periodic || batch != 1 || plane_smem > kPlaneSmemLimit) return 0;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const int xh = m[0] / 2 + 1;
  for (int cl = 8; cl >= 2; --cl) {
    if (cl > m[1] || cl > xh || m[2] * cl > nsm) continue;
    const size_t smem = plane_cluster_smem(m, cl);
    if (cudaFuncSetAttribute(k_fft_planes_cluster<true, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(m[2] * cl));
    cfg.blockDim = dim3(kFftThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, (const void*)k_fft_planes_cluster<true, 0>, &cfg) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (nclusters >= m[2]) return cl;     // every plane's cluster resident at once
  }
  return 0;
}

namespace {

// The cube edge compiled into the single-cell kernels (16 or 20), 0 for other boxes.
int compiled_edge(const int m[3]) {
  return (m[0] == m[1] && m[1] == m[2] && (m[0] == 16 || m[0] == 20)) ? m[0] : 0;
}

template <bool FWD>
cudaError_t launch_planes_cluster(double2* work, const int m[3], int cl, const double2* tw0, const double2* tw1,
                                  const FftPlanArgs& p0, const FftPlanArgs& p1, const double* rho, int xc,
                                  double* vhxc, cudaStream_t s, const ResidualArgs* ra = nullptr) {
  const int xh = m[0] / 2 + 1;
  const int rmax = (m[1] + cl - 1) / cl, cmax = (xh + cl - 1) / cl;
  const size_t smem = plane_cluster_smem(m, cl);
  const int edge = compiled_edge(m);
  auto kern = edge == 20 ? k_fft_planes_cluster<FWD, 20> : edge == 16 ? k_fft_planes_cluster<FWD, 16>
                                                                       : k_fft_planes_cluster<FWD, 0>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // one thread per element of the larger line set (rows or columns)
  int threads = rmax * m[0] > cmax * m[1] ? rmax * m[0] : cmax * m[1];
  threads = (threads + 31) / 32 * 32;
  if (threads > kFftThreads) threads = kFftThreads;
  const double* vpred = ra ? ra->vpred : nullptr;
  double* partials = ra ? ra->partials : nullptr;
  unsigned* ticket = ra ? ra->ticket : nullptr;
  double* res = ra ? ra->res : nullptr;
  const int decide = ra ? ra->decide : 0;
  const double thr = ra ? ra->thr : 0.0;
  double* vnext = ra ? ra->vnext : nullptr;
  double* fb = ra ? ra->fb : nullptr;
  const cudaGraphConditionalHandle handle = ra ? ra->handle : cudaGraphConditionalHandle{};
  return launch_pdl(kern, dim3((unsigned)(m[2] * cl)), dim3((unsigned)threads), smem, s, cl, work, m[0], m[1], xh,
                    tw0, tw1, p0, p1, rho, xc, vhxc, rmax, cmax, vpred, partials, ticket, res, decide, thr, vnext,
                    fb, handle);
}

// z pass of one cell for the cluster plane path: LZ lines per CTA so that the CTAs about fill the SMs;
// with xc > 0 further CTAs write V_xc(rho) to vxc
cudaError_t launch_zcol(double2* work, const int m[3], const double2* tw2, const FftPlanArgs& p2,
                        const double* pfac, const double* rho, int xc, double* vxc, cudaStream_t s) {
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int xh = m[0] / 2 + 1, nlines = xh * m[1];
  int LZ = (nlines + nsm - 1) / nsm;
  while (LZ > 1 && LZ * m[2] > kFftThreads) --LZ;
  int threads = (LZ * m[2] + 31) / 32 * 32;
  if (threads > kFftThreads) threads = kFftThreads;
  const size_t smem = ((size_t)m[2] + 2 * (size_t)LZ * m[2]) * sizeof(double2);
  const int edge = compiled_edge(m);
  auto kern = edge == 20 ? k_fft_zcol<20> : edge == 16 ? k_fft_zcol<16> : k_fft_zcol<0>;
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
    return e;
  const int nzb = (nlines + LZ - 1) / LZ;
  const int nxb = xc > 0 ? (m[0] * m[1] * m[2] + threads - 1) / threads : 0;
  return launch_pdl(kern, dim3((unsigned)(nzb + nxb)), dim3((unsigned)threads), smem, s, 0, work, m[0], m[1], m[2],
                    xh, LZ, tw2, p2, pfac, rho, xc, vxc);
}

}  // namespace

// Hartree (periodic 4 pi / G^2, or Hockney with the kernel spectrum ghat) + exchange in five line
// passes: x forward from the real density, y forward, z forward-multiply-inverse, y inverse, and
// x inverse writing vhxc (see FftHooks).  Periodic boxes whose xy-plane fits in shared memory take
// three launches instead: xy planes forward, the z pass, xy planes inverse with the epilogue
// (k_fft_planes).  *nlaunch (nullable) receives the number of launches.
cudaError_t launch_hartree_xc_fused(double2* work, const int m[3], const int n[3], int batch, int periodic,
                                    const double h[3], const double* ghat, double gscale,
                                    double2* const tw[3], const int* const rad[3], const int nrad[3],
                                    const double* rho, int xc, double* vhxc, cudaStream_t s, int* nlaunch,
                                    int plane_cl, ResidualArgs* resid) {
  FftHooks base;
  std::memset(&base, 0, sizeof(base));
  base.n0 = n[0]; base.n1 = n[1]; base.n2 = n[2];
  const int lo_x = periodic ? 0 : n[1], hi_xy = periodic ? 0 : n[2];
  cudaError_t e;
  const size_t plane_smem = ((size_t)m[0] + m[1] + 2 * (size_t)m[0] * m[1]) * sizeof(double2);
  if (periodic && plane_smem <= kPlaneSmemLimit && nrad[0] <= kMaxRadices && nrad[1] <= kMaxRadices) {
    // three launches: xy planes forward, z forward-multiply-inverse, xy planes inverse + exchange
    FftPlanArgs p0, p1;
    p0.nrad = nrad[0];
    p1.nrad = nrad[1];
    for (int i = 0; i < nrad[0]; ++i) p0.rad[i] = rad[0][i];
    for (int i = 0; i < nrad[1]; ++i) p1.rad[i] = rad[1][i];
    const int grid = m[2] * batch;
    // the y and z passes only on the x frequencies kx <= m0/2 (see k_fft_planes)
    const int xhp = m[0] / 2 + 1;
    const bool split = plane_cl >= 2 && batch == 1 && ghat && nrad[2] <= kMaxRadices;
    if (split) {
      if ((e = launch_planes_cluster<true>(work, m, plane_cl, tw[0], tw[1], p0, p1, rho, 0, nullptr, s)) !=
          cudaSuccess)
        return e;
    } else {
      if ((e = cudaFuncSetAttribute(k_fft_planes<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)plane_smem)) != cudaSuccess) return e;
      if ((e = cudaFuncSetAttribute(k_fft_planes<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)plane_smem)) != cudaSuccess) return e;
      k_fft_planes<true><<<grid, kFftThreads, plane_smem, s>>>(work, m[0], m[1], m[2], tw[0], tw[1], p0, p1, rho,
                                                               0, nullptr, xhp);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (split) {
      FftPlanArgs p2;
      p2.nrad = nrad[2];
      for (int i = 0; i < nrad[2]; ++i) p2.rad[i] = rad[2][i];
      if ((e = launch_zcol(work, m, tw[2], p2, ghat, rho, xc, vhxc, s)) != cudaSuccess) return e;
    } else {
      FftHooks h3 = base;
      h3.spectral = 1;
      for (int a = 0; a < 3; ++a) h3.L[a] = m[a] * h[a];
      h3.inv_n = 1.0 / ((double)m[0] * m[1] * m[2]);
      h3.ghat = ghat;
      if ((e = launch_fft_axis_hooked(work, m, 2, -1, tw[2], rad[2], nrad[2], s, batch, 0, 0, &h3,
                                      xhp)) != cudaSuccess)
        return e;
    }
    if (nlaunch) *nlaunch = 3;
    if (resid && resid->decide && !split) return cudaErrorInvalidValue;   // the caller expected the fused form
    if (split) {
      const bool with_res = resid && resid->vpred && m[2] * plane_cl <= 304;   // partials [304][2]
      e = launch_planes_cluster<false>(work, m, plane_cl, tw[0], tw[1], p0, p1, rho, xc, vhxc, s,
                                       with_res ? resid : nullptr);
      if (e == cudaSuccess && with_res) resid->done = 1;
      return e;
    }
    k_fft_planes<false><<<grid, kFftThreads, plane_smem, s>>>(work, m[0], m[1], m[2], tw[0], tw[1], p0, p1, rho,
                                                              xc, vhxc, xhp);
    return cudaGetLastError();
  }
  if (nlaunch) *nlaunch = 5;
  // The density is real and the Poisson factor (4 pi / G^2, or the spectrum of the even Green's
  // function) real and even, so every x line of the spectrum, after the y and z transforms in
  // either direction, satisfies X(m0 - k) = conj(X(k)): the y and z passes only transform the
  // x frequencies k <= m0/2, and the inverse x pass rebuilds the rest.
  const int xh = m[0] / 2 + 1;
  FftHooks h1 = base;
  h1.load_real = 1;
  h1.rsrc = rho;
  h1.store_lim = xh;
  if ((e = launch_fft_axis_hooked(work, m, 0, -1, tw[0], rad[0], nrad[0], s, batch, lo_x, hi_xy, &h1)) != cudaSuccess) return e;
  // the padded box (isolated) is written only where the density is: the forward y and z passes
  // read the rest as zeros
  FftHooks h2 = base;
  h2.zero_from = periodic ? 0 : n[1];
  if ((e = launch_fft_axis_hooked(work, m, 1, -1, tw[1], rad[1], nrad[1], s, batch, xh, hi_xy, &h2)) != cudaSuccess) return e;
  FftHooks h3 = base;
  h3.zero_from = periodic ? 0 : n[2];
  h3.spectral = periodic ? 1 : 2;
  for (int a = 0; a < 3; ++a) h3.L[a] = m[a] * h[a];
  h3.inv_n = 1.0 / ((double)m[0] * m[1] * m[2]);
  h3.ghat = ghat;
  h3.gscale = gscale;
  if ((e = launch_fft_axis_hooked(work, m, 2, -1, tw[2], rad[2], nrad[2], s, batch, 0, 0, &h3, xh)) != cudaSuccess) return e;
  if ((e = launch_fft_axis_hooked(work, m, 1, +1, tw[1], rad[1], nrad[1], s, batch, xh, hi_xy, &base)) != cudaSuccess) return e;
  FftHooks h5 = base;
  h5.herm = xh > 0 ? 1 : 0;
  h5.store_epi = 1;
  h5.vhxc = vhxc;
  h5.rho = rho;
  h5.xc = xc;
  return launch_fft_axis_hooked(work, m, 0, +1, tw[0], rad[0], nrad[0], s, batch, lo_x, hi_xy, &h5);
}

cudaError_t launch_pack_real(const double* src, const int n[3], double2* dst, const int m[3],
                             cudaStream_t s) {
  const long long tot = (long long)m[0] * m[1] * m[2];
  k_pack_real<<<grid_for(tot, 256), 256, 0, s>>>(src, n[0], n[1], n[2], dst, m[0], m[1], m[2]);
  return cudaGetLastError();
}

cudaError_t launch_poisson_scale_periodic(double2* data, const int n[3], const double h[3],
                                          cudaStream_t s, int batch) {
  const long long tot = (long long)n[0] * n[1] * n[2] * batch;
  k_poisson_periodic<<<grid_for(tot, 256), 256, 0, s>>>(data, n[0], n[1], n[2], n[0] * h[0],
                                                         n[1] * h[1], n[2] * h[2], batch);
  return cudaGetLastError();
}

cudaError_t launch_scale_by_real(double2* data, const double* ghat, double scale, size_t count,
                                 cudaStream_t s) {
  k_scale_by_real<<<grid_for((long long)count, 256), 256, 0, s>>>(data, ghat, scale, (long long)count);
  return cudaGetLastError();
}

cudaError_t launch_hxc_epilogue(const double2* fft, const int m[3], const double* rho,
                                const int n[3], double scale_h, int hartree, int xc, double* vhxc,
                                cudaStream_t s) {
  const long long tot = (long long)n[0] * n[1] * n[2];
  k_hxc_epilogue<<<grid_for(tot, 256), 256, 0, s>>>(fft, m[0], m[1], rho, n[0], n[1], n[2],
                                                     scale_h, hartree, xc, vhxc);
  return cudaGetLastError();
}

cudaError_t launch_combine_potential(const double* vloc, const double* v1, double a,
                                     const double* v2, double b, double* v64, float* v32, int npts,
                                     cudaStream_t s, int batch) {
  const long long n = (long long)npts * batch;
  k_combine<<<grid_for(n, 256), 256, 0, s>>>(vloc, v1, a, v2, b, v64, v32, npts, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_density(const typename Cplx<T>::type* psi, int nk, int norb, int npts,
                           const double* kw, double* rho, cudaStream_t s) {
  k_density<<<grid_for(npts, 256), 256, 0, s>>>(psi, nk, norb, npts, kw, rho);
  return cudaGetLastError();
}
template cudaError_t launch_density<float>(const float2*, int, int, int, const double*, double*, cudaStream_t);
template cudaError_t launch_density<double>(const double2*, int, int, int, const double*, double*, cudaStream_t);

template <typename T>
cudaError_t launch_kick(typename Cplx<T>::type* psi, int norb_tot, const int n[3], const double h[3],
                        int periodic, const double kappa[3], cudaStream_t s) {
  const long long tot = (long long)n[0] * n[1] * n[2] * norb_tot;
  k_kick<<<grid_for(tot, 256), 256, 0, s>>>(psi, norb_tot, n[0], n[1], n[2], h[0], h[1], h[2],
                                            periodic, kappa[0], kappa[1], kappa[2]);
  return cudaGetLastError();
}
template cudaError_t launch_kick<float>(float2*, int, const int*, const double*, int, const double*, cudaStream_t);
template cudaError_t launch_kick<double>(double2*, int, const int*, const double*, int, const double*, cudaStream_t);

cudaError_t launch_vloc_isolated(double* v, const int n[3], const double h[3], const double* atoms,
                                 int natom, cudaStream_t s) {
  const long long tot = (long long)n[0] * n[1] * n[2];
  k_vloc_isolated<<<grid_for(tot, 256), 256, 0, s>>>(v, n[0], n[1], n[2], h[0], h[1], h[2], atoms, natom);
  return cudaGetLastError();
}

cudaError_t launch_hockney_kernel(double2* g, const int m[3], const int n[3], const double h[3],
                                  double g0, cudaStream_t s) {
  const long long tot = (long long)m[0] * m[1] * m[2];
  k_hockney<<<grid_for(tot, 256), 256, 0, s>>>(g, m[0], m[1], m[2], n[0], n[1], n[2], h[0], h[1], h[2], g0);
  return cudaGetLastError();
}

cudaError_t launch_poisson_table(double* t, const int m[3], const double h[3], cudaStream_t s) {
  const long long tot = (long long)m[0] * m[1] * m[2];
  k_poisson_table<<<grid_for(tot, 256), 256, 0, s>>>(t, m[0], m[1], m[2], m[0] * h[0], m[1] * h[1], m[2] * h[2],
                                                     1.0 / (double)tot);
  return cudaGetLastError();
}

cudaError_t launch_real_part(const double2* src, double* dst, size_t count, double scale, cudaStream_t s) {
  k_real_part<<<grid_for((long long)count, 256), 256, 0, s>>>(src, dst, (long long)count, scale);
  return cudaGetLastError();
}

cudaError_t launch_f32_from_f64(const double* src, float* dst, size_t count, cudaStream_t s) {
  k_f32<<<grid_for((long long)count, 256), 256, 0, s>>>(src, dst, (long long)count);
  return cudaGetLastError();
}

cudaError_t launch_dipole(const double* rho, const double* rho0, const int n[3], const double h[3],
                          int periodic, double* partials, unsigned* ticket, double* out, cudaStream_t s) {
  const long long total = (long long)n[0] * n[1] * n[2];
  k_dipole<<<grid_sum_blocks(total, kRedThreads), kRedThreads, 0, s>>>(rho, rho0, n[0], n[1], n[2], h[0], h[1],
                                                                       h[2], periodic, partials, ticket, out);
  return cudaGetLastError();
}

cudaError_t launch_reduce_current(const double* orb_obs, int nk, int norb, const double* kw,
                                  double inv_omega, int periodic, double* out, cudaStream_t s, int ncell) {
  k_reduce_current<<<ncell, 256, 0, s>>>(orb_obs, nk, norb, kw, inv_omega, periodic, out);
  return cudaGetLastError();
}

// Leapfrog of (1/c^2) A_tt - A_XX = (4 pi / c) I on the interior, first-order Mur at both ends, and
// the cells' A' = A/c along z at t + dt/2 (mean of both levels) and t + dt.
__global__ void k_maxwell(const double* __restrict__ Ap, const double* __restrict__ An, double* __restrict__ Anext,
                          const double* __restrict__ I, int nX, int m0, int ncell, double cdx, double src,
                          double inv_c, double* __restrict__ mid, double* __restrict__ end) {
  for (int X = 1 + threadIdx.x; X < nX - 1; X += blockDim.x)
    Anext[X] = 2.0 * An[X] - Ap[X] + cdx * cdx * (An[X + 1] - 2.0 * An[X] + An[X - 1]) + src * I[X];
  __syncthreads();
  if (threadIdx.x == 0) {
    const double k = (cdx - 1.0) / (cdx + 1.0);
    Anext[0] = An[1] + k * (Anext[1] - An[0]);
    Anext[nX - 1] = An[nX - 2] + k * (Anext[nX - 2] - An[nX - 1]);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
    const int X = m0 + c;
    mid[3 * c] = 0.0; mid[3 * c + 1] = 0.0; mid[3 * c + 2] = 0.5 * (An[X] + Anext[X]) * inv_c;
    end[3 * c] = 0.0; end[3 * c + 1] = 0.0; end[3 * c + 2] = Anext[X] * inv_c;
  }
}

// Longitudinal geometry: d^2 A'_ind / dt^2 = 4 pi J, one leapfrog step per TDKS step from the current
// J(t_n) in step_obs[0..2]; lg = {A_ind^n[3], A_ind^{n-1}[3]} is advanced in place.  The first step
// starts from rest (zero A_ind and zero velocity: A^1 = A^0 + 2 pi dt^2 J).  The A' of the step's
// Taylor stages (mid) and of its end (end) add the external field.
__global__ void k_longitudinal(const double* __restrict__ step_obs, double* __restrict__ lg, int first, double dt,
                               double3 ext_mid, double3 ext_end, double* __restrict__ mid, double* __restrict__ end) {
  const int a = threadIdx.x;
  if (a >= 3) return;
  const double J = step_obs[a];
  const double An = lg[a], Ap = lg[3 + a];
  const double src = 4.0 * kPi * dt * dt * J;
  const double Anext = first ? An + 0.5 * src : 2.0 * An - Ap + src;
  lg[3 + a] = An;
  lg[a] = Anext;
  const double em = a == 0 ? ext_mid.x : (a == 1 ? ext_mid.y : ext_mid.z);
  const double ee = a == 0 ? ext_end.x : (a == 1 ? ext_end.y : ext_end.z);
  mid[a] = em + 0.5 * (An + Anext);
  end[a] = ee + Anext;
}

__global__ void k_ms_current(const double* __restrict__ step_obs, int ncell, int m0, double* __restrict__ I) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x)
    I[m0 + c] = step_obs[(size_t)c * 8 + 2];
}

cudaError_t launch_longitudinal(const double* step_obs, double* lg, int first, double dt, const double ext_mid[3],
                                const double ext_end[3], double* ap_mid, double* ap_end, cudaStream_t s) {
  k_longitudinal<<<1, 32, 0, s>>>(step_obs, lg, first, dt, make_double3(ext_mid[0], ext_mid[1], ext_mid[2]),
                                  make_double3(ext_end[0], ext_end[1], ext_end[2]), ap_mid, ap_end);
  return cudaGetLastError();
}

cudaError_t launch_maxwell(const double* A_prev, const double* A_now, double* A_next, const double* I,
                           int nX, int m0, int ncell, double c_dt_dX, double src, double inv_c,
                           double* ap_mid, double* ap_end, cudaStream_t s) {
  k_maxwell<<<1, 1024, 0, s>>>(A_prev, A_now, A_next, I, nX, m0, ncell, c_dt_dX, src, inv_c, ap_mid, ap_end);
  return cudaGetLastError();
}

cudaError_t launch_ms_current(const double* step_obs, int ncell, int m0, double* I, cudaStream_t s) {
  k_ms_current<<<(ncell + 255) / 256, 256, 0, s>>>(step_obs, ncell, m0, I);
  return cudaGetLastError();
}

cudaError_t launch_fold_density(const float* rho32, int nk, int npts, const float* wsplit, double* rho,
                                cudaStream_t s, int ncell) {
  const long long n = (long long)npts * ncell;
  if (n * kFoldLanes >= (1LL << 31) || n * nk >= (1LL << 31)) return cudaErrorInvalidValue;   // 32-bit indices
  k_fold_density<<<grid_for(n * kFoldLanes, 256), 256, 0, s>>>(rho32, nk, npts, wsplit, rho, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_orbital_dots(const typename Cplx<T>::type* u, const typename Cplx<T>::type* hu,
                                int norb_tot, int npts, double dV, double* out, cudaStream_t s) {
  k_orbital_dots<<<norb_tot, 256, 0, s>>>(u, hu, npts, dV, out);
  return cudaGetLastError();
}
template cudaError_t launch_orbital_dots<float>(const float2*, const float2*, int, int, double, double*, cudaStream_t);
template cudaError_t launch_orbital_dots<double>(const double2*, const double2*, int, int, double, double*, cudaStream_t);

}  // namespace tdks
