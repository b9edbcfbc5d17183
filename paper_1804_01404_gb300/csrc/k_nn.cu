// Learned potential predictor: a 3-layer 3D convolutional network (4 -> 16 -> 16 -> 1 channels,
// 3^3 kernels, SiLU) that predicts the Hartree-exchange potential of the next step from the last
// four, replacing the predictor half-step of the predictor-corrector scheme (Program summary).
//
// Storage: activations and weights that feed a convolution are BF16 values (weights are kept as
// FP32 masters and read through their BF16 rounding); every product is accumulated in FP32.
// Training is plain backpropagation with Adam; the weight gradient is reduced over grid points by
// per-block partials summed in a fixed order, so a training run is deterministic.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "grid_sum.cuh"
#include "pdl.cuh"
#include "tdks_internal.h"

namespace tdks {

namespace {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ int nb_index(const NNGrid& g, int x, int y, int z, int dx, int dy, int dz) {
  int xx = x + dx, yy = y + dy, zz = z + dz;
  if (g.periodic) {
    xx += (xx < 0) ? g.nx : 0; xx -= (xx >= g.nx) ? g.nx : 0;
    yy += (yy < 0) ? g.ny : 0; yy -= (yy >= g.ny) ? g.ny : 0;
    zz += (zz < 0) ? g.nz : 0; zz -= (zz >= g.nz) ? g.nz : 0;
  } else if (xx < 0 || xx >= g.nx || yy < 0 || yy >= g.ny || zz < 0 || zz >= g.nz) {
    return -1;
  }
  return (zz * g.ny + yy) * g.nx + xx;
}

__device__ __forceinline__ void coords(const NNGrid& g, int p, int& x, int& y, int& z) {
  x = p % g.nx;
  const int r = p / g.nx;
  y = r % g.ny;
  z = r / g.ny;
}

__device__ __forceinline__ float silu(float y) { return y / (1.0f + expf(-y)); }
__device__ __forceinline__ float dsilu(float y) {
  const float s = 1.0f / (1.0f + expf(-y));
  return s * (1.0f + y * (1.0f - s));
}

__device__ __forceinline__ double cubic(double v0, double v1, double v2, double v3) {
  return 4.0 * v0 - 6.0 * v1 + 4.0 * v2 - v3;
}

// N consecutive BF16 values (N = 4 or a multiple of 8, address aligned to 2N bytes) as floats.
template <int N>
__device__ __forceinline__ void load_bf16(const bf16* p, float* out) {
  static_assert(N == 4 || N % 8 == 0, "vector width");
  if constexpr (N == 4) {
    const uint2 r = *reinterpret_cast<const uint2*>(p);
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&r.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&r.y));
    out[0] = a.x; out[1] = a.y; out[2] = b.x; out[3] = b.y;
  } else {
#pragma unroll
    for (int v = 0; v < N / 8; ++v) {
      const uint4 r = reinterpret_cast<const uint4*>(p)[v];
      const unsigned w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[j]));
        out[8 * v + 2 * j] = f.x;
        out[8 * v + 2 * j + 1] = f.y;
      }
    }
  }
}

// y[co][p] = b[co] + sum_{kk, ci} W[co][ci][kk] x[ci][nb(p, kk)];  a = bf16(SiLU(y)) if ACT.
// Each point is shared by G = (COUT / COP) * CIS adjacent lanes: a lane forms COP outputs over
// CIN / CIS input channels, and lanes that split the input channels add their sums by shuffles.
// (A point per thread would leave most SMs idle on the grids of these cells.)
// Layouts: channel-first x[ci][p], y[co][p], a[co][p] (training), or, with CL, channel-last
// x[p][ci] and a[p][co] read and written with vector accesses, y not stored (prediction only).
// PRED (COUT = 1): also vpred[p] = cubic(V0..V3)[p] + s3 * y[p], the network's potential prediction.
template <int CIN, int COUT, bool ACT, int COP, int CIS, bool PRED = false, bool CL = false>
__global__ void __launch_bounds__(256) k_nn_fwd(NNGrid g, const bf16* __restrict__ x,
                                                const float* __restrict__ W, const float* __restrict__ b,
                                                float* __restrict__ y, bf16* __restrict__ a,
                                                NNPredict pr = NNPredict{}, const double* __restrict__ stats = nullptr) {
  static_assert(!PRED || COUT == 1, "the prediction epilogue follows the single-channel layer");
  constexpr int GO = COUT / COP, G = GO * CIS, CIP = CIN / CIS;
  static_assert(GO * COP == COUT && CIP * CIS == CIN && 32 % G == 0, "lane split");
  __shared__ float Ws[27][CIN][COUT];
  for (int i = threadIdx.x; i < COUT * CIN * 27; i += blockDim.x) {
    const int co = i / (CIN * 27), r = i % (CIN * 27), ci = r / 27, kk = r % 27;
    Ws[kk][ci][co] = W[i];
  }
  __syncthreads();
  const long long total = (long long)g.npts * G;
  for (long long t0 = (long long)blockIdx.x * blockDim.x; t0 < total; t0 += (long long)gridDim.x * blockDim.x) {
    const long long t = t0 + threadIdx.x;           // every lane of the warp runs the iteration
    const bool act = t < total;
    const int p = act ? (int)(t / G) : 0;
    const int gi = (int)(t % G);
    const int og = gi % GO, cs = gi / GO;           // output group, input-channel split
    int px, py, pz;
    coords(g, p, px, py, pz);
    float acc[COP];
#pragma unroll
    for (int o = 0; o < COP; ++o) acc[o] = (cs == 0) ? b[og * COP + o] : 0.f;
    for (int kk = 0; kk < 27; ++kk) {
      const int q = act ? nb_index(g, px, py, pz, kk % 3 - 1, (kk / 3) % 3 - 1, kk / 9 - 1) : -1;
      if (q < 0) continue;
      if constexpr (CL) {
        float xv[CIP];
        load_bf16<CIP>(x + (size_t)q * CIN + cs * CIP, xv);
#pragma unroll
        for (int c = 0; c < CIP; ++c)
#pragma unroll
          for (int o = 0; o < COP; ++o) acc[o] = fmaf(Ws[kk][cs * CIP + c][og * COP + o], xv[c], acc[o]);
      } else {
#pragma unroll
        for (int c = 0; c < CIP; ++c) {
          const int ci = cs * CIP + c;
          const float xv = __bfloat162float(x[(size_t)ci * g.npts + q]);
#pragma unroll
          for (int o = 0; o < COP; ++o) acc[o] = fmaf(Ws[kk][ci][og * COP + o], xv, acc[o]);
        }
      }
    }
    if (CIS > 1) {
#pragma unroll
      for (int sft = GO; sft < G; sft <<= 1)
#pragma unroll
        for (int o = 0; o < COP; ++o) acc[o] += __shfl_xor_sync(0xffffffffu, acc[o], sft);
    }
    if (act && cs == 0) {
      if constexpr (CL && ACT && COP == 4) {
        const __nv_bfloat162 lo = __floats2bfloat162_rn(silu(acc[0]), silu(acc[1]));
        const __nv_bfloat162 hi = __floats2bfloat162_rn(silu(acc[2]), silu(acc[3]));
        uint2 r;
        r.x = *reinterpret_cast<const unsigned*>(&lo);
        r.y = *reinterpret_cast<const unsigned*>(&hi);
        *reinterpret_cast<uint2*>(a + (size_t)p * COUT + og * COP) = r;
      } else {
        static_assert(!CL || !ACT || COP == 4, "channel-last activations are stored four at a time");
#pragma unroll
        for (int o = 0; o < COP; ++o) {
          const int co = og * COP + o;
          if (!CL) y[(size_t)co * g.npts + p] = acc[o];
          if (ACT) a[(size_t)co * g.npts + p] = __float2bfloat16(silu(acc[o]));
        }
      }
      if (PRED) pr.vpred[p] = cubic(pr.V0[p], pr.V1[p], pr.V2[p], pr.V3[p]) + stats[2] * (double)acc[0];
    }
  }
}

// dyprev[ci][q] = SiLU'(yprev[ci][q]) * sum_{kk, co} W[co][ci][kk] dy[co][p],  nb(p, kk) = q
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) k_nn_bwd_data(NNGrid g, const float* __restrict__ dy,
                                                     const float* __restrict__ W,
                                                     const float* __restrict__ yprev,
                                                     float* __restrict__ dyprev) {
  __shared__ float Ws[27][COUT][CIN];
  for (int i = threadIdx.x; i < COUT * CIN * 27; i += blockDim.x) {
    const int co = i / (CIN * 27), r = i % (CIN * 27), ci = r / 27, kk = r % 27;
    Ws[kk][co][ci] = W[i];
  }
  __syncthreads();
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < g.npts; q += gridDim.x * blockDim.x) {
    int qx, qy, qz;
    coords(g, q, qx, qy, qz);
    float acc[CIN];
#pragma unroll
    for (int ci = 0; ci < CIN; ++ci) acc[ci] = 0.0f;
    for (int kk = 0; kk < 27; ++kk) {
      const int p = nb_index(g, qx, qy, qz, -(kk % 3 - 1), -((kk / 3) % 3 - 1), -(kk / 9 - 1));
      if (p < 0) continue;
#pragma unroll
      for (int co = 0; co < COUT; ++co) {
        const float d = dy[(size_t)co * g.npts + p];
#pragma unroll
        for (int ci = 0; ci < CIN; ++ci) acc[ci] = fmaf(Ws[kk][co][ci], d, acc[ci]);
      }
    }
#pragma unroll
    for (int ci = 0; ci < CIN; ++ci)
      dyprev[(size_t)ci * g.npts + q] = acc[ci] * dsilu(yprev[(size_t)ci * g.npts + q]);
  }
}

constexpr int PB = 128;   // grid points per weight-gradient block

// part[blk][w]: w < COUT*CIN*27 -> sum_p dy[co][p] x[ci][nb(p, kk)], else bias: sum_p dy[co][p]
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) k_nn_bwd_weight(NNGrid g, const float* __restrict__ dy,
                                                       const bf16* __restrict__ x,
                                                       float* __restrict__ part) {
  __shared__ float dys[COUT][PB];
  __shared__ int nbs[27][PB];
  constexpr int NW = COUT * CIN * 27 + COUT;
  const int p0 = blockIdx.x * PB;
  const int np = min(PB, g.npts - p0);
  for (int i = threadIdx.x; i < COUT * PB; i += blockDim.x) {
    const int co = i / PB, j = i % PB;
    dys[co][j] = (j < np) ? dy[(size_t)co * g.npts + p0 + j] : 0.0f;
  }
  for (int i = threadIdx.x; i < 27 * PB; i += blockDim.x) {
    const int kk = i / PB, j = i % PB;
    int q = -1;
    if (j < np) {
      int px, py, pz;
      coords(g, p0 + j, px, py, pz);
      q = nb_index(g, px, py, pz, kk % 3 - 1, (kk / 3) % 3 - 1, kk / 9 - 1);
    }
    nbs[kk][j] = q;
  }
  __syncthreads();
  for (int w = threadIdx.x; w < NW; w += blockDim.x) {
    float acc = 0.0f;
    if (w < COUT * CIN * 27) {
      const int co = w / (CIN * 27), r = w % (CIN * 27), ci = r / 27, kk = r % 27;
      const bf16* xc = x + (size_t)ci * g.npts;
      for (int j = 0; j < np; ++j) {
        const int q = nbs[kk][j];
        if (q >= 0) acc = fmaf(dys[co][j], __bfloat162float(xc[q]), acc);
      }
    } else {
      const int co = w - COUT * CIN * 27;
      for (int j = 0; j < np; ++j) acc += dys[co][j];
    }
    part[(size_t)blockIdx.x * NW + w] = acc;
  }
}

// grad[w] += sum_blk part[blk][w]   (fixed order)
__global__ void k_nn_reduce(const float* __restrict__ part, int nblk, int nw, float* __restrict__ grad) {
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += gridDim.x * blockDim.x) {
    float acc = 0.0f;
    for (int b = 0; b < nblk; ++b) acc += part[(size_t)b * nw + w];
    grad[w] += acc;
  }
}

// dout = 2 (out - t) / n; loss partial sums per block, then added to *loss in fixed order
__global__ void __launch_bounds__(256) k_nn_loss(const float* __restrict__ out, const float* __restrict__ t,
                                                 int n, float* __restrict__ dout, double* loss) {
  __shared__ double red[256];
  float acc = 0.0f;
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    const float d = out[p] - t[p];
    dout[p] = 2.0f * d / (float)n;
    acc += d * d;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss += red[0] / n;
}

// Adam on FP32 masters; wq = parameters rounded through BF16 (what the convolutions read)
__global__ void k_nn_adam(float* __restrict__ p, float* __restrict__ g, float* __restrict__ m,
                          float* __restrict__ v, float* __restrict__ wq, int n, float lr, float b1,
                          float b2, float eps, float c1, float c2, float gscale) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i] * gscale;
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    wq[i] = __bfloat162float(__float2bfloat16(pi));
    g[i] = 0.0f;
  }
}

__global__ void k_nn_round(const float* __restrict__ p, float* __restrict__ wq, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    wq[i] = __bfloat162float(__float2bfloat16(p[i]));
}

// Differences D1 = V0 - V1, D2 = V0 - 2 V1 + V2, D3 = V0 - 3 V1 + 3 V2 - V3 (formed in FP64).
// stats = {s1, s2, s3, mean V0, s_V}: root mean squares of D1, D2, D3 and V0 - mean V0, each
// floored at 1e-13 rms(V0); summed over all CTAs by grid_sum.
__global__ void __launch_bounds__(256) k_nn_stats(const double* __restrict__ V0, const double* __restrict__ V1,
                                                  const double* __restrict__ V2, const double* __restrict__ V3,
                                                  int n, double* partials, unsigned* ticket, double* stats) {
  __shared__ double tot[5];
  double acc[5] = {0, 0, 0, 0, 0};
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const double v0 = V0[p], v1 = V1[p], v2 = V2[p], v3 = V3[p];
    const double d1 = v0 - v1, d2 = d1 - (v1 - v2), d3 = d2 - ((v1 - v2) - (v2 - v3));
    acc[0] += d1 * d1; acc[1] += d2 * d2; acc[2] += d3 * d3; acc[3] += v0; acc[4] += v0 * v0;
  }
  if (!grid_sum<5>(acc, partials, ticket, tot)) return;
  if (threadIdx.x == 0) {
    const double mean = tot[3] / n;
    const double fl = 1e-13 * sqrt(tot[4] / n) + 1e-300;
    stats[0] = fmax(sqrt(tot[0] / n), fl);
    stats[1] = fmax(sqrt(tot[1] / n), fl);
    stats[2] = fmax(sqrt(tot[2] / n), fl);
    stats[3] = mean;
    stats[4] = fmax(sqrt(fmax(tot[4] / n - mean * mean, 0.0)), fl);
  }
}

// Network inputs x[c][p] (channel-first) or x[p][c] (cl = 1), c = scaled D1, D2, D3, V0 - mean.
__global__ void k_nn_pack(const double* __restrict__ V0, const double* __restrict__ V1,
                          const double* __restrict__ V2, const double* __restrict__ V3,
                          const double* __restrict__ Vnext, const double* __restrict__ stats, int n,
                          int cl, bf16* __restrict__ x, float* __restrict__ target) {
  const double s1 = stats[0], s2 = stats[1], s3 = stats[2], m = stats[3], sv = stats[4];
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const double d1 = V0[p] - V1[p], d2 = V0[p] - 2.0 * V1[p] + V2[p];
    const double d3 = V0[p] - 3.0 * V1[p] + 3.0 * V2[p] - V3[p];
    const bf16 c0 = __float2bfloat16((float)(d1 / s1)), c1 = __float2bfloat16((float)(d2 / s2));
    const bf16 c2 = __float2bfloat16((float)(d3 / s3)), c3 = __float2bfloat16((float)((V0[p] - m) / sv));
    if (cl) {
      x[4 * (size_t)p] = c0; x[4 * (size_t)p + 1] = c1; x[4 * (size_t)p + 2] = c2; x[4 * (size_t)p + 3] = c3;
    } else {
      x[p] = c0; x[(size_t)n + p] = c1; x[2 * (size_t)n + p] = c2; x[3 * (size_t)n + p] = c3;
    }
    if (Vnext) target[p] = (float)((Vnext[p] - cubic(V0[p], V1[p], V2[p], V3[p])) / s3);
  }
}

// mode 0: V~ = 2 V0 - V1;  1: cubic 4 V0 - 6 V1 + 4 V2 - V3;  2: cubic + s3 * out
__global__ void k_nn_apply(const double* __restrict__ V0, const double* __restrict__ V1,
                           const double* __restrict__ V2, const double* __restrict__ V3,
                           const float* __restrict__ out, const double* __restrict__ stats, int n,
                           int mode, double* __restrict__ vpred) {
  const double s3 = (mode == 2) ? stats[2] : 0.0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    double v;
    if (mode == 0) v = 2.0 * V0[p] - V1[p];
    else v = cubic(V0[p], V1[p], V2[p], V3[p]) + (mode == 2 ? s3 * (double)out[p] : 0.0);
    vpred[p] = v;
  }
}

// res = ||Vnew - Vpred||_2 / ||Vnew||_2, summed over all CTAs by grid_sum
__global__ void __launch_bounds__(256) k_residual(const double* __restrict__ Vnew, const double* __restrict__ Vpred,
                                                  int n, double* partials, unsigned* ticket, double* res) {
  pdl_trigger();
  pdl_wait();
  __shared__ double tot[2];
  double acc[2] = {0, 0};
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const double d = Vnew[p] - Vpred[p], v = Vnew[p];
    acc[0] += d * d;
    acc[1] += v * v;
  }
  if (!grid_sum<2>(acc, partials, ticket, tot)) return;
  if (threadIdx.x == 0) *res = sqrt(tot[0] / fmax(tot[1], 1e-300));
}

// Accept or reject a predicted potential on the device: every thread reads the misfit the residual
// kernel left, and if it is finite and within the threshold copies V_Hxc(t+dt) of the predicted step
// into the step potential; thread 0 of block 0 otherwise counts a fallback and sets the graph's
// conditional handle, which runs the conditional body (the restore and the plain predictor-corrector
// step).  One thread sets the handle, so there are no racing calls.
__global__ void __launch_bounds__(256) k_decide(const double* __restrict__ res, double thr,
                                                const double* __restrict__ vnew, double* __restrict__ vhxc,
                                                double* __restrict__ vnext, int n, double* fb,
                                                cudaGraphConditionalHandle handle) {
  const double r = *res;
  const bool ok = (r <= thr) && (r == r) && (r < 1e300);   // finite and within the threshold
  if (ok)
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
      const double v = vnew[p];
      vhxc[p] = v;
      vnext[p] = v;
    }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (!ok) *fb += 1.0;
    cudaGraphSetConditional(handle, ok ? 0u : 1u);
  }
}

__global__ void k_store6(double* dst, double a0, double a1, double a2, double a3, double a4, double a5) {
  if (threadIdx.x == 0) {
    dst[0] = a0; dst[1] = a1; dst[2] = a2; dst[3] = a3; dst[4] = a4; dst[5] = a5;
  }
}

// ---------------------------------------------------------------------------------------------
// The whole prediction in one cooperative launch: statistics, input packing and the three layers are
// phases separated by grid barriers (every CTA is resident, so a CTA waits only for the others to
// finish the phase before).  Layer 2 (16 -> 16 channels, the bulk of the work) is an implicit GEMM on
// the tensor cores: a warp takes 16 grid points, and for each of the 27 taps multiplies the 16 x 16
// BF16 matrix of its points' neighbour activations by the tap's 16 x 16 BF16 weight matrix with
// mma.sync (m16n8k16, two n-halves), accumulating in FP32.  Layers 1 and 3 (4 -> 16 and 16 -> 1) are
// small and run on the CUDA cores.  Arithmetic per value is that of k_nn_stats, k_nn_pack and k_nn_fwd.
// ---------------------------------------------------------------------------------------------
constexpr int kFusedThreads = 256;
constexpr int kFusedMaxBlocks = 304;   // partials of the statistics: [304][5]

struct FusedArgs {
  NNGrid g;
  const double *V0, *V1, *V2, *V3;
  double* vpred;
  const double *vloc, *vhxc; // optional: the corrector's step potential from V~ (see NNPredict)
  double* vstep64;
  float* vstep32;
  const uint4* wpack;        // FusedWeights image of the BF16-rounded parameters
  bf16 *x0, *a1, *a2;        // channel-last [npts][4], [npts][16], [npts][16]
  double* stats;             // out: s1, s2, s3, mean V0, s_V
  double* part;              // [gridDim.x][5]
  double inv_n;              // 1 / points
  unsigned* bar;             // [2] grid-barrier counter and exit counter, zero at launch (the kernel resets them)
  int* err;                  // TDKS_ETIMEOUT if a barrier wait gives up
  long long limit;           // polls per barrier wait
};

// Grid barrier number k (targets k * gridDim.x arrivals) with a bounded wait: false (and *err set) if
// the other CTAs did not all arrive within the poll limit.
__device__ __forceinline__ bool fused_barrier(const FusedArgs& A, unsigned k, int* ok_s) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(A.bar, 1u);
    const unsigned target = k * gridDim.x;
    long long it = 0;
    unsigned v = *(volatile unsigned*)A.bar;
    while (v < target && ++it < A.limit) v = *(volatile unsigned*)A.bar;
    __threadfence();
    *ok_s = v >= target;
    if (!*ok_s) atomicExch(A.err, 4);            // TDKS_ETIMEOUT
  }
  __syncthreads();
  return *ok_s != 0;
}

__device__ __forceinline__ unsigned pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const unsigned*>(&v);
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Neighbour indices of the 27 taps (the layer loops are fully unrolled so that every neighbour's load
// is issued before the arithmetic that uses it; these layers are bound by load latency).
// Built from the three wrapped (or, outside an isolated box, invalid) coordinates per axis; an invalid
// coordinate contributes a large negative offset, so every neighbour it touches gets q < 0.
__device__ __forceinline__ void tap_index(const NNGrid& g, int x, int y, int z, bool valid, int (&q)[27]) {
  constexpr int kOut = -(1 << 29);
  int xo[3], yo[3], zo[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    int xx = x + d - 1, yy = y + d - 1, zz = z + d - 1;
    if (g.periodic) {
      xx += (xx < 0) ? g.nx : 0; xx -= (xx >= g.nx) ? g.nx : 0;
      yy += (yy < 0) ? g.ny : 0; yy -= (yy >= g.ny) ? g.ny : 0;
      zz += (zz < 0) ? g.nz : 0; zz -= (zz >= g.nz) ? g.nz : 0;
    }
    xo[d] = (xx >= 0 && xx < g.nx) ? xx : kOut;
    yo[d] = (yy >= 0 && yy < g.ny) ? yy * g.nx : kOut;
    zo[d] = (zz >= 0 && zz < g.nz) ? zz * g.nx * g.ny : kOut;
  }
#pragma unroll
  for (int kk = 0; kk < 27; ++kk) {
    const int v = zo[kk / 9] + yo[(kk / 3) % 3] + xo[kk % 3];
    q[kk] = (valid && v >= 0) ? v : -1;
  }
}

// sqrt(a) and 1 / sqrt(a) of a normal, positive a to FP64 accuracy without the FP64 square-root and
// division sequences (slow on this GPU): an FP32 reciprocal square root refined by two Newton steps
// y <- y (3 - a y^2) / 2, whose error squares at each step (about 1e-7, 1e-14, 1e-28).  Arguments
// outside the FP32 range take the exact route.
__device__ __forceinline__ void sqrt_and_rsqrt(double a, double& s, double& r) {
  if (a > 1e-30 && a < 1e30) {
    double y = (double)rsqrtf((float)a);
    y = y * (1.5 - 0.5 * a * y * y);
    y = y * (1.5 - 0.5 * a * y * y);
    r = y;
    s = a * y;
  } else {
    s = sqrt(a);
    r = 1.0 / s;
  }
}

// The weights as the prediction kernel holds them in shared memory, laid out once per parameter update
// (k_nn_pack_weights) so that every CTA copies them with a few 16-byte loads per thread.
struct alignas(16) FusedWeights {
  float W1s[27][4][16];
  float W3s[27][16];
  float b1s[16], b2s[16];
  float b3s[4];
  uint2 Bf[27][2][32];      // layer-2 weights as mma B fragments [tap][n-half][lane]
};
static_assert(sizeof(FusedWeights) % 16 == 0, "copied as uint4");
constexpr int kFusedWeightVecs = sizeof(FusedWeights) / 16;

static_assert(kNNOff[1] == 1728 && kNNOff[2] == 1744 && kNNOff[3] == 8656 && kNNOff[4] == 8672 && kNNOff[5] == 9104,
              "parameter offsets used by k_nn_pack_weights");
__global__ void k_nn_pack_weights(const float* __restrict__ wq, FusedWeights* __restrict__ out) {
  const float* W1 = wq + 0;
  const float* W2 = wq + 1744;
  const float* W3 = wq + 8672;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 16 * 4 * 27; i += gridDim.x * blockDim.x) {
    const int co = i / (4 * 27), r = i % (4 * 27), ci = r / 27, kk = r % 27;
    out->W1s[kk][ci][co] = W1[i];
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 16 * 27; i += gridDim.x * blockDim.x)
    out->W3s[i % 27][i / 27] = W3[i];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 16; i += gridDim.x * blockDim.x) {
    out->b1s[i] = wq[1728 + i];
    out->b2s[i] = wq[8656 + i];
    if (i < 4) out->b3s[i] = (i == 0) ? wq[9104] : 0.f;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 27 * 2 * 32; i += gridDim.x * blockDim.x) {
    const int kk = i / 64, h = (i / 32) % 2, l = i % 32;
    const int n = 8 * h + (l >> 2), k0 = 2 * (l & 3);
    auto w = [&](int ci) { return W2[(n * 16 + ci) * 27 + kk]; };
    out->Bf[kk][h][l] = make_uint2(pack_bf16x2(w(k0), w(k0 + 1)), pack_bf16x2(w(k0 + 8), w(k0 + 9)));
  }
}

__global__ void __launch_bounds__(kFusedThreads, 1) k_nn_predict(FusedArgs A) {
  __shared__ FusedWeights Ws;
  float (&W1s)[27][4][16] = Ws.W1s;
  float (&W3s)[27][16] = Ws.W3s;
  float (&b1s)[16] = Ws.b1s;
  float (&b2s)[16] = Ws.b2s;
  uint2 (&Bf)[27][2][32] = Ws.Bf;
  __shared__ double st[5];
  __shared__ int ok_s;
  const NNGrid& g = A.g;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long nthr = (long long)gridDim.x * blockDim.x;
  const long long gtid = (long long)blockIdx.x * blockDim.x + tid;
  // weights (read through their BF16 rounding, as stored): the packed image, all loads in flight at once
  {
    constexpr int PER = (kFusedWeightVecs + kFusedThreads - 1) / kFusedThreads;
    uint4 tmp[PER];
    uint4* dst = reinterpret_cast<uint4*>(&Ws);
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int i = tid + j * kFusedThreads;
      if (i < kFusedWeightVecs) tmp[j] = __ldg(A.wpack + i);
    }
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int i = tid + j * kFusedThreads;
      if (i < kFusedWeightVecs) dst[i] = tmp[j];
    }
  }
  __syncthreads();
  const float b3s = Ws.b3s[0];

  // phase 1: statistics of the backward differences (FP64), per-CTA partials
  {
    double acc[5] = {0, 0, 0, 0, 0};
    for (long long p = gtid; p < g.npts; p += nthr) {
      const double v0 = A.V0[p], v1 = A.V1[p], v2 = A.V2[p], v3 = A.V3[p];
      const double d1 = v0 - v1, d2 = d1 - (v1 - v2), d3 = d2 - ((v1 - v2) - (v2 - v3));
      acc[0] += d1 * d1; acc[1] += d2 * d2; acc[2] += d3 * d3; acc[3] += v0; acc[4] += v0 * v0;
    }
    // the CTA's sums: warp j takes value j of all threads (eight adds per lane, then a shuffle
    // tree), 13 FP64 additions in a warp's chain instead of 25 shuffle steps plus 8 (one warp's FP64
    // instructions do not overlap on this GPU)
    __shared__ double rs[5][kFusedThreads];
#pragma unroll
    for (int j = 0; j < 5; ++j) rs[j][tid] = acc[j];
    __syncthreads();
    if (warp < 5) {
      double x = 0;
#pragma unroll
      for (int i = 0; i < kFusedThreads / 32; ++i) x += rs[warp][lane + 32 * i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) A.part[(size_t)blockIdx.x * 5 + warp] = x;
    }
  }
  if (!fused_barrier(A, 1, &ok_s)) return;
  if (warp < 5) {       // totals in a fixed order: lane l sums CTAs l, l + 32, ..., then a shuffle tree
    double xs[kFusedMaxBlocks / 32 + 1];
#pragma unroll
    for (int j = 0; j <= kFusedMaxBlocks / 32; ++j) {   // every load in flight at once
      const unsigned b = lane + 32u * j;
      xs[j] = b < gridDim.x ? __ldcg(&A.part[(size_t)b * 5 + warp]) : 0.0;
    }
    double x = 0;
    const int nb32 = (int)((gridDim.x + 31) >> 5);   // only the words that hold partials
#pragma unroll
    for (int j = 0; j <= kFusedMaxBlocks / 32; ++j) {
      if (j >= nb32) break;
      x += xs[j];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) st[warp] = x;
  }
  __syncthreads();
  // the four scales s_j = max(rms_j, floor) and their reciprocals, one thread each (an FP32 seed and
  // Newton steps; FP64 square roots and divisions are slow on this GPU)
  __shared__ double sc[9];
  if (tid < 4) {
    const double mean = st[3] * A.inv_n;
    // rms(V0) only sets the floor of the scales: FP32 is enough (and off the FP64 pipe)
    const double s0 = (double)sqrtf((float)fmin(st[4] * A.inv_n, 1e30));
    const double fl = 1e-13 * s0 + 1e-300;
    const double a = (tid < 3) ? st[tid] * A.inv_n : fmax(st[4] * A.inv_n - mean * mean, 0.0);
    double sj = 0.0, rj = 0.0;
    if (a > 0.0) sqrt_and_rsqrt(a, sj, rj);
    if (!(sj >= fl)) { sj = fl; rj = 1.0 / fl; }                    // floored (degenerate history)
    sc[2 * tid] = sj;
    sc[2 * tid + 1] = rj;
    if (tid == 0) sc[8] = mean;
  }
  __syncthreads();
  const double r1 = sc[1], r2 = sc[3], r3 = sc[5], rv = sc[7], s3 = sc[4], mean = sc[8];
  if (blockIdx.x == 0 && tid == 0) {
    A.stats[0] = sc[0]; A.stats[1] = sc[2]; A.stats[2] = sc[4]; A.stats[3] = mean; A.stats[4] = sc[6];
  }
  // phase 2: the four input channels of every point (BF16, channel-last)
  for (long long p = gtid; p < g.npts; p += nthr) {
    const double v0 = A.V0[p], v1 = A.V1[p], v2 = A.V2[p], v3 = A.V3[p];
    const double d1 = v0 - v1, d2 = v0 - 2.0 * v1 + v2, d3 = v0 - 3.0 * v1 + 3.0 * v2 - v3;
    uint2 r;
    r.x = *reinterpret_cast<const unsigned*>(&(const __nv_bfloat162&)make_bfloat162(
        __float2bfloat16((float)(d1 * r1)), __float2bfloat16((float)(d2 * r2))));
    r.y = *reinterpret_cast<const unsigned*>(&(const __nv_bfloat162&)make_bfloat162(
        __float2bfloat16((float)(d3 * r3)), __float2bfloat16((float)((v0 - mean) * rv))));
    *reinterpret_cast<uint2*>(A.x0 + 4 * p) = r;
  }
  if (!fused_barrier(A, 2, &ok_s)) return;
  // phase 3: layer 1 (4 -> 16), four lanes per point, four outputs each
  for (long long t = gtid; t < 4LL * g.npts; t += nthr) {
    const int p = (int)(t >> 2), og = (int)(t & 3);
    int px, py, pz;
    coords(g, p, px, py, pz);
    int q[27];
    tap_index(g, px, py, pz, true, q);
    uint2 raw[27];
#pragma unroll
    for (int kk = 0; kk < 27; ++kk)
      raw[kk] = q[kk] >= 0 ? *reinterpret_cast<const uint2*>(A.x0 + 4 * (size_t)q[kk]) : make_uint2(0u, 0u);
    float acc[4];
#pragma unroll
    for (int o = 0; o < 4; ++o) acc[o] = b1s[og * 4 + o];
#pragma unroll
    for (int kk = 0; kk < 27; ++kk) {
      const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&raw[kk].x));
      const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&raw[kk].y));
      const float xv[4] = {lo.x, lo.y, hi.x, hi.y};
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int o = 0; o < 4; ++o) acc[o] = fmaf(W1s[kk][c][og * 4 + o], xv[c], acc[o]);
    }
    uint2 r;
    r.x = pack_bf16x2(silu(acc[0]), silu(acc[1]));
    r.y = pack_bf16x2(silu(acc[2]), silu(acc[3]));
    *reinterpret_cast<uint2*>(A.a1 + 16 * (size_t)p + 4 * og) = r;
  }
  if (!fused_barrier(A, 3, &ok_s)) return;
  // phase 4: layer 2 (16 -> 16) on the tensor cores: a warp task is 16 points and one half (8) of the
  // output channels, so that the tasks cover every warp of the grid
  {
    const int grp = lane >> 2, tq = lane & 3;
    const int ntask = 2 * ((g.npts + 15) / 16);
    const int nwarp = gridDim.x * (blockDim.x / 32);
    const unsigned* a1w = reinterpret_cast<const unsigned*>(A.a1);   // 8 words per point
    unsigned* a2w = reinterpret_cast<unsigned*>(A.a2);
    for (int task = blockIdx.x * (blockDim.x / 32) + warp; task < ntask; task += nwarp) {
      const int tile = task >> 1, h = task & 1;
      const int r0 = tile * 16 + grp, r1 = r0 + 8;
      const bool v0ok = r0 < g.npts, v1ok = r1 < g.npts;
      int x0, y0, z0, x1, y1, z1;
      coords(g, v0ok ? r0 : 0, x0, y0, z0);
      coords(g, v1ok ? r1 : 0, x1, y1, z1);
      float d[4] = {0, 0, 0, 0};
      int q0[27], q1[27];
      tap_index(g, x0, y0, z0, v0ok, q0);
      tap_index(g, x1, y1, z1, v1ok, q1);
      unsigned a[27][4];                      // every tap's words loaded before the 27 MMAs
#pragma unroll
      for (int kk = 0; kk < 27; ++kk) {
        a[kk][0] = q0[kk] >= 0 ? a1w[8 * (size_t)q0[kk] + tq] : 0u;
        a[kk][1] = q1[kk] >= 0 ? a1w[8 * (size_t)q1[kk] + tq] : 0u;
        a[kk][2] = q0[kk] >= 0 ? a1w[8 * (size_t)q0[kk] + tq + 4] : 0u;
        a[kk][3] = q1[kk] >= 0 ? a1w[8 * (size_t)q1[kk] + tq + 4] : 0u;
      }
#pragma unroll
      for (int kk = 0; kk < 27; ++kk) {
        const uint2 b = Bf[kk][h][lane];
        mma_bf16_16816(d, a[kk], b.x, b.y);
      }
      const int c0 = 8 * h + 2 * tq;
      if (v0ok) a2w[8 * (size_t)r0 + 4 * h + tq] = pack_bf16x2(silu(d[0] + b2s[c0]), silu(d[1] + b2s[c0 + 1]));
      if (v1ok) a2w[8 * (size_t)r1 + 4 * h + tq] = pack_bf16x2(silu(d[2] + b2s[c0]), silu(d[3] + b2s[c0 + 1]));
    }
  }
  if (!fused_barrier(A, 4, &ok_s)) return;
  // every CTA is past the last barrier (none polls the counter any more): the last CTA to get here
  // resets both counters for the next launch
  if (tid == 0 && atomicAdd(A.bar + 1, 1u) == gridDim.x - 1) {
    atomicExch(A.bar, 0u);
    atomicExch(A.bar + 1, 0u);
  }
  // phase 5: layer 3 (16 -> 1), four lanes per point splitting the channels, and the prediction
  for (long long t0 = (long long)blockIdx.x * blockDim.x; t0 < 4LL * g.npts; t0 += nthr) {
    const long long t = t0 + tid;                  // every lane of the warp takes part in the shuffles
    const bool act = t < 4LL * g.npts;
    const int p = act ? (int)(t >> 2) : 0, cs = (int)(t & 3);
    int px, py, pz;
    coords(g, p, px, py, pz);
    int q[27];
    tap_index(g, px, py, pz, act, q);
    uint2 raw[27];
#pragma unroll
    for (int kk = 0; kk < 27; ++kk)
      raw[kk] = q[kk] >= 0 ? *reinterpret_cast<const uint2*>(A.a2 + 16 * (size_t)q[kk] + 4 * cs) : make_uint2(0u, 0u);
    float acc = (cs == 0) ? b3s : 0.f;
#pragma unroll
    for (int kk = 0; kk < 27; ++kk) {
      const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&raw[kk].x));
      const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&raw[kk].y));
      acc = fmaf(W3s[kk][4 * cs], lo.x, acc);
      acc = fmaf(W3s[kk][4 * cs + 1], lo.y, acc);
      acc = fmaf(W3s[kk][4 * cs + 2], hi.x, acc);
      acc = fmaf(W3s[kk][4 * cs + 3], hi.y, acc);
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    if (act && cs == 0) {
      const double vp = cubic(A.V0[p], A.V1[p], A.V2[p], A.V3[p]) + s3 * (double)acc;
      A.vpred[p] = vp;
      if (A.vstep64) {                             // V_loc + (V_Hxc(t) + V~)/2, as k_combine forms it
        double v = A.vloc[p];
        v += 0.5 * A.vhxc[p];
        v += 0.5 * vp;
        A.vstep64[p] = v;
        if (A.vstep32) A.vstep32[p] = (float)v;
      }
    }
  }
}

int blocks_for(int n) {
  int b = (n + 255) / 256;
  return b > 152 * 8 ? 152 * 8 : (b < 1 ? 1 : b);
}

}  // namespace

int nn_part_blocks(int npts) { return (npts + PB - 1) / PB; }

inline const bf16* B16(const unsigned short* p) { return reinterpret_cast<const bf16*>(p); }
inline bf16* B16(unsigned short* p) { return reinterpret_cast<bf16*>(p); }

cudaError_t nn_forward(const NNBuffers& B, const NNGrid& g, cudaStream_t s, const NNPredict* pred) {
  // four lanes per point in every layer (4 outputs each; the last layer splits its 16 inputs)
  // (the prediction reads channel-last inputs, see nn_inputs, and keeps its activations channel-last)
  const int nb = blocks_for(4 * g.npts);
  if (pred) {
    k_nn_fwd<4, 16, true, 4, 1, false, true><<<nb, 256, 0, s>>>(g, B16(B.x0), B.wq + kNNOff[0], B.wq + kNNOff[1],
                                                                 nullptr, B16(B.a1));
    k_nn_fwd<16, 16, true, 4, 1, false, true><<<nb, 256, 0, s>>>(g, B16(B.a1), B.wq + kNNOff[2], B.wq + kNNOff[3],
                                                                  nullptr, B16(B.a2));
    k_nn_fwd<16, 1, false, 1, 4, true, true><<<nb, 256, 0, s>>>(g, B16(B.a2), B.wq + kNNOff[4], B.wq + kNNOff[5],
                                                                 B.out, nullptr, *pred, B.stats);
    return cudaGetLastError();
  }
  k_nn_fwd<4, 16, true, 4, 1><<<nb, 256, 0, s>>>(g, B16(B.x0), B.wq + kNNOff[0], B.wq + kNNOff[1], B.y1, B16(B.a1));
  k_nn_fwd<16, 16, true, 4, 1><<<nb, 256, 0, s>>>(g, B16(B.a1), B.wq + kNNOff[2], B.wq + kNNOff[3], B.y2, B16(B.a2));
  k_nn_fwd<16, 1, false, 1, 4><<<nb, 256, 0, s>>>(g, B16(B.a2), B.wq + kNNOff[4], B.wq + kNNOff[5], B.out, nullptr);
  return cudaGetLastError();
}

cudaError_t nn_backward(const NNBuffers& B, const NNGrid& g, cudaStream_t s) {
  const int nb = blocks_for(g.npts);
  const int nblk = nn_part_blocks(g.npts);
  // layer 3: weight gradient and the gradient into layer 2
  k_nn_bwd_weight<16, 1><<<nblk, 256, 0, s>>>(g, B.dout, B16(B.a2), B.part);
  k_nn_reduce<<<blocks_for(16 * 27 + 1), 256, 0, s>>>(B.part, nblk, 16 * 27 + 1, B.grad + kNNOff[4]);
  k_nn_bwd_data<16, 1><<<nb, 256, 0, s>>>(g, B.dout, B.wq + kNNOff[4], B.y2, B.dy2);
  // layer 2
  k_nn_bwd_weight<16, 16><<<nblk, 256, 0, s>>>(g, B.dy2, B16(B.a1), B.part);
  k_nn_reduce<<<blocks_for(16 * 16 * 27 + 16), 256, 0, s>>>(B.part, nblk, 16 * 16 * 27 + 16, B.grad + kNNOff[2]);
  k_nn_bwd_data<16, 16><<<nb, 256, 0, s>>>(g, B.dy2, B.wq + kNNOff[2], B.y1, B.dy1);
  // layer 1 (no gradient into the inputs)
  k_nn_bwd_weight<4, 16><<<nblk, 256, 0, s>>>(g, B.dy1, B16(B.x0), B.part);
  k_nn_reduce<<<blocks_for(16 * 4 * 27 + 16), 256, 0, s>>>(B.part, nblk, 16 * 4 * 27 + 16, B.grad + kNNOff[0]);
  return cudaGetLastError();
}

cudaError_t nn_loss(const NNBuffers& B, const NNGrid& g, double* loss_acc, cudaStream_t s) {
  k_nn_loss<<<1, 256, 0, s>>>(B.out, B.target, g.npts, B.dout, loss_acc);
  return cudaGetLastError();
}

cudaError_t nn_adam(const NNBuffers& B, float lr, int t, float gscale, cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
  k_nn_adam<<<blocks_for(kNNParams), 256, 0, s>>>(B.params, B.grad, B.m, B.v, B.wq, kNNParams, lr, b1, b2,
                                                   1e-8f, c1, c2, gscale);
  k_nn_pack_weights<<<8, 256, 0, s>>>(B.wq, reinterpret_cast<FusedWeights*>(B.wpack));
  return cudaGetLastError();
}

cudaError_t nn_round_weights(const NNBuffers& B, cudaStream_t s) {
  k_nn_round<<<blocks_for(kNNParams), 256, 0, s>>>(B.params, B.wq, kNNParams);
  k_nn_pack_weights<<<8, 256, 0, s>>>(B.wq, reinterpret_cast<FusedWeights*>(B.wpack));
  return cudaGetLastError();
}

size_t nn_wpack_bytes() { return sizeof(FusedWeights); }

cudaError_t nn_inputs(const NNBuffers& B, const NNGrid& g, const double* V0, const double* V1,
                      const double* V2, const double* V3, const double* Vnext, cudaStream_t s,
                      bool channel_last) {
  k_nn_stats<<<grid_sum_blocks(g.npts, 256), 256, 0, s>>>(V0, V1, V2, V3, g.npts, B.red, B.ticket, B.stats);
  k_nn_pack<<<blocks_for(g.npts), 256, 0, s>>>(V0, V1, V2, V3, Vnext, B.stats, g.npts, channel_last ? 1 : 0,
                                               B16(B.x0), B.target);
  return cudaGetLastError();
}

cudaError_t nn_apply(const NNBuffers& B, const NNGrid& g, const double* V0, const double* V1,
                     const double* V2, const double* V3, int mode, double* vpred, cudaStream_t s) {
  k_nn_apply<<<blocks_for(g.npts), 256, 0, s>>>(V0, V1, V2, V3, B.out, B.stats, g.npts, mode, vpred);
  return cudaGetLastError();
}

cudaError_t nn_predict_fused(const NNBuffers& B, const NNGrid& g, const NNPredict& pr, long long wait_limit,
                             cudaStream_t s) {
  static int nsm = 0, occ = 0;
  if (nsm == 0) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_nn_predict, kFusedThreads, 0);
    if (e != cudaSuccess) { nsm = 0; return e; }
  }
  long long want = (4LL * g.npts + kFusedThreads - 1) / kFusedThreads;
  long long nb = (long long)nsm * occ;
  if (nb > kFusedMaxBlocks) nb = kFusedMaxBlocks;
  if (nb > want) nb = want;
  if (nb < 1) nb = 1;
  FusedArgs A{g, pr.V0, pr.V1, pr.V2, pr.V3, pr.vpred, pr.vloc, pr.vhxc, pr.vstep64, pr.vstep32, B.wpack,
              B16(B.x0), B16(B.a1), B16(B.a2), B.stats, B.red, 1.0 / (double)g.npts, B.bar, B.err, wait_limit};
  void* args[] = {&A};
  return cudaLaunchCooperativeKernel((const void*)k_nn_predict, dim3((unsigned)nb), dim3(kFusedThreads), args, 0, s);
}

cudaError_t launch_decide(const double* res, double thr, const double* vnew, double* vhxc, double* vnext, int n,
                          double* fb, cudaGraphConditionalHandle handle, cudaStream_t s) {
  int nb = (n + 255) / 256;
  nb = nb < 1 ? 1 : (nb > 152 ? 152 : nb);
  k_decide<<<nb, 256, 0, s>>>(res, thr, vnew, vhxc, vnext, n, fb, handle);
  return cudaGetLastError();
}

cudaError_t launch_store6(double* dst, const double v[6], cudaStream_t s) {
  k_store6<<<1, 32, 0, s>>>(dst, v[0], v[1], v[2], v[3], v[4], v[5]);
  return cudaGetLastError();
}

cudaError_t launch_residual(const double* Vnew, const double* Vpred, int n, double* partials, unsigned* ticket,
                            double* res, cudaStream_t s) {
  return launch_pdl(k_residual, dim3((unsigned)grid_sum_blocks(n, 256)), dim3(256), 0, s, 0, Vnew, Vpred, n, partials,
                    ticket, res);
}

}  // namespace tdks
