// Orbital kernels with the whole orbital resident in shared memory.
//
// One CTA owns one orbital (k, n).  It copies the orbital into shared memory once, applies the
// Hamiltonian of Eq. (TDKS_solid) -- 25-point Laplacian, -i q.grad (9-point first derivative
// per axis), |q|^2/2 + V, and the Kleinman-Bylander projectors with the gauge phase of Sec. 4.1
// -- and, for the Taylor propagator, runs all four Horner stages
//     v <- psi + (-i dt / m) H v,   m = 4, 3, 2, 1
// without leaving the SM, so one Taylor step reads and writes the orbital in HBM once.
// The density of Eq. (rho) is accumulated from the final stage (FP64 atomics).
#include <cuda_runtime.h>

#include "tdks_internal.h"

namespace tdks {

namespace {

template <typename T> struct Vec;
template <> struct Vec<float> {
  using C = float2;
  static __device__ __forceinline__ void sincos_(float x, float* s, float* c) { sincosf(x, s, c); }
};
template <> struct Vec<double> {
  using C = double2;
  static __device__ __forceinline__ void sincos_(double x, double* s, double* c) { sincos(x, s, c); }
};

template <typename T>
struct SmemLayout {
  using C = typename Cplx<T>::type;
  C* v;      // [npts] current Horner vector
  C* ph;     // [nsph] exp(i q.d)
  C* ec;     // [natom*4] E_p * c_ap
};

template <typename T>
__device__ __forceinline__ SmemLayout<T> carve(unsigned char* raw, int npts, int nsph) {
  using C = typename Cplx<T>::type;
  SmemLayout<T> L;
  L.v = reinterpret_cast<C*>(raw);
  L.ph = L.v + npts;
  L.ec = L.ph + nsph;
  return L;
}

// point index -> (x, y, z) without integer division (exact for the grid sizes used here)
__device__ __forceinline__ void unpack(int p, int nx, int ny, float inx, float iny, int& x, int& y,
                                       int& z) {
  int row = __float2int_rd((p + 0.5f) * inx);
  x = p - row * nx;
  z = __float2int_rd((row + 0.5f) * iny);
  y = row - z * ny;
}

// Projections of the shared-memory vector: ec[a*4+p] = E_p * dV * sum_i beta_ip ph_i v(idx_i).
template <typename T, int NT>
__device__ __forceinline__ void project(const OrbArgs<T>& a, SmemLayout<T> L) {
  using C = typename Cplx<T>::type;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int at = warp; at < a.natom; at += NT / 32) {
    T acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int e0 = a.atom_off[at], e1 = a.atom_off[at + 1];
    for (int i = e0 + lane; i < e1; i += 32) {
      const C v = L.v[a.sph_idx[i]];
      const C ph = L.ph[i];
      const T re = v.x * ph.x - v.y * ph.y;
      const T im = v.x * ph.y + v.y * ph.x;
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const T b = a.sph_beta[i * 4 + p];
        acc[2 * p] += b * re;
        acc[2 * p + 1] += b * im;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
    if (lane < 4) {
      const T s = a.atomE[at * 4 + lane] * a.dV;
      C c;
      c.x = acc[2 * lane] * s;
      c.y = acc[2 * lane + 1] * s;
      L.ec[at * 4 + lane] = c;
    }
  }
}

// (H_q v)(p) from the shared-memory vector.
template <typename T, bool PER>
__device__ __forceinline__ typename Cplx<T>::type apply_h(const OrbArgs<T>& a, SmemLayout<T> L,
                                                          int p, int x, int y, int z, T diag,
                                                          const T* gx, const T* gy, const T* gz) {
  using C = typename Cplx<T>::type;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int sxy = nx * ny;
  const C u0 = L.v[p];
  const T vloc = a.V[p] + diag;
  T re = vloc * u0.x, im = vloc * u0.y;
  const int row = p - x;
  // x neighbours
#pragma unroll
  for (int m = 1; m <= 4; ++m) {
    int xp = x + m, xm = x - m;
    C up, um;
    if (PER) {
      xp -= (xp >= nx) ? nx : 0;
      xm += (xm < 0) ? nx : 0;
      up = L.v[row + xp];
      um = L.v[row + xm];
    } else {
      up = (xp < nx) ? L.v[row + xp] : C{0, 0};
      um = (xm >= 0) ? L.v[row + xm] : C{0, 0};
    }
    const T sr = up.x + um.x, si = up.y + um.y, dr = up.x - um.x, di = up.y - um.y;
    re += a.c2x[m] * sr;
    im += a.c2x[m] * si;
    if (PER) { re += gx[m - 1] * di; im -= gx[m - 1] * dr; }
  }
  // y neighbours
  const int plane = z * sxy + x;
#pragma unroll
  for (int m = 1; m <= 4; ++m) {
    int yp = y + m, ym = y - m;
    C up, um;
    if (PER) {
      yp -= (yp >= ny) ? ny : 0;
      ym += (ym < 0) ? ny : 0;
      up = L.v[plane + yp * nx];
      um = L.v[plane + ym * nx];
    } else {
      up = (yp < ny) ? L.v[plane + yp * nx] : C{0, 0};
      um = (ym >= 0) ? L.v[plane + ym * nx] : C{0, 0};
    }
    const T sr = up.x + um.x, si = up.y + um.y, dr = up.x - um.x, di = up.y - um.y;
    re += a.c2y[m] * sr;
    im += a.c2y[m] * si;
    if (PER) { re += gy[m - 1] * di; im -= gy[m - 1] * dr; }
  }
  // z neighbours
  const int col = p - z * sxy;
#pragma unroll
  for (int m = 1; m <= 4; ++m) {
    int zp = z + m, zm = z - m;
    C up, um;
    if (PER) {
      zp -= (zp >= nz) ? nz : 0;
      zm += (zm < 0) ? nz : 0;
      up = L.v[col + zp * sxy];
      um = L.v[col + zm * sxy];
    } else {
      up = (zp < nz) ? L.v[col + zp * sxy] : C{0, 0};
      um = (zm >= 0) ? L.v[col + zm * sxy] : C{0, 0};
    }
    const T sr = up.x + um.x, si = up.y + um.y, dr = up.x - um.x, di = up.y - um.y;
    re += a.c2z[m] * sr;
    im += a.c2z[m] * si;
    if (PER) { re += gz[m - 1] * di; im -= gz[m - 1] * dr; }
  }
  // nonlocal: sum over projector entries touching this point
  const int e0 = a.pt_off[p], e1 = a.pt_off[p + 1];
  for (int e = e0; e < e1; ++e) {
    const int i = a.pt_ent[e];
    const int at = a.ent_atom[i];
    T sr = 0, si = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const T b = a.sph_beta[i * 4 + q];
      const C c = L.ec[at * 4 + q];
      sr += b * c.x;
      si += b * c.y;
    }
    const C ph = L.ph[i];   // multiply by conj(ph)
    re += sr * ph.x + si * ph.y;
    im += si * ph.x - sr * ph.y;
  }
  return C{re, im};
}

template <typename T>
__device__ __forceinline__ void orbital_q(const OrbArgs<T>& a, int k, T q[3]) {
  q[0] = (T)(a.kpts[3 * k] + a.Ap[0]);
  q[1] = (T)(a.kpts[3 * k + 1] + a.Ap[1]);
  q[2] = (T)(a.kpts[3 * k + 2] + a.Ap[2]);
}

// Load the orbital and the per-entry phases exp(i q.d); returns diag term c0 sum + |q|^2/2 and
// the first-derivative weights q_a d_m / h_a.
template <typename T, int NT, bool PER>
__device__ __forceinline__ T prologue(const OrbArgs<T>& a, SmemLayout<T> L,
                                      const typename Cplx<T>::type* psi, T gx[4], T gy[4],
                                      T gz[4]) {
  const int k = blockIdx.x / a.norb;
  T q[3];
  orbital_q(a, k, q);
  for (int p = threadIdx.x; p < a.npts; p += NT) L.v[p] = psi[p];
  for (int i = threadIdx.x; i < a.nsph; i += NT) {
    const T arg = q[0] * a.sph_d[3 * i] + q[1] * a.sph_d[3 * i + 1] + q[2] * a.sph_d[3 * i + 2];
    T s, c;
    Vec<T>::sincos_(arg, &s, &c);
    L.ph[i] = typename Cplx<T>::type{c, s};
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    gx[m] = PER ? q[0] * a.d1x[m] : T(0);
    gy[m] = PER ? q[1] * a.d1y[m] : T(0);
    gz[m] = PER ? q[2] * a.d1z[m] : T(0);
  }
  return a.c2x[0] + a.c2y[0] + a.c2z[0] + T(0.5) * (q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
}

// MODE 0: psi_out = H psi_in.  MODE 1: psi_out = T4 psi_in (Horner), rho += 2 w_k |psi_out|^2.
// DBUF: the next Horner vector goes to a second shared-memory buffer; otherwise to the
// orbital's slice of a global scratch array (large FP64 cells), copied back after a barrier.
template <typename T, int NT, int MODE, bool PER, bool DBUF>
__global__ void __launch_bounds__(NT) k_smem_orbital(OrbArgs<T> a, typename Cplx<T>::type* scratch) {
  using C = typename Cplx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmemLayout<T> L = carve<T>(smem_raw, a.npts, a.nsph);
  C* nxt = DBUF ? L.ec + 4 * a.natom : scratch + (size_t)blockIdx.x * a.npts;
  const int orb = blockIdx.x;
  const C* psi = a.psi_in + (size_t)orb * a.npts;
  C* out = a.psi_out + (size_t)orb * a.npts;
  T gx[4], gy[4], gz[4];
  const T diag = prologue<T, NT, PER>(a, L, psi, gx, gy, gz);
  const float inx = 1.0f / a.nx, iny = 1.0f / a.ny;
  const double w = (MODE == 1 && a.rho) ? 2.0 * a.kw[orb / a.norb] : 0.0;
  __syncthreads();
  constexpr int NSTAGE = (MODE == 1) ? 4 : 1;
#pragma unroll 1
  for (int st = 0; st < NSTAGE; ++st) {
    if (a.natom > 0) {
      project<T, NT>(a, L);
      __syncthreads();
    }
    const T coef = a.dt / T(4 - st);
    const bool last = (st + 1 == NSTAGE);
#pragma unroll 1
    for (int p = threadIdx.x; p < a.npts; p += NT) {
      int x, y, z;
      unpack(p, a.nx, a.ny, inx, iny, x, y, z);
      const C hv = apply_h<T, PER>(a, L, p, x, y, z, diag, gx, gy, gz);
      C r;
      if (MODE == 1) {
        const C ps = psi[p];
        r = C{ps.x + coef * hv.y, ps.y - coef * hv.x};   // psi + (-i coef) H v
      } else {
        r = hv;
      }
      if (!last) {
        nxt[p] = r;
      } else {
        if (MODE == 0 || a.write_out) out[p] = r;
        if (MODE == 1 && a.rho) atomicAdd(&a.rho[p], w * ((double)r.x * r.x + (double)r.y * r.y));
      }
    }
    if (!last) {
      __syncthreads();
      if (DBUF) {
        C* t = L.v; L.v = nxt; nxt = t;
      } else {
        for (int p = threadIdx.x; p < a.npts; p += NT) L.v[p] = nxt[p];
        __syncthreads();
      }
    }
  }
}

// Per-orbital observables: norm, local and nonlocal current, <u|H_q|u> (a.V = V_loc).
template <typename T, int NT, bool PER>
__global__ void __launch_bounds__(NT) k_smem_observables(OrbArgs<T> a, double* obs) {
  using C = typename Cplx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmemLayout<T> L = carve<T>(smem_raw, a.npts, a.nsph);
  __shared__ double red[NT / 32][8];
  const int orb = blockIdx.x;
  const C* psi = a.psi_in + (size_t)orb * a.npts;
  T gx[4], gy[4], gz[4];
  const T diag = prologue<T, NT, PER>(a, L, psi, gx, gy, gz);
  const int k = orb / a.norb;
  T q[3];
  orbital_q(a, k, q);
  const float inx = 1.0f / a.nx, iny = 1.0f / a.ny;
  __syncthreads();
  if (a.natom > 0) {
    project<T, NT>(a, L);
    __syncthreads();
  }
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const int nx = a.nx, ny = a.ny, nz = a.nz, sxy = nx * ny;
  for (int p = threadIdx.x; p < a.npts; p += NT) {
    int x, y, z;
    unpack(p, nx, ny, inx, iny, x, y, z);
    const C u = L.v[p];
    const C hv = apply_h<T, PER>(a, L, p, x, y, z, diag, gx, gy, gz);
    const double uu = (double)u.x * u.x + (double)u.y * u.y;
    acc[0] += uu;
    acc[7] += (double)u.x * hv.x + (double)u.y * hv.y;
    if (PER) {
      // Im(conj(u) D1_a u) + q_a |u|^2
      const int row = p - x, plane = z * sxy + x, col = p - z * sxy;
      double d1[3][2] = {{0, 0}, {0, 0}, {0, 0}};
      for (int m = 1; m <= 4; ++m) {
        int xp = x + m, xm = x - m, yp = y + m, ym = y - m, zp = z + m, zm = z - m;
        xp -= (xp >= nx) ? nx : 0; xm += (xm < 0) ? nx : 0;
        yp -= (yp >= ny) ? ny : 0; ym += (ym < 0) ? ny : 0;
        zp -= (zp >= nz) ? nz : 0; zm += (zm < 0) ? nz : 0;
        const C ax = L.v[row + xp], bx = L.v[row + xm];
        const C ay = L.v[plane + yp * nx], by = L.v[plane + ym * nx];
        const C az = L.v[col + zp * sxy], bz = L.v[col + zm * sxy];
        d1[0][0] += a.d1x[m - 1] * ((double)ax.x - bx.x); d1[0][1] += a.d1x[m - 1] * ((double)ax.y - bx.y);
        d1[1][0] += a.d1y[m - 1] * ((double)ay.x - by.x); d1[1][1] += a.d1y[m - 1] * ((double)ay.y - by.y);
        d1[2][0] += a.d1z[m - 1] * ((double)az.x - bz.x); d1[2][1] += a.d1z[m - 1] * ((double)az.y - bz.y);
      }
      for (int c = 0; c < 3; ++c)
        acc[1 + c] += (double)u.x * d1[c][1] - (double)u.y * d1[c][0] + (double)q[c] * uu;
    }
  }
  // nonlocal current: sum_ap 2 E_p Im(conj(b_ap^(c)) c_ap), one warp per atom
  if (PER) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int at = warp; at < a.natom; at += NT / 32) {
      double cb[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
      double bb[3][4][2];
      for (int c = 0; c < 3; ++c)
        for (int pp = 0; pp < 4; ++pp) bb[c][pp][0] = bb[c][pp][1] = 0;
      for (int i = a.atom_off[at] + lane; i < a.atom_off[at + 1]; i += 32) {
        const C v = L.v[a.sph_idx[i]];
        const C ph = L.ph[i];
        const double re = (double)v.x * ph.x - (double)v.y * ph.y;
        const double im = (double)v.x * ph.y + (double)v.y * ph.x;
        for (int pp = 0; pp < 4; ++pp) {
          const double b = a.sph_beta[i * 4 + pp];
          cb[pp][0] += b * re;
          cb[pp][1] += b * im;
          for (int c = 0; c < 3; ++c) {
            const double dd = a.sph_d[3 * i + c];
            bb[c][pp][0] += dd * b * re;
            bb[c][pp][1] += dd * b * im;
          }
        }
      }
      for (int o = 16; o > 0; o >>= 1)
        for (int pp = 0; pp < 4; ++pp) {
          cb[pp][0] += __shfl_xor_sync(0xffffffffu, cb[pp][0], o);
          cb[pp][1] += __shfl_xor_sync(0xffffffffu, cb[pp][1], o);
          for (int c = 0; c < 3; ++c) {
            bb[c][pp][0] += __shfl_xor_sync(0xffffffffu, bb[c][pp][0], o);
            bb[c][pp][1] += __shfl_xor_sync(0xffffffffu, bb[c][pp][1], o);
          }
        }
      if (lane == 0) {
        const double dv2 = (double)a.dV * (double)a.dV;
        for (int c = 0; c < 3; ++c) {
          double s = 0;
          for (int pp = 0; pp < 4; ++pp) {
            // Im(conj(b) c) = b.re c.im - b.im c.re
            s += 2.0 * (double)a.atomE[at * 4 + pp] *
                 (bb[c][pp][0] * cb[pp][1] - bb[c][pp][1] * cb[pp][0]);
          }
          acc[4 + c] += s * dv2;
        }
      }
    }
  }
  // block reduction
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = 0; j < 8; ++j) {
    double v = acc[j];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][j] = v;
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    double v = 0;
    for (int w = 0; w < NT / 32; ++w) v += red[w][threadIdx.x];
    const double scale = (threadIdx.x >= 4 && threadIdx.x < 7) ? 1.0 : (double)a.dV;
    obs[orb * 8 + threadIdx.x] = v * scale;
  }
}

template <typename T, int NT, int MODE, bool PER, bool DBUF>
cudaError_t launch_one(const OrbArgs<T>& a, typename Cplx<T>::type* scratch, size_t smem,
                       cudaStream_t s) {
  auto kern = k_smem_orbital<T, NT, MODE, PER, DBUF>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<a.nk * a.norb, NT, smem, s>>>(a, scratch);
  return cudaGetLastError();
}

template <typename T, int NT, bool PER, bool DBUF>
cudaError_t launch_mode(const OrbArgs<T>& a, int mode, typename Cplx<T>::type* scratch,
                        size_t smem, cudaStream_t s) {
  return mode == 0 ? launch_one<T, NT, 0, PER, DBUF>(a, scratch, smem, s)
                   : launch_one<T, NT, 1, PER, DBUF>(a, scratch, smem, s);
}

constexpr int kNT = 512;

}  // namespace

template <typename T>
size_t smem_orbital_bytes(int npts, int nsph, int natom) {
  using C = typename Cplx<T>::type;
  return sizeof(C) * ((size_t)npts + nsph + 4 * (size_t)natom);
}

constexpr size_t kSmemLimit = 220 * 1024;

template <typename T>
bool smem_orbital_fits(int npts, int nsph, int natom) {
  return smem_orbital_bytes<T>(npts, nsph, natom) <= kSmemLimit;
}

template <typename T>
bool smem_orbital_needs_scratch(int npts, int nsph, int natom) {
  using C = typename Cplx<T>::type;
  return smem_orbital_bytes<T>(npts, nsph, natom) + sizeof(C) * (size_t)npts > kSmemLimit;
}

template <typename T>
cudaError_t launch_smem_orbital(const OrbArgs<T>& a, int mode, typename Cplx<T>::type* scratch,
                                cudaStream_t s) {
  using C = typename Cplx<T>::type;
  const size_t base = smem_orbital_bytes<T>(a.npts, a.nsph, a.natom);
  const bool dbuf = base + sizeof(C) * (size_t)a.npts <= kSmemLimit;
  if (!dbuf && mode == 1 && !scratch) return cudaErrorInvalidValue;
  const size_t smem = dbuf ? base + sizeof(C) * (size_t)a.npts : base;
  if (a.periodic)
    return dbuf ? launch_mode<T, kNT, true, true>(a, mode, scratch, smem, s)
                : launch_mode<T, kNT, true, false>(a, mode, scratch, smem, s);
  return dbuf ? launch_mode<T, kNT, false, true>(a, mode, scratch, smem, s)
              : launch_mode<T, kNT, false, false>(a, mode, scratch, smem, s);
}

template <typename T>
cudaError_t launch_orbital_observables(const OrbArgs<T>& a, double* out, cudaStream_t s) {
  const size_t smem = smem_orbital_bytes<T>(a.npts, a.nsph, a.natom);
  const int grid = a.nk * a.norb;
  if (a.periodic) {
    auto kern = k_smem_observables<T, kNT, true>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kNT, smem, s>>>(a, out);
  } else {
    auto kern = k_smem_observables<T, kNT, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kNT, smem, s>>>(a, out);
  }
  return cudaGetLastError();
}

template size_t smem_orbital_bytes<float>(int, int, int);
template size_t smem_orbital_bytes<double>(int, int, int);
template bool smem_orbital_fits<float>(int, int, int);
template bool smem_orbital_fits<double>(int, int, int);
template bool smem_orbital_needs_scratch<float>(int, int, int);
template bool smem_orbital_needs_scratch<double>(int, int, int);
template cudaError_t launch_smem_orbital<float>(const OrbArgs<float>&, int, float2*, cudaStream_t);
template cudaError_t launch_smem_orbital<double>(const OrbArgs<double>&, int, double2*, cudaStream_t);
template cudaError_t launch_orbital_observables<float>(const OrbArgs<float>&, double*, cudaStream_t);
template cudaError_t launch_orbital_observables<double>(const OrbArgs<double>&, double*, cudaStream_t);

}  // namespace tdks
