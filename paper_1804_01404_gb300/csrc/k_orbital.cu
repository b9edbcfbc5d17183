// Orbital kernels with the whole orbital resident in shared memory ("cell" kernels).
//
// One CTA owns one orbital (k, n).  It copies the orbital into shared memory once, applies the
// Hamiltonian of Eq. (TDKS_solid) -- 25-point Laplacian, -i q.grad (9-point first derivative per
// axis), |q|^2/2 + V, and the Kleinman-Bylander projectors with the gauge phase of Sec. 4.1 -- and,
// for the Taylor propagator, runs all four Horner stages
//     v <- psi + (-i dt / m) H v,   m = 4, 3, 2, 1
// without leaving the SM, so one Taylor step reads and writes the orbital in HBM once.
//
// Work split inside the CTA: a thread owns one (x, y) column segment and marches along z,
// keeping the nine z-values u(z-4..z+4) of its column in registers; the 16 x/y neighbours come
// from shared memory through offsets computed once per column.  Two buffer schemes:
//   * two buffers (DBUF): a stage reads one shared-memory copy and writes the other (or a global
//     scratch slice when two copies do not fit);
//   * one buffer swept in place (IP, planes of up to kNTip points): one thread per column, all
//     columns advance through z together, and the result of plane z replaces the input after a
//     barrier, once every thread has read that input plane.  The input planes 0..3 that periodic
//     columns still need at the end of the sweep (their images beyond the last plane) are kept in
//     a small side buffer.  Half the shared memory lets two CTAs share an SM, so one CTA's loads,
//     projections and barriers overlap the other's stencil work.  Complex FP32 arithmetic uses the
// packed f32x2 instructions.  The nonlocal scatter runs as a separate pass over the grid points
// that lie inside a projector sphere.  The last pass writes the orbital, accumulates the density
// of Eq. (rho) (FP64 atomics; FP32 orbitals add into per-k FP32 partials folded in FP64) and, on
// request, the norm and the current of Eq. (macro_current).
#include <cuda_runtime.h>

#include <cstdint>

#include <type_traits>

#include "ff.cuh"
#include "tdks_internal.h"
#include "warp_sum.cuh"

namespace tdks {

namespace {

// ------------------------------------------------------------------ complex helpers
template <typename T> struct CM;

template <> struct CM<float> {
  using C = float2;
  // packed f32x2 arithmetic (one instruction for the real and imaginary parts)
  static __device__ __forceinline__ C add(C a, C b) { return __fadd2_rn(a, b); }
  static __device__ __forceinline__ C sub(C a, C b) { return __ffma2_rn(make_float2(-1.0f, -1.0f), b, a); }
  // acc + s * a  (s real, broadcast to both lanes)
  static __device__ __forceinline__ C fma(float s, C a, C acc) { return __ffma2_rn(make_float2(s, s), a, acc); }
  static __device__ __forceinline__ C mul(float s, C a) { return __fmul2_rn(make_float2(s, s), a); }
  static __device__ __forceinline__ void sincos_(float x, float* s, float* c) { sincosf(x, s, c); }
};

template <> struct CM<double> {
  using C = double2;
  static __device__ __forceinline__ C add(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
  static __device__ __forceinline__ C sub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
  static __device__ __forceinline__ C fma(double s, C a, C acc) {
    return C{__fma_rn(s, a.x, acc.x), __fma_rn(s, a.y, acc.y)};
  }
  static __device__ __forceinline__ C mul(double s, C a) { return C{s * a.x, s * a.y}; }
  static __device__ __forceinline__ void sincos_(double x, double* s, double* c) { sincos(x, s, c); }
};

// ------------------------------------------------------------------ shared-memory layout
template <typename T>
struct Smem {
  using C = typename Cplx<T>::type;
  C* v;      // [nz * pstride] current vector
  C* nxt;    // [nz * pstride] next vector (double-buffer mode)
  C* ph;     // [nsph] exp(i q.d)
  C* ec;     // [natom*4] E_p * dV * c_ap
  C* sv;     // IP, periodic: [4][nx*ny] input planes 0..3 of the current stage
};

template <typename T>
__host__ __device__ inline size_t cell_smem_bytes(int nz, int pstride, int nsph, int natom, bool dbuf) {
  using C = typename Cplx<T>::type;
  const size_t vsz = (size_t)nz * pstride;
  return sizeof(C) * (vsz * (dbuf ? 2 : 1) + nsph + 4 * (size_t)natom);
}

// Threads per CTA (upper bound): 25 warps for FP32 (two z-segments per column of a 20^2 plane; the
// warps-per-scheduler count caps registers at 72), 16 warps for FP64 so that its wider values get
// 128 registers per thread.
template <typename T> constexpr int kNTof() { return sizeof(T) == 4 ? 800 : 512; }
// Column segments: about one per thread in FP32; two per thread in FP64, whose CTA of 16 warps then
// spreads the FP64 work evenly over the four schedulers of the SM (one segment per column of a
// 20 x 20 plane leaves one scheduler 3.5 warps of work and the others 3).
template <typename T> constexpr int kSegThreads() { return sizeof(T) == 4 ? kNTof<T>() : 2 * kNTof<T>(); }
constexpr size_t kSmemLimit = 220 * 1024;
// In-place sweep: at most kNTip columns (one thread each); FP32 CTAs are sized for two per SM
// (72 registers per thread), FP64 CTAs for one.
constexpr int kNTip = 448;
// FP32 fixed geometries (GEOM != 0): two x-adjacent points per thread, at most kNTpair threads.
constexpr int kNTpair = 416;
// ... and with two copies (scheme 2) kProjWarpsGeom further warps that only project: the projection
// of a stage reads the current copy while the stencil writes the other, so it runs beside the
// local pass instead of delaying the warps that would otherwise take an atom each before their
// column segments (the barrier after the local pass waits for the slowest warp).
constexpr int kProjWarpsGeom = 2;
// ... and with one copy swept in place (scheme 3): one thread per column pair, at most kNTpairIP, two
// CTAs per SM.
constexpr int kNTpairIP = 224;
template <typename T, bool IP, int GEOM = 0> constexpr int kMaxThreads() {
  return (GEOM != 0 && sizeof(T) == 4) ? (IP ? kNTpairIP : kNTpair + 32 * kProjWarpsGeom)
                                       : (IP ? kNTip : kNTof<T>());
}
template <typename T, bool IP> constexpr int kMinBlocks() { return (IP && sizeof(T) == 4) ? 2 : 1; }

// Fixed geometries also hold the projector tables of the sphere entries in shared memory: beta_ip
// (4 values, 16-byte aligned) and the point index with the atom in bits 16..30 and, in the sign bit,
// whether the point lies inside more than one sphere.
template <typename T>
__host__ __device__ inline size_t cell_smem_bytes_ip(int nx, int ny, int nz, int pstride, int nsph, int natom,
                                                     bool periodic) {
  using C = typename Cplx<T>::type;
  return sizeof(C) * ((size_t)nz * pstride + nsph + 4 * (size_t)natom + (periodic ? 4 * (size_t)nx * ny : 0));
}
// ip: after the layout of the in-place sweep (one copy and the saved planes) instead of two copies
template <typename T>
__host__ __device__ inline size_t geom_table_offset(int nx, int ny, int nz, int pstride, int nsph, int natom,
                                                    bool ip) {
  const size_t base = ip ? cell_smem_bytes_ip<T>(nx, ny, nz, pstride, nsph, natom, true)
                         : cell_smem_bytes<T>(nz, pstride, nsph, natom, true);
  return (base + 15) & ~size_t(15);
}
template <typename T>
inline size_t cell_smem_bytes_geom(int nx, int ny, int nz, int pstride, int nsph, int natom, bool ip) {
  return geom_table_offset<T>(nx, ny, nz, pstride, nsph, natom, ip) + (size_t)nsph * (4 * sizeof(T) + sizeof(int));
}

// Projections of the shared-memory vector:  ec[a*4+p] = E_p dV sum_i beta_ip ph_i v(idx_i), one warp
// per atom.
template <typename T>
__device__ __forceinline__ void project(const OrbArgs<T>& a, const typename Cplx<T>::type* v,
                                        const typename Cplx<T>::type* ph,
                                        typename Cplx<T>::type* ec) {
  using C = typename Cplx<T>::type;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int at = warp; at < a.natom; at += nw) {
    T acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int e1 = a.atom_off[at + 1];
    for (int i = a.atom_off[at] + lane; i < e1; i += 32) {
      const C u = v[a.sph_sidx[i]];
      const C f = ph[i];
      const T re = u.x * f.x - u.y * f.y, im = u.x * f.y + u.y * f.x;
      const T* b = a.sph_beta + 4 * i;
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        acc[2 * p] += b[p] * re;
        acc[2 * p + 1] += b[p] * im;
      }
    }
    const T tot = warp_split_sum<8>(acc);        // lane L: total of acc[L >> 2]
    if ((lane & 3) == 0) {
      const int j = lane >> 2, p = j >> 1;          // acc[2p]: Re, acc[2p+1]: Im of projector p
      reinterpret_cast<T*>(ec)[2 * (at * 4 + p) + (j & 1)] = tot * (a.atomE[at * 4 + p] * a.dV);
    }
  }
}

template <typename T, bool PER>
struct Column {
  int col, x, y, z0, z1;
  int ix[8], iy[8];   // in-plane index of x+-m, y+-m neighbours (pad index when outside)
};

template <typename T, bool PER>
__device__ __forceinline__ Column<T, PER> make_column(const OrbArgs<T>& a, int item) {
  Column<T, PER> c;
  const int nxy = a.nx * a.ny;
  c.col = item % nxy;
  const int seg = item / nxy;
  c.y = c.col / a.nx;
  c.x = c.col - c.y * a.nx;
  c.z0 = seg * a.zlen;
  c.z1 = min(a.nz, c.z0 + a.zlen);
#pragma unroll
  for (int m = 1; m <= 4; ++m) {
    int xp = c.x + m, xm = c.x - m, yp = c.y + m, ym = c.y - m;
    if (PER) {
      xp -= (xp >= a.nx) ? a.nx : 0; xm += (xm < 0) ? a.nx : 0;
      yp -= (yp >= a.ny) ? a.ny : 0; ym += (ym < 0) ? a.ny : 0;
      c.ix[2 * (m - 1)] = c.y * a.nx + xp;
      c.ix[2 * (m - 1) + 1] = c.y * a.nx + xm;
      c.iy[2 * (m - 1)] = yp * a.nx + c.x;
      c.iy[2 * (m - 1) + 1] = ym * a.nx + c.x;
    } else {
      c.ix[2 * (m - 1)] = (xp < a.nx) ? c.y * a.nx + xp : nxy;
      c.ix[2 * (m - 1) + 1] = (xm >= 0) ? c.y * a.nx + xm : nxy;
      c.iy[2 * (m - 1)] = (yp < a.ny) ? yp * a.nx + c.x : nxy;
      c.iy[2 * (m - 1) + 1] = (ym >= 0) ? ym * a.nx + c.x : nxy;
    }
  }
  return c;
}

template <typename T, bool PER>
__device__ __forceinline__ typename Cplx<T>::type zload(const OrbArgs<T>& a,
                                                        const typename Cplx<T>::type* v, int zz,
                                                        int col) {
  using C = typename Cplx<T>::type;
  if (PER) {
    zz += (zz < 0) ? a.nz : 0;
    zz -= (zz >= a.nz) ? a.nz : 0;
  } else if (zz < 0 || zz >= a.nz) {
    return C{0, 0};
  }
  return v[zz * a.pstride + col];
}

// Local part of (H v) at one point: diag*v + S + (-i) q.D.  nb(j) gives the in-plane neighbours
// (j = 2(m-1): x+m, 2(m-1)+1: x-m, 8 + 2(m-1): y+m, 8 + 2(m-1)+1: y-m), wz(j) the z-values
// u(z-4+j), j = 0..8.
// WD (periodic cells): also return the per-axis first-derivative sums D1_a v in Dout[3], with one
// accumulator per axis.  Otherwise each neighbour distance m uses one Laplacian and one derivative
// coefficient, the axes entering through the fixed ratios (c2y = ry c2x, d1y = ty d1x, ...):
//   S += c2x[m] (X_m + ry Y_m + rz Z_m),  q.D += d1x[m] (q_x X'_m + ty q_y Y'_m + tz q_z Z'_m)
// (X_m: x+m plus x-m values, X'_m: their difference), which halves the coefficient registers.
// FMA64 (FP64, periodic, without the per-axis sums): each neighbour pair of axis a and distance m
// enters as S += c2_a[m] (u+ + u-) - i (q_a d1_a[m]) (u+ - u-), two adds and four FMAs, which leaves
// 100 FP64 instructions per point instead of 113 (the FP64 pipe bounds these kernels).
template <typename T, bool PER, bool WD, typename NB, typename WZ, bool FMA64 = true>
__device__ __forceinline__ typename Cplx<T>::type local_h_at(const OrbArgs<T>& a, NB nb, WZ wz, T diag,
                                                             const T* q, typename Cplx<T>::type* Dout) {
  using C = typename Cplx<T>::type;
  using M = CM<T>;
  if constexpr (FMA64 && sizeof(T) == 8 && PER && !WD) {
    C S = M::fma(diag, wz(4), C{0, 0});
#pragma unroll
    for (int m = 1; m <= 4; ++m) {
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        const C up = ax == 0 ? nb(2 * (m - 1)) : (ax == 1 ? nb(8 + 2 * (m - 1)) : wz(4 + m));
        const C um = ax == 0 ? nb(2 * (m - 1) + 1) : (ax == 1 ? nb(8 + 2 * (m - 1) + 1) : wz(4 - m));
        const T c2 = ax == 0 ? a.c2x[m] : (ax == 1 ? a.c2y[m] : a.c2z[m]);
        const T b = q[ax] * (ax == 0 ? a.d1x[m - 1] : (ax == 1 ? a.d1y[m - 1] : a.d1z[m - 1]));
        const T sr = up.x + um.x, si = up.y + um.y, dr = up.x - um.x, di = up.y - um.y;
        S.x = fma(b, di, fma(c2, sr, S.x));
        S.y = fma(-b, dr, fma(c2, si, S.y));
      }
    }
    return S;
  }
  if (WD) {
    // independent accumulators per axis keep the FMA chains short
    C Sx = M::fma(diag, wz(4), C{0, 0}), Sy = C{0, 0}, Sz = C{0, 0};
    C Dx = C{0, 0}, Dy = C{0, 0}, Dz = C{0, 0};
#pragma unroll
    for (int m = 1; m <= 4; ++m) {
      const C xp = nb(2 * (m - 1)), xm = nb(2 * (m - 1) + 1);
      const C yp = nb(8 + 2 * (m - 1)), ym = nb(8 + 2 * (m - 1) + 1);
      const C zp = wz(4 + m), zm = wz(4 - m);
      Sx = M::fma(a.c2x[m], M::add(xp, xm), Sx);
      Sy = M::fma(a.c2y[m], M::add(yp, ym), Sy);
      Sz = M::fma(a.c2z[m], M::add(zp, zm), Sz);
      Dx = M::fma(a.d1x[m - 1], M::sub(xp, xm), Dx);
      Dy = M::fma(a.d1y[m - 1], M::sub(yp, ym), Dy);
      Dz = M::fma(a.d1z[m - 1], M::sub(zp, zm), Dz);
    }
    C S = M::add(M::add(Sx, Sy), Sz);
    const C D = M::fma(q[2], Dz, M::fma(q[1], Dy, M::fma(q[0], Dx, C{0, 0})));
    Dout[0] = Dx; Dout[1] = Dy; Dout[2] = Dz;
    return C{S.x + D.y, S.y - D.x};   // + (-i) q.D
  }
  C S = M::fma(diag, wz(4), C{0, 0});
  C D = C{0, 0};
  const T qy = q[1] * a.ty, qz = q[2] * a.tz;
#pragma unroll
  for (int m = 1; m <= 4; ++m) {
    const C xp = nb(2 * (m - 1)), xm = nb(2 * (m - 1) + 1);
    const C yp = nb(8 + 2 * (m - 1)), ym = nb(8 + 2 * (m - 1) + 1);
    const C zp = wz(4 + m), zm = wz(4 - m);
    S = M::fma(a.c2x[m], M::fma(a.rz, M::add(zp, zm), M::fma(a.ry, M::add(yp, ym), M::add(xp, xm))), S);
    if (PER)
      D = M::fma(a.d1x[m - 1],
                 M::fma(qz, M::sub(zp, zm), M::fma(qy, M::sub(yp, ym), M::mul(q[0], M::sub(xp, xm)))), D);
  }
  if (PER) S = C{S.x + D.y, S.y - D.x};   // + (-i) q.D
  return S;
}

// local_h_at for a column: in-plane neighbours at the column's precomputed offsets in plane zb,
// z-values from the window w.
template <typename T, bool PER, bool WD, bool FMA64 = true>
__device__ __forceinline__ typename Cplx<T>::type local_h(const OrbArgs<T>& a,
                                                          const Column<T, PER>& c,
                                                          const typename Cplx<T>::type* v,
                                                          const typename Cplx<T>::type* w, int zb,
                                                          T diag, const T* q,
                                                          typename Cplx<T>::type* Dout) {
  auto nb = [&](int j) { return v[zb + (j < 8 ? c.ix[j] : c.iy[j - 8])]; };
  auto wz = [&](int j) { return w[j]; };
  return local_h_at<T, PER, WD, decltype(nb), decltype(wz), FMA64>(a, nb, wz, diag, q, Dout);
}

// Projections from the shared-memory tables (fixed geometries): as project(), with beta_ip and the
// point index of entry i read from tbeta[4i..4i+3] and tidx[i] & 0xffff.
template <typename T>
__device__ __forceinline__ void project_tab(const OrbArgs<T>& a, const typename Cplx<T>::type* v,
                                            const typename Cplx<T>::type* ph, const int* tidx,
                                            const T* tbeta, typename Cplx<T>::type* ec, int warp, int nw) {
  using C = typename Cplx<T>::type;
  const int lane = threadIdx.x & 31;
  for (int at = warp; at < a.natom; at += nw) {
    T acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int e1 = a.atom_off[at + 1];
    for (int i = a.atom_off[at] + lane; i < e1; i += 32) {
      const C u = v[tidx[i] & 0xffff];
      const C f = ph[i];
      const T re = u.x * f.x - u.y * f.y, im = u.x * f.y + u.y * f.x;
      const T* b = tbeta + 4 * i;
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        acc[2 * p] += b[p] * re;
        acc[2 * p + 1] += b[p] * im;
      }
    }
    const T tot = warp_split_sum<8>(acc);        // lane L: total of acc[L >> 2]
    if ((lane & 3) == 0) {
      const int j = lane >> 2, p = j >> 1;
      reinterpret_cast<T*>(ec)[2 * (at * 4 + p) + (j & 1)] = tot * (a.atomE[at * 4 + p] * a.dV);
    }
  }
}

// Nonlocal scatter from the shared-memory tables, one sphere entry per thread: entry i of atom a adds
// conj(ph_i) sum_p beta_ip ec_ap (MODE 0), or -i coef times that (a Horner stage), to the next vector
// at its point.  A point inside one sphere only (tidx >= 0) is updated by a plain read-modify-write;
// a point inside several (the sign bit of tidx set) receives one shared-memory atomic add per entry.
template <typename T, int MODE>
__device__ __forceinline__ void scatter_tab(const OrbArgs<T>& a, const typename Cplx<T>::type* ph,
                                            const typename Cplx<T>::type* ec, const int* tidx,
                                            const T* tbeta, typename Cplx<T>::type* nxt, T coef) {
  using C = typename Cplx<T>::type;
  for (int i = threadIdx.x; i < a.nsph; i += blockDim.x) {
    const int pk = tidx[i];
    const int at = (pk >> 16) & 0x7fff;
    const T* b = tbeta + 4 * i;
    T sr = 0, si = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const C cc = ec[at * 4 + q];
      sr += b[q] * cc.x;
      si += b[q] * cc.y;
    }
    const C f = ph[i];
    C nl = C{sr * f.x + si * f.y, si * f.x - sr * f.y};
    if (MODE == 1) nl = C{coef * nl.y, -coef * nl.x};
    C* dst = nxt + (pk & 0xffff);
    if (pk < 0) {
      atomicAdd(&dst->x, nl.x);
      atomicAdd(&dst->y, nl.y);
    } else {
      C r = *dst;
      r.x += nl.x;
      r.y += nl.y;
      *dst = r;
    }
  }
}

// ------------------------------------------------------------------ fixed cell geometries
// Periodic cells whose size is a template parameter (GEOM 1: 20^3, GEOM 2: 16^3; 0: any size).  A
// thread's column segment is unrolled over its ZL planes: the z window rotates by renaming registers,
// and every shared-memory access of the segment is one of 18 per-thread base addresses plus a
// compile-time plane offset, so the loads and stores need no address arithmetic.
template <int GEOM> struct Geom;
template <> struct Geom<1> { static constexpr int NX = 20, NY = 20, NZ = 20; };
template <> struct Geom<2> { static constexpr int NX = 16, NY = 16, NZ = 16; };

// the column split of cell_split for this geometry
template <typename T, int GEOM>
struct GeomT {
  static constexpr int NX = Geom<GEOM>::NX, NY = Geom<GEOM>::NY, NZ = Geom<GEOM>::NZ, NXY = NX * NY;
  static constexpr int S0 = kSegThreads<T>() / NXY;
  static constexpr int S = S0 < 1 ? 1 : (S0 > NZ ? NZ : S0);
  static constexpr int ZL = (NZ + S - 1) / S;
  static constexpr int NSEG = (NZ + ZL - 1) / ZL;
};

__device__ __forceinline__ float2 lds_c(unsigned addr, float) {
  float2 r;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(r.x), "=f"(r.y) : "r"(addr));
  return r;
}
__device__ __forceinline__ double2 lds_c(unsigned addr, double) {
  double2 r;
  asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(r.x), "=d"(r.y) : "r"(addr));
  return r;
}
__device__ __forceinline__ void sts_c(unsigned addr, float2 v) {
  asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y));
}
__device__ __forceinline__ void sts_c(unsigned addr, double2 v) {
  asm volatile("st.shared.v2.f64 [%0], {%1, %2};" ::"r"(addr), "d"(v.x), "d"(v.y));
}

// One column segment of a Taylor stage (MODE 1: psi + (-i coef) H v) or of H v (MODE 0) for a fixed
// geometry: reads the shared-memory vector at byte address sv, writes the next one at sn.  ACC: also
// add |u|^2 and Im(conj(u) D1_a u) of the input to os (the first stage of OBS 2).
template <typename T, int GEOM, int MODE, bool ACC>
__device__ __forceinline__ void fixed_column(const OrbArgs<T>& a, int item, unsigned sv, unsigned sn,
                                             const T* __restrict__ Vc,
                                             const typename Cplx<T>::type* __restrict__ psi, T diag0,
                                             const T* q, T coef, T os[5]) {
  using C = typename Cplx<T>::type;
  using M = CM<T>;
  using G = GeomT<T, GEOM>;
  constexpr int NX = G::NX, NY = G::NY, NZ = G::NZ, NXY = G::NXY, ZL = G::ZL;
  constexpr bool RAGGED = (NZ % ZL) != 0;
  constexpr unsigned CB = sizeof(C), PB = NXY * sizeof(C);   // bytes per point, per plane
  const int col = item % NXY, seg = item / NXY;
  const int y = col / NX, x = col - y * NX;
  const int z0 = seg * ZL;
  const unsigned p0 = (unsigned)(z0 * NXY) * CB;
  unsigned nbA[16];                                  // plane z0: x+-m, y+-m (periodic images)
#pragma unroll
  for (int m = 1; m <= 4; ++m) {
    const int xp = x + m - (x + m >= NX ? NX : 0), xm = x - m + (x - m < 0 ? NX : 0);
    const int yp = y + m - (y + m >= NY ? NY : 0), ym = y - m + (y - m < 0 ? NY : 0);
    nbA[2 * (m - 1)] = sv + p0 + (unsigned)(y * NX + xp) * CB;
    nbA[2 * (m - 1) + 1] = sv + p0 + (unsigned)(y * NX + xm) * CB;
    nbA[8 + 2 * (m - 1)] = sv + p0 + (unsigned)(yp * NX + x) * CB;
    nbA[8 + 2 * (m - 1) + 1] = sv + p0 + (unsigned)(ym * NX + x) * CB;
  }
  const unsigned cA = sv + p0 + (unsigned)col * CB, oA = sn + p0 + (unsigned)col * CB;
  C w[9];                                            // plane z0 + k - 4 + j in w[(k + j) % 9]
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    int zz = z0 - 4 + j;
    zz += zz < 0 ? NZ : 0;
    zz -= zz >= NZ ? NZ : 0;
    w[j] = lds_c(sv + (unsigned)(zz * NXY + col) * CB, T());
  }
  const T* Vp = Vc + z0 * NXY + col;
  const C* Pp = psi + z0 * NXY + col;
  const int len = NZ - z0;
#pragma unroll
  for (int k = 0; k < ZL; ++k) {
    if (RAGGED && k >= len) break;
    const T diag = diag0 + Vp[k * NXY];
    C Dd[3];
    const C hv = local_h_at<T, true, ACC>(
        a, [&](int j) { return lds_c(nbA[j] + (unsigned)k * PB, T()); }, [&](int j) { return w[(k + j) % 9]; },
        diag, q, Dd);
    if (ACC) {                                       // |u|^2 and Im(conj(u) D1_a u)
      const C u0 = w[(k + 4) % 9];
      os[0] += u0.x * u0.x + u0.y * u0.y;
#pragma unroll
      for (int d = 0; d < 3; ++d) os[1 + d] += u0.x * Dd[d].y - u0.y * Dd[d].x;
    }
    C r;
    if (MODE == 1) r = M::fma(coef, C{hv.y, -hv.x}, Pp[k * NXY]);   // psi + (-i coef) H v
    else r = hv;
    sts_c(oA + (unsigned)k * PB, r);
    if (k < ZL - 1) {                                // plane z + 5 replaces plane z - 4
      const bool wrap = z0 + k + 5 >= NZ;
      w[k % 9] = lds_c(cA + (unsigned)(k + 5) * PB - (wrap ? (unsigned)NZ * PB : 0u), T());
    }
  }
}

// FP32 fixed geometries: a thread owns two x-adjacent points (x even) of a column segment.  The
// points of a row pair are one 16-byte shared-memory load, so the 16 x-neighbours of the two points
// come from four loads and their 16 y-neighbours from eight: 13 loads per two points with the z
// window, against 17 per point for one point per thread.
template <int GEOM>
struct GeomP {
  static constexpr int NX = Geom<GEOM>::NX, NY = Geom<GEOM>::NY, NZ = Geom<GEOM>::NZ, NXY = NX * NY;
  static constexpr int NP = NXY / 2;                       // point pairs per plane
  static constexpr int S0 = kNTpair / NP;
  static constexpr int S = S0 < 1 ? 1 : (S0 > NZ ? NZ : S0);
  static constexpr int ZL = (NZ + S - 1) / S;
  static constexpr int NSEG = (NZ + ZL - 1) / ZL;
  static_assert(NX % 2 == 0, "point pairs need an even nx");
};

__device__ __forceinline__ float4 lds_c2(unsigned addr) {
  float4 r;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w) : "r"(addr));
  return r;
}
__device__ __forceinline__ void sts_c2(unsigned addr, float4 v) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w));
}
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

template <int GEOM, int MODE, bool ACC>
__device__ __forceinline__ void fixed_pair(const OrbArgs<float>& a, int item, unsigned sv, unsigned sn,
                                           const float* __restrict__ Vc, const float2* __restrict__ psi,
                                           float diag0, const float* q, float coef, float os[5]) {
  using M = CM<float>;
  using G = GeomP<GEOM>;
  constexpr int NX = G::NX, NY = G::NY, NZ = G::NZ, NXY = G::NXY, ZL = G::ZL;
  constexpr bool RAGGED = (NZ % ZL) != 0;
  constexpr unsigned CB = sizeof(float2), PB = NXY * sizeof(float2);
  const int pi = item % G::NP, seg = item / G::NP;
  const int col = 2 * pi;
  const int y = col / NX, x = col - y * NX;          // x even
  const int z0 = seg * ZL;
  const unsigned p0 = sv + (unsigned)(z0 * NXY) * CB;
  auto wx = [](int v) { return v < 0 ? v + NX : (v >= NX ? v - NX : v); };
  auto wy = [](int v) { return v < 0 ? v + NY : (v >= NY ? v - NY : v); };
  // pairs (x-4, x-3), (x-2, x-1), (x+2, x+3), (x+4, x+5) of row y; the pair (x, x+1) of rows y +- m
  const unsigned xa0 = p0 + (unsigned)(y * NX + wx(x - 4)) * CB, xa1 = p0 + (unsigned)(y * NX + wx(x - 2)) * CB;
  const unsigned xa2 = p0 + (unsigned)(y * NX + wx(x + 2)) * CB, xa3 = p0 + (unsigned)(y * NX + wx(x + 4)) * CB;
  unsigned ya[8];
#pragma unroll
  for (int m = 1; m <= 4; ++m) {
    ya[2 * (m - 1)] = p0 + (unsigned)(wy(y + m) * NX + x) * CB;
    ya[2 * (m - 1) + 1] = p0 + (unsigned)(wy(y - m) * NX + x) * CB;
  }
  const unsigned cA = p0 + (unsigned)col * CB, oA = sn + (unsigned)(z0 * NXY + col) * CB;
  float4 w[9];                                       // plane z0 + k - 4 + j in w[(k + j) % 9]
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    int zz = z0 - 4 + j;
    zz += zz < 0 ? NZ : 0;
    zz -= zz >= NZ ? NZ : 0;
    w[j] = lds_c2(sv + (unsigned)(zz * NXY + col) * CB);
  }
  const float* Vp = Vc + z0 * NXY + col;
  const float2* Pp = psi + z0 * NXY + col;
  const int len = NZ - z0;
#pragma unroll
  for (int k = 0; k < ZL; ++k) {
    if (RAGGED && k >= len) break;
    const unsigned ko = (unsigned)k * PB;
    const float4 XM4 = lds_c2(xa0 + ko), XM2 = lds_c2(xa1 + ko), XP2 = lds_c2(xa2 + ko), XP4 = lds_c2(xa3 + ko);
    float4 Y[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) Y[j] = lds_c2(ya[j] + ko);
    const float4 Wc = w[(k + 4) % 9];
    const float2 Vv = *reinterpret_cast<const float2*>(Vp + k * NXY);
    // in-plane neighbours of point A (x) and B (x + 1), in local_h_at's order
    auto nbA = [&](int j) -> float2 {
      switch (j) {
        case 0: return hi2(Wc);  case 1: return hi2(XM2); case 2: return lo2(XP2); case 3: return lo2(XM2);
        case 4: return hi2(XP2); case 5: return hi2(XM4); case 6: return lo2(XP4); case 7: return lo2(XM4);
        default: return lo2(Y[j - 8]);
      }
    };
    auto nbB = [&](int j) -> float2 {
      switch (j) {
        case 0: return lo2(XP2); case 1: return lo2(Wc);  case 2: return hi2(XP2); case 3: return hi2(XM2);
        case 4: return lo2(XP4); case 5: return lo2(XM2); case 6: return hi2(XP4); case 7: return hi2(XM4);
        default: return hi2(Y[j - 8]);
      }
    };
    float2 DdA[3], DdB[3];
    const float2 hA = local_h_at<float, true, ACC>(a, nbA, [&](int j) { return lo2(w[(k + j) % 9]); },
                                                   diag0 + Vv.x, q, DdA);
    const float2 hB = local_h_at<float, true, ACC>(a, nbB, [&](int j) { return hi2(w[(k + j) % 9]); },
                                                   diag0 + Vv.y, q, DdB);
    if (ACC) {                                       // |u|^2 and Im(conj(u) D1_a u) of both points
      const float2 uA = lo2(Wc), uB = hi2(Wc);
      os[0] += uA.x * uA.x + uA.y * uA.y;
#pragma unroll
      for (int d = 0; d < 3; ++d) os[1 + d] += uA.x * DdA[d].y - uA.y * DdA[d].x;
      os[0] += uB.x * uB.x + uB.y * uB.y;
#pragma unroll
      for (int d = 0; d < 3; ++d) os[1 + d] += uB.x * DdB[d].y - uB.y * DdB[d].x;
    }
    float2 rA = hA, rB = hB;
    if (MODE == 1) {                                 // psi + (-i coef) H v
      const float4 P = *reinterpret_cast<const float4*>(Pp + k * NXY);
      rA = M::fma(coef, make_float2(hA.y, -hA.x), lo2(P));
      rB = M::fma(coef, make_float2(hB.y, -hB.x), hi2(P));
    }
    sts_c2(oA + ko, make_float4(rA.x, rA.y, rB.x, rB.y));
    if (k < ZL - 1) {                                // plane z + 5 replaces plane z - 4
      const bool wrap = z0 + k + 5 >= NZ;
      w[k % 9] = lds_c2(cA + (unsigned)(k + 5) * PB - (wrap ? (unsigned)NZ * PB : 0u));
    }
  }
}

// One Taylor stage of an FP32 fixed geometry with one copy swept in place (scheme 3): a thread owns
// the column pair pi (x = 2 pi mod nx even) over all planes, and all threads advance through z
// together; the result of plane z replaces the input after a barrier, once every thread has read that
// input plane as a neighbour plane.  The z window keeps the input values of planes z-4 .. z+4 in
// registers (loaded before they are replaced); the input planes 0..3, which the last planes need as
// their periodic images, are kept in the side buffer at ssv.  Inactive threads (act = false) take
// part in the barriers only.
template <int GEOM, bool ACC>
__device__ __forceinline__ void fixed_ip_pair(const OrbArgs<float>& a, int pi, bool act, unsigned sv, unsigned ssv,
                                              const float* __restrict__ Vc, const float2* __restrict__ psi,
                                              float diag0, const float* q, float coef, float os[5]) {
  using M = CM<float>;
  using G = GeomP<GEOM>;
  constexpr int NX = G::NX, NY = G::NY, NZ = G::NZ, NXY = G::NXY;
  constexpr unsigned CB = sizeof(float2), PB = NXY * sizeof(float2);
  const int col = act ? 2 * pi : 0;
  const int y = col / NX, x = col - y * NX;
  auto wx = [](int v) { return v < 0 ? v + NX : (v >= NX ? v - NX : v); };
  auto wy = [](int v) { return v < 0 ? v + NY : (v >= NY ? v - NY : v); };
  const unsigned xa0 = sv + (unsigned)(y * NX + wx(x - 4)) * CB, xa1 = sv + (unsigned)(y * NX + wx(x - 2)) * CB;
  const unsigned xa2 = sv + (unsigned)(y * NX + wx(x + 2)) * CB, xa3 = sv + (unsigned)(y * NX + wx(x + 4)) * CB;
  unsigned ya[8];
#pragma unroll
  for (int m = 1; m <= 4; ++m) {
    ya[2 * (m - 1)] = sv + (unsigned)(wy(y + m) * NX + x) * CB;
    ya[2 * (m - 1) + 1] = sv + (unsigned)(wy(y - m) * NX + x) * CB;
  }
  const unsigned cA = sv + (unsigned)col * CB, sA = ssv + (unsigned)col * CB;
  float4 w[9];                                       // plane z - 4 + j in w[(z + j) % 9]
  if (act) {
#pragma unroll
    for (int j = 0; j < 9; ++j) w[j] = lds_c2(cA + (unsigned)((j - 4 + NZ) % NZ) * PB);
#pragma unroll
    for (int j = 0; j < 4; ++j) {                  // input planes 0..3 (8-byte accesses: the side
      sts_c(sA + (unsigned)j * PB, lo2(w[4 + j])); // buffer is only 8-byte aligned)
      sts_c(sA + (unsigned)j * PB + CB, hi2(w[4 + j]));
    }
  }
#pragma unroll
  for (int z = 0; z < NZ; ++z) {
    float4 rr = make_float4(0.f, 0.f, 0.f, 0.f);
    if (act) {
      const unsigned ko = (unsigned)z * PB;
      const float4 XM4 = lds_c2(xa0 + ko), XM2 = lds_c2(xa1 + ko), XP2 = lds_c2(xa2 + ko), XP4 = lds_c2(xa3 + ko);
      float4 Y[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) Y[j] = lds_c2(ya[j] + ko);
      const float4 Wc = w[(z + 4) % 9];
      const float2 Vv = *reinterpret_cast<const float2*>(Vc + z * NXY + col);
      auto nbA = [&](int j) -> float2 {
        switch (j) {
          case 0: return hi2(Wc);  case 1: return hi2(XM2); case 2: return lo2(XP2); case 3: return lo2(XM2);
          case 4: return hi2(XP2); case 5: return hi2(XM4); case 6: return lo2(XP4); case 7: return lo2(XM4);
          default: return lo2(Y[j - 8]);
        }
      };
      auto nbB = [&](int j) -> float2 {
        switch (j) {
          case 0: return lo2(XP2); case 1: return lo2(Wc);  case 2: return hi2(XP2); case 3: return hi2(XM2);
          case 4: return lo2(XP4); case 5: return lo2(XM2); case 6: return hi2(XP4); case 7: return hi2(XM4);
          default: return hi2(Y[j - 8]);
        }
      };
      float2 DdA[3], DdB[3];
      const float2 hA = local_h_at<float, true, ACC>(a, nbA, [&](int j) { return lo2(w[(z + j) % 9]); },
                                                     diag0 + Vv.x, q, DdA);
      const float2 hB = local_h_at<float, true, ACC>(a, nbB, [&](int j) { return hi2(w[(z + j) % 9]); },
                                                     diag0 + Vv.y, q, DdB);
      if (ACC) {
        const float2 uA = lo2(Wc), uB = hi2(Wc);
        os[0] += uA.x * uA.x + uA.y * uA.y;
#pragma unroll
        for (int d = 0; d < 3; ++d) os[1 + d] += uA.x * DdA[d].y - uA.y * DdA[d].x;
        os[0] += uB.x * uB.x + uB.y * uB.y;
#pragma unroll
        for (int d = 0; d < 3; ++d) os[1 + d] += uB.x * DdB[d].y - uB.y * DdB[d].x;
      }
      const float4 P = *reinterpret_cast<const float4*>(psi + z * NXY + col);
      const float2 rA = M::fma(coef, make_float2(hA.y, -hA.x), lo2(P));   // psi + (-i coef) H v
      const float2 rB = M::fma(coef, make_float2(hB.y, -hB.x), hi2(P));
      rr = make_float4(rA.x, rA.y, rB.x, rB.y);
      // input plane z + 5: not yet replaced below nz; beyond, one of the saved planes 0..3
      if (z + 5 < NZ) w[z % 9] = lds_c2(cA + (unsigned)(z + 5) * PB);
      else if (z + 5 - NZ < 4) {
        const float2 l = lds_c(sA + (unsigned)(z + 5 - NZ) * PB, 0.f), h = lds_c(sA + (unsigned)(z + 5 - NZ) * PB + CB, 0.f);
        w[z % 9] = make_float4(l.x, l.y, h.x, h.y);
      }
    }
    __syncthreads();                                 // every thread has read input plane z
    if (act) sts_c2(cA + (unsigned)z * PB, rr);
  }
}

// Final pass of an FP32 fixed geometry over one column-pair segment of the propagated vector at
// shared-memory address sv: writes the orbital (out, nullable), adds 2 |u|^2 to the per-k density
// partial rho32 (nullable), and with OBS adds |u|^2 and Im(conj(u) D1_a u) (a = x, y, z) to os.
template <int GEOM, bool OBS>
__device__ __forceinline__ void fixed_final_pair(const OrbArgs<float>& a, int item, unsigned sv,
                                                 float2* __restrict__ out, float* __restrict__ rho32,
                                                 float os[5]) {
  using M = CM<float>;
  using G = GeomP<GEOM>;
  constexpr int NX = G::NX, NY = G::NY, NZ = G::NZ, NXY = G::NXY, ZL = G::ZL;
  constexpr bool RAGGED = (NZ % ZL) != 0;
  constexpr unsigned CB = sizeof(float2), PB = NXY * sizeof(float2);
  const int pi = item % G::NP, seg = item / G::NP;
  const int col = 2 * pi;
  const int y = col / NX, x = col - y * NX;
  const int z0 = seg * ZL;
  const unsigned p0 = sv + (unsigned)(z0 * NXY) * CB;
  auto wx = [](int v) { return v < 0 ? v + NX : (v >= NX ? v - NX : v); };
  auto wy = [](int v) { return v < 0 ? v + NY : (v >= NY ? v - NY : v); };
  const unsigned cA = p0 + (unsigned)col * CB;
  unsigned xa0 = 0, xa1 = 0, xa2 = 0, xa3 = 0, ya[8];
  float4 w[9];
  if (OBS) {
    xa0 = p0 + (unsigned)(y * NX + wx(x - 4)) * CB; xa1 = p0 + (unsigned)(y * NX + wx(x - 2)) * CB;
    xa2 = p0 + (unsigned)(y * NX + wx(x + 2)) * CB; xa3 = p0 + (unsigned)(y * NX + wx(x + 4)) * CB;
#pragma unroll
    for (int m = 1; m <= 4; ++m) {
      ya[2 * (m - 1)] = p0 + (unsigned)(wy(y + m) * NX + x) * CB;
      ya[2 * (m - 1) + 1] = p0 + (unsigned)(wy(y - m) * NX + x) * CB;
    }
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      int zz = z0 - 4 + j;
      zz += zz < 0 ? NZ : 0;
      zz -= zz >= NZ ? NZ : 0;
      w[j] = lds_c2(sv + (unsigned)(zz * NXY + col) * CB);
    }
  }
  const int len = NZ - z0;
#pragma unroll
  for (int k = 0; k < ZL; ++k) {
    if (RAGGED && k >= len) break;
    const unsigned ko = (unsigned)k * PB;
    const float4 Wc = OBS ? w[(k + 4) % 9] : lds_c2(cA + ko);
    const int pg = (z0 + k) * NXY + col;
    if (out) *reinterpret_cast<float4*>(out + pg) = Wc;
    const float2 rA = lo2(Wc), rB = hi2(Wc);
    const float rrA = rA.x * rA.x + rA.y * rA.y, rrB = rB.x * rB.x + rB.y * rB.y;
    if (rho32) {
      atomicAdd(rho32 + pg, 2.0f * rrA);
      atomicAdd(rho32 + pg + 1, 2.0f * rrB);
    }
    if (OBS) {
      const float4 XM4 = lds_c2(xa0 + ko), XM2 = lds_c2(xa1 + ko), XP2 = lds_c2(xa2 + ko), XP4 = lds_c2(xa3 + ko);
      float4 Y[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) Y[j] = lds_c2(ya[j] + ko);
      // x +- m of point A (x) and B (x + 1), as in fixed_pair
      const float2 axp[4] = {hi2(Wc), lo2(XP2), hi2(XP2), lo2(XP4)}, axm[4] = {hi2(XM2), lo2(XM2), hi2(XM4), lo2(XM4)};
      const float2 bxp[4] = {lo2(XP2), hi2(XP2), lo2(XP4), hi2(XP4)}, bxm[4] = {lo2(Wc), hi2(XM2), lo2(XM2), hi2(XM4)};
      float2 dA[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}}, dB[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
      for (int m = 1; m <= 4; ++m) {
        dA[0] = M::fma(a.d1x[m - 1], M::sub(axp[m - 1], axm[m - 1]), dA[0]);
        dB[0] = M::fma(a.d1x[m - 1], M::sub(bxp[m - 1], bxm[m - 1]), dB[0]);
        dA[1] = M::fma(a.d1y[m - 1], M::sub(lo2(Y[2 * (m - 1)]), lo2(Y[2 * (m - 1) + 1])), dA[1]);
        dB[1] = M::fma(a.d1y[m - 1], M::sub(hi2(Y[2 * (m - 1)]), hi2(Y[2 * (m - 1) + 1])), dB[1]);
        dA[2] = M::fma(a.d1z[m - 1], M::sub(lo2(w[(k + 4 + m) % 9]), lo2(w[(k + 4 - m) % 9])), dA[2]);
        dB[2] = M::fma(a.d1z[m - 1], M::sub(hi2(w[(k + 4 + m) % 9]), hi2(w[(k + 4 - m) % 9])), dB[2]);
      }
      os[0] += rrA + rrB;
#pragma unroll
      for (int d = 0; d < 3; ++d) os[1 + d] += (rA.x * dA[d].y - rA.y * dA[d].x) + (rB.x * dB[d].y - rB.y * dB[d].x);
      if (k < ZL - 1) {
        const bool wrap = z0 + k + 5 >= NZ;
        w[k % 9] = lds_c2(cA + (unsigned)(k + 5) * PB - (wrap ? (unsigned)NZ * PB : 0u));
      }
    }
  }
}

// Nonlocal value at sphere point s: sum over its entries of conj(ph_i) sum_p beta_ip ec_ap.
template <typename T>
__device__ __forceinline__ typename Cplx<T>::type nonlocal_at(const OrbArgs<T>& a, int s,
                                                              const typename Cplx<T>::type* ph,
                                                              const typename Cplx<T>::type* ec) {
  using C = typename Cplx<T>::type;
  T re = 0, im = 0;
  const int e1 = a.sp_off[s + 1];
  for (int e = a.sp_off[s]; e < e1; ++e) {
    const int i = a.pt_ent[e];
    const int at = a.ent_atom[i];
    T sr = 0, si = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const T b = a.sph_beta[i * 4 + q];
      const C cc = ec[at * 4 + q];
      sr += b * cc.x;
      si += b * cc.y;
    }
    const C f = ph[i];
    re += sr * f.x + si * f.y;
    im += si * f.x - sr * f.y;
  }
  return C{re, im};
}

template <typename T>
__device__ __forceinline__ void set_phases(const OrbArgs<T>& a, typename Cplx<T>::type* ph,
                                           const T q[3]) {
  for (int i = threadIdx.x; i < a.nsph; i += blockDim.x) {
    const T arg = q[0] * a.sph_d[3 * i] + q[1] * a.sph_d[3 * i + 1] + q[2] * a.sph_d[3 * i + 2];
    T s, c;
    CM<T>::sincos_(arg, &s, &c);
    ph[i] = typename Cplx<T>::type{c, s};
  }
}

// Accumulators of the per-orbital sums.  FP64 arithmetic runs at a small fraction of the FP32 rate
// on this GPU, so FP32 kernels accumulate in compensated float-float form (ff.cuh); FP64 kernels
// use double.
template <typename T> struct Acc;
template <> struct Acc<float> {
  using type = FF;
  static __device__ __forceinline__ FF zero() { return FF{0.f, 0.f}; }
  static __device__ __forceinline__ FF add(FF a, float x) { return ff_add(a, FF{x, 0.f}); }
  static __device__ __forceinline__ FF addv(FF a, FF b) { return ff_add(a, b); }
  // a float-float in one double slot of a shared array
  static __device__ __forceinline__ void store(double* r, int i, FF a) { reinterpret_cast<FF*>(r)[i] = a; }
  static __device__ __forceinline__ FF load(const double* r, int i) { return reinterpret_cast<const FF*>(r)[i]; }
  static __device__ __forceinline__ FF warp_sum(FF a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a = ff_add(a, ff_shfl_xor(a, o));
    return a;
  }
  static __device__ __forceinline__ double to_double(FF a) { return (double)a.hi + (double)a.lo; }
  static __device__ __forceinline__ FF from_double(double x) {
    const float h = (float)x;
    return FF{h, (float)(x - (double)h)};
  }
};
template <> struct Acc<double> {
  using type = double;
  static __device__ __forceinline__ double zero() { return 0.0; }
  static __device__ __forceinline__ double add(double a, double x) { return a + x; }
  static __device__ __forceinline__ double addv(double a, double b) { return a + b; }
  static __device__ __forceinline__ void store(double* r, int i, double a) { r[i] = a; }
  static __device__ __forceinline__ double load(const double* r, int i) { return r[i]; }
  static __device__ __forceinline__ double warp_sum(double a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    return a;
  }
  static __device__ __forceinline__ double to_double(double a) { return a; }
  static __device__ __forceinline__ double from_double(double x) { return x; }
};

// Per-orbital observables from per-thread partial sums v = {sum |u|^2, sum Im(conj(u) D1_a u) (a = x,
// y, z), sum Re(conj(u) (H u))}: warp sums in the accumulator type, one barrier, then thread j < 8 adds
// the warps' sums in the accumulator type (float-float for FP32 orbitals: a chain of dependent FP64
// adds would wait on the narrow FP64 pipe at every step) and writes out[j] = {norm, J_loc[3], J_nl[3],
// e} with J_loc_a = (sum Im(conj(u) D1_a u) + qo_a sum |u|^2) dV and J_nl from s_jnl.
// red: [8][32] shared doubles.
template <typename T>
__device__ __forceinline__ void reduce_obs(const T v[5], const T qo[3], double dV, const double* s_jnl,
                                           double* red, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  typename Acc<T>::type x[5];
#pragma unroll
  for (int j = 0; j < 5; ++j) x[j] = Acc<T>::warp_sum(Acc<T>::add(Acc<T>::zero(), v[j]));
  __syncthreads();                                 // red and s_jnl complete, red free
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < 5; ++j) Acc<T>::store(red, j * 32 + warp, x[j]);
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    const int j = threadIdx.x;
    typename Acc<T>::type s0 = Acc<T>::zero(), s1 = Acc<T>::zero();
    const int src = (j == 7) ? 4 : (j < 4 ? j : -1);
    if (src >= 0)
      for (int w = 0; w < nw; ++w) {
        s0 = Acc<T>::addv(s0, Acc<T>::load(red, src * 32 + w));
        s1 = Acc<T>::addv(s1, Acc<T>::load(red, w));
      }
    const double t[2] = {Acc<T>::to_double(s0), Acc<T>::to_double(s1)};
    double r;
    if (j == 0 || j == 7) r = t[0] * dV;
    else if (j < 4) r = (t[0] + (double)qo[j - 1] * t[1]) * dV;
    else r = s_jnl[j - 4];
    out[j] = r;
  }
}

// Nonlocal current of one orbital, sum over atoms of sum_p 2 E_p Im(conj(b_ap^(d)) c_ap) dV^2, with
// c_ap = sum_i beta_ip ph_i v_i and b_ap^(d) = sum_i d_i beta_ip ph_i v_i.  Every warp takes a chunk of
// one atom's sphere points (atoms in batches of kNLBatch, each split over the warps), partial sums
// meet in shared memory (part: [kNLBatch][32] of T), and thread a of the batch forms the products
// of atom a and adds it to s_jnl[3] (shared; zeroed by the caller).
// TAB: the point indices and beta_ip come from the shared-memory tables of the fixed geometries.
constexpr int kNLBatch = 16;
template <typename T, bool TAB = false>
__device__ __forceinline__ void nonlocal_current(const OrbArgs<T>& a, const typename Cplx<T>::type* v,
                                                 const typename Cplx<T>::type* ph, T* part,
                                                 double* s_jnl, const int* tidx = nullptr,
                                                 const T* tbeta = nullptr) {
  using C = typename Cplx<T>::type;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int ab = 0; ab < a.natom; ab += kNLBatch) {
    const int nb = min(kNLBatch, a.natom - ab);
    const int nch = max(1, nw / nb);               // chunks per atom
    for (int i = threadIdx.x; i < kNLBatch * 32; i += blockDim.x) part[i] = T(0);
    __syncthreads();
    for (int job = warp; job < nb * nch; job += nw) {
      const int at = ab + job / nch, ch = job % nch;
      T acc[32];                                  // [c, b_x, b_y, b_z][Re, Im of projector 0..3]
#pragma unroll
      for (int j = 0; j < 32; ++j) acc[j] = 0;
      for (int i = a.atom_off[at] + ch * 32 + lane; i < a.atom_off[at + 1]; i += 32 * nch) {
        const C u = v[TAB ? (tidx[i] & 0xffff) : a.sph_sidx[i]];
        const C f = ph[i];
        const T re = u.x * f.x - u.y * f.y, im = u.x * f.y + u.y * f.x;
        const T d0 = a.sph_d[3 * i], d1 = a.sph_d[3 * i + 1], d2 = a.sph_d[3 * i + 2];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          const T b = TAB ? tbeta[i * 4 + p] : a.sph_beta[i * 4 + p];
          acc[2 * p] += b * re; acc[2 * p + 1] += b * im;
          acc[8 + 2 * p] += d0 * b * re; acc[8 + 2 * p + 1] += d0 * b * im;
          acc[16 + 2 * p] += d1 * b * re; acc[16 + 2 * p + 1] += d1 * b * im;
          acc[24 + 2 * p] += d2 * b * re; acc[24 + 2 * p + 1] += d2 * b * im;
        }
      }
      const T tot = warp_split_sum<32>(acc);       // lane L: total of acc[L]
      atomicAdd(&part[(at - ab) * 32 + lane], tot);
    }
    __syncthreads();
    if (threadIdx.x < nb) {
      const int at = ab + threadIdx.x;
      const T* pa = part + threadIdx.x * 32;
      const double dv2 = (double)a.dV * (double)a.dV;
      for (int d = 0; d < 3; ++d) {
        // the products in the orbitals' precision (the sums in pa are of that precision already): for
        // FP32 orbitals no dependent FP64 chain on the narrow FP64 pipe
        T sacc = 0;
        for (int p = 0; p < 4; ++p) {
          const T br = pa[8 + 8 * d + 2 * p], bi = pa[8 + 8 * d + 2 * p + 1];
          const T im = fma(br, pa[2 * p + 1], -(bi * pa[2 * p]));   // Im(conj(b) c)
          sacc = fma(T(2) * a.atomE[at * 4 + p], im, sacc);
        }
        atomicAdd(&s_jnl[d], (double)sacc * dv2);
      }
    }
    __syncthreads();
  }
}

// MODE 0: out = H v.   MODE 1: out = T4 v (Horner), rho += 2 w_k |out|^2, optional fused
// observables.   MODE 2: observables only (norm, current, <v|H|v> with a.V).
// DBUF: next vector in shared memory; otherwise in the orbital's slice of `scratch`.
// OBS (MODE 1): 0 none; 1 norm and current of the propagated orbital, in an extra pass after the
// last stage; 2 norm and current of the input orbital, accumulated during the first stage from the
// per-axis derivative sums that stage forms anyway (no extra pass).  MODE 2 always uses 1.
template <typename T, int MODE, bool PER, bool DBUF, int OBS, bool IP, int GEOM = 0>
__global__ void __launch_bounds__(kMaxThreads<T, IP, GEOM>(), kMinBlocks<T, IP>())
    k_cell(OrbArgs<T> a, typename Cplx<T>::type* scratch) {
  static_assert(!IP || (MODE == 1 && !DBUF), "the in-place sweep serves the Taylor stages with one buffer");
  static_assert(GEOM == 0 || (PER && (DBUF || IP) && MODE != 2), "fixed geometries: periodic, two copies or in place");
  static_assert(!(GEOM != 0 && IP) || sizeof(T) == 4, "the fixed in-place sweep is FP32");
  using C = typename Cplx<T>::type;
  using M = CM<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[8 * 32];
  __shared__ T nl_part[kNLBatch * 32];
  __shared__ double s_jnl[3];
  const int nxy = a.nx * a.ny;
  const int ps = a.pstride;
  const int vsz = a.nz * ps;
  Smem<T> L;
  L.v = reinterpret_cast<C*>(smem_raw);
  L.nxt = IP ? L.v : L.v + vsz;
  L.ph = L.v + (DBUF ? 2 * vsz : vsz);
  L.ec = L.ph + a.nsph;
  L.sv = L.ec + 4 * a.natom;
  // fixed geometries: projector tables in shared memory (loaded below)
  T* tbeta = reinterpret_cast<T*>(smem_raw + geom_table_offset<T>(a.nx, a.ny, a.nz, ps, a.nsph, a.natom, IP));
  int* tidx = reinterpret_cast<int*>(tbeta + 4 * (size_t)a.nsph);
  const int orb = blockIdx.x;
  const int cell = orb / (a.nk * a.norb);
  const int k = (orb - cell * a.nk * a.norb) / a.norb;
  const C* psi = a.psi_in + (size_t)orb * a.npts;
  C* gnxt = DBUF ? nullptr : scratch + (size_t)orb * a.npts;
  const double* ap = a.Ap_cell ? a.Ap_cell + 3 * cell : a.Ap;
  const T* Vc = a.V + (size_t)cell * a.vstride;
  T q[3];
  q[0] = (T)(a.kpts[3 * k] + ap[0]);
  q[1] = (T)(a.kpts[3 * k + 1] + ap[1]);
  q[2] = (T)(a.kpts[3 * k + 2] + ap[2]);
  const T diag0 = a.c2x[0] + a.c2y[0] + a.c2z[0] + T(0.5) * (q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);

  // load the orbital (pad elements zero), phases; a predicted step also keeps a copy of its input
  // (the fallback restores it), written here while the values pass through
  C* bk = a.backup ? a.backup + (size_t)orb * a.npts : nullptr;
  if (PER && ps == nxy && ((vsz * sizeof(C)) & 15) == 0 && ((reinterpret_cast<uintptr_t>(psi) & 15) == 0)) {
    // a contiguous orbital: 16-byte copies, eight per thread in flight at once (a plain loop waits
    // for each load before the next); the next buffer needs no clearing (every point is written)
    const int nv = vsz * (int)sizeof(C) / 16;
    const uint4* src = reinterpret_cast<const uint4*>(psi);
    uint4* dst = reinterpret_cast<uint4*>(L.v);
    uint4* bkv = reinterpret_cast<uint4*>(bk);
    constexpr int U = 8;
    for (int base = threadIdx.x; base < nv; base += U * blockDim.x) {
      uint4 t[U];
#pragma unroll
      for (int j = 0; j < U; ++j) {
        const int i = base + j * blockDim.x;
        if (i < nv) t[j] = __ldg(src + i);
      }
#pragma unroll
      for (int j = 0; j < U; ++j) {
        const int i = base + j * blockDim.x;
        if (i < nv) {
          dst[i] = t[j];
          if (bkv) bkv[i] = t[j];
        }
      }
    }
  } else {
    for (int i = threadIdx.x; i < vsz; i += blockDim.x) {
      const int z = i / ps, r = i - z * ps;
      const C u = (r < nxy) ? psi[z * nxy + r] : C{0, 0};
      L.v[i] = u;
      if (bk && r < nxy) bk[z * nxy + r] = u;
      if (DBUF && !IP) L.nxt[i] = C{0, 0};
    }
  }
  if constexpr (GEOM != 0) {
    for (int i = threadIdx.x; i < a.nsph; i += blockDim.x) {
      const int pg = a.sph_idx[i];                 // periodic cells: the same as the shared-memory index
      const bool several = a.pt_off[pg + 1] - a.pt_off[pg] > 1;
      tidx[i] = a.sph_sidx[i] | (a.ent_atom[i] << 16) | (several ? (int)0x80000000u : 0);
#pragma unroll
      for (int p = 0; p < 4; ++p) tbeta[4 * i + p] = a.sph_beta[4 * i + p];
    }
  }
  // wave vector of the observables: k + A'_obs (OBS 1: end of the step; OBS 2: its start)
  auto obs_q = [&](T qo[3]) {
    qo[0] = q[0]; qo[1] = q[1]; qo[2] = q[2];
    if (OBS != 0 && MODE == 1) {
      const double* apo = a.Ap_obs_cell ? a.Ap_obs_cell + 3 * cell : a.Ap_obs;
      for (int d = 0; d < 3; ++d) qo[d] = (T)(a.kpts[3 * k + d] + apo[d]);
    }
  };
  if (OBS != 0 && threadIdx.x < 3) s_jnl[threadIdx.x] = 0.0;
  if (OBS == 2 && PER && a.natom > 0) {          // nonlocal current of the input orbital
    T qo[3];
    obs_q(qo);
    set_phases<T>(a, L.ph, qo);
    __syncthreads();                               // also completes the table load
    if constexpr (GEOM != 0) nonlocal_current<T, true>(a, L.v, L.ph, nl_part, s_jnl, tidx, tbeta);
    else nonlocal_current<T>(a, L.v, L.ph, nl_part, s_jnl);
  }
  set_phases<T>(a, L.ph, q);
  __syncthreads();

  const int nitems = nxy * a.nseg;
  constexpr int NSTAGE = (MODE == 1) ? 4 : 1;
  // two copies with the grid size built in (FP32): the last kProjWarpsGeom warps project, the nit
  // threads before them take the column segments
  const bool sep_proj = GEOM != 0 && !IP && sizeof(T) == 4 && a.natom > 0;
  const int nit = sep_proj ? (int)blockDim.x - 32 * kProjWarpsGeom : (int)blockDim.x;
  // per-thread partial sums of the observables {|u|^2, Im(conj(u) D1_a u) x3, Re(conj(u) H u)}
  T os[5] = {0, 0, 0, 0, 0};
#pragma unroll 1
  for (int st = 0; st < NSTAGE; ++st) {
    if constexpr (GEOM != 0) {
      // the projection only reads the current vector; the scatter that reads ec waits for the
      // barrier after the local pass (the in-place sweep replaces the vector: it waits here)
      if (a.natom > 0) {
        const int w = threadIdx.x >> 5;
        if (!sep_proj) project_tab<T>(a, L.v, L.ph, tidx, tbeta, L.ec, w, blockDim.x >> 5);
        else if (w >= nit / 32) project_tab<T>(a, L.v, L.ph, tidx, tbeta, L.ec, w - nit / 32, kProjWarpsGeom);
      }
      if (IP) __syncthreads();
    } else if (a.natom > 0) {
      project<T>(a, L.v, L.ph, L.ec);
      __syncthreads();
    }
    const T coef = a.dt / T(4 - st);
    // local part for every column segment; the first stage of OBS 2 also sums the observables of
    // its input (a separate instance of the loop, so the other stages compile as without them)
    auto local_pass = [&](auto acc_tag) {
      constexpr bool ACC = decltype(acc_tag)::value;
      if constexpr (IP && GEOM != 0) {
        const unsigned sv = (unsigned)__cvta_generic_to_shared(L.v), ssv = (unsigned)__cvta_generic_to_shared(L.sv);
        const int pi = threadIdx.x;
        fixed_ip_pair<GEOM, ACC && PER>(a, pi, pi < GeomP<GEOM>::NP, sv, ssv, Vc, psi, diag0, q, coef, os);
      } else if constexpr (IP) {
        const int col = threadIdx.x;
        const bool act = col < nxy;
        const Column<T, PER> c = make_column<T, PER>(a, act ? col : 0);
        C w[9];
        T vnext = T(0);
        C pnext = C{0, 0};
        if (act) {
#pragma unroll
          for (int j = 0; j < 9; ++j) w[j] = zload<T, PER>(a, L.v, j - 4, col);
          if (PER) {
#pragma unroll
            for (int j = 0; j < 4; ++j) L.sv[j * nxy + col] = w[4 + j];   // input planes 0..3
          }
          vnext = Vc[col];
          pnext = psi[col];
        }
#pragma unroll 1
        for (int z = 0; z < a.nz; ++z) {
          const int zb = z * ps;
          C r = C{0, 0};
          if (act) {
            const int pg = z * nxy + col;
            const T diag = diag0 + vnext;
            const C pv = pnext;
            if (z + 1 < a.nz) {                 // prefetch the next plane's V and psi
              vnext = Vc[pg + nxy];
              pnext = psi[pg + nxy];
            }
            C Dd[3];
            // (the in-place sweep keeps the separate Laplacian and derivative sums: fewer registers)
            const C hv = local_h<T, PER, ACC && PER, false>(a, c, L.v, w, zb, diag, q, Dd);
            if (ACC) {
              const C u0 = w[4];
              os[0] += u0.x * u0.x + u0.y * u0.y;
              if (PER) {
#pragma unroll
                for (int d = 0; d < 3; ++d) os[1 + d] += u0.x * Dd[d].y - u0.y * Dd[d].x;
              }
            }
            r = M::fma(coef, C{hv.y, -hv.x}, pv);   // psi + (-i coef) H v
#pragma unroll
            for (int j = 0; j < 8; ++j) w[j] = w[j + 1];
            // input plane z + 5: not yet replaced below nz; its periodic image beyond the last
            // plane is one of the saved planes 0..3 (the value loaded at the last plane is unused)
            const int zn = z + 5;
            if (zn < a.nz) w[8] = L.v[zn * ps + col];
            else if (PER && zn - a.nz < 4) w[8] = L.sv[(zn - a.nz) * nxy + col];
            else w[8] = C{0, 0};
          }
          __syncthreads();                      // every thread has read input plane z
          if (act) L.v[zb + col] = r;
        }
      } else if constexpr (GEOM != 0) {
        const unsigned sv = (unsigned)__cvta_generic_to_shared(L.v), sn = (unsigned)__cvta_generic_to_shared(L.nxt);
        if constexpr (sizeof(T) == 4) {
          constexpr int npair_items = GeomP<GEOM>::NP * GeomP<GEOM>::NSEG;
#pragma unroll 1
          for (int item = threadIdx.x; item < npair_items && (int)threadIdx.x < nit; item += nit)
            fixed_pair<GEOM, MODE, ACC && PER>(a, item, sv, sn, Vc, psi, diag0, q, coef, os);
        } else {
#pragma unroll 1
          for (int item = threadIdx.x; item < nitems; item += blockDim.x)
            fixed_column<T, GEOM, MODE, ACC && PER>(a, item, sv, sn, Vc, psi, diag0, q, coef, os);
        }
      } else {
#pragma unroll 1
        for (int item = threadIdx.x; item < nitems; item += blockDim.x) {
          const Column<T, PER> c = make_column<T, PER>(a, item);
          C w[9];
#pragma unroll
          for (int j = 0; j < 9; ++j) w[j] = zload<T, PER>(a, L.v, c.z0 - 4 + j, c.col);
          T vnext = Vc[c.z0 * nxy + c.col];
          C pnext = (MODE == 1) ? psi[c.z0 * nxy + c.col] : C{0, 0};
#pragma unroll 1
          for (int z = c.z0; z < c.z1; ++z) {
            const int zb = z * ps;
            const int pg = z * nxy + c.col;
            const T diag = diag0 + vnext;
            const C pv = pnext;
            if (z + 1 < c.z1) {                   // prefetch the next plane's V and psi
              vnext = Vc[pg + nxy];
              if (MODE == 1) pnext = psi[pg + nxy];
            }
            C Dd[3];
            const C hv = local_h<T, PER, ACC && PER>(a, c, L.v, w, zb, diag, q, Dd);
            if (ACC) {                            // |u|^2 and Im(conj(u) D1_a u)
              const C u0 = w[4];
              os[0] += u0.x * u0.x + u0.y * u0.y;
              if (PER) {
#pragma unroll
                for (int d = 0; d < 3; ++d) os[1 + d] += u0.x * Dd[d].y - u0.y * Dd[d].x;
              }
            }
            C r;
            if (MODE == 1) {
              r = M::fma(coef, C{hv.y, -hv.x}, pv);   // psi + (-i coef) H v
            } else {
              r = hv;
            }
            if (DBUF) L.nxt[zb + c.col] = r; else gnxt[pg] = r;
#pragma unroll
            for (int j = 0; j < 8; ++j) w[j] = w[j + 1];
            w[8] = zload<T, PER>(a, L.v, z + 5, c.col);
          }
        }
      }
    };
    if (OBS == 2 && st == 0) local_pass(std::integral_constant<bool, true>{});
    else local_pass(std::integral_constant<bool, false>{});
    if (OBS == 2 && st == 0) {                   // observables of the input orbital are complete
      T qo[3];
      obs_q(qo);
      reduce_obs<T>(os, qo, a.dV, s_jnl, red, a.obs + (size_t)orb * 8);
    }
    __syncthreads();
    // nonlocal scatter at sphere points
    if (GEOM != 0 && a.natom > 0) {
      scatter_tab<T, MODE>(a, L.ph, L.ec, tidx, tbeta, L.nxt, coef);
      __syncthreads();
    } else if (a.natom > 0) {
      for (int s = threadIdx.x; s < a.nsp; s += blockDim.x) {
        const C nl = nonlocal_at<T>(a, s, L.ph, L.ec);
        const int pg = a.sp_pt[s];
        const int zz = pg / nxy;
        const int pidx = (DBUF || IP) ? pg + zz * (ps - nxy) : pg;
        C* dst = (DBUF || IP) ? L.nxt : gnxt;
        C r = dst[pidx];
        if (MODE == 1) r = M::fma(coef, C{nl.y, -nl.x}, r);
        else r = M::add(r, nl);
        dst[pidx] = r;
      }
      __syncthreads();
    }
    if (MODE != 2 && !IP) {
      if (DBUF) {
        C* t = L.v; L.v = L.nxt; L.nxt = t;
      } else {
        for (int i = threadIdx.x; i < vsz; i += blockDim.x) {
          const int z = i / ps, r = i - z * ps;
          if (r < nxy) L.v[i] = gnxt[z * nxy + r];
        }
        __syncthreads();
      }
    }
  }

  // final pass: write, density, observables (OBS 1)
  const double wk = 2.0 * a.kw[k];
  C* out = a.psi_out ? a.psi_out + (size_t)orb * a.npts : nullptr;
  constexpr bool FINAL_OBS = (OBS == 1);
  if constexpr (GEOM != 0 && sizeof(T) == 4) {
    const unsigned sv = (unsigned)__cvta_generic_to_shared(L.v);
    float2* o = (MODE == 0 || (MODE == 1 && a.write_out)) ? out : nullptr;
    float* r32 = (MODE == 1 && a.rho32) ? a.rho32 + ((size_t)cell * a.nk + k) * a.npts : nullptr;
    constexpr int npair_items = GeomP<GEOM>::NP * GeomP<GEOM>::NSEG;
#pragma unroll 1
    for (int item = threadIdx.x; item < npair_items; item += blockDim.x)
      fixed_final_pair<GEOM, FINAL_OBS>(a, item, sv, o, r32, os);
  } else
#pragma unroll 1
  for (int item = threadIdx.x; item < (IP ? nxy : nitems); item += blockDim.x) {
    Column<T, PER> c = make_column<T, PER>(a, item);
    if (IP) { c.z0 = 0; c.z1 = a.nz; }           // whole columns
    C w[9];
    if (FINAL_OBS) {
#pragma unroll
      for (int j = 0; j < 9; ++j) w[j] = zload<T, PER>(a, L.v, c.z0 - 4 + j, c.col);
    }
#pragma unroll 1
    for (int z = c.z0; z < c.z1; ++z) {
      const int zb = z * ps;
      const int pg = z * nxy + c.col;
      const C r = L.v[zb + c.col];
      const T rr = r.x * r.x + r.y * r.y;
      if (MODE == 0 || (MODE == 1 && a.write_out)) out[pg] = r;
      if (MODE == 1) {
        if (a.rho32) atomicAdd(&a.rho32[((size_t)cell * a.nk + k) * a.npts + pg], 2.0f * (float)rr);
        else if (a.rho) atomicAdd(&a.rho[(size_t)cell * a.npts + pg], wk * (double)rr);
      }
      if (FINAL_OBS) {
        os[0] += rr;
        if (MODE == 2) {
          const C hv = DBUF ? L.nxt[zb + c.col] : gnxt[pg];
          os[4] += r.x * hv.x + r.y * hv.y;
        }
        if (PER) {
          // Im(conj(r) D1_a r) + q_a |r|^2
          C dx = C{0, 0}, dy = C{0, 0}, dz = C{0, 0};
#pragma unroll
          for (int m = 1; m <= 4; ++m) {
            dx = M::fma(a.d1x[m - 1], M::sub(L.v[zb + c.ix[2 * (m - 1)]], L.v[zb + c.ix[2 * (m - 1) + 1]]), dx);
            dy = M::fma(a.d1y[m - 1], M::sub(L.v[zb + c.iy[2 * (m - 1)]], L.v[zb + c.iy[2 * (m - 1) + 1]]), dy);
            dz = M::fma(a.d1z[m - 1], M::sub(w[4 + m], w[4 - m]), dz);
          }
          os[1] += r.x * dx.y - r.y * dx.x;
          os[2] += r.x * dy.y - r.y * dy.x;
          os[3] += r.x * dz.y - r.y * dz.x;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) w[j] = w[j + 1];
        w[8] = zload<T, PER>(a, L.v, z + 5, c.col);
      }
    }
  }
  if (!FINAL_OBS) return;

  // nonlocal current with the final phases: sum_ap 2 E_p Im(conj(b_ap^(d)) c_ap)
  T qo[3];
  obs_q(qo);
  if (PER && a.natom > 0) {
    __syncthreads();
    set_phases<T>(a, L.ph, qo);
    __syncthreads();
    if constexpr (GEOM != 0) nonlocal_current<T, true>(a, L.v, L.ph, nl_part, s_jnl, tidx, tbeta);
    else nonlocal_current<T>(a, L.v, L.ph, nl_part, s_jnl);
  }
  reduce_obs<T>(os, qo, a.dV, s_jnl, red, a.obs + (size_t)orb * 8);
}

template <typename T, int MODE, bool PER, bool DBUF, int OBS, bool IP = false, int GEOM = 0>
cudaError_t launch_cell(const OrbArgs<T>& a, typename Cplx<T>::type* scratch, size_t smem, int nt,
                        cudaStream_t s) {
  auto kern = k_cell<T, MODE, PER, DBUF, OBS, IP, GEOM>;
  // Shared-memory carveout: just enough shared memory for the CTAs that can be resident (registers,
  // threads and the footprint allow), the rest of the unified storage left as L1 for the reads that
  // stay global (the input orbital of every stage, the potential, the projector tables).  Computed
  // once per kernel and launch shape.
  static size_t last_smem = 0;
  static int last_nt = 0, carve = -1;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (carve < 0 || last_smem != smem || last_nt != nt) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, nt, smem);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    const size_t per_sm = 228 * 1024, need = (size_t)(nb > 0 ? nb : 1) * (smem + fa.sharedSizeBytes + 1024);
    int pct = (int)((need * 100 + per_sm - 1) / per_sm);
    carve = pct > 100 ? 100 : pct;
    last_smem = smem;
    last_nt = nt;
  }
  e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, carve);
  if (e != cudaSuccess) return e;
  kern<<<a.ncell * a.nk * a.norb, nt, smem, s>>>(a, scratch);
  return cudaGetLastError();
}

template <typename T, int MODE, int OBS>
cudaError_t dispatch(const OrbArgs<T>& a, typename Cplx<T>::type* scratch, cudaStream_t s) {
  const bool dbuf = cell_smem_bytes<T>(a.nz, a.pstride, a.nsph, a.natom, true) <= kSmemLimit;
  if (!dbuf && !scratch) return cudaErrorInvalidValue;
  const size_t smem = cell_smem_bytes<T>(a.nz, a.pstride, a.nsph, a.natom, dbuf);
  const int items = a.nx * a.ny * a.nseg;
  int nt = ((items + 31) / 32) * 32;
  if (nt > kNTof<T>()) nt = kNTof<T>();
  if (a.periodic)
    return dbuf ? launch_cell<T, MODE, true, true, OBS>(a, scratch, smem, nt, s)
                : launch_cell<T, MODE, true, false, OBS>(a, scratch, smem, nt, s);
  return dbuf ? launch_cell<T, MODE, false, true, OBS>(a, scratch, smem, nt, s)
              : launch_cell<T, MODE, false, false, OBS>(a, scratch, smem, nt, s);
}

// The built-in geometry (1 or 2) of a's grid for the Taylor stages of cell_variant 2, or 0: periodic,
// planes unpadded, two shared-memory copies, the column split of cell_split.
template <typename T, int GEOM>
bool geom_is(const OrbArgs<T>& a) {
  using G = GeomT<T, GEOM>;
  return a.periodic && a.nx == G::NX && a.ny == G::NY && a.nz == G::NZ && a.pstride == G::NXY &&
         a.zlen == G::ZL && a.nseg == G::NSEG && a.natom < 32768 &&
         cell_smem_bytes_geom<T>(a.nx, a.ny, a.nz, a.pstride, a.nsph, a.natom, false) <= kSmemLimit;
}

template <typename T>
int cell_geom(const OrbArgs<T>& a) {
  if (geom_is<T, 1>(a)) return 1;
  if (geom_is<T, 2>(a)) return 2;
  return 0;
}

// Taylor stages with a built-in geometry (cell_variant 2).
template <typename T, int OBS>
cudaError_t dispatch_geom(const OrbArgs<T>& a, cudaStream_t s) {
  const int g = cell_geom<T>(a);
  if (g == 0) return cudaErrorInvalidValue;
  const size_t smem = cell_smem_bytes_geom<T>(a.nx, a.ny, a.nz, a.pstride, a.nsph, a.natom, false);
  const int items = sizeof(T) == 4 ? (g == 1 ? GeomP<1>::NP * GeomP<1>::NSEG : GeomP<2>::NP * GeomP<2>::NSEG)
                                   : a.nx * a.ny * a.nseg;
  int nt = ((items + 31) / 32) * 32;
  const int ntmax = sizeof(T) == 4 ? kNTpair : kNTof<T>();
  if (nt > ntmax) nt = ntmax;
  if (sizeof(T) == 4 && a.natom > 0) nt += 32 * kProjWarpsGeom;   // the projecting warps (see k_cell)
  return g == 1 ? launch_cell<T, 1, true, true, OBS, false, 1>(a, nullptr, smem, nt, s)
                : launch_cell<T, 1, true, true, OBS, false, 2>(a, nullptr, smem, nt, s);
}

// Taylor stages of an FP32 built-in geometry swept in place, two points per thread (cell_variant 3).
template <typename T, int OBS>
cudaError_t dispatch_geom_ip(const OrbArgs<T>& a, cudaStream_t s) {
  if constexpr (sizeof(T) != 4) {
    return cudaErrorInvalidValue;
  } else {
    const int g = cell_geom<T>(a);
    if (g == 0) return cudaErrorInvalidValue;
    const size_t smem = cell_smem_bytes_geom<T>(a.nx, a.ny, a.nz, a.pstride, a.nsph, a.natom, true);
    if (smem > kSmemLimit) return cudaErrorInvalidValue;
    const int np = g == 1 ? GeomP<1>::NP : GeomP<2>::NP;
    const int nt = ((np + 31) / 32) * 32;
    if (nt > kNTpairIP) return cudaErrorInvalidValue;
    return g == 1 ? launch_cell<T, 1, true, false, OBS, true, 1>(a, nullptr, smem, nt, s)
                  : launch_cell<T, 1, true, false, OBS, true, 2>(a, nullptr, smem, nt, s);
  }
}

// Taylor stages with the in-place sweep (cell_variant 1).
template <typename T, int OBS>
cudaError_t dispatch_ip(const OrbArgs<T>& a, cudaStream_t s) {
  const size_t smem = cell_smem_bytes_ip<T>(a.nx, a.ny, a.nz, a.pstride, a.nsph, a.natom, a.periodic != 0);
  const int nt = ((a.nx * a.ny + 31) / 32) * 32;
  if (a.periodic) return launch_cell<T, 1, true, false, OBS, true>(a, nullptr, smem, nt, s);
  return launch_cell<T, 1, false, false, OBS, true>(a, nullptr, smem, nt, s);
}

}  // namespace

template <typename T>
bool smem_orbital_ip_ok(int nx, int ny, int nz, int pstride, int nsph, int natom, int periodic) {
  return nx * ny <= kNTip && cell_smem_bytes_ip<T>(nx, ny, nz, pstride, nsph, natom, periodic != 0) <= kSmemLimit;
}

template <typename T>
bool smem_orbital_fits(int nz, int pstride, int nsph, int natom) {
  return cell_smem_bytes<T>(nz, pstride, nsph, natom, false) <= kSmemLimit;
}

template <typename T>
bool smem_orbital_needs_scratch(int nz, int pstride, int nsph, int natom) {
  return cell_smem_bytes<T>(nz, pstride, nsph, natom, true) > kSmemLimit;
}

void cell_split(int nx, int ny, int nz, int elem_bytes, int* nseg, int* zlen) {
  const int ncol = nx * ny;
  int s = (elem_bytes == 8 ? kSegThreads<float>() : kSegThreads<double>()) / ncol;
  if (s < 1) s = 1;
  if (s > nz) s = nz;
  *zlen = (nz + s - 1) / s;
  *nseg = (nz + *zlen - 1) / *zlen;
}

template <typename T>
cudaError_t launch_smem_orbital(const OrbArgs<T>& a, int mode, typename Cplx<T>::type* scratch,
                                cudaStream_t s) {
  if (mode == 0) return dispatch<T, 0, 0>(a, scratch, s);
  if (mode == 1) {
    if (a.cell_variant == 1) {
      if (!smem_orbital_ip_ok<T>(a.nx, a.ny, a.nz, a.pstride, a.nsph, a.natom, a.periodic))
        return cudaErrorInvalidValue;
      if (!a.obs) return dispatch_ip<T, 0>(a, s);
      return a.obs_at_start ? dispatch_ip<T, 2>(a, s) : dispatch_ip<T, 1>(a, s);
    }
    if (a.cell_variant == 2) {
      if (!a.obs) return dispatch_geom<T, 0>(a, s);
      return a.obs_at_start ? dispatch_geom<T, 2>(a, s) : dispatch_geom<T, 1>(a, s);
    }
    if (a.cell_variant == 3) {
      if (!a.obs) return dispatch_geom_ip<T, 0>(a, s);
      return a.obs_at_start ? dispatch_geom_ip<T, 2>(a, s) : dispatch_geom_ip<T, 1>(a, s);
    }
    if (!a.obs) return dispatch<T, 1, 0>(a, scratch, s);
    return a.obs_at_start ? dispatch<T, 1, 2>(a, scratch, s) : dispatch<T, 1, 1>(a, scratch, s);
  }
  return dispatch<T, 2, 1>(a, scratch, s);
}

template <typename T>
bool smem_orbital_geom_ok(int nx, int ny, int nz, int pstride, int nsph, int natom, int periodic, int nseg, int zlen) {
  OrbArgs<T> a{};
  a.nx = nx; a.ny = ny; a.nz = nz; a.pstride = pstride; a.nsph = nsph; a.natom = natom;
  a.periodic = periodic; a.nseg = nseg; a.zlen = zlen;
  return cell_geom<T>(a) != 0;
}

template <typename T>
bool smem_orbital_geom_ip_ok(int nx, int ny, int nz, int pstride, int nsph, int natom, int periodic, int nseg,
                             int zlen) {
  if (sizeof(T) != 4 || !smem_orbital_geom_ok<T>(nx, ny, nz, pstride, nsph, natom, periodic, nseg, zlen)) return false;
  return cell_smem_bytes_geom<T>(nx, ny, nz, pstride, nsph, natom, true) <= kSmemLimit;
}

template bool smem_orbital_geom_ip_ok<float>(int, int, int, int, int, int, int, int, int);
template bool smem_orbital_geom_ip_ok<double>(int, int, int, int, int, int, int, int, int);
template bool smem_orbital_geom_ok<float>(int, int, int, int, int, int, int, int, int);
template bool smem_orbital_geom_ok<double>(int, int, int, int, int, int, int, int, int);
template bool smem_orbital_ip_ok<float>(int, int, int, int, int, int, int);
template bool smem_orbital_ip_ok<double>(int, int, int, int, int, int, int);
template bool smem_orbital_fits<float>(int, int, int, int);
template bool smem_orbital_fits<double>(int, int, int, int);
template bool smem_orbital_needs_scratch<float>(int, int, int, int);
template bool smem_orbital_needs_scratch<double>(int, int, int, int);
template cudaError_t launch_smem_orbital<float>(const OrbArgs<float>&, int, float2*, cudaStream_t);
template cudaError_t launch_smem_orbital<double>(const OrbArgs<double>&, int, double2*, cudaStream_t);

}  // namespace tdks
