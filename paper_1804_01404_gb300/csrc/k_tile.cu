// Large isolated grids: one Horner stage (or one H application) per launch, tiled in x-y and
// marching in z.
//
// A CTA owns a TX x TY column tile of one orbital and walks z = 0..nz-1.  Planes of the tile plus
// a 4-point halo in x and y arrive in a ring of NS shared-memory slots by TMA
// (cp.async.bulk.tensor.4d); coordinates outside the box are zero-filled by the copy engine, which
// is exactly the vacuum boundary of an isolated system (Sec. 2.1).  The CTA is warp-specialised:
// one producer warp issues the plane copies (completion on a "full" mbarrier per slot) and refills
// a slot once every consumer warp has released it (an "empty" mbarrier per slot); eight consumer
// warps each own two rows of the tile and keep the nine z-values of their columns in registers, so
// each plane is read from HBM once, the 16 in-plane neighbours come from shared memory at
// compile-time offsets, and no block-wide barrier is taken per plane.  The nonlocal projectors are
// applied by the separate gather/scatter kernels below.  Every mbarrier wait gives up after a
// bounded number of polls: the CTA then sets the context error flag, the producer drains its own
// copies (again bounded) and all warps exit.
#include <cstring>

#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "tdks_internal.h"
#include "warp_sum.cuh"

namespace tdks {

namespace {

constexpr int TX = 32, TY = 16, NS = 8;
constexpr int SX = TX + 8, SY = TY + 8;          // slot shape (complex elements)
constexpr int RPT = 2;                           // tile rows per consumer thread
constexpr int NCW = TX * TY / RPT / 32;          // consumer warps
constexpr int NT = (NCW + 1) * 32;               // + one producer warp
constexpr long long kSpinLimit = 1LL << 22;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool volatile_abort(int* flag) {
  return *reinterpret_cast<volatile int*>(flag) != 0;
}

// bounded wait; returns false on timeout
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, long long limit = kSpinLimit) {
  for (long long i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            int c3, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2),
        "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2),
        "r"(smem_u32(bar))
      : "memory");
}

// L2 prefetch of one box of a tensor map (no shared memory, no completion to wait for).
__device__ __forceinline__ void tma_prefetch_4d(const CUtensorMap* map, int c0, int c1, int c2, int c3) {
  asm volatile("cp.async.bulk.prefetch.tensor.4d.L2.global.tile [%0, {%1, %2, %3, %4}];"
               ::"l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
               : "memory");
}

// Producer of a plane ring: one thread issues the TMA copy of every plane z = -4 .. nz+3 of the
// (SXx x SYx)-element window whose interior starts at (x0, y0), refilling a slot once all consumer
// warps have arrived on its "empty" barrier.  The ring alone keeps only NSx - 5 planes in flight (the
// consumers hold five); with pf > 0 the producer also asks L2 for the plane pf ahead of each copy,
// and, given pmap (the Horner base psi, interior box), for the psi plane the consumers reach about
// pf planes later, so DRAM sees enough requests in flight without more shared memory.  On a
// timed-out wait it raises the abort flag and the error word; in every case it waits (bounded) for
// its own most recent copies before returning, so no copy is in flight when the CTA exits.
// limit: polls per wait (the drain at the end always uses the full kSpinLimit, so copies in flight
// land before the CTA exits).  stop_after >= 0 issues only that many planes (the timeout test: the
// consumers then wait for a plane that never comes and must give up).
// Side planes (optional): with smap, slot j also receives the interior box of the potential (a 3D
// map of floats) at plane j - 4, the plane whose stencil uses slot j as its centre, into sring; with
// qmap, the interior box of the Horner base psi at the same plane into qring.  Both complete on the
// slot's "full" barrier, so the stencil warps read V and psi from shared memory.
template <typename C, int NSx, int SXx, int SYx>
__device__ __forceinline__ void tile_producer(const CUtensorMap* map, const CUtensorMap* pmap, int pf,
                                              C* ring, unsigned long long* full,
                                              unsigned long long* empty, int* abort_flag, int* err,
                                              int x0, int y0, int orb, int nplanes, long long limit,
                                              int stop_after, const CUtensorMap* smap = nullptr,
                                              float* sring = nullptr, unsigned sbytes = 0,
                                              const CUtensorMap* qmap = nullptr, C* qring = nullptr,
                                              unsigned qbytes = 0) {
  constexpr int E = sizeof(C) / 8;
  constexpr unsigned kSlotBytes = SXx * SYx * sizeof(C);
  const int nz = nplanes - 8;
  int issued = 0;
  bool ok = true;
  for (int j = 0; j < nplanes; ++j) {
    if (stop_after >= 0 && j >= stop_after) break;
    const int slot = j % NSx;
    if (j >= NSx && !mbar_wait(&empty[slot], ((j / NSx) - 1) & 1, limit)) { ok = false; break; }
    if (volatile_abort(abort_flag)) { ok = false; break; }
    if (pf > 0) {
      const int zp = j + pf - 4;                   // plane of the ring source pf ahead
      if (zp >= 0 && zp < nz) tma_prefetch_4d(map, E * (x0 - 4), y0 - 4, zp, orb);
      const int zq = j + pf - NSx - 4;             // psi plane the consumers reach ~pf planes later
      if (pmap && zq >= 0 && zq < nz) tma_prefetch_4d(pmap, E * x0, y0, zq, orb);
    }
    mbar_expect_tx(&full[slot], kSlotBytes + (smap ? sbytes : 0u) + (qmap ? qbytes : 0u));
    tma_load_4d(ring + slot * SXx * SYx, map, E * (x0 - 4), y0 - 4, j - 4, orb, &full[slot]);
    if (smap) tma_load_3d(sring + slot * (sbytes / sizeof(float)), smap, x0, y0, j - 4, &full[slot]);
    if (qmap) tma_load_4d(qring + slot * (qbytes / sizeof(C)), qmap, E * x0, y0, j - 4, orb, &full[slot]);
    issued = j + 1;
  }
  if (!ok) {
    atomicExch(abort_flag, 1);
    atomicExch(err, (int)TDKS_ETIMEOUT);
  }
  for (int j = (issued > NSx ? issued - NSx : 0); j < issued; ++j) mbar_wait(&full[j % NSx], (j / NSx) & 1);
}

// Complex-by-real arithmetic of the stencil.  K is the coefficient operand: a duplicated pair for the
// packed FP32 instructions (so one register pair per coefficient is built once, outside the loop),
// a scalar for FP64.
template <typename T> struct TM;
template <> struct TM<float> {
  using C = float2;
  using K = float2;
  static __device__ __forceinline__ K k(float s) { return make_float2(s, s); }
  static __device__ __forceinline__ C add(C a, C b) { return __fadd2_rn(a, b); }
  static __device__ __forceinline__ C fma(K s, C a, C acc) { return __ffma2_rn(s, a, acc); }
};
template <> struct TM<double> {
  using C = double2;
  using K = double;
  static __device__ __forceinline__ K k(double s) { return s; }
  static __device__ __forceinline__ C add(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
  static __device__ __forceinline__ C fma(K s, C a, C acc) {
    return C{__fma_rn(s, a.x, acc.x), __fma_rn(s, a.y, acc.y)};
  }
};

// MODE 0: out = H_loc v.  MODE 1: out = psi + (-i coef) H_loc v.   (H_loc: everything but V_NL;
// q = 0 for isolated systems.)
template <typename T, int MODE, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_tile(const __grid_constant__ CUtensorMap vmap,
                                             const __grid_constant__ CUtensorMap pmap, TileArgs<T> a) {
  using C = typename Cplx<T>::type;
  using M = TM<T>;
  extern __shared__ unsigned char smem_raw[];
  // TMA destinations 128-byte aligned (the launch requests 128 spare bytes)
  C* ring = reinterpret_cast<C*>((reinterpret_cast<size_t>(smem_raw) + 127) & ~size_t(127));
  __shared__ __align__(8) unsigned long long full[NS], empty[NS];
  __shared__ int s_abort;

  const int tilesx = (a.nx + TX - 1) / TX;
  const int bx = blockIdx.x % tilesx, by = blockIdx.x / tilesx;
  const int orb = blockIdx.y;
  const int x0 = bx * TX, y0 = by * TY;
  const int nplanes = a.nz + 8;                    // z = -4 .. nz+3
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int i = 0; i < NS; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], NCW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == NCW) {
    if (lane == 0)
      tile_producer<C, NS, SX, SY>(&vmap, MODE == 1 ? &pmap : nullptr, a.prefetch, ring, full, empty, &s_abort,
                                   a.err, x0, y0, orb, nplanes, a.wait_limit, a.stop_after);
    return;
  }

  // ---------------- consumer warps: thread (tx, ty) owns rows ty and ty + TY/2 of column tx
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int x = x0 + tx;
  const int yr[RPT] = {y0 + ty, y0 + ty + TY / 2};
  const int own[RPT] = {(ty + 4) * SX + (tx + 4), (ty + TY / 2 + 4) * SX + (tx + 4)};
  bool inside[RPT];
  const size_t plane = (size_t)a.nx * a.ny;
  const size_t obase = (size_t)orb * plane * a.nz;
  size_t col[RPT];
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    inside[r] = (x < a.nx) && (yr[r] < a.ny);
    col[r] = (size_t)yr[r] * a.nx + x;
  }
  // c2y[m] = ry c2x[m] and c2z[m] = rz c2x[m] (the axes differ only by 1/h^2): one coefficient per
  // neighbour distance, S = (diag + V) u + sum_m c2x[m] (X_m + ry Y_m + rz Z_m)
  using K = typename M::K;
  const K ry = M::k(a.ry), rz = M::k(a.rz);
  bool timeout = false;
  C w[RPT][9];
  // window planes j = 0..7 (z = -4..3); planes 0..3 are released right away
  for (int j = 0; j < 8; ++j) {
    if (!timeout && !mbar_wait(&full[j % NS], (j / NS) & 1, a.wait_limit)) timeout = true;
#pragma unroll
    for (int r = 0; r < RPT; ++r) w[r][j] = ring[(j % NS) * SX * SY + own[r]];
    if (j < 4) {
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[j % NS]);
    }
  }
  const T coef = a.coef;
  // psi one plane ahead; V (L2-resident, shared by all orbitals) VD planes ahead, two when the
  // register cap leaves room for it
  constexpr int VD = MINB <= 2 ? 2 : 1;
  C pnext[RPT];
  T vq[RPT][VD];
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    pnext[r] = C{0, 0};
#pragma unroll
    for (int d = 0; d < VD; ++d) vq[r][d] = 0;
    if (inside[r]) {
      if (MODE == 1) pnext[r] = a.psi[obase + col[r]];
#pragma unroll
      for (int d = 0; d < VD; ++d)
        if (d < a.nz) vq[r][d] = a.V[(size_t)d * plane + col[r]];
    }
  }
  for (int z = 0; z < a.nz; ++z) {
    if (timeout || volatile_abort(&s_abort)) break;
    const int jc = z + 4;
    const int jn = z + 8;
    if (!mbar_wait(&full[jn % NS], (jn / NS) & 1, a.wait_limit)) { timeout = true; break; }
    const C* sbase = ring + (jc % NS) * SX * SY;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      w[r][8] = ring[(jn % NS) * SX * SY + own[r]];
      const C pv = pnext[r];
      const T vv = vq[r][0];
#pragma unroll
      for (int d = 0; d + 1 < VD; ++d) vq[r][d] = vq[r][d + 1];
      if (inside[r] && z + 1 < a.nz) {             // prefetch psi of plane z+1 and V of plane z+VD
        if (MODE == 1) pnext[r] = a.psi[obase + (size_t)(z + 1) * plane + col[r]];
        if (z + VD < a.nz) vq[r][VD - 1] = a.V[(size_t)(z + VD) * plane + col[r]];
      }
      const C* sp = sbase + own[r];
      C S = M::fma(M::k(a.diag + vv), w[r][4], C{0, 0});
#pragma unroll
      for (int m = 1; m <= 4; ++m)
        S = M::fma(M::k(a.c2x[m]), M::fma(rz, M::add(w[r][4 + m], w[r][4 - m]),
                                          M::fma(ry, M::add(sp[m * SX], sp[-m * SX]), M::add(sp[m], sp[-m]))), S);
      if (inside[r]) {
        const size_t o = obase + (size_t)z * plane + col[r];
        if (MODE == 1) a.out[o] = M::fma(M::k(coef), C{S.y, -S.x}, pv);   // psi + (-i coef) H v
        else a.out[o] = S;
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) w[r][j] = w[r][j + 1];
    }
    __syncwarp();                                  // this warp is done with plane jc
    if (lane == 0) mbar_arrive(&empty[jc % NS]);
  }
  if (timeout) {
    atomicExch(&s_abort, 1);
    atomicExch(a.err, (int)TDKS_ETIMEOUT);
  }
}

// FP32 variant with 2 x 2 register blocking.  Shared-memory bandwidth, not HBM, limits the kernel
// above on this GPU: it reads 17 complex values (136 B) from shared memory per output point,
// while the shared-memory / HBM bandwidth ratio leaves room for about 90 B per point at full HBM
// speed.  Here each consumer thread owns two adjacent columns of two adjacent rows: one 16-byte
// load brings both columns of a row, the x-neighbours of a row pair come from four such loads,
// and the y-neighbours are shared by the two rows, so shared-memory traffic falls to 72 B per
// point and the instruction count roughly halves.  A warp covers 16 column pairs x 2 row pairs of
// a 32 x (4 NCW) tile.  The z loop is unrolled by the window length 9, so the register window
// rotates by renaming instead of moving values.
// ROWS = 1: the same with one row per thread (2 x 1 points, 104 B of shared memory per point and
// about half the registers), a 32 x (2 NCW) tile.
template <int NCW, int ROWS = 2>
struct B4 {
  static constexpr int TX = 32, TY = 2 * ROWS * NCW, NS = 8;
  static constexpr int SX = TX + 8, SY = TY + 8;
  static constexpr int NT = (NCW + 1) * 32;
  // resident CTAs per SM the register budget allows
  static constexpr int MINB = ROWS == 1 ? (NCW == 4 ? 4 : 2) : (NCW == 4 ? 2 : 1);
};

__device__ __forceinline__ float4 lds4(const float2* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float2 lo(float4 q) { return make_float2(q.x, q.y); }
__device__ __forceinline__ float2 hi(float4 q) { return make_float2(q.z, q.w); }
__device__ __forceinline__ float2 sum2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fma2s(float s, float2 a, float2 acc) {
  return __ffma2_rn(make_float2(s, s), a, acc);
}

// SV: the potential (and, for a Horner stage, psi) of each plane arrive by TMA beside the orbital
// plane (side rings after the orbital ring) instead of as per-thread global loads.
template <int MODE, int NCW, int ROWS = 2, bool SV = false>
__global__ void __launch_bounds__(B4<NCW, ROWS>::NT, B4<NCW, ROWS>::MINB)
    k_tile4(const __grid_constant__ CUtensorMap vmap, const __grid_constant__ CUtensorMap pmap,
            const __grid_constant__ CUtensorMap potmap, TileArgs<float> a) {
  using G = B4<NCW, ROWS>;
  static_assert(ROWS == 1 || ROWS == 2, "one or two rows per thread");
  constexpr int TX = G::TX, TY = G::TY, NS = G::NS, SX = G::SX, SY = G::SY, SS = SX * SY;
  extern __shared__ unsigned char smem_raw[];
  float2* ring = reinterpret_cast<float2*>((reinterpret_cast<size_t>(smem_raw) + 127) & ~size_t(127));
  float* sring = reinterpret_cast<float*>(ring + NS * SS);        // [NS][TY][TX] potential
  float2* qring = reinterpret_cast<float2*>(sring + NS * TX * TY);  // [NS][TY][TX] psi (MODE 1)
  __shared__ __align__(8) unsigned long long full[NS], empty[NS];
  __shared__ int s_abort;

  const int tilesx = (a.nx + TX - 1) / TX;
  const int x0 = (blockIdx.x % tilesx) * TX, y0 = (blockIdx.x / tilesx) * TY;
  const int orb = blockIdx.y;
  const int nz = a.nz;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int i = 0; i < NS; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], NCW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (warp == NCW) {
    if (lane == 0 && SV)
      tile_producer<float2, NS, SX, SY>(&vmap, nullptr, a.prefetch, ring, full, empty, &s_abort, a.err, x0, y0,
                                        orb, nz + 8, a.wait_limit, a.stop_after, &potmap, sring,
                                        TX * TY * sizeof(float), MODE == 1 ? &pmap : nullptr, qring,
                                        TX * TY * sizeof(float2));
    else if (lane == 0)
      tile_producer<float2, NS, SX, SY>(&vmap, MODE == 1 ? &pmap : nullptr, a.prefetch, ring, full, empty,
                                        &s_abort, a.err, x0, y0, orb, nz + 8, a.wait_limit, a.stop_after);
    return;
  }

  const int lx = 2 * (lane & 15);                  // tile column of the pair (even)
  const int ly = 2 * ROWS * warp + ROWS * (lane >> 4);   // first of the thread's tile rows
  const int x = x0 + lx, y = y0 + ly;
  // nx is even, so both columns of a pair are inside together
  const bool in0 = (x < a.nx) && (y < a.ny), in1 = ROWS == 2 && (x < a.nx) && (y + 1 < a.ny);
  const int o0 = (ly + 4) * SX + (lx + 4);         // slot offset of the row-0 pair (16-byte aligned)
  const int o1 = o0 + SX;
  const size_t plane = (size_t)a.nx * a.ny;
  const size_t g0 = (size_t)orb * plane * nz + (size_t)y * a.nx + x;   // row-0 pair, plane z = 0
  const size_t v0 = (size_t)y * a.nx + x;

  float2 w0a[9], w0b[9], w1a[9], w1b[9];
  bool timeout = false;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    if (!timeout && !mbar_wait(&full[j % NS], (j / NS) & 1, a.wait_limit)) timeout = true;
    const float4 p0 = lds4(ring + (j % NS) * SS + o0);
    w0a[j] = lo(p0); w0b[j] = hi(p0);
    if (ROWS == 2) {
      const float4 p1 = lds4(ring + (j % NS) * SS + o1);
      w1a[j] = lo(p1); w1b[j] = hi(p1);
    }
    if (j < 4) {
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[j % NS]);
    }
  }
  // c2y[m] = ry c2x[m] and c2z[m] = rz c2x[m] for every m (the axes differ only by 1/h^2), so each
  // neighbour distance costs one coefficient: S += c2x[m] (X_m + ry Y_m + rz Z_m)
  const float2 c1 = make_float2(a.c2x[1], a.c2x[1]), c2 = make_float2(a.c2x[2], a.c2x[2]);
  const float2 c3 = make_float2(a.c2x[3], a.c2x[3]), c4 = make_float2(a.c2x[4], a.c2x[4]);
  const float2 ry = make_float2(a.ry, a.ry), rz = make_float2(a.rz, a.rz);
  const float diag = a.diag, coef = a.coef;
  float2 vn0 = make_float2(0.f, 0.f), vn1 = vn0;
  float4 pn0 = make_float4(0.f, 0.f, 0.f, 0.f), pn1 = pn0;
  if (!SV && in0) {
    vn0 = *reinterpret_cast<const float2*>(a.V + v0);
    if (MODE == 1) pn0 = *reinterpret_cast<const float4*>(a.psi + g0);
  }
  if (!SV && in1) {
    vn1 = *reinterpret_cast<const float2*>(a.V + v0 + a.nx);
    if (MODE == 1) pn1 = *reinterpret_cast<const float4*>(a.psi + g0 + a.nx);
  }

  for (int zb = 0; zb < nz && !timeout; zb += 9) {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int z = zb + k;
      if (z >= nz) break;
      if (volatile_abort(&s_abort)) { timeout = true; break; }
      const int jc = z + 4, jn = z + 8;
      // register slots of planes z .. z+8 (z multiple-of-9 aligned at zb)
      const int rc = (k + 4) % 9, rn = (k + 8) % 9;
      if (!mbar_wait(&full[jn % NS], (jn / NS) & 1, a.wait_limit)) { timeout = true; break; }
      {
        const float2* sn = ring + (jn % NS) * SS;
        const float4 p0 = lds4(sn + o0);
        w0a[rn] = lo(p0); w0b[rn] = hi(p0);
        if (ROWS == 2) {
          const float4 p1 = lds4(sn + o1);
          w1a[rn] = lo(p1); w1b[rn] = hi(p1);
        }
      }
      const float2* sc = ring + (jc % NS) * SS;
      float2 V0 = vn0, V1 = vn1;
      float4 P0 = pn0, P1 = pn1;
      if (SV) {                                    // this plane's V and psi from the side rings
        V0 = *reinterpret_cast<const float2*>(sring + (jc % NS) * TX * TY + ly * TX + lx);
        if (MODE == 1) P0 = *reinterpret_cast<const float4*>(qring + (jc % NS) * TX * TY + ly * TX + lx);
        if (ROWS == 2) {
          V1 = *reinterpret_cast<const float2*>(sring + (jc % NS) * TX * TY + (ly + 1) * TX + lx);
          if (MODE == 1) P1 = *reinterpret_cast<const float4*>(qring + (jc % NS) * TX * TY + (ly + 1) * TX + lx);
        }
      } else if (z + 1 < nz) {                     // prefetch the next plane's V and psi
        const size_t dz = (size_t)(z + 1) * plane;
        if (in0) {
          vn0 = *reinterpret_cast<const float2*>(a.V + v0 + dz);
          if (MODE == 1) pn0 = *reinterpret_cast<const float4*>(a.psi + g0 + dz);
        }
        if (in1) {
          vn1 = *reinterpret_cast<const float2*>(a.V + v0 + a.nx + dz);
          if (MODE == 1) pn1 = *reinterpret_cast<const float4*>(a.psi + g0 + a.nx + dz);
        }
      }
      // The three axes are summed in turn (z from the register window, then y, then x from shared
      // memory), with a compiler fence between the phases so that at most eight 16-byte loads are in
      // registers next to the window: S = (diag + V) u + rz Tz + ry Ty + Tx, T_a = sum_m c_m (pair sums).
#define TDKS_AXIS(T, l1, r1, l2, r2, l3, r3, l4, r4)                                           \
  T = __ffma2_rn(c4, sum2(l4, r4), __ffma2_rn(c3, sum2(l3, r3),                                  \
      __ffma2_rn(c2, sum2(l2, r2), __ffma2_rn(c1, sum2(l1, r1), T))));
#define TDKS_ZPART(S, dv, W)                                                                     \
  {                                                                                              \
    float2 Tz = make_float2(0.f, 0.f);                                                           \
    TDKS_AXIS(Tz, W[(k + 3) % 9], W[(k + 5) % 9], W[(k + 2) % 9], W[(k + 6) % 9],                \
              W[(k + 1) % 9], W[(k + 7) % 9], W[k % 9], W[(k + 8) % 9])                          \
    S = __ffma2_rn(rz, Tz, fma2s(dv, W[rc], make_float2(0.f, 0.f)));                             \
  }
      float2 S0a, S0b, S1a = make_float2(0.f, 0.f), S1b = S1a;
      TDKS_ZPART(S0a, diag + V0.x, w0a)
      TDKS_ZPART(S0b, diag + V0.y, w0b)
      if (ROWS == 2) {
        TDKS_ZPART(S1a, diag + V1.x, w1a)
        TDKS_ZPART(S1b, diag + V1.y, w1b)
      }
      asm volatile("" ::: "memory");
      if (ROWS == 1) {
        // y-neighbour pairs: rows ly-1 .. ly-4 and ly+1 .. ly+4
        const float4 Ym1 = lds4(sc + o0 - SX), Ym2 = lds4(sc + o0 - 2 * SX), Ym3 = lds4(sc + o0 - 3 * SX), Ym4 = lds4(sc + o0 - 4 * SX);
        const float4 Yp1 = lds4(sc + o0 + SX), Yp2 = lds4(sc + o0 + 2 * SX), Yp3 = lds4(sc + o0 + 3 * SX), Yp4 = lds4(sc + o0 + 4 * SX);
        float2 T0a = make_float2(0.f, 0.f), T0b = T0a;
        TDKS_AXIS(T0a, lo(Ym1), lo(Yp1), lo(Ym2), lo(Yp2), lo(Ym3), lo(Yp3), lo(Ym4), lo(Yp4))
        TDKS_AXIS(T0b, hi(Ym1), hi(Yp1), hi(Ym2), hi(Yp2), hi(Ym3), hi(Yp3), hi(Ym4), hi(Yp4))
        S0a = __ffma2_rn(ry, T0a, S0a);
        S0b = __ffma2_rn(ry, T0b, S0b);
      } else {
        // y-neighbour pairs: rows ly-1 .. ly-4 and ly+2 .. ly+5
        const float4 Ym1 = lds4(sc + o0 - SX), Ym2 = lds4(sc + o0 - 2 * SX), Ym3 = lds4(sc + o0 - 3 * SX), Ym4 = lds4(sc + o0 - 4 * SX);
        const float4 Yp1 = lds4(sc + o1 + SX), Yp2 = lds4(sc + o1 + 2 * SX), Yp3 = lds4(sc + o1 + 3 * SX), Yp4 = lds4(sc + o1 + 4 * SX);
        float2 T0a = make_float2(0.f, 0.f), T0b = T0a, T1a = T0a, T1b = T0a;
        TDKS_AXIS(T0a, lo(Ym1), w1a[rc], lo(Ym2), lo(Yp1), lo(Ym3), lo(Yp2), lo(Ym4), lo(Yp3))
        TDKS_AXIS(T0b, hi(Ym1), w1b[rc], hi(Ym2), hi(Yp1), hi(Ym3), hi(Yp2), hi(Ym4), hi(Yp3))
        TDKS_AXIS(T1a, w0a[rc], lo(Yp1), lo(Ym1), lo(Yp2), lo(Ym2), lo(Yp3), lo(Ym3), lo(Yp4))
        TDKS_AXIS(T1b, w0b[rc], hi(Yp1), hi(Ym1), hi(Yp2), hi(Ym2), hi(Yp3), hi(Ym3), hi(Yp4))
        S0a = __ffma2_rn(ry, T0a, S0a);
        S0b = __ffma2_rn(ry, T0b, S0b);
        S1a = __ffma2_rn(ry, T1a, S1a);
        S1b = __ffma2_rn(ry, T1b, S1b);
      }
      asm volatile("" ::: "memory");
      {
        // x-neighbour pairs of row 0 (offsets -4/-3, -2/-1, +2/+3, +4/+5)
        const float4 Am2 = lds4(sc + o0 - 4), Am1 = lds4(sc + o0 - 2), Ap1 = lds4(sc + o0 + 2), Ap2 = lds4(sc + o0 + 4);
        TDKS_AXIS(S0a, hi(Am1), w0b[rc], lo(Am1), lo(Ap1), hi(Am2), hi(Ap1), lo(Am2), lo(Ap2))
        TDKS_AXIS(S0b, w0a[rc], lo(Ap1), hi(Am1), hi(Ap1), lo(Am1), lo(Ap2), hi(Am2), hi(Ap2))
      }
      if (ROWS == 2) {
        // row 1
        const float4 Am2 = lds4(sc + o1 - 4), Am1 = lds4(sc + o1 - 2), Ap1 = lds4(sc + o1 + 2), Ap2 = lds4(sc + o1 + 4);
        TDKS_AXIS(S1a, hi(Am1), w1b[rc], lo(Am1), lo(Ap1), hi(Am2), hi(Ap1), lo(Am2), lo(Ap2))
        TDKS_AXIS(S1b, w1a[rc], lo(Ap1), hi(Am1), hi(Ap1), lo(Am1), lo(Ap2), hi(Am2), hi(Ap2))
      }
      __syncwarp();                                // this warp is done with plane jc
      if (lane == 0) mbar_arrive(&empty[jc % NS]);
#undef TDKS_ZPART
#undef TDKS_AXIS
      const size_t o = g0 + (size_t)z * plane;
      if (MODE == 1) {
        // psi + (-i coef) S = psi + coef (S.y, -S.x)
        const float2 mc = make_float2(coef, -coef);
        const float2 r0a = __ffma2_rn(mc, make_float2(S0a.y, S0a.x), lo(P0));
        const float2 r0b = __ffma2_rn(mc, make_float2(S0b.y, S0b.x), hi(P0));
        const float2 r1a = __ffma2_rn(mc, make_float2(S1a.y, S1a.x), lo(P1));
        const float2 r1b = __ffma2_rn(mc, make_float2(S1b.y, S1b.x), hi(P1));
        if (in0) *reinterpret_cast<float4*>(a.out + o) = make_float4(r0a.x, r0a.y, r0b.x, r0b.y);
        if (ROWS == 2 && in1) *reinterpret_cast<float4*>(a.out + o + a.nx) = make_float4(r1a.x, r1a.y, r1b.x, r1b.y);
      } else {
        if (in0) *reinterpret_cast<float4*>(a.out + o) = make_float4(S0a.x, S0a.y, S0b.x, S0b.y);
        if (ROWS == 2 && in1) *reinterpret_cast<float4*>(a.out + o + a.nx) = make_float4(S1a.x, S1a.y, S1b.x, S1b.y);
      }
    }
  }
  if (timeout) {
    atomicExch(&s_abort, 1);
    atomicExch(a.err, (int)TDKS_ETIMEOUT);
  }
}

// Projections for large grids.  A CTA takes one atom and kOB orbitals, one warp per kOB / 4 of them;
// the lanes stride over the atom's sphere points and each loaded index and beta row serves every
// orbital of the warp, so the index -> value load chain is paid once per point, not once per orbital.
// ec[orb][a][p] = E_p dV sum_i beta_ip v(idx_i)   (isolated: q = 0, no phase)
constexpr int kOB = 16;
template <typename T>
__global__ void __launch_bounds__(128) k_gproject(TileArgs<T> a, const typename Cplx<T>::type* v) {
  using C = typename Cplx<T>::type;
  constexpr int OW = kOB / 4;                      // orbitals per warp
  const int at = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ob = blockIdx.y * kOB + warp * OW;
  const int i0 = a.atom_off[at], i1 = a.atom_off[at + 1];
  T acc[OW][8];
#pragma unroll
  for (int o = 0; o < OW; ++o)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[o][j] = 0;
  for (int i = i0 + lane; i < i1; i += 32) {
    const int idx = a.sph_idx[i];
    T b[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) b[p] = a.sph_beta[4 * i + p];
    C x[OW];
#pragma unroll
    for (int o = 0; o < OW; ++o) x[o] = ob + o < a.norb_tot ? v[(size_t)(ob + o) * a.npts + idx] : C{0, 0};
#pragma unroll
    for (int o = 0; o < OW; ++o)
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        acc[o][2 * p] += b[p] * x[o].x;
        acc[o][2 * p + 1] += b[p] * x[o].y;
      }
  }
  // all OW x 8 sums at once: lane L receives acc[L / 8][L % 8] (Re of projector p on even L, Im on
  // the odd partner)
  static_assert(OW * 8 == 32, "one value per lane");
  const T tot = warp_split_sum<32>(&acc[0][0]);
  const T im = __shfl_xor_sync(0xffffffffu, tot, 1);
  const int o = lane >> 3, p = (lane & 7) >> 1;
  if ((lane & 1) == 0 && ob + o < a.norb_tot) {
    const T sc = a.atomE[at * 4 + p] * a.dV;
    a.ec[((size_t)(ob + o) * a.natom + at) * 4 + p] = C{tot * sc, im * sc};
  }
}

// FP32 projections as a batched dense contraction on the tensor cores.  For one atom the projections of
// all orbitals are the matrix product C = U B: U [orbitals x sphere points] holds the orbitals' values at
// the atom's sphere points (real and imaginary parts as two matrices), B [sphere points x 4] the real
// projectors.  A CTA takes 16 orbitals; its warps walk interleaved steps of 8 sphere points with
// mma.sync m16n8k8 TF32 (the four projectors padded to n = 8), FP32 accumulation, and their partial
// products are added in shared memory in a fixed order.  Each operand is
// split into a TF32 head and a TF32 tail (x = hi + lo, both exact in FP32) and the product is formed
// as hi*hi + hi*lo + lo*hi, which keeps the sum at FP32 accuracy (three TF32 products per step).
// Fragments (PTX ISA, m16n8k8 .tf32): A a0 (row g, col t), a1 (g+8, t), a2 (g, t+4), a3 (g+8, t+4);
// B b0 (row t, col g), b1 (t+4, g); C c0 (g, 2t), c1 (g, 2t+1), c2 (g+8, 2t), c3 (g+8, 2t+1), with
// g = lane / 4 and t = lane % 4.  Rows are orbitals, columns of B and C are projectors.
// kPW (template parameter): warps per CTA, all on the same 16 orbitals, each on every kPW-th step of
// 8 sphere points; the context's tuner picks 2, 4 or 8 (TileArgs::proj_variant 0, 1, 2).

__device__ __forceinline__ unsigned tf32_rna(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void split_tf32(float x, unsigned& hi, unsigned& lo) {
  hi = tf32_rna(x);
  lo = tf32_rna(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32_1688(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int kPW>
__global__ void __launch_bounds__(32 * kPW) k_gproject_mma(TileArgs<float> a, const float2* __restrict__ v) {
  __shared__ float part[kPW][32][8];
  const int at = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int ob = blockIdx.y * 16;
  const int i0 = a.atom_off[at], i1 = a.atom_off[at + 1];
  const bool r0 = ob + g < a.norb_tot, r1 = ob + g + 8 < a.norb_tot;
  const float2* u0 = v + (size_t)(r0 ? ob + g : 0) * a.npts;
  const float2* u1 = v + (size_t)(r1 ? ob + g + 8 : 0) * a.npts;
  float dre[4] = {0, 0, 0, 0}, dim[4] = {0, 0, 0, 0};
  for (int k0 = i0 + 8 * warp; k0 < i1; k0 += 8 * kPW) {
    const int ia = k0 + t, ib = k0 + t + 4;
    const bool va = ia < i1, vb = ib < i1;
    const int xa = va ? a.sph_idx[ia] : 0, xb = vb ? a.sph_idx[ib] : 0;
    const float2 z = make_float2(0.f, 0.f);
    const float2 p0a = (va && r0) ? u0[xa] : z, p1a = (va && r1) ? u1[xa] : z;
    const float2 p0b = (vb && r0) ? u0[xb] : z, p1b = (vb && r1) ? u1[xb] : z;
    const float ba = (va && g < 4) ? a.sph_beta[4 * ia + g] : 0.f;
    const float bb = (vb && g < 4) ? a.sph_beta[4 * ib + g] : 0.f;
    unsigned bh0, bl0, bh1, bl1;
    split_tf32(ba, bh0, bl0);
    split_tf32(bb, bh1, bl1);
    unsigned ah[4], al[4];
    // real parts
    split_tf32(p0a.x, ah[0], al[0]); split_tf32(p1a.x, ah[1], al[1]);
    split_tf32(p0b.x, ah[2], al[2]); split_tf32(p1b.x, ah[3], al[3]);
    mma_tf32_1688(dre, al, bh0, bh1);
    mma_tf32_1688(dre, ah, bl0, bl1);
    mma_tf32_1688(dre, ah, bh0, bh1);
    // imaginary parts
    split_tf32(p0a.y, ah[0], al[0]); split_tf32(p1a.y, ah[1], al[1]);
    split_tf32(p0b.y, ah[2], al[2]); split_tf32(p1b.y, ah[3], al[3]);
    mma_tf32_1688(dim, al, bh0, bh1);
    mma_tf32_1688(dim, ah, bl0, bl1);
    mma_tf32_1688(dim, ah, bh0, bh1);
  }
  // the warps' partial products meet in shared memory (fixed order)
#pragma unroll
  for (int j = 0; j < 4; ++j) { part[warp][lane][j] = dre[j]; part[warp][lane][4 + j] = dim[j]; }
  __syncthreads();
  if (warp != 0 || t >= 2) return;        // columns 2t, 2t+1 are projectors 0..3
#pragma unroll
  for (int w = 1; w < kPW; ++w)
#pragma unroll
    for (int j = 0; j < 4; ++j) { dre[j] += part[w][lane][j]; dim[j] += part[w][lane][4 + j]; }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int p = 2 * t + j;
    const float sc = a.atomE[at * 4 + p] * a.dV;
    if (r0) a.ec[((size_t)(ob + g) * a.natom + at) * 4 + p] = make_float2(dre[j] * sc, dim[j] * sc);
    if (r1) a.ec[((size_t)(ob + g + 8) * a.natom + at) * 4 + p] = make_float2(dre[2 + j] * sc, dim[2 + j] * sc);
  }
}

// out[p] += f * V_NL v at sphere points, f = 1 (H) or -i coef (Horner stage); one thread per
// (sphere point, orbital).
template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_gscatter(TileArgs<T> a, typename Cplx<T>::type* out) {
  using C = typename Cplx<T>::type;
  const int orb = blockIdx.y;
  const C* ec = a.ec + (size_t)orb * a.natom * 4;
  C* o = out + (size_t)orb * a.npts;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < a.nsp; s += gridDim.x * blockDim.x) {
    T re = 0, im = 0;
    for (int e = a.sp_off[s]; e < a.sp_off[s + 1]; ++e) {
      const int i = a.pt_ent[e];
      const int at = a.ent_atom[i];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const T b = a.sph_beta[i * 4 + q];
        const C c = ec[at * 4 + q];
        re += b * c.x;
        im += b * c.y;
      }
    }
    const int p = a.sp_pt[s];
    C r = o[p];
    if (MODE == 1) { r.x += a.coef * im; r.y -= a.coef * re; }
    else { r.x += re; r.y += im; }
    o[p] = r;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

template <typename T>
bool encode_map(CUtensorMap* map, const void* base, int nx, int ny, int nz, int norb_tot, int bx, int by) {
  auto enc = get_encode();
  if (!enc) return false;
  constexpr int E = sizeof(typename Cplx<T>::type) / 8;
  const cuuint64_t dims[4] = {(cuuint64_t)E * nx, (cuuint64_t)ny, (cuuint64_t)nz, (cuuint64_t)norb_tot};
  const cuuint64_t strides[3] = {(cuuint64_t)8 * E * nx, (cuuint64_t)8 * E * nx * ny,
                                 (cuuint64_t)8 * E * nx * ny * nz};
  const cuuint32_t box[4] = {(cuuint32_t)(E * bx), (cuuint32_t)by, 1, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = enc(map, E == 1 ? CU_TENSOR_MAP_DATA_TYPE_INT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4,
                   const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// 3D map of the FP32 potential [nz][ny][nx] with an interior box bx x by (needs nx % 4 == 0).
bool encode_pot_map(CUtensorMap* map, const float* V, int nx, int ny, int nz, int bx, int by) {
  auto enc = get_encode();
  if (!enc || nx % 4 != 0) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  const cuuint64_t strides[2] = {(cuuint64_t)4 * nx, (cuuint64_t)4 * nx * ny};
  const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(V), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int MODE, int NCW, int ROWS, bool SV>
cudaError_t launch_tile4(const TileArgs<float>& a, const CUtensorMap& pmap, const void* vin, cudaStream_t s) {
  using G = B4<NCW, ROWS>;
  CUtensorMap map, potmap;
  std::memset(&potmap, 0, sizeof(potmap));
  if (!encode_map<float>(&map, vin, a.nx, a.ny, a.nz, a.norb_tot, G::SX, G::SY)) return cudaErrorInvalidValue;
  if (SV && !encode_pot_map(&potmap, a.V, a.nx, a.ny, a.nz, G::TX, G::TY)) return cudaErrorInvalidValue;
  const dim3 grid(((a.nx + G::TX - 1) / G::TX) * ((a.ny + G::TY - 1) / G::TY), a.norb_tot);
  size_t smem = (size_t)G::NS * G::SX * G::SY * sizeof(float2) + 128;
  if (SV) smem += (size_t)G::NS * G::TX * G::TY * (sizeof(float) + (MODE == 1 ? sizeof(float2) : 0));
  cudaError_t e = cudaFuncSetAttribute(k_tile4<MODE, NCW, ROWS, SV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_tile4<MODE, NCW, ROWS, SV><<<grid, G::NT, smem, s>>>(map, pmap, potmap, a);
  return cudaGetLastError();
}

template <typename T, int MINB>
cudaError_t launch_tile_plain(const TileArgs<T>& a, const CUtensorMap& pmap, const void* vin, int mode,
                              cudaStream_t s) {
  CUtensorMap map;
  if (!encode_map<T>(&map, vin, a.nx, a.ny, a.nz, a.norb_tot, SX, SY)) return cudaErrorInvalidValue;
  const dim3 grid(((a.nx + TX - 1) / TX) * ((a.ny + TY - 1) / TY), a.norb_tot);   // NT threads
  const size_t smem = (size_t)NS * SX * SY * sizeof(typename Cplx<T>::type) + 128;
  if (mode == 1) {
    cudaError_t e = cudaFuncSetAttribute(k_tile<T, 1, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_tile<T, 1, MINB><<<grid, NT, smem, s>>>(map, pmap, a);
  } else {
    cudaError_t e = cudaFuncSetAttribute(k_tile<T, 0, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_tile<T, 0, MINB><<<grid, NT, smem, s>>>(map, pmap, a);
  }
  return cudaGetLastError();
}

}  // namespace

bool tile_variant_ok(int variant, int nx, int elem_bytes) {
  if (elem_bytes == 16) return variant == 0 || variant == 1;
  if (variant == 5 || variant == 6) return nx % 4 == 0;     // the potential's tensor-map rows
  return variant >= 0 && variant < kTileVariants;
}

bool tile_supported(int nx, int ny, int nz, int elem_bytes) {
  // row stride must be a multiple of 16 bytes for the tensor map
  return ((size_t)nx * elem_bytes) % 16 == 0 && nz >= 1 && get_encode() != nullptr;
}

// Variant table of the tile stencil (kernel, resident CTAs per SM the registers are capped for, L2
// prefetch distance in planes).  FP32: 0 = k_tile, 3 CTAs, no prefetch; 1 = k_tile, 2 CTAs, 8;
// 2 = k_tile4<8> (2 x 2 points per thread), 8; 3 = k_tile4<8, 1 row> (2 x 1 points per thread,
// 2 CTAs), 8; 4 = k_tile4<4, 1 row> (4 consumer warps, 4 CTAs), 8; 5, 6 = variants 3, 4 with V and psi
// staged by TMA beside the orbital planes (nx % 4 == 0).  FP64 (one CTA per SM, as the ring fills
// shared memory): 0 = no prefetch, 1 = prefetch 8.
template <typename T>
cudaError_t launch_tile_stage(const TileArgs<T>& a0, const void* vin, int mode, cudaStream_t s) {
  TileArgs<T> a = a0;
  a.prefetch = a.variant == 0 ? 0 : 8;
  // psi map (interior box): the L2 prefetch of the Horner base, or (variants 5, 6) its TMA loads;
  // unused in mode 0
  CUtensorMap pmap;
  std::memset(&pmap, 0, sizeof(pmap));
  if (mode == 1 && a.prefetch > 0) {
    int by = TY;
    if (sizeof(T) == 4 && a.variant == 2) by = B4<8>::TY;
    if (sizeof(T) == 4 && (a.variant == 3 || a.variant == 5)) by = B4<8, 1>::TY;
    if (sizeof(T) == 4 && (a.variant == 4 || a.variant == 6)) by = B4<4, 1>::TY;
    if (!encode_map<T>(&pmap, a.psi, a.nx, a.ny, a.nz, a.norb_tot, TX, by)) return cudaErrorInvalidValue;
  }
  if constexpr (sizeof(T) == 4) {
    if (a.variant == 2)
      return mode == 1 ? launch_tile4<1, 8, 2, false>(a, pmap, vin, s) : launch_tile4<0, 8, 2, false>(a, pmap, vin, s);
    if (a.variant == 3)
      return mode == 1 ? launch_tile4<1, 8, 1, false>(a, pmap, vin, s) : launch_tile4<0, 8, 1, false>(a, pmap, vin, s);
    if (a.variant == 4)
      return mode == 1 ? launch_tile4<1, 4, 1, false>(a, pmap, vin, s) : launch_tile4<0, 4, 1, false>(a, pmap, vin, s);
    if (a.variant == 5)
      return mode == 1 ? launch_tile4<1, 8, 1, true>(a, pmap, vin, s) : launch_tile4<0, 8, 1, true>(a, pmap, vin, s);
    if (a.variant == 6)
      return mode == 1 ? launch_tile4<1, 4, 1, true>(a, pmap, vin, s) : launch_tile4<0, 4, 1, true>(a, pmap, vin, s);
    if (a.variant == 1) return launch_tile_plain<T, 2>(a, pmap, vin, mode, s);
    return launch_tile_plain<T, 3>(a, pmap, vin, mode, s);
  } else {
    return launch_tile_plain<T, 1>(a, pmap, vin, mode, s);
  }
}

template <typename T>
cudaError_t launch_tile_project(const TileArgs<T>& a, const typename Cplx<T>::type* v, cudaStream_t s) {
  if (a.natom == 0) return cudaSuccess;
  if constexpr (sizeof(T) == 4) {      // FP32: tensor cores (3xTF32); the schedule of the projection
    const dim3 grid(a.natom, (a.norb_tot + 15) / 16);   // tuner: 2, 4 or 8 warps per CTA
    if (a.proj_variant == 0) k_gproject_mma<2><<<grid, 64, 0, s>>>(a, v);
    else if (a.proj_variant == 2) k_gproject_mma<8><<<grid, 256, 0, s>>>(a, v);
    else k_gproject_mma<4><<<grid, 128, 0, s>>>(a, v);
  } else {
    const dim3 grid(a.natom, (a.norb_tot + kOB - 1) / kOB);
    k_gproject<T><<<grid, 128, 0, s>>>(a, v);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tile_scatter(const TileArgs<T>& a, typename Cplx<T>::type* out, int mode, cudaStream_t s) {
  if (a.natom == 0 || a.nsp == 0) return cudaSuccess;
  const dim3 grid((a.nsp + 255) / 256, a.norb_tot);
  if (mode == 1) k_gscatter<T, 1><<<grid, 256, 0, s>>>(a, out);
  else k_gscatter<T, 0><<<grid, 256, 0, s>>>(a, out);
  return cudaGetLastError();
}

template cudaError_t launch_tile_stage<float>(const TileArgs<float>&, const void*, int, cudaStream_t);
template cudaError_t launch_tile_stage<double>(const TileArgs<double>&, const void*, int, cudaStream_t);
template cudaError_t launch_tile_project<float>(const TileArgs<float>&, const float2*, cudaStream_t);
template cudaError_t launch_tile_project<double>(const TileArgs<double>&, const double2*, cudaStream_t);
template cudaError_t launch_tile_scatter<float>(const TileArgs<float>&, float2*, int, cudaStream_t);
template cudaError_t launch_tile_scatter<double>(const TileArgs<double>&, double2*, int, cudaStream_t);

}  // namespace tdks
