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
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "tdks_internal.h"

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
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
  for (long long i = 0; i < kSpinLimit; ++i)
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

template <typename T> struct TM;
template <> struct TM<float> {
  using C = float2;
  static __device__ __forceinline__ C add(C a, C b) { return __fadd2_rn(a, b); }
  static __device__ __forceinline__ C fma(float s, C a, C acc) { return __ffma2_rn(make_float2(s, s), a, acc); }
};
template <> struct TM<double> {
  using C = double2;
  static __device__ __forceinline__ C add(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
  static __device__ __forceinline__ C fma(double s, C a, C acc) {
    return C{__fma_rn(s, a.x, acc.x), __fma_rn(s, a.y, acc.y)};
  }
};

// MODE 0: out = H_loc v.  MODE 1: out = psi + (-i coef) H_loc v.   (H_loc: everything but V_NL;
// q = 0 for isolated systems.)
template <typename T, int MODE>
__global__ void __launch_bounds__(NT) k_tile(const __grid_constant__ CUtensorMap vmap, TileArgs<T> a) {
  using C = typename Cplx<T>::type;
  using M = TM<T>;
  constexpr int E = sizeof(C) / 8;                 // 8-byte tensor elements per complex value
  constexpr unsigned kSlotBytes = SX * SY * sizeof(C);
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
    // ---------------- producer warp: one lane issues every plane copy
    if (lane == 0) {
      int issued = 0;
      bool ok = true;
      for (int j = 0; j < nplanes && ok; ++j) {
        const int slot = j % NS;
        if (j >= NS && !mbar_wait(&empty[slot], ((j / NS) - 1) & 1)) { ok = false; break; }
        if (volatile_abort(&s_abort)) { ok = false; break; }
        mbar_expect_tx(&full[slot], kSlotBytes);
        tma_load_4d(ring + slot * SX * SY, &vmap, E * (x0 - 4), y0 - 4, j - 4, orb, &full[slot]);
        issued = j + 1;
      }
      if (!ok) {
        atomicExch(&s_abort, 1);
        atomicExch(a.err, (int)TDKS_ETIMEOUT);
      }
      // the most recent copy of every slot has landed before this warp leaves, so no copy is in
      // flight when the CTA's shared memory is released (bounded waits)
      for (int j = (issued > NS ? issued - NS : 0); j < issued; ++j) mbar_wait(&full[j % NS], (j / NS) & 1);
    }
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
  bool timeout = false;
  C w[RPT][9];
  // window planes j = 0..7 (z = -4..3); planes 0..3 are released right away
  for (int j = 0; j < 8; ++j) {
    if (!timeout && !mbar_wait(&full[j % NS], (j / NS) & 1)) timeout = true;
#pragma unroll
    for (int r = 0; r < RPT; ++r) w[r][j] = ring[(j % NS) * SX * SY + own[r]];
    if (j < 4) {
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[j % NS]);
    }
  }
  const T coef = a.coef;
  C pnext[RPT];
  T vnext[RPT];
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    pnext[r] = C{0, 0};
    vnext[r] = 0;
    if (inside[r]) {
      if (MODE == 1) pnext[r] = a.psi[obase + col[r]];
      vnext[r] = a.V[col[r]];
    }
  }
  for (int z = 0; z < a.nz; ++z) {
    if (timeout || volatile_abort(&s_abort)) break;
    const int jc = z + 4;
    const int jn = z + 8;
    if (!mbar_wait(&full[jn % NS], (jn / NS) & 1)) { timeout = true; break; }
    const C* sbase = ring + (jc % NS) * SX * SY;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      w[r][8] = ring[(jn % NS) * SX * SY + own[r]];
      const C pv = pnext[r];
      const T vv = vnext[r];
      if (inside[r] && z + 1 < a.nz) {             // prefetch the next plane's psi and V
        if (MODE == 1) pnext[r] = a.psi[obase + (size_t)(z + 1) * plane + col[r]];
        vnext[r] = a.V[(size_t)(z + 1) * plane + col[r]];
      }
      const C* s = sbase + own[r];
      C Sx = M::fma(a.diag + vv, w[r][4], C{0, 0}), Sy = C{0, 0}, Sz = C{0, 0};
#pragma unroll
      for (int m = 1; m <= 4; ++m) {
        Sx = M::fma(a.c2x[m], M::add(s[m], s[-m]), Sx);
        Sy = M::fma(a.c2y[m], M::add(s[m * SX], s[-m * SX]), Sy);
        Sz = M::fma(a.c2z[m], M::add(w[r][4 + m], w[r][4 - m]), Sz);
      }
      const C S = M::add(M::add(Sx, Sy), Sz);
      if (inside[r]) {
        const size_t o = obase + (size_t)z * plane + col[r];
        if (MODE == 1) a.out[o] = M::fma(coef, C{S.y, -S.x}, pv);   // psi + (-i coef) H v
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

// Projections for large grids: one CTA per orbital, one warp per atom at a time.
// ec[orb][a][p] = E_p dV sum_i beta_ip v(idx_i)   (isolated: q = 0, no phase)
template <typename T>
__global__ void __launch_bounds__(256) k_gproject(TileArgs<T> a, const typename Cplx<T>::type* v) {
  using C = typename Cplx<T>::type;
  const int orb = blockIdx.x;
  const C* u = v + (size_t)orb * a.npts;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int at = warp; at < a.natom; at += nw) {
    T acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = a.atom_off[at] + lane; i < a.atom_off[at + 1]; i += 32) {
      const C x = u[a.sph_idx[i]];
      const T* b = a.sph_beta + 4 * i;
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        acc[2 * p] += b[p] * x.x;
        acc[2 * p + 1] += b[p] * x.y;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
    if (lane < 4) {
      const T sc = a.atomE[at * 4 + lane] * a.dV;
      a.ec[((size_t)orb * a.natom + at) * 4 + lane] = C{acc[2 * lane] * sc, acc[2 * lane + 1] * sc};
    }
  }
}

// out[p] += f * V_NL v at sphere points, f = 1 (H) or -i coef (Horner stage).
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
bool encode_map(CUtensorMap* map, const void* base, int nx, int ny, int nz, int norb_tot) {
  auto enc = get_encode();
  if (!enc) return false;
  constexpr int E = sizeof(typename Cplx<T>::type) / 8;
  const cuuint64_t dims[4] = {(cuuint64_t)E * nx, (cuuint64_t)ny, (cuuint64_t)nz, (cuuint64_t)norb_tot};
  const cuuint64_t strides[3] = {(cuuint64_t)8 * E * nx, (cuuint64_t)8 * E * nx * ny,
                                 (cuuint64_t)8 * E * nx * ny * nz};
  const cuuint32_t box[4] = {(cuuint32_t)(E * SX), (cuuint32_t)SY, 1, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = enc(map, E == 1 ? CU_TENSOR_MAP_DATA_TYPE_INT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4,
                   const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

bool tile_supported(int nx, int ny, int nz, int elem_bytes) {
  // row stride must be a multiple of 16 bytes for the tensor map
  return ((size_t)nx * elem_bytes) % 16 == 0 && nz >= 1 && get_encode() != nullptr;
}

template <typename T>
cudaError_t launch_tile_stage(const TileArgs<T>& a, const void* vin, int mode, cudaStream_t s) {
  CUtensorMap map;
  if (!encode_map<T>(&map, vin, a.nx, a.ny, a.nz, a.norb_tot)) return cudaErrorInvalidValue;
  const dim3 grid(((a.nx + TX - 1) / TX) * ((a.ny + TY - 1) / TY), a.norb_tot);   // NT threads
  const size_t smem = (size_t)NS * SX * SY * sizeof(typename Cplx<T>::type) + 128;
  if (mode == 1) {
    cudaError_t e = cudaFuncSetAttribute(k_tile<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_tile<T, 1><<<grid, NT, smem, s>>>(map, a);
  } else {
    cudaError_t e = cudaFuncSetAttribute(k_tile<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_tile<T, 0><<<grid, NT, smem, s>>>(map, a);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tile_project(const TileArgs<T>& a, const typename Cplx<T>::type* v, cudaStream_t s) {
  if (a.natom == 0) return cudaSuccess;
  k_gproject<T><<<a.norb_tot, 256, 0, s>>>(a, v);
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
