// tdks_hxc_noalloc: the Hartree + exchange potential of a density, for callers that cannot
// allocate device memory.
//
// The FFT work area lives in one file-scope device array (g_noalloc) instead of memory from
// cudaMalloc.  Every GPU that loads the library holds the array until the process exits.  Host
// code cannot pass the array's name to a kernel (on the host that name is only a stand-in), so
// the first call on each device asks the runtime for the array's device address with
// cudaGetSymbolAddress and caches it.  The cached address belongs to the device's current context:
// after cudaDeviceReset the module is loaded again and the array may move, so a process that resets
// a device must not call this entry point on it again.  All calls share the array: concurrent calls
// on different streams race.
#include <cmath>
#include <mutex>

#include "tdks_internal.h"

namespace {

constexpr int kNoallocMaxLine = 64;                                   // points per FFT axis
constexpr size_t kNoallocMaxPoints = (size_t)64 * 64 * 64;            // FFT points in total
constexpr int kMaxDevices = 64;

struct NoallocArea {
  double2 fft[kNoallocMaxPoints];        // transform buffer
  double ghat[kNoallocMaxPoints];        // spectrum of the Hockney Green's function (isolated)
  double2 tw[3][kNoallocMaxLine];        // twiddles exp(-2 pi i t / m) per axis
};

static __device__ __align__(256) NoallocArea g_noalloc;

NoallocArea* g_noalloc_addr[kMaxDevices] = {nullptr};
std::mutex g_noalloc_mu;

tdks_status noalloc_fail(tdks_status s, const char* msg) {
  tdks::set_last_error(msg);
  return s;
}

__global__ void k_noalloc_twiddles(double2* tw, int m) {
  for (int t = threadIdx.x; t < m; t += blockDim.x) {
    double s, c;
    sincospi(2.0 * t / m, &s, &c);
    tw[t] = double2{c, -s};
  }
}

// factor m into the radices the FFT kernel takes (4, 2, then odd primes up to 31), without heap
// storage
int noalloc_radices(int m, int* r) {
  int k = 0;
  while (m % 4 == 0) { r[k++] = 4; m /= 4; }
  while (m % 2 == 0) { r[k++] = 2; m /= 2; }
  for (int p = 3; p <= 31; p += 2)
    while (m % p == 0) { r[k++] = p; m /= p; }
  return m == 1 ? k : -1;
}

}  // namespace

extern "C" tdks_status tdks_hxc_noalloc(const tdks_grid* grid, const double* rho_dev, double* vhxc_dev,
                                        int hartree, int xc, void* stream) {
  using namespace tdks;
  if (!grid || !rho_dev || !vhxc_dev) return noalloc_fail(TDKS_EINVAL, "null grid, density or output");
  if (xc < 0 || xc > 2) return noalloc_fail(TDKS_EINVAL, "tdks_hxc_noalloc: xc must be 0, 1 or 2");
  int m[3];
  int rad[3][16];
  int nrad[3];
  size_t total = 1;
  for (int a = 0; a < 3; ++a) {
    if (grid->n[a] < 4 || !(grid->h[a] > 0.0)) return noalloc_fail(TDKS_EINVAL, "grid needs n >= 4 and h > 0 per axis");
    m[a] = grid->periodic ? grid->n[a] : 2 * grid->n[a];
    if (m[a] > kNoallocMaxLine)
      return noalloc_fail(TDKS_EUNSUPPORTED,
                          "tdks_hxc_noalloc: FFT length above 64 per axis (periodic n <= 64, isolated n <= 32)");
    nrad[a] = noalloc_radices(m[a], rad[a]);
    if (nrad[a] < 0) return noalloc_fail(TDKS_EUNSUPPORTED, "tdks_hxc_noalloc: FFT length with a prime factor above 31");
    total *= (size_t)m[a];
  }
  if (total > kNoallocMaxPoints)
    return noalloc_fail(TDKS_EUNSUPPORTED, "tdks_hxc_noalloc: more than 64^3 FFT points");

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(TDKS_ECUDA, "tdks_hxc_noalloc: no usable current device");
  NoallocArea* area = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc);
      if (e != cudaSuccess || !p) return noalloc_fail(TDKS_ECUDA, "tdks_hxc_noalloc: cudaGetSymbolAddress failed");
      g_noalloc_addr[dev] = static_cast<NoallocArea*>(p);
    }
    area = g_noalloc_addr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int n[3] = {grid->n[0], grid->n[1], grid->n[2]};
  const double dV = grid->h[0] * grid->h[1] * grid->h[2];
  for (int a = 0; a < 3; ++a) k_noalloc_twiddles<<<1, 64, 0, s>>>(area->tw[a], m[a]);
  if (cudaGetLastError() != cudaSuccess) return noalloc_fail(TDKS_ECUDA, "tdks_hxc_noalloc: twiddle launch failed");

  auto fft3d = [&](int dir) -> bool {
    for (int a = 0; a < 3; ++a)
      if (launch_fft_axis(area->fft, m, a, dir, area->tw[a], rad[a], nrad[a], s) != cudaSuccess) return false;
    return true;
  };
  if (hartree) {
    if (!grid->periodic) {
      // spectrum of the zero-padded Green's function, rebuilt on every call
      const double g0 = cell_mean_inverse_distance(grid->h[0], grid->h[1], grid->h[2]);
      if (launch_hockney_kernel(area->fft, m, n, grid->h, g0, s) != cudaSuccess || !fft3d(-1) ||
          launch_real_part(area->fft, area->ghat, total, 1.0, s) != cudaSuccess)
        return noalloc_fail(TDKS_ECUDA, "tdks_hxc_noalloc: Green's function launch failed");
    }
    if (launch_pack_real(rho_dev, n, area->fft, m, s) != cudaSuccess || !fft3d(-1))
      return noalloc_fail(TDKS_ECUDA, "tdks_hxc_noalloc: forward transform failed");
    const cudaError_t e = grid->periodic
                              ? launch_poisson_scale_periodic(area->fft, m, grid->h, s)
                              : launch_scale_by_real(area->fft, area->ghat, dV / (double)total, total, s);
    if (e != cudaSuccess || !fft3d(+1)) return noalloc_fail(TDKS_ECUDA, "tdks_hxc_noalloc: inverse transform failed");
  }
  if (launch_hxc_epilogue(area->fft, m, rho_dev, n, 1.0, hartree, xc, vhxc_dev, s) != cudaSuccess)
    return noalloc_fail(TDKS_ECUDA, "tdks_hxc_noalloc: epilogue launch failed");
  return TDKS_OK;
}
