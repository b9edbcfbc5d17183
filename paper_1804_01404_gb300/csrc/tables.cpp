// Host-side set-up tables: Kleinman-Bylander projector spheres, the periodic local potential in
// G-space, the Hockney self-term and FFT factorisations.  Plain C++, run once per context.
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "tdks_internal.h"

namespace tdks {

static double coord(const tdks_grid& g, int axis, int j) {
  return g.periodic ? j * g.h[axis] : (j - 0.5 * (g.n[axis] - 1)) * g.h[axis];
}

bool build_projector_tables(const tdks_grid& g, const tdks_atom* atoms, int natom,
                            const tdks_projector* proj, int nproj, ProjectorTables& T,
                            std::string& err) {
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const long long npts = 1LL * nx * ny * nz;
  const double dV = g.h[0] * g.h[1] * g.h[2];
  const double L[3] = {nx * g.h[0], ny * g.h[1], nz * g.h[2]};
  T = ProjectorTables();
  T.atom_off.push_back(0);
  for (int ia = 0; ia < natom; ++ia) {
    const tdks_atom& at = atoms[ia];
    if (at.proj < 0) continue;
    if (at.proj >= nproj) { err = "atom projector index out of range"; return false; }
    const tdks_projector& P = proj[at.proj];
    const double rc = P.r_cut, w = P.width;
    if (!(rc > 0.0) || !(w > 0.0)) { err = "projector r_cut and width must be positive"; return false; }
    if (g.periodic && rc >= 0.5 * std::min(L[0], std::min(L[1], L[2]))) {
      err = "projector sphere wider than half the periodic cell";
      return false;
    }
    // candidate indices per axis with |d_axis| < rc (nearest image for periodic cells)
    std::vector<int> cand[3];
    std::vector<double> disp[3];
    for (int a = 0; a < 3; ++a) {
      for (int j = 0; j < g.n[a]; ++j) {
        double dd = coord(g, a, j) - at.R[a];
        if (g.periodic) dd -= L[a] * std::nearbyint(dd / L[a]);
        if (std::fabs(dd) < rc) { cand[a].push_back(j); disp[a].push_back(dd); }
      }
    }
    const size_t first = T.idx.size();
    double nrm[4] = {0, 0, 0, 0};
    for (size_t kz = 0; kz < cand[2].size(); ++kz)
      for (size_t ky = 0; ky < cand[1].size(); ++ky)
        for (size_t kx = 0; kx < cand[0].size(); ++kx) {
          const double dx = disp[0][kx], dy = disp[1][ky], dz = disp[2][kz];
          const double r2 = dx * dx + dy * dy + dz * dz;
          if (!(r2 < rc * rc)) continue;
          const double s = 1.0 - r2 / (rc * rc);
          const double gv = std::exp(-r2 / (2.0 * w * w)) * s * s;
          const double b[4] = {gv, dx * gv, dy * gv, dz * gv};
          T.idx.push_back((cand[2][kz] * ny + cand[1][ky]) * nx + cand[0][kx]);
          for (int p = 0; p < 4; ++p) { T.beta.push_back(b[p]); nrm[p] += b[p] * b[p] * dV; }
          T.d.push_back(dx); T.d.push_back(dy); T.d.push_back(dz);
          T.ent_atom.push_back(T.natom);
        }
    for (int p = 0; p < 4; ++p) {
      if (!(nrm[p] > 0.0)) { err = "projector has no grid points (r_cut below the spacing)"; return false; }
      const double inv = 1.0 / std::sqrt(nrm[p]);
      for (size_t i = first; i < T.idx.size(); ++i) T.beta[i * 4 + p] *= inv;
    }
    T.E.push_back(P.E_s); T.E.push_back(P.E_p); T.E.push_back(P.E_p); T.E.push_back(P.E_p);
    T.natom += 1;
    T.atom_off.push_back((int)T.idx.size());
  }
  // point -> entry CSR
  const size_t nsph = T.idx.size();
  T.pt_off.assign(npts + 1, 0);
  for (size_t i = 0; i < nsph; ++i) T.pt_off[T.idx[i] + 1] += 1;
  for (long long p = 0; p < npts; ++p) T.pt_off[p + 1] += T.pt_off[p];
  T.pt_ent.assign(nsph, 0);
  std::vector<int> fill(T.pt_off.begin(), T.pt_off.end() - 1);
  for (size_t i = 0; i < nsph; ++i) T.pt_ent[fill[T.idx[i]]++] = (int)i;
  T.sp_pt.clear();
  T.sp_off.clear();
  for (long long p = 0; p < npts; ++p)
    if (T.pt_off[p + 1] > T.pt_off[p]) {
      T.sp_pt.push_back((int)p);
      T.sp_off.push_back(T.pt_off[p]);
    }
  T.sp_off.push_back((int)nsph);
  return true;
}

static double fft_frequency(int m, int n) { return (m <= (n - 1) / 2) ? m : m - n; }

void local_potential_gspace(const tdks_grid& g, const tdks_atom* atoms, int natom,
                            std::vector<double>& vg) {
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const double L[3] = {nx * g.h[0], ny * g.h[1], nz * g.h[2]};
  const double omega = L[0] * L[1] * L[2];
  vg.assign(2ULL * nx * ny * nz, 0.0);
  for (int iz = 0; iz < nz; ++iz)
    for (int iy = 0; iy < ny; ++iy)
      for (int ix = 0; ix < nx; ++ix) {
        const double G[3] = {2.0 * kPi * fft_frequency(ix, nx) / L[0],
                             2.0 * kPi * fft_frequency(iy, ny) / L[1],
                             2.0 * kPi * fft_frequency(iz, nz) / L[2]};
        const double G2 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
        if (G2 == 0.0) continue;
        double re = 0.0, im = 0.0;
        for (int a = 0; a < natom; ++a) {
          const double amp = -4.0 * kPi * atoms[a].Z / G2 *
                             std::exp(-G2 * atoms[a].sigma * atoms[a].sigma / 4.0);
          const double ph = G[0] * atoms[a].R[0] + G[1] * atoms[a].R[1] + G[2] * atoms[a].R[2];
          re += amp * std::cos(ph);
          im -= amp * std::sin(ph);
        }
        const size_t o = ((size_t)(iz * ny + iy) * nx + ix) * 2;
        vg[o] = re / omega;
        vg[o + 1] = im / omega;
      }
}

// integral of 1/|r| over [0,a]x[0,b]x[0,c] (Newton potential of a uniform box at its corner)
static double box_corner_integral(double a, double b, double c) {
  const double d = std::sqrt(a * a + b * b + c * c);
  return a * b * std::log((c + d) / std::hypot(a, b)) + b * c * std::log((a + d) / std::hypot(b, c)) +
         c * a * std::log((b + d) / std::hypot(c, a)) - 0.5 * a * a * std::atan(b * c / (a * d)) -
         0.5 * b * b * std::atan(c * a / (b * d)) - 0.5 * c * c * std::atan(a * b / (c * d));
}

double cell_mean_inverse_distance(double hx, double hy, double hz) {
  return 8.0 * box_corner_integral(0.5 * hx, 0.5 * hy, 0.5 * hz) / (hx * hy * hz);
}

bool fft_radices(int n, std::vector<int>& r) {
  r.clear();
  if (n < 1) return false;
  while (n % 4 == 0) { r.push_back(4); n /= 4; }
  while (n % 2 == 0) { r.push_back(2); n /= 2; }
  for (int p = 3; p <= n; p += 2)
    while (n % p == 0) {
      if (p > 31) return false;   // large prime factors are not supported
      r.push_back(p);
      n /= p;
    }
  return true;
}

}  // namespace tdks
