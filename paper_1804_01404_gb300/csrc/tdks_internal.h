// Internal declarations shared by the libtdks translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/tdks.h"

namespace tdks {

// 8th-order central differences, 4 neighbours per side:
// f'' ~ (1/h^2)[c0 f0 + sum_m c_m (f_m + f_-m)],  f' ~ (1/h) sum_m d_m (f_m - f_-m).
constexpr double kFD2[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};
constexpr double kFD1[4] = {4.0 / 5.0, -1.0 / 5.0, 4.0 / 105.0, -1.0 / 280.0};
constexpr double kPi = 3.14159265358979323846;

template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };

// Host-built projector tables (Kleinman-Bylander s, px, py, pz per atom with projectors).
struct ProjectorTables {
  int natom = 0;                  // atoms that carry projectors
  std::vector<int> atom_off;      // [natom+1] entry ranges
  std::vector<int> idx;           // [nsph] grid index (z*ny + y)*nx + x
  std::vector<double> beta;       // [nsph*4] normalised beta_s, beta_px, beta_py, beta_pz
  std::vector<double> d;          // [nsph*3] displacement from the atom (nearest image)
  std::vector<double> E;          // [natom*4] E_s, E_p, E_p, E_p
  std::vector<int> pt_off;        // [npts+1] point -> entries (CSR)
  std::vector<int> pt_ent;        // [nsph]  entry ids sorted by grid point
  std::vector<int> ent_atom;      // [nsph]  atom of each entry
  std::vector<int> sp_pt;         // [nsp]   unique grid points inside at least one sphere
  std::vector<int> sp_off;        // [nsp+1] their entry ranges in pt_ent
};

// Shared-memory layout of one orbital: plane stride nx*ny (+1 pad element that stays zero for
// isolated cells, so out-of-box x/y neighbours read 0 without a branch).
inline int smem_plane_stride(const tdks_grid& g) { return g.n[0] * g.n[1] + (g.periodic ? 0 : 1); }

// Set the thread-local message returned by tdks_last_error().
void set_last_error(const char* msg);

// Build projector tables; returns false with a message on invalid input.
bool build_projector_tables(const tdks_grid& g, const tdks_atom* atoms, int natom,
                            const tdks_projector* proj, int nproj, ProjectorTables& out,
                            std::string& err);

// Periodic local potential in G-space on the FFT grid, layout [nz][ny][nx] complex (re, im):
// V(G) = (1/Omega) sum_a (-4 pi Z / G^2) exp(-G^2 sigma^2/4) exp(-i G.R), V(0) = 0.
void local_potential_gspace(const tdks_grid& g, const tdks_atom* atoms, int natom,
                            std::vector<double>& vg_interleaved);

// Mean of 1/|r| over one grid cell centred at the origin, times nothing: returns
// (1/dV) * integral over [-hx/2,hx/2]x[-hy/2,hy/2]x[-hz/2,hz/2] of 1/|r|.
double cell_mean_inverse_distance(double hx, double hy, double hz);

// Factorisation of an FFT length into radices (4, 2, 3, 5, then any prime).
bool fft_radices(int n, std::vector<int>& radices);

// ---------------------------------------------------------------------------------------------
// device-side argument blocks
// ---------------------------------------------------------------------------------------------
template <typename T>
struct OrbArgs {
  using C = typename Cplx<T>::type;
  const C* psi_in;          // [norb_tot][npts]
  C* psi_out;               // output (Hu, or the propagated orbital); may alias psi_in for Taylor
  const T* V;               // [npts] local potential of this call
  int nx, ny, nz, npts, periodic;
  T c2x[5], c2y[5], c2z[5]; // -1/2 * FD2[m] / h^2
  T d1x[4], d1y[4], d1z[4]; // FD1[m] / h
  T ry, rz;                 // hx^2/hy^2, hx^2/hz^2: c2y = ry c2x, c2z = rz c2x
  T ty, tz;                 // hx/hy, hx/hz: d1y = ty d1x, d1z = tz d1x
  int norb, nk;
  const double* kpts;       // [nk*3]
  double Ap[3];             // A'(t) added to every k
  // projectors
  int natom, nsph;
  const int* atom_off;
  const int* sph_idx;
  const T* sph_beta;        // [nsph*4]
  const T* sph_d;           // [nsph*3]
  const T* atomE;           // [natom*4]
  const int* pt_off;
  const int* pt_ent;
  const int* ent_atom;
  T dV;
  T dt;
  double* rho;              // nullable: rho += 2 w_k |u_out|^2 (FP64 orbitals)
  float* rho32;             // FP32 orbitals: rho32[k][p] += 2 |u_out|^2, folded into rho later
  const double* kw;
  int write_out;            // write psi_out (Taylor) -- predictor passes only accumulate rho
  // shared-memory cell kernels
  int pstride;              // shared-memory plane stride (see smem_plane_stride)
  int nseg, zlen;           // threads per column = nseg, each marching zlen planes
  const int* sph_sidx;      // [nsph] shared-memory index of each sphere entry
  int nsp;                  // unique sphere points
  const int* sp_pt;         // [nsp] global index
  const int* sp_off;        // [nsp+1]
  double Ap_obs[3];         // A' for the fused observables
  double* obs;              // nullable: per-orbital {norm, jloc[3], jnl[3], 0}
  int obs_at_start;         // 1: observables of the input orbital (first stage), 0: of the output
  C* backup;                // nullable: copy of the input orbitals, written while they are loaded
  // batches of cells (multiscale): orbitals are [ncell][nk][norb], potentials [ncell][npts]
  int ncell;                // cells in the batch (1 for a single system)
  long long vstride;        // offset of a cell's potential (0: one potential shared by all)
  const double* Ap_cell;    // nullable: [ncell][3] A' per cell, replaces Ap
  const double* Ap_obs_cell;// nullable: [ncell][3], replaces Ap_obs
  int cell_variant;         // Taylor stages: 0 two buffers, 1 one buffer swept in place, 2 two
                            // buffers with the grid size fixed at compile time (smem_orbital_geom_ok),
                            // 3 one buffer swept in place with the grid size fixed (FP32)
};

// Orbital kernels (k_orbital.cu)
// Shared-memory cell kernels.  mode 0: H u; 1: T4 (Horner) with optional density and fused
// observables (a.obs); 2: observables of u (norm, current, <u|H|u> with a.V) into a.obs.
// scratch = [norb_tot][npts] global buffer, needed only when smem_orbital_needs_scratch().
// Mode 1 with a.cell_variant = 1 sweeps one shared-memory buffer in place (smem_orbital_ip_ok).
template <typename T>
cudaError_t launch_smem_orbital(const OrbArgs<T>& a, int mode, typename Cplx<T>::type* scratch,
                                cudaStream_t s);
template <typename T>
bool smem_orbital_fits(int nz, int pstride, int nsph, int natom);
template <typename T>
bool smem_orbital_needs_scratch(int nz, int pstride, int nsph, int natom);
template <typename T>
bool smem_orbital_ip_ok(int nx, int ny, int nz, int pstride, int nsph, int natom, int periodic);
// Mode 1 with a.cell_variant = 2: a periodic grid of a size built into the kernels (20^3, 16^3)
template <typename T>
bool smem_orbital_geom_ok(int nx, int ny, int nz, int pstride, int nsph, int natom, int periodic, int nseg,
                          int zlen);
// Mode 1 with a.cell_variant = 3: the same grids swept in place, FP32 (two CTAs per SM)
template <typename T>
bool smem_orbital_geom_ip_ok(int nx, int ny, int nz, int pstride, int nsph, int natom, int periodic, int nseg,
                             int zlen);
// column segments of the cell kernels; elem_bytes = bytes of one complex value (8: FP32, 16: FP64)
void cell_split(int nx, int ny, int nz, int elem_bytes, int* nseg, int* zlen);

// Large isolated grids (k_tile.cu): one Horner stage / H application per launch.
template <typename T>
struct TileArgs {
  using C = typename Cplx<T>::type;
  int nx, ny, nz, npts, norb_tot;
  const C* psi;             // Horner base (mode 1)
  C* out;
  const T* V;               // [npts]
  T c2x[5], c2y[5], c2z[5]; // -1/2 FD2[m] / h^2
  T diag;                   // c2x[0] + c2y[0] + c2z[0]
  T ry, rz;                 // hx^2 / hy^2 and hx^2 / hz^2 (c2y = ry c2x, c2z = rz c2x)
  T coef;                   // dt / m (mode 1)
  int* err;                 // device error word (TDKS_ETIMEOUT on a timed-out wait)
  long long wait_limit;     // polls per mbarrier wait before giving up (TDKS_ETIMEOUT)
  int stop_after;           // >= 0: the producer issues only this many planes (timeout test)
  int variant;              // stencil variant (kernel + L2 prefetch), see launch_tile_stage
  int proj_variant;         // FP32 projection schedule: 0, 1, 2 = 2, 4, 8 warps per CTA
  int prefetch;             // L2 prefetch distance in planes (set by launch_tile_stage)
  // projectors (q = 0)
  int natom, nsp;
  const int* atom_off;
  const int* sph_idx;
  const T* sph_beta;
  const T* atomE;
  T dV;
  C* ec;                    // [norb_tot][natom][4] E_p dV c_ap
  const int* sp_pt;
  const int* sp_off;
  const int* pt_ent;
  const int* ent_atom;
};
bool tile_supported(int nx, int ny, int nz, int elem_bytes);
constexpr int kTileVariants = 7;
constexpr int kProjVariants = 3;
// whether a tile variant applies to rows of nx points of elem_bytes-byte complex values
bool tile_variant_ok(int variant, int nx, int elem_bytes);
// local part of one stage: mode 0 out = H_loc vin, mode 1 out = psi + (-i coef) H_loc vin
template <typename T>
cudaError_t launch_tile_stage(const TileArgs<T>& a, const void* vin, int mode, cudaStream_t s);
template <typename T>
cudaError_t launch_tile_project(const TileArgs<T>& a, const typename Cplx<T>::type* v, cudaStream_t s);
// out += V_NL (mode 0) or out += (-i coef) V_NL (mode 1) at sphere points, from a.ec
template <typename T>
cudaError_t launch_tile_scatter(const TileArgs<T>& a, typename Cplx<T>::type* out, int mode, cudaStream_t s);
// per-orbital out[o*8+0] = sum |u|^2 dV, out[o*8+7] = Re sum conj(u) hu dV (hu nullable)
template <typename T>
cudaError_t launch_orbital_dots(const typename Cplx<T>::type* u, const typename Cplx<T>::type* hu,
                                int norb_tot, int npts, double dV, double* out, cudaStream_t s);

// Learned potential predictor (k_nn.cu).  Parameter layout (FP32 masters, as in the oracle):
// W1 [16][4][27], b1 [16], W2 [16][16][27], b2 [16], W3 [1][16][27], b3 [1].
constexpr int kNNParams = 9105;
constexpr int kNNOff[6] = {0, 1728, 1744, 8656, 8672, 9104};
struct NNGrid { int nx, ny, nz, npts, periodic; };
struct NNBuffers {
  unsigned short *x0, *a1, *a2;                   // BF16 conv inputs [4|16|16][npts]
  float *y1, *y2, *out, *target, *dout, *dy1, *dy2, *part;
  float *params, *grad, *m, *v, *wq;              // [kNNParams]; wq = BF16-rounded params
  double* stats;                                  // rms D1, rms D2, rms D3, mean V0, rms(V0 - mean)
  double* loss;                                   // accumulator
  double* red;                                    // [304][5] grid_sum partials of the statistics
  unsigned* ticket;                               // grid_sum ticket (zero between launches)
  unsigned* bar;                                  // [2] grid-barrier counters of the fused prediction (zero between launches)
  uint4* wpack;                                   // shared-memory image of the prediction's weights
  int* err;                                       // context error word (TDKS_ETIMEOUT of a barrier wait)
};
int nn_part_blocks(int npts);
// channel_last: inputs for nn_forward with a prediction epilogue (which reads them channel-last)
cudaError_t nn_inputs(const NNBuffers& B, const NNGrid& g, const double* V0, const double* V1,
                      const double* V2, const double* V3, const double* Vnext, cudaStream_t s,
                      bool channel_last = false);
// Optional epilogue of the last layer: vpred = cubic(V0..V3) + s3 * out (the predictor's mode 2).
// With it the layers run on channel-last inputs and activations (nn_inputs with channel_last) and
// leave no pre-activations for a backward pass.
struct NNPredict {
  const double *V0, *V1, *V2, *V3;
  double* vpred;
  // optional (nn_predict_fused): also the corrector's step potential V_loc + (V_Hxc(t) + V~)/2 into
  // vstep64 and, if not null, its FP32 copy vstep32
  const double* vloc = nullptr;
  const double* vhxc = nullptr;
  double* vstep64 = nullptr;
  float* vstep32 = nullptr;
};
cudaError_t nn_forward(const NNBuffers& B, const NNGrid& g, cudaStream_t s, const NNPredict* pred = nullptr);
// The prediction V~ = cubic + s3 * NN in one cooperative launch (statistics, inputs and three layers
// separated by grid barriers whose waits give up after wait_limit polls and set *B.err).  Same values
// as nn_inputs + nn_forward(pred) up to the FP32 summation order of the tensor-core layer.
cudaError_t nn_predict_fused(const NNBuffers& B, const NNGrid& g, const NNPredict& pr, long long wait_limit,
                             cudaStream_t s);
cudaError_t nn_loss(const NNBuffers& B, const NNGrid& g, double* loss_acc, cudaStream_t s);
cudaError_t nn_backward(const NNBuffers& B, const NNGrid& g, cudaStream_t s);   // grad +=
cudaError_t nn_adam(const NNBuffers& B, float lr, int t, float gscale, cudaStream_t s);
cudaError_t nn_round_weights(const NNBuffers& B, cudaStream_t s);
size_t nn_wpack_bytes();   // size of NNBuffers::wpack
// vpred: mode 0 = 2 V0 - V1, 1 = cubic 4 V0 - 6 V1 + 4 V2 - V3, 2 = cubic + s3 * out
cudaError_t nn_apply(const NNBuffers& B, const NNGrid& g, const double* V0, const double* V1,
                     const double* V2, const double* V3, int mode, double* vpred, cudaStream_t s);
// partials: [304][2] doubles, ticket: one unsigned that is zero between launches (grid_sum)
cudaError_t launch_residual(const double* Vnew, const double* Vpred, int n, double* partials, unsigned* ticket,
                            double* res, cudaStream_t s);
// Device-side acceptance of a predicted potential (a kernel inside a captured graph that owns `handle`):
// vhxc <- vnew and vnext <- vnew (the potential history's next slot) if *res <= thr (finite), else
// *fb += 1 and the conditional `handle` is set to 1 (0 when accepted).
cudaError_t launch_decide(const double* res, double thr, const double* vnew, double* vhxc, double* vnext, int n,
                          double* fb, cudaGraphConditionalHandle handle, cudaStream_t s);
// dst[0..5] <- v[0..5] (six doubles passed by value, so the host buffer may change right after the call)
cudaError_t launch_store6(double* dst, const double v[6], cudaStream_t s);

// Grid kernels (k_grid.cu)
// The misfit of a predicted potential, sqrt(sum (V - vpred)^2 / sum V^2) over the points of V (as
// launch_residual forms it), when the Hartree solve can form it in its last launch: partials
// [304][2] and ticket as for grid_sum; done is set to 1 when it did.  With decide set (inside a
// step graph) that launch also takes the decision k_decide takes: the potential goes to vnext as
// well, and the last CTA counts a fallback in *fb and sets the graph's conditional `handle` to 1
// when the misfit is above thr or not finite (0 otherwise).
struct ResidualArgs {
  const double* vpred;
  double* partials;
  unsigned* ticket;
  double* res;
  int done;
  int decide;
  double thr;
  double* vnext;
  double* fb;
  cudaGraphConditionalHandle handle;
};
// Hartree + exchange in five fused FFT line passes (three for periodic boxes whose xy-plane fits in
// shared memory): vhxc = V_H[rho] (+ V_x[rho] if xc).  work: the transform box m^3 per cell (m = n
// periodic, 2n isolated); batch: cells (periodic only); ghat: the periodic Poisson factors
// (launch_poisson_table) or the Hockney spectrum.  plane_cl >= 2 (one periodic cell): the xy-plane
// passes split each plane over a cluster of plane_cl CTAs (hartree_plane_cluster).
cudaError_t launch_hartree_xc_fused(double2* work, const int m[3], const int n[3], int batch, int periodic,
                                    const double h[3], const double* ghat, double gscale,
                                    double2* const tw[3], const int* const rad[3], const int nrad[3],
                                    const double* rho, int xc, double* vhxc, cudaStream_t s,
                                    int* nlaunch = nullptr, int plane_cl = 0, ResidualArgs* resid = nullptr);
// Cluster size for the xy-plane passes of one periodic cell of transform box m: the largest of 8 .. 2
// whose clusters (one CTA per SM) are all resident at once, 0 where the split does not apply.
int hartree_plane_cluster(const int m[3], int batch, int periodic);
// batch = number of consecutive [dims2][dims1][dims0] arrays transformed together
// lim_lo / lim_hi > 0: transform only the lines whose two other coordinates (lo: the faster of
// them, hi: the slower, batch included for the last axis) are below the limits
cudaError_t launch_fft_axis(double2* data, const int dims[3], int axis, int dir,
                            const double2* tw, const int* radices, int nrad, cudaStream_t s,
                            int batch = 1, int lim_lo = 0, int lim_hi = 0);
cudaError_t launch_pack_real(const double* src, const int n[3], double2* dst, const int m[3],
                             cudaStream_t s);
cudaError_t launch_poisson_scale_periodic(double2* data, const int n[3], const double h[3],
                                          cudaStream_t s, int batch = 1);
cudaError_t launch_scale_by_real(double2* data, const double* ghat, double scale, size_t count,
                                 cudaStream_t s);
// vhxc = scale_h * Re(fft[crop]) (if hartree) + V_x[rho] (if xc)
cudaError_t launch_hxc_epilogue(const double2* fft, const int m[3], const double* rho,
                                const int n[3], double scale_h, int hartree, int xc,
                                double* vhxc, cudaStream_t s);
// vstep64 = vloc + a*v1 + b*v2 (v2 nullable), and vstep32 = (float)vstep64 (nullable);
// v1, v2, v64, v32 hold `batch` potentials of npts points, vloc one shared potential
cudaError_t launch_combine_potential(const double* vloc, const double* v1, double a,
                                     const double* v2, double b, double* v64, float* v32,
                                     int npts, cudaStream_t s, int batch = 1);
template <typename T>
cudaError_t launch_density(const typename Cplx<T>::type* psi, int nk, int norb, int npts,
                           const double* kw, double* rho, cudaStream_t s);
template <typename T>
cudaError_t launch_kick(typename Cplx<T>::type* psi, int norb_tot, const int n[3],
                        const double h[3], int periodic, const double kappa[3], cudaStream_t s);
cudaError_t launch_vloc_isolated(double* v, const int n[3], const double h[3],
                                 const double* atoms /*[natom*5]: R, Z, sigma*/, int natom,
                                 cudaStream_t s);
cudaError_t launch_hockney_kernel(double2* g, const int m[3], const int n[3], const double h[3],
                                  double g0, cudaStream_t s);
cudaError_t launch_real_part(const double2* src, double* dst, size_t count, double scale,
                             cudaStream_t s);
// t[(z m1 + y) m0 + x] = 4 pi / G^2 / (m0 m1 m2) of the periodic box m x h, 0 at G = 0
cudaError_t launch_poisson_table(double* t, const int m[3], const double h[3], cudaStream_t s);
// dipole: partials then final (deterministic two-pass); out[3..5] = d, out[6] = int rho
// out[3..5] = dipole, out[6] = electron count; partials: [304][4] doubles, ticket: grid_sum ticket
cudaError_t launch_dipole(const double* rho, const double* rho0, const int n[3], const double h[3],
                          int periodic, double* partials, unsigned* ticket, double* out,
                          cudaStream_t s);
// J from per-orbital observables; writes out[c*8 + 0..2] = J of cell c (zero if isolated)
cudaError_t launch_reduce_current(const double* orb_obs, int nk, int norb, const double* kw,
                                  double inv_omega, int periodic, double* out, cudaStream_t s,
                                  int ncell = 1);
// 1D Maxwell leapfrog (Eq. Maxwell_ms) with Mur boundaries; A'(X) of the cells at t+dt/2 and t+dt
// Ground-state subspace kernels (k_scf.cu): out[k][i][j] = dV sum conj(A_i) B_j;
// out[k][j] = a V_j + c0 U_j + b sum_i U_i M[k][i][j]; vin <- vout <- vin + mix (vout - vin).
template <typename T>
cudaError_t launch_gram(const typename Cplx<T>::type* A, const typename Cplx<T>::type* B, int nk, int norb, int npts,
                        double dV, double2* out, cudaStream_t s);
template <typename T>
cudaError_t launch_basis(const typename Cplx<T>::type* U, const typename Cplx<T>::type* V, const double2* M, int nk,
                         int norb, int npts, double a, double c0, double b, typename Cplx<T>::type* out,
                         cudaStream_t s);
cudaError_t launch_mix_potential(double* vin, double* vout, long long n, double mix, cudaStream_t s);
// out = a A + b B + g C over n complex values (Cv may be NULL when g = 0)
template <typename T>
cudaError_t launch_lincomb3(const typename Cplx<T>::type* A, const typename Cplx<T>::type* B,
                            const typename Cplx<T>::type* Cv, double a, double b, double g, long long n,
                            typename Cplx<T>::type* out, cudaStream_t s);

// TB-mBJ exchange (k_mbj.cu): V += v_x^mBJ[rho, tau~ of u]; c = c_fixed (> 0) or computed into *c_dev.
// part: [nchunk][5][npts] doubles; partials / ticket: a grid_sum work area.  nlaunch: kernels launched.
int mbj_chunks(long long npts, int norb_tot);
template <typename T>
cudaError_t launch_mbj(const typename Cplx<T>::type* u, int nk, int norb, const int n[3], int periodic,
                       const double h[3], const double* kpts, const double* kw, const double* rho, double c_fixed,
                       double* part, int nchunk, double* partials, unsigned* ticket, double* c_dev, double* V,
                       cudaStream_t s, int* nlaunch);

// longitudinal geometry: one leapfrog step of A'_ind from J(t_n) = step_obs[0..2] (see k_grid.cu)
cudaError_t launch_longitudinal(const double* step_obs, double* lg, int first, double dt, const double ext_mid[3],
                                const double ext_end[3], double* ap_mid, double* ap_end, cudaStream_t s);
cudaError_t launch_maxwell(const double* A_prev, const double* A_now, double* A_next, const double* I,
                           int nX, int m0, int ncell, double c_dt_dX, double src, double inv_c,
                           double* ap_mid, double* ap_end, cudaStream_t s);
// I[m0 + c] = step_obs[c*8 + 2]
cudaError_t launch_ms_current(const double* step_obs, int ncell, int m0, double* I, cudaStream_t s);
cudaError_t launch_f32_from_f64(const double* src, float* dst, size_t count, cudaStream_t s);
// rho[c][p] = sum_k w_k rho32[c][k][p] in FP64 (fixed order); wsplit[2k], wsplit[2k+1]: w_k as a
// float pair, hi = (float)w_k and lo = (float)(w_k - hi)
cudaError_t launch_fold_density(const float* rho32, int nk, int npts, const float* wsplit, double* rho,
                                cudaStream_t s, int ncell = 1);

}  // namespace tdks
