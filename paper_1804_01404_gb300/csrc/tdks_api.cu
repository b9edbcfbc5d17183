// C ABI entry points of libtdks: context set-up and the orchestration of one TDKS step.
// All arithmetic of the step runs in the kernels of k_orbital.cu and k_grid.cu; this file only
// validates arguments, owns device buffers and enqueues launches on the context's stream.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "host_linalg.h"
#include "tdks_internal.h"

using namespace tdks;

namespace {
thread_local std::string g_err;

tdks_status fail(tdks_status s, const std::string& msg) {
  g_err = msg;
  return s;
}
}  // namespace

void tdks::set_last_error(const char* msg) { g_err = msg; }

namespace {
// seeded uniform numbers (splitmix64) for initial network parameters and buffer states
unsigned long long splitmix64(unsigned long long& x) {
  unsigned long long z = (x += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
double uniform01(unsigned long long& x) { return (splitmix64(x) >> 11) * (1.0 / 9007199254740992.0); }
}  // namespace

#define TDKS_CUDA(call)                                                                    \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail(TDKS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));         \
  } while (0)

#define TDKS_TRY(expr)                      \
  do {                                      \
    tdks_status s_ = (expr);                \
    if (s_ != TDKS_OK) return s_;           \
  } while (0)

// One pulse of Eq. (pulse), delayed: A'(t) = A0 cos^2[pi (t' - T/2)/T] sin[-omega (t' - T/2) - 2 pi cep],
// t' = t - delay, 0 < t' < T.
struct PulseDef {
  double A0[3], omega, T, cep, delay;
};
constexpr int kMaxPulses = 8;

struct tdks_ctx {
  tdks_grid grid{};
  tdks_cell cell_in{};
  std::vector<tdks_atom> atoms_in;
  std::vector<tdks_projector> proj_in;
  double vnl_bound = 0.0;        // upper bound of ||V_NL|| (Gershgorin on the projector overlaps)
  int npts = 0, nk = 0, norb = 0, ncell = 1;
  // multiscale: A(X) at three time levels (ring), cell currents I(X), per-cell A'
  int nX = 0, m0 = 0, ms_head = 0;
  double dX = 0;
  bool ms_ready = false;
  double *d_A[3] = {nullptr, nullptr, nullptr}, *d_I = nullptr, *d_ap_mid = nullptr, *d_ap_end = nullptr;
  const double *cur_ap_mid = nullptr, *cur_ap_end = nullptr;
  tdks_options opt{};
  double dV = 0, omega = 0;
  std::vector<double> kpts, kw;
  cudaStream_t stream = nullptr;
  // field
  int field_kind = TDKS_FIELD_NONE;
  double A0[3] = {0, 0, 0};                 // TDKS_FIELD_STEP
  std::vector<PulseDef> pulses;             // TDKS_FIELD_PULSE: A' is their sum
  std::vector<double> ftable;               // TDKS_FIELD_TABLE: [nt][3] samples of A'
  double tab_t0 = 0.0, tab_dt = 0.0;
  int longitudinal = 0, lg_first = 1;       // longitudinal geometry (tdks_set_longitudinal)
  // TB-mBJ exchange (xc = 3): c fixed (> 0) or from the density; per-chunk kinetic-density sums;
  // the predictor's orbitals (their kinetic energy density enters the predicted potential)
  double mbj_c_fixed = 0.0;
  double* d_mbj_c = nullptr;
  double* d_mbj_part = nullptr;
  int mbj_nchunk = 0;
  void* d_porb = nullptr;
  double* d_lg = nullptr;                   // {A'_ind^n[3], A'_ind^{n-1}[3]}
  // projector tables
  int natom = 0, nsph = 0;
  int *d_atom_off = nullptr, *d_sph_idx = nullptr, *d_pt_off = nullptr, *d_pt_ent = nullptr,
      *d_ent_atom = nullptr, *d_sph_sidx = nullptr, *d_sp_pt = nullptr, *d_sp_off = nullptr;
  int nsp = 0, pstride = 0, nseg = 1, zlen = 1;
  double *d_beta64 = nullptr, *d_d64 = nullptr, *d_E64 = nullptr;
  float *d_beta32 = nullptr, *d_d32 = nullptr, *d_E32 = nullptr;
  double *d_kpts = nullptr, *d_kw = nullptr;
  float* d_kwsplit = nullptr;    // [nk][2]: each k weight as a float pair (the density fold)
  // grid arrays
  double *d_vloc = nullptr, *d_vhxc = nullptr, *d_vpred = nullptr, *d_rho = nullptr,
         *d_rho0 = nullptr, *d_rho_tmp = nullptr, *d_v64 = nullptr;
  float* d_v32 = nullptr;
  float* d_rho32 = nullptr;      // [nk][npts] per-k FP32 density partials (FP32 orbitals); zero
                                 // outside an orbital kernel and its fold (zeroed after each fold)
  bool defer_r32_zero = false;   // the caller zeroes d_rho32 after the fold (a parallel graph branch)
  void* d_scratch = nullptr;     // [norb_tot][npts] complex, only for cells whose two copies exceed smem
  // large isolated grids (tile kernels): two Horner buffers and the projection coefficients
  bool tiled = false;
  int tile_variant[2] = {0, 0};  // stencil variant of the tiled path for H v / Horner stages
  int proj_variant = 1;          // FP32 projection schedule of the tiled path (2, 4, 8 warps per CTA)
  float proj_ms[kProjVariants] = {-1.f, -1.f, -1.f};   // its tuning times (-1: not timed)
  long long wait_limit = 1LL << 22;  // polls per device-side wait of the tile kernels
  int stop_after = -1;              // timeout test: planes the tile producer issues (-1: all)
  float tile_ms[2][kTileVariants] = {{-1.f, -1.f, -1.f, -1.f, -1.f, -1.f, -1.f},
                                     {-1.f, -1.f, -1.f, -1.f, -1.f, -1.f, -1.f}};
  int cell_variant = 0;          // Taylor launches of the cell kernels: 0 two buffers, 1 in-place sweep,
                                 // 2 two buffers with the grid size built in, 3 in-place sweep with it
  cudaStream_t side = nullptr;   // tile path: the projections run here beside the stencil
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  float cell_ms[4] = {-1.f, -1.f, -1.f, -1.f};  // tuning time of one Taylor launch per variant (-1: not available)
  void *d_bufA = nullptr, *d_bufB = nullptr, *d_ec = nullptr;
  int* d_err = nullptr;
  bool have_rho0 = false, have_potential = false;
  // FFT
  int m[3] = {0, 0, 0};
  std::vector<int> rad[3];
  double2* d_fft = nullptr;
  double2* d_tw[3] = {nullptr, nullptr, nullptr};
  double* d_ghat = nullptr;
  ResidualArgs* res_args = nullptr;  // set around a predicted step's Hartree solve (see predicted_main)
  // while a step graph is captured: its conditional handle, and whether the Hartree solve's last
  // launch took the decision (then the graph has no k_decide and its V_Hxc went straight to d_vhxc)
  bool cap_decide = false;
  cudaGraphConditionalHandle cap_handle = 0;
  bool cap_decided = false;
  int plane_cl = 0;               // cluster size of the Hartree xy-plane passes (0: one CTA per plane)
  // observables
  double* d_orb_obs = nullptr;   // [nk*norb*8]
  double* d_step_obs = nullptr;  // [8]: J[3], d[3], N
  double* d_partials = nullptr;   // [304][4] grid_sum partials (residual, dipole)
  unsigned* d_ticket = nullptr;   // grid_sum ticket, zero between launches
  double* d_partials_obs = nullptr;   // the same for the dipole of a step graph's parallel branch
  unsigned* d_ticket_obs = nullptr;
  int red_blocks = 0;
  std::vector<void*> allocs;
  // potential history (V_Hxc at t, t-dt, t-2dt, t-3dt) and the predictor
  double* d_vhist = nullptr;     // [4][npts] ring
  int hist_head = 0, hist_count = 0;
  int pred_mode = TDKS_PRED_PC;
  double pred_thr = 1e-5;
  double* d_vnew = nullptr;      // V_Hxc(t+dt) of a predicted step before acceptance
  double* d_resid = nullptr;     // device residual
  double* h_resid = nullptr;     // pinned host buffer [16] (step observables, misfit, fallbacks; c of TB-mBJ)
  void* d_backup = nullptr;      // orbitals at t (predicted steps)
  void* cur_backup = nullptr;    // set while the corrector of a predicted step writes the backup
  double fallbacks = 0, last_resid = 0;
  // Predicted steps run as one CUDA graph per slot of the potential history ring (the slot sets which
  // buffers hold V_Hxc(t .. t-3dt)): prediction, corrector, Hartree-exchange, misfit, the decision
  // kernel and a conditional node whose body restores the orbitals and runs the plain
  // predictor-corrector step, then the history update and the observables.  The vector potentials
  // come from device memory, so a graph serves every step with the same orbital array and settings.
  struct Rec { int phase; cudaEvent_t a, b; };
  struct StepGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<Rec> recs;       // phase events recorded by the graph (profiling on)
    long long launches = 0;      // launches of one execution without the fallback body
    long long calls[TDKS_NPHASE] = {0};
    bool pending = false;        // recs hold times of an execution not yet added to ms[]
  } sg[4];
  struct StepKey {
    const void* u = nullptr;
    double dt = 0, thr = 0, mbj_c = 0;
    int mode = -1, lg = -1, has_obs = -1, obs_start = -1, cell_variant = -1, tile0 = -1, tile1 = -1, prof = -1;
    int proj = -1;
    bool operator==(const StepKey& o) const {
      return u == o.u && dt == o.dt && thr == o.thr && mbj_c == o.mbj_c && mode == o.mode && lg == o.lg &&
             has_obs == o.has_obs && obs_start == o.obs_start && cell_variant == o.cell_variant && tile0 == o.tile0 &&
             tile1 == o.tile1 && prof == o.prof && proj == o.proj;
    }
  } sg_key;
  // multiscale steps as graphs, one per rotation of the three A levels (c->ms_head), built from the
  // second tdks_ms_step on (the first runs on the stream)
  StepGraph msg[3];
  struct MsKey {
    const void* u = nullptr;
    double dt = 0, mbj_c = 0;
    int cell_variant = -1, tile0 = -1, tile1 = -1, prof = -1;
    bool operator==(const MsKey& o) const {
      return u == o.u && dt == o.dt && mbj_c == o.mbj_c && cell_variant == o.cell_variant && tile0 == o.tile0 &&
             tile1 == o.tile1 && prof == o.prof;
    }
  } msg_key;
  long long ms_steps = 0;        // multiscale steps since tdks_ms_init / tdks_set_state
  long long body_launches = 0;   // launches of the fallback body
  long long body_calls[TDKS_NPHASE] = {0};   // phase calls of the fallback body
  int step_graph = 1;            // predicted steps as step graphs (1) or stream launches with a host decision (0)
  std::vector<Rec>* cap_recs = nullptr;   // set while a step graph is captured with profiling on
  cudaStream_t cap = nullptr, cap2 = nullptr;   // private streams the graphs are captured on
  cudaStream_t side2 = nullptr;      // side stream of the tile path inside a fallback body
  cudaStream_t body_side = nullptr;  // set to side2 while a fallback body is captured
  cudaStream_t obs_side = nullptr;   // parallel branch of a step graph: J and the dipole
  cudaEvent_t ev_obs_fork = nullptr, ev_obs_join = nullptr;
  double* d_apf = nullptr;       // [6] A'(t+dt/2) and A' of the observables, read by the step graph
  double* d_fb = nullptr;        // fallback count (device)
  double fb_seen = 0;            // fallbacks already added to the launch count
  bool nn_ready = false;
  NNBuffers nn{};
  int nn_step = 0;
  // profiling
  bool profiling = false;
  bool prof_stencil_only = false;   // record events around the orbital stencil kernel launches only
  long long launches = 0;
  long long calls[TDKS_NPHASE] = {0};
  double ms[TDKS_NPHASE] = {0};
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> event_pool;
};

namespace {

template <typename P>
tdks_status dalloc(tdks_ctx* c, P** p, size_t count) {
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(P));
  if (e != cudaSuccess) return fail(TDKS_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  c->allocs.push_back((void*)*p);
  return TDKS_OK;
}

template <typename P>
tdks_status upload(tdks_ctx* c, P** p, const std::vector<P>& h) {
  TDKS_TRY(dalloc(c, p, h.size()));
  if (!h.empty()) TDKS_CUDA(cudaMemcpyAsync(*p, h.data(), h.size() * sizeof(P), cudaMemcpyHostToDevice, c->stream));
  return TDKS_OK;
}

void field_at(const tdks_ctx* c, double t, double out[3]) {
  out[0] = out[1] = out[2] = 0.0;
  if (!c->grid.periodic) return;
  if (c->field_kind == TDKS_FIELD_STEP) {
    if (t > 0.0) for (int a = 0; a < 3; ++a) out[a] = c->A0[a];
  } else if (c->field_kind == TDKS_FIELD_PULSE) {
    for (const PulseDef& p : c->pulses) {
      const double tt = t - p.delay;
      if (tt > 0.0 && tt < p.T) {
        const double env = std::cos(kPi * (tt - 0.5 * p.T) / p.T);
        const double s = std::sin(-p.omega * (tt - 0.5 * p.T) - 2.0 * kPi * p.cep);
        for (int a = 0; a < 3; ++a) out[a] += p.A0[a] * env * env * s;
      }
    }
  } else if (c->field_kind == TDKS_FIELD_TABLE) {
    // linear between the samples t0 + i dt, the end samples outside
    const int nt = (int)(c->ftable.size() / 3);
    const double x = (t - c->tab_t0) / c->tab_dt;
    if (nt == 1 || x <= 0.0) {
      for (int a = 0; a < 3; ++a) out[a] = c->ftable[a];
    } else if (x >= nt - 1) {
      for (int a = 0; a < 3; ++a) out[a] = c->ftable[3 * (nt - 1) + a];
    } else {
      const int i = (int)std::floor(x);
      const double f = x - i;
      for (int a = 0; a < 3; ++a) out[a] = (1.0 - f) * c->ftable[3 * i + a] + f * c->ftable[3 * (i + 1) + a];
    }
  }
}

template <typename T>
OrbArgs<T> make_args(const tdks_ctx* c, const void* in, void* out, const T* V, const double Ap[3],
                     double dt, double* rho, int write_out) {
  OrbArgs<T> a;
  std::memset(&a, 0, sizeof(a));
  using C = typename Cplx<T>::type;
  a.psi_in = static_cast<const C*>(in);
  a.psi_out = static_cast<C*>(out);
  a.V = V;
  a.nx = c->grid.n[0]; a.ny = c->grid.n[1]; a.nz = c->grid.n[2];
  a.npts = c->npts;
  a.periodic = c->grid.periodic;
  for (int m = 0; m < 5; ++m) {
    a.c2x[m] = (T)(-0.5 * kFD2[m] / (c->grid.h[0] * c->grid.h[0]));
    a.c2y[m] = (T)(-0.5 * kFD2[m] / (c->grid.h[1] * c->grid.h[1]));
    a.c2z[m] = (T)(-0.5 * kFD2[m] / (c->grid.h[2] * c->grid.h[2]));
  }
  for (int m = 0; m < 4; ++m) {
    a.d1x[m] = (T)(kFD1[m] / c->grid.h[0]);
    a.d1y[m] = (T)(kFD1[m] / c->grid.h[1]);
    a.d1z[m] = (T)(kFD1[m] / c->grid.h[2]);
  }
  {
    const double hx = c->grid.h[0], hy = c->grid.h[1], hz = c->grid.h[2];
    a.ry = (T)(hx * hx / (hy * hy));
    a.rz = (T)(hx * hx / (hz * hz));
    a.ty = (T)(hx / hy);
    a.tz = (T)(hx / hz);
  }
  a.norb = c->norb; a.nk = c->nk;
  a.kpts = c->d_kpts;
  for (int i = 0; i < 3; ++i) a.Ap[i] = Ap ? Ap[i] : 0.0;
  a.natom = c->natom; a.nsph = c->nsph;
  a.atom_off = c->d_atom_off; a.sph_idx = c->d_sph_idx;
  a.ncell = c->ncell;
  a.vstride = c->ncell > 1 ? c->npts : 0;
  a.Ap_cell = c->cur_ap_mid;
  a.Ap_obs_cell = c->cur_ap_end;
  a.backup = static_cast<C*>(c->cur_backup);
  if (sizeof(T) == 8) {
    a.sph_beta = (const T*)c->d_beta64; a.sph_d = (const T*)c->d_d64; a.atomE = (const T*)c->d_E64;
  } else {
    a.sph_beta = (const T*)c->d_beta32; a.sph_d = (const T*)c->d_d32; a.atomE = (const T*)c->d_E32;
  }
  a.pt_off = c->d_pt_off; a.pt_ent = c->d_pt_ent; a.ent_atom = c->d_ent_atom;
  a.pstride = c->pstride; a.nseg = c->nseg; a.zlen = c->zlen;
  a.sph_sidx = c->d_sph_sidx; a.nsp = c->nsp; a.sp_pt = c->d_sp_pt; a.sp_off = c->d_sp_off;
  a.dV = (T)c->dV;
  a.dt = (T)dt;
  a.rho = rho;
  a.kw = c->d_kw;
  a.write_out = write_out;
  a.cell_variant = c->cell_variant;
  return a;
}

bool is_f32(const tdks_ctx* c) { return c->opt.precision == TDKS_F32; }

double* hist_slot(tdks_ctx* c, int j) {   // V_Hxc(t - j dt)
  return c->d_vhist + (size_t)((c->hist_head - j + 8) % 4) * c->npts;
}

tdks_status hist_push(tdks_ctx* c, const double* v) {
  c->hist_head = (c->hist_head + 1) % 4;
  TDKS_CUDA(cudaMemcpyAsync(hist_slot(c, 0), v, c->npts * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  if (c->hist_count < 4) c->hist_count += 1;
  return TDKS_OK;
}

NNGrid nn_grid(const tdks_ctx* c) {
  return NNGrid{c->grid.n[0], c->grid.n[1], c->grid.n[2], c->npts, c->grid.periodic};
}

cudaEvent_t take_event(tdks_ctx* c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// RAII phase marker: records an event pair on the context stream when profiling is on.
struct Phase {
  tdks_ctx* c;
  int phase;
  cudaEvent_t a = nullptr;
  Phase(tdks_ctx* c_, int p) : c(c_), phase(p) {
    c->calls[p] += 1;
    if (c->profiling && (!c->prof_stencil_only || p == 6) && (a = take_event(c)) != nullptr) record(a);
  }
  ~Phase() {
    if (!a) return;
    cudaEvent_t b = take_event(c);
    if (!b) { c->event_pool.push_back(a); return; }
    record(b);
    (c->cap_recs ? *c->cap_recs : c->recs).push_back({phase, a, b});
  }
  // while a step graph is captured the event becomes an event-record node of the graph
  void record(cudaEvent_t e) {
    if (c->cap_recs) cudaEventRecordWithFlags(e, c->stream, cudaEventRecordExternal);
    else cudaEventRecord(e, c->stream);
  }
};

// V used by the next orbital kernel: V_loc + a * V_Hxc + b * V_pred
// Whether the density of an orbital kernel is written whole (FP32 cell kernels: per-k partials folded
// into rho) rather than accumulated into a zeroed rho (FP64 atomics, the tile path).
bool rho_overwritten(const tdks_ctx* c) { return is_f32(c) && !c->tiled; }

tdks_status set_step_potential(tdks_ctx* c, double a, const double* v2, double b) {
  Phase ph(c, 5);
  TDKS_CUDA(launch_combine_potential(c->d_vloc, c->d_vhxc, a, v2, b, c->d_v64,
                                     is_f32(c) ? c->d_v32 : nullptr, c->npts, c->stream, c->ncell));
  c->launches += 1;
  return TDKS_OK;
}

template <typename T>
TileArgs<T> make_tile_args(const tdks_ctx* c, const T* V) {
  TileArgs<T> a;
  std::memset(&a, 0, sizeof(a));
  a.nx = c->grid.n[0]; a.ny = c->grid.n[1]; a.nz = c->grid.n[2];
  a.npts = c->npts;
  a.norb_tot = c->nk * c->norb;
  a.V = V;
  for (int m = 0; m < 5; ++m) {
    a.c2x[m] = (T)(-0.5 * kFD2[m] / (c->grid.h[0] * c->grid.h[0]));
    a.c2y[m] = (T)(-0.5 * kFD2[m] / (c->grid.h[1] * c->grid.h[1]));
    a.c2z[m] = (T)(-0.5 * kFD2[m] / (c->grid.h[2] * c->grid.h[2]));
  }
  a.diag = a.c2x[0] + a.c2y[0] + a.c2z[0];
  a.ry = (T)((c->grid.h[0] * c->grid.h[0]) / (c->grid.h[1] * c->grid.h[1]));
  a.rz = (T)((c->grid.h[0] * c->grid.h[0]) / (c->grid.h[2] * c->grid.h[2]));
  a.variant = c->tile_variant[0];
  a.proj_variant = c->proj_variant;
  a.wait_limit = c->wait_limit;
  a.stop_after = c->stop_after;
  a.err = c->d_err;
  a.natom = c->natom; a.nsp = c->nsp;
  a.atom_off = c->d_atom_off; a.sph_idx = c->d_sph_idx;
  a.sph_beta = sizeof(T) == 8 ? (const T*)c->d_beta64 : (const T*)c->d_beta32;
  a.atomE = sizeof(T) == 8 ? (const T*)c->d_E64 : (const T*)c->d_E32;
  a.dV = (T)c->dV;
  a.ec = static_cast<typename Cplx<T>::type*>(c->d_ec);
  a.sp_pt = c->d_sp_pt; a.sp_off = c->d_sp_off; a.pt_ent = c->d_pt_ent; a.ent_atom = c->d_ent_atom;
  return a;
}

// Large isolated grids: H u (mode 0) or T4 u (mode 1, Horner through the two work buffers).
template <typename T>
tdks_status tiled_kernel(tdks_ctx* c, int mode, const void* in, void* out, double dt, double* rho,
                         int write_out) {
  using C = typename Cplx<T>::type;
  const T* V = sizeof(T) == 8 ? (const T*)c->d_v64 : (const T*)c->d_v32;
  TileArgs<T> a = make_tile_args<T>(c, V);
  // the projections of the input (side stream) overlap the stencil (context stream); the scatter,
  // which needs both, waits for the projections
  // (while the fallback body of a step graph is captured, the side stream of the enclosing capture
  // is still part of that capture, so the body forks to a second one)
  cudaStream_t side = c->body_side ? c->body_side : c->side;
  auto project = [&](const C* v) -> cudaError_t {
    cudaError_t e = cudaEventRecord(c->ev_fork, c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(side, c->ev_fork, 0);
    if (e == cudaSuccess) e = launch_tile_project<T>(a, v, side);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_join, side);
    return e;
  };
  auto join = [&]() { return cudaStreamWaitEvent(c->stream, c->ev_join, 0); };
  if (mode == 0) {
    a.out = static_cast<C*>(out);
    TDKS_CUDA(project(static_cast<const C*>(in)));
    {
      Phase pk(c, 6);
      TDKS_CUDA(launch_tile_stage<T>(a, in, 0, c->stream));
    }
    TDKS_CUDA(join());
    TDKS_CUDA(launch_tile_scatter<T>(a, a.out, 0, c->stream));
    c->launches += 3;
    return TDKS_OK;
  }
  const C* u = static_cast<const C*>(in);
  C* A = static_cast<C*>(c->d_bufA);
  C* B = static_cast<C*>(c->d_bufB);
  C* fin = write_out ? static_cast<C*>(out) : B;
  C* dst[4] = {A, B, A, fin};
  const C* v = u;
  a.psi = u;
  a.variant = c->tile_variant[1];
  for (int st = 0; st < 4; ++st) {
    a.coef = (T)(dt / (4 - st));
    a.out = dst[st];
    TDKS_CUDA(project(v));
    {
      Phase pk(c, 6);
      TDKS_CUDA(launch_tile_stage<T>(a, v, 1, c->stream));
    }
    TDKS_CUDA(join());
    TDKS_CUDA(launch_tile_scatter<T>(a, a.out, 1, c->stream));
    c->launches += 3;
    v = a.out;
  }
  if (rho) {
    TDKS_CUDA(launch_density<T>(fin, c->nk, c->norb, c->npts, c->d_kw, rho, c->stream));
    c->launches += 1;
  }
  return TDKS_OK;
}

// phase: profiling phase (-1: H u -> hpsi, a written Taylor result -> corrector, else predictor)
tdks_status orbital_kernel(tdks_ctx* c, int mode, const void* in, void* out, const double Ap[3],
                           double dt, double* rho, int write_out, const double* Ap_obs = nullptr,
                           bool obs_start = false, int phase = -1) {
  Phase ph(c, phase >= 0 ? phase : (mode == 0 ? 2 : (write_out ? 1 : 0)));
  if (c->tiled)
    return is_f32(c) ? tiled_kernel<float>(c, mode, in, out, dt, rho, write_out)
                     : tiled_kernel<double>(c, mode, in, out, dt, rho, write_out);
  c->launches += 1;
  if (is_f32(c)) {
    auto a = make_args<float>(c, in, out, c->d_v32, Ap, dt, rho, write_out);
    if (rho) {
      // per-k FP32 partial densities (zero on entry), folded into rho in FP64 afterwards and zeroed
      // again by a memset (cheaper in a step than zeroing them in the fold kernel, measured)
      a.rho = nullptr;
      a.rho32 = c->d_rho32;
    }
    if (Ap_obs) {
      a.obs = c->d_orb_obs;
      a.obs_at_start = obs_start ? 1 : 0;
      for (int i = 0; i < 3; ++i) a.Ap_obs[i] = Ap_obs[i];
    }
    {
      Phase pk(c, 6);
      TDKS_CUDA(launch_smem_orbital<float>(a, mode, static_cast<float2*>(c->d_scratch), c->stream));
    }
    if (rho) {
      TDKS_CUDA(launch_fold_density(c->d_rho32, c->nk, c->npts, c->d_kwsplit, rho, c->stream, c->ncell));
      c->launches += 1;
      if (!c->defer_r32_zero)
        TDKS_CUDA(cudaMemsetAsync(c->d_rho32, 0, sizeof(float) * (size_t)c->ncell * c->nk * c->npts, c->stream));
    }
  } else {
    auto a = make_args<double>(c, in, out, c->d_v64, Ap, dt, rho, write_out);
    if (Ap_obs) {
      a.obs = c->d_orb_obs;
      a.obs_at_start = obs_start ? 1 : 0;
      for (int i = 0; i < 3; ++i) a.Ap_obs[i] = Ap_obs[i];
    }
    {
      Phase pk(c, 6);
      TDKS_CUDA(launch_smem_orbital<double>(a, mode, static_cast<double2*>(c->d_scratch), c->stream));
    }
  }
  return TDKS_OK;
}

tdks_status density(tdks_ctx* c, const void* u, double* rho) {
  const size_t per = (size_t)c->nk * c->norb * c->npts;
  for (int cell = 0; cell < c->ncell; ++cell) {
    c->launches += 1;
    double* r = rho + (size_t)cell * c->npts;
    if (is_f32(c))
      TDKS_CUDA(launch_density<float>(static_cast<const float2*>(u) + cell * per, c->nk, c->norb, c->npts, c->d_kw, r, c->stream));
    else
      TDKS_CUDA(launch_density<double>(static_cast<const double2*>(u) + cell * per, c->nk, c->norb, c->npts, c->d_kw, r, c->stream));
  }
  return TDKS_OK;
}

tdks_status fft3d(tdks_ctx* c, int dir) {
  for (int ax = 0; ax < 3; ++ax)
    TDKS_CUDA(launch_fft_axis(c->d_fft, c->m, ax, dir, c->d_tw[ax], c->rad[ax].data(),
                              (int)c->rad[ax].size(), c->stream, c->ncell));
  c->launches += 3;
  return TDKS_OK;
}

// vhxc = V_H[rho] + V_xc[rho]; u: the orbitals rho comes from (their kinetic energy density
// enters the TB-mBJ exchange of xc = 3, added after the Hartree + correlation kernels)
tdks_status hxc_lda(tdks_ctx* c, const double* rho, double* vhxc);
tdks_status hxc(tdks_ctx* c, const double* rho, double* vhxc, const void* u) {
  TDKS_TRY(hxc_lda(c, rho, vhxc));
  if (c->opt.xc != 3) return TDKS_OK;
  Phase ph(c, 3);
  int nl = 0;
  if (is_f32(c))
    TDKS_CUDA(launch_mbj<float>(static_cast<const float2*>(u), c->nk, c->norb, c->grid.n, c->grid.periodic, c->grid.h,
                                c->d_kpts, c->d_kw, rho, c->mbj_c_fixed, c->d_mbj_part, c->mbj_nchunk, c->d_partials,
                                c->d_ticket, c->d_mbj_c, vhxc, c->stream, &nl));
  else
    TDKS_CUDA(launch_mbj<double>(static_cast<const double2*>(u), c->nk, c->norb, c->grid.n, c->grid.periodic,
                                 c->grid.h, c->d_kpts, c->d_kw, rho, c->mbj_c_fixed, c->d_mbj_part, c->mbj_nchunk,
                                 c->d_partials, c->d_ticket, c->d_mbj_c, vhxc, c->stream, &nl));
  c->launches += nl;
  return TDKS_OK;
}

tdks_status hxc_lda(tdks_ctx* c, const double* rho, double* vhxc) {
  Phase ph(c, 3);
  // a batch of periodic cells is handled as one grid stacked along z for the pointwise kernels
  const int ns[3] = {c->grid.n[0], c->grid.n[1], c->grid.n[2] * c->ncell};
  const int ms[3] = {c->m[0], c->m[1], c->m[2] * c->ncell};
  if (c->opt.hartree) {
    // three (periodic xy planes in shared memory) or five line passes with the packing, the
    // Poisson factor and the exchange epilogue fused in
    const double npad = (double)c->m[0] * c->m[1] * c->m[2];
    const int* rad[3] = {c->rad[0].data(), c->rad[1].data(), c->rad[2].data()};
    const int nrad[3] = {(int)c->rad[0].size(), (int)c->rad[1].size(), (int)c->rad[2].size()};
    int nl = 0;
    TDKS_CUDA(launch_hartree_xc_fused(c->d_fft, c->m, c->grid.n, c->ncell, c->grid.periodic, c->grid.h,
                                      c->d_ghat, c->dV / npad, c->d_tw, rad, nrad, rho, c->opt.xc,
                                      vhxc, c->stream, &nl, c->plane_cl, c->res_args));
    c->launches += nl;
    return TDKS_OK;
  }
  c->launches += 1;
  TDKS_CUDA(launch_hxc_epilogue(c->d_fft, ms, rho, ns, 1.0, 0, c->opt.xc, vhxc, c->stream));
  return TDKS_OK;
}

// per-orbital norm, current and <u|T_q + V_loc + V_NL|u> into d_orb_obs (cell kernel mode 2)
tdks_status orbital_observables(tdks_ctx* c, const void* u, const double Ap[3]) {
  if (c->tiled) {   // isolated: no current; H u with V_loc into the work buffer, then dots
    TDKS_TRY(set_step_potential(c, 0.0, nullptr, 0.0));
    TDKS_TRY(orbital_kernel(c, 0, u, c->d_bufA, Ap, 0.0, nullptr, 1));
    c->launches += 1;
    if (is_f32(c))
      TDKS_CUDA(launch_orbital_dots<float>(static_cast<const float2*>(u), static_cast<const float2*>(c->d_bufA),
                                           c->nk * c->norb, c->npts, c->dV, c->d_orb_obs, c->stream));
    else
      TDKS_CUDA(launch_orbital_dots<double>(static_cast<const double2*>(u), static_cast<const double2*>(c->d_bufA),
                                            c->nk * c->norb, c->npts, c->dV, c->d_orb_obs, c->stream));
    return TDKS_OK;
  }
  c->launches += is_f32(c) ? 2 : 1;
  if (is_f32(c)) {
    TDKS_CUDA(launch_f32_from_f64(c->d_vloc, c->d_v32, c->npts, c->stream));
    auto a = make_args<float>(c, u, nullptr, c->d_v32, Ap, 0.0, nullptr, 0);
    a.obs = c->d_orb_obs;
    TDKS_CUDA(launch_smem_orbital<float>(a, 2, static_cast<float2*>(c->d_scratch), c->stream));
  } else {
    auto a = make_args<double>(c, u, nullptr, c->d_vloc, Ap, 0.0, nullptr, 0);
    a.obs = c->d_orb_obs;
    TDKS_CUDA(launch_smem_orbital<double>(a, 2, static_cast<double2*>(c->d_scratch), c->stream));
  }
  return TDKS_OK;
}

tdks_status check_ctx(const tdks_ctx* c) {
  if (!c) return fail(TDKS_EINVAL, "null context");
  return TDKS_OK;
}

// The calls that form the density-dependent potential from the orbitals need every orbital's density;
// a context that holds one shard of the orbitals (options.norb_total > norb) has only its own.
tdks_status check_whole_set(const tdks_ctx* c, const char* what) {
  if (c->opt.norb_total > c->norb)
    return fail(TDKS_EUNSUPPORTED, std::string(what) + " needs every orbital: this context holds a shard "
                "(norb < norb_total) and this build has no density exchange between shards");
  return TDKS_OK;
}

}  // namespace

// Stencil autotuner of the tiled path: every variant runs the stencil alone (H v, and a Horner stage
// with psi = v) on the zeroed work buffers, one untimed and two timed launches each, and the fastest
// per mode is kept.
tdks_status tune_tile(tdks_ctx* c) {
  c->tile_variant[0] = c->tile_variant[1] = 0;
  if (!c->tiled) return TDKS_OK;
  const int nvar = is_f32(c) ? kTileVariants : 2;   // FP64 has variants 0 and 1
  const size_t n = (size_t)c->npts * c->nk * c->norb;
  const size_t csz = is_f32(c) ? sizeof(float2) : sizeof(double2);
  TDKS_CUDA(cudaMemsetAsync(c->d_bufA, 0, n * csz, c->stream));
  TDKS_CUDA(cudaMemsetAsync(c->d_v32, 0, (size_t)c->npts * sizeof(float), c->stream));
  TDKS_CUDA(cudaMemsetAsync(c->d_v64, 0, (size_t)c->npts * sizeof(double), c->stream));
  cudaEvent_t e0, e1;
  TDKS_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return fail(TDKS_ECUDA, "event"); }
  cudaError_t err = cudaSuccess;
  const int eb = is_f32(c) ? 8 : 16;
  for (int mode = 0; mode < 2 && err == cudaSuccess; ++mode) {
    float best = -1.f;
    for (int v = 0; v < nvar && err == cudaSuccess; ++v) {
      if (!tile_variant_ok(v, c->grid.n[0], eb)) continue;
      auto run = [&]() -> cudaError_t {
        if (is_f32(c)) {
          TileArgs<float> a = make_tile_args<float>(c, c->d_v32);
          a.variant = v;
          a.psi = static_cast<const float2*>(c->d_bufA);
          a.out = static_cast<float2*>(c->d_bufB);
          a.coef = 0.01f;
          return launch_tile_stage<float>(a, c->d_bufA, mode, c->stream);
        }
        TileArgs<double> a = make_tile_args<double>(c, c->d_v64);
        a.variant = v;
        a.psi = static_cast<const double2*>(c->d_bufA);
        a.out = static_cast<double2*>(c->d_bufB);
        a.coef = 0.01;
        return launch_tile_stage<double>(a, c->d_bufA, mode, c->stream);
      };
      err = run();
      if (err == cudaSuccess) err = cudaEventRecord(e0, c->stream);
      for (int r = 0; r < 2 && err == cudaSuccess; ++r) err = run();
      if (err == cudaSuccess) err = cudaEventRecord(e1, c->stream);
      if (err == cudaSuccess) err = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
      if (err != cudaSuccess) break;
      c->tile_ms[mode][v] = 0.5f * ms;
      if (best < 0.f || c->tile_ms[mode][v] < best) { best = c->tile_ms[mode][v]; c->tile_variant[mode] = v; }
    }
  }
  // the schedule of the FP32 tensor-core projection: 2, 4 or 8 warps per CTA over the sphere points
  if (is_f32(c) && c->natom > 0) {
    float best = -1.f;
    for (int v = 0; v < kProjVariants && err == cudaSuccess; ++v) {
      TileArgs<float> a = make_tile_args<float>(c, c->d_v32);
      a.proj_variant = v;
      err = launch_tile_project<float>(a, static_cast<const float2*>(c->d_bufA), c->stream);
      if (err == cudaSuccess) err = cudaEventRecord(e0, c->stream);
      for (int r = 0; r < 3 && err == cudaSuccess; ++r)
        err = launch_tile_project<float>(a, static_cast<const float2*>(c->d_bufA), c->stream);
      if (err == cudaSuccess) err = cudaEventRecord(e1, c->stream);
      if (err == cudaSuccess) err = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
      if (err != cudaSuccess) break;
      c->proj_ms[v] = ms / 3.f;
      if (best < 0.f || c->proj_ms[v] < best) { best = c->proj_ms[v]; c->proj_variant = v; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return fail(TDKS_ECUDA, std::string("tile tuning: ") + cudaGetErrorString(err));
  int h_err = 0;
  TDKS_CUDA(cudaMemcpy(&h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h_err != 0) return fail((tdks_status)h_err, "tile tuning: a stencil kernel gave up waiting for its copies");
  return TDKS_OK;
}

bool cell_ip_ok(const tdks_ctx* c) {
  const int* n = c->grid.n;
  return !c->tiled &&
         (is_f32(c) ? smem_orbital_ip_ok<float>(n[0], n[1], n[2], c->pstride, c->nsph, c->natom, c->grid.periodic)
                    : smem_orbital_ip_ok<double>(n[0], n[1], n[2], c->pstride, c->nsph, c->natom, c->grid.periodic));
}

bool cell_geom_ok(const tdks_ctx* c) {
  const int* n = c->grid.n;
  return !c->tiled &&
         (is_f32(c) ? smem_orbital_geom_ok<float>(n[0], n[1], n[2], c->pstride, c->nsph, c->natom, c->grid.periodic,
                                                  c->nseg, c->zlen)
                    : smem_orbital_geom_ok<double>(n[0], n[1], n[2], c->pstride, c->nsph, c->natom,
                                                   c->grid.periodic, c->nseg, c->zlen));
}

bool cell_geom_ip_ok(const tdks_ctx* c) {
  const int* n = c->grid.n;
  return !c->tiled && is_f32(c) &&
         smem_orbital_geom_ip_ok<float>(n[0], n[1], n[2], c->pstride, c->nsph, c->natom, c->grid.periodic, c->nseg,
                                        c->zlen);
}

bool cell_variant_ok(const tdks_ctx* c, int v) {
  switch (v) {
    case 0: return !c->tiled;
    case 1: return cell_ip_ok(c);
    case 2: return cell_geom_ok(c);
    default: return cell_geom_ip_ok(c);
  }
}

// Times one Taylor launch of each cell-kernel scheme that applies on zero orbitals -- up to 1216 of
// them (eight waves of one CTA per SM) -- and keeps the fastest.  The launch is the corrector's:
// four Horner stages with the per-orbital observables of the context's choice (input or output
// state), no orbital or density output.
tdks_status tune_cell(tdks_ctx* c) {
  c->cell_variant = 0;
  c->cell_ms[0] = c->cell_ms[1] = c->cell_ms[2] = c->cell_ms[3] = -1.f;
  if (!cell_ip_ok(c) && !cell_geom_ok(c)) return TDKS_OK;
  const int nsub = std::min(c->ncell * c->nk * c->norb, 1216);
  const size_t csz = is_f32(c) ? sizeof(float2) : sizeof(double2);
  void* buf = nullptr;
  TDKS_CUDA(cudaMalloc(&buf, csz * (size_t)nsub * c->npts));
  cudaError_t err = cudaMemsetAsync(buf, 0, csz * (size_t)nsub * c->npts, c->stream);
  if (err == cudaSuccess)
    err = is_f32(c) ? cudaMemsetAsync(c->d_v32, 0, (size_t)c->npts * sizeof(float), c->stream)
                    : cudaMemsetAsync(c->d_v64, 0, (size_t)c->npts * sizeof(double), c->stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (err == cudaSuccess) err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  float best = 0.f;
  for (int v = 0; v < 4 && err == cudaSuccess; ++v) {
    if (!cell_variant_ok(c, v)) continue;
    auto run = [&]() -> cudaError_t {
      if (is_f32(c)) {
        auto a = make_args<float>(c, buf, buf, c->d_v32, nullptr, 0.02, nullptr, 0);
        a.ncell = 1; a.nk = 1; a.norb = nsub; a.vstride = 0; a.Ap_cell = a.Ap_obs_cell = nullptr;
        a.backup = nullptr;
        a.obs = c->d_orb_obs;
        a.obs_at_start = c->opt.obs_at_start;
        a.cell_variant = v;
        return launch_smem_orbital<float>(a, 1, static_cast<float2*>(c->d_scratch), c->stream);
      }
      auto a = make_args<double>(c, buf, buf, c->d_v64, nullptr, 0.02, nullptr, 0);
      a.ncell = 1; a.nk = 1; a.norb = nsub; a.vstride = 0; a.Ap_cell = a.Ap_obs_cell = nullptr;
      a.backup = nullptr;
      a.obs = c->d_orb_obs;
      a.obs_at_start = c->opt.obs_at_start;
      a.cell_variant = v;
      return launch_smem_orbital<double>(a, 1, static_cast<double2*>(c->d_scratch), c->stream);
    };
    err = run();
    if (err == cudaSuccess) err = cudaEventRecord(e0, c->stream);
    for (int r = 0; r < 2 && err == cudaSuccess; ++r) err = run();
    if (err == cudaSuccess) err = cudaEventRecord(e1, c->stream);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err != cudaSuccess) break;
    c->cell_ms[v] = 0.5f * ms;
    if (v == 0 || c->cell_ms[v] < best) { best = c->cell_ms[v]; c->cell_variant = v; }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(c->stream);
  cudaFree(buf);
  if (err != cudaSuccess) return fail(TDKS_ECUDA, std::string("cell tuning: ") + cudaGetErrorString(err));
  return TDKS_OK;
}

extern "C" {

const char* tdks_last_error(void) { return g_err.c_str(); }
int tdks_abi_version(void) { return TDKS_ABI_VERSION; }

tdks_status tdks_check_options(const tdks_grid* grid, int nk, int norb, const tdks_options* opts) {
  if (!grid || !opts) return fail(TDKS_EINVAL, "null grid or options");
  if (nk < 1 || norb < 1) return fail(TDKS_EINVAL, "nk and norb must be >= 1");
  if (opts->precision != TDKS_F64 && opts->precision != TDKS_F32)
    return fail(TDKS_EINVAL, "precision must be TDKS_F64 or TDKS_F32");
  if (opts->ncell < 0 || opts->ncell > 65536) return fail(TDKS_EINVAL, "ncell must be in [0, 65536]");
  if (opts->ncell > 1 && !grid->periodic) return fail(TDKS_EINVAL, "ncell > 1 needs a periodic grid");
  for (int a = 0; a < 3; ++a) {
    if (grid->n[a] < 4 || grid->n[a] > 1024) return fail(TDKS_EINVAL, "grid points per axis must be in [4, 1024]");
    if (!(grid->h[a] > 0.0)) return fail(TDKS_EINVAL, "grid spacing must be positive");
  }
  if (opts->obs_at_start != 0 && opts->obs_at_start != 1) return fail(TDKS_EINVAL, "obs_at_start must be 0 or 1");
  if (opts->xc < 0 || opts->xc > 3)
    return fail(TDKS_EINVAL, "xc must be 0 (none), 1 (exchange), 2 (exchange + correlation) or 3 (TB-mBJ exchange + correlation)");
  if (opts->xc == 3 && opts->ncell > 1) return fail(TDKS_EUNSUPPORTED, "xc = 3 (TB-mBJ) needs ncell = 1");
  if (opts->hartree != 0 && opts->hartree != 1) return fail(TDKS_EINVAL, "hartree must be 0 or 1");
  if (opts->norb_total < 0 || opts->norb_offset < 0) return fail(TDKS_EINVAL, "norb_offset and norb_total must be >= 0");
  if (opts->norb_total == 0 && opts->norb_offset != 0)
    return fail(TDKS_EINVAL, "norb_offset needs norb_total (0 means the whole set, offset 0)");
  if (opts->norb_total > 0 && (long long)opts->norb_offset + norb > opts->norb_total)
    return fail(TDKS_EINVAL, "orbital range norb_offset .. norb_offset + norb - 1 exceeds norb_total");
  return TDKS_OK;
}

tdks_status tdks_init(const tdks_grid* grid, const tdks_cell* cell, const tdks_atom* atoms,
                      int natom, const tdks_projector* projectors, int nproj, const double* kpts,
                      const double* kw, int nk, int norb, const tdks_options* opts, void* stream,
                      tdks_ctx** out) {
  if (!out) return fail(TDKS_EINVAL, "out is null");
  *out = nullptr;
  if (!grid || !opts || !kpts || !kw) return fail(TDKS_EINVAL, "null grid, options or k-points");
  if (natom < 0 || (natom > 0 && !atoms)) return fail(TDKS_EINVAL, "bad atom list");
  if (nproj < 0 || (nproj > 0 && !projectors)) return fail(TDKS_EINVAL, "bad projector list");
  TDKS_TRY(tdks_check_options(grid, nk, norb, opts));
  if (grid->periodic) {
    if (!cell) return fail(TDKS_EINVAL, "periodic grid needs a cell");
    for (int a = 0; a < 3; ++a)
      if (std::fabs(cell->L[a] - grid->n[a] * grid->h[a]) > 1e-9 * cell->L[a])
        return fail(TDKS_EINVAL, "cell length differs from n*h");
  }
  double wsum = 0.0;
  for (int k = 0; k < nk; ++k) wsum += kw[k];
  if (std::fabs(wsum - 1.0) > 1e-9) return fail(TDKS_EINVAL, "k-point weights must sum to 1");

  tdks_ctx* c = new tdks_ctx();
  c->grid = *grid;
  c->npts = grid->n[0] * grid->n[1] * grid->n[2];
  c->ncell = opts->ncell > 1 ? opts->ncell : 1;
  c->nk = nk;
  c->norb = norb;
  c->opt = *opts;
  c->dV = grid->h[0] * grid->h[1] * grid->h[2];
  c->omega = c->dV * c->npts;
  c->kpts.assign(kpts, kpts + 3 * nk);
  c->kw.assign(kw, kw + nk);
  c->stream = static_cast<cudaStream_t>(stream);

  auto bail = [&](tdks_status s) { tdks_destroy(c); return s; };

  ProjectorTables T;
  std::string err;
  if (!build_projector_tables(*grid, atoms, natom, projectors, nproj, T, err))
    return bail(fail(TDKS_EINVAL, err));
  // the set-up inputs (the ground-state solver builds a sibling context with a larger orbital block)
  if (cell) c->cell_in = *cell;
  if (natom > 0) c->atoms_in.assign(atoms, atoms + natom);
  if (nproj > 0) c->proj_in.assign(projectors, projectors + nproj);
  // bound on the norm of the nonlocal operator: max |E_p| times the largest row sum of |<beta_i|beta_j>|
  // (Gershgorin), the overlaps bounded pointwise through the point -> entries table
  {
    std::vector<double> row((size_t)T.natom * 4, 0.0);
    double emax = 0.0;
    for (double e : T.E) emax = std::max(emax, std::fabs(e));
    for (size_t pt = 0; pt + 1 < T.pt_off.size(); ++pt)
      for (int e1 = T.pt_off[pt]; e1 < T.pt_off[pt + 1]; ++e1)
        for (int e2 = T.pt_off[pt]; e2 < T.pt_off[pt + 1]; ++e2) {
          const int i = T.pt_ent[e1], j = T.pt_ent[e2];
          double bj = 0.0;
          for (int q = 0; q < 4; ++q) bj += std::fabs(T.beta[4 * (size_t)j + q]);
          for (int p = 0; p < 4; ++p)
            row[(size_t)T.ent_atom[i] * 4 + p] += std::fabs(T.beta[4 * (size_t)i + p]) * bj * c->dV;
        }
    double rmax = 0.0;
    for (double r : row) rmax = std::max(rmax, r);
    c->vnl_bound = emax * rmax;
  }
  c->natom = T.natom;
  c->nsph = (int)T.idx.size();
  c->nsp = (int)T.sp_pt.size();
  c->pstride = smem_plane_stride(*grid);
  cell_split(grid->n[0], grid->n[1], grid->n[2], is_f32(c) ? 8 : 16, &c->nseg, &c->zlen);
  const bool fits = is_f32(c) ? smem_orbital_fits<float>(grid->n[2], c->pstride, c->nsph, c->natom)
                              : smem_orbital_fits<double>(grid->n[2], c->pstride, c->nsph, c->natom);
  if (!fits) {
    const int eb = is_f32(c) ? 8 : 16;
    if (grid->periodic || !tile_supported(grid->n[0], grid->n[1], grid->n[2], eb))
      return bail(fail(TDKS_EUNSUPPORTED,
                       "grid too large for the shared-memory cell kernels; the tiled kernels need an "
                       "isolated grid with nx * element size a multiple of 16 bytes"));
    c->tiled = true;
  }

  tdks_status s;
  if ((s = upload(c, &c->d_atom_off, T.atom_off)) != TDKS_OK) return bail(s);
  if ((s = upload(c, &c->d_sph_idx, T.idx)) != TDKS_OK) return bail(s);
  if ((s = upload(c, &c->d_pt_off, T.pt_off)) != TDKS_OK) return bail(s);
  if ((s = upload(c, &c->d_pt_ent, T.pt_ent)) != TDKS_OK) return bail(s);
  if ((s = upload(c, &c->d_ent_atom, T.ent_atom)) != TDKS_OK) return bail(s);
  {
    const int nxy = grid->n[0] * grid->n[1];
    std::vector<int> sidx(T.idx.size());
    for (size_t i = 0; i < T.idx.size(); ++i) sidx[i] = T.idx[i] + (T.idx[i] / nxy) * (c->pstride - nxy);
    if ((s = upload(c, &c->d_sph_sidx, sidx)) != TDKS_OK) return bail(s);
    if ((s = upload(c, &c->d_sp_pt, T.sp_pt)) != TDKS_OK) return bail(s);
    if ((s = upload(c, &c->d_sp_off, T.sp_off)) != TDKS_OK) return bail(s);
  }
  if ((s = upload(c, &c->d_beta64, T.beta)) != TDKS_OK) return bail(s);
  if ((s = upload(c, &c->d_d64, T.d)) != TDKS_OK) return bail(s);
  if ((s = upload(c, &c->d_E64, T.E)) != TDKS_OK) return bail(s);
  {
    std::vector<float> b(T.beta.begin(), T.beta.end()), d(T.d.begin(), T.d.end()), E(T.E.begin(), T.E.end());
    if ((s = upload(c, &c->d_beta32, b)) != TDKS_OK) return bail(s);
    if ((s = upload(c, &c->d_d32, d)) != TDKS_OK) return bail(s);
    if ((s = upload(c, &c->d_E32, E)) != TDKS_OK) return bail(s);
  }
  if ((s = upload(c, &c->d_kpts, c->kpts)) != TDKS_OK) return bail(s);
  if ((s = upload(c, &c->d_kw, c->kw)) != TDKS_OK) return bail(s);
  {
    std::vector<float> ws(2 * c->kw.size());
    for (size_t k = 0; k < c->kw.size(); ++k) {
      const float hi = (float)c->kw[k];
      ws[2 * k] = hi;
      ws[2 * k + 1] = (float)(c->kw[k] - (double)hi);
    }
    if ((s = upload(c, &c->d_kwsplit, ws)) != TDKS_OK) return bail(s);
  }

  const size_t np = c->npts;
  const size_t npc = np * c->ncell;        // per-cell arrays
  double** grids[] = {&c->d_vhxc, &c->d_vpred, &c->d_rho, &c->d_rho0, &c->d_rho_tmp, &c->d_v64};
  if ((s = dalloc(c, &c->d_vloc, np)) != TDKS_OK) return bail(s);
  for (double** g : grids) {
    if ((s = dalloc(c, g, npc)) != TDKS_OK) return bail(s);
    if (cudaMemsetAsync(*g, 0, npc * sizeof(double), c->stream) != cudaSuccess)
      return bail(fail(TDKS_ECUDA, "memset"));
  }
  if ((s = dalloc(c, &c->d_v32, npc)) != TDKS_OK) return bail(s);
  if ((s = dalloc(c, &c->d_err, 1)) != TDKS_OK) return bail(s);
  if ((s = dalloc(c, &c->d_vhist, 4 * np)) != TDKS_OK) return bail(s);
  if ((s = dalloc(c, &c->d_vnew, npc)) != TDKS_OK) return bail(s);
  // the step observables of every cell, then the misfit (2) and the fallback count: one block, so that
  // tdks_read_step_observables of a single cell is one copy into pinned memory
  if ((s = dalloc(c, &c->d_step_obs, 8 * (size_t)c->ncell + 4)) != TDKS_OK) return bail(s);
  c->d_resid = c->d_step_obs + 8 * (size_t)c->ncell;
  c->d_fb = c->d_resid + 2;
  if (cudaMemsetAsync(c->d_step_obs, 0, (8 * (size_t)c->ncell + 4) * sizeof(double), c->stream) != cudaSuccess)
    return bail(fail(TDKS_ECUDA, "memset"));
  if ((s = dalloc(c, &c->d_apf, 6)) != TDKS_OK) return bail(s);
  if (cudaMallocHost((void**)&c->h_resid, 16 * sizeof(double)) != cudaSuccess) return bail(fail(TDKS_ENOMEM, "pinned"));
  if (is_f32(c) && !c->tiled) {
    if ((s = dalloc(c, &c->d_rho32, npc * (size_t)nk)) != TDKS_OK) return bail(s);
    cudaMemsetAsync(c->d_rho32, 0, sizeof(float) * npc * (size_t)nk, c->stream);
  }
  cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
  if (c->tiled) {
    const size_t csz = is_f32(c) ? sizeof(float2) : sizeof(double2);
    unsigned char *pa = nullptr, *pb = nullptr, *pe = nullptr;
    if ((s = dalloc(c, &pa, csz * np * (size_t)nk * norb)) != TDKS_OK) return bail(s);
    if ((s = dalloc(c, &pb, csz * np * (size_t)nk * norb)) != TDKS_OK) return bail(s);
    if ((s = dalloc(c, &pe, csz * 4 * (size_t)(c->natom > 0 ? c->natom : 1) * nk * norb)) != TDKS_OK) return bail(s);
    c->d_bufA = pa; c->d_bufB = pb; c->d_ec = pe;
  }
  const bool scratch = !c->tiled &&
      (is_f32(c) ? smem_orbital_needs_scratch<float>(grid->n[2], c->pstride, c->nsph, c->natom)
                 : smem_orbital_needs_scratch<double>(grid->n[2], c->pstride, c->nsph, c->natom));
  if (scratch) {
    const size_t csz = is_f32(c) ? sizeof(float2) : sizeof(double2);
    unsigned char* p = nullptr;
    if ((s = dalloc(c, &p, csz * npc * (size_t)nk * norb)) != TDKS_OK) return bail(s);
    c->d_scratch = p;
  }
  if ((s = dalloc(c, &c->d_orb_obs, (size_t)c->ncell * nk * norb * 8)) != TDKS_OK) return bail(s);
  if (opts->xc == 3) {
    const size_t csz = is_f32(c) ? sizeof(float2) : sizeof(double2);
    unsigned char* p = nullptr;
    c->mbj_nchunk = mbj_chunks((long long)np, nk * norb);
    if ((s = dalloc(c, &c->d_mbj_part, (size_t)c->mbj_nchunk * 5 * np)) != TDKS_OK) return bail(s);
    if ((s = dalloc(c, &c->d_mbj_c, 1)) != TDKS_OK) return bail(s);
    if ((s = dalloc(c, &p, csz * np * (size_t)nk * norb)) != TDKS_OK) return bail(s);
    c->d_porb = p;
    cudaMemsetAsync(c->d_mbj_c, 0, sizeof(double), c->stream);
  }
  c->red_blocks = 304;
  if ((s = dalloc(c, &c->d_partials, (size_t)c->red_blocks * 4)) != TDKS_OK) return bail(s);
  if ((s = dalloc(c, &c->d_ticket, 1)) != TDKS_OK) return bail(s);
  cudaMemsetAsync(c->d_ticket, 0, sizeof(unsigned), c->stream);
  if ((s = dalloc(c, &c->d_partials_obs, (size_t)c->red_blocks * 4)) != TDKS_OK) return bail(s);
  if ((s = dalloc(c, &c->d_ticket_obs, 1)) != TDKS_OK) return bail(s);
  cudaMemsetAsync(c->d_ticket_obs, 0, sizeof(unsigned), c->stream);

  // FFT set-up: periodic transforms are n^3, isolated ones (2n)^3 (zero padding)
  for (int a = 0; a < 3; ++a) {
    c->m[a] = grid->periodic ? grid->n[a] : 2 * grid->n[a];
    if (!fft_radices(c->m[a], c->rad[a]))
      return bail(fail(TDKS_EUNSUPPORTED, "FFT length with a prime factor above 31"));
    std::vector<double2> tw(c->m[a]);
    for (int t = 0; t < c->m[a]; ++t)
      tw[t] = double2{std::cos(2.0 * kPi * t / c->m[a]), -std::sin(2.0 * kPi * t / c->m[a])};
    if ((s = upload(c, &c->d_tw[a], tw)) != TDKS_OK) return bail(s);
  }
  const size_t nfft = (size_t)c->m[0] * c->m[1] * c->m[2];
  if ((s = dalloc(c, &c->d_fft, nfft * c->ncell)) != TDKS_OK) return bail(s);

  // local potential
  if (grid->periodic) {
    std::vector<double> vg;
    local_potential_gspace(*grid, atoms, natom, vg);
    if (cudaMemcpyAsync(c->d_fft, vg.data(), vg.size() * sizeof(double), cudaMemcpyHostToDevice,
                        c->stream) != cudaSuccess)
      return bail(fail(TDKS_ECUDA, "upload V(G)"));
    for (int ax = 0; ax < 3; ++ax)
      if (launch_fft_axis(c->d_fft, c->m, ax, +1, c->d_tw[ax], c->rad[ax].data(), (int)c->rad[ax].size(),
                          c->stream, 1) != cudaSuccess)
        return bail(fail(TDKS_ECUDA, "V_loc transform"));
    if (launch_real_part(c->d_fft, c->d_vloc, np, 1.0, c->stream) != cudaSuccess)
      return bail(fail(TDKS_ECUDA, "real part"));
    // the Poisson factor of every wave vector, read by the z pass of the Hartree solve
    if ((s = dalloc(c, &c->d_ghat, np)) != TDKS_OK) return bail(s);
    if (launch_poisson_table(c->d_ghat, c->m, grid->h, c->stream) != cudaSuccess)
      return bail(fail(TDKS_ECUDA, "Poisson factor table"));
    c->plane_cl = hartree_plane_cluster(c->m, c->ncell, 1);
  } else {
    std::vector<double> at(5 * (size_t)natom);
    for (int i = 0; i < natom; ++i) {
      for (int a = 0; a < 3; ++a) at[5 * i + a] = atoms[i].R[a];
      at[5 * i + 3] = atoms[i].Z;
      at[5 * i + 4] = atoms[i].sigma;
      if (!(atoms[i].sigma > 0.0)) return bail(fail(TDKS_EINVAL, "atom sigma must be positive"));
    }
    double* d_at = nullptr;
    if ((s = upload(c, &d_at, at)) != TDKS_OK) return bail(s);
    if (launch_vloc_isolated(c->d_vloc, grid->n, grid->h, d_at, natom, c->stream) != cudaSuccess)
      return bail(fail(TDKS_ECUDA, "vloc"));
    // Hockney Green's function spectrum
    const double g0 = cell_mean_inverse_distance(grid->h[0], grid->h[1], grid->h[2]);
    if (launch_hockney_kernel(c->d_fft, c->m, grid->n, grid->h, g0, c->stream) != cudaSuccess)
      return bail(fail(TDKS_ECUDA, "hockney"));
    if ((s = fft3d(c, -1)) != TDKS_OK) return bail(s);
    if ((s = dalloc(c, &c->d_ghat, nfft)) != TDKS_OK) return bail(s);
    if (launch_real_part(c->d_fft, c->d_ghat, nfft, 1.0, c->stream) != cudaSuccess)
      return bail(fail(TDKS_ECUDA, "ghat"));
  }
  if (c->tiled) {
    if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess)
      return bail(fail(TDKS_ECUDA, "side stream for the projections"));
  }
  if ((s = tune_tile(c)) != TDKS_OK) return bail(s);
  if ((s = tune_cell(c)) != TDKS_OK) return bail(s);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess)
    return bail(fail(TDKS_ECUDA, std::string("init: ") + cudaGetErrorString(cudaGetLastError())));
  *out = c;
  return TDKS_OK;
}

void tdks_destroy(tdks_ctx* c) {
  if (!c) return;
  if (c->stream || !c->allocs.empty()) cudaStreamSynchronize(c->stream);
  for (auto& r : c->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (cudaEvent_t e : c->event_pool) cudaEventDestroy(e);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->ev_obs_fork) cudaEventDestroy(c->ev_obs_fork);
  if (c->ev_obs_join) cudaEventDestroy(c->ev_obs_join);
  if (c->side) cudaStreamDestroy(c->side);
  for (void* p : c->allocs) cudaFree(p);
  if (c->h_resid) cudaFreeHost(c->h_resid);
  for (auto* gs : {&c->sg[0], &c->sg[1], &c->sg[2], &c->sg[3], &c->msg[0], &c->msg[1], &c->msg[2]}) {
    auto& g = *gs;
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
    for (auto& r : g.recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  }
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->cap2) cudaStreamDestroy(c->cap2);
  if (c->side2) cudaStreamDestroy(c->side2);
  if (c->obs_side) cudaStreamDestroy(c->obs_side);
  delete c;
}

tdks_status tdks_set_field(tdks_ctx* c, int kind, const double A0[3], double omega, double T, double cep) {
  TDKS_TRY(check_ctx(c));
  if (kind < TDKS_FIELD_NONE || kind > TDKS_FIELD_PULSE) return fail(TDKS_EINVAL, "unknown field kind");
  if (kind != TDKS_FIELD_NONE && !A0) return fail(TDKS_EINVAL, "null A0");
  if (kind == TDKS_FIELD_PULSE && !(T > 0.0)) return fail(TDKS_EINVAL, "pulse duration must be positive");
  c->field_kind = kind;
  for (int a = 0; a < 3; ++a) c->A0[a] = (A0 && kind == TDKS_FIELD_STEP) ? A0[a] : 0.0;
  c->pulses.clear();
  c->ftable.clear();
  if (kind == TDKS_FIELD_PULSE) {
    PulseDef p;
    for (int a = 0; a < 3; ++a) p.A0[a] = A0[a];
    p.omega = omega; p.T = T; p.cep = cep; p.delay = 0.0;
    c->pulses.push_back(p);
  }
  return TDKS_OK;
}

tdks_status tdks_field_at(tdks_ctx* c, double t, double Ap[3], double E[3]) {
  TDKS_TRY(check_ctx(c));
  if (!Ap && !E) return fail(TDKS_EINVAL, "null outputs");
  if (!std::isfinite(t)) return fail(TDKS_EINVAL, "t must be finite");
  if (Ap) field_at(c, t, Ap);
  if (E) {   // E = -dA'/dt by a central difference (h = 1e-6 max(1, |t|))
    const double h = 1e-6 * std::max(1.0, std::fabs(t));
    double ap[3], am[3];
    field_at(c, t + h, ap);
    field_at(c, t - h, am);
    for (int a = 0; a < 3; ++a) E[a] = -(ap[a] - am[a]) / (2.0 * h);
  }
  return TDKS_OK;
}

namespace {
// cholesky_inverse_h (host_linalg.h) on the double2 matrices the Gram kernels write
bool cholesky_inverse_h(const double2* S, int n, double2* Cout) {
  std::vector<std::complex<double>> a((size_t)n * n), c((size_t)n * n);
  for (size_t i = 0; i < a.size(); ++i) a[i] = std::complex<double>(S[i].x, S[i].y);
  if (!tdks::cholesky_inverse_h(a.data(), n, c.data())) return false;
  for (size_t i = 0; i < c.size(); ++i) Cout[i] = double2{c[i].real(), c[i].imag()};
  return true;
}
}  // namespace

tdks_status tdks_ground_state(tdks_ctx* c, void* u, int max_iter, double tol, double degree, double mix,
                              double* out) {
  TDKS_TRY(check_ctx(c));
  TDKS_TRY(check_whole_set(c, "tdks_ground_state"));
  if (!u) return fail(TDKS_EINVAL, "null orbitals");
  if (c->ncell != 1) return fail(TDKS_EUNSUPPORTED, "tdks_ground_state needs ncell = 1");
  if (c->norb > 64) return fail(TDKS_EUNSUPPORTED, "tdks_ground_state handles at most 64 orbitals per k-point");
  if (max_iter < 1 || !(tol > 0.0) || !(mix > 0.0 && mix <= 1.0) || !std::isfinite(degree))
    return fail(TDKS_EINVAL, "need max_iter >= 1, tol > 0, 0 < mix <= 1 and a finite filter degree");
  const int m = degree > 0.0 ? std::max(2, std::min(60, (int)std::lround(degree))) : 10;
  const int nk = c->nk, no = c->norb, np = c->npts;
  const int nb = std::min(no + std::max(4, (no + 3) / 4), np);      // the block: occupied + buffer states
  const bool f32 = is_f32(c);
  const size_t csz = f32 ? sizeof(float2) : sizeof(double2);
  const size_t nblk = (size_t)nk * nb * np;                          // complex values of one block
  const size_t nmat = (size_t)nk * nb * nb;
  using Z = std::complex<double>;
  std::vector<Z> hM(nmat), hC(nmat);
  std::vector<double> hv((size_t)np), hvin((size_t)np), hvl((size_t)np), eig((size_t)nk * nb, 0.0);
  void* Bf[4] = {nullptr, nullptr, nullptr, nullptr};
  double2 *dM = nullptr, *dC = nullptr;
  double* d_vin = nullptr;
  tdks_ctx* sib = nullptr;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  for (auto& b : Bf) chk(cudaMalloc(&b, nblk * csz));
  chk(cudaMalloc(&dM, nmat * sizeof(double2)));
  chk(cudaMalloc(&dC, nmat * sizeof(double2)));
  chk(cudaMalloc(&d_vin, (size_t)np * sizeof(double)));
  auto cleanup = [&]() {
    cudaStreamSynchronize(c->stream);
    for (auto& b : Bf) cudaFree(b);
    cudaFree(dM); cudaFree(dC); cudaFree(d_vin);
    if (sib) tdks_destroy(sib);
  };
  if (e != cudaSuccess) { cleanup(); return fail(TDKS_ENOMEM, "tdks_ground_state: device memory"); }
  // a context of the same system with nb orbitals per k-point applies H to the block
  {
    tdks_options o2 = c->opt;
    o2.hartree = 0; o2.xc = 0; o2.pc = 0; o2.ncell = 1; o2.obs_at_start = 0; o2.norb_offset = 0; o2.norb_total = 0;
    const tdks_status st = tdks_init(&c->grid, &c->cell_in, c->atoms_in.empty() ? nullptr : c->atoms_in.data(),
                                     (int)c->atoms_in.size(), c->proj_in.empty() ? nullptr : c->proj_in.data(),
                                     (int)c->proj_in.size(), c->kpts.data(), c->kw.data(), nk, nb, &o2, c->stream, &sib);
    if (st != TDKS_OK) { cleanup(); return st; }
  }
  const double zeroA[3] = {0.0, 0.0, 0.0};
  auto H = [&](const void* in, void* o) -> tdks_status {                   // o = H in, the block
    TDKS_TRY(set_step_potential(sib, 1.0, nullptr, 0.0));
    return orbital_kernel(sib, 0, in, o, zeroA, 0.0, nullptr, 1);
  };
  auto gram = [&](const void* A, const void* B, double2* o) {
    return f32 ? launch_gram<float>((const float2*)A, (const float2*)B, nk, nb, np, c->dV, o, c->stream)
               : launch_gram<double>((const double2*)A, (const double2*)B, nk, nb, np, c->dV, o, c->stream);
  };
  auto basis = [&](const void* U, const void* V, const double2* M, double a, double c0, double b, void* o) {
    return f32 ? launch_basis<float>((const float2*)U, (const float2*)V, M, nk, nb, np, a, c0, b, (float2*)o, c->stream)
               : launch_basis<double>((const double2*)U, (const double2*)V, M, nk, nb, np, a, c0, b, (double2*)o,
                                      c->stream);
  };
  auto lincomb = [&](const void* A, const void* B, const void* C3, double a, double b, double g, void* o) {
    return f32 ? launch_lincomb3<float>((const float2*)A, (const float2*)B, (const float2*)C3, a, b, g,
                                        (long long)nblk, (float2*)o, c->stream)
               : launch_lincomb3<double>((const double2*)A, (const double2*)B, (const double2*)C3, a, b, g,
                                         (long long)nblk, (double2*)o, c->stream);
  };
  auto vec = [&](void* base, int k, int n) {        // start of vector n of k-point k in a block
    return static_cast<unsigned char*>(base) + (((size_t)k * nb + n) * np) * csz;
  };
  // orthonormal block: dst = src L^{-H} with src^H src dV = L L^H
  auto ortho = [&](const void* src, void* dst) -> tdks_status {
    TDKS_CUDA(gram(src, src, dM));
    TDKS_CUDA(cudaMemcpyAsync(hM.data(), dM, nmat * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
    TDKS_CUDA(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < nk; ++k)
      if (!cholesky_inverse_h(&hM[(size_t)k * nb * nb], nb, &hC[(size_t)k * nb * nb]))
        return fail(TDKS_EINVAL, "tdks_ground_state: the orbitals are linearly dependent");
    TDKS_CUDA(cudaMemcpyAsync(dC, hC.data(), nmat * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
    TDKS_CUDA(basis(src, nullptr, dC, 0.0, 0.0, 1.0, dst));
    c->launches += 2;
    return TDKS_OK;
  };
  // Rayleigh-Ritz of the orthonormal block X (HX its H image, W a work block): the eigenpairs of the
  // projected H per k (host Jacobi), X and HX rotated into Ritz vectors, eig their values
  auto ritz = [&](void*& X, void*& HX, void*& W) -> tdks_status {
    TDKS_TRY(H(X, HX));
    TDKS_CUDA(gram(X, HX, dM));
    TDKS_CUDA(cudaMemcpyAsync(hM.data(), dM, nmat * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
    TDKS_CUDA(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < nk; ++k) {
      std::vector<Z> A(hM.begin() + (size_t)k * nb * nb, hM.begin() + (size_t)(k + 1) * nb * nb), Y;
      for (int i2 = 0; i2 < nb; ++i2)                  // the projected H is Hermitian up to rounding
        for (int j2 = 0; j2 < i2; ++j2) {
          const Z h = 0.5 * (A[(size_t)i2 * nb + j2] + std::conj(A[(size_t)j2 * nb + i2]));
          A[(size_t)i2 * nb + j2] = h;
          A[(size_t)j2 * nb + i2] = std::conj(h);
        }
      std::vector<double> w;
      herm_eig(A, nb, w, Y);
      for (int n = 0; n < nb; ++n) eig[(size_t)k * nb + n] = w[n];
      std::copy(Y.begin(), Y.end(), hC.begin() + (size_t)k * nb * nb);
    }
    TDKS_CUDA(cudaMemcpyAsync(dC, hC.data(), nmat * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
    TDKS_CUDA(basis(X, nullptr, dC, 0.0, 0.0, 1.0, W));
    std::swap(X, W);
    TDKS_CUDA(basis(HX, nullptr, dC, 0.0, 0.0, 1.0, W));
    std::swap(HX, W);
    c->launches += 3;
    return TDKS_OK;
  };
  // the input orbitals must be independent: their own overlap
  {
    std::vector<Z> S((size_t)nk * no * no), Cn((size_t)nk * no * no);
    const tdks_status st = [&]() -> tdks_status {
      TDKS_CUDA(f32 ? launch_gram<float>((const float2*)u, (const float2*)u, nk, no, np, c->dV, dM, c->stream)
                    : launch_gram<double>((const double2*)u, (const double2*)u, nk, no, np, c->dV, dM, c->stream));
      TDKS_CUDA(cudaMemcpyAsync(S.data(), dM, S.size() * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
      TDKS_CUDA(cudaStreamSynchronize(c->stream));
      for (int k = 0; k < nk; ++k)
        if (!cholesky_inverse_h(&S[(size_t)k * no * no], no, &Cn[(size_t)k * no * no]))
          return fail(TDKS_EINVAL, "tdks_ground_state: the orbitals are linearly dependent");
      return TDKS_OK;
    }();
    if (st != TDKS_OK) { cleanup(); return st; }
  }
  auto free_blocks = [&](const void* X, const void* HX, void* (&fr)[2]) {   // the two blocks not in use
    int n = 0;
    for (void* bb : Bf)
      if (bb != X && bb != HX && n < 2) fr[n++] = bb;
  };
  auto solve = [&]() -> tdks_status {
    void* X = Bf[0];
    void* HX = Bf[1];
    void* P = Bf[2];
    // initial block in P: the input orbitals, then seeded random buffer states; orthonormalised into X
    {
      std::vector<unsigned char> hb((size_t)(nb - no) * np * csz);
      unsigned long long sd = 0x243F6A8885A308D3ULL;
      for (size_t i2 = 0; i2 < (size_t)(nb - no) * np; ++i2) {
        const double re = 2.0 * uniform01(sd) - 1.0, im = 2.0 * uniform01(sd) - 1.0;
        if (f32) reinterpret_cast<float2*>(hb.data())[i2] = float2{(float)re, (float)im};
        else reinterpret_cast<double2*>(hb.data())[i2] = double2{re, im};
      }
      for (int k = 0; k < nk; ++k) {
        TDKS_CUDA(cudaMemcpyAsync(vec(P, k, 0), static_cast<unsigned char*>(u) + (size_t)k * no * np * csz,
                                  (size_t)no * np * csz, cudaMemcpyDeviceToDevice, c->stream));
        TDKS_CUDA(cudaMemcpyAsync(vec(P, k, no), hb.data(), hb.size(), cudaMemcpyHostToDevice, c->stream));
      }
      TDKS_CUDA(cudaStreamSynchronize(c->stream));
    }
    TDKS_TRY(ortho(P, X));
    // the potential of the input density
    TDKS_TRY(density(c, u, c->d_rho));
    TDKS_TRY(hxc(c, c->d_rho, c->d_vhxc, u));
    TDKS_CUDA(cudaMemcpyAsync(d_vin, c->d_vhxc, (size_t)np * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    TDKS_CUDA(cudaMemcpyAsync(sib->d_vhxc, c->d_vhxc, (size_t)np * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    TDKS_TRY(ritz(X, HX, P));
    // upper bound of the spectrum: the FD kinetic symbol (its largest value per axis 3.26 / h^2, the
    // first-derivative term at most 2.09 |q| / h, plus |q|^2 / 2), the largest potential, ||V_NL||
    double kin = 0.0;
    for (int k = 0; k < nk; ++k) {
      double kk = 0.0, q2 = 0.0;
      for (int a = 0; a < 3; ++a) {
        const double q = c->kpts[3 * k + a], h = c->grid.h[a];
        kk += 3.26 / (h * h) + 2.09 * std::fabs(q) / h;
        q2 += q * q;
      }
      kin = std::max(kin, kk + 0.5 * q2);
    }
    TDKS_CUDA(cudaMemcpyAsync(hvl.data(), c->d_vloc, (size_t)np * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    double resid = 0.0;
    int it = 0;
    for (it = 1; it <= max_iter; ++it) {
      // bounds of the filter: damp [a, b] (a = the block's highest Ritz value), normalised at the lowest
      TDKS_CUDA(cudaMemcpyAsync(hv.data(), sib->d_vhxc, (size_t)np * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      TDKS_CUDA(cudaStreamSynchronize(c->stream));
      double vmax = -1e300;
      for (int i2 = 0; i2 < np; ++i2) vmax = std::max(vmax, hvl[i2] + hv[i2]);
      double elo = 1e300, ehi = -1e300;
      for (int k = 0; k < nk; ++k) {
        elo = std::min(elo, eig[(size_t)k * nb]);
        ehi = std::max(ehi, eig[(size_t)k * nb + nb - 1]);
      }
      const double b = kin + vmax + c->vnl_bound;
      const double a = ehi;
      if (!(b > a && a > elo)) return fail(TDKS_ECUDA, "tdks_ground_state: inconsistent spectral bounds");
      const double ee = 0.5 * (b - a), cc = 0.5 * (b + a);
      double sig = ee / (elo - cc);
      const double sig1 = sig;
      // Chebyshev filter of degree m (three-term recurrence, scaled so the lowest end stays of order 1):
      // Y1 = (H - cc) X sig1 / ee;  Y_{j+1} = 2 sig' / ee (H - cc) Y_j - sig sig' Y_{j-1}.  The buffers
      // rotate over the four blocks; HX (needed only by the first term) then holds H Y_j.
      void* fr[2];
      free_blocks(X, HX, fr);
      void* prev = X;
      void* cur = fr[0];
      void* nxt = fr[1];
      TDKS_CUDA(lincomb(HX, X, nullptr, sig1 / ee, -cc * sig1 / ee, 0.0, cur));
      c->launches += 1;
      for (int jj = 2; jj <= m; ++jj) {
        const double sig2 = 1.0 / (2.0 / sig1 - sig);
        TDKS_TRY(H(cur, HX));
        TDKS_CUDA(lincomb(HX, cur, prev, 2.0 * sig2 / ee, -2.0 * cc * sig2 / ee, -sig * sig2, nxt));
        c->launches += 1;
        void* t = prev;
        prev = cur;
        cur = nxt;
        nxt = t;
        sig = sig2;
      }
      // orthonormalise the filtered block into a free block, then Rayleigh-Ritz
      X = (prev != cur) ? prev : nxt;
      TDKS_TRY(ortho(cur, X));
      free_blocks(X, HX, fr);
      P = fr[0];
      TDKS_TRY(ritz(X, HX, P));
      free_blocks(X, HX, fr);
      P = fr[0];
      // residual of the occupied Ritz pairs, R = HX - X diag(e)
      {
        std::vector<Z> D(nmat, Z(0.0, 0.0));
        for (int k = 0; k < nk; ++k)
          for (int n = 0; n < nb; ++n) D[(size_t)k * nb * nb + (size_t)n * nb + n] = eig[(size_t)k * nb + n];
        TDKS_CUDA(cudaMemcpyAsync(dC, D.data(), nmat * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
        TDKS_CUDA(basis(X, HX, dC, 1.0, 0.0, -1.0, P));
        TDKS_CUDA(gram(P, P, dM));
        TDKS_CUDA(cudaMemcpyAsync(hM.data(), dM, nmat * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
        TDKS_CUDA(cudaStreamSynchronize(c->stream));
        double r2 = 0.0;
        for (int k = 0; k < nk; ++k)
          for (int n = 0; n < no; ++n) r2 += hM[(size_t)k * nb * nb + (size_t)n * nb + n].real();
        resid = std::sqrt(r2 / (nk * no));
        c->launches += 2;
      }
      // the occupied states into u, their density and potential, mixing
      for (int k = 0; k < nk; ++k)
        TDKS_CUDA(cudaMemcpyAsync(static_cast<unsigned char*>(u) + (size_t)k * no * np * csz, vec(X, k, 0),
                                  (size_t)no * np * csz, cudaMemcpyDeviceToDevice, c->stream));
      TDKS_TRY(density(c, u, c->d_rho));
      TDKS_TRY(hxc(c, c->d_rho, c->d_vhxc, u));                                   // V_out
      TDKS_CUDA(cudaMemcpyAsync(hv.data(), c->d_vhxc, (size_t)np * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      TDKS_CUDA(cudaMemcpyAsync(hvin.data(), d_vin, (size_t)np * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      TDKS_CUDA(cudaStreamSynchronize(c->stream));
      double a2 = 0.0, b2 = 0.0;
      for (int i2 = 0; i2 < np; ++i2) { a2 += (hv[i2] - hvin[i2]) * (hv[i2] - hvin[i2]); b2 += hv[i2] * hv[i2]; }
      const double dv = std::sqrt(a2 / std::max(b2, 1e-300));
      if (resid < tol && dv < tol) break;
      TDKS_CUDA(launch_mix_potential(d_vin, c->d_vhxc, np, mix, c->stream));
      TDKS_CUDA(cudaMemcpyAsync(sib->d_vhxc, c->d_vhxc, (size_t)np * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
      c->launches += 1;
    }
    // the ground state's own potential and reference density
    TDKS_TRY(density(c, u, c->d_rho));
    TDKS_TRY(hxc(c, c->d_rho, c->d_vhxc, u));
    TDKS_CUDA(cudaMemcpyAsync(c->d_rho0, c->d_rho, (size_t)np * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    c->have_rho0 = true;
    c->have_potential = true;
    c->hist_count = 0;
    TDKS_TRY(hist_push(c, c->d_vhxc));
    if (out) {
      double eb = 0.0;
      for (int k = 0; k < nk; ++k)
        for (int n = 0; n < no; ++n) eb += 2.0 * c->kw[k] * eig[(size_t)k * nb + n];
      out[0] = std::min(it, max_iter);
      out[1] = resid;
      out[2] = eb;
    }
    return TDKS_OK;
  };
  const tdks_status st = solve();
  cleanup();
  return st;
}

tdks_status tdks_excited_pairs(tdks_ctx* c, const void* u, const void* u_gs, double* n_eh) {
  TDKS_TRY(check_ctx(c));
  if (!u || !u_gs || !n_eh) return fail(TDKS_EINVAL, "null argument");
  if (c->ncell != 1) return fail(TDKS_EUNSUPPORTED, "tdks_excited_pairs needs ncell = 1");
  const int nk = c->nk, no = c->norb;
  const size_t nmat = (size_t)nk * no * no;
  double2* dO = nullptr;
  if (cudaMalloc(&dO, nmat * sizeof(double2)) != cudaSuccess) return fail(TDKS_ENOMEM, "tdks_excited_pairs: device memory");
  std::vector<double2> hO(nmat);
  std::vector<double> kw((size_t)nk);
  cudaError_t e = is_f32(c)
      ? launch_gram<float>((const float2*)u_gs, (const float2*)u, nk, no, c->npts, c->dV, dO, c->stream)
      : launch_gram<double>((const double2*)u_gs, (const double2*)u, nk, no, c->npts, c->dV, dO, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hO.data(), dO, nmat * sizeof(double2), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(kw.data(), c->d_kw, nk * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(dO);
  if (e != cudaSuccess) return fail(TDKS_ECUDA, std::string("tdks_excited_pairs: ") + cudaGetErrorString(e));
  c->launches += 1;
  double n = 0.0;
  for (int k = 0; k < nk; ++k) {
    double f2 = 0.0;     // sum_{m,n} |<phi_m|psi_n>|^2: the occupied weight kept in the ground-state subspace
    for (size_t i = 0; i < (size_t)no * no; ++i) {
      const double2 o = hO[(size_t)k * no * no + i];
      f2 += o.x * o.x + o.y * o.y;
    }
    n += 2.0 * kw[k] * (no - f2);
  }
  *n_eh = n / c->omega;
  return TDKS_OK;
}

tdks_status tdks_orbital_energies(tdks_ctx* c, void* u, const double Ap[3], int rotate, double* eps) {
  TDKS_TRY(check_ctx(c));
  if (!u || !eps) return fail(TDKS_EINVAL, "null argument");
  if (rotate != 0 && rotate != 1) return fail(TDKS_EINVAL, "rotate must be 0 or 1");
  if (c->ncell != 1) return fail(TDKS_EUNSUPPORTED, "tdks_orbital_energies needs ncell = 1");
  if (c->norb > 64) return fail(TDKS_EUNSUPPORTED, "tdks_orbital_energies handles at most 64 orbitals per k-point");
  if (!c->have_potential) return fail(TDKS_EINVAL, "call tdks_update_potential or tdks_ground_state first");
  const int nk = c->nk, no = c->norb, np = c->npts;
  const bool f32 = is_f32(c);
  const size_t nob = (size_t)nk * no * np * (f32 ? sizeof(float2) : sizeof(double2)), nmat = (size_t)nk * no * no;
  const double zeroA[3] = {0.0, 0.0, 0.0};
  void* HU = nullptr;
  double2 *dM = nullptr, *dS = nullptr;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  chk(cudaMalloc(&HU, nob));
  chk(cudaMalloc(&dM, nmat * sizeof(double2)));
  chk(cudaMalloc(&dS, nmat * sizeof(double2)));
  auto cleanup = [&]() {
    cudaStreamSynchronize(c->stream);
    cudaFree(HU); cudaFree(dM); cudaFree(dS);
  };
  if (e != cudaSuccess) { cleanup(); return fail(TDKS_ENOMEM, "tdks_orbital_energies: device memory"); }
  auto run = [&]() -> tdks_status {
    std::vector<double2> hM(nmat), hS(nmat), hX(nmat), hZ(nmat);
    TDKS_TRY(set_step_potential(c, 1.0, nullptr, 0.0));
    TDKS_TRY(orbital_kernel(c, 0, u, HU, Ap ? Ap : zeroA, 0.0, nullptr, 1));       // H_q u
    if (f32) {
      TDKS_CUDA(launch_gram<float>((const float2*)u, (const float2*)HU, nk, no, np, c->dV, dM, c->stream));
      TDKS_CUDA(launch_gram<float>((const float2*)u, (const float2*)u, nk, no, np, c->dV, dS, c->stream));
    } else {
      TDKS_CUDA(launch_gram<double>((const double2*)u, (const double2*)HU, nk, no, np, c->dV, dM, c->stream));
      TDKS_CUDA(launch_gram<double>((const double2*)u, (const double2*)u, nk, no, np, c->dV, dS, c->stream));
    }
    c->launches += 2;
    TDKS_CUDA(cudaMemcpyAsync(hM.data(), dM, nmat * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
    TDKS_CUDA(cudaMemcpyAsync(hS.data(), dS, nmat * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
    TDKS_CUDA(cudaStreamSynchronize(c->stream));
    using Zc = std::complex<double>;
    for (int k = 0; k < nk; ++k) {
      // S = L L^H, X = L^{-H}: the projected problem M z = e S z becomes A y = e y with A = X^H M X, z = X y
      const size_t o = (size_t)k * no * no;
      if (!cholesky_inverse_h(&hS[o], no, &hX[o]))
        return fail(TDKS_EINVAL, "tdks_orbital_energies: the orbitals are linearly dependent");
      std::vector<Zc> X((size_t)no * no), MX((size_t)no * no), A((size_t)no * no), Y;
      for (size_t i = 0; i < (size_t)no * no; ++i) X[i] = Zc(hX[o + i].x, hX[o + i].y);
      for (int i = 0; i < no; ++i)
        for (int j = 0; j < no; ++j) {
          Zc sacc = 0.0;
          for (int l = 0; l < no; ++l) sacc += Zc(hM[o + (size_t)i * no + l].x, hM[o + (size_t)i * no + l].y) * X[(size_t)l * no + j];
          MX[(size_t)i * no + j] = sacc;
        }
      for (int i = 0; i < no; ++i)
        for (int j = 0; j < no; ++j) {
          Zc sacc = 0.0;
          for (int l = 0; l < no; ++l) sacc += std::conj(X[(size_t)l * no + i]) * MX[(size_t)l * no + j];
          A[(size_t)i * no + j] = sacc;
        }
      for (int i = 0; i < no; ++i)                                               // symmetrise the rounding
        for (int j = i + 1; j < no; ++j) {
          const Zc m = 0.5 * (A[(size_t)i * no + j] + std::conj(A[(size_t)j * no + i]));
          A[(size_t)i * no + j] = m;
          A[(size_t)j * no + i] = std::conj(m);
        }
      std::vector<double> w;
      herm_eig(A, no, w, Y);
      for (int n = 0; n < no; ++n) eps[(size_t)k * no + n] = w[n];
      for (int i = 0; i < no; ++i)                                               // Z = X Y
        for (int j = 0; j < no; ++j) {
          Zc sacc = 0.0;
          for (int l = 0; l < no; ++l) sacc += X[(size_t)i * no + l] * Y[(size_t)l * no + j];
          hZ[o + (size_t)i * no + j] = double2{sacc.real(), sacc.imag()};
        }
    }
    if (rotate) {   // u_j <- sum_i u_i Z_ij through the work buffer
      TDKS_CUDA(cudaMemcpyAsync(dM, hZ.data(), nmat * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
      if (f32)
        TDKS_CUDA(launch_basis<float>((const float2*)u, nullptr, dM, nk, no, np, 0.0, 0.0, 1.0, (float2*)HU, c->stream));
      else
        TDKS_CUDA(launch_basis<double>((const double2*)u, nullptr, dM, nk, no, np, 0.0, 0.0, 1.0, (double2*)HU,
                                       c->stream));
      TDKS_CUDA(cudaMemcpyAsync(u, HU, nob, cudaMemcpyDeviceToDevice, c->stream));
      c->launches += 1;
    }
    return TDKS_OK;
  };
  const tdks_status st = run();
  cleanup();
  return st;
}

tdks_status tdks_set_mbj(tdks_ctx* c, double cval) {
  TDKS_TRY(check_ctx(c));
  if (c->opt.xc != 3) return fail(TDKS_EUNSUPPORTED, "tdks_set_mbj needs a context with xc = 3");
  if (!std::isfinite(cval)) return fail(TDKS_EINVAL, "tdks_set_mbj: c must be finite");
  c->mbj_c_fixed = cval > 0.0 ? cval : 0.0;
  return TDKS_OK;
}

tdks_status tdks_mbj_c(tdks_ctx* c, double* cval) {
  TDKS_TRY(check_ctx(c));
  if (!cval) return fail(TDKS_EINVAL, "null output");
  if (c->opt.xc != 3) return fail(TDKS_EUNSUPPORTED, "tdks_mbj_c needs a context with xc = 3");
  if (c->mbj_c_fixed > 0.0) {
    *cval = c->mbj_c_fixed;
    return TDKS_OK;
  }
  TDKS_CUDA(cudaMemcpyAsync(c->h_resid, c->d_mbj_c, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  TDKS_CUDA(cudaStreamSynchronize(c->stream));
  *cval = *c->h_resid;
  return TDKS_OK;
}

tdks_status tdks_set_longitudinal(tdks_ctx* c, int enable, const void* u, double t0) {
  TDKS_TRY(check_ctx(c));
  if (enable != 0 && enable != 1) return fail(TDKS_EINVAL, "enable must be 0 or 1");
  if (!enable) {
    c->longitudinal = 0;
    return TDKS_OK;
  }
  if (!c->grid.periodic || c->ncell != 1 || c->ms_ready)
    return fail(TDKS_EUNSUPPORTED, "the longitudinal geometry needs one periodic cell outside the multiscale mode");
  if (c->opt.obs_at_start) return fail(TDKS_EUNSUPPORTED, "the longitudinal geometry needs obs_at_start = 0");
  if (!u) return fail(TDKS_EINVAL, "null orbitals");
  if (!c->d_lg) TDKS_TRY(dalloc(c, &c->d_lg, 6));
  if (!c->d_ap_mid) {
    TDKS_TRY(dalloc(c, &c->d_ap_mid, 3 * (size_t)c->ncell));
    TDKS_TRY(dalloc(c, &c->d_ap_end, 3 * (size_t)c->ncell));
  }
  TDKS_CUDA(cudaMemsetAsync(c->d_lg, 0, 6 * sizeof(double), c->stream));
  double A[3];
  field_at(c, t0, A);
  // J(t0) of u (A'_ind = 0 at t0) into the step observables, where the first step reads it
  TDKS_TRY(orbital_observables(c, u, A));
  TDKS_CUDA(launch_reduce_current(c->d_orb_obs, c->nk, c->norb, c->d_kw, 1.0 / c->omega, 1, c->d_step_obs,
                                  c->stream, c->ncell));
  c->launches += 1;
  c->lg_first = 1;
  c->longitudinal = 1;
  return TDKS_OK;
}

tdks_status tdks_longitudinal_read(tdks_ctx* c, double A_ind[3]) {
  TDKS_TRY(check_ctx(c));
  if (!A_ind) return fail(TDKS_EINVAL, "null output");
  if (!c->d_lg) {
    A_ind[0] = A_ind[1] = A_ind[2] = 0.0;
    return TDKS_OK;
  }
  TDKS_CUDA(cudaMemcpyAsync(A_ind, c->d_lg, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  TDKS_CUDA(cudaStreamSynchronize(c->stream));
  return TDKS_OK;
}

tdks_status tdks_add_pulse(tdks_ctx* c, const double A0[3], double omega, double T, double cep, double t_delay) {
  TDKS_TRY(check_ctx(c));
  if (c->field_kind != TDKS_FIELD_PULSE) return fail(TDKS_EINVAL, "tdks_add_pulse needs a field of kind TDKS_FIELD_PULSE");
  if (!A0) return fail(TDKS_EINVAL, "null A0");
  if (!(T > 0.0)) return fail(TDKS_EINVAL, "pulse duration must be positive");
  if (!std::isfinite(t_delay)) return fail(TDKS_EINVAL, "pulse delay must be finite");
  if ((int)c->pulses.size() >= kMaxPulses) return fail(TDKS_EINVAL, "at most 8 pulses");
  PulseDef p;
  for (int a = 0; a < 3; ++a) p.A0[a] = A0[a];
  p.omega = omega; p.T = T; p.cep = cep; p.delay = t_delay;
  c->pulses.push_back(p);
  return TDKS_OK;
}

tdks_status tdks_set_field_table(tdks_ctx* c, const double* Ap, int nt, double t0, double dt_table) {
  TDKS_TRY(check_ctx(c));
  if (!Ap) return fail(TDKS_EINVAL, "null table");
  if (nt < 1 || nt > (1 << 26)) return fail(TDKS_EINVAL, "table length outside 1..2^26");
  if (!(dt_table > 0.0) || !std::isfinite(t0)) return fail(TDKS_EINVAL, "table spacing must be positive");
  for (size_t i = 0; i < 3 * (size_t)nt; ++i)
    if (!std::isfinite(Ap[i])) return fail(TDKS_EINVAL, "non-finite value in the field table");
  c->field_kind = TDKS_FIELD_TABLE;
  c->pulses.clear();
  for (int a = 0; a < 3; ++a) c->A0[a] = 0.0;
  c->ftable.assign(Ap, Ap + 3 * (size_t)nt);
  c->tab_t0 = t0;
  c->tab_dt = dt_table;
  return TDKS_OK;
}

tdks_status tdks_kick(tdks_ctx* c, void* u, const double kappa[3]) {
  TDKS_TRY(check_ctx(c));
  if (!u || !kappa) return fail(TDKS_EINVAL, "null argument");
  const int tot = c->nk * c->norb;
  if (is_f32(c))
    TDKS_CUDA(launch_kick<float>(static_cast<float2*>(u), tot, c->grid.n, c->grid.h, c->grid.periodic, kappa, c->stream));
  else
    TDKS_CUDA(launch_kick<double>(static_cast<double2*>(u), tot, c->grid.n, c->grid.h, c->grid.periodic, kappa, c->stream));
  return TDKS_OK;
}

tdks_status tdks_update_potential(tdks_ctx* c, const void* u) {
  TDKS_TRY(check_ctx(c));
  TDKS_TRY(check_whole_set(c, "tdks_update_potential"));
  if (!u) return fail(TDKS_EINVAL, "null orbitals");
  TDKS_TRY(density(c, u, c->d_rho));
  TDKS_TRY(hxc(c, c->d_rho, c->d_vhxc, u));
  if (!c->have_rho0) {
    TDKS_CUDA(cudaMemcpyAsync(c->d_rho0, c->d_rho, c->npts * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    c->have_rho0 = true;
  }
  c->have_potential = true;
  c->hist_count = 0;
  TDKS_TRY(hist_push(c, c->d_vhxc));
  return TDKS_OK;
}

tdks_status tdks_hpsi(tdks_ctx* c, const void* u, void* hu, const double Ap[3]) {
  TDKS_TRY(check_ctx(c));
  if (!u || !hu) return fail(TDKS_EINVAL, "null orbitals");
  if (u == hu) return fail(TDKS_EINVAL, "u and hu must not alias");
  TDKS_TRY(set_step_potential(c, 1.0, nullptr, 0.0));
  return orbital_kernel(c, 0, u, hu, Ap, 0.0, nullptr, 1);
}

tdks_status tdks_taylor_step(tdks_ctx* c, void* u, double dt, const double Ap[3]) {
  TDKS_TRY(check_ctx(c));
  if (!u) return fail(TDKS_EINVAL, "null orbitals");
  TDKS_TRY(set_step_potential(c, 1.0, nullptr, 0.0));
  return orbital_kernel(c, 1, u, u, Ap, dt, nullptr, 1);
}

// plain predictor-corrector (or single Taylor step) from u; leaves V_Hxc(t+dt) in d_vhxc and the
// predictor's potential in d_vpred
// Aobs: A' of the fused per-orbital observables (nullptr: none); obs_start: they belong to the input
// state (formed by the first orbital kernel of the step) instead of the propagated one.
tdks_status pc_step(tdks_ctx* c, void* u, const double Amid[3], const double* Aobs, bool obs_start,
                    double dt) {
  const size_t gb = (size_t)c->ncell * c->npts * sizeof(double);
  const bool pc = c->opt.pc && (c->opt.hartree || c->opt.xc);
  if (pc) {
    // predictor: T4 with V(t); only its density is kept
    TDKS_TRY(set_step_potential(c, 1.0, nullptr, 0.0));
    if (!rho_overwritten(c)) {
      Phase ph(c, 5);
      TDKS_CUDA(cudaMemsetAsync(c->d_rho_tmp, 0, gb, c->stream));
    }
    // (TB-mBJ needs the predicted orbitals themselves: they are written to d_porb)
    void* pout = c->d_porb ? c->d_porb : u;
    TDKS_TRY(orbital_kernel(c, 1, u, pout, Amid, dt, c->d_rho_tmp, c->d_porb ? 1 : 0, obs_start ? Aobs : nullptr,
                            obs_start, 0));
    TDKS_TRY(hxc(c, c->d_rho_tmp, c->d_vpred, pout));
    // corrector: T4 with the mid-point potential
    TDKS_TRY(set_step_potential(c, 0.5, c->d_vpred, 0.5));
  } else {
    TDKS_TRY(set_step_potential(c, 1.0, nullptr, 0.0));
  }
  if (!rho_overwritten(c)) {
    Phase ph(c, 5);
    TDKS_CUDA(cudaMemsetAsync(c->d_rho, 0, gb, c->stream));
  }
  // corrector; it also forms the per-orbital observables unless the predictor already did
  const bool corr_obs = !(pc && obs_start);
  TDKS_TRY(orbital_kernel(c, 1, u, u, Amid, dt, c->d_rho, 1, corr_obs ? Aobs : nullptr, obs_start));
  TDKS_TRY(hxc(c, c->d_rho, c->d_vhxc, u));
  if (pc) {   // the PC's own misfit, for scale
    TDKS_CUDA(launch_residual(c->d_vhxc, c->d_vpred, c->npts * c->ncell, c->d_partials, c->d_ticket, c->d_resid, c->stream));
    c->launches += 1;
  }
  return TDKS_OK;
}

// Read the device fallback count (synchronises the stream); the launches of the fallback bodies that
// ran since the last read join the launch count.
static tdks_status sync_fallbacks(tdks_ctx* c) {
  double fb = 0.0;
  TDKS_CUDA(cudaMemcpyAsync(&fb, c->d_fb, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  TDKS_CUDA(cudaStreamSynchronize(c->stream));
  if (fb > c->fb_seen) {
    const long long n = (long long)(fb - c->fb_seen);
    c->launches += n * c->body_launches;
    for (int p = 0; p < TDKS_NPHASE; ++p) c->calls[p] += n * c->body_calls[p];
  }
  c->fb_seen = fb;
  c->fallbacks = fb;
  return TDKS_OK;
}

// Predicted step, main path (inside a step-graph capture): the prediction of V~(t+dt) from the
// history (the network or the cubic), the corrector T4[V_loc + (V_Hxc(t) + V~)/2] with its density,
// V_Hxc(t+dt) into d_vnew and the misfit into d_resid.
// J (from the orbital kernel's per-orbital sums) and the dipole of rho, into the step observables;
// `partials` / `ticket` are the grid_sum buffers of the dipole.
static tdks_status step_observables(tdks_ctx* c, bool at_start, double* partials, unsigned* ticket) {
  Phase ph(c, 4);
  if (c->grid.periodic) {
    TDKS_CUDA(launch_reduce_current(c->d_orb_obs, c->nk, c->norb, c->d_kw, 1.0 / c->omega, 1, c->d_step_obs,
                                    c->stream, c->ncell));
    c->launches += 1;
  } else {
    TDKS_CUDA(cudaMemsetAsync(c->d_step_obs, 0, 3 * sizeof(double), c->stream));
  }
  if (!at_start) {
    TDKS_CUDA(launch_dipole(c->d_rho, c->d_rho0, c->grid.n, c->grid.h, c->grid.periodic, partials, ticket,
                            c->d_step_obs, c->stream));
    c->launches += 1;
  }
  return TDKS_OK;
}

// Inside a step graph the step's J and dipole run on a parallel branch beside the Hartree solve
// (whose FFT kernels occupy few SMs): they need only what the orbital kernel left (the per-orbital
// sums and the density).  The graph joins the branch before the accept / fallback decision, and a
// fallback body computes them again from its own orbitals.
static tdks_status fork_step_observables(tdks_ctx* c, bool at_start, bool zero_r32) {
  TDKS_CUDA(cudaEventRecord(c->ev_obs_fork, c->stream));
  TDKS_CUDA(cudaStreamWaitEvent(c->obs_side, c->ev_obs_fork, 0));
  const cudaStream_t main = c->stream;
  c->stream = c->obs_side;
  tdks_status st = step_observables(c, at_start, c->d_partials_obs, c->d_ticket_obs);
  if (st == TDKS_OK && zero_r32 &&   // the per-k density partials, consumed by the fold
      cudaMemsetAsync(c->d_rho32, 0, sizeof(float) * (size_t)c->ncell * c->nk * c->npts, c->stream) != cudaSuccess)
    st = fail(TDKS_ECUDA, "memset of the density partials");
  c->stream = main;
  TDKS_TRY(st);
  TDKS_CUDA(cudaEventRecord(c->ev_obs_join, c->obs_side));
  return TDKS_OK;
}

// The history slot the next step reads as V0: an accepted step's decision writes V_Hxc(t+dt)
// there, a fallback body copies it at its end.
static double* next_hist_slot(tdks_ctx* c) { return c->d_vhist + (size_t)((c->hist_head + 1) % 4) * c->npts; }

static tdks_status predicted_main(tdks_ctx* c, void* u, const double Amid[3], double dt, const double* Aobs,
                                  bool obs_start, bool obs_branch = false) {
  const size_t gb = c->npts * sizeof(double);
  const size_t obytes = (size_t)c->nk * c->norb * c->npts * (is_f32(c) ? sizeof(float2) : sizeof(double2));
  const NNGrid g = nn_grid(c);
  bool step_pot_done = false;
  {
    Phase ph(c, 5);
    if (c->pred_mode == TDKS_PRED_LEARNED) {   // statistics, inputs and the three layers: one launch
      NNPredict pr{hist_slot(c, 0), hist_slot(c, 1), hist_slot(c, 2), hist_slot(c, 3), c->d_vpred};
      if (c->ncell == 1) {   // the corrector's step potential too (what set_step_potential forms)
        pr.vloc = c->d_vloc; pr.vhxc = c->d_vhxc; pr.vstep64 = c->d_v64; pr.vstep32 = is_f32(c) ? c->d_v32 : nullptr;
      }
      TDKS_CUDA(nn_predict_fused(c->nn, g, pr, c->wait_limit, c->stream));
      c->launches += 1;
      step_pot_done = c->ncell == 1;
    } else {
      TDKS_CUDA(nn_apply(c->nn, g, hist_slot(c, 0), hist_slot(c, 1), hist_slot(c, 2), hist_slot(c, 3), 1,
                         c->d_vpred, c->stream));
      c->launches += 1;
    }
    // the shared-memory cell kernel writes the backup while it loads the orbitals; the tile path
    // copies it first
    if (c->tiled) TDKS_CUDA(cudaMemcpyAsync(c->d_backup, u, obytes, cudaMemcpyDeviceToDevice, c->stream));
    if (!rho_overwritten(c)) TDKS_CUDA(cudaMemsetAsync(c->d_rho, 0, gb, c->stream));
  }
  if (!step_pot_done) TDKS_TRY(set_step_potential(c, 0.5, c->d_vpred, 0.5));
  c->cur_backup = c->tiled ? nullptr : c->d_backup;
  // in a step graph the per-k density partials are zeroed on the observables branch
  const bool defer = obs_branch && rho_overwritten(c);
  c->defer_r32_zero = defer;
  const tdks_status cs = orbital_kernel(c, 1, u, u, Amid, dt, c->d_rho, 1, Aobs, obs_start);
  c->defer_r32_zero = false;
  c->cur_backup = nullptr;
  TDKS_TRY(cs);
  if (obs_branch) TDKS_TRY(fork_step_observables(c, obs_start, defer));
  // the misfit: formed by the Hartree solve's last launch where it can (one periodic cell, xc
  // without the TB-mBJ exchange, which is added after it), else by its own kernel.  In a step graph
  // that launch also takes the accept decision: V_Hxc(t+dt) goes straight to d_vhxc and to the next
  // history slot (a fallback body restores d_vhxc from the history first).
  const bool fuse = c->opt.xc != 3 && c->opt.hartree && c->plane_cl >= 2;
  const bool decide = obs_branch && c->cap_decide && fuse;
  ResidualArgs ra{c->d_vpred, c->d_partials, c->d_ticket, c->d_resid, 0, decide ? 1 : 0, c->pred_thr,
                  decide ? next_hist_slot(c) : nullptr, c->d_fb, c->cap_handle};
  c->res_args = c->opt.xc != 3 ? &ra : nullptr;
  const tdks_status hs = hxc(c, c->d_rho, decide ? c->d_vhxc : c->d_vnew, u);
  c->res_args = nullptr;
  TDKS_TRY(hs);
  c->cap_decided = decide && ra.done;
  if (!ra.done) {
    TDKS_CUDA(launch_residual(c->d_vnew, c->d_vpred, c->npts, c->d_partials, c->d_ticket, c->d_resid, c->stream));
    c->launches += 1;
  }
  return TDKS_OK;
}



// Add the step-graph timings of the last execution of slot v to the phase times.
static tdks_status collect_graph(tdks_ctx* c, tdks_ctx::StepGraph& g) {
  if (!g.pending) return TDKS_OK;
  for (auto& r : g.recs) {
    float ms = 0.f;
    TDKS_CUDA(cudaEventSynchronize(r.b));
    TDKS_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
    c->ms[r.phase] += ms;
  }
  g.pending = false;
  return TDKS_OK;
}

static tdks_status collect_step_graph(tdks_ctx* c, int v) { return collect_graph(c, c->sg[v]); }

static void drop_graph(tdks_ctx* c, tdks_ctx::StepGraph& g) {
  collect_graph(c, g);
  if (g.exec) cudaGraphExecDestroy(g.exec);
  if (g.graph) cudaGraphDestroy(g.graph);
  for (auto& r : g.recs) { c->event_pool.push_back(r.a); c->event_pool.push_back(r.b); }
  g = tdks_ctx::StepGraph{};
}

static void drop_step_graphs(tdks_ctx* c) {
  cudaStreamSynchronize(c->stream);
  for (int v = 0; v < 4; ++v) drop_graph(c, c->sg[v]);
}

static void drop_ms_graphs(tdks_ctx* c) {
  cudaStreamSynchronize(c->stream);
  for (int v = 0; v < 3; ++v) drop_graph(c, c->msg[v]);
}

// Capture the step graph of history slot v = c->hist_head (see tdks_ctx::StepGraph).
static tdks_status build_step_graph(tdks_ctx* c, void* u, double dt, const double* Aobs, bool obs_start) {
  auto& g = c->sg[c->hist_head];
  if (!c->cap) TDKS_CUDA(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
  if (!c->cap2) TDKS_CUDA(cudaStreamCreateWithFlags(&c->cap2, cudaStreamNonBlocking));
  if (c->tiled && !c->side2) TDKS_CUDA(cudaStreamCreateWithFlags(&c->side2, cudaStreamNonBlocking));
  if (!c->obs_side) TDKS_CUDA(cudaStreamCreateWithFlags(&c->obs_side, cudaStreamNonBlocking));
  if (!c->ev_obs_fork) TDKS_CUDA(cudaEventCreateWithFlags(&c->ev_obs_fork, cudaEventDisableTiming));
  if (!c->ev_obs_join) TDKS_CUDA(cudaEventCreateWithFlags(&c->ev_obs_join, cudaEventDisableTiming));
  const cudaStream_t main = c->stream;
  const bool prof = c->profiling;
  const long long launches0 = c->launches;
  long long calls0[TDKS_NPHASE];
  std::memcpy(calls0, c->calls, sizeof(calls0));
  const size_t obytes = (size_t)c->nk * c->norb * c->npts * (is_f32(c) ? sizeof(float2) : sizeof(double2));
  const double zero[3] = {0.0, 0.0, 0.0};
  c->cur_ap_mid = c->longitudinal ? c->d_ap_mid : c->d_apf;
  c->cur_ap_end = c->longitudinal ? c->d_ap_end : c->d_apf + 3;
  c->stream = c->cap;
  c->cap_recs = prof ? &g.recs : nullptr;
  long long body0 = 0, body1 = 0;
  tdks_status st = TDKS_OK;
  cudaError_t e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    cudaStreamCaptureStatus cst;
    cudaGraphConditionalHandle handle = 0;
    cudaGraphNode_t cn = nullptr;
    cudaGraph_t body = nullptr;
    // the conditional handle first: the Hartree solve's last launch may set it (see predicted_main)
    e = cudaStreamGetCaptureInfo(c->cap, &cst, nullptr, &cg, nullptr, nullptr, nullptr);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&handle, cg, 0, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
      c->cap_decide = true;
      c->cap_handle = handle;
      c->cap_decided = false;
      st = predicted_main(c, u, zero, dt, Aobs, obs_start, true);   // the kernels read A' from the device pointers
      c->cap_decide = false;
    }
    if (st == TDKS_OK && e == cudaSuccess) e = cudaStreamWaitEvent(c->cap, c->ev_obs_join, 0);   // join J and the dipole
    if (st == TDKS_OK && e == cudaSuccess && !c->cap_decided) {
      Phase ph(c, 5);
      e = launch_decide(c->d_resid, c->pred_thr, c->d_vnew, c->d_vhxc, next_hist_slot(c), c->npts, c->d_fb, handle,
                        c->stream);
      c->launches += 1;
    }
    if (st == TDKS_OK && e == cudaSuccess) e = cudaStreamGetCaptureInfo(c->cap, &cst, nullptr, &cg, &deps, nullptr, &ndeps);
    if (st == TDKS_OK && e == cudaSuccess) {
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = handle;
      cp.conditional.type = cudaGraphCondTypeIf;
      cp.conditional.size = 1;
      e = cudaGraphAddNode(&cn, cg, deps, nullptr, ndeps, &cp);
      if (e == cudaSuccess) body = cp.conditional.phGraph_out[0];
    }
    if (st == TDKS_OK && e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(c->cap, &cn, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (st == TDKS_OK && e == cudaSuccess) {
      // the fallback body: restore the orbitals, plain predictor-corrector (no profiling events: a
      // conditional body holds kernels, copies and memsets only)
      c->stream = c->cap2;
      c->body_side = c->side2;
      c->cap_recs = nullptr;
      c->profiling = false;
      body0 = c->launches;
      long long bc0[TDKS_NPHASE];
      std::memcpy(bc0, c->calls, sizeof(bc0));
      e = cudaStreamBeginCaptureToGraph(c->cap2, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
      if (e == cudaSuccess) {
        // V_Hxc(t) back from the history (the predicted step may have written its own into d_vhxc),
        // and the orbitals from the backup
        e = cudaMemcpyAsync(c->d_vhxc, hist_slot(c, 0), c->npts * sizeof(double), cudaMemcpyDeviceToDevice,
                            c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(u, c->d_backup, obytes, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess) st = pc_step(c, u, zero, Aobs ? zero : nullptr, obs_start, dt);
        if (e == cudaSuccess && st == TDKS_OK) st = step_observables(c, obs_start, c->d_partials, c->d_ticket);
        if (e == cudaSuccess && st == TDKS_OK)
          e = cudaMemcpyAsync(next_hist_slot(c), c->d_vhxc, c->npts * sizeof(double), cudaMemcpyDeviceToDevice,
                              c->stream);
        const cudaError_t e2 = cudaStreamEndCapture(c->cap2, &body);
        if (e == cudaSuccess) e = e2;
      }
      body1 = c->launches;
      for (int p = 0; p < TDKS_NPHASE; ++p) c->body_calls[p] = c->calls[p] - bc0[p];
      c->stream = c->cap;
      c->body_side = nullptr;
      c->cap_recs = prof ? &g.recs : nullptr;
      c->profiling = prof;
    }
    const cudaError_t e2 = cudaStreamEndCapture(c->cap, &g.graph);
    if (e == cudaSuccess) e = e2;
  }
  c->body_launches = body1 - body0;
  g.launches = c->launches - launches0 - c->body_launches;
  for (int p = 0; p < TDKS_NPHASE; ++p) g.calls[p] = c->calls[p] - calls0[p] - c->body_calls[p];
  c->launches = launches0;
  std::memcpy(c->calls, calls0, sizeof(calls0));
  c->stream = main;
  c->profiling = prof;
  c->cap_recs = nullptr;
  c->cur_ap_mid = c->cur_ap_end = nullptr;
  if (e == cudaSuccess && st == TDKS_OK) e = cudaGraphInstantiate(&g.exec, g.graph, 0);
  if (e != cudaSuccess || st != TDKS_OK) {
    cudaGetLastError();
    if (g.graph) cudaGraphDestroy(g.graph);
    for (auto& r : g.recs) { c->event_pool.push_back(r.a); c->event_pool.push_back(r.b); }
    g = tdks_ctx::StepGraph{};
    if (st != TDKS_OK) return st;
    return fail(TDKS_ECUDA, std::string("capture of the predicted step: ") + cudaGetErrorString(e));
  }
  return TDKS_OK;
}

// A predicted step without the step graph (tdks_set_step_graph(ctx, 0)): the same launches on the
// stream, the misfit read on the host (one synchronisation) and the fallback enqueued from the host.
// The caller adds the history update and the observables.
static tdks_status predicted_step_host(tdks_ctx* c, void* u, const double Amid[3], const double* Aobs,
                                       bool obs_start, double dt) {
  TDKS_TRY(predicted_main(c, u, Amid, dt, Aobs, obs_start));
  double r = 0.0;
  TDKS_CUDA(cudaMemcpyAsync(&r, c->d_resid, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  TDKS_CUDA(cudaStreamSynchronize(c->stream));
  const size_t gb = c->npts * sizeof(double);
  if (std::isfinite(r) && r <= c->pred_thr) {
    TDKS_CUDA(cudaMemcpyAsync(c->d_vhxc, c->d_vnew, gb, cudaMemcpyDeviceToDevice, c->stream));
    return TDKS_OK;
  }
  const size_t obytes = (size_t)c->nk * c->norb * c->npts * (is_f32(c) ? sizeof(float2) : sizeof(double2));
  TDKS_CUDA(cudaMemcpyAsync(u, c->d_backup, obytes, cudaMemcpyDeviceToDevice, c->stream));
  TDKS_TRY(sync_fallbacks(c));
  c->fallbacks += 1.0;
  c->fb_seen = c->fallbacks;
  TDKS_CUDA(cudaMemcpy(c->d_fb, &c->fallbacks, sizeof(double), cudaMemcpyHostToDevice));
  return pc_step(c, u, Amid, Aobs, obs_start, dt);
}

// One predicted step: the vector potentials to the device, then the step graph of the current history
// slot (built on first use).  No host synchronisation.
static tdks_status predicted_step(tdks_ctx* c, void* u, const double Amid[3], const double* Aobs, bool obs_start,
                                  double dt) {
  tdks_ctx::StepKey key;
  key.u = u; key.dt = dt; key.thr = c->pred_thr; key.mbj_c = c->mbj_c_fixed; key.mode = c->pred_mode;
  key.lg = c->longitudinal ? 1 : 0; key.has_obs = Aobs ? 1 : 0; key.obs_start = obs_start ? 1 : 0;
  key.cell_variant = c->cell_variant; key.tile0 = c->tile_variant[0]; key.tile1 = c->tile_variant[1];
  key.prof = c->profiling ? (c->prof_stencil_only ? 2 : 1) : 0;
  key.proj = c->proj_variant;
  if (!(key == c->sg_key)) {
    drop_step_graphs(c);
    c->sg_key = key;
  }
  if (!c->longitudinal) {
    Phase ph(c, 5);
    const double v[6] = {Amid[0], Amid[1], Amid[2], Aobs ? Aobs[0] : 0.0, Aobs ? Aobs[1] : 0.0, Aobs ? Aobs[2] : 0.0};
    TDKS_CUDA(launch_store6(c->d_apf, v, c->stream));
    c->launches += 1;
  }
  const int v = c->hist_head;
  auto& g = c->sg[v];
  if (!g.exec) TDKS_TRY(build_step_graph(c, u, dt, Aobs, obs_start));
  TDKS_TRY(collect_step_graph(c, v));
  TDKS_CUDA(cudaGraphLaunch(g.exec, c->stream));
  g.pending = c->profiling;
  c->launches += g.launches;
  for (int p = 0; p < TDKS_NPHASE; ++p) c->calls[p] += g.calls[p];
  c->hist_head = (v + 1) % 4;
  return TDKS_OK;
}

tdks_status tdks_step(tdks_ctx* c, void* u, double t, double dt) {
  TDKS_TRY(check_ctx(c));
  TDKS_TRY(check_whole_set(c, "tdks_step"));
  if (!u) return fail(TDKS_EINVAL, "null orbitals");
  if (!c->have_potential) return fail(TDKS_EINVAL, "call tdks_update_potential before tdks_step");
  double Amid[3], Aend[3], Astart[3];
  field_at(c, t + 0.5 * dt, Amid);
  field_at(c, t + dt, Aend);
  field_at(c, t, Astart);
  // observables of the input state (J(t), dipole of rho(t)) or of the propagated one
  const bool at_start = c->opt.obs_at_start != 0;
  const double* Aobs = c->grid.periodic ? (at_start ? Astart : Aend) : nullptr;
  if (at_start) {
    Phase ph(c, 4);
    TDKS_CUDA(launch_dipole(c->d_rho, c->d_rho0, c->grid.n, c->grid.h, c->grid.periodic,
                            c->d_partials, c->d_ticket, c->d_step_obs, c->stream));   // cell 0
    c->launches += 1;
  }
  if (c->longitudinal) {   // A' = A'_ext + A'_ind, A'_ind advanced from J(t) on the device
    Phase ph(c, 5);
    TDKS_CUDA(launch_longitudinal(c->d_step_obs, c->d_lg, c->lg_first, dt, Amid, Aend, c->d_ap_mid, c->d_ap_end,
                                  c->stream));
    c->launches += 1;
    c->lg_first = 0;
    c->cur_ap_mid = c->d_ap_mid;
    c->cur_ap_end = c->d_ap_end;
  }
  const bool predicted = c->pred_mode != TDKS_PRED_PC && c->hist_count >= 4 && (c->opt.hartree || c->opt.xc);
  if (predicted && c->step_graph) {
    const tdks_status st = predicted_step(c, u, Amid, Aobs, at_start, dt);   // history, J and dipole inside
    c->cur_ap_mid = c->cur_ap_end = nullptr;
    return st;
  }
  const tdks_status st = predicted ? predicted_step_host(c, u, Amid, Aobs, at_start, dt)
                                   : pc_step(c, u, Amid, Aobs, at_start, dt);
  c->cur_ap_mid = c->cur_ap_end = nullptr;
  TDKS_TRY(st);
  TDKS_TRY(hist_push(c, c->d_vhxc));
  return step_observables(c, at_start, c->d_partials, c->d_ticket);   // cell 0's dipole
}

tdks_status tdks_ms_init(tdks_ctx* c, int nX, int m0, double dX, const double* A_now, const double* A_prev) {
  TDKS_TRY(check_ctx(c));
  if (c->longitudinal) return fail(TDKS_EUNSUPPORTED, "the multiscale mode and the longitudinal geometry exclude each other");
  if (!c->grid.periodic) return fail(TDKS_EINVAL, "the multiscale mode needs periodic cells");
  if (!A_now || !A_prev || nX < 3 || m0 < 1 || m0 + c->ncell > nX - 1 || !(dX > 0.0))
    return fail(TDKS_EINVAL, "need nX >= 3, 1 <= m0, m0 + ncell <= nX - 1, dX > 0 and both A levels");
  if (!c->ms_ready || nX != c->nX) {
    for (int i = 0; i < 3; ++i) TDKS_TRY(dalloc(c, &c->d_A[i], nX));
    TDKS_TRY(dalloc(c, &c->d_I, nX));
    if (!c->d_ap_mid) {
      TDKS_TRY(dalloc(c, &c->d_ap_mid, 3 * (size_t)c->ncell));
      TDKS_TRY(dalloc(c, &c->d_ap_end, 3 * (size_t)c->ncell));
    }
  }
  drop_ms_graphs(c);
  c->ms_steps = 0;
  c->nX = nX; c->m0 = m0; c->dX = dX; c->ms_head = 0;
  TDKS_CUDA(cudaMemcpyAsync(c->d_A[0], A_now, nX * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  TDKS_CUDA(cudaMemcpyAsync(c->d_A[2], A_prev, nX * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  TDKS_CUDA(cudaMemsetAsync(c->d_I, 0, nX * sizeof(double), c->stream));
  TDKS_CUDA(cudaStreamSynchronize(c->stream));
  c->ms_ready = true;
  return TDKS_OK;
}

// One coupled multiscale step on c->stream: the Maxwell update of the macroscopic grid (A' of every
// cell at the half and full step), the predictor-corrector step of all cells with their own A', and
// the currents back to the grid.  Reads the three A levels selected by c->ms_head.
static tdks_status ms_step_body(tdks_ctx* c, void* u, double dt) {
  const double cl = 137.035999084;
  const int h = c->ms_head;
  double* Aprev = c->d_A[(h + 2) % 3];
  double* Anow = c->d_A[h];
  double* Anext = c->d_A[(h + 1) % 3];
  {
    Phase ph(c, 5);
    TDKS_CUDA(launch_maxwell(Aprev, Anow, Anext, c->d_I, c->nX, c->m0, c->ncell, cl * dt / c->dX,
                             4.0 * kPi * cl * dt * dt, 1.0 / cl, c->d_ap_mid, c->d_ap_end, c->stream));
    c->launches += 1;
  }
  const double zero[3] = {0.0, 0.0, 0.0};
  c->cur_ap_mid = c->d_ap_mid;
  c->cur_ap_end = c->d_ap_end;
  const tdks_status st = pc_step(c, u, zero, zero, false, dt);   // per-cell A' via cur_ap_*
  c->cur_ap_mid = c->cur_ap_end = nullptr;
  TDKS_TRY(st);
  Phase ph(c, 4);
  TDKS_CUDA(launch_reduce_current(c->d_orb_obs, c->nk, c->norb, c->d_kw, 1.0 / c->omega, 1,
                                  c->d_step_obs, c->stream, c->ncell));
  TDKS_CUDA(launch_ms_current(c->d_step_obs, c->ncell, c->m0, c->d_I, c->stream));
  c->launches += 2;
  return TDKS_OK;
}

// Capture ms_step_body for the current c->ms_head into c->msg[c->ms_head].
static tdks_status build_ms_graph(tdks_ctx* c, void* u, double dt) {
  auto& g = c->msg[c->ms_head];
  if (!c->cap) TDKS_CUDA(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
  const cudaStream_t main = c->stream;
  const long long launches0 = c->launches;
  long long calls0[TDKS_NPHASE];
  std::memcpy(calls0, c->calls, sizeof(calls0));
  c->stream = c->cap;
  c->cap_recs = c->profiling ? &g.recs : nullptr;
  tdks_status st = TDKS_OK;
  cudaError_t e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    st = ms_step_body(c, u, dt);
    const cudaError_t e2 = cudaStreamEndCapture(c->cap, &g.graph);
    if (e == cudaSuccess) e = e2;
  }
  g.launches = c->launches - launches0;
  for (int p = 0; p < TDKS_NPHASE; ++p) g.calls[p] = c->calls[p] - calls0[p];
  c->launches = launches0;
  std::memcpy(c->calls, calls0, sizeof(calls0));
  c->stream = main;
  c->cap_recs = nullptr;
  if (e == cudaSuccess && st == TDKS_OK) e = cudaGraphInstantiate(&g.exec, g.graph, 0);
  if (e != cudaSuccess || st != TDKS_OK) {
    cudaGetLastError();
    if (g.graph) cudaGraphDestroy(g.graph);
    for (auto& r : g.recs) { c->event_pool.push_back(r.a); c->event_pool.push_back(r.b); }
    g = tdks_ctx::StepGraph{};
    if (st != TDKS_OK) return st;
    return fail(TDKS_ECUDA, std::string("capture of the multiscale step: ") + cudaGetErrorString(e));
  }
  return TDKS_OK;
}

tdks_status tdks_ms_step(tdks_ctx* c, void* u, double t, double dt) {
  TDKS_TRY(check_ctx(c));
  TDKS_TRY(check_whole_set(c, "tdks_ms_step"));
  if (!u) return fail(TDKS_EINVAL, "null orbitals");
  if (!c->ms_ready) return fail(TDKS_EINVAL, "call tdks_ms_init first");
  if (!c->have_potential) return fail(TDKS_EINVAL, "call tdks_update_potential before tdks_ms_step");
  (void)t;
  const int h = c->ms_head;
  if (c->step_graph && c->ms_steps > 0) {
    // a replay of the step's graph: one launch, no host work between the kernels
    tdks_ctx::MsKey key;
    key.u = u; key.dt = dt; key.mbj_c = c->mbj_c_fixed; key.cell_variant = c->cell_variant;
    key.tile0 = c->tile_variant[0]; key.tile1 = c->tile_variant[1];
    key.prof = c->profiling ? (c->prof_stencil_only ? 2 : 1) : 0;
    if (!(key == c->msg_key)) {
      drop_ms_graphs(c);
      c->msg_key = key;
    }
    auto& g = c->msg[h];
    if (!g.exec) TDKS_TRY(build_ms_graph(c, u, dt));
    TDKS_TRY(collect_graph(c, g));
    TDKS_CUDA(cudaGraphLaunch(g.exec, c->stream));
    g.pending = c->profiling;
    c->launches += g.launches;
    for (int p = 0; p < TDKS_NPHASE; ++p) c->calls[p] += g.calls[p];
  } else {
    TDKS_TRY(ms_step_body(c, u, dt));
  }
  c->ms_steps += 1;
  c->ms_head = (h + 1) % 3;
  return TDKS_OK;
}

tdks_status tdks_ms_size(const tdks_ctx* c, int* nX) {
  TDKS_TRY(check_ctx(c));
  if (!nX) return fail(TDKS_EINVAL, "null output");
  *nX = c->ms_ready ? c->nX : 0;
  return TDKS_OK;
}

tdks_status tdks_ms_read(tdks_ctx* c, double* A_host, double* I_host) {
  TDKS_TRY(check_ctx(c));
  if (!c->ms_ready) return fail(TDKS_EINVAL, "call tdks_ms_init first");
  if (A_host) TDKS_CUDA(cudaMemcpyAsync(A_host, c->d_A[c->ms_head], c->nX * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (I_host) TDKS_CUDA(cudaMemcpyAsync(I_host, c->d_I, c->nX * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  TDKS_CUDA(cudaStreamSynchronize(c->stream));
  return TDKS_OK;
}


namespace {

// Enqueue the copy of the step-observable block of the first cell (J[3], dipole[3], n_elec, 0,
// misfit, 0, fallback count) into h on the context stream.
cudaError_t copy_step_obs(tdks_ctx* c, double* h) {
  if (c->ncell == 1)         // J, dipole, N, misfit, fallback count: one copy
    return cudaMemcpyAsync(h, c->d_step_obs, TDKS_STEP_OBS_DOUBLES * sizeof(double), cudaMemcpyDeviceToHost,
                           c->stream);
  cudaError_t e = cudaMemcpyAsync(h, c->d_step_obs, 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h + 8, c->d_resid, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  return e;
}

// Fill o from a copied block; fallbacks seen for the first time add the launches and phase calls of
// the predictor-corrector body they ran to the context's counters.
void unpack_step_obs(tdks_ctx* c, const double* h, tdks_obs* o) {
  const double fb = h[10];
  if (fb > c->fb_seen) {
    const long long n = (long long)(fb - c->fb_seen);
    c->launches += n * c->body_launches;
    for (int p = 0; p < TDKS_NPHASE; ++p) c->calls[p] += n * c->body_calls[p];
    c->fb_seen = fb;
  }
  if (fb > c->fallbacks) c->fallbacks = fb;
  std::memset(o, 0, sizeof(*o));
  for (int a = 0; a < 3; ++a) { o->J[a] = h[a]; o->dipole[a] = h[3 + a]; }
  o->n_elec = h[6];
  o->residual = h[8];
  o->fallbacks = fb;
}

}  // namespace

tdks_status tdks_read_step_observables(tdks_ctx* c, tdks_obs* o) {
  TDKS_TRY(check_ctx(c));
  if (!o) return fail(TDKS_EINVAL, "null output");
  TDKS_CUDA(copy_step_obs(c, c->h_resid));
  TDKS_CUDA(cudaStreamSynchronize(c->stream));
  unpack_step_obs(c, c->h_resid, o);
  return TDKS_OK;
}

tdks_status tdks_copy_step_observables(tdks_ctx* c, double* host_dst) {
  TDKS_TRY(check_ctx(c));
  if (!host_dst) return fail(TDKS_EINVAL, "null host buffer");
  TDKS_CUDA(copy_step_obs(c, host_dst));
  return TDKS_OK;
}

tdks_status tdks_unpack_step_observables(tdks_ctx* c, const double* host_src, tdks_obs* o) {
  TDKS_TRY(check_ctx(c));
  if (!host_src || !o) return fail(TDKS_EINVAL, "null argument");
  unpack_step_obs(c, host_src, o);
  return TDKS_OK;
}

tdks_status tdks_observables(tdks_ctx* c, const void* u, const double Ap[3], double* rho_out, tdks_obs* o) {
  TDKS_TRY(check_ctx(c));
  if (!u || !o) return fail(TDKS_EINVAL, "null argument");
  if (c->ncell > 1) return fail(TDKS_EUNSUPPORTED, "tdks_observables needs ncell = 1");
  double A[3] = {0, 0, 0};
  if (Ap && c->grid.periodic) for (int a = 0; a < 3; ++a) A[a] = Ap[a];
  TDKS_TRY(density(c, u, c->d_rho_tmp));
  if (rho_out)
    TDKS_CUDA(cudaMemcpyAsync(rho_out, c->d_rho_tmp, c->npts * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  const double* r0 = c->have_rho0 ? c->d_rho0 : c->d_rho_tmp;
  TDKS_CUDA(launch_dipole(c->d_rho_tmp, r0, c->grid.n, c->grid.h, c->grid.periodic, c->d_partials, c->d_ticket, c->d_step_obs, c->stream));
  TDKS_TRY(orbital_observables(c, u, A));
  const size_t no = (size_t)c->nk * c->norb;
  std::vector<double> ob(no * 8);
  double so[8];
  TDKS_CUDA(cudaMemcpyAsync(ob.data(), c->d_orb_obs, ob.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  TDKS_CUDA(cudaMemcpyAsync(so, c->d_step_obs, sizeof(so), cudaMemcpyDeviceToHost, c->stream));
  TDKS_CUDA(cudaStreamSynchronize(c->stream));
  std::memset(o, 0, sizeof(*o));
  o->norm_min = 1e300;
  o->norm_max = -1e300;
  double J[3] = {0, 0, 0}, eb = 0.0;
  bool finite = true;
  for (int k = 0; k < c->nk; ++k) {
    double js[3] = {0, 0, 0}, es = 0.0;
    for (int n = 0; n < c->norb; ++n) {
      const double* v = &ob[((size_t)k * c->norb + n) * 8];
      for (int a = 0; a < 3; ++a) js[a] += v[1 + a] + v[4 + a];
      es += v[7];
      o->norm_min = std::fmin(o->norm_min, v[0]);
      o->norm_max = std::fmax(o->norm_max, v[0]);
      if (!std::isfinite(v[0])) finite = false;
    }
    for (int a = 0; a < 3; ++a) J[a] += 2.0 * c->kw[k] * js[a];
    eb += 2.0 * c->kw[k] * es;
  }
  for (int a = 0; a < 3; ++a) {
    o->J[a] = c->grid.periodic ? -J[a] / c->omega : 0.0;
    o->dipole[a] = so[3 + a];
  }
  o->e_band = eb;
  o->n_elec = so[6];
  if (!finite) return fail(TDKS_ENONFINITE, "non-finite orbital norm");
  return TDKS_OK;
}

tdks_status tdks_get_grid_array(tdks_ctx* c, int which, double* dst) {
  TDKS_TRY(check_ctx(c));
  if (!dst) return fail(TDKS_EINVAL, "null destination");
  const double* src = nullptr;
  switch (which) {
    case 0: src = c->d_vloc; break;
    case 1: src = c->d_vhxc; break;
    case 2: src = c->d_rho; break;
    case 3: src = c->d_rho0; break;
    default: return fail(TDKS_EINVAL, "unknown grid array");
  }
  TDKS_CUDA(cudaMemcpyAsync(dst, src, c->npts * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  return TDKS_OK;
}

tdks_status tdks_check(tdks_ctx* c) {
  TDKS_TRY(check_ctx(c));
  TDKS_CUDA(cudaStreamSynchronize(c->stream));
  TDKS_CUDA(cudaGetLastError());
  int err = 0;
  TDKS_CUDA(cudaMemcpy(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err != 0) {
    cudaMemset(c->d_err, 0, sizeof(int));
    // a prediction whose grid barrier gave up left its counters behind
    if (c->nn_ready) cudaMemset(c->nn.bar, 0, 2 * sizeof(unsigned));
    return fail((tdks_status)err, "a device-side wait timed out (kernel gave up and returned)");
  }
  return TDKS_OK;
}

tdks_status tdks_set_step_graph(tdks_ctx* c, int enable) {
  TDKS_TRY(check_ctx(c));
  if (enable != 0 && enable != 1) return fail(TDKS_EINVAL, "enable must be 0 or 1");
  if (!enable) {
    drop_step_graphs(c);
    drop_ms_graphs(c);
  }
  c->step_graph = enable;
  return TDKS_OK;
}

tdks_status tdks_set_predictor(tdks_ctx* c, int mode, double threshold) {
  TDKS_TRY(check_ctx(c));
  if (mode < TDKS_PRED_PC || mode > TDKS_PRED_LEARNED) return fail(TDKS_EINVAL, "unknown predictor mode");
  if (!(threshold > 0.0)) return fail(TDKS_EINVAL, "threshold must be positive");
  if (mode == TDKS_PRED_LEARNED && !c->nn_ready) return fail(TDKS_EINVAL, "call tdks_nn_init first");
  if (mode != TDKS_PRED_PC && c->ncell > 1) return fail(TDKS_EUNSUPPORTED, "predicted steps need ncell = 1");
  if (mode != TDKS_PRED_PC && !c->d_backup) {
    const size_t obytes = (size_t)c->nk * c->norb * c->npts * (is_f32(c) ? sizeof(float2) : sizeof(double2));
    unsigned char* p = nullptr;
    TDKS_TRY(dalloc(c, &p, obytes));
    c->d_backup = p;
  }
  if (mode != TDKS_PRED_PC && !c->nn_ready) {   // the extrapolation uses the network's buffers too
    TDKS_TRY(tdks_nn_init(c, 0));
  }
  c->pred_mode = mode;
  c->pred_thr = threshold;
  return TDKS_OK;
}


tdks_status tdks_nn_init(tdks_ctx* c, unsigned long long seed) {
  TDKS_TRY(check_ctx(c));
  NNBuffers& B = c->nn;
  const size_t np = c->npts;
  if (!c->nn_ready) {
    TDKS_TRY(dalloc(c, &B.x0, 4 * np));
    TDKS_TRY(dalloc(c, &B.a1, 16 * np));
    TDKS_TRY(dalloc(c, &B.a2, 16 * np));
    TDKS_TRY(dalloc(c, &B.y1, 16 * np));
    TDKS_TRY(dalloc(c, &B.y2, 16 * np));
    TDKS_TRY(dalloc(c, &B.dy1, 16 * np));
    TDKS_TRY(dalloc(c, &B.dy2, 16 * np));
    TDKS_TRY(dalloc(c, &B.out, np));
    TDKS_TRY(dalloc(c, &B.target, np));
    TDKS_TRY(dalloc(c, &B.dout, np));
    TDKS_TRY(dalloc(c, &B.part, (size_t)nn_part_blocks(c->npts) * (16 * 16 * 27 + 16)));
    TDKS_TRY(dalloc(c, &B.params, kNNParams));
    TDKS_TRY(dalloc(c, &B.grad, kNNParams));
    TDKS_TRY(dalloc(c, &B.m, kNNParams));
    TDKS_TRY(dalloc(c, &B.v, kNNParams));
    TDKS_TRY(dalloc(c, &B.wq, kNNParams));
    TDKS_TRY(dalloc(c, &B.stats, 8));
    TDKS_TRY(dalloc(c, &B.loss, 1));
    TDKS_TRY(dalloc(c, &B.red, 304 * 5));
    TDKS_TRY(dalloc(c, &B.ticket, 1));
    TDKS_TRY(dalloc(c, &B.bar, 2));
    TDKS_CUDA(cudaMemsetAsync(B.bar, 0, 2 * sizeof(unsigned), c->stream));
    TDKS_TRY(dalloc(c, &B.wpack, nn_wpack_bytes() / sizeof(uint4)));
    TDKS_CUDA(cudaMemsetAsync(B.ticket, 0, sizeof(unsigned), c->stream));
    B.err = c->d_err;
  }
  std::vector<float> p(kNNParams, 0.0f);
  const int fan[3] = {4 * 27, 16 * 27, 16 * 27};
  const int woff[3] = {kNNOff[0], kNNOff[2], kNNOff[4]}, wlen[3] = {16 * 4 * 27, 16 * 16 * 27, 16 * 27};
  unsigned long long st = seed * 0x2545F4914F6CDD1DULL + 1;
  for (int l = 0; l < 3; ++l) {
    const double bound = (l == 2 ? 0.1 : 1.0) / std::sqrt((double)fan[l]);
    for (int i = 0; i < wlen[l]; ++i) p[woff[l] + i] = (float)((2.0 * uniform01(st) - 1.0) * bound);
  }
  TDKS_CUDA(cudaMemcpyAsync(B.params, p.data(), kNNParams * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  TDKS_CUDA(cudaMemsetAsync(B.grad, 0, kNNParams * sizeof(float), c->stream));
  TDKS_CUDA(cudaMemsetAsync(B.m, 0, kNNParams * sizeof(float), c->stream));
  TDKS_CUDA(cudaMemsetAsync(B.v, 0, kNNParams * sizeof(float), c->stream));
  TDKS_CUDA(nn_round_weights(B, c->stream));
  TDKS_CUDA(cudaStreamSynchronize(c->stream));
  c->nn_ready = true;
  c->nn_step = 0;
  return TDKS_OK;
}

tdks_status tdks_nn_params(tdks_ctx* c, float* host, int n, int set) {
  TDKS_TRY(check_ctx(c));
  if (!c->nn_ready) return fail(TDKS_EINVAL, "call tdks_nn_init first");
  if (!host || n != kNNParams) return fail(TDKS_EINVAL, "host buffer must hold TDKS_NN_NPARAMS floats");
  if (set) {
    TDKS_CUDA(cudaMemcpyAsync(c->nn.params, host, n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    TDKS_CUDA(nn_round_weights(c->nn, c->stream));
  } else {
    TDKS_CUDA(cudaMemcpyAsync(host, c->nn.params, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  }
  TDKS_CUDA(cudaStreamSynchronize(c->stream));
  return TDKS_OK;
}

tdks_status tdks_nn_train(tdks_ctx* c, const double* vseq, int nt, int epochs, int batch, double lr,
                          unsigned long long seed, double* loss_out) {
  TDKS_TRY(check_ctx(c));
  if (!c->nn_ready) return fail(TDKS_EINVAL, "call tdks_nn_init first");
  if (!vseq || nt < 5 || epochs < 1 || batch < 1 || !(lr > 0.0)) return fail(TDKS_EINVAL, "bad training arguments");
  const NNGrid g = nn_grid(c);
  const size_t np = c->npts;
  std::vector<int> order;
  for (int t = 3; t + 1 < nt; ++t) order.push_back(t);
  unsigned long long st = seed * 0x9E3779B97F4A7C15ULL + 7;
  for (int ep = 0; ep < epochs; ++ep) {
    for (size_t i = order.size(); i > 1; --i) std::swap(order[i - 1], order[splitmix64(st) % i]);
    TDKS_CUDA(cudaMemsetAsync(c->nn.loss, 0, sizeof(double), c->stream));
    for (size_t b0 = 0; b0 < order.size(); b0 += batch) {
      const size_t b1 = std::min(order.size(), b0 + (size_t)batch);
      for (size_t i = b0; i < b1; ++i) {
        const int t = order[i];
        const double* V0 = vseq + (size_t)t * np;
        TDKS_CUDA(nn_inputs(c->nn, g, V0, V0 - np, V0 - 2 * np, V0 - 3 * np, V0 + np, c->stream));
        TDKS_CUDA(nn_forward(c->nn, g, c->stream));
        TDKS_CUDA(nn_loss(c->nn, g, c->nn.loss, c->stream));
        TDKS_CUDA(nn_backward(c->nn, g, c->stream));
        c->launches += 15;
      }
      c->nn_step += 1;
      TDKS_CUDA(nn_adam(c->nn, (float)lr, c->nn_step, 1.0f / (float)(b1 - b0), c->stream));
      c->launches += 1;
    }
    double l = 0.0;
    TDKS_CUDA(cudaMemcpyAsync(&l, c->nn.loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    TDKS_CUDA(cudaStreamSynchronize(c->stream));
    if (loss_out) loss_out[ep] = l / (double)order.size();
  }
  return TDKS_OK;
}

tdks_status tdks_nn_predict(tdks_ctx* c, const double* vhist, double* vpred, int mode) {
  TDKS_TRY(check_ctx(c));
  if (!c->nn_ready) return fail(TDKS_EINVAL, "call tdks_nn_init first");
  if (!vhist || !vpred) return fail(TDKS_EINVAL, "null argument");
  if (mode < 0 || mode > 2) return fail(TDKS_EINVAL, "mode must be 0 (linear), 1 (cubic) or 2 (network)");
  const NNGrid g = nn_grid(c);
  const size_t np = c->npts;
  if (mode == 2) {
    const NNPredict pr{vhist, vhist + np, vhist + 2 * np, vhist + 3 * np, vpred};
    TDKS_CUDA(nn_predict_fused(c->nn, g, pr, c->wait_limit, c->stream));
    c->launches += 1;
  } else {
    TDKS_CUDA(nn_inputs(c->nn, g, vhist, vhist + np, vhist + 2 * np, vhist + 3 * np, nullptr, c->stream, false));
    TDKS_CUDA(nn_apply(c->nn, g, vhist, vhist + np, vhist + 2 * np, vhist + 3 * np, mode, vpred, c->stream));
    c->launches += 3;
  }
  return TDKS_OK;
}

tdks_status tdks_nn_gradient(tdks_ctx* c, const double* vhist, const double* vnext, double* loss,
                             float* grad) {
  TDKS_TRY(check_ctx(c));
  if (!c->nn_ready) return fail(TDKS_EINVAL, "call tdks_nn_init first");
  if (!vhist || !vnext || !loss || !grad) return fail(TDKS_EINVAL, "null argument");
  const NNGrid g = nn_grid(c);
  const size_t np = c->npts;
  TDKS_CUDA(cudaMemsetAsync(c->nn.grad, 0, kNNParams * sizeof(float), c->stream));
  TDKS_CUDA(cudaMemsetAsync(c->nn.loss, 0, sizeof(double), c->stream));
  TDKS_CUDA(nn_inputs(c->nn, g, vhist, vhist + np, vhist + 2 * np, vhist + 3 * np, vnext, c->stream));
  TDKS_CUDA(nn_forward(c->nn, g, c->stream));
  TDKS_CUDA(nn_loss(c->nn, g, c->nn.loss, c->stream));
  TDKS_CUDA(nn_backward(c->nn, g, c->stream));
  TDKS_CUDA(cudaMemcpyAsync(grad, c->nn.grad, kNNParams * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  TDKS_CUDA(cudaMemcpyAsync(loss, c->nn.loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  TDKS_CUDA(cudaMemsetAsync(c->nn.grad, 0, kNNParams * sizeof(float), c->stream));
  TDKS_CUDA(cudaStreamSynchronize(c->stream));
  return TDKS_OK;
}

tdks_status tdks_profile(tdks_ctx* c, int enable) {
  TDKS_TRY(check_ctx(c));
  if (enable < 0 || enable > 2) return fail(TDKS_EINVAL, "enable must be 0, 1 or 2");
  c->profiling = enable != 0;
  c->prof_stencil_only = enable == 2;
  return TDKS_OK;
}

tdks_status tdks_stats_read(tdks_ctx* c, tdks_stats* out, int reset) {
  TDKS_TRY(check_ctx(c));
  if (!out) return fail(TDKS_EINVAL, "null output");
  TDKS_TRY(sync_fallbacks(c));
  for (int v = 0; v < 4; ++v) TDKS_TRY(collect_step_graph(c, v));
  for (int v = 0; v < 3; ++v) TDKS_TRY(collect_graph(c, c->msg[v]));
  for (auto& r : c->recs) {
    float ms = 0.0f;
    TDKS_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
    c->ms[r.phase] += ms;
    c->event_pool.push_back(r.a);
    c->event_pool.push_back(r.b);
  }
  c->recs.clear();
  out->launches = c->launches;
  for (int p = 0; p < TDKS_NPHASE; ++p) { out->calls[p] = c->calls[p]; out->ms[p] = c->ms[p]; }
  if (reset) {
    c->launches = 0;
    for (int p = 0; p < TDKS_NPHASE; ++p) { c->calls[p] = 0; c->ms[p] = 0.0; }
  }
  return TDKS_OK;
}

tdks_status tdks_project_variant(tdks_ctx* c, int set, int* variant, float* tune_ms) {
  TDKS_TRY(check_ctx(c));
  if (set < -1 || set >= kProjVariants) return fail(TDKS_EINVAL, "projection schedule outside -1..2");
  if (!c->tiled || !is_f32(c))
    return fail(TDKS_EUNSUPPORTED, "the projection schedules belong to the FP32 tile kernels");
  if (set >= 0) c->proj_variant = set;
  if (variant) *variant = c->proj_variant;
  if (tune_ms)
    for (int v = 0; v < kProjVariants; ++v) tune_ms[v] = c->proj_ms[v];
  return TDKS_OK;
}

tdks_status tdks_tile_variant(tdks_ctx* c, int set, int* variant, float* tune_ms) {
  TDKS_TRY(check_ctx(c));
  if (set < -1 || set >= kTileVariants) return fail(TDKS_EINVAL, "tile variant outside -1..6");
  if (!c->tiled) return fail(TDKS_EUNSUPPORTED, "this context does not use the tile kernels");
  if (set > 1 && !is_f32(c)) return fail(TDKS_EUNSUPPORTED, "tile variants 2 to 6 are FP32 only");
  if (set >= 0 && !tile_variant_ok(set, c->grid.n[0], is_f32(c) ? 8 : 16))
    return fail(TDKS_EUNSUPPORTED, "tile variants 5 and 6 need nx divisible by 4");
  if (set >= 0) c->tile_variant[0] = c->tile_variant[1] = set;
  if (variant) { variant[0] = c->tile_variant[0]; variant[1] = c->tile_variant[1]; }
  if (tune_ms)
    for (int m = 0; m < 2; ++m)
      for (int v = 0; v < kTileVariants; ++v) tune_ms[m * kTileVariants + v] = c->tile_ms[m][v];
  return TDKS_OK;
}

tdks_status tdks_cell_variant(tdks_ctx* c, int set, int* variant, float* tune_ms) {
  TDKS_TRY(check_ctx(c));
  if (set < -1 || set > 3) return fail(TDKS_EINVAL, "cell variant outside -1..3");
  if (c->tiled) return fail(TDKS_EUNSUPPORTED, "this context uses the tile kernels");
  if (set == 1 && !cell_ip_ok(c))
    return fail(TDKS_EUNSUPPORTED, "the in-place sweep needs nx * ny <= 448 and one orbital copy in shared memory");
  if (set == 2 && !cell_geom_ok(c))
    return fail(TDKS_EUNSUPPORTED, "the built-in geometries are the periodic 20^3 and 16^3 grids with two "
                                   "orbital copies in shared memory");
  if (set == 3 && !cell_geom_ip_ok(c))
    return fail(TDKS_EUNSUPPORTED, "the built-in geometries swept in place are the periodic 20^3 and 16^3 grids "
                                   "with FP32 orbitals");
  if (set >= 0) c->cell_variant = set;
  if (variant) *variant = c->cell_variant;
  if (tune_ms)
    for (int v = 0; v < 4; ++v) tune_ms[v] = c->cell_ms[v];
  return TDKS_OK;
}

tdks_status tdks_set_wait_test(tdks_ctx* c, long long wait_limit, int stop_after) {
  TDKS_TRY(check_ctx(c));
  if (wait_limit < 0) return fail(TDKS_EINVAL, "wait_limit must be >= 0");
  c->wait_limit = wait_limit > 0 ? wait_limit : (1LL << 22);
  c->stop_after = stop_after < 0 ? -1 : stop_after;
  return TDKS_OK;
}

// ------------------------------------------------------------------ checkpoint
namespace {
struct StateHeader {
  char magic[8];            // "TDKSSTA2"
  int npts, ncell, nk, norb, precision, natom, periodic;
  int hartree, xc, pc;
  int have_rho0, have_potential;
  int hist_head, hist_count;
  int pred_mode, nn_ready;
  double pred_thr, fallbacks, last_resid;
  int field_kind;
  double A0[3];
  int npulse;
  PulseDef pulse[kMaxPulses];
  int ntable;                 // field table rows, stored after the arrays
  double tab_t0, tab_dt;
  int longitudinal, lg_first;
  double lg[6], lg_J[3];      // A'_ind levels and the current J(t_n) the next leapfrog step reads
  int ms_ready, nX, m0, ms_head;
  double dX;
};

size_t state_bytes(const tdks_ctx* c) {
  const size_t npc = (size_t)c->npts * c->ncell;
  size_t b = sizeof(StateHeader) + sizeof(double) * (3 * npc + 4 * (size_t)c->npts);
  if (c->nn_ready) b += sizeof(float) * kNNParams;
  if (c->ms_ready) b += sizeof(double) * 4 * (size_t)c->nX;
  b += sizeof(double) * c->ftable.size();
  return b;
}
}  // namespace

tdks_status tdks_state_size(const tdks_ctx* c, size_t* bytes) {
  TDKS_TRY(check_ctx(c));
  if (!bytes) return fail(TDKS_EINVAL, "null output");
  *bytes = state_bytes(c);
  return TDKS_OK;
}

tdks_status tdks_get_state(tdks_ctx* c, void* host, size_t bytes) {
  TDKS_TRY(check_ctx(c));
  if (!host || bytes < state_bytes(c)) return fail(TDKS_EINVAL, "state buffer smaller than tdks_state_size");
  TDKS_TRY(sync_fallbacks(c));
  StateHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, "TDKSSTA2", 8);
  h.npts = c->npts; h.ncell = c->ncell; h.nk = c->nk; h.norb = c->norb; h.precision = c->opt.precision;
  h.natom = c->natom; h.periodic = c->grid.periodic;
  h.hartree = c->opt.hartree; h.xc = c->opt.xc; h.pc = c->opt.pc;
  h.have_rho0 = c->have_rho0; h.have_potential = c->have_potential;
  h.hist_head = c->hist_head; h.hist_count = c->hist_count;
  h.pred_mode = c->pred_mode; h.nn_ready = c->nn_ready;
  h.pred_thr = c->pred_thr; h.fallbacks = c->fallbacks; h.last_resid = c->last_resid;
  h.field_kind = c->field_kind;
  for (int a = 0; a < 3; ++a) h.A0[a] = c->A0[a];
  h.npulse = (int)c->pulses.size();
  for (int i = 0; i < h.npulse; ++i) h.pulse[i] = c->pulses[i];
  h.ntable = (int)(c->ftable.size() / 3);
  h.tab_t0 = c->tab_t0; h.tab_dt = c->tab_dt;
  h.longitudinal = c->longitudinal; h.lg_first = c->lg_first;
  if (c->d_lg) {
    TDKS_CUDA(cudaMemcpyAsync(h.lg, c->d_lg, 6 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    TDKS_CUDA(cudaMemcpyAsync(h.lg_J, c->d_step_obs, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    TDKS_CUDA(cudaStreamSynchronize(c->stream));
  }
  h.ms_ready = c->ms_ready; h.nX = c->nX; h.m0 = c->m0; h.ms_head = c->ms_head; h.dX = c->dX;
  unsigned char* o = static_cast<unsigned char*>(host);
  std::memcpy(o, &h, sizeof(h));
  o += sizeof(h);
  const size_t npc = (size_t)c->npts * c->ncell;
  auto d2h = [&](const void* src, size_t nbytes) -> cudaError_t {
    const cudaError_t e = cudaMemcpyAsync(o, src, nbytes, cudaMemcpyDeviceToHost, c->stream);
    o += nbytes;
    return e;
  };
  TDKS_CUDA(d2h(c->d_vhxc, npc * sizeof(double)));
  TDKS_CUDA(d2h(c->d_rho, npc * sizeof(double)));
  TDKS_CUDA(d2h(c->d_rho0, npc * sizeof(double)));
  TDKS_CUDA(d2h(c->d_vhist, 4 * (size_t)c->npts * sizeof(double)));
  if (c->nn_ready) TDKS_CUDA(d2h(c->nn.params, kNNParams * sizeof(float)));
  if (c->ms_ready) {
    for (int i = 0; i < 3; ++i) TDKS_CUDA(d2h(c->d_A[i], c->nX * sizeof(double)));
    TDKS_CUDA(d2h(c->d_I, c->nX * sizeof(double)));
  }
  if (!c->ftable.empty()) std::memcpy(o, c->ftable.data(), sizeof(double) * c->ftable.size());
  TDKS_CUDA(cudaStreamSynchronize(c->stream));
  return TDKS_OK;
}

tdks_status tdks_set_state(tdks_ctx* c, const void* host, size_t bytes) {
  TDKS_TRY(check_ctx(c));
  if (!host || bytes < sizeof(StateHeader)) return fail(TDKS_EINVAL, "state buffer too small");
  StateHeader h;
  std::memcpy(&h, host, sizeof(h));
  if (std::memcmp(h.magic, "TDKSSTA2", 8) != 0) return fail(TDKS_EINVAL, "not a tdks state (bad magic)");
  if (h.field_kind < TDKS_FIELD_NONE || h.field_kind > TDKS_FIELD_TABLE || h.npulse < 0 || h.npulse > kMaxPulses ||
      h.ntable < 0 || (h.field_kind == TDKS_FIELD_TABLE && (h.ntable < 1 || !(h.tab_dt > 0.0))))
    return fail(TDKS_EINVAL, "state holds an invalid field description");
  if (h.npts != c->npts || h.ncell != c->ncell || h.nk != c->nk || h.norb != c->norb ||
      h.precision != c->opt.precision || h.natom != c->natom || h.periodic != c->grid.periodic ||
      h.hartree != c->opt.hartree || h.xc != c->opt.xc || h.pc != c->opt.pc)
    return fail(TDKS_EINVAL, "state was written by a context of another system or options");
  if (h.nn_ready && !c->nn_ready) TDKS_TRY(tdks_nn_init(c, 0));
  if (h.ms_ready && (!c->ms_ready || c->nX != h.nX)) {
    for (int i = 0; i < 3; ++i) TDKS_TRY(dalloc(c, &c->d_A[i], h.nX));
    TDKS_TRY(dalloc(c, &c->d_I, h.nX));
    if (!c->d_ap_mid) {
      TDKS_TRY(dalloc(c, &c->d_ap_mid, 3 * (size_t)c->ncell));
      TDKS_TRY(dalloc(c, &c->d_ap_end, 3 * (size_t)c->ncell));
    }
  }
  // sizes as the writer had them
  const size_t npc = (size_t)c->npts * c->ncell;
  size_t need = sizeof(StateHeader) + sizeof(double) * (3 * npc + 4 * (size_t)c->npts);
  if (h.nn_ready) need += sizeof(float) * kNNParams;
  if (h.ms_ready) need += sizeof(double) * 4 * (size_t)h.nX;
  need += sizeof(double) * 3 * (size_t)h.ntable;
  if (bytes < need) return fail(TDKS_EINVAL, "state buffer shorter than its header says");
  if (h.pred_mode != TDKS_PRED_PC) TDKS_TRY(tdks_set_predictor(c, h.pred_mode, h.pred_thr));
  else c->pred_mode = TDKS_PRED_PC;
  const unsigned char* in = static_cast<const unsigned char*>(host) + sizeof(h);
  auto h2d = [&](void* dst, size_t nbytes) -> cudaError_t {
    const cudaError_t e = cudaMemcpyAsync(dst, in, nbytes, cudaMemcpyHostToDevice, c->stream);
    in += nbytes;
    return e;
  };
  TDKS_CUDA(h2d(c->d_vhxc, npc * sizeof(double)));
  TDKS_CUDA(h2d(c->d_rho, npc * sizeof(double)));
  TDKS_CUDA(h2d(c->d_rho0, npc * sizeof(double)));
  TDKS_CUDA(h2d(c->d_vhist, 4 * (size_t)c->npts * sizeof(double)));
  if (h.nn_ready) {
    TDKS_CUDA(h2d(c->nn.params, kNNParams * sizeof(float)));
    TDKS_CUDA(nn_round_weights(c->nn, c->stream));
  }
  if (h.ms_ready) {
    for (int i = 0; i < 3; ++i) TDKS_CUDA(h2d(c->d_A[i], h.nX * sizeof(double)));
    TDKS_CUDA(h2d(c->d_I, h.nX * sizeof(double)));
  }
  c->have_rho0 = h.have_rho0; c->have_potential = h.have_potential;
  c->hist_head = h.hist_head; c->hist_count = h.hist_count;
  c->pred_thr = h.pred_thr; c->fallbacks = h.fallbacks; c->last_resid = h.last_resid;
  c->fb_seen = h.fallbacks;
  TDKS_CUDA(cudaMemcpyAsync(c->d_fb, &c->fallbacks, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  c->field_kind = h.field_kind;
  for (int a = 0; a < 3; ++a) c->A0[a] = h.A0[a];
  c->pulses.assign(h.pulse, h.pulse + h.npulse);
  c->ftable.resize(3 * (size_t)h.ntable);
  if (h.ntable > 0) std::memcpy(c->ftable.data(), in, sizeof(double) * c->ftable.size());
  in += sizeof(double) * c->ftable.size();
  c->tab_t0 = h.tab_t0; c->tab_dt = h.tab_dt;
  if (h.longitudinal) {
    if (!c->grid.periodic || c->ncell != 1 || c->opt.obs_at_start)
      return fail(TDKS_EINVAL, "state holds the longitudinal geometry, which this context cannot use");
    if (!c->d_lg) TDKS_TRY(dalloc(c, &c->d_lg, 6));
    if (!c->d_ap_mid) {
      TDKS_TRY(dalloc(c, &c->d_ap_mid, 3 * (size_t)c->ncell));
      TDKS_TRY(dalloc(c, &c->d_ap_end, 3 * (size_t)c->ncell));
    }
    TDKS_CUDA(cudaMemcpyAsync(c->d_lg, h.lg, 6 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  }
  c->longitudinal = h.longitudinal; c->lg_first = h.lg_first;
  c->ms_ready = h.ms_ready; c->nX = h.nX; c->m0 = h.m0; c->ms_head = h.ms_head; c->dX = h.dX;
  drop_ms_graphs(c);
  c->ms_steps = 0;
  // the step potential follows from V_Hxc at the next step; the observables buffer is reset
  TDKS_CUDA(cudaMemsetAsync(c->d_step_obs, 0, 8 * sizeof(double) * c->ncell, c->stream));
  if (h.longitudinal)   // the current the next leapfrog step of A'_ind reads
    TDKS_CUDA(cudaMemcpyAsync(c->d_step_obs, h.lg_J, 3 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  TDKS_CUDA(cudaStreamSynchronize(c->stream));
  return TDKS_OK;
}

tdks_status tdks_query(const tdks_ctx* c, int* npts, int* nk, int* norb, int* precision, int* nsph) {
  TDKS_TRY(check_ctx(c));
  if (npts) *npts = c->npts;
  if (nk) *nk = c->nk;
  if (norb) *norb = c->norb;
  if (precision) *precision = c->opt.precision;
  if (nsph) *nsph = c->nsph;
  return TDKS_OK;
}

}  // extern "C"
