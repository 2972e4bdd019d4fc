// C ABI of the GB300 PIC library (declared in include/pic.h): validation,
// device memory layout, step scheduling, diagnostics and state access.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/pic.h"
#include "pic_kernels.cuh"
#include "pic_batch.cuh"

using namespace pg;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
  g_err = msg;
  return code;
}

#define PIC_CUDA(call)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(PIC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));       \
  } while (0)

constexpr size_t kAlign = 256;
constexpr int kSpecMax = 65536;
constexpr int kThreads = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Everything derived from the inputs, shared by pic_query and pic_create.
struct Plan {
  pic_grid g;
  std::vector<pic_layer> layers;
  pic_pulse pulse;
  int rsz;  // bytes per real
  double dt, omega, E0, V;
  double Tsin2;  // sine-squared envelope duration
  int NW, n_mplanes;
  long long nxy, nfield, ncell, nmat, n_neutrals, cap;
  std::vector<int> lop, mplane, kplane, vplane;
  int nb_scan, diag_blocks_p, diag_blocks_g;
  // arena offsets
  size_t off_E[3], off_B[3], off_Bh[3], off_J4, off_P[3], off_Q[3];
  size_t off_lop, off_mplane, off_kplane, off_vplane, off_lk, off_lr;
  size_t off_win, off_pm, off_eamp, off_ckey, off_T, off_alive, off_leave;
  size_t off_pc[2], off_po[2][3], off_pu[2][3], off_pt[2], off_pid[2];
  size_t off_cnt, off_bsum, off_total, off_nslots, off_step, off_acc, off_err;
  size_t off_work, off_work_n, off_leave16;
  size_t off_imax, off_prof;
  size_t off_clist, off_cn;  // collision cell list and its counters
  size_t off_hot;            // hot-plane stamps (n_mplanes + 1)
  size_t off_jtouch;         // deposit-plane marks (nz + 2)
  size_t off_cpar, off_cord, off_clike, off_cunl;  // collision work (coll_every > 0)
  int imax_every;  // steps between intensity records, 0 = off
  int ppc_max;
  size_t off_ne, off_ed, off_rho, off_spec, off_part;
  size_t off_flux_part;
  size_t off_ktab;               // elliptic tables (elliptic_table > 0)
  size_t off_psi[12];            // absorbing-layer convolution terms (pml_cells > 0):
                                 // eight, then the B terms after a closing half step
  size_t off_pmlb;               // their decay factors: E along x, y; B along x, y
  std::vector<double> pmlb;      // the same factors on the host
  std::vector<double> ktab;      // the same tables on the host, K and E interleaved
  int flux_plane[2];  // node planes of the Poynting split (front, back)
  int flux_blocks;    // blocks per flux plane
  size_t total;
};

int validate_and_plan(const pic_grid *grid, const pic_material *mat, const pic_pulse *pulse,
                      Plan &P) {
  if (!grid || !mat || !pulse) return fail(PIC_EINVAL, "null configuration pointer");
  const pic_grid &g = *grid;
  if (g.nx < 4 || g.ny < 4 || g.nz < 8) return fail(PIC_EINVAL, "grid needs nx, ny >= 4, nz >= 8");
  if (g.nz >= 65535) return fail(PIC_EINVAL, "grid needs nz < 65535 (one launch row per z plane)");
  if (!(g.dx > 0 && g.dy > 0 && g.dz > 0)) return fail(PIC_EINVAL, "cell sizes must be > 0");
  if (!(g.cfl > 0 && g.cfl <= 1.0)) return fail(PIC_EINVAL, "cfl must be in (0, 1]");
  if (g.precision != PIC_FP64 && g.precision != PIC_FP32)
    return fail(PIC_EINVAL, "unknown precision");
  if (!(g.pool_factor >= 0)) return fail(PIC_EINVAL, "pool_factor must be >= 0");
  if (g.keldysh_terms < 0 || g.sort_interval < 0 || g.coll_every < 0)
    return fail(PIC_EINVAL, "negative count");
  if (g.elliptic_table != 0 && (g.elliptic_table < 2 || g.elliptic_table > 1000000))
    return fail(PIC_EINVAL, "elliptic_table must be 0 or 2 .. 1000000 points");
  if (g.pml_cells < 0 || 2 * g.pml_cells >= g.nx || 2 * g.pml_cells >= g.ny)
    return fail(PIC_EINVAL, "pml_cells must be >= 0 with 2 pml_cells < nx, ny");
  if (mat->n_layers < 0 || mat->n_layers > PIC_MAX_LAYERS || (mat->n_layers && !mat->layers))
    return fail(PIC_EINVAL, "bad layer count");
  if (!(pulse->lambda > 0 && pulse->fwhm > 0 && pulse->fluence >= 0) ||
      (pulse->pol != 0 && pulse->pol != 1))
    return fail(PIC_EINVAL, "bad pulse");
  P.g = g;
  if (P.g.keldysh_terms == 0) P.g.keldysh_terms = 500;
  if (P.g.sort_interval == 0) P.g.sort_interval = 16;
  P.pulse = *pulse;
  P.layers.assign(mat->layers, mat->layers + mat->n_layers);
  P.rsz = g.precision == PIC_FP64 ? 8 : 4;
  P.nxy = (long long)g.nx * g.ny;
  P.ncell = P.nxy * g.nz;
  P.nfield = P.nxy * (g.nz + 1);
  if (P.ncell >= (1ll << 31)) return fail(PIC_EINVAL, "grid has >= 2^31 cells");
  P.dt = g.cfl / (kC * std::sqrt(1.0 / (g.dx * g.dx) + 1.0 / (g.dy * g.dy) + 1.0 / (g.dz * g.dz)));
  P.omega = 2.0 * kPi * kC / pulse->lambda;
  P.V = g.dx * g.dy * g.dz;
  P.NW = (int)std::ceil(pulse->lambda / (kC * P.dt));
  // the paper records the intensity map every 0.5 fs (Sec. 5)
  P.imax_every = g.imax_every > 0
                     ? g.imax_every
                     : (g.imax_every == 0 ? (int)std::max(1.0, std::round(0.5e-15 / P.dt)) : 0);
  if (pulse->shape != 0 && pulse->shape != 1) return fail(PIC_EINVAL, "unknown pulse shape");
  if (!(pulse->w0 >= 0.0)) return fail(PIC_EINVAL, "spot radius must be >= 0");
  // cos^4 falls to one half at pi t / T = acos(2^(-1/4)); int cos^4 = 3 T / 8
  P.Tsin2 = pulse->fwhm / (2.0 * std::acos(std::pow(2.0, -0.25)) / kPi);
  if (pulse->shape == 1)
    P.E0 = std::sqrt(16.0 * pulse->fluence / (3.0 * kC * kEps0 * P.Tsin2));
  else
    P.E0 = std::sqrt(2.0 * pulse->fluence /
                   (kC * kEps0 * pulse->fwhm * std::sqrt(kPi / (4.0 * std::log(2.0)))));
  P.lop.assign(g.nz, -1);
  P.n_neutrals = 0;
  for (int L = 0; L < mat->n_layers; ++L) {
    const pic_layer &ly = mat->layers[L];
    if (ly.z0 < 2 || ly.z1 > g.nz - 2 || ly.z0 >= ly.z1)
      return fail(PIC_EINVAL, "layer " + std::to_string(L) + " must satisfy 2 <= z0 < z1 <= nz-2");
    if (ly.ppc < 1 || ly.ppc > 32) return fail(PIC_EINVAL, "ppc must be in 1..32");
    if (!(ly.n_index >= 1 && ly.gap_eV > 0 && ly.me_star > 0 && ly.mh_star > 0 && ly.n_mol > 0 &&
          ly.omega0_eV > 0 && ly.damping >= 0 && ly.temp_eV >= 0 && ly.mol_mass_amu > 0 &&
          ly.e_melt >= 0 && ly.e_boil >= 0 && ly.e_dissoc >= 0))
      return fail(PIC_EINVAL, "layer " + std::to_string(L) + " has a non-physical parameter");
    if (std::isfinite(ly.omega0_eV) && ly.omega0_eV * kQe / kHbar <= P.omega)
      return fail(PIC_EINVAL, "Lorentz pole must lie above the laser frequency");
    for (int k = ly.z0; k < ly.z1; ++k) {
      if (P.lop[k] >= 0) return fail(PIC_EINVAL, "layers overlap");
      P.lop[k] = L;
    }
    P.n_neutrals += (long long)(ly.z1 - ly.z0) * P.nxy * ly.ppc;
  }
  P.mplane.assign(g.nz, -1);
  P.kplane.clear();
  for (int k = 0; k < g.nz; ++k)
    if (P.lop[k] >= 0) {
      P.mplane[k] = (int)P.kplane.size();
      P.kplane.push_back(k);
    }
  P.n_mplanes = (int)P.kplane.size();
  // interior node planes without material: the E step's vacuum launch
  P.vplane.clear();
  for (int k = 1; k < g.nz; ++k)
    if (P.lop[k] < 0) P.vplane.push_back(k);
  // Poynting planes: halfway between the entrance face and the first
  // material plane, and between the last one and the far face (a quarter
  // and three quarters of the box without material), within 1 .. nz - 1
  {
    const int nz = g.nz;
    const int f = P.kplane.empty() ? nz / 4 : P.kplane.front() / 2;
    const int b = P.kplane.empty() ? (3 * nz) / 4 : (P.kplane.back() + 1 + nz) / 2;
    P.flux_plane[0] = std::min(std::max(f, 1), nz - 1);
    P.flux_plane[1] = std::min(std::max(b, 1), nz - 1);
  }
  P.nmat = (long long)P.n_mplanes * P.nxy;
  P.cap = (long long)std::ceil(g.pool_factor * (double)P.n_neutrals) + 1024;
  if (P.cap >= (1ll << 31)) return fail(PIC_EINVAL, "particle pool of >= 2^31 slots");
  P.nb_scan = (int)((P.ncell + kScanChunk - 1) / kScanChunk);
  P.diag_blocks_p = 152 * 8;
  P.diag_blocks_g = (int)((P.nfield + kThreads - 1) / kThreads);
  // arena layout
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + std::max<size_t>(bytes, 1));
    return at;
  };
  const size_t R = P.rsz;
  for (int d = 0; d < 3; ++d) P.off_E[d] = take(P.nfield * R);
  for (int d = 0; d < 3; ++d) P.off_B[d] = take(P.nfield * R);
  for (int d = 0; d < 3; ++d) P.off_Bh[d] = take(P.nfield * R);
  P.off_J4 = take(P.nfield * 4 * R);
  for (int d = 0; d < 3; ++d) P.off_P[d] = take(P.nmat * R);
  for (int d = 0; d < 3; ++d) P.off_Q[d] = take(P.nmat * R);

  P.off_lop = take(g.nz * sizeof(int));
  P.off_mplane = take(g.nz * sizeof(int));
  P.off_kplane = take(std::max(1, P.n_mplanes) * sizeof(int));
  P.off_vplane = take(std::max<size_t>(1, P.vplane.size()) * sizeof(int));
  P.off_lk = take(std::max(1, mat->n_layers) * sizeof(LayerK));
  P.off_lr = take(std::max(1, mat->n_layers) * std::max(sizeof(LayerR<double>), sizeof(LayerR<float>)));
  P.off_win = take((size_t)P.NW * P.nmat * R);
  P.off_pm = take(P.nmat * R);
  P.off_eamp = take(P.nmat * R);
  P.off_ckey = take(P.nmat * R);
  P.off_T = take(P.nmat * 8);
  P.off_alive = take(P.nmat * 4);
  P.off_leave = take(P.nmat * 4);
  for (int b = 0; b < 2; ++b) {
    P.off_pc[b] = take(P.cap * 4);
    for (int d = 0; d < 3; ++d) P.off_po[b][d] = take(P.cap * R);
    for (int d = 0; d < 3; ++d) P.off_pu[b][d] = take(P.cap * R);
    P.off_pt[b] = take(P.cap * 4);
    P.off_pid[b] = take(P.cap * 8);
  }
  P.ppc_max = 1;
  for (const pic_layer &ly : P.layers) P.ppc_max = std::max(P.ppc_max, ly.ppc);
  P.off_leave16 = take(std::max<long long>(P.nmat, 1) * P.ppc_max * 2);
  P.off_work = take(std::max<long long>(P.nmat, 1) * 4);
  P.off_imax = take(P.ncell * R);
  // collisions: per-cell parameters indexed by cell; listed cells hold >= 2
  // particles, so there are at most cap / 2 like items or unlike columns
  const bool coll = g.coll_every > 0;
  P.off_clist = take(coll ? P.ncell * 2 * 4 : 4);
  P.off_cn = take(32);
  P.off_hot = take((size_t)(P.n_mplanes + 1) * sizeof(uint32_t));
  P.off_jtouch = take((size_t)(g.nz + 2) * sizeof(uint32_t));
  P.off_cpar = take((size_t)(coll ? P.ncell : 1) *
                    std::max(sizeof(CollParam<double>), sizeof(CollParam<float>)));
  P.off_cord = take(coll ? P.cap * 4 : 4);
  P.off_clike = take((size_t)(coll ? P.cap / 2 + 1 : 1) * 8);
  P.off_cunl = take((size_t)(coll ? P.cap / 2 + 1 : 1) * 8);
  P.off_prof = take((size_t)(2 * (g.nz + 1) + g.nz) * 8);
  P.off_work_n = take(16);
  P.off_cnt = take(P.ncell * 4);
  P.off_bsum = take((size_t)P.nb_scan * 4);
  P.off_total = take(8);
  P.off_nslots = take(8);
  P.off_step = take(8);
  P.off_acc = take(16 * 8);
  P.flux_blocks = (int)std::min<long long>(std::max<long long>((P.nxy + kThreads - 1) / kThreads, 1),
                                            kFluxMaxBlocks);
  P.off_flux_part = take(2 * kFluxMaxBlocks * 2 * 8);
  P.off_ktab = take((size_t)2 * std::max(g.elliptic_table, 1) * R);
  P.ktab.clear();
  for (int i = 0; i < g.elliptic_table; ++i) {
    const double m = (double)i / (double)g.elliptic_table;
    double K, KmE;
    ellip_k_kme<double>(m, 1.0 - m, K, KmE);
    P.ktab.push_back(K);
    P.ktab.push_back(K - KmE);
  }
  // absorbing layers: eight convolution terms over the field points and the
  // decay factors b = exp(-sigma h / eps0) of each position, E (integer
  // positions, h = dt) then B (half-integer ones, h = dt / 2), x then y
  const bool pml = g.pml_cells > 0;
  for (int q = 0; q < 12; ++q) P.off_psi[q] = take(pml ? P.nfield * R : 1);
  P.off_pmlb = take((size_t)2 * (g.nx + g.ny) * R);
  P.pmlb.clear();
  if (pml) {
    const int L = g.pml_cells;
    const int n[2] = {g.nx, g.ny};
    const double cell[2] = {g.dx, g.dy};
    for (int half = 0; half < 2; ++half)
      for (int ax = 0; ax < 2; ++ax)
        for (int i = 0; i < n[ax]; ++i) {
          const double p = i + 0.5 * half, h = half ? 0.5 * P.dt : P.dt;
          const double d = p < L ? L - p : (p > n[ax] - L ? p - (n[ax] - L) : 0.0);
          const double smax = 0.8 * 4.0 / (kMu0 * kC * cell[ax]), r = d / L;
          P.pmlb.push_back(d > 0.0 ? std::exp(-smax * r * r * r * h / kEps0) : 1.0);
        }
  }
  P.off_err = take(16);
  P.off_ne = take(P.nfield * 8);
  P.off_ed = take(P.nfield * 8);
  P.off_rho = take(P.nfield * 8);
  P.off_spec = take(kSpecMax * 8);
  P.off_part = take((size_t)std::max(3 * P.diag_blocks_p, 5 * P.diag_blocks_g) * 8);
  P.total = o;
  return PIC_OK;
}

// Per-layer constants (double) and the amplitude below which the Keldysh
// threshold is zero: the largest E of a 1% geometric grid up to which every
// grid value has p 2^64 < 1/16 (W grows like E^(2N) there, N >= 3, so the
// values between grid points stay below 1).
std::vector<LayerK> layer_constants(const Plan &P) {
  std::vector<LayerK> out;
  for (const pic_layer &ly : P.layers) {
    LayerK k{};
    const bool st = !std::isfinite(ly.omega0_eV);
    const double n2m1 = ly.n_index * ly.n_index - 1.0;
    k.is_static = st;
    if (st) {
      k.deps = n2m1;
      k.w0sq = 0.0;
    } else {
      const double w0 = ly.omega0_eV * kQe / kHbar;
      k.deps = n2m1 * (1.0 - P.omega * P.omega / (w0 * w0));
      k.w0sq = w0 * w0;
    }
    k.damping = ly.damping;
    k.ppc = ly.ppc;
    k.wmac = ly.n_mol * P.V / ly.ppc;
    k.mass[0] = ly.me_star * kMe;
    k.mass[1] = ly.mh_star * kMe;
    k.qm[0] = -kQe / k.mass[0];
    k.qm[1] = kQe / k.mass[1];
    const double mstar = kMe / (1.0 / ly.me_star + 1.0 / ly.mh_star);
    k.gapJ = ly.gap_eV * kQe;
    k.kG = P.omega * std::sqrt(mstar * k.gapJ) / kQe;
    k.kX = (2.0 / kPi) * k.gapJ / (kHbar * P.omega);
    k.kP = 2.0 * (2.0 * P.omega / (9.0 * kPi)) * std::pow(mstar * P.omega / kHbar, 1.5) * P.dt /
           ly.n_mol;
    k.sigv = std::sqrt(ly.temp_eV * kQe / (ly.mol_mass_amu * kAmu));
    double e = 1e3, last_ok = 0.0;
    k.e_skip = 0.0;
    for (int it = 0; it < 4000; ++it, e *= 1.01) {
      const double p = keldysh_probability<double>(e, k, P.g.keldysh_terms, nullptr,
                                                   P.ktab.empty() ? nullptr : P.ktab.data(),
                                                   P.g.elliptic_table);
      if (p * 18446744073709551616.0 >= 1.0 / 16.0) break;
      last_ok = e;
    }
    k.e_skip = last_ok;
    out.push_back(k);
  }
  return out;
}

template <class R>
std::vector<LayerR<R>> layer_working(const Plan &P, const std::vector<LayerK> &lk) {
  std::vector<LayerR<R>> out;
  const double h = P.dt;
  const double dl[3] = {P.g.dx, P.g.dy, P.g.dz};
  for (const LayerK &k : lk) {
    LayerR<R> r{};
    r.deps = R(k.deps);
    r.is_static = k.is_static;
    r.ppc = k.ppc;
    if (k.is_static) {
      r.inv_den = R(1.0 / (1.0 + k.deps));
    } else {
      r.cn_g = R(h);
      r.cn_a = R(0.5 * h * h * k.w0sq);
      r.cn_b = R(0.25 * h * h * k.w0sq * k.deps);
      r.inv_den = R(1.0 / (1.0 + 0.25 * h * h * k.w0sq * (1.0 + k.deps) + 0.5 * k.damping * h));
      r.two_over_h = R(2.0 / h);
    }
    for (int s = 0; s < 2; ++s) {
      const double q = s ? kQe : -kQe;
      r.qmdt2[s] = R(0.5 * k.qm[s] * h);
      for (int d = 0; d < 3; ++d) r.jpref[s][d] = R(-q * k.wmac * dl[d] / (P.V * h));
      r.inv_mass_c2[s] = R(1.0 / (k.mass[s] * kC * kC));
    }
    r.kG = R(k.kG);
    r.kX = R(k.kX);
    r.kP = R(k.kP);
    r.e_skip = R(k.e_skip);
    r.sig_v = R(k.sigv);
    r.mhat[0] = R(k.mass[0] / kMe);
    r.mhat[1] = R(k.mass[1] / kMe);
    r.wmac = R(k.wmac);
    out.push_back(r);
  }
  return out;
}

}  // namespace

// Lets the allocation-free entry point (its own translation unit) report
// errors through pic_last_error().
namespace pg_internal {
void set_last_error(const std::string &msg) { g_err = msg; }
}  // namespace pg_internal

struct pic_ctx {
  Plan P;
  std::vector<LayerK> lk;
  cudaStream_t stream = nullptr;
  char *arena = nullptr;
  // side stream of a step: the window, Keldysh and ionisation passes run on
  // it while the B step runs on `stream` (fork after the E step, join before
  // the step end)
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // set while a batch captures this member's steps: the batch's graph runs
  // its members side by side already, and keeps one branch per member
  bool in_batch = false;
  bool own_arena = false;
  uint64_t seed = 0;
  long long step = 0;
  int since_sort = 0;
  Ctx<double> c64{};
  Ctx<float> c32{};
  bool fp64 = true;
  int sticky = PIC_OK;
  long long launches = 0;
  long long h2d_bytes = 0, d2h_bytes = 0;  // host <-> device bytes copied so far
  int push_blocks = 0;                      // resident blocks of k_push on this device
  int coll_blocks = 0;                      // resident blocks of k_collide
  int field_v = 1;  // x points per thread of the field and window kernels
  // the E step in separate launches for the faces, the interior vacuum
  // planes and the material planes (when the vacuum planes are many)
  bool efull_split = false;
  // Bh = B - (dt/2) curl E holds (B^{n+1/2} from B^n, E^n): set by each
  // field pass, cleared when the host writes E or B
  bool bh_valid = false;
  // profiling: (class, start, stop) event triples, reused across reads
  bool profiling = false;
  struct Rec {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  size_t used = 0;
  int open_cls = -1;
  // NVTX range per kernel class, for timeline tools (ids, not the thread's
  // push/pop stack, so a range an error path leaves open unbalances nothing)
  nvtxRangeId_t nvtx[4] = {};
  int nvtx_n = 0;
};

namespace {

template <class R>
Ctx<R> &ctx_of(pic_ctx *h);
template <>
Ctx<double> &ctx_of<double>(pic_ctx *h) { return h->c64; }
template <>
Ctx<float> &ctx_of<float>(pic_ctx *h) { return h->c32; }

template <class R>
void bind(pic_ctx *h) {
  const Plan &P = h->P;
  char *A = h->arena;
  Ctx<R> &X = ctx_of<R>(h);
  Dev<R> &D = X.d;
  D.nx = P.g.nx;
  D.ny = P.g.ny;
  D.nz = P.g.nz;
  D.nxy = (int)P.nxy;
  D.nfield = P.nfield;
  D.nmat = P.nmat;
  D.ncell = P.ncell;
  D.NW = P.NW;
  D.keldysh_terms = P.g.keldysh_terms;
  D.n_layers = (int)P.layers.size();
  D.pol = P.pulse.pol;
  D.dt = R(P.dt);
  D.idx = R(1.0 / P.g.dx);
  D.idy = R(1.0 / P.g.dy);
  D.idz = R(1.0 / P.g.dz);
  D.alpha = R(kC * P.dt / P.g.dz);
  D.c2dt = R(kC * kC * P.dt);
  D.dtdx = R(P.dt / P.g.dx);
  D.dtdy = R(P.dt / P.g.dy);
  D.dtdz = R(P.dt / P.g.dz);
  D.dt_d = P.dt;
  D.V_d = P.V;
  D.dx_d = P.g.dx;
  D.dy_d = P.g.dy;
  D.dz_d = P.g.dz;
  D.E0 = P.E0;
  D.omega = P.omega;
  D.fwhm = P.pulse.fwhm;
  D.t_peak = P.pulse.t_peak;
  D.shape = P.pulse.shape;
  D.Tsin2 = P.Tsin2;
  D.w0 = P.pulse.w0;
  D.xc = 0.5 * P.g.nx * P.g.dx;
  D.yc = 0.5 * P.g.ny * P.g.dy;
  D.cep = P.pulse.cep;
  for (int d = 0; d < 3; ++d) {
    D.E[d] = (R *)(A + P.off_E[d]);
    D.B[d] = (R *)(A + P.off_B[d]);
    D.Bh[d] = (R *)(A + P.off_Bh[d]);
    D.P[d] = (R *)(A + P.off_P[d]);
    D.Q[d] = (R *)(A + P.off_Q[d]);
  }
  D.J4 = (R *)(A + P.off_J4);
  D.layer_of_plane = (const int *)(A + P.off_lop);
  D.hot = (uint32_t *)(A + P.off_hot);
  D.jtouch = (uint32_t *)(A + P.off_jtouch);
  D.mplane = (const int *)(A + P.off_mplane);
  D.kplane = (const int *)(A + P.off_kplane);
  D.vplane = (const int *)(A + P.off_vplane);
  D.layers = (const LayerK *)(A + P.off_lk);
  D.win = (R *)(A + P.off_win);
  D.pm = (R *)(A + P.off_pm);
  D.eamp = (R *)(A + P.off_eamp);
  D.ckey = (R *)(A + P.off_ckey);
  D.T = (unsigned long long *)(A + P.off_T);
  D.alive = (uint32_t *)(A + P.off_alive);
  D.leave_step = (uint32_t *)(A + P.off_leave);
  D.pcell = (int32_t *)(A + P.off_pc[0]);
  for (int d = 0; d < 3; ++d) {
    D.po[d] = (R *)(A + P.off_po[0][d]);
    D.pu[d] = (R *)(A + P.off_pu[0][d]);
    X.ao[d] = (R *)(A + P.off_po[1][d]);
    X.au[d] = (R *)(A + P.off_pu[1][d]);
  }
  D.ptag = (uint32_t *)(A + P.off_pt[0]);
  D.pid = (unsigned long long *)(A + P.off_pid[0]);
  X.acell = (int32_t *)(A + P.off_pc[1]);
  X.atag = (uint32_t *)(A + P.off_pt[1]);
  X.aid = (unsigned long long *)(A + P.off_pid[1]);
  D.cap = (unsigned long long)P.cap;
  D.nslots = (unsigned long long *)(A + P.off_nslots);
  D.step = (long long *)(A + P.off_step);
  D.imax = (R *)(A + P.off_imax);
  D.imax_every = P.imax_every;
  D.inv_e0sq = R(P.E0 > 0.0 ? 1.0 / (P.E0 * P.E0) : 1.0);
  D.acc = (double *)(A + P.off_acc);
  D.ktab = P.ktab.empty() ? nullptr : (const R *)(A + P.off_ktab);
  D.ntab = P.g.elliptic_table;
  D.pml = P.g.pml_cells;
  for (int q = 0; q < 8; ++q) D.psi[q] = D.pml ? (R *)(A + P.off_psi[q]) : nullptr;
  for (int q = 0; q < 4; ++q) D.psi_close[q] = D.pml ? (R *)(A + P.off_psi[8 + q]) : nullptr;
  {
    const R *b = (const R *)(A + P.off_pmlb);
    D.pml_bE[0] = b;
    D.pml_bE[1] = b + P.g.nx;
    D.pml_bB[0] = b + P.g.nx + P.g.ny;
    D.pml_bB[1] = b + 2 * P.g.nx + P.g.ny;
  }
  D.flux_k[0] = P.flux_plane[0];
  D.flux_k[1] = P.flux_plane[1];
  D.flux_scale = kC * kEps0 * P.g.dx * P.g.dy * P.dt;
  D.flux_part = (double *)(A + P.off_flux_part);
  D.err = (int *)(A + P.off_err);
  D.seed = h->seed;
  X.lr = (const LayerR<R> *)(A + P.off_lr);
  X.work = (int *)(A + P.off_work);
  X.work_n = (int *)(A + P.off_work_n);
  X.leave16 = (uint16_t *)(A + P.off_leave16);
  X.ppc_max = P.ppc_max;
}

int grid_blocks(long long n) { return (int)std::max<long long>(1, (n + kThreads - 1) / kThreads); }
constexpr int kPersistentBlocks = 152 * 8;

const char *const kProfNames[PIC_PROF_N] = {"pic push",   "pic fields", "pic keldysh",
                                             "pic window", "pic ionize", "pic sort",
                                             "pic other",  "pic collide"};

// Event pair around a group of launches of one class (no-op unless
// profiling), inside an NVTX range named for the class.
void prof_begin(pic_ctx *h, int cls) {
  if (h->nvtx_n < 4) h->nvtx[h->nvtx_n++] = nvtxRangeStartA(kProfNames[cls]);
  if (!h->profiling) return;
  if (h->used == h->recs.size()) {
    pic_ctx::Rec r{cls, nullptr, nullptr};
    cudaEventCreate(&r.a);
    cudaEventCreate(&r.b);
    h->recs.push_back(r);
  }
  h->recs[h->used].cls = cls;
  cudaEventRecord(h->recs[h->used].a, h->stream);
  h->open_cls = cls;
}

void prof_end(pic_ctx *h) {
  if (h->nvtx_n > 0) nvtxRangeEnd(h->nvtx[--h->nvtx_n]);
  if (!h->profiling || h->open_cls < 0) return;
  cudaEventRecord(h->recs[h->used].b, h->stream);
  h->used++;
  h->open_cls = -1;
}

// Counting sort of the pool: by cell (by_frame false: the collision pass
// needs each cell's particles in one range, with cnt holding the cell ends)
// or by deposit-frame base node (the periodic sort, for the push).
template <class R>
int sort_pool(pic_ctx *h, bool by_frame) {
  Ctx<R> &X = ctx_of<R>(h);
  const Plan &P = h->P;
  cudaStream_t s = h->stream;
  unsigned int *cnt = (unsigned int *)(h->arena + P.off_cnt);
  unsigned int *bsum = (unsigned int *)(h->arena + P.off_bsum);
  unsigned long long *total = (unsigned long long *)(h->arena + P.off_total);
  prof_begin(h, PIC_PROF_SORT);
  PIC_CUDA(cudaMemsetAsync(cnt, 0, P.ncell * 4, s));
  if (by_frame)
    k_hist<true, R><<<kPersistentBlocks, kThreads, 0, s>>>(X.d, cnt);
  else
    k_hist<false, R><<<kPersistentBlocks, kThreads, 0, s>>>(X.d, cnt);
  k_scan_reduce<<<P.nb_scan, kScanThreads, 0, s>>>(cnt, P.ncell, bsum);
  k_scan_blocks<<<1, kScanThreads, 0, s>>>(bsum, P.nb_scan, total);
  k_scan_final<<<P.nb_scan, kScanThreads, 0, s>>>(cnt, P.ncell, bsum);
  if (by_frame)
    k_scatter<true, R><<<kPersistentBlocks, kThreads, 0, s>>>(X, cnt);
  else
    k_scatter<false, R><<<kPersistentBlocks, kThreads, 0, s>>>(X, cnt);
  k_set_slots<<<1, 1, 0, s>>>(X.d.nslots, total);
  prof_end(h);
  h->launches += 6;
  std::swap(X.d.pcell, X.acell);
  for (int d = 0; d < 3; ++d) {
    std::swap(X.d.po[d], X.ao[d]);
    std::swap(X.d.pu[d], X.au[d]);
  }
  std::swap(X.d.ptag, X.atag);
  std::swap(X.d.pid, X.aid);
  PIC_CUDA(cudaGetLastError());
  return PIC_OK;
}

// Calls f(std::true_type) for grids with absorbing transverse layers (the
// field kernels instantiated with their terms), else f(std::false_type).
template <class F>
void with_layers(bool on, F &&f) {
  if (on) f(std::true_type{});
  else f(std::false_type{});
}

// Bh = B - (dt/2) curl E from the current fields, unless the last field
// pass left it valid (nothing but the host writes E or B between passes).
template <class R>
int prime_bh(pic_ctx *h) {
  if (h->bh_valid) return PIC_OK;
  const Plan &P = h->P;
  Ctx<R> &X = ctx_of<R>(h);
  cudaStream_t s = h->stream;
  with_layers(P.g.pml_cells > 0, [&](auto lay) {
    constexpr bool kLay = decltype(lay)::value;
    if constexpr (sizeof(R) == 4) {
      if (h->field_v == 4) {
        const dim3 grid(grid_blocks(P.nxy / 4), (unsigned)(P.g.nz + 1));
        k_bstep<4, kPrime, R, kLay><<<grid, kThreads, 0, s>>>(X.d);
      }
    }
    if (h->field_v == 1) {
      const dim3 grid(grid_blocks(P.nxy), (unsigned)(P.g.nz + 1));
      k_bstep<1, kPrime, R, kLay><<<grid, kThreads, 0, s>>>(X.d);
    }
  });
  PIC_CUDA(cudaGetLastError());
  h->launches += 1;
  h->bh_valid = true;
  return PIC_OK;
}

template <class R>
int enqueue(pic_ctx *h, int mask) {
  Ctx<R> &X = ctx_of<R>(h);
  const Plan &P = h->P;
  cudaStream_t s = h->stream;
  // A whole step (fields, window and ionisation) overlaps the B step with
  // the material passes, which read E^{n+1} only; with profiling on, every
  // class runs in order on the simulation's stream so that each is timed.
  constexpr int kOverlapMask = PIC_PHASE_FIELDS | PIC_PHASE_WINDOW | PIC_PHASE_IONIZE;
  const bool overlap =
      !h->profiling && !h->in_batch && P.nmat > 0 && (mask & kOverlapMask) == kOverlapMask;
  // window and Keldysh threshold, then ionisation, on stream st
  auto material_passes = [&](cudaStream_t st, bool window, bool ionize) -> int {
    if (window && P.nmat > 0) {
      prof_begin(h, PIC_PROF_WINDOW);
      PIC_CUDA(cudaMemsetAsync(X.work_n, 0, sizeof(int), st));
      if constexpr (sizeof(R) == 4) {
        if (h->field_v == 4)
          k_window<4, R><<<dim3(grid_blocks(P.nxy / 4), P.n_mplanes), kThreads, 0, st>>>(X);
      }
      if (h->field_v == 1)
        k_window<1, R><<<dim3(grid_blocks(P.nxy), P.n_mplanes), kThreads, 0, st>>>(X);
      prof_end(h);
      prof_begin(h, PIC_PROF_KELDYSH);
      k_keldysh<R><<<kPersistentBlocks, kThreads, 0, st>>>(X);
      prof_end(h);
      h->launches += 2;
    }
    if (ionize && P.nmat > 0) {
      prof_begin(h, PIC_PROF_IONIZE);
      k_ionize<R><<<dim3(grid_blocks((P.nxy + kIonizeCells - 1) / kIonizeCells), P.n_mplanes),
                    kThreads, 0, st>>>(X);
      prof_end(h);
      h->launches += 1;
    }
    return PIC_OK;
  };
  if (mask & PIC_PHASE_PARTICLES) {
    prof_begin(h, PIC_PROF_PUSH);
    k_push<R><<<h->push_blocks, kThreads, 0, s>>>(X);
    prof_end(h);
    h->launches += 1;
  }
  if ((mask & PIC_PHASE_COLLIDE) && P.g.coll_every > 0 && (h->step + 1) % P.g.coll_every == 0) {
    // pairs are formed per cell: the pool is sorted first (cell ends in cnt)
    const int rc = sort_pool<R>(h, false);
    if (rc) return rc;
    prof_begin(h, PIC_PROF_COLLIDE);
    CollConst K;
    K.K1 = kQe * kQe * kQe * kQe / (4.0 * kPi * kEps0 * kEps0 * kC * kC * kC * kMe * kMe);
    K.re = kQe * kQe / (4.0 * kPi * kEps0 * kMe * kC * kC);
    K.lc = 2.0 * kPi * kHbar / (kMe * kC);
    K.kD = 4.0 * kPi * K.re;
    K.capc = std::cbrt(4.0 * kPi / 3.0) * kC;
    const unsigned int *cend = (const unsigned int *)(h->arena + P.off_cnt);
    CollWork<R> W;
    int *clist = (int *)(h->arena + P.off_clist);
    W.list = clist;
    W.n = (int *)(h->arena + P.off_cn);
    W.ncell = P.ncell;
    W.par = (CollParam<R> *)(h->arena + P.off_cpar);
    W.ord = (int *)(h->arena + P.off_cord);
    W.like = (unsigned long long *)(h->arena + P.off_clike);
    W.unl = (unsigned long long *)(h->arena + P.off_cunl);
    W.lcap = (int)(P.cap / 2 + 1);
    PIC_CUDA(cudaMemsetAsync(W.n, 0, 8 * sizeof(int), s));
    k_coll_cells<<<grid_blocks((P.ncell + kCellsPerThread - 1) / kCellsPerThread), kThreads, 0, s>>>(
        cend, P.ncell, clist, W.n);
    const double dtc = P.dt * P.g.coll_every;
    // twice the resident warps of one pass: the thread-per-cell preparation
    // waits on its scattered particle loads
    k_coll_prep_small<R><<<kPersistentBlocks * 2, 128, 0, s>>>(X, cend, W, dtc);
    k_coll_prep<R><<<h->coll_blocks, 32 * kCollWarps, 0, s>>>(X, cend, W, dtc);
    k_coll_like<R><<<kPersistentBlocks, kThreads, 0, s>>>(X, W, K);
    k_coll_unlike<R><<<kPersistentBlocks, kThreads, 0, s>>>(X, W, K);
    prof_end(h);
    h->launches += 5;
  }
  if (mask & PIC_PHASE_FIELDS) {
    prof_begin(h, PIC_PROF_FIELDS);
    const int rp = prime_bh<R>(h);
    if (rp) return rp;
    with_layers(P.g.pml_cells > 0, [&](auto lay) {
      constexpr bool kLay = decltype(lay)::value;
      // the E step: one launch over every plane, or, when the interior
      // planes without material are many, three launches each compiled for
      // its planes only: the two faces (boundary, laser source), the vacuum
      // planes (a lean kernel, four blocks per SM), the material planes
      const unsigned nv = (unsigned)P.vplane.size(), nm = (unsigned)P.n_mplanes;
      const bool split = h->efull_split;
      auto estep = [&](auto vt) {
        constexpr int V = decltype(vt)::value;
        const unsigned gx = grid_blocks(P.nxy / V);
        if (!split) {
          k_efull<V, R, kLay, 0><<<dim3(gx, P.g.nz + 1), kThreads, 0, s>>>(X);
          return;
        }
        k_efull<V, R, kLay, 3><<<dim3(gx, 2), kThreads, 0, s>>>(X);
        if (nv) k_efull<V, R, kLay, 1><<<dim3(gx, nv), kThreads, 0, s>>>(X);
        if (nm) k_efull<V, R, kLay, 2><<<dim3(gx, nm), kThreads, 0, s>>>(X);
      };
      if constexpr (sizeof(R) == 4) {
        if (h->field_v == 4) estep(std::integral_constant<int, 4>{});
      }
      if (h->field_v == 1) estep(std::integral_constant<int, 1>{});
    });
    if (overlap) {
      // fork: the window, Keldysh and ionisation passes need E^{n+1} only
      PIC_CUDA(cudaEventRecord(h->ev_fork, s));
      PIC_CUDA(cudaStreamWaitEvent(h->aux, h->ev_fork, 0));
      const int rw = material_passes(h->aux, true, true);
      if (rw) return rw;
      PIC_CUDA(cudaEventRecord(h->ev_join, h->aux));
    }
    with_layers(P.g.pml_cells > 0, [&](auto lay) {
      constexpr bool kLay = decltype(lay)::value;
      if constexpr (sizeof(R) == 4) {
        if (h->field_v == 4)
          k_bstep<4, kFullRecord, R, kLay>
              <<<dim3(grid_blocks(P.nxy / 4), P.g.nz + 1), kThreads, 0, s>>>(X.d);
      }
      if (h->field_v == 1)
        k_bstep<1, kFullRecord, R, kLay><<<dim3(grid_blocks(P.nxy), P.g.nz + 1), kThreads, 0, s>>>(
            X.d);
    });
    if (overlap) PIC_CUDA(cudaStreamWaitEvent(s, h->ev_join, 0));  // join
    prof_end(h);
    // E step (one launch, or faces + vacuum + material) and the B step
    h->launches += h->efull_split ? 2 + (P.vplane.empty() ? 0 : 1) + (P.n_mplanes ? 1 : 0) : 2;
    h->bh_valid = true;
  }
  if (!overlap) {
    const int rw = material_passes(s, (mask & PIC_PHASE_WINDOW) != 0,
                                   (mask & PIC_PHASE_IONIZE) != 0);
    if (rw) return rw;
  }
  if (mask & PIC_PHASE_ADVANCE) {
    prof_begin(h, PIC_PROF_OTHER);
    k_flux_advance<R><<<dim3(P.flux_blocks, 2), kThreads, 0, s>>>(X.d);
    prof_end(h);
    h->launches += 1;
    h->step++;
    if (++h->since_sort >= P.g.sort_interval) {
      h->since_sort = 0;
      const int rc = sort_pool<R>(h, true);
      if (rc) return rc;
    }
  }
  PIC_CUDA(cudaGetLastError());
  return PIC_OK;
}

int enqueue_any(pic_ctx *h, int mask) { return h->fp64 ? enqueue<double>(h, mask) : enqueue<float>(h, mask); }

template <class R>
int init_state(pic_ctx *h) {
  const Plan &P = h->P;
  cudaStream_t s = h->stream;
  PIC_CUDA(cudaMemsetAsync(h->arena, 0, P.total, s));
  // the push is persistent: exactly as many blocks as are resident at once
  int dev = 0, nsm = 0, per_sm = 0;
  PIC_CUDA(cudaGetDevice(&dev));
  PIC_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  PIC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_push<R>, kThreads, 0));
  h->push_blocks = std::max(1, nsm) * std::max(1, per_sm);
  PIC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coll_prep<R>, 32 * kCollWarps, 0));
  h->coll_blocks = std::max(1, nsm) * std::max(1, per_sm);
  if (!h->aux) {
    // the side stream at the highest priority: its passes are the longer
    // branch of a step, the B step fills the SMs they leave
    int lo = 0, hi = 0;
    PIC_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    PIC_CUDA(cudaStreamCreateWithPriority(&h->aux, cudaStreamNonBlocking, hi));
    PIC_CUDA(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    PIC_CUDA(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
  }
  PIC_CUDA(cudaMemcpyAsync(h->arena + P.off_lop, P.lop.data(), P.lop.size() * sizeof(int),
                           cudaMemcpyHostToDevice, s));
  PIC_CUDA(cudaMemcpyAsync(h->arena + P.off_mplane, P.mplane.data(), P.mplane.size() * sizeof(int),
                           cudaMemcpyHostToDevice, s));
  h->h2d_bytes += (long long)((P.lop.size() + P.mplane.size() + P.kplane.size()) * sizeof(int));
  if (!P.kplane.empty())
    PIC_CUDA(cudaMemcpyAsync(h->arena + P.off_kplane, P.kplane.data(),
                             P.kplane.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  if (!P.vplane.empty())
    PIC_CUDA(cudaMemcpyAsync(h->arena + P.off_vplane, P.vplane.data(),
                             P.vplane.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  h->h2d_bytes += (long long)(P.vplane.size() * sizeof(int));
  if (!h->lk.empty()) {
    PIC_CUDA(cudaMemcpyAsync(h->arena + P.off_lk, h->lk.data(), h->lk.size() * sizeof(LayerK),
                             cudaMemcpyHostToDevice, s));
    std::vector<LayerR<R>> lr = layer_working<R>(P, h->lk);
    PIC_CUDA(cudaMemcpyAsync(h->arena + P.off_lr, lr.data(), lr.size() * sizeof(LayerR<R>),
                             cudaMemcpyHostToDevice, s));
    h->h2d_bytes += (long long)(h->lk.size() * sizeof(LayerK) + lr.size() * sizeof(LayerR<R>));
    PIC_CUDA(cudaStreamSynchronize(s));  // lr is a host temporary
  }
  if (!P.pmlb.empty()) {
    std::vector<R> pb(P.pmlb.begin(), P.pmlb.end());
    PIC_CUDA(cudaMemcpyAsync(h->arena + P.off_pmlb, pb.data(), pb.size() * sizeof(R),
                             cudaMemcpyHostToDevice, h->stream));
    PIC_CUDA(cudaStreamSynchronize(h->stream));
  }
  if (!P.ktab.empty()) {
    std::vector<R> kt(P.ktab.begin(), P.ktab.end());
    PIC_CUDA(cudaMemcpyAsync(h->arena + P.off_ktab, kt.data(), kt.size() * sizeof(R),
                             cudaMemcpyHostToDevice, s));
    h->h2d_bytes += (long long)(kt.size() * sizeof(R));
    PIC_CUDA(cudaStreamSynchronize(s));  // kt is a host temporary
  }
  if (P.nmat > 0) k_init_material<R><<<grid_blocks(P.nmat), kThreads, 0, s>>>(ctx_of<R>(h));
  PIC_CUDA(cudaGetLastError());
  PIC_CUDA(cudaStreamSynchronize(s));
  return PIC_OK;
}

int check_sticky(pic_ctx *h) {
  int e = 0;
  const Plan &P = h->P;
  PIC_CUDA(cudaMemcpyAsync(&e, h->arena + P.off_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  h->d2h_bytes += (long long)sizeof(int);
  PIC_CUDA(cudaStreamSynchronize(h->stream));
  if (e & kErrPool) h->sticky = PIC_EPOOL;
  if (e & kErrColl) h->sticky = PIC_ECOLL;
  if (h->sticky == PIC_EPOOL)
    return fail(PIC_EPOOL, "ionisation outgrew the charged-particle pool (raise pool_factor)");
  if (h->sticky == PIC_ECOLL)
    return fail(PIC_ECOLL, "a cell held more charged particles than a collision pass handles");
  return PIC_OK;
}

template <class R>
void to_double(const std::vector<char> &raw, size_t n, double *dst) {
  const R *src = (const R *)raw.data();
  for (size_t q = 0; q < n; ++q) dst[q] = (double)src[q];
}

template <class R>
void from_double(const double *src, size_t n, std::vector<char> &raw) {
  raw.resize(n * sizeof(R));
  R *d = (R *)raw.data();
  for (size_t q = 0; q < n; ++q) d[q] = (R)src[q];
}

int copy_in(pic_ctx *h, size_t off, const void *src, size_t bytes) {
  PIC_CUDA(cudaMemcpyAsync(h->arena + off, src, bytes, cudaMemcpyHostToDevice, h->stream));
  h->h2d_bytes += (long long)bytes;
  PIC_CUDA(cudaStreamSynchronize(h->stream));
  return PIC_OK;
}

int copy_out(pic_ctx *h, size_t off, void *dst, size_t bytes) {
  PIC_CUDA(cudaMemcpyAsync(dst, h->arena + off, bytes, cudaMemcpyDeviceToHost, h->stream));
  h->d2h_bytes += (long long)bytes;
  PIC_CUDA(cudaStreamSynchronize(h->stream));
  return PIC_OK;
}

// device offset of a pointer inside the arena
size_t off_of(pic_ctx *h, const void *p) { return (size_t)((const char *)p - h->arena); }

}  // namespace

// ---------------------------------------------------------------------------
// Exported entry points
// ---------------------------------------------------------------------------
extern "C" {

const char *pic_last_error(void) { return g_err.c_str(); }

int pic_query(const pic_grid *grid, const pic_material *mat, const pic_pulse *pulse,
              pic_info *out) {
  Plan P;
  const int rc = validate_and_plan(grid, mat, pulse, P);
  if (rc) return rc;
  if (!out) return fail(PIC_EINVAL, "null output");
  std::memset(out, 0, sizeof(*out));
  out->dt = P.dt;
  out->E0 = P.E0;
  out->NW = P.NW;
  out->n_mplanes = P.n_mplanes;
  out->nfield = P.nfield;
  out->nmat = P.nmat;
  out->n_neutrals = P.n_neutrals;
  out->capacity = P.cap;
  out->arena_bytes = P.total;
  return PIC_OK;
}

int pic_create(const pic_grid *grid, const pic_material *mat, const pic_pulse *pulse,
               uint64_t seed, void *stream, void *d_arena, size_t arena_bytes, pic_handle *out) {
  if (!out) return fail(PIC_EINVAL, "null handle pointer");
  *out = nullptr;
  pic_ctx *h = new pic_ctx();
  int rc = validate_and_plan(grid, mat, pulse, h->P);
  if (rc) {
    delete h;
    return rc;
  }
  h->seed = seed;
  h->stream = (cudaStream_t)stream;
  h->fp64 = h->P.g.precision == PIC_FP64;
  h->field_v = (!h->fp64 && h->P.g.nx % 4 == 0) ? 4 : 1;
  // Splitting the E step saves about 1.3 ps per interior vacuum point (the
  // lean kernel streams at four blocks per SM) and costs about 17 us of
  // launches and tails per step (measured on the 256 x 256 x 1024 mirror,
  // 51 M such points, and the 128 x 128 x 512 silica slab, 2.6 M): split
  // from 16 M points.
  h->efull_split = (long long)h->P.vplane.size() * h->P.nxy >= (16ll << 20);
  h->lk = layer_constants(h->P);
  if (d_arena) {
    if (arena_bytes < h->P.total || ((uintptr_t)d_arena % kAlign)) {
      delete h;
      return fail(PIC_ENOMEM, "caller arena smaller than " + std::to_string(h->P.total) +
                                  " bytes or not 256-byte aligned");
    }
    h->arena = (char *)d_arena;
  } else {
    cudaError_t e = cudaMalloc((void **)&h->arena, h->P.total);
    if (e != cudaSuccess) {
      delete h;
      return fail(PIC_ENOMEM, std::string("cudaMalloc of the state failed: ") + cudaGetErrorString(e));
    }
    h->own_arena = true;
  }
  bind<double>(h);
  bind<float>(h);
  rc = h->fp64 ? init_state<double>(h) : init_state<float>(h);
  if (rc) {
    if (h->own_arena) cudaFree(h->arena);
    delete h;
    return rc;
  }
  *out = h;
  return PIC_OK;
}

// ---------------------------------------------------------------------------
// Batches
// ---------------------------------------------------------------------------
}  // extern "C"

struct pic_batch_ctx {
  std::vector<pic_ctx *> m;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int period = 32;
  cudaGraphExec_t exec = nullptr;
  std::vector<long long> step_at_capture_end;  // members' host steps after capture
  std::vector<long long> launches_per_period;  // kernels one replay runs per member
  std::vector<cudaEvent_t> ev;
  // batch launches (one per phase for all members): device tables, and the
  // parity of the members' pool halves relative to the tables' first copy
  bool multi = false;
  bool one_launch = false;  // batch launches allowed (pic_batch_set_launches)
  char *tab = nullptr;
  size_t tab_bytes = 0;
  int parity = 0;
  int push_blocks = 0;   // resident blocks of k_push_batch
  // the push's launch shape, picked by batch_tune: particles per block task
  // and grid (a multiple of the resident blocks)
  long long push_chunk = 2048;
  int push_grid_mult = 1;
  bool tuned = false;
  std::vector<long long> tune_chunk;
  std::vector<int> tune_mult;
  std::vector<double> tune_ms;     // push time over the tuning period
  std::vector<double> tune_cost;   // push time per particle push [ns]
  int tune_pick = -1;
  // while tuning, event pairs around every push of the captured period
  bool time_push = false;
  std::vector<cudaEvent_t> tev;
  // byte offsets in tab
  size_t o_ctx[2] = {0, 0}, o_sort[2] = {0, 0}, o_cnt = 0;
  struct Flat {
    size_t o_start = 0, o_gx = 0;
    int total = 0;
  } g_field, g_window, g_ionize, g_flux, g_scan, g_zero;
};

namespace {
long long gcd_ll(long long a, long long b) { return b ? gcd_ll(b, a % b) : a; }

// Work already queued on a member's own stream (a pic_step outside the batch)
// comes before the batch's next graph: the batch stream waits on every member.
int join_members_into_batch(pic_batch_ctx *b) {
  for (size_t q = 0; q < b->m.size(); ++q) {
    PIC_CUDA(cudaEventRecord(b->ev[1 + q], b->m[q]->stream));
    PIC_CUDA(cudaStreamWaitEvent(b->stream, b->ev[1 + q], 0));
  }
  return PIC_OK;
}

// And a member's later work (its own pic_step, state reads after pic_sync)
// comes after the graph: every member stream waits on the batch stream.
int join_batch_into_members(pic_batch_ctx *b) {
  PIC_CUDA(cudaEventRecord(b->ev[0], b->stream));
  for (size_t q = 0; q < b->m.size(); ++q) PIC_CUDA(cudaStreamWaitEvent(b->m[q]->stream, b->ev[0], 0));
  return PIC_OK;
}

// Batch launches are used when every member has the same precision, the
// same points per thread in the field kernels and the same pool-sort
// schedule, and no member runs collisions.
bool batch_uniform(const pic_batch_ctx *b) {
  if (!b->one_launch || b->m.size() > (size_t)kMaxBatch) return false;
  const pic_ctx *a = b->m[0];
  for (const pic_ctx *h : b->m)
    if (h->fp64 != a->fp64 || h->field_v != a->field_v ||
        h->P.g.sort_interval != a->P.g.sort_interval || h->since_sort != a->since_sort ||
        h->P.g.coll_every > 0)
      return false;
  return true;
}

FlatGrid flat_of(const pic_batch_ctx *b, const pic_batch_ctx::Flat &f) {
  return FlatGrid{(const int *)(b->tab + f.o_start), (const int *)(b->tab + f.o_gx), (int)b->m.size()};
}

// Lay out and upload the device tables of the current members (synchronous,
// outside any capture): the Ctx of every member as it is now and with its
// pool halves swapped, the sort buffers for both, the flat block tables and
// the chunk counters.
template <class R>
int batch_tables(pic_batch_ctx *b) {
  // a replay still running reads the current tables
  PIC_CUDA(cudaStreamSynchronize(b->stream));
  const int n = (int)b->m.size();
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = (o + bytes + 255) / 256 * 256;
    return at;
  };
  b->o_ctx[0] = take(n * sizeof(Ctx<R>));
  b->o_ctx[1] = take(n * sizeof(Ctx<R>));
  b->o_sort[0] = take(n * sizeof(SortBufs));
  b->o_sort[1] = take(n * sizeof(SortBufs));
  b->o_cnt = take(kCntN * sizeof(unsigned int));
  pic_batch_ctx::Flat *fl[6] = {&b->g_field, &b->g_window, &b->g_ionize, &b->g_flux, &b->g_scan,
                                &b->g_zero};
  for (pic_batch_ctx::Flat *f : fl) {
    f->o_start = take((n + 1) * sizeof(int));
    f->o_gx = take(n * sizeof(int));
  }
  if (o > b->tab_bytes) {
    if (b->tab) cudaFree(b->tab);
    b->tab = nullptr;
    b->tab_bytes = 0;
    PIC_CUDA(cudaMalloc((void **)&b->tab, o));
    b->tab_bytes = o;
  }
  std::vector<char> host(o, 0);
  std::vector<Ctx<R>> cx(n), cy(n);
  std::vector<SortBufs> sb(n);
  std::vector<std::vector<int>> gx(6, std::vector<int>(n)), st(6, std::vector<int>(n + 1, 0));
  long long blocks[6] = {0, 0, 0, 0, 0, 0};
  for (int q = 0; q < n; ++q) {
    pic_ctx *h = b->m[q];
    const Plan &P = h->P;
    Ctx<R> X = ctx_of<R>(h);
    cx[q] = X;
    // the same Ctx after a sort: pool halves swapped
    std::swap(X.d.pcell, X.acell);
    for (int d = 0; d < 3; ++d) {
      std::swap(X.d.po[d], X.ao[d]);
      std::swap(X.d.pu[d], X.au[d]);
    }
    std::swap(X.d.ptag, X.atag);
    std::swap(X.d.pid, X.aid);
    cy[q] = X;
    sb[q] = SortBufs{(unsigned int *)(h->arena + P.off_cnt), (unsigned int *)(h->arena + P.off_bsum),
                     (unsigned long long *)(h->arena + P.off_total), P.ncell, P.nb_scan, 0};
    const int V = h->field_v;
    const int gxs[6] = {grid_blocks(P.nxy / V), grid_blocks(P.nxy / V),
                        grid_blocks((P.nxy + kIonizeCells - 1) / kIonizeCells),
                        P.flux_blocks, P.nb_scan, grid_blocks(P.ncell)};
    const long long gys[6] = {P.g.nz + 1, P.n_mplanes, P.n_mplanes, 2, 1, 1};
    for (int k = 0; k < 6; ++k) {
      gx[k][q] = gxs[k];
      st[k][q] = (int)blocks[k];
      blocks[k] += (long long)gxs[k] * gys[k];
      if (blocks[k] >= (1ll << 31)) return fail(PIC_EINVAL, "batch grid above 2^31 blocks");
    }
  }
  for (int k = 0; k < 6; ++k) {
    st[k][n] = (int)blocks[k];
    fl[k]->total = (int)blocks[k];
    std::memcpy(host.data() + fl[k]->o_start, st[k].data(), (n + 1) * sizeof(int));
    std::memcpy(host.data() + fl[k]->o_gx, gx[k].data(), n * sizeof(int));
  }
  std::memcpy(host.data() + b->o_ctx[0], cx.data(), n * sizeof(Ctx<R>));
  std::memcpy(host.data() + b->o_ctx[1], cy.data(), n * sizeof(Ctx<R>));
  std::memcpy(host.data() + b->o_sort[0], sb.data(), n * sizeof(SortBufs));
  std::memcpy(host.data() + b->o_sort[1], sb.data(), n * sizeof(SortBufs));
  PIC_CUDA(cudaMemcpy(b->tab, host.data(), o, cudaMemcpyHostToDevice));
  int dev = 0, nsm = 0, per_sm = 0;
  PIC_CUDA(cudaGetDevice(&dev));
  PIC_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  PIC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_push_batch<R>, kThreads, 0));
  b->push_blocks = std::max(1, nsm) * std::max(1, per_sm);
  b->parity = 0;
  return PIC_OK;
}

// One full step of every member as batch launches on the batch stream; the
// members' host state advances as enqueue would advance it.
template <class R>
int enqueue_batch(pic_batch_ctx *b, int st) {
  cudaStream_t s = b->stream;
  const int n = (int)b->m.size();
  const Ctx<R> *cx = (const Ctx<R> *)(b->tab + b->o_ctx[b->parity]);
  unsigned int *cnt = (unsigned int *)(b->tab + b->o_cnt);
  const int V = b->m[0]->field_v;
  long long launched = 0;
  k_batch_prep<R><<<grid_blocks(std::max(n, (int)kCntN)), kThreads, 0, s>>>(cx, n, cnt);
  // external record nodes: inside a capture a plain record is only an edge
  if (b->time_push) PIC_CUDA(cudaEventRecordWithFlags(b->tev[2 * st], s, cudaEventRecordExternal));
  k_push_batch<R><<<b->push_blocks * b->push_grid_mult, kThreads, 0, s>>>(cx, n, cnt,
                                                                        b->push_chunk);
  if (b->time_push)
    PIC_CUDA(cudaEventRecordWithFlags(b->tev[2 * st + 1], s, cudaEventRecordExternal));
  launched += 2;
  if (b->g_field.total > 0) {
    const FlatGrid G = flat_of(b, b->g_field);
    bool any_layers = false;
    for (const pic_ctx *h : b->m) any_layers |= h->P.g.pml_cells > 0;
    with_layers(any_layers, [&](auto lay) {
      constexpr bool kLay = decltype(lay)::value;
      if constexpr (sizeof(R) == 4) {
        if (V == 4) {
          k_efull_batch<4, R, kLay><<<b->g_field.total, kThreads, 0, s>>>(cx, G);
          k_bstep_batch<4, R, kLay><<<b->g_field.total, kThreads, 0, s>>>(cx, G);
        }
      }
      if (V == 1) {
        k_efull_batch<1, R, kLay><<<b->g_field.total, kThreads, 0, s>>>(cx, G);
        k_bstep_batch<1, R, kLay><<<b->g_field.total, kThreads, 0, s>>>(cx, G);
      }
    });
    launched += 2;
  }
  if (b->g_window.total > 0) {
    const FlatGrid G = flat_of(b, b->g_window);
    if constexpr (sizeof(R) == 4) {
      if (V == 4) k_window_batch<4, R><<<b->g_window.total, kThreads, 0, s>>>(cx, G);
    }
    if (V == 1) k_window_batch<1, R><<<b->g_window.total, kThreads, 0, s>>>(cx, G);
    k_keldysh_batch<R><<<kPersistentBlocks, kThreads, 0, s>>>(cx, n, cnt);
    k_ionize_batch<R><<<b->g_ionize.total, kThreads, 0, s>>>(cx, flat_of(b, b->g_ionize));
    launched += 3;
  }
  k_flux_advance_batch<R><<<b->g_flux.total, kThreads, 0, s>>>(cx, flat_of(b, b->g_flux));
  launched += 1;
  PIC_CUDA(cudaGetLastError());
  bool sort = false;
  for (pic_ctx *h : b->m) {
    h->step++;
    h->bh_valid = true;
    if (++h->since_sort >= h->P.g.sort_interval) {
      h->since_sort = 0;
      sort = true;
    }
  }
  if (sort) {
    const SortBufs *sb = (const SortBufs *)(b->tab + b->o_sort[b->parity]);
    k_zero_cnt_batch<<<b->g_zero.total, kThreads, 0, s>>>(sb, flat_of(b, b->g_zero));
    k_hist_batch<R><<<kPersistentBlocks, kThreads, 0, s>>>(cx, sb, n, cnt);
    k_scan_reduce_batch<<<b->g_scan.total, kScanThreads, 0, s>>>(sb, flat_of(b, b->g_scan));
    k_scan_blocks_batch<<<n, kScanThreads, 0, s>>>(sb);
    k_scan_final_batch<<<b->g_scan.total, kScanThreads, 0, s>>>(sb, flat_of(b, b->g_scan));
    k_scatter_batch<R><<<kPersistentBlocks, kThreads, 0, s>>>(cx, sb, n, cnt);
    k_set_slots_batch<R><<<grid_blocks(n), kThreads, 0, s>>>(cx, sb, n);
    launched += 7;
    PIC_CUDA(cudaGetLastError());
    // every member's pool halves swap, as sort_pool swaps them
    for (pic_ctx *h : b->m) {
      Ctx<R> &X = ctx_of<R>(h);
      std::swap(X.d.pcell, X.acell);
      for (int d = 0; d < 3; ++d) {
        std::swap(X.d.po[d], X.ao[d]);
        std::swap(X.d.pu[d], X.au[d]);
      }
      std::swap(X.d.ptag, X.atag);
      std::swap(X.d.pid, X.aid);
    }
    b->parity ^= 1;
  }
  b->m[0]->launches += launched;  // the batch's launches, counted once
  return PIC_OK;
}

int batch_capture(pic_batch_ctx *b) {
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  cudaStream_t s = b->stream;
  // Bh is made valid outside the graph, so that replays do not recompute it
  for (pic_ctx *h : b->m) {
    const int rp = h->fp64 ? prime_bh<double>(h) : prime_bh<float>(h);
    if (rp) return rp;
  }
  std::vector<long long> l0;
  for (pic_ctx *h : b->m) l0.push_back(h->launches);
  b->multi = batch_uniform(b);
  if (b->multi) {
    const int rt = b->m[0]->fp64 ? batch_tables<double>(b) : batch_tables<float>(b);
    if (rt) return rt;
  }
  if (const int rj = join_members_into_batch(b)) return rj;
  PIC_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  int rc = PIC_OK;
  cudaError_t e = cudaSuccess;
  if (b->multi) {
    // one launch per phase for all members, on the batch stream
    for (int st = 0; st < b->period && rc == PIC_OK; ++st)
      rc = b->m[0]->fp64 ? enqueue_batch<double>(b, st) : enqueue_batch<float>(b, st);
  } else {
    e = cudaEventRecord(b->ev[0], s);
    for (size_t q = 0; q < b->m.size() && e == cudaSuccess; ++q)
      e = cudaStreamWaitEvent(b->m[q]->stream, b->ev[0], 0);
    for (pic_ctx *h : b->m) h->in_batch = true;
    for (int st = 0; st < b->period && rc == PIC_OK && e == cudaSuccess; ++st)
      for (size_t q = 0; q < b->m.size() && rc == PIC_OK; ++q) rc = enqueue_any(b->m[q], PIC_PHASE_ALL);
    for (pic_ctx *h : b->m) h->in_batch = false;
    for (size_t q = 0; q < b->m.size() && e == cudaSuccess; ++q) {
      e = cudaEventRecord(b->ev[1 + q], b->m[q]->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->ev[1 + q], 0);
    }
  }
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(s, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return fail(PIC_ECUDA, std::string("graph capture: ") +
                               cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  const cudaError_t e3 = cudaGraphInstantiate(&b->exec, g, 0);
  cudaGraphDestroy(g);
  if (e3 != cudaSuccess) return fail(PIC_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e3));
  // the capture advanced every member's host state by one period; the first
  // replay makes the device catch up
  b->step_at_capture_end.clear();
  b->launches_per_period.clear();
  for (size_t q = 0; q < b->m.size(); ++q) {
    b->step_at_capture_end.push_back(b->m[q]->step);
    b->launches_per_period.push_back(b->m[q]->launches - l0[q]);
  }
  PIC_CUDA(cudaGraphLaunch(b->exec, s));
  return join_batch_into_members(b);
}
// One replay of the captured period, ordered after the members' own work and
// before their later work; the members' host state advances by the period.
int batch_replay(pic_batch_ctx *b, cudaEvent_t t0 = nullptr, cudaEvent_t t1 = nullptr) {
  if (const int rj = join_members_into_batch(b)) return rj;
  if (t0) PIC_CUDA(cudaEventRecord(t0, b->stream));
  PIC_CUDA(cudaGraphLaunch(b->exec, b->stream));
  if (t1) PIC_CUDA(cudaEventRecord(t1, b->stream));
  if (const int rj = join_batch_into_members(b)) return rj;
  for (size_t q = 0; q < b->m.size(); ++q) {
    b->m[q]->step += b->period;
    b->m[q]->launches += b->launches_per_period[q];
    b->step_at_capture_end[q] = b->m[q]->step;
  }
  return PIC_OK;
}

// The push's launch shape in batch launches, picked on the batch itself:
// each candidate (particles per block task; grid of 1 or 2 times the
// resident blocks) is captured with event pairs around its push launches and
// run for one period; its cost is the push time over the particle pushes of
// that period, so the growth of the particle count while the candidates take
// turns does not favour the earlier ones.  The cheapest is kept.  Every
// tuning period is a real one (the candidates differ only in how the same
// work spreads over the GPU); it takes one period per candidate, when the
// step request has them.
int batch_pushes(pic_batch_ctx *b, double *out) {
  double sum = 0.0;
  for (pic_ctx *h : b->m) {
    double acc[5];
    const int rc = copy_out(h, h->P.off_acc, acc, sizeof(acc));
    if (rc) return rc;
    sum += acc[4];
  }
  *out = sum;
  return PIC_OK;
}

// Slots in use over all members (synchronous).
int batch_slots(pic_batch_ctx *b, double *out) {
  double sum = 0.0;
  for (pic_ctx *h : b->m) {
    unsigned long long n = 0;
    const int rc = copy_out(h, h->P.off_nslots, &n, sizeof(n));
    if (rc) return rc;
    sum += (double)std::min<unsigned long long>(n, (unsigned long long)h->P.cap);
  }
  *out = sum;
  return PIC_OK;
}

int batch_tune(pic_batch_ctx *b, int &n_steps) {
  static const long long kChunk[] = {1024, 2048, 4096, 2048};
  static const int kMult[] = {1, 1, 1, 2};
  constexpr int kCand = 4;
  if (n_steps < kCand * b->period) return PIC_OK;
  // a push with too few particles measures nothing: tune once the members
  // hold four particles per resident push thread (or a 64th of their
  // pools, for batches too small to reach that)
  {
    PIC_CUDA(cudaStreamSynchronize(b->stream));
    double slots = 0.0, cap = 0.0;
    if (const int rs = batch_slots(b, &slots)) return rs;
    for (pic_ctx *h : b->m) cap += (double)h->P.cap;
    if (slots < std::min(4.0 * (double)b->push_blocks * kThreads, cap / 64.0)) return PIC_OK;
  }
  if (b->tev.empty()) {
    b->tev.resize(2 * (size_t)b->period);
    for (auto &e : b->tev) PIC_CUDA(cudaEventCreate(&e));
  }
  b->tune_chunk.clear();
  b->tune_mult.clear();
  b->tune_ms.clear();
  b->tune_cost.clear();
  int rc = PIC_OK;
  for (int c = 0; c < kCand && rc == PIC_OK; ++c) {
    b->push_chunk = kChunk[c];
    b->push_grid_mult = kMult[c];
    double before = 0.0, after = 0.0;
    PIC_CUDA(cudaStreamSynchronize(b->stream));
    rc = batch_pushes(b, &before);
    if (rc) break;
    b->time_push = true;
    rc = batch_capture(b);  // captures with the timing events and runs one period
    b->time_push = false;
    if (rc) break;
    PIC_CUDA(cudaStreamSynchronize(b->stream));
    double ms = 0.0;
    for (int st = 0; st < b->period; ++st) {
      float t = 0.f;
      const cudaError_t et = cudaEventElapsedTime(&t, b->tev[2 * st], b->tev[2 * st + 1]);
      if (et != cudaSuccess) {
        rc = fail(PIC_ECUDA, std::string("batch tuning: event timing: ") + cudaGetErrorString(et));
        break;
      }
      ms += t;
    }
    if (rc) break;
    rc = batch_pushes(b, &after);
    if (rc) break;
    b->tune_chunk.push_back(kChunk[c]);
    b->tune_mult.push_back(kMult[c]);
    b->tune_ms.push_back(ms);
    b->tune_cost.push_back(ms * 1e6 / std::max(after - before, 1.0));
    n_steps -= b->period;
  }
  if (rc) return rc;
  int best = 0;
  for (int c = 1; c < (int)b->tune_cost.size(); ++c)
    if (b->tune_cost[c] < b->tune_cost[best]) best = c;
  b->tune_pick = best;
  b->push_chunk = b->tune_chunk[best];
  b->push_grid_mult = b->tune_mult[best];
  b->tuned = true;
  if (b->exec) {  // the next period captures with the pick, without events
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  return PIC_OK;
}
}  // namespace

extern "C" {

int pic_batch_create(pic_handle const *members, int n, void *stream, pic_batch *out) {
  if (!members || n <= 0 || !out) return fail(PIC_EINVAL, "bad batch arguments");
  *out = nullptr;
  pic_batch_ctx *b = new pic_batch_ctx();
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {
    const cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete b;
      return fail(PIC_ECUDA, std::string("cudaStreamCreateWithFlags: ") + cudaGetErrorString(e));
    }
    b->own_stream = true;
  }
  long long per = 2;
  for (int q = 0; q < n; ++q) {
    pic_ctx *h = members[q];
    if (!h || !h->stream || h->stream == b->stream) {
      if (b->own_stream) cudaStreamDestroy(b->stream);
      delete b;
      return fail(PIC_EINVAL, "batch members need non-NULL streams other than the batch stream");
    }
    if (h->profiling) {
      if (b->own_stream) cudaStreamDestroy(b->stream);
      delete b;
      return fail(PIC_ESTATE, "a batch member is profiling");
    }
    // the host schedule (pool sorts, collision passes) and the parity of the
    // double-buffered pool repeat after lcm(2 sort_interval, 2 coll_every)
    const long long p2 = 2ll * h->P.g.sort_interval;
    per = per / gcd_ll(per, p2) * p2;
    if (h->P.g.coll_every > 0) {
      const long long p3 = 2ll * h->P.g.coll_every;
      per = per / gcd_ll(per, p3) * p3;
    }
    b->m.push_back(h);
  }
  if (per > 4096) {
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return fail(PIC_EINVAL, "members' sort intervals give a graph period above 4096 steps");
  }
  b->period = (int)per;
  b->ev.resize(n + 1);
  for (auto &e : b->ev) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  *out = b;
  return PIC_OK;
}

int pic_batch_set_launches(pic_batch b, int one_launch_per_phase) {
  if (!b) return fail(PIC_EINVAL, "null batch");
  const bool on = one_launch_per_phase != 0;
  if (on != b->one_launch) {
    PIC_CUDA(cudaStreamSynchronize(b->stream));  // a replay may still run
    b->one_launch = on;
    if (b->exec) {  // the next step captures in the requested form
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
  }
  return PIC_OK;
}

int pic_batch_step(pic_batch b, int n_steps) {
  if (!b || n_steps < 0) return fail(PIC_EINVAL, "bad batch step arguments");
  for (pic_ctx *h : b->m)
    if (h->sticky) return fail(h->sticky, "a batch member holds a device error");
  while (n_steps > 0) {
    // tune the batch's push once its members hold particles (checked before
    // every period until then)
    if (!b->tuned && batch_uniform(b) && b->push_blocks > 0) {
      const int rt = batch_tune(b, n_steps);
      if (rt) return rt;
      if (n_steps <= 0) break;
    }
    if (n_steps < b->period) {
      // tail: members step one by one on their streams, ordered after the batch stream
      PIC_CUDA(cudaEventRecord(b->ev[0], b->stream));
      for (size_t q = 0; q < b->m.size(); ++q) {
        PIC_CUDA(cudaStreamWaitEvent(b->m[q]->stream, b->ev[0], 0));
        for (int st = 0; st < n_steps; ++st) {
          const int rc = enqueue_any(b->m[q], PIC_PHASE_ALL);
          if (rc) return rc;
        }
        PIC_CUDA(cudaEventRecord(b->ev[1 + q], b->m[q]->stream));
        PIC_CUDA(cudaStreamWaitEvent(b->stream, b->ev[1 + q], 0));
      }
      return PIC_OK;
    }
    bool valid = b->exec != nullptr && b->step_at_capture_end.size() == b->m.size();
    for (size_t q = 0; valid && q < b->m.size(); ++q)
      valid = b->m[q]->step == b->step_at_capture_end[q];
    if (!valid) {
      const int rc = batch_capture(b);
      if (rc) return rc;
    } else {
      const int rc = batch_replay(b);
      if (rc) return rc;
    }
    n_steps -= b->period;
  }
  return PIC_OK;
}

int pic_batch_tuning(pic_batch b, int cap, long long *chunk, int *grid_mult, double *ms,
                     double *ns_per_push, int *n, int *pick, int *batch_launches) {
  if (!b || !n || !pick) return fail(PIC_EINVAL, "null pointer");
  *n = (int)b->tune_ms.size();
  *pick = b->tune_pick;
  if (batch_launches) *batch_launches = b->multi ? 1 : 0;
  for (int c = 0; c < *n && c < cap; ++c) {
    if (chunk) chunk[c] = b->tune_chunk[c];
    if (grid_mult) grid_mult[c] = b->tune_mult[c];
    if (ms) ms[c] = b->tune_ms[c];
    if (ns_per_push) ns_per_push[c] = b->tune_cost[c];
  }
  return PIC_OK;
}

int pic_batch_sync(pic_batch b) {
  if (!b) return fail(PIC_EINVAL, "null batch");
  PIC_CUDA(cudaStreamSynchronize(b->stream));
  for (pic_ctx *h : b->m) {
    const int rc = pic_sync(h);
    if (rc) return rc;
  }
  return PIC_OK;
}

int pic_batch_destroy(pic_batch b) {
  if (!b) return PIC_OK;
  cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->tab) cudaFree(b->tab);
  for (auto &e : b->tev) cudaEventDestroy(e);
  for (auto &e : b->ev) cudaEventDestroy(e);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
  return PIC_OK;
}

int pic_profile(pic_handle h, int enable) {
  if (!h) return fail(PIC_EINVAL, "null handle");
  h->profiling = enable != 0;
  h->used = 0;
  h->open_cls = -1;
  return PIC_OK;
}

int pic_profile_read(pic_handle h, double ms[PIC_PROF_N], long long launches[PIC_PROF_N]) {
  if (!h || !ms || !launches) return fail(PIC_EINVAL, "null pointer");
  PIC_CUDA(cudaStreamSynchronize(h->stream));
  for (int c = 0; c < PIC_PROF_N; ++c) {
    ms[c] = 0.0;
    launches[c] = 0;
  }
  for (size_t q = 0; q < h->used; ++q) {
    float t = 0.f;
    PIC_CUDA(cudaEventElapsedTime(&t, h->recs[q].a, h->recs[q].b));
    ms[h->recs[q].cls] += t;
    launches[h->recs[q].cls] += 1;
  }
  h->used = 0;
  return PIC_OK;
}

int pic_destroy(pic_handle h) {
  if (!h) return PIC_OK;
  cudaStreamSynchronize(h->stream);
  if (h->aux) {
    cudaStreamSynchronize(h->aux);
    cudaStreamDestroy(h->aux);
  }
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  for (auto &r : h->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  if (h->own_arena) cudaFree(h->arena);
  delete h;
  return PIC_OK;
}

int pic_step(pic_handle h, int n_steps) {
  if (!h) return fail(PIC_EINVAL, "null handle");
  if (n_steps < 0) return fail(PIC_EINVAL, "negative step count");
  if (h->sticky) return fail(h->sticky, "handle holds a device error");
  for (int q = 0; q < n_steps; ++q) {
    const int rc = enqueue_any(h, PIC_PHASE_ALL);
    if (rc) return rc;
  }
  return PIC_OK;
}

int pic_step_phases(pic_handle h, int mask) {
  if (!h) return fail(PIC_EINVAL, "null handle");
  if (mask & ~PIC_PHASE_ALL) return fail(PIC_EINVAL, "unknown phase bits");
  if (h->sticky) return fail(h->sticky, "handle holds a device error");
  return enqueue_any(h, mask);
}

int pic_sync(pic_handle h) {
  if (!h) return fail(PIC_EINVAL, "null handle");
  PIC_CUDA(cudaStreamSynchronize(h->stream));
  return check_sticky(h);
}

int pic_info_get(pic_handle h, pic_info *out) {
  if (!h || !out) return fail(PIC_EINVAL, "null pointer");
  const Plan &P = h->P;
  std::memset(out, 0, sizeof(*out));
  out->dt = P.dt;
  out->E0 = P.E0;
  out->NW = P.NW;
  out->n_mplanes = P.n_mplanes;
  out->nfield = P.nfield;
  out->nmat = P.nmat;
  out->n_neutrals = P.n_neutrals;
  out->capacity = P.cap;
  out->arena_bytes = P.total;
  unsigned long long ns = 0;
  const int rc = copy_out(h, P.off_nslots, &ns, 8);
  if (rc) return rc;
  out->n_particles = (long long)std::min<unsigned long long>(ns, P.cap);
  long long dstep = 0;
  const int rc1 = copy_out(h, P.off_step, &dstep, 8);
  if (rc1) return rc1;
  out->step = dstep;
  out->launches = h->launches;
  double acc[5];
  const int rc2 = copy_out(h, P.off_acc, acc, sizeof(acc));
  if (rc2) return rc2;
  out->particle_steps = acc[4];
  out->h2d_bytes = h->h2d_bytes;  // including this call's own reads
  out->d2h_bytes = h->d2h_bytes;
  return PIC_OK;
}

int pic_damage(pic_handle h, const int region[4], double *ne_z, double *ed_z, double *layer_out,
               int *layer_flags, double *n_crit) {
  if (!h || !region) return fail(PIC_EINVAL, "null pointer");
  const Plan &P = h->P;
  const int nx = P.g.nx, ny = P.g.ny, nz = P.g.nz;
  if (region[0] < 0 || region[1] > nx || region[0] >= region[1] || region[2] < 0 ||
      region[3] > ny || region[2] >= region[3])
    return fail(PIC_EINVAL, "region must be a non-empty box inside [0, nx) x [0, ny)");
  int rc = check_sticky(h);
  if (rc) return rc;
  cudaStream_t s = h->stream;
  char *A = h->arena;
  double *ne = (double *)(A + P.off_ne), *ed = (double *)(A + P.off_ed),
         *rho = (double *)(A + P.off_rho), *spec = (double *)(A + P.off_spec),
         *part = (double *)(A + P.off_part), *prof = (double *)(A + P.off_prof);
  PIC_CUDA(cudaMemsetAsync(ne, 0, P.nfield * 8, s));
  PIC_CUDA(cudaMemsetAsync(ed, 0, P.nfield * 8, s));
  PIC_CUDA(cudaMemsetAsync(rho, 0, P.nfield * 8, s));
  const int4 r0 = make_int4(0, nx, 0, ny);
  const int2 r1 = make_int2(0, nz);
  if (h->fp64) {
    k_diag_particles<double><<<P.diag_blocks_p, kThreads, 0, s>>>(h->c64, ne, ed, rho, spec, 0, 0.0,
                                                                  1.0, r0, r1, part);
    k_imax_plane<double><<<nz, kThreads, 0, s>>>(h->c64.d.imax, (int)P.nxy, prof + 2 * (nz + 1));
  } else {
    k_diag_particles<float><<<P.diag_blocks_p, kThreads, 0, s>>>(h->c32, ne, ed, rho, spec, 0, 0.0,
                                                                 1.0, r0, r1, part);
    k_imax_plane<float><<<nz, kThreads, 0, s>>>(h->c32.d.imax, (int)P.nxy, prof + 2 * (nz + 1));
  }
  k_profile<<<nz + 1, kThreads, 0, s>>>(ne, ed, nx, ny,
                                        make_int4(region[0], region[1], region[2], region[3]), prof);
  PIC_CUDA(cudaGetLastError());
  std::vector<double> hp(3 * nz + 2);
  PIC_CUDA(cudaMemcpyAsync(hp.data(), prof, hp.size() * 8, cudaMemcpyDeviceToHost, s));
  PIC_CUDA(cudaStreamSynchronize(s));
  h->d2h_bytes += (long long)(hp.size() * 8);
  // region means per node plane; per layer the peaks over its planes and
  // the verdicts (critical density of free electrons at the laser frequency,
  // 9% of four valence electrons per molecule, the layer's energy densities)
  const double cnt = (double)(region[1] - region[0]) * (double)(region[3] - region[2]);
  const double ncrit = kEps0 * kMe * P.omega * P.omega / (kQe * kQe);
  for (int k = 0; k <= nz; ++k) {
    if (ne_z) ne_z[k] = hp[2 * k] / cnt;
    if (ed_z) ed_z[k] = hp[2 * k + 1] / cnt;
  }
  for (size_t L = 0; L < P.layers.size(); ++L) {
    const pic_layer &ly = P.layers[L];
    double mne = 0.0, med = 0.0, mi = 0.0;
    for (int k = ly.z0; k < ly.z1; ++k) {
      mne = std::max(mne, hp[2 * k] / cnt);
      med = std::max(med, hp[2 * k + 1] / cnt);
      mi = std::max(mi, hp[2 * (nz + 1) + k]);
    }
    const double ninst = 0.09 * 4.0 * ly.n_mol;
    if (layer_out) {
      layer_out[4 * L] = mne;
      layer_out[4 * L + 1] = med;
      layer_out[4 * L + 2] = mi;
      layer_out[4 * L + 3] = ninst;
    }
    if (layer_flags) {
      int f = 0;
      if (mne >= ncrit) f |= 1;
      if (mne >= ninst) f |= 2;
      if (ly.e_melt > 0.0 && med >= ly.e_melt) f |= 4;
      if (ly.e_boil > 0.0 && med >= ly.e_boil) f |= 8;
      if (ly.e_dissoc > 0.0 && med >= ly.e_dissoc) f |= 16;
      layer_flags[L] = f;
    }
  }
  if (n_crit) *n_crit = ncrit;
  return PIC_OK;
}

int pic_get_intensity_max(pic_handle h, double *dst) {
  if (!h || !dst) return fail(PIC_EINVAL, "null pointer");
  const Plan &P = h->P;
  std::vector<char> raw((size_t)P.ncell * P.rsz);
  const int rc = copy_out(h, P.off_imax, raw.data(), raw.size());
  if (rc) return rc;
  if (h->fp64)
    to_double<double>(raw, (size_t)P.ncell, dst);
  else
    to_double<float>(raw, (size_t)P.ncell, dst);
  return PIC_OK;
}

int pic_diagnostics(pic_handle h, pic_diag *dg) {
  if (!h || !dg) return fail(PIC_EINVAL, "null pointer");
  if (dg->n_bins < 0 || dg->n_bins > kSpecMax) return fail(PIC_EINVAL, "n_bins out of range");
  if (dg->n_bins > 0 && (!dg->spectrum || !(dg->e_max_eV > dg->e_min_eV)))
    return fail(PIC_EINVAL, "spectrum needs a buffer and e_max > e_min");
  int rc = check_sticky(h);
  if (rc) return rc;
  const Plan &P = h->P;
  cudaStream_t s = h->stream;
  char *A = h->arena;
  double *ne = (double *)(A + P.off_ne), *ed = (double *)(A + P.off_ed),
         *rho = (double *)(A + P.off_rho), *spec = (double *)(A + P.off_spec),
         *part = (double *)(A + P.off_part);
  PIC_CUDA(cudaMemsetAsync(ne, 0, P.nfield * 8, s));
  PIC_CUDA(cudaMemsetAsync(ed, 0, P.nfield * 8, s));
  PIC_CUDA(cudaMemsetAsync(rho, 0, P.nfield * 8, s));
  PIC_CUDA(cudaMemsetAsync(spec, 0, kSpecMax * 8, s));
  const int4 r0 = make_int4(dg->region[0], dg->region[1], dg->region[2], dg->region[3]);
  const int2 r1 = make_int2(dg->region[4], dg->region[5]);
  std::vector<double> pp(3 * P.diag_blocks_p), pg5(5 * P.diag_blocks_g);
  if (h->fp64) {
    k_diag_particles<double><<<P.diag_blocks_p, kThreads, 0, s>>>(
        h->c64, ne, ed, rho, spec, dg->n_bins, dg->e_min_eV, dg->e_max_eV, r0, r1, part);
  } else {
    k_diag_particles<float><<<P.diag_blocks_p, kThreads, 0, s>>>(
        h->c32, ne, ed, rho, spec, dg->n_bins, dg->e_min_eV, dg->e_max_eV, r0, r1, part);
  }
  PIC_CUDA(cudaGetLastError());
  PIC_CUDA(cudaMemcpyAsync(pp.data(), part, pp.size() * 8, cudaMemcpyDeviceToHost, s));
  PIC_CUDA(cudaStreamSynchronize(s));
  if (h->fp64)
    k_diag_grid<double><<<P.diag_blocks_g, kThreads, 0, s>>>(h->c64, ne, ed, rho, part);
  else
    k_diag_grid<float><<<P.diag_blocks_g, kThreads, 0, s>>>(h->c32, ne, ed, rho, part);
  PIC_CUDA(cudaGetLastError());
  PIC_CUDA(cudaMemcpyAsync(pg5.data(), part, pg5.size() * 8, cudaMemcpyDeviceToHost, s));
  double acc[12];
  PIC_CUDA(cudaMemcpyAsync(acc, A + P.off_acc, sizeof(acc), cudaMemcpyDeviceToHost, s));
  // the Poynting split: every flux block's running sums, added in block order
  std::vector<double> fpart((size_t)4 * P.flux_blocks);
  PIC_CUDA(cudaMemcpyAsync(fpart.data(), A + P.off_flux_part, fpart.size() * sizeof(double),
                           cudaMemcpyDeviceToHost, s));
  if (dg->n_bins > 0)
    PIC_CUDA(cudaMemcpyAsync(dg->spectrum, spec, dg->n_bins * 8, cudaMemcpyDeviceToHost, s));
  PIC_CUDA(cudaStreamSynchronize(s));
  h->d2h_bytes +=
      (long long)((pp.size() + pg5.size() + 12 + fpart.size() + std::max(dg->n_bins, 0)) * 8);
  double kin = 0, nel = 0, nho = 0;
  for (int b = 0; b < P.diag_blocks_p; ++b) {
    kin += pp[3 * b];
    nel += pp[3 * b + 1];
    nho += pp[3 * b + 2];
  }
  double uf = 0, mne = 0, med = 0, mrho = 0, mg = 0;
  for (int b = 0; b < P.diag_blocks_g; ++b) {
    uf += pg5[5 * b];
    mne = std::max(mne, pg5[5 * b + 1]);
    med = std::max(med, pg5[5 * b + 2]);
    mrho = std::max(mrho, pg5[5 * b + 3]);
    mg = std::max(mg, pg5[5 * b + 4]);
  }
  // the peak fluence times the sum of spot^2 dx dy over the entrance nodes
  // of the polarised component (F Lx Ly for a plane wave)
  double area = 0.0;
  for (int j = 0; j < P.g.ny; ++j)
    for (int i = 0; i < P.g.nx; ++i) {
      const double x = (i + (P.pulse.pol == 0 ? 0.5 : 0.0)) * P.g.dx;
      const double y = (j + (P.pulse.pol == 0 ? 0.0 : 0.5)) * P.g.dy;
      double sp = 1.0;
      if (P.pulse.w0 > 0.0) {
        const double xc = 0.5 * P.g.nx * P.g.dx, yc = 0.5 * P.g.ny * P.g.dy;
        sp = std::exp(-((x - xc) * (x - xc) + (y - yc) * (y - yc)) / (P.pulse.w0 * P.pulse.w0));
      }
      area += sp * sp * P.g.dx * P.g.dy;
    }
  dg->U_incident = P.pulse.fluence * area;
  dg->U_kinetic = kin;
  dg->U_ionization = acc[2];
  dg->U_absorbed = kin + acc[2];
  dg->frac_absorbed = dg->U_incident > 0 ? dg->U_absorbed / dg->U_incident : 0.0;
  dg->U_joule = acc[0];
  dg->U_field = uf * P.V;
  dg->N_pairs = acc[1];
  dg->n_e_peak = mne;
  dg->energy_density_peak = med;
  dg->gauss_residual_max = mg;
  dg->rho_max = mrho;
  dg->n_electrons_macro = nel;
  dg->n_holes_macro = nho;
  dg->step = h->step;
  dg->flux_plane[0] = P.flux_plane[0];
  dg->flux_plane[1] = P.flux_plane[1];
  double U[4] = {0.0, 0.0, 0.0, 0.0};  // fwd, bwd at the front plane, then the back
  for (int q = 0; q < 2; ++q)
    for (int x = 0; x < P.flux_blocks; ++x) {
      U[2 * q] += fpart[2 * ((size_t)q * P.flux_blocks + x)];
      U[2 * q + 1] += fpart[2 * ((size_t)q * P.flux_blocks + x) + 1];
    }
  dg->U_fwd[0] = U[0];
  dg->U_bwd[0] = U[1];
  dg->U_fwd[1] = U[2];
  dg->U_bwd[1] = U[3];
  dg->frac_reflected = dg->frac_transmitted = dg->frac_absorbed_flux = 0.0;
  if (U[0] > 0.0) {
    dg->frac_reflected = U[1] / U[0];
    dg->frac_transmitted = U[2] / U[0];
    dg->frac_absorbed_flux = ((U[0] - U[1]) - (U[2] - U[3])) / U[0];
  }
  return PIC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// State access
// ---------------------------------------------------------------------------
namespace {
template <class R>
int get_fields_t(pic_ctx *h, double *dst) {
  const Plan &P = h->P;
  Ctx<R> &X = ctx_of<R>(h);
  std::vector<char> raw(std::max(4 * P.nfield, P.nmat) * sizeof(R));
  R *const *arrs[2] = {X.d.E, X.d.B};
  for (int g3 = 0; g3 < 2; ++g3)
    for (int d = 0; d < 3; ++d) {
      int rc = copy_out(h, off_of(h, arrs[g3][d]), raw.data(), P.nfield * sizeof(R));
      if (rc) return rc;
      to_double<R>(raw, P.nfield, dst + (size_t)(3 * g3 + d) * P.nfield);
    }
  {
    int rc = copy_out(h, off_of(h, X.d.J4), raw.data(), 4 * P.nfield * sizeof(R));
    if (rc) return rc;
    const R *j = (const R *)raw.data();
    for (int d = 0; d < 3; ++d)
      for (long long o = 0; o < P.nfield; ++o) dst[(size_t)(6 + d) * P.nfield + o] = (double)j[4 * o + d];
  }
  std::vector<double> tmp(P.nmat);
  R *const *pq[2] = {X.d.P, X.d.Q};
  for (int g2 = 0; g2 < 2; ++g2)
    for (int d = 0; d < 3; ++d) {
      double *out = dst + (size_t)(9 + 3 * g2 + d) * P.nfield;
      std::fill(out, out + P.nfield, 0.0);
      if (!P.nmat) continue;
      int rc = copy_out(h, off_of(h, pq[g2][d]), raw.data(), P.nmat * sizeof(R));
      if (rc) return rc;
      to_double<R>(raw, P.nmat, tmp.data());
      for (int mp = 0; mp < P.n_mplanes; ++mp)
        std::memcpy(out + (size_t)P.kplane[mp] * P.nxy, tmp.data() + (size_t)mp * P.nxy,
                    P.nxy * sizeof(double));
    }
  return PIC_OK;
}

template <class R>
int set_fields_t(pic_ctx *h, const double *src) {
  const Plan &P = h->P;
  Ctx<R> &X = ctx_of<R>(h);
  std::vector<char> raw;
  R *const *arrs[2] = {X.d.E, X.d.B};
  for (int g3 = 0; g3 < 2; ++g3)
    for (int d = 0; d < 3; ++d) {
      from_double<R>(src + (size_t)(3 * g3 + d) * P.nfield, P.nfield, raw);
      int rc = copy_in(h, off_of(h, arrs[g3][d]), raw.data(), raw.size());
      if (rc) return rc;
    }
  {
    std::vector<double> j4(4 * P.nfield, 0.0);
    for (int d = 0; d < 3; ++d)
      for (long long o = 0; o < P.nfield; ++o) j4[4 * o + d] = src[(size_t)(6 + d) * P.nfield + o];
    from_double<R>(j4.data(), j4.size(), raw);
    int rc = copy_in(h, off_of(h, X.d.J4), raw.data(), raw.size());
    if (rc) return rc;
    // the next E step reads the current on every plane
    const uint32_t all = 1u;
    rc = copy_in(h, P.off_jtouch + (size_t)P.g.nz * sizeof(uint32_t), &all, sizeof(all));
    if (rc) return rc;
  }
  std::vector<double> tmp(P.nmat);
  R *const *pq[2] = {X.d.P, X.d.Q};
  for (int g2 = 0; g2 < 2; ++g2)
    for (int d = 0; d < 3; ++d) {
      if (!P.nmat) continue;
      const double *in = src + (size_t)(9 + 3 * g2 + d) * P.nfield;
      for (int mp = 0; mp < P.n_mplanes; ++mp)
        std::memcpy(tmp.data() + (size_t)mp * P.nxy, in + (size_t)P.kplane[mp] * P.nxy,
                    P.nxy * sizeof(double));
      from_double<R>(tmp.data(), P.nmat, raw);
      int rc = copy_in(h, off_of(h, pq[g2][d]), raw.data(), raw.size());
      if (rc) return rc;
    }
  return PIC_OK;
}

template <class R>
int get_particles_t(pic_ctx *h, long long *n, uint64_t *id, int32_t *cell, double *off, double *u,
                    uint32_t *tag) {
  const Plan &P = h->P;
  Ctx<R> &X = ctx_of<R>(h);
  unsigned long long ns = 0;
  int rc = copy_out(h, P.off_nslots, &ns, 8);
  if (rc) return rc;
  ns = std::min<unsigned long long>(ns, P.cap);
  std::vector<int32_t> c(ns);
  if (ns) {
    rc = copy_out(h, off_of(h, X.d.pcell), c.data(), ns * 4);
    if (rc) return rc;
  }
  long long live = 0;
  for (unsigned long long q = 0; q < ns; ++q) live += c[q] >= 0;
  *n = live;
  if (!id || !cell || !off || !u || !tag) return PIC_OK;
  std::vector<char> raw(std::max<size_t>(ns, 1) * sizeof(R));
  std::vector<double> tmp(ns);
  std::vector<double> o3(3 * ns), u3(3 * ns);
  for (int d = 0; d < 3; ++d) {
    if (!ns) break;
    rc = copy_out(h, off_of(h, X.d.po[d]), raw.data(), ns * sizeof(R));
    if (rc) return rc;
    to_double<R>(raw, ns, tmp.data());
    for (unsigned long long q = 0; q < ns; ++q) o3[3 * q + d] = tmp[q];
    rc = copy_out(h, off_of(h, X.d.pu[d]), raw.data(), ns * sizeof(R));
    if (rc) return rc;
    to_double<R>(raw, ns, tmp.data());
    for (unsigned long long q = 0; q < ns; ++q) u3[3 * q + d] = tmp[q];
  }
  std::vector<uint32_t> t(ns);
  std::vector<unsigned long long> ids(ns);
  if (ns) {
    rc = copy_out(h, off_of(h, X.d.ptag), t.data(), ns * 4);
    if (rc) return rc;
    rc = copy_out(h, off_of(h, X.d.pid), ids.data(), ns * 8);
    if (rc) return rc;
  }
  long long w = 0;
  for (unsigned long long q = 0; q < ns; ++q) {
    if (c[q] < 0) continue;
    id[w] = ids[q];
    cell[w] = c[q];
    for (int d = 0; d < 3; ++d) {
      off[3 * w + d] = o3[3 * q + d];
      u[3 * w + d] = u3[3 * q + d];
    }
    tag[w] = t[q];
    ++w;
  }
  return PIC_OK;
}

template <class R>
int set_particles_t(pic_ctx *h, long long n, const uint64_t *id, const int32_t *cell,
                    const double *off, const double *u, const uint32_t *tag) {
  const Plan &P = h->P;
  Ctx<R> &X = ctx_of<R>(h);
  if (n < 0 || n > P.cap) return fail(PIC_EINVAL, "particle count exceeds the pool");
  for (long long q = 0; q < n; ++q) {
    if (cell[q] < 0 || cell[q] >= P.ncell) return fail(PIC_EINVAL, "particle cell out of range");
    const int k = (int)(cell[q] / P.nxy);
    if (k < 2 || k >= P.g.nz - 2) return fail(PIC_EINVAL, "particle inside the z outflow band");
    if ((int)(tag[q] >> 1) >= (int)P.layers.size()) return fail(PIC_EINVAL, "tag names no layer");
    for (int d = 0; d < 3; ++d)
      if (!(off[3 * q + d] >= 0.0 && off[3 * q + d] < 1.0))
        return fail(PIC_EINVAL, "particle offset outside [0, 1)");
  }
  std::vector<double> tmp(std::max<long long>(n, 1));
  std::vector<char> raw;
  int rc;
  for (int d = 0; d < 3; ++d) {
    for (long long q = 0; q < n; ++q) tmp[q] = off[3 * q + d];
    from_double<R>(tmp.data(), n, raw);
    if (n && (rc = copy_in(h, off_of(h, X.d.po[d]), raw.data(), raw.size()))) return rc;
    for (long long q = 0; q < n; ++q) tmp[q] = u[3 * q + d];
    from_double<R>(tmp.data(), n, raw);
    if (n && (rc = copy_in(h, off_of(h, X.d.pu[d]), raw.data(), raw.size()))) return rc;
  }
  if (n) {
    if ((rc = copy_in(h, off_of(h, X.d.pcell), cell, n * 4))) return rc;
    if ((rc = copy_in(h, off_of(h, X.d.ptag), tag, n * 4))) return rc;
    if ((rc = copy_in(h, off_of(h, X.d.pid), id, n * 8))) return rc;
  }
  unsigned long long ns = (unsigned long long)n;
  return copy_in(h, P.off_nslots, &ns, 8);
}

template <class R>
int get_material_t(pic_ctx *h, uint32_t *alive, double *eamp, uint64_t *T) {
  const Plan &P = h->P;
  if (!P.nmat) return PIC_OK;
  int rc;
  if (alive && (rc = copy_out(h, P.off_alive, alive, P.nmat * 4))) return rc;
  if (T && (rc = copy_out(h, P.off_T, T, P.nmat * 8))) return rc;
  if (eamp) {
    std::vector<char> raw(P.nmat * sizeof(R));
    if ((rc = copy_out(h, P.off_eamp, raw.data(), raw.size()))) return rc;
    to_double<R>(raw, P.nmat, eamp);
  }
  return PIC_OK;
}

// Raw history -> block form: after sample t = step - 1 with position
// s = t mod NW, slots 0..s keep this block's samples, slots above s the
// suffix maxima of the previous block, pm the prefix max of this block.
template <class R>
int set_material_t(pic_ctx *h, const uint32_t *alive, const double *win) {
  const Plan &P = h->P;
  if (!P.nmat) return PIC_OK;
  int rc;
  // k_ionize skips no plane until the next window pass stamps them again
  const uint32_t all = 0xFFFFFFFFu;
  if ((rc = copy_in(h, P.off_hot + (size_t)P.n_mplanes * sizeof(uint32_t), &all, sizeof(all))))
    return rc;
  if (alive && (rc = copy_in(h, P.off_alive, alive, P.nmat * 4))) return rc;
  if (win) {
    const int NW = P.NW;
    std::vector<double> W(win, win + (size_t)NW * P.nmat), pm(P.nmat, 0.0);
    if (h->step > 0) {
      const int s = (int)((h->step - 1) % NW);
      for (long long m = 0; m < P.nmat; ++m) {
        double run = 0.0;
        for (int q = NW - 1; q > s; --q) {
          run = std::max(run, W[(size_t)q * P.nmat + m]);
          W[(size_t)q * P.nmat + m] = run;
        }
        double pre = 0.0;
        for (int q = 0; q <= s; ++q) pre = std::max(pre, W[(size_t)q * P.nmat + m]);
        if (s == NW - 1) {
          double r2 = 0.0;
          for (int q = NW - 1; q >= 0; --q) {
            r2 = std::max(r2, W[(size_t)q * P.nmat + m]);
            W[(size_t)q * P.nmat + m] = r2;
          }
        }
        pm[m] = pre;
      }
    }
    std::vector<char> raw;
    from_double<R>(W.data(), W.size(), raw);
    if ((rc = copy_in(h, P.off_win, raw.data(), raw.size()))) return rc;
    from_double<R>(pm.data(), pm.size(), raw);
    if ((rc = copy_in(h, P.off_pm, raw.data(), raw.size()))) return rc;
  }
  // thresholds are recomputed at the next window phase
  std::vector<double> inval(P.nmat, -1.0);
  std::vector<char> raw;
  from_double<R>(inval.data(), inval.size(), raw);
  return copy_in(h, P.off_ckey, raw.data(), raw.size());
}
}  // namespace

extern "C" {

int pic_get_fields(pic_handle h, double *dst) {
  if (!h || !dst) return fail(PIC_EINVAL, "null pointer");
  PIC_CUDA(cudaStreamSynchronize(h->stream));
  return h->fp64 ? get_fields_t<double>(h, dst) : get_fields_t<float>(h, dst);
}

int pic_set_fields(pic_handle h, const double *src) {
  if (!h || !src) return fail(PIC_EINVAL, "null pointer");
  PIC_CUDA(cudaStreamSynchronize(h->stream));
  h->bh_valid = false;  // the next field pass recomputes Bh from the new E, B
  return h->fp64 ? set_fields_t<double>(h, src) : set_fields_t<float>(h, src);
}

int pic_get_particles(pic_handle h, long long *n, uint64_t *id, int32_t *cell, double *off,
                      double *u, uint32_t *tag) {
  if (!h || !n) return fail(PIC_EINVAL, "null pointer");
  PIC_CUDA(cudaStreamSynchronize(h->stream));
  return h->fp64 ? get_particles_t<double>(h, n, id, cell, off, u, tag)
                 : get_particles_t<float>(h, n, id, cell, off, u, tag);
}

int pic_set_particles(pic_handle h, long long n, const uint64_t *id, const int32_t *cell,
                      const double *off, const double *u, const uint32_t *tag) {
  if (!h || (n > 0 && (!id || !cell || !off || !u || !tag))) return fail(PIC_EINVAL, "null pointer");
  PIC_CUDA(cudaStreamSynchronize(h->stream));
  return h->fp64 ? set_particles_t<double>(h, n, id, cell, off, u, tag)
                 : set_particles_t<float>(h, n, id, cell, off, u, tag);
}

int pic_get_material(pic_handle h, uint32_t *alive, double *eamp, uint64_t *T) {
  if (!h) return fail(PIC_EINVAL, "null handle");
  PIC_CUDA(cudaStreamSynchronize(h->stream));
  return h->fp64 ? get_material_t<double>(h, alive, eamp, T) : get_material_t<float>(h, alive, eamp, T);
}

int pic_set_material(pic_handle h, const uint32_t *alive, const double *win) {
  if (!h) return fail(PIC_EINVAL, "null handle");
  PIC_CUDA(cudaStreamSynchronize(h->stream));
  return h->fp64 ? set_material_t<double>(h, alive, win) : set_material_t<float>(h, alive, win);
}

int pic_get_scalars(pic_handle h, long long *step, double out[4]) {
  if (!h || !out) return fail(PIC_EINVAL, "null pointer");
  if (step) *step = h->step;
  return copy_out(h, h->P.off_acc, out, 32);
}

int pic_set_scalars(pic_handle h, long long step, const double in[4]) {
  if (!h || !in || step < 0) return fail(PIC_EINVAL, "bad arguments");
  int rc = copy_in(h, h->P.off_acc, in, 32);
  if (rc) return rc;
  h->step = step;
  return copy_in(h, h->P.off_step, &step, 8);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Checkpoints: the configuration, the host-side step state and the arena.
// Every device-side quantity of a simulation lives in its arena, so writing
// the arena back into a simulation created from the same configuration
// resumes it exactly.  The two pool halves are the exception: only the live
// half holds state, and only its first nslots entries (slots at or past
// nslots are written before they are read, and the other half is written by
// the sort before it becomes live), so those are all that is stored.
// ---------------------------------------------------------------------------
namespace {

constexpr char kCkptMagic[8] = {'P', 'I', 'C', 'C', 'K', 'P', 'T', '1'};
constexpr uint32_t kCkptVersion = 4;
constexpr size_t kStageBytes = size_t(64) << 20;

struct CkptHeader {
  char magic[8];
  uint32_t version, n_layers;
  pic_grid grid;
  pic_pulse pulse;
  uint64_t seed;
  int64_t step;
  int32_t since_sort, bh_valid;
  uint64_t arena_bytes;  // layout check: the plan's total size
  uint64_t pool_lo, pool_hi;  // arena span of the two pool halves
  uint64_t nslots;       // live slots stored
};

struct Span {
  size_t off, elem;
};

// arrays of pool half b with their element sizes
std::vector<Span> pool_arrays(const Plan &P, int b) {
  std::vector<Span> a{{P.off_pc[b], 4}};
  for (int d = 0; d < 3; ++d) a.push_back({P.off_po[b][d], (size_t)P.rsz});
  for (int d = 0; d < 3; ++d) a.push_back({P.off_pu[b][d], (size_t)P.rsz});
  a.push_back({P.off_pt[b], 4});
  a.push_back({P.off_pid[b], 8});
  return a;
}

size_t pool_hi(const Plan &P) { return align_up(P.off_pid[1] + std::max<size_t>(P.cap * 8, 1)); }

// pinned host buffer through which the arena streams to or from a file
struct Stage {
  char *buf = nullptr;
  ~Stage() {
    if (buf) cudaFreeHost(buf);
  }
};

struct File {
  FILE *f = nullptr;
  ~File() {
    if (f) std::fclose(f);
  }
};

int write_span(pic_ctx *h, FILE *f, char *st, size_t off, size_t bytes) {
  while (bytes) {
    const size_t n = std::min(bytes, kStageBytes);
    PIC_CUDA(cudaMemcpyAsync(st, h->arena + off, n, cudaMemcpyDeviceToHost, h->stream));
    PIC_CUDA(cudaStreamSynchronize(h->stream));
    h->d2h_bytes += (long long)n;
    if (std::fwrite(st, 1, n, f) != n) return fail(PIC_EIO, "checkpoint write failed");
    off += n;
    bytes -= n;
  }
  return PIC_OK;
}

int read_span(pic_ctx *h, FILE *f, char *st, size_t off, size_t bytes) {
  while (bytes) {
    const size_t n = std::min(bytes, kStageBytes);
    if (std::fread(st, 1, n, f) != n) return fail(PIC_EIO, "checkpoint file is truncated");
    PIC_CUDA(cudaMemcpyAsync(h->arena + off, st, n, cudaMemcpyHostToDevice, h->stream));
    PIC_CUDA(cudaStreamSynchronize(h->stream));
    h->h2d_bytes += (long long)n;
    off += n;
    bytes -= n;
  }
  return PIC_OK;
}

// header and layers of a checkpoint file, checked for magic, version and
// layer count
int read_head(FILE *f, CkptHeader &hd, std::vector<pic_layer> &layers) {
  if (std::fread(&hd, sizeof(hd), 1, f) != 1) return fail(PIC_EIO, "not a checkpoint (short header)");
  if (std::memcmp(hd.magic, kCkptMagic, sizeof(kCkptMagic)) != 0)
    return fail(PIC_EIO, "not a checkpoint (bad magic)");
  if (hd.version != kCkptVersion) return fail(PIC_EIO, "unsupported checkpoint version");
  if (hd.n_layers > PIC_MAX_LAYERS) return fail(PIC_EIO, "checkpoint has a bad layer count");
  layers.resize(hd.n_layers);
  if (hd.n_layers && std::fread(layers.data(), sizeof(pic_layer), hd.n_layers, f) != hd.n_layers)
    return fail(PIC_EIO, "checkpoint file is truncated");
  return PIC_OK;
}

}  // namespace

extern "C" {

int pic_save(pic_handle h, const char *path) {
  if (!h || !path) return fail(PIC_EINVAL, "null pointer");
  PIC_CUDA(cudaStreamSynchronize(h->stream));
  int rc = check_sticky(h);
  if (rc) return rc;
  const Plan &P = h->P;
  unsigned long long ns = 0;
  rc = copy_out(h, P.off_nslots, &ns, 8);
  if (rc) return rc;
  ns = std::min<unsigned long long>(ns, (unsigned long long)P.cap);
  CkptHeader hd;
  std::memset(&hd, 0, sizeof(hd));
  std::memcpy(hd.magic, kCkptMagic, sizeof(kCkptMagic));
  hd.version = kCkptVersion;
  hd.n_layers = (uint32_t)P.layers.size();
  hd.grid = P.g;
  hd.pulse = P.pulse;
  hd.seed = h->seed;
  hd.step = h->step;
  hd.since_sort = h->since_sort;
  hd.bh_valid = h->bh_valid ? 1 : 0;
  hd.arena_bytes = P.total;
  hd.pool_lo = P.off_pc[0];
  hd.pool_hi = pool_hi(P);
  hd.nslots = ns;
  // the live pool half: the one the particle pointers address
  const int32_t *pcell = h->fp64 ? h->c64.d.pcell : h->c32.d.pcell;
  const int live = (const char *)pcell == h->arena + P.off_pc[1] ? 1 : 0;
  // written to path.tmp and renamed, so that a failed save leaves no
  // partial file under the final name
  const std::string tmp = std::string(path) + ".tmp";
  {
    Stage st;
    PIC_CUDA(cudaMallocHost((void **)&st.buf, kStageBytes));
    File f;
    f.f = std::fopen(tmp.c_str(), "wb");
    if (!f.f) return fail(PIC_EIO, "cannot open " + tmp + " for writing");
    if (std::fwrite(&hd, sizeof(hd), 1, f.f) != 1 ||
        (hd.n_layers &&
         std::fwrite(P.layers.data(), sizeof(pic_layer), hd.n_layers, f.f) != hd.n_layers))
      rc = fail(PIC_EIO, "checkpoint write failed");
    if (!rc) rc = write_span(h, f.f, st.buf, 0, hd.pool_lo);
    if (!rc) rc = write_span(h, f.f, st.buf, hd.pool_hi, P.total - hd.pool_hi);
    for (const Span &a : pool_arrays(P, live))
      if (!rc) rc = write_span(h, f.f, st.buf, a.off, ns * a.elem);
    if (!rc && std::fflush(f.f) != 0) rc = fail(PIC_EIO, "checkpoint write failed");
    const int closed = std::fclose(f.f);
    f.f = nullptr;
    if (!rc && closed != 0) rc = fail(PIC_EIO, "checkpoint write failed");
  }
  if (rc) {
    std::remove(tmp.c_str());
    return rc;
  }
  if (std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return fail(PIC_EIO, std::string("cannot rename the checkpoint to ") + path);
  }
  return PIC_OK;
}

int pic_checkpoint_config(const char *path, pic_grid *grid, pic_pulse *pulse, pic_layer *layers,
                          int *n_layers, uint64_t *seed, long long *step) {
  if (!path || !grid || !pulse || !layers || !n_layers || !seed)
    return fail(PIC_EINVAL, "null pointer");
  File f;
  f.f = std::fopen(path, "rb");
  if (!f.f) return fail(PIC_EIO, std::string("cannot open ") + path);
  CkptHeader hd;
  std::vector<pic_layer> ly;
  const int rc = read_head(f.f, hd, ly);
  if (rc) return rc;
  *grid = hd.grid;
  *pulse = hd.pulse;
  std::copy(ly.begin(), ly.end(), layers);
  *n_layers = (int)hd.n_layers;
  *seed = hd.seed;
  if (step) *step = hd.step;
  return PIC_OK;
}

int pic_load(const char *path, void *stream, void *d_arena, size_t arena_bytes, pic_handle *out) {
  if (!path || !out) return fail(PIC_EINVAL, "null pointer");
  *out = nullptr;
  File f;
  f.f = std::fopen(path, "rb");
  if (!f.f) return fail(PIC_EIO, std::string("cannot open ") + path);
  CkptHeader hd;
  std::vector<pic_layer> ly;
  int rc = read_head(f.f, hd, ly);
  if (rc) return rc;
  pic_material m;
  std::memset(&m, 0, sizeof(m));
  m.n_layers = (int)hd.n_layers;
  m.layers = ly.data();
  pic_handle h = nullptr;
  rc = pic_create(&hd.grid, &m, &hd.pulse, hd.seed, stream, d_arena, arena_bytes, &h);
  if (rc) return rc;
  const Plan &P = h->P;
  if (hd.arena_bytes != P.total || hd.pool_lo != P.off_pc[0] || hd.pool_hi != pool_hi(P) ||
      hd.nslots > (uint64_t)P.cap || hd.step < 0) {
    pic_destroy(h);
    return fail(PIC_EIO, "checkpoint layout does not match this library's");
  }
  {
    Stage st;
    cudaError_t e = cudaMallocHost((void **)&st.buf, kStageBytes);
    if (e != cudaSuccess) rc = fail(PIC_ECUDA, std::string("cudaMallocHost: ") + cudaGetErrorString(e));
    // pic_create's initialisation is on the same stream, before these copies
    if (!rc) rc = read_span(h, f.f, st.buf, 0, hd.pool_lo);
    if (!rc) rc = read_span(h, f.f, st.buf, hd.pool_hi, P.total - hd.pool_hi);
    for (const Span &a : pool_arrays(P, 0))
      if (!rc) rc = read_span(h, f.f, st.buf, a.off, hd.nslots * a.elem);
    if (!rc && std::fgetc(f.f) != EOF) rc = fail(PIC_EIO, "checkpoint file has trailing data");
  }
  if (rc) {
    pic_destroy(h);
    return rc;
  }
  h->step = hd.step;
  h->since_sort = hd.since_sort;
  h->bh_valid = hd.bh_valid != 0;
  *out = h;
  return PIC_OK;
}

}  // extern "C"
