// Kernels of one PIC step on sm_103a.  Every step of the hot path runs here:
//   k_push      gather (TSC) + relativistic Boris + move + Esirkepov deposit;
//               marks the cell planes it deposits from
//   k_bstep     B half steps (Faraday): B and Bh around the particle phase
//   k_efull     E step with the Lorentz polarisation current (trapezoidal
//               oscillator), Silver-Mueller z faces with the laser source,
//               Joule work, J read and cleared near the marked planes
//   k_window    cell-centred |E|, exact sliding maximum over one optical
//               cycle (van Herk / Gil-Werman blocks), the per-cell threshold
//               cache with an exact low-field skip, the work list for
//   k_keldysh   Keldysh thresholds of the cells whose amplitude changed
//   k_ionize    Philox draws per alive neutral, electron + hole appends
//               (planes with no cell above the skip amplitude return at once)
//   k_hist / k_scan* / k_scatter   counting sort of the pool by cell
//   k_coll_*    binary collisions (cell lists, per-cell preparation, pairs)
//   k_diag_*    FP64 diagnostics and damage metrics
#pragma once
#include "pic_device.cuh"

namespace pg {

// Per-layer constants in the working precision (no double math in kernels).
template <class R>
struct LayerR {
  R deps, cn_a, cn_b, cn_g, inv_den, two_over_h;  // trapezoidal oscillator
  int is_static, ppc;
  R qmdt2[2];   // q dt / (2 m)
  R jpref[2][3];// -q w dl_d / (V dt) per species and axis
  R kG, kX, kP, e_skip;
  R sig_v;
  R inv_mass_c2[2];
  R mhat[2];  // carrier masses / m_e (collisions)
  R wmac;     // real particles per macroparticle (collisions)
};

template <class R>
struct Ctx {
  Dev<R> d;
  const LayerR<R> *lr;
  // the other half of the double-buffered pool (sorting)
  int32_t *acell;
  R *ao[3], *au[3];
  uint32_t *atag;
  unsigned long long *aid;
  // material cells whose Keldysh threshold must be recomputed this step
  int *work;
  int *work_n;
  // per-neutral leave steps in units of 64 steps (nmat x ppc_max)
  uint16_t *leave16;
  int ppc_max;
};

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Block coordinates of a launch: blockIdx and gridDim for a simulation's own
// launch, or, for a batch launch that covers many simulations, the block's
// place (x, y) in one member's grid of gx x gy blocks.
struct Blk {
  int x, y, gx, gy;
};
__device__ __forceinline__ Blk blk_here() {
  return Blk{(int)blockIdx.x, (int)blockIdx.y, (int)gridDim.x, (int)gridDim.y};
}

// Absorbing transverse layers (the paper's outflow faces, Sec. 3.1): a
// convolutional PML (Roden and Gedney 2000; kappa = 1, alpha = 0) of
// D.pml cells on each side of the periodic x and y seams.  A derivative df
// of the curl inside them becomes df + psi with psi <- b psi + (b - 1) df;
// b is 1 outside, where psi stays 0.
enum { kPsiEYX = 0, kPsiEZX, kPsiEXY, kPsiEZY, kPsiBYX, kPsiBZX, kPsiBXY, kPsiBZY };

template <class R>
__device__ __forceinline__ bool pml_point(const Dev<R> &D, int i, int j) {
  return D.pml > 0 && (i < D.pml || i >= D.nx - D.pml || j < D.pml || j >= D.ny - D.pml);
}

template <class R>
__device__ __forceinline__ R pml_step(R *psi, R b, R df) {
  const R p = b * *psi + (b - R(1)) * df;
  *psi = p;
  return df + p;
}

// A B point's layer derivative over the pass's half steps, all with the same
// E: d1 and d2 for the closing half step of this step and the opening one of
// the next (two convolution steps; the state after the first is kept in
// psi_c), or, for kMode 0, the opening half step alone, from the state that
// the last closing half step left in psi_c (so a Bh primed again after a
// host write advances the convolution once, as the opening half step does).
template <int kMode, class R>
__device__ __forceinline__ void pml_two(R *psi, R *psi_c, R b, R df, R &d1, R &d2) {
  if constexpr (kMode == 0) {
    const R p = b * *psi_c + (b - R(1)) * df;
    d1 = d2 = df + p;
    *psi = p;
  } else {
    const R p1 = b * *psi + (b - R(1)) * df;
    d1 = df + p1;
    *psi_c = p1;
    const R p2 = b * p1 + (b - R(1)) * df;
    d2 = df + p2;
    *psi = p2;
  }
}

template <class R>
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double part[32];
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) part[w] = v;
  __syncthreads();
  double tot = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tot += part[q];
  return tot;
}


template <class R>
__device__ __forceinline__ void shape_int(R d, R w[3], int &b) {
  const int s = d >= R(0.5);
  const R e = d - R(s);
  b = s - 1;
  const R hm = R(0.5) - e, hp = R(0.5) + e;
  w[0] = R(0.5) * hm * hm;
  w[1] = R(0.75) - e * e;
  w[2] = R(0.5) * hp * hp;
}

template <class R>
__device__ __forceinline__ void shape_half(R d, R w[3]) {
  const R e = d - R(0.5);
  const R hm = R(0.5) - e, hp = R(0.5) + e;
  w[0] = R(0.5) * hm * hm;
  w[1] = R(0.75) - e * e;
  w[2] = R(0.5) * hp * hp;
}

// sum_c wz[c] sum_b wy[b] sum_a wx[a] f[zo_c + yo_b + x_a]; zo, yo are plane
// and row offsets in elements
template <class R>
__device__ __forceinline__ R gather27(const R *__restrict__ f, const int xs[3], const int yo[3],
                                      const int zo[3], const R wx[3], const R wy[3],
                                      const R wz[3]) {
  R acc = R(0);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    R accy = R(0);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const R *row = f + (zo[c] + yo[b]);
      const R accx = wx[0] * __ldg(row + xs[0]) + wx[1] * __ldg(row + xs[1]) +
                     wx[2] * __ldg(row + xs[2]);
      accy += wy[b] * accx;
    }
    acc += wz[c] * accy;
  }
  return acc;
}

template <class R>
__device__ __forceinline__ void atomic_add(R *p, R v) {
  atomicAdd(p, v);
}

// Adds (a, b, c) to the interleaved current of one field point: one
// red.global.add.v4.f32 in FP32, three scalar atomics in FP64.
template <class R>
__device__ __forceinline__ void red_add3(R *p, R a, R b, R c);
template <>
__device__ __forceinline__ void red_add3<float>(float *p, float a, float b, float c) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c),
               "f"(0.0f)
               : "memory");
}
template <>
__device__ __forceinline__ void red_add3<double>(double *p, double a, double b, double c) {
  if (a != 0.0) atomicAdd(p, a);
  if (b != 0.0) atomicAdd(p + 1, b);
  if (c != 0.0) atomicAdd(p + 2, c);
}

// Esirkepov deposit on a 4-node frame per axis (moves are below one cell):
// with S0, S1 the old and new shape, DS = S1 - S0, A = S0 + DS/2 and C_d the
// running sum of DS_d along d,
//   J_x(a,b,c) = jpref_x C_x[a] (A_y[b] A_z[c] + DS_y[b] DS_z[c] / 12)
// and cyclically; the three components of one node go out in one vector
// reduction.  C_d is exactly 0 on the last node of the support.  A particle
// whose support shifts on no axis (nearly every one on a given step) takes a
// 3 x 3 x 3 loop with no per-node frame test.
template <class R>
__device__ __forceinline__ void esirkepov(const Dev<R> &D, const R jpref[3], const int co[3],
                                          const R oo[3], const int cn[3], const R on[3]) {
  R DS[3][4], A[3][4], Cs[3][4];
  int nn[3], off[3][4];
  const int nx = D.nx, ny = D.ny, nxy = D.nxy;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    R wo[3], wn[3];
    int bo, bn;
    shape_int(oo[d], wo, bo);
    shape_int(on[d], wn, bn);
    const int i0o = co[d] + bo + 1, i0n = cn[d] + bn + 1;
    const int s = i0n - i0o;
    const bool lo = s < 0, hi = s > 0;
    const int base = i0o - 1 - (lo ? 1 : 0);
    nn[d] = 3 + (s != 0);
    const R S0[4] = {lo ? R(0) : wo[0], lo ? wo[0] : wo[1], lo ? wo[1] : wo[2], lo ? wo[2] : R(0)};
    const R S1[4] = {hi ? R(0) : wn[0], hi ? wn[0] : wn[1], hi ? wn[1] : wn[2], hi ? wn[2] : R(0)};
    R run = R(0);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      DS[d][q] = S1[q] - S0[q];
      A[d][q] = S0[q] + R(0.5) * DS[d][q];
      run += DS[d][q];
      Cs[d][q] = q < nn[d] - 1 ? jpref[d] * run : R(0);
      const int g = base + q;
      off[d][q] = d == 0 ? wrap(g, nx) : (d == 1 ? wrap(g, ny) * nx : g * nxy);
    }
  }
  R *__restrict__ J = D.J4;
  const R twelfth = R(1.0 / 12.0);
  auto node = [&](int a, int b, int c) {
    const R jx = Cs[0][a] * (A[1][b] * A[2][c] + DS[1][b] * DS[2][c] * twelfth);
    const R jy = Cs[1][b] * (A[2][c] * A[0][a] + DS[2][c] * DS[0][a] * twelfth);
    const R jz = Cs[2][c] * (A[0][a] * A[1][b] + DS[0][a] * DS[1][b] * twelfth);
    if (jx == R(0) && jy == R(0) && jz == R(0)) return;
    red_add3(J + 4 * (off[2][c] + off[1][b] + off[0][a]), jx, jy, jz);
  };
  if ((nn[0] | nn[1] | nn[2]) == 3) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int a = 0; a < 3; ++a) node(a, b, c);
  } else {
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int a = 0; a < 4; ++a)
          if (a < nn[0] && b < nn[1] && c < nn[2]) node(a, b, c);
  }
}

// Blocks per SM for the push: two (128 registers).  In FP32, 64 and 80
// registers (four and three blocks) measured slower: the gather's loads in
// flight per thread matter more than resident warps.
template <class R> struct PushOcc { static constexpr int v = 2; };
// blocks of consecutive slots a block of the push takes before it jumps a
// grid ahead (1: plain grid stride)
constexpr int kPushRun = 4;

// Pushes slots below last (and below the slots in use) in runs of `run`
// consecutive blocks of threads: the thread's slots are first + threadIdx.x
// + i blockDim.x + j stride (i < run); returns how many live particles this
// thread pushed.
template <class R>
__device__ __forceinline__ double push_items(const Ctx<R> &X, unsigned long long first,
                                             unsigned long long last, unsigned long long stride,
                                             int run = 1) {
  const Dev<R> &D = X.d;
  const unsigned long long n = min(min(*D.nslots, D.cap), last);
  const int nx = D.nx, ny = D.ny, nz = D.nz;
  const R dl_inv[3] = {D.idx, D.idy, D.idz};
  const R c2inv = R(1.0 / (kC * kC));
  double pushed = 0.0;
  const uint32_t jstamp = D.jtouch[D.nz + 1] + 1u;  // the next field pass
  unsigned long long p = first + threadIdx.x;
  int ip = 0;  // place of p in its run
  const unsigned long long bd = blockDim.x, jump = stride - (unsigned long long)(run - 1) * bd;
  unsigned long long pn = 0;
  int ipn = 0;
  // each thread loads its next particle's state one iteration ahead, so that
  // round trip overlaps the current particle's gather and deposit
  int cell_n = -1;
  R off_n[3] = {R(0), R(0), R(0)}, u_n[3] = {R(0), R(0), R(0)};
  uint32_t tag_n = 0;
  if (p < n) {
    cell_n = D.pcell[p];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      off_n[d] = D.po[d][p];
      u_n[d] = D.pu[d][p];
    }
    tag_n = D.ptag[p];
  }
  for (; p < n; p = pn, ip = ipn) {
    // the thread's next slot: one block of threads on in the run, or the
    // start of the next run
    ipn = ip + 1 < run ? ip + 1 : 0;
    pn = ip + 1 < run ? p + bd : p + jump;
    const int cell = cell_n;
    R off[3] = {off_n[0], off_n[1], off_n[2]};
    R u[3] = {u_n[0], u_n[1], u_n[2]};
    const uint32_t tag = tag_n;
    if (pn < n) {
      const unsigned long long q = pn;
      cell_n = D.pcell[q];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        off_n[d] = D.po[d][q];
        u_n[d] = D.pu[d][q];
      }
      tag_n = D.ptag[q];
    }
    if (cell < 0) continue;
    pushed += 1.0;
    const int ci = cell % nx, t = cell / nx, cj = t % ny, ck = t / ny;
    const LayerR<R> &L = X.lr[tag >> 1];
    const int sp = tag & 1u;
    // shapes on the integer and half-integer grids; node offsets in elements
    R wi[3][3], wh[3][3];
    int xi[3], xh[3], yi[3], yh[3], zi[3], zh[3];
    {
      const int nxy = D.nxy;
      int b;
      shape_int(off[0], wi[0], b);
      shape_half(off[0], wh[0]);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        xi[a] = wrap(ci + b + a, nx);
        xh[a] = wrap(ci - 1 + a, nx);
      }
      shape_int(off[1], wi[1], b);
      shape_half(off[1], wh[1]);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        yi[a] = wrap(cj + b + a, ny) * nx;
        yh[a] = wrap(cj - 1 + a, ny) * nx;
      }
      shape_int(off[2], wi[2], b);
      shape_half(off[2], wh[2]);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        zi[a] = (ck + b + a) * nxy;
        zh[a] = (ck - 1 + a) * nxy;
      }
    }
    const R Ex = gather27(D.E[0], xh, yi, zi, wh[0], wi[1], wi[2]);
    const R Ey = gather27(D.E[1], xi, yh, zi, wi[0], wh[1], wi[2]);
    const R Ez = gather27(D.E[2], xi, yi, zh, wi[0], wi[1], wh[2]);
    const R Bx = gather27(D.B[0], xi, yh, zh, wi[0], wh[1], wh[2]);
    const R By = gather27(D.B[1], xh, yi, zh, wh[0], wi[1], wh[2]);
    const R Bz = gather27(D.B[2], xh, yh, zi, wh[0], wh[1], wi[2]);
    // relativistic Boris rotation between two half electric kicks
    const R h = L.qmdt2[sp];
    R um[3] = {u[0] + h * Ex, u[1] + h * Ey, u[2] + h * Ez};
    const R gm = sqrt(R(1) + (um[0] * um[0] + um[1] * um[1] + um[2] * um[2]) * c2inv);
    const R hg = h / gm;
    const R tv[3] = {hg * Bx, hg * By, hg * Bz};
    const R t2 = tv[0] * tv[0] + tv[1] * tv[1] + tv[2] * tv[2];
    const R sf = R(2) / (R(1) + t2);
    const R sv[3] = {sf * tv[0], sf * tv[1], sf * tv[2]};
    const R up[3] = {um[0] + (um[1] * tv[2] - um[2] * tv[1]), um[1] + (um[2] * tv[0] - um[0] * tv[2]),
                     um[2] + (um[0] * tv[1] - um[1] * tv[0])};
    u[0] = um[0] + (up[1] * sv[2] - up[2] * sv[1]) + h * Ex;
    u[1] = um[1] + (up[2] * sv[0] - up[0] * sv[2]) + h * Ey;
    u[2] = um[2] + (up[0] * sv[1] - up[1] * sv[0]) + h * Ez;
    const R g = sqrt(R(1) + (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) * c2inv);
    const R dtg = D.dt / g;
    const int co[3] = {ci, cj, ck};
    int cn[3];
    R on[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      R nd = off[d] + dtg * u[d] * dl_inv[d];
      int cc = co[d];
      if (nd < R(0)) {
        nd += R(1);
        cc -= 1;
      }
      if (nd >= R(1)) {
        nd -= R(1);
        cc += 1;
      }
      cn[d] = cc;
      on[d] = nd;
    }
    // the frame reaches node planes ck - 2 .. ck + 3: mark ck for k_efull
    if (D.jtouch[ck] != jstamp) D.jtouch[ck] = jstamp;
    esirkepov(D, L.jpref[sp], co, off, cn, on);
    const int ni = wrap(cn[0], nx), nj = wrap(cn[1], ny);
    if (cn[2] < 2 || cn[2] >= nz - 2 || pml_point(D, ni, nj)) {
      D.pcell[p] = -1;  // outflow through a z face or into an absorbing layer
      continue;
    }
    D.pcell[p] = (cn[2] * ny + nj) * nx + ni;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      D.po[d][p] = on[d];
      D.pu[d][p] = u[d];
    }
  }
  return pushed;
}

template <class R>
__global__ void __launch_bounds__(256, PushOcc<R>::v) k_push(Ctx<R> X) {
  // runs of kPushRun blocks of consecutive slots of the cell-sorted pool, a
  // grid of runs apart: a block's particles stay in a compact region for a
  // few iterations, so its gathers reuse field lines in L1
  const unsigned long long run = (unsigned long long)kPushRun * blockDim.x;
  const double pushed = push_items(X, blockIdx.x * run, ~0ull, gridDim.x * run, kPushRun);
  const double tot = block_sum<R>(pushed);
  if (threadIdx.x == 0 && tot != 0.0) atomicAdd(X.d.acc + 4, tot);
}

// ---------------------------------------------------------------------------
// Fields
// ---------------------------------------------------------------------------
// Points per thread of the field and window kernels: V consecutive x points
// of one row.  V = 4 (FP32, nx a multiple of 4) moves them with 16-byte
// vector loads and stores; the launch is (row chunks, z planes).
template <int V, class R>
__device__ __forceinline__ void ldv(R *d, const R *p) {
  if constexpr (V == 4 && sizeof(R) == 4) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    d[0] = v.x;
    d[1] = v.y;
    d[2] = v.z;
    d[3] = v.w;
  } else {
#pragma unroll
    for (int l = 0; l < V; ++l) d[l] = p[l];
  }
}
template <int V, class R>
__device__ __forceinline__ void stv(R *p, const R *d) {
  if constexpr (V == 4 && sizeof(R) == 4) {
    *reinterpret_cast<float4 *>(p) = make_float4(d[0], d[1], d[2], d[3]);
  } else {
#pragma unroll
    for (int l = 0; l < V; ++l) p[l] = d[l];
  }
}

// Fold |E|^2 / E0^2 at the V cell centres from point o into the intensity
// map: each component is the mean of its four edge values around the centre.
// Kept out of line and reloading its operands so that the B half step it is
// called from keeps close to the register count (and occupancy) of the plain
// step.
template <int V, class R>
__device__ __noinline__ void record_intensity(const R *ex0, const R *ey0, const R *ez0, R *imax,
                                              long long o, long long oj, long long ov,
                                              long long ojv, int nxy, R inv_e0sq) {
  R a[V], b[V], c[V], d[V], a2[V];
  ldv<V>(a, ex0 + o);
  ldv<V>(b, ex0 + oj);
  ldv<V>(c, ex0 + o + nxy);
  ldv<V>(d, ex0 + oj + nxy);
#pragma unroll
  for (int l = 0; l < V; ++l) {
    const R ax = R(0.25) * (((a[l] + b[l]) + c[l]) + d[l]);
    a2[l] = ax * ax;
  }
  R e[V + 1], f[V + 1];
  ldv<V>(e, ey0 + o);
  e[V] = ey0[ov];
  ldv<V>(f, ey0 + o + nxy);
  f[V] = ey0[ov + nxy];
#pragma unroll
  for (int l = 0; l < V; ++l) {
    const R ay = R(0.25) * (((e[l] + e[l + 1]) + f[l]) + f[l + 1]);
    a2[l] += ay * ay;
  }
  ldv<V>(e, ez0 + o);
  e[V] = ez0[ov];
  ldv<V>(f, ez0 + oj);
  f[V] = ez0[ojv];
#pragma unroll
  for (int l = 0; l < V; ++l) {
    const R az = R(0.25) * (((e[l] + e[l + 1]) + f[l]) + f[l + 1]);
    a2[l] = (a2[l] + az * az) * inv_e0sq;
  }
  R *const cell = imax + o;
  ldv<V>(a, cell);
#pragma unroll
  for (int l = 0; l < V; ++l) a[l] = fmax(a[l], a2[l]);
  stv<V>(cell, a);
}

// Faraday half steps on V points of plane blockIdx.y, t = curl E / 2 dt.
// Both half steps of B around the particle phase use the same E: the one
// after the E update (B^{n+1} = B^{n+1/2} - t) and the one that opens the
// next step (B^{n+3/2} = B^{n+1} - t).  So a field pass keeps B at integer
// time (read by the push and the diagnostics) and Bh at the next half time
// (read by the E update), and kFull computes both from Bh and E^{n+1} in one
// pass, each rounded as two separate half steps would be.  kPrime sets Bh =
// B - t from the current B and E (at creation, and after the host has
// written the fields).  kRecord (with kFull): on the steps where the
// intensity map is recorded, also fold |E^{n+1}|^2 / E0^2 at the V cell
// centres into it.
enum { kPrime = 0, kFull = 1, kFullRecord = 2 };

// t1 is the curl term of the first half step, t2 of the second (they differ
// only inside the absorbing layers).
template <int V, int kMode, class R>
__device__ __forceinline__ void b_out(const Dev<R> &D, int d, long long o, const R *t1,
                                      const R *t2) {
  const R h = R(0.5) * D.dt;
  R b[V];
  ldv<V>(b, (kMode == kPrime ? D.B[d] : D.Bh[d]) + o);
#pragma unroll
  for (int l = 0; l < V; ++l) b[l] -= h * t1[l];
  if constexpr (kMode == kPrime) {
    stv<V>(D.Bh[d] + o, b);
  } else {
    stv<V>(D.B[d] + o, b);
#pragma unroll
    for (int l = 0; l < V; ++l) b[l] -= h * t2[l];
    stv<V>(D.Bh[d] + o, b);
  }
}

template <int V, int kMode, bool kLay = false, class R>
__device__ __forceinline__ void bstep_body(const Dev<R> &D, Blk bk) {
  const int nx = D.nx, ny = D.ny, nxy = D.nxy;
  // the E step of this pass has read the current: count the pass and clear
  // the host-write flag
  if (kMode != kPrime && bk.x == 0 && bk.y == 0 && threadIdx.x == 0) {
    D.jtouch[D.nz + 1] += 1u;
    D.jtouch[D.nz] = 0u;
  }
  const int r = (bk.x * blockDim.x + threadIdx.x) * V;
  if (r >= nxy) return;
  const int k = bk.y;
  const int j = r / nx, i = r - j * nx;
  const long long o = (long long)k * nxy + r;
  const long long oj = (j == ny - 1) ? o - (long long)(ny - 1) * nx : o + nx;
  const long long ov = (i + V == nx) ? o + V - nx : o + V;  // x + 1 of the last point
  R ex[V], ey[V + 1], exj[V], t[V], t2[V];
  ldv<V>(ex, D.E[0] + o);
  ldv<V>(ey, D.E[1] + o);
  ey[V] = D.E[1][ov];
  ldv<V>(exj, D.E[0] + oj);
  // a thread with a point in the absorbing layers takes the layer terms
  // (kLay: instantiated for grids that have them)
  const bool lay = kLay && (pml_point(D, i, j) || pml_point(D, i + V - 1, j));
#pragma unroll
  for (int l = 0; l < V; ++l) t[l] = (ey[l + 1] - ey[l]) * D.idx - (exj[l] - ex[l]) * D.idy;
  if (lay) {
#pragma unroll
    for (int l = 0; l < V; ++l) {
      t2[l] = t[l];
      if (pml_point(D, i + l, j)) {
        R x1, x2, y1, y2;
        pml_two<kMode>(D.psi[kPsiBZX] + o + l, D.psi_close[kPsiBZX - kPsiBYX] + o + l,
                       D.pml_bB[0][i + l], (ey[l + 1] - ey[l]) * D.idx, x1, x2);
        pml_two<kMode>(D.psi[kPsiBZY] + o + l, D.psi_close[kPsiBZY - kPsiBYX] + o + l,
                       D.pml_bB[1][j], (exj[l] - ex[l]) * D.idy, y1, y2);
        t[l] = x1 - y1;
        t2[l] = x2 - y2;
      }
    }
    b_out<V, kMode>(D, 2, o, t, t2);
  } else {
    b_out<V, kMode>(D, 2, o, t, t);
  }
  if (k < D.nz) {
    R ez[V + 1], ezj[V], eyk[V], exk[V];
    ldv<V>(ez, D.E[2] + o);
    ez[V] = D.E[2][ov];
    ldv<V>(ezj, D.E[2] + oj);
    ldv<V>(eyk, D.E[1] + o + nxy);
    ldv<V>(exk, D.E[0] + o + nxy);
#pragma unroll
    for (int l = 0; l < V; ++l) t[l] = (ezj[l] - ez[l]) * D.idy - (eyk[l] - ey[l]) * D.idz;
    if (lay) {
#pragma unroll
      for (int l = 0; l < V; ++l) {
        t2[l] = t[l];
        if (pml_point(D, i + l, j)) {
          R y1, y2;
          pml_two<kMode>(D.psi[kPsiBXY] + o + l, D.psi_close[kPsiBXY - kPsiBYX] + o + l,
                         D.pml_bB[1][j], (ezj[l] - ez[l]) * D.idy, y1, y2);
          const R dz = (eyk[l] - ey[l]) * D.idz;
          t[l] = y1 - dz;
          t2[l] = y2 - dz;
        }
      }
      b_out<V, kMode>(D, 0, o, t, t2);
    } else {
      b_out<V, kMode>(D, 0, o, t, t);
    }
#pragma unroll
    for (int l = 0; l < V; ++l) t[l] = (exk[l] - ex[l]) * D.idz - (ez[l + 1] - ez[l]) * D.idx;
    if (lay) {
#pragma unroll
      for (int l = 0; l < V; ++l) {
        t2[l] = t[l];
        if (pml_point(D, i + l, j)) {
          R x1, x2;
          pml_two<kMode>(D.psi[kPsiBYX] + o + l, D.psi_close[0] + o + l, D.pml_bB[0][i + l],
                         (ez[l + 1] - ez[l]) * D.idx, x1, x2);
          const R dz = (exk[l] - ex[l]) * D.idz;
          t[l] = dz - x1;
          t2[l] = dz - x2;
        }
      }
      b_out<V, kMode>(D, 1, o, t, t2);
    } else {
      b_out<V, kMode>(D, 1, o, t, t);
    }
    if constexpr (kMode == kFullRecord) {
      const int every = D.imax_every;
      if (every > 0 && ((unsigned)*D.step + 1u) % (unsigned)every == 0u)
        record_intensity<V, R>(D.E[0], D.E[1], D.E[2], D.imax, o, oj, ov,
                               (i + V == nx) ? oj + V - nx : oj + V, nxy, D.inv_e0sq);
    }
  }
}

template <int V, int kMode, class R, bool kLay = false>
__global__ void __launch_bounds__(256) k_bstep(Dev<R> D) {
  bstep_body<V, kMode, kLay>(D, blk_here());
}

template <class R>
__device__ __forceinline__ R block_sum_r(R v) {
  __shared__ R part_r[32];
#pragma unroll
  for (int sft = 16; sft > 0; sft >>= 1) v += __shfl_xor_sync(0xffffffffu, v, sft);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) part_r[w] = v;
  __syncthreads();
  R tot = R(0);
  if (threadIdx.x == 0)
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tot += part_r[q];
  return tot;
}

__device__ __forceinline__ void load_j3(const float *j4, float &a, float &b, float &c) {
  const float4 v = *reinterpret_cast<const float4 *>(j4);
  a = v.x;
  b = v.y;
  c = v.z;
}
__device__ __forceinline__ void load_j3(const double *j4, double &a, double &b, double &c) {
  const double2 v = *reinterpret_cast<const double2 *>(j4);
  a = v.x;
  b = v.y;
  c = j4[2];
}
__device__ __forceinline__ void clear_j3(float *j4) {
  *reinterpret_cast<float4 *>(j4) = make_float4(0.f, 0.f, 0.f, 0.f);
}
__device__ __forceinline__ void clear_j3(double *j4) {
  reinterpret_cast<double2 *>(j4)[0] = make_double2(0.0, 0.0);
  j4[2] = 0.0;
}

template <class R>
__device__ __forceinline__ R e_point(const LayerR<R> &L, R e0, R a, R &p, R &q) {
  R dp;
  if (L.is_static) {
    dp = (R(2) * (L.deps * e0 - p) + L.deps * a) * L.inv_den;
    q = R(0);
  } else {
    // trapezoidal oscillator coupled implicitly to E^{n+1}
    dp = (L.cn_g * q + L.cn_a * (L.deps * e0 - p) + L.cn_b * a) * L.inv_den;
    q = L.two_over_h * dp - q;
  }
  p += dp;
  return e0 + a - dp;
}

// E step on V points of plane blockIdx.y: Ampere with B^{n+1/2} (Bh), J and
// the polarisation current, Silver-Mueller faces at k = 0 (with the incident field) and k = nz,
// Joule work J.(E^n + E^{n+1})/2, J cleared for the next deposit.  Three
// blocks per SM (80 registers) measured faster than two at 100 registers.
// kPlanes: 0 every node plane (k = bk.y); 1 the interior planes without
// material (D.vplane[bk.y]); 2 the material planes (D.kplane[bk.y]); 3 the
// two faces (bk.y 0: k = 0, 1: k = nz).  Each compiles only the code its
// planes need (face boundary and laser source, polarisation).
template <int V, bool kLay = false, int kPlanes = 0, class R>
__device__ __forceinline__ void efull_body(const Ctx<R> &X, Blk bk) {
  const Dev<R> &D = X.d;
  const int nx = D.nx, ny = D.ny, nz = D.nz, nxy = D.nxy;
  const int r = (bk.x * blockDim.x + threadIdx.x) * V;
  constexpr bool kFaces = kPlanes == 0 || kPlanes == 3;
  constexpr bool kMaterial = kPlanes == 0 || kPlanes == 2;
  const int k = kPlanes == 0   ? bk.y
                : kPlanes == 1 ? D.vplane[bk.y]
                : kPlanes == 2 ? D.kplane[bk.y]
                               : (bk.y == 0 ? 0 : D.nz);
  // the current is nonzero only on node planes within reach of a particle
  // deposited since the last field pass (cell planes k - 3 .. k + 2) or
  // after a host write
  bool jt = D.jtouch[nz] != 0u;
  {
    const uint32_t jstamp = D.jtouch[nz + 1] + 1u;  // this pass
    for (int q = max(0, k - 3); q <= min(nz - 1, k + 2); ++q) jt |= D.jtouch[q] == jstamp;
  }
  R joule = R(0);
  if (r < nxy) {
    const int j = r / nx, i = r - j * nx;
    const long long o = (long long)k * nxy + r;
    const long long omv = (i == 0) ? o + (nx - 1) : o - 1;  // x - 1 of the first point
    const long long omj = (j == 0) ? o + (long long)(ny - 1) * nx : o - nx;
    const R c2dt = D.c2dt, dtie = R(D.dt_d / kEps0);
    // bz[0] is the x - 1 neighbour of the first point, bz[1..V] the points
    R bz[V + 1], bzj[V], bx[V], by[V];
    bz[0] = D.Bh[2][omv];
    ldv<V>(bz + 1, D.Bh[2] + o);
    ldv<V>(bzj, D.Bh[2] + omj);
    ldv<V>(bx, D.Bh[0] + o);
    ldv<V>(by, D.Bh[1] + o);
    R jx[V], jy[V], jz[V];
    if (jt) {
#pragma unroll
      for (int l = 0; l < V; ++l) load_j3(D.J4 + 4 * (o + l), jx[l], jy[l], jz[l]);
    } else {
#pragma unroll
      for (int l = 0; l < V; ++l) jx[l] = jy[l] = jz[l] = R(0);
    }
    R ex0[V], ey0[V], ex1[V], ey1[V], dBz_dy[V], dBz_dx[V];
    ldv<V>(ex0, D.E[0] + o);
    ldv<V>(ey0, D.E[1] + o);
#pragma unroll
    for (int l = 0; l < V; ++l) {
      dBz_dy[l] = (bz[l + 1] - bzj[l]) * D.idy;
      dBz_dx[l] = (bz[l + 1] - bz[l]) * D.idx;
    }
    // absorbing layers: the convolution terms of the x and y derivatives
    const bool lay = kLay && (pml_point(D, i, j) || pml_point(D, i + V - 1, j));
    if (lay) {
#pragma unroll
      for (int l = 0; l < V; ++l)
        if (pml_point(D, i + l, j)) {
          dBz_dy[l] = pml_step(D.psi[kPsiEXY] + o + l, D.pml_bE[1][j], dBz_dy[l]);
          dBz_dx[l] = pml_step(D.psi[kPsiEYX] + o + l, D.pml_bE[0][i + l], dBz_dx[l]);
        }
    }
    const int L = (kMaterial && k < nz) ? D.layer_of_plane[k] : -1;
    const long long m = L >= 0 ? (long long)D.mplane[k] * nxy + r : -1;
    if (kFaces && (k == 0 || k == nz)) {
      const R al = D.alpha, cc = R(kC);
      const R inv = R(1) / (R(1) + al);
      if (k == 0) {
        // incident field at t^{n+1/2}, computed in double: Gaussian or
        // sine-squared envelope, times the spot profile at the polarised
        // component's node (Ex at ((i + 1/2) dx, j dy), Ey at (i dx, (j + 1/2) dy))
        const double t = ((double)(*D.step) + 0.5) * D.dt_d - D.t_peak;
        double env;
        if (D.shape == 1) {
          const double x = kPi * t / D.Tsin2;
          env = fabs(t) < 0.5 * D.Tsin2 ? cos(x) * cos(x) : 0.0;
        } else {
          env = exp(-2.0 * 0.69314718055994531 * t * t / (D.fwhm * D.fwhm));
        }
        const double einc = D.E0 * env * cos(D.omega * t + D.cep);
#pragma unroll
        for (int l = 0; l < V; ++l) {
          double sp = 1.0;
          if (D.w0 > 0.0) {
            const double x = (i + l + (D.pol == 0 ? 0.5 : 0.0)) * D.dx_d - D.xc;
            const double y = (j + (D.pol == 0 ? 0.0 : 0.5)) * D.dy_d - D.yc;
            sp = exp(-(x * x + y * y) / (D.w0 * D.w0));
          }
          const R exi = D.pol == 0 ? R(einc * sp) : R(0), eyi = D.pol == 0 ? R(0) : R(einc * sp);
          ex1[l] = ((R(1) - al) * ex0[l] - R(2) * al * cc * by[l] + R(4) * al * exi +
                    (c2dt * dBz_dy[l] - dtie * jx[l])) * inv;
          ey1[l] = ((R(1) - al) * ey0[l] + R(2) * al * cc * bx[l] + R(4) * al * eyi -
                    (c2dt * dBz_dx[l] + dtie * jy[l])) * inv;
        }
      } else {
        R bxm[V], bym[V];
        ldv<V>(bxm, D.Bh[0] + o - nxy);
        ldv<V>(bym, D.Bh[1] + o - nxy);
#pragma unroll
        for (int l = 0; l < V; ++l) {
          ex1[l] = ((R(1) - al) * ex0[l] + R(2) * al * cc * bym[l] +
                    (c2dt * dBz_dy[l] - dtie * jx[l])) * inv;
          ey1[l] = ((R(1) - al) * ey0[l] - R(2) * al * cc * bxm[l] -
                    (c2dt * dBz_dx[l] + dtie * jy[l])) * inv;
        }
      }
    } else {
      R bxm[V], bym[V], ax[V], ay[V];
      ldv<V>(bxm, D.Bh[0] + o - nxy);
      ldv<V>(bym, D.Bh[1] + o - nxy);
#pragma unroll
      for (int l = 0; l < V; ++l) {
        ax[l] = c2dt * (dBz_dy[l] - (by[l] - bym[l]) * D.idz) - dtie * jx[l];
        ay[l] = c2dt * ((bx[l] - bxm[l]) * D.idz - dBz_dx[l]) - dtie * jy[l];
      }
      if (m >= 0) {
        const LayerR<R> &Ly = X.lr[L];
        R px[V], qx[V], py[V], qy[V];
        ldv<V>(px, D.P[0] + m);
        ldv<V>(qx, D.Q[0] + m);
        ldv<V>(py, D.P[1] + m);
        ldv<V>(qy, D.Q[1] + m);
#pragma unroll
        for (int l = 0; l < V; ++l) {
          ex1[l] = e_point(Ly, ex0[l], ax[l], px[l], qx[l]);
          ey1[l] = e_point(Ly, ey0[l], ay[l], py[l], qy[l]);
        }
        stv<V>(D.P[0] + m, px);
        stv<V>(D.Q[0] + m, qx);
        stv<V>(D.P[1] + m, py);
        stv<V>(D.Q[1] + m, qy);
      } else {
#pragma unroll
        for (int l = 0; l < V; ++l) {
          ex1[l] = ex0[l] + ax[l];
          ey1[l] = ey0[l] + ay[l];
        }
      }
    }
#pragma unroll
    for (int l = 0; l < V; ++l) {
      joule += jx[l] * R(0.5) * (ex0[l] + ex1[l]) + jy[l] * R(0.5) * (ey0[l] + ey1[l]);
      if (jt) clear_j3(D.J4 + 4 * (o + l));
    }
    stv<V>(D.E[0] + o, ex1);
    stv<V>(D.E[1] + o, ey1);
    if (k < nz) {
      R bxj[V], ez0[V], ez1[V], az[V];
      const R byp = D.Bh[1][omv];
      ldv<V>(bxj, D.Bh[0] + omj);
      ldv<V>(ez0, D.E[2] + o);
      R dby_dx[V], dbx_dy[V];
#pragma unroll
      for (int l = 0; l < V; ++l) {
        dby_dx[l] = (by[l] - (l ? by[l - 1] : byp)) * D.idx;
        dbx_dy[l] = (bx[l] - bxj[l]) * D.idy;
      }
      if (lay) {
#pragma unroll
        for (int l = 0; l < V; ++l)
          if (pml_point(D, i + l, j)) {
            dby_dx[l] = pml_step(D.psi[kPsiEZX] + o + l, D.pml_bE[0][i + l], dby_dx[l]);
            dbx_dy[l] = pml_step(D.psi[kPsiEZY] + o + l, D.pml_bE[1][j], dbx_dy[l]);
          }
      }
#pragma unroll
      for (int l = 0; l < V; ++l) az[l] = c2dt * (dby_dx[l] - dbx_dy[l]) - dtie * jz[l];
      if (m >= 0) {
        R pz[V], qz[V];
        ldv<V>(pz, D.P[2] + m);
        ldv<V>(qz, D.Q[2] + m);
#pragma unroll
        for (int l = 0; l < V; ++l) ez1[l] = e_point(X.lr[L], ez0[l], az[l], pz[l], qz[l]);
        stv<V>(D.P[2] + m, pz);
        stv<V>(D.Q[2] + m, qz);
      } else {
#pragma unroll
        for (int l = 0; l < V; ++l) ez1[l] = ez0[l] + az[l];
      }
#pragma unroll
      for (int l = 0; l < V; ++l) joule += jz[l] * R(0.5) * (ez0[l] + ez1[l]);
      stv<V>(D.E[2] + o, ez1);
    }
  }
  // Joule work: block sum in the working precision, one FP64 atomic per block
  const R tot = block_sum_r(joule);
  if (threadIdx.x == 0 && tot != R(0)) atomicAdd(D.acc + 0, (double)tot * D.dt_d * D.V_d);
}

template <int V, class R, bool kLay = false, int kPlanes = 0>
__global__ void __launch_bounds__(256, kPlanes == 1 ? 4 : 3) k_efull(Ctx<R> X) {
  efull_body<V, kLay, kPlanes>(X, blk_here());
}

// ---------------------------------------------------------------------------
// Amplitude window + Keldysh threshold, one thread per material cell
// ---------------------------------------------------------------------------
template <int V, class R>
__device__ __forceinline__ void window_body(const Ctx<R> &X, Blk bk) {
  const Dev<R> &D = X.d;
  const int nx = D.nx, ny = D.ny, nxy = D.nxy;
  const int r = (bk.x * blockDim.x + threadIdx.x) * V;
  const int mp = bk.y;
  const long long m = (long long)mp * nxy + r;
  uint32_t miss = 0;  // cells whose threshold k_keldysh must recompute
  bool hot = false;   // a cell at or above the skip amplitude
  if (r < nxy) {
    const int j = r / nx, i = r - j * nx;
    const int k = D.kplane[mp];
    const long long o = (long long)k * nxy + r;
    const long long oj = (j == ny - 1) ? o - (long long)(ny - 1) * nx : o + nx;
    const long long ov = (i + V == nx) ? o + V - nx : o + V;     // x + 1 of the last point
    const long long ojv = (i + V == nx) ? oj + V - nx : oj + V;  // and one row up
    // cell-centred amplitude: mean of the four edge values of each component
    R ex[V], exj[V], exk[V], exjk[V], ey[V + 1], eyk[V + 1], ez[V + 1], ezj[V + 1];
    ldv<V>(ex, D.E[0] + o);
    ldv<V>(exj, D.E[0] + oj);
    ldv<V>(exk, D.E[0] + o + nxy);
    ldv<V>(exjk, D.E[0] + oj + nxy);
    ldv<V>(ey, D.E[1] + o);
    ey[V] = D.E[1][ov];
    ldv<V>(eyk, D.E[1] + o + nxy);
    eyk[V] = D.E[1][ov + nxy];
    ldv<V>(ez, D.E[2] + o);
    ez[V] = D.E[2][ov];
    ldv<V>(ezj, D.E[2] + oj);
    ezj[V] = D.E[2][ojv];
    R a[V];
#pragma unroll
    for (int l = 0; l < V; ++l) {
      const R ax = R(0.25) * (((ex[l] + exj[l]) + exk[l]) + exjk[l]);
      const R ay = R(0.25) * (((ey[l] + ey[l + 1]) + eyk[l]) + eyk[l + 1]);
      const R az = R(0.25) * (((ez[l] + ez[l + 1]) + ezj[l]) + ezj[l + 1]);
      a[l] = sqrt(ax * ax + ay * ay + az * az);
    }
    // sliding maximum: slots <= s hold this block's samples, slots > s the
    // suffix maxima of the previous block; pm is the running block prefix max
    const int NW = D.NW;
    const int s = (int)((unsigned)*D.step % (unsigned)NW);
    R *__restrict__ W = D.win + m;
    const long long st = D.nmat;
    stv<V>(W + s * st, a);
    R pm[V], amp[V];
    if (s == 0) {
#pragma unroll
      for (int l = 0; l < V; ++l) pm[l] = a[l];
    } else {
      ldv<V>(pm, D.pm + m);
#pragma unroll
      for (int l = 0; l < V; ++l) pm[l] = fmax(pm[l], a[l]);
    }
    stv<V>(D.pm + m, pm);
    if (s + 1 < NW) {
      ldv<V>(amp, W + (s + 1) * st);
#pragma unroll
      for (int l = 0; l < V; ++l) amp[l] = fmax(pm[l], amp[l]);
    } else {
#pragma unroll
      for (int l = 0; l < V; ++l) amp[l] = pm[l];
    }
    if (s == NW - 1) {
      R run[V], w[V];
#pragma unroll
      for (int l = 0; l < V; ++l) run[l] = a[l];
      for (int q = NW - 2; q >= 0; --q) {
        ldv<V>(w, W + q * st);
#pragma unroll
        for (int l = 0; l < V; ++l) run[l] = fmax(run[l], w[l]);
        stv<V>(W + q * st, run);
      }
    }
    stv<V>(D.eamp + m, amp);
    R key[V];
    ldv<V>(key, D.ckey + m);
    const R e_skip = X.lr[D.layer_of_plane[k]].e_skip;
#pragma unroll
    for (int l = 0; l < V; ++l) {
      hot |= amp[l] >= e_skip;
      if (key[l] == amp[l]) continue;  // threshold cached for this exact amplitude
      if (!(amp[l] >= e_skip)) {
        D.T[m + l] = 0ull;
        D.ckey[m + l] = amp[l];
      } else {
        miss |= 1u << l;
      }
    }
  }
  // stamp the plane for k_ionize, which skips planes without such cells
  if (__syncthreads_or(hot) && threadIdx.x == 0) D.hot[mp] = (uint32_t)*D.step + 1u;
  if (threadIdx.x == 0 && bk.x == 0 && mp == 0) D.hot[bk.gy] = (uint32_t)*D.step + 1u;
  // warp-aggregated append of the misses to k_keldysh's work list
  const int cnt = __popc(miss);
  int incl = cnt;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int sft = 1; sft < 32; sft <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, sft);
    if (lane >= sft) incl += v;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  int base = 0;
  if (lane == 31 && total) base = atomicAdd(X.work_n, total);
  base = __shfl_sync(0xffffffffu, base, 31) + incl - cnt;
  for (; miss; miss &= miss - 1) X.work[base++] = (int)(m + __ffs(miss) - 1);
}

template <int V, class R>
__global__ void __launch_bounds__(256) k_window(Ctx<R> X) {
  window_body<V>(X, blk_here());
}

// Keldysh thresholds of the queued cells, one thread per cell: queue
// entries q = first + threadIdx.x + j stride below last.
template <class R>
__device__ __forceinline__ void keldysh_items(const Ctx<R> &X, int first, int last, int stride) {
  const Dev<R> &D = X.d;
  for (int q = first + threadIdx.x; q < last; q += stride) {
    const long long m = X.work[q];
    const int k = D.kplane[(int)(m / D.nxy)];
    const R amp = D.eamp[m];
    D.T[m] = keldysh_threshold<R>(amp, D.layers[D.layer_of_plane[k]], D.keldysh_terms, nullptr,
                                  D.ktab, D.ntab);
    D.ckey[m] = amp;
  }
}

template <class R>
__global__ void __launch_bounds__(256) k_keldysh(Ctx<R> X) {
  keldysh_items(X, blockIdx.x * blockDim.x, *X.work_n, gridDim.x * blockDim.x);
}

// ---------------------------------------------------------------------------
// Ionisation: one thread per material (birth) cell.  A neutral is force-free,
// at x0 + v0 t with x0, v0 regenerated from Philox; it is drawn against the
// threshold of the cell it occupies at t^{n+1}.  k_init_material computes
// from each neutral's own x0, v0 the step before which it cannot have crossed
// a face (with a margin for the rounding of the run-time position), so until
// then the birth cell's threshold decides without regenerating any state.
// ---------------------------------------------------------------------------
template <class R>
struct Neutral {
  int cell[3];
  R off[3];
  R u[3];
};

template <class R>
__device__ __forceinline__ void neutral_pos(const Dev<R> &D, uint32_t c, uint32_t s, R off0[3]) {
  const uint4 w = draw(D.seed, 0u, c, s, kStreamPos);
  const R top = R(1) - Eps<R>::v();
  off0[0] = fmin(unit_open<R>(w.x), top);
  off0[1] = fmin(unit_open<R>(w.y), top);
  off0[2] = fmin(unit_open<R>(w.z), top);
}

template <class R>
__device__ __forceinline__ void neutral_vel(const Dev<R> &D, R sig, uint32_t c, uint32_t s, R v[3]) {
  const uint4 w = draw(D.seed, 0u, c, s, kStreamVel);
  const R r1 = sqrt(R(-2) * log(unit_open<R>(w.x)));
  const R r2 = sqrt(R(-2) * log(unit_open<R>(w.z)));
  R s1, c1, s2, c2;
  sincospi(R(2) * unit_open<R>(w.y), &s1, &c1);
  sincospi(R(2) * unit_open<R>(w.w), &s2, &c2);
  v[0] = sig * r1 * c1;
  v[1] = sig * r1 * s1;
  v[2] = sig * r2 * c2;
}

// Position at time t of neutral (c, s) born in cell (i, j, k); false if it
// left the grid along z.
template <class R>
__device__ __forceinline__ bool neutral_at(const Dev<R> &D, R sig, int i, int j, int k, uint32_t c,
                                           uint32_t s, R t, Neutral<R> &nu) {
  R off0[3], v[3];
  neutral_pos(D, c, s, off0);
  neutral_vel(D, sig, c, s, v);
  const R il[3] = {D.idx, D.idy, D.idz};
  int cc[3] = {i, j, k};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    R nd = off0[d] + v[d] * t * il[d];
    if (nd < R(0)) {
      nd += R(1);
      cc[d] -= 1;
    }
    if (nd >= R(1)) {
      nd -= R(1);
      cc[d] += 1;
    }
    nu.off[d] = nd;
  }
  nu.cell[0] = wrap(cc[0], D.nx);
  nu.cell[1] = wrap(cc[1], D.ny);
  nu.cell[2] = cc[2];
  const R v2 = (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) * R(1.0 / (kC * kC));
  const R gm = R(1) / sqrt(R(1) - v2);
  nu.u[0] = gm * v[0];
  nu.u[1] = gm * v[1];
  nu.u[2] = gm * v[2];
  return cc[2] >= 0 && cc[2] < D.nz;
}

template <class R>
__device__ __forceinline__ unsigned long long threshold_at(const Dev<R> &D, int i, int j, int k) {
  if (k < 0 || k >= D.nz) return 0ull;
  const int mp = D.mplane[k];
  if (mp < 0) return 0ull;
  return D.T[(long long)mp * D.nxy + (long long)j * D.nx + i];
}

// A neutral in slot s ionises when its 64-bit uniform (h16 << 48 | lo48) is
// below T = floor(p 2^64) (T = ~0: always).  h16 is the 16-bit half
// (s & 1: high) of word (s & 7) >> 1 of the block (step, cell, s >> 3, 3),
// shared by eight slots; lo48 comes from the block (step, cell, s, 4), drawn
// only when h16 equals the top 16 bits of T (otherwise those decide), which
// happens once in 2^16 draws.
__device__ __forceinline__ uint32_t ion_h16(const uint4 &w, uint32_t s) {
  const uint32_t q = (s & 7u) >> 1;
  const uint32_t v = q == 0 ? w.x : (q == 1 ? w.y : (q == 2 ? w.z : w.w));
  return (s & 1u) ? (v >> 16) : (v & 0xFFFFu);
}
__device__ __forceinline__ bool ionises(uint32_t h16, unsigned long long T, unsigned long long seed,
                                        uint32_t step, uint32_t cell, uint32_t s) {
  if (T == ~0ull) return true;
  const uint32_t th = (uint32_t)(T >> 48);
  if (h16 != th) return h16 < th;
  const uint4 b = draw(seed, step, cell, s, kStreamIonLow);
  const unsigned long long lo48 = ((unsigned long long)(b.y & 0xFFFFu) << 32) | b.x;
  return lo48 < (T & 0xFFFFFFFFFFFFull);
}

// The eight 16-bit halves of one block against the top 16 bits th of a
// threshold: bit t of *lt is set when slot 8g + t is decided (below), of *eq
// when its low 48 bits must decide.
__device__ __forceinline__ void ion_compare8(const uint4 &w, uint32_t th, uint32_t &lt,
                                             uint32_t &eq) {
  lt = 0;
  eq = 0;
  // nearly every block has all eight halves above th: their minimum says so
  // in a few instructions, before any per-slot comparison
  const uint32_t m2 = __vminu2(__vminu2(w.x, w.y), __vminu2(w.z, w.w));
  if (min(m2 & 0xFFFFu, m2 >> 16) > th) return;
  // two halves per instruction: __vcmpltu2 / __vcmpeq2 set a halfword to
  // 0xFFFF where the unsigned comparison holds
  const uint32_t v[4] = {w.x, w.y, w.z, w.w};
  const uint32_t th2 = th | (th << 16);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint32_t l = __vcmpltu2(v[q], th2), e = __vcmpeq2(v[q], th2);
    lt |= ((l & 1u) | ((l >> 15) & 2u)) << (2 * q);
    eq |= ((e & 1u) | ((e >> 15) & 2u)) << (2 * q);
  }
}

// Decisions for the neutrals of cell (i, j, k) in the bits of exc, which
// may have crossed a face: exact position at t^{n+1}, threshold of the cell
// it is in.
template <class R>
__device__ __forceinline__ uint32_t ion_exc(const Dev<R> &D, R sig, int i, int j, int k,
                                            uint32_t c, uint32_t exc, uint32_t step, R t1) {
  uint32_t ion = 0;
  for (uint32_t bits = exc; bits; bits &= bits - 1) {
    const uint32_t s = __ffs(bits) - 1;
    Neutral<R> nu;
    const unsigned long long Tuse = neutral_at(D, sig, i, j, k, c, s, t1, nu)
                                        ? threshold_at(D, nu.cell[0], nu.cell[1], nu.cell[2])
                                        : 0ull;
    if (Tuse == 0ull) continue;
    const uint4 w = draw(D.seed, step, c, s >> 3, kStreamIon);
    if (ionises(ion_h16(w, s), Tuse, D.seed, step, c, s)) ion |= 1u << s;
  }
  return ion;
}

// Electron + hole for each neutral in the bits of ion of cell r of the
// plane (material index m, alive word alive): pool slots reserved once per
// warp (every lane of the warp calls this; most warps ionise nothing).
template <class R>
__device__ __forceinline__ void ion_append(const Ctx<R> &X, long long m, int r, int k, int L,
                                           uint32_t c, uint32_t alive, uint32_t ion, R t1) {
  const Dev<R> &D = X.d;
  if (__ballot_sync(0xffffffffu, ion != 0u) == 0u) return;
  const int npair = __popc(ion);
  int incl = npair;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int sft = 1; sft < 32; sft <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, sft);
    if (lane >= sft) incl += v;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  unsigned long long basew = 0;
  if (lane == 31 && total) basew = atomicAdd(D.nslots, 2ull * (unsigned long long)total);
  basew = __shfl_sync(0xffffffffu, basew, 31);
  if (!npair) return;
  const int j = r / D.nx, i = r - j * D.nx;
  unsigned long long slot = basew + 2ull * (unsigned long long)(incl - npair);
  const LayerR<R> &Ly = X.lr[L];
  const int ppc = Ly.ppc;
  uint32_t done = 0;
  for (uint32_t bits = ion; bits; bits &= bits - 1, slot += 2) {
    const uint32_t s = __ffs(bits) - 1;
    if (slot + 1 >= D.cap) {
      atomicOr(D.err, kErrPool);
      break;
    }
    Neutral<R> nu;
    neutral_at(D, Ly.sig_v, i, j, k, c, s, t1, nu);
    const int ncell = (nu.cell[2] * D.ny + nu.cell[1]) * D.nx + nu.cell[0];
    const unsigned long long gid = (unsigned long long)c * ppc + s;
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
      const unsigned long long q = slot + sp;
      D.pid[q] = 2ull * gid + sp;
      D.pcell[q] = ncell;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        D.po[d][q] = nu.off[d];
        D.pu[d][q] = nu.u[d];
      }
      D.ptag[q] = ((uint32_t)L << 1) | (uint32_t)sp;
    }
    done |= 1u << s;
  }
  D.alive[m] = alive & ~done;
  const double nd = (double)__popc(done);
  const LayerK &LK = D.layers[L];
  atomicAdd(D.acc + 1, nd * LK.wmac);
  atomicAdd(D.acc + 2, nd * LK.wmac * LK.gapJ);
  atomicAdd(D.acc + 3, nd);
}

// Each thread takes kIonizeCells material cells of a plane, a grid row of
// threads apart, and loads the next cell's three words while it draws for
// the current one.  (A thread per slot pair measured twice as
// slow as a thread per cell: four threads repeat the cell's index and
// threshold loads.)  FP32: six blocks per SM (40 registers): the kernel
// waits on its loads, and 64 registers (four blocks) measured 22% slower.
// The cells with neutrals that may have crossed a face (under 1% of them)
// are queued in shared memory and decided after the block's other cells,
// one per thread, so that a warp no longer runs that long path for one lane
// while the other 31 wait; a full queue sends the rest down the path at once.
constexpr int kIonizeCells = 4;
constexpr int kExcQueue = 256;

template <class R>
__device__ __forceinline__ void ionize_body(const Ctx<R> &X, Blk bk) {
  const Dev<R> &D = X.d;
  const int mp = bk.y;
  {
    // only cells at or above the skip amplitude can have a nonzero
    // threshold; a neutral may sit in the plane above or below its birth
    // plane, so a plane is skipped when neither it nor those hold one
    const uint32_t stamp = D.hot[bk.gy];
    if (stamp != 0xFFFFFFFFu && D.hot[mp] != stamp && (mp == 0 || D.hot[mp - 1] != stamp) &&
        (mp + 1 == bk.gy || D.hot[mp + 1] != stamp))
      return;
  }
  __shared__ int xq_r[kExcQueue];
  __shared__ uint32_t xq_bits[kExcQueue];
  __shared__ int xq_n;
  if (threadIdx.x == 0) xq_n = 0;
  __syncthreads();
  const int nx = D.nx, nxy = D.nxy;
  const long long step = *D.step;
  const int k = D.kplane[mp], L = D.layer_of_plane[k];
  const long long mbase = (long long)mp * nxy;
  const int stride = bk.gx * blockDim.x;
  const R sig = X.lr[L].sig_v;
  R t1;
  if constexpr (sizeof(R) == 4)
    t1 = R((int)(step + 1)) * D.dt;
  else
    t1 = R((double)(step + 1) * D.dt_d);
  // the cell's three words, loaded one cell ahead
  uint32_t alive_n = 0, leave_n = 0;
  unsigned long long T_n = 0;
  {
    const int r = bk.x * blockDim.x + threadIdx.x;
    if (r < nxy) {
      alive_n = D.alive[mbase + r];
      T_n = D.T[mbase + r];
      leave_n = D.leave_step[mbase + r];
    }
  }
  for (int r0 = bk.x * blockDim.x; r0 < nxy; r0 += stride) {
    const int r = r0 + threadIdx.x;
    const long long m = mbase + r;
    const uint32_t alive = alive_n, leave = leave_n;
    const unsigned long long Town = T_n;
    if (r + stride < nxy) {
      alive_n = D.alive[m + stride];
      T_n = D.T[m + stride];
      leave_n = D.leave_step[m + stride];
    } else {
      // past the plane's last cell (a ragged last row of threads): nothing
      alive_n = 0;
      T_n = 0;
      leave_n = 0;
    }
    uint32_t ion = 0, c = 0;
    if (alive) {
      c = (uint32_t)((long long)k * nxy + r);
      // neutrals that may have left the birth cell by t^{n+1}: their own
      // leave step (64-step units, rounded down) has been reached
      uint32_t exc = 0;
      if ((unsigned long long)(step + 1) >= (unsigned long long)leave) {
        const uint16_t *ls = X.leave16 + m * X.ppc_max;
        for (uint32_t bits = alive; bits; bits &= bits - 1) {
          const uint32_t s = __ffs(bits) - 1;
          if ((unsigned long long)(step + 1) >= 64ull * ls[s]) exc |= 1u << s;
        }
      }
      // birth-cell threshold for every other alive neutral: one block per
      // group of eight slots decides on the top 16 bits; the rare ties draw
      // their low 48 bits afterwards
      if (Town == ~0ull) {
        ion = alive & ~exc;
      } else if (Town != 0ull) {
        const uint32_t th = (uint32_t)(Town >> 48);
        uint32_t tie = 0;
        for (uint32_t bits = alive & ~exc; bits;) {
          const uint32_t g = (uint32_t)(__ffs(bits) - 1) >> 3;
          const uint32_t gm = 0xFFu << (8 * g);
          uint32_t lt, eq;
          ion_compare8(draw(D.seed, (uint32_t)step, c, g, kStreamIon), th, lt, eq);
          ion |= bits & gm & (lt << (8 * g));
          tie |= bits & gm & (eq << (8 * g));
          bits &= ~gm;
        }
        for (; tie; tie &= tie - 1) {
          const uint32_t s = __ffs(tie) - 1;
          const uint4 b = draw(D.seed, (uint32_t)step, c, s, kStreamIonLow);
          const unsigned long long lo48 = ((unsigned long long)(b.y & 0xFFFFu) << 32) | b.x;
          if (lo48 < (Town & 0xFFFFFFFFFFFFull)) ion |= 1u << s;
        }
      }
      if (exc) {
        const int q = atomicAdd(&xq_n, 1);
        if (q < kExcQueue) {
          xq_r[q] = r;
          xq_bits[q] = exc;
        } else {
          const int j = r / nx, i = r - j * nx;
          ion |= ion_exc(D, sig, i, j, k, c, exc, (uint32_t)step, t1);
        }
      }
    }
    ion_append(X, m, r, k, L, c, alive, ion, t1);
  }
  // the queued cells: their alive words as this block's appends left them
  __syncthreads();
  const int nq = min(xq_n, kExcQueue);
  for (int q0 = 0; q0 < nq; q0 += blockDim.x) {
    const int q = q0 + threadIdx.x;
    uint32_t ion = 0, c = 0, alive = 0;
    int r = 0;
    if (q < nq) {
      r = xq_r[q];
      alive = D.alive[mbase + r];
      c = (uint32_t)((long long)k * nxy + r);
      const int j = r / nx, i = r - j * nx;
      ion = ion_exc(D, sig, i, j, k, c, xq_bits[q] & alive, (uint32_t)step, t1);
    }
    ion_append(X, mbase + r, r, k, L, c, alive, ion, t1);
  }
}

template <class R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 6 : 3) k_ionize(Ctx<R> X) {
  ionize_body(X, blk_here());
}

// First step index at which any neutral of a cell could have left it.
template <class R>
__global__ void k_init_material(Ctx<R> X) {
  const Dev<R> &D = X.d;
  const long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (m >= D.nmat) return;
  const int nx = D.nx, nxy = D.nxy;
  const int mp = (int)(m / nxy);
  const int r = (int)(m - (long long)mp * nxy);
  const int k = D.kplane[mp];
  const LayerK &L = D.layers[D.layer_of_plane[k]];
  const uint32_t c = (uint32_t)((long long)k * nxy + r);
  const int ppc = L.ppc;
  D.alive[m] = ppc >= 32 ? 0xFFFFFFFFu : ((1u << ppc) - 1u);
  double smin = 4e9;
  const double dl[3] = {D.dx_d, D.dy_d, D.dz_d};
  // offset error of the position the working precision computes at run time
  // (birth offset, Box-Muller velocity and the product v t / dl rounded)
  const double eps = 16.0 * (sizeof(R) == 4 ? 0x1p-24 : 0x1p-53);
  uint16_t *ls = X.leave16 + m * X.ppc_max;
  for (int s = 0; s < ppc; ++s) {
    // the neutral's own birth offset and velocity (the same Philox draws the
    // step uses), in double
    const uint4 w = draw(D.seed, 0u, c, (uint32_t)s, kStreamPos);
    const double o3[3] = {unit_open<double>(w.x), unit_open<double>(w.y), unit_open<double>(w.z)};
    const uint4 wv = draw(D.seed, 0u, c, (uint32_t)s, kStreamVel);
    const double r1 = sqrt(-2.0 * log(unit_open<double>(wv.x)));
    const double r2 = sqrt(-2.0 * log(unit_open<double>(wv.z)));
    double s1, c1, s2, c2;
    sincospi(2.0 * unit_open<double>(wv.y), &s1, &c1);
    sincospi(2.0 * unit_open<double>(wv.w), &s2, &c2);
    const double v[3] = {L.sigv * r1 * c1, L.sigv * r1 * s1, L.sigv * r2 * c2};
    // time at which it may reach a face along any axis, less the time the
    // rounding of its run-time offset can be early by
    double t = 1e300;
    for (int d = 0; d < 3; ++d) {
      const double av = fabs(v[d]);
      if (!(av > 0.0)) continue;
      const double dist = (v[d] > 0.0 ? 1.0 - o3[d] : o3[d]) - eps;
      t = fmin(t, fmax(dist, 0.0) * dl[d] / av);
    }
    // steps before which this neutral is certainly inside its birth cell
    const double st = fmin(fmax(floor(t / D.dt_d) - 1.0, 0.0), 4e9);
    smin = fmin(smin, st);
    ls[s] = (uint16_t)fmin(floor(st / 64.0), 65535.0);
  }
  D.leave_step[m] = smin >= 4e9 ? 0xFFFFFFFFu : (uint32_t)smin;
  D.pm[m] = R(0);
  D.eamp[m] = R(0);
  D.ckey[m] = R(-1);
  D.T[m] = 0ull;
  (void)nx;
}

// End of a step: the Poynting split at the two flux planes (blockIdx.y = 0
// front, 1 back; a fixed number of blocks per plane over a fixed partition
// of its points) and the step counter.  At node plane k the transverse E (Ex and
// Ey of the plane) is paired with B averaged over planes k - 1 and k (By and
// Bx at k - 1/2 and k + 1/2, the same transverse positions) and split into
// the waves going along +z, ((Ex + c By) / 2, (Ey - c Bx) / 2), and along -z,
// ((Ex - c By) / 2, (Ey + c Bx) / 2).  Each block adds its FP64 sums of
// |fwd|^2 and |bwd|^2 over its points, times c eps0 dx dy dt, to its own
// running pair: the time integrals are the sums of the blocks' pairs, which
// the diagnostics form in block order (no reduction across blocks, no
// atomic, no last block per step).  The first block advances the step.
// Blocks per flux plane: one field point per thread (ceil(nxy / 256)), at
// most kFluxMaxBlocks, so each thread makes one round trip to memory.
constexpr int kFluxMaxBlocks = 256;

template <class R>
__device__ __forceinline__ void flux_advance_body(const Dev<R> &D, Blk bk) {
  const int q = bk.y;
  const long long base = (long long)D.flux_k[q] * D.nxy, basem = base - D.nxy;
  double f = 0.0, b = 0.0;
  for (int r = bk.x * blockDim.x + threadIdx.x; r < D.nxy; r += bk.gx * blockDim.x) {
    const double cby = kC * 0.5 * ((double)D.B[1][basem + r] + (double)D.B[1][base + r]);
    const double cbx = kC * 0.5 * ((double)D.B[0][basem + r] + (double)D.B[0][base + r]);
    const double ex = (double)D.E[0][base + r], ey = (double)D.E[1][base + r];
    const double fx = 0.5 * (ex + cby), fy = 0.5 * (ey - cbx);
    const double bx = 0.5 * (ex - cby), by = 0.5 * (ey + cbx);
    f += fx * fx + fy * fy;
    b += bx * bx + by * by;
  }
  const double fs = block_sum<R>(f);
  __syncthreads();
  const double bs = block_sum<R>(b);
  // each block adds its partial sums, times dt and the plane's area, to its
  // own running pair (no reduction across blocks per step: the diagnostics
  // sum the blocks' pairs in a fixed order)
  if (threadIdx.x == 0) {
    double *p = D.flux_part + 2 * (q * bk.gx + bk.x);
    p[0] += fs * D.flux_scale;
    p[1] += bs * D.flux_scale;
    if (bk.x == 0 && q == 0) *D.step += 1;  // nothing in this launch reads it
  }
}

template <class R>
__global__ void __launch_bounds__(256) k_flux_advance(Dev<R> D) {
  flux_advance_body(D, blk_here());
}

// ---------------------------------------------------------------------------
// Counting sort of the pool (dead slots dropped).  The key is the cell (the
// collision pass forms its pairs per cell), or (kByFrame) the lowest node of
// the particle's 3 x 3 x 3 deposit frame: its nearest integer node minus one
// on each axis, x and y wrapped.  Sorted by frame, the particles a warp
// pushes together share frame rows, so each of the deposit's vector
// reductions touches a few consecutive nodes of one grid row instead of up
// to four rows per cell.  Both keys lie in [0, ncell).
// ---------------------------------------------------------------------------
template <bool kByFrame, class R>
__device__ __forceinline__ int sort_key(const Dev<R> &D, int c, unsigned long long p) {
  if constexpr (!kByFrame) {
    return c;
  } else {
    const int nx = D.nx, ny = D.ny;
    const int ci = c % nx, t = c / nx, cj = t % ny, ck = t / ny;
    const int i0 = wrap(ci + (D.po[0][p] >= R(0.5) ? 0 : -1), nx);
    const int j0 = wrap(cj + (D.po[1][p] >= R(0.5) ? 0 : -1), ny);
    const int k0 = ck + (D.po[2][p] >= R(0.5) ? 0 : -1);
    return (k0 * ny + j0) * nx + i0;
  }
}

// Slots first + threadIdx.x + j stride below last (and below the slots in use).
template <bool kByFrame, class R>
__device__ __forceinline__ void hist_items(const Dev<R> &D, unsigned int *cnt,
                                           unsigned long long first, unsigned long long last,
                                           unsigned long long stride) {
  const unsigned long long n = min(min(*D.nslots, D.cap), last);
  for (unsigned long long p = first + threadIdx.x; p < n; p += stride) {
    const int c = D.pcell[p];
    if (c >= 0) atomicAdd(cnt + sort_key<kByFrame>(D, c, p), 1u);
  }
}

template <bool kByFrame, class R>
__global__ void k_hist(Dev<R> D, unsigned int *cnt) {
  hist_items<kByFrame>(D, cnt, blockIdx.x * (unsigned long long)blockDim.x, ~0ull,
                       (unsigned long long)gridDim.x * blockDim.x);
}

constexpr int kScanThreads = 256, kScanItems = 16, kScanChunk = kScanThreads * kScanItems;

__device__ __forceinline__ unsigned int block_excl_scan(unsigned int v, unsigned int &total) {
  __shared__ unsigned int warp_tot[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned int incl = v;
#pragma unroll
  for (int s = 1; s < 32; s <<= 1) {
    const unsigned int t = __shfl_up_sync(0xffffffffu, incl, s);
    if (lane >= s) incl += t;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    unsigned int x = lane < nw ? warp_tot[lane] : 0u;
    unsigned int xi = x;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
      const unsigned int t = __shfl_up_sync(0xffffffffu, xi, s);
      if (lane >= s) xi += t;
    }
    if (lane < nw) warp_tot[lane] = xi - x;
    if (lane == nw - 1) warp_tot[31] = xi;
  }
  __syncthreads();
  const unsigned int excl = warp_tot[w] + incl - v;
  total = warp_tot[31];
  __syncthreads();
  return excl;
}

__device__ __forceinline__ void scan_reduce_body(const unsigned int *cnt, long long n,
                                                 unsigned int *bsum, int bx) {
  const long long base = (long long)bx * kScanChunk;
  unsigned int s = 0;
  for (int q = 0; q < kScanItems; ++q) {
    const long long idx = base + (long long)q * kScanThreads + threadIdx.x;
    if (idx < n) s += cnt[idx];
  }
  unsigned int tot;
  block_excl_scan(s, tot);
  if (threadIdx.x == 0) bsum[bx] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const unsigned int *cnt, long long n,
                                                               unsigned int *bsum) {
  scan_reduce_body(cnt, n, bsum, blockIdx.x);
}

__global__ void __launch_bounds__(kScanThreads) k_scan_blocks(unsigned int *bsum, int nb,
                                                               unsigned long long *total_out) {
  unsigned int carry = 0;
  for (int base = 0; base < nb; base += kScanThreads) {
    const int idx = base + threadIdx.x;
    const unsigned int v = idx < nb ? bsum[idx] : 0u;
    unsigned int tot;
    const unsigned int ex = block_excl_scan(v, tot);
    if (idx < nb) bsum[idx] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) *total_out = carry;
}

// Each thread scans kScanItems consecutive counts, moved as 16-byte vectors
// (the arena is 256-byte aligned, so a thread's run starts on a 64-byte
// boundary); a ragged last run goes element by element.
__device__ __forceinline__ void scan_final_body(unsigned int *cnt, long long n,
                                                const unsigned int *bsum, int bx) {
  const long long base = (long long)bx * kScanChunk + (long long)threadIdx.x * kScanItems;
  const bool full = base + kScanItems <= n;
  unsigned int v[kScanItems];
  if (full) {
    const uint4 *p4 = reinterpret_cast<const uint4 *>(cnt + base);
#pragma unroll
    for (int q = 0; q < kScanItems / 4; ++q) {
      const uint4 t = p4[q];
      v[4 * q] = t.x;
      v[4 * q + 1] = t.y;
      v[4 * q + 2] = t.z;
      v[4 * q + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) v[q] = base + q < n ? cnt[base + q] : 0u;
  }
  unsigned int s = 0;
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) s += v[q];
  unsigned int tot;
  unsigned int ex = block_excl_scan(s, tot) + bsum[bx];
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    const unsigned int e = ex;
    ex += v[q];
    v[q] = e;
  }
  if (full) {
    uint4 *p4 = reinterpret_cast<uint4 *>(cnt + base);
#pragma unroll
    for (int q = 0; q < kScanItems / 4; ++q)
      p4[q] = make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  } else {
#pragma unroll
    for (int q = 0; q < kScanItems; ++q)
      if (base + q < n) cnt[base + q] = v[q];
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_final(unsigned int *cnt, long long n,
                                                              const unsigned int *bsum) {
  scan_final_body(cnt, n, bsum, blockIdx.x);
}

// Slots first + threadIdx.x + j stride below last (and below the slots in use).
template <bool kByFrame, class R>
__device__ __forceinline__ void scatter_items(const Ctx<R> &X, unsigned int *cursor,
                                              unsigned long long first, unsigned long long last,
                                              unsigned long long stride) {
  const Dev<R> &D = X.d;
  const unsigned long long n = min(min(*D.nslots, D.cap), last);
  for (unsigned long long p = first + threadIdx.x; p < n; p += stride) {
    const int c = D.pcell[p];
    if (c < 0) continue;
    const unsigned int q = atomicAdd(cursor + sort_key<kByFrame>(D, c, p), 1u);
    X.acell[q] = c;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      X.ao[d][q] = D.po[d][p];
      X.au[d][q] = D.pu[d][p];
    }
    X.atag[q] = D.ptag[p];
    X.aid[q] = D.pid[p];
  }
}

template <bool kByFrame, class R>
__global__ void __launch_bounds__(256) k_scatter(Ctx<R> X, unsigned int *cursor) {
  scatter_items<kByFrame>(X, cursor, blockIdx.x * (unsigned long long)blockDim.x, ~0ull,
                          (unsigned long long)gridDim.x * blockDim.x);
}

__global__ void k_set_slots(unsigned long long *nslots, const unsigned long long *total) {
  *nslots = *total;
}

// ---------------------------------------------------------------------------
// Diagnostics (FP64): per-particle deposits and sums, per-node reductions.
// Block partials are reduced on the host in a fixed order.
// ---------------------------------------------------------------------------
template <class R>
__global__ void __launch_bounds__(256) k_diag_particles(Ctx<R> X, double *ne, double *ed,
                                                         double *rho, double *spec, int nbins,
                                                         double emin, double emax, int4 r0,
                                                         int2 r1, double *partials) {
  const Dev<R> &D = X.d;
  const unsigned long long n = min(*D.nslots, D.cap);
  const int nx = D.nx, ny = D.ny;
  double kin = 0.0, nel = 0.0, nho = 0.0;
  for (unsigned long long p = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; p < n;
       p += (unsigned long long)gridDim.x * blockDim.x) {
    const int cell = D.pcell[p];
    if (cell < 0) continue;
    const int ci = cell % nx, t = cell / nx, cj = t % ny, ck = t / ny;
    const uint32_t tag = D.ptag[p];
    const LayerK &L = D.layers[tag >> 1];
    const int sp = tag & 1u;
    const double ux = D.pu[0][p], uy = D.pu[1][p], uz = D.pu[2][p];
    const double g = sqrt(1.0 + (ux * ux + uy * uy + uz * uz) / (kC * kC));
    const double ek = (g - 1.0) * L.mass[sp] * kC * kC;
    kin += L.wmac * ek;
    const double q = (sp ? kQe : -kQe) * L.wmac / D.V_d;
    double w[3][3];
    int b[3];
    const double o3[3] = {(double)D.po[0][p], (double)D.po[1][p], (double)D.po[2][p]};
    for (int d = 0; d < 3; ++d) {
      const int s = o3[d] >= 0.5;
      const double e = o3[d] - s;
      b[d] = s - 1;
      w[d][0] = 0.5 * (0.5 - e) * (0.5 - e);
      w[d][1] = 0.75 - e * e;
      w[d][2] = 0.5 * (0.5 + e) * (0.5 + e);
    }
    const bool el = sp == 0;
    const double vne = L.wmac / D.V_d, ved = L.wmac * ek / D.V_d;
    for (int c = 0; c < 3; ++c)
      for (int bb = 0; bb < 3; ++bb)
        for (int a = 0; a < 3; ++a) {
          const long long o = ((long long)(ck + b[2] + c) * ny + wrap(cj + b[1] + bb, ny)) * nx +
                              wrap(ci + b[0] + a, nx);
          const double wt = w[0][a] * w[1][bb] * w[2][c];
          atomicAdd(rho + o, q * wt);
          if (el) {
            atomicAdd(ne + o, vne * wt);
            atomicAdd(ed + o, ved * wt);
          }
        }
    if (el) {
      nel += 1.0;
      if (nbins > 0 && ci >= r0.x && ci < r0.y && cj >= r0.z && cj < r0.w && ck >= r1.x &&
          ck < r1.y) {
        const double ev = ek / kQe;
        if (ev >= emin && ev < emax) {
          const int bin = (int)floor((ev - emin) / (emax - emin) * nbins);
          if (bin >= 0 && bin < nbins) atomicAdd(spec + bin, L.wmac);
        }
      }
    } else {
      nho += 1.0;
    }
  }
  const double a = block_sum<R>(kin);
  __syncthreads();
  const double bq = block_sum<R>(nel);
  __syncthreads();
  const double cq = block_sum<R>(nho);
  if (threadIdx.x == 0) {
    partials[3 * blockIdx.x + 0] = a;
    partials[3 * blockIdx.x + 1] = bq;
    partials[3 * blockIdx.x + 2] = cq;
  }
}

__device__ __forceinline__ double block_max(double v) {
  __shared__ double part[32];
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, s));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) part[w] = v;
  __syncthreads();
  double tot = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tot = fmax(tot, part[q]);
  return tot;
}

template <class R>
__global__ void __launch_bounds__(256) k_diag_grid(Ctx<R> X, const double *ne, const double *ed,
                                                    const double *rho, double *partials) {
  const Dev<R> &D = X.d;
  const long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double uf = 0.0, mne = 0.0, med = 0.0, mrho = 0.0, mg = 0.0;
  if (o < D.nfield) {
    const int nx = D.nx, ny = D.ny, nz = D.nz, nxy = D.nxy;
    const int k = (int)(o / nxy);
    const int r = (int)(o - (long long)k * nxy);
    const int j = r / nx, i = r - j * nx;
    for (int d = 0; d < 3; ++d) {
      const double e = D.E[d][o], b = D.B[d][o];
      uf += 0.5 * kEps0 * e * e + 0.5 * b * b / kMu0;
    }
    mne = ne[o];
    med = ed[o];
    mrho = fabs(rho[o]);
    if (k >= 4 && k <= nz - 4) {
      const long long omi = (i == 0) ? o + (nx - 1) : o - 1;
      const long long omj = (j == 0) ? o + (long long)(ny - 1) * nx : o - nx;
      const long long omk = o - nxy;
      auto pol = [&](int d, long long oo, int kk) -> double {
        const int mp = D.mplane[kk];
        if (mp < 0) return 0.0;
        return (double)D.P[d][(long long)mp * nxy + (oo - (long long)kk * nxy)];
      };
      const double dxv = ((double)D.E[0][o] + pol(0, o, k)) - ((double)D.E[0][omi] + pol(0, omi, k));
      const double dyv = ((double)D.E[1][o] + pol(1, o, k)) - ((double)D.E[1][omj] + pol(1, omj, k));
      const double dzv =
          ((double)D.E[2][o] + pol(2, o, k)) - ((double)D.E[2][omk] + pol(2, omk, k - 1));
      const double div = dxv / D.dx_d + dyv / D.dy_d + dzv / D.dz_d;
      mg = fabs(kEps0 * div - rho[o]);
    }
  }
  const double v0 = block_sum<R>(uf);
  __syncthreads();
  const double v1 = block_max(mne);
  __syncthreads();
  const double v2 = block_max(med);
  __syncthreads();
  const double v3 = block_max(mrho);
  __syncthreads();
  const double v4 = block_max(mg);
  if (threadIdx.x == 0) {
    double *p = partials + 5 * blockIdx.x;
    p[0] = v0;
    p[1] = v1;
    p[2] = v2;
    p[3] = v3;
    p[4] = v4;
  }
}

// ---------------------------------------------------------------------------
// Binary collisions among electrons and holes (Sec. 2.2).  Nanbu's
// cumulative small-angle scattering (Phys. Rev. E 55, 4642, 1997) in the
// relativistic centre-of-mass frame of Perez et al. (Phys. Plasmas 19,
// 083104, 2012), Coulomb logarithm bounded below by 1 (Sec. 2.2), screening
// no shorter than the interparticle spacing and the low-temperature cap on
// the collision parameter.  One warp per cell of the cell-sorted pool.  The
// arithmetic is in the working precision with momenta in units of m_e c and
// masses in m_e (every float quantity then stays in range); the SI
// prefactors come from the host in double.
// ---------------------------------------------------------------------------
constexpr int kCollMax = 128;  // charged particles per cell a pass handles
constexpr int kCollWarps = 4;  // cells per block

// SI constants of the normalised collision arithmetic (host-computed).
struct CollConst {
  double K1;    // e^4 / (4 pi eps0^2 c^3 m_e^2)            [m^3 / s]
  double re;    // e^2 / (4 pi eps0 m_e c^2)                 [m]
  double lc;    // h / (m_e c)                               [m]
  double kD;    // e^2 / (eps0 m_e c^2) = 4 pi re            [m]
  double capc;  // (4 pi / 3)^(1/3) c                         [m/s]
};

// e^2 / (eps0 m_e c^2) = 4 pi r_e [m]: the Debye sum in normalised units.
constexpr double K_KD = kQe * kQe / (kEps0 * kMe * kC * kC);

// Arithmetic of the collision pass in the working precision.  FP32, whose
// results are held to 1e-5 of the FP64 oracle, takes the hardware's
// approximate division, reciprocal square root, exponential and logarithm
// (each within a few ulp over the ranges met here); FP64 the correctly
// rounded operations.
template <class R>
struct CollMath {
  __device__ static R div(R a, R b) { return a / b; }
  __device__ static R rcp(R x) { return R(1) / x; }
  __device__ static R sqrt_(R x) { return sqrt(x); }
  __device__ static R exp_(R x) { return exp(x); }
  __device__ static R log_(R x) { return log(x); }
  __device__ static R one_minus_exp_m2(R A) { return -expm1(R(-2) * A); }  // 1 - exp(-2A)
};
template <>
struct CollMath<float> {
  __device__ static float div(float a, float b) { return __fdividef(a, b); }
  __device__ static float rcp(float x) { return __fdividef(1.0f, x); }
  __device__ static float sqrt_(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }
  __device__ static float exp_(float x) { return __expf(x); }
  __device__ static float log_(float x) { return __logf(x); }
  // only for A >= 0.5, where 1 - exp(-2A) >= 0.63 does not cancel
  __device__ static float one_minus_exp_m2(float A) { return 1.0f - __expf(-2.0f * A); }
};

template <class R> struct CollTol;
template <> struct CollTol<double> { static constexpr double v = 4e-16, small = 1e-4; };
template <> struct CollTol<float> { static constexpr float v = 4e-7f, small = 0.5f; };

// Langevin function coth A - 1/A (its series where the difference cancels).
template <class R>
__device__ __forceinline__ R langevin(R A) {
  if (A < CollTol<R>::small) {
    const R A2 = A * A;
    if (sizeof(R) == 8) return A / R(3) - A * A2 / R(45);
    return A * (R(1) / R(3) + A2 * (R(-1) / R(45) + A2 * (R(2) / R(945) +
                A2 * (R(-1) / R(4725) + A2 * (R(2) / R(93555))))));
  }
  return R(1) / tanh(A) - R(1) / A;
}

// Derivative of the Langevin function, 1/A^2 - 1/sinh^2 A (its series
// where the difference cancels).
template <class R>
__device__ __forceinline__ R langevin_d(R A) {
  if (A < R(sizeof(R) == 8 ? 1e-2 : 0.5)) {
    const R A2 = A * A;
    return R(1) / R(3) + A2 * (R(-1) / R(15) + A2 * (R(2) / R(189) + A2 * (R(-1) / R(675))));
  }
  const R sh = sinh(A);
  return R(1) / (A * A) - R(1) / (sh * sh);
}

// The Langevin function and its derivative at A together: the series below
// the thresholds where the differences cancel, else from one d = 1 -
// exp(-2A): coth A = (2 - d)/d and 1/sinh^2 A = 4 (1 - d)/d^2.
template <class R>
__device__ __forceinline__ void langevin_both(R A, R &L, R &Ld) {
  const R A2 = A * A;
  const bool smallL = A < CollTol<R>::small, smallD = A < R(sizeof(R) == 8 ? 1e-2 : 0.5);
  if (smallL && smallD) {
    L = langevin(A);
    Ld = langevin_d(A);
    return;
  }
  using M = CollMath<R>;
  const R d = M::one_minus_exp_m2(A), id = M::rcp(d), iA = M::rcp(A);
  L = smallL ? langevin(A) : (R(2) - d) * id - iA;
  Ld = smallD ? langevin_d(A) : iA * iA - R(4) * (R(1) - d) * id * id;
}

// Nanbu's parameter A(s): the root of coth A - 1/A = exp(-s).  Newton from
// the left (the function is increasing and concave, so the iterates rise
// monotonically to the root), started at 0.95 of Cohen's Pade inverse
// t (3 - t^2) / (1 - t^2) of the Langevin function, t = exp(-s): that lies
// 0 to 4.94% above the root for 0.1 <= s < 6, so the start is below it, and
// two steps reach FP32 precision; at most 40 steps.
template <class R>
__device__ R nanbu_A(R s) {
  using M = CollMath<R>;
  const R t = M::exp_(-s);
  R A = R(0.95) * t * M::div(R(3) - t * t, R(1) - t * t);
  for (int it = 0; it < 40; ++it) {
    R L, Ld;
    langevin_both(A, L, Ld);
    const R dA = M::div(t - L, Ld);
    A += dA;
    if (!(fabs(dA) > CollTol<R>::v * A)) break;
  }
  return A;
}

// cos chi for parameter s and uniform U: 1 + s ln U for s < 0.1, isotropic
// for s >= 6, otherwise the inverse of A exp(A cos chi) / (2 sinh A).
template <class R>
__device__ R nanbu_cos(R s, R U) {
  using M = CollMath<R>;
  R c;
  if (s < R(0.1)) {
    c = R(1) + s * M::log_(U);
  } else if (s < R(6)) {
    const R A = nanbu_A(s);
    c = M::log_(M::exp_(-A) + R(2) * U * sinh(A)) * M::rcp(A);
  } else {
    c = R(2) * U - R(1);
  }
  return fmin(R(1), fmax(R(-1), c));
}

// One collision of a and b: normalised momenta u (units of c, u = gamma v),
// masses m (units of m_e), weights w; centre-of-mass momentum rotated by
// (chi, phi), then back to the lab frame; each side moves with probability
// w_other / max(w_a, w_b).  nd = neff * dtc (density factor times the
// collision interval); na23, nb23 the group densities to the power 2/3
// (per cell); lD the screening length.  Quotients by a common denominator
// are products with its reciprocal.
template <class R>
__device__ void collide_pair(R ua[3], R ub[3], R ma, R mb, R wa, R wb, R nd, R na23, R nb23, R lD,
                             const CollConst &K, const R U[4]) {
  using M = CollMath<R>;
  const R ga = M::sqrt_(R(1) + (ua[0] * ua[0] + ua[1] * ua[1] + ua[2] * ua[2]));
  const R gb = M::sqrt_(R(1) + (ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2]));
  const R Et = ma * ga + mb * gb;
  const R iga = M::rcp(ga), igb = M::rcp(gb), iEt = M::rcp(Et);
  R vc[3], va[3], vb[3], pa[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    pa[d] = ma * ua[d];
    va[d] = ua[d] * iga;
    vb[d] = ub[d] * igb;
    vc[d] = (pa[d] + mb * ub[d]) * iEt;
  }
  const R vc2 = vc[0] * vc[0] + vc[1] * vc[1] + vc[2] * vc[2];
  const R gc = M::rcp(M::sqrt_(R(1) - vc2));
  const R kc = M::div(gc * gc, gc + R(1));  // (gamma_c - 1) / v_c^2
  const R vcva = vc[0] * va[0] + vc[1] * va[1] + vc[2] * va[2];
  const R vcvb = vc[0] * vb[0] + vc[1] * vb[1] + vc[2] * vb[2];
  R ps[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) ps[d] = pa[d] + (kc * vcva - gc) * ma * ga * vc[d];
  const R gsa = (R(1) - vcva) * gc * ga, gsb = (R(1) - vcvb) * gc * gb;
  const R p2 = ps[0] * ps[0] + ps[1] * ps[1] + ps[2] * ps[2];
  const R pm = M::sqrt_(p2);
  if (!(pm > R(0))) return;
  const R ipm = M::rcp(pm);
  const R mab = ma * gsa * mb * gsb;
  const R mm = M::div(mab, p2) + R(1);
  const R b0 = R(K.re) * gc * iEt * mm;
  const R bmin = fmax(R(K.lc) * R(0.5) * ipm, b0);
  const R lnL = fmax(R(1), R(0.5) * M::log_(R(1) + M::div(lD * lD, bmin * bmin)));
  const R sv = M::div(nd * R(K.K1) * lnL * gc * pm, ma * ga * mb * gb * Et) * mm * mm;
  const R vrel = M::div(Et * pm, mab * gc);
  const R dens = fmax(ma * na23, mb * nb23);
  const R scap = M::div(nd * R(K.capc) * (ma + mb), dens) * vrel;
  const R s = fmin(sv, scap);
  const R cx = nanbu_cos(s, U[0]);
  const R sx = M::sqrt_(fmax(R(0), R(1) - cx * cx));
  R sp, cp;
  sincospi(R(2) * U[1], &sp, &cp);  // phi = 2 pi U
  const R u[3] = {ps[0] * ipm, ps[1] * ipm, ps[2] * ipm};
  R e1[3], e2v[3];
  if (fabs(u[2]) < R(0.9)) {
    const R in = M::rcp(M::sqrt_(u[0] * u[0] + u[1] * u[1]));
    e1[0] = u[1] * in;
    e1[1] = -u[0] * in;
    e1[2] = R(0);
  } else {
    const R in = M::rcp(M::sqrt_(u[1] * u[1] + u[2] * u[2]));
    e1[0] = R(0);
    e1[1] = u[2] * in;
    e1[2] = -u[1] * in;
  }
  e2v[0] = u[1] * e1[2] - u[2] * e1[1];
  e2v[1] = u[2] * e1[0] - u[0] * e1[2];
  e2v[2] = u[0] * e1[1] - u[1] * e1[0];
  R pn[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) pn[d] = pm * (cx * u[d] + sx * (cp * e1[d] + sp * e2v[d]));
  const R vpa = vc[0] * pn[0] + vc[1] * pn[1] + vc[2] * pn[2];
  // (a side whose partner weighs at least as much always moves: the same
  // as U w_max < w_other for every U < 1, and safe when a float U rounds to 1)
  const R wmax = fmax(wa, wb);
  if (wb >= wmax || U[2] * wmax < wb) {
    const R ima = M::rcp(ma);
#pragma unroll
    for (int d = 0; d < 3; ++d) ua[d] = (pn[d] + (kc * vpa + ma * gsa * gc) * vc[d]) * ima;
  }
  if (wa >= wmax || U[3] * wmax < wa) {
    const R imb = M::rcp(mb);
#pragma unroll
    for (int d = 0; d < 3; ++d) ub[d] = (-pn[d] + (-kc * vpa + mb * gsb * gc) * vc[d]) * imb;
  }
}

template <class R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Per-warp shared state of one cell while it is prepared.
template <class R>
struct CollCell {
  uint32_t key[kCollMax];
  unsigned long long id[kCollMax];
  R v[3][kCollMax];  // velocity / c
  R m[kCollMax];     // mass / m_e
  R w[kCollMax];     // weight
  uint8_t sp[kCollMax];
};

// A prepared cell: where its particles start in the sorted pool, its group
// sizes, the collision parameters shared by its pairs and the Philox index
// of its first unlike pair.  ord (global, indexed like the pool) lists the
// cell's slots in pairing order: electrons, then holes.
template <class R>
struct CollParam {
  unsigned int st, cell;
  int nE, nH;
  R ndl[2];  // like pairs: group density x collision interval
  R ndu;     // unlike pairs: n_e n_h / n_ab x collision interval
  R dens23[2], lD;  // group densities to the power 2/3 (collide_pair's spacing cap)
  uint32_t qu;
};

// Work items: bits 0-31 the cell, bit 32 the group, bit 33 a triplet,
// bits 34-49 the pair (or unlike column) index.
__device__ __forceinline__ unsigned long long coll_item(int cidx, int sp, int tri, int k) {
  return (unsigned long long)(unsigned)cidx | ((unsigned long long)sp << 32) |
         ((unsigned long long)tri << 33) | ((unsigned long long)k << 34);
}

// Pair q of a cell (pool slots pa, pb): both particles read from and written
// back to the pool.  Out of line: one copy of the pair arithmetic for all
// call sites keeps the kernels within the instruction cache.
template <class R>
__device__ __noinline__ void collide_pool(const Dev<R> &D, const LayerR<R> *__restrict__ lr,
                                          unsigned long long pa, unsigned long long pb,
                                          uint32_t step, uint32_t c, uint32_t q, R nd, R na23,
                                          R nb23, R lD, const CollConst &K) {
  const uint32_t ta = D.ptag[pa], tb = D.ptag[pb];
  const LayerR<R> &La = lr[ta >> 1], &Lb = lr[tb >> 1];
  const R ic = R(1.0 / kC);
  R ua[3], ub[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    ua[d] = D.pu[d][pa] * ic;
    ub[d] = D.pu[d][pb] * ic;
  }
  const uint4 w = draw(D.seed, step, c, q, kStreamCollPair);
  const R U[4] = {unit_open<R>(w.x), unit_open<R>(w.y), unit_open<R>(w.z), unit_open<R>(w.w)};
  collide_pair(ua, ub, La.mhat[ta & 1u], Lb.mhat[tb & 1u], La.wmac, Lb.wmac, nd, na23, nb23, lD, K,
               U);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    D.pu[d][pa] = ua[d] * R(kC);
    D.pu[d][pb] = ub[d] * R(kC);
  }
}

constexpr int kCollSmall = 8;  // cells up to this size are prepared by one thread

// Cells that hold two or more charged particles after the sort: those of at
// most kCollSmall in list (count n[0]), larger ones in list + ncell (n[4]).
// Each thread classifies kCellsPerThread consecutive cells and each block
// reserves its entries with one atomic per list (the order of the lists
// does not matter: every cell's collisions are independent).
constexpr int kCellsPerThread = 4;

__global__ void __launch_bounds__(256) k_coll_cells(const unsigned int *cend, long long ncell,
                                                    int *list, int *n) {
  __shared__ int wsum[2][8], wbase[2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long c0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) * kCellsPerThread;
  uint32_t small = 0, large = 0;  // bit q: cell c0 + q
  unsigned int prev = (c0 > 0 && c0 <= ncell) ? cend[c0 - 1] : 0u;
#pragma unroll
  for (int q = 0; q < kCellsPerThread; ++q) {
    const long long c = c0 + q;
    const unsigned int e = c < ncell ? cend[c] : prev;
    const unsigned int m = e - prev;
    prev = e;
    small |= (uint32_t)(m >= 2u && m <= (unsigned)kCollSmall) << q;
    large |= (uint32_t)(m > (unsigned)kCollSmall) << q;
  }
  int cnt[2] = {__popc(small), __popc(large)}, incl[2] = {cnt[0], cnt[1]};
#pragma unroll
  for (int sft = 1; sft < 32; sft <<= 1) {
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      const int v = __shfl_up_sync(0xffffffffu, incl[g], sft);
      if (lane >= sft) incl[g] += v;
    }
  }
  if (lane == 31) {
    wsum[0][warp] = incl[0];
    wsum[1][warp] = incl[1];
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    const int g = threadIdx.x;
    int tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      const int v = wsum[g][w];
      wsum[g][w] = tot;
      tot += v;
    }
    wbase[g] = tot ? atomicAdd(n + 4 * g, tot) : 0;
  }
  __syncthreads();
#pragma unroll
  for (int g = 0; g < 2; ++g) {
    int at = wbase[g] + wsum[g][warp] + incl[g] - cnt[g];
    int *const dst = list + g * ncell;
    for (uint32_t bits = g ? large : small; bits; bits &= bits - 1) dst[at++] = (int)(c0 + __ffs(bits) - 1);
  }
}

// Collision work of one pass, in global memory.
template <class R>
struct CollWork {
  const int *list;               // listed cells: small ones (count n[0]), large at + ncell (n[4])
  int *n;                        // [0] small cells [1] like pairs [2] unlike columns of
                                 // one collision [3] like triplets [4] large cells
                                 // [5] unlike columns of two or more collisions
  long long ncell;
  int lcap;                      // entries of like and unl: pairs and one-collision
                                 // columns fill them from the front, triplets and
                                 // longer columns from the back (each list holds at
                                 // most half the particles, so the ends never meet),
                                 // so that a warp's threads do equal work
  CollParam<R> *par;             // indexed by cell
  int *ord;                      // pool-indexed pairing order of every listed cell
  unsigned long long *like, *unl;  // work items
};

// Prepare one listed cell (one warp): order each group by its Philox keys,
// take the group densities, kinetic temperatures and screening length, and
// append the cell's like pairs, triplets and unlike columns as work items.
template <class R>
__device__ void coll_prep_cell(const Dev<R> &D, const LayerR<R> *__restrict__ lr, CollCell<R> &S,
                               const unsigned int *cend, int cidx, const CollWork<R> &W,
                               double dtc) {
  const int lane = threadIdx.x & 31;
  const long long c = cidx;
  const unsigned int st = c ? cend[c - 1] : 0u, en = cend[c];
  const int n = (int)(en - st);
  if (n > kCollMax) {
    if (lane == 0) atomicOr(D.err, kErrColl);
    return;
  }
  const uint32_t step = (uint32_t)*D.step;
  const R ic = R(1.0 / kC);
  int cnt[2] = {0, 0};
  for (int i0 = 0; i0 < n; i0 += 32) {
    const int i = i0 + lane;
    uint8_t sp = 2;
    if (i < n) {
      const unsigned long long p = st + i;
      const unsigned long long id = D.pid[p];
      S.id[i] = id;
      S.key[i] = draw(D.seed, step, (uint32_t)id, (uint32_t)(id >> 32), kStreamCollOrder).x;
      const uint32_t t = D.ptag[p];
      sp = (uint8_t)(t & 1u);
      S.sp[i] = sp;
      S.m[i] = lr[t >> 1].mhat[sp];
      S.w[i] = lr[t >> 1].wmac;
      const R u0 = D.pu[0][p] * ic, u1 = D.pu[1][p] * ic, u2 = D.pu[2][p] * ic;
      const R g = sqrt(R(1) + (u0 * u0 + u1 * u1 + u2 * u2));
      S.v[0][i] = u0 / g;
      S.v[1][i] = u1 / g;
      S.v[2][i] = u2 / g;
    }
    cnt[0] += __popc(__ballot_sync(0xffffffffu, sp == 0));
    cnt[1] += __popc(__ballot_sync(0xffffffffu, sp == 1));
  }
  __syncwarp();
  for (int i = lane; i < n; i += 32) {
    const uint32_t ki = S.key[i];
    const unsigned long long idi = S.id[i];
    const uint8_t si = S.sp[i];
    int r = 0;
    for (int j = 0; j < n; ++j)
      if (S.sp[j] == si && (S.key[j] < ki || (S.key[j] == ki && S.id[j] < idi))) ++r;
    W.ord[st + (si ? cnt[0] : 0) + r] = (int)(st + i);
  }
  // densities and kinetic temperatures of the two groups: mean mass times
  // the weighted velocity variance, written as a sum over pairs (exactly 0
  // for one particle or equal velocities, no cancellation); T / (m_e c^2)
  R ws[2] = {R(0), R(0)}, wm[2] = {R(0), R(0)}, Sv[2] = {R(0), R(0)};
  for (int i = lane; i < n; i += 32) {
    const int sp = S.sp[i];
    ws[sp] += S.w[i];
    wm[sp] += S.w[i] * S.m[i];
    for (int j = i + 1; j < n; ++j) {
      if (S.sp[j] != sp) continue;
      const R d0 = S.v[0][i] - S.v[0][j], d1 = S.v[1][i] - S.v[1][j], d2 = S.v[2][i] - S.v[2][j];
      Sv[sp] += S.w[i] * S.w[j] * (d0 * d0 + d1 * d1 + d2 * d2);
    }
  }
  const R V = R(D.V_d);
  R dens[2], inv_l2 = R(0);
#pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
    ws[sp] = warp_sum(ws[sp]);
    wm[sp] = warp_sum(wm[sp]);
    Sv[sp] = warp_sum(Sv[sp]);
    const R T = ws[sp] > R(0) ? wm[sp] / ws[sp] * Sv[sp] / (R(3) * ws[sp] * ws[sp]) : R(0);
    dens[sp] = ws[sp] / V;
    if (T > R(0)) inv_l2 += dens[sp] * R(K_KD) / T;
  }
  __syncwarp();  // ord is complete
  const R ni = dens[1] > R(0) ? dens[1] : dens[0];
  const R ra = pow(R(4 * kPi / 3) * ni, R(-1) / R(3));
  const R lD = inv_l2 > R(0) ? fmax(R(1) / sqrt(inv_l2), ra) : ra;
  const R dt = R(dtc);
  const int nlike[2] = {cnt[0] < 2 ? 0 : ((cnt[0] & 1) ? 3 + (cnt[0] - 3) / 2 : cnt[0] / 2),
                        cnt[1] < 2 ? 0 : ((cnt[1] & 1) ? 3 + (cnt[1] - 3) / 2 : cnt[1] / 2)};
  R ndu = R(0);
  if (cnt[0] > 0 && cnt[1] > 0) {
    const int A = cnt[0] >= cnt[1] ? 0 : 1, B = 1 - A;
    const int nA = cnt[A], nB = cnt[B];
    const int *oA = W.ord + st + (A ? cnt[0] : 0), *oB = W.ord + st + (B ? cnt[0] : 0);
    R nab = R(0);
    for (int i = lane; i < nA; i += 32)
      nab += fmin(lr[D.ptag[oA[i]] >> 1].wmac, lr[D.ptag[oB[i % nB]] >> 1].wmac) / V;
    nab = warp_sum(nab);
    ndu = dens[0] * (dens[1] / nab) * dt;
  }
  if (lane == 0) {
    CollParam<R> P;
    P.st = st;
    P.cell = (unsigned)c;
    P.nE = cnt[0];
    P.nH = cnt[1];
    P.ndl[0] = dens[0] * dt;
    P.ndl[1] = dens[1] * dt;
    P.ndu = ndu;
    P.dens23[0] = pow(dens[0], R(2) / R(3));
    P.dens23[1] = pow(dens[1], R(2) / R(3));
    P.lD = lD;
    P.qu = (uint32_t)(nlike[0] + nlike[1]);
    W.par[c] = P;
  }
  // work items: the triplet and like pairs of each group, then the unlike
  // columns, each list's entries reserved with one atomic per cell
  int tri[2], rest[2];
#pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
    const int m = cnt[sp];
    tri[sp] = m >= 3 && (m & 1);
    rest[sp] = m < 2 ? 0 : (tri[sp] ? (m - 3) / 2 : m / 2);
  }
  const int np = rest[0] + rest[1], nt = tri[0] + tri[1];
  const int nB = (cnt[0] > 0 && cnt[1] > 0) ? min(cnt[0], cnt[1]) : 0;
  const int nA = max(cnt[0], cnt[1]);
  const int nm = nB ? max(0, min(nB, nA - nB)) : 0;  // columns j < nA - nB collide twice or more
  int b[4] = {0, 0, 0, 0};
  if (lane == 0) {
    if (np) b[0] = atomicAdd(W.n + 1, np);
    if (nt) b[1] = atomicAdd(W.n + 3, nt);
    if (nB - nm) b[2] = atomicAdd(W.n + 2, nB - nm);
    if (nm) b[3] = atomicAdd(W.n + 5, nm);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) b[q] = __shfl_sync(0xffffffffu, b[q], 0);
  for (int e = lane; e < np; e += 32) {
    const int sp = e < rest[0] ? 0 : 1;
    W.like[b[0] + e] = coll_item(cidx, sp, 0, sp ? e - rest[0] : e);
  }
  if (lane < nt) W.like[W.lcap - 1 - (b[1] + lane)] = coll_item(cidx, (lane == 0 && tri[0]) ? 0 : 1, 1, 0);
  for (int j = lane; j < nB; j += 32) {
    if (j < nm)
      W.unl[W.lcap - 1 - (b[3] + j)] = coll_item(cidx, 0, 0, j);
    else
      W.unl[b[2] + j - nm] = coll_item(cidx, 0, 0, j);
  }
}

template <class R>
__global__ void __launch_bounds__(32 * kCollWarps) k_coll_prep(Ctx<R> X, const unsigned int *cend,
                                                                CollWork<R> W, double dtc) {
  __shared__ CollCell<R> cells[kCollWarps];
  const int wp = threadIdx.x >> 5;
  const int nl = W.n[4];
  // each warp takes every (number of warps)-th large cell
  for (int q = blockIdx.x * kCollWarps + wp; q < nl; q += gridDim.x * kCollWarps) {
    coll_prep_cell(X.d, X.lr, cells[wp], cend, W.list[W.ncell + q], W, dtc);
    __syncwarp();
  }
}

// Warp-aggregated append of k items per lane (all lanes take part).
__device__ __forceinline__ int reserve_items(int *count, int k) {
  const int lane = threadIdx.x & 31;
  int incl = k;
#pragma unroll
  for (int sft = 1; sft < 32; sft <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, sft);
    if (lane >= sft) incl += v;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  int base = 0;
  if (lane == 31 && total) base = atomicAdd(count, total);
  return __shfl_sync(0xffffffffu, base, 31) + incl - k;
}

// Small cells (2 .. kCollSmall particles): one thread each, the same
// ordering, statistics and work items as the warp version.
template <class R>
__global__ void __launch_bounds__(128) k_coll_prep_small(Ctx<R> X, const unsigned int *cend,
                                                         CollWork<R> W, double dtc) {
  const Dev<R> &D = X.d;
  const LayerR<R> *__restrict__ lr = X.lr;
  const int ns = W.n[0];
  const uint32_t step = (uint32_t)*D.step;
  const R ic = R(1.0 / kC), V = R(D.V_d), dt = R(dtc);
  const int stride = gridDim.x * blockDim.x;
  for (int t0 = blockIdx.x * blockDim.x; t0 < ns; t0 += stride) {
    const int t = t0 + threadIdx.x;
    const bool have = t < ns;
    int nl = 0, nu = 0, c = 0, cnt[2] = {0, 0};
    unsigned int st = 0;
    bool tri[2] = {false, false};
    int rest[2] = {0, 0};
    if (have) {
      c = W.list[t];
      st = c ? cend[c - 1] : 0u;
      const int n = (int)(cend[c] - st);
      uint32_t key[kCollSmall];
      unsigned long long id[kCollSmall];
      int sp[kCollSmall];
      R m[kCollSmall], w[kCollSmall], v[3][kCollSmall];
      for (int i = 0; i < n; ++i) {
        const unsigned long long p = st + i;
        id[i] = D.pid[p];
        key[i] = draw(D.seed, step, (uint32_t)id[i], (uint32_t)(id[i] >> 32), kStreamCollOrder).x;
        const uint32_t tg = D.ptag[p];
        sp[i] = (int)(tg & 1u);
        ++cnt[sp[i]];
        m[i] = lr[tg >> 1].mhat[sp[i]];
        w[i] = lr[tg >> 1].wmac;
        const R u0 = D.pu[0][p] * ic, u1 = D.pu[1][p] * ic, u2 = D.pu[2][p] * ic;
        const R g = sqrt(R(1) + (u0 * u0 + u1 * u1 + u2 * u2));
        v[0][i] = u0 / g;
        v[1][i] = u1 / g;
        v[2][i] = u2 / g;
      }
      int ordl[2][kCollSmall];
      for (int i = 0; i < n; ++i) {
        int r = 0;
        for (int j = 0; j < n; ++j)
          if (sp[j] == sp[i] && (key[j] < key[i] || (key[j] == key[i] && id[j] < id[i]))) ++r;
        ordl[sp[i]][r] = i;
        W.ord[st + (sp[i] ? cnt[0] : 0) + r] = (int)(st + i);
      }
      R ws[2] = {R(0), R(0)}, wm[2] = {R(0), R(0)}, Sv[2] = {R(0), R(0)};
      for (int i = 0; i < n; ++i) {
        ws[sp[i]] += w[i];
        wm[sp[i]] += w[i] * m[i];
        for (int j = i + 1; j < n; ++j) {
          if (sp[j] != sp[i]) continue;
          const R d0 = v[0][i] - v[0][j], d1 = v[1][i] - v[1][j], d2 = v[2][i] - v[2][j];
          Sv[sp[i]] += w[i] * w[j] * (d0 * d0 + d1 * d1 + d2 * d2);
        }
      }
      R dens[2], inv_l2 = R(0);
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        const R T = ws[g] > R(0) ? wm[g] / ws[g] * Sv[g] / (R(3) * ws[g] * ws[g]) : R(0);
        dens[g] = ws[g] / V;
        if (T > R(0)) inv_l2 += dens[g] * R(K_KD) / T;
      }
      const R ni = dens[1] > R(0) ? dens[1] : dens[0];
      const R ra = pow(R(4 * kPi / 3) * ni, R(-1) / R(3));
      const R lD = inv_l2 > R(0) ? fmax(R(1) / sqrt(inv_l2), ra) : ra;
      R ndu = R(0);
      if (cnt[0] > 0 && cnt[1] > 0) {
        const int A = cnt[0] >= cnt[1] ? 0 : 1, B = 1 - A;
        R nab = R(0);
        for (int i = 0; i < cnt[A]; ++i) nab += fmin(w[ordl[A][i]], w[ordl[B][i % cnt[B]]]) / V;
        ndu = dens[0] * (dens[1] / nab) * dt;
        nu = cnt[B];
      }
      int nlike[2];
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        tri[g] = cnt[g] >= 3 && (cnt[g] & 1);
        rest[g] = cnt[g] < 2 ? 0 : (tri[g] ? (cnt[g] - 3) / 2 : cnt[g] / 2);
        nlike[g] = cnt[g] < 2 ? 0 : (tri[g] ? 3 + rest[g] : rest[g]);
        nl += (tri[g] ? 1 : 0) + rest[g];
      }
      CollParam<R> P;
      P.st = st;
      P.cell = (unsigned)c;
      P.nE = cnt[0];
      P.nH = cnt[1];
      P.ndl[0] = dens[0] * dt;
      P.ndl[1] = dens[1] * dt;
      P.ndu = ndu;
      P.dens23[0] = pow(dens[0], R(2) / R(3));
      P.dens23[1] = pow(dens[1], R(2) / R(3));
      P.lD = lD;
      P.qu = (uint32_t)(nlike[0] + nlike[1]);
      W.par[c] = P;
    }
    // pairs and one-collision columns from the front of their lists,
    // triplets and longer columns from the back
    const int np = rest[0] + rest[1], nt = nl - np;
    const int nm = nu ? max(0, min(nu, max(cnt[0], cnt[1]) - nu)) : 0;
    int bp = reserve_items(W.n + 1, np);
    int bt = reserve_items(W.n + 3, nt);
    const int bs = reserve_items(W.n + 2, nu - nm);
    const int bm = reserve_items(W.n + 5, nm);
    if (have) {
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        if (tri[g]) W.like[W.lcap - 1 - bt++] = coll_item(c, g, 1, 0);
        for (int k = 0; k < rest[g]; ++k) W.like[bp++] = coll_item(c, g, 0, k);
      }
      for (int j = 0; j < nu; ++j) {
        if (j < nm)
          W.unl[W.lcap - 1 - (bm + j)] = coll_item(c, 0, 0, j);
        else
          W.unl[bs + j - nm] = coll_item(c, 0, 0, j);
      }
    }
  }
}

// Like pairs (one thread per pair) and triplets (one thread each, three
// pairs in order): the pairs first, then the triplets, so that warps do
// equal work.  Pair q: electrons' like pairs first, then the holes'.
template <class R>
__global__ void __launch_bounds__(256) k_coll_like(Ctx<R> X, CollWork<R> W, CollConst K) {
  const Dev<R> &D = X.d;
  const int npair = W.n[1], nitems = npair + W.n[3];
  const uint32_t step = (uint32_t)*D.step;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nitems; t += gridDim.x * blockDim.x) {
    const unsigned long long it = W.like[t < npair ? t : W.lcap - 1 - (t - npair)];
    const int cidx = (int)(unsigned)it, sp = (int)(it >> 32) & 1, tri = (int)(it >> 33) & 1;
    const int k = (int)(it >> 34) & 0xFFFF;
    const CollParam<R> P = W.par[cidx];
    const int m = sp ? P.nH : P.nE;
    const int *ord = W.ord + P.st + (sp ? P.nE : 0);
    const uint32_t q0 = sp ? (uint32_t)(P.nE < 2 ? 0 : ((P.nE & 1) ? 3 + (P.nE - 3) / 2 : P.nE / 2))
                           : 0u;
    if (tri) {
      const int a[3] = {0, 0, 1}, b[3] = {1, 2, 2};
      for (int r = 0; r < 3; ++r)
        collide_pool(D, X.lr, ord[a[r]], ord[b[r]], step, P.cell, q0 + r, R(0.5) * P.ndl[sp],
                     P.dens23[sp], P.dens23[sp], P.lD, K);
    } else {
      const int start = (m & 1) ? 3 : 0;
      collide_pool(D, X.lr, ord[start + 2 * k], ord[start + 2 * k + 1], step, P.cell,
                   q0 + start + k, P.ndl[sp], P.dens23[sp], P.dens23[sp], P.lD, K);
    }
  }
}

// Unlike pairs (A_i, B_{i mod |B|}), A the larger group: one thread per
// column j of B takes i = j, j + |B|, ... in order, which is the order of the
// rounds; columns share no particle.  Columns of one collision come first,
// then the longer ones.
template <class R>
__global__ void __launch_bounds__(256) k_coll_unlike(Ctx<R> X, CollWork<R> W, CollConst K) {
  const Dev<R> &D = X.d;
  const int n1 = W.n[2], nitems = n1 + W.n[5];
  const uint32_t step = (uint32_t)*D.step;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nitems; t += gridDim.x * blockDim.x) {
    const unsigned long long it = W.unl[t < n1 ? t : W.lcap - 1 - (t - n1)];
    const int cidx = (int)(unsigned)it, j = (int)(it >> 34) & 0xFFFF;
    const CollParam<R> P = W.par[cidx];
    const int A = P.nE >= P.nH ? 0 : 1;
    const int nA = A ? P.nH : P.nE, nB = A ? P.nE : P.nH;
    const int *oE = W.ord + P.st, *oH = W.ord + P.st + P.nE;
    const int *oA = A ? oH : oE, *oB = A ? oE : oH;
    for (int i = j; i < nA; i += nB) {
      const unsigned long long pA = oA[i], pB = oB[j];
      collide_pool(D, X.lr, A == 0 ? pA : pB, A == 0 ? pB : pA, step, P.cell, P.qu + i, P.ndu,
                   P.dens23[0], P.dens23[1], P.lD, K);
    }
  }
}

// Damage profiles: one block per node plane k sums the deposited n_e and
// energy density over the transverse node box [reg.x, reg.y) x [reg.z, reg.w)
// in a fixed order; out[2k], out[2k + 1].
__global__ void __launch_bounds__(256) k_profile(const double *ne, const double *ed, int nx, int ny,
                                                  int4 reg, double *out) {
  const long long base = (long long)blockIdx.x * nx * ny;
  const int w = reg.y - reg.x, n = w * (reg.w - reg.z);
  double a = 0.0, b = 0.0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const long long o = base + (long long)(reg.z + q / w) * nx + (reg.x + q % w);
    a += ne[o];
    b += ed[o];
  }
  const double sa = block_sum<double>(a);
  __syncthreads();
  const double sb = block_sum<double>(b);
  if (threadIdx.x == 0) {
    out[2 * blockIdx.x] = sa;
    out[2 * blockIdx.x + 1] = sb;
  }
}

// Largest recorded intensity on cell plane blockIdx.x.
template <class R>
__global__ void __launch_bounds__(256) k_imax_plane(const R *imax, int nxy, double *out) {
  const long long base = (long long)blockIdx.x * nxy;
  double m = 0.0;
  for (int q = threadIdx.x; q < nxy; q += blockDim.x) m = fmax(m, (double)imax[base + q]);
  const double v = block_max(m);
  if (threadIdx.x == 0) out[blockIdx.x] = v;
}

}  // namespace pg
