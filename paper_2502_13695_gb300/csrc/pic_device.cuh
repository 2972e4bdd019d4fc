// Device-side building blocks of the GB300 PIC library: physical constants,
// the per-simulation device view, Philox4x32-10, complete elliptic integrals,
// the Dawson integral and the Keldysh ionisation threshold.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pg {

// CODATA 2018
constexpr double kC = 299792458.0;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kMu0 = 1.0 / (kEps0 * kC * kC);
constexpr double kQe = 1.602176634e-19;
constexpr double kMe = 9.1093837015e-31;
constexpr double kHbar = 1.054571817e-34;
constexpr double kAmu = 1.66053906660e-27;
constexpr double kPi = 3.14159265358979323846;

enum : uint32_t {
  kStreamPos = 1u,
  kStreamVel = 2u,
  kStreamIon = 3u,
  kStreamIonLow = 4u,
  kStreamCollOrder = 5u,
  kStreamCollPair = 6u
};
enum : int { kErrPool = 1, kErrBadCell = 2, kErrColl = 4 };

// Per-layer constants, prepared on the host in double precision.
struct LayerK {
  double deps;      // Lorentz strength (or static eps - 1)
  double w0sq;      // pole frequency squared (unused when is_static)
  double damping;   // [rad/s]
  double wmac;      // real molecules per macroparticle
  double qm[2];     // charge / mass: electron, hole
  double mass[2];   // [kg]
  double kG;        // Keldysh gamma = kG / E
  double kX;        // x = kX * E(gamma2) / sqrt(gamma1)
  double kP;        // per-step rate = kP * gamma1^(-3/4) * Q * exp(-N a)
  double e_skip;    // amplitude below which the threshold is 0
  double sigv;      // neutral thermal speed per component [m/s]
  double gapJ;      // band gap [J]
  int is_static;
  int ppc;
};

// Device view of one simulation; passed by value to every kernel.
template <class R>
struct Dev {
  int nx, ny, nz, nxy;
  long long nfield, nmat, ncell;
  int NW, keldysh_terms, n_layers, pol;
  R dt, idx, idy, idz, alpha;
  R c2dt;                         // c^2 dt
  R dtdx, dtdy, dtdz;             // dt / dx ...
  double dt_d, V_d, dx_d, dy_d, dz_d;
  double E0, omega, fwhm, t_peak, cep;
  int shape;             // 0 Gaussian, 1 sine-squared envelope
  double Tsin2;          // full duration of the sine-squared field envelope
  double w0, xc, yc;     // spot radius (0: plane wave) and centre
  // fields: nfield each (E, B at integer time, Bh at the next half time),
  // J interleaved (Jx, Jy, Jz, 0) per point, nmat each (P, Q)
  R *E[3], *B[3], *Bh[3], *J4, *P[3], *Q[3];
  const int *layer_of_plane;      // nz, -1 vacuum
  const int *mplane;              // nz, -1 vacuum
  const int *kplane;              // n_mplanes: z plane of material plane
  const int *vplane;              // the other node planes 0 .. nz (no material)
  const LayerK *layers;
  // amplitude window and Keldysh threshold, per material cell
  R *win;                         // NW x nmat
  R *pm, *eamp, *ckey;
  unsigned long long *T;
  uint32_t *alive;
  uint32_t *leave_step;           // first step index at which a neutral may have left its cell
  // per material plane the stamp (step + 1) of the last window pass that
  // found a cell at or above its layer's skip amplitude (only such cells
  // can have a nonzero threshold); [n_mplanes] that pass's stamp, all ones
  // when the host has written the material since
  uint32_t *hot;
  // per cell plane the number of the field pass that must read the current
  // a push deposited from a particle in it (completed passes + 1); [nz]
  // nonzero when the host wrote the current (the next E step reads every
  // plane); [nz + 1] the number of completed field passes
  uint32_t *jtouch;
  // charged particles (SoA)
  int32_t *pcell;
  R *po[3], *pu[3];
  uint32_t *ptag;
  unsigned long long *pid;
  unsigned long long cap;
  unsigned long long *nslots;     // slots in use
  long long *step;                // device step counter
  // intensity map: per cell the largest recorded |E|^2 / E0^2, recorded when
  // (step + 1) % imax_every == 0 (0: never)
  R *imax;
  int imax_every;
  R inv_e0sq;
  const R *ktab;                  // elliptic tables (K, E interleaved), or null
  int ntab;
  // absorbing transverse layers of pml cells on each side of the x and y
  // seams (0: periodic): the convolution terms of the layer derivatives
  // (nfield each; order Ey/x, Ez/x, Ex/y, Ez/y, By/x, Bz/x, Bx/y, Bz/y) and
  // the decay factors b per position: [0] along x, [1] along y, at integer
  // positions over dt (E step) and half-integer ones over dt / 2 (B)
  int pml;
  R *psi[8];
  R *psi_close[4];  // the B terms after the closing half step of the last
                    // fused pass: a re-primed Bh (after a host write) takes
                    // the opening half step's convolution from here
  const R *pml_bE[2], *pml_bB[2];
  double *acc;                    // [0] joule [1] N_pairs [2] U_ion [3] events
                                  // [4] pushes
  // Poynting split: node planes (front, back), c eps0 dx dy dt, and each
  // block's running sums over the steps (2 planes x blocks per plane x
  // {fwd, bwd}; the diagnostics add them up)
  int flux_k[2];
  double flux_scale;
  double *flux_part;
  int *err;
  unsigned long long seed;
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two
// 32x32->64 multiplies with Weyl-sequence key bumps.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
#ifdef __CUDA_ARCH__
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
#else
    const uint64_t m0 = (uint64_t)0xD2511F53u * c.x, m1 = (uint64_t)0xCD9E8D57u * c.z;
    const uint32_t hi0 = (uint32_t)(m0 >> 32), lo0 = (uint32_t)m0;
    const uint32_t hi1 = (uint32_t)(m1 >> 32), lo1 = (uint32_t)m1;
#endif
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

__host__ __device__ __forceinline__ uint4 draw(unsigned long long seed, uint32_t step,
                                               uint32_t cell, uint32_t slot, uint32_t stream) {
  return philox4x32_10(make_uint4(step, cell, slot, stream),
                       make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

template <class R>
__host__ __device__ __forceinline__ R unit_open(uint32_t w) {
  return (R(w) + R(0.5)) * R(2.3283064365386963e-10);  // (w + 1/2) 2^-32
}

template <class R> struct Eps;
template <> struct Eps<double> {
  __host__ __device__ static constexpr double v() { return 1.1102230246251565e-16; }
};
template <> struct Eps<float> {
  __host__ __device__ static constexpr float v() { return 5.9604645e-08f; }
};

// ---------------------------------------------------------------------------
// Complete elliptic integrals K(m), K(m) - E(m) in the parameter convention,
// by the arithmetic-geometric mean with Legendre's sum of squared
// half-differences; m and its complement are both passed to keep precision.
// ---------------------------------------------------------------------------
template <class R>
__host__ __device__ __forceinline__ void ellip_k_kme(R m, R mc, R &K, R &KmE) {
  R a = R(1), b = sqrt(mc), s = R(0.5) * m, w = R(0.5);
  for (int it = 0; it < 16; ++it) {
    const R half_diff = R(0.5) * (a - b);
    const R mean = R(0.5) * (a + b);
    b = sqrt(a * b);
    a = mean;
    w += w;
    s += w * half_diff * half_diff;
    if (fabs(half_diff) <= R(4) * Eps<R>::v() * a) break;
  }
  K = R(kPi) / (R(2) * a);
  KmE = K * s;
}

// ---------------------------------------------------------------------------
// Dawson integral F(z), z >= 0, by Rybicki's exponential-sum method
// (G. B. Rybicki, Computers in Physics 3, 85 (1989)):
//   F(z) ~ (1/sqrt(pi)) sum_{k odd} exp(-(d - k h)^2) / (n0 + k),
// z = n0 h + d with n0 the even integer nearest z / h; a Taylor series near
// 0 and the asymptotic series sum (2k-1)!! / (2 z^2)^k / (2 z) for large z.
// ---------------------------------------------------------------------------
template <class R> struct DawsonCfg;
template <> struct DawsonCfg<double> {
  static constexpr double h = 0.25, z_small = 0.2, z_large = 8.0;
  static constexpr int pairs = 26, taylor = 10, asym = 20;
};
template <> struct DawsonCfg<float> {
  static constexpr float h = 0.4f, z_small = 0.2f, z_large = 5.0f;
  static constexpr int pairs = 7, taylor = 5, asym = 9;
};

template <class R>
__host__ __device__ __forceinline__ R dawson(R z) {
  using Cf = DawsonCfg<R>;
  if (z < R(Cf::z_small)) {
    // z (1 - (2z^2/3)(1 - (2z^2/5)(1 - ...)))
    const R t = R(2) * z * z;
    R s = R(1);
    for (int n = Cf::taylor; n >= 1; --n) s = R(1) - t / R(2 * n + 1) * s;
    return z * s;
  }
  if (z >= R(Cf::z_large)) {
    const R inv = R(1) / (R(2) * z * z);
    R s = R(1);
    for (int k = Cf::asym; k >= 1; --k) s = R(1) + R(2 * k - 1) * inv * s;
    return s / (R(2) * z);
  }
  const R h = R(Cf::h);
  const R n0 = R(2) * rint(z / (R(2) * h));
  const R d = z - n0 * h;
  R s = R(0);
  for (int q = Cf::pairs - 1; q >= 0; --q) {
    const R k = R(2 * q + 1);
    const R a = d - k * h, b = d + k * h;
    s += exp(-a * a) / (n0 + k) + exp(-b * b) / (n0 - k);
  }
  return s * R(0.56418958354775628);  // 1/sqrt(pi)
}

// FP32 evaluation on the device: piecewise degree-8 polynomials on
// [0.2, 5) (generated by gen_dawson_f32.py, 1.3e-7 relative), the series
// above elsewhere.  FP64 keeps the exponential-sum method everywhere.
#include "dawson_f32_table.inc"

template <class R>
__host__ __device__ __forceinline__ R dawson_w(R z) {
  return dawson<R>(z);
}
template <>
__host__ __device__ __forceinline__ float dawson_w<float>(float z) {
#ifdef __CUDA_ARCH__
  if (z >= PG_DAWSON_LO && z < 5.0f) {
    const float u = (z - PG_DAWSON_LO) * PG_DAWSON_INV_W;
    const int iv = min((int)u, PG_DAWSON_NINT - 1);
    const float t = 2.0f * (u - (float)iv) - 1.0f;
    const float *c = kDawsonF32[iv];
    float acc = c[PG_DAWSON_DEG];
#pragma unroll
    for (int q = PG_DAWSON_DEG - 1; q >= 0; --q) acc = fmaf(acc, t, c[q]);
    return acc;
  }
#endif
  return dawson<float>(z);
}

// Dawson's F at z = sqrt(y), y > 0, for the Keldysh series (which has y).
// FP32 on the device: r = rsqrt(y); below z = 5 the table at z = y r (the
// rsqrt is within a few ulp; the table is good to 1.3e-7); from z = 5 the
// asymptotic series with 1/(2 z^2) = r^2 / 2 and 1/(2 z) = r / 2, so with no
// division.  Elsewhere the correctly rounded root and dawson_w.
template <class R>
__host__ __device__ __forceinline__ R dawson_of_square(R y) {
  return dawson_w<R>(sqrt(y));
}
template <>
__host__ __device__ __forceinline__ float dawson_of_square<float>(float y) {
#ifdef __CUDA_ARCH__
  const float r = rsqrtf(y);
  if (y >= 25.0f) {
    const float inv = 0.5f * r * r;
    float s = 1.0f;
#pragma unroll
    for (int k = DawsonCfg<float>::asym; k >= 1; --k) s = fmaf(float(2 * k - 1) * inv, s, 1.0f);
    return s * (0.5f * r);
  }
  return dawson_w<float>(y * r);
#else
  return dawson_w<float>(sqrtf(y));
#endif
}

// ---------------------------------------------------------------------------
// Keldysh threshold (Sec. 2.1, corrected form) for one cell:
//   gamma = kG / E, gamma1 = g^2/(1+g^2), gamma2 = 1/(1+g^2),
//   x = kX E(gamma2)/sqrt(gamma1), N = floor(x+1), a = pi (K-E)(g1)/E(g2),
//   Q = sqrt(pi/(2K(g2))) sum_n e^{-n a} F(sqrt(pi^2 (N - x + n)/(2 K(g2) E(g2)))),
//   rate dt / n_mol = kP gamma1^(-3/4) Q e^{-N a},  p = -expm1(-rate),
//   T = floor(p 2^64), or ~0 (all ones) when p rounds to 1.
// The series stops once the remaining tail, bounded by term * r/(1-r) with
// r = e^{-a} (every later Dawson factor is smaller past the maximum of F),
// is below half an ulp of the sum, or after `nterms` terms.
// ---------------------------------------------------------------------------
// K and K - E from an N-point table (K(i/N), E(i/N) interleaved, i < N;
// linear in m between neighbouring entries) while m lies inside it, else by
// the AGM.
template <class R>
__host__ __device__ __forceinline__ void ellip_tab_k_kme(R m, R mc, const R *tab, int ntab, R &K,
                                                         R &KmE) {
  if (tab) {
    const R u = m * R(ntab);
    const R fi = floor(u);
    if (fi >= R(0) && fi < R(ntab - 1)) {
      const int i = (int)fi;
      const R f = u - fi;
      const R k = tab[2 * i] + f * (tab[2 * i + 2] - tab[2 * i]);
      const R e = tab[2 * i + 1] + f * (tab[2 * i + 3] - tab[2 * i + 1]);
      K = k;
      KmE = k - e;
      return;
    }
  }
  ellip_k_kme(m, mc, K, KmE);
}

template <class R>
__host__ __device__ inline R keldysh_probability(R E, const LayerK &L, int nterms,
                                                 int *terms_out = nullptr,
                                                 const R *tab = nullptr, int ntab = 0) {
  if (terms_out) *terms_out = 0;
  if (!(E > R(0))) return R(0);
  const R g = R(L.kG) / E;
  const R g2 = g * g;
  if (!(g2 < R(1e30))) return R(0);
  const R gam1 = g2 / (R(1) + g2), gam2 = R(1) / (R(1) + g2);
  R K1, KmE1, K2, KmE2;
  ellip_tab_k_kme(gam1, gam2, tab, ntab, K1, KmE1);
  ellip_tab_k_kme(gam2, gam1, tab, ntab, K2, KmE2);
  const R E2 = K2 - KmE2;
  const R x = R(L.kX) * E2 / sqrt(gam1);
  const R N = floor(x + R(1));
  const R a = R(kPi) * KmE1 / E2;
  const R r = exp(-a);
  const R tail = r / (R(1) - r);
  const R cd = R(kPi * kPi) / (R(2) * K2 * E2);
  const R base = N - x;
  R sum = R(0), rn = R(1);
  int n = 0;
  for (; n < nterms; ++n) {
    const R y = cd * (base + R(n));  // the Dawson argument squared
    const R term = rn * dawson_of_square<R>(y);
    sum += term;
    if (y > R(0.85414564) && term * tail <= R(0.5) * Eps<R>::v() * sum) {  // z > 0.9242
      ++n;
      break;
    }
    rn *= r;
  }
  if (terms_out) *terms_out = n;
  const R Q = sqrt(R(kPi) / (R(2) * K2)) * sum;
  const R rate = R(L.kP) * pow(gam1, R(-0.75)) * Q * exp(-N * a);
  return -expm1(-rate);
}

template <class R>
__host__ __device__ inline unsigned long long keldysh_threshold(R E, const LayerK &L, int nterms,
                                                                int *terms_out = nullptr,
                                                                const R *tab = nullptr,
                                                                int ntab = 0) {
  const R p = keldysh_probability<R>(E, L, nterms, terms_out, tab, ntab);
  if (!(p < R(1))) return ~0ull;
  const double scaled = (double)p * 18446744073709551616.0;  // exact: power of 2
  return (unsigned long long)scaled;
}

}  // namespace pg
