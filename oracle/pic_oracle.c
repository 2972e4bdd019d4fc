/*
 * FP64 CPU oracle for the per-timestep 3D particle-in-cell cycle of a
 * few-cycle laser pulse driving a dielectric (Smith et al., arXiv 2502.13695).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA library; the CUDA library never
 * loads it.
 *
 * Plain loops in the order the step is defined, all arithmetic in double:
 *   particle pass  : TSC gather (Sec. 4.1 "shape function"), relativistic Boris
 *                    push, Esirkepov charge-conserving deposit, z outflow and
 *                    outflow into the absorbing transverse layers
 *   field pass     : Yee update with a Lorentz polarisation current (Sec. 2.3,
 *                    refraction) advanced by a Crank-Nicolson oscillator step,
 *                    laser injected through a Silver-Mueller boundary (Sec. 3),
 *                    optional convolutional PML layers at the x and y seams
 *                    (the outflow transverse faces of Sec. 3.1)
 *   amplitude      : maximum of |E| over the last optical cycle (Sec. 2.1,
 *                    rolling window)
 *   Keldysh rate   : Sec. 2.1, Eqs. for x, W and Q, first 500 terms of Q;
 *                    K and E in situ or from N-point tables (Sec. 2.1)
 *   ionisation     : one event per molecule (Sec. 2.1), electron + hole with
 *                    the Table 1 effective masses (Sec. 3.2)
 *   diagnostics    : energies, TSC number and energy density (Sec. 4.1-4.2),
 *                    spectra (Sec. 4.3), Gauss residual, and the Poynting
 *                    split into +z and -z waves at two planes
 * Counter-based Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) supplies
 * every random number, keyed by (seed) with counter (step, cell, slot, stream).
 * A neutral's 64-bit ionisation uniform takes its top 16 bits from the block
 * (step, cell, slot >> 3, 3) shared by eight slots and its low 48 bits from
 * the block (step, cell, slot, 4) (or_ion_uniform).
 *
 * Parity pins for every function here live in tests/test_oracle_*.py.
 *
 * The same source also builds with OpenMP (liboracle_omp.so), used only to
 * time the oracle on all host cores: the loops whose iterations write
 * disjoint data (the field updates and the intensity record over z planes,
 * the window and Keldysh pass over material planes) then run in parallel;
 * the particle and ionisation passes stay serial.  Only the summation order
 * of the Joule work differs from the serial build.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_C 299792458.0
#define OR_EPS0 8.8541878128e-12
#define OR_MU0 (1.0 / (OR_EPS0 * OR_C * OR_C))
#define OR_QE 1.602176634e-19
#define OR_ME 9.1093837015e-31
#define OR_HBAR 1.054571817e-34
#define OR_AMU 1.66053906660e-27
#define OR_PI 3.14159265358979323846

#define OR_MAX_LAYERS 128
#define OR_STREAM_POS 1u
#define OR_STREAM_VEL 2u
#define OR_STREAM_ION 3u
#define OR_STREAM_ION_LOW 4u
#define OR_STREAM_COLL_ORDER 5u
#define OR_STREAM_COLL_PAIR 6u

/* ------------------------------------------------------------------------ */
/* Configuration (mirrors the library's inputs, declared independently)     */
/* ------------------------------------------------------------------------ */
typedef struct {
  int z0, z1; /* layer occupies z cells [z0, z1) */
  int ppc;    /* neutral macroparticles per cell */
  int pad_;
  double n_index;      /* refractive index at the laser wavelength */
  double gap_eV;       /* band gap (Table 1) */
  double me_star;      /* electron effective mass / m_e (Table 1) */
  double mh_star;      /* hole effective mass / m_e (Table 1) */
  double n_mol;        /* molecular density [m^-3] */
  double omega0_eV;    /* Lorentz pole photon energy; INFINITY = static eps */
  double damping;      /* Lorentz damping [rad/s] */
  double temp_eV;      /* neutral temperature */
  double mol_mass_amu; /* molecular mass */
  double e_melt, e_boil, e_dissoc; /* damage energy densities [J/m^3], 0 = none */
} or_layer;

typedef struct {
  int nx, ny, nz, pol;
  double dx, dy, dz, cfl;
  double lambda, fwhm, fluence, cep, t_peak;
  uint64_t seed;
  int keldysh_terms;
  int n_layers;
  int imax_every; /* intensity record interval in steps: 0 = 0.5 fs, < 0 off */
  int coll_every; /* steps between binary-collision passes, 0 = none */
  int shape;      /* temporal envelope: 0 Gaussian, 1 sine-squared (Sec. 3) */
  int elliptic_table; /* 0: K and E in situ; N >= 2: read from N-point tables */
  double w0;      /* Gaussian spot radius (1/e^2 of the intensity), 0 = plane wave */
  int pml_cells;  /* 0: periodic x and y; L > 0: absorbing layers of L cells on each
                     side of the x and y seams, particles entering them removed */
  int pad_pml;
  or_layer layers[OR_MAX_LAYERS];
} or_config;

typedef struct {
  double U_incident, U_kinetic, U_ionization, U_absorbed, frac_absorbed;
  double U_joule, U_field, N_pairs, n_e_peak, energy_density_peak;
  double gauss_residual_max, rho_max;
  double n_electrons_macro, n_holes_macro, step;
  /* Poynting split (reading K17): node planes, time integrals of the +z and
   * -z wave power through each, and the balance they give */
  double flux_front, flux_back;
  double U_fwd_front, U_bwd_front, U_fwd_back, U_bwd_back;
  double frac_reflected, frac_transmitted, frac_absorbed_flux;
} or_diag;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10                                                             */
/* ------------------------------------------------------------------------ */
void or_philox(const uint32_t ctr_in[4], const uint32_t key_in[2],
               uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; r++) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

static void philox_draw(uint64_t seed, uint32_t step, uint32_t cell,
                        uint32_t slot, uint32_t stream, uint32_t out[4]) {
  uint32_t ctr[4] = {step, cell, slot, stream};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  or_philox(ctr, key, out);
}

static double u01(uint32_t w) { return ((double)w + 0.5) * 0x1p-32; }

/* The uniform 64-bit number a neutral draws at a step: bits 63..48 are the
 * 16-bit half (slot & 1: high half) of word (slot & 7) >> 1 of the block
 * (step, cell, slot >> 3, ION); bits 47..0 are the low 16 bits of word 1
 * above word 0 of the block (step, cell, slot, ION_LOW).  It ionises when it
 * is below the threshold T = floor(p 2^64). */
uint64_t or_ion_uniform(uint64_t seed, uint32_t step, uint32_t cell, uint32_t slot) {
  uint32_t a[4], b[4];
  philox_draw(seed, step, cell, slot >> 3, OR_STREAM_ION, a);
  philox_draw(seed, step, cell, slot, OR_STREAM_ION_LOW, b);
  uint32_t w = a[(slot & 7u) >> 1];
  uint64_t hi16 = (slot & 1u) ? (w >> 16) : (w & 0xFFFFu);
  uint64_t lo48 = ((uint64_t)(b[1] & 0xFFFFu) << 32) | (uint64_t)b[0];
  return (hi16 << 48) | lo48;
}

/* ------------------------------------------------------------------------ */
/* Complete elliptic integrals, parameter convention (reading K1):           */
/*   K(m) = int_0^{pi/2} (1 - m sin^2 t)^(-1/2) dt, E(m) likewise.           */
/* Gauss arithmetic-geometric mean with the Legendre sum (DLMF 19.8.1 and     */
/* 19.8.6): K = pi / (2 AGM(1, sqrt(1-m))), K - E = K * sum 2^(n-1) c_n^2.    */
/* The complementary parameter mc = 1 - m is passed separately so that both   */
/* ends of [0, 1] keep full precision.                                        */
/* ------------------------------------------------------------------------ */
void or_ellip_KE(double m, double mc, double *K, double *KmE) {
  double a = 1.0, b = sqrt(mc);
  double pw = 0.5, sum = 0.5 * m; /* n = 0 term: 2^-1 c_0^2, c_0^2 = m */
  for (int it = 0; it < 64; it++) {
    double an = 0.5 * (a + b);
    double bn = sqrt(a * b);
    double cn = 0.5 * (a - b);
    pw *= 2.0;
    sum += pw * cn * cn;
    a = an;
    b = bn;
    if (fabs(cn) <= 1e-15 * a) break; /* later terms are below roundoff */
  }
  *K = OR_PI / (2.0 * a);
  *KmE = *K * sum;
}

/* ------------------------------------------------------------------------ */
/* Dawson integral  F(z) = exp(-z^2) int_0^z exp(y^2) dy  (Sec. 2.1 Phi).    */
/*   |z| < 7   : exp(-z^2) * sum_n z^(2n+1) / (n! (2n+1)), which is the      */
/*               term-by-term integral of exp(y^2); every term is positive,   */
/*               summed with compensation.                                   */
/*   |z| >= 7  : asymptotic series (1/2z) sum_k (2k-1)!! / (2 z^2)^k, cut     */
/*               once a term is below 2^-60 of the sum, which happens before */
/*               the smallest term (about 1e-20 relative at z = 7).          */
/* ------------------------------------------------------------------------ */
double or_dawson(double z) {
  double az = fabs(z), r;
  if (az == 0.0) return 0.0;
  if (az < 7.0) {
    double z2 = az * az, t = az, s = 0.0, comp = 0.0;
    for (int n = 0; n < 2000; n++) {
      double term = t / (2.0 * n + 1.0);
      double y = term - comp;
      double ts = s + y;
      comp = (ts - s) - y;
      s = ts;
      if ((double)n > z2 && term < 1e-19 * s) break;
      t *= z2 / (double)(n + 1);
    }
    r = s * exp(-z2);
  } else {
    double inv = 1.0 / (2.0 * az * az), term = 1.0, s = 1.0;
    for (int k = 1; k < 400 && (double)k < az * az; k++) {
      term *= (2.0 * k - 1.0) * inv;
      s += term;
      if (term < 0x1p-60 * s) break;
    }
    r = s / (2.0 * az);
  }
  return z < 0 ? -r : r;
}

/* ------------------------------------------------------------------------ */
/* Keldysh photoionisation rate W [m^-3 s^-1], Sec. 2.1 (corrected form).    */
/*   gamma = omega sqrt(m* Delta) / (e E),  gamma1 = g^2/(1+g^2),            */
/*   gamma2 = 1/(1+g^2),                                                     */
/*   x = (2/pi) (Delta / hbar omega) eps(gamma2) / sqrt(gamma1),             */
/*   W = 2 (2 omega / 9 pi) (m* omega / (hbar sqrt(gamma1)))^(3/2)           */
/*       Q(gamma, x) exp(-pi floor(x+1) (K(g1) - E(g1)) / E(g2)),            */
/*   Q = sqrt(pi / (2 K(g2))) sum_{n>=0} exp(-n pi (K(g1)-E(g1))/E(g2))      */
/*       Phi( sqrt( pi^2 (floor(x+1) - x + n) / (2 K(g2) E(g2)) ) ).          */
/* The sum takes the first nterms terms (500 in Sec. 2.1).  It stops earlier  */
/* only once the Dawson argument is past the maximum of Phi (so every later   */
/* term is smaller) and the current term is below a quarter ulp of the sum,   */
/* where adding it, or any later term, leaves the double sum unchanged: the    */
/* result is bit-identical to summing all nterms terms.                       */
/* ------------------------------------------------------------------------ */
/* Keldysh rate W (returned) and, when parts is not NULL, its pieces:
 * parts[0] = gamma, [1] = x, [2] = floor(x + 1), [3] = Q(gamma, x). */
/* The paper reads K and E from tabulated data files of 1000 points (Sec.
 * 2.1); their range, spacing and interpolation are not given.  Reading:
 * tabK[i] = K(i / N), tabE[i] = E(i / N) for i = 0 .. N - 1 (N = 1000 in the
 * paper), linear interpolation in m between the two neighbouring entries,
 * and, past the last entry (m > 1 - 1/N, where K diverges logarithmically
 * and no finite table reaches), the in-situ value.  Returns K and K - E as
 * or_ellip_KE does. */
void or_ellip_table(const double *tabK, const double *tabE, int N, double m, double mc,
                    double *K, double *KmE) {
  double u = m * (double)N;
  double fi = floor(u);
  if (tabK && N >= 2 && fi >= 0.0 && fi < (double)(N - 1)) {
    int i = (int)fi;
    double f = u - fi;
    double k = tabK[i] + f * (tabK[i + 1] - tabK[i]);
    double e = tabE[i] + f * (tabE[i + 1] - tabE[i]);
    *K = k;
    *KmE = k - e;
    return;
  }
  or_ellip_KE(m, mc, K, KmE);
}

static double keldysh_rate(double E, double omega, double gap_J, double mstar_kg, int nterms,
                           int *terms_used, double parts[4], const double *tabK,
                           const double *tabE, int ntab);

double or_keldysh_parts(double E, double omega, double gap_J, double mstar_kg,
                        int nterms, int *terms_used, double parts[4]) {
  return keldysh_rate(E, omega, gap_J, mstar_kg, nterms, terms_used, parts, NULL, NULL, 0);
}

/* The rate with K and E from N-point tables (or_ellip_table). */
double or_keldysh_W_table(double E, double omega, double gap_J, double mstar_kg, int nterms,
                          const double *tabK, const double *tabE, int ntab) {
  return keldysh_rate(E, omega, gap_J, mstar_kg, nterms, NULL, NULL, tabK, tabE, ntab);
}

static double keldysh_rate(double E, double omega, double gap_J, double mstar_kg, int nterms,
                           int *terms_used, double parts[4], const double *tabK,
                           const double *tabE, int ntab) {
  if (terms_used) *terms_used = 0;
  if (parts) parts[0] = parts[1] = parts[2] = parts[3] = 0.0;
  if (!(E > 0.0)) return 0.0;
  double g = omega * sqrt(mstar_kg * gap_J) / (OR_QE * E);
  double g2 = g * g;
  if (parts) parts[0] = g;
  if (!(g2 < 1e300)) return 0.0;
  double gam1 = g2 / (1.0 + g2), gam2 = 1.0 / (1.0 + g2);
  double K1, KmE1, K2, KmE2;
  or_ellip_table(tabK, tabE, ntab, gam1, gam2, &K1, &KmE1);
  or_ellip_table(tabK, tabE, ntab, gam2, gam1, &K2, &KmE2);
  double E2 = K2 - KmE2;
  double x = (2.0 / OR_PI) * (gap_J / (OR_HBAR * omega)) * E2 / sqrt(gam1);
  double N = floor(x + 1.0);
  double a = OR_PI * KmE1 / E2;
  double cd = OR_PI * OR_PI / (2.0 * K2 * E2);
  double sum = 0.0;
  int n;
  for (n = 0; n < nterms; n++) {
    double arg = sqrt(cd * (N - x + (double)n));
    double term = exp(-(double)n * a) * or_dawson(arg);
    if (arg > 0.9241 && sum > 0.0) {
      double ulp = nextafter(sum, INFINITY) - sum;
      if (term < 0.25 * ulp) break;
    }
    sum += term;
  }
  if (terms_used) *terms_used = n;
  double Q = sqrt(OR_PI / (2.0 * K2)) * sum;
  if (parts) {
    parts[1] = x;
    parts[2] = N;
    parts[3] = Q;
  }
  double pref = 2.0 * (2.0 * omega / (9.0 * OR_PI)) *
                pow(mstar_kg * omega / (OR_HBAR * sqrt(gam1)), 1.5);
  return pref * Q * exp(-N * a);
}

double or_keldysh_W(double E, double omega, double gap_J, double mstar_kg,
                    int nterms, int *terms_used) {
  return or_keldysh_parts(E, omega, gap_J, mstar_kg, nterms, terms_used, NULL);
}

/* Probability that one molecule ionises in one step (reading K5):
 * p = 1 - exp(-(W / n_mol) dt); threshold T = floor(p 2^64), or "always"
 * when p reaches 1 (reading K16). */
static void ion_threshold(double W, double n_mol, double dt, uint64_t *T,
                          uint8_t *always) {
  double p = -expm1(-(W / n_mol) * dt);
  if (p >= 1.0) {
    *T = UINT64_MAX;
    *always = 1;
  } else {
    *T = (uint64_t)floor(ldexp(p, 64));
    *always = 0;
  }
}

/* ------------------------------------------------------------------------ */
/* Relativistic Boris push (u = gamma v), uniform E, B at the particle.      */
/* ------------------------------------------------------------------------ */
void or_boris(double qm, double dt, const double E[3], const double B[3],
              double u[3]) {
  double h = 0.5 * qm * dt;
  double um[3] = {u[0] + h * E[0], u[1] + h * E[1], u[2] + h * E[2]};
  double gm = sqrt(1.0 + (um[0] * um[0] + um[1] * um[1] + um[2] * um[2]) /
                             (OR_C * OR_C));
  double t[3] = {h * B[0] / gm, h * B[1] / gm, h * B[2] / gm};
  double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
  double s[3] = {2.0 * t[0] / (1.0 + t2), 2.0 * t[1] / (1.0 + t2),
                 2.0 * t[2] / (1.0 + t2)};
  double up[3] = {um[0] + (um[1] * t[2] - um[2] * t[1]),
                  um[1] + (um[2] * t[0] - um[0] * t[2]),
                  um[2] + (um[0] * t[1] - um[1] * t[0])};
  double upl[3] = {um[0] + (up[1] * s[2] - up[2] * s[1]),
                   um[1] + (up[2] * s[0] - up[0] * s[2]),
                   um[2] + (up[0] * s[1] - up[1] * s[0])};
  u[0] = upl[0] + h * E[0];
  u[1] = upl[1] + h * E[1];
  u[2] = upl[2] + h * E[2];
}

/* Quadratic (TSC) weights for one axis.  'half' selects the grid of
 * half-integer nodes.  Returns the node (relative to the particle's cell
 * index) that carries w[0]; w[1], w[2] sit on the next two nodes. */
static int tsc(double delta, int half, double w[3]) {
  int base;
  double d;
  if (half) {
    d = delta - 0.5;
    base = -1;
  } else {
    int s = delta >= 0.5;
    d = delta - (double)s;
    base = s - 1;
  }
  w[0] = 0.5 * (0.5 - d) * (0.5 - d);
  w[1] = 0.75 - d * d;
  w[2] = 0.5 * (0.5 + d) * (0.5 + d);
  return base;
}

/* ------------------------------------------------------------------------ */
/* Simulation state                                                          */
/* ------------------------------------------------------------------------ */
enum { FEX, FEY, FEZ, FBX, FBY, FBZ, FJX, FJY, FJZ, FPX, FPY, FPZ, FQX, FQY,
       FQZ, NCOMP };
/* staggering (x, y, z) of each E/B/J component: 1 = half-integer position */
static const int stag_E[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
static const int stag_B[3][3] = {{0, 1, 1}, {1, 0, 1}, {1, 1, 0}};

typedef struct {
  or_config cfg;
  double dt, omega, alpha, E0, V;
  int NW, nxy;
  long nfield, nmat;
  double *F[NCOMP];
  int *layer_of_plane, *mplane;
  double *win, *eamp;
  uint64_t *T;
  uint8_t *Talways;
  uint32_t *alive;
  /* per layer */
  double deps[OR_MAX_LAYERS], kosc[OR_MAX_LAYERS], wmac[OR_MAX_LAYERS];
  double qm[OR_MAX_LAYERS][2], mass[OR_MAX_LAYERS][2];
  double mstar[OR_MAX_LAYERS], gapJ[OR_MAX_LAYERS], sigv[OR_MAX_LAYERS];
  int is_static[OR_MAX_LAYERS];
  /* charged macroparticles */
  long np, cap;
  uint64_t *pid;
  int32_t *pcell;
  double *poff, *pu;
  uint32_t *ptag;
  long step;
  double U_joule, N_pairs, U_ion, n_events;
  /* maximum over the recorded steps of |E|^2 / E0^2 at each cell centre */
  double *imax;
  int imax_every;
  double Tsin2; /* full duration of the sine-squared field envelope */
  /* Poynting split: node planes (front, back) and the time integrals of
   * the +z (fwd) and -z (bwd) wave power through them */
  int flux_plane[2];
  double U_fwd[2], U_bwd[2];
  /* elliptic tables (elliptic_table > 0): K(i / N), E(i / N) */
  double *tabK, *tabE;
  int ntab;
  /* absorbing transverse layers: the convolution terms of the x and y
   * derivatives in the curl (pml_cells > 0) */
  double *psi[8];
} or_sim;

enum { PEYX, PEZX, PEXY, PEZY, PBYX, PBZX, PBXY, PBZY };

static long fidx(const or_sim *s, int i, int j, int k) {
  int nx = s->cfg.nx, ny = s->cfg.ny;
  i %= nx;
  if (i < 0) i += nx;
  j %= ny;
  if (j < 0) j += ny;
  return ((long)k * ny + j) * nx + i;
}

static void grow(or_sim *s, long need) {
  if (need <= s->cap) return;
  long nc = s->cap ? s->cap : 1024;
  while (nc < need) nc *= 2;
  s->pid = realloc(s->pid, nc * sizeof(uint64_t));
  s->pcell = realloc(s->pcell, nc * sizeof(int32_t));
  s->poff = realloc(s->poff, 3 * nc * sizeof(double));
  s->pu = realloc(s->pu, 3 * nc * sizeof(double));
  s->ptag = realloc(s->ptag, nc * sizeof(uint32_t));
  s->cap = nc;
}

/* Incident field at the z_min plane (Sec. 3), at the spot centre: a
 * Gaussian intensity envelope of FWHM tau (reading K14), or the paper's
 * sine-squared pulse read as the field envelope cos^2(pi (t - t_peak) / T)
 * on |t - t_peak| < T / 2, whose intensity (cos^4) has FWHM tau; E0 from
 * the peak fluence F = int c eps0 E^2 dt. */
static double e_inc(const or_sim *s, double t) {
  double tau = s->cfg.fwhm, tt = t - s->cfg.t_peak, env;
  if (s->cfg.shape == 1) {
    double x = OR_PI * tt / s->Tsin2;
    env = fabs(tt) < 0.5 * s->Tsin2 ? cos(x) * cos(x) : 0.0;
  } else {
    env = exp(-2.0 * log(2.0) * tt * tt / (tau * tau));
  }
  return s->E0 * env * cos(s->omega * tt + s->cfg.cep);
}

/* Transverse profile of the incident field, exp(-r^2 / w0^2) about the box
 * centre (the spot radius of Sec. 3, where F = 2 E_las / (pi w0^2) is the
 * peak fluence); 1 for a plane wave. */
double or_spot(const or_sim *s, double x, double y) {
  if (!(s->cfg.w0 > 0.0)) return 1.0;
  double xc = 0.5 * s->cfg.nx * s->cfg.dx, yc = 0.5 * s->cfg.ny * s->cfg.dy;
  double r2 = (x - xc) * (x - xc) + (y - yc) * (y - yc);
  return exp(-r2 / (s->cfg.w0 * s->cfg.w0));
}

or_sim *or_create(const or_config *cfg) {
  const int nx = cfg->nx, ny = cfg->ny, nz = cfg->nz;
  if (nx < 4 || ny < 4 || nz < 8 || cfg->n_layers < 0 ||
      cfg->n_layers > OR_MAX_LAYERS || cfg->pml_cells < 0 || 2 * cfg->pml_cells >= nx ||
      2 * cfg->pml_cells >= ny)
    return NULL;
  or_sim *s = calloc(1, sizeof(or_sim));
  s->cfg = *cfg;
  s->nxy = nx * ny;
  s->nfield = (long)s->nxy * (nz + 1);
  s->dt = cfg->cfl / (OR_C * sqrt(1.0 / (cfg->dx * cfg->dx) +
                                  1.0 / (cfg->dy * cfg->dy) +
                                  1.0 / (cfg->dz * cfg->dz)));
  s->omega = 2.0 * OR_PI * OR_C / cfg->lambda;
  s->alpha = OR_C * s->dt / cfg->dz;
  s->V = cfg->dx * cfg->dy * cfg->dz;
  s->NW = (int)ceil(cfg->lambda / (OR_C * s->dt));
  /* cos^4 falls to one half at pi t / T = acos(2^(-1/4)) */
  s->Tsin2 = cfg->fwhm / (2.0 * acos(pow(2.0, -0.25)) / OR_PI);
  if (cfg->shape == 1) /* int cos^4 over the pulse = 3 T / 8 */
    s->E0 = sqrt(16.0 * cfg->fluence / (3.0 * OR_C * OR_EPS0 * s->Tsin2));
  else
    s->E0 = sqrt(2.0 * cfg->fluence /
                 (OR_C * OR_EPS0 * cfg->fwhm * sqrt(OR_PI / (4.0 * log(2.0)))));
  for (int c = 0; c < NCOMP; c++) s->F[c] = calloc(s->nfield, sizeof(double));
  s->layer_of_plane = malloc(nz * sizeof(int));
  s->mplane = malloc(nz * sizeof(int));
  for (int k = 0; k < nz; k++) s->layer_of_plane[k] = -1;
  for (int L = 0; L < cfg->n_layers; L++) {
    const or_layer *ly = &cfg->layers[L];
    if (ly->z0 < 2 || ly->z1 > nz - 2 || ly->z0 >= ly->z1 || ly->ppc < 1 ||
        ly->ppc > 32) {
      free(s);
      return NULL;
    }
    for (int k = ly->z0; k < ly->z1; k++) s->layer_of_plane[k] = L;
    /* Lorentz pole at the band gap with the strength that gives the stated
     * index at the laser frequency (reading K9); static eps when the pole is
     * at infinity (Sec. 2.3). */
    double n2m1 = ly->n_index * ly->n_index - 1.0;
    if (isinf(ly->omega0_eV)) {
      s->is_static[L] = 1;
      s->deps[L] = n2m1;
      s->kosc[L] = INFINITY;
    } else {
      double w0 = ly->omega0_eV * OR_QE / OR_HBAR;
      s->is_static[L] = 0;
      s->deps[L] = n2m1 * (1.0 - s->omega * s->omega / (w0 * w0));
      s->kosc[L] = w0 * w0;
    }
    s->wmac[L] = ly->n_mol * s->V / ly->ppc;
    s->mass[L][0] = ly->me_star * OR_ME;
    s->mass[L][1] = ly->mh_star * OR_ME;
    s->qm[L][0] = -OR_QE / s->mass[L][0];
    s->qm[L][1] = OR_QE / s->mass[L][1];
    s->mstar[L] = OR_ME / (1.0 / ly->me_star + 1.0 / ly->mh_star);
    s->gapJ[L] = ly->gap_eV * OR_QE;
    s->sigv[L] = sqrt(ly->temp_eV * OR_QE / (ly->mol_mass_amu * OR_AMU));
  }
  int nm = 0;
  for (int k = 0; k < nz; k++)
    s->mplane[k] = s->layer_of_plane[k] >= 0 ? nm++ : -1;
  /* Poynting planes: halfway between the entrance face and the first
   * material plane, and halfway between the last one and the far face
   * (a quarter and three quarters of the box without material), inside
   * 1 .. nz - 1 so that the B planes on both sides exist */
  {
    int zlo = -1, zhi = -1;
    for (int k = 0; k < nz; k++)
      if (s->layer_of_plane[k] >= 0) {
        if (zlo < 0) zlo = k;
        zhi = k + 1;
      }
    int f = zlo < 0 ? nz / 4 : zlo / 2;
    int b = zlo < 0 ? (3 * nz) / 4 : (zhi + nz) / 2;
    s->flux_plane[0] = f < 1 ? 1 : (f > nz - 1 ? nz - 1 : f);
    s->flux_plane[1] = b < 1 ? 1 : (b > nz - 1 ? nz - 1 : b);
  }
  s->nmat = (long)nm * s->nxy;
  s->win = calloc((size_t)s->NW * (s->nmat ? s->nmat : 1), sizeof(double));
  s->eamp = calloc(s->nmat ? s->nmat : 1, sizeof(double));
  s->T = calloc(s->nmat ? s->nmat : 1, sizeof(uint64_t));
  s->Talways = calloc(s->nmat ? s->nmat : 1, 1);
  s->alive = calloc(s->nmat ? s->nmat : 1, sizeof(uint32_t));
  s->imax = calloc((size_t)s->nxy * nz, sizeof(double));
  if (cfg->pml_cells > 0)
    for (int q = 0; q < 8; q++) s->psi[q] = calloc(s->nfield, sizeof(double));
  if (cfg->elliptic_table >= 2) {
    s->ntab = cfg->elliptic_table;
    s->tabK = malloc((size_t)s->ntab * sizeof(double));
    s->tabE = malloc((size_t)s->ntab * sizeof(double));
    for (int i = 0; i < s->ntab; i++) {
      double m = (double)i / (double)s->ntab, K, KmE;
      or_ellip_KE(m, 1.0 - m, &K, &KmE);
      s->tabK[i] = K;
      s->tabE[i] = K - KmE;
    }
  }
  /* the paper records the intensity every 0.5 fs (Sec. 5, Plasma Screening) */
  s->imax_every = cfg->imax_every > 0
                      ? cfg->imax_every
                      : (cfg->imax_every == 0 ? (int)fmax(1.0, round(0.5e-15 / s->dt)) : 0);
  for (int k = 0; k < nz; k++) {
    int L = s->layer_of_plane[k];
    if (L < 0) continue;
    uint32_t bits = cfg->layers[L].ppc == 32
                        ? 0xFFFFFFFFu
                        : ((1u << cfg->layers[L].ppc) - 1u);
    for (int q = 0; q < s->nxy; q++)
      s->alive[(long)s->mplane[k] * s->nxy + q] = bits;
  }
  return s;
}

void or_destroy(or_sim *s) {
  if (!s) return;
  free(s->tabK);
  free(s->tabE);
  for (int q = 0; q < 8; q++) free(s->psi[q]);
  free(s->imax);
  for (int c = 0; c < NCOMP; c++) free(s->F[c]);
  free(s->layer_of_plane);
  free(s->mplane);
  free(s->win);
  free(s->eamp);
  free(s->T);
  free(s->Talways);
  free(s->alive);
  free(s->pid);
  free(s->pcell);
  free(s->poff);
  free(s->pu);
  free(s->ptag);
  free(s);
}

/* ------------------------------------------------------------------------ */
/* Particle pass: gather, Boris, move, Esirkepov deposit, z outflow.         */
/* ------------------------------------------------------------------------ */
static double gather(const or_sim *s, const double *f, const int st[3], int ci,
                     int cj, int ck, const double off[3]) {
  double wx[3], wy[3], wz[3];
  int bx = tsc(off[0], st[0], wx), by = tsc(off[1], st[1], wy),
      bz = tsc(off[2], st[2], wz);
  double acc = 0.0;
  for (int c = 0; c < 3; c++)
    for (int b = 0; b < 3; b++)
      for (int a = 0; a < 3; a++)
        acc += wx[a] * wy[b] * wz[c] *
               f[fidx(s, ci + bx + a, cj + by + b, ck + bz + c)];
  return acc;
}

/* Integer-node TSC shape of one axis on a 5-node frame starting at
 * (old nearest node - 2).  shift = new nearest node - old nearest node. */
static void frame_shape(double delta, int shift, double S[5]) {
  double w[3];
  tsc(delta, 0, w);
  for (int m = 0; m < 5; m++) S[m] = 0.0;
  S[1 + shift] = w[0];
  S[2 + shift] = w[1];
  S[3 + shift] = w[2];
}

static void esirkepov(or_sim *s, double qw, const int cold[3],
                      const double dold[3], const int cnew[3],
                      const double dnew[3]) {
  const double dl[3] = {s->cfg.dx, s->cfg.dy, s->cfg.dz};
  double S0[3][5], DS[3][5];
  int base[3];
  for (int d = 0; d < 3; d++) {
    int n0 = cold[d] + (dold[d] >= 0.5);
    int n1 = cnew[d] + (dnew[d] >= 0.5);
    double S1[5];
    frame_shape(dold[d], 0, S0[d]);
    frame_shape(dnew[d], n1 - n0, S1);
    for (int m = 0; m < 5; m++) DS[d][m] = S1[m] - S0[d][m];
    base[d] = n0 - 2;
  }
  /* W1 = DSx (S0y S0z + DSy S0z/2 + S0y DSz/2 + DSy DSz/3), cyclic for W2,
   * W3 (Esirkepov 2001); J_d accumulates -q w dl_d / (V dt) W_d along d. */
  for (int d = 0; d < 3; d++) {
    int e = (d + 1) % 3, f = (d + 2) % 3;
    double pref = -qw * dl[d] / (s->V * s->dt);
    double *J = s->F[FJX + d];
    for (int b = 0; b < 5; b++)
      for (int c = 0; c < 5; c++) {
        double wtr = S0[e][b] * S0[f][c] + 0.5 * DS[e][b] * S0[f][c] +
                     0.5 * S0[e][b] * DS[f][c] +
                     (1.0 / 3.0) * DS[e][b] * DS[f][c];
        double run = 0.0;
        for (int a = 0; a < 5; a++) {
          run += pref * DS[d][a] * wtr;
          if (run == 0.0) continue;
          int idx[3];
          idx[d] = base[d] + a;
          idx[e] = base[e] + b;
          idx[f] = base[f] + c;
          J[fidx(s, idx[0], idx[1], idx[2])] += run;
        }
      }
  }
}

void or_particle_pass(or_sim *s) {
  const int nx = s->cfg.nx, ny = s->cfg.ny, nz = s->cfg.nz;
  const double dl[3] = {s->cfg.dx, s->cfg.dy, s->cfg.dz};
  long w = 0;
  for (long p = 0; p < s->np; p++) {
    int32_t cell = s->pcell[p];
    int c[3] = {cell % nx, (cell / nx) % ny, cell / (nx * ny)};
    double *off = &s->poff[3 * p], *u = &s->pu[3 * p];
    uint32_t tag = s->ptag[p];
    int L = (int)(tag >> 1), sp = (int)(tag & 1u);
    double E[3], B[3];
    for (int d = 0; d < 3; d++) {
      E[d] = gather(s, s->F[FEX + d], stag_E[d], c[0], c[1], c[2], off);
      B[d] = gather(s, s->F[FBX + d], stag_B[d], c[0], c[1], c[2], off);
    }
    or_boris(s->qm[L][sp], s->dt, E, B, u);
    double g = sqrt(1.0 + (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) /
                              (OR_C * OR_C));
    int cn[3];
    double dn[3];
    for (int d = 0; d < 3; d++) {
      double nd = off[d] + s->dt * u[d] / (g * dl[d]);
      int cc = c[d];
      if (nd < 0.0) {
        nd += 1.0;
        cc -= 1;
      }
      if (nd >= 1.0) {
        nd -= 1.0;
        cc += 1;
      }
      cn[d] = cc;
      dn[d] = nd;
    }
    double q = sp ? OR_QE : -OR_QE;
    esirkepov(s, q * s->wmac[L], c, off, cn, dn);
    if (cn[2] < 2 || cn[2] >= nz - 2) continue; /* outflow: deleted */
    cn[0] = (cn[0] % nx + nx) % nx;
    cn[1] = (cn[1] % ny + ny) % ny;
    {
      /* outflow through the absorbing transverse layers */
      int L = s->cfg.pml_cells;
      if (L > 0 && (cn[0] < L || cn[0] >= nx - L || cn[1] < L || cn[1] >= ny - L)) continue;
    }
    s->pid[w] = s->pid[p];
    s->pcell[w] = (int32_t)(((long)cn[2] * ny + cn[1]) * nx + cn[0]);
    for (int d = 0; d < 3; d++) {
      s->poff[3 * w + d] = dn[d];
      s->pu[3 * w + d] = u[d];
    }
    s->ptag[w] = tag;
    w++;
  }
  s->np = w;
}

/* ------------------------------------------------------------------------ */
/* Field pass: B half step, E with Lorentz polarisation and Silver-Mueller   */
/* z faces, B half step, J cleared.                                          */
/* ------------------------------------------------------------------------ */
/* Absorbing transverse layers (the paper's outflow boundaries, Sec. 3.1):
 * a convolutional perfectly matched layer (Roden and Gedney, Microw. Opt.
 * Technol. Lett. 27, 334 (2000)) with kappa = 1 and alpha = 0, of L cells on
 * each side of the periodic seam of x (and of y), so that a wave leaving
 * through either face crosses 2 L graded cells.  A position p (in cells)
 * lies at depth d = L - p below L, p - (n - L) above n - L, else 0; the
 * conductivity is sigma = sigma_max (d / L)^3, sigma_max = 0.8 (3 + 1) /
 * (eta0 delta) for cells of size delta.  Over a time step h a derivative df
 * of the curl becomes df + psi, psi <- b psi + (b - 1) df, with
 * b = exp(-sigma h / eps0) (1 outside the layers, where psi stays 0). */
static double pml_b(const or_sim *s, double p, int n, double delta, double h) {
  int L = s->cfg.pml_cells;
  double d = p < L ? L - p : (p > n - L ? p - (n - L) : 0.0);
  if (!(d > 0.0)) return 1.0;
  double smax = 0.8 * 4.0 / (OR_MU0 * OR_C * delta);
  double r = d / L;
  return exp(-smax * r * r * r * h / OR_EPS0);
}

/* The layer's derivative: df + psi with psi advanced in place. */
static double pml_d(const or_sim *s, int q, long o, double b, double df) {
  if (!s->psi[q]) return df;
  s->psi[q][o] = b * s->psi[q][o] + (b - 1.0) * df;
  return df + s->psi[q][o];
}

static void b_half(or_sim *s) {
  const int nx = s->cfg.nx, ny = s->cfg.ny, nz = s->cfg.nz;
  const double h = 0.5 * s->dt, dx = s->cfg.dx, dy = s->cfg.dy,
               dz = s->cfg.dz;
  double *Ex = s->F[FEX], *Ey = s->F[FEY], *Ez = s->F[FEZ];
  double *Bx = s->F[FBX], *By = s->F[FBY], *Bz = s->F[FBZ];
#pragma omp parallel for schedule(static)
  for (int k = 0; k <= nz; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        long o = fidx(s, i, j, k);
        /* x derivatives at x = i + 1/2, y derivatives at y = j + 1/2 */
        double bxh = pml_b(s, i + 0.5, nx, dx, h), byh = pml_b(s, j + 0.5, ny, dy, h);
        if (k < nz) {
          double dEz_dy = pml_d(s, PBXY, o, byh, (Ez[fidx(s, i, j + 1, k)] - Ez[o]) / dy);
          double dEz_dx = pml_d(s, PBYX, o, bxh, (Ez[fidx(s, i + 1, j, k)] - Ez[o]) / dx);
          Bx[o] -= h * (dEz_dy - (Ey[fidx(s, i, j, k + 1)] - Ey[o]) / dz);
          By[o] -= h * ((Ex[fidx(s, i, j, k + 1)] - Ex[o]) / dz - dEz_dx);
        }
        double dEy_dx = pml_d(s, PBZX, o, bxh, (Ey[fidx(s, i + 1, j, k)] - Ey[o]) / dx);
        double dEx_dy = pml_d(s, PBZY, o, byh, (Ex[fidx(s, i, j + 1, k)] - Ex[o]) / dy);
        Bz[o] -= h * (dEy_dx - dEx_dy);
      }
}

/* One E point: a = dt (c^2 curl B - J / eps0) is the vacuum increment.  In a
 * Lorentz cell the oscillator P'' + G P' + w0^2 P = w0^2 eps0 deps E is
 * advanced by the trapezoidal (Crank-Nicolson) rule, coupled implicitly to
 * E^{n+1} (the explicit leapfrog form is unstable at CFL 0.95 for a 9 eV pole
 * at 25 nm cells).  p = P/eps0 and q = (dP/dt)/eps0 at integer times; the
 * polarisation current of Ampere's law is eps0 (p1 - p0)/dt. */
static double e_point(const or_sim *s, int L, double E0v, double a, double *p,
                      double *q) {
  if (L < 0) return E0v + a;
  double de = s->deps[L];
  double dp;
  if (s->is_static[L]) {
    dp = (2.0 * (de * E0v - *p) + de * a) / (1.0 + de);
    *p += dp;
    *q = 0.0;
  } else {
    double h = s->dt, k = s->kosc[L], g = s->cfg.layers[L].damping;
    double num = h * (*q) + 0.5 * h * h * k * (de * E0v - *p) +
                 0.25 * h * h * k * de * a;
    double den = 1.0 + 0.25 * h * h * k * (1.0 + de) + 0.5 * g * h;
    dp = num / den;
    *q = 2.0 * dp / h - *q;
    *p += dp;
  }
  return E0v + a - dp;
}

static void e_full(or_sim *s) {
  const int nx = s->cfg.nx, ny = s->cfg.ny, nz = s->cfg.nz;
  const double dt = s->dt, c2 = OR_C * OR_C, dx = s->cfg.dx, dy = s->cfg.dy,
               dz = s->cfg.dz, al = s->alpha;
  double *Ex = s->F[FEX], *Ey = s->F[FEY], *Ez = s->F[FEZ];
  double *Bx = s->F[FBX], *By = s->F[FBY], *Bz = s->F[FBZ];
  double *Jx = s->F[FJX], *Jy = s->F[FJY], *Jz = s->F[FJZ];
  double einc = e_inc(s, (s->step + 0.5) * dt);
  double exi = s->cfg.pol == 0 ? einc : 0.0, eyi = s->cfg.pol == 0 ? 0.0 : einc;
  double joule = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : joule)
  for (int k = 0; k <= nz; k++) {
    int L = k < nz ? s->layer_of_plane[k] : -1;
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        long o = fidx(s, i, j, k);
        /* x derivatives at x = i, y derivatives at y = j (absorbing layers) */
        double bxi = pml_b(s, (double)i, nx, dx, dt), byi = pml_b(s, (double)j, ny, dy, dt);
        double dBz_dy = pml_d(s, PEXY, o, byi, (Bz[o] - Bz[fidx(s, i, j - 1, k)]) / dy);
        double dBz_dx = pml_d(s, PEYX, o, bxi, (Bz[o] - Bz[fidx(s, i - 1, j, k)]) / dx);
        double ex0 = Ex[o], ey0 = Ey[o], ex1, ey1;
        if (k == 0) {
          /* the polarised component's own node: Ex at ((i + 1/2) dx, j dy),
           * Ey at (i dx, (j + 1/2) dy) */
          double spx = or_spot(s, (i + 0.5) * dx, j * dy), spy = or_spot(s, i * dx, (j + 0.5) * dy);
          ex1 = ((1.0 - al) * ex0 - 2.0 * al * OR_C * By[o] + 4.0 * al * exi * spx +
                 dt * (c2 * dBz_dy - Jx[o] / OR_EPS0)) /
                (1.0 + al);
          ey1 = ((1.0 - al) * ey0 + 2.0 * al * OR_C * Bx[o] + 4.0 * al * eyi * spy -
                 dt * (c2 * dBz_dx + Jy[o] / OR_EPS0)) /
                (1.0 + al);
        } else if (k == nz) {
          long om = fidx(s, i, j, k - 1);
          ex1 = ((1.0 - al) * ex0 + 2.0 * al * OR_C * By[om] +
                 dt * (c2 * dBz_dy - Jx[o] / OR_EPS0)) /
                (1.0 + al);
          ey1 = ((1.0 - al) * ey0 - 2.0 * al * OR_C * Bx[om] -
                 dt * (c2 * dBz_dx + Jy[o] / OR_EPS0)) /
                (1.0 + al);
        } else {
          long om = fidx(s, i, j, k - 1);
          double ax = dt * (c2 * (dBz_dy - (By[o] - By[om]) / dz) -
                            Jx[o] / OR_EPS0);
          double ay = dt * (c2 * ((Bx[o] - Bx[om]) / dz - dBz_dx) -
                            Jy[o] / OR_EPS0);
          ex1 = e_point(s, L, ex0, ax, &s->F[FPX][o], &s->F[FQX][o]);
          ey1 = e_point(s, L, ey0, ay, &s->F[FPY][o], &s->F[FQY][o]);
        }
        joule += Jx[o] * 0.5 * (ex0 + ex1) + Jy[o] * 0.5 * (ey0 + ey1);
        Ex[o] = ex1;
        Ey[o] = ey1;
        if (k < nz) {
          double dBy_dx = pml_d(s, PEZX, o, bxi, (By[o] - By[fidx(s, i - 1, j, k)]) / dx);
          double dBx_dy = pml_d(s, PEZY, o, byi, (Bx[o] - Bx[fidx(s, i, j - 1, k)]) / dy);
          double az = dt * (c2 * (dBy_dx - dBx_dy) - Jz[o] / OR_EPS0);
          double ez0 = Ez[o];
          double ez1 = e_point(s, L, ez0, az, &s->F[FPZ][o], &s->F[FQZ][o]);
          joule += Jz[o] * 0.5 * (ez0 + ez1);
          Ez[o] = ez1;
        }
      }
  }
  s->U_joule += joule * dt * s->V;
}

/* Accumulated intensity map (Sec. 5, Plasma Screening, Fig. 7c): every
 * imax_every steps, |E^{n+1}|^2 at each cell centre (4-edge means, as the
 * amplitude window) over E0^2 (the incident peak amplitude; raw |E|^2 when
 * E0 = 0), kept as the running maximum. */
static void record_intensity(or_sim *s) {
  const int nx = s->cfg.nx, ny = s->cfg.ny, nz = s->cfg.nz;
  const double *Ex = s->F[FEX], *Ey = s->F[FEY], *Ez = s->F[FEZ];
  const double norm = s->E0 > 0.0 ? 1.0 / (s->E0 * s->E0) : 1.0;
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nz; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        double ax = 0.25 * (((Ex[fidx(s, i, j, k)] + Ex[fidx(s, i, j + 1, k)]) +
                             Ex[fidx(s, i, j, k + 1)]) +
                            Ex[fidx(s, i, j + 1, k + 1)]);
        double ay = 0.25 * (((Ey[fidx(s, i, j, k)] + Ey[fidx(s, i + 1, j, k)]) +
                             Ey[fidx(s, i, j, k + 1)]) +
                            Ey[fidx(s, i + 1, j, k + 1)]);
        double az = 0.25 * (((Ez[fidx(s, i, j, k)] + Ez[fidx(s, i + 1, j, k)]) +
                             Ez[fidx(s, i, j + 1, k)]) +
                            Ez[fidx(s, i + 1, j + 1, k)]);
        double v = (ax * ax + ay * ay + az * az) * norm;
        long c = ((long)k * ny + j) * nx + i;
        if (v > s->imax[c]) s->imax[c] = v;
      }
}

void or_field_pass(or_sim *s) {
  b_half(s);
  e_full(s);
  b_half(s);
  for (int d = 0; d < 3; d++) memset(s->F[FJX + d], 0, s->nfield * sizeof(double));
  if (s->imax_every > 0 && (s->step + 1) % s->imax_every == 0) record_intensity(s);
}

/* ------------------------------------------------------------------------ */
/* Amplitude window (Sec. 2.1, reading K6) and Keldysh threshold per cell.   */
/* ------------------------------------------------------------------------ */
void or_window_keldysh_pass(or_sim *s) {
  const int nx = s->cfg.nx, ny = s->cfg.ny, nz = s->cfg.nz, NW = s->NW;
  double *Ex = s->F[FEX], *Ey = s->F[FEY], *Ez = s->F[FEZ];
  int slot = (int)(s->step % NW);
#pragma omp parallel for schedule(dynamic)
  for (int k = 0; k < nz; k++) {
    int L = s->layer_of_plane[k];
    if (L < 0) continue;
    const or_layer *ly = &s->cfg.layers[L];
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        long m = (long)s->mplane[k] * s->nxy + (long)j * nx + i;
        double ax = 0.25 * (((Ex[fidx(s, i, j, k)] + Ex[fidx(s, i, j + 1, k)]) +
                             Ex[fidx(s, i, j, k + 1)]) +
                            Ex[fidx(s, i, j + 1, k + 1)]);
        double ay = 0.25 * (((Ey[fidx(s, i, j, k)] + Ey[fidx(s, i + 1, j, k)]) +
                             Ey[fidx(s, i, j, k + 1)]) +
                            Ey[fidx(s, i + 1, j, k + 1)]);
        double az = 0.25 * (((Ez[fidx(s, i, j, k)] + Ez[fidx(s, i + 1, j, k)]) +
                             Ez[fidx(s, i, j + 1, k)]) +
                            Ez[fidx(s, i + 1, j + 1, k)]);
        double a = sqrt(ax * ax + ay * ay + az * az);
        s->win[(long)slot * s->nmat + m] = a;
        double mx = 0.0;
        for (int q = 0; q < NW; q++) {
          double v = s->win[(long)q * s->nmat + m];
          if (v > mx) mx = v;
        }
        s->eamp[m] = mx;
        double W = keldysh_rate(mx, s->omega, s->gapJ[L], s->mstar[L],
                                s->cfg.keldysh_terms, NULL, NULL, s->tabK, s->tabE, s->ntab);
        ion_threshold(W, ly->n_mol, s->dt, &s->T[m], &s->Talways[m]);
      }
  }
}

/* ------------------------------------------------------------------------ */
/* Ionisation draws and pair creation (Sec. 2.1 "ionized once", Sec. 3.2).   */
/* ------------------------------------------------------------------------ */
static void neutral_state(const or_sim *s, int L, uint32_t cell, uint32_t slot,
                          double off0[3], double v0[3]) {
  uint32_t r[4];
  philox_draw(s->cfg.seed, 0, cell, slot, OR_STREAM_POS, r);
  off0[0] = u01(r[0]);
  off0[1] = u01(r[1]);
  off0[2] = u01(r[2]);
  philox_draw(s->cfg.seed, 0, cell, slot, OR_STREAM_VEL, r);
  double sg = s->sigv[L];
  double r1 = sqrt(-2.0 * log(u01(r[0]))), t1 = 2.0 * OR_PI * u01(r[1]);
  double r2 = sqrt(-2.0 * log(u01(r[2]))), t2 = 2.0 * OR_PI * u01(r[3]);
  v0[0] = sg * r1 * cos(t1);
  v0[1] = sg * r1 * sin(t1);
  v0[2] = sg * r2 * cos(t2);
}

void or_ionize_pass(or_sim *s) {
  const int nx = s->cfg.nx, ny = s->cfg.ny, nz = s->cfg.nz;
  const double dl[3] = {s->cfg.dx, s->cfg.dy, s->cfg.dz};
  const double t1 = (double)(s->step + 1) * s->dt;
  for (int k = 0; k < nz; k++) {
    int L = s->layer_of_plane[k];
    if (L < 0) continue;
    int ppc = s->cfg.layers[L].ppc;
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        long m = (long)s->mplane[k] * s->nxy + (long)j * nx + i;
        uint32_t cell = (uint32_t)(((long)k * ny + j) * nx + i);
        for (int sl = 0; sl < ppc; sl++) {
          if (!((s->alive[m] >> sl) & 1u)) continue;
          double off0[3], v0[3];
          neutral_state(s, L, cell, (uint32_t)sl, off0, v0);
          int cc[3] = {i, j, k};
          double dn[3];
          for (int d = 0; d < 3; d++) {
            double nd = off0[d] + v0[d] * t1 / dl[d];
            int c0 = cc[d];
            if (nd < 0.0) {
              nd += 1.0;
              c0 -= 1;
            }
            if (nd >= 1.0) {
              nd -= 1.0;
              c0 += 1;
            }
            cc[d] = c0;
            dn[d] = nd;
          }
          cc[0] = (cc[0] % nx + nx) % nx;
          cc[1] = (cc[1] % ny + ny) % ny;
          uint64_t T = 0;
          int always = 0;
          if (cc[2] >= 0 && cc[2] < nz && s->mplane[cc[2]] >= 0) {
            long m2 = (long)s->mplane[cc[2]] * s->nxy + (long)cc[1] * nx + cc[0];
            T = s->T[m2];
            always = s->Talways[m2];
          }
          uint64_t r64 = or_ion_uniform(s->cfg.seed, (uint32_t)s->step, cell, (uint32_t)sl);
          if (!(always || r64 < T)) continue;
          s->alive[m] &= ~(1u << sl);
          double v2 = v0[0] * v0[0] + v0[1] * v0[1] + v0[2] * v0[2];
          double gm = 1.0 / sqrt(1.0 - v2 / (OR_C * OR_C));
          grow(s, s->np + 2);
          uint64_t gid = (uint64_t)cell * (uint64_t)ppc + (uint64_t)sl;
          int32_t ncell = (int32_t)(((long)cc[2] * ny + cc[1]) * nx + cc[0]);
          for (int sp = 0; sp < 2; sp++) {
            long p = s->np++;
            s->pid[p] = 2 * gid + (uint64_t)sp;
            s->pcell[p] = ncell;
            for (int d = 0; d < 3; d++) {
              s->poff[3 * p + d] = dn[d];
              s->pu[3 * p + d] = gm * v0[d];
            }
            s->ptag[p] = ((uint32_t)L << 1) | (uint32_t)sp;
          }
          s->n_events += 1.0;
          s->N_pairs += s->wmac[L];
          s->U_ion += s->wmac[L] * s->gapJ[L];
        }
      }
  }
}

/* ------------------------------------------------------------------------ */
/* Binary collisions among electrons and holes (Sec. 2.2: the Perez/Nanbu    */
/* module, here written from the published methods: Nanbu, Phys. Rev. E 55,  */
/* 4642 (1997) for the cumulative scattering angle; Perez et al., Phys.      */
/* Plasmas 19, 083104 (2012) for the relativistic centre-of-mass frame, the  */
/* Coulomb logarithm and the low-temperature cap).                           */
/* ------------------------------------------------------------------------ */
#define OR_H (2.0 * OR_PI * OR_HBAR)

/* Nanbu's parameter A(s): the root of coth A - 1/A = exp(-s). */
double or_nanbu_A(double s) {
  double target = exp(-s);
  double lo = 1e-12, hi = 1e12;
  for (int it = 0; it < 200; it++) { /* bisection on log A */
    double mid = sqrt(lo * hi);
    double g = mid < 1e-4 ? mid / 3.0 - mid * mid * mid / 45.0 : 1.0 / tanh(mid) - 1.0 / mid;
    if (g < target)
      lo = mid;
    else
      hi = mid;
    if (hi / lo < 1.0 + 4e-16) break;
  }
  return sqrt(lo * hi);
}

/* cos chi of the cumulative scattering angle for parameter s and uniform U
 * (Nanbu): small s 1 + s ln U; large s isotropic; between, the inverse of
 * the distribution A exp(A cos chi) / (2 sinh A). */
double or_nanbu_cos(double s, double U) {
  double c;
  if (s < 0.1) {
    c = 1.0 + s * log(U);
  } else if (s < 6.0) {
    double A = or_nanbu_A(s);
    c = log(exp(-A) + 2.0 * U * sinh(A)) / A;
  } else {
    c = 2.0 * U - 1.0;
  }
  return c < -1.0 ? -1.0 : (c > 1.0 ? 1.0 : c);
}

/* One binary collision of macroparticles a and b (u = gamma v per unit mass,
 * masses m, weights w, charges of magnitude e), Perez et al.: transform to
 * the centre-of-mass frame, rotate the relative momentum by the sampled
 * (chi, phi), transform back.  neff = n_a n_b / n_ab (inter) or n (intra),
 * times `frac` (1/2 for the odd-count triplet); na, nb the group densities;
 * lambda_D the screening length; dtc the collision interval; U[4] uniforms:
 * angle, azimuth, acceptance of a, acceptance of b.  Returns s. */
double or_collide_pair(double ua[3], double ub[3], double ma, double mb, double wa, double wb,
                       double neff, double na, double nb, double lambda_D, double dtc,
                       const double U[4]) {
  const double c = OR_C, c2 = OR_C * OR_C;
  double ga = sqrt(1.0 + (ua[0] * ua[0] + ua[1] * ua[1] + ua[2] * ua[2]) / c2);
  double gb = sqrt(1.0 + (ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2]) / c2);
  double pa[3], pb[3], va[3], vb[3], vc[3];
  double Etot = ma * ga + mb * gb; /* total energy / c^2 */
  for (int d = 0; d < 3; d++) {
    pa[d] = ma * ua[d];
    pb[d] = mb * ub[d];
    va[d] = ua[d] / ga;
    vb[d] = ub[d] / gb;
    vc[d] = (pa[d] + pb[d]) / Etot;
  }
  double vc2 = vc[0] * vc[0] + vc[1] * vc[1] + vc[2] * vc[2];
  double gc = 1.0 / sqrt(1.0 - vc2 / c2);
  double kc = gc * gc / (c2 * (gc + 1.0)); /* (gamma_c - 1) / v_c^2 */
  double vcva = vc[0] * va[0] + vc[1] * va[1] + vc[2] * va[2];
  double vcvb = vc[0] * vb[0] + vc[1] * vb[1] + vc[2] * vb[2];
  double pst[3];
  for (int d = 0; d < 3; d++) pst[d] = pa[d] + (kc * vcva - gc) * ma * ga * vc[d];
  double gsa = (1.0 - vcva / c2) * gc * ga, gsb = (1.0 - vcvb / c2) * gc * gb;
  double p2 = pst[0] * pst[0] + pst[1] * pst[1] + pst[2] * pst[2];
  double pm = sqrt(p2);
  if (!(pm > 0.0)) return 0.0;
  double e2 = OR_QE * OR_QE;
  double mm = ma * gsa * mb * gsb * c2 / p2 + 1.0;
  double b0 = e2 / (4.0 * OR_PI * OR_EPS0 * c2) * gc / Etot * mm;
  double bmin = fmax(OR_H / (2.0 * pm), b0);
  double lnL = fmax(1.0, 0.5 * log(1.0 + lambda_D * lambda_D / (bmin * bmin)));
  double sv = neff * dtc * lnL * e2 * e2 /
              (4.0 * OR_PI * OR_EPS0 * OR_EPS0 * c2 * c2 * ma * ga * mb * gb) * gc * pm / Etot *
              mm * mm;
  /* low-temperature cap: collisions no faster than the mean interparticle
   * spacing allows (Perez et al.) */
  double vrel = Etot * pm / (ma * gsa * mb * gsb * gc);
  double dens = fmax(ma * pow(na, 2.0 / 3.0), mb * pow(nb, 2.0 / 3.0));
  double scap = neff * dtc * pow(4.0 * OR_PI / 3.0, 1.0 / 3.0) * (ma + mb) / dens * vrel;
  double s = fmin(sv, scap);
  double cx = or_nanbu_cos(s, U[0]);
  double sx = sqrt(fmax(0.0, 1.0 - cx * cx));
  double phi = 2.0 * OR_PI * U[1];
  double u[3] = {pst[0] / pm, pst[1] / pm, pst[2] / pm}, e1[3], e2v[3];
  if (fabs(u[2]) < 0.9) {
    double n = sqrt(u[0] * u[0] + u[1] * u[1]);
    e1[0] = u[1] / n;
    e1[1] = -u[0] / n;
    e1[2] = 0.0;
  } else {
    double n = sqrt(u[1] * u[1] + u[2] * u[2]);
    e1[0] = 0.0;
    e1[1] = u[2] / n;
    e1[2] = -u[1] / n;
  }
  e2v[0] = u[1] * e1[2] - u[2] * e1[1];
  e2v[1] = u[2] * e1[0] - u[0] * e1[2];
  e2v[2] = u[0] * e1[1] - u[1] * e1[0];
  double cp = cos(phi), sp = sin(phi), pn[3];
  for (int d = 0; d < 3; d++) pn[d] = pm * (cx * u[d] + sx * (cp * e1[d] + sp * e2v[d]));
  /* back to the lab frame; b takes -pn in the centre-of-mass frame */
  double vpa = vc[0] * pn[0] + vc[1] * pn[1] + vc[2] * pn[2];
  double wmax = fmax(wa, wb);
  if (U[2] * wmax < wb)
    for (int d = 0; d < 3; d++) ua[d] = (pn[d] + (kc * vpa + ma * gsa * gc) * vc[d]) / ma;
  if (U[3] * wmax < wa)
    for (int d = 0; d < 3; d++) ub[d] = (-pn[d] + (-kc * vpa + mb * gsb * gc) * vc[d]) / mb;
  return s;
}

typedef struct {
  uint32_t key;
  uint64_t id;
  long p;
} coll_item;

static int cmp_coll(const void *x, const void *y) {
  const coll_item *a = x, *b = y;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  return a->id < b->id ? -1 : (a->id > b->id ? 1 : 0);
}

/* One collision pass: in every cell, electrons and holes each in the random
 * order of their keys (Philox (step, id) stream 5); like-species pairs
 * (0,1),(2,3),... with an odd count's first three colliding pairwise at half
 * strength (Takizuka & Abe); then unlike pairs (A_i, B_{i mod |B|}) with A
 * the larger group.  Pair q of the cell (in that order) draws Philox
 * (step, cell, q) stream 6. */
void or_collide_pass(or_sim *s) {
  if (s->cfg.coll_every <= 0 || (s->step + 1) % s->cfg.coll_every != 0) return;
  const int nx = s->cfg.nx, ny = s->cfg.ny, nz = s->cfg.nz;
  const long ncell = (long)nx * ny * nz;
  const double dtc = s->dt * s->cfg.coll_every;
  long *cnt = calloc(ncell + 1, sizeof(long));
  for (long p = 0; p < s->np; p++) cnt[s->pcell[p] + 1]++;
  for (long c = 0; c < ncell; c++) cnt[c + 1] += cnt[c];
  long *pos = malloc(ncell * sizeof(long)), *idx = malloc((s->np ? s->np : 1) * sizeof(long));
  for (long c = 0; c < ncell; c++) pos[c] = cnt[c];
  for (long p = 0; p < s->np; p++) idx[pos[s->pcell[p]]++] = p;
  for (long c = 0; c < ncell; c++) {
    long n = cnt[c + 1] - cnt[c];
    if (n < 2) continue;
    coll_item *grp[2];
    long gn[2] = {0, 0};
    grp[0] = malloc(n * sizeof(coll_item));
    grp[1] = malloc(n * sizeof(coll_item));
    double dens[2] = {0, 0}, wsum[2] = {0, 0}, wm[2] = {0, 0}, T[2] = {0, 0};
    for (long q = cnt[c]; q < cnt[c + 1]; q++) {
      long p = idx[q];
      int sp = (int)(s->ptag[p] & 1u), L = (int)(s->ptag[p] >> 1);
      uint32_t r[4];
      philox_draw(s->cfg.seed, (uint32_t)s->step, (uint32_t)s->pid[p],
                  (uint32_t)(s->pid[p] >> 32), OR_STREAM_COLL_ORDER, r);
      grp[sp][gn[sp]].key = r[0];
      grp[sp][gn[sp]].id = s->pid[p];
      grp[sp][gn[sp]].p = p;
      gn[sp]++;
      wsum[sp] += s->wmac[L];
      wm[sp] += s->wmac[L] * s->mass[L][sp];
    }
    for (int sp = 0; sp < 2; sp++) {
      qsort(grp[sp], gn[sp], sizeof(coll_item), cmp_coll);
      dens[sp] = wsum[sp] / s->V;
    }
    /* kinetic temperature of each group: mean mass times the weighted
     * velocity variance, written as a sum over pairs so that it is exactly 0
     * for one particle or equal velocities (no cancellation) */
    for (int sp = 0; sp < 2; sp++) {
      double S = 0.0;
      for (long i = 0; i < gn[sp]; i++)
        for (long j = i + 1; j < gn[sp]; j++) {
          long pi = grp[sp][i].p, pj = grp[sp][j].p;
          const double *ui = &s->pu[3 * pi], *uj = &s->pu[3 * pj];
          double gi = sqrt(1.0 + (ui[0] * ui[0] + ui[1] * ui[1] + ui[2] * ui[2]) / (OR_C * OR_C));
          double gj = sqrt(1.0 + (uj[0] * uj[0] + uj[1] * uj[1] + uj[2] * uj[2]) / (OR_C * OR_C));
          double dv2 = 0.0;
          for (int d = 0; d < 3; d++) {
            double dv = ui[d] / gi - uj[d] / gj;
            dv2 += dv * dv;
          }
          S += s->wmac[s->ptag[pi] >> 1] * s->wmac[s->ptag[pj] >> 1] * dv2;
        }
      if (wsum[sp] > 0.0) T[sp] = wm[sp] / wsum[sp] * S / (3.0 * wsum[sp] * wsum[sp]);
    }
    double inv_l2 = 0.0;
    for (int sp = 0; sp < 2; sp++)
      if (T[sp] > 0.0) inv_l2 += dens[sp] * OR_QE * OR_QE / (OR_EPS0 * T[sp]);
    /* screening no shorter than the interparticle spacing of the holes (the
     * ions), or of the electrons in a cell without holes */
    double ni = dens[1] > 0.0 ? dens[1] : dens[0];
    double ra = pow(4.0 * OR_PI * ni / 3.0, -1.0 / 3.0);
    double lD = inv_l2 > 0.0 ? fmax(1.0 / sqrt(inv_l2), ra) : ra;
    uint32_t q = 0;
    /* like-species pairs */
    for (int sp = 0; sp < 2; sp++) {
      long m = gn[sp];
      if (m < 2) continue;
      long start = 0;
      if (m % 2 == 1) {
        const long tri[3][2] = {{0, 1}, {0, 2}, {1, 2}};
        for (int t = 0; t < 3; t++) {
          long pa = grp[sp][tri[t][0]].p, pb = grp[sp][tri[t][1]].p;
          int La = (int)(s->ptag[pa] >> 1), Lb = (int)(s->ptag[pb] >> 1);
          uint32_t r[4];
          philox_draw(s->cfg.seed, (uint32_t)s->step, (uint32_t)c, q++, OR_STREAM_COLL_PAIR, r);
          double U[4] = {u01(r[0]), u01(r[1]), u01(r[2]), u01(r[3])};
          or_collide_pair(&s->pu[3 * pa], &s->pu[3 * pb], s->mass[La][sp], s->mass[Lb][sp],
                          s->wmac[La], s->wmac[Lb], 0.5 * dens[sp], dens[sp], dens[sp], lD, dtc, U);
        }
        start = 3;
      }
      for (long i = start; i + 1 < m; i += 2) {
        long pa = grp[sp][i].p, pb = grp[sp][i + 1].p;
        int La = (int)(s->ptag[pa] >> 1), Lb = (int)(s->ptag[pb] >> 1);
        uint32_t r[4];
        philox_draw(s->cfg.seed, (uint32_t)s->step, (uint32_t)c, q++, OR_STREAM_COLL_PAIR, r);
        double U[4] = {u01(r[0]), u01(r[1]), u01(r[2]), u01(r[3])};
        or_collide_pair(&s->pu[3 * pa], &s->pu[3 * pb], s->mass[La][sp], s->mass[Lb][sp],
                        s->wmac[La], s->wmac[Lb], dens[sp], dens[sp], dens[sp], lD, dtc, U);
      }
    }
    /* unlike pairs: every particle of the larger group once */
    if (gn[0] > 0 && gn[1] > 0) {
      int A = gn[0] >= gn[1] ? 0 : 1, B = 1 - A;
      double nab = 0.0;
      for (long i = 0; i < gn[A]; i++) {
        long pa = grp[A][i].p, pb = grp[B][i % gn[B]].p;
        nab += fmin(s->wmac[s->ptag[pa] >> 1], s->wmac[s->ptag[pb] >> 1]) / s->V;
      }
      double neff = dens[0] * dens[1] / nab;
      for (long i = 0; i < gn[A]; i++) {
        /* (electron, hole) order inside the pair */
        long pA = grp[A][i].p, pB = grp[B][i % gn[B]].p;
        long pe = A == 0 ? pA : pB, ph = A == 0 ? pB : pA;
        int Le = (int)(s->ptag[pe] >> 1), Lh = (int)(s->ptag[ph] >> 1);
        uint32_t r[4];
        philox_draw(s->cfg.seed, (uint32_t)s->step, (uint32_t)c, q++, OR_STREAM_COLL_PAIR, r);
        double U[4] = {u01(r[0]), u01(r[1]), u01(r[2]), u01(r[3])};
        or_collide_pair(&s->pu[3 * pe], &s->pu[3 * ph], s->mass[Le][0], s->mass[Lh][1],
                        s->wmac[Le], s->wmac[Lh], neff, dens[0], dens[1], lD, dtc, U);
      }
    }
    free(grp[0]);
    free(grp[1]);
  }
  free(cnt);
  free(pos);
  free(idx);
}

/* Phases of one step: 1 particle, 32 collisions, 2 field, 4 window + Keldysh,
 * 8 ionisation, 16 advance the step counter.  A full step is 63. */
/* Poynting split (reading K17: the reflected and transmitted energy from
 * the waves going along -z and +z).  At node plane k the transverse E of
 * the plane (Ex at (i + 1/2, j, k), Ey at (i, j + 1/2, k)) is paired with B
 * averaged over the two half-integer planes k - 1/2 and k + 1/2 (By and Bx
 * share those transverse positions).  A wave along +z has Ex = c By and
 * Ey = -c Bx, one along -z the opposite signs, so
 *   fwd = ((Ex + c By) / 2, (Ey - c Bx) / 2),
 *   bwd = ((Ex - c By) / 2, (Ey + c Bx) / 2),
 * and c eps0 (|fwd|^2 - |bwd|^2) is the Poynting flux (E x B)_z / mu0.
 * Called once per step at the end of the step (E^{n+1}, B^{n+1}); each
 * plane's sum of c eps0 |fwd|^2 dx dy and c eps0 |bwd|^2 dx dy, times dt, is
 * added to the time integrals. */
static void poynting_split(or_sim *s) {
  const int nx = s->cfg.nx, ny = s->cfg.ny;
  const double *Ex = s->F[FEX], *Ey = s->F[FEY], *Bx = s->F[FBX], *By = s->F[FBY];
  for (int q = 0; q < 2; q++) {
    int k = s->flux_plane[q];
    double f = 0.0, b = 0.0;
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        long o = fidx(s, i, j, k), om = fidx(s, i, j, k - 1);
        double cby = OR_C * 0.5 * (By[om] + By[o]);
        double cbx = OR_C * 0.5 * (Bx[om] + Bx[o]);
        double fx = 0.5 * (Ex[o] + cby), fy = 0.5 * (Ey[o] - cbx);
        double bx = 0.5 * (Ex[o] - cby), by = 0.5 * (Ey[o] + cbx);
        f += fx * fx + fy * fy;
        b += bx * bx + by * by;
      }
    double scale = OR_C * OR_EPS0 * s->cfg.dx * s->cfg.dy * s->dt;
    s->U_fwd[q] += f * scale;
    s->U_bwd[q] += b * scale;
  }
}

void or_step_phases(or_sim *s, int mask) {
  if (mask & 1) or_particle_pass(s);
  if (mask & 32) or_collide_pass(s);
  if (mask & 2) or_field_pass(s);
  if (mask & 4) or_window_keldysh_pass(s);
  if (mask & 8) or_ionize_pass(s);
  if (mask & 16) {
    poynting_split(s);
    s->step++;
  }
}

void or_step(or_sim *s, int n) {
  for (int q = 0; q < n; q++) or_step_phases(s, 63);
}

/* ------------------------------------------------------------------------ */
/* Diagnostics (Sec. 4.1 number density, Sec. 4.2 energy density, Sec. 4.3   */
/* spectra; readings K17, K18).                                              */
/* ------------------------------------------------------------------------ */
static void deposit_node(const or_sim *s, double *grid, int ci, int cj, int ck,
                         const double off[3], double val) {
  double wx[3], wy[3], wz[3];
  int bx = tsc(off[0], 0, wx), by = tsc(off[1], 0, wy), bz = tsc(off[2], 0, wz);
  for (int c = 0; c < 3; c++)
    for (int b = 0; b < 3; b++)
      for (int a = 0; a < 3; a++)
        grid[fidx(s, ci + bx + a, cj + by + b, ck + bz + c)] +=
            val * wx[a] * wy[b] * wz[c];
}

/* Charge density at integer nodes with the TSC shape, C/m^3. */
void or_rho(const or_sim *s, double *rho) {
  const int nx = s->cfg.nx, ny = s->cfg.ny;
  memset(rho, 0, s->nfield * sizeof(double));
  for (long p = 0; p < s->np; p++) {
    int32_t cell = s->pcell[p];
    int L = (int)(s->ptag[p] >> 1), sp = (int)(s->ptag[p] & 1u);
    double q = (sp ? OR_QE : -OR_QE) * s->wmac[L] / s->V;
    deposit_node(s, rho, cell % nx, (cell / nx) % ny, cell / (nx * ny),
                 &s->poff[3 * p], q);
  }
}

/* Damage metrics (Sec. 4.1-4.2 criteria, Sec. 5): n_e and the electron
 * energy density (number density x mean kinetic energy, i.e. the deposited
 * w E_k / V) on the nodes with the TSC shape; their mean over the nodes
 * (i, j) of the transverse box [r0, r1) x [r2, r3) on every node plane k
 * (ne_z, ed_z: nz + 1 values); per layer the largest profile value on its
 * node planes z0 <= k < z1, the largest recorded intensity over its cells,
 * and the verdicts (bit 0: n_e >= critical density eps0 m_e w^2 / e^2 of
 * free electrons; bit 1: n_e >= 9% of the valence density, four valence
 * electrons per molecule; bits 2-4: energy density >= melting, boiling,
 * dissociation energy density, where given).  out_layers holds 4 doubles
 * per layer: ne_peak, ed_peak, imax_peak, instability density.  Returns the
 * critical density. */
double or_damage(const or_sim *s, const int region[4], double *ne_z, double *ed_z,
                 double *out_layers, int *flags) {
  const int nx = s->cfg.nx, ny = s->cfg.ny, nz = s->cfg.nz;
  double *ne = calloc(s->nfield, sizeof(double));
  double *ed = calloc(s->nfield, sizeof(double));
  for (long p = 0; p < s->np; p++) {
    int32_t cell = s->pcell[p];
    int L = (int)(s->ptag[p] >> 1), sp = (int)(s->ptag[p] & 1u);
    if (sp != 0) continue;
    int ci = cell % nx, cj = (cell / nx) % ny, ck = cell / (nx * ny);
    const double *u = &s->pu[3 * p];
    double g = sqrt(1.0 + (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) / (OR_C * OR_C));
    double ek = (g - 1.0) * s->mass[L][0] * OR_C * OR_C;
    deposit_node(s, ne, ci, cj, ck, &s->poff[3 * p], s->wmac[L] / s->V);
    deposit_node(s, ed, ci, cj, ck, &s->poff[3 * p], s->wmac[L] * ek / s->V);
  }
  double cnt = (double)(region[1] - region[0]) * (double)(region[3] - region[2]);
  double *pz = malloc((size_t)(nz + 1) * 2 * sizeof(double));
  for (int k = 0; k <= nz; k++) {
    double a = 0.0, b = 0.0;
    for (int j = region[2]; j < region[3]; j++)
      for (int i = region[0]; i < region[1]; i++) {
        a += ne[fidx(s, i, j, k)];
        b += ed[fidx(s, i, j, k)];
      }
    pz[2 * k] = cnt > 0.0 ? a / cnt : 0.0;
    pz[2 * k + 1] = cnt > 0.0 ? b / cnt : 0.0;
    if (ne_z) ne_z[k] = pz[2 * k];
    if (ed_z) ed_z[k] = pz[2 * k + 1];
  }
  double ncrit = OR_EPS0 * OR_ME * s->omega * s->omega / (OR_QE * OR_QE);
  for (int L = 0; L < s->cfg.n_layers; L++) {
    const or_layer *ly = &s->cfg.layers[L];
    double mne = 0.0, med = 0.0, mi = 0.0;
    for (int k = ly->z0; k < ly->z1; k++) {
      if (pz[2 * k] > mne) mne = pz[2 * k];
      if (pz[2 * k + 1] > med) med = pz[2 * k + 1];
      for (long q = 0; q < s->nxy; q++)
        if (s->imax[(long)k * s->nxy + q] > mi) mi = s->imax[(long)k * s->nxy + q];
    }
    double ninst = 0.09 * 4.0 * ly->n_mol;
    if (out_layers) {
      out_layers[4 * L] = mne;
      out_layers[4 * L + 1] = med;
      out_layers[4 * L + 2] = mi;
      out_layers[4 * L + 3] = ninst;
    }
    if (flags) {
      int f = 0;
      if (mne >= ncrit) f |= 1;
      if (mne >= ninst) f |= 2;
      if (ly->e_melt > 0.0 && med >= ly->e_melt) f |= 4;
      if (ly->e_boil > 0.0 && med >= ly->e_boil) f |= 8;
      if (ly->e_dissoc > 0.0 && med >= ly->e_dissoc) f |= 16;
      flags[L] = f;
    }
  }
  free(pz);
  free(ne);
  free(ed);
  return ncrit;
}

void or_get_imax(const or_sim *s, double *out) {
  memcpy(out, s->imax, (size_t)s->nxy * s->cfg.nz * sizeof(double));
}

void or_diagnostics(const or_sim *s, or_diag *dg, int n_bins, double e_min_eV,
                    double e_max_eV, const int region[6], double *spectrum) {
  const int nx = s->cfg.nx, ny = s->cfg.ny, nz = s->cfg.nz;
  memset(dg, 0, sizeof(*dg));
  double *ne = calloc(s->nfield, sizeof(double));
  double *ed = calloc(s->nfield, sizeof(double));
  double *rho = calloc(s->nfield, sizeof(double));
  if (spectrum)
    for (int b = 0; b < n_bins; b++) spectrum[b] = 0.0;
  double kin = 0.0;
  for (long p = 0; p < s->np; p++) {
    int32_t cell = s->pcell[p];
    int ci = cell % nx, cj = (cell / nx) % ny, ck = cell / (nx * ny);
    int L = (int)(s->ptag[p] >> 1), sp = (int)(s->ptag[p] & 1u);
    const double *u = &s->pu[3 * p];
    double g = sqrt(1.0 + (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) /
                              (OR_C * OR_C));
    double ek = (g - 1.0) * s->mass[L][sp] * OR_C * OR_C;
    double w = s->wmac[L];
    kin += w * ek;
    deposit_node(s, rho, ci, cj, ck, &s->poff[3 * p],
                 (sp ? OR_QE : -OR_QE) * w / s->V);
    if (sp == 0) {
      dg->n_electrons_macro += 1.0;
      deposit_node(s, ne, ci, cj, ck, &s->poff[3 * p], w / s->V);
      deposit_node(s, ed, ci, cj, ck, &s->poff[3 * p], w * ek / s->V);
      if (spectrum && n_bins > 0 && ci >= region[0] && ci < region[1] &&
          cj >= region[2] && cj < region[3] && ck >= region[4] &&
          ck < region[5]) {
        double ev = ek / OR_QE;
        if (ev >= e_min_eV && ev < e_max_eV) {
          int b = (int)floor((ev - e_min_eV) / (e_max_eV - e_min_eV) * n_bins);
          if (b >= 0 && b < n_bins) spectrum[b] += w;
        }
      }
    } else {
      dg->n_holes_macro += 1.0;
    }
  }
  double uf = 0.0;
  for (long o = 0; o < s->nfield; o++) {
    for (int d = 0; d < 3; d++) {
      double e = s->F[FEX + d][o], b = s->F[FBX + d][o];
      uf += 0.5 * OR_EPS0 * e * e + 0.5 * b * b / OR_MU0;
    }
    if (ne[o] > dg->n_e_peak) dg->n_e_peak = ne[o];
    if (ed[o] > dg->energy_density_peak) dg->energy_density_peak = ed[o];
    if (fabs(rho[o]) > dg->rho_max) dg->rho_max = fabs(rho[o]);
  }
  double gmax = 0.0;
  for (int k = 4; k <= nz - 4; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        long o = fidx(s, i, j, k);
        long ox = fidx(s, i - 1, j, k), oy = fidx(s, i, j - 1, k),
             oz = fidx(s, i, j, k - 1);
        double div =
            ((s->F[FEX][o] + s->F[FPX][o]) - (s->F[FEX][ox] + s->F[FPX][ox])) /
                s->cfg.dx +
            ((s->F[FEY][o] + s->F[FPY][o]) - (s->F[FEY][oy] + s->F[FPY][oy])) /
                s->cfg.dy +
            ((s->F[FEZ][o] + s->F[FPZ][o]) - (s->F[FEZ][oz] + s->F[FPZ][oz])) /
                s->cfg.dz;
        double r = fabs(OR_EPS0 * div - rho[o]);
        if (r > gmax) gmax = r;
      }
  dg->gauss_residual_max = gmax;
  dg->U_field = uf * s->V;
  dg->U_kinetic = kin;
  dg->U_ionization = s->U_ion;
  dg->U_absorbed = kin + s->U_ion;
  /* incident energy: the peak fluence times the sum over the entrance
   * nodes of the polarised component of spot^2 dx dy (F Lx Ly for a plane
   * wave, pi w0^2 F / 2 for a spot well inside the box) */
  double area = 0.0;
  for (int j = 0; j < ny; j++)
    for (int i = 0; i < nx; i++) {
      double sp = s->cfg.pol == 0 ? or_spot(s, (i + 0.5) * s->cfg.dx, j * s->cfg.dy)
                                  : or_spot(s, i * s->cfg.dx, (j + 0.5) * s->cfg.dy);
      area += sp * sp * s->cfg.dx * s->cfg.dy;
    }
  dg->U_incident = s->cfg.fluence * area;
  dg->frac_absorbed = dg->U_absorbed / dg->U_incident;
  dg->U_joule = s->U_joule;
  dg->N_pairs = s->N_pairs;
  dg->step = (double)s->step;
  /* Poynting balance: reflected and transmitted fractions of the energy
   * that came in through the front plane, and the net energy that stayed
   * between the planes (1 - R - T when nothing enters through the back) */
  dg->flux_front = s->flux_plane[0];
  dg->flux_back = s->flux_plane[1];
  dg->U_fwd_front = s->U_fwd[0];
  dg->U_bwd_front = s->U_bwd[0];
  dg->U_fwd_back = s->U_fwd[1];
  dg->U_bwd_back = s->U_bwd[1];
  if (s->U_fwd[0] > 0.0) {
    dg->frac_reflected = s->U_bwd[0] / s->U_fwd[0];
    dg->frac_transmitted = s->U_fwd[1] / s->U_fwd[0];
    dg->frac_absorbed_flux =
        ((s->U_fwd[0] - s->U_bwd[0]) - (s->U_fwd[1] - s->U_bwd[1])) / s->U_fwd[0];
  }
  free(ne);
  free(ed);
  free(rho);
}

/* ------------------------------------------------------------------------ */
/* State access for the tests                                               */
/* ------------------------------------------------------------------------ */
void or_info(const or_sim *s, double *dt, int *NW, long *nfield, long *nmat,
             long *np, long *step, double *E0) {
  *dt = s->dt;
  *NW = s->NW;
  *nfield = s->nfield;
  *nmat = s->nmat;
  *np = s->np;
  *step = s->step;
  *E0 = s->E0;
}

void or_get_fields(const or_sim *s, double *out) {
  for (int c = 0; c < NCOMP; c++)
    memcpy(out + (long)c * s->nfield, s->F[c], s->nfield * sizeof(double));
}

void or_set_fields(or_sim *s, const double *in) {
  for (int c = 0; c < NCOMP; c++)
    memcpy(s->F[c], in + (long)c * s->nfield, s->nfield * sizeof(double));
}

static const or_sim *g_sort_sim;
static int cmp_id(const void *a, const void *b) {
  uint64_t x = g_sort_sim->pid[*(const long *)a],
           y = g_sort_sim->pid[*(const long *)b];
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* Particles in ascending id order. */
void or_get_particles(const or_sim *s, uint64_t *id, int32_t *cell,
                      double *off, double *u, uint32_t *tag) {
  long *ord = malloc((s->np ? s->np : 1) * sizeof(long));
  for (long p = 0; p < s->np; p++) ord[p] = p;
  g_sort_sim = s;
  qsort(ord, s->np, sizeof(long), cmp_id);
  for (long q = 0; q < s->np; q++) {
    long p = ord[q];
    id[q] = s->pid[p];
    cell[q] = s->pcell[p];
    for (int d = 0; d < 3; d++) {
      off[3 * q + d] = s->poff[3 * p + d];
      u[3 * q + d] = s->pu[3 * p + d];
    }
    tag[q] = s->ptag[p];
  }
  free(ord);
}

void or_set_particles(or_sim *s, long n, const uint64_t *id,
                      const int32_t *cell, const double *off, const double *u,
                      const uint32_t *tag) {
  grow(s, n);
  s->np = n;
  memcpy(s->pid, id, n * sizeof(uint64_t));
  memcpy(s->pcell, cell, n * sizeof(int32_t));
  memcpy(s->poff, off, 3 * n * sizeof(double));
  memcpy(s->pu, u, 3 * n * sizeof(double));
  memcpy(s->ptag, tag, n * sizeof(uint32_t));
}

void or_get_material(const or_sim *s, uint32_t *alive, double *win,
                     double *eamp, uint64_t *T, uint8_t *Talways) {
  if (alive) memcpy(alive, s->alive, s->nmat * sizeof(uint32_t));
  if (win) memcpy(win, s->win, (size_t)s->NW * s->nmat * sizeof(double));
  if (eamp) memcpy(eamp, s->eamp, s->nmat * sizeof(double));
  if (T) memcpy(T, s->T, s->nmat * sizeof(uint64_t));
  if (Talways) memcpy(Talways, s->Talways, s->nmat);
}

void or_set_material(or_sim *s, const uint32_t *alive, const double *win) {
  if (alive) memcpy(s->alive, alive, s->nmat * sizeof(uint32_t));
  if (win) memcpy(s->win, win, (size_t)s->NW * s->nmat * sizeof(double));
}

void or_get_scalars(const or_sim *s, double out[4]) {
  out[0] = s->U_joule;
  out[1] = s->N_pairs;
  out[2] = s->U_ion;
  out[3] = s->n_events;
}

void or_set_scalars(or_sim *s, long step, const double in[4]) {
  s->step = step;
  s->U_joule = in[0];
  s->N_pairs = in[1];
  s->U_ion = in[2];
  s->n_events = in[3];
}

/* Poynting time integrals [fwd front, bwd front, fwd back, bwd back]. */
void or_get_flux(const or_sim *s, double out[4]) {
  out[0] = s->U_fwd[0];
  out[1] = s->U_bwd[0];
  out[2] = s->U_fwd[1];
  out[3] = s->U_bwd[1];
}

void or_set_flux(or_sim *s, const double in[4]) {
  s->U_fwd[0] = in[0];
  s->U_bwd[0] = in[1];
  s->U_fwd[1] = in[2];
  s->U_bwd[1] = in[3];
}

/* K and K - E of a simulation as its rate sees them (its tables or in situ). */
void or_sim_ellip(const or_sim *s, double m, double *K, double *KmE) {
  or_ellip_table(s->tabK, s->tabE, s->ntab, m, 1.0 - m, K, KmE);
}

/* Threads the parallel loops use: 1 in the serial build. */
int or_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Incident field value, for the boundary tests. */
double or_incident(const or_sim *s, double t) { return e_inc(s, t); }

/* Ionisation threshold of a cell of layer L at window amplitude E: the rate
 * and the threshold exactly as the window/Keldysh pass computes them (for
 * item-by-item checks of a larger run's thresholds). */
void or_cell_threshold(const or_sim *s, int L, double E, uint64_t *T, int *always) {
  uint8_t a = 0;
  double W = keldysh_rate(E, s->omega, s->gapJ[L], s->mstar[L], s->cfg.keldysh_terms, NULL, NULL,
                          s->tabK, s->tabE, s->ntab);
  ion_threshold(W, s->cfg.layers[L].n_mol, s->dt, T, &a);
  *always = a;
}
