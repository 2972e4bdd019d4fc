/*
 * pic.h - C ABI of the GB300 (sm_103a) particle-in-cell library for few-cycle
 * laser pulses driving dielectrics (Smith et al., arXiv 2502.13695).
 *
 * One time step (pic_step) advances, entirely in CUDA kernels on one GPU:
 *   - field gather with quadratic (TSC) weights, relativistic Boris push,
 *     charge-conserving Esirkepov current deposition (Sec. 1: macroparticles
 *     advanced by the Lorentz force; Sec. 4.1: shape function);
 *   - the Yee update of E and B with the dielectric's polarisation current
 *     (Sec. 2.3, refraction), the laser entering through the z_min boundary
 *     and outflow faces (Sec. 3, Sec. 3.1);
 *   - the per-cell maximum of |E| over the last optical cycle (Sec. 2.1,
 *     rolling window) and the Keldysh photoionisation rate (Sec. 2.1, Eqs.
 *     for x, W and Q);
 *   - counter-based Philox4x32-10 draws keyed by (seed, step, cell, slot group) that
 *     ionise each molecule at most once (Sec. 2.1) into an electron and a
 *     hole with the Table 1 effective masses (Sec. 3.2).
 *
 * Conventions
 *   - Units are SI.  Cell (i, j, k) spans [i dx, (i+1) dx) x ...; linear cell
 *     id c = (k ny + j) nx + i.  The laser travels along +z; x and y are
 *     periodic; z has absorbing (Silver-Mueller) faces, the laser enters at
 *     z = 0.  Charged particles that come within two cells of a z face leave.
 *   - Field arrays have nx * ny * (nz + 1) entries (z planes 0..nz); a
 *     component at a half-integer z position k + 1/2 is stored at plane k and
 *     plane nz is unused for it.  Staggering (Yee): Ex (i+1/2, j, k),
 *     Ey (i, j+1/2, k), Ez (i, j, k+1/2), Bx (i, j+1/2, k+1/2),
 *     By (i+1/2, j, k+1/2), Bz (i+1/2, j+1/2, k); J like E.
 *   - Polarisation state is stored in field units: P/eps0 [V/m] and
 *     (dP/dt)/eps0 [V/(m s)], at the E points.
 *   - A field point on plane k belongs to cell (i, j, k); a layer [z0, z1)
 *     makes the E points of planes z0 .. z1-1 polarisable.
 *
 * Errors: every call returns PIC_OK (0) or a negative PIC_E* code and sets a
 * thread-local message readable with pic_last_error().  No call aborts the
 * process or traps the GPU.  Device-detected errors (pool overflow) are
 * latched in the handle and reported by the next pic_sync / pic_diagnostics
 * / state read.  A handle is not thread-safe.
 */
#ifndef PIC_GB300_H
#define PIC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIC_OK 0
#define PIC_EINVAL (-1)   /* bad sizes, layer outside the grid, CFL > 1 ... */
#define PIC_ENOMEM (-2)   /* device memory or caller arena too small */
#define PIC_EPOOL (-3)    /* ionisation outgrew the charged-particle pool */
#define PIC_ETIMEOUT (-4) /* a bounded device wait gave up */
#define PIC_ECUDA (-5)    /* any CUDA runtime error */
#define PIC_ESTATE (-6)   /* call not valid in the handle's current state */
#define PIC_ECOLL (-7)    /* a cell held more charged particles than a collision
                             pass handles (128) */
#define PIC_EIO (-8)      /* a checkpoint file could not be opened, written or
                             read, or does not match this library's layout */

#define PIC_FP64 0
#define PIC_FP32 1
#define PIC_MAX_LAYERS 128

/* Step phases for pic_step_phases (a full step is PIC_PHASE_ALL). */
#define PIC_PHASE_PARTICLES 1 /* gather, Boris, move, deposit, z outflow */
#define PIC_PHASE_FIELDS 2    /* B half step, E (+ polarisation), B half */
#define PIC_PHASE_WINDOW 4    /* |E| window and Keldysh threshold per cell */
#define PIC_PHASE_IONIZE 8    /* ionisation draws and pair creation */
#define PIC_PHASE_ADVANCE 16  /* Poynting split of the step's end fields, step
                                 counter += 1 */
#define PIC_PHASE_COLLIDE 32  /* binary collisions (when coll_every divides step + 1);
                                 runs after the particles, before the fields */
#define PIC_PHASE_ALL 63

typedef struct pic_ctx *pic_handle;

/* Grid and numerical parameters. */
typedef struct {
  int nx, ny, nz;      /* cells; nx, ny >= 4, 8 <= nz < 65535 */
  int precision;       /* PIC_FP64 or PIC_FP32 (fields, push, deposit) */
  double dx, dy, dz;   /* cell sizes [m] */
  double cfl;          /* dt = cfl / (c sqrt(1/dx^2+1/dy^2+1/dz^2)), 0 < cfl <= 1
                          (Sec. 3.1 uses 0.95) */
  double pool_factor;  /* charged-slot capacity = pool_factor * neutrals + 1024 */
  int keldysh_terms;   /* terms of the Q series cap (Sec. 2.1: 500) */
  int sort_interval;   /* steps between cell sorts of the pool (0: 16) */
  int imax_every;      /* steps between records of the intensity map (Sec. 5
                          records every 0.5 fs): 0 = round(0.5 fs / dt), < 0 off */
  int coll_every;      /* steps between binary-collision passes among electrons
                          and holes (Sec. 2.2), each over coll_every * dt; 0 = none */
  int elliptic_table;  /* complete elliptic integrals of the Keldysh rate: 0 in
                          situ (arithmetic-geometric mean); N >= 2 from N-point
                          tables as the paper reads them (Sec. 2.1: 1000
                          points): K(i/N), E(i/N), i < N, linear in the
                          parameter between entries, in situ past the last */
  int pml_cells;       /* transverse faces (Sec. 3.1 uses outflow faces): 0
                          periodic in x and y; L > 0 (2 L < nx, ny) absorbing
                          layers of L cells on each side of the x = 0 and y = 0
                          seams: a convolutional PML (Roden and Gedney 2000,
                          kappa 1, alpha 0, conductivity sigma_max (d / L)^3 at
                          depth d, sigma_max = 0.8 * 4 / (eta0 * cell size)),
                          and a particle that ends a push inside them leaves
                          the simulation, as through the z faces.  Their
                          convolution state lives in the arena (checkpoints
                          keep it); pic_set_fields / pic_set_state leave it
                          as the run left it */
} pic_grid;

/* One dielectric layer: z cells [z0, z1) over the whole transverse plane.
 * Table 1 (Sec. 3.2) supplies gap, masses and density; the Lorentz pole
 * (omega0_eV, INFINITY for a static permittivity) and the index fix the
 * polarisation; temp_eV and mol_mass_amu the neutrals' thermal velocity. */
typedef struct {
  int z0, z1;         /* 2 <= z0 < z1 <= nz - 2, layers must not overlap */
  int ppc;            /* neutral macroparticles per cell, 1..32 */
  int reserved;
  double n_index;     /* refractive index at the laser wavelength */
  double gap_eV;      /* band gap Delta */
  double me_star;     /* electron effective mass / m_e */
  double mh_star;     /* hole effective mass / m_e */
  double n_mol;       /* molecular density [m^-3] */
  double omega0_eV;   /* Lorentz pole photon energy, INFINITY = static eps */
  double damping;     /* Lorentz damping rate [rad/s] */
  double temp_eV;     /* neutral temperature */
  double mol_mass_amu;/* molecular mass */
  double e_melt;      /* damage energy densities [J/m^3] (Sec. 4.2, Sec. 5: */
  double e_boil;      /*   melting, boiling, dissociation); 0 = not given */
  double e_dissoc;
} pic_layer;

typedef struct {
  int n_layers;             /* 0..PIC_MAX_LAYERS */
  int reserved;
  const pic_layer *layers;  /* host array, copied by pic_create */
} pic_material;

/* Laser (Sec. 3): a wave along +z injected through the z = 0 face.  Time
 * envelope: Gaussian in intensity with FWHM fwhm, or the paper's
 * sine-squared pulse (field envelope cos^2(pi (t - t_peak) / T) for
 * |t - t_peak| < T / 2, T chosen so that the intensity FWHM is fwhm).
 * Transverse profile: plane wave, or a Gaussian spot exp(-r^2 / w0^2) about
 * the box centre (x and y stay periodic).  fluence is the peak fluence
 * F = int c eps0 E^2 dt at the spot centre (for a spot, F = 2 E_las /
 * (pi w0^2), Sec. 3). */
typedef struct {
  double lambda;   /* wavelength [m] */
  double fwhm;     /* intensity FWHM [s] */
  double fluence;  /* [J/m^2] */
  double cep;      /* carrier-envelope phase [rad] */
  double t_peak;   /* time of the envelope peak at z = 0 [s] */
  int pol;         /* 0: E along x, 1: E along y */
  int shape;       /* 0: Gaussian, 1: sine-squared */
  double w0;       /* spot radius [m] (1/e^2 of the intensity); 0: plane wave */
} pic_pulse;

/* Sizes and derived constants of a configuration (pic_query / pic_info). */
typedef struct {
  double dt;                 /* time step [s] */
  double E0;                 /* laser peak field [V/m] */
  int NW;                    /* samples in the amplitude window (one cycle) */
  int n_mplanes;             /* z planes that hold material */
  long long nfield;          /* nx * ny * (nz + 1) */
  long long nmat;            /* material cells */
  long long n_neutrals;      /* initial neutral macroparticles */
  long long capacity;        /* charged-particle slots */
  long long n_particles;     /* charged-particle slots in use (pic_info) */
  long long step;            /* steps the device has completed (pic_info) */
  size_t arena_bytes;        /* device bytes pic_create needs */
  long long launches;        /* kernels launched on the handle so far (pic_info) */
  double particle_steps;     /* charged-particle pushes done so far (pic_info) */
  long long h2d_bytes;       /* host-to-device bytes the library has copied for
                                this handle: create tables, state writes (pic_info) */
  long long d2h_bytes;       /* device-to-host bytes it has copied: state reads,
                                diagnostics, error checks (pic_info) */
} pic_info;

/* Kernel classes reported by pic_profile_read. */
#define PIC_PROF_PUSH 0    /* gather + Boris + deposit */
#define PIC_PROF_FIELDS 1  /* B half step, E + polarisation + z faces, B half step */
#define PIC_PROF_KELDYSH 2 /* Keldysh thresholds of the cells whose amplitude changed */
#define PIC_PROF_WINDOW 3  /* cell-centred |E| window and Keldysh cache check */
#define PIC_PROF_IONIZE 4  /* ionisation draws + pair appends */
#define PIC_PROF_SORT 5    /* pool sort (all its kernels) */
#define PIC_PROF_OTHER 6   /* step counter */
#define PIC_PROF_COLLIDE 7 /* binary collisions (their sort included) */
#define PIC_PROF_N 8

/* FP64 diagnostics (Sec. 4.1 number density, Sec. 4.2 energy density,
 * Sec. 4.3 spectra).  Inputs: n_bins, e_min_eV, e_max_eV, region, spectrum;
 * everything else is output. */
typedef struct {
  double U_incident;         /* F * transverse area [J] */
  double U_kinetic;          /* sum w (gamma - 1) m c^2 over carriers [J] */
  double U_ionization;       /* sum over events w * gap [J] */
  double U_absorbed;         /* U_kinetic + U_ionization [J] */
  double frac_absorbed;      /* U_absorbed / U_incident */
  double U_joule;            /* time integral of sum J.E dV [J] */
  double U_field;            /* sum (eps0 E^2 + B^2 / mu0) / 2 dV [J] */
  double N_pairs;            /* real electron-hole pairs created */
  double n_e_peak;           /* max over nodes of TSC electron density [m^-3] */
  double energy_density_peak;/* max over nodes of TSC electron energy density [J/m^3] */
  double gauss_residual_max; /* max |eps0 div(E + P/eps0) - rho| on planes 4..nz-4 [C/m^3] */
  double rho_max;            /* max |rho| [C/m^3] */
  double n_electrons_macro;  /* electron macroparticles */
  double n_holes_macro;      /* hole macroparticles */
  long long step;            /* steps taken */
  int n_bins;                /* spectrum bins (0: no spectrum) */
  int reserved;
  double e_min_eV, e_max_eV; /* spectrum range, uniform bins */
  int region[6];             /* cell box [i0, i1) x [j0, j1) x [k0, k1) */
  int reserved2[2];
  double *spectrum;          /* caller-owned host array of n_bins: real
                                electrons per bin (electron kinetic energy) */
  /* Poynting split (the reflected and transmitted energy behind the absorbed
   * fraction, Sec. 4.2 and Sec. 5): at a node plane k the transverse E of the
   * plane is paired with B averaged over the planes k - 1/2 and k + 1/2, and
   * split into the wave going along +z, ((Ex + c By) / 2, (Ey - c Bx) / 2),
   * and the one going along -z, ((Ex - c By) / 2, (Ey + c Bx) / 2); c eps0
   * |.|^2 of each, summed over the plane times dx dy, is its power.  The
   * split is taken once per step, at the end of the step (the advance
   * phase), and its powers are summed times dt from step 0.  The planes are
   * halfway between the entrance face and the first material plane and
   * halfway between the last material plane and the far face (nz / 4 and
   * 3 nz / 4 without material), clamped to 1 .. nz - 1. */
  int flux_plane[2];         /* out: node planes of the split (front, back) */
  double U_fwd[2];           /* out: energy carried along +z through each [J] */
  double U_bwd[2];           /* out: energy carried along -z through each [J] */
  double frac_reflected;     /* out: U_bwd[0] / U_fwd[0] (0 while U_fwd[0] = 0) */
  double frac_transmitted;   /* out: U_fwd[1] / U_fwd[0] */
  double frac_absorbed_flux; /* out: (U_fwd[0] - U_bwd[0] - U_fwd[1] + U_bwd[1]) /
                                U_fwd[0], the energy that stayed between the
                                planes (1 - R - T when nothing enters through
                                the back plane) */
} pic_diag;

/* Sizes of a configuration without creating it.  Returns PIC_EINVAL for an
 * invalid configuration. */
int pic_query(const pic_grid *grid, const pic_material *mat,
              const pic_pulse *pulse, pic_info *out);

/* Create a simulation: validate, lay out the device state, initialise the
 * neutrals (Philox streams, no host RNG) and zero the fields.
 *   stream      : cudaStream_t to run on (NULL: the legacy default stream)
 *   d_arena     : caller-owned device memory of >= arena_bytes (pic_query),
 *                 256-byte aligned, or NULL to let the library cudaMalloc it
 *   arena_bytes : size of d_arena (ignored when d_arena is NULL)
 * The caller keeps ownership of d_arena and must keep it alive until
 * pic_destroy. */
int pic_create(const pic_grid *grid, const pic_material *mat,
               const pic_pulse *pulse, uint64_t seed, void *stream,
               void *d_arena, size_t arena_bytes, pic_handle *out);

/* Enqueue n_steps full steps on the handle's stream (asynchronous). */
int pic_step(pic_handle h, int n_steps);

/* Enqueue selected phases of the current step (PIC_PHASE_* mask). */
int pic_step_phases(pic_handle h, int mask);

/* Wait for the handle's stream; report latched device errors. */
int pic_sync(pic_handle h);

/* Per-kernel timing with CUDA events recorded on the handle's stream around
 * every launch (enable != 0 starts a fresh record, 0 stops recording).
 * pic_profile_read synchronises and returns, per PIC_PROF_* class, the summed
 * device milliseconds and launch counts since the last enable. */
int pic_profile(pic_handle h, int enable);
int pic_profile_read(pic_handle h, double ms[PIC_PROF_N], long long launches[PIC_PROF_N]);

/* Synchronous FP64 diagnostics of the current state. */
int pic_diagnostics(pic_handle h, pic_diag *inout);

/* Damage metrics of the current state (Sec. 4.1 electron density and its
 * critical and instability densities, Sec. 4.2 energy density and its
 * melting / boiling / dissociation thresholds, Sec. 5 accumulated intensity).
 * Synchronous; FP64.
 *   region      in: transverse node box [region[0], region[1]) x
 *               [region[2], region[3]) (x then y), 0 <= r0 < r1 <= nx,
 *               0 <= r2 < r3 <= ny.
 *   ne_z, ed_z  out (host, nz + 1 doubles each, or NULL): the mean over the
 *               box's nodes of the TSC-deposited electron density [m^-3] and
 *               electron kinetic-energy density [J/m^3] on every node plane.
 *   layer_out   out (host, 4 doubles per layer, or NULL): per layer the
 *               largest ne_z and ed_z on its node planes z0 <= k < z1, the
 *               largest recorded |E|^2 / E0^2 over its cells, and its
 *               instability density 0.09 * 4 * n_mol (four valence electrons
 *               per molecule).
 *   layer_flags out (host, n_layers ints, or NULL): bit 0 n_e >= the critical
 *               density, bit 1 n_e >= the instability density, bits 2-4 the
 *               energy density >= e_melt, e_boil, e_dissoc (given ones only).
 *   n_crit      out (or NULL): critical density eps0 m_e omega^2 / e^2 of free
 *               electrons at the laser frequency [m^-3].
 * Errors: PIC_EINVAL for a bad region or null handle; PIC_ECUDA. */
int pic_damage(pic_handle h, const int region[4], double *ne_z, double *ed_z,
               double *layer_out, int *layer_flags, double *n_crit);

/* The intensity map: per cell (x fastest, nz * ny * nx doubles into the host
 * array dst) the largest |E^{n+1}|^2 / E0^2 at the cell centre over the
 * recorded steps (every imax_every steps; E0 the incident peak amplitude,
 * raw |E|^2 when the fluence is 0).  Synchronous. */
int pic_get_intensity_max(pic_handle h, double *dst);

int pic_info_get(pic_handle h, pic_info *out);
int pic_destroy(pic_handle h);
const char *pic_last_error(void);

/* ---- state access (synchronous; host pointers; used for per-step parity
 *      and checkpointing) ------------------------------------------------- */

/* 15 * nfield doubles: Ex Ey Ez Bx By Bz Jx Jy Jz Px Py Pz Qx Qy Qz, each in
 * the field layout above; P and Q are P/eps0 and (dP/dt)/eps0 and are zero
 * outside material planes. */
int pic_get_fields(pic_handle h, double *dst);
int pic_set_fields(pic_handle h, const double *src);

/* Charged particles in slot order (unsorted).  *n receives the count; with
 * any array NULL only the count is returned.  off and u are n x 3 (offset in
 * [0,1) within the cell; u = gamma v [m/s]); tag = (birth layer << 1) |
 * species (0 electron, 1 hole); id = 2 gid (+1 for the hole) with
 * gid = birth cell * ppc + slot. */
int pic_get_particles(pic_handle h, long long *n, uint64_t *id, int32_t *cell,
                      double *off, double *u, uint32_t *tag);
int pic_set_particles(pic_handle h, long long n, const uint64_t *id,
                      const int32_t *cell, const double *off, const double *u,
                      const uint32_t *tag);

/* Per material cell m = mplane(k) nx ny + j nx + i: alive neutral bitmask,
 * window amplitude of the last window phase, and the ionisation threshold
 * T = floor(p 2^64) (UINT64_MAX: p = 1).  Any pointer may be NULL. */
int pic_get_material(pic_handle h, uint32_t *alive, double *eamp, uint64_t *T);

/* Load alive bits and the raw amplitude history: win is NW x nmat, slot q
 * holding the most recent sample whose index is q mod NW (samples are
 * numbered by the step that wrote them).  Either pointer may be NULL. */
int pic_set_material(pic_handle h, const uint32_t *alive, const double *win);

/* Accumulators: [U_joule, N_pairs, U_ionization, events]. */
int pic_get_scalars(pic_handle h, long long *step, double out[4]);
int pic_set_scalars(pic_handle h, long long step, const double in[4]);

/* ---- checkpoints ---------------------------------------------------------
 * The paper has no counterpart (its runs are single jobs); this is the
 * resume path of long runs and of a serving loop that parks simulations.
 * pic_save writes the handle's configuration, step state and every
 * device-side quantity to the file at path (host path, created or
 * replaced; written to path.tmp first and renamed, so a failed save leaves
 * no partial file under path).  The particle pool is stored up to its live
 * slot count, so the file holds roughly the state, not the pool capacity.
 * Synchronous on the handle's stream; a handle holding a latched device
 * error (PIC_EPOOL, PIC_ECOLL) is not saved.
 * pic_load creates a handle from such a file, as pic_create would from the
 * stored configuration (same stream / d_arena / arena_bytes rules; the
 * arena size is pic_query's for the configuration that
 * pic_checkpoint_config returns), and restores the state: stepping it gives
 * the results the saved handle would have given.  Files are read by the
 * library build and machine family that wrote them.
 * pic_checkpoint_config reads only the stored configuration: grid, pulse,
 * layers (the caller provides PIC_MAX_LAYERS entries), layer count, seed
 * and the step the file was written at (step may be NULL).
 * Errors: PIC_EINVAL for null pointers; PIC_EIO for a file that cannot be
 * opened, written or read, is not a checkpoint, or does not match this
 * library's state layout; otherwise as pic_create. */
int pic_save(pic_handle h, const char *path);
int pic_checkpoint_config(const char *path, pic_grid *grid, pic_pulse *pulse,
                          pic_layer *layers, int *n_layers, uint64_t *seed,
                          long long *step);
int pic_load(const char *path, void *stream, void *d_arena, size_t arena_bytes,
             pic_handle *out);

/* ---- batches: many simulations advanced by one CUDA graph ----------------
 * Advances uneven simulations together (the batched fluence scan): the
 * batch captures one period of steps of every member into a CUDA graph, each
 * member's kernels on that member's own stream, forked from and joined to
 * the batch stream, and replays it; the period is the least common multiple
 * of 2 sort_interval over the members, after which every member's buffers
 * are back in their starting order.  Members keep their own state and may be
 * read (or stepped alone) between batch calls; a member stepped alone makes
 * the next batch call capture again.
 *   members : n handles, each created on a non-NULL stream (members may share
 *             one, which serialises them)
 *   stream  : batch stream, not a member's; NULL lets the batch create and
 *             own one
 * pic_batch_step enqueues asynchronously; pic_batch_sync waits for the batch
 * and reports member errors as pic_sync does. */
typedef struct pic_batch_ctx *pic_batch;
int pic_batch_create(pic_handle const *members, int n, void *stream, pic_batch *out);
int pic_batch_step(pic_batch b, int n_steps);
int pic_batch_sync(pic_batch b);
int pic_batch_destroy(pic_batch b);

/* How a batch steps.  By default the graph holds every member's own
 * launches, each on its stream (branches the device runs side by side).
 * pic_batch_set_launches(b, 1) asks for batch launches instead: when every
 * member has the same precision, the same points per thread in the field
 * kernels (FP32 with nx a multiple of 4, or not) and the same pool-sort
 * schedule, and none runs collisions, the graph then holds one launch per
 * phase of a step for all members together (fixed grids laid end to end
 * over the members, particle and Keldysh loops in chunks handed out from a
 * counter), so that launches per step do not grow with the member count.
 * Measured on one GB300, member branches were faster both for the 64-member
 * fluence scan (4.25 s against 4.39 s) and for the serving trace (time to
 * result p99 2.0 s against 2.9 s), so they stay the default.  The setting
 * takes effect at the next capture; 0 returns to member branches.  With
 * batch launches, a
 * pic_batch_step with at least 4 periods left tunes the push's launch shape
 * on the batch itself once the members hold particles (four per resident
 * push thread, or a 64th of their pools; checked before each period
 * until then): four candidates (particles per block task, grid as 1 or 2
 * times the resident blocks), each captured with CUDA events around its push
 * launches and run for one period; the one with the least push time per
 * particle push is kept (every tuning period is a real step of every
 * member).
 *   cap            : entries the arrays hold
 *   chunk, grid_mult, ms, ns_per_push : per candidate (any may be NULL): the
 *                    shape, its push time over the period [ms] and per
 *                    particle push [ns]
 *   n, pick        : candidates tuned (0: not yet) and the index kept (-1)
 *   batch_launches : 1 when the batch steps with batch launches
 * The paper has no counterpart (its runs are single jobs). */
int pic_batch_set_launches(pic_batch b, int one_launch_per_phase);
int pic_batch_tuning(pic_batch b, int cap, long long *chunk, int *grid_mult, double *ms,
                     double *ns_per_push, int *n, int *pick, int *batch_launches);

/* ---- serving: continuous batching of submitted simulations ---------------
 * The paper runs one simulation per job; this is the request loop of a
 * fluence or stack sweep served on one GPU.  A server owns a host worker
 * thread on the device current at pic_serve_create.  Submitted requests
 * wait in submission order and are admitted as soon as their state
 * (pic_query's arena_bytes) fits budget_bytes next to the running
 * simulations, whose state stays resident on the device until they finish.
 * A request that fits may be admitted before earlier ones that do not,
 * unless the oldest waiting request has waited 1 s or more: then nothing
 * passes it and memory frees up for it.  The state lives in the server's
 * own device memory: chunks of 16 GiB (or one request's size) reserved with
 * cudaMalloc when no free range fits, never more than budget_bytes in all,
 * kept until pic_serve_destroy and handed out first-fit, so that admitting
 * and finishing requests allocates and frees no device memory.
 * The running simulations with at least `quantum` steps left advance
 * together from one CUDA graph (pic_batch_*, rebuilt when that set
 * changes); one with fewer steps left takes them alone.  A finished
 * request's FP64 diagnostics are kept until its ticket is polled, and its
 * device memory is released at once.
 *   pic_serve_create  : budget_bytes >= 1, quantum >= 1 steps.
 *   pic_serve_submit  : copies the configuration (as pic_create takes it)
 *                       and returns a ticket (a request that cannot get
 *                       device memory even with nothing running ends with
 *                       PIC_ENOMEM).  n_bins, e_min_eV, e_max_eV
 *                       ask for the spectrum of pic_diagnostics (n_bins 0:
 *                       none); fields_out, if not NULL, is a host array of
 *                       15 * nfield doubles (layout of pic_get_fields) that
 *                       receives the final fields and must stay valid until
 *                       the ticket is polled done.  PIC_EINVAL for a bad
 *                       configuration or request, PIC_ENOMEM for one whose
 *                       state alone exceeds the budget.
 *   pic_serve_poll    : waits up to wait_ms for the ticket; *done = 1 once it
 *                       has finished, then fills diag (its spectrum pointer
 *                       must hold the submitted n_bins) and times =
 *                       {submitted, admitted, finished} in seconds since
 *                       pic_serve_create, releases the ticket and returns
 *                       the request's own status (PIC_OK, or the error that
 *                       ended it: PIC_EPOOL, PIC_ECOLL, PIC_ENOMEM, PIC_ECUDA).
 *                       *done = 0 with PIC_OK while it runs or waits;
 *                       PIC_EINVAL for an unknown ticket.
 *   pic_serve_destroy : stops the worker after its current quantum; requests
 *                       not yet finished are dropped with their state.
 * The server is thread-safe: submit and poll may come from any thread. */
typedef struct pic_server_ctx *pic_server;
int pic_serve_create(double budget_bytes, int quantum, pic_server *out);
int pic_serve_submit(pic_server s, const pic_grid *grid, const pic_material *mat,
                     const pic_pulse *pulse, uint64_t seed, long long n_steps,
                     int n_bins, double e_min_eV, double e_max_eV,
                     double *fields_out, long long *ticket);
int pic_serve_poll(pic_server s, long long ticket, int wait_ms, int *done,
                   pic_diag *diag, double times[3]);
int pic_serve_destroy(pic_server s);

/* ---- allocation-free field energy -------------------------------------
 * The paper has no counterpart: this is a service for callers that cannot
 * allocate device memory, such as a process whose device memory is planned
 * up front by another allocator (a serving loop holding a fixed budget, or a
 * host framework whose caching allocator owns the device), where a stray
 * cudaMalloc can fail or fragment the plan.  It
 * computes sum over n field points of (eps0 |E|^2 + |B|^2 / mu0) / 2 times
 * cell_volume, the U_field of pic_diagnostics, with no allocation: its
 * scratch is one FP64 partial per block of 2048 points in a static device
 * array of 512 KiB that every GPU loading this library keeps until the
 * process exits.
 *   precision   : PIC_FP32 or PIC_FP64, the element type of the six arrays
 *   Ex..Bz      : device arrays of n elements each (caller-owned)
 *   n           : 0 .. 134217728 (65536 blocks of 2048); larger is PIC_EINVAL
 *   d_out       : device pointer to one double, written on `stream`
 *   stream      : cudaStream_t (NULL: the legacy default stream)
 * The result is deterministic (fixed partition, fixed summation order).  The
 * first call on each device looks up the scratch address
 * (cudaGetSymbolAddress) with that device current; make it before any stream
 * capture.  The address is then kept for the device until the process exits,
 * so it does not survive cudaDeviceReset.  All calls share the scratch: calls
 * that overlap on the GPU (on different streams, or from different threads)
 * race and must be serialised by the caller.  A CUDA error that earlier work
 * left pending on the calling thread is reported as this call's PIC_ECUDA. */
int pic_field_energy_noalloc(int precision, const void *Ex, const void *Ey, const void *Ez,
                             const void *Bx, const void *By, const void *Bz, long long n,
                             double cell_volume, double *d_out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* PIC_GB300_H */
