/*
 * prad.h - C ABI of the GB300 (sm_103a) synchrotron-emission particle step.
 *
 * Implements the per-timestep particle hot path of E. Wallin, A. Gonoskov and
 * M. Marklund, "Effects of high energy photon emissions in laser generated
 * ultra-relativistic plasmas: real-time synchrotron simulations"
 * (arXiv:1409.5574):
 *
 *   field gather -> Boris push -> effective field H_eff and omega_c (Eq. (1))
 *   -> Monte Carlo emission of synchrotron macro-photons sampled from
 *   Eqs. (7)-(8) with the S(x) noise-reduction proposal (Eqs. (11)-(13))
 *   -> photon append -> emitted-energy ledger booked beside the
 *   Landau-Lifshitz loss of Eq. (4) (the comparison of Fig. 3).
 *
 * Conventions shared by every call
 * --------------------------------
 * - All calls return int: PRAD_OK (0), a negative PRAD_ERR_* code, or a
 *   positive PRAD_WARN_* code.  They never abort, print or throw;
 *   prad_last_error() returns a message for the last failing call of a
 *   context.
 * - Pointers named "device" must be CUDA device (or managed) memory of the
 *   context's device; "host" pointers are ordinary host memory.  The library
 *   never frees memory it did not allocate.
 * - Units.  The problem is described in SI (dt in s, fields in V/m and T,
 *   wavelength in m).  Particle state is normalised by a reference angular
 *   frequency omega_ref: time in 1/omega_ref, length in c/omega_ref,
 *   momentum u = p/(m_e c).  Photon and ledger energies are in m_e c^2.
 * - Every kernel of a context runs on the context's stream (cfg.stream).
 *   push_emit is asynchronous; get_photons, energy_budget and get_ledger
 *   synchronise that stream before returning.
 * - Random numbers: Philox4x32-10 with key (seed_lo, seed_hi) and counter
 *   (pid, step, 0, ensemble); results do not depend on launch shape, on how
 *   a run is split into calls, or on the number of substeps per launch.
 */
#ifndef PRAD_H
#define PRAD_H

#ifndef __CUDACC_RTC__
#include <stdint.h>
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define PRAD_OK 0
#define PRAD_ERR_ARG -1      /* invalid argument (null, size, enum, alignment) */
#define PRAD_ERR_CUDA -2     /* a CUDA runtime call failed */
#define PRAD_ERR_CAPACITY -3 /* a buffer of capacity 0 was given */
#define PRAD_ERR_TIMEOUT -4  /* a bounded device wait gave up */
#define PRAD_ERR_STATE -5    /* call made in the wrong state (e.g. no fields) */
#define PRAD_WARN_NAN 1      /* non-finite particles were found and frozen */

/* ---- enums ------------------------------------------------------------- */
enum prad_precision { PRAD_FP32 = 0, PRAD_FP64 = 1 };
enum prad_sampler {
  PRAD_SAMPLER_TABLE = 0,        /* S(x) proposal + tabulated F, Eq. (13) */
  PRAD_SAMPLER_MLP = 1,          /* learned inverse CDF (no fallback)     */
  PRAD_SAMPLER_MLP_FALLBACK = 2  /* learned inverse CDF, table fallback   */
};
enum prad_rr_mode {
  PRAD_RR_OFF = 0,    /* no LL ledger, no LL kick                          */
  PRAD_RR_LEDGER = 1, /* book the LL loss of Eq. (4), no momentum change   */
  PRAD_RR_APPLY = 2   /* book it and apply the LL force to the momentum    */
};
enum prad_heff_form {
  PRAD_HEFF_FIELD = 0,   /* H^2 = |E + beta x B|^2 - (E.beta)^2            */
  PRAD_HEFF_MOMENTUM = 1 /* Eq. (9), from the momentum change of the step  */
};
enum prad_field_kind {
  PRAD_FIELD_CONST = 0,      /* uniform constant E, B                      */
  PRAD_FIELD_PLANE_WAVE = 1, /* circularly polarised plane wave along +-x  */
  PRAD_FIELD_YEE2D = 2       /* staggered 2D Yee grid, quadratic splines   */
};

/* ---- configuration ----------------------------------------------------- */
typedef struct prad_config {
  int32_t precision;        /* prad_precision: FP32 push (FP64 ledger) or FP64 */
  int32_t sampler;          /* prad_sampler (MLP samplers: FP32 only)        */
  int32_t rr_mode;          /* prad_rr_mode                                  */
  int32_t heff_form;        /* prad_heff_form                                */
  double dt;                /* time step [s], > 0                            */
  double omega_ref;         /* reference angular frequency [rad/s], > 0      */
  double charge;            /* particle charge in e: -1 electron, +1 positron */
  uint64_t seed;            /* Philox key                                     */
  uint32_t ensemble;        /* Philox counter word 3                          */
  int32_t steps_per_launch; /* substeps fused per kernel launch; 0 = 1       */
  int64_t photon_capacity;  /* photon records held on the device, >= 1       */
  int64_t max_particles;    /* per-particle ledger entries, >= 1             */
  void* stream;             /* cudaStream_t for every launch; NULL = default */
  int32_t block_size;       /* threads per block (0 = 256); multiple of 32   */
  int32_t blocks_per_sm;    /* blocks per SM of the persistent grid, capped
                               at the kernel's occupancy (0 = occupancy)   */
  int32_t sort_interval;    /* YEE2D with a pid array: reorder particles by
                               32 x 32-cell tile (and cell) every this many
                               steps and gather from shared-memory field
                               tiles (0 = never sort; plain gather)       */
  int32_t batch_chunk;      /* push_emit_batch: particles per work item
                               (0 = 2048); multiple of 32                 */
  int32_t use_graph;        /* push_emit_batch: capture the launches of a
                               call in a CUDA graph and replay it when the
                               next call has the same shape (0 = off)     */
  /* Super-photon control (Sec. "Monte Carlo method": the number of
   * super-photons per super-particle and time step, and the number of real
   * photons one represents, set at runtime).  n_try trials per particle and
   * step (0 = 1; table sampler only), each with its own Philox block (tag 0
   * for trial 0, 0x10000 + j for trial j) and 1/n_try of dN; a particle
   * takes part in a step's emission with probability select_prob (decided
   * by Philox word 3 of trial 0; 0 = 1) and its records then carry weight
   * k w / select_prob.  Both keep the expected emission unchanged. */
  int32_t n_try;
  int32_t diagnostics;      /* bit mask of PRAD_DIAG_*                        */
  int32_t specialize;       /* 1 = run the standard FP32 step of the plane
                               wave (any sampler) and of the Yee grid (plain
                               and tile-staged), without control or
                               diagnostics, through kernels compiled at run
                               time by NVRTC with this context's constants
                               (time step, wave or grid geometry, Philox key
                               ...) as literals: the same results, fewer
                               loads.  Each variant is compiled (~0.3-0.7 s)
                               at its first launch and kept until
                               prad_destroy; every distinct set of constants
                               (prad_set_fields with another wave or grid)
                               compiles its own, so it suits runs whose
                               constants stay fixed.  Make the first call of
                               a variant outside CUDA-graph capture (it loads
                               a module).  prad_push_emit fails with
                               PRAD_ERR_CUDA if NVRTC or the driver cannot
                               provide a kernel.  NVRTC is the toolkit's
                               libnvrtc.so.13, or the library the environment
                               variable PRAD_NVRTC_LIBRARY names.
                               0 = compiled-in kernels only.  */
  double select_prob;
} prad_config;

/* Diagnostics counted in prad_stats when enabled in prad_config.diagnostics */
#define PRAD_DIAG_WIGGLER 1 /* steps outside the synchrotron (wiggler) regime:
                               Omega tau_EM < 1 with tau_EM the field period
                               the particle sees, 1 / (omega_L |1 - dir beta_x|)
                               (Eq. (3) context; PLANE_WAVE fields only)   */
/* Angular spread of the emission (Eqs. (5)-(6), the circular-motion
 * spectrum by angle), an option beside the paper's collinear photons:
 * every record's direction is turned out of the plane of the step's orbit
 * (the plane of u^n and u^(n+1)) by theta = psi / gamma, gamma of the step's
 * mean momentum, psi drawn from Eq. (5)'s density at the record's
 * x = omega / omega_c, proportional to (1 + psi^2)^2 K_2/3(xi)^2 +
 * (1 + psi^2) psi^2 K_1/3(xi)^2 with xi = (x/2)(1 + psi^2)^(3/2) (Eq. (6)).
 * The uniform and the sign come from Philox block (pid, step, 0x20000 + j,
 * ensemble), j the trial; the draw of psi is a table lookup (~2e-4
 * relative in psi).  Energies, weights, ledgers and counters are those of
 * the collinear run.  Table sampler only (prad_init fails with
 * PRAD_ERR_ARG otherwise), not in batched calls (prad_push_emit_batch and
 * prad_autotune_batch fail with PRAD_ERR_ARG); the context holds a 225 KB
 * device table, built on the host at the first such prad_init of the
 * process (~0.3 s). */
#define PRAD_DIAG_ANGLE_SPREAD 2
/* Geometry of the angular spread's table (prad_angle_table): PRAD_ANG_NL
 * rows uniform in ln x over [PRAD_ANG_LX0, PRAD_ANG_LX1] and PRAD_ANG_NV
 * columns uniform in v = sqrt(-ln(1 - u)) over [0, PRAD_ANG_VMAX]; entry
 * (row, column) is psi / (v s(x)) with s(x) = (2/x)^(1/3) (1 + x)^(-1/6)
 * (0 in column 0). */
#define PRAD_ANG_NL 225
#define PRAD_ANG_NV 257
#define PRAD_ANG_LX0 (-18.420680743952367) /* ln 1e-8 */
#define PRAD_ANG_LX1 3.6888794541139363    /* ln 40   */
#define PRAD_ANG_VMAX 4.8

/* ---- field description ------------------------------------------------- */
typedef struct prad_fields {
  int32_t kind;      /* prad_field_kind                                      */
  int32_t dir;       /* PLANE_WAVE: +1 propagates along +x, -1 along -x      */
  int32_t hand;      /* PLANE_WAVE: +1 / -1 handedness of the polarisation  */
  int32_t periodic;  /* YEE2D: 1 = wrap positions and indices (only mode)    */
  double E[3];       /* CONST: E [V/m]                                       */
  double B[3];       /* CONST: B [T]                                         */
  double a0;         /* PLANE_WAVE: normalised amplitude e E0 / (m c omega_L) */
  double lambda;     /* PLANE_WAVE: wavelength [m]                           */
  double phase0;     /* PLANE_WAVE: phase at t = 0, x = 0 [rad]              */
  /* YEE2D: six device planes Ex Ey Ez Bx By Bz, float32, row-major [ny][nx],
   * normalised (E in m c omega_ref / e, B in m omega_ref / e).  Staggering:
   * Ex (i+1/2, j), Ey (i, j+1/2), Ez (i, j), Bx (i, j+1/2), By (i+1/2, j),
   * Bz (i+1/2, j+1/2).  BORROWED: the caller keeps them alive and unchanged
   * until the next prad_set_fields or prad_destroy. */
  const float* yee[6];
  int32_t nx, ny;    /* YEE2D grid size, >= 4 each                           */
  double dx, dy;     /* YEE2D cell size [c/omega_ref]                        */
  double x0, y0;     /* YEE2D position of node (0, 0) [c/omega_ref]          */
} prad_fields;

/* ---- particles ---------------------------------------------------------- */
typedef struct prad_particles {
  /* Device SoA arrays of n entries, float (FP32 precision) or double (FP64),
   * advanced in place.  BORROWED for the duration of the call's kernels.
   * x, y, ux, uy, uz, w are required; z may be NULL for YEE2D (2D3V).
   * u holds u^{n-1/2} on entry and u^{n+nsteps-1/2} on return; w is the
   * macro-particle weight (read only). */
  void *x, *y, *z, *ux, *uy, *uz;
  void* w;  /* read only in push_emit; reordered by prad_sort_by_tile */
  /* Optional device array of n particle ids (NULL: particle i has id
   * pid0 + i).  The id is Philox counter word 0 and selects the ledger entry
   * ledger_offset + (id - pid0), so ids move with particles that a tile sort
   * reorders.  Ids outside [pid0, pid0 + max_particles - ledger_offset) are
   * not booked (status bit 1 is set). */
  uint32_t* pid;
  int64_t ledger_offset; /* ledger entry of id pid0                        */
  uint32_t pid0;
  uint32_t pad0;
  int64_t t0;            /* global index of the first step (time t0*dt)  */
} prad_particles;

/* ---- photon records ------------------------------------------------------ */
typedef struct prad_photons {
  /* Caller-owned arrays of at least `cap` entries (float32 / uint32).
   * Position x^{n+1} [c/omega_ref], unit direction of the emitting particle's
   * mean velocity (collinear approximation), energy x hbar omega_c [m c^2],
   * weight = multiplicity * macro weight, emitting particle id and step. */
  float *x, *y, *z, *nx, *ny, *nz, *eps, *weight;
  uint32_t *pid, *step;
} prad_photons;

typedef struct prad_stats {
  int64_t records;      /* photon records written since init               */
  int64_t dropped;      /* records lost to a full buffer since init        */
  int64_t dn_gt1;       /* trials with dN > 1 (multiplicity > 1 possible)  */
  int64_t clamped;      /* steps where dp_perp/p was limited to 1          */
  int64_t chi_gt1;      /* steps with chi > 1 (outside classical validity) */
  int64_t mlp_fallback; /* learned-sampler draws that fell back to table   */
  int64_t nan_frozen;   /* particle-launches skipped as non-finite         */
  int32_t status;       /* sticky device status word (0 = ok): bit 1 an id
                         * outside the ledger; bit 2 a bounded tensor-core
                         * wait of the learned sampler ran out (the block
                         * stopped; its remaining records keep energy 0)   */
  int32_t spec_launches; /* launches through run-time specialised kernels
                          * since init (saturates at INT32_MAX)            */
  int64_t wiggler_invalid; /* PRAD_DIAG_WIGGLER: steps outside the regime  */
} prad_stats;

typedef struct prad_ctx prad_ctx;

/* Create a context on the current CUDA device: allocates the photon buffer
 * (10 x 4 B x photon_capacity), the per-particle FP64 ledger
 * (2 x 8 B x max_particles), the sampling tables, counters and reduction
 * scratch.  *out receives the handle (NULL on error).  Follows the problem
 * statement of the Numerical implementation section (emission per particle
 * and step, photons as particles).  Errors: PRAD_ERR_ARG for a null pointer,
 * a non-positive dt/omega_ref/capacity/max_particles or a bad enum;
 * PRAD_ERR_CUDA if an allocation fails. */
int prad_init(prad_ctx** out, const prad_config* cfg);

/* Free everything the context allocated.  Safe on NULL. */
int prad_destroy(prad_ctx* ctx);

/* Message of the last failing call on ctx ("" if none).  With ctx == NULL,
 * the message of the last failed prad_init of this thread. */
const char* prad_last_error(const prad_ctx* ctx);

/* Set the field model (the E, B that enter the Lorentz force and H_eff).
 * Copies everything except the YEE2D planes, which are borrowed.
 * Errors: PRAD_ERR_ARG (null, bad kind, bad sizes, misaligned planes). */
int prad_set_fields(prad_ctx* ctx, const prad_fields* f);

/* Advance n particles by nsteps steps in place, emitting photons.  Per
 * particle and step, in order:
 *   1. gather E, B at x^n, t^n;
 *   2. Boris push u^{n-1/2} -> u^{n+1/2} (Numerical implementation section);
 *   3. u_avg = (u^{n-1/2} + u^{n+1/2})/2 gives gamma and beta;
 *   4. H_eff by the configured form, limited by Omega dt <= gamma
 *      (dp_perp/p <= 1);
 *   5. omega_c = (3/2) Omega gamma^2 (Eq. (1)), chi = (2/3) hbar omega_c /
 *      (gamma m c^2);
 *   6. LL ledger += w (2/3) alpha hbar Omega^2 gamma^2 beta^2 dt (Eq. (4));
 *      rr_mode APPLY also scales u by 1/(1 + K gamma dt),
 *      K = (2/3) alpha hbar Omega^2 / (m c^2);
 *   7. x^{n+1} = x^n + dt u^{n+1/2}/gamma^{n+1/2};
 *   8. x = P^-1(R') from the proposal of Eqs. (11)-(12);
 *      dN = (sqrt3/2pi) alpha Omega dt F(x)/(x S(x)) (Eq. (13) per unit x);
 *      k = floor(dN) + [R < frac(dN)];
 *   9. if k > 0 and w > 0: append one record (weight k w, energy
 *      x hbar omega_c) and add k w x hbar omega_c to the emit ledger.
 * Records beyond the capacity are counted as dropped, never written.
 * For YEE2D with sort_interval > 0 and a pid array, the particles are
 * reordered by tile (prad_sort_by_tile) before every sort_interval steps.
 * Errors: PRAD_ERR_ARG (null pointers, n < 0, nsteps < 0, ledger range
 * outside max_particles, misaligned arrays), PRAD_ERR_STATE (no fields),
 * PRAD_ERR_CUDA (launch failure).  n == 0 or nsteps == 0 is a no-op. */
int prad_push_emit(prad_ctx* ctx, const prad_particles* p, int64_t n,
                   int32_t nsteps);

/* ---- batched ensembles ---------------------------------------------------- */
typedef struct prad_ensemble {
  prad_particles p;  /* arrays, ids, ledger offset and t0 of this ensemble */
  int64_t n;         /* particles (>= 0)                                   */
  prad_fields field; /* CONST or PLANE_WAVE (the batch kernel has no Yee)  */
  uint32_t ensemble; /* Philox counter word 3 for this ensemble            */
  uint32_t pad0;
} prad_ensemble;

/* Advance n_ens independent ensembles of uneven size by nsteps steps in ONE
 * persistent kernel per steps_per_launch chunk: a grid of SMs x blocks_per_sm
 * blocks takes work items (batch_chunk particles of one ensemble) from an
 * atomic counter until none are left, so large and small ensembles share
 * the GPU without a launch per ensemble.  Each ensemble has its own field
 * and Philox word 3; dt, omega_ref, seed, sampler (table or learned; FP32
 * only) and rr_mode are the context's.  With a learned sampler a block
 * evaluates its queued emissions before it moves to another ensemble.  With
 * use_graph the launches of a call are captured in a CUDA graph and
 * replayed by later calls of the same shape (same n_ens, sizes, nsteps,
 * sampler and launch parameters); ensemble contents (arrays, t0, fields)
 * may change between calls.  No kernel waits on another: nothing can spin.
 * Results per ensemble equal those of prad_push_emit with the same field
 * and ensemble word (state, counters and photon records bit for bit; the
 * emitted-energy ledger of a learned sampler up to the order of its FP64
 * atomic adds).  Errors: PRAD_ERR_ARG (bad ensemble, ledger range, Yee
 * field, n_ens < 1, FP64 context), PRAD_ERR_CUDA. */
int prad_push_emit_batch(prad_ctx* ctx, const prad_ensemble* ens, int32_t n_ens,
                         int32_t nsteps);

typedef struct prad_tuning {
  int32_t block_size, blocks_per_sm, batch_chunk, steps_per_launch;
  double particle_steps_per_s; /* throughput of the chosen configuration  */
  int32_t candidates;          /* configurations timed                   */
  int32_t pad0;
} prad_tuning;

/* Autotune the batch launch for this ensemble set: time candidate
 * (block_size, blocks_per_sm, batch_chunk, steps_per_launch) on scratch
 * copies of up to `sample` particles per ensemble for probe_steps steps
 * (CUDA events, after a warm-up), keep the fastest, store it in the
 * context's configuration (used by later batch calls) and in *out.  The
 * caller's particles, ledgers and photon records are left unchanged.
 * A later call with the same ensemble sizes and GPU returns the cached
 * result without timing.  Errors as for prad_push_emit_batch. */
int prad_autotune_batch(prad_ctx* ctx, const prad_ensemble* ens, int32_t n_ens,
                        int32_t probe_steps, int64_t sample, prad_tuning* out);

/* Reorder n particles in place (x, y, z, ux, uy, uz, w and the pid array,
 * which is required) by the 32 x 32-cell tile of the YEE2D grid that holds
 * them and, inside each tile, by cell (row-major in the tile), so that
 * neighbouring threads read the same staged field values (counting sorts:
 * histogram, scan, scatter, then a per-tile histogram of cells; the order
 * within a cell is not deterministic), and record the tile ranges that
 * push_emit uses to gather from shared-memory field tiles.  push_emit calls it itself every
 * sort_interval steps when sort_interval > 0.  Uses the context's scratch
 * (max_particles x 32 B).  Errors: PRAD_ERR_STATE (fields not YEE2D),
 * PRAD_ERR_ARG (null arrays, no pid array, n > max_particles). */
int prad_sort_by_tile(prad_ctx* ctx, const prad_particles* p, int64_t n);

/* Load balance of the last prad_push_emit_batch call (a measurement of the
 * batched form; the paper defines no such quantity): each CTA of its
 * persistent launches accumulates the SM clocks from its start to its exit
 * (summed over the call's launches); *efficiency (host) = mean / max over
 * the CTAs, 1 when every CTA was busy as long as the slowest.  *ctas (host,
 * may be NULL) receives the CTA count.  PRAD_ERR_ARG for a null context or
 * efficiency pointer, PRAD_ERR_STATE before the first batched call,
 * PRAD_ERR_CUDA if the copy fails.  Synchronises. */
int prad_batch_balance(prad_ctx* ctx, double* efficiency, int32_t* ctas);

/* Copy up to `cap` photon records into `out` (device arrays if
 * out_on_device, else host arrays; any pointer of out may be NULL to skip
 * that field), in slot order (nondeterministic across runs: records carry
 * pid and step).  *n_out receives the number of records held, *n_dropped
 * the records lost since the last drain.  With drain != 0 the buffer is
 * emptied afterwards.  cap may be 0 with out == NULL to query or drain only.
 * Synchronises the context stream. */
int prad_get_photons(prad_ctx* ctx, prad_photons* out, int64_t cap,
                     int64_t* n_out, int64_t* n_dropped, int32_t drain,
                     int32_t out_on_device);

/* Totals of the per-particle ledgers over all max_particles entries, by a
 * deterministic two-pass Kahan-compensated FP64 reduction on the device:
 * *emitted = sum of k w x hbar omega_c, *rr_loss = sum of the LL loss, both
 * in m c^2 (multiply by m_e c^2 for joules).  Either output may be NULL.
 * s (may be NULL) receives the counters.  Synchronises the stream. */
int prad_energy_budget(prad_ctx* ctx, double* emitted, double* rr_loss,
                       prad_stats* s);

/* Copy ledger entries [offset, offset + n) into emit/ll (device arrays if
 * out_on_device, else host); either may be NULL.  Synchronises. */
int prad_get_ledger(prad_ctx* ctx, double* emit, double* ll, int64_t offset,
                    int64_t n, int32_t out_on_device);

/* Zero the ledgers, counters and photon buffer. */
int prad_reset(prad_ctx* ctx);

/* ---- learned sampler (PRAD_SAMPLER_MLP, PRAD_SAMPLER_MLP_FALLBACK) --------
 * A 3 -> 64 -> 64 -> 1 MLP (SiLU, activations rounded to IEEE half, BF16
 * weights, FP32 accumulate) plus a fixed prior ln(-ln(1 - r)) + 2 (1 - r) ln r
 * maps
 * (r, gamma, omega_c dt) to ln x with G(x) = r, G the photon-number CDF of
 * the spectrum of Eqs. (7)-(8), int_0^x F(t)/t dt / (5 pi / 3).  With an MLP
 * sampler, push_emit uses the direct scheme: the photons of a step have mean
 * (5 sqrt3 / 6) alpha Omega dt (the integral over x of the rate of Eq. (13)),
 * multiplicity k = floor + [R < frac], and x = exp(MLP(r', gamma, omega_c dt))
 * for a uniform r' (records carry weight k w, as in the table path).  Uniforms
 * outside the trained range [1e-7, 1 - 1e-7], and with MLP_FALLBACK also
 * non-finite or out-of-range outputs, take x from a tabulated G^-1 instead
 * (counted in prad_stats.mlp_fallback).  FP32 precision only.  Parameters:
 * 4481 floats, W1[64][3], b1[64], W2[64][64] (row = output unit), b2[64],
 * W3[64], b3.  A new context starts from a fixed Glorot initialisation. */
#define PRAD_MLP_NUM_PARAMS 4481

/* Host FP32 parameter vector in/out (n must be PRAD_MLP_NUM_PARAMS).
 * set_weights also resets the optimiser state. */
int prad_mlp_set_weights(prad_ctx* ctx, const float* params, int64_t n);
int prad_mlp_get_weights(prad_ctx* ctx, float* params, int64_t n);

/* Train the context's network on the GPU: `steps` Adam steps (lr with a
 * cosine decay to 0) on minibatches of `batch` samples generated on the
 * device (r uniform in the trained range, gamma log-uniform in [10, 1e4],
 * H_eff log-uniform in [1e2, 1e6] T, omega_c dt from the context's dt;
 * target ln G^-1(r) from the device table), loss = mean over samples of
 * w (o - (ln x - prior(r)))^2 with o the network output, the fixed prior
 * ln(-ln(1 - r)) + 2 (1 - r) ln r and the energy weight w = (1 + x)/1.308.
 * *final_loss (host, may be NULL) receives the last minibatch loss.
 * Synchronises. */
int prad_mlp_train(prad_ctx* ctx, int64_t steps, int32_t batch, float lr, uint64_t seed,
                   float* final_loss);

/* Gradient of the mean loss over n explicit samples (device float4 each:
 * r, gamma, omega_c dt, target ln x) with respect to the parameter vector,
 * by the training kernels; grad (host, PRAD_MLP_NUM_PARAMS floats) and loss
 * (host) receive the results.  Synchronises. */
int prad_mlp_grad(prad_ctx* ctx, const float* samples, int64_t n, float* grad,
                  double* loss);

/* ln x = MLP(r, gamma, omega_c dt) for n device triples `in` (3 floats each)
 * into device `lnx`, with the tile evaluator of the learned sampler's
 * finishing kernel.  Synchronises.  PRAD_ERR_TIMEOUT if a bounded
 * tensor-core wait ran out (status bit 2 is then set). */
int prad_mlp_eval(prad_ctx* ctx, const float* in, float* lnx, int64_t n);

/* Self-test of the bounded tensor-core waits: runs the evaluator on one
 * 128-row tile with every MMA completion withheld, so each wait on the
 * tensor cores runs out (about 2 s of SM clocks in all); the kernel then
 * releases its tensor memory and reports through a status word of its own
 * (the context's status is untouched).  Returns PRAD_ERR_TIMEOUT when the
 * timeout was reported, as it should be (PRAD_ERR_STATE if it was not,
 * PRAD_ERR_CUDA on a runtime error); the context stays usable.
 * Synchronises. */
int prad_mlp_wait_selftest(prad_ctx* ctx);

/* ln G^-1(r) from the device table for n device uniforms. */
int prad_ginv_eval(prad_ctx* ctx, const float* r, float* lnx, int64_t n);

/* Angular spread (Eqs. (5)-(6), PRAD_DIAG_ANGLE_SPREAD): psi = gamma theta
 * as the step kernels draw it, for n photons of device x[i] (omega/omega_c,
 * float32) and device Philox words words[2i] (the uniform
 * (w + 1/2) 2^-32 of psi's one-sided CDF) and words[2i + 1] (bit 31: the
 * sign), into device psi[i].  Asynchronous on the context's stream.
 * PRAD_ERR_STATE if the context was created without
 * PRAD_DIAG_ANGLE_SPREAD; PRAD_ERR_ARG for a NULL array with n > 0 or
 * n < 0. */
int prad_angle_eval(prad_ctx* ctx, const float* x, const uint32_t* words, float* psi,
                    int64_t n);

/* The angular spread's table as the library builds it for
 * PRAD_DIAG_ANGLE_SPREAD contexts, written to host out (row-major,
 * PRAD_ANG_NL x PRAD_ANG_NV floats; geometry above).  Host only: needs no
 * device and no context (built once per process, ~0.3 s on first use).
 * PRAD_ERR_ARG if out is NULL or n < PRAD_ANG_NL * PRAD_ANG_NV. */
int prad_angle_table(float* out, int64_t n);

/* ---- angular distribution (Fig. 4) -------------------------------------------
 * Histogram of the emitted energy (record energy x weight) of the photon
 * records currently held, by direction: polar angle theta from `axis`, bins
 * uniform over [0, theta_max] (theta_max = pi/2: the front hemisphere), and
 * azimuth phi around the axis measured from the component of `ref`
 * perpendicular to it (phi = pi/2 along axis x ref), bins uniform over
 * [0, 2 pi).  Records with theta > theta_max are not counted.  out (host,
 * ntheta x nphi doubles, row-major [theta][phi]) receives energies in
 * m c^2.  Angles are computed in FP64 from the float records; bin sums use
 * FP64 atomics (order-dependent in the last bits).  Errors: PRAD_ERR_ARG
 * (null pointers, ntheta or nphi < 1, ntheta x nphi > 8192, theta_max
 * outside (0, pi], zero axis, ref parallel to axis), PRAD_ERR_CUDA.
 * Synchronises. */
int prad_angular_histogram(prad_ctx* ctx, const double axis[3], const double ref[3],
                           int32_t ntheta, int32_t nphi, double theta_max, double* out);

/* ---- totals without allocation ---------------------------------------------
 * The paper has no counterpart to this call; it serves callers that cannot
 * allocate device memory where they need the totals: a host code that owns
 * a fixed device memory pool, or a time loop in which a cudaMalloc (which
 * synchronises the device and may fail once the pool holds the memory) is
 * not acceptable.  It needs no context.
 *
 * The same deterministic two-pass Kahan totals as prad_energy_budget, of
 * two caller-owned device FP64 arrays emit[n] and rr[n] (for example the
 * caller's own per-particle ledgers), written to out[0] (sum of emit) and
 * out[1] (sum of rr), a caller-owned device array of 2 doubles, on `stream`
 * (cudaStream_t; NULL = default stream); asynchronous.  The per-block
 * partials live in a file-scope device array of 4096 x 4 doubles (128 KB,
 * held by every GPU that loads the library until the process exits), so
 * n is limited to 4096 x 65536 = 268435456 entries; larger n returns
 * PRAD_ERR_ARG.  No cudaMalloc, cudaFree or allocating library routine is
 * called.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the array and it keeps the
 * last call's contents (each call writes every partial it reads), so calls
 * that overlap on the GPU race: order them on one stream or synchronise.
 * n == 0 writes zeros (emit and rr may then be NULL).  The device address
 * looked up by the first call stays in use for the life of the process:
 * calls after a cudaDeviceReset of that device are not supported.
 * Errors: PRAD_ERR_ARG (null pointer, n < 0, n too large), PRAD_ERR_CUDA;
 * prad_ledger_totals_noalloc_error() returns the message of this thread's
 * last call if it failed, and an empty string after a call that succeeded. */
int prad_ledger_totals_noalloc(const double* emit, const double* rr, int64_t n, double* out,
                               void* stream);
const char* prad_ledger_totals_noalloc_error(void);

/* ---- diagnostics (same device functions as the hot kernel) --------------- */

/* Philox4x32-10 on n device counters (uint32 x 4 each) with key (k0, k1),
 * writing n x 4 words to device `out`. */
int prad_philox(prad_ctx* ctx, const uint32_t* ctr, uint32_t k0, uint32_t k1,
                uint32_t* out, int64_t n);

/* Run the sampler of step 8 on n Philox blocks (device uint32 x 4 each):
 * x_out[i] = P^-1(R') and g_out[i] = F(x)/S(x) from the device table, in the
 * context precision's type (float or double device arrays). */
int prad_eval_sampler(prad_ctx* ctx, const uint32_t* words, void* x_out,
                      void* g_out, int64_t n);

#ifdef __cplusplus
}
#endif
#endif /* PRAD_H */
