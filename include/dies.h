/*
 * dies.h -- C ABI of the GB300 immediate re-emission (IRE) dust radiative
 * transfer library (Juvela 2024, "DIES: Parallel dust radiative transfer
 * program with the immediate re-emission method").
 *
 * Problem statement (Sect. 2.1): a spherically symmetric cloud of concentric
 * shells, each with one density; dust absorption and scattering coefficients
 * and a Henyey-Greenstein asymmetry parameter per frequency; an isotropic
 * external radiation field and/or a central point source.  The luminosity of
 * each source is split over N photon packages of equal energy.  Packages are
 * followed shell by shell with independent free paths for absorption and
 * scattering (Eqs. 1 and 4); each absorption adds the package energy to its
 * shell, updates the shell temperature at once and re-emits the same energy
 * isotropically at a frequency drawn from the difference between the shell's
 * emission spectra at the new and old temperatures.  Optional weighting
 * (Sect. 2.2): background directions mu = u^k_bg (Eq. 5), directions of
 * re-emission and scattering (Eqs. 6-7), free paths (Eq. 8) and a forced
 * first interaction on the extinction or the absorption depth (Eqs. 9-12).
 *
 * Conventions shared by every call:
 *   - All array arguments are HOST pointers unless a name says otherwise.
 *     Inputs are copied during the call; the caller keeps ownership.
 *     Outputs are written to caller-allocated host arrays of the stated size.
 *   - Every call returns a dies_status (0 = success).  On failure the call
 *     has no effect on the handle, and dies_last_error() returns a
 *     thread-local, human-readable description.
 *   - Calls on one handle are not thread-safe; distinct handles are
 *     independent.  Setters after a run mark the derived tables stale; the
 *     next run rebuilds them on the device.
 *   - Units: radii in "length units" (length_unit_cm centimetres each);
 *     kappa * density is an opacity per length unit; frequencies in Hz;
 *     intensities in erg s^-1 cm^-2 Hz^-1 sr^-1; luminosities in erg s^-1.
 *   - Device work is enqueued on the handle's CUDA stream (default: the
 *     legacy default stream).  dies_run and dies_run_frozen return after the
 *     stream has completed; dies_run_async only enqueues.
 */
#ifndef DIES_H
#define DIES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DIES_MAX_FREQ 64      /* frequency bins per package (6-bit index) */
#define DIES_MAX_SHELLS 65536 /* shells per model */
#define DIES_MAX_TNODES 4096  /* temperature-table nodes */

typedef enum {
  DIES_OK = 0,
  DIES_EINVAL = -1,   /* invalid argument (sizes, ordering, NaN, range) */
  DIES_ENOMEM = -2,   /* host or device allocation failed, or workspace too small */
  DIES_ECUDA = -3,    /* a CUDA runtime call failed (no device, launch error, ...) */
  DIES_ESTATE = -4,   /* call not valid in the handle's state (e.g. run before dust) */
  DIES_ETIMEOUT = -5, /* the transport kernel hit its wall-clock budget and stopped */
  DIES_ERANGE = -6    /* a result left its representable range: an absorbed-energy counter of
                         the all-FP32 form passed ~1e38 (use DIES_PREC_MIXED for such sources) */
} dies_status;

/* Precision forms of the transport (Sect. 2.3 discusses FP32 only). */
enum {
  DIES_PREC_MIXED = 0, /* FP32 stepping and sampling; FP64 crossing distances in the
                          innermost shells, FP64 absorbed-energy accumulators and
                          temperature lookup (default) */
  DIES_PREC_FP32 = 1,  /* everything FP32; absorbed energies in two FP32 counters per
                          shell (all previous batches + current batch) over n_batches
                          sequential batches (Sect. 2.3) */
  DIES_PREC_FP64 = 2   /* FP64 geometry, sampling and accumulation */
};

/* flags of dies_run_frozen */
enum {
  DIES_FROZEN_REEMIT = 0,          /* absorption re-emits from the full cell spectrum */
  DIES_FROZEN_ABSORB_TERMINAL = 1, /* absorption ends the package (pure-absorber tests) */
  DIES_FROZEN_FORM = 2             /* with DIES_FROZEN_ABSORB_TERMINAL only: run the pass in the
                                      handle's precision form (dies_set_precision: the MIXED or
                                      FP32 stepping, FP64 inner crossings, forced first
                                      interaction) instead of the FP64 form; no per-package
                                      records */
};

typedef struct dies_model dies_model; /* opaque; owned by the library until destroyed */
typedef struct dies_batch dies_batch; /* opaque; many models in one launch */

/* Counters of the last run (all packages of all sources and models). */
typedef struct {
  uint64_t injected;      /* packages started */
  uint64_t escaped;       /* packages that left through the outer surface */
  uint64_t absorbed;      /* absorption (+ re-emission) events */
  uint64_t scattered;     /* scattering events */
  uint64_t crossed;       /* shell-boundary crossings, including the final exit */
  uint64_t killed_weight; /* packages ended by the weight floor (Sect. 2.2.1) */
  uint64_t killed_cap;    /* packages ended by the per-package event cap */
  uint64_t clamp_hi;      /* absorptions whose energy exceeded the table top */
  uint64_t forced;        /* packages given a forced first interaction */
  double E_injected;      /* erg/s carried by injected packages (with weights) */
  double E_escaped;       /* erg/s leaving the model (SED total) */
  double E_lost;          /* erg/s of packages ended by the floor or the cap */
  double E_direct;        /* erg/s tallied as the direct-escape part of forced packages */
  double table_ms;        /* device time of the table build of this run (0 if cached) */
  double kernel_ms;       /* device time from the accumulator reset to the end of the temperature kernel */
  double transport_ms;    /* device time of the transport launch(es) alone */
  uint32_t status_word;   /* device-side error flags: 0 = none, 1 = time budget reached, 8 = flight
                             watchdog tripped, 16 = a package left unfinished, 32 = FP32
                             counter out of range (DIES_ERANGE) */
  uint32_t launches;      /* kernels launched by this run */
  uint32_t diag[16];      /* diag[0] = 1: state of the first package ended by the flight
                             watchdog (state, cell, freq, n, s, p^2, tauA, tauS (FP32
                             forms: column travelled, column limit), kA, kS, w as
                             float bits, package, model) */
  double upload_ms;       /* device time of the input uploads that open the table build
                             (part of table_ms; 0 if cached).  Together with table_ms and
                             kernel_ms: the split of a run into upload, table build and
                             transport + temperatures that Sect. 3.1 reports as total vs
                             kernel time */
  uint32_t grid;          /* transport launch of the run: CTAs (0 after dies_run_frozen_static) */
  uint32_t block;         /* threads per CTA */
  uint32_t variant;       /* DIES_VARIANT_* bits of the transport kernel that ran */
} dies_stats;

/* dies_stats.variant: compile-time variants of the transport kernel, chosen
 * per run from the options and the launch (results do not depend on them
 * beyond FP32 rounding order). */
#define DIES_VARIANT_PLAIN_WEIGHTING 1u  /* FP32 forms: every weighting option but k_bg neutral,
                                            the weighting code not compiled in */
#define DIES_VARIANT_STAGED_GEOMETRY 2u  /* one model: geometry records copied to shared memory
                                            per CTA (dies_launch.stage_geometry) */
#define DIES_VARIANT_PACKAGE_POOL 4u     /* two packages per thread (launch knob) */
#define DIES_VARIANT_FP64_CROSSINGS 8u   /* mixed form: FP64 crossing distances in inner shells */

/* ------------------------------------------------------------ one model */

/* Create a model of n_shells shells from n_radii = n_shells + 1 strictly
 * increasing radii (radii[0] >= 0; r < radii[0] is a transparent void) and
 * n_shells densities (>= 0, finite) -- Sect. 2.1, one density per shell.
 * length_unit_cm > 0 converts radii to cm.  Host-only: no CUDA call is made.
 * Returns DIES_EINVAL on bad sizes or values, DIES_ENOMEM on host OOM. */
int dies_create_model(const double *radii, int n_radii, const double *densities, int n_shells,
                      double length_unit_cm, dies_model **out);

/* Dust per frequency (Sect. 2.1, Eq. 4 coefficients; HG phase function of
 * Sect. 2.2.1): n_freq in [2, DIES_MAX_FREQ] strictly increasing frequencies,
 * kappa_abs, kappa_sca >= 0 and g in (-1, 1).  Spectral integrals use bin
 * widths dnu_k = nu_k * (ln-nu width of bin k), the ln-nu width being half
 * the distance to the two neighbours (the full distance at the two ends). */
int dies_set_dust(dies_model *m, const double *freq_hz, int n_freq, const double *kappa_abs,
                  const double *kappa_sca, const double *g);

/* Radiation sources (Sect. 2.1): J_ext[n_freq] isotropic external intensity
 * (NULL = none) and/or a central point source of luminosity L_point > 0 with
 * spectral shape point_spectrum[n_freq] (any scale; NULL only if L_point == 0).
 * At least one source is required.  Call after dies_set_dust. */
int dies_set_sources(dies_model *m, const double *J_ext, double L_point, const double *point_spectrum);

/* Forced first interaction modes (Sect. 2.2.2). */
enum {
  DIES_FFI_OFF = 0,
  /* one interaction forced on the first flight with weight 1 - exp(-tau0),
   * tau0 the extinction optical depth of the whole ray (Eqs. 9-12); the
   * direct-escape part exp(-tau0) is tallied in the escaping SED */
  DIES_FFI_EXTINCTION = 1,
  /* the variant on the absorption optical depth only: a package whose plain
   * scattering free path outlasts the whole first ray is absorbed inside it
   * with weight 1 - exp(-tau_A0) (exp(-tau_A0) tallied as a direct escape);
   * any other package makes an unforced first flight (unbiased with
   * scattering) */
  DIES_FFI_ABSORPTION = 2
};

/* Weighting (Sect. 2.2): background directions mu = u^k_bg with package
 * weight 2 k_bg mu^(2 - 1/k_bg) (Eq. 5), k_bg in (0, 1], 0.5 = unweighted;
 * forced_first_interaction one of DIES_FFI_* (DIES_EINVAL otherwise). */
int dies_set_weighting(dies_model *m, double k_bg, int forced_first_interaction);

/* All weighting options of Sect. 2.2 (Table 1).  Directional weighting of
 * re-emission (Eq. 6) and scattering (Eq. 7) draws the new direction from a
 * Henyey-Greenstein function about the reference direction (towards the
 * centre for packages of the external field, away from it for the point
 * source) and multiplies the package weight by the ratio of the true to the
 * sampling density; free-path weighting (Eq. 8) draws tau from k e^(-k tau)
 * with weight e^(tau (k - 1)) / k.  With these options a package's weight
 * changes along its path, so energy is conserved in expectation only (the
 * injected energy counts the source's share before any free-path weight). */
typedef struct {
  double k_bg;                   /* Eq. 5, (0, 1], 0.5 = unweighted */
  int forced_first_interaction;  /* DIES_FFI_*: Eqs. 9-12 on the extinction or the absorption depth */
  double g_E;                    /* Eq. 6, (-1, 1), 0 = isotropic re-emission (off) */
  int scatter_weighting;         /* Eq. 7 on (g_S = 0 is isotropic about the reference, not off) */
  double g_S;                    /* Eq. 7 parameter, (-1, 1) */
  double k_A, k_S;               /* Eq. 8 factors, > 0, 1 = off */
  int k_A_density;               /* 1: k_A per shell, linear in log density from
                                    k_A_low_density (lowest shell density; also the
                                    void and empty shells) to k_A_high_density (highest) */
  double k_A_low_density, k_A_high_density;
  int reemit_uniform_in_cell;    /* 1: re-emit from a point uniform over the absorbing
                                    shell's volume instead of the absorption point (the
                                    test variant discussed in Sect. 4; not a weighting) */
} dies_weighting;

/* Sets every weighting option at once (see dies_weighting).  Errors:
 * DIES_EINVAL for NULL or out-of-range fields. */
int dies_set_weighting_ex(dies_model *m, const dies_weighting *w);

/* Precision form (DIES_PREC_*) and, for DIES_PREC_FP32, the number of
 * sequential batches n_batches >= 1 (Sect. 2.3).  fp64_radius: in
 * DIES_PREC_MIXED, shells whose outer radius is below fp64_radius * R use
 * FP64 crossing distances (0 = none). */
int dies_set_precision(dies_model *m, int mode, int n_batches, double fp64_radius);

/* Temperature table: n_nodes in [16, DIES_MAX_TNODES] nodes T_j log-spaced
 * from T_min to T_max (defaults 2.7 K, 1500 K, 1024).  Temperatures below
 * T_min are reported as T_min; absorbed energies above the table top are
 * counted in dies_stats.clamp_hi and reported as T_max. */
int dies_set_tgrid(dies_model *m, double T_min, double T_max, int n_nodes);

/* CUDA stream for all device work of this handle (cudaStream_t as void*). */
int dies_set_stream(dies_model *m, void *cuda_stream);

/* Launch shape of the transport kernel: block_size a multiple of 32 in
 * [64, 256], blocks_per_sm >= 0 (0 = occupancy maximum, larger values are
 * clamped to it), rare_batch in [1, 32]: a warp runs its scatterings,
 * absorptions and package starts together once this many of its lanes wait
 * for one (or when no lane can move on); inner_moves in [1, 64]: boundary
 * crossings a lane may make between two such rare-event passes (taken in
 * blocks of 8, rounded up, the warp checking its parked lanes after each);
 * aggregate_atomics 0 or 1 (FP32 forms): lanes of a warp absorbing in the
 * same shell in the same pass add their energies with one atomic, each lane
 * taking as its E_old the returned value plus the energies of the lower
 * lanes (the order of a serial run; for absorption-heavy models with hot
 * inner shells; a kernel variant, not used by the two-packages-per-thread
 * kernels).  Defaults 256, 0, 16, 32, 0.  Results do not depend on
 * these values beyond FP32 rounding. */
int dies_set_launch(dies_model *m, int block_size, int blocks_per_sm, int rare_batch, int inner_moves,
                    int aggregate_atomics);

/* Re-emission table layouts of the FP32 forms (dies_launch.reemit_table). */
enum {
  DIES_TABLE_ALIAS = 0, /* one alias-table row per T interval: one probe and one compare */
  DIES_TABLE_CDF = 1    /* one FP32 CDF row per T interval: binary search of six probes */
};

/* The full launch configuration, all knobs of the autotuner (no counterpart
 * in the paper; Sect. 2.3 runs one work item per package).  The first five
 * fields are those of dies_set_launch, with the same ranges; then
 *   refill_divisor       in [0, 4096]: a warp takes about 1/refill_divisor of
 *                        its share of the launch per trip to the device work
 *                        counter (32 to 1024 packages, a multiple of 32, so 1
 *                        to 32 packages per lane); 0 = 64.  Relative to the
 *                        launch, so one value serves every package count;
 *   reemit_table         DIES_TABLE_ALIAS or DIES_TABLE_CDF: a kernel variant of
 *                        the mixed form's single-model runs without forced
 *                        first interaction; every other run uses alias rows
 *                        (the FP64 form searches FP64 CDF rows);
 *   packages_per_thread  1 (or 0) or 2: with 2 (FP32 forms without forced
 *                        first interaction; other runs ignore it) each lane
 *                        owns two slots of a per-warp pool of packages in
 *                        shared memory besides the package in its registers:
 *                        a stopped package waits there for its event while
 *                        the lane moves another, and events run in passes of
 *                        one kind.
 * Both sample the same discrete distributions (to within 2^-23 per bin);
 * results do not depend on the configuration beyond FP32 rounding. */
typedef struct dies_launch {
  int block_size;
  int blocks_per_sm;
  int rare_batch;
  int inner_moves;
  int aggregate_atomics;
  int refill_divisor;
  int reemit_table;
  int packages_per_thread;
  int stage_geometry;  /* 1: a single model (FP32 forms, no FP64 crossings, no package
                          pools) has its geometry records (16 bytes + a density per
                          shell and the void) copied to shared memory by every CTA
                          and read there at each crossing, wherever that costs no
                          resident CTA; 0: read through L1.  Default 1;
                          dies_set_launch leaves it as it is */
} dies_launch;
int dies_set_launch_ex(dies_model *m, const dies_launch *launch);

/* Package range of the next run on this handle: checkpoint and resume at a
 * package index (no counterpart in the paper; its N_B batches of Sect. 2.3
 * split a run the same way).  The next dies_run, dies_run_async or
 * dies_run_frozen call with n_packages = N runs only packages
 * [first, first + count) of each active source of that N-package run: the
 * same Philox streams and package energies L / N as the whole run.  With
 * resume = 1 it adds to the absorbed energies, escaping SED, counters and
 * energy sums the handle holds from its previous run instead of starting
 * from zero (DIES_ESTATE if there was none); temperatures are those of all
 * the packages so far.  Consecutive ranges covering [0, N) therefore compute
 * the whole run: in the frozen pass the same per-package event counts and
 * path hashes bit for bit (rows outside the range are left untouched); in IRE
 * runs the same estimator, with the deposits of a later range ordered after
 * those of earlier ones.  The setting applies to the next run only; a range
 * outside [0, N) fails that run with DIES_EINVAL.  Graph mode is bypassed for
 * a ranged run. */
int dies_set_package_range(dies_model *m, uint64_t first, uint64_t count, int resume);

/* Wall-clock budget of one transport launch in seconds (default 120).  A
 * launch that reaches it stops early and the run returns DIES_ETIMEOUT. */
int dies_set_time_budget(dies_model *m, double seconds);

/* Graph mode (no counterpart in the paper; launch-overhead removal for
 * repeated runs such as seed ensembles): enable = 1 makes each run replay
 * one CUDA graph of the per-run device work (accumulator reset, transport,
 * tallies, temperatures), captured on the first run of a configuration and
 * captured again when the package count, precision, launch shape, tables'
 * sizes or workspace change.  The seed reaches the kernels through a pinned
 * host word that the graph copies first, so in graph mode dies_run_async
 * waits for the handle's previous run before enqueueing.  Results are the
 * same as without a graph.  enable must be 0 or 1 (default 0). */
int dies_set_graph(dies_model *m, int enable);

/* Device memory.  By default the library allocates its own device memory.
 * Alternatively the caller provides one device buffer of at least
 * dies_workspace_bytes() bytes (256-byte aligned, e.g. from a PyTorch
 * tensor); the caller then owns it and must keep it alive while the handle
 * uses it.  Call after the setters that fix sizes (create, dust, tgrid). */
int dies_workspace_bytes(const dies_model *m, size_t *bytes);
int dies_set_workspace(dies_model *m, void *device_ptr, size_t bytes);

/* Run n_packages packages per active source with Philox seed `seed` (full
 * IRE transport, Sect. 2.1).  Builds the emission and re-emission tables on
 * the device when stale, zeroes the accumulators, runs the transport kernel
 * and the temperature kernel, waits for the stream and reads the counters.
 * n_packages >= 1.  Errors: DIES_ESTATE (dust/sources missing), DIES_ECUDA,
 * DIES_ENOMEM, DIES_ETIMEOUT. */
int dies_run(dies_model *m, uint64_t n_packages, uint64_t seed);

/* As dies_run but only enqueues the work on the handle's stream; results
 * and counters become readable after the stream completes (the getters
 * synchronise it). */
int dies_run_async(dies_model *m, uint64_t n_packages, uint64_t seed);

/* Results of the last run (synchronise the stream first).  n must equal the
 * number of shells / frequencies.  Temperatures in K from the absorbed energy
 * per shell by log-log interpolation in the emission table; absorbed energy
 * per shell in erg/s; escaping SED in erg/s per frequency bin. */
int dies_get_temperatures(dies_model *m, double *T_out, int n_shells);
int dies_get_absorbed(dies_model *m, double *E_out, int n_shells);
int dies_get_escaping_sed(dies_model *m, double *L_out, int n_freq);
int dies_get_stats(dies_model *m, dies_stats *out);

/* Frozen-temperature transfer pass in FP64 (parity diagnostic): the shell
 * temperatures are fixed to T_frozen[n_shells] (> 0), an absorption only
 * tallies its energy and re-emits from the full shell spectrum
 * kappa_abs B(T_i) dnu (or ends the package with DIES_FROZEN_ABSORB_TERMINAL).
 * Uses the Philox stream layout of the FP64 form.  Optional per-package
 * outputs (NULL to skip), package j of active source s at row s*n + j:
 * n_events_out[rows*3] = (scatterings, absorptions, crossings) and
 * path_hash_out[rows] = 64-bit FNV-1a hash of the event sequence.
 * With flags = DIES_FROZEN_ABSORB_TERMINAL | DIES_FROZEN_FORM the pass runs
 * the handle's own precision form instead (the stepping, sampling and
 * forced-interaction code of dies_run, Sect. 2.1 and Eq. 4, with each
 * absorption ending its package): a pure absorber's per-shell absorbed
 * energy then has a closed form (impact-parameter quadrature for the
 * external field, radial for the point source) that pins the FP32 geometry.
 * Absorbed energies are tallied in FP64 in every form; T_frozen is unused
 * by the physics of this mode but still required; records must be NULL
 * (else DIES_EINVAL). */
int dies_run_frozen(dies_model *m, const double *T_frozen, uint64_t n_packages, uint64_t seed, int flags,
                    uint32_t *n_events_out, uint64_t *path_hash_out);

void dies_destroy_model(dies_model *m);

/* Frozen-temperature pass that allocates no device memory.  The paper has no
 * counterpart: this entry point serves callers that cannot call cudaMalloc
 * (plug-ins whose host application owns all device memory, code whose
 * memory budget is fixed up front, allocators that forbid side
 * allocations).  It computes the absorbed energies, the escaping SED, the
 * per-package event counts and the path hashes that dies_run_frozen
 * computes, but every input and output is a caller-owned DEVICE pointer and
 * the pass's scratch (per-shell re-emission CDFs, work counter, event
 * counters, status word, SED partials) lives in one fixed array inside the
 * library, DIES_STATIC_SCRATCH_BYTES bytes on every GPU that loads it, kept
 * until the process exits.  The handle's temperatures, absorbed energies and
 * SED (dies_get_temperatures / _absorbed / _escaping_sed) keep the values of
 * its last dies_run.  To learn whether the pass completed, call
 * dies_get_stats on the handle afterwards (it waits for the stream): it
 * returns DIES_ETIMEOUT when the kernel stopped at the handle's time budget
 * (dies_set_time_budget) and fills the counters and energies of the pass;
 * it reads them from the shared scratch, so call it before the next static
 * pass on any handle.
 *   T_frozen_dev  [n_shells] shell temperatures (> 0), device memory
 *   E_abs_dev     [n_shells] out: absorbed energy per shell (erg/s)
 *   sed_dev       [n_freq]   out: escaping luminosity per bin (erg/s)
 *   n_events_dev  [rows*3]   out or NULL, path_hash_dev [rows] out or NULL,
 *                 rows = n_packages * active sources (layout of dies_run_frozen)
 * Requirements: n_shells <= DIES_STATIC_MAX_SHELLS (else DIES_EINVAL); the
 * handle must already hold its device workspace and tables, i.e. one
 * dies_run / dies_run_async must have completed set-up on it (else
 * DIES_ESTATE).  The call only enqueues work on the handle's stream.  Its
 * first call on a device looks up the scratch array's device address; make
 * that first call before any stream capture.  All calls share the one
 * scratch array, so calls whose work overlaps on the GPU (other streams,
 * other threads) race and must be serialised by the caller. */
#define DIES_STATIC_MAX_SHELLS 4096
#define DIES_STATIC_SCRATCH_BYTES (DIES_STATIC_MAX_SHELLS * 64 * 8 + 4096)
int dies_run_frozen_static(dies_model *m, const double *T_frozen_dev, uint64_t n_packages, uint64_t seed, int flags,
                           double *E_abs_dev, double *sed_dev, uint32_t *n_events_dev, uint64_t *path_hash_dev);

/* ------------------------------------------------ batched parameter study */

/* n_models models in one persistent launch.  Model i has shells
 * [shell_offsets[i], shell_offsets[i+1]) of the concatenated densities array
 * and radii rows radii[shell_offsets[i] + i ... shell_offsets[i+1] + i]
 * (n_i + 1 radii per model, concatenated).  source_kind[i] = 1 external
 * field, 2 point source, 3 both.  All models share one dust table, one
 * external field and one point-source spectrum/luminosity. */
int dies_create_batch(int n_models, const int *shell_offsets, const double *radii, const double *densities,
                      const int *source_kind, double length_unit_cm, dies_batch **out);
int dies_batch_set_dust(dies_batch *b, const double *freq_hz, int n_freq, const double *kappa_abs,
                        const double *kappa_sca, const double *g);
int dies_batch_set_sources(dies_batch *b, const double *J_ext, double L_point, const double *point_spectrum);
int dies_batch_set_stream(dies_batch *b, void *cuda_stream);
int dies_batch_set_launch(dies_batch *b, int block_size, int blocks_per_sm, int rare_batch, int inner_moves,
                          int aggregate_atomics);
int dies_batch_set_launch_ex(dies_batch *b, const dies_launch *launch);
/* Weighting for all models of the batch (as dies_set_weighting_ex; with
 * k_A_density the density range is each model's own). */
int dies_batch_set_weighting(dies_batch *b, const dies_weighting *w);
/* Precision form of the batch (as dies_set_precision; the N_B batches of the
 * FP32 form then split every model's packages). */
int dies_batch_set_precision(dies_batch *b, int mode, int n_batches, double fp64_radius);
/* Graph mode for the batch, as dies_set_graph. */
int dies_batch_set_graph(dies_batch *b, int enable);
int dies_run_batch(dies_batch *b, uint64_t n_packages_per_model, uint64_t seed);
int dies_run_batch_async(dies_batch *b, uint64_t n_packages_per_model, uint64_t seed);
/* Results: concatenated per-shell arrays (n_total = shell_offsets[n_models])
 * and per-model SEDs (n_models * n_freq, model-major). */
int dies_batch_get_temperatures(dies_batch *b, double *T_out, int n_total_shells);
int dies_batch_get_escaping_sed(dies_batch *b, double *L_out, int n_values);
int dies_batch_get_stats(dies_batch *b, dies_stats *out);
void dies_destroy_batch(dies_batch *b);

/* --------------------------------------------------------------- misc */

/* Thread-local description of the last failure of a call on this thread. */
const char *dies_last_error(void);

/* Number of kernels this library has launched in this process. */
uint64_t dies_launch_count(void);

/* Library version string. */
const char *dies_version(void);

/* ------------------------------------------------------- measurement */

/* Measured rates of the units that bound the transport (no counterpart in
 * the paper; the roofline denominators of its hot path): whole-GPU
 * operations per second of FP32 fused multiply-add, 32-bit integer
 * multiply-add, MUFU base-2 logarithm and FP64 fused multiply-add (each from
 * 8 independent chains per thread, 8 CTAs of 256 threads per SM), and of the
 * L2 FP64 atomic add with return that each absorption performs (Sect. 2.1),
 * to 2^20 distinct addresses, to 64 addresses and to one address. */
typedef struct {
  double fp32_fma_per_s;
  double int_mad_per_s;
  double mufu_per_s;
  double fp64_fma_per_s;
  double atomic_f64_ret_distinct_per_s;
  double atomic_f64_ret_64addr_per_s;
  double atomic_f64_ret_same_per_s;
  int sm_count;
} dies_peaks;

/* Runs the microbenchmarks on the current device (legacy default stream,
 * ~0.3 s, 8 MiB of device memory allocated and freed).  Errors:
 * DIES_EINVAL (out NULL), DIES_ENOMEM, DIES_ECUDA (no device, launch
 * failure). */
int dies_measure_peaks(dies_peaks *out);

#ifdef __cplusplus
}
#endif

#endif /* DIES_H */
