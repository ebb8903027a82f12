/*
 * flipmc.h -- C ABI of a GB300 (sm_103a) flip Monte Carlo library for the
 * triangular three-site molecular glass-former of arXiv 2506.21290
 * ("Molecular motion at the experimental glass transition", Sec. II).
 *
 * Model (Sec. II.A).  M molecules of three atoms; atom (site) i belongs to
 * molecule i/3.  Types 0=A, 1=B, 2=C with diameters sigma_A, sigma_B, sigma_C
 * (paper: 0.9, 1, 1.1).  Every pair, intra- and intermolecular, interacts by
 * the WCA potential of Eq. 1 with sigma_ab = (sigma_a + sigma_b)/2 and cutoff
 * 2^(1/6) sigma_ab; the three bonds of a molecule add the FENE potential of
 * Eq. 2, -K eps ln(1 - (r / (R0 sigma_ab))^2) (paper: K = 33.75, R0 = 1.5).
 * Cubic periodic box of side L.
 *
 * Chain (Sec. II.B).  Metropolis moves, N = 3M attempts per sweep (one MC time
 * step).  Move types: atom translation (uniform in [-d_atom, d_atom]^3), flip
 * (pick a molecule and one of its three median axes; swap the types of the two
 * other atoms), and two rigid-body moves the paper does not use (molecule
 * translation, molecule rotation about the centroid).  Sweeps follow a
 * checkerboard schedule: a random 32-bit shift of an n_c^3 cell grid per sweep,
 * 8 colours in order, every cell of a colour updated concurrently, a cell with
 * n atoms running n attempts; a move that would take an atom out of its cell,
 * or that writes an atom outside the active cell, is rejected.  Random numbers
 * are Philox4x32-10 keyed on (seed) and counted on (attempt, cell, sweep), so a
 * run is reproducible bit for bit and independent of the launch layout.
 *
 * Precision.  MC_PREC_FP64 evaluates every Delta E in FP64 with one rounding per
 * operation, summed in a fixed order (moved atom ascending, then partner index
 * ascending); it reproduces the library's FP64 reference trajectory exactly.
 * MC_PREC_FP32 evaluates pair terms in FP32 and decides in FP32 when
 * |dE32 - threshold| exceeds recheck_gap times the sum of term magnitudes plus
 * the threshold's own error bound (the FP32 decision then equals the FP64 one);
 * otherwise it recomputes Delta E and the threshold in the FP64 order above.
 * Total energies are FP64 in both modes; the running total is accumulated in
 * FP64 (in FP32 mode from per-cell FP32 sums of the accepted FP32 Delta E).
 *
 * Conventions.  All functions return 0 (MC_OK) or a negative MC_ERR_* code;
 * mc_last_error() returns a message for the calling thread's last error.
 * Pointers named host_* or without a prefix are host memory and are only read
 * or written during the call; inputs are copied, the caller keeps ownership.
 * Pointers named dev_* are device memory of the handle's GPU, owned by the
 * caller.  The library owns the device memory it allocates until
 * mc_destroy().  Arrays are site-major: xyz[3*i + axis], types[i], molecule
 * m = sites 3m, 3m+1, 3m+2.  Batched handles concatenate replicas in order.
 * Work is enqueued on the handle's stream (mc_set_stream); functions that
 * return data synchronise that stream.  A handle must not be used by two
 * threads at once.
 */
#ifndef FLIPMC_H
#define FLIPMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MC_OK 0
#define MC_ERR_INVALID_ARG (-1)   /* a size, pointer or parameter is out of range         */
#define MC_ERR_BAD_STATE (-2)     /* input state has a broken bond or a non-finite energy */
#define MC_ERR_CUDA (-3)          /* a CUDA runtime call failed                            */
#define MC_ERR_TIMEOUT (-4)       /* a bounded device wait gave up                         */
#define MC_ERR_CELL_OVERFLOW (-5) /* a cell neighbourhood exceeded the staging capacity    */
#define MC_ERR_NO_DEVICE (-6)     /* no usable CUDA device                                 */

#define MC_PREC_FP64 0
#define MC_PREC_FP32 1

#define MC_MOVE_ATOM 0
#define MC_MOVE_FLIP 1
#define MC_MOVE_MOL_TRANS 2
#define MC_MOVE_MOL_ROT 3

/* Status of one attempted move in the attempt log. */
#define MC_ST_EVALUATED 0   /* Delta E computed and Metropolis applied           */
#define MC_ST_LEFT_CELL 1   /* proposal took an atom out of the active cell      */
#define MC_ST_BOND_BREAK 2  /* a proposed bond length reached R0 sigma_ab        */
#define MC_ST_NOT_IN_CELL 3 /* an atom the move writes lies outside the cell     */

typedef struct mc_handle mc_handle;

/* Potential of Eq. 1-2: sigma[type], eps, FENE prefactor K (energy in units of
 * eps) and FENE range factor R0. */
typedef struct {
    double sigma[3];
    double eps;
    double fene_k;
    double fene_r0;
} mc_params;

/* Move mix: probabilities p[MC_MOVE_*] (non-negative, summing to 1 within
 * 1e-9), atom step half-width d_atom, molecule step half-width d_mol (length
 * units), and rot_a: the rotation quaternion is (1, rot_a v)/|.| with v
 * uniform in (-1,1)^3.  Paper mix: p = {0.8, 0.2, 0, 0}. */
typedef struct {
    double p[4];
    double d_atom;
    double d_mol;
    double rot_a;
} mc_move_mix;

/* Creation options.  precision: MC_PREC_FP64 or MC_PREC_FP32.  n_cells: cells
 * per axis (even, >= 2), 0 picks the largest even n_c whose cell side is at
 * least R0 * max bonded sigma_ab (the longest possible interaction).
 * recheck_gap: FP32 decision margin as a fraction of the summed term
 * magnitudes (0 picks 1e-5).  The FP32 Delta E differs from the FP64 one by at
 * most about 6.3e-6 of that sum (distances to 9 units of FP32 rounding, each
 * term's sensitivity to them, its own evaluation and the sums), so with the
 * default every decision taken in FP32 is the one FP64 takes; smaller values
 * trade that guarantee for fewer FP64 rechecks.  device: CUDA device
 * ordinal.  stencil_cap: atoms staged per cell neighbourhood (0 = automatic).
 * warps_per_cell: 1, 2, 4 or 8 warps per cell, each evaluating one of the cell's
 * consecutive attempts, committed in order (0 = chosen from the number of
 * cells); results do not depend on it.  launch_mode: 0 = one persistent
 * cooperative launch per mc_sweep call when the device supports it, else a
 * CUDA graph per sweep; 1 = graphs; 2 = persistent (INVALID_ARG if
 * unsupported).  recompute_every: k > 0 makes every k-th sweep of
 * mc_sweep / mc_sweep_batch / mc_corr_run (counted across calls) end with an
 * FP64 recompute of each replica's total energy on the device: the relative
 * drift |e_run - E| / |E| of the running total is recorded in mc_stats and
 * e_run restarts from E (0 = off; the chain itself is unchanged).
 * wait_limit_log2: 0 = the
 * default bounds of the device-side waits between blocks; 1..30 = every such
 * wait gives up after 2^k polls and reports MC_ERR_TIMEOUT (for tests of the
 * timeout path; a wait that gives up leaves the state undefined). */
typedef struct {
    int precision;
    int n_cells;
    int device;
    int stencil_cap;
    double recheck_gap;
    int warps_per_cell;
    int launch_mode;
    int recompute_every;
    int wait_limit_log2;
} mc_options;

/* Per-replica counters since creation (or mc_reset_stats). */
typedef struct {
    uint64_t attempts[4];
    uint64_t accepts[4];
    uint64_t rejected_geometry; /* MC_ST_LEFT_CELL + MC_ST_NOT_IN_CELL          */
    uint64_t rejected_bond;     /* MC_ST_BOND_BREAK                              */
    uint64_t pair_evals;        /* site-pair evaluations of the cell-list method: per
                                   evaluated attempt 2 (rigid moves: 6) times the atoms
                                   of the active cell's neighbourhood (old and new)   */
    uint64_t fp64_rechecks;     /* FP32 mode: decisions retaken in FP64          */
    uint64_t pair_interactions; /* pair-potential evaluations inside their range, old
                                   and new configuration counted apart: WCA terms with
                                   r < 2^(1/6) sigma_ab and FENE terms (FP32 mode: the
                                   FP32 pass; FP64 mode: the FP64 sum)              */
    uint64_t sweeps;
    double e_run;               /* running FP64 energy: initial + sum of accepted dE */
    uint64_t recomputes;        /* FP64 recomputes made by recompute_every           */
    double drift_last;          /* relative drift |e_run - E| / |E| at the last one  */
    double drift_max;           /* largest such drift                                */
} mc_stats;

/* Static facts of a handle. */
typedef struct {
    int n_rep;
    int precision;
    int stencil_cap;
    int total_sites;
    int total_cells;
    int max_cells_per_axis;
    double recheck_gap;
    int warps_per_cell;
    int active_cells_per_colour;
    int launch_mode;          /* 1: a CUDA graph per sweep; 2: one persistent launch per call */
    int persistent_blocks;    /* blocks of the persistent launch (0 with graphs) */
    int recompute_every;      /* as in mc_options */
    int binary_version;       /* compute capability the sweep kernels were built for (103 = sm_103) */
} mc_info;

/* One attempted move as recorded by mc_sweep_logged(). */
typedef struct {
    int32_t site;      /* site index within its replica                         */
    int16_t move;      /* MC_MOVE_*                                             */
    int16_t flags;     /* bit 0: FP32 decision retaken in FP64                  */
    int32_t status;    /* MC_ST_*                                               */
    int32_t accepted;  /* 1 if accepted                                         */
    double dE;         /* Delta E as the mode computed it (FP32 value in FP32)  */
    double dE64;       /* FP64 Delta E when computed (FP64 mode, or recheck)    */
    double scale;      /* sum of term magnitudes used for the FP32 margin       */
} mc_log_entry;

/*
 * Create a single-replica handle.  L: box side (> 0).  n_mol: molecules (>= 1).
 * xyz: 9*n_mol positions (any real; wrapped into [0,L) and quantised to 32-bit
 * fixed point, q = floor(frac(x/L) 2^32)).  types: 3*n_mol values in {0,1,2}.
 * params/opts: NULL picks the paper's potential and FP32 defaults.
 * Errors: INVALID_ARG (sizes, types, box smaller than two cells of side
 * R0*max sigma), BAD_STATE (a bond at or beyond R0 sigma_ab, or a non-finite
 * energy), NO_DEVICE, CUDA; of several invalid inputs the one met first in
 * replica, then site, then bond order is reported.  Host work: the packing and
 * validation of more than 8192 molecules runs on up to 16 host threads started
 * and joined inside the call; the handle keeps a page-locked staging buffer
 * (16 to 28 bytes per atom) for the state's copies.  Model: Sec. II.A; schedule as
 * described above.
 */
int mc_create(mc_handle **out, double L, int n_mol, const double *xyz, const int32_t *types,
              const mc_params *params, const mc_options *opts);

/*
 * Create a handle of n_rep independent replicas (the paper runs 10 to 100
 * independent samples per temperature, Sec. III.B) advanced together.
 * L[n_rep], n_mol[n_rep]; xyz and types concatenate the replicas in order.
 * Errors as mc_create.
 */
int mc_create_batch(mc_handle **out, int n_rep, const double *L, const int32_t *n_mol, const double *xyz,
                     const int32_t *types, const mc_params *params, const mc_options *opts);

/*
 * The cell grid mc_create picks for one replica (host only, no GPU): the
 * longest interaction range (the WCA cutoff 2^(1/6) sigma_ab of any type pair
 * and R0 sigma_ab of any pair bonded in some molecule) into *range_out
 * (nullable), and n_c: request if it is even, >= 2 and leaves cells at least
 * that wide, else the largest such even n_c (request = 0).  Errors:
 * INVALID_ARG (as mc_create: sizes, types, a box smaller than twice the
 * range, a request that makes cells too narrow).
 */
int mc_cell_grid(double L, int n_mol, const int32_t *types, const mc_params *params, int request, int *nc_out,
                 double *range_out);

/* Free all device memory and graphs of the handle.  NULL is ignored. */
void mc_destroy(mc_handle *h);

/* Enqueue subsequent work on this cudaStream_t (NULL: the handle's own stream). */
int mc_set_stream(mc_handle *h, void *stream);

/*
 * Run n_sweeps sweeps (each N = 3M attempts per replica, Sec. II.B) at
 * temperature T with the given move mix and 64-bit seed; the sweep counter
 * persists in the handle, so consecutive calls continue one chain.  For a
 * batched handle T and seed apply to every replica.  Asynchronous: returns
 * after enqueuing; device-side errors surface at the next synchronising call.
 * Errors: INVALID_ARG (T <= 0, bad mix, n_sweeps < 0), CUDA.
 */
int mc_sweep(mc_handle *h, int n_sweeps, double T, const mc_move_mix *mix, uint64_t seed);

/* Batched variant: T[n_rep] and seeds[n_rep] per replica. */
int mc_sweep_batch(mc_handle *h, int n_sweeps, const double *T, const mc_move_mix *mix, const uint64_t *seeds);

/*
 * As mc_sweep, recording every attempt in log_out (host, n_sweeps * total_sites
 * entries, layout [replica][sweep][slot], slot = cell start + attempt number).
 * Synchronous.  For tests and audits; slower than mc_sweep.
 */
int mc_sweep_logged(mc_handle *h, int n_sweeps, const double *T, const mc_move_mix *mix, const uint64_t *seeds,
                    mc_log_entry *log_out);

/* Wait for enqueued work; return the first device-side error, if any. */
int mc_sync(mc_handle *h);

/*
 * Total energy of each replica, recomputed from the state in FP64 over the
 * cell neighbourhoods (Eq. 1 + Eq. 2, every pair once): E_out[n_rep].
 * Synchronous.
 */
int mc_energy(mc_handle *h, double *E_out);

/*
 * Pressure of each replica from the virial (Sec. II.C quotes P = 30 at T = 1,
 * rho = 1.2): out[2r] = W, the sum over all pairs i < j of -r dphi/dr (the
 * derivative of Eq. 1 and, for the three bonds of a molecule, Eq. 2), FP64
 * over the cell neighbourhoods; out[2r+1] = N T[r] / V + W / (3 V) with N
 * the replica's atoms and V = L^3.  T: n_rep temperatures (host).
 * Synchronous.  Errors: INVALID_ARG (NULL, T <= 0), CUDA.
 */
int mc_pressure(mc_handle *h, const double *T, double *out);

/*
 * Static structure factor of the atoms (Sec. IV.A, Eq. sq):
 * out[r * n_q + k] = |sum_i exp(i q_k . x_i)|^2 / N per replica r and
 * wavevector qvec[3k..3k+2], over the N atoms of the replica at their wrapped
 * positions x in [0, L)^3, FP64.  This is the double sum of Eq. sq with the
 * i = j terms (each 1) included; the sum over i != j alone is out - 1.  Use
 * wavevectors of the reciprocal lattice, q = 2 pi n / L, for which the result
 * does not depend on the periodic image.  1 <= n_q <= 65535.  Synchronous.
 */
int mc_structure_factor(mc_handle *h, const double *qvec, int n_q, double *out);

/*
 * Pair-distance histogram of the atoms (Sec. IV.A, Eq. gr): counts[r * n_bins
 * + b] = the number of pairs i < j of replica r whose minimum-image distance
 * r_ij satisfies floor(r_ij / dr) = b, with r_ij from the int32 fixed-point
 * differences in FP64 (each product and sum rounded once, x then y then z,
 * then sqrt, then the division).  g (nullable, n_rep * n_bins doubles) gets
 * g(r) = 2 counts / (N rho V_shell) with rho = N / V and V_shell the volume of
 * the bin's spherical shell.  0 < dr, 1 <= n_bins <= 4096, n_bins dr <= L / 2
 * for every replica.  Synchronous.  Errors: INVALID_ARG, CUDA.
 */
int mc_pair_histogram(mc_handle *h, double dr, int n_bins, uint64_t *counts, double *g);

/*
 * As mc_energy, but only enqueued on the handle's stream: dev_E_out is a
 * device buffer of n_rep doubles owned by the caller (for example a torch
 * tensor).  No synchronisation; errors surface at the next mc_sync.
 */
int mc_energy_device(mc_handle *h, double *dev_E_out);

/*
 * Run n_sweeps sweeps without graphs, timing each stage with CUDA events on
 * the handle's stream: ms_out[0] = cell-list build, ms_out[1] = the 8 colour
 * phases, ms_out[2] = per-sweep finalisation, each the total over the sweeps
 * in milliseconds.  Same chain as mc_sweep_batch.  Synchronous.  For
 * measurements; mc_sweep is the production path.
 */
int mc_sweep_timed(mc_handle *h, int n_sweeps, const double *T, const mc_move_mix *mix, const uint64_t *seeds,
                   double *ms_out);

/*
 * Copy the state out: xyz_out[3*total_sites] (wrapped, x = q L / 2^32),
 * types_out[total_sites], stats_out[n_rep]; any pointer may be NULL.
 * Synchronous; more than 65536 atoms are converted on up to 16 host threads
 * started and joined inside the call.
 */
int mc_state(mc_handle *h, double *xyz_out, int32_t *types_out, mc_stats *stats_out);

/*
 * Exact state: q_out[3*total_sites] fixed-point positions, X_out[3*total_sites]
 * unwrapped fixed point (q + 2^32 * periodic images crossed), types_out.  Any
 * pointer may be NULL.  Synchronous.
 */
int mc_state_fixed(mc_handle *h, uint32_t *q_out, int64_t *X_out, int32_t *types_out);

/*
 * Replace the state from host arrays (same layout and quantisation as
 * mc_create).  Stats and the sweep counter are kept; e_run is reset to the new
 * total energy; image counters are cleared.  Errors as mc_create.
 */
int mc_set_state(mc_handle *h, const double *xyz, const int32_t *types);

/*
 * Exact restore (checkpoint resume): q[3*total_sites] fixed-point positions,
 * X[3*total_sites] unwrapped fixed point or NULL (image counters restored from
 * (X - q) / 2^32, else cleared), types[total_sites].  Same checks and
 * e_run reset as mc_set_state.
 */
int mc_set_state_fixed(mc_handle *h, const uint32_t *q, const int64_t *X, const int32_t *types);

/* Set the sweep counter (checkpoint resume).  Random numbers depend only on
 * (seed, sweep, cell, attempt), so resuming reproduces an uninterrupted run. */
int mc_set_sweep(mc_handle *h, uint64_t sweep);

/* Clear the counters of mc_stats (not e_run), the drift figures included. */
int mc_reset_stats(mc_handle *h);

/*
 * Record the time origin of the correlation functions (Sec. III.B): the
 * unwrapped positions, and per molecule the reference atom k (the atom of
 * type B now; Eq. 7) and the orientation vector u(0) from the centroid to k.
 */
int mc_set_t0(mc_handle *h);

/*
 * Time correlations against the last mc_set_t0 (Sec. III.B, Eq. 5-7):
 * out[3*r + 0] = F_s(q,t) over atoms and the n_qa wavevectors qvec_atom[3*n_qa],
 * out[3*r + 1] = F_s^cm over molecules and the n_qc vectors qvec_cm,
 * out[3*r + 2] = C_2(t) = <P_2(u(t).u(0))>.
 * Optional per-particle outputs (NULL to skip): fs_atom[total_sites],
 * fscm_mol[total_mol], c2_mol[total_mol].  FP64.  Synchronous.
 * Errors: INVALID_ARG (no t0, n_q < 1 or > 256).
 */
int mc_observables(mc_handle *h, const double *qvec_atom, int n_qa, const double *qvec_cm, int n_qc,
                   double *out, double *fs_atom, double *fscm_mol, double *c2_mol);

/*
 * Time correlations over many time origins, the statistics of Sec. III.E-F
 * built on Eq. 5-7.  mc_corr_setup starts a correlation clock t at 0 (the
 * current state is time 0); from then on t counts the sweeps that
 * mc_corr_run makes.  At every time t, in this order:
 *   1. each live origin o with t - t_o = lags[l] adds its per-particle
 *      correlations at t to the sums of lag l (below), per replica;
 *   2. an origin with t - t_o >= lags[n_lags-1] stops being live;
 *   3. if t is a multiple of origin_every and fewer than max_origins origins
 *      are live, the current state becomes a new origin (the positions, per
 *      molecule the atom of type B and the orientation u(0), as mc_set_t0),
 *      and if lags[0] = 0 it adds its lag-0 sample.
 * lags: n_lags (1..1024) strictly increasing sweep counts >= 0; origin_every
 * >= 1; max_origins 1..1024; the wavevectors as in mc_observables.  The
 * origins are kept on the device (3 int64 per site and 4 doubles per
 * molecule per origin).  A new setup replaces the previous one.
 * Errors: INVALID_ARG, CUDA (out of device memory).
 */
int mc_corr_setup(mc_handle *h, int n_lags, const int64_t *lags, int origin_every, int max_origins,
                  const double *qvec_atom, int n_qa, const double *qvec_cm, int n_qc);

/*
 * The origin schedule of mc_corr_setup / mc_corr_run, replayed on the host
 * alone (no handle, no GPU): counts[n_lags] = the number of samples each lag
 * holds after n_sweeps sweeps (n_sweeps >= 0).  Same rules for the arguments
 * as mc_corr_setup.  Errors: INVALID_ARG.
 */
int mc_corr_schedule(int n_lags, const int64_t *lags, int origin_every, int max_origins, int64_t n_sweeps,
                     int64_t *counts);

/*
 * n_sweeps sweeps (as mc_sweep_batch: the chain is the one that call would
 * make) with the correlation events of each time on the way.  Sweeps between
 * two event times run as one launch.  Asynchronous like mc_sweep_batch.
 * Errors: INVALID_ARG (no setup, bad arguments), CUDA.
 */
int mc_corr_run(mc_handle *h, int n_sweeps, const double *T, const mc_move_mix *mix, const uint64_t *seeds);

/*
 * The raw sums, FP64, sums[(r * n_lags + l) * MC_CORR_NSUM + j] for replica r
 * and lag l; over the n samples (origins measured at that lag) and, for the
 * per-particle sums, over the particles of each sample (F_s: the N atoms;
 * F_s^cm and C_2: the M molecules):
 *   j = 0: n;
 *   1, 2: sum of F_s, of F_s^2;     3, 4: sum of fs_i, of fs_i^2;
 *   5, 6: sum of F_s^cm, of its square;  7, 8: sum of fcm_i, of fcm_i^2;
 *   9, 10: sum of C_2, of C_2^2;    11, 12: sum of c2_i, of c2_i^2;
 *   13: sum of c2_i fcm_i;  14, 15: 0.
 * Sums of replicas at the same state point add.  Synchronous.
 */
#define MC_CORR_NSUM 16
int mc_corr_sums(mc_handle *h, double *sums);

/*
 * Derived per (replica, lag), out[(r * n_lags + l) * MC_CORR_NRES + j]:
 *   j = 0: n; 1-3: the averages F_s(q,t), F_s^cm(q,t), C_2(t) (Eq. 5-7);
 *   4-6: chi_4 = P (<C^2> - <C>^2) of F_s (P = N), F_s^cm and C_2 (P = M)
 *        (Eq. chi4 of Sec. III.E; <> over the samples);
 *   7-9: chi_4^self = <C_i^2> - <C_i>^2 of the same three (over particles
 *        and samples);
 *   10: the Pearson coefficient of c2_i and fcm_i (Eq. pearson of Sec. III.F).
 * NaN where n = 0 (and for rho where a variance is 0).  Synchronous.
 */
#define MC_CORR_NRES 11
int mc_corr_results(mc_handle *h, double *out);

/*
 * The derivation of mc_corr_results on its own (host only, no handle): n_rows
 * rows of MC_CORR_NSUM sums (layout of mc_corr_sums) into rows of
 * MC_CORR_NRES results, n_atoms[k] the atoms N of row k's replica (a positive
 * multiple of 3).  Errors: INVALID_ARG.
 */
int mc_corr_derive(int n_rows, const double *sums, const int32_t *n_atoms, double *out);

/*
 * Relaxation time per replica (Sec. III.C: the time at which a correlation
 * function reaches e^-1): the first lag l (in increasing order, lags with no
 * sample skipped) at which the average of which = 0 (F_s), 1 (F_s^cm) or
 * 2 (C_2) is <= level, interpolated linearly in ln t from the previous lag
 * (linearly in t when that lag is 0), or lags[l] itself when it is the first
 * lag sampled.  tau[n_rep] (host); NaN where the series stays above level.
 * Synchronous.  Errors: INVALID_ARG (no setup, which out of range).
 */
int mc_corr_relaxation_time(mc_handle *h, int which, double level, double *tau);

/*
 * The same interpolation on one series (host only): values[l] at lags[l]
 * (increasing), counts[l] > 0 where the lag has samples; *tau as above.
 * Errors: INVALID_ARG.
 */
int mc_relaxation_time(int n_lags, const int64_t *lags, const double *values, const double *counts, double level,
                       double *tau);

/*
 * Molecular dynamics of the same model (Sec. II.D: NVT, time step 0.001,
 * Nose-Hoover thermostat with relaxation time 1), FP64, m = 1.  One step is
 * the symmetric splitting
 *   xi += dt/2 (2K - gT)/Q; eta += dt/2 xi; v *= exp(-xi dt/2); v += dt/2 F;
 *   q += rint(v dt / h) (the fixed-point positions; periodic images counted);
 *   F = -grad U (Eq. 1 and 2) from the rebuilt cell list;
 *   v += dt/2 F; v *= exp(-xi dt/2); xi += dt/2 (2K - gT)/Q; eta += dt/2 xi,
 * with K = sum v^2 / 2 per replica (fixed order), g = 3N, Q = g T tau_T^2.
 * mc_md_setup: dt > 0; tau_T > 0, or <= 0 for no thermostat (constant
 * energy); T[n_rep] the bath temperatures; v0[3 N] the initial velocities in
 * site order (host, copied); xi = eta = 0.  The positions are the handle's
 * state; MD steps and MC sweeps may alternate (after MD steps the running
 * MC energy restarts from a recompute).  force_precision: MC_PREC_FP64 (pair
 * forces in FP64, the oracle-parity path) or MC_PREC_FP32 (pair terms and
 * their per-atom sums in FP32, from the exact int32 differences; velocities,
 * positions, the thermostat and energies stay FP64).
 * mc_md_run: n_steps steps, each one CUDA graph.  Asynchronous.
 * mc_md_state: v_out[3 N] (nullable) and per replica out[5 r + {0..4}] =
 * K, U, xi, eta, and the conserved K + U + Q xi^2/2 + g T eta (K + U without
 * a thermostat).  Synchronous.
 * Errors: INVALID_ARG (NULL, dt <= 0, T <= 0, no setup), CUDA.
 */
int mc_md_setup(mc_handle *h, double dt, double tau_T, const double *T, const double *v0, int force_precision);
int mc_md_run(mc_handle *h, int n_steps);
int mc_md_state(mc_handle *h, double *v_out, double *out);

/* Pick the cell schedule: run n_sweeps sweeps (>= 1) with each schedule (1,
 * 2, 4 and 8 warps per cell, as one persistent launch per call and as one
 * CUDA graph per sweep) from the same state, time them on the handle's stream
 * and keep the fastest.  The state, the sweep counters, the running energies and
 * the statistics are restored afterwards: the chain continues exactly as if
 * the call had not been made (the schedule never changes the chain).  The
 * arguments T, mix and seeds are those of mc_sweep_batch.  results (nullable,
 * host, 8 doubles): ms per sweep for W = 1, 2, 4, 8 persistent, then W = 1, 2, 4, 8
 * graphs; a schedule that cannot run reads -1.  Not part of the paper's method:
 * an engineering choice of the library.  Errors: INVALID_ARG, CUDA. */
int mc_autotune(mc_handle *h, int n_sweeps, const double *T, const mc_move_mix *mix, const uint64_t *seeds,
                double *results);

/* Static facts of the handle. */
int mc_get_info(mc_handle *h, mc_info *info);

/*
 * Total FP64 energy (the quantity mc_energy returns, every pair once) of one
 * configuration that already sits in the caller's device memory, for callers
 * that cannot allocate device memory: code running inside another framework's
 * memory pool or under a fixed device-memory budget, or code that may only
 * enqueue kernels on a stream it was given.  The paper has no counterpart;
 * this is an interface convenience.
 *   L: box side; n_mol: molecules, 1 <= n_mol <= 21845 (at most 65536 atoms);
 *   dev_q: 3*3*n_mol fixed-point positions (q = floor(frac(x/L) 2^32)),
 *   dev_types: 3*n_mol types in {0,1,2}, dev_E_out: one double, all three
 *   device memory of the current device, owned by the caller;
 *   params: host, NULL picks the paper's potential; stream: cudaStream_t
 *   (NULL: the legacy default stream).
 * Allocates nothing: the working space is a fixed __device__ array of this
 * library (about 3.5 MB on every GPU that loads it, kept until exit).  All
 * calls on a device share that array: calls whose work overlaps on the GPU
 * race and must be serialised by the caller.  The first call on a device
 * looks up the array's address and should come before any stream capture.
 * The call only enqueues kernels and device-memory clears on the stream (it
 * copies nothing from host memory); the result is ready when the stream
 * reaches it.  A type outside {0,1,2} or a broken bond gives NaN (or +inf);
 * the next valid call clears that state.
 * Errors: INVALID_ARG (sizes beyond the maximum, NULL pointers, box smaller
 * than two interaction ranges), NO_DEVICE, CUDA.
 */
int mc_energy_noalloc(double L, int n_mol, const uint32_t *dev_q, const int32_t *dev_types, const mc_params *params,
                      double *dev_E_out, void *stream);

/*
 * Test hook for the library's failure paths (the paper has no counterpart):
 * after this call, the device allocation number `after` (0 = the next one)
 * made by mc_create / mc_create_batch fails as if the device were out of
 * memory; that call then frees what it had allocated and returns
 * MC_ERR_CUDA.  The hook disarms itself once it has fired; after < 0 disarms
 * it.  Process-wide; not meant for production use.
 */
void mc_test_fail_alloc(int after);

/* Message describing the calling thread's last error ("" if none). */
const char *mc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FLIPMC_H */
