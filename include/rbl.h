/*
 * rbl.h -- C ABI of librbl, a GB300 (sm_103a) implementation of the random-batch
 * list (RBL) short-range force step for Lennard-Jones molecular dynamics
 * (Liang, Xu & Zhao, arXiv 2105.04884).
 *
 * Method (Sec. 2 of the paper): each particle keeps a core neighbour list
 * (r < r_c) summed directly (Eq. (3)) and a shell list (r_c <= r < r_s) from which a
 * random batch of p neighbours is drawn and scaled by N_s/p (Eq. (4)); the mean
 * force is subtracted (Appendix A, F_cor) and the Langevin equation (Eq. (2)) is
 * advanced with a velocity-Verlet splitting (Algorithm 1; Sec. 3).  The pair kernel
 * is LJ 12-6 (Eq. (1)), optionally plus the Ewald real-space Coulomb term, the
 * extension the paper names for other short-range kernels (Sec. 2, closing
 * remarks; Sec. 4).
 *
 * Conventions shared by every entry point
 *  - Units: reduced LJ units, sigma = epsilon = m = k_B = 1; charges such that two
 *    unit charges at distance r have Coulomb energy 1/r.
 *  - Particle arrays passed in or out are in TAG order (row t describes the particle
 *    whose tag is t), AoS [N][3] doubles for positions/velocities/forces.  Inside the
 *    context particles are kept in cell order; the library translates.
 *  - Replicas: a context holds R >= 1 independent systems (rbl_create: R = 1;
 *    rbl_create_batch: any R), advanced together by one launch per kernel.  Per-
 *    particle arrays then hold the replicas' rows one after another ("packed": rows
 *    in0_r .. in0_r + N_r - 1 for replica r, in0_r = N_0 + ... + N_{r-1}); tags and
 *    neighbour tags are numbers within a replica.  Per-replica outputs (rbl_obs,
 *    exact energies, histograms) are arrays of R.
 *  - "ptr_is_device": 0 means the pointer is host memory (the call copies through
 *    the context's stream and synchronises), 1 means device memory on the context's
 *    device (the call is asynchronous on the context's stream).
 *  - Memory: the caller owns one device workspace of rbl_workspace_size() bytes
 *    (any allocator; 256-byte aligned) and passes it to rbl_create; the context
 *    carves every device array out of it and never allocates device memory itself.
 *    The workspace must outlive the context.
 *  - Streams: every kernel runs on the stream given to rbl_create (NULL = legacy
 *    default stream).  Calls on one context must not run concurrently.
 *  - Errors: every call returns an rbl_status; rbl_last_error() describes the last
 *    failure on that context.  Device-side problems (row overflow, non-finite
 *    positions, bounded waits that expired) are recorded in device flags and
 *    reported by the next call that synchronises (rbl_step, rbl_forces with a host
 *    pointer, rbl_observables, rbl_get_*).  No kernel traps.
 *  - Random numbers: Philox4x32-10 (Salmon et al., SC'11), counter
 *    (step_lo, step_hi, tag, stream<<24 | block), key (seed_lo, seed_hi); stream 0
 *    draws the batches, stream 1 the thermostat noise.  Results therefore depend
 *    only on (parameters, initial state, seed, step counter), never on launch
 *    configuration.
 */
#ifndef RBL_H
#define RBL_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rbl_ctx rbl_ctx;

typedef enum {
    RBL_OK = 0,
    RBL_EINVAL = 1,      /* bad argument (message in rbl_last_error) */
    RBL_ENOMEM = 2,      /* workspace too small */
    RBL_EOVERFLOW = 3,   /* a list row or cell exceeded its capacity; recreate with larger caps */
    RBL_ENONFINITE = 4,  /* a non-finite position, velocity or force was produced, a force left the
                            fixed-point range (|F| >= 2^29: overlapping particles), or a particle moved
                            more than a box length in one step */
    RBL_ETIMEOUT = 5,    /* a bounded device wait gave up */
    RBL_ECUDA = 6        /* a CUDA runtime call failed (message in rbl_last_error) */
} rbl_status;

enum { RBL_FP64 = 0, RBL_FP32 = 1 };

/* Where the shell batch is drawn from (Sec. 2):
 *  RBL_SAMPLE_SHELL   (default) the shell list, j with max(r_c - skin, 0) <= r <
 *                     r_s + skin at the last build; scale N_s / p.  Cells of width
 *                     >= (r_s + skin) / K, stencil (2K + 1)^3.
 *  RBL_SAMPLE_STENCIL the paper's own pool: every other particle of the
 *                     (2 floor(r_s / r_c) + 3)^3 stencil of cells of edge >= r_c + skin
 *                     around the particle's cell; scale N_I / p.  No shell list is
 *                     built (the core list comes from the 27 nearest cells), but only
 *                     about one draw in ten lands in the shell, so the estimator's
 *                     variance is larger at the same p.  Needs r_s / r_c < 3 and
 *                     full_list = 0; cells_per_cutoff is not used. */
enum { RBL_SAMPLE_SHELL = 0, RBL_SAMPLE_STENCIL = 1 };

/* Pair potential of every pair with r < r_s (the RBL applies to any short-range
 * kernel, Sec. 2 closing remarks and Sec. 4, which name the Ewald real-space term):
 *  RBL_POT_LJ        (default) u(r) = 4 (r^-12 - r^-6)
 *  RBL_POT_LJ_EWALD  u(r) = 4 (r^-12 - r^-6) + q_i q_j erfc(alpha r) / r, the short-
 *                    range part of the Coulomb interaction in an Ewald splitting;
 *                    r . f adds q_i q_j (erfc(alpha r) / r + 2 alpha / sqrt(pi)
 *                    exp(-alpha^2 r^2)).  Charges come from rbl_set_charges (all
 *                    zero until then).  The reciprocal-space and self terms of the
 *                    Ewald sum are not part of this library. */
enum { RBL_POT_LJ = 0, RBL_POT_LJ_EWALD = 1 };

typedef struct {
    double L[3];          /* periodic box lengths; each >= 2 (r_s + skin) */
    double r_c;           /* core radius: pairs r < r_c summed directly (Eq. (3)) */
    double r_s;           /* cutoff radius: pairs r_c <= r < r_s sampled (Eq. (4)) */
    double skin;          /* Verlet skin; lists rebuilt when a particle moved > skin/2 */
    int p;                /* batch size, 1 <= p <= 128 */
    double dt;            /* time step */
    double T;             /* bath temperature (k_B T) */
    double gamma;         /* Langevin friction; 0 = plain velocity-Verlet (NVE) */
    unsigned long long seed;
    int precision;        /* RBL_FP32: binary32 pair math, int64 fixed-point force sums;
                             RBL_FP64: FP64 pair math and sums */
    int full_list;        /* 1: classical cutoff with one full Verlet list (no batch) */
    int subtract_net_force; /* 1 (default): subtract the mean force (Appendix A) */
    int cells_per_cutoff; /* K: cell width >= (r_s + skin)/K, stencil (2K+1)^3; 1..3 */
    int cap_core;         /* core row capacity; 0 = derived from the density */
    int cap_stencil;      /* capacity of a cell's culled candidate table (shell
                             sampling: the stencil members within r_s + skin of the
                             cell's particles; shell rows are bitmasks over it);
                             0 = derived from the density */
    double rho_cap;       /* number density the derived capacities are sized for;
                             0 = the mean density N/V.  Set it to the densest
                             region's density for inhomogeneous systems (a liquid
                             slab in vapour), else rows overflow (RBL_EOVERFLOW). */
    int sampling;         /* RBL_SAMPLE_SHELL (default) or RBL_SAMPLE_STENCIL */
    int potential;        /* RBL_POT_LJ (default) or RBL_POT_LJ_EWALD */
    double alpha;         /* Ewald splitting parameter (> 0) for RBL_POT_LJ_EWALD */
} rbl_params;

typedef struct {
    double U_est;         /* RBL energy estimate: 1/2 sum_i [sum_core u + s_i sum_B u] */
    double W_est;         /* RBL virial estimate, same weights, W = sum r.f */
    double K;             /* kinetic energy sum v^2 / 2 */
    double T_kin;         /* 2K / (3N) */
    double P;             /* rho T_kin + W_est / (3V) (no tail) */
    double U_tail;        /* per-particle LJ tail energy (8/3) pi rho (r_s^-9/3 - r_s^-3) */
    double P_tail;        /* LJ tail pressure (16/3) pi rho^2 (2 r_s^-9/3 - r_s^-3) */
    double net_momentum[3];
    long long step;       /* step counter */
    long long n_rebuild;  /* list builds so far */
    double Ns_mean;       /* mean shell (or full) row length at the last build */
    double Nc_mean;       /* mean core row length at the last build */
    double Mc_mean;       /* mean stencil population of a particle's home cell at the last build */
    int Ns_max;           /* longest shell (or full) row at the last build */
    int Nc_max;           /* longest core row at the last build */
} rbl_obs;

/* Fills *prm with defaults: cells_per_cutoff 2, subtract_net_force 1, precision FP32,
 * gamma 0, caps 0 (automatic).  Box, radii, p, dt, T, seed must still be set. */
void rbl_params_default(rbl_params *prm);

/* Bytes of device workspace a context for N particles with these parameters needs.
 * Returns RBL_EINVAL for invalid parameters (see rbl_create). */
rbl_status rbl_workspace_size(const rbl_params *prm, int N, size_t *bytes);

/* Creates a context (host memory for the handle only).  Validates: N >= 2,
 * 0 < r_c < r_s, skin >= 0, 1 <= p <= 128, dt > 0, T >= 0, gamma >= 0, finite values,
 * every L_a >= 2 (r_s + skin), K in 1..3, potential RBL_POT_LJ or RBL_POT_LJ_EWALD
 * (then alpha > 0 and finite).  stream is a cudaStream_t (or NULL).
 * The initial state is zero; load one with rbl_set_state. */
rbl_status rbl_create(const rbl_params *prm, int N, void *workspace, size_t workspace_bytes, void *stream,
                      rbl_ctx **out);

/* Batched ensemble: R independent replicas of N[r] particles each, with parameters
 * prm[r] (each validated as for rbl_create).  Replicas may differ in the box L, the
 * bath temperature T, the seed and N; every other field must equal prm[0]'s
 * (RBL_EINVAL otherwise).  Each replica evolves exactly as a context of its own
 * would: its own Philox streams (its seed, its tags), its own net-force correction,
 * and its own rebuild decisions (a replica's lists are rebuilt only when one of its
 * own particles moved more than skin/2).  Every kernel launch covers all replicas,
 * and the steady-state step is one CUDA graph for the whole ensemble.  Particle
 * slots are allocated per replica in multiples of 256, so a workspace for R small
 * replicas is larger than one for a single system of the same total N. */
rbl_status rbl_workspace_size_batch(const rbl_params *prm, int R, const int *N, size_t *bytes);
rbl_status rbl_create_batch(const rbl_params *prm, int R, const int *N, void *workspace, size_t workspace_bytes,
                            void *stream, rbl_ctx **out);

/* Number of replicas of a context (0 for NULL). */
int rbl_replicas(const rbl_ctx *ctx);

/* Loads positions x[N][3] (wrapped into [0, L)), velocities v[N][3] (may be NULL:
 * zero) and the step counter; marks the lists stale.  Rejects non-finite input. */
rbl_status rbl_set_state(rbl_ctx *ctx, const double *x, const double *v, long long step, int ptr_is_device);

/* Charges q[N] in tag order (packed over replicas) for RBL_POT_LJ_EWALD; they stay
 * with their particles through every rebuild and rbl_set_state.  Marks the force
 * stale.  RBL_EINVAL on a context without charges (RBL_POT_LJ) or for a non-finite
 * charge (checked on the host copy, so host pointers only). */
rbl_status rbl_set_charges(rbl_ctx *ctx, const double *q);

/* Copies positions and velocities (either may be NULL) out in tag order, and the
 * step counter (may be NULL). */
rbl_status rbl_get_state(rbl_ctx *ctx, double *x, double *v, long long *step, int ptr_is_device);

/* Checkpoint and resume (Algorithm 1: each step's batches are keyed by (seed, step,
 * tag) and drawn from the rows of the last list build, so a resumed run needs those
 * rows, not a fresh build).  A checkpoint holds the positions and velocities (tag
 * order), the fixed-point images the lists were last built from, the step counter
 * and each replica's rebuild count: rbl_checkpoint_size() bytes, an opaque byte
 * buffer (host or device memory, 8-byte aligned).  rbl_load_checkpoint into a
 * context created with the same parameters and sizes rebuilds the lists from the
 * saved images and recomputes the force at the saved step when it is next needed,
 * so the steps that follow are bit-identical to continuing the saved context (every
 * replica, either precision); it needs no extra rebuild at the resume step.  Charges
 * (RBL_POT_LJ_EWALD) are not part of a checkpoint: set them with rbl_set_charges,
 * before or after loading.  RBL_EINVAL for a buffer that is not a checkpoint or that
 * was saved from a context of other sizes or precision.  Both calls synchronise. */
rbl_status rbl_checkpoint_size(const rbl_ctx *ctx, size_t *bytes);
rbl_status rbl_save_checkpoint(rbl_ctx *ctx, void *buf, int ptr_is_device);
rbl_status rbl_load_checkpoint(rbl_ctx *ctx, const void *buf, int ptr_is_device);

/* Builds the cell list and the two-level neighbour lists from the current positions
 * (Sec. 2: linked cells, core list r < r_c + skin, shell list
 * max(r_c - skin, 0) <= r < r_s + skin; or the full list r < r_s + skin).
 * rbl_step rebuilds by itself when needed; this forces a build now. */
rbl_status rbl_build_lists(rbl_ctx *ctx);

/* One force evaluation at the current positions with the batch drawn for the
 * current step counter (Eqs. (3)-(4); mean force subtracted when enabled).
 * F_out[N][3] in tag order (may be NULL: the force stays in the context), and the
 * energy/virial estimates are refreshed for rbl_observables. Builds lists if stale. */
rbl_status rbl_forces(rbl_ctx *ctx, double *F_out, int ptr_is_device);

/* Advances n >= 0 steps of Algorithm 1: velocity-Verlet kick/drift with the Langevin
 * O-step between the drifts (BAOAB) when gamma > 0, list rebuild whenever some
 * particle moved more than skin/2 since the last build, RBL force, final kick.
 * Between two steps the closing half kick of one and the opening half kick of the
 * next are one kick of dt, also across calls: a call ends after its last force
 * evaluation and the next call's first step applies the pending half kick with its
 * own, so a run gives the same trajectory however it is split into calls.  The
 * velocities that rbl_get_state, rbl_observables and checkpoints report or keep are
 * those at the end of the last step (the pending half kick included in what is
 * reported; a checkpoint keeps it pending).  rbl_set_charges and rbl_build_lists
 * apply a pending half kick first (it is due with the current force); rbl_set_state
 * discards it.  Synchronises at the end and reports device flags. */
rbl_status rbl_step(rbl_ctx *ctx, int n);

/* rbl_step without the wait: enqueues the n steps on the context's stream and returns.
 * Device flags are reported by the next call that synchronises.  With phase timing
 * enabled it is rbl_step. */
rbl_status rbl_step_async(rbl_ctx *ctx, int n);

/* Scalars of the current state (kinetic terms from the current velocities, energy
 * and virial from the last force evaluation), out[R]: one per replica.
 * Synchronises. */
rbl_status rbl_observables(rbl_ctx *ctx, rbl_obs *out);

/* rbl_observables without the wait: enqueues on the context's stream the kinetic sums,
 * the assembly of the same rbl_obs[R] values on the device, and their delivery into
 * out[R] (host memory, or device memory with ptr_is_device = 1), and returns.  Page-
 * locked host memory and device memory are written by the assembling kernel itself;
 * other host memory receives a copy, which is asynchronous only if that memory is
 * page-locked.  out is valid once the stream has reached the
 * copy (synchronise the stream, or make any synchronising call).  Device flags are
 * not read here; the next synchronising call reports them.  For reading the scalars
 * every step without stalling the step sequence. */
rbl_status rbl_observables_async(rbl_ctx *ctx, rbl_obs *out, int ptr_is_device);

/* The energy and virial of the truncated potential at the current positions, with
 * no sampling: *U = sum over pairs i<j with r_ij < r_s of u(r_ij), *W the virial
 * sum r.f over the same pairs (Sec. 3 observables; the quantities the RBL estimates
 * U_est, W_est are unbiased for).  Every core entry with r < r_c and every shell
 * entry with r_c <= r < r_s is summed once per ordered pair and halved, so the cost
 * is that of a full-list force pass; nothing in the context's force state changes.
 * Pair terms in the context's precision, per-particle sums then FP64.  Builds lists
 * if stale.  U[R], W[R]: one per replica.  Synchronises; host pointers. */
rbl_status rbl_exact_energy(rbl_ctx *ctx, double *U, double *W);

/* Parity hooks.  kind 0 = core rows, 1 = shell rows (full rows when full_list).
 * rows[N][cap] receives neighbour TAGS in the canonical row order (stencil slot of
 * the neighbour's cell, then the neighbour's 32-bit x image, then tag), counts[N]
 * the lengths; host pointers.  Rows
 * longer than cap return RBL_EOVERFLOW. Builds lists if stale. */
rbl_status rbl_get_lists(rbl_ctx *ctx, int kind, int *rows, int cap, int *counts);

/* The same rows for m selected particles only: which[m] are packed row indices,
 * rows[m][cap] and counts[m] receive their rows as rbl_get_lists would.  Copies
 * only those particles' list data, so it suits very large systems.  Builds lists
 * if stale; host pointers. */
rbl_status rbl_get_rows(rbl_ctx *ctx, int kind, const long long *which, int m, int *rows, int cap, int *counts);

/* The batch B(i) the force would use at step counter `step` with the current
 * lists: batch[N][p] neighbour tags in ascending row position, counts[N] = min(p,
 * N_s); host pointers. */
rbl_status rbl_get_batch(rbl_ctx *ctx, long long step, int *batch, int *counts);

/* Pair-distance histogram for g(r) (Sec. 3): adds to hist[b] the number of ordered
 * pairs i != j with r < r_s and floor(sqrt(r2) / dr) = b < nbins, each pair taken
 * from the list that classifies it like the force does (core rows for r < r_c,
 * shell rows for r_c <= r < r_s; full rows in full-list mode).  Requires
 * nbins * dr <= r_s.  hist[R][nbins] int64 (one histogram per replica), host
 * pointer, accumulated (not cleared).  Builds lists if stale. */
rbl_status rbl_rdf(rbl_ctx *ctx, float dr, int nbins, long long *hist);

/* Density profile along axis (0 = x, 1 = y, 2 = z) at the current positions
 * (Sec. 3 observables; the slab benchmark's z profile): adds to hist[r][b] the
 * number of particles of replica r with floor(u_a nbins / 2^32) = b, u_a the
 * particle's 32-bit fixed-point image along the axis (bins of width L_a / nbins).
 * 1 <= nbins <= 12288.  hist[R][nbins] int64, host pointer, accumulated (not
 * cleared).  Synchronises. */
rbl_status rbl_density_profile(rbl_ctx *ctx, int axis, int nbins, long long *hist);

/* Launch shapes, which no result depends on (the tests check this bit for bit):
 * threads per block of the force kernel (64, 128 or 256; default 256 for FP32 with
 * shell sampling or the full list, 128 otherwise) and home
 * cells (warps) per block of the list build (2, 4 or 8; default 4).
 * rbl_autotune times every candidate of each on the current state (`trials`
 * launches each, after one warm-up) and keeps the fastest, reporting the choice
 * through the optional out pointers.  It times the list build on the images of the
 * last build, so the lists, the particle order, the state, the step counter and the
 * per-replica counters are as they were afterwards.  Synchronises. */
rbl_status rbl_set_launch_config(rbl_ctx *ctx, int force_threads, int build_warps);
rbl_status rbl_autotune(rbl_ctx *ctx, int trials, int *force_threads, int *build_warps);

/* Cell size by measurement (the linked cells of Sec. 2 / Fig. 1: cells of width
 * >= (r_s + skin)/K, stencil (2K + 1)^3).  K is not a launch shape: the canonical row
 * order follows the cell stencil, so K decides which batch each step draws (every K
 * samples the same shell rows uniformly; the oracle reproduces each K's batches), and
 * it is chosen before a run.  rbl_tune_cells runs the caller's system (positions x,
 * velocities v, [N][3] tag-order host arrays, read only) for K = 1, 2 and 3 in turn,
 * each in a context of its own created in `workspace` (device memory of at least
 * rbl_tune_cells_workspace_size bytes, the largest of the three workspaces; the call
 * allocates nothing) with its launch shapes autotuned: `steps` warm-up steps, then
 * `steps` steps timed with CUDA events on `stream` (use steps >= 10 so that the
 * timing includes list rebuilds).  It returns the fastest K in *K_best and, when
 * ms_per_step is not NULL, the three times in ms_per_step[3] (-1 for a K that the
 * parameters do not allow or that does not fit the workspace).  prm's own
 * cells_per_cutoff is ignored.  Errors of the trial runs are returned as they occur
 * (a blow-up of the given state, RBL_ENONFINITE, for instance).  Synchronises. */
rbl_status rbl_tune_cells_workspace_size(const rbl_params *prm, int N, size_t *bytes);
rbl_status rbl_tune_cells(const rbl_params *prm, int N, const double *x, const double *v, void *workspace,
                          size_t workspace_bytes, void *stream, int steps, int *K_best, float *ms_per_step);

/* Phase timing.  While enabled, rbl_step launches each step's phases directly (no
 * graph replay) and brackets them with CUDA events on the context's stream:
 * phase 0 = kick/drift/thermostat kernel, 1 = cell hash, scan, sort and permutation,
 * 2 = list build (1 and 2 are device-conditional: their kernels return at once when
 * no rebuild is due), 3 = force kernel alone, 4 = force reduction.  rbl_phase_times
 * writes the elapsed milliseconds of every timed step since the last reset, summed
 * per phase, to ms[5] and reports the number of timed steps; reset = 1 clears them. */
rbl_status rbl_set_phase_timing(rbl_ctx *ctx, int enable);
rbl_status rbl_phase_times(rbl_ctx *ctx, double ms[5], long long *steps, int reset);

/* With phase timing enabled, every rebuild made outside the step loop (rbl_build_lists,
 * and the first force evaluation after a new state) is timed on its own: ms[0] the cell
 * sort chain, ms[1] the list build, summed over *rebuilds such rebuilds (host pointers;
 * either may be NULL).  These carry none of the skipped rebuild launches that the
 * phase-timed steps which do not rebuild make.  reset = 1 clears the sums after reading. */
rbl_status rbl_rebuild_times(rbl_ctx *ctx, double ms[2], long long *rebuilds, int reset);

/* Allocation-free force evaluation (the paper has no counterpart; this is a service
 * for callers that may not allocate).  Some callers cannot allocate device memory
 * when they need forces: a plugin called inside another engine's time step whose
 * host application owns all device memory through its own pool and forbids
 * cudaMalloc (it can fail or synchronise the device mid-run), or code bound by a
 * no-allocation rule after initialisation.  This call computes, like rbl_forces on
 * a fresh context, the mean-subtracted RBL (or full-list) force of positions
 * x[N][3] (device pointer, tag order) at step counter `step` into F[N][3] (device
 * pointer, tag order), on `stream`, and synchronises that stream.  It allocates
 * nothing: its working memory is one file-scope device array of 48 MiB, which every
 * device where the library's module is loaded (at the latest on the first call of
 * this function there) holds until the process exits.  The first call on a device,
 * made with that device current, sets the array up there and looks up its device
 * address; make that first call before any stream capture.  Later calls look the
 * address up again (a device reset may move it).  Systems whose workspace (as
 * rbl_workspace_size reports) exceeds 48 MiB are rejected with RBL_ENOMEM (about
 * 44,000 particles at rho* = 0.8 with the default radii); invalid parameters with
 * RBL_EINVAL, and so is RBL_POT_LJ_EWALD (this call takes no charges).  Every call
 * shares the array, so calls that overlap on the GPU (two streams, two host threads)
 * race: serialise them.  Each call resets the parts it reads; the array keeps the
 * last call's contents otherwise. */
rbl_status rbl_forces_static(const rbl_params *prm, int N, const double *x, long long step, double *F, void *stream);

/* Releases the handle (the workspace stays the caller's). NULL is ignored. */
void rbl_destroy(rbl_ctx *ctx);

/* Text of the last error on ctx ("" if none); valid until the next call. */
const char *rbl_last_error(const rbl_ctx *ctx);

/* Short name of a status code. */
const char *rbl_status_string(rbl_status s);

#ifdef __cplusplus
}
#endif

#endif /* RBL_H */
