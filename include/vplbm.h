/*
 * vplbm.h -- C ABI of a GB300 (sm_103a) volume-penalized lattice Boltzmann
 * solver: D2Q9 VP-LBM with the two fluid-force estimators compared by
 * Liberge & Beghein, "About fluid forces computation for Volume Penalization
 * coupled with Lattice Boltzmann method" (arXiv 2110.00967).
 *
 * Conventions for every entry point:
 *   - Every call returns a vplbm_status and never aborts, exits or prints.
 *     The text of the last failure is available from vplbm_last_error().
 *   - The library never allocates device memory.  The caller hands it one
 *     device workspace at creation (vplbm_workspace_bytes tells the size) and
 *     owns it; vplbm_destroy does not free it.  Pointers documented as
 *     "device" are caller-owned device memory, pointers documented as "host"
 *     are caller-owned host memory.
 *   - All GPU work is queued on the caller's CUDA stream given at creation
 *     (or vplbm_set_stream).  vplbm_step only queues work; calls that return
 *     host values synchronise that stream.
 *   - Lattice node (i, j) sits at x = i, y = j (lattice units, dx = dt = 1);
 *     i runs fastest.  Fields of a lattice are laid out [j][i]; populations
 *     are laid out [a][j][i] with the D2Q9 numbering of the paper's Fig. d2q9:
 *     a = 0 rest, 1 (1,0), 2 (0,1), 3 (-1,0), 4 (0,-1), 5 (1,1), 6 (-1,1),
 *     7 (-1,-1), 8 (1,-1).
 *   - Forces are the force exerted by the fluid on the body (Eqs. MMEL and
 *     defFf); torques are taken about the body reference point (x_c, y_c).
 */
#ifndef VPLBM_H
#define VPLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vplbm_ctx vplbm_ctx;

typedef enum {
  VPLBM_OK = 0,
  VPLBM_EINVAL = 1,    /* bad argument or configuration */
  VPLBM_ENOMEM = 2,    /* workspace too small */
  VPLBM_ECUDA = 3,     /* a CUDA runtime call failed */
  VPLBM_EUNSTABLE = 4, /* a non-finite or non-positive density was met (latched) */
  VPLBM_ETIMEOUT = 5,  /* a bounded device-side wait ran out */
  VPLBM_ESTATE = 6     /* call not valid in the current state (no body, no step yet,
                          SIM point without a fluid node) */
} vplbm_status;

/* Storage of the populations.  All forms store offsets h_a = f_a - E_a from
 * E_a = feq_a(1, u_ref) (config.u_ref; zero gives the lattice weights w_a).
 * F64 computes in FP64; the others compute the step in FP32.  F16_OFS and
 * BF16_OFS round each stored value to nearest even; F16_SR and BF16_SR round
 * it stochastically: up or down with probabilities in proportion to its
 * distances from the two neighbouring 16-bit values, drawn from a counter-
 * based hash of the lattice's step count, the node and the population
 * (reproducible run to run).  Rounding to nearest leaves a steady flow in a
 * quantized state offset from the exact one, which time averages keep;
 * stochastic rounding has no such offset on average.  Force sums are exact
 * 64-bit fixed-point integers converted to FP64; the rigid-body update is
 * FP64 in every form. */
typedef enum {
  VPLBM_F64 = 0,
  VPLBM_F32 = 1,
  VPLBM_F16_OFS = 2,
  VPLBM_BF16_OFS = 3,
  VPLBM_F16_SR = 4,
  VPLBM_BF16_SR = 5
} vplbm_dtype;

/* Collision operator: BGK (Sec. 2.2) or TRT (Eq. TRT) with
 * tau- = Lambda / (tau+ - 1/2) + 1/2. */
typedef enum { VPLBM_BGK = 0, VPLBM_TRT = 1 } vplbm_collision;

/* How the forcing term F_a (Guo et al., cited with Eq. eqBd) enters TRT:
 * PAPER multiplies all of F_a by (1 - 1/(2 tau+)) as Eq. TRT prints it;
 * SPLIT multiplies its antisymmetric part by (1 - 1/(2 tau-)) instead.
 * Both are the same for BGK. */
typedef enum { VPLBM_FORCING_PAPER = 0, VPLBM_FORCING_SPLIT = 1 } vplbm_forcing;

/* Side conditions (Sec. 3.1 and 3.2).  x sides: PERIODIC (both), INLET_BB
 * (half-way bounce-back from a wall moving at u_in), OUTLET_CONVECTIVE (x_hi
 * only; convective condition with U_c = |u_in|), OUTLET_FREE (x_hi only; the
 * "free flow" outlet of Sec. 3.2 read as a zero normal gradient: populations
 * entering the last column copy those of the column before it), NOSLIP_BB.  y sides:
 * PERIODIC (both), SYMMETRY (specular reflection), NOSLIP_BB.  Walls sit half
 * a cell beyond the edge nodes. */
typedef enum {
  VPLBM_PERIODIC = 0,
  VPLBM_INLET_BB = 1,
  VPLBM_OUTLET_CONVECTIVE = 2,
  VPLBM_SYMMETRY = 3,
  VPLBM_NOSLIP_BB = 4,
  VPLBM_OUTLET_FREE = 5
} vplbm_bc;

typedef enum { VPLBM_BODY_NONE = 0, VPLBM_BODY_DISK = 1, VPLBM_BODY_NACA4 = 2 } vplbm_body_kind;

/* force estimators: momentum exchange (Sec. 2.3.1), stress integration
 * (Sec. 2.3.2), and the volume integral of Eq. Angotforce (Sec. 2.3), which
 * the paper reports as failing and which only the history read-backs offer */
typedef enum { VPLBM_MEM = 0, VPLBM_SIM = 1, VPLBM_ANGOT = 2 } vplbm_estimator;

typedef struct {
  int32_t nx, ny;          /* lattice size, each >= 3 */
  int32_t dtype;           /* vplbm_dtype */
  int32_t collision;       /* vplbm_collision */
  int32_t forcing;         /* vplbm_forcing */
  int32_t bc[4];           /* vplbm_bc for x_lo, x_hi, y_lo, y_hi */
  int32_t sim_every;       /* evaluate SIM every k-th step (0: never) */
  int32_t max_sim_points;  /* capacity for SIM points (0: 4096) */
  int32_t history_len;     /* per-step force history ring length (0: 1024) */
  int32_t sim_order;       /* SIM stress at a point: 0 copied from the first fluid node along
                              the sampling direction (Sec. 2.3.2); 1 extrapolated linearly
                              from the first two (not in the paper) */
  double tau_plus;         /* > 1/2; nu = (tau+ - 1/2)/3 (Eq. tauvisco) */
  double lambda_trt;       /* TRT magic parameter Lambda (1/6 in Sec. 2.2) */
  double eta;              /* penalization factor, > 0 (1e-6 in Sec. 3) */
  double u_in[2];          /* inlet velocity and the initial fluid velocity */
  double body_force[2];    /* uniform force density on every node (0 in the paper) */
  double u_ref[2];         /* populations are stored as f_a - feq_a(1, u_ref): (0, 0)
                              stores the offsets from the lattice weights; the
                              free-stream velocity keeps undisturbed regions near
                              zero (smaller rounding in FP32 / 16-bit storage);
                              |u_ref| < 0.3 */
} vplbm_config;

typedef struct {
  int32_t kind;            /* vplbm_body_kind */
  int32_t moving;          /* 1: integrate Eqs. dep1 and theta2 each step (disk only) */
  int32_t n_sim_points;    /* SIM points (0: disk ceil(2 pi R / 0.5), airfoil 849);
                              airfoil counts are odd */
  int32_t estimator;       /* vplbm_estimator driving a moving body */
  double length;           /* disk diameter D or chord C (lattice units) */
  double thickness;        /* NACA 4-digit thickness ratio t (0.12); ignored for a disk */
  double x_c, y_c;         /* disk centre, or airfoil pivot point */
  double angle;            /* airfoil angle of attack in radians, positive nose up;
                              disk: initial rotation angle */
  double pivot_chord_frac; /* airfoil pivot position along the chord (0.25) */
  double u[2];             /* rigid translational velocity */
  double omega;            /* rigid angular velocity (counter-clockwise) */
  double density_ratio;    /* rho_s / rho (moving body) */
  double gravity[2];       /* gravity acting on a moving body (Eq. dep1) */
} vplbm_body;

/* Device bytes a lattice with this configuration needs (population ping-pong
 * buffers, mask, outlet column, force partials, SIM points, histories).
 * Returns EINVAL for an invalid configuration (same checks as vplbm_create). */
vplbm_status vplbm_workspace_bytes(const vplbm_config *cfg, size_t *bytes);

/* Creates a lattice in the caller's device workspace (dev_workspace, at least
 * vplbm_workspace_bytes, 256-byte aligned) on the device that is current.
 * cuda_stream is a cudaStream_t (NULL: the legacy default stream).  EINVAL on
 * nx or ny < 3, tau+ <= 1/2, eta <= 0, a bad side combination or dtype;
 * ENOMEM when bytes is too small.  The lattice holds no body until
 * vplbm_set_body. */
vplbm_status vplbm_create(const vplbm_config *cfg, void *dev_workspace, size_t bytes,
                          void *cuda_stream, vplbm_ctx **out);

/* Replaces the stream used by later calls. */
vplbm_status vplbm_set_stream(vplbm_ctx *ctx, void *cuda_stream);

/* Places the body: rasterises chi (Eq. fcar: 1 on nodes inside or on the
 * body), builds the SIM polygon (Eq. defFf quadrature, points on the body
 * surface with their outward normals and lengths), resets the step counter,
 * force histories and averages, and sets the initial state f = feq(1, u0)
 * with u0 = u_in on fluid nodes and the rigid velocity on solid nodes.
 * kind NONE gives an empty lattice.  EINVAL when the body does not fit in
 * the lattice, n_sim_points exceeds the capacity, or a NACA body is moving.
 * The step graphs (vplbm_step) are kept when the new body has the same SIM
 * point count and constant part, force-region block count, motion and SIM
 * cadence as the old one (the same body placed again); otherwise they are
 * dropped and captured again at the next run.  Synchronises the stream. */
vplbm_status vplbm_set_body(vplbm_ctx *ctx, const vplbm_body *body);

/* Queues nsteps time steps (nsteps >= 0).  One step, for every node:
 * moments and penalized velocity (Eqs. updatestep .. updatestepm), force
 * density G = -rho (chi/eta)(u - u_s) + body force, equilibrium and
 * collision with the forcing term (Eq. TRT / BGK), streaming with the side
 * conditions (Eq. eqBd, Sec. 3.1); the MEM force of Eq. MMEL / Eq. fluidtorque
 * on the post-collision populations; the SIM force of Eq. defFf on the
 * pre-collision populations (when due); and, for a moving body, the FP64
 * rigid-body update of Eqs. dep1 / theta2 followed by re-rasterising chi.
 * Runs of steps are replayed from CUDA graphs of 1, 2, 4, ..., 32 steps,
 * captured (all of them, from either population buffer) at the first run
 * that can use one: when the lattice is past its first step and SIM runs
 * every step or never.  The call returns with the last step's forces in the
 * history. */
vplbm_status vplbm_step(vplbm_ctx *ctx, int32_t nsteps);

/* Captures and uploads, now, the step graphs that runs of nsteps steps use
 * (a run of more than 32 steps is replayed in 32-step graphs and one graph of
 * the remainder), so that the first run of that length pays for no capture
 * and replays one graph where it would otherwise replay several (20 steps:
 * one graph instead of 16 + 4).  No counterpart in the paper; it changes no
 * result.  The prepared length is kept until the context is destroyed (graphs
 * dropped by vplbm_set_body or a change of launch form are captured again at
 * the next run).  Synchronises the stream.  ESTATE before vplbm_set_body.
 * Lattices whose SIM runs on some steps only (sim_every > 1) queue their
 * steps one by one; the call does nothing for them. */
vplbm_status vplbm_prepare(vplbm_ctx *ctx, int32_t nsteps);

/* Force (F[0], F[1]) and torque (*T) of the last step from MEM (Eq. MMEL,
 * Eq. fluidtorque), host outputs.  Synchronises the stream.  ESTATE before the
 * first step; EUNSTABLE when the instability flag is set. */
vplbm_status vplbm_force_mem(vplbm_ctx *ctx, double F[2], double *T);

/* Same for SIM (Eq. defFf): the last step on which SIM was evaluated.
 * ESTATE when SIM has not run or a point found no fluid node. */
vplbm_status vplbm_force_sim(vplbm_ctx *ctx, double F[2], double *T);

/* Volume-integral force of the last step (Eq. Angotforce, Sec. 2.3): the
 * penalization force density reversed and summed over the solid nodes,
 * sum rho (chi/eta)(u - u_s) with u the penalized velocity of Eq.
 * updatestepm (the printed formula has lost its 1/eta), evaluated with the
 * collision of the step; torque about the body reference point.  Host
 * outputs; synchronises the stream.  ESTATE before the first step.  A
 * diagnostic: the paper reports that this estimator fails. */
vplbm_status vplbm_force_angot(vplbm_ctx *ctx, double F[2], double *T);

/* Queues a copy of the last step's forces into caller host memory without
 * waiting: out[6] = MEM (F_x, F_y, T) then SIM (F_x, F_y, T) (SIM entries are
 * NaN on steps where SIM was not evaluated).  out should be page-locked for
 * the copy to be asynchronous; it is valid once the stream has been
 * synchronised.  ESTATE before the first step. */
vplbm_status vplbm_forces_async(vplbm_ctx *ctx, double *out);

/* Last `count` per-step forces of one estimator (MEM, SIM or ANGOT), oldest first, host output
 * out[count][3] = (F_x, F_y, T).  EINVAL when count exceeds the history length
 * or the number of steps taken. */
vplbm_status vplbm_force_history(vplbm_ctx *ctx, int32_t estimator, int32_t count, double *out);

/* The last `count` history rows, queued into caller host memory without
 * waiting: out[count][9] = MEM (F_x, F_y, T), SIM (F_x, F_y, T; NaN on steps
 * without SIM), volume integral (F_x, F_y, T), oldest first.  out should be
 * page-locked for the copy to be asynchronous; it is valid once the stream
 * has been synchronised, and a later vplbm_step that wraps the ring past
 * these rows must be queued after the copy (the same stream orders it).
 * EINVAL when count exceeds the history length or the steps taken. */
vplbm_status vplbm_force_history_async(vplbm_ctx *ctx, int32_t count, double *out);

/* FP64 sums of (F_x, F_y, T) of both estimators since the last reset and the
 * number of steps summed (host outputs sums[6] = MEM then SIM, n[2]). */
vplbm_status vplbm_force_sums(vplbm_ctx *ctx, double sums[6], int64_t n[2]);
vplbm_status vplbm_reset_sums(vplbm_ctx *ctx);

/* Number of steps taken since vplbm_set_body (host output). */
vplbm_status vplbm_step_count(vplbm_ctx *ctx, int64_t *n);

/* Pre-collision populations f_a of the current time level (the streamed
 * field: Eq. eqBd's left-hand side) as FP64 into caller host memory
 * f[9][ny][nx].  Synchronises the stream.  The rows are staged a few at a
 * time in the population buffer that does not hold the state, so the call
 * needs no device memory beyond the workspace.  ESTATE before
 * vplbm_set_body. */
vplbm_status vplbm_get_f(vplbm_ctx *ctx, double *f);

/* Macroscopic fields of the current time level (Eqs. updatestep,
 * updatestepm: rho, and the penalized velocity u on solid nodes) as FP64 into
 * caller host memory rho[ny][nx], ux[ny][nx], uy[ny][nx].  Synchronises the
 * stream; staged as vplbm_get_f.  ESTATE before vplbm_set_body. */
vplbm_status vplbm_get_fields(vplbm_ctx *ctx, double *rho, double *ux, double *uy);

/* The same two read-backs into caller device memory (f_dev[9][ny][nx];
 * rho_dev, ux_dev, uy_dev [ny][nx] each), queued on the stream without
 * waiting. */
vplbm_status vplbm_get_f_dev(vplbm_ctx *ctx, double *f_dev);
vplbm_status vplbm_get_fields_dev(vplbm_ctx *ctx, double *rho_dev, double *ux_dev, double *uy_dev);

/* Overwrites the state from caller device FP64 buffers [9][ny][nx].
 * post_collision = 0: f_dev is the pre-collision field of the current time
 * level (prev_dev ignored).  post_collision = 1: f_dev is the post-collision
 * field of the previous level and prev_dev that level's pre-collision field
 * (only its x_hi column is read, for the convective outlet; may be NULL when
 * x_hi is not an outlet).  Converted to the storage form (16-bit forms round
 * to nearest even).  The step counter is kept.  Queued. */
vplbm_status vplbm_set_state(vplbm_ctx *ctx, const double *f_dev, const double *prev_dev,
                             int32_t post_collision);

/* Mask chi of the current time level (Eq. fcar: 1 on nodes inside or on
 * the body, 0 elsewhere) into caller host memory chi[ny][nx] bytes.
 * Synchronises the stream; staged as vplbm_get_f. */
vplbm_status vplbm_get_mask(vplbm_ctx *ctx, uint8_t *chi);

/* The mask into caller device memory chi_dev[ny][nx], queued. */
vplbm_status vplbm_get_mask_dev(vplbm_ctx *ctx, uint8_t *chi_dev);

/* ---- checkpoint and restart ----
 * No counterpart in the paper (its runs are single uninterrupted solves).
 * A snapshot holds everything a lattice continues from: the stored
 * populations of the current time level, the outlet columns, the mask, the
 * SIM polygon and its sampled nodes, the force histories, running sums and
 * counts, the step counter, the body and force-region states (FP64) and the
 * library's host-side bookkeeping, as raw bytes.  A lattice restored from it
 * continues bit for bit as the saved one would have: the same populations,
 * forces, body trajectory and sums, in every storage form, fixed or moving
 * body.
 *
 * vplbm_state_bytes: the snapshot size of this lattice (host output).
 * vplbm_save_state: writes the snapshot into caller host memory of at least
 *   that many bytes (the pending force sums are finalized first, so the
 *   history is complete); synchronises the stream.  ESTATE before
 *   vplbm_set_body; EINVAL when bytes is too small.
 * vplbm_load_state: restores a snapshot into this lattice, which may be the
 *   one it was taken from or another created with an identical
 *   configuration (any workspace address); the body placed by the snapshot
 *   replaces the current one.  Synchronises the stream.  EINVAL for a buffer
 *   that is not a snapshot of this library's format, or of a lattice with
 *   another configuration.  Step graphs are rebuilt at the next step. */
vplbm_status vplbm_state_bytes(vplbm_ctx *ctx, size_t *bytes);
vplbm_status vplbm_save_state(vplbm_ctx *ctx, void *host, size_t bytes);
vplbm_status vplbm_load_state(vplbm_ctx *ctx, const void *host, size_t bytes);

/* Body state (x_c, y_c, angle, u_x, u_y, omega), host output.  Synchronises. */
vplbm_status vplbm_get_body(vplbm_ctx *ctx, double state[6]);

/* Lattice node index j*nx + i sampled by each SIM point at its last
 * evaluation (-1: none), host output nodes[n_sim_points]; *n gets the count.
 * Synchronises. */
vplbm_status vplbm_get_sim_nodes(vplbm_ctx *ctx, int32_t *nodes, int32_t capacity, int32_t *n);

/* Latched device status: OK, EUNSTABLE or ETIMEOUT.  Synchronises. */
vplbm_status vplbm_check(vplbm_ctx *ctx);

/* Number of kernels the library has launched on this lattice so far. */
vplbm_status vplbm_launch_count(vplbm_ctx *ctx, int64_t *n);

/* ---- launch forms of the bulk kernel and their tuner ----
 * No counterpart in the paper.  The kernel that updates every node away
 * from the edges and the body comes in three launch forms which compute the
 * same values bit for bit: FP32/FP64 storage, blocks of one, two or four
 * 128 x 2 tiles; 16-bit storage, eight nodes per thread at 96 or 126
 * registers, or four nodes per thread.
 * Form 0 is the default.
 *
 * vplbm_autotune times the forms on this lattice's own steps: three passes
 * over the forms, each form running 32 untimed steps (its step graph is
 * captured there) and then `trials` steps timed with CUDA events on the
 * lattice's stream (1 <= trials <= 10000); each form's fastest pass counts.
 * It keeps the fastest form and writes its index to *variant (may be NULL).
 * The lattice advances by 9 * (32 + trials) steps, which give the same state,
 * histories and sums as vplbm_step of that count (the forms agree bit for
 * bit).  Synchronises the stream.  ESTATE before vplbm_set_body.  Step graphs
 * are rebuilt after a change of form; batches re-capture theirs at their
 * next step.
 *
 * vplbm_set_bulk_variant selects a form (0 .. 2, else EINVAL);
 * vplbm_bulk_variant reads the current one. */
vplbm_status vplbm_autotune(vplbm_ctx *ctx, int32_t trials, int32_t *variant);
vplbm_status vplbm_set_bulk_variant(vplbm_ctx *ctx, int32_t variant);
vplbm_status vplbm_bulk_variant(vplbm_ctx *ctx, int32_t *variant);

/* ---- batches: several lattices stepped together ----
 * A batch steps n independent lattices (any sizes and storage types, one
 * device).  The lattices share no data, so each runs its steps on a stream of
 * its own, forked from the batch's stream and joined back into it at the end
 * of every vplbm_batch_step: steps of different lattices overlap, and one
 * lattice's latency-bound work (force reductions, a moving body's update) runs
 * while others use the memory bandwidth.  Each lattice ends in the state, with
 * the force histories and sums, that stepping it alone would give.  Each
 * lattice's steps are replayed from its own step graphs (runs of 1, 2, 4, ...,
 * 32 steps, as vplbm_step replays them) where they apply, and the lattices
 * meet only at the end of the call, so that none waits for another between
 * runs; a step count prepared with vplbm_batch_prepare is one graph launch
 * holding every lattice's runs side by side.  The parameter studies of Sec. 4 (one lattice per angle of attack, per
 * estimator, per resolution) are such batches; the paper itself steps one
 * lattice at a time. */
typedef struct vplbm_batch vplbm_batch;

/* ctxs: host array of n >= 1 distinct contexts created on the current device.
 * The batch keeps the pointers: destroy it before any of its contexts.
 * cuda_stream: the stream the batch's steps are queued on; each
 * vplbm_batch_step first orders that stream after every lattice's own stream
 * and afterwards orders every lattice's own stream after it.  EINVAL for an
 * empty list, a NULL or repeated context, or a context of another device.
 * Failures of the batch calls are reported through vplbm_last_error(NULL). */
vplbm_status vplbm_batch_create(vplbm_ctx *const *ctxs, int32_t n, void *cuda_stream,
                                vplbm_batch **out);

/* Queues nsteps time steps (nsteps >= 0) of every lattice of the batch, each
 * step as vplbm_step defines it.  ESTATE when a lattice has no body placed
 * (nothing is queued then).  A vplbm_set_body on a member between calls is
 * seen by the next call. */
vplbm_status vplbm_batch_step(vplbm_batch *batch, int32_t nsteps);

/* vplbm_prepare for every lattice of the batch (the runs of a batch call are
 * at most 32 steps per lattice; each graph is uploaded on its lattice's chain
 * stream).  It also builds a call of nsteps steps as one graph: every
 * lattice's run of step graphs as a chain of child graphs, the chains side by
 * side, for the lattices' current buffers and for the other ones (where they
 * stand after an odd step count).  A later vplbm_batch_step of nsteps steps
 * is then one graph launch on the batch's stream, as long as every lattice
 * starts from a buffer it was built for and none of the step graphs was
 * rebuilt since (vplbm_set_body, vplbm_load_state, a change of launch form);
 * other calls take the per-lattice path, with the same results.  At most
 * eight such graphs are kept per batch.  Synchronises.  ESTATE when a
 * lattice has no body placed. */
vplbm_status vplbm_batch_prepare(vplbm_batch *batch, int32_t nsteps);

/* The bulk kernel's launch form per lattice of the batch, timed on the
 * batch's own steps.  Lattices of one size (nx, ny) and storage type form a
 * class and share a form.  Three passes visit the classes in turn; for one
 * class every form runs 32 untimed batch steps (its step graphs are captured
 * there) and then `trials` batch steps timed with CUDA events on the batch's
 * stream (1 <= trials <= 10000), the other classes held at their current
 * forms, and the class keeps the form with the fastest time seen so far.
 * With one class this is vplbm_autotune on the whole batch.  The batch
 * advances by 9 * G * (32 + trials) steps (G classes), which give every
 * lattice the state, histories and sums of that many vplbm_batch_step steps
 * (the forms agree bit for bit).  variants: host array of n entries that
 * receives each lattice's form, in the order of vplbm_batch_create (may be
 * NULL).  Synchronises the batch's stream.  ESTATE when a lattice has no body
 * placed. */
vplbm_status vplbm_batch_autotune(vplbm_batch *batch, int32_t trials, int32_t *variants);

/* Releases the batch (never its contexts).  NULL is accepted. */
void vplbm_batch_destroy(vplbm_batch *batch);

/* The SIM force (F[0], F[1], T about ref) of a state the caller supplies,
 * computed without any device allocation by the caller or the library.  For
 * callers that cannot allocate device memory: code embedded in a host
 * application whose allocator has already claimed the device memory, or
 * latency-bound callers that cannot afford the device-wide synchronisation
 * that cudaMalloc and cudaFree imply.  No counterpart in the paper: it
 * evaluates the same SIM sum as vplbm_step (nearest node, or both nodes of an
 * exact tie, walk along the lattice direction closest to the normal to the
 * first fluid node, stress averaged over the candidates, summed in point
 * order in FP64) on the inputs given here.
 *   cfg     nx, ny, tau_plus and body_force are used; sim_order must be 0 (the
 *           stress copied from the sampled node, as Sec. 2.3.2 describes;
 *           EINVAL otherwise);
 *   f_dev   device, FP64 pre-collision populations [9][ny][nx];
 *   chi_dev device, mask [ny][nx] (0 fluid, nonzero solid);
 *   pts     host, n_pts rows (x - ref_x, y - ref_y, n_x, n_y, S);
 *   ref     host, the reference point; out host, (F_x, F_y, T).
 * The scratch is one fixed device array in the library of
 * 8 * (8 + 4096) doubles (256 KiB), held by every GPU that loads the library
 * until the process exits: n_pts above 4096 is rejected with EINVAL.  Every
 * call takes that array's device address with the device current
 * (cudaGetSymbolAddress, which allocates nothing); the first call on a device
 * also loads the library's device code there, so make it before any stream
 * capture.  Every call uses the same array and leaves its contents behind
 * (the call clears what must start at zero), so calls whose GPU work
 * overlaps -- on two streams or from two threads -- race.  Synchronises
 * cuda_stream; ESTATE when a point finds no fluid node (out then sums the
 * other points); the text of a failure is vplbm_last_error(NULL). */
vplbm_status vplbm_sim_force_static(const vplbm_config *cfg, const double *f_dev,
                                    const uint8_t *chi_dev, int32_t n_pts, const double *pts,
                                    const double ref[2], double out[3], void *cuda_stream);

/* Releases the host-side context; never touches the caller's workspace.
 * NULL is accepted. */
void vplbm_destroy(vplbm_ctx *ctx);

/* Text of the last failure on ctx (never NULL; "" when none).  ctx may be
 * NULL for failures of vplbm_create / vplbm_workspace_bytes. */
const char *vplbm_last_error(const vplbm_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* VPLBM_H */
