/*
 * plbm.h - C ABI of the GB300 (sm_103a) parametric lattice Boltzmann solver.
 *
 * Method: J. W. Shim, "Parametric Lattice Boltzmann Method" (arXiv:1402.5487).
 *   f^eq_i = rho r_i                                  (Eq. eq:eqdist)
 *   r_i    = sum_{j=1}^{q} c_ij mu_{j-1}              (Eq. eq:rdr)
 *   c_ij   = coefficient of v^{j-1} in the Lagrange polynomial through
 *            (v_k, delta_ik); C = V^{-1}, V_{n,k} = v_k^n   (Appendix)
 *   mu_n   = n-th moment of the Maxwell-Boltzmann distribution (Appendix)
 *   2D     : tensor product of 1D rules (Sec. 2.1)
 *   step   : f_i(x + v_i, t + 1) = (1 - omega) f_i(x, t) + omega f^eq_i(x, t)
 *            (Eq. eq:srt, lattice units dx = dt = 1)
 *
 * Conventions shared by every call:
 *   - Lattice units.  Velocities are integers (on-lattice sets, Sec. 2.4).
 *   - Field arrays are FP64, row-major [ny][nx] (ny = 1 in 1D).
 *   - Population arrays at the boundary are FP64 [q][ny][nx], q = q1^dim,
 *     population p = ix*q1 + iy has velocity (v[ix], v[iy]) in 2D, p = ix in 1D.
 *   - The stored state is the post-collision state; a step is "pull-stream,
 *     then collide", which yields the same sequence of states as Eq. (eq:srt).
 *   - Moments: rho = sum f, rho u = sum v f, d rho theta = sum |v - u|^2 f.
 *   - The caller owns every array it passes.  The handle owns its device
 *     populations unless a workspace was supplied in the descriptor.
 *   - Calls are asynchronous on the handle's stream, except those that return
 *     host data or a status read from the device (documented per call).
 *   - Every call returns a plbm_status.  Errors are sticky per handle: after
 *     PLBM_E_DIVERGED or PLBM_E_CUDA only plbm_destroy, plbm_get_populations,
 *     plbm_last_error and plbm_diagnostics are accepted.
 *   - Thread safety: a handle must not be used from two threads at once.
 *   - No call falls back to the CPU: without a usable CUDA device,
 *     plbm_create returns PLBM_E_CUDA.
 */
#ifndef PLBM_H
#define PLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PLBM_ABI_VERSION 2
#define PLBM_MAX_Q1 8

typedef struct plbm_s *plbm_handle;

typedef enum {
    PLBM_OK = 0,
    PLBM_E_ARG = -1,           /* invalid argument or descriptor */
    PLBM_E_CUDA = -2,          /* a CUDA runtime call failed */
    PLBM_E_INADMISSIBLE = -3,  /* r_i < 0 for the requested state (Sec. 3.1) */
    PLBM_E_DIVERGED = -4,      /* non-finite, rho <= 0 or theta <= 0 seen on the device */
    PLBM_E_TIMEOUT = -5,       /* a bounded device-side wait ran out */
    PLBM_E_STATE = -6,         /* call not valid in the handle's state */
    PLBM_E_CHECKSUM = -7,      /* checkpoint checksum or header mismatch */
    PLBM_E_NOMEM = -8          /* device allocation failed or workspace too small */
} plbm_status;

/* Storage precision of the populations.  F64 stores f itself and does the
 * arithmetic in FP64.  F32, F16DEV and BF16DEV store the deviation
 * g = f - w0 from the rest equilibrium w0 = f^eq(rho = 1, u = 0, theta0) in
 * 32 or 16 bits and do the arithmetic in FP32. */
typedef enum { PLBM_F64 = 0, PLBM_F32 = 1, PLBM_F16DEV = 2, PLBM_BF16DEV = 3 } plbm_prec;

/* PERIODIC: periodic in every direction.  FIXED_ENDS: nodes left of x = 0 and
 * right of x = nx-1 hold f^eq(left_state) and f^eq(right_state) for ever (the
 * shock-tube ends "maintained by C_L and C_R", Sec. 3.2); y stays periodic. */
typedef enum { PLBM_PERIODIC = 0, PLBM_FIXED_ENDS = 1 } plbm_bc;

/* Descriptor flags. */
#define PLBM_FLAG_ISOTHERMAL 0x1u      /* theta in f^eq held at theta0 (Eq. eq:1d3v models) */
#define PLBM_FLAG_SKIP_ADMISSIBILITY 0x2u /* do not run the positivity gate at create */
#define PLBM_FLAG_PLAIN_LAYOUT 0x4u    /* 2D: keep the plain layout [q][ny][pitch] (one node per
                                          thread) where the row-paired one would be taken */

typedef struct {
    int dim;                   /* 1, 2 or 3 */
    int q1;                    /* velocities per axis: 3..8 in 1D and 2D (D1Q3..D1Q8,
                                  D2Q9..D2Q64; n* = q1 - 1 moments reproduced), 3..5 in 3D
                                  (D3Q27..D3Q125) */
    const int *v;              /* q1 distinct integer velocities (copied at create) */
    double omega;              /* BGK relaxation constant, 0 < omega < 2 */
    double theta0;             /* reference temperature (rest state, isothermal models) */
    int nx, ny;                /* grid; ny must be 1 when dim == 1 */
    plbm_prec prec;
    plbm_bc bc;
    const double *left_state;  /* (rho, u, theta) at the left end, FIXED_ENDS only */
    const double *right_state; /* (rho, u, theta) at the right end, FIXED_ENDS only */
    void *stream;              /* cudaStream_t for every launch; NULL = default stream */
    unsigned flags;            /* PLBM_FLAG_* */
    int check_every;           /* plbm_step reads the device status every this many
                                  steps and at its end (0 = never inside plbm_step) */
    double u_max;              /* positivity gate: r_i >= 0 required for |u| <= u_max
                                  at theta0 (0 = check the rest state only) */
    void *workspace;           /* optional caller-owned device memory of at least
                                  plbm_workspace_bytes(desc) bytes, 256-byte aligned;
                                  NULL = the handle allocates its own */
    size_t workspace_bytes;
    int device;                /* CUDA device ordinal */
    int nz;                    /* nodes along z when dim == 3 (Sec. 2.1's tensor product
                                  in three dimensions: periodic only; 16/32-bit storage
                                  needs a thermal set v = (0, a, -a, b, -b), FP64 takes
                                  any); ignored for dim 1 and 2 */
} plbm_desc;

/* Global diagnostics of the stored state, all accumulated in FP64. */
typedef struct {
    double mass;      /* sum over nodes of rho */
    double jx, jy;    /* sum of rho u */
    double energy;    /* sum of sum_p |v_p|^2 f_p  (= sum of d rho theta + rho |u|^2) */
    double rho_min, theta_min;
    uint32_t status;  /* PLBM_STATUS_* bits seen since create */
    int64_t steps;    /* steps taken since create (or since the last set_populations) */
} plbm_diag;

#define PLBM_STATUS_NONFINITE 0x1u
#define PLBM_STATUS_RHO_NONPOS 0x2u
#define PLBM_STATUS_THETA_NONPOS 0x4u

/* Library and ABI version; never fails. */
int plbm_abi_version(void);

/* Coefficients c_ij of Eq. (eq:rdr) for a velocity set, in FP64, computed on
 * the host by expanding the Lagrange polynomials of the Appendix
 * (C = V^{-1}).  C_out: q1*q1 doubles, C_out[i*q1 + n] multiplies mu_n in r_i.
 * Errors: PLBM_E_ARG for q1 out of range or repeated velocities. */
plbm_status plbm_coefficients(int q1, const int *v, double *C_out);

/* Positivity range of Sec. 3.1 for the lattice described by desc: *min_r =
 * min over i and over |u| <= u_max (401 samples along one axis) of r_i(u, theta0)
 * (Eq. eq:rdr).  The rule is admissible there when *min_r >= 0; plbm_create runs
 * the same test with desc->u_max.  Host computation (no GPU). */
plbm_status plbm_positivity(const plbm_desc *desc, double u_max, double *min_r);

/* Linear (von Neumann) stability of the lattice described by desc around the
 * uniform state f^eq(rho = 1, u = (ux, 0), theta0): the largest |lambda| of the
 * one-step operator A(k) = J S(k) over the wave vectors k = 2 pi (a, b) / nk,
 * where S(k) = diag(exp(-i k.v_p)) is the pull of Eq. (eq:srt) and J the
 * Jacobian of its BGK collision with the equilibrium of Eq. (eq:rdr) (exact to
 * rounding, complex-step).  The lattice is linearly stable there when the
 * result is <= 1 (up to rounding: conserved modes sit at exactly 1).  Both
 * k axes are also scanned at 8 nk points (narrow unstable bands of tensor-
 * product lattices lie there).  For symmetric velocity sets only
 * 0 <= k_y <= pi is scanned (mirror symmetry).
 * stop_above > 0 lets the scan stop at the first |lambda| above that value (the
 * result is then a lower bound above it); 0 scans every k.  Host computation
 * (no GPU), multithreaded over k.  Used to screen parameter draws of batched
 * sweeps.  Errors: PLBM_E_ARG for an invalid descriptor, nk outside 1..256 or
 * a non-finite ux. */
plbm_status plbm_linear_stability(const plbm_desc *desc, double ux, int nk, double stop_above,
                                  double *max_abs_lambda);

/* Device bytes a handle with this descriptor needs (two population arrays,
 * reduction scratch, status words).  Returns 0 for an invalid descriptor. */
size_t plbm_workspace_bytes(const plbm_desc *desc);

/* Create a solver (Secs. 2-4).  Validates the descriptor, computes c_ij in FP64
 * on the host, runs the positivity gate of Sec. 3.1 (every r_i(u, theta0) >= 0
 * for |u| <= desc->u_max along each axis, unless PLBM_FLAG_SKIP_ADMISSIBILITY),
 * and allocates or adopts device memory.  Populations are undefined until
 * plbm_init or plbm_set_populations.  Synchronous.
 * Errors: PLBM_E_ARG, PLBM_E_INADMISSIBLE, PLBM_E_NOMEM, PLBM_E_CUDA; *out is
 * NULL on error and the reason is available from plbm_last_error(NULL). */
plbm_status plbm_create(const plbm_desc *desc, plbm_handle *out);

/* Release the handle and the memory it owns.  Accepts NULL.  Synchronises the
 * handle's stream. */
plbm_status plbm_destroy(plbm_handle h);

/* Initial state f = f^eq(rho, u, theta) at every node (Eq. eq:eqdist), computed
 * on the device and stored in the handle's precision: in FP64, except for
 * FP32/FP16/BF16 handles with a symmetric five-velocity set (0, +-a, +-b), which
 * evaluate f^eq - w0 in the FP32 deviation arithmetic of their own collision
 * from rho - 1, u and theta - theta0 (formed in FP64).  Fields: FP64 [ny][nx];
 * uy may be NULL in 1D; theta may be NULL for isothermal handles.
 * on_device != 0: the pointers are device memory, read on the handle's stream
 * (asynchronous); otherwise host memory, copied before return (through a
 * staging buffer of 4 nx ny doubles that the handle keeps after first use, in
 * row bands whose copies overlap the kernel).  Resets the step counter and
 * the status word, then checks the fields on the device: a non-finite value,
 * rho <= 0 or theta <= 0 sets the matching PLBM_STATUS_* bit.  With host
 * pointers plbm_init then returns PLBM_E_ARG and leaves the handle
 * uninitialised; with device pointers (asynchronous) the next plbm_check, or
 * plbm_step with check_every > 0, returns PLBM_E_DIVERGED. */
plbm_status plbm_init(plbm_handle h, const double *rho, const double *ux, const double *uy,
                      const double *theta, int on_device);

/* Advance n >= 0 steps of Eq. (eq:srt) (pull-stream + BGK collision of the
 * equilibrium of Eq. eq:rdr).  Asynchronous unless check_every > 0, in which
 * case the device status is read (with a stream synchronisation) every
 * check_every steps and at the end; a set status returns PLBM_E_DIVERGED.
 * Lattices of at most 2^18 nodes, whose steps are too short to hide the
 * launches, advance by replays of a CUDA graph of 32 steps (captured at first
 * use on a private stream, launched on the handle's stream; not when
 * check_every > 0 or while the handle's stream is being captured). */
plbm_status plbm_step(plbm_handle h, long n);

/* Read the device status word (synchronises the stream).  Returns
 * PLBM_E_DIVERGED if any PLBM_STATUS_* bit has been set. */
plbm_status plbm_check(plbm_handle h);

/* Macroscopic fields of the stored state: rho, u_x, u_y, theta as FP64
 * [ny][nx] (uy may be NULL).  FP32/FP16/BF16 handles sum their stored
 * deviations in float-float arithmetic (~2^-48 relative), then form the fields
 * in FP64.  on_device != 0: device pointers, asynchronous; otherwise host
 * pointers, synchronous (the staging buffer of plbm_init). */
plbm_status plbm_moments(plbm_handle h, double *rho, double *ux, double *uy, double *theta,
                         int on_device);

/* Global FP64 sums and extrema of the stored state plus the status word.
 * Synchronous. */
plbm_status plbm_diagnostics(plbm_handle h, plbm_diag *out);

/* Advance n >= 1 steps as plbm_step does, the last one fused with the
 * reductions of plbm_diagnostics (the step kernel's blocks form the FP64 partial
 * sums of the moments it computes anyway: mass, momentum and energy are those of
 * the state after the step, as collision conserves them; the minima are of the
 * pulled state's rho and theta).  Synchronous.  3D handles take plbm_step and
 * plbm_diagnostics.  Errors: those of plbm_step; PLBM_E_ARG for n < 1. */
plbm_status plbm_step_diagnostics(plbm_handle h, long n, plbm_diag *out);

/* Conserved sums out[4] = (mass, jx, jy, energy) of the stored state, FP64.
 * Synchronous.  (3D handles: plbm_conserved3.) */
plbm_status plbm_conserved(plbm_handle h, double out[4]);

/* Three-dimensional handles (dim == 3, Sec. 2.1: f^eq = rho r^x r^y r^z with one
 * theta; theta = (sum |v|^2 f / rho - |u|^2) / 3).  Fields are FP64
 * [nz][ny][nx]; populations [q][nz][ny][nx] with q = q1^3 and p = (a q1 + b) q1 + c
 * for the velocity (v[a], v[b], v[c]).  plbm_init, plbm_moments and
 * plbm_conserved return PLBM_E_ARG for 3D handles; these take their place.
 * on_device as in plbm_init / plbm_moments, with the same check of the fields. */
plbm_status plbm_init3(plbm_handle h, const double *rho, const double *ux, const double *uy, const double *uz,
                       const double *theta, int on_device);
plbm_status plbm_moments3(plbm_handle h, double *rho, double *ux, double *uy, double *uz, double *theta,
                          int on_device);
/* out[5] = (mass, jx, jy, jz, energy) of the stored state, FP64.  Synchronous. */
plbm_status plbm_conserved3(plbm_handle h, double out[5]);

/* Populations as FP64 [q][ny][nx] ([q][nz][ny][nx] in 3D; for F16DEV/BF16DEV:
 * w0 + g).  on_device as in plbm_moments. */
plbm_status plbm_get_populations(plbm_handle h, double *f, int on_device);

/* Replace the stored state with FP64 populations [q][ny][nx], rounded to the
 * handle's precision.  Resets the step counter to `step`. */
plbm_status plbm_set_populations(plbm_handle h, const double *f, int on_device, int64_t step);

/* Checkpoint and resume.  A checkpoint is a header (format version, ABI
 * version, dim, q1, velocities, omega, theta0, sizes, storage precision and
 * layout, a digest of the fixed-end states, step counter) followed by the
 * stored population array byte for byte, in the handle's own precision and
 * layout, so that resuming continues bit for bit as if uninterrupted.  A
 * 64-bit FNV-1a checksum covers header and payload.
 * plbm_checkpoint_bytes: size of a checkpoint of h (0 for NULL).
 * plbm_checkpoint_save: writes it to host memory buf (bytes >= that size);
 *   synchronous.  Errors: PLBM_E_ARG, PLBM_E_STATE (not initialised).
 * plbm_checkpoint_load: replaces h's state and step counter from buf after
 *   verifying the checksum and that the header describes h's lattice; the
 *   status word is reset.  Synchronous.  PLBM_E_CHECKSUM for a corrupted or
 *   truncated checkpoint or one of another lattice (nothing is changed). */
size_t plbm_checkpoint_bytes(plbm_handle h);
plbm_status plbm_checkpoint_save(plbm_handle h, void *buf, size_t bytes);
plbm_status plbm_checkpoint_load(plbm_handle h, const void *buf, size_t bytes);

/* Descriptor facts of a live handle. */
plbm_status plbm_get_info(plbm_handle h, int *q, int *pitch, size_t *population_bytes);

/* Raw device pointer of the current population array (storage layout
 * [q][ny][pitch] in the handle's precision).  For profiling and tests. */
plbm_status plbm_device_populations(plbm_handle h, void **ptr);

/* ------------------------------------------------------------------------
 * Batched runner: many independent lattices advanced together.
 * The paper runs one lattice at a time; batching is a throughput service for
 * parameter sweeps over its models.  Each instance is an ordinary handle
 * (plbm_batch_instance) for init, moments, diagnostics and checkpoints; the
 * batch advances all of them with one of four launch schemes:
 *   PLBM_BATCH_PERSISTENT           one persistent launch per step and group of
 *                                   instances (CTAs walk a global tile list;
 *                                   per-instance parameters in a device table);
 *   PLBM_BATCH_PERSISTENT_GRAPH     the same, two steps per CUDA graph replay;
 *   PLBM_BATCH_PER_INSTANCE         one launch per instance per step;
 *   PLBM_BATCH_PER_INSTANCE_GRAPH   the same, captured in a CUDA graph.
 * All four give bit-identical populations.
 * ------------------------------------------------------------------------ */
typedef struct plbm_batch_s *plbm_batch;

#define PLBM_BATCH_PERSISTENT 0
#define PLBM_BATCH_PERSISTENT_GRAPH 1
#define PLBM_BATCH_PER_INSTANCE 2
#define PLBM_BATCH_PER_INSTANCE_GRAPH 3

/* Create n instances from n descriptors (one device; each a 2D lattice that
 * passes plbm_create's checks, with 3 to 5 velocities per axis unless it takes
 * the row-paired layout).  Instances may differ in size, velocity set, omega,
 * theta0, storage precision, boundary and model (thermal or isothermal).  The
 * batch advances them in groups, one persistent launch per group and step:
 * periodic thermal lattices with v = (0, a, -a, b, -b) and FP32/FP16/BF16
 * storage by the kernel of the row-paired layout, one group per precision
 * (even ny: a node pair per thread; odd ny: the plain layout, one node per
 * thread, same arithmetic); all others (FP64 storage, isothermal models, other
 * velocity sets) by a one-node-per-thread kernel, one group per (precision, q1).
 * One device allocation holds all instances' populations; descs[i].workspace
 * and .stream are ignored.  stream: cudaStream_t for every launch (NULL: the
 * batch creates its own non-blocking stream, as graph capture cannot use the
 * legacy default stream).  Synchronous. */
plbm_status plbm_batch_create(const plbm_desc *descs, int n, void *stream, plbm_batch *out);

/* How the batch splits: instances in the five-velocity thermal 16/32-bit groups
 * (row-paired or plain layout), instances in the other groups, and persistent
 * launches per step (one per group). */
plbm_status plbm_batch_groups(plbm_batch b, int *paired_instances, int *plain_instances, int *launches_per_step);

/* Release the batch, its instances and its memory.  Accepts NULL. */
plbm_status plbm_batch_destroy(plbm_batch b);

/* Handle of instance i (owned by the batch; plbm_destroy refuses it). */
plbm_status plbm_batch_instance(plbm_batch b, int i, plbm_handle *h);

/* Advance every instance n steps (Eq. eq:srt) with launch scheme `mode`.  All
 * instances must be initialised and at the same step parity.  Asynchronous. */
plbm_status plbm_batch_step(plbm_batch b, long n, int mode);

/* Read every instance's status word (synchronous).  PLBM_E_DIVERGED names the
 * first bad instance in *first_bad (else -1). */
plbm_status plbm_batch_check(plbm_batch b, int *first_bad);

/* Launch shape of the row-paired persistent kernel: block_x in {64, 128, 256}
 * threads (one tile = block_x node pairs of one pair row), ctas_per_sm
 * persistent CTAs per SM (0 = as many as fit).  The plain-layout groups always
 * take 128-node tiles and as many CTAs as fit. */
plbm_status plbm_batch_set_config(plbm_batch b, int block_x, int ctas_per_sm);

/* Order in which the persistent CTAs take the tiles (all instances' tiles form
 * one list, instance by instance, pair row by pair row).  CONTIGUOUS: CTA c takes
 * the range [c T / G, (c + 1) T / G) of the T tiles (G CTAs) and reloads an
 * instance's parameters only at the few instance boundaries it meets.
 * INTERLEAVED (default): CTA c takes tiles c, c + G, c + 2G, ..., so the tiles in
 * flight at any moment are neighbours in memory, as in a plain grid; the
 * instance of each tile comes from a per-tile table.  Errors: PLBM_E_ARG. */
#define PLBM_BATCH_ORDER_CONTIGUOUS 0
#define PLBM_BATCH_ORDER_INTERLEAVED 1
plbm_status plbm_batch_set_order(plbm_batch b, int order);
/* Current order, or -1 for a NULL batch. */
int plbm_batch_get_order(plbm_batch b);

/* Current launch shape and the occupancy limit for it. */
plbm_status plbm_batch_info(plbm_batch b, int *ninst, int *total_tiles, int *block_x, int *ctas,
                            int *max_ctas_per_sm);

/* Autotuner: times steps_per_trial persistent steps for both orders, every
 * block_x and every ctas_per_sm up to the occupancy limit and keeps the
 * fastest (plbm_batch_get_order reads the order it chose).  It advances the
 * instances (initialise them again afterwards if the state matters). */
plbm_status plbm_batch_tune(plbm_batch b, int steps_per_trial, int *best_block_x, int *best_ctas_per_sm,
                            double *best_ms_per_step);

/* Text of the last error of the batch (or of the calling thread when NULL). */
const char *plbm_batch_last_error(plbm_batch b);

/* ------------------------------------------------------------------------
 * Learned surrogate (not in the paper; a throughput service around its solver,
 * which generates the training data and stays the fallback and the reference).
 * A 6-layer 3x3 CNN with circular padding, channels 4 -> 64 -> 64 -> 64 -> 64
 * -> 64 -> 4, ReLU after the first five layers, BF16 weights and activations
 * with FP32 accumulation, maps the normalised fields (rho, u_x, u_y, theta)
 * of a periodic H x W lattice to the normalised change of those fields over K
 * lattice steps.  FP32 master weights, Adam, mean squared error.
 * Tensors are NHWC on the device: network input bf16 [B][H][W][4], targets and
 * outputs fp32 [B][H][W][4].  W must be a multiple of 128.
 * ------------------------------------------------------------------------ */
typedef struct plbm_surrogate_s *plbm_surrogate;

/* Number of FP32 parameters; flat layout per layer W[3][3][cin][cout], b[cout]. */
int plbm_sur_num_params(void);

/* Network for batches of up to max_batch lattices of H x W nodes, He-initialised
 * from `seed` (last layer scaled by 0.1).  stream: cudaStream_t (NULL: own).
 * PLBM_E_ARG unless 1 <= max_batch <= 65535, H >= 3 and W is a multiple of 128. */
plbm_status plbm_sur_create(int max_batch, int H, int W, unsigned long long seed, void *stream,
                            plbm_surrogate *out);
plbm_status plbm_sur_destroy(plbm_surrogate s);

/* Options: PLBM_SUR_OPT_TENSOR_PATH selects the kernels of the 64 -> 64
 * convolutions, their backward-data passes and their weight gradients: 1
 * (default) tcgen05.mma with tensor-memory accumulators, 0 mma.sync (kept as a
 * cross-check). */
#define PLBM_SUR_OPT_TENSOR_PATH 1
/* PLBM_SUR_OPT_CONSERVE: 1 shifts each lattice's predicted conserved densities
 * (rho, rho u, E = rho (d theta + |u|^2)) uniformly so that their totals equal
 * those of the old fields before the drift gate of plbm_sur_advance, which then
 * only rejects non-finite or non-positive predictions (and FP32 rounding);
 * 0 (default) gates the network's own prediction. */
#define PLBM_SUR_OPT_CONSERVE 2
/* PLBM_SUR_OPT_WAIT_NS: budget in nanoseconds (>= 1; default 2 x 10^9) of each
 * bounded wait of the tcgen05 kernels (a warp waiting for staged inputs, for
 * an accumulator or for a free buffer).  A wait that runs out makes the kernel
 * stop issuing work, wait for the MMAs and copies it issued (a fixed bound of
 * 2 s, whatever this budget), free its tensor memory and return, and sets the
 * flag plbm_sur_check reads; the results of that pass are then invalid.  A
 * budget of a few nanoseconds makes the waits of the next pass run out, which
 * exercises this path without a fault. */
#define PLBM_SUR_OPT_WAIT_NS 3
plbm_status plbm_sur_set_option(plbm_surrogate s, int option, int value);

/* PLBM_E_TIMEOUT if a bounded wait of a tensor-core kernel ran out since the
 * last call; the flag is cleared once reported (synchronous). */
plbm_status plbm_sur_check(plbm_surrogate s);

/* Replace (host FP32, resets Adam) or read the parameters and the last gradients. */
plbm_status plbm_sur_set_params(plbm_surrogate s, const float *params);
plbm_status plbm_sur_get_params(plbm_surrogate s, float *params, float *grads);

/* Per-field normalisation: input (x - mean_in) / std_in, target
 * (x_{t+K} - x_t - mean_d) / std_d.  Four values each, host memory. */
plbm_status plbm_sur_set_norm(plbm_surrogate s, const float *mean_in, const float *std_in, const float *mean_d,
                              const float *std_d);

/* Forward pass of B samples; out (device fp32, may be NULL) receives the output. */
plbm_status plbm_sur_forward(plbm_surrogate s, int B, const void *x, float *out);

/* Forward and backward pass for the upstream gradient dout (device fp32) of the
 * output; the gradients are then read with plbm_sur_get_params. */
plbm_status plbm_sur_backward(plbm_surrogate s, int B, const void *x, const float *dout);

/* Copy a stored tensor of the last pass for B samples to dst (device):
 * kind 0: output of layer 1..5 (bf16 [B][H][W][64], after ReLU) or 6 (fp32
 * [B][H][W][4]); kind 1 (after a backward pass): gradient of the loss with
 * respect to the convolution output of layer 1..5 (bf16 [B][H][W][64]).
 * Synchronous. */
plbm_status plbm_sur_copy(plbm_surrogate s, int kind, int layer, int B, void *dst);

/* Training loss = mean squared error + lambda x mean over samples and fields of
 * the squared lattice-mean error (the mean over all pixels of prediction minus
 * target).  The second term aims the network at the global sums the drift gate
 * of plbm_sur_advance checks.  lambda >= 0 (default 0); PLBM_E_ARG otherwise. */
plbm_status plbm_sur_set_mean_penalty(plbm_surrogate s, float lambda);

/* One Adam step on the training loss (above) against target.  loss (host, may be
 * NULL) receives its mean squared error part, which synchronises the stream. */
plbm_status plbm_sur_train_step(plbm_surrogate s, int B, const void *x, const float *target, float lr,
                                float *loss);

/* FP32 NHWC fields [n][4] from four FP64 planes (device). */
plbm_status plbm_sur_pack_fields(const double *rho, const double *ux, const double *uy, const double *theta,
                                 long long n, float *out, void *stream);

/* Training batch from a stack of field snapshots (device fp32 [S][npix][4]):
 * for b < B with pairs[2b] = s0, pairs[2b+1] = s1 (device int32), x[b] is the
 * normalised snapshot s0 (bf16) and y[b] the normalised change s1 - s0 (fp32). */
plbm_status plbm_sur_assemble(plbm_surrogate s, const float *snaps, long long npix, const int *pairs, int B,
                              void *x, float *y);

/* The same with sigma x a standard normal number added to every normalised input
 * element before its bf16 rounding (training on inputs perturbed like the
 * network's own predictions keeps repeated advances stable).  The numbers come
 * from a counter-based generator: element e = 4 (b npix + pixel) + field draws
 * SplitMix64(seed xor SplitMix64(e)) (SplitMix64: z += 0x9e3779b97f4a7c15,
 * z = (z ^ z >> 30) 0xbf58476d1ce4e5b9, z = (z ^ z >> 27) 0x94d049bb133111eb,
 * z ^ z >> 31), whose bits 40..63 and 16..39 give u1 = (k + 1) / 2^24 and
 * u2 = k / 2^24, and Box-Muller sqrt(-2 ln u1) cos(2 pi u2).  sigma = 0: no
 * noise.  PLBM_E_ARG for a negative or non-finite sigma. */
plbm_status plbm_sur_assemble_noise(plbm_surrogate s, const float *snaps, long long npix, const int *pairs, int B,
                                    void *x, float *y, float sigma, unsigned long long seed);

/* Advance n lattices (handles of H x W periodic 2D lattices, 16/32/64-bit
 * storage) by K steps with the network: fields from the populations, predicted
 * change, and the FP64 global drift of mass, energy (relative) and momentum
 * (relative to 0.1 x mass) between the old and the predicted fields.  Drift <=
 * tol: the populations are rebuilt by Chapman-Enskog reconstruction (f^eq plus
 * -((1 - omega) / omega) D f^eq with Euler time derivatives, projected so the
 * conserved moments equal the predicted fields) and the step counter advances
 * by K.  Otherwise (or for a non-finite prediction) the lattice runs K ordinary
 * steps (Eq. eq:srt); fallback lattices in the row-paired layout of one
 * precision take them together, one persistent launch per step, without the
 * check_every status reads of plbm_step (plbm_check reads the status).
 * fell_back[b] (host, may be NULL) reports which.  Synchronous up to the drift
 * read; the lattices' streams are ordered after the work it queues. */
plbm_status plbm_sur_advance(plbm_surrogate s, plbm_handle *hs, int n, int K, double tol, int *fell_back);

/* Drift values (as defined for plbm_sur_advance) of the first n lattices of the
 * last advance, into out[n] (host).  PLBM_E_ARG if n exceeds that advance's
 * lattice count. */
plbm_status plbm_sur_last_drift(plbm_surrogate s, double *out, int n);

/* Text of the last error of s (or of the calling thread when NULL). */
const char *plbm_sur_last_error(plbm_surrogate s);

/* ------------------------------------------------------------------------
 * Domain decomposition along y.  A step of Eq. (eq:srt) (pull, then the local
 * BGK collision) reads a node's populations from at most w = max|v| rows away
 * (integer velocities, Sec. 2.4), so a slab of consecutive rows advances on its
 * own once the w rows on each side of it hold its neighbours' current state:
 * the rows below it are read only by populations with v_y > 0, the rows above
 * only by those with v_y < 0.
 * ------------------------------------------------------------------------ */

/* Rows of slab k when ny rows are split into nslabs slabs as evenly as
 * possible (the first ny mod nslabs slabs take one row more): rows y0 ..
 * y0 + rows - 1.  Host computation.  PLBM_E_ARG unless 1 <= nslabs <= ny and
 * 0 <= k < nslabs. */
plbm_status plbm_slab_rows(int ny, int nslabs, int k, int *y0, int *rows);

/* Halo width w = max |v_i| of a velocity set (-1 for bad arguments). */
int plbm_halo_width(int q1, const int *v);

/* Populations (index p = ix q1 + iy, ascending) that a slab's halo must hold:
 * side -1, the w rows below the slab (populations with v_y > 0); side +1, the
 * w rows above it (v_y < 0).  pops may be NULL to query *count (at most
 * q1 * q1).  Host computation. */
plbm_status plbm_halo_plan(int q1, const int *v, int side, int *pops, int *count);

/* A periodic 2D lattice (desc: dim 2, PLBM_PERIODIC) split into nslabs slabs of
 * rows (plbm_slab_rows) on desc->device.  Slab k is an ordinary handle of
 * rows_k + 2w rows: its own rows at w .. w + rows_k - 1 between a lower and an
 * upper halo of w rows.  A decomposed step copies the halo populations of
 * plbm_halo_plan from the neighbouring slabs' own rows (periodic in y, one
 * launch for all slabs), then steps every slab; the halo rows' own results are
 * discarded.  Every own row is computed from the same values by the same code
 * as in the undivided lattice, so the result equals it bit for bit: where the
 * undivided lattice takes the row-paired layout (even ny, see plbm_desc.prec)
 * the slabs take an even number of rows each (ny / 2 row pairs split by
 * plbm_slab_rows) and the row-paired layout too; otherwise every slab keeps the
 * plain layout (PLBM_FLAG_PLAIN_LAYOUT).  Each slab needs at least w rows.
 * Every launch goes to desc->stream (it must not be the legacy default stream,
 * as step pairs are captured in a CUDA graph; NULL: s creates its own).   Errors: PLBM_E_ARG, PLBM_E_NOMEM, PLBM_E_CUDA, and
 * those of plbm_create. */
typedef struct plbm_slabs_s *plbm_slabs;
plbm_status plbm_slabs_create(const plbm_desc *desc, int nslabs, plbm_slabs *out);
plbm_status plbm_slabs_destroy(plbm_slabs s);
/* Handle, first row and row count of slab k (the handle is owned by s). */
plbm_status plbm_slabs_slab(plbm_slabs s, int k, plbm_handle *h, int *y0, int *rows);
/* Equilibrium initial state from host FP64 fields [ny][nx] of the whole
 * lattice (the halo rows take the neighbours' rows).  Synchronous. */
plbm_status plbm_slabs_init(plbm_slabs s, const double *rho, const double *ux, const double *uy,
                            const double *theta);
/* n decomposed steps (pairs of them replay a CUDA graph).  Asynchronous. */
plbm_status plbm_slabs_step(plbm_slabs s, long n);
/* Fields [ny][nx] or populations [q][ny][nx] of the whole lattice, FP64 host
 * memory, gathered from the slabs' own rows.  Synchronous. */
plbm_status plbm_slabs_moments(plbm_slabs s, double *rho, double *ux, double *uy, double *theta);
plbm_status plbm_slabs_get_populations(plbm_slabs s, double *f);
/* Text of the last error of s (or of the calling thread's last slab call when NULL). */
const char *plbm_slabs_last_error(plbm_slabs s);

/* Largest lattice (nx * ny nodes) plbm_diagnostics_noalloc accepts: its
 * static scratch array holds one 64-byte record per 256 nodes (1 MiB). */
#define PLBM_NOALLOC_MAX_NODES (1 << 22)

/* Diagnostics for callers that cannot allocate device memory.  The paper has
 * no counterpart; this is a service of the library.  Some callers cannot call
 * cudaMalloc: plug-ins whose host application owns every allocation, or
 * embedded set-ups that forbid allocation after start-up.
 * This call needs no handle, allocates nothing (no cudaMalloc or cudaFree, no
 * allocating library routine) and keeps its only scratch in a static device
 * array of PLBM_NOALLOC_MAX_NODES / 256 records (1 MiB) that every GPU loading
 * the library holds until the process exits.
 *   f:   device pointer, FP64 populations [q][ny][nx] (q = q1^dim, the layout of
 *        plbm_get_populations), velocities v (q1 integers, host memory).
 *   out: device pointer to 6 doubles: mass, jx, jy, energy (sum |v|^2 f),
 *        rho_min, theta_min, with the moment definitions of this header.
 * Runs on `stream` (cudaStream_t, NULL = default) in the CUDA context current
 * on the calling thread and returns without synchronising.  Any context is
 * supported: the runtime's primary context of a device, or a context the
 * caller created and made current with the driver API.  The static array has
 * its own address in each context; the first call in a context looks that
 * address up (cudaGetSymbolAddress) and caches it under the context's unique
 * ID (cuCtxGetId), for up to 64 contexts at a time.  All calls share the one
 * array of their context:
 * calls that overlap on the GPU race and may return wrong sums, so serialise
 * them.
 * Errors: PLBM_E_ARG for bad arguments or nx * ny > PLBM_NOALLOC_MAX_NODES;
 * PLBM_E_CUDA for a failed lookup, a failed launch (the message names the
 * kernel) or a CUDA error that earlier work left pending (reported, not
 * cleared); text in plbm_last_error(NULL). */
plbm_status plbm_diagnostics_noalloc(int dim, int q1, const int *v, int nx, int ny, const double *f,
                                     double *out, void *stream);

/* Text of the last error of h (or of the calling thread when h is NULL). */
const char *plbm_last_error(plbm_handle h);

/* Name of a status code. */
const char *plbm_status_string(plbm_status s);

#ifdef __cplusplus
}
#endif

#endif /* PLBM_H */
