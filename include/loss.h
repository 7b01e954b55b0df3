/*
 * loss.h -- C ABI of the GB300 (sm_103a) implementation of the distributed local spline simulator
 * (LOSS) time step: Guo, Li, Xiong, "Distributed local spline simulator for wave propagation",
 * arXiv 2301.05127.
 *
 * What one step computes (paper Sec. 2 and 3):
 *   - along every grid line of every axis, cubic-B-spline collocation (c_{i-1} + 4 c_i + c_{i+1})/6 = f_i
 *     solved patch by patch (Eq. spline_cofficient_eq_piece), each patch closed by the perfectly matched
 *     boundary condition (PMBC, Eqs. PMBC / PMBC_coeffcients and the end closures of Sec. 3.2):
 *     truncated sums over n_nb samples on each side of every junction;
 *   - first derivatives (c_{i+1} - c_{i-1})/(2h) (Eq. derivative_approximation);
 *   - the acoustic (Eq. acoustic_wave) or elastic velocity-stress update (Sec. 2) advanced by the Strang
 *     splitting "half A, full B, half A" of Sec. 3.3 (A: velocities, B: stresses).
 *
 * Conventions shared by every entry point:
 *   - A grid axis has n intervals and n + 1 points.  Axis 0 is z (slowest), axis 1 is y (3-D only),
 *     the last axis is x (contiguous).  In 2-D the axes are (z, x) and n[2], p[2], h[2] are ignored.
 *   - Each axis is cut into p patches of M = n / p intervals; junction points are stored once.
 *   - Host-visible arrays are dense, row-major [z][y][x] (2-D: [z][x]); "flat index" means the offset in
 *     that dense array.
 *   - Field arrays are in the working precision of the grid (double for LOSS_FP64, float otherwise).
 *     Model arrays (vp, vs, rho) are always double.
 *   - mem = LOSS_MEM_HOST for host pointers, LOSS_MEM_DEVICE for device pointers of the current CUDA
 *     device.  Caller buffers are only read or written during the call, or, for device pointers, by work
 *     queued on the handle's stream before the call returns; loss_sync() waits for that work.
 *   - The library owns every device allocation it makes (through the caller's allocator if one is given)
 *     and frees them in loss_destroy().
 *   - Every entry point returns a status and never aborts.  After LOSS_E_CUDA or LOSS_E_TIMEOUT the handle
 *     is poisoned: every later call except loss_destroy / loss_last_error returns the same status.
 *     loss_last_error() describes the most recent failure on a handle.
 */
#ifndef LOSS_H_
#define LOSS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct loss_ctx* loss_handle_t; /* opaque; owned by the library */

typedef enum {
  LOSS_OK = 0,
  LOSS_E_ARG = 1,         /* bad argument (null pointer, out-of-range index, unknown enum) */
  LOSS_E_SHAPE = 2,       /* grid shape violates a rule listed at loss_create_grid */
  LOSS_E_NOMEM = 3,       /* device or host allocation failed */
  LOSS_E_CUDA = 4,        /* a CUDA call failed; handle poisoned */
  LOSS_E_STATE = 5,       /* call not valid in the handle's current state */
  LOSS_E_TIMEOUT = 6,     /* a bounded device wait expired; handle poisoned */
  LOSS_E_NUMERIC = 7,     /* non-finite values detected */
  LOSS_E_UNSUPPORTED = 8  /* valid request this build cannot serve (e.g. a line longer than fits on chip) */
} loss_status_t;

enum { LOSS_ACOUSTIC = 0, LOSS_ELASTIC = 1 };
enum { LOSS_FP64 = 0, LOSS_FP32 = 1, LOSS_FP32_KAHAN = 2 };
enum { LOSS_MEM_HOST = 0, LOSS_MEM_DEVICE = 1 };

/* Field identifiers.  Acoustic grids use V1, V3 (2-D) or V1, V2, V3 (3-D) and SIGMA (the pressure, which
 * shares the slot of S11).  Elastic grids use all nine. */
enum {
  LOSS_FIELD_V1 = 0, LOSS_FIELD_V2 = 1, LOSS_FIELD_V3 = 2,
  LOSS_FIELD_S11 = 3, LOSS_FIELD_S22 = 4, LOSS_FIELD_S33 = 5,
  LOSS_FIELD_S12 = 6, LOSS_FIELD_S13 = 7, LOSS_FIELD_S23 = 8,
  LOSS_FIELD_SIGMA = 3,
  LOSS_NUM_FIELDS = 9
};

/* Source kinds (bit mask).  PRESSURE acts on the acoustic pressure, EXPLOSIVE on S11, S22, S33, SHEAR_XZ
 * on S13 (all in the stress sub-step B, evaluated at t_n + dt/2); FORCE_X, FORCE_Y, FORCE_Z are body forces
 * f_1, f_2, f_3 of the momentum equation (paper Sec. 2, Eq. conservation_momentum) on V1, V2, V3 in each half of
 * the velocity sub-step A (at t_n and t_{n+1}); the three together are the paper's source of Sec. 4.3. */
enum {
  LOSS_SRC_PRESSURE = 1u, LOSS_SRC_EXPLOSIVE = 2u, LOSS_SRC_SHEAR_XZ = 4u, LOSS_SRC_FORCE_Z = 8u,
  LOSS_SRC_FORCE_X = 16u, LOSS_SRC_FORCE_Y = 32u
};

typedef struct {
  int32_t dim;       /* 2 or 3 */
  int32_t physics;   /* LOSS_ACOUSTIC or LOSS_ELASTIC (elastic requires dim == 3) */
  int32_t precision; /* LOSS_FP64, LOSS_FP32 or LOSS_FP32_KAHAN */
  int32_t n_nb;      /* PMBC halo width (paper Sec. 3.2): terms m = -n_nb..n_nb around each junction */
  int64_t n[3];      /* intervals per axis (axis 0 = z) */
  int32_t p[3];      /* patches per axis */
  double h[3];       /* grid spacing per axis [m] */
  double dt;         /* time step [s] */
} loss_grid_desc_t;

/* Optional device allocator.  alloc(ctx, bytes, stream) returns device memory (or NULL on failure);
 * free(ctx, ptr, stream) releases it.  stream is the handle's cudaStream_t. */
typedef struct {
  void* ctx;
  void* (*alloc)(void* ctx, size_t bytes, void* stream);
  void (*free)(void* ctx, void* ptr, void* stream);
} loss_allocator_t;

/* Version string of the library. */
const char* loss_version(void);

/* Human-readable name of a status code (static storage). */
const char* loss_status_str(loss_status_t status);

/* Text of the last failure on this handle (empty if none); valid until the next call on the handle. */
const char* loss_last_error(loss_handle_t handle);

/* Create a handle holding n_shots independent grids (shots), all resident on the current CUDA device and
 * advanced together by loss_step.  descs[s] describes shot s (paper Sec. 3.2 for the patch layout).
 * Shape rules (else LOSS_E_SHAPE): dim in {2, 3}; every used n[a] >= 2 and n[a] % p[a] == 0;
 * M = n/p >= 2 and n_nb <= M on every axis; n_nb >= 1; h > 0; dt > 0; elastic only with dim == 3.
 * Lines longer than fit in one thread block's shared memory give LOSS_E_UNSUPPORTED.
 * alloc may be NULL (then cudaMallocAsync / cudaFreeAsync on the stream are used).  cuda_stream is a
 * cudaStream_t (NULL = legacy default stream).  On success *out is a new handle; on failure *out = NULL.
 * Fields, compensation terms and the model start at zero; the source is off; no receivers. */
loss_status_t loss_create_grid(const loss_grid_desc_t* descs, int32_t n_shots, const loss_allocator_t* alloc,
                               void* cuda_stream, loss_handle_t* out);

/* Release every resource of the handle (waits for its stream first).  NULL is accepted. */
loss_status_t loss_destroy(loss_handle_t handle);

/* Set the model of one shot from dense double arrays of the grid shape: P velocity vp, S velocity vs
 * (elastic only; pass NULL for acoustic grids) and density rho.  Stored as kappa = rho vp^2 and b = 1/rho
 * (acoustic) or lambda = rho (vp^2 - 2 vs^2), mu = rho vs^2, b = 1/rho (elastic), paper Sec. 2.
 * Arrays are copied.  FP32 grids store these coefficients with loss_round_fp32_unbiased (key = 3 i + m for
 * point i of coefficient array m), so that a region of constant coefficients carries no common rounding bias.
 * LOSS_E_ARG if rho <= 0 anywhere or a required pointer is NULL. */
loss_status_t loss_set_model(loss_handle_t handle, int32_t shot, const double* vp, const double* vs,
                             const double* rho, int32_t mem);

/* Host-side conversion of n doubles to FP32 by unbiased (stochastic) rounding: a value that FP32 does not
 * hold exactly becomes one of its two FP32 neighbours lo < x < hi, hi with probability (x - lo) / (hi - lo),
 * so that the expected result is x.  The uniform variate of element i is the top 53 bits of the SplitMix64
 * output (Steele, Lea and Flood, OOPSLA 2014) for the input key0 + i, scaled to [0, 1): the conversion is
 * deterministic.  Values FP32 holds exactly, and non-finite values, convert as by a cast.  Needs no GPU and no
 * handle.  LOSS_E_ARG if n < 0 or a pointer is NULL while n > 0. */
loss_status_t loss_round_fp32_unbiased(const double* x, float* out, int64_t n, uint64_t key0);

/* Ricker source f_r(t) = (1 - 2 a) exp(-a), a = (pi f0 (t - t0))^2 (paper Sec. 4.2), with the Gaussian
 * spatial amplitude of Sec. 4.2: exp(-|o|^2 / 8) over integer offsets o (standard deviation 2 cells per
 * axis), truncated to |o_a| <= 12 and to the grid, scaled so that its sum times the cell volume equals amp.
 * idx = centre point (z, y, x); for 2-D idx[1] is ignored.  kind_mask = 0 switches the source off. */
loss_status_t loss_set_source(loss_handle_t handle, int32_t shot, const int64_t idx[3], uint32_t kind_mask,
                              double amp, double f0, double t0);

/* Absorbing layer: the ADE-PML of paper Sec. 3.3 in the outer `width` points of every axis (width = 0 turns it
 * off), with profiles d = d0 r^2, k = 1 + (k_max - 1) r, alpha = pi f0 (1 - r) at normalised depth r, and
 * d0 = -3 c_max log(R) / (2 width h), c_max = max vp of the model (so loss_set_model must come first, else
 * LOSS_E_STATE).  Memory variables start at zero.  Each sub-step integrates the memory variables exactly
 * with the other subsystem frozen (the exponential operator splitting of Sec. 3.3).
 * LOSS_E_ARG unless 2 * width <= n on every axis, 0 < R < 1, k_max > 0 and f0 > 0 (the study of Sec. 4.1
 * takes k_max from 0.5 to 19; k_max = 1 absorbs best). */
loss_status_t loss_set_pml(loss_handle_t handle, int32_t shot, int32_t width, double R, double k_max, double f0);

/* Record field `field` of shot `shot` at the n dense flat indices flat_idx (int64, copied) after every
 * step.  Replaces any earlier receiver set of that field; n = 0 removes it.  Recorded values are the
 * fields at integer time levels t_{k} (k = steps taken so far). */
loss_status_t loss_set_receivers(loss_handle_t handle, int32_t shot, int32_t field, const int64_t* flat_idx,
                                 int64_t n, int32_t mem);

/* Copy a dense field (working precision) into the state of one shot; resets that field's compensation. */
loss_status_t loss_set_field(loss_handle_t handle, int32_t shot, int32_t field, const void* src, int32_t mem);

/* Copy one field of one shot at the current integer time level into a dense array (working precision). */
loss_status_t loss_get_field(loss_handle_t handle, int32_t shot, int32_t field, void* dst, int32_t mem);

/* Advance every shot by n_steps Strang steps (paper Sec. 3.3), recording receivers after each step.
 * Asynchronous on the handle's stream. */
loss_status_t loss_step(loss_handle_t handle, int64_t n_steps);

/* Number of recorded time levels and receivers of one shot (receivers of all fields, in increasing field
 * id, each field in the order given to loss_set_receivers). */
loss_status_t loss_record_count(loss_handle_t handle, int32_t shot, int64_t* n_steps, int64_t* n_receivers);

/* Copy the traces of one shot, [n_steps][n_receivers] in working precision, and clear them. */
loss_status_t loss_record(loss_handle_t handle, int32_t shot, void* out, int32_t mem);

/* First (d1) and, if d2 != NULL, second (d2) LOSS derivative along `axis` of the dense field f given in the
 * grid shape of `shot` (working precision; d1, d2 dense of the same shape).  d1 follows Eq.
 * derivative_approximation with the PMBC closure; d2 = (c_{i-1} - 2 c_i + c_{i+1})/h^2 from the same local
 * coefficients, averaged over the two patches at a shared junction.  axis: 0 = z, 1 = y (3-D), last = x. */
loss_status_t loss_derivative(loss_handle_t handle, int32_t shot, int32_t axis, const void* f, void* d1, void* d2,
                              int32_t mem);

/* PMBC closure values phi (paper Eqs. PMBC and end closures) of the dense field f along `axis`: out has
 * shape [lines][p + 1] in double, lines ordered as the dense array with `axis` removed. */
loss_status_t loss_pmbc_phi(loss_handle_t handle, int32_t shot, int32_t axis, const void* f, double* phi, int32_t mem);

/* Transposed LOSS first derivative along `axis`: out = D^T g, with D the operator of loss_derivative (same
 * arrays, layouts and memory rules; out is overwritten).  Per line D = (3/h) P with P f = e the compact solve
 * of every patch closed by the PMBC junction values (Sec. 3.2); P^T runs the same symmetric tridiagonal solve
 * on the patch interiors (zero junction values) and scatters the junction adjoints back with the PMBC weights.
 * On an axis with knots (loss_set_coordinates) it is the transpose of that axis's spline derivative: the patch
 * slope systems are not symmetric there, so their transposed factors are used.
 * The paper has no counterpart: it is the building block of loss_gradient.  Errors as loss_derivative. */
loss_status_t loss_derivative_adjoint(loss_handle_t handle, int32_t shot, int32_t axis, const void* g, void* out,
                                      int32_t mem);

/* Seismogram misfit J = 1/2 sum_{n < n_steps} sum_r (trace_{n,r} - d_obs_{n,r})^2 of shot `shot` and its gradient
 * with respect to the model grids, by the discrete adjoint of the time step the library takes (the paper has
 * no adjoint).  The shot is reset to rest (every field, compensation term and PML memory variable zero, step 0,
 * recorded traces dropped), advanced n_steps steps with its model, source, absorbing layers and receivers, and
 * then the adjoint runs backwards, recomputing the forward states segment by segment from checkpoints taken
 * every checkpoint_every steps (0 = ceil(sqrt(n_steps))); device memory for about n_steps / C + C states.
 * d_obs: [n_steps][n_receivers] doubles in the order of loss_record.  g_vp, g_vs (elastic only; NULL allowed for
 * acoustic grids), g_rho: dense arrays of the grid shape, doubles, written.  mem says where d_obs and the
 * gradients live.  The gradient is dJ/d(model) with the time step, the absorbing profile (whose damping uses
 * the largest vp) and the source fixed.  Afterwards the shot is at step n_steps with its traces recorded.
 * Built for 2-D acoustic and 3-D elastic grids with stress-type sources; LOSS_E_UNSUPPORTED for a body force,
 * LOSS_E_STATE without a model or receivers, LOSS_E_ARG for bad arguments. */
loss_status_t loss_gradient(loss_handle_t handle, int32_t shot, const double* d_obs, int32_t checkpoint_every,
                            int64_t n_steps, double* misfit, double* g_vp, double* g_vs, double* g_rho, int32_t mem);

/* Serialise / restore the full time-stepping state of every shot (fields, compensation terms, step
 * counters) at the current integer time level.  loss_get_state with blob = NULL returns the size. */
loss_status_t loss_get_state(loss_handle_t handle, void* blob, size_t* bytes);
loss_status_t loss_set_state(loss_handle_t handle, const void* blob, size_t bytes);

/* Number of steps taken by shot `shot`. */
loss_status_t loss_get_step(loss_handle_t handle, int32_t shot, int64_t* step);

/* Kernel identifiers for loss_profile_read. */
enum {
  LOSS_KERNEL_ACOUSTIC_X = 0, /* 2-D acoustic: stress sub-step and x part of the velocity sub-step on x lines */
  LOSS_KERNEL_ACOUSTIC_Z = 1, /* 2-D acoustic: z part of the velocity sub-step and d_z v3 on z lines */
  LOSS_KERNEL_GATHER = 2,     /* receiver gather */
  LOSS_KERNEL_DERIVATIVE = 3, /* stand-alone derivative / phi (loss_derivative, loss_pmbc_phi) */
  LOSS_KERNEL_ELASTIC_X = 4,  /* 3-D elastic passes on x lines */
  LOSS_KERNEL_ELASTIC_Y = 5,  /* 3-D elastic passes on y lines */
  LOSS_KERNEL_ELASTIC_Z = 6,  /* 3-D elastic passes on z lines */
  LOSS_KERNEL_CLOCK = 7,      /* batched schedule: end-of-step advance of the device step counters */
  LOSS_KERNEL_ADJOINT = 8,    /* adjoint terms and the transposed derivative (loss_gradient, loss_derivative_adjoint) */
  LOSS_KERNEL_ACOUSTIC_X2 = 9,  /* 2-D acoustic FP32 tiles: x part of the velocity sub-step (the stress sub-step is
                                   LOSS_KERNEL_ACOUSTIC_X) */
  LOSS_KERNEL_ACOUSTIC_Z2 = 10, /* 2-D acoustic FP32 tiles: d_z v3 for the next step (the z velocity part is
                                   LOSS_KERNEL_ACOUSTIC_Z) */
  LOSS_KERNEL_WATCH = 11,       /* non-finite watchdog pass (loss_set_watchdog) */
  LOSS_NUM_KERNELS = 16
};

/* Launch shape of one kernel family of the handle: lines_per_block = number of whole grid lines one thread block
 * holds on chip (power of two, 1..32) and chunk_log2 = log2 of the number of unknowns one thread solves serially
 * (3 or 4; FP64 grids always use 4); 0 = the built-in choice.  Applies to every shot; shapes that do not fit
 * fall back to smaller bundles at launch.  Used by the autotuner. */
loss_status_t loss_set_launch(loss_handle_t handle, int32_t kernel, int32_t lines_per_block, int32_t chunk_log2);

/* Tile shape of one kernel family given as a block size: threads_per_block (32..1024, 512 at most for FP64 grids)
 * is the thread count a block of this kernel aims at; every shot then takes the widest power-of-two bundle of
 * whole lines whose chunks fit in it (so shots of different sizes share one block size in a batched launch).
 * chunk_log2 as in loss_set_launch.  0 = the built-in choice.  An explicit lines_per_block (loss_set_launch)
 * takes precedence.  For the truncated-convolution z tiles (LOSS_KERNEL_ACOUSTIC_Z = Z1, LOSS_KERNEL_ACOUSTIC_Z2 =
 * Z2) chunk_log2 is the number of z positions one warp row of a tile takes (8 or 16; 0 = 16) and fixes the block
 * size, 32 x ceil(M / chunk); threads_per_block does not apply to them.  Used by the autotuner.  LOSS_E_ARG for
 * values out of range. */
loss_status_t loss_set_tile(loss_handle_t handle, int32_t kernel, int32_t threads_per_block, int32_t chunk_log2);

/* Schedule of loss_step: the batched multi-shot schedule (the paper's MPI design runs one process per patch
 * instead).  batched != 0 (the default): a handle whose shots are all 2-D acoustic grids of one precision advances
 * them together, each step being one persistent launch per kernel over the work of all shots, one launch per
 * receiver phase and a clock tick.  The kernels are those of the per-shot step: with the truncated-convolution
 * family (FP32, when every shot qualifies) the x kernel over row units of all shots, then Z1 and Z2 over the z
 * tiles of all shots; otherwise the line kernels, x and z over bundles of whole lines.  The source amplitude and
 * the trace row of each step are read from per-shot device counters, so the launches of every step are
 * identical.  graph_steps > 0: such handles (also with a single shot) capture graph_steps steps
 * once in a CUDA graph and replay it (the remainder of a loss_step call runs as plain launches); the graph is
 * captured again when shapes, buffers or the shot set change.  Results are those of the per-shot schedule.
 * Other handles (3-D elastic) always use per-shot launches.  Per-kernel timing (loss_profile) is not available
 * for steps replayed from a graph; launches are counted.  LOSS_E_ARG if graph_steps < 0. */
loss_status_t loss_set_schedule(loss_handle_t handle, int32_t batched, int32_t graph_steps);

/* Kernel family of the per-shot FP32 2-D acoustic step: LOSS_KERNELS_LINE = whole grid lines on chip with the
 * chunked Thomas solve of the patch systems (the form every other grid and the batched schedule use);
 * LOSS_KERNELS_CONVOLUTION (the default) = the truncated-convolution form: the same patch systems solved through
 * the closed-form inverse of the (1, 4, 1) operator, truncated where |sqrt(3) - 2|^k < 1e-9, with exact patch-end
 * corrections from the PMBC junction values (x rows pipelined through TMA bulk copies, z lines on independent
 * 32-column x one-patch tiles; rows the pipelined kernel does not take, longer than 2049 points or with patches
 * whose length is not a multiple of 8, go to independent (row, patch) items in two launches);
 * LOSS_KERNELS_CONVOLUTION_ITEMS = the same with every row on (row, patch) items.  All agree with the FP64 oracle
 * at the FP32 tolerance; they differ in rounding.  LOSS_E_ARG for another value. */
enum { LOSS_KERNELS_LINE = 0, LOSS_KERNELS_CONVOLUTION = 1, LOSS_KERNELS_CONVOLUTION_ITEMS = 2 };
loss_status_t loss_set_kernels(loss_handle_t handle, int32_t family);

/* One autotuner result: the tile shape chosen for a kernel family and its measured mean launch time. */
typedef struct {
  int32_t kernel;            /* LOSS_KERNEL_* */
  int32_t threads_per_block; /* as loss_set_tile */
  int32_t chunk_log2;
  double ms;                 /* mean device time of one launch of the chosen shape */
} loss_tune_entry_t;

/* Project-written autotuner (for the batched multi-shot schedule): times every candidate tile shape (threads per
 * block 128..1024, chunk_log2 3 or 4; for the convolution kernels the z chunk of Z1 and Z2) of each kernel family the
 * handle's time step uses, on a scratch copy of the handle (same grids, models, absorbing layers, kernel family
 * and schedule; zero fields), with `steps` timed steps per candidate
 * after one warm-up step, and applies the fastest shape of each family to the handle (loss_set_tile).  The
 * handle's own state is not touched.  out (capacity cap entries, may be NULL) receives one entry per tuned
 * family and *n_out their number.  Needs device memory for a second copy of the handle's arrays.
 * Returns LOSS_E_ARG for steps < 1, the error of the first failing call otherwise. */
loss_status_t loss_autotune(loss_handle_t handle, int32_t steps, loss_tune_entry_t* out, int32_t cap, int32_t* n_out);

/* Reset the per-kernel counters of the handle and switch CUDA-event timing of every kernel launch on
 * (enable != 0) or off.  Launches are always counted. */
loss_status_t loss_profile(loss_handle_t handle, int32_t enable);

/* Launches of kernel `kernel` since the last loss_profile call and, if timing was on, their summed device
 * duration in milliseconds (waits for the stream).  kernel = -1 gives the totals over all kernels. */
loss_status_t loss_profile_read(loss_handle_t handle, int32_t kernel, double* total_ms, int64_t* launches);

/* First LOSS derivative along `axis` for callers that cannot allocate device memory (code running under another
 * framework's allocator, which owns every device allocation of the process, or under a memory budget that forbids
 * allocations after start-up), so they cannot create a handle.  The paper has no counterpart: this is a deployment
 * variant of loss_derivative.
 * desc: the grid; only dim, n, p, h, n_nb and precision are read and checked as in loss_create_grid (physics and
 * dt are ignored); f, d1: DEVICE pointers to dense arrays of the grid shape in the working precision of
 * desc->precision; cuda_stream: the stream to run on.
 * Nothing is allocated: the PMBC weights and Thomas factors are written into a 64 KiB static device array that
 * every GPU loading this library keeps until the process exits.  Limit: (p + 1) * (2 n_nb + 1) <= 8096 on the
 * axis, else LOSS_E_UNSUPPORTED before any work is queued.  Every call rewrites the whole table it reads, so no
 * state carries over between calls; but each device holds one copy of the array, so calls on the same device
 * whose work overlaps on the GPU (different streams) race on it: serialise them.  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) with that device current.
 * Returns LOSS_E_ARG / LOSS_E_SHAPE for bad arguments, LOSS_E_CUDA if a CUDA call fails. */
loss_status_t loss_derivative_noalloc(const loss_grid_desc_t* desc, int32_t axis, const void* f, void* d1,
                                      void* cuda_stream);

/* Non-uniform grid spacing along one axis (paper Sec. 3: the construction carries over to non-uniform grids; the
 * conclusion names it as future work).  x: HOST array of n[axis] + 1 finite, strictly increasing knot coordinates,
 * copied; NULL returns the axis to the uniform spacing h[axis].  On such an axis loss_derivative (first and second
 * derivatives) and loss_pmbc_phi use the cubic spline on these knots: the PMBC weights are the junction rows of the
 * global natural spline's slope operator, truncated to |m| <= n_nb (FP64, built on the host), and each patch solves
 * its own slope system with the junction values as ends; the second derivative is the patch spline's, averaged
 * over the two patches at a junction.  Layout and precision of the fields are unchanged.
 * loss_step on such a shot (2-D acoustic) takes the literal Strang step of Sec. 3.3 with every derivative on the
 * knots (other axes of the shot get equally spaced knots); the state stays at the integer time level.  An
 * absorbing layer (loss_set_pml, before or after this call) takes its profiles on the physical distance into the
 * layer: on each side L = the layer's physical width and d0 = -3 vmax ln R / (2 L), the normalised depth of a knot
 * its distance past the first physical knot over L.  A pressure source takes its Gaussian amplitude (width 2 h) on
 * the physical distance from the source knot over the same 25 knots per axis, normalised with the knots' dual cell
 * volumes so that it injects the uniform grid's total.  loss_derivative_adjoint on the axis applies the exact
 * transpose of this derivative.  Returns LOSS_E_ARG for a bad axis or knots; afterwards loss_gradient on the shot
 * and loss_step on other shot kinds return LOSS_E_UNSUPPORTED. */
loss_status_t loss_set_coordinates(loss_handle_t handle, int32_t shot, int32_t axis, const double* x);

/* Poll limit of the bounded waits of the staged FP32 x kernels (each block waits on an mbarrier for the bulk copies
 * of its next row).  A wait that runs out sets the handle's device error flag; the block then waits (with a fixed
 * limit) for its own copies in flight and stops, so the CUDA context stays usable, and the next loss_sync returns
 * LOSS_E_TIMEOUT and poisons the handle.  polls < 0 restores the default (2^24 polls, far beyond any copy's
 * latency); polls = 0 makes every such wait give up without polling, which is how the failure path is tested.
 * This is a library control with no counterpart in the paper.  Takes effect from the next loss_step (a captured
 * graph is recaptured).  Returns LOSS_E_ARG for a NULL handle. */
loss_status_t loss_set_wait_limit(loss_handle_t handle, int64_t polls);

/* Non-finite watchdog (a library control with no counterpart in the paper): with every_steps > 0, at the end of
 * each loss_step call that completes another every_steps steps (counted from this call), one streaming pass over
 * every field of every shot checks for Inf and NaN (kernel LOSS_KERNEL_WATCH, one read of each field).  The first
 * non-finite field found is reported by the next loss_sync as LOSS_E_NUMERIC, with the shot and field in
 * loss_last_error; the report clears the flag and does not poison the handle (fields may be reset with
 * loss_set_field).  every_steps = 0 (the default) turns the watchdog off.  Returns LOSS_E_ARG for every_steps < 0. */
loss_status_t loss_set_watchdog(loss_handle_t handle, int64_t every_steps);

/* Wait for all work queued on the handle's stream.  Returns LOSS_E_TIMEOUT (sticky) if a kernel gave up on a
 * bounded wait, LOSS_E_NUMERIC if the watchdog found a non-finite field, LOSS_E_CUDA if the stream failed. */
loss_status_t loss_sync(loss_handle_t handle);

#ifdef __cplusplus
}
#endif

#endif /* LOSS_H_ */
