/*
 * cavity.h -- C ABI of the GB300 (sm_103a) buoyancy-driven-cavity step.
 *
 * One explicit time step of the artificial-compressibility Boussinesq solver
 * of Xue & Roy (arXiv 2006.02602): fields p, u, v, w, T on a unit cube with n
 * interior nodes per axis, walls at the nodes 0 and n+1 (h = 1/(n+1)), a
 * pressure ghost beyond every wall.  Per step (Section 2, Eqs. 1-3; Section
 * 3.1, Fig. 1; Section 4.5, Listings 1-2):
 *   dt from the previous step's spectral-radius max-reduce,
 *   fused residual + explicit Euler update of every interior node (13-point
 *   pressure star, 7-point star for u, v, w, T),
 *   FP64 residual sums, centre-pressure rescale, wall conditions,
 *   ghost-face pack/unpack between the blocks of a decomposition held on one
 *   device (p at depth 2, u, v, w, T at depth 1), hot/cold wall Nusselt.
 *
 * Nondimensional (thermal) scaling: rho = 1, alpha = 1, nu = Pr,
 * g sigma = Ra Pr.  Hot wall x = 0, cold wall x = 1, other walls adiabatic,
 * no slip everywhere; buoyancy along +gravity_axis.
 *
 * Conventions for every entry point:
 *  - return 0 (CAVITY_OK) or a negative CAVITY_ERR_* code; cavity_strerror()
 *    names a code, cavity_last_error() gives the last message of a handle;
 *  - the library owns all device memory of a handle; the caller owns every
 *    host buffer and must keep it valid for the duration of the call;
 *  - host arrays of interior fields are FP64, ordered (f, k, j, i) with i
 *    fastest and f in p, u, v, w, T order restricted to the mask;
 *  - cavity_step() only enqueues work on the handle's stream; every getter
 *    synchronises that stream first;
 *  - a handle is not thread safe; distinct handles are independent.
 */
#ifndef BDC_CAVITY_H
#define BDC_CAVITY_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define CAVITY_API __attribute__((visibility("default")))
#else
#define CAVITY_API
#endif

/* status codes */
#define CAVITY_OK 0
#define CAVITY_ERR_INVALID_ARG (-1) /* bad pointer, size, mask or parameter */
#define CAVITY_ERR_OOM (-2)         /* device or host allocation failed */
#define CAVITY_ERR_CUDA (-3)        /* a CUDA runtime call failed (see cavity_last_error) */
#define CAVITY_ERR_NONFINITE (-4)   /* a residual or the spectral radius became NaN/Inf */
#define CAVITY_ERR_TIMEOUT (-5)     /* a bounded device-side wait gave up */
#define CAVITY_ERR_UNSUPPORTED (-6) /* valid request this build does not implement */

/* arithmetic forms */
#define CAVITY_FP64 0       /* every field and every operation in FP64 */
#define CAVITY_FP32_MIXED 1 /* u, v, w in FP32; p and T as FP32 hi/lo pairs; FP64 reductions */

/* field masks */
#define CAVITY_FIELD_P 1
#define CAVITY_FIELD_U 2
#define CAVITY_FIELD_V 4
#define CAVITY_FIELD_W 8
#define CAVITY_FIELD_T 16
#define CAVITY_FIELD_ALL 31

typedef struct cavity cavity_t; /* opaque, library owned */

/* Geometry, decomposition and initial condition.
 *  nx, ny, nz   interior nodes per axis (h_d = 1/(n_d+1));
 *  px, py, pz   block grid; the cavity is split as evenly as possible along
 *               each axis (Section 3.2), every block at least 2 nodes thick;
 *               1,1,1 = a single block;
 *  precision    CAVITY_FP64 or CAVITY_FP32_MIXED;
 *  seed, noise_amp  initial T = t_hot + (t_cold - t_hot) x + noise_amp (2U - 1),
 *               U from splitmix64(seed * 2^40 + global interior index);
 *               u = v = w = p = 0;
 *  device       CUDA device ordinal;
 *  stream       cudaStream_t to run on, or NULL for a stream the handle owns. */
typedef struct {
  int nx, ny, nz;
  int px, py, pz;
  int precision;
  unsigned long long seed;
  double noise_amp;
  int device;
  void *stream;
} cavity_desc;

/* Physical and numerical parameters (Section 2; the paper gives no formula for
 * beta, eps or dt, so the forms below are readings of its text).  Negative
 * u_ref or NaN t_inf select their defaults:
 * u_ref = max(1, sqrt(Ra Pr)), t_inf = (t_hot + t_cold) / 2.
 *  beta^2 = max(|V|^2, kappa u_ref^2)                 (Section 2)
 *  eps_d  = c4 lambda_d h_d^3 / beta^2                 (Eq. 1 dissipation)
 *  dt     = cfl / max[sum_d lambda_d/h_d + 2 max(nu,alpha) sum_d 1/h_d^2]
 *  gravity_axis 1 (y) or 2 (z).
 * Ra >= 0, Pr, cfl, kappa, u_ref > 0, c4 >= 0, finite distinct wall
 * temperatures, and kappa u_ref^2 in [2^-126, 1e300]; anything else gives
 * CAVITY_ERR_INVALID_ARG where the parameters are set. */
typedef struct {
  double Ra, Pr, cfl, kappa, c4, u_ref, t_inf, t_hot, t_cold;
  int gravity_axis;
} cavity_params;

/* Fill *p with the default parameters (Ra 1e5, Pr 0.71, cfl 0.5, kappa 0.1,
 * c4 1/32, u_ref and t_inf defaulted, t_hot 1, t_cold 0, gravity_axis 2). */
CAVITY_API int cavity_default_params(cavity_params *p);

/* Allocate the handle and its device state, initialise the fields from desc
 * (Section 2 problem statement), apply the walls, exchange ghosts and compute
 * the first dt.  Uses the default parameters until cavity_set_params().
 * On error *out is NULL and nothing is leaked. */
CAVITY_API int cavity_create(const cavity_desc *desc, cavity_t **out);

/* Set the parameters.  Before the first step the state is re-initialised
 * from the descriptor's seed and noise under the new parameters; after it the
 * fields are kept and only the walls and the next dt are recomputed. */
CAVITY_API int cavity_set_params(cavity_t *h, const cavity_params *p);

/* Temperature of an isothermal wall (Section 2: the left and right vertical
 * walls are held at fixed temperatures): wall 0 = hot (x = 0), 1 = cold
 * (x = 1).  host holds ny*nz values, (j-1) + ny (k-1) order; n must equal
 * ny*nz (CAVITY_ERR_INVALID_ARG otherwise, or for a wall other than 0 or 1).
 * Replaces the uniform t_hot / t_cold on that wall; walls are re-applied.
 * The caller keeps the host array; the call copies it and synchronises. */
CAVITY_API int cavity_set_wall_temperature(cavity_t *h, int wall, const double *host, size_t n);

/* Enqueue nsteps explicit steps (nsteps >= 0) on the handle's stream.  One
 * step is the first-order explicit update in (pseudo) time of Section 2 with
 * the second-order central differences and fourth-difference pressure
 * dissipation of Eqs. 1-3 on the stencils of Section 3.1 (Fig. 1), the
 * centre-pressure rescale and wall extrapolations of Section 2, and, for a
 * decomposed cavity, the ghost-face pack/unpack of Section 4.5 (Listings
 * 1-2, V3).  Asynchronous: errors of the device work (non-finite state, a
 * timed-out wait) surface at the next getter or cavity_sync();
 * CAVITY_ERR_INVALID_ARG for nsteps < 0. */
CAVITY_API int cavity_step(cavity_t *h, int nsteps);

/* One step's record in a step log (cavity_set_step_log): the state's counters
 * and diagnostics after the step, as the getters would return them then
 * (step count, time, the next dt, the residual norms of Section 4.2, the
 * Nusselt numbers, flags: bit 0 non-finite, bit 1 a timed-out wait). */
typedef struct {
  long long step;
  double t, dt;
  double res[5];
  double nu_hot, nu_cold;
  long long flags;
} cavity_step_record;

/* Step log in host memory: after each step the device writes that step's
 * record of cavity c (0 for a single cavity) to host[((step - 1) % capacity)
 * * ncav + c], in the launch that finishes the step, so a caller that wants
 * every step's diagnostics reads them from host memory when it next
 * synchronises, without a synchronising getter per step.  host must be
 * page-locked host memory (cudaHostAlloc, cudaHostRegister, a pinned torch
 * tensor) of capacity * ncav records, kept alive while attached; NULL
 * detaches.  Records of steps the adjoint's reverse sweep recomputes are
 * written again.  CAVITY_ERR_INVALID_ARG for capacity < 1 or memory the device
 * cannot address. */
CAVITY_API int cavity_set_step_log(cavity_t *h, cavity_step_record *host, long long capacity);

/* Page-locked, zeroed host memory for `records` step records (records >= 1),
 * and its release; CAVITY_ERR_OOM if the allocation fails. */
CAVITY_API int cavity_step_log_alloc(long long records, cavity_step_record **out);
CAVITY_API int cavity_step_log_free(cavity_step_record *p);

/* RMS over the interior of dq/dt of the last step, p, u, v, w, T
 * (Section 4.2 residual norms).  Zeros before the first step.
 * Returns CAVITY_ERR_NONFINITE (after filling out) once a step produced
 * a NaN/Inf residual or spectral radius. */
CAVITY_API int cavity_residual(cavity_t *h, double out[5]);

/* Hot- and cold-wall Nusselt numbers of the current state: mean over the
 * ny*nz wall nodes of the one-sided second-order wall heat flux divided by
 * (t_hot - t_cold).  The paper defines no Nusselt number; this is the
 * hot-wall Nusselt number the benchmark configurations of this cavity ask
 * for (the 32^3, Ra 1e4 run reports it), taken with the second-order
 * one-sided difference that matches the scheme's order (Section 2).  Either
 * pointer may be NULL.  Synchronises; returns the sticky status. */
CAVITY_API int cavity_nusselt(cavity_t *h, double *hot, double *cold);

/* Copy interior fields of the whole cavity to host (FP64; FP32 fields
 * widened, the p pair summed): the state p, u, v, w, T of Eqs. 1-3 on the
 * interior nodes of Section 3.1's grid, gathered across the blocks of the
 * Section 3.2 decomposition, p after the centre rescale (Section 2).  count
 * must equal popcount(mask)*nx*ny*nz (CAVITY_ERR_INVALID_ARG otherwise).
 * Synchronises the stream; the caller owns host. */
CAVITY_API int cavity_get_fields(cavity_t *h, int field_mask, double *host, size_t count);

/* Copy a box of interior nodes (global 1-based node ranges i0 .. i0+ni-1,
 * j0 .. j0+nj-1, k0 .. k0+nk-1) of the fields in the mask to host, FP64,
 * ordered (f, k, j, i); count must equal popcount(mask)*ni*nj*nk.  For
 * probes and sampled checks of cavities too large to copy whole. */
CAVITY_API int cavity_get_fields_box(cavity_t *h, int field_mask, int i0, int j0, int k0, int ni, int nj, int nk,
                                     double *host, size_t count);

/* Overwrite interior fields from host (layout as cavity_get_fields), then
 * re-apply the Section 2 wall conditions, exchange ghosts (Section 4.5) and
 * recompute dt; the state can then be stepped as if the scheme had reached
 * it (checkpoint/restart of the Section 2 iteration).  Step count and time
 * are kept.  FP32-mixed handles round u, v, w to FP32 and split p and T
 * into FP32 pairs.  count as cavity_get_fields; synchronises. */
CAVITY_API int cavity_set_fields(cavity_t *h, int field_mask, const double *host, size_t count);

/* Step counter, simulated (pseudo) time t = sum of the global dt of the
 * steps taken, and the dt the next step will use: cfl over the largest
 * spectral-radius bound of the current state (the stable explicit step of
 * Section 2).  Any pointer may be NULL.  Synchronises; returns the sticky
 * status. */
CAVITY_API int cavity_get_time(cavity_t *h, long long *step, double *t, double *dt);

/* Number of blocks (px*py*pz). */
CAVITY_API int cavity_num_blocks(cavity_t *h);

/* Whole stored array `field` of one block, walls and ghosts included, as
 * stored (p before the pending centre shift), (k, j, i) order over local
 * nodes -1 .. n+2 of each axis: count = (nx_b+4)(ny_b+4)(nz_b+4).  Array
 * index: FP64 form p, u, v, w, T (0..4); FP32-mixed form p_hi, p_lo, u, v,
 * w, T_hi, T_lo (0..6).  The FP32-mixed step forms p's wall and ghost values
 * and the adiabatic T where it reads them, so those stored entries are only
 * refreshed by state changes (creation, set_fields, parameters).
 * dims (optional) receives nx_b, ny_b, nz_b, ox, oy, oz (global node index
 * = o + local index).  For checks of the ghost exchange. */
CAVITY_API int cavity_get_block_array(cavity_t *h, int block, int field, double *host, size_t count, int dims[6]);

/* The packed buffer of one cut face of one block (Section 4.5 layout:
 * p at depth 2 with depth fastest, then u, v, w, T at depth 1), widened to
 * FP64; count must equal 6*nb*nc (FP64 form) or 9*nb*nc (FP32-mixed form:
 * p_hi then p_lo at depth 2, then u, v, w, T_hi, T_lo at depth 1), packed
 * from the current state by this call: the values every exchange of this
 * state sends (the step's exchange writes the neighbour's ghost layers
 * without the buffer).  Synchronises.  CAVITY_ERR_INVALID_ARG if the face is
 * a wall. */
CAVITY_API int cavity_get_face_buffer(cavity_t *h, int block, int face, double *host, size_t count);

/* Pack and unpack every cut face of the current state (a7, a8 alone). */
CAVITY_API int cavity_exchange(cavity_t *h);

/* Batch of independent cavities advanced together (the batched form of the
 * step): every launch covers all cavities through one block descriptor table
 * and one work list per kernel, and each cavity's reductions finalise in
 * parallel (one last-CTA counter per cavity).  descs[i] gives cavity i's size,
 * seed and noise; each member is a single block (px = py = pz = 1); precision,
 * device and stream come from descs[0].  params[i] are cavity i's parameters
 * (params may be NULL for the defaults).  The single-cavity getters and
 * cavity_set_wall_temperature address cavity 0; cavity_set_params sets every
 * cavity. */
CAVITY_API int cavity_create_batch(const cavity_desc *descs, const cavity_params *params, int n, cavity_t **out);

/* Number of cavities of a handle (1 for cavity_create). */
CAVITY_API int cavity_batch_size(cavity_t *h);

/* State of cavity `cav`: out[0] step, out[1] t, out[2] next dt, out[3..7]
 * RMS dq/dt of p, u, v, w, T of the last step, out[8] hot- and out[9]
 * cold-wall Nusselt number. */
CAVITY_API int cavity_batch_state(cavity_t *h, int cav, double out[10]);

/* Interior fields of cavity `cav` (layout of cavity_get_fields, that
 * cavity's nx, ny, nz). */
CAVITY_API int cavity_batch_get_fields(cavity_t *h, int cav, int field_mask, double *host, size_t count);

/* Autotuner of the FP32-mixed step kernel: times every compiled tile shape
 * (x-y tile extent, z-chunk length, ring depth) for `steps` graph-replayed
 * steps on this handle's own cavities, times the four fastest once more
 * (each keeps its better time) and keeps the fastest.  The state is
 * saved before the trials and restored after them (the step counter and the
 * fields are as before the call).  out (optional) receives the chosen tile
 * height (8 or 16 rows of 32 nodes), z-chunk, ring depth, kernel form (3:
 * two nodes per thread, the z neighbours below the plane in registers, the
 * one form) and microseconds per step.  Every shape gives the same fields.
 * With the environment variable BDC_F32_TILE
 * ("TY,KC,R,form", a compiled shape, read at creation) the shape is pinned and
 * no trials run (out[4] = 0).  FP64 handles have a single shape (32 x 4
 * threads, 8-plane chunks; BDC_F64_TY=8, read at creation, selects 32 x 8):
 * CAVITY_ERR_UNSUPPORTED. */
CAVITY_API int cavity_autotune(cavity_t *h, int steps, double out[5]);

/* Discrete adjoint, part 1: from the current state run nsteps steps and
 * return J = (1/nsteps) sum over steps 1..nsteps of the hot-wall Nusselt
 * number.  The state every ckpt steps is kept on the device (checkpoints)
 * for cavity_adjoint_backward.  Single-block, single-cavity handles with
 * global time stepping and (nx+4)(ny+4)(nz+4) < 2^31 only
 * (CAVITY_ERR_UNSUPPORTED otherwise).  The state afterwards is the state
 * after the nsteps steps. */
CAVITY_API int cavity_adjoint_forward(cavity_t *h, int nsteps, int ckpt, double *J);

/* Discrete adjoint, part 2: gradient of the J of the last
 * cavity_adjoint_forward with respect to the hot-wall temperature field
 * (grad_wall: ny*nz host values, (j-1) + ny (k-1) order; n must equal
 * ny*nz; may be NULL) and to Ra (grad_ra, may be NULL).  Reverse sweep of
 * the step (Section 2 scheme; dt, beta^2 and |V| differentiated along the
 * forward branch), each ckpt-step segment recomputed from its checkpoint.
 * The sweep runs in the forward form's arithmetic: FP64 after an FP64
 * forward; FP32 adjoint arrays with FP64 node sums after an FP32-mixed
 * forward (linearised about its FP32 trajectory); the returned gradients
 * are FP64 either way.  When u_ref was left to its default it follows Ra
 * (u_ref^2 = Ra Pr) in the derivative.  The state is restored to the one
 * after the forward run. */
CAVITY_API int cavity_adjoint_backward(cavity_t *h, double *grad_wall, size_t n, double *grad_ra);

/* Measurement: mean duration in ms, from CUDA events on the handle's stream
 * around every launch, of the dominant kernel of the last
 * cavity_adjoint_backward: the reverse of the rates (k_adj_gather after an
 * FP32-mixed forward, k_adj_rates after an FP64 one), one launch per reverse
 * step.  CAVITY_ERR_INVALID_ARG before the first reverse sweep. */
CAVITY_API int cavity_adjoint_kernel_ms(cavity_t *h, double *ms);

/* Interior/shell split with overlap (Section 4.7): when on, each step first
 * computes the nodes within two layers of a cut face, then exchanges the new
 * ghost layers (pack + unpack) on a second stream while the remaining nodes
 * are stepped, and applies the walls and the reductions after both.  Fields
 * are bit-identical to the plain schedule; the residual sums are reduced in
 * another order.  FP64 single-cavity handles (CAVITY_ERR_UNSUPPORTED
 * otherwise); without cut faces there is nothing to overlap and the call
 * changes nothing.  on = 0 returns to the plain schedule. */
CAVITY_API int cavity_set_overlap(cavity_t *h, int on);

/* Time stepping.  CAVITY_DT_GLOBAL (default): every node advances by the one
 * stable step dt = cfl / max_n S_n (time accurate, Section 2).  CAVITY_DT_LOCAL:
 * node n advances by its own dt_n = cfl / S_n, S_n its spectral bound in the
 * state before the step -- the iteration in pseudo time towards a steady
 * state (Section 3.1); residuals, Nusselt numbers and the centre rescale are
 * unchanged, and the time t keeps summing the global dt.  Both precisions and
 * batch handles; CAVITY_ERR_INVALID_ARG for another mode. */
#define CAVITY_DT_GLOBAL 0
#define CAVITY_DT_LOCAL 1
CAVITY_API int cavity_set_time_stepping(cavity_t *h, int mode);

/* Measurement: run nsteps steps as plain launches (no graph replay) with CUDA
 * events around every kernel on the handle's stream.  ms[0..3] receive the
 * mean duration per launch of the fused step kernel, the wall/finalise
 * kernel, the pack kernel and the unpack kernel (0 where a kernel does not
 * run).  The steps are real steps of the state. */
CAVITY_API int cavity_time_kernels(cavity_t *h, int nsteps, double ms[4]);

/* Self-check of the FP64 square root the fused FP64 step uses for the wave
 * speeds lambda_d = (|V_d| + sqrt(V_d^2 + 4 beta^2)) / 2 (Section 2): a
 * Newton iteration seeded by the approximate reciprocal square root.  On the
 * current CUDA device, evaluates it and CUDA's correctly rounded sqrt for the
 * n host values x (positive, normal, finite; copied in and out by the call,
 * which synchronises) and returns the largest relative difference in
 * *max_rel and the number of values where the two differ in *n_diff.
 * CAVITY_ERR_INVALID_ARG for n < 1 or n > 2^26, a null pointer or a value
 * outside that range; CAVITY_ERR_OOM / CAVITY_ERR_CUDA on a CUDA error. */
CAVITY_API int cavity_check_sqrt(const double *x, long long n, double *max_rel, long long *n_diff);

/* Self-check of the division by 3 in the adiabatic wall value
 * T_w = (4 T_1 - T_2) / 3 (the one-sided second-order zero-flux condition of
 * Section 2) of the FP64 wall kernel: a rounded reciprocal of 3 and one
 * residual correction through fused multiply-adds (Markstein 1990).  On the
 * current CUDA device, evaluates it and CUDA's correctly rounded division for
 * the n host values x (finite, |x| >= 4 DBL_MIN, so that the quotient is
 * normal; copied in and out by the call, which synchronises) and returns in
 * *n_diff the number of values where the two differ.
 * CAVITY_ERR_INVALID_ARG for n < 1 or n > 2^26, a null pointer or a value
 * outside that range; CAVITY_ERR_OOM / CAVITY_ERR_CUDA on a CUDA error. */
CAVITY_API int cavity_check_div3(const double *x, long long n, long long *n_diff);

/* Measurement (no counterpart in the paper): the FP64 FMA throughput of CUDA
 * device `device` in TFLOP/s (2 flops per FMA), the ceiling of the FP64 step
 * kernel, whose 190 FP64 operations per 80 bytes of state put it far on the
 * arithmetic side of GB300's FP64 roofline.  Independent FMA chains on every
 * resident thread of every SM, timed with CUDA events over one launch of
 * about 0.1 s after a warm-up launch; the best of three.  Allocates and frees
 * a few kilobytes; synchronises its own stream.  CAVITY_ERR_INVALID_ARG for a
 * null pointer or a device that does not exist. */
CAVITY_API int cavity_measure_fp64_peak(int device, double *tflops);

/* Allocation-free step of one caller-held block.  The paper has no
 * counterpart; this exists for callers that must not call cudaMalloc, such as
 * code running inside another framework's caching allocator or a fixed,
 * pre-sized memory arena, where a driver allocation behind the allocator's
 * back would break its accounting and its out-of-memory handling.
 *
 * Runs the fused residual + explicit-update kernel (the one cavity_step uses)
 * once over a single block whose walls and ghosts the caller has already
 * filled, then reduces the rates:
 *  q_in   device, 5 fields (p, u, v, w, T) one after another, each a dense
 *         (nz+4)(ny+4)(nx+4) FP64 array over local nodes -1 .. n+2 with x
 *         fastest (the layout cavity_get_block_array returns); read only;
 *  q_out  device, same layout, distinct from q_in; the interior nodes are
 *         written (p_new = p - pshift + dt dp/dt, q_new = q + dt dq/dt),
 *         walls and ghosts are left untouched;
 *  p      parameters (defaults resolved as in cavity_set_params);
 *  dt     the time step; pshift a pending centre-pressure shift (0 if none);
 *  out6   device, 6 doubles: RMS dq/dt of p, u, v, w, T and the next dt;
 *  stream cudaStream_t (NULL = the legacy default stream); the call only
 *         enqueues work.
 * Nothing is allocated: the per-CTA reduction partials and the kernel
 * descriptors live in one fixed array compiled into the library, about
 * 1 MiB, held on every GPU that loads the library until the process exits.
 * Limit: ceil(nx/32) ceil(ny/8) ceil(nz/16) <= CAVITY_NOALLOC_MAX_TILES
 * (e.g. 256^3 fits, 512^3 does not); larger blocks return
 * CAVITY_ERR_INVALID_ARG.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current.  All
 * calls share the array and it
 * keeps the last call's contents (each call rewrites all it reads): calls
 * that overlap on the GPU (other streams, other threads) race and must not
 * be issued. */
#define CAVITY_NOALLOC_MAX_TILES 16384
CAVITY_API int cavity_step_block_noalloc(const double *q_in, double *q_out, int nx, int ny, int nz,
                                         const cavity_params *p, double dt, double pshift, double *out6,
                                         void *stream);

/* Test hook of the failure detection (the paper has none): the FP32-mixed
 * step kernels wait on shared-memory barriers for each TMA plane load, every
 * wait bounded; a wait that gives up sets the cavity's sticky timeout flag,
 * lets the CTA's issued copies land (again bounded) and returns, so the
 * context stays usable and cavity_sync() / the getters report
 * CAVITY_ERR_TIMEOUT.  This sets the limit of each wait (wait_cycles, SM
 * clock cycles in [1000, 4e9]; 4e9, about 2 s, is the default) and, with
 * withhold_plane >= 0, leaves the load of that plane of every tile (0 = the
 * first halo plane below the tile's z range) unissued, so that its waits run
 * out; withhold_plane = -1 issues every load.  The step graphs are rebuilt.
 * FP32-mixed handles only (CAVITY_ERR_UNSUPPORTED otherwise); the state of a
 * handle whose wait ran out is not a step of the scheme: destroy it. */
CAVITY_API int cavity_test_wait_timeout(cavity_t *h, long long wait_cycles, int withhold_plane);

/* Synchronise the handle's stream; returns the sticky status: CAVITY_ERR_TIMEOUT
 * once a bounded device-side wait gave up, else CAVITY_ERR_NONFINITE once a
 * step produced a non-finite residual or spectral radius, else CAVITY_OK. */
CAVITY_API int cavity_sync(cavity_t *h);

/* Release everything the handle owns.  NULL is accepted. */
CAVITY_API int cavity_destroy(cavity_t *h);

/* Static description of a status code. */
CAVITY_API const char *cavity_strerror(int code);

/* Last error message recorded on a handle (empty string if none). */
CAVITY_API const char *cavity_last_error(cavity_t *h);

#ifdef __cplusplus
}
#endif

#endif /* BDC_CAVITY_H */
