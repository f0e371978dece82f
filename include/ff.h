/*
 * ff.h -- C ABI of the GB300 Fireflies hot path.
 *
 * Fireflies (Merrison-Hort, arXiv 1505.00344) visualises an N-dimensional ODE
 * by integrating millions of independent trajectories ("particles") with a
 * constant-step fourth-order Runge-Kutta method and drawing each particle's
 * current state as a point of light.  This library is that data-parallel path
 * on one GPU: seed particle groups, step them forward or backward in time,
 * change parameters between steps, project onto a 2D or 3D view and splat into
 * a point-density image.  Every step runs in hand-written CUDA kernels for
 * sm_103a.
 *
 * Conventions that hold for every entry point:
 *   - Return value: FF_OK, or an error code with a message available from
 *     ff_last_error() (per thread).  Arguments are checked on the host before
 *     anything is enqueued; a rejected call changes nothing.
 *   - Ownership: a system owns its particle state and group tables (device
 *     memory allocated by ff_create_system).  Buffers passed in by the caller
 *     (images, state copies, parameter vectors) stay owned by the caller and
 *     are only borrowed for the duration of the call.
 *   - Streams: all device work of a system is enqueued on the CUDA stream
 *     given at creation (NULL = the legacy default stream).  Calls return after
 *     enqueueing unless documented as synchronising.
 *   - Device: a system is bound to the device that was current when it was
 *     created; every call makes that device current for its own work and
 *     restores the caller's device before returning.
 *   - Threads: a system must not be used from two threads at once.
 *   - Numerics: state is single precision (the paper's choice, Appendix A);
 *     parameters are accepted in double and rounded to float for the kernels;
 *     simulated time is accumulated in double on the host.
 */
#ifndef FF_H
#define FF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ff_status {
    FF_OK = 0,
    FF_ERR_INVALID_ARG = 1,  /* a pointer, size, index or value is out of range */
    FF_ERR_CUDA = 2,         /* a CUDA call or kernel launch failed */
    FF_ERR_OOM = 3,          /* device or host allocation failed */
    FF_ERR_STATE = 4,        /* the call is not allowed in the system's current state */
    FF_ERR_UNSUPPORTED = 5,  /* valid request that this build does not implement */
    FF_ERR_TIMEOUT = 6       /* a bounded device wait gave up */
} ff_status;

/* Right-hand sides f(x, p).  Parameter vectors (length n_params) in order:
 *   FF_RHS_LINEAR        dim 1..8, dx/dt = A x, p = A row-major (dim*dim).
 *   FF_RHS_HARMONIC      dim 2, (x, v): dx = v, dv = -w^2 x; p = [w].
 *   FF_RHS_WILSON_COWAN  dim 2, paper Eq. 1-2 as an E-I pair:
 *                        tauE dE = -E + S(wEE E - wEI I + P),
 *                        tauI dI = -I + S(wIE E - wII I + Q),
 *                        S(a) = 1 / (1 + exp(-gain (a - threshold)));
 *                        p = [wEE, wEI, wIE, wII, P, Q, tauE, tauI, gain, threshold].
 *   FF_RHS_LORENZ        dim 3, paper Eq. 3-5; p = [sigma, r, beta].
 *   FF_RHS_HH3           dim 15, three Hodgkin-Huxley neurons (paper Eq. 6-11)
 *                        with state (V, m, h, n, s) per neuron, rate functions
 *                        of Hodgkin & Huxley 1952 with rest near -65 mV and
 *                        all-to-all synaptic coupling sum_{j != i} s_j;
 *                        p = [C, gNa, gK, gL, ENa, EK, EL, gsyn, Esyn, I1, I2, I3,
 *                             tau_r, tau_d, sig, theta]. */
enum { FF_RHS_LINEAR = 0, FF_RHS_HARMONIC = 1, FF_RHS_WILSON_COWAN = 2, FF_RHS_LORENZ = 3,
       FF_RHS_HH3 = 4 };

/* Time steppers: classical RK4 (the paper's solver, Sec. 2.1) or explicit Euler. */
enum { FF_RK4 = 0, FF_EULER = 1 };

/* ff_create_system flags. */
#define FF_FLAG_KAHAN 1u  /* compensated (Kahan) summation of the state update */

#define FF_MAX_DIM 16
#define FF_MAX_PARAMS 64
#define FF_MAX_GROUPS 16

typedef struct ff_system ff_system;

/* A render technique (paper Appendix A): which state variables are drawn and
 * how they map to pixels.
 *   ndim_view = 2: column = floor((x[axes[0]] - lo[0]) * (width  / (hi[0]-lo[0]))),
 *                  row    = floor((x[axes[1]] - lo[1]) * (height / (hi[1]-lo[1]))),
 *                  the scale factors formed in double and rounded to float,
 *                  every other operation in float with its own rounding.
 *   ndim_view = 3: clip = M [x[axes[0]], x[axes[1]], x[axes[2]], 1] with M the
 *                  column-major Model-View-Projection matrix mvp (element
 *                  (row j, col c) at mvp[4c + j], each row summed left to
 *                  right); particles with clip.w <= 0 are dropped; otherwise
 *                  (clip.x / clip.w, clip.y / clip.w) in [-1, 1) maps to the
 *                  image with the 2D rule.
 * A particle is drawn iff its pixel lies inside the image (this also drops
 * non-finite coordinates).  Row 0 is the bottom of the view (lo[1] / ndc -1).
 * An axis index equal to the system's dim selects the per-particle parameter
 * (the paper's extra state variable with zero time derivative).
 * group_mask bit g selects group g; accumulate = 0 clears the image first. */
typedef struct ff_view {
    int ndim_view;
    int axes[3];
    double lo[2];
    double hi[2];
    float mvp[16];
    int width;
    int height;
    uint32_t group_mask;
    int accumulate;
} ff_view;

/* Create a system: its right-hand side, parameter vector, stepper and room
 * for `capacity` particles (paper Appendix A, "Initialization": an array of
 * N * P single-precision values).  The state is stored structure-of-arrays,
 * one plane of `pitch` floats per state variable, pitch = capacity rounded up
 * to a multiple of 256.  cuda_stream is a cudaStream_t (or NULL).
 * Errors: FF_ERR_INVALID_ARG for an unknown rhs_id/method, a dim or n_params
 * that does not fit rhs_id, capacity < 1, non-finite parameters or unknown
 * flags; FF_ERR_OOM if device memory runs out. */
ff_status ff_create_system(int rhs_id, int dim, const double* params, int n_params, int method,
                           unsigned flags, int64_t capacity, void* cuda_stream, ff_system** out);

/* Release the system and its device memory (synchronises its stream). NULL is a no-op. */
ff_status ff_destroy_system(ff_system* sys);

/* Append a particle group (paper Appendix A, "Particle Group"): `count`
 * particles with initial conditions uniform in the box [lo[k], hi[k]) of each
 * state variable, integrated forward (direction +1) or backward (-1) in time.
 * Group particle j, state variable k takes draw n = j*dim + k + 1 of the
 * SplitMix64 stream seeded with `seed`; the top 24 bits give u in [0, 1) and
 * x = lo + (hi - lo) * u is formed in double and rounded to float.  Groups
 * occupy consecutive index ranges in creation order.  *group_id_out (may be
 * NULL) receives the group's index.
 * Errors: FF_ERR_STATE after the first ff_step (until ff_reset) or with
 * FF_MAX_GROUPS groups; FF_ERR_INVALID_ARG for count < 1, more particles than
 * the capacity, lo/hi NULL, non-finite or lo > hi, direction not +-1. */
ff_status ff_seed_particles(ff_system* sys, int64_t count, const double* lo, const double* hi,
                            int direction, uint64_t seed, int* group_id_out);

/* One contiguous slice of a larger particle group, for splitting one ensemble
 * across GPUs (one process per GPU, each holding a contiguous range of the
 * particle indices; the paper runs one GPU, Sec. 4): the `count` particles
 * appended are particles first .. first + count - 1 of a group of `total`
 * particles with this box, direction and seed.  Particle j of the slice takes
 * the draws of group particle first + j (n = (first + j)*dim + k + 1), and an
 * in-kernel reset (ff_set_reset) re-draws it as that group particle, so the
 * union of the slices is, bit for bit, the ensemble of a system that seeds the
 * whole group.  ff_seed_particles(sys, count, ...) is the slice (0, count).
 * Errors: as ff_seed_particles, and FF_ERR_INVALID_ARG unless
 * 0 <= first <= total - count. */
ff_status ff_seed_particles_slice(ff_system* sys, int64_t count, int64_t first, int64_t total, const double* lo,
                                  const double* hi, int direction, uint64_t seed, int* group_id_out);

/* Restart: re-seed every group from its box and seed, clear the Kahan
 * compensation and simulated times (the paper re-initialises the GPU when a
 * system is modified, Appendix A). Per-particle parameters are kept. */
ff_status ff_reset(ff_system* sys);

/* Dynamic bifurcation diagram (paper Sec. 2.1 and 2.2, last paragraphs):
 * parameter `param_index` becomes a per-particle value, particle i of the P
 * particles seeded so far getting lo + (hi - lo) * (i / (P - 1)) (double,
 * rounded to float; lo for P = 1).  param_index = -1 switches it off.
 * Errors: FF_ERR_INVALID_ARG for an index out of range or non-finite bounds;
 * FF_ERR_STATE if no particles are seeded. */
ff_status ff_set_particle_param(ff_system* sys, int param_index, double lo, double hi);

/* The same linspace for a system holding particles first .. first + P - 1 of
 * an ensemble of `total` (one GPU's share of a split ensemble): its particle j
 * gets lo + (hi - lo) * ((first + j) / (total - 1)), the value particle
 * first + j has in the whole ensemble.  ff_set_particle_param is the slice
 * (0, P).  Errors: as ff_set_particle_param, and FF_ERR_INVALID_ARG unless
 * 0 <= first <= total - P. */
ff_status ff_set_particle_param_slice(ff_system* sys, int param_index, double lo, double hi, int64_t first,
                                      int64_t total);

/* Same, with caller-supplied per-particle values (P floats, host or device). */
ff_status ff_set_particle_param_values(ff_system* sys, int param_index, const float* values,
                                       int values_is_device);

/* Copy the per-particle parameter values out (P floats, host or device; a
 * host copy synchronises).  *param_index_out (may be NULL) receives the
 * parameter they replace, -1 if none.  Errors: FF_ERR_STATE if no per-particle
 * parameter was ever set. */
ff_status ff_get_particle_param(ff_system* sys, float* dst, int dst_is_device, int* param_index_out);

/* Particle reset (paper Sec. 2.1 and Appendix A: a trajectory that leaves the
 * bounds of any state variable, or has not been reset for more than T_max, is
 * given new random initial conditions from its group's box).  The paper does
 * this on the CPU a batch per frame; here the integrator does it in-kernel:
 * after each step a particle's age grows by one step, and at global step
 * numbers (steps since the last ff_reset, counted over all ff_step calls) that
 * are multiples of check_every, a particle whose float state lies outside
 * [bound_lo[k], bound_hi[k]] for some k (or is not finite), or whose age has
 * reached ceil(t_max / |dt|) steps, is re-drawn: its r-th reset takes draws
 * n = (r * count + j) * dim + k + 1 of its group's SplitMix64 stream (j its
 * index in the group, count the group's size) -- the blocks after its
 * initial-condition draws -- and its age restarts at 0.
 *   bound_lo/bound_hi: dim values each (rounded to float), or both NULL for no
 *   bounds; t_max <= 0: no age limit; check_every >= 1 enables the reset,
 *   0 disables it.  Ages and reset counts start at 0 and are cleared by ff_reset
 *   and ff_set_state.  Resetting particles run the scalar integrator (one
 *   particle per thread).
 * Errors: FF_ERR_INVALID_ARG for check_every < 0, only one of the bounds
 * given, non-finite or inverted bounds, non-finite t_max; FF_ERR_OOM. */
ff_status ff_set_reset(ff_system* sys, const double* bound_lo, const double* bound_hi, double t_max,
                       int check_every);

/* Copy per-particle ages (steps since the last reset) and reset counts out (P
 * uint32 each, host or device; either may be NULL; a host copy synchronises).
 * Errors: FF_ERR_STATE if the reset was never enabled. */
ff_status ff_get_reset_state(ff_system* sys, uint32_t* age, uint32_t* resets, int dst_is_device);

/* Advance every particle by n_steps constant steps (RK4 or Euler) of size
 * direction_g * dt (paper Sec. 2.1; Appendix A "Running the Simulation":
 * negative steps integrate backward).  The integrator keeps each particle's
 * state in registers for all n_steps steps of a launch.  n_steps = 0 is a
 * no-op.  Errors: FF_ERR_INVALID_ARG for n_steps < 0 or non-finite dt;
 * FF_ERR_STATE if no particles are seeded; FF_ERR_CUDA on a launch failure. */
ff_status ff_step(ff_system* sys, int64_t n_steps, double dt);

/* Replace the system parameter vector between steps (paper Sec. 2.1 and
 * Appendix A: sliders write the parameter values; the change is seen by the
 * next step).  Ordered with ff_step on the system's stream.  A per-particle
 * parameter keeps overriding its entry.
 * Errors: FF_ERR_INVALID_ARG for a wrong n_params or non-finite values. */
ff_status ff_set_params(ff_system* sys, const double* params, int n_params);

/* Project every selected particle through `view` and add one count to its
 * pixel of the uint32 image [height][width] (paper Appendix A, vertex,
 * geometry and fragment shaders with additive blending).  image is a device
 * pointer (image_is_device = 1) or host memory (0; the call then stages the
 * image on the device and synchronises).
 * Errors: FF_ERR_INVALID_ARG for a NULL image/view, ndim_view not 2 or 3, an
 * axis out of range (or equal to dim without a per-particle parameter),
 * width/height < 1 or width*height >= 2^31, lo >= hi or non-finite bounds. */
ff_status ff_project_splat(ff_system* sys, const ff_view* view, uint32_t* image,
                           int image_is_device);

/* One frame: exactly ff_step(n_steps, dt) followed by
 * ff_project_splat(view, image, image_is_device), with the same results.  When
 * the group-uniform packed Lorenz kernel runs (plain RK4, 2 or 4 particles per
 * thread, 4-aligned groups, per-particle parameter absent or r, no reset, no
 * tape, device image) the projection and splat are fused into the last
 * integrator launch, which counts each particle from the registers that hold
 * its final state; otherwise the two calls run one after the other.  Errors:
 * those of ff_step and ff_project_splat. */
ff_status ff_step_splat(ff_system* sys, int64_t n_steps, double dt, const ff_view* view, uint32_t* image,
                        int image_is_device);

/* Soft sprites (paper Appendix A: the geometry shader emits a screen-facing
 * square around each projected particle, the fragment shader gives each of its
 * pixels an intensity falling off smoothly with the distance from the centre,
 * and glBlendFunc(GL_SRC_ALPHA, GL_ONE) adds intensity x colour to the pixel).
 * The particle's centre is the view's pixel coordinate before the floor (the
 * 2D window map, or the 3D map after the perspective divide), so sprites keep
 * a constant size on the screen.  Pixel (col, row) is sampled at its centre
 * (col + 1/2, row + 1/2); with q = d^2 / radius^2, computed in float with every
 * operation rounded on its own, a pixel with q < 1 gains
 *     gain * (1 - q)^2 * colour[g][k]     in channel k = 0..3
 * for a particle of group g; q >= 1 (the square's corners) gains nothing.
 * Colours may have any sign.  Sums are FP32 in an unspecified order. */
#define FF_SPRITE_MAX_RADIUS 32.0f
/* How the fragments are summed (the covered pixels and their weights are the
 * same; only the order of the FP32 additions differs):
 *   FF_SPRITE_DIRECT  one 16-byte global vector reduction per fragment;
 *   FF_SPRITE_TILED   particles binned by 32 x 32 pixel tiles, each tile summed
 *                     in shared memory and added to the image once (needs at
 *                     most 8192 tiles; FF_ERR_UNSUPPORTED otherwise);
 *   FF_SPRITE_AUTO    the direct technique, which measured faster on every
 *                     workload tried (L2 vector reductions outrun shared-memory
 *                     atomics on the dense tiles of an attractor). */
enum { FF_SPRITE_AUTO = 0, FF_SPRITE_DIRECT = 1, FF_SPRITE_TILED = 2 };
typedef struct ff_sprite {
    float radius;                    /* half-side of the square, pixels: 0 < radius <= 32 */
    float gain;                      /* factor on every contribution */
    float colour[FF_MAX_GROUPS][4];  /* channel weights of each group */
    int technique;                   /* FF_SPRITE_AUTO / DIRECT / TILED */
} ff_sprite;

/* Draw every selected particle of `view` as a soft sprite into the float image
 * [height][width][4] (channels interleaved).  view->accumulate = 0 clears the
 * image first; group_mask selects groups as in ff_project_splat.  image is a
 * device pointer aligned to 16 bytes (image_is_device = 1) or host memory (0;
 * the call then stages the image on the device and synchronises).
 * Errors: those of ff_project_splat; FF_ERR_INVALID_ARG for a NULL sprite, a
 * radius outside (0, 32], non-finite gain or colours, an unknown technique, or
 * a device image not aligned to 16 bytes; FF_ERR_UNSUPPORTED for
 * FF_SPRITE_TILED on an image of more than 8192 tiles. */
ff_status ff_project_sprites(ff_system* sys, const ff_view* view, const ff_sprite* sprite, float* image,
                             int image_is_device);

/* Copy the state out, SoA [dim][P] with P the number of seeded particles
 * (dst holds dim*P floats; host or device).  A host copy synchronises. */
ff_status ff_get_state(ff_system* sys, float* dst, int dst_is_device);

/* Overwrite the state of all P seeded particles from SoA [dim][P] (host or
 * device), e.g. to resume a checkpoint.  Clears the Kahan compensation. */
ff_status ff_set_state(ff_system* sys, const float* src, int src_is_device);

/* Statistics (synchronises): number of escaped particles (some component
 * non-finite or above 1e30 in magnitude), and the simulated time of the
 * forward and backward groups.  Any output pointer may be NULL. */
ff_status ff_stats(ff_system* sys, int64_t* n_escaped, double* t_fwd, double* t_bwd);

/* Size information: seeded particles, plane pitch, dim, groups (NULL-able). */
ff_status ff_system_info(ff_system* sys, int64_t* n_particles, int64_t* pitch, int* dim,
                         int* n_groups);

/* What the last ff_step or ff_step_splat on this system launched (the paper's
 * main loop, App. A "Running the Simulation", one integration call per frame;
 * this call only reports, it launches nothing).  All outputs are NULL-able:
 *   kernel, kernel_len   the integrator kernel of the call's last launch, its
 *                        demangled C++ name (e.g. "void ff::lorenz_rk4_x2u_kernel
 *                        <false, 2, true>(ff::IntegrateArgs)"), truncated to
 *                        kernel_len - 1 characters and NUL-terminated; "" before
 *                        the first launch;
 *   grid, block          that launch's grid and block size;
 *   fused_splat          1 if the projection and count splat ran inside that
 *                        launch (ff_step_splat on the fused path), else 0;
 *   integrator_launches  integrator launches the call made (a call is split at
 *                        ff_set_launch's max_steps_per_launch and at 2^30 steps);
 *   splat_launches       separate splat kernels of the last ff_step_splat or
 *                        ff_project_splat (0 when the splat was fused).
 * An ff_step of 0 steps launches nothing and leaves these values as they were.
 * Errors: FF_ERR_INVALID_ARG for a NULL system or kernel_len < 1 with a
 * kernel buffer; FF_ERR_CUDA if the runtime cannot name the kernel. */
ff_status ff_last_launch(ff_system* sys, char* kernel, int kernel_len, int* grid, int* block, int* fused_splat,
                         int64_t* integrator_launches, int64_t* splat_launches);

/* Launch shape of the integrator: particles per thread (1, 2 or 4; at 2 and 4
 * each plane is read with one 8- or 16-byte access, and RK4 on Lorenz, plain or
 * compensated, then runs two particles per packed f32x2 instruction; HH3 takes
 * 1 or 2, and plain RK4 at 2 runs all three neurons of two particles packed,
 * bit-identical to 1, when the pairs fill one wave (3 x 128 per SM; smaller
 * ensembles run one particle per thread); the default is 4 for RK4 on Lorenz, 2 when compensated,
 * 2 for plain RK4 on HH3, and 1 otherwise; 0 keeps the current value),
 * threads per block (a multiple of 32 up to 1024, default 512 for RK4 on
 * Lorenz and 256 otherwise, 0 keeps the current value; clamped to the kernel's
 * maximum, 512 for the 2- and 3-dimensional systems and 256 for LINEAR and
 * HH3, and narrowed in whole warps when the particles would not give every SM
 * a block, so that a small ensemble spreads over all SMs), resident blocks per
 * SM of the persistent grid (0 = as many as fit), and the most steps per
 * launch (0 = all steps of an ff_step call in one launch; launches are also
 * split at 2^30 steps).  Errors: FF_ERR_INVALID_ARG for values out of range. */
ff_status ff_set_launch(ff_system* sys, int particles_per_thread, int block, int blocks_per_sm,
                        int64_t max_steps_per_launch);

/* Gradients through the integration (not part of the paper): the discrete
 * adjoint of the RK4 / Euler map, for losses of the final states.
 *
 * ff_tape_begin starts recording at the current state: every later ff_step
 * stores a checkpoint of the state every checkpoint_every steps (1..256) and
 * whenever the parameters or dt changed since the last checkpoint, up to
 * max_steps steps in total; the checkpoints take
 * (ceil(max_steps / checkpoint_every) + 16) * dim * pitch floats (a later
 * ff_tape_begin reuses them when they are enough; ff_tape_end releases them).
 * The integrator writes the checkpoints inside its launches.  Every
 * system has an adjoint; FF_ERR_UNSUPPORTED while particle reset is on (a
 * re-draw is not differentiable).  ff_reset and ff_set_state end the tape.
 * Errors: FF_ERR_INVALID_ARG for checkpoint_every outside 1..256 or
 * max_steps < 1; FF_ERR_STATE without particles; FF_ERR_OOM. */
ff_status ff_tape_begin(ff_system* sys, int64_t checkpoint_every, int64_t max_steps);

/* Release the tape's memory (no-op without a tape). */
ff_status ff_tape_end(ff_system* sys);

/* Reverse sweep over the tape.  dL_dxT_dev: dL/dx at the current state, SoA
 * [dim][P] (device, contiguous); dL_dx0_dev receives dL/dx at the tape's start
 * (device, same layout; may be the same buffer); dL_dp_host receives n_params
 * doubles: dL/dp summed over all taped steps (parameters changed mid-tape are
 * treated as one vector), and with a per-particle parameter its entry is the
 * sum over particles of the derivatives with respect to their own values.
 * The recomputation runs plain FP32 steps from the checkpoints; the
 * per-particle parameter sums are FP64 and reduced in a fixed order.
 * Memory: for the 15-dimensional system the first call allocates a scratch
 * area for one recomputed chunk per resident thread, (resident threads) x
 * checkpoint_every x 40 floats for RK4 (10 for Euler): about 0.9 GB at
 * checkpoint_every = 100 on a 152-SM GPU; it is kept with the tape and
 * released by ff_tape_end.  The other systems' sweeps need none.
 * Synchronises.  Errors: FF_ERR_STATE without a tape or after it ended,
 * FF_ERR_INVALID_ARG for NULL buffers, FF_ERR_OOM, FF_ERR_CUDA. */
ff_status ff_backward(ff_system* sys, const float* dL_dxT_dev, float* dL_dx0_dev, double* dL_dp_host);

/* Batched stepping (not part of the paper): several systems -- each with its
 * own right-hand side, method, parameters, groups and particle count -- advance
 * together.  Members of one family (same right-hand side, method and presence
 * of a per-particle parameter) run in one persistent launch over a table of work tiles, each block taking tiles
 * round-robin; the families are parallel branches of one CUDA graph, captured
 * once per step count and replayed by every ff_batch_step with that count.
 * The systems keep owning their state; the batch borrows them until
 * ff_batch_destroy, and they must not be destroyed, re-seeded, taped (other
 * than by ff_batch_tape_begin) or given a particle reset, and must keep or
 * lack their per-particle parameter meanwhile (ff_batch_step then returns
 * FF_ERR_STATE).
 * Members run the scalar integrator (no packed Lorenz kernel, no fused splat).
 *
 * ff_batch_create: systems on one device, each with particles, no Kahan flag,
 *   no reset, no tape; cuda_stream orders the batch's work (NULL = legacy
 *   default stream).  Errors: FF_ERR_INVALID_ARG (NULL/duplicate systems,
 *   different devices), FF_ERR_UNSUPPORTED (Kahan, reset, tape), FF_ERR_STATE
 *   (no particles), FF_ERR_CUDA / FF_ERR_OOM.
 * ff_batch_step: n_steps (0..2^30) steps; dt[i] is the step of system i
 *   (host array of n_systems doubles).  Parameters set with ff_set_params
 *   take effect at the next call.  Asynchronous.
 * ff_batch_autotune: times every launch shape (particles per thread 1/2/4 for
 *   dimension <= 4, blocks of 64..512 threads) of each family on the members'
 *   own data for trial_steps steps (twice), keeps the fastest, then times the
 *   same trial split into 2 and 4 launches (steps per launch) and keeps a split
 *   if it is faster; restores the members' states exactly.  Synchronises.
 * ff_batch_describe: one line per family: members, launch shape, tiles, tuned
 *   rate (NUL-terminated, truncated to text_len).
 *
 * Batched gradients.  ff_batch_tape_begin starts every member's tape
 * (ff_tape_begin with the same arguments; on failure none is left started).
 * While taped, ff_batch_step runs in segments that end wherever a member's
 * chunk ends (every checkpoint_every steps, or where its parameters or dt
 * changed); the first launch of a chunk stores the member's checkpoint from the
 * state it loads.  ff_batch_backward then runs one reverse-sweep launch per
 * family over tiles of 128 particles of one member (80 for the 15-dimensional
 * system, whose family keeps one scratch area as ff_backward's, sized for its
 * longest chunk and released by ff_batch_destroy), with the arithmetic of
 * ff_backward (dL/dx0 bit-identical to it), and reduces each member's
 * parameter gradient over its tiles in a fixed order:
 *   dL_dxT_dev[i], dL_dx0_dev[i]: device SoA [dim_i][P_i] buffers of member i
 *     (host arrays of n_systems pointers; a member's two may alias);
 *   dL_dp_host: n_systems * FF_MAX_PARAMS doubles, member i's gradient at
 *     [i * FF_MAX_PARAMS + q] for q < its n_params (zeros after).
 *   Synchronises.  Errors: FF_ERR_STATE without a batch tape, FF_ERR_INVALID_ARG
 *   for NULL arrays or buffers.
 * ff_batch_tape_end ends every member's tape. */
typedef struct ff_batch ff_batch;
ff_status ff_batch_create(ff_system* const* systems, int n_systems, void* cuda_stream, ff_batch** out);
ff_status ff_batch_step(ff_batch* batch, int64_t n_steps, const double* dt);
ff_status ff_batch_autotune(ff_batch* batch, const double* dt, int64_t trial_steps);
ff_status ff_batch_describe(ff_batch* batch, char* text, int text_len);
ff_status ff_batch_tape_begin(ff_batch* batch, int64_t checkpoint_every, int64_t max_steps);
ff_status ff_batch_tape_end(ff_batch* batch);
ff_status ff_batch_backward(ff_batch* batch, const float* const* dL_dxT_dev, float* const* dL_dx0_dev,
                            double* dL_dp_host);
ff_status ff_batch_destroy(ff_batch* batch);

/* Instruction kinds of ff_pipe_rate. */
#define FF_PIPE_FFMA 0  /* fma.rn.f32: one lane operation (2 flops) per thread instruction */
#define FF_PIPE_FFMA2 1 /* fma.rn.f32x2: two lane operations per thread instruction */
#define FF_PIPE_EX2 2   /* ex2.approx.ftz.f32 (multi-function unit) */
#define FF_PIPE_RCP 3   /* rcp.approx.ftz.f32 (multi-function unit), each followed by an FP32 add,
                           since a chain of reciprocals alone is an involution the compiler removes */
#define FF_PIPE_LOGISTIC 4 /* 1 / (1 + 2^-a): ex2, add, rcp -- the sigmoid of the Wilson-Cowan
                              right-hand side; counts two operations (ex2 and rcp) per step */

/* Issue-rate microbenchmark of one instruction kind on `device` (not part of
 * the paper's method: it supplies the measured denominators of the
 * integrators' ALU rooflines, Table 1's per-step cost being their arithmetic).
 * Every thread of a full-occupancy grid runs eight independent dependency
 * chains of the instruction for 4,096 iterations; the launch is timed with
 * events after one warm-up launch.  *lane_ops_per_s receives the lane
 * operations per second over the whole device (an FFMA2 counts two, a logistic
 * step its two multi-function operations; multiply FMA rates by 2 for flops).  The call allocates a small buffer, creates and
 * destroys its own stream and events, synchronises, and takes a few
 * milliseconds.  Errors: FF_ERR_INVALID_ARG for a NULL output or unknown op,
 * FF_ERR_CUDA if the device cannot run it. */
ff_status ff_pipe_rate(int op, int device, double* lane_ops_per_s);

/* Most groups ff_count_escaped_noalloc accepts (its fixed scratch holds one
 * 64-bit counter per group: 2 KB per GPU). */
#define FF_NOALLOC_MAX_GROUPS 256

/* Count escaped particles per group without allocating any memory.  The paper
 * has no counterpart: this serves callers that may not allocate device memory
 * when they ask, e.g. a plugin handed device buffers by a host application
 * that owns the whole memory budget, a render loop that cannot afford the
 * device synchronisation cudaMalloc may imply, or code whose memory comes
 * from a fixed pool sized up front.
 *   state_dev     SoA state on the device, plane k at state_dev + k * pitch
 *                 (any device buffer, e.g. one filled by ff_get_state).
 *   dim, n_particles, pitch   planes, particles, floats between planes.
 *   group_starts  host array of n_groups non-decreasing first indices,
 *                 group_starts[0] == 0; group g covers [starts[g],
 *                 starts[g+1]) and the last group ends at n_particles.
 *   n_groups      1 .. FF_NOALLOC_MAX_GROUPS.
 *   cuda_stream   stream for the work (NULL = legacy default stream).
 *   counts_out    host array of n_groups int64: escaped particles per group,
 *                 with the escape test of ff_stats (a component non-finite or
 *                 above 1e30 in magnitude).
 * The call synchronises the stream before returning, and it copies the
 * counts to pageable host memory.  It calls no cudaMalloc or cudaFree: its
 * only scratch is a fixed device array of FF_NOALLOC_MAX_GROUPS counters in
 * the library, present on every GPU that loads the library until the process
 * exits.  The first call on each device does a one-time set-up: it looks up
 * that array's device address (cudaGetSymbolAddress) and keeps it for the
 * process, so make that first call on a device before any stream capture
 * begins.  After cudaDeviceReset on a device the kept address is stale, so do
 * not call this entry point on that device again.
 * All calls on a device share the array and each clears the counters it
 * uses: calls that overlap on the GPU (concurrent streams or threads) race
 * and give wrong counts.
 * Errors: FF_ERR_INVALID_ARG for NULL pointers, dim outside 1..FF_MAX_DIM,
 * n_particles < 0, pitch < n_particles, n_groups outside
 * 1..FF_NOALLOC_MAX_GROUPS, or badly ordered group_starts; FF_ERR_CUDA if a
 * CUDA call fails. */
ff_status ff_count_escaped_noalloc(const float* state_dev, int dim, int64_t n_particles, int64_t pitch,
                                   const int64_t* group_starts, int n_groups, void* cuda_stream,
                                   int64_t* counts_out);

/* Message describing the last error returned on the calling thread. */
const char* ff_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FF_H */
