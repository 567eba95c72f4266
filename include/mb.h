/*
 * mb.h — C ABI of the GB300 multiblob inertial-coupling library (libmb.so).
 *
 * The library advances neutrally buoyant multiblob colloids coupled to an incompressible
 * fluid on a periodic staggered (MAC) grid, following Vazquez-Quesada, Balboa Usabiaga and
 * Delgado-Buscalioni, "A multiblob approach to colloidal hydrodynamics with inherent
 * lubrication" (arXiv:1407.5600).  Section and equation labels below are that paper's.
 *
 * Common rules for every entry point
 * ----------------------------------
 *  - Status: every call returns an mb_status and never aborts the process.  On any error
 *    the context is left as it was before the call and mb_last_error() describes the error.
 *  - Streams: all device work is enqueued on the CUDA stream given to mb_create_grid and is
 *    ordered with respect to other work on that stream.  A call that writes into HOST memory
 *    synchronises that stream before it returns.
 *  - Pointers: array arguments may be device pointers (on the context's device) or host
 *    pointers (pageable or pinned); the library finds out which with
 *    cudaPointerGetAttributes and stages host arrays through its own device buffers (the
 *    FP32-grid mb_step reads page-locked external forces directly instead).  Input arrays in
 *    device or page-locked memory are read in stream order, like cudaMemcpyAsync: keep them
 *    unchanged until the stream has reached the call.  The caller owns every array it
 *    passes; no caller pointer is used by work enqueued after the call returns.
 *  - Environment (read when a context is created; for comparisons and tuning, the defaults
 *    are the fast path): MB_FFT_PASSES=5 runs the fluid solve as five one-axis passes instead
 *    of three; MB_NO_GRAPH=1 launches every FP32-grid step directly instead of replaying its
 *    captured CUDA graph; MB_NO_AUTOTUNE=1 keeps the default spreading tile;
 *    MB_NO_FUSE_INTERP=1 runs the corrector and the next predictor as separate passes.
 *    MB_FAULT_ALLOC=k makes the k-th device allocation fail (tests of the error paths).
 *  - Layouts: blob arrays are [n][3] row-major FP64 (x, y, z).  A velocity or force grid of
 *    one box is 3 component arrays stored one after another, each [nz][ny][nx] with x
 *    fastest, in the context's grid precision (float for precision 0, double for 1); a
 *    batched grid is [batch] such boxes.  Component a lives on the faces normal to a:
 *    v_x[k][j][i] at (i h, (j+1/2) h, (k+1/2) h), v_y at ((i+1/2) h, j h, (k+1/2) h),
 *    v_z at ((i+1/2) h, (j+1/2) h, k h).  Blob positions are taken modulo the box.
 *  - Kernel: every blob-grid coupling uses delta_h(r) = h^-3 prod_a Phi(r_a / h), Eq. (delta),
 *    with Phi the three-point Peskin function of Roma, Peskin and Berger.
 */
#ifndef MB_H
#define MB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mb_ctx mb_ctx;

typedef enum {
    MB_OK = 0,
    MB_EINVAL = 1,   /* an argument is out of range or inconsistent */
    MB_ENOMEM = 2,   /* a device or host allocation failed */
    MB_ECUDA = 3,    /* a CUDA call or kernel launch failed */
    MB_ESTATE = 4,   /* the call is not valid in the context's current state */
    MB_ETIMEOUT = 5  /* a bounded device-side wait gave up */
} mb_status;

/* Grid and fluid description.
 *   nx, ny, nz   cells per box side: powers of two in [4, 256].  Sides above 128 run the
 *                fluid solve as five one-axis passes (see MB_FFT_PASSES above).
 *   batch        number of independent periodic boxes B >= 1 sharing the same geometry.
 *   h            mesh size (> 0); box side L_a = n_a h.
 *   rho, eta     fluid density and shear viscosity (> 0).
 *   dt           time step (> 0).
 *   precision    0: grid, spreading, interpolation and FFT in FP32 (blob positions, forces and
 *                the mean fluid momentum stay FP64); 1: FP64 storage and arithmetic, except
 *                that the FFT of grids with every side at most 128 computes in double-float
 *                (a pair of floats, about 48 significant bits; its error stays near 1e-14
 *                relative), where grid values below 2^-74 in magnitude keep 24 bits.
 *   deterministic  0 or 1.  With precision 1, 1 makes a run bitwise reproducible: blobs are
 *                ordered within their bin cells and spreading accumulates in 64-bit fixed point
 *                (order-independent sums); every other stage already has a fixed order.  In
 *                FP32-grid mode the flag has no effect: the in-cell order, the spring sums at
 *                an icosahedron's centre and the grid additions of neighbouring spreading
 *                tiles follow the order of atomics, so runs agree to FP32 rounding.
 *   advection    0, or 1 for the convective stress rho v v of Eq. (vf) (integrator 0 only;
 *                every measurement in the paper is at vanishing Reynolds number, so it is off
 *                by default).  It enters the momentum right-hand side as -rho D.M(v^n)
 *                (explicit in time), M placed like the thermal stress: M_aa at cell centres,
 *                the square of the mean of the two v_a faces; M_ab (b != a) on the (a, b)
 *                edges, v_a averaged along b times v_b averaged along a.  This centred
 *                conservative form keeps momentum exactly and, for a divergence-free field,
 *                kinetic energy.  mb_fluid_update includes it too.
 *   mean_mode    0: the k = 0 fluid mode carries the net momentum, rho L^3 d(mean v)/dt =
 *                sum of blob forces (+ mean body force); 1: the k = 0 mode is held at zero
 *                (the frame of Hasimoto's periodic drag, Eq. rhinf).
 *   kT           thermal energy, >= 0.  kT > 0 adds the fluctuating stress of Sec. 3 (the
 *                Gaussian stress sigma~ of Eq. vf; integrator 0 only): every step the fluid
 *                receives -D.sigma~ with sigma~ = sqrt(2 eta kT/(h^3 dt)) W, W a
 *                non-symmetric 3x3 tensor of standard normals per cell (W_aa at cell
 *                centres, W_ab on the edges at integer a and b coordinates), so that the
 *                fluid velocity samples Eq. (ef), variance kT/(rho h^3) per projected mode.
 *                The normals of box b at step index n are drawn for groups of four cells
 *                along x (cell m = 4 G + r, x fastest): five Philox4x64-10 blocks, key
 *                (seed, 0), counters (G, n, b, j), j = 0..4, give the 64-bit words
 *                x0..x19; word x_p gives the Box-Muller pair p (u1 = (low 32 bits + 1/2)/
 *                2^32, u2 = (high 32 bits + 1/2)/2^32, normals z_2p, z_2p+1 =
 *                sqrt(-2 ln u1) (cos, sin)(2 pi u2)), and cell r takes z_9r .. z_9r+8 as
 *                W_xx, W_xy, W_xz, W_yx, W_yy, W_yz, W_zx, W_zy, W_zz.  No drift term is
 *                added (neutrally buoyant blobs, m_e = 0).
 *   seed         key of the thermal stress (see kT).
 *   integrator   0: the inertial coupling method (Sec. 3: fluid and blob inertia, midpoint
 *                predictor/corrector for the blobs, Crank-Nicolson for the fluid).  1: its
 *                Stokes limit (Sc -> infinity, the regime of the paper's viscosity runs): each
 *                half step solves the steady zero-mean Stokes flow of the current forces,
 *                v = P (-eta L)^{-1} (S F + f_body), and the blobs follow u = J v with the
 *                explicit midpoint rule; rho is not used, mean_mode must be 1, and the velocity
 *                field of the context is the flow of the last half step.  Each grid
 *                precision keeps its blob arithmetic (FP64 positions and forces with
 *                precision 1; float-float positions and FP32 forces with precision 0); the
 *                step adjoint is not provided for it. */
typedef struct {
    int nx, ny, nz;
    int batch;
    double h, rho, eta, dt;
    int precision;
    int deterministic;
    int advection;
    int mean_mode;
    double kT;
    uint64_t seed;
    int integrator;
} mb_grid_desc;

/* Creates a context: validates *desc, allocates every grid buffer on the current CUDA
 * device and zeroes the fluid velocity of all boxes.  cuda_stream is a cudaStream_t (NULL =
 * the legacy default stream).  *out receives the context, or NULL on error.  Problem
 * statement: Sec. 3, Eq. (vf) on a periodic box. */
mb_status mb_create_grid(const mb_grid_desc* desc, void* cuda_stream, mb_ctx** out);

/* Releases every buffer of ctx after synchronising its stream.  ctx may be NULL. */
mb_status mb_destroy(mb_ctx* ctx);

/* Sets the blobs of box `box` (0 <= box < batch), replacing any previous ones.
 *   pos          [n_blobs][3] blob positions q_i.
 *   particle_id  [n_blobs] particle index of each blob, in [0, n_particles); a particle is
 *                the set of blobs sharing an id (Sec. 2: 12 icosahedron vertices + centre).
 *   bonds        [n_bonds][2] box-local blob index pairs tied by harmonic springs of rest
 *                length rest_len[e] and stiffness k_spring (Fig. ico: hard springs).
 *   k_rep, r_cut soft repulsion k_rep (r_cut - r) r_hat between blobs of different particles
 *                closer than r_cut (0 disables it); r_cut <= min(nx, ny, nz) h / 2.
 * n_blobs may be 0 (an empty box).  The blob forces of a step are the spring, repulsion and
 * external forces evaluated at the midpoint positions. */
mb_status mb_set_particles(mb_ctx* ctx, int box, int64_t n_blobs, const double* pos,
                           const int32_t* particle_id, int64_t n_bonds, const int32_t* bonds,
                           const double* rest_len, double k_spring, double k_rep, double r_cut);

/* Advances all boxes by n_steps time steps of the neutrally buoyant inertial coupling method
 * (m_e = 0, so the blob-fluid force is minus the blob force, Eqs. blob1 and vf):
 *   u^n       = J(q^n) v^n                                   (no-slip, Eq. ju)
 *   q^{n+1/2} = q^n + dt/2 u^n
 *   F         = springs + repulsion + ext at q^{n+1/2}
 *   (rho/dt - eta/2 L) v^{n+1} = P[(rho/dt + eta/2 L) v^n + S(q^{n+1/2}) F + f_body]
 *   q^{n+1}   = q^n + dt J(q^{n+1/2}) (v^n + v^{n+1})/2
 * with L the 7-point Laplacian of each MAC component and P the exact discrete projection
 * onto divergence-free fields, solved by FFT.
 *   ext_blob_force  [total blobs][3] external blob forces, boxes in order (NULL = none); the
 *                   same forces are applied in every one of the n_steps.
 *   body_force      HOST array of 4 doubles {f0, axis, wave_dir, j} giving the force density
 *                   f0 sin(2 pi j x_w / L_w) along `axis`, x_w the node coordinate along
 *                   wave_dir (the viscosity protocol of Sec. 10), or NULL.
 * Every box must have had mb_set_particles called (possibly with 0 blobs). */
mb_status mb_step(mb_ctx* ctx, int n_steps, const double* ext_blob_force,
                  const double* body_force);

/* Reads the current state.  Each output may be NULL.
 *   blob_vel    [total blobs][3] u_i = J_i v at the current positions (Eq. ju).
 *   blob_pos    [total blobs][3] current positions, wrapped into [0, L).
 *   particle_U  [total particles][3] U0 = (1/N) sum_i u_i (Sec. 2), particles of box 0
 *               first, then box 1, and so on.
 *   grid_v      [batch] grids of the fluid velocity, in the context's precision. */
mb_status mb_get_velocities(mb_ctx* ctx, double* blob_vel, double* blob_pos,
                            double* particle_U, void* grid_v);

/* Particle translational and angular velocities: U0 = (1/N) sum u_i and Omega solving
 * I0 Omega = sum_i s_i x (u_i - U0), I0 = sum_i (s_i^2 1 - s_i s_i), s_i = q_i - q_0
 * (Sec. 3.2, Eqs. torque and miner0).  Both [total particles][3]; either may be NULL. */
mb_status mb_get_particle_velocities(mb_ctx* ctx, double* particle_U, double* particle_Omega);

/* Replaces the fluid velocity of all boxes ([batch] grids in the context's precision), for
 * example to resume from a checkpoint.  The field should be divergence-free. */
mb_status mb_set_velocity_field(mb_ctx* ctx, const void* grid_v);

/* Standalone spreading S (Sec. 2): grid_out = sum_i delta_h(r - q_i) F_i on one box of the
 * context's geometry.  pos, F are [n][3]; grid_out is one box grid (3 components). */
mb_status mb_spread(mb_ctx* ctx, int64_t n, const double* pos, const double* F, void* grid_out);

/* Standalone interpolation J (Eq. ju): u_out_i = sum over nodes of prod Phi * v, on one box
 * grid grid_v.  pos, u_out are [n][3]. */
mb_status mb_interp(mb_ctx* ctx, int64_t n, const double* pos, const void* grid_v,
                    double* u_out);

/* Standalone fluid update of one box (Eq. vf with the viscous stress, Crank-Nicolson):
 *   (rho/dt - eta/2 L) v_out = P[(rho/dt + eta/2 L) v_in + f + f_body - rho D.M(v_in)],
 * the last term only with advection = 1 (no thermal stress here).
 * The k = 0 mode follows the grid (mean_mode 0) or is zeroed (mean_mode 1).  v_in, f and
 * v_out are one box grid each; body_force as in mb_step (HOST, or NULL).
 * In a Stokes-limit context (integrator 1) it is the steady solve of that integrator,
 *   -eta L v_out = P[f + f_body], k = 0 mode zero,
 * and v_in is not read (may be NULL). */
mb_status mb_fluid_update(mb_ctx* ctx, const void* v_in, const void* f,
                          const double* body_force, void* v_out);

/* The midpoint positions q^{n+1/2} and blob forces F (springs + repulsion + external) of the
 * last step taken, each [total blobs][3]; either may be NULL.  Before the first step both
 * are undefined (MB_ESTATE). */
mb_status mb_get_forces(mb_ctx* ctx, double* blob_force, double* midpoint_pos);

/* Per-stage device timing for profiling.  With timing enabled, mb_step records a CUDA event
 * on the context stream between consecutive stages of every step (no synchronisation; every
 * 64th step waits for the previous 64 to finish and accumulates their times).  Enabling (or
 * disabling) resets the totals.  mb_get_stage_times waits for the recorded steps, then copies
 * up to max_stages totals (milliseconds) and call counts, and sets *n_stages to the number of
 * stages; mb_stage_name gives a stage's name ("" if out of range).
 * Stages, in launch order: interp_predict, bin, forces, force_sum, spread, fluid_stress,
 * fluid_x_fwd, fluid_y_fwd, fluid_z_solve, fluid_y_inv, fluid_x_inv, interp_correct. */
mb_status mb_set_stage_timing(mb_ctx* ctx, int enable);
mb_status mb_get_stage_times(mb_ctx* ctx, int max_stages, double* ms_total,
                             int64_t* calls, int* n_stages);
const char* mb_stage_name(int stage);

/* The step index n that keys the thermal stress of the next step (see kT above).  It starts
 * at 0 when the context is created and every step of a context with kT > 0 advances it by one;
 * setting it, together with mb_set_positions and mb_set_velocity_field, resumes a
 * fluctuating run from a checkpoint with the same noise.  The paper has no counterpart of
 * this index: it fixes the random-number stream that its Gaussian stress (Sec. 3) leaves
 * open.  mb_get_step_index waits for the context stream. */
mb_status mb_set_step_index(mb_ctx* ctx, uint64_t step);
mb_status mb_get_step_index(mb_ctx* ctx, uint64_t* step);

/* Number of CUDA kernels the context's steps have launched so far. */
mb_status mb_get_launch_count(const mb_ctx* ctx, int64_t* launches);

/* Replaces the blob positions of all boxes ([total blobs][3], the same blobs and order as set
 * by mb_set_particles), for example to resume from a checkpoint.  Positions are taken modulo
 * the box.  mb_get_forces is undefined until the next step. */
mb_status mb_set_positions(mb_ctx* ctx, const double* pos);

/* Reverse-mode derivative of one mb_step (the adjoint of the step map).  Given the state the
 * step started from (pos_n [total blobs][3], grid_v_n one box grid) and the gradients of a
 * scalar loss with respect to the state after the step, it overwrites
 *   grad_pos  (in: dL/dq^{n+1}; out: dL/dq^n)            [total blobs][3]
 *   grad_v    (in: dL/dv^{n+1}; out: dL/dv^n)            one box grid
 * and adds dL/dk_spring of this step to *grad_k_spring (may be NULL).  ext_blob_force and
 * body_force must be those of the forward step (either may be NULL).  The step is recomputed
 * from (pos_n, grid_v_n), then its stages are transposed in reverse order: the transpose of J
 * is h^3 S and of S is h^-3 J; the position derivatives of J and S use the derivative of the
 * kernel Phi (Eq. delta, Phi is C^1); the fluid update v^{n+1} = A v^n + T f has symmetric A
 * and T (Eq. vf: the projection P, the Laplacian and the CN factors are symmetric and commute),
 * so its transpose reuses the forward solver; the blob-force transpose is the force Hessian
 * applied to the incoming gradient (forces derive from a potential).  Provided for FP64
 * contexts (precision 1) with batch 1, integrator 0, kT = 0 and advection = 0; MB_EINVAL
 * otherwise.  Arrays may be host or device. */
mb_status mb_adjoint_step(mb_ctx* ctx, const double* pos_n, const void* grid_v_n,
                          const double* ext_blob_force, const double* body_force,
                          double* grad_pos, void* grad_v, double* grad_k_spring);

/* Adjoint of the blob velocities u = J(q) v (Eq. ju) at positions pos and field grid_v:
 * grad_pos += (du/dq)^T grad_u and grad_v += J^T grad_u = h^3 S(q) grad_u.  FP64 contexts with
 * batch 1.  Arrays may be host or device. */
mb_status mb_velocity_adjoint(mb_ctx* ctx, const double* pos, const void* grid_v,
                              const double* grad_u, double* grad_pos, void* grad_v);

/* Adjoint of the particle velocities U0_p = (1/N_p) sum_{i in p} J_i(q) v (Sec. 2, the
 * translational velocity of a particle as the mean of its blob velocities, with Eq. ju) at
 * positions pos and field grid_v:
 *   grad_pos [total blobs][3] += (dU0/dq)^T grad_U,
 *   grad_v   one grid (context precision) += (dU0/dv)^T grad_U,
 * grad_U being [total particles][3].  Equivalent to mb_velocity_adjoint with
 * grad_u_i = grad_U_p(i) / N_p(i).  FP64 contexts with batch 1; arrays may be host or device;
 * MB_EINVAL for null arrays or other contexts. */
mb_status mb_particle_velocity_adjoint(mb_ctx* ctx, const double* pos, const void* grid_v,
                                       const double* grad_U, double* grad_pos, void* grad_v);

/* Spreading tile (nodes per block along x, y, z) in use and the fastest time of one spreading
 * launch with it when it was chosen (0 if not timed).  In FP32-grid mode the first step after
 * mb_set_particles times a set of candidate tile shapes on the actual blob distribution, in
 * several rounds, and keeps the one with the fastest launch (synchronising the stream after
 * each timed launch; set MB_NO_AUTOTUNE=1 to keep the default); choices are cached per
 * geometry and blob count for the life of the process. */
mb_status mb_get_tuning(const mb_ctx* ctx, int* spread_tile, float* spread_ms);

/* Number of blobs and particles of all boxes together. */
mb_status mb_get_counts(const mb_ctx* ctx, int64_t* total_blobs, int64_t* total_particles);

/* Spreading that allocates nothing.  The paper has no counterpart: this entry point exists
 * for callers that cannot allocate device memory (a plugin running inside another framework's
 * memory budget, or code that must not trigger an allocation mid-run).  It needs no context:
 * it computes the same grid_out = sum_i delta_h(r - q_i) F_i as mb_spread, for one box of the
 * geometry in *desc (only nx, ny, nz, h and precision are read), using a fixed scratch array
 * compiled into the library instead of buffers it would otherwise have to allocate.
 *   pos, F       [n][3] FP64 DEVICE arrays (positions are taken modulo the box).
 *   grid_out     one box grid (3 components, desc->precision) in DEVICE memory, overwritten.
 *   cuda_stream  stream of the current device the work is enqueued on (NULL = legacy default
 *                stream); a stream of another device is rejected with MB_EINVAL.
 * Limits: 0 <= n <= 262144 blobs, grids up to 128^3; larger sizes, host pointers and device
 * pointers of a GPU other than the current device are rejected with MB_EINVAL.  The scratch array (about 5 MiB) is held by every GPU that loads
 * the library until the process exits.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) and caches it; make that first call before any stream
 * capture.  Every call reuses the same array, so calls that overlap on the GPU (on different
 * streams, or from different threads) race and corrupt each other's results.  Errors are
 * reported through mb_last_error(NULL). */
mb_status mb_spread_static(const mb_grid_desc* desc, int64_t n, const double* pos,
                           const double* F, void* grid_out, void* cuda_stream);

/* Message of the last error on ctx (or, when ctx is NULL, of the last failed context-free
 * call: mb_create_grid or mb_spread_static).  The string stays valid until the next call on
 * ctx. */
const char* mb_last_error(const mb_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* MB_H */
