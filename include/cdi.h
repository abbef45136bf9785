/*
 * cdi.h -- C ABI of libcdi.so: one GPU time step of the conservative diffuse
 * interface (CDI) two-phase incompressible solver with the GNBC contact-line
 * treatment of Brown, Mirjalili, Khanwale & Mani, "A mass-conserving contact
 * line treatment for second-order conservative phase field methods based on
 * the generalized Navier boundary condition" (arXiv 2412.16843).
 *
 * Problem statement (Sec. 2 and Sec. 4 of the paper):
 *   d(phi)/dt + div(u phi) = div R,  R = gamma [eps grad phi - phi(1-phi) n]   Eq. (CDI)
 *   d(rho u)/dt + div[(rho u - S) x u] = -grad P + div[mu(grad u + grad u^T)]
 *                                        + F_ST                               Eq. (NS_momentum)
 *   div u = 0                                                                   Eq. (NS_incompressibility)
 *   F_ST = mu_c grad phi, mu_c from psi = eps ln(phi/(1-phi))                  Eqs. (EB), (chemical potential)
 *   walls: R.n = 0, u.n = 0, u_slip = u_slip^v + u_slip^Y (Model 4A)           Eqs. (no-flux BC), (no-penetration BC),
 *                                                                               (slip BC), (u_slip_v), (u_slip_Y)
 * on a uniform staggered grid (phi, p at cell centres, velocity components on
 * the faces normal to them), second-order central differences inside,
 * second-order one-sided wall-normal stencils in the wall rows, first-order
 * linear extrapolation of the slip-model quantities to the wall, classical
 * RK4 in time (Sec. 4).  The pressure solve is a geometric multigrid.
 *
 * Geometry: 2D grids are nx x ny with walls at y = 0 and y = ny*h; 3D grids
 * are nx x ny x nz with walls at z = 0 and z = nz*h.  All other axes are
 * periodic.  The spacing h = Lx/nx is uniform and must equal Ly/ny (and Lz/nz).
 *
 * Host array layout (every call that copies fields): contiguous, row-major,
 * x fastest, no halo.  Cell fields hold nx*ny(*nz) doubles.  The velocity
 * component normal to the walls (v in 2D, w in 3D) holds one extra face
 * plane: nx*(ny+1) in 2D, nx*ny*(nz+1) in 3D; its first and last planes lie
 * on the walls and are zero.  The tangential components hold nx*ny(*nz)
 * values; entry (i, ...) sits on the face between cells i-1 and i.
 *
 * Ownership: the library owns the context.  Device memory is ONE workspace
 * the caller allocates (size from cdi_workspace_bytes) and binds with
 * cdi_bind_workspace; the library allocates no device memory.  Host arrays
 * are copied in or out before the call returns; the caller keeps them.
 * All device work is issued on the stream given to cdi_bind_workspace.
 *
 * Errors: every call returns a cdi_status and never aborts, exits or traps.
 * cdi_last_error() holds a one-line description of the last failure.
 * No C++ exception crosses this interface.  Calls on one context are not
 * thread safe.
 */
#ifndef CDI_H
#define CDI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cdi_ctx cdi_ctx;

typedef enum {
    CDI_OK = 0,
    CDI_EINVAL = 1,   /* invalid argument (size, range, NaN parameter)            */
    CDI_ESTATE = 2,   /* call out of order (e.g. step before a workspace is bound) */
    CDI_ECUDA = 3,    /* a CUDA runtime call failed; the text says which           */
    CDI_ENOCONV = 4,  /* the pressure solve hit max_vcycles above its tolerance    */
    CDI_ENAN = 5,     /* a non-finite value appeared in the state                  */
    CDI_ETIMEOUT = 6  /* a bounded device-side wait gave up                        */
} cdi_status;

enum { CDI_FP64 = 0, CDI_FP32_MIXED = 1 };
enum { CDI_WALL_LO = 0, CDI_WALL_HI = 1, CDI_WALL_BOTH = 2 };
/* first guess of each pressure solve: the last solve's pressure, zero, the
 * same RK stage of the two previous steps extrapolated linearly in time, or
 * the prediction of the network attached with cdi_set_warm_unet
 * (launch-per-kernel execution) */
enum { CDI_WARM_PREV = 0, CDI_WARM_ZERO = 1, CDI_WARM_EXTRAP = 2, CDI_WARM_UNET = 3 };
/* how cdi_step runs: one persistent cooperative launch per call; one launch
 * per stencil kernel with each pressure solve one CUDA graph, its V-cycle
 * loop decided on the device (the host waits once per solve); or (default)
 * the first for grids up to 2^20 cells and the second above */
enum { CDI_EXEC_PERSISTENT = 0, CDI_EXEC_KERNELS = 1, CDI_EXEC_AUTO = 2 };
/* slip models of Sec. 3, Eqs. (Model 1A) .. (Model 4B); 4A is the default */
enum { CDI_MODEL_1A = 0, CDI_MODEL_1B, CDI_MODEL_2A, CDI_MODEL_2B,
       CDI_MODEL_3A, CDI_MODEL_3B, CDI_MODEL_4A, CDI_MODEL_4B };

/* Create a context for a dim-D grid (Sec. 4: uniform staggered Cartesian grid,
 * periodic sides, walls on the last axis).  dim is 2 or 3; nz is ignored in
 * 2D.  Every periodic extent must be even and >= 2, the wall extent >= 4;
 * multigrid coarsens all axes by 2 while every extent stays even and >= 2 and
 * the coarsest grid must hold at most 64 cells.  precision is CDI_FP64 or
 * CDI_FP32_MIXED (FP32 state and stencils, FP64 reductions, residuals and
 * coarse solve).  wall_mask must be 3 (both walls present).
 * On success *out owns a new context; on failure *out is NULL. */
cdi_status cdi_init_grid(cdi_ctx** out, int dim, int nx, int ny, int nz,
                         double Lx, double Ly, double Lz, unsigned wall_mask,
                         int precision);

/* Bytes of device workspace the context needs (256-byte aligned start). */
cdi_status cdi_workspace_bytes(const cdi_ctx* ctx, size_t* bytes);

/* Bind the caller's device workspace (at least cdi_workspace_bytes, 256-byte
 * aligned) and the CUDA stream (a cudaStream_t, NULL for the legacy default
 * stream) all later work runs on.  Zeroes the state (phi = 0, u = 0, p = 0). */
cdi_status cdi_bind_workspace(cdi_ctx* ctx, void* dev_ptr, size_t bytes,
                              void* cuda_stream);

/* Fluid properties: rho = (rho1-rho2) phi + rho2, mu = (mu1-mu2) phi + mu2
 * (Sec. 2), surface tension sigma (Eq. chemical potential), interface
 * thickness eps and regularisation strength gamma (Eq. CDI).  gamma >= 0 is
 * used as given; gamma < 0 selects gamma = max(2.5 |u|_max, -gamma) with
 * |u|_max the largest face velocity magnitude at the start of each step
 * (Sec. 5.1).  rho1, rho2 > 0; mu1, mu2 >= 0; eps > 0. */
cdi_status cdi_set_fluids(cdi_ctx* ctx, double rho1, double rho2, double mu1,
                          double mu2, double sigma, double eps, double gamma);

/* Wall properties (Eqs. slip BC, u_slip_v, u_slip_Y): equilibrium contact
 * angle theta_eq (radians, in (0, pi)), slip length l >= 0 giving the
 * friction beta_i = mu_i / l of each fluid (l = 0: no slip), and the wall's
 * x velocity U_wall (the tangential direction is +x on both walls).
 * wall is CDI_WALL_LO, CDI_WALL_HI or CDI_WALL_BOTH.  Call after
 * cdi_set_fluids (beta uses mu_i). */
cdi_status cdi_set_wall(cdi_ctx* ctx, int wall, double theta_eq_rad,
                        double slip_length, double U_wall);

/* The paper's own form of the wall friction: beta = (beta1-beta2) phi + beta2
 * (Sec. 2), beta1, beta2 > 0, or both +inf for no slip. */
cdi_status cdi_set_wall_beta(cdi_ctx* ctx, int wall, double beta1, double beta2);

/* Tangential wall velocity (Ux, Uy); Uy is used in 3D only. */
cdi_status cdi_set_wall_velocity(cdi_ctx* ctx, int wall, double Ux, double Uy);

/* Slip model of Sec. 3 (CDI_MODEL_*); Model 4A (Eq. u_slip_Y) by default. */
cdi_status cdi_set_model(cdi_ctx* ctx, int model);

/* Copy the phase field from host memory (cell layout above).  A value that is
 * not finite returns CDI_ENAN (checked on the device after the copy; the
 * field is then undefined). */
cdi_status cdi_set_phi(cdi_ctx* ctx, const double* phi_host);

/* Copy the face velocities from host memory (face layouts above); w is
 * ignored in 2D.  The wall planes of the wall-normal component are forced to
 * zero (Eq. no-penetration BC).  A value that is not finite returns CDI_ENAN
 * (checked on the device; the velocity is then undefined). */
cdi_status cdi_set_velocity(cdi_ctx* ctx, const double* u, const double* v,
                            const double* w);

/* Pressure solve controls: relative residual tolerance ||f - A p||_2 <=
 * tol ||f||_2, cap on V-cycles per solve, and the first guess
 * (CDI_WARM_PREV, CDI_WARM_ZERO, CDI_WARM_EXTRAP or CDI_WARM_UNET).  Setting
 * the state (cdi_set_phi, cdi_set_velocity) or the solver restarts the
 * extrapolation history. */
cdi_status cdi_set_solver(cdi_ctx* ctx, double tol, int max_vcycles, int warm);

/* Advance nsteps RK4 steps of size dt (Sec. 4): each stage evaluates the phi
 * flux, wall rows, momentum right-hand side, and projects the stage velocity
 * (4 pressure solves per step).  Returns CDI_ENOCONV, CDI_ENAN or
 * CDI_ETIMEOUT on the first failing step, which leaves the state undefined. */
cdi_status cdi_step(cdi_ctx* ctx, double dt, int nsteps);

/* Total phase volume sum(phi) h^dim, summed in FP64 in a fixed order
 * (Sec. 2: conserved by the no-flux and no-penetration walls). */
cdi_status cdi_mass(cdi_ctx* ctx, double* mass_out);

/* Contact angle and wetted length on one wall (Sec. 3.1: angle of the
 * phi = 0.5 contour with the wall, cos(theta) = -d_n psi / |grad psi|; Sec. 5.1:
 * wetted length).  phi and the psi gradient are linearly extrapolated to the
 * wall; the crossings of phi_w = 0.5 are found by linear interpolation,
 * scanning +x from the column of smallest phi_w.  2D: theta is the mean of
 * the two crossings and *wetted_len = x_R - x_L.  3D: theta is the mean over
 * every x line of the wall plane and *wetted_len is the diameter of the disc
 * of the wetted area.  No crossing: theta = NaN, wetted_len = 0. */
cdi_status cdi_contact_angle(cdi_ctx* ctx, int wall, double* theta_rad,
                             double* wetted_len);

/* Copy the state to host memory (any pointer may be NULL); p with its mean
 * removed (mean(p) = 0). */
cdi_status cdi_get_fields(cdi_ctx* ctx, double* phi, double* u, double* v,
                          double* w, double* p);

/* Stage-level evaluations on the current state (used by the parity tests):
 * right-hand sides of phi (cell layout) and of the face momentum (face
 * layouts) for the given gamma (gamma < 0: the step's rule). */
cdi_status cdi_eval_rhs(cdi_ctx* ctx, double gamma, double* rhs_phi,
                        double* rhs_u, double* rhs_v, double* rhs_w);

/* GNBC quantities on the current state: u^Y and the ghost velocity of every
 * tangential component, layout [wall][component][wall-plane position]
 * (wall-plane positions: nx in 2D, nx*ny in 3D, x fastest). */
cdi_status cdi_eval_wall(cdi_ctx* ctx, double* uY, double* ghost);

/* Pressure solve alone with the current phi: div(grad p / rho_f) = f - mean(f);
 * p holds the first guess on entry and the zero-mean solution on exit. */
cdi_status cdi_solve_pressure(cdi_ctx* ctx, const double* f, double* p);

/* Statistics of the last pressure solve: V-cycles, relative residual; and
 * of the last cdi_step call: largest V-cycle count of one solve and the
 * V-cycles of all its solves (any pointer may be NULL). */
cdi_status cdi_last_stats(cdi_ctx* ctx, int* vcycles, double* resid,
                          int* max_vcycles_step, int* total_vcycles_call);

/* Number of kernel launches the last cdi_step issued per time step, rounded
 * up (the persistent mode issues one launch per cdi_step call and reports 1). */
cdi_status cdi_launches_per_step(cdi_ctx* ctx, long* launches);

/* Execution mode of cdi_step: CDI_EXEC_PERSISTENT runs all steps of the call
 * in one cooperative launch with bounded grid barriers (a barrier that waits
 * longer than 2 s ends the call with CDI_ETIMEOUT); CDI_EXEC_KERNELS launches
 * every stencil and multigrid kernel separately; CDI_EXEC_AUTO (default)
 * takes the persistent launch for grids up to 2^20 cells, where launch
 * latency dominates, and separate kernels above, where the separate kernels
 * keep more warps resident for the bandwidth-bound sweeps.  All take the same
 * discretisation and solver; they order some FP32 operations of the V-cycle
 * differently, so their results agree to the pressure tolerance, not bit for
 * bit. */
cdi_status cdi_set_exec(cdi_ctx* ctx, int mode);

/* Red-black Gauss-Seidel sweeps before and after the coarse-grid correction
 * on every multigrid level (each in [1, 4]; default 1 and 1 in 2D, 1 and 2 in
 * 3D: measured fastest per step of a single 2D or 3D grid; in batched
 * execution, where an instance's barriers are CTA barriers, 2 and 2 measured
 * faster on the 2D sweep).  The solve
 * still iterates to its tolerance; the counts trade work per V-cycle against
 * V-cycles per solve. */
cdi_status cdi_set_smoothing(cdi_ctx* ctx, int npre, int npost);

/* Red-black sweeps before and after the coarse-grid correction on the levels
 * below the finest that the launch-per-kernel V-cycle runs as separate
 * launches (the levels the single-CTA tail takes, and the persistent and
 * batched kernels, keep the counts of cdi_set_smoothing).  Each in [0, 4]
 * with npre + npost >= 1; npre = npost = -1 (the default) takes the counts of
 * cdi_set_smoothing.  On these levels every sweep is two launches of a few
 * microseconds, so the counts trade launches against V-cycles per solve; the
 * solve still iterates to its tolerance.  Returns CDI_EINVAL outside those
 * ranges. */
cdi_status cdi_set_coarse_smoothing(cdi_ctx* ctx, int npre, int npost);

/* Relaxation factor omega of the finest level's red-black sweeps on the
 * launch-per-kernel path: each update is e <- e + omega (e_GS - e), e_GS the
 * Gauss-Seidel value (omega in (0, 2); default 1.15 on 3D grids, 1 on 2D
 * grids, where 1 is Gauss-Seidel).  A preconditioner setting: the solve
 * still iterates to its tolerance. */
cdi_status cdi_set_relaxation(cdi_ctx* ctx, double omega);

/* Smoother kernel of the finest multigrid level of 3D grids on the
 * launch-per-kernel path (the pressure solve of Eq. NS_incompressibility;
 * the solver is this library's choice): CDI_SWEEP_ONEPASS runs each
 * red-black Gauss-Seidel sweep as one launch that marches along z over
 * 64 x 16 tiles with planes staged in shared memory, reading the correction
 * from one buffer and writing it to another (both colours in one pass over
 * memory; needs nx a multiple of 64 and ny of 16); tiles whose halo lies
 * inside the grid stage each plane with TMA copies, the tiles on the periodic
 * seams with 16-byte cp.async copies; CDI_SWEEP_ONEPASS_CPASYNC is the same
 * sweep with cp.async staging on every tile; CDI_SWEEP_COLOUR runs one
 * launch per colour; CDI_SWEEP_AUTO (default) takes the one-pass sweep where
 * the grid has enough tiles to fill the GPU.  All compute the same
 * red-then-black update (each cell's terms in the same order).  A staged
 * copy that does not complete within its bounded wait (1 s) makes cdi_step
 * return CDI_ETIMEOUT. */
enum { CDI_SWEEP_AUTO = 0, CDI_SWEEP_ONEPASS = 1, CDI_SWEEP_COLOUR = 2, CDI_SWEEP_ONEPASS_CPASYNC = 3 };
cdi_status cdi_set_level0_sweep(cdi_ctx* ctx, int mode);

/* Longest wait (nanoseconds, 0 .. 6e10; default 2e9) of a grid barrier in the
 * persistent step kernel before the call ends with CDI_ETIMEOUT.  A timed-out
 * call leaves the state undefined but the context and the device usable. */
cdi_status cdi_set_barrier_timeout(cdi_ctx* ctx, long long ns);

/* Launch profiler (diagnostics): from now on record a CUDA event pair on the
 * launching stream around each of the next max_launches launches of one
 * kernel class ("step" = the persistent step kernel, one launch per cdi_step
 * call; separate kernels: "rbgs0" = red-black sweep on the finest level,
 * "mom", "phi_rhs", "wall", "cell", "psi", "stage_phi", "stage_mom", "div",
 * "rbgs", "resid_restrict0", "prolong0", "coarse", "resid", "project").
 * Creates events (host objects); allocates no device memory. */
cdi_status cdi_profile_start(cdi_ctx* ctx, const char* kernel, int max_launches);

/* Stop the launch profiler: total device time of the recorded launches (ms)
 * and their number.  Synchronises the stream. */
cdi_status cdi_profile_stop(cdi_ctx* ctx, double* total_ms, long* launches);

/* Text of the last error on this context ("" if none); NULL ctx gives the
 * last error of cdi_init_grid. */
const char* cdi_last_error(const cdi_ctx* ctx);

/* Release the context (not the caller's workspace). NULL is accepted. */
void cdi_destroy(cdi_ctx* ctx);

/* ---------------------------------------------------------------------------
 * Batched sweep: many independent problems (e.g. a theta_eq / slip length /
 * capillary number sweep) advanced together by ONE kernel launch.  Each
 * problem is an ordinary context (initialised, parameters set, workspace
 * bound, state set); the batch only schedules them: one CTA takes one
 * instance (largest first) and runs all its steps, so instances never wait
 * for each other.  The arithmetic of every instance is exactly that of
 * cdi_step (Sec. 4 time step), so results equal those of stepping each
 * context alone.  All instances need the same dimension and precision and
 * must stay alive while the batch exists.
 * ------------------------------------------------------------------------- */
typedef struct cdi_batch cdi_batch;

/* Create a batch over n contexts (the batch does not own them). */
cdi_status cdi_batch_create(cdi_batch** out, int n, cdi_ctx* const* instances);

/* Device workspace of the batch itself (instance descriptors and outcomes;
 * about 4 KB per instance). */
cdi_status cdi_batch_workspace_bytes(const cdi_batch* b, size_t* bytes);

/* Bind the batch workspace (256-byte aligned) and the stream of its launches. */
cdi_status cdi_batch_bind_workspace(cdi_batch* b, void* dev_ptr, size_t bytes,
                                    void* cuda_stream);

/* Advance every instance by nsteps RK4 steps; dt[i] is instance i's step.
 * Returns the first failing instance's status (its context holds the text). */
cdi_status cdi_batch_step(cdi_batch* b, const double* dt, int nsteps);

/* Threads per CTA of the batched kernel: 256, 512 (default) or 1024. */
cdi_status cdi_batch_set_threads(cdi_batch* b, int threads);

/* Shared-memory budget (bytes, 8 KiB .. the device's opt-in limit - 4 KiB;
 * default 100 KiB) of one CTA's multigrid tail: every instance's coarse
 * levels that fit run in shared memory inside the CTA; the larger the budget,
 * the more levels run there and the fewer CTAs fit on an SM. */
cdi_status cdi_batch_set_tail_budget(cdi_batch* b, size_t bytes);

/* Autotuner: time trial_steps steps of the whole batch for every pair of CTA
 * size (256, 512, 1024 threads) and tail budget (32 KiB, 64 KiB, 100 KiB and
 * the device's opt-in limit less 4 KiB) that launches, and keep the fastest;
 * ms_out (12 entries, [budget][CTA size], -1 where the pair does not
 * launch; may be NULL) receives the times.  The trial steps advance the
 * instances. */
cdi_status cdi_batch_autotune(cdi_batch* b, const double* dt, int trial_steps,
                              int* threads_out, size_t* tail_bytes_out, double* ms_out);

/* Outcome of instance i in the last cdi_batch_step: status, largest V-cycle
 * count of one solve, total V-cycles; and the launch's device time (ms). */
cdi_status cdi_batch_stats(cdi_batch* b, int i, int* status, int* max_vcycles,
                           int* total_vcycles, float* last_ms);

/* Last error of the batch (NULL: of the last failed cdi_batch_create). */
const char* cdi_batch_last_error(const cdi_batch* b);

/* Release the batch (not its contexts or workspace). NULL is accepted. */
void cdi_batch_destroy(cdi_batch* b);

/* ---------------------------------------------------------------------------
 * Learned first guess of the pressure solve (a form of the solver; the paper
 * has no network).  A 3D U-Net with four levels (16, 32, 64, 128 channels,
 * one 3x3x3 convolution per level with zero padding and ReLU, 2x2x2 average
 * pooling, nearest upsampling, skip connections by concatenation, a 1x1x1
 * head; 726,993 parameters) maps (f / rms(f), rho_f / max(rho1, rho2)) to
 * p / (rms(f) max(rho1, rho2) h^2) (h: grid spacing) for the pressure equation
 * div(grad p / rho_f) = f of the projection (Sec. 4).  Convolutions run on the
 * tensor cores with BF16 weights and activations and FP32 accumulation;
 * master weights and Adam moments are FP32.  Arrays are channels-last with x
 * fastest: input [nz][ny][nx][2], output [nz][ny][nx].  The prediction only
 * starts the multigrid solve, which still iterates to its tolerance.
 * ------------------------------------------------------------------------- */
typedef struct cdi_unet cdi_unet;

/* Create a network for nx*ny*nz grids; every extent a multiple of 8 and the
 * grid at most 2^28 voxels. */
cdi_status cdi_unet_create(cdi_unet** out, int nx, int ny, int nz);

/* Device workspace (parameters, gradients, Adam moments, activations). */
cdi_status cdi_unet_workspace_bytes(const cdi_unet* net, size_t* bytes);

/* Bind the workspace (256-byte aligned, cleared here) and the stream. */
cdi_status cdi_unet_bind_workspace(cdi_unet* net, void* dev_ptr, size_t bytes,
                                   void* cuda_stream);

/* Number of parameters (726,993). */
cdi_status cdi_unet_param_count(size_t* n);

/* Copy the parameters from / to host memory (n doubles, stored as FP32 on
 * the device).  Flat order: for the layers e0, e1, e2, b, d2, d1, d0, head,
 * the weights [taps][Cout][Cin] (tap (dz+1)*9 + (dy+1)*3 + (dx+1)) then the
 * biases [Cout].  Setting the parameters resets the Adam moments. */
cdi_status cdi_unet_set_params(cdi_unet* net, const double* params, size_t n);
cdi_status cdi_unet_get_params(cdi_unet* net, double* params, size_t n);

/* Forward pass on host arrays: x [N][2] -> y [N]. */
cdi_status cdi_unet_forward(cdi_unet* net, const double* x, double* y);

/* Forward pass on device arrays, FP32 x [N][2] -> FP32 y [N], issued on the
 * network's stream without host copies or synchronisation. */
cdi_status cdi_unet_forward_device(cdi_unet* net, const float* x, float* y);

/* One training step on host arrays x [N][2], target [N]: forward, the mean
 * squared error (written to loss before the update, may be NULL), the
 * gradients of every parameter (written to grads in the flat order when not
 * NULL) and, when lr > 0, one Adam step (b1 0.9, b2 0.999, eps 1e-8). */
cdi_status cdi_unet_train_step(cdi_unet* net, const double* x, const double* target,
                               double lr, double* loss, double* grads);

/* Kernels of the convolutions: 1 (default) the tcgen05 implicit GEMMs: the
 * 3x3x3 forward and data gradient (M = 128 voxels, accumulator in tensor
 * memory, input tile with halo staged once in shared memory for all 27 taps)
 * and every layer's weight and bias gradient (M = 128 rows of taps x input
 * channels plus a row of ones, N = output channels, K = voxels; voxel splits
 * added in a fixed order, no atomics); 0 the warp-level mma.sync implicit
 * GEMMs (weight gradients summed with FP32 atomics); 2 the tcgen05
 * convolutions with the mma.sync weight gradients (to compare the two weight
 * gradients on the same forward pass).  All compute the same sums in FP32. */
cdi_status cdi_unet_set_conv_kernel(cdi_unet* net, int tensor_core);

/* Last error of the network (NULL: of the last failed cdi_unet_create). */
const char* cdi_unet_last_error(const cdi_unet* net);

/* Release the network (not its workspace). NULL is accepted. */
void cdi_unet_destroy(cdi_unet* net);

/* Attach a network (NULL detaches) whose extents equal the context's grid
 * (3D only).  With CDI_WARM_UNET every pressure solve of cdi_step starts from
 * the network's prediction; cdi_step then launches kernel by kernel.  The
 * network must stay alive while attached and share the context's stream. */
cdi_status cdi_set_warm_unet(cdi_ctx* ctx, cdi_unet* net);

/* The right-hand side (mean removed) and the solution of the last pressure
 * solve of cdi_step or cdi_solve_pressure, cell layout (either pointer may
 * be NULL): training pairs for the network. */
cdi_status cdi_last_pressure(cdi_ctx* ctx, double* f, double* p);

/* Total phase volume sum(phi) * cell_volume of n doubles at phi_dev (device
 * memory), written as one double to mass_dev (device memory), with work
 * issued on cuda_stream (a cudaStream_t, NULL for the legacy default stream).
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory -- code running inside an allocator or
 * memory-pool callback, or in a program whose device memory is all reserved
 * up front -- and so cannot supply the workspace a context needs.  It
 * allocates nothing: its scratch (one FP64 partial per 8192 elements) is a
 * fixed 32 KiB array inside the library, present on every GPU that loads the
 * library until the process exits.  Hence n must lie in [1, 33554432];
 * other n returns CDI_EINVAL.  The first call on a device looks up the
 * scratch address on that device (make that first call before any stream
 * capture) and keeps it for the life of the process: a device reset while
 * the library is loaded is not supported.  A CUDA error already pending
 * from earlier work is reported as such (CDI_ECUDA) before any launch.  Every call on a device shares the scratch and leaves its partial
 * sums there; calls whose kernels overlap on the GPU race with each other.
 * Blocks sum fixed chunks in a fixed order, so the result is deterministic.
 * On failure a one-line message is copied into err (err_len bytes, may be
 * NULL). */
cdi_status cdi_mass_noalloc(const double* phi_dev, long long n, double cell_volume,
                            double* mass_dev, void* cuda_stream, char* err,
                            size_t err_len);

#ifdef __cplusplus
}
#endif

#endif /* CDI_H */
