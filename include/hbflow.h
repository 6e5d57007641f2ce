/* hbflow: one time step of Papanastasiou-regularised Herschel-Bulkley
 * incompressible flow on a uniform grid, on one GB300 GPU (sm_103a).
 *
 * Method: Sverdrup, Nikiforakis & Almgren, "Highly parallelisable simulations
 * of time-dependent viscoplastic fluid flow with structured adaptive mesh
 * refinement" (arXiv:1803.00417), Sec. III: the approximate projection method
 * with a Godunov edge-state predictor, a semi-implicit tensor viscous solve and
 * a nodal projection (Sec. III A, Eqs. 11-19), and the regularised viscosity
 * of Sec. III B (Eq. 23).
 *
 * Conventions for every entry point:
 *  - returns an hbf_status (0 on success); on failure hbf_last_error() holds a
 *    one-line reason.  Outputs are valid only on HBF_OK, except that
 *    HBF_ERR_NOT_CONVERGED leaves the last iterate and filled stats.
 *  - work is queued on the CUDA stream given to hbf_init_grid; calls that return
 *    solver statistics synchronise that stream (they read residual norms).
 *  - the context owns every device buffer it allocates; pointers passed in by
 *    the caller stay owned by the caller and are never freed by the library.
 *  - layouts: cell fields are structure-of-arrays, component-major, x fastest:
 *    element (c, i, j, k) of a d-component field sits at
 *    c*ncell + i + nx*(j + ny*k); nodal fields (pressure) have (nx+1)(ny+1)(nz+1)
 *    points, i + (nx+1)*(j + (ny+1)*k).  In 2D nz = 1 and k = 0.
 *  - every face of the box is a no-slip wall with a prescribed tangential
 *    velocity, except the faces normal to the axes made periodic by
 *    hbf_set_periodic.
 */
#ifndef HBFLOW_H
#define HBFLOW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hbf_ctx hbf_ctx;

enum hbf_status {
  HBF_OK = 0,
  HBF_ERR_ARG = -1,           /* invalid argument; nothing was done */
  HBF_ERR_OOM = -2,           /* device allocation failed */
  HBF_ERR_CUDA = -3,          /* a CUDA call failed; the message names it */
  HBF_ERR_NOT_CONVERGED = -4, /* a multigrid solve hit max_cycles */
  HBF_ERR_TIMEOUT = -5,       /* reserved: a bounded device-side wait gave up */
  HBF_ERR_NONFINITE = -6      /* a residual norm was NaN or Inf */
};

enum hbf_precision {
  HBF_FP64 = 0,  /* every solve in FP64 */
  HBF_MIXED = 1  /* FP64 defect correction around FP32 V-cycles */
};

/* Fields that can be copied in or out with hbf_set_field / hbf_get_field.
 * Sizes in doubles (hbf_field_size): U, USTAR, RHS, GP, LU: d*ncell; P: nnode;
 * ETA, PHI_MAC: ncell; UADV, UMAC: sum over axes a of nface[a] (axis-major);
 * UL, UR: sum over axes a of d*nface[a] (axis-major, then component);
 * ETA_FACES: sum over axes of nface[a]; SLOPES, HATS: d*d*ncell; NRES0: nnode;
 * VRES0, VCORR: d*ncell. */
enum hbf_field {
  HBF_U = 0,       /* cell velocity u^m (set) / u^{m+1} (after a step) */
  HBF_P = 1,       /* nodal pressure p^{m-1/2} / p^{m+1/2} */
  HBF_ETA = 2,     /* cell apparent viscosity eta^m (Eq. 23) */
  HBF_USTAR = 3,   /* provisional velocity u* (Eq. 16) */
  HBF_UADV = 4,    /* face advection velocity u^adv (normal component) */
  HBF_UMAC = 5,    /* MAC-projected face velocity u^MAC */
  HBF_RHS = 6,     /* right-hand side of the viscous solve (Eq. 16) */
  HBF_PHI_MAC = 7, /* MAC projection potential */
  HBF_GP = 8,      /* cell-centred G p^{m-1/2} */
  HBF_LU = 9,      /* div(eta^m (grad u^m + grad u^m^T)) at cells */
  HBF_UL = 10,     /* left face states (Eq. 14a) */
  HBF_UR = 11,     /* right face states (Eq. 14b) */
  HBF_ETA_FACES = 12, /* face eta of the finest level (axis-major) */
  HBF_SLOPES = 13, /* limited slopes, d*d*ncell, [axis][component] */
  HBF_HATS = 14,   /* transverse terms, d*d*ncell, [axis][component] */
  HBF_NRES0 = 15,  /* nodal projection: warm-start residual b - L p of the last hbf_project */
  HBF_VRES0 = 16,  /* viscous solve: b - A x at the start of the last solve, after the initial guess
                      (d*ncell; needs hbf_set_visc_record) */
  HBF_VCORR = 17   /* viscous solve: u* minus that starting point (d*ncell; needs hbf_set_visc_record) */
};

typedef struct {
  int cycles;      /* V-cycles (outer defect-correction iterations in mixed mode) */
  int converged;   /* 1 if ||b - A x||_inf <= rtol ||b||_inf */
  double r0;       /* initial residual norm */
  double rnorm;    /* final residual norm */
  double bnorm;    /* ||b||_inf (after removing the mean of a singular rhs) */
  int guess;       /* nodal projection: 1 if the learned initial guess was used */
} hbf_solve_stats;

typedef struct {
  hbf_solve_stats mac, visc, nodal;
} hbf_step_stats;

/* Create a context for a box of n[0] x n[1] (x n[2]) cells of size h, all
 * faces no-slip walls.  wall_u[(a*2 + s)*3 + c] is component c of the velocity
 * of the wall normal to axis a on side s (0 low, 1 high); its normal component
 * must be 0.  Every n[a] must be even (the multigrid coarsens by two down to at
 * least two cells per axis).  stream: a cudaStream_t, NULL for the default
 * stream.  precision: an hbf_precision.  Allocates all device buffers.
 * (Sec. IV: the lid-driven cavity; Sec. III A: cell-centred velocity, nodal
 * pressure.) */
int hbf_init_grid(hbf_ctx** out, int dim, const int64_t n[3], double h, const double wall_u[18],
                  int precision, void* stream);

/* Make axis a periodic (periodic[a] != 0) or bounded by walls (0), for the
 * channel flows with which the method is checked (plane Couette and Poiseuille
 * flow between walls, periodic along the flow).  A periodic axis needs an even
 * cell count; the walls normal to it are dropped (their velocities set to 0).
 * Nodal fields keep n+1 points along a periodic axis, the last a copy of the
 * first: fields set with hbf_set_field must repeat node 0 there (the library
 * keeps the copy equal).  Call before stepping; the exact bottom inverses are
 * rebuilt.  HBF_ERR_ARG for an odd count.  Not available in a batch. */
int hbf_set_periodic(hbf_ctx* ctx, const int periodic[3]);

/* Regularised Herschel-Bulkley law, Eq. 23 with mu -> K and 1/epsilon -> m:
 *   eta = (2^(n-1) K g^n + tau_y/2) F(g),  F(g) = (1 - exp(-m g))/g, F(0) = m,
 * g = |gamma_dot| = sqrt(1/2 tr(D D^T)) (Eq. 1).  reg_power = 0 regularises only
 * the yield term: eta = 2^(n-1) K g^(n-1) + tau_y/2 F(g) (then n >= 1).
 * Requires K >= 0, n > 0, tau_y >= 0, m > 0. */
int hbf_set_rheology(hbf_ctx* ctx, double K, double n, double tau_y, double m, int reg_power);

/* Constant density rho > 0 (Eq. 2b) and body force f (Eq. 2b, f^m in Eq. 15). */
int hbf_set_density(hbf_ctx* ctx, double rho);
int hbf_set_body_force(hbf_ctx* ctx, const double f[3]);

/* Include the explicit stress divergence in the edge-state forcing of Eq. 14
 * (1) or leave it out (0, default; see the library documentation). */
int hbf_set_predictor_viscous(hbf_ctx* ctx, int on);

/* Implicit weight theta of the viscous term: the solve of stage 6 is
 * (I - theta dt/rho L_eta) u* = u^m - dt [u.grad u] + dt/rho (-G p +
 * (1 - theta) L_eta u^m + f).  theta = 1/2 (default) is the Crank-Nicolson
 * form of Eqs. 15-16; theta = 1 is backward Euler, which damps the modes
 * with dt eta / (rho h^2) >> 1 that Crank-Nicolson leaves oscillating.
 * HBF_ERR_ARG outside [1/2, 1]. */
int hbf_set_theta(hbf_ctx* ctx, double theta);

/* Multigrid controls: stop when ||b - A x||_inf <= rtol ||b||_inf or after
 * max_cycles V-cycles; nu1/nu2 pre/post smoothing sweeps; nu_bottom sweeps on
 * the coarsest level.  Defaults 1e-10, 200, 2, 2, 40. */
int hbf_set_solver(hbf_ctx* ctx, double rtol, int max_cycles, int nu1, int nu2, int nu_bottom);
/* HBF_MIXED viscous solve (Eq. 16): each pass of the FP64 defect correction
 * runs the FP32 BiCGStab on A e = r until its residual has dropped by this
 * factor (or 40 iterations), then recomputes r in FP64.  Default 1e-3; FP32
 * limits a useful drop to about 1e-6.  HBF_ERR_ARG outside [1e-7, 1). */
int hbf_set_inner_drop(hbf_ctx* ctx, double drop);
/* HBF_MIXED viscous solve, 3D with walls on every axis and an even x extent:
 * on = 1 (default) keeps the FP32 finest-level vectors of the solve in the
 * colour-split layout (the cells with i + j + k even, then the odd ones, each
 * row-major with n_x / 2 cells per row), so that each red-black sweep reads
 * and writes unit-stride runs of one colour; on = 0 keeps the natural layout.
 * The values are the same bit for bit; only the memory traffic differs.  The
 * TMA-staged and one-launch sweep forms, when enabled, take the natural
 * layout.  HBF_ERR_ARG unless on is 0 or 1. */
int hbf_set_split_layout(hbf_ctx* ctx, int on);
/* The fused tail of the V-cycles (the multigrid scheme of Sec. III B): from
 * the first level with at most max_cells cells down to the exact bottom solve
 * and back runs as one launch of one thread block, with block barriers
 * between the colour sweeps; the arithmetic and its order are those of the
 * level-by-level launches.  0 disables it; default 512.  HBF_ERR_ARG for a
 * negative count. */
int hbf_set_tail(hbf_ctx* ctx, int max_cells);
/* The 3D FP32 finest-level viscous smoothing of HBF_MIXED contexts: 1 runs
 * each component's red-black Gauss-Seidel sweep (Sec. III A's tensor solve,
 * smoothed as in hbf_set_solver) as one launch that stages z-marching tiles
 * in shared memory and writes to a second array; 0 (default) runs the red
 * and the black cells as two launches in place.  The two give the same
 * update of every cell (bit for bit); the one-launch form reads 24 instead
 * of 36 bytes per cell but measured slower on GB300 (370 against 2 x 110 us
 * per 256^3 component sweep). */
int hbf_set_fused_sweep(hbf_ctx* ctx, int on);
/* The same two-launch red-black sweeps of the 3D FP32 finest level with their
 * operands staged in shared memory by the tensor memory accelerator: each
 * block owns a tile_x x 8-cell tile of a plane (tile_x 64 or 128) and streams
 * tile_z planes in z through a ring of shared-memory stages, so that the
 * loads of the next planes are in flight while the block updates the current
 * one.  Every interior cell's update is the same arithmetic on the same
 * values as in the unstaged sweeps (bit for bit).  Taken when the level has
 * walls on every axis and n[0] % 4 == 0 (the staged rows must start on
 * 16-byte boundaries); otherwise the unstaged sweeps run.  tile_x = 0
 * disables it (default).  A block whose bounded wait for its loads gives up
 * stops updating and the viscous solve returns HBF_ERR_TIMEOUT.
 * HBF_ERR_ARG for another width or tile_z outside [1, 4096]. */
int hbf_set_staged_sweep(hbf_ctx* ctx, int tile_x, int tile_z);
/* The 3D FP32 finest-level viscous operator u - beta L_eta u and residual
 * b - (u - beta L_eta u) of the mixed solve (the BiCGStab products and the
 * preconditioner's finest residual) with their operands staged the same way:
 * tiles of 64 x rows cells (rows 4 or 8) and tile_z planes per block.  Every
 * interior cell's value is the same arithmetic on the same values as in the
 * unstaged operator (bit for bit).  Taken under the rules of
 * hbf_set_staged_sweep; rows = 0 disables it.  A block whose bounded wait
 * gives up stops and the viscous solve returns HBF_ERR_TIMEOUT.  HBF_ERR_ARG
 * for other rows or tile_z outside [1, 4096]. */
int hbf_set_staged_op(hbf_ctx* ctx, int rows, int tile_z);

/* Number of doubles of a field (see enum hbf_field), or a negative status. */
int64_t hbf_field_size(const hbf_ctx* ctx, int which);

/* Copy a field in or out.  src/dst may be host or device pointers (unified
 * addressing); the copy is ordered on the context stream and the host side
 * must stay valid until hbf_sync. */
int hbf_set_field(hbf_ctx* ctx, int which, const double* src);
int hbf_get_field(hbf_ctx* ctx, int which, double* dst);

/* Stage 1 (Sec. III B, Eq. 23): eta^m from U. */
int hbf_compute_viscosity(hbf_ctx* ctx);

/* Stages 2-3 (Sec. III A, Eqs. 11-14): G p, div tau(u^m), limited slopes,
 * transverse terms, left/right face states and the advection velocity u^adv.
 * Needs ETA (hbf_compute_viscosity) for the current U. */
int hbf_predict(hbf_ctx* ctx, double dt);

/* Stage 4: MAC projection of u^adv: solve the cell-centred Poisson problem
 * D^MAC G^MAC phi = D^MAC u^adv (Neumann walls, mean-zero phi) and set
 * u^MAC = u^adv - G^MAC phi.  stats may be NULL. */
int hbf_mac_project(hbf_ctx* ctx, hbf_solve_stats* stats);

/* Stage 5 (Eqs. 15-16): upwind the face states with u^MAC, form the convective
 * term and the viscous right-hand side RHS. */
int hbf_advect_rhs(hbf_ctx* ctx, double dt);

/* Stage 6 (Eq. 16): solve (I - theta dt/rho L_eta) u = rhs (theta = 1/2
 * unless hbf_set_theta changed it) with the context's current ETA, L_eta u = div(eta (grad u + grad u^T)), walls at their
 * velocity.  rhs_dev, u_dev: device arrays of d*ncell doubles; u_dev holds the
 * initial guess on entry and the solution on exit.  stats may be NULL. */
int hbf_solve_viscous(hbf_ctx* ctx, double dt, const double* rhs_dev, double* u_dev,
                      hbf_solve_stats* stats);

/* Stage 7 (Eqs. 17-19): nodal projection.  Solves L phi = rho D(u/dt + G p/rho)
 * with the finite-element nodal Laplacian (Neumann walls, mean-zero phi), then
 * u <- u + dt/rho (G p - G phi) and p <- phi.  u_dev: device d*ncell doubles
 * (u* in, u^{m+1} out); p_dev: device nnode doubles (p^{m-1/2} in, also the
 * initial guess; p^{m+1/2} out).  stats may be NULL. */
int hbf_project(hbf_ctx* ctx, double dt, double* u_dev, double* p_dev, hbf_solve_stats* stats);

/* One full step m -> m+1 of stages 1-7 on the context's U and P.  stats may be
 * NULL.  Returns HBF_ERR_NOT_CONVERGED if any solve did not converge. */
int hbf_step(hbf_ctx* ctx, double dt, hbf_step_stats* stats);

/* dt = cfl h / max(max|u|, 1) for the current U (synchronises).  Returns NaN
 * (and hbf_last_error says why) when U holds a NaN or an Inf or a CUDA call
 * failed. */
double hbf_cfl_dt(hbf_ctx* ctx, double cfl);

/* Event timing of launches, per kernel class (slot):
 *   0 viscous smoother, 1 viscous residual/operator, 2 nodal smoother,
 *   3 nodal residual, 4 MAC smoother, 5 MAC residual (slots 0-5: finest level
 *   only), 6 explicit stages; with level 2 also 7 coarsest-level solves,
 *   8 transfers and conversions, 9 reductions, 10 Krylov vector updates,
 *   11 smoothing and residuals on coarse levels, 12 learned-guess sections
 *   (the network passes, their transfers and the acceptance tests, timed as
 *   whole regions whose launches also count in their own slots).
 * hbf_profile_enable(ctx, level) synchronises, clears the accumulators and
 * records at that level (0 off, 1 slots 0-6, 2 all); hbf_profile_read
 * synchronises and returns the summed device time in milliseconds and the
 * number of launches recorded for a slot. */
int hbf_profile_enable(hbf_ctx* ctx, int on);
int hbf_profile_read(hbf_ctx* ctx, int slot, double* total_ms, int64_t* launches);

/* Number of kernels the context has launched since it was created. */
int64_t hbf_launch_count(const hbf_ctx* ctx);

/* Allocation-free variant of hbf_cfl_dt for callers that cannot allocate
 * device memory: code recorded inside a CUDA graph capture (cudaMalloc is not
 * permitted there), hosts whose device memory belongs to another runtime's pool
 * allocator, or drivers that reserve every byte up front.  The paper has no
 * counterpart; it is a service of this library.
 *
 * Computes dt = cfl h / max(max_i |u_dev[i]|, 1) on the device and writes it to
 * dt_dev (one double in device memory).  u_dev: n doubles in device memory
 * (any layout, e.g. all velocity components).  stream: a cudaStream_t or NULL.
 * The work is queued on the stream; nothing is allocated and nothing
 * synchronises.
 *
 * Scratch: a file-scope device array of 32768 doubles (256 KiB), present on
 * every GPU that loads the library until the process exits, so
 * n <= HBF_NOALLOC_MAX_N (32768 * 2048 = 67,108,864 doubles); larger n returns
 * HBF_ERR_ARG without touching the GPU, as do null pointers or h, cfl <= 0.
 * The first call on a device looks up the array's device address (with that
 * device current) and caches it; make that first call before any stream
 * capture.  All calls share the one array and each overwrites the slots it
 * reads, so nothing carries over between calls, but calls whose GPU work
 * overlaps (different streams, or concurrent host threads) race on it.
 *
 * A NaN or Inf in u_dev makes *dt_dev NaN.  The call cannot report that in
 * its return value without waiting for the GPU, which a caller inside a
 * stream capture may not do; check the written dt (isnan) where that matters.
 * Returns HBF_OK, HBF_ERR_ARG, or HBF_ERR_CUDA (a launch failed, or an error
 * from earlier work was already pending: it is left for the caller to read
 * and nothing is launched). */
#define HBF_NOALLOC_MAX_N 67108864LL
int hbf_cfl_dt_noalloc(const double* u_dev, int64_t n, double h, double cfl, double* dt_dev, void* stream);

/* ---------------------------------------------------------------------------
 * Learned initial guess for the nodal projection solve (Eq. 17).  The paper
 * has no learned part; this network is an addition whose output only changes
 * the multigrid's starting point: the solve still runs to the same tolerance.
 *
 * A 4-level U-Net (16-32-64-128 channels, 3^d convolutions, ReLU, 2^d average
 * pooling, nearest upsampling with skip concatenation, 1x1 head) on a box of
 * n[0] x n[1] (x n[2]) points, each a multiple of 8.  BF16 weights and
 * activations, FP32 accumulation on the tensor cores, FP32 master weights.
 * Parameters are a flat FP32 vector, layer by layer: W[tap][c_out][c_in] then
 * b[c_out] for the 14 convolutions (taps in lexicographic order over
 * {-1,0,1}^d, x slowest; the first layer has c_in = 16 of which only channel 0
 * is used), then the head's 16 weights and 1 bias.  Arrays x, y, t, mask are
 * FP32 on the device, one value per point, x fastest.
 * ------------------------------------------------------------------------- */
typedef struct hbf_unet hbf_unet;

/* train = 0 allocates only what inference needs.  seed: He-normal init. */
int hbf_unet_create(hbf_unet** out, int dim, const int64_t n[3], int train, uint64_t seed, void* stream);
void hbf_unet_destroy(hbf_unet* net);
const char* hbf_unet_last_error(const hbf_unet* net);
int64_t hbf_unet_param_count(const hbf_unet* net);
/* copy the FP32 parameters (or, after backward, their gradients) out/in;
 * host or device pointers; synchronises */
int hbf_unet_get_params(hbf_unet* net, float* dst);
int hbf_unet_set_params(hbf_unet* net, const float* src);
int hbf_unet_get_grads(hbf_unet* net, float* dst);
/* Tensor-core path of the 3^d convolutions (forward and input-gradient):
 * 0 = warp-level mma.sync, 1 = tcgen05.mma with TMEM accumulators (default)
 * (128 points x Cout per CTA, operands staged in shared memory, completion
 * on an mbarrier with a bounded wait).  Both accumulate in FP32.  The weight
 * gradient always uses mma.sync. */
int hbf_unet_set_tensor_path(hbf_unet* net, int path);
/* Synchronises; HBF_ERR_TIMEOUT (and clears it) if a tcgen05 convolution
 * gave up waiting for the tensor cores since the last call, else HBF_OK. */
int hbf_unet_tensor_status(hbf_unet* net);
/* y = net(x); y_dev may be NULL (the output stays inside the network) */
int hbf_unet_forward(hbf_unet* net, const float* x_dev, float* y_dev);
/* masked mean squared error of the last forward output against t; writes the
 * output gradient to gy_dev and the loss to *loss (synchronises).  Returns
 * HBF_ERR_TIMEOUT (and clears the flag) when a tcgen05 convolution gave up
 * waiting for the tensor cores since the flag was last cleared: the forward
 * output, the loss and the gradient are then not valid. */
int hbf_unet_loss(hbf_unet* net, const float* t_dev, const float* mask_dev, float* gy_dev, double* loss);
/* accumulate parameter gradients of the last forward for output gradient gy */
int hbf_unet_backward(hbf_unet* net, const float* gy_dev);
int hbf_unet_zero_grads(hbf_unet* net);
/* one Adam step on the accumulated gradients, which it then clears */
int hbf_unet_adam(hbf_unet* net, double lr, double beta1, double beta2, double eps);

/* Use net (NULL disables) for the initial guess of every nodal projection
 * solve of ctx: with r0 = b - L p the warm-start residual, the candidate guess
 * is p + |r0|_inf net(r0 / |r0|_inf); it is kept only if its residual is
 * smaller than |r0|_inf, otherwise the solve starts from p (also when a
 * tcgen05 convolution of that forward pass gave up waiting for the tensor
 * cores, whose flag the step then clears).  The network's
 * box must hold the (n+1)^d nodes: each of its sizes >= n[a] + 1. */
int hbf_set_guess_model(hbf_ctx* ctx, hbf_unet* net);
/* The same with the network on the nodes of multigrid level `level` (0 = the
 * finest grid; each level halves the cells per axis): the warm-start residual
 * is restricted to that level by nodal full weighting, the network's output
 * is interpolated back to the finest nodes, and the step and acceptance rule
 * are as above.  A coarse level makes the network 2^(d*level) times cheaper;
 * the correction it has to predict is the smooth part.  The box must hold
 * that level's nodes.  HBF_ERR_ARG if the level does not exist. */
int hbf_set_guess_model_level(hbf_ctx* ctx, hbf_unet* net, int level);

/* ---------------------------------------------------------------------------
 * Initial guess of the viscous solve (Eq. 16) in HBF_MIXED contexts.  Not in
 * the paper: the solve starts from u^m there, and here too with mode 0.  The
 * guess only moves the starting point; the solve still runs to its FP64
 * tolerance.  From x = u^m and its residual r = b - A x, minimal-residual
 * steps along up to two directions d, each taken only if it lowers max |r|:
 * w = A d (homogeneous walls), alpha = (r, w)/(w, w), x += alpha d.
 *   mode 1: d = the previous step's increment u*^{m-1} - u^{m-1} (kept by
 *           hbf_step; cleared when U is set).  Where dt eta / (rho h^2) >> 1
 *           Crank-Nicolson leaves modes flipping sign from step to step, so
 *           alpha comes out near -1.
 *   mode 2: also the direction of the network set by
 *           hbf_set_visc_guess_model for the remaining residual.
 * hbf_solve_stats.guess of the viscous solve: bit 0 the increment's step was
 * taken, bit 1 the network's.  HBF_ERR_ARG for another mode or an FP64
 * context. */
int hbf_set_visc_guess(hbf_ctx* ctx, int mode);
/* The network of mode 2 (NULL disables): each velocity component of the
 * residual, divided by its max norm over all components, is restricted to
 * the cells of multigrid level `level` by averaging, mapped by one forward
 * pass, and the output interpolated back to the finest cells (multilinear,
 * odd reflection at the walls).  The network's box must hold that level's
 * cells (each size >= n[a] >> level). */
int hbf_set_visc_guess_model(hbf_ctx* ctx, hbf_unet* net, int level);
/* Keep the fields HBF_VRES0 and HBF_VCORR of every viscous solve of hbf_step
 * (training pairs for the network: the residual at the start and the
 * correction the solver found).  HBF_MIXED contexts. */
int hbf_set_visc_record(hbf_ctx* ctx, int on);
/* One level of the multigrid restriction applied to caller data (device
 * pointers): kind 0 a d-component cell field, 1 a cell scalar (mean of the
 * 2^d children), 2 a nodal field (full weighting); from level `level` to
 * level + 1.  HBF_ERR_ARG if level + 1 does not exist. */
int hbf_restrict(hbf_ctx* ctx, int kind, int level, const double* src, double* dst);

int hbf_sync(hbf_ctx* ctx);
const char* hbf_last_error(const hbf_ctx* ctx);
void hbf_destroy(hbf_ctx* ctx);

/* ---------------------------------------------------------------------------
 * Start-up, steady state and cessation of the lid-driven cavity (Sec. III A:
 * the steady criterion; Sec. IV: start-up from rest, steady state, the lid
 * stopped and the fluid brought to rest in finite time; yield surfaces,
 * stagnant and plug zones; Sec. IV and V: centre-line profiles and vortex
 * centres), and the checkpoint record of a context.  The diagnostics read
 * the context's current U and synchronise its stream.
 * ------------------------------------------------------------------------- */

/* Everything hbf_step reads besides U and P, plus the time and step count. */
typedef struct {
  int32_t dim;               /* 2 or 3 */
  int32_t precision;         /* an hbf_precision (informative on restore) */
  int64_t n[3];              /* cells per axis (n[2] = 1 in 2D) */
  double h;                  /* cell size */
  double t;                  /* time: sum of the dt of the steps taken */
  int64_t step;              /* steps taken (hbf_step, hbf_batch_step) */
  double K, nexp, tau_y, m;  /* as given to hbf_set_rheology */
  int32_t reg_power;
  int32_t predictor_viscous; /* hbf_set_predictor_viscous */
  double theta;              /* hbf_set_theta */
  int32_t periodic[3];       /* hbf_set_periodic */
  double rho;                /* hbf_set_density */
  double f[3];               /* hbf_set_body_force */
  double wall_u[18];         /* layout of hbf_init_grid */
} hbf_state;

/* Fill *state and, where not NULL, copy U (d*ncell doubles) and P (nnode
 * doubles) out to host or device memory.  Synchronises. */
int hbf_get_state(hbf_ctx* ctx, hbf_state* state, double* u, double* p);
/* Restore a record of hbf_get_state: dim, n and h must be the context's
 * (HBF_ERR_ARG otherwise; the precision may differ); sets the rheology,
 * density, body force, predictor form, walls, time and step count, and copies
 * U and P in where not NULL (host or device).  Synchronises. */
int hbf_set_state(hbf_ctx* ctx, const hbf_state* state, const double* u, const double* p);

/* Replace the wall velocities (layout and rules of hbf_init_grid): the
 * cessation study stops the lid this way.  HBF_ERR_ARG for a non-zero normal
 * component.  Also valid on a batch cavity (its tables are rebuilt). */
int hbf_set_walls(hbf_ctx* ctx, const double wall_u[18]);

/* The steady criterion of Sec. III A for the last hbf_step:
 * max|u^{m+1} - u^m| / max|u^m|.  The paper's pointwise quotient is undefined
 * where u^m = 0, so the two maxima are taken separately; +inf when u^m = 0.
 * HBF_ERR_ARG when U was set, or a batched step taken, since that step. */
int hbf_step_change(hbf_ctx* ctx, double* change);

typedef struct {
  double tau_max;     /* max over cells of |tau| = 2 eta |gamma_dot| (tau = 2 eta gamma_dot; norm of Eq. 1) */
  int64_t yielded;    /* cells with |tau| > tau_y */
  int64_t cells[3];   /* unyielded cells in stagnant [0], plug [1] and attached [2] zones */
  int64_t zones[3];   /* number of zones of each kind */
} hbf_yield_info;
/* Yield state of the current U, with eta(|gamma_dot|) of Eq. 23: a cell is
 * unyielded where |tau| <= tau_y (Sec. IV: the yield surface is the contour
 * |tau| = tau_0).  Unyielded cells sharing a face form zones: a zone touching
 * a wall at rest is stagnant, one touching no wall a plug (Sec. IV), one
 * touching moving walls only attached.  labels: NULL, or ncell int32 (host or
 * device, cell layout): -1 for a yielded cell, else the smallest cell index
 * of its zone. */
int hbf_yield(hbf_ctx* ctx, hbf_yield_info* info, int32_t* labels);

typedef struct {
  int64_t steps;          /* steps taken by the call */
  double t;               /* the context's time after the call */
  double change;          /* hbf_run_steady: the last step's change */
  double tau_ratio;       /* hbf_run_cessation: max |tau| / tau_y after the last step */
  double t_c;             /* hbf_run_cessation: time from the call to the first state with no yielded cell */
  double t_c_interp;      /* the same with max|tau|/tau_y = 1 interpolated linearly between the last two steps */
  int32_t reached;        /* 1 if the criterion was met within max_steps */
  int32_t not_converged;  /* steps at which a solve stopped at its cycle cap */
} hbf_run_info;

/* Start-up (Sec. IV): hbf_step(dt) until hbf_step_change falls below tol
 * (1e-5 in the paper) or max_steps steps were taken (then reached = 0).  An
 * error of a step other than HBF_ERR_NOT_CONVERGED ends the run and is
 * returned. */
int hbf_run_steady(hbf_ctx* ctx, double dt, double tol, int64_t max_steps, hbf_run_info* info);
/* Cessation (Sec. IV): set every wall at rest, then hbf_step(dt) until no
 * cell is yielded (t_c) or max_steps steps were taken.  The first damp_steps
 * steps use theta = 1 (backward Euler in the viscous term, see
 * hbf_set_theta), the rest the context's theta: stopping the lid excites
 * modes with dt eta / (rho h^2) >> 1, which Crank-Nicolson carries on with
 * an amplification factor near -1 (Rannacher's damped start after a
 * discontinuity; 0 keeps the context's scheme throughout).  HBF_ERR_ARG
 * without a yield stress.  Errors as for hbf_run_steady. */
int hbf_run_cessation(hbf_ctx* ctx, double dt, int64_t max_steps, int damp_steps, hbf_run_info* info);

/* Velocity component comp along the line parallel to axis `along` through
 * the box centre (Sec. IV and V centre-line profiles): n[along] values; across
 * each other axis the mean of the two middle cells for an even count, the
 * middle cell for an odd one.  out: host or device. */
int hbf_centreline(hbf_ctx* ctx, int comp, int along, double* out);
/* Stream function of the centre plane and the primary vortex centre
 * (Sec. IV, V A).  The plane is the box in 2D and the plane normal to y
 * through the centre in 3D (u_x averaged across y as for hbf_centreline);
 * (a, b) = (x, y) in 2D, (x, z) in 3D.  psi: NULL or (n_a+1)(n_b+1) doubles,
 * a fastest: psi = 0 on the low b wall and psi(i, j+1) = psi(i, j) + h u_x
 * with u_x on the a-face i of cell row j the mean of its two cells (0 on the
 * walls normal to a).  centre: the node where |psi| is largest (the smallest
 * index among ties), refined by a parabola through its two neighbours along
 * each in-plane axis, in coordinates of the plane (node k at k h); psi_c: psi
 * at that node. */
int hbf_vortex(hbf_ctx* ctx, double* psi, double centre[2], double* psi_c);

/* ---------------------------------------------------------------------------
 * Batched sweep: ncav independent cavities (sizes, rheology and time steps of
 * their own) each advanced by the step of hbf_step (Sec. III A) in one call.
 * The paper runs one problem at a time; batching is a service of this
 * library for parameter sweeps.  Every stage is one persistent kernel launch
 * over a work list of tiles (cavity, element range) spanning all cavities;
 * the multigrid levels of all cavities are smoothed together; each cavity
 * keeps its own solver state and tolerance and drops out of the launches once
 * it has converged.  Fixed launch sequences (the explicit stages, V-cycles)
 * are recorded once as CUDA graphs and replayed.  Per cavity the arithmetic
 * is the single-context step's; only the summation order of norms and dot
 * products differs.
 *
 * Each cavity must coarsen to an exact bottom solve: its coarsest level
 * (sizes halved while even and >= 4) has at most 128 unknowns in each of the
 * three solves, e.g. every size a power of two, or 3 * 2^k.  No learned
 * initial guess is used in the batch.
 * ------------------------------------------------------------------------- */
typedef struct hbf_batch hbf_batch;

/* dim 2 or 3; n: ncav x 3 cell counts (the third ignored in 2D); h: ncav cell
 * sizes; wall_u: ncav x 18 wall velocities laid out as for hbf_init_grid, or
 * NULL for resting walls; precision HBF_FP64 or HBF_MIXED (all cavities);
 * stream: a cudaStream_t, or NULL to let the batch create its own (graphs
 * need a stream other than the legacy default one).  Host arrays. */
int hbf_batch_create(hbf_batch** out, int dim, int ncav, const int64_t* n, const double* h, const double* wall_u,
                     int precision, void* stream);
void hbf_batch_destroy(hbf_batch* b);
/* Borrow cavity i's context for hbf_set_rheology / _density / _body_force /
 * _solver / _predictor_viscous and hbf_set_field / hbf_get_field.  The batch
 * owns it: do not destroy it.  Settings are read at the next hbf_batch_step. */
int hbf_batch_cavity(hbf_batch* b, int i, hbf_ctx** ctx);
/* per-cavity time steps (ncav positive values, host) */
int hbf_batch_set_dt(hbf_batch* b, const double* dt);
/* One step of every cavity.  stats: NULL or ncav entries.  Returns HBF_OK,
 * HBF_ERR_NOT_CONVERGED when some solve stopped at its cycle cap (the step
 * still completes), or an error.  All cavities share the nu1/nu2 counts. */
int hbf_batch_step(hbf_batch* b, hbf_step_stats* stats);
/* Work-list tiling: elements per tile (>= 32) and the persistent grid size
 * (152 x blocks_per_sm blocks at most per launch). */
int hbf_batch_set_tiling(hbf_batch* b, int tile, int blocks_per_sm);
int hbf_batch_get_tiling(const hbf_batch* b, int* tile, int* blocks_per_sm, int64_t* tiles_level0);
/* Multigrid levels on which every cavity has at most max_cells cells (and
 * all coarser levels) run as one launch per V-cycle, one thread block per
 * cavity, with block barriers between colour sweeps; the arithmetic and its
 * order are those of the level-by-level launches.  0 disables it; default
 * 4096. */
int hbf_batch_set_tail(hbf_batch* b, int max_cells);
/* Time a representative launch sequence (explicit stages and one viscous
 * V-cycle of every cavity; no cavity state changes) for each tiling
 * candidate, reps times each, and keep the fastest.  Outputs may be NULL. */
int hbf_batch_autotune(hbf_batch* b, int reps, int* best_tile, int* best_blocks_per_sm, double* best_ms);
/* Phase timing of the following steps (on != 0 starts and resets it, 0
 * stops it): CUDA events between the stages, so each step then ends with a
 * synchronisation.  phase_ms[7]: explicit predictor stages, MAC solve, MAC
 * correction and advective rhs, viscous solve, nodal rhs, nodal solve,
 * projection update, summed over the timed steps.  trips[3]: batched
 * iterations of the MAC, viscous (inner Krylov) and nodal loops, counted
 * whether timing is on or not since the last hbf_batch_profile call. */
int hbf_batch_profile(hbf_batch* b, int on);
int hbf_batch_profile_read(const hbf_batch* b, double phase_ms[7], int64_t trips[3], int64_t* steps);
int64_t hbf_batch_launch_count(const hbf_batch* b);
int hbf_batch_sync(hbf_batch* b);
const char* hbf_batch_last_error(const hbf_batch* b);

#ifdef __cplusplus
}
#endif

#endif /* HBFLOW_H */
