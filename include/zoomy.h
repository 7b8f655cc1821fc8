/*
 * zoomy.h -- C ABI of the GB300 finite-volume library for the shallow-water (level 0) to
 * shallow-moment (level N) hierarchy.
 *
 * The library advances   d_t Q + div F(Q) + B(Q) grad Q = S(Q)    (Eq. (PDE-structure), Sec. 1)
 * for the shallow-moment system of Eq. (sme) (1D) and its 2D form in Sec. 3.4, with the explicit
 * path-conservative finite-volume step named in Sec. 2.1.2 ("hyperbolic_step", after Dumbser,
 * Enaux & Toro 2008 and Castro et al. 2009), hydrostatic reconstruction at the bed, the slip /
 * Newtonian friction closure of Sec. 3.4 (plus Manning), wet/dry handling, SSP-RK2 stages and the
 * adaptive CFL step of the Sec. 3.1 runner (timestepping.adaptive(CFL=0.45)).
 *
 * State layout (every entry point): Q is structure-of-arrays, Q[v * ld + i] for variable v and
 * cell i, with ld >= number of cells.  Variable order:
 *   1D: (h, h alpha_0, h alpha_1, ..., h alpha_N)                       nv = N + 2
 *   2D: (h, h alpha_0, h beta_0, h alpha_1..h alpha_N, h beta_1..h beta_N) nv = 2N + 3
 * where alpha_k / beta_k are the Legendre moments of the x / y velocity (alpha_0 = mean u).
 * Element type: float (dtype 0) or double (dtype 1), as set by zoomy_model_set.
 * Structured 2D cells are numbered j * nx + i; triangle meshes use the library's cell order
 * (see zoomy_mesh_permutation).
 *
 * Ownership: descriptors and host arrays passed in are read during the call only.  Q buffers are
 * owned by the caller.  The context owns its device copies of the mesh, the bed, the stage buffer
 * and the reduction scalars; zoomy_mesh_destroy frees them.
 *
 * Streams: all device work of a context is ordered on its stream (zoomy_mesh_create /
 * zoomy_set_stream).  Calls that return a host value synchronise that stream.
 *
 * Errors: every call returns a zoomy_status and never aborts.  Invalid arguments are rejected
 * before any device work.  zoomy_last_error() describes the last failure of the calling thread.
 */
#ifndef ZOOMY_H
#define ZOOMY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ZOOMY_OK = 0,
    ZOOMY_EINVAL = 1,     /* invalid argument (checked before any launch) */
    ZOOMY_ENOMEM = 2,     /* device or host allocation failed */
    ZOOMY_ECUDA = 3,      /* CUDA runtime error; see zoomy_last_error() */
    ZOOMY_ENAN = 4,       /* a step produced a non-finite state */
    ZOOMY_ENEGDEPTH = 5,  /* a step produced a negative depth */
    ZOOMY_ECFL = 6,       /* no positive finite wave speed: the CFL step is undefined */
    ZOOMY_ETIMEOUT = 7,   /* a device-side wait gave up (persistent ensemble kernel) */
    ZOOMY_ESTATE = 8,     /* call out of order (e.g. zoomy_step before zoomy_model_set) */
    ZOOMY_EBOUNDS = 9     /* bounds-checking build only: a kernel met a gather index outside its buffer
                             (the access was redirected to element 0 and flagged) */
} zoomy_status;

typedef struct zoomy_ctx zoomy_ctx; /* opaque, library-owned */

enum { ZOOMY_MESH_1D = 0, ZOOMY_MESH_2D = 1, ZOOMY_MESH_TRI = 2 };
enum { ZOOMY_BC_TRANSMISSIVE = 0, ZOOMY_BC_WALL = 1 };
enum { ZOOMY_FRICTION_NONE = 0, ZOOMY_FRICTION_SLIP_NEWTONIAN = 1, ZOOMY_FRICTION_MANNING = 2 };
enum { ZOOMY_FP32 = 0, ZOOMY_FP64 = 1 };

/* Mesh description (caller-owned, read during zoomy_mesh_create only).
 *   kind ZOOMY_MESH_1D : nx uniform cells on [x0, x1]; bc[0] left, bc[1] right.
 *   kind ZOOMY_MESH_2D : nx * ny rectangles on [x0,x1] x [y0,y1]; bc = {x-, x+, y-, y+}.
 *   kind ZOOMY_MESH_TRI: ntris triangles over nverts vertices (verts_xy[2*nverts], tris[3*ntris],
 *                        host memory, either orientation); every boundary edge takes bc[0].
 * bathymetry: host array of the bed level b per cell in the caller's cell numbering, or NULL
 * for a flat bed.  morton_reorder (triangles only): 1 = number the cells along a Morton curve of
 * their centroids for locality of the neighbour gathers. */
typedef struct {
    int32_t kind;
    int64_t nx, ny;
    double x0, x1, y0, y1;
    int32_t bc[4];
    int64_t nverts, ntris;
    const double *verts_xy;
    const int32_t *tris;
    const double *bathymetry;
    int32_t morton_reorder;
} zoomy_mesh_desc;

/* Friction closure (Sec. 3.4): Navier slip at the bed sigma|_0 = C u|_0 with the Newtonian bulk
 * stress sigma = nu d_z u (kind SLIP_NEWTONIAN), or the Manning bottom stress g n^2 |u_b| u_b /
 * h^(1/3) (kind MANNING, parameter manning_n).  rho divides the stresses (kinematic: rho = 1). */
typedef struct {
    int32_t kind;
    double C, nu, rho, manning_n;
} zoomy_friction;

/* Version of the C ABI (major * 10000 + minor * 100 + patch). */
int32_t zoomy_version(void);

/* Create a context for a mesh.  stream: a cudaStream_t (NULL = legacy default stream) on which
 * all device work of the context is queued.  On success *out receives the context. */
zoomy_status zoomy_mesh_create(const zoomy_mesh_desc *desc, void *stream, zoomy_ctx **out);

/* Free the context and every device buffer it owns.  NULL is accepted. */
zoomy_status zoomy_mesh_destroy(zoomy_ctx *ctx);

/* Change the stream of the context. */
zoomy_status zoomy_set_stream(zoomy_ctx *ctx, void *stream);

/* Number of cells and min_i Delta_i with Delta_i = 2 |Omega_i| / P_i (the CFL length). */
zoomy_status zoomy_mesh_info(zoomy_ctx *ctx, int64_t *ncells, double *min_delta);

/* Cell permutation of a triangle mesh: perm_out[new] = caller's index (host, ncells int64).
 * Structured meshes return the identity. */
zoomy_status zoomy_mesh_permutation(zoomy_ctx *ctx, int64_t *perm_out);

/* Select the model: level N in [0, 4] (Eq. (sme)), friction closure (may be NULL = none),
 * gravity g > 0, CFL number cfl in (0, 1], dry threshold h_dry >= 0 (velocities are zero where
 * h <= h_dry), dtype ZOOMY_FP32 (FP32 state and flux; FP64-exact bed/surface differences; FP64
 * mass sums) or ZOOMY_FP64.  Allocates the stage buffer. */
zoomy_status zoomy_model_set(zoomy_ctx *ctx, int32_t level, const zoomy_friction *friction, double g, double cfl,
                             double h_dry, int32_t dtype);

/* Time treatment of the friction source (Sec. 3.4 closure, Eq. (PDE-source)).  mode 0 (default):
 * each stage adds the Newtonian bulk stress explicitly and then applies the bottom stress linearly
 * implicitly (rank-1 Sherman-Morrison).  mode 1: the paper's step_source_implicit: each stage takes
 * the hyperbolic update only and then applies the whole friction, bulk plus bottom stress, by one
 * backward-Euler step per cell, (I + dt K) z = y with K_ki = (2k+1) c + (nu/rho)/h^2 C_ik/M_k
 * (C_ik = int phi_i' phi_k'; h and the bottom coefficient c frozen at the stage result); stable for
 * stiff thin layers where dt nu/h^2 >> 1.  Structured and triangle contexts; EINVAL for ensembles,
 * a context with the learned closure, or another mode. */
zoomy_status zoomy_source_mode(zoomy_ctx *ctx, int32_t mode);

/* Order in space.  1 (default): the first-order scheme above.  2: MUSCL reconstruction (the
 * second-order building block the paper names with its gradient reconstruction, Sec. 2.1.2): per
 * direction, minmod-limited slopes of (h, eta = h + b, velocity moments), zero next to dry cells;
 * face states w +- slope/2 with the bed b +- (slope_eta - slope_h)/2; the first-order face term
 * (hydrostatic reconstruction, path-conservative Rusanov flux, pressure difference, path integral
 * of the nonconservative product) between reconstructed face states; per cell and direction the
 * interior terms g (h_+ + h_-)/2 (eta_+ - eta_-) on the normal mean momentum and
 * Btilde(Q_- -> Q_+)(Q_+ - Q_-).  Well-balanced (lake at rest), second order on smooth solutions,
 * no new extrema at shocks; the CFL step is still taken from the cell wave speeds (a CFL number of
 * at most 0.3 is advisable).  1D and structured 2D contexts, FP32 or FP64; EINVAL for triangles,
 * ensembles, a context with the learned closure, or another order. */
zoomy_status zoomy_space_order(zoomy_ctx *ctx, int32_t order);

/* The non-hydrostatic VAM model in 1D (Sec. "Unsteady Vertically Averaged Momentum Equations in
 * 1D"), without friction, over the context's bathymetry b (flat when none was given), as the paper's
 * predictor-corrector splitting (Eq. (PDE-hyperbolic), (PDE-non-hydrostatic),
 * (PDE-non-hydrostatic-update)).  enable = 1 switches a 1D FP64 context (after zoomy_model_set) to the
 * state Q = (h, h u0, h u1, h w0, h w1) (nv = 5, zoomy_nvars), w2 = -(w0 + w1) + (u0 + u1) b_x; every
 * zoomy_step step is then: predictor Q* by the path-conservative Rusanov scheme with hydrostatic
 * reconstruction for the VAM flux and nonconservative product (dt from s = |u0| + sqrt(g h + u1^2) +
 * |u1|, CFL number of the context, or fixed); corrector: the non-hydrostatic pressure (p0, p1) per
 * cell that makes Q** = Q* - dt S(p), S = (0, d(h p0)/dx + 2 p1 b_x, d(h p1)/dx - (3 p0 - p1) dh/dx -
 * 6 (p0 - p1) b_x, -2 p1, 6 (p0 - p1)), satisfy h du0/dx + d(h u1)/dx/3 + u1 dh/dx/3 + 2 (w0 - u0 b_x)
 * = 0 and h du0/dx + u1 dh/dx + 2 (u1 b_x - w1) = 0 (central differences, mirrored ghosts; a
 * block-tridiagonal linear system, two cells per block, solved on the GPU by cyclic reduction);
 * Q^{n+1} = Q**.  The depth must stay positive (ZOOMY_ENEGDEPTH otherwise).  enable = 0 returns to the
 * level-N model, and so does a later zoomy_model_set.  EINVAL for other contexts, enable outside
 * {0, 1}, the learned closure, order 2 or the implicit friction mode; zoomy_max_wavespeed and
 * zoomy_lift3d are not defined in this mode (EINVAL). */
zoomy_status zoomy_vam_set(zoomy_ctx *ctx, int32_t enable);

/* Number of variables nv of the current model. */
zoomy_status zoomy_nvars(zoomy_ctx *ctx, int32_t *nv);

/* Advance Q (device pointer, SoA [nv][ld], dtype of the model) by nsteps SSP-RK2 steps:
 *   Q1 = R(Q^n + dt L(Q^n)),  Q^{n+1} = 1/2 (Q^n + R(Q1 + dt L(Q1)))
 * dt > 0: fixed step.  dt == 0: dt = cfl * min Delta / max_i s_i(Q^n), recomputed on the device
 * every step (no host round trip).  Q is updated in place.
 * t_advanced (host) != NULL: the stream is synchronised, *t_advanced receives the simulated time
 * advanced since the last status read (see zoomy_sync) and device-detected errors are returned (ZOOMY_ENAN / ZOOMY_ENEGDEPTH / ZOOMY_ECFL; Q then
 * holds the state after the step that raised it, and the later steps of the call are skipped).
 * t_advanced == NULL: the call only queues work; zoomy_sync reports the outcome. */
zoomy_status zoomy_step(zoomy_ctx *ctx, void *Q, int64_t ld, double dt, int32_t nsteps, double *t_advanced);

/* Same step with Q in HOST memory (pinned for full copy speed): copies Q to a context-owned
 * device buffer, steps, copies the result back, synchronises. */
zoomy_status zoomy_step_host(zoomy_ctx *ctx, void *Q_host, int64_t ld, double dt, int32_t nsteps,
                             double *t_advanced);

/* Wait for the queued steps; *t_total (may be NULL) receives the time advanced by all steps
 * queued since the last status read (a zoomy_step with t_advanced, zoomy_step_host or
 * zoomy_sync), and the first device-detected error among them is returned.  An error is sticky:
 * once raised, later queued steps are skipped until it is read here. */
zoomy_status zoomy_sync(zoomy_ctx *ctx, double *t_total);

/* max_i s_i(Q) (device Q, synchronises): s = |u_mean| + sqrt(g h + sum_{k>=1}|a_k|^2) +
 * sum_{k>=2}|a_k|, the bound on the spectral radius of the quasilinear matrix (Sec. 2.1.1,
 * eigenstructure of A . n) used for the CFL step. */
zoomy_status zoomy_max_wavespeed(zoomy_ctx *ctx, const void *Q, int64_t ld, double *out);

/* Advance Q (device) to the time t_end from now with CFL steps and land on t_end exactly: chunks of
 * at most `chunk` steps, each sized from the current maximum wave speed (zoomy_max_wavespeed, one
 * synchronisation per chunk) to stay below t_end, then one or two fixed steps of equal length once
 * fewer than about 1.25 CFL steps remain (neither longer than the CFL step).  The paper's solver runs
 * to a final time the same way (Sec. 3.1: adaptive step, end time).  *t_out: time advanced (t_end
 * up to rounding), *steps_out: steps taken (both may be NULL).  Errors as zoomy_step; ZOOMY_EINVAL
 * for t_end < 0 or chunk < 1. */
zoomy_status zoomy_advance(zoomy_ctx *ctx, void *Q, int64_t ld, double t_end, int32_t chunk, double *t_out,
                           int64_t *steps_out);

/* sum_i |Omega_i| h_i accumulated in FP64 in a fixed order (device Q, synchronises). */
zoomy_status zoomy_mass(zoomy_ctx *ctx, const void *Q, int64_t ld, double *out);

/* Work decomposition of the structured 2D kernels (a performance knob; results do not depend
 * on it): each warp marches over rows_per_warp rows of a 30-column strip, warps_per_block warps
 * per CTA.  rows_per_warp in [1, 4096], warps_per_block in [1, 32].  Until this or zoomy_autotune
 * sets it, rows_per_warp follows the grid: about 24 warps per SM (16 for the learned-closure stage),
 * within [8, 64] rows. */
zoomy_status zoomy_tune_set(zoomy_ctx *ctx, int32_t rows_per_warp, int32_t warps_per_block);

/* Launch shape of the first-order 1D line (a performance knob; the state is bitwise the same for every
 * setting).  The 1D kernels run one warp per 31 cells, each lane evaluating one face.  mode:
 * ZOOMY_LAUNCH_AUTO (0) and ZOOMY_LAUNCH_PER_STAGE (1): two kernel launches per SSP-RK2 step (with
 * programmatic dependent launch); ZOOMY_LAUNCH_PERSISTENT (2): all steps of a zoomy_step call in one
 * cooperative launch whose CTAs meet at a grid barrier after each stage (taken where every CTA of the
 * line can be resident at once and stage profiling is off; otherwise the call falls back to two launches
 * per step).  warps_per_cta: 0 = automatic (1 below 65536 cells, else 8), or 1..8.  EINVAL for other
 * values. */
enum { ZOOMY_LAUNCH_AUTO = 0, ZOOMY_LAUNCH_PER_STAGE = 1, ZOOMY_LAUNCH_PERSISTENT = 2 };
zoomy_status zoomy_tune_1d(zoomy_ctx *ctx, int32_t mode, int32_t warps_per_cta);

/* Autotuner of the structured 2D decomposition: times both stage kernels on the state Q (device,
 * left unchanged; a temporary copy is used for the in-place stage) for each candidate rows_per_warp
 * (and warps_per_block where the kernel has that freedom) and keeps the fastest pair in the context.
 * cache_path (may be NULL): a JSON-lines file; an entry for the same (grid, level, dtype, device)
 * is reused without measuring, a new measurement is appended.  *rows_per_warp_out and
 * *us_per_step_out (may be NULL) receive the choice and its measured stage-1 + stage-2 time. */
zoomy_status zoomy_autotune(zoomy_ctx *ctx, const void *Q, int64_t ld, const char *cache_path,
                            int32_t *rows_per_warp_out, double *us_per_step_out);

/* ---- Learned closure ---------------------------------------------------------------------------
 * Turns a structured 2D level-1 FP32 context into the level-1 solver closed with learned level-4
 * moments: the level-4 system restricted to the rows of (h, h alpha_0, h beta_0, h alpha_1,
 * h beta_1), with alpha_2..4, beta_2..4 predicted per cell at every stage input by the MLP
 *   x = (h, u_m, v_m, alpha_1, beta_1, lambda) * in_scale -> 64 -> 64 -> 6 (GELU, tanh form)
 *   (alpha_2, alpha_3, alpha_4, beta_2, beta_3, beta_4) = y * out_scale
 * run on the tensor cores inside the stage kernel (BF16 weights and layer inputs, FP32
 * accumulation).  The paper's model hierarchy truncates the moments; the "material closure" it
 * calls exchangeable is here a learned one.  params: 4998 host floats W1[6][64], b1[64],
 * W2[64][64], b2[64], W3[64][6], b3[6] (weights rounded to BF16 on upload); lambda: the slip
 * feature (normally the context's slip coefficient).  zoomy_step then advances the closed model;
 * zoomy_closure_clear returns to the plain level-1 model. */
zoomy_status zoomy_closure_set(zoomy_ctx *ctx, const float *params, const float *in_scale, const float *out_scale,
                               double lambda);
zoomy_status zoomy_closure_clear(zoomy_ctx *ctx);

/* The closure MLP alone, with the solver's tensor-core code: feat (device, SoA [6][n], unscaled
 * features) -> out (device, SoA [6][n], the six predicted moments).  Queued on the context's
 * stream; a tensor-core completion wait that gives up is reported as ZOOMY_ETIMEOUT by the next
 * synchronising call (zoomy_sync). */
zoomy_status zoomy_closure_eval(zoomy_ctx *ctx, const float *feat, float *out, int64_t n);

/* Tensor-core engine of the closure network: 0 (default) = tcgen05.mma with FP32 accumulators in
 * tensor memory, 128 cells per MMA tile; 1 = warp-level mma.sync (m16n8k16).  Both round the
 * weights and the layer inputs to BF16 and accumulate in FP32; they differ only in the order of
 * the FP32 accumulation.  EINVAL for other values. */
zoomy_status zoomy_closure_engine(zoomy_ctx *ctx, int32_t engine);

/* When the closure network is evaluated (the paper's material closure of Sec. 1 / Sec. 3.4 is
 * exchangeable and leaves this open; reading R21): schedule 0 (default) on every SSP-RK2 stage
 * input; schedule 1 once per step on Q^n, its predicted velocity moments held for both stages (each
 * stage input closes with its own depth and dry cut).  Schedule 1 halves the network evaluations;
 * the two differ by O(dt) at a fixed end time.  EINVAL for other values. */
zoomy_status zoomy_closure_schedule(zoomy_ctx *ctx, int32_t schedule);

/* ---- Training the closure MLP ------------------------------------------------------------------
 * Full-batch (or caller-sliced mini-batch) training of the closure network above by hand-written
 * kernels: forward and backward passes one thread per sample (FP32, weights in shared memory), the
 * weight gradients as split-K reductions summed in a fixed order (deterministic), Adam (Kingma &
 * Ba: beta1 0.9, beta2 0.999, eps 1e-8) on FP32 master weights.  Loss = mean over the n samples and
 * the 6 outputs of (y - t)^2 in the scaled output space.  X: device [n][6] scaled features, T:
 * device [n][6] scaled targets (row-major, sample-major).  The paper builds no learned closure; this
 * trains the "material closure" of Sec. 1 / Sec. 3.4 as a data-driven one.
 *   zoomy_mlp_create: params = 4998 host floats in the order of zoomy_closure_set; stream = the
 *     stream every later call queues on (NULL = legacy default stream).
 *   zoomy_mlp_grad: loss (host, may be NULL) and gradient (host [4998], may be NULL) of the current
 *     parameters; synchronises the stream when either is requested.
 *   zoomy_mlp_train_step: one Adam step with learning rate lr > 0 on the batch; loss (may be NULL:
 *     no synchronisation) is the loss BEFORE the step.
 *   zoomy_mlp_get_params: the current FP32 parameters into host params [4998] (synchronises).
 * The workspace grows to the largest n seen (~1.6 kB per sample).  ZOOMY_EINVAL on NULL pointers,
 * n < 1 or lr <= 0; ZOOMY_ECUDA on launch or allocation failures. */
typedef struct zoomy_mlp zoomy_mlp; /* opaque, library-owned */
zoomy_status zoomy_mlp_create(const float *params, void *stream, zoomy_mlp **out);
zoomy_status zoomy_mlp_destroy(zoomy_mlp *mlp);
zoomy_status zoomy_mlp_get_params(zoomy_mlp *mlp, float *params);
zoomy_status zoomy_mlp_grad(zoomy_mlp *mlp, const float *X, const float *T, int64_t n, float *loss, float *grad);
zoomy_status zoomy_mlp_train_step(zoomy_mlp *mlp, const float *X, const float *T, int64_t n, float lr, float *loss);

/* Training samples from a structured 2D level-`level` FP32 state Q[v][ld] (device): for each of the
 * n listed cells (device int64 indices), X[s] = (h, u_m, v_m, alpha_1, beta_1, lambda) * in_scale and
 * T[s] = (alpha_2, alpha_3, alpha_4, beta_2, beta_3, beta_4) / out_scale (moments above `level` are
 * zero; velocities are zero where h <= h_dry).  in_scale / out_scale: device [6]; X, T: device
 * [n][6].  Queued on `stream`. */
zoomy_status zoomy_closure_samples(const float *Q, int64_t ld, int32_t level, const int64_t *cells, int64_t n,
                                   double lambda, double h_dry, const float *in_scale, const float *out_scale,
                                   float *X, float *T, void *stream);

/* Scale factors of a training set X, T (device, [n][6] each; the closure network's features and
 * targets): in_scale[j] = 1 / max_s |X[s][j]|, out_scale[j] = max_s |T[s][j]| (floored at 1e-12),
 * into host arrays [6].  Synchronises `stream`.  The paper trains no network; this serves the
 * learned closure (zoomy_closure_set). */
zoomy_status zoomy_sample_scales(const float *X, const float *T, int64_t n, float *in_scale, float *out_scale,
                                 void *stream);

/* In place on the device: X[s][j] *= in_scale[j], T[s][j] /= out_scale[j] for s < n (in_scale,
 * out_scale: device [6]).  Queued on `stream`. */
zoomy_status zoomy_sample_scale(float *X, float *T, int64_t n, const float *in_scale, const float *out_scale,
                                void *stream);

/* ---- Lifting to three-dimensional fields ---------------------------------------------------------
 * The paper's interpolate_3d postprocessing (Sec. "Postprocessing"): from the state Q (device,
 * [nv][ld], the context's dtype and cell order) the fields u, v, w, p at the K sigma levels zeta[j]
 * (host, in [0, 1]; elevation z = b + zeta h) of every cell:
 *   u = sum_k alpha_k phi_k(zeta), v = sum_k beta_k phi_k(zeta)   (the moment expansion),
 *   w = -sum_k [d_x(h alpha_k) + d_y(h beta_k)] Phi_k(zeta) + u (d_x b + zeta d_x h) + v (d_y b + zeta d_y h)
 *       (continuity integrated from the bed, where w = u . grad b),
 *   p = g h (1 - zeta)   (hydrostatic, rho = 1);
 * horizontal derivatives by Green-Gauss with face values (q_i + q_j)/2 (q_j = q_i on boundary
 * faces); u = v = w = 0 in dry cells.  out (device, the context's dtype): plane (f, j) of field
 * f in (u, v, w, p) at out + (f K + j) ldo, ldo >= ncells.  1 <= K <= 64.  Any mesh kind, any
 * level; queued on the context's stream (no synchronisation).  EINVAL on bad arguments or zeta
 * outside [0, 1]. */
zoomy_status zoomy_lift3d(zoomy_ctx *ctx, const void *Q, int64_t ld, int32_t K, const double *zeta, void *out,
                          int64_t ldo);

/* ---- Batched ensembles (independent runs of uneven sizes in one launch) -------------------------
 * nmembers square grids of side sides[m] on the unit square with walls, each with its own slip
 * coefficient C[m] (Navier slip, rho = 1) and the Newtonian viscosity nu, level `level`, FP32
 * state, its own CFL step (cfl, g, h_dry as in zoomy_model_set).  The members' states are
 * concatenated: member m's cell (i, j) is at offsets[m] + j sides[m] + i of each variable plane of
 * one SoA array Q[v][ld], ld >= offsets[nmembers] (zoomy_ensemble_offsets). */
zoomy_status zoomy_ensemble_create(int32_t nmembers, const int64_t *sides, const double *C, int32_t level,
                                   double nu, double g, double cfl, double h_dry, void *stream, zoomy_ctx **out);

/* offsets[0..nmembers] (host): start of each member in the concatenated state, and the total. */
zoomy_status zoomy_ensemble_offsets(zoomy_ctx *ctx, int64_t *offsets);

/* Advance every member by nsteps SSP-RK2 steps with its own CFL step.  mode 0: one persistent
 * cooperative launch (grid-wide barriers between phases, dynamic work distribution over
 * (member, strip, row segment) items) captured in a CUDA graph; mode 1: the same launch without the
 * graph; mode 2: one launch per phase (2 nsteps + 1) captured in a CUDA graph; mode 3: those launches
 * without the graph.  All modes give bitwise the same result.  Synchronises; t_members (host,
 * nmembers, may be NULL) receives each member's simulated time.  A barrier wait that exceeds its
 * spin limit makes the kernel return and the call report ZOOMY_ETIMEOUT. */
zoomy_status zoomy_ensemble_step(zoomy_ctx *ctx, void *Q, int64_t ld, int32_t nsteps, int32_t mode,
                                 double *t_members);

/* Pick the row-segment height of the ensemble's work items by timing two persistent steps per
 * candidate on a scratch copy of Q (Q is left unchanged). */
zoomy_status zoomy_ensemble_autotune(zoomy_ctx *ctx, void *Q, int64_t ld, int32_t *rows_per_warp_out,
                                     double *us_per_step_out);

/* Barrier settings of the persistent ensemble kernel: spin_limit bounds every wait (iterations of a
 * ~64 ns sleep; default 2e7); extra_participants > 0 makes every barrier wait for participants that
 * never arrive, which exercises the timeout path (testing). */
zoomy_status zoomy_ensemble_set_barrier(zoomy_ctx *ctx, int64_t spin_limit, int32_t extra_participants);

/* Per-launch timing of the stage kernels with CUDA events recorded on the context's stream
 * around every stage launch (on = 1) or off (on = 0, default).  zoomy_profile_read waits for
 * the stream and returns the launch counts and the summed device time in milliseconds of the
 * stage-1 kernels, the stage-2 kernels and the learned closure's prediction kernels (in that
 * order) since profiling was enabled, then resets the counters.  Arrays of length 3 (host). */
zoomy_status zoomy_profile_enable(zoomy_ctx *ctx, int32_t on);
zoomy_status zoomy_profile_read(zoomy_ctx *ctx, int64_t *launches, double *total_ms);

/* Size of the fixed device scratch used by zoomy_step_noalloc (bytes). */
#define ZOOMY_NOALLOC_SCRATCH_BYTES (32u << 20)

/* zoomy_step with no allocation, for callers that cannot call cudaMalloc: code running where the
 * device allocator is off limits (a host callback or driver hook, an application whose external
 * memory manager owns every device allocation, a real-time loop that cannot take the implicit
 * synchronisation of an allocation).  The paper has no counterpart; it is a service of this
 * library.  It advances a structured 2D grid (cells j * nx + i on [x0,x1] x [y0,y1], bc = {x-, x+,
 * y-, y+}) with the FP32 state path of zoomy_step: Q is the caller's device state [nv][ld]
 * (nv = 2 level + 3, ld >= nx ny), bed the caller's device bed level [nx ny] (required; zeros for a
 * flat bed), and the other arguments mean what they mean for zoomy_mesh_create / zoomy_model_set /
 * zoomy_step (the same friction parameters are refused).  Q and bed must be float-aligned, and
 * nx ny must fit a 32-bit cell index.  The stage buffer and the step's control block live in one
 * array of ZOOMY_NOALLOC_SCRATCH_BYTES compiled into the library, reserved on every GPU that loads
 * it until the process exits: a state needing more (256 + 4 nv ld bytes) is rejected with
 * ZOOMY_EINVAL and a message naming the limit.  Every rejection happens before any device work.
 * The call allocates nothing (no cudaMalloc, no cudaFree, no allocating library routine); it clears
 * the control block it needs zeroed at its start, because the array keeps the previous call's
 * contents.  All calls share that one array: calls whose device work overlaps (other streams or
 * threads, without ordering) race on it.  Every call looks up the array's device address on the
 * current device (so a device reset between calls is harmless); the first call on a device also
 * loads the library's device code there, so make that first call before any stream capture.
 * t_advanced != NULL synchronises the stream and reports device-detected errors as zoomy_step
 * does; with t_advanced == NULL nothing is read back. */
zoomy_status zoomy_step_noalloc(int64_t nx, int64_t ny, double x0, double x1, double y0, double y1,
                                const int32_t *bc, int32_t level, const zoomy_friction *friction, double g,
                                double cfl, double h_dry, const float *bed, float *Q, int64_t ld, double dt,
                                int32_t nsteps, void *stream, double *t_advanced);

/* Text of the last error of the calling thread (static storage, never NULL). */
const char *zoomy_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* ZOOMY_H */
