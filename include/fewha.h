/*
 * fewha.h -- C ABI of the GB300 (sm_103a) FEWHA reconstructor.
 *
 * FEWHA (Finite Element Wavelet Hybrid Algorithm, Stadler & Ramlau, "Performance of
 * an iterative wavelet reconstructor for MAORY") solves, once per frame, the MAP
 * tomography system of Eq. (5),
 *
 *     M c = b,   M = W (sum_g P_g^T Gamma_g^T C_hat_g^-1 Gamma_g P_g) W^T + alpha D,
 *                b = W sum_g P_g^T Gamma_g^T C_hat_g^-1 s_g,
 *
 * with a fixed number of Jacobi-preconditioned CG iterations (Eq. 7, Sec. 3.3),
 * warm-started from the previous frame, then fits the DMs, a~ = F W^T c, and applies
 * the control law (Algorithm 1: open loop, or closed loop with FEWHA_FLAG_CLOSED_LOOP).
 * Options: the augmented PCG of Sec. 3.4 (FEWHA_FLAG_AUGMENTED), the LGS spot-elongation
 * noise model of Eq. 3 (fewha_params.alpha_eta); batches of uneven instances; gradients
 * of the converged map (fewha_backward) and of the fixed-iteration frame
 * (fewha_frame_vjp); least-squares DM fitting over fitting directions in place of the
 * projection F (fewha_fit_ls, Sec. 4.1).
 *
 * Conventions shared by every entry point
 *   - All functions return FEWHA_OK (0) or a negative FEWHA_ERR_* code; the text of
 *     the last error of a handle is fewha_last_error(handle).
 *   - "d_" pointers are CUDA device pointers owned by the caller; "h_" pointers are
 *     host pointers owned by the caller.  The library owns its handle and all of the
 *     handle's internal device state.  No entry point keeps a caller pointer after
 *     it returns, except that a captured frame graph is re-captured when the caller
 *     passes different device pointers.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     Device work is enqueued on it in order; entry points taking only device
 *     pointers return before the work finishes (no host synchronisation), entry
 *     points taking host pointers synchronise on `stream` before returning.
 *   - Element type: a handle created with params.precision == 32 computes every
 *     operator in float (inner products and the CG scalars alpha, beta in double);
 *     precision == 64 computes everything in double.  Entry points with typed
 *     pointers exist in float and _f64 twins; the void* operator entry points take
 *     the handle's element type.
 *   - A handle is not thread-safe; distinct handles are independent.
 *
 * Layouts
 *   - coefficient vector c, b (n_coeffs): layers concatenated in creation order;
 *     layer l is an n_l x n_l row-major array in Mallat layout (after `levels`
 *     analysis steps on rows then columns: [LL LH; HL HH], recursion on LL).
 *   - layer (finite-element) vector phi: same sizes, row-major node values; node
 *     (i, j) of layer l sits at x = (j - n_l/2) delta_l, y = (i - n_l/2) delta_l.
 *   - node vector (n_nodes): sensors concatenated; sensor g holds (N_g+1)^2 aperture
 *     nodes, N_g = n_sub * nb, node (a, b) at x = -D/2 + b d_g, y = -D/2 + a d_g.
 *   - slope vector s (n_slopes): sensors concatenated; sensor g holds the x-slopes of
 *     its active subapertures in row-major order, then the y-slopes in the same
 *     order.  A subaperture is active iff its centre radius r satisfies
 *     obs*D/2 <= r <= D/2.  A slope is the phase difference across the subaperture
 *     (radians).  For a coarse sensor (nb > 1) the active units are coarse
 *     subapertures.
 *   - DM vector (n_act): DMs concatenated, each n_act_m x n_act_m row-major,
 *     actuator (p, q) at x = (q - (n_act_m-1)/2) spacing_m, y likewise with p.
 */
#ifndef FEWHA_H
#define FEWHA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FEWHA_OK 0
#define FEWHA_ERR_INVALID_ARG (-1) /* null pointer, bad count, precision mismatch   */
#define FEWHA_ERR_GEOMETRY (-2)    /* footprint outside a layer grid, n not 2^k ... */
#define FEWHA_ERR_OOM (-3)         /* device allocation failed                      */
#define FEWHA_ERR_CUDA (-4)        /* a CUDA runtime call failed                    */
#define FEWHA_ERR_NONFINITE (-5)   /* a NaN/Inf was found in the input slopes, or a
                                      recurrence being differentiated stopped          */
#define FEWHA_ERR_LIMIT (-6)       /* a size exceeds a compiled-in maximum          */
#define FEWHA_ERR_TIMEOUT (-7)     /* a grid-wide wait of the persistent frame ran out
                                      of polls (FEWHA_FLAG_PERSISTENT)                 */

#define FEWHA_MAX_LAYERS 16
#define FEWHA_MAX_WFS 16
#define FEWHA_MAX_DMS 4
#define FEWHA_MAX_GRID 128   /* largest layer grid side n                           */
#define FEWHA_MAX_NFINE 80   /* largest fine subaperture count per side, n_sub*nb   */
#define FEWHA_MAX_COARSE 4   /* largest coarse subaperture count per side (nb > 1)  */
#define FEWHA_MAX_ITERS 64

#define FEWHA_FLAG_GRAPH 1u         /* replay each frame as a captured CUDA graph    */
#define FEWHA_FLAG_WARM_RESIDUAL 2u /* r0 = (b - b_prev) + r_prev (Algorithm 1)     */
#define FEWHA_FLAG_PDL 4u           /* programmatic dependent launch: each kernel lets
                                       the next one launch its CTAs early (the cluster
                                       kernels from a barrier in their middle), which
                                       wait on the device for it to finish; shortens
                                       the gap between dependent kernels (the Python
                                       binding sets it by default)                     */
#define FEWHA_FLAG_AUGMENTED 8u     /* augmented PCG (Sec. 3.4, the augPCG step of
                                       Algorithm 1): the previous frame's search
                                       directions P and their images Q = M P are kept;
                                       the start is corrected over span(P) and every new
                                       direction is made M-conjugate to P.  Needs
                                       iters <= FEWHA_AUG_MAX_ITERS.  The directions are
                                       dropped by update_params, reset and set_state (the
                                       next frame runs unaugmented).  Not available in
                                       batched frames (FEWHA_ERR_INVALID_ARG).         */
#define FEWHA_AUG_MAX_ITERS 8
#define FEWHA_FLAG_CLOSED_LOOP 16u  /* closed-loop control (Algorithm 1): the slopes passed
                                       in are residual slopes; the frame first forms the
                                       pseudo-open-loop slopes s + Gamma P_DM a^(i-1)
                                       (the DM shapes of two frames back, bilinear between
                                       actuators, seen by each sensor like a layer) and
                                       ends with a^(i+1) = a^(i) + gain (a~ - a^(i-1)).
                                       fewha_reset zeroes a^(i) and a^(i-1); set_state
                                       sets a^(i) only.  Every DM must sit below every
                                       LGS (FEWHA_ERR_GEOMETRY).  Not available in
                                       batched frames (FEWHA_ERR_INVALID_ARG).         */

#define FEWHA_FLAG_PERSISTENT 32u  /* run each frame (right-hand side, initial residual,
                                       PCG iterations, fit: Algorithm 1) as ONE cooperative
                                       launch of thread-block clusters whose stages are
                                       separated by grid-wide waits instead of kernel
                                       boundaries.  Every wait gives up after a bounded
                                       number of polls (fewha_set_wait_limit); the frame
                                       then stops and FEWHA_ERR_TIMEOUT is reported by the
                                       host-buffer entry points, fewha_run_loop and
                                       fewha_check_input.  Not with FEWHA_FLAG_AUGMENTED or
                                       FEWHA_FLAG_CLOSED_LOOP (FEWHA_ERR_INVALID_ARG);
                                       batched frames ignore it.                          */

/* Telescope aperture: diameter D [m], central obstruction as a diameter ratio. */
typedef struct fewha_telescope {
    double D;
    double obs;
} fewha_telescope;

/* One Shack-Hartmann sensor (Sec. 2; Table 4).  n_sub subapertures per side; nb > 1
 * makes a coarse sensor whose slope is (1/nb) x the sum of the fine slopes of the
 * active fine subapertures in its nb x nb block.  An LGS (is_lgs = 1) sits at height
 * H [m] (cone effect, s_l = 1 - h_l/H) and has its tip/tilt removed by the projector
 * of Sec. 3.2; an NGS sits at infinity.  theta: direction [rad]; sigma: noise standard
 * deviation per slope [rad], C_g = sigma^2 I (Eq. 2). */
typedef struct fewha_wfs {
    int n_sub;
    int nb;
    int is_lgs;
    double theta_x, theta_y;
    double H;
    double sigma;
    /* LGS spot elongation (Eq. 3), used when fewha_params.alpha_eta, na_fwhm and
     * spot_fwhm are all > 0: laser launch position (launch_x, launch_y) [m] in the pupil
     * plane, FWHM of the sodium profile na_fwhm [m], FWHM of the non-elongated spot
     * spot_fwhm [rad].  Subaperture (i, j) with midpoint (x, y) then has the 2 x 2 noise
     * covariance sigma^2 (I + (alpha_eta / spot_fwhm)^2 beta beta^T), beta =
     * (na_fwhm / H^2) ((x, y) - (launch_x, launch_y)).  Zero for an NGS. */
    double launch_x, launch_y;
    double na_fwhm;
    double spot_fwhm;
} fewha_wfs;

/* One reconstruction layer (Sec. 3.1; Table 2): altitude h [m], Cn2 weight, grid
 * spacing [m], periodic grid side n = 2^J, number of wavelet levels (1..J). */
typedef struct fewha_layer {
    double h;
    double cn2_weight;
    double spacing;
    int n;
    int levels;
} fewha_layer;

/* One deformable mirror (Sec. 4.1; Table 3): altitude [m], actuator spacing [m],
 * actuators per side. */
typedef struct fewha_dm {
    double h;
    double spacing;
    int n_act;
} fewha_dm;

/* Method parameters (Table 5): regularisation alpha, preconditioner threshold tau
 * (Eq. 7), loop gain (Algorithm 1), von Karman r0 [m at 500 nm] and L0 [m] of the
 * prior D, PCG iterations, precision (32 or 64) and FEWHA_FLAG_* bits. */
typedef struct fewha_params {
    double alpha;
    double tau;
    double gain;
    double r0;
    double L0;
    int iters;
    int precision;
    unsigned flags;
    double alpha_eta;   /* spot-elongation tuning of Eq. 3 (Table 5); 0 = C_g = sigma^2 I */
    int warm_refresh;   /* with FEWHA_FLAG_WARM_RESIDUAL: after this many frames in a row on
                           the warm recurrence r0 = (b - b_prev) + r_prev, one frame forms the
                           explicit r0 = b - M c0, which bounds the recurrence's drift in
                           single precision; 0 = never */
} fewha_params;

typedef struct fewha_handle fewha_handle;

/* Build an instance: validates the geometry (FEWHA_ERR_GEOMETRY if a projected
 * aperture or DM footprint leaves a layer grid, n is not a power of two, or levels
 * is out of range; FEWHA_ERR_LIMIT above the FEWHA_MAX_* sizes), computes the
 * interpolation tables, the prior D (Sec. 3.1) and the exact Jacobi diagonal of
 * Eq. (7) on the GPU, allocates the state (warm start c = 0, a_prev = 0) on the
 * current CUDA device.  Synchronous.  *out receives the handle; on failure *out is
 * NULL and the return code says why. */
int fewha_create(const fewha_telescope* tel, const fewha_wfs* wfs, int n_wfs,
                 const fewha_layer* layers, int n_layers, const fewha_dm* dms, int n_dms,
                 const fewha_params* params, fewha_handle** out);
void fewha_destroy(fewha_handle* h);
const char* fewha_last_error(const fewha_handle* h);
/* Text of the last error of a failed fewha_create (thread-local). */
const char* fewha_create_error(void);

/* Vector sizes of an instance (any pointer may be NULL). */
int fewha_sizes(const fewha_handle* h, int64_t* n_slopes, int64_t* n_coeffs, int64_t* n_act,
                int64_t* n_nodes);

/* On-the-fly system update (Sec. 1, Sec. 4.3): new alpha, tau, gain, r0, L0, iters
 * and optionally new layer Cn2 weights (n_layers values) and sensor noise sigmas
 * (n_wfs values); recomputes D and the Jacobi diagonal, discards the warm residual.
 * precision and the geometry cannot change.  Synchronous. */
int fewha_update_params(fewha_handle* h, const fewha_params* params, const double* cn2_weights,
                        const double* sigmas);

/* Zero the warm-start state (c, a_prev, residual history). Stream-ordered. */
int fewha_reset(fewha_handle* h, void* stream);

/* One frame of Algorithm 1 (open loop): r0 = b - M c0 from d_slopes (formed as
 * W P^T Gamma^T C^-1 (s - Gamma P W^T c0) - alpha D c0, without b; the warm residual
 * form with FEWHA_FLAG_WARM_RESIDUAL and the augmented start form b first), `iters` PCG
 * iterations, DM fit and gain.  d_x_warm (n_coeffs) is the warm start, read and overwritten with the new c;
 * NULL uses the handle's internal state.  d_dm_out (n_act) receives the commands
 * a = (1 - gain) a_prev + gain a~.  Asynchronous on `stream`. */
int fewha_reconstruct(fewha_handle* h, const float* d_slopes, float* d_x_warm, float* d_dm_out,
                      void* stream);
int fewha_reconstruct_f64(fewha_handle* h, const double* d_slopes, double* d_x_warm,
                          double* d_dm_out, void* stream);

/* The same frame from and to HOST memory (pinned or pageable): copies the slopes in,
 * runs the frame on the internal warm state, copies the commands out and synchronises
 * on `stream`.  Returns FEWHA_ERR_NONFINITE (commands still written) if the slopes
 * held a NaN or Inf. */
int fewha_reconstruct_host(fewha_handle* h, const float* h_slopes, float* h_dm_out, void* stream);
int fewha_reconstruct_host_f64(fewha_handle* h, const double* h_slopes, double* h_dm_out,
                               void* stream);

/* Warm-start state of the frame loop (checkpoint / resume): the wavelet coefficients c
 * (n_coeffs) and the previous commands a_prev (n_act), device pointers of the handle's
 * element type, either may be NULL.  set_state also discards the warm residual (the next
 * frame forms r0 = b - M c explicitly).  Stream-ordered. */
int fewha_get_state(fewha_handle* h, void* d_c, void* d_a_prev, void* stream);
int fewha_set_state(fewha_handle* h, const void* d_c, const void* d_a_prev, void* stream);

/* The residual r and right-hand side b of the last frame's PCG (the recurrence residual;
 * Sec. 3.3), n_coeffs each, copied into device buffers of the handle's element type
 * (either pointer may be NULL).  Inspection only: ||r|| / ||b|| measures how far the
 * fixed iteration count left the frame from M c = b.  b exists only for the frame forms
 * that keep it (FEWHA_FLAG_WARM_RESIDUAL, _AUGMENTED, _PERSISTENT): the plain explicit
 * frame forms r0 = b - M c0 from the slopes' residual in one chain and never forms b, and
 * a request for it returns FEWHA_ERR_INVALID_ARG (fewha_rhs computes b from the slopes).
 * Stream-ordered. */
int fewha_get_residual(fewha_handle* h, void* d_r, void* d_b, void* stream);

/* Reverse mode through the fixed-iteration frame (a build addition; the paper has no
 * gradients).  The map is the frame of Algorithm 1 started from the warm start d_c0
 * (n_coeffs) with the explicit initial residual r0 = b(s) - M c0, params.iters PCG
 * iterations (Sec. 3.3) and the fit, without the control law: a~ = F W^T c_k(s), written
 * to d_dm_out (n_act, nullable).  With d_grad_dm = dJ/da~ (n_act; NULL: forward only) it
 * writes dJ/ds (n_slopes) to d_grad_slopes by running the recurrence backwards, the
 * adjoint of every statement in reverse order.  Device pointers of the handle's element
 * type.  The handle's warm state is untouched; the warm-residual, augmented and
 * closed-loop flags do not apply.  FEWHA_ERR_NONFINITE if the recurrence stopped
 * (r.z or p.q vanished).  Synchronous on `stream`. */
int fewha_frame_vjp(fewha_handle* h, const void* d_slopes, const void* d_c0, const void* d_grad_dm,
                    void* d_dm_out, void* d_grad_slopes, void* stream);

/* Real-time frame loop (Algorithm 1 run frame after frame, open loop): frame k reads
 * the host slopes h_slopes + k * n_slopes, is warm-started from frame k - 1 (the
 * handle's internal state, so frame 0 continues from whatever the handle holds), and
 * writes its commands to h_dm_out + k * n_act.  Each frame is one host->device copy,
 * one replay of the captured frame graph (with FEWHA_FLAG_GRAPH) and one
 * device->host copy, then a synchronise: the frame's commands are on the host when
 * its latency sample is taken.  Frame k is released at t0 + k * period_us (t0 = the
 * call; the host busy-waits until then); period_us = 0 runs the frames back to back.
 * Per frame, wall_us (nullable, n_frames floats) gets the host-clock time from the
 * later of the frame's release and the end of the previous frame to its commands
 * being on the host, and device_us (nullable) the CUDA-event time from the start of
 * the slope copy to the end of the command copy.  *n_late (nullable) counts frames
 * whose commands arrived after the next frame's release.  Host buffers should be
 * pinned for the copies to be asynchronous.  A frame whose slopes hold a NaN or Inf
 * still runs; the call then returns FEWHA_ERR_NONFINITE after the last frame, naming
 * the first such frame in fewha_last_error.  Synchronous on `stream`. */
int fewha_run_loop(fewha_handle* h, const float* h_slopes, int n_frames, float* h_dm_out,
                   double period_us, float* wall_us, float* device_us, int* n_late, void* stream);
int fewha_run_loop_f64(fewha_handle* h, const double* h_slopes, int n_frames, double* h_dm_out,
                       double period_us, float* wall_us, float* device_us, int* n_late,
                       void* stream);

/* Non-finite flag of the slopes read by frames since the last call (1 if any NaN or
 * Inf was seen), then cleared.  Returns FEWHA_ERR_TIMEOUT (the flag still written) if a
 * persistent frame since the last call stopped because a grid-wide wait ran out.
 * Synchronises on `stream`. */
int fewha_check_input(fewha_handle* h, int* nonfinite, void* stream);

/* ---- operator entry points (the handle's element type; asynchronous) ----------- */

/* q = M c (Eq. 6). */
int fewha_apply_M(fewha_handle* h, const void* d_c, void* d_q, void* stream);
/* b = W sum_g P_g^T Gamma_g^T C_hat_g^-1 s_g (Sec. 3.1, Algorithm 1). */
int fewha_rhs(fewha_handle* h, const void* d_slopes, void* d_b, void* stream);
/* c = W phi and phi = W^T c, every layer with its own level count (Sec. 3.1). */
int fewha_dwt(fewha_handle* h, const void* d_phi, void* d_c, void* stream);
int fewha_idwt(fewha_handle* h, const void* d_c, void* d_phi, void* stream);
/* nodes = P phi (all sensors, Sec. 2) and its transpose phi = sum_g P_g^T nodes_g. */
int fewha_project(fewha_handle* h, const void* d_phi, void* d_nodes, void* stream);
int fewha_project_adj(fewha_handle* h, const void* d_nodes, void* d_phi, void* stream);
/* s = Gamma nodes (Sec. 2) and nodes = Gamma^T s. */
int fewha_slopes(fewha_handle* h, const void* d_nodes, void* d_s, void* stream);
int fewha_slopes_adj(fewha_handle* h, const void* d_s, void* d_nodes, void* stream);
/* out = C_hat^-1 s: (I - T) sigma^-2 (I - T) s for an LGS, sigma^-2 s for an NGS
 * (Eq. 2, Sec. 3.2). */
int fewha_noise_weight(fewha_handle* h, const void* d_s, void* d_out, void* stream);
/* s = A phi = Gamma P phi (Eq. 1) and phi = A^T s. */
int fewha_forward(fewha_handle* h, const void* d_phi, void* d_s, void* stream);
int fewha_forward_adj(fewha_handle* h, const void* d_s, void* d_phi, void* stream);
/* a~ = F W^T c (Algorithm 1, fitting step) and c = (F W^T)^T a. */
int fewha_fit(fewha_handle* h, const void* d_c, void* d_dm, void* stream);
int fewha_fit_adj(fewha_handle* h, const void* d_dm, void* d_c, void* stream);
/* `iters` Jacobi-PCG iterations on M c = b from c (in/out) with r0 = b - M c. */
int fewha_pcg(fewha_handle* h, const void* d_b, void* d_c, int iters, void* stream);
/* Copies of the handle's diagonals (n_coeffs each, handle element type, NULL skips):
 * D of Sec. 3.1 and J of Eq. (7). */
int fewha_get_diagonals(fewha_handle* h, void* d_D, void* d_J, void* stream);

/* ---- least-squares DM fitting over fitting directions ---------------------------
 * Sec. 4.1 notes that reconstructing more layers than there are DMs turns the fitting
 * step into a least-squares problem of its own, in place of the projection F.  Here the
 * commands minimise
 *
 *     sum_k w_k || Pi (A_k a - L_k phi) ||^2 + eps ||a||^2,    phi = W^T c,
 *
 * over the fitting directions theta_k: the pupil nodes x (n_fit + 1 per side, spacing
 * D / n_fit from -D/2, those with obs*D/2 <= |x| <= D/2) see layer l bilinearly at
 * x + theta_k h_l (L_k; the sample must stay inside the layer grid, else
 * FEWHA_ERR_GEOMETRY) and DM m as the sum of its actuators' bilinear hats at
 * x + theta_k h_m (A_k; zero beyond the outer actuators), and Pi removes the mean over
 * the pupil nodes (piston is not fitted).  The normal equations
 * (sum_k w_k A_k^T Pi A_k + eps I) a = sum_k w_k A_k^T Pi L_k phi are solved by
 * (unpreconditioned) CG from a = 0 until the recurrence residual falls to tol times the
 * right-hand side's norm or max_iters iterations have run; the CG inner products and
 * scalars are double, the operators the handle's element type. */
#define FEWHA_MAX_FIT_DIRS 32
#define FEWHA_MAX_FIT_NODES 256  /* largest n_fit                                      */
typedef struct fewha_lsfit {
    int n_dirs;              /* 1 .. FEWHA_MAX_FIT_DIRS                                */
    const double* theta_x;   /* direction of each [rad], host arrays of n_dirs          */
    const double* theta_y;
    const double* weight;    /* w_k >= 0, not all zero                                  */
    int n_fit;               /* pupil intervals per side, 1 .. FEWHA_MAX_FIT_NODES       */
    double eps;              /* Tikhonov weight >= 0                                    */
} fewha_lsfit;

/* d_c: coefficient vector (n_coeffs), d_dm_out: commands (n_act), both device pointers of
 * the handle's element type.  The fitting tables and CG vectors are built and kept in the
 * handle on the first call and rebuilt when the configuration changes (FEWHA_ERR_OOM if
 * their allocation fails).  Synchronises on `stream` (convergence is checked from the host
 * every FEWHA_MAX_ITERS iterations).  *iters_done and *rel_residual (both nullable) give
 * the iterations run and the final relative recurrence residual.  FEWHA_ERR_INVALID_ARG
 * for a null pointer, a count or n_fit out of range, a negative weight or eps, or no
 * positive weight; FEWHA_ERR_NONFINITE if the residual is not finite. */
int fewha_fit_ls(fewha_handle* h, const fewha_lsfit* cfg, const void* d_c, void* d_dm_out, double tol,
                 int max_iters, int* iters_done, double* rel_residual, void* stream);

/* ---- measurement --------------------------------------------------------------- */

/* Hot-path stages of one PCG iteration and of the frame, for timing one kernel alone. */
#define FEWHA_STAGE_IDWT 0      /* p = z + beta p and phi = W^T p, one CTA per layer       */
#define FEWHA_STAGE_SENSOR 1    /* sum of the pair terms, Gamma_g, C_hat_g^-1, Gamma_g^T    */
#define FEWHA_STAGE_LAYER 2     /* sum of the pair terms, W, + alpha D p, p.q               */
#define FEWHA_STAGE_VECTOR 3    /* x += a p, r -= a q, z = J^-1 r, r.z                     */
#define FEWHA_STAGE_RHS 4       /* C_hat^-1 and Gamma^T of the measured slopes             */
#define FEWHA_STAGE_FIT 5       /* DM fit and gain                                          */
#define FEWHA_STAGE_PROJ 6      /* R_y phi_l R_x^T per (sensor, layer) pair                  */
#define FEWHA_STAGE_PROJT 7     /* R_y^T u_g R_x per (sensor, layer) pair                    */
#define FEWHA_NUM_STAGES 8

/* Enqueue `reps` back-to-back launches of one stage's kernel on `stream`, working on the
 * handle's internal buffers (for timing with events around the call).  It overwrites
 * the handle's warm-start state: use a handle dedicated to measurement, or call
 * fewha_reset afterwards.  Asynchronous. */
int fewha_bench_stage(fewha_handle* h, int stage, int reps, void* stream);
/* Kernel launches one frame enqueues (for the launch count of a timed region; for
 * FEWHA_FLAG_AUGMENTED, a frame that has the previous frame's directions). */
int fewha_frame_launches(const fewha_handle* h, int* launches);

/* Device memory held by the instance (its own allocations, made at creation and on first
 * use of an option: the augmented PCG's directions, the reverse pass's record, the double
 * copy of a single-precision instance's converged solves), in bytes. */
int fewha_device_bytes(const fewha_handle* h, int64_t* bytes);

/* Test hook of the allocation-failure paths: the device allocations of the calling thread
 * succeed `after` more times, then one fails as if the device were out of memory (the
 * call making it returns FEWHA_ERR_OOM and releases what it had allocated); after < 0
 * turns the injection off.  Returns FEWHA_OK. */
int fewha_test_fail_alloc(int after);

/* Grid-wide waits of the persistent frame (FEWHA_FLAG_PERSISTENT): each gives up after
 * `polls` polls of its arrival counter (each poll a load and a 64 ns sleep; default
 * 1 << 20, well under a second).  `extra` is added to every wait's target; any value > 0 makes every wait run
 * out (tests of the timeout path).  Applies to frames enqueued after the call. */
int fewha_set_wait_limit(fewha_handle* h, unsigned polls, unsigned extra);

/* ---- differentiable reconstruction (a build addition: the paper has no gradients) --
 * The differentiable map is the CONVERGED reconstruction: c* solves M c = b (Eq. 6) to a
 * tolerance, the MAP estimate of Sec. 3.1, and a~ = F W^T c* (no gain).  Gradients follow
 * from implicit differentiation: lambda = M^-1 (F W^T)^T g_a by a second PCG on the
 * symmetric M, then dJ/ds = C_hat^-1 Gamma P W^T lambda, dJ/dalpha = -lambda^T D c* and
 * dJ/dw_l = alpha lambda_l^T D_l c*_l / w_l (D_l is proportional to 1 / w_l).
 * These calls use the frame's work vectors: they discard the warm residual (the next
 * frame forms r0 = b - M c explicitly) but keep the frame's warm start c.  Synchronous. */

/* x = M^-1 b by PCG from x = 0 (one recurrence, no restarts), until
 * sqrt(r^T J^-1 r / b^T J^-1 b) <= tol or max_iters iterations; the test is made every
 * FEWHA_MAX_ITERS - 1 iterations.  Precision 64: r is the recursively updated residual.
 * Precision 32 (mixed precision): the recurrence runs in float on a residual scaled to
 * unit norm, its iterate is accumulated in double, and whenever the float residual has
 * dropped tenfold the TRUE residual r = b - M x is formed in double (by an internal
 * double-precision copy of the instance, created on the first such call) and replaces it
 * (reliable updates); the test uses that true residual, so both precisions reach the same
 * tolerance.  *iters_done (nullable) counts the recurrence's iterations, *rel_residual
 * (nullable) the final relative residual; reaching max_iters is not an error.  Device
 * pointers of the handle's element type. */
int fewha_solve(fewha_handle* h, const void* d_b, void* d_x, double tol, int max_iters,
                int* iters_done, double* rel_residual, void* stream);

/* a~ = F W^T M^-1 b(s) with the solve above; the handle keeps c* for fewha_backward (in
 * double for precision 32, where b(s) and the fit are formed in double as well).
 * The solve (and the adjoint solve of fewha_backward) starts from the handle's previous
 * solution, if any: a nearby b or M (parameter sweeps, consecutive frames) converges in
 * fewer iterations. */
int fewha_reconstruct_converged(fewha_handle* h, const void* d_slopes, void* d_dm_out, double tol,
                                int max_iters, int* iters_done, double* rel_residual, void* stream);

/* Given d_grad_dm = dJ/da~ (n_act), the gradients of J at the last converged
 * reconstruction: d_grad_slopes (n_slopes, nullable), *grad_alpha (nullable) and
 * grad_cn2[n_layers] (nullable), the adjoint solve using the same tolerance and
 * iteration limit (precision 32: the adjoint solve as above, F^T, the slope map and the
 * per-layer sums in double, the slope gradient rounded to float at the end).  FEWHA_ERR_INVALID_ARG if no converged reconstruction is held (none
 * yet, or fewha_update_params since). */
int fewha_backward(fewha_handle* h, const void* d_grad_dm, void* d_grad_slopes, double* grad_alpha,
                   double* grad_cn2, void* stream);

/* ---- batched frames of many instances ------------------------------------------
 * Independent instances of uneven size (telescope, sensors, layers, DMs) reconstruct one
 * frame each in one CUDA-graph replay.  The frame of Algorithm 1 is the same sequence of
 * steps for every instance (right-hand side, initial residual, `iters` PCG iterations,
 * fit), so each step runs as ONE kernel launch over a work list of (instance, unit)
 * items, a unit being a layer, a sensor, a (sensor, layer) pair or a CTA of the vector
 * and fit kernels.  Results are bit-identical to the instances' own fewha_reconstruct.
 * All instances must share the device, precision, iteration count and warm-residual
 * mode; each runs on its own internal warm state (as fewha_reconstruct with
 * d_x_warm = NULL).  A handle may belong to several batches but not twice to one; a
 * batch whose member was destroyed fails with FEWHA_ERR_INVALID_ARG.  A batch is not
 * thread-safe, and no member may run other work concurrently with it. */
typedef struct fewha_batch fewha_batch;

/* Launch shape of a batch (what the autotuner chooses). */
typedef struct {
    int order;       /* 0: work items in the given instance order; 1: costliest instance first */
    int groups;      /* 1..FEWHA_BATCH_MAX_GROUPS: instances split (by balanced cost) into this
                        many independent launch chains that run concurrently */
    int vec_passes;  /* 1..8: passes of 4 elements per thread of the vector kernel's CTAs */
    int pair_threads;/* threads per CTA of the (sensor, layer) projection kernels: 0 = the
                        single-instance size (512 in single, 256 in double precision), or
                        half of it */
    int proj_taps;   /* unrolled taps of the adjoint projection: 0 = as few as every member's
                        geometry allows, 4 (only if every member allows it) or 8 */
    int vec_threads; /* threads per CTA of the vector kernel: 0 = 256, 256 or 512 */
} fewha_batch_config;

#define FEWHA_BATCH_MAX_GROUPS 8
#define FEWHA_BATCH_MAX_COUNT 4096

int fewha_batch_create(fewha_handle* const* handles, int count, fewha_batch** out);
void fewha_batch_destroy(fewha_batch* b);
const char* fewha_batch_last_error(const fewha_batch* b);
int fewha_batch_set_config(fewha_batch* b, const fewha_batch_config* cfg);
int fewha_batch_get_config(const fewha_batch* b, fewha_batch_config* cfg);

/* One frame of every instance: d_slopes[i] (device, the handle's element type) ->
 * d_dm_out[i].  Asynchronous on `stream`.  The graph is captured on the first call and
 * re-captured when the configuration, the warm-residual state or a member's parameters
 * change; new slope / command pointers only refresh a device argument table (uploaded on
 * `stream`). */
int fewha_batch_reconstruct(fewha_batch* b, const void* const* d_slopes, void* const* d_dm_out,
                            void* stream);

/* Autotuner: times the candidate configurations on `reps` batched frames of the given
 * slopes (CUDA events on `stream`): first every order x groups x vec_passes with the default
 * kernel shapes, then, from the best of those, every pair_threads x proj_taps x vec_threads
 * (the CTA sizes of the projection and vector kernels and the adjoint projection's tap
 * unroll, as far as the members' geometry allows), and keeps the fastest
 * in the batch and in a process-wide table keyed by the instances' shapes (a later batch
 * of the same shapes starts from it), and restores every member's warm state afterwards.
 * *best_us (nullable) receives the chosen configuration's mean frame time.  Synchronous. */
int fewha_batch_autotune(fewha_batch* b, const void* const* d_slopes, void* const* d_dm_out,
                         int reps, float* best_us, void* stream);

/* The same frame without a batch object: a batch for this exact handle list is created on
 * first use and cached (dropped when a member is destroyed). */
int fewha_reconstruct_batched(fewha_handle* const* handles, int count, const float* const* d_slopes,
                              float* const* d_dm_out, void* stream);
int fewha_reconstruct_batched_f64(fewha_handle* const* handles, int count,
                                  const double* const* d_slopes, double* const* d_dm_out,
                                  void* stream);

/* ---- no-allocation variant ------------------------------------------------------
 * The paper has no counterpart to this entry point; it serves callers that may not
 * allocate device memory at the time they need the operator.  A real-time control
 * loop typically allocates everything at start-up and then forbids cudaMalloc and
 * cudaFree, which can synchronise the whole device and take unbounded time; a
 * monitoring thread of such a loop may still want q = M c (for instance to check a
 * residual) without touching the handle's own scratch, which the frame uses.
 *
 * fewha_apply_M_noalloc computes the same q = M c as fewha_apply_M, but its
 * intermediate layer values, aperture-node vector and p.q partial sums live in one
 * static device block of FEWHA_NOALLOC_SCRATCH_BYTES inside the library (held by every
 * GPU that loads the library until the process exits), not in the handle.  It calls
 * no cudaMalloc, cudaFree or allocating routine.  It returns FEWHA_ERR_LIMIT, doing
 * nothing, when the instance needs more scratch than the block holds.  The need is
 * round256(n_coeffs * e) + round256(n_nodes * e) + 256 bytes, e the element size (4 or
 * 8) and round256 rounding up to a multiple of 256 (the MAORY-size instance needs
 * 1 455 872 bytes in double precision).  The first call on each device looks up the
 * block's device address (cudaGetSymbolAddress) with that device current and keeps it
 * for the life of the process: make that first call before any stream capture, and do
 * not tear the device's primary context down (cudaDeviceReset) while the library is in
 * use, since the kept address would then be stale.  All calls share the one block and leave their intermediates in it:
 * calls whose device work overlaps (different streams, or different handles on one
 * device) race on it and must be serialised by the caller.  Asynchronous on `stream`;
 * d_c and d_q are device pointers of the handle's element type. */
#define FEWHA_NOALLOC_SCRATCH_BYTES (2u << 20)
#define FEWHA_NOALLOC_MAX_DEVICES 64
int fewha_apply_M_noalloc(fewha_handle* h, const void* d_c, void* d_q, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FEWHA_H */
