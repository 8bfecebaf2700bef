/*
 * swf.h -- C ABI of the GB300 (sm_103a) scattered-wave-function (SWF) Dirac solver.
 *
 * The method (G. Torgrimsson, "Solving the Dirac equation on a GPU for strong-field processes
 * in multidimensional background fields"):
 *   Sec. II, Eq. 6:  (i D-slash - 1) psi_scat = A-slash psi_back, D_mu = d_mu + i A_mu (Eq. 2),
 *                    psi_scat(t_out) = 0 (Eq. 7), marched back to t_in.
 *   Sec. II.A:       spatial derivatives by FFT (Eq. 10); Dormand-Prince 5(4) in time.
 *   Sec. II, Eq. 8:  pair number N(m, n) from overlaps (Eq. 9) at t_in.
 *   Sec. IV:         Breit-Wheeler amplitude M = M_ss + M_bs + M_sb (Eqs. 13-14), finite-time
 *                    part accumulated during the march (Eqs. 17, 33-35), past part at t_in
 *                    (Eqs. 24-27) with the energy projectors of Eq. 23.
 *
 * Conventions shared by every entry point:
 *   - units c = hbar = m = 1; metric (+,-,-,-); A_mu covariant; Dirac representation.
 *   - Hamiltonian form of Eq. 6:  d psi_s/dt = -i [ H0 psi_s + V (psi_s + psi_b) ],
 *     H0 = alpha.kappa + beta per Fourier mode e^{i kappa.x}, V = A_0 + alpha^k A_k.
 *   - spinors u_s(p) = (1 + p-slash) R_s / sqrt(2 p0 (p0 - p^x)), v_s(p) = (1 - p-slash) R_s / ...
 *     with R_+ = (1,1,1,1)/2, R_- = (1,-1,-1,1)/2 (Eqs. A44-A45); spin s = +1 or -1.
 *   - grid: n[a] points on [-L[a]/2, L[a]/2) per axis a = x, y, z; mode kappa_j =
 *     2 pi j'/L with j' = j for j < (n+1)/2 and j - n otherwise.  n[a] = 1 marks a trivial axis:
 *     the field does not depend on it, its delta function is stripped, and the marched wave
 *     carries its background's momentum along it.
 *   - a spinor field on the grid is stored planar per component, x fastest:
 *     element (c, z, y, x) at index ((c*nz + z)*ny + y)*nx + x, complex (re, im) interleaved,
 *     complex64 (8 B) or complex128 (16 B) per the precision.
 *
 * Ownership and errors: the caller owns every pointer it passes; the library owns its
 * workspace inside swf_ctx.  Every entry point returns a status, never aborts or traps, leaves
 * outputs untouched on a validation error, and records a message for swf_last_error().
 * Device-pointer entry points ("_dev") are asynchronous on the given stream (NULL = the
 * context's stream); the host-pointer entry point solve_swf is synchronous.
 */
#ifndef SWF_H
#define SWF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SWF_OK = 0,
  SWF_EINVAL = 1,       /* invalid argument (message says which) */
  SWF_ENOMEM = 2,       /* device allocation failed or exceeds the context's workspace limit */
  SWF_ECUDA = 3,        /* a CUDA runtime call failed */
  SWF_ENUMERIC = 4,     /* a non-finite value appeared in the march */
  SWF_ETIMEOUT = 5,     /* a bounded device-side wait gave up */
  SWF_EUNSUPPORTED = 6  /* valid request outside what the library implements */
} swf_status;

typedef enum { SWF_SCHWINGER = 0, SWF_BREIT_WHEELER = 1 } swf_process;

/* March precision.  SWF_C128: complex128 march and FP64 everywhere.  SWF_C64: complex64
 * march with FP32 accumulation; phases of the plane waves are formed in FP64 and rounded once;
 * the projections at t_in (FFT and spinor overlaps) run in FP64. */
typedef enum { SWF_C128 = 0, SWF_C64 = 1 } swf_precision;

/* Background field kinds; prm[] holds the parameters in the order listed. */
typedef enum {
  SWF_FIELD_ZERO = 0,          /* A = 0 */
  SWF_FIELD_SAUTER_GAUSS = 1,  /* {E, omega, lambda}: A_1 = (E/omega) sech^2(omega t) exp(-r^2/lambda^2),
                                  r over the non-trivial axes; lambda <= 0 means no spatial envelope */
  SWF_FIELD_PULSE_GAUSS = 2,   /* {a0, omega0, tau, w, wy}: A_1 = a0 sin(omega0 (t - y))
                                  exp(-(t-y)^2/tau^2 - x^2/w^2) [* exp(-y^2/wy^2) if wy > 0] */
  SWF_FIELD_SINGLE_E = 3,      /* {E0, omega, kx, ky, kz}: Eq. 11, A_0 = -(E0/kx) sin(kx x)
                                  exp(-(omega t)^2 - (kx x)^2 - (ky y)^2 - (kz z)^2) */
  SWF_FIELD_DOUBLE_E = 4       /* {E0, omega, kx, ky, kz, Dx}: Eq. 12, A_0^one(x+Dx) + A_0^one(x-Dx) */
} swf_field_kind;

typedef struct {
  int32_t kind;     /* swf_field_kind */
  int32_t reserved;
  double prm[8];
} swf_field;

typedef struct {
  int32_t n[3];     /* points per axis (1 = trivial axis); each n > 1 must factor into 2, 3, 5 and be <= 512 */
  int32_t n_steps;  /* fixed Dormand-Prince steps from t_out down to t_in */
  double L[3];      /* box lengths (ignored on trivial axes) */
  double t_in, t_out;
} swf_grid;

/* One problem instance.  Schwinger: an electron m = (s, p) (one U march) and optionally a
 * positron n = (r, q) (one V march when SWF_WANT_FULL_N).  Breit-Wheeler: electron (s, p),
 * positron (r, q) and photon (k, eps); U and V are marched together. */
typedef struct {
  swf_field field;
  swf_grid grid;
  double p[3]; int32_t s;
  int32_t r;   double q[3];
  double k[3]; double eps[3];  /* photon momentum (a grid mode) and polarisation eps_mu = (0, eps) */
  int32_t flags;               /* SWF_WANT_* */
  int32_t reserved;
} swf_instance;

#define SWF_WANT_SPECTRUM 1  /* Schwinger: |C(m,(r,q))|^2 for every grid positron q */
#define SWF_WANT_FULL_N   2  /* Schwinger: march V too and return both lines of Eq. 8 */
#define SWF_ADAPTIVE      4  /* step-size-controlled march (Sec. II.A: Dopri5 with relative and
                                absolute tolerances, swf_set_tolerances); the first step is
                                (t_in - t_out)/n_steps and at most 100 n_steps + 100 attempts are made
                                (SWF_ENUMERIC beyond); pass kernels only.  Breit-Wheeler: U and V share
                                the controller (the larger of their error norms decides), the
                                integrand of Eq. 17 is integrated over the accepted steps (Eq. 35);
                                not with SWF_BW_PARTIAL (SWF_EUNSUPPORTED) */
#define SWF_BW_PARTIAL    8  /* Breit-Wheeler: integrate the partial-integration integrands of Sec. IV
                                (Eqs. 30-33) during the march instead of adding the past terms of
                                Eqs. 25-27 to the finite-time terms of Eq. 17; amp holds the same three
                                terms and M.  Each weighted stage transforms the stage value and the
                                source term -iV(psi_s + psi_b) of both waves on the grid (about twice
                                the work of the default form) */

/* Per-instance scalar results (complex values as (re, im) pairs).
 * Schwinger: amp = {C(m,n), D(m,n), A(m,n), B(m,n)} for the listed positron n = (r, q);
 *            prob = {|C + D|^2, |A + B|^2}.  Without SWF_WANT_FULL_N: amp = {C(m,(r,q)),
 *            C(m,(-r,q)), 0, 0} and prob = {|C(m,(r,q))|^2, |C(m,(-r,q))|^2}.
 * Breit-Wheeler: amp = {M_ss, M_bs, M_sb, M}, prob = {|M|^2, 0}.
 * diag = {||psi_U(t_in)||^2, ||psi_V(t_in)||^2} (grid inner product, Eq. 9). */
typedef struct {
  double amp[8];
  double prob[2];
  double diag[2];
} swf_result;

typedef struct swf_ctx swf_ctx;

/* Create a context on CUDA device `device` with its own stream.  Returns SWF_ECUDA if the
 * device is absent.  *ctx is NULL on failure. */
swf_status swf_create(swf_ctx** ctx, int device);

/* Release the context and all its device memory.  NULL is accepted. */
swf_status swf_destroy(swf_ctx* ctx);

/* Thread-local message for the last non-OK status of this thread ("" if none). */
const char* swf_last_error(void);

/* Highest-level call: solve n_inst instances (host descriptors) and write host outputs.
 * results:  n_inst swf_result (required).
 * spectrum: optional (NULL = not wanted); for Schwinger instances with SWF_WANT_SPECTRUM,
 *           |C(m,(r,q))|^2 for r = +1, -1 and every grid mode j, laid out per instance as
 *           [2][nz][ny][nx] doubles, instances back to back in input order (instances without
 *           the flag take no room).  The positron at mode index j has q = -kappa_j.
 * Synchronous: returns after the results are in host memory. */
swf_status solve_swf(swf_ctx* ctx, int n_inst, const swf_instance* inst, swf_process process,
                     swf_precision prec, swf_result* results, double* spectrum);

/* Same as solve_swf with device output buffers (results: n_inst swf_result in device memory;
 * spectrum as above, in device memory), asynchronous on `stream`. */
swf_status solve_swf_dev(swf_ctx* ctx, int n_inst, const swf_instance* inst, swf_process process,
                         swf_precision prec, swf_result* results_dev, double* spectrum_dev,
                         void* stream);

/* Full Schwinger pair numbers N(m, n) (Eq. 8, both lines; Eq. 9 inner product) for every
 * electron m = (s, p) of `electrons` and every positron n = (r, q) of `positrons`, as a scan over
 * momenta (Sec. II.A).  All instances must share field, grid and time window (EINVAL
 * otherwise); along trivial axes (n = 1) every p must be equal and every q = -p.  Only p, s of
 * the electrons and q, r of the positrons are read.  Marches each electron's U wave and each
 * positron's V wave once (n_e + n_p marches rather than 2 n_e n_p) and forms C, A, B and D as
 * complex FP64 matrix products over the grid (components x sites).
 * results: host array of n_e * n_p swf_result, row-major [m][n], with the layout of a
 * SWF_WANT_FULL_N instance: amp = {C, D, A, B}, prob = {|C + D|^2, |A + B|^2},
 * diag = {||psi_U,m||^2, ||psi_V,n||^2}.  Synchronous; uses the context's stream and workspace. */
swf_status swf_pair_matrix(swf_ctx* ctx, int n_e, const swf_instance* electrons, int n_p,
                           const swf_instance* positrons, swf_precision prec, swf_result* results);

/* Breit-Wheeler photon scan (Sec. IV): the photon enters only the integrals of Eq. 14, not the
 * Dirac equations for U and V, so one march of the instance's U and V (its p, s, q, r, field and
 * grid; its own k and eps are not read) gives the amplitude M(k_j, eps_j) of every photon of a list,
 * each with the past/finite split of Eqs. 17 and 25-27.  A photon wave packet sampled on grid
 * momenta (Sec. IV, closing paragraphs) is, by linearity, sum_j w_j M(k_j, eps_j).
 * k, eps: host [n_photons][3] (each k a grid mode along non-trivial axes, k = p + q along trivial
 *         ones, k != 0; eps real, eps_mu = (0, eps)).
 * weights: host [n_photons] complex (re, im) or NULL; packet_out: host 4 complex (8 doubles):
 *         sum_j w_j (M_ss, M_bs, M_sb, M)_j, or NULL (needs weights).
 * amp_out: host [n_photons][4] complex (8 doubles per photon): M_ss, M_bs, M_sb, M.
 * Instances with SWF_ADAPTIVE or SWF_BW_PARTIAL give SWF_EUNSUPPORTED; invalid photons SWF_EINVAL
 * (outputs untouched).  Synchronous; uses the context's stream and workspace. */
swf_status swf_bw_photons(swf_ctx* ctx, const swf_instance* inst, int n_photons, const double* k,
                          const double* eps, const double* weights, swf_precision prec,
                          double* amp_out, double* packet_out);

/* Lower-level: march n_inst instances' electron (bg = 0, background u_s(p) e^{-ipx}) or
 * positron (bg = 1, background v_r(q) e^{+iqx}) scattered wave from psi_s(t_out) = 0 to t_in
 * (Eqs. 6-7) and write psi_s(t_in) to psi_out_dev: per instance 4*nx*ny*nz complex values in
 * the march precision, instances back to back.  All instances must share the grid. */
swf_status swf_march_dev(swf_ctx* ctx, int n_inst, const swf_instance* inst, int bg,
                         swf_precision prec, void* psi_out_dev, void* stream);

/* Lower-level: one evaluation of the right-hand side of Eq. 6,
 * out = -i [ H0 psi + V(t) (psi + psi_b(t)) ], for one instance and background bg (0 = U,
 * 1 = V), psi and out in the march precision and the layout above (device memory, may not
 * alias).  Uses a workspace of one spinor field held by the context. */
swf_status swf_rhs_dev(swf_ctx* ctx, const swf_instance* inst, int bg, swf_precision prec,
                       double t, const void* psi_dev, void* out_dev, void* stream);

/* Lower-level: the C-spectrum of Eq. 8's line 2 first term for n_inst electron waves at t_in:
 * C(m,(r,q)) = (U_scat(m) | V_back(r,q)) for every grid mode, in FP64.  psi_dev as written by
 * swf_march_dev (march precision); c_out_dev receives complex128 [inst][2][nz][ny][nx],
 * prob_out_dev (optional) the |C|^2 doubles in the same layout. */
swf_status swf_spectrum_dev(swf_ctx* ctx, int n_inst, const swf_instance* inst,
                            swf_precision prec, const void* psi_dev, double* c_out_dev,
                            double* prob_out_dev, void* stream);

/* Kernel timing hook (tracing).  When enabled, the context records a CUDA event pair on the
 * launching stream around every kernel it launches and accumulates the elapsed time per kernel
 * family.  swf_profile_read synchronises the context's events and returns up to max_entries
 * families: names (max_entries * 32 chars, NUL-terminated), total milliseconds and launch counts;
 * it then clears the accumulators.  *total_launches (optional) receives every kernel launched by
 * the context since the previous read, timed or not. */
swf_status swf_profile_enable(swf_ctx* ctx, int on);
swf_status swf_profile_read(swf_ctx* ctx, int max_entries, char* names, double* total_ms,
                            long long* launches, int* n_entries, long long* total_launches);

/* March path selection: 0 = automatic (the fused cluster kernel for (2+1)D 256 x 256
 * complex64 marches that keep the z-spin sectors apart, the pass kernels otherwise; a large
 * fused march gives some of its fields to the pass kernels, run concurrently on the SMs that the
 * 16-CTA clusters leave free), 1 = pass kernels only, 2 = the fused kernel of path 0 (the
 * pushed-transpose kernel of path 5) for every field, 3 = fused kernel with two CTAs per SM, 4 = fused kernel whose threads pull the two
 * transposes of an evaluation through distributed shared memory, 5 = fused kernel whose
 * transposes are pushed by the bulk-copy engine while the threads compute (2 to 5 still fall back
 * to the pass kernels where the fused kernel does not apply).  All fused variants give the same
 * arithmetic in the same order. */
swf_status swf_set_march_path(swf_ctx* ctx, int path);

/* Status of the context's last march on the pushed-transpose fused kernel (march paths 0, 2
 * and 5): *status = 0 when every transpose arrived, 1 when a CTA's receive wait ran out (after
 * about half a second), in which case that CTA stopped copying and wrote NaN for its rows while
 * keeping to the cluster's barriers, so the kernel still ended.  Synchronises the context's
 * device (the march may have run on a caller's stream).  0 if no such march has run. */
swf_status swf_fused_status(swf_ctx* ctx, int* status);
/* Diagnostic for the bounded waits above: on = 1 makes the pushed-transpose kernel issue none of
 * its transposes, so that every receive wait runs out (tests only; default 0). */
swf_status swf_set_fused_drop(swf_ctx* ctx, int on);

/* Tolerances of step-size-controlled marches (SWF_ADAPTIVE): a Dormand-Prince 5(4) step is
 * accepted when the RMS over the field's complex entries of |e|/(atol + rtol max(|y_n|, |y_n+1|))
 * is at most 1 (the largest over the fields of one call), e the difference of the fifth- and
 * fourth-order solutions; the next step is h min(10, max(0.2, 0.9 err^(-1/5))).  Defaults: the
 * paper's rtol = 1e-5, atol = 1e-10 (Sec. II.A). */
swf_status swf_set_tolerances(swf_ctx* ctx, double rtol, double atol);
/* Accepted and rejected steps of the context's last step-size-controlled march. */
swf_status swf_march_stats(swf_ctx* ctx, long long* accepted, long long* rejected);

/* Step-size-controlled marches of this context that ran as one graph launch with the attempt
 * loop on the device (a while node of a CUDA graph: every attempt, its acceptance or rejection
 * and the stop decided by the controller kernel; Sec. II.A's Dopri5 control with no host round
 * trip per attempt).  Where that graph form is unavailable, or kernel timing is on, the march
 * replays attempts from the host in growing chunks instead (the same attempts and results). */
swf_status swf_device_loop_marches(swf_ctx* ctx, long long* count);

/* Repeated marches.  on = 1 (default): within one call, a field whose march repeats another's
 * is marched once: the same field, window and background wave, or (with the z axis trivial,
 * p_z = 0 and A_3 = 0, where the spin along z is conserved) the other spin s = -1 vs +1 (or r),
 * whose scattered wave is exactly the first with components 1 and 2 negated (R_- = diag(1, -1,
 * -1, 1) R_+ and every operator of Eq. 6 keeps {0, 3} and {1, 2} apart; App. A.5 Eq. A44).
 * on = 0 marches every field.  Results agree either way (up to the sign of zeros). */
swf_status swf_set_dedupe(swf_ctx* ctx, int on);

/* Batching of uneven grids (Sec. II.A: many instances marched at once).  Instance groups of one
 * call that sit on different grids but share the time grid (t_out, t_in, step count) and the
 * non-trivial axes, and that run on the pass kernels at fixed steps (Schwinger, and
 * Breit-Wheeler with the integrand of Eq. 17), can be marched together, up to eight groups at a
 * time: one launch per pass serves all of them, persistent blocks taking (group, block) work
 * items from a device counter, largest grids first, and one CUDA graph replays their step
 * pairs.  Each group's results are bitwise those of marching it alone.
 * mode = 1 (default): together when the groups hold fewer than 4 Mi fields x grid points (above
 * that each group fills the GPU alone); 2: always together; 0: one group after another. */
swf_status swf_set_multi_grid(swf_ctx* ctx, int mode);
/* Fields (U or V waves) actually marched by this context since its creation (a diagnostic of
 * the library; the paper has no counterpart). */
swf_status swf_fields_marched(swf_ctx* ctx, long long* count);
/* Of those, the fields marched by the fused cluster kernel (the rest ran on the pass kernels). */
swf_status swf_fields_fused(swf_ctx* ctx, long long* count);
/* The split of an n_fields fused march (path 0) between the fused kernel and the pass kernels run
 * concurrently on the SMs its clusters leave free, for `clusters` resident 16-CTA clusters on a
 * device of `sms` SMs: *pass_fields receives the number of fields (the last ones) given to the
 * pass kernels, 0 for no split.  Host-only (no device needed); SWF_EINVAL for negative counts or
 * a NULL pointer. */
swf_status swf_plan_split(int n_fields, int clusters, int sms, int* pass_fields);

/* Launch shapes of the pass kernels (rows per block of the x passes, tile width of the y and z
 * passes, 256 or 128 threads per block).  on = 1 (default): the first march of each grid
 * shape in this context times the candidate shapes (a few launches each, before the march
 * starts) and keeps the fastest;
 * on = 0: a fixed rule from the grid size.  A shape only decides which lines a block
 * transforms, so results are bitwise the same either way.  Part of the batching design
 * (Sec. II.A: many instances per launch); the paper names no tuner. */
swf_status swf_set_autotune(swf_ctx* ctx, int on);

/* Allocation-free variant of swf_rhs_dev (the paper has no counterpart: this is a service of
 * the library).  Some callers cannot call cudaMalloc: host applications that own all device
 * memory and hand it out from a pool of their own, and latency-critical loops that cannot
 * absorb the device-wide synchronisation that cudaFree brings.  This entry point allocates
 * nothing: it needs no context and takes its workspace from one fixed device array of about
 * 4.1 MiB that every GPU loading the library holds until the process exits.  The caller passes
 * inputs and outputs exactly as for swf_rhs_dev; the evaluation runs on the current CUDA
 * device, on `stream` (NULL = the default stream), asynchronously.
 * Limit: grids of at most 65536 points (for example 256 x 256 or 64 x 64 x 16) in either
 * precision; larger grids return SWF_EINVAL with a message.
 * The first call on a device (and the first after the device's context was reset) looks up
 * the array's device address (cudaGetSymbolAddress) and sets the kernels' shared-memory limits;
 * make that first call before any stream capture begins.  All calls on a device share the
 * array and it keeps the last call's contents (every value a call reads is written earlier by
 * the same call), so calls that overlap on the GPU -- on different streams or from different
 * host threads -- race on it and must be serialised by the caller. */
swf_status swf_rhs_noalloc(const swf_instance* inst, int bg, swf_precision prec, double t,
                           const void* psi_dev, void* out_dev, void* stream);

/* Caps the context's device workspace (bytes; 0 = no cap).  Requests that need more return
 * SWF_ENOMEM before touching the device. */
swf_status swf_set_workspace_limit(swf_ctx* ctx, size_t bytes);

/* ---------------------------------------------------------------------------------------
 * Surrogate network for parameter and momentum scans.  The paper scans with the worldline-
 * instanton approximation (App. A) and improves points with the SWF solver (Sec. V); here a
 * multilayer perceptron trained on solver outputs plays that screening role:
 *   x = (E, omega, lambda, p_x, p_y, s) -> 4 x [256, GELU] -> (mu, log sigma^2),
 * mu estimating ln P with P = sum_r |C((s,p),(r,q = -p))|^2 and sigma its own error estimate
 * (Gaussian negative log-likelihood L = mean[(y - mu)^2 exp(-l) + l]/2 on the standardised
 * target).  BF16 operands on the tensor cores, FP32 accumulation, FP32 master weights, Adam.
 * Parameters: per layer W [out][in] row-major then b [out], layers 6->256->256->256->256->2,
 * FP32, swf_mlp_param_count() values in all.  norm (14 floats): feature shifts [6], feature
 * scales [6] (x' = (x - shift) * scale), target shift y0 and scale ys (y' = (y - y0) * ys).
 * x: [B][6] float, y: [B] float, out: [B][2] float (mu and log sigma^2 in the target's units),
 * all device pointers; calls are asynchronous on `stream` (NULL = default stream). */
typedef struct swf_mlp swf_mlp;
int swf_mlp_param_count(void);
swf_status swf_mlp_create(swf_mlp** m, int device, const float* init_params /* host */, int max_batch,
                          const float* norm /* host, 14 floats */);
swf_status swf_mlp_destroy(swf_mlp* m);
/* Inference over any number of rows B >= 1 (one persistent tensor-core kernel, no workspace
 * beyond the network's own). */
swf_status swf_mlp_forward(swf_mlp* m, const float* x_dev, int B, float* out_dev, void* stream);
/* Waits for the network's last inference call and reports SWF_ETIMEOUT if one of its waits on
 * the tensor cores or on a weight copy gave up (about two seconds each; the kernel then returns
 * with its outputs incomplete), else SWF_OK. */
swf_status swf_mlp_status(swf_mlp* m);
/* Gradient of the loss on one batch (B <= max_batch) into grad_dev (param_count floats,
 * optional) and the loss into loss_dev (optional); parameters unchanged. */
swf_status swf_mlp_gradients(swf_mlp* m, const float* x_dev, const float* y_dev, int B, float* grad_dev,
                             float* loss_dev, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on one batch with learning rate lr. */
swf_status swf_mlp_train_step(swf_mlp* m, const float* x_dev, const float* y_dev, int B, float lr,
                              float* loss_dev, void* stream);
/* The network's activation GELU(x) = x Phi(x) and its derivative Phi(x) + x phi(x),
 * elementwise on n device floats, as the network's kernels evaluate them (erf by Abramowitz and
 * Stegun's formula 7.1.26, |error| <= 1.5e-7); asynchronous on `stream`. */
swf_status swf_mlp_activation(const float* x_dev, int n, float* gelu_dev, float* grad_dev, void* stream);
swf_status swf_mlp_get_params(swf_mlp* m, float* params_host);

#ifdef __cplusplus
}
#endif

#endif /* SWF_H */
