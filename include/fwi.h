/*
 * fwi.h -- C ABI of the GB300 (sm_103a) library for the preconditioned
 * time-domain full-waveform-inversion gradient of Huang, Wang & Ren, "Two New
 * Gradient Precondition Schemes for Full Waveform Inversion" (arXiv:1406.1864).
 *
 * The library computes, for every shot of one velocity model:
 *   forward modelling of the constant-density acoustic wave equation
 *     1/v^2 u_tt - lap u = delta(x - x_s) f_s(t)                  [Sec. 2]
 *   traces d_s(x_r, t_n) = u_s(x_r, t_n) at the receivers         [Sec. 2]
 *   the OLS misfit J = 1/2 sum_s sum_r sum_n (d - d_obs)^2         [Sec. 2]
 *   or the time-integral misfit J = 1/2 || int_0^t (d - d_obs) ||^2 [Eq. 2]
 *   the adjoint (back-propagated residual) wavefield and the zero-lag
 *   cross-correlation gradient g = 2/v^3 sum_s int u_tt v_s dt      [Sec. 2]
 *   the shot illumination / pseudo-diagonal Hessian sum_s sum_n u^2 dt [Eq. 1]
 *   the diagonal of the localized subsurface-offset Hessian,
 *     H(x,h) = sum_s sum_n u(x + h e_x) u(x - h e_x) dt, h = 0..hmax [Sec. 3]
 *   and the preconditioned gradient g / (P + eps max P)             [Sec. 3.1]
 *
 * Discretisation (the paper names only "time domain finite difference"):
 * 8th-order centred Laplacian, second-order leapfrog in time, and an absorbing
 * sponge u_tt + 2 eta u_t of `sponge` cells added outside the model on every
 * side, the velocity there replicating the nearest model cell. The gradient is
 * the exact derivative of the discrete misfit; the part that falls on sponge
 * cells is added to the model edge cell they replicate.
 *
 * Conventions for every entry point:
 *   - Arrays are caller-owned, contiguous, C order. "DEVICE" arrays live in
 *     CUDA device memory of the current device; "HOST" arrays in host memory.
 *   - Physical-grid shapes only: [nz][nx] in 2-D, [nz][ny][nx] in 3-D.
 *     Padding is internal.
 *   - float is IEEE binary32 (the stencil arithmetic), double is binary64
 *     (misfit reductions only).
 *   - `ws` is a DEVICE workspace of at least the size reported by
 *     fwi_workspace_bytes() for the same operation and arguments; the library
 *     allocates no device memory of its own and keeps no state between calls,
 *     except the forward checkpoints that fwi_forward(save=1) leaves in `ws`
 *     for a following fwi_adjoint_apply().
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream). Work is
 *     queued on it; the call returns after queueing, except that argument
 *     errors are found before anything is queued and a status flag written by
 *     the kernels (timeouts, non-finite wavefields) is read back at the end of
 *     the call, which synchronises `stream` once.
 *   - Return value: FWI_OK or an error code; fwi_last_error() then gives a
 *     message (per host thread). On error the outputs are unspecified.
 *   - Dimensions: every entry point takes 2-D grids (ndim = 2). 3-D grids
 *     (ndim = 3; 25-point Laplacian, source f / dx^3) are taken by
 *     fwi_workspace_bytes, fwi_forward (save = 1 with ckpt =
 *     FWI_CKPT_SNAPSHOT and all shots in one group), fwi_adjoint_apply,
 *     fwi_adjoint_gradient (ckpt = FWI_CKPT_SNAPSHOT), fwi_illumination,
 *     fwi_offset_hessian_diag, fwi_precondition and fwi_autotune*, with
 *     [nz][ny][nx] model arrays and [hmax+1][nz][ny][nx] offset Hessians
 *     (offsets along x); the other entry points return FWI_ERR_INVALID_ARG
 *     for them.
 */
#ifndef FWI_H
#define FWI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FWI_OK = 0,
    FWI_ERR_INVALID_ARG = 1, /* bad size, index, pointer or option           */
    FWI_ERR_CFL = 2,         /* v dt / dx above the stability limit           */
    FWI_ERR_NOMEM = 3,       /* workspace smaller than fwi_workspace_bytes()  */
    FWI_ERR_CUDA = 4,        /* a CUDA runtime call failed                    */
    FWI_ERR_TIMEOUT = 5,     /* a bounded device wait gave up                 */
    FWI_ERR_UNSTABLE = 6     /* a wavefield became non-finite                 */
} fwi_status;

/* Stability limits of the leapfrog schemes: every cell needs
   v dt / dx <= FWI_CFL_LIMIT_2D (2-D, 17-point Laplacian) or
   FWI_CFL_LIMIT_3D (3-D, 25-point); calls over it return FWI_ERR_CFL. */
#define FWI_CFL_LIMIT_2D 0.5546f
#define FWI_CFL_LIMIT_3D 0.4528f

enum { FWI_MISFIT_OLS = 0, FWI_MISFIT_TIME_INTEGRAL = 1 };
enum { FWI_ILLUM_U2 = 0, FWI_ILLUM_UTT2 = 1 };
enum { FWI_PRECOND_NONE = 0, FWI_PRECOND_ILLUM = 1, FWI_PRECOND_OFFSET = 2 };
enum { FWI_CKPT_SPONGE = 0, FWI_CKPT_SNAPSHOT = 1 };
enum { FWI_SNAP_F32 = 0, FWI_SNAP_BF16 = 1, FWI_SNAP_F16S = 2 };
enum {
    FWI_OP_FORWARD = 0,        /* fwi_forward(save = 0)                     */
    FWI_OP_FORWARD_SAVE = 1,   /* fwi_forward(save = 1) + fwi_adjoint_apply */
    FWI_OP_GRADIENT = 2,       /* fwi_adjoint_gradient                      */
    FWI_OP_ILLUMINATION = 3,   /* fwi_illumination                          */
    FWI_OP_OFFSET_HESSIAN = 4, /* fwi_offset_hessian_diag                   */
    FWI_OP_PRECONDITION = 5,   /* fwi_precondition                          */
    FWI_OP_BORN = 6,           /* fwi_born                                  */
    FWI_OP_GN_HVP = 7,         /* fwi_gauss_newton_hvp                      */
    FWI_OP_MISFIT = 8,         /* fwi_misfit                                */
    FWI_OP_RECEIVER_FACTOR = 9, /* fwi_receiver_factor (kind from opts.precond
                                   is not used: see fwi_receiver_factor)     */
    FWI_OP_PRECONDITION_RECEIVER = 10, /* fwi_precondition_receiver        */
    FWI_OP_EXT_BORN = 11,      /* fwi_extended_born (any hext)              */
    FWI_OP_EXT_MIGRATION = 12, /* fwi_extended_migration (any hext)         */
    FWI_OP_PM_HESSIAN = 13     /* fwi_plessix_mulder_hessian                */
};

#define FWI_HMAX_LIMIT 12 /* largest offset (cells) of the offset Hessian */

/* Grid and time axis. */
typedef struct {
    int ndim;     /* 2, or 3 for the entry points that take 3-D grids        */
    int nz;       /* model rows (depth)                                       */
    int ny;       /* 1 in 2-D; model rows across in 3-D                       */
    int nx;       /* model columns                                            */
    float dx;     /* grid spacing (m), the same on every axis                 */
    float dt;     /* time step (s)                                            */
    int nt;       /* number of time levels t_n = n dt, n = 0..nt-1 (>= 2)     */
    int sponge;   /* sponge width P (cells), 1..64                            */
    float vref;   /* speed (m/s) that sets the damping; independent of v      */
    float refl;   /* sponge strength R in (0,1): eta_max = 3 vref ln(1/R)/(2 P dx) */
} fwi_grid;

/* Acquisition: one point source and nrec receivers per shot. */
typedef struct {
    int nshots;          /* >= 1                                                */
    int nrec;            /* receivers per shot, >= 0                             */
    const int *src;      /* HOST [nshots][3]: (z, y, x) model cell of the source; y = 0 in 2-D */
    const int *rec;      /* HOST [nshots][nrec][3]: (z, y, x) of each receiver   */
    const float *wavelet;/* DEVICE [nshots][nt]: source time function f_s(t_n)  */
} fwi_geometry;

/* What to compute besides the plain gradient. */
typedef struct {
    int misfit;     /* FWI_MISFIT_OLS or FWI_MISFIT_TIME_INTEGRAL              */
    int illum_mode; /* FWI_ILLUM_U2: sum u^2 dt; FWI_ILLUM_UTT2: sum u_tt^2 dt
                       (the omega^4 weighting of Eq. 1, by Parseval)           */
    int hmax;       /* offsets 0..hmax of the offset Hessian, 0..FWI_HMAX_LIMIT;
                       -1: not computed                                        */
    int precond;    /* FWI_PRECOND_*: preconditioner applied for grad_pre      */
    float eps;      /* water level of the division, > 0 (e.g. 1e-3)           */
    int ckpt;       /* forward state kept for the adjoint pass:
                       FWI_CKPT_SPONGE: every time level's sponge cells (exact;
                         the model part is rebuilt by reverse time stepping);
                         nshots * nt * sponge cells * 4 bytes
                       FWI_CKPT_SNAPSHOT: the whole field every snap_interval
                         levels, each segment re-propagated from its snapshot
                         during the adjoint pass (about sqrt(nt) snapshots) */
    int snap_prec;  /* snapshot storage: FWI_SNAP_F32 (u^n, u^{n-1} exact),
                       FWI_SNAP_BF16 / FWI_SNAP_F16S (u^n and u^n - u^{n-1},
                       each scaled by its own max-abs, as bfloat16 / float16) */
    int snap_interval; /* levels between snapshots; 0: ceil(sqrt(nt))       */
    int shot_group; /* 3-D: shots modelled at a time (the workspace holds one
                       group; the sums over groups are the sums over shots);
                       0: all shots at once                                    */
    int hess_v6;    /* 1: the illumination and offset-Hessian outputs, and the
                       preconditioners built from them, carry the 4 / v(x)^6
                       prefactor of H_a's diagonal [Sec. 3]; 0: without (Eq. 1
                       as printed)                                             */
} fwi_options;

/* Per-phase device times of the last call on this host thread, when enabled
   with fwi_profile_enable(1); CUDA events recorded on the call's stream. */
typedef struct {
    float forward_ms;    /* forward time loop (all shots)                      */
    float adjoint_ms;    /* backward time loop: adjoint, reconstruction, imaging */
    float other_ms;      /* set-up, misfit, fold, preconditioning              */
    int forward_launches;/* kernel launches in the forward time loop          */
    int adjoint_launches;/* kernel launches in the backward time loop         */
    int other_launches;  /* all other kernel launches of the call             */
} fwi_phase_times;

/* Workspace size (bytes) of operation `op` (FWI_OP_*) for these arguments.
   The returned size covers the padded wavefields, the sponge checkpoints of
   the adjoint pass (largest part: nshots * nt * sponge cells * 4 bytes) and
   the traces. opts may be NULL for FWI_OP_FORWARD. */
fwi_status fwi_workspace_bytes(const fwi_grid *grid, const fwi_geometry *geom,
                               const fwi_options *opts, int op, size_t *bytes);

/* Forward modelling of every shot [Sec. 2].
   v     DEVICE [nz][nx] velocity (m/s)
   seis  DEVICE [nshots][nt][nrec] output traces d_s^n(r) = u_s^n(x_r)
   save  1: leave the checkpoints for fwi_adjoint_apply() in ws (workspace of
         FWI_OP_FORWARD_SAVE); 0: do not (FWI_OP_FORWARD). */
fwi_status fwi_forward(const fwi_grid *grid, const fwi_geometry *geom, const fwi_options *opts,
                       const float *v, float *seis, int save, void *ws, size_t ws_bytes,
                       void *stream);

/* Gradient, with respect to v, of sum_s sum_n sum_r adj_src[s][n][r] * d_s^n(r):
   the adjoint of the Jacobian applied to adj_src [Sec. 2, zero-lag
   cross-correlation of forward and back-propagated wavefields]. Needs the
   checkpoints of a preceding fwi_forward(save = 1) with the same grid,
   geometry, options (opts->ckpt, snap_prec, snap_interval), v and ws, and
   nothing else on ws in between. The call overwrites the forward buffers of
   ws: a second fwi_adjoint_apply needs a new fwi_forward(save = 1).
   adj_src DEVICE [nshots][nt][nrec]; grad DEVICE [nz][nx] output. */
fwi_status fwi_adjoint_apply(const fwi_grid *grid, const fwi_geometry *geom,
                             const fwi_options *opts, const float *v, const float *adj_src,
                             float *grad, void *ws, size_t ws_bytes, void *stream);

/* The whole preconditioned gradient of one model [Sec. 2, Eq. 1-2, Sec. 3]:
   forward modelling, misfit (opts->misfit), adjoint source, back-propagation,
   imaging, illumination (always) and offset Hessian (opts->hmax >= 0).
   v        DEVICE [nz][nx] velocity
   d_obs    DEVICE [nshots][nt][nrec] observed traces
   grad     DEVICE [nz][nx] gradient dJ/dv
   grad_pre DEVICE [nz][nx] preconditioned gradient (opts->precond), or NULL
   misfit   DEVICE double, the misfit J, or NULL
   illum    DEVICE [nz][nx] illumination (opts->illum_mode), or NULL
   offh     DEVICE [hmax+1][nz][nx] offset-Hessian diagonal, or NULL */
fwi_status fwi_adjoint_gradient(const fwi_grid *grid, const fwi_geometry *geom,
                                const fwi_options *opts, const float *v, const float *d_obs,
                                float *grad, float *grad_pre, double *misfit, float *illum,
                                float *offh, void *ws, size_t ws_bytes, void *stream);

/* Preconditioned gradients of nmodels independent models of different sizes,
   computed together [Sec. 2, Eq. 1-2, Sec. 3, each model as in
   fwi_adjoint_gradient]: every time level of all models is one launch of the
   forward step and one of the backward step, whose CTAs take (model, tile,
   shots) chunks from one counter, so small models fill the GPU next to large
   ones. 1 <= nmodels <= FWI_BATCH_MAX. grids, geoms: HOST arrays [nmodels];
   every grid has the same nt (dx, dt, sponge and sizes may differ); opts is
   shared and needs ckpt = FWI_CKPT_SPONGE when nmodels > 1.
   v, d_obs, grad: HOST arrays [nmodels] of DEVICE pointers (model k's arrays
   as in fwi_adjoint_gradient); grad_pre, illum, offh: the same or NULL (and
   entries may be NULL); misfit: DEVICE double [nmodels] or NULL.
   Workspace: fwi_batch_workspace_bytes(). Errors name the model. */
#define FWI_BATCH_MAX 4
fwi_status fwi_batch_workspace_bytes(int nmodels, const fwi_grid *grids, const fwi_geometry *geoms,
                                     const fwi_options *opts, size_t *bytes);
fwi_status fwi_batch_gradient(int nmodels, const fwi_grid *grids, const fwi_geometry *geoms,
                              const fwi_options *opts, const float *const *v, const float *const *d_obs,
                              float *const *grad, float *const *grad_pre, double *misfit, float *const *illum,
                              float *const *offh, void *ws, size_t ws_bytes, void *stream);

/* Misfit only [Sec. 2 OLS misfit, or Eq. 2 with misfit =
   FWI_MISFIT_TIME_INTEGRAL]: forward modelling of every shot, the residual
   against d_obs and J in FP64, without checkpoints or the adjoint pass (the
   trial steps of a line search). v DEVICE [nz][nx]; d_obs DEVICE
   [nshots][nt][nrec]; misfit DEVICE double, written. opts may be NULL (OLS).
   Workspace of FWI_OP_MISFIT. 2-D. */
fwi_status fwi_misfit(const fwi_grid *grid, const fwi_geometry *geom, const fwi_options *opts, const float *v,
                      const float *d_obs, double *misfit, void *ws, size_t ws_bytes, void *stream);

/* Receiver-side factor R of the diagonal Hessian for a fixed receiver spread
   (every shot records at the same cells) [Sec. 1 and Sec. 3: H_a's sum over
   receivers of G(x, x_r) G(y, x_r), which Eq. 1 drops]. The source-side
   preconditioners (illumination, offset-Hessian diagonal) times R give the
   receiver-inclusive diagonal Hessian (fwi_precondition_receiver).
   kind = FWI_RECV_PLESSIX_MULDER: Plessix and Mulder's analytic factor,
     R(x) = asinh((x_max - x) / z) - asinh((x_min - x) / z), x_min, x_max the
     spread's extent along x (m), z the depth below the receivers' mean row
     (m), floored at dx / 2; out [nz][nx]; v may be NULL; no workspace.
   kind = FWI_RECV_GREEN: receiver Green's-function correlations,
     R(x, h) = sum_r sum_n G_r^n(x + h e_x) G_r^n(x - h e_x) dt, h = 0 ..
     max(hmax, 0) (opts->hmax; opts NULL: 0), G_r the wavefield of a source
     at receiver r with shot 0's wavelet, modelled in v; out
     [max(hmax, 0) + 1][nz][nx]; workspace of FWI_OP_RECEIVER_FACTOR (the
     receivers are modelled as nrec simultaneous independent sources).
   A geometry whose shots do not share one receiver spread is refused
   (FWI_ERR_INVALID_ARG). 2-D. */
enum { FWI_RECV_PLESSIX_MULDER = 0, FWI_RECV_GREEN = 1 };
fwi_status fwi_receiver_factor(const fwi_grid *grid, const fwi_geometry *geom, const fwi_options *opts, int kind,
                               const float *v, float *out, void *ws, size_t ws_bytes, void *stream);

/* Plessix and Mulder's approximate diagonal Hessian [Sec. 1], for any
   acquisition: out(x) = sum_s W_s(x) I_s(x), I_s the illumination of shot s
   (sum_n u^2 dt, or u_tt^2 dt with opts->illum_mode = FWI_ILLUM_UTT2; opts may
   be NULL) and W_s(x) = asinh((x_max(s) - x)/z_s) - asinh((x_min(s) - x)/z_s)
   from shot s's receiver extent along x and depth below its receivers' mean
   row (floored at dx / 2), as in fwi_receiver_factor. Consecutive shots with
   the same receiver cells share one illumination pass, so a fixed spread
   costs one pass of all shots and a spread that moves with every shot one
   pass per shot. v DEVICE [nz][nx]; out DEVICE [nz][nx]. Workspace of
   FWI_OP_PM_HESSIAN. 2-D; needs receivers. As a preconditioner:
   fwi_precondition(kind = FWI_PRECOND_ILLUM, scale = out). */
fwi_status fwi_plessix_mulder_hessian(const fwi_grid *grid, const fwi_geometry *geom, const fwi_options *opts,
                                      const float *v, float *out, void *ws, size_t ws_bytes, void *stream);

/* Preconditioning by a source-side scale times a receiver factor
   [Sec. 3.1 with the receiver term]: fwi_precondition with the scale
   P(x, h) = scale(x, h) * recv(x, min(h, recv_planes - 1)), recv_planes = 1
   (one factor for every offset, e.g. Plessix-Mulder's) or hmax + 1.
   kind FWI_PRECOND_ILLUM (scale [nz][nx], h = 0 only) or FWI_PRECOND_OFFSET
   (scale [hmax+1][nz][nx]). Workspace of FWI_OP_PRECONDITION_RECEIVER. */
fwi_status fwi_precondition_receiver(const fwi_grid *grid, const float *grad, const float *scale, int kind,
                                     int hmax, const float *recv, int recv_planes, float eps, float *out, void *ws,
                                     size_t ws_bytes, void *stream);

/* Extended Born modelling [Eq. 5]: traces of an extended velocity
   perturbation dv_ext(x, h) with horizontal subsurface offsets
   h = -hext..hext: the incident field at x + h scatters from x - h, with the
   scattering strength 2 c2(x) dv_ext(x, h) / v(x) of fwi_born (at hext = 0
   exactly fwi_born's operator up to rounding). dv_ext is edge-replicated into
   the sponge for every h. v DEVICE [nz][nx]; dv_ext DEVICE [2 hext + 1][nz][nx]
   (plane k is h = k - hext); dseis DEVICE [nshots][nt][nrec] output.
   0 <= hext <= FWI_HEXT_LIMIT. Workspace of FWI_OP_EXT_BORN. 2-D, sponge
   checkpoints (opts may be NULL). */
#define FWI_HEXT_LIMIT 6
fwi_status fwi_extended_born(const fwi_grid *grid, const fwi_geometry *geom, const fwi_options *opts, int hext,
                             const float *v, const float *dv_ext, float *dseis, void *ws, size_t ws_bytes,
                             void *stream);

/* Extended migration [Eq. 6], the adjoint of fwi_extended_born: the image
   [2 hext + 1][nz][nx] of the adjoint source adj_src [nshots][nt][nrec]
   (the generalized imaging condition: the back-propagated field at x - h
   correlated with the incident field at x + h; with the residual as adj_src,
   the subsurface-offset extended gradient, whose h = 0 plane is
   fwi_adjoint_gradient's grad). Forward modelling with sponge checkpoints,
   then the adjoint pass with the extended imaging. Workspace of
   FWI_OP_EXT_MIGRATION. 2-D (opts may be NULL). */
fwi_status fwi_extended_migration(const fwi_grid *grid, const fwi_geometry *geom, const fwi_options *opts, int hext,
                                  const float *v, const float *adj_src, float *image, void *ws, size_t ws_bytes,
                                  void *stream);

/* Self-test of failure detection on the GPU: one warp waits on an mbarrier
   that no thread arrives at, with the bounded wait every step kernel uses
   (%globaltimer limit of limit_us microseconds, 1 .. 10,000,000). The wait
   gives up, the kernel raises the timeout status and returns, and the call
   returns FWI_ERR_TIMEOUT, as a step kernel's wait that ran out would; the
   context stays usable. ws: DEVICE, >= 256 bytes, 256-byte aligned (the
   status word). Any other return value is a failure of the mechanism. */
fwi_status fwi_selftest_wait(unsigned limit_us, void *ws, size_t ws_bytes, void *stream);

/* Born modelling [Eq. 4, as the exact derivative of fwi_forward's discrete
   traces]: dseis = J dv, the change of the traces along the velocity change
   dv, by the tangent-linear scheme (u and du = J dv advanced together).
   v, dv DEVICE [nz][nx]; dseis DEVICE [nshots][nt][nrec] output. Workspace
   of FWI_OP_BORN. 2-D, sponge checkpoints (opts may be NULL). */
fwi_status fwi_born(const fwi_grid *grid, const fwi_geometry *geom, const fwi_options *opts, const float *v,
                    const float *dv, float *dseis, void *ws, size_t ws_bytes, void *stream);

/* Gauss-Newton Hessian-vector product [Sec. 3, the Hessian of the
   linearised problem]: hv = J^T W^T W J dv, Born modelling of dv followed by
   the adjoint pass with the weighted Born traces as adjoint source (the
   gradient's imaging and fold: hv has the units of fwi_adjoint_gradient's
   grad). W is the misfit's data weighting: the identity for the OLS misfit
   (opts NULL or misfit = FWI_MISFIT_OLS), the time integral C of Eq. 2 for
   misfit = FWI_MISFIT_TIME_INTEGRAL. v, dv DEVICE [nz][nx]; hv DEVICE
   [nz][nx] output. Workspace of FWI_OP_GN_HVP. 2-D, sponge checkpoints. */
fwi_status fwi_gauss_newton_hvp(const fwi_grid *grid, const fwi_geometry *geom, const fwi_options *opts,
                                const float *v, const float *dv, float *hv, void *ws, size_t ws_bytes,
                                void *stream);

/* Tile autotuning: times every compiled tile variant and shot-chunk size of
   the gradient's forward step (with the offset Hessian if opts->hmax >= 0)
   and of its backward step, for a few time levels of this very problem (v,
   geometry, a workspace of FWI_OP_GRADIENT), and keeps the fastest for the
   process, keyed by kind of step, padded grid shape and shot count: later
   plans of the same shape use them (a batch uses model 0's). choice: NULL
   or int[4] = forward variant, forward chunk, backward variant, backward
   chunk. The timing leaves ws in an unspecified state (the next call's
   set-up rewrites it). fwi_autotune_reset() forgets all choices.
   3-D grids (opts as for a 3-D gradient: ckpt = FWI_CKPT_SNAPSHOT): the
   compiled ring-depth / CTAs-per-SM variants of the 3-D forward and backward
   steps are timed on the first shot group, keyed by padded shape and group
   size. A 3-D item is one z-segment of one column (64 x 8 cells) of one
   shot; the chunks are the z-segments per column, which fwi_autotune
   chooses from the item count and the resident CTAs of the chosen variant
   (and reports), and fwi_autotune_set takes as given (0: that choice). */
fwi_status fwi_autotune(const fwi_grid *grid, const fwi_geometry *geom, const fwi_options *opts, const float *v,
                        void *ws, size_t ws_bytes, void *stream, int *choice);
/* Keep a given choice (int[4] as above) for this problem's shape, as if
   fwi_autotune had picked it: to reproduce a tuning, or to pin a variant. */
fwi_status fwi_autotune_set(const fwi_grid *grid, const fwi_geometry *geom, const fwi_options *opts,
                            const int *choice);
fwi_status fwi_autotune_reset(void);

/* A recorded gradient: fwi_exec_gradient_create() checks its arguments as
   fwi_batch_gradient() does (nmodels = 1 is fwi_adjoint_gradient), uploads
   the geometry tables into ws, and records the call's device work -- set-up,
   both time loops, misfit, outputs: some 2 nt kernel launches -- into a CUDA
   graph bound to these buffers. fwi_exec_run() replays it on `stream` (one
   graph launch) and reads the status like a direct call; change the contents
   of v[] and d_obs[] between runs, not their addresses. `stream` must not be
   the legacy default stream (it cannot be captured). The exec holds no
   device memory of its own; ws and the buffers must outlive it. */
typedef struct fwi_exec_s fwi_exec;
fwi_status fwi_exec_gradient_create(int nmodels, const fwi_grid *grids, const fwi_geometry *geoms,
                                    const fwi_options *opts, const float *const *v, const float *const *d_obs,
                                    float *const *grad, float *const *grad_pre, double *misfit,
                                    float *const *illum, float *const *offh, void *ws, size_t ws_bytes,
                                    void *stream, fwi_exec **out);
fwi_status fwi_exec_run(fwi_exec *ex, void *stream);
fwi_status fwi_exec_destroy(fwi_exec *ex);
/* Overlap the upload of the observed traces with the forward pass: the
   recorded gradient reads d_obs only after its forward time loop, and waits
   there for the exec's input event. fwi_exec_input_ready() records that
   event on `stream` (typically the stream copying d_obs from the host),
   after the work already queued on it. Call it before fwi_exec_run(); runs
   without a new call proceed once the last recording has completed (at
   once if it was never recorded). The caller orders the next write of
   d_obs after the run (e.g. `stream` waits for the run's stream). */
fwi_status fwi_exec_input_ready(fwi_exec *ex, void *stream);

/* Shot illumination, the pseudo-diagonal Hessian of Eq. 1:
   illum DEVICE [nz][nx] = sum_s sum_n u_s^n(x)^2 dt (FWI_ILLUM_U2) or
   sum_s sum_n (u_tt)_s^n(x)^2 dt (FWI_ILLUM_UTT2), from a forward modelling. */
fwi_status fwi_illumination(const fwi_grid *grid, const fwi_geometry *geom,
                            const fwi_options *opts, const float *v, float *illum, void *ws,
                            size_t ws_bytes, void *stream);

/* Diagonal of the localized subsurface-offset Hessian [Sec. 3], source side,
   horizontal offsets h = 0..opts->hmax (opts->hmax >= 0):
   offh DEVICE [hmax+1][nz][nx] = sum_s sum_n u_s^n(x + h e_x) u_s^n(x - h e_x) dt,
   u = 0 outside the padded grid. offh[0] equals the illumination. 3-D grids:
   offh [hmax+1][nz][ny][nx], offsets along x, shots in groups of
   opts->shot_group. Workspace of FWI_OP_OFFSET_HESSIAN. */
fwi_status fwi_offset_hessian_diag(const fwi_grid *grid, const fwi_geometry *geom,
                                   const fwi_options *opts, const float *v, float *offh,
                                   void *ws, size_t ws_bytes, void *stream);

/* Diagonal preconditioning [Sec. 3.1, Fig. 5]: out = grad / (P + eps max P),
   P = scale[0] (kind FWI_PRECOND_ILLUM: scale is an illumination [nz][nx]) or
   P = |scale[0]| + 2 sum_{h=1..hmax} |scale[h]| (FWI_PRECOND_OFFSET: scale is an
   offset Hessian [hmax+1][nz][nx]); on 3-D grids [nz][ny][nx] and
   [hmax+1][nz][ny][nx]. All DEVICE; ws of FWI_OP_PRECONDITION (geometry and
   options not needed). */
fwi_status fwi_precondition(const fwi_grid *grid, const float *grad, const float *scale, int kind,
                            int hmax, float eps, float *out, void *ws, size_t ws_bytes,
                            void *stream);

/* Forward modelling without a caller workspace (no counterpart in the paper:
   a deployment aid). For callers that cannot allocate device memory -- code
   where cudaMalloc is not allowed or not wanted, a host framework that owns
   all device memory through its own pool, a plugin handed only its inputs and
   outputs -- this computes exactly what fwi_forward(save = 0) computes, in a
   scratch array the library holds itself: FWI_NOALLOC_SCRATCH_BYTES of device
   memory, reserved on every GPU that loads this part of the library and kept
   until the process exits. It allocates no device memory.
   Only 2-D grids (ndim = 2).
   v     DEVICE [nz][nx] velocity; seis DEVICE [nshots][nt][nrec] output traces.
   Errors, all returned before any device work: FWI_ERR_INVALID_ARG for a NULL
   or 3-D grid, a NULL geometry, bad coordinates, a NULL v or (nrec > 0) a NULL
   seis, as fwi_forward; FWI_ERR_NOMEM (with a message giving both sizes) when
   the problem's forward workspace, fwi_workspace_bytes(..., FWI_OP_FORWARD,
   ...), exceeds FWI_NOALLOC_SCRATCH_BYTES. Like fwi_forward, the call waits
   for its stream at the end to read the kernels' status word.
   The first call on a device (and the first after a device reset) looks up
   the scratch array's device address (cudaGetSymbolAddress).
   All calls share the one array, which keeps the previous call's contents
   (every call clears what must start at zero): calls that may overlap on the
   GPU -- on different streams, or from different host threads -- race and
   corrupt each other's results; serialise them. */
#define FWI_NOALLOC_SCRATCH_BYTES (32u << 20)
fwi_status fwi_forward_noalloc(const fwi_grid *grid, const fwi_geometry *geom, const float *v,
                               float *seis, void *stream);

/* Per-call phase timing with CUDA events (off by default). */
fwi_status fwi_profile_enable(int on);
fwi_status fwi_profile_last(fwi_phase_times *out);

/* Message of the last error on this host thread ("" if none). */
const char *fwi_last_error(void);

/* Library version, 100 * major + minor. */
int fwi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FWI_H */
