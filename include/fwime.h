/*
 * libfwime -- C ABI of the GB300 (sm_103a) implementation of the FWIME operators.
 *
 * Barnier, Biondi, Clapp & Biondi, "Full waveform inversion by model extension:
 * practical applications" (arXiv 2206.02362).  Every entry point below applies
 * one operator named in the paper's Theory section:
 *   fwime_forward       f(m)            nonlinear forward modelling, Eq. 1
 *   fwime_born          B(m) dm         non-extended Born modelling, Eq. 8
 *   fwime_born_adj      B*(m) d         its adjoint (Born gradient operator), Eq. 8
 *   fwime_born_ext      B~(m) p~        Born extended with horizontal subsurface
 *                                       offsets, Eq. 1 (data-correcting term)
 *   fwime_born_ext_adj  B~*(m) d        extended imaging condition, Eqs. 2-5
 *   fwime_tomo          T(m,p~) dm      data-space tomographic operator, Eq. 9
 *   fwime_tomo_adj      T*(m,p~) d      its adjoint (tomographic gradient), Eq. 9
 *   fwime_gradient      Phi_eps and B* r + T* r with r = f + B~ p~ - d_obs at a
 *                       fixed p~ (Eqs. 1, 7-9), the spline operator S = I.
 *
 * Discretisation (the paper defers it to a companion paper; this library fixes
 * one reading and documents it): 2-D acoustic constant-density wave equation,
 * 2nd order in time, 8th order in space on a uniform grid; a Cerjan-type sponge
 * of `sponge` points on every side plus a 4-point zero halo; point sources with
 * amplitude w[n]/(dx dz); receivers record the pressure at time n dt, n=0..nt-1
 * (sample 0 is always zero).  Subsurface offsets h = (ih - (nh-1)/2) dx act
 * along x with the symmetric convention: p~(x, h) couples the source wavefield
 * at x-h to the receiver side at x+h.
 *
 * Memory layout, all row-major with x fastest, FP32:
 *   v        [nz][nx]            velocity in m/s (the model m of the paper, S = I)
 *   w        [nshot][nt]         source wavelet of each shot
 *   d        [nshot][nt][nrec]   data (shot records), time-major per shot
 *   dv, grad [nz][nx]            model-space perturbation / gradient
 *   pt       [nh][nz][nx]        extended perturbation p~ (on the FD grid)
 *
 * Ownership: every float pointer is caller-owned and is a DEVICE pointer unless
 * the context was switched to host I/O with FWIME_OPT_HOST_IO, in which case it
 * is a host pointer (pinned memory recommended) and the library copies through
 * its own device staging buffers.  The library never frees caller memory.  The
 * context owns its workspace (wavefields, rings, checkpoints, status word).
 *
 * Execution: calls enqueue work on the context's CUDA stream and return without
 * waiting, except that with FWIME_OPT_HOST_IO the call waits for its outputs.
 * Device-side errors are latched in a status word read by fwime_sync().
 *
 * Errors: every int-returning call returns FWIME_OK (0) or a negative code;
 * no exception, abort or trap crosses the ABI.  fwime_last_error_detail()
 * returns a one-line description of the last failure on that context.
 */
#ifndef FWIME_H
#define FWIME_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FWIME_OK        0
#define FWIME_EINVAL   -1   /* bad argument, shape or geometry */
#define FWIME_ENOMEM   -2   /* workspace does not fit the budget or cudaMalloc failed */
#define FWIME_ECFL     -3   /* dt * vmax * sqrt(6.5016 (1/dx^2 + 1/dz^2)) >= 2 */
#define FWIME_ECUDA    -4   /* a CUDA runtime call failed */
#define FWIME_ETIMEOUT -5   /* a device-side bounded wait gave up */
#define FWIME_EBUSY    -6   /* the context is in use (graph capture in progress) */

typedef struct fwime_ctx fwime_ctx;

/* Physical grid nz x nx at spacing dz, dx; `sponge` absorbing points per side;
 * nt time samples at dt; nh subsurface offsets (odd, 1 = non-extended). */
typedef struct {
    int nz, nx, sponge, nt, nh;
    float dz, dx, dt;
} fwime_grid;

/* One point source per shot and a fixed receiver spread, physical-grid indices.
 * The arrays are host memory and are copied by fwime_create. */
typedef struct {
    int nshot;
    const int *src_iz, *src_ix;
    int nrec;
    const int *rec_iz, *rec_ix;
} fwime_geom;

/* Options for fwime_set_option / fwime_get_option. */
enum {
    FWIME_OPT_SHOTS_PER_BATCH = 1, /* shots advanced together per launch; 0 = as many as fit */
    FWIME_OPT_SEGMENT = 2,         /* checkpoint/ring segment length K in time steps; 0 = auto */
    FWIME_OPT_PLAIN = 3,           /* 1 = plain path: one shot per launch, host-driven steps */
    FWIME_OPT_GRAPH = 4,           /* 1 = capture each operator call in a CUDA graph and replay */
    FWIME_OPT_HOST_IO = 5,         /* 1 = I/O pointers are host memory */
    FWIME_OPT_ZCHUNK = 6,          /* rows per warp in the stencil kernel; 0 = auto */
    FWIME_OPT_LAUNCHES = 7,        /* read-only: kernels launched by the last operator call */
    FWIME_OPT_WORKSPACE = 8,       /* read-only: bytes of device workspace held */
    FWIME_OPT_PROFILE = 9,         /* 1 = bracket every kernel launch with CUDA events (no graphs) */
    FWIME_OPT_REUSE_BACKGROUND = 10, /* 1 = B / B~ keep the background wavefield's segment-start states of
                                       every shot (when they fit in device memory) and a following B* / B~*
                                       with the SAME v and w pointers starts from them instead of its own
                                       checkpointing sweep (one propagation fewer).  The caller guarantees
                                       that v and w are not modified in between; any other operator call
                                       drops the states.  0 (default) frees them. */
    FWIME_OPT_BACKGROUND_REUSED = 11, /* read-only: 1 if the last call started from states an earlier call
                                         kept (the background states above, or the state of
                                         fwime_gradient_forward) */
    FWIME_OPT_TIME_LAG = 12,        /* 0 (default): B~ / B~* extend with nh horizontal subsurface offsets;
                                       L > 0: with nh time lags tau_i = (i - (nh-1)/2) L dt, the symmetric
                                       convention (source side at t - tau, receiver side at t + tau):
                                       e^n(x) = sum_i b p~(x,i) D2t q0^{n - 2 (i-(nh-1)/2) L}(x).  Every
                                       operator (B~, B~*, T, T*, gradient, objective, VP solve) then uses
                                       the lag form. */
    FWIME_OPT_FREE_SURFACE = 13,    /* 1: pressure-release free surface at the top physical row (iz = 0)
                                       instead of the top sponge: q = 0 there and the 4 rows above hold
                                       the odd mirror of the 4 rows below after every step (forward and
                                       adjoint); receivers on the surface row record 0.  Not available in
                                       fwime_forward_group. */
    FWIME_OPT_BATCH_USED = 15       /* read-only: shots per batch the last operator call planned (the
                                       planner splits the shots into equal batches that fit) */
};

/* Kernel families, for fwime_profile_read. */
enum {
    FWIME_K_PROP = 0,     /* wave-equation time step (forward and adjoint) */
    FWIME_K_SCATTER = 1,  /* extended scattering and its transpose */
    FWIME_K_IMAGE = 2,    /* imaging-condition reductions */
    FWIME_K_POINTS = 3,   /* receiver recording / injection */
    FWIME_K_OTHER = 4     /* model preparation, copies, reductions */
};

/* Operators, for fwime_workspace_bytes. */
enum {
    FWIME_OP_FORWARD = 0, FWIME_OP_BORN, FWIME_OP_BORN_ADJ, FWIME_OP_BORN_EXT,
    FWIME_OP_BORN_EXT_ADJ, FWIME_OP_TOMO, FWIME_OP_TOMO_ADJ, FWIME_OP_GRADIENT, FWIME_OP_OBJECTIVE
};

/* Creates a context on the current CUDA device.  `max_workspace_bytes` caps the
 * device memory the context may hold (0 = no cap); `cuda_stream` is a
 * cudaStream_t (NULL = legacy default stream).  Returns FWIME_EINVAL for an
 * invalid grid/geometry (receivers or sources outside the physical grid, nh
 * even, nt < 2, non-positive spacing). */
int fwime_create(fwime_ctx **out, const fwime_grid *g, const fwime_geom *geo,
                 size_t max_workspace_bytes, void *cuda_stream);

/* Device bytes operator `op` needs for `shots_per_batch` shots advanced
 * together with segment length `segment` (0 = the defaults). */
int fwime_workspace_bytes(const fwime_grid *g, const fwime_geom *geo, int op,
                          int shots_per_batch, int segment, size_t *bytes);

int fwime_set_option(fwime_ctx *ctx, int option, long long value);
int fwime_get_option(fwime_ctx *ctx, int option, long long *value);

/* f(m): d[nshot][nt][nrec] = recorded pressure of every shot (Eq. 1). */
int fwime_forward(fwime_ctx *ctx, const float *v, const float *w, float *d);

/* B(m) dv: Born data of the velocity perturbation dv[nz][nx] (Eq. 8). */
int fwime_born(fwime_ctx *ctx, const float *v, const float *w, const float *dv, float *d);

/* B*(m) d: dv[nz][nx] (=, or += when accumulate=1) summed over shots. */
int fwime_born_adj(fwime_ctx *ctx, const float *v, const float *w, const float *d,
                   float *dv, int accumulate);

/* B~(m) p~: data of the extended perturbation pt[nh][nz][nx] (Eq. 1). */
int fwime_born_ext(fwime_ctx *ctx, const float *v, const float *w, const float *pt, float *d);

/* B~*(m) d: extended image pt[nh][nz][nx] (=, or +=), summed over shots. */
int fwime_born_ext_adj(fwime_ctx *ctx, const float *v, const float *w, const float *d,
                       float *pt, int accumulate);

/* T(m, p~) dv: derivative of m -> B~(m) p~ along dv (Eq. 9). */
int fwime_tomo(fwime_ctx *ctx, const float *v, const float *w, const float *pt,
               const float *dv, float *d);

/* T*(m, p~) d: dv[nz][nx] (=, or +=), summed over shots (Eq. 9). */
int fwime_tomo_adj(fwime_ctx *ctx, const float *v, const float *w, const float *pt,
                   const float *d, float *dv, int accumulate);

/* FWIME objective at fixed p~ and its gradient (Eqs. 1, 7-9):
 *   r = f(m) + B~(m) p~ - d_obs,  Phi = 1/2 ||r||^2 + eps^2/2 ||D p~||^2,
 *   grad[nz][nx] = B* r + T* r (overwritten), *objective = Phi (host double,
 *   written when the call's work has completed, i.e. after fwime_sync).
 * D = diag(|ih - (nh-1)/2| + 1) is this library's reading of the paper's
 * invertible, modified DSO operator; it does not enter the gradient. */
int fwime_gradient(fwime_ctx *ctx, const float *v, const float *w, const float *pt,
                   const float *dobs, float eps, float *grad, double *objective);

/* The objective Phi of fwime_gradient alone (Eq. 1 at fixed p~): the forward
 * sweep f + B~ p~ and the residual norm, without the adjoint sweep -- the
 * extra objective evaluation a line search makes (Computational aspects).
 * *objective (host double) is written when the work has completed. */
int fwime_objective(fwime_ctx *ctx, const float *v, const float *w, const float *pt,
                    const float *dobs, float eps, double *objective);

/* The FWIME gradient of fwime_gradient in two calls, for reverse-mode differentiation (Eqs. 1, 7-9):
 *
 * fwime_gradient_forward runs the forward sweep only -- f + B~ p~, the residual r = f + B~ p~ - d_obs and
 * Phi (*objective, host double, written at the next fwime_sync) -- and keeps what the adjoint sweep needs in
 * the context: the background and scattered wavefields' states at every segment start for every shot
 * (4 nseg nshot padded fields) and r (nshot nt nrec floats).  No adjoint kernel runs.  When that state does
 * not fit in device memory next to the adjoint sweep's workspace (or with FWIME_OPT_TIME_LAG or the plain
 * path), only Phi is computed and nothing is kept.
 *
 * fwime_gradient_backward runs the adjoint sweep -- B* r + T* r into grad[nz][nx] (=, or += when
 * accumulate) -- from that state when it was kept for the same v, w and pt pointers (the caller guarantees
 * that their contents did not change in between), and releases it; otherwise it runs the whole gradient
 * (the forward sweep again, then the adjoint sweep), which needs dobs and eps.  FWIME_OPT_BACKGROUND_REUSED
 * reads 1 after a backward call that started from the kept state.  Device pointers only. */
int fwime_gradient_forward(fwime_ctx *ctx, const float *v, const float *w, const float *pt, const float *dobs,
                           float eps, double *objective);
int fwime_gradient_backward(fwime_ctx *ctx, const float *v, const float *w, const float *pt, const float *dobs,
                            float eps, float *grad, int accumulate);

/* Variable projection step (Theory section, Eqs. 2-5): approximately minimises
 *   Phi_eps,m(p~) = 1/2 ||B~(m) p~ - dres||^2 + eps^2/2 ||D p~||^2
 * with `niter` iterations of linear conjugate gradients on the normal
 * equations (B~* B~ + eps^2 D* D) p~ = B~* dres, starting from and overwriting
 * pt[nh][nz][nx].  dres[nshot][nt][nrec] = d_obs - f(m); both device pointers.
 * history (host, niter+1 doubles, may be NULL) receives Phi_eps,m at every
 * iterate, written at the next fwime_sync.  Each iteration applies B~ and B~*
 * once (4 propagations + the background recomputation); the scalars stay on
 * the device.  D = diag(|ih - (nh-1)/2| + 1) as in fwime_gradient. */
int fwime_vp_solve(fwime_ctx *ctx, const float *v, const float *w, const float *dres, float eps, int niter,
                   float *pt, double *history);

/* Linear spline re-parametrisation S of the model (Theory section, Eq. 1: m lives on a coarse spline
 * grid and the wave equation sees v = S m; gradients map back with S*, Eqs. 7-9).  Nodes zs[nzs] x xs[nxs]
 * are host arrays in metres, strictly increasing (they may extend past the grid); the physical grid
 * point (iz, ix) sits at (iz dz, ix dx).  Between nodes k and k+1 a point takes the weights 1 - a and a,
 * a = (c - node_k) / (node_k+1 - node_k); beyond the end nodes it takes the end node's value (bilinear
 * in 2-D).  adjoint = 0: out[nz][nx] (=, or += when accumulate) = S in[nzs][nxs];
 * adjoint = 1: out[nzs][nxs] (=, or +=) = S* in[nz][nx].  in and out are device pointers;
 * FWIME_EINVAL for unsorted or non-finite nodes. */
int fwime_spline(fwime_ctx *ctx, int nzs, const float *zs, int nxs, const float *xs, const float *in, float *out,
                 int adjoint, int accumulate);

/* Model-space multiscale step (Theory section, the model-space multi-scale workflow after Eq. 9: the model
 * inverted on one spline grid is the starting model on a finer one; the Marmousi2 example halves the spline
 * spacing whenever the step-length search fails).  mf[nzf][nxf] = the linear spline of mc[nzc][nxc] on the
 * coarse nodes zc x xc (the S of fwime_spline) evaluated at the fine nodes zf x xf.  When every coarse node
 * is also a fine node, S on the fine nodes applied to mf equals S on the coarse nodes applied to mc.  Node
 * arrays are host memory (metres, strictly increasing, finite; else FWIME_EINVAL); mc and mf are device
 * pointers.  Asynchronous on the context's stream. */
int fwime_spline_refine(fwime_ctx *ctx, int nzc, const float *zc, int nxc, const float *xc, const float *mc, int nzf,
                        const float *zf, int nxf, const float *xf, float *mf);

/* f(m) for a group of contexts at once (Eq. 1; the Computational-aspects
 * section's shots are independent): ctxs[i] has its own grid, record length
 * and shots, with model v[i], wavelets w[i] and output d[i] (device pointers,
 * layouts as fwime_forward).  Each time step of all members runs as ONE
 * kernel launch (plus one recording launch): shots of uneven grid sizes share
 * the launch, members drop out as their nt ends.  All members must use the
 * same stream and fit all their shots in one batch (else FWIME_ENOMEM); at most
 * 4096 members.  Results equal n separate fwime_forward calls bit for bit. */
int fwime_forward_group(fwime_ctx *const *ctxs, int n, const float *const *v, const float *const *w,
                        float *const *d);

/* Autotuner of the stencil kernel's tiling: plans the workspace of operator
 * `op` (so the batch size is the one the operator will use), then times the
 * time-step kernel on that batch for candidate rows-per-warp chunkings with
 * CUDA events (two passes, the faster of each kept) and keeps the fastest,
 * except that among chunkings within 1 % of it the one whose last wave of
 * resident warps is fullest wins (FWIME_OPT_ZCHUNK).  Synchronous.  Returns
 * the chosen chunking and its time per launch (either pointer may be NULL). */
int fwime_autotune(fwime_ctx *ctx, int op, int *zchunk, float *us_per_launch);

/* ---- Request server (continuous batching; Computational aspects: shots are independent modelling
 * tasks that a host layer dispatches to the GPU) ----
 *
 * A server is a context created by fwime_server_create; it takes requests, not operator calls.  Each
 * request is one forward-modelling job f(m) (Eq. 1) or one FWIME-gradient job (Phi and B* r + T* r at a
 * fixed p~, Eqs. 1, 7-9) with its own grid, geometry, record length and nh.  fwime_submit copies the
 * request's grid and geometry, checks it and queues it; it returns at once with a ticket.  A dispatcher
 * thread admits queued requests in submission order as soon as the request's device memory
 * (fwime_request_bytes: the operator's workspace with all its shots in one batch, as fwime_workspace_bytes
 * plans it, plus staging when host_io = 1) fits under memory_budget and fewer than max_active requests are
 * in flight -- while earlier requests are still running.  Each admitted request runs on a context and a
 * CUDA stream of its own, so admitted requests overlap on the GPU; forward requests admitted together
 * share one launch per time step (as fwime_forward_group).  Completion is detected with CUDA events; the
 * request's memory then returns to the budget.  fwime_poll (non-blocking) and fwime_wait (blocking)
 * collect a finished request's result once; the ticket is then forgotten.
 *
 * Buffers: with host_io = 0 every pointer is a DEVICE pointer; with host_io = 1 they are host pointers
 * (pinned memory recommended) that the server stages through device memory counted in the admission.
 * Either way they are the caller's and must stay valid and unchanged until the request is collected.
 * Layouts as for fwime_forward (v, w, d) and fwime_gradient (pt, dobs, grad).
 *
 * Errors: fwime_submit returns FWIME_EINVAL for a bad request (unknown kind, grid, geometry, missing
 * buffer) and FWIME_ENOMEM when the request alone needs more than the budget (it could never be
 * admitted); a message is then available from fwime_server_last_error (per calling thread).  A request
 * that fails on the GPU side is collected with its error code in fwime_result.status.  fwime_sync on a
 * server context waits until every submitted request has finished; fwime_destroy waits for them too,
 * then stops the server's threads. */
enum { FWIME_REQ_FORWARD = 0, FWIME_REQ_GRADIENT = 1 };
#define FWIME_SERVE_PLAIN 1   /* fwime_server_create option: one request at a time, one shot per launch,
                                 host-driven steps (the comparison path) */

typedef struct {
    int kind;                      /* FWIME_REQ_FORWARD or FWIME_REQ_GRADIENT */
    fwime_grid grid;
    fwime_geom geom;               /* host arrays, copied by fwime_submit */
    int host_io;                   /* 1: the buffers below are host memory */
    const float *v, *w;            /* v[nz][nx], w[nshot][nt] */
    const float *pt, *dobs;        /* gradient: p~[nh][nz][nx], d_obs[nshot][nt][nrec] */
    float *d;                      /* forward output d[nshot][nt][nrec] */
    float *grad;                   /* gradient output grad[nz][nx] */
    float eps;                     /* gradient: DSO weight of Phi */
} fwime_request;

typedef struct {
    int done;                      /* 1: finished, outputs written (result collected) */
    int status;                    /* FWIME_OK or the request's error code */
    double objective;              /* gradient requests: Phi */
    double queued_s;               /* submission to admission, seconds */
    double latency_s;              /* submission to completion seen by the server, seconds */
    double enqueue_s;              /* host time spent enqueuing the request's launches (its launch group's) */
} fwime_result;

/* memory_budget: device bytes the admitted requests may hold together (0 = 80 % of the free memory now);
 * max_active: requests in flight at most (1..1024); options: 0 or FWIME_SERVE_PLAIN. */
int fwime_server_create(fwime_ctx **out, size_t memory_budget, int max_active, int options);
/* Device bytes the server admits a request with (workspace + staging). */
int fwime_request_bytes(const fwime_request *req, size_t *bytes);
int fwime_submit(fwime_ctx *server, const fwime_request *req, uint64_t *ticket);
/* Non-blocking: res->done = 0 while the request runs; on 1 the result is collected and the ticket freed.
 * FWIME_EINVAL for an unknown (or already collected) ticket. */
int fwime_poll(fwime_ctx *server, uint64_t ticket, fwime_result *res);
/* Blocks until the request has finished, then collects it as fwime_poll does. */
int fwime_wait(fwime_ctx *server, uint64_t ticket, fwime_result *res);
int fwime_server_last_error(char *buf, size_t n);

/* Schedule autotuner for operator `op`: segment length K (the automatic one, half and double, unless
 * FWIME_OPT_SEGMENT fixes it) x shots per launch S (the largest equal batch that fits at that K, and half
 * of it) x the stencil's rows per warp.  At every (K, S) it plans the operator's workspace, picks the stencil
 * chunking as fwime_autotune does, times the operator's extension kernels once over a full segment of K x S
 * (step, shot) pairs with CUDA events, and models the time per shot as
 *   ((nt - 1) props t_stencil + nseg (scatters t_scatter + images t_image)) / S
 * with the operator's launches per step and per segment.  The fastest schedule is set as the context's
 * FWIME_OPT_SEGMENT, FWIME_OPT_SHOTS_PER_BATCH and FWIME_OPT_ZCHUNK and returned.  Synchronous; the
 * workspace contents are overwritten (no operator state survives it).  Not with the plain path. */
typedef struct {
    int segment, shots_per_batch, zchunk;
    float us_stencil, us_scatter, us_image;   /* per launch at the chosen schedule */
    double us_per_shot;                       /* modelled operator time per shot */
} fwime_schedule;
int fwime_autotune_schedule(fwime_ctx *ctx, int op, fwime_schedule *res);

/* Waits for the context's stream and returns the latched device status
 * (FWIME_OK, FWIME_ECFL, FWIME_ETIMEOUT) or FWIME_ECUDA; clears the latch. */
int fwime_sync(fwime_ctx *ctx);

/* With FWIME_OPT_PROFILE on: waits for the stream, then returns for kernel
 * family `kernel` the summed CUDA-event duration (ms) of its launches since the
 * last reset, the number of launches, and the algorithmic bytes they moved
 * (the compulsory reads/writes of the operator's definition, e.g. 16 bytes per
 * grid-point update of a plain time step).  reset = 1 clears the counters. */
int fwime_profile_read(fwime_ctx *ctx, int kernel, double *ms, long long *launches, double *bytes, int reset);

int fwime_last_error_detail(fwime_ctx *ctx, char *buf, size_t n);

/* ---- Allocation-free forward modelling (the paper has no counterpart) ----
 * For callers that cannot call cudaMalloc (inside another allocator or memory
 * pool, with device memory reserved up front, or on a thread that must not
 * enter the driver's allocator): f(m) of fwime_forward with no context and no
 * allocation.  Its scratch (padded model, sponge tables, offsets, a status
 * word, two wavefields per shot) is one file-scope device array of
 * FWIME_STATIC_SCRATCH_BYTES held by every GPU that loads the library until
 * the process exits.  v[nz][nx], w[nshot][nt] and d[nshot][nt][nrec] are
 * caller-owned DEVICE pointers; work is enqueued on cuda_stream (NULL = legacy
 * default stream).  Every call looks up the array's address on the current
 * device (cudaGetSymbolAddress, which allocates nothing), copies the source
 * and receiver offsets in from host memory and waits for the model check on
 * its stream; the time steps are then enqueued and the call returns without
 * waiting for them.  Every call shares the array and leaves its contents
 * behind (wavefields and status are cleared at the start of a call); calls
 * whose work overlaps on the GPU race on it and must be serialised by the
 * caller.  Returns FWIME_ECFL (d untouched, no time step run) for a velocity
 * that is not positive or breaks the stability bound of FWIME_ECFL;
 * FWIME_ENOMEM when the problem needs more than FWIME_STATIC_SCRATCH_BYTES
 * (see fwime_static_scratch_bytes); FWIME_EINVAL for a bad grid or geometry;
 * each with a message for fwime_static_last_error. */
#define FWIME_STATIC_SCRATCH_BYTES ((size_t)32 << 20)
size_t fwime_static_scratch_bytes(const fwime_grid *g, const fwime_geom *geo);
int fwime_forward_static(const fwime_grid *g, const fwime_geom *geo, const float *v, const float *w,
                         float *d, void *cuda_stream);
int fwime_static_last_error(char *buf, size_t n);
const char *fwime_strerror(int code);
void fwime_destroy(fwime_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* FWIME_H */
