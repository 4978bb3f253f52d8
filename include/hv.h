/*
 * hv.h -- C ABI of libhv, a single-GPU (sm_103a) library for the matrix-free
 * Gauss-Newton Hessian-vector product of 2D acoustic seismic inversion, and
 * the forward map, Born map, migration and misfit gradient built from the same
 * wave solves.
 *
 * Paper: M. Hu, N. Alger, R. Nammour, O. Ghattas, "Accelerating seismic
 * inversion and uncertainty quantification with efficient high-rank Hessian
 * approximations" (arXiv 2507.10804).
 *
 *  - forward map f(m), data d = f(m) + noise ........... section 2, eq. (pde), eq. (data)
 *  - Born operator F = grad f, migration F* ............ section 2.1, eq. (grad)
 *  - misfit Phi = 1/2 |f(m) - d|^2_{Gamma^-1}, grad .... section 2.1, eq. (grad) (no prior term)
 *  - H_d v = F* Gamma^-1 F v, two wave solves per source
 *    (plus the forward field) .......................... section 3, opening of the section
 *
 * Discretisation (the paper fixes only the continuous equation
 * (1/m^2) u_tt - lap u = s(t) delta(x - x_s) with m the wave speed):
 *  - padded grid NZ = nz + 2 nb rows by NX = nx + 2 nb columns, spacing h,
 *    zero (Dirichlet) values outside it;
 *  - 8th-order central Laplacian, 2nd-order leapfrog in time;
 *  - absorbing sponge of nb cells on all four sides: (1/m^2)(u_tt + q u_t) - lap u = f,
 *    q = q_max (d/(nb h))^2 with d the distance into the sponge,
 *    q_max = 3 vmax ln(1/R) / (2 nb h), q = max over the two axes in corners;
 *  - Ricker source s(t) = (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2)
 *    injected as s(n dt)/h^2 at one node per shot;
 *  - receivers sample u^{n+1} at their node after step n (d[n][r], n < nt);
 *  - the model on the sponge is the interior model replicated from the
 *    nearest edge cell (operator E); gradients and Hessian outputs are folded
 *    back onto the interior by E^T;
 *  - Gamma_noise = sigma^2 I.
 *
 * Conventions for every call below:
 *  - Return value: HV_OK (0) or an HV_E* code; hv_last_error() returns a
 *    thread-local message for the last failure of the calling thread.
 *  - All array arguments of the compute calls are DEVICE pointers owned by the
 *    caller, on the device that was current at hv_create; the library keeps
 *    no reference to them after the call is enqueued.
 *  - Models, vectors, gradients and Hessian outputs are interior fields
 *    [nz][nx] (x fastest), float32 unless stated.  Data are [ns][nt][nr]
 *    float32 (Born data: [k][ns][nt][nr]).
 *  - Every compute call is asynchronous on `stream` (a cudaStream_t passed as
 *    void*; NULL is the legacy default stream).  Outputs are valid once the
 *    stream reaches the point of the call.
 *  - Scratch memory: the caller passes `ws`, a device buffer of at least the
 *    size hv_workspace_size() reports for the same operation, k and budget,
 *    aligned to 256 bytes.  Calls enqueued on different streams must use
 *    different workspaces.  The library never allocates device memory inside
 *    a compute call.
 *  - Checkpoint budget `ckpt`: number of wavefield snapshots (each a pair of
 *    time levels) kept per shot for the adjoint sweep; HV_CKPT_ALL keeps every
 *    time level instead (no recomputation).  With 1 <= ckpt < nt - 1 the
 *    forward field is recomputed from snapshots by an optimal binomial
 *    schedule; results are bitwise identical to HV_CKPT_ALL.
 */
#ifndef HV_H
#define HV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define HV_OK 0
#define HV_EINVAL 1     /* an argument failed validation (message says which)      */
#define HV_ENOMEM 2     /* a workspace or host allocation was too small / failed   */
#define HV_ECUDA 3      /* a CUDA runtime call failed (message carries its string) */
#define HV_ETIMEOUT 4   /* a bounded device or host wait ran out                   */
#define HV_EBUSY 5      /* the resource is in use (server queue full, ...)         */
#define HV_ENOTSUP 6    /* the operation is declared but not provided              */

#define HV_CKPT_ALL (-1)

/* Operations for hv_workspace_size. */
#define HV_OP_FWD 0         /* hv_fwd_model                      */
#define HV_OP_BORN 1        /* hv_born                           */
#define HV_OP_MIGRATE 2     /* hv_migrate                        */
#define HV_OP_GRAD 3        /* hv_misfit_grad                    */
#define HV_OP_HV 4          /* hv_hessian_apply(_f64out)         */
#define HV_OP_WAVEFIELD 5   /* hv_wavefield                      */
#define HV_OP_MISFIT 6      /* hv_misfit                         */
#define HV_OP_MISFITS 7     /* hv_misfit_models (k = models)     */

/* Interior grid and sponge.  h in metres. */
typedef struct hv_grid {
    int nz, nx;     /* interior rows (depth) and columns, >= 1            */
    int nb;         /* sponge width in cells on every side, >= 0          */
    double h;       /* grid spacing [m], > 0                              */
} hv_grid;

/* Acquisition and time axis.  Node indices are interior (iz, ix), int32,
 * host pointers read only during hv_create. */
typedef struct hv_acq {
    int ns;                 /* shots, >= 1                                      */
    const int *src_iz;      /* [ns] source node row, 0 <= iz < nz               */
    const int *src_ix;      /* [ns] source node column, 0 <= ix < nx            */
    int nr;                 /* receivers per shot, >= 1                         */
    const int *rec_iz;      /* [ns*nr] receiver rows (distinct nodes per shot)  */
    const int *rec_ix;      /* [ns*nr] receiver columns                         */
    int nt;                 /* time steps, >= 1                                 */
    double dt;              /* time step [s]; stable for vmax dt / h < 0.5547   */
    double f0;              /* Ricker peak frequency [Hz]                       */
    double t0;              /* Ricker delay [s]                                 */
    double vmax;            /* velocity that sizes the sponge rate [m/s], > 0   */
    double R;               /* sponge target reflection coefficient, (0, 1)     */
    double sigma;           /* noise standard deviation, > 0                    */
} hv_acq;

typedef struct hv_handle hv_handle;

/* Thread-local description of the calling thread's last failure ("" if none). */
const char *hv_last_error(void);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int hv_version(void);

/* Validate the problem and create a handle on the current device.  Copies
 * the acquisition arrays; precomputes the source wavelet, the sponge profiles
 * and the receiver tables on the device (small allocations owned by the
 * handle).  Rejects: non-positive sizes, out-of-range or duplicate receiver
 * nodes, out-of-range source nodes, non-positive h/dt/vmax/sigma, R outside
 * (0, 1).  Blocks until the set-up kernels finish. */
int hv_create(const hv_grid *grid, const hv_acq *acq, hv_handle **out);

/* Release the handle and its device memory (synchronises the device). */
int hv_destroy(hv_handle *h);

/* Bytes of workspace needed by operation `op` (HV_OP_*) with k vectors and
 * checkpoint budget ckpt (ignored by HV_OP_FWD/BORN/WAVEFIELD). */
int hv_workspace_size(const hv_handle *h, int op, int k, int ckpt, size_t *bytes);

/* Forward map f(m): d[ns][nt][nr] = receiver samples of u.  m: [nz][nx] wave
 * speed [m/s], every value > 0. */
int hv_fwd_model(hv_handle *h, const float *m, float *d, void *ws, size_t ws_bytes, void *stream);

/* Forward wavefields at n_out selected steps: out[i][s][NZ][NX] = u^{steps[i]+1}
 * of shot s on the padded grid (steps: HOST array, ascending, each in [0, nt)). */
int hv_wavefield(hv_handle *h, const float *m, int n_out, const int *steps, float *out,
                 void *ws, size_t ws_bytes, void *stream);

/* Born map F dm for k perturbations: dd[k][ns][nt][nr]; dm: [k][nz][nx]. */
int hv_born(hv_handle *h, const float *m, const float *dm, int k, float *dd,
            void *ws, size_t ws_bytes, void *stream);

/* Migration F^T r for data r[ns][nt][nr]: g[nz][nx]. */
int hv_migrate(hv_handle *h, const float *m, const float *r, float *g, int ckpt,
               void *ws, size_t ws_bytes, void *stream);

/* Misfit and gradient: phi (DEVICE double scalar) = (1/(2 sigma^2)) sum (f(m) - d_obs)^2,
 * grad[nz][nx] = F^T (f(m) - d_obs) / sigma^2.  Reductions in FP64, fixed order. */
int hv_misfit_grad(hv_handle *h, const float *m, const float *d_obs, double *phi, float *grad,
                   int ckpt, void *ws, size_t ws_bytes, void *stream);

/* Misfit only: phi (DEVICE double) = (1/(2 sigma^2)) sum (f(m) - d_obs)^2, the
 * negative log-likelihood of section 2 (one forward solve per shot; what a
 * gpCN proposal needs, paper section 2.3). */
int hv_misfit(hv_handle *h, const float *m, const float *d_obs, double *phi, void *ws, size_t ws_bytes, void *stream);

/* Misfits at k different models in one forward sweep: phi[i] = (1/(2 sigma^2))
 * sum (f(m[i]) - d_obs[i])^2 for i < k, the negative log-likelihoods that k
 * gpCN chains (section 2.3) need for their k proposals.  m, d_obs and phi are
 * HOST arrays of k DEVICE pointers (m[i]: [nz][nx] velocity; d_obs[i]:
 * [ns][nt][nr]; phi[i]: one double), read during the call; the models' k x ns
 * forward fields advance together, one launch per time step.  Every phi[i]
 * is bitwise what hv_misfit gives for m[i] and d_obs[i] alone.  Workspace:
 * hv_workspace_size(h, HV_OP_MISFITS, k, 0, &bytes); 1 <= k <= 65535.
 * Errors: HV_EINVAL for a null array or entry or k out of range, HV_ENOMEM
 * for a short workspace (nothing is launched then). */
int hv_misfit_models(hv_handle *h, int k, const float *const *m, const float *const *d_obs,
                     double *const *phi, void *ws, size_t ws_bytes, void *stream);

/* Misfit engine: misfit requests (as hv_misfit) that join a running forward
 * sweep at its next time step instead of waiting for it to end.  The engine
 * has `slots` slots; each holds one model with its own step counter.
 * hv_engine_join enqueues the model's preparation and the zeroing of its
 * fields on `stream` and takes a free slot (HV_EBUSY when none is free);
 * every hv_engine_tick enqueues one launch that advances every occupied slot
 * by one time step (slot i at step ticks-since-its-join); after a slot's
 * nt-th step the same tick reduces its misfit into the slot's phi (bitwise
 * what hv_misfit gives for that model and data), frees the slot and reports
 * it in done[0 .. *n_done) (done: HOST array of `slots` ints).  A tick with
 * no occupied slot launches nothing.  m, d_obs, phi: DEVICE pointers that
 * must stay valid until the slot is reported done.  All calls of one engine
 * go to one stream, from one thread.  Device memory: the caller's workspace
 * of hv_engine_workspace_size bytes (256-byte aligned), owned by the engine
 * until hv_engine_destroy (which neither synchronises nor frees it). */
typedef struct hv_engine hv_engine;
int hv_engine_workspace_size(const hv_handle *h, int slots, size_t *bytes);
int hv_engine_create(hv_handle *h, int slots, void *ws, size_t ws_bytes, hv_engine **out);
int hv_engine_join(hv_engine *e, const float *m, const float *d_obs, double *phi, void *stream, int *slot);
int hv_engine_tick(hv_engine *e, void *stream, int *done, int *n_done);
int hv_engine_active(const hv_engine *e, int *active);
int hv_engine_destroy(hv_engine *e);

/* The engine's device-resident request loop: requests are posted into device
 * memory and a loop running on the GPU admits them at its next time step,
 * advances every occupied slot and reports each finished misfit to the host,
 * with no host launch per step.  The loop is one CUDA graph launch: a
 * conditional while node whose body is one iteration (the forward step of the
 * occupied slots, admission and the loop's conditions, the misfits of the
 * slots that took their last step).
 *  - hv_engine_post takes a free slot (HV_EBUSY when none is), enqueues on
 *    `stream` the model's preparation, the zeroing of the slot's fields and
 *    the post itself (the request's data and phi pointers and a sequence
 *    number written to device memory after the preparation), and returns the
 *    slot.  Any stream may be used, also while the loop runs on another.
 *  - hv_engine_serve launches the loop on `stream` unless it is running.  One
 *    launch ends after 2000 iterations with no occupied slot and no waiting
 *    request, after 2^20 iterations, or at the end of the iteration in which
 *    hv_engine_stop's request is seen; occupied slots keep their state across
 *    launches.  A post that lands as a launch ends waits for the next
 *    hv_engine_serve: call it again when hv_engine_poll reports the loop not
 *    running while posted requests are not done.
 *  - hv_engine_poll reports, in done[0 .. *n_done) (HOST array of `slots`
 *    ints), the slots whose misfit has been written to its phi (bitwise what
 *    hv_misfit gives) since the last poll, frees them, and sets *running
 *    (may be NULL) to whether the loop is running.
 * The first post switches the engine to this mode: hv_engine_join and
 * hv_engine_tick are refused from then on (and posting while joined slots
 * run is refused).  hv_engine_destroy ends a running loop (a stop request and
 * a wait for its current iteration) before it frees the engine.  Host memory:
 * a small pinned, mapped mailbox per engine (allocated at the first post). */
int hv_engine_post(hv_engine *e, const float *m, const float *d_obs, double *phi, void *stream, int *slot);
int hv_engine_serve(hv_engine *e, void *stream);
int hv_engine_poll(hv_engine *e, int *done, int *n_done, int *running);
int hv_engine_stop(hv_engine *e);

/* Gauss-Newton Hessian apply: Hv[j] = F^T F v[j] / sigma^2 for j < k; v and Hv
 * are [k][nz][nx].  Images accumulate in FP64 and are summed over shots in a
 * fixed order, so results do not depend on batching. */
int hv_hessian_apply(hv_handle *h, const float *m, const float *v, int k, float *Hv, int ckpt,
                     void *ws, size_t ws_bytes, void *stream);

/* As hv_hessian_apply with a double output Hv[k][nz][nx]. */
int hv_hessian_apply_f64out(hv_handle *h, const float *m, const float *v, int k, double *Hv, int ckpt,
                            void *ws, size_t ws_bytes, void *stream);

/* Merged calls on one model: Hessian applies, misfit gradients and misfits
 * at the same m (the quantities sections 2.1-2.3 ask for: an optimiser's
 * gradient and Gauss-Newton products, an MCMC chain's misfit) share one
 * forward sweep.  The H v vectors of all entries and one vector per gradient
 * run as one batch of Born vectors; a gradient's vector is zero (its Born
 * field stays zero) and its adjoint source is the residual f(m) - d_obs
 * instead of Born data; misfits are reduced from the forward data.  Every
 * output is bitwise what the separate call gives (hv_hessian_apply per entry,
 * hv_misfit_grad, hv_misfit).
 *  - hv_batch: HOST arrays of DEVICE pointers.  Entry i of n_hv: v[i]
 *    [k[i]][nz][nx] -> Hv[i] [k[i]][nz][nx]; gradient g of n_grad:
 *    grad_dobs[g] [ns][nt][nr] -> grad_phi[g] (device double), grad[g]
 *    [nz][nx]; misfit q of n_misfit: misfit_dobs[q] -> misfit_phi[q].  At
 *    least one entry in all; sum k[i] + n_grad <= 65535.
 *  - hv_batch_workspace_size: bytes of `ws` hv_apply_batch needs for this
 *    batch shape and checkpoint budget.
 *  - hv_apply_batch: enqueues the batch on `stream` (no CUDA graph).  The
 *    library's request server merges queued requests on one problem and
 *    model into such calls. */
typedef struct hv_batch {
    int n_hv;
    const float *const *v;
    const int *k;
    float *const *Hv;
    int n_grad;
    const float *const *grad_dobs;
    double *const *grad_phi;
    float *const *grad;
    int n_misfit;
    const float *const *misfit_dobs;
    double *const *misfit_phi;
} hv_batch;
int hv_batch_workspace_size(const hv_handle *h, const hv_batch *b, int ckpt, size_t *bytes);
int hv_apply_batch(hv_handle *h, const float *m, const hv_batch *b, int ckpt, void *ws, size_t ws_bytes, void *stream);

/* The Hessian apply split over sources (section 3: H_d v is a sum over
 * sources of two wave solves each; eq. (grad) sums the imaging over
 * sources), for one process per GPU, each owning a block of shots:
 *  - hv_hessian_apply_partial: the extended image of this handle's shots,
 *    before the fold E^T: ext[k][NZ][NX] (DEVICE doubles, padded grid NZ =
 *    nz + 2 nb, NX = nx + 2 nb, x fastest) = G^T S^-T P^T Gamma^-1 P S^-1 G E v
 *    restricted to the handle's shots, i.e. 2 / (m_ext h^2) sum_s sum_n
 *    lam_s^n (L_h u_s^n + s_n) with the shot groups summed in FP64.  Same
 *    workspace (HV_OP_HV), arguments and checkpointing as hv_hessian_apply.
 *  - hv_image_fold: out[k][nz][nx] = E^T ext (the sponge nodes added onto
 *    their nearest interior nodes, FP64 sums), written as float (out) and/or
 *    double (out64); either may be NULL, not both.  Any handle of the same
 *    grid may fold.
 * The ranks' extended images summed in a fixed rank order, then folded once,
 * give H_d v of all shots (to FP64 rounding of the order of the sums). */
int hv_hessian_apply_partial(hv_handle *h, const float *m, const float *v, int k, double *ext, int ckpt,
                             void *ws, size_t ws_bytes, void *stream);
int hv_image_fold(hv_handle *h, const double *ext, int k, float *out, double *out64, void *stream);

/* Allocation-free Gauss-Newton Hessian apply.  The paper has no counterpart;
 * this entry point exists for callers that cannot allocate device memory
 * where they call it (an application that owns every byte of device memory
 * through its own pool, a real-time loop that must not stall in an
 * allocator, or code that cannot size and pass a workspace).  It takes the
 * problem description directly (no handle) and computes what
 * hv_hessian_apply computes, with the same kernels, but keeps every table
 * and scratch field in one fixed device array of HV_STATIC_SCRATCH_BYTES
 * inside the library, which each GPU that loads the library holds until the
 * process exits.  It calls no cudaMalloc/cudaFree and no allocating library
 * routine.
 *  - m, v, Hv: DEVICE pointers as for hv_hessian_apply; grid/acq: host
 *    structs as for hv_create (validated the same way).
 *  - Problems whose tables plus workspace exceed the array are rejected with
 *    HV_ENOMEM and a message giving the bytes needed (64 MiB holds, e.g., a
 *    104 x 104 padded grid, 1 shot, 600 steps, k = 1, with every time level
 *    stored).
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current.
 *  - Never call it while `stream` is being captured into a CUDA graph: it
 *    copies its tables from host memory that is freed when it returns, so it
 *    returns HV_EINVAL under capture.
 *  - Every call shares the one array and overwrites the previous call's
 *    contents (whatever must start at zero is cleared on each call): calls
 *    that may overlap on the GPU (different streams, different host threads
 *    on the same device) race and must be serialised by the caller.
 *  - It runs tile configuration 0 for every kernel kind and the default
 *    (programmatic dependent launch) ordering, so its results are bitwise
 *    those of hv_hessian_apply with the same settings (and of any tiles).
 *  - Asynchronous on `stream` like the other compute calls.
 *  - hv_static_status reports a bounded device wait that ran out in any
 *    call since it was last read: it synchronises the device, writes HV_OK
 *    or HV_ETIMEOUT (the outputs of those calls are then invalid) and clears
 *    the word, which sits at the start of the array. */
#define HV_STATIC_SCRATCH_BYTES (64u * 1024u * 1024u)
int hv_hessian_apply_static(const hv_grid *grid, const hv_acq *acq, const float *m, const float *v, int k,
                            float *Hv, int ckpt, void *stream);
int hv_static_status(int *device_status);

/* Device status of the handle's kernels since the last call of hv_status:
 * HV_OK, or HV_ETIMEOUT if a bounded on-device wait (for a bulk tile copy, or
 * in the dataflow launch mode for the neighbouring tiles of an earlier step)
 * ran out and the kernel returned early (the outputs of the calls since the
 * last hv_status are then invalid).  Synchronises the device, then clears the
 * status. */
int hv_status(hv_handle *h, int *device_status);

/* Limit of every bounded wait inside the handle's stencil kernels, in seconds
 * (default 2; 1e-4 <= seconds <= 60, else HV_EINVAL).  A wait that runs out
 * sets the device status (hv_status) and the CTA returns without leaving a
 * copy in flight.  Applies to calls enqueued afterwards. */
int hv_set_wait_limit(hv_handle *h, double seconds);

/* Testing the timeout path without a fault: the next stencil step that the
 * dataflow launch mode orders by tile counters (HV_LAUNCH_DATAFLOW, see
 * hv_set_launch_mode) waits for a count that no step reaches.  Its CTAs wait
 * out the limit before they issue any copy, the first one sets HV_ETIMEOUT,
 * and every later wait of the call gives up at once on seeing the status;
 * the call's outputs are invalid and hv_status reports HV_ETIMEOUT.  One-shot:
 * cleared when a step takes it.  No effect in the other launch modes. */
int hv_inject_wait_timeout(hv_handle *h);

/* Hessian approximations built from batched H v.
 *
 * Point spread functions (section 3.2) in the PsiDO row form of section 3.5:
 * a PSF is H_d applied to a delta at a sample point x_k, read around x_k,
 *   p_k(d) = (H_d e_{x_k})[x_k + d],
 * and H_d ~ (2 pi)^2 sum_k D_{w_k} F^-1 D_{conj(p_k^)} F, i.e. on the grid
 *   (H~ v)(x) = sum_k w_k(x) sum_{|d|_inf <= R} p_k(d) v(x + d)   (v = 0 off the grid).
 * Sample points: the lattice of spacing S = spacing_cells on the interior grid
 * starting at (S/2, S/2) (integer division), all points with iz < nz, ix < nx,
 * point (a, b) numbered k = a * nb + b.  n_batches = B * B (B = 1..8): batch
 * (a mod B) * B + (b mod B) holds the sum of unit impulses at its points, and
 * one hv_hessian_apply with k = B * B vectors yields every PSF.  Window radius
 * R = (B S - 1) / 2 (windows of one batch never overlap; at most 40); PSF
 * values whose x_k + d leaves the grid are zero.  Weights w_k: bilinear hat
 * functions on the lattice (a partition of unity), constant beyond the
 * outermost points.  The paper leaves the window, the weights and the batch
 * layout open; these are this library's choices.
 *
 *  - hv_approx_psf_workspace_size: bytes of `ws` hv_approx_build_psf needs for
 *    n_batches and checkpoint budget ckpt (as in hv_hessian_apply).
 *  - hv_approx_build_psf: builds the approximation at model m ([nz][nx]
 *    device) on `stream`; *out receives a new object that owns its device
 *    memory (PSFs [r][2R+1][2R+1] floats).  HV_EINVAL on a bad argument
 *    (spacing < 1, n_batches not a square of 1..8, R > 40, first sample point
 *    off the grid), HV_ENOMEM if ws is too small.
 *  - hv_approx_apply: out[k][nz][nx] = H~ v[k][nz][nx] (device, k >= 1) on
 *    `stream`, mode HV_APPROX_H.  The other modes return HV_ENOTSUP for a PSF
 *    approximation; the square-root forms below and the LR approximation
 *    provide them.
 *  - hv_approx_info: info[11] = {kind (0 = PSF), r, R, na, nb, S, B, cz0,
 *    cx0, nz, nx}.
 *  - hv_approx_psfs: copies the PSFs [r][2R+1][2R+1] into a device buffer.
 *  - hv_approx_destroy: frees the object (NULL is allowed).
 *
 * Pseudo-differential operator probing (section 3.4, appendix A), applied in
 * the low-rank-symbol form of section 3.3, eq. (lr-psido):
 *   H~ v = Re sum_k D_{a_k} F^-1 D_{b_k} F v,  F the 2D DFT of the nz x nx grid.
 * Sample frequencies xi_k = rho0 (cos theta_k, sin theta_k) [rad/m], theta_k =
 * 2 pi k / r (r even, 2..32; the paper uses 8), each snapped to the nearest
 * DFT frequency (signed index rounded half to even), so the probe
 * v_p = sum_k exp(i x . xi_k) is real.  One hv_hessian_apply to v_p; the
 * symbol column a_k(x) = s(x, xi_k) is the part of the spectrum of H v_p
 * inside the disc of radius rho0 sin(pi / r) around xi_k, moved to the origin
 * and transformed back; b_k(xi) = (|xi| / |xi_k|) w_k(theta) with w_k the
 * trigonometric interpolation basis of the r nominal angles (linear in the
 * magnitude, Fourier over the angle).  rho0 + rho0 sin(pi / r) must stay below
 * the Nyquist frequency pi / h; the paper's choice is rho0 ~ 2 pi f_max / c_max.
 *  - hv_approx_pdo_workspace_size: bytes of `ws` the build needs for budget ckpt.
 *  - hv_approx_build_pdo: builds it at model m on `stream` (one H v, cuFFT
 *    transforms); the object owns its columns, weights, FFT plans and scratch.
 *    HV_EINVAL on a bad r or rho0, HV_ENOMEM if ws is too small.
 *  - hv_approx_apply on a PDO object: one forward and r inverse transforms per
 *    vector; applies of one object from different streams run one after
 *    another (they share its FFT scratch).
 *  - hv_approx_pdo_symbol: copies a_k and/or b_k ([r][nz][nx] complex each,
 *    interleaved re/im floats; b in DFT order) to device buffers.
 *  - hv_approx_info on a PDO object: {1, r, spd, 0, 0, 0, 0, 0, 0, nz, nx}
 *    (spd = 1 for the square-root form below).
 *
 * PSF+ (section 3.6): hv_approx_build_psfplus(psf, pdo, tol, out, stream)
 * combines a PSF and a PDO approximation of the same grid and device into a
 * low-rank symbol A B: the PSF symbol rows s(x_k, xi) = sum_d p_k(d) e^{i xi.d}
 * (conjugated DFTs of the PSFs at the origin), their SVD through the Gram
 * matrix (FP64, Hermitian Jacobi on the host) giving the
 * basis B of the r' <= 32 singular directions with sigma >= tol sigma_1 and
 * A0 = W U Sigma (W the PSF lattice weights), then A = (S_c B_c^H + alpha A0)
 * (B_c B_c^H + alpha I)^-1 with S_c the PDO columns, B_c the basis at the PDO
 * sample frequencies and alpha = ||B_c||_F^2 / ||B||_F^2.  At most 256 PSFs;
 * synchronous on `stream` (waits for the PDO object's build).  The result is
 * applied with hv_approx_apply (kind 2; hv_approx_pdo_symbol returns A and B);
 * hv_approx_info gives {2, r', spd, 0, ..., nz, nx}.  HV_EINVAL for mismatched
 * inputs or tol outside (0, 1).
 *
 * Low-rank approximation (section 3.1) with the Matern prior of section 2.1,
 * R = Gamma_pr^-1 = A^2, A = delta I - gamma Lap_h (Lap_h the 5-point
 * Laplacian with homogeneous Neumann conditions, mirror ghost cells):
 *  - hv_prior_apply: out = A v (op 0), A^-1 v (1), R v (2) or R^-1 v (3) for
 *    k fields [k][nz][nx] on the device (A^-1 by the 2D DCT-II that
 *    diagonalises A, computed with one real 2D DFT of the reordered field).
 *    Builds and frees its tables on every call; synchronous on `stream`.
 *  - hv_approx_lr_workspace_size: bytes of `ws` hv_approx_build_lr needs for
 *    k test vectors and budget ckpt.
 *  - hv_approx_build_lr: the `rank` leading eigenpairs of H_d v = lambda R v
 *    (V^T R V = I) at model m by the randomized double pass with the caller's
 *    test matrix omega [k][nz][nx] (device; normally standard Gaussian, drawn
 *    by the caller): Y = R^-1 H_d omega, Q its R-orthonormal basis (the
 *    eigen-decomposition of the R-Gram matrix in FP64, dropping directions
 *    below 1e-12 of the largest, twice), T = Q^T H_d Q, V = Q S[:, :rank].
 *    Two batched H v (k vectors each).  1 <= rank <= k <= 256; HV_EINVAL if
 *    omega spans fewer than `rank` directions.  Synchronous on `stream`.
 *  - hv_approx_apply on an LR object: HV_APPROX_H gives R V Lambda V^T R v
 *    (the approximation of H_d, so that H~_d + R = R + R V Lambda V^T R);
 *    HV_APPROX_INVSQRT gives (I - V S V^T R) A^-1 v with S = I - (Lambda +
 *    I)^-1/2, which maps N(0, I) to N(0, (H~_d + R)^-1), the Laplace
 *    approximation of the posterior; HV_APPROX_SQRT returns HV_ENOTSUP.
 *  - hv_approx_lr_eigs: lambda[rank] (host, descending) and/or V (device
 *    [rank][nz][nx]).  hv_approx_info gives {3, rank, 0, ..., nz, nx}.
 *
 * Square-root (SPD) forms (section 3.7): the square root of H_d is
 * approximated by the same procedure with the pointwise square root
 * sqrt(max(Re s, 0)) of the computed symbol columns (PDO) or rows and columns
 * (PSF+), giving a factor B = Re sum_k D_{a_k} F^-1 D_{b_k} F, and H~_d = B B^T
 * is symmetric positive semi-definite.
 *  - hv_approx_sqrt_pdo: from a PDO approximation of H_d (kind 1, not itself a
 *    square root), a new object with a_k = sqrt(max(Re a_k, 0)) and weights
 *    of radial order 1/2: b_k(xi) = (|xi| / |xi_k|)^(1/2) w_k(theta) (the
 *    square root of the order-1 symbol is of order 1/2).
 *  - hv_approx_build_psfplus_sqrt: as hv_approx_build_psfplus with the PSF
 *    symbol rows and the PDO columns replaced by sqrt(max(Re s, 0)) before the
 *    SVD and the refinement.
 *  - hv_approx_apply on such an object (hv_approx_info()[2] == 1):
 *    HV_APPROX_H gives B B^T v, HV_APPROX_SQRT B v, HV_APPROX_SQRT_T
 *    B^T v = Re F^-1 sum_k conj(b_k) F (conj(a_k) v); HV_APPROX_INVSQRT returns
 *    HV_ENOTSUP (posterior samples need a solve with B B^T + R: see
 *    hv_posterior_sample).  On a PDO or PSF+ approximation of H_d itself only
 *    HV_APPROX_H (B v) is provided.
 *
 * hv_set_fused_transforms(enable): for PDO, PSF+ and quadratic-model objects
 * created afterwards in this process (default on), the applies of the
 * low-rank-symbol form run the library's own 2D DFTs with the symbol products
 * fused into them where nz and nx are powers of two from 16 to 512 (the r-term
 * spectra are written once and read once per vector); other grids, and
 * objects created with the setting off, use cuFFT transforms and separate
 * product kernels.  The two agree to FP32 rounding (about 1e-6 relative), not
 * bitwise.  Returns HV_OK.
 *
 * hv_util_hermitian_eig: eigenvalues (descending) into w[n] and eigenvectors
 * (columns, row-major, interleaved re/im doubles) into V[n*n*2] of the
 * Hermitian matrix A[n*n*2] (interleaved re/im, row-major), n <= 4096: the host
 * routine the PSF+ build uses.  HV_EINVAL if A is not Hermitian. */
typedef struct hv_approx hv_approx;
#define HV_APPROX_H 0           /* apply the approximation of H_d            */
#define HV_APPROX_SQRT 1        /* apply its square-root factor B            */
#define HV_APPROX_INVSQRT 2     /* apply the posterior sampling factor       */
#define HV_APPROX_SQRT_T 3      /* apply the transpose B^T of the factor     */
int hv_approx_psf_workspace_size(hv_handle *h, int n_batches, int ckpt, size_t *bytes);
int hv_approx_build_psf(hv_handle *h, const float *m, int spacing_cells, int n_batches, int ckpt, hv_approx **out,
                        void *ws, size_t ws_bytes, void *stream);
int hv_approx_pdo_workspace_size(hv_handle *h, int ckpt, size_t *bytes);
int hv_approx_build_pdo(hv_handle *h, const float *m, double rho0, int r, int ckpt, hv_approx **out, void *ws,
                        size_t ws_bytes, void *stream);
int hv_approx_pdo_symbol(const hv_approx *a, float *cols, float *weights, void *stream);
int hv_approx_build_psfplus(const hv_approx *psf, const hv_approx *pdo, double tol, hv_approx **out, void *stream);
int hv_approx_sqrt_pdo(const hv_approx *pdo, hv_approx **out, void *stream);
int hv_approx_build_psfplus_sqrt(const hv_approx *psf, const hv_approx *pdo, double tol, hv_approx **out,
                                 void *stream);
int hv_util_hermitian_eig(int n, const double *A, double *w, double *V);
int hv_prior_apply(int nz, int nx, double h, double delta, double gamma, const float *v, int k, float *out, int op,
                   void *stream);
int hv_approx_lr_workspace_size(hv_handle *h, int k, int ckpt, size_t *bytes);
int hv_approx_build_lr(hv_handle *h, const float *m, double delta, double gamma, int rank, const float *omega, int k,
                       int ckpt, hv_approx **out, void *ws, size_t ws_bytes, void *stream);
int hv_approx_lr_eigs(const hv_approx *a, double *lambda, float *V, void *stream);
int hv_approx_apply(const hv_approx *a, const float *v, int k, float *out, int mode, void *stream);
int hv_set_fused_transforms(int enable);
int hv_approx_info(const hv_approx *a, int *info);
int hv_approx_psfs(const hv_approx *a, float *psf, void *stream);
int hv_approx_destroy(hv_approx *a);

/* Operators given by the caller.  hv_operator describes a linear operator on
 * nz x nx fields with spacing h: apply(ctx, v, k, out, stream) writes
 * out[k][nz][nx] = Op v[k][nz][nx] (device buffers, stream-ordered on
 * `stream`) and returns HV_OK or an HV_E* code.  The *_op builds construct the
 * approximations of such an operator exactly as the builds above do from
 * hv_hessian_apply (same arguments and results; the build's scratch is
 * allocated on the device and freed before return).  The operator is called
 * with k = n_batches (PSF), 1 (PDO) or k then at most k (LR) vectors. */
typedef int (*hv_op_fn)(void *ctx, const float *v, int k, float *out, void *stream);
typedef struct hv_operator {
    int nz, nx;
    double h;
    hv_op_fn apply;
    void *ctx;
} hv_operator;
int hv_approx_build_psf_op(const hv_operator *op, int spacing_cells, int n_batches, hv_approx **out, void *stream);
int hv_approx_build_pdo_op(const hv_operator *op, double rho0, int r, hv_approx **out, void *stream);
int hv_approx_build_lr_op(const hv_operator *op, double delta, double gamma, int rank, const float *omega, int k,
                          hv_approx **out, void *stream);

/* High-pass filter before the PSF and PDO approximations (sections 3.2 and
 * 3.7: the low-frequency part of H_d -- transmission, non-local PSFs, too low
 * for spectral separation -- is removed before approximating and left to the
 * low-rank correction).  The paper does not specify the filter; this library
 * uses the radial Gaussian high-pass on the periodic 2D DFT of the nz x nx
 * grid, F_hp v = Re F^-1 (phi(|xi|) F v), phi(rho) = 1 - exp(-rho^2 /
 * (2 rho_c^2)), xi = (2 pi k_z / (nz h), 2 pi k_x / (nx h)) for the signed DFT
 * indices, rho_c [rad/m] the cutoff, and applies it on both sides,
 * F_hp H_d F_hp, so the approximated operator stays symmetric.
 *  - hv_highpass_apply: out = F_hp v for k fields [k][nz][nx] (device; out
 *    may be v); builds and frees its transforms; synchronous on `stream`.
 *  - hv_set_highpass(h, rho_c): hv_approx_build_psf and hv_approx_build_pdo on
 *    this handle approximate F_hp H_d F_hp (rho_c > 0) or H_d (0, the default).
 *    The filtered builds allocate the filter's transforms and a scratch of
 *    n_batches (PSF) or 1 (PDO) fields, freed before they return.
 *  - hv_filtered_create(inner, rho_c, max_k, out): F_hp inner F_hp as an
 *    object that owns the transforms and a scratch of max_k fields;
 *    hv_filtered_operator fills an hv_operator that applies it (in chunks of
 *    max_k fields; applies on one object are ordered by an event, also across
 *    streams), for the *_op builds; hv_filtered_destroy frees it (the inner
 *    operator must outlive it). */
typedef struct hv_filtered hv_filtered;
int hv_highpass_apply(int nz, int nx, double h, double rho_c, const float *v, int k, float *out, void *stream);
int hv_set_highpass(hv_handle *h, double rho_c);
int hv_filtered_create(const hv_operator *inner, double rho_c, int max_k, hv_filtered **out);
int hv_filtered_operator(hv_filtered *f, hv_operator *op);
int hv_filtered_destroy(hv_filtered *f);

/* The ideal quadratic test model (section 4.1).  Misfit Hessian
 *   H_d = A A^T + V_r Lambda_r V_r^T                        (eq. (toy-hess))
 * with A the order-1/2 PsiDO of eq. (toy-symbol),
 *   s_A(x, xi) = w(x) P(|xi|) (0.1 + cos^2(arg xi + pi x / x_max)) / (0.1 + (z / z_max)^2),
 * applied through its rank-3 expansion (compound angle) a_1 = w / d(z),
 * a_2 = w cos(2 pi x / x_max) / d(z), a_3 = w sin(2 pi x / x_max) / d(z),
 * b_1 = 0.6 P, b_2 = cos(2 arg xi) P / 2, b_3 = -sin(2 arg xi) P / 2,
 * d(z) = 0.1 + (z / z_max)^2, as A v = Re sum_k a_k F^-1 b_k F v.  The paper
 * describes P, w and V_r qualitatively; this library takes
 * P(rho) = (rho / rho_c)^(1/2) exp(-(rho / rho_c)^4) (rho in rad/m), w = the
 * window W = the product of 1D tapers sin^2(pi/2 (i + 1/2) / L) over the L =
 * taper_cells cells next to each edge, z = iz h, x = ix h, z_max = nz h,
 * x_max = nx h, arg xi = atan2(xi_z, xi_x), and for p = 1 .. nlr/2 the unit-norm
 * modes e^{-8 z / z_max} cos(2 pi p x / x_max) and e^{-8 z / z_max} sin(...)
 * (orthonormal on the grid) with eigenvalues lam[nlr] >= 0.  The objective is
 * Phi(m) = Phi_d(W m) + 1/2 m^T R m = 1/2 (W m - m*)^T H_d (W m - m*) + 1/2 m^T R m
 * with the Matern prior R = (delta I - gamma Lap_h)^2 (as hv_prior_apply).
 *  - hv_quad_create: builds the tables (FP64 on the host, stored FP32) on the
 *    current device; HV_EINVAL for nz, nx < 4, h or rho_c <= 0, a taper wider
 *    than half the grid, an odd nlr, nlr / 2 >= nx / 2 or a negative lam.
 *  - hv_quad_apply: out = op v for k fields [k][nz][nx] (device):
 *    HV_QUAD_HD the misfit Hessian of Phi_d(W m), W (A A^T + V Lambda V^T) W;
 *    HV_QUAD_A, HV_QUAD_AT: A and A^T; HV_QUAD_HD_RAW: A A^T + V Lambda V^T.
 *  - hv_quad_objective: phi[k] (device doubles, FP64 sums) and, unless grad
 *    is NULL, grad[k][nz][nx] = W H_d (W m - m*) + R m for k states m (device);
 *    one_target != 0: mstar is one field for every state, else k fields.
 *  - hv_quad_tables: device copies of a, b ([3][nz][nx] complex each, b in
 *    DFT order), V [nlr][nz][nx] and W [nz][nx] (any may be NULL).
 *  - hv_quad_operator: fills *op with HV_QUAD_HD of q (valid while q lives).
 * Calls on one model from several streams run one after another (shared
 * scratch). */
typedef struct hv_quad hv_quad;
#define HV_QUAD_HD 0
#define HV_QUAD_A 1
#define HV_QUAD_AT 2
#define HV_QUAD_HD_RAW 3
int hv_quad_create(int nz, int nx, double h, double rho_c, int taper_cells, int nlr, const double *lam, double delta,
                   double gamma, hv_quad **out);
int hv_quad_apply(hv_quad *q, int op, const float *v, int k, float *out, void *stream);
int hv_quad_objective(hv_quad *q, const float *m, const float *mstar, int k, int one_target, double *phi, float *grad,
                      void *stream);
int hv_quad_tables(const hv_quad *q, float *a, float *b, float *V, float *W, void *stream);
int hv_quad_operator(hv_quad *q, hv_operator *op);
int hv_quad_destroy(hv_quad *q);

/* Laplace approximation of the posterior (sections 2.2, 3.1, 3.7).  A
 * posterior object holds H0 = H~_d + R, R = (delta I - gamma Lap_h)^2 the
 * Matern prior (as hv_prior_apply) and H~_d = B B^T the square-root
 * approximation `approx` (hv_approx_sqrt_pdo / hv_approx_build_psfplus_sqrt;
 * borrowed, it must outlive the posterior) or H~_d = 0 (approx NULL), plus an
 * optional low-rank correction, H~ = H0 + H0 V Lambda V^T H0.
 *  - hv_posterior_create: on the current device; HV_EINVAL for an approx that
 *    is not a square-root form or lives on another grid or device, or for
 *    max_k outside 1..256.  All device memory the object needs is allocated
 *    here, sized for calls of at most max_k fields (solves, applies, samples
 *    and correction test vectors; a correction's rank is at most max_k):
 *    the calls below allocate nothing and return HV_EINVAL for a larger k.
 *  - hv_posterior_solve: x = (Op + R)^-1 b for k fields, Op = the caller's
 *    operator or, if op is NULL, H~_d (so H0 x = b; the correction is not
 *    included).  Preconditioned conjugate gradients (preconditioner R^-1),
 *    FP32 vectors with FP64 dot products and step lengths, started from 0, until
 *    every ||r_j|| <= rtol ||b_j||; *iters = the iterations taken.  HV_ETIMEOUT
 *    after max_iter iterations (x then holds the last iterate).
 *  - hv_posterior_apply: out = H~ v.
 *  - hv_posterior_sample: zeta ~ N(0, H~^-1) from standard normals n1, n2
 *    [k][nz][nx] (caller-drawn, device): z = H0^-1 (A n1 + B n2) (by the solve
 *    above; for approx NULL z = A^-1 n1 exactly and n2 is unused), then
 *    zeta = (I - V S_r V^T H0) z, S_r = I - (Lambda + I)^-1/2.
 *  - hv_posterior_correct: the low-rank correction: the `rank` leading
 *    eigenpairs of (H_d - H~_d) v = lambda H0 v, V^T H0 V = I, H_d the operator
 *    hd, by the randomized double pass with the test matrix omega [k][nz][nx]
 *    (the section 3.1 method with H0 in place of R; the solves with H0 as
 *    above): Z = (H_d - H~_d) omega, Y = H0^-1 Z, Q = Y M from the
 *    eigen-decomposition of Y^T Z (= Y^T H0 Y; FP64, directions below 1e-12 of
 *    the largest dropped; twice), T = Q^T (H_d - H~_d) Q = S Lambda S^T,
 *    V = Q S[:, :rank].  1 <= rank <= k <= 256; HV_EINVAL if a kept eigenvalue
 *    is <= -1 (H~ would not be positive definite).  Replaces an earlier
 *    correction.  With approx NULL this is the low-rank approximation of
 *    section 3.1.
 *  - hv_posterior_eigs: lambda[rank] (host) and/or V [rank][nz][nx] (device).
 *  - hv_posterior_rank: the correction rank (0 without one; -1 for NULL).
 * Calls on one posterior are serialised (shared scratch); they synchronise
 * `stream` where a solve checks convergence.
 *
 * gpCN (section 2.3), c chains of n = nz * nx values each (device arrays):
 *  - hv_gpcn_propose: m_new[c] = m_map + sqrt(1 - beta^2)(m[c] - m_map) +
 *    beta zeta[c] and, unless d_new is NULL, d_new[c] = m_new[c] - m_map;
 *    0 < beta < 1.
 *  - hv_gpcn_accept (allocates nothing): Delta' = phi_new[c] - 1/2 d_new[c] . Hd_new[c] (FP64;
 *    Hd_new = H~ d_new, e.g. by hv_posterior_apply); the proposal is accepted
 *    iff log_u[c] < delta_cur[c] - Delta', u ~ U(0, 1) drawn by the caller,
 *    i.e. with probability min(1, exp(Delta(m_k) - Delta(m'))); then m[c] <-
 *    m_new[c] and delta_cur[c] <- Delta'.  accepted[c] = 1 or 0.  log_u = -inf
 *    accepts unconditionally (initialises delta_cur). */
typedef struct hv_posterior hv_posterior;
int hv_posterior_create(int nz, int nx, double h, double delta, double gamma, const hv_approx *approx, int max_k,
                        hv_posterior **out);
int hv_posterior_solve(hv_posterior *p, const hv_operator *op, const float *b, int k, float *x, double rtol,
                       int max_iter, int *iters, void *stream);
int hv_posterior_apply(hv_posterior *p, const float *v, int k, float *out, void *stream);
int hv_posterior_sample(hv_posterior *p, const float *n1, const float *n2, int k, float *zeta, double rtol,
                        int max_iter, int *iters, void *stream);
int hv_posterior_correct(hv_posterior *p, const hv_operator *hd, const float *omega, int k, int rank, double rtol,
                         int max_iter, void *stream);
int hv_posterior_eigs(const hv_posterior *p, double *lambda, float *V, void *stream);
int hv_posterior_rank(const hv_posterior *p);
int hv_posterior_destroy(hv_posterior *p);
int hv_gpcn_propose(int n, int c, const float *m, const float *m_map, const float *zeta, double beta, float *m_new,
                    float *d_new, void *stream);
int hv_gpcn_accept(int n, int c, const double *phi_new, const float *m_new, const float *d_new, const float *Hd_new,
                   const double *log_u, float *m, double *delta_cur, int *accepted, void *stream);

/* Output checks: *count (DEVICE unsigned long long) = the number of NaN and
 * +-Inf entries of the DEVICE array x[0, n) (a scan of any output, e.g. of an
 * H v whose model violates the time step's stability bound).  The paper has no
 * counterpart; it serves the checks of a run.  HV_EINVAL for a null count, or
 * a null x with n > 0. */
int hv_count_nonfinite(const float *x, size_t n, unsigned long long *count, void *stream);

/* Serving.  A server owns one device arena of hbm_budget bytes (allocated at
 * creation) and max_concurrent CUDA streams on the current device.  Requests
 * (H v, gradient, misfit, and the apply of a built Hessian approximation) on
 * any problems or approximations created on that device are queued
 * by hv_submit; a scheduler thread admits them in arrival order, letting a
 * later request pass one that is waiting for memory, whenever a stream is free
 * and the request's workspace fits in the arena, and runs each on its own
 * stream, so the work of requests that arrive while others run overlaps on
 * the GPU; queued requests on one problem and model are merged into one call
 * (hv_server_set_batching).  Results are bitwise the same as the direct calls.  Inputs and
 * outputs are caller-owned device buffers that must stay valid until the
 * request is done.  Request status: HV_REQ_QUEUED, HV_REQ_RUNNING, HV_OK when
 * done, or an HV_E* code. */
#define HV_REQ_HV 0
#define HV_REQ_GRAD 1
#define HV_REQ_MISFIT 2
#define HV_REQ_APPROX 3         /* hv_approx_apply(approx, v, k, out, approx_mode); needs no workspace */
#define HV_REQ_QUEUED 100
#define HV_REQ_RUNNING 101
typedef struct hv_server hv_server;
typedef struct hv_request {
    int kind;               /* HV_REQ_*                                           */
    hv_handle *problem;     /* problem the request runs on (unused by APPROX)     */
    const float *m;         /* model [nz][nx] (unused by APPROX)                  */
    const float *v;         /* HV, APPROX: vectors [k][nz][nx]                    */
    int k;                  /* HV, APPROX: number of vectors                      */
    const float *d_obs;     /* GRAD, MISFIT: observed data [ns][nt][nr]           */
    float *out;             /* HV, APPROX: [k][nz][nx]; GRAD: gradient [nz][nx]   */
    double *phi;            /* GRAD, MISFIT: device scalar                        */
    int ckpt;               /* HV, GRAD: checkpoint budget                        */
    const hv_approx *approx; /* APPROX: a built approximation                     */
    int approx_mode;        /* APPROX: HV_APPROX_* mode of hv_approx_apply         */
} hv_request;
typedef struct hv_request_info {
    int kind, status;
    double t_submit, t_start, t_done;   /* seconds since the server started        */
    size_t ws_bytes;                     /* arena bytes the request held (alone)     */
    int batch;                           /* requests that ran merged with it (1: alone); for a misfit
                                            that joined a lane, the lane's occupied slots at its join */
} hv_request_info;
int hv_server_create(size_t hbm_budget, int max_concurrent, hv_server **out);
/* Stops admitting, waits (bounded by timeout_s) for running requests, frees the arena. */
int hv_server_destroy(hv_server *s, double timeout_s);
int hv_submit(hv_server *s, const hv_request *r, unsigned long long *id);
int hv_poll(hv_server *s, unsigned long long id, int *status);
/* Waits until the request is done or failed; HV_ETIMEOUT after timeout_s. */
int hv_wait(hv_server *s, unsigned long long id, double timeout_s, int *status);
int hv_request_get_info(hv_server *s, unsigned long long id, hv_request_info *info);
/* Continuous batching: when the scheduler admits an H v, gradient or misfit
 * request, the queued requests on the same problem and model (H v and
 * gradients with the same checkpoint budget) join it, up to max_vectors Born
 * vectors in all (a gradient counts as one, a misfit as none), and run as one
 * hv_apply_batch on one stream and one arena block, if that fits; their
 * results are bitwise those of separate calls.  Queued applies of one
 * approximation in one mode likewise join into one hv_approx_apply of up to
 * max_vectors vectors (gathered into and scattered from an arena block of
 * 2 x vectors x nz x nx floats).  max_vectors < 2 turns merging off (each
 * request runs alone).  Default 64.  Applies to later admissions. */
int hv_server_set_batching(hv_server *s, int max_vectors);
/* Misfit lanes (continuous batching by time step): with slots > 0 (default
 * 64) a second scheduler thread gives each problem that receives misfit
 * requests a misfit engine (hv_engine_*) of up to `slots` slots, sized to at
 * most an eighth of the arena and to 16384 CTAs per step, on a stream of its
 * own.  A queued misfit request on that problem joins the engine at its next
 * time step, whatever step the other slots have reached, and is done after
 * its own nt steps (its phi bitwise hv_misfit's).  By default the thread
 * enqueues the engine's ticks (hv_engine_join / hv_engine_tick), keeping a few
 * in flight; with hv_server_set_engine_loop(s, 1), lanes created afterwards
 * are served by the engine's device-resident loop instead (requests posted
 * with hv_engine_post on a second stream of the lane, completions polled with
 * hv_engine_poll, the loop relaunched when it has ended while requests are
 * out).  A lane's arena block is released after it has been idle for 0.2 s.  When no lane fits in the
 * arena, misfits run as calls (merged as hv_server_set_batching says; queued
 * misfits at different models then run as one hv_misfit_models).  slots = 0
 * turns lanes off.  Applies to lanes created later. */
int hv_server_set_engine(hv_server *s, int slots);
int hv_server_set_engine_loop(hv_server *s, int enable);

/* Tile configurations.  The stencil kernels come in a small menu of
 * configurations: a tile shape (TX x TZ points per CTA), a copy-pipeline depth
 * (stages; stages - 1 shots in flight per CTA) and the number of 8-shot groups
 * one CTA walks.  The choice per kernel kind (cfg[0]: forward + Born step,
 * cfg[1]: forward-only step, cfg[2]: adjoint step) does not change any result
 * bit, only speed.
 *  - hv_tile_menu_size: number of menu entries.
 *  - hv_tile_menu: shape of menu entry `index` (HV_EINVAL past the end).
 *  - hv_tile_menu_info: info[5] = {TX, TZ, threads per CTA, stages, shot
 *    groups per CTA} of entry `index` (HV_EINVAL past the end or info NULL).
 *  - hv_autotune: times every entry for the three kernels on this handle's
 *    grid with k vectors, using `ws` (at least hv_workspace_size(HV_OP_HV, k,
 *    ckpt = 1) bytes; contents overwritten) on `stream`, the timed launches'
 *    fields rotating through the workspace's batches as in a sweep (each
 *    launch reads what the previous one wrote), keeps the fastest
 *    in the handle and writes the choice to chosen[3] and the per-launch
 *    times to ms[menu * 3] (either may be NULL).  Synchronous.  In the
 *    dataflow launch mode the three choices share one tile shape (the shape
 *    of least weighted time, weights 1 / 1.8 / 1 for the three kinds).  With
 *    step fusion on, the forward-only kind is timed as fused double steps
 *    (per step).
 *    Tune after setting the launch mode.
 *  - hv_set_tiles / hv_get_tiles: apply or read a choice (e.g. a cached one). */
int hv_tile_menu_size(void);
int hv_tile_menu(int index, int *TX, int *TZ);
int hv_tile_menu_info(int index, int *info);
int hv_autotune(hv_handle *h, int k, void *ws, size_t ws_bytes, void *stream, int *chosen, float *ms);
int hv_set_tiles(hv_handle *h, const int *cfg);
int hv_get_tiles(const hv_handle *h, int *cfg);

/* CUDA graphs.  When enabled (and profiling is off), the first
 * hv_hessian_apply with a given workspace pointer, size, k, budget and tile
 * choice records its whole launch sequence between model preparation and the
 * final fold as a CUDA graph (captured on a private stream); later calls with
 * the same key replay it with one launch.  The workspace contents are not
 * part of the key: they are rewritten by every call. */
int hv_set_graphs(hv_handle *h, int enable);

/* Launch modes of the stencil steps (every mode gives bitwise the same
 * results; graphs captured in one mode are not reused in another):
 *  - HV_LAUNCH_PLAIN: each step starts after the previous kernel completes.
 *  - HV_LAUNCH_PDL (default): programmatic dependent launch; a step's CTAs
 *    become resident and do their set-up while the previous step's last CTAs
 *    run, and touch no field before every earlier kernel has completed.
 *  - HV_LAUNCH_DATAFLOW: as PDL, and a CTA starts its tile as soon as the
 *    previous steps have finished that tile and its 8 neighbours (per-tile
 *    completion counters in the workspace, acquire/release at GPU scope,
 *    waits bounded by a deadline), so the tail of one step overlaps the start
 *    of the next.  Used when the three kernel kinds share a tile shape and
 *    nothing else was launched between two steps; otherwise the step falls
 *    back to the PDL wait.  On GB300 the release each CTA makes before it
 *    exits costs more than the overlap gains (about 3% slower than PDL on the
 *    384 x 1152 benchmark grid), hence not the default.
 * HV_EINVAL for another mode. */
/* Step fusion (off by default): the recomputation from snapshots runs two
 * forward steps per launch wherever two follow each other, reading u^n (with
 * an 8-cell halo) and u^{n-1} once (16 instead of 24 bytes per point for two
 * steps); results are bitwise those of single steps.  Not used in the
 * dataflow launch mode.  On GB300 the recomputed 4-cell ring (35-70% more
 * stencil work on the benchmark's tiles) and the extra barrier cost more than
 * the traffic saved: a fused launch takes about 120 us where two single steps
 * take 94 us on the 384 x 1152, 32-shot grid. */
int hv_set_step_fusion(hv_handle *h, int enable);
/* Shared-memory-resident H v.  With resident enabled, hv_hessian_apply with
 * every forward level stored (HV_CKPT_ALL, or a budget >= nt - 1) runs, on
 * grids whose padded field fits twice in one CTA's shared memory (NX a multiple
 * of 4; hv_resident_fits), three persistent kernels instead of one launch per
 * time step: the forward field of each shot (writing Q^n = Lh u^n + s_n for
 * every step), then the Born field of each (shot, vector) pair, then its
 * adjoint field, each held in shared memory for all nt steps.  Q^n, the Born
 * data and the adjoint fields are bitwise those of the tiled kernels; the image
 * is accumulated per pair over all steps in double-float arithmetic and summed
 * over shots in FP64, an order different from the tiled path's shot-group sums,
 * so results agree with it to rounding (about 1e-7 relative), not bitwise, and
 * are bitwise the same for any k and with or without graphs.  The workspace
 * size (hv_workspace_size) depends on the setting.  Off by default. */
int hv_set_resident(hv_handle *h, int enable);
int hv_resident_fits(const hv_handle *h);

/* Precision of the zero-lag imaging sum (section 3, the sum over time steps
 * and sources of the Hessian action and the gradient).
 *  - HV_IMAGE_PAIRS (default): per step, a CTA sums the products lam^n Q^n of
 *    the (at most 8) shots of its shot group in FP32 in shot order and adds
 *    that sum to the group's image held as a double-float pair (hi, lo) of
 *    FP32 values by an error-free TwoSum; the groups are summed in FP64.
 *  - HV_IMAGE_FP64: a check of the default's rounding: every shot's product,
 *    exact in FP64, is added to an FP64 image of its group in every step
 *    (a slower adjoint on a fixed 64 x 8 tile; not with the resident kernels).
 * Applies to calls enqueued afterwards; HV_EINVAL for another mode. */
#define HV_IMAGE_PAIRS 0
#define HV_IMAGE_FP64 1
int hv_set_image_precision(hv_handle *h, int mode);

#define HV_LAUNCH_PLAIN 0
#define HV_LAUNCH_PDL 1
#define HV_LAUNCH_DATAFLOW 2
int hv_set_launch_mode(hv_handle *h, int mode);

/* Profiling.  While enabled on a handle, each kernel launch the handle makes
 * is bracketed by CUDA events on the launching stream.  hv_profile_read waits
 * for those events and returns, per kernel kind (HV_K_*), the number of
 * launches and their summed device time [ms], then clears the record.  Not
 * thread-safe: profile one call stream at a time per handle. */
#define HV_K_FWD 0       /* forward step of the first sweep (with Born fields)  */
#define HV_K_ADVANCE 1   /* forward recomputation step during the reversal      */
#define HV_K_ADJ 2       /* adjoint step with zero-lag imaging                  */
#define HV_K_OTHER 3     /* model preparation, residual, reductions, fold, copies */
#define HV_K_COUNT 4
int hv_profile(hv_handle *h, int enable);
int hv_profile_read(hv_handle *h, long long *launches, double *ms);

/* Number of kernels the library has launched in this process (all handles). */
long long hv_kernel_launches(void);

/* Host-only: the checkpoint schedule the library runs for nt steps and `slots`
 * snapshots.  Writes up to max_actions triples (op, arg0, arg1) into actions
 * (HOST int array of 3*max_actions) and the counts; ops: 0 = forward step n
 * (first sweep), 1 = save current state to slot, 2 = restore slot (-1: zero
 * state), 3 = recompute one forward step, 4 = adjoint step n.  n_advances is
 * the number of recomputed forward steps.  No GPU needed. */
int hv_checkpoint_schedule(int nt, int slots, int *actions, int max_actions, int *n_actions,
                           long long *n_advances);

#ifdef __cplusplus
}
#endif

#endif /* HV_H */
