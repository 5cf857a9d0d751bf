/*
 * csem.h -- C ABI of the GB300 fictitious-wave CSEM gradient engine.
 *
 * The engine computes, for a cell-centred resistivity model on a stretched
 * tensor-product grid, the frequency-domain electric field of point dipoles
 * through the fictitious-wave correspondence of Yang (2211.16665):
 *   Sec. 2, Eq. 1      diffusive Maxwell system, time convention d/dt <-> -i w;
 *   Sec. 2, Eq. 2-3    sigma = 2 w0 eps, J' = k J, E' = E, k = sqrt(-i w / 2 w0);
 *   Sec. 2, Eq. 4      fictitious-time wave system, leap-frog staggered grid;
 *   Sec. 2, Eq. 6      on-the-fly damped transform into every frequency at once;
 * the misfit and weighted residual (Sec. 3.1, Eq. 7), the adjoint field
 * from the same engine (Sec. 3.2, Eq. 14) driven by time series built from
 * the regularised basis functions (Sec. 3.3, Eq. 8-13), and the resistivity
 * gradient (Sec. 3.1 isotropic gradient, Sec. 3.5 ln-rho chain rule).
 *
 * Conventions shared by every call
 *  - Grid: nx, ny, nz cells including an npml-cell CPML on every face; node
 *    coordinates x_0..x_nx etc. (metres, z down).  Yee placement:
 *    Ex(i,j,k) at (x_{i+1/2}, y_j, z_k), Ey at (x_i, y_{j+1/2}, z_k),
 *    Ez at (x_i, y_j, z_{k+1/2}); rho(i,j,k) at the cell centre.
 *  - Cell arrays (rho, gradient): [nz][ny][nx], x fastest.
 *  - Edge volumes ("vol"): per (source, component, frequency) a block of
 *    (nz+1)*(ny+1)*pitch complex entries, index (k*(ny+1) + j)*pitch + i,
 *    pitch >= nx+1 from csem_get_info(); entries off a component's lattice
 *    and in the row padding are zero.  Layout [n_src][3][n_freq][block].
 *  - Complex numbers are interleaved (re, im).  "real" below means float
 *    when the context's precision is 32 and double when it is 64; receiver
 *    data and residuals are always complex128.
 *  - Device pointers (suffix _dev) are CUDA global memory on the current
 *    device; the caller owns them.  The library owns only what a context
 *    allocates (fields, CPML memory, tables, graphs).
 *  - stream is a cudaStream_t passed as void*; NULL means the legacy
 *    default stream.  Calls are asynchronous on it unless stated otherwise.
 *  - Every call returns CSEM_OK (0) or a negative status and never throws;
 *    csem_last_error() then holds a message for the calling thread.
 */
#ifndef CSEM_H
#define CSEM_H

#ifdef __cplusplus
extern "C" {
#endif

#define CSEM_OK                 0
#define CSEM_ERR_INVALID_ARG   -1   /* bad size, pointer, ordering or option */
#define CSEM_ERR_OUT_OF_DOMAIN -2   /* a source or receiver lies outside the grid */
#define CSEM_ERR_CFL           -3   /* explicit dt above the stability limit */
#define CSEM_ERR_OOM           -4   /* device allocation failed */
#define CSEM_ERR_NONFINITE     -5   /* non-finite input or result */
#define CSEM_ERR_TIMEOUT       -6   /* a bounded device wait gave up */
#define CSEM_ERR_CUDA          -7   /* a CUDA runtime call failed */

typedef struct csem_ctx csem_ctx;

/* Stretched tensor-product grid (Sec. 2 and Sec. 4.2: non-uniform grid with
 * PML padding).  Host arrays, read during csem_create only. */
typedef struct {
    int nx, ny, nz;               /* cells per axis including the CPML, >= 2*npml + 2 */
    const double *xn, *yn, *zn;   /* node coordinates, strictly increasing */
    int npml;                     /* CPML thickness in cells on every face, >= 0 */
} csem_grid;

/* Point sources or receivers (Sec. 3.1: restriction operator R).  Host arrays. */
typedef struct {
    int n;                        /* number of points */
    const double *x, *y, *z;      /* coordinates [m] */
    const int *comp;              /* electric component per point: 0 = x, 1 = y, 2 = z */
} csem_points;

/* Problem options.  Host data, read during csem_create only. */
typedef struct {
    double f0;          /* reference frequency of the correspondence [Hz], w0 = 2 pi f0 (Eq. 2) */
    double rho_max;     /* resistivity that freezes the CFL step and the CPML damping [ohm-m] */
    double dt;          /* fictitious time step [s]; <= 0: s / (v(rho_max) sqrt(max 1/hx^2+1/hy^2+1/hz^2)) */
    int nt;             /* steps per run; <= 0: ceil(35 / (min_k sqrt(w_k w0) dt)) */
    double cfl_safety;  /* s above; <= 0 means 0.99 */
    int precision;      /* 32 (FP32 stencil) or 64 (FP64 stencil) */
    int kahan;          /* 1: compensated volumetric transform (FP32 only) */
    int n_freq;         /* number of inversion frequencies, 1..8 */
    const double *freqs;/* [n_freq] frequencies [Hz] */
    int max_src;        /* largest source batch any call will pass */
    int max_rec;        /* largest receiver (or adjoint-source) count */
    int anisotropy;     /* 0: isotropic, models and gradients [cells]; 1: VTI (Sec. 2:
                           sigma_h = sigma_xx = sigma_yy on the x and y edges, sigma_v =
                           sigma_zz on the z edges), models [2][cells] = (rho_h, rho_v)
                           and gradients [2][cells] = (h, v) (Sec. 3.1, Eq. 15) */
    int order;          /* spatial order of the staggered differences (Sec. 2: high-order
                           differences on the non-uniform grid): 0 or 2 = Yee; 4 = four-point
                           differences, at each half node from the nodes p-1..p+2 and at each
                           node from the half nodes q-2..q+1, the derivative of the cubic
                           through the four points (exact for cubics on any spacing), the
                           two-point difference where four points do not fit (next to the
                           outer boundary); dt <= 0 then gives 2 s / (v(rho_max) sqrt(sum over
                           axes of the largest absolute weight-row sum squared)).  Order 4 runs
                           its own H and E kernels (csem_set_launch accepts no other family) */
    int ring_slots;     /* cap on the ring of E snapshots kept per source for the deferred damped
                           transform: <= 0 takes the largest of 129, 65, 33 and 17 slots that fits
                           in 85 % of the free device memory beside the rest of the workspace; a
                           positive value also caps it (17 slots at least).  A larger ring allows
                           longer transform blocks (csem_set_launch) */
} csem_opts;

typedef struct {
    int nx, ny, nz, npml;
    int pitch;                    /* row pitch of edge volumes (elements) */
    long long vol_elems;          /* (nz+1)*(ny+1)*pitch: complex entries per (src, comp, freq) */
    double dt;                    /* time step in use */
    int nt;                       /* steps per run */
    int precision, kahan, n_freq, max_src, max_rec;
    long long workspace_bytes;    /* device memory the context holds */
    int transform_block;          /* E snapshots per damped-transform flush (16, 32, 64 or 128) */
    int anisotropy;               /* as in csem_opts */
    int order;                    /* 2 or 4, as in csem_opts */
} csem_info;

/* Creates a context on the current device: validates the grid and options,
 * derives dt / nt, builds the spacing, CPML and transform tables and
 * allocates the workspaces for max_src sources.  *ctx is set on success.
 * Errors: INVALID_ARG, CFL (dt given above the limit), OOM, CUDA. */
int csem_create(csem_ctx **ctx, const csem_grid *grid, const csem_opts *opts);

/* Releases every device and host resource of ctx (synchronises the device).  NULL is a no-op. */
void csem_destroy(csem_ctx *ctx);

/* Fills *info with the layout and derived quantities of ctx. */
int csem_get_info(const csem_ctx *ctx, csem_info *info);

/* Forward modelling (Sec. 2, Eq. 2-6; data d_syn = R u, Sec. 3.1).
 *  rho_dev   [nz][ny][nx] real resistivity [ohm-m], > 0; for a VTI context
 *            (anisotropy = 1) [2][nz][ny][nx] = (rho_h, rho_v).
 *  src       src->n unit x/y/z electric dipoles (1 A m), one per batch entry
 *            (1 <= src->n <= max_src); each is injected trilinearly on its
 *            component's lattice at t_{n+1/2}.
 *  rec       receivers (0 <= rec->n <= max_rec), sampled trilinearly at t_n.
 *  d_syn_dev [src->n][rec->n][n_freq] complex128 out: E(x_r, w_k) per source,
 *            normalised to a unit diffusive dipole, E = k_k Ehat_k / What_k.
 *  Evol_dev  NULL, or [src->n][3][n_freq][vol] complex(real) out: the same
 *            normalised E(w_k) on every edge, kept for the gradient.
 * Errors: INVALID_ARG, OUT_OF_DOMAIN, NONFINITE (rho), CUDA. */
int csem_fwd_model(csem_ctx *ctx, const void *rho_dev, const csem_points *src, const csem_points *rec,
                   double *d_syn_dev, void *Evol_dev, void *stream);

/* Adjoint-source basis (Sec. 3.3, Eq. 8-13), FP64 on the device, solved by
 * conjugate gradients on the regularised normal equations (CGNR) with B
 * formed on the fly; one unit right-hand side per column.
 *  B rows: exp(-a_k t_n) cos(a_k t_n), then exp(-a_k t_n) sin(a_k t_n),
 *          a_k = sqrt(2 pi f_k 2 pi f0), t_n = (n + 1/2) dt (injection times).
 *  gamma     regularisation; if gamma_is_relative it multiplies the largest
 *            eigenvalue of B B^T.
 *  max_iter, tol  CG stops when ||B^T(e_j - B x) - gamma x|| <= tol ||B^T e_j||.
 *  basis_dev [nt][2 n_freq] double out: the columns b_j of B+.
 *  fit_residual_host  out (may be NULL): max |B B+ - I|.
 *  iters_host         out (may be NULL): largest CG iteration count used.
 * Blocks the calling thread until the result is on the host.  Allocates
 * (and frees) 2 n_freq * nt * 16 bytes of scratch on the stream.
 * Errors: INVALID_ARG, OOM, CUDA. */
int csem_estimate_adjoint_basis(double dt, int nt, const double *freqs_host, int n_freq, double f0,
                                double gamma, int gamma_is_relative, int max_iter, double tol,
                                double *basis_dev, double *fit_residual_host, int *iters_host,
                                void *stream);

/* Same result as csem_estimate_adjoint_basis, for callers that cannot
 * allocate device memory (the paper has no counterpart; this is a deployment
 * variant).  Some applications own all device memory through their own
 * allocator (a framework's caching pool, a fixed arena) and must not see
 * foreign allocations, or run on a path where an allocation's implicit
 * synchronisation or possible failure is not acceptable.  This entry point
 * calls no cudaMalloc, cudaFree or other allocating routine: its CG work
 * vectors live in one file-scope device array of 8 MiB that every device
 * which loads the library keeps until the process exits.
 *  Limits: nt <= 32768 and n_freq <= 8, else INVALID_ARG with a message.
 *  Every call looks the array's device address up (cudaGetSymbolAddress)
 *  with the caller's device current.  With lazy module loading (the CUDA
 *  default) the first such lookup on a device loads the library's module,
 *  which reserves the array and may synchronise the device: make one call
 *  during setup, before any stream capture or latency-critical path.  After
 *  cudaDeviceReset the next call loads the module again and finds the new
 *  address.
 *  Every call shares the one array and clears the part it uses on the
 *  stream first, so
 *  calls that overlap on the GPU (two streams, two threads) race: serialise
 *  them.  Arguments, outputs and blocking behaviour are those of
 *  csem_estimate_adjoint_basis.
 * Errors: INVALID_ARG, CUDA. */
int csem_estimate_adjoint_basis_noalloc(double dt, int nt, const double *freqs_host, int n_freq, double f0,
                                        double gamma, int gamma_is_relative, int max_iter, double tol,
                                        double *basis_dev, double *fit_residual_host, int *iters_host,
                                        void *stream);

/* Misfit and weighted residual (Sec. 3.1, Eq. 7):
 *   phi = 1/2 sum |w (d_obs - d_syn)|^2,  resid = w^2 (d_obs - d_syn).
 *  n            number of complex entries.
 *  weight_dev   NULL (w = 1) or [n] double real weights.
 *  resid_dev    [n] complex128 out;  phi_dev  1 double out.
 * Errors: INVALID_ARG, CUDA. */
int csem_misfit(int n, const double *d_obs_dev, const double *d_syn_dev, const double *weight_dev,
                double *resid_dev, double *phi_dev, void *stream);

/* Adjoint modelling (Sec. 3.2, Eq. 14 with the conjugation trick; Sec. 3.3).
 * Each receiver becomes an electric dipole whose diffusive moment is
 * conj(resid); its fictitious series is B+ [Re c; Im c] with
 * c_k = k_k conj(resid_k) / dt, injected like a forward source, and the
 * output is conj(v) = dt * (damped transform of the adjoint field).
 *  rho_dev    as in csem_fwd_model.
 *  rec        the receivers of the residual (0 < rec->n <= max_rec).
 *  n_src      batch size (1..max_src).
 *  resid_dev  [n_src][rec->n][n_freq] complex128 weighted residual W^T W (d - R u).
 *  basis_dev  [nt][2 n_freq] double from csem_estimate_adjoint_basis.
 *  Vvol_dev   [n_src][3][n_freq][vol] complex(real) out: conj(v) on every edge.
 * Errors: INVALID_ARG, OUT_OF_DOMAIN, NONFINITE, CUDA. */
int csem_adjoint_model(csem_ctx *ctx, const void *rho_dev, const csem_points *rec, int n_src,
                       const double *resid_dev, const double *basis_dev, void *Vvol_dev, void *stream);

/* Resistivity gradient (Sec. 3.1 isotropic form, scaled by the cell volume;
 * Sec. 3.5 chain rule).  Edge form -Re sum_s sum_k conj(v)_e E_e dV_e mapped
 * to cells by the transpose of the edge conductivity average
 * sigma_e = sum_c V_c sigma_c / sum_c V_c.  For a VTI context (Sec. 3.1,
 * Eq. 15) the x and y edges of a cell give its sigma_h gradient and the z
 * edges its sigma_v gradient.
 *  Evol_dev, Vvol_dev  [n_src][3][n_freq][vol] from the two runs.
 *  wrt        0: d phi / d sigma_c;  1: d phi / d ln(rho_c) = -sigma_c d phi / d sigma_c
 *             (per part for VTI: -sigma_h d phi / d sigma_h, -sigma_v d phi / d sigma_v).
 *  grad_dev   [nz][ny][nx] real ([2][nz][ny][nx] = (h, v) for VTI),
 *             ACCUMULATED (+=) so batches can be summed.
 * Errors: INVALID_ARG, CUDA. */
int csem_gradient(csem_ctx *ctx, const void *rho_dev, const void *Evol_dev, const void *Vvol_dev,
                  int n_src, int wrt, void *grad_dev, void *stream);

/* Time-domain adjoint gradient (the paper's appendix): the exact gradient of
 * the discrete scheme, a second route to the one above that needs no basis
 * estimate.  The adjoint of the leap-frog scheme is the same scheme run in
 * reversed fictitious time, m = nt - 1 - n, driven at the receivers like a
 * source by q^{nt-1-m}, q^n = Re sum_k conj(r_k) alpha_k w_{k,n}
 * (alpha_k = k_k / What_k the forward normalisation, w_{k,n} the transform
 * weights exp((-1+i) a_k n dt)); with E^n the forward E after n steps and
 * Et^m the adjoint E after m steps,
 *     dphi/dsigma_e = -1 / (2 w0 dt) sum_{m<nt} dV_e Et_e^m (E_e^{nt-m} - E_e^{nt-1-m})
 * (appendix: dphi/dsigma = -(1 / 2 w0) int Et . dE/dt' dt'), mapped to cells
 * and to ln rho as in csem_gradient.  Because the forward field is consumed
 * backwards in time, the forward run is replayed in segments of `segment`
 * steps from checkpoints of its state (H, the E snapshot, the CPML memory)
 * kept by a first pass; each replayed segment's E snapshots sit in a ring in
 * the workspace while the adjoint run advances through them.  Forward steps:
 * (ceil(nt / segment) - 1) * segment + nt; adjoint steps: nt.
 *
 * csem_td_plan: workspace for n_src sources and n_rec receivers.  In:
 *  *segment_out > 0 asks for that segment length (even); else the call picks
 *  the length with the least replayed steps whose workspace fits budget_bytes
 *  (budget_bytes <= 0: the smallest workspace).  Out: *segment_out, and
 *  *bytes_out the workspace size.  The size depends on the launch
 *  configuration in force (csem_autotune, csem_set_launch): plan after it.
 *  Errors: INVALID_ARG, OOM (no plan fits the budget).
 * csem_gradient_td:
 *  rho_dev    as in csem_fwd_model.
 *  src, rec   sources (1..max_src) and receivers (1..max_rec) of the residual.
 *  resid_dev  [src->n][rec->n][n_freq] complex128 weighted residual, as for
 *             csem_adjoint_model (the data of the same model and sources).
 *  segment    from csem_td_plan (even, >= 2).
 *  wrt, grad_dev  as in csem_gradient (ACCUMULATED, += ; summed over sources).
 *  work_dev   device workspace of work_bytes >= the plan's bytes, 256-byte
 *             aligned, owned by the caller; its contents are scratch.
 * Overwrites the context's field state.
 * Errors: INVALID_ARG (also a workspace too small), OUT_OF_DOMAIN, CUDA. */
int csem_td_plan(const csem_ctx *ctx, int n_src, int n_rec, long long budget_bytes, int *segment_out,
                 long long *bytes_out);
int csem_gradient_td(csem_ctx *ctx, const void *rho_dev, const csem_points *src, const csem_points *rec,
                     const double *resid_dev, int segment, int wrt, void *grad_dev, void *work_dev,
                     long long work_bytes, void *stream);

/* Early end of forward data runs (Sec. 2: the stepping can stop once the
 * frequency-domain field has reached its steady state, checked regularly during
 * the run).  tol > 0: csem_fwd_model calls that keep no volumes (Evol_dev NULL,
 * at least one receiver) check, after every 64 steps, the running transform
 * R_c[s][r][k] = sum_{n < 64 (c+1)} w_{k,n} E^n(x_r) and end after the first
 * chunk c >= 1 with |R_c - R_{c-1}| <= tol |R_c| for every source, receiver and
 * frequency; the data are then alpha_k R_c.  The transform is flushed after each
 * block (never overlapped) in these runs.  tol = 0 turns the check off (the
 * default).  Runs that keep volumes, adjoint runs and csem_gradient_td always
 * take nt steps.  The first call with tol > 0 allocates the check's buffers.
 * csem_last_run_steps: the steps whose snapshots the last csem_fwd_model or
 * csem_adjoint_model run includes (nt unless it ended early, here or through
 * csem_set_early_stop_volumes); synchronises stream.
 * Errors: INVALID_ARG, OOM, CUDA. */
int csem_set_early_stop(csem_ctx *ctx, double tol);
int csem_last_run_steps(csem_ctx *ctx, void *stream, int *steps);

/* Early end of runs that keep volumes (csem_fwd_model with Evol_dev, csem_adjoint_model;
 * the same reading of Sec. 2 on the volumetric transform).  tol > 0: after every 64
 * steps one pass over the accumulators checks every entry of every source, component
 * and frequency k: t_k |acc - acc at the previous check| <= tol max(|acc|, floor_frac
 * A_k), A_k the largest |acc| of frequency k at the previous check and t_k = |q| / |1 - q|,
 * q = exp((-1 + i) a_k 64 dt), the remainder an endless run would still add per unit of
 * the last chunk's change if the field stayed as it was (the weights' geometric tail) --
 * entries of at least floor_frac of the largest converge in relative terms, smaller ones
 * to tol floor_frac A_k (floor_frac in [0, 1]); the run ends after the first chunk c >= 1
 * where every entry passes (the decision taken in FP32).  The volumes (and the receivers of a forward run) then hold
 * the transform of the steps up to that chunk; csem_last_run_steps reports them.  The
 * host waits for each chunk's verdict before issuing the next, so nothing runs past the
 * end.  tol = 0 turns it off (the default); the first call with tol > 0 allocates a
 * copy of max_src volumes.  The time-domain gradient always takes nt steps.
 * Errors: INVALID_ARG, OOM, CUDA. */
int csem_set_early_stop_volumes(csem_ctx *ctx, double tol, double floor_frac);

/* Picks the launch shape of the H and E stepping kernels -- z planes per
 * thread (1, 2, 4, 8), the register budget (4, 6 or 8 resident 256-thread
 * blocks per SM), and for FP32 one or four cells per thread along x, the
 * bulk-copy-staged kernels (1, 2 or 4 rows per block, 2-16 planes) or the
 * lean four-cell kernels (1, 2 or 4 planes; see csem_set_launch) -- by
 * timing each candidate on n_src sources of this grid;
 * later calls use the fastest.  It then times the fused H+E step kernels (the
 * tiled one with z blocking 4, 8 or 16; for FP32 the one-pass, warp-specialised
 * and wave-ordered steps) against the best split pair and keeps the fastest, and
 * last, when nt >= 256, the transform flush over 128 steps: the register
 * kernel or (FP32) the bulk-copy kernel, over 16, 32, 64 or 128 snapshots, run after
 * its block or on a second stream overlapping the next block (needs a ring of
 * 2 * snapshots + 1 slots; the results are the same bit for bit).  kz_out
 * (may be NULL, else 4 ints) receives, for H and E, 16 * planes + blocks
 * (+ 256 for the FP32 four-cells-per-thread kernel, + 1024 * rows for the
 * bulk-copy-staged kernel, + 8192 * cells per thread for the lean kernel), then 4 * snapshots per flush + flush mode (as in
 * csem_set_launch), then the step's form: 0 split, 4/8/16 the fused z
 * blocking, 10000 + code the one-pass kernel, 30000 + code the
 * warp-specialised fused kernel, 50000 + code the wave-ordered step.  Overwrites the
 * context's field state and blocks until the timing is done.
 * Errors: INVALID_ARG, CUDA. */
int csem_autotune(csem_ctx *ctx, int n_src, int *kz_out, void *stream);

/* Sets the launch configuration by hand instead of csem_autotune (tests run
 * every variant through it): cfg = {H z planes, H blocks/SM, E z planes,
 * E blocks/SM, step form (0 = split kernels; 4, 8 or 16 = the tiled fused
 * kernel's z blocking; 10000 + planes * 100 + rows * 10 + blocks = the one-pass
 * kernel with TMA-staged planes; 30000 + planes * 100 + rows * 10 + blocks = the
 * warp-specialised fused kernel: producer warps compute H^{n+1/2} of the tile and
 * its one-cell halo into shared memory, consumer warps the E step from it; rows
 * and blocks (4,2), (4,3), (6,2), (8,1), (8,2); FP32, second order; 50000 + lag * 100 +
 * planes * 10 + blocks = the wave-ordered step: the lean H and E tiles (2 cells per
 * thread, 2 or 4 planes, 6 or 8 blocks/SM) of one step in one launch, each block taking
 * the next ticket of a counter, E of z block c after H of z block c + lag, so that E reads
 * E^n and H^{n+1/2} while they are still in L2; an E tile waits (bounded) until H of its
 * z block and the one below is complete; FP32, second order, nx a multiple of 4), flush mode (bit 0: bulk
 * copy, FP32 only, else register kernel; bit 1: overlapped with the next
 * block on a second stream), snapshots per flush (16, 32, 64 or 128; the
 * context's ring of 17, 33, 65 or 129 slots must hold snapshots + 1, or
 * 2 * snapshots + 1 when overlapped; runs with an early end flush at most 64 at
 * a time), H four-cells-per-thread (0/1, FP32, 4 or 6 blocks/SM),
 * E four-cells-per-thread (0/1), H bulk-copy-staged rows per block (0, or
 * 1/2/4 for FP32 when the staged planes fit shared memory; z planes 2-16),
 * E bulk-copy-staged rows per block, H lean kernel (0 off, or 1 or 2 cells
 * per thread: FP32 with nx a multiple of 4 and room for the CPML memory in 12
 * volume arrays per source; 1, 2 or 4 planes; blocks of 128 threads, 6 or 8
 * resident per SM, or 4, 6 or 8 with 2 cells), E lean kernel (0, 1 or 2)}
 * -- 13 ints.  The
 * lean kernel takes precedence over the staged and four-cell ones.
 * Synchronises the device.
 * Errors: INVALID_ARG. */
int csem_set_launch(csem_ctx *ctx, const int *cfg);

/* Test hooks.
 * csem_set_wavelet: forward source time function J'(t_{n+1/2}) (host [nt]
 * doubles, copied), or NULL for the unit impulse J'_0 = 1/dt.  The forward
 * normalisation divides by its damped transform, so E does not depend on it.
 * csem_set_trace: when trace_dev ([max_src][rec n][nt] double) is non-NULL,
 * later forward runs also store the sampled E(x_r, t_n). */
int csem_set_wavelet(csem_ctx *ctx, const double *wavelet_host);
int csem_set_trace(csem_ctx *ctx, double *trace_dev);

/* Test hook for failure detection: with extra_bytes > 0 (a multiple of 16, at most 4096)
 * the first shared-memory stage of every block of the bulk-copy kernels (the transform
 * flush, the row-staged step kernels, the fused one-pass step) expects extra_bytes more
 * than its copies bring, so the bounded wait on it runs out after about a second: the
 * block leaves without writing results, and the next csem_check reports CSEM_ERR_TIMEOUT.
 * The copies themselves complete; nothing faults.  In the warp-specialised fused step,
 * whose warps hand planes over through shared memory without copies, the producer warps
 * skip their first arrival instead, so the consumers' bounded wait runs out (and then the
 * producers' own).  In the wave-ordered step the E tiles wait for one H tile more than
 * there are, so the first wave of E tiles gives up after about a second and the rest skip
 * the wait.  0 restores normal operation (the
 * field state of the run that timed out is not usable).  Synchronises the device.
 * Errors: INVALID_ARG. */
int csem_set_copy_fault(csem_ctx *ctx, int extra_bytes);

/* Synchronises stream and reports problems seen on the device since the last
 * check: TIMEOUT if a bulk-copy kernel gave up waiting for its copies (about a
 * second per wait; a transform flush then leaves its block's accumulators
 * unchanged, a step kernel its block's fields; the message names the kernel
 * family), NONFINITE if a resistivity was non-positive or non-finite (such
 * cells get zero conductivity). */
int csem_check(csem_ctx *ctx, void *stream);

/* Measurement hooks.
 * csem_launch_count: number of CUDA kernels this library has launched in the
 * process so far (each replay of a captured chunk counts its kernel nodes).
 * csem_time_step_kernels: on the state left by the last run of ctx, launches
 * each stepping kernel `launches` times for n_src sources and returns the mean
 * duration of one launch in milliseconds, from CUDA events on stream:
 * ms_out[0] = split H half-step, ms_out[1] = fused H+E step when the
 * autotuner selected it (else 0), ms_out[2] = split E step (with the source
 * injection of the last forward run; without injection when the last run was
 * an adjoint run),
 * ms_out[3] = one damped-transform flush of transform_block snapshots
 * into vol_dev ([n_src][3][n_freq][vol] complex(real), overwritten).  Field
 * values are overwritten. */
long long csem_launch_count(void);
int csem_time_step_kernels(csem_ctx *ctx, int n_src, void *vol_dev, int launches, double *ms_out, void *stream);

/* Message of the last failing call on this thread ("" if none). */
const char *csem_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CSEM_H */
