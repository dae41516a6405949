/*
 * oam.h - C ABI of liboam.so: GB300 (sm_103a) model-based AR-OAM inversion.
 *
 * Method: Li et al., "Broadband model-based inversion enables optoacoustic
 * microscopy beyond the acoustic diffraction limit" (arXiv:2009.10173).
 *
 * Data layouts (all device arrays are FP32, row-major, caller-owned):
 *   volume  H[py][px][nz]   voxel (y, x, depth k), depth fastest;
 *   signals s[py][px][nt]   A-mode signal of scan position (y, x), time fastest.
 * Voxel (y, x) sits under scan position (y, x): the lateral voxel grid equals
 * the scan grid (Results: the voxels' lateral positions match the scanning
 * positions).  Depth k is at z0_rel + k*dz relative to the focal depth, sample
 * n at time t0 + n/fs.
 *
 * Model slab (Eqs. 3-4 and "Efficient reconstruction based on scanning
 * symmetries"): S[b][a][k][n], b, a in [-R, R], R = (win-1)/2, is the signal
 * at sample n from a unit voxel at lateral offset (a*dx, b*dy) and depth k
 * relative to one scan position.  It sums, over M sensor-surface patches j of
 * area w_j at distance d_j, (w_j[mm^2] / d_j[mm]) * e'(n - fs*(d_j/c - t0)),
 * where e is the electrical impulse response (a Gaussian-windowed cosine at
 * fc whose -6 dB amplitude bandwidth is frac_bw*fc, cut at trunc_sigma
 * standard deviations) and e' its time derivative (the d/dt of Eq. 1).
 *
 *   forward  (Eq. 4, s = A_s H):  s[y][x][n] = sum_{b,a,k} S[b][a][k][n] H[y+b][x+a][k]
 *   adjoint  (A_s^T):             H[y][x][k] = sum_{b,a,n} S[b][a][k][n] s[y-b][x-a][n]
 * with H and s zero outside their grids (no wrap-around).
 *
 * Conventions for every entry point:
 *   - Returns an oam_status; nothing throws or aborts across the ABI.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Work is enqueued asynchronously on it; results are valid after the stream
 *     is synchronised, unless the function says it synchronises.
 *   - Device pointers must be distinct, non-overlapping and 16-byte aligned.
 *   - The library owns a model and its device memory; the caller owns every
 *     other buffer.  A model serves one stream at a time: concurrent calls on
 *     the same model race on its internal staging buffers.
 *   - Invalid arguments are rejected before any allocation or launch.
 */
#ifndef OAM_H
#define OAM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  OAM_OK = 0,
  OAM_ERR_INVALID_ARG = 1, /* bad pointer, size or parameter */
  OAM_ERR_WINDOW = 2,      /* arrivals fall outside [0, nt) for the time origin */
  OAM_ERR_OOM = 3,         /* device or host allocation failed */
  OAM_ERR_CUDA = 4,        /* a CUDA runtime call failed */
  OAM_ERR_DEVICE = 5,      /* a kernel reported an internal inconsistency */
  OAM_ERR_TIMEOUT = 6,     /* a bounded device-side wait ran out */
  OAM_ERR_BUSY = 7,        /* resource in use (batch / server) */
  OAM_ERR_UNSUPPORTED = 8  /* option not implemented, or GPU is not sm_103 */
} oam_status;

typedef enum {
  OAM_PREC_FP32 = 0,  /* plain FP32 slab and FP32 CUDA-core operators */
  OAM_PREC_BF16X3 = 1, /* split-BF16 (hi+lo) slab and iterate on tcgen05 tensor cores,
                          FP32 accumulation in tensor memory: hi*hi + hi*lo + lo*hi */
  OAM_PREC_FFT = 2     /* FP32 lateral-FFT form of the same operators: both are 2-D
                          correlations over the scan grid (Methods, Efficient
                          reconstruction based on scanning symmetries), restated
                          exactly by the correlation theorem on a zero-padded
                          P x P grid (P a power of two >= max(py, px) + R, at most
                          2048), with the slab's real lateral spectrum stored once
                          per frequency orbit */
} oam_precision;

/* How Eq. 1 is discretised into the model slab.
 * OAM_DISC_POINT (default): point voxels and the analytic time derivative of
 *   the EIR: S = sum_j (w_j / d_j) e'(n - fs (d_j / c - t0)).
 * OAM_DISC_TRILINEAR: the paper's two-step discretisation (Methods, Forward
 *   modeling): the surface integral of Eq. 1 over the sphere |x - x'| = ct is
 *   taken of the trilinear interpolation of the voxel values -- each voxel is
 *   the tent L(x/dx) L(y/dy) L(z/dz), L(u) = max(0, 1 - |u|), and across a
 *   tent's support the sphere is a plane, so the integral is the tent's
 *   planar Radon transform R_j (in closed form) -- and the time derivative is
 *   a central finite difference on the sample grid; the patch sum of Eq. 3
 *   and the EIR sampled at whole samples follow:
 *     I_j(m) = R_j(c t_m - r_j) / (c t_m),  t_m = t0 + m / fs,
 *     S(n)   = sum_j w_j sum_m e(n - m) (I_j(m + 1) - I_j(m - 1)) / 2,
 *   lengths in mm (arbitrary units, Eq. 2; for tents much smaller than a
 *   wavelength it tends to (dx dy dz fs / c) times the point model).  Its
 *   arrivals reach ceil(fs (dx + dy + dz) / c) + 2 samples beyond the point
 *   model's, which the automatic time origin and the window check include. */
typedef enum {
  OAM_DISC_POINT = 0,
  OAM_DISC_TRILINEAR = 1
} oam_discretisation;

/* Spherically focused sensor (AR-OAM set-up): focal length F, aperture
 * diameter D < 2F, optional central hole h < D, speed of sound c, and the
 * number M of surface patches (Eq. 3), a positive multiple of 8. */
typedef struct {
  double focal_m, aperture_m, hole_m, c_mps;
  int32_t n_patches;
} oam_sensor;

/* Scan / voxel / time grid.  win odd, 1 <= win; nt a multiple of 4.
 * t0_s = NaN selects the automatic time origin
 * t0 = (floor(fs*dmin/c - trunc_sigma*sigma_s) - 2) / fs, dmin the shortest
 * voxel-patch distance in the slab; the window check then requires
 * fs*(dmax/c - t0) + trunc_sigma*sigma_s < nt (else OAM_ERR_WINDOW). */
typedef struct {
  int32_t px, py, nz, nt, win;
  double dx_m, dy_m, dz_m, z0_rel_m, fs_hz, t0_s;
} oam_grid;

/* Electrical impulse response: centre frequency, fractional -6 dB amplitude
 * bandwidth, truncation in standard deviations (Results: EIR / SIR split). */
typedef struct {
  double fc_hz, frac_bw, trunc_sigma;
} oam_eir;

typedef struct oam_model oam_model; /* opaque */

typedef struct {
  double t0_s;         /* time of sample 0 */
  int32_t n_lo, n_hi;  /* every slab entry is zero outside samples [n_lo, n_hi) */
  int32_t n_orbits;    /* distinct lateral offsets stored (mirror symmetry) */
  int32_t precision;   /* oam_precision of forward / adjoint */
  int64_t nnz;         /* nonzero slab entries over all win*win*nz columns */
  double flops_per_op; /* algorithmic flops of one forward (= one adjoint): 2*px*py*nnz_in_grid */
  size_t device_bytes; /* device memory owned by the model */
  double exec_flops_forward, exec_flops_adjoint; /* flops issued per application: tensor-core
                                                    flops (3 BF16 products, band and tile padding)
                                                    for OAM_PREC_BF16X3, banded spectral products
                                                    and FFTs for OAM_PREC_FFT; 0 for OAM_PREC_FP32 */
  double op_bytes;     /* OAM_PREC_FFT: device bytes read + written per application (the
                          spectral slab dominates); 0 otherwise */
  int32_t filter_half_len; /* L of the band-pass filter set by oam_model_set_filter, -1: none */
  int32_t filter_size;     /* its transform length NF (0: none) */
} oam_model_info;

/* Build the model slab on the device (Methods: Forward modeling, Eqs. 1-4;
 * "it was sufficient to generate the model matrix for a single scanning
 * position").  Synchronises `stream` (the time origin and band layout are
 * planned from device results).  On success *out owns all device memory.
 * Errors: OAM_ERR_INVALID_ARG, OAM_ERR_WINDOW, OAM_ERR_OOM, OAM_ERR_CUDA,
 * OAM_ERR_UNSUPPORTED (no sm_103 device). */
oam_status oam_build_model(const oam_sensor *sensor, const oam_grid *grid, const oam_eir *eir,
                           oam_precision precision, void *stream, oam_model **out);

/* Device bytes oam_build_model would allocate for these parameters (the
 * model's device_bytes after the build; a band-pass filter set later adds
 * its own), computed on the host before anything is allocated.  The paper's
 * compressed model is a single scanning position's, so its size depends on
 * the window, depths, samples and sensor, not on the number of scan
 * positions (Results; Methods, Efficient reconstruction based on scanning
 * symmetries) -- only the tensor-core staging buffers grow with the scan.
 * The bands are planned from host-side distances with two samples of margin
 * per band edge, so the result bounds the built model's device_bytes from
 * above (by a few per cent).  Same argument errors as oam_build_model
 * (OAM_ERR_WINDOW up to rounding at the window's exact edge;
 * OAM_ERR_UNSUPPORTED for shapes a kernel does not take); no device call. */
oam_status oam_model_bytes(const oam_sensor *sensor, const oam_grid *grid, const oam_eir *eir,
                           oam_precision precision, size_t *bytes);

/* Options of oam_build_model_ex / oam_model_bytes_ex (NULL = defaults). */
typedef struct {
  int32_t discretisation; /* oam_discretisation */
} oam_model_opts;

/* oam_build_model with options (the slab's discretisation of Eq. 1). */
oam_status oam_build_model_ex(const oam_sensor *sensor, const oam_grid *grid, const oam_eir *eir,
                              oam_precision precision, const oam_model_opts *opts, void *stream, oam_model **out);
/* oam_model_bytes with options. */
oam_status oam_model_bytes_ex(const oam_sensor *sensor, const oam_grid *grid, const oam_eir *eir,
                              oam_precision precision, const oam_model_opts *opts, size_t *bytes);

/* Release a model (NULL is accepted).  Synchronises the device first. */
oam_status oam_model_free(oam_model *model);

/* Fill *info (host memory). */
oam_status oam_model_get_info(const oam_model *model, oam_model_info *info);

/* Write slab column S[b][a][k][0..nt) to device memory d_out (nt floats),
 * b, a in [-R, R], 0 <= k < nz.  For inspection and tests. */
oam_status oam_model_slab_column(const oam_model *model, int32_t b, int32_t a, int32_t k,
                                 float *d_out, void *stream);

/* s = A H (Eq. 4 applied over the scan grid).  d_H: py*px*nz floats (input),
 * d_s: py*px*nt floats (output, fully overwritten). */
oam_status oam_forward(const oam_model *model, const float *d_H, float *d_s, void *stream);

/* H = A^T s.  d_s: py*px*nt floats (input), d_H: py*px*nz floats (output,
 * fully overwritten). */
oam_status oam_adjoint(const oam_model *model, const float *d_s, float *d_H, void *stream);

/* ------------------------------------------------------ band-pass filtering */
/* Results (second simulation, in vivo): the raw signals and the model matrix
 * are band-pass filtered (0.5-80 MHz; 1-120 MHz in vivo) before inversion.
 * The filter F is a zero-phase FIR with 2L + 1 even taps h[-L..L] (h[-m] =
 * h[m]), run along time over every A-line of nt samples with samples outside
 * [0, nt) taken as zero and the centred nt outputs kept:
 *   (F s)[y][x][n] = sum_{m=-L}^{L} h[|m|] s[y][x][n - m].
 * Filtering every slab column S[b][a][k][:] with F turns A into F A (F runs
 * along time, A laterally and over depth, so they commute), and F is
 * symmetric, so the filtered adjoint is A^T F. */
#define OAM_MAX_FIR_HALF 8191

/* Design taps[0..half_len] (host memory, half_len + 1 doubles) of the
 * Blackman-windowed sinc band-pass [f_lo_hz, f_hi_hz]:
 *   h[m] = w[m] (2 f_hi/fs sinc(2 f_hi m/fs) - 2 f_lo/fs sinc(2 f_lo m/fs)),
 *   w[m] = 0.42 + 0.5 cos(pi m/(L+1)) + 0.08 cos(2 pi m/(L+1)),
 * sinc(x) = sin(pi x)/(pi x).  Host only (no device call).  Errors:
 * OAM_ERR_INVALID_ARG unless 0 <= f_lo < f_hi <= fs/2, 0 <= half_len <=
 * OAM_MAX_FIR_HALF and taps != NULL. */
oam_status oam_bandpass_taps(double f_lo_hz, double f_hi_hz, double fs_hz, int32_t half_len, double *taps);

/* Make the model's forward operator F A and its adjoint A^T F (also inside
 * the solvers, batches and autotuning) for the even FIR taps[0..half_len]
 * (host memory, copied).  taps == NULL or half_len < 0 removes the filter.
 * The transform length is the smallest power of two NF >= nt + min(L, nt-1);
 * NF > 8192 is rejected (OAM_ERR_INVALID_ARG), as are non-finite taps.
 * Allocates the filter's spectrum and one signal-sized staging buffer (owned
 * by the model, counted in device_bytes) on `stream` and synchronises it.
 * A batch that uses the model records its graph again on its next run. */
oam_status oam_model_set_filter(oam_model *model, const double *taps, int32_t half_len, void *stream);

/* d_out = F d_in over py*px A-lines of nt samples with the model's filter
 * (OAM_ERR_INVALID_ARG when none is set).  d_in and d_out may be the same
 * buffer.  Use it on measured signals before solving with a filtered model. */
oam_status oam_filter_signals(const oam_model *model, const float *d_in, float *d_out, void *stream);

/* ---------------------------------------------------------------- solvers */
/* MB-L2: Eq. 5 with the Tikhonov term of Eq. 6 (lambda = damp^2), solved by
 * LSQR (Paige & Saunders) from x0 = 0 for `iters` iterations.  Vectors are
 * FP32; norms, the bidiagonalisation scalars and the plane-rotation
 * recurrence are FP64 on the device; no host synchronisation inside the loop.
 * An exact zero alpha or beta stops early (stop_reason 1). */
typedef struct {
  int32_t iters;
  double damp;
} oam_lsqr_opts;

typedef struct {
  int32_t iters_done, stop_reason;
  double rnorm;  /* |phibar|: ||s - A x|| (damp = 0) */
  double arnorm; /* |phibar * alpha * c| */
  double anorm;  /* Frobenius-norm estimate of the bidiagonal */
} oam_lsqr_info;

/* d_s: signals (input), d_x: volume (output).  d_work / work_bytes: caller
 * workspace of at least oam_solver_work_bytes(model, 0) bytes, 256-byte
 * aligned.  If info != NULL the call synchronises `stream` and fills it. */
oam_status oam_lsqr(const oam_model *model, const float *d_s, float *d_x, const oam_lsqr_opts *opts,
                    oam_lsqr_info *info, void *d_work, size_t work_bytes, void *stream);

/* MB-L1: Eq. 5 with the L1 term of Eq. 7, f(H) = ||s - A H||^2 + lambda ||H||_1
 * (no factor 1/2), solved by FISTA (Beck & Teboulle) with constant step 1/L:
 * grad = 2 A^T (A Y - s), x = prox(Y - grad/L, lambda/L), t' = (1 + sqrt(1+4t^2))/2,
 * Y = x + ((t-1)/t')(x - x_prev), from x0 = Y = 0, t = 1.
 * L <= 0: L = 2 * 1.01 * mu, mu from `power_iters` steps of A^T A started at
 * d_power_v0 (volume-sized; NULL = all ones).  lambda < 0: lambda =
 * lambda_rel * max|A^T s|.  nonneg != 0 projects onto H >= 0. */
typedef struct {
  int32_t iters, power_iters, nonneg, compute_objective;
  double lambda, lambda_rel, L;
  const float *d_power_v0;
} oam_fista_opts;

typedef struct {
  int32_t iters_done;
  double L, lambda, mu;
  double objective; /* f at the returned x when compute_objective, else NaN */
} oam_fista_info;

oam_status oam_l1_fista(const oam_model *model, const float *d_s, float *d_x, const oam_fista_opts *opts,
                        oam_fista_info *info, void *d_work, size_t work_bytes, void *stream);

/* LSQR without any device allocation (the paper has no counterpart; this is a
 * library service).  For callers that cannot call cudaMalloc at solve time:
 * hosts that reserve all device memory up front for their own allocator, and
 * latency-critical loops that cannot take an allocation's implicit device
 * synchronisation.  Same arguments and results as oam_lsqr, but the workspace
 * is a 32 MiB array in this library's static device memory (every GPU that
 * loads the library holds it until the process exits), so problems whose
 * oam_solver_work_bytes(model, 0) exceeds 32 MiB are rejected with
 * OAM_ERR_INVALID_ARG.  Each call outside stream capture looks the array's
 * device address up in the current context (cudaGetSymbolAddress, which does
 * not allocate); a call made while `stream` is capturing reuses the address
 * of the last uncaptured call on that device, so the first call on a device
 * must come before any capture (else OAM_ERR_INVALID_ARG), and a context that
 * is reset must see an uncaptured call again before the next capture.
 * Every call on a device shares the one array, which keeps
 * the previous call's contents (each call initialises what it reads); calls
 * that overlap on the GPU race and give wrong results.  No cudaMalloc,
 * cudaFree or allocating library routine is called. */
oam_status oam_lsqr_noalloc(const oam_model *model, const float *d_s, float *d_x, const oam_lsqr_opts *opts,
                            oam_lsqr_info *info, void *stream);

/* Tikhonov sweep: MB-L2 (Eq. 5 with Eq. 6) for n_damps weights lambda_i =
 * damps[i]^2 at once.  LSQR's Golub-Kahan bidiagonalisation (u, v, alpha,
 * beta) does not depend on the damp, only the plane rotations and the x and w
 * updates do, so one forward and one adjoint per iteration serve every damp;
 * each damp keeps its own rotations and its own w.  Result i is the same as
 * oam_lsqr with damp = damps[i] and the same iters (same kernels, same
 * reduction order).  d_x: host array of n_damps device pointers to volumes
 * (outputs, 16-byte aligned); damps: host, finite, >= 0; 1 <= n_damps <=
 * OAM_MAX_SWEEP.  d_work: at least oam_lsqr_sweep_work_bytes(model, n_damps)
 * bytes, 256-byte aligned.  If infos != NULL (n_damps entries) the call
 * synchronises `stream` and fills them. */
#define OAM_MAX_SWEEP 32
oam_status oam_lsqr_sweep(const oam_model *model, const float *d_s, int32_t n_damps, const double *damps,
                          float *const *d_x, int32_t iters, oam_lsqr_info *infos, void *d_work, size_t work_bytes,
                          void *stream);
oam_status oam_lsqr_sweep_work_bytes(const oam_model *model, int32_t n_damps, size_t *bytes);

/* Workspace bytes for solver 0 = LSQR, 1 = FISTA. */
oam_status oam_solver_work_bytes(const oam_model *model, int32_t solver, size_t *bytes);

/* ------------------------------------------------------------- autotuning */
/* Pick the tensor-core kernels' tile shape for this model's shapes by timing
 * each candidate (CUDA events on `stream`, `reps` runs each after one
 * warm-up): per direction, the number of fold warps (4, 8 or 16 warps that
 * build the folded split-BF16 operand, each folding 32, 16 or 8 of a stage's
 * 32 K elements per item) and the item-ring depth (slab tiles in shared
 * memory and folded operands in tensor memory, 2 up to the deepest that
 * fits), and the position tiling (oam_model_set_tiling).  The choice is kept
 * in the model (read it with oam_model_get_tiles and oam_model_get_tiling).
 * Allocates and frees a scratch volume and signal buffer; synchronises
 * `stream`.  No-op for the other precisions.  The paper has no counterpart
 * (tuning of this implementation). */
oam_status oam_model_autotune(oam_model *model, int32_t reps, void *stream, int32_t *ring_forward,
                              int32_t *ring_adjoint);
/* Tile shape of the split-BF16 kernels, direction 0 = forward, 1 = adjoint:
 * fold warps and the ring depth in use.  OAM_ERR_UNSUPPORTED for the other
 * precisions. */
oam_status oam_model_get_tiles(const oam_model *model, int32_t direction, int32_t *fold_warps, int32_t *ring);
/* Set that shape (fold_warps 4, 8 or 16; ring 0 = deepest that fits, else
 * 2 .. deepest); OAM_ERR_INVALID_ARG leaves the model unchanged.  Results do
 * not depend on the shape (fixed summation order per accumulator). */
oam_status oam_model_set_tiles(oam_model *model, int32_t direction, int32_t fold_warps, int32_t ring);
/* Position tiling of the split-BF16 kernels, direction 0 or 1: the grid whose
 * 128 consecutive positions a block takes.  1 = the padded scan grid (rows of
 * px + R positions, the R padding positions per row computed and dropped;
 * strips of 128 + 2R staged rows), 2 = the scan grid itself (every position an
 * output; a tile that wraps w scan rows stages 128 + (w + 2) R rows, so it
 * needs w + 2 <= 128 / R and more shared memory), 0 = automatic (the scan grid
 * unless it leaves a shallower item ring).  get returns the tiling in use (1
 * or 2); set returns OAM_ERR_INVALID_ARG for other values and
 * OAM_ERR_UNSUPPORTED when the tiling does not fit, leaving the model
 * unchanged in both cases.  oam_model_autotune searches it too.  Results do not
 * depend on it. */
oam_status oam_model_get_tiling(const oam_model *model, int32_t direction, int32_t *tiling);
oam_status oam_model_set_tiling(oam_model *model, int32_t direction, int32_t tiling);

/* --------------------------------------------------------------- batching */
/* Many uneven reconstructions in one CUDA-graph launch (the paper reconstructs
 * one volume at a time; this is a serving feature).  Each job is LSQR (MB-L2)
 * and/or FISTA (MB-L1) on a model, signals, images and a workspace (at least
 * the larger of oam_solver_work_bytes(model, 0/1)); jobs run on separate
 * branches of one graph, so their kernels overlap on the GPU.  Jobs that use
 * the same model (whose staging buffers serve one stream at a time) or
 * overlapping workspaces share one branch and run in job order.  The graph
 * is recorded on the first oam_batch_run after any oam_batch_set_job and
 * replayed afterwards.  Buffers must stay valid until the run completes. */
typedef struct oam_batch oam_batch;
oam_status oam_batch_create(int32_t n_jobs, oam_batch **out);
/* d_x_l2 / d_x_l1 may be NULL when the matching iteration count is 0. */
oam_status oam_batch_set_job(oam_batch *batch, int32_t job, const oam_model *model, const float *d_s,
                             float *d_x_l2, float *d_x_l1, const oam_lsqr_opts *lsqr, const oam_fista_opts *fista,
                             void *d_work, size_t work_bytes);
/* Launch every job on `stream` (asynchronous; synchronise the stream for results). */
oam_status oam_batch_run(oam_batch *batch, void *stream);
oam_status oam_batch_free(oam_batch *batch);

/* ---------------------------------------------------------------- serving */
/* A continuous-batching request server (no counterpart in the paper).  A host
 * thread admits queued requests first-in first-out while a slot (CUDA stream)
 * is free and the device-memory reservation stays within hbm_budget_bytes
 * (oam_request_footprint: the model's planned bytes, signals, two images and
 * the solver workspace; reconciled upward with the built model's bytes if
 * they ever exceed it); each admitted request builds its model, copies its host signals
 * in, runs LSQR then FISTA, and copies both images out on its slot's stream,
 * so requests on different slots overlap on the GPU.  Finished requests
 * release their memory and slot to the next queued request.  Results do not
 * depend on what else runs (all kernels are deterministic). */
typedef struct oam_server oam_server;
typedef struct {
  size_t hbm_budget_bytes;
  int32_t max_slots;
  int32_t precision;                       /* oam_precision */
  int32_t lsqr_iters, fista_iters, power_iters;
  double lambda_rel;                       /* FISTA lambda = lambda_rel * max|A^T s| */
} oam_server_opts;
typedef struct {
  int32_t state;     /* 0 queued, 1 running, 2 done, 3 failed */
  int32_t error;     /* oam_status of a failed request */
  double latency_s;  /* submit to completion (done or failed), else -1 */
} oam_request_info;
typedef struct {
  int32_t queued, running, peak_running;
  size_t reserved_bytes, peak_reserved_bytes;
} oam_server_stats_t;
/* Device bytes the server reserves for one request before admitting it:
 * oam_model_bytes plus its signals, two images and solver workspace (an
 * upper bound of what the request allocates).  Host only.  A request whose
 * model cannot be built (oam_model_bytes fails) fails at admission with that
 * status. */
oam_status oam_request_footprint(int32_t precision, const oam_sensor *sensor, const oam_grid *grid,
                                 const oam_eir *eir, size_t *bytes);
oam_status oam_server_create(const oam_server_opts *opts, oam_server **out);
/* h_s: host signals (py*px*nt floats), h_x_l2 / h_x_l1: host images
 * (py*px*nz floats, may be NULL); all must stay valid until the request ends.
 * Submit plans the request's device footprint on the host (oam_model_bytes
 * plus buffers and workspace) and keeps the plan by geometry (the bytes of
 * sensor, grid and eir), so requests that repeat a geometry skip the planning. */
oam_status oam_server_submit(oam_server *server, const oam_sensor *sensor, const oam_grid *grid, const oam_eir *eir,
                             const float *h_s, float *h_x_l2, float *h_x_l1, int64_t *request_id);
oam_status oam_server_poll(oam_server *server, int64_t request_id, oam_request_info *info);
/* Block until the request ends or timeout_s passes (OAM_ERR_TIMEOUT). */
oam_status oam_server_wait(oam_server *server, int64_t request_id, double timeout_s);
oam_status oam_server_stats(oam_server *server, oam_server_stats_t *stats);
/* Finish queued and running requests, then release the server. */
oam_status oam_server_stop(oam_server *server);

/* ---------------------------------------------------------------- timing */
/* Device time of the operator kernels, measured with CUDA events recorded on
 * the caller's stream around the main kernel of every forward / adjoint
 * (including those inside the solvers).  The band-pass filter of a filtered
 * model runs outside these events. */
typedef struct {
  int64_t forward_calls, adjoint_calls;
  double forward_ms, adjoint_ms; /* summed event-to-event durations */
} oam_profile;

/* enable != 0 starts (and resets) event timing on this model; 0 stops it. */
oam_status oam_profile_enable(oam_model *model, int32_t enable);

/* Synchronise on the last recorded event and fill *out (host memory). */
oam_status oam_profile_read(oam_model *model, oam_profile *out);

/* Number of kernel launches this library has issued in this process. */
int64_t oam_launch_count(void);

/* Static description of a status code. */
const char *oam_status_string(oam_status status);

/* Library version (major*10000 + minor*100 + patch). */
int32_t oam_version(void);

#ifdef __cplusplus
}
#endif
#endif /* OAM_H */
