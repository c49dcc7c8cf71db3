/*
 * enufft.h -- C ABI of the B300 (sm_103a) ENUFFT hot-path library.
 *
 * The library evaluates, for every cell of an unstructured triangular or hexagonal grid, the
 * windowed quadrature sum of the paper "Elastic Non-Uniform FFT (ENUFFT)" (arxiv 2606.21278),
 *
 *     h_mn = 1/|D| sum_q win_q w_q h_q exp(-i (k_m x'_q + k_n y'_q)),   k_m = 2 pi m / L,
 *
 * (App. B, Eq. discrete_quadrature, with the local window of App. A), by a type-1 NUFFT
 * (Sec. 2.1.2: spread, FFT, deconvolve) with an exponential-of-semicircle kernel (or the paper's
 * Kaiser-Bessel kernel), and then the
 * Elastic Mode Selection of Sec. 2.2 on each spectrum.  It also provides the adjoint (type-2)
 * needed for gradients of the EMS-retained power with respect to the samples and weights.
 *
 * Conventions shared by every call
 *   - Pointers prefixed d_ are caller-owned DEVICE memory on the plan's device; nothing is
 *     copied to or from the host during execution calls, and the library never frees them.
 *   - Samples are grouped by cell in CSR form: cell j owns samples [offsets[j], offsets[j+1]).
 *     x, y are local tangent-plane coordinates; h is elevation; w is the quadrature weight.
 *     Arrays are plain SoA vectors of float (ENUFFT_FP32 / ENUFFT_MIXED plans) or double
 *     (ENUFFT_FP64 plans).
 *   - Coefficients are complex (interleaved re, im) float or double, laid out
 *     coeffs[cell][n + P/2][m + P/2] for m, n in [-P/2, P/2) (row index n is the y mode).
 *     They follow the paper's phase origin x' = u + H (App. A), so a cell's spectrum is
 *     exactly the quadrature sum above.
 *   - Every execution call is asynchronous and stream-ordered on the plan's stream; argument
 *     errors are returned synchronously before anything is launched.  Conditions detected on
 *     the device (non-finite coordinates, exhausted bounded waits) are latched in a device
 *     status word and reported by enufft_sync_status().  The library never aborts or traps.
 *   - A plan is bound to one device, one set of cells and one CSR offset vector; sample values
 *     may change from call to call.  A plan is not thread-safe; distinct plans are.
 */
#ifndef ENUFFT_H
#define ENUFFT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct enufft_plan_s *enufft_plan;

typedef enum {
    ENUFFT_OK = 0,
    ENUFFT_ERR_ARG = 1,          /* invalid argument (null pointer, bad size, bad option)       */
    ENUFFT_ERR_CUDA = 2,         /* a CUDA runtime call failed                                   */
    ENUFFT_ERR_NOMEM = 3,        /* device allocation failed                                     */
    ENUFFT_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up                           */
    ENUFFT_ERR_UNSUPPORTED = 5,  /* option combination not implemented on this build             */
    ENUFFT_ERR_DEVICE = 6        /* device-detected data error (e.g. non-finite coordinates)     */
} enufft_status;

typedef enum {
    ENUFFT_FP64 = 0,   /* everything in binary64 (inputs/outputs double)                         */
    ENUFFT_FP32 = 1,   /* plain binary32 per-cell launches (the comparison path)                 */
    ENUFFT_MIXED = 2   /* product path: binary32 spreading/FFT with exact-binary32 coordinate
                          transforms from binary64 per-cell constants, binary64 EMS sums          */
} enufft_precision;

typedef enum { ENUFFT_MASK_CELL = 0, ENUFFT_MASK_SQUARE = 1, ENUFFT_MASK_CIRCLE = 2 } enufft_mask;

/* Spreading kernel (Sec. 2.1.2).  Either choice reaches the same quadrature sum within the
 * plan's tolerance; the kernel only changes how the spread/FFT/deconvolve route gets there (the
 * tensor-core direct sum uses no kernel).
 *   ES: exponential of semicircle phi(z) = exp(beta (sqrt(1 - z^2) - 1)), z = 2 tau / w,
 *       beta = 2.30 w at sigma = 2 (scaled by (1 - 1/(2 sigma)) / 0.75 otherwise); Phi by
 *       Gauss-Legendre quadrature at plan time.
 *   KB: Kaiser-Bessel, Eq. kb_compact with half-width a = w/2 grid points and the shape of
 *       Eq. kaisal_bessel_coeffs (beta = 2.34, gamma = pi sqrt((2 a beta / pi)^2 - 0.8)),
 *       normalised to phi(0) = 1 (a constant factor that the deconvolution divides out); Phi
 *       from the closed form of Eq. kb_fourier. */
typedef enum { ENUFFT_KERNEL_ES = 0, ENUFFT_KERNEL_KB = 1 } enufft_kernel;

/* Orientation of each cell's local frame (App. A).  Both use the centroid x-bar as origin and the
 * square B = [-H, H]^2, H = (eta/2) max extent measured in the frame, x' = u + H.
 *   CENTROID: the original axes, u = x - x-bar.
 *   EDGE:     u = R (x - x-bar) with R = [[cos t, sin t], [-sin t, cos t]] (Eq. rotation_matrix),
 *             (cos t, sin t) = e / |e| for the longest polygon edge e = v_(i+1) - v_i (the first one
 *             on a tie), so that edge runs along +x.  Each execution call then starts with one
 *             extra kernel that writes every sample's local coordinates, in binary64 arithmetic,
 *             into plan-owned scratch (n_points x 2 values of the plan's precision), taking the
 *             window decision there on the exact binary64 coordinates; binary32 plans store the
 *             rounded coordinates, moved by at most a few units in the last place toward the
 *             centroid where rounding would otherwise carry a windowed sample across the window's
 *             boundary.  enufft_voronoi_weights is not built for these plans. */
typedef enum { ENUFFT_FRAME_CENTROID = 0, ENUFFT_FRAME_EDGE = 1 } enufft_frame;

typedef struct {
    int modes;            /* P, retained modes per dimension: even, 2..128                       */
    double oversamp;      /* sigma >= 2: fine grid n_f = smallest power of two >= sigma * P      */
    int kernel_width;     /* w (grid points) of the spreading kernel, 2..16                      */
    double tol;           /* requested relative accuracy; w is raised to ceil(log10(1/tol)) + 1
                             when that is larger (0 = use kernel_width as given)                  */
    enufft_precision prec;
    enufft_mask mask;     /* App. A support mask                                                 */
    double eta;           /* App. A window expansion factor: H = (eta/2) * max extent            */
    int tc_max_points;    /* cells with at most this many samples take the tensor-core direct
                             sum (Eq. discrete_quadrature as a dense contraction); 0 = off.
                             Mixed-precision plans with modes <= 64 only: other plans with a
                             positive value return ENUFFT_ERR_UNSUPPORTED                       */
    enufft_kernel kernel; /* spreading kernel (default ES)                                       */
    enufft_frame frame;   /* local frame orientation (default CENTROID)                          */
    int autotune;         /* 1: tune the execution routes at plan creation (see enufft_tuning):
                             the tensor-core routing threshold, at most tc_max_points, and the
                             fused kernel's blocks per SM, or for n_f = 256 plans the tile side of
                             the sorted spreading; 0 (default): take tc_max_points as given and
                             tiles of 32.  Mixed-precision plans only; elsewhere it has no effect */
    const char *tune_cache;   /* NULL, or a JSON file of earlier tunings (read, and written on a
                                 miss) keyed by GPU name, SM count, P, n_f, w, precision, kernel,
                                 frame and tc_max_points                                        */
    int deterministic;    /* 1 (default) or 0.  Every route is bit-reproducible run to run (the
                             spreading sums are integer, every other reduction has a fixed
                             order), so both values select the same code; other values return
                             ENUFFT_ERR_ARG                                                      */
} enufft_opts;

typedef struct {
    int k_min, k_max;                 /* spectral budget K_min <= K* <= K_max (Eq. k_elastic)     */
    double alpha_min, alpha_max;      /* Eq. alpha_c                                              */
    double delta;                     /* Eq. s_delta                                              */
    double w1, w2;                    /* Eq. c_score                                              */
    int sum_over;                     /* 0: sums over the top J_max = min(J*, K_max) energies
                                         (footnote of Eq. alpha_c); 1: over all J* energies        */
    int include_dc;                   /* 0: the (0,0) mode is not a candidate                     */
} enufft_ems_params;

/* Defaults: P = 64, sigma = 2, w = 7, tol = 0, MIXED, cell mask, eta = 1.5, no tensor-core path,
 * ES kernel, centroid-aligned frame, no autotuning, no tuning cache, deterministic. */
void enufft_default_opts(enufft_opts *opts);
/* Defaults of the paper's EMS illustration (Sec. 2.2): K_min 1, K_max 12, alpha 0..0.7,
 * delta 0.02, w1 = w2 = 0.5, HEAD sums, DC excluded. */
void enufft_default_ems(enufft_ems_params *params);

/*
 * Create a plan for n_cells cells (App. A window, Sec. 2.1.3 per-cell transforms).
 *   d_cell_offsets  int64[n_cells + 1], non-decreasing, offsets[0] = 0 (device)
 *   d_cell_nverts   int32[n_cells], convex polygon vertex counts in 3..6 (device)
 *   d_cell_verts    double[n_cells][6][2] polygon vertices, either orientation (device)
 *   cuda_stream     cudaStream_t for every call of this plan (NULL = legacy default stream)
 * Computes the per-cell frames (centroid, H, L, |D|) on the device in binary64, copies the
 * offsets to the host once to order cells by size and to route small cells, and allocates the
 * plan's device state.  This call synchronises the stream.  On failure *out is NULL.
 */
enufft_status enufft_plan_create(enufft_plan *out, const enufft_opts *opts, int64_t n_cells,
                                 const int64_t *d_cell_offsets, const int32_t *d_cell_nverts,
                                 const double *d_cell_verts, void *cuda_stream);

/* Release every resource of the plan (synchronises its stream first). NULL is accepted. */
enufft_status enufft_plan_destroy(enufft_plan plan);

/*
 * Type-1 transform of every cell (Sec. 2.1.2 steps 1-4 with the App. A/B window and weights):
 *   d_x, d_y, d_h, d_w  [N] samples (N = offsets[n_cells])
 *   d_coeffs            [n_cells][P][P] complex output, every entry written
 * Cells with no sample inside their window get all-zero coefficients.
 */
enufft_status enufft_type1(enufft_plan plan, const void *d_x, const void *d_y, const void *d_h,
                           const void *d_w, void *d_coeffs);

/*
 * Elastic Mode Selection (Sec. 2.2, Eqs. energy .. k_elastic) on every cell's spectrum:
 *   d_coeffs          [n_cells][P][P] complex (as written by enufft_type1)
 *   d_mode_weights    NULL (all 1), double[P][P] shared by all cells (per_cell = 0) or
 *                     double[n_cells][P][P] (per_cell = 1); a pair takes the weight of its
 *                     half-plane member (Eq. weighted_e)
 *   d_kstar           int32[n_cells]                  selected count K*
 *   d_sel             int32[n_cells][k_max]           selected pair indices in decreasing energy,
 *                     -1 padded; a pair +-(m,n) is named by its member with n > 0 or (n = 0,
 *                     m > 0), encoded p = (n + P/2) * P + (m + P/2)
 *   d_retained_power  double[n_cells]                 sum of the K* selected (weighted) energies
 * Candidates are the pairs of the symmetric box |m|, |n| <= P/2 - 1.  Energies are formed in
 * binary32 from binary32 coefficients (binary64 for FP64 plans); ranking ties go to the lower
 * pair index; the cumulative power and its threshold test are binary64.
 */
enufft_status enufft_ems(enufft_plan plan, const void *d_coeffs, const double *d_mode_weights,
                         int mode_weights_per_cell, const enufft_ems_params *params,
                         int32_t *d_kstar, int32_t *d_sel, double *d_retained_power);

/* enufft_type1 followed by enufft_ems, fused into one pass where the plan allows it (the
 * spectrum is selected while it is still on chip).  Same arguments and results as the two calls. */
enufft_status enufft_type1_ems(enufft_plan plan, const void *d_x, const void *d_y, const void *d_h,
                               const void *d_w, void *d_coeffs, const double *d_mode_weights,
                               int mode_weights_per_cell, const enufft_ems_params *params,
                               int32_t *d_kstar, int32_t *d_sel, double *d_retained_power);

/*
 * enufft_type1_ems through a CUDA graph that the plan owns (batching of many cells into a fixed
 * launch sequence; no counterpart in the paper, whose transforms run on a CPU).  Same arguments,
 * results and errors as enufft_type1_ems.  The first call, and every call whose pointers, mode-
 * weight layout or EMS parameters differ from the captured ones, captures the call's kernels on a
 * plan-owned stream and instantiates the graph; every call then launches the graph on the plan's
 * stream.  A replay reads the buffers named at capture: their contents may change between calls,
 * their addresses may not without a new capture (which happens automatically).  The graph is
 * destroyed with the plan.  Argument errors are returned before any capture; a failed capture
 * leaves the plan without a graph and returns the error of the failing step.
 */
enufft_status enufft_type1_ems_graph(enufft_plan plan, const void *d_x, const void *d_y, const void *d_h,
                                     const void *d_w, void *d_coeffs, const double *d_mode_weights,
                                     int mode_weights_per_cell, const enufft_ems_params *params,
                                     int32_t *d_kstar, int32_t *d_sel, double *d_retained_power);

/*
 * Gradient of the EMS-retained power with the selection held fixed:
 *   G_mu = 2 * grad_power[j] * W_p * h_mu on both members of each selected pair of cell j, 0 elsewhere,
 * i.e. G = dL/dRe(h) + i dL/dIm(h) for L = sum_j grad_power[j] * retained_power[j].
 *   d_coeffs, d_mode_weights, per_cell, d_kstar, d_sel as for enufft_ems (k_max from params)
 *   d_grad_power      double[n_cells]
 *   d_grad_coeffs     [n_cells][P][P] complex output (same precision as the coefficients)
 */
enufft_status enufft_ems_backward(enufft_plan plan, const void *d_coeffs, const double *d_mode_weights,
                                  int mode_weights_per_cell, const enufft_ems_params *params,
                                  const int32_t *d_kstar, const int32_t *d_sel,
                                  const double *d_grad_power, void *d_grad_coeffs);

/*
 * Adjoint of enufft_type1 (a type-2 NUFFT: deconvolve, inverse FFT, interpolate):
 *   d_grad_coeffs  [n_cells][P][P] complex G = dL/dRe(h_mn) + i dL/dIm(h_mn)
 *   d_grad_h       [N] dL/dh_q = win_q w_q v_q / |D|     (may be NULL)
 *   d_grad_w       [N] dL/dw_q = win_q h_q v_q / |D|     (may be NULL)
 *   with v_q = Re sum_mn G_mn exp(+i (k_m x'_q + k_n y'_q)).
 * Every route: the fused adjoint kernel for n_f <= 128 (cells of the tensor-core route included),
 * two kernels per batch for n_f = 256 (inverse transforms into the batch's fine grids, then
 * interpolation from staged windows of them).  Plain FP32 plans return ENUFFT_ERR_UNSUPPORTED.
 */
enufft_status enufft_type1_backward(enufft_plan plan, const void *d_grad_coeffs, const void *d_x,
                                    const void *d_y, const void *d_h, const void *d_w, void *d_grad_h,
                                    void *d_grad_w);

/*
 * Voronoi quadrature weights by raster sampling (App. A, Eqs. raster_grid .. voronoi_weights) for
 * the samples of every cell, on the plan's stream, binary32 plans only (binary64 plans return
 * ENUFFT_ERR_UNSUPPORTED):
 *   - raster points at the centres of an ng x ng grid over the cell's square B, kept when inside
 *     the window (the plan's mask);
 *   - each kept point goes to its nearest windowed sample (Eq. nn_assignment: the squared
 *     distance in binary64, every operation rounded as written, ties to the lowest sample index;
 *     the search runs in binary32 and re-decides in binary64 where the binary32 gap to the
 *     second-nearest sample is within its certified rounding bound); n_q counts its points;
 *   - d_w[q] = max(n_q, 1/2) |D| / sum_q' max(n_q', 1/2) (a sample no point reached takes the
 *     floor 1/2; the weights of a cell sum to |D|), 0 for samples outside the window.
 * d_w [N] binary32 (caller-owned) is also the count scratch while the call runs.  ng in [2, 1024];
 * the work is ng^2 x (windowed samples) distance evaluations per cell.
 */
enufft_status enufft_voronoi_weights(enufft_plan plan, const void *d_x, const void *d_y, int ng, void *d_w);

/*
 * Reconstruction diagnostics of Sec. 3.2 from coefficients and an EMS selection (as written by
 * enufft_type1_ems / enufft_ems on this plan).  The mode set is the selected pairs and their
 * partners: for k < kstar[j], p = sel[j][k] marks (m, n) with p = (n + P/2) P + (m + P/2), and
 * (-m, -n).  On the plan's stream, per cell j:
 *   d_hrec[q]        h_rec(x_q) = Re sum over the set of h_mn exp(+i (k_m x'_q + k_n y'_q)), the
 *                    truncated series of Eq. tri_series at the samples (0 outside the window;
 *                    may be NULL); float or double as the plan's samples
 *   d_stats[4 j + 0] eps_rel = sqrt(sum_q (h_q - h_rec(x_q))^2 / sum_q h_q^2) over the windowed
 *                    samples (Eq. alps_relative_rmse; 0 when every h_q is 0)
 *   d_stats[4 j + 1] sigma2_phys = (1/|D|) sum_q w_q h_q^2 over the windowed samples
 *   d_stats[4 j + 2] sigma2_spec over the selected set, (m, n) != (0, 0)
 *   d_stats[4 j + 3] sigma2_spec over the whole P x P box, (m, n) != (0, 0)   (Eq. spectral_variance)
 * The paper evaluates these on deplaned elevations (h minus the cell's weighted mean); the call
 * uses h as given.  k_max is the row length of d_sel (1..64).  Built on the adjoint's kernels of
 * each route; plain FP32 plans return ENUFFT_ERR_UNSUPPORTED; NULL pointers or a bad k_max return
 * ENUFFT_ERR_ARG.
 */
enufft_status enufft_reconstruct(enufft_plan plan, const void *d_coeffs, const int32_t *d_kstar,
                                 const int32_t *d_sel, int k_max, const void *d_x, const void *d_y,
                                 const void *d_h, const void *d_w, void *d_hrec, double *d_stats);

/* Re-bind the plan to another stream of the same device (e.g. the caller's current stream);
 * work already queued on the old stream is not waited for.  NULL selects the legacy default. */
enufft_status enufft_set_stream(enufft_plan plan, void *cuda_stream);

/*
 * enufft_ems without a plan and without any device allocation (the paper has no counterpart; it
 * is a deployment convenience).  For callers that cannot allocate device memory when they need
 * the selection -- where a cudaMalloc would synchronise the device inside a latency-bound
 * pipeline, where another allocator owns the device memory, or in plug-ins that may not own
 * device memory.  Same arguments and results as enufft_ems for binary32 (complex64) spectra of
 * n_cells cells with P = modes, on the given stream.
 *   - n_cells must not exceed 2048 (the fixed scratch): larger batches return ENUFFT_ERR_ARG
 *     with a message and launch nothing.
 *   - The scratch is one static device array (about 2.2 MB) held by every GPU that loads the
 *     library until the process exits, shared by all calls: calls whose work overlaps on the GPU
 *     (different streams, or different host threads) race on it and must be serialised by the
 *     caller.  Nothing in it needs to start at zero.
 *   - The first call on each device looks up the array's device address (with that device
 *     current); make that first call before any stream capture.  The address is kept for the
 *     life of the process: after cudaDeviceReset (or any other teardown of the device's primary
 *     context) it is stale, so do not call this entry point again in that process.
 */
enufft_status enufft_ems_noalloc(int modes, int64_t n_cells, const void *d_coeffs,
                                 const double *d_mode_weights, int mode_weights_per_cell,
                                 const enufft_ems_params *params, int32_t *d_kstar, int32_t *d_sel,
                                 double *d_retained_power, void *cuda_stream);

/*
 * Self-test of the failure path of the bounded device-side waits (the paper has no counterpart).
 * Launches, on the plan's stream, one block that waits on an mbarrier nothing ever arrives at,
 * giving up after `polls` polls exactly as the tensor-core kernel does when a hand-off never
 * comes: the block latches the timeout bit in the plan's status word and returns, so the context
 * stays usable.  The next enufft_sync_status then returns ENUFFT_ERR_TIMEOUT ("bounded wait
 * expired").  Each poll suspends the waiting warp for at most about 20 us, so the wait ends within
 * about polls * 20 us.  polls must be in [1, 2^17]; a NULL plan or a bad count returns ENUFFT_ERR_ARG.
 */
enufft_status enufft_selftest_wait_timeout(enufft_plan plan, unsigned polls);

/* Synchronise the plan's stream and report (then clear) any latched device-side condition:
 * non-finite samples (skipped), degenerate cell polygons (cells skipped), an edge-frame sample
 * placed at its cell centroid (ENUFFT_ERR_DEVICE for these; the message names each), or an
 * exhausted bounded wait (ENUFFT_ERR_TIMEOUT). */
enufft_status enufft_sync_status(enufft_plan plan);
/* The same call under the name of the plan it reports on. */
enufft_status enufft_plan_sync_status(enufft_plan plan);

/* Human-readable text of the last error on this plan (plan == NULL: of the calling thread). */
const char *enufft_last_error(enufft_plan plan);

/* Read-only plan facts: fine grid size, effective kernel width and shape parameter, how many
 * cells take each execution route (cells_plain: the plain binary32 per-cell path of ENUFFT_FP32
 * plans), and how many kernels one enufft_type1_ems call launches.  Returns ENUFFT_ERR_ARG for a
 * NULL plan or output. */
typedef struct {
    int modes, fine_grid, kernel_width;
    double beta, oversamp_effective;   /* beta: the kernel's shape (ES beta, or KB gamma)       */
    int64_t n_cells, n_points, cells_fused, cells_tensor, cells_large;
    int precision;
    int64_t cells_plain, kernels_per_type1_ems;
    int kernel;                        /* enufft_kernel of the plan                             */
    int frame;                         /* enufft_frame of the plan                              */
    int tc_max_points;                 /* routing threshold in effect (tuned or as given)       */
    int autotuned;                     /* 1 if the routes were tuned at plan creation           */
    int fused_blocks_per_sm;           /* persistent blocks per SM of the fused kernel          */
    int large_tile;                    /* n_f = 256 route: tile side of its sorted spreading
                                          (16, 32 or 64; 0 for other routes)                     */
} enufft_plan_info;
enufft_status enufft_get_plan_info(enufft_plan plan, enufft_plan_info *info);

/*
 * Route tuning (the paper has no counterpart; it is part of running the batched method well on this
 * hardware).  With opts.autotune = 1 the plan times, on synthetic batches drawn from its own cells
 * (each synthetic cell copies the frame of a plan cell, with Q samples spread uniformly over its
 * window), the fused spread/FFT kernel against the tensor-core direct sum at Q = 128, 256, 512,
 * 1024, 2048, 3072, 4096, 6144 (those not above tc_max_points) and keeps as threshold the largest Q
 * at which the direct sum was faster per sample (0 = none); and the fused kernel with one against
 * two resident blocks per SM, at the plan's median cell size.  For n_f = 256 plans it instead times
 * the sorted tile spreading of the plan's first batch (its own cells, synthetic samples) with tiles
 * of 16, 32 and 64 nodes and keeps the fastest: then ladder[] holds the sides tried and ns_fused[]
 * the route's ns per sample with each.  Results are identical either way within the accuracy of
 * each route; only the time changes.
 *   ladder[i], ns_fused[i], ns_tc[i]: the measured ns per sample of each route at Q = ladder[i]
 *   from_cache: 1 if the record was read from opts.tune_cache instead of measured
 */
typedef struct {
    int tc_max_points;
    int fused_blocks_per_sm;
    int n_ladder;
    int ladder[8];
    double ns_fused[8];
    double ns_tc[8];
    int from_cache;
    int large_tile;   /* n_f = 256 plans: the tile side kept (0 in records of other plans) */
} enufft_tuning;
/* The plan's tuning record; ENUFFT_ERR_ARG if the plan was not tuned. */
enufft_status enufft_get_tuning(enufft_plan plan, enufft_tuning *out);
/* Host-only access to a tuning cache file (no GPU needed): look up the record of `key`
 * (ENUFFT_OK, or ENUFFT_ERR_ARG when the file is missing or malformed or has no such key), and
 * store one (the file is created, or rewritten with the key added or replaced; a malformed file is
 * replaced; keys may not contain '"' or '\\'). */
enufft_status enufft_tune_cache_lookup(const char *path, const char *key, enufft_tuning *out);
enufft_status enufft_tune_cache_store(const char *path, const char *key, const enufft_tuning *t);

/*
 * Compute peaks of the current GPU for the roofline terms (the paper has no counterpart; a
 * measurement aid).  Each figure is one launch of fixed work on every SM, timed with CUDA events on
 * cuda_stream (best of three after a warm-up):
 *   fp32_tflops               binary32 FMA, 8 independent chains per thread, 2 blocks of 512 per SM
 *   f16_tflops                tcgen05.mma kind::f16 (binary16 operands in shared memory, binary32
 *                             accumulator in tensor memory), 128 x 256 x 16 per instruction, one
 *                             issuing thread per SM, dense flops 2 M N K per instruction
 *   smem_red_u32_gops         shared-memory 32-bit integer reductions, every lane in its own bank
 *   smem_red_u32_random_gops  the same at random words (bank conflicts as they fall)
 *   smem_red_f32_gops         shared-memory binary32 add reductions, every lane in its own bank
 * (reductions per second over the whole GPU, in units of 1e9).  Allocates and frees two small
 * buffers; synchronises the stream.  ENUFFT_ERR_TIMEOUT if a tensor-core block's bounded wait
 * expired.
 */
typedef struct {
    double fp32_tflops, f16_tflops;
    double smem_red_u32_gops, smem_red_u32_random_gops, smem_red_f32_gops;
    int num_sms;
} enufft_peaks;
enufft_status enufft_probe_peaks(enufft_peaks *out, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* ENUFFT_H */
