/*
 * dd.h -- C-ABI of the GB300 damage-diffusion field library (libdd.so).
 *
 * The library evaluates the cumulative damage field of a scanned Gaussian electron
 * probe (Javadi Rad et al., "Fast Simulation of Damage Diffusion Distribution in
 * STEM", Sec. 2):
 *
 *   phi_i(r,t) = Q0/(4 pi D) [E1(|r-r_i|^2/(2Ds+4D(t-t_i))) - E1(|r-r_i|^2/w0)]
 *       w0 = 2Ds                     while the beam is on,  t_i <= t <= t_i+tau_i  (Eq. 1)
 *       w0 = 2Ds + 4D(t-t_i-tau_i)   after it,              t > t_i+tau_i          (Eq. 2)
 *       with Ds = r_s^2 (r_s = probe sigma) and the ln forms of Eq. 3/4 at r = r_i;
 *   psi(r,t)   = sum over visits i, in visit order, of phi_i(r,t)             (Eq. 5)
 *       (a visit that has not started, t <= t_i, adds nothing).
 *
 * Conventions shared by every entry point:
 *   - Units are SI: metres, seconds, m^2/s, u/s; fields are returned in u/m^2.
 *   - Every call returns a dd_status; on failure dd_last_error() gives a message
 *     (thread-local, valid until the next call on the same thread).  No C++
 *     exception crosses this boundary.
 *   - The caller owns every input and output buffer.  dd_create_scan deep-copies
 *     the arrays it is given.  A dd_scan is immutable after creation and may be
 *     used from several threads; calls that write the same output race.
 *   - Pointers marked "host or device" may point to host memory or to CUDA device
 *     memory of the current device (detected with cudaPointerGetAttributes).
 *     With device inputs and outputs the call only enqueues work on `cuda_stream`
 *     (NULL = the legacy default stream) and returns.  With a host input or output
 *     the call synchronises the stream before it returns (host outputs are then
 *     written), except when a stream other than NULL is given and every host buffer
 *     of the call is page-locked (cudaHostAlloc / cudaHostRegister): then its copies
 *     stay enqueued on `cuda_stream` like its kernels, and the caller synchronises
 *     the stream before reading the outputs or reusing the inputs.
 *   - Device scratch of a call is handed back with an event recorded on its stream
 *     and reused by later calls (at once on the same stream, on another once that
 *     event has completed; up to 8 GiB per device kept); new scratch comes from a
 *     memory pool the library owns per device (freed memory up to 4 GiB stays
 *     mapped).  A scan caches its probe list per device, in blocks that destroyed
 *     scans give back.  Streams are told apart by their handles: a stream destroyed
 *     while calls enqueued on it are still running must not be followed by calls on a
 *     new stream before that work has completed (the new stream can receive the old
 *     handle, and scratch released on the old one would be taken at once).
 */
#ifndef DD_H
#define DD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dd_scan dd_scan;          /* opaque, library-owned */

typedef enum {
    DD_OK = 0,
    DD_EINVAL = -1,     /* an argument is out of range, NULL where not allowed, or not finite */
    DD_ENOMEM = -2,     /* host or device allocation failed */
    DD_ECUDA = -3,      /* a CUDA runtime call failed (message names it) */
    DD_ETIMEOUT = -4,   /* a bounded device wait ran out (status word set by a kernel) */
    DD_ENOTSUP = -5     /* valid request that this library does not implement */
} dd_status;

/* Scan strategies of Sec. 1: raster; alternating (serpentine); interleaved, which
   skips fixed grid points; random; or an explicit list of grid positions. */
typedef enum {
    DD_RASTER = 0,       /* rows in order, each left to right */
    DD_SERPENTINE = 1,   /* even rows left to right, odd rows right to left */
    DD_INTERLEAVED = 2,  /* stride S: S*S passes over the sub-lattices (iy%S, ix%S), in
                            raster order of the sub-lattice, each pass in raster order */
    DD_RANDOM = 3,       /* Fisher-Yates permutation driven by SplitMix64(seed) */
    DD_CUSTOM = 4        /* custom_visit[] lists grid indices in visit order */
} dd_order;

typedef enum {
    DD_FP64 = 0,         /* every step in FP64 */
    DD_MIXED = 1         /* per-pair terms in FP32; per-(visit, snapshot) coefficients,
                            per-block sums and the output in FP64 */
} dd_precision;

/* Problem statement of Sec. 2 (assumptions) and Sec. 1 (scan strategies).
   Probe (ix, iy) sits at (ix * pitch_m, iy * pitch_m); its grid index is iy*nx + ix. */
typedef struct {
    int32_t nx, ny;               /* probe grid, each >= 1, nx*ny <= 2^26 */
    double pitch_m;               /* probe pitch [m], > 0 */
    double sigma_m;               /* Gaussian probe sigma r_s [m], > 0; Ds = sigma^2 */
    double D_m2s;                 /* diffusion coefficient D [m^2/s], > 0 */
    double Q0;                    /* deposition rate [u/s], finite */
    double dwell_s;               /* dwell tau [s], > 0 (also the time unit used inside) */
    double flyback_s;             /* dead time when a raster/serpentine scan changes row, >= 0;
                                     must be 0 for the other orders */
    int32_t order;                /* dd_order */
    int32_t interleave_stride;    /* S >= 1 for DD_INTERLEAVED, ignored otherwise */
    uint64_t seed;                /* seed of the random order / kept subset */
    double keep_fraction;         /* in (0, 1]; < 1 keeps round(f*nx*ny) positions: the first
                                     ones of the seeded permutation (visited in that order for
                                     DD_RANDOM, in the order's own sequence otherwise) */
    const uint8_t *mask;          /* host, nx*ny, row-major; NULL = all; 0 = not visited.
                                     Must be NULL when keep_fraction < 1 or order is CUSTOM */
    const int32_t *custom_visit;  /* host, n_custom grid indices for DD_CUSTOM, NULL otherwise */
    int32_t n_custom;
    const double *dwell_per_visit;/* host, optional per-visit dwell tau_i [s] (Eq. 1/2 allow a
                                     different tau_i per probe); NULL = dwell_s for all */
    double blank_s;               /* beam-blanker travel: dead time [s] before a visit whose
                                     position lies more than one pitch from the previous
                                     visit's (random, interleaved, masked or subsampled scans,
                                     Sec. 1), >= 0; 0 = none */
    double blank_s_per_m;         /* further dead time per metre of such a jump [s/m], >= 0 */
} dd_scan_desc;

/* Build a scan: the visit list in visit order and each visit's start time
   t_k = k*dwell (uniform dwell, no flyback, no blanker travel), otherwise
   t_{k+1} = t_k + tau_k (+ flyback_s when a raster/serpentine scan changes row)
   (+ blank_s + blank_s_per_m * |r_{k+1} - r_k| when that jump is longer than one pitch;
   flyback and travel add up at a row change).  The beam deposits nothing during either
   dead time.  Host-only; touches no GPU.  *out is set to a new scan owned by the caller
   (free with dd_destroy).
   Errors: DD_EINVAL (bad description; *out untouched), DD_ENOMEM. */
dd_status dd_create_scan(const dd_scan_desc *desc, dd_scan **out);

/* Number of visits of the scan. */
dd_status dd_scan_size(const dd_scan *scan, int64_t *n_visits);

/* Copy the visit list out: grid_index[k] (may be NULL), t_start_s[k] and
   dwell_s[k] (each may be NULL), k < n_visits.  Host pointers. */
dd_status dd_scan_visits(const dd_scan *scan, int32_t *grid_index, double *t_start_s,
                         double *dwell_s);

/* Cumulative field psi (Eq. 5) at n_pts points and n_t snapshot times:
     out[it * n_pts + ip] = psi((pts_xy_m[2*ip], pts_xy_m[2*ip+1]), times_s[it])   [u/m^2]
   pts_xy_m: host or device, 2*n_pts doubles (x, y interleaved) [m].
   times_s:  host or device, n_t doubles [s], any order (a device array is copied
             to the host first, which synchronises the stream).
   out:      host or device, n_t*n_pts doubles, row = snapshot.
   n_pts == 0 or n_t == 0 is a no-op.  Times at or before the first visit give 0.
   Errors: DD_EINVAL (NULL scan/buffer with a non-zero size, negative sizes,
   non-finite times, bad precision), DD_ENOMEM, DD_ECUDA. */
dd_status dd_field_at_times(const dd_scan *scan, const double *pts_xy_m, int64_t n_pts,
                            const double *times_s, int64_t n_t, dd_precision prec,
                            double *out, void *cuda_stream);

/* Cumulative field psi (Eq. 5) on a rectilinear grid of evaluation points (the paper's
   simulation grid of pixel side delta_s, Sec. 3): point (c, r) sits at
   (x0_m + c * dx_m, y0_m + r * dy_m) for c < n_cols, r < n_rows (each product and sum
   rounded once in FP64, no fused multiply-add), and
     out[it * n_cols * n_rows + r * n_cols + c] = psi(point (c, r), times_s[it])   [u/m^2]
   -- the result of dd_field_at_times on those points in row-major order, without a point
   buffer.  In FP32-mixed precision the grid lets a tile of 128 columns x 4 rows split the
   low-degree pair terms into column and row factors (fewer exponentials per pair); and on
   grids of at least 64 x 64 points, the visits whose pair terms are on the degree-2 series
   at every point of the grid (the older ones) are summed as a matrix product of those
   factors on the tensor cores (BF16 pieces of the FP32 factors, FP32 accumulation); the
   result then differs from dd_field_at_times by the FP32 rounding, within the same error
   budget.  times_s and out as in dd_field_at_times.  A grid with no columns, rows or
   snapshots is a no-op.
   Errors: DD_EINVAL (NULL scan/buffer, negative sizes, non-finite origin or spacing, more
   than 2^31 points), DD_ENOMEM, DD_ECUDA.  A tensor-core wait that gave up (an
   iteration-limited wait for the MMAs' completion) leaves NaN in the affected points and
   is reported by dd_field_check. */
dd_status dd_field_on_grid(const dd_scan *scan, double x0_m, double y0_m, double dx_m, double dy_m,
                           int64_t n_cols, int64_t n_rows, const double *times_s, int64_t n_t,
                           dd_precision prec, double *out, void *cuda_stream);

/* The split dd_field_on_grid makes in FP32-mixed precision, host-only (no GPU work):
   prefix[it] = the number of leading visits (in visit order) whose pair terms at snapshot
   times_s[it] (host array) are summed on the tensor cores, and prefix_deg2[it] (NULL: not
   wanted) how many of them in the degree-2 form; the visits after prefix[it] go to the
   CUDA-core tile kernel.  A visit qualifies when its pair term is on the degree-2 (degree-4)
   series at every point of the grid: h = rho^2 dq <= 0.04 (0.33) for rho^2 up to the
   largest squared distance between the grid's box and the visits' box, with dq bounded
   through the scan's longest dwell (dq <= c / ((w1 - c) w1), c = 4 D tau_max, at
   w1 = 2 sigma^2 + 4 D (t - t_i)), so the qualifying visits are those started by
   t - dT*: prefixes.  0 for grids smaller than 64 x 64 points and for snapshots with no
   qualifying visit; the degree-4 band is left out where its coefficients of (rho^2)^4
   would leave the FP32 normal range, and the path falls back to 0 everywhere if the
   split's partial sums would exceed its 1 GiB workspace budget.
   Errors: DD_EINVAL (NULL scan or buffers, negative sizes, non-finite grid or times,
   device arrays). */
dd_status dd_field_grid_split(const dd_scan *scan, double x0_m, double y0_m, double dx_m, double dy_m,
                              int64_t n_cols, int64_t n_rows, const double *times_s, int64_t n_t,
                              int64_t *prefix, int64_t *prefix_deg2);

/* Synchronise the device and return DD_ETIMEOUT (clearing the flag) if a tensor-core
   contraction of dd_field_on_grid gave up waiting for its MMAs since the last check,
   DD_OK otherwise. */
dd_status dd_field_check(void);

/* Dwell-start dose of every visit: the field at the probe's own position when
   its dwell starts, from the visits before it,
     out[j] = psi_{j-1}(r_j, t_j) = sum_{i<j} phi_i(r_j, t_j)   (Eq. 5 at r_j, t_j)
   in visit order.  out: host or device, n_visits doubles.  With a uniform dwell and no
   flyback (t_k = k*tau) the pair coefficients depend on the lag j - i only and come
   from a table of n_visits records; otherwise (per-visit dwells, flyback) they are
   formed per pair in FP64, which costs more per pair.
   Errors: DD_EINVAL, DD_ENOMEM, DD_ECUDA. */
dd_status dd_per_probe_dose(const dd_scan *scan, dd_precision prec, double *out,
                            void *cuda_stream);

/* Dwell-start dose of the visits j0 <= j < j1 only (0 <= j0 <= j1 <= n_visits):
     out[j - j0] = psi_{j-1}(r_j, t_j)   (as dd_per_probe_dose, Eq. 5 at r_j, t_j)
   The paper partitions the sum into independent tasks over subsets of the probe positions
   (Sec. 3); this is that partition for the dose, so that several GPUs (or processes)
   can each evaluate a range of targets.  Visit j's dose costs about j pair terms, so equal
   work needs ranges that shrink towards the end of the scan.  out: host or device,
   j1 - j0 doubles; j1 == j0 is a no-op.  Results agree with dd_per_probe_dose within the
   precision's rounding (the lag blocks are sized for the range, so the summation order
   may differ).  Errors: DD_EINVAL, DD_ENOMEM, DD_ECUDA. */
dd_status dd_per_probe_dose_range(const dd_scan *scan, dd_precision prec, int64_t j0, int64_t j1,
                                  double *out, void *cuda_stream);

/* Allocation-free variant of dd_per_probe_dose (the paper has no counterpart: this
   entry point exists for callers that cannot allocate device memory while they run,
   e.g. an acquisition loop that reserves its whole GPU memory budget before the scan
   starts, or a host whose device allocator belongs to another framework).  Same
   result as dd_per_probe_dose.  It calls no device allocator: its scratch lives in
   one file-scope __device__ array of 8 MiB, which every GPU that loads the library
   holds until the process exits, so scans of at most 16384 visits are accepted
   (larger ones: DD_EINVAL with a message).  out must be device memory (else
   DD_EINVAL).  The first call on each device looks up the array's device address
   (cudaGetSymbolAddress); make that first call before any stream capture.  All calls
   share the array, which keeps the previous call's contents: every byte a kernel
   reads is written earlier in the same call, and calls that overlap on the GPU (two
   streams, or two host threads) race on it.  The call synchronises `cuda_stream`
   before returning.  The scan must stay alive until the call returns.
   Errors: DD_EINVAL, DD_ENOTSUP (non-uniform dwell or flyback), DD_ECUDA. */
dd_status dd_per_probe_dose_noalloc(const dd_scan *scan, dd_precision prec, double *out,
                                    void *cuda_stream);

/* Many independent scans in one persistent launch (the paper's task partition
   over probe subsets, Sec. 3, applied across scans).  Scan k is evaluated at
   points pts_xy_m[2*pt_offsets[k] .. 2*pt_offsets[k+1]) and the single time
   times_s[k]; its field goes to out[pt_offsets[k] .. pt_offsets[k+1]).
   scans: host array of n_scans handles.  pt_offsets: host, n_scans+1 entries,
   non-decreasing, pt_offsets[0] == 0.  times_s: host, n_scans.  pts_xy_m and out:
   host or device.  Work items are cost-sorted and claimed by an atomic counter.
   Errors: DD_EINVAL, DD_ENOMEM, DD_ECUDA. */
dd_status dd_field_batch(const dd_scan *const *scans, int32_t n_scans, const int64_t *pt_offsets,
                         const double *pts_xy_m, const double *times_s, dd_precision prec,
                         double *out, void *cuda_stream);

/* Reusable plan of a batch (same arguments as dd_field_batch without the buffers):
   validates, builds the cost-sorted work list, uploads the tables and allocates its
   device buffers (cudaMalloc; synchronous).  The scans must outlive the plan.
   dd_batch_run evaluates it: the launch sequence is captured into a CUDA graph on
   the first run (and again when the point/output pointers or the kernel variant
   change) and replayed with cudaGraphLaunch on `cuda_stream`; with device buffers the
   call only enqueues.  pts_xy_m/out: host or device, as in dd_field_batch.
   dd_batch_tune times each kernel variant once on device points pts_xy_m, keeps the
   fastest for this plan and records it for (GPU, precision, batch size) in-process and
   in the JSON file named by the environment variable DD_TUNE_CACHE, if set; plans
   created later with the same key start from the recorded variant.
   dd_batch_info: work items, causal pair-terms per run and the kernel variant.
   dd_batch_destroy synchronises the device and frees the plan (NULL is a no-op). */
typedef struct dd_batch dd_batch;
/* dd_batch_create_grid: the same plan with each scan evaluated on a rectilinear grid of
   points instead of a point list: grid_xy[4k..4k+3] = (x0, y0, dx, dy) [m] and
   grid_wh[2k], grid_wh[2k+1] = (columns W_k, rows H_k) of scan k; point (c, r) of scan k
   sits at (x0 + c dx, y0 + r dy) (one product and one sum each, no fused multiply-add) and
   its field goes to out[off_k + r W_k + c], off_k = sum over the earlier scans of W H.
   dd_batch_run and dd_batch_tune then take pts_xy_m = NULL.  In FP32-mixed precision the
   grid lets tiles of 32 x 32 points split the low-degree pair terms into column and row
   factors (as dd_field_on_grid does), and for grids of at least 64 x 64 points each scan's
   visits on the degree-2 (then degree-4) series at every point of its grid are summed as
   matrix products on the tensor cores, the prefixes dd_field_grid_split reports, with the
   same completion waits and NaN-on-timeout rule as dd_field_on_grid (dd_field_check); the
   result differs from the point-list plan by FP32 rounding only.  Errors: DD_EINVAL (sizes,
   non-finite origin or spacing, more than 2^31 points), DD_ENOMEM, DD_ECUDA. */
dd_status dd_batch_create_grid(const dd_scan *const *scans, int32_t n_scans, const double *grid_xy,
                               const int64_t *grid_wh, const double *times_s, dd_precision prec,
                               dd_batch **out);
dd_status dd_batch_create(const dd_scan *const *scans, int32_t n_scans, const int64_t *pt_offsets,
                          const double *times_s, dd_precision prec, dd_batch **out);
dd_status dd_batch_run(dd_batch *batch, const double *pts_xy_m, double *out, void *cuda_stream);
dd_status dd_batch_tune(dd_batch *batch, const double *pts_xy_m, int32_t *chosen_variant);
dd_status dd_batch_info(const dd_batch *batch, int64_t *n_items, int64_t *pair_terms,
                        int32_t *variant);
void dd_batch_destroy(dd_batch *batch);

/* Free a scan and its per-device caches (device caches are freed on their own
   devices).  NULL, or a handle that was already destroyed, is a no-op.  Blocks until the
   work already enqueued by calls on this scan is done: on each stream that such a call
   used, up to that call's last launch or copy (other work in flight is not waited for),
   or the whole device once a batch plan was built on the scan (a plan may run on any
   stream).  The handle must not be passed to a call made after (or during) dd_destroy.
   Testing hook: with the environment variable DD_FAULT=alloc, the field workspace
   allocation reports cudaErrorMemoryAllocation (the call returns DD_ENOMEM). */
void dd_destroy(dd_scan *scan);

/* Message of the last failed call on this thread ("" if none). */
const char *dd_last_error(void);

/* ---- Learned surrogate of the field map (no counterpart in the paper) ----------------
   Building blocks of a small convolutional network that maps input planes of a scan
   (visit-time map, visited mask, standardised log D and log dwell) to the final
   log-damage map; it is trained on fields from the batched exact path, which also
   serves as its fallback.  All tensors are device memory, NHWC, BF16 unless noted;
   weights are [cout][3*3][cin] BF16 (tap = ky*3 + kx).  W must be a multiple of 64;
   (cin, cout) in {(16,32), (32,32), (32,16), (16,16)}.  Calls enqueue on cuda_stream.

   dd_sur_conv3x3: 3x3 convolution with dilation d in 1..32 (tap (ky, kx) reads the input
   at (y + (ky-1) d, x + (kx-1) d)), zero "same" padding, implicit GEMM on the tensor
   cores (BF16 x BF16 -> FP32; tcgen05.mma with the accumulator in tensor memory when W
   is a multiple of 128, mma.sync otherwise).  epilogue 0: out = bf16(relu(z + bias)) [B,H,W,cout];
   1: out = float(z + bias) of channel 0 only [B,H,W]; 2: out = bf16(z * (mask > 0))
   with mask [B,H,W,cout] (the data gradient through a ReLU, using the flipped weights
   that dd_sur_adam writes; bias unused).
   dd_sur_wgrad: grad[cout*9*cin + cout] (FP32) = weight gradient [cout][9][cin] followed
   by the bias gradient of the dilation-d convolution, from layer input x [B,H,W,cin] and output gradient dz
   [B,H,W,cout]; part (FP32, part_floats >= 608 * (cout*9*cin + cout)) holds per-CTA
   partial sums, reduced in a fixed order.
   dd_sur_mse: loss_sum[0] (FP64, device) = sum (pred - target)^2 over n elements, and
   dz [n][16] BF16 = (2 (pred - target) / n, 0, ..., 0); block_sums: ceil(n/256) doubles.
   dd_sur_adam: Adam (bias-corrected, step >= 1) on FP32 param with grad, moments m, v;
   when w_bf16 is given also writes the BF16 copy and the flipped copy [cin][8-tap][cout].
   dd_sur_planes: x [B,H,W,16] BF16 from tmap [B,H,W] (visit time / total scan time,
   < 0 where not visited) and scal [B][2] (standardised log D, log dwell).
   dd_sur_wmse: the same with per-element weights weight[n] (FP32): loss_sum[0] =
   sum w (pred - target)^2, dz = (2 w (pred - target) / n, 0, ..., 0).
   dd_sur_weights: w [n_maps*hw] FP32 = alpha hw f_p^2 / sum_q f_q^2 + (1 - alpha) per map,
   f = 10^(target sigma + mu) from normalised targets (alpha in [0, 1]): the squared log
   error weighted so, summed over a map and divided by hw, approximates (relative L2 error of
   the linear map / ln 10)^2, the surrogate's accuracy measure.
   dd_sur_targets: out [n_maps*hw] FP32 = (log10(max(f, peak * 10^floor_rel_log10)) - mu)
   / sigma with f = psi*scale[map] and peak = max of f over the map (floor_rel_log10 < 0):
   the network's normalised target from exact fields psi [n_maps*hw] (u/m^2, FP64) and
   per-map scale[] = 4 pi D / Q0 (the dimensionless field).
   dd_sur_fields: psi [n_maps*hw] (u/m^2, FP64) = 10^(pred*sigma + mu) / scale[map].
   dd_sur_spot_error: err[m] = relative L2 error over k spot points of map m between the
   field of pred [n_maps][hw] plus add [n_maps][hw] (u/m^2, FP64; an exactly computed part
   of the field, or NULL) and exact [n_maps][k] (u/m^2) at canvas indices idx [n_maps][k].
   dd_sur_check: synchronises the device and returns DD_ETIMEOUT (clearing the flag) if a
   tensor-memory convolution since the last check gave up waiting for its MMAs (an
   iteration-limited wait; its output is then not written), DD_OK otherwise. */
dd_status dd_sur_conv3x3(const void *in, const void *w, const float *bias, const void *mask, void *out,
                         int32_t B, int32_t H, int32_t W, int32_t cin, int32_t cout, int32_t dilation,
                         int32_t epilogue, void *cuda_stream);
dd_status dd_sur_wgrad(const void *x, const void *dz, int32_t B, int32_t H, int32_t W, int32_t cin,
                       int32_t cout, int32_t dilation, float *part, int64_t part_floats, float *grad,
                       void *cuda_stream);
dd_status dd_sur_mse(const float *pred, const float *target, int64_t n, void *dz, double *block_sums,
                     double *loss_sum, void *cuda_stream);
dd_status dd_sur_adam(float *param, const float *grad, float *m, float *v, int64_t n, float lr,
                      float beta1, float beta2, float eps, int32_t step, void *w_bf16,
                      void *w_flip_bf16, int32_t cin, int32_t cout, void *cuda_stream);
dd_status dd_sur_planes(const float *tmap, const float *scal, int32_t B, int32_t H, int32_t W, void *x,
                        void *cuda_stream);
/* dd_sur_planes_bg: the planes of dd_sur_planes from scal3 [B][3] (standardised log D,
   standardised log dwell, kappa = D dwell / pitch^2), tmap holding 1 / age (age in dwells
   at the end of the scan, 1 for the last visit), plus channel 4: the own term of each
   background visit (age > k_exact) at its position, ln(w1/w0) of Eq. 3/4 with
   w1 = 2 s + 4 kappa age, w0 = 2 s + 4 kappa (age - 1), s = probe sigma^2 / pitch^2, as
   (log10 - mu) / sigma, 0 elsewhere; channel 5: 1 on those visits; channels 6..15 zero. */
dd_status dd_sur_planes_bg(const float *tmap, const float *scal3, float s_dim, int32_t k_exact, float mu,
                           float sigma, int32_t B, int32_t H, int32_t W, void *x, void *cuda_stream);
dd_status dd_sur_wmse(const float *pred, const float *target, const float *weight, int64_t n, void *dz,
                      double *block_sums, double *loss_sum, void *cuda_stream);
dd_status dd_sur_weights(const float *target, int64_t n_maps, int64_t hw, float mu, float sigma, float alpha,
                         float *w, void *cuda_stream);
dd_status dd_sur_targets(const double *psi, const double *scale, int64_t n_maps, int64_t hw,
                         double floor_rel_log10, float mu, float sigma, float *out, void *cuda_stream);
dd_status dd_sur_fields(const float *pred, const double *scale, int64_t n_maps, int64_t hw, float mu,
                        float sigma, double *psi, void *cuda_stream);
dd_status dd_sur_spot_error(const float *pred, const int32_t *idx, const double *exact,
                            const double *scale, const double *add, int32_t n_maps, int32_t hw, int32_t k,
                            float mu, float sigma, double *err, void *cuda_stream);
dd_status dd_sur_check(void);

/* Tracing (no counterpart in the paper): per-kernel device time of this library's
   own launches.  While enabled, each launch is bracketed by two CUDA events on its
   stream (do not enable it while a stream is being captured into a graph).
   dd_profile_read waits for the recorded events and fills up to max_entries rows:
   names[64*k] is the NUL-terminated kernel name (at most 63 chars), launches[k]
   the count and total_ms[k] the summed device time since the last reset;
   *n_entries receives the number of distinct kernels.  Host pointers. */
dd_status dd_profile_enable(int32_t on);
dd_status dd_profile_reset(void);
dd_status dd_profile_read(char *names, int64_t *launches, double *total_ms, int32_t max_entries,
                          int32_t *n_entries);

/* Library version string. */
const char *dd_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DD_H */
