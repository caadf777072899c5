/*
 * rick.h -- C ABI of librick, a GB300 (sm_103a) w-stacking imager: the hot
 * path of RICK (arXiv 2504.00959) -- convolutional gridding onto w-planes,
 * a per-plane 2D inverse FFT, and the w-term phase-screen correction that
 * stacks the planes into one dirty image.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Coordinates u, v, w are in wavelengths (float32 arrays of length nvis).
 *   Visibilities are complex64: interleaved (re, im) float32 pairs, 2*nvis
 *   floats.  Weights are float32 (NULL = unit weights).
 * - Grid: n x n cells per w-plane, cell j <-> u = (j - n/2) * du with
 *   du = 1 / (n * pixel_rad); planes are row-major [v cell][u cell].
 * - Image: n x n pixels, row-major [y][x]; pixel (x, y) <-> l = (x - n/2) *
 *   pixel_rad, m = (y - n/2) * pixel_rad; the phase centre is pixel (n/2, n/2).
 * - w-planes: nw uniform bins over [w_min, w_max]; a measurement goes to the
 *   plane floor((w - w_min) / dw) clamped to [0, nw-1] (the closest plane,
 *   Sec. 2.1), or with rick_params.w_support > 1 to the planes of its
 *   w-footprint (Eq. 3's kernel in w); plane k has centre w_k = w_min +
 *   (k + 1/2) dw.
 * - Kernel footprint: cells f .. f+S-1 on each axis, f = floor(p - S/2) + 1,
 *   p = u / du + n/2; taps normalised to sum 1 per axis.  A measurement whose
 *   footprint leaves the grid, or with a non-finite coordinate, weight or
 *   value, is dropped and counted (not an error).
 * - Device pointers unless a call says "host".  All work is enqueued on the
 *   handle's stream (rick_set_stream); calls return once the work is
 *   enqueued, except where a call says it synchronises.  Caller-owned buffers
 *   must stay valid until that work has run.  The library owns only its
 *   internal workspace, plans and handles.
 * - Every call returns a rick_status; RICK_OK (0) on success.  No exceptions
 *   cross the ABI and no device trap is used.  rick_last_error(h) gives a
 *   message for the last failure on h.
 * - A handle is not thread-safe: one host thread at a time per handle.
 */
#ifndef RICK_H
#define RICK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t rick_status;
#define RICK_OK 0
#define RICK_ERR_ARG 1      /* invalid argument (null pointer, bad size, bad parameter) */
#define RICK_ERR_OOM 2      /* device memory would not fit; nothing was launched */
#define RICK_ERR_CUDA 3     /* a CUDA runtime call failed */
#define RICK_ERR_CUFFT 4    /* a cuFFT call failed */
#define RICK_ERR_TIMEOUT 5  /* a bounded device wait ran out */
#define RICK_ERR_STATE 6    /* call out of order (e.g. degrid before any grid) */

#define RICK_KERNEL_GAUSS 0 /* exp(-x^2 / (2 sigma^2)), kernel_param = sigma in cells (0: S/6) */
#define RICK_KERNEL_KB 1    /* I0(beta sqrt(1 - (2x/S)^2)), kernel_param = beta (0: 2.34 S) */

#define RICK_GRID_CORRECT 1u   /* divide the image by the kernel's Fourier transform (taper) */
#define RICK_REAL_IMAGE 2u     /* output Re(image) as float[n*n]; else complex float[2*n*n] */
#define RICK_APPLY_N 4u        /* multiply the image by n = sqrt(1 - l^2 - m^2) (Eq. 1 LHS) */
#define RICK_UNIFORM_WEIGHT 8u /* weight / (gridded measurements sharing the nearest cell) */
#define RICK_HERMITIAN_FOLD 32u /* real images only (with RICK_REAL_IMAGE): a measurement with
                                  w < 0 is imaged as its Hermitian mirror (-u, -v, -w, conj V),
                                  which leaves Re(image) unchanged, so the w-planes need only
                                  cover the folded range (w_min, w_max >= 0 typically: half the
                                  planes for the same plane spacing) */
#define RICK_FFT_2D 64u         /* transform the planes with cuFFT's 2D plan and stack them in a
                                  separate pass, also where the library would otherwise split
                                  the column transform and fuse its last factor with the
                                  w-screen and the stack (single images with n >= 2048) */
#define RICK_FFT_SPLIT 128u     /* the split transform for any power-of-two n in [64, 16384]
                                  (single images; the default from n = 2048 on, for tests and
                                  measurement below).  Not with RICK_FFT_2D.  Either way the
                                  result is the same up to rounding */

/* Problem statement of Sec. 2.1: grid size, pixel scale, w-planes, kernel.
 * n: grid side, even, >= 2*support.  nw >= 1.  w_max > w_min when nw > 1.
 * support: kernel support S in cells, 1..16.  plane_group: w-planes resident
 * in HBM at once (0 = as many as fit).  tile: uv tile side of the gridder,
 * 16, 32 or 64 (0 = automatic); must be >= support.  w_support: planes each
 * measurement is gridded onto, Eq. 3's kernel in w (0 or 1: the nearest
 * plane, Sec. 2.1; 2..16, at most nw: the sw planes fk .. fk+sw-1 around
 * its continuous plane coordinate pw = (w - w_min)/dw - 1/2, fk =
 * floor(pw - sw/2) + 1, with normalised taps of the kernel family of u and v
 * (support sw, sigma sw/6 or beta 2.34 sw), and the image divided by that
 * kernel's Fourier transform at dw (n - 1)).  Taps on planes outside
 * 0 .. nw-1 are dropped, so [w_min, w_max] should extend sw/2 plane widths
 * beyond the measurements' w.  The planes must sample the w-term: creation
 * fails (RICK_ERR_ARG) when the correction falls below 1e-2 anywhere in the
 * image (dw (1 - n) at the corners beyond the w-kernel's passband; add
 * planes).  Not available for batched handles. */
typedef struct rick_params {
    int32_t n;
    int32_t nw;
    double pixel_rad;
    double w_min;
    double w_max;
    int32_t kernel;
    int32_t support;
    double kernel_param;
    int32_t plane_group;
    int32_t tile;
    uint32_t flags;
    int32_t w_support;
} rick_params;

typedef struct rick_stats {
    int64_t n_gridded;      /* measurements gridded since the last reset */
    int64_t n_dropped;      /* measurements dropped since the last reset */
    int64_t n_entries;      /* (measurement, tile) entries after footprint splitting */
    double sum_weights;     /* sum of the effective weights gridded */
    int32_t plane_group;    /* planes resident per group */
    int32_t tile;           /* uv tile side in use */
    int64_t workspace_bytes;/* device bytes the handle holds */
} rick_stats;

typedef struct rick_imager* rick_handle;

/* Fill *p with defaults (Gaussian, support 7, grid correction + real image). */
rick_status rick_params_default(rick_params* p);

/* Create an imager for the problem *p on the current CUDA device: plans, taper,
 * plane buffers.  Fails with RICK_ERR_OOM (and allocates nothing) when the
 * plane group does not fit in free device memory. *out receives the handle. */
rick_status rick_create(const rick_params* p, rick_handle* out);

/* Release every resource of h (synchronises its stream).  NULL is a no-op. */
rick_status rick_destroy(rick_handle h);

/* Enqueue all later work of h on `cuda_stream` (a cudaStream_t; NULL = legacy
 * default stream). */
rick_status rick_set_stream(rick_handle h, void* cuda_stream);

/* Device bytes rick_create + one rick_grid of max_vis measurements need. */
rick_status rick_workspace_size(const rick_params* p, int64_t max_vis, size_t* bytes);

/* Forget all gridded measurements, weight sums, counters and the uniform-
 * weighting density. */
rick_status rick_reset(rick_handle h);

/* Step 1-2 of the workflow (Sec. 2.1) for one chunk of measurements: place
 * each on its w-plane and footprint, bin by (w-plane, uv tile) with a
 * counting sort, and store the weighted visibility with its continuous cell
 * coordinates.  Calls accumulate (chunks, Sec. 2.2); the planes themselves
 * are gridded (Eq. 3) inside rick_fft_and_stack, so the inputs may be freed
 * as soon as this call's work has run.  vis: float[2*nvis]; u, v, w:
 * float[nvis]; weights: float[nvis] or NULL.  nvis >= 0. */
rick_status rick_grid(rick_handle h, const float* vis, const float* u, const float* v,
                      const float* w, const float* weights, int64_t nvis);

/* Uniform weighting over several chunks: add the nearest-cell counts of one
 * chunk to the density grid before the first rick_grid of the batch.  With a
 * single chunk rick_grid computes the density itself. */
rick_status rick_add_density(rick_handle h, const float* vis, const float* u, const float* v,
                             const float* w, const float* weights, int64_t nvis);

/* Steps 2-4 of the workflow for everything gridded since the last reset:
 * for each plane group, grid the planes (Eq. 3), inverse-FFT each plane
 * (cuFFT, unnormalised, exponent +), multiply by the phase screen
 * exp(+2 pi i w_k (n-1)) and sum over planes (Eq. 1); then divide by the
 * weight sum and, per flags, by the taper and times n.  image: float[n*n]
 * (RICK_REAL_IMAGE) or float[2*n*n] complex, fully overwritten.  For
 * power-of-two n from 2048 to 16384 (or with RICK_FFT_SPLIT) the column
 * transform is split, n = 16 * (n / 16): cuFFT transforms the rows, one
 * library kernel the first (n / 16-point) column factor of every plane of
 * the group in place, and one kernel the last 16-point column factor
 * together with the screen and the sum, reading each plane once more;
 * otherwise cuFFT's 2D plan and a separate screen-and-sum pass
 * (RICK_FFT_2D). */
rick_status rick_fft_and_stack(rick_handle h, float* image);

/* Eq. 3 alone: the gridded planes k0 .. k0+nk-1 as complex float
 * [nk][n][n] (no fftshift sign), fully overwritten. */
rick_status rick_grid_planes(rick_handle h, int32_t k0, int32_t nk, float* planes);

/* Adjoint of the measurement-to-image map (degridding; not in the paper):
 * vis_grad = A^H image_grad, where A maps visibilities to the image
 * rick_fft_and_stack would produce for the measurements (u, v, w, weights)
 * with the current weight sum and density.  image_grad: float[n*n]
 * (RICK_REAL_IMAGE) or float[2*n*n]; vis_grad: float[2*nvis] (complex),
 * overwritten; dropped measurements get 0.  Planes are recomputed from
 * image_grad per plane group (phase screen conjugate, forward FFT, gather
 * with the same taps).  RICK_ERR_STATE when nothing has been gridded. */
rick_status rick_degrid(rick_handle h, const float* image_grad, const float* u, const float* v,
                        const float* w, const float* weights, int64_t nvis, float* vis_grad);

/* Model visibilities from a model image (prediction by degridding; the
 * paper has no counterpart): vis[i] = the measurement equation (Eq. 2 with
 * the image in place of I/n) sum_{x,y} model(x,y) exp(-2 pi i (u l + v m +
 * w (n-1))), evaluated the w-stacking way: model / taper (RICK_GRID_CORRECT)
 * x n (RICK_APPLY_N), conjugate w-screen per plane, forward FFT, gather with
 * the gridding taps.  It is the adjoint of the unweighted, unnormalised
 * imaging map (rick_degrid with unit weights, times the weight sum); weights
 * and uniform weighting play no part.  model: float[n*n] (RICK_REAL_IMAGE)
 * or float[2*n*n]; vis: float[2*nvis] (complex), overwritten; measurements
 * whose footprint leaves the grid get 0.  Needs no forward pass. */
rick_status rick_predict(rick_handle h, const float* model, const float* u, const float* v,
                         const float* w, int64_t nvis, float* vis);

/* End to end with HOST buffers: copy the inputs to the device, reset, grid,
 * fft_and_stack, copy the image back to image_host, synchronise.  Host
 * arrays as in rick_grid / rick_fft_and_stack (pinned memory is faster). */
rick_status rick_image_host(rick_handle h, const float* vis_host, const float* u_host,
                            const float* v_host, const float* w_host,
                            const float* weights_host, int64_t nvis, float* image_host);

/* Pipelined form of rick_image_host for a stream of images (the paper's
 * chunk loop reads the next data while it images, Sec. 2.2): enqueues the
 * upload of the inputs, the imaging and the download of the image, and
 * returns without waiting.  Uploads and downloads run on the handle's own
 * copy streams into two device slots, ordered against the handle's stream
 * by events, so image i's compute overlaps the upload of image i+1 and the
 * download of image i-1.  Host arrays must stay valid and unmodified, and
 * image_host must not be read, until rick_synchronize; they should be
 * pinned (pageable memory makes the copies synchronous).  Same arguments,
 * layouts and errors as rick_image_host. */
rick_status rick_image_host_async(rick_handle h, const float* vis_host, const float* u_host,
                                  const float* v_host, const float* w_host,
                                  const float* weights_host, int64_t nvis, float* image_host);

/* Wait for everything enqueued on the handle (its stream and copy streams). */
rick_status rick_synchronize(rick_handle h);

/* Batched multi-channel imaging (not in the paper; it repeats the chunk loop
 * of Sec. 2.2 over frequency channels in one pass): nchan channels share n,
 * pixel_rad, the kernel and the w-plane count p->nw, each with its own
 * w-range [w_min[c], w_max[c]] (host arrays).  Channel c owns w-planes
 * c*nw .. (c+1)*nw-1 of one plane stack; all channels are sorted, gridded,
 * transformed (one launch of each transform kernel per plane group) and
 * stacked together.
 * Uniform weighting is not available here.  Only rick_image_batch,
 * rick_set_stream, rick_get_stats, rick_set_timing / rick_get_timing and
 * rick_destroy apply to a batched handle. */
rick_status rick_create_batch(const rick_params* p, int32_t nchan, const double* w_min, const double* w_max,
                              rick_handle* out);
/* (Batched handles transform their plane groups like single images from
 * n = 1024 on -- cuFFT's rows, the library's first column factor, and one
 * launch of the last column factor fused with every channel's w-screen and
 * stack -- and with cuFFT's 2D plan and a separate stack per channel below,
 * or with RICK_FFT_2D.  Hermitian fold works per channel; each channel's
 * w-range is then its folded one.) */

/* One dirty image per channel: channel c's measurements are entries
 * chan_offsets[c] .. chan_offsets[c+1]-1 (host array of nchan+1, starting at
 * 0, non-decreasing) of vis / u / v / w / weights (device, as rick_grid).
 * images: float[nchan][n*n] (RICK_REAL_IMAGE) or float[nchan][2*n*n],
 * overwritten.  With use_graph != 0 the whole step is captured into a CUDA
 * graph on the first call and replayed by later calls with the same pointers
 * and offsets (needs a non-default stream, rick_set_stream); the entry
 * buffers are persistent and grow outside the capture.  With two or more
 * plane groups (plane_group smaller than nchan * nw) and room for a second
 * plane buffer, the groups are pipelined: group g + 1 is gridded on the
 * handle's stream while group g is transformed and stacked on a second
 * stream of the handle (event-ordered; joined before the call returns its
 * work to the handle's stream).  With phase timing on, groups run one by
 * one. */
rick_status rick_image_batch(rick_handle h, const float* vis, const float* u, const float* v, const float* w,
                             const float* weights, const int64_t* chan_offsets, float* images, int32_t use_graph);

/* Autotuner for batched imaging: times rick_image_batch of the given data
 * (the median of three steps after one untimed step) for every tile side
 * (16, 32, 64, at least the support) and plane group (all channels, half, a
 * quarter of them), then, on the fastest of those, the measurements per
 * block of the sort kernels (rick_set_prep_blocks: 8 -- the default, 0 --
 * against 4, 16 and 32 blocks per SM), and returns the fastest in *tile_out,
 * *plane_group_out and *prep_blocks_out (may be NULL; 0 = the default), the
 * device time in *ms_out (may be NULL).  When the environment variable
 * RICK_AUTOTUNE_CACHE names a file, results are looked up there first and
 * appended after tuning (key: the device's name and SM count, this build of
 * the library, n, nw, nchan, support, kernel, flags, log2 of the
 * measurement count). */
rick_status rick_autotune_batch(const rick_params* p, int32_t nchan, const double* w_min, const double* w_max,
                                const float* vis, const float* u, const float* v, const float* w,
                                const float* weights, const int64_t* chan_offsets, int32_t* tile_out,
                                int32_t* plane_group_out, int32_t* prep_blocks_out, double* ms_out);

/* Blocks per SM of the sort kernels (placement + counting sort) of this
 * handle, i.e. how many measurements each block takes: M / (SMs x
 * blocks_per_sm); 0 = the default 8, at most 64.  A batched handle re-captures
 * its graph on the next call.  RICK_ERR_ARG outside [0, 64]. */
rick_status rick_set_prep_blocks(rick_handle h, int32_t blocks_per_sm);

/* Eq. 3 alone for one set of measurements, into caller-provided planes,
 * WITHOUT allocating any device memory.  The paper has no counterpart.  It is
 * for callers that cannot call cudaMalloc: code inside a framework that owns
 * the whole device heap through its own allocator, real-time loops that
 * forbid allocation after start-up.  No handle is needed.  planes: complex float [nw][n][n] (no fftshift sign),
 * fully overwritten -- the same result as rick_create + rick_grid +
 * rick_grid_planes(0, nw).  The working memory is one fixed 64 MiB array in
 * the library's static device data.  Under CUDA's default lazy module
 * loading that array is committed on a device at this function's first call
 * there (the first cudaGetSymbolAddress loads its module), not when the
 * library is loaded, and stays until the process exits; so make the first
 * call before a framework claims the rest of the device heap.  What a call needs -- counters, kernel-tap
 * polynomials, the uint32 tile counters (nw * ceil(n/tile)^2 of them, each
 * padded to up to 32 words while the padded array stays within 2^16 words)
 * and the tile offsets (nw * ceil(n/tile)^2 + 1 words), the scan totals, n*n uint32 of density with RICK_UNIFORM_WEIGHT,
 * and 64 bytes per measurement (16 when support is 1), each piece 256-byte
 * aligned -- must fit in those 64 MiB; otherwise RICK_ERR_ARG before any
 * launch, with the reason written to err (err_len bytes; err may be NULL).
 * All calls on a device share the array and it keeps the last call's
 * contents, so calls whose GPU work overlaps race: the caller must order
 * them.  The first call on a device, and the first for each kernel
 * configuration, looks up the array's device address and fits the kernel
 * taps, synchronising cuda_stream once; make that first call before any
 * stream capture.  Work goes to cuda_stream (a cudaStream_t, NULL = legacy
 * default stream). */
rick_status rick_grid_planes_static(const rick_params* p, const float* vis, const float* u,
                                    const float* v, const float* w, const float* weights,
                                    int64_t nvis, float* planes, void* cuda_stream, char* err,
                                    size_t err_len);

/* Sharding one image over several GPUs (the paper reduces the gridded
 * w-planes of its sectors across ranks, Sec. 2.2; here each rank finishes its
 * share of the image and the ranks sum images).  Every step of imaging is
 * linear in the planes and in the measurements, and the finalisation (sign,
 * 1 / weight sum, taper, n) is per pixel, so images of disjoint shares made
 * with the same weight sum add up to the image of everything.
 *
 * rick_set_plane_range: this handle grids, transforms and stacks only the
 * w-planes k0 .. k1-1 (0 <= k0 < k1 <= nw; the default is all of them); every
 * measurement is still placed, weighted (uniform weighting counts all) and
 * counted in the weight sum, so ranks that each see all measurements and
 * take disjoint plane ranges produce images that sum to the full image.
 * rick_degrid then covers the same planes (its gradients sum likewise).
 * Call it after rick_create or rick_reset, before rick_grid (RICK_ERR_STATE
 * otherwise).  Not for batched handles. */
rick_status rick_set_plane_range(rick_handle h, int32_t k0, int32_t k1);

/* rick_set_weight_sum: normalise images (and the adjoint) by sum_w instead
 * of the handle's own weight sum -- for ranks that each grid a share of the
 * measurements: the caller sums the ranks' weight sums (rick_get_stats)
 * and sets the total on every rank before rick_fft_and_stack.  sum_w < 0
 * returns to the handle's own sum.  Synchronises the handle's stream.  Not
 * for batched handles. */
rick_status rick_set_weight_sum(rick_handle h, double sum_w);

/* Test hook of the error path of the fused column-transform kernel (the
 * split transform of rick_fft_and_stack; the paper has no counterpart).
 * Every wait of that kernel on its shared-memory pipeline is bounded; with
 * skip_slot >= 0 the kernel's producer leaves out the copy of that pipeline
 * slot (plane nk - 1 - skip_slot of a group of nk), so every thread block's
 * wait on it runs out after wait_ns nanoseconds (<= 0: the default 1 s), the
 * block waits for its other copies, leaves, and the failure is recorded:
 * the next rick_get_stats returns RICK_ERR_TIMEOUT until rick_reset.  The
 * image of such a call is invalid; the CUDA context stays usable.
 * skip_slot = -1 restores normal operation (wait_ns still sets the bound).
 * For tests of the timeout handling only; RICK_ERR_ARG for skip_slot < -1. */
rick_status rick_debug_colstack(rick_handle h, int32_t skip_slot, int64_t wait_ns);

/* Counters since the last reset (synchronises the stream).  RICK_ERR_TIMEOUT
 * when a bounded wait inside the fused column-transform kernel ran out since
 * the last reset (the image of that call is invalid; the context stays usable). */
rick_status rick_get_stats(rick_handle h, rick_stats* out);

/* Per-phase device time of the library's own work, from CUDA events recorded
 * on the handle's stream around each phase (no synchronisation while timing
 * is on).  Phases: prep = placement + counting sort (rick_grid); grid = the
 * gridding kernel (Eq. 3); fft = cuFFT plane transforms (the rows only when
 * the column transform is split); colfft = the first column factor of the
 * split transform (the library's own kernel); stack = phase screen + plane
 * reduction + finalisation (with the split: the last column factor too);
 * degrid = the whole adjoint.  Times are sums over all calls since timing
 * was enabled; *_calls count the phase executions; kernel_launches counts
 * librick's own kernel launches (cuFFT's not included). */
typedef struct rick_timing {
    double prep_ms, grid_ms, fft_ms, stack_ms, degrid_ms;
    int64_t prep_calls, grid_calls, fft_calls, stack_calls, degrid_calls;
    int64_t kernel_launches;
    double colfft_ms;
    int64_t colfft_calls;
} rick_timing;

/* Turn phase timing on (enable != 0, resets the sums) or off. */
rick_status rick_set_timing(rick_handle h, int32_t enable);

/* Phase times since timing was enabled (synchronises the stream). */
rick_status rick_get_timing(rick_handle h, rick_timing* out);

/* Message for the last failure on h (static storage of the handle); with
 * h = NULL, the message of the last failed rick_create / rick_create_batch
 * on the calling thread. */
const char* rick_last_error(rick_handle h);

/* Name of a status code. */
const char* rick_status_string(rick_status s);

#ifdef __cplusplus
}
#endif

#endif /* RICK_H */
