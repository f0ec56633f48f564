/*
 * gaborbank.h - C ABI of a GB300 (sm_103a) library computing the 2-D complex Gabor filter
 * bank and the 2-D localized sliding DFT of Um, Kim and Min, "Fast 2-D Complex Gabor Filter
 * with Kernel Decomposition" (arXiv 1704.05231).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Images are single-channel FP32, row-major: pixel (x, y) is img[y * pitch + x], x the
 *    column (the paper's k / m index, horizontal), y the row (l / n, vertical).
 *    pitch >= W counts elements, not bytes.
 *  - Outputs are complex64: interleaved (re, im) float pairs, plane-major, each plane H x W
 *    with row stride W.  The library never allocates or frees caller buffers.
 *  - The image is zero outside [0, W) x [0, H); every output has the input's size.
 *  - The Gaussian is S_sigma(d) = exp(-d^2 / (2 sigma^2)) / (sqrt(2 pi) sigma), truncated
 *    to |d| <= R = ceil(radius_factor * sigma), not renormalised (Sec. II).
 *  - Functions taking device pointers are asynchronous with respect to the host: they
 *    enqueue work on `stream` (a cudaStream_t; NULL = the legacy default stream) and return.
 *    Arguments are validated synchronously.  An asynchronous CUDA error surfaces as
 *    GB_ERR_CUDA from a later call.  Functions taking host pointers are synchronous.
 *  - A handle must not be used from two host threads, or on two streams, at the same time.
 *  - No C++ exception and no abort crosses this interface.  On failure a function returns
 *    a negative gb_status and gabor_bank_last_error() describes the failure; outputs are
 *    then unspecified.
 *  - Work queued by one call may still run when the next call on another stream starts.
 *    Calls on one stream run in order.
 */
#ifndef GABORBANK_H
#define GABORBANK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gabor_bank *gabor_bank_t; /* opaque; owned by the library */

typedef enum {
    GB_OK = 0,
    GB_ERR_INVALID_ARG = -1,   /* NULL pointer, bad size, non-finite or non-positive value */
    GB_ERR_OUT_OF_MEMORY = -2, /* a device or host allocation failed */
    GB_ERR_CUDA = -3,          /* a CUDA runtime call failed (possibly from earlier work) */
    GB_ERR_UNSUPPORTED = -4,   /* valid but not implemented: odd M, too large a radius ... */
    GB_ERR_BUDGET = -5,        /* the request does not fit the handle's memory budget */
    GB_ERR_TIMEOUT = -6        /* a bounded device wait gave up (see gabor_bank_device_status) */
} gb_status;

typedef enum {
    GB_FP32 = 0,    /* FP32 CUDA-core path: |err| <= 1e-5 * max|out| against FP64 */
    GB_FP16_TC = 1, /* tcgen05 tensor cores, FP16 operands, FP32 accumulation */
    GB_BF16_TC = 2  /* tcgen05 tensor cores, BF16 operands, FP32 accumulation; the filter bank
                       splits every operand into BF16 hi + lo parts (three products per step,
                       lo x lo dropped), which makes it more accurate than GB_FP16_TC */
} gb_precision;

/*
 * gabor_bank_create - build a filter-bank plan (Algorithm 1, inputs Sigma, Omega, Theta).
 *
 * theta[n_theta]   orientations in radians, any order and any value.  When both theta and
 *                  pi - theta (to 1e-9 rad) are present, the horizontal pass of theta is
 *                  computed once and reused for pi - theta through J_{pi-theta} = J*_theta
 *                  (Eq. 13-16).
 * omega[n_freq]    centre frequencies in radians per pixel (finite).
 * sigma[n_freq]    Gaussian standard deviations in pixels (> 0), one per frequency.  The
 *                  paper ties sigma to omega inconsistently (Algorithm 1 vs Fig. 1); the
 *                  library takes sigma as given.
 * radius_factor    R_s = ceil(radius_factor * sigma_s); 0 selects 3.
 * prec             arithmetic of gabor_bank_filter / gabor_bank_sdft (see gb_precision).
 * max_H, max_W     largest image the handle will see, used to size internal tables now
 *                  (0, 0: size them on first use).
 * n_theta = n_freq = 0 creates an SDFT-only handle.
 * Returns GB_OK and *out, or an error (and *out = NULL).  The handle owns device tables and
 * workspace; it binds to the CUDA device current at creation.
 */
gb_status gabor_bank_create(gabor_bank_t *out, const double *theta, int n_theta,
                            const double *omega, const double *sigma, int n_freq,
                            double radius_factor, gb_precision prec, int max_H, int max_W);

/* gabor_bank_destroy - synchronise the device and free everything; NULL is allowed. */
gb_status gabor_bank_destroy(gabor_bank_t h);

/*
 * gabor_bank_filter - the 2-D complex Gabor filter bank of Eq. 1 for every (omega_s,
 * theta_k) of the plan, computed by the kernel decomposition of Sec. II (Eq. 3-10) with
 * the orientation reuse of Sec. II-B (Eq. 11-16, Algorithm 1).
 *
 * d_img  device FP32 image, H x W, row stride `pitch` elements (pitch >= W).
 * d_out  device complex64 buffer of n_freq * n_theta * H * W elements (8 bytes each):
 *        out[s][k][y][x] = F_{omega_s, theta_k, sigma_s}(x, y).  8-byte aligned.
 * stream cudaStream_t or NULL.
 * A call needs no per-image-shape device data: after the handle's first call (which builds
 * its tables), calls on new image shapes up to max_H x max_W allocate nothing, except that a
 * GB_FP16_TC handle without a workspace (gabor_bank_set_workspace) grows its own
 * intermediate buffer when an image needs more than it holds.
 * Asynchronous.  Errors: GB_ERR_INVALID_ARG (NULL, H/W <= 0, pitch < W, misaligned),
 * GB_ERR_UNSUPPORTED (a radius above 96 px on tensor cores; a GB_BF16_TC bank under
 * GB_OPT_ROW_PASS = 1), GB_ERR_BUDGET (attached workspace too small), GB_ERR_CUDA.
 * gabor_bank_create refuses radii above 160 px.
 */
gb_status gabor_bank_filter(gabor_bank_t h, const float *d_img, int H, int W, int64_t pitch,
                            void *d_out, void *stream);

/*
 * gabor_bank_filter_host - gabor_bank_filter on HOST buffers: copies the image to the
 * device, filters, copies the result back and synchronises `stream`.  h_out holds
 * n_freq * n_theta * H * W complex64.  Pinned (page-locked) host buffers give full copy
 * bandwidth; pageable ones work too.  Device staging buffers are owned by the handle and
 * grow on demand.  On FP32 handles with the plane-major layout and several frequencies the
 * bank runs as one launch per frequency (cheapest first) and the planes of each finished
 * frequency are copied back on a second, handle-owned stream while the next ones compute;
 * results are bitwise those of one launch.  Synchronous.  Errors as gabor_bank_filter, plus
 * GB_ERR_OUT_OF_MEMORY.
 */
gb_status gabor_bank_filter_host(gabor_bank_t h, const float *h_img, int H, int W,
                                 int64_t pitch, void *h_out, void *stream);

/*
 * gabor_bank_sdft - the 2-D localized sliding DFT with a Gaussian window (Eq. 17-26,
 * Algorithm 2): for every pixel (x, y) and bin (u, v), u in [0, Mx), v in [0, My),
 *   F_{u,v}(x,y) = sum_{a=0}^{Mx-1} sum_{b=0}^{My-1} f(xhat + a, yhat + b)
 *                  exp(-i 2 pi (u a / Mx + v b / My)) S(a - Mx/2) S(b - My/2),
 * xhat = x - Mx/2, yhat = y - My/2 (the M_x x M_y window of Eq. 17).
 *
 * sigma          Gaussian standard deviation (> 0); the paper suggests floor(M/2) = 3 sigma.
 * My, Mx         window size, even, 2..64 each (odd sizes break the integer shift x - M/2
 *                and the conjugate symmetry F_{M-u,M-v} = F*_{u,v}: GB_ERR_UNSUPPORTED).
 * half_spectrum  0: d_out holds My * Mx planes, out[v][u][y][x].
 *                1: only v = 0 .. My/2 are written, out[v][u][y][x] with My/2 + 1 planes
 *                   of v; the rest follow from F_{u,v} = F*_{(Mx-u)%Mx,(My-v)%My}.
 * d_out          device complex64, 8-byte aligned.
 * The handle's precision selects the FP32 separable path (Algorithm 2) or the tensor-core
 * windowed-DFT contraction (Mx * My <= 256).  For Mx in {8, 16, 32, 64} with Mx * My a
 * multiple of 64 the tensor-core path first writes a row-unfolded FP16/BF16 copy of the image,
 * (H + My) * W * Mx * 2 bytes, into a handle-owned buffer that grows when an image needs more
 * (the call then synchronizes the stream once); other windows need no per-image buffer.
 * Asynchronous.  Errors as gabor_bank_filter; GB_ERR_UNSUPPORTED when a tensor-core window's
 * operands do not fit in shared memory.
 */
gb_status gabor_bank_sdft(gabor_bank_t h, const float *d_img, int H, int W, int64_t pitch,
                          double sigma, int My, int Mx, int half_spectrum, void *d_out,
                          void *stream);

/*
 * gabor_bank_filter_batch - gabor_bank_filter for n independent images of possibly
 * different sizes, in one persistent launch (one CTA per SM pulls cost-sorted (image, unit,
 * strip, segment) items from a device work queue).  d_imgs[i], H[i], W[i], pitch[i],
 * d_outs[i] as in gabor_bank_filter; the host arrays are read during the call only.
 * Asynchronous.  Results are bitwise identical to n separate gabor_bank_filter calls with the
 * same handle.  A call whose pointers and shapes equal the previous call's (and whose tables
 * already exist) enqueues only a memset and the kernel, so it can be captured in a CUDA graph.
 * FP32 handles: one launch.  Tensor-core handles: four launches for the whole batch (image
 * min / max, the constant-image tables, the row pass and the column pass over every image's
 * tiles), with intermediates in a handle-owned batch workspace (about 4 bytes per pixel and
 * horizontal pass, plus halo rows), allocated on the first call with a new set of pointers and
 * shapes; plans that need the step-by-step kernels (GB_OPT_ROW_PASS = 1, radii above 96 px)
 * run one bank pass per image.  A batch call on a set of pointers and shapes other than the
 * previous one synchronises the stream once.
 */
gb_status gabor_bank_filter_batch(gabor_bank_t h, int n, const float *const *d_imgs,
                                  const int *H, const int *W, const int64_t *pitch,
                                  void *const *d_outs, void *stream);

/* Runtime options (gabor_bank_set_option). */
typedef enum {
    /* 1 (default): reuse J_theta for pi - theta (Algorithm 1).  0: recompute the
       horizontal pass for every orientation (the paper's "no reuse" comparison). */
    GB_OPT_REUSE = 1,
    /* Rows per streamed chunk in the FP32 bank kernel: 0 = automatic, else 16, 32 or 64. */
    GB_OPT_TILE_ROWS = 2,
    /* Row segments per image column strip: 0 = automatic, else 1 .. 64. */
    GB_OPT_SEGMENTS = 3,
    /* How the image extends beyond its edges (gb_boundary; default GB_BOUNDARY_ZERO).  Applies
       to gabor_bank_filter, _filter_host, _filter_batch and gabor_bank_sdft. */
    GB_OPT_BOUNDARY = 4,
    /* Bank output layout (gb_layout; default GB_LAYOUT_PLANES). */
    GB_OPT_LAYOUT = 5,
    /* The 1-D Gaussian of the bank's passes (gb_smoother; default GB_SMOOTHER_FIR). */
    GB_OPT_SMOOTHER = 6,
    /* Pass order of the FP32 SDFT (Sec. III-B): 0 = automatic (horizontal first), 1 =
       horizontal first, 2 = vertical first.  Vertical first needs fewer FMAs when My > Mx but
       runs on a transposed copy of the image (a handle-owned buffer of H * W floats) with
       stores across output rows, which costs more than it saves on this store-bound kernel.
       Full spectra only (half_spectrum = 1 always runs horizontal first).  Results agree to
       FP32 rounding. */
    GB_OPT_SDFT_ORDER = 7,
    /* FP32 bank kernel schedule: 0 automatic (= 1), 1 phased (all 16 warps of a CTA run a
       chunk's row pass, then its column pass), 2 pipelined (8 warps run the row passes of
       chunk k while the other 8 run the column pass of chunk k - 1; the ring buffer holds two
       chunks of at most 32 rows, hand-over by mbarriers with bounded waits, which report
       device status 35 and GB_ERR_TIMEOUT when they give up).  Results are identical: the
       schedules compute every output with the same operations in the same order. */
    GB_OPT_PIPELINE = 8,
    /* Form of the FP32 bank's row pass (Eq. 5-6), J(x) = sum_d S(d) f(x + d) exp(-i omega^c d):
       0 automatic (= 2), 1 demodulate by (cos, sin)(omega^c x), smooth with the real Gaussian,
       remodulate (the three steps as the paper writes them), 2 one pass with the modulated
       taps S(d) exp(-i omega^c d) (the same sum in one step; the same packed FMAs, no
       demodulated copy of the rows).  The column pass is the same in both.  Results agree to
       FP32 rounding (each within 1e-5 max|out| of the FP64 oracle). */
    GB_OPT_ROW_PASS = 9,
    /* FP32 bank CTAs per SM: 0 automatic (= 1), 1 one CTA of 16 warps, 2 two CTAs of 8 warps
       (each with half of the SM's shared memory, so smaller row tiles for large radii; falls
       back to 1 where a frequency does not fit, and under GB_OPT_PIPELINE = 2).  Results are
       identical. */
    GB_OPT_BANK_CTAS = 10,
    /* Form of the FP32 SDFT passes (Eq. 19-24): 0 automatic (= 2), 1 demodulate, smooth with
       the real Gaussian, remodulate, in both passes (the steps as the paper writes them), 2 one
       convolution with the modulated taps S(a - Mx/2) exp(-i w0 u a) per pass: J_u is read
       straight from its ring for every v, and F_{Mx-u,v} comes from the same four real sums
       over J*_u.  Results agree to FP32 rounding.  The tensor-core SDFT is unaffected. */
    GB_OPT_SDFT_FORM = 11,
    /* Reuse in the FP32 SDFT (Sec. III-B, Algorithm 2): 1 (default) computes the row pass J_u
       once per u <= Mx/2 and reuses it for every v <= My/2, with F_{Mx-u,v} from J*_u
       (Eq. 25-26); 0 is the paper's "no reuse" comparison: J_u is recomputed for every
       (u, v) with u in [0, Mx), v in [0, My/2], nothing is derived from J*_u, and only the
       conjugate fill F_{u,v} = F*_{Mx-u,My-v} stays.  Results agree to FP32 rounding.  The
       tensor-core SDFT is unaffected. */
    GB_OPT_SDFT_REUSE = 12,
    /* Tile shapes of the tensor-core bank's modulated-tap kernels: value = row + 256 * column,
       row = image rows per row-pass item, column = output rows per column-pass job, each 0
       (automatic: 64 where the operands fit in shared memory, else 32) or 32 or 64 (taken when
       it fits, else the automatic value).  Results do not change (every output takes the same
       products).  Used by the autotuner.  Synchronises the device. */
    GB_OPT_TC_TILES = 13
} gb_option;

/* 1-D Gaussian smoothers (GB_OPT_SMOOTHER). */
typedef enum {
    GB_SMOOTHER_FIR = 0,       /* S_sigma truncated at R: exact against Eq. 1 (all precisions) */
    GB_SMOOTHER_IIR = 1        /* Young-van Vliet third-order forward / backward recursion (the
                                  smoother of Sec. II): approximate, cost independent of sigma; FP32
                                  handles, sigma >= 0.5.  Each signal is extended by P = ceil(12 sigma)
                                  + 32 samples per side under the boundary rule; the recursions start
                                  from zero state.  Evaluated in difference form, chunk-parallel along
                                  every line.  Uses a library-owned workspace of about
                                  8 * n_units * (H + 2 P) * W bytes (J of every horizontal pass) plus
                                  1.5 bytes per column-pass sample; extended rows (W + 2 P) longer than
                                  about 20000 samples return GB_ERR_UNSUPPORTED. */
} gb_smoother;

/* Image extension rules (GB_OPT_BOUNDARY).  The paper leaves the border unstated. */
typedef enum {
    GB_BOUNDARY_ZERO = 0,      /* f = 0 outside [0, W) x [0, H) */
    GB_BOUNDARY_REPLICATE = 1, /* the nearest edge pixel */
    GB_BOUNDARY_MIRROR = 2     /* mirrored about the pixel edges: f(-1) = f(0), f(W) = f(W-1), period 2W */
} gb_boundary;

/* Bank output layouts (GB_OPT_LAYOUT); both hold n_freq * n_theta * H * W complex64. */
typedef enum {
    GB_LAYOUT_PLANES = 0,      /* out[s][k][y][x]: one H x W plane per filter */
    GB_LAYOUT_PIXELS = 1       /* out[y][x][s][k]: the n_freq x n_theta feature vector of each pixel */
} gb_layout;

/* gabor_bank_set_option - set an option; GB_ERR_INVALID_ARG on an unknown key or value. */
gb_status gabor_bank_set_option(gabor_bank_t h, int key, int64_t value);

/*
 * gabor_bank_set_tiling - tile geometry of the FP32 bank kernel for frequency s (s = -1: all
 * frequencies): rows per streamed chunk (0 = automatic, or 8, 16, 32, 64) and row segments per
 * column strip (0 = automatic, or 1 .. 64).  This trades the 2R-row halo recomputed per
 * segment against load balance; results do not change (the arithmetic of every output is the
 * same).  Used by the autotuner.  Synchronises the device.  GB_ERR_INVALID_ARG on bad values.
 */
gb_status gabor_bank_set_tiling(gabor_bank_t h, int s, int tile_rows, int segments);

/*
 * gabor_bank_device_status - wait for `stream`, then read and clear the handle's device
 * error word: GB_OK; GB_ERR_TIMEOUT if a bounded device wait (tensor-core pipeline barriers)
 * gave up since the last read; GB_ERR_UNSUPPORTED if a GB_FP16_TC bank met an image whose
 * centre level c = (min + max) / 2 is beyond its FP16 operands' range (|c| above about 2^24;
 * GB_BF16_TC has no such limit), whose results are then wrong.  Synchronous.
 */
gb_status gabor_bank_device_status(gabor_bank_t h, void *stream);

/*
 * gabor_fp32_fma_probe - FP32 CUDA-core throughput probe (the measured peak that the FP32
 * bank's roofline fraction divides by; the paper has no counterpart).  Enqueues `blocks` CTAs
 * of 256 threads on the current device; every thread runs 16 independent FMA chains for
 * `iters` iterations: 32 * iters FLOP per thread, scalar fmaf (packed = 0) or packed FP32x2
 * FMA (packed = 1).  d_out: a device float the kernel may write.  Time it with CUDA events.
 * Asynchronous.  GB_ERR_INVALID_ARG on NULL or non-positive arguments.
 */
gb_status gabor_fp32_fma_probe(void *d_out, int blocks, int iters, int packed, void *stream);

/*
 * gabor_store_probe - store-bandwidth probe for the tensor-core SDFT's output pattern (the
 * paper has no counterpart).  Writes nplanes x H x W complex64 values to d_out (plane-major,
 * the SDFT's output layout, caller-owned device memory of 8 * nplanes * H * W bytes) the way
 * that kernel's epilogue does, without its arithmetic: `ctas` CTAs of 16 warps, tiles of 128
 * pixels of one row, a warp storing 32 consecutive pixels of one plane per instruction.  The
 * values are non-zero (a zero fill runs faster through the memory's zero compression).  Time
 * it with CUDA events.  Asynchronous.  GB_ERR_INVALID_ARG on NULL or non-positive arguments or
 * W not a multiple of 128.
 */
gb_status gabor_store_probe(void *d_out, int64_t nplanes, int H, int W, int ctas, void *stream);

/*
 * gabor_bank_selftest_wait - failure-detection self-test of the bounded device waits.  Enqueues
 * a one-warp kernel whose thread 0 waits on a shared-memory mbarrier with the same bounded
 * wait the tensor-core kernels use.  signal = 1: the barrier is signalled first and the wait
 * succeeds.  signal = 0: nothing signals it; the wait gives up after limit_ms (0 < limit_ms
 * <= 2000), writes code 90 to the handle's device status word and the kernel returns, leaving
 * the CUDA context usable.  gabor_bank_device_status then reports GB_ERR_TIMEOUT.  The paper
 * has no counterpart; this checks the library's own error path.  Asynchronous.
 */
gb_status gabor_bank_selftest_wait(gabor_bank_t h, int signal, double limit_ms, void *stream);

/*
 * gabor_sdft_noalloc - the FP32 localized sliding DFT of gabor_bank_sdft (same arguments and
 * output layout, FP32 CUDA-core path, zero boundary rule) for callers that cannot allocate
 * device memory: code inside a custom allocator or memory pool that forbids cudaMalloc, or an
 * application whose device-memory budget is fixed before it starts.  No handle is needed and
 * the call allocates nothing.  The paper has no counterpart; this is a deployment convenience.
 *
 * Its tables (Gaussian taps and twiddles of both window axes) live in one fixed 2 KiB
 * __device__ array of the library, which every GPU that loads the library holds until the
 * process exits.  Limits: My, Mx even, 2 .. 64 (GB_ERR_UNSUPPORTED beyond).  The first call on
 * a device does a one-time set-up on that device (the array's device address, kernel
 * attributes) under a process-wide mutex; make that first call before any CUDA stream
 * capture.  Every call then enqueues two kernels on `stream`: one that rewrites the whole
 * table (1600 bytes, from by-value parameters; no host-to-device copy) and the SDFT kernel.
 * Because every call rewrites the shared table, calls that overlap on the GPU (for example on
 * two streams) race; serialise them on one stream.  Asynchronous like gabor_bank_sdft; argument
 * checks and errors as gabor_bank_sdft.
 */
gb_status gabor_sdft_noalloc(const float *d_img, int H, int W, int64_t pitch, double sigma,
                             int My, int Mx, int half_spectrum, void *d_out, void *stream);

/*
 * gabor_bank_workspace_bytes - device bytes of intermediate a GB_FP16_TC / GB_BF16_TC handle
 * needs to filter an H x W image: the FP16 signals between the row and the column pass (by
 * default Re J and Im J of every horizontal pass, Eq. 5-6; under GB_OPT_ROW_PASS = 1 the
 * column signals of Eq. 10), each image column padded by zero rows above and below, followed
 * by the bank's response to a constant image, one row and one column table per horizontal
 * pass, the operands that add it back in the column pass's matrix products (4 KB per 64
 * image columns and per 32 image rows of every horizontal pass), and the row pass's operand
 * image (f - c) 2^-e (2 bytes per pixel, 4 under GB_BF16_TC, rows padded to 8 pixels), which
 * the zero rule's row pass loads by TMA.  Sized for the larger of the two forms.  0 for FP32
 * handles (their intermediates stay on chip) and for invalid arguments.  Host-only; no device
 * work.
 */
int64_t gabor_bank_workspace_bytes(gabor_bank_t h, int H, int W);

/*
 * gabor_bank_set_workspace - make the handle use the caller's device buffer d_ws (16-byte
 * aligned, `bytes` long) as its tensor-core intermediate from the next call on, instead of a
 * buffer of its own; d_ws = NULL, bytes = 0 returns to the handle's own buffer.  The caller
 * keeps ownership and must keep the buffer alive and unused by other work while calls that
 * use it run.  Several handles may share one workspace when their calls are ordered (one
 * stream).  A filter call whose image needs more than `bytes` fails with GB_ERR_BUDGET.
 * Host-only; no device work.  GB_ERR_INVALID_ARG on a NULL handle, misalignment or a
 * non-positive size.
 */
gb_status gabor_bank_set_workspace(gabor_bank_t h, void *d_ws, int64_t bytes);

/*
 * Device-memory arena: one allocation made at creation, handed out in 256-byte aligned
 * ranges (first fit by address, neighbours merged on free).  Used to admit work by a fixed
 * HBM budget: an allocation that does not fit fails at once with GB_ERR_BUDGET instead of
 * growing device memory.  Book-keeping is host-only and thread-safe; the arena never
 * synchronises, so a range may be freed only when the device work that uses it has
 * finished (or when later users are ordered after it on one stream).
 */
typedef struct gabor_arena *gabor_arena_t;

/* gabor_arena_create - cudaMalloc `bytes` (> 0) on the current device.
   GB_ERR_OUT_OF_MEMORY if the device cannot provide it. */
gb_status gabor_arena_create(gabor_arena_t *out, int64_t bytes);
/* gabor_arena_wrap - an arena over caller-owned device memory d_base (256-byte aligned,
   `bytes` long); gabor_arena_destroy then leaves the memory to the caller. */
gb_status gabor_arena_wrap(gabor_arena_t *out, void *d_base, int64_t bytes);
/* gabor_arena_alloc - *d_ptr = a free range of `bytes` (> 0), or GB_ERR_BUDGET (and NULL). */
gb_status gabor_arena_alloc(gabor_arena_t a, int64_t bytes, void **d_ptr);
/* gabor_arena_free - return a range from gabor_arena_alloc; GB_ERR_INVALID_ARG otherwise. */
gb_status gabor_arena_free(gabor_arena_t a, void *d_ptr);
/* gabor_arena_stats - capacity, bytes in use and the largest free range (any may be NULL). */
gb_status gabor_arena_stats(gabor_arena_t a, int64_t *capacity, int64_t *in_use, int64_t *largest_free);
/* gabor_arena_destroy - free the arena (and its device allocation if gabor_arena_create made
   it); outstanding ranges become invalid.  NULL is allowed. */
gb_status gabor_arena_destroy(gabor_arena_t a);

/* gabor_bank_output_elems - complex elements gabor_bank_filter writes for an H x W image. */
int64_t gabor_bank_output_elems(gabor_bank_t h, int H, int W);

/* gabor_bank_last_error - message of the last failure on this host thread ("" if none). */
const char *gabor_bank_last_error(void);

/* gabor_bank_version - library version string. */
const char *gabor_bank_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GABORBANK_H */
