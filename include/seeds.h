/*
 * seeds.h -- C ABI of libseeds.so: SEEDS superpixels on one GB300 (sm_103a).
 *
 * Method: M. Van den Bergh, X. Boix, G. Roig, L. Van Gool, "SEEDS:
 * Superpixels Extracted via Energy-Driven Sampling", arXiv 1309.3848.
 * The library runs the paper's hill climbing (Sec. 5): a grid start
 * (Sec. 5.1), block moves from the largest block level down to the
 * smallest, then pixel moves (Sec. 5.2), each judged by the histogram
 * intersection test (Prop. 1) and, for pixels, the label-patch test
 * (Prop. 2), with incremental histogram updates (Sec. 5.3).
 *
 * Fixed readings (the same ones the bundled CPU oracle follows):
 *  - colour bins from the RGB bytes, or from their 8-bit CIE L*a*b* codes
 *    (color_space = 1, Sec. 6.2): bin(v) = floor(v*B/256) per channel,
 *    j = bR*B*B + bG*B + bB;
 *  - grid: gx = max(1, round(sqrt(K*W/H))), gy = max(1, round(K/gx)),
 *    K_actual = gx*gy; level-l block edges floor(i*W/(gx*2^(L-l+1)));
 *  - every level runs iters_per_level iterations of four parity phases
 *    (py,px) = (0,0),(0,1),(1,0),(1,1); a phase judges all its units against
 *    the state at phase start and applies the accepted moves together;
 *  - a unit may leave superpixel k only if k stays 4-connected around it
 *    (local 8-ring test); candidates are the distinct neighbour labels,
 *    best score wins, ties to the smallest label, accept on strict gain;
 *  - pixel score D*c_An(j) + gamma*(G_n + |K_p|) against
 *    D*c_{Ak\p}(j) + gamma*G_k with D = 81 (Prop. 1 + Prop. 2); blocks use
 *    the intersection alone; all compares are exact int64 products, except
 *    in the optional means-based pixel iterations (Sec. 6.3, 6.5), which
 *    compare fixed-order single-precision distances.
 * Results are deterministic: the same image and parameters give the same
 * labels on any stream, in any batch, at any tuning.
 *
 * Memory and streams.  Device pointers (d_*) are CUDA device addresses
 * owned by the caller (e.g. torch tensor data_ptr()).  Host pointers (h_*)
 * are ordinary host memory; pinned memory makes their copies asynchronous.
 * `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 * Calls on one context must be issued from one host thread at a time and
 * are ordered by the stream they are given; a context keeps its state (bin
 * maps, label grids, histograms) resident on the device between calls.
 *
 * Errors.  Every entry point returns an int status: SEEDS_OK or one of the
 * negative codes below.  No exception crosses the ABI.  Device-side faults
 * that the kernels detect themselves (a grid-barrier wait that ran out; in
 * the bounds-checked debug build, an index outside its buffer) are recorded
 * in the context's error word and
 * reported by seeds_status().
 */
#ifndef SEEDS_H
#define SEEDS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SEEDS_OK 0
#define SEEDS_ERR_INVALID (-1)     /* bad argument or parameter */
#define SEEDS_ERR_GEOMETRY (-2)    /* gx*2^L > W or gy*2^L > H */
#define SEEDS_ERR_INT64 (-3)       /* exact int64 products could overflow */
#define SEEDS_ERR_NO_MEMORY (-4)   /* device allocation failed */
#define SEEDS_ERR_CUDA (-5)        /* a CUDA runtime call failed */
#define SEEDS_ERR_DEVICE (-6)      /* device-side timeout or bounds trip */
#define SEEDS_ERR_STATIC_SIZE (-7) /* image too large for seeds_run_static */

#define SEEDS_MAX_LEVELS 12
#define SEEDS_MAX_BATCH 4096
#define SEEDS_STATIC_SCRATCH_BYTES (32u << 20) /* device scratch of seeds_run_static */

typedef struct seeds_ctx seeds_ctx;

/* Parameters of one image (Sec. 6.2 fixes gamma = 1, a 3x3 patch, 5 bins,
 * and LAB colour).
 *   width, height      image size, 1..32768 each, width*height < 2^31
 *   num_superpixels    requested K (>= 1); the grid gives gx*gy <= 65535
 *   block_levels       L >= 0 (0 = pixel moves only)
 *   bins_per_channel   B in 1..16; histograms have B^3 bins
 *   iters_per_level    0..1000, for every block level and the pixel level;
 *                      0 only with means_iters > 0: SPM on its own (Sec.
 *                      6.3), the means iterations start from the grid
 *   patch              0 (no boundary term) or 3 (3x3 patches, Prop. 2)
 *   gamma_num/den      gamma = num/den, 0 <= num <= 1024, 1 <= den <= 1024
 *   color_space        0: bins of the RGB bytes; 1: bins of the 8-bit CIE
 *                      L*a*b* code of each pixel (sRGB under D65; L* scaled
 *                      by 255/100, a* and b* offset by 128, rounded half up),
 *                      computed in exact integer fixed point: the sRGB
 *                      decoding curve as linear light * 2^24, the sRGB to
 *                      XYZ matrix rows divided by the D65 white * 2^20,
 *                      f(t) * 2^20 by an exact integer cube root
 *   means_iters        0..1000 more pixel-level iterations after the
 *                      histogram ones in which a pixel moves to the neighbour
 *                      superpixel whose mean is nearest in SLIC's distance
 *                      (Sec. 6.3 SPM, run as post-processing, Sec. 6.5): the
 *                      squared distance of its colour code to the mean code
 *                      plus (m/S)^2 times the squared distance to the
 *                      centroid, S^2 = W*H/K; strictly nearer than its own
 *                      superpixel's mean (with the pixel in it), ties to the
 *                      smallest label, IEEE single precision without fused
 *                      operations (a mean is its sum times 1/size)
 *   compactness        m in 0..1024 (0 = colour only)
 *   edge_threshold     0..765, 0 = off: edge snapping (the edge prior of
 *                      Sec. 6.4).  Two 4-neighbour pixels are across a colour
 *                      edge when the L1 distance of their colour codes (the
 *                      bytes the bins come from) is at least this; a pixel
 *                      with a 4-neighbour of another label across an edge
 *                      no longer moves (pixel and means phases)
 *   compact_prior      0..1024, 0 = off: the compactness prior of Sec. 6.4 in
 *                      the histogram pixel phases.  Every option's score
 *                      loses w*D*d^2/S^2, d^2 the squared distance of the
 *                      pixel to the option's centre of gravity (its own
 *                      superpixel's with the pixel in it), S^2 = W*H/K,
 *                      D = 81, w = compact_prior/16; with the prior on, the
 *                      pixel score is compared in IEEE single precision in a
 *                      fixed order (colour term a/s by one division, centre
 *                      as sum times 1/size) instead of exact integers */
typedef struct {
    int32_t width, height;
    int32_t num_superpixels;
    int32_t block_levels;
    int32_t bins_per_channel;
    int32_t iters_per_level;
    int32_t patch;
    int32_t gamma_num, gamma_den;
    int32_t color_space;
    int32_t means_iters;
    int32_t compactness;
    int32_t edge_threshold;
    int32_t compact_prior;
} seeds_params;

/* Result-invariant launch knobs (any value gives identical labels).
 *   threads_per_block  128, 256, 512 or 1024 (0 = the largest whose
 *                      shared scratch fits, 1024 unless B^3 is large)
 *   blocks_per_sm      resident CTAs per SM of the persistent kernel,
 *                      0 = as many as fit
 *   hist_layout        0: hist[k][j] (label-major), 1: hist[j][k] (bin-major)
 *   pixel_tile_rows    unit rows of a pixel-phase warp tile (32 units wide):
 *                      2 or 4 (0 = 4); shorter tiles balance small images
 *   small_block_area   blocks of at most this many pixels are judged by one
 *                      thread, larger ones by a warp (1..16; 0 = default)
 *   block_tiles        wide steps: phases of warp-judged block levels in
 *                      warp tiles (32 x 1 units, labels staged in shared
 *                      memory, only boundary blocks judged) and catch-ups
 *                      with more units per lane: 0 = steps with at least two
 *                      tiles per warp slot of the GPU (the default),
 *                      1 = never, 2 = every step */
typedef struct {
    int32_t threads_per_block;
    int32_t blocks_per_sm;
    int32_t hist_layout;
    int32_t small_block_area;
    int32_t pixel_tile_rows;
    int32_t block_tiles;
} seeds_tuning;

/* Fill p with the paper's defaults for a W x H image and K superpixels
 * (Sec. 6.2 for the bins, the 3x3 patch and gamma; Sec. 5.1 for the block
 * levels): 4 block levels (clamped to what the grid allows), 5 bins per
 * channel, 2 iterations, 3x3 patch, gamma = 1; RGB, no means iterations, no
 * edge snapping.  Host only. */
int seeds_params_default(seeds_params *p, int32_t width, int32_t height, int32_t num_superpixels);

/* Largest block_levels the grid geometry of *p allows (>= 0), ignoring
 * p->block_levels itself: the block hierarchy of Sec. 5.1, where each level
 * halves the block size down to blocks of a few pixels.  Host only;
 * SEEDS_ERR_INVALID for bad sizes. */
int seeds_feasible_levels(const seeds_params *p, int32_t *max_levels);

/* Validate *p and compute its grid without allocating: K_actual = gx*gy
 * (the initial partition of Sec. 5.1).  Returns SEEDS_ERR_GEOMETRY /
 * SEEDS_ERR_INT64 exactly as seeds_create would; the int64 bound covers the
 * cross-multiplied compares of Prop. 1 and Prop. 2 (Sec. 5.3). */
int seeds_check_params(const seeds_params *p, int32_t *gx, int32_t *gy);

/* Device bytes a context for these images would hold (for admission
 * control by footprint).  The paper has no counterpart: it sizes the state
 * of Sec. 5.1 (bin map, label grids of every level, Sec. 4 histograms).
 * Host only. */
int seeds_footprint(const seeds_params *p, int32_t n, int64_t *bytes);

/* One entry of a step schedule (seeds_plan): work of image `img` in one
 * step, handed to the kernel as `units` units of `group` threads each (1: a
 * thread per unit, 32: a warp per unit; pixel tiles and init rectangles are
 * warp units), starting at virtual thread vt_begin of its step.
 *   op      0 init, 1 phase, 2 descent, 3 output, 4 catch-up (replays the
 *           moves of op opidx-1 into the buffer that op read), 5 start of
 *           the means iterations, 6 means phase
 *   level   the op's level (0 = pixels; a catch-up: the level of op opidx-1)
 *   phase   parity phase (py*2 + px) of a phase or catch-up entry
 *   opidx   the image's op number, which selects its state buffers
 *   cphase  a phase entry whose units first replay the previous phase of
 *           the same level (that phase's parity), or -1 */
typedef struct {
    int32_t img, op, level, phase, opidx, units, group, cphase;
    int64_t vt_begin;
} seeds_plan_entry;

/* The step schedule (the hill climbing of Sec. 5.2-5.3 as parity phases,
 * level by level) a launch over the n images p[0..n) uses on a GPU with
 * sm_count SMs, planned on the host alone (no device is touched): one step
 * per op (the images of a batch share each step), a catch-up entry where a
 * phase's moves are replayed beside the next op, and the fusion of replays
 * into block or pixel phases that the step's size calls for.  Image i runs
 * its ops [op_begin[i], op_end[i]) (NULL = from the first op / to the last:
 * a full run); a range that starts after a phase catches up that phase's
 * moves first, as a launch resuming a stopped run does.  t: launch knobs
 * (NULL = defaults; only small_block_area and pixel_tile_rows shape a
 * schedule).  Always writes *n_entries and *n_steps.  With out,
 * step_first and step_threads all NULL it stops there; otherwise out[cap]
 * receives the entries in step order, step_first[step_cap] the index of
 * every step's first entry and one past the last (step_cap >= *n_steps+1),
 * and step_threads (if not NULL) every step's padded thread count.
 * Returns SEEDS_ERR_INVALID for bad parameters or buffers too small, and
 * seeds_check_params' errors.  Host only. */
int seeds_plan(const seeds_params *p, int32_t n, const seeds_tuning *t, int32_t sm_count, const int32_t *op_begin,
               const int32_t *op_end, seeds_plan_entry *out, int32_t cap, int32_t *n_entries, int32_t *step_first,
               int64_t *step_threads, int32_t step_cap, int32_t *n_steps);

/* Create a context for one image on the current CUDA device: validates the
 * parameters (the partition into K superpixels of Sec. 3, its initial grid
 * and block levels of Sec. 5.1, the int64 bound of the exact compares of
 * Sec. 5.3) and allocates all device state.  Host call, synchronous. */
int seeds_create(const seeds_params *p, seeds_ctx **out);

/* Run the whole schedule on one image: quantise, grid, histograms (Sec. 4,
 * Sec. 5.1), block levels L..1 and the pixel level (Sec. 5.2-5.3), for
 * iters_per_level iterations each (the stopping rule of Sec. 5.4 as a fixed
 * iteration count).  d_rgb: device, H rows of W*3 uint8 (R,G,B),
 * row_stride_bytes >= 3*W apart.  Asynchronous on `stream`; d_rgb must stay
 * valid until the stream reaches this work.  Re-initialises from the image
 * on every call. */
int seeds_iterate(seeds_ctx *c, const uint8_t *d_rgb, int64_t row_stride_bytes, void *stream);

/* Write the labels of the last seeds_iterate, the partition s of Sec. 3 (one
 * superpixel label per pixel): d_labels_out is a device int32 H x W
 * row-major buffer (caller-owned), values in [0, K_actual).  Asynchronous on
 * `stream`. */
int seeds_labels(seeds_ctx *c, int32_t *d_labels_out, void *stream);

/* K_actual = gx*gy of image 0 of the context: the number of superpixels K
 * of Sec. 3, fixed by the initial grid of Sec. 5.1. */
int seeds_num_superpixels(const seeds_ctx *c, int32_t *k_out);

/* Wait for the context's last launched work and report device-side errors:
 * SEEDS_OK, SEEDS_ERR_DEVICE (the error word was set; it is cleared), or
 * SEEDS_ERR_CUDA.  Failure reporting has no counterpart in the paper. */
int seeds_status(seeds_ctx *c);

/* Free the context (waits for its work first).  Resource handling has no
 * counterpart in the paper. */
int seeds_destroy(seeds_ctx *c);

/* ---- batches: many images of any sizes in one persistent launch ------- */

/* Context for n images (1..SEEDS_MAX_BATCH); p[i] are their parameters.
 * Each image is partitioned independently as in seeds_create (Sec. 3,
 * Sec. 5.1); running many images in one launch has no counterpart in the
 * paper. */
int seeds_batch_create(const seeds_params *p, int32_t n, seeds_ctx **out);

/* Number of images of the context (batching has no counterpart in the
 * paper). */
int seeds_batch_size(const seeds_ctx *c, int32_t *n_out);
/* K_actual of image i: its superpixel count K (Sec. 3) after the grid of
 * Sec. 5.1. */
int seeds_batch_num_superpixels(const seeds_ctx *c, int32_t i, int32_t *k_out);

/* Run all images through the schedule of seeds_iterate (Sec. 5.1-5.3):
 * h_rgb_ptrs[i] is the DEVICE address of image i (an array of n device
 * pointers held in host memory), h_row_strides[i] its row stride in bytes.
 * One persistent kernel launch.  Asynchronous. */
int seeds_batch_iterate(seeds_ctx *c, const uint8_t *const *h_rgb_ptrs, const int64_t *h_row_strides,
                        void *stream);

/* Write every image's labels (its partition s, Sec. 3): h_label_ptrs[i] is
 * the device address of an int32 H_i x W_i buffer.  Asynchronous. */
int seeds_batch_labels(seeds_ctx *c, int32_t *const *h_label_ptrs, void *stream);

/* seeds_batch_iterate and seeds_batch_labels fused into one launch (the
 * whole of Sec. 5.1-5.3 and the partition of Sec. 3).  Once a
 * context has run this call, a repeat of it on the same buffers allocates
 * and synchronises nothing (a pointer upload, a barrier reset and the
 * persistent kernel), so it can be captured into a CUDA graph and replayed;
 * after replays, synchronise the replay stream before seeds_status. */
int seeds_batch_run(seeds_ctx *c, const uint8_t *const *h_rgb_ptrs, const int64_t *h_row_strides,
                    int32_t *const *h_label_ptrs, void *stream);

/* Anytime termination (Sec. 5.4).  As seeds_batch_run, but the launch may
 * stop early: at the first step boundary where max_steps steps have run
 * (max_steps > 0) or budget_ns nanoseconds of device time have passed since
 * the launch began (budget_ns > 0), whichever comes first; 0 for both runs
 * every step.  A step is one op of every image, and image i's ops are, in
 * order: the initialisation; for each block level L..1 its 4*iters parity
 * phases and the descent to the next finer level; the 4*iters pixel phases;
 * the output.  An image whose output op has not run when the launch stops
 * gets the partition after its ops done so far, each pixel labelled by the
 * unit that holds it at the level the image stands at; it is a valid
 * partition (every superpixel non-empty and 4-connected).  Asynchronous;
 * seeds_anytime_steps tells how many steps ran.  The context's state is then
 * that of the stop, so seeds_batch_labels / seeds_labels return
 * SEEDS_ERR_INVALID until the next seeds_batch_iterate or run.
 * Errors: SEEDS_ERR_INVALID for a negative limit or a null pointer. */
int seeds_batch_run_anytime(seeds_ctx *c, const uint8_t *const *h_rgb_ptrs, const int64_t *h_row_strides,
                            int32_t *const *h_label_ptrs, int32_t max_steps, int64_t budget_ns, void *stream);

/* Steps the last seeds_batch_run_anytime launch ran (waits for it); 0 if
 * there was none.  The anytime stop of Sec. 5.4. */
int seeds_anytime_steps(seeds_ctx *c, int32_t *steps);

/* End to end from HOST memory: copies every image host->device into
 * context-owned staging buffers, runs the batch (Sec. 5.1-5.3), and copies
 * the labels (Sec. 3) device->host.  h_rgb[i]: H_i rows of 3*W_i bytes, h_row_strides[i] apart;
 * h_labels[i]: int32 H_i x W_i.  Asynchronous on `stream` (the host buffers
 * must stay valid until the stream completes; pinned buffers overlap). */
int seeds_run_host(seeds_ctx *c, const uint8_t *const *h_rgb, const int64_t *h_row_strides, int32_t *const *h_labels,
                   void *stream);

/* seeds_run_host over a stream of n_batches batches of the context's shape
 * (Sec. 5.1-5.3 for each), with the copies of one batch overlapping the
 * launch of another: batch b's host->device copies run while batch b-1 is
 * segmented, and its labels go back while batch b+1 is.  Two sets of
 * staging buffers alternate; the copies run on two streams of the
 * context's own, and `stream` waits for all of them before the call's work
 * counts as done, so stream order holds for the whole sequence.
 * h_rgb, h_row_strides, h_labels: n_batches * n pointers (n the batch
 * size), batch-major (entry b*n + i is image i of batch b), as in
 * seeds_run_host; the same host buffer may serve several batches.
 * Asynchronous on `stream`; host buffers must stay valid until it completes
 * (pinned buffers make the copies asynchronous).  Errors:
 * SEEDS_ERR_INVALID for n_batches < 1, a null pointer, a row stride below
 * 3*W, or `stream` under capture into a CUDA graph. */
int seeds_run_host_stream(seeds_ctx *c, int32_t n_batches, const uint8_t *const *h_rgb,
                          const int64_t *h_row_strides, int32_t *const *h_labels, void *stream);

/* Launch knobs; see seeds_tuning.  They change no label, so the paper has
 * no counterpart. */
int seeds_set_tuning(seeds_ctx *c, const seeds_tuning *t);

/* The search seeds_autotune runs, with the timing supplied by the caller:
 * coordinate descent from *start over threads_per_block {128, 256, 512,
 * 1024}, blocks_per_sm {0..3}, hist_layout {0, 1}, small_block_area {4, 9,
 * 16}, pixel_tile_rows {2, 4} and block_tiles {0, 1, 2}, in that order, one
 * pass; a value is kept
 * only if cost() reports it at least 2% faster than the current setting.
 * cost returns milliseconds (a huge value for a setting that cannot run).
 * Writes the setting found to *best.  Host only; no device is touched.  The
 * knobs change no label, so the paper has no counterpart. */
typedef float (*seeds_tune_cost_fn)(const seeds_tuning *t, void *user);
int seeds_tune_search(const seeds_tuning *start, seeds_tune_cost_fn cost, void *user, seeds_tuning *best);
/* The context's current launch knobs (no counterpart in the paper). */
int seeds_get_tuning(const seeds_ctx *c, seeds_tuning *t);

/* Pick the fastest result-invariant knobs for this context's images by
 * timing candidate settings on them (the labels do not depend on the
 * choice), apply them, and return them in *best (may be NULL).  Runs
 * `reps` timed batches per candidate on `stream` and synchronises.  The
 * inputs are as for seeds_batch_run (device images and label buffers).  No
 * counterpart in the paper. */
int seeds_autotune(seeds_ctx *c, const uint8_t *const *h_rgb_ptrs, const int64_t *h_row_strides,
                   int32_t *const *h_label_ptrs, int32_t reps, void *stream, seeds_tuning *best);

/* ---- serving: continuous batching over a device arena ------------------
 *
 * The server keeps images resident in slots of one device arena and runs
 * them in epochs: one persistent launch advances every resident image by up
 * to epoch_steps of its ops (a step = one parity phase, a descent, the init
 * or the output of Sec. 5), so an image admitted while others run joins them
 * at the next epoch.  Requests are admitted first come first served when a
 * slot is free and their footprint (seeds_footprint plus 7 bytes per pixel
 * of image and label staging) fits the arena.  Each image's labels are the
 * same alone or in any mix.  All work runs on the server's own streams:
 * one for the launches and one each for the copies in and out, which
 * overlap the launches; a finished image's arena space is reused only once
 * its labels have reached the host. */
typedef struct seeds_server seeds_server;

typedef struct {
    int64_t arena_bytes;           /* device memory for resident images (>= 1 MiB) */
    int32_t max_slots;             /* images resident at once, 1..128 */
    int32_t epoch_steps;           /* ops per image per launch, 1..1024 */
    int32_t max_bins_per_channel;  /* largest B a request may use, 1..16 */
} seeds_server_config;

typedef struct {
    int32_t queued, resident;
    int64_t arena_free_bytes;  /* free now: a finished request's space counts once its labels have reached the host */
    int64_t epochs, launches, admitted;
    double host_ms;  /* host time since creation, on the clock done_ms uses */
} seeds_server_stats_t;

/* A server over a device arena (continuous batching has no counterpart in
 * the paper; each served image runs the schedule of Sec. 5.1-5.3). */
int seeds_server_create(const seeds_server_config *cfg, seeds_server **out);
/* Free the server (waits for its work).  No counterpart in the paper. */
int seeds_server_destroy(seeds_server *s);

/* Queue one request (one image to partition, Sec. 3).  h_rgb: host, H rows
 * of 3*W bytes, row_stride_bytes apart; h_labels: host int32 H x W that
 * receives the labels.  Both must stay
 * valid until the request is reported done by seeds_server_poll (pinned
 * memory makes the copies asynchronous).  *id receives the request id.
 * SEEDS_ERR_NO_MEMORY if the image could never fit the arena. */
int seeds_server_submit(seeds_server *s, const seeds_params *p, const uint8_t *h_rgb, int64_t row_stride_bytes,
                        int32_t *h_labels, int64_t *id);

/* Admit what fits, then launch one epoch over the resident images
 * (asynchronous; blocks only while two epochs are already queued): up to
 * epoch_steps ops of each image's schedule (Sec. 5.2-5.3).
 * *resident receives the number of images in the epoch (0: nothing to do). */
int seeds_server_step(seeds_server *s, int32_t *resident);

/* Requests finished since the last call (non-blocking): ids[i] and the
 * device-side completion time done_ms[i] in ms since the server was created,
 * for i < *n <= cap.  No counterpart in the paper. */
int seeds_server_poll(seeds_server *s, int64_t *ids, float *done_ms, int32_t cap, int32_t *n);

/* Wait for all launched work; report device-side errors as seeds_status.
 * No counterpart in the paper. */
int seeds_server_drain(seeds_server *s);

/* Queue, residency, arena and epoch counters (no counterpart in the
 * paper). */
int seeds_server_stats(const seeds_server *s, seeds_server_stats_t *out);

/* ---- one image without allocating ----------------------------------------
 *
 * The paper has no counterpart to this entry point; it exists for callers
 * that must not allocate device memory themselves or through a library: code
 * that runs inside a framework which owns the whole device memory through its
 * own pool and budget, or a latency-critical loop that cannot afford the
 * device-wide synchronisation and unpredictable time a cudaMalloc/cudaFree
 * can bring.  It runs the same schedule as seeds_iterate + seeds_labels on
 * one image and gives the same labels, but keeps every byte of its device
 * state (bin map, label grids, histograms, move lists, schedule, barrier) in
 * one file-scope static device array of SEEDS_STATIC_SCRATCH_BYTES (32 MiB)
 * inside libseeds.so.  Every GPU that loads the library holds that array
 * until the process exits.  No cudaMalloc, cudaFree, host heap or other
 * allocating routine is called.
 *
 *   p              image parameters, as for seeds_create
 *   d_rgb          device, H rows of W*3 uint8, row_stride_bytes apart
 *   d_labels_out   device int32 H x W, written with labels in [0, K_actual)
 *   d_status       device int32 or NULL; receives the run's device error word
 *                  (0 = no device-side timeout or bounds trip)
 *   stream         cudaStream_t as void*; the call is asynchronous on it
 *
 * Returns SEEDS_ERR_STATIC_SIZE, without launching anything, when the
 * image's state does not fit the array (about 4 Mpixel at 5 bins per
 * channel; a 1920x1080 image with 1000 superpixels needs about 17 MiB),
 * and the usual codes for bad parameters.  The first call on each device
 * looks up the array's device address (with that device current) and
 * caches it (calls outside a stream capture look it up again), and every
 * call with color_space = 1 made outside a capture copies the 1 KB LAB
 * tables into a static device array on `stream` (no allocation); make the
 * first call on each device, and the first after a device reset, before any
 * stream capture.  All calls
 * share the one array, which keeps the previous call's contents: each call
 * re-initialises everything it reads, but calls whose work overlaps on the
 * GPU (other streams, other host threads) race on it and must be serialised
 * by the caller. */
int seeds_run_static(const seeds_params *p, const uint8_t *d_rgb, int64_t row_stride_bytes, int32_t *d_labels_out,
                     int32_t *d_status, void *stream);

/* ---- test hooks --------------------------------------------------------- */

/* Operation list of image i (the schedule of Sec. 5.1-5.3, Sec. 6.5 for the
 * means iterations): op 0 quantises and builds the grid and the
 * histograms; then one op per phase (level L..0, iteration, phase 0..3)
 * with one descent op after each block level; with means_iters > 0 an op
 * that sums every superpixel's colour codes and coordinates, then one op per
 * means-based pixel phase; the last op is the output (only run by
 * seeds_batch_run).  kind: 0 init, 1 phase, 2 descend, 3 output, 5 start of
 * the means iterations, 6 means-based phase. */
int seeds_debug_num_ops(const seeds_ctx *c, int32_t i, int32_t *n_ops);
/* Kind, level and parity phase of op `op` of image i (Sec. 5.2-5.3). */
int seeds_debug_op_info(const seeds_ctx *c, int32_t i, int32_t op, int32_t *kind, int32_t *level, int32_t *phase);

/* Run ops [op_begin, op_end) of every image (clamped to each image's list)
 * from the current device state; inputs as seeds_batch_iterate.  A single
 * op is one parity phase of the hill climbing (Sec. 5.2-5.3), a descent, the
 * initialisation (Sec. 5.1) or the output. */
int seeds_debug_run_ops(seeds_ctx *c, const uint8_t *const *h_rgb_ptrs, const int64_t *h_row_strides, int32_t op_begin,
                        int32_t op_end, void *stream);

/* Synchronous read of image i's state (the labels, the colour histograms of
 * Sec. 4 and the superpixel sizes |A_k| of Prop. 1) into host buffers (any
 * may be NULL):
 * h_labels: the label grid of `level` (level 0 = pixels, H x W; level l >=
 * 1: its block grid), h_hist: K x B^3 int32 label-major, h_sizes: K int32,
 * h_bins: H x W int32. */
int seeds_debug_read_state(seeds_ctx *c, int32_t i, int32_t level, int32_t *h_labels, int32_t *h_hist, int32_t *h_sizes,
                           int32_t *h_bins);

/* Replace image i's labels at `level` (host int32 grid as above, values in
 * [0,K)) and recount its histograms (Sec. 4) and sizes on the device from
 * the current bin map, so that the next op judges from that partition
 * (Sec. 5.3).  Synchronous. */
int seeds_debug_set_labels(seeds_ctx *c, int32_t i, int32_t level, const int32_t *h_labels);

/* Set the context's device error word (host-side fault injection: the next
 * seeds_status() must report SEEDS_ERR_DEVICE).  No counterpart in the
 * paper. */
int seeds_debug_inject_error(seeds_ctx *c);

/* Failure test of the device-side wait: the grid barrier of this context's
 * next launches gives up after timeout_ns nanoseconds instead of 2 s (0 =
 * the default), and, with withhold_step >= 0, CTA 0 does not arrive at the
 * barrier that ends step withhold_step, so that every CTA's wait there runs
 * out: each sets the error word (SEEDS_ERR_DEVICE at the next seeds_status)
 * and leaves the kernel; no output is written.  (0, -1) restores normal
 * launches.  No GPU fault is involved, and the paper has no counterpart. */
int seeds_debug_barrier_test(seeds_ctx *c, int64_t timeout_ns, int32_t withhold_step);

/* Kernel launches issued by the context so far (every launch of the
 * persistent kernel and of the small pointer-upload kernel counts one).  No
 * counterpart in the paper. */
int seeds_debug_launch_count(const seeds_ctx *c, int64_t *n);

/* ---- profiling ---------------------------------------------------------- */

/* enable != 0: record a CUDA event pair on the launch stream around every
 * persistent-kernel launch of this context (off by default).  Profiling has
 * no counterpart in the paper. */
int seeds_profile_enable(seeds_ctx *c, int32_t enable);

/* Device time in ms of the context's most recent persistent-kernel launch
 * (waits for it).  SEEDS_ERR_INVALID if profiling was off for it.  No
 * counterpart in the paper. */
int seeds_profile_last_ms(seeds_ctx *c, float *ms);

/* Step stamps of the most recent profiled persistent launch: *n = 1 +
 * steps values (ns since the kernel began, read on the device's global
 * timer by one thread): [0] start, [1+s] the end of step s (one op of every
 * image, Sec. 5.2-5.3).  Call with h_ns = NULL to get *n. */
int seeds_profile_steps(seeds_ctx *c, int64_t *h_ns, int32_t cap, int32_t *n);

#ifdef __cplusplus
}
#endif

#endif /* SEEDS_H */
