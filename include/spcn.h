/*
 * spcn.h -- C ABI of the B300 (sm_103a) implementation of the improved
 * structure-preserving colour normalisation (SPCN) of Ramakrishnan, Anand &
 * Sethi, "Fast GPU-Enabled Color Normalization for Digital Pathology"
 * (arXiv 1901.03088).
 *
 * The per-pixel path, by the paper's steps:
 *   Eq. 1      optical density  v = log(i0 / i), with the channel-wise,
 *              image-wise i0 of §3.1 item 1;
 *   Eq. 2      two-stain sparse NMF: the basis W from sampled non-white
 *              pixels (§3.1 item 2, §3.2 item 2), and for every pixel the
 *              stain densities h = argmin_{h>=0} 1/2||v - W h||^2 + lambda|h|_1;
 *   Eq. 3      per-stain scaling by the ratio of 99th percentiles, taken over
 *              non-white pixels (§3.1 item 2);
 *   Eq. 4      inverse optical density i' = i0 exp(-v');
 *   §3.1 item 3  hematoxylin is the column with the larger OD(red)-OD(blue).
 *
 * Conventions shared by every entry point
 *   - Images are 8-bit RGB, interleaved (R,G,B per pixel), row-major, in
 *     DEVICE memory unless the entry point says otherwise.  Row y starts at
 *     data + y * pitch_bytes; pitch_bytes >= 3 * width.  Rows whose start
 *     (and, for outputs, destination) is 16-byte aligned take the vector
 *     path; any other layout is accepted and handled byte by byte.
 *     Limits: width * height < 2^36 pixels and height * ceil(width / 16)
 *     < 2^32 (chunk indices are 32-bit); larger images are INVALID_ARG.
 *   - The caller owns every image, output and density buffer.  The library
 *     never frees caller memory; it allocates only the scratch held by the
 *     context (grown on demand, released by spcn_context_destroy).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is stream-ordered.  An entry point blocks the host
 *     only when it returns results in host memory (documented per call).
 *   - Return value: SPCN_OK (0) or a negative spcn_status.  On error the
 *     output buffers hold unspecified contents.  Conditions found on the
 *     device by an asynchronous call (no tissue, a wait that gave up) are
 *     returned by the next call that synchronises: spcn_synchronize() or
 *     any call returning host results.
 *   - A context is bound to one device and is not thread-safe; use one
 *     context per host thread.
 */
#ifndef SPCN_H
#define SPCN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SPCN_OK = 0,
  SPCN_ERR_INVALID_ARG = -1,      /* null/misaligned pointer, bad size or parameter */
  SPCN_ERR_CUDA = -2,             /* a CUDA runtime call failed */
  SPCN_ERR_OOM = -3,              /* device scratch allocation failed */
  SPCN_ERR_NO_TISSUE = -4,        /* no non-white pixel where one is needed */
  SPCN_ERR_DEGENERATE_BASIS = -5, /* stain vectors (nearly) parallel or vanished */
  SPCN_ERR_TIMEOUT = -6,          /* a grid-wide wait gave up (kernel returned) */
  SPCN_ERR_SCRATCH_LIMIT = -7     /* request larger than spcn_estimate_basis_noalloc's fixed scratch */
} spcn_status;

typedef enum {
  SPCN_SAMPLE_ALL = 0,      /* every pixel, raster order */
  SPCN_SAMPLE_HASH = 1,     /* round(rate*N) SplitMix64 draws with replacement */
  SPCN_SAMPLE_PATCHES = 2   /* patches at least half non-white (§3.2 item 2) */
} spcn_sample_mode;

/* Variants of the method, bits of spcn_params.flags.  With no bit set the
 * library computes the improved method as the rest of this header describes
 * it; each bit restores one of the paper's earlier choices (for A/B
 * comparisons).  Unknown bits are rejected with SPCN_ERR_INVALID_ARG.
 *
 * SPCN_FLAG_I0_255: spcn_estimate_basis (and the estimation inside
 *   spcn_normalize_estimated) sets i0 = 255 for every channel, the original
 *   method's fixed maximum intensity (§2.1 Eq. 1), instead of the P80 of the
 *   bright sample pixels (§3.1 item 1).
 * SPCN_FLAG_ORDER_BLUE: the stains are ordered by the original heuristic
 *   that §3.1 item 3 replaces: hematoxylin is the column with the larger
 *   blue optical density (ties keep the learnt order).
 * SPCN_FLAG_P99_SAMPLED: spcn_normalize and spcn_normalize_estimated scale
 *   with the source percentile that basis estimation reports (over the
 *   sub-sampled non-white pixels, §3.1 item 2; or the patch median below)
 *   instead of the exact whole-image percentile: pass 1 is skipped and the
 *   step reads and writes each pixel once.  spcn_normalize takes that value
 *   from src_st->p99 (> 0 where a stain is present; 0 gives scale 1).
 * SPCN_FLAG_P99_PATCH_MEDIAN: basis estimation reports, per stain, the
 *   median over the kept patches of each patch's non-white percentile
 *   (§3.2 item 4) as p99.  Requires SPCN_SAMPLE_PATCHES and n_patches <= 4096.
 * SPCN_FLAG_H_PINV: the densities that are measured, scaled and reconstructed
 *   are H = pinv(W) v (§2.1) instead of the non-negative lasso of Eq. 2: in
 *   the reported and exact percentiles, spcn_stain_densities, and both
 *   passes.  They are signed, so a percentile can be negative; outputs above
 *   255 are clamped.  The basis itself is still learnt with Eq. 2.  Not
 *   available for batches and the float (differentiable) entry points.
 * SPCN_FLAG_I0_OUT_255: Eq. 4 reconstructs with the neutral white 255 in
 *   every channel instead of the target's i0 (so background maps to white,
 *   not to the target's background tint); in spcn_normalize,
 *   spcn_normalize_estimated, batches and the float entry points.
 */
#define SPCN_FLAG_I0_255 0x1u
#define SPCN_FLAG_ORDER_BLUE 0x2u
#define SPCN_FLAG_P99_SAMPLED 0x4u
#define SPCN_FLAG_P99_PATCH_MEDIAN 0x8u
#define SPCN_FLAG_H_PINV 0x10u
#define SPCN_FLAG_I0_OUT_255 0x20u

/* An 8-bit interleaved RGB image. */
typedef struct {
  const uint8_t* data;      /* device pointer to pixel (0,0) */
  int32_t width;            /* pixels per row, >= 1 */
  int32_t height;           /* rows, >= 1 */
  int64_t pitch_bytes;      /* bytes between row starts, >= 3*width */
} spcn_image;

/* Method parameters; spcn_params_default() gives the paper's constants. */
typedef struct {
  float lambda;             /* Eq. 2 sparsity weight (0.1, §2.1), >= 0 */
  int32_t white_thresh;     /* bright: all channels > t; non-white otherwise (220, §3.1) */
  float i0_pct;             /* percentile of bright pixels taken as i0 (80, §3.1 item 1) */
  float stain_pct;          /* stain-density percentile of Eq. 3 (99) */
  int32_t i0_max_samples;   /* cap on bright pixels used for i0 (100000, §3.1 item 1) */
  int32_t sample_mode;      /* spcn_sample_mode used by spcn_estimate_basis */
  float sample_rate;        /* SPCN_SAMPLE_HASH: fraction of pixels drawn (0.01) */
  int32_t n_patches;        /* SPCN_SAMPLE_PATCHES: patches kept (<= 4*n_patches tried) */
  int32_t patch_size;       /* SPCN_SAMPLE_PATCHES: patch side in pixels */
  int32_t max_iter;         /* dictionary-learning iteration cap (200) */
  float tol;                /* stop when max|dW| < tol (1e-6) */
  uint32_t flags;           /* SPCN_FLAG_* variants (0: the improved method) */
  uint64_t seed;            /* SplitMix64 seed of the sampling */
} spcn_params;

/* Per-image statistics: everything the per-pixel passes need.  A plain host
 * record; it can be stored and reused (e.g. one target for many sources). */
typedef struct {
  float W[6];               /* basis, column-major 3x2: W[0..2] = hematoxylin OD
                               (R,G,B), W[3..5] = eosin OD; entries >= 0 */
  float i0[3];              /* background intensity per channel, in [1, 255] */
  double p99[2];            /* Eq. 3 percentile of each stain's density.  From
                               spcn_estimate_basis: over the sampled non-white
                               pixels (§3.1 item 2); from spcn_stain_percentile:
                               exact over all non-white pixels of the image */
  int32_t iters;            /* dictionary-learning iterations run */
  int32_t status;           /* spcn_status of the call that produced the record */
  int64_t n_sample;         /* pixels in the basis sample */
  int64_t n_nonwhite;       /* non-white pixels in the sample */
  int64_t n_bright;         /* bright pixels in the sample */
  double objective;         /* Eq. 2 objective (1/2-scaled) at the last H-step */
} spcn_stats;

/* Fill *p with the paper's constants: lambda 0.1, threshold 220, i0 from the
 * 80th percentile of <= 100000 bright pixels, 99th-percentile scaling, hash
 * sampling at 1%, 200 patches of 256 px, 200 iterations, tol 1e-6, seed 0. */
void spcn_params_default(spcn_params* p);

/* Create a context on CUDA device `device`.  Allocates the fixed scratch
 * (a few tens of MB) on that device.  *ctx is set on success. */
int spcn_context_create(void** ctx, int device);

/* Release the context and all its device scratch.  NULL is accepted. */
int spcn_context_destroy(void* ctx);

/* Basis estimation (§3.1 items 1-3, §3.2 item 2, Eq. 2): sample pixels by
 * params->sample_mode, estimate i0 (P80 of <= i0_max_samples bright sample
 * pixels), run the sparse NMF on the sample's non-white pixels, order the
 * stains by OD(red)-OD(blue), and set p99 to the percentile of the sampled
 * non-white pixels' densities (SPCN_FLAG_I0_255, SPCN_FLAG_ORDER_BLUE and
 * SPCN_FLAG_P99_PATCH_MEDIAN select the paper's earlier choices for these).  Writes the host record *out.  Blocks the
 * host until the stream has finished this call's work.
 * Errors: INVALID_ARG, NO_TISSUE (no non-white sample pixel or patch),
 * DEGENERATE_BASIS, TIMEOUT, CUDA, OOM. */
int spcn_estimate_basis(void* ctx, const spcn_image* img, const spcn_params* params,
                        spcn_stats* out, void* stream);

/* Exact Eq. 3 percentile (params->stain_pct) of each stain's density over
 * all non-white pixels of `img`, for the basis and i0 in *st (st->p99, if
 * positive, only guides the search window; SPCN_FLAG_P99_SAMPLED does not
 * apply to this call).  Writes p99_out[2] (host).
 * Blocks the host.  Errors: INVALID_ARG, NO_TISSUE, DEGENERATE_BASIS,
 * TIMEOUT, CUDA. */
int spcn_stain_percentile(void* ctx, const spcn_image* img, const spcn_stats* st,
                          const spcn_params* params, double* p99_out, void* stream);

/* Stain densities (Eq. 2 H-step for the basis and i0 in *st) of every pixel,
 * written planar to device memory: H[j * h_stride + y * width + x] for stain
 * j = 0 (hematoxylin), 1 (eosin); h_stride >= width*height.  Asynchronous. */
int spcn_stain_densities(void* ctx, const spcn_image* img, const spcn_stats* st,
                         const spcn_params* params, float* H, int64_t h_stride,
                         void* stream);

/* Stain separation of a whole image in one stream-ordered call (the
 * §4.3 use of the densities as a module of their own): the work of
 * spcn_estimate_basis, then spcn_stain_densities with the estimated basis
 * and i0, whose table stays on the device (no host round trip).  H, h_stride
 * as for spcn_stain_densities; the values are those of the two calls in
 * sequence.  If st_out (host) is non-NULL the call blocks and returns the
 * estimated statistics there (p99: the sample percentile); otherwise it is
 * asynchronous and an estimation error is returned by the next synchronising
 * call (the densities of a failed estimation are zeros).
 * Errors: as spcn_estimate_basis and spcn_stain_densities. */
int spcn_stain_densities_estimated(void* ctx, const spcn_image* img, const spcn_params* params,
                                   float* H, int64_t h_stride, spcn_stats* st_out,
                                   void* stream);

/* Normalise `src` to the target statistics (Eq. 1-4): pass 1 computes the
 * source's exact non-white P99 per stain on the device (src_st->p99 only
 * guides the search window), pass 2 recomputes every pixel's densities,
 * scales them by tgt_st->p99 / P99_src, mixes them with the target basis and
 * writes i0_tgt * exp(-v') rounded half-to-even into `out` (device, same
 * width/height as src, row pitch out_pitch >= 3*width; must not overlap
 * src).  If src_p99_out (host, 2 doubles) is non-NULL the call blocks and
 * returns the source percentiles there; otherwise it is asynchronous.
 * With SPCN_FLAG_P99_SAMPLED there is no pass 1: src_st->p99 (finite, and
 * >= 0 unless SPCN_FLAG_H_PINV) is the source percentile.
 * Errors: INVALID_ARG, DEGENERATE_BASIS, CUDA (and, when blocking,
 * NO_TISSUE/TIMEOUT). */
int spcn_normalize(void* ctx, const spcn_image* src, const spcn_stats* src_st,
                   const spcn_stats* tgt_st, const spcn_params* params,
                   uint8_t* out, int64_t out_pitch, double* src_p99_out, void* stream);

/* Basis estimation and normalisation of `src` in one stream-ordered call:
 * the work of spcn_estimate_basis followed by spcn_normalize with the
 * estimated statistics, except that the statistics stay on the device (the
 * source table is built from the estimated basis and i0, and the P99 search
 * window from the sample percentile) so there is no host round trip between
 * the two.  The search window covers a binomial band of the sample's order
 * statistics around the percentile.  The output bytes are those of the two
 * calls in sequence.
 * Without src_st_out the call puts only kernels and memsets into the stream,
 * every argument passed by value: once the context's sample buffers have the
 * size the call needs (after a first call with the same sampling) and with
 * kernel timing off, it can be captured into a CUDA graph; replays use the
 * pointers, parameters and target statistics of the capture.
 * If src_st_out (host) is non-NULL the call blocks and returns the estimated
 * source statistics there, with p99 = the percentile the scale used (the
 * exact one of the whole source; with SPCN_FLAG_P99_SAMPLED the sample's,
 * and no pass 1 runs); otherwise it is asynchronous and errors of the estimation (no
 * tissue, degenerate basis) are returned by the next synchronising call.
 * Errors: as spcn_estimate_basis and spcn_normalize. */
int spcn_normalize_estimated(void* ctx, const spcn_image* src, const spcn_stats* tgt_st,
                             const spcn_params* params, uint8_t* out, int64_t out_pitch,
                             spcn_stats* src_st_out, void* stream);

/* Wait for the context's work on `stream` and return the first error any
 * asynchronous call recorded on the device since the last synchronising
 * call (the record is then cleared). */
int spcn_synchronize(void* ctx, void* stream);

/* Differentiable normalisation of float images (Eq. 1-4 without the final
 * rounding), for training pipelines.  x and y: device FP32, planar
 * (batch, 3, height, width), intensities in [0, 255].  src_stats: one host
 * record per image (W, i0 and the exact p99 of that image's source); the
 * Eq. 3 scale tgt_stats->p99 / src p99 and both i0 are held constant.  wt:
 * device pointer to the target basis (6 floats, column-major like
 * spcn_stats.W), the variable the backward differentiates.  Asynchronous.
 * Errors: INVALID_ARG, DEGENERATE_BASIS, CUDA. */
int spcn_normalize_f32(void* ctx, const float* x, int32_t batch, int32_t height, int32_t width,
                       const spcn_stats* src_stats, const spcn_stats* tgt_stats, const float* wt,
                       const spcn_params* params, float* y, void* stream);

/* Backward of spcn_normalize_f32 for L = sum(gy * y): writes gx = dL/dx
 * (same layout as x) and gwt = dL/dW_target (device, 6 floats, column-major).
 * The densities are recomputed, not stored; through the lasso the derivative
 * follows each pixel's active set (inactive densities have zero derivative),
 * through Eq. 1 it is -1/x (0 where the clamp at 1 is active).  The W_target
 * sum is reduced in a fixed order (deterministic), in FP64, launch by launch
 * for batches larger than one launch; any batch the forward accepts is
 * accepted.  Asynchronous.  Errors: INVALID_ARG, DEGENERATE_BASIS, CUDA. */
int spcn_normalize_f32_backward(void* ctx, const float* x, const float* gy, int32_t batch,
                                int32_t height, int32_t width, const spcn_stats* src_stats,
                                const spcn_stats* tgt_stats, const float* wt,
                                const spcn_params* params, float* gx, float* gwt, void* stream);

/* Basis estimation for callers that cannot allocate device memory (no
 * counterpart in the paper; it exists for deployment).  Hosts that own all
 * GPU memory through their own pool, plugin hosts that forbid cudaMalloc, and
 * pipelines that must not call the allocator (it can stall the device) cannot
 * create a context.  This entry point needs none: it runs the same work as
 * spcn_estimate_basis on the current device, with all scratch taken from one
 * fixed array inside the library (about 6.8 MB, resident on every GPU that
 * loads the library until the process exits).  It allocates nothing.
 *   Limits: at most 524288 sample pixels (SPCN_SAMPLE_ALL: width*height;
 *   SPCN_SAMPLE_HASH: round(rate*N); SPCN_SAMPLE_PATCHES:
 *   n_patches*patch_size^2) and at most 4096 patches; larger requests return
 *   SPCN_ERR_SCRATCH_LIMIT without touching the device.  Invalid images or
 *   parameters return SPCN_ERR_INVALID_ARG before any size is derived.
 *   The first call on a device does a one-time set-up (resolves the array's
 *   device address, reads launch attributes); make that first call before
 *   any stream capture.  All calls share the one array, so calls that
 *   overlap on the GPU (other host threads, other streams) race; serialise
 *   them.  Blocks the host like spcn_estimate_basis; same other errors. */
int spcn_estimate_basis_noalloc(const spcn_image* img, const spcn_params* params,
                                spcn_stats* out, void* stream);

/* ------------------------------------------------------------------ batches
 * Batched normalisation (§3.2: a batch of source images normalised to one
 * target).  Many tiles of any sizes, each with its own source statistics (W,
 * i0; p99 only guides the search window, as in spcn_normalize), are
 * normalised to one target by a fixed short sequence of launches on one
 * stream, whatever the number of tiles.  Every tile's output bytes and
 * percentiles are identical to what spcn_normalize gives for that tile
 * alone; only the schedule differs.
 *
 * A batch object fixes the tile table (pointers, sizes, pitches, statistics,
 * outputs) and owns the device state of a run; spcn_batch_run can then be
 * repeated, and captured into a CUDA graph, as long as the buffers it names
 * stay allocated.  A run first sets each tile's window start from a sample
 * of the tile (one block per tile).  Work is then split into items of
 * `item_chunks` 16-pixel chunks: pass-1 items (densities, non-white count,
 * keys at or above the window start), then pass-2 items (reconstruction) of
 * tiles whose percentile is known.  The default schedule (SPCN_SCHED_STAGED)
 * runs pass 1, the per-tile selects and pass 2 as separate launches; the
 * other two run every item in one cooperative persistent launch, where the
 * last block to finish a tile's pass 1 selects its percentile.  Tiles whose
 * ranks fell below the window start are finished at the end of the run by an
 * exact radix select over the whole grid (a cooperative launch that returns
 * at once when no tile needs it). */

typedef enum {
  SPCN_SCHED_PHASED = 0,       /* all pass-1 items, then all pass-2 items */
  SPCN_SCHED_INTERLEAVED = 1,  /* groups of about group_px pixels: pass 1 of group g+1
                                  is queued before pass 2 of group g, so pass 2
                                  rereads recently read tiles */
  SPCN_SCHED_STAGED = 2,       /* separate launches, each with the whole shared memory
                                  and register budget of its pass: pass 1 of every
                                  tile (with the single-image chunk skips and
                                  per-warp stack), the per-tile selects, pass 2 of
                                  every tile, then the cooperative kernel for the
                                  exact fallback only.  Both passes split the chunks
                                  of all tiles (the tiles of one table adjacent)
                                  into equal contiguous shares, one per block, so
                                  item_chunks has no effect.  Needs fewer than
                                  2^32 chunks per tile (else INVALID_ARG) */
  SPCN_SCHED_PERSISTENT = 3    /* the staged schedule's steps (window starts, pass 1,
                                  the per-tile selects, pass 2) as phases of ONE
                                  cooperative persistent launch, one block per SM,
                                  separated by grid barriers; the cooperative
                                  fallback launch follows as in the staged
                                  schedule.  Needs the grid-wide select (at most
                                  1024 tiles) and the same block count for both
                                  passes (else INVALID_ARG); item_chunks has no
                                  effect */
} spcn_schedule;

typedef struct {
  int32_t item_chunks;   /* chunks (16 px) per work item, >= 1024; multiple of 1024 */
  int32_t schedule;      /* spcn_schedule */
  int64_t group_px;      /* SPCN_SCHED_INTERLEAVED: pixels per group */
  float ms;              /* spcn_batch_tune: measured mean time of one run */
  int32_t pad;
} spcn_batch_config;

/* Create a batch of n >= 1 tiles on ctx's device.  tiles[i], tile_stats[i],
 * outs[i] (device, out_pitches[i] >= 3 * width) describe tile i; tgt_st is
 * the one target.  The host arrays are copied; the device buffers are not
 * (the caller keeps them allocated while the batch is used).  An output must
 * not overlap its own source (INVALID_ARG); it must not overlap another
 * tile's source or output either (not checked: results are then undefined).
 * Builds the per-statistics tables (tiles with bitwise-equal W and i0 share
 * one) and allocates the batch state; blocks the host.  Every tile's
 * percentile is measured (SPCN_FLAG_P99_SAMPLED is rejected; the other flags
 * concern basis estimation and have no effect here).  Errors: INVALID_ARG,
 * DEGENERATE_BASIS, OOM, CUDA. */
int spcn_batch_create(void* ctx, int32_t n, const spcn_image* tiles,
                      const spcn_stats* tile_stats, const spcn_stats* tgt_st,
                      const spcn_params* params, uint8_t* const* outs,
                      const int64_t* out_pitches, void** batch);

/* Normalise every tile of the batch on `stream`: one memset of the batch
 * state, the window-start launch, then the launches of the configured
 * schedule (SPCN_SCHED_STAGED: pass 1, three select launches, pass 2 and the
 * cooperative fallback launch; the other schedules: one cooperative launch).
 * Asynchronous, allocates nothing and may be captured into a CUDA graph.
 * Errors: INVALID_ARG, CUDA. */
int spcn_batch_run(void* batch, void* stream);

/* Wait for the batch's last run on `stream` and read its results: p99_out
 * (host, 2n doubles, tile-major: tile i's stains at 2i, 2i+1), status_out
 * (host, n: SPCN_OK or SPCN_ERR_NO_TISSUE per tile) and fallback_out (host,
 * n: 1 where the tile's percentile needed the exact radix select over its
 * pixels because a rank lay below the window), each optional.  Returns
 * SPCN_ERR_TIMEOUT if a wait of the run gave up, else SPCN_OK. */
int spcn_batch_results(void* batch, double* p99_out, int32_t* status_out, int32_t* fallback_out,
                       void* stream);

/* Read or replace the batch's schedule (spcn_batch_set_config rebuilds the
 * work queue; blocks the host). */
int spcn_batch_get_config(void* batch, spcn_batch_config* cfg);
int spcn_batch_set_config(void* batch, const spcn_batch_config* cfg);

/* Autotuner: run the batch under each candidate schedule (item sizes x
 * phased / interleaved groups), one untimed run then `reps` timed runs each
 * (CUDA events on `stream`), keep the fastest.  trials (host, optional,
 * max_trials entries) receives every candidate with its mean time;
 * *n_trials the number written.  The outputs are rewritten by every run
 * (with the same bytes).  Blocks the host. */
int spcn_batch_tune(void* batch, int32_t reps, spcn_batch_config* trials, int32_t max_trials,
                    int32_t* n_trials, void* stream);

/* Release the batch's device state.  NULL is accepted. */
int spcn_batch_destroy(void* batch);

/* One-shot form: create, run, read the results, destroy.  p99_out and
 * status_out as in spcn_batch_results.  Blocks the host. */
int spcn_normalize_batched(void* ctx, int32_t n, const spcn_image* tiles,
                           const spcn_stats* tile_stats, const spcn_stats* tgt_st,
                           const spcn_params* params, uint8_t* const* outs,
                           const int64_t* out_pitches, double* p99_out, int32_t* status_out,
                           void* stream);

/* Number of kernels the context has launched since creation (for launch
 * accounting in benchmarks). */
int64_t spcn_launch_count(void* ctx);

/* Number of whole-image percentiles (Eq. 3's exact P99, §3.1 item 2) that
 * this context resolved with the exact radix select over the image because a
 * rank fell outside pass 1's window, since the context was created.  Waits
 * for the context's device.  Errors: INVALID_ARG, CUDA. */
int spcn_exact_fallbacks(void* ctx, int64_t* count);

/* Kernels whose launches can be timed (spcn_kernel_timing). */
typedef enum {
  SPCN_KERNEL_PASS1 = 0,    /* pass 1: densities, non-white count, P99 window histogram */
  SPCN_KERNEL_SELECT = 1,   /* exact radix select for ranks outside the window */
  SPCN_KERNEL_PASS2 = 2,    /* pass 2: densities, Eq. 3 scaling, Eq. 4, store */
  SPCN_KERNEL_DENSITY = 3,  /* density output pass */
  SPCN_KERNEL_F32_FWD = 4,  /* differentiable forward (float images) */
  SPCN_KERNEL_F32_BWD = 5,  /* differentiable backward (float images) */
  SPCN_KERNEL_BATCH = 6,    /* the launches of spcn_batch_run after the window start */
  SPCN_KERNEL_LADDER = 7,   /* window-miss recovery: counting passes over key ladders */
  SPCN_KERNEL_COUNT = 8
} spcn_kernel;

/* Enable (1) or disable (0) CUDA-event timing of the kernels above on the
 * streams they are launched on, and clear the accumulated times.  Timing
 * records two events per timed launch; it does not synchronise. */
int spcn_kernel_timing(void* ctx, int enable);

/* Total device time (ms) and number of timed launches of kernel `kernel`
 * since timing was enabled.  Waits for the recorded events. */
int spcn_kernel_times(void* ctx, int kernel, double* total_ms, int64_t* launches);

/* Static description of a status code. */
const char* spcn_strerror(int status);

/* Test hook for failure detection: launch a cooperative kernel whose grid
 * barrier waits for `extra_arrivals` more blocks than exist; the wait gives
 * up after timeout_ns, the kernel records SPCN_ERR_TIMEOUT and returns, and
 * the call (which blocks) returns that status.  extra_arrivals = 0 must
 * return SPCN_OK.  No fault or hang is ever raised. */
int spcn_debug_barrier_timeout(void* ctx, int32_t extra_arrivals, int64_t timeout_ns,
                               void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SPCN_H */
