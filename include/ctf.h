/*
 * ctf.h -- C ABI of the GB300 collaborative texture filtering library.
 *
 * Collaborative texture filtering (Akenine-Moller, Ebelin, Pharr, Wronski,
 * "Collaborative Texture Filtering", HPG 2025, arXiv 2506.17770): the 32
 * pixels of a warp find the texels their bilinear footprints need, each
 * needed texel is evaluated ("produced") once by one lane, and every pixel
 * gathers its four taps from the lanes that produced them (Sec. 3, the
 * three-step flow: collect, produce, gather and filter).  Warps whose texel
 * set is too large, or that contain a minified pixel, fall back to one-tap
 * stochastic texture filtering (STF, Sec. 3.4 opening).
 *
 * Conventions shared by every call:
 *  - Pixel arrays are row-major [height][width]:
 *      uv       float[2] per pixel, texture coordinates in [0,1]-normalised
 *               texture space (texel x covers u in [x/Wt, (x+1)/Wt));
 *      jac      float[4] per pixel = (du/dx, dv/dx, du/dy, dv/dy), the UV
 *               Jacobian in normalised UV per pixel;
 *      coverage uint8 per pixel, 0 = not covered (nullable = all covered);
 *      out_rgba float[4] per pixel (RGBA, values in [0,1]);
 *      out_evals uint8 per pixel: texel evaluations made by that pixel's lane.
 *  - Texel-space position of a pixel: (u*Wt - 0.5, v*Ht - 0.5), upper-left
 *    texel = floor, (s,t) = fraction (Appendix code, first lines), each a
 *    single IEEE float32 operation.
 *  - A pixel is active when it is inside the frame, covered, and its
 *    texel-space position is finite with magnitude below 2^22; inactive
 *    pixels get RGBA (0,0,0,0) and 0 evaluations.
 *  - Warp tiles are tile_w x tile_h pixels (tile_w*tile_h = 32) aligned to
 *    the frame origin; lane = ty*tile_w + tx.  Partial tiles at the right
 *    and bottom edges have inactive lanes.
 *  - Device pointers are CUDA device (or managed) memory on the current
 *    device; "host" entry points take host memory.  The library never keeps
 *    a caller pointer after a call returns.  The stream is borrowed; NULL is
 *    the legacy default stream.
 *  - Every function returns CTF_OK (0) or a negative ctf_status.  Arguments
 *    are validated before any work is queued; errors of kernels already
 *    queued show up as CTF_ERR_CUDA on a later synchronising call.
 *    ctf_last_error() gives a thread-local message for the last failure.
 */
#ifndef CTF_H
#define CTF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CTF_OK = 0,
    CTF_ERR_ARG = -1,         /* bad argument (null, size, enum, shape) */
    CTF_ERR_ALIGN = -2,       /* pointer not aligned as documented */
    CTF_ERR_UNSUPPORTED = -3, /* combination not built */
    CTF_ERR_OOM = -4,         /* device allocation failed */
    CTF_ERR_CUDA = -5,        /* CUDA runtime error */
    CTF_ERR_TIMEOUT = -6,     /* a bounded device wait gave up */
    CTF_ERR_CORRUPT = -7,     /* corrupt or mismatched file */
    CTF_ERR_BOUNDS = -8       /* debug build: a kernel index fell outside its buffer */
} ctf_status;

/* Filtering algorithm.
 *  CTF_ALG_4TAP        per-pixel bilinear: every pixel evaluates its 4 texels
 *                      (the reference every collaborative success must equal).
 *  CTF_ALG_STF         one-tap STF for every pixel (Sec. 3.4 opening).
 *  CTF_ALG_LIST_MERGE  exact union of the wave's 2x2 texel lists (Sec. 3.1).
 *  CTF_ALG_BOX         bounding box of the wave's footprints, texel i at
 *                      (i mod w, i div w) from its corner (Sec. 3.2).
 *  CTF_ALG_MASK        bit mask over the bounding box, texel i = i-th set bit
 *                      h(i,B) (Sec. 3.3, Fig. 3); mask_dim 16 or 11. */
typedef enum {
    CTF_ALG_4TAP = 0,
    CTF_ALG_STF = 1,
    CTF_ALG_LIST_MERGE = 2,
    CTF_ALG_BOX = 3,
    CTF_ALG_MASK = 4
} ctf_algorithm;

/* How a texel value is produced ("texel evaluation", Sec. 3, step 2). */
typedef enum {
    CTF_EVAL_BLOCK = 0,    /* exact decode of 4x4-texel blocks */
    CTF_EVAL_MLP_FP16 = 1, /* learned decode, FP16 MLP over latent grids */
    CTF_EVAL_MLP_FP8 = 2   /* learned decode, FP8 E4M3 with per-channel scales */
} ctf_eval_mode;

typedef struct ctf_texture_s *ctf_texture;

/* Texture description for ctf_texture_create.
 * CTF_EVAL_BLOCK: width and height multiples of 4 in [4, 65536]; blocks
 *   points to (width/4)*(height/4) records of 8 bytes, row-major by block:
 *   bytes 0-1 endpoint c0 (RGB565, little endian), bytes 2-3 endpoint c1,
 *   bytes 4-7 the 2-bit palette indices, texel (x&3, y&3) at bits
 *   2*(4*(y&3)+(x&3)).  Decode: endpoints bit-replicated to 8 bits, palette
 *   c0, c1, (2c0+c1+1)/3, (c0+2c1+1)/3 per channel, alpha 255; value = v/255
 *   correctly rounded.  The paper leaves the format open ("a texel stored in
 *   a custom format", Sec. 3); this one is the library's.
 *   blocks may be host or device memory; it is copied. */
typedef struct {
    int width, height;
    ctf_eval_mode mode;
    const void *blocks;
} ctf_texture_desc;

/* Filter options; NULL means the defaults in brackets.
 *   tile_w, tile_h  warp pixel tile, 8x4, 4x8 or 16x2            [8 x 4]
 *   budget          texels one warp may produce, 1..32 (one per lane,
 *                   Sec. 3 "at most one texel evaluation per lane"), up to
 *                   64 with two texels per lane                 [32]
 *   mask_dim        Mask Sampling mask side, 16 or 11 (Sec. 3.3)  [16]
 *   edge_remap      1: producer of texel i is the i-th active lane h(i,A)
 *                   (supplemental Sec. 2), success needs n <= popcount(A);
 *                   0: lane i produces texel i and lanes 0..n-1 must be
 *                   active                                        [1]
 *   group_dedup     learned textures, algorithms other than 4TAP: the
 *                   texels a CTA's group of 8 consecutive warp tiles
 *                   (tile index order) produces are evaluated once per
 *                   distinct (clamped) texel instead of once per warp, the
 *                   shared-memory extension of Sec. 3 that Sec. 6 proposes;
 *                   outputs and out_evals are unchanged, ctf_stats
 *                   texel_evals_unique counts the evaluations done.  0 or 1
 *                                                                 [0]
 *   fallback        magnified tiles over budget: 0 one-tap STF, 1 fallback
 *                   C, 2 fallback C+ (Sec. 3.4: every active lane draws its
 *                   STF texel; C produces them, C+ produces the distinct
 *                   ones and spends the other lanes on further texels of
 *                   the footprints (eq. 2); each pixel blends the produced
 *                   texels of its footprint by eq. 1).  Minified tiles take
 *                   one-tap STF.  Block and learned textures (on learned
 *                   ones not together with group_dedup, and in
 *                   ctf_filter_batch block views only)            [0]
 *   texels_per_lane 0 or 1: one texel evaluation per lane; 2: up to two
 *                   (Sec. 5: at magnification 1 an 8x4 wave needs at most
 *                   54 texels, so two per lane always succeed once every
 *                   pixel is magnified).  Texel i is evaluated for lane
 *                   h(i mod na, A) (or lane i mod 32 without edge
 *                   remapping), whose count becomes 2 when it has two;
 *                   success needs n <= 2 popcount(A).  Block and learned
 *                   textures (as for fallback)                    [1]
 *   filter          0 bilinear (2x2 footprint); 1 cubic B-spline, 2
 *                   Catmull-Rom (4x4 footprint, Sec. 4.2: the same
 *                   algorithms with the footprint, weights and mask bits of
 *                   the larger filter; one-tap STF draws a tap per axis by
 *                   |w|, scaled by the signed sums for Catmull-Rom's
 *                   negative lobes).  The bicubic filters take one texel per
 *                   lane and the STF fallback, block textures, single views
 *                   (CTF_ERR_UNSUPPORTED otherwise)            [0] */
typedef struct {
    int tile_w, tile_h;
    int budget;
    int mask_dim;
    int edge_remap;
    int group_dedup;
    int fallback;
    int texels_per_lane;
    int filter;
} ctf_filter_opts;

/* Per-call counters (filled only when a stats pointer is given). */
typedef struct {
    int64_t tiles_total;             /* warp tiles in the frame */
    int64_t tiles_empty;             /* tiles with no active pixel */
    int64_t tiles_direct;            /* tiles filtered by 4TAP or STF algorithms */
    int64_t tiles_success;           /* collaborative tiles on the success path */
    int64_t tiles_fallback_budget;   /* collaborative tiles over budget -> STF */
    int64_t tiles_fallback_minified; /* collaborative tiles with a minified pixel -> STF */
    int64_t pixels_active;
    int64_t texel_evals;             /* sum of out_evals */
    int64_t texel_evals_unique;      /* texel evaluations done: texel_evals,
                                        less the repeats group_dedup removed */
} ctf_stats;

/* Library and device information. */
const char *ctf_version(void);
const char *ctf_status_string(int status);
/* Thread-local message of the last failing call on this thread ("" if none). */
const char *ctf_last_error(void);

/* Create a texture; the library copies the data into its own device memory
 * on the current device.  *out receives the handle.  Errors: CTF_ERR_ARG,
 * CTF_ERR_UNSUPPORTED (mode not built), CTF_ERR_OOM, CTF_ERR_CUDA. */
int ctf_texture_create(const ctf_texture_desc *desc, ctf_texture *out);

/* Destroy a texture (synchronises the device first).  NULL is accepted. */
int ctf_texture_destroy(ctf_texture tex);

/* Filter one view (Sec. 3 flow for the collaborative algorithms).
 *   uv [H][W][2], jac [H][W][4], coverage [H][W] (nullable): device memory;
 *   uv 8-byte and jac 16-byte aligned (else CTF_ERR_ALIGN).
 *   width, height in [0, 32768] (0 = nothing to do).
 *   view_id: third word of the STF counter (px, py, view_id, 0).
 *   seed: Philox4x32-10 key (low word, high word) of the STF choice; pixel
 *   (px,py) takes the right neighbour when (r0>>8)*2^-24 < s and the lower
 *   one when (r1>>8)*2^-24 < t, so each tap is chosen with probability equal
 *   to its bilinear weight (Sec. 3.4 opening).
 *   out_rgba [H][W][4] device, 16-byte aligned; out_evals [H][W] device or
 *   NULL.
 *   stats: host pointer or NULL; when given, the call waits for the stream
 *   and fills it.
 *   stream: cudaStream_t or NULL.
 * The call is asynchronous unless stats is given. */
int ctf_filter(ctf_texture tex, const float *uv, const float *jac, const uint8_t *coverage, int width,
               int height, int view_id, ctf_algorithm alg, uint64_t seed, const ctf_filter_opts *opts,
               float *out_rgba, uint8_t *out_evals, ctf_stats *stats, void *stream);

/* ctf_filter on HOST buffers: copies uv, jac (and coverage) to device memory
 * that the library owns and reuses, filters, copies the image and counts
 * back, and waits for the stream before returning.  Host buffers that are
 * page-locked (cudaHostAlloc / cudaHostRegister) are not copied at all:
 * the kernel reads the inputs and writes the image in host memory in place (over NVLink-C2C on a Grace-Blackwell node), and the
 * counts come back in one copy from library-owned device memory (so
 * out_evals_host need not be page-locked).  Otherwise, views of at least 2^20 pixels (without group_dedup) go
 * in 4 bands of whole tile rows, so that the copy-in of one band, the
 * filtering of the previous one and the copy-out of the one before overlap
 * (two library-owned copy streams; the filter runs on `stream`); each band
 * is filtered as the part of the view it is.  The results always equal
 * those of ctf_filter on the whole view. */
int ctf_filter_host(ctf_texture tex, const float *uv_host, const float *jac_host, const uint8_t *coverage_host,
                    int width, int height, int view_id, ctf_algorithm alg, uint64_t seed,
                    const ctf_filter_opts *opts, float *out_rgba_host, uint8_t *out_evals_host,
                    ctf_stats *stats, void *stream);

/* Learned texel decode (the paper's costly texel evaluation, Sec. 4.3.1:
 * a neural decompressor run "on sample").  Texel (x, y) of a W x H texture
 * is decoded as
 *   f    = concat over grids g = 0, 1 of the bilinear sample of latent grid
 *          L_g (latent_w[g] x latent_h[g] texels, 8 channels, clamp-to-edge)
 *          at grid position ((x+0.5)*latent_w[g]/W - 0.5, (y+0.5)*latent_h[g]/H - 0.5)
 *   h1   = relu(W1 f + b1), h2 = relu(W2 h1 + b2)       (16 -> 64 -> 64)
 *   rgba = clamp(W3 h2 + b3, 0, 1)                     (64 -> 4)
 * on the tensor cores, FP32 accumulation.  CTF_EVAL_MLP_FP16: latents and
 * weights rounded to FP16 (nearest), activations FP16.  CTF_EVAL_MLP_FP8:
 * latents FP16; every layer input k is scaled by a_k = act_absmax_k / 448
 * and rounded to E4M3 (nearest, saturating); weights W'[o][k] = W[o][k]*a_k
 * are stored as E4M3 after division by s_o = max_k |W'[o][k]| / 448, and the
 * layer output is s_o * sum_k + b_o.  Biases stay FP32.
 * All arrays are FP32, row-major, host or device memory; they are copied and
 * quantised by the library.  latent[g] is [latent_h][latent_w][8]; w1 [64][16],
 * w2 [64][64], w3 [4][64] (output x input); act_absmax[l] (FP8 only) holds
 * the largest |input| of layer l per input channel (16, 64, 64 values). */
typedef struct {
    int width, height;
    ctf_eval_mode mode;
    int latent_w[2], latent_h[2];
    const float *latent[2];
    const float *w1, *b1, *w2, *b2, *w3, *b3;
    const float *act_absmax[3];
} ctf_mlp_desc;

/* Create a learned-decode texture (copies and quantises the parameters).
 * Errors: CTF_ERR_ARG (sizes, NULL or non-finite values), CTF_ERR_OOM,
 * CTF_ERR_CUDA.  ctf_filter on such a texture runs every algorithm with the
 * learned decode as texel evaluation; alpha comes from the network. */
int ctf_texture_create_mlp(const ctf_mlp_desc *desc, ctf_texture *out);

/* The parameters exactly as stored, as floats, into caller-owned host
 * arrays (any pointer may be NULL): latents (FP16 values), weights (FP16
 * values, or E4M3 values before scaling), biases, and for FP8 the weight
 * scales s (64, 64, 4) and activation scales a (16, 64, 64).  The effective
 * FP8 weight is s_o * q[o][k] / a_k. */
typedef struct {
    float *latent[2];
    float *w1, *b1, *w2, *b2, *w3, *b3;
    float *weight_scale[3];
    float *act_scale[3];
} ctf_mlp_params;
int ctf_mlp_export(ctf_texture tex, const ctf_mlp_params *out);

/* Decode n texels of a learned-decode texture: xy is int32 [n][2] (x, y),
 * clamped to the texture; out_rgba float [n][4].  Device memory, xy 8-byte
 * and out 16-byte aligned.  Asynchronous on the stream. */
int ctf_mlp_decode(ctf_texture tex, const int32_t *xy, int n, float *out_rgba, void *stream);

/* Wait for the stream and report any failure of work queued on it:
 * CTF_ERR_CUDA for CUDA errors, CTF_ERR_TIMEOUT if a kernel of this library
 * on the current device gave up a bounded wait since the last check,
 * CTF_ERR_BOUNDS if (debug build) a kernel index fell outside its buffer
 * (the record is then cleared). */
int ctf_sync_check(void *stream);

/* The same as ctf_sync_check, under the name of the problem statement's
 * interface (asynchronous device errors are reported by the next call or
 * by this one). */
int ctf_stream_status(void *stream);

/* Self-test of the bounded waits: one CTA waits on an mbarrier that nothing
 * arrives on, gives up after `polls` tries (1..2^24) as the library's kernels
 * do when an MMA does not complete, and records CTF_ERR_TIMEOUT, which the
 * next ctf_sync_check reports (and clears).  The context stays usable.
 * Returns CTF_ERR_ARG for polls outside the range, else the launch status. */
int ctf_selftest_bounded_wait(uint32_t polls, void *stream);

/* Host-side fault injection for tests (the paper has no counterpart).  Every
 * device allocation the library makes (textures, trainers, batch plans, the
 * staging and stats scratch, the decode tables) goes through one internal
 * routine.  ctf_debug_device_allocations returns how many times it has been
 * called in this process, failed attempts included; a test reads it before
 * and after a call to show that the call allocated nothing.
 * ctf_debug_live_allocations returns how many of them succeeded and have not
 * been freed yet (a call that fails must leave it as it found it).
 * ctf_debug_fail_allocations(skip, n) lets the next `skip` allocations
 * through and makes the n after them fail as if the device were out of
 * memory, without calling CUDA: the entry point that needed the memory
 * returns CTF_ERR_OOM after freeing what it had taken, and the CUDA context
 * stays usable.  n = 0 disarms it; negative arguments return CTF_ERR_ARG.
 * Both are thread-safe. */
int64_t ctf_debug_device_allocations(void);
int64_t ctf_debug_live_allocations(void);
int ctf_debug_fail_allocations(int skip, int n);

/* Debug build.  The library also builds as libctf_debug.so (compiled with
 * -DCTF_DEBUG): the same entry points and results, and every data-dependent
 * index its kernels use to reach a texel (block or latent cell), a pixel of
 * the view, or an entry of a shared-memory table (decode tables, rank
 * slots, List Merge and fallback tables, texel lists, chain rows, per-pixel
 * words) is checked against its buffer first.  An index outside it is
 * recorded in the device error word and replaced by 0, so the access stays
 * inside the buffer and the kernel runs on to its end (no trap); the next
 * ctf_sync_check returns CTF_ERR_BOUNDS, and ctf_last_error names the site,
 * the index and the bound of the first record.
 * ctf_debug_build returns 1 in that library and 0 in the release one.
 * ctf_debug_selftest_bounds(index, stream) has one thread read element
 * `index` of a 32-int shared array through the same check: in the debug
 * library an index outside [0, 32) is recorded (site "self-test") and 0 is
 * read instead, so the next ctf_sync_check returns CTF_ERR_BOUNDS; the
 * release library does no unchecked read and returns CTF_ERR_UNSUPPORTED
 * without launching.  Otherwise returns the launch status. */
int ctf_debug_build(void);
int ctf_debug_selftest_bounds(int index, void *stream);

/* Training of the learned decode on texels of an exact block texture (the
 * decoder the network stands in for, which also judges its error).  A
 * trainer holds FP32 master parameters (latents, weights, biases) and Adam
 * moments on the device.  One step draws `batch` texels with Philox4x32-10
 * (counter (i, step, 0x5A4D, 0), key = seed; x = (r0 * W) >> 32,
 * y = (r1 * H) >> 32), decodes their exact values as targets, and minimises
 * L = (1/batch) sum_i sum_c (y_ic - target_ic)^2 over the unclamped network
 * output, all four channels.  Gradients are summed in 64-bit fixed point
 * (2^-44 resolution), so every step is deterministic and a run resumed from
 * a checkpoint is bit-identical to an uninterrupted one.  Learning rates
 * decay linearly from lr_* to lr_* * lr_final_frac over `total_steps`.
 * The paper trains no network; this is the project's stand-in for the
 * neural decompressor of Sec. 4.3.1. */
typedef struct {
    int latent_w[2], latent_h[2]; /* latent grid sizes, e.g. W/4 x H/4 and W/8 x H/8 */
    int batch;                    /* texels per step, 1 .. 4194304 */
    int64_t total_steps;          /* length of the learning-rate schedule */
    float lr_weights, lr_latents; /* Adam step sizes */
    float lr_final_frac;          /* final fraction of the step sizes */
    float beta1, beta2, eps;      /* Adam */
    uint64_t seed;                /* sampling and initialisation */
} ctf_train_desc;

typedef struct ctf_trainer_s *ctf_trainer;

/* Create a trainer on an exact block texture (which must outlive it), with
 * seeded initial parameters: latents ~ N(0, 0.5^2), weights uniform in
 * +-sqrt(6 / fan_in), biases 0 except b3 = 0.5. */
int ctf_trainer_create(ctf_texture exact_src, const ctf_train_desc *desc, ctf_trainer *out);
int ctf_trainer_destroy(ctf_trainer tr);

/* Run `steps` optimisation steps on the stream (asynchronous). */
int ctf_trainer_step(ctf_trainer tr, int64_t steps, void *stream);

/* Steps taken so far. */
int64_t ctf_trainer_steps_done(ctf_trainer tr);

/* Loss and gradients for explicit texels without updating anything:
 * xy int32 [n][2] (device), targets from the exact texture.  Gradients go
 * to host arrays (any may be NULL) shaped like the parameters; loss to a
 * host double.  Synchronises the stream. */
typedef struct {
    float *latent[2];
    float *w1, *b1, *w2, *b2, *w3, *b3;
} ctf_mlp_arrays;
int ctf_trainer_gradients(ctf_trainer tr, const int32_t *xy, int n, double *loss, const ctf_mlp_arrays *grads,
                          void *stream);

/* Copy the FP32 master parameters to host arrays, or replace them from host
 * or device arrays (Adam moments are kept).  Synchronous. */
int ctf_trainer_get_params(ctf_trainer tr, const ctf_mlp_arrays *out);
int ctf_trainer_set_params(ctf_trainer tr, const ctf_mlp_arrays *in);

/* Quantise the current parameters into a learned-decode texture of the
 * given mode.  For CTF_EVAL_MLP_FP8 the activation ranges are measured on
 * the GPU over every texel of the texture first. */
int ctf_trainer_export(ctf_trainer tr, ctf_eval_mode mode, ctf_texture *out);

/* Checkpoint: parameters, Adam moments, step count and description in a
 * versioned binary file with an FNV-1a checksum.  Loading checks the
 * magic, version, sizes and checksum (CTF_ERR_CORRUPT on mismatch) and
 * needs the same exact source texture size. */
int ctf_trainer_save(ctf_trainer tr, const char *path);
int ctf_trainer_load(ctf_texture exact_src, const char *path, ctf_trainer *out);

/* Error of a learned-decode texture against an exact block texture of the
 * same size over every texel: mean squared error of RGB (alpha excluded)
 * and the largest absolute channel difference.  PSNR = -10 log10(mse).
 * Synchronous. */
int ctf_texture_compare(ctf_texture exact_ref, ctf_texture learned, double *mse_rgb, double *max_abs, void *stream);

/* One-call training of a learned texture on the exact decode of exact_src
 * (the paper's costly texel evaluation, Sec. 4.3.1, here a neural decoder
 * fitted to the block texture): a trainer with `desc` runs
 * desc->total_steps steps on the stream, its parameters are exported as a
 * learned texture of `mode` (*out_mlp, owned by the caller), that texture
 * is compared with exact_src over every texel, and the trainer is
 * destroyed.  report (nullable, host) receives the steps, texels sampled,
 * wall time and error.  Synchronous.  Errors: those of ctf_trainer_create,
 * ctf_trainer_step, ctf_trainer_export and ctf_texture_compare; nothing is
 * returned on failure. */
typedef struct {
    int64_t steps, texels;   /* optimisation steps and texels sampled */
    double seconds;          /* wall time of the steps, stream drained */
    double mse_rgb, max_abs; /* exported texture vs exact_src, every texel */
    double psnr_db;          /* -10 log10(mse_rgb) */
} ctf_train_report;
int ctf_mlp_train(ctf_texture exact_src, const ctf_train_desc *desc, ctf_eval_mode mode, ctf_texture *out_mlp,
                  ctf_train_report *report, void *stream);

/* Texture checkpoints: a block texture's blocks, or a learned texture's
 * stored (quantised) parameters, in a versioned binary file with an FNV-1a
 * checksum.  ctf_checkpoint_load reads and checks the whole file (magic,
 * version, mode, sizes, checksum: CTF_ERR_CORRUPT on a mismatch, CTF_ERR_ARG
 * if it cannot be read) before any device work, then builds a texture on
 * the current device that filters bit for bit like the saved one (*out,
 * owned by the caller).  Layout, little-endian: "CTFTEX01", uint32 version
 * 1, int32 mode, width, height, latent_w[0], latent_h[0], latent_w[1],
 * latent_h[1] (0 for block textures); the payload: the blocks, or float32
 * latent[0], latent[1], w1, b1, w2, b2, w3, b3 as stored and, for FP8,
 * weight_scale[0..2] and act_scale[0..2]; then the uint64 FNV-1a of every
 * byte before it. */
int ctf_checkpoint_save(ctf_texture tex, const char *path);
int ctf_checkpoint_load(const char *path, ctf_texture *out);

/* Batched filtering: many views, each with its own texture (block or
 * learned), size, magnification and buffers.  Views of at least solo_tiles
 * warp tiles run as their own launches of the single-view kernels (they fill
 * the GPU alone); the others share two persistent launches on the stream,
 * one per kind of texel evaluation (block views first).  Block views: CTAs
 * of 8 warps, every warp takes items of 32 warp tiles from an atomic
 * counter.  Learned views: CTAs of 4 warps that keep their tensor memory
 * for the whole launch take items of 8 warp tiles (4 for per-pixel 4-tap)
 * that share MLP chains, items_per_fetch at a time.  Every view is filtered
 * exactly as ctf_filter would filter it with the same options. */
typedef struct {
    ctf_texture tex;            /* block or learned-decode texture */
    const float *uv, *jac;      /* device, [height][width][2] and [4] */
    const uint8_t *coverage;    /* device or NULL */
    int width, height;          /* [0, 32768] */
    int view_id;                /* third word of the STF counter */
    float *out_rgba;            /* device [height][width][4] */
    uint8_t *out_evals;         /* device [height][width] or NULL */
} ctf_view;

/* Launch shape of a batch; NULL means the defaults in brackets.
 *   filter           tile shape, budget, mask_dim, edge_remap (as ctf_filter)
 *   items_per_fetch  learned views: items taken per fetch, 1..64      [4]
 *   ctas_per_sm      learned views: persistent CTAs per SM, 1..4       [4]
 *   solo_tiles       views of at least this many warp tiles get their own
 *                    launch; 0: every view in the persistent launches [16384]
 * (the block-view launch always fills every SM to its occupancy limit). */
typedef struct {
    ctf_filter_opts filter;
    int items_per_fetch;
    int ctas_per_sm;
    int solo_tiles;
} ctf_batch_opts;

/* Filter nviews (1..4096) views in one launch (asynchronous unless stats is
 * given, in which case the counters are summed over all views). */
int ctf_filter_batch(const ctf_view *views, int nviews, ctf_algorithm alg, uint64_t seed, const ctf_batch_opts *opts,
                     ctf_stats *stats, void *stream);

/* The same batch captured once into a CUDA graph (the solo launches, the
 * counter reset and both persistent launches) and replayed with
 * ctf_batch_graph_launch.  The views'
 * buffers are baked in: they must stay valid and at the same addresses. */
typedef struct ctf_batch_graph_s *ctf_batch_graph;
int ctf_batch_graph_create(const ctf_view *views, int nviews, ctf_algorithm alg, uint64_t seed,
                           const ctf_batch_opts *opts, ctf_batch_graph *out);
int ctf_batch_graph_launch(ctf_batch_graph g, void *stream);
int ctf_batch_graph_destroy(ctf_batch_graph g);

/* Time every warp tile (8x4, 4x8, 16x2) x items_per_fetch (1, 2, 4, 8) x
 * ctas_per_sm (2, 4) on these views, then solo_tiles (0, 4096, 16384,
 * 65536) at the best of those (best of 3 runs each, CUDA events on the
 * stream), and return the fastest in *best (budget, mask_dim and edge_remap
 * from *base, or the defaults).  Note that the warp tile changes which
 * warps succeed, hence the texel choices: every tile shape is a valid
 * filtering, and results are reproducible for a fixed shape. */
int ctf_batch_autotune(const ctf_view *views, int nviews, ctf_algorithm alg, uint64_t seed, const ctf_batch_opts *base,
                       ctf_batch_opts *best, double *best_ms, void *stream);

/* ctf_filter_host for callers that cannot let the library allocate device
 * memory.  The paper has no counterpart: this is a deployment variant.
 * ctf_filter_host stages the host arrays in device buffers that the library
 * allocates (and re-allocates for larger views) with cudaMalloc; a renderer
 * or plug-in whose video memory is reserved up front by its own allocator,
 * or a frame loop that cannot afford the device-wide synchronisation that
 * cudaMalloc and cudaFree may cause, cannot allow that.  This call keeps all
 * of its scratch (staging of uv, jac, coverage, image and counts, plus the
 * stats counters) in one fixed __device__ array of CTF_NOALLOC_SCRATCH_BYTES
 * that exists on every GPU that loads the library until the process exits,
 * and it never calls cudaMalloc, cudaFree or any other allocating routine.
 * Same arguments and results as ctf_filter_host, with these limits:
 *  - the view must fit: 256 bytes plus, each rounded up to 256 bytes,
 *    8 + 16 + 16 + 1 + 1 bytes per pixel (about 798,000 pixels; 1024x768
 *    fits); larger views return CTF_ERR_ARG and queue nothing;
 *  - all calls on a device share the array and it keeps the last call's
 *    contents (the stats counters are cleared at the start of each call);
 *    calls whose GPU work overlaps (other streams, other threads) race on
 *    it, so serialise them;
 *  - the first call on a device looks up the device addresses of the array
 *    and of the library's error word (a static __device__ int, which the
 *    learned-decode kernels use to report a wait that gave up) and caches
 *    them; make that first call before any stream capture. */
#define CTF_NOALLOC_SCRATCH_BYTES (32u << 20)
int ctf_filter_host_noalloc(ctf_texture tex, const float *uv_host, const float *jac_host,
                            const uint8_t *coverage_host, int width, int height, int view_id, ctf_algorithm alg,
                            uint64_t seed, const ctf_filter_opts *opts, float *out_rgba_host,
                            uint8_t *out_evals_host, ctf_stats *stats, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CTF_H */
