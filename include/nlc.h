/*
 * nlc.h -- C ABI of the GB300 (sm_103a) parallel local-autoregressive image
 * compressor ("Parallel Neural Local Lossless Compression", Zhang, Townsend,
 * Kang, Barber).
 *
 * Model (Section 2.1, Eq. 3): pixel (i, j) of a coding unit depends only on
 * rows i-h..i-1, columns j-h..j+h and on row i, columns j-h..j-1 (zero
 * outside the unit).  The local PixelCNN is a masked first layer over that
 * context (3 -> C channels), n_res residual blocks of two 1x1 layers with ELU,
 * and a 1x1 head to a K-component discretized logistic mixture with
 * channel-coupled RGB means.  Stream coder: 32-bit rANS (ANS, Section 2),
 * one stream per unit row.  Decoding follows Algorithm 1 (Section 3): at step
 * t every pixel with j = t - (h+1) i is decoded in one batch, so an H x W
 * unit takes W + (H-1)(h+1) steps instead of H W; independent P x P patches
 * of an image are decoded concurrently.
 *
 * Conventions for every entry point:
 *   - Pointers named d_* are device pointers on the current CUDA device;
 *     h_* are host pointers.  The caller owns every buffer it passes; the
 *     library owns only the context and a device workspace that it grows on
 *     demand (so the first call with a larger batch allocates).
 *   - Images are uint8 H x W x 3 (RGB), C-contiguous, row stride 3 W bytes.
 *     Kernels read image buffers (the inputs of the compress calls and of
 *     nlc_forward, and the outputs of the decode calls, whose decoded pixels
 *     are the context of later ones) in naturally aligned 4-byte words: the
 *     up to 3 bytes before an image's first byte and after its last byte
 *     that share such a word with it are read and their values ignored.
 *     Such a word never crosses a page, so any buffer of cudaMalloc or of
 *     a caching allocator qualifies.
 *     Container buffers (d_out of the compress calls, d_in of
 *     nlc_decompress) must be 16-byte aligned (NLC_ERR_ARG otherwise).
 *   - Calls taking a `stream` are asynchronous on that stream (NULL = the
 *     legacy default stream).  Argument errors are detected synchronously and
 *     returned.  Errors found on the device (corrupt stream, weight mismatch,
 *     capacity overflow, a bounded wait that timed out) are recorded in the
 *     context's device status word and returned by nlc_sync_status().
 *   - Calls on one context must not overlap on different streams: they share
 *     the context's workspace.
 *   - Every function returns an nlc_status; nlc_last_error() describes the
 *     last failure of the calling thread.
 */
#ifndef NLC_H
#define NLC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NLC_ABI_VERSION 1

typedef struct nlc_ctx nlc_ctx;
typedef struct CUstream_st* nlc_stream;

typedef enum {
  NLC_OK = 0,
  NLC_ERR_ARG = 1,         /* invalid argument (synchronous)                 */
  NLC_ERR_CAPACITY = 2,    /* output buffer too small                        */
  NLC_ERR_CORRUPT = 3,     /* malformed container or rANS stream            */
  NLC_ERR_WEIGHTS = 4,     /* container made with other weights / precision */
  NLC_ERR_CUDA = 5,        /* a CUDA call failed                             */
  NLC_ERR_TIMEOUT = 6,     /* a bounded device wait gave up                  */
  NLC_ERR_UNSUPPORTED = 7  /* configuration outside the compiled limits     */
} nlc_status;

/* Network arithmetic.  NLC_BF16_SHEARED is the BF16 network with its first
 * layer evaluated as Section 3.1's sheared kernels (Fig. 5) over the h+1 rows
 * of the h(h+2) sheared columns before the pixel (ShearLoC): the same model
 * function, rounded differently, so its containers are its own; its
 * wavefront decoder keeps the decoded pixels in a sheared layout and reads
 * each front's context as one rectangular window. */
typedef enum { NLC_FP32 = 0, NLC_BF16 = 1, NLC_BF16_SHEARED = 2 } nlc_precision;

/* Decode schedules.  All three decode the same container to the same pixels
 * (Section 4: every schedule has the same compression rate). */
typedef enum {
  NLC_SCHED_RASTER = 0,      /* one pixel per unit per step, raster order      */
  NLC_SCHED_WAVEFRONT = 1,   /* Algorithm 1: the whole front j = t-(h+1)i     */
  NLC_SCHED_SEQUENTIAL = 2   /* one pixel per image per step: the units of an
                                image one after another, raster inside each
                                (the paper's sequential decoder)             */
} nlc_schedule;

/* Stream layouts. */
typedef enum {
  NLC_LAYOUT_UNIT = 0,  /* one stream per unit, raster order (sequential only) */
  NLC_LAYOUT_ROW = 1    /* one stream per unit row: decodable by every schedule */
} nlc_layout;

/* Model configuration: horizon h (1..3), channels C (16, 32, 48 or 64),
 * residual blocks n_res (0..4), mixture components K (1..16), network
 * precision (FP32 SIMT, or BF16 on tcgen05 tensor cores with FP32
 * accumulation).  The mixture, CDF and coder are FP32/integer in both. */
typedef struct {
  int32_t h, C, n_res, K, precision;
} nlc_model_cfg;

typedef struct {
  const uint8_t* data; /* device pointer, H x W x 3 */
  int32_t H, W;
} nlc_image_in;

typedef struct {
  uint8_t* data; /* device pointer, H x W x 3, written by the decoder */
  int32_t H, W;
} nlc_image_out;

/* Thread-local description of the last error (never NULL). */
const char* nlc_last_error(void);
int nlc_abi_version(void);

/* Number of FP32 weights of cfg; the flat layout is
 *   W0[C][F] b0[C] { W1[C][C] b1[C] W2[C][C] b2[C] } x n_res WH[10K][C] bH[10K]
 * with F = 6h(h+1): feature 3p + c of W0 is channel c of context tap p, the
 * taps enumerating rows -h..-1 (columns -h..h) then row 0 (columns -h..-1),
 * i.e. the unmasked taps of a (2h+1)^2 type-A masked kernel in raster order.
 * Head outputs: [0,K) mixture logits, [K,4K) means, [4K,7K) log-scales
 * (clamped at -7), [7K,10K) raw coupling coefficients (tanh).  Returns 0 for
 * an invalid cfg. */
size_t nlc_num_weights(const nlc_model_cfg* cfg);

/* Creates a context on the current device with the given host weights
 * (n_weights must equal nlc_num_weights(cfg)).  Synchronous.  The first call
 * on a device also checks, over every pair of adjacent floats (all floats for
 * ex2.approx, [1, +inf] for rcp.approx), that the device's ex2.approx and
 * rcp.approx are monotone (a few milliseconds); the frequency tables are
 * computed one boundary at a time and rely on it.  If the check fails:
 * NLC_ERR_UNSUPPORTED. */
int nlc_create(const nlc_model_cfg* cfg, const float* h_weights, size_t n_weights, nlc_ctx** out);
int nlc_destroy(nlc_ctx* ctx);

/* Copies the current FP32 weights to / from the host (synchronous).  Setting
 * weights also resets the optimizer state. */
int nlc_get_weights(nlc_ctx* ctx, float* h_weights, size_t n_weights);
int nlc_set_weights(nlc_ctx* ctx, const float* h_weights, size_t n_weights);

/* 64-bit content hash of (cfg, weights), stored in every container. */
int nlc_weight_hash(nlc_ctx* ctx, uint64_t* h_hash);

/* Waits for `stream`, returns the device status recorded since the last call
 * (NLC_OK if none) and clears it. */
int nlc_sync_status(nlc_ctx* ctx, nlc_stream stream);

/* Decoder tuning: the decoder assigns about px_per_cta pixels of every step
 * to each CTA (default 8) and uses at most max_ctas CTAs (0 = as many as can
 * be co-resident). */
int nlc_set_tuning(nlc_ctx* ctx, int px_per_cta, int max_ctas);

/* Limits of the decoder's bounded waits (also the sampler's): polls of the
 * grid barrier between wavefront steps and of an MMA's completion before the
 * wait gives up (0 = the defaults, 2^25 and 2^22 polls, far beyond any
 * normal wait).  A wait that gives up records NLC_ERR_TIMEOUT in the
 * context's status and releases every CTA of the launch, which leaves the
 * decode loop (an MMA wait first waits, bounded, for the MMAs it issued);
 * the context stays usable.  Small limits exist to exercise that path: a
 * reduced MMA limit counts non-blocking tests of the completion. */
int nlc_set_wait_limits(nlc_ctx* ctx, uint32_t grid_polls, uint32_t mma_polls);

/* Decoder phase profile (per-step latency against the dependency-bound step
 * count of Section 3).  enable != 0 makes the following nlc_decompress calls
 * and nlc_plan_run calls (a captured graph keeps the setting of its capture)
 * run an instrumented build of the decoder (same results, slower: its
 * counters' state costs registers) that records, in thread 0 of every CTA,
 * clock64 cycles spent per phase; a
 * non-NULL h_counters (16 uint64) receives the totals accumulated since the
 * last read, summed over CTAs, and clears them:
 *   [0] front bookkeeping, [1] tile slot assignment, [2] context gather and
 *   local network, [3] per-pixel CDF + rANS coding, [4] grid barrier,
 *   [5] tiles processed, [6] CTAs, [7] decode steps (of CTA 0);
 *   within [3], for the pixels coded by warp 0: [8] mixture and channel
 *   set-up, [9] CDF symbol search, [10] rANS state update, [11] posterior
 *   update, [12] pixels; within [2], for thread 0 (BF16 network): [13]
 *   context gather, [14] tensor-core MMA issue to completion, [15] epilogues
 *   (TMEM loads, bias/ELU, operand stores, CTA barriers).
 * Synchronises the device when reading or changing the mode. */
int nlc_decode_profile(nlc_ctx* ctx, int enable, uint64_t* h_counters);

/* Step end times of the following nlc_decompress and nlc_plan_run calls (a
 * captured graph keeps the buffer of its capture): the decoder zeroes
 * d_times[0 .. n) and writes, in %globaltimer nanoseconds, d_times[0] = its
 * start and d_times[t + 1] = the time at which every CTA has finished
 * wavefront step t (the release of the grid barrier after it; the last step:
 * the latest CTA end), for the entries below n.  With the unit partition and
 * Algorithm 1's step count W_u + (H_u - 1)(h + 1) of each unit (all units
 * start at step 0 under the wavefront schedule), an image's decode latency
 * in a batch is d_times[T_i] - d_times[0], T_i its units' largest step
 * count.  d_times = NULL (n = 0) stops the stamping; the caller owns the
 * buffer, which must outlive the calls that use it. */
int nlc_decode_step_times(nlc_ctx* ctx, uint64_t* d_times, int64_t n);

/* Upper bound of the compressed size of n images with the given sizes, unit
 * partition and layout: per image 32 + 4 n_streams + 6 H W + 4 n_streams
 * bytes, rounded up to 16.  `patch` = side of the square coding units (0 =
 * the whole image is one unit). */
int nlc_compress_bound(const int32_t* h_H, const int32_t* h_W, int n, int patch, int layout,
                       size_t* h_bytes);

/* Compresses n images.  Container i is written to d_out + d_offsets[i] and
 * ends at d_offsets[i+1]; d_offsets (n+1 uint64, device) is written by the
 * library.  Container: 32-byte header ("NLC1", version 2, h, layout,
 * precision, H, W, patch, n_streams, weight hash), n_streams stream lengths
 * (uint16 when 6 x the pixels of the image's largest stream + 4 < 2^16 --
 * a row of at most 10,921 pixels with one stream per row -- else uint32),
 * the streams (rANS, 4-byte big-endian final state then bytes), zero padding
 * to 16 bytes.  If the total exceeds `cap` nothing is written
 * and the device status becomes NLC_ERR_CAPACITY (d_offsets still holds the
 * sizes).  The encoder computes every pixel's frequency tables in parallel
 * with the decoder's own device code (the paper's encoder reruns the
 * decoder's procedure for the same reason, Section 4). */
int nlc_compress(nlc_ctx* ctx, const nlc_image_in* h_imgs, int n, int patch, int layout,
                 uint8_t* d_out, size_t cap, uint64_t* d_offsets, nlc_stream stream);

/* Scratch capacity of nlc_compress_noalloc, in bytes.  A batch needs about
 * 18 bytes per pixel, 16 per rANS stream and 100 per coding unit and image
 * (32 MiB holds e.g. one 1024 x 1024 image or forty 256 x 256 images). */
#define NLC_NOALLOC_SCRATCH_BYTES (32u << 20)

/* nlc_compress without any device allocation.  The paper has no counterpart:
 * this serves callers that cannot call cudaMalloc at the time they compress,
 * e.g. a process whose framework allocator has reserved all device memory,
 * a real-time thread that cannot absorb cudaMalloc's implicit device
 * synchronisation and unbounded latency, or a deployment whose device memory
 * budget is fixed when the library is loaded.  Same arguments, output and
 * asynchrony as nlc_compress (byte-identical containers), but the call's
 * scratch (batch plan, per-symbol tables, per-stream bytes) is a file-scope
 * device array of NLC_NOALLOC_SCRATCH_BYTES that every GPU loading the
 * library holds until exit; the caller still owns the images, d_out and
 * d_offsets.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress, with the device current); make that first
 * call before any stream capture.  Like nlc_compress, every call copies the
 * batch's unit table to the device (cudaMemcpyAsync on `stream`) from host
 * memory that the call owns and releases before it returns.  Batches needing more scratch are rejected
 * with NLC_ERR_CAPACITY before anything is launched.  All calls share the one
 * array, which keeps the last call's contents (nothing in it needs to start
 * at zero): calls that overlap on the GPU, from any context or stream, race,
 * so serialise them.  The context must already exist (nlc_create allocates);
 * this call itself allocates nothing. */
int nlc_compress_noalloc(nlc_ctx* ctx, const nlc_image_in* h_imgs, int n, int patch, int layout,
                         uint8_t* d_out, size_t cap, uint64_t* d_offsets, nlc_stream stream);

/* Decompresses n containers (d_in + d_offsets[i] .. d_offsets[i+1]) into
 * caller-allocated images whose H, W must match the containers.  `patch`
 * and `layout` must be those used to compress; `schedule` is an
 * nlc_schedule (NLC_LAYOUT_UNIT needs RASTER or SEQUENTIAL).  The wavefront
 * decode is one persistent cooperative kernel: the pixels of every step are
 * split across all CTAs, which meet at a bounded grid barrier between steps. */
int nlc_decompress(nlc_ctx* ctx, const uint8_t* d_in, const uint64_t* d_offsets,
                   const nlc_image_out* h_outs, int n, int patch, int layout, int schedule,
                   nlc_stream stream);

/* Decode plan: the host side of nlc_decompress for a fixed batch of output
 * images (unit partition, wavefront schedule of Algorithm 1, device unit
 * tables, grid size), done once.  nlc_plan_decode allocates the plan's
 * device buffers and copies its unit tables synchronously; the plan keeps
 * the output pointers of h_outs (they must stay valid) and uses the
 * context's weights at run time.  Arguments and errors as nlc_decompress. */
typedef struct nlc_plan nlc_plan;
int nlc_plan_decode(nlc_ctx* ctx, const nlc_image_out* h_outs, int n, int patch, int layout,
                    int schedule, nlc_plan** out);

/* Decodes containers laid out as the plan's images (d_in 16-byte aligned,
 * d_offsets n+1 device uint64) into the plan's outputs.  Issues device work
 * only (no allocation, no host copy, no synchronisation), so it may be
 * captured in a CUDA graph; a graph replay decodes whatever containers are
 * at d_in then.  Device-side errors go to the context's status word.  Runs
 * of one plan, and of plans sharing a context, must not overlap. */
int nlc_plan_run(nlc_plan* plan, const uint8_t* d_in, const uint64_t* d_offsets,
                 nlc_stream stream);

/* Autotuner of the decoder's front packing: for px_per_cta in 1, 2, 4, ...,
 * 128 (pixels of each step per CTA, which sets the grid), runs the plan once
 * to warm up and `reps` times timed with CUDA events, and keeps the fastest
 * setting in the plan.  Synchronous; decodes (reps + 1) x candidates times.
 * h_px_per_cta / h_ms (either may be NULL) receive the choice and its time
 * per decode. */
int nlc_plan_tune(nlc_plan* plan, const uint8_t* d_in, const uint64_t* d_offsets, int reps,
                  nlc_stream stream, int* h_px_per_cta, float* h_ms);

/* Frees the plan (synchronises the device). */
int nlc_plan_destroy(nlc_plan* plan);

/* Draws n images from the model (Section 5: the parallel schedules serve
 * sampling from a local autoregressive model as they serve decoding): the
 * decoder's schedule, network and quantised tables, with each symbol taken
 * by inverse-CDF sampling of its channel's table, v such that cum_v <= u <
 * cum_{v+1}, where u is the top 16 bits of output k of SplitMix64 (Steele,
 * Lea, Flood 2014) seeded with `seed`, k = ((i 2^21 + y) 2^21 + x) 3 + c for
 * channel c of pixel (y, x) of image i of the batch.  Every schedule gives
 * the same images.  h_outs as nlc_decompress (caller-allocated, sides and n
 * below 2^21); `patch` partitions them into independent units as in the
 * codec (0 = whole images). */
int nlc_sample(nlc_ctx* ctx, const nlc_image_out* h_outs, int n, int patch, uint64_t seed,
               int schedule, nlc_stream stream);

/* Network outputs (d_params: sum H W x 10K floats, images in order, pixels
 * in raster order) and/or the model code length -log2 p(x_ij) of every pixel
 * (d_bits: sum H W floats); either may be NULL.  Context zero outside the
 * units of the given patch partition. */
int nlc_forward(nlc_ctx* ctx, const nlc_image_in* h_imgs, int n, int patch, float* d_params,
                float* d_bits, nlc_stream stream);

/* Frequency tables of n pixels from given network outputs (d_params: n x 10K)
 * and pixel values (d_pixels: n x 3): d_cum (n x 3 x 257 uint32) receives
 * cum_0..cum_256 of the R, G|r and B|r,g coding distributions. */
int nlc_tables(nlc_ctx* ctx, const float* d_params, const uint8_t* d_pixels, int64_t n,
               uint32_t* d_cum, nlc_stream stream);

/* rANS stage alone.  Stream s codes symbols [d_sym_off[s], d_sym_off[s+1])
 * given as (start, freq) with 16-bit probability scale; it is written to the
 * LAST d_len[s] bytes of the slot d_bytes + s * stride (stride >= 2 nsym + 4). */
int nlc_rans_encode(const uint32_t* d_start, const uint32_t* d_freq, const int64_t* d_sym_off,
                    int n_streams, uint8_t* d_bytes, int64_t stride, int32_t* d_len,
                    nlc_stream stream);

/* Decodes the streams laid out as nlc_rans_encode writes them, with one
 * cumulative table (257 uint32) per symbol.  A stream that does not end in
 * the initial state with every byte consumed sets NLC_ERR_CORRUPT in the
 * context's status (ctx may not be NULL). */
int nlc_rans_decode(nlc_ctx* ctx, const uint8_t* d_bytes, int64_t stride, const int32_t* d_len,
                    const uint32_t* d_cum, const int64_t* d_sym_off, int n_streams,
                    int32_t* d_sym, nlc_stream stream);

/* Maximum-likelihood training (Eq. 2).  One Adam step (beta 0.9/0.999,
 * eps 1e-8) on the mean code length in bits per dimension of N H x W images
 * (d_batch, each image one unit); h_loss (may be NULL) receives the loss
 * before the step, which makes the call synchronous. */
int nlc_train_step(nlc_ctx* ctx, const uint8_t* d_batch, int N, int H, int W, float lr,
                   float* h_loss, nlc_stream stream);

/* Loss (bits per dimension, d_loss: 1 float) and its gradient with respect
 * to the FP32 weights (d_grad: nlc_num_weights floats) -- the adjoint of the
 * network and of the mixture likelihood (Eq. 2).  A BF16 context computes
 * the forward and the adjoint on the tensor cores (tcgen05, BF16 operands,
 * FP32 accumulation; the mixture likelihood and its gradient in FP32) when
 * its tiles fit in one CTA's shared memory (every h and K with C <= 64 and
 * n_res <= 3, and C <= 48 with n_res = 4); FP32 contexts use the FP32 SIMT
 * adjoint, which holds models up to n_res = 2 at C = 64 (larger ones:
 * NLC_ERR_UNSUPPORTED).  Deterministic: the same inputs give the same bits. */
int nlc_loss_grad(nlc_ctx* ctx, const uint8_t* d_batch, int N, int H, int W, float* d_loss,
                  float* d_grad, nlc_stream stream);

/* Adjoint of the local network alone (Section 2.1): given the gradient
 * d_dparams (N H W x 10K floats, the layout of nlc_forward's outputs for the
 * N images of d_batch, each one unit) of some scalar with respect to the
 * network outputs, writes its gradient with respect to the FP32 weights to
 * d_dweights (nlc_num_weights floats).  Same arithmetic and path choice as
 * nlc_loss_grad (the BF16 path rounds d_dparams to BF16). */
int nlc_backward(nlc_ctx* ctx, const uint8_t* d_batch, int N, int H, int W, const float* d_dparams,
                 float* d_dweights, nlc_stream stream);

/* Replaces the weights with n_weights FP32 values from device memory
 * (asynchronous on `stream`; the optimizer state is kept). */
int nlc_load_weights(nlc_ctx* ctx, const float* d_weights, size_t n_weights, nlc_stream stream);

/* Measurement utility (no counterpart in the paper): the device's rate of
 * the MUFU instruction pair of one logistic term of the symbol search,
 * rcp.approx(1 + ex2.approx(z)), in MUFU operations per second.  Runs
 * independent chains of the pair at full occupancy on every SM, `iters`
 * pairs per chain (about 2e4 gives ~20 ms on a GB300), timed with CUDA
 * events on `stream`; synchronous.  h_ms (may be NULL) receives the timed
 * kernel's duration.  This rate is the denominator of the decoder's MUFU
 * roofline. */
int nlc_measure_mufu(int iters, nlc_stream stream, double* h_ops_per_s, double* h_ms);

#ifdef __cplusplus
}
#endif

#endif /* NLC_H */
