/*
 * glassnet.h — C ABI of the GlassNet per-pixel forward pass on sm_103a.
 *
 * Method: Zhang & Simo-Serra, "Neural Scene Baking for Permutation Invariant
 * Transparency Rendering with Real-time Global Illumination" (arXiv
 * 2405.19056).  The network (Sec. 3.3-3.4, Fig. 2) in its per-pixel MLP form:
 *
 *   sigma = F(s)                          scene encoder, once per scene
 *   v_k   = h([b_k ; sigma])              shared per-layer network (Eq. 5)
 *   pool  = [max_k v_k ; mean_k v_k]      symmetric function over valid layers
 *   r     = rho(pool)   (r = 0 when a pixel has no valid layer)
 *   y     = B([g ; r ; sigma])            final blending network
 *   rgb   = sigmoid(R(y))                 rendering network
 *
 * Widths: hidden H, latent Z with (H, Z) = (64, 128) or (128, 256); scene
 * vector 32 floats; transparency layer 12 channels; opaque G-buffer 14
 * channels; 3 output channels.  Every linear layer is followed by ReLU except
 * the last one of R, which is followed by a sigmoid.
 *
 * Conventions for every entry point:
 *  - Return value: GN_OK or a negative gn_status.  Nothing is thrown across
 *    the ABI and nothing aborts.  glassnet_last_error() gives a message for the
 *    last failure on the calling thread.
 *  - Arguments are validated on the host before any launch; a call that
 *    returns an error has enqueued no work.
 *  - Buffers are owned by the caller; gn_model and gn_latent objects are owned
 *    by the library and released with the matching free function.
 *  - Device work is asynchronous on the given stream (0 = legacy default
 *    stream).  Conditions only the device can see (a layer count above K, an
 *    exact-sum overflow, a device-side wait that timed out) set sticky bits in
 *    the model's error word; glassnet_check() synchronises the stream and
 *    returns them as GN_EINVAL, GN_ERANGE or GN_ETIMEOUT.
 *  - Image buffers are structure-of-arrays, row-major pixels p = y*w + x:
 *      gbuf        float [14][h][w]      opaque G-buffer (device)
 *      tbuf        float [K][12][h][w]   transparency layers (device);
 *                  slots k >= layer_count[p] are never read into the result
 *                  and may hold any bits, including NaN
 *      layer_count uint8 [h][w]          valid layers per pixel, 0..K (device)
 *      out         float [3][h][w]       RGB in (0, 1) (device)
 *    All pointers must be 4-byte aligned (uint8 counts: any alignment).
 */
#ifndef GLASSNET_H_
#define GLASSNET_H_

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gn_status {
  GN_OK = 0,
  GN_EINVAL = -1,       /* bad argument, or a layer count above K seen on device */
  GN_ENOMEM = -2,       /* device or host allocation failed */
  GN_ECUDA = -3,        /* a CUDA runtime call failed */
  GN_EFORMAT = -4,      /* weight blob: bad magic, version, sizes or checksum */
  GN_ETIMEOUT = -5,     /* a device-side wait exceeded its time limit */
  GN_EUNSUPPORTED = -6, /* widths or precision the library does not provide */
  GN_ERANGE = -7,       /* exact set-sum left its fixed-point range (see below) */
  GN_ESATURATED = -8    /* FP8: an input beyond its calibrated range was clamped */
} gn_status;

typedef enum gn_precision {
  GN_FP32_PLAIN = 0, /* unfused concat form, one kernel per layer, FP32 CUDA cores */
  GN_BF16_FUSED = 1, /* one fused tcgen05 kernel, BF16 operands, FP32 accumulate */
  GN_FP8_FUSED = 2   /* fused kernel with E4M3 operands and FP32 scales */
} gn_precision;

/* Symmetric function of Eq. 5 that pools a pixel's per-layer phi outputs.
 * GN_POOL_MAX_MEAN: pool = [max ; mean] over the valid layers, then
 *   r = ReLU(W_rho pool + b_rho) (r = 0 without layers) enters B.
 * GN_POOL_SUM: the paper's own form, tau = sum of the phi outputs (the zero
 *   vector without layers) enters B directly; rho is not used. */
typedef enum gn_pooling {
  GN_POOL_MAX_MEAN = 0,
  GN_POOL_SUM = 1
} gn_pooling;

typedef struct gn_model gn_model;   /* device weights of one network */
typedef struct gn_latent gn_latent; /* one encoded scene: sigma and folded biases */

/* ------------------------------------------------------------------------
 * Weight blob.  A 48-byte header followed by float32 tensors, each W as
 * [out][in] row-major (y = W x + b) followed by its b [out], in the order
 * F1, F2, phi1, phi2, rho, B1, B2, R1, R2 with shapes (concat form):
 *   F1 [Z][32]   F2 [Z][Z]   phi1 [H][12+Z]   phi2 [H][H]   rho [H][2H]
 *   B1 [H][14+H+Z]   B2 [H][H]   R1 [H][H]   R2 [3][H]
 * phi1's input is [layer ; sigma]; B1's input is [gbuf ; r ; sigma]; rho's
 * input is [max ; mean].  checksum = FNV-1a 64 over the payload bytes.
 * ---------------------------------------------------------------------- */
#define GN_BLOB_MAGIC 0x544E4C47u /* bytes "GLNT" */
#define GN_BLOB_VERSION 1u

typedef struct gn_blob_header {
  uint32_t magic;
  uint32_t version;
  uint32_t hidden;        /* H */
  uint32_t latent;        /* Z */
  uint32_t scene_dim;     /* 32 */
  uint32_t tbuf_channels; /* 12 */
  uint32_t gbuf_channels; /* 14 */
  uint32_t out_channels;  /* 3 */
  uint64_t payload_floats;
  uint64_t checksum;
} gn_blob_header;

/*
 * Validates a weight blob (host memory) and uploads it for one precision.
 * The network's weights are trained jointly (Sec. 3.4); the blob is the
 * trained (or synthetic) parameter set.  For GN_BF16_FUSED the weights are
 * rounded to BF16 (round to nearest even) and packed into the tensor-core
 * operand layout; GN_FP32_PLAIN keeps them as given.
 * Errors: GN_EINVAL (null pointers, unknown precision), GN_EFORMAT (size,
 * magic, version, channel counts or checksum), GN_EUNSUPPORTED ((H, Z) not
 * (64, 128) or (128, 256)), GN_ENOMEM, GN_ECUDA.  Synchronous.
 */
int glassnet_load_weights(const void* blob, size_t nbytes, int precision, gn_model** out);

/* Form of the network a blob is loaded as. */
typedef struct gn_model_config {
  int precision; /* gn_precision */
  int pooling;   /* gn_pooling */
  /* Positional encoding of the inputs (Sec. 3.4, after Mildenhall et al.):
   * L = pe_freqs frequency bands, 0 = inputs as given.  Every input of n
   * channels -- the scene vector, each transparency layer and the G-buffer --
   * enters its first linear layer as the n (1 + 2L) values
   *   [x ; sin(2^0 pi x) ; cos(2^0 pi x) ; ... ; sin(2^(L-1) pi x) ; cos(2^(L-1) pi x)]
   * (blocks of n, in that order), so F1, phi1 and B1 are wider:
   *   F1 [Z][32 e]   phi1 [H][12 e + Z]   B1 [H][14 e + H + Z],  e = 1 + 2L. */
  int pe_freqs;
  /* Kernel size of R's first layer (Sec. 3.4: larger kernels ahead of the
   * 1x1 end of R): 1 (or 0) = per pixel; 3 = a 3x3 kernel over the frame's
   * neural buffer y (B's output), q(p) = ReLU(b + sum over (dy, dx) in
   * {-1,0,1}^2 of W[:, :, dy+1, dx+1] y(p + (dy, dx))), y = 0 outside the
   * frame.  R1 is then stored as [H][9 H], the [out][in][3][3] kernel
   * flattened (column k 9 + (dy+1) 3 + dx+1).  R2 stays 1x1. */
  int r_kernel;
} gn_model_config;

/*
 * As glassnet_load_weights, for the form in `config`;
 * glassnet_load_weights is this call with {precision, GN_POOL_MAX_MEAN, 0, 1}.
 * The blob's payload must hold the widths of that form (the header's H and Z
 * with pe_freqs), else GN_EFORMAT.
 * Pooling: a GN_POOL_SUM network has no rho; its blob keeps the rho tensor
 *   and bias slots (any values; zeros for a network trained in that form),
 *   which are never read.  The sum uses the same exact fixed-point
 *   accumulator as the mean (range [0, 2^11) per pixel-channel, GN_ERANGE
 *   beyond it), so the BF16 result is bit-identical under any order of a
 *   pixel's layers.
 * Positional encoding: pe_freqs 0..10 for GN_FP32_PLAIN; 0..4 at H = 64 and
 *   H = 128 for GN_BF16_FUSED (the encoded operands are sized for 4; at
 *   H = 128 they and the resident weights fill the shared memory, so the
 *   per-pixel weights stream from device memory through a two-stage ring
 *   in each CTA, with the same arithmetic); 0..4 at H = 64 and H = 128 for
 *   GN_FP8_FUSED with the 1x1 R (E4M3 operands take half the bytes).
 *   The fused kernels compute sin(pi x) and cos(pi x) of each input
 *   channel with exact argument reduction and the higher bands by the
 *   double-angle identities in FP32, then round every band to BF16, or to
 *   E4M3: band 0 as codes of its channel's calibrated scale, the sine and
 *   cosine bands as codes of 256 v (|v| <= 1).
 * GN_POOL_SUM serves every precision (for GN_FP8_FUSED the sum enters B1 as
 * codes of B1's input scale, calibrated on the FP32 path's sum form).
 * pe_freqs > 0 serves every render, batch, graph, server and streaming call
 * of GN_FP32_PLAIN / GN_BF16_FUSED models and every render, batch, graph and
 * server call of GN_FP8_FUSED models (pe_freqs above 4, or with r_kernel = 3,
 * returns GN_EUNSUPPORTED there).
 * r_kernel = 3 serves every render, batch, graph and server call of every
 *   precision (streaming: GN_BF16_FUSED) (any pooling; with pe_freqs as
 *   above): the fused kernel writes each frame's neural buffer (BF16, H 2
 *   bytes per pixel, in the launch's workspace, so glassnet_workspace_bytes
 *   grows by about h w H 2 bytes), then a tcgen05 kernel per frame runs the
 *   3x3 layer, R2 and the sigmoid (streaming: the resolve writes the neural
 *   buffer into the pool's own, then the 3x3 kernel runs).  GN_FP8_FUSED
 *   models write B2's output in real units as BF16 and share the BF16 3x3
 *   kernel.
 * Errors: those of glassnet_load_weights, GN_EINVAL (NULL config, unknown
 * pooling, pe_freqs outside 0..10, r_kernel not 0, 1 or 3), GN_EUNSUPPORTED.
 */
int glassnet_load_weights_ex(const void* blob, size_t nbytes, const gn_model_config* config,
                             gn_model** out);
/* The form a model was loaded as.  Errors: GN_EINVAL (NULL argument). */
int glassnet_model_config(const gn_model* model, gn_model_config* config);

/* Widths and precision of a loaded model (any pointer may be NULL). */
int glassnet_model_info(const gn_model* model, int* hidden, int* latent, int* precision);

/*
 * Scene encoder F (Sec. 3.4) on one scene vector, and the per-scene folded
 * biases c_phi = W_phi1[:, 12:] sigma + b_phi1 and c_B = W_B1[:, 14+H:] sigma
 * + b_B1 (exact algebra of the concat form).  `scene` is 32 floats in host
 * memory, copied before the call returns.  Allocates the latent (device
 * memory) and enqueues the encoder on `stream`.
 * Errors: GN_EINVAL, GN_ENOMEM, GN_ECUDA.
 */
int glassnet_encode_scene(gn_model* model, const float* scene, gn_latent** out,
                          cudaStream_t stream);

/* Re-encodes into an existing latent from a device scene vector (32 floats);
 * allocates nothing. */
int glassnet_encode_scene_device(gn_model* model, const float* scene_dev, gn_latent* latent,
                                 cudaStream_t stream);

/* Copies sigma (Z floats) or the folded biases (H floats each) of a latent
 * to device buffers, enqueued on `stream`.  Any destination may be NULL. */
int glassnet_latent_read(const gn_latent* latent, float* sigma_dev, float* c_phi_dev,
                         float* c_b_dev, cudaStream_t stream);

/*
 * Renders one frame: the per-pixel network over every pixel (Sec. 3.2-3.4).
 * K is the number of layer slots in tbuf (0..8); K = 0 renders the
 * opaque-only path (r = 0) and tbuf may be NULL.  h, w >= 1, 12*max(K,1)*h*w < 2^31.
 * Precision is the model's.  GN_BF16_FUSED / GN_FP8_FUSED: the tile-plan
 * kernel and one fused kernel (and the 3x3 R kernel for r_kernel = 3),
 * output bit-identical under any permutation of each pixel's valid layers.
 * GN_FP32_PLAIN: one kernel per layer.  The workspace (FP32 intermediates,
 * or the fused tile plan with its tile counter and, for r_kernel = 3, the
 * neural buffer) is owned by the model and grows on demand (a growing call
 * synchronises the device), so renders of one model must be ordered on one
 * stream; concurrent renders of one model on different streams must use
 * glassnet_render_ws with separate workspaces.
 * Errors: GN_EINVAL (bad sizes, NULL pointers, misalignment, latent of another
 * width), GN_ENOMEM, GN_ECUDA.
 */
int glassnet_render(const gn_model* model, const gn_latent* latent, const float* gbuf,
                    const float* tbuf, const uint8_t* layer_count, int K, int h, int w, float* out,
                    cudaStream_t stream);

/* Workspace bytes glassnet_render_ws needs for this model and frame size
 * (0 for the fused precisions). */
int glassnet_workspace_bytes(const gn_model* model, int K, int h, int w, size_t* bytes);

/* glassnet_render with a caller-owned device workspace of at least
 * glassnet_workspace_bytes() bytes (256-byte aligned). */
int glassnet_render_ws(const gn_model* model, const gn_latent* latent, const float* gbuf,
                       const float* tbuf, const uint8_t* layer_count, int K, int h, int w,
                       float* out, void* workspace, size_t workspace_bytes, cudaStream_t stream);

/*
 * End-to-end render from HOST buffers (same layouts as glassnet_render):
 * copies gbuf, the K slots of tbuf and the counts to device staging owned by
 * the model, renders, copies RGB back to `out_host` and synchronises
 * `stream`.  Host buffers should be page-locked for full copy bandwidth.
 * Staging grows on demand.  Not safe to call concurrently on one model.
 */
int glassnet_render_host(gn_model* model, const gn_latent* latent, const float* gbuf_host,
                         const float* tbuf_host, const uint8_t* count_host, int K, int h, int w,
                         float* out_host, cudaStream_t stream);

/*
 * Streaming (incremental) rendering: the pooled set representation of Eq. 5
 * built one transparency layer at a time (the paper's memory argument, Sec. 5
 * and Fig. 9: the cost of a frame grows with the number of objects, the
 * memory held need not).  A pool holds, per pixel, the running max and the
 * exact fixed-point sum of phi over the layers accumulated so far and their
 * number; the pooling is exact and order-independent, so accumulating a
 * frame's layers in any order and resolving gives the same bits as
 * glassnet_render of that frame (tested).
 *
 * Pool state: (H/2 + H) * 4 + 1 bytes per pixel in device memory (769 B at
 * H = 128), plus a tile plan; owned by the pool object.
 *
 * glassnet_pool_create: a pool for h x w frames of this model (precision
 *   GN_BF16_FUSED; GN_EUNSUPPORTED otherwise), empty (no layers).
 * glassnet_pool_reset: empties the pool (stream-ordered).
 * glassnet_accumulate_layer: phi of one transparency layer `layer` (device,
 *   [12][h][w] f32, the channel layout of a tbuf slot) pooled into the pixels
 *   it covers: `covered` (device, [h][w] u8, 0 or 1; NULL: every pixel).  At
 *   most 8 layers per pool (Eq. 5's exact sum is bounded for K <= 8): a ninth
 *   call returns GN_EINVAL.  Values other than 0 and 1 in `covered` set the
 *   count error (GN_EINVAL at the next glassnet_check).
 * glassnet_resolve: rho, B and R of the pooled state with the G-buffer `gbuf`
 *   (device, [14][h][w] f32) -> `out` (device, [3][h][w] f32); for a
 *   GN_POOL_SUM model the pooled sum enters B directly.  Pixels with no
 *   layer take the opaque-only path (r = 0), as in glassnet_render.
 * All three are asynchronous on `stream`; calls on one pool must be ordered
 * (one stream); different pools may run concurrently.  Alignment rules are
 * those of glassnet_render.
 */
typedef struct gn_pool gn_pool;
int glassnet_pool_create(const gn_model* model, int h, int w, gn_pool** out);
int glassnet_pool_reset(gn_pool* pool, cudaStream_t stream);
int glassnet_accumulate_layer(const gn_model* model, const gn_latent* latent, gn_pool* pool,
                              const float* layer, const uint8_t* covered, cudaStream_t stream);
int glassnet_resolve(const gn_model* model, const gn_latent* latent, const gn_pool* pool,
                     const float* gbuf, float* out, cudaStream_t stream);
void glassnet_pool_free(gn_pool* pool);

/* One frame of a batched launch. */
typedef struct gn_frame {
  const gn_latent* latent;
  const float* gbuf;
  const float* tbuf;
  const uint8_t* layer_count;
  int K, h, w;
  float* out;
} gn_frame;

/*
 * Renders n frames of mixed sizes, layer counts and scenes in one persistent
 * launch of the fused kernel (fused precisions only).  `frames` is host
 * memory; the descriptor table is copied into a model-owned device buffer,
 * so one model must not run two batches concurrently.  Each frame's output
 * equals glassnet_render of that frame alone, bit for bit.
 */
int glassnet_render_batch(const gn_model* model, const gn_frame* frames, int n,
                          cudaStream_t stream);

/*
 * FP8 variant.  A model loaded with GN_FP8_FUSED runs every layer's GEMM with
 * E4M3 operands and FP32 accumulation: weights are quantised per output
 * channel (scale = channel |max| / 448), the network's two input tensors
 * (transparency layers, G-buffer) per input channel and the hidden
 * activations per tensor, with static scales taken from one calibration
 * render.  An input channel's scale is folded into its weight column (the
 * weights quantised are W[n][c] s[c]), so it costs nothing at render time.
 * The per-scene folded biases stay exact (a BF16 hi/lo MMA), the set pooling
 * stays exact and order-independent (it runs on the dequantised phi output).
 * An input value beyond its channel's calibrated range is clamped to the
 * largest E4M3 code and reported (GN_ESATURATED at the next glassnet_check);
 * the frame is still rendered.  The paper fixes no precision for the
 * network; this is a deployment variant.
 *
 * glassnet_calibrate_fp8 renders the given frame with the FP32 plain path
 * (intermediates in the model's FP32 workspace, grown on demand), takes the
 * |max| of each layer input over it (each channel of t over the valid slots,
 * each channel of g; then U, pool, r, y, y2, q) and sets scale = 8 |max| / 448
 * for the input channels and 4 |max| / 448 for the others (headroom against
 * inputs beyond the calibration frame's range; 1 where the maximum is 0),
 * then packs the E4M3 image.  Synchronous.  Until it has run, rendering with
 * the model returns GN_EINVAL.  It may be called again to recalibrate (no
 * render may be in flight).  Errors: GN_EINVAL (not an FP8 model, bad frame),
 * GN_ENOMEM, GN_ECUDA.
 *
 * glassnet_fp8_scales copies the GN_FP8_SCALES = 32 scales (the real value of
 * a code x is x * scale) to host memory, in the order: the 12 channels of t,
 * the 14 channels of g, then U, pool, r, y, y2, q.
 */
#define GN_FP8_SCALES 32
int glassnet_calibrate_fp8(gn_model* model, const gn_latent* latent, const float* gbuf,
                           const float* tbuf, const uint8_t* layer_count, int K, int h, int w,
                           cudaStream_t stream);
int glassnet_fp8_scales(const gn_model* model, float* scales);

/*
 * CUDA graphs of batched launches.  A graph holds the launch sequence of
 * glassnet_render_batch (the tile-plan kernel and the fused kernel) for one
 * batch shape: the number of frames and each frame's h, w and K.  The paper
 * has no counterpart (its Sec. 5 times single frames); this is the serving
 * layer's way to replay a shape bucket without rebuilding its launches.
 *
 * glassnet_graph_create validates the batch as glassnet_render_batch does,
 * allocates the graph's own tile-plan workspace (device memory, so graphs of
 * one model may replay concurrently on different streams) and captures the
 * launches with the given buffers and latents.  Synchronous; call it outside
 * any stream capture.  Errors: those of glassnet_render_batch, GN_ENOMEM,
 * GN_ECUDA.
 *
 * glassnet_graph_launch replays the graph on `stream`: same buffers, same
 * latents (whose contents may have changed), fresh contents read at replay.
 * Each replay's output equals glassnet_render_batch of the same frames, bit
 * for bit.  Replays of one graph must not overlap on the GPU (they share the
 * graph's workspace).
 *
 * glassnet_graph_update rebinds the graph to other buffers and latents of
 * the same shapes (n, and per frame h, w, K; GN_EINVAL otherwise).  Call it
 * when no replay of the graph is in flight.
 */
typedef struct gn_graph gn_graph;
int glassnet_graph_create(const gn_model* model, const gn_frame* frames, int n, gn_graph** out);
int glassnet_graph_launch(gn_graph* graph, cudaStream_t stream);
int glassnet_graph_update(gn_graph* graph, const gn_frame* frames, int n);
void glassnet_graph_free(gn_graph* graph);

/*
 * Serving loop.  A server owns `n_streams` lanes; each lane is a CUDA stream
 * with a device arena for the largest request (max_h x max_w, max_K) and a
 * CUDA graph per request shape (h, w, K) captured on first use.  Requests
 * carry HOST buffers (page-locked for full copy bandwidth; they must stay
 * valid until glassnet_server_wait returns for the request).  A dispatcher
 * thread admits requests in arrival order once a lane is free and the bytes
 * of all admitted requests stay within `budget_bytes`; on the lane's stream it
 * copies the scene latent and the inputs to the device, replays the graph and
 * copies RGB back.  Lanes run concurrently, so copies overlap kernels.  A
 * completion thread records each request's latency (submission to result in
 * host memory).  Scenes are encoded once (glassnet_server_add_scene) and kept
 * resident; when `max_scenes` are resident the least recently used one is
 * replaced (after its requests finish).  Each request's image equals
 * glassnet_render_host of the same inputs alone, bit for bit.  The paper has
 * no counterpart (its Sec. 5 times single frames); device errors of the
 * kernels accumulate in the model's error word (glassnet_check).
 *
 * Functions may be called from any thread; glassnet_server_destroy waits for
 * every submitted request, then joins the threads and frees the server.
 * Errors: GN_EINVAL (bad config, request outside the maximum or the budget,
 * unknown scene or ticket), GN_ENOMEM, GN_ECUDA (a request whose device work
 * failed; glassnet_server_wait returns it).
 */
typedef struct gn_server gn_server;
typedef struct gn_server_config {
  int n_streams;        /* lanes, 1..16 */
  int max_scenes;       /* resident scene latents */
  size_t budget_bytes;  /* device bytes of admitted requests' buffers */
  int max_h, max_w;     /* largest request */
  int max_K;            /* largest layer-slot count, 0..8 */
} gn_server_config;
typedef struct gn_request {
  int scene;                  /* id from glassnet_server_add_scene */
  const float* gbuf;          /* host [14][h][w] */
  const float* tbuf;          /* host [K][12][h][w] (NULL if K = 0) */
  const uint8_t* layer_count; /* host [h][w] */
  int K, h, w;
  float* out;                 /* host [3][h][w] */
} gn_request;
typedef struct gn_server_stats {
  uint64_t submitted, completed;
  double p50_ms, p99_ms, mean_ms, max_ms;  /* latency of completed requests */
  double pixels;                           /* pixels of completed requests */
} gn_server_stats;
int glassnet_server_create(gn_model* model, const gn_server_config* config, gn_server** out);
/* Encodes `scene` (host, 32 floats) on a private stream and keeps its latent
 * resident; concurrent calls take different slots, and a call waits while
 * every slot is being encoded by another call or used by requests in flight. */
int glassnet_server_add_scene(gn_server* server, const float* scene, int* scene_id);
/* Captures the graph of the shape bucket (h, w, K) on every lane now, so that
 * the first requests of that shape do not wait for a capture.  Call it while
 * no request is queued or in flight (GN_EINVAL otherwise).  Synchronous. */
int glassnet_server_prepare(gn_server* server, int h, int w, int K);
int glassnet_server_submit(gn_server* server, const gn_request* request, uint64_t* ticket);
int glassnet_server_wait(gn_server* server, uint64_t ticket, double* latency_ms);
/* Where a request's latency went (milliseconds).  Host clock: waiting in
 * the queue for a lane and the budget, enqueueing its copies and graph on
 * the lane's stream, and from then until the completion thread saw the
 * lane's event (device_ms); total = the sum, as glassnet_server_wait reports
 * it.  Device clock (CUDA events on the lane's stream), the parts of
 * device_ms: copies of the latent and the inputs (including any wait for a
 * copy engine), the plan and fused kernels (including any wait for SMs) and
 * the read-back of the image. */
typedef struct gn_request_times {
  double queue_ms, enqueue_ms, device_ms, total_ms;
  double copy_in_ms, render_ms, copy_out_ms;
} gn_request_times;
/* As glassnet_server_wait, with the latency's parts. */
int glassnet_server_wait_times(gn_server* server, uint64_t ticket, gn_request_times* times);
int glassnet_server_stats(gn_server* server, gn_server_stats* stats);
void glassnet_server_destroy(gn_server* server);

/*
 * Synchronises `stream`, then returns and clears the model's device error
 * bits: GN_ETIMEOUT (a device wait gave up), GN_EINVAL (a layer count above
 * K), GN_ERANGE (a pixel's exact set-sum reached 2^11 and lost exactness),
 * GN_ESATURATED (an FP8 input was clamped), in that order of precedence, or
 * GN_OK.  GN_ECUDA if the stream reports a CUDA error.
 */
int glassnet_check(const gn_model* model, cudaStream_t stream);

/*
 * Test hook for the device-side timeout path (the paper has no counterpart).
 * The next fused launch of this GN_BF16_FUSED or GN_FP8_FUSED model (one
 * render, batch or streamed launch; either layer schedule) makes its MMA warp
 * wait `stall_ns` nanoseconds (1 ns .. 1 s) on a barrier that nothing arrives
 * on, after the weights are in shared memory and before any MMA is issued;
 * the wait gives up, every warp of the kernel leaves through its exit path
 * (which leaves no MMA or bulk copy in flight and frees the tensor memory),
 * the frame is not written, and the next glassnet_check returns GN_ETIMEOUT.
 * Later launches render normally.  Do not arm it around a graph capture (the
 * stall would be captured).
 * Errors: GN_EINVAL (NULL model, GN_FP32_PLAIN, stall out of range).
 */
int glassnet_debug_stall_next_render(gn_model* model, uint64_t stall_ns);

/* How the fused BF16 kernel runs the ragged layer work of Eq. 5 (each pixel
 * pools over its own c_p <= K layers).
 * GN_SCHEDULE_SORTED (default): 128-pixel tiles whose pixels are sorted by
 *   layer count within windows of 512 pixels; a tile runs as many layer slots
 *   as its largest count (1.42 executed rows per valid (pixel, layer) row at
 *   Poisson(3) counts).
 * GN_SCHEDULE_COMPACT: the valid (pixel, layer) rows of 256 pixels are packed
 *   slot-major into 128-row layer tiles (about 1.08 executed rows per valid
 *   row) and each pixel's pool is kept in shared memory.  Built for H = 64
 *   without positional encoding and with the 1x1 R (the pool of 256 pixels
 *   takes 128 KB of shared memory beside the operands). */
typedef enum gn_schedule {
  GN_SCHEDULE_SORTED = 0,
  GN_SCHEDULE_COMPACT = 1
} gn_schedule;

/*
 * Selects the layer schedule of a GN_BF16_FUSED model's frame renders
 * (glassnet_render*, the server).  Both schedules give bit-identical frames;
 * streamed layers (glassnet_accumulate_layer / glassnet_resolve) always use
 * the sorted kernel.  Call it outside stream capture (it sets the kernel's
 * attributes) and not while a render of the model is being enqueued.
 * Errors: GN_EINVAL (NULL model, unknown schedule), GN_EUNSUPPORTED
 * (GN_SCHEDULE_COMPACT for another precision, H != 64, positional encoding
 * or a 3x3 R), GN_ECUDA.
 */
int glassnet_set_layer_schedule(gn_model* model, int schedule);

/*
 * The FP32 plain render with no device allocation.  The paper has no
 * counterpart; this is an ABI convenience.  glassnet_render grows a
 * model-owned workspace with cudaMalloc (synchronising the device) when it
 * meets a larger frame, and glassnet_render_ws needs a workspace allocated by
 * the caller.  Callers that cannot allocate device memory at render time (a
 * program whose device memory is all handed out up front by its own pooling
 * allocator, a frame loop that must never block in the allocator) use this
 * entry point instead: its scratch is a 48 MiB array in device memory that
 * the library defines statically.  A GPU maps it when the first
 * GN_FP32_PLAIN model is loaded on it (glassnet_load_weights looks up the
 * array's address with the model's device current) and holds it until the
 * process exits; this call itself maps and allocates nothing.
 *  - The model must have precision GN_FP32_PLAIN.  Other arguments and the
 *    result are those of glassnet_render.
 *  - Frames whose plain-path scratch (glassnet_workspace_bytes) exceeds
 *    48 MiB are rejected with GN_EINVAL and a message giving both sizes, e.g.
 *    base widths K = 4 fit up to about 14,000 pixels, doubled widths K = 8 up
 *    to about 4,400 pixels.
 *  - Every call only launches kernels (the address lookup is done at model
 *    load).  cudaDeviceReset invalidates every model and latent of the
 *    device, this entry point's set-up included: load the model again.
 *  - All calls on a device share the one array, and it keeps the previous
 *    call's contents (every call overwrites all scratch it reads).  Calls
 *    whose work overlaps on the GPU (different streams, no ordering between
 *    them) race on the scratch and give wrong results: serialise them.
 *  - Allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 */
int glassnet_render_fp32_static(const gn_model* model, const gn_latent* latent, const float* gbuf,
                                const float* tbuf, const uint8_t* layer_count, int K, int h, int w,
                                float* out, cudaStream_t stream);

void glassnet_free_latent(gn_latent* latent);
void glassnet_free_model(gn_model* model);

/* Message for the last failing call on this thread ("" if none). */
const char* glassnet_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GLASSNET_H_ */
