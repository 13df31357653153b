/*
 * libjde: JDE detect-and-track on one GB300 (sm_103a), C ABI.
 *
 * The operation follows the tracking-by-detection pipeline of
 * "Faster object tracking pipeline for real time tracking" (Soni, Shah, Vyas):
 * a Joint Detection and Embedding network (Sec. 3.1: DarkNet-53 backbone, FPN,
 * predictions from three layers, YOLOv3-style detection) turns a batch of
 * frames into per-frame detection rows of 518 values (Appendix A, first item:
 * 4 location values, object confidence, class score, 512-d embedding), which
 * are filtered by confidence, non-max suppressed (Appendix A, items 2-3) and
 * then associated to tracks per video stream with a Kalman filter, cosine
 * cost, motion gating, Hungarian assignment and a track lifecycle (Sec. 3
 * "Location Estimation" / "Association", Appendix A items 4-9).
 *
 * Conventions for every call:
 *  - Every call returns a jde_status; nothing throws, exits or traps.  On an
 *    error the handle keeps a message for jde_last_error().
 *  - "device" pointers are CUDA global-memory pointers on the handle's device;
 *    "host" pointers are ordinary (preferably pinned) host memory.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *    with device outputs are asynchronous on that stream; calls with host
 *    outputs synchronise it before returning.
 *  - The caller owns every buffer it passes; the library owns the weights,
 *    activations and per-stream tracker state inside the handle.
 *  - One handle is used by one host thread at a time.
 */
#ifndef JDE_H
#define JDE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct jde_handle jde_handle;

typedef enum {
  JDE_OK = 0,
  JDE_ERR_INVALID_ARG = 1, /* a size, pointer or option is out of range */
  JDE_ERR_OOM = 2,         /* device allocation failed */
  JDE_ERR_CUDA = 3,        /* a CUDA runtime call failed */
  JDE_ERR_CAPACITY = 4,    /* an output or state buffer is too small; counts hold the true sizes */
  JDE_ERR_ADMISSION = 5,   /* a stream slot cannot be granted within the HBM budget */
  JDE_ERR_TIMEOUT = 6,     /* a device-side bounded wait gave up (kernel error word) */
  JDE_ERR_NOT_FOUND = 7,   /* unknown stream id or tensor id */
  JDE_ERR_WEIGHTS = 8,     /* weights blob malformed or does not match the layer table */
  JDE_ERR_UNSUPPORTED = 9  /* option not built into this library */
} jde_status;

/* JDE_FP8_E4M3: convolutions from the first stride-2 stage's output on take E4M3 activations
 * (one scale per stored tensor, amax / 448, set with jde_set_act_amax) and E4M3 weights (one
 * scale per output channel, max |W'| / 448 of the BN-folded weights, computed at create time),
 * accumulate in f32 and store E4M3 outputs; the stem and the next three layers run in BF16 and
 * the heads are written in f32. */
typedef enum { JDE_FP32 = 0, JDE_BF16 = 1, JDE_FP8_E4M3 = 2 } jde_precision;

/* Track states reported by jde_track_step (Appendix A: active / lost; the association cascade adds
 * unconfirmed tracks: born after a stream's first frame and not matched since). */
enum { JDE_TRACK_TRACKED = 1, JDE_TRACK_LOST = 2, JDE_TRACK_UNCONFIRMED = 3 };

/* Values a detection row carries (Appendix A: [n, num_detections, 518]). */
#define JDE_ROW 518
#define JDE_EMB 512
#define JDE_NUM_LAYERS 78

typedef struct {
  int precision;        /* jde_precision of the convolutions */
  int max_batch;        /* most frames per jde_detect_batch / jde_forward call */
  int max_in_w;         /* largest model input width  (multiple of 32) */
  int max_in_h;         /* largest model input height (multiple of 32) */
  int max_src_w;        /* largest source frame width  (for host->device staging) */
  int max_src_h;        /* largest source frame height */
  int max_cand;         /* K_max: candidates kept per frame after the confidence filter, <= 4096 */
  float conf_thresh;    /* keep conf >= conf_thresh (Appendix A item 2), default 0.5 */
  float nms_iou;        /* suppress IoU > nms_iou (Appendix A item 3), default 0.4 */
  float assign_thresh;  /* reject assigned pairs with cost > assign_thresh (item 7), default 0.7 */
  double gate_chi2;     /* gate squared Mahalanobis distance > gate_chi2 (item 6), default 9.487729036781154 */
  int lost_max_frames;  /* remove tracks lost for more frames (item 9), default 30 */
  float emb_momentum;   /* gallery update e <- norm(m e + (1-m) d), default 0.9 */
  int max_streams;      /* tracker state slots (video streams), default 64 */
  int max_tracks;       /* tracks per stream, default 1024 */
  int max_track_dets;   /* detections per frame entering the tracker, default 1024 */
  int device;           /* CUDA device ordinal */
  int keep_layer_outputs; /* 0 (default): in BF16-stored residual stages each block's 3x3 conv adds
                             its output into the block input's storage in place (the residual add
                             of Sec. 3 done by a TMA reduce-add), so the blocks' inputs are not kept,
                             and on tensor-core handles the stem runs fused with the first stride-2
                             conv, so the stem's output (layer 0) is never stored; jde_get_tensor /
                             jde_act_amax refuse those tensors; 1: every conv layer keeps its own
                             output tensor (per-layer inspection, calibration); 2: as 1, except that
                             the stem stays fused (inspection of the fused path; layer 0 refused) */
  int sparse_emb;       /* tensor-core handles, 1 (default): the embedding heads (Sec. 3.1, the linear
                           3x3 -> 512 of each scale) are evaluated only at the detections kept by NMS,
                           inside the post-processing of the handle's own forward (jde_detect_batch,
                           jde_postprocess with heads NULL), from copies of their input maps; their
                           dense maps are not computed (jde_get_tensor and jde_act_amax refuse them).
                           0: dense embedding maps */
  int assoc_cascade;    /* 0 (default): the single-stage association of Appendix A (items 5-9).  1: the
                           three-stage association of the cited JDE tracker: (1) confirmed tracks (tracked
                           or lost) against all detections on motion_lambda (1 - cos) + (1 - motion_lambda)
                           d^2 (d^2 the squared Mahalanobis distance, gated as in item 6), rejected above
                           assign_thresh; (2) the confirmed tracks left that were tracked before the frame,
                           against the detections left, on 1 - IoU(Kalman-predicted box, detection box),
                           rejected above iou_cost2; (3) unconfirmed tracks against the detections still
                           left on 1 - IoU, rejected above iou_cost3, an unmatched unconfirmed track being
                           removed; detections left start tracks, tracked on a stream's first frame and
                           unconfirmed after it */
  double motion_lambda; /* cascade stage 1 weight of the appearance cost, default 0.98 */
  double iou_cost2;     /* cascade stage 2 rejection threshold on 1 - IoU, default 0.5 */
  double iou_cost3;     /* cascade stage 3 rejection threshold on 1 - IoU, default 0.3 */
  int fuse_block1;      /* tensor-core handles with keep_layer_outputs = 0: 1 runs the first stage's
                           residual block (layers 2 and 3, Sec. 3.1) as one kernel whose 1x1 output
                           never leaves shared memory and whose output goes to its own tensor (tensor 2
                           is then refused by jde_get_tensor; 0.6 GB less DRAM traffic per batch-16
                           step, the same time alone, 2% slower when two batches share the GPU);
                           0 (default): two kernels, the block in place */
  int dependent_launch; /* tensor-core handles, 1 (default): each convolution kernel is launched as a
                           programmatic dependent of the kernel before it in the stream, so its launch and
                           set-up (barriers, tensor memory, cluster) overlap the previous layer's last work
                           units; it waits for that kernel to complete before it reads or writes global
                           memory, so results are identical; 0: plain stream order */
} jde_config;

/* One layer of the network as this library builds it (for the weights blob). */
typedef struct {
  int cin, cout, k, stride;
  int has_bn;        /* 1: BN statistics follow the weights in the blob, 0: a bias follows */
  int res_nblocks;   /* block count of the residual stage if the conv closes a residual branch, else 0 */
} jde_layer_desc;

/* Detection output of jde_detect_batch / jde_postprocess for n frames.
 * rows[f][i][0..517] = x1, y1, x2, y2 (source-frame pixels), conf, cls, unit embedding[512]
 * in kept order (confidence descending, canonical anchor index ascending).
 * count[f] is the number of kept detections of frame f (it may exceed `cap`,
 * in which case only `cap` rows were written).  anchor_index (optional) holds
 * the canonical anchor index of each row: off_s + (a H_s + y) W_s + x with the
 * heads ordered by stride 32, 16, 8. */
typedef struct {
  float* rows;            /* [n][cap][518] */
  int32_t* count;         /* [n] */
  int32_t* anchor_index;  /* [n][cap] or NULL */
  int cap;
  int on_device;          /* 1: all pointers are device pointers, 0: host pointers */
} jde_dets;

/* Track output of jde_track_step for n streams: the tracks alive after the
 * step, in track order (creation order).  box is the Kalman state mean as
 * x1, y1, x2, y2 in source-frame pixels; det is the row of the frame's
 * detection assigned to the track this step, or -1. */
typedef struct {
  int64_t* id;      /* [n][cap] */
  float* box;       /* [n][cap][4] */
  int32_t* state;   /* [n][cap] JDE_TRACK_* */
  int32_t* det;     /* [n][cap] */
  int32_t* count;   /* [n] */
  int cap;
  int on_device;
} jde_tracks;

/* Fill *cfg with the defaults listed above (precision BF16, max_batch 16, 1088x608 from 1920x1080). */
void jde_default_config(jde_config* cfg);

/* Copy the layer table (JDE_NUM_LAYERS entries, weights-blob order) into out[0..cap).
 * Returns the number of layers.  Pure host code; needs no GPU. */
int jde_layer_table(jde_layer_desc* out, int cap);

/* Create a handle on cfg->device.  `weights` (host, nbytes) is a blob:
 *   "JDEW", u32 version = 1, u32 n_layers, u32 0, then per layer
 *   u32 cin, cout, k, stride, flags (1 = BN, 2 = bias), 0, 0, 0 and f32
 *   W[cout][cin][k][k] followed by gamma, beta, mean, var [cout] (BN, eps 1e-5)
 *   or bias[cout].
 * The blob is copied; BN is folded and weights are packed on the device.
 * Errors: JDE_ERR_WEIGHTS if the blob does not match jde_layer_table,
 * JDE_ERR_OOM, JDE_ERR_CUDA, JDE_ERR_INVALID_ARG. */
jde_status jde_create(const jde_config* cfg, const void* weights, size_t nbytes, jde_handle** out);

/* Release everything the handle owns.  jde_destroy(NULL) is a no-op. */
void jde_destroy(jde_handle* h);

/* Message of the last failed call on h (or of the last failed jde_create when h is NULL). */
const char* jde_last_error(jde_handle* h);

/* Letterbox + network forward (Sec. 3.1) for n frames of src_w x src_h uint8
 * RGB (HWC, rows tightly packed, frames contiguous) into the handle's head
 * tensors at model input in_w x in_h.  `frames` is a device pointer when
 * on_device, else host memory copied inside the call on `stream`.
 * Letterbox: r = min(in_w/src_w, in_h/src_h), resized size floor(src r + 0.5),
 * centred, bilinear with half-pixel centres, /255, pad value 0.5. */
jde_status jde_forward(jde_handle* h, const uint8_t* frames, int n, int src_w, int src_h,
                       int in_w, int in_h, int on_device, void* stream);

/* Decode, confidence filter, NMS and embedding gather/L2-normalise (Sec. 3.2,
 * Appendix A items 1-3) for n frames.  heads[0..2] are the detection maps of
 * strides 32, 16, 8 ([n][H_s][W_s][24] f32, channels 6a..6a+5 = tx, ty, tw, th,
 * t_obj, t_cls of anchor a), heads[3..5] the embedding maps
 * ([n][H_s][W_s][512] f32), all device pointers; NULL heads means the
 * handle's own heads from the last jde_forward (with sparse_emb, its embedding
 * head is then evaluated at the kept detections only, from the input maps that
 * forward kept).  Boxes are mapped back to src_w x src_h frame pixels. */
jde_status jde_postprocess(jde_handle* h, const float* const* heads, int n, int in_w, int in_h,
                           int src_w, int src_h, jde_dets* out, void* stream);

/* Head tensors are double-buffered: the k-th jde_forward on a handle writes
 * set k mod 2 and jde_postprocess(heads = NULL) reads the set of the last
 * forward (the copies of the embedding head's input maps kept for sparse_emb
 * follow the same two sets).  So the post-processing of batch k, enqueued on a second stream
 * after an event recorded behind forward k, may run while forward k+1 runs;
 * forward k+2 overwrites the set of batch k and must be ordered after that
 * post-processing by the caller (e.g. cudaStreamWaitEvent). */

/* jde_forward followed by jde_postprocess on the handle's heads. */
jde_status jde_detect_batch(jde_handle* h, const uint8_t* frames, int n, int src_w, int src_h,
                            int in_w, int in_h, int on_device, jde_dets* out, void* stream);

/* One tracker step (Appendix A items 4-9) for n streams: stream_ids[i] (host
 * array, distinct ids in [0, max_streams)) consumes frame i of `dets` (device
 * rows as written by jde_postprocess).  Tracker state stays on the device. */
jde_status jde_track_step(jde_handle* h, int n, const int32_t* stream_ids, const jde_dets* dets,
                          jde_tracks* out, void* stream);

/* Forget all tracks of a stream and restart its ids at 1 (asynchronous on stream). */
jde_status jde_stream_reset(jde_handle* h, int stream_id, void* stream);

/* Copy an internal tensor to `dst` (device pointer, dst_bytes capacity) for
 * inspection: id 0..77 = output of conv layer id (after its fused epilogue:
 * bias, leaky-ReLU, residual add), 100 = letterboxed input.  dims receives {n, h, w, c} of the unpadded tensor, *dtype
 * 0 = f32, 1 = bf16, 2 = E4M3 codes (value = code * amax / 448 of its tensor); the copy is
 * the unpadded tensor in NHWC order.  dst NULL
 * only reports dims and dtype.  JDE_ERR_NOT_FOUND for the input of an in-place residual block
 * (its storage holds the block's output; see keep_layer_outputs). */
jde_status jde_get_tensor(jde_handle* h, int id, void* dst, size_t dst_bytes, int* dims, int* dtype,
                          void* stream);

/* Device error word accumulated by the kernels (bit 0: bounded wait timed out,
 * bit 1: capacity overflow); reading it synchronises `stream` and clears it. */
jde_status jde_kernel_errors(jde_handle* h, int* word, void* stream);

/* E4M3 handles: per-layer output amax (n = JDE_NUM_LAYERS values, layer order of the weights
 * blob, finite and >= 0) from calibration frames, e.g. the elementwise maximum of
 * jde_act_amax over calibration batches run on a BF16 handle.  The scale of a stored tensor is
 * amax / 448; a concat buffer takes the larger amax of the two layers writing into it.  Must be
 * called before the handle's first jde_forward (else that returns JDE_ERR_INVALID_ARG); calling
 * it again replaces the scales.  Other handles: JDE_ERR_INVALID_ARG. */
jde_status jde_set_act_amax(jde_handle* h, const float* amax, int n);

/* max |value| of every layer output of the handle's last jde_forward (all its frames), into
 * amax[JDE_NUM_LAYERS] (host); synchronises `stream`.  Heads and BF16/f32 tensors as stored;
 * E4M3 tensors as code times scale.  Needs every layer output: JDE_ERR_UNSUPPORTED unless the
 * handle keeps them (keep_layer_outputs = 1, or an FP32 handle). */
jde_status jde_act_amax(jde_handle* h, float* amax, void* stream);

/* Tile autotuner (tensor-core handles): for batches of n frames at in_w x in_h, times every
 * built tile width (64/128/256 output channels, 32 where that is the default; 256 runs on CTA
 * pairs; for the stride-1 3x3 convs also 128 channels x 256 rows per CTA, tile code 129; for the
 * other BF16 convs of 128-byte k-blocks also 128 channels on CTA pairs, tile code 130) of every
 * convolution that has more than one, on `stream` with CUDA events on the handle's
 * activation buffers (the median of five launches, each right after a launch of the layer before it,
 * so the input is as cached as in a forward), and keeps the fastest for later forwards of that shape.  Results do not
 * change: every tile computes each output with the same K order.  Synchronises `stream`;
 * overwrites intermediate activations (the next forward recomputes them).  E4M3 handles need
 * their scales first. */
jde_status jde_autotune(jde_handle* h, int n, int in_w, int in_h, void* stream);

/* Tile code used per layer (bn[JDE_NUM_LAYERS]) for batches of n at in_w x in_h: the tuned
 * choice if jde_autotune ran for that shape, else the default rule.  The code is the tile's output
 * channel count, plus 1 when each CTA computes two 128-row sub-tiles (256 rows) per tile, plus 2
 * when a 128-wide tile runs on a CTA pair. */
jde_status jde_tile_choice(jde_handle* h, int n, int in_w, int in_h, int* bn);

/* Set the tile code of every layer (bn[JDE_NUM_LAYERS]; 0 = the default rule) for batches of n at
 * in_w x in_h, as jde_autotune would (e.g. to reuse its choice, read with jde_tile_choice, in
 * another process).  Plans are rebuilt on the host at once: a code a layer cannot run (a width
 * its channel count is not a multiple of, a layer with one tile shape, code 129 where the
 * windows do not fit, or code 130 on a flat-window or E4M3 conv) returns JDE_ERR_INVALID_ARG or JDE_ERR_UNSUPPORTED and keeps the previous
 * choice.  Results do not change (same K order for every tile). */
jde_status jde_set_tile_choice(jde_handle* h, int n, int in_w, int in_h, const int* bn);

/* Device memory the handle holds now (weights, activation buffers of every
 * input size used so far, post-processing and tracker state, staging), in bytes. */
jde_status jde_device_bytes(jde_handle* h, size_t* out);

/* Device memory a handle created with *cfg holds once it has run batches of
 * cfg->max_batch frames at in_w x in_h with device-resident frames (host-fed
 * frames add max_batch * src_w * src_h * 3 bytes of staging).  For admission
 * against a memory budget before jde_create; allocates nothing. */
jde_status jde_estimate_device_bytes(const jde_config* cfg, int in_w, int in_h, size_t* out);

/* Number of kernels libjde has launched in this process (all handles), for launch accounting. */
unsigned long long jde_launch_count(void);

/* Stage timing: when set (cudaEvent_t values, or NULL to stop), jde_forward
 * records forward_begin before the letterbox, conv_begin before the first
 * convolution and conv_end after the last one, on the call's stream.  The
 * events stay owned by the caller. */
jde_status jde_set_profile_events(jde_handle* h, void* forward_begin, void* conv_begin, void* conv_end);

/* Sets the handle's jde_config.dependent_launch (0 or 1) for the launches it makes from now on (a CUDA
 * graph captured earlier keeps the launches it captured).  Dependent launches shorten one forward
 * stream's convolution chain; where two forwards share the GPU on two streams, plain stream order lets
 * each fill the SMs the other's layer tails leave idle.  Results are identical either way.
 * JDE_ERR_INVALID_ARG for another value. */
jde_status jde_set_dependent_launch(jde_handle* h, int on);

/* Failure-detection self-test (no counterpart in the paper).  Every kernel that waits on another warp
 * or CTA waits on an mbarrier with a cycle limit (about 2^32 SM cycles, two seconds); when the limit
 * passes, the kernel sets bit 0 of the handle's error word, skips its remaining work and returns, so a
 * lost signal never hangs the GPU.  This call exercises that path: one thread waits on a phase of a
 * fresh mbarrier that nothing completes, with limit_cycles (1 .. 2^31) as the limit.  The call then
 * reads and clears the error word (synchronising `stream`) into *word and returns JDE_ERR_TIMEOUT
 * with bit 0 set; nothing traps and the context stays usable. */
jde_status jde_selftest_wait(jde_handle* h, long long limit_cycles, int* word, void* stream);

/* Post-processing for callers that cannot allocate device memory: code that
 * runs after a host application has reserved all device memory, a real-time
 * loop where a cudaMalloc (which can synchronise the device) is not allowed,
 * or a plugin that receives device pointers but no allocator.  The paper has
 * no counterpart; this is a deployment variant of jde_postprocess.
 * Same computation and rows as jde_postprocess with the thresholds passed in
 * (conf_thresh, nms_iou, max_cand = K_max, a multiple of 64 in [64, 4096]).
 * It needs no handle and calls no cudaMalloc, cudaFree or allocating library
 * routine: heads[0..5] (device, layout as in jde_postprocess) and the outputs
 * (device; out->on_device must be 1) are the caller's, and all scratch comes
 * from one fixed 32 MiB device array compiled into the library.  CUDA loads
 * that array onto a device the first time its address is looked up there -
 * by jde_create for the handle's device, or else by the first call of this
 * function on that device - and the device holds the 32 MiB from then until
 * the process exits; so create a handle, or make that first call, before the
 * application reserves the device's memory.  in_w, in_h <= 16384.  A call needs about
 * n * (8 * anchors + max_cand * (36 + max_cand / 8)) bytes of it (anchors =
 * 4 * (in_w*in_h/1024 + in_w*in_h/256 + in_w*in_h/64)); a larger request
 * returns JDE_ERR_CAPACITY with the sizes in err_msg (e.g. 16 frames at
 * 1088x608 fit with max_cand <= 2048).
 * The first call on a device with no handle looks up the array's device
 * address (cudaGetSymbolAddress) with that device current: make that first
 * call before any stream capture.  Every call uses the same array and leaves its
 * contents behind; two calls that can overlap on the GPU (different streams
 * or host threads) race, so the caller must serialise them.
 * err_msg (optional, err_len bytes) receives the reason of a failure. */
jde_status jde_postprocess_noalloc(const float* const* heads, int n, int in_w, int in_h, int src_w, int src_h,
                                   float conf_thresh, float nms_iou, int max_cand, jde_dets* out, void* stream,
                                   char* err_msg, size_t err_len);

/* ---------------------------------------------------------------------------------------------
 * Serving many video streams in one process (the paper's capture -> prediction -> post-processing
 * pipeline of Sec. 4.3-4.4, Fig. 4, generalised from one video to many).
 *
 * A server groups streams by model input size.  A group owns one handle (created from
 * cfg.group with max_in_w/h = the group's size, max_src_w/h = src_w/h, max_streams =
 * max_streams_per_group), one CUDA stream and its batch buffers.  jde_stream_open admits a stream
 * into the group of its size when that group has a free tracker slot, or creates the group when
 * jde_estimate_device_bytes of its handle plus its batch buffers fits in what hbm_budget_bytes has
 * left (else JDE_ERR_ADMISSION, nothing allocated).  jde_submit queues one frame of a stream;
 * jde_poll, which never blocks, collects finished batches and starts, in every group with no batch on
 * the device, a batch of the queued frames (at most max_batch, at most one per stream, oldest first).
 * A batch is forward + post-processing + tracker step of its frames on the group's stream.  With
 * use_graphs the launch sequence of a batch of n frames is captured into a CUDA graph the second
 * time a batch of n frames starts in that group (the first runs eagerly and sets everything up)
 * and replayed from then on.  The server is not thread-safe: one host thread drives it.
 * ------------------------------------------------------------------------------------------- */
typedef struct jde_server jde_server;

typedef struct {
  jde_config group;          /* template of each group's handle (precision, max_batch = frames per batch,
                                thresholds, tracker options, device); sizes are set per group as above.
                                With caller_heads the handles compute the embedding heads densely
                                (sparse_emb forced to 0), so the forward does all of its work. */
  int src_w, src_h;          /* size of every stream's frames (uint8 RGB, HWC, rows tightly packed) */
  int max_streams_per_group; /* tracker slots of a group, 1..1024 */
  size_t hbm_budget_bytes;   /* device bytes the groups may be charged in total */
  int det_cap;               /* detection rows kept per frame (jde_dets.cap of the groups) */
  int track_cap;             /* tracks reported per frame (jde_tracks.cap) */
  int caller_heads;          /* 1: every frame is submitted with its six head tensors (layout of
                                jde_postprocess), which the post-processing reads instead of the
                                network's; 0: the network's own heads */
  int collect_net_heads;     /* 1: the network's three detection maps of each frame are kept and can be
                                returned through jde_frame_out.net_det */
  int use_graphs;            /* 1: replay each batch size's launch sequence as a CUDA graph */
  int prewarm;               /* 1: a new group runs every batch size it can see (1 .. min(max_batch,
                                max_streams_per_group)) once on zeroed inputs and captures its graph
                                before its first stream is admitted, so no set-up or capture delays a
                                served batch; its tracker slots are reset afterwards */
} jde_server_config;

/* Host buffers a frame's results are written to when jde_poll returns it (each optional, NULL to
 * skip; they must stay valid until then).  Track arrays hold track_cap entries, rows det_cap rows
 * of JDE_ROW values, net_det[k] the [H_k][W_k][24] f32 detection map of stride 32, 16, 8 (needs
 * collect_net_heads). */
typedef struct {
  int64_t* track_id;
  float* track_box;     /* [track_cap][4] */
  int32_t* track_state; /* JDE_TRACK_* */
  int32_t* track_det;   /* row of the frame's detection assigned to the track, or -1 */
  float* rows;          /* [det_cap][518] as jde_postprocess writes them */
  float* net_det[3];
} jde_frame_out;

typedef struct {
  long long ticket;   /* as returned by jde_submit */
  int stream_id;
  int n_dets;         /* detections kept (rows beyond det_cap were not written) */
  int n_tracks;       /* tracks alive after the step (beyond track_cap not reported) */
  int errors;         /* kernel error word of the frame's batch (jde_kernel_errors), 0 if none; -1
                         when the batch could not be launched or did not complete (nothing else of
                         the result is filled in) */
  float done_ms;      /* device time at which the frame's batch finished, ms after the server's clock
                         start (jde_server_create or jde_server_reset_clock) */
} jde_frame_result;

/* Fill *cfg with defaults: jde_default_config for the groups, 1920x1080 sources, 16 streams per group,
 * budget 64 GiB, det_cap 256, track_cap 256, network heads, no collection, graphs on, prewarm on. */
void jde_default_server_config(jde_server_config* cfg);

/* Create a server (no device memory until a stream is opened).  `weights` is the blob of
 * jde_create, copied.  Errors: JDE_ERR_INVALID_ARG, JDE_ERR_CUDA. */
jde_status jde_server_create(const jde_server_config* cfg, const void* weights, size_t nbytes, jde_server** out);

/* Wait for the device work of every group, then release everything.  NULL is a no-op. */
void jde_server_destroy(jde_server* s);

/* Message of the last failed call on s. */
const char* jde_server_last_error(jde_server* s);

/* Restart the clock of done_ms: records the start event and waits for it. */
jde_status jde_server_reset_clock(jde_server* s);

/* Admit a stream with model input size in_w x in_h (multiples of 32); its tracker slot starts empty.
 * *stream_id receives its id (ids are never reused).  JDE_ERR_ADMISSION when neither a free slot
 * nor the budget allows it; JDE_ERR_OOM / JDE_ERR_WEIGHTS / JDE_ERR_CUDA from creating a group. */
jde_status jde_stream_open(jde_server* s, int in_w, int in_h, int* stream_id);

/* Finish the stream's submitted frames (their results stay queued for jde_poll), free its slot, and
 * destroy its group, returning the group's charge to the budget, when no stream is left in it.
 * JDE_ERR_NOT_FOUND for an unknown id. */
jde_status jde_stream_close(jde_server* s, int stream_id);

/* Queue one frame of a stream.  `frame` (device, src_h x src_w x 3 uint8) and, with caller_heads,
 * heads[0..5] (device) must stay unchanged until the frame's result is returned by jde_poll.
 * ready_event (a cudaEvent_t, or NULL): the server's first read of the frame's inputs waits on the
 * device for the event as recorded when the frame's batch starts, so a caller that fills the inputs
 * on its own CUDA stream need not synchronise.  `out` (copied) names host buffers for its results,
 * or NULL.  *ticket (optional) receives the frame's ticket, increasing from 1.  Frames of a stream
 * are processed in submission order. */
jde_status jde_submit(jde_server* s, int stream_id, const uint8_t* frame, const float* const* heads,
                      void* ready_event, const jde_frame_out* out, long long* ticket);

/* Advance the server without blocking (see above) and move up to cap results of finished frames
 * into results[0..*n), in completion order.  A failed launch or batch returns its status (the
 * message in jde_server_last_error); its frames still get their results, with errors = -1, so every
 * submitted frame gets exactly one result. */
jde_status jde_poll(jde_server* s, jde_frame_result* results, int cap, int* n);

/* Device bytes a group of in_w x in_h is charged at creation: jde_estimate_device_bytes of its handle's
 * configuration plus its batch buffers (frames, caller heads, detection rows, track outputs, the
 * network's detection maps when collected, stream slots).  Pure host arithmetic; needs no GPU. */
jde_status jde_server_group_cost(const jde_server_config* cfg, int in_w, int in_h, size_t* out);

/* Block until every submitted frame has finished (results stay queued for jde_poll). */
jde_status jde_server_flush(jde_server* s);

/* *charged: bytes charged to the budget by the open groups; *held: device bytes their handles hold
 * (jde_device_bytes) plus their batch buffers.  Either pointer may be NULL. */
jde_status jde_server_device_bytes(jde_server* s, size_t* charged, size_t* held);

/* Counters of the server: batches launched eagerly, graphs captured, graph replays. */
jde_status jde_server_stats(jde_server* s, long long* eager, long long* captured, long long* replays);

/* ---------------------------------------------------------------------------------------------
 * Device decode of compressed frames (the capture stage of Sec. 4.4, on the GPU, for Motion-JPEG
 * video streams).  A decoder turns baseline JPEG bitstreams in host memory into interleaved 8-bit
 * RGB frames in device memory (n x h x w x 3, the layout jde_forward and jde_submit read) with
 * nvJPEG: on the GPU's JPEG decode engines (JDE_DECODE_HARDWARE) when they are available, else with
 * the GPU-assisted hybrid backend (JDE_DECODE_GPU_HYBRID).  libnvjpeg is loaded at run time; where
 * it is absent every decoder call returns JDE_ERR_UNSUPPORTED.
 * ------------------------------------------------------------------------------------------- */
typedef struct jde_decoder jde_decoder;
enum { JDE_DECODE_HARDWARE = 1, JDE_DECODE_GPU_HYBRID = 2 };

/* Create a decoder on `device` for batches of up to max_batch frames (1..1024); hardware = 1 asks
 * for the JPEG engines.  JDE_ERR_UNSUPPORTED when nvJPEG cannot be loaded or set up. */
jde_status jde_decoder_create(int device, int max_batch, int hardware, jde_decoder** out);

/* Release the decoder (synchronises its device).  NULL is a no-op. */
void jde_decoder_destroy(jde_decoder* d);

/* Message of the last failed call on d. */
const char* jde_decoder_last_error(jde_decoder* d);

/* The backend in use: JDE_DECODE_HARDWARE or JDE_DECODE_GPU_HYBRID (0 for NULL). */
int jde_decoder_backend(jde_decoder* d);

/* Decode n (1..max_batch) JPEG bitstreams (host pointers and lengths; each must be a 3-component
 * w x h image, checked on the host from its headers before any device work: JDE_ERR_INVALID_ARG
 * otherwise) into frames (device, n x h x w x 3 uint8, frames contiguous) on `stream`.  The
 * bitstreams must stay valid until the call returns. */
jde_status jde_decode_jpeg(jde_decoder* d, const uint8_t* const* bitstreams, const size_t* lengths, int n, int w,
                           int h, uint8_t* frames, void* stream);

/* Encode n frames (device, n x h x w x 3 uint8 RGB) as baseline JPEG with 4:2:0 chroma subsampling at
 * `quality` (1..100) into out[i] (host buffers; lengths[i] holds each buffer's capacity on entry and
 * the bitstream's length on return).  A buffer too small returns JDE_ERR_CAPACITY with the length it
 * needs in lengths[i].  Synchronises `stream`.  For making synthetic compressed streams. */
jde_status jde_encode_jpeg(jde_decoder* d, const uint8_t* frames, int n, int w, int h, int quality,
                           uint8_t* const* out, size_t* lengths, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* JDE_H */
