// Internal interfaces between the translation units of libjde.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/jde.h"
#include "common.cuh"

// One convolution launch: out = act(conv(in, W) + bias) (+ res), optionally
// written 2x2-replicated (nearest upsample) into a concat slice.
struct ConvSpec {
  int k, stride, cin, cout;
  TView in, out, res;   // res.ptr == nullptr: no residual
  int Ho, Wo;           // conv output size (before any upsample)
  int act;              // 1: leaky-ReLU(0.1), 0: linear
  int upsample;         // 1: write each output pixel to a 2x2 block of `out`
  const float* bias;    // [cout_pad] f32
  int* err;
  // FP8 (E4M3) operands: acc * mult[co] + bias[co] (mult = input scale * weight scale of channel co)
  int q;                // 1: input and weights are E4M3 codes
  const float* mult;    // [cout_pad] f32 when q
  float res_scale;      // value of one residual code (res.dtype == 2)
  float out_inv_scale;  // 1 / scale of the output tensor (out.dtype == 2)
};

// SIMT f32 path: weights [K_pad16][cout_pad64] f32, K = (ky*k + kx)*cin + ci.
void conv_simt_launch(const ConvSpec& c, const float* w_kn, int cout_pad64, cudaStream_t st);

// tcgen05 bf16 path.  Weights [cout_pad][K] bf16 (K-major), K = (ky*k + kx)*cin + ci.
struct TcPlan {
  alignas(64) CUtensorMap a[4];  // activations: flat 2-D map, or 4 stride-2 phase maps
  alignas(64) CUtensorMap b;     // weights
  alignas(64) CUtensorMap o;     // output (TMA-stored epilogue), valid when tma_out
  alignas(64) CUtensorMap r;     // residual (TMA-loaded into the staging tile), valid when tma_res
  int tma_out, tma_res;
  int red_res;                   // output aliases the residual: the epilogue reduce-adds into it
  int mode;                      // 0 flat (stride 1 over the padded pixel array), 1 patch (stride 2),
                                 // 2 stem gather, 3 32-channel window, 4 flat window (stride-1 3x3)
  int bn, bkc;
  int kt_total, cin_blocks;
  int m_tiles, n_tiles;
  int M_total, Hp, Wp;
  int TW, TH, tiles_x, tiles_y;
  int WW, WH, win_bytes, plane;  // mode 3: (sub-)window pixels, bytes per buffer, bytes per 8-channel plane
  int nwin;                      // modes 3, 4: window buffers in the ring
  int wnb, whb;                  // mode 4: TMA boxes per window, pixel rows per box
  int cg;                        // 2: 256-wide tiles on CTA pairs (cta_group::2), else 1
  int q;                         // 1: E4M3 operands (kind::f8f6f4)
  int kel;                       // elements of one k-block along K (bf16: bkc, E4M3: 2 * bkc)
  int msub;                      // mode 4: M tiles of 128 rows per CTA and work unit (1 or 2)
  int w4deep;                    // mode 4 with 128-byte k-blocks: 1 = the deeper weight ring
  int pdl;                       // 1: launched as a programmatic dependent of the previous kernel
  ConvSpec spec;
};
// Fill plan (tensor maps and grid) for a conv whose input is a padded bf16
// view and whose weights are w ([cout_pad][K] bf16).  Returns false with a
// message if the shape is not supported by the tensor-core path.
// w: [cout_pad][K] bf16, or E4M3 codes when c.q.
// msub = 2 (flat-window 3x3 convs with bn = 128 only): each CTA computes 256 rows x bn columns per
// work unit, two M=128 sub-tiles sharing every weight tile and one window.
// pair128 = 1 (stride-1 flat and stride-2 patch convs with bn = 128 only): the 128-wide tiles run on CTA
// pairs (M = 256 per MMA, each CTA loading half of every weight tile).
bool conv_tc_plan(TcPlan& plan, const ConvSpec& c, const void* w, int cout_pad, int bn, char* msg,
                  size_t msg_len, int msub = 1, int pair128 = 0);
cudaError_t conv_tc_launch(const TcPlan& plan, cudaStream_t st);
// Point a planned conv at another output buffer of the same shape (the double-buffered heads);
// re-encodes the output tensor map of a TMA-stored f32 head.  False if the map cannot be built.
bool conv_tc_retarget(TcPlan& plan, void* out);
int conv_tc_pick_bn(int cout);

// Letterbox geometry tables (per output column / row): source index pair and weight.
struct LbAxis {
  int i0, i1;
  float f;
  int inside;   // 1 inside the resized image, 0 in the letterbox padding
};
void letterbox_tables_launch(LbAxis* xs, LbAxis* ys, int src_w, int src_h, int dst_w, int dst_h, double r,
                             int nw, int nh, int px, int py, cudaStream_t st);
void letterbox_f32_launch(const uint8_t* frames, int n, int src_w, int src_h, const LbAxis* xs, const LbAxis* ys,
                          TView out, cudaStream_t st);
void letterbox_bf16x4_launch(const uint8_t* frames, int n, int src_w, int src_h, const LbAxis* xs,
                             const LbAxis* ys, TView out, cudaStream_t st);

// Post-processing.
struct HeadGeom {
  int n;
  int gh[3], gw[3];      // grid per head (strides 32, 16, 8)
  int off[4];            // canonical index offsets, off[3] = anchors per frame
  float anchor_w[12], anchor_h[12];
  int stride[3];
  float ratio, pad_x, pad_y;
  int epad;              // embedding maps carry a zero halo of this width (0 or 1)
};
struct PostBufs {
  uint64_t* cand_keys;   // [n][cand_cap]
  int* cand_count;       // [n]
  int cand_cap;
  uint64_t* sorted;      // [n][kmax]
  int* n_sorted;         // [n]
  float4* boxes;         // [n][kmax] letterbox xyxy
  float* conf;           // [n][kmax]
  float* cls;            // [n][kmax]
  unsigned long long* mask;  // [n][kmax][kmax/64]
  int* keep_idx;         // [n][kmax] positions in sorted order
  int* n_keep;           // [n]
  int kmax;
  int4* emb_list;        // [3][n * kmax] sparse embedding head: (frame, row, y, x) per kept detection
  int* emb_count;        // [3] kept detections per scale
};
// Sparse embedding head (Sec. 3.1, the linear 3x3 -> 512 of each scale) evaluated only at the
// locations kept by NMS: per scale the head's input feature map, its weights and epilogue constants.
struct EmbSparse {
  TView in[3];           // padded NHWC input of the head (bf16 or E4M3 codes)
  const void* w[3];      // [cout_pad][K] bf16, or E4M3 codes when q[s]
  const float* bias[3];  // [>= 512]
  const float* mult[3];  // E4M3: input scale x weight scale per channel, else null
  int cin[3];
  int ldw[3];            // elements per weight row (= 9 cin, a multiple of 64)
  int q[3];
};
// es != null: the embedding maps heads[3..5] are not read; the kept detections' embeddings are
// computed from es (sparse head, tensor cores) into their rows, then normalised.  Returns the launch
// status (cudaErrorInvalidValue when the sparse head's weight tensor maps cannot be built).
cudaError_t post_launch(const float* const* heads, const HeadGeom& g, float conf_thresh, float nms_iou, PostBufs& b,
                        float* rows, int32_t* count, int32_t* anchor_index, int cap, int* err, cudaStream_t st,
                        const EmbSparse* es = nullptr);

// Loads the fixed scratch array of jde_postprocess_noalloc onto the current device and records its
// address; 0 on success, else 1 with a reason in msg.
int noalloc_scratch_setup(char* msg, size_t len);

// Stem (layer 0) and the first stride-2 conv (layer 1) fused into one tcgen05 kernel: the stem's output
// stays in shared memory.  lb: the bf16 RGB0 letterbox (haloed); out: layer 1's output (bf16, 64
// channels, haloed); w0b: the stem's packed bf16 weights [32][32] with its bias in K columns 27..29;
// w1: layer 1's packed bf16 weights [64][320]; b1b: layer 1's bias parts [64][32] (K columns 0..2).
// stem_s2_pack writes w0b and b1b (bias = sum of three bf16 parts) from the packed weights and biases.
struct StemS2Plan;
constexpr size_t STEM_S2_PACK_BYTES = 32 * 32 * 2 + 64 * 32 * 2;   // w0b + b1b
cudaError_t stem_s2_pack(const void* w0, const float* bias0, const float* bias1, void* w0b, void* b1b,
                         cudaStream_t st);
StemS2Plan* stem_s2_plan_new(const TView& lb, const TView& out, const void* w0b, const void* w1, const void* b1b,
                             int* err, char* msg, size_t msg_len);
void stem_s2_plan_free(StemS2Plan* p);
cudaError_t stem_s2_launch(const StemS2Plan* p, cudaStream_t st);

// The first stage's residual block (1x1 64 -> 32, 3x3 32 -> 64, + input) fused into one tcgen05 kernel:
// the 1x1's output stays in shared memory.  x: the block input, out: the block output (another tensor:
// x is read on every patch's halo); w1: the 1x1's packed bf16 weights [32][64], w2: the 3x3's [64][320];
// b1, b2: their folded biases.  The output is leaky(3x3 + b2) + x rounded once to bf16.
struct Res1Plan;
Res1Plan* res1_plan_new(const TView& x, const TView& out, const void* w1, const void* w2, const float* b1,
                        const float* b2, int* err, char* msg, size_t msg_len);
void res1_plan_free(Res1Plan* p);
cudaError_t res1_launch(const Res1Plan* p, cudaStream_t st);

// jde_track_step whose kernels read the call's stream slots from dev_slots (device, n entries, the same
// values as stream_ids) instead of kernel arguments, so that a captured CUDA graph of the step serves
// any batch of n streams after the caller rewrites dev_slots.
jde_status track_step_device_slots(jde_handle* h, int n, const int32_t* stream_ids, const int* dev_slots,
                                   const jde_dets* dets, jde_tracks* out, cudaStream_t st);
