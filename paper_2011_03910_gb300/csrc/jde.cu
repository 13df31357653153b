// libjde C ABI: handle, layer table, weights, forward orchestration, post-processing glue.
//
// Network (Sec. 3.1 names DarkNet-53 + FPN + three prediction layers; the
// layer table itself is not printed, this is the reading used throughout):
//   stem 3x3 3->32; five stride-2 3x3 downsamples (64, 128, 256, 512, 1024)
//   each followed by 1/2/8/8/4 residual blocks (1x1 c->c/2, 3x3 c/2->c, add);
//   per scale (stride 32, 16, 8; mid 512, 256, 128): 1x1 mid, 3x3 2mid,
//   1x1 mid, 3x3 2mid, 1x1 mid -> F; detection 3x3 mid->2mid + linear 1x1
//   2mid->24; embedding linear 3x3 mid->512; lateral 1x1 mid->mid/2 upsampled
//   2x into channels [0, mid/2) of the next scale's concat, whose remaining
//   channels hold the backbone skip (C4 / C3).  BN is folded (eps 1e-5),
//   leaky-ReLU slope 0.1 after every conv except the two linear heads.
// Memory: every activation is NHWC with a 1-pixel zero halo, one buffer per
// layer output (no reuse: the whole pyramid of a max-size batch stays
// resident, a few GB of HBM), allocated per model-input resolution.  The
// backbone skips are written straight into their concat slices and the
// laterals' upsample is fused into their epilogue, so no concat copy runs.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/jde.h"
#include "internal.h"
#include "track.h"

static std::atomic<unsigned long long> g_launches{0};
void jde_count_launch(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace {

thread_local std::string g_create_error;

struct LayerDef {
  int cin, cout, k, stride, has_bn, res_nb;
};

std::vector<LayerDef> build_layers() {
  std::vector<LayerDef> L;
  L.push_back({3, 32, 3, 1, 1, 0});
  const int stage_c[5] = {64, 128, 256, 512, 1024};
  const int stage_n[5] = {1, 2, 8, 8, 4};
  for (int s = 0; s < 5; ++s) {
    const int c = stage_c[s];
    L.push_back({c / 2, c, 3, 2, 1, 0});
    for (int b = 0; b < stage_n[s]; ++b) {
      L.push_back({c, c / 2, 1, 1, 1, 0});
      L.push_back({c / 2, c, 3, 1, 1, stage_n[s]});
    }
  }
  const int head_cin[3] = {1024, 768, 384}, head_mid[3] = {512, 256, 128};
  for (int h = 0; h < 3; ++h) {
    const int ci = head_cin[h], m = head_mid[h];
    L.push_back({ci, m, 1, 1, 1, 0});
    L.push_back({m, 2 * m, 3, 1, 1, 0});
    L.push_back({2 * m, m, 1, 1, 1, 0});
    L.push_back({m, 2 * m, 3, 1, 1, 0});
    L.push_back({2 * m, m, 1, 1, 1, 0});
    L.push_back({m, 2 * m, 3, 1, 1, 0});   // det 3x3
    L.push_back({2 * m, 24, 1, 1, 0, 0});  // det 1x1 (linear)
    L.push_back({m, 512, 3, 1, 0, 0});     // emb 3x3 (linear)
    if (h < 2) L.push_back({m, m / 2, 1, 1, 1, 0});  // lateral
  }
  return L;
}

const std::vector<LayerDef>& layers() {
  static const std::vector<LayerDef> L = build_layers();
  return L;
}

int align_up(int v, int a) { return (v + a - 1) / a * a; }

// Weights folded and packed for both precisions' kernels.
struct LayerW {
  float* w_kn = nullptr;           // f32 [K_pad16][cout_pad64]
  __nv_bfloat16* w_nk = nullptr;   // bf16 [cout_pad_tc][K_tc]
  uint8_t* w_q = nullptr;          // E4M3 codes [cout_pad_tc][K_tc] (E4M3 layers)
  double* wscale = nullptr;        // E4M3 layers: per-channel weight scale [cout_pad_tc] (exact, for rounding)
  float* mult = nullptr;           // E4M3 layers: input scale * weight scale [cout_pad_tc]
  std::vector<double> wscale_host;
  float* bias = nullptr;           // f32 [bias_len]
  int cout_pad64 = 0, cout_pad_tc = 0, bn = 0, k_tc = 0;
  int q = 0;                       // 1: E4M3 operands
};

// E4M3 handles: layer outputs from this layer on are stored as E4M3 codes, and the layers
// after it take E4M3 inputs (the stem and the 32/64-channel layers before stay BF16).
constexpr int FP8_FIRST_OUT = 4;
bool is_q_layer(int precision, int l) { return precision == JDE_FP8_E4M3 && l > FP8_FIRST_OUT; }
int el_size(int dt) { return dt == 0 ? 4 : (dt == 1 ? 2 : 1); }
// Sparse embedding head: tensor-core handles with sparse_emb set.
bool sparse_emb_cfg(const jde_config& c) { return c.sparse_emb && c.precision != JDE_FP32; }
// Stem and first stride-2 conv fused (the stem's output is never stored): tensor-core handles, unless
// they keep every layer output (keep_layer_outputs = 1).
bool fused_stem_cfg(const jde_config& c) { return c.precision != JDE_FP32 && c.keep_layer_outputs != 1; }
// The first stage's residual block (layers 2 and 3) fused into one kernel whose 1x1 output (layer 2) is
// never stored and whose output (layer 3) goes to its own tensor: tensor-core handles with the default
// keep_layer_outputs = 0.
bool fused_res1_cfg(const jde_config& c) {
  return c.precision != JDE_FP32 && c.keep_layer_outputs == 0 && c.fuse_block1 != 0;
}

// Where each conv reads and writes (tensor ids below, -1 = none).
struct LayerIO {
  int in, out, res;
  int out_slice;   // channel offset inside `out` (concat slices)
  int upsample;
  int act;
  int head;        // output is a head tensor (f32, unpadded): 0..2 det, 3..5 emb, -1 otherwise
};

// Tensor ids: 0..77 = output of layer l, 78 = cat16, 79 = cat8, 80 = letterbox, 81..83 = copies of
// the embedding heads' input maps (strides 32, 16, 8) kept for the sparse embedding head of the
// post-processing (two sets, like the heads).
enum { T_CAT16 = 78, T_CAT8 = 79, T_LB = 80, T_PF = 81, T_COUNT = 84 };

struct TensorDesc {
  int h, w, c;     // unpadded size at the given input resolution (per frame)
  int pad;
  int dt;          // storage: 0 f32, 1 bf16, 2 E4M3 codes
  int alias;       // >= 0: lives inside tensor `alias` at channel offset `alias_off`
  int alias_off;
};

struct ResBuffers {
  int in_w = 0, in_h = 0;
  std::vector<TensorDesc> td;
  std::vector<void*> mem;          // owned allocations (per tensor id, null for aliases)
  std::vector<size_t> bytes;
  std::vector<size_t> set_bytes;   // head tensors hold two sets (double buffer); bytes of one set
};

struct Plan {
  int n = 0;
  std::vector<ConvSpec> specs;     // per layer
  std::vector<TcPlan> tc;          // per layer (BF16)
  std::shared_ptr<StemS2Plan> stem_s2;   // layers 0 and 1 fused (their tc plans unused)
  std::shared_ptr<Res1Plan> res1;        // layers 2 and 3 fused (their tc plans unused)
};

}  // namespace

struct jde_handle {
  jde_config cfg;
  std::string err;
  int* d_err = nullptr;
  std::vector<LayerW> w;
  std::vector<LayerIO> io;
  std::map<std::pair<int, int>, ResBuffers> res;
  std::map<std::tuple<int, int, int>, Plan> plans;
  ResBuffers* cur = nullptr;
  int cur_n = 0, cur_src_w = 0, cur_src_h = 0;
  // letterbox
  LbAxis* lb_x = nullptr;
  LbAxis* lb_y = nullptr;
  int lb_key[4] = {0, 0, 0, 0};
  uint8_t* frames_dev = nullptr;
  size_t frames_cap = 0;
  // post-processing
  PostBufs pb{};
  int pb_n = 0;
  float* rows_stage = nullptr;
  int32_t* count_stage = nullptr;
  int32_t* aidx_stage = nullptr;
  size_t rows_stage_cap = 0;
  TrackState trk{};
  cudaEvent_t prof[3] = {nullptr, nullptr, nullptr};
  int head_set = 0;   // head-tensor set the next forward writes
  int cur_set = 0;    // set written by the last forward
  size_t weight_bytes = 0;   // device bytes of the packed weights
  // E4M3 handles: scale of each stored tensor (per tensor id; concat buffers shared), set by
  // jde_set_act_amax
  std::vector<float> act_scale = std::vector<float>(T_COUNT, 1.0f);
  bool scales_set = false;
  float* d_amax = nullptr;   // jde_act_amax scratch [JDE_NUM_LAYERS]
  void* stem_pack = nullptr; // tensor-core handles: fused stem weights with bias parts, then layer 1's bias parts
  // jde_autotune: tile width per layer for (in_w, in_h, n); 0 = the default rule
  std::map<std::tuple<int, int, int>, std::vector<int>> tuned_bn;
};

namespace {

jde_status fail(jde_handle* h, jde_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (h)
    h->err = buf;
  else
    g_create_error = buf;
  return s;
}

#define CUDA_OR(h, call)                                                                        \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess) return fail((h), JDE_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

bool dmalloc(void** p, size_t bytes) {
  if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return false;
  }
  return true;
}

// ----------------------------------------------------------------------------- network wiring
// In-place residual stages: every block's 3x3 adds its output into the storage of the block's
// input (TMA reduce-add), so a stage's chain lives in one buffer.  Tensor-core handles whose
// stage outputs are stored in BF16 (all stages of a BF16 handle; the first stride-2 stage of an
// E4M3 handle), unless the handle keeps every layer output.
bool inplace_stage(const jde_config& cfg, int first_layer) {
  if (cfg.keep_layer_outputs || cfg.precision == JDE_FP32) return false;
  return cfg.precision == JDE_BF16 || first_layer < FP8_FIRST_OUT;
}

std::vector<LayerIO> build_io(const jde_config& cfg) {
  const auto& L = layers();
  std::vector<LayerIO> io(L.size());
  int l = 0;
  auto set = [&](int in, int res, int act) {
    io[l] = {in, l, res, 0, 0, act, -1};
    return l++;
  };
  int x = set(T_LB, -1, 1);  // stem (input: letterbox or its im2col rows)
  const int stage_n[5] = {1, 2, 8, 8, 4};
  int c3 = -1, c4 = -1;
  for (int s = 0; s < 5; ++s) {
    x = set(x, -1, 1);
    const bool chain = inplace_stage(cfg, x);
    // the skips of stages 3 and 4 end in a concat slice: an in-place chain lives there from its start
    if (chain && (s == 2 || s == 3)) {
      io[x].out = s == 2 ? T_CAT8 : T_CAT16;
      io[x].out_slice = s == 2 ? 128 : 256;
    }
    for (int b = 0; b < stage_n[s]; ++b) {
      const int r = x;
      const int t = set(x, -1, 1);
      x = set(t, r, 1);
      if (chain && !(s == 0 && fused_res1_cfg(cfg))) {   // the fused first block writes its own tensor
        io[x].out = io[r].out;               // the block output overwrites its input
        io[x].out_slice = io[r].out_slice;
      }
    }
    if (s == 2) c3 = x;
    if (s == 3) c4 = x;
  }
  // backbone skips live inside the concat buffers
  io[c3].out = T_CAT8;
  io[c3].out_slice = 128;
  io[c4].out = T_CAT16;
  io[c4].out_slice = 256;
  const int c5 = x;
  int in = c5;
  for (int h = 0; h < 3; ++h) {
    int f = in;
    for (int j = 0; j < 5; ++j) f = set(f, -1, 1);
    const int d3 = set(f, -1, 1);
    const int d1 = set(d3, -1, 0);
    io[d1].head = h;
    const int e = set(f, -1, 0);
    io[e].head = 3 + h;
    if (h < 2) {
      const int lat = set(f, -1, 1);
      io[lat].out = h == 0 ? T_CAT16 : T_CAT8;
      io[lat].out_slice = 0;
      io[lat].upsample = 1;
      in = h == 0 ? T_CAT16 : T_CAT8;
    }
  }
  return io;
}

// Resolve a tensor id to (storage id, channel offset); layer outputs may alias a concat slice.
void tensor_desc_table(const jde_handle* h, int in_w, int in_h, std::vector<TensorDesc>& td) {
  const auto& L = layers();
  td.assign(T_COUNT, TensorDesc{0, 0, 0, 1, 0, -1, 0});
  const bool bf16 = h->cfg.precision != JDE_FP32;   // tensor-core path (BF16 / E4M3)
  // spatial size of every layer output follows the input chain
  std::vector<int> oh(L.size()), ow(L.size());
  auto in_hw = [&](int tid, int& hh, int& ww) {
    if (tid == T_LB) {
      hh = in_h;
      ww = in_w;
    } else if (tid == T_CAT16) {
      hh = in_h / 16;
      ww = in_w / 16;
    } else if (tid == T_CAT8) {
      hh = in_h / 8;
      ww = in_w / 8;
    } else {
      hh = oh[tid];
      ww = ow[tid];
    }
  };
  for (size_t l = 0; l < L.size(); ++l) {
    int hh, ww;
    in_hw(h->io[l].in, hh, ww);
    oh[l] = (hh + 2 * (L[l].k / 2) - L[l].k) / L[l].stride + 1;
    ow[l] = (ww + 2 * (L[l].k / 2) - L[l].k) / L[l].stride + 1;
    const int prec = h->cfg.precision;
    const int dt = (prec == JDE_FP32 || h->io[l].head >= 0) ? 0
                   : (prec == JDE_FP8_E4M3 && (int)l >= FP8_FIRST_OUT) ? 2 : 1;
    TensorDesc d{oh[l], ow[l], L[l].cout, 1, dt, -1, 0};
    // heads are unpadded f32, except the tensor-core path's embedding maps, which keep the zero
    // halo so that their convs store whole flat tiles with TMA
    if (h->io[l].head >= 0) d.pad = (bf16 && h->io[l].head >= 3) ? 1 : 0;
    if (h->io[l].out != (int)l) {
      d.alias = h->io[l].out;
      d.alias_off = h->io[l].out_slice;
      if (h->io[l].upsample) {
        d.h *= 2;
        d.w *= 2;
      }
    }
    td[l] = d;
  }
  const int cat_dt = !bf16 ? 0 : (h->cfg.precision == JDE_FP8_E4M3 ? 2 : 1);
  td[T_CAT16] = TensorDesc{in_h / 16, in_w / 16, 768, 1, cat_dt, -1, 0};
  td[T_CAT8] = TensorDesc{in_h / 8, in_w / 8, 384, 1, cat_dt, -1, 0};
  td[T_LB] = TensorDesc{in_h, in_w, bf16 ? 4 : 3, 1, bf16 ? 1 : 0, -1, 0};
  // copies of the embedding heads' inputs (sparse head): same shape and storage type as the map
  for (size_t l = 0; l < L.size(); ++l)
    if (h->io[l].head >= 3) {
      const int src = h->io[l].in;
      td[T_PF + h->io[l].head - 3] = td[src];
      if (!sparse_emb_cfg(h->cfg)) td[T_PF + h->io[l].head - 3].alias = src;   // not kept
    }
}

// Storage of a tensor id in two sets (written by alternate forwards): the heads and, for the
// sparse embedding head, the copies of its input maps.
bool two_sets(const jde_handle* h, int t) {
  return (t < JDE_NUM_LAYERS && h->io[t].head >= 0) || (t >= T_PF && t < T_PF + 3);
}
// Tensor not allocated: the embedding heads when they are evaluated sparsely, the stem's output when
// it is fused into the next conv.
bool not_stored(const jde_handle* h, int t) {
  if (t == 0 && fused_stem_cfg(h->cfg)) return true;
  if (t == 2 && fused_res1_cfg(h->cfg)) return true;
  return t < JDE_NUM_LAYERS && t >= 0 && h->io[t].head >= 3 && sparse_emb_cfg(h->cfg);
}

size_t tensor_bytes(const TensorDesc& d, int n) {
  const size_t el = el_size(d.dt);
  return (size_t)n * (d.h + 2 * d.pad) * (d.w + 2 * d.pad) * d.c * el;
}

jde_status get_res(jde_handle* h, int in_w, int in_h, ResBuffers** out) {
  auto key = std::make_pair(in_w, in_h);
  auto it = h->res.find(key);
  if (it != h->res.end()) {
    *out = &it->second;
    return JDE_OK;
  }
  ResBuffers rb;
  rb.in_w = in_w;
  rb.in_h = in_h;
  tensor_desc_table(h, in_w, in_h, rb.td);
  rb.mem.assign(T_COUNT, nullptr);
  rb.bytes.assign(T_COUNT, 0);
  rb.set_bytes.assign(T_COUNT, 0);
  const int n = h->cfg.max_batch;
  const bool bf16 = h->cfg.precision != JDE_FP32;   // tensor-core path (BF16 / E4M3)
  for (int t = 0; t < T_COUNT; ++t) {
    if (rb.td[t].alias >= 0 || not_stored(h, t)) continue;
    rb.set_bytes[t] = tensor_bytes(rb.td[t], n);
    const size_t b = rb.set_bytes[t] * (two_sets(h, t) ? 2 : 1);
    if (!dmalloc(&rb.mem[t], b)) {
      for (void* p : rb.mem)
        if (p) cudaFree(p);
      return fail(h, JDE_ERR_OOM, "allocating %zu bytes for tensor %d at %dx%d", b, t, in_w, in_h);
    }
    rb.bytes[t] = b;
    // the zero halo is never written again
    if (cudaMemset(rb.mem[t], 0, b) != cudaSuccess) return fail(h, JDE_ERR_CUDA, "memset of activation buffer");
  }
  auto res = h->res.emplace(key, std::move(rb));
  *out = &res.first->second;
  return JDE_OK;
}

TView view_of(const ResBuffers& rb, int tid, int n) {
  const TensorDesc& d = rb.td[tid];
  TView v;
  if (d.alias >= 0) {
    const TensorDesc& p = rb.td[d.alias];
    const size_t el = el_size(p.dt);
    v.ptr = static_cast<char*>(rb.mem[d.alias]) + (size_t)d.alias_off * el;
    v.n = n;
    v.h = d.h;
    v.w = d.w;
    v.c = d.c;
    v.pad = p.pad;
    v.pixstride = p.c;
    v.dtype = p.dt;
  } else {
    v.ptr = rb.mem[tid];
    v.n = n;
    v.h = d.h;
    v.w = d.w;
    v.c = d.c;
    v.pad = d.pad;
    v.pixstride = d.c;
    v.dtype = d.dt;
  }
  if (tid == T_LB && d.c == 4) v.c = 3;   // bf16 letterbox stores RGB + one zero channel
  return v;
}

// True for a layer output that a later layer overwrites in place (the input of an in-place block).
bool overwritten(const jde_handle* h, int tid) {
  for (int l = tid + 1; l < JDE_NUM_LAYERS; ++l)
    if (h->io[l].res == tid && h->io[l].out == h->io[tid].out && h->io[l].out_slice == h->io[tid].out_slice &&
        h->io[l].out != l)
      return true;
  return false;
}

// Storage tensor of tensor id `tid` (a concat buffer for the layers writing into one).
int buffer_of(const jde_handle* h, int tid) {
  if (tid >= 0 && tid < JDE_NUM_LAYERS && h->io[tid].out != tid) return h->io[tid].out;
  return tid;
}

jde_status get_plan(jde_handle* h, ResBuffers* rb, int n, Plan** out) {
  auto key = std::make_tuple(rb->in_w, rb->in_h, n);
  auto it = h->plans.find(key);
  if (it != h->plans.end()) {
    *out = &it->second;
    return JDE_OK;
  }
  const auto& L = layers();
  Plan p;
  p.n = n;
  p.specs.resize(L.size());
  const bool bf16 = h->cfg.precision != JDE_FP32;   // tensor-core path (BF16 / E4M3)
  if (bf16) p.tc.resize(L.size());
  for (size_t l = 0; l < L.size(); ++l) {
    const LayerIO& io = h->io[l];
    if (not_stored(h, (int)l)) continue;   // sparse embedding head: evaluated in the post-processing
    ConvSpec c;
    memset(&c, 0, sizeof(c));
    c.k = L[l].k;
    c.stride = L[l].stride;
    c.cin = L[l].cin;
    c.cout = L[l].cout;
    c.in = view_of(*rb, io.in, n);
    c.out = view_of(*rb, (int)l, n);
    c.res.ptr = nullptr;
    if (io.res >= 0) c.res = view_of(*rb, io.res, n);
    c.Ho = rb->td[l].h / (io.upsample ? 2 : 1);
    c.Wo = rb->td[l].w / (io.upsample ? 2 : 1);
    c.act = io.act;
    c.upsample = io.upsample;
    c.bias = h->w[l].bias;
    c.err = h->d_err;
    c.q = h->w[l].q;
    c.mult = h->w[l].mult;
    if (c.res.ptr && c.res.dtype == 2) c.res_scale = h->act_scale[buffer_of(h, io.res)];
    if (c.out.dtype == 2) c.out_inv_scale = 1.0f / h->act_scale[buffer_of(h, (int)l)];
    p.specs[l] = c;
    if (bf16 && l == 1 && fused_stem_cfg(h->cfg)) continue;   // runs inside the fused stem kernel
    if (bf16 && l == 3 && fused_res1_cfg(h->cfg)) continue;   // runs inside the fused block kernel
    if (bf16) {
      char msg[256];
      const void* w = c.q ? static_cast<const void*>(h->w[l].w_q) : static_cast<const void*>(h->w[l].w_nk);
      int bn = h->w[l].bn;
      auto tb = h->tuned_bn.find(key);
      if (tb != h->tuned_bn.end() && tb->second[l] > 0) bn = tb->second[l];
      // tile code: output channels per tile, + 1 for two 128-row M sub-tiles per CTA (flat-window 3x3)
      if (!conv_tc_plan(p.tc[l], c, w, h->w[l].cout_pad_tc, bn & ~3, msg, sizeof(msg), (bn & 1) ? 2 : 1,
                        (bn & 2) ? 1 : 0))
        return fail(h, JDE_ERR_UNSUPPORTED, "layer %zu: %s", l, msg);
      p.tc[l].pdl = h->cfg.dependent_launch;
    }
  }
  if (bf16 && fused_stem_cfg(h->cfg)) {
    char msg[256];
    StemS2Plan* fp = stem_s2_plan_new(view_of(*rb, T_LB, n), view_of(*rb, 1, n), h->stem_pack, h->w[1].w_nk,
                                      static_cast<char*>(h->stem_pack) + 32 * 32 * 2, h->d_err, msg, sizeof(msg));
    if (!fp) return fail(h, JDE_ERR_UNSUPPORTED, "layers 0-1: %s", msg);
    p.stem_s2.reset(fp, stem_s2_plan_free);
  }
  if (bf16 && fused_res1_cfg(h->cfg)) {
    char msg[256];
    Res1Plan* rp = res1_plan_new(view_of(*rb, 1, n), view_of(*rb, 3, n), h->w[2].w_nk, h->w[3].w_nk, h->w[2].bias,
                                 h->w[3].bias, h->d_err, msg, sizeof(msg));
    if (!rp) return fail(h, JDE_ERR_UNSUPPORTED, "layers 2-3: %s", msg);
    p.res1.reset(rp, res1_plan_free);
  }
  auto res = h->plans.emplace(key, std::move(p));
  *out = &res.first->second;
  return JDE_OK;
}

// ----------------------------------------------------------------------------- weights
__global__ void pack_kernel(const float* W, const float* gamma, const float* beta, const float* mean,
                            const float* var, const float* bias_in, int cin, int cout, int k, int K, int kpad16,
                            int cp64, float* w_kn, int cptc, int ktc, __nv_bfloat16* w_nk, float* bias_out,
                            int bias_len) {
  // one thread per (k index, output channel) of the largest padded layout
  const int rows = kpad16 > ktc ? kpad16 : ktc;
  const int cols = cp64 > cptc ? cp64 : cptc;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)rows * cols) return;
  const int kk = (int)(idx / cols), co = (int)(idx % cols);
  double scale = 1.0;
  if (co < cout && gamma) scale = (double)gamma[co] / sqrt((double)var[co] + 1e-5);
  double v = 0.0;
  if (co < cout && kk < K) {
    const int tap = kk / cin, ci = kk % cin;
    const int ky = tap / k, kx = tap % k;
    v = (double)W[(((size_t)co * cin + ci) * k + ky) * k + kx] * scale;
  }
  if (w_kn && kk < kpad16 && co < cp64) w_kn[(size_t)kk * cp64 + co] = (float)v;
  // one rounding of the exact folded value (a float intermediate would round twice)
  if (w_nk && kk < ktc && co < cptc) w_nk[(size_t)co * ktc + kk] = __double2bfloat16(v);
  if (kk == 0 && co < bias_len) {
    double b = 0.0;
    if (co < cout) b = gamma ? (double)beta[co] - (double)mean[co] * scale : (double)bias_in[co];
    bias_out[co] = (float)b;
  }
}

// E4M3 layers: per output channel, scale = max |W'[co]| / 448 of the folded weights (1 for a zero channel).
__global__ void wscale_kernel(const float* W, const float* gamma, const float* var, int cin, int cout, int k,
                              double* wscale, int cptc) {
  const int co = blockIdx.x;
  __shared__ double red[256];
  double m = 0.0;
  if (co < cout) {
    const double scale = gamma ? (double)gamma[co] / sqrt((double)var[co] + 1e-5) : 1.0;
    const size_t nper = (size_t)cin * k * k;
    for (size_t i = threadIdx.x; i < nper; i += blockDim.x) m = fmax(m, fabs((double)W[co * nper + i] * scale));
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0 && co < cptc) wscale[co] = red[0] > 0.0 ? red[0] / 448.0 : 1.0;
}

// E4M3 code of a double, rounded once from the exact quotient (no float intermediate, whose own
// rounding can land on a midpoint of the 8-bit grid): binade 2^k (k >= -6; below that the
// subnormal spacing 2^-9), spacing 2^(k-3), nearest with ties to even, finite values saturate
// at 448; then the bit fields (sign, exponent k + 7, 3 mantissa bits; exponent 0 = subnormal).
__device__ uint8_t e4m3_code(double v) {
  if (v != v) return 0x7F;
  const uint8_t sign = v < 0.0 ? 0x80 : 0x00;
  const double a = fabs(v);
  int ex = 0;
  frexp(a, &ex);
  int k = a > 0.0 ? ex - 1 : -6;
  if (k < -6) k = -6;
  double r = rint(a / ldexp(1.0, k - 3)) * ldexp(1.0, k - 3);
  if (r > 448.0) r = 448.0;
  if (r == 0.0) return sign;
  frexp(r, &ex);
  const int kr = ex - 1;
  if (kr < -6) return sign | (uint8_t)rint(r / ldexp(1.0, -9));
  return sign | (uint8_t)((kr + 7) << 3) | (uint8_t)((int)rint(r / ldexp(1.0, kr - 3)) - 8);
}

// E4M3 layers: w_q[co][kk] = E4M3(W'[co][kk] / wscale[co]), K index = tap * cin + ci.
__global__ void pack_q_kernel(const float* W, const float* gamma, const float* var, int cin, int cout, int k,
                              const double* wscale, uint8_t* w_q, int cptc, int ktc) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)cptc * ktc) return;
  const int co = (int)(idx / ktc), kk = (int)(idx % ktc);
  double v = 0.0;
  const int K = cin * k * k;
  if (co < cout && kk < K) {
    const double scale = gamma ? (double)gamma[co] / sqrt((double)var[co] + 1e-5) : 1.0;
    const int tap = kk / cin, ci = kk % cin;
    const double w = (double)W[(((size_t)co * cin + ci) * k + tap / k) * k + tap % k] * scale;
    v = w / wscale[co];
  }
  w_q[idx] = e4m3_code(v);
}

// Device bytes of one layer's packed weights (bias + tensor-core or SIMT layout).
size_t layer_weight_bytes(const LayerDef& L, int precision, int l) {
  const bool bf16 = precision != JDE_FP32;
  const int K = L.k * L.k * L.cin;
  const int cout_pad64 = align_up(L.cout, 64);
  const int bn = conv_tc_pick_bn(L.cout);
  const int cout_pad_tc = align_up(L.cout, bn);
  const int k_tc = l == 0 ? 32 : (L.cin == 32 && L.k == 3 ? 320 : K);
  const int bias_len = (cout_pad64 > cout_pad_tc ? cout_pad64 : cout_pad_tc) + 256;
  size_t b = sizeof(float) * (size_t)bias_len;
  if (is_q_layer(precision, l))
    b += (size_t)cout_pad_tc * k_tc + (sizeof(double) + sizeof(float)) * (size_t)cout_pad_tc;
  else
    b += bf16 ? sizeof(__nv_bfloat16) * (size_t)cout_pad_tc * k_tc : sizeof(float) * (size_t)align_up(K, 16) * cout_pad64;
  return b;
}

// Device bytes of the post-processing scratch for n frames.
size_t post_bytes(int n, int anchors, int kmax) {
  const size_t N = (size_t)n, K = (size_t)kmax;
  return N * anchors * sizeof(uint64_t) + N * sizeof(int) + N * K * sizeof(uint64_t) + N * sizeof(int) +
         N * K * sizeof(float4) + 2 * N * K * sizeof(float) + N * K * (K / 64) * sizeof(unsigned long long) +
         N * K * sizeof(int) + N * sizeof(int) + 3 * N * K * sizeof(int4) + 3 * sizeof(int);
}

int anchors_for(int in_w, int in_h) {
  return 4 * ((in_w / 32) * (in_h / 32) + (in_w / 16) * (in_h / 16) + (in_w / 8) * (in_h / 8));
}

jde_status load_weights(jde_handle* h, const void* blob, size_t nbytes) {
  const auto& L = layers();
  const uint8_t* p = static_cast<const uint8_t*>(blob);
  if (!blob || nbytes < 16 || memcmp(p, "JDEW", 4) != 0) return fail(h, JDE_ERR_WEIGHTS, "bad weights magic");
  uint32_t hdr[3];
  memcpy(hdr, p + 4, 12);
  if (hdr[0] != 1) return fail(h, JDE_ERR_WEIGHTS, "weights version %u != 1", hdr[0]);
  if (hdr[1] != L.size()) return fail(h, JDE_ERR_WEIGHTS, "weights have %u layers, expected %zu", hdr[1], L.size());
  std::vector<size_t> offs(L.size());
  size_t off = 16;
  for (size_t l = 0; l < L.size(); ++l) {
    if (off + 32 > nbytes) return fail(h, JDE_ERR_WEIGHTS, "weights truncated at layer %zu", l);
    uint32_t lh[8];
    memcpy(lh, p + off, 32);
    const uint32_t want_flags = L[l].has_bn ? 1u : 2u;
    if ((int)lh[0] != L[l].cin || (int)lh[1] != L[l].cout || (int)lh[2] != L[l].k || (int)lh[3] != L[l].stride ||
        lh[4] != want_flags)
      return fail(h, JDE_ERR_WEIGHTS, "layer %zu header (%u,%u,%u,%u,%u) does not match the layer table", l, lh[0],
                  lh[1], lh[2], lh[3], lh[4]);
    offs[l] = off + 32;
    off += 32 + 4ull * L[l].cout * L[l].cin * L[l].k * L[l].k + 4ull * L[l].cout * (L[l].has_bn ? 4 : 1);
    if (off > nbytes) return fail(h, JDE_ERR_WEIGHTS, "weights truncated in layer %zu", l);
  }
  if (off != nbytes) return fail(h, JDE_ERR_WEIGHTS, "weights blob has %zu trailing bytes", nbytes - off);
  void* dblob = nullptr;
  if (!dmalloc(&dblob, nbytes)) return fail(h, JDE_ERR_OOM, "weights staging (%zu bytes)", nbytes);
  CUDA_OR(h, cudaMemcpy(dblob, blob, nbytes, cudaMemcpyHostToDevice));
  const bool bf16 = h->cfg.precision != JDE_FP32;   // tensor-core path (BF16 / E4M3)
  h->w.resize(L.size());
  for (size_t l = 0; l < L.size(); ++l) {
    LayerW& lw = h->w[l];
    const int K = L[l].k * L[l].k * L[l].cin;
    const int kpad16 = align_up(K, 16);
    lw.cout_pad64 = align_up(L[l].cout, 64);
    lw.bn = conv_tc_pick_bn(L[l].cout);
    lw.cout_pad_tc = align_up(L[l].cout, lw.bn);
    // stem: 27 taps x channels padded to 32; 32-channel 3x3: 9 taps padded to 10 (two taps per K=64 block)
    lw.k_tc = l == 0 ? 32 : (L[l].cin == 32 && L[l].k == 3 ? 320 : K);
    const int bias_len = (lw.cout_pad64 > lw.cout_pad_tc ? lw.cout_pad64 : lw.cout_pad_tc) + 256;
    bool ok = dmalloc((void**)&lw.bias, sizeof(float) * bias_len);
    lw.q = is_q_layer(h->cfg.precision, (int)l) ? 1 : 0;
    if (lw.q)
      ok = ok && dmalloc((void**)&lw.w_q, (size_t)lw.cout_pad_tc * lw.k_tc) &&
           dmalloc((void**)&lw.wscale, sizeof(double) * lw.cout_pad_tc) &&
           dmalloc((void**)&lw.mult, sizeof(float) * lw.cout_pad_tc);
    else if (bf16)
      ok = ok && dmalloc((void**)&lw.w_nk, sizeof(__nv_bfloat16) * (size_t)lw.cout_pad_tc * lw.k_tc);
    else
      ok = ok && dmalloc((void**)&lw.w_kn, sizeof(float) * (size_t)kpad16 * lw.cout_pad64);
    if (!ok) {
      cudaFree(dblob);
      return fail(h, JDE_ERR_OOM, "weights of layer %zu", l);
    }
    cudaMemset(lw.bias, 0, sizeof(float) * bias_len);
    h->weight_bytes += layer_weight_bytes(L[l], h->cfg.precision, (int)l);
    const float* base = reinterpret_cast<const float*>(static_cast<uint8_t*>(dblob) + offs[l]);
    const size_t nw = (size_t)L[l].cout * L[l].cin * L[l].k * L[l].k;
    const float* W = base;
    const float *gamma = nullptr, *beta = nullptr, *mean = nullptr, *var = nullptr, *bias = nullptr;
    if (L[l].has_bn) {
      gamma = W + nw;
      beta = gamma + L[l].cout;
      mean = beta + L[l].cout;
      var = mean + L[l].cout;
    } else {
      bias = W + nw;
    }
    const int rows = bf16 ? lw.k_tc : kpad16;
    const int cols = bf16 ? lw.cout_pad_tc : lw.cout_pad64;
    const long long total = (long long)rows * cols;
    jde_count_launch();
    pack_kernel<<<(unsigned)((total + 255) / 256), 256>>>(
        W, gamma, beta, mean, var, bias, L[l].cin, L[l].cout, L[l].k, K, bf16 ? 0 : kpad16, bf16 ? 0 : lw.cout_pad64,
        lw.w_kn, bf16 ? lw.cout_pad_tc : 0, bf16 ? lw.k_tc : 0, lw.w_nk, lw.bias, bias_len);   // E4M3 layers:
                                                                                           // bias only (w_nk NULL)
    if (lw.q) {
      jde_count_launch(2);
      wscale_kernel<<<lw.cout_pad_tc, 256>>>(W, gamma, var, L[l].cin, L[l].cout, L[l].k, lw.wscale, lw.cout_pad_tc);
      const long long nq = (long long)lw.cout_pad_tc * lw.k_tc;
      pack_q_kernel<<<(unsigned)((nq + 255) / 256), 256>>>(W, gamma, var, L[l].cin, L[l].cout, L[l].k, lw.wscale,
                                                            lw.w_q, lw.cout_pad_tc, lw.k_tc);
      lw.wscale_host.resize(lw.cout_pad_tc);
      CUDA_OR(h, cudaMemcpy(lw.wscale_host.data(), lw.wscale, sizeof(double) * lw.cout_pad_tc, cudaMemcpyDeviceToHost));
    }
  }
  if (bf16) {
    // the fused stem kernel's weights: the stem's with its bias parts, and layer 1's bias parts
    if (!dmalloc(&h->stem_pack, STEM_S2_PACK_BYTES)) {
      cudaFree(dblob);
      return fail(h, JDE_ERR_OOM, "fused stem weights");
    }
    h->weight_bytes += STEM_S2_PACK_BYTES;
    if (stem_s2_pack(h->w[0].w_nk, h->w[0].bias, h->w[1].bias, h->stem_pack,
                     static_cast<char*>(h->stem_pack) + 32 * 32 * 2, 0) != cudaSuccess) {
      cudaFree(dblob);
      return fail(h, JDE_ERR_CUDA, "packing the fused stem weights");
    }
  }
  cudaError_t e = cudaDeviceSynchronize();
  cudaFree(dblob);
  if (e != cudaSuccess) return fail(h, JDE_ERR_CUDA, "packing weights: %s", cudaGetErrorString(e));
  return JDE_OK;
}

// ----------------------------------------------------------------------------- helpers
void geometry(int src_w, int src_h, int in_w, int in_h, double& r, int& nw, int& nh, int& px, int& py) {
  r = fmin((double)in_w / src_w, (double)in_h / src_h);
  nw = (int)floor(src_w * r + 0.5);
  nh = (int)floor(src_h * r + 0.5);
  px = (in_w - nw) / 2;
  py = (in_h - nh) / 2;
}

// The post-processing scratch is allocated once, for max_batch frames, at the first call: it never moves
// afterwards, so a CUDA graph that captured a post-processing launch stays valid for any later batch size.
jde_status ensure_post(jde_handle* h, int n) {
  if (h->pb_n >= n && h->pb.cand_keys) return JDE_OK;
  n = h->cfg.max_batch;
  PostBufs& b = h->pb;
  void* ptrs[] = {b.cand_keys, b.cand_count, b.sorted, b.n_sorted, b.boxes, b.conf, b.cls, b.mask, b.keep_idx,
                  b.n_keep, b.emb_list, b.emb_count};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  const int kmax = h->cfg.max_cand;
  const int anchors = anchors_for(h->cfg.max_in_w, h->cfg.max_in_h);
  b.cand_cap = anchors;
  b.kmax = kmax;
  bool ok = dmalloc((void**)&b.cand_keys, sizeof(uint64_t) * (size_t)n * anchors) &&
            dmalloc((void**)&b.cand_count, sizeof(int) * n) &&
            dmalloc((void**)&b.sorted, sizeof(uint64_t) * (size_t)n * kmax) &&
            dmalloc((void**)&b.n_sorted, sizeof(int) * n) && dmalloc((void**)&b.boxes, sizeof(float4) * (size_t)n * kmax) &&
            dmalloc((void**)&b.conf, sizeof(float) * (size_t)n * kmax) &&
            dmalloc((void**)&b.cls, sizeof(float) * (size_t)n * kmax) &&
            dmalloc((void**)&b.mask, sizeof(unsigned long long) * (size_t)n * kmax * (kmax / 64)) &&
            dmalloc((void**)&b.keep_idx, sizeof(int) * (size_t)n * kmax) && dmalloc((void**)&b.n_keep, sizeof(int) * n) &&
            dmalloc((void**)&b.emb_list, sizeof(int4) * 3 * (size_t)n * kmax) &&
            dmalloc((void**)&b.emb_count, sizeof(int) * 3);
  if (!ok) return fail(h, JDE_ERR_OOM, "post-processing buffers for %d frames", n);
  h->pb_n = n;
  return JDE_OK;
}

__global__ void gather_view_kernel(TView v, void* dst, int el) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)v.n * v.h * v.w * v.c;
  if (idx >= total) return;
  const int c = (int)(idx % v.c);
  long long p = idx / v.c;
  const int x = (int)(p % v.w);
  p /= v.w;
  const int y = (int)(p % v.h);
  const int n = (int)(p / v.h);
  const size_t o = tview_off(v, n, y, x) + c;
  if (el == 4)
    static_cast<float*>(dst)[idx] = static_cast<const float*>(v.ptr)[o];
  else if (el == 2)
    static_cast<__nv_bfloat16*>(dst)[idx] = static_cast<const __nv_bfloat16*>(v.ptr)[o];
  else
    static_cast<uint8_t*>(dst)[idx] = static_cast<const uint8_t*>(v.ptr)[o];
}

// max |value| of a tensor view (E4M3 codes times `scale`), folded into *out with an integer max
// (non-negative floats order like their bit patterns).
__global__ void amax_kernel(TView v, float scale, float* out) {
  const long long total = (long long)v.n * v.h * v.w * v.c;
  float m = 0.f;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(idx % v.c);
    long long p = idx / v.c;
    const int x = (int)(p % v.w);
    p /= v.w;
    const int y = (int)(p % v.h);
    const int n = (int)(p / v.h);
    const size_t o = tview_off(v, n, y, x) + c;
    float a;
    if (v.dtype == 0)
      a = static_cast<const float*>(v.ptr)[o];
    else if (v.dtype == 1)
      a = __bfloat162float(static_cast<const __nv_bfloat16*>(v.ptr)[o]);
    else
      a = e4m3x2_to_float2(static_cast<const uint8_t*>(v.ptr)[o]).x * scale;
    m = fmaxf(m, fabsf(a));
  }
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int*>(out), __float_as_int(m));
}

// Self-test of the bounded waits: one thread waits on phase 0 of a fresh mbarrier, which nothing
// completes, with the given cycle limit; the wait gives up and the error word gets the timeout bit.
__global__ void wait_selftest_kernel(int* err, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0u, limit)) flag_error(err, KERR_TIMEOUT);
}

}  // namespace

// ============================================================================= C ABI
extern "C" {

void jde_default_config(jde_config* c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->precision = JDE_BF16;
  c->max_batch = 16;
  c->max_in_w = 1088;
  c->max_in_h = 608;
  c->max_src_w = 1920;
  c->max_src_h = 1080;
  c->max_cand = 4096;
  c->conf_thresh = 0.5f;
  c->nms_iou = 0.4f;
  c->assign_thresh = 0.7f;
  c->gate_chi2 = 9.487729036781154;
  c->lost_max_frames = 30;
  c->emb_momentum = 0.9f;
  c->max_streams = 64;
  c->max_tracks = 1024;
  c->max_track_dets = 1024;
  c->device = 0;
  c->sparse_emb = 1;
  c->assoc_cascade = 0;
  c->motion_lambda = 0.98;
  c->iou_cost2 = 0.5;
  c->iou_cost3 = 0.3;
  c->fuse_block1 = 0;
  c->dependent_launch = 1;
}

int jde_layer_table(jde_layer_desc* out, int cap) {
  const auto& L = layers();
  for (int i = 0; i < (int)L.size() && i < cap && out; ++i)
    out[i] = jde_layer_desc{L[i].cin, L[i].cout, L[i].k, L[i].stride, L[i].has_bn, L[i].res_nb};
  return (int)L.size();
}

const char* jde_last_error(jde_handle* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

void jde_destroy(jde_handle* h) {
  if (!h) return;
  cudaSetDevice(h->cfg.device);
  cudaDeviceSynchronize();
  for (auto& lw : h->w) {
    cudaFree(lw.w_kn);
    cudaFree(lw.w_nk);
    cudaFree(lw.w_q);
    cudaFree(lw.wscale);
    cudaFree(lw.mult);
    cudaFree(lw.bias);
  }
  cudaFree(h->d_amax);
  cudaFree(h->stem_pack);
  for (auto& kv : h->res)
    for (void* p : kv.second.mem)
      if (p) cudaFree(p);
  PostBufs& b = h->pb;
  void* ptrs[] = {b.cand_keys, b.cand_count, b.sorted, b.n_sorted, b.boxes, b.conf, b.cls, b.mask, b.keep_idx,
                  b.n_keep, b.emb_list, b.emb_count, h->lb_x, h->lb_y, h->frames_dev, h->rows_stage,
                  h->count_stage, h->aidx_stage, h->d_err};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  track_free(h->trk);
  delete h;
}

jde_status jde_create(const jde_config* cfg, const void* weights, size_t nbytes, jde_handle** out) {
  if (!out) return fail(nullptr, JDE_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!cfg) return fail(nullptr, JDE_ERR_INVALID_ARG, "cfg is NULL");
  const jde_config& c = *cfg;
  if (c.precision != JDE_FP32 && c.precision != JDE_BF16 && c.precision != JDE_FP8_E4M3)
    return fail(nullptr, JDE_ERR_UNSUPPORTED, "precision %d not supported", c.precision);
  if (c.max_batch < 1 || c.max_in_w < 32 || c.max_in_h < 32 || c.max_in_w % 32 || c.max_in_h % 32 ||
      c.max_src_w < 1 || c.max_src_h < 1 || c.max_cand < 64 || c.max_cand > 4096 || c.max_cand % 64 ||
      c.max_streams < 1 || c.max_tracks < 1 || c.max_track_dets < 1 || c.max_track_dets > 4096 ||
      c.max_tracks > 4096 || c.keep_layer_outputs < 0 || c.keep_layer_outputs > 2 || c.assoc_cascade < 0 ||
      c.assoc_cascade > 1 || !(c.motion_lambda >= 0.0 && c.motion_lambda <= 1.0) || !(c.iou_cost2 >= 0.0) ||
      !(c.iou_cost3 >= 0.0) || c.fuse_block1 < 0 || c.fuse_block1 > 1 || c.dependent_launch < 0 ||
      c.dependent_launch > 1)
    return fail(nullptr, JDE_ERR_INVALID_ARG, "config out of range");
  if (cudaSetDevice(c.device) != cudaSuccess) return fail(nullptr, JDE_ERR_CUDA, "cudaSetDevice(%d)", c.device);
  jde_handle* h = new jde_handle();
  h->cfg = c;
  h->io = build_io(h->cfg);
  jde_status s = JDE_OK;
  if (!dmalloc((void**)&h->d_err, sizeof(int))) s = fail(h, JDE_ERR_OOM, "error word");
  if (s == JDE_OK) cudaMemset(h->d_err, 0, sizeof(int));
  if (s == JDE_OK) s = load_weights(h, weights, nbytes);
  if (s == JDE_OK && !(dmalloc((void**)&h->lb_x, sizeof(LbAxis) * c.max_in_w) &&
                       dmalloc((void**)&h->lb_y, sizeof(LbAxis) * c.max_in_h)))
    s = fail(h, JDE_ERR_OOM, "letterbox tables");
  if (s == JDE_OK && track_alloc(h->trk, c) != 0) s = fail(h, JDE_ERR_OOM, "tracker state");
  if (s == JDE_OK) {
    // the scratch array of jde_postprocess_noalloc is loaded onto this device now, with the handle's
    // other device memory, rather than by that entry point's first call
    char msg[200] = {0};
    if (noalloc_scratch_setup(msg, sizeof(msg)) != 0) s = fail(h, JDE_ERR_CUDA, "no-alloc scratch set-up: %s", msg);
  }
  if (s != JDE_OK) {
    g_create_error = h->err;
    jde_destroy(h);
    return s;
  }
  *out = h;
  return JDE_OK;
}

jde_status jde_forward(jde_handle* h, const uint8_t* frames, int n, int src_w, int src_h, int in_w, int in_h,
                       int on_device, void* stream) {
  if (!h) return fail(nullptr, JDE_ERR_INVALID_ARG, "handle is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!frames || n < 1 || n > h->cfg.max_batch || in_w % 32 || in_h % 32 || in_w < 32 || in_h < 32 ||
      in_w > h->cfg.max_in_w || in_h > h->cfg.max_in_h || src_w < 1 || src_h < 1)
    return fail(h, JDE_ERR_INVALID_ARG, "jde_forward: bad arguments (n=%d in=%dx%d src=%dx%d)", n, in_w, in_h, src_w,
                src_h);
  if (h->cfg.precision == JDE_FP8_E4M3 && !h->scales_set)
    return fail(h, JDE_ERR_INVALID_ARG, "jde_forward: E4M3 handle has no activation scales (call jde_set_act_amax)");
  const size_t fbytes = (size_t)n * src_w * src_h * 3;
  if (!on_device) {
    if (fbytes > h->frames_cap) {
      cudaFree(h->frames_dev);
      h->frames_dev = nullptr;
      if (!dmalloc((void**)&h->frames_dev, fbytes)) return fail(h, JDE_ERR_OOM, "frame staging");
      h->frames_cap = fbytes;
    }
    CUDA_OR(h, cudaMemcpyAsync(h->frames_dev, frames, fbytes, cudaMemcpyHostToDevice, st));
    frames = h->frames_dev;
  }
  ResBuffers* rb;
  jde_status s = get_res(h, in_w, in_h, &rb);
  if (s != JDE_OK) return s;
  Plan* plan;
  s = get_plan(h, rb, n, &plan);
  if (s != JDE_OK) return s;
  const int key[4] = {src_w, src_h, in_w, in_h};
  if (memcmp(key, h->lb_key, sizeof(key)) != 0) {
    double r;
    int nw, nh, px, py;
    geometry(src_w, src_h, in_w, in_h, r, nw, nh, px, py);
    letterbox_tables_launch(h->lb_x, h->lb_y, src_w, src_h, in_w, in_h, r, nw, nh, px, py, st);
    memcpy(h->lb_key, key, sizeof(key));
  }
  const TView lb = view_of(*rb, T_LB, n);
  const bool bf16 = h->cfg.precision != JDE_FP32;   // tensor-core path (BF16 / E4M3)
  if (h->prof[0]) cudaEventRecord(h->prof[0], st);
  if (bf16) {
    letterbox_bf16x4_launch(frames, n, src_w, src_h, h->lb_x, h->lb_y, lb, st);
  } else {
    letterbox_f32_launch(frames, n, src_w, src_h, h->lb_x, h->lb_y, lb, st);
  }
  const auto& L = layers();
  // head tensors are double-buffered: this forward writes set head_set
  const int set = h->head_set;
  for (size_t l = 0; l < L.size(); ++l) {
    if (h->io[l].head < 0 || not_stored(h, (int)l)) continue;
    void* p = static_cast<char*>(rb->mem[l]) + (size_t)set * rb->set_bytes[l];
    plan->specs[l].out.ptr = p;
    if (bf16 && !conv_tc_retarget(plan->tc[l], p))
      return fail(h, JDE_ERR_CUDA, "layer %zu: output tensor map for head set %d", l, set);
  }
  if (h->prof[1]) cudaEventRecord(h->prof[1], st);
  for (size_t l = 0; l < L.size(); ++l) {
    if (not_stored(h, (int)l)) continue;
    if (bf16) {
      const cudaError_t e = (l == 1 && plan->stem_s2) ? stem_s2_launch(plan->stem_s2.get(), st)
                            : (l == 3 && plan->res1) ? res1_launch(plan->res1.get(), st)
                                                      : conv_tc_launch(plan->tc[l], st);
      if (e != cudaSuccess) return fail(h, JDE_ERR_CUDA, "conv layer %zu: %s", l, cudaGetErrorString(e));
    } else {
      conv_simt_launch(plan->specs[l], h->w[l].w_kn, h->w[l].cout_pad64, st);
    }
  }
  // sparse embedding head: keep this forward's head inputs for its post-processing (set `set`)
  for (int s = 0; s < 3; ++s) {
    const int t = T_PF + s;
    if (!rb->mem[t]) continue;
    int src = -1;
    for (size_t l = 0; l < L.size(); ++l)
      if (h->io[l].head == 3 + s) src = h->io[l].in;
    const size_t bytes = tensor_bytes(rb->td[src], n);
    CUDA_OR(h, cudaMemcpyAsync(static_cast<char*>(rb->mem[t]) + (size_t)set * rb->set_bytes[t], rb->mem[src], bytes,
                               cudaMemcpyDeviceToDevice, st));
  }
  if (h->prof[2]) cudaEventRecord(h->prof[2], st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(h, JDE_ERR_CUDA, "forward launch: %s", cudaGetErrorString(e));
  h->cur = rb;
  h->cur_n = n;
  h->cur_src_w = src_w;
  h->cur_src_h = src_h;
  h->cur_set = set;
  h->head_set = set ^ 1;
  return JDE_OK;
}

jde_status jde_postprocess(jde_handle* h, const float* const* heads, int n, int in_w, int in_h, int src_w, int src_h,
                           jde_dets* out, void* stream) {
  if (!h) return fail(nullptr, JDE_ERR_INVALID_ARG, "handle is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!out || !out->rows || !out->count || out->cap < 1 || n < 1 || n > h->cfg.max_batch || in_w % 32 ||
      in_h % 32 || in_w > h->cfg.max_in_w || in_h > h->cfg.max_in_h || in_w < 32 || in_h < 32 || src_w < 1 ||
      src_h < 1)
    return fail(h, JDE_ERR_INVALID_ARG, "jde_postprocess: bad arguments");
  const float* hp[6];
  if (heads) {
    for (int i = 0; i < 6; ++i) {
      if (!heads[i]) return fail(h, JDE_ERR_INVALID_ARG, "jde_postprocess: head %d is NULL", i);
      hp[i] = heads[i];
    }
  } else {
    if (!h->cur || h->cur->in_w != in_w || h->cur->in_h != in_h || h->cur_n < n)
      return fail(h, JDE_ERR_INVALID_ARG, "jde_postprocess: no forward result at %dx%d for %d frames", in_w, in_h, n);
    const auto& L = layers();
    for (size_t l = 0; l < L.size(); ++l)
      if (h->io[l].head >= 0)
        hp[h->io[l].head] = reinterpret_cast<const float*>(static_cast<const char*>(h->cur->mem[l]) +
                                                            (size_t)h->cur_set * h->cur->set_bytes[l]);
  }
  jde_status s = ensure_post(h, n);
  if (s != JDE_OK) return s;
  HeadGeom g;
  memset(&g, 0, sizeof(g));
  g.n = n;
  if (!heads)   // the handle's own embedding maps (padded on the tensor-core path)
    for (size_t l = 0; l < layers().size(); ++l)
      if (h->io[l].head == 3) g.epad = h->cur->td[l].pad;
  const int strides[3] = {32, 16, 8};
  const float base[3] = {128.f, 32.f, 8.f};
  g.off[0] = 0;
  for (int i = 0; i < 3; ++i) {
    g.stride[i] = strides[i];
    g.gh[i] = in_h / strides[i];
    g.gw[i] = in_w / strides[i];
    g.off[i + 1] = g.off[i] + 4 * g.gh[i] * g.gw[i];
    for (int a = 0; a < 4; ++a) {
      const double w = base[i] * pow(sqrt(2.0), a);
      g.anchor_w[i * 4 + a] = (float)w;
      g.anchor_h[i * 4 + a] = (float)(3.0 * w);
    }
  }
  double r;
  int nw, nh, px, py;
  geometry(src_w, src_h, in_w, in_h, r, nw, nh, px, py);
  g.ratio = (float)r;
  g.pad_x = (float)px;
  g.pad_y = (float)py;
  float* rows = out->rows;
  int32_t* count = out->count;
  int32_t* aidx = out->anchor_index;
  const size_t need = (size_t)n * out->cap;
  if (!out->on_device) {
    if (need > h->rows_stage_cap) {
      cudaFree(h->rows_stage);
      cudaFree(h->count_stage);
      cudaFree(h->aidx_stage);
      h->rows_stage = nullptr;
      h->count_stage = nullptr;
      h->aidx_stage = nullptr;
      if (!(dmalloc((void**)&h->rows_stage, sizeof(float) * 518 * need) &&
            dmalloc((void**)&h->count_stage, sizeof(int32_t) * h->cfg.max_batch) &&
            dmalloc((void**)&h->aidx_stage, sizeof(int32_t) * need)))
        return fail(h, JDE_ERR_OOM, "detection staging");
      h->rows_stage_cap = need;
    }
    rows = h->rows_stage;
    count = h->count_stage;
    aidx = out->anchor_index ? h->aidx_stage : nullptr;
  }
  // the handle's own forward with a sparse embedding head: its input maps of the last forward
  EmbSparse es;
  memset(&es, 0, sizeof(es));
  const bool sparse = !heads && sparse_emb_cfg(h->cfg);
  if (sparse) {
    const auto& L = layers();
    for (size_t l = 0; l < L.size(); ++l) {
      const int hd = h->io[l].head;
      if (hd < 3) continue;
      const int s = hd - 3, t = T_PF + s;
      TView v = view_of(*h->cur, h->io[l].in, n);
      v.ptr = static_cast<char*>(h->cur->mem[t]) + (size_t)h->cur_set * h->cur->set_bytes[t];
      const LayerW& lw = h->w[l];
      es.in[s] = v;
      es.w[s] = lw.q ? static_cast<const void*>(lw.w_q) : static_cast<const void*>(lw.w_nk);
      es.bias[s] = lw.bias;
      es.mult[s] = lw.q ? lw.mult : nullptr;
      es.cin[s] = L[l].cin;
      es.ldw[s] = lw.k_tc;
      es.q[s] = lw.q;
    }
  }
  cudaError_t e = post_launch(hp, g, h->cfg.conf_thresh, h->cfg.nms_iou, h->pb, rows, count, aidx, out->cap,
                              h->d_err, st, sparse ? &es : nullptr);
  if (e != cudaSuccess) return fail(h, JDE_ERR_CUDA, "post-processing launch: %s", cudaGetErrorString(e));
  if (!out->on_device) {
    CUDA_OR(h, cudaMemcpyAsync(out->count, count, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
    CUDA_OR(h, cudaStreamSynchronize(st));
    int maxc = 0;
    for (int i = 0; i < n; ++i) maxc = out->count[i] > maxc ? out->count[i] : maxc;
    const int rows_copy = maxc < out->cap ? maxc : out->cap;
    for (int i = 0; i < n && rows_copy > 0; ++i) {
      const int ci = out->count[i] < out->cap ? out->count[i] : out->cap;
      if (ci <= 0) continue;
      CUDA_OR(h, cudaMemcpyAsync(out->rows + (size_t)i * out->cap * 518, rows + (size_t)i * out->cap * 518,
                                 sizeof(float) * 518 * ci, cudaMemcpyDeviceToHost, st));
      if (out->anchor_index)
        CUDA_OR(h, cudaMemcpyAsync(out->anchor_index + (size_t)i * out->cap, aidx + (size_t)i * out->cap,
                                   sizeof(int32_t) * ci, cudaMemcpyDeviceToHost, st));
    }
    CUDA_OR(h, cudaStreamSynchronize(st));
    if (maxc > out->cap) return fail(h, JDE_ERR_CAPACITY, "a frame kept %d detections, cap is %d", maxc, out->cap);
  }
  return JDE_OK;
}

jde_status jde_detect_batch(jde_handle* h, const uint8_t* frames, int n, int src_w, int src_h, int in_w, int in_h,
                            int on_device, jde_dets* out, void* stream) {
  jde_status s = jde_forward(h, frames, n, src_w, src_h, in_w, in_h, on_device, stream);
  if (s != JDE_OK) return s;
  return jde_postprocess(h, nullptr, n, in_w, in_h, src_w, src_h, out, stream);
}

jde_status jde_get_tensor(jde_handle* h, int id, void* dst, size_t dst_bytes, int* dims, int* dtype, void* stream) {
  if (!h) return fail(nullptr, JDE_ERR_INVALID_ARG, "handle is NULL");
  if (!h->cur) return fail(h, JDE_ERR_NOT_FOUND, "no forward has run");
  int tid;
  if (id >= 0 && id < JDE_NUM_LAYERS && not_stored(h, id))
    return fail(h, JDE_ERR_NOT_FOUND,
                id == 0   ? "tensor 0: the stem's output stays on chip, fused into layer 1 (keep_layer_outputs = 1 keeps it)"
                : id == 2 ? "tensor 2: the first residual block's 1x1 output stays on chip, fused into layer 3 "
                            "(keep_layer_outputs = 1 or 2 keeps it)"
                          : "tensor %d: the embedding head runs only at kept detections (sparse_emb)",
                id);
  if (id >= 0 && id < JDE_NUM_LAYERS && overwritten(h, id))
    return fail(h, JDE_ERR_NOT_FOUND, "tensor %d is overwritten in place by its residual block (keep_layer_outputs)", id);
  if (id >= 0 && id < JDE_NUM_LAYERS)
    tid = id;
  else if (id == 100)
    tid = T_LB;
  else
    return fail(h, JDE_ERR_NOT_FOUND, "unknown tensor id %d", id);
  TView v = view_of(*h->cur, tid, h->cur_n);
  if (tid < JDE_NUM_LAYERS && h->io[tid].head >= 0)
    v.ptr = static_cast<char*>(v.ptr) + (size_t)h->cur_set * h->cur->set_bytes[tid];
  if (dims) {
    dims[0] = v.n;
    dims[1] = v.h;
    dims[2] = v.w;
    dims[3] = v.c;
  }
  if (dtype) *dtype = v.dtype;
  if (!dst) return JDE_OK;
  const int el = el_size(v.dtype);
  const long long total = (long long)v.n * v.h * v.w * v.c;
  if ((size_t)total * el > dst_bytes) return fail(h, JDE_ERR_CAPACITY, "jde_get_tensor: dst too small");
  (jde_count_launch(), gather_view_kernel<<<(unsigned)((total + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(v, dst, el));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(h, JDE_ERR_CUDA, "gather: %s", cudaGetErrorString(e));
  return JDE_OK;
}

jde_status jde_set_act_amax(jde_handle* h, const float* amax, int n) {
  if (!h) return fail(nullptr, JDE_ERR_INVALID_ARG, "handle is NULL");
  if (h->cfg.precision != JDE_FP8_E4M3)
    return fail(h, JDE_ERR_INVALID_ARG, "jde_set_act_amax: only E4M3 handles take activation scales");
  if (!amax || n != JDE_NUM_LAYERS) return fail(h, JDE_ERR_INVALID_ARG, "jde_set_act_amax: need %d values", JDE_NUM_LAYERS);
  for (int l = 0; l < n; ++l)
    if (!(amax[l] >= 0.f) || !isfinite(amax[l]))
      return fail(h, JDE_ERR_INVALID_ARG, "jde_set_act_amax: amax[%d] = %g", l, (double)amax[l]);
  // scale of a stored tensor = amax / 448; a concat buffer takes the larger amax of its writers
  std::vector<float> bmax(T_COUNT, 0.f);
  for (int l = 0; l < n; ++l) {
    const int b = buffer_of(h, l);
    bmax[b] = fmaxf(bmax[b], amax[l]);
  }
  for (int t = 0; t < T_COUNT; ++t) h->act_scale[t] = (bmax[t] > 0.f ? bmax[t] : 1.0f) / 448.0f;
  for (int l = 0; l < n; ++l) {
    LayerW& lw = h->w[l];
    if (!lw.q) continue;
    const float s_in = h->act_scale[buffer_of(h, h->io[l].in)];
    std::vector<float> m(lw.cout_pad_tc);
    for (int co = 0; co < lw.cout_pad_tc; ++co) m[co] = (float)((double)s_in * lw.wscale_host[co]);
    CUDA_OR(h, cudaMemcpy(lw.mult, m.data(), sizeof(float) * m.size(), cudaMemcpyHostToDevice));
  }
  h->plans.clear();   // plans carry the scales
  h->scales_set = true;
  return JDE_OK;
}

jde_status jde_act_amax(jde_handle* h, float* amax, void* stream) {
  if (!h) return fail(nullptr, JDE_ERR_INVALID_ARG, "handle is NULL");
  if (!amax) return fail(h, JDE_ERR_INVALID_ARG, "jde_act_amax: amax is NULL");
  if (!h->cur) return fail(h, JDE_ERR_INVALID_ARG, "jde_act_amax: no forward has run");
  for (int l = 0; l < JDE_NUM_LAYERS; ++l)
    if (overwritten(h, l) || not_stored(h, l))
      return fail(h, JDE_ERR_UNSUPPORTED,
                  "jde_act_amax: layer outputs are not kept (needs keep_layer_outputs = 1, sparse_emb = 0)");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!h->d_amax && !dmalloc((void**)&h->d_amax, sizeof(float) * JDE_NUM_LAYERS))
    return fail(h, JDE_ERR_OOM, "amax scratch");
  CUDA_OR(h, cudaMemsetAsync(h->d_amax, 0, sizeof(float) * JDE_NUM_LAYERS, st));
  for (int l = 0; l < JDE_NUM_LAYERS; ++l) {
    TView v = view_of(*h->cur, l, h->cur_n);
    if (h->io[l].head >= 0) v.ptr = static_cast<char*>(v.ptr) + (size_t)h->cur_set * h->cur->set_bytes[l];
    jde_count_launch();
    amax_kernel<<<152, 256, 0, st>>>(v, h->act_scale[buffer_of(h, l)], h->d_amax + l);
  }
  CUDA_OR(h, cudaMemcpyAsync(amax, h->d_amax, sizeof(float) * JDE_NUM_LAYERS, cudaMemcpyDeviceToHost, st));
  CUDA_OR(h, cudaStreamSynchronize(st));
  return JDE_OK;
}

jde_status jde_autotune(jde_handle* h, int n, int in_w, int in_h, void* stream) {
  if (!h) return fail(nullptr, JDE_ERR_INVALID_ARG, "handle is NULL");
  if (h->cfg.precision == JDE_FP32) return fail(h, JDE_ERR_UNSUPPORTED, "jde_autotune: tensor-core handles only");
  if (n < 1 || n > h->cfg.max_batch || in_w % 32 || in_h % 32 || in_w < 32 || in_h < 32 || in_w > h->cfg.max_in_w ||
      in_h > h->cfg.max_in_h)
    return fail(h, JDE_ERR_INVALID_ARG, "jde_autotune: bad arguments");
  if (h->cfg.precision == JDE_FP8_E4M3 && !h->scales_set)
    return fail(h, JDE_ERR_INVALID_ARG, "jde_autotune: E4M3 handle has no activation scales");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ResBuffers* rb;
  jde_status s = get_res(h, in_w, in_h, &rb);
  if (s != JDE_OK) return s;
  const auto key = std::make_tuple(in_w, in_h, n);
  h->tuned_bn.erase(key);
  h->plans.erase(key);
  Plan* plan;
  s = get_plan(h, rb, n, &plan);
  if (s != JDE_OK) return s;
  std::vector<int> best(JDE_NUM_LAYERS, 0);
  constexpr int REPS = 5;
  cudaEvent_t e0[REPS], e1[REPS];
  for (int r = 0; r < REPS; ++r) {
    CUDA_OR(h, cudaEventCreate(&e0[r]));
    CUDA_OR(h, cudaEventCreate(&e1[r]));
  }
  // the launch before layer l in a forward: its output is (mostly) layer l's input, so re-running it
  // before each timed launch recreates the cache state a forward gives layer l
  auto previous = [&](int l) -> cudaError_t {
    for (int k = l - 1; k >= 0; --k) {
      if (not_stored(h, k)) continue;
      if (k == 1 && plan->stem_s2) return stem_s2_launch(plan->stem_s2.get(), st);
      if (k == 3 && plan->res1) return res1_launch(plan->res1.get(), st);
      return conv_tc_launch(plan->tc[k], st);
    }
    return cudaSuccess;
  };
  for (int l = 0; l < JDE_NUM_LAYERS; ++l) {
    if (not_stored(h, l)) continue;                  // sparse embedding head: not a conv launch
    if (l == 1 && plan->stem_s2) continue;           // fused with the stem: one tile shape
    if (l == 3 && plan->res1) continue;              // fused residual block: one tile shape
    const TcPlan& def = plan->tc[l];
    if (def.mode == 2 || def.mode == 3) continue;    // stem and window convs have one tile shape
    const LayerW& lw = h->w[l];
    const void* w = lw.q ? static_cast<const void*>(lw.w_q) : static_cast<const void*>(lw.w_nk);
    float best_ms = 1e30f;
    for (int code : {32, 64, 128, 256, 129, 130}) {
      const int bn = code & ~3, msub = (code & 1) ? 2 : 1, pair128 = (code & 2) ? 1 : 0;
      // 32-wide tiles only where they are the default (the 24-channel heads, 32-channel outputs)
      if (lw.cout_pad_tc % bn || (bn == 32 && lw.bn != 32)) continue;
      TcPlan cand;
      char msg[256];
      if (!conv_tc_plan(cand, plan->specs[l], w, lw.cout_pad_tc, bn, msg, sizeof(msg), msub, pair128)) continue;
      // same addressing mode and k-block width: the same order of the K sum
      if (cand.mode != def.mode || cand.bkc != def.bkc || cand.msub != msub) continue;
      if (msub == 2 && !cand.tma_out) continue;
      if (conv_tc_launch(cand, st) != cudaSuccess) {   // shape without a built configuration
        cudaGetLastError();
        continue;
      }
      for (int r = 0; r < REPS; ++r) {
        CUDA_OR(h, previous(l));
        CUDA_OR(h, cudaEventRecord(e0[r], st));
        CUDA_OR(h, conv_tc_launch(cand, st));
        CUDA_OR(h, cudaEventRecord(e1[r], st));
      }
      CUDA_OR(h, cudaEventSynchronize(e1[REPS - 1]));
      float t[REPS];
      for (int r = 0; r < REPS; ++r) CUDA_OR(h, cudaEventElapsedTime(&t[r], e0[r], e1[r]));
      std::sort(t, t + REPS);
      const float ms = t[REPS / 2];   // median launch
      if (ms < best_ms) {
        best_ms = ms;
        best[l] = code;
      }
    }
  }
  for (int r = 0; r < REPS; ++r) {
    cudaEventDestroy(e0[r]);
    cudaEventDestroy(e1[r]);
  }
  h->tuned_bn[key] = best;
  h->plans.erase(key);   // rebuilt with the chosen tiles on the next forward
  return JDE_OK;
}

jde_status jde_set_tile_choice(jde_handle* h, int n, int in_w, int in_h, const int* bn) {
  if (!h || !bn) return fail(h, JDE_ERR_INVALID_ARG, "jde_set_tile_choice: NULL argument");
  if (h->cfg.precision == JDE_FP32) return fail(h, JDE_ERR_UNSUPPORTED, "jde_set_tile_choice: tensor-core handles only");
  if (n < 1 || n > h->cfg.max_batch || in_w % 32 || in_h % 32 || in_w < 32 || in_h < 32 || in_w > h->cfg.max_in_w ||
      in_h > h->cfg.max_in_h)
    return fail(h, JDE_ERR_INVALID_ARG, "jde_set_tile_choice: bad arguments");
  std::vector<int> codes(bn, bn + JDE_NUM_LAYERS);
  for (int l = 0; l < JDE_NUM_LAYERS; ++l)
    if (!(codes[l] == 0 || codes[l] == 32 || codes[l] == 64 || codes[l] == 128 || codes[l] == 256 || codes[l] == 129 ||
          codes[l] == 130))
      return fail(h, JDE_ERR_INVALID_ARG, "jde_set_tile_choice: layer %d: tile code %d", l, codes[l]);
  ResBuffers* rb;
  jde_status s = get_res(h, in_w, in_h, &rb);
  if (s != JDE_OK) return s;
  const auto key = std::make_tuple(in_w, in_h, n);
  auto prev = h->tuned_bn.find(key);
  const bool had = prev != h->tuned_bn.end();
  const std::vector<int> old = had ? prev->second : std::vector<int>();
  h->tuned_bn[key] = codes;
  h->plans.erase(key);
  Plan* plan;
  s = get_plan(h, rb, n, &plan);
  if (s == JDE_OK) {
    // a code the layer cannot run as asked (e.g. two sub-tiles whose windows do not fit) is refused
    for (int l = 0; l < JDE_NUM_LAYERS && s == JDE_OK; ++l) {
      if (codes[l] == 0 || plan->tc.empty() || not_stored(h, l) || (l == 1 && plan->stem_s2) ||
          (l == 3 && plan->res1))
        continue;
      const TcPlan& t = plan->tc[l];
      // the default tile's addressing mode: another mode would sum K in another order
      TcPlan def;
      char msg[256];
      const LayerW& lw = h->w[l];
      const void* w = lw.q ? static_cast<const void*>(lw.w_q) : static_cast<const void*>(lw.w_nk);
      const bool def_ok = conv_tc_plan(def, plan->specs[l], w, lw.cout_pad_tc, lw.bn, msg, sizeof(msg));
      if (t.bn != (codes[l] & ~3) || t.msub != ((codes[l] & 1) ? 2 : 1) || ((codes[l] & 2) && t.cg != 2) || !def_ok ||
          def.mode != t.mode || def.bkc != t.bkc)
        s = fail(h, JDE_ERR_UNSUPPORTED, "jde_set_tile_choice: layer %d cannot run tile code %d", l, codes[l]);
    }
  }
  if (s != JDE_OK) {
    if (had)
      h->tuned_bn[key] = old;
    else
      h->tuned_bn.erase(key);
    h->plans.erase(key);
    return s;
  }
  return JDE_OK;
}

jde_status jde_tile_choice(jde_handle* h, int n, int in_w, int in_h, int* bn) {
  if (!h || !bn) return fail(h, JDE_ERR_INVALID_ARG, "jde_tile_choice: NULL argument");
  auto tb = h->tuned_bn.find(std::make_tuple(in_w, in_h, n));
  for (int l = 0; l < JDE_NUM_LAYERS; ++l)
    bn[l] = (tb != h->tuned_bn.end() && tb->second[l] > 0) ? tb->second[l] : h->w[l].bn;
  return JDE_OK;
}

jde_status jde_device_bytes(jde_handle* h, size_t* out) {
  if (!h || !out) return fail(h, JDE_ERR_INVALID_ARG, "jde_device_bytes: NULL argument");
  size_t b = h->weight_bytes + sizeof(int) + sizeof(LbAxis) * (size_t)(h->cfg.max_in_w + h->cfg.max_in_h);
  for (const auto& kv : h->res)
    for (size_t t : kv.second.bytes) b += t;
  if (h->pb.cand_keys) b += post_bytes(h->pb_n, h->pb.cand_cap, h->pb.kmax);
  b += h->frames_cap;
  if (h->rows_stage) b += h->rows_stage_cap * sizeof(float) + sizeof(int32_t) * (size_t)h->cfg.max_batch +
                         h->rows_stage_cap / 518 * sizeof(int32_t);
  b += track_bytes(h->cfg);
  *out = b;
  return JDE_OK;
}

jde_status jde_estimate_device_bytes(const jde_config* cfg, int in_w, int in_h, size_t* out) {
  if (!cfg || !out || in_w < 32 || in_h < 32 || in_w % 32 || in_h % 32 || in_w > cfg->max_in_w ||
      in_h > cfg->max_in_h || cfg->max_batch < 1)
    return fail(nullptr, JDE_ERR_INVALID_ARG, "jde_estimate_device_bytes: bad arguments");
  jde_handle tmp;
  tmp.cfg = *cfg;
  tmp.io = build_io(tmp.cfg);
  const bool bf16 = cfg->precision != JDE_FP32;
  const auto& L = layers();
  size_t b = sizeof(int) + sizeof(LbAxis) * (size_t)(cfg->max_in_w + cfg->max_in_h);
  for (size_t l = 0; l < L.size(); ++l) b += layer_weight_bytes(L[l], cfg->precision, (int)l);
  if (bf16) b += STEM_S2_PACK_BYTES;
  std::vector<TensorDesc> td;
  tensor_desc_table(&tmp, in_w, in_h, td);
  for (int t = 0; t < T_COUNT; ++t) {
    if (td[t].alias >= 0 || not_stored(&tmp, t)) continue;
    b += tensor_bytes(td[t], cfg->max_batch) * (two_sets(&tmp, t) ? 2 : 1);
  }
  b += post_bytes(cfg->max_batch, anchors_for(cfg->max_in_w, cfg->max_in_h), cfg->max_cand);
  b += track_bytes(*cfg);
  *out = b;
  return JDE_OK;
}

jde_status jde_kernel_errors(jde_handle* h, int* word, void* stream) {
  if (!h || !word) return fail(h, JDE_ERR_INVALID_ARG, "jde_kernel_errors: NULL argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CUDA_OR(h, cudaMemcpyAsync(word, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CUDA_OR(h, cudaStreamSynchronize(st));
  CUDA_OR(h, cudaMemsetAsync(h->d_err, 0, sizeof(int), st));
  return JDE_OK;
}

jde_status jde_track_step(jde_handle* h, int n, const int32_t* stream_ids, const jde_dets* dets, jde_tracks* out,
                          void* stream) {
  if (!h) return fail(nullptr, JDE_ERR_INVALID_ARG, "handle is NULL");
  char msg[256] = {0};
  const int r = track_step(h->trk, h->cfg, n, stream_ids, dets, out, h->d_err, static_cast<cudaStream_t>(stream), msg,
                           sizeof(msg));
  if (r != JDE_OK) return fail(h, (jde_status)r, "jde_track_step: %s", msg);
  return JDE_OK;
}

}  // extern "C"

jde_status track_step_device_slots(jde_handle* h, int n, const int32_t* stream_ids, const int* dev_slots,
                                   const jde_dets* dets, jde_tracks* out, cudaStream_t st) {
  if (!h || !dev_slots) return fail(h, JDE_ERR_INVALID_ARG, "track_step_device_slots: NULL argument");
  if (!dets->on_device || !out->on_device)
    return fail(h, JDE_ERR_INVALID_ARG, "track_step_device_slots: detections and tracks must be on the device");
  char msg[256] = {0};
  const int r = track_step(h->trk, h->cfg, n, stream_ids, dets, out, h->d_err, st, msg, sizeof(msg), dev_slots);
  if (r != JDE_OK) return fail(h, (jde_status)r, "jde_track_step: %s", msg);
  return JDE_OK;
}

extern "C" {

unsigned long long jde_launch_count(void) { return g_launches.load(); }

jde_status jde_selftest_wait(jde_handle* h, long long limit_cycles, int* word, void* stream) {
  if (!h) return fail(nullptr, JDE_ERR_INVALID_ARG, "handle is NULL");
  if (!word || limit_cycles < 1 || limit_cycles > (1ll << 31))
    return fail(h, JDE_ERR_INVALID_ARG, "jde_selftest_wait: word NULL or limit out of [1, 2^31]");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  jde_count_launch();
  wait_selftest_kernel<<<1, 32, 0, st>>>(h->d_err, limit_cycles);
  CUDA_OR(h, cudaGetLastError());
  CUDA_OR(h, cudaMemcpyAsync(word, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CUDA_OR(h, cudaStreamSynchronize(st));
  CUDA_OR(h, cudaMemsetAsync(h->d_err, 0, sizeof(int), st));
  CUDA_OR(h, cudaStreamSynchronize(st));
  if (*word & KERR_TIMEOUT)
    return fail(h, JDE_ERR_TIMEOUT, "bounded device wait gave up after %lld cycles (error word 0x%x)", limit_cycles,
                *word);
  return JDE_OK;
}

jde_status jde_set_profile_events(jde_handle* h, void* forward_begin, void* conv_begin, void* conv_end) {
  if (!h) return fail(nullptr, JDE_ERR_INVALID_ARG, "handle is NULL");
  h->prof[0] = static_cast<cudaEvent_t>(forward_begin);
  h->prof[1] = static_cast<cudaEvent_t>(conv_begin);
  h->prof[2] = static_cast<cudaEvent_t>(conv_end);
  return JDE_OK;
}

jde_status jde_set_dependent_launch(jde_handle* h, int on) {
  if (!h) return fail(nullptr, JDE_ERR_INVALID_ARG, "handle is NULL");
  if (on != 0 && on != 1) return fail(h, JDE_ERR_INVALID_ARG, "jde_set_dependent_launch: %d is not 0 or 1", on);
  h->cfg.dependent_launch = on;
  for (auto& kv : h->plans)
    for (TcPlan& t : kv.second.tc) t.pdl = on;
  return JDE_OK;
}

jde_status jde_stream_reset(jde_handle* h, int stream_id, void* stream) {
  if (!h) return fail(nullptr, JDE_ERR_INVALID_ARG, "handle is NULL");
  if (stream_id < 0 || stream_id >= h->cfg.max_streams)
    return fail(h, JDE_ERR_NOT_FOUND, "stream id %d out of range", stream_id);
  if (track_reset(h->trk, stream_id, static_cast<cudaStream_t>(stream)) != 0)
    return fail(h, JDE_ERR_CUDA, "stream reset failed");
  return JDE_OK;
}

}  // extern "C"
