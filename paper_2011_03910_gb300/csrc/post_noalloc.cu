// jde_postprocess_noalloc: the post-processing chain (decode, confidence
// filter, sort, NMS, embedding gather + L2) with no device allocation at all.
//
// Who needs it: callers that cannot call cudaMalloc once they run - a host
// application that reserves all device memory up front and hands out only
// fixed buffers, a hard real-time loop where a driver allocation (which may
// synchronise the device and take milliseconds) is not allowed, or a plugin
// that is given device pointers but no allocator.  jde_create/jde_postprocess
// allocate their scratch with cudaMalloc; this entry point takes its scratch
// from a fixed array compiled into the library instead.
//
// The array below lives in the device code of this file.  CUDA loads that code
// onto a device lazily, the first time the array's address is looked up there,
// and the load reserves the 32 MiB, which the device then holds until the
// process exits.  The look-up (cudaGetSymbolAddress, once per device, with that
// device current) happens in jde_create for the handle's device and otherwise
// in the first jde_postprocess_noalloc call on a device.  Host code must not
// use the array's name as a device pointer: on the host it is only a stand-in.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "../../include/jde.h"
#include "internal.h"

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = 32ull << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = JDE_MAX_DEVICES;
std::mutex g_setup_mutex;
void* g_scratch_addr[MAX_DEVICES] = {nullptr};

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Largest model input side the entry point accepts (keeps every size computation far from overflow).
constexpr int NOALLOC_MAX_SIDE = 16384;

// Device address of the scratch array on the current device, looked up once per device.
void* scratch_address(int* dev_out, char* msg, size_t len) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
    if (msg && len) snprintf(msg, len, "no usable current CUDA device");
    return nullptr;
  }
  if (dev_out) *dev_out = dev;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      if (msg && len) snprintf(msg, len, "cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return nullptr;
    }
    g_scratch_addr[dev] = p;
  }
  return g_scratch_addr[dev];
}

void say(char* msg, size_t len, const char* text) {
  if (msg && len) snprintf(msg, len, "%s", text);
}

}  // namespace

// Loads the scratch array onto the current device and records its address (called by jde_create).
int noalloc_scratch_setup(char* msg, size_t len) { return scratch_address(nullptr, msg, len) ? 0 : 1; }

extern "C" jde_status jde_postprocess_noalloc(const float* const* heads, int n, int in_w, int in_h, int src_w,
                                              int src_h, float conf_thresh, float nms_iou, int max_cand,
                                              jde_dets* out, void* stream, char* err_msg, size_t err_len) {
  char buf[256];
  if (!heads || !out || !out->rows || !out->count || out->cap < 1 || !out->on_device || n < 1 || in_w < 32 ||
      in_h < 32 || in_w % 32 || in_h % 32 || in_w > NOALLOC_MAX_SIDE || in_h > NOALLOC_MAX_SIDE || src_w < 1 ||
      src_h < 1 || max_cand < 64 || max_cand > 4096 || max_cand % 64) {
    say(err_msg, err_len,
        "jde_postprocess_noalloc: bad arguments (device outputs required; sizes multiples of 32 up to 16384; "
        "max_cand a multiple of 64 in [64, 4096])");
    return JDE_ERR_INVALID_ARG;
  }
  {
    // n frames of 4 * (in_w in_h / 1024 + in_w in_h / 256 + in_w in_h / 64) anchors, counted in size_t
    const size_t px = (size_t)in_w * (size_t)in_h;
    const size_t anchors = 4 * (px / 1024 + px / 256 + px / 64);
    if ((size_t)n * anchors * sizeof(uint64_t) > NOALLOC_SCRATCH_BYTES) {
      snprintf(buf, sizeof(buf),
               "jde_postprocess_noalloc: %d frames at %dx%d need more than the fixed scratch of %zu bytes "
               "for their candidate keys alone; use fewer frames per call",
               n, in_w, in_h, NOALLOC_SCRATCH_BYTES);
      say(err_msg, err_len, buf);
      return JDE_ERR_CAPACITY;
    }
  }
  for (int i = 0; i < 6; ++i)
    if (!heads[i]) {
      say(err_msg, err_len, "jde_postprocess_noalloc: a head pointer is NULL");
      return JDE_ERR_INVALID_ARG;
    }

  // geometry of the three heads (strides 32, 16, 8), anchors and letterbox
  HeadGeom g;
  memset(&g, 0, sizeof(g));
  g.n = n;
  const int strides[3] = {32, 16, 8};
  const float base[3] = {128.f, 32.f, 8.f};
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
  const double r = fmin((double)in_w / src_w, (double)in_h / src_h);
  const int nw = (int)floor(src_w * r + 0.5), nh = (int)floor(src_h * r + 0.5);
  g.ratio = (float)r;
  g.pad_x = (float)((in_w - nw) / 2);
  g.pad_y = (float)((in_h - nh) / 2);

  // carve the scratch: every buffer the post-processing kernels need
  const size_t A = (size_t)g.off[3], K = (size_t)max_cand;
  size_t off = 0;
  const size_t o_keys = off;
  off = align256(off + sizeof(uint64_t) * n * A);
  const size_t o_cnt = off;
  off = align256(off + sizeof(int) * n);
  const size_t o_sorted = off;
  off = align256(off + sizeof(uint64_t) * n * K);
  const size_t o_nsorted = off;
  off = align256(off + sizeof(int) * n);
  const size_t o_boxes = off;
  off = align256(off + sizeof(float4) * n * K);
  const size_t o_conf = off;
  off = align256(off + sizeof(float) * n * K);
  const size_t o_cls = off;
  off = align256(off + sizeof(float) * n * K);
  const size_t o_mask = off;
  off = align256(off + sizeof(unsigned long long) * n * K * (K / 64));
  const size_t o_keep = off;
  off = align256(off + sizeof(int) * n * K);
  const size_t o_nkeep = off;
  off = align256(off + sizeof(int) * n);
  if (off > NOALLOC_SCRATCH_BYTES) {
    snprintf(buf, sizeof(buf),
             "jde_postprocess_noalloc: %d frames at %dx%d with max_cand %d need %zu bytes of scratch, "
             "the fixed scratch holds %zu; use fewer frames per call or a smaller max_cand",
             n, in_w, in_h, max_cand, off, NOALLOC_SCRATCH_BYTES);
    say(err_msg, err_len, buf);
    return JDE_ERR_CAPACITY;
  }

  // once per device (with that device current): the device address of the scratch array
  char why[160] = {0};
  void* base_ptr = scratch_address(nullptr, why, sizeof(why));
  if (!base_ptr) {
    snprintf(buf, sizeof(buf), "jde_postprocess_noalloc: %s", why);
    say(err_msg, err_len, buf);
    return JDE_ERR_CUDA;
  }
  unsigned char* s = static_cast<unsigned char*>(base_ptr);
  PostBufs b{};   // the sparse-embedding scratch stays null: caller heads carry dense embedding maps
  b.cand_keys = reinterpret_cast<uint64_t*>(s + o_keys);
  b.cand_count = reinterpret_cast<int*>(s + o_cnt);   // zeroed by post_launch before the filter runs
  b.cand_cap = (int)A;
  b.sorted = reinterpret_cast<uint64_t*>(s + o_sorted);
  b.n_sorted = reinterpret_cast<int*>(s + o_nsorted);
  b.boxes = reinterpret_cast<float4*>(s + o_boxes);
  b.conf = reinterpret_cast<float*>(s + o_conf);
  b.cls = reinterpret_cast<float*>(s + o_cls);
  b.mask = reinterpret_cast<unsigned long long*>(s + o_mask);
  b.keep_idx = reinterpret_cast<int*>(s + o_keep);
  b.n_keep = reinterpret_cast<int*>(s + o_nkeep);
  b.kmax = max_cand;
  const cudaError_t e = post_launch(heads, g, conf_thresh, nms_iou, b, out->rows, out->count, out->anchor_index,
                                    out->cap, nullptr, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    snprintf(buf, sizeof(buf), "jde_postprocess_noalloc: launch failed: %s", cudaGetErrorString(e));
    say(err_msg, err_len, buf);
    return JDE_ERR_CUDA;
  }
  return JDE_OK;
}
