// Device decode of compressed frames: the capture stage of the paper's pipeline (Sec. 4.4 reads video
// frames on the host and queues them) moved onto the GPU for Motion-JPEG streams.  Each frame is a
// baseline JPEG bitstream in host memory; nvJPEG decodes a batch of them into interleaved 8-bit RGB
// frames in device memory, the layout jde_forward reads.  The hardware backend runs on the GPU's JPEG
// decode engines; where that backend is not available the GPU-assisted hybrid backend is used and
// reported.  An encoder (nvJPEG, quality and 4:2:0 chroma subsampling chosen by the caller) makes the
// bitstreams of synthetic streams.
//
// libnvjpeg is loaded at run time (dlopen), so libjde builds and loads where it is absent; the calls
// then return JDE_ERR_UNSUPPORTED.  The few nvJPEG declarations needed are written out below.
#include <dlfcn.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace {

// nvJPEG's C interface: opaque handles, int-valued enums, and the image descriptor (per component a
// pointer and a pitch, four components).
typedef void* NvjHandle;
typedef void* NvjState;
typedef void* NvjEncState;
typedef void* NvjEncParams;
struct NvjImage {
  unsigned char* channel[4];
  size_t pitch[4];
};
constexpr int NVJ_SUCCESS = 0;
constexpr int NVJ_BACKEND_GPU_HYBRID = 2;
constexpr int NVJ_BACKEND_HARDWARE = 3;
constexpr int NVJ_OUTPUT_RGBI = 5;
constexpr int NVJ_INPUT_RGBI = 5;
constexpr int NVJ_CSS_420 = 2;

struct Nvj {
  int (*create_ex)(int, void*, void*, unsigned, NvjHandle*) = nullptr;
  int (*destroy)(NvjHandle) = nullptr;
  int (*state_create)(NvjHandle, NvjState*) = nullptr;
  int (*state_destroy)(NvjState) = nullptr;
  int (*image_info)(NvjHandle, const unsigned char*, size_t, int*, int*, int*, int*) = nullptr;
  int (*batched_init)(NvjHandle, NvjState, int, int, int) = nullptr;
  int (*batched)(NvjHandle, NvjState, const unsigned char* const*, const size_t*, NvjImage*, cudaStream_t) = nullptr;
  int (*enc_state_create)(NvjHandle, NvjEncState*, cudaStream_t) = nullptr;
  int (*enc_state_destroy)(NvjEncState) = nullptr;
  int (*enc_params_create)(NvjHandle, NvjEncParams*, cudaStream_t) = nullptr;
  int (*enc_params_destroy)(NvjEncParams) = nullptr;
  int (*enc_quality)(NvjEncParams, int, cudaStream_t) = nullptr;
  int (*enc_sampling)(NvjEncParams, int, cudaStream_t) = nullptr;
  int (*encode_image)(NvjHandle, NvjEncState, NvjEncParams, const NvjImage*, int, int, int, cudaStream_t) = nullptr;
  int (*retrieve)(NvjHandle, NvjEncState, unsigned char*, size_t*, cudaStream_t) = nullptr;
  bool ok = false;
  std::string why;
};

Nvj& nvj() {
  static Nvj n;
  static std::once_flag once;
  std::call_once(once, [] {
    const char* names[] = {"libnvjpeg.so.13", "libnvjpeg.so", "/usr/local/cuda/lib64/libnvjpeg.so.13",
                           "/usr/local/cuda/targets/sbsa-linux/lib/libnvjpeg.so.13",
                           "/usr/local/cuda/targets/x86_64-linux/lib/libnvjpeg.so.13"};
    void* lib = nullptr;
    for (const char* nm : names)
      if ((lib = dlopen(nm, RTLD_NOW | RTLD_LOCAL))) break;
    if (!lib) {
      n.why = "libnvjpeg not found";
      return;
    }
    bool all = true;
    auto sym = [&](auto& fp, const char* name) {
      fp = reinterpret_cast<std::remove_reference_t<decltype(fp)>>(dlsym(lib, name));
      all = all && fp;
    };
    sym(n.create_ex, "nvjpegCreateEx");
    sym(n.destroy, "nvjpegDestroy");
    sym(n.state_create, "nvjpegJpegStateCreate");
    sym(n.state_destroy, "nvjpegJpegStateDestroy");
    sym(n.image_info, "nvjpegGetImageInfo");
    sym(n.batched_init, "nvjpegDecodeBatchedInitialize");
    sym(n.batched, "nvjpegDecodeBatched");
    sym(n.enc_state_create, "nvjpegEncoderStateCreate");
    sym(n.enc_state_destroy, "nvjpegEncoderStateDestroy");
    sym(n.enc_params_create, "nvjpegEncoderParamsCreate");
    sym(n.enc_params_destroy, "nvjpegEncoderParamsDestroy");
    sym(n.enc_quality, "nvjpegEncoderParamsSetQuality");
    sym(n.enc_sampling, "nvjpegEncoderParamsSetSamplingFactors");
    sym(n.encode_image, "nvjpegEncodeImage");
    sym(n.retrieve, "nvjpegEncodeRetrieveBitstream");
    n.ok = all;
    if (!all) n.why = "libnvjpeg lacks a required entry point";
  });
  return n;
}

}  // namespace

struct jde_decoder {
  int device = 0;
  int max_batch = 0;
  int backend = 0;               // JDE_DECODE_HARDWARE or JDE_DECODE_GPU_HYBRID
  NvjHandle h = nullptr;         // decode handle (the backend above)
  NvjState state = nullptr;
  int init_batch = 0;            // batch size the batched decoder was initialised for
  NvjHandle eh = nullptr;        // encode handle (GPU-assisted backend)
  NvjEncState es = nullptr;
  NvjEncParams ep = nullptr;
  std::vector<NvjImage> dst;
  std::string err;
};

namespace {

jde_status dfail(jde_decoder* d, jde_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (d) d->err = buf;
  return st;
}

}  // namespace

extern "C" {

jde_status jde_decoder_create(int device, int max_batch, int hardware, jde_decoder** out) {
  if (!out || max_batch < 1 || max_batch > 1024) return JDE_ERR_INVALID_ARG;
  *out = nullptr;
  Nvj& n = nvj();
  if (!n.ok) return JDE_ERR_UNSUPPORTED;
  if (cudaSetDevice(device) != cudaSuccess) return JDE_ERR_CUDA;
  jde_decoder* d = new jde_decoder();
  d->device = device;
  d->max_batch = max_batch;
  int r = 1;
  if (hardware) {
    r = n.create_ex(NVJ_BACKEND_HARDWARE, nullptr, nullptr, 0, &d->h);
    if (r == NVJ_SUCCESS) d->backend = JDE_DECODE_HARDWARE;
  }
  if (r != NVJ_SUCCESS) {
    d->h = nullptr;
    r = n.create_ex(NVJ_BACKEND_GPU_HYBRID, nullptr, nullptr, 0, &d->h);
    if (r == NVJ_SUCCESS) d->backend = JDE_DECODE_GPU_HYBRID;
  }
  if (r != NVJ_SUCCESS || n.state_create(d->h, &d->state) != NVJ_SUCCESS) {
    if (d->h) n.destroy(d->h);
    delete d;
    return JDE_ERR_UNSUPPORTED;
  }
  d->dst.resize(max_batch);
  *out = d;
  return JDE_OK;
}

void jde_decoder_destroy(jde_decoder* d) {
  if (!d) return;
  Nvj& n = nvj();
  cudaSetDevice(d->device);
  cudaDeviceSynchronize();
  if (d->ep) n.enc_params_destroy(d->ep);
  if (d->es) n.enc_state_destroy(d->es);
  if (d->eh) n.destroy(d->eh);
  if (d->state) n.state_destroy(d->state);
  if (d->h) n.destroy(d->h);
  delete d;
}

const char* jde_decoder_last_error(jde_decoder* d) { return d ? d->err.c_str() : ""; }

int jde_decoder_backend(jde_decoder* d) { return d ? d->backend : 0; }

jde_status jde_decode_jpeg(jde_decoder* d, const uint8_t* const* bitstreams, const size_t* lengths, int n, int w,
                           int h, uint8_t* frames, void* stream) {
  if (!d || !bitstreams || !lengths || !frames) return dfail(d, JDE_ERR_INVALID_ARG, "NULL argument");
  if (n < 1 || n > d->max_batch || w < 1 || h < 1)
    return dfail(d, JDE_ERR_INVALID_ARG, "n = %d (at most %d), %dx%d", n, d->max_batch, w, h);
  Nvj& nv = nvj();
  cudaSetDevice(d->device);
  // every bitstream must hold a 3-component w x h image (headers parsed on the host, nothing decoded)
  for (int i = 0; i < n; ++i) {
    if (!bitstreams[i] || lengths[i] < 4) return dfail(d, JDE_ERR_INVALID_ARG, "bitstream %d is empty", i);
    int comps = 0, css = 0, ws[4] = {0}, hs[4] = {0};
    if (nv.image_info(d->h, bitstreams[i], lengths[i], &comps, &css, ws, hs) != NVJ_SUCCESS)
      return dfail(d, JDE_ERR_INVALID_ARG, "bitstream %d: not a JPEG image nvJPEG can parse", i);
    if (comps != 3 || ws[0] != w || hs[0] != h)
      return dfail(d, JDE_ERR_INVALID_ARG, "bitstream %d: %d components of %dx%d, expected 3 of %dx%d", i, comps,
                   ws[0], hs[0], w, h);
  }
  if (d->init_batch != n) {
    if (nv.batched_init(d->h, d->state, n, 1, NVJ_OUTPUT_RGBI) != NVJ_SUCCESS)
      return dfail(d, JDE_ERR_CUDA, "batched decoder initialisation for %d frames failed", n);
    d->init_batch = n;
  }
  for (int i = 0; i < n; ++i) {
    memset(&d->dst[i], 0, sizeof(NvjImage));
    d->dst[i].channel[0] = frames + (size_t)i * w * h * 3;
    d->dst[i].pitch[0] = (size_t)w * 3;
  }
  const int r = nv.batched(d->h, d->state, bitstreams, lengths, d->dst.data(), static_cast<cudaStream_t>(stream));
  if (r != NVJ_SUCCESS) {
    d->init_batch = 0;   // a failed batch needs a fresh initialisation
    return dfail(d, JDE_ERR_CUDA, "nvjpegDecodeBatched failed (status %d)", r);
  }
  return JDE_OK;
}

jde_status jde_encode_jpeg(jde_decoder* d, const uint8_t* frames, int n, int w, int h, int quality,
                           uint8_t* const* out, size_t* lengths, void* stream) {
  if (!d || !frames || !out || !lengths) return dfail(d, JDE_ERR_INVALID_ARG, "NULL argument");
  if (n < 1 || w < 1 || h < 1 || quality < 1 || quality > 100)
    return dfail(d, JDE_ERR_INVALID_ARG, "n = %d, %dx%d, quality %d", n, w, h, quality);
  Nvj& nv = nvj();
  cudaSetDevice(d->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!d->eh) {
    if (nv.create_ex(NVJ_BACKEND_GPU_HYBRID, nullptr, nullptr, 0, &d->eh) != NVJ_SUCCESS) {
      d->eh = nullptr;
      return dfail(d, JDE_ERR_UNSUPPORTED, "no nvJPEG encoder");
    }
    if (nv.enc_state_create(d->eh, &d->es, st) != NVJ_SUCCESS ||
        nv.enc_params_create(d->eh, &d->ep, st) != NVJ_SUCCESS ||
        nv.enc_sampling(d->ep, NVJ_CSS_420, st) != NVJ_SUCCESS)
      return dfail(d, JDE_ERR_UNSUPPORTED, "nvJPEG encoder set-up failed");
  }
  if (nv.enc_quality(d->ep, quality, st) != NVJ_SUCCESS) return dfail(d, JDE_ERR_INVALID_ARG, "quality %d", quality);
  for (int i = 0; i < n; ++i) {
    NvjImage src;
    memset(&src, 0, sizeof(src));
    src.channel[0] = const_cast<unsigned char*>(frames + (size_t)i * w * h * 3);
    src.pitch[0] = (size_t)w * 3;
    if (nv.encode_image(d->eh, d->es, d->ep, &src, NVJ_INPUT_RGBI, w, h, st) != NVJ_SUCCESS)
      return dfail(d, JDE_ERR_CUDA, "encoding frame %d failed", i);
    size_t len = 0;
    if (nv.retrieve(d->eh, d->es, nullptr, &len, st) != NVJ_SUCCESS)
      return dfail(d, JDE_ERR_CUDA, "bitstream size of frame %d", i);
    if (cudaStreamSynchronize(st) != cudaSuccess) return dfail(d, JDE_ERR_CUDA, "encode synchronisation");
    if (len > lengths[i]) {
      lengths[i] = len;
      return dfail(d, JDE_ERR_CAPACITY, "frame %d needs %zu bytes", i, len);
    }
    if (nv.retrieve(d->eh, d->es, out[i], &len, st) != NVJ_SUCCESS)
      return dfail(d, JDE_ERR_CUDA, "bitstream of frame %d", i);
    if (cudaStreamSynchronize(st) != cudaSuccess) return dfail(d, JDE_ERR_CUDA, "encode synchronisation");
    lengths[i] = len;
  }
  return JDE_OK;
}

}  // extern "C"
