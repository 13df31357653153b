// Letterbox resize of uint8 RGB frames to the network input.
//
// Geometry (the paper only states FullHD input, Sec. 5.1): r = min(dst_w/src_w,
// dst_h/src_h); the image is resized to floor(src r + 0.5) on each axis,
// centred (pad = floor((dst - new)/2) on the left/top), sampled bilinearly with
// half-pixel centres src = (dst + 0.5)/r - 0.5 clamped to the image, scaled by
// 1/255; the padding holds 0.5.  The per-column and per-row sample positions
// are computed once in double precision; the per-pixel blend is f32.
#include "internal.h"

namespace {

__global__ void tables_kernel(LbAxis* xs, LbAxis* ys, int src_w, int src_h, int dst_w, int dst_h, double r, int nw,
                              int nh, int px, int py) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < dst_w) {
    LbAxis a = {0, 0, 0.f, 0};
    const int d = i - px;
    if (d >= 0 && d < nw) {
      double s = (d + 0.5) / r - 0.5;
      s = fmin(fmax(s, 0.0), (double)(src_w - 1));
      const int i0 = (int)floor(s);
      a.i0 = i0;
      a.i1 = min(i0 + 1, src_w - 1);
      a.f = (float)(s - i0);
      a.inside = 1;
    }
    xs[i] = a;
  }
  if (i < dst_h) {
    LbAxis a = {0, 0, 0.f, 0};
    const int d = i - py;
    if (d >= 0 && d < nh) {
      double s = (d + 0.5) / r - 0.5;
      s = fmin(fmax(s, 0.0), (double)(src_h - 1));
      const int i0 = (int)floor(s);
      a.i0 = i0;
      a.i1 = min(i0 + 1, src_h - 1);
      a.f = (float)(s - i0);
      a.inside = 1;
    }
    ys[i] = a;
  }
}

__device__ __forceinline__ void sample(const uint8_t* img, int src_w, const LbAxis& ax, const LbAxis& ay,
                                       float (&v)[3]) {
  if (!(ax.inside && ay.inside)) {
    v[0] = v[1] = v[2] = 0.5f;
    return;
  }
  const uint8_t* r0 = img + (size_t)ay.i0 * src_w * 3;
  const uint8_t* r1 = img + (size_t)ay.i1 * src_w * 3;
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    const float p00 = r0[ax.i0 * 3 + ch], p01 = r0[ax.i1 * 3 + ch];
    const float p10 = r1[ax.i0 * 3 + ch], p11 = r1[ax.i1 * 3 + ch];
    const float top = p00 * (1.f - ax.f) + p01 * ax.f;
    const float bot = p10 * (1.f - ax.f) + p11 * ax.f;
    v[ch] = (top * (1.f - ay.f) + bot * ay.f) / 255.f;
  }
}

// f32, 3 channels, into the interior of a haloed view
__global__ void letterbox_f32_kernel(const uint8_t* frames, int n, int src_w, int src_h, const LbAxis* xs,
                                     const LbAxis* ys, TView out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)n * out.h * out.w;
  if (idx >= total) return;
  const int x = (int)(idx % out.w);
  const int y = (int)((idx / out.w) % out.h);
  const int f = (int)(idx / ((long long)out.w * out.h));
  float v[3];
  sample(frames + (size_t)f * src_w * src_h * 3, src_w, xs[x], ys[y], v);
  float* o = static_cast<float*>(out.ptr) + tview_off(out, f, y, x);
  o[0] = v[0];
  o[1] = v[1];
  o[2] = v[2];
}

// bf16, 4 channels (RGB, 0), 8 bytes per pixel, into the interior of a haloed view
__global__ void letterbox_bf16x4_kernel(const uint8_t* frames, int n, int src_w, int src_h, const LbAxis* xs,
                                        const LbAxis* ys, TView out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)n * out.h * out.w;
  if (idx >= total) return;
  const int x = (int)(idx % out.w);
  const int y = (int)((idx / out.w) % out.h);
  const int f = (int)(idx / ((long long)out.w * out.h));
  float v[3];
  sample(frames + (size_t)f * src_w * src_h * 3, src_w, xs[x], ys[y], v);
  __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]);
  __nv_bfloat162 b = __floats2bfloat162_rn(v[2], 0.f);
  uint2 q = make_uint2(*reinterpret_cast<uint32_t*>(&a), *reinterpret_cast<uint32_t*>(&b));
  *reinterpret_cast<uint2*>(static_cast<__nv_bfloat16*>(out.ptr) + tview_off(out, f, y, x)) = q;
}

// bf16 RGB0 as above, one block per (output row, frame): the block copies the two source rows the
// output row samples into shared memory with coalesced loads (16-byte, 4-byte or 1-byte units, the
// widest that every source row's start allows), then blends its pixels from there.  The arithmetic is
// sample()'s, term for term.
constexpr int LB_THREADS = 256;

__global__ void __launch_bounds__(LB_THREADS) letterbox_bf16x4_rows_kernel(const uint8_t* frames, int src_w,
                                                                           int src_h, const LbAxis* xs,
                                                                           const LbAxis* ys, TView out, int unit) {
  extern __shared__ __align__(16) uint8_t srow[];   // [2][row_bytes]
  const int f = blockIdx.y, y = blockIdx.x;
  const LbAxis ay = ys[y];
  __nv_bfloat16* const o = static_cast<__nv_bfloat16*>(out.ptr);
  const int row_bytes = src_w * 3;
  if (ay.inside) {
    const uint8_t* img = frames + (size_t)f * src_w * src_h * 3;
    const uint8_t* rows[2] = {img + (size_t)ay.i0 * row_bytes, img + (size_t)ay.i1 * row_bytes};
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      uint8_t* dst = srow + r * row_bytes;
      if (unit == 16) {
        const uint4* src = reinterpret_cast<const uint4*>(rows[r]);
        for (int w = threadIdx.x; w < row_bytes / 16; w += LB_THREADS)
          reinterpret_cast<uint4*>(dst)[w] = __ldg(src + w);
      } else if (unit == 4) {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(rows[r]);
        for (int w = threadIdx.x; w < row_bytes / 4; w += LB_THREADS)
          reinterpret_cast<uint32_t*>(dst)[w] = __ldg(src + w);
      } else {
        for (int b = threadIdx.x; b < row_bytes; b += LB_THREADS) dst[b] = __ldg(rows[r] + b);
      }
    }
  }
  __syncthreads();
  for (int x = threadIdx.x; x < out.w; x += LB_THREADS) {
    float v[3];
    const LbAxis ax = xs[x];
    if (!(ax.inside && ay.inside)) {
      v[0] = v[1] = v[2] = 0.5f;
    } else {
      const uint8_t* r0 = srow;
      const uint8_t* r1 = srow + row_bytes;
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        const float p00 = r0[ax.i0 * 3 + ch], p01 = r0[ax.i1 * 3 + ch];
        const float p10 = r1[ax.i0 * 3 + ch], p11 = r1[ax.i1 * 3 + ch];
        const float top = p00 * (1.f - ax.f) + p01 * ax.f;
        const float bot = p10 * (1.f - ax.f) + p11 * ax.f;
        v[ch] = (top * (1.f - ay.f) + bot * ay.f) / 255.f;
      }
    }
    __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]);
    __nv_bfloat162 b = __floats2bfloat162_rn(v[2], 0.f);
    *reinterpret_cast<uint2*>(o + tview_off(out, f, y, x)) =
        make_uint2(*reinterpret_cast<uint32_t*>(&a), *reinterpret_cast<uint32_t*>(&b));
  }
}

}  // namespace

void letterbox_tables_launch(LbAxis* xs, LbAxis* ys, int src_w, int src_h, int dst_w, int dst_h, double r, int nw,
                             int nh, int px, int py, cudaStream_t st) {
  const int n = dst_w > dst_h ? dst_w : dst_h;
  jde_count_launch();
  tables_kernel<<<(n + 255) / 256, 256, 0, st>>>(xs, ys, src_w, src_h, dst_w, dst_h, r, nw, nh, px, py);
}

void letterbox_f32_launch(const uint8_t* frames, int n, int src_w, int src_h, const LbAxis* xs, const LbAxis* ys,
                          TView out, cudaStream_t st) {
  const long long total = (long long)n * out.h * out.w;
  jde_count_launch();
  letterbox_f32_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(frames, n, src_w, src_h, xs, ys, out);
}

void letterbox_bf16x4_launch(const uint8_t* frames, int n, int src_w, int src_h, const LbAxis* xs,
                             const LbAxis* ys, TView out, cudaStream_t st) {
  // the row kernel holds two whole source rows in shared memory (up to 48 KB: src_w <= 8192)
  const size_t smem = (size_t)2 * src_w * 3;
  jde_count_launch();
  if (smem <= 48 * 1024 && out.h <= 65535 && n <= 65535) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(frames);
    const size_t rb = (size_t)src_w * 3;
    const int unit = (a % 16 == 0 && rb % 16 == 0) ? 16 : (a % 4 == 0 && rb % 4 == 0) ? 4 : 1;
    dim3 grid((unsigned)out.h, (unsigned)n);
    letterbox_bf16x4_rows_kernel<<<grid, LB_THREADS, smem, st>>>(frames, src_w, src_h, xs, ys, out, unit);
    return;
  }
  const long long total = (long long)n * out.h * out.w;
  letterbox_bf16x4_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(frames, n, src_w, src_h, xs, ys, out);
}
