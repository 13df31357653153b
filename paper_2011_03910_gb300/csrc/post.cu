// Post-processing of the JDE heads (Sec. 3.2, Appendix A items 1-3):
// anchor decode, confidence filter, sort, greedy NMS, embedding gather + L2.
//
// Decode (YOLOv3 manner, Sec. 3.1): anchor a of head s at cell (y, x) uses
// channels 6a..6a+5 = (tx, ty, tw, th, t_obj, t_cls):
//   cx = (x + sigmoid(tx)) * stride, cy = (y + sigmoid(ty)) * stride,
//   w = anchor_w * exp(clamp(tw, -10, 10)), h = anchor_h * exp(clamp(th, -10, 10)),
//   conf = sigmoid(t_obj), cls = sigmoid(t_cls); box xyxy in letterbox pixels.
// Canonical anchor index g = off_s + (a * H_s + y) * W_s + x, heads ordered by
// stride 32, 16, 8.  Candidates (conf >= threshold) are ordered by conf
// descending then g ascending through one 64-bit key per candidate:
// key = (~bits(conf)) << 32 | g, sorted ascending.  At most kmax survive.
// NMS: bit j of mask word (i, j/64) says IoU(i, j) > threshold for j > i in
// sorted order; one warp per frame then scans the rows in order, keeping a row
// unless an earlier kept row suppressed it - exactly the greedy result.
#include <mutex>

#include "internal.h"

namespace {

constexpr int SORT_CAP = 8192;   // candidates sorted in shared memory without pre-selection

__device__ __forceinline__ float sigm(float t) { return 1.f / (1.f + expf(-t)); }

__device__ __forceinline__ void locate(const HeadGeom& g, int gi, int& s, int& a, int& y, int& x) {
  s = gi < g.off[1] ? 0 : (gi < g.off[2] ? 1 : 2);
  int l = gi - g.off[s];
  x = l % g.gw[s];
  l /= g.gw[s];
  y = l % g.gh[s];
  a = l / g.gh[s];
}

__global__ void filter_kernel(const float* d0, const float* d1, const float* d2, HeadGeom g, float thr,
                              uint64_t* keys, int* count, int cap) {
  const int n = blockIdx.y;
  const int gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= g.off[3]) return;
  int s, a, y, x;
  locate(g, gi, s, a, y, x);
  const float* d = s == 0 ? d0 : (s == 1 ? d1 : d2);
  const float t = d[((size_t)(n * g.gh[s] + y) * g.gw[s] + x) * 24 + 6 * a + 4];
  const float conf = sigm(t);
  if (conf >= thr) {
    const int slot = atomicAdd(&count[n], 1);
    if (slot < cap) keys[(size_t)n * cap + slot] = ((uint64_t)(~__float_as_uint(conf)) << 32) | (uint32_t)gi;
  }
}

__device__ void bitonic_sort(uint64_t* s, int P) {
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const bool up = (i & k) == 0;
          const uint64_t a = s[i], b = s[ixj];
          if ((a > b) == up) {
            s[i] = b;
            s[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
}

// One CTA per frame: sort the candidates (or select the kmax smallest keys by
// an 8-pass radix select first when there are more than SORT_CAP).
__global__ void __launch_bounds__(1024) select_sort_kernel(const uint64_t* keys, const int* count, int cap,
                                                           uint64_t* sorted, int* n_sorted, int kmax) {
  extern __shared__ uint64_t s[];
  __shared__ unsigned hist[256];
  __shared__ uint64_t s_prefix, s_mask;
  __shared__ int s_rank, s_cnt;
  const int n = blockIdx.x;
  const uint64_t* kin = keys + (size_t)n * cap;
  const int C = min(count[n], cap);
  int use;
  if (C <= SORT_CAP) {
    int P = 1;
    while (P < C) P <<= 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x) s[i] = i < C ? kin[i] : ~0ull;
    __syncthreads();
    bitonic_sort(s, P);
    use = min(C, kmax);
  } else {
    if (threadIdx.x == 0) {
      s_prefix = 0;
      s_mask = 0;
      s_rank = kmax - 1;
      s_cnt = 0;
    }
    __syncthreads();
    for (int pass = 0; pass < 8; ++pass) {
      const int shift = 56 - 8 * pass;
      for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
      __syncthreads();
      const uint64_t pre = s_prefix, msk = s_mask;
      for (int i = threadIdx.x; i < C; i += blockDim.x) {
        const uint64_t k = kin[i];
        if ((k & msk) == pre) atomicAdd(&hist[(k >> shift) & 255], 1u);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        unsigned cum = 0;
        int rank = s_rank;
        for (int d = 0; d < 256; ++d) {
          if (cum + hist[d] > (unsigned)rank) {
            s_prefix = pre | ((uint64_t)d << shift);
            s_rank = rank - (int)cum;
            break;
          }
          cum += hist[d];
        }
        s_mask = msk | (0xFFull << shift);
      }
      __syncthreads();
    }
    const uint64_t kth = s_prefix;
    for (int i = threadIdx.x; i < C; i += blockDim.x) {
      const uint64_t k = kin[i];
      if (k <= kth) {
        const int p = atomicAdd(&s_cnt, 1);
        if (p < kmax) s[p] = k;
      }
    }
    __syncthreads();
    int P = 1;
    while (P < kmax) P <<= 1;
    for (int i = kmax + threadIdx.x; i < P; i += blockDim.x) s[i] = ~0ull;
    __syncthreads();
    bitonic_sort(s, P);
    use = kmax;
  }
  for (int i = threadIdx.x; i < use; i += blockDim.x) sorted[(size_t)n * kmax + i] = s[i];
  if (threadIdx.x == 0) n_sorted[n] = use;
}

__global__ void prep_kernel(const float* d0, const float* d1, const float* d2, HeadGeom g, const uint64_t* sorted,
                            const int* n_sorted, int kmax, float4* boxes, float* conf, float* cls) {
  const int n = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_sorted[n]) return;
  const int gi = (int)(sorted[(size_t)n * kmax + i] & 0xFFFFFFFFu);
  int s, a, y, x;
  locate(g, gi, s, a, y, x);
  const float* d = (s == 0 ? d0 : (s == 1 ? d1 : d2)) + ((size_t)(n * g.gh[s] + y) * g.gw[s] + x) * 24 + 6 * a;
  const float st = (float)g.stride[s];
  const float cx = ((float)x + sigm(d[0])) * st;
  const float cy = ((float)y + sigm(d[1])) * st;
  const float w = g.anchor_w[s * 4 + a] * expf(fminf(fmaxf(d[2], -10.f), 10.f));
  const float h = g.anchor_h[s * 4 + a] * expf(fminf(fmaxf(d[3], -10.f), 10.f));
  const size_t o = (size_t)n * kmax + i;
  boxes[o] = make_float4(cx - w / 2.f, cy - h / 2.f, cx + w / 2.f, cy + h / 2.f);
  conf[o] = sigm(d[4]);
  cls[o] = sigm(d[5]);
}

__device__ __forceinline__ bool iou_above(const float4& a, const float4& b, float thr) {
  const float iw = fmaxf(0.f, fminf(a.z, b.z) - fmaxf(a.x, b.x));
  const float ih = fmaxf(0.f, fminf(a.w, b.w) - fmaxf(a.y, b.y));
  const float inter = iw * ih;
  const float uni = (a.z - a.x) * (a.w - a.y) + (b.z - b.x) * (b.w - b.y) - inter;
  const float iou = uni > 0.f ? inter / uni : 0.f;
  return iou > thr;
}

// grid (col block, row block, frame), 64 threads: row i = rb*64 + t against columns cb*64 .. +63
__global__ void nms_mask_kernel(const float4* boxes, const int* n_sorted, int kmax, float thr,
                                unsigned long long* mask) {
  const int n = blockIdx.z, rb = blockIdx.y, cb = blockIdx.x;
  const int K = n_sorted[n];
  if (cb < rb || rb * 64 >= K || cb * 64 >= K) return;
  __shared__ float4 cols[64];
  const int t = threadIdx.x;
  const float4* bx = boxes + (size_t)n * kmax;
  if (cb * 64 + t < K) cols[t] = bx[cb * 64 + t];
  __syncthreads();
  const int i = rb * 64 + t;
  if (i >= K) return;
  const float4 bi = bx[i];
  unsigned long long word = 0;
  const int jend = min(64, K - cb * 64);
  for (int u = 0; u < jend; ++u) {
    const int j = cb * 64 + u;
    if (j > i && iou_above(bi, cols[u], thr)) word |= 1ull << u;
  }
  mask[((size_t)n * kmax + i) * (kmax / 64) + cb] = word;
}

// one warp per frame: greedy scan of the bitmask in sorted order
__global__ void nms_scan_kernel(const unsigned long long* mask, const int* n_sorted, int kmax, int* keep_idx,
                                int* n_keep, int nframes) {
  extern __shared__ unsigned long long removed_all[];
  const int warps = blockDim.x / 32;
  const int wid = threadIdx.x / 32, lane = threadIdx.x & 31;
  const int n = blockIdx.x * warps + wid;
  const int words = kmax / 64;
  unsigned long long* removed = removed_all + wid * words;
  for (int i = lane; i < words; i += 32) removed[i] = 0;
  __syncwarp();
  if (n >= nframes) return;
  const int K = n_sorted[n];
  const int nb = (K + 63) / 64;
  const unsigned long long* m = mask + (size_t)n * kmax * words;
  int nkeep = 0;
  for (int b = 0; b < nb; ++b) {
    const int i0 = b * 64 + lane, i1 = i0 + 32;
    const unsigned long long d0 = i0 < K ? m[(size_t)i0 * words + b] : 0ull;
    const unsigned long long d1 = i1 < K ? m[(size_t)i1 * words + b] : 0ull;
    unsigned long long w = removed[b];
    const int rows = min(64, K - b * 64);
    unsigned long long kept = 0;
    for (int t = 0; t < rows; ++t) {
      const unsigned long long src = t < 32 ? d0 : d1;
      const unsigned long long dm = __shfl_sync(0xffffffffu, src, t & 31);
      if (!((w >> t) & 1ull)) {
        kept |= 1ull << t;
        w |= dm;
      }
    }
    // kept rows in order
    if (lane == 0) {
      unsigned long long kb = kept;
      while (kb) {
        const int t = __ffsll((long long)kb) - 1;
        kb &= kb - 1;
        keep_idx[(size_t)n * kmax + nkeep++] = b * 64 + t;
      }
    }
    nkeep = __shfl_sync(0xffffffffu, nkeep, 0);
    for (int bb = b + 1 + lane; bb < nb; bb += 32) {
      unsigned long long acc = removed[bb];
      unsigned long long kb = kept;
      while (kb) {
        const int t = __ffsll((long long)kb) - 1;
        kb &= kb - 1;
        acc |= m[(size_t)(b * 64 + t) * words + bb];
      }
      removed[bb] = acc;
    }
    __syncwarp();
  }
  if (lane == 0) n_keep[n] = nkeep;
}

// one warp per kept detection: row = box (frame px), conf, cls, unit embedding
__global__ void emit_kernel(const float* e0, const float* e1, const float* e2, HeadGeom g, const uint64_t* sorted,
                            const float4* boxes, const float* conf, const float* cls, const int* keep_idx,
                            const int* n_keep, int kmax, float* rows, int32_t* count, int32_t* anchor_index, int cap) {
  const int n = blockIdx.y;
  const int r = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  const int nk = n_keep[n];
  if (r == 0 && lane == 0) count[n] = nk;
  if (r >= nk || r >= cap) return;
  const int p = keep_idx[(size_t)n * kmax + r];
  const size_t o = (size_t)n * kmax + p;
  const int gi = (int)(sorted[o] & 0xFFFFFFFFu);
  int s, a, y, x;
  locate(g, gi, s, a, y, x);
  float* row = rows + ((size_t)n * cap + r) * 518;
  const int ep = g.epad;
  // sparse head (e0 null): the raw embedding was written into the row by emb_gemm_kernel
  const float* e = e0 == nullptr ? row + 6
                                 : (s == 0 ? e0 : (s == 1 ? e1 : e2)) +
                                       ((size_t)(n * (g.gh[s] + 2 * ep) + y + ep) * (g.gw[s] + 2 * ep) + x + ep) * 512;
  float v[16];
  float ss = 0.f;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float2 t = *reinterpret_cast<const float2*>(e + q * 64 + lane * 2);
    v[2 * q] = t.x;
    v[2 * q + 1] = t.y;
    ss += t.x * t.x + t.y * t.y;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, off);
  const float nrm = sqrtf(ss);
  const float inv = nrm > 0.f ? 1.f / nrm : 0.f;
#pragma unroll
  for (int q = 0; q < 8; ++q)
    *reinterpret_cast<float2*>(row + 6 + q * 64 + lane * 2) = make_float2(v[2 * q] * inv, v[2 * q + 1] * inv);
  if (lane == 0) {
    const float4 b = boxes[o];
    row[0] = (b.x - g.pad_x) / g.ratio;
    row[1] = (b.y - g.pad_y) / g.ratio;
    row[2] = (b.z - g.pad_x) / g.ratio;
    row[3] = (b.w - g.pad_y) / g.ratio;
    row[4] = conf[o];
    row[5] = cls[o];
    if (anchor_index) anchor_index[(size_t)n * cap + r] = gi;
  }
}

// Sparse embedding head, step 1: the kept detections of every frame, listed per scale as
// (frame, row, y, x).
__global__ void emb_list_kernel(HeadGeom g, const uint64_t* sorted, const int* keep_idx, const int* n_keep, int kmax,
                                int cap, int4* list, int* count) {
  const int n = blockIdx.x;
  const int nk = min(n_keep[n], cap);
  for (int r = threadIdx.x; r < nk; r += blockDim.x) {
    const int p = keep_idx[(size_t)n * kmax + r];
    const int gi = (int)(sorted[(size_t)n * kmax + p] & 0xFFFFFFFFu);
    int s, a, y, x;
    locate(g, gi, s, a, y, x);
    const int slot = atomicAdd(&count[s], 1);
    list[(size_t)s * g.n * kmax + slot] = make_int4(n, r, y, x);
  }
}

__device__ __forceinline__ float e4m3_value(uint8_t code) { return e4m3x2_to_float2((uint32_t)code).x; }

// Sparse embedding head, step 2: for the listed detections of scale blockIdx.z, out[o] = sum_k
// W[o][k] x[k] over K = (tap, channel) of the 3x3 input patch around (y, x), times the E4M3
// dequantisation multiplier, plus the bias; the raw (unnormalised) values go into the detection's
// row.  Tiles of 64 detections x 128 outputs (8 x 4 per thread), fp32 accumulation, K in chunks
// of 32 channels of one tap, operands read with 16-byte loads.
constexpr int EG_D = 64, EG_O = 128, EG_K = 32;
// 16 bytes -> 8 bf16 values, or 16 E4M3 codes (Q)
template <int Q>
__device__ __forceinline__ void unpack16b(const uint4 v, float (&out)[16]) {
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
  if (Q) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 lo = e4m3x2_to_float2(w[i] & 0xFFFFu), hi = e4m3x2_to_float2(w[i] >> 16);
      out[4 * i] = lo.x;
      out[4 * i + 1] = lo.y;
      out[4 * i + 2] = hi.x;
      out[4 * i + 3] = hi.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[i]));
      out[2 * i] = f.x;
      out[2 * i + 1] = f.y;
    }
  }
}
template <int Q>
__global__ void __launch_bounds__(256) emb_gemm_kernel(EmbSparse es, const int4* list, const int* count, int list_stride,
                                                       float* rows, int cap) {
  const int s = blockIdx.z;
  const int o0 = blockIdx.y * EG_O;
  const int total = count[s];
  const TView in = es.in[s];
  const int cin = es.cin[s], K = 9 * cin, ldw = es.ldw[s];
  constexpr int es_b = Q ? 1 : 2;             // bytes per element
  constexpr int vec = 16 / es_b;              // elements per 16-byte load
  __shared__ __align__(16) float As[EG_K][EG_D + 4];
  __shared__ __align__(16) float Bs[EG_K][EG_O + 4];
  __shared__ int4 ent[EG_D];
  const int t = threadIdx.x;
  const int td = (t / 32) * 8;                // 8 detections
  const int to = (t % 32) * 4;                // 4 outputs
  for (int d0 = blockIdx.x * EG_D; d0 < total; d0 += gridDim.x * EG_D) {
    __syncthreads();
    if (t < EG_D) ent[t] = d0 + t < total ? list[(size_t)s * list_stride + d0 + t] : make_int4(-1, -1, 0, 0);
    __syncthreads();
    float acc[8][4] = {};
    for (int k0 = 0; k0 < K; k0 += EG_K) {
      const int tap = k0 / cin, c0 = k0 % cin;
      const int ky = tap / 3, kx = tap % 3;
      // A: 64 detections x 32 channels of one tap
      for (int i = t; i < EG_D * (EG_K / vec); i += 256) {
        const int d = i / (EG_K / vec), part = i % (EG_K / vec);
        const int4 e = ent[d];
        float v[16];
        if (e.x >= 0) {
          const size_t off = tview_off(in, e.x, e.z + ky - 1, e.w + kx - 1) + c0 + part * vec;
          unpack16b<Q>(__ldg(reinterpret_cast<const uint4*>(static_cast<const uint8_t*>(in.ptr) + off * es_b)), v);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] = 0.f;
        }
#pragma unroll
        for (int j = 0; j < vec; ++j) As[part * vec + j][d] = v[j];
      }
      // B: 128 outputs x 32 K
      for (int i = t; i < EG_O * (EG_K / vec); i += 256) {
        const int o = i / (EG_K / vec), part = i % (EG_K / vec);
        const size_t off = (size_t)(o0 + o) * ldw + k0 + part * vec;
        float v[16];
        unpack16b<Q>(__ldg(reinterpret_cast<const uint4*>(static_cast<const uint8_t*>(es.w[s]) + off * es_b)), v);
#pragma unroll
        for (int j = 0; j < vec; ++j) Bs[part * vec + j][o] = v[j];
      }
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < EG_K; ++kk) {
        const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][td]);
        const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][td + 4]);
        const float4 b = *reinterpret_cast<const float4*>(&Bs[kk][to]);
        const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float bb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int4 e = ent[td + i];
      if (e.x < 0) continue;
      float* row = rows + ((size_t)e.x * cap + e.y) * 518 + 6;
      float v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int o = o0 + to + j;
        v[j] = acc[i][j] * (Q ? es.mult[s][o] : 1.f) + es.bias[s][o];
      }
      // rows are 518 floats: 8-byte aligned only
      reinterpret_cast<float2*>(row + o0 + to)[0] = make_float2(v[0], v[1]);
      reinterpret_cast<float2*>(row + o0 + to)[1] = make_float2(v[2], v[3]);
    }
  }
}

}  // namespace

void post_launch(const float* const* heads, const HeadGeom& g, float conf_thresh, float nms_iou, PostBufs& b,
                 float* rows, int32_t* count, int32_t* anchor_index, int cap, int* err, cudaStream_t st,
                 const EmbSparse* es) {
  (void)err;
  {
    // the kernel's dynamic shared-memory limit is a per-device attribute: set it once per device
    static std::mutex mu;
    static bool attr[JDE_MAX_DEVICES] = {false};
    int dev = -1;
    if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < JDE_MAX_DEVICES) {
      std::lock_guard<std::mutex> lock(mu);
      if (!attr[dev] && cudaFuncSetAttribute(select_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             SORT_CAP * (int)sizeof(uint64_t)) == cudaSuccess)
        attr[dev] = true;
    }
  }
  const int n = g.n;
  cudaMemsetAsync(b.cand_count, 0, sizeof(int) * n, st);
  dim3 gf((g.off[3] + 255) / 256, n);
  jde_count_launch();
  filter_kernel<<<gf, 256, 0, st>>>(heads[0], heads[1], heads[2], g, conf_thresh, b.cand_keys, b.cand_count,
                                    b.cand_cap);
  jde_count_launch();
  select_sort_kernel<<<n, 1024, SORT_CAP * sizeof(uint64_t), st>>>(b.cand_keys, b.cand_count, b.cand_cap, b.sorted,
                                                                   b.n_sorted, b.kmax);
  dim3 gp((b.kmax + 127) / 128, n);
  jde_count_launch();
  prep_kernel<<<gp, 128, 0, st>>>(heads[0], heads[1], heads[2], g, b.sorted, b.n_sorted, b.kmax, b.boxes, b.conf,
                                  b.cls);
  dim3 gm(b.kmax / 64, b.kmax / 64, n);
  jde_count_launch();
  nms_mask_kernel<<<gm, 64, 0, st>>>(b.boxes, b.n_sorted, b.kmax, nms_iou, b.mask);
  const int wpb = 4;
  jde_count_launch();
  nms_scan_kernel<<<(n + wpb - 1) / wpb, 32 * wpb, wpb * (b.kmax / 64) * sizeof(unsigned long long), st>>>(
      b.mask, b.n_sorted, b.kmax, b.keep_idx, b.n_keep, n);
  if (es) {
    cudaMemsetAsync(b.emb_count, 0, sizeof(int) * 3, st);
    jde_count_launch();
    emb_list_kernel<<<n, 256, 0, st>>>(g, b.sorted, b.keep_idx, b.n_keep, b.kmax, cap, b.emb_list, b.emb_count);
    const int per = n * (cap < b.kmax ? cap : b.kmax);   // most detections of one scale
    int gx = (per + EG_D - 1) / EG_D;
    if (gx > 64) gx = 64;
    jde_count_launch();
    // the three heads of a handle are all BF16 or all E4M3
    if (es->q[0])
      emb_gemm_kernel<1><<<dim3(gx, 512 / EG_O, 3), 256, 0, st>>>(*es, b.emb_list, b.emb_count, n * b.kmax, rows, cap);
    else
      emb_gemm_kernel<0><<<dim3(gx, 512 / EG_O, 3), 256, 0, st>>>(*es, b.emb_list, b.emb_count, n * b.kmax, rows, cap);
  }
  dim3 ge((b.kmax + 3) / 4, n);
  jde_count_launch();
  emit_kernel<<<ge, 128, 0, st>>>(es ? nullptr : heads[3], heads[4], heads[5], g, b.sorted, b.boxes, b.conf, b.cls,
                                  b.keep_idx, b.n_keep, b.kmax, rows, count, anchor_index, cap);
}
