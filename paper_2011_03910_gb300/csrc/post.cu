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
// One block (two warps) per 64-row block of a frame's sorted candidates, looping over the column blocks
// at or right of the diagonal that hold candidates: lane r of a warp holds row r's box and, per column
// block, columns lane and lane + 32; for each of the warp's 32 rows the row box is broadcast and two
// ballots give the row's 64-bit word (bit u: column cb * 64 + u comes later and overlaps it by IoU > thr),
// which lane r keeps and stores.
__global__ void __launch_bounds__(64) nms_mask_kernel(const float4* boxes, const int* n_sorted, int kmax, float thr,
                                                      unsigned long long* mask) {
  const int n = blockIdx.y, rb = blockIdx.x;
  const int K = n_sorted[n];
  if (rb * 64 >= K) return;
  const int nb = (K + 63) / 64, words = kmax / 64;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float4* bx = boxes + (size_t)n * kmax;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  const int row0 = rb * 64 + 32 * warp;
  const int i_lane = row0 + lane;
  const float4 mine = i_lane < K ? bx[i_lane] : zero;
  const int rows = min(32, K - row0);   // warp-uniform; <= 0 for an empty half block
  unsigned long long* out = mask + ((size_t)n * kmax + i_lane) * words;
  for (int cb = rb; cb < nb; ++cb) {
    const int j0 = cb * 64 + lane, j1 = j0 + 32;
    const float4 c0 = j0 < K ? bx[j0] : zero, c1 = j1 < K ? bx[j1] : zero;
    unsigned long long word = 0;
    for (int r = 0; r < rows; ++r) {
      const int i = row0 + r;
      float4 bi;
      bi.x = __shfl_sync(0xffffffffu, mine.x, r);
      bi.y = __shfl_sync(0xffffffffu, mine.y, r);
      bi.z = __shfl_sync(0xffffffffu, mine.z, r);
      bi.w = __shfl_sync(0xffffffffu, mine.w, r);
      const unsigned lo = __ballot_sync(0xffffffffu, j0 < K && j0 > i && iou_above(bi, c0, thr));
      const unsigned hi = __ballot_sync(0xffffffffu, j1 < K && j1 > i && iou_above(bi, c1, thr));
      if (lane == r) word = ((unsigned long long)hi << 32) | lo;
    }
    if (i_lane < K) out[cb] = word;
  }
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
  // sparse head (e0 null): the raw embedding was written into the row by emb_tc_kernel
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

// Sparse embedding head, step 2 (tensor cores): for the listed detections of scale blockIdx.z,
// out[o] = sum_k W[o][k] x[k] over K = (tap, channel) of the 3x3 input patch around (y, x), times the
// E4M3 dequantisation multiplier, plus the bias; the raw (unnormalised) values go into the
// detection's row.  One CTA computes 128 detections x 256 outputs (blockIdx.y: which half of 512):
//   * warps 0..3 gather, per k-block (one 128-byte slice of one tap: 64 bf16 or 128 E4M3 channels),
//     each detection's input row into a 128-byte-swizzled A tile; warp 0 / lane 0 loads the weight
//     tile (256 output rows x 128 bytes) with TMA; a 4-deep ring;
//   * warp 4 / lane 0 issues tcgen05.mma (M = 128, N = 256, K = 16 bf16 or 32 E4M3) into a TMEM
//     accumulator and frees ring slots with tcgen05.commit;
//   * warps 4..7 read the accumulator rows (TMEM lane = detection) and write the row values.
// Waits are bounded; on a timeout the CTA flags the error word and stops.
constexpr int EMB_M = 128, EMB_N = 256, EMB_STAGES = 4;
constexpr int EMB_A_BYTES = EMB_M * 128, EMB_B_BYTES = EMB_N * 128;
constexpr int EMB_SMEM = EMB_STAGES * (EMB_A_BYTES + EMB_B_BYTES) + 1024 + 256;

struct EmbMaps {
  alignas(64) CUtensorMap w[3];   // weights [512][K] of each scale, boxes {128 bytes of K, 256 rows}
};
struct EmbArgs {
  EmbSparse es;
  const int4* list;
  const int* count;
  int list_stride;
  float* rows;
  int cap;
  int* err;
};

template <int Q>
__global__ void __launch_bounds__(256, 1) emb_tc_kernel(const __grid_constant__ EmbMaps maps, const EmbArgs a) {
  const int sc = blockIdx.z, n0 = blockIdx.y * EMB_N, d0 = blockIdx.x * EMB_M;
  const int total = a.count[sc];
  if (d0 >= total) return;   // the whole CTA
  extern __shared__ uint8_t smem_raw[];
  __shared__ int s_abort;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + EMB_STAGES * EMB_A_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + EMB_STAGES * (EMB_A_BYTES + EMB_B_BYTES));
  uint64_t* empty = full + EMB_STAGES;
  uint64_t* acc_full = empty + EMB_STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_full + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const TView in = a.es.in[sc];
  const int cin = a.es.cin[sc];
  constexpr int KEL = Q ? 128 : 64;          // elements of one 128-byte k-block
  constexpr int ES = Q ? 1 : 2;              // bytes per element
  const int nkb = 9 * cin / KEL;
  if (threadIdx.x == 0) {
    for (int i = 0; i < EMB_STAGES; ++i) {
      mbar_init(&full[i], 5);                // four gather warps + the weight load
      mbar_init(&empty[i], 1);
    }
    mbar_init(acc_full, 1);
    fence_barrier_init();
    s_abort = 0;
  }
  if (warp == 4) tmem_alloc(tmem_slot, EMB_N);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp < 4) {
    // ---------------- gather: detection row t of the tile, one 128-byte k-block slice per stage
    const int t = threadIdx.x;
    const int det = d0 + t;
    int4 e = make_int4(-1, 0, 0, 0);
    if (det < total) e = a.list[(size_t)sc * a.list_stride + det];
    for (int kb = 0; kb < nkb; ++kb) {
      const int st = kb % EMB_STAGES;
      bool ok = true;
      if (lane == 0 && kb >= EMB_STAGES) ok = mbar_wait(&empty[st], ((kb / EMB_STAGES) - 1) & 1);
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (!ok || *((volatile int*)&s_abort)) {
        if (lane == 0) {
          flag_error(a.err, KERR_TIMEOUT);
          atomicExch(&s_abort, 1);
        }
        break;
      }
      if (threadIdx.x == 0) {
        mbar_expect_tx(&full[st], EMB_B_BYTES);
        tma_load_2d(sB + st * EMB_B_BYTES, &maps.w[sc], &full[st], kb * KEL, n0);
      }
      const int k0 = kb * KEL, tap = k0 / cin, c0 = k0 - tap * cin;
      uint4 v[8];
      if (e.x >= 0) {
        const uint8_t* src = static_cast<const uint8_t*>(in.ptr) +
                             (tview_off(in, e.x, e.z + tap / 3 - 1, e.w + tap % 3 - 1) + c0) * ES;
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldg(reinterpret_cast<const uint4*>(src) + u);
      } else {
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = make_uint4(0u, 0u, 0u, 0u);
      }
      uint8_t* dst = sA + st * EMB_A_BYTES + t * 128;
#pragma unroll
      for (int u = 0; u < 8; ++u) *reinterpret_cast<uint4*>(dst + ((u ^ (t & 7)) << 4)) = v[u];
      fence_proxy_async();                   // generic-proxy writes -> visible to the MMAs
      __syncwarp();
      if (lane == 0) mbar_arrive(&full[st]);
    }
  } else {
    if (warp == 4 && lane == 0) {
      // ---------------- MMA issuer
      constexpr uint32_t idesc = Q ? idesc_e4m3(EMB_M, EMB_N) : idesc_bf16(EMB_M, EMB_N);
      const uint64_t a0 = smem_desc(smem_u32(sA), 1024, 2u);   // 128-byte rows, 128-byte swizzle
      const uint64_t b0 = smem_desc(smem_u32(sB), 1024, 2u);
      bool ok = true;
      for (int kb = 0; kb < nkb; ++kb) {
        const int st = kb % EMB_STAGES;
        if (!mbar_wait(&full[st], (kb / EMB_STAGES) & 1)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint64_t ad = desc_add(a0, (uint32_t)(st * EMB_A_BYTES) >> 4);
        const uint64_t bd = desc_add(b0, (uint32_t)(st * EMB_B_BYTES) >> 4);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {     // 32 bytes of K per MMA
          if (Q)
            umma_e4m3(tmem, desc_add(ad, 2 * kk), desc_add(bd, 2 * kk), idesc, (kb | kk) != 0 ? 1u : 0u);
          else
            umma_bf16(tmem, desc_add(ad, 2 * kk), desc_add(bd, 2 * kk), idesc, (kb | kk) != 0 ? 1u : 0u);
        }
        umma_commit(&empty[st]);
      }
      umma_commit(acc_full);
      if (!ok) {
        flag_error(a.err, KERR_TIMEOUT);
        atomicExch(&s_abort, 1);
      }
    }
    // ---------------- epilogue: TMEM lane = detection row of the tile
    __syncwarp();
    const int quarter = warp & 3;
    const int t = quarter * 32 + lane;
    const int det = d0 + t;
    bool ok = lane == 0 ? mbar_wait(acc_full, 0) : true;
    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    if (!ok && lane == 0) flag_error(a.err, KERR_TIMEOUT);
    tc_fence_after();
    float* row = nullptr;
    if (det < total && ok && !*((volatile int*)&s_abort)) {
      const int4 e = a.list[(size_t)sc * a.list_stride + det];
      row = a.rows + ((size_t)e.x * a.cap + e.y) * 518 + 6 + n0;
    }
#pragma unroll 1
    for (int c0 = 0; c0 < EMB_N; c0 += 32) {
      uint32_t r[32];
      tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0, r);
      tmem_ld_wait();
      if (row) {
#pragma unroll
        for (int j = 0; j < 32; j += 2) {
          const int o = n0 + c0 + j;
          float v0 = __uint_as_float(r[j]), v1 = __uint_as_float(r[j + 1]);
          if (Q) {
            v0 *= a.es.mult[sc][o];
            v1 *= a.es.mult[sc][o + 1];
          }
          // rows are 518 floats: 8-byte aligned only
          reinterpret_cast<float2*>(row + c0 + j)[0] = make_float2(v0 + a.es.bias[sc][o], v1 + a.es.bias[sc][o + 1]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 4) tmem_dealloc(tmem, EMB_N);
}

typedef CUresult (*EmbEncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Weight tensor maps of the three scales; false if the driver entry point or an encoding fails.
bool emb_maps(const EmbSparse& es, EmbMaps& m) {
  static EmbEncodeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EmbEncodeFn>(p);
  });
  if (!fn) return false;
  for (int sc = 0; sc < 3; ++sc) {
    const int es_b = es.q[sc] ? 1 : 2;
    const cuuint64_t K = (cuuint64_t)es.ldw[sc];
    cuuint64_t dims[2] = {K, 512};
    cuuint64_t strides[1] = {K * es_b};
    cuuint32_t box[2] = {(cuuint32_t)(128 / es_b), EMB_N};
    cuuint32_t el[2] = {1, 1};
    if (fn(&m.w[sc], es.q[sc] ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
           const_cast<void*>(es.w[sc]), dims, strides, box, el, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

}  // namespace

cudaError_t post_launch(const float* const* heads, const HeadGeom& g, float conf_thresh, float nms_iou, PostBufs& b,
                        float* rows, int32_t* count, int32_t* anchor_index, int cap, int* err, cudaStream_t st,
                        const EmbSparse* es) {
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
  dim3 gm(b.kmax / 64, n);
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
    const int gx = (per + EMB_M - 1) / EMB_M;
    EmbMaps maps;
    EmbArgs ea;
    ea.es = *es;
    ea.list = b.emb_list;
    ea.count = b.emb_count;
    ea.list_stride = n * b.kmax;
    ea.rows = rows;
    ea.cap = cap;
    ea.err = err;
    if (emb_maps(*es, maps)) {
      {
        // dynamic shared-memory limit of the two instantiations, once per device
        static std::mutex mu;
        static bool attr[JDE_MAX_DEVICES] = {false};
        int dev = -1;
        if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < JDE_MAX_DEVICES) {
          std::lock_guard<std::mutex> lock(mu);
          if (!attr[dev] &&
              cudaFuncSetAttribute(emb_tc_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, EMB_SMEM) ==
                  cudaSuccess &&
              cudaFuncSetAttribute(emb_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, EMB_SMEM) ==
                  cudaSuccess)
            attr[dev] = true;
        }
      }
      jde_count_launch();
      // the three heads of a handle are all BF16 or all E4M3
      if (es->q[0])
        emb_tc_kernel<1><<<dim3(gx, 512 / EMB_N, 3), 256, EMB_SMEM, st>>>(maps, ea);
      else
        emb_tc_kernel<0><<<dim3(gx, 512 / EMB_N, 3), 256, EMB_SMEM, st>>>(maps, ea);
    } else {
      return cudaErrorInvalidValue;   // the weight tensor maps could not be built
    }
  }
  dim3 ge((b.kmax + 3) / 4, n);
  jde_count_launch();
  emit_kernel<<<ge, 128, 0, st>>>(es ? nullptr : heads[3], heads[4], heads[5], g, b.sorted, b.boxes, b.conf, b.cls,
                                  b.keep_idx, b.n_keep, b.kmax, rows, count, anchor_index, cap);
  return cudaGetLastError();
}
