// Plain FP32 implicit-GEMM convolution on the CUDA cores.
//
// GEMM view: M = output pixels (n, oy, ox), N = output channels, K = (ky, kx, ci).
// A[m][k] = in[n, oy*s + ky - p, ox*s + kx - p, ci] read from the zero-haloed
// input (p = k/2 <= halo, so no bounds checks are needed); B = packed weights
// [K_pad16][cout_pad64].  Epilogue: + bias, leaky-ReLU, + residual, store
// (optionally 2x2-replicated for the FPN upsample).  128x64 output tile per
// 256-thread CTA, 8x4 outputs per thread, BK = 16, double-buffered smem.
#include "internal.h"

namespace {

constexpr int BM = 128, BN = 64, BK = 16;

struct SimtArgs {
  ConvSpec c;
  const float* w;
  int ldw;      // cout_pad64
  int K;        // k*k*cin
  int M;        // n*Ho*Wo
};

template <bool VEC>
__device__ __forceinline__ void load_a(const SimtArgs& a, int m0, int k0, float (&ra)[8]) {
  const ConvSpec& c = a.c;
  const int tid = threadIdx.x;
  const float* base = static_cast<const float*>(c.in.ptr);
  const int p = c.k / 2;
  if (VEC) {
    // 16 consecutive k of one tap are 16 consecutive channels: row r = tid/2, half = tid%2.
    const int r = tid >> 1, half = tid & 1;
    const int m = m0 + r;
    const int tap = k0 / c.cin, ci = k0 % c.cin + half * 8;
    if (m < a.M) {
      const int hw = c.Ho * c.Wo;
      const int n = m / hw, rem = m % hw, oy = rem / c.Wo, ox = rem % c.Wo;
      const int ky = tap / c.k, kx = tap % c.k;
      const float* src = base + tview_off(c.in, n, oy * c.stride + ky - p, ox * c.stride + kx - p) + ci;
      const float4 v0 = *reinterpret_cast<const float4*>(src);
      const float4 v1 = *reinterpret_cast<const float4*>(src + 4);
      ra[0] = v0.x; ra[1] = v0.y; ra[2] = v0.z; ra[3] = v0.w;
      ra[4] = v1.x; ra[5] = v1.y; ra[6] = v1.z; ra[7] = v1.w;
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) ra[j] = 0.f;
    }
  } else {
    // generic: element e = tid + 256*j -> (r = e / BK, kk = e % BK)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int e = tid + 256 * j;
      const int r = e / BK, kk = e % BK;
      const int m = m0 + r, k = k0 + kk;
      float v = 0.f;
      if (m < a.M && k < a.K) {
        const int hw = c.Ho * c.Wo;
        const int n = m / hw, rem = m % hw, oy = rem / c.Wo, ox = rem % c.Wo;
        const int tap = k / c.cin, ci = k % c.cin;
        const int ky = tap / c.k, kx = tap % c.k;
        v = base[tview_off(c.in, n, oy * c.stride + ky - p, ox * c.stride + kx - p) + ci];
      }
      ra[j] = v;
    }
  }
}

template <bool VEC>
__device__ __forceinline__ void store_a(float (*As)[BM + 4], const float (&ra)[8]) {
  const int tid = threadIdx.x;
  if (VEC) {
    const int r = tid >> 1, half = tid & 1;
#pragma unroll
    for (int j = 0; j < 8; ++j) As[half * 8 + j][r] = ra[j];
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int e = tid + 256 * j;
      As[e % BK][e / BK] = ra[j];
    }
  }
}

template <bool VEC>
__global__ void __launch_bounds__(256) conv_simt_kernel(const SimtArgs a) {
  __shared__ __align__(16) float As[2][BK][BM + 4];
  __shared__ __align__(16) float Bs[2][BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int KT = (a.K + BK - 1) / BK;

  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

  float ra[8];
  float4 rb;
  const int brow = tid / 16, bcol = (tid % 16) * 4;
  load_a<VEC>(a, m0, 0, ra);
  rb = *reinterpret_cast<const float4*>(a.w + (size_t)brow * a.ldw + n0 + bcol);
  store_a<VEC>(As[0], ra);
  *reinterpret_cast<float4*>(&Bs[0][brow][bcol]) = rb;
  __syncthreads();

  for (int kt = 0; kt < KT; ++kt) {
    const int cur = kt & 1;
    if (kt + 1 < KT) {
      load_a<VEC>(a, m0, (kt + 1) * BK, ra);
      rb = *reinterpret_cast<const float4*>(a.w + (size_t)((kt + 1) * BK + brow) * a.ldw + n0 + bcol);
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[cur][kk][ty * 8]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[cur][kk][ty * 8 + 4]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[cur][kk][tx * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (kt + 1 < KT) {
      store_a<VEC>(As[cur ^ 1], ra);
      *reinterpret_cast<float4*>(&Bs[cur ^ 1][brow][bcol]) = rb;
    }
    __syncthreads();
  }

  // epilogue
  const ConvSpec& c = a.c;
  const int co = n0 + tx * 4;
  if (co >= c.cout) return;
  const int nc = min(4, c.cout - co);
  float bias[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) bias[j] = c.bias[co + j];
  const int hw = c.Ho * c.Wo;
  float* outp = static_cast<float*>(c.out.ptr);
  const float* resp = static_cast<const float*>(c.res.ptr);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int m = m0 + ty * 8 + i;
    if (m >= a.M) break;
    const int n = m / hw, rem = m % hw, oy = rem / c.Wo, ox = rem % c.Wo;
    float v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      v[j] = acc[i][j] + bias[j];
      if (c.act) v[j] = leaky01(v[j]);
    }
    if (resp) {
      const float* r = resp + tview_off(c.res, n, oy, ox) + co;
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (j < nc) v[j] += r[j];
    }
    const int reps = c.upsample ? 4 : 1;
    for (int q = 0; q < reps; ++q) {
      const int y = c.upsample ? 2 * oy + (q >> 1) : oy;
      const int x = c.upsample ? 2 * ox + (q & 1) : ox;
      float* o = outp + tview_off(c.out, n, y, x) + co;
      if (nc == 4) {
        *reinterpret_cast<float4*>(o) = make_float4(v[0], v[1], v[2], v[3]);
      } else {
        for (int j = 0; j < nc; ++j) o[j] = v[j];
      }
    }
  }
}

}  // namespace

void conv_simt_launch(const ConvSpec& c, const float* w_kn, int cout_pad64, cudaStream_t st) {
  SimtArgs a;
  a.c = c;
  a.w = w_kn;
  a.ldw = cout_pad64;
  a.K = c.k * c.k * c.cin;
  a.M = c.in.n * c.Ho * c.Wo;
  dim3 grid((a.M + BM - 1) / BM, cout_pad64 / BN);
  if (c.cin % BK == 0)
    (jde_count_launch(), conv_simt_kernel<true><<<grid, 256, 0, st>>>(a));
  else
    (jde_count_launch(), conv_simt_kernel<false><<<grid, 256, 0, st>>>(a));
}
