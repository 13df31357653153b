// BF16 / E4M3 implicit-GEMM convolution on the 5th-generation tensor cores (tcgen05).
//
// GEMM view: D[M = pixels][N = out channels] = sum_k A[m][k] B[n][k], K = (tap, ci).
// A persistent CTA (or CTA pair: M = 256 over two SMs, cta_group::2) computes 128 x BN tiles
// with the f32 accumulator in TMEM:
//   * warp 0 / lane 0 streams A and B k-blocks (64-byte or 128-byte rows of one tap) into a
//     STAGES-deep shared-memory ring with TMA (cp.async.bulk.tensor), swizzled, completion
//     tracked by mbarriers (the windowed modes load an input window once per k-block instead);
//   * warp 1 / lane 0 issues tcgen05.mma (M=128 or 256, N=BN, K=16 bf16 / 32 E4M3) per k-block
//     and frees the ring slot with tcgen05.commit;
//   * two groups of four epilogue warps read the accumulator rows (TMEM lane = tile row) with
//     tcgen05.ld and run the fused epilogue: x E4M3 dequantisation, + bias (BN folded),
//     leaky-ReLU, + residual (or a TMA reduce-add into the residual's own storage), bf16 / E4M3 /
//     f32 staged TMA stores, or direct stores with the 2x2 upsample into a concat slice.
// Activation addressing (implicit im2col) needs no gather:
//   * stride 1 ("flat"): activations keep a 1-pixel zero halo, so for tap
//     (ky, kx) the A rows of output pixels m0..m0+127 (flattened over the
//     padded image) are input rows m0 + (ky-1)*Wp + (kx-1): one 2-D TMA box.
//     Rows that fall on the halo are computed and discarded.
//   * stride 2 ("patch"): the padded input is split into its four
//     (row parity, column parity) sub-lattices, each described by its own 4-D
//     tensor map; tap (ky, kx) of a TH x TW output patch is a dense box of
//     sub-lattice (ky&1, kx&1) at offset (ky>>1, kx>>1).
// Every wait is bounded; on a timeout the CTA flags the error word, skips
// its stores, releases TMEM and exits.
#include <stdio.h>

#include <mutex>

#include "internal.h"

namespace {

struct TcArgs {
  int mode, k, cin_blocks, kt_total;
  int M_total, Hp, Wp;
  int TW, TH, tiles_x, tiles_y, n_tiles, total_tiles;
  int tma_out, tma_res;
  int red_res;                     // output aliases the residual: stores are TMA reduce-adds
  int stride, WW, WH, win_bytes;   // mode 3: window (or parity sub-window) size in pixels, bytes per buffer
  int plane;                       // mode 3: bytes between (parity) windows of one buffer (1024-aligned)
  int plane_tx;                    // mode 3: bytes one window load delivers (WW * WH * 64)
  int nwin;                        // modes 3, 4: window buffers in the ring (2 .. MAX_WIN)
  int total_units;                 // work units: tiles, or (CTA pairs) pairs of M tiles x N tiles
  int kel;                         // elements of one k-block along K (E4M3: twice the bf16 count, same bytes)
  int wnb, whb;                    // mode 4: TMA boxes per window, pixel rows per box
  int msub;                        // mode 4: 128-row M sub-tiles per CTA and unit (1 or 2)
  ConvSpec c;
};

// Modes: 0 flat stride-1 (TMA per tap), 1 stride-2 patch (TMA per tap from parity maps),
// 2 stem (im2col gathered from the letterbox), 3 32-channel 3x3: the input window of an
// 8x16 output patch (stride 2: its four parity sub-windows) is loaded once, 64 bytes per pixel
// with the 64-byte swizzle; the MMAs apply the swizzle to absolute shared-memory addresses, so
// each tap is the same window at another descriptor start (pixel offset); weights resident.
// 4 stride-1 3x3 with 64-byte k-blocks (32 bf16 / 64 E4M3 channels): per k-block the flat input
// rows m0 - Wp - 1 .. m0 + 128 + Wp (the nine taps' rows of the tile) are loaded once into a
// 64-byte-swizzled window; tap (ky, kx) is the window at row offset ky * Wp + kx; the weights
// stream through the ring, one (tap, k-block) tile per stage.
__device__ __forceinline__ bool patch_mode(int mode) { return mode == 1 || mode == 3; }

// warp 0: TMA producer; warp 1: MMA issuer + TMEM owner; warps 2..9: epilogue in two
// groups of four, group g draining TMEM accumulator buffer g (tiles alternate).
constexpr int EPI_WARPS = 8;
constexpr int MAX_WIN = 16;   // modes 3, 4: most window buffers in flight
__host__ __device__ constexpr int tc_threads(int gw) { return 32 * (gw + 1 + EPI_WARPS); }

// CG = 2: a CTA pair computes a 256 x BN tile with one M=256 MMA; each CTA holds its own
// 128 rows of A and half (BN/2 rows) of B.
// Q = 1: E4M3 operands (one byte per element; a k-block row holds 2 * BKC elements, the same
// bytes as BKC bf16 ones) and E4M3 staged outputs.
// WM = 1: mode 4 (flat window); the ring holds weight tiles only, the windows are sized at launch.
// WM = 2: mode 4 with two M sub-tiles per CTA: a unit is 256 rows x BN columns per CTA (512 x BN per
// pair), each weight tile feeding the MMAs of both sub-tiles, whose accumulators sit side by side
// (columns [0, BN) and [BN, 2 BN) of the unit's TMEM buffer); epilogue group g drains sub-tile g.
template <int BN, int BKC, int STAGES, int CG = 1, int Q = 0, int WM = 0>
struct TcCfg {
  static constexpr int MS = WM == 2 ? 2 : 1;            // M sub-tiles per unit
  static constexpr int ACC = BN * MS;                   // TMEM columns of one unit's accumulators
  static constexpr int A_BYTES = 128 * BKC * 2;
  static constexpr int B_BYTES = (BN / CG) * BKC * 2;
  static constexpr int STAGE_BYTES = WM ? B_BYTES : A_BYTES + B_BYTES;
  static constexpr int SWC = BN < 64 ? BN : 64;         // columns staged per epilogue pass
  static constexpr int PASSES = BN / SWC;
  static constexpr int SUB = SWC < 64 ? SWC : 64;       // channels per TMA store box (64 or 128-byte rows)
  static constexpr int NSUB = SWC / SUB;
  static constexpr int SUB_BYTES = 128 * SUB * 2;
  static constexpr int C_BYTES = Q ? 128 * SWC : NSUB * SUB_BYTES;   // one staging tile (one epilogue pass)
  static constexpr uint32_t WROW = BKC * 2;             // mode 4: bytes per window row (one k-block)
  static constexpr int BIAS_BYTES = 2 * BN * 4 * (Q ? 2 : 1);   // per epilogue group: bias (and E4M3 scale) slice
  static constexpr int BAR_BYTES = 768;                 // mbarriers + TMEM address slot
  // staging tiles per epilogue group: two, unless the ring then leaves no room (flat windows of
  // 128-byte rows, deep rings of 256-wide tiles): one
  static constexpr int SDEPTH =
      (WM && BKC == 64) ||
              STAGES * STAGE_BYTES + 4 * C_BYTES + 1024 + BAR_BYTES + BIAS_BYTES > 227 * 1024 - 64
          ? 1
          : 2;
  static constexpr int SMEM =
      STAGES * STAGE_BYTES + 2 * SDEPTH * C_BYTES + 1024 /*align*/ + BAR_BYTES + BIAS_BYTES;
  static constexpr uint32_t LAYOUT = BKC == 64 ? 2u : 4u;     // SW128 : SW64 (MMA operand tiles)
  static constexpr uint32_t SBO = 8 * BKC * 2;                 // bytes per 8-row group
  static constexpr int NBUF = ACC <= 128 ? 4 : 2;              // TMEM accumulator buffers
  // 256-wide tiles (two TMEM buffers): both epilogue groups drain every tile, each half of its
  // columns (WM = 2: each one sub-tile), so a buffer is free again in half the time; narrower
  // tiles alternate between groups
  static constexpr bool SPLIT = ACC == 256;
  static constexpr uint32_t TMEM_COLS = NBUF * ACC;
  static_assert(SMEM <= 227 * 1024 - 64, "shared memory budget (64 bytes left for static shared variables)");
  static_assert((2 * STAGES + 2 * NBUF + 2 + 2 * MAX_WIN + 1) * 8 + 4 <= BAR_BYTES, "barrier region");
  static_assert(TMEM_COLS >= 32 && TMEM_COLS <= 512, "TMEM budget");
};

// 16-byte unit `unit` of staged row `row` inside a SUB-channel box written by TMA with
// 128-byte (SUB 64) or 64-byte (SUB 32) swizzle: the unit index is XORed with the
// address bits 7..9 (resp. 7..8) of the row start.
template <int SUB>
__device__ __forceinline__ uint32_t stage_off(int row, int unit) {
  if (SUB == 64) return (uint32_t)(row * 128 + ((unit ^ (row & 7)) << 4));
  return (uint32_t)(row * 64 + ((unit ^ ((row >> 1) & 3)) << 4));
}

__device__ __forceinline__ void store_chunk(const ConvSpec& c, int n, int y, int x, int ch0, int nvalid,
                                            const float (&v)[32]) {
  const int reps = c.upsample ? 4 : 1;
  for (int q = 0; q < reps; ++q) {
    const int yy = c.upsample ? 2 * y + (q >> 1) : y;
    const int xx = c.upsample ? 2 * x + (q & 1) : x;
    const size_t off = tview_off(c.out, n, yy, xx) + ch0;
    if (c.out.dtype == 1) {
      __nv_bfloat16* o = static_cast<__nv_bfloat16*>(c.out.ptr) + off;
      if (nvalid == 32) {
        uint32_t packed[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
          packed[j] = *reinterpret_cast<uint32_t*>(&h2);
        }
        uint4* o4 = reinterpret_cast<uint4*>(o);
#pragma unroll
        for (int j = 0; j < 4; ++j)
          o4[j] = make_uint4(packed[4 * j], packed[4 * j + 1], packed[4 * j + 2], packed[4 * j + 3]);
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (j < nvalid) o[j] = __float2bfloat16_rn(v[j]);
      }
    } else if (c.out.dtype == 2) {
      uint8_t* o = static_cast<uint8_t*>(c.out.ptr) + off;
      if (nvalid == 32) {
        uint32_t packed[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
          packed[j] = e4m3x2(v[4 * j] * c.out_inv_scale, v[4 * j + 1] * c.out_inv_scale) |
                      (e4m3x2(v[4 * j + 2] * c.out_inv_scale, v[4 * j + 3] * c.out_inv_scale) << 16);
        uint4* o4 = reinterpret_cast<uint4*>(o);
        o4[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
        o4[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (j < nvalid) o[j] = (uint8_t)(e4m3x2(v[j] * c.out_inv_scale, 0.f) & 0xFFu);
      }
    } else {
      float* o = static_cast<float*>(c.out.ptr) + off;
      if ((nvalid & 3) == 0) {
        float4* o4 = reinterpret_cast<float4*>(o);
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (4 * j < nvalid) o4[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (j < nvalid) o[j] = v[j];
      }
    }
  }
}

struct TileCoord {
  int n0, m0, img, oy0, ox0;
};

__device__ __forceinline__ TileCoord tile_coord(const TcArgs& a, int tile, int bn) {
  TileCoord t;
  const int n_tile = tile % a.n_tiles;   // consecutive tiles share the activation tile
  const int m_tile = tile / a.n_tiles;
  t.n0 = n_tile * bn;
  t.m0 = 0;
  t.img = 0;
  t.oy0 = 0;
  t.ox0 = 0;
  if (!patch_mode(a.mode)) {
    t.m0 = m_tile * 128 * a.msub;
  } else {
    const int per_img = a.tiles_x * a.tiles_y;
    t.img = m_tile / per_img;
    const int r = m_tile % per_img;
    t.oy0 = (r / a.tiles_x) * a.TH;
    t.ox0 = (r % a.tiles_x) * a.TW;
  }
  return t;
}

__device__ __forceinline__ bool aborted(const int* flag) { return *((volatile const int*)flag) != 0; }

// One K step of the tile's MMA: M = 128 (CG = 2: 256 over the CTA pair), N = BN, bf16 or E4M3.
template <int CG, int Q>
__device__ __forceinline__ void mma_step(uint32_t d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t accum) {
  if constexpr (CG == 2 && Q)
    umma_e4m3_pair(d, ad, bd, idesc, accum);
  else if constexpr (CG == 2)
    umma_bf16_pair(d, ad, bd, idesc, accum);
  else if constexpr (Q)
    umma_e4m3(d, ad, bd, idesc, accum);
  else
    umma_bf16(d, ad, bd, idesc, accum);
}

// Tile of work unit u for this CTA.  CG = 1: unit = tile.  CG = 2: unit = (M-tile pair, N tile);
// CTA `rank` of the pair takes M tile 2 * pair + rank.
template <int CG>
__device__ __forceinline__ int unit_tile(const TcArgs& a, int u, uint32_t rank) {
  if (CG == 1) return u;
  const int n_tile = u % a.n_tiles, m_pair = u / a.n_tiles;
  return (2 * m_pair + (int)rank) * a.n_tiles + n_tile;
}

// False for the idle second tile of a CTA pair whose M tile lies past the end.
__device__ __forceinline__ bool tile_live(const TcArgs& a, const TileCoord& t) {
  if (!patch_mode(a.mode)) return t.m0 < a.M_total;
  return t.img < a.c.out.n;
}

// Persistent CTA (one per SM): work units blockIdx.x, blockIdx.x + gridDim.x, ... (CG = 2:
// per CTA pair of a 2-CTA cluster, the leader CTA of the pair issuing the M=256 MMAs).
// Warps 0..GW-1 produce (GW = 1: lane 0 of warp 0 issues TMA; the stem uses GW gather
// warps), warp GW issues the MMAs and owns TMEM, the last 8 warps run the epilogue.
template <int BN, int BKC, int STAGES, int GW, int CG, int Q, int WM>
__global__ void __launch_bounds__(tc_threads(GW), 1) conv_tc_kernel(const __grid_constant__ TcPlan plan, const TcArgs a) {
  using Cfg = TcCfg<BN, BKC, STAGES, CG, Q, WM>;
  const uint32_t rank = CG == 2 ? cluster_rank() : 0u;
  const int u0 = CG == 2 ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
  const int ustep = CG == 2 ? (int)(gridDim.x >> 1) : (int)gridDim.x;
  const int nunits = CG == 2 ? a.total_units : a.total_tiles;
  extern __shared__ uint8_t smem_raw[];
  __shared__ int s_abort;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  // mode 3: [windows][resident B][staging]; mode 4: [windows][B ring][staging];
  // otherwise [A ring][B ring][staging]
  uint8_t* sWin = smem;
  uint8_t* sA = smem;
  uint8_t* sB = a.mode >= 3 ? smem + a.nwin * a.win_bytes : smem + STAGES * Cfg::A_BYTES;
  const int b_region = a.mode == 3 ? a.kt_total * Cfg::B_BYTES : STAGES * Cfg::B_BYTES;
  uint8_t* sC = sB + b_region;                           // 2 staging tiles
  uint64_t* full = reinterpret_cast<uint64_t*>(sC + 2 * Cfg::SDEPTH * Cfg::C_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;   // [NBUF] MMA -> epilogue group
  uint64_t* acc_empty = acc_full + Cfg::NBUF;   // [NBUF] epilogue group -> MMA
  uint64_t* res_full = acc_empty + Cfg::NBUF;   // [2] residual tile landed in staging tile g
  uint64_t* win_full = res_full + 2;     // [MAX_WIN] modes 3, 4: input window landed
  uint64_t* win_empty = win_full + MAX_WIN;   // [MAX_WIN] modes 3, 4: window consumed by the MMAs
  uint64_t* b_full = win_empty + MAX_WIN;     // mode 3: resident weights landed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(b_full + 1);
  float* const sBiasAll = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(full) + Cfg::BAR_BYTES);   // [2][BN]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const ConvSpec& c = a.c;

  if (threadIdx.x == 0) {
    // stem: TMA (B) arrival + the gather warp's arrival
    const int full_count = a.mode == 2 ? 2 : 1;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], full_count);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < Cfg::NBUF; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], CG * (Cfg::SPLIT ? EPI_WARPS : EPI_WARPS / 2));   // CG = 2: both CTAs' warps
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&res_full[b], 1);
    }
    for (int b = 0; b < MAX_WIN; ++b) {
      mbar_init(&win_full[b], 1);
      mbar_init(&win_empty[b], 1);      // tcgen05.commit after the tile's MMAs
    }
    mbar_init(b_full, 1);
    fence_barrier_init();
    s_abort = 0;
  }
  if (warp == GW) {
    if constexpr (CG == 2)
      tmem_alloc_pair(tmem_slot, Cfg::TMEM_COLS);
    else
      tmem_alloc(tmem_slot, Cfg::TMEM_COLS);
  }
  tc_fence_before();
  __syncthreads();
  if constexpr (CG == 2) cluster_sync();   // both CTAs' barriers initialised before any remote signal
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // launched as a dependent of the previous layer's kernel: the set-up above overlaps its tail, and
  // no thread touches global memory (that kernel's output, or this one's) before it has completed
  grid_dep_wait();

  if (warp < GW && a.mode == 2) {
    // ---------------- stem producer: gather warp w fills the stage of every GW-th tile with the
    // 3x3x3 im2col rows (27 bf16 values padded to 32, order (ky, kx, c)) read from the haloed
    // RGB0 letterbox image, in the 64-byte swizzle the MMA expects; its lane 0 streams the weights.
    if (lane == 0 && warp == 0) tma_prefetch(&plan.b);
    const __nv_bfloat16* lb = static_cast<const __nv_bfloat16*>(c.in.ptr);
    const int plane = a.Hp * a.Wp;
    uint32_t lt = 0;   // local tile index of this CTA
    for (int u = u0; u < nunits && !aborted(&s_abort); u += ustep, ++lt) {
      if ((int)(lt % GW) != warp) continue;
      const int tile = unit_tile<CG>(a, u, rank);
      const TileCoord tc = tile_coord(a, tile, BN);
      const uint32_t s = lt % STAGES;
      const uint32_t ph = (lt / STAGES) & 1u;
      bool ok = true;
      if (lane == 0 && lt >= (uint32_t)STAGES) ok = mbar_wait(&empty[s], ph ^ 1u);
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (!ok) {
        if (lane == 0) {
          flag_error(c.err, KERR_TIMEOUT);
          atomicExch(&s_abort, 1);
        }
        break;
      }
      if (lane == 0) {
        mbar_expect_tx(&full[s], Cfg::B_BYTES);
        tma_load_2d(sB + s * Cfg::B_BYTES, &plan.b, &full[s], 0, tc.n0);
      }
      uint8_t* dA = sA + s * Cfg::A_BYTES;
      // tap (ky, kx) of a pixel is a constant element offset from the pixel itself (the letterbox
      // and the flat tile share the padded grid); the letterbox halo is zero, so every tap of an
      // in-image pixel is addressable
      const int tap_step = a.Wp * c.in.pixstride;
      uint2 q[4][9];
#pragma unroll
      for (int i = 0; i < 4; ++i) {          // issue all 36 loads before using any
        const int r = lane + 32 * i;
        const int m = tc.m0 + r;
        const int n = m / plane, rem = m % plane;
        const int y = rem / a.Wp - 1, x = rem % a.Wp - 1;
        const bool in = m < a.M_total && y >= 0 && y < c.Ho && x >= 0 && x < c.Wo;
        const __nv_bfloat16* pix = lb + tview_off(c.in, n, y, x);
#pragma unroll
        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
          for (int kx = 0; kx < 3; ++kx)
            q[i][ky * 3 + kx] = in ? __ldg(reinterpret_cast<const uint2*>(pix + (ky - 1) * tap_step +
                                                                           (kx - 1) * c.in.pixstride))
                                   : make_uint2(0u, 0u);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = lane + 32 * i;
        __nv_bfloat16 v[32];
#pragma unroll
        for (int t = 0; t < 9; ++t) {
          const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&q[i][t]);
          v[3 * t] = e[0];
          v[3 * t + 1] = e[1];
          v[3 * t + 2] = e[2];
        }
#pragma unroll
        for (int j = 27; j < 32; ++j) v[j] = __float2bfloat16_rn(0.f);
        const uint4* v4 = reinterpret_cast<const uint4*>(v);
#pragma unroll
        for (int u = 0; u < 4; ++u) *reinterpret_cast<uint4*>(dA + stage_off<32>(r, u)) = v4[u];
      }
      fence_proxy_async();              // generic-proxy smem writes -> visible to tcgen05.mma
      __syncwarp();
      if (lane == 0) mbar_arrive(&full[s]);
    }
  } else if (warp == 0 && GW == 1 && a.mode == 3) {
    if (lane == 0) {
      // ---------------- window producer: resident weights once, then per patch the 8-channel
      // planes of its input window (stride 2: of its four parity sub-windows)
      mbar_expect_tx(b_full, (uint32_t)(a.kt_total * Cfg::B_BYTES));
      for (int kb = 0; kb < a.kt_total; ++kb) tma_load_2d(sB + kb * Cfg::B_BYTES, &plan.b, b_full, kb * 64, 0);
      const int npar = a.stride == 2 ? 4 : 1;
      uint32_t lt = 0;
      for (int u = u0; u < nunits && !aborted(&s_abort); u += ustep, ++lt) {
        const int tile = unit_tile<CG>(a, u, rank);
        const uint32_t wb = lt % (uint32_t)a.nwin;
        if (lt >= (uint32_t)a.nwin && !mbar_wait(&win_empty[wb], ((lt / (uint32_t)a.nwin) - 1) & 1u)) {
          flag_error(c.err, KERR_TIMEOUT);
          atomicExch(&s_abort, 1);
          break;
        }
        const TileCoord tc = tile_coord(a, tile, BN);
        if ((smem_u32(sWin + wb * a.win_bytes) | (uint32_t)a.plane) & 1023u) {   // swizzled TMA destinations
          flag_error(c.err, KERR_TIMEOUT);
          atomicExch(&s_abort, 1);
          break;
        }
        mbar_expect_tx(&win_full[wb], (uint32_t)(npar * a.plane_tx));
        for (int par = 0; par < npar; ++par)
          tma_load_4d(sWin + wb * a.win_bytes + par * a.plane, &plan.a[par], &win_full[wb], 0, tc.ox0, tc.oy0, tc.img);
      }
    }
  } else if (WM && warp == 0) {
    if (lane == 0) {
      // ---------------- flat-window producer: per k-block the tile's window rows, then its nine
      // weight tiles (tap-major); CG = 2: both CTAs' bytes are counted on the leader's barriers
      tma_prefetch(&plan.a[0]);
      tma_prefetch(&plan.b);
      uint32_t s = 0, ph = 0, nb = 0, w = 0, wph = 0, nw = 0;   // ring slots, phases, loads issued
      const uint32_t full_leader0 = CG == 2 ? mapa_rank(smem_u32(&full[0]), 0) : 0u;
      const uint32_t wfull_leader0 = CG == 2 ? mapa_rank(smem_u32(&win_full[0]), 0) : 0u;
      const uint32_t box_bytes = (uint32_t)a.whb * Cfg::WROW;
      bool ok = true;
      for (int u = u0; ok && u < nunits && !aborted(&s_abort); u += ustep) {
        const TileCoord tc = tile_coord(a, unit_tile<CG>(a, u, rank), BN);
        const int row0 = tc.m0 - a.Wp - 1;   // input row of the window's first pixel (may be < 0: zero fill)
        for (int cb = 0; ok && cb < a.cin_blocks; ++cb) {
          if (nw >= (uint32_t)a.nwin && !mbar_wait(&win_empty[w], wph ^ 1u)) {
            ok = false;
            break;
          }
          uint8_t* dW = sWin + w * a.win_bytes;
          if ((smem_u32(dW) | box_bytes) & 1023u) {   // swizzled TMA destinations
            ok = false;
            break;
          }
          if constexpr (CG == 2) {
            if (rank == 0) mbar_expect_tx(&win_full[w], 2u * (uint32_t)a.wnb * box_bytes);
            for (int j = 0; j < a.wnb; ++j)
              tma_load_2d_pair(dW + j * box_bytes, &plan.a[0], wfull_leader0 + w * 8u, cb * a.kel, row0 + j * a.whb);
          } else {
            mbar_expect_tx(&win_full[w], (uint32_t)a.wnb * box_bytes);
            for (int j = 0; j < a.wnb; ++j)
              tma_load_2d(dW + j * box_bytes, &plan.a[0], &win_full[w], cb * a.kel, row0 + j * a.whb);
          }
          ++nw;
          if (++w == (uint32_t)a.nwin) {
            w = 0;
            wph ^= 1u;
          }
          for (int tap = 0; tap < 9; ++tap) {
            if (nb >= (uint32_t)STAGES && !mbar_wait(&empty[s], ph ^ 1u)) {
              ok = false;
              break;
            }
            ++nb;
            const int kcol = tap * a.c.cin + cb * a.kel;   // weights: K = (tap, channel)
            if constexpr (CG == 2) {
              if (rank == 0) mbar_expect_tx(&full[s], 2u * (uint32_t)Cfg::B_BYTES);
              tma_load_2d_pair(sB + s * Cfg::B_BYTES, &plan.b, full_leader0 + s * 8u, kcol, tc.n0 + (int)rank * (BN / 2));
            } else {
              mbar_expect_tx(&full[s], (uint32_t)Cfg::B_BYTES);
              tma_load_2d(sB + s * Cfg::B_BYTES, &plan.b, &full[s], kcol, tc.n0);
            }
            if (++s == (uint32_t)STAGES) {
              s = 0;
              ph ^= 1u;
            }
          }
        }
      }
      if (!ok) {
        flag_error(c.err, KERR_TIMEOUT);
        atomicExch(&s_abort, 1);
      }
    }
  } else if (warp == 0 && GW == 1) {
    if (lane == 0) {
      // ---------------- TMA producer
      for (int i = 0; i < 4; ++i)
        if (a.mode == 1 || i == 0) tma_prefetch(&plan.a[i]);
      tma_prefetch(&plan.b);
      uint32_t it = 0;
      const uint32_t full_leader0 = CG == 2 ? mapa_rank(smem_u32(&full[0]), 0) : 0u;
      for (int u = u0; u < nunits && !aborted(&s_abort); u += ustep) {
        const int tile = unit_tile<CG>(a, u, rank);
        const TileCoord tc = tile_coord(a, tile, BN);
        for (int kt = 0; kt < a.kt_total; ++kt, ++it) {
          const uint32_t s = it % STAGES;
          const uint32_t ph = (it / STAGES) & 1u;
          if (it >= (uint32_t)STAGES && !mbar_wait(&empty[s], ph ^ 1u)) {
            flag_error(c.err, KERR_TIMEOUT);
            atomicExch(&s_abort, 1);
            break;
          }
          const int tap = kt / a.cin_blocks, cb = kt % a.cin_blocks;
          const int ky = tap / a.k, kx = tap % a.k;
          uint8_t* dA = sA + s * Cfg::A_BYTES;
          if constexpr (CG == 2) {
            // both CTAs' bytes are counted on the leader's full[s]
            const uint32_t bar = full_leader0 + s * 8u;
            if (rank == 0) mbar_expect_tx(&full[s], 2 * Cfg::STAGE_BYTES);
            if (a.mode == 0) {
              const int shift = a.k == 3 ? (ky - 1) * a.Wp + (kx - 1) : 0;
              tma_load_2d_pair(dA, &plan.a[0], bar, cb * a.kel, tc.m0 + shift);
            } else {
              tma_load_4d_pair(dA, &plan.a[(ky & 1) * 2 + (kx & 1)], bar, cb * a.kel, tc.ox0 + (kx >> 1),
                               tc.oy0 + (ky >> 1), tc.img);
            }
            tma_load_2d_pair(sB + s * Cfg::B_BYTES, &plan.b, bar, kt * a.kel, tc.n0 + (int)rank * (BN / 2));
          } else {
            mbar_expect_tx(&full[s], Cfg::STAGE_BYTES);
            if (a.mode == 0) {
              const int shift = a.k == 3 ? (ky - 1) * a.Wp + (kx - 1) : 0;
              tma_load_2d(dA, &plan.a[0], &full[s], cb * a.kel, tc.m0 + shift);
            } else {
              tma_load_4d(dA, &plan.a[(ky & 1) * 2 + (kx & 1)], &full[s], cb * a.kel, tc.ox0 + (kx >> 1),
                          tc.oy0 + (ky >> 1), tc.img);
            }
            tma_load_2d(sB + s * Cfg::B_BYTES, &plan.b, &full[s], kt * a.kel, tc.n0);
          }
        }
      }
    }
  } else if (warp == GW) {
    if (lane == 0 && rank == 0) {
      // ---------------- MMA issuer (CG = 2: the leader CTA, for both CTAs of the pair)
      constexpr uint32_t idesc = Q ? idesc_e4m3(128 * CG, BN) : idesc_bf16(128 * CG, BN);
      uint32_t local = 0;
      uint32_t s = 0, ph = 0;   // ring slot and its phase parity
      uint32_t w4 = 0, w4ph = 0;   // mode 4: window slot and its phase parity
      // Descriptors are built once: the start address (16-byte units, bits 0..13) of every
      // operand tile is the base descriptor plus a constant offset, so issuing an MMA costs one add.
      const uint64_t a_desc0 = smem_desc(smem_u32(sA), Cfg::SBO, Cfg::LAYOUT);
      const uint64_t b_desc0 = smem_desc(smem_u32(sB), Cfg::SBO, Cfg::LAYOUT);
      constexpr int NW = 18;                      // mode 3: 9 taps x two K=16 MMAs per tile
      uint32_t w_aoff[NW], w_boff[NW];
      uint64_t w_desc0 = 0;
      if (CG == 1 && !Q && a.mode == 3) {
        // 64-byte-swizzled window, 8-row groups one window row (WW pixels x 64 bytes) apart
        w_desc0 = smem_desc(smem_u32(sWin), (uint32_t)(a.WW * 64), 4u);
#pragma unroll
        for (int i = 0; i < NW; ++i) {
          const int tap = i / 2, kk = i % 2;
          const int ky = tap / 3, kx = tap % 3;
          const int par = a.stride == 2 ? (ky & 1) * 2 + (kx & 1) : 0;
          const int pix = a.stride == 2 ? (ky >> 1) * a.WW + (kx >> 1) : ky * a.WW + kx;
          const int kidx = tap * 32 + kk * 16;   // K index of this MMA's first element
          w_aoff[i] = (uint32_t)(par * a.plane + pix * 64 + kk * 32) >> 4;
          w_boff[i] = (uint32_t)((kidx >> 6) * Cfg::B_BYTES + (kidx & 63) * 2) >> 4;
        }
      }
      for (int u = u0; u < nunits; u += ustep, ++local) {
        const uint32_t buf = local % Cfg::NBUF, use = local / Cfg::NBUF;
        if (local >= (uint32_t)Cfg::NBUF && !mbar_wait(&acc_empty[buf], (use - 1) & 1u)) {
          flag_error(c.err, KERR_TIMEOUT);
          atomicExch(&s_abort, 1);
          break;
        }
        if (local == 0 && a.mode == 3 && !mbar_wait(b_full, 0)) {
          flag_error(c.err, KERR_TIMEOUT);
          atomicExch(&s_abort, 1);
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + buf * Cfg::ACC;
        if constexpr (CG == 1 && !Q) if (a.mode == 3) {
          const uint32_t wb = local % (uint32_t)a.nwin;
          if (!mbar_wait(&win_full[wb], (local / (uint32_t)a.nwin) & 1u)) {
            flag_error(c.err, KERR_TIMEOUT);
            atomicExch(&s_abort, 1);
            break;
          }
          tc_fence_after();
          // window buffer wb, each tap at its pixel offset in the swizzled window
          const uint64_t ad0 = desc_add(w_desc0, (wb * (uint32_t)a.win_bytes) >> 4);
#pragma unroll
          for (int i = 0; i < NW; ++i)
            umma_bf16(d, desc_add(ad0, w_aoff[i]), desc_add(b_desc0, w_boff[i]), idesc, i != 0 ? 1u : 0u);
          umma_commit(&acc_full[buf]);
          umma_commit(&win_empty[wb]);
          continue;
        }
        if constexpr (WM != 0) {
          // mode 4: per k-block one window; tap (ky, kx) starts ky * Wp + kx rows into it
          // window rows of WROW bytes (64: 64-byte swizzle, 128: 128-byte swizzle), 8-row groups
          const uint64_t w_base = smem_desc(smem_u32(sWin), 8u * Cfg::WROW, Cfg::LAYOUT);
          bool wok = true;
          for (int cb = 0; cb < a.cin_blocks; ++cb) {
            if (!mbar_wait(&win_full[w4], w4ph)) {
              wok = false;
              break;
            }
            tc_fence_after();
            const uint64_t wd = desc_add(w_base, (w4 * (uint32_t)a.win_bytes) >> 4);
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) {
              if (!mbar_wait(&full[s], ph)) {
                wok = false;
                break;
              }
              tc_fence_after();
              const uint64_t ad_t = desc_add(wd, (uint32_t)((tap / 3) * a.Wp + tap % 3) * (Cfg::WROW / 16u));
              const uint64_t bd_s = desc_add(b_desc0, (s * (uint32_t)Cfg::B_BYTES) >> 4);
#pragma unroll
              for (int kk = 0; kk < BKC / 16; ++kk)
#pragma unroll
                for (int ms = 0; ms < Cfg::MS; ++ms)   // sub-tile ms: 128 window rows (8 KB) further on
                  mma_step<CG, Q>(d + (uint32_t)(ms * BN), desc_add(ad_t, 2 * kk + ms * 8 * Cfg::WROW),
                                  desc_add(bd_s, 2 * kk),
                                  idesc, (cb | tap | kk) != 0 ? 1u : 0u);
              if constexpr (CG == 2)
                umma_commit_pair(&empty[s], 3);
              else
                umma_commit(&empty[s]);
              if (++s == (uint32_t)STAGES) {
                s = 0;
                ph ^= 1u;
              }
            }
            if (!wok) break;
            if constexpr (CG == 2)
              umma_commit_pair(&win_empty[w4], 3);   // the window is free in both CTAs
            else
              umma_commit(&win_empty[w4]);
            if (++w4 == (uint32_t)a.nwin) {
              w4 = 0;
              w4ph ^= 1u;
            }
          }
          if constexpr (CG == 2)
            umma_commit_pair(&acc_full[buf], 3);
          else
            umma_commit(&acc_full[buf]);
          if (!wok) {
            flag_error(c.err, KERR_TIMEOUT);
            atomicExch(&s_abort, 1);
            break;
          }
          continue;
        }
        bool ok = true;
        for (int kt = 0; kt < a.kt_total; ++kt) {
          if (!mbar_wait(&full[s], ph)) {
            flag_error(c.err, KERR_TIMEOUT);
            atomicExch(&s_abort, 1);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint64_t ad_s = desc_add(a_desc0, (s * (uint32_t)Cfg::A_BYTES) >> 4);
          const uint64_t bd_s = desc_add(b_desc0, (s * (uint32_t)Cfg::B_BYTES) >> 4);
#pragma unroll
          for (int kk = 0; kk < BKC / 16; ++kk) {
            const uint64_t ad = desc_add(ad_s, 2 * kk);     // +32 bytes per K=16 (bf16) / K=32 (E4M3) step
            const uint64_t bd = desc_add(bd_s, 2 * kk);
            const uint32_t accum = (kt | kk) != 0 ? 1u : 0u;
            if constexpr (CG == 2 && Q)
              umma_e4m3_pair(d, ad, bd, idesc, accum);
            else if constexpr (CG == 2)
              umma_bf16_pair(d, ad, bd, idesc, accum);
            else if constexpr (Q)
              umma_e4m3(d, ad, bd, idesc, accum);
            else
              umma_bf16(d, ad, bd, idesc, accum);
          }
          if constexpr (CG == 2)
            umma_commit_pair(&empty[s], 3);      // the stage is free in both CTAs
          else
            umma_commit(&empty[s]);
          if (++s == (uint32_t)STAGES) {
            s = 0;
            ph ^= 1u;
          }
        }
        if constexpr (CG == 2)
          umma_commit_pair(&acc_full[buf], 3);
        else
          umma_commit(&acc_full[buf]);
        if (!ok) break;
      }
    }
  } else if (warp > GW) {
    // ---------------- epilogue: group g takes the tiles whose local index has parity g (256-wide
    // tiles: every tile, its half g of the columns)
    const int ew = warp - GW - 1;
    const int g = ew >> 2;
    const int quarter = warp & 3;           // TMEM lanes a warp may read: 32 * (warp % 4) ...
    const int row = quarter * 32 + lane;
    const bool elected = (ew & 3) == 0 && lane == 0;
    const int bar_id = 1 + g;
    // WM = 2: group g drains sub-tile g (rows 128 g .. 128 g + 127 of the unit, TMEM columns g BN ..)
    const int mrow = WM == 2 ? g * 128 : 0;
    const uint32_t cbase = WM == 2 ? (uint32_t)(g * BN) : 0u;
    // the group's SDEPTH staging tiles take the passes in turn, so a pass only waits for the
    // store issued SDEPTH passes earlier to have read its tile
    uint8_t* const stg_base = sC + g * Cfg::SDEPTH * Cfg::C_BYTES;
    uint8_t* stg = stg_base;
    uint32_t res_uses = 0, local = 0, npass = 0;
    // bias of the group's current N tile, in shared memory (refilled when the N tile changes)
    float* const sBias = sBiasAll + g * BN;
    float* const sMult = sBiasAll + 2 * BN + g * BN;       // Q: input scale x weight scale per channel
    const int gtid = (ew & 3) * 32 + lane;
    int bias_n0 = -1;
    float4 breg[8];                         // 32-wide tiles: the tile's bias in registers
    // CG = 2: the accumulator buffer is released on the leader's barrier
    const uint32_t acc_empty_leader0 = CG == 2 ? mapa_rank(smem_u32(&acc_empty[0]), 0) : 0u;
    for (int u = u0; u < nunits; u += ustep, ++local) {
      if (!Cfg::SPLIT && (local & 1u) != (uint32_t)g) continue;
      const int tile = unit_tile<CG>(a, u, rank);
      const uint32_t buf = local % Cfg::NBUF, use = local / Cfg::NBUF;
      bool ok = mbar_wait(&acc_full[buf], use & 1u);
      if (!ok) {
        flag_error(c.err, KERR_TIMEOUT);
        atomicExch(&s_abort, 1);
      }
      // the CTA's last accumulator is complete: only its epilogue is left, so the next layer's kernel
      // may launch and set up (it waits for this grid before touching global memory)
      if (u + ustep >= nunits && gtid == 0) grid_dep_trigger();
      ok = bar_and(ok, bar_id, 128);        // the group's four warps take the same path
      tc_fence_after();
      const TileCoord tc = tile_coord(a, tile, BN);
      if (tc.n0 != bias_n0) {
        // the group finished reading the previous slice before the last pass's barrier
        for (int i = gtid; i < BN; i += 128) {
          sBias[i] = c.bias[tc.n0 + i];
          if (Q) sMult[i] = c.mult[tc.n0 + i];
        }
        named_bar(bar_id, 128);
        bias_n0 = tc.n0;
        if (BN == 32) {
#pragma unroll
          for (int i = 0; i < 8; ++i) breg[i] = reinterpret_cast<const float4*>(sBias)[i];
        }
      }
      int n = 0, y = 0, x = 0;
      bool valid;
      if (!patch_mode(a.mode)) {
        const int m = tc.m0 + mrow + row;
        const int plane = a.Hp * a.Wp;
        n = m / plane;
        const int r = m % plane;
        y = r / a.Wp - 1;
        x = r % a.Wp - 1;
        valid = m < a.M_total && y >= 0 && y < c.Ho && x >= 0 && x < c.Wo;
      } else {
        n = tc.img;
        y = tc.oy0 + row / a.TW;
        x = tc.ox0 + row % a.TW;
        valid = y < c.Ho && x < c.Wo && tile_live(a, tc);
      }
      if (a.tma_out && c.out.dtype == 0) {
        // staged f32 (the embedding heads): sub-passes of FW columns, each one staging tile
        // (128-byte rows with the 128-byte swizzle, or 64-byte rows with the 64-byte one) and one
        // TMA store box; rows on the halo are written as zeros
        constexpr int FW = Cfg::C_BYTES / (128 * 4);
        constexpr int NSP = BN / FW;
        const int sp_begin = Cfg::SPLIT && WM != 2 ? g * (NSP / 2) : 0;
        const int sp_end = Cfg::SPLIT && WM != 2 ? sp_begin + NSP / 2 : NSP;
        for (int sp = sp_begin; sp < sp_end; ++sp) {
          stg = stg_base + (npass++ % Cfg::SDEPTH) * Cfg::C_BYTES;
          const bool live = WM == 2 ? tc.m0 + mrow < a.M_total : tile_live(a, tc);
          const int c0 = sp * FW;
          uint32_t r[32];
          const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + buf * Cfg::ACC + cbase + (uint32_t)c0;
          if (FW == 32)
            tmem_ld32(taddr, r);
          else
            tmem_ld16(taddr, r);
          if (elected) bulk_wait_read<Cfg::SDEPTH - 1>();   // the store that last used this staging tile has read it
          named_bar(bar_id, 128);
          float v[FW];
#pragma unroll
          for (int j = 0; j < FW; ++j) v[j] = sBias[c0 + j];
          float m[FW];
          if (Q) {
#pragma unroll
            for (int j = 0; j < FW; ++j) m[j] = sMult[c0 + j];
          }
          tmem_ld_wait();
#pragma unroll
          for (int j = 0; j < FW; ++j) {
            const float acc = Q ? __uint_as_float(r[j]) * m[j] : __uint_as_float(r[j]);
            const float t = acc + v[j];
            v[j] = c.act ? leaky01f(t) : t;
          }
#pragma unroll
          for (int u = 0; u < FW / 4; ++u) {
            uint8_t* q = stg + (FW == 32 ? stage_off<64>(row, u) : stage_off<32>(row, u));
            *reinterpret_cast<uint4*>(q) =
                valid ? make_uint4(__float_as_uint(v[4 * u]), __float_as_uint(v[4 * u + 1]),
                                   __float_as_uint(v[4 * u + 2]), __float_as_uint(v[4 * u + 3]))
                      : make_uint4(0u, 0u, 0u, 0u);
          }
          if (sp == sp_end - 1) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {                   // accumulator buffer free for the MMA
              if (CG == 2)
                mbar_arrive_cluster(acc_empty_leader0 + buf * 8u);
              else
                mbar_arrive(&acc_empty[buf]);
            }
          }
          fence_proxy_async();               // staging writes visible to the TMA store
          named_bar(bar_id, 128);
          if (elected && ok && live && !aborted(&s_abort)) {
            if (!patch_mode(a.mode))
              tma_store_2d(&plan.o, stg, tc.n0 + c0, tc.m0 + mrow);
            else
              tma_store_4d(&plan.o, stg, tc.n0 + c0, tc.ox0 + 1, tc.oy0 + 1, tc.img);
            bulk_commit();
          }
        }
      } else if (a.tma_out) {
        // staged: TMEM -> (scale, bias, leaky, + residual) -> bf16 or E4M3 staging tile -> TMA store.
        // Rows on the halo are written as zeros, which keeps the halo zero.  E4M3 rows are SWC
        // bytes (64-byte swizzle), one box per pass.
        const bool o8 = c.out.dtype == 2;
        const uint32_t vmask = valid ? 0xFFFFFFFFu : 0u;   // rows on the halo are stored as zeros
        const int nsub = o8 ? 1 : Cfg::NSUB;
        const int sub_ch = o8 ? Cfg::SWC : Cfg::SUB;
        const int sub_bytes = o8 ? 128 * Cfg::SWC : Cfg::SUB_BYTES;
        const int p_begin = Cfg::SPLIT && WM != 2 ? g * (Cfg::PASSES / 2) : 0;
        const int p_end = Cfg::SPLIT && WM != 2 ? p_begin + Cfg::PASSES / 2 : Cfg::PASSES;
        for (int p = p_begin; p < p_end; ++p) {
          stg = stg_base + (npass++ % Cfg::SDEPTH) * Cfg::C_BYTES;
          const bool live = WM == 2 ? tc.m0 + mrow < a.M_total : tile_live(a, tc);
          const bool use_res = a.tma_res && ok && live;
          if (elected) {
            bulk_wait_read<Cfg::SDEPTH - 1>();   // the store that last used this staging tile has read it
            if (use_res) {
              mbar_expect_tx(&res_full[g], (uint32_t)(nsub * sub_bytes));
              for (int j = 0; j < nsub; ++j) {
                const int ch = tc.n0 + p * Cfg::SWC + j * sub_ch;
                if (patch_mode(a.mode))
                  tma_load_4d(stg + j * sub_bytes, &plan.r, &res_full[g], ch, tc.ox0 + 1, tc.oy0 + 1, tc.img);
                else
                  tma_load_2d(stg + j * sub_bytes, &plan.r, &res_full[g], ch, tc.m0 + mrow);
              }
            }
          }
          named_bar(bar_id, 128);
          if (use_res) {
            if (!mbar_wait(&res_full[g], res_uses & 1u)) {
              flag_error(c.err, KERR_TIMEOUT);
              atomicExch(&s_abort, 1);
            }
            ++res_uses;
          }
#pragma unroll 1
          for (int c0 = 0; c0 < Cfg::SWC; c0 += 32) {
            uint32_t r[32];
            tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + buf * Cfg::ACC + cbase + (uint32_t)(p * Cfg::SWC + c0), r);
            // the chunk's shared-memory operands (bias, scale, residual) are all read before any of
            // its stores, so the loads overlap each other and the TMEM read
            const int nu = o8 ? 2 : 4;               // 16-byte staging units of the chunk's 32 columns
            uint8_t* qa[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int col = o8 ? c0 + 16 * u : c0 + 8 * u;   // first column of unit u inside the pass
              qa[u] = o8 ? stg + stage_off<32>(row, col >> 4)
                         : stg + (col / Cfg::SUB) * Cfg::SUB_BYTES + stage_off<Cfg::SUB>(row, (col % Cfg::SUB) >> 3);
            }
            const float4* b4 = reinterpret_cast<const float4*>(sBias + p * Cfg::SWC + c0);
            float4 bb[8], mm[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) bb[i] = BN == 32 ? breg[i] : b4[i];
            if (Q) {
              const float4* m4 = reinterpret_cast<const float4*>(sMult + p * Cfg::SWC + c0);
#pragma unroll
              for (int i = 0; i < 8; ++i) mm[i] = m4[i];
            }
            uint4 rq[4];
            if (use_res) {
#pragma unroll
              for (int u = 0; u < 4; ++u)
                if (u < nu) rq[u] = *reinterpret_cast<const uint4*>(qa[u]);
            }
            tmem_ld_wait();
            float v[32];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              float a4[4] = {__uint_as_float(r[4 * i]), __uint_as_float(r[4 * i + 1]), __uint_as_float(r[4 * i + 2]),
                             __uint_as_float(r[4 * i + 3])};
              if (Q) {
                a4[0] *= mm[i].x;
                a4[1] *= mm[i].y;
                a4[2] *= mm[i].z;
                a4[3] *= mm[i].w;
              }
              v[4 * i] = a4[0] + bb[i].x;
              v[4 * i + 1] = a4[1] + bb[i].y;
              v[4 * i + 2] = a4[2] + bb[i].z;
              v[4 * i + 3] = a4[3] + bb[i].w;
            }
            if (c.act) {
#pragma unroll
              for (int e = 0; e < 32; ++e) v[e] = leaky01f(v[e]);
            }
            uint4 outv[4];
            if (o8) {
              // 32 columns = two 16-byte units of the 64-byte E4M3 row
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                if (use_res) {
                  const uint32_t rv[4] = {rq[h].x, rq[h].y, rq[h].z, rq[h].w};
#pragma unroll
                  for (int e = 0; e < 4; ++e) {
                    const float2 lo = e4m3x2_to_float2(rv[e] & 0xFFFFu), hi = e4m3x2_to_float2(rv[e] >> 16);
                    v[16 * h + 4 * e] += lo.x * c.res_scale;
                    v[16 * h + 4 * e + 1] += lo.y * c.res_scale;
                    v[16 * h + 4 * e + 2] += hi.x * c.res_scale;
                    v[16 * h + 4 * e + 3] += hi.y * c.res_scale;
                  }
                }
                uint32_t pk[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                  const float* w = v + 16 * h + 4 * e;
                  pk[e] = valid ? (e4m3x2(w[0] * c.out_inv_scale, w[1] * c.out_inv_scale) |
                                   (e4m3x2(w[2] * c.out_inv_scale, w[3] * c.out_inv_scale) << 16))
                                : 0u;
                }
                outv[h] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
              }
            } else {
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                float* t = v + 8 * u;
                if (use_res) {
                  const uint32_t rv[4] = {rq[u].x, rq[u].y, rq[u].z, rq[u].w};
#pragma unroll
                  for (int e = 0; e < 4; ++e) {
                    const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&rv[e]));
                    t[2 * e] += f.x;
                    t[2 * e + 1] += f.y;
                  }
                }
                uint32_t pk[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) pk[e] = pack_bf16x2(t[2 * e], t[2 * e + 1]) & vmask;
                outv[u] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
              }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (u < nu) *reinterpret_cast<uint4*>(qa[u]) = outv[u];
          }
          if (p == p_end - 1) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {                   // accumulator buffer free for the MMA
              if (CG == 2)
                mbar_arrive_cluster(acc_empty_leader0 + buf * 8u);
              else
                mbar_arrive(&acc_empty[buf]);
            }
          }
          fence_proxy_async();               // staging writes visible to the TMA store
          named_bar(bar_id, 128);
          if (elected && ok && live && !aborted(&s_abort)) {
            for (int j = 0; j < nsub; ++j) {
              const int ch = tc.n0 + p * Cfg::SWC + j * sub_ch;
              // in place over the residual: the tile is added to it (the residual add of the block)
              if (!patch_mode(a.mode)) {
                if (a.red_res)
                  tma_reduce_add_2d(&plan.o, stg + j * sub_bytes, ch, tc.m0 + mrow);
                else
                  tma_store_2d(&plan.o, stg + j * sub_bytes, ch, tc.m0 + mrow);
              } else {
                if (a.red_res)
                  tma_reduce_add_4d(&plan.o, stg + j * sub_bytes, ch, tc.ox0 + 1, tc.oy0 + 1, tc.img);
                else
                  tma_store_4d(&plan.o, stg + j * sub_bytes, ch, tc.ox0 + 1, tc.oy0 + 1, tc.img);
              }
            }
            bulk_commit();
          }
        }
      } else {
        // direct: one pixel row per thread (f32 heads, upsampled laterals)
        if (!ok || aborted(&s_abort)) valid = false;
#pragma unroll 1
        for (int c0 = Cfg::SPLIT ? g * (BN / 2) : 0; c0 < (Cfg::SPLIT ? (g + 1) * (BN / 2) : BN); c0 += 32) {
          uint32_t r[32];
          tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + buf * Cfg::ACC + (uint32_t)c0, r);
          tmem_ld_wait();
          const int ch0 = tc.n0 + c0;
          if (valid && ch0 < c.cout) {
            const int nvalid = min(32, c.cout - ch0);
            float v[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const float acc = Q ? __uint_as_float(r[j]) * sMult[c0 + j] : __uint_as_float(r[j]);
              const float t = acc + sBias[c0 + j];
              v[j] = c.act ? leaky01f(t) : t;
            }
            if (c.res.ptr) {
              const size_t ro = tview_off(c.res, n, y, x) + ch0;
#pragma unroll
              for (int j = 0; j < 32; ++j)
                if (j < nvalid) {
                  if (c.res.dtype == 2) {
                    const uint8_t code = static_cast<const uint8_t*>(c.res.ptr)[ro + j];
                    v[j] += e4m3x2_to_float2(code).x * c.res_scale;
                  } else {
                    v[j] += __bfloat162float(static_cast<const __nv_bfloat16*>(c.res.ptr)[ro + j]);
                  }
                }
            }
            store_chunk(c, n, y, x, ch0, nvalid, v);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          if (CG == 2)
            mbar_arrive_cluster(acc_empty_leader0 + buf * 8u);
          else
            mbar_arrive(&acc_empty[buf]);
        }
      }
      if (!ok) break;
    }
    if (elected) bulk_wait0();               // stores done before the CTA (and its smem) goes away
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if constexpr (CG == 2) cluster_sync();   // no CTA leaves while its peer may still signal it
  if (warp == GW) {
    if constexpr (CG == 2)
      tmem_dealloc_pair(tmem, Cfg::TMEM_COLS);
    else
      tmem_dealloc(tmem, Cfg::TMEM_COLS);
  }
}

// ----------------------------------------------------------------------------- host side
// mode 4: weight-ring depth, and the shared memory of an instantiation besides its windows
// E4M3 weight tiles are consumed twice as fast (K = 32 per MMA), so their ring is deeper
constexpr int W4_STAGES = 8;
constexpr int W4_STAGES_Q = 12;
constexpr int W4M2_STAGES = 12;   // two sub-tiles: half-size weight tiles (64 rows per CTA), each used twice
// 128-byte window rows: 16 KB weight tiles, 512 MMA cycles each; the deeper ring where two windows
// still fit next to it (the narrower images), else the shallower one
constexpr int W4W_STAGES = 5;
constexpr int W4W_STAGES_DEEP = 7;
template <int BN, int BKC, int CG, int Q, int WM, int SW = W4W_STAGES>
constexpr int w4_fixed() {
  constexpr int S = BKC == 64 ? SW : WM == 2 ? W4M2_STAGES : (Q ? W4_STAGES_Q : W4_STAGES);
  using C = TcCfg<BN, BKC, S, CG, Q, WM>;
  return S * C::B_BYTES + 2 * C::SDEPTH * C::C_BYTES + 1024 + C::BAR_BYTES + C::BIAS_BYTES;
}
int w4_fixed_bytes(int bn, int q, int msub, int wide, int deep = 0) {
  if (wide && deep) return q ? w4_fixed<256, 64, 2, 1, 1, W4W_STAGES_DEEP>() : w4_fixed<256, 64, 2, 0, 1, W4W_STAGES_DEEP>();
  if (wide) return q ? w4_fixed<256, 64, 2, 1, 1>() : w4_fixed<256, 64, 2, 0, 1>();
  if (msub == 2) return q ? w4_fixed<128, 32, 2, 1, 2>() : w4_fixed<128, 32, 2, 0, 2>();
  if (bn == 128) return q ? w4_fixed<128, 32, 2, 1, 1>() : w4_fixed<128, 32, 2, 0, 1>();
  return q ? w4_fixed<256, 32, 2, 1, 1>() : w4_fixed<256, 32, 2, 0, 1>();
}
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// bkc: elements of the innermost box dimension; its bytes (2 per bf16, 1 per E4M3 code when u8)
// choose the swizzle: 128 -> 128-byte, 64 -> 64-byte, 32 -> 32-byte, otherwise none.
// f32: the box's inner extent `bkc` counts f32 elements (4 bytes each).
bool encode(CUtensorMap* m, int rank, void* base, const cuuint64_t* dims, const cuuint64_t* strides_bytes,
            const cuuint32_t* box, int bkc, bool u8 = false, bool f32 = false) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint32_t es[5] = {1, 1, 1, 1, 1};
  const int row_bytes = bkc * (f32 ? 4 : (u8 ? 1 : 2));
  const CUtensorMapSwizzle swz = row_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                 : row_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                 : row_bytes == 32 ? CU_TENSOR_MAP_SWIZZLE_32B
                                                   : CU_TENSOR_MAP_SWIZZLE_NONE;
  const CUtensorMapDataType dt = f32  ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : u8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                      : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  CUresult r = fn(m, dt, (cuuint32_t)rank, base,
                  dims, strides_bytes, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Per-device launch facts (SM count, kernel attributes, cluster occupancy) are cached per device
// ordinal under one mutex: a process may drive several GPUs, from several host threads.
std::mutex g_launch_mutex;

int current_device() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  return dev >= 0 && dev < JDE_MAX_DEVICES ? dev : -1;
}

int sm_count(int dev) {
  static int n[JDE_MAX_DEVICES] = {0};
  std::lock_guard<std::mutex> lock(g_launch_mutex);
  if (!n[dev]) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
    n[dev] = v;
  }
  return n[dev];
}

template <int BN, int BKC, int STAGES, int GW = 1, int CG = 1, int Q = 0, int WM = 0>
cudaError_t launch_cfg(const TcPlan& p, const TcArgs& a, cudaStream_t st, int smem = 0) {
  using Cfg = TcCfg<BN, BKC, STAGES, CG, Q, WM>;
  auto kernel = conv_tc_kernel<BN, BKC, STAGES, GW, CG, Q, WM>;
  if (!smem) smem = Cfg::SMEM;
  const int dev = current_device();
  if (dev < 0) return cudaErrorInvalidDevice;
  const int sms = sm_count(dev);
  // the dynamic shared-memory attribute is a per-device property of the kernel
  static int attr_set[JDE_MAX_DEVICES] = {0};
  {
    std::lock_guard<std::mutex> lock(g_launch_mutex);
    if (attr_set[dev] < smem) {
      cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return e;
      attr_set[dev] = smem;
    }
  }
  // p.pdl: a programmatic dependent of the kernel before it in the stream (its set-up overlaps that
  // kernel's last work units; the kernel waits for it before touching global memory)
  cudaLaunchAttribute dep;
  dep.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  dep.val.programmaticStreamSerializationAllowed = 1;
  if (CG == 1) {
    const int tiles = p.m_tiles * p.n_tiles;
    const int grid = tiles < sms ? tiles : sms;
    jde_count_launch();
    if (!p.pdl) {
      kernel<<<grid, tc_threads(GW), smem, st>>>(p, a);
      return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg1 = {};
    cfg1.gridDim = dim3(grid);
    cfg1.blockDim = dim3(tc_threads(GW));
    cfg1.dynamicSmemBytes = (size_t)smem;
    cfg1.stream = st;
    cfg1.attrs = &dep;
    cfg1.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg1, kernel, p, a);
  }
  // CTA pairs: 2-CTA clusters, as many as can be resident at once (persistent)
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(tc_threads(GW));
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  static int max_clusters[JDE_MAX_DEVICES] = {0};
  int mc;
  {
    std::lock_guard<std::mutex> lock(g_launch_mutex);
    if (!max_clusters[dev]) {
      cfg.gridDim = dim3(2 * (sms / 2));
      int n = 0;
      if (cudaOccupancyMaxActiveClusters(&n, kernel, &cfg) != cudaSuccess || n < 1) {
        cudaGetLastError();
        n = sms / 2;
      }
      max_clusters[dev] = n;
    }
    mc = max_clusters[dev];
  }
  const int clusters = a.total_units < mc ? a.total_units : mc;
  cfg.gridDim = dim3(2 * clusters);
  if (p.pdl) {
    attr[1] = dep;
    cfg.numAttrs = 2;
  }
  jde_count_launch();
  return cudaLaunchKernelEx(&cfg, kernel, p, a);
}

}  // namespace

int conv_tc_pick_bn(int cout) {
  if (cout <= 32) return 32;
  if (cout <= 64) return 64;
  if (cout <= 128) return 128;
  return 256;
}

bool conv_tc_plan(TcPlan& plan, const ConvSpec& c, const void* w_any, int cout_pad, int bn, char* msg,
                  size_t msg_len, int msub, int pair128) {
  const __nv_bfloat16* w = static_cast<const __nv_bfloat16*>(w_any);
  plan = TcPlan();
  plan.spec = c;
  plan.msub = 1;
  if (msub != 1 && (msub != 2 || bn != 128 || c.k != 3 || c.stride != 1)) {
    snprintf(msg, msg_len, "two M sub-tiles: flat-window 3x3 convs with 128-wide tiles only");
    return false;
  }
  if (c.cin == 3 && c.k == 3 && c.stride == 1 && c.in.dtype == 1 && c.in.pad == 1 && c.in.pixstride == 4 &&
      (bn == 32 || bn == 64)) {
    // stem: im2col rows gathered in the kernel (K = 27 padded to 32), flat over the padded image
    plan.mode = 2;
    plan.bn = bn;
    plan.bkc = 32;
    plan.cin_blocks = 1;
    plan.kt_total = 1;
    plan.n_tiles = cout_pad / bn;
    plan.Hp = c.in.h + 2;
    plan.Wp = c.in.w + 2;
    plan.M_total = c.in.n * plan.Hp * plan.Wp;
    plan.m_tiles = (plan.M_total + 127) / 128;
    cuuint64_t dims[2] = {32, (cuuint64_t)cout_pad};
    cuuint64_t strides[1] = {32 * 2};
    cuuint32_t box[2] = {32, (cuuint32_t)bn};
    bool ok = encode(&plan.b, 2, const_cast<__nv_bfloat16*>(w), dims, strides, box, 32);
    const int sub = bn < 64 ? bn : 64;
    plan.tma_out = c.out.dtype == 1 && c.out.pad == 1 && !c.upsample && c.cout % sub == 0;
    if (plan.tma_out) {
      cuuint64_t od[2] = {(cuuint64_t)c.cout, (cuuint64_t)plan.M_total};
      cuuint64_t os[1] = {(cuuint64_t)c.out.pixstride * 2};
      cuuint32_t ob[2] = {(cuuint32_t)sub, 128};
      ok &= encode(&plan.o, 2, c.out.ptr, od, os, ob, sub);
    }
    if (!ok) snprintf(msg, msg_len, "cuTensorMapEncodeTiled failed (stem)");
    return ok;
  }
  // window mode: 32-channel 3x3 convs (64-byte pixels, two K=16 MMAs per tap)
  if (c.cin == 32 && bn == 64 && c.cout == 64 && c.k == 3 && cout_pad == bn && c.in.dtype == 1 && c.in.pad == 1 &&
      c.out.dtype == 1 && c.out.pad == 1 && !c.upsample) {
    // the input window of each 8-wide, 16-high output patch
    plan.mode = 3;
    plan.bn = bn;
    plan.bkc = 64;
    plan.cin_blocks = 1;
    plan.kt_total = 5;                          // resident weights: 9 taps x 32 channels, padded to 320
    plan.n_tiles = 1;
    plan.TW = 8;
    plan.TH = 16;
    plan.tiles_x = (c.Wo + plan.TW - 1) / plan.TW;
    plan.tiles_y = (c.Ho + plan.TH - 1) / plan.TH;
    plan.m_tiles = c.in.n * plan.tiles_x * plan.tiles_y;
    const int st = c.stride;
    plan.WW = st == 1 ? plan.TW + 2 : plan.TW + 1;   // (sub-)window width in pixels
    plan.WH = st == 1 ? plan.TH + 2 : plan.TH + 1;
    // every plane is a TMA destination: its shared-memory address must be 128-byte aligned
    plan.plane = (plan.WW * plan.WH * 64 + 1023) / 1024 * 1024;
    plan.win_bytes = (st == 1 ? 1 : 4) * plan.plane;
    {
      // as many window buffers as shared memory holds next to the resident weights and the two
      // staging tiles per epilogue group (at most MAX_WIN)
      const int fixed = plan.kt_total * bn * 64 * 2 + 2 * 2 * 128 * bn * 2 + 1024 + 768 + 2 * bn * 4;
      plan.nwin = (227 * 1024 - 64 - fixed) / plan.win_bytes;
      if (plan.nwin > MAX_WIN) plan.nwin = MAX_WIN;
    }
    if (plan.nwin < 2) {
      snprintf(msg, msg_len, "window ring does not fit in shared memory");
      return false;
    }
    if (plan.plane % 1024 || plan.win_bytes % 1024) {
      snprintf(msg, msg_len, "window planes not 128-byte aligned");
      return false;
    }
    const int Hp = c.in.h + 2, Wp = c.in.w + 2;
    plan.Hp = Hp;
    plan.Wp = Wp;
    bool ok = true;
    const size_t ps = (size_t)c.in.pixstride;
    for (int par = 0; par < (st == 2 ? 4 : 1); ++par) {
      // 4-D view (32 channels, x, y, image), 64-byte swizzle; stride 2: parity sub-lattice (py, px)
      const int py = par >> 1, px = par & 1;
      const int ch = 32;
      void* base = static_cast<__nv_bfloat16*>(c.in.ptr) + (st == 2 ? ((size_t)py * Wp + px) * ps : 0);
      cuuint64_t dims[4] = {(cuuint64_t)ch, (cuuint64_t)(st == 2 ? Wp / 2 : Wp), (cuuint64_t)(st == 2 ? Hp / 2 : Hp),
                            (cuuint64_t)c.in.n};
      cuuint64_t strides[3] = {(cuuint64_t)st * ps * 2, (cuuint64_t)st * Wp * ps * 2, (cuuint64_t)Hp * Wp * ps * 2};
      cuuint32_t box[4] = {(cuuint32_t)ch, (cuuint32_t)plan.WW, (cuuint32_t)plan.WH, 1};
      ok &= encode(&plan.a[par], 4, base, dims, strides, box, ch);
    }
    {
      const int Kt = plan.kt_total * 64;
      cuuint64_t dims[2] = {(cuuint64_t)Kt, (cuuint64_t)bn};
      cuuint64_t strides[1] = {(cuuint64_t)Kt * 2};
      cuuint32_t box[2] = {64, (cuuint32_t)bn};
      ok &= encode(&plan.b, 2, const_cast<__nv_bfloat16*>(w), dims, strides, box, 64);
    }
    plan.tma_out = 1;
    {
      cuuint64_t dims[4] = {(cuuint64_t)c.cout, (cuuint64_t)(c.Wo + 2), (cuuint64_t)(c.Ho + 2), (cuuint64_t)c.out.n};
      cuuint64_t strides[3] = {(cuuint64_t)c.out.pixstride * 2, (cuuint64_t)(c.Wo + 2) * c.out.pixstride * 2,
                               (cuuint64_t)(c.Ho + 2) * (c.Wo + 2) * c.out.pixstride * 2};
      cuuint32_t box[4] = {(cuuint32_t)bn, (cuuint32_t)plan.TW, (cuuint32_t)plan.TH, 1};
      ok &= encode(&plan.o, 4, c.out.ptr, dims, strides, box, bn);
    }
    plan.red_res = c.res.ptr != nullptr && c.res.ptr == c.out.ptr && c.res.dtype == 1 &&
                   c.res.pixstride == c.out.pixstride && c.res.pad == 1;
    plan.tma_res = !plan.red_res && c.res.ptr != nullptr && c.res.dtype == 1 && c.res.pad == 1;
    if (plan.tma_res) {
      cuuint64_t dims[4] = {(cuuint64_t)c.cout, (cuuint64_t)(c.Wo + 2), (cuuint64_t)(c.Ho + 2), (cuuint64_t)c.res.n};
      cuuint64_t strides[3] = {(cuuint64_t)c.res.pixstride * 2, (cuuint64_t)(c.Wo + 2) * c.res.pixstride * 2,
                               (cuuint64_t)(c.Ho + 2) * (c.Wo + 2) * c.res.pixstride * 2};
      cuuint32_t box[4] = {(cuuint32_t)bn, (cuuint32_t)plan.TW, (cuuint32_t)plan.TH, 1};
      ok &= encode(&plan.r, 4, c.res.ptr, dims, strides, box, bn);
    }
    if (!ok) snprintf(msg, msg_len, "cuTensorMapEncodeTiled failed (32-channel window conv)");
    return ok;
  }
  // k-block: 128-byte rows (64 bf16 or 128 E4M3 elements), or 64-byte rows for narrower inputs
  const bool q = c.q != 0;
  const int ie = q ? 1 : 2;                 // bytes per input / weight element
  const int kel = q ? ((c.cin % 128 == 0) ? 128 : (c.cin % 64 == 0 ? 64 : 0))
                    : ((c.cin % 64 == 0) ? 64 : (c.cin % 32 == 0 ? 32 : 0));
  const int bkc = q ? kel / 2 : kel;        // the kernel's row unit: row bytes / 2
  const bool o8 = c.out.dtype == 2;
  if (!kel || c.in.dtype != (q ? 2 : 1) || c.in.pad != 1 || !(c.k == 1 || c.k == 3) ||
      !(c.stride == 1 || c.stride == 2) || (c.stride == 2 && c.k != 3) ||
      (bn != 32 && bn != 64 && bn != 128 && bn != 256) || cout_pad % bn || (o8 && bn < 64) ||
      (q && c.out.dtype == 1)) {
    snprintf(msg, msg_len, "tensor-core conv: unsupported shape cin=%d k=%d s=%d bn=%d q=%d out=%d", c.cin, c.k,
             c.stride, bn, (int)q, c.out.dtype);
    return false;
  }
  plan.bn = bn;
  plan.bkc = bkc;
  plan.kel = kel;
  plan.q = q;
  plan.cin_blocks = c.cin / kel;
  plan.kt_total = c.k * c.k * plan.cin_blocks;
  plan.n_tiles = cout_pad / bn;
  const int K = c.k * c.k * c.cin;
  const int Hp = c.in.h + 2, Wp = c.in.w + 2;
  plan.Hp = Hp;
  plan.Wp = Wp;
  void* base = c.in.ptr;
  bool ok = true;
  if (c.stride == 1) {
    plan.mode = 0;
    plan.M_total = c.in.n * Hp * Wp;
    plan.m_tiles = (plan.M_total + 127) / 128;
    // 3x3 with 128- or 256-wide tiles: flat windows (mode 4) when at least two fit in shared memory
    // (measured: E4M3 convs of two 64-byte k-blocks, 128 input channels, run faster flat)
    // 256-wide tiles take 128-byte k-blocks (64 bf16 / 128 E4M3 channels) when two such windows fit:
    // half the TMA rows per byte, the 128-byte swizzle; otherwise 64-byte k-blocks
    const int wide0 = bn == 256 && msub == 1 && c.cin % (q ? 128 : 64) == 0;
    for (int wide = wide0; wide >= 0 && plan.mode != 4; --wide) {
      const int kel4 = q ? (wide ? 128 : 64) : (wide ? 64 : 32);   // channels per k-block
      const int rowb = wide ? 128 : 64;                             // bytes per window row
      if (!(c.k == 3 && (bn == 128 || bn == 256) && c.cin % kel4 == 0 && !(q && !wide && c.cin / kel4 == 2)))
        continue;
      const int npx = 128 * msub + 2 * Wp + 2;   // rows m0 - Wp - 1 .. m0 + 128 msub + Wp
      const int wnb = (npx + 255) / 256;     // a TMA box spans at most 256 rows
      const int whb = ((npx + wnb - 1) / wnb + 15) / 16 * 16;   // rows per box: 1024-byte multiples
      const int win_bytes = wnb * whb * rowb;
      int deep = wide && (227 * 1024 - 64 - w4_fixed_bytes(bn, q, msub, wide, 1)) / win_bytes >= 2;
      int nwin = (227 * 1024 - 64 - w4_fixed_bytes(bn, q, msub, wide, deep)) / win_bytes;
      if (nwin > MAX_WIN) nwin = MAX_WIN;
      if (nwin >= 2) {
        plan.mode = 4;
        plan.w4deep = deep;
        plan.msub = msub;
        plan.m_tiles = (plan.M_total + 128 * msub - 1) / (128 * msub);
        plan.wnb = wnb;
        plan.whb = whb;
        plan.win_bytes = win_bytes;
        plan.nwin = nwin;
        plan.kel = kel4;
        plan.bkc = rowb / 2;
        plan.cin_blocks = c.cin / kel4;
        plan.kt_total = 9 * plan.cin_blocks;
      }
    }
    cuuint64_t dims[2] = {(cuuint64_t)c.cin, (cuuint64_t)plan.M_total};
    cuuint64_t strides[1] = {(cuuint64_t)c.in.pixstride * ie};
    cuuint32_t box[2] = {(cuuint32_t)plan.kel, plan.mode == 4 ? (cuuint32_t)plan.whb : 128u};
    ok &= encode(&plan.a[0], 2, base, dims, strides, box, plan.kel, q);
  } else {
    plan.mode = 1;
    if ((c.in.h & 1) || (c.in.w & 1)) {
      snprintf(msg, msg_len, "tensor-core conv: stride-2 input must have even size");
      return false;
    }
    // output patch shape: 128 pixels, widest tile that keeps the waste lowest
    int best_tw = 128, best_cost = 1 << 30;
    for (int tw = 8; tw <= 128; tw *= 2) {
      const int th = 128 / tw;
      const int cost = ((c.Wo + tw - 1) / tw) * tw * ((c.Ho + th - 1) / th) * th;
      if (cost < best_cost) best_cost = cost, best_tw = tw;
    }
    plan.TW = best_tw;
    plan.TH = 128 / best_tw;
    plan.tiles_x = (c.Wo + plan.TW - 1) / plan.TW;
    plan.tiles_y = (c.Ho + plan.TH - 1) / plan.TH;
    plan.m_tiles = c.in.n * plan.tiles_x * plan.tiles_y;
    for (int py = 0; py < 2; ++py)
      for (int px = 0; px < 2; ++px) {
        void* pb = static_cast<uint8_t*>(base) + ((size_t)py * Wp + px) * c.in.pixstride * ie;
        cuuint64_t dims[4] = {(cuuint64_t)c.cin, (cuuint64_t)(Wp / 2), (cuuint64_t)(Hp / 2), (cuuint64_t)c.in.n};
        cuuint64_t strides[3] = {(cuuint64_t)2 * c.in.pixstride * ie, (cuuint64_t)2 * Wp * c.in.pixstride * ie,
                                 (cuuint64_t)Hp * Wp * c.in.pixstride * ie};
        cuuint32_t box[4] = {(cuuint32_t)kel, (cuuint32_t)plan.TW, (cuuint32_t)plan.TH, 1};
        ok &= encode(&plan.a[py * 2 + px], 4, pb, dims, strides, box, kel, q);
      }
  }
  // 256-wide tiles run on CTA pairs (M = 256 per MMA, each CTA loads half of B)
  // CTA pairs: 256-wide tiles, and every flat-window tile (each CTA holds half of the weight tile)
  plan.cg = (bn == 256 && (bkc == 64 || plan.mode == 4)) || (bn == 128 && plan.mode == 4) ? 2 : 1;
  if (pair128) {
    if (bn != 128 || bkc != 64 || q || !(plan.mode == 0 || plan.mode == 1)) {
      snprintf(msg, msg_len, "128-wide tiles on CTA pairs: stride-1 flat or stride-2 BF16 convs of 128-byte k-blocks only");
      return false;
    }
    plan.cg = 2;
  }
  {
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)cout_pad};
    cuuint64_t strides[1] = {(cuuint64_t)K * ie};
    cuuint32_t box[2] = {(cuuint32_t)plan.kel, (cuuint32_t)(bn / plan.cg)};
    ok &= encode(&plan.b, 2, const_cast<void*>(w_any), dims, strides, box, plan.kel, q);
  }
  // TMA-stored epilogue: bf16 or E4M3 padded outputs written in place (no upsample), channel
  // count a multiple of the store box (64 channels, or 32 for 32-wide bf16 tiles)
  const int sub = o8 ? 64 : (bn < 64 ? bn : 64);
  const int oe = o8 ? 1 : 2;
  plan.tma_out = (c.out.dtype == 1 || o8) && !c.upsample && c.out.pad == 1 && c.cout % sub == 0;
  // f32 outputs (padded embedding heads) of flat tiles: boxes of fw channels (64- or 128-byte rows)
  const int fw = q ? 16 : 32;
  const bool o32 = c.out.dtype == 0 && !c.upsample && c.out.pad == 1 && bn >= 64 && c.cout % fw == 0 &&
                   (plan.mode == 0 || plan.mode == 4);
  if (o32) plan.tma_out = 1;
  // residual stored in place under the output (bf16): added by the store itself (TMA reduce-add)
  plan.red_res = plan.tma_out && c.res.ptr != nullptr && c.res.ptr == c.out.ptr && c.out.dtype == 1 &&
                 c.res.dtype == 1 && c.res.pixstride == c.out.pixstride && c.res.pad == 1;
  plan.tma_res = !plan.red_res && plan.tma_out && c.res.ptr != nullptr && c.stride == 1 &&
                 c.res.dtype == c.out.dtype && c.res.pad == 1;
  if (q && !o8 && !o32 && plan.tma_out) {
    snprintf(msg, msg_len, "E4M3 conv: staged outputs must be E4M3");
    return false;
  }
  if (plan.tma_out) {
    const int Ho = c.Ho, Wo = c.Wo;
    if (o32) {
      cuuint64_t dims[2] = {(cuuint64_t)c.cout, (cuuint64_t)plan.M_total};
      cuuint64_t strides[1] = {(cuuint64_t)c.out.pixstride * 4};
      cuuint32_t box[2] = {(cuuint32_t)fw, 128};
      ok &= encode(&plan.o, 2, c.out.ptr, dims, strides, box, fw, false, true);
    } else if (plan.mode == 0 || plan.mode == 4) {
      cuuint64_t dims[2] = {(cuuint64_t)c.cout, (cuuint64_t)plan.M_total};
      cuuint64_t strides[1] = {(cuuint64_t)c.out.pixstride * oe};
      cuuint32_t box[2] = {(cuuint32_t)sub, 128};
      ok &= encode(&plan.o, 2, c.out.ptr, dims, strides, box, sub, o8);
    } else {
      cuuint64_t dims[4] = {(cuuint64_t)c.cout, (cuuint64_t)(Wo + 2), (cuuint64_t)(Ho + 2), (cuuint64_t)c.out.n};
      cuuint64_t strides[3] = {(cuuint64_t)c.out.pixstride * oe, (cuuint64_t)(Wo + 2) * c.out.pixstride * oe,
                               (cuuint64_t)(Ho + 2) * (Wo + 2) * c.out.pixstride * oe};
      cuuint32_t box[4] = {(cuuint32_t)sub, (cuuint32_t)plan.TW, (cuuint32_t)plan.TH, 1};
      ok &= encode(&plan.o, 4, c.out.ptr, dims, strides, box, sub, o8);
    }
  }
  if (plan.tma_res) {
    cuuint64_t dims[2] = {(cuuint64_t)c.cout, (cuuint64_t)plan.M_total};
    cuuint64_t strides[1] = {(cuuint64_t)c.res.pixstride * oe};
    cuuint32_t box[2] = {(cuuint32_t)sub, 128};
    ok &= encode(&plan.r, 2, c.res.ptr, dims, strides, box, sub, o8);
  }
  if (!ok) {
    snprintf(msg, msg_len, "cuTensorMapEncodeTiled failed (cin=%d k=%d s=%d)", c.cin, c.k, c.stride);
    return false;
  }
  return true;
}

bool conv_tc_retarget(TcPlan& p, void* out) {
  p.spec.out.ptr = out;
  if (!p.tma_out) return true;
  if (p.spec.out.dtype != 0 || !(p.mode == 0 || p.mode == 4)) return false;   // only f32 heads move
  const int fw = p.q ? 16 : 32;
  cuuint64_t dims[2] = {(cuuint64_t)p.spec.cout, (cuuint64_t)p.M_total};
  cuuint64_t strides[1] = {(cuuint64_t)p.spec.out.pixstride * 4};
  cuuint32_t box[2] = {(cuuint32_t)fw, 128};
  return encode(&p.o, 2, out, dims, strides, box, fw, false, true);
}

cudaError_t conv_tc_launch(const TcPlan& p, cudaStream_t st) {
  TcArgs a;
  a.mode = p.mode;
  a.k = p.spec.k;
  a.cin_blocks = p.cin_blocks;
  a.kt_total = p.kt_total;
  a.M_total = p.M_total;
  a.Hp = p.Hp;
  a.Wp = p.Wp;
  a.TW = p.TW;
  a.TH = p.TH;
  a.tiles_x = p.tiles_x;
  a.tiles_y = p.tiles_y;
  a.n_tiles = p.n_tiles;
  a.total_tiles = p.m_tiles * p.n_tiles;
  a.total_units = p.cg == 2 ? (p.m_tiles + 1) / 2 * p.n_tiles : a.total_tiles;
  a.tma_out = p.tma_out;
  a.tma_res = p.tma_res;
  a.red_res = p.red_res;
  a.stride = p.spec.stride;
  a.WW = p.WW;
  a.WH = p.WH;
  a.win_bytes = p.win_bytes;
  a.nwin = p.nwin;
  a.kel = p.kel ? p.kel : p.bkc;
  a.plane = p.plane;
  a.plane_tx = p.WW * p.WH * 64;
  a.wnb = p.wnb;
  a.whb = p.whb;
  a.msub = p.msub > 1 ? p.msub : 1;
  a.c = p.spec;
  if (p.mode == 2) {
    if (p.bn == 32) return launch_cfg<32, 32, 16, 4>(p, a, st);
    if (p.bn == 64) return launch_cfg<64, 32, 12, 4>(p, a, st);
    return cudaErrorInvalidValue;
  }
  if (p.mode == 4) {
    const int wide = p.bkc == 64;
    const int smem = p.nwin * p.win_bytes + w4_fixed_bytes(p.bn, p.q, p.msub, wide, p.w4deep);
    if (smem > 227 * 1024 - 64) return cudaErrorInvalidValue;
    if (wide) {
      if (p.bn != 256 || p.cg != 2 || p.msub != 1) return cudaErrorInvalidValue;
      if (p.w4deep)
        return p.q ? launch_cfg<256, 64, W4W_STAGES_DEEP, 1, 2, 1, 1>(p, a, st, smem)
                   : launch_cfg<256, 64, W4W_STAGES_DEEP, 1, 2, 0, 1>(p, a, st, smem);
      return p.q ? launch_cfg<256, 64, W4W_STAGES, 1, 2, 1, 1>(p, a, st, smem)
                 : launch_cfg<256, 64, W4W_STAGES, 1, 2, 0, 1>(p, a, st, smem);
    }
    if (p.msub == 2) {
      if (p.bn != 128 || p.cg != 2 || !p.tma_out) return cudaErrorInvalidValue;
      return p.q ? launch_cfg<128, 32, W4M2_STAGES, 1, 2, 1, 2>(p, a, st, smem)
                 : launch_cfg<128, 32, W4M2_STAGES, 1, 2, 0, 2>(p, a, st, smem);
    }
    if (p.bn == 128 && p.cg == 2)
      return p.q ? launch_cfg<128, 32, W4_STAGES_Q, 1, 2, 1, 1>(p, a, st, smem)
                 : launch_cfg<128, 32, W4_STAGES, 1, 2, 0, 1>(p, a, st, smem);
    if (p.bn == 256 && p.cg == 2)
      return p.q ? launch_cfg<256, 32, W4_STAGES_Q, 1, 2, 1, 1>(p, a, st, smem)
                 : launch_cfg<256, 32, W4_STAGES, 1, 2, 0, 1>(p, a, st, smem);
    return cudaErrorInvalidValue;
  }
  if (p.mode == 3) {
    if (p.bn == 64) {
      using Cfg8 = TcCfg<64, 64, 6>;
      const int smem = p.nwin * p.win_bytes + p.kt_total * Cfg8::B_BYTES + 2 * Cfg8::SDEPTH * Cfg8::C_BYTES + 1024 +
                       Cfg8::BAR_BYTES + Cfg8::BIAS_BYTES;
      if (smem > 227 * 1024 - 64) return cudaErrorInvalidValue;
      return launch_cfg<64, 64, 6, 1>(p, a, st, smem);
    }
    return cudaErrorInvalidValue;
  }
  if (p.q) {
    // E4M3 operands: 64-bf16-unit rows hold 128 codes, 32-unit rows 64 codes
    if (p.bkc == 64) {
      switch (p.bn) {
        case 32: return launch_cfg<32, 64, 10, 1, 1, 1>(p, a, st);
        case 64: return launch_cfg<64, 64, 8, 1, 1, 1>(p, a, st);
        case 128: return launch_cfg<128, 64, 5, 1, 1, 1>(p, a, st);
        case 256:
          if (p.cg == 2) return launch_cfg<256, 64, 5, 1, 2, 1>(p, a, st);
          break;
      }
    } else if (p.bkc == 32 && p.bn == 128) {
      return launch_cfg<128, 32, 11, 1, 1, 1>(p, a, st);
    }
    return cudaErrorInvalidValue;
  }
  if (p.bkc == 64) {
    switch (p.bn) {
      case 32: return launch_cfg<32, 64, 9>(p, a, st);
      case 64: return launch_cfg<64, 64, 6>(p, a, st);
      case 128:
        if (p.cg == 2) return launch_cfg<128, 64, 8, 1, 2>(p, a, st);
        return launch_cfg<128, 64, 5>(p, a, st);
      case 256:
        if (p.cg == 2) return launch_cfg<256, 64, 4, 1, 2>(p, a, st);
        return launch_cfg<256, 64, 3>(p, a, st);
    }
  } else {
    switch (p.bn) {
      case 32: return launch_cfg<32, 32, 16>(p, a, st);
      case 64: return launch_cfg<64, 32, 12>(p, a, st);
      case 128: return launch_cfg<128, 32, 10>(p, a, st);
      case 256: return launch_cfg<256, 32, 6>(p, a, st);
    }
  }
  return cudaErrorInvalidValue;
}
