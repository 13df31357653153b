// The stem (3x3, 3 -> 32, stride 1) and the first stride-2 conv (3x3, 32 -> 64) of the backbone
// (Sec. 3.1, DarkNet-53) fused into one persistent tcgen05 kernel: the stem's output, the largest
// tensor of the network, never leaves shared memory.
//
// Work unit: one TW x TH = 8 x 16 patch of the stride-2 conv's output (M = 128).  It reads the stem
// output on a (2 TH + 1) x (2 TW + 1) = 33 x 17 window, which needs the letterbox on a 35 x 19 window.
// Per unit:
//   * warp 0 / lane 0 loads the letterbox window (RGB0 bf16, 8 bytes per pixel) with one TMA box;
//   * eight gather warps build the stem's im2col rows of the 561 window pixels (27 values, (ky, kx, c)
//     order, then three 1.0 columns, padded to 32 bf16) in five 128-row, 64-byte-swizzled operand
//     tiles in shared memory, one row per thread: warps 1-4 fill tiles 0, 2 and 4, warps 14-17
//     tiles 1 and 3, each tile with its own full / empty barriers, so a tile is refilled for the next
//     unit as soon as its own MMAs are done; a pixel outside the image gets an all-zero row;
//   * the MMA warp issues the stem GEMM (5 tiles x M=128, N=32, K=32) into TMEM: the stem weights carry
//     the folded BN bias in their K columns 27..29, split into three bfloat16 parts whose sum is the
//     float32 bias, so the accumulator holds conv + bias, and exactly zero outside the image (the
//     stride-2 conv's zero padding); then the stride-2 conv of the previous unit (9 taps x two K=16
//     MMAs, M=128, N=64, plus one K=16 MMA of a constant-ones tile against its bias parts), whose A
//     operand is the same four-parity-plane window layout as the 32-channel window mode of the
//     unfused kernel;
//   * four stem-epilogue warps read the stem accumulators, apply leaky-ReLU and store the bf16 values
//     into the parity planes (64-byte swizzle by absolute address);
//   * four output-epilogue warps read the stride-2 conv's accumulators, apply leaky-ReLU, round to
//     bf16 into a 128-byte-swizzled staging tile and TMA-store it.
// The epilogues therefore do no per-element bias add and no per-element select.
// Letterbox windows, stem accumulators, parity windows and output accumulators are double-buffered;
// the im2col tiles are single-buffered, handed over tile by tile.  Every wait is bounded: on a
// timeout the CTA flags the error word, stops issuing work, and releases TMEM.
#include <stdio.h>

#include <mutex>

#include "internal.h"

namespace {

constexpr int F_TW = 8, F_TH = 16;                        // stride-2 conv output patch
constexpr int F_WX = 2 * F_TW + 1, F_WY = 2 * F_TH + 1;   // stem window: 17 x 33 pixels
constexpr int F_WPIX = F_WX * F_WY;                       // 561
constexpr int F_MT = (F_WPIX + 127) / 128;                // 5 stem M tiles
constexpr int F_LBX = 2 * F_TW + 4;                       // letterbox window columns (20, even start)
constexpr int F_LBY = F_WY + 2;                           // letterbox window rows (35)
constexpr int F_LB_ROW = F_LBX * 8;                       // bytes per letterbox window row (RGB0 bf16)
constexpr int F_LB_BYTES = F_LBY * F_LB_ROW;              // 5600
constexpr int F_LB_SLOT = 6144;
constexpr int F_PW = F_TW + 1;                            // parity plane: 9 x 17 pixels of 64 bytes
constexpr int F_PLANE = 10240;                            // 9792 rounded up to 1024
constexpr int F_WIN = 4 * F_PLANE;
constexpr int F_COL_TILE = 128 * 64;                      // one im2col tile: 128 rows x 32 bf16
constexpr int F_W0_BYTES = 32 * 64;                       // stem weights: 32 rows x 32 bf16
constexpr int F_W1_KB = 5;                                // stride-2 weights: 9 taps x 32 ch, padded to 320
constexpr int F_W1_BYTES = F_W1_KB * 64 * 128;
constexpr int F_STG = 128 * 128;                          // output staging: 128 pixels x 64 bf16
constexpr int F_ONES = 128 * 64;                          // constant-ones A tile (128 rows x 32 bf16)
constexpr int F_B1B = 64 * 64;                            // stride-2 bias parts: 64 rows x 32 bf16
constexpr int F_GATHER = 8;                               // gather warps: 1..4 and 14..17
constexpr int F_THREADS = 18 * 32;

// shared-memory carve-up (offsets from a 1024-aligned base)
constexpr int O_LB = 0;
constexpr int O_COL = O_LB + 2 * F_LB_SLOT;
constexpr int O_WIN = O_COL + F_MT * F_COL_TILE;
constexpr int O_W0 = O_WIN + 2 * F_WIN;
constexpr int O_W1 = O_W0 + 2048;
constexpr int O_STG = O_W1 + F_W1_BYTES;
constexpr int O_ONES = O_STG + 2 * F_STG;
constexpr int O_B1B = O_ONES + F_ONES;
constexpr int O_BAR = O_B1B + F_B1B;
constexpr int F_SMEM = O_BAR + 256 + 1024;
static_assert(F_SMEM <= 227 * 1024, "fused stem shared memory");
static_assert(O_COL % 1024 == 0 && O_WIN % 1024 == 0 && O_W0 % 1024 == 0 && O_W1 % 1024 == 0 && O_STG % 1024 == 0 &&
                  O_ONES % 1024 == 0 && O_B1B % 1024 == 0,
              "swizzled operand tiles need 1024-byte alignment");

// TMEM columns: two stem accumulator sets (5 x 32) and two output accumulators (64)
constexpr uint32_t T_STEM = 0, T_OUT = 320, T_COLS = 512;

struct FusedArgs {
  int n, H, W;        // letterbox (stem input and output) size, unpadded
  int Ho, Wo;         // stride-2 conv output size
  int tiles_x, tiles_y, total;
  int* err;
};

struct FusedMaps {
  alignas(64) CUtensorMap lb;   // letterbox: {Wp * 4, Hp, n} bf16
  alignas(64) CUtensorMap w0;   // stem weights {32, 32} with the bias parts in K columns 27..29
  alignas(64) CUtensorMap w1;   // stride-2 weights {320, 64}
  alignas(64) CUtensorMap o;    // output {64, Wo + 2, Ho + 2, n}
  alignas(64) CUtensorMap b1;   // stride-2 bias parts {32, 64} (K columns 0..2)
};

__device__ __forceinline__ bool f_aborted(const int* flag) { return *((volatile const int*)flag) != 0; }

__global__ void __launch_bounds__(F_THREADS, 1) stem_s2_kernel(const __grid_constant__ FusedMaps maps, const FusedArgs a) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ int s_abort;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sLB = smem + O_LB;
  uint8_t* sCol = smem + O_COL;
  uint8_t* sWin = smem + O_WIN;
  uint8_t* sW0 = smem + O_W0;
  uint8_t* sW1 = smem + O_W1;
  uint8_t* sStg = smem + O_STG;
  uint8_t* sOnes = smem + O_ONES;
  uint8_t* sB1b = smem + O_B1B;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + O_BAR);
  uint64_t* lb_full = bar;          // [2]
  uint64_t* lb_empty = bar + 2;     // [2]
  uint64_t* col_full = bar + 4;     // [F_MT] im2col tile t gathered
  uint64_t* col_empty = bar + 9;    // [F_MT] im2col tile t consumed by its MMAs
  uint64_t* sacc_full = bar + 14;   // [2]
  uint64_t* sacc_empty = bar + 16;  // [2]
  uint64_t* win_full = bar + 18;    // [2]
  uint64_t* win_empty = bar + 20;   // [2]
  uint64_t* acc_full = bar + 22;    // [2]
  uint64_t* acc_empty = bar + 24;   // [2]
  uint64_t* w_full = bar + 26;      // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 27);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&lb_full[i], 1);
      mbar_init(&lb_empty[i], F_GATHER);
      mbar_init(&sacc_full[i], 1);
      mbar_init(&sacc_empty[i], 4);
      mbar_init(&win_full[i], 4);
      mbar_init(&win_empty[i], 1);
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], 4);
    }
    for (int t = 0; t < F_MT; ++t) {
      mbar_init(&col_full[t], F_GATHER / 2);   // the four warps of the tile's gather group
      mbar_init(&col_empty[t], 1);
    }
    mbar_init(w_full, 1);
    fence_barrier_init();
    s_abort = 0;
  }
  // rows 561..639 of the last im2col tile are never gathered: zero them once; the ones tile (bf16 1.0)
  for (int i = threadIdx.x; i < (F_MT * 128 - F_WPIX) * 4; i += blockDim.x)
    reinterpret_cast<uint4*>(sCol + F_WPIX * 64)[i] = make_uint4(0u, 0u, 0u, 0u);
  for (int i = threadIdx.x; i < F_ONES / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(sOnes)[i] = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
  if (warp == 5) tmem_alloc(tmem_slot, T_COLS);
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int u0 = blockIdx.x, ustep = gridDim.x;
  const int per_img = a.tiles_x * a.tiles_y;

  if (warp == 0) {
    // ---------------- producer: weights once, then one letterbox window per unit
    if (lane == 0) {
      tma_prefetch(&maps.lb);
      mbar_expect_tx(w_full, F_W0_BYTES + F_W1_BYTES + F_B1B);
      tma_load_2d(sW0, &maps.w0, w_full, 0, 0);
      tma_load_2d(sB1b, &maps.b1, w_full, 0, 0);
      for (int kb = 0; kb < F_W1_KB; ++kb) tma_load_2d(sW1 + kb * 64 * 128, &maps.w1, w_full, kb * 64, 0);
      uint32_t lt = 0;
      for (int u = u0; u < a.total && !f_aborted(&s_abort); u += ustep, ++lt) {
        const uint32_t b = lt & 1u;
        if (lt >= 2 && !mbar_wait(&lb_empty[b], ((lt >> 1) - 1) & 1u)) {
          flag_error(a.err, KERR_TIMEOUT);
          atomicExch(&s_abort, 1);
          break;
        }
        const int img = u / per_img, r = u % per_img;
        const int oy0 = (r / a.tiles_x) * F_TH, ox0 = (r % a.tiles_x) * F_TW;
        // padded letterbox rows 2 oy0 - 1 .. 2 oy0 + 33, columns 2 ox0 - 2 .. 2 ox0 + 17 (an even pixel, so
        // the box starts on a 16-byte boundary); rows outside the image read the zero fill
        mbar_expect_tx(&lb_full[b], F_LB_BYTES);
        tma_load_3d(sLB + b * F_LB_SLOT, &maps.lb, &lb_full[b], (2 * ox0 - 2) * 4, 2 * oy0 - 1, img);
      }
    }
  } else if ((warp >= 1 && warp <= 4) || warp >= 14) {
    // ---------------- gather: im2col rows of the stem window from the letterbox window; group 0
    // (warps 1-4) fills tiles 0, 2, 4 and group 1 (warps 14-17) tiles 1, 3, one row per thread
    const int grp = warp <= 4 ? 0 : 1;
    const int rr = warp <= 4 ? threadIdx.x - 32 : threadIdx.x - 14 * 32;   // tile row 0..127
    uint32_t lt = 0;
    for (int u = u0; u < a.total; u += ustep, ++lt) {
      if (__shfl_sync(0xffffffffu, f_aborted(&s_abort) ? 1 : 0, 0)) break;   // warp-uniform
      const uint32_t b = lt & 1u;
      bool ok = lane == 0 ? mbar_wait(&lb_full[b], (lt >> 1) & 1u) : true;
      const uint8_t* lbw = sLB + b * F_LB_SLOT;
      const int r_g = u % per_img;
      const int oy0 = (r_g / a.tiles_x) * F_TH, ox0 = (r_g % a.tiles_x) * F_TW;
      for (int t = grp; t < F_MT; t += 2) {
        if (lane == 0 && ok && lt >= 1) ok = mbar_wait(&col_empty[t], (lt - 1) & 1u);   // the tile's last MMAs
        if (!__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) break;   // the warp takes one path
        const int m = 128 * t + rr;            // window pixel = im2col row
        if (m < F_WPIX) {
          const int wy = m / F_WX, wx = m - (m / F_WX) * F_WX;
          uint8_t* row = sCol + t * F_COL_TILE;
          const int sy = 2 * oy0 - 1 + wy, sx = 2 * ox0 - 1 + wx;
          // outside the image: an all-zero row (so a zero accumulator), selected without a branch; every tap
          // of the window lies inside the loaded letterbox window, so the loads below are always in bounds
          const uint32_t keep = (sy >= 0 && sy < a.H && sx >= 0 && sx < a.W) ? 0xFFFFFFFFu : 0u;
          // tap (ky, kx) of window pixel (wy, wx): letterbox window row wy + ky, column wx + kx + 1; a tap is
          // 8 bytes, lo = (R, G), hi = (B, 0) as bf16 pairs
          uint2 q[9];
          const uint8_t* src = lbw + wy * F_LB_ROW + (wx + 1) * 8;
#pragma unroll
          for (int ky = 0; ky < 3; ++ky)
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) q[ky * 3 + kx] = *reinterpret_cast<const uint2*>(src + ky * F_LB_ROW + kx * 8);
          // the 27 values (tap, channel) packed two per word, then 1.0 x 3 (the bias columns) and 0 x 2:
          // taps 2i, 2i+1 give three words (R G | B R' | G' B')
          uint32_t w[16];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const uint2 ta = q[2 * i], tb = q[2 * i + 1];
            w[3 * i] = ta.x;
            w[3 * i + 1] = __byte_perm(ta.y, tb.x, 0x5410);
            w[3 * i + 2] = __byte_perm(tb.x, tb.y, 0x5432);
          }
          w[12] = q[8].x;
          w[13] = (q[8].y & 0xFFFFu) | 0x3F800000u;
          w[14] = 0x3F803F80u;
          w[15] = 0u;
#pragma unroll
          for (int k = 0; k < 4; ++k)
            *reinterpret_cast<uint4*>(row + rr * 64 + ((k ^ ((rr >> 1) & 3)) << 4)) =
                make_uint4(w[4 * k] & keep, w[4 * k + 1] & keep, w[4 * k + 2] & keep, w[4 * k + 3] & keep);
        }
        fence_proxy_async();   // generic-proxy writes -> visible to the MMAs
        __syncwarp();
        if (lane == 0) mbar_arrive(&col_full[t]);
      }
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;   // lane 0's waits decide for the warp
      if (!ok) {
        if (lane == 0) {
          flag_error(a.err, KERR_TIMEOUT);
          atomicExch(&s_abort, 1);
        }
        break;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&lb_empty[b]);   // the letterbox window is read
    }
  } else if (warp == 5) {
    // ---------------- MMA issuer: stem of unit lt, then the stride-2 conv of unit lt - 1
    if (lane == 0) {
      constexpr uint32_t id0 = idesc_bf16(128, 32);
      constexpr uint32_t id1 = idesc_bf16(128, 64);
      const uint64_t col_d = smem_desc(smem_u32(sCol), 512, 4u);    // 64-byte rows, 64-byte swizzle
      const uint64_t w0_d = smem_desc(smem_u32(sW0), 512, 4u);
      const uint64_t w1_d = smem_desc(smem_u32(sW1), 1024, 2u);    // 128-byte rows, 128-byte swizzle
      const uint64_t win_d = smem_desc(smem_u32(sWin), (uint32_t)(F_PW * 64), 4u);
      const uint64_t ones_d = smem_desc(smem_u32(sOnes), 512, 4u);
      const uint64_t b1b_d = smem_desc(smem_u32(sB1b), 512, 4u);
      uint32_t aoff[18], boff[18];
#pragma unroll
      for (int i = 0; i < 18; ++i) {
        const int tap = i / 2, kk = i % 2;
        const int ky = tap / 3, kx = tap % 3;
        const int par = (ky & 1) * 2 + (kx & 1);
        const int pix = (ky >> 1) * F_PW + (kx >> 1);
        const int kidx = tap * 32 + kk * 16;
        aoff[i] = (uint32_t)(par * F_PLANE + pix * 64 + kk * 32) >> 4;
        boff[i] = (uint32_t)((kidx >> 6) * (64 * 128) + (kidx & 63) * 2) >> 4;
      }
      bool ok = mbar_wait(w_full, 0);
      uint32_t lt = 0;
      auto stage2 = [&](uint32_t t) -> bool {   // the stride-2 conv of unit t
        const uint32_t wb = t & 1u;
        if (!mbar_wait(&win_full[wb], (t >> 1) & 1u)) return false;
        if (t >= 2 && !mbar_wait(&acc_empty[wb], ((t >> 1) - 1) & 1u)) return false;
        tc_fence_after();
        const uint64_t ad = desc_add(win_d, (wb * (uint32_t)F_WIN) >> 4);
        const uint32_t d = tmem + T_OUT + wb * 64;
#pragma unroll
        for (int i = 0; i < 18; ++i) umma_bf16(d, desc_add(ad, aoff[i]), desc_add(w1_d, boff[i]), id1, i != 0 ? 1u : 0u);
        umma_bf16(d, ones_d, b1b_d, id1, 1u);   // + bias (ones x bias parts, K columns 0..15)
        umma_commit(&win_empty[wb]);
        umma_commit(&acc_full[wb]);
        return true;
      };
      for (int u = u0; ok && u < a.total && !f_aborted(&s_abort); u += ustep, ++lt) {
        const uint32_t sb = lt & 1u;
        if (lt >= 2) ok = mbar_wait(&sacc_empty[sb], ((lt >> 1) - 1) & 1u);
        if (!ok) break;
        const uint32_t d0 = tmem + T_STEM + sb * (F_MT * 32);
        // each im2col tile as soon as its gather group has filled it; its barrier frees it for the next unit
#pragma unroll
        for (int t = 0; t < F_MT; ++t) {
          if (!(ok = mbar_wait(&col_full[t], lt & 1u))) break;
          tc_fence_after();
#pragma unroll
          for (int kk = 0; kk < 2; ++kk)
            umma_bf16(d0 + t * 32, desc_add(col_d, (uint32_t)(t * F_COL_TILE) / 16 + 2 * kk), desc_add(w0_d, 2 * kk),
                      id0, kk);
          umma_commit(&col_empty[t]);
        }
        if (!ok) break;
        umma_commit(&sacc_full[sb]);
        if (lt >= 1) ok = stage2(lt - 1);
      }
      if (ok && lt >= 1) ok = stage2(lt - 1);
      if (!ok) {
        flag_error(a.err, KERR_TIMEOUT);
        atomicExch(&s_abort, 1);
      }
    }
  } else if (warp >= 6 && warp <= 9) {
    // ---------------- stem epilogue: TMEM -> bias, leaky-ReLU, zero outside the image -> parity planes
    const int quarter = warp & 3;
    const int r = quarter * 32 + lane;   // TMEM lane = row of each stem tile
    uint32_t lt = 0;
    for (int u = u0; u < a.total; u += ustep, ++lt) {
      if (__shfl_sync(0xffffffffu, f_aborted(&s_abort) ? 1 : 0, 0)) break;   // warp-uniform
      const uint32_t sb = lt & 1u;
      bool ok = true;
      if (lane == 0) {
        ok = mbar_wait(&sacc_full[sb], (lt >> 1) & 1u);
        if (ok && lt >= 2) ok = mbar_wait(&win_empty[sb], ((lt >> 1) - 1) & 1u);
        if (!ok) {
          flag_error(a.err, KERR_TIMEOUT);
          atomicExch(&s_abort, 1);
        }
      }
      if (!__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) break;   // the warp takes one path
      tc_fence_after();
      uint8_t* win = sWin + sb * F_WIN;
      const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + T_STEM + sb * (F_MT * 32);
      // two tiles' accumulator rows in flight per wait (TMEM load latency overlaps)
#pragma unroll 1
      for (int t0 = 0; t0 < F_MT; t0 += 2) {
        uint32_t v[2][32];
        tmem_ld32(tbase + t0 * 32, v[0]);
        if (t0 + 1 < F_MT) tmem_ld32(tbase + (t0 + 1) * 32, v[1]);
        tmem_ld_wait();
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int t = t0 + q;
          const int m = 128 * t + r;
          if (t >= F_MT || m >= F_WPIX) continue;
          const int wy = m / F_WX, wx = m - (m / F_WX) * F_WX;
          uint32_t pk[16];   // bias already in the accumulator; zero outside the image stays zero
#pragma unroll
          for (int j = 0; j < 16; ++j)
            pk[j] = pack_bf16x2(leaky01f(__uint_as_float(v[q][2 * j])), leaky01f(__uint_as_float(v[q][2 * j + 1])));
          const int par = (wy & 1) * 2 + (wx & 1);
          const int pix = (wy >> 1) * F_PW + (wx >> 1);
          uint8_t* dst = win + par * F_PLANE + pix * 64;
#pragma unroll
          for (int k = 0; k < 4; ++k)
            *reinterpret_cast<uint4*>(dst + ((k ^ ((pix >> 1) & 3)) << 4)) =
                make_uint4(pk[4 * k], pk[4 * k + 1], pk[4 * k + 2], pk[4 * k + 3]);
        }
      }
      tc_fence_before();
      fence_proxy_async();               // window writes -> visible to the MMAs
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&sacc_empty[sb]);
        mbar_arrive(&win_full[sb]);
      }
    }
  } else {
    // ---------------- output epilogue: TMEM -> bias, leaky-ReLU -> bf16 staging -> TMA store
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;   // output pixel (row / 8, row % 8) of the patch
    const bool elected = warp == 10 && lane == 0;
    uint32_t lt = 0;
    for (int u = u0; u < a.total; u += ustep, ++lt) {   // a failed wait ends it (bar_and below)
      const uint32_t ab = lt & 1u;
      bool ok = lane == 0 ? mbar_wait(&acc_full[ab], (lt >> 1) & 1u) : true;
      // the CTA's last accumulator is complete: the next layer's kernel may launch and set up
      if (u + ustep >= a.total && elected) grid_dep_trigger();
      ok = bar_and(ok, 1, 128);               // the four warps take one path
      if (!ok) {
        if (lane == 0) {
          flag_error(a.err, KERR_TIMEOUT);
          atomicExch(&s_abort, 1);
        }
        break;
      }
      tc_fence_after();
      const int img = u / per_img, rr = u % per_img;
      const int oy0 = (rr / a.tiles_x) * F_TH, ox0 = (rr % a.tiles_x) * F_TW;
      const bool valid = oy0 + row / F_TW < a.Ho && ox0 + row % F_TW < a.Wo;
      if (elected) bulk_wait_read<1>();   // the store that used this staging tile two units ago has read it
      named_bar(1, 128);
      uint8_t* stg = sStg + ab * F_STG;
      uint32_t v2[2][32];                     // both halves of 32 channels in flight
      tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + T_OUT + ab * 64, v2[0]);
      tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + T_OUT + ab * 64 + 32, v2[1]);
      tmem_ld_wait();
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint32_t* v = v2[h];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          uint32_t pk[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int c = 8 * k + 2 * e;   // bias already in the accumulator
            pk[e] = pack_bf16x2(leaky01f(__uint_as_float(v[c])), leaky01f(__uint_as_float(v[c + 1])));
          }
          const int unit = 4 * h + k;        // 16-byte unit of the 128-byte row
          // rows past the output's edge (ragged patches only) are stored as zeros into the halo
          *reinterpret_cast<uint4*>(stg + row * 128 + ((unit ^ (row & 7)) << 4)) =
              valid ? make_uint4(pk[0], pk[1], pk[2], pk[3]) : make_uint4(0u, 0u, 0u, 0u);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[ab]);
      fence_proxy_async();
      named_bar(1, 128);
      if (elected && !f_aborted(&s_abort)) {
        tma_store_4d(&maps.o, stg, 0, ox0 + 1, oy0 + 1, img);
        bulk_commit();
      }
    }
    if (elected) bulk_wait0();
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (warp == 5) tmem_dealloc(tmem, T_COLS);
}

typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*, const cuuint64_t*,
                             const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                             CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn f_encode_fn() {
  static EncodeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
  });
  return fn;
}

bool f_encode(CUtensorMap* m, int rank, const void* base, const cuuint64_t* dims, const cuuint64_t* strides,
              const cuuint32_t* box, CUtensorMapSwizzle swz) {
  EncodeFn fn = f_encode_fn();
  if (!fn) return false;
  cuuint32_t es[5] = {1, 1, 1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

struct StemS2Plan {
  FusedMaps maps;
  FusedArgs args;
};

namespace {
// b = p0 + p1 + p2 with each part a bfloat16 (the remainders are exact in float32), to float32 accuracy.
__device__ void split_bf16x3(float b, __nv_bfloat16* p) {
  p[0] = __float2bfloat16_rn(b);
  const float r1 = b - __bfloat162float(p[0]);
  p[1] = __float2bfloat16_rn(r1);
  p[2] = __float2bfloat16_rn(r1 - __bfloat162float(p[1]));
}

__global__ void stem_s2_pack_kernel(const __nv_bfloat16* w0, const float* bias0, const float* bias1,
                                    __nv_bfloat16* w0b, __nv_bfloat16* b1b) {
  const int n = threadIdx.x;   // 64 threads
  if (n < 32) {
    __nv_bfloat16* row = w0b + n * 32;
    for (int k = 0; k < 32; ++k) row[k] = k < 27 ? w0[n * 32 + k] : __float2bfloat16_rn(0.f);
    split_bf16x3(bias0[n], row + 27);
  }
  __nv_bfloat16* row = b1b + n * 32;
  for (int k = 0; k < 32; ++k) row[k] = __float2bfloat16_rn(0.f);
  split_bf16x3(bias1[n], row);
}
}  // namespace

cudaError_t stem_s2_pack(const void* w0, const float* bias0, const float* bias1, void* w0b, void* b1b,
                         cudaStream_t st) {
  jde_count_launch();
  stem_s2_pack_kernel<<<1, 64, 0, st>>>(static_cast<const __nv_bfloat16*>(w0), bias0, bias1,
                                         static_cast<__nv_bfloat16*>(w0b), static_cast<__nv_bfloat16*>(b1b));
  return cudaGetLastError();
}

StemS2Plan* stem_s2_plan_new(const TView& lb, const TView& out, const void* w0b, const void* w1, const void* b1b,
                             int* err, char* msg, size_t msg_len) {
  // letterbox: bf16 RGB0 (pixstride 4) with a one-pixel halo; output: bf16, 64 channels, halo, even input size
  if (lb.dtype != 1 || lb.pad != 1 || lb.pixstride != 4 || out.dtype != 1 || out.pad != 1 || out.c != 64 ||
      (lb.h & 1) || (lb.w & 1) || out.h != lb.h / 2 || out.w != lb.w / 2 || out.n != lb.n || out.pixstride < 64 ||
      (out.pixstride % 8)) {
    snprintf(msg, msg_len, "fused stem: unsupported shapes");
    return nullptr;
  }
  StemS2Plan* p = new StemS2Plan();
  FusedArgs& a = p->args;
  a.n = lb.n;
  a.H = lb.h;
  a.W = lb.w;
  a.Ho = out.h;
  a.Wo = out.w;
  a.tiles_x = (a.Wo + F_TW - 1) / F_TW;
  a.tiles_y = (a.Ho + F_TH - 1) / F_TH;
  a.total = a.n * a.tiles_x * a.tiles_y;
  a.err = err;
  const int Hp = lb.h + 2, Wp = lb.w + 2;
  bool ok = true;
  {
    cuuint64_t dims[3] = {(cuuint64_t)Wp * 4, (cuuint64_t)Hp, (cuuint64_t)lb.n};
    cuuint64_t strides[2] = {(cuuint64_t)Wp * 4 * 2, (cuuint64_t)Hp * Wp * 4 * 2};
    cuuint32_t box[3] = {(cuuint32_t)F_LBX * 4, (cuuint32_t)F_LBY, 1};
    ok &= f_encode(&p->maps.lb, 3, lb.ptr, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_NONE);
  }
  {
    cuuint64_t dims[2] = {32, 32};
    cuuint64_t strides[1] = {64};
    cuuint32_t box[2] = {32, 32};
    ok &= f_encode(&p->maps.w0, 2, w0b, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_64B);
  }
  {
    cuuint64_t dims[2] = {32, 64};
    cuuint64_t strides[1] = {64};
    cuuint32_t box[2] = {32, 64};
    ok &= f_encode(&p->maps.b1, 2, b1b, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_64B);
  }
  {
    cuuint64_t dims[2] = {(cuuint64_t)F_W1_KB * 64, 64};
    cuuint64_t strides[1] = {(cuuint64_t)F_W1_KB * 64 * 2};
    cuuint32_t box[2] = {64, 64};
    ok &= f_encode(&p->maps.w1, 2, w1, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_128B);
  }
  {
    const size_t ps = (size_t)out.pixstride * 2;
    cuuint64_t dims[4] = {64, (cuuint64_t)(out.w + 2), (cuuint64_t)(out.h + 2), (cuuint64_t)out.n};
    cuuint64_t strides[3] = {ps, (cuuint64_t)(out.w + 2) * ps, (cuuint64_t)(out.h + 2) * (out.w + 2) * ps};
    cuuint32_t box[4] = {64, (cuuint32_t)F_TW, (cuuint32_t)F_TH, 1};
    ok &= f_encode(&p->maps.o, 4, out.ptr, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_128B);
  }
  if (!ok) {
    snprintf(msg, msg_len, "fused stem: cuTensorMapEncodeTiled failed");
    delete p;
    return nullptr;
  }
  return p;
}

void stem_s2_plan_free(StemS2Plan* p) { delete p; }

cudaError_t stem_s2_launch(const StemS2Plan* p, cudaStream_t st) {
  static std::mutex mu;
  static bool attr[JDE_MAX_DEVICES] = {false};
  static int sms[JDE_MAX_DEVICES] = {0};
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= JDE_MAX_DEVICES) return cudaErrorInvalidDevice;
  int nsm;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!attr[dev]) {
      cudaError_t e = cudaFuncSetAttribute(stem_s2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, F_SMEM);
      if (e != cudaSuccess) return e;
      int v = 0;
      if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
      sms[dev] = v;
      attr[dev] = true;
    }
    nsm = sms[dev];
  }
  const int grid = p->args.total < nsm ? p->args.total : nsm;
  jde_count_launch();
  stem_s2_kernel<<<grid, F_THREADS, F_SMEM, st>>>(p->maps, p->args);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------- fused residual block
// The first stage's residual block (Sec. 3.1, DarkNet-53: x -> 1x1 64 -> 32 -> 3x3 32 -> 64, added to
// x) as one persistent tcgen05 kernel: the 1x1's output t never leaves shared memory.
//
// Work unit: one TW x TH = 8 x 16 patch of the block output.  Its 3x3 reads t on the (TW + 2) x (TH + 2)
// = 10 x 18 window around the patch, and t there is the 1x1 of x on the same window.  Per unit:
//   * warp 0 / lane 0 loads the x window (180 pixels x 64 channels, 128-byte rows, 128-byte swizzle)
//     with one TMA box; the weights of both convs are loaded once and stay resident;
//   * the MMA warp runs the 1x1 over the window (two M=128 tiles, N=32, K=64) into TMEM, then the 3x3
//     of the previous unit: nine taps x two K=16 MMAs (M=128, N=64) reading the t window at a pixel
//     offset per tap (64-byte rows, 64-byte swizzle by absolute address, 8-row groups one window row
//     apart), the layout of the 32-channel window convs;
//   * four t-epilogue warps add the 1x1's bias, apply leaky-ReLU, round to bf16 and write t into the t
//     window, zero at window pixels outside the image (the 3x3's zero padding);
//   * four output epilogue warps add the 3x3's bias, apply leaky-ReLU, add the block input x (read from
//     global memory, where the window load has just brought it into L2) in float32, round once to bf16
//     and TMA-store the patch into the block's output tensor, which is not the input tensor:
//     neighbouring patches read x on their halos.
// An x window is released as soon as the 1x1 has read it (three buffers, so the loads run two units
// ahead); t windows and both accumulators are double-buffered; every wait is bounded.
namespace {

constexpr int R_TW = 8, R_TH = 16;
constexpr int R_WX = R_TW + 2, R_WY = R_TH + 2;   // 10 x 18 window
constexpr int R_WPIX = R_WX * R_WY;               // 180
constexpr int R_XW = 256 * 128;                   // x window slot: two 128-row operand tiles of 128 bytes
constexpr int R_NXW = 3;                          // x window slots
constexpr int R_NB = 2;                           // t windows and accumulator sets
constexpr int R_XW_TX = R_WPIX * 128;             // bytes one x window load delivers
constexpr int R_TWB = 12288;                      // t window slot: 180 x 64 bytes, rounded up to 1024
constexpr int R_W1 = 32 * 128;                    // 1x1 weights: 32 rows x 64 bf16
constexpr int R_W2_KB = 5;                        // 3x3 weights: 9 taps x 32 channels, padded to 320
constexpr int R_W2 = R_W2_KB * 64 * 128;
constexpr int R_STG = 128 * 128;                  // output staging: 128 pixels x 64 bf16
constexpr int R_THREADS = 10 * 32;

constexpr int RO_XW = 0;
constexpr int RO_TW = RO_XW + R_NXW * R_XW;
constexpr int RO_W1 = RO_TW + R_NB * R_TWB;
constexpr int RO_W2 = RO_W1 + R_W1;
constexpr int RO_STG = RO_W2 + R_W2;
constexpr int RO_BIAS = RO_STG + 2 * R_STG;       // 32 + 64 floats
constexpr int RO_BAR = RO_BIAS + 512;
constexpr int R_SMEM = RO_BAR + 256 + 1024;
static_assert(R_SMEM <= 227 * 1024, "fused residual block shared memory");
static_assert(RO_TW % 1024 == 0 && RO_W1 % 1024 == 0 && RO_W2 % 1024 == 0 && RO_STG % 1024 == 0 && R_TWB % 1024 == 0,
              "swizzled operand tiles need 1024-byte alignment");

// TMEM columns: R_NB 1x1 accumulator sets (2 tiles x 32) and R_NB 3x3 accumulators (64)
constexpr uint32_t RT_A1 = 0, RT_A2 = 64 * R_NB, RT_COLS = 256;
static_assert(RT_A2 + 64 * R_NB <= RT_COLS, "TMEM columns");

struct Res1Args {
  int n, H, W;        // block input / output size, unpadded
  const __nv_bfloat16* x;   // block input (haloed, x_ps elements per pixel), for the residual
  int x_ps;
  int tiles_x, tiles_y, total;
  const float* b1;    // 1x1 bias [32]
  const float* b2;    // 3x3 bias [64]
  int* err;
};

struct Res1Maps {
  alignas(64) CUtensorMap x;    // block input {64, W + 2, H + 2, n}
  alignas(64) CUtensorMap w1;   // 1x1 weights {64, 32}
  alignas(64) CUtensorMap w2;   // 3x3 weights {320, 64}
  alignas(64) CUtensorMap o;    // block output {64, W + 2, H + 2, n}
};

__global__ void __launch_bounds__(R_THREADS, 1) res1_kernel(const __grid_constant__ Res1Maps maps, const Res1Args a) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ int s_abort;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sXW = smem + RO_XW;
  uint8_t* sTW = smem + RO_TW;
  uint8_t* sW1 = smem + RO_W1;
  uint8_t* sW2 = smem + RO_W2;
  uint8_t* sStg = smem + RO_STG;
  float* sB1 = reinterpret_cast<float*>(smem + RO_BIAS);
  float* sB2 = sB1 + 32;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + RO_BAR);
  uint64_t* xw_full = bar;                 // [R_NXW] x window landed
  uint64_t* xw_empty = xw_full + R_NXW;    // [R_NXW] x window read by the 1x1
  uint64_t* a1_full = xw_empty + R_NXW;    // [R_NB] 1x1 accumulators ready
  uint64_t* a1_empty = a1_full + R_NB;     // [R_NB] 1x1 accumulators drained
  uint64_t* tw_full = a1_empty + R_NB;     // [R_NB] t window written
  uint64_t* tw_empty = tw_full + R_NB;     // [R_NB] t window read by the 3x3
  uint64_t* a2_full = tw_empty + R_NB;     // [R_NB] 3x3 accumulator ready
  uint64_t* a2_empty = a2_full + R_NB;     // [R_NB] 3x3 accumulator drained
  uint64_t* w_full = a2_empty + R_NB;      // [1] weights landed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(w_full + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < R_NXW; ++i) {
      mbar_init(&xw_full[i], 1);
      mbar_init(&xw_empty[i], 1);   // tcgen05.commit after the unit's 1x1
    }
    for (int i = 0; i < R_NB; ++i) {
      mbar_init(&a1_full[i], 1);
      mbar_init(&a1_empty[i], 4);
      mbar_init(&tw_full[i], 4);
      mbar_init(&tw_empty[i], 1);
      mbar_init(&a2_full[i], 1);
      mbar_init(&a2_empty[i], 4);
    }
    mbar_init(w_full, 1);
    fence_barrier_init();
    s_abort = 0;
  }
  for (int i = threadIdx.x; i < 96; i += blockDim.x) sB1[i] = i < 32 ? a.b1[i] : a.b2[i - 32];
  if (warp == 1) tmem_alloc(tmem_slot, RT_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int u0 = blockIdx.x, ustep = gridDim.x;
  const int per_img = a.tiles_x * a.tiles_y;

  if (warp == 0) {
    // ---------------- producer: weights once, then one x window per unit
    if (lane == 0) {
      tma_prefetch(&maps.x);
      mbar_expect_tx(w_full, R_W1 + R_W2);
      tma_load_2d(sW1, &maps.w1, w_full, 0, 0);
      for (int kb = 0; kb < R_W2_KB; ++kb) tma_load_2d(sW2 + kb * 64 * 128, &maps.w2, w_full, kb * 64, 0);
      uint32_t lt = 0;
      for (int u = u0; u < a.total && !f_aborted(&s_abort); u += ustep, ++lt) {
        const uint32_t b = lt % R_NXW;
        if (lt >= (uint32_t)R_NXW && !mbar_wait(&xw_empty[b], ((lt / R_NXW) - 1) & 1u)) {
          flag_error(a.err, KERR_TIMEOUT);
          atomicExch(&s_abort, 1);
          break;
        }
        const int img = u / per_img, r = u % per_img;
        const int oy0 = (r / a.tiles_x) * R_TH, ox0 = (r % a.tiles_x) * R_TW;
        // padded pixels (oy0 .. oy0 + 17, ox0 .. ox0 + 9): image rows oy0 - 1 .. oy0 + 16; past the
        // tensor's end the box reads the zero fill
        mbar_expect_tx(&xw_full[b], R_XW_TX);
        tma_load_4d(sXW + b * R_XW, &maps.x, &xw_full[b], 0, ox0, oy0, img);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: the 1x1 of unit lt, then the 3x3 of unit lt - 1
    if (lane == 0) {
      constexpr uint32_t id1 = idesc_bf16(128, 32);
      constexpr uint32_t id2 = idesc_bf16(128, 64);
      const uint64_t xw_d = smem_desc(smem_u32(sXW), 1024, 2u);        // 128-byte rows, 128-byte swizzle
      const uint64_t w1_d = smem_desc(smem_u32(sW1), 1024, 2u);
      const uint64_t tw_d = smem_desc(smem_u32(sTW), (uint32_t)(R_WX * 64), 4u);   // window rows R_WX pixels apart
      const uint64_t w2_d = smem_desc(smem_u32(sW2), 1024, 2u);
      uint32_t aoff[18], boff[18];
#pragma unroll
      for (int i = 0; i < 18; ++i) {
        const int tap = i / 2, kk = i % 2;
        const int ky = tap / 3, kx = tap % 3;
        const int kidx = tap * 32 + kk * 16;
        aoff[i] = (uint32_t)((ky * R_WX + kx) * 64 + kk * 32) >> 4;
        boff[i] = (uint32_t)((kidx >> 6) * (64 * 128) + (kidx & 63) * 2) >> 4;
      }
      bool ok = mbar_wait(w_full, 0);
      uint32_t lt = 0;
      auto conv3 = [&](uint32_t t) -> bool {   // the 3x3 of unit t
        const uint32_t b = t % R_NB;
        if (!mbar_wait(&tw_full[b], (t / R_NB) & 1u)) return false;
        if (t >= (uint32_t)R_NB && !mbar_wait(&a2_empty[b], ((t / R_NB) - 1) & 1u)) return false;
        tc_fence_after();
        const uint64_t ad = desc_add(tw_d, (b * (uint32_t)R_TWB) >> 4);
        const uint32_t d = tmem + RT_A2 + b * 64;
#pragma unroll
        for (int i = 0; i < 18; ++i) umma_bf16(d, desc_add(ad, aoff[i]), desc_add(w2_d, boff[i]), id2, i != 0 ? 1u : 0u);
        umma_commit(&tw_empty[b]);
        umma_commit(&a2_full[b]);
        return true;
      };
      for (int u = u0; ok && u < a.total && !f_aborted(&s_abort); u += ustep, ++lt) {
        const uint32_t b = lt % R_NB, xb = lt % R_NXW;
        ok = mbar_wait(&xw_full[xb], (lt / R_NXW) & 1u);
        if (ok && lt >= (uint32_t)R_NB) ok = mbar_wait(&a1_empty[b], ((lt / R_NB) - 1) & 1u);
        if (!ok) break;
        tc_fence_after();
        const uint32_t d = tmem + RT_A1 + b * 64;
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            umma_bf16(d + mt * 32, desc_add(xw_d, (xb * (uint32_t)R_XW + mt * 128 * 128) / 16 + 2 * kk),
                      desc_add(w1_d, 2 * kk), id1, kk != 0 ? 1u : 0u);
        umma_commit(&xw_empty[xb]);
        umma_commit(&a1_full[b]);
        if (lt >= 1) ok = conv3(lt - 1);
      }
      if (ok && lt >= 1) ok = conv3(lt - 1);
      if (!ok) {
        flag_error(a.err, KERR_TIMEOUT);
        atomicExch(&s_abort, 1);
      }
    }
  } else if (warp >= 2 && warp <= 5) {
    // ---------------- t epilogue: TMEM -> bias, leaky-ReLU, zero outside the image -> t window
    const int quarter = warp & 3;
    const int r = quarter * 32 + lane;   // TMEM lane = row of each 1x1 tile
    uint32_t lt = 0;
    for (int u = u0; u < a.total; u += ustep, ++lt) {
      if (__shfl_sync(0xffffffffu, f_aborted(&s_abort) ? 1 : 0, 0)) break;   // warp-uniform
      const uint32_t b = lt % R_NB;
      bool ok = true;
      if (lane == 0) {
        ok = mbar_wait(&a1_full[b], (lt / R_NB) & 1u);
        if (ok && lt >= (uint32_t)R_NB) ok = mbar_wait(&tw_empty[b], ((lt / R_NB) - 1) & 1u);
        if (!ok) {
          flag_error(a.err, KERR_TIMEOUT);
          atomicExch(&s_abort, 1);
        }
      }
      if (!__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) break;   // the warp takes one path
      tc_fence_after();
      const int rr = u % per_img;
      const int oy0 = (rr / a.tiles_x) * R_TH, ox0 = (rr % a.tiles_x) * R_TW;
      uint32_t v[2][32];
      const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + RT_A1 + b * 64;
      tmem_ld32(tbase, v[0]);
      tmem_ld32(tbase + 32, v[1]);
      tmem_ld_wait();
      uint8_t* tw = sTW + b * R_TWB;
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int m = 128 * mt + r;   // window pixel
        if (m >= R_WPIX) continue;
        const int wy = m / R_WX, wx = m - (m / R_WX) * R_WX;
        const int iy = oy0 + wy - 1, ix = ox0 + wx - 1;
        const uint32_t keep = (iy >= 0 && iy < a.H && ix >= 0 && ix < a.W) ? 0xFFFFFFFFu : 0u;
        uint32_t pk[16];
#pragma unroll
        for (int j = 0; j < 16; ++j)
          pk[j] = pack_bf16x2(leaky01f(__uint_as_float(v[mt][2 * j]) + sB1[2 * j]),
                              leaky01f(__uint_as_float(v[mt][2 * j + 1]) + sB1[2 * j + 1])) &
                  keep;
        uint8_t* dst = tw + m * 64;
#pragma unroll
        for (int k = 0; k < 4; ++k)
          *reinterpret_cast<uint4*>(dst + ((k ^ ((m >> 1) & 3)) << 4)) =
              make_uint4(pk[4 * k], pk[4 * k + 1], pk[4 * k + 2], pk[4 * k + 3]);
      }
      tc_fence_before();
      fence_proxy_async();   // window writes -> visible to the MMAs
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&a1_empty[b]);
        mbar_arrive(&tw_full[b]);
      }
    }
  } else {
    // ---------------- output epilogue: TMEM -> bias, leaky-ReLU, + x -> bf16 staging -> TMA store
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;   // output pixel (row / 8, row % 8) of the patch
    const bool elected = warp == 6 && lane == 0;
    uint32_t lt = 0;
    for (int u = u0; u < a.total; u += ustep, ++lt) {   // a failed wait ends it (bar_and below)
      const uint32_t b = lt % R_NB, sb = lt & 1u;
      const int img = u / per_img, rr = u % per_img;
      const int oy0 = (rr / a.tiles_x) * R_TH, ox0 = (rr % a.tiles_x) * R_TW;
      const int oy = oy0 + row / R_TW, ox = ox0 + row % R_TW;
      const bool valid = oy < a.H && ox < a.W;
      // the block input at this pixel (64 channels, 128 bytes): loaded before the wait for the unit's
      // accumulator, so the load overlaps it
      uint4 xv[8];
      if (valid) {
        const uint4* xr = reinterpret_cast<const uint4*>(
            a.x + (((size_t)img * (a.H + 2) + oy + 1) * (a.W + 2) + ox + 1) * (size_t)a.x_ps);
#pragma unroll
        for (int k = 0; k < 8; ++k) xv[k] = __ldg(xr + k);
      } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) xv[k] = make_uint4(0u, 0u, 0u, 0u);
      }
      bool ok = lane == 0 ? mbar_wait(&a2_full[b], (lt / R_NB) & 1u) : true;
      ok = bar_and(ok, 1, 128);               // the four warps take one path
      if (!ok) {
        if (lane == 0) {
          flag_error(a.err, KERR_TIMEOUT);
          atomicExch(&s_abort, 1);
        }
        break;
      }
      tc_fence_after();
      if (elected) bulk_wait_read<1>();   // the store that used this staging tile two units ago has read it
      named_bar(1, 128);
      uint8_t* stg = sStg + sb * R_STG;
      uint32_t v2[2][32];
      tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + RT_A2 + b * 64, v2[0]);
      tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + RT_A2 + b * 64 + 32, v2[1]);
      tmem_ld_wait();
#pragma unroll
      for (int k = 0; k < 8; ++k) {           // 16-byte unit k: channels 8k .. 8k + 7
        const uint32_t* v = v2[k >> 2];
        const uint32_t xw[4] = {xv[k].x, xv[k].y, xv[k].z, xv[k].w};
        uint32_t pk[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int c = 8 * k + 2 * e;
          const float2 xf = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&xw[e]));
          const float y0 = leaky01f(__uint_as_float(v[c & 31]) + sB2[c]) + xf.x;
          const float y1 = leaky01f(__uint_as_float(v[(c + 1) & 31]) + sB2[c + 1]) + xf.y;
          pk[e] = pack_bf16x2(y0, y1);
        }
        // rows past the output's edge (ragged patches only) are stored as zeros into the halo
        *reinterpret_cast<uint4*>(stg + row * 128 + ((k ^ (row & 7)) << 4)) =
            valid ? make_uint4(pk[0], pk[1], pk[2], pk[3]) : make_uint4(0u, 0u, 0u, 0u);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&a2_empty[b]);
      fence_proxy_async();
      named_bar(1, 128);
      if (elected && !f_aborted(&s_abort)) {
        tma_store_4d(&maps.o, stg, 0, ox0 + 1, oy0 + 1, img);
        bulk_commit();
      }
    }
    if (elected) bulk_wait0();
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, RT_COLS);
}

}  // namespace

struct Res1Plan {
  Res1Maps maps;
  Res1Args args;
};

Res1Plan* res1_plan_new(const TView& x, const TView& out, const void* w1, const void* w2, const float* b1,
                        const float* b2, int* err, char* msg, size_t msg_len) {
  // block input and output: bf16, 64 channels, one-pixel halo, same size, 16-byte pixel strides
  if (x.dtype != 1 || x.pad != 1 || x.c != 64 || (x.pixstride % 8) || out.dtype != 1 || out.pad != 1 ||
      out.c != 64 || (out.pixstride % 8) || out.h != x.h || out.w != x.w || out.n != x.n || x.ptr == out.ptr) {
    snprintf(msg, msg_len, "fused residual block: unsupported shapes");
    return nullptr;
  }
  Res1Plan* p = new Res1Plan();
  Res1Args& a = p->args;
  a.n = x.n;
  a.H = x.h;
  a.W = x.w;
  a.tiles_x = (a.W + R_TW - 1) / R_TW;
  a.tiles_y = (a.H + R_TH - 1) / R_TH;
  a.total = a.n * a.tiles_x * a.tiles_y;
  a.b1 = b1;
  a.b2 = b2;
  a.err = err;
  a.x = static_cast<const __nv_bfloat16*>(x.ptr);
  a.x_ps = x.pixstride;
  bool ok = true;
  auto map4 = [&](CUtensorMap* m, const TView& v, int bx, int by) {
    const size_t ps = (size_t)v.pixstride * 2;
    cuuint64_t dims[4] = {64, (cuuint64_t)(v.w + 2), (cuuint64_t)(v.h + 2), (cuuint64_t)v.n};
    cuuint64_t strides[3] = {ps, (cuuint64_t)(v.w + 2) * ps, (cuuint64_t)(v.h + 2) * (v.w + 2) * ps};
    cuuint32_t box[4] = {64, (cuuint32_t)bx, (cuuint32_t)by, 1};
    return f_encode(m, 4, v.ptr, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_128B);
  };
  ok &= map4(&p->maps.x, x, R_WX, R_WY);
  ok &= map4(&p->maps.o, out, R_TW, R_TH);
  {
    cuuint64_t dims[2] = {64, 32};
    cuuint64_t strides[1] = {128};
    cuuint32_t box[2] = {64, 32};
    ok &= f_encode(&p->maps.w1, 2, w1, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_128B);
  }
  {
    cuuint64_t dims[2] = {(cuuint64_t)R_W2_KB * 64, 64};
    cuuint64_t strides[1] = {(cuuint64_t)R_W2_KB * 64 * 2};
    cuuint32_t box[2] = {64, 64};
    ok &= f_encode(&p->maps.w2, 2, w2, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_128B);
  }
  if (!ok) {
    snprintf(msg, msg_len, "fused residual block: cuTensorMapEncodeTiled failed");
    delete p;
    return nullptr;
  }
  return p;
}

void res1_plan_free(Res1Plan* p) { delete p; }

cudaError_t res1_launch(const Res1Plan* p, cudaStream_t st) {
  static std::mutex mu;
  static bool attr[JDE_MAX_DEVICES] = {false};
  static int sms[JDE_MAX_DEVICES] = {0};
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= JDE_MAX_DEVICES) return cudaErrorInvalidDevice;
  int nsm;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!attr[dev]) {
      cudaError_t e = cudaFuncSetAttribute(res1_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, R_SMEM);
      if (e != cudaSuccess) return e;
      int v = 0;
      if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
      sms[dev] = v;
      attr[dev] = true;
    }
    nsm = sms[dev];
  }
  const int grid = p->args.total < nsm ? p->args.total : nsm;
  jde_count_launch();
  res1_kernel<<<grid, R_THREADS, R_SMEM, st>>>(p->maps, p->args);
  return cudaGetLastError();
}
