// Tracker step on the device (Sec. 3 "Location Estimation" / "Association",
// Appendix A items 4-9), for several video streams per launch.
//
//   prep   : Kalman predict of every active/lost track (x <- F x,
//            P <- F P F^T + Q, Q from the pre-prediction height), then the
//            innovation covariance S = H P H^T + R (R from the predicted
//            height) and its Cholesky factor for gating and update;
//   cost   : C[k][j] = 1 - <e_k, d_j> (compensated f32 dot of unit embeddings), replaced by
//            the "infinite" 1e5 when the squared Mahalanobis distance
//            |L^-1 (z_j - H x_k)|^2 exceeds the chi-square gate;
//   cascade (jde_config.assoc_cascade): cost holds lambda (1 - cos) + (1 - lambda) d^2 (gated), and
//            assign_cascade runs three Hungarian stages on sub-matrices (confirmed tracks on that cost;
//            the tracked ones left on 1 - IoU of the predicted box; unconfirmed tracks on 1 - IoU),
//            removes unmatched unconfirmed tracks and confirms births only on a stream's first step;
//   assign : shortest-augmenting-path Hungarian in f64 (one warp per stream;
//            rows = the smaller side, tracks in creation order, detections in
//            kept order; columns scanned ascending, first minimum wins), pairs
//            costing more than the threshold rejected, Kalman update
//            (K = P H^T S^-1, x += K y, P -= K S K^T) and gallery update of
//            the assigned tracks, lost/removal bookkeeping, births in
//            detection order, output.
// Noise model: constant velocity on (cx, cy, a = w/h, h), dt = 1, sigma_p =
// 1/20 and sigma_v = 1/160 of the height (the paper names the Kalman filter
// but not its model).
// Track data never moves: each stream has a pool of slots, an `order` list
// (slot of the k-th track in creation order) and a free-slot stack.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "common.cuh"
#include "track.h"

namespace {

constexpr double SP = 1.0 / 20.0;
constexpr double SV = 1.0 / 160.0;
constexpr double INF_COST = 1e5;
constexpr int MAXB = 64;
constexpr int ASSIGN_COST_CACHE = 8192;   // doubles of cost matrix the assignment keeps in shared memory

struct Slots {
  int stream[MAXB];
};

struct StepArgs {
  TrackState t;
  const float* rows;      // [n][cap][518]
  const int32_t* count;   // [n]
  int cap;
  int n;
  double gate;
  float assign_thresh;
  int lost_max;
  float momentum;
  const int* dslots;      // device stream slots of the call (graph replays), else null: the by-value slots
  int cascade;            // three-stage association
  double lam, iou2, iou3; // cascade: appearance weight of stage 1, rejection thresholds of stages 2 and 3
  int* err;
  // outputs
  long long* o_id;
  float* o_box;
  int32_t* o_state;
  int32_t* o_det;
  int32_t* o_count;
  int o_cap;
};

__device__ __forceinline__ int det_count(const StepArgs& a, int b) {
  const int c = a.count[b];
  const int d = c < a.cap ? c : a.cap;
  return d < a.t.max_dets ? d : a.t.max_dets;
}

__device__ void measurement(const float* row, double (&z)[4]) {
  const double x1 = row[0], y1 = row[1], x2 = row[2], y2 = row[3];
  const double w = x2 - x1, h = y2 - y1;
  z[0] = x1 + w / 2;
  z[1] = y1 + h / 2;
  z[2] = w / h;
  z[3] = h;
}

__global__ void reset_kernel(TrackState t, int s) {
  const int T = t.max_tracks;
  for (int k = threadIdx.x; k < T; k += blockDim.x) {
    t.free_stack[(size_t)s * T + k] = T - 1 - k;
    t.order[(size_t)s * T + k] = -1;
  }
  if (threadIdx.x == 0) {
    t.n_tracks[s] = 0;
    t.next_id[s] = 1;
    t.free_top[s] = T;
    t.frames[s] = 0;
  }
}

// ---------------------------------------------------------------- predict + gating factors
__global__ void prep_kernel(StepArgs a, Slots sl) {
  const int b = blockIdx.y;
  const int s = a.dslots ? a.dslots[b] : sl.stream[b];
  const int T = a.t.max_tracks;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.t.n_tracks[s]) return;
  const int slot = a.t.order[(size_t)s * T + k];
  double* m = a.t.mean + ((size_t)s * T + slot) * 8;
  double* P = a.t.cov + ((size_t)s * T + slot) * 64;
  double mm[8], p[64], tmp[64];
#pragma unroll
  for (int i = 0; i < 8; ++i) mm[i] = m[i];
#pragma unroll
  for (int i = 0; i < 64; ++i) p[i] = P[i];
  const double h = mm[3];
  // x <- F x
#pragma unroll
  for (int i = 0; i < 4; ++i) mm[i] = mm[i] + mm[i + 4];
  // P <- (F P) F^T + Q
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) tmp[i * 8 + j] = i < 4 ? p[i * 8 + j] + p[(i + 4) * 8 + j] : p[i * 8 + j];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) p[i * 8 + j] = j < 4 ? tmp[i * 8 + j] + tmp[i * 8 + j + 4] : tmp[i * 8 + j];
  const double qp = (SP * h) * (SP * h), qv = (SV * h) * (SV * h);
  p[0] += qp;
  p[9] += qp;
  p[18] += 1e-2 * 1e-2;
  p[27] += qp;
  p[36] += qv;
  p[45] += qv;
  p[54] += 1e-5 * 1e-5;
  p[63] += qv;
#pragma unroll
  for (int i = 0; i < 8; ++i) m[i] = mm[i];
#pragma unroll
  for (int i = 0; i < 64; ++i) P[i] = p[i];
  // S = H P H^T + R, Cholesky S = L L^T
  const double hp = mm[3];
  const double rp = (SP * hp) * (SP * hp);
  double S[16];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) S[i * 4 + j] = p[i * 8 + j];
  S[0] += rp;
  S[5] += rp;
  S[10] += 1e-1 * 1e-1;
  S[15] += rp;
  double L[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) L[i] = 0.0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    double sj = S[j * 4 + j];
#pragma unroll
    for (int q = 0; q < j; ++q) sj -= L[j * 4 + q] * L[j * 4 + q];
    L[j * 4 + j] = sqrt(sj);
#pragma unroll
    for (int i = j + 1; i < 4; ++i) {
      double v = S[i * 4 + j];
#pragma unroll
      for (int q = 0; q < j; ++q) v -= L[i * 4 + q] * L[j * 4 + q];
      L[i * 4 + j] = v / L[j * 4 + j];
    }
  }
  double* gl = a.t.gate_l + ((size_t)b * T + slot) * 16;
  double* gz = a.t.gate_z + ((size_t)b * T + slot) * 4;
#pragma unroll
  for (int i = 0; i < 16; ++i) gl[i] = L[i];
#pragma unroll
  for (int i = 0; i < 4; ++i) gz[i] = mm[i];
}

// ---------------------------------------------------------------- cost + gate
// 32 tracks x 32 detections per tile, 256 threads: thread (tx, ty) owns det tx, tracks 4ty..4ty+3.
// The blocks of a stream (blockIdx.y) loop over the tiles its track and detection counts need (the
// counts live on the device), so the grid does not scale with the track and detection capacities.
constexpr int COST_BLOCKS = 8;   // blocks per stream
__global__ void cost_kernel(StepArgs a, Slots sl) {
  const int b = blockIdx.y;
  const int s = a.dslots ? a.dslots[b] : sl.stream[b];
  const int T = a.t.max_tracks;
  const int nt = a.t.n_tracks[s];
  const int D = det_count(a, b);
  const int ntx = (nt + 31) / 32, nty = (D + 31) / 32;
  __shared__ float Es[32][33];
  __shared__ float Ds[32][33];
  __shared__ int slot_s[32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int tile = blockIdx.x; tile < ntx * nty; tile += gridDim.x) {
    const int k0 = (tile % ntx) * 32, j0 = (tile / ntx) * 32;
    __syncthreads();   // the previous tile's reads of slot_s are done
    if (threadIdx.x < 32) slot_s[threadIdx.x] = k0 + threadIdx.x < nt ? a.t.order[(size_t)s * T + k0 + threadIdx.x] : -1;
    __syncthreads();
    // compensated f32 dot product: each product's rounding error (fma) and each sum's rounding error
    // (Neumaier) go into c, so s + c is the dot product of the f32 inputs to ~1e-7, well inside the
    // 1e-6 band in which a threshold decision counts as a tie
    float acc[4] = {0.f, 0.f, 0.f, 0.f}, comp[4] = {0.f, 0.f, 0.f, 0.f};
    const float* rows = a.rows + (size_t)b * a.cap * 518;
    for (int c0 = 0; c0 < 512; c0 += 32) {
      for (int e = threadIdx.x; e < 32 * 32; e += 256) {
        const int r = e >> 5, cc = e & 31;
        const int sl2 = slot_s[r];
        Es[r][cc] = sl2 >= 0 ? a.t.emb[((size_t)s * T + sl2) * 512 + c0 + cc] : 0.f;
        Ds[r][cc] = j0 + r < D ? rows[(size_t)(j0 + r) * 518 + 6 + c0 + cc] : 0.f;
      }
      __syncthreads();
#pragma unroll 8
      for (int cc = 0; cc < 32; ++cc) {
        const float dv = Ds[tx][cc];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float ev = Es[ty * 4 + q][cc];
          const float p = ev * dv;
          const float pe = fmaf(ev, dv, -p);       // exact product error
          const float t = acc[q] + p;
          comp[q] += (fabsf(acc[q]) >= fabsf(p) ? (acc[q] - t) + p : (p - t) + acc[q]) + pe;
          acc[q] = t;
        }
      }
      __syncthreads();
    }
    const int j = j0 + tx;
    if (j >= D) continue;
    double z[4];
    measurement(rows + (size_t)j * 518, z);
    const bool trans = nt > D;
    const int M = trans ? nt : D;
    double* A = a.t.cost + (size_t)b * T * a.t.max_dets;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = k0 + ty * 4 + q;
      if (k >= nt) break;
      const int slot = slot_s[ty * 4 + q];
      const double* L = a.t.gate_l + ((size_t)b * T + slot) * 16;
      const double* zh = a.t.gate_z + ((size_t)b * T + slot) * 4;
      double w[4], d2 = 0.0;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        double v = z[i] - zh[i];
#pragma unroll
        for (int c = 0; c < i; ++c) v -= L[i * 4 + c] * w[c];
        w[i] = v / L[i * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) d2 += w[i] * w[i];
      double cost = 1.0 - ((double)acc[q] + (double)comp[q]);
      if (a.cascade) {   // motion-fused cost, tracks x detections row-major
        cost = d2 > a.gate ? INF_COST : a.lam * cost + (1.0 - a.lam) * d2;
        A[(size_t)k * D + j] = cost;
        continue;
      }
      if (d2 > a.gate) cost = INF_COST;
      if (trans)
        A[(size_t)j * M + k] = cost;
      else
        A[(size_t)k * M + j] = cost;
    }
  }
}

// ---------------------------------------------------------------- assignment, update, lifecycle
__device__ __forceinline__ void argmin_warp(double& v, int& j) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, off);
    const int oj = __shfl_xor_sync(0xffffffffu, j, off);
    if (ov < v || (ov == v && oj < j)) {
      v = ov;
      j = oj;
    }
  }
}

// Shortest-augmenting-path Hungarian with row and column potentials on the R x M cost matrix A
// (row-major, R <= M), run by one warp.  On return p[j] is the 1-based row assigned to column j (0 =
// none).  Columns are scanned in ascending order and the first minimum wins.  Returns false when a step
// finds no finite free column (the matrix holds NaN).  This form keeps every column's state in shared
// memory (any M); hungarian_warp_reg keeps it in the registers of the column's lane.
__device__ bool hungarian_warp_smem(const double* A, int R, int M, double* u, double* v, double* minv, int* p, int* way,
                                    uint8_t* used) {
  const int lane = threadIdx.x & 31;
  for (int j = lane; j <= M; j += 32) {
    v[j] = 0.0;
    p[j] = 0;
    way[j] = 0;
  }
  for (int i = lane; i <= R; i += 32) u[i] = 0.0;
  __syncwarp();
  bool fail = false;
  for (int i = 1; i <= R && !fail; ++i) {
    if (lane == 0) p[0] = i;
    for (int j = lane; j <= M; j += 32) {
      minv[j] = INFINITY;
      used[j] = 0;
    }
    __syncwarp();
    int j0 = 0;
    for (int iter = 0; iter <= M; ++iter) {
      if (lane == 0) used[j0] = 1;
      __syncwarp();
      const int i0 = p[j0];
      const double ui0 = u[i0];
      const double* arow = A + (size_t)(i0 - 1) * M;
      double best = INFINITY;
      int bestj = 0x7fffffff;
      for (int j = lane + 1; j <= M; j += 32) {
        if (!used[j]) {
          const double cur = (arow[j - 1] - ui0) - v[j];
          if (cur < minv[j]) {
            minv[j] = cur;
            way[j] = j0;
          }
          if (minv[j] < best) {
            best = minv[j];
            bestj = j;
          }
        }
      }
      argmin_warp(best, bestj);
      if (bestj == 0x7fffffff) {   // no finite free column
        fail = true;
        break;
      }
      const double delta = best;
      for (int j = lane; j <= M; j += 32) {
        if (used[j]) {
          u[p[j]] += delta;
          v[j] -= delta;
        } else {
          minv[j] -= delta;
        }
      }
      __syncwarp();
      j0 = bestj;
      if (p[j0] == 0) break;
    }
    __syncwarp();
    if (lane == 0 && !fail) {
      int jj = j0;
      for (int guard = 0; guard <= M && jj; ++guard) {
        const int j1 = way[jj];
        p[jj] = p[j1];
        jj = j1;
      }
    }
    __syncwarp();
  }
  return !fail;
}

// The same algorithm with the state of column j (1-based) held by lane (j - 1) % 32 in registers: its
// potential v, its slack minv and whether it is used; way and p stay in shared memory (lane 0 walks
// them to augment, every lane reads p for the row potentials).  Columns are visited, compared and
// updated with the same operations in the same order as in hungarian_warp_smem, so the assignment is
// the same.  M <= 32 * CPL.
template <int CPL>
__device__ bool hungarian_warp_reg(const double* A, int R, int M, double* u, int* p, int* way) {
  const int lane = threadIdx.x & 31;
  double vr[CPL], mr[CPL];
  bool ur[CPL];
#pragma unroll
  for (int c = 0; c < CPL; ++c) vr[c] = 0.0;
  for (int j = lane; j <= M; j += 32) {
    p[j] = 0;
    way[j] = 0;
  }
  for (int i = lane; i <= R; i += 32) u[i] = 0.0;
  __syncwarp();
  bool fail = false;
  for (int i = 1; i <= R && !fail; ++i) {
    if (lane == 0) p[0] = i;
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      mr[c] = INFINITY;
      ur[c] = false;
    }
    __syncwarp();
    int j0 = 0;
    for (int iter = 0; iter <= M; ++iter) {
      if (j0 > 0 && ((j0 - 1) & 31) == lane) {   // column j0 becomes used (column 0 always is)
#pragma unroll
        for (int c = 0; c < CPL; ++c)
          if (c == ((j0 - 1) >> 5)) ur[c] = true;
      }
      const int i0 = p[j0];
      const double ui0 = u[i0];
      const double* arow = A + (size_t)(i0 - 1) * M;
      double best = INFINITY;
      int bestj = 0x7fffffff;
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        const int j = lane + 1 + 32 * c;
        if (j <= M && !ur[c]) {
          const double cur = (arow[j - 1] - ui0) - vr[c];
          if (cur < mr[c]) {
            mr[c] = cur;
            way[j] = j0;
          }
          if (mr[c] < best) {
            best = mr[c];
            bestj = j;
          }
        }
      }
      argmin_warp(best, bestj);
      if (bestj == 0x7fffffff) {   // no finite free column
        fail = true;
        break;
      }
      const double delta = best;
      if (lane == 0) u[p[0]] += delta;   // column 0 (the row being added) is used
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        const int j = lane + 1 + 32 * c;
        if (j > M) continue;
        if (ur[c]) {
          u[p[j]] += delta;
          vr[c] -= delta;
        } else {
          mr[c] -= delta;
        }
      }
      __syncwarp();
      j0 = bestj;
      if (p[j0] == 0) break;
    }
    __syncwarp();
    if (lane == 0 && !fail) {
      int jj = j0;
      for (int guard = 0; guard <= M && jj; ++guard) {
        const int j1 = way[jj];
        p[jj] = p[j1];
        jj = j1;
      }
    }
    __syncwarp();
  }
  return !fail;
}

__device__ bool hungarian_warp(const double* A, int R, int M, double* u, double* v, double* minv, int* p, int* way,
                               uint8_t* used) {
  if (M <= 64) return hungarian_warp_reg<2>(A, R, M, u, p, way);
  if (M <= 128) return hungarian_warp_reg<4>(A, R, M, u, p, way);
  return hungarian_warp_smem(A, R, M, u, v, minv, p, way, used);
}

__global__ void __launch_bounds__(256) assign_kernel(StepArgs a, Slots sl) {
  extern __shared__ uint8_t smem[];
  const int b = blockIdx.x;
  const int s = a.dslots ? a.dslots[b] : sl.stream[b];
  const int T = a.t.max_tracks;
  const int Dmax = a.t.max_dets;
  const int nt = a.t.n_tracks[s];
  const int D = det_count(a, b);
  const bool trans = nt > D;
  const int R = trans ? D : nt;   // rows
  const int M = trans ? nt : D;   // cols
  const int MM = T > Dmax ? T : Dmax;
  // the block's cost matrix, read once per Hungarian step, is kept in shared memory when it fits
  double* const cache = reinterpret_cast<double*>(smem);
  double* u = cache + ASSIGN_COST_CACHE;
  double* v = u + (MM + 1);
  double* minv = v + (MM + 1);
  int* p = reinterpret_cast<int*>(minv + (MM + 1));
  int* way = p + (MM + 1);
  int* trk_det = way + (MM + 1);     // [T] by order index
  int* det_trk = trk_det + T;        // [Dmax]
  int* new_order = det_trk + Dmax;   // [T]
  uint8_t* used = reinterpret_cast<uint8_t*>(new_order + T);
  __shared__ int s_fail, s_nnew;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double* const Ag = a.t.cost + (size_t)b * T * Dmax;
  const bool cached = (long long)R * M <= ASSIGN_COST_CACHE;
  for (int k = tid; cached && k < R * M; k += blockDim.x) cache[k] = Ag[k];
  const double* A = cached ? cache : Ag;
  const float* rows = a.rows + (size_t)b * a.cap * 518;
  for (int k = tid; k < T; k += blockDim.x) trk_det[k] = -1;
  for (int j = tid; j < Dmax; j += blockDim.x) det_trk[j] = -1;
  if (tid == 0) s_fail = 0;
  __syncthreads();

  if (warp == 0 && R > 0) {
    if (!hungarian_warp(A, R, M, u, v, minv, p, way, used) && lane == 0) s_fail = 1;
    __syncwarp();
    // pairs, rejected when the (gated) cost is above the threshold
    for (int j = lane + 1; j <= M; j += 32) {
      if (!p[j] || s_fail) continue;
      const int r = p[j] - 1, c = j - 1;
      const double cost = A[(size_t)r * M + c];
      if (cost > (double)a.assign_thresh || cost >= INF_COST) continue;
      const int k = trans ? c : r, d = trans ? r : c;
      trk_det[k] = d;
      det_trk[d] = k;
    }
  }
  __syncthreads();
  if (s_fail) flag_error(a.err, KERR_TIMEOUT);

  // Kalman update of assigned tracks and lost bookkeeping: eight lanes per track (four tracks per
  // warp), lane i forming row i of the gain K, of the mean and of the covariance; every element is
  // computed with the operations, in the order, of the one-thread form (kalman_update)
  {
    const int row = lane & 7;
    const unsigned gmask = 0xFFu << (lane & 24);   // the track's eight lanes
    for (int k0 = warp * 4; k0 < nt; k0 += (blockDim.x / 32) * 4) {
      const int k = k0 + (lane >> 3);
      if (k >= nt) continue;                       // the whole eight-lane group takes this branch
      const int slot = a.t.order[(size_t)s * T + k];
      const size_t ts = (size_t)s * T + slot;
      const int d = trk_det[k];
      if (d < 0) {
        if (row == 0) {
          a.t.state[ts] = JDE_TRACK_LOST;
          a.t.since[ts] += 1;
          a.t.last_det[ts] = -1;
        }
        continue;
      }
      double z[4];
      measurement(rows + (size_t)d * 518, z);
      double* m = a.t.mean + ts * 8;
      double* P = a.t.cov + ts * 64;
      const double* L = a.t.gate_l + ((size_t)b * T + slot) * 16;
      const double hp = m[3];
      const double rp = (SP * hp) * (SP * hp);
      double S[16];
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) S[i * 4 + j] = P[i * 8 + j];
      S[0] += rp;
      S[5] += rp;
      S[10] += 1e-1 * 1e-1;
      S[15] += rp;
      // row `row` of K solves (L L^T) k = (P H^T)[row]
      double Kr[4];
      {
        double t[4];
        for (int r = 0; r < 4; ++r) {
          double vv = P[row * 8 + r];
          for (int c = 0; c < r; ++c) vv -= L[r * 4 + c] * t[c];
          t[r] = vv / L[r * 4 + r];
        }
        for (int r = 3; r >= 0; --r) {
          double vv = t[r];
          for (int c = r + 1; c < 4; ++c) vv -= L[c * 4 + r] * Kr[c];
          Kr[r] = vv / L[r * 4 + r];
        }
      }
      double y[4];
      for (int r = 0; r < 4; ++r) y[r] = z[r] - m[r];
      __syncwarp(gmask);                           // every lane has read m and P before any writes them
      {
        double acc = 0.0;
        for (int r = 0; r < 4; ++r) acc += Kr[r] * y[r];
        m[row] += acc;
      }
      double KS[4];
      for (int c = 0; c < 4; ++c) {
        double acc = 0.0;
        for (int r = 0; r < 4; ++r) acc += Kr[r] * S[r * 4 + c];
        KS[c] = acc;
      }
      for (int j = 0; j < 8; ++j) {
        double Kj[4];
        for (int c = 0; c < 4; ++c) Kj[c] = __shfl_sync(gmask, Kr[c], (lane & 24) + j);
        double acc = 0.0;
        for (int c = 0; c < 4; ++c) acc += KS[c] * Kj[c];
        P[row * 8 + j] -= acc;
      }
      if (row == 0) {
        a.t.state[ts] = JDE_TRACK_TRACKED;
        a.t.since[ts] = 0;
        a.t.last_det[ts] = d;
      }
    }
  }
  __syncthreads();
  // gallery update of assigned tracks (one warp per track): e <- normalise(m e + (1 - m) d)
  for (int k = warp; k < nt; k += blockDim.x / 32) {
    const int d = trk_det[k];
    if (d < 0) continue;
    const int slot = a.t.order[(size_t)s * T + k];
    float* e = a.t.emb + ((size_t)s * T + slot) * 512;
    const float* dv = rows + (size_t)d * 518 + 6;
    float vals[16], ss = 0.f;
    for (int q = 0; q < 16; ++q) {
      const int c = q * 32 + lane;
      vals[q] = a.momentum * e[c] + (1.f - a.momentum) * dv[c];
      ss += vals[q] * vals[q];
    }
    for (int off = 16; off > 0; off >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, off);
    const float inv = ss > 0.f ? 1.f / sqrtf(ss) : 0.f;
    for (int q = 0; q < 16; ++q) e[q * 32 + lane] = vals[q] * inv;
  }
  __syncthreads();
  // removal, order compaction and births (serial bookkeeping on one thread; O(T + D) integer work)
  if (tid == 0) {
    int nn = 0;
    int top = a.t.free_top[s];
    for (int k = 0; k < nt; ++k) {
      const int slot = a.t.order[(size_t)s * T + k];
      const size_t ts = (size_t)s * T + slot;
      if (a.t.state[ts] == JDE_TRACK_LOST && a.t.since[ts] > a.lost_max) {
        a.t.free_stack[(size_t)s * T + top++] = slot;
        continue;
      }
      new_order[nn++] = slot;
    }
    long long nid = a.t.next_id[s];
    for (int j = 0; j < D; ++j) {
      if (det_trk[j] >= 0) continue;
      if (top == 0 || nn >= T) {
        flag_error(a.err, KERR_CAPACITY);
        break;
      }
      const int slot = a.t.free_stack[(size_t)s * T + --top];
      const size_t ts = (size_t)s * T + slot;
      a.t.id[ts] = nid++;
      a.t.state[ts] = JDE_TRACK_TRACKED;
      a.t.since[ts] = 0;
      a.t.last_det[ts] = j;
      det_trk[j] = -2 - slot;   // marks the birth slot for the parallel init below
      new_order[nn++] = slot;
    }
    a.t.next_id[s] = nid;
    a.t.free_top[s] = top;
    s_nnew = nn;
  }
  __syncthreads();
  const int nn = s_nnew;
  for (int k = tid; k < nn; k += blockDim.x) a.t.order[(size_t)s * T + k] = new_order[k];
  // initialise born tracks: x = (z, 0), P0 from the measured height, gallery = detection embedding
  for (int j = tid; j < D; j += blockDim.x) {
    if (det_trk[j] > -2) continue;
    const int slot = -2 - det_trk[j];
    const size_t ts = (size_t)s * T + slot;
    double z[4];
    measurement(rows + (size_t)j * 518, z);
    double* m = a.t.mean + ts * 8;
    double* P = a.t.cov + ts * 64;
    for (int i = 0; i < 4; ++i) {
      m[i] = z[i];
      m[i + 4] = 0.0;
    }
    for (int i = 0; i < 64; ++i) P[i] = 0.0;
    const double h = z[3];
    const double sp2 = (2 * SP * h) * (2 * SP * h), sv2 = (10 * SV * h) * (10 * SV * h);
    P[0] = sp2;
    P[9] = sp2;
    P[18] = 1e-2 * 1e-2;
    P[27] = sp2;
    P[36] = sv2;
    P[45] = sv2;
    P[54] = 1e-5 * 1e-5;
    P[63] = sv2;
  }
  for (int j = warp; j < D; j += blockDim.x / 32) {
    if (det_trk[j] > -2) continue;
    const int slot = -2 - det_trk[j];
    float* e = a.t.emb + ((size_t)s * T + slot) * 512;
    const float* dv = rows + (size_t)j * 518 + 6;
    for (int q = 0; q < 16; ++q) e[q * 32 + lane] = dv[q * 32 + lane];
  }
  if (tid == 0) {
    a.t.n_tracks[s] = nn;
    a.t.frames[s] += 1;
  }
  __syncthreads();
  // output in track order
  if (tid == 0) a.o_count[b] = nn;
  for (int k = tid; k < nn && k < a.o_cap; k += blockDim.x) {
    const int slot = new_order[k];
    const size_t ts = (size_t)s * T + slot;
    const double* m = a.t.mean + ts * 8;
    const size_t o = (size_t)b * a.o_cap + k;
    const double w = m[2] * m[3];
    a.o_id[o] = a.t.id[ts];
    a.o_box[o * 4 + 0] = (float)(m[0] - w / 2);
    a.o_box[o * 4 + 1] = (float)(m[1] - m[3] / 2);
    a.o_box[o * 4 + 2] = (float)(m[0] + w / 2);
    a.o_box[o * 4 + 3] = (float)(m[1] + m[3] / 2);
    a.o_state[o] = a.t.state[ts];
    if (a.o_det) a.o_det[o] = a.t.last_det[ts];
  }
}


// IoU of the track's Kalman box (state mean: cx, cy, a, h) and a detection row's box (x1, y1, x2, y2).
__device__ double iou_mean_row(const double* m, const float* row) {
  const double w = m[2] * m[3];
  const double ax1 = m[0] - w / 2, ay1 = m[1] - m[3] / 2, ax2 = m[0] + w / 2, ay2 = m[1] + m[3] / 2;
  const double bx1 = row[0], by1 = row[1], bx2 = row[2], by2 = row[3];
  const double iw = fmax(0.0, fmin(ax2, bx2) - fmax(ax1, bx1));
  const double ih = fmax(0.0, fmin(ay2, by2) - fmax(ay1, by1));
  const double inter = iw * ih;
  const double uni = (ax2 - ax1) * (ay2 - ay1) + (bx2 - bx1) * (by2 - by1) - inter;
  return uni > 0.0 ? inter / uni : 0.0;
}

// Kalman update of track slot ts with measurement z (K = P H^T S^-1 through the factor L of S,
// x += K (z - H x), P -= K S K^T).
__device__ void kalman_update(double* m, double* P, const double* L, const double (&z)[4]) {
  const double hp = m[3];
  const double rp = (SP * hp) * (SP * hp);
  double S[16];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) S[i * 4 + j] = P[i * 8 + j];
  S[0] += rp;
  S[5] += rp;
  S[10] += 1e-1 * 1e-1;
  S[15] += rp;
  double K[32];
  for (int i = 0; i < 8; ++i) {
    double t[4];
    for (int r = 0; r < 4; ++r) {
      double vv = P[i * 8 + r];
      for (int c = 0; c < r; ++c) vv -= L[r * 4 + c] * t[c];
      t[r] = vv / L[r * 4 + r];
    }
    for (int r = 3; r >= 0; --r) {
      double vv = t[r];
      for (int c = r + 1; c < 4; ++c) vv -= L[c * 4 + r] * K[i * 4 + c];
      K[i * 4 + r] = vv / L[r * 4 + r];
    }
  }
  double y[4];
  for (int r = 0; r < 4; ++r) y[r] = z[r] - m[r];
  for (int i = 0; i < 8; ++i) {
    double acc = 0.0;
    for (int r = 0; r < 4; ++r) acc += K[i * 4 + r] * y[r];
    m[i] += acc;
  }
  double KS[32];
  for (int i = 0; i < 8; ++i)
    for (int c = 0; c < 4; ++c) {
      double acc = 0.0;
      for (int r = 0; r < 4; ++r) acc += K[i * 4 + r] * S[r * 4 + c];
      KS[i * 4 + c] = acc;
    }
  for (int i = 0; i < 8; ++i)
    for (int j = 0; j < 8; ++j) {
      double acc = 0.0;
      for (int c = 0; c < 4; ++c) acc += KS[i * 4 + c] * K[j * 4 + c];
      P[i * 8 + j] -= acc;
    }
}

// Three-stage association (one block per stream): stage 1 confirmed tracks x all detections on the fused
// cost, stage 2 the confirmed tracks left that were tracked before the step x the detections left on
// 1 - IoU, stage 3 unconfirmed tracks x the detections still left on 1 - IoU.  Each stage's sub-matrix
// (rows in creation order, columns in kept order, transposed when it has more rows) is solved by the
// warp Hungarian; pairs above the stage's threshold (or "infinite") are rejected.  Then Kalman and
// gallery updates of every matched track, lost bookkeeping of unmatched confirmed tracks, removal of
// unmatched unconfirmed ones, births (confirmed on the stream's first step, else unconfirmed), output.
constexpr int STATE_REMOVED = 0;
__global__ void __launch_bounds__(256) assign_cascade_kernel(StepArgs a, Slots sl) {
  extern __shared__ uint8_t smem[];
  const int b = blockIdx.x;
  const int s = a.dslots ? a.dslots[b] : sl.stream[b];
  const int T = a.t.max_tracks;
  const int Dmax = a.t.max_dets;
  const int nt = a.t.n_tracks[s];
  const int D = det_count(a, b);
  const int MM = T > Dmax ? T : Dmax;
  double* const cache = reinterpret_cast<double*>(smem);
  double* u = cache + ASSIGN_COST_CACHE;
  double* v = u + (MM + 1);
  double* minv = v + (MM + 1);
  int* p = reinterpret_cast<int*>(minv + (MM + 1));
  int* way = p + (MM + 1);
  int* trk_det = way + (MM + 1);     // [T] by order index
  int* det_trk = trk_det + T;        // [Dmax]
  int* new_order = det_trk + Dmax;   // [T]
  int* ridx = new_order + T;         // [MM] rows of the current stage (order indices)
  int* cidx = ridx + MM;             // [MM] columns of the current stage (detection rows)
  int* pstate = cidx + MM;           // [T] state of each track before the step
  uint8_t* used = reinterpret_cast<uint8_t*>(pstate + T);
  __shared__ int s_fail, s_nr, s_nc, s_nnew;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double* const full = a.t.cost + (size_t)b * T * Dmax;    // stage-1 cost [nt][D]
  double* const big = a.t.cost2 + (size_t)b * T * Dmax;          // sub-matrices above the shared cache
  const float* rows = a.rows + (size_t)b * a.cap * 518;
  for (int k = tid; k < T; k += blockDim.x) trk_det[k] = -1;
  for (int j = tid; j < Dmax; j += blockDim.x) det_trk[j] = -1;
  for (int k = tid; k < nt; k += blockDim.x) pstate[k] = a.t.state[(size_t)s * T + a.t.order[(size_t)s * T + k]];
  if (tid == 0) s_fail = 0;
  __syncthreads();

  for (int stage = 0; stage < 3; ++stage) {
    if (tid == 0) {   // the stage's rows and columns, in order (O(T + D) integer work)
      int nr = 0, nc = 0;
      for (int k = 0; k < nt; ++k) {
        const int ps = pstate[k];
        const bool take = stage == 0   ? ps != JDE_TRACK_UNCONFIRMED
                          : stage == 1 ? (ps == JDE_TRACK_TRACKED && trk_det[k] < 0)
                                       : ps == JDE_TRACK_UNCONFIRMED;
        if (take) ridx[nr++] = k;
      }
      for (int j = 0; j < D; ++j)
        if (det_trk[j] < 0) cidx[nc++] = j;
      s_nr = nr;
      s_nc = nc;
    }
    __syncthreads();
    const int nr = s_nr, nc = s_nc;
    if (nr == 0 || nc == 0 || s_fail) continue;   // block-uniform
    const bool trans = nr > nc;
    const int R = trans ? nc : nr, M = trans ? nr : nc;
    double* const A = (long long)R * M <= ASSIGN_COST_CACHE ? cache : big;
    for (int e = tid; e < R * M; e += blockDim.x) {
      const int r = e / M, c = e - (e / M) * M;
      const int k = ridx[trans ? c : r], j = cidx[trans ? r : c];
      double cost;
      if (stage == 0) {
        cost = full[(size_t)k * D + j];
      } else {
        const int slot = a.t.order[(size_t)s * T + k];
        cost = 1.0 - iou_mean_row(a.t.mean + ((size_t)s * T + slot) * 8, rows + (size_t)j * 518);
      }
      A[e] = cost;
    }
    __syncthreads();
    if (warp == 0) {
      const bool ok = hungarian_warp(A, R, M, u, v, minv, p, way, used);
      if (!ok && lane == 0) s_fail = 1;
      const double thr = stage == 0 ? (double)a.assign_thresh : (stage == 1 ? a.iou2 : a.iou3);
      for (int jj = lane + 1; ok && jj <= M; jj += 32) {
        if (!p[jj]) continue;
        const int r = p[jj] - 1, c = jj - 1;
        const double cost = A[(size_t)r * M + c];
        if (cost > thr || cost >= INF_COST) continue;
        const int k = ridx[trans ? c : r], j = cidx[trans ? r : c];
        trk_det[k] = j;
        det_trk[j] = k;
      }
    }
    __syncthreads();
  }
  if (s_fail) flag_error(a.err, KERR_TIMEOUT);

  // Kalman update of matched tracks; lost bookkeeping; unmatched unconfirmed tracks marked removed
  for (int k = tid; k < nt; k += blockDim.x) {
    const int slot = a.t.order[(size_t)s * T + k];
    const size_t ts = (size_t)s * T + slot;
    const int d = trk_det[k];
    if (d >= 0) {
      double z[4];
      measurement(rows + (size_t)d * 518, z);
      kalman_update(a.t.mean + ts * 8, a.t.cov + ts * 64, a.t.gate_l + ((size_t)b * T + slot) * 16, z);
      a.t.state[ts] = JDE_TRACK_TRACKED;
      a.t.since[ts] = 0;
      a.t.last_det[ts] = d;
    } else if (pstate[k] == JDE_TRACK_UNCONFIRMED) {
      a.t.state[ts] = STATE_REMOVED;
      a.t.last_det[ts] = -1;
    } else {
      a.t.state[ts] = JDE_TRACK_LOST;
      a.t.since[ts] += 1;
      a.t.last_det[ts] = -1;
    }
  }
  __syncthreads();
  // gallery update of matched tracks (one warp per track): e <- normalise(m e + (1 - m) d)
  for (int k = warp; k < nt; k += blockDim.x / 32) {
    const int d = trk_det[k];
    if (d < 0) continue;
    const int slot = a.t.order[(size_t)s * T + k];
    float* e = a.t.emb + ((size_t)s * T + slot) * 512;
    const float* dv = rows + (size_t)d * 518 + 6;
    float vals[16], ss = 0.f;
    for (int q = 0; q < 16; ++q) {
      const int c = q * 32 + lane;
      vals[q] = a.momentum * e[c] + (1.f - a.momentum) * dv[c];
      ss += vals[q] * vals[q];
    }
    for (int off = 16; off > 0; off >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, off);
    const float inv = ss > 0.f ? 1.f / sqrtf(ss) : 0.f;
    for (int q = 0; q < 16; ++q) e[q * 32 + lane] = vals[q] * inv;
  }
  __syncthreads();
  // removals, order compaction and births (one thread; O(T + D) integer work)
  if (tid == 0) {
    int nn = 0;
    int top = a.t.free_top[s];
    for (int k = 0; k < nt; ++k) {
      const int slot = a.t.order[(size_t)s * T + k];
      const size_t ts = (size_t)s * T + slot;
      if (a.t.state[ts] == STATE_REMOVED || (a.t.state[ts] == JDE_TRACK_LOST && a.t.since[ts] > a.lost_max)) {
        a.t.free_stack[(size_t)s * T + top++] = slot;
        continue;
      }
      new_order[nn++] = slot;
    }
    const int born_state = a.t.frames[s] == 0 ? JDE_TRACK_TRACKED : JDE_TRACK_UNCONFIRMED;
    long long nid = a.t.next_id[s];
    for (int j = 0; j < D; ++j) {
      if (det_trk[j] >= 0) continue;
      if (top == 0 || nn >= T) {
        flag_error(a.err, KERR_CAPACITY);
        break;
      }
      const int slot = a.t.free_stack[(size_t)s * T + --top];
      const size_t ts = (size_t)s * T + slot;
      a.t.id[ts] = nid++;
      a.t.state[ts] = born_state;
      a.t.since[ts] = 0;
      a.t.last_det[ts] = j;
      det_trk[j] = -2 - slot;   // marks the birth slot for the parallel init below
      new_order[nn++] = slot;
    }
    a.t.next_id[s] = nid;
    a.t.free_top[s] = top;
    s_nnew = nn;
  }
  __syncthreads();
  const int nn = s_nnew;
  for (int k = tid; k < nn; k += blockDim.x) a.t.order[(size_t)s * T + k] = new_order[k];
  for (int j = tid; j < D; j += blockDim.x) {
    if (det_trk[j] > -2) continue;
    const int slot = -2 - det_trk[j];
    const size_t ts = (size_t)s * T + slot;
    double z[4];
    measurement(rows + (size_t)j * 518, z);
    double* m = a.t.mean + ts * 8;
    double* P = a.t.cov + ts * 64;
    for (int i = 0; i < 4; ++i) {
      m[i] = z[i];
      m[i + 4] = 0.0;
    }
    for (int i = 0; i < 64; ++i) P[i] = 0.0;
    const double h = z[3];
    const double sp2 = (2 * SP * h) * (2 * SP * h), sv2 = (10 * SV * h) * (10 * SV * h);
    P[0] = sp2;
    P[9] = sp2;
    P[18] = 1e-2 * 1e-2;
    P[27] = sp2;
    P[36] = sv2;
    P[45] = sv2;
    P[54] = 1e-5 * 1e-5;
    P[63] = sv2;
  }
  for (int j = warp; j < D; j += blockDim.x / 32) {
    if (det_trk[j] > -2) continue;
    const int slot = -2 - det_trk[j];
    float* e = a.t.emb + ((size_t)s * T + slot) * 512;
    const float* dv = rows + (size_t)j * 518 + 6;
    for (int q = 0; q < 16; ++q) e[q * 32 + lane] = dv[q * 32 + lane];
  }
  if (tid == 0) {
    a.t.n_tracks[s] = nn;
    a.t.frames[s] += 1;
    a.o_count[b] = nn;
  }
  __syncthreads();
  for (int k = tid; k < nn && k < a.o_cap; k += blockDim.x) {
    const int slot = new_order[k];
    const size_t ts = (size_t)s * T + slot;
    const double* m = a.t.mean + ts * 8;
    const size_t o = (size_t)b * a.o_cap + k;
    const double w = m[2] * m[3];
    a.o_id[o] = a.t.id[ts];
    a.o_box[o * 4 + 0] = (float)(m[0] - w / 2);
    a.o_box[o * 4 + 1] = (float)(m[1] - m[3] / 2);
    a.o_box[o * 4 + 2] = (float)(m[0] + w / 2);
    a.o_box[o * 4 + 3] = (float)(m[1] + m[3] / 2);
    a.o_state[o] = a.t.state[ts];
    if (a.o_det) a.o_det[o] = a.t.last_det[ts];
  }
}

size_t assign_smem(const TrackState& t) {
  const int MM = t.max_tracks > t.max_dets ? t.max_tracks : t.max_dets;
  return sizeof(double) * ASSIGN_COST_CACHE + sizeof(double) * 3 * (MM + 1) + sizeof(int) * 2 * (MM + 1) + sizeof(int) * (2 * t.max_tracks + t.max_dets) +
         (MM + 1) + 16;
}
// the cascade adds the stage's row and column lists and the tracks' states before the step
size_t cascade_smem(const TrackState& t) {
  const int MM = t.max_tracks > t.max_dets ? t.max_tracks : t.max_dets;
  return assign_smem(t) + sizeof(int) * (2 * (size_t)MM + t.max_tracks);
}

bool dalloc(void** p, size_t bytes) {
  if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return false;
  }
  return true;
}

}  // namespace

size_t track_bytes(const jde_config& cfg) {
  const size_t S = cfg.max_streams, T = cfg.max_tracks, D = cfg.max_track_dets;
  const size_t B = cfg.max_batch < MAXB ? cfg.max_batch : MAXB;
  return sizeof(int) * S + sizeof(long long) * S + 2 * sizeof(int) * S * T + sizeof(int) * S +
         sizeof(long long) * S * T + 2 * sizeof(int) * S * T + sizeof(double) * S * T * (8 + 64) +
         sizeof(float) * S * T * 512 + sizeof(int) * S * T + sizeof(double) * B * T * (16 + 4) +
         sizeof(double) * B * T * D * (cfg.assoc_cascade ? 2 : 1) + sizeof(int) * B + sizeof(int) * S;
}

int track_alloc(TrackState& t, const jde_config& cfg) {
  t.max_streams = cfg.max_streams;
  t.max_tracks = cfg.max_tracks;
  t.max_dets = cfg.max_track_dets;
  t.max_batch = cfg.max_batch < MAXB ? cfg.max_batch : MAXB;
  const size_t S = t.max_streams, T = t.max_tracks, B = t.max_batch, D = t.max_dets;
  bool ok = dalloc((void**)&t.n_tracks, sizeof(int) * S) && dalloc((void**)&t.next_id, sizeof(long long) * S) &&
            dalloc((void**)&t.order, sizeof(int) * S * T) && dalloc((void**)&t.free_stack, sizeof(int) * S * T) &&
            dalloc((void**)&t.free_top, sizeof(int) * S) && dalloc((void**)&t.id, sizeof(long long) * S * T) &&
            dalloc((void**)&t.state, sizeof(int) * S * T) && dalloc((void**)&t.since, sizeof(int) * S * T) &&
            dalloc((void**)&t.mean, sizeof(double) * S * T * 8) && dalloc((void**)&t.cov, sizeof(double) * S * T * 64) &&
            dalloc((void**)&t.emb, sizeof(float) * S * T * 512) && dalloc((void**)&t.last_det, sizeof(int) * S * T) &&
            dalloc((void**)&t.gate_l, sizeof(double) * B * T * 16) && dalloc((void**)&t.gate_z, sizeof(double) * B * T * 4) &&
            dalloc((void**)&t.cost, sizeof(double) * B * T * D) && dalloc((void**)&t.slot_stream, sizeof(int) * B) &&
            dalloc((void**)&t.frames, sizeof(int) * S);
  t.cascade = cfg.assoc_cascade ? 1 : 0;
  if (ok && t.cascade) ok = dalloc((void**)&t.cost2, sizeof(double) * B * T * D);
  if (!ok) return 1;
  if (t.cascade && cudaFuncSetAttribute(assign_cascade_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)cascade_smem(t)) != cudaSuccess)
    return 1;
  if (cudaFuncSetAttribute(assign_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)assign_smem(t)) !=
      cudaSuccess)
    return 1;
  for (int s = 0; s < t.max_streams; ++s) {
    jde_count_launch();
    reset_kernel<<<1, 256>>>(t, s);
  }
  return cudaDeviceSynchronize() == cudaSuccess ? 0 : 1;
}

void track_free(TrackState& t) {
  void* ptrs[] = {t.n_tracks, t.next_id, t.order, t.free_stack, t.free_top, t.id, t.state, t.since, t.mean, t.cov,
                  t.emb, t.last_det, t.gate_l, t.gate_z, t.cost, t.cost2, t.frames, t.slot_stream, t.rows_stage, t.count_stage,
                  t.o_id, t.o_box, t.o_state, t.o_det, t.o_count};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  t = TrackState();
}

int track_reset(TrackState& t, int s, cudaStream_t st) {
  jde_count_launch();
  reset_kernel<<<1, 256, 0, st>>>(t, s);
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

int track_step(TrackState& t, const jde_config& cfg, int n, const int32_t* stream_ids, const jde_dets* dets,
               jde_tracks* out, int* err, cudaStream_t st, char* msg, size_t msg_len, const int* dev_slots) {
  if (n < 1 || n > t.max_batch || !stream_ids || !dets || !out || !dets->rows || !dets->count || dets->cap < 1 ||
      !out->id || !out->box || !out->state || !out->count || out->cap < 1) {
    snprintf(msg, msg_len, "bad arguments (n=%d, at most %d streams per call)", n, t.max_batch);
    return JDE_ERR_INVALID_ARG;
  }
  Slots sl;
  for (int i = 0; i < n; ++i) {
    if (stream_ids[i] < 0 || stream_ids[i] >= t.max_streams) {
      snprintf(msg, msg_len, "stream id %d out of range", stream_ids[i]);
      return JDE_ERR_NOT_FOUND;
    }
    for (int j = 0; j < i; ++j)
      if (stream_ids[j] == stream_ids[i]) {
        snprintf(msg, msg_len, "stream id %d appears twice in one call", stream_ids[i]);
        return JDE_ERR_INVALID_ARG;
      }
    sl.stream[i] = stream_ids[i];
  }
  const float* rows = dets->rows;
  const int32_t* count = dets->count;
  if (!dets->on_device) {
    const size_t need = (size_t)t.max_batch * dets->cap * 518;
    if (!t.rows_stage || need > t.rows_stage_cap) {
      cudaFree(t.rows_stage);
      cudaFree(t.count_stage);
      if (!dalloc((void**)&t.rows_stage, sizeof(float) * need) ||
          !dalloc((void**)&t.count_stage, sizeof(int32_t) * t.max_batch)) {
        snprintf(msg, msg_len, "detection staging");
        return JDE_ERR_OOM;
      }
      t.rows_stage_cap = need;
    }
    if (cudaMemcpyAsync(t.rows_stage, dets->rows, sizeof(float) * (size_t)n * dets->cap * 518, cudaMemcpyHostToDevice,
                        st) != cudaSuccess ||
        cudaMemcpyAsync(t.count_stage, dets->count, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      snprintf(msg, msg_len, "staging copy failed");
      return JDE_ERR_CUDA;
    }
    rows = t.rows_stage;
    count = t.count_stage;
  }
  StepArgs a;
  a.t = t;
  a.rows = rows;
  a.count = count;
  a.cap = dets->cap;
  a.n = n;
  a.gate = cfg.gate_chi2;
  a.assign_thresh = cfg.assign_thresh;
  a.lost_max = cfg.lost_max_frames;
  a.momentum = cfg.emb_momentum;
  a.dslots = dev_slots;
  a.cascade = t.cascade;
  a.lam = cfg.motion_lambda;
  a.iou2 = cfg.iou_cost2;
  a.iou3 = cfg.iou_cost3;
  a.err = err;
  a.o_cap = out->cap;
  if (out->on_device) {
    a.o_id = reinterpret_cast<long long*>(out->id);
    a.o_box = out->box;
    a.o_state = out->state;
    a.o_det = out->det;
    a.o_count = out->count;
  } else {
    if (!t.o_id || out->cap > t.o_cap) {
      void* ptrs[] = {t.o_id, t.o_box, t.o_state, t.o_det, t.o_count};
      for (void* p : ptrs)
        if (p) cudaFree(p);
      const size_t c = (size_t)t.max_batch * out->cap;
      if (!(dalloc((void**)&t.o_id, sizeof(long long) * c) && dalloc((void**)&t.o_box, sizeof(float) * 4 * c) &&
            dalloc((void**)&t.o_state, sizeof(int32_t) * c) && dalloc((void**)&t.o_det, sizeof(int32_t) * c) &&
            dalloc((void**)&t.o_count, sizeof(int32_t) * t.max_batch))) {
        snprintf(msg, msg_len, "track output staging");
        return JDE_ERR_OOM;
      }
      t.o_cap = out->cap;
      a.t = t;
    }
    a.o_id = t.o_id;
    a.o_box = t.o_box;
    a.o_state = t.o_state;
    a.o_det = t.o_det;
    a.o_count = t.o_count;
  }
  dim3 gp((t.max_tracks + 127) / 128, n);
  jde_count_launch();
  prep_kernel<<<gp, 128, 0, st>>>(a, sl);
  dim3 gc(COST_BLOCKS, n);
  jde_count_launch();
  cost_kernel<<<gc, 256, 0, st>>>(a, sl);
  jde_count_launch();
  if (t.cascade)
    assign_cascade_kernel<<<n, 256, cascade_smem(t), st>>>(a, sl);
  else
    assign_kernel<<<n, 256, assign_smem(t), st>>>(a, sl);
  if (cudaGetLastError() != cudaSuccess) {
    snprintf(msg, msg_len, "tracker launch failed");
    return JDE_ERR_CUDA;
  }
  if (!out->on_device) {
    const size_t c = (size_t)n * out->cap;
    bool ok = cudaMemcpyAsync(out->count, a.o_count, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
              cudaMemcpyAsync(out->id, a.o_id, sizeof(long long) * c, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
              cudaMemcpyAsync(out->box, a.o_box, sizeof(float) * 4 * c, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
              cudaMemcpyAsync(out->state, a.o_state, sizeof(int32_t) * c, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
              (!out->det ||
               cudaMemcpyAsync(out->det, a.o_det, sizeof(int32_t) * c, cudaMemcpyDeviceToHost, st) == cudaSuccess) &&
              cudaStreamSynchronize(st) == cudaSuccess;
    if (!ok) {
      snprintf(msg, msg_len, "track output copy failed");
      return JDE_ERR_CUDA;
    }
    for (int i = 0; i < n; ++i)
      if (out->count[i] > out->cap) {
        snprintf(msg, msg_len, "stream %d has %d tracks, cap is %d", stream_ids[i], out->count[i], out->cap);
        return JDE_ERR_CAPACITY;
      }
  }
  return JDE_OK;
}
