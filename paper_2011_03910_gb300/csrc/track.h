// Device-resident multi-stream tracker state and the tracker step (Appendix A items 4-9).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/jde.h"

struct TrackState {
  int max_streams = 0, max_tracks = 0, max_dets = 0, max_batch = 0;
  // per stream slot
  int* n_tracks = nullptr;          // [S]
  long long* next_id = nullptr;     // [S]
  int* order = nullptr;             // [S][T]  slot of the k-th track in track (creation) order
  int* free_stack = nullptr;        // [S][T]  free track slots
  int* free_top = nullptr;          // [S]
  // per stream slot x track (SoA)
  long long* id = nullptr;          // [S][T]
  int* state = nullptr;             // [S][T]
  int* since = nullptr;             // [S][T]  frames since the last update
  double* mean = nullptr;           // [S][T][8]
  double* cov = nullptr;            // [S][T][64]
  float* emb = nullptr;             // [S][T][512]
  int* last_det = nullptr;          // [S][T]  detection row assigned in the last step, -1 if none
  int* frames = nullptr;            // [S]     steps since the stream's reset (births on step 0 are confirmed)
  // per call slot scratch (call slot b < max_batch)
  double* gate_l = nullptr;         // [B][T][16]  Cholesky factor of S (row-major 4x4)
  double* gate_z = nullptr;         // [B][T][4]   projected mean H x
  double* cost = nullptr;           // [B][T*D]    gated cost, rows = min(T, D); cascade: fused cost [T][D]
  double* cost2 = nullptr;          // [B][T*D]    cascade: a stage's sub-matrix when it exceeds the shared cache
  int cascade = 0;                  // three-stage association (jde_config.assoc_cascade)
  int* slot_stream = nullptr;       // [B]
  float* rows_stage = nullptr;      // [B][cap][518] host-provided detections staged on the device
  size_t rows_stage_cap = 0;        // floats rows_stage holds
  int32_t* count_stage = nullptr;   // [B]
  // output staging for host outputs
  long long* o_id = nullptr;
  float* o_box = nullptr;
  int32_t* o_state = nullptr;
  int32_t* o_det = nullptr;
  int32_t* o_count = nullptr;
  int o_cap = 0;
};

int track_alloc(TrackState& t, const jde_config& cfg);
size_t track_bytes(const jde_config& cfg);   // device bytes track_alloc takes
void track_free(TrackState& t);
int track_reset(TrackState& t, int stream_id, cudaStream_t st);
// Returns a jde_status value; msg receives a reason on failure.  dev_slots (device, n ints, optional): the
// kernels read the stream slots from it instead of the by-value copy of stream_ids (a captured CUDA graph
// then serves any set of streams; stream_ids is still validated and must hold the same ids).
int track_step(TrackState& t, const jde_config& cfg, int n, const int32_t* stream_ids, const jde_dets* dets,
               jde_tracks* out, int* err, cudaStream_t st, char* msg, size_t msg_len, const int* dev_slots = nullptr);
