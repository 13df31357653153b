// Serving many video streams through one process (the GB300 counterpart of the paper's capture ->
// prediction -> post-processing processes connected by queues, Sec. 4.3-4.4): admission by a device-memory
// budget, continuous batching per model input size, and CUDA-graph replay of each batch's launch sequence.
//
// Structure:
//   * a group per model input size: one library handle (weights, activations, post-processing scratch,
//     the tracker state of its streams), one CUDA stream, and the group's batch buffers (frames, optional
//     caller head tensors, detection rows, track outputs, the network's detection maps when collected);
//   * jde_stream_open admits a stream into the group of its size if the group has a free tracker slot, or
//     creates the group if its device memory (the handle's allocation rule plus the group buffers) fits in
//     what the budget has left; jde_stream_close frees the slot and destroys an empty group;
//   * jde_submit queues a frame of a stream; jde_poll collects finished batches (event queries, no
//     blocking) and launches, in every group with no batch on the device, the queued frames (at most
//     max_batch, at most one per stream: a stream's tracker steps are sequential);
//   * a batch of n frames is: device copies of its frames (and caller heads) into the group buffers, the
//     stream slots copied to the device, then forward + post-processing + tracker step, either eagerly or
//     as a CUDA graph captured at the first eager-warmed launch of that n; then the outputs are copied to
//     pinned host memory and an event closes the batch.
// Every computation runs in libjde's kernels; this file only schedules and moves buffers.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <deque>
#include <map>
#include <string>
#include <vector>

#include "../../include/jde.h"
#include "internal.h"

namespace {

struct Pending {
  long long ticket;
  int stream_id;
  const uint8_t* frame;     // device, src_h x src_w x 3
  const float* heads[6];    // device per-frame head tensors (caller_heads), else null
  cudaEvent_t ready;        // the frame's inputs are complete when this event has completed, or null
  jde_frame_out out;        // host outputs filled when the frame's result is collected
};

struct Group;

struct StreamRec {
  Group* g = nullptr;
  int slot = -1;
  int inflight = 0;         // frames submitted and not yet collected
};

struct Batch {
  std::vector<Pending> frames;
  cudaEvent_t done = nullptr;
  int n = 0;
};

struct Group {
  int in_w = 0, in_h = 0;
  jde_handle* h = nullptr;
  cudaStream_t st = nullptr;
  std::vector<int> free_slots;
  std::deque<Pending> queue;
  std::deque<Batch> inflight;
  size_t charged = 0;
  // device batch buffers
  uint8_t* frames = nullptr;
  float* heads[6] = {nullptr};
  size_t head_bytes[6] = {0};   // bytes of one frame's head tensor
  float* rows = nullptr;
  int32_t* count = nullptr;
  int64_t* t_id = nullptr;
  float* t_box = nullptr;
  int32_t* t_state = nullptr;
  int32_t* t_det = nullptr;
  int32_t* t_count = nullptr;
  float* net_det[3] = {nullptr};
  size_t net_bytes[3] = {0};    // bytes of one frame's detection map
  int* d_slots = nullptr;
  int* h_slots = nullptr;       // pinned
  // pinned host staging of the outputs of the batch in flight
  int32_t* p_count = nullptr;
  int64_t* p_id = nullptr;
  float* p_box = nullptr;
  int32_t* p_state = nullptr;
  int32_t* p_tcount = nullptr;
  int32_t* p_det = nullptr;
  float* p_rows = nullptr;
  float* p_net[3] = {nullptr};
  std::map<int, cudaGraphExec_t> graphs;   // per batch size
  std::map<int, int> warmed;               // eager launches done per batch size
};

}  // namespace

struct jde_server {
  jde_server_config cfg;
  std::vector<uint8_t> weights;
  std::map<std::pair<int, int>, Group*> groups;
  std::map<int, StreamRec> streams;
  int next_stream = 0;
  long long next_ticket = 1;
  size_t used = 0;
  cudaEvent_t start = nullptr;
  std::deque<jde_frame_result> ready;
  std::string err;
  std::vector<int> det_layers;
  long long eager = 0, captured = 0, replays = 0;
};

namespace {

jde_status sfail(jde_server* s, jde_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (s) s->err = buf;
  return st;
}

#define S_CUDA(s, call)                                                                              \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess) return sfail((s), JDE_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

jde_config group_config(const jde_server_config& sc, int in_w, int in_h) {
  jde_config c = sc.group;
  c.max_in_w = in_w;
  c.max_in_h = in_h;
  c.max_src_w = sc.src_w;
  c.max_src_h = sc.src_h;
  c.max_streams = sc.max_streams_per_group;
  if (sc.caller_heads) c.sparse_emb = 0;
  return c;
}

// Device bytes of a group's own buffers (next to its handle).
size_t group_buffer_bytes(const jde_server_config& sc, int in_w, int in_h) {
  const size_t B = (size_t)sc.group.max_batch;
  const int st[3] = {32, 16, 8};
  size_t cells = 0;
  for (int k = 0; k < 3; ++k) cells += (size_t)(in_w / st[k]) * (in_h / st[k]);
  size_t b = B * sc.src_w * sc.src_h * 3;                     // frames
  if (sc.caller_heads) b += B * cells * (24 + 512) * 4;        // caller heads
  b += B * sc.det_cap * 518 * 4 + B * 4;                      // rows, count
  b += B * sc.track_cap * (8 + 16 + 4 + 4) + B * 4;           // id, box, state, det; count
  if (sc.collect_net_heads) b += B * cells * 24 * 4;           // the network's detection maps
  b += B * sizeof(int);                                       // stream slots
  return b;
}

bool server_config_ok(const jde_server_config& c) {
  return c.max_streams_per_group >= 1 && c.max_streams_per_group <= 1024 && c.src_w >= 1 && c.src_h >= 1 &&
         c.src_w <= 16384 && c.src_h <= 16384 && c.det_cap >= 1 && c.track_cap >= 1 && c.group.max_batch >= 1 &&
         c.group.max_batch <= 64;
}

bool galloc(void** p, size_t bytes) {
  if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return false;
  }
  return true;
}
bool halloc(void** p, size_t bytes) {
  if (cudaHostAlloc(p, bytes ? bytes : 16, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return false;
  }
  return true;
}

void group_free(Group* g) {
  if (!g) return;
  if (g->st) cudaStreamSynchronize(g->st);
  for (auto& kv : g->graphs) cudaGraphExecDestroy(kv.second);
  for (auto& b : g->inflight)
    if (b.done) cudaEventDestroy(b.done);
  void* dev[] = {g->frames, g->heads[0], g->heads[1], g->heads[2], g->heads[3], g->heads[4], g->heads[5], g->rows,
                 g->count, g->t_id, g->t_box, g->t_state, g->t_det, g->t_count, g->net_det[0], g->net_det[1],
                 g->net_det[2], g->d_slots};
  for (void* p : dev)
    if (p) cudaFree(p);
  void* host[] = {g->h_slots, g->p_count, g->p_id, g->p_box, g->p_state, g->p_tcount, g->p_det, g->p_rows, g->p_net[0],
                  g->p_net[1], g->p_net[2]};
  for (void* p : host)
    if (p) cudaFreeHost(p);
  if (g->h) jde_destroy(g->h);
  if (g->st) cudaStreamDestroy(g->st);
  delete g;
}

jde_status group_new(jde_server* s, int in_w, int in_h, Group** out) {
  Group* g = new Group();
  g->in_w = in_w;
  g->in_h = in_h;
  jde_config c = group_config(s->cfg, in_w, in_h);
  jde_status st = jde_create(&c, s->weights.data(), s->weights.size(), &g->h);
  if (st != JDE_OK) {
    s->err = std::string("group handle: ") + jde_last_error(nullptr);
    delete g;
    return st;
  }
  const size_t B = (size_t)s->cfg.group.max_batch;
  const int strides[3] = {32, 16, 8};
  bool ok = cudaStreamCreateWithFlags(&g->st, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && galloc((void**)&g->frames, B * s->cfg.src_w * s->cfg.src_h * 3);
  for (int k = 0; k < 3; ++k) {
    const size_t cells = (size_t)(in_w / strides[k]) * (in_h / strides[k]);
    g->head_bytes[k] = cells * 24 * 4;
    g->head_bytes[3 + k] = cells * 512 * 4;
    g->net_bytes[k] = cells * 24 * 4;
  }
  for (int k = 0; k < 6 && s->cfg.caller_heads; ++k) ok = ok && galloc((void**)&g->heads[k], B * g->head_bytes[k]);
  for (int k = 0; k < 3 && s->cfg.collect_net_heads; ++k) {
    ok = ok && galloc((void**)&g->net_det[k], B * g->net_bytes[k]);
    ok = ok && halloc((void**)&g->p_net[k], B * g->net_bytes[k]);
  }
  const size_t dc = (size_t)s->cfg.det_cap, tc = (size_t)s->cfg.track_cap;
  ok = ok && galloc((void**)&g->rows, B * dc * 518 * 4) && galloc((void**)&g->count, B * 4) &&
       galloc((void**)&g->t_id, B * tc * 8) && galloc((void**)&g->t_box, B * tc * 16) &&
       galloc((void**)&g->t_state, B * tc * 4) && galloc((void**)&g->t_det, B * tc * 4) &&
       galloc((void**)&g->t_count, B * 4) && galloc((void**)&g->d_slots, B * sizeof(int));
  ok = ok && halloc((void**)&g->h_slots, B * sizeof(int)) && halloc((void**)&g->p_count, B * 4) &&
       halloc((void**)&g->p_id, B * tc * 8) && halloc((void**)&g->p_box, B * tc * 16) &&
       halloc((void**)&g->p_state, B * tc * 4) && halloc((void**)&g->p_tcount, B * 4) &&
       halloc((void**)&g->p_det, B * tc * 4) &&
       halloc((void**)&g->p_rows, B * dc * 518 * 4);
  if (!ok) {
    group_free(g);
    return sfail(s, JDE_ERR_OOM, "group buffers for %dx%d", in_w, in_h);
  }
  for (int k = s->cfg.max_streams_per_group - 1; k >= 0; --k) g->free_slots.push_back(k);
  *out = g;
  return JDE_OK;
}

// The launch sequence of a batch of n frames on the group's stream (capturable: no allocation once warm,
// no synchronisation): forward, the network's detection maps (when collected), post-processing, tracker.
jde_status batch_sequence(jde_server* s, Group* g, int n, const std::vector<int>& ids) {
  jde_status st = jde_forward(g->h, g->frames, n, s->cfg.src_w, s->cfg.src_h, g->in_w, g->in_h, 1, g->st);
  if (st != JDE_OK) return sfail(s, st, "forward: %s", jde_last_error(g->h));
  if (s->cfg.collect_net_heads)
    for (int k = 0; k < 3; ++k) {
      st = jde_get_tensor(g->h, s->det_layers[k], g->net_det[k], (size_t)n * g->net_bytes[k], nullptr, nullptr, g->st);
      if (st != JDE_OK) return sfail(s, st, "detection maps: %s", jde_last_error(g->h));
    }
  jde_dets d{g->rows, g->count, nullptr, s->cfg.det_cap, 1};
  const float* hp[6];
  for (int k = 0; k < 6; ++k) hp[k] = g->heads[k];
  st = jde_postprocess(g->h, s->cfg.caller_heads ? hp : nullptr, n, g->in_w, g->in_h, s->cfg.src_w, s->cfg.src_h, &d,
                       g->st);
  if (st != JDE_OK) return sfail(s, st, "post-processing: %s", jde_last_error(g->h));
  jde_tracks t{g->t_id, g->t_box, g->t_state, g->t_det, g->t_count, s->cfg.track_cap, 1};
  st = track_step_device_slots(g->h, n, ids.data(), g->d_slots, &d, &t, g->st);
  if (st != JDE_OK) return sfail(s, st, "tracker: %s", jde_last_error(g->h));
  return JDE_OK;
}

// The CUDA graph of the group's batch of n frames, captured from batch_sequence if it is not there yet.
jde_status ensure_graph(jde_server* s, Group* g, int n, const std::vector<int>& ids) {
  if (g->graphs.count(n)) return JDE_OK;
  cudaGraph_t graph = nullptr;
  S_CUDA(s, cudaStreamBeginCapture(g->st, cudaStreamCaptureModeThreadLocal));
  jde_status st = batch_sequence(s, g, n, ids);
  const cudaError_t ce = cudaStreamEndCapture(g->st, &graph);
  if (st != JDE_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (ce != cudaSuccess) return sfail(s, JDE_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ce));
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) return sfail(s, JDE_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ie));
  g->graphs[n] = exec;
  s->captured += 1;
  return JDE_OK;
}

// A new group runs every batch size it can see once (1 .. min(max_batch, tracker slots)) on zeroed
// inputs, with slots 0 .. n-1, and captures its graph, so no plan, scratch allocation or capture
// happens while streams are served; then it clears the error word and resets the slots it used.
jde_status prewarm_group(jde_server* s, Group* g) {
  const int B = s->cfg.group.max_batch < s->cfg.max_streams_per_group ? s->cfg.group.max_batch
                                                                        : s->cfg.max_streams_per_group;
  const size_t fbytes = (size_t)s->cfg.src_w * s->cfg.src_h * 3;
  S_CUDA(s, cudaMemsetAsync(g->frames, 0, (size_t)B * fbytes, g->st));
  for (int k = 0; k < 6 && s->cfg.caller_heads; ++k)
    S_CUDA(s, cudaMemsetAsync(g->heads[k], 0, (size_t)B * g->head_bytes[k], g->st));
  for (int n = 1; n <= B; ++n) {
    std::vector<int> ids(n);
    for (int i = 0; i < n; ++i) ids[i] = g->h_slots[i] = i;
    S_CUDA(s, cudaMemcpyAsync(g->d_slots, g->h_slots, sizeof(int) * n, cudaMemcpyHostToDevice, g->st));
    jde_status st = batch_sequence(s, g, n, ids);
    if (st != JDE_OK) return st;
    g->warmed[n] += 1;
    if (s->cfg.use_graphs) {
      st = ensure_graph(s, g, n, ids);
      if (st != JDE_OK) return st;
    }
    S_CUDA(s, cudaStreamSynchronize(g->st));   // the pinned slot array is rewritten for the next n
  }
  int word = 0;
  jde_status st = jde_kernel_errors(g->h, &word, g->st);
  if (st != JDE_OK) return sfail(s, st, "error word: %s", jde_last_error(g->h));
  for (int i = 0; i < B; ++i) {
    st = jde_stream_reset(g->h, i, g->st);
    if (st != JDE_OK) return sfail(s, st, "reset: %s", jde_last_error(g->h));
  }
  S_CUDA(s, cudaStreamSynchronize(g->st));
  return JDE_OK;
}

// Frames whose batch could not be launched or did not complete: their results are returned with
// errors = -1 (nothing else filled in), so every submitted frame gets exactly one result.
void fail_frames(jde_server* s, const std::vector<Pending>& frames) {
  for (const Pending& p : frames) {
    jde_frame_result r;
    memset(&r, 0, sizeof(r));
    r.ticket = p.ticket;
    r.stream_id = p.stream_id;
    r.errors = -1;
    s->ready.push_back(r);
    auto it = s->streams.find(p.stream_id);
    if (it != s->streams.end()) it->second.inflight -= 1;
  }
}

jde_status launch_frames(jde_server* s, Group* g, Batch& b);

jde_status launch_batch(jde_server* s, Group* g) {
  Batch b;
  std::deque<Pending> rest;
  std::vector<int> seen;
  while (!g->queue.empty()) {
    Pending p = g->queue.front();
    g->queue.pop_front();
    bool dup = false;
    for (int id : seen) dup = dup || id == p.stream_id;
    if (dup || (int)b.frames.size() >= s->cfg.group.max_batch) {
      rest.push_back(p);
    } else {
      seen.push_back(p.stream_id);
      b.frames.push_back(p);
    }
  }
  g->queue.swap(rest);
  b.n = (int)b.frames.size();
  const jde_status st = launch_frames(s, g, b);
  if (st != JDE_OK) {
    if (b.done) cudaEventDestroy(b.done);
    fail_frames(s, b.frames);
  }
  return st;
}

// Copies, launch sequence (graph or eager) and output copies of batch b; on success the batch is in
// flight with its done event.
jde_status launch_frames(jde_server* s, Group* g, Batch& b) {
  const int n = b.n;
  const size_t fbytes = (size_t)s->cfg.src_w * s->cfg.src_h * 3;
  std::vector<int> ids(n);
  for (int i = 0; i < n; ++i) {
    const Pending& p = b.frames[i];
    ids[i] = s->streams[p.stream_id].slot;
    g->h_slots[i] = ids[i];
    if (p.ready) S_CUDA(s, cudaStreamWaitEvent(g->st, p.ready, 0));
    S_CUDA(s, cudaMemcpyAsync(g->frames + (size_t)i * fbytes, p.frame, fbytes, cudaMemcpyDeviceToDevice, g->st));
    for (int k = 0; k < 6 && s->cfg.caller_heads; ++k)
      S_CUDA(s, cudaMemcpyAsync(reinterpret_cast<char*>(g->heads[k]) + (size_t)i * g->head_bytes[k], p.heads[k],
                                g->head_bytes[k], cudaMemcpyDeviceToDevice, g->st));
  }
  S_CUDA(s, cudaMemcpyAsync(g->d_slots, g->h_slots, sizeof(int) * n, cudaMemcpyHostToDevice, g->st));
  if (s->cfg.use_graphs && g->warmed[n] >= 1) {
    jde_status st = ensure_graph(s, g, n, ids);
    if (st != JDE_OK) return st;
    S_CUDA(s, cudaGraphLaunch(g->graphs[n], g->st));
    s->replays += 1;
  } else {
    jde_status st = batch_sequence(s, g, n, ids);
    if (st != JDE_OK) return st;
    g->warmed[n] += 1;
    s->eager += 1;
  }
  // outputs of the batch to pinned host memory
  const size_t dc = (size_t)s->cfg.det_cap, tc = (size_t)s->cfg.track_cap;
  S_CUDA(s, cudaMemcpyAsync(g->p_count, g->count, 4 * n, cudaMemcpyDeviceToHost, g->st));
  S_CUDA(s, cudaMemcpyAsync(g->p_tcount, g->t_count, 4 * n, cudaMemcpyDeviceToHost, g->st));
  S_CUDA(s, cudaMemcpyAsync(g->p_id, g->t_id, 8 * tc * n, cudaMemcpyDeviceToHost, g->st));
  S_CUDA(s, cudaMemcpyAsync(g->p_box, g->t_box, 16 * tc * n, cudaMemcpyDeviceToHost, g->st));
  S_CUDA(s, cudaMemcpyAsync(g->p_state, g->t_state, 4 * tc * n, cudaMemcpyDeviceToHost, g->st));
  S_CUDA(s, cudaMemcpyAsync(g->p_det, g->t_det, 4 * tc * n, cudaMemcpyDeviceToHost, g->st));
  bool want_rows = false, want_net = false;
  for (const Pending& p : b.frames) {
    want_rows = want_rows || p.out.rows;
    want_net = want_net || p.out.net_det[0];
  }
  if (want_rows) S_CUDA(s, cudaMemcpyAsync(g->p_rows, g->rows, 518 * 4 * dc * n, cudaMemcpyDeviceToHost, g->st));
  if (want_net && s->cfg.collect_net_heads)
    for (int k = 0; k < 3; ++k)
      S_CUDA(s, cudaMemcpyAsync(g->p_net[k], g->net_det[k], g->net_bytes[k] * n, cudaMemcpyDeviceToHost, g->st));
  S_CUDA(s, cudaEventCreateWithFlags(&b.done, cudaEventDefault));
  S_CUDA(s, cudaEventRecord(b.done, g->st));
  g->inflight.push_back(b);
  b.done = nullptr;   // owned by the in-flight copy
  return JDE_OK;
}

// A finished batch: results into the ready list, outputs into the callers' host buffers.
void collect_batch(jde_server* s, Group* g, Batch& b, int errors) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, s->start, b.done);
  const int dc = s->cfg.det_cap, tc = s->cfg.track_cap;
  for (int i = 0; i < b.n; ++i) {
    const Pending& p = b.frames[i];
    jde_frame_result r;
    r.ticket = p.ticket;
    r.stream_id = p.stream_id;
    r.n_dets = g->p_count[i];
    r.n_tracks = g->p_tcount[i];
    r.errors = errors;
    r.done_ms = ms;
    const int nt = r.n_tracks < tc ? r.n_tracks : tc;
    const int nd = r.n_dets < dc ? r.n_dets : dc;
    if (p.out.track_id) memcpy(p.out.track_id, g->p_id + (size_t)i * tc, 8 * (size_t)nt);
    if (p.out.track_box) memcpy(p.out.track_box, g->p_box + (size_t)i * tc * 4, 16 * (size_t)nt);
    if (p.out.track_state) memcpy(p.out.track_state, g->p_state + (size_t)i * tc, 4 * (size_t)nt);
    if (p.out.track_det) memcpy(p.out.track_det, g->p_det + (size_t)i * tc, 4 * (size_t)nt);
    if (p.out.rows) memcpy(p.out.rows, g->p_rows + (size_t)i * dc * 518, 518 * 4 * (size_t)nd);
    for (int k = 0; k < 3; ++k)
      if (p.out.net_det[k] && s->cfg.collect_net_heads)
        memcpy(p.out.net_det[k], reinterpret_cast<char*>(g->p_net[k]) + (size_t)i * g->net_bytes[k], g->net_bytes[k]);
    s->ready.push_back(r);
    auto it = s->streams.find(p.stream_id);
    if (it != s->streams.end()) it->second.inflight -= 1;
  }
  cudaEventDestroy(b.done);
  b.done = nullptr;
}

jde_status poll_groups(jde_server* s) {
  for (auto& kv : s->groups) {
    Group* g = kv.second;
    while (!g->inflight.empty()) {
      const cudaError_t q = cudaEventQuery(g->inflight.front().done);
      if (q == cudaErrorNotReady) break;
      if (q != cudaSuccess) {
        Batch& bad = g->inflight.front();
        fail_frames(s, bad.frames);
        cudaEventDestroy(bad.done);
        g->inflight.pop_front();
        return sfail(s, JDE_ERR_CUDA, "batch: %s", cudaGetErrorString(q));
      }
      // the batch is done, so reading the handle's error word waits for nothing
      int word = 0;
      jde_status st = jde_kernel_errors(g->h, &word, g->st);
      if (st != JDE_OK) return sfail(s, st, "error word: %s", jde_last_error(g->h));
      collect_batch(s, g, g->inflight.front(), word);
      g->inflight.pop_front();
    }
    if (g->inflight.empty() && !g->queue.empty()) {
      jde_status st = launch_batch(s, g);
      if (st != JDE_OK) return st;
    }
  }
  return JDE_OK;
}

}  // namespace

extern "C" {

void jde_default_server_config(jde_server_config* c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  jde_default_config(&c->group);
  c->src_w = 1920;
  c->src_h = 1080;
  c->max_streams_per_group = 16;
  c->hbm_budget_bytes = (size_t)64 << 30;
  c->det_cap = 256;
  c->track_cap = 256;
  c->caller_heads = 0;
  c->collect_net_heads = 0;
  c->use_graphs = 1;
  c->prewarm = 1;
}

jde_status jde_server_create(const jde_server_config* cfg, const void* weights, size_t nbytes, jde_server** out) {
  if (!out || !cfg || !weights) return JDE_ERR_INVALID_ARG;
  *out = nullptr;
  const jde_server_config& c = *cfg;
  if (!server_config_ok(c) || nbytes == 0) return JDE_ERR_INVALID_ARG;
  jde_server* s = new jde_server();
  s->cfg = c;
  s->weights.assign(static_cast<const uint8_t*>(weights), static_cast<const uint8_t*>(weights) + nbytes);
  jde_layer_desc L[JDE_NUM_LAYERS];
  jde_layer_table(L, JDE_NUM_LAYERS);
  for (int l = 0; l < JDE_NUM_LAYERS; ++l)
    if (L[l].cout == 24) s->det_layers.push_back(l);
  if (cudaSetDevice(c.group.device) != cudaSuccess || cudaEventCreate(&s->start) != cudaSuccess ||
      cudaEventRecord(s->start, 0) != cudaSuccess) {
    delete s;
    return JDE_ERR_CUDA;
  }
  *out = s;
  return JDE_OK;
}

void jde_server_destroy(jde_server* s) {
  if (!s) return;
  cudaSetDevice(s->cfg.group.device);
  for (auto& kv : s->groups) group_free(kv.second);
  if (s->start) cudaEventDestroy(s->start);
  delete s;
}

const char* jde_server_last_error(jde_server* s) { return s ? s->err.c_str() : ""; }

jde_status jde_server_reset_clock(jde_server* s) {
  if (!s) return JDE_ERR_INVALID_ARG;
  cudaSetDevice(s->cfg.group.device);
  S_CUDA(s, cudaEventRecord(s->start, 0));
  S_CUDA(s, cudaEventSynchronize(s->start));
  return JDE_OK;
}

jde_status jde_stream_open(jde_server* s, int in_w, int in_h, int* stream_id) {
  if (!s || !stream_id) return JDE_ERR_INVALID_ARG;
  *stream_id = -1;
  if (in_w < 32 || in_h < 32 || in_w % 32 || in_h % 32) return sfail(s, JDE_ERR_INVALID_ARG, "input size %dx%d", in_w, in_h);
  cudaSetDevice(s->cfg.group.device);
  const auto key = std::make_pair(in_w, in_h);
  auto it = s->groups.find(key);
  Group* g = it == s->groups.end() ? nullptr : it->second;
  if (!g) {
    size_t cost = 0;
    jde_status st = jde_server_group_cost(&s->cfg, in_w, in_h, &cost);
    if (st != JDE_OK) return sfail(s, st, "estimate: %s", jde_last_error(nullptr));
    if (s->used + cost > s->cfg.hbm_budget_bytes)
      return sfail(s, JDE_ERR_ADMISSION, "a %dx%d group needs %zu bytes, %zu of %zu left", in_w, in_h, cost,
                   s->cfg.hbm_budget_bytes - s->used, s->cfg.hbm_budget_bytes);
    st = group_new(s, in_w, in_h, &g);
    if (st != JDE_OK) return st;
    if (s->cfg.prewarm) {
      st = prewarm_group(s, g);
      if (st != JDE_OK) {
        group_free(g);
        return st;
      }
    }
    g->charged = cost;
    s->used += cost;
    s->groups[key] = g;
  }
  if (g->free_slots.empty()) return sfail(s, JDE_ERR_ADMISSION, "the %dx%d group has no free tracker slot", in_w, in_h);
  const int slot = g->free_slots.back();
  g->free_slots.pop_back();
  jde_status st = jde_stream_reset(g->h, slot, g->st);
  if (st != JDE_OK) return sfail(s, st, "reset: %s", jde_last_error(g->h));
  const int id = s->next_stream++;
  StreamRec r;
  r.g = g;
  r.slot = slot;
  s->streams[id] = r;
  *stream_id = id;
  return JDE_OK;
}

jde_status jde_stream_close(jde_server* s, int stream_id) {
  if (!s) return JDE_ERR_INVALID_ARG;
  auto it = s->streams.find(stream_id);
  if (it == s->streams.end()) return sfail(s, JDE_ERR_NOT_FOUND, "stream %d", stream_id);
  cudaSetDevice(s->cfg.group.device);
  // its queued and in-flight frames finish first
  while (it->second.inflight > 0) {
    jde_status st = poll_groups(s);
    if (st != JDE_OK) return st;
    S_CUDA(s, cudaStreamSynchronize(it->second.g->st));
  }
  Group* g = it->second.g;
  g->free_slots.push_back(it->second.slot);
  s->streams.erase(it);
  bool empty = true;
  for (auto& kv : s->streams) empty = empty && kv.second.g != g;
  if (empty) {
    s->used -= g->charged;
    s->groups.erase(std::make_pair(g->in_w, g->in_h));
    group_free(g);
  }
  return JDE_OK;
}

jde_status jde_submit(jde_server* s, int stream_id, const uint8_t* frame, const float* const* heads, void* ready_event,
                      const jde_frame_out* out, long long* ticket) {
  if (!s || !frame) return JDE_ERR_INVALID_ARG;
  auto it = s->streams.find(stream_id);
  if (it == s->streams.end()) return sfail(s, JDE_ERR_NOT_FOUND, "stream %d", stream_id);
  if (s->cfg.caller_heads && !heads) return sfail(s, JDE_ERR_INVALID_ARG, "this server takes per-frame heads");
  Pending p;
  memset(&p, 0, sizeof(p));
  p.ticket = s->next_ticket++;
  p.stream_id = stream_id;
  p.frame = frame;
  p.ready = static_cast<cudaEvent_t>(ready_event);
  for (int k = 0; k < 6 && s->cfg.caller_heads; ++k) {
    if (!heads[k]) return sfail(s, JDE_ERR_INVALID_ARG, "head %d is NULL", k);
    p.heads[k] = heads[k];
  }
  if (out) p.out = *out;
  it->second.g->queue.push_back(p);
  it->second.inflight += 1;
  if (ticket) *ticket = p.ticket;
  return JDE_OK;
}

jde_status jde_poll(jde_server* s, jde_frame_result* results, int cap, int* n) {
  if (!s || !n || (cap > 0 && !results)) return JDE_ERR_INVALID_ARG;
  *n = 0;
  cudaSetDevice(s->cfg.group.device);
  jde_status st = poll_groups(s);
  while (*n < cap && !s->ready.empty()) {
    results[(*n)++] = s->ready.front();
    s->ready.pop_front();
  }
  return st;
}

jde_status jde_server_group_cost(const jde_server_config* cfg, int in_w, int in_h, size_t* out) {
  if (!cfg || !out || !server_config_ok(*cfg)) return JDE_ERR_INVALID_ARG;
  jde_config c = group_config(*cfg, in_w, in_h);
  size_t est = 0;
  jde_status st = jde_estimate_device_bytes(&c, in_w, in_h, &est);
  if (st != JDE_OK) return st;
  *out = est + group_buffer_bytes(*cfg, in_w, in_h);
  return JDE_OK;
}

jde_status jde_server_flush(jde_server* s) {
  if (!s) return JDE_ERR_INVALID_ARG;
  cudaSetDevice(s->cfg.group.device);
  for (;;) {
    jde_status st = poll_groups(s);
    if (st != JDE_OK) return st;
    bool busy = false;
    for (auto& kv : s->groups) {
      busy = busy || !kv.second->inflight.empty() || !kv.second->queue.empty();
      if (!kv.second->inflight.empty()) S_CUDA(s, cudaStreamSynchronize(kv.second->st));
    }
    if (!busy) return JDE_OK;
  }
}

jde_status jde_server_stats(jde_server* s, long long* eager, long long* captured, long long* replays) {
  if (!s) return JDE_ERR_INVALID_ARG;
  if (eager) *eager = s->eager;
  if (captured) *captured = s->captured;
  if (replays) *replays = s->replays;
  return JDE_OK;
}

jde_status jde_server_device_bytes(jde_server* s, size_t* charged, size_t* held) {
  if (!s) return JDE_ERR_INVALID_ARG;
  if (charged) *charged = s->used;
  if (held) {
    size_t b = 0;
    for (auto& kv : s->groups) {
      size_t hb = 0;
      jde_device_bytes(kv.second->h, &hb);
      b += hb + group_buffer_bytes(s->cfg, kv.second->in_w, kv.second->in_h);
    }
    *held = b;
  }
  return JDE_OK;
}

}  // extern "C"
