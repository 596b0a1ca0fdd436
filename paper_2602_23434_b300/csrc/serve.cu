// serve.cu -- host side of the serving entry points (include/part.h).
//
// A server holds a table of resident snapshots (padded f32 fields + geometry
// of PART_MIXED contexts) and a work list in its device workspace.  Each
// round copies the work list from the caller's pinned staging buffer and
// runs the persistent kernel; both are captured once into a CUDA graph and
// replayed.  Items are validated on the host before every round, so the
// kernel never sees an out-of-range request slice.
#include <cmath>
#include <cstring>
#include <new>

#include "part_internal.cuh"

static_assert(sizeof(part_work_item) == 72, "part_work_item layout is part of the ABI");

struct part_server {
  part_ctx* snaps[64];
  int nsnap;
  int max_items;
  int shape, dim;
  cudaStream_t stream;
  char* ws;
  ServeHeader* d_hdr;
  part_work_item* d_items;
  SnapEntry* d_snaps;
  int* d_status;
  char* h_stage;
  size_t stage_bytes;
  int grid, threads;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  bool captured;
  std::string err;
};

namespace {

constexpr int kMaxSnaps = 64;
size_t up256(size_t v) { return (v + 255) / 256 * 256; }

struct SrvLayout {
  size_t hdr, items, snaps, status, total, stage;
};

SrvLayout srv_layout(int nsnap, int max_items) {
  SrvLayout L;
  L.hdr = 0;
  L.items = sizeof(ServeHeader);                                   // 256 bytes
  L.snaps = up256(L.items + (size_t)max_items * sizeof(part_work_item));
  L.status = up256(L.snaps + (size_t)nsnap * sizeof(SnapEntry));
  L.total = L.status + 256;
  L.stage = L.snaps;  // header + items are staged on the host and copied as one block
  return L;
}

part_status sfail(part_server* s, part_status st, const std::string& m) {
  if (s) s->err = m;
  return fail(nullptr, st, m);
}

}  // namespace

extern "C" {

part_status part_server_sizes(int nsnap, int max_items, size_t* device_bytes,
                              size_t* host_bytes) {
  if (nsnap < 1 || nsnap > kMaxSnaps) return fail(nullptr, PART_EINVAL, "nsnap in [1, 64]");
  if (max_items < 1 || max_items > (1 << 24))
    return fail(nullptr, PART_EINVAL, "max_items in [1, 2^24]");
  SrvLayout L = srv_layout(nsnap, max_items);
  if (device_bytes) *device_bytes = L.total;
  if (host_bytes) *host_bytes = L.stage;
  return PART_OK;
}

part_status part_server_init(part_server** out, part_ctx* const* snapshots, int nsnap,
                             int max_items, void* workspace, size_t ws_bytes, void* host_stage,
                             size_t host_bytes, void* cuda_stream, int threads,
                             int ctas_per_sm) {
  if (!out) return fail(nullptr, PART_EINVAL, "out is NULL");
  *out = nullptr;
  size_t need = 0, hneed = 0;
  part_status st = part_server_sizes(nsnap, max_items, &need, &hneed);
  if (st != PART_OK) return st;
  if (!snapshots || !workspace || !host_stage)
    return fail(nullptr, PART_EINVAL, "snapshots, workspace and host_stage must be given");
  if (((uintptr_t)workspace & 255u) != 0)
    return fail(nullptr, PART_EINVAL, "workspace must be 256-byte aligned");
  if (ws_bytes < need || host_bytes < hneed)
    return fail(nullptr, PART_ENOMEM, "workspace or staging buffer smaller than part_server_sizes()");
  if (threads < 128 || threads > 512 || threads % 32 != 0)
    return fail(nullptr, PART_EINVAL, "threads must be a multiple of 32 in [128, 512]");
  if (ctas_per_sm < 1 || ctas_per_sm > 16)
    return fail(nullptr, PART_EINVAL, "ctas_per_sm in [1, 16]");
  if (cuda_stream == nullptr || cuda_stream == (void*)cudaStreamLegacy ||
      cuda_stream == (void*)cudaStreamPerThread)
    return fail(nullptr, PART_EINVAL,
                "serving needs a created stream: a default stream cannot be captured");
  for (int i = 0; i < nsnap; ++i) {
    const part_ctx* c = snapshots[i];
    if (!c || c->prec != PART_MIXED || c->mode != PART_BORIS || !c->fields_set)
      return fail(nullptr, PART_EINVAL, "snapshots must be PART_MIXED Boris contexts with fields");
    if (c->geo.any_open)
      return fail(nullptr, PART_EUNSUPPORTED, "serving needs periodic snapshots");
    if (c->shape != snapshots[0]->shape || c->geo.dim != snapshots[0]->geo.dim)
      return fail(nullptr, PART_EINVAL, "snapshots must share shape and dim");
  }
  part_server* s = new (std::nothrow) part_server();
  if (!s) return fail(nullptr, PART_ENOMEM, "host allocation of the server failed");
  SrvLayout L = srv_layout(nsnap, max_items);
  for (int i = 0; i < nsnap; ++i) s->snaps[i] = snapshots[i];
  s->nsnap = nsnap;
  s->max_items = max_items;
  s->shape = snapshots[0]->shape;
  s->dim = snapshots[0]->geo.dim;
  s->stream = (cudaStream_t)cuda_stream;
  s->ws = (char*)workspace;
  s->d_hdr = (ServeHeader*)(s->ws + L.hdr);
  s->d_items = (part_work_item*)(s->ws + L.items);
  s->d_snaps = (SnapEntry*)(s->ws + L.snaps);
  s->d_status = (int*)(s->ws + L.status);
  s->h_stage = (char*)host_stage;
  s->stage_bytes = L.stage;
  s->threads = threads;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      nsm < 1) {
    delete s;
    return fail(nullptr, PART_ECUDA, "cudaGetDevice / multiprocessor count query failed");
  }
  s->grid = nsm * ctas_per_sm;
  std::memset(s->h_stage, 0, L.stage);
  SnapEntry tab[kMaxSnaps];
  for (int i = 0; i < nsnap; ++i) {
    tab[i].fp = (const float*)snapshots[i]->fpad;
    tab[i].g = snapshots[i]->geo;
  }
  cudaError_t e = cudaMemcpy(s->d_snaps, tab, sizeof(SnapEntry) * nsnap, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(s->d_status, 0, 256);
  if (e == cudaSuccess) e = cudaMemset(s->d_hdr, 0, sizeof(ServeHeader));
  if (e != cudaSuccess) {
    delete s;
    return fail(nullptr, PART_ECUDA, std::string("part_server_init: ") + cudaGetErrorString(e));
  }
  *out = s;
  return PART_OK;
}

part_work_item* part_server_items(part_server* s) {
  return s ? (part_work_item*)(s->h_stage + sizeof(ServeHeader)) : nullptr;
}

part_status part_server_run(part_server* s, int nitems) {
  if (!s) return fail(nullptr, PART_EINVAL, "server is NULL");
  if (nitems < 0 || nitems > s->max_items)
    return sfail(s, PART_EINVAL, "nitems must be in [0, max_items]");
  const part_work_item* it = part_server_items(s);
  // the chunks of one request share their state arrays: look each array set
  // up once (cudaPointerGetAttributes is a host call per pointer)
  const void *ok_cell = nullptr, *ok_off = nullptr, *ok_u = nullptr;
  for (int i = 0; i < nitems; ++i) {
    const part_work_item& w = it[i];
    if (w.snapshot < 0 || w.snapshot >= s->nsnap)
      return sfail(s, PART_EINVAL, "work item " + std::to_string(i) + ": snapshot out of range");
    if (w.count < 0 || w.nsteps < 0 || w.first < 0 || w.first + w.count > w.stride)
      return sfail(s, PART_EINVAL, "work item " + std::to_string(i) + ": bad slice");
    if (w.count > 0 && (!w.cell || !w.off || !w.u))
      return sfail(s, PART_EINVAL, "work item " + std::to_string(i) + ": NULL state");
    if (w.count > 0 && !(w.cell == ok_cell && w.off == ok_off && w.u == ok_u)) {
      if (((uintptr_t)w.cell | (uintptr_t)w.off | (uintptr_t)w.u) % 4 != 0 ||
          !device_accessible(s->snaps[0]->device, w.cell) ||
          !device_accessible(s->snaps[0]->device, w.off) ||
          !device_accessible(s->snaps[0]->device, w.u))
        return sfail(s, PART_EINVAL,
                     "work item " + std::to_string(i) + ": state not aligned or not reachable");
      ok_cell = w.cell;
      ok_off = w.off;
      ok_u = w.u;
    }
    if (!std::isfinite(w.q_over_m) || !std::isfinite(w.dt) || w.dt == 0.0)
      return sfail(s, PART_EINVAL, "work item " + std::to_string(i) + ": bad q_over_m / dt");
  }
  ((ServeHeader*)s->h_stage)->nitems = nitems;
  ((ServeHeader*)s->h_stage)->next = 0;
  cudaError_t e = cudaSuccess;
  if (!s->captured) {
    e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess)
      return sfail(s, PART_ECUDA, std::string("begin capture: ") + cudaGetErrorString(e));
    e = cudaMemcpyAsync(s->d_hdr, s->h_stage, s->stage_bytes, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
      e = launch_serve_kernel(s->shape, s->dim, s->d_hdr, s->d_items, s->d_snaps, s->nsnap,
                              s->d_status, s->grid, s->threads, s->stream);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(s->stream, &g);  // always close an open capture
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&s->exec, g, 0);
    if (e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return sfail(s, PART_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    s->graph = g;
    s->captured = true;
  }
  e = cudaGraphLaunch(s->exec, s->stream);
  if (e != cudaSuccess)
    return sfail(s, PART_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
  return PART_OK;
}

part_status part_server_sync(part_server* s) {
  if (!s) return fail(nullptr, PART_EINVAL, "server is NULL");
  int st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, s->d_status, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess)
    return sfail(s, PART_ECUDA, std::string("part_server_sync: ") + cudaGetErrorString(e));
  if (st == 0) return PART_OK;
  e = cudaMemsetAsync(s->d_status, 0, sizeof(int), s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (st & ST_NONFINITE) return sfail(s, PART_ENONFINITE, "non-finite particle state");
  return sfail(s, PART_EDOMAIN, "a particle cell or item snapshot was out of range");
}

part_status part_server_destroy(part_server* s) {
  if (!s) return fail(nullptr, PART_EINVAL, "server is NULL");
  if (s->captured) {
    cudaGraphExecDestroy(s->exec);
    cudaGraphDestroy(s->graph);
  }
  delete s;
  return PART_OK;
}

}  // extern "C"
