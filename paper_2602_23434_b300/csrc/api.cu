// api.cu -- host side of the C ABI declared in include/part.h.
//
// Validates arguments before any launch, carves the caller's workspace,
// encodes the TMA tensor map of the padded field copy, and dispatches the
// kernels on the context's stream.  Allocates no device memory.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include <cudaTypedefs.h>

#include "part_internal.cuh"

cudaError_t launch_lp_sample_rho(part_ctx* c);

namespace {
thread_local std::string g_err = "";
}  // namespace

part_status fail(part_ctx* c, part_status s, const std::string& msg) {
  if (c) c->err = msg;
  g_err = msg;
  return s;
}

// Memory a kernel on `device` may touch: device memory of that device,
// managed memory, or pinned host memory mapped into the unified address space
// at the same address (read or written over the host link).  Pageable host
// memory and other devices' memory are refused: a kernel would fault on them.
// NULL passes (optional arrays).
bool device_accessible(int device, const void* p) {
  if (!p) return true;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // clear the non-sticky error
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  if (a.type == cudaMemoryTypeDevice) return a.device == device;
  if (a.type == cudaMemoryTypeHost) return a.devicePointer == p;
  return false;
}

part_status cuda_fail(part_ctx* c, cudaError_t e, const char* where) {
  return fail(c, PART_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

namespace {

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// Element alignment of a caller array (the kernels load whole elements).
bool misaligned(const void* p, size_t elem) {
  return p && (reinterpret_cast<uintptr_t>(p) % elem) != 0;
}

// Element sizes of the particle planes of this context: positions (or cells),
// offsets, u, w.
size_t pos_elem(const part_ctx* c) { return c->prec == PART_MIXED ? 4 : 8; }
size_t real_elem(const part_ctx* c) { return c->prec == PART_MIXED ? 4 : 8; }

}  // namespace

part_status check_access(part_ctx* c, const void* p, const char* what) {
  if (device_accessible(c->device, p)) return PART_OK;
  return fail(c, PART_EINVAL,
              std::string(what) + " is not memory the kernels can reach (device memory of the "
                                  "context's device, managed memory or pinned host memory)");
}

namespace {

part_status check_planes(part_ctx* c, const void* x, const void* off, const void* u,
                         const void* w, const void* id, const void* chi, const void* eng,
                         const void* n_old) {
  if (misaligned(x, pos_elem(c)) || misaligned(off, 4) || misaligned(u, real_elem(c)) ||
      misaligned(w, real_elem(c)) || misaligned(id, 8) || misaligned(chi, 8) ||
      misaligned(eng, 8) || misaligned(n_old, 8))
    return fail(c, PART_EINVAL, "a particle array is not aligned to its element size");
  const void* planes[8] = {x, off, u, w, id, chi, eng, n_old};
  for (const void* q : planes)
    if (check_access(c, q, "a particle array") != PART_OK) return PART_EINVAL;
  return PART_OK;
}

}  // namespace

part_status check_grid(const part_grid* g) {
  if (!g) return fail(nullptr, PART_EINVAL, "grid is NULL");
  if (g->dim != 2 && g->dim != 3) return fail(nullptr, PART_EINVAL, "dim must be 2 or 3");
  for (int a = 0; a < 3; ++a) {
    if (g->n[a] < 1) return fail(nullptr, PART_EINVAL, "n[a] must be >= 1");
    if (!(g->dx[a] > 0.0) || !std::isfinite(g->dx[a]))
      return fail(nullptr, PART_EINVAL, "dx[a] must be finite and > 0");
    if (!std::isfinite(g->xmin[a])) return fail(nullptr, PART_EINVAL, "xmin must be finite");
  }
  if (g->dim == 2 && g->n[2] != 1) return fail(nullptr, PART_EINVAL, "dim 2 needs n[2] == 1");
  int64_t G = (int64_t)g->n[0] * g->n[1] * g->n[2];
  if (G > ((int64_t)1 << 30)) return fail(nullptr, PART_EINVAL, "grid larger than 2^30 cells");
  return PART_OK;
}

void make_geo(const part_grid* gr, int esize, Geo* g) {
  std::memset(g, 0, sizeof(Geo));
  g->dim = gr->dim;
  const int b3[3] = {8, 8, 8}, b2[3] = {16, 16, 1};
  for (int a = 0; a < 3; ++a) {
    g->n[a] = gr->n[a];
    g->b[a] = gr->dim == 3 ? b3[a] : b2[a];
    g->nb[a] = (g->n[a] + g->b[a] - 1) / g->b[a];
    g->h[a] = (a < gr->dim) ? 1 : 0;
    g->e[a] = g->b[a] + 2 * g->h[a];
    g->xmin[a] = gr->xmin[a];
    g->dx[a] = gr->dx[a];
    g->inv_dx[a] = 1.0 / gr->dx[a];
    g->L[a] = (double)gr->n[a] * gr->dx[a];
    g->xmax[a] = gr->xmin[a] + g->L[a];
    g->invn[a] = 1.0f / (float)gr->n[a];
    g->xminf[a] = (float)g->xmin[a];
    g->inv_dxf[a] = (float)g->inv_dx[a];
    g->xmin_cells[a] = (float)(std::fabs(g->xmin[a]) * g->inv_dx[a]);
  }
  // FP64: component planes with the x pitch rounded to 16 bytes.  f32 (mixed
  // form): cells interleave 8 floats (32 bytes), so no x rounding is needed.
  const int q = esize == 4 ? 1 : 16 / esize;
  g->pn[0] = (g->n[0] + 2 * g->h[0] + q - 1) / q * q;
  g->pn[1] = g->n[1] + 2 * g->h[1];
  g->pn[2] = g->n[2] + 2 * g->h[2];
  g->box[0] = (g->b[0] + 2 * g->h[0] + q - 1) / q * q;
  g->box[1] = g->b[1] + 2 * g->h[1];
  g->box[2] = g->b[2] + 2 * g->h[2];
  g->V = g->b[0] * g->b[1] * g->b[2];
  for (int a = 0; a < 3; ++a) {
    g->bshift[a] = 0;
    while ((1 << g->bshift[a]) < g->b[a]) ++g->bshift[a];
  }
  g->vshift = g->bshift[0] + g->bshift[1] + g->bshift[2];
  g->any_open = 0;
  for (int a = 0; a < 3; ++a) {
    g->open[a] = a < gr->dim && !gr->periodic[a] ? 1 : 0;
    g->any_open |= g->open[a];
  }
  g->ev = g->e[0] * g->e[1] * g->e[2];
  g->G = (int64_t)g->n[0] * g->n[1] * g->n[2];
  g->nbricks = (int64_t)g->nb[0] * g->nb[1] * g->nb[2];
  g->nkeys = g->nbricks * g->V;
  g->pplane = (int64_t)g->pn[0] * g->pn[1] * g->pn[2];
}

namespace {

struct Layout {
  size_t fpad, keys0, keys1, vals0, vals1, hist, hsum, cstart, tmp, dpart, samples, status,
      alt_x, alt_off, alt_u, alt_w, alt_id, shock_r, shock_q, shock_list, shock_rs, shock_qs,
      cstart_alt, bcount,
      bsum, bslot, lpcache, fpair, fxq, fxq_bytes, smap, total;
};

int ncomp_of(part_mode m) { return m == PART_BORIS ? 6 : 7; }
int esize_of(part_prec p) { return p == PART_FP64 ? 8 : 4; }
// components stored per cell of the padded copy: the mixed form keeps E, B
// and two zero pads interleaved per cell (one 32-byte record)
int fcomp_of(part_prec p, part_mode m) { return p == PART_MIXED ? 8 : ncomp_of(m); }

Layout layout_of(const Geo& g, part_prec prec, part_mode mode, int64_t cap, int nbins) {
  Layout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  const int64_t c1 = cap > 0 ? cap : 1;
  const int64_t ntiles = (c1 + kSortTile - 1) / kSortTile;
  const int64_t hlen = ntiles * kRadix;
  const int64_t nblk = (hlen + kScanBlock - 1) / kScanBlock;
  L.fpad = take((size_t)fcomp_of(prec, mode) * g.pplane * esize_of(prec));
  L.keys0 = take((size_t)(c1 + 1) * 4);  // +1: compaction scans n + 1 flags
  L.keys1 = take((size_t)(c1 + 1) * 4);  // +1: the exchange scans n + 1 flags per side
  L.vals0 = take((size_t)c1 * 4);
  L.vals1 = take((size_t)c1 * 4);
  L.hist = take((size_t)hlen * 4);
  L.hsum = take((size_t)(nblk + 1) * 4);
  L.cstart = take((size_t)(g.nkeys + 1) * 4);
  size_t tmpb = (size_t)c1 * 8;
  if ((size_t)nbins * 16 > tmpb) tmpb = (size_t)nbins * 16;
  L.tmp = take(tmpb);
  L.dpart = take(mode == PART_BORIS ? (size_t)g.nbricks * 3 * g.ev * 8 : 0);
  L.samples = take(mode == PART_LP_RK2 ? (size_t)4 * c1 * 8 : 0);
  L.status = take(256);
  // alternate particle buffers of the Boris modes (sorted state awaiting the push)
  const bool alt = mode == PART_BORIS;
  const size_t e = esize_of(prec);
  L.alt_x = take(alt ? (size_t)c1 * (prec == PART_FP64 ? 3 * 8 : 4) : 0);
  L.alt_off = take(alt && prec == PART_MIXED ? (size_t)c1 * 12 : 0);
  L.alt_u = take(alt ? (size_t)c1 * (prec == PART_MIXED ? 6 : 3) * e : 0);
  L.alt_w = take(alt ? (size_t)c1 * e : 0);
  L.alt_id = take(alt ? (size_t)c1 * 8 : 0);
  // LP mode: shock cells and the list of LPs shocked by the last push
  const bool lp = mode == PART_LP_RK2;
  L.shock_r = take(lp ? (size_t)g.G * 8 : 0);
  L.shock_q = take(lp ? (size_t)g.G * 8 : 0);
  L.shock_list = take(lp ? (size_t)(c1 + 1) * 4 : 0);
  L.shock_rs = take(lp ? (size_t)c1 * 8 : 0);
  L.shock_qs = take(lp ? (size_t)c1 * 8 : 0);
  L.lpcache = take(lp ? (size_t)6 * c1 * 8 : 0);
  L.fpair = take(lp ? (size_t)16 * g.pplane * 4 : 0);
  // x quadratics of the FP64 fields: the LP gathers and the FP64 Boris
  // kernels (TSC) read the fields through them
  const bool xq = lp || (mode == PART_BORIS && prec == PART_FP64);
  L.fxq_bytes = xq ? (size_t)(lp ? 7 : 6) * 4 * g.pplane * 8 : 0;
  L.fxq = take(L.fxq_bytes);
  L.smap = take(lp ? (size_t)3 * c1 * 8 : 0);
  // Boris modes: second cell_start and the brick counts of the incremental sort
  L.cstart_alt = take(alt ? (size_t)(g.nkeys + 1) * 4 : 0);
  L.bcount = take(alt ? (size_t)(g.nbricks + 1) * 4 : 0);
  L.bsum = take(alt ? (size_t)((g.nbricks + 1 + kScanBlock - 1) / kScanBlock + 1) * 4 : 0);
  L.bslot = take(alt ? (size_t)g.nbricks * 27 * 4 : 0);
  L.total = off;
  return L;
}

part_status check_combo(part_prec prec, part_shape shape, part_mode mode, int64_t cap,
                        int nbins) {
  if (prec != PART_FP64 && prec != PART_MIXED) return fail(nullptr, PART_EINVAL, "bad prec");
  if (shape != PART_CIC && shape != PART_TSC) return fail(nullptr, PART_EINVAL, "bad shape");
  if (mode != PART_BORIS && mode != PART_LP_RK2) return fail(nullptr, PART_EINVAL, "bad mode");
  if (mode == PART_LP_RK2 && prec != PART_FP64)
    return fail(nullptr, PART_EUNSUPPORTED, "LP mode keeps FP64 spectra: use PART_FP64");
  if (cap < 0 || cap > ((int64_t)1 << 31) - 1)
    return fail(nullptr, PART_EINVAL, "capacity must be in [0, 2^31)");
  if (mode == PART_LP_RK2 && (nbins < 1 || nbins > 4096))
    return fail(nullptr, PART_EINVAL, "nbins must be in [1, 4096]");
  return PART_OK;
}

part_status encode_tmap(part_ctx* c) {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e =
      cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess || fn == nullptr || q != cudaDriverEntryPointSuccess)
    return fail(c, PART_ECUDA, "cuTensorMapEncodeTiled entry point unavailable");
  auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  const Geo& g = c->geo;
  const cuuint64_t es = (cuuint64_t)c->esize;
  cuuint64_t dims[4] = {(cuuint64_t)g.pn[0], (cuuint64_t)g.pn[1], (cuuint64_t)g.pn[2],
                        (cuuint64_t)c->ncomp};
  cuuint64_t strides[3] = {(cuuint64_t)g.pn[0] * es, (cuuint64_t)g.pn[0] * g.pn[1] * es,
                           (cuuint64_t)g.pplane * es};
  cuuint32_t box[4] = {(cuuint32_t)g.box[0], (cuuint32_t)g.box[1], (cuuint32_t)g.box[2],
                       (cuuint32_t)c->ncomp};
  if (c->fcomp == 8) {  // cell-interleaved f32: (comp, x, y, z), 32 bytes per cell
    const cuuint64_t cb = 8 * es;
    dims[0] = 8;
    dims[1] = (cuuint64_t)g.pn[0];
    dims[2] = (cuuint64_t)g.pn[1];
    dims[3] = (cuuint64_t)g.pn[2];
    strides[0] = cb;
    strides[1] = cb * g.pn[0];
    strides[2] = cb * g.pn[0] * g.pn[1];
    box[0] = 8;
    box[1] = (cuuint32_t)g.box[0];
    box[2] = (cuuint32_t)g.box[1];
    box[3] = (cuuint32_t)g.box[2];
  }
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = encode(&c->tmap,
                      c->esize == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                    : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                      4, c->fpad, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(c, PART_ECUDA, "cuTensorMapEncodeTiled failed");
  if (c->fcomp == 8 && g.dim == 3) {  // one tile plane per copy (rolling staging)
    box[3] = 1;
    r = encode(&c->tmap_plane, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, c->fpad, dims, strides, box,
               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(c, PART_ECUDA, "cuTensorMapEncodeTiled failed");
  }
  c->tmap_ok = true;
  return PART_OK;
}

}  // namespace

part_status check_ctx(part_ctx* c) {
  if (!c) return fail(nullptr, PART_EINVAL, "ctx is NULL");
  return PART_OK;
}

extern "C" {

part_status part_brick_dims(const part_grid* grid, int brick[3], int64_t* nkeys) {
  part_status s = check_grid(grid);
  if (s != PART_OK) return s;
  Geo g;
  make_geo(grid, 8, &g);
  if (brick)
    for (int a = 0; a < 3; ++a) brick[a] = g.b[a];
  if (nkeys) *nkeys = g.nkeys;
  return PART_OK;
}

part_status part_workspace_size(const part_grid* grid, part_prec prec, part_mode mode,
                                int64_t capacity, int nbins, size_t* bytes) {
  part_status s = check_grid(grid);
  if (s != PART_OK) return s;
  if ((s = check_combo(prec, PART_TSC, mode, capacity, nbins)) != PART_OK) return s;
  if (!bytes) return fail(nullptr, PART_EINVAL, "bytes is NULL");
  Geo g;
  make_geo(grid, esize_of(prec), &g);
  *bytes = layout_of(g, prec, mode, capacity, nbins).total;
  return PART_OK;
}

part_status part_init(part_ctx** out, const part_grid* grid, part_prec prec, part_shape shape,
                      part_mode mode, int64_t capacity, int nbins, void* workspace,
                      size_t ws_bytes, void* cuda_stream) {
  if (!out) return fail(nullptr, PART_EINVAL, "out is NULL");
  *out = nullptr;
  part_status s = check_grid(grid);
  if (s != PART_OK) return s;
  if ((s = check_combo(prec, shape, mode, capacity, nbins)) != PART_OK) return s;
  if (!workspace) return fail(nullptr, PART_EINVAL, "workspace is NULL");
  if (((uintptr_t)workspace & 255u) != 0)
    return fail(nullptr, PART_EINVAL, "workspace must be 256-byte aligned");
  part_ctx* c = new (std::nothrow) part_ctx();
  if (!c) return fail(nullptr, PART_ENOMEM, "host allocation of the context failed");
  c->grid = *grid;
  c->prec = prec;
  c->shape = shape;
  c->mode = mode;
  c->capacity = capacity;
  c->nbins = mode == PART_LP_RK2 ? nbins : 0;
  c->stream = (cudaStream_t)cuda_stream;
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device) !=
          cudaSuccess || c->sms < 1) {
    delete c;
    return fail(nullptr, PART_ECUDA, "cudaGetDevice / multiprocessor count query failed");
  }
  c->ncomp = ncomp_of(mode);
  c->fcomp = fcomp_of(prec, mode);
  c->esize = esize_of(prec);
  make_geo(grid, c->esize, &c->geo);
  Layout L = layout_of(c->geo, prec, mode, capacity, c->nbins);
  if (ws_bytes < L.total) {
    delete c;
    return fail(nullptr, PART_ENOMEM, "workspace smaller than part_workspace_size()");
  }
  c->ws = (char*)workspace;
  c->ws_bytes = ws_bytes;
  c->fpad = c->ws + L.fpad;
  c->keys[0] = (uint32_t*)(c->ws + L.keys0);
  c->keys[1] = (uint32_t*)(c->ws + L.keys1);
  c->vals[0] = (uint32_t*)(c->ws + L.vals0);
  c->vals[1] = (uint32_t*)(c->ws + L.vals1);
  c->hist = (uint32_t*)(c->ws + L.hist);
  c->hsum = (uint32_t*)(c->ws + L.hsum);
  c->cstart = (uint32_t*)(c->ws + L.cstart);
  c->tmp = c->ws + L.tmp;
  c->dpart = mode == PART_BORIS ? (double*)(c->ws + L.dpart) : nullptr;
  c->samples = mode == PART_LP_RK2 ? (double*)(c->ws + L.samples) : nullptr;
  c->status = (int*)(c->ws + L.status);
  if (mode == PART_BORIS) {
    c->alt_x = c->ws + L.alt_x;
    c->alt_off = prec == PART_MIXED ? c->ws + L.alt_off : nullptr;
    c->alt_u = c->ws + L.alt_u;
    c->alt_w = c->ws + L.alt_w;
    c->alt_id = (uint64_t*)(c->ws + L.alt_id);
    c->cstart_alt = (uint32_t*)(c->ws + L.cstart_alt);
    c->bcount = (uint32_t*)(c->ws + L.bcount);
    c->bsum = (uint32_t*)(c->ws + L.bsum);
    c->bslot = (uint32_t*)(c->ws + L.bslot);
  }
  if (mode == PART_LP_RK2) {
    c->shock_r = (double*)(c->ws + L.shock_r);
    c->shock_list = (uint32_t*)(c->ws + L.shock_list);
    c->shock_rs = (double*)(c->ws + L.shock_rs);
    c->shock_q = (double*)(c->ws + L.shock_q);
    c->shock_qs = (double*)(c->ws + L.shock_qs);
    c->lpcache = (double*)(c->ws + L.lpcache);
    c->fpair = (float*)(c->ws + L.fpair);
    c->smap = (double*)(c->ws + L.smap);
  }
  c->fxq = L.fxq_bytes ? (double*)(c->ws + L.fxq) : nullptr;
  cudaError_t e = cudaMemsetAsync(c->status, 0, 256, c->stream);
  if (e != cudaSuccess) {
    part_status r = cuda_fail(nullptr, e, "status reset");
    delete c;
    return r;
  }
  if ((s = encode_tmap(c)) != PART_OK) {
    delete c;
    return s;
  }
  *out = c;
  return PART_OK;
}

part_status part_destroy(part_ctx* c) {
  if (!c) return fail(nullptr, PART_EINVAL, "ctx is NULL");
  delete c;
  return PART_OK;
}

part_status part_set_fields(part_ctx* c, const void* fields, int ncomp, part_prec field_prec) {
  if (check_ctx(c)) return PART_EINVAL;
  if (!fields) return fail(c, PART_EINVAL, "fields is NULL");
  if (ncomp != c->ncomp)
    return fail(c, PART_EINVAL, c->mode == PART_BORIS ? "Boris mode needs ncomp = 6 (E, B)"
                                                      : "LP mode needs ncomp = 7 (v, rho, B)");
  if (field_prec != c->prec) return fail(c, PART_EINVAL, "field_prec must match the context");
  if (misaligned(fields, c->prec == PART_MIXED ? 4 : 8))
    return fail(c, PART_EINVAL, "fields are not aligned to their element size");
  if (check_access(c, fields, "fields") != PART_OK) return PART_EINVAL;
  cudaError_t e = launch_pad_fields(c, fields);
  if (e == cudaSuccess && c->mode == PART_LP_RK2) e = launch_pad_pair_lp(c);
  if (e == cudaSuccess && c->fxq && (c->mode == PART_LP_RK2 || c->shape == PART_TSC))
    e = launch_pad_xq(c);
  if (e == cudaSuccess && c->shk) e = launch_shock_cells(c);
  if (e != cudaSuccess) return cuda_fail(c, e, "part_set_fields");
  c->fields_set = true;
  c->lp_cache_ok = false;  // the fields changed
  return PART_OK;
}

part_status part_bind_particles(part_ctx* c, int64_t n, void* x_or_cell, void* off, void* u,
                                void* w, uint64_t* id, double* chi, double* eng,
                                double* n_old) {
  if (check_ctx(c)) return PART_EINVAL;
  if (n < 0 || n > c->capacity) return fail(c, PART_EINVAL, "n must be in [0, capacity]");
  // the previous arrays get their current state first (Boris: the sorted
  // copy; LP: the spectra as (chi, eps))
  if (c->cur_alt || c->perm_pend || c->spec_inv || c->maps_pending) {
    cudaError_t e = flush_pending(c);
    if (e != cudaSuccess) return cuda_fail(c, e, "part_bind_particles");
  }
  if (n > 0 && !x_or_cell) return fail(c, PART_EINVAL, "positions are NULL");
  if (check_planes(c, x_or_cell, off, u, w, id, chi, eng, n_old)) return PART_EINVAL;
  if (c->mode == PART_BORIS) {
    if (n > 0 && !u) return fail(c, PART_EINVAL, "u is NULL");
    if (c->prec == PART_MIXED && n > 0 && !off)
      return fail(c, PART_EINVAL, "mixed form needs the f32 offsets");
  } else {
    if (n > 0 && (!chi || !eng || !n_old))
      return fail(c, PART_EINVAL, "LP mode needs chi, eng and n_old");
  }
  c->n = n;
  c->x = x_or_cell;
  c->off = c->prec == PART_MIXED ? off : nullptr;
  c->u = c->mode == PART_BORIS ? u : nullptr;
  c->w = c->mode == PART_BORIS ? w : nullptr;
  c->id = id;
  c->chi = c->mode == PART_LP_RK2 ? chi : nullptr;
  c->eng = c->mode == PART_LP_RK2 ? eng : nullptr;
  c->n_old = c->mode == PART_LP_RK2 ? n_old : nullptr;
  c->shk = nullptr;  // shock flags belong to the previous particle set
  c->outmask = nullptr;
  c->shock_listed = false;
  c->order_kept = false;
  c->lp_cache_ok = false;
  c->bound = true;
  c->sorted = false;
  c->deposit_ready = false;
  c->samples_ready = false;
  return PART_OK;
}

part_status part_sort(part_ctx* c) {
  if (check_ctx(c)) return PART_EINVAL;
  if (!c->bound) return fail(c, PART_EINVAL, "no particles bound");
  cudaError_t e = cudaSuccess;
  // every particle moved by less than one cell since the last sort: the
  // per-brick incremental sort gives the same permutation at a fraction of
  // the radix passes
  double dxmin = c->geo.dx[0];
  for (int a = 1; a < c->geo.dim; ++a) dxmin = std::min(dxmin, c->geo.dx[a]);
  const bool inc = c->order_kept && c->cstart_alt && c->moved < dxmin && !c->geo.any_open;
  // the deferred LP spectra: each LP's map applied before the LPs move
  if (c->maps_pending) e = launch_spec_to_plain(c);
  if (e == cudaSuccess) e = inc ? launch_sort_incremental(c) : launch_sort(c);
  if (e != cudaSuccess) return cuda_fail(c, e, "part_sort");
  c->sorted = true;
  c->order_kept = true;
  c->moved = 0.0;
  c->samples_ready = false;  // LP samples are in the old particle order
  c->lp_cache_ok = false;
  c->shock_listed = false;
  return PART_OK;
}

part_status part_compact(part_ctx* c, const uint8_t* deleted, int64_t* n_new) {
  if (check_ctx(c)) return PART_EINVAL;
  if (!c->bound) return fail(c, PART_EINVAL, "no particles bound");
  if (!n_new) return fail(c, PART_EINVAL, "n_new is NULL");
  if (c->n > 0 && !deleted) return fail(c, PART_EINVAL, "deleted mask is NULL");
  if (check_access(c, deleted, "deleted") != PART_OK) return PART_EINVAL;
  cudaError_t e = flush_pending(c);
  int64_t nn = c->n;
  if (e == cudaSuccess) e = launch_compact(c, deleted, &nn);
  if (e != cudaSuccess) return cuda_fail(c, e, "part_compact");
  c->n = nn;
  *n_new = nn;
  c->sorted = false;
  c->order_kept = false;
  c->lp_cache_ok = false;
  c->deposit_ready = false;
  c->samples_ready = false;
  c->shock_listed = false;
  return PART_OK;
}

part_status part_inject(part_ctx* c, int64_t k, const void* x_or_cell, const void* off,
                        const void* u, const void* w, const uint64_t* id, const double* chi,
                        const double* eng, const double* n_old) {
  if (check_ctx(c)) return PART_EINVAL;
  if (!c->bound) return fail(c, PART_EINVAL, "no particles bound");
  if (k < 0 || k > c->capacity - c->n)
    return fail(c, PART_EINVAL, "k must be in [0, capacity - n]");
  if (k > 0) {
    if (!x_or_cell) return fail(c, PART_EINVAL, "new positions are NULL");
    if (c->mode == PART_BORIS && !u) return fail(c, PART_EINVAL, "new u is NULL");
    if (c->prec == PART_MIXED && !off) return fail(c, PART_EINVAL, "new offsets are NULL");
    if (c->mode == PART_LP_RK2 && (!chi || !eng || !n_old))
      return fail(c, PART_EINVAL, "LP mode needs the new chi, eng and n_old");
    if (c->w && !w) return fail(c, PART_EINVAL, "w is bound: the new w are needed");
    if (c->id && !id) return fail(c, PART_EINVAL, "id is bound: the new ids are needed");
    if (check_planes(c, x_or_cell, off, u, w, id, chi, eng, n_old)) return PART_EINVAL;
  }
  cudaError_t e = flush_pending(c);
  const InjectSrc src{x_or_cell, off, u, w, id, chi, eng, n_old};
  if (e == cudaSuccess) e = launch_inject(c, k, src);
  if (e != cudaSuccess) return cuda_fail(c, e, "part_inject");
  if (k == 0) return PART_OK;
  c->n += k;
  c->sorted = false;
  c->order_kept = false;
  c->lp_cache_ok = false;
  c->deposit_ready = false;
  c->samples_ready = false;
  c->shock_listed = false;
  return PART_OK;
}

part_status part_set_outflow(part_ctx* c, uint8_t* mask) {
  if (check_ctx(c)) return PART_EINVAL;
  if (mask && !c->geo.any_open) return fail(c, PART_EINVAL, "the grid has no open axis");
  if (check_access(c, mask, "mask") != PART_OK) return PART_EINVAL;
  c->outmask = mask;
  return PART_OK;
}

part_status part_flush(part_ctx* c) {
  if (check_ctx(c)) return PART_EINVAL;
  cudaError_t e = flush_pending(c);
  if (e != cudaSuccess) return cuda_fail(c, e, "part_flush");
  return PART_OK;
}

part_status part_set_lp_order(part_ctx* c, int order) {
  if (check_ctx(c)) return PART_EINVAL;
  if (c->mode != PART_LP_RK2) return fail(c, PART_EINVAL, "the RK order is an LP-mode setting");
  if (order != 2 && order != 3) return fail(c, PART_EINVAL, "order must be 2 or 3");
  c->lp_order = order;
  return PART_OK;
}

part_status part_set_spec_lazy(part_ctx* c, int lazy) {
  if (check_ctx(c)) return PART_EINVAL;
  if (c->mode != PART_LP_RK2) return fail(c, PART_EINVAL, "the spectra are an LP-mode setting");
  if (lazy != 0 && lazy != 1) return fail(c, PART_EINVAL, "lazy must be 0 or 1");
  if (lazy != c->spec_lazy) {  // the bound spectra as (chi, eps) first
    cudaError_t e = launch_spec_to_plain(c);
    if (e != cudaSuccess) return cuda_fail(c, e, "part_set_spec_lazy");
  }
  c->spec_lazy = lazy;
  return PART_OK;
}

part_status part_set_lp_arith(part_ctx* c, int paired) {
  if (check_ctx(c)) return PART_EINVAL;
  if (c->mode != PART_LP_RK2) return fail(c, PART_EINVAL, "the LP arithmetic is an LP-mode setting");
  if (paired != 0 && paired != 1) return fail(c, PART_EINVAL, "paired must be 0 or 1");
  if (paired != c->lp_paired) c->lp_cache_ok = false;  // the cache is kept in the push's format
  c->lp_paired = paired;
  return PART_OK;
}

part_status part_enable_shocks(part_ctx* c, double r_min, uint8_t* state) {
  if (check_ctx(c)) return PART_EINVAL;
  if (c->mode != PART_LP_RK2) return fail(c, PART_EINVAL, "shocks need LP mode");
  if (!state) {
    c->shk = nullptr;
    c->shock_listed = false;
    return PART_OK;
  }
  if (!(std::isfinite(r_min) && r_min > 1.0)) return fail(c, PART_EINVAL, "r_min must be > 1");
  if (check_access(c, state, "state") != PART_OK) return PART_EINVAL;
  if (!c->bound) return fail(c, PART_EINVAL, "bind the particles first");
  if (!c->fields_set) return fail(c, PART_EINVAL, "part_set_fields first");
  c->shk = state;
  c->r_min = r_min;
  c->shock_listed = false;
  cudaError_t e = launch_shock_cells(c);
  if (e != cudaSuccess) return cuda_fail(c, e, "part_enable_shocks");
  return PART_OK;
}

part_status part_set_shock_slope(part_ctx* c, int relativistic) {
  if (check_ctx(c)) return PART_EINVAL;
  if (c->mode != PART_LP_RK2) return fail(c, PART_EINVAL, "shocks need LP mode");
  if (relativistic != 0 && relativistic != 1)
    return fail(c, PART_EINVAL, "relativistic must be 0 or 1");
  c->shock_rel = relativistic;
  if (!c->shk) return PART_OK;  // taken up by the next part_enable_shocks
  cudaError_t e = launch_shock_cells(c);
  if (e != cudaSuccess) return cuda_fail(c, e, "part_set_shock_slope");
  return PART_OK;
}

part_status part_shock_slopes(part_ctx* c, const double** q_cell, int64_t* ncells) {
  if (check_ctx(c)) return PART_EINVAL;
  if (!q_cell || !ncells) return fail(c, PART_EINVAL, "NULL output");
  if (!c->shk) return fail(c, PART_EINVAL, "shocks are not enabled");
  *q_cell = c->shock_q;
  *ncells = c->geo.G;
  return PART_OK;
}

part_status part_shock_cells(part_ctx* c, const double** r_cell, int64_t* ncells) {
  if (check_ctx(c)) return PART_EINVAL;
  if (!r_cell || !ncells) return fail(c, PART_EINVAL, "NULL output");
  if (!c->shk) return fail(c, PART_EINVAL, "shocks are not enabled");
  *r_cell = c->shock_r;
  *ncells = c->geo.G;
  return PART_OK;
}

part_status part_cell_start(part_ctx* c, const uint32_t** cs, int64_t* nkeys) {
  if (check_ctx(c)) return PART_EINVAL;
  if (cs) *cs = c->cstart;
  if (nkeys) *nkeys = c->geo.nkeys;
  return PART_OK;
}

part_status part_enable_deposit(part_ctx* c, int on) {
  if (check_ctx(c)) return PART_EINVAL;
  if (c->mode != PART_BORIS) return fail(c, PART_EINVAL, "deposit is a Boris-mode feature");
  c->deposit_on = on != 0;
  return PART_OK;
}

part_status part_gather_push(part_ctx* c, double q_over_m, double dt, int nsteps) {
  if (check_ctx(c)) return PART_EINVAL;
  if (!c->bound) return fail(c, PART_EINVAL, "no particles bound");
  if (!c->fields_set) return fail(c, PART_EINVAL, "part_set_fields first");
  if (nsteps < 1) return fail(c, PART_EINVAL, "nsteps must be >= 1");
  if (!std::isfinite(dt) || dt == 0.0) return fail(c, PART_EINVAL, "dt must be finite, != 0");
  cudaError_t e;
  if (c->mode == PART_BORIS) {
    if (!std::isfinite(q_over_m)) return fail(c, PART_EINVAL, "q_over_m must be finite");
    if (c->deposit_on && nsteps != 1)
      return fail(c, PART_EINVAL, "deposit needs nsteps == 1 (fused steps are test particles)");
    if (c->deposit_on && !c->sorted)
      return fail(c, PART_EINVAL, "deposit needs part_sort since the last push");
    // the brick kernel (sorted, one step) reads the current buffer through
    // the sort's permutation; every other path needs the state in the bound
    // arrays first
    if (!(c->sorted && nsteps == 1)) {
      e = flush_pending(c);
      if (e != cudaSuccess) return cuda_fail(c, e, "part_gather_push");
    }
    e = launch_boris(c, q_over_m, dt, nsteps);
    c->moved += std::fabs(dt) * nsteps;  // |v| < 1: displacement bound
    if (e == cudaErrorNotSupported)
      return fail(c, PART_EUNSUPPORTED, "no kernel implements this precision/mode combination");
    c->deposit_ready = c->deposit_on;
  } else {
    if (nsteps != 1) return fail(c, PART_EINVAL, "LP mode advances one step per call");
    e = launch_lp_push(c, dt, nsteps);
    c->order_kept = false;  // fluid speeds are not bounded by the library
    c->samples_ready = true;
    c->shock_listed = c->shk != nullptr;
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "part_gather_push");
  c->sorted = false;
  return PART_OK;
}

part_status part_deposit(part_ctx* c, double* grid_out) {
  if (check_ctx(c)) return PART_EINVAL;
  if (!grid_out) return fail(c, PART_EINVAL, "grid_out is NULL");
  if (misaligned(grid_out, 8)) return fail(c, PART_EINVAL, "grid_out is not 8-byte aligned");
  if (check_access(c, grid_out, "grid_out") != PART_OK) return PART_EINVAL;
  if (c->mode != PART_BORIS || !c->deposit_ready)
    return fail(c, PART_EINVAL, "no deposit pending: enable it and push first");
  cudaError_t e = launch_deposit_combine(c, grid_out);
  if (e != cudaSuccess) return cuda_fail(c, e, "part_deposit");
  return PART_OK;
}

part_status spec_update(part_ctx* c, double dt, double c0, double u_rad) {
  if (check_ctx(c)) return PART_EINVAL;
  if (c->mode != PART_LP_RK2) return fail(c, PART_EINVAL, "spec_update needs LP mode");
  if (!c->samples_ready) return fail(c, PART_EINVAL, "no LP push since the last update");
  if (!std::isfinite(dt) || !std::isfinite(c0) || !std::isfinite(u_rad))
    return fail(c, PART_EINVAL, "dt, c0, u_rad must be finite");
  cudaError_t e = launch_spec_update(c, dt, c0, u_rad);
  if (e == cudaSuccess && c->shock_listed) e = launch_shock_convolve(c);
  c->shock_listed = false;
  if (e != cudaSuccess) return cuda_fail(c, e, "spec_update");
  c->samples_ready = false;
  return PART_OK;
}

part_status part_init_particles(part_ctx* c, uint64_t seed, double u_th, double eps_min,
                                double eps_max, double p_index, double N0) {
  if (check_ctx(c)) return PART_EINVAL;
  if (!c->bound) return fail(c, PART_EINVAL, "no particles bound");
  if (c->mode == PART_LP_RK2) {
    if (!c->fields_set) return fail(c, PART_EINVAL, "part_set_fields first (n_old = rho)");
    if (!(eps_min > 0.0) || !(eps_max > eps_min) || !std::isfinite(eps_max) ||
        !std::isfinite(p_index) || p_index == 1.0 || !std::isfinite(N0))
      return fail(c, PART_EINVAL, "need 0 < eps_min < eps_max, finite p_index != 1, N0");
  } else if (!std::isfinite(u_th) || u_th < 0.0) {
    return fail(c, PART_EINVAL, "u_th must be finite and >= 0");
  }
  c->cur_alt = false;  // every bound array is overwritten
  c->perm_pend = nullptr;
  c->spec_inv = false;
  c->maps_pending = false;
  cudaError_t e = launch_init(c, seed, u_th, eps_min, eps_max, p_index, N0);
  if (e != cudaSuccess) return cuda_fail(c, e, "part_init_particles");
  c->sorted = false;
  c->order_kept = false;
  c->lp_cache_ok = false;
  c->samples_ready = false;
  c->deposit_ready = false;
  return PART_OK;
}

part_status part_sync(part_ctx* c) {
  if (check_ctx(c)) return PART_EINVAL;
  int st = 0;
  cudaError_t e = flush_pending(c);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "part_sync");
  if (st == 0) return PART_OK;
  e = cudaMemsetAsync(c->status, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "part_sync reset");
  if (st & ST_TIMEOUT) return fail(c, PART_ETIMEOUT, "a bounded device wait ran out");
  if (st & ST_NONFINITE) return fail(c, PART_ENONFINITE, "non-finite particle state or sample");
  return fail(c, PART_EDOMAIN, "a particle was outside the cell it was sorted by");
}

const char* part_last_error(const part_ctx* c) {
  if (c) return c->err.c_str();
  return g_err.c_str();
}

int64_t part_launch_count(const part_ctx* c) { return c ? c->launches : 0; }

part_status part_selftest_wait(part_ctx* c, int64_t limit_ns, int arrive) {
  if (check_ctx(c)) return PART_EINVAL;
  if (limit_ns <= 0 || limit_ns > 10000000000LL)
    return fail(c, PART_EINVAL, "limit_ns must be in (0, 1e10]");
  if (arrive != 0 && arrive != 1) return fail(c, PART_EINVAL, "arrive must be 0 or 1");
  cudaError_t e = launch_selftest_wait(c, limit_ns, arrive);
  if (e != cudaSuccess) return cuda_fail(c, e, "part_selftest_wait");
  return PART_OK;
}

}  // extern "C"
