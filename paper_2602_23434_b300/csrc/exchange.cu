// exchange.cu -- the multi-rank pieces of the particle step.
//
// Particle exchange between subdomains (Sec. 3.3, "Multi-core
// communication"): along one axis at a time, the particles that left a
// rank's interior cells are flagged and counted, packed in index order into
// one send buffer per neighbour (left, right), shifted into the receiver's
// frame, and removed by the hole/filler compaction of Sec. 3.2; the received
// ones are appended (part_exchange_unpack).  The host protocol around these
// calls (counts first, non-blocking sends and receives, buffer resizing) is
// the caller's.
//
// Deposit halos: a rank's deposit reaches one cell beyond its interior; those
// halo planes are packed (part_box_pack), sent, and added to the owner's
// interior (part_box_add).
//
// Replicated grids: with the particles partitioned over ranks and the fields
// replicated, every rank deposits onto the whole grid; part_sum_ordered adds
// the ranks' grids in rank order, so every rank gets the same bits whatever
// the transport.
#include "part_internal.cuh"

namespace {

// Byte offsets of the planes of a packed exchange buffer for k particles: the
// bound planes in a fixed order, 8-byte ones first (ids, then FP64 state), so
// every plane is aligned to its element size when the buffer is.
struct XLayout {
  size_t id, x, off, u, w, chi, eng, nold, shk, total;
};
constexpr size_t kAbsent = ~(size_t)0;

XLayout xlayout(const part_ctx* c, int64_t k) {
  XLayout L{kAbsent, kAbsent, kAbsent, kAbsent, kAbsent, kAbsent, kAbsent, kAbsent, kAbsent, 0};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t r = o;
    o += bytes;
    return r;
  };
  const size_t kk = (size_t)k;
  if (c->id) L.id = take(8 * kk);
  if (c->mode == PART_BORIS && c->prec == PART_FP64) {
    L.x = take(24 * kk);
    L.u = take(24 * kk);
    if (c->w) L.w = take(8 * kk);
  } else if (c->mode == PART_BORIS) {
    L.x = take(4 * kk);
    L.off = take(12 * kk);
    L.u = take(24 * kk);
    if (c->w) L.w = take(4 * kk);
  } else {
    L.x = take(24 * kk);
    L.chi = take(8 * kk * c->nbins);
    L.eng = take(8 * kk * c->nbins);
    L.nold = take(8 * kk);
    if (c->shk) L.shk = take(kk);
  }
  L.total = o;
  return L;
}

// Flag the particles whose cell along `axis` lies below lo (left) or at or
// above hi (right).  FP64 and LP: s = (x - xmin) / dx in cell units with the
// library's roundings, left if s < lo, right if s >= hi (floor(s) < lo and
// floor(s) >= hi); mixed: the cell index itself.  NaN positions stay.
__global__ void k_exch_classify(const Geo g, int axis, int lo, int hi, const double* __restrict__ x,
                                const int32_t* __restrict__ cell, int64_t n,
                                uint32_t* __restrict__ fl, uint32_t* __restrict__ fr,
                                uint8_t* __restrict__ leaving) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p <= n;
       p += (int64_t)gridDim.x * blockDim.x) {
    if (p == n) {
      fl[n] = 0;
      fr[n] = 0;
      continue;
    }
    bool L = false, R = false;
    if (cell) {
      int j[3];
      cell_coords(g, cell[p], j);
      L = j[axis] < lo;
      R = j[axis] >= hi;
    } else {
      const double s = __dmul_rn(__dsub_rn(x[axis * n + p], g.xmin[axis]), g.inv_dx[axis]);
      L = s < (double)lo;
      R = s >= (double)hi;
    }
    fl[p] = L ? 1u : 0u;
    fr[p] = R ? 1u : 0u;
    leaving[p] = (L || R) ? 1 : 0;
  }
}

// Copy the flagged particles of one plane (rows x n, row stride n) into the
// left / right buffers (row strides kl, kr) at their scanned positions.
template <typename T>
__global__ void k_pack_plane(const T* __restrict__ src, int rows, int64_t n,
                             const uint32_t* __restrict__ sl, const uint32_t* __restrict__ sr,
                             T* __restrict__ dl, int64_t kl, T* __restrict__ dr, int64_t kr) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t a = sl[p], b = sr[p];
    if (sl[p + 1] != a) {
      for (int r = 0; r < rows; ++r) dl[(int64_t)r * kl + a] = src[(int64_t)r * n + p];
    } else if (sr[p + 1] != b) {
      for (int r = 0; r < rows; ++r) dr[(int64_t)r * kr + b] = src[(int64_t)r * n + p];
    }
  }
}

// Positions into the receiver's frame.  FP64 / LP: x_axis += dx (0, or the
// global period across the periodic seam: the same single rounding as the
// wrap of a one-domain run).
__global__ void k_shift_x(double* __restrict__ xa, int64_t k, double dx) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k;
       i += (int64_t)gridDim.x * blockDim.x)
    xa[i] = xa[i] + dx;
}

// Mixed form: the cell index re-based, j_axis += dj, and re-linearised with the
// receiver's cell count n_axis along the axis (the others are shared).
__global__ void k_shift_cell(const Geo g, int axis, int32_t* __restrict__ cell, int64_t k, int dj,
                             int n_axis) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k;
       i += (int64_t)gridDim.x * blockDim.x) {
    int j[3];
    cell_coords(g, cell[i], j);
    j[axis] += dj;
    int nn[3] = {g.n[0], g.n[1], g.n[2]};
    nn[axis] = n_axis;
    cell[i] = (int32_t)(((int64_t)j[2] * nn[1] + j[1]) * nn[0] + j[0]);
  }
}

__global__ void k_box_copy(const double* __restrict__ src, int ncomp, int nx, int ny, int nz,
                           int lx, int ly, int lz, int ex, int ey, int ez,
                           double* __restrict__ dst, int add) {
  const int64_t per = (int64_t)ex * ey * ez;
  const int64_t tot = per * ncomp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i / per);
    int64_t r = i - c * per;
    const int z = (int)(r / ((int64_t)ex * ey));
    r -= (int64_t)z * ex * ey;
    const int y = (int)(r / ex);
    const int xx = (int)(r - (int64_t)y * ex);
    const int64_t a = (((int64_t)c * nz + lz + z) * ny + ly + y) * nx + lx + xx;
    if (add)
      dst[a] = dst[a] + src[i];   // box_add: src packed, dst the full array
    else
      dst[i] = src[a];            // box_pack: src the full array, dst packed
  }
}

// out may alias parts' first row (each element is read before it is written)
__global__ void k_sum_ordered(double* out, const double* parts, int64_t count, int nparts) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = parts[i];
    for (int r = 1; r < nparts; ++r) s = s + parts[(int64_t)r * count + i];
    out[i] = s;
  }
}

int grid_of(int sms, int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > (int64_t)sms * 32) b = (int64_t)sms * 32;
  return (int)b;
}

int sms_current() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  return sms;
}

bool box_ok(const int dims[3], const int lo[3], const int ext[3]) {
  for (int a = 0; a < 3; ++a)
    if (dims[a] < 1 || lo[a] < 0 || ext[a] < 0 || (int64_t)lo[a] + ext[a] > dims[a]) return false;
  return true;
}

part_status box_call(const double* src, int ncomp, const int dims[3], const int lo[3],
                     const int ext[3], double* dst, void* stream, int add, const char* what) {
  if (!src || !dst || !dims || !lo || !ext || ncomp < 1)
    return fail(nullptr, PART_EINVAL, std::string(what) + ": NULL argument or ncomp < 1");
  if (!box_ok(dims, lo, ext))
    return fail(nullptr, PART_EINVAL, std::string(what) + ": box outside the array");
  if ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) % 8 != 0)
    return fail(nullptr, PART_EINVAL, std::string(what) + ": arrays must be 8-byte aligned");
  int dev = 0;
  const int sms = sms_current();
  if (cudaGetDevice(&dev) != cudaSuccess || sms < 1)
    return fail(nullptr, PART_ECUDA, std::string(what) + ": device query failed");
  if (!device_accessible(dev, src) || !device_accessible(dev, dst))
    return fail(nullptr, PART_EINVAL, std::string(what) + ": arrays the kernels cannot reach");
  const int64_t tot = (int64_t)ext[0] * ext[1] * ext[2] * ncomp;
  if (tot == 0) return PART_OK;
  k_box_copy<<<grid_of(sms, tot), 256, 0, (cudaStream_t)stream>>>(
      src, ncomp, dims[0], dims[1], dims[2], lo[0], lo[1], lo[2], ext[0], ext[1],
      ext[2], dst, add);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(nullptr, PART_ECUDA, std::string(what) + ": " +
                                                              cudaGetErrorString(e));
  return PART_OK;
}

}  // namespace

extern "C" {

part_status part_exchange_bytes(const part_ctx* c, int64_t k, size_t* bytes) {
  if (!c || !bytes || k < 0) return fail(nullptr, PART_EINVAL, "part_exchange_bytes: bad argument");
  *bytes = xlayout(c, k).total;
  return PART_OK;
}

part_status part_exchange_pack(part_ctx* c, int axis, int lo, int hi, const part_xshift* to_left,
                               const part_xshift* to_right, void* send_left, size_t left_bytes,
                               void* send_right, size_t right_bytes, uint8_t* leaving,
                               int64_t counts[2]) {
  if (check_ctx(c)) return PART_EINVAL;
  if (!c->bound) return fail(c, PART_EINVAL, "part_exchange_pack: no particles bound");
  if (axis < 0 || axis >= c->geo.dim || lo < 0 || hi <= lo || hi > c->geo.n[axis])
    return fail(c, PART_EINVAL, "part_exchange_pack: need 0 <= axis < dim, 0 <= lo < hi <= n");
  if (!to_left || !to_right || !counts || (c->n > 0 && !leaving))
    return fail(c, PART_EINVAL, "part_exchange_pack: NULL shift, counts or leaving");
  if (c->prec == PART_MIXED)
    for (const part_xshift* s : {to_left, to_right})
      if (s->n_axis < 1) return fail(c, PART_EINVAL, "part_exchange_pack: n_axis must be >= 1");
  if (check_access(c, leaving, "leaving") != PART_OK) return PART_EINVAL;
  if ((send_left && check_access(c, send_left, "send_left") != PART_OK) ||
      (send_right && check_access(c, send_right, "send_right") != PART_OK))
    return PART_EINVAL;
  if ((reinterpret_cast<uintptr_t>(send_left) | reinterpret_cast<uintptr_t>(send_right)) % 8)
    return fail(c, PART_EINVAL, "part_exchange_pack: send buffers must be 8-byte aligned");
  cudaError_t e = flush_pending(c);  // state home, spectra as (chi, eps)
  if (e != cudaSuccess) return cuda_fail(c, e, "part_exchange_pack");
  const int64_t n = c->n;
  counts[0] = counts[1] = 0;
  if (n == 0) return PART_OK;
  uint32_t* FL = c->keys[0];
  uint32_t* FR = c->keys[1];
  const bool mixed = c->prec == PART_MIXED;
  k_exch_classify<<<grid_for(c, n + 1, 256), 256, 0, c->stream>>>(
      c->geo, axis, lo, hi, mixed ? nullptr : (const double*)c->x,
      mixed ? (const int32_t*)c->x : nullptr, n, FL, FR, leaving);
  c->launches++;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_exclusive_scan(c, FL, n + 1, c->vals[0]);
  if (e == cudaSuccess) e = launch_exclusive_scan(c, FR, n + 1, c->vals[1]);
  uint32_t kl = 0, kr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&kl, FL + n, 4, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&kr, FR + n, 4, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "part_exchange_pack");
  counts[0] = kl;
  counts[1] = kr;
  const XLayout A = xlayout(c, kl), B = xlayout(c, kr);
  if ((kl > 0 && (!send_left || A.total > left_bytes)) ||
      (kr > 0 && (!send_right || B.total > right_bytes)))
    return fail(c, PART_ENOMEM,
                "part_exchange_pack: a send buffer is smaller than part_exchange_bytes(count); "
                "counts are set, nothing was packed");
  char* bl = (char*)send_left;
  char* br = (char*)send_right;
  const int gb = grid_for(c, n, 256);
  auto plane = [&](auto tag, const void* src, int rows, size_t offl, size_t offr) {
    using T = decltype(tag);
    if (!src || offl == kAbsent) return;
    k_pack_plane<T><<<gb, 256, 0, c->stream>>>((const T*)src, rows, n, FL, FR,
                                               (T*)(bl ? bl + offl : nullptr), kl,
                                               (T*)(br ? br + offr : nullptr), kr);
    c->launches++;
  };
  plane(uint64_t{}, c->id, 1, A.id, B.id);
  if (c->mode == PART_BORIS && !mixed) {
    plane(double{}, c->x, 3, A.x, B.x);
    plane(double{}, c->u, 3, A.u, B.u);
    plane(double{}, c->w, 1, A.w, B.w);
  } else if (c->mode == PART_BORIS) {
    plane(int32_t{}, c->x, 1, A.x, B.x);
    plane(float{}, c->off, 3, A.off, B.off);
    plane(float{}, c->u, 6, A.u, B.u);
    plane(float{}, c->w, 1, A.w, B.w);
  } else {
    plane(double{}, c->x, 3, A.x, B.x);
    plane(double{}, c->chi, c->nbins, A.chi, B.chi);
    plane(double{}, c->eng, c->nbins, A.eng, B.eng);
    plane(double{}, c->n_old, 1, A.nold, B.nold);
    plane(uint8_t{}, c->shk, 1, A.shk, B.shk);
  }
  // into the receivers' frames
  if (mixed) {
    if (kl > 0) {
      k_shift_cell<<<grid_for(c, kl, 256), 256, 0, c->stream>>>(
          c->geo, axis, (int32_t*)(bl + A.x), kl, to_left->dj, to_left->n_axis);
      c->launches++;
    }
    if (kr > 0) {
      k_shift_cell<<<grid_for(c, kr, 256), 256, 0, c->stream>>>(
          c->geo, axis, (int32_t*)(br + B.x), kr, to_right->dj, to_right->n_axis);
      c->launches++;
    }
  } else {
    if (kl > 0 && to_left->dx != 0.0) {
      k_shift_x<<<grid_for(c, kl, 256), 256, 0, c->stream>>>((double*)(bl + A.x) + axis * kl, kl,
                                                             to_left->dx);
      c->launches++;
    }
    if (kr > 0 && to_right->dx != 0.0) {
      k_shift_x<<<grid_for(c, kr, 256), 256, 0, c->stream>>>((double*)(br + B.x) + axis * kr, kr,
                                                             to_right->dx);
      c->launches++;
    }
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "part_exchange_pack");
  return PART_OK;
}

part_status part_exchange_unpack(part_ctx* c, int64_t k, const void* recv, size_t recv_bytes) {
  if (check_ctx(c)) return PART_EINVAL;
  if (!c->bound) return fail(c, PART_EINVAL, "part_exchange_unpack: no particles bound");
  if (k < 0 || k > c->capacity - c->n)
    return fail(c, PART_EINVAL, "part_exchange_unpack: k must be in [0, capacity - n]");
  if (k == 0) return PART_OK;
  const XLayout L = xlayout(c, k);
  if (!recv || recv_bytes < L.total || reinterpret_cast<uintptr_t>(recv) % 8)
    return fail(c, PART_EINVAL,
                "part_exchange_unpack: recv is NULL, unaligned or smaller than "
                "part_exchange_bytes(k)");
  if (check_access(c, recv, "recv") != PART_OK) return PART_EINVAL;
  const char* b = (const char*)recv;
  auto at = [&](size_t o) -> const void* { return o == kAbsent ? nullptr : b + o; };
  InjectSrc src{at(L.x), at(L.off), at(L.u), at(L.w), (const uint64_t*)at(L.id),
                (const double*)at(L.chi), (const double*)at(L.eng), (const double*)at(L.nold)};
  const int64_t n0 = c->n;
  cudaError_t e = flush_pending(c);
  if (e == cudaSuccess) e = launch_inject(c, k, src);
  // the shock flags travel with their LPs (injection clears new ones)
  if (e == cudaSuccess && c->shk && L.shk != kAbsent)
    e = cudaMemcpyAsync(c->shk + n0, b + L.shk, (size_t)k, cudaMemcpyDeviceToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "part_exchange_unpack");
  c->n += k;
  c->sorted = false;
  c->order_kept = false;
  c->lp_cache_ok = false;
  c->deposit_ready = false;
  c->samples_ready = false;
  c->shock_listed = false;
  return PART_OK;
}

part_status part_box_pack(const double* src, int ncomp, const int dims[3], const int lo[3],
                          const int ext[3], double* dst, void* cuda_stream) {
  return box_call(src, ncomp, dims, lo, ext, dst, cuda_stream, 0, "part_box_pack");
}

part_status part_box_add(double* dst, int ncomp, const int dims[3], const int lo[3],
                         const int ext[3], const double* src, void* cuda_stream) {
  return box_call(src, ncomp, dims, lo, ext, dst, cuda_stream, 1, "part_box_add");
}

part_status part_sum_ordered(double* out, const double* parts, int64_t count, int nparts,
                             void* cuda_stream) {
  if (!out || !parts || count < 0 || nparts < 1)
    return fail(nullptr, PART_EINVAL, "part_sum_ordered: NULL array, count < 0 or nparts < 1");
  if ((reinterpret_cast<uintptr_t>(out) | reinterpret_cast<uintptr_t>(parts)) % 8 != 0)
    return fail(nullptr, PART_EINVAL, "part_sum_ordered: arrays must be 8-byte aligned");
  int dev = 0;
  const int sms = sms_current();
  if (cudaGetDevice(&dev) != cudaSuccess || sms < 1)
    return fail(nullptr, PART_ECUDA, "part_sum_ordered: device query failed");
  if (!device_accessible(dev, out) || !device_accessible(dev, parts))
    return fail(nullptr, PART_EINVAL, "part_sum_ordered: arrays the kernels cannot reach");
  if (count == 0) return PART_OK;
  k_sum_ordered<<<grid_of(sms, count), 256, 0, (cudaStream_t)cuda_stream>>>(out, parts, count,
                                                                           nparts);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(nullptr, PART_ECUDA, std::string("part_sum_ordered: ") + cudaGetErrorString(e));
  return PART_OK;
}

}  // extern "C"
