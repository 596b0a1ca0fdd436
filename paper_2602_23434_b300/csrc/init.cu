// init.cu -- device-side particle initialisation and field padding.
//
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32 -> 64-bit multiplies (multipliers 0xD2511F53, 0xCD9E8D57), a word
// permutation, and a Weyl key schedule (0x9E3779B9, 0xBB67AE85).
// Particle p draws counter (p, 0) for its position and (p, 1) for three
// Box-Muller normals; key = seed.  LPs get the power law of Eq. initSpec.
#include "part_internal.cuh"

cudaError_t launch_lp_sample_rho(part_ctx* c);

namespace {

__device__ __forceinline__ void philox10(uint32_t* c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t a = c[0], b = c[2];
    const uint32_t hi0 = __umulhi(0xD2511F53u, a), lo0 = 0xD2511F53u * a;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, b), lo1 = 0xCD9E8D57u * b;
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// (r + 1/2) 2^-32: open interval (0, 1), exact in double
__device__ __forceinline__ double unit_open(uint32_t r) {
  return ((double)r + 0.5) * 2.3283064365386963e-10;
}

struct Draw {
  double x[3];
  double g[3];
};

__device__ __forceinline__ Draw draw_particle(const Geo& g, uint64_t seed, int64_t p) {
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  uint32_t c0[4] = {(uint32_t)p, (uint32_t)((uint64_t)p >> 32), 0u, 0u};
  uint32_t c1[4] = {(uint32_t)p, (uint32_t)((uint64_t)p >> 32), 1u, 0u};
  philox10(c0, k0, k1);
  philox10(c1, k0, k1);
  Draw d;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double v = __dadd_rn(g.xmin[a], __dmul_rn(g.L[a], unit_open(c0[a])));
    if (v < g.xmin[a]) v = v + g.L[a];
    else if (v >= g.xmax[a]) v = v - g.L[a];
    d.x[a] = v;
  }
  const double r0 = sqrt(-2.0 * log(unit_open(c1[0])));
  const double r1 = sqrt(-2.0 * log(unit_open(c1[2])));
  const double ph0 = (2.0 * 3.141592653589793) * unit_open(c1[1]);
  const double ph1 = (2.0 * 3.141592653589793) * unit_open(c1[3]);
  d.g[0] = r0 * cos(ph0);
  d.g[1] = r0 * sin(ph0);
  d.g[2] = r1 * cos(ph1);
  return d;
}

__global__ void k_init_boris_f64(const Geo g, int64_t n, uint64_t seed, double u_th,
                                 double* __restrict__ x, double* __restrict__ u,
                                 double* __restrict__ w, uint64_t* __restrict__ id) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    Draw d = draw_particle(g, seed, p);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      x[a * n + p] = d.x[a];
      u[a * n + p] = u_th * d.g[a];
    }
    if (w) w[p] = 1.0;
    if (id) id[p] = (uint64_t)p;
  }
}

// Mixed form: int32 linear cell + f32 offset from the cell centre.
__global__ void k_init_boris_mixed(const Geo g, int64_t n, uint64_t seed, double u_th,
                                   int32_t* __restrict__ cell, float* __restrict__ off,
                                   float* __restrict__ u, float* __restrict__ w,
                                   uint64_t* __restrict__ id) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    Draw d = draw_particle(g, seed, p);
    int j[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float dd = 0.0f;
      if (a < g.dim) {
        double s = __dmul_rn(__dsub_rn(d.x[a], g.xmin[a]), g.inv_dx[a]);
        double f = floor(s);
        j[a] = f >= (double)g.n[a] ? g.n[a] - 1 : (f < 0.0 ? 0 : (int)f);
        dd = (float)((s - (double)j[a]) - 0.5);
      }
      off[a * n + p] = dd;
      const double ua = u_th * d.g[a];
      const float hi = (float)ua;
      u[a * n + p] = hi;                        // u = hi + lo, the compensated pair
      u[(a + 3) * n + p] = (float)(ua - (double)hi);
    }
    cell[p] = (int32_t)(((int64_t)j[2] * g.n[1] + j[1]) * g.n[0] + j[0]);
    if (w) w[p] = 1.0f;
    if (id) id[p] = (uint64_t)p;
  }
}

// Node table of Eq. initSpec: eps_i log-spaced over [emin, emax] (both ends),
// chi_i = N0 (1-p)/(emax^(1-p) - emin^(1-p)) eps_i^-p.
__global__ void k_spec_table(int nb, double emin, double emax, double pidx, double N0,
                             double* __restrict__ tab) {
  const double la = log(emin), lb = log(emax);
  const double norm = N0 * (1.0 - pidx) / (pow(emax, 1.0 - pidx) - pow(emin, 1.0 - pidx));
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    const double e = nb > 1 ? exp(la + (lb - la) * ((double)i / (double)(nb - 1))) : emin;
    tab[i] = e;
    tab[nb + i] = norm * pow(e, -pidx);
  }
}

__global__ void k_init_lp(const Geo g, int64_t n, int nb, uint64_t seed,
                          const double* __restrict__ tab, double* __restrict__ x,
                          double* __restrict__ chi, double* __restrict__ eng,
                          uint64_t* __restrict__ id) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    Draw d = draw_particle(g, seed, p);
#pragma unroll
    for (int a = 0; a < 3; ++a) x[a * n + p] = d.x[a];
    for (int i = 0; i < nb; ++i) {
      eng[(int64_t)i * n + p] = tab[i];
      chi[(int64_t)i * n + p] = tab[nb + i];
    }
    if (id) id[p] = (uint64_t)p;
  }
}

// Ghost-filled padded copy: padded (px, py, pz) <- cell ((px-h) mod n, ...);
// x columns beyond n + 2 (row-pitch padding) are zero.
// Source cell of padded coordinate i (cell index, -h <= i < n + h with h <= 1):
// periodic image, or the edge cell on an open axis (zero-gradient ghost layer).
__device__ __forceinline__ int ghost_src(int i, int n, int open) {
  if (open) return i < 0 ? 0 : (i >= n ? n - 1 : i);
  return i < 0 ? i + n : (i >= n ? i - n : i);
}

// One warp per padded row (component, pz, py): the row's source row is fixed,
// so the lanes read it coalesced (x ghosts aside) and write the padded row
// contiguously; U loads per lane are in flight before the stores (the source
// may be pinned host memory read over the link).
template <typename T>
__global__ void k_pad_fields(const T* __restrict__ src, T* __restrict__ dst, const Geo g,
                             int ncomp) {
  constexpr int U = 4;
  const int lane = threadIdx.x & 31;
  const int64_t rows = (int64_t)ncomp * g.pn[2] * g.pn[1];
  const int64_t wstride = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int nx = g.n[0] + 2 * g.h[0];
  for (int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); r < rows;
       r += wstride) {
    const int py = (int)(r % g.pn[1]);
    const int64_t t = r / g.pn[1];
    const int pz = (int)(t % g.pn[2]);
    const int c = (int)(t / g.pn[2]);
    const int sy = ghost_src(py - g.h[1], g.n[1], g.open[1]);
    const int sz = ghost_src(pz - g.h[2], g.n[2], g.open[2]);
    const T* srow = src + (int64_t)c * g.G + ((int64_t)sz * g.n[1] + sy) * g.n[0];
    T* drow = dst + r * g.pn[0];
    for (int px0 = 0; px0 < g.pn[0]; px0 += 32 * U) {
      T v[U];
#pragma unroll
      for (int k = 0; k < U; ++k) {
        const int px = px0 + k * 32 + lane;
        v[k] = T(0);
        if (px < nx) v[k] = srow[ghost_src(px - g.h[0], g.n[0], g.open[0])];
      }
#pragma unroll
      for (int k = 0; k < U; ++k) {
        const int px = px0 + k * 32 + lane;
        if (px < g.pn[0]) drow[px] = v[k];
      }
    }
  }
}

// Mixed form: cell-interleaved copy, 8 floats per padded cell (6 components,
// 2 zero pads), so one stencil point is two 16-byte loads.  With the six
// components E0 E1 E2 B0 B1 B2 the record holds them as E0 E1 B0 B1 E2 B2, so
// that the push's paired arithmetic finds (E0, E1), (B0, B1) and (E2, B2) as
// aligned pairs.  One warp per padded row (pz, py); each lane gathers one
// cell's components (coalesced per component across the warp) and writes its
// 32 bytes as two 16-byte stores.
__global__ void k_pad_fields_aos8(const float* __restrict__ src, float* __restrict__ dst,
                                  const Geo g, int ncomp) {
  const int lane = threadIdx.x & 31;
  const int64_t rows = (int64_t)g.pn[2] * g.pn[1];
  const int64_t wstride = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int nx = g.n[0] + 2 * g.h[0];
  for (int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); r < rows;
       r += wstride) {
    const int py = (int)(r % g.pn[1]);
    const int pz = (int)(r / g.pn[1]);
    const int sy = ghost_src(py - g.h[1], g.n[1], g.open[1]);
    const int sz = ghost_src(pz - g.h[2], g.n[2], g.open[2]);
    const float* srow = src + ((int64_t)sz * g.n[1] + sy) * g.n[0];
    for (int px = lane; px < g.pn[0]; px += 32) {
      float v[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) v[c] = 0.0f;
      if (px < nx) {
        const int sx = ghost_src(px - g.h[0], g.n[0], g.open[0]);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          // the component in record slot c
          const int k = ncomp != 6 || c < 2 ? c : (c < 4 ? c + 1 : (c == 4 ? 2 : 5));
          if (c < ncomp) v[c] = srow[(int64_t)k * g.G + sx];
        }
      }
      float4* d = reinterpret_cast<float4*>(dst + (r * g.pn[0] + px) * 8);
      d[0] = make_float4(v[0], v[1], v[2], v[3]);
      d[1] = make_float4(v[4], v[5], v[6], v[7]);
    }
  }
}

// The x quadratics of the padded FP64 fields, used by the TSC gathers that
// read the fields from global memory in FP64: along x the three weighted
// cells of a stencil row sum to q0 + d (q1 + d q2), d the offset from the
// cell centre, with q0 = (F[-1] + F[1]) / 8 + 3 F[0] / 4,
// q1 = (F[1] - F[-1]) / 2 and q2 = (F[-1] + F[1]) / 2 - F[0] (the TSC weights
// expanded in d).  For each component and padded cell with both x neighbours,
// (q0, q1, q2, 0) as one 32-byte record; 0 elsewhere (never read).
__global__ void k_pad_xq(const double* __restrict__ fp, const Geo g, int ncomp,
                         double* __restrict__ fxq) {
  const int64_t pp = g.pplane;
  double4_32a* __restrict__ q4 = reinterpret_cast<double4_32a*>(fxq);
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < pp;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int px = (int)(q % g.pn[0]);
    const bool in = px >= 1 && px <= g.pn[0] - 2;
    for (int c = 0; c < ncomp; ++c) {
      double4_32a o;
      o.x = o.y = o.z = o.w = 0.0;
      if (in) {
        const double fm = fp[c * pp + q - 1], f0 = fp[c * pp + q], fq = fp[c * pp + q + 1];
        const double sp = fm + fq;
        o.x = fma(0.75, f0, 0.125 * sp);
        o.y = 0.5 * (fq - fm);
        o.z = fma(0.5, sp, -f0);
      }
      q4[c * pp + q] = o;
    }
  }
}

}  // namespace

cudaError_t launch_pad_fields(part_ctx* c, const void* src) {
  // one warp per padded row, 8 warps per CTA
  const int64_t rows = (int64_t)c->geo.pn[2] * c->geo.pn[1];
  if (c->fcomp == 8 && c->esize == 4)
    k_pad_fields_aos8<<<grid_for(c, rows * 32, 256), 256, 0, c->stream>>>(
        (const float*)src, (float*)c->fpad, c->geo, c->ncomp);
  else if (c->esize == 8)
    k_pad_fields<double><<<grid_for(c, rows * c->ncomp * 32, 256), 256, 0, c->stream>>>(
        (const double*)src, (double*)c->fpad, c->geo, c->ncomp);
  else
    k_pad_fields<float><<<grid_for(c, rows * c->ncomp * 32, 256), 256, 0, c->stream>>>(
        (const float*)src, (float*)c->fpad, c->geo, c->ncomp);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_init(part_ctx* c, uint64_t seed, double u_th, double emin, double emax,
                        double pidx, double N0) {
  const int64_t n = c->n;
  if (n == 0) return cudaSuccess;
  const int gb = grid_for(c, n, 256);
  if (c->mode == PART_BORIS && c->prec == PART_FP64) {
    k_init_boris_f64<<<gb, 256, 0, c->stream>>>(c->geo, n, seed, u_th, (double*)c->x,
                                                (double*)c->u, (double*)c->w, c->id);
    c->launches++;
  } else if (c->mode == PART_BORIS) {
    k_init_boris_mixed<<<gb, 256, 0, c->stream>>>(c->geo, n, seed, u_th, (int32_t*)c->x,
                                                  (float*)c->off, (float*)c->u, (float*)c->w,
                                                  c->id);
    c->launches++;
  } else {
    double* tab = (double*)c->tmp;
    k_spec_table<<<1, 128, 0, c->stream>>>(c->nbins, emin, emax, pidx, N0, tab);
    k_init_lp<<<gb, 256, 0, c->stream>>>(c->geo, n, c->nbins, seed, tab, (double*)c->x,
                                         c->chi, c->eng, c->id);
    c->launches += 2;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_lp_sample_rho(c);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------- wait self-test
// One thread waits on a shared-memory mbarrier with the kernels' bounded wait.
// With arrive = 1 it arrives first (the wait succeeds at once); with arrive = 0
// nothing ever arrives, the wait gives up after limit_ns and ST_TIMEOUT is
// latched, exactly as a brick kernel does when its TMA copy never lands.
namespace {
__global__ void k_selftest_wait(int* __restrict__ status, uint64_t limit_ns, int arrive) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  if (arrive)
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&bar)) : "memory");
  if (!mbar_wait_for(&bar, 0, limit_ns)) atomicOr(status, ST_TIMEOUT);
}
}  // namespace

cudaError_t launch_selftest_wait(part_ctx* c, int64_t limit_ns, int arrive) {
  k_selftest_wait<<<1, 32, 0, c->stream>>>(c->status, (uint64_t)limit_ns, arrive);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_pad_xq(part_ctx* c) {
  k_pad_xq<<<grid_for(c, c->geo.pplane, 256), 256, 0, c->stream>>>(
      (const double*)c->fpad, c->geo, c->ncomp, c->fxq);
  c->launches++;
  return cudaGetLastError();
}
