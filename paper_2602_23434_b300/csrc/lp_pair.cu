// lp_pair.cu -- the LP step (Eq. push, Heun RK2 or SSP-RK3, with the samples
// for Eq. cr_chi) in paired-f32 arithmetic (pair.cuh).
//
// The FP64 kernel (lp.cu) is bound by B300's FP64 pipe: about 440 FP64
// instructions per LP-step, at ~1/64 of the f32 rate.  Here positions stay
// FP64 in memory and are converted to pairs once on load and once on store
// (conversions run at the FP64 rate too); offsets, weights, the stencil sums
// and the position updates are pair arithmetic on the f32 pipes, two field
// components per packed f32x2 instruction.  The fields are read from a
// paired copy, 64 bytes per padded cell: hi(vx, vy, vz, rho),
// hi(Bx, By, Bz, 0), lo(...), lo(...).  The v, B cache is kept as pairs; the
// samples for spec_update are FP64, as the FP64 push leaves them.
//
// Accuracy: a pair carries ~48 bits, and every step is arranged so that the
// errors are absolute at that level: the in-cell offset is (x - c_j)/dx with
// c_j the cell's lower face, not (x - xmin)/dx - j (which would lose
// log2(n) bits), and the stencil sums are Dot2 accumulations.  Offsets come
// out within ~1e-13 cell, positions within ~1e-15 of the FP64 step.
#include "lp_shock.cuh"
#include "lp_spec.cuh"
#include "pair.cuh"
#include "part_internal.cuh"

namespace {

struct PairGeo {
  f2 xmin[3], dx[3], inv_dx[3], L[3], xmax[3];
  float nf[3];  // cells per axis
};

__device__ __forceinline__ f2 wrap_p(const Geo& g, const PairGeo& pg, int a, f2 v) {
  if (g.open[a]) return v;
  if (f2_lt(v, pg.xmin[a])) return f2_add(v, pg.L[a]);
  if (!f2_lt(v, pg.xmax[a])) return f2_sub(v, pg.L[a]);
  return v;
}

// TSC / CIC weights from the in-cell offset d (|d| <= 1/2): TSC in the
// factored forms (1/2 - d)^2/2, 3/4 - d^2, (1/2 + d)^2/2
template <int SHAPE>
__device__ __forceinline__ void weights_p(f2 d, f2* w) {
  if (SHAPE == PART_TSC) {
    const f2 a = f2_addf(f2_neg(d), 0.5f), b = f2_addf(d, 0.5f);
    w[0] = f2_scale(f2_norm(f2_sqr_u(a)), 0.5f);
    w[1] = f2_addf(f2_neg(f2_norm(f2_sqr_u(d))), 0.75f);
    w[2] = f2_scale(f2_norm(f2_sqr_u(b)), 0.5f);
  } else {
    const f2 z = {0.0f, 0.0f};
    const bool neg = d.h < 0.0f;
    w[0] = neg ? f2_neg(d) : z;
    w[2] = neg ? z : d;
    w[1] = f2_addf(neg ? d : f2_neg(d), 1.0f);
  }
}

// The two float4 of a 32-byte load (one sector).
__device__ __forceinline__ void split32(const ulonglong4_32a v, float4& a, float4& b) {
  a = make_float4(__uint_as_float((uint32_t)v.x), __uint_as_float((uint32_t)(v.x >> 32)),
                  __uint_as_float((uint32_t)v.y), __uint_as_float((uint32_t)(v.y >> 32)));
  b = make_float4(__uint_as_float((uint32_t)v.z), __uint_as_float((uint32_t)(v.z >> 32)),
                  __uint_as_float((uint32_t)v.w), __uint_as_float((uint32_t)(v.w >> 32)));
}

template <int SHAPE, int DIM>
struct StencilP {
  int64_t base;  // padded index of the (-1,-1,-1) corner
  int64_t cell;  // linear index of the cell containing the position
  f2 wx[3], wy[3], wz[3];
  bool finite;
  __device__ __forceinline__ StencilP(const Geo& g, const PairGeo& pg, const f2* X) {
    int j[3] = {0, 0, 0};
    f2 d[3] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
    finite = true;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const f2 s = f2_mul(f2_sub(X[a], pg.xmin[a]), pg.inv_dx[a]);  // cells from xmin
      const int nm = g.n[a] - 1;
      if (!(isfinite(s.h) && isfinite(s.l))) {
        finite = false;
        continue;                                   // j = 0, d = 0
      }
      if (g.open[a] && (s.h < 0.0f || (s.h == 0.0f && s.l < 0.0f))) {
        d[a] = {-0.5f, 0.0f};                         // sampled at the lower face
        continue;
      }
      if (g.open[a] && !f2_lt(s, {pg.nf[a], 0.0f})) {
        j[a] = nm;
        d[a] = {0.5f, 0.0f};                          // sampled at the upper face
        continue;
      }
      float fl = floorf(s.h);
      if (fl == s.h && s.l < 0.0f) fl -= 1.0f;
      int jj = (int)fl;
      jj = jj < 0 ? 0 : (jj > nm ? nm : jj);
      j[a] = jj;
      // d = (x - c_j)/dx - 1/2, c_j = xmin + j dx: the difference is formed
      // between two O(1) pairs, so it keeps their absolute accuracy
      const f2 jd = f2_mul_u(pg.dx[a], {(float)jj, 0.0f});
      const f2 cj = f2_add(pg.xmin[a], f2_norm(jd));
      const f2 f = f2_mul(f2_sub(X[a], cj), pg.inv_dx[a]);
      const f2 t = f2_two_sum(f.h, -0.5f);
      d[a] = f2_two_sum(t.h, t.l + f.l);
    }
    weights_p<SHAPE>(d[0], wx);
    weights_p<SHAPE>(d[1], wy);
    wz[0] = {0.0f, 0.0f};
    wz[1] = {1.0f, 0.0f};
    wz[2] = {0.0f, 0.0f};
    if (DIM == 3) weights_p<SHAPE>(d[2], wz);
    base = ((int64_t)j[2] * g.pn[1] + j[1]) * g.pn[0] + j[0];
    cell = ((int64_t)j[2] * g.n[1] + j[1]) * g.n[0] + j[0];
  }
  // stencil sums of NP component pairs: pairs 0, 1 = (vx, vy), (vz, rho);
  // pairs 2, 3 = (Bx, By), (Bz, 0).  (ah + al) per component on return.
  template <int NP>
  __device__ __forceinline__ void gather(const float4* __restrict__ fq, const Geo& g, float2* ah,
                                         float2* al) const {
#pragma unroll
    for (int c = 0; c < NP; ++c) ah[c] = al[c] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int kz = (DIM == 3 ? 0 : 1); kz < (DIM == 3 ? 3 : 2); ++kz) {
      const int zo = DIM == 3 ? kz : 0;
#pragma unroll
      for (int ky = 0; ky < 3; ++ky) {
        const f2 wzy = f2_mul_u(wz[kz], wy[ky]);
        const int64_t row = base + ((int64_t)zo * g.pn[1] + ky) * g.pn[0];
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
          const f2 ww = f2_mul_u(wzy, wx[kx]);
          // one 32-byte load per half record: (v, rho) high and low parts, then
          // (B, 0) high and low parts
          const ulonglong4_32a* q = reinterpret_cast<const ulonglong4_32a*>(fq + 4 * (row + kx));
          float4 h0, l0;
          split32(q[0], h0, l0);
          dot2_acc2(ah[0], al[0], ww, make_float2(h0.x, h0.y), make_float2(l0.x, l0.y));
          dot2_acc2(ah[1], al[1], ww, make_float2(h0.z, h0.w), make_float2(l0.z, l0.w));
          if (NP == 4) {
            float4 h1, l1;
            split32(q[1], h1, l1);
            dot2_acc2(ah[2], al[2], ww, make_float2(h1.x, h1.y), make_float2(l1.x, l1.y));
            dot2_acc2(ah[3], al[3], ww, make_float2(h1.z, h1.w), make_float2(l1.z, l1.w));
          }
        }
      }
    }
  }
};

__device__ __forceinline__ void unpack(const float2* ah, const float2* al, int k, f2* out) {
  out[0] = f2_two_sum(ah[k].x, al[k].x);
  out[1] = f2_two_sum(ah[k].y, al[k].y);
}

__device__ __forceinline__ f2 norm2_p(const f2* v) {
  return f2_add(f2_add(f2_norm(f2_sqr_u(v[0])), f2_norm(f2_sqr_u(v[1]))), f2_norm(f2_sqr_u(v[2])));
}

struct StepDt {
  f2 dt, half, quarter, sixth;
};

// cache: [12][n] floats, v.h[3], v.l[3], B.h[3], B.l[3].  LPs [p0, p1) of
// the n bound (the row stride of every array).
// The push of one LP, leaving its samples (density, <|B|^2>, 1/gamma_g) as
// pairs.
template <int SHAPE, int DIM, bool SHOCK, int ORDER, bool CACHED>
struct PushPair {
  LpArgs A;   // A.fp: the paired copy (float4 records); A.cache: [12][n] floats
  PairGeo pg;
  StepDt sd;
  __device__ __forceinline__ void pairs(int64_t p, f2* smp) const {
    const float4* __restrict__ fq = reinterpret_cast<const float4*>(A.fp);
    const Geo& g = A.g;
    double* __restrict__ x = A.x;
    const int64_t n = A.n;
    int* __restrict__ status = A.status;
    float* __restrict__ cache = reinterpret_cast<float*>(A.cache);
    uint8_t* __restrict__ outmask = A.outmask;
    f2 X0[3] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
    double x0d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      x0d[a] = x[a * n + p];
      if (a < DIM) X0[a] = f2_of(x0d[a]);
    }
    f2 v1[3], b0[3];
    bool fin;
    if (CACHED) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        v1[c] = {cache[c * n + p], cache[(3 + c) * n + p]};
        b0[c] = {cache[(6 + c) * n + p], cache[(9 + c) * n + p]};
      }
      fin = isfinite(x0d[0]) && isfinite(x0d[1]) && isfinite(x0d[2]);
    } else {
      StencilP<SHAPE, DIM> s0(g, pg, X0);
      float2 ah[4], al[4];
      s0.template gather<4>(fq, g, ah, al);
      f2 t[2];
      unpack(ah, al, 0, t);
      v1[0] = t[0];
      v1[1] = t[1];
      unpack(ah, al, 1, t);
      v1[2] = t[0];
      unpack(ah, al, 2, t);
      b0[0] = t[0];
      b0[1] = t[1];
      unpack(ah, al, 3, t);
      b0[2] = t[0];
      fin = s0.finite;
    }
    f2 XS[3] = {X0[0], X0[1], X0[2]};
#pragma unroll
    for (int a = 0; a < DIM; ++a) XS[a] = wrap_p(g, pg, a, f2_add(X0[a], f2_mul(sd.dt, v1[a])));
    StencilP<SHAPE, DIM> ss(g, pg, XS);
    f2 v2[3];
    {
      float2 ah[2], al[2];
      ss.template gather<2>(fq, g, ah, al);
      f2 t[2];
      unpack(ah, al, 0, t);
      v2[0] = t[0];
      v2[1] = t[1];
      unpack(ah, al, 1, t);
      v2[2] = t[0];
    }
    fin = fin && ss.finite;
    f2 X1[3] = {X0[0], X0[1], X0[2]};
    if (ORDER == 2) {
#pragma unroll
      for (int a = 0; a < DIM; ++a)
        X1[a] = wrap_p(g, pg, a, f2_add(X0[a], f2_mul(sd.half, f2_add(v1[a], v2[a]))));
    } else {
      f2 XB[3] = {X0[0], X0[1], X0[2]};
#pragma unroll
      for (int a = 0; a < DIM; ++a)
        XB[a] = wrap_p(g, pg, a, f2_add(X0[a], f2_mul(sd.quarter, f2_add(v1[a], v2[a]))));
      StencilP<SHAPE, DIM> sb(g, pg, XB);
      f2 k3[3];
      {
        float2 ah[2], al[2];
        sb.template gather<2>(fq, g, ah, al);
        f2 t[2];
        unpack(ah, al, 0, t);
        k3[0] = t[0];
        k3[1] = t[1];
        unpack(ah, al, 1, t);
        k3[2] = t[0];
      }
      fin = fin && sb.finite;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        const f2 k = f2_add(f2_add(v1[a], v2[a]), f2_scale(k3[a], 4.0f));
        X1[a] = wrap_p(g, pg, a, f2_add(X0[a], f2_mul(sd.sixth, k)));
      }
    }
    StencilP<SHAPE, DIM> s1(g, pg, X1);
    f2 v3[3], b1[3], r;
    {
      float2 ah[4], al[4];
      s1.template gather<4>(fq, g, ah, al);
      f2 t[2];
      unpack(ah, al, 0, t);
      v3[0] = t[0];
      v3[1] = t[1];
      unpack(ah, al, 1, t);
      v3[2] = t[0];
      r = t[1];
      unpack(ah, al, 2, t);
      b1[0] = t[0];
      b1[1] = t[1];
      unpack(ah, al, 3, t);
      b1[2] = t[0];
    }
    double x1d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      x1d[a] = a < DIM ? f2_to(X1[a]) : x0d[a];
      x[a * n + p] = x1d[a];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      cache[c * n + p] = v3[c].h;
      cache[(3 + c) * n + p] = v3[c].l;
      cache[(6 + c) * n + p] = b1[c].h;
      cache[(9 + c) * n + p] = b1[c].l;
    }
    if (outmask) outmask[p] = outside_open(g, x1d);
    const f2 bm = f2_scale(f2_add(norm2_p(b0), norm2_p(b1)), 0.5f);
    const f2 om = f2_add({1.0f, 0.0f}, f2_neg(norm2_p(v3)));   // 1 - |v|^2
    // 1/gamma_g; not a number where 1 - |v|^2 <= 0 (flagged below, as in FP64)
    const f2 ig = om.h > 0.0f ? f2_sqrt(om) : f2{__int_as_float(0x7fc00000), 0.0f};
    smp[0] = r;
    smp[1] = bm;
    smp[2] = ig;
    if (!(fin && s1.finite && ig.h > 0.0f && isfinite(r.h) && r.h > 0.0f))
      atomicOr(status, ST_NONFINITE);
    if (SHOCK) shock_mark(p, s1.cell, A.shock_r, A.shock_q, A.shk, A.list, A.rs, A.qs);
  }
};

// The samples [4][n] for spec_update (lp_samples): the step's logarithm and
// exponential in FP64 on the pipe the paired push leaves idle.
template <int SHAPE, int DIM, bool SHOCK, int ORDER, bool CACHED>
__global__ void __launch_bounds__(256, 2)
    k_lp_pair(const PushPair<SHAPE, DIM, SHOCK, ORDER, CACHED> push, double* __restrict__ samples,
              int64_t p0, int64_t p1) {
  const int64_t n = push.A.n;
  for (int64_t p = p0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < p1;
       p += (int64_t)gridDim.x * blockDim.x) {
    f2 t[3];
    push.pairs(p, t);
    double s4[4];
    lp_samples(push.A.n_old[p], f2_to(t[0]), f2_to(t[1]), f2_to(t[2]), s4);
#pragma unroll
    for (int k = 0; k < 4; ++k) samples[k * n + p] = s4[k];
  }
}

// The paired copy of the padded LP fields (7 FP64 planes -> 64 B per cell).
__global__ void k_pad_pair_lp(const double* __restrict__ fp, int64_t pplane,
                              float4* __restrict__ fq) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < pplane;
       q += (int64_t)gridDim.x * blockDim.x) {
    float h[8], l[8];
#pragma unroll
    for (int c = 0; c < 7; ++c) {
      const f2 v = f2_of(fp[c * pplane + q]);
      h[c] = v.h;
      l[c] = v.l;
    }
    h[7] = l[7] = 0.0f;
    // 32-byte halves: (v, rho) high, low; (B, 0) high, low
    fq[4 * q + 0] = make_float4(h[0], h[1], h[2], h[3]);
    fq[4 * q + 1] = make_float4(l[0], l[1], l[2], l[3]);
    fq[4 * q + 2] = make_float4(h[4], h[5], h[6], h[7]);
    fq[4 * q + 3] = make_float4(l[4], l[5], l[6], l[7]);
  }
}

PairGeo pair_geo(const Geo& g) {
  PairGeo pg;
  for (int a = 0; a < 3; ++a) {
    pg.xmin[a] = f2_host(g.xmin[a]);
    pg.dx[a] = f2_host(g.dx[a]);
    pg.inv_dx[a] = f2_host(g.inv_dx[a]);
    pg.L[a] = f2_host(g.L[a]);
    pg.xmax[a] = f2_host(g.xmax[a]);
    pg.nf[a] = (float)g.n[a];
  }
  return pg;
}

template <int SHAPE, int DIM, bool SHOCK, int ORDER, bool CACHED>
PushPair<SHAPE, DIM, SHOCK, ORDER, CACHED> push_pair(part_ctx* c, double dt) {
  PushPair<SHAPE, DIM, SHOCK, ORDER, CACHED> f;
  f.A = lp_args(c, dt);
  f.A.fp = reinterpret_cast<const double*>(c->fpair);
  f.pg = pair_geo(c->geo);
  f.sd = {f2_host(dt), f2_host(0.5 * dt), f2_host(0.25 * dt), f2_host(dt * (1.0 / 6.0))};
  return f;
}

template <int SHAPE, int DIM, int ORDER, bool CACHED>
cudaError_t lp_pair_launch(part_ctx* c, double dt, const LpLaunch& L) {
  double* smp = c->samples;
  if (c->shk)
    k_lp_pair<<<L.grid, 256, 0, L.stream>>>(push_pair<SHAPE, DIM, true, ORDER, CACHED>(c, dt),
                                            smp, L.p0, L.p1);
  else
    k_lp_pair<<<L.grid, 256, 0, L.stream>>>(push_pair<SHAPE, DIM, false, ORDER, CACHED>(c, dt),
                                            smp, L.p0, L.p1);
  c->launches++;
  return cudaGetLastError();
}

template <int SHAPE, int DIM>
cudaError_t lp_pair_dispatch(part_ctx* c, double dt, const LpLaunch& L) {
  if (c->lp_order == 3)
    return L.cached ? lp_pair_launch<SHAPE, DIM, 3, true>(c, dt, L)
                    : lp_pair_launch<SHAPE, DIM, 3, false>(c, dt, L);
  return L.cached ? lp_pair_launch<SHAPE, DIM, 2, true>(c, dt, L)
                  : lp_pair_launch<SHAPE, DIM, 2, false>(c, dt, L);
}

}  // namespace

cudaError_t launch_lp_push_pair_range(part_ctx* c, double dt, const LpLaunch& L) {
  if (L.p1 <= L.p0) return cudaSuccess;
  if (c->shape == PART_TSC)
    return c->geo.dim == 3 ? lp_pair_dispatch<PART_TSC, 3>(c, dt, L)
                           : lp_pair_dispatch<PART_TSC, 2>(c, dt, L);
  return c->geo.dim == 3 ? lp_pair_dispatch<PART_CIC, 3>(c, dt, L)
                         : lp_pair_dispatch<PART_CIC, 2>(c, dt, L);
}

cudaError_t launch_pad_pair_lp(part_ctx* c) {
  k_pad_pair_lp<<<grid_for(c, c->geo.pplane, 256), 256, 0, c->stream>>>(
      (const double*)c->fpad, c->geo.pplane, reinterpret_cast<float4*>(c->fpair));
  c->launches++;
  return cudaGetLastError();
}
