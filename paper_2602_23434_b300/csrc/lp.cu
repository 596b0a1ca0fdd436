// lp.cu -- Lagrangian-particle advection (Eq. push, Heun RK2 or SSP-RK3) and the
// per-bin spectral update of Eq. cr_chi (exact characteristics).
//
// Fields: padded FP64 copy with 7 components: v[3], rho, B[3] (the fluid
// quantities an LP samples, Sec. 2).  Spectra are bin-major [nb][n], so every
// bin access of a warp is one coalesced 256-byte row.
#include <algorithm>

#include "lp_shock.cuh"
#include "lp_spec.cuh"
#include "part_internal.cuh"

namespace {

// Periodic wrap of coordinate a, or none on an open axis.
__device__ __forceinline__ double wrap_axis(const Geo& g, int a, double v) {
  if (g.open[a]) return v;
  if (v < g.xmin[a]) v = v + g.L[a];
  else if (v >= g.xmax[a]) v = v - g.L[a];
  return v;
}

// Stencil of position x: padded row origin and weights per axis.
template <int SHAPE, int DIM>
struct Stencil {
  int64_t base;     // padded index of the (-1,-1,-1) corner
  int64_t cell;     // linear index of the cell containing x
  double wx[3], wy[3], wz[3];
  double dxo;       // offset from the cell centre along x, in cells (the TSC x quadratic)
  bool finite;
  __device__ __forceinline__ Stencil(const Geo& g, const double* xp) {
    int j[3] = {0, 0, 0};
    double d[3] = {0.0, 0.0, 0.0};
    finite = true;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      double s = __dmul_rn(__dsub_rn(xp[a], g.xmin[a]), g.inv_dx[a]);
      if (!finite_bits(s)) {
        finite = false;
        s = 0.0;
      }
      if (g.open[a]) s = fmin(fmax(s, 0.0), (double)g.n[a]);  // sample at the boundary
      j[a] = floor_clamp_bits(s, g.n[a] - 1);
      d[a] = __dsub_rn(__dsub_rn(s, (double)j[a]), 0.5);
    }
    dxo = d[0];
    shape_weights<SHAPE>(d[0], wx);
    shape_weights<SHAPE>(d[1], wy);
    wz[0] = 0.0;
    wz[1] = 1.0;
    wz[2] = 0.0;
    if (DIM == 3) shape_weights<SHAPE>(d[2], wz);
    base = ((int64_t)j[2] * g.pn[1] + j[1]) * g.pn[0] + j[0];
    cell = ((int64_t)j[2] * g.n[1] + j[1]) * g.n[0] + j[0];
  }
  // sum over the stencil of components [c0, c0 + NC); the 27 weight products
  // are formed once for all NC components
  template <int NC>
  __device__ __forceinline__ void gather(const double* __restrict__ fp, const Geo& g, int c0,
                                         double* out) const {
#pragma unroll
    for (int c = 0; c < NC; ++c) out[c] = 0.0;
#pragma unroll
    for (int kz = (DIM == 3 ? 0 : 1); kz < (DIM == 3 ? 3 : 2); ++kz) {
      const int zo = DIM == 3 ? kz : 0;
#pragma unroll
      for (int ky = 0; ky < 3; ++ky) {
        const double wzy = wz[kz] * wy[ky];
        const int64_t row = base + ((int64_t)zo * g.pn[1] + ky) * g.pn[0];
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
          const double ww = wzy * wx[kx];
#pragma unroll
          for (int c = 0; c < NC; ++c)
            out[c] += ww * __ldg(fp + (int64_t)(c0 + c) * g.pplane + row + kx);
        }
      }
    }
  }
  // TSC from the x quadratics (fxq): along x the three weighted cells of a
  // row are q0 + d (q1 + d q2) with d the offset from the cell centre, where
  // q0 = (F[-1] + F[1]) / 8 + 3 F[0] / 4, q1 = (F[1] - F[-1]) / 2 and
  // q2 = (F[-1] + F[1]) / 2 - F[0] (the expansion of the TSC weights in d):
  // two FMAs per row and component, one 32-byte load, no x weight products.
  template <int NC>
  __device__ __forceinline__ void gather_xq(const double* __restrict__ fxq, const Geo& g, int c0,
                                            double* out) const {
    const double4_32a* __restrict__ q4 = reinterpret_cast<const double4_32a*>(fxq);
#pragma unroll
    for (int c = 0; c < NC; ++c) out[c] = 0.0;
#pragma unroll
    for (int kz = (DIM == 3 ? 0 : 1); kz < (DIM == 3 ? 3 : 2); ++kz) {
      const int zo = DIM == 3 ? kz : 0;
#pragma unroll
      for (int ky = 0; ky < 3; ++ky) {
        const double wzy = wz[kz] * wy[ky];
        const int64_t rc = base + ((int64_t)zo * g.pn[1] + ky) * g.pn[0] + 1;  // row centre
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const double4_32a q = q4[(int64_t)(c0 + c) * g.pplane + rc];
          out[c] = fma(wzy, fma(dxo, fma(dxo, q.z, q.y), q.x), out[c]);
        }
      }
    }
  }
  // components {0,1,2} (v) and {4,5,6} (B) in one pass, from the x quadratics
  __device__ __forceinline__ void gather_vb_xq(const double* __restrict__ fxq, const Geo& g,
                                               double* v, double* b) const {
    const double4_32a* __restrict__ q4 = reinterpret_cast<const double4_32a*>(fxq);
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c] = b[c] = 0.0;
#pragma unroll
    for (int kz = (DIM == 3 ? 0 : 1); kz < (DIM == 3 ? 3 : 2); ++kz) {
      const int zo = DIM == 3 ? kz : 0;
#pragma unroll
      for (int ky = 0; ky < 3; ++ky) {
        const double wzy = wz[kz] * wy[ky];
        const int64_t rc = base + ((int64_t)zo * g.pn[1] + ky) * g.pn[0] + 1;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const double4_32a qv = q4[(int64_t)c * g.pplane + rc];
          const double4_32a qb = q4[(int64_t)(4 + c) * g.pplane + rc];
          v[c] = fma(wzy, fma(dxo, fma(dxo, qv.z, qv.y), qv.x), v[c]);
          b[c] = fma(wzy, fma(dxo, fma(dxo, qb.z, qb.y), qb.x), b[c]);
        }
      }
    }
  }
  // the gathers the push uses: the x quadratics for TSC, the weights for CIC
  template <int NC>
  __device__ __forceinline__ void gather_lp(const double* __restrict__ fp,
                                            const double* __restrict__ fxq, const Geo& g, int c0,
                                            double* out) const {
    if (SHAPE == PART_TSC)
      gather_xq<NC>(fxq, g, c0, out);
    else
      gather<NC>(fp, g, c0, out);
  }
  __device__ __forceinline__ void gather_vb_lp(const double* __restrict__ fp,
                                               const double* __restrict__ fxq, const Geo& g,
                                               double* v, double* b) const {
    if (SHAPE == PART_TSC)
      gather_vb_xq(fxq, g, v, b);
    else
      gather_vb(fp, g, v, b);
  }
  // components {0,1,2} (v) and {4,5,6} (B) in one stencil pass
  __device__ __forceinline__ void gather_vb(const double* __restrict__ fp, const Geo& g,
                                            double* v, double* b) const {
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c] = b[c] = 0.0;
#pragma unroll
    for (int kz = (DIM == 3 ? 0 : 1); kz < (DIM == 3 ? 3 : 2); ++kz) {
      const int zo = DIM == 3 ? kz : 0;
#pragma unroll
      for (int ky = 0; ky < 3; ++ky) {
        const double wzy = wz[kz] * wy[ky];
        const int64_t row = base + ((int64_t)zo * g.pn[1] + ky) * g.pn[0];
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
          const double ww = wzy * wx[kx];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            v[c] += ww * __ldg(fp + (int64_t)c * g.pplane + row + kx);
            b[c] += ww * __ldg(fp + (int64_t)(4 + c) * g.pplane + row + kx);
          }
        }
      }
    }
  }
};

// ORDER 2: Heun, x' = x + dt (k1 + k2)/2.  ORDER 3: three-stage SSP
// Runge-Kutta (Shu & Osher) in stage-velocity form, k3 = v(x + dt (k1+k2)/4),
// x' = x + dt (k1 + k2 + 4 k3)/6; the wrap only enters the sampled positions.
// Each update is one FMA with dt/2, dt/4 or dt/6 (no division per LP).
// CACHED: v and B at x (from the previous step's samples at its new
// position, the same stencil at the same point) are read instead of gathered;
// every step leaves v and B at x' for the next one (cache [6][n]).
// LPs [p0, p1) of the n bound (the row stride of every array).
// The push of one LP, leaving its samples (density, <|B|^2>, 1/gamma_g) in
// s3.
template <int SHAPE, int DIM, bool SHOCK, int ORDER, bool CACHED>
struct PushF64 {
  LpArgs A;
  __device__ __forceinline__ void operator()(int64_t p, double* s3) const {
    const double* __restrict__ fp = A.fp;
    const Geo& g = A.g;
    double* __restrict__ x = A.x;
    const int64_t n = A.n;
    const double dt = A.dt;
    int* __restrict__ status = A.status;
    double* __restrict__ cache = A.cache;
    uint8_t* __restrict__ outmask = A.outmask;
    double x0[3], xs[3], x1[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) x0[a] = xs[a] = x1[a] = x[a * n + p];
    double v1[3], b0[3], v2[3], v3[3], b1[3], r;
    bool fin;
    if (CACHED) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        v1[c] = cache[c * n + p];
        b0[c] = cache[(3 + c) * n + p];
      }
      fin = finite_bits(x0[0]) && finite_bits(x0[1]) && finite_bits(x0[2]);
    } else {
      Stencil<SHAPE, DIM> s0(g, x0);
      s0.gather_vb_lp(fp, A.fxq, g, v1, b0);
      fin = s0.finite;
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a) xs[a] = wrap_axis(g, a, fma(dt, v1[a], x0[a]));
    Stencil<SHAPE, DIM> ss(g, xs);
    ss.template gather_lp<3>(fp, A.fxq, g, 0, v2);
    fin = fin && ss.finite;
    if (ORDER == 2) {
#pragma unroll
      for (int a = 0; a < DIM; ++a)
        x1[a] = wrap_axis(g, a, fma(0.5 * dt, v1[a] + v2[a], x0[a]));
    } else {
      double xb[3] = {x0[0], x0[1], x0[2]}, k3[3];
      const double dt6 = dt * (1.0 / 6.0);
#pragma unroll
      for (int a = 0; a < DIM; ++a)
        xb[a] = wrap_axis(g, a, fma(0.25 * dt, v1[a] + v2[a], x0[a]));
      Stencil<SHAPE, DIM> sb(g, xb);
      sb.template gather_lp<3>(fp, A.fxq, g, 0, k3);
      fin = fin && sb.finite;
#pragma unroll
      for (int a = 0; a < DIM; ++a)
        x1[a] = wrap_axis(g, a, fma(dt6, fma(4.0, k3[a], v1[a] + v2[a]), x0[a]));
    }
    Stencil<SHAPE, DIM> s1(g, x1);
    {
      double o[7];  // v, rho, B at the new position in one stencil pass
      s1.template gather_lp<7>(fp, A.fxq, g, 0, o);
      v3[0] = o[0];
      v3[1] = o[1];
      v3[2] = o[2];
      r = o[3];
      b1[0] = o[4];
      b1[1] = o[5];
      b1[2] = o[6];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) x[a * n + p] = x1[a];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      cache[c * n + p] = v3[c];
      cache[(3 + c) * n + p] = b1[c];
    }
    if (outmask) outmask[p] = outside_open(g, x1);
    const double bb0 = fma(b0[2], b0[2], fma(b0[1], b0[1], b0[0] * b0[0]));
    const double bb1 = fma(b1[2], b1[2], fma(b1[1], b1[1], b1[0] * b1[0]));
    const double vv = fma(v3[2], v3[2], fma(v3[1], v3[1], v3[0] * v3[0]));
    const double igam = sqrt(1.0 - vv);  // 1/gamma_g: d tau = dt / gamma_g = dt * igam
    s3[0] = r;
    s3[1] = 0.5 * (bb0 + bb1);
    s3[2] = igam;
    if (!(fin && s1.finite && igam > 0.0 && isfinite(r) && r > 0.0))
      atomicOr(status, ST_NONFINITE);
    if (SHOCK) shock_mark(p, s1.cell, A.shock_r, A.shock_q, A.shk, A.list, A.rs, A.qs);
  }
};

// Two CTAs per SM (128 registers): the x-quadratic gathers take more
// registers than one CTA per SM can hide the FP64 latency with.
template <int SHAPE, int DIM, bool SHOCK, int ORDER, bool CACHED>
__global__ void __launch_bounds__(256, 2)
    k_lp_rk2(const LpArgs a, double* __restrict__ samples, int64_t p0, int64_t p1) {
  const PushF64<SHAPE, DIM, SHOCK, ORDER, CACHED> push{a};
  for (int64_t p = p0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < p1;
       p += (int64_t)gridDim.x * blockDim.x) {
    double s3[3], s4[4];
    push(p, s3);
    lp_samples(a.n_old[p], s3[0], s3[1], s3[2], s4);
#pragma unroll
    for (int k = 0; k < 4; ++k) samples[k * a.n + p] = s4[k];
  }
}

// The spectral update (spec_lp) of LPs [p0, p1) from the samples [4][n] the
// last push left.
template <bool FROM_PLAIN>
__global__ void __launch_bounds__(256)
    k_spec_update(double* __restrict__ chi, double* __restrict__ eng, double* __restrict__ n_old,
                  const double* __restrict__ samples, int64_t n, int nb, double dt, double c0,
                  double u_rad, int* __restrict__ status, int64_t p0, int64_t p1) {
  for (int64_t p = p0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < p1;
       p += (int64_t)gridDim.x * blockDim.x) {
    double s4[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) s4[k] = samples[k * n + p];
    spec_lp<FROM_PLAIN>(SpecArgs{chi, eng, n_old, nb, dt, c0, u_rad}, p, n, s4, status);
  }
}

// Back from (y, psi) to (chi, eps): eps = 1/y, chi = psi y^2; one thread
// per LP, eight bins per batch inversion.
__global__ void __launch_bounds__(256)
    k_spec_to_plain(double* __restrict__ chi, double* __restrict__ eng, int64_t n, int nb) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    double* ep = eng + p;
    double* cp = chi + p;
    int i = 0;
    for (; i + 8 <= nb; i += 8) {
      double y[8], ps[8], r[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        y[k] = ep[(int64_t)(i + k) * n];
        ps[k] = cp[(int64_t)(i + k) * n];
      }
      recip8(y, r);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        ep[(int64_t)(i + k) * n] = r[k];
        cp[(int64_t)(i + k) * n] = (ps[k] * y[k]) * y[k];
      }
    }
    for (; i < nb; ++i) {
      const double y = ep[(int64_t)i * n], ps = cp[(int64_t)i * n];
      ep[(int64_t)i * n] = __drcp_rn(y);
      cp[(int64_t)i * n] = (ps * y) * y;
    }
  }
}

template <int SHAPE, int DIM, int ORDER, bool CACHED>
cudaError_t lp_launch_range(part_ctx* c, double dt, const LpLaunch& L) {
  const LpArgs a = lp_args(c, dt);
  if (c->shk)
    k_lp_rk2<SHAPE, DIM, true, ORDER, CACHED><<<L.grid, 256, 0, L.stream>>>(a, c->samples, L.p0,
                                                                           L.p1);
  else
    k_lp_rk2<SHAPE, DIM, false, ORDER, CACHED><<<L.grid, 256, 0, L.stream>>>(a, c->samples,
                                                                            L.p0, L.p1);
  c->launches++;
  return cudaGetLastError();
}

template <int SHAPE, int DIM>
cudaError_t lp_launch(part_ctx* c, double dt, const LpLaunch& L) {
  if (c->lp_order == 3)
    return L.cached ? lp_launch_range<SHAPE, DIM, 3, true>(c, dt, L)
                    : lp_launch_range<SHAPE, DIM, 3, false>(c, dt, L);
  return L.cached ? lp_launch_range<SHAPE, DIM, 2, true>(c, dt, L)
                  : lp_launch_range<SHAPE, DIM, 2, false>(c, dt, L);
}

// Shock cells from the padded fields (periodic ghost layer of one cell):
// along each axis a < dim, a converging flow across the cell (v_a(+1) -
// v_a(-1) < 0) with neighbour density ratio max/min >= r_min marks it; the
// cell keeps the largest such ratio r (the first axis reaching it), 0 if
// none, and the index q of Eq. slope: 3r/(r-1), or with REL the relativistic
// index of Keshet & Waxman (2005) from the shock-frame normal speeds of the
// lower-density (upstream) and denser (downstream) neighbours along that
// axis.  The shock frame moves at the speed that conserves the lab-frame
// mass D = rho/sqrt(1 - |v|^2) across the front (c = 1):
// v_sh = (D_d v_d - D_u v_u)/(D_d - D_u); there the normal speeds are
// |v - v_sh|/(1 - v v_sh).  Where no such frame exists (a speed >= 1,
// D_d = D_u, |v_sh| >= 1, no slowdown) q stays 3r/(r-1).
__device__ __forceinline__ bool shock_frame_speeds(double vu, double s2u, double rhou, double vd,
                                                   double s2d, double rhod, double& bu,
                                                   double& bd) {
  if (!(s2u < 1.0 && s2d < 1.0)) return false;
  const double Du = rhou / sqrt(1.0 - s2u), Dd = rhod / sqrt(1.0 - s2d);
  if (!(Dd != Du)) return false;
  const double vsh = (Dd * vd - Du * vu) / (Dd - Du);
  if (!(fabs(vsh) < 1.0)) return false;
  bu = fabs((vu - vsh) / (1.0 - vu * vsh));
  bd = fabs((vd - vsh) / (1.0 - vd * vsh));
  return bd < bu;
}

template <bool REL>
__global__ void k_shock_cells(const double* __restrict__ fp, const Geo g, double r_min,
                              double* __restrict__ r_cell, double* __restrict__ q_cell) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < g.G;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int jx = (int)(c % g.n[0]);
    const int jy = (int)((c / g.n[0]) % g.n[1]);
    const int jz = (int)(c / ((int64_t)g.n[0] * g.n[1]));
    const int64_t q = ((int64_t)(jz + g.h[2]) * g.pn[1] + (jy + g.h[1])) * g.pn[0] + (jx + g.h[0]);
    double best = 0.0;
    int axis = -1;
    int64_t up = 0, down = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a >= g.dim) break;
      const int64_t st = a == 0 ? 1 : a == 1 ? (int64_t)g.pn[0] : (int64_t)g.pn[0] * g.pn[1];
      const double dv = fp[a * g.pplane + q + st] - fp[a * g.pplane + q - st];
      if (dv < 0.0) {
        const double rp = fp[3 * g.pplane + q + st], rm = fp[3 * g.pplane + q - st];
        const double hi = rp > rm ? rp : rm, lo = rp > rm ? rm : rp;
        const double ratio = hi / lo;
        if (ratio > best) {
          best = ratio;
          axis = a;
          down = rp > rm ? q + st : q - st;
          up = rp > rm ? q - st : q + st;
        }
      }
    }
    const bool shock = best >= r_min;
    double qi = 0.0;
    if (shock) {
      qi = 3.0 * best / (best - 1.0);
      if (REL) {
        double s2u = 0.0, s2d = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const double vu = fp[a * g.pplane + up], vd = fp[a * g.pplane + down];
          s2u += vu * vu;
          s2d += vd * vd;
        }
        double bu, bd;
        if (shock_frame_speeds(fp[axis * g.pplane + up], s2u, fp[3 * g.pplane + up],
                               fp[axis * g.pplane + down], s2d, fp[3 * g.pplane + down], bu, bd))
          qi = (3.0 * bu - 2.0 * bu * bd * bd + bd * bd * bd) / (bu - bd);
      }
    }
    r_cell[c] = shock ? best : 0.0;
    q_cell[c] = qi;
  }
}

// Eq. convolution_spectra for each listed LP, one warp per LP, so only
// shocked LPs do the work and a few thousand of them still fill the GPU.
// With chi_in the power law through adjacent bin values, the kernel
// (eps_i/e)^(2-q) separates: chi_out_i = cn S_i / w_i, w = eps^(q-2),
// S_i = sum_{j<=i} dln eps_j h_{j-1} expm1(d_j)/d_j, h = chi w,
// d_j = ln(h_j/h_{j-1}) -- a prefix sum over the bins: each lane takes 4
// consecutive bins of a 128-bin tile, sums them, and a warp scan (shuffles)
// adds the lanes before it; tiles carry their last bin and running sum.
// q from the LP's shock cell (Eq. slope, with or without q_R), cn = q/r (for
// a non-relativistic shock: particle number per unit fluid density conserved
// across the jump).
// FORM: how the bound arrays hold the spectra -- 0 (chi, eps); 1 (y, psi) =
// (1/eps, chi eps^2); 2 the deferred form (chi0, eps0) with the LP's map
// smap = (alpha, beta, S), where eps = eps0/t and chi = S chi0 t^2 with
// t = alpha + beta eps0: the LP's bins are written back as (chi, eps) and
// its map reset to the identity.
template <int FORM>
__global__ void __launch_bounds__(256)
    k_shock_convolve(const uint32_t* __restrict__ list, const double* __restrict__ rs,
                     const double* __restrict__ qs, double* __restrict__ chi,
                     double* __restrict__ eng, double* __restrict__ smap, int64_t n, int nb,
                     int* __restrict__ status) {
  constexpr bool INV = FORM == 1;
  constexpr int K = 4;
  const uint32_t cnt = list[0];
  const int lane = threadIdx.x & 31;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < cnt; t += warps) {
    const int64_t p = list[1 + t];
    const double r = rs[t];
    const double q = qs[t];
    const double cn = q / r;
    const double qm2 = q - 2.0;
    double cS = 0.0, cE = 0.0, cL = 0.0, cH = 0.0;  // carry: running sum, last bin
    bool ok = true;
    double al = 1.0, be = 0.0, sc = 1.0;  // FORM 2: the LP's pending map
    if (FORM == 2) {
      al = smap[p];
      be = smap[n + p];
      sc = smap[2 * n + p];
    }
    for (int t0 = 0; t0 < nb; t0 += 32 * K) {
      double e[K], le[K], w[K], h[K], S[K];
#pragma unroll
      for (int i = 0; i < K; ++i) {
        const int j = t0 + lane * K + i;
        // INV: the arrays hold y = 1/eps and psi = chi eps^2 (see k_spec_update)
        const double ev = j < nb ? eng[(int64_t)j * n + p] : 1.0;
        double c = j < nb ? chi[(int64_t)j * n + p] : 0.0;
        e[i] = INV ? __drcp_rn(ev) : ev;
        if (INV) c = (c * ev) * ev;
        if (FORM == 2 && j < nb) {
          const double tt = fma(be, ev, al);
          e[i] = ev / tt;
          c = (sc * c) * (tt * tt);
        }
        le[i] = log(e[i]);
        w[i] = exp(qm2 * le[i]);
        h[i] = c * w[i];
      }
      // the bin before this lane's first: the previous lane's last, or the carry
      double pe = __shfl_up_sync(0xffffffffu, e[K - 1], 1);
      double pl = __shfl_up_sync(0xffffffffu, le[K - 1], 1);
      double ph = __shfl_up_sync(0xffffffffu, h[K - 1], 1);
      if (lane == 0) {
        pe = cE;
        pl = cL;
        ph = cH;
      }
      double run = 0.0;
#pragma unroll
      for (int i = 0; i < K; ++i) {
        const int j = t0 + lane * K + i;
        double seg = 0.0;
        if (j >= 1 && j < nb && ph > 0.0 && h[i] > 0.0 && e[i] > pe) {
          const double d = log(h[i] / ph);
          const double D = le[i] - pl;
          seg = d == 0.0 ? D * ph : D * ph * (expm1(d) / d);
        }
        run += seg;
        S[i] = run;
        pe = e[i];
        pl = le[i];
        ph = h[i];
      }
      // prefix of the lane totals; the exclusive one is the previous lane's
      // inclusive value (not incl - run: h can grow by orders of magnitude
      // from bin to bin, and that difference would cancel)
      double incl = run;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const double v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      double excl = __shfl_up_sync(0xffffffffu, incl, 1);
      if (lane == 0) excl = 0.0;
      const double before = cS + excl;
#pragma unroll
      for (int i = 0; i < K; ++i) {
        const int j = t0 + lane * K + i;
        if (j < nb) {
          const double out = j == 0 ? 0.0 : cn * ((before + S[i]) / w[i]);
          ok = ok && isfinite(out);
          chi[(int64_t)j * n + p] = INV ? (out * e[i]) * e[i] : out;
          if (FORM == 2) eng[(int64_t)j * n + p] = e[i];
        }
      }
      cS = __shfl_sync(0xffffffffu, cS + incl, 31);
      cE = __shfl_sync(0xffffffffu, e[K - 1], 31);
      cL = __shfl_sync(0xffffffffu, le[K - 1], 31);
      cH = __shfl_sync(0xffffffffu, h[K - 1], 31);
    }
    if (!ok) atomicOr(status, ST_NONFINITE);
    if (FORM == 2 && lane == 0) {  // the bins now hold the LP's spectrum as it is
      smap[p] = 1.0;
      smap[n + p] = 0.0;
      smap[2 * n + p] = 1.0;
    }
  }
}

// The deferred form of the spectral update (part_set_spec_lazy): the bins
// stay as they were at the last materialisation, (chi0, eps0), and each LP
// carries the composition of its steps' maps in y = 1/eps and psi = chi eps^2,
// y = alpha y0 + beta, psi = S psi0; a step (coefficients A, C as in
// k_spec_update) composes one more: alpha <- A alpha, beta <- A beta + C,
// S <- S / A.  O(1) per LP instead of O(N_b).  FIRST: no map pending (the
// identity).
template <bool FIRST>
__global__ void __launch_bounds__(256)
    k_spec_lazy(const SpecArgs sa, const double* __restrict__ samples, double* __restrict__ smap,
                int64_t n, int* __restrict__ status) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const SpecCoef k = spec_coeffs(sa, samples[n + p], samples[2 * n + p], samples[3 * n + p],
                                   status);
    double al = 1.0, be = 0.0, sc = 1.0;
    if (!FIRST) {
      al = smap[p];
      be = smap[n + p];
      sc = smap[2 * n + p];
    }
    smap[p] = k.A * al;
    smap[n + p] = fma(k.A, be, k.C);
    smap[2 * n + p] = sc * k.iA;
    sa.n_old[p] = samples[p];
  }
}

// Materialise the deferred form: every LP's map applied to its bins, with
// t = alpha + beta eps0: eps = eps0 / t, chi = S chi0 t^2 (eight reciprocals
// at a time by recip8).  The maps become the identity (implicitly).
__global__ void __launch_bounds__(256)
    k_spec_apply(double* __restrict__ chi, double* __restrict__ eng,
                 const double* __restrict__ smap, int64_t n, int nb) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const double al = smap[p], be = smap[n + p], sc = smap[2 * n + p];
    double* ep = eng + p;
    double* cp = chi + p;
    int i = 0;
    for (; i + 8 <= nb; i += 8) {
      double e0[8], c0[8], t[8], r[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        e0[k] = ep[(int64_t)(i + k) * n];
        c0[k] = cp[(int64_t)(i + k) * n];
        t[k] = fma(be, e0[k], al);
      }
      recip8(t, r);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        ep[(int64_t)(i + k) * n] = e0[k] * r[k];
        cp[(int64_t)(i + k) * n] = (sc * c0[k]) * (t[k] * t[k]);
      }
    }
    for (; i < nb; ++i) {
      const double e0 = ep[(int64_t)i * n], c0 = cp[(int64_t)i * n];
      const double t = fma(be, e0, al);
      ep[(int64_t)i * n] = e0 * __drcp_rn(t);
      cp[(int64_t)i * n] = (sc * c0) * (t * t);
    }
  }
}

}  // namespace

cudaError_t launch_lp_push_range(part_ctx* c, double dt, const LpLaunch& L) {
  if (L.p1 <= L.p0) return cudaSuccess;
  if (c->shape == PART_TSC)
    return c->geo.dim == 3 ? lp_launch<PART_TSC, 3>(c, dt, L) : lp_launch<PART_TSC, 2>(c, dt, L);
  return c->geo.dim == 3 ? lp_launch<PART_CIC, 3>(c, dt, L) : lp_launch<PART_CIC, 2>(c, dt, L);
}

cudaError_t launch_lp_push(part_ctx* c, double dt, int nsteps) {
  (void)nsteps;
  if (c->n == 0) return cudaSuccess;
  if (c->shk) {
    cudaError_t e = cudaMemsetAsync(c->shock_list, 0, sizeof(uint32_t), c->stream);
    if (e != cudaSuccess) return e;
  }
  const LpLaunch L{0, c->n, grid_for(c, c->n, 256), c->stream, c->lp_cache_ok};
  cudaError_t e = c->lp_paired ? launch_lp_push_pair_range(c, dt, L)
                               : launch_lp_push_range(c, dt, L);
  if (e == cudaSuccess) {
    c->lp_cache_ok = true;
  }
  return e;
}

cudaError_t launch_shock_cells(part_ctx* c) {
  if (c->shock_rel)
    k_shock_cells<true><<<grid_for(c, c->geo.G, 256), 256, 0, c->stream>>>(
        (const double*)c->fpad, c->geo, c->r_min, c->shock_r, c->shock_q);
  else
    k_shock_cells<false><<<grid_for(c, c->geo.G, 256), 256, 0, c->stream>>>(
        (const double*)c->fpad, c->geo, c->r_min, c->shock_r, c->shock_q);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_shock_convolve(part_ctx* c) {
  if (c->n == 0) return cudaSuccess;
  int64_t b = (c->n + 7) / 8;            // 8 warps (LPs) per block
  if (b > (int64_t)c->sms * 16) b = (int64_t)c->sms * 16;
  auto go = [&](auto kern) {
    kern<<<(unsigned)b, 256, 0, c->stream>>>(c->shock_list, c->shock_rs, c->shock_qs, c->chi,
                                             c->eng, c->smap, c->n, c->nbins, c->status);
  };
  if (c->maps_pending) go(k_shock_convolve<2>);
  else if (c->spec_inv) go(k_shock_convolve<1>);
  else go(k_shock_convolve<0>);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_spec_range(part_ctx* c, double dt, double c0, double u_rad, bool from_plain,
                              const LpLaunch& L) {
  if (L.p1 <= L.p0) return cudaSuccess;
  auto go = [&](auto kern) {
    kern<<<L.grid, 256, 0, L.stream>>>(c->chi, c->eng, c->n_old, c->samples, c->n, c->nbins, dt,
                                       c0, u_rad, c->status, L.p0, L.p1);
  };
  if (from_plain)
    go(k_spec_update<true>);
  else
    go(k_spec_update<false>);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_spec_update(part_ctx* c, double dt, double c0, double u_rad) {
  if (c->n == 0) return cudaSuccess;
  const int gb = grid_for(c, c->n, 256);
  if (c->spec_lazy) {  // the deferred form: compose the step into each LP's map
    const SpecArgs sa{c->chi, c->eng, c->n_old, c->nbins, dt, c0, u_rad};
    auto go = [&](auto kern) {
      kern<<<gb, 256, 0, c->stream>>>(sa, c->samples, c->smap, c->n, c->status);
    };
    if (c->maps_pending)
      go(k_spec_lazy<false>);
    else
      go(k_spec_lazy<true>);
    c->launches++;
    c->maps_pending = true;
    return cudaGetLastError();
  }
  const LpLaunch L{0, c->n, gb, c->stream, false};
  cudaError_t e = launch_spec_range(c, dt, c0, u_rad, !c->spec_inv, L);
  if (e == cudaSuccess) c->spec_inv = true;
  return e;
}

cudaError_t launch_spec_to_plain(part_ctx* c) {
  if (c->maps_pending) {  // the deferred form: apply the maps
    c->maps_pending = false;
    if (c->n > 0 && c->nbins > 0) {
      k_spec_apply<<<grid_for(c, c->n, 256), 256, 0, c->stream>>>(c->chi, c->eng, c->smap, c->n,
                                                                  c->nbins);
      c->launches++;
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  if (!c->spec_inv) return cudaSuccess;
  c->spec_inv = false;
  if (c->n == 0 || c->nbins == 0) return cudaSuccess;
  k_spec_to_plain<<<grid_for(c, c->n, 256), 256, 0, c->stream>>>(c->chi, c->eng, c->n, c->nbins);
  c->launches++;
  return cudaGetLastError();
}

// Gather of one scalar component, used by the LP initialisation.
template <int SHAPE, int DIM>
__global__ void k_lp_sample_rho(const double* __restrict__ fp, const double* __restrict__ fxq,
                                const Geo g, const double* __restrict__ x, int64_t n,
                                double* __restrict__ n_old) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    double xp[3] = {x[p], x[n + p], x[2 * n + p]};
    Stencil<SHAPE, DIM> s(g, xp);
    double r;
    s.template gather_lp<1>(fp, fxq, g, 3, &r);  // as the push samples rho
    n_old[p] = r;
  }
}

cudaError_t launch_lp_sample_rho(part_ctx* c) {
  if (c->n == 0) return cudaSuccess;
  const int gb = grid_for(c, c->n, 256);
  const double* fp = (const double*)c->fpad;
  const double* x = (const double*)c->x;
  if (c->shape == PART_TSC) {
    if (c->geo.dim == 3)
      k_lp_sample_rho<PART_TSC, 3><<<gb, 256, 0, c->stream>>>(fp, c->fxq, c->geo, x, c->n, c->n_old);
    else
      k_lp_sample_rho<PART_TSC, 2><<<gb, 256, 0, c->stream>>>(fp, c->fxq, c->geo, x, c->n, c->n_old);
  } else {
    if (c->geo.dim == 3)
      k_lp_sample_rho<PART_CIC, 3><<<gb, 256, 0, c->stream>>>(fp, c->fxq, c->geo, x, c->n, c->n_old);
    else
      k_lp_sample_rho<PART_CIC, 2><<<gb, 256, 0, c->stream>>>(fp, c->fxq, c->geo, x, c->n, c->n_old);
  }
  c->launches++;
  return cudaGetLastError();
}
