// lp_spec.cuh -- the arguments of the LP kernels and the per-LP spectral
// update of Eq. cr_chi.
#pragma once
#include "part_internal.cuh"

// r[k] = 1/v[k] for eight values by Montgomery's simultaneous inversion:
// prefix products, one correctly rounded reciprocal, then unwinding (three
// multiplies per value instead of a reciprocal each).  Products that leave
// the double range fall back to eight reciprocals.
static __device__ __forceinline__ void recip8(const double* v, double* r) {
  double pre[8];
  pre[0] = v[0];
#pragma unroll
  for (int k = 1; k < 8; ++k) pre[k] = pre[k - 1] * v[k];
  double inv = __drcp_rn(pre[7]);
  if (finite_bits(inv) && inv != 0.0 && finite_bits(pre[7]) && pre[7] != 0.0) {
#pragma unroll
    for (int k = 7; k > 0; --k) {
      r[k] = inv * pre[k - 1];
      inv = inv * v[k];
    }
    r[0] = inv;
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) r[k] = __drcp_rn(v[k]);
  }
}

// Everything an LP push reads and writes (the bound LPs, the fields, the
// shock bookkeeping); fp: the padded FP64 fields, or the paired copy.
struct LpArgs {
  const double* fp;
  Geo g;
  double* x;
  int64_t n;
  double dt;
  int* status;
  const double* shock_r;
  const double* shock_q;
  uint8_t* shk;
  uint32_t* list;
  double* rs;
  double* qs;
  uint8_t* outmask;
  double* cache;
};

// The push arguments of a context (fp: the FP64 padded fields).
static inline LpArgs lp_args(part_ctx* c, double dt) {
  LpArgs a;
  a.fp = (const double*)c->fpad;
  a.g = c->geo;
  a.x = (double*)c->x;
  a.n = c->n;
  a.dt = dt;
  a.status = c->status;
  a.shock_r = c->shock_r;
  a.shock_q = c->shock_q;
  a.shk = c->shk;
  a.list = c->shock_list;
  a.rs = c->shock_rs;
  a.qs = c->shock_qs;
  a.outmask = c->outmask;
  a.cache = c->lpcache;
  return a;
}

struct SpecArgs {
  double* chi;
  double* eng;
  double* n_old;
  int nb;
  double dt, c0, u_rad;
};

// Eq. cr_chi along exact characteristics for LP p, in the variables the step
// is linear in: y = 1/eps and psi = chi eps^2.  With a3 and c_r frozen over
// the step, dy/dtau = a3 y + c_r gives y1 = A y0 + C, A = exp(a3 dtau) =
// (n_old/n_new)^(1/3), C = c_r dtau expm1(a3 dtau)/(a3 dtau); number
// conservation along the characteristic (chi deps fixed) gives
// chi1 = chi0 (y1/y0)^2 / A, i.e. psi1 = psi0 / A.  Per bin that is one FMA
// and one multiply, so the pass is bound by HBM instead of the FP64 rate.
// FROM_PLAIN: the arrays still hold chi and eps (first update since they
// were bound, initialised or brought back) and are converted on the way.
// nn, b2, igam: the push's samples (density, <|B|^2>, 1/gamma_g at the new
// position); dtau = dt / gamma_g.  Spectra are bin-major [nb][n].
// The step's coefficients for LP p: y1 = A y0 + C, psi1 = psi0 iA, iA = 1/A.
struct SpecCoef {
  double A, C, iA;
};
static __device__ __forceinline__ SpecCoef spec_coeffs(const SpecArgs& a, int64_t p, double nn,
                                                       double b2, double igam,
                                                       int* __restrict__ status) {
  const double dtau = a.dt * igam;
  const double L = log(a.n_old[p] / nn) * (1.0 / 3.0);  // a3 dtau
  const double em = expm1(L);                            // A - 1, no cancellation
  SpecCoef k;
  k.A = 1.0 + em;
  k.iA = __drcp_rn(k.A);
  const double cr = a.c0 * (0.5 * b2 + a.u_rad);
  k.C = cr * dtau * (L == 0.0 ? 1.0 : em / L);
  if (!(isfinite(k.A) && k.A > 0.0 && isfinite(k.C) && isfinite(k.iA)))
    atomicOr(status, ST_NONFINITE);
  return k;
}

template <bool FROM_PLAIN>
static __device__ __forceinline__ void spec_lp(const SpecArgs& a, int64_t p, int64_t n,
                                               double nn, double b2, double igam,
                                               int* __restrict__ status) {
  const SpecCoef kc = spec_coeffs(a, p, nn, b2, igam, status);
  const double A = kc.A, C = kc.C, iA = kc.iA;
  double* ep = a.eng + p;
  double* cp = a.chi + p;
  const int nb = a.nb;
  int i = 0;
  for (; i + 8 <= nb; i += 8) {  // eight rows' loads in flight per thread
    double y[8], ps[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      y[k] = ep[(int64_t)(i + k) * n];
      ps[k] = cp[(int64_t)(i + k) * n];
    }
    if (FROM_PLAIN) {  // y[] holds eps: psi = chi eps^2, y = 1/eps
      double r[8];
      recip8(y, r);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        ps[k] = (ps[k] * y[k]) * y[k];
        y[k] = r[k];
      }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      ep[(int64_t)(i + k) * n] = fma(A, y[k], C);
      cp[(int64_t)(i + k) * n] = ps[k] * iA;
    }
  }
  for (; i < nb; ++i) {
    double y = ep[(int64_t)i * n], ps = cp[(int64_t)i * n];
    if (FROM_PLAIN) {
      ps = (ps * y) * y;
      y = __drcp_rn(y);
    }
    ep[(int64_t)i * n] = fma(A, y, C);
    cp[(int64_t)i * n] = ps * iA;
  }
  a.n_old[p] = nn;
}

