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
  const double* fxq;  // x quadratics of fp (TSC gathers), 4 doubles per (component, cell)
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
  const double* n_old;  // n at the old positions, for the samples
};

// The push arguments of a context (fp: the FP64 padded fields).
static inline LpArgs lp_args(part_ctx* c, double dt) {
  LpArgs a;
  a.fp = (const double*)c->fpad;
  a.fxq = c->fxq;
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
  a.n_old = c->n_old;
  return a;
}

struct SpecArgs {
  double* chi;
  double* eng;
  double* n_old;
  int nb;
  double dt, c0, u_rad;
};

// The samples an LP push leaves for spec_update ([4][n] doubles): the
// density n_new at the new position, <|B|^2>, and the step's factors that do
// not depend on spec_update's arguments, em = A - 1 and
// G = (1/gamma_g) expm1(L)/L (1/gamma_g at L = 0), L = a3 dtau =
// ln(n_old/n_new)/3, A = exp(L).  The transcendental functions run in the
// push kernels, whose FP64 pipe has room (the paired push is bound by the
// f32 pipes); the spectral update only combines them with dt, c0, u_rad.
// With u = n_old/n_new - 1, em = (1 + u)^(1/3) - 1 and
// expm1(L)/L = em / (ln(1 + u)/3); for |u| < 1/16 (a step's density change
// is small) both come from their Taylor series in u, 13 terms each (the
// truncation is below 1e-18 relative there): kLpA are the binomial
// coefficients C(1/3, k), k = 1..13, kLpB the series of the ratio, from
// u^0 to u^12.  Elsewhere log and expm1.
__device__ __constant__ static const double kLpA[13] = {
    1.0 / 3, -1.0 / 9, 5.0 / 81, -10.0 / 243, 22.0 / 729, -154.0 / 6561, 374.0 / 19683,
    -935.0 / 59049, 21505.0 / 1594323, -55913.0 / 4782969, 147407.0 / 14348907,
    -1179256.0 / 129140163, 3174920.0 / 387420489};
__device__ __constant__ static const double kLpB[13] = {
    1.0, 1.0 / 6, -7.0 / 108, 25.0 / 648, -523.0 / 19440, 7139.0 / 349920,
    -239543.0 / 14696640, 1189813.0 / 88179840, -38985989.0 / 3401222400.0,
    1418545769.0 / 142851340800.0, -16473859861.0 / 1885637698560.0,
    1320722958449.0 / 169707392870400.0, -3244822448357701.0 / 463301182536192000.0};

static __device__ __forceinline__ void lp_samples(double n_old, double nn, double b2,
                                                  double igam, double* s4) {
  const double u = (n_old - nn) / nn;
  double em, h;
  if (fabs(u) < 0.0625) {
    double pa = kLpA[12], pb = kLpB[12];
#pragma unroll
    for (int k = 11; k >= 0; --k) {
      pa = fma(pa, u, kLpA[k]);
      pb = fma(pb, u, kLpB[k]);
    }
    em = u * pa;
    h = pb;
  } else {
    const double L = log(n_old / nn) * (1.0 / 3.0);
    em = expm1(L);  // A - 1, no cancellation
    h = L == 0.0 ? 1.0 : em / L;
  }
  s4[0] = nn;
  s4[1] = b2;
  s4[2] = em;
  s4[3] = igam * h;
}

// The step's coefficients: y1 = A y0 + C, psi1 = psi0 iA, iA = 1/A, with
// dtau = dt / gamma_g and C = c_r dtau expm1(L)/L = c_r dt G.
struct SpecCoef {
  double A, C, iA;
};
static __device__ __forceinline__ SpecCoef spec_coeffs(const SpecArgs& a, double b2, double em,
                                                       double G, int* __restrict__ status) {
  SpecCoef k;
  k.A = 1.0 + em;
  k.iA = __drcp_rn(k.A);
  const double cr = a.c0 * (0.5 * b2 + a.u_rad);
  k.C = (cr * a.dt) * G;
  if (!(isfinite(k.A) && k.A > 0.0 && isfinite(k.C) && isfinite(k.iA)))
    atomicOr(status, ST_NONFINITE);
  return k;
}

// Eq. cr_chi along exact characteristics for LP p, in the variables the step
// is linear in: y = 1/eps and psi = chi eps^2.  With a3 and c_r frozen over
// the step, dy/dtau = a3 y + c_r gives y1 = A y0 + C, A = exp(a3 dtau) =
// (n_old/n_new)^(1/3), C = c_r dtau expm1(a3 dtau)/(a3 dtau); number
// conservation along the characteristic (chi deps fixed) gives
// chi1 = chi0 (y1/y0)^2 / A, i.e. psi1 = psi0 / A.  Per bin that is one FMA
// and one multiply and 32 bytes moved: on B300 the pass keeps both the FP64
// pipe and HBM busy (measured: FP64 pipe ~74%, DRAM ~0.87 of a copy).
// FROM_PLAIN: the arrays still hold chi and eps (first update since they
// were bound, initialised or brought back) and are converted on the way.
// s4: the push's samples (lp_samples).  Spectra are bin-major [nb][n].
template <bool FROM_PLAIN>
static __device__ __forceinline__ void spec_lp(const SpecArgs& a, int64_t p, int64_t n,
                                               const double* s4, int* __restrict__ status) {
  const SpecCoef kc = spec_coeffs(a, s4[1], s4[2], s4[3], status);
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
  a.n_old[p] = s4[0];
}

