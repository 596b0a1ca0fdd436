// push_boris.cu -- gather + relativistic Boris push (+ fused force deposit).
//
// Brick kernel (sorted particles, one CTA per 8x8x8 / 16x16 cell brick;
// with the deposit, warp-specialised: 8 push warps, 8 deposit warps):
//   1. CIC: one thread issues a 4-D TMA copy of the brick's haloed field box
//      (all components) into shared memory.  TSC: nothing is staged; each
//      stencil row of each component is one 32-byte record (q0, q1, q2) of
//      the fields' x quadratics, read through L1, and the row's three
//      weighted cells are q0 + d (q1 + d q2).  cell_start of the brick is read;
//   2. the CTA walks the brick's particles in chunks of blockDim: weights,
//      gather, Boris kick, drift, periodic wrap, coalesced SoA loads/stores;
//   3. deposit (optional): each particle leaves its weights and force in
//      shared memory; then warp w takes the chunk's source cells with x index
//      w mod 8, one lane per stencil offset: every lane loops over the same
//      particles (no divergence) and adds into the warp's private window of
//      haloed-tile columns, in a fixed order.  No atomics;
//   4. the windows are combined in warp order into the brick's haloed tile,
//      written as this brick's partial; a second kernel
//      adds, per grid cell, the partials of the bricks covering it in fixed
//      order.  The result is bitwise reproducible.
// Particle-order kernel (any order, no deposit): nsteps fused steps with the
// state in registers and the stencil read from the padded global copy.
#include "part_internal.cuh"

namespace {

constexpr int kT = kPushThreads;

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Shared-memory carve of the brick kernel.
constexpr int kRS = kT + 1;      // record row stride (doubles): odd, so rows hit other banks
constexpr int kWarps = kT / 32;

// Deposit windows: warp w owns the source cells whose x index is w mod 8, so
// its targets lie in the ext-tile columns w..w+2 (and w+8..w+10 for 16-wide
// 2D bricks): kSlots(DIM) columns x e1 x e2 targets x 3 components.
__host__ __device__ constexpr int kslots(int dim) { return dim == 3 ? 3 : 6; }

struct BrickSmem {
  size_t box, cs, bar, rec, win, total;
};
// dep: two record buffers [2][18][kRS] and the deposit windows follow the box
__host__ __device__ inline BrickSmem brick_smem(const Geo& g, int ncomp, int esize, bool dep) {
  BrickSmem s;
  s.box = 0;
  size_t bbytes = (size_t)ncomp * g.box[0] * g.box[1] * g.box[2] * esize;
  s.cs = align_up(bbytes, 128);
  s.bar = align_up(s.cs + (size_t)(g.V + 1) * 4, 16);
  s.rec = align_up(s.bar + 16, 128);
  s.win = align_up(s.rec + (dep ? (size_t)2 * 18 * kRS * 8 : 0), 128);
  s.total = s.win + (dep ? (size_t)kWarps * kslots(g.dim) * g.e[1] * g.e[2] * 3 * 8 : 0);
  return s;
}

__device__ __forceinline__ double wrap_axis(double v, double lo, double hi, double L) {
  if (v < lo) v = v + L;
  else if (v >= hi) v = v - L;
  return v;
}

// 1 + |v|^2 as three FMAs
__device__ __forceinline__ double one_plus_norm2(double a, double b, double c) {
  return fma(c, c, fma(b, b, fma(a, a, 1.0)));
}

// Relativistic Boris kick (c = 1): half E kick, rotation about B with
// t = h B / gamma-, s = 2t/(1+t^2), half E kick; h = (q/m) dt / 2.
__device__ __forceinline__ void boris_f64(double* u, const double* E, const double* B, double h) {
  double um0 = u[0] + h * E[0], um1 = u[1] + h * E[1], um2 = u[2] + h * E[2];
  double gi = rsqrt(one_plus_norm2(um0, um1, um2));
  double hg = h * gi;
  double t0 = hg * B[0], t1 = hg * B[1], t2 = hg * B[2];
  // 2/x = 2 * rn(1/x) exactly (scaling by two is exact): the reciprocal
  // alone, not a general division
  double sf = 2.0 * __drcp_rn(one_plus_norm2(t0, t1, t2));
  double s0 = sf * t0, s1 = sf * t1, s2 = sf * t2;
  // u' = u- + u- x t and u+ = u- + u' x s, each component as two FMAs
  double p0 = fma(um1, t2, fma(-um2, t1, um0));
  double p1 = fma(um2, t0, fma(-um0, t2, um1));
  double p2 = fma(um0, t1, fma(-um1, t0, um2));
  double q0 = fma(p1, s2, fma(-p2, s1, um0));
  double q1 = fma(p2, s0, fma(-p0, s2, um1));
  double q2 = fma(p0, s1, fma(-p1, s0, um2));
  u[0] = q0 + h * E[0];
  u[1] = q1 + h * E[1];
  u[2] = q2 + h * E[2];
}

// ---------------------------------------------------------------- brick kernel, FP64
// One particle of a chunk: weights, gather from the staged box, Boris, drift,
// wrap, store; with DEP, its deposit record (9 z-y weight products and the 9
// x-weighted force terms) is returned in wyz / fxc (zero if it has none).
struct PState64 {
  double x[3], u[3], w;
  uint64_t id;
};
__device__ __forceinline__ void load_state64(PState64& s, uint32_t q, const double* xs,
                                             const double* us, const double* ws,
                                             const uint64_t* ids, int64_t n) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    s.x[a] = xs[a * n + q];
    s.u[a] = us[a * n + q];
  }
  s.w = ws ? ws[q] : 1.0;
  s.id = ids ? ids[q] : 0ull;
}

template <int SHAPE, int DIM, bool DEP, bool OPEN, bool XQ>
__device__ __forceinline__ void push_one(const Geo& g, const double* sbox, int bvol,
                                         const double* __restrict__ fxq,
                                         const uint32_t* scs, const int* org, uint32_t p,
                                         uint32_t q, const double* xs, const double* us,
                                         const double* ws, const uint64_t* ids, double* x,
                                         double* u, double* wd, uint64_t* idd, int64_t n,
                                         double h, double dt, double inv_dt, int* status,
                                         uint8_t* outmask, double* wyz, double* fxc,
                                         const PState64* pre = nullptr) {
  double xp[3], up[3], uo[3];
  PState64 st;
  if (pre) st = *pre;
  else load_state64(st, q, xs, us, ws, ids, n);
#pragma unroll
  for (int a = 0; a < 3; ++a) {  // particle q of the current buffer goes to slot p
    xp[a] = st.x[a];
    up[a] = st.u[a];
    uo[a] = up[a];
  }
  const double wp = st.w;
  if (ws && wd != ws) wd[p] = wp;             // carry the read-only planes over
  if (ids && idd != ids) idd[p] = st.id;
  int l[3] = {0, 0, 0};
  double d[3] = {0.0, 0.0, 0.0};
  bool ok = true;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    double sa = __dmul_rn(__dsub_rn(xp[a], g.xmin[a]), g.inv_dx[a]);
    const bool fa = finite_bits(sa);
    if (OPEN && g.open[a]) sa = fmin(fmax(sa, 0.0), (double)g.n[a]);  // sample at the boundary
    int j = floor_clamp_bits(sa, g.n[a] - 1);
    d[a] = __dsub_rn(__dsub_rn(sa, (double)j), 0.5);
    l[a] = j - org[a];
    ok = ok && l[a] >= 0 && l[a] < g.b[a] && fa;
  }
  if (ok) {  // the particle must sit in the cell it was sorted into
    const int lc = (l[2] * g.b[1] + l[1]) * g.b[0] + l[0];
    ok = p >= scs[lc] && p < scs[lc + 1];
  }
  if (!ok) {
    atomicOr(status, ST_DOMAIN);
#pragma unroll
    for (int a = 0; a < 3; ++a) {  // left as it was
      x[a * n + p] = xp[a];
      u[a * n + p] = up[a];
    }
    if (OPEN && outmask) outmask[p] = outside_open(g, xp);
    return;
  }
  double wx[3], wy[3], wz[3] = {0.0, 1.0, 0.0};
  shape_weights<SHAPE>(d[0], wx);
  shape_weights<SHAPE>(d[1], wy);
  if (DIM == 3) shape_weights<SHAPE>(d[2], wz);
  double f[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
  for (int kz = (DIM == 3 ? 0 : 1); kz < (DIM == 3 ? 3 : 2); ++kz) {
    const int zz = DIM == 3 ? l[2] + kz : 0;
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
      const double wzy = wz[kz] * wy[ky];
      if (DEP) wyz[kz * 3 + ky] = wzy;
      if (XQ) {
        // TSC along x from the row's x quadratics (read through L1): the
        // three weighted cells are q0 + d (q1 + d q2); padded index of cell
        // j is j + 1, so the row centre is at the particle's own padded x
        const double4_32a* __restrict__ q4 = reinterpret_cast<const double4_32a*>(fxq);
        const int64_t rc = ((int64_t)(org[2] + zz) * g.pn[1] + org[1] + l[1] + ky) * g.pn[0] +
                           org[0] + l[0] + 1;
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          const double4_32a q = q4[(int64_t)c * g.pplane + rc];
          f[c] = fma(wzy, fma(d[0], fma(d[0], q.z, q.y), q.x), f[c]);
        }
      } else {
        const int row = (zz * g.box[1] + l[1] + ky) * g.box[0] + l[0];
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
          const double ww = wzy * wx[kx];
          const double* sp = sbox + row + kx;
#pragma unroll
          for (int c = 0; c < 6; ++c) f[c] += ww * sp[c * bvol];
        }
      }
    }
  }
  boris_f64(up, f, f + 3, h);
  const double gi = rsqrt(one_plus_norm2(up[0], up[1], up[2]));
  const double dgi = dt * gi;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    const double xa = fma(up[a], dgi, xp[a]);
    xp[a] = OPEN && g.open[a] ? xa : wrap_axis(xa, g.xmin[a], g.xmax[a], g.L[a]);
  }
  bool fin = finite_bits(up[0]) && finite_bits(up[1]) && finite_bits(up[2]) &&
             finite_bits(xp[0]) && finite_bits(xp[1]) && finite_bits(xp[2]);
  if (!fin) atomicOr(status, ST_NONFINITE);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    x[a * n + p] = xp[a];
    u[a * n + p] = up[a];
  }
  if (outmask) outmask[p] = outside_open(g, xp);
  if (DEP) {
    const double wdt = wp * inv_dt;
    double F[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) F[a] = (up[a] - uo[a]) * wdt;
#pragma unroll
    for (int kx = 0; kx < 3; ++kx)
#pragma unroll
      for (int c = 0; c < 3; ++c) fxc[kx * 3 + c] = wx[kx] * F[c];
  }
}

// First index i in [lo, hi] with s[i] > v (s nondecreasing), hi if none.
__device__ __forceinline__ int first_above64(const uint32_t* s, int lo, int hi, uint32_t v) {
  while (lo < hi) {
    const int m = (lo + hi) >> 1;
    if (s[m] > v)
      hi = m;
    else
      lo = m + 1;
  }
  return lo;
}

// Deposit of one chunk [base, bend) by deposit warp `warp` (0..7): the cells
// s with s mod 8 == warp, one lane per stencil offset; every lane loops over
// the same particles, so the loop does not diverge.  Adds into the warp's
// private window in a fixed order.  cfirst: first cell with particles at or
// after base (carried across chunks).
template <int DIM>
__device__ __forceinline__ void deposit_chunk(const Geo& g, const uint32_t* scs,
                                              const double* rw, const double* rf, double* win,
                                              int wsize, int warp, int lane, uint32_t base,
                                              uint32_t bend, int& cfirst) {
  // the chunk's cells by two binary searches of the brick's cell_start
  cfirst = first_above64(scs, 1, g.V, base) - 1;
  const int clast = first_above64(scs, 0, g.V, bend - 1) - 1;
  const int s0 = cfirst + ((warp - cfirst % 8) + 8) % 8;
  for (int sc = s0; sc <= clast; sc += 8) {
    uint32_t r0 = scs[sc], r1 = scs[sc + 1];
    r0 = r0 > base ? r0 : base;
    r1 = r1 < bend ? r1 : bend;
    const int nk = DIM == 3 ? 27 : 9;
    if (lane < nk && r0 < r1) {
      const int kz = DIM == 3 ? lane / 9 : 1;
      const int ky = DIM == 3 ? (lane / 3) % 3 : lane / 3;
      const int kx = lane % 3;
      const double* pw = rw + (kz * 3 + ky) * kRS;
      const double* pf = rf + (kx * 3) * kRS;
      double a0 = 0.0, a1 = 0.0, a2 = 0.0;
      for (uint32_t r = r0; r < r1; ++r) {
        const int i = (int)(r - base);
        const double ww = pw[i];
        a0 += ww * pf[i];
        a1 += ww * pf[kRS + i];
        a2 += ww * pf[2 * kRS + i];
      }
      const int lx = sc & (g.b[0] - 1), ly = (sc >> g.bshift[0]) & (g.b[1] - 1),
                lz = sc >> (g.bshift[0] + g.bshift[1]);   // brick sides are powers of two
      const int ex = lx + kx, ey = ly + ky, ez = DIM == 3 ? lz + kz : 0;
      const int col = ex - warp < 3 ? ex - warp : ex - warp - 5;   // slot in the window
      double* wp = win + warp * wsize + ((col * g.e[2] + ez) * g.e[1] + ey) * 3;
      wp[0] += a0;
      wp[1] += a1;
      wp[2] += a2;
    }
    __syncwarp();
  }
}

// Combine the deposit windows in warp order into the brick's haloed tile.
template <int DIM>
__device__ __forceinline__ void combine_windows(const Geo& g, const double* win, int wsize,
                                                int64_t brick, double* dpart, int t0,
                                                int stride) {
  for (int t = t0; t < g.ev; t += stride) {
    const int ex = t % g.e[0], ey = (t / g.e[0]) % g.e[1], ez = t / (g.e[0] * g.e[1]);
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int w = 0; w < kWarps; ++w) {
      int col = ex - w;
      if (col < 0) continue;
      if (col >= 3) {
        if (DIM == 3 || col < 8 || col >= 11) continue;
        col -= 5;
      }
      const double* wp = win + w * wsize + ((col * g.e[2] + ez) * g.e[1] + ey) * 3;
      s0 += wp[0];
      s1 += wp[1];
      s2 += wp[2];
    }
    dpart[(brick * 3 + 0) * g.ev + t] = s0;
    dpart[(brick * 3 + 1) * g.ev + t] = s1;
    dpart[(brick * 3 + 2) * g.ev + t] = s2;
  }
}

__device__ __forceinline__ void named_bar_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
__device__ __forceinline__ void named_bar_arrive(int id, int nthreads) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Common prologue: TMA of the haloed box on an mbarrier (bounded wait),
// cell_start of the brick, zeroed windows.  Returns false (after reporting
// ST_TIMEOUT) if the copy did not land.
template <int NT, bool STAGE>
__device__ __forceinline__ bool brick_prologue(const CUtensorMap* tmap, const Geo& g,
                                               double* sbox, int bvol, uint32_t* scs,
                                               uint64_t* bar, int* sflag, double* win,
                                               int nwin, const uint32_t* cstart,
                                               int64_t brick, const int* org, int* status) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(bar, 1);
    *sflag = 0;
  }
  __syncthreads();
  if (STAGE && tid == 0) {
    mbar_arrive_expect_tx(bar, (uint32_t)(6 * bvol * 8));
    // padded index of cell c is c + h, so the box starting one cell below the
    // brick origin starts at padded coordinate o
    tma_load_4d(sbox, tmap, bar, org[0], org[1], org[2], 0);
  }
  for (int i = tid; i <= g.V; i += NT) scs[i] = cstart[brick * g.V + i];
  for (int i = tid; i < nwin; i += NT) win[i] = 0.0;
  if (STAGE && !mbar_wait_bounded(bar, 0)) atomicOr(sflag, 1);
  __syncthreads();
  if (*sflag) {
    if (tid == 0) {
      atomicOr(status, ST_TIMEOUT);
      mbar_wait_bounded(bar, 0);
    }
    return false;
  }
  return true;
}

// Without deposit: 256 threads walk the brick's particles in chunks.  OPEN:
// the grid has an open axis (no wrap there, sampling clamped, outflow mask).
template <int SHAPE, int DIM, bool OPEN>
__global__ void __launch_bounds__(kT, 2)
    k_boris_brick_f64(const __grid_constant__ CUtensorMap tmap, const Geo g,
                      const double* __restrict__ fxq, const double* xs, const double* us, const double* ws,
                      const uint64_t* ids, double* x, double* u, double* wd, uint64_t* idd,
                      int64_t n, const uint32_t* __restrict__ perm,
                      const uint32_t* __restrict__ cstart, double* __restrict__ dpart,
                      double qm, double dt, double inv_dt, int* __restrict__ status,
                      uint8_t* __restrict__ outmask) {
  constexpr bool XQ = SHAPE == PART_TSC;  // gather from the x quadratics
  extern __shared__ __align__(128) unsigned char smem[];
  const BrickSmem L = brick_smem(g, XQ ? 0 : 6, 8, false);
  const int tid = threadIdx.x;
  const int bvol = g.box[0] * g.box[1] * g.box[2];
  double* sbox = reinterpret_cast<double*>(smem);
  uint32_t* scs = reinterpret_cast<uint32_t*>(smem + L.cs);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar);
  int* sflag = reinterpret_cast<int*>(smem + L.bar + 8);
  const int64_t brick = blockIdx.x;
  const int org[3] = {(int)(brick % g.nb[0]) * g.b[0],
                      (int)((brick / g.nb[0]) % g.nb[1]) * g.b[1],
                      (int)(brick / ((int64_t)g.nb[0] * g.nb[1])) * g.b[2]};
  if (!brick_prologue<kT, !XQ>(&tmap, g, sbox, bvol, scs, bar, sflag, nullptr, 0, cstart, brick,
                               org, status))
    return;
  const double h = 0.5 * qm * dt;
  const uint32_t p0 = scs[0], p1 = scs[g.V];
  // the next particle's permutation entry and state are loaded while the
  // current one is pushed
  PState64 nxt;
  uint32_t qnext = 0;
  if (p0 + tid < p1) {
    qnext = perm ? perm[p0 + tid] : p0 + tid;
    load_state64(nxt, qnext, xs, us, ws, ids, n);
  }
  for (uint32_t p = p0 + tid; p < p1; p += kT) {
    const PState64 cur = nxt;
    const uint32_t qcur = qnext;
    if (p + kT < p1) {
      qnext = perm ? perm[p + kT] : p + kT;
      load_state64(nxt, qnext, xs, us, ws, ids, n);
    }
    push_one<SHAPE, DIM, false, OPEN, XQ>(g, sbox, bvol, fxq, scs, org, p, qcur, xs, us, ws, ids,
                                          x, u, wd, idd, n, h, dt, inv_dt, status, outmask,
                                          nullptr, nullptr, &cur);
  }
}

// With deposit: warp-specialised, 512 threads.  Warps 0-7 push chunk k of 256
// particles and leave its records in buffer k & 1; warps 8-15 deposit chunk
// k - 1 from the other buffer at the same time.  The hand-off uses named
// barriers (FULL_b: records of buffer b written; EMPTY_b: buffer b read), so
// both phases keep the FP64 pipe busy and neither waits for the other's
// latency.  Both groups derive the same chunk count from cell_start.
template <int SHAPE, int DIM, bool OPEN>
__global__ void __launch_bounds__(2 * kT, 1)
    k_boris_brick_f64_dep(const __grid_constant__ CUtensorMap tmap, const Geo g,
                          const double* __restrict__ fxq, const double* xs, const double* us, const double* ws,
                          const uint64_t* ids, double* x, double* u, double* wd,
                          uint64_t* idd, int64_t n, const uint32_t* __restrict__ perm,
                          const uint32_t* __restrict__ cstart,
                          double* __restrict__ dpart, double qm, double dt, double inv_dt,
                          int* __restrict__ status, uint8_t* __restrict__ outmask) {
  constexpr int NT = 2 * kT;
  constexpr int kFull = 1, kEmpty = 3;  // named barrier ids (0 is __syncthreads)
  constexpr bool XQ = SHAPE == PART_TSC;  // gather from the x quadratics
  extern __shared__ __align__(128) unsigned char smem[];
  const BrickSmem L = brick_smem(g, XQ ? 0 : 6, 8, true);
  const int tid = threadIdx.x;
  const int bvol = g.box[0] * g.box[1] * g.box[2];
  double* sbox = reinterpret_cast<double*>(smem);
  uint32_t* scs = reinterpret_cast<uint32_t*>(smem + L.cs);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar);
  int* sflag = reinterpret_cast<int*>(smem + L.bar + 8);
  double* rec = reinterpret_cast<double*>(smem + L.rec);  // [2][18][kRS]
  double* win = reinterpret_cast<double*>(smem + L.win);  // [warp][slot][e2][e1][3]
  constexpr int NS = kslots(DIM);
  const int wsize = NS * g.e[1] * g.e[2] * 3;
  const int64_t brick = blockIdx.x;
  const int org[3] = {(int)(brick % g.nb[0]) * g.b[0],
                      (int)((brick / g.nb[0]) % g.nb[1]) * g.b[1],
                      (int)(brick / ((int64_t)g.nb[0] * g.nb[1])) * g.b[2]};
  if (!brick_prologue<NT, !XQ>(&tmap, g, sbox, bvol, scs, bar, sflag, win, kWarps * wsize,
                               cstart, brick, org, status))
    return;
  const uint32_t p0 = scs[0], p1 = scs[g.V];
  const int nchunks = (int)((p1 - p0 + kT - 1) / kT);
  if (tid < kT) {  // producer warps: push
    const double h = 0.5 * qm * dt;
    // each thread's particle of the next chunk is loaded while this one is
    // finished, so a chunk never starts with the permutation and state reads
    PState64 nxt;
    uint32_t qnext = 0;
    {
      const uint32_t pn = p0 + tid;
      if (pn < p1) {
        qnext = perm ? perm[pn] : pn;
        load_state64(nxt, qnext, xs, us, ws, ids, n);
      }
    }
    for (int k = 0; k < nchunks; ++k) {
      const int b = k & 1;
      const uint32_t p = p0 + (uint32_t)k * kT + tid;
      double wyz[9], fxc[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) wyz[q] = fxc[q] = 0.0;
      if (p < p1) {
        const PState64 cur = nxt;
        const uint32_t qcur = qnext;
        if (p + kT < p1) {
          qnext = perm ? perm[p + kT] : p + kT;
          load_state64(nxt, qnext, xs, us, ws, ids, n);
        }
        push_one<SHAPE, DIM, true, OPEN, XQ>(g, sbox, bvol, fxq, scs, org, p, qcur, xs, us, ws,
                                             ids, x, u, wd, idd, n, h, dt, inv_dt, status,
                                             outmask, wyz, fxc, &cur);
      }
      if (k >= 2) named_bar_sync(kEmpty + b, NT);  // deposit of chunk k-2 has read it
      double* rw = rec + (size_t)b * 18 * kRS;
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        rw[q * kRS + tid] = wyz[q];
        rw[(9 + q) * kRS + tid] = fxc[q];
      }
      named_bar_arrive(kFull + b, NT);
    }
    // complete the EMPTY instances of the last two chunks
    for (int k = nchunks > 2 ? nchunks - 2 : 0; k < nchunks; ++k)
      named_bar_sync(kEmpty + (k & 1), NT);
  } else {  // consumer warps: deposit
    const int dw = (tid - kT) >> 5, lane = tid & 31;
    int cfirst = 0;
    for (int k = 0; k < nchunks; ++k) {
      const int b = k & 1;
      named_bar_sync(kFull + b, NT);
      const uint32_t base = p0 + (uint32_t)k * kT;
      const uint32_t bend = base + kT < p1 ? base + kT : p1;
      const double* rw = rec + (size_t)b * 18 * kRS;
      deposit_chunk<DIM>(g, scs, rw, rw + 9 * kRS, win, wsize, dw, lane, base, bend, cfirst);
      named_bar_arrive(kEmpty + b, NT);
    }
  }
  __syncthreads();
  combine_windows<DIM>(g, win, wsize, brick, dpart, tid, NT);
}

// ---------------------------------------------------------------- particle order, FP64
template <int SHAPE, int DIM, bool OPEN>
__global__ void __launch_bounds__(256)
    k_boris_particles_f64(const double* __restrict__ fp, const double* __restrict__ fxq,
                          const Geo g, double* __restrict__ x,
                          double* __restrict__ u, int64_t n, double qm, double dt, int nsteps,
                          int* __restrict__ status, uint8_t* __restrict__ outmask) {
  const double h = 0.5 * qm * dt;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    double xp[3], up[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      xp[a] = x[a * n + p];
      up[a] = u[a * n + p];
    }
    bool bad = false;
    // a particle that has left through an open face is not advanced further
    for (int st = 0; st < nsteps && !(OPEN && outside_open(g, xp)); ++st) {
      int j[3] = {0, 0, 0};
      double d[3] = {0.0, 0.0, 0.0};
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        double s = __dmul_rn(__dsub_rn(xp[a], g.xmin[a]), g.inv_dx[a]);
        if (!finite_bits(s)) {
          bad = true;
          s = 0.0;
        }
        if (OPEN && g.open[a]) s = fmin(fmax(s, 0.0), (double)g.n[a]);
        j[a] = floor_clamp_bits(s, g.n[a] - 1);
        d[a] = __dsub_rn(__dsub_rn(s, (double)j[a]), 0.5);
      }
      double wx[3], wy[3], wz[3] = {0.0, 1.0, 0.0};
      if (SHAPE != PART_TSC) shape_weights<SHAPE>(d[0], wx);
      shape_weights<SHAPE>(d[1], wy);
      if (DIM == 3) shape_weights<SHAPE>(d[2], wz);
      double f[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
      for (int kz = (DIM == 3 ? 0 : 1); kz < (DIM == 3 ? 3 : 2); ++kz) {
        const int zz = DIM == 3 ? j[2] + kz : 0;
#pragma unroll
        for (int ky = 0; ky < 3; ++ky) {
          const double wzy = wz[kz] * wy[ky];
          const int64_t row = ((int64_t)zz * g.pn[1] + j[1] + ky) * g.pn[0] + j[0];
          if (SHAPE == PART_TSC) {  // the row from its x quadratics, as in the brick kernels
            const double4_32a* __restrict__ q4 = reinterpret_cast<const double4_32a*>(fxq);
#pragma unroll
            for (int c = 0; c < 6; ++c) {
              const double4_32a q = q4[(int64_t)c * g.pplane + row + 1];
              f[c] = fma(wzy, fma(d[0], fma(d[0], q.z, q.y), q.x), f[c]);
            }
          } else {
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
              const double ww = wzy * wx[kx];
#pragma unroll
              for (int c = 0; c < 6; ++c) f[c] += ww * __ldg(fp + c * g.pplane + row + kx);
            }
          }
        }
      }
      boris_f64(up, f, f + 3, h);
      const double gi = rsqrt(one_plus_norm2(up[0], up[1], up[2]));
      const double dgi = dt * gi;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        const double xa = fma(up[a], dgi, xp[a]);
        xp[a] = OPEN && g.open[a] ? xa : wrap_axis(xa, g.xmin[a], g.xmax[a], g.L[a]);
      }
      if (bad) break;
    }
    if (bad || !(isfinite(up[0]) && isfinite(up[1]) && isfinite(up[2]) && isfinite(xp[0]) &&
                 isfinite(xp[1]) && isfinite(xp[2])))
      atomicOr(status, ST_NONFINITE);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      x[a * n + p] = xp[a];
      u[a * n + p] = up[a];
    }
    if (OPEN && outmask) outmask[p] = outside_open(g, xp);
  }
}

// ---------------------------------------------------------------- deposit combine
// out[c][g] = sum over the bricks whose haloed tile covers cell g (or one of
// its periodic images), in fixed (z, y, x, image) order, of their partials.
__global__ void __launch_bounds__(256)
    k_dep_combine(const double* __restrict__ dpart, double* __restrict__ out, const Geo g,
                  bool fast) {
  for (int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gi < g.G;
       gi += (int64_t)gridDim.x * blockDim.x) {
    int j[3];
    if (g.G <= INT32_MAX) {
      cell_coords(g, (int32_t)gi, j);  // float-reciprocal divmod, no 64-bit division
    } else {
      j[0] = (int)(gi % g.n[0]);
      j[1] = (int)((gi / g.n[0]) % g.n[1]);
      j[2] = (int)(gi / ((int64_t)g.n[0] * g.n[1]));
    }
    if (fast) {
      // full bricks and at least three per active axis: the cell is in its
      // own brick's tile, and in one neighbour's halo when it is on a face
      // of its brick.  A warp's lanes share y and z, so the loop over the
      // (y, z) tiles is uniform; along x a lane has its own tile's partial and
      // at most one neighbour's (on an x face), added as one pair (0 where
      // there is none).  The rows are then summed in (z, y) order, starting
      // from the first: the FP64 adds (this pass's bound) are all full-warp.
      int cb[3][3], ce[3][3], cnt[3];
#pragma unroll
      for (int a = 1; a < 3; ++a) {
        const int bj = j[a] >> g.bshift[a], l = j[a] & (g.b[a] - 1);
        cnt[a] = 0;
        if (g.h[a] != 0 && l == 0) {
          cb[a][cnt[a]] = bj == 0 ? g.nb[a] - 1 : bj - 1;
          ce[a][cnt[a]++] = g.b[a] + 1;
        }
        cb[a][cnt[a]] = bj;
        ce[a][cnt[a]++] = l + g.h[a];
        if (g.h[a] != 0 && l == g.b[a] - 1) {
          cb[a][cnt[a]] = bj == g.nb[a] - 1 ? 0 : bj + 1;
          ce[a][cnt[a]++] = 0;
        }
      }
      const int bx = j[0] >> g.bshift[0], lx = j[0] & (g.b[0] - 1);
      int xb = -1, xe = 0;  // the x neighbour whose halo holds the cell, if any
      if (lx == 0) {
        xb = bx == 0 ? g.nb[0] - 1 : bx - 1;
        xe = g.b[0] + 1;
      } else if (lx == g.b[0] - 1) {
        xb = bx == g.nb[0] - 1 ? 0 : bx + 1;
        xe = 0;
      }
      double s0 = 0.0, s1 = 0.0, s2 = 0.0;
      for (int qz = 0; qz < cnt[2]; ++qz)
        for (int qy = 0; qy < cnt[1]; ++qy) {
          const int64_t rb = ((int64_t)cb[2][qz] * g.nb[1] + cb[1][qy]) * g.nb[0];
          const int trow = (ce[2][qz] * g.e[1] + ce[1][qy]) * g.e[0];
          const double* po = dpart + (rb + bx) * 3 * g.ev + trow + lx + 1;
          double e0 = 0.0, e1 = 0.0, e2 = 0.0;
          if (xb >= 0) {
            const double* pe = dpart + (rb + xb) * 3 * g.ev + trow + xe;
            e0 = pe[0];
            e1 = pe[g.ev];
            e2 = pe[2 * (int64_t)g.ev];
          }
          const double t0 = po[0] + e0, t1 = po[g.ev] + e1, t2 = po[2 * (int64_t)g.ev] + e2;
          if (qz == 0 && qy == 0) {
            s0 = t0;
            s1 = t1;
            s2 = t2;
          } else {
            s0 += t0;
            s1 += t1;
            s2 += t2;
          }
        }
      out[gi] = s0;
      out[g.G + gi] = s1;
      out[2 * g.G + gi] = s2;
      continue;
    }
    int cb[3][9], ce[3][9], cnt[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cnt[a] = 0;
      if (g.h[a] == 0) {
        cb[a][0] = j[a] / g.b[a];
        ce[a][0] = j[a] - cb[a][0] * g.b[a];
        cnt[a] = 1;
        continue;
      }
      const int bj = j[a] / g.b[a];
      if (g.open[a]) {
        // no periodic images; the edge cell also collects what was deposited
        // beyond its face (global cell -1 or n), the adjoint of the
        // zero-gradient gather
        for (int t = (j[a] == 0 ? -1 : j[a]); t <= (j[a] == g.n[a] - 1 ? g.n[a] : j[a]); ++t)
          for (int db = -1; db <= 1; ++db) {
            const int bb = bj + db;
            if (bb < 0 || bb >= g.nb[a]) continue;
            const int ee = t - bb * g.b[a] + g.h[a];
            if (ee >= 0 && ee < g.e[a] && cnt[a] < 9) {
              cb[a][cnt[a]] = bb;
              ce[a][cnt[a]] = ee;
              cnt[a]++;
            }
          }
        continue;
      }
      for (int db = -1; db <= 1; ++db) {
        int bb = ((bj + db) % g.nb[a] + g.nb[a]) % g.nb[a];
        bool dup = false;
        for (int q = 0; q < cnt[a]; ++q) dup = dup || (cb[a][q] == bb);
        if (dup) continue;
        for (int m = -1; m <= 1; ++m) {
          int ee = j[a] + m * g.n[a] - bb * g.b[a] + g.h[a];
          if (ee >= 0 && ee < g.e[a] && cnt[a] < 9) {
            cb[a][cnt[a]] = bb;
            ce[a][cnt[a]] = ee;
            cnt[a]++;
          }
        }
      }
    }
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int qz = 0; qz < cnt[2]; ++qz)
      for (int qy = 0; qy < cnt[1]; ++qy)
        for (int qx = 0; qx < cnt[0]; ++qx) {
          const int64_t br = ((int64_t)cb[2][qz] * g.nb[1] + cb[1][qy]) * g.nb[0] + cb[0][qx];
          const int t = (ce[2][qz] * g.e[1] + ce[1][qy]) * g.e[0] + ce[0][qx];
          const double* pp = dpart + br * 3 * g.ev + t;
          s0 += pp[0];
          s1 += pp[g.ev];
          s2 += pp[2 * (int64_t)g.ev];
        }
    out[gi] = s0;
    out[g.G + gi] = s1;
    out[2 * g.G + gi] = s2;
  }
}

template <int SHAPE, int DIM, bool DEP>
cudaError_t brick_f64(part_ctx* c, double qm, double dt) {
  const bool open = c->geo.any_open != 0;
  auto kern = DEP ? (open ? k_boris_brick_f64_dep<SHAPE, DIM, true>
                          : k_boris_brick_f64_dep<SHAPE, DIM, false>)
                  : (open ? k_boris_brick_f64<SHAPE, DIM, true>
                          : k_boris_brick_f64<SHAPE, DIM, false>);
  constexpr bool XQ = SHAPE == PART_TSC;  // no staged box: the x quadratics
  const BrickSmem L = brick_smem(c->geo, XQ ? 0 : 6, 8, DEP);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)L.total);
  if (e != cudaSuccess) return e;
  // read the current buffer (through the sort's permutation, if one is
  // pending, into the other buffer; else in place)
  const PState src = state_of(c, c->cur_alt);
  const PState dst = c->perm_pend ? state_of(c, !c->cur_alt) : src;
  kern<<<(unsigned)c->geo.nbricks, DEP ? 2 * kT : kT, L.total, c->stream>>>(
      c->tmap, c->geo, c->fxq, (const double*)src.x, (const double*)src.u, (const double*)src.w, src.id,
      (double*)dst.x, (double*)dst.u, (double*)dst.w, dst.id, c->n, c->perm_pend, c->cstart,
      c->dpart, qm, dt, 1.0 / dt, c->status, c->outmask);
  c->launches++;
  if (c->perm_pend) {
    c->perm_pend = nullptr;
    c->cur_alt = !c->cur_alt;
  }
  return cudaGetLastError();
}

template <int SHAPE, int DIM>
cudaError_t particles_f64(part_ctx* c, double qm, double dt, int nsteps) {
  auto kern = c->geo.any_open ? k_boris_particles_f64<SHAPE, DIM, true>
                              : k_boris_particles_f64<SHAPE, DIM, false>;
  const int t = threads_for_spread(c, c->n);
  kern<<<grid_for(c, c->n, t), t, 0, c->stream>>>(
      (const double*)c->fpad, c->fxq, c->geo, (double*)c->x, (double*)c->u, c->n, qm, dt, nsteps,
      c->status, c->outmask);
  c->launches++;
  return cudaGetLastError();
}

template <int SHAPE, int DIM>
cudaError_t dispatch_f64(part_ctx* c, double qm, double dt, int nsteps) {
  if (c->sorted && nsteps == 1) {
    return c->deposit_on ? brick_f64<SHAPE, DIM, true>(c, qm, dt)
                         : brick_f64<SHAPE, DIM, false>(c, qm, dt);
  }
  return particles_f64<SHAPE, DIM>(c, qm, dt, nsteps);
}

}  // namespace

cudaError_t launch_boris(part_ctx* c, double qm, double dt, int nsteps) {
  if (c->n == 0) return cudaSuccess;
  const int dim = c->geo.dim;
  if (c->prec == PART_FP64) {
    if (c->shape == PART_TSC)
      return dim == 3 ? dispatch_f64<PART_TSC, 3>(c, qm, dt, nsteps)
                      : dispatch_f64<PART_TSC, 2>(c, qm, dt, nsteps);
    return dim == 3 ? dispatch_f64<PART_CIC, 3>(c, qm, dt, nsteps)
                    : dispatch_f64<PART_CIC, 2>(c, qm, dt, nsteps);
  }
  return launch_boris_mixed(c, qm, dt, nsteps);
}

cudaError_t launch_deposit_combine(part_ctx* c, double* out) {
  const Geo& g = c->geo;
  bool fast = true;
  for (int a = 0; a < 3; ++a)
    if (g.h[a] != 0 && (g.nb[a] < 3 || g.n[a] % g.b[a] != 0 || g.open[a])) fast = false;
  k_dep_combine<<<grid_for(c, g.G, 256), 256, 0, c->stream>>>(c->dpart, out, g, fast);
  c->launches++;
  return cudaGetLastError();
}
