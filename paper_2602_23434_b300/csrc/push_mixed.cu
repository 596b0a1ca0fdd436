// push_mixed.cu -- mixed-precision form of the gather + Boris push (+ deposit).
//
// State: int32 linear cell + f32 offset from the cell centre (cell units, in
// [-1/2, 1/2)) + the momentum as a compensated f32 pair u[6] = (hi[3], lo[3])
// (+ optional f32 w).  Fields are staged as f32.  The
// push runs in f32.  The deposit sums each source cell's particles in f32
// (a handful of terms: ~8 at 8 particles per cell), adds those per-cell sums
// into compensated (two-float, about 48-bit) accumulators of the brick's
// haloed tile, and leaves FP64 partials that are combined in FP64.
//
// Brick kernel (sorted): TMA stages the brick's haloed f32 field box; the
// brick's particles are processed in super-chunks of up to kM particles:
//   A. one thread per particle: weights from the offsets, gather, Boris, move
//      (offset += dt v/dx, integer cell carry, periodic wrap); the old offsets
//      and the force w du/dt are left in shared memory.  du is formed from the
//      Boris rotation increment (u' x s + 2hE), not as u_new - u_old, so f32
//      cancellation does not enter the force;
//   B. one thread per (source cell, force component) sums its particles' 27
//      contributions in registers, then 27 passes (one per stencil offset,
//      separated by barriers) add them into the haloed tile's two-float
//      accumulators: in a pass no two threads share a target, and the order
//      is fixed.  Super-chunks of 640 particles (about 80 cells, so about
//      240 of the 255 phase-B lanes busy) keep shared memory at ~74 KB and
//      the registers at 80, so three CTAs share an SM.
// Each thread loads the state of its first particle of the next super-chunk
// before the deposit of the current one, so phase A never starts cold.
// Particle-order kernel: nsteps fused steps, state in registers, stencil read
// from the padded global f32 copy (test particles, serving).
#include "part_internal.cuh"

namespace {

constexpr int kT = kPushThreads;
constexpr int kM = 640;   // particles per super-chunk (~80 cells: 240 of the 255 phase-B lanes)
// Row stride of the record planes: kM + 11 floats puts the three force rows
// (read at once by a cell's three component lanes) on different banks.
constexpr int kR = kM + 11;

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct MixedSmem {
  size_t cs, bar, rec, acc, total;
  int evp;  // component stride of the two-float tile (in float2)
};
__host__ __device__ inline MixedSmem mixed_smem(const Geo& g) {
  MixedSmem s;
  size_t bbytes = (size_t)8 * g.box[0] * g.box[1] * g.box[2] * 4;  // 8 floats per cell
  s.cs = align_up(bbytes, 128);
  s.bar = align_up(s.cs + (size_t)(g.V + 1) * 4, 16);
  s.rec = align_up(s.bar + 16, 128);
  s.acc = align_up(s.rec + (size_t)6 * kR * 4, 16);
  // components (hi, lo) strided by evp = 6 mod 16 float2: the three component
  // lanes of a cell, adding to the same target offset, land on different banks
  s.evp = g.ev + ((6 - g.ev % 16) + 16) % 16;
  s.total = s.acc + (size_t)3 * s.evp * 8;
  return s;
}

// Knuth's TwoSum: returns s = fl(a + b) and sets e so that s + e = a + b.
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float s = a + b;
  const float bp = s - a;
  e = (a - (s - bp)) + (b - bp);
  return s;
}

// Paired f32 arithmetic (two lanes per instruction, each rounded to nearest
// as its scalar form).  sub2 is b * (-1) + a, one rounding of a - b.
__device__ __forceinline__ float2 sp2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
__device__ __forceinline__ float2 two_sum2(float2 a, float2 b, float2& e) {
  const float2 s = add2(a, b);
  const float2 bp = sub2(s, a);
  e = add2(sub2(a, sub2(s, bp)), sub2(b, bp));
  return s;
}
// 1/x to about an ulp (the hardware approximation); every use below corrects
// the quotient with its exact remainder.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// f32 relativistic Boris kick of the compensated momentum u + ul (ul the f32
// residual of u).  The momentum is kept as that pair because rounding it to
// f32 after every step is a random walk that the gyrophase budget (1e-5 rad
// per 1000 steps) cannot absorb, least of all for particles gyrating on a
// small circle: the step's increment u^{n+1} - u^n is added to the pair
// exactly (TwoSum), so only the increment's own rounding (a fraction of the
// rotation angle's worth) enters each step.
// The rotation parameters are the quantities whose rounding repeats
// identically every step (in a steady field), so they are formed to about
// half an ulp with error-free transformations (TwoProd by fma, exact residuals
// of 1 + q): 1/gamma- is refined from rsqrtf by one Newton step evaluated in
// two-float, h = h_hi + h_lo is the two-float half step, t = h B / gamma- and
// s = 2 t / (1 + |t|^2) are each kept as an f32 value plus its f32 residual
// (2 / (1 + |t|^2) from the approximate reciprocal and the exact remainder of
// the quotient, so the value plus residual is good to about 2^-46).
// The rotation, being linear in u-, is applied to u-'s value and, to first
// order, to its residual.
// Components 0 and 1 of every vector go as one pair (paired instructions);
// the cross products mix components and stay scalar.  f holds the gathered
// fields as the pairs (E0, E1), (B0, B1), (E2, B2).
// du gets u^{n+1} - u^n from the rotation increment and the two half-kicks.
__device__ __forceinline__ void boris_f32(float* u, float* ul, const float2* f, float h,
                                          float hl, float* du) {
  const float2 E01 = f[0], B01 = f[1];
  const float E2 = f[2].x, B2 = f[2].y;
  // half kick k = h E with the two-float h
  const float2 k01 = fma2(sp2(h), E01, mul2(sp2(hl), E01));
  const float k2 = fmaf(h, E2, hl * E2);
  // u- = u + k as a pair (um, ml)
  float2 e01;
  float e2;
  const float2 um01 = two_sum2(make_float2(u[0], u[1]), k01, e01);
  const float um2 = two_sum(u[2], k2, e2);
  const float2 ml01 = add2(make_float2(ul[0], ul[1]), e01);
  const float ml2 = ul[2] + e2;
  const float um0 = um01.x, um1 = um01.y, ml0 = ml01.x, ml1 = ml01.y;
  const float q = fmaf(um2, um2, fmaf(um1, um1, um0 * um0));
  const float a = 1.0f + q;
  const float res = q - (a - 1.0f);             // exact: a + res = 1 + q
  const float y = rsqrtf(a);
  const float yp = y * y;
  const float ype = fmaf(y, y, -yp);            // y^2 = yp + ype exactly
  const float r = fmaf(-a, yp, 1.0f) - fmaf(a, ype, res * yp);  // 1 - (1+q) y^2
  const float gl = 0.5f * y * r;                // 1/gamma- = y + gl
  const float hg = h * y;
  const float hge = fmaf(h, y, -hg) + fmaf(h, gl, hl * y);      // h/gamma- = hg + hge
  // t = (h/gamma-) B and its residual tl: t_true = t + tl to ~2^-46 relative
  const float2 hb01 = mul2(sp2(hge), B01);
  const float2 t01 = fma2(sp2(hg), B01, hb01);
  const float2 tl01 = sub2(hb01, fma2(sp2(-hg), B01, t01));
  const float hb2 = hge * B2;
  const float t2 = fmaf(hg, B2, hb2);
  const float tl2 = fmaf(hg, B2, -t2) + hb2;
  const float t0 = t01.x, t1 = t01.y, tl0 = tl01.x, tl1 = tl01.y;
  const float tt = fmaf(t2, t2, fmaf(t1, t1, t0 * t0));
  const float d = 1.0f + tt;
  const float dres = tt - (d - 1.0f);           // exact: d + dres = 1 + |t|^2
  const float rd = rcp_approx(d);
  const float sf = 2.0f * rd;                   // 2 / (1 + |t|^2) to about an ulp
  const float sfl = (fmaf(-sf, d, 2.0f) - sf * dres) * rd;      // ... = sf + sfl
  const float2 s01 = fma2(sp2(sf), t01, mul2(sp2(sfl), t01));
  const float2 sl01 =
      sub2(fma2(sp2(sfl), t01, mul2(sp2(sf), tl01)), fma2(sp2(-sf), t01, s01));
  const float s2 = fmaf(sf, t2, sfl * t2);
  const float sl2 = fmaf(sf, t2, -s2) + fmaf(sfl, t2, sf * tl2);
  const float s0 = s01.x, s1 = s01.y, sl0 = sl01.x, sl1 = sl01.y;
  // u' = u- + u- x t and u+ - u- = u' x s with t, s carried as value +
  // residual: the residual terms are first-order small and enter in plain f32,
  // so the rotation angle carries no rounding that repeats from step to step
  const float2 p01 = add2(um01, add2(make_float2(um1 * t2 - um2 * t1, um2 * t0 - um0 * t2),
                                     make_float2(um1 * tl2 - um2 * tl1, um2 * tl0 - um0 * tl2)));
  const float p2 = um2 + ((um0 * t1 - um1 * t0) + (um0 * tl1 - um1 * tl0));
  const float p0 = p01.x, p1 = p01.y;
  const float2 r01 = add2(make_float2(p1 * s2 - p2 * s1, p2 * s0 - p0 * s2),
                          make_float2(p1 * sl2 - p2 * sl1, p2 * sl0 - p0 * sl2));  // u+ - u-
  const float r2 = (p0 * s1 - p1 * s0) + (p0 * sl1 - p1 * sl0);
  // the same rotation of u-'s residual, to first order
  const float2 pl01 = add2(ml01, make_float2(ml1 * t2 - ml2 * t1, ml2 * t0 - ml0 * t2));
  const float pl2 = ml2 + (ml0 * t1 - ml1 * t0);
  const float pl0 = pl01.x, pl1 = pl01.y;
  const float2 rl01 = make_float2(pl1 * s2 - pl2 * s1, pl2 * s0 - pl0 * s2);
  const float rl2 = pl0 * s1 - pl1 * s0;
  // increment D = r + rl + 2 h E, added to the pair exactly:
  // (u + ul) + D = su + (ul + g + f + rl) with d + f = r + 2k, su + g = u + d
  float2 f01, g01;
  float f2, g2;
  const float2 d01 = two_sum2(r01, add2(k01, k01), f01);
  const float d2 = two_sum(r2, 2.0f * k2, f2);
  du[0] = d01.x;
  du[1] = d01.y;
  du[2] = d2;
  const float2 su01 = two_sum2(make_float2(u[0], u[1]), d01, g01);
  const float su2 = two_sum(u[2], d2, g2);
  const float2 lo01 = add2(make_float2(ul[0], ul[1]), add2(g01, add2(f01, rl01)));
  const float lo2 = ul[2] + (g2 + (f2 + rl2));
  // renormalise (FastTwoSum: |su| >= |lo|)
  const float2 un01 = add2(su01, lo01);
  const float2 uln01 = sub2(lo01, sub2(un01, su01));
  u[0] = un01.x;
  u[1] = un01.y;
  u[2] = su2 + lo2;
  ul[0] = uln01.x;
  ul[1] = uln01.y;
  ul[2] = lo2 - (u[2] - su2);
}

// Knuth's TwoSum into a (hi, lo) pair: hi + lo carries the sum with the
// rounding error of hi.
__device__ __forceinline__ float2 two_sum_add(float2 v, float x) {
  const float s = v.x + x;
  const float bp = s - v.x;
  v.y += (v.x - (s - bp)) + (x - bp);
  v.x = s;
  return v;
}

// Stencil point accumulate: six field components of one cell (two 16-byte
// loads of the cell-interleaved copy, whose record holds E0 E1 B0 B1 E2 B2)
// weighted by ww, as three paired FMAs into (E0, E1), (B0, B1), (E2, B2).
__device__ __forceinline__ void acc_point(float2* f, float ww, float4 a, float4 b) {
  const float2 w2 = make_float2(ww, ww);
  f[0] = __ffma2_rn(w2, make_float2(a.x, a.y), f[0]);
  f[1] = __ffma2_rn(w2, make_float2(a.z, a.w), f[1]);
  f[2] = __ffma2_rn(w2, make_float2(b.x, b.y), f[2]);
}

// Move in cell units: off += dv; whole cells carry into j (periodic).  On an
// open axis a particle that leaves is held at the face (edge cell, offset
// -1/2 or +1/2) and marked out.
__device__ __forceinline__ void move_axis(float& off, int& j, float dv, int n, int open,
                                          bool& out) {
  off = off + dv;
  const float k = floorf(off + 0.5f);
  off = off - k;
  int jj = j + (int)k;
  if (jj < 0 || jj >= n) {
    if (open) {
      out = true;
      off = jj < 0 ? -0.5f : 0.5f;
      jj = jj < 0 ? 0 : n - 1;
    } else {
      jj = ((jj % n) + n) % n;
    }
  }
  j = jj;
}

// First index i in [lo, hi] with s[i] > v (s nondecreasing), hi if none.
__device__ __forceinline__ int first_above(const uint32_t* s, int lo, int hi, uint32_t v) {
  while (lo < hi) {
    const int m = (lo + hi) >> 1;
    if (s[m] > v)
      hi = m;
    else
      lo = m + 1;
  }
  return lo;
}

template <int SHAPE, int DIM, bool DEP>
__global__ void __launch_bounds__(kT, 3)
    k_boris_brick_mixed(const __grid_constant__ CUtensorMap tmap, const Geo g,
                        const int32_t* cells, const float* offs, const float* us,
                        const float* w, const uint64_t* ids, int32_t* cell, float* off,
                        float* u, float* wd, uint64_t* idd, int64_t n,
                        const uint32_t* __restrict__ perm,
                        const uint32_t* __restrict__ cstart, double* __restrict__ dpart,
                        float h, float hl, float dtdx0, float dtdx1, float dtdx2, float inv_dt,
                        int* __restrict__ status, uint8_t* __restrict__ outmask) {
  extern __shared__ __align__(128) unsigned char smem[];
  const MixedSmem L = mixed_smem(g);
  const int tid = threadIdx.x;
  const int bvol = g.box[0] * g.box[1] * g.box[2];
  float* sbox = reinterpret_cast<float*>(smem);
  uint32_t* scs = reinterpret_cast<uint32_t*>(smem + L.cs);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar);
  int* sflag = reinterpret_cast<int*>(smem + L.bar + 8);
  float* rd = reinterpret_cast<float*>(smem + L.rec);  // [3][kR] old offsets
  float* rF = rd + 3 * kR;                              // [3][kR] force
  float2* acc = reinterpret_cast<float2*>(smem + L.acc);  // [3][evp] (hi, lo)

  const int64_t brick = blockIdx.x;
  const int bx = (int)(brick % g.nb[0]);
  const int by = (int)((brick / g.nb[0]) % g.nb[1]);
  const int bz = (int)(brick / ((int64_t)g.nb[0] * g.nb[1]));
  const int org[3] = {bx * g.b[0], by * g.b[1], bz * g.b[2]};

  if (tid == 0) {
    mbar_init(bar, 1);
    *sflag = 0;
  }
  __syncthreads();
  if (tid == 0) {
    mbar_arrive_expect_tx(bar, (uint32_t)(8 * bvol * 4));
    tma_load_4d(sbox, &tmap, bar, 0, org[0], org[1], org[2]);
  }
  for (int i = tid; i <= g.V; i += kT) scs[i] = cstart[brick * g.V + i];
  if (DEP)
    for (int i = tid; i < 3 * L.evp; i += kT) acc[i] = make_float2(0.0f, 0.0f);
  if (!mbar_wait_bounded(bar, 0)) atomicOr(sflag, 1);
  __syncthreads();
  if (*sflag) {
    if (tid == 0) {
      atomicOr(status, ST_TIMEOUT);
      mbar_wait_bounded(bar, 0);
    }
    return;
  }

  const float dtdx[3] = {dtdx0, dtdx1, dtdx2};
  const uint32_t p0 = scs[0], p1 = scs[g.V];
  int cfirst = 0;  // first brick cell with particles at or after the super-chunk start
  // state of each thread's first particle of a super-chunk, loaded before the
  // previous super-chunk's deposit so that phase A starts with it at hand
  int32_t nc = 0;
  float no[3] = {0.f, 0.f, 0.f}, nu[3] = {0.f, 0.f, 0.f}, nl[3] = {0.f, 0.f, 0.f}, nw = 1.0f;
  uint32_t qc = 0, qn = 0;
  auto prefetch = [&](uint32_t sbx) {
    const uint32_t sex = p1 - sbx < (uint32_t)kM ? p1 : sbx + kM;
    const uint32_t px = sbx + tid;
    qc = px;
    qn = px + kT;
    if (perm) {
      if (px < sex) qc = perm[px];
      if (px + kT < sex) qn = perm[px + kT];
    }
    if (px < sex) {
      nc = cells[qc];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        no[a] = offs[a * n + qc];
        nu[a] = us[a * n + qc];
        nl[a] = us[(a + 3) * n + qc];
      }
      if (w) nw = w[qc];
    }
  };
  prefetch(p0);
  for (uint32_t sb = p0; sb < p1; sb += kM) {
    const uint32_t se = p1 - sb < (uint32_t)kM ? p1 : sb + kM;
    // ---- A: push, one thread per particle; the next particle's state is
    // loaded before the current one is computed
    // particle q of the current buffer goes to slot p; the permutation is
    // read two slots ahead and the state one slot ahead of the computation
    uint32_t p = sb + tid;
    for (; p < se; p += kT) {
      const int i = (int)(p - sb);
      const int32_t ccur = nc;
      float o[3] = {no[0], no[1], no[2]}, up[3] = {nu[0], nu[1], nu[2]};
      float ul[3] = {nl[0], nl[1], nl[2]};
      const float wcur = nw;
      const uint32_t qcur = qc;
      if (p + kT < se) {
        qc = qn;
        if (p + 2 * kT < se) qn = perm ? perm[p + 2 * kT] : p + 2 * kT;
        nc = cells[qc];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          no[a] = offs[a * n + qc];
          nu[a] = us[a * n + qc];
          nl[a] = us[(a + 3) * n + qc];
        }
        if (w) nw = w[qc];
      }
      if (w && wd != w) wd[p] = wcur;             // carry the read-only planes over
      if (ids && idd != ids) idd[p] = ids[qcur];
      int j[3];
      cell_coords(g, ccur, j);
      int l[3];
      bool ok = true;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        l[a] = j[a] - org[a];
        ok = ok && l[a] >= 0 && l[a] < g.b[a];
      }
      if (ok) {  // the particle must sit in the cell it was sorted into
        const int lc = (l[2] * g.b[1] + l[1]) * g.b[0] + l[0];
        ok = p >= scs[lc] && p < scs[lc + 1];
      }
      float F[3] = {0.0f, 0.0f, 0.0f};
      float d0[3] = {0.0f, 0.0f, 0.0f};
      if (!ok) {
        atomicOr(status, ST_DOMAIN);
        if (outmask) outmask[p] = 0;
        cell[p] = ccur;  // left as it was
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          off[a * n + p] = o[a];
          u[a * n + p] = up[a];
          u[(a + 3) * n + p] = ul[a];
        }
      } else {
        float wx[3], wy[3], wz[3] = {0.0f, 1.0f, 0.0f};
        shape_weights<SHAPE>(o[0], wx);
        shape_weights<SHAPE>(o[1], wy);
        if (DIM == 3) shape_weights<SHAPE>(o[2], wz);
        float2 f2[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        const float4* sb4 = reinterpret_cast<const float4*>(sbox);
#pragma unroll
        for (int kz = (DIM == 3 ? 0 : 1); kz < (DIM == 3 ? 3 : 2); ++kz) {
          const int zz = DIM == 3 ? l[2] + kz : 0;
#pragma unroll
          for (int ky = 0; ky < 3; ++ky) {
            const float wzy = wz[kz] * wy[ky];
            const int row = (zz * g.box[1] + l[1] + ky) * g.box[0] + l[0];
#pragma unroll
            for (int kx = 0; kx < 3; ++kx)
              acc_point(f2, wzy * wx[kx], sb4[2 * (row + kx)], sb4[2 * (row + kx) + 1]);
          }
        }
        float du[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) d0[a] = o[a];
        boris_f32(up, ul, f2, h, hl, du);
        const float gi = rsqrtf(1.0f + (up[0] * up[0] + up[1] * up[1] + up[2] * up[2]));
        bool out = false;
#pragma unroll
        for (int a = 0; a < DIM; ++a)
          move_axis(o[a], j[a], up[a] * gi * dtdx[a], g.n[a], g.open[a], out);
        if (!(isfinite(up[0]) && isfinite(up[1]) && isfinite(up[2]) && isfinite(o[0]) &&
              isfinite(o[1]) && isfinite(o[2])))
          atomicOr(status, ST_NONFINITE);
        if (outmask) outmask[p] = out ? 1 : 0;
        cell[p] = (j[2] * g.n[1] + j[1]) * g.n[0] + j[0];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          off[a * n + p] = o[a];
          u[a * n + p] = up[a];
          u[(a + 3) * n + p] = ul[a];
        }
        if (DEP) {
          const float wdt = wcur * inv_dt;
#pragma unroll
          for (int a = 0; a < 3; ++a) F[a] = du[a] * wdt;
        }
      }
      if (DEP) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          rd[a * kR + i] = d0[a];
          rF[a * kR + i] = F[a];
        }
      }
    }
    if (sb + kM < p1) prefetch(sb + kM);
    if (!DEP) continue;
    __syncthreads();
    // ---- B: one thread per (source cell, component) of this super-chunk
    // sums its particles' 27 contributions, then 27 (3^dim) ordered passes
    const int hz = DIM == 3 ? 1 : 0;
    // cells of this super-chunk: cfirst holds slot sb, clast is the last cell
    // with a slot below se (binary searches of the brick's cell_start)
    cfirst = first_above(scs, 1, g.V, sb) - 1;
    const int clast = first_above(scs, 0, g.V, se - 1) - 1;
    constexpr int CB = kT / 3;  // cells per batch
    const int comp = tid % 3;
    for (int c0 = cfirst; c0 <= clast; c0 += CB) {
      const int ls = c0 + tid / 3;
      float T[27];
#pragma unroll
      for (int k = 0; k < 27; ++k) T[k] = 0.0f;
      bool any = false;
      int lx = 0, ly = 0, lz = 0;
      if (tid < 3 * CB && ls <= clast) {
        lx = ls & (g.b[0] - 1);   // brick sides are powers of two
        ly = (ls >> g.bshift[0]) & (g.b[1] - 1);
        lz = ls >> (g.bshift[0] + g.bshift[1]);
        uint32_t r0 = scs[ls], r1 = scs[ls + 1];
        r0 = r0 > sb ? r0 : sb;
        r1 = r1 < se ? r1 : se;
        for (uint32_t r = r0; r < r1; ++r) {
          const int i = (int)(r - sb);
          float wx[3], wy[3], wz[3] = {0.0f, 1.0f, 0.0f};
          shape_weights<SHAPE>(rd[i], wx);
          shape_weights<SHAPE>(rd[kR + i], wy);
          if (DIM == 3) shape_weights<SHAPE>(rd[2 * kR + i], wz);
          const float Fc = rF[comp * kR + i];
          const float wxF[3] = {wx[0] * Fc, wx[1] * Fc, wx[2] * Fc};
#pragma unroll
          for (int kz = (DIM == 3 ? 0 : 1); kz < (DIM == 3 ? 3 : 2); ++kz)
#pragma unroll
            for (int ky = 0; ky < 3; ++ky) {
              const float wzy = wz[kz] * wy[ky];
#pragma unroll
              for (int kx = 0; kx < 3; ++kx)
                T[(kz * 3 + ky) * 3 + kx] = fmaf(wzy, wxF[kx], T[(kz * 3 + ky) * 3 + kx]);
            }
          any = true;
        }
      }
      // target of stencil offset (kx, ky, kz) in the haloed tile:
      // a0 + kz * sz + ky * e0 + kx
      const int sz = g.e[0] * g.e[1];
      float2* a0 = acc + comp * L.evp + ((lz + hz - 1) * g.e[1] + ly) * g.e[0] + lx;
#pragma unroll
      for (int kz = (DIM == 3 ? 0 : 1); kz < (DIM == 3 ? 3 : 2); ++kz)
#pragma unroll
        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
          for (int kx = 0; kx < 3; ++kx) {
            if (any) {
              float2* a = a0 + kz * sz + ky * g.e[0] + kx;
              *a = two_sum_add(*a, T[(kz * 3 + ky) * 3 + kx]);
            }
            __syncthreads();
          }
    }
  }
  if (DEP) {
    __syncthreads();
    for (int t = tid; t < g.ev; t += kT)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        dpart[(brick * 3 + c) * g.ev + t] =
            (double)acc[c * L.evp + t].x + (double)acc[c * L.evp + t].y;
  }
}

// ---- 3D brick kernel with deposit, one brick plane at a time --------------
// The brick's 8^3 cells are numbered x fastest, so each z-plane of 8 x 8
// cells holds a contiguous range of the sorted particles.  A plane's
// particles are taken in chunks of up to kM3 (one chunk unless the plane
// holds more than kM3 particles); per chunk:
//   A.  push, one thread per particle, as in the kernel above; a record of the
//       gather weights (at x^n) and the force w du/dt goes to shared memory;
//   B1. one thread per (cell, kz) sums, over the cell's particles in index
//       order, the 27 contributions (ky, kx, component) that land in tile
//       plane lz + kz: the same f32 products, summed in the same order, as
//       the per-cell sums of the kernel above.  Cells are handed to threads
//       fullest first, so a warp's lanes loop over similar counts;
//   B2. the sums go to shared memory (over the records, no longer needed);
//   B3. one thread per (pair of x-adjacent targets, component, kz) takes the
//       sums of the up to 9 source cells that reach each target, in a fixed
//       order, into a two-float value (TwoSum), and adds that into a rolling
//       window of three tile planes held as two-float accumulators.  No two
//       threads share a target, so no ordered passes are needed.
//   B4. tile planes that no later source plane reaches are written out as
//       FP64 partials (hi + lo) and their window slots cleared, by the threads
//       that B1 leaves idle (the rest at the end of the brick).
// Four barriers per chunk, where the kernel above takes 27 per batch of
// cells.  The field box is staged as a ring of four tile planes, each copied
// by TMA once no plane's stencil needs the one it replaces: 52 KB of shared
// memory, three CTAs per SM, and room left in L1 for the state's loads
// through the sort's permutation.
constexpr int kB3 = 8;             // brick side (3D)
constexpr int kE3 = kB3 + 2;       // haloed tile side
constexpr int kPC = kB3 * kB3;     // cells in a brick plane
constexpr int kPT = kE3 * kE3;     // cells in a tile plane
constexpr int kM3 = 640;           // particles per chunk (a plane holds ~512 at 8 per cell)
// record floats: (F[3], wx0), (wy[3], wx1), (wz[3], wx2) -- F and wy start
// 16-byte rows, so the per-cell sums read (F0, F1) and (wy0, wy1) as aligned
// pairs for the paired multiplies
constexpr int kRec = 12;
// stride of the plane sums per (component, kz): 9 * 64 + 11 floats, so the
// three kz lanes of a cell store to different banks
constexpr int kTS = 9 * kPC + 11;

constexpr int kSlots = 4;          // tile planes staged at once (a ring)
constexpr int kPlaneF = 8 * kPT;   // floats per staged tile plane (8 per cell)

struct Mixed3Smem {
  size_t cs, bar, rec, win, total;
};
__host__ __device__ inline Mixed3Smem mixed3_smem() {
  Mixed3Smem s;
  s.cs = align_up((size_t)kSlots * kPlaneF * 4, 128);
  s.bar = align_up(s.cs + (size_t)(kB3 * kB3 * kB3 + 1) * 4, 16);
  s.rec = align_up(s.bar + 8 * kSlots + 16 + 32 * 4 + 64, 128);
  const size_t rb = (size_t)kM3 * kRec * 4, tb = (size_t)9 * kTS * 4;
  s.win = align_up(s.rec + (rb > tb ? rb : tb), 16);
  s.total = s.win + (size_t)3 * 3 * kPT * 8;
  return s;
}

// Knuth's TwoSum on two lanes: s + v = s' + err exactly in each; err joins e.
__device__ __forceinline__ void two_sum_acc2(float2& s, float2& e, float2 v) {
  const float2 t = add2(s, v);
  const float2 bp = sub2(t, s);
  e = add2(e, add2(sub2(s, sub2(t, bp)), sub2(v, bp)));
  s = t;
}

// Warp 0: order the 64 cells of a brick plane by their particle count in the
// slot range [sb, se), fullest first (counts above 31 rank as 31), so that
// the lanes of each B1 warp loop over cells of similar counts.  ord[r] is the
// cell of rank r.  Equal counts come in any order: which thread sums a cell
// does not change its sums.
__device__ __forceinline__ void rank_cells(const uint32_t* cs, uint32_t sb, uint32_t se,
                                           int* cur, uint8_t* ord, int lane) {
  auto count = [&](int c) -> int {
    const uint32_t a = cs[c] > sb ? cs[c] : sb, b = cs[c + 1] < se ? cs[c + 1] : se;
    const int k = b > a ? (int)(b - a) : 0;
    return k < 31 ? k : 31;
  };
  const int na = count(lane), nb = count(lane + 32);
  cur[lane] = 0;
  __syncwarp();
  atomicAdd(&cur[na], 1);
  atomicAdd(&cur[nb], 1);
  __syncwarp();
  // cells with a count above v, for lane v: a suffix sum over the lanes
  const int h = cur[lane];
  int suf = h;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int t = __shfl_down_sync(0xffffffffu, suf, d);
    if (lane + d < 32) suf += t;
  }
  __syncwarp();
  cur[lane] = suf - h;
  __syncwarp();
  ord[atomicAdd(&cur[na], 1)] = (uint8_t)lane;
  ord[atomicAdd(&cur[nb], 1)] = (uint8_t)(lane + 32);
}

template <int SHAPE>
__global__ void __launch_bounds__(kT, 3)
    k_boris_brick_mixed3_dep(const __grid_constant__ CUtensorMap tmap, const Geo g,
                             const int32_t* cells, const float* offs, const float* us,
                             const float* w, const uint64_t* ids, int32_t* cell, float* off,
                             float* u, float* wd, uint64_t* idd, int64_t n,
                             const uint32_t* __restrict__ perm,
                             const uint32_t* __restrict__ cstart, double* __restrict__ dpart,
                             float h, float hl, float dtdx0, float dtdx1, float dtdx2,
                             float inv_dt, int* __restrict__ status,
                             uint8_t* __restrict__ outmask) {
  extern __shared__ __align__(128) unsigned char smem[];
  const Mixed3Smem L = mixed3_smem();
  const int tid = threadIdx.x;
  constexpr int kV3 = kB3 * kB3 * kB3;
  float* sbox = reinterpret_cast<float*>(smem);           // [slot][100 cells][8]
  uint32_t* scs = reinterpret_cast<uint32_t*>(smem + L.cs);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar);  // one per slot
  int* sflag = reinterpret_cast<int*>(smem + L.bar + 8 * kSlots);
  int* scur = reinterpret_cast<int*>(smem + L.bar + 8 * kSlots + 16);      // [32] cell ranking
  uint8_t* sord = reinterpret_cast<uint8_t*>(smem + L.bar + 8 * kSlots + 16 + 32 * 4);  // [64]
  float* rec = reinterpret_cast<float*>(smem + L.rec);   // chunk records, then plane sums
  float2* win = reinterpret_cast<float2*>(smem + L.win);  // [slot][component][100] (hi, lo)

  const int64_t brick = blockIdx.x;
  const int bx = (int)(brick % g.nb[0]);
  const int by = (int)((brick / g.nb[0]) % g.nb[1]);
  const int bz = (int)(brick / ((int64_t)g.nb[0] * g.nb[1]));
  const int org[3] = {bx * kB3, by * kB3, bz * kB3};

  // Tile plane tz (0..9) is staged in slot tz % kSlots; its copy completes
  // phase tz / kSlots of that slot's barrier.  Thread 0 issues the copies:
  // planes 0..3 now, plane lz + 4 once source plane lz is done with plane lz.
  auto stage = [&](int tz) {
    mbar_arrive_expect_tx(&bar[tz % kSlots], (uint32_t)(kPlaneF * 4));
    tma_load_4d(sbox + (tz % kSlots) * kPlaneF, &tmap, &bar[tz % kSlots], 0, org[0], org[1],
                org[2] + tz);
  };
  auto staged = [&](int tz) { return mbar_wait_bounded(&bar[tz % kSlots], (tz / kSlots) & 1); };
  if (tid == 0) {
    for (int k = 0; k < kSlots; ++k) mbar_init(&bar[k], 1);
    *sflag = 0;
  }
  __syncthreads();
  if (tid == 0)
    for (int tz = 0; tz < kSlots; ++tz) stage(tz);
  for (int i = tid; i <= kV3; i += kT) scs[i] = cstart[brick * kV3 + i];
  for (int i = tid; i < 3 * 3 * kPT; i += kT) win[i] = make_float2(0.0f, 0.0f);
  __syncthreads();

  const float dtdx[3] = {dtdx0, dtdx1, dtdx2};
  const uint32_t p1 = scs[kV3];
  // end of the chunk that starts at slot s (s < p1): the end of s's plane or
  // s + kM3, whichever comes first
  auto chunk_end = [&](uint32_t s) -> uint32_t {
    int z = 0;
    while (scs[(z + 1) * kPC] <= s) ++z;
    const uint32_t pe = scs[(z + 1) * kPC];
    return pe - s < (uint32_t)kM3 ? pe : s + kM3;
  };
  // state of each thread's first particle of a chunk, loaded before the
  // previous chunk's deposit so that phase A starts with it at hand
  int32_t nc = 0;
  float no[3] = {0.f, 0.f, 0.f}, nu[3] = {0.f, 0.f, 0.f}, nl[3] = {0.f, 0.f, 0.f}, nw = 1.0f;
  uint32_t qc = 0, qn = 0;
  auto prefetch = [&](uint32_t sbx, uint32_t sex) {
    const uint32_t px = sbx + tid;
    qc = px;
    qn = px + kT;
    if (perm) {
      if (px < sex) qc = perm[px];
      if (px + kT < sex) qn = perm[px + kT];
    }
    if (px < sex) {
      nc = cells[qc];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        no[a] = offs[a * n + qc];
        nu[a] = us[a * n + qc];
        nl[a] = us[(a + 3) * n + qc];
      }
      if (w) nw = w[qc];
    }
  };
  if (scs[0] < p1) prefetch(scs[0], chunk_end(scs[0]));

  const int blc = tid / 3, bkz = tid - 3 * (tid / 3);  // B1 role (tid < 3 * kPC)
  // tile planes below zw have been written out; tile plane z is complete
  // once source plane z is, and is written out by the threads that B1 leaves
  // idle (before the next pull needs its slot), or at the end
  int zw = 0;
  auto write_out = [&](int z, int t0, int nt) {
    float2* ws = win + (z % 3) * 3 * kPT;
    for (int i = t0; i < 3 * kPT; i += nt) {
      const int c = i / kPT, t = i - c * kPT;
      const float2 v = ws[i];
      dpart[(brick * 3 + c) * g.ev + z * kPT + t] = (double)v.x + (double)v.y;
      ws[i] = make_float2(0.0f, 0.0f);
    }
  };
  for (int lz = 0; lz < kB3; ++lz) {
    const uint32_t pb = scs[lz * kPC], pe = scs[(lz + 1) * kPC];
    // the stencils of plane lz reach tile planes lz .. lz + 2
    if (pb < pe && !(staged(lz) && staged(lz + 1) && staged(lz + 2))) atomicOr(sflag, 1);
    const float4* pz[3] = {reinterpret_cast<const float4*>(sbox + (lz % kSlots) * kPlaneF),
                           reinterpret_cast<const float4*>(sbox + ((lz + 1) % kSlots) * kPlaneF),
                           reinterpret_cast<const float4*>(sbox + ((lz + 2) % kSlots) * kPlaneF)};
    for (uint32_t sb = pb; sb < pe; sb += kM3) {
      const uint32_t se = pe - sb < (uint32_t)kM3 ? pe : sb + kM3;
      if (tid < 32) rank_cells(scs + lz * kPC, sb, se, scur, sord, tid);
      // ---- A: push, one thread per particle; the permutation is read two
      // slots ahead and the state one slot ahead of the computation
      for (uint32_t p = sb + tid; p < se; p += kT) {
        const int i = (int)(p - sb);
        const int32_t ccur = nc;
        float o[3] = {no[0], no[1], no[2]}, up[3] = {nu[0], nu[1], nu[2]};
        float ul[3] = {nl[0], nl[1], nl[2]};
        const float wcur = nw;
        const uint32_t qcur = qc;
        if (p + kT < se) {
          qc = qn;
          if (p + 2 * kT < se) qn = perm ? perm[p + 2 * kT] : p + 2 * kT;
          nc = cells[qc];
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            no[a] = offs[a * n + qc];
            nu[a] = us[a * n + qc];
            nl[a] = us[(a + 3) * n + qc];
          }
          if (w) nw = w[qc];
        }
        if (w && wd != w) wd[p] = wcur;  // carry the read-only planes over
        if (ids && idd != ids) idd[p] = ids[qcur];
        int j[3];
        cell_coords(g, ccur, j);
        int l[3];
        bool ok = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          l[a] = j[a] - org[a];
          ok = ok && l[a] >= 0 && l[a] < kB3;
        }
        if (ok) {  // the particle must sit in the cell it was sorted into
          const int lc = (l[2] * kB3 + l[1]) * kB3 + l[0];
          ok = p >= scs[lc] && p < scs[lc + 1];
        }
        float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0;
        if (!ok) {
          atomicOr(status, ST_DOMAIN);
          if (outmask) outmask[p] = 0;
          cell[p] = ccur;  // left as it was
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            off[a * n + p] = o[a];
            u[a * n + p] = up[a];
            u[(a + 3) * n + p] = ul[a];
          }
        } else {
          float wx[3], wy[3], wz[3];
          shape_weights<SHAPE>(o[0], wx);
          shape_weights<SHAPE>(o[1], wy);
          shape_weights<SHAPE>(o[2], wz);
          float2 f2[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
          const int c0 = 2 * (l[1] * kE3 + l[0]);  // the stencil's first cell in a tile plane
#pragma unroll
          for (int kz = 0; kz < 3; ++kz)
#pragma unroll
            for (int ky = 0; ky < 3; ++ky) {
              const float wzy = wz[kz] * wy[ky];
              const float4* row = pz[kz] + c0 + 2 * ky * kE3;
#pragma unroll
              for (int kx = 0; kx < 3; ++kx)
                acc_point(f2, wzy * wx[kx], row[2 * kx], row[2 * kx + 1]);
            }
          float du[3];
          boris_f32(up, ul, f2, h, hl, du);
          const float gi = rsqrtf(1.0f + (up[0] * up[0] + up[1] * up[1] + up[2] * up[2]));
          bool out = false;
#pragma unroll
          for (int a = 0; a < 3; ++a)
            move_axis(o[a], j[a], up[a] * gi * dtdx[a], g.n[a], g.open[a], out);
          if (!(isfinite(up[0]) && isfinite(up[1]) && isfinite(up[2]) && isfinite(o[0]) &&
                isfinite(o[1]) && isfinite(o[2])))
            atomicOr(status, ST_NONFINITE);
          if (outmask) outmask[p] = out ? 1 : 0;
          cell[p] = (j[2] * g.n[1] + j[1]) * g.n[0] + j[0];
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            off[a * n + p] = o[a];
            u[a * n + p] = up[a];
            u[(a + 3) * n + p] = ul[a];
          }
          const float wdt = wcur * inv_dt;
          r0 = make_float4(du[0] * wdt, du[1] * wdt, du[2] * wdt, wx[0]);
          r1 = make_float4(wy[0], wy[1], wy[2], wx[1]);
          r2 = make_float4(wz[0], wz[1], wz[2], wx[2]);
        }
        float4* rq = reinterpret_cast<float4*>(rec + i * kRec);
        rq[0] = r0;
        rq[1] = r1;
        rq[2] = r2;
      }
      if (se < p1) prefetch(se, chunk_end(se));
      __syncthreads();
      if (*sflag) {  // a staging copy did not complete: wait for ours (bounded), give up
        if (tid == 0) {
          atomicOr(status, ST_TIMEOUT);
          for (int tz = lz; tz < kE3 && tz < lz + kSlots; ++tz) staged(tz);
        }
        return;
      }
      // ---- B1: one thread per (cell, kz) of this plane
      float2 T01[9];  // (component 0, component 1) of target (ky, kx): index ky * 3 + kx
      float2 T2p[3];  // component 2 of targets (0, kx) and (1, kx)
      float T2s[3];   // component 2 of target (2, kx)
#pragma unroll
      for (int k = 0; k < 9; ++k) T01[k] = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        T2p[k] = make_float2(0.0f, 0.0f);
        T2s[k] = 0.0f;
      }
      if (tid >= 3 * kPC) {
        for (int z = zw; z < lz; ++z) write_out(z, tid - 3 * kPC, kT - 3 * kPC);
      } else {
        const int cl = sord[blc];  // the cell of rank blc
        uint32_t ra = scs[lz * kPC + cl], rb = scs[lz * kPC + cl + 1];
        ra = ra > sb ? ra : sb;
        rb = rb < se ? rb : se;
        const float4* q = reinterpret_cast<const float4*>(rec) + (ra - sb) * (kRec / 4);
        for (uint32_t r = ra; r < rb; ++r, q += kRec / 4) {
          const float4 a = q[0], b = q[1], c4 = q[2];
          const float wzk = bkz == 0 ? c4.x : (bkz == 1 ? c4.y : c4.z);
          const float2 P01 = __fmul2_rn(make_float2(wzk, wzk), make_float2(b.x, b.y));
          const float P2 = wzk * b.z;
          const float P[3] = {P01.x, P01.y, P2};
          const float2 F01 = make_float2(a.x, a.y);
          const float wx[3] = {a.w, b.w, c4.w};
#pragma unroll
          for (int kx = 0; kx < 3; ++kx) {
            const float2 Q01 = __fmul2_rn(make_float2(wx[kx], wx[kx]), F01);
            const float Q2 = wx[kx] * a.z;
#pragma unroll
            for (int ky = 0; ky < 3; ++ky)
              T01[ky * 3 + kx] = __ffma2_rn(make_float2(P[ky], P[ky]), Q01, T01[ky * 3 + kx]);
            T2p[kx] = __ffma2_rn(P01, make_float2(Q2, Q2), T2p[kx]);
            T2s[kx] = fmaf(P2, Q2, T2s[kx]);
          }
        }
      }
      __syncthreads();
      // ---- B2: the chunk's per-cell sums to shared memory
      if (tid < 3 * kPC) {
        const int cl = sord[blc];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          rec[(0 * 3 + bkz) * kTS + k * kPC + cl] = T01[k].x;
          rec[(1 * 3 + bkz) * kTS + k * kPC + cl] = T01[k].y;
          rec[(2 * 3 + bkz) * kTS + k * kPC + cl] =
              k < 3 ? T2p[k].x : (k < 6 ? T2p[k - 3].y : T2s[k - 6]);
        }
      }
      __syncthreads();
      // ---- B3: pull into the window, targets (tx, tx + 1) of tile row ty in
      // tile plane lz + kz, one component
      for (int it = tid; it < 3 * 3 * kE3 * (kE3 / 2); it += kT) {
        const int txp = it % (kE3 / 2);
        int r = it / (kE3 / 2);
        const int ty = r % kE3;
        r /= kE3;
        const int kz = r % 3;
        const int c = r / 3;
        const int tx = 2 * txp;
        const float* Tb = rec + (c * 3 + kz) * kTS;
        float2 s = make_float2(0.0f, 0.0f), e = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int ky = 0; ky < 3; ++ky) {
          const int ly = ty - ky;
          const bool yok = ly >= 0 && ly < kB3;
#pragma unroll
          for (int kx = 0; kx < 3; ++kx) {
            const int la = tx - kx, lb = tx + 1 - kx;
            const float* row = Tb + (ky * 3 + kx) * kPC + ly * kB3;
            float2 v = make_float2(0.0f, 0.0f);
            if (yok && la >= 0 && la < kB3) v.x = row[la];
            if (yok && lb >= 0 && lb < kB3) v.y = row[lb];
            two_sum_acc2(s, e, v);
          }
        }
        float4* wp = reinterpret_cast<float4*>(win + (((lz + kz) % 3) * 3 + c) * kPT + ty * kE3 + tx);
        const float4 acc = *wp;  // (hi, lo) of target tx, then of tx + 1
        float2 hi = make_float2(acc.x, acc.z), lo = make_float2(acc.y, acc.w);
        two_sum_acc2(hi, lo, s);
        lo = add2(lo, e);
        *wp = make_float4(hi.x, lo.x, hi.y, lo.y);
      }
      __syncthreads();
      zw = lz;
    }
    // tile plane lz is read by no later plane: its slot takes plane lz + 4
    // (after the slot's previous copy, bounded, should nobody have waited)
    if (tid == 0 && lz + kSlots < kE3) {
      if (staged(lz))
        stage(lz + kSlots);
      else
        atomicOr(sflag, 1);  // seen after the next barrier
    }
  }
  // ---- B4: the tile planes not yet written out
  for (int z = zw; z < kE3; ++z) write_out(z, tid, kT);
  // the copies into slots that were not refilled: waited for before the exit
  // (at once if a plane's stencils already did)
  if (tid == 0) {
    bool ok = *sflag == 0;
    for (int tz = kE3 - kSlots; tz < kE3; ++tz) ok = staged(tz) && ok;
    if (!ok) atomicOr(status, ST_TIMEOUT);
  }
}

// nsteps fused steps of one particle in registers: gather from the padded
// global f32 copy, Boris, move.  Shared by the particle-order kernel and the
// serving kernel so a particle gets the same bits whichever runs it.
template <int SHAPE, int DIM>
__device__ __forceinline__ void advance_mixed(const float* __restrict__ fp, const Geo& g, int* j,
                                              float* o, float* up, float* ul, float h, float hl,
                                              const float* dtdx, int nsteps, bool& out) {
  for (int st = 0; st < nsteps && !out; ++st) {
    float wx[3], wy[3], wz[3] = {0.0f, 1.0f, 0.0f};
    shape_weights<SHAPE>(o[0], wx);
    shape_weights<SHAPE>(o[1], wy);
    if (DIM == 3) shape_weights<SHAPE>(o[2], wz);
    float2 f2[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    const ulonglong4_32a* __restrict__ fp8 = reinterpret_cast<const ulonglong4_32a*>(fp);
#pragma unroll
    for (int kz = (DIM == 3 ? 0 : 1); kz < (DIM == 3 ? 3 : 2); ++kz) {
      const int zz = DIM == 3 ? j[2] + kz : 0;
#pragma unroll
      for (int ky = 0; ky < 3; ++ky) {
        const float wzy = wz[kz] * wy[ky];
        const int64_t row = ((int64_t)zz * g.pn[1] + j[1] + ky) * g.pn[0] + j[0];
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
          // one 32-byte load per stencil point (the cell's 8 floats)
          const ulonglong4_32a v = fp8[row + kx];
          acc_point(f2, wzy * wx[kx],
                    make_float4(__uint_as_float((uint32_t)v.x), __uint_as_float((uint32_t)(v.x >> 32)),
                                __uint_as_float((uint32_t)v.y), __uint_as_float((uint32_t)(v.y >> 32))),
                    make_float4(__uint_as_float((uint32_t)v.z), __uint_as_float((uint32_t)(v.z >> 32)),
                                0.0f, 0.0f));
        }
      }
    }
    float du[3];
    boris_f32(up, ul, f2, h, hl, du);
    const float gi = rsqrtf(1.0f + (up[0] * up[0] + up[1] * up[1] + up[2] * up[2]));
#pragma unroll
    for (int a = 0; a < DIM; ++a)
      move_axis(o[a], j[a], up[a] * gi * dtdx[a], g.n[a], g.open[a], out);
  }
}

// Load one particle (stride = row stride of the SoA arrays), advance, store.
template <int SHAPE, int DIM>
__device__ __forceinline__ void particle_mixed(const float* __restrict__ fp, const Geo& g,
                                               int32_t* __restrict__ cell, float* __restrict__ off,
                                               float* __restrict__ u, int64_t stride, int64_t p,
                                               float h, float hl, const float* dtdx, int nsteps,
                                               int* __restrict__ status,
                                               uint8_t* __restrict__ outmask) {
  int32_t c = cell[p];
  bool bad = false;
  if (c < 0 || c >= g.G) {
    bad = true;
    c = 0;
  }
  int j[3];
  cell_coords(g, c, j);
  float o[3], up[3], ul[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    o[a] = off[a * stride + p];
    up[a] = u[a * stride + p];
    ul[a] = u[(a + 3) * stride + p];
  }
  bool out = false;
  advance_mixed<SHAPE, DIM>(fp, g, j, o, up, ul, h, hl, dtdx, nsteps, out);
  if (outmask) outmask[p] = out ? 1 : 0;
  if (bad || !(isfinite(up[0]) && isfinite(up[1]) && isfinite(up[2]) && isfinite(o[0]) &&
               isfinite(o[1]) && isfinite(o[2])))
    atomicOr(status, bad ? ST_DOMAIN : ST_NONFINITE);
  cell[p] = (j[2] * g.n[1] + j[1]) * g.n[0] + j[0];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    off[a * stride + p] = o[a];
    u[a * stride + p] = up[a];
    u[(a + 3) * stride + p] = ul[a];
  }
}

template <int SHAPE, int DIM>
__global__ void __launch_bounds__(256)
    k_boris_particles_mixed(const float* __restrict__ fp, const Geo g, int32_t* __restrict__ cell,
                            float* __restrict__ off, float* __restrict__ u, int64_t n, float h,
                            float hl, float dtdx0, float dtdx1, float dtdx2, int nsteps,
                            int* __restrict__ status, uint8_t* __restrict__ outmask) {
  const float dtdx[3] = {dtdx0, dtdx1, dtdx2};
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x)
    particle_mixed<SHAPE, DIM>(fp, g, cell, off, u, n, p, h, hl, dtdx, nsteps, status, outmask);
}

// Persistent serving kernel: each CTA claims the next unclaimed work item
// (one atomic on the work list's counter per item; the host lists the items
// costliest first), so CTAs finish a round together however uneven the
// items are.  No CTA waits on another.  Each item is a slice of one
// request's particles to advance nsteps steps against one resident field
// snapshot; every particle gets the same arithmetic whichever CTA takes it.
// The per-item step parameters are formed in FP64 exactly as the host forms
// them for part_gather_push.
template <int SHAPE, int DIM>
__global__ void __launch_bounds__(512)
    k_serve_mixed(ServeHeader* __restrict__ hdr, const part_work_item* __restrict__ items,
                  const SnapEntry* __restrict__ snaps, int nsnap, int* __restrict__ status) {
  __shared__ part_work_item s_it;
  __shared__ SnapEntry s_sn;
  __shared__ float s_par[5];
  __shared__ int s_next;
  const int nitems = hdr->nitems;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_next = (int)atomicAdd(&hdr->next, 1u);
    __syncthreads();
    const int it = s_next;
    if (it >= nitems) break;
    if (threadIdx.x == 0) {
      s_it = items[it];
      int sn = s_it.snapshot;
      if (sn < 0 || sn >= nsnap) {
        atomicOr(status, ST_DOMAIN);
        s_it.count = 0;
        sn = 0;
      }
      s_sn = snaps[sn];
      const double hd = 0.5 * s_it.q_over_m * s_it.dt;
      s_par[0] = (float)hd;
      s_par[1] = (float)(hd - (double)s_par[0]);
      for (int a = 0; a < 3; ++a) s_par[2 + a] = (float)(s_it.dt / s_sn.g.dx[a]);
    }
    __syncthreads();
    const float dtdx[3] = {s_par[2], s_par[3], s_par[4]};
    for (int64_t q = threadIdx.x; q < s_it.count; q += blockDim.x)
      particle_mixed<SHAPE, DIM>(s_sn.fp, s_sn.g, s_it.cell, s_it.off, s_it.u, s_it.stride,
                                 s_it.first + q, s_par[0], s_par[1], dtdx, s_it.nsteps, status,
                                 nullptr);
  }
}

struct MixedArgs {
  float h, hl, dtdx[3], inv_dt;  // h + hl: the half step (q/m) dt/2 as two floats
};

MixedArgs mixed_args(const part_ctx* c, double qm, double dt) {
  MixedArgs a;
  const double hd = 0.5 * qm * dt;
  a.h = (float)hd;
  a.hl = (float)(hd - (double)a.h);
  for (int k = 0; k < 3; ++k) a.dtdx[k] = (float)(dt / c->geo.dx[k]);
  a.inv_dt = (float)(1.0 / dt);
  return a;
}

template <int SHAPE, int DIM, bool DEP>
cudaError_t brick_mixed(part_ctx* c, const MixedArgs& a) {
  // 3D with deposit: the plane-by-plane kernel (8^3 bricks, 10^3 staged box)
  const bool planes = DIM == 3 && DEP;
  if (planes && (c->geo.V != kB3 * kB3 * kB3 || c->geo.box[0] != kE3 ||
                 c->geo.box[1] != kE3 || c->geo.box[2] != kE3 || c->geo.ev != kE3 * kE3 * kE3))
    return cudaErrorInvalidConfiguration;
  auto kern = planes ? k_boris_brick_mixed3_dep<SHAPE> : k_boris_brick_mixed<SHAPE, DIM, DEP>;
  const size_t smem_bytes = planes ? mixed3_smem().total : mixed_smem(c->geo).total;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_bytes);
  if (e != cudaSuccess) return e;
  // read the current buffer (through the sort's permutation, if one is
  // pending, into the other buffer; else in place)
  const PState src = state_of(c, c->cur_alt);
  const PState dst = c->perm_pend ? state_of(c, !c->cur_alt) : src;
  kern<<<(unsigned)c->geo.nbricks, kT, smem_bytes, c->stream>>>(
      planes ? c->tmap_plane : c->tmap, c->geo, (const int32_t*)src.x, (const float*)src.off, (const float*)src.u,
      (const float*)src.w, src.id, (int32_t*)dst.x, (float*)dst.off, (float*)dst.u,
      (float*)dst.w, dst.id, c->n, c->perm_pend, c->cstart, c->dpart, a.h, a.hl, a.dtdx[0],
      a.dtdx[1], a.dtdx[2], a.inv_dt, c->status, c->outmask);
  c->launches++;
  if (c->perm_pend) {
    c->perm_pend = nullptr;
    c->cur_alt = !c->cur_alt;
  }
  return cudaGetLastError();
}

template <int SHAPE, int DIM>
cudaError_t dispatch_mixed(part_ctx* c, double qm, double dt, int nsteps) {
  const MixedArgs a = mixed_args(c, qm, dt);
  if (c->sorted && nsteps == 1)
    return c->deposit_on ? brick_mixed<SHAPE, DIM, true>(c, a)
                         : brick_mixed<SHAPE, DIM, false>(c, a);
  const int t = threads_for_spread(c, c->n);
  k_boris_particles_mixed<SHAPE, DIM><<<grid_for(c, c->n, t), t, 0, c->stream>>>(
      (const float*)c->fpad, c->geo, (int32_t*)c->x, (float*)c->off, (float*)c->u, c->n, a.h,
      a.hl, a.dtdx[0], a.dtdx[1], a.dtdx[2], nsteps, c->status, c->outmask);
  c->launches++;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_boris_mixed(part_ctx* c, double qm, double dt, int nsteps) {
  if (c->n == 0) return cudaSuccess;
  const int dim = c->geo.dim;
  if (c->shape == PART_TSC)
    return dim == 3 ? dispatch_mixed<PART_TSC, 3>(c, qm, dt, nsteps)
                    : dispatch_mixed<PART_TSC, 2>(c, qm, dt, nsteps);
  return dim == 3 ? dispatch_mixed<PART_CIC, 3>(c, qm, dt, nsteps)
                  : dispatch_mixed<PART_CIC, 2>(c, qm, dt, nsteps);
}

cudaError_t launch_serve_kernel(int shape, int dim, ServeHeader* hdr,
                                const part_work_item* items, const SnapEntry* snaps, int nsnap,
                                int* status, int grid, int threads, cudaStream_t stream) {
  if (shape == PART_TSC) {
    if (dim == 3)
      k_serve_mixed<PART_TSC, 3><<<grid, threads, 0, stream>>>(hdr, items, snaps, nsnap, status);
    else
      k_serve_mixed<PART_TSC, 2><<<grid, threads, 0, stream>>>(hdr, items, snaps, nsnap, status);
  } else {
    if (dim == 3)
      k_serve_mixed<PART_CIC, 3><<<grid, threads, 0, stream>>>(hdr, items, snaps, nsnap, status);
    else
      k_serve_mixed<PART_CIC, 2><<<grid, threads, 0, stream>>>(hdr, items, snaps, nsnap, status);
  }
  return cudaGetLastError();
}
