// sort.cu -- bit-exact stable cell sort of the bound particles.
//
// keys  : brick-ordered cell key of every particle (integer arithmetic on the
//         cell index j = floor((x - xmin) * (1/dx)), both roundings explicit).
// radix : LSD radix sort of (key, index), 8-bit digits, reduce-then-scan:
//         per-tile digit histograms -> exclusive scan (digit-major) -> stable
//         per-tile scatter ranked with warp match masks.  No inter-CTA waits.
// incremental: after a push that moved every particle by less than a cell,
//         a per-brick stable counting sort over the brick's own and adjacent
//         old cells replaces the radix passes (same permutation).
// permute: Boris modes leave the permutation to the next brick push, which
//         reads the current copy of the state through it and writes the
//         other copy (apply_perm does the same gather when no push follows);
//         LP mode gathers each bound array through the scratch row and copies
//         it back.
// cell_start: cs[k] = first sorted particle with key >= k, k in [0, nkeys].
#include <algorithm>
#include "part_internal.cuh"

namespace {

// Brick sides are powers of two (8^3, 16^2), so the split is by shifts.
__device__ __forceinline__ uint32_t brick_key(const Geo& g, int jx, int jy, int jz) {
  const int bx = jx >> g.bshift[0], by = jy >> g.bshift[1], bz = jz >> g.bshift[2];
  const int lx = jx & (g.b[0] - 1), ly = jy & (g.b[1] - 1), lz = jz & (g.b[2] - 1);
  const uint32_t brick = (uint32_t)((bz * g.nb[1] + by) * g.nb[0] + bx);
  return (brick << g.vshift) |
         (uint32_t)((((lz << g.bshift[1]) | ly) << g.bshift[0]) | lx);
}

// Cell index floor((x - xmin) inv_dx), rounded as in FP64, clamped to
// [0, n-1].  The FP64 rate bounds a pass that only computes keys, so the
// floor is first taken from an f32 image of the same expression: x's f32
// image by truncating its significand on the integer pipe (relative error
// <= 2^-23), then an f32 subtract and multiply.  That value is within
// 1.3 * 2^-22 * (|xmin| inv_dx + |s|) of the exact s, and the FP64 s is
// within a few ulp of it, so whenever the f32 value is farther than
// 4e-7 * (|xmin| inv_dx + |s| + 1) from an integer both floors agree.  The
// rest (about 1e-4 of the positions per axis, and non-finite or huge
// coordinates) take the FP64 expression.
__device__ __forceinline__ int cell_of(const Geo& g, int a, double xa, int* status) {
  {
    const uint32_t hi = (uint32_t)__double2hiint(xa), lo = (uint32_t)__double2loint(xa);
    const int e = (int)((hi >> 20) & 0x7ffu);
    // binary64 exponents that are normal in binary32; +-0 is exact as well
    const bool zero = ((hi & 0x7fffffffu) | lo) == 0u;
    if ((e >= 1023 - 126 && e <= 1023 + 127) || zero) {
      const float xf = zero ? 0.0f
                            : __uint_as_float((hi & 0x80000000u) | ((uint32_t)(e - 896) << 23) |
                                              ((hi & 0xfffffu) << 3) | (lo >> 29));
      const float sf = (xf - g.xminf[a]) * g.inv_dxf[a];
      if (fabsf(sf) < 4194304.0f) {  // 2^22: floorf and the fraction are exact
        const float fl = floorf(sf);
        const float fr = sf - fl;
        const float m = 4e-7f * (g.xmin_cells[a] + fabsf(sf) + 1.0f);
        if (fr > m && fr < 1.0f - m) {
          const int j = (int)fl;
          return j < 0 ? 0 : (j > g.n[a] - 1 ? g.n[a] - 1 : j);
        }
      }
    }
  }
  double s = __dmul_rn(__dsub_rn(xa, g.xmin[a]), g.inv_dx[a]);
  if (!finite_bits(s)) {
    atomicOr(status, ST_NONFINITE);
    return 0;
  }
  return floor_clamp_bits(s, g.n[a] - 1);
}

__global__ void k_keys_f64(const double* __restrict__ x, int64_t n, Geo g,
                           uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                           int* status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int j[3] = {0, 0, 0};
    for (int a = 0; a < g.dim; ++a) j[a] = cell_of(g, a, x[a * n + i], status);
    keys[i] = brick_key(g, j[0], j[1], j[2]);
    vals[i] = (uint32_t)i;
  }
}

__global__ void k_keys_cell(const int32_t* __restrict__ cell, int64_t n, Geo g,
                            uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                            int* status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t c = cell[i];
    if (c < 0 || c >= g.G) {
      atomicOr(status, ST_DOMAIN);
      c = c < 0 ? 0 : (int32_t)(g.G - 1);
    }
    int j[3];
    cell_coords(g, c, j);
    keys[i] = brick_key(g, j[0], j[1], j[2]);
    vals[i] = (uint32_t)i;
  }
}

__global__ void __launch_bounds__(kSortThreads)
    k_radix_hist(const uint32_t* __restrict__ keys, int64_t n, int shift,
                 uint32_t* __restrict__ hist, int64_t ntiles) {
  __shared__ uint32_t h[kRadix];
  const int tid = threadIdx.x;
  h[tid] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll 4
  for (int it = 0; it < kSortItems; ++it) {
    int64_t i = base + it * kSortThreads + tid;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & (kRadix - 1)], 1u);
  }
  __syncthreads();
  hist[(int64_t)tid * ntiles + blockIdx.x] = h[tid];
}

// Block-wide exclusive scan of one value per thread (256 threads).
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_tot,
                                                         uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint32_t wv = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
    uint32_t wi = wv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < (int)(blockDim.x >> 5)) warp_tot[lane] = wi - wv;
    if (lane == 31) *total = wi;
  }
  __syncthreads();
  uint32_t r = warp_tot[warp] + inc - v;
  __syncthreads();
  return r;
}

// Scan phase 1: sums of kScanBlock-element blocks.
__global__ void __launch_bounds__(256) k_scan_reduce(const uint32_t* __restrict__ a, int64_t m,
                                                     uint32_t* __restrict__ sums) {
  __shared__ uint32_t wt[8];
  __shared__ uint32_t tot;
  const int64_t base = (int64_t)blockIdx.x * kScanBlock;
  uint32_t s = 0;
  for (int k = 0; k < kScanBlock / 256; ++k) {
    int64_t i = base + k * 256 + threadIdx.x;
    if (i < m) s += a[i];
  }
  block_exclusive_scan(s, wt, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Scan phase 2: exclusive scan of the block sums in one CTA.  Each thread
// takes a contiguous segment (one block scan in all, whatever the count).
// total (if given) gets the sum of all blocks.
__global__ void __launch_bounds__(256) k_scan_top(uint32_t* __restrict__ sums, int64_t nblk,
                                                  uint32_t* __restrict__ total = nullptr) {
  __shared__ uint32_t wt[8];
  __shared__ uint32_t tot;
  const int64_t per = (nblk + 255) / 256;
  const int64_t b0 = (int64_t)threadIdx.x * per;
  const int64_t b1 = b0 + per < nblk ? b0 + per : nblk;
  uint32_t s = 0;
  for (int64_t i = b0; i < b1; ++i) s += sums[i];
  uint32_t e = block_exclusive_scan(s, wt, &tot);
  for (int64_t i = b0; i < b1; ++i) {
    const uint32_t v = sums[i];
    sums[i] = e;
    e += v;
  }
  if (total && threadIdx.x == 0) *total = tot;
}

// Scan phase 3: exclusive scan inside each block plus its block offset.
__global__ void __launch_bounds__(256) k_scan_down(uint32_t* __restrict__ a, int64_t m,
                                                   const uint32_t* __restrict__ sums) {
  __shared__ uint32_t wt[8];
  __shared__ uint32_t tot;
  const int64_t base = (int64_t)blockIdx.x * kScanBlock;
  const int per = kScanBlock / 256;
  uint32_t v[kScanBlock / 256];
  uint32_t s = 0;
  for (int k = 0; k < per; ++k) {
    int64_t i = base + (int64_t)threadIdx.x * per + k;
    v[k] = i < m ? a[i] : 0;
    s += v[k];
  }
  uint32_t e = block_exclusive_scan(s, wt, &tot) + sums[blockIdx.x];
  for (int k = 0; k < per; ++k) {
    int64_t i = base + (int64_t)threadIdx.x * per + k;
    if (i < m) a[i] = e;
    e += v[k];
  }
}

// Stable scatter of one radix pass.  Warp w of the tile owns the contiguous
// key segment [w*32*ITEMS, (w+1)*32*ITEMS); keys are ranked within the warp
// in index order, then offset by the counts of lower warps and by the scanned
// tile histogram.
__global__ void __launch_bounds__(kSortThreads)
    k_radix_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                    uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n,
                    int shift, const uint32_t* __restrict__ hscan, int64_t ntiles) {
  constexpr int W = kSortThreads / 32;
  __shared__ uint32_t wh[W][kRadix];
  __shared__ uint32_t tbase[kRadix];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < W * kRadix; i += kSortThreads) (&wh[0][0])[i] = 0;
  tbase[tid] = hscan[(int64_t)tid * ntiles + blockIdx.x];
  __syncthreads();
  const int64_t seg = (int64_t)blockIdx.x * kSortTile + (int64_t)warp * 32 * kSortItems;
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t kk[kSortItems], vv[kSortItems], pos[kSortItems];
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    int64_t i = seg + r * 32 + lane;
    bool valid = i < n;
    uint32_t key = valid ? kin[i] : 0u;
    uint32_t val = valid ? vin[i] : 0u;
    uint32_t d = valid ? ((key >> shift) & (kRadix - 1)) : (uint32_t)kRadix;
    uint32_t peers = __match_any_sync(0xffffffffu, d);
    uint32_t rank = __popc(peers & lt);
    int leader = __ffs(peers) - 1;
    uint32_t before = valid ? wh[warp][d] : 0u;
    __syncwarp();
    if (valid && lane == leader) wh[warp][d] = before + __popc(peers);
    __syncwarp();
    kk[r] = key;
    vv[r] = val;
    pos[r] = before + rank;
  }
  __syncthreads();
  {
    uint32_t run = 0;
    for (int w = 0; w < W; ++w) {
      uint32_t t = wh[w][tid];
      wh[w][tid] = run;
      run += t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    int64_t i = seg + r * 32 + lane;
    if (i < n) {
      uint32_t d = (kk[r] >> shift) & (kRadix - 1);
      uint32_t dst = tbase[d] + wh[warp][d] + pos[r];
      if (dst < (uint64_t)n) {  // always true for a consistent histogram
        kout[dst] = kk[r];
        vout[dst] = vv[r];
      }
    }
  }
}

template <typename T>
__global__ void k_gather(const T* __restrict__ src, T* __restrict__ dst,
                         const uint32_t* __restrict__ perm, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
  {
    const uint32_t s = perm[i];
    dst[i] = s < (uint64_t)n ? src[s] : T(0);
  }
}

__global__ void k_cell_start(const uint32_t* __restrict__ sk, int64_t n, int64_t nkeys,
                             uint32_t* __restrict__ cs) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t lo = i == 0 ? 0 : (int64_t)sk[i - 1] + 1;
    int64_t hi = i == n ? nkeys : (int64_t)sk[i];
    if (hi > nkeys) hi = nkeys;
    for (int64_t c = lo; c <= hi; ++c) cs[c] = (uint32_t)i;
  }
}

// One pass over the permutation: every bound plane of particle perm[i] of one
// copy of the state is written to slot i of the other copy.  NX planes of the
// position-like array (3 doubles, or 1 int32 cell) by the template.
template <typename TX, int NX, typename TV, int NU>
__global__ void k_gather_state(const TX* __restrict__ x, const float* __restrict__ off,
                               const TV* __restrict__ u, const TV* __restrict__ w,
                               const uint64_t* __restrict__ id, TX* __restrict__ ax,
                               float* __restrict__ aoff, TV* __restrict__ au,
                               TV* __restrict__ aw, uint64_t* __restrict__ aid,
                               const uint32_t* __restrict__ perm, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t s = perm[i];
    if (s >= (uint64_t)n) continue;  // never for a consistent permutation
#pragma unroll
    for (int a = 0; a < NX; ++a) ax[a * n + i] = x[a * n + s];
    if (off)
#pragma unroll
      for (int a = 0; a < 3; ++a) aoff[a * n + i] = off[a * n + s];
#pragma unroll
    for (int a = 0; a < NU; ++a) au[a * n + i] = u[a * n + s];
    if (w) aw[i] = w[s];
    if (id) aid[i] = id[s];
  }
}

// ---- incremental sort.  When the bound arrays are still in the order of the
// previous sort (old cell_start cs_old: old brick ob owns the contiguous
// segment [cs_old[ob V], cs_old[(ob+1) V])) and every particle has moved by
// less than one cell since, each particle's new brick is its old brick or one
// of the 26 around it: a slot d in 0..26 (per axis: same, +1, -1, periodic).
//   count : per old brick, particles per slot               (coalesced)
//   dest  : per new brick b, its sources in increasing id -> where each
//           source's particles start among b's members; b's member count
//   place : per old brick, each particle's position among its new brick's
//           members, in old-index order (stable within the source)
//   cells : per new brick, stable counting sort of its members by local
//           cell -> perm and the new cell_start
// Members of b in old-index order, sorted stably by local cell, is exactly
// the stable sort by key, so the permutation equals the radix sort's.
constexpr int kIncT = 256;
constexpr int kIncMaxV = 512;

__device__ __forceinline__ void brick_coords(const Geo& g, int64_t b, int* c) {
  c[0] = (int)(b % g.nb[0]);
  c[1] = (int)((b / g.nb[0]) % g.nb[1]);
  c[2] = (int)(b / ((int64_t)g.nb[0] * g.nb[1]));
}

// slot of new brick db seen from old brick ob, or -1 if it is not a
// neighbour (the particle moved more than one cell)
__device__ __forceinline__ int inc_slot(const Geo& g, const int* oc, int64_t db) {
  int dc[3];
  brick_coords(g, db, dc);
  int slot = 0;
  for (int a = 2; a >= 0; --a) {
    const int d = ((dc[a] - oc[a]) % g.nb[a] + g.nb[a]) % g.nb[a];
    const int code = d == 0 ? 0 : d == 1 ? 1 : d == g.nb[a] - 1 ? 2 : -1;
    if (code < 0) return -1;
    slot = slot * 3 + code;
  }
  return slot;
}

// The 27 (possibly repeated) neighbour bricks of ob and their slots, so that
// a particle's slot is a table lookup; ob itself (the common case) is slot 0.
__device__ __forceinline__ void inc_table(const Geo& g, int64_t ob, uint32_t* nid) {
  const int t = threadIdx.x;
  if (t < 27) {
    int oc[3];
    brick_coords(g, ob, oc);
    const int code[3] = {t % 3, (t / 3) % 3, t / 9};  // slot = (cz*3 + cy)*3 + cx
    int nc[3];
    for (int a = 0; a < 3; ++a) {
      const int d = code[a] == 0 ? 0 : code[a] == 1 ? 1 : -1;
      nc[a] = ((oc[a] + d) % g.nb[a] + g.nb[a]) % g.nb[a];
    }
    // a direction that does not exist on this grid (or repeats another) is
    // never the slot a particle gets from inc_slot; keep it out of the table
    const int64_t id = ((int64_t)nc[2] * g.nb[1] + nc[1]) * g.nb[0] + nc[0];
    nid[t] = inc_slot(g, oc, id) == t ? (uint32_t)id : 0xffffffffu;
  }
}

__device__ __forceinline__ int inc_lookup(const uint32_t* nid, uint32_t ob, uint32_t db) {
  if (db == ob) return 0;
  for (int k = 1; k < 27; ++k)
    if (nid[k] == db) return k;
  return -1;
}

// Keys from the current positions (same arithmetic as the full sort) and the
// particle count of every (old brick, slot).  Each thread has kIncItems
// elements in flight: their loads are issued before any of them is used.
constexpr int kIncItems = 4;
template <bool CELL>
__global__ void __launch_bounds__(kIncT)
    k_inc_count(const void* __restrict__ xv, int64_t n, const uint32_t* __restrict__ cs_old, Geo g,
                uint32_t* __restrict__ keys, uint32_t* __restrict__ cnt, int* status) {
  __shared__ uint32_t h[27], nid[27];
  const int64_t ob = blockIdx.x;
  if (threadIdx.x < 27) h[threadIdx.x] = 0;
  inc_table(g, ob, nid);
  __syncthreads();
  const uint32_t s0 = cs_old[ob * g.V], s1 = cs_old[(ob + 1) * g.V];
  // uniform trip count per warp
  for (uint32_t c0 = s0; c0 < s1; c0 += kIncT * kIncItems) {
    int32_t cv[kIncItems];
    double xr[kIncItems][3];
#pragma unroll
    for (int r = 0; r < kIncItems; ++r) {
      const uint32_t i = c0 + r * kIncT + threadIdx.x;
      if (CELL) {
        cv[r] = i < s1 ? ((const int32_t*)xv)[i] : 0;
      } else {
#pragma unroll
        for (int a = 0; a < 3; ++a)
          xr[r][a] = i < s1 && a < g.dim ? ((const double*)xv)[a * n + i] : 0.0;
      }
    }
#pragma unroll
    for (int r = 0; r < kIncItems; ++r) {
      const uint32_t i = c0 + r * kIncT + threadIdx.x;
      int slot = 27;
      if (i < s1) {
        uint32_t key;
        if (CELL) {
          int32_t c = cv[r];
          if (c < 0 || c >= g.G) {
            atomicOr(status, ST_DOMAIN);
            c = c < 0 ? 0 : (int32_t)(g.G - 1);
          }
          int jc[3];
          cell_coords(g, c, jc);
          key = brick_key(g, jc[0], jc[1], jc[2]);
        } else {
          int j[3] = {0, 0, 0};
#pragma unroll
          for (int a = 0; a < 3; ++a)
            if (a < g.dim) j[a] = cell_of(g, a, xr[r][a], status);
          key = brick_key(g, j[0], j[1], j[2]);
        }
        keys[i] = key;
        slot = inc_lookup(nid, (uint32_t)ob, (key >> g.vshift));
        if (slot < 0) {
          atomicOr(status, ST_DOMAIN);
          slot = 27;
        }
      }
      const uint32_t peers = __match_any_sync(0xffffffffu, (uint32_t)slot);
      if (slot < 27 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&h[slot], __popc(peers));
    }
  }
  __syncthreads();
  if (threadIdx.x < 27) cnt[ob * 27 + threadIdx.x] = h[threadIdx.x];
}

// One warp per new brick b: lane d < 27 takes the source brick b - delta(d);
// repeated sources (one or two bricks along an axis) keep their first lane.
// In increasing source id, the count of each (source, slot) is replaced by
// its start among b's members; b's member count goes to bcount.
__global__ void __launch_bounds__(256)
    k_inc_dest(uint32_t* __restrict__ cnt, Geo g, uint32_t* __restrict__ bcount) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < g.nbricks;
       b += nw) {
    int bc[3];
    brick_coords(g, b, bc);
    uint64_t id = ~0ull;
    uint32_t c = 0, slot = 0;
    if (lane < 27 && (g.dim == 3 || lane / 9 == 1)) {
      const int d[3] = {lane % 3 - 1, (lane / 3) % 3 - 1, lane / 9 - 1};
      int sc[3];
      for (int a = 0; a < 3; ++a) sc[a] = ((bc[a] - d[a]) % g.nb[a] + g.nb[a]) % g.nb[a];
      id = ((uint64_t)sc[2] * g.nb[1] + sc[1]) * g.nb[0] + sc[0];
      slot = (uint32_t)inc_slot(g, sc, b);
    }
    const uint32_t peers = __match_any_sync(0xffffffffu, id);
    const bool keep = id != ~0ull && lane == __ffs(peers) - 1;
    if (keep) c = cnt[id * 27 + slot];
    // exclusive prefix of the kept counts in increasing source id
    uint32_t before = 0, total = 0;
    for (int k = 0; k < 27; ++k) {
      const uint64_t idk = __shfl_sync(0xffffffffu, id, k);
      const uint32_t ck = __shfl_sync(0xffffffffu, keep ? c : 0u, k);
      const bool kk = __shfl_sync(0xffffffffu, keep ? 1 : 0, k) != 0;
      if (kk) {
        total += ck;
        if (idk < id) before += ck;
      }
    }
    if (keep) cnt[id * 27 + slot] = before;
    if (lane == 0) bcount[b] = total;
  }
}

// Position of every particle of old brick ob among its new brick's members:
// bbase[db] + start of (ob, slot) + rank within (ob, slot) in index order.
// The brick's particles go in tiles of kIncT * kIncItems; warp w takes the
// tile's w-th run of 32 * kIncItems consecutive particles, so index order is
// (tile, warp, item, lane).  Ranks: earlier lanes of the same item by
// match_any, earlier items of the warp by a per-warp running count, earlier
// warps and tiles by a prefix over the warps' counts.
__global__ void __launch_bounds__(kIncT)
    k_inc_place(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ cs_old, Geo g,
                const uint32_t* __restrict__ start, const uint32_t* __restrict__ bbase,
                uint32_t* __restrict__ memb, uint32_t* __restrict__ mlc, int64_t n) {
  constexpr int W = kIncT / 32;
  __shared__ uint32_t wc[W][28], run[28], nid[27];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t ob = blockIdx.x;
  inc_table(g, ob, nid);
  if (tid < 28) run[tid] = 0;
  const uint32_t s0 = cs_old[ob * g.V], s1 = cs_old[(ob + 1) * g.V];
  const uint32_t lt = (1u << lane) - 1u;
  for (uint32_t c0 = s0; c0 < s1; c0 += kIncT * kIncItems) {
    for (int q = tid; q < W * 28; q += kIncT) (&wc[0][0])[q] = 0;
    __syncthreads();
    const uint32_t seg = c0 + (uint32_t)warp * 32 * kIncItems;
    uint32_t key[kIncItems], rank[kIncItems];
    int slot[kIncItems];
#pragma unroll
    for (int r = 0; r < kIncItems; ++r) {
      const uint32_t i = seg + r * 32 + lane;
      key[r] = i < s1 ? keys[i] : 0u;
    }
#pragma unroll
    for (int r = 0; r < kIncItems; ++r) {
      const uint32_t i = seg + r * 32 + lane;
      int sl = i < s1 ? inc_lookup(nid, (uint32_t)ob, (key[r] >> g.vshift)) : 27;
      if (sl < 0) sl = 27;  // moved too far: reported by the count pass
      slot[r] = sl;
      const uint32_t peers = __match_any_sync(0xffffffffu, (uint32_t)sl);
      rank[r] = wc[warp][sl] + __popc(peers & lt);  // this warp's earlier items
      __syncwarp();
      if (lane == __ffs(peers) - 1) wc[warp][sl] += __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    if (tid < 28) {  // exclusive prefix over the warps, on top of the running count
      uint32_t acc = run[tid];
      for (int w = 0; w < W; ++w) {
        const uint32_t t = wc[w][tid];
        wc[w][tid] = acc;
        acc += t;
      }
      run[tid] = acc;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kIncItems; ++r) {
      if (slot[r] < 27) {
        const uint32_t i = seg + r * 32 + lane;
        const uint32_t db = (key[r] >> g.vshift);
        const uint64_t pos =
            (uint64_t)bbase[db] + start[ob * 27 + slot[r]] + wc[warp][slot[r]] + rank[r];
        if (pos < (uint64_t)n) {
          memb[pos] = i;
          mlc[pos] = (key[r] & (uint32_t)(g.V - 1));
        }
      }
    }
    __syncthreads();
  }
}

// Per new brick: stable counting sort of its members (old-index order) by
// local cell into perm, and the new cell_start of its cells.
__global__ void __launch_bounds__(kIncT)
    k_inc_cells(const uint32_t* __restrict__ bbase, const uint32_t* __restrict__ memb,
                const uint32_t* __restrict__ mlc, Geo g, uint32_t* __restrict__ perm,
                uint32_t* __restrict__ cs_new) {
  constexpr int W = kIncT / 32;
  constexpr int ITEMS = 8;
  __shared__ uint32_t wh[W][kIncMaxV];
  __shared__ uint32_t cofs[kIncMaxV], crun[kIncMaxV];
  __shared__ uint32_t wt[8], tot;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t b = blockIdx.x;
  const uint32_t base = bbase[b], count = bbase[b + 1] - bbase[b];
  for (int lc = tid; lc < g.V; lc += kIncT) crun[lc] = 0;
  __syncthreads();
  for (uint32_t m = tid; m < count; m += kIncT) atomicAdd(&crun[mlc[base + m]], 1u);
  __syncthreads();
  {
    const int q = g.V / kIncT;  // V is 256 or 512
    uint32_t c[kIncMaxV / kIncT], sum = 0;
    for (int r = 0; r < q; ++r) {
      c[r] = crun[tid * q + r];
      sum += c[r];
    }
    uint32_t e = block_exclusive_scan(sum, wt, &tot);
    for (int r = 0; r < q; ++r) {
      cofs[tid * q + r] = e;
      cs_new[b * g.V + tid * q + r] = base + e;
      e += c[r];
    }
  }
  __syncthreads();
  for (int lc = tid; lc < g.V; lc += kIncT) crun[lc] = 0;
  __syncthreads();
  const uint32_t lt = (1u << lane) - 1u;
  for (uint32_t tb = 0; tb < count; tb += W * 32 * ITEMS) {
    for (int q = tid; q < W * kIncMaxV; q += kIncT) (&wh[0][0])[q] = 0;
    __syncthreads();
    const uint32_t seg = tb + (uint32_t)warp * 32 * ITEMS;
    uint32_t li[ITEMS], ll[ITEMS], pos[ITEMS];
#pragma unroll
    for (int r = 0; r < ITEMS; ++r) {
      const uint32_t m = seg + r * 32 + lane;
      const bool valid = m < count;
      const uint32_t lc = valid ? mlc[base + m] : (uint32_t)kIncMaxV;
      const uint32_t peers = __match_any_sync(0xffffffffu, lc);
      const uint32_t rank = __popc(peers & lt);
      const int leader = __ffs(peers) - 1;
      const uint32_t before = valid ? wh[warp][lc] : 0u;
      __syncwarp();
      if (valid && lane == leader) wh[warp][lc] = before + __popc(peers);
      __syncwarp();
      li[r] = valid ? memb[base + m] : 0u;
      ll[r] = lc;
      pos[r] = before + rank;
    }
    __syncthreads();
    for (int lc = tid; lc < g.V; lc += kIncT) {
      uint32_t acc = crun[lc];
      for (int w = 0; w < W; ++w) {
        const uint32_t t = wh[w][lc];
        wh[w][lc] = acc;
        acc += t;
      }
      crun[lc] = acc;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < ITEMS; ++r) {
      const uint32_t m = seg + r * 32 + lane;
      if (m < count) {
        const uint32_t dst = cofs[ll[r]] + wh[warp][ll[r]] + pos[r];
        if (dst < count) perm[base + dst] = li[r];
      }
    }
    __syncthreads();
  }
}

// cs_new[nkeys] = total; a total below n means some particle moved further
// than one cell since the previous sort (the arrays were changed outside).
__global__ void k_inc_finish(const uint32_t* __restrict__ bbase, int64_t nbricks, int64_t nkeys,
                             int64_t n, uint32_t* __restrict__ cs_new, int* status) {
  const uint32_t total = bbase[nbricks];
  cs_new[nkeys] = total;
  if ((int64_t)total != n) atomicOr(status, ST_DOMAIN);
}

// ---- compaction (Sec. 3.2): D = exclusive scan of the deletion flags over
// n + 1 entries (D[n] = N_del); the k-th hole below n_keep = n - N_del takes
// the k-th surviving particle at or beyond n_keep.
// The scan of the deletion flags reads the mask itself: phase 1 sums the
// flags of each kScanBlock block of the n + 1 entries (entry n is 0), phase 2
// is k_scan_top (which also leaves N_del), and phase 3 writes D and, for each
// deleted slot below n_keep, hole_pos[D[i]] = i.
__global__ void __launch_bounds__(256) k_del_reduce(const uint8_t* __restrict__ del, int64_t n,
                                                    uint32_t* __restrict__ sums) {
  __shared__ uint32_t wt[8];
  __shared__ uint32_t tot;
  const int64_t base = (int64_t)blockIdx.x * kScanBlock;
  uint32_t s = 0;
  for (int k = 0; k < kScanBlock / 256; ++k) {
    const int64_t i = base + k * 256 + threadIdx.x;
    if (i < n && del[i]) ++s;
  }
  block_exclusive_scan(s, wt, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(256) k_del_down(const uint8_t* __restrict__ del, int64_t n,
                                                  const uint32_t* __restrict__ sums,
                                                  const uint32_t* __restrict__ ndel,
                                                  uint32_t* __restrict__ D,
                                                  uint32_t* __restrict__ hole_pos) {
  __shared__ uint32_t wt[8];
  __shared__ uint32_t tot;
  const int64_t nkeep = n - (int64_t)*ndel;
  const int64_t base = (int64_t)blockIdx.x * kScanBlock;
  constexpr int per = kScanBlock / 256;
  uint32_t v[per];
  uint32_t s = 0;
  for (int k = 0; k < per; ++k) {
    const int64_t i = base + (int64_t)threadIdx.x * per + k;
    v[k] = i < n && del[i] ? 1u : 0u;
    s += v[k];
  }
  uint32_t e = block_exclusive_scan(s, wt, &tot) + sums[blockIdx.x];
  for (int k = 0; k < per; ++k) {
    const int64_t i = base + (int64_t)threadIdx.x * per + k;
    if (i <= n) D[i] = e;
    if (v[k] && i < nkeep) hole_pos[e] = (uint32_t)i;
    e += v[k];
  }
}

// Move the fillers of every plane of every array (rows planes of stride n,
// elements of 1, 4 or 8 bytes) in one launch: filler i -> its hole.
struct FillArr {
  void* base;
  int rows, esize;
};
struct FillSet {
  FillArr a[6];
  int k;
};
template <typename T>
__device__ __forceinline__ void fill_planes(void* base, int rows, int64_t n, int64_t h, int64_t i) {
  T* a = reinterpret_cast<T*>(base);
  for (int r = 0; r < rows; ++r) a[r * n + h] = a[r * n + i];
}
__global__ void k_fill_all(const FillSet fs, const uint8_t* __restrict__ del,
                           const uint32_t* __restrict__ D, const uint32_t* __restrict__ hole_pos,
                           int64_t n) {
  const int64_t nkeep = n - (int64_t)D[n];
  const int64_t base = (int64_t)D[nkeep];
  for (int64_t i = nkeep + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (del[i]) continue;
    const int64_t k = (i - nkeep) - ((int64_t)D[i] - base);  // filler rank
    const int64_t h = hole_pos[k];
#pragma unroll
    for (int q = 0; q < 6; ++q) {  // unrolled: the set stays in the parameter space
      if (q >= fs.k) break;
      const FillArr& f = fs.a[q];
      if (f.esize == 8)
        fill_planes<uint64_t>(f.base, f.rows, n, h, i);
      else if (f.esize == 4)
        fill_planes<uint32_t>(f.base, f.rows, n, h, i);
      else
        fill_planes<uint8_t>(f.base, f.rows, n, h, i);
    }
  }
}

template <typename T>
cudaError_t permute_plane(part_ctx* c, T* arr, const uint32_t* perm) {
  const int64_t n = c->n;
  k_gather<T><<<grid_for(c, n, 256), 256, 0, c->stream>>>(arr, (T*)c->tmp, perm, n);
  c->launches++;
  return cudaMemcpyAsync(arr, c->tmp, sizeof(T) * n, cudaMemcpyDeviceToDevice, c->stream);
}

cudaError_t permute_all(part_ctx* c, const uint32_t* perm);

}  // namespace

cudaError_t launch_sort(part_ctx* c) {
  const Geo& g = c->geo;
  const int64_t n = c->n;
  cudaStream_t s = c->stream;
  cudaError_t e = apply_perm(c);  // a permutation not yet used by a push
  if (e != cudaSuccess) return e;
  const void* xcur = state_of(c, c->cur_alt).x;
  if (n > 0) {
    if (c->mode == PART_BORIS && c->prec == PART_MIXED)
      k_keys_cell<<<grid_for(c, n, 256), 256, 0, s>>>((const int32_t*)xcur, n, g, c->keys[0],
                                                   c->vals[0], c->status);
    else
      k_keys_f64<<<grid_for(c, n, 256), 256, 0, s>>>((const double*)xcur, n, g, c->keys[0],
                                                  c->vals[0], c->status);
    c->launches++;
    int bits = 0;
    while (bits < 32 && ((int64_t)1 << bits) < g.nkeys) ++bits;
    const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
    const int64_t m = ntiles * kRadix;
    const int64_t nblk = (m + kScanBlock - 1) / kScanBlock;
    int cur = 0;
    for (int shift = 0; shift < bits; shift += kRadixBits) {
      k_radix_hist<<<(unsigned)ntiles, kSortThreads, 0, s>>>(c->keys[cur], n, shift, c->hist,
                                                             ntiles);
      k_scan_reduce<<<(unsigned)nblk, 256, 0, s>>>(c->hist, m, c->hsum);
      k_scan_top<<<1, 256, 0, s>>>(c->hsum, nblk);
      k_scan_down<<<(unsigned)nblk, 256, 0, s>>>(c->hist, m, c->hsum);
      k_radix_scatter<<<(unsigned)ntiles, kSortThreads, 0, s>>>(
          c->keys[cur], c->vals[cur], c->keys[cur ^ 1], c->vals[cur ^ 1], n, shift, c->hist,
          ntiles);
      c->launches += 5;
      cur ^= 1;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const uint32_t* perm = c->vals[cur];
    const uint32_t* sk = c->keys[cur];
    k_cell_start<<<grid_for(c, n + 1, 256), 256, 0, s>>>(sk, n, g.nkeys, c->cstart);
    c->launches++;
    return permute_all(c, perm);
  } else {
    k_cell_start<<<1, 256, 0, s>>>(c->keys[0], 0, g.nkeys, c->cstart);
    c->launches++;
  }
  return cudaGetLastError();
}

// Incremental path: keys + per-(brick, slot) counts, destinations, scan,
// placement, per-brick cell sort (see the kernels above).
cudaError_t launch_sort_incremental(part_ctx* c) {
  const Geo& g = c->geo;
  const int64_t n = c->n;
  cudaStream_t s = c->stream;
  if (n == 0) return launch_sort(c);
  cudaError_t e = apply_perm(c);
  if (e != cudaSuccess) return e;
  const void* xcur = state_of(c, c->cur_alt).x;
  const unsigned nbk = (unsigned)g.nbricks;
  if (c->mode == PART_BORIS && c->prec == PART_MIXED)
    k_inc_count<true><<<nbk, kIncT, 0, s>>>(xcur, n, c->cstart, g, c->keys[0], c->bslot,
                                            c->status);
  else
    k_inc_count<false><<<nbk, kIncT, 0, s>>>(xcur, n, c->cstart, g, c->keys[0], c->bslot,
                                             c->status);
  k_inc_dest<<<grid_for(c, g.nbricks * 32, 256), 256, 0, s>>>(c->bslot, g, c->bcount);
  e = cudaMemsetAsync(c->bcount + g.nbricks, 0, sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  const int64_t m = g.nbricks + 1;
  const int64_t nblk = (m + kScanBlock - 1) / kScanBlock;
  k_scan_reduce<<<(unsigned)nblk, 256, 0, s>>>(c->bcount, m, c->bsum);
  k_scan_top<<<1, 256, 0, s>>>(c->bsum, nblk);
  k_scan_down<<<(unsigned)nblk, 256, 0, s>>>(c->bcount, m, c->bsum);
  k_inc_place<<<nbk, kIncT, 0, s>>>(c->keys[0], c->cstart, g, c->bslot, c->bcount, c->vals[1],
                                    c->keys[1], n);
  k_inc_cells<<<nbk, kIncT, 0, s>>>(c->bcount, c->vals[1], c->keys[1], g, c->vals[0],
                                    c->cstart_alt);
  k_inc_finish<<<1, 1, 0, s>>>(c->bcount, g.nbricks, g.nkeys, n, c->cstart_alt, c->status);
  c->launches += 8;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  std::swap(c->cstart, c->cstart_alt);
  return permute_all(c, c->vals[0]);
}

namespace {

// Permute every bound array by perm (Boris modes: only recorded, see above).
cudaError_t permute_all(part_ctx* c, const uint32_t* perm) {
  const int64_t n = c->n;
  cudaStream_t s = c->stream;
  cudaError_t e;
  {
    // Boris modes with alternate buffers: the next brick push (or
    // apply_perm) moves the particles; nothing is copied here
    if (c->mode == PART_BORIS && c->alt_x) {
      c->perm_pend = perm;
      (void)s;
      return cudaGetLastError();
    }
    if (c->mode == PART_BORIS && c->prec == PART_FP64) {
      for (int a = 0; a < 3; ++a) {
        if ((e = permute_plane<double>(c, (double*)c->x + a * n, perm))) return e;
        if ((e = permute_plane<double>(c, (double*)c->u + a * n, perm))) return e;
      }
      if (c->w && (e = permute_plane<double>(c, (double*)c->w, perm))) return e;
    } else if (c->mode == PART_BORIS) {
      if ((e = permute_plane<int32_t>(c, (int32_t*)c->x, perm))) return e;
      for (int a = 0; a < 3; ++a)
        if ((e = permute_plane<float>(c, (float*)c->off + a * n, perm))) return e;
      for (int a = 0; a < 6; ++a)
        if ((e = permute_plane<float>(c, (float*)c->u + a * n, perm))) return e;
      if (c->w && (e = permute_plane<float>(c, (float*)c->w, perm))) return e;
    } else {
      for (int a = 0; a < 3; ++a)
        if ((e = permute_plane<double>(c, (double*)c->x + a * n, perm))) return e;
      for (int b = 0; b < c->nbins; ++b) {
        if ((e = permute_plane<double>(c, c->chi + (int64_t)b * n, perm))) return e;
        if ((e = permute_plane<double>(c, c->eng + (int64_t)b * n, perm))) return e;
      }
      if (c->n_old && (e = permute_plane<double>(c, c->n_old, perm))) return e;
      if (c->shk && (e = permute_plane<uint8_t>(c, c->shk, perm))) return e;
    }
    if (c->id && (e = permute_plane<uint64_t>(c, c->id, perm))) return e;
  }
  return cudaGetLastError();
}

}  // namespace

// Gather the current buffer through the pending permutation into the other
// buffer, which becomes current.
cudaError_t apply_perm(part_ctx* c) {
  if (!c->perm_pend) return cudaSuccess;
  const uint32_t* perm = c->perm_pend;
  c->perm_pend = nullptr;
  const int64_t n = c->n;
  if (n == 0) return cudaSuccess;
  const PState a = state_of(c, c->cur_alt), b = state_of(c, !c->cur_alt);
  if (c->prec == PART_FP64)
    k_gather_state<double, 3, double, 3><<<grid_for(c, n, 256), 256, 0, c->stream>>>(
        (const double*)a.x, nullptr, (const double*)a.u, (const double*)a.w, a.id,
        (double*)b.x, nullptr, (double*)b.u, (double*)b.w, b.id, perm, n);
  else
    k_gather_state<int32_t, 1, float, 6><<<grid_for(c, n, 256), 256, 0, c->stream>>>(
        (const int32_t*)a.x, (const float*)a.off, (const float*)a.u, (const float*)a.w, a.id,
        (int32_t*)b.x, (float*)b.off, (float*)b.u, (float*)b.w, b.id, perm, n);
  c->launches++;
  c->cur_alt = !c->cur_alt;
  return cudaGetLastError();
}

// Bring the current state into the caller's arrays, in sorted order.
cudaError_t flush_pending(part_ctx* c) {
  cudaError_t r = launch_spec_to_plain(c);
  if (r != cudaSuccess) return r;
  r = apply_perm(c);
  if (r != cudaSuccess || !c->cur_alt) return r;
  c->cur_alt = false;
  const int64_t n = c->n;
  if (n == 0) return cudaSuccess;
  const size_t e = c->prec == PART_FP64 ? 8 : 4;
  const int nx = c->prec == PART_FP64 ? 3 : 1;
  r = cudaMemcpyAsync(c->x, c->alt_x, e * nx * n, cudaMemcpyDeviceToDevice, c->stream);
  if (r == cudaSuccess && c->off)
    r = cudaMemcpyAsync(c->off, c->alt_off, 12 * n, cudaMemcpyDeviceToDevice, c->stream);
  if (r == cudaSuccess)
    r = cudaMemcpyAsync(c->u, c->alt_u, u_rows(c) * e * n, cudaMemcpyDeviceToDevice,
                        c->stream);
  if (r == cudaSuccess && c->w)
    r = cudaMemcpyAsync(c->w, c->alt_w, e * n, cudaMemcpyDeviceToDevice, c->stream);
  if (r == cudaSuccess && c->id)
    r = cudaMemcpyAsync(c->id, c->alt_id, 8 * n, cudaMemcpyDeviceToDevice, c->stream);
  return r;
}

namespace {

// ---- one row moved within its own buffer: dst[i] = src[i], i < len, where
// the two ranges may overlap (the new row stride after a compaction or an
// injection).  Blocks of kMoveB elements are taken in copy order (ascending
// when dst < src, descending when dst > src) through a ticket counter; a
// block reads its source into registers, publishes that it has read, and
// writes only after the at most two blocks whose sources its destination
// covers have published the same.  Those blocks hold earlier tickets and read
// before they wait on anything, so every wait ends; each is bounded all the
// same (ST_TIMEOUT, and the block's writes are skipped).  flags[0] is the
// ticket counter, flags[1 + b] block b's published read; both start at 0.
constexpr int kMoveT = 256, kMoveE = 8, kMoveB = kMoveT * kMoveE;

template <typename T>
__device__ __forceinline__ void move_row_body(const T* src, T* dst, int64_t len, uint32_t* flags,
                                              int* status) {
  __shared__ int64_t s_b;
  __shared__ int s_ok;
  const int64_t nblk = (len + kMoveB - 1) / kMoveB;
  const bool up = dst > src;
  const int64_t d = dst - src;  // destination offset in source elements
  for (;;) {
    if (threadIdx.x == 0) {
      const int64_t t = (int64_t)atomicAdd(&flags[0], 1u);
      s_b = t < nblk ? (up ? nblk - 1 - t : t) : -1;
    }
    __syncthreads();
    const int64_t b = s_b;
    if (b < 0) break;
    const int64_t i0 = b * kMoveB;
    T v[kMoveE];
#pragma unroll
    for (int k = 0; k < kMoveE; ++k) {
      const int64_t i = i0 + k * kMoveT + threadIdx.x;
      if (i < len) v[k] = src[i];
    }
    __syncthreads();  // the whole block has read
    if (threadIdx.x == 0) {
      __threadfence();
      atomicExch(&flags[1 + b], 1u);
      // source blocks that the destination [i0 + d, i1 + d) covers
      const int64_t i1 = i0 + kMoveB < len ? i0 + kMoveB : len;
      int64_t lo = (i0 + d) / kMoveB, hi = (i1 - 1 + d) / kMoveB;
      if (i0 + d < 0) lo = -1;  // floor for negative offsets (no such block)
      lo = lo < 0 ? 0 : lo;
      hi = hi < nblk - 1 ? hi : nblk - 1;
      bool ok = true;
      for (int64_t q = lo; q <= hi && ok; ++q) {
        if (q == b) continue;
        const uint64_t t0 = global_ns();
        uint32_t it = 0;
        while (atomicAdd(&flags[1 + q], 0u) == 0u) {
          if (++it > (1u << 24) || global_ns() - t0 > kWaitLimitNs) {
            ok = false;
            break;
          }
        }
      }
      __threadfence();
      if (!ok) atomicOr(status, ST_TIMEOUT);
      s_ok = ok ? 1 : 0;
    }
    __syncthreads();
    if (s_ok) {
#pragma unroll
      for (int k = 0; k < kMoveE; ++k) {
        const int64_t i = i0 + k * kMoveT + threadIdx.x;
        if (i < len) dst[i] = v[k];
      }
    }
    __syncthreads();  // s_b and s_ok are reused
  }
}

template <typename T>
__global__ void __launch_bounds__(kMoveT)
    k_move_row(const T* src, T* dst, int64_t len, uint32_t* flags, int* status) {
  move_row_body<T>(src, dst, len, flags, status);
}

// Row r of a compaction, for up to three arrays of element type T in one
// launch: from stride n to stride nnew = n - D[n], with D[n] (the deletion
// count) read on the device, so the host need not wait for it.  The arrays'
// rows move one after the other, each with its own ticket counter and flags
// (at flags + a * fstride); arrays with rows <= r are skipped.
template <typename T>
struct MoveRows {
  T* base[3];
  int rows[3];
  int k;
};
template <typename T>
__global__ void __launch_bounds__(kMoveT)
    k_move_rows_compact(const MoveRows<T> m, int64_t n, int64_t r,
                        const uint32_t* __restrict__ dn, uint32_t* flags, int64_t fstride,
                        int* status) {
  const int64_t nnew = n - (int64_t)*dn;
  if (nnew == n) return;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a >= m.k) break;
    if (r < m.rows[a])
      move_row_body<T>(m.base[a] + r * n, m.base[a] + r * nnew, nnew, flags + a * fstride,
                       status);
    __syncthreads();  // the body's shared ticket slot is reused by the next array
  }
}

// Move len elements from src to dst in the stream, overlap allowed.
template <typename T>
cudaError_t move_row(part_ctx* c, const T* src, T* dst, int64_t len) {
  if (len <= 0 || src == dst) return cudaSuccess;
  if (src + len <= dst || dst + len <= src)
    return cudaMemcpyAsync(dst, src, sizeof(T) * len, cudaMemcpyDeviceToDevice, c->stream);
  const int64_t nblk = (len + kMoveB - 1) / kMoveB;
  uint32_t* flags = (uint32_t*)c->tmp;  // (1 + nblk) words; tmp holds 8 * capacity bytes
  cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(uint32_t) * (1 + nblk), c->stream);
  if (e != cudaSuccess) return e;
  const int64_t grid = std::min<int64_t>(nblk, (int64_t)c->sms * 8);
  k_move_row<T><<<(unsigned)grid, kMoveT, 0, c->stream>>>(src, dst, len, flags, c->status);
  c->launches++;
  return cudaGetLastError();
}

// Move rows r >= 1 of up to three arrays of one element type (their holes
// already filled) from stride n to stride nnew (the deletion count stays on
// the device: D[n]); row r of every array in one launch.
template <typename T>
cudaError_t shrink_rows(part_ctx* c, const MoveRows<T>& m, int64_t n) {
  // Rows r >= 1 move from stride n to stride nnew: row r shifts down by
  // r (n - nnew) elements, in place, lowest row first (a row only overwrites
  // source rows already moved, and its own source as the move allows).
  const int64_t nblk = (n + kMoveB - 1) / kMoveB;
  const int64_t grid = std::min<int64_t>(m.k * nblk, (int64_t)c->sms * 8);
  const int64_t fstride = 1 + nblk;
  // k (1 + nblk) words; tmp holds 8 * capacity bytes
  uint32_t* flags = (uint32_t*)c->tmp;
  int rows = 0;
  for (int a = 0; a < m.k; ++a) rows = m.rows[a] > rows ? m.rows[a] : rows;
  for (int r = 1; r < rows; ++r) {
    cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(uint32_t) * m.k * fstride, c->stream);
    if (e != cudaSuccess) return e;
    k_move_rows_compact<T><<<(unsigned)grid, kMoveT, 0, c->stream>>>(
        m, n, r, c->keys[0] + n, flags, fstride, c->status);
    c->launches++;
  }
  return cudaGetLastError();
}

// Injection: rows r >= 1 move up from stride n to stride n + k (row r by
// r k elements), in place, the highest row first so that a row only
// overwrites source rows already moved (and its own source as k_move_row
// allows).  Then the k new elements of each row go to its slots n..n+k-1.
template <typename T>
cudaError_t grow_rows(part_ctx* c, T* base, int rows, int64_t n, int64_t k, const T* src) {
  cudaError_t e = cudaSuccess;
  const int64_t m = n + k;
  for (int r = rows - 1; r >= 1 && n > 0 && k > 0 && e == cudaSuccess; --r)
    e = move_row<T>(c, base + (int64_t)r * n, base + (int64_t)r * m, n);
  for (int r = 0; r < rows && k > 0 && e == cudaSuccess; ++r)
    e = cudaMemcpyAsync(base + (int64_t)r * m + n, src + (int64_t)r * k, sizeof(T) * k,
                        cudaMemcpyDeviceToDevice, c->stream);
  return e;
}

}  // namespace

cudaError_t launch_inject(part_ctx* c, int64_t k, const InjectSrc& s) {
  const int64_t n = c->n;
  cudaError_t e = cudaSuccess;
  if (k == 0) return e;
  if (c->mode == PART_BORIS && c->prec == PART_FP64) {
    e = grow_rows<double>(c, (double*)c->x, 3, n, k, (const double*)s.x);
    if (e == cudaSuccess) e = grow_rows<double>(c, (double*)c->u, 3, n, k, (const double*)s.u);
    if (e == cudaSuccess && c->w)
      e = grow_rows<double>(c, (double*)c->w, 1, n, k, (const double*)s.w);
  } else if (c->mode == PART_BORIS) {
    e = grow_rows<int32_t>(c, (int32_t*)c->x, 1, n, k, (const int32_t*)s.x);
    if (e == cudaSuccess) e = grow_rows<float>(c, (float*)c->off, 3, n, k, (const float*)s.off);
    if (e == cudaSuccess) e = grow_rows<float>(c, (float*)c->u, 6, n, k, (const float*)s.u);
    if (e == cudaSuccess && c->w)
      e = grow_rows<float>(c, (float*)c->w, 1, n, k, (const float*)s.w);
  } else {
    e = grow_rows<double>(c, (double*)c->x, 3, n, k, (const double*)s.x);
    if (e == cudaSuccess) e = grow_rows<double>(c, c->chi, c->nbins, n, k, s.chi);
    if (e == cudaSuccess) e = grow_rows<double>(c, c->eng, c->nbins, n, k, s.eng);
    if (e == cudaSuccess) e = grow_rows<double>(c, c->n_old, 1, n, k, s.n_old);
    if (e == cudaSuccess && c->shk) e = cudaMemsetAsync(c->shk + n, 0, (size_t)k, c->stream);
  }
  if (e == cudaSuccess && c->id) e = grow_rows<uint64_t>(c, c->id, 1, n, k, s.id);
  return e;
}

// In-place exclusive scan of m 32-bit counts (m <= capacity + 1); sums needs
// (m + kScanBlock - 1) / kScanBlock + 1 entries.  a[m - 1] ends as the total
// of the first m - 1 counts when the last count is 0.
cudaError_t launch_exclusive_scan(part_ctx* c, uint32_t* a, int64_t m, uint32_t* sums) {
  const int64_t nblk = (m + kScanBlock - 1) / kScanBlock;
  k_scan_reduce<<<(unsigned)nblk, 256, 0, c->stream>>>(a, m, sums);
  k_scan_top<<<1, 256, 0, c->stream>>>(sums, nblk);
  k_scan_down<<<(unsigned)nblk, 256, 0, c->stream>>>(a, m, sums);
  c->launches += 3;
  return cudaGetLastError();
}

cudaError_t launch_compact(part_ctx* c, const uint8_t* del, int64_t* nnew_out) {
  const int64_t n = c->n;
  cudaStream_t s = c->stream;
  if (n == 0) {
    *nnew_out = 0;
    return cudaSuccess;
  }
  const int gb = grid_for(c, n + 1, 256);
  const int64_t m = n + 1;
  const int64_t nblk = (m + kScanBlock - 1) / kScanBlock;
  uint32_t* D = c->keys[0];
  uint32_t* sums = c->vals[1];
  k_del_reduce<<<(unsigned)nblk, 256, 0, s>>>(del, n, sums);
  k_scan_top<<<1, 256, 0, s>>>(sums, nblk, sums + nblk);
  k_del_down<<<(unsigned)nblk, 256, 0, s>>>(del, n, sums, sums + nblk, D, c->keys[1]);
  c->launches += 3;
  // every array is filled (one launch) and its rows moved on the device (the
  // kernels read the deletion count D[n] there); the host reads the count
  // once, at the end
  FillSet fs{};
  auto add = [&](void* p, int rows, int esize) {
    if (p) fs.a[fs.k++] = FillArr{p, rows, esize};
  };
  if (c->mode == PART_BORIS && c->prec == PART_FP64) {
    add(c->x, 3, 8);
    add(c->u, 3, 8);
    add(c->w, 1, 8);
  } else if (c->mode == PART_BORIS) {
    add(c->x, 1, 4);
    add(c->off, 3, 4);
    add(c->u, 6, 4);
    add(c->w, 1, 4);
  } else {
    add(c->x, 3, 8);
    add(c->chi, c->nbins, 8);
    add(c->eng, c->nbins, 8);
    add(c->n_old, 1, 8);
    add(c->shk, 1, 1);
  }
  add(c->id, 1, 8);
  k_fill_all<<<gb, 256, 0, s>>>(fs, del, D, c->keys[1], n);
  c->launches++;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (c->mode == PART_BORIS && c->prec == PART_FP64) {
    const MoveRows<double> m{{(double*)c->x, (double*)c->u, nullptr}, {3, 3, 0}, 2};
    if ((e = shrink_rows<double>(c, m, n))) return e;
  } else if (c->mode == PART_BORIS) {
    const MoveRows<float> m{{(float*)c->off, (float*)c->u, nullptr}, {3, 6, 0}, 2};
    if ((e = shrink_rows<float>(c, m, n))) return e;
  } else {
    const MoveRows<double> m{{(double*)c->x, c->chi, c->eng}, {3, c->nbins, c->nbins}, 3};
    if ((e = shrink_rows<double>(c, m, n))) return e;
  }
  uint32_t ndel = 0;
  e = cudaMemcpyAsync(&ndel, D + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  *nnew_out = n - (int64_t)ndel;
  return cudaGetLastError();
}
