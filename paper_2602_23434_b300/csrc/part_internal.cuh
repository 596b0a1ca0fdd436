// part_internal.cuh -- shared definitions of the CUDA particle library.
//
// Geometry, status bits, the context record and the small PTX wrappers
// (mbarrier, TMA tensor copies) used by the kernels.  sm_103a only.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "part.h"

// ---------------------------------------------------------------- status bits
// Latched by kernels with atomicOr into the workspace status word.
enum : int {
  ST_TIMEOUT = 1,     // a bounded mbarrier wait ran out
  ST_NONFINITE = 2,   // NaN / Inf in particle state or samples
  ST_DOMAIN = 4,      // particle outside the cell range it was sorted into
};

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;   // keys per radix tile
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kScanBlock = 1024;                      // elements per scan block
constexpr int kPushThreads = 256;                     // brick kernel CTA size

// Geometry handed to kernels by value.
struct Geo {
  int dim;
  int n[3];
  int b[3];        // brick (cell tile) dims
  int nb[3];       // bricks per axis (last may be partial)
  int h[3];        // stencil halo per axis: 1, or 0 for z in 2D
  int e[3];        // extended (haloed) tile dims b + 2h
  int pn[3];       // padded field dims: x pitch, y, z (ghost layer of h)
  int box[3];      // TMA box dims (x rounded to a 16-byte multiple)
  int V;           // cells per brick
  int ev;          // cells per extended tile
  int64_t G;       // cells
  int64_t nkeys;   // key-space size = bricks * V
  int64_t nbricks;
  int64_t pplane;  // padded elements per field component
  double xmin[3], dx[3], inv_dx[3], L[3], xmax[3];
  float invn[3];   // 1/n per axis, for the float-reciprocal cell decode
  float xminf[3], inv_dxf[3], xmin_cells[3];  // f32 images of xmin, inv_dx; |xmin| inv_dx
  int bshift[3];   // log2 b per axis (brick sides are powers of two)
  int vshift;      // log2 V
  int open[3];     // 1: open (outflow) axis, 0: periodic
  int any_open;
};

// Every member has a default initializer: a context built on the stack (the
// no-allocation sort) starts with null buffers and no pending state.
struct part_ctx {
  part_grid grid{};
  part_prec prec{};
  part_shape shape{};
  part_mode mode{};
  int64_t capacity{};
  int nbins{};
  cudaStream_t stream{};
  int device{};       // CUDA device current at part_init
  int sms{};          // its multiprocessor count (launch shapes)
  Geo geo{};
  int ncomp{};        // field components (6 Boris, 7 LP)
  int fcomp{};        // components per cell as stored: SoA ncomp, or 8 (cell-interleaved f32)
  int esize{};        // field element bytes
  // workspace carve-up
  char* ws{};
  size_t ws_bytes{};
  void* fpad{};       // padded fields [ncomp][pz][py][px]
  uint32_t* keys[2] = {};
  uint32_t* vals[2] = {};
  uint32_t* hist{};   // radix tile histograms (digit-major)
  uint32_t* hsum{};   // scan block sums
  uint32_t* cstart{}; // cell_start [nkeys + 1]
  uint32_t* cstart_alt{};  // the other cell_start buffer (incremental sort)
  uint32_t* bcount{};      // [nbricks + 1] particles per brick, then their offsets
  uint32_t* bsum{};        // scan block sums of bcount
  uint32_t* bslot{};       // [nbricks][27] particles per (old brick, neighbour slot)
  void* tmp{};        // permute scratch, 8 bytes * capacity
  double* dpart{};    // deposit partials [nbricks][3][ev]
  double* samples{};  // LP samples [3][capacity]: n_new, b2m, 1/gamma_g
  double* lpcache{};  // LP v, B at the current positions [6][capacity] (paired: [12] f32)
  bool lp_cache_ok{}; // lpcache matches the bound LPs, their order and the fields
  float* fpair{};     // LP: paired-f32 copy of the padded fields, 16 floats per cell
  double* fxq{};      // x quadratics of the padded FP64 fields (LP; FP64 Boris), 4 doubles per (component, cell)
  int lp_paired{};    // LP push arithmetic: 0 FP64, 1 paired f32
  double* smap{};     // LP deferred spectra: per-LP map (alpha, beta, S) [3][capacity]
  int spec_lazy{};    // spec_update composes maps instead of updating every bin
  bool maps_pending{};  // some LP's map is not the identity (bins not materialised)
  // Boris modes: alternate particle buffers.  part_sort only computes the
  // permutation (perm_pend); the next brick push reads the current buffer
  // through it and writes the other one, so no separate permutation pass is
  // needed.  The current state then alternates between the caller's arrays
  // and these buffers; part_flush / part_sync bring it home.
  void* alt_x{};      // FP64: double[3][cap]   mixed: int32 cell[cap]
  void* alt_off{};    // mixed: float[3][cap]
  void* alt_u{};      // FP64: double[3][cap]   mixed: float[6][cap] (hi, lo)
  void* alt_w{};      // FP64: double[cap]      mixed: float[cap]
  uint64_t* alt_id{}; // uint64[cap]
  uint8_t* outmask{};             // caller's outflow flags (open axes), or NULL
  bool cur_alt{};                 // the current state is in the alternate buffers
  const uint32_t* perm_pend{};    // new slot -> index in the current buffer, or NULL
  int* status{};      // device status word
  CUtensorMap tmap{};  // TMA map of fpad
  CUtensorMap tmap_plane{};  // the same with a one-plane box (3D cell-interleaved f32)
  bool tmap_ok{};
  // bound particles
  int64_t n{};
  void* x{};
  void* off{};
  void* u{};
  void* w{};
  uint64_t* id{};
  double* chi{};
  double* eng{};
  double* n_old{};
  // LP shocks (Eq. convolution_spectra)
  double* shock_r{};       // [G] compression ratio of each shock cell, 0 elsewhere
  uint32_t* shock_list{};  // [0]: count; [1 + k]: LPs shocked by the last push
  double* shock_rs{};      // [k]: compression ratio each listed LP saw
  double* shock_q{};       // [G] Eq. slope index q of each shock cell, 0 elsewhere
  double* shock_qs{};      // [k]: the index q each listed LP saw
  uint8_t* shk{};          // caller's per-LP "in a shock cell" flags; NULL: shocks off
  double r_min{};
  int shock_rel{};         // 1: q with the relativistic correction q_R
  int lp_order{2};         // LP time marching: 2 (Heun) or 3 (SSP-RK3)
  bool shock_listed{};     // the last push filled the list
  // incremental sort: the arrays are in the order of the last sort, and
  // `moved` bounds every particle's displacement since (|v| < c = 1)
  bool order_kept{};
  double moved{};
  // LP spectra: the bound chi/eng arrays hold psi = chi eps^2 and y = 1/eps
  // (the variables the spectral step is linear in) until the next flush
  bool spec_inv{};
  bool bound{}, fields_set{}, sorted{}, deposit_on{}, deposit_ready{}, samples_ready{};
  int64_t launches{};
  std::string err;
};

// Serving: the device header of a work list and one resident snapshot.
struct ServeHeader {
  int nitems;
  unsigned next;  // next unclaimed item (the staged copy carries 0 into every round)
  int pad[62];
};
struct SnapEntry {
  const float* fp;  // padded f32 field copy of the snapshot's context
  Geo g;
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Nanoseconds of the GPU's global timer.
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait: polls until the phase completes, limit_ns have passed on the
// global timer, or (should the timer stall) 2^26 polls were made; returns
// false when it gave up.
constexpr uint64_t kWaitLimitNs = 1000000000ull;  // 1 s: far above any TMA copy
__device__ __forceinline__ bool mbar_wait_for(uint64_t* bar, uint32_t parity,
                                              uint64_t limit_ns) {
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0; it < (1u << 26); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
  return false;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  return mbar_wait_for(bar, parity, kWaitLimitNs);
}

// 4-D tiled TMA load global -> shared, completion signalled on bar.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
      "r"(smem_addr(bar))
      : "memory");
}

// Finite test on the exponent bits (integer pipe): true unless v is Inf/NaN.
__device__ __forceinline__ bool finite_bits(double v) {
  return ((unsigned)__double2hiint(v) & 0x7ff00000u) != 0x7ff00000u;
}

// min(floor(s), hi) for s >= 0, and 0 for s < 0, from the bits of s on the
// integer pipe (exactly the value floor() gives; floor and compares would be
// FP64-pipe instructions).  s >= 2^31, +Inf and NaN give hi: callers test
// finiteness separately.
__device__ __forceinline__ int floor_clamp_bits(double s, int hi) {
  const long long b = __double_as_longlong(s);
  if (b < 0) return 0;                            // negative, or -0.0
  const int e = (int)(b >> 52) - 1023;            // unbiased exponent
  if (e < 0) return 0;                            // 0 <= s < 1
  if (e >= 31) return hi;
  const long long m = (b & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL;
  const int j = (int)(m >> (52 - e));
  return j > hi ? hi : j;
}

// q = c / n, r = c % n for 0 <= c < 2^24 by a float reciprocal and one exact
// integer correction (the float quotient is within 1 of the true one).
__device__ __forceinline__ int divmod_f(int c, int n, float invn, int* r) {
  int q = (int)(__int2float_rn(c) * invn);
  int rr = c - q * n;
  if (rr < 0) {
    --q;
    rr += n;
  } else if (rr >= n) {
    ++q;
    rr -= n;
  }
  *r = rr;
  return q;
}

// Cell coordinates of a linear cell index c = (jz n1 + jy) n0 + jx.
__device__ __forceinline__ void cell_coords(const Geo& g, int32_t c, int* j) {
  if (g.G <= (1 << 24) && c >= 0) {
    const int r = divmod_f(c, g.n[0], g.invn[0], &j[0]);
    j[2] = divmod_f(r, g.n[1], g.invn[1], &j[1]);
  } else {
    j[0] = c % g.n[0];
    const int r = c / g.n[0];
    j[1] = r % g.n[1];
    j[2] = r / g.n[1];
  }
}

// 1 if x lies outside the domain along an open axis (NaN counts as outside).
__device__ __forceinline__ uint8_t outside_open(const Geo& g, const double* x) {
  bool out = false;
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (g.open[a]) out = out || !(x[a] >= g.xmin[a] && x[a] < g.xmax[a]);
  return out ? 1 : 0;
}

// ---------------------------------------------------------------- shape weights
// Three-point weights at offsets k = -1, 0, +1 from the particle's cell for
// offset d = (s - j) - 1/2 in [-1/2, 1/2].  TSC: quadratic B-spline; CIC: hat
// (one of the outer weights is zero).
template <int SHAPE, typename T>
__device__ __forceinline__ void shape_weights(T d, T* w) {
  if (SHAPE == PART_TSC && sizeof(T) == 8) {
    // FP64: the three quadratics in Horner form, 1/8 -+ d/2 + d^2/2 and
    // 3/4 - d^2: five FMAs where the factored form takes seven FP64
    // instructions (measured faster on B300's FP64 pipe; not in f32)
    w[0] = fma(d, fma(T(0.5), d, T(-0.5)), T(0.125));
    w[1] = fma(-d, d, T(0.75));
    w[2] = fma(d, fma(T(0.5), d, T(0.5)), T(0.125));
  } else if (SHAPE == PART_TSC) {
    T a = T(0.5) - d, b = T(0.5) + d;
    w[0] = T(0.5) * (a * a);
    w[1] = T(0.75) - d * d;
    w[2] = T(0.5) * (b * b);
  } else {
    w[0] = d < T(0) ? -d : T(0);
    w[1] = T(1) - (d < T(0) ? -d : d);
    w[2] = d > T(0) ? d : T(0);
  }
}

// ---------------------------------------------------------------- host glue
// Host helpers of api.cu: record an error message, validate a grid, derive
// the kernel geometry for a field element size.
part_status fail(part_ctx* c, part_status s, const std::string& msg);
bool device_accessible(int device, const void* p);  // see api.cu
part_status check_grid(const part_grid* g);
void make_geo(const part_grid* gr, int esize, Geo* g);

// Kernel launchers implemented in the .cu files; each returns a cudaError_t
// of its launch and counts the launches it made in *launches.
cudaError_t launch_pad_fields(part_ctx* c, const void* src);
cudaError_t launch_sort(part_ctx* c);
cudaError_t flush_pending(part_ctx* c);  // current state into the bound arrays, in order
cudaError_t apply_perm(part_ctx* c);     // a pending permutation into the other buffer

// Rows of the momentum array: FP64 u[3][n]; mixed u[6][n], the f32 momentum
// in rows 0-2 and its f32 residual in rows 3-5 (u = hi + lo, a compensated
// pair, so the stored momentum is not rounded to f32 every step).
inline int u_rows(const part_ctx* c) { return c->prec == PART_MIXED ? 6 : 3; }

// Particle arrays of one buffer (the caller's or the alternate one).
struct PState {
  void* x;
  void* off;
  void* u;
  void* w;
  uint64_t* id;
};
inline PState state_of(const part_ctx* c, bool alt) {
  if (!alt) return {c->x, c->off, c->u, c->w, c->id};
  return {c->alt_x, c->off ? c->alt_off : nullptr, c->alt_u, c->w ? c->alt_w : nullptr,
          c->id ? c->alt_id : nullptr};
}
cudaError_t launch_compact(part_ctx* c, const uint8_t* del, int64_t* nnew);
cudaError_t launch_exclusive_scan(part_ctx* c, uint32_t* a, int64_t m, uint32_t* sums);
part_status check_ctx(part_ctx* c);                                    // api.cu
part_status cuda_fail(part_ctx* c, cudaError_t e, const char* where);  // api.cu
part_status check_access(part_ctx* c, const void* p, const char* what);  // api.cu
struct InjectSrc {
  const void *x, *off, *u, *w;
  const uint64_t* id;
  const double *chi, *eng, *n_old;
};
cudaError_t launch_inject(part_ctx* c, int64_t k, const InjectSrc& src);  // sort.cu
cudaError_t launch_sort_incremental(part_ctx* c);  // see sort.cu
// One launch of an LP kernel over LPs [p0, p1) (of the n bound) on a stream;
// cached: v and B at x come from the cache of the previous push.
struct LpLaunch {
  int64_t p0, p1;
  int grid;
  cudaStream_t stream;
  bool cached;
};
cudaError_t launch_lp_push_range(part_ctx* c, double dt, const LpLaunch& L);       // FP64
cudaError_t launch_lp_push_pair_range(part_ctx* c, double dt, const LpLaunch& L);  // paired f32
cudaError_t launch_spec_range(part_ctx* c, double dt, double c0, double u_rad, bool from_plain,
                              const LpLaunch& L);
cudaError_t launch_pad_pair_lp(part_ctx* c);               // fpair from fpad
cudaError_t launch_pad_xq(part_ctx* c);                    // fxq from fpad (FP64)
cudaError_t launch_shock_cells(part_ctx* c);       // shock_r, shock_q from the padded LP fields
cudaError_t launch_shock_convolve(part_ctx* c);    // Eq. convolution_spectra on the list
cudaError_t launch_boris(part_ctx* c, double qm, double dt, int nsteps);
cudaError_t launch_boris_mixed(part_ctx* c, double qm, double dt, int nsteps);
cudaError_t launch_serve_kernel(int shape, int dim, ServeHeader* hdr,
                                const part_work_item* items, const SnapEntry* snaps, int nsnap,
                                int* status, int grid, int threads, cudaStream_t stream);
cudaError_t launch_deposit_combine(part_ctx* c, double* out);
cudaError_t launch_lp_push(part_ctx* c, double dt, int nsteps);
cudaError_t launch_spec_update(part_ctx* c, double dt, double c0, double u_rad);
// (y, psi) back to (chi, eps) in the bound arrays, if the updates left them so
cudaError_t launch_spec_to_plain(part_ctx* c);

// Launch shapes.  The SM count is read from the device at part_init
// (cudaDevAttrMultiProcessorCount: 148 on a full B300, fewer on a smaller
// SKU or a MIG slice); grid-stride kernels are capped at 64 CTAs per SM.
inline int grid_for(const part_ctx* c, int64_t n, int threads) {
  const int64_t cap = (int64_t)(c->sms > 0 ? c->sms : 1) * 64;
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}
// CTA size (256, 128 or 64 threads, one particle each) that spreads a set too
// small to fill the GPU most evenly over the SMs: the one whose fullest SM
// holds the fewest particles (65,536 particles on 148 SMs: 64 threads, 448 per
// SM instead of 512).  Sets of a full wave or more keep 256.
inline int threads_for_spread(const part_ctx* c, int64_t n) {
  const int64_t sms = c->sms > 0 ? c->sms : 1;
  if (n >= sms * 2048) return 256;
  int best = 256;
  int64_t best_load = INT64_MAX;
  for (int t : {256, 128, 64}) {
    const int64_t blocks = (n + t - 1) / t;
    const int64_t load = (blocks + sms - 1) / sms * t;
    if (load < best_load) {
      best_load = load;
      best = t;
    }
  }
  return best;
}
cudaError_t launch_selftest_wait(part_ctx* c, int64_t limit_ns, int arrive);  // init.cu
cudaError_t launch_init(part_ctx* c, uint64_t seed, double u_th, double emin, double emax,
                        double p, double N0);
