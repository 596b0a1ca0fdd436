// noalloc.cu -- part_sort_fp64_noalloc: the cell sort without any device
// allocation and without a caller workspace.
//
// Some callers cannot allocate device memory at the moment they need a sort:
// a plug-in whose host application owns every device byte through its own
// pool, or a latency-critical loop where an allocation (which may synchronise
// the device) is not acceptable.  This entry point takes its scratch from one fixed
// array compiled into the library instead.
//
// The scratch is a file-scope static __device__ array of
// PART_NOALLOC_SORT_SCRATCH_BYTES.  Every GPU that loads the library holds it
// until the process exits.  Host code never dereferences the array's name
// (on the host that name is only a stand-in, not a device address): the
// first call on each device, with that device current, looks the device
// address up with cudaGetSymbolAddress and caches it.  That first call should
// therefore come before any stream capture.  All calls share the one array
// and it keeps whatever the last call left there, so calls that overlap on
// the GPU (different streams, or different host threads on one device) race
// and must be serialised by the caller.  No cudaMalloc, cudaFree or
// allocating library routine is called.
#include <mutex>

#include "part_internal.cuh"

namespace {

constexpr int64_t kMaxN = PART_NOALLOC_SORT_MAX_N;
constexpr int64_t kTiles = (kMaxN + kSortTile - 1) / kSortTile;
constexpr int64_t kHistLen = kTiles * kRadix;
constexpr int64_t kBlocks = (kHistLen + kScanBlock - 1) / kScanBlock;

constexpr size_t up256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kOffKeys0 = 0;
constexpr size_t kOffKeys1 = kOffKeys0 + up256(kMaxN * 4);
constexpr size_t kOffVals0 = kOffKeys1 + up256(kMaxN * 4);
constexpr size_t kOffVals1 = kOffVals0 + up256(kMaxN * 4);
constexpr size_t kOffHist = kOffVals1 + up256(kMaxN * 4);
constexpr size_t kOffHsum = kOffHist + up256(kHistLen * 4);
constexpr size_t kOffTmp = kOffHsum + up256((kBlocks + 1) * 4);
constexpr size_t kOffStatus = kOffTmp + up256(kMaxN * 8);
constexpr size_t kBytes = kOffStatus + 256;
static_assert(kBytes == PART_NOALLOC_SORT_SCRATCH_BYTES,
              "part.h states the scratch size; keep the two in step");

static __device__ __align__(256) unsigned char g_sort_scratch[kBytes];

constexpr int kMaxDevices = 128;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch on the current device (looked up once).
part_status scratch_for_current_device(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(nullptr, PART_ECUDA, std::string("cudaGetDevice: ") +
                                                             cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices)
    return fail(nullptr, PART_EUNSUPPORTED, "device ordinal beyond the scratch table");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sort_scratch);
    if (e != cudaSuccess || p == nullptr)
      return fail(nullptr, PART_ECUDA, std::string("cudaGetSymbolAddress of the sort "
                                                   "scratch: ") + cudaGetErrorString(e));
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return PART_OK;
}

}  // namespace

extern "C" part_status part_sort_fp64_noalloc(const part_grid* grid, int64_t n, double* x,
                                              double* u, double* w, uint64_t* id,
                                              uint32_t* cell_start, void* cuda_stream) {
  part_status s = check_grid(grid);
  if (s != PART_OK) return s;
  if (n < 0 || n > kMaxN)
    return fail(nullptr, PART_EINVAL,
                "n must be in [0, PART_NOALLOC_SORT_MAX_N = 1048576] for the no-allocation "
                "sort; use part_sort with a workspace for more particles");
  if (n > 0 && (!x || !u)) return fail(nullptr, PART_EINVAL, "x and u must not be NULL");
  if (!cell_start) return fail(nullptr, PART_EINVAL, "cell_start must not be NULL");
  if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(u) |
       reinterpret_cast<uintptr_t>(w) | reinterpret_cast<uintptr_t>(id)) % 8 != 0 ||
      reinterpret_cast<uintptr_t>(cell_start) % 4 != 0)
    return fail(nullptr, PART_EINVAL, "an array is not aligned to its element size");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return fail(nullptr, PART_ECUDA, "cudaGetDevice / multiprocessor count query failed");
  if (!device_accessible(dev, x) || !device_accessible(dev, u) || !device_accessible(dev, w) ||
      !device_accessible(dev, id) || !device_accessible(dev, cell_start))
    return fail(nullptr, PART_EINVAL, "an array is not memory the kernels can reach");
  void* base = nullptr;
  if ((s = scratch_for_current_device(&base)) != PART_OK) return s;
  char* b = static_cast<char*>(base);

  // A context on the host stack that points into the static scratch and at
  // the caller's arrays; the sort below is the same launch sequence as
  // part_sort's.
  part_ctx c;
  c.grid = *grid;
  c.prec = PART_FP64;
  c.shape = PART_TSC;
  c.mode = PART_BORIS;
  c.capacity = kMaxN;
  c.nbins = 0;
  c.stream = (cudaStream_t)cuda_stream;
  c.device = dev;
  c.sms = sms;
  c.ncomp = 6;
  c.esize = 8;
  make_geo(grid, 8, &c.geo);
  c.ws = b;
  c.ws_bytes = kBytes;
  c.fpad = nullptr;
  c.keys[0] = reinterpret_cast<uint32_t*>(b + kOffKeys0);
  c.keys[1] = reinterpret_cast<uint32_t*>(b + kOffKeys1);
  c.vals[0] = reinterpret_cast<uint32_t*>(b + kOffVals0);
  c.vals[1] = reinterpret_cast<uint32_t*>(b + kOffVals1);
  c.hist = reinterpret_cast<uint32_t*>(b + kOffHist);
  c.hsum = reinterpret_cast<uint32_t*>(b + kOffHsum);
  c.cstart = cell_start;
  c.tmp = b + kOffTmp;
  c.dpart = nullptr;
  c.samples = nullptr;
  c.status = reinterpret_cast<int*>(b + kOffStatus);
  c.tmap_ok = false;
  c.n = n;
  c.x = x;
  c.off = nullptr;
  c.u = u;
  c.w = w;
  c.id = id;
  c.chi = c.eng = c.n_old = nullptr;
  c.bound = true;
  c.fields_set = c.sorted = c.deposit_on = c.deposit_ready = c.samples_ready = false;
  c.launches = 0;

  // The status word is the only scratch that must start at zero; every other
  // region is written before it is read within one call.
  cudaError_t e = cudaMemsetAsync(c.status, 0, sizeof(int), c.stream);
  if (e == cudaSuccess) e = launch_sort(&c);
  if (e != cudaSuccess)
    return fail(nullptr, PART_ECUDA, std::string("part_sort_fp64_noalloc: ") +
                                         cudaGetErrorString(e));
  return PART_OK;
}
