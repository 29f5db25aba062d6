// pip_project_noalloc: the plain projection for callers that must not
// allocate device memory while they run.
//
// Some callers cannot call cudaMalloc (or anything that may call it) at the
// point where they project: code running under a CUDA stream capture that
// must not allocate, real-time paths where an allocation's latency or a
// failure is not acceptable, and hosts whose memory is fixed up front. This
// entry point takes its scratch (residual queue, binned residual, superbin
// counts and offsets, scan partials, counters) from one file-scope device
// array of fixed size instead of allocating it.
#include <mutex>

#include "pip_internal.cuh"

namespace pip {
pip_status project_device_scratch(pip_set_s* S, const double* lon, const double* lat, int64_t n,
                                  int32_t* out, cudaStream_t s, Residual* queue, Residual* binned,
                                  uint32_t* hist2, uint64_t* off, uint64_t* scan_tmp, int64_t scan_len,
                                  uint32_t* ctr);
}

namespace {

constexpr int64_t NOALLOC_MAX_POINTS = 1 << 18;      // points per call
constexpr int64_t NOALLOC_MAX_SUPERBINS = 1 << 19;   // superbins of the set
constexpr int64_t SCAN_TMP = 2 * 256;                // 2 x ceil(2^19 / 4096) partials
constexpr size_t BYTES_RES = (size_t)NOALLOC_MAX_POINTS * 16;        // queue, binned
constexpr size_t BYTES_HIST = (size_t)NOALLOC_MAX_SUPERBINS * 8;     // counts + cursors
constexpr size_t BYTES_OFF = (size_t)NOALLOC_MAX_SUPERBINS * 8;
constexpr size_t BYTES_SCAN = (size_t)SCAN_TMP * 8;
constexpr size_t BYTES_CTR = 256;
constexpr size_t SCRATCH_BYTES = 2 * BYTES_RES + BYTES_HIST + BYTES_OFF + BYTES_SCAN + BYTES_CTR;

// The scratch: about 16 MB in every GPU context that loads the library,
// held until the process exits, shared by every call.
static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

// Device address of g_scratch, resolved once per device with that device
// current (in host code the symbol is only a host-side stand-in).
std::mutex g_mu;
void* g_addr[64] = {nullptr};

pip_status scratch_address(int dev, unsigned char** p) {
  if (dev < 0 || dev >= 64) return pip::fail(PIP_EINVAL, "pip_project_noalloc: device index");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* a = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&a, g_scratch);
    if (e != cudaSuccess) return pip::cuda_fail(e, "pip_project_noalloc: cudaGetSymbolAddress");
    g_addr[dev] = a;
  }
  *p = (unsigned char*)g_addr[dev];
  return PIP_OK;
}

}  // namespace

using namespace pip;

// No allocation happens here: every scratch buffer is carved from
// g_scratch. The first call on a device resolves the array's address (make
// that first call before any stream capture). Calls that overlap on the GPU
// (other streams, other threads) share the array and race: serialise them.
extern "C" pip_status pip_project_noalloc(pip_set set, const double* lon, const double* lat, int64_t n,
                                          int32_t* out, void* stream) {
  if (!set) return fail(PIP_EINVAL, "pip_project_noalloc: NULL set");
  if (n < 0) return fail(PIP_EINVAL, "pip_project_noalloc: n < 0");
  if (n == 0) return PIP_OK;
  if (!lon || !lat || !out) return fail(PIP_EINVAL, "pip_project_noalloc: NULL pointer with n > 0");
  if (n > NOALLOC_MAX_POINTS)
    return fail(PIP_EINVAL, "pip_project_noalloc: at most 262144 points per call");
  if ((int64_t)set->view.n_sb > NOALLOC_MAX_SUPERBINS)
    return fail(PIP_EINVAL, "pip_project_noalloc: the set has more than 524288 superbins");
  if (!is_device_ptr(lon) || !is_device_ptr(lat) || !is_device_ptr(out))
    return fail(PIP_EINVAL, "pip_project_noalloc: lon, lat and out must be device memory");
  int dev = 0;
  PIP_CUDA(cudaGetDevice(&dev));
  if (dev != set->device) return fail(PIP_EINVAL, "pip_project_noalloc: the set lives on another device");
  unsigned char* base = nullptr;
  pip_status st = scratch_address(dev, &base);
  if (st != PIP_OK) return st;
  Residual* queue = (Residual*)base;
  Residual* binned = (Residual*)(base + BYTES_RES);
  uint32_t* hist2 = (uint32_t*)(base + 2 * BYTES_RES);
  uint64_t* off = (uint64_t*)(base + 2 * BYTES_RES + BYTES_HIST);
  uint64_t* scan_tmp = (uint64_t*)(base + 2 * BYTES_RES + BYTES_HIST + BYTES_OFF);
  uint32_t* ctr = (uint32_t*)(base + 2 * BYTES_RES + BYTES_HIST + BYTES_OFF + BYTES_SCAN);
  return project_device_scratch(set, lon, lat, n, out, (cudaStream_t)stream, queue, binned, hist2, off,
                                scan_tmp, SCAN_TMP, ctr);
}
