// Error plumbing, device memory, exclusive scans and the diagnostic
// quantizer entry point.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <mutex>
#include <string>

#include "pip_internal.cuh"

namespace pip {

static thread_local std::string g_last_error;
static std::atomic<int64_t> g_launches{0};

void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void set_error(const std::string& msg) { g_last_error = msg; }

pip_status fail(pip_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

pip_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return e == cudaErrorMemoryAllocation ? PIP_ENOMEM : PIP_ECUDA;
}

int num_sms() {
  static std::atomic<int> cached[64];  // per device; 0 = not read yet
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  int v = cached[dev].load(std::memory_order_relaxed);
  if (!v) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    v = n > 0 ? n : 1;
    cached[dev].store(v, std::memory_order_relaxed);
  }
  return v;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void* Alloc::get(size_t bytes, cudaStream_t s) {
  if (bytes == 0) return nullptr;
  if (has_hook) return hook.alloc(bytes, (void*)s, hook.ctx);
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void Alloc::put(void* p, cudaStream_t s) {
  if (!p) return;
  if (has_hook) {
    hook.free(p, (void*)s, hook.ctx);
    return;
  }
  cudaFreeAsync(p, s);
}

// ---------------------------------------------------------------------------
// Exclusive scan: 4096 elements per block (256 threads x 16), block sums
// scanned recursively, then each block rescans with its offset.
// ---------------------------------------------------------------------------
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ uint64_t warp_incl_scan(uint64_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint64_t t = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v += t;
  }
  return v;
}

// Exclusive scan of one value per thread across the block; returns the
// block total through *total.
__device__ __forceinline__ uint64_t block_excl_scan(uint64_t v, uint64_t* total) {
  __shared__ uint64_t warp_sums[SCAN_THREADS / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t incl = warp_incl_scan(v);
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint64_t w = lane < SCAN_THREADS / 32 ? warp_sums[lane] : 0;
    const uint64_t wi = warp_incl_scan(w);
    if (lane < SCAN_THREADS / 32) warp_sums[lane] = wi - w;
    if (lane == SCAN_THREADS / 32 - 1) *total = wi;
  }
  __syncthreads();
  const uint64_t r = warp_sums[warp] + incl - v;
  __syncthreads();
  return r;
}

template <class In>
__global__ void k_block_sums(const In* __restrict__ in, int64_t n, uint64_t* __restrict__ sums) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  uint64_t s = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i)
    if (base + i < n) s += (uint64_t)in[base + i];
  __shared__ uint64_t total;
  block_excl_scan(s, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

template <class In>
__global__ void k_block_scan(const In* __restrict__ in, uint64_t* __restrict__ out, int64_t n,
                             const uint64_t* __restrict__ offs, uint64_t* total_dev) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  uint64_t v[SCAN_ITEMS];
  uint64_t s = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    v[i] = base + i < n ? (uint64_t)in[base + i] : 0;
    s += v[i];
  }
  __shared__ uint64_t total;
  uint64_t run = block_excl_scan(s, &total) + (offs ? offs[blockIdx.x] : 0);
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
  if (total_dev && blockIdx.x == gridDim.x - 1 && threadIdx.x == SCAN_THREADS - 1) *total_dev = run;
}

template <class In>
static pip_status scan_impl(Alloc& al, const In* in, uint64_t* out, int64_t n, uint64_t* total_dev,
                            cudaStream_t s) {
  if (n <= 0) {
    if (total_dev) PIP_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(uint64_t), s));
    return PIP_OK;
  }
  const int64_t blocks = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (blocks == 1) {
    k_block_scan<In><<<1, SCAN_THREADS, 0, s>>>(in, out, n, nullptr, total_dev);
    PIP_CUDA(cudaGetLastError());
    count_launches(1);
    return PIP_OK;
  }
  DBuf<uint64_t> sums, offs;
  if (!sums.alloc(&al, blocks, s) || !offs.alloc(&al, blocks, s))
    return fail(PIP_ENOMEM, "scan: scratch allocation failed");
  k_block_sums<In><<<(unsigned)blocks, SCAN_THREADS, 0, s>>>(in, n, sums.p);
  PIP_CUDA(cudaGetLastError());
  pip_status st = scan_impl<uint64_t>(al, sums.p, offs.p, blocks, nullptr, s);
  if (st != PIP_OK) return st;
  k_block_scan<In><<<(unsigned)blocks, SCAN_THREADS, 0, s>>>(in, out, n, offs.p, total_dev);
  PIP_CUDA(cudaGetLastError());
  count_launches(2);
  return PIP_OK;
}

// The same exclusive scan without allocating: block sums live in caller
// scratch `tmp` of at least 2 * ceil(n / 4096) entries; n <= 4096 * 4096.
pip_status scan_u32_to_u64_scratch(const uint32_t* in, uint64_t* out, int64_t n, uint64_t* tmp,
                                   int64_t tmp_len, cudaStream_t s) {
  if (n <= 0) return PIP_OK;
  const int64_t blocks = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (blocks == 1) {
    k_block_scan<uint32_t><<<1, SCAN_THREADS, 0, s>>>(in, out, n, nullptr, nullptr);
    PIP_CUDA(cudaGetLastError());
    count_launches(1);
    return PIP_OK;
  }
  if (blocks > SCAN_TILE || 2 * blocks > tmp_len) return fail(PIP_EINVAL, "scan: scratch too small");
  k_block_sums<uint32_t><<<(unsigned)blocks, SCAN_THREADS, 0, s>>>(in, n, tmp);
  k_block_scan<uint64_t><<<1, SCAN_THREADS, 0, s>>>(tmp, tmp + blocks, blocks, nullptr, nullptr);
  k_block_scan<uint32_t><<<(unsigned)blocks, SCAN_THREADS, 0, s>>>(in, out, n, tmp + blocks, nullptr);
  PIP_CUDA(cudaGetLastError());
  count_launches(3);
  return PIP_OK;
}

pip_status scan_u32_to_u64(Alloc& al, const uint32_t* in, uint64_t* out, int64_t n,
                           uint64_t* total_dev, cudaStream_t s) {
  return scan_impl<uint32_t>(al, in, out, n, total_dev, s);
}

pip_status scan_u64(Alloc& al, const uint64_t* in, uint64_t* out, int64_t n, uint64_t* total_dev,
                    cudaStream_t s) {
  return scan_impl<uint64_t>(al, in, out, n, total_dev, s);
}

__global__ void k_quantize(const double* __restrict__ v, int64_t n, int32_t* __restrict__ q,
                           uint8_t* __restrict__ valid) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t r = 0;
    const bool ok = quantize_double(v[i], r);
    q[i] = ok ? r : 0;
    valid[i] = ok ? 1 : 0;
  }
}

}  // namespace pip

using namespace pip;

extern "C" const char* pip_last_error(void) { return g_last_error.c_str(); }

// 1.1.0: compact leaves and the split-ratio fallback (options and set facts), pip_locate,
// per-slot leaf records.
extern "C" int32_t pip_version(void) { return 10100; }

extern "C" int64_t pip_kernel_launches(void) { return g_launches.load(); }

extern "C" pip_status pip_quantize(const double* v, int64_t n, int32_t* q, uint8_t* valid,
                                   void* stream) {
  if (n < 0) return fail(PIP_EINVAL, "pip_quantize: n < 0");
  if (n == 0) return PIP_OK;
  if (!v || !q || !valid) return fail(PIP_EINVAL, "pip_quantize: NULL pointer");
  if (!is_device_ptr(v) || !is_device_ptr(q) || !is_device_ptr(valid))
    return fail(PIP_EINVAL, "pip_quantize: pointers must be device memory");
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 8);
  k_quantize<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(v, n, q, valid);
  PIP_CUDA(cudaGetLastError());
  return PIP_OK;
}
