// The host-memory form of pip_project: lon/lat/out in host memory (pinned
// for full speed) are streamed through two device staging buffers on two
// streams, so one chunk's copies overlap the other chunk's projection.
//
// The second stream, the staging buffers and each stream's projection
// scratch are reserved at a set's first host-memory call and kept with the
// set. Allocating them per call (stream-ordered, on a fresh stream) left a
// call waiting now and then for the pool to map memory or for the other
// stream's frees: on the national workload single 1e8-point calls took
// 20-300 ms against 8.55 ms, the copy bound being 8.37 ms.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "pip_internal.cuh"

namespace pip {

struct HostStage {
  std::mutex mu;  // host-memory calls on one set run one at a time
  cudaStream_t s2 = nullptr;
  cudaEvent_t start = nullptr;
  DBuf<double> x[2], y[2];
  DBuf<int32_t> o[2];
  ProjScratch w[2];
  int64_t cap = 0;
};

HostStage* host_stage_new() { return new HostStage(); }

void host_stage_free(HostStage* h) {
  if (!h) return;
  if (h->s2) cudaStreamSynchronize(h->s2);
  for (int b = 0; b < 2; ++b) {  // stream-ordered frees on s2
    h->x[b].release();
    h->y[b].release();
    h->o[b].release();
    h->w[b] = ProjScratch();
  }
  if (h->s2) {
    cudaStreamSynchronize(h->s2);
    cudaStreamDestroy(h->s2);
  }
  if (h->start) cudaEventDestroy(h->start);
  delete h;
}

// Reserve staging and scratch for chunks of `chunk` points (on s2, then
// synchronised, so both streams may use them).
static pip_status host_stage_reserve(pip_set_s* S, HostStage& H, int64_t chunk) {
  if (!H.s2) PIP_CUDA(cudaStreamCreateWithFlags(&H.s2, cudaStreamNonBlocking));
  if (!H.start) PIP_CUDA(cudaEventCreateWithFlags(&H.start, cudaEventDisableTiming));
  bool fits = H.cap >= chunk;
  for (int b = 0; b < 2; ++b) fits = fits && proj_scratch_fits(S, H.w[b], chunk);
  if (fits) return PIP_OK;
  Alloc* al = &S->alloc;
  H.cap = 0;
  for (int b = 0; b < 2; ++b) {
    if (!H.x[b].alloc(al, chunk, H.s2) || !H.y[b].alloc(al, chunk, H.s2) || !H.o[b].alloc(al, chunk, H.s2))
      return fail(PIP_ENOMEM, "pip_project: staging buffers");
    pip_status st = proj_scratch_alloc(S, H.w[b], chunk, H.s2);
    if (st != PIP_OK) return st;
  }
  PIP_CUDA(cudaStreamSynchronize(H.s2));
  H.cap = chunk;
  return PIP_OK;
}

pip_status project_host(pip_set_s* S, const double* lon, const double* lat, int64_t n, int32_t* out,
                        cudaStream_t s, pip_project_stats* stats) {
  const int64_t CH = 1ll << 24;        // largest chunk: 16M points (256 MB of lon/lat)
  const int64_t CH_MIN = 1ll << 21;    // first and last chunks: 2M points
  if (!S->host) return fail(PIP_EINVAL, "pip_project: set has no host staging");
  HostStage& H = *S->host;
  std::lock_guard<std::mutex> lock(H.mu);
  pip_status res = host_stage_reserve(S, H, std::min<int64_t>(CH, n));
  if (res != PIP_OK) return res;
  cudaStream_t st[2] = {s, H.s2};
  PIP_CUDA(cudaEventRecord(H.start, s));
  PIP_CUDA(cudaStreamWaitEvent(H.s2, H.start, 0));
  int64_t residual = 0, items = 0;
  // chunk sizes ramp up from CH_MIN and down again at the end, so the copy
  // of the first chunk and the compute + copy-back of the last one (the
  // parts no other chunk overlaps) stay short
  int64_t c = 0;
  for (int64_t a = 0, i = 0; a < n && res == PIP_OK; a += c, ++i) {
    const int b = (int)(i & 1);
    const int64_t rem = n - a;
    c = std::min<int64_t>({H.cap, CH_MIN << std::min<int64_t>(i, 20), std::max<int64_t>(CH_MIN, rem / 2), rem});
    cudaError_t e = cudaMemcpyAsync(H.x[b].p, lon + a, c * sizeof(double), cudaMemcpyDefault, st[b]);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(H.y[b].p, lat + a, c * sizeof(double), cudaMemcpyDefault, st[b]);
    if (e != cudaSuccess) {
      res = cuda_fail(e, "pip_project: host-to-device copy");
      break;
    }
    pip_project_stats ps{};
    res = project_device_with(S, H.x[b].p, H.y[b].p, c, H.o[b].p, st[b], stats ? &ps : nullptr, &H.w[b]);
    if (res != PIP_OK) break;
    residual += ps.residual;
    items += ps.items;
    e = cudaMemcpyAsync(out + a, H.o[b].p, c * sizeof(int32_t), cudaMemcpyDefault, st[b]);
    if (e != cudaSuccess) res = cuda_fail(e, "pip_project: device-to-host copy");
  }
  // both streams' work is done when this returns, so the buffers are free
  // for the next call
  cudaError_t e0 = cudaStreamSynchronize(H.s2);
  cudaError_t e1 = cudaStreamSynchronize(s);
  if (res == PIP_OK && e0 != cudaSuccess) res = cuda_fail(e0, "pip_project: stream");
  if (res == PIP_OK && e1 != cudaSuccess) res = cuda_fail(e1, "pip_project: stream");
  if (stats && res == PIP_OK) {
    stats->n = n;
    stats->residual = residual;
    stats->items = items;
  }
  return res;
}

}  // namespace pip

pip_set_s::~pip_set_s() {
  pip::host_stage_free(host);
  for (cudaEvent_t e : prof_ev) cudaEventDestroy(e);
}
