// The host-memory form of pip_project: lon/lat/out in host memory (pinned
// for full speed) are streamed through two device staging buffers on two
// streams, so one chunk's copies overlap the other chunk's projection.
#include <algorithm>
#include <cstring>

#include "pip_internal.cuh"

namespace pip {

pip_status project_device(pip_set_s* S, const double* lon, const double* lat, int64_t n, int32_t* out,
                          cudaStream_t s, pip_project_stats* stats);

pip_status project_host(pip_set_s* S, const double* lon, const double* lat, int64_t n, int32_t* out,
                        cudaStream_t s, pip_project_stats* stats) {
  const int64_t CH = 1ll << 24;        // largest chunk: 16M points (256 MB of lon/lat)
  const int64_t CH_MIN = 1ll << 21;    // first and last chunks: 2M points
  const int64_t chunk = std::min<int64_t>(CH, n);
  Alloc* al = &S->alloc;
  cudaStream_t st[2] = {s, nullptr};
  PIP_CUDA(cudaStreamCreateWithFlags(&st[1], cudaStreamNonBlocking));
  struct Buf {
    DBuf<double> x, y;
    DBuf<int32_t> o;
  } buf[2];
  pip_status res = PIP_OK;
  cudaEvent_t start_ev;
  cudaEventCreateWithFlags(&start_ev, cudaEventDisableTiming);
  cudaEventRecord(start_ev, s);
  cudaStreamWaitEvent(st[1], start_ev, 0);
  for (int b = 0; b < 2 && res == PIP_OK; ++b) {
    if (!buf[b].x.alloc(al, chunk, st[b]) || !buf[b].y.alloc(al, chunk, st[b]) ||
        !buf[b].o.alloc(al, chunk, st[b]))
      res = fail(PIP_ENOMEM, "pip_project: staging buffers");
  }
  int64_t residual = 0, items = 0;
  // chunk sizes ramp up from CH_MIN and down again at the end, so the copy
  // of the first chunk and the compute + copy-back of the last one (the
  // parts no other chunk overlaps) stay short
  int64_t c = 0;
  for (int64_t a = 0, i = 0; a < n && res == PIP_OK; a += c, ++i) {
    const int b = (int)(i & 1);
    const int64_t rem = n - a;
    c = std::min<int64_t>({chunk, CH_MIN << std::min<int64_t>(i, 20), std::max<int64_t>(CH_MIN, rem / 2), rem});
    cudaError_t e = cudaMemcpyAsync(buf[b].x.p, lon + a, c * sizeof(double), cudaMemcpyDefault, st[b]);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(buf[b].y.p, lat + a, c * sizeof(double), cudaMemcpyDefault, st[b]);
    if (e != cudaSuccess) {
      res = cuda_fail(e, "pip_project: host-to-device copy");
      break;
    }
    pip_project_stats ps{};
    res = project_device(S, buf[b].x.p, buf[b].y.p, c, buf[b].o.p, st[b], stats ? &ps : nullptr);
    if (res != PIP_OK) break;
    residual += ps.residual;
    items += ps.items;
    e = cudaMemcpyAsync(out + a, buf[b].o.p, c * sizeof(int32_t), cudaMemcpyDefault, st[b]);
    if (e != cudaSuccess) res = cuda_fail(e, "pip_project: device-to-host copy");
  }
  for (int b = 0; b < 2; ++b) {
    buf[b].x.release();
    buf[b].y.release();
    buf[b].o.release();
  }
  cudaError_t e0 = cudaStreamSynchronize(st[1]);
  cudaError_t e1 = cudaStreamSynchronize(st[0]);
  cudaStreamDestroy(st[1]);
  cudaEventDestroy(start_ev);
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
