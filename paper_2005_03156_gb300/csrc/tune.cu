// Autotuner: picks the cell size (top-grid cell log2 and the subdivision
// ratio / leaf size that shape the trie), the points per crossing work item
// and the shared-memory staging depth for a set, by timing projections of a
// sample of the caller's points with CUDA events; and points per item and
// staging for a batched plan by timing whole plan runs.
#include <algorithm>
#include <vector>

#include "pip_internal.cuh"

namespace pip {
pip_status build_index(pip_set_s* S, cudaStream_t s);
pip_status project_device(pip_set_s* S, const double* lon, const double* lat, int64_t n, int32_t* out,
                          cudaStream_t s, pip_project_stats* stats);
pip_status plan_set_knobs(pip_plan plan, uint32_t ppc, int staged);

// Median device time (ms) of `reps` projections of the sample.
static pip_status time_projection(pip_set_s* S, const double* lon, const double* lat, int64_t n,
                                  int32_t* out, cudaStream_t s, int reps, float& ms) {
  cudaEvent_t a, b;
  PIP_CUDA(cudaEventCreate(&a));
  PIP_CUDA(cudaEventCreate(&b));
  pip_status st = project_device(S, lon, lat, n, out, s, nullptr);  // warm
  std::vector<float> t;
  for (int r = 0; r < reps && st == PIP_OK; ++r) {
    cudaEventRecord(a, s);
    st = project_device(S, lon, lat, n, out, s, nullptr);
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float x = 0;
    cudaEventElapsedTime(&x, a, b);
    t.push_back(x);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (st != PIP_OK) return st;
  std::sort(t.begin(), t.end());
  ms = t[t.size() / 2];
  return PIP_OK;
}

}  // namespace pip

using namespace pip;

extern "C" pip_status pip_set_tune(pip_set set, const double* lon, const double* lat, int64_t n_sample,
                                   void* stream, pip_build_opts* chosen) {
  if (!set) return fail(PIP_EINVAL, "pip_set_tune: NULL set");
  if (n_sample <= 0 || !lon || !lat) return fail(PIP_EINVAL, "pip_set_tune: empty sample");
  if (!is_device_ptr(lon) || !is_device_ptr(lat))
    return fail(PIP_EINVAL, "pip_set_tune: sample must be device memory");
  cudaStream_t s = (cudaStream_t)stream;
  DBuf<int32_t> out;
  if (!out.alloc(&set->alloc, (size_t)n_sample, s)) return fail(PIP_ENOMEM, "pip_set_tune: output");
  const pip_build_opts start = set->opts;  // resolved options of the current index
  pip_build_opts best = start;
  float best_ms = 1e30f;
  // 1) index shape: top cell size, subdivision ratio, leaf size
  const int s0 = start.cell_log2;
  for (int dc = -1; dc <= 1; ++dc)
    for (int ratio : {16, 32, 64, 128})
      for (int le : {4, 8}) {
        pip_build_opts o = start;
        o.cell_log2 = std::max(4, std::min(30, s0 + dc));
        o.size_ratio = ratio;
        o.leaf_edges = le;
        o.max_depth = 0;
        set->opts = o;
        if (build_index(set, s) != PIP_OK) continue;  // too large: skip this shape
        float ms = 0;
        pip_status st = time_projection(set, lon, lat, n_sample, out.p, s, 3, ms);
        if (st != PIP_OK) return st;
        if (ms < best_ms) {
          best_ms = ms;
          best = set->opts;
        }
      }
  // 2) compact leaves on the best shape
  {
    pip_build_opts o = best;
    o.compact_edges = 3;
    set->opts = o;
    if (build_index(set, s) == PIP_OK) {
      float ms = 0;
      pip_status st = time_projection(set, lon, lat, n_sample, out.p, s, 3, ms);
      if (st != PIP_OK) return st;
      if (ms < best_ms) {
        best_ms = ms;
        best = set->opts;
      }
    }
  }
  // 3) crossing work items on the best index
  set->opts = best;
  pip_status st = build_index(set, s);
  if (st != PIP_OK) return st;
  for (int ppc : {128, 256, 512, 1024})
    for (int stages : {-1, 1, 2}) {
      set->opts.pts_per_cta = ppc;
      set->opts.stage_depth = stages;
      float ms = 0;
      st = time_projection(set, lon, lat, n_sample, out.p, s, 3, ms);
      if (st != PIP_OK) return st;
      if (ms < best_ms) {
        best_ms = ms;
        best = set->opts;
      }
    }
  set->opts = best;
  set->info.pts_per_cta = best.pts_per_cta;
  set->info.stage_depth = best.stage_depth;
  PIP_CUDA(cudaStreamSynchronize(s));
  if (chosen) *chosen = best;
  return PIP_OK;
}

extern "C" pip_status pip_plan_tune(pip_plan plan, const pip_query* q, int32_t n_q, void* stream,
                                    int32_t* pts_per_cta, int32_t* staged) {
  if (!plan) return fail(PIP_EINVAL, "pip_plan_tune: NULL plan");
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t a, b;
  PIP_CUDA(cudaEventCreate(&a));
  PIP_CUDA(cudaEventCreate(&b));
  float best_ms = 1e30f;
  int best_ppc = 256, best_st = 0;
  pip_status st = PIP_OK;
  for (int stg : {0, 1}) {
    for (int ppc : {128, 256, 512, 1024}) {
      if ((st = plan_set_knobs(plan, (uint32_t)ppc, stg)) != PIP_OK) break;
      if ((st = pip_plan_run(plan, q, n_q, stream)) != PIP_OK) break;  // warm / capture
      std::vector<float> t;
      for (int r = 0; r < 3; ++r) {
        cudaEventRecord(a, s);
        if ((st = pip_plan_run(plan, q, n_q, stream)) != PIP_OK) break;
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float x = 0;
        cudaEventElapsedTime(&x, a, b);
        t.push_back(x);
      }
      if (st != PIP_OK) break;
      std::sort(t.begin(), t.end());
      if (t[1] < best_ms) {
        best_ms = t[1];
        best_ppc = ppc;
        best_st = stg;
      }
    }
    if (st != PIP_OK) break;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (st != PIP_OK) return st;
  st = plan_set_knobs(plan, (uint32_t)best_ppc, best_st);
  if (st != PIP_OK) return st;
  st = pip_plan_check(plan, stream);
  if (pts_per_cta) *pts_per_cta = best_ppc;
  if (staged) *staged = best_st;
  return st;
}
