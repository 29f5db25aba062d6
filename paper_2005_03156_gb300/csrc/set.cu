// Polygon-set lifecycle: load (host or device arrays), rebuild, info, free.
#include <algorithm>
#include <cstring>
#include <memory>

#include "pip_internal.cuh"

namespace pip {
pip_status build_index(pip_set_s* S, cudaStream_t s);
pip_status load_validate(pip_set_s* S, cudaStream_t s);
pip_status quantize_vertices(const double* x, const double* y, int64_t n, int32_t* qx, int32_t* qy,
                             Alloc* al, cudaStream_t s);
pip_status top_candidates_export(pip_set_s* S, int mode, int64_t* off, int32_t* ids, int64_t cap,
                                 cudaStream_t s);

__global__ void k_max_i32(const int32_t* __restrict__ a, int64_t n, int* __restrict__ out) {
  int m = -1;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, a[i]);
  atomicMax(out, m);
}

template <class T>
static pip_status to_device(DBuf<T>& dst, const T* src, int64_t n, Alloc* al, cudaStream_t s,
                            const char* what) {
  if (!dst.alloc(al, (size_t)n + 1, s)) return fail(PIP_ENOMEM, std::string("pip_set_load: ") + what);
  if (n > 0) PIP_CUDA(cudaMemcpyAsync(dst.p, src, n * sizeof(T), cudaMemcpyDefault, s));
  return PIP_OK;
}

template <class V>
static pip_status load_common(const V* vx, const V* vy, int64_t n_vert, const int64_t* ring_off,
                              int64_t n_ring, const int64_t* poly_ring_off, int32_t n_poly,
                              const int32_t* const* parent, int32_t n_levels,
                              const pip_build_opts* opts, const pip_allocator* alloc, void* stream,
                              pip_set* out) {
  if (!out) return fail(PIP_EINVAL, "pip_set_load: out is NULL");
  *out = nullptr;
  if (n_vert < 0 || n_ring < 0 || n_poly < 0 || n_levels < 0)
    return fail(PIP_EINVAL, "pip_set_load: negative size");
  if (n_poly >= (1 << 30)) return fail(PIP_EINVAL, "pip_set_load: n_poly must be < 2^30");
  if (n_levels > MAX_LEVELS - 2) return fail(PIP_EINVAL, "pip_set_load: too many hierarchy levels");
  if ((n_vert > 0 && (!vx || !vy)) || !ring_off || !poly_ring_off)
    return fail(PIP_EINVAL, "pip_set_load: NULL array");
  if (n_levels > 0 && !parent) return fail(PIP_EINVAL, "pip_set_load: parent is NULL");
  for (int l = 0; l < n_levels; ++l)
    if (!parent[l]) return fail(PIP_EINVAL, "pip_set_load: parent level is NULL");
  if (alloc && (!alloc->alloc || !alloc->free)) return fail(PIP_EINVAL, "pip_set_load: incomplete allocator");
  cudaStream_t s = (cudaStream_t)stream;
  std::unique_ptr<pip_set_s> S(new pip_set_s());
  PIP_CUDA(cudaGetDevice(&S->device));
  S->host = host_stage_new();
  if (alloc) {
    S->alloc.hook = *alloc;
    S->alloc.has_hook = true;
  }
  if (opts) S->opts = *opts;
  S->n_vert = n_vert;
  S->n_ring = n_ring;
  S->n_poly = n_poly;
  Alloc* al = &S->alloc;
  pip_status st;
  if (!S->vx.alloc(al, (size_t)n_vert + 1, s) || !S->vy.alloc(al, (size_t)n_vert + 1, s))
    return fail(PIP_ENOMEM, "pip_set_load: vertices");
  if (std::is_same<V, int32_t>::value) {
    if (n_vert > 0) {
      PIP_CUDA(cudaMemcpyAsync(S->vx.p, vx, n_vert * sizeof(int32_t), cudaMemcpyDefault, s));
      PIP_CUDA(cudaMemcpyAsync(S->vy.p, vy, n_vert * sizeof(int32_t), cudaMemcpyDefault, s));
    }
  } else {
    DBuf<double> dx, dy;
    if ((st = to_device(dx, (const double*)vx, n_vert, al, s, "vx")) != PIP_OK) return st;
    if ((st = to_device(dy, (const double*)vy, n_vert, al, s, "vy")) != PIP_OK) return st;
    if (n_vert > 0 && (st = quantize_vertices(dx.p, dy.p, n_vert, S->vx.p, S->vy.p, al, s)) != PIP_OK)
      return st;
  }
  if ((st = to_device(S->ring_off, ring_off, n_ring + 1, al, s, "ring_off")) != PIP_OK) return st;
  if ((st = to_device(S->poly_ring_off, poly_ring_off, (int64_t)n_poly + 1, al, s, "poly_ring_off")) != PIP_OK)
    return st;
  S->level_len.assign(1, n_poly);
  S->parent.resize(n_levels);
  DBuf<int> mx;
  if (!mx.alloc(al, 1, s)) return fail(PIP_ENOMEM, "pip_set_load: scratch");
  for (int l = 0; l < n_levels; ++l) {
    const int64_t len = S->level_len[l];
    if ((st = to_device(S->parent[l], parent[l], len, al, s, "parent")) != PIP_OK) return st;
    const int init = -1;
    PIP_CUDA(cudaMemcpyAsync(mx.p, &init, sizeof(int), cudaMemcpyHostToDevice, s));
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((len + 255) / 256, 4096));
    k_max_i32<<<g, 256, 0, s>>>(S->parent[l].p, len, mx.p);
    PIP_CUDA(cudaGetLastError());
    int m = -1;
    PIP_CUDA(cudaMemcpyAsync(&m, mx.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    PIP_CUDA(cudaStreamSynchronize(s));
    S->level_len.push_back(std::max<int64_t>(1, (int64_t)m + 1));
  }
  if (!S->status.alloc(al, 2, s)) return fail(PIP_ENOMEM, "pip_set_load: status word");
  PIP_CUDA(cudaMemsetAsync(S->status.p, 0, 2 * sizeof(uint32_t), s));
  if ((st = load_validate(S.get(), s)) != PIP_OK) return st;
  if ((st = build_index(S.get(), s)) != PIP_OK) return st;
  PIP_CUDA(cudaStreamSynchronize(s));
  *out = S.release();
  return PIP_OK;
}

}  // namespace pip

using namespace pip;

extern "C" pip_status pip_set_load_i32(const int32_t* vx, const int32_t* vy, int64_t n_vert,
                                       const int64_t* ring_off, int64_t n_ring,
                                       const int64_t* poly_ring_off, int32_t n_poly,
                                       const int32_t* const* parent, int32_t n_levels,
                                       const pip_build_opts* opts, const pip_allocator* alloc,
                                       void* stream, pip_set* out) {
  return load_common<int32_t>(vx, vy, n_vert, ring_off, n_ring, poly_ring_off, n_poly, parent, n_levels,
                              opts, alloc, stream, out);
}

extern "C" pip_status pip_set_load_f64(const double* vx, const double* vy, int64_t n_vert,
                                       const int64_t* ring_off, int64_t n_ring,
                                       const int64_t* poly_ring_off, int32_t n_poly,
                                       const int32_t* const* parent, int32_t n_levels,
                                       const pip_build_opts* opts, const pip_allocator* alloc,
                                       void* stream, pip_set* out) {
  return load_common<double>(vx, vy, n_vert, ring_off, n_ring, poly_ring_off, n_poly, parent, n_levels,
                             opts, alloc, stream, out);
}

extern "C" pip_status pip_set_rebuild(pip_set set, const pip_build_opts* opts, void* stream) {
  if (!set) return fail(PIP_EINVAL, "pip_set_rebuild: NULL set");
  const pip_build_opts saved = set->opts;
  set->opts = opts ? *opts : pip_build_opts{};
  cudaStream_t s = (cudaStream_t)stream;
  pip_status st = build_index(set, s);
  if (st != PIP_OK) {
    set->opts = saved;
    pip_status st2 = build_index(set, s);  // restore the previous index
    (void)st2;
    return st;
  }
  PIP_CUDA(cudaStreamSynchronize(s));
  return PIP_OK;
}

extern "C" pip_status pip_set_info(pip_set set, pip_set_info_t* info) {
  if (!set || !info) return fail(PIP_EINVAL, "pip_set_info: NULL argument");
  *info = set->info;
  return PIP_OK;
}

extern "C" pip_status pip_set_free(pip_set set) {
  if (!set) return PIP_OK;
  int cur = 0;  // free on the set's own device (its streams and pool live there)
  const int dev = set->device;
  cudaGetDevice(&cur);
  if (cur != dev) cudaSetDevice(dev);
  cudaDeviceSynchronize();
  delete set;
  cudaDeviceSynchronize();
  if (cur != dev) cudaSetDevice(cur);
  return PIP_OK;
}

extern "C" pip_status pip_set_check(pip_set set, void* stream) {
  if (!set) return fail(PIP_EINVAL, "pip_set_check: NULL set");
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t w = 0;
  PIP_CUDA(cudaMemcpyAsync(&w, set->status.p, sizeof(w), cudaMemcpyDeviceToHost, s));
  PIP_CUDA(cudaStreamSynchronize(s));
  if (w) {
    PIP_CUDA(cudaMemsetAsync(set->status.p, 0, sizeof(uint32_t), s));
    PIP_CUDA(cudaStreamSynchronize(s));
    return fail(PIP_ETIMEOUT, "a bounded device wait ran out (status word set)");
  }
  return PIP_OK;
}

extern "C" pip_status pip_set_top_candidates(pip_set set, int32_t cand_mode, int64_t* off,
                                             int32_t* ids, int64_t cap) {
  if (!set || !off || (cap > 0 && !ids)) return fail(PIP_EINVAL, "pip_set_top_candidates: NULL argument");
  if (cand_mode != 1 && cand_mode != 2) return fail(PIP_EINVAL, "pip_set_top_candidates: mode 1 or 2");
  pip_status st = top_candidates_export(set, cand_mode, off, ids, cap, 0);
  return st;
}

extern "C" pip_status pip_profile_enable(pip_set set, int32_t capacity) {
  if (!set || capacity < 0) return fail(PIP_EINVAL, "pip_profile_enable: bad argument");
  cudaDeviceSynchronize();
  for (cudaEvent_t e : set->prof_ev) cudaEventDestroy(e);
  set->prof_ev.clear();
  set->prof_cap = 0;
  set->prof_n = 0;
  for (int32_t i = 0; i < 4 * capacity; ++i) {
    cudaEvent_t e;
    PIP_CUDA(cudaEventCreate(&e));
    set->prof_ev.push_back(e);
  }
  set->prof_cap = capacity;
  return PIP_OK;
}

extern "C" pip_status pip_profile_read(pip_set set, double* k1_ms, double* bin_ms, double* k3_ms,
                                       int32_t* n) {
  if (!set || !n || *n < 0) return fail(PIP_EINVAL, "pip_profile_read: bad argument");
  PIP_CUDA(cudaDeviceSynchronize());
  const int32_t m = std::min(*n, set->prof_n);
  for (int32_t i = 0; i < m; ++i) {
    float a = 0, b = 0, c = 0;
    PIP_CUDA(cudaEventElapsedTime(&a, set->prof_ev[4 * i + 0], set->prof_ev[4 * i + 1]));
    PIP_CUDA(cudaEventElapsedTime(&b, set->prof_ev[4 * i + 1], set->prof_ev[4 * i + 2]));
    PIP_CUDA(cudaEventElapsedTime(&c, set->prof_ev[4 * i + 2], set->prof_ev[4 * i + 3]));
    if (k1_ms) k1_ms[i] = a;
    if (bin_ms) bin_ms[i] = b;
    if (k3_ms) k3_ms[i] = c;
  }
  *n = m;
  set->prof_n = 0;
  return PIP_OK;
}

namespace pip {
struct ParentChain {
  const int32_t* level[MAX_LEVELS];
  int32_t n_levels;
};

// out[i] = the level-`level` ancestor of block ids[i] (-1 stays -1).
__global__ void k_parent_ids(ParentChain pc, const int32_t* __restrict__ ids, int64_t n,
                             int32_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t v = ids[i];
    for (int l = 0; l < pc.n_levels && v >= 0; ++l) v = pc.level[l][v];
    out[i] = v;
  }
}
}  // namespace pip

extern "C" pip_status pip_parent_ids(pip_set set, const int32_t* ids, int64_t n, int32_t level,
                                     int32_t* out, void* stream) {
  if (!set) return fail(PIP_EINVAL, "pip_parent_ids: NULL set");
  if (n < 0 || level < 0 || level > (int32_t)set->parent.size())
    return fail(PIP_EINVAL, "pip_parent_ids: bad n or level");
  if (n == 0) return PIP_OK;
  if (!ids || !out || !is_device_ptr(ids) || !is_device_ptr(out))
    return fail(PIP_EINVAL, "pip_parent_ids: ids and out must be device memory");
  ParentChain pc{};
  pc.n_levels = level;
  for (int l = 0; l < level; ++l) pc.level[l] = set->parent[l].p;
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, num_sms() * 8));
  k_parent_ids<<<g, 256, 0, (cudaStream_t)stream>>>(pc, ids, n, out);
  PIP_CUDA(cudaGetLastError());
  count_launches(1);
  return PIP_OK;
}

// Which cell of the index answers each lattice point (Sec. IV: interior
// cells answer without a test; boundary cells keep the crossing test). The
// walk is the one the classify kernels take.
__global__ void k_locate(IndexView ix, const int32_t* __restrict__ qx, const int32_t* __restrict__ qy,
                         int64_t n, uint32_t* __restrict__ code) {
  const uint32_t m = (1u << NODE_K) - 1u;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = qx[i], y = qy[i];
    const uint32_t dx = (uint32_t)x - (uint32_t)ix.gx0, dy = (uint32_t)y - (uint32_t)ix.gy0;
    const uint32_t cx = dx >> ix.s0, cy = dy >> ix.s0;
    if (x < ix.gx0 || y < ix.gy0 || cx >= ix.nx || cy >= ix.ny) {
      code[i] = PIP_LOC_OUTSIDE;
      continue;
    }
    uint32_t d = ix.table[(size_t)cy * ix.nx + cx];
    uint32_t depth = 0;
    int s = ix.s0;
    while (!ix.compact && (d >> 30) == TAG_CHILD) {  // 16-byte entries
      s = s > NODE_K ? s - NODE_K : 0;
      const uint4 e = ix.nodes[d & PAYLOAD_MASK];
      if ((e.y >> 30) == E16_NODE) ++depth;  // leaf and id entries belong to their parent's level
      d = entry_step(e, (((dy >> s) & m) << NODE_K) | ((dx >> s) & m));
    }
    while ((d >> 30) == TAG_CHILD && !(d & DESC_COMPACT)) {
      s -= NODE_K;
      const uint32_t* w = reinterpret_cast<const uint32_t*>(ix.nodes + 2 * (size_t)(d & SLOT_MASK));
      NodeWords nw;
      for (int k = 0; k < 8; ++k) nw.w[k] = w[k];
      d = node_step<true>(nw, (((dy >> s) & m) << NODE_K) | ((dx >> s) & m));
      ++depth;
    }
    const uint32_t tag = d >> 30;
    const uint32_t kind = tag == TAG_EMPTY ? PIP_LOC_EMPTY
                        : tag == TAG_INTERIOR ? PIP_LOC_INTERIOR
                        : tag == TAG_LEAF ? PIP_LOC_RESIDUAL : PIP_LOC_COMPACT;
    code[i] = kind | (depth << 8);
  }
}

extern "C" pip_status pip_locate(pip_set set, const int32_t* qx, const int32_t* qy, int64_t n, uint32_t* code,
                                 void* stream) {
  if (!set) return fail(PIP_EINVAL, "pip_locate: NULL set");
  if (n < 0) return fail(PIP_EINVAL, "pip_locate: n < 0");
  if (n == 0) return PIP_OK;
  if (!qx || !qy || !code || !is_device_ptr(qx) || !is_device_ptr(qy) || !is_device_ptr(code))
    return fail(PIP_EINVAL, "pip_locate: qx, qy and code must be device memory");
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, num_sms() * 8));
  k_locate<<<g, 256, 0, (cudaStream_t)stream>>>(set->view, qx, qy, n, code);
  PIP_CUDA(cudaGetLastError());
  count_launches(1);
  return PIP_OK;
}
