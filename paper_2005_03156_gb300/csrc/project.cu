// The plain projection path: K1 classify -> K2 bin -> K3 cross on one
// stream, plus the chunked host-memory pipeline.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>

#include "kernels.cuh"

namespace pip {

// ------------------------------------------------------------------- K1
// Loads of one step: 4 consecutive points per thread.
template <bool VEC>
__device__ __forceinline__ void load4(const double* __restrict__ lon, const double* __restrict__ lat,
                                      int64_t n, int64_t g, double (&x)[4], double (&y)[4]) {
  const int64_t i0 = g * 4;
  if (VEC && i0 + 3 < n) {
    const double2 a0 = __ldcs(reinterpret_cast<const double2*>(lon) + 2 * g);
    const double2 a1 = __ldcs(reinterpret_cast<const double2*>(lon) + 2 * g + 1);
    const double2 b0 = __ldcs(reinterpret_cast<const double2*>(lat) + 2 * g);
    const double2 b1 = __ldcs(reinterpret_cast<const double2*>(lat) + 2 * g + 1);
    x[0] = a0.x; x[1] = a0.y; x[2] = a1.x; x[3] = a1.y;
    y[0] = b0.x; y[1] = b0.y; y[2] = b1.x; y[3] = b1.y;
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const bool have = i0 + j < n;
      x[j] = have ? lon[i0 + j] : __longlong_as_double(0x7FF8000000000000ll);  // NaN: invalid
      y[j] = have ? lat[i0 + j] : 0.0;
    }
  }
}

// VEC: lon/lat/out are 16-byte aligned; each thread takes 4 consecutive
// points per step (two double2 loads per coordinate, one int4 store). The
// grid is persistent (one wave) and the next step's loads are issued before
// the current step's trie walk, so the stream's DRAM latency overlaps the
// dependent lookups.
template <bool VEC>
__global__ void __launch_bounds__(K1_THREADS, 3) k_classify_points(
    IndexView ix, const double* __restrict__ lon, const double* __restrict__ lat, int64_t n,
    int32_t* __restrict__ out, Residual* __restrict__ queue, uint32_t* __restrict__ qcount,
    uint32_t* __restrict__ hist) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t groups = (n + 3) / 4;
  // iterate whole warps together so warp-level appends stay uniform
  const int64_t rounds = (groups + stride - 1) / stride;
  double nx[4], ny[4];
  load4<VEC>(lon, lat, n, tid, nx, ny);
  for (int64_t it = 0; it < rounds; ++it) {
    const int64_t g = it * stride + tid;
    const int64_t i0 = g * 4;
    double x[4], y[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      x[j] = nx[j];
      y[j] = ny[j];
    }
    if (it + 1 < rounds) load4<VEC>(lon, lat, n, g + stride, nx, ny);
    int32_t id[4], qx[4], qy[4];
    uint32_t d[4];
    uint32_t mask = classify4(ix, x, y, id, qx, qy, d);
    if (VEC && i0 + 3 < n) {
      __stcs(reinterpret_cast<int4*>(out) + g, make_int4(id[0], id[1], id[2], id[3]));
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (i0 + j < n) out[i0 + j] = id[j];
    }
    append_residual(mask, qx, qy, d, (uint32_t)i0, queue, qcount, hist, 0u);
  }
}

// ------------------------------------------------------ K1, deferred-queue form
// In the lockstep form above a lane walks its 4 points level by level, so at
// every level the warp waits for the deepest of its 128 points (in the state
// workload ~39 % of points stop at the top grid, ~38 % one level down, ~20 %
// two, ~3 % three, yet nearly every warp takes all three node levels). Here
// a step of 4 points per lane only quantizes them, reads their top-grid
// descriptors and, with 16-byte entries, the first trie level (whose
// entries stay in L2; 7 % faster than leaving it to the ring); points whose
// cell is split further go onto a per-warp ring in shared memory, and
// whenever the ring holds 128 entries the warp takes one trie level for all
// of them at once (4 per lane) and puts back the ones that are still split. Every dependent index load then serves a live point, and
// the lanes stay converged. Ids of points resolved below the top grid are
// stored one by one; their sectors were written by the step's 16-byte store
// moments before and are still in L2. Residual points go straight to the
// global queue through a ChunkWriter (per-warp chunks reserved one ahead;
// holes are marked and skipped by K2; the residual count is qcount[2]).
// Shared memory holds only the ring (17 KB a CTA): the rest of the SM's
// 256 KB stays L1, which holds the sectors of the index loads in flight; a
// larger carve-out measurably throttles them.
constexpr int DQ_THREADS = 128;

template <bool VEC, bool COMPACT>
__global__ void __launch_bounds__(DQ_THREADS, 5) k_classify_dq(
    IndexView ix, const double* __restrict__ lon, const double* __restrict__ lat, int64_t n,
    int32_t* __restrict__ out, Residual* __restrict__ queue, uint32_t* __restrict__ qcount,
    uint32_t* __restrict__ hist) {
  __shared__ uint4 ring[DQ_THREADS / 32][TRING];
  __shared__ uint8_t ring_sh[DQ_THREADS / 32][TRING];
  const uint32_t full = 0xffffffffu;
  const uint64_t pol = policy_evict_last();
  TrieRing tr;
  tr.rq = ring[threadIdx.x >> 5];
  tr.rs = ring_sh[threadIdx.x >> 5];
  ChunkWriter res;  // residual entries of this warp

  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t groups = (n + 3) / 4;
  const int64_t rounds = (groups + stride - 1) / stride;  // whole warps iterate together
  double nx[4], ny[4];
  load4<VEC>(lon, lat, n, tid, nx, ny);
#pragma unroll 1
  for (int64_t it = 0; it < rounds; ++it) {
    const int64_t g = it * stride + tid;
    const int64_t i0 = g * 4;
    double x[4], y[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      x[j] = nx[j];
      y[j] = ny[j];
    }
    if (it + 1 < rounds) load4<VEC>(lon, lat, n, g + stride, nx, ny);
    int32_t qx[4], qy[4], id[4];
    uint32_t d[4], idx[4];
    int sh[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      qx[j] = qy[j] = 0;
      const bool ok = quantize_double(x[j], qx[j]) & quantize_double(y[j], qy[j]);
      const uint32_t dx = (uint32_t)qx[j] - (uint32_t)ix.gx0, dy = (uint32_t)qy[j] - (uint32_t)ix.gy0;
      const uint32_t cx = dx >> ix.s0, cy = dy >> ix.s0;
      const bool in = ok & (cx < ix.nx) & (cy < ix.ny) & (qx[j] >= ix.gx0) & (qy[j] >= ix.gy0);
      d[j] = in ? ld_index_u32(ix.table + (size_t)cy * ix.nx + cx, pol) : 0u;
      idx[j] = (uint32_t)i0 + j;
      sh[j] = ix.s0 - NODE_K;
    }
    if (!COMPACT) {  // the first trie level at once (its entries stay in L2): only
                     // points that need a second level go to the ring
      uint4 e[4];
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if ((d[j] >> 30) == TAG_CHILD) e[j] = ld_entry(ix.nodes, d[j] & PAYLOAD_MASK, pol);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if ((d[j] >> 30) == TAG_CHILD) {
          const uint32_t dx = (uint32_t)qx[j] - (uint32_t)ix.gx0, dy = (uint32_t)qy[j] - (uint32_t)ix.gy0;
          const uint32_t m = (1u << NODE_K) - 1u;
          d[j] = entry_step(e[j], (((dy >> sh[j]) & m) << NODE_K) | ((dx >> sh[j]) & m));
          sh[j] = sh[j] > NODE_K ? sh[j] - NODE_K : 0;
        }
      }
    }
    uint32_t leaf = 0, split = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t tag = d[j] >> 30;
      id[j] = tag == TAG_INTERIOR ? (int32_t)(d[j] & PAYLOAD_MASK) : -1;
      if (tag == TAG_LEAF && ix.approx_id) id[j] = ix.approx_id[d[j] & PAYLOAD_MASK];  // approximate mode
      else leaf |= (tag == TAG_LEAF ? 1u : 0u) << j;
      split |= (tag == TAG_CHILD ? 1u : 0u) << j;
    }
    if (VEC && i0 + 3 < n) {
      reinterpret_cast<int4*>(out)[g] = make_int4(id[0], id[1], id[2], id[3]);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (i0 + j < n) out[i0 + j] = id[j];
    }
    if (__any_sync(full, leaf != 0u))
      res.put(leaf, qx, qy, d, [&](int j) { return idx[j]; }, queue, qcount, hist, 0u);
    if (__any_sync(full, split != 0u)) tr.push(split, qx, qy, idx, d, sh);
#pragma unroll 1
    while (tr.count >= 128u) tr.step<COMPACT>(128u, ix, pol, out, 0u, res, queue, qcount, hist, 0u);
  }
#pragma unroll 1
  while (tr.count > 0u)
    tr.step<COMPACT>(tr.count < 128u ? tr.count : 128u, ix, pol, out, 0u, res, queue, qcount, hist, 0u);
  res.finish(queue, qcount + 2);
}

// ------------------------------------------------------------------- K2
// Counting sort by superbin: off = exclusive scan of hist (in points).
__global__ void k_scatter(const Residual* __restrict__ queue, const uint32_t* __restrict__ qcount,
                          const uint64_t* __restrict__ off, uint32_t* __restrict__ cursor,
                          Residual* __restrict__ binned) {
  scatter_by_superbin(queue, *qcount, off, cursor, binned, blockIdx.x * blockDim.x + threadIdx.x,
                      gridDim.x * blockDim.x);
}

// ------------------------------------------------------------------- K3
struct PlainStore {
  int32_t* out;
  __device__ __forceinline__ void operator()(const Residual& r, int32_t id) const { out[r.z] = id; }
};

template <int STAGES>
__global__ void __launch_bounds__(K3_THREADS) k_cross(IndexView ix, const Residual* __restrict__ binned,
                                                      const uint32_t* __restrict__ qcount, uint32_t ppc,
                                                      uint32_t* __restrict__ item_ctr,
                                                      int32_t* __restrict__ out,
                                                      uint32_t* __restrict__ status,
                                                      uint32_t stage_bytes) {
  extern __shared__ __align__(128) uint4 stage_mem[];
  __shared__ __align__(8) uint64_t bar[STAGES];
  __shared__ uint32_t s_item[STAGES];
  __shared__ uint32_t s_staged[STAGES];
  __shared__ uint32_t s_region[STAGES];
  __shared__ uint32_t s_abort;
  const uint32_t n_res = *qcount;
  const uint32_t n_items = (n_res + ppc - 1) / ppc;
  const uint32_t stage16 = stage_bytes >> 4;
  if (threadIdx.x == 0) {
    for (int i = 0; i < STAGES; ++i) mbar_init(&bar[i], 1);
    fence_barrier_init();
    s_abort = 0;
  }
  __syncthreads();
  uint32_t phase[STAGES];
  bool pending[STAGES];  // thread 0: a copy into this stage is in flight
#pragma unroll
  for (int i = 0; i < STAGES; ++i) {
    phase[i] = 0;
    pending[i] = false;
  }

  // thread 0: claim the next chunk into stage st and start its copy when the
  // records of the chunk's superbins (one contiguous range) fit the stage
  auto claim = [&](int st) {
    const uint32_t w = atomicAdd(item_ctr, 1u);
    s_item[st] = w;
    s_staged[st] = 0;
    if (w < n_items) {
      const uint32_t first = w * ppc;
      const uint32_t last = min(first + ppc, n_res) - 1;
      // binned points are sorted by superbin (not by slot within one): stage
      // whole superbins, from the first point's to the last point's
      const uint32_t da = ix.slot_off[(binned[first].w >> SB_LOG2) << SB_LOG2];
      const uint32_t db = ix.slot_off[((binned[last].w >> SB_LOG2) + 1) << SB_LOG2];
      const uint32_t len16 = db - da;
      if (len16 <= stage16) {
        fence_proxy_async();
        bulk_load(stage_mem + (size_t)st * stage16, ix.blobs + da, len16 * 16u, &bar[st]);
        s_staged[st] = 1;
        s_region[st] = da;
        pending[st] = true;
      }
    }
  };

  if (threadIdx.x == 0) claim(0);
  __syncthreads();
  int cur = 0;
  while (true) {
    const uint32_t w = s_item[cur];
    if (w >= n_items || s_abort) break;
    if (STAGES == 2 && threadIdx.x == 0) claim(cur ^ 1);
    const uint32_t first = w * ppc;
    const uint32_t count = min(ppc, n_res - first);
    const uint4* staged = nullptr;
    if (s_staged[cur]) {
      if (mbar_wait(&bar[cur], phase[cur])) {
        phase[cur] ^= 1u;
        pending[cur] = false;
      } else {
        atomicOr(status, 1u);
        s_abort = 1;
      }
      staged = stage_mem + (size_t)cur * stage16;
    }
    if (!s_abort) test_chunk(ix, binned, first, count, staged, s_region[cur], PlainStore{out});
    __syncthreads();
    if (STAGES == 2) {
      cur ^= 1;
    } else {
      if (threadIdx.x == 0) claim(0);
      __syncthreads();
    }
  }
  // never leave with a copy in flight: wait (bounded) for any issued copy
  // that no iteration consumed
  if (threadIdx.x == 0) {
    for (int st = 0; st < STAGES; ++st)
      if (pending[st]) mbar_wait(&bar[st], phase[st]);
  }
}

// K3 without shared-memory staging: records are read through L1/L2. Best
// when a chunk's points are spread over more superbins than fit a stage.
__global__ void __launch_bounds__(K3_THREADS) k_cross_direct(IndexView ix,
                                                             const Residual* __restrict__ binned,
                                                             const uint32_t* __restrict__ qcount,
                                                             uint32_t ppc, uint32_t* __restrict__ item_ctr,
                                                             int32_t* __restrict__ out) {
  __shared__ uint32_t s_w;
  const uint32_t n_res = *qcount;
  const uint32_t n_items = (n_res + ppc - 1) / ppc;
  while (true) {
    if (threadIdx.x == 0) s_w = atomicAdd(item_ctr, 1u);
    __syncthreads();
    const uint32_t w = s_w;
    __syncthreads();
    if (w >= n_items) break;
    const uint32_t first = w * ppc;
    test_chunk(ix, binned, first, min(ppc, n_res - first), nullptr, 0u, PlainStore{out});
  }
}

// Failure path of the bounded waits: one CTA waits on an mbarrier that
// nothing completes; the wait gives up after limit_ns, the kernel records
// the outcome (1 = ran out, 2 = completed) and returns.
__global__ void k_bounded_wait_probe(uint32_t* __restrict__ outcome, unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) *outcome = mbar_wait(&bar, 0u, limit_ns) ? 2u : 1u;
}

// ------------------------------------------------------------------- host
static void init_pool_once() {
  static std::once_flag f[64];
  int dev = 0;
  cudaGetDevice(&dev);
  std::call_once(f[dev & 63], [dev] {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
  });
}

static int k3_smem_config(int stages, uint32_t& stage_bytes) {
  stage_bytes = stages == 2 ? 48u * 1024u : 96u * 1024u;
  return (int)(stage_bytes * stages);
}

static pip_status k3_launch(const IndexView& ix, int stages, const Residual* binned,
                            const uint32_t* qcount, uint32_t ppc, uint32_t* item_ctr,
                            int32_t* out, uint32_t* status, cudaStream_t s) {
  if (stages < 0) {
    static std::atomic<int> occ_cache{0};  // same on every device of one architecture
    int occ = occ_cache.load(std::memory_order_relaxed);
    if (!occ) {
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cross_direct, K3_THREADS, 0);
      occ = std::max(1, occ);
      occ_cache.store(occ, std::memory_order_relaxed);
    }
    const unsigned grid = (unsigned)(num_sms() * occ);
    k_cross_direct<<<grid, K3_THREADS, 0, s>>>(ix, binned, qcount, ppc, item_ctr, out);
    PIP_CUDA(cudaGetLastError());
    return PIP_OK;
  }
  uint32_t stage_bytes = 0;
  const int smem = k3_smem_config(stages, stage_bytes);
  static std::atomic<uint32_t> attr_set[64];  // per device: bit `stages` once the attribute is set
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!(attr_set[dev].load(std::memory_order_acquire) & (1u << stages))) {
    if (stages == 2)
      PIP_CUDA(cudaFuncSetAttribute(k_cross<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    else
      PIP_CUDA(cudaFuncSetAttribute(k_cross<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    attr_set[dev].fetch_or(1u << stages, std::memory_order_acq_rel);
  }
  const int ctas_per_sm = std::max(1, (int)((200 * 1024) / (smem + 2048)));
  const unsigned grid = (unsigned)(num_sms() * std::min(ctas_per_sm, 4));
  if (stages == 2)
    k_cross<2><<<grid, K3_THREADS, smem, s>>>(ix, binned, qcount, ppc, item_ctr, out, status,
                                              stage_bytes);
  else
    k_cross<1><<<grid, K3_THREADS, smem, s>>>(ix, binned, qcount, ppc, item_ctr, out, status,
                                              stage_bytes);
  PIP_CUDA(cudaGetLastError());
  return PIP_OK;
}

pip_status k3_launch_public(const IndexView& ix, int stages, const Residual* binned,
                            const uint32_t* qcount, uint32_t ppc, uint32_t* item_ctr, int32_t* out,
                            uint32_t* status, cudaStream_t s) {
  return k3_launch(ix, stages, binned, qcount, ppc, item_ctr, out, status, s);
}

// K1 grid: one persistent wave of the deferred-queue kernel.
static unsigned k1_grid(int64_t n) {
  static std::atomic<int> occ_cache{0};
  int occ = occ_cache.load(std::memory_order_relaxed);
  if (!occ) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_classify_dq<true, true>, DQ_THREADS, 0) != cudaSuccess)
      occ = 1;
    occ = std::max(1, occ);
    occ_cache.store(occ, std::memory_order_relaxed);
  }
  const int64_t groups = (n + 3) / 4;
  return (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((groups + DQ_THREADS - 1) / DQ_THREADS, (int64_t)num_sms() * occ));
}

// Queue entries K1 may use for n points: n plus two reserved chunks per warp.
int64_t k1_queue_entries(int64_t n) {
  return n + 2 * (int64_t)QCHUNK * (DQ_THREADS / 32) * k1_grid(n);
}

// K1 over n points (deferred-queue form): 16-byte loads and stores when lon,
// lat and out are 16-byte aligned, else scalar ones. qcount[0] counts queue
// entries including holes, qcount[2] the residual points; the queue holds
// k1_queue_entries(n) entries.
cudaError_t k1_launch(const IndexView& ix, const double* lon, const double* lat, int64_t n,
                      int32_t* out, Residual* queue, uint32_t* qcount, uint32_t* hist, cudaStream_t s) {
  const bool vec = ((uintptr_t)lon % 16 == 0) && ((uintptr_t)lat % 16 == 0) && ((uintptr_t)out % 16 == 0);
  const unsigned g1 = k1_grid(n);
  if (vec && ix.compact)
    k_classify_dq<true, true><<<g1, DQ_THREADS, 0, s>>>(ix, lon, lat, n, out, queue, qcount, hist);
  else if (vec)
    k_classify_dq<true, false><<<g1, DQ_THREADS, 0, s>>>(ix, lon, lat, n, out, queue, qcount, hist);
  else if (ix.compact)
    k_classify_dq<false, true><<<g1, DQ_THREADS, 0, s>>>(ix, lon, lat, n, out, queue, qcount, hist);
  else
    k_classify_dq<false, false><<<g1, DQ_THREADS, 0, s>>>(ix, lon, lat, n, out, queue, qcount, hist);
  return cudaGetLastError();
}

// K1 in the lockstep form: no reserved chunks, so the queue needs only n
// entries and qcount[0] is the residual count.
cudaError_t k1_launch_lockstep(const IndexView& ix, const double* lon, const double* lat, int64_t n,
                               int32_t* out, Residual* queue, uint32_t* qcount, uint32_t* hist,
                               cudaStream_t s) {
  static std::atomic<int> occ_cache{0};
  int occ = occ_cache.load(std::memory_order_relaxed);
  if (!occ) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_classify_points<true>, K1_THREADS, 0);
    if (e != cudaSuccess) return e;
    occ = std::max(1, occ);
    occ_cache.store(occ, std::memory_order_relaxed);
  }
  const bool vec = ((uintptr_t)lon % 16 == 0) && ((uintptr_t)lat % 16 == 0) && ((uintptr_t)out % 16 == 0);
  const int64_t groups = (n + 3) / 4;
  const unsigned g1 = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((groups + K1_THREADS - 1) / K1_THREADS, (int64_t)num_sms() * occ));
  if (vec)
    k_classify_points<true><<<g1, K1_THREADS, 0, s>>>(ix, lon, lat, n, out, queue, qcount, hist);
  else
    k_classify_points<false><<<g1, K1_THREADS, 0, s>>>(ix, lon, lat, n, out, queue, qcount, hist);
  return cudaGetLastError();
}

// Binning the residual by superbin before the unstaged crossing test did not
// pay at any density measured (state workload, 1e8 points, split ratios 128
// / 48 / 16 / 8, i.e. 0.44 / 2.8 / 24 / 75 residual points per superbin:
// the test over the queue in arrival order took 0.141 / 0.295 / 0.733 /
// 1.162 ms against 0.206 / 0.361 / 0.770 / 1.251 ms for binning + test).
// Each point reads its own leaf record either way; the binning's scan and
// scatter cost more than the locality they buy. So the plain path bins only
// when asked to or when the staged crossing kernel needs it.


// Binning by superbin: when asked for, or for the staged crossing kernel,
// which needs each chunk's records contiguous.
static bool bins_residual(const pip_set_s* S) { return S->opts.stage_depth > 0 || S->opts.bin_residual > 0; }

pip_status proj_scratch_alloc(pip_set_s* S, ProjScratch& w, int64_t n, cudaStream_t s) {
  Alloc* al = &S->alloc;
  const int64_t n_sb = std::max<int64_t>(1, S->view.n_sb);
  const bool bin = bins_residual(S);
  w.cap = 0;
  w.binned.release();
  if (!w.queue.alloc(al, k1_queue_entries(n), s) || (bin && !w.binned.alloc(al, n, s)) ||
      !w.hist.alloc(al, 2 * n_sb, s) || !w.off.alloc(al, n_sb, s) || !w.ctr.alloc(al, 4, s))
    return fail(PIP_ENOMEM, "pip_project: scratch allocation failed");
  w.cap = n;
  w.n_sb = n_sb;
  w.bin = bin;
  return PIP_OK;
}

bool proj_scratch_fits(const pip_set_s* S, const ProjScratch& w, int64_t n) {
  return w.cap >= n && w.n_sb == std::max<int64_t>(1, S->view.n_sb) && (w.bin || !bins_residual(S));
}

pip_status project_device(pip_set_s* S, const double* lon, const double* lat, int64_t n, int32_t* out,
                          cudaStream_t s, pip_project_stats* stats) {
  return project_device_with(S, lon, lat, n, out, s, stats, nullptr);
}

pip_status project_device_with(pip_set_s* S, const double* lon, const double* lat, int64_t n, int32_t* out,
                               cudaStream_t s, pip_project_stats* stats, ProjScratch* pre) {
  if (n <= 0) return PIP_OK;
  if (n >= (1ll << 32) - 1 || k1_queue_entries(n) >= (1ll << 32))
    return fail(PIP_EINVAL, "pip_project: too many points for one device call (queue indices are 32-bit)");
  init_pool_once();
  Alloc* al = &S->alloc;
  const IndexView& ix = S->view;
  const int64_t n_sb = std::max<int64_t>(1, ix.n_sb);
  const uint32_t ppc = (uint32_t)std::max(1, S->opts.pts_per_cta);
  const bool bin = bins_residual(S);
  ProjScratch own;
  if (!pre || !proj_scratch_fits(S, *pre, n)) {
    pip_status a = proj_scratch_alloc(S, own, n, s);
    if (a != PIP_OK) return a;
    pre = &own;
  }
  ProjScratch& w = *pre;
  uint32_t* hist = w.hist.p;
  uint32_t* cursor = w.hist.p + n_sb;
  int prof = -1;
  if (S->prof_cap > 0 && S->prof_n < S->prof_cap) {
    prof = S->prof_n++;
    PIP_CUDA(cudaEventRecord(S->prof_ev[4 * prof + 0], s));
  }
  PIP_CUDA(cudaMemsetAsync(w.hist.p, 0, 2 * n_sb * sizeof(uint32_t), s));
  PIP_CUDA(cudaMemsetAsync(w.ctr.p, 0, 4 * sizeof(uint32_t), s));
  PIP_CUDA(k1_launch(ix, lon, lat, n, out, w.queue.p, w.ctr.p, hist, s));
  if (prof >= 0) PIP_CUDA(cudaEventRecord(S->prof_ev[4 * prof + 1], s));
  pip_status st = PIP_OK;
  if (bin) {
    st = scan_u32_to_u64(*al, hist, w.off.p, n_sb, nullptr, s);
    if (st != PIP_OK) return st;
    k_scatter<<<(unsigned)(num_sms() * 8), 256, 0, s>>>(w.queue.p, w.ctr.p, w.off.p, cursor, w.binned.p);
    PIP_CUDA(cudaGetLastError());
  }
  if (prof >= 0) PIP_CUDA(cudaEventRecord(S->prof_ev[4 * prof + 2], s));
  // K3 over the binned points, or over the whole queue in arrival order
  // (its unused reserved entries are skipped)
  st = bin ? k3_launch(ix, S->opts.stage_depth, w.binned.p, w.ctr.p + 2, ppc, w.ctr.p + 1, out, S->status.p, s)
           : k3_launch(ix, -1, w.queue.p, w.ctr.p + 0, ppc, w.ctr.p + 1, out, S->status.p, s);
  if (st != PIP_OK) return st;
  if (prof >= 0) PIP_CUDA(cudaEventRecord(S->prof_ev[4 * prof + 3], s));
  count_launches(bin ? 3 : 2);  // K1, scatter, K3 (the scan counts its own)
  if (stats) {
    uint32_t c[3];
    PIP_CUDA(cudaMemcpyAsync(c, w.ctr.p, sizeof(c), cudaMemcpyDeviceToHost, s));
    PIP_CUDA(cudaStreamSynchronize(s));
    stats->n = n;
    stats->residual = c[2];
    stats->items = (c[2] + ppc - 1) / ppc;
  }
  return PIP_OK;
}

// The same K1 -> scan -> scatter -> K3 sequence with every scratch buffer
// supplied by the caller (used by the entry point that allocates nothing).
// queue/binned hold n entries, hist 2 * n_sb, off n_sb, scan_tmp scan_len,
// ctr 4 words.
pip_status project_device_scratch(pip_set_s* S, const double* lon, const double* lat, int64_t n,
                                  int32_t* out, cudaStream_t s, Residual* queue, Residual* binned,
                                  uint32_t* hist2, uint64_t* off, uint64_t* scan_tmp, int64_t scan_len,
                                  uint32_t* ctr) {
  const IndexView& ix = S->view;
  const int64_t n_sb = std::max<int64_t>(1, ix.n_sb);
  const uint32_t ppc = (uint32_t)std::max(1, S->opts.pts_per_cta);
  PIP_CUDA(cudaMemsetAsync(hist2, 0, 2 * n_sb * sizeof(uint32_t), s));
  PIP_CUDA(cudaMemsetAsync(ctr, 0, 4 * sizeof(uint32_t), s));
  PIP_CUDA(k1_launch_lockstep(ix, lon, lat, n, out, queue, ctr, hist2, s));
  pip_status st = scan_u32_to_u64_scratch(hist2, off, n_sb, scan_tmp, scan_len, s);
  if (st != PIP_OK) return st;
  k_scatter<<<(unsigned)(num_sms() * 8), 256, 0, s>>>(queue, ctr, off, hist2 + n_sb, binned);
  PIP_CUDA(cudaGetLastError());
  st = k3_launch(ix, S->opts.stage_depth, binned, ctr, ppc, ctr + 1, out, S->status.p, s);
  if (st != PIP_OK) return st;
  count_launches(3);
  return PIP_OK;
}

// Host-memory inputs/outputs: see host.cu.
pip_status project_host(pip_set_s* S, const double* lon, const double* lat, int64_t n, int32_t* out,
                        cudaStream_t s, pip_project_stats* stats);

}  // namespace pip

using namespace pip;

extern "C" pip_status pip_project_ex(pip_set set, const double* lon, const double* lat, int64_t n,
                                     int32_t* out, void* stream, pip_project_stats* stats) {
  if (!set) return fail(PIP_EINVAL, "pip_project: NULL set");
  if (n < 0) return fail(PIP_EINVAL, "pip_project: n < 0");
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (n == 0) return PIP_OK;
  if (!lon || !lat || !out) return fail(PIP_EINVAL, "pip_project: NULL pointer with n > 0");
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != set->device) PIP_CUDA(cudaSetDevice(set->device));
  cudaStream_t s = (cudaStream_t)stream;
  const bool dev = is_device_ptr(lon) && is_device_ptr(lat) && is_device_ptr(out);
  pip_status st = dev ? project_device(set, lon, lat, n, out, s, stats)
                      : project_host(set, lon, lat, n, out, s, stats);
  if (cur != set->device) cudaSetDevice(cur);
  return st;
}

extern "C" pip_status pip_project(pip_set set, const double* lon, const double* lat, int64_t n,
                                  int32_t* out, void* stream) {
  return pip_project_ex(set, lon, lat, n, out, stream, nullptr);
}

extern "C" pip_status pip_selftest_bounded_wait(int64_t limit_ns, void* stream) {
  if (limit_ns <= 0 || limit_ns > 10ll * 1000 * 1000 * 1000)
    return fail(PIP_EINVAL, "pip_selftest_bounded_wait: 0 < limit_ns <= 1e10");
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t* d = nullptr;
  PIP_CUDA(cudaMallocAsync((void**)&d, sizeof(uint32_t), s));
  PIP_CUDA(cudaMemsetAsync(d, 0, sizeof(uint32_t), s));
  k_bounded_wait_probe<<<1, 32, 0, s>>>(d, (unsigned long long)limit_ns);
  cudaError_t e = cudaGetLastError();
  uint32_t h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFreeAsync(d, s);
  if (e != cudaSuccess) return cuda_fail(e, "pip_selftest_bounded_wait");
  count_launches(1);
  if (h == 1u) return fail(PIP_ETIMEOUT, "pip_selftest_bounded_wait: the wait ran out (expected)");
  return h == 2u ? PIP_OK : fail(PIP_ECUDA, "pip_selftest_bounded_wait: no outcome recorded");
}
