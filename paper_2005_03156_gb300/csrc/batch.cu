// Batched form: many uneven queries over many resident sets in one
// persistent, work-stealing, cooperative launch captured in a CUDA graph.
//
// Phases of the one kernel, separated by grid-wide barriers (bounded waits:
// a barrier that does not complete within 2 s sets the status word and the
// kernel runs to its end without further waiting):
//   0 classify   CTAs take 4096-point tiles from an atomic counter; each
//                point is quantized, looked up in its query's set trie and
//                either answered (EMPTY / INTERIOR) or appended to the
//                residual queue with a global slot (set base + leaf slot).
//   1 scan       exclusive scan of the per-superbin counts of all sets.
//   2 scatter    counting sort of the residual by global superbin.
//   3 cross      CTAs take chunks of pts_per_cta binned points; a chunk whose
//                points all belong to one set and whose records fit a stage
//                is staged with one cp.async.bulk copy; then the exact
//                crossing test runs per point and the id is written to its
//                query's output.
// Phases 1 and 2 run only with staging, which needs a chunk's records
// contiguous; unstaged (the default), phase 3 reads the residual queue in
// arrival order, as the plain path does: binning cost more than it saved.
// The results equal separate plain projections bit for bit: same index,
// same arithmetic, same rule.
#include <algorithm>
#include <cstring>
#include <memory>
#include <vector>

#include "kernels.cuh"

namespace pip {

constexpr int B_THREADS = 256;
constexpr int TILE = 4096;
static_assert(TILE == 4096, "tile offsets use 12 bits");
constexpr int MAX_SETS = 64;

struct DevSet {
  IndexView view;
  uint32_t sb_base;  // first global superbin of the set
  uint32_t pad[3];
};

struct DevQuery {
  const double* lon;
  const double* lat;
  int32_t* out;
  uint32_t set;
  uint32_t n;
};

// Layout of the per-run table block (host pinned -> device in one copy).
struct RunHeader {
  uint32_t n_q, n_sets, n_tiles, total_points;
  uint32_t n_sb_total, ppc, stage16;
  uint32_t sub_log2;  // phase-0 work item: 2^sub_log2 points of a tile (10..12)
};

struct PlanBufs {
  RunHeader* hdr;         // header
  DevSet* sets;           // [MAX_SETS]
  DevQuery* queries;      // [max_queries]
  uint32_t* qoff;         // [max_queries + 1] point offsets
  uint4* tiles;           // [max_tiles] (query, start, count, global offset)
  Residual* queue;        // [max_points]
  Residual* binned;       // [max_points]
  uint32_t* hist;         // [sb_cap] counts
  uint32_t* cursor;       // [sb_cap]
  uint64_t* off;          // [sb_cap]
  uint64_t* partial;      // [grid + 1]
  uint32_t* ctr;          // [0] queue slots [1] tile ctr [2] chunk ctr [3] barrier count [4] barrier gen [5] residual count
  uint32_t* status;       // bounded-wait status word
};

__device__ __forceinline__ void grid_barrier(const PlanBufs& B, uint32_t nblocks) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile uint32_t* vgen = B.ctr + 4;
    const uint32_t g = *vgen;
    __threadfence();
    if (atomicAdd(B.ctr + 3, 1u) == nblocks - 1) {
      B.ctr[3] = 0;
      __threadfence();
      atomicAdd(B.ctr + 4, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (*vgen == g) {
        if (global_ns() - t0 > WAIT_NS) {
          atomicOr(B.status, 2u);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// Residual entries of the batched form carry z = tile << 12 | offset in the
// tile (tiles never cross queries), so the output slot is two cached loads.
constexpr int TILE_LOG2 = 12;

struct BatchStore {
  const uint4* tiles;
  const DevQuery* queries;
  __device__ __forceinline__ void operator()(const Residual& r, int32_t id) const {
    const uint4 tl = tiles[r.z >> TILE_LOG2];
    queries[tl.x].out[tl.y + (r.z & (TILE - 1))] = id;
  }
};

// Set of a global slot (sets in increasing sb_base order).
__device__ __forceinline__ uint32_t set_of_slot(const DevSet* sets, uint32_t n_sets, uint32_t gslot) {
  const uint32_t gsb = gslot >> SB_LOG2;
  uint32_t s = 0;
  while (s + 1 < n_sets && sets[s + 1].sb_base <= gsb) ++s;
  return s;
}

// Crossing test of one chunk whose points may span several sets.
__device__ __forceinline__ void batch_test_chunk(const DevSet* sets, uint32_t n_sets,
                                                 const Residual* __restrict__ binned, uint32_t first,
                                                 uint32_t count, const uint4* staged, uint32_t region16,
                                                 BatchStore store) {
  const int lane = threadIdx.x & 31;
  for (uint32_t base = threadIdx.x & ~31u; base < count; base += blockDim.x) {
    const uint32_t t = base + lane;
    bool active = t < count;
    Residual r = make_uint4(0, 0, 0, 0);
    const uint4* bp = nullptr;
    if (active) r = binned[first + t];
    active &= r.w != RES_HOLE;  // the queue in arrival order keeps its unused entries
    if (active) {
      const DevSet& S = sets[set_of_slot(sets, n_sets, r.w)];
      const uint32_t off = S.view.slot_off[r.w - (S.sb_base << SB_LOG2)];
      bp = staged ? staged + (off - region16) : S.view.blobs + off;
    }
    LeafRec b{nullptr, nullptr};
    if (active) b = leaf_rec(bp);
    const bool is_long = active && leaf_edges(b) > (uint32_t)LONG_LIST;
    int32_t id = -1;
    if (active && !is_long) id = test_point(b, (int32_t)r.x, (int32_t)r.y);
    uint32_t lm = __ballot_sync(0xffffffffu, is_long);
    while (lm) {
      const int j = __ffs(lm) - 1;
      lm &= lm - 1;
      const int32_t px = (int32_t)__shfl_sync(0xffffffffu, r.x, j);
      const int32_t py = (int32_t)__shfl_sync(0xffffffffu, r.y, j);
      const unsigned long long pj = __shfl_sync(0xffffffffu, (unsigned long long)(uintptr_t)bp, j);
      const int32_t v = test_point_warp(leaf_rec((const uint4*)(uintptr_t)pj), px, py);
      if (lane == j) id = v;
    }
    if (active) store(r, id);
  }
}

// COMPACT = false when no set of the run holds compact leaves (a leaner
// trie step: the kernel is sensitive to its code size and registers).
template <int STAGED, bool COMPACT>
__global__ void __launch_bounds__(B_THREADS, 3) k_batch(PlanBufs B) {
  extern __shared__ __align__(128) uint4 stage_mem[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t s_w, s_staged, s_region;  // phase 3
  __shared__ DevSet s_sets[MAX_SETS];
  __shared__ uint64_t s_scan[B_THREADS / 32];
  const uint32_t nblocks = gridDim.x;
  const RunHeader H = *B.hdr;
  for (uint32_t i = threadIdx.x; i < H.n_sets * (sizeof(DevSet) / 4); i += blockDim.x)
    reinterpret_cast<uint32_t*>(s_sets)[i] = reinterpret_cast<const uint32_t*>(B.sets)[i];
  if (STAGED && threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  __syncthreads();

  // ---- phase 0: classify tiles. Each warp takes work items of 2^sub_log2
  // points of one tile: a step reads the top-grid descriptors of 128 points,
  // points in split cells wait in the warp's trie ring (walked one level for
  // 128 entries at a time) and the ring is drained at the end of the item, so
  // its entries share the tile's set and output array. Large batches use
  // whole tiles (fewer drains); small ones 1024-point items (whole tiles per
  // warp made a small batch's latency 4x that of a CTA-wide tile).
  {
    __shared__ uint4 ring[B_THREADS / 32][TRING];
    __shared__ uint8_t ring_sh[B_THREADS / 32][TRING];
    const uint32_t full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint64_t pol = policy_evict_last();
    TrieRing tr;
    tr.rq = ring[threadIdx.x >> 5];
    tr.rs = ring_sh[threadIdx.x >> 5];
    ChunkWriter res;  // this warp's residual entries
    while (true) {
      uint32_t item = 0;
      if (lane == 0) item = atomicAdd(B.ctr + 1, 1u);
      item = __shfl_sync(full, item, 0);
      const uint32_t per_tile_log2 = TILE_LOG2 - H.sub_log2;
      if (item >= (H.n_tiles << per_tile_log2)) break;
      const uint32_t w = item >> per_tile_log2;
      const uint4 tl = B.tiles[w];  // (query, start, count, global offset)
      const uint32_t g_begin = (item & ((1u << per_tile_log2) - 1u)) << H.sub_log2;
      if (g_begin >= tl.z) continue;
      const uint32_t g_end = min(tl.z, g_begin + (1u << H.sub_log2));
      const DevQuery q = B.queries[tl.x];
      const DevSet& S = s_sets[q.set];
      const IndexView& ix = S.view;
      const uint32_t slot_add = S.sb_base << SB_LOG2;
      const uint32_t code0 = w << TILE_LOG2;
      const double* lon = q.lon + tl.y;
      const double* lat = q.lat + tl.y;
      int32_t* out = q.out + tl.y;
      // 16-byte loads / stores when the tile's three arrays are aligned
      const bool vec = (((uintptr_t)lon | (uintptr_t)lat | (uintptr_t)out) & 15u) == 0;
      auto load = [&](uint32_t j0, double(&x)[4], double(&y)[4]) {
        if (vec && j0 + 3 < tl.z) {
          const double2 a0 = __ldcs(reinterpret_cast<const double2*>(lon + j0));
          const double2 a1 = __ldcs(reinterpret_cast<const double2*>(lon + j0) + 1);
          const double2 b0 = __ldcs(reinterpret_cast<const double2*>(lat + j0));
          const double2 b1 = __ldcs(reinterpret_cast<const double2*>(lat + j0) + 1);
          x[0] = a0.x; x[1] = a0.y; x[2] = a1.x; x[3] = a1.y;
          y[0] = b0.x; y[1] = b0.y; y[2] = b1.x; y[3] = b1.y;
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const bool have = j0 + j < tl.z;
            x[j] = have ? __ldcs(lon + j0 + j) : __longlong_as_double(0x7FF8000000000000ll);
            y[j] = have ? __ldcs(lat + j0 + j) : 0.0;
          }
        }
      };
      double nx[4], ny[4];
      load(g_begin + 4 * lane, nx, ny);
#pragma unroll 1
      for (uint32_t g0 = g_begin; g0 < g_end; g0 += 128u) {
        const uint32_t j0 = g0 + 4 * lane;  // offset within the tile
        double x[4], y[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          x[j] = nx[j];
          y[j] = ny[j];
        }
        if (g0 + 128u < g_end) load(j0 + 128u, nx, ny);
        int32_t qx[4], qy[4], id[4];
        uint32_t d[4], z[4];
        int sh[4];
        const uint32_t s0 = (uint32_t)ix.s0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          qx[j] = qy[j] = 0;
          const bool ok = quantize_double(x[j], qx[j]) & quantize_double(y[j], qy[j]);
          const uint32_t dx = (uint32_t)qx[j] - (uint32_t)ix.gx0, dy = (uint32_t)qy[j] - (uint32_t)ix.gy0;
          const uint32_t cx = dx >> s0, cy = dy >> s0;
          const bool in = ok & (cx < ix.nx) & (cy < ix.ny) & (qx[j] >= ix.gx0) & (qy[j] >= ix.gy0);
          d[j] = in ? ld_index_u32(ix.table + (size_t)cy * ix.nx + cx, pol) : 0u;
          z[j] = j0 + j;
          sh[j] = (int)s0 - NODE_K;
        }
        if (!COMPACT) {  // the first trie level at once, as the plain classify kernel
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
        if (vec && j0 + 3 < tl.z) {
          *reinterpret_cast<int4*>(out + j0) = make_int4(id[0], id[1], id[2], id[3]);
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (j0 + j < tl.z) out[j0 + j] = id[j];
        }
        if (__any_sync(full, leaf != 0u))
          res.put(leaf, qx, qy, d, [&](int j) { return code0 + z[j]; }, B.queue, B.ctr + 0, B.hist, slot_add);
        if (__any_sync(full, split != 0u)) tr.push(split, qx, qy, z, d, sh);
#pragma unroll 1
        while (tr.count >= 128u)
          tr.step<COMPACT>(128u, ix, pol, out, code0, res, B.queue, B.ctr + 0, B.hist, slot_add);
      }
#pragma unroll 1
      while (tr.count > 0u)
        tr.step<COMPACT>(tr.count < 128u ? tr.count : 128u, ix, pol, out, code0, res, B.queue, B.ctr + 0, B.hist,
                         slot_add);
    }
    res.finish(B.queue, B.ctr + 5);
  }
  grid_barrier(B, nblocks);

  const uint32_t n_slots = *(volatile uint32_t*)(B.ctr + 0);  // queue entries, holes included
  const uint32_t n_res = *(volatile uint32_t*)(B.ctr + 5);
  if (STAGED) {  // binning: only the staged crossing phase needs chunks sorted by superbin
    // ---- phase 1: exclusive scan of hist[0, n_sb_total) over all CTAs
    const uint32_t nsb = H.n_sb_total;
    const uint32_t seg = (nsb + nblocks - 1) / nblocks;
    const uint32_t a = min(nsb, blockIdx.x * seg), e = min(nsb, a + seg);
    {
      uint64_t part = 0;
      for (uint32_t i = a + threadIdx.x; i < e; i += blockDim.x) part += B.hist[i];
      for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      if ((threadIdx.x & 31) == 0) s_scan[threadIdx.x >> 5] = part;
      __syncthreads();
      if (threadIdx.x == 0) {
        uint64_t t = 0;
        for (int i = 0; i < B_THREADS / 32; ++i) t += s_scan[i];
        B.partial[blockIdx.x] = t;
      }
    }
    grid_barrier(B, nblocks);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      uint64_t run = 0;
      for (uint32_t c = 0; c < nblocks; ++c) {
        const uint64_t v = B.partial[c];
        B.partial[c] = run;
        run += v;
      }
    }
    grid_barrier(B, nblocks);
    {  // block-wide scan of this CTA's segment, blockDim values per step
      uint64_t run = B.partial[blockIdx.x];
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
      for (uint32_t base = a; base < e; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        const uint64_t v = i < e ? B.hist[i] : 0;
        uint64_t incl = v;
  #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint64_t t = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += t;
        }
        if (lane == 31) s_scan[warp] = incl;
        __syncthreads();
        uint64_t wbase = 0, total = 0;
        for (int k = 0; k < B_THREADS / 32; ++k) {
          if (k < warp) wbase += s_scan[k];
          total += s_scan[k];
        }
        if (i < e) B.off[i] = run + wbase + incl - v;
        run += total;
        __syncthreads();
      }
    }
    grid_barrier(B, nblocks);

    // ---- phase 2: scatter by global superbin (queue slots include holes)
    scatter_by_superbin(B.queue, n_slots, B.off, B.cursor, B.binned, blockIdx.x * blockDim.x + threadIdx.x,
                        nblocks * blockDim.x);
    grid_barrier(B, nblocks);
  }

  // ---- phase 3: crossing tests, chunks of ppc binned points (staged), or
  // of the residual queue in arrival order, its unused entries skipped
  const Residual* __restrict__ cross_in = STAGED ? B.binned : B.queue;
  const uint32_t n_cross = STAGED ? n_res : n_slots;
  const uint32_t ppc = H.ppc;
  const uint32_t n_items = (n_cross + ppc - 1) / ppc;
  const BatchStore store{B.tiles, B.queries};
  uint32_t phase = 0;
  while (true) {
    if (threadIdx.x == 0) {
      const uint32_t w = atomicAdd(B.ctr + 2, 1u);
      s_w = w;
      s_staged = 0;
      if (STAGED && w < n_items) {
        const uint32_t first = w * ppc, last = min(first + ppc, n_res) - 1;
        const uint32_t ga = B.binned[first].w, gb = B.binned[last].w;
        const uint32_t sa = set_of_slot(s_sets, H.n_sets, ga), sb = set_of_slot(s_sets, H.n_sets, gb);
        if (sa == sb) {
          const DevSet& S = s_sets[sa];
          // whole superbins (binned order sorts superbins, not slots)
          const uint32_t da = S.view.slot_off[((ga >> SB_LOG2) - S.sb_base) << SB_LOG2];
          const uint32_t db = S.view.slot_off[((gb >> SB_LOG2) - S.sb_base + 1) << SB_LOG2];
          const uint32_t len16 = db - da;
          if (len16 <= H.stage16) {
            fence_proxy_async();
            bulk_load(stage_mem, S.view.blobs + da, len16 * 16u, &bar);
            s_staged = 1;
            s_region = da;
          }
        }
      }
    }
    __syncthreads();
    const uint32_t w = s_w;
    if (w >= n_items) break;
    const uint4* staged = nullptr;
    if (STAGED && s_staged) {
      if (!mbar_wait(&bar, phase)) atomicOr(B.status, 1u);
      phase ^= 1u;
      staged = stage_mem;
    }
    const uint32_t first = w * ppc;
    batch_test_chunk(s_sets, H.n_sets, cross_in, first, min(ppc, n_cross - first), staged, s_region,
                     store);
    __syncthreads();
  }
}

}  // namespace pip

using namespace pip;

struct pip_plan_s {
  int device = 0;
  int64_t max_points = 0;
  int32_t max_queries = 0;
  int64_t max_tiles = 0;
  int64_t sb_cap = 0;
  int grid = 0;
  int staged = 0;      // 0 unstaged, 1 staged
  bool compact = false;  // the captured kernel handles compact leaves
  bool compact_fixed = false;  // keep `compact` for runs without compact sets
  uint32_t ppc = 256;
  uint32_t stage_bytes = 16 * 1024;  // small: the one kernel's other phases want L1
  Alloc alloc;
  DBuf<uint8_t> tables;  // header | sets | queries | qoff | tiles
  size_t tables_bytes = 0;
  DBuf<Residual> queue, binned;
  DBuf<uint32_t> hist;   // counts | cursors
  DBuf<uint64_t> off, partial;
  DBuf<uint32_t> ctr, status;
  // two pinned table buffers and two graphs: the host fills one while the
  // previous run's graph may still be copying the other
  uint8_t* host_tables[2] = {nullptr, nullptr};
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaEvent_t done[2] = {nullptr, nullptr};
  bool used[2] = {false, false};
  int turn = 0;
  PlanBufs bufs{};
  size_t off_sets = 0, off_q = 0, off_qoff = 0, off_tiles = 0;
  void drop_graphs() {
    for (int i = 0; i < 2; ++i) {
      if (exec[i]) cudaGraphExecDestroy(exec[i]);
      if (graph[i]) cudaGraphDestroy(graph[i]);
      exec[i] = nullptr;
      graph[i] = nullptr;
    }
  }
  ~pip_plan_s() {
    drop_graphs();
    for (int i = 0; i < 2; ++i) {
      if (host_tables[i]) cudaFreeHost(host_tables[i]);
      if (done[i]) cudaEventDestroy(done[i]);
    }
  }
};

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

static pip_status plan_alloc_sb(pip_plan_s* P, int64_t need, cudaStream_t s) {
  if (need <= P->sb_cap) return PIP_OK;
  const int64_t cap = std::max<int64_t>(need, 2 * P->sb_cap);
  if (!P->hist.alloc(&P->alloc, 2 * cap + 2, s) || !P->off.alloc(&P->alloc, cap + 1, s))
    return fail(PIP_ENOMEM, "pip_plan: superbin buffers");
  P->sb_cap = cap;
  P->drop_graphs();  // buffers moved: capture again
  return PIP_OK;
}

static int batch_smem(int staged, uint32_t stage_bytes) { return staged ? (int)stage_bytes : 0; }

// The kernel instantiation for the plan's knobs.
static void (*batch_kernel(int staged, bool compact))(PlanBufs) {
  if (staged) return compact ? k_batch<1, true> : k_batch<1, false>;
  return compact ? k_batch<0, true> : k_batch<0, false>;
}

static pip_status plan_grid(pip_plan_s* P) {
  int occ = 0;
  const int smem = batch_smem(P->staged, P->stage_bytes);
  auto k = batch_kernel(P->staged, P->compact);
  if (P->staged) PIP_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  PIP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, B_THREADS, smem));
  if (occ < 1) return fail(PIP_ECUDA, "pip_plan: batched kernel does not fit an SM");
  P->grid = num_sms() * occ;
  return PIP_OK;
}

// Capture: table copy -> memsets of the counters -> cooperative kernel.
static pip_status plan_capture(pip_plan_s* P, int t, cudaStream_t s) {
  if (P->exec[t]) return PIP_OK;
  cudaStream_t cs;
  PIP_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  pip_status res = PIP_OK;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaMemcpyAsync(P->tables.p, P->host_tables[t], P->tables_bytes, cudaMemcpyHostToDevice, cs);
    cudaMemsetAsync(P->ctr.p, 0, 8 * sizeof(uint32_t), cs);
    if (P->staged) cudaMemsetAsync(P->hist.p, 0, (2 * P->sb_cap + 2) * sizeof(uint32_t), cs);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)P->grid);
    cfg.blockDim = dim3(B_THREADS);
    cfg.dynamicSmemBytes = (size_t)batch_smem(P->staged, P->stage_bytes);
    cfg.stream = cs;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, batch_kernel(P->staged, P->compact), P->bufs);
    cudaError_t e2 = cudaStreamEndCapture(cs, &P->graph[t]);
    if (e != cudaSuccess) res = cuda_fail(e, "pip_plan: cooperative launch capture");
    else if (e2 != cudaSuccess) res = cuda_fail(e2, "pip_plan: end capture");
    else {
      e = cudaGraphInstantiate(&P->exec[t], P->graph[t], 0);
      if (e != cudaSuccess) res = cuda_fail(e, "pip_plan: graph instantiate");
    }
  } else {
    res = cuda_fail(e, "pip_plan: begin capture");
  }
  cudaStreamDestroy(cs);
  (void)s;
  return res;
}

extern "C" pip_status pip_plan_create(int64_t max_points, int32_t max_queries, void* stream,
                                      pip_plan* out) {
  if (!out) return fail(PIP_EINVAL, "pip_plan_create: out is NULL");
  *out = nullptr;
  if (max_points <= 0 || max_points >= (1ll << 32) - 1 || max_queries <= 0)
    return fail(PIP_EINVAL, "pip_plan_create: 0 < max_points < 2^32 - 1 and max_queries > 0");
  cudaStream_t s = (cudaStream_t)stream;
  std::unique_ptr<pip_plan_s> P(new pip_plan_s());
  PIP_CUDA(cudaGetDevice(&P->device));
  P->max_points = max_points;
  P->max_queries = max_queries;
  P->max_tiles = max_points / TILE + max_queries + 1;
  if (P->max_tiles >= (1ll << (32 - TILE_LOG2)))
    return fail(PIP_EINVAL, "pip_plan_create: too many tiles (max_points / 4096 + max_queries < 2^20)");
  P->off_sets = align_up(sizeof(RunHeader), 256);
  P->off_q = align_up(P->off_sets + sizeof(DevSet) * MAX_SETS, 256);
  P->off_qoff = align_up(P->off_q + sizeof(DevQuery) * (size_t)max_queries, 256);
  P->off_tiles = align_up(P->off_qoff + sizeof(uint32_t) * ((size_t)max_queries + 1), 256);
  P->tables_bytes = align_up(P->off_tiles + sizeof(uint4) * (size_t)P->max_tiles, 256);
  Alloc* al = &P->alloc;
  // queue: max_points plus two reserved chunks per warp of the largest grid
  int occ_max = 1;
  for (int staged = 0; staged < 2; ++staged)
    for (int compact = 0; compact < 2; ++compact) {
      auto k = batch_kernel(staged, compact != 0);
      int occ = 0;
      if (staged)
        PIP_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, batch_smem(1, P->stage_bytes)));
      PIP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, B_THREADS, batch_smem(staged, P->stage_bytes)));
      occ_max = std::max(occ_max, occ);
    }
  const int64_t queue_len = max_points + 2 * (int64_t)QCHUNK * (B_THREADS / 32) * num_sms() * occ_max;
  if (queue_len >= (1ll << 32)) return fail(PIP_EINVAL, "pip_plan_create: max_points too large");
  if (!P->tables.alloc(al, P->tables_bytes, s) || !P->queue.alloc(al, queue_len, s) ||
      !P->binned.alloc(al, max_points, s) || !P->ctr.alloc(al, 8, s) || !P->status.alloc(al, 2, s))
    return fail(PIP_ENOMEM, "pip_plan_create: device buffers");
  for (int i = 0; i < 2; ++i) {
    PIP_CUDA(cudaMallocHost((void**)&P->host_tables[i], P->tables_bytes));
    std::memset(P->host_tables[i], 0, P->tables_bytes);
    PIP_CUDA(cudaEventCreateWithFlags(&P->done[i], cudaEventDisableTiming));
  }
  PIP_CUDA(cudaMemsetAsync(P->status.p, 0, 2 * sizeof(uint32_t), s));
  pip_status st = plan_alloc_sb(P.get(), 1 << 16, s);
  if (st != PIP_OK) return st;
  st = plan_grid(P.get());
  if (st != PIP_OK) return st;
  if (!P->partial.alloc(al, (size_t)P->grid + 1, s)) return fail(PIP_ENOMEM, "pip_plan_create: partials");
  PIP_CUDA(cudaStreamSynchronize(s));
  *out = P.release();
  return PIP_OK;
}

static void plan_fill_bufs(pip_plan_s* P) {
  PlanBufs& B = P->bufs;
  uint8_t* t = P->tables.p;
  B.hdr = (RunHeader*)t;
  B.sets = (DevSet*)(t + P->off_sets);
  B.queries = (DevQuery*)(t + P->off_q);
  B.qoff = (uint32_t*)(t + P->off_qoff);
  B.tiles = (uint4*)(t + P->off_tiles);
  B.queue = P->queue.p;
  B.binned = P->binned.p;
  B.hist = P->hist.p;
  B.cursor = P->hist.p + P->sb_cap;
  B.off = P->off.p;
  B.partial = P->partial.p;
  B.ctr = P->ctr.p;
  B.status = P->status.p;
}

extern "C" pip_status pip_plan_run(pip_plan plan, const pip_query* q, int32_t n_q, void* stream) {
  if (!plan) return fail(PIP_EINVAL, "pip_plan_run: NULL plan");
  if (n_q < 0 || n_q > plan->max_queries) return fail(PIP_EINVAL, "pip_plan_run: too many queries");
  if (n_q > 0 && !q) return fail(PIP_EINVAL, "pip_plan_run: NULL queries");
  cudaStream_t s = (cudaStream_t)stream;
  // distinct sets in order of first use
  std::vector<pip_set> sets;
  std::vector<uint32_t> qset(n_q);
  int64_t total = 0;
  for (int i = 0; i < n_q; ++i) {
    if (!q[i].set || q[i].n < 0) return fail(PIP_EINVAL, "pip_plan_run: bad query");
    if (q[i].n > 0 && (!q[i].lon || !q[i].lat || !q[i].out))
      return fail(PIP_EINVAL, "pip_plan_run: NULL query array");
    auto it = std::find(sets.begin(), sets.end(), q[i].set);
    if (it == sets.end()) {
      if ((int)sets.size() == MAX_SETS) return fail(PIP_EINVAL, "pip_plan_run: more than 64 sets");
      sets.push_back(q[i].set);
      it = sets.end() - 1;
    }
    qset[i] = (uint32_t)(it - sets.begin());
    total += q[i].n;
  }
  if (total > plan->max_points) return fail(PIP_EINVAL, "pip_plan_run: more points than max_points");
  int64_t sb_total = 0;
  std::vector<uint32_t> sb_base(sets.size());
  for (size_t i = 0; i < sets.size(); ++i) {
    sb_base[i] = (uint32_t)sb_total;
    sb_total += std::max<int64_t>(1, sets[i]->view.n_sb);
  }
  if ((sb_total << SB_LOG2) >= (1ll << 32)) return fail(PIP_ERANGE, "pip_plan_run: too many leaf slots");
  pip_status st = plan_alloc_sb(plan, sb_total + 1, s);
  if (st != PIP_OK) return st;
  // tables into pinned host memory (the buffer of this turn, once its last
  // run has finished reading it)
  const int t = plan->turn;
  if (plan->used[t]) PIP_CUDA(cudaEventSynchronize(plan->done[t]));
  RunHeader H{};
  uint8_t* h = plan->host_tables[t];
  DevSet* hs = (DevSet*)(h + plan->off_sets);
  bool any_compact = false;
  for (size_t i = 0; i < sets.size(); ++i) {
    hs[i].view = sets[i]->view;
    hs[i].sb_base = sb_base[i];
    any_compact |= sets[i]->view.compact != 0;
  }
  if (plan->compact_fixed) any_compact |= plan->compact;
  if (any_compact != plan->compact) {  // the other kernel instantiation: capture again
    PIP_CUDA(cudaDeviceSynchronize());
    plan->drop_graphs();
    plan->compact = any_compact;
    st = plan_grid(plan);
    if (st != PIP_OK) return st;
    if (!plan->partial.alloc(&plan->alloc, (size_t)plan->grid + 1, s))
      return fail(PIP_ENOMEM, "pip_plan: partials");
  }
  DevQuery* hq = (DevQuery*)(h + plan->off_q);
  uint32_t* hqoff = (uint32_t*)(h + plan->off_qoff);
  uint4* ht = (uint4*)(h + plan->off_tiles);
  uint32_t n_tiles = 0, acc = 0;
  for (int i = 0; i < n_q; ++i) {
    hq[i] = DevQuery{q[i].lon, q[i].lat, q[i].out, qset[i], (uint32_t)q[i].n};
    hqoff[i] = acc;
    acc += (uint32_t)q[i].n;
  }
  hqoff[n_q] = acc;
  // tiles grouped by set (queries in order within a set): the CTAs, which
  // take tiles in list order, then classify mostly one set's points at a
  // time, so one index at a time competes for L2 (4,096 queries over 8
  // sets: 3.06 against 3.87 ms a launch)
  for (uint32_t k = 0; k < (uint32_t)sets.size(); ++k)
    for (int i = 0; i < n_q; ++i) {
      if (qset[i] != k) continue;
      for (int64_t t0 = 0; t0 < q[i].n; t0 += TILE)
        ht[n_tiles++] = make_uint4((uint32_t)i, (uint32_t)t0, (uint32_t)std::min<int64_t>(TILE, q[i].n - t0),
                                   hqoff[i] + (uint32_t)t0);
    }
  H.n_q = (uint32_t)n_q;
  H.n_sets = (uint32_t)sets.size();
  H.n_tiles = n_tiles;
  H.total_points = acc;
  // whole tiles per warp when every warp gets several (the ring drains once
  // per item); 1024-point items for small batches, whose latency is one item
  H.sub_log2 = (int64_t)acc >= (int64_t)plan->grid * (B_THREADS / 32) * 4 * TILE ? 12u : 10u;
  H.n_sb_total = (uint32_t)sb_total;
  H.ppc = plan->ppc;
  H.stage16 = plan->stage_bytes / 16;
  std::memcpy(h, &H, sizeof(H));
  plan_fill_bufs(plan);
  st = plan_capture(plan, t, s);
  if (st != PIP_OK) return st;
  PIP_CUDA(cudaGraphLaunch(plan->exec[t], s));
  PIP_CUDA(cudaEventRecord(plan->done[t], s));
  plan->used[t] = true;
  plan->turn = t ^ 1;
  count_launches(1);
  return PIP_OK;
}

extern "C" pip_status pip_plan_check(pip_plan plan, void* stream) {
  if (!plan) return fail(PIP_EINVAL, "pip_plan_check: NULL plan");
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t w = 0;
  PIP_CUDA(cudaMemcpyAsync(&w, plan->status.p, sizeof(w), cudaMemcpyDeviceToHost, s));
  PIP_CUDA(cudaStreamSynchronize(s));
  if (w) {
    PIP_CUDA(cudaMemsetAsync(plan->status.p, 0, sizeof(uint32_t), s));
    PIP_CUDA(cudaStreamSynchronize(s));
    return fail(PIP_ETIMEOUT, w & 2u ? "batched launch: a grid barrier wait ran out"
                                     : "batched launch: a staging wait ran out");
  }
  return PIP_OK;
}

extern "C" pip_status pip_plan_destroy(pip_plan plan) {
  if (!plan) return PIP_OK;
  cudaDeviceSynchronize();
  delete plan;
  return PIP_OK;
}

// Plan knobs used by the autotuner (internal).
namespace pip {
// Make a plan ready for runs over a known family of sets: superbin buffers
// for `superbins` in all (the sum over the sets a run may use), the kernel
// instantiation for `compact` kept for every run, and both graphs captured
// and uploaded, so no run over those sets allocates or captures.
pip_status plan_prepare(pip_plan plan, int64_t superbins, bool compact, cudaStream_t s) {
  pip_status st = plan_alloc_sb(plan, superbins + 1, s);
  if (st != PIP_OK) return st;
  if (compact != plan->compact) {
    plan->drop_graphs();
    plan->compact = compact;
    st = plan_grid(plan);
    if (st != PIP_OK) return st;
    if (!plan->partial.alloc(&plan->alloc, (size_t)plan->grid + 1, s))
      return fail(PIP_ENOMEM, "pip_plan: partials");
  }
  plan->compact_fixed = true;
  plan_fill_bufs(plan);
  for (int t = 0; t < 2; ++t) {
    st = plan_capture(plan, t, s);
    if (st != PIP_OK) return st;
    PIP_CUDA(cudaGraphUpload(plan->exec[t], s));
  }
  PIP_CUDA(cudaStreamSynchronize(s));
  return PIP_OK;
}

pip_status plan_set_knobs(pip_plan plan, uint32_t ppc, int staged) {
  if (plan->ppc == ppc && plan->staged == staged) return PIP_OK;
  plan->ppc = ppc;
  plan->drop_graphs();  // the header carries ppc, but the graph holds the launch shape
  if (plan->staged != staged) {
    plan->staged = staged;
    pip_status st = plan_grid(plan);
    if (st != PIP_OK) return st;
    if (!plan->partial.alloc(&plan->alloc, (size_t)plan->grid + 1, 0))
      return fail(PIP_ENOMEM, "pip_plan: partials");
    cudaDeviceSynchronize();
  }
  return PIP_OK;
}
}  // namespace pip

extern "C" pip_status pip_project_batch(const pip_query* q, int32_t n_q, void* stream) {
  if (n_q < 0 || (n_q > 0 && !q)) return fail(PIP_EINVAL, "pip_project_batch: bad arguments");
  if (n_q == 0) return PIP_OK;
  int64_t total = 0;
  for (int i = 0; i < n_q; ++i) total += std::max<int64_t>(0, q[i].n);
  pip_plan plan = nullptr;
  pip_status st = pip_plan_create(std::max<int64_t>(1, total), n_q, stream, &plan);
  if (st != PIP_OK) return st;
  st = pip_plan_run(plan, q, n_q, stream);
  if (st == PIP_OK) st = pip_plan_check(plan, stream);
  pip_plan_destroy(plan);
  return st;
}
