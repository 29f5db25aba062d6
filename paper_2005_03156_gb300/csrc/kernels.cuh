// Device code of the projection path, shared by the plain and the batched
// forms.
//
//   K1 classify   streams the points (two 16-byte loads of lon and two of lat
//                 per 4 points), quantizes them with integer instructions and
//                 reads their top-grid descriptors (and the first trie level
//                 when the trie is stored as 16-byte entries); EMPTY and
//                 INTERIOR cells answer at once (Sec. IV true-hit filtering).
//                 Points in cells split further wait in a per-warp ring
//                 (TrieRing) that is walked one trie level for 128 points at
//                 a time. Points in boundary
//                 leaves go to the residual queue through per-warp chunks
//                 (ChunkWriter) and are counted per superbin.
//   K2 bin        counting sort of the residual by superbin: scan of the
//                 counts and a scatter, so points that share polygons sit
//                 together (the GPU form of sorting the points so many share
//                 one polygon call, Sec. III-A / III).
//   K3 cross      persistent CTAs take chunks of pts_per_cta binned points
//                 from an atomic counter. A chunk covers a contiguous range
//                 of leaf slots whose records (candidates + clipped edges) are
//                 contiguous in HBM; when they fit, one cp.async.bulk copy
//                 completed on an mbarrier stages them in shared memory
//                 (double-buffered: the next chunk's copy flies while the
//                 current one is tested). The exact crossing-number test
//                 (Sec. III-A) then runs per point; points whose leaf holds a
//                 long edge list are tested by the whole warp: lanes take
//                 strided edges and a ballot + popc gives the parity.
#pragma once

#include "pip_internal.cuh"

namespace pip {

constexpr int K1_THREADS = 256;
constexpr int K3_THREADS = 256;
constexpr int LONG_LIST = 48;  // edges above which a point is tested by its whole warp
constexpr unsigned long long WAIT_NS = 2000000000ull;  // bounded waits: 2 s

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// --------------------------------------------------------------- K1 pieces
// Trie walk for 4 points at once so their dependent loads overlap.
__device__ __forceinline__ void lookup4(const IndexView& ix, const int32_t (&qx)[4],
                                        const int32_t (&qy)[4], const bool (&ok)[4],
                                        uint32_t (&d)[4]) {
  const uint64_t pol = policy_evict_last();
  uint32_t dx[4], dy[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    dx[j] = (uint32_t)qx[j] - (uint32_t)ix.gx0;
    dy[j] = (uint32_t)qy[j] - (uint32_t)ix.gy0;
    const uint32_t cx = dx[j] >> ix.s0, cy = dy[j] >> ix.s0;
    const bool in = ok[j] & (cx < ix.nx) & (cy < ix.ny) & (qx[j] >= ix.gx0) & (qy[j] >= ix.gy0);
    d[j] = in ? ld_index_u32(ix.table + (size_t)cy * ix.nx + cx, pol) : 0u;
  }
  int s = ix.s0;
  const uint32_t m = (1u << NODE_K) - 1u;
  if (!ix.compact) {  // 16-byte entries
#pragma unroll 1
    while (((d[0] >> 30) == TAG_CHILD) | ((d[1] >> 30) == TAG_CHILD) | ((d[2] >> 30) == TAG_CHILD) |
           ((d[3] >> 30) == TAG_CHILD)) {
      s = s > NODE_K ? s - NODE_K : 0;  // leaf and id entries sit one level below their cell
      uint4 e[4];
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if ((d[j] >> 30) == TAG_CHILD) e[j] = ld_entry(ix.nodes, d[j] & PAYLOAD_MASK, pol);
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if ((d[j] >> 30) == TAG_CHILD) d[j] = entry_step(e[j], (((dy[j] >> s) & m) << NODE_K) | ((dx[j] >> s) & m));
    }
    return;
  }
#pragma unroll 1
  while (((d[0] >> 30) == TAG_CHILD) | ((d[1] >> 30) == TAG_CHILD) | ((d[2] >> 30) == TAG_CHILD) |
         ((d[3] >> 30) == TAG_CHILD)) {
    s -= NODE_K;
    NodeWords nw[4];
#pragma unroll
    for (int j = 0; j < 4; ++j)  // issue the node loads of all four points first
      if ((d[j] >> 30) == TAG_CHILD) nw[j] = ld_node(ix.nodes, d[j] & SLOT_MASK, pol);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if ((d[j] >> 30) == TAG_CHILD) {
        if (d[j] & DESC_COMPACT) {  // compact leaf: answered here
          const int32_t v = compact_answer(nw[j], ix.nodes, d[j] & SLOT_MASK,
                                           ((d[j] >> DESC_SLOTS_SHIFT) & 3u) + 1u, qx[j], qy[j], pol);
          d[j] = v < 0 ? make_desc(TAG_EMPTY, 0) : make_desc(TAG_INTERIOR, (uint32_t)v);
        } else {
          const uint32_t sub = (((dy[j] >> s) & m) << NODE_K) | ((dx[j] >> s) & m);
          d[j] = node_step(nw[j], sub);
        }
      }
    }
  }
}

// Append up to 4 residual points of this lane to the queue with one atomic
// per warp; count them per superbin (hist may be offset per set). idx_of(j)
// is the index of slot j's point.
template <class IdxOf>
__device__ __forceinline__ void append_residual_at(uint32_t mask, const int32_t (&qx)[4],
                                                   const int32_t (&qy)[4], const uint32_t (&d)[4],
                                                   IdxOf idx_of, Residual* __restrict__ queue,
                                                   uint32_t* __restrict__ qcount,
                                                   uint32_t* __restrict__ hist, uint32_t slot_add) {
  const uint32_t full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  if (!__any_sync(full, mask != 0u)) return;
  const uint32_t r = __popc(mask);
  uint32_t incl = r;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(full, incl, o);
    if (lane >= o) incl += t;
  }
  uint32_t base = 0;
  if (lane == 31) base = atomicAdd(qcount, incl);
  base = __shfl_sync(full, base, 31) + incl - r;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (mask & (1u << j)) {
      const uint32_t slot = (d[j] & PAYLOAD_MASK) + slot_add;
      queue[base++] = make_uint4((uint32_t)qx[j], (uint32_t)qy[j], idx_of(j), slot);
      atomicAdd(hist + (slot >> SB_LOG2), 1u);
    }
  }
}

// Slot j holds point idx0 + j.
__device__ __forceinline__ void append_residual(uint32_t mask, const int32_t (&qx)[4],
                                                const int32_t (&qy)[4], const uint32_t (&d)[4],
                                                uint32_t idx0, Residual* __restrict__ queue,
                                                uint32_t* __restrict__ qcount,
                                                uint32_t* __restrict__ hist, uint32_t slot_add) {
  append_residual_at(mask, qx, qy, d, [idx0](int j) { return idx0 + (uint32_t)j; }, queue, qcount,
                     hist, slot_add);
}

// Residual entries of one warp into queue chunks of QCHUNK entries. The first
// chunk is reserved when the warp meets its first residual point; from then
// on lane 0 holds the base of the next chunk, reserved one chunk ahead, so
// an append waits on the queue counter only once per warp. (Atomics on one
// address are serialised in L2: one per warp and step of 128 points cost as
// much as a whole trie walk.) Entries reserved but not filled are marked
// RES_HOLE at the end; the warp's residual count is added to *real then.
// A warp holds at most 2 * QCHUNK unused entries, so the queue needs
// n + 2 * QCHUNK * warps entries. All lanes of the warp call every method.
constexpr uint32_t QCHUNK = 256;  // >= 128, the most one call appends

struct ChunkWriter {
  uint32_t cb = 0, cu = 0, nb = 0, real = 0;  // cb, cu, real: warp-uniform; nb: lane 0
  bool have = false;                          // warp-uniform: a chunk is reserved

  template <class IdxOf>
  __device__ __forceinline__ void put(uint32_t mask, const int32_t (&qx)[4], const int32_t (&qy)[4],
                                      const uint32_t (&d)[4], IdxOf idx_of, Residual* __restrict__ queue,
                                      uint32_t* __restrict__ count, uint32_t* __restrict__ hist,
                                      uint32_t slot_add) {
    const uint32_t full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint32_t c = __popc(mask);
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(full, incl, o);
      if (lane >= o) incl += t;
    }
    const uint32_t tot = __shfl_sync(full, incl, 31);
    if (tot == 0u) return;
    if (!have) {
      uint32_t b = 0;
      if (lane == 0) b = atomicAdd(count, QCHUNK);
      cb = __shfl_sync(full, b, 0);
      cu = 0;
      if (lane == 0) nb = atomicAdd(count, QCHUNK);
      have = true;
    }
    const uint32_t nbb = __shfl_sync(full, nb, 0);
    uint32_t r = cu + incl - c;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if ((mask >> j) & 1u) {
        const uint32_t slot = (d[j] & PAYLOAD_MASK) + slot_add;
        const uint32_t at = r < QCHUNK ? cb + r : nbb + (r - QCHUNK);
        queue[at] = make_uint4((uint32_t)qx[j], (uint32_t)qy[j], idx_of(j), slot);
        atomicAdd(hist + (slot >> SB_LOG2), 1u);
        ++r;
      }
    }
    cu += tot;
    real += tot;
    if (cu >= QCHUNK) {  // the next chunk becomes current; reserve another
      cb = nbb;
      cu -= QCHUNK;
      if (lane == 0) nb = atomicAdd(count, QCHUNK);
    }
  }

  __device__ __forceinline__ void finish(Residual* __restrict__ queue, uint32_t* __restrict__ real_count) {
    if (!have) return;
    const int lane = threadIdx.x & 31;
    const uint32_t nbb = __shfl_sync(0xffffffffu, nb, 0);
    for (uint32_t k = cu + lane; k < QCHUNK; k += 32) queue[cb + k] = make_uint4(0u, 0u, 0u, RES_HOLE);
    for (uint32_t k = lane; k < QCHUNK; k += 32) queue[nbb + k] = make_uint4(0u, 0u, 0u, RES_HOLE);
    if (lane == 0) atomicAdd(real_count, real);
  }
};

// Per-warp ring of points whose cell is split (K1, deferred-queue form): a
// step reads the top-grid descriptors of 4 points per lane and pushes the
// split ones here; step() then walks one trie level for up to 128 entries at
// once (4 per lane), stores INTERIOR ids, hands boundary leaves to the
// residual writer and pushes back the entries still split. Entry: (qx, qy, z,
// node) plus the shift of the node's children; the point's id goes to
// out_base[z] and its residual index is code_base + z. The ring lives in
// shared memory (TRING entries, at most TRING - 1 held); all lanes call.
constexpr uint32_t TRING = 256;

struct TrieRing {
  uint4* rq;
  uint8_t* rs;
  uint32_t head = 0, count = 0;  // warp-uniform

  __device__ __forceinline__ void push(uint32_t mask, const int32_t (&qx)[4], const int32_t (&qy)[4],
                                       const uint32_t (&z)[4], const uint32_t (&d)[4], const int (&sh)[4]) {
    const uint32_t full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint32_t c = __popc(mask);
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(full, incl, o);
      if (lane >= o) incl += t;
    }
    uint32_t pos = head + count + incl - c;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if ((mask >> j) & 1u) {
        const uint32_t p = pos++ & (TRING - 1);
        rq[p] = make_uint4((uint32_t)qx[j], (uint32_t)qy[j], z[j], d[j] & PAYLOAD_MASK);
        rs[p] = (uint8_t)sh[j];
      }
    }
    count += __shfl_sync(full, incl, 31);
  }

  // one trie level for the ring's first `take` entries (take <= 128,
  // uniform); COMPACT = false for a trie without compact leaves
  template <bool COMPACT = true>
  __device__ __forceinline__ void step(uint32_t take, const IndexView& ix, uint64_t pol,
                                       int32_t* __restrict__ out_base, uint32_t code_base,
                                       ChunkWriter& res, Residual* __restrict__ queue,
                                       uint32_t* __restrict__ qcount, uint32_t* __restrict__ hist,
                                       uint32_t slot_add) {
    const uint32_t full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint32_t m = (1u << NODE_K) - 1u;
    __syncwarp();
    int32_t qx[4], qy[4];
    uint32_t z[4], d[4];
    int sh[4];
    uint32_t have = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t k = (uint32_t)lane + 32u * j;
      qx[j] = qy[j] = 0;
      z[j] = d[j] = 0u;
      sh[j] = 0;
      if (k < take) {
        const uint32_t p = (head + k) & (TRING - 1);
        const uint4 e = rq[p];
        qx[j] = (int32_t)e.x;
        qy[j] = (int32_t)e.y;
        z[j] = e.z;
        d[j] = e.w;
        sh[j] = rs[p];
        have |= 1u << j;
      }
    }
    head += take;
    count -= take;
    __syncwarp();  // every entry is read before the pushes below reuse slots
    NodeWords nw[4];
    uint4 ne[4];
    const uint64_t cold = policy_evict_first();
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (COMPACT) {
        const uint32_t sl = d[j] & SLOT_MASK;
        if ((have >> j) & 1u) nw[j] = ld_node(ix.nodes, sl, sl < ix.hot_nodes ? pol : cold);
      } else {
        const uint32_t sl = d[j] & PAYLOAD_MASK;
        if ((have >> j) & 1u) ne[j] = ld_entry(ix.nodes, sl, sl < ix.hot_nodes ? pol : cold);
      }
    }
    uint32_t leaf = 0, again = 0;
    if (COMPACT) {  // compact leaves: answered here, one entry per pass of a
                    // rolled loop (one copy of the evaluation keeps the code small)
      uint32_t cm = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) cm |= (((have >> j) & 1u) && (d[j] & DESC_COMPACT) ? 1u : 0u) << j;
      have &= ~cm;
#pragma unroll 1
      while (cm) {
        const int j = __ffs(cm) - 1;
        cm &= cm - 1;
        uint32_t w[8];
#pragma unroll
        for (int k = 0; k < 8; ++k)
          w[k] = j == 0 ? nw[0].w[k] : j == 1 ? nw[1].w[k] : j == 2 ? nw[2].w[k] : nw[3].w[k];
        const uint32_t dj = j == 0 ? d[0] : j == 1 ? d[1] : j == 2 ? d[2] : d[3];
        const int32_t px = j == 0 ? qx[0] : j == 1 ? qx[1] : j == 2 ? qx[2] : qx[3];
        const int32_t py = j == 0 ? qy[0] : j == 1 ? qy[1] : j == 2 ? qy[2] : qy[3];
        const uint32_t zj = j == 0 ? z[0] : j == 1 ? z[1] : j == 2 ? z[2] : z[3];
        const uint32_t sl = dj & SLOT_MASK;
        const int32_t v = compact_answer_words(w[0], w[1], w[2], w[3], w[4], w[5], w[6], w[7], ix.nodes, sl,
                                               ((dj >> DESC_SLOTS_SHIFT) & 3u) + 1u, px, py,
                                               sl < ix.hot_nodes ? pol : cold);
        if (v >= 0) out_base[zj] = v;
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if ((have >> j) & 1u) {
        const uint32_t dx = (uint32_t)qx[j] - (uint32_t)ix.gx0, dy = (uint32_t)qy[j] - (uint32_t)ix.gy0;
        const uint32_t sub = (((dy >> sh[j]) & m) << NODE_K) | ((dx >> sh[j]) & m);
        if (COMPACT) d[j] = node_step<true>(nw[j], sub);
        else d[j] = entry_step(ne[j], sub);
        const uint32_t tag = d[j] >> 30;
        if (tag == TAG_INTERIOR) out_base[z[j]] = (int32_t)(d[j] & PAYLOAD_MASK);
        if (tag == TAG_LEAF && ix.approx_id) {  // approximate mode: the leaf's own answer
          out_base[z[j]] = ix.approx_id[d[j] & PAYLOAD_MASK];
        } else {
          leaf |= (tag == TAG_LEAF ? 1u : 0u) << j;
        }
        again |= (tag == TAG_CHILD ? 1u : 0u) << j;
        sh[j] = sh[j] > NODE_K ? sh[j] - NODE_K : 0;  // 16-byte leaf / id entries sit one level below
      }
    }
    if (__any_sync(full, leaf != 0u))
      res.put(leaf, qx, qy, d, [&](int j) { return code_base + z[j]; }, queue, qcount, hist, slot_add);
    if (__any_sync(full, again != 0u)) push(again, qx, qy, z, d, sh);
  }
};

// K2 body: queue entries [0, n) go to binned[off[sb] + rank], rank taken from
// cursor[sb]; RES_HOLE entries are skipped. (Four entries per thread with
// their atomics issued back to back measured slower: 0.29 vs 0.27 ms.)
__device__ __forceinline__ void scatter_by_superbin(const Residual* __restrict__ queue, uint32_t n,
                                                    const uint64_t* __restrict__ off,
                                                    uint32_t* __restrict__ cursor,
                                                    Residual* __restrict__ binned, uint32_t tid,
                                                    uint32_t stride) {
  for (uint64_t i = tid; i < n; i += stride) {
    const Residual e = queue[i];
    if (e.w == RES_HOLE) continue;
    const uint32_t sb = e.w >> SB_LOG2;
    binned[(uint32_t)off[sb] + atomicAdd(cursor + sb, 1u)] = e;
  }
}

// Classify 4 points; returns their ids (-1 for residual ones) and the
// residual mask.
__device__ __forceinline__ uint32_t classify4(const IndexView& ix, const double (&x)[4],
                                              const double (&y)[4], int32_t (&id)[4],
                                              int32_t (&qx)[4], int32_t (&qy)[4], uint32_t (&d)[4]) {
  bool ok[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    qx[j] = 0;
    qy[j] = 0;
    ok[j] = quantize_double(x[j], qx[j]) & quantize_double(y[j], qy[j]);
  }
  lookup4(ix, qx, qy, ok, d);
  uint32_t mask = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const uint32_t tag = d[j] >> 30;
    id[j] = tag == TAG_INTERIOR ? (int32_t)(d[j] & PAYLOAD_MASK) : -1;
    if (tag == TAG_LEAF && ix.approx_id) id[j] = ix.approx_id[d[j] & PAYLOAD_MASK];  // approximate mode
    else mask |= (tag == TAG_LEAF ? 1u : 0u) << j;
  }
  return mask;
}

// --------------------------------------------------------------- K3 pieces
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Thread 0: expect `bytes` on bar and start the bulk copy global -> shared.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Bounded wait for phase `parity` of bar; false when it ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          unsigned long long limit_ns = WAIT_NS) {
  const uint32_t a = smem_addr(bar);
  uint32_t done = 0;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(done)
      : "r"(a), "r"(parity)
      : "memory");
  if (done) return true;
  const unsigned long long t0 = global_ns();
  while (true) {
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

// One leaf slot's record (layout in pip_internal.cuh).
struct LeafRec {
  const uint32_t* w;  // nc, cand[nc], edge_end[nc]
  const int4* edges;
};

__device__ __forceinline__ LeafRec leaf_rec(const uint4* base) {
  LeafRec r;
  r.w = (const uint32_t*)base;
  r.edges = (const int4*)(base + ((1u + 2u * r.w[0] + 3u) >> 2));
  return r;
}

// Crossing test of one point against its leaf's candidates, in id order.
__device__ __forceinline__ int32_t test_point(const LeafRec& b, int32_t qx, int32_t qy) {
  const uint32_t nc = b.w[0];
  const uint32_t* cand = b.w + 1;
  const uint32_t* eend = cand + nc;
  uint32_t e = 0;
  for (uint32_t c = 0; c < nc; ++c) {
    const uint32_t cw = cand[c];
    uint32_t par = cw >> 31;
    const uint32_t e1 = eend[c];
    for (; e < e1; ++e) par ^= edge_crosses(b.edges[e], qx, qy);
    if (par) return (int32_t)(cw & 0x7FFFFFFFu);
  }
  return -1;
}

// The same test done by the whole warp for one point (broadcast values):
// lanes take edges lane, lane+32, ...; the parity is the popcount of the
// ballot of the lanes' partial parities.
__device__ __forceinline__ int32_t test_point_warp(const LeafRec& b, int32_t qx, int32_t qy) {
  const int lane = threadIdx.x & 31;
  const uint32_t nc = b.w[0];
  const uint32_t* cand = b.w + 1;
  const uint32_t* eend = cand + nc;
  uint32_t e0 = 0;
  for (uint32_t c = 0; c < nc; ++c) {
    const uint32_t cw = cand[c];
    uint32_t part = 0;
    const uint32_t e1 = eend[c];
    for (uint32_t e = e0 + lane; e < e1; e += 32) part ^= edge_crosses(b.edges[e], qx, qy);
    e0 = e1;
    const uint32_t par = (cw >> 31) ^ (__popc(__ballot_sync(0xffffffffu, part)) & 1u);
    if (par) return (int32_t)(cw & 0x7FFFFFFFu);
  }
  return -1;
}

__device__ __forceinline__ uint32_t leaf_edges(const LeafRec& b) {
  const uint32_t nc = b.w[0];
  return nc ? b.w[nc + nc] : 0u;
}

// Crossing tests of the binned residual points [first, first + count),
// count <= 32, one per lane of the calling warp. Each point's leaf record
// (two dependent reads: the slot's offset, then the record with candidates
// and edges together) lives either in the staged copy of the chunk's
// contiguous record range (staged != nullptr, starting at 16-byte unit
// region16 of the blobs) or in global memory. Points whose leaf holds a long
// edge list are tested by the whole warp. Ids go through `store`.
template <class Store>
__device__ __forceinline__ void test_warp_slice(const IndexView& ix, const Residual* __restrict__ binned,
                                                uint32_t first, uint32_t count, const uint4* staged,
                                                uint32_t region16, Store store) {
  const int lane = threadIdx.x & 31;
  bool active = (uint32_t)lane < count;
  Residual r = make_uint4(0, 0, 0, 0);
  const uint4* bp = ix.blobs;
  if (active) r = binned[first + lane];
  active &= r.w != RES_HOLE;  // a queue read in arrival order keeps its unused reserved entries
  if (active) {
    const uint32_t off = ix.slot_off[r.w];
    bp = staged ? staged + (off - region16) : ix.blobs + off;
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

// Test the residual points [first, first + count) of one work item: the
// CTA's warps take 32-point slices of it.
template <class Store>
__device__ __forceinline__ void test_chunk(const IndexView& ix, const Residual* __restrict__ binned,
                                           uint32_t first, uint32_t count, const uint4* staged,
                                           uint32_t region16, Store store) {
  for (uint32_t base = threadIdx.x & ~31u; base < count; base += blockDim.x)
    test_warp_slice(ix, binned, first + base, min(32u, count - base), staged, region16, store);
}

}  // namespace pip
