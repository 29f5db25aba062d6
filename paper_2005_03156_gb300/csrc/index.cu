// Device index build for one polygon set.
//
// The paper's two filters, re-designed for the GPU:
//   * Sec. III: bounding boxes, tested down the region -> county -> tract ->
//     block hierarchy, pick the polygons a point must be tested against.
//     Here they pick the candidate polygons of each top-level grid cell: a
//     polygon is a candidate of a cell iff its closed box meets the cell's
//     closed lattice rectangle. Found by descending the box hierarchy (one
//     thread per cell) or, equivalently, by rasterizing block boxes.
//   * Sec. IV: cells that lie wholly inside one polygon answer without a
//     point-in-polygon test; boundary cells are subdivided so most of the
//     area is covered by such interior cells ("true hit filtering").
//
// Per cell and candidate, every edge is classified against the cell row
// [y0, y1) x [x0, x1) (lattice points x0..x1-1, y0..y1-1):
//   drop  the edge's y-span [ymin, ymax) misses [y0, y1-1], or it lies
//         wholly at or left of x0 (it can never count for a point here);
//   fold  it lies wholly right of x1-1 and spans the whole row: it counts
//         for every point of the cell, so it only flips the base parity;
//   keep  otherwise.
// Then, for every point p of the cell, inside(P, p) = base XOR (sum of kept
// crossings), exactly. A candidate with no kept edge has a constant answer:
// base 0 -> never inside (dropped); base 1 -> inside everywhere, which also
// ends the candidate list (higher ids can never be the smallest). A cell
// whose list is empty is EMPTY; a cell whose list is one such full candidate
// is INTERIOR; otherwise it is a boundary cell: split into 4^k children
// (whose edges are re-clipped from the parent's kept edges) or a leaf.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstring>
#include <vector>

#include "kernels.cuh"

namespace pip {

namespace {

constexpr int TB = 256;

inline unsigned blocks_for(int64_t n, int per = TB) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + per - 1) / per, 1 << 30));
}

__device__ __forceinline__ bool box_meets(int4 b, long long x0, long long y0, long long x1m,
                                          long long y1m) {
  // b = (xmin, ymin, xmax, ymax), closed; empty boxes have xmin > xmax
  return b.x <= b.z && (long long)b.x <= x1m && (long long)b.z >= x0 && (long long)b.y <= y1m &&
         (long long)b.w >= y0;
}

// ----------------------------------------------------------------- B0, B1
__global__ void k_validate_csr(const int64_t* __restrict__ ring_off, int64_t n_ring,
                               const int64_t* __restrict__ pro, int64_t n_poly, int64_t n_vert,
                               uint32_t* err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n_ring; i += stride) {
    const int64_t v = ring_off[i];
    if (v < 0 || v > n_vert || (i > 0 && v < ring_off[i - 1])) atomicOr(err, 1u);
    if (i == 0 && v != 0) atomicOr(err, 1u);
    if (i == n_ring && v != n_vert) atomicOr(err, 1u);
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n_poly; i += stride) {
    const int64_t r = pro[i];
    if (r < 0 || r > n_ring || (i > 0 && r < pro[i - 1])) atomicOr(err, 1u);
    if (i == 0 && r != 0) atomicOr(err, 1u);
    if (i == n_poly && r != n_ring) atomicOr(err, 1u);
  }
}

// Polygon boxes (warp per polygon) and the edge-span check (bit 2).
__global__ void k_poly_box(const int32_t* __restrict__ vx, const int32_t* __restrict__ vy,
                           const int64_t* __restrict__ ring_off, const int64_t* __restrict__ pro,
                           int64_t n_poly, int4* __restrict__ box, uint32_t* err) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = (((int64_t)blockIdx.x * blockDim.x) + threadIdx.x) >> 5; p < n_poly; p += warps) {
    int xmin = INT32_MAX, ymin = INT32_MAX, xmax = INT32_MIN, ymax = INT32_MIN;
    bool bad = false;
    for (int64_t r = pro[p]; r < pro[p + 1]; ++r) {
      const int64_t a = ring_off[r], b = ring_off[r + 1];
      for (int64_t i = a + lane; i < b; i += 32) {
        const int64_t j = (i + 1 == b) ? a : i + 1;
        const int x = vx[i], y = vy[i];
        xmin = min(xmin, x); xmax = max(xmax, x);
        ymin = min(ymin, y); ymax = max(ymax, y);
        const long long dx = (long long)vx[j] - x, dy = (long long)vy[j] - y;
        bad |= (dx >= (1ll << 31)) | (dx <= -(1ll << 31)) | (dy >= (1ll << 31)) | (dy <= -(1ll << 31));
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      xmin = min(xmin, __shfl_xor_sync(0xffffffffu, xmin, o));
      ymin = min(ymin, __shfl_xor_sync(0xffffffffu, ymin, o));
      xmax = max(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
      ymax = max(ymax, __shfl_xor_sync(0xffffffffu, ymax, o));
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(err, 2u);
    if (lane == 0) box[p] = make_int4(xmin, ymin, xmax, ymax);
  }
}

__global__ void k_union_box(const int4* __restrict__ box, int64_t n, int* __restrict__ out4) {
  int xmin = INT32_MAX, ymin = INT32_MAX, xmax = INT32_MIN, ymax = INT32_MIN;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int4 b = box[i];
    if (b.x > b.z) continue;
    xmin = min(xmin, b.x); ymin = min(ymin, b.y);
    xmax = max(xmax, b.z); ymax = max(ymax, b.w);
  }
  atomicMin(out4 + 0, xmin);
  atomicMin(out4 + 1, ymin);
  atomicMax(out4 + 2, xmax);
  atomicMax(out4 + 3, ymax);
}

__global__ void k_f64_to_lattice(const double* __restrict__ x, const double* __restrict__ y,
                                 int64_t n, int32_t* __restrict__ qx, int32_t* __restrict__ qy,
                                 uint32_t* err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t a = 0, b = 0;
    const bool ok = quantize_double(x[i], a) & quantize_double(y[i], b);
    if (!ok) atomicOr(err, 2u);
    qx[i] = a;
    qy[i] = b;
  }
}

// ----------------------------------------------------------------- B3
__global__ void k_count_children(const int32_t* __restrict__ parent, int64_t n,
                                 uint32_t* __restrict__ cnt, int64_t n_parent, uint32_t* err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t q = parent[i];
    if (q < 0 || q >= n_parent) {
      atomicOr(err, 1u);
      continue;
    }
    atomicAdd(cnt + q, 1u);
  }
}

__global__ void k_fill_children(const int32_t* __restrict__ parent, int64_t n,
                                const uint64_t* __restrict__ off, uint32_t* __restrict__ cur,
                                int32_t* __restrict__ child, int4* __restrict__ pbox,
                                const int4* __restrict__ cbox, int64_t n_parent) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t q = parent[i];
    if (q < 0 || q >= n_parent) continue;
    const uint32_t k = atomicAdd(cur + q, 1u);
    child[off[q] + k] = (int32_t)i;
    const int4 b = cbox[i];
    if (b.x > b.z) continue;
    int* pb = (int*)(pbox + q);
    atomicMin(pb + 0, b.x);
    atomicMin(pb + 1, b.y);
    atomicMax(pb + 2, b.z);
    atomicMax(pb + 3, b.w);
  }
}

__global__ void k_fill_int4(int4* p, int64_t n, int4 v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

struct Hier {
  int levels;                        // top level index (0 = flat)
  int64_t len[MAX_LEVELS];           // nodes per level
  const int4* box[MAX_LEVELS];       // per level
  const uint64_t* coff[MAX_LEVELS];  // [l >= 1]: children CSR of level-l nodes
  const int32_t* cids[MAX_LEVELS];   // [l >= 1]: child ids (level l-1 nodes)
};

struct Grid {
  long long gx0, gy0;
  uint32_t nx, ny;
  int s0;
};

// ----------------------------------------------------------------- B4
// One thread per top cell: depth-first descent of the box hierarchy. With
// `ids == nullptr` it counts, otherwise it writes the candidate polygons.
__global__ void k_top_hier(Hier h, Grid g, uint32_t* __restrict__ cnt,
                           const uint64_t* __restrict__ off, int32_t* __restrict__ ids) {
  const int64_t cells = (int64_t)g.nx * g.ny;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < cells;
       c += (int64_t)gridDim.x * blockDim.x) {
    const long long cx = c % g.nx, cy = c / g.nx;
    const long long x0 = g.gx0 + (cx << g.s0), y0 = g.gy0 + (cy << g.s0);
    const long long x1m = x0 + (1ll << g.s0) - 1, y1m = y0 + (1ll << g.s0) - 1;
    uint64_t cur[MAX_LEVELS], end[MAX_LEVELS];
    int l = h.levels;
    cur[l] = 0;
    end[l] = (uint64_t)h.len[l];
    uint32_t n = 0;
    uint64_t w = ids ? off[c] : 0;
    while (true) {
      if (cur[l] == end[l]) {
        if (l == h.levels) break;
        ++l;
        continue;
      }
      const int64_t node = (l == h.levels) ? (int64_t)cur[l] : (int64_t)h.cids[l + 1][cur[l]];
      ++cur[l];
      if (!box_meets(h.box[l][node], x0, y0, x1m, y1m)) continue;
      if (l == 0) {
        if (ids) ids[w++] = (int32_t)node;
        ++n;
        continue;
      }
      cur[l - 1] = h.coff[l][node];
      end[l - 1] = h.coff[l][node + 1];
      --l;
    }
    if (!ids) cnt[c] = n;
  }
}

// One thread per polygon: its box covers top cells [cx0..cx1] x [cy0..cy1].
__global__ void k_top_raster(const int4* __restrict__ box, int64_t n_poly, Grid g,
                             uint32_t* __restrict__ cnt, const uint64_t* __restrict__ off,
                             uint32_t* __restrict__ cur, int32_t* __restrict__ ids) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_poly;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int4 b = box[p];
    if (b.x > b.z) continue;
    const long long cx0 = ((long long)b.x - g.gx0) >> g.s0, cx1 = ((long long)b.z - g.gx0) >> g.s0;
    const long long cy0 = ((long long)b.y - g.gy0) >> g.s0, cy1 = ((long long)b.w - g.gy0) >> g.s0;
    for (long long cy = cy0; cy <= cy1; ++cy)
      for (long long cx = cx0; cx <= cx1; ++cx) {
        const int64_t c = cy * g.nx + cx;
        if (!ids) {
          atomicAdd(cnt + c, 1u);
        } else {
          const uint32_t k = atomicAdd(cur + c, 1u);
          ids[off[c] + k] = (int32_t)p;
        }
      }
  }
}

// Sort each cell's candidate ids ascending (lists are short).
__global__ void k_sort_segments(const uint64_t* __restrict__ off, int64_t n_seg,
                                int32_t* __restrict__ ids) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n_seg;
       s += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t a = off[s], b = off[s + 1];
    for (uint64_t i = a + 1; i < b; ++i) {
      const int32_t v = ids[i];
      uint64_t j = i;
      while (j > a && ids[j - 1] > v) {
        ids[j] = ids[j - 1];
        --j;
      }
      ids[j] = v;
    }
  }
}

// ----------------------------------------------------------------- frontier
// One level of cells being classified. Candidate c of the frontier belongs
// to cell cd_cell[c]; its edges come either from polygon cd_poly[c]'s rings
// (level 0) or from the parent's kept edges [cd_src[c], cd_src[c] + cd_srcn[c]).
struct Level {
  int shift;  // log2 cell side at this level
};

__device__ __forceinline__ void cell_rect(const Grid& g, int shift, uint32_t cx, uint32_t cy,
                                          long long& x0, long long& y0, long long& x1,
                                          long long& y1) {
  x0 = g.gx0 + ((long long)cx << shift);
  y0 = g.gy0 + ((long long)cy << shift);
  x1 = x0 + (1ll << shift);
  y1 = y0 + (1ll << shift);
}

// Does the segment a-b meet the closed rectangle [x0, x1m] x [y0, y1m]?
// Separating-axis test: the box axes (coordinate overlap) and the segment's
// normal (all four corners strictly on one side), in exact 128-bit integers.
__device__ __forceinline__ bool seg_meets_rect(long long ax, long long ay, long long bx, long long by,
                                               long long x0, long long y0, long long x1m,
                                               long long y1m) {
  if (max(ax, bx) < x0 || min(ax, bx) > x1m || max(ay, by) < y0 || min(ay, by) > y1m) return false;
  const __int128 dx = bx - ax, dy = by - ay;
  int pos = 0, neg = 0;
  const long long cx[4] = {x0, x1m, x0, x1m}, cy[4] = {y0, y0, y1m, y1m};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __int128 v = dx * (__int128)(cy[i] - ay) - dy * (__int128)(cx[i] - ax);
    pos += v > 0;
    neg += v < 0;
  }
  return !(pos == 4 || neg == 4);
}

// Crossing rule of one normalised edge (ay < by) for the point (px, py).
__device__ __forceinline__ uint32_t crosses_ll(int4 e, long long px, long long py) {
  if (py < e.y || py >= e.w) return 0;
  if (px >= (long long)max(e.x, e.z)) return 0;
  if (px < (long long)min(e.x, e.z)) return 1;
  const __int128 l = (__int128)(e.z - e.x) * (__int128)(py - e.y);
  const __int128 r = (__int128)(e.w - e.y) * (__int128)(px - e.x);
  return l > r ? 1u : 0u;
}

// 0 drop, 1 fold, 2 keep; the edge is normalised so that ay < by.
__device__ __forceinline__ int clip_edge(int ax, int ay, int bx, int by, long long x0, long long y0,
                                         long long x1, long long y1, int4& out) {
  if (ay == by) return 0;
  if (ay > by) {
    int t = ax; ax = bx; bx = t;
    t = ay; ay = by; by = t;
  }
  if ((long long)by <= y0 || (long long)ay >= y1) return 0;      // y-span misses the row
  if ((long long)max(ax, bx) <= x0) return 0;                   // wholly at or left
  if ((long long)min(ax, bx) >= x1 && (long long)ay <= y0 && (long long)by >= y1) return 1;  // fold
  out = make_int4(ax, ay, bx, by);
  return 2;
}

// Count (emit == nullptr) or emit the kept edges of each frontier candidate,
// and compute its base parity. When no edge of the candidate meets the
// cell's closed lattice rectangle, its parity is the same at every lattice
// point of the cell: two lattice segments that do not meet are at least
// 1/(sqrt(2) W) apart, more than the infinitesimal shift that settles ties,
// so no edge separates two points of the cell. The candidate then keeps no
// edge and its base becomes that constant, taken at the lower-left point.
template <bool FROM_POLY>
__global__ void k_clip(Grid g, int shift, int64_t n_cand, const uint32_t* __restrict__ cd_cell,
                       const uint32_t* __restrict__ fc_x, const uint32_t* __restrict__ fc_y,
                       const int32_t* __restrict__ cd_poly, const uint64_t* __restrict__ cd_src,
                       const uint32_t* __restrict__ cd_srcn, const int4* __restrict__ src_edges,
                       const int32_t* __restrict__ vx, const int32_t* __restrict__ vy,
                       const int64_t* __restrict__ ring_off, const int64_t* __restrict__ pro,
                       uint32_t* __restrict__ cd_kept, uint8_t* __restrict__ cd_base,
                       const uint64_t* __restrict__ emit_off, int4* __restrict__ emit) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cand;
       c += (int64_t)gridDim.x * blockDim.x) {
    if (emit && emit_off[c] == emit_off[c + 1]) continue;
    long long x0, y0, x1, y1;
    const uint32_t cell = cd_cell[c];
    cell_rect(g, shift, fc_x[cell], fc_y[cell], x0, y0, x1, y1);
    uint32_t kept = 0, fold = 0, at_corner = 0;
    bool touch = false;
    uint64_t w = emit ? emit_off[c] : 0;
    int4 e;
    auto visit = [&](int ax, int ay, int bx, int by) {
      const bool meets = seg_meets_rect(ax, ay, bx, by, x0, y0, x1 - 1, y1 - 1);
      touch |= meets;
      int k;
      if (ay == by) {
        // a horizontal edge never counts, but one that crosses the cell
        // separates inside from outside: keep it so sub-cells see it
        k = meets ? 2 : 0;
        e = make_int4(ax, ay, bx, by);
      } else {
        k = clip_edge(ax, ay, bx, by, x0, y0, x1, y1, e);
      }
      fold ^= (k == 1);
      if (k == 2) {
        if (emit) emit[w++] = e;
        at_corner ^= crosses_ll(e, x0, y0);
        ++kept;
      }
    };
    if (FROM_POLY) {
      const int32_t p = cd_poly[c];
      for (int64_t r = pro[p]; r < pro[p + 1]; ++r) {
        const int64_t a = ring_off[r], b = ring_off[r + 1];
        for (int64_t i = a; i < b; ++i) {
          const int64_t j = (i + 1 == b) ? a : i + 1;
          visit(vx[i], vy[i], vx[j], vy[j]);
        }
      }
    } else {
      const uint64_t a = cd_src[c], b = a + cd_srcn[c];
      for (uint64_t i = a; i < b; ++i) {
        const int4 s = src_edges[i];
        visit(s.x, s.y, s.z, s.w);
      }
    }
    if (!emit) {
      if (!touch) {
        cd_kept[c] = 0;
        cd_base[c] ^= (uint8_t)(fold ^ at_corner);
      } else {
        cd_kept[c] = kept;
        cd_base[c] ^= (uint8_t)fold;
      }
    }
  }
}

// Cell classification (thread per frontier cell). Writes the descriptor of
// EMPTY / INTERIOR cells, and for boundary cells the number of kept
// candidates and edges, the keep flag of each candidate and split / leaf.
__global__ void k_classify(int64_t n_cell, const uint64_t* __restrict__ fc_coff,
                           const int32_t* __restrict__ cd_poly, const uint32_t* __restrict__ cd_kept,
                           const uint8_t* __restrict__ cd_base, uint8_t* __restrict__ cd_keep,
                           const int4* __restrict__ poly_box, const uint32_t* __restrict__ fc_slot,
                           uint32_t* __restrict__ desc, uint32_t* __restrict__ fc_nk,
                           uint32_t* __restrict__ fc_ne, uint32_t* __restrict__ fc_leaf,
                           uint32_t* __restrict__ fc_split, int32_t* __restrict__ fc_val, int shift,
                           int can_split, uint32_t leaf_edges, int size_ratio, long long approx,
                           int compact_early, unsigned long long* counters) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cell;
       c += (int64_t)gridDim.x * blockDim.x) {
    uint32_t nk = 0, ne = 0, first = 0xFFFFFFFFu;
    bool first_full = false;
    long long min_ext = LLONG_MAX;
    for (uint64_t i = fc_coff[c]; i < fc_coff[c + 1]; ++i) {
      const uint32_t k = cd_kept[i];
      const uint8_t b = cd_base[i];
      const bool keep = (k > 0) || b;
      cd_keep[i] = keep;
      if (!keep) continue;
      if (nk == 0) {
        first = (uint32_t)i;
        first_full = (k == 0);
      }
      ++nk;
      ne += k;
      if (k > 0) {
        const int4 bx = poly_box[cd_poly[i]];
        const long long ext = max((long long)bx.z - bx.x, (long long)bx.w - bx.y);
        min_ext = min(min_ext, ext);
      }
      if (k == 0) {  // inside everywhere: higher ids never win in this cell
        for (uint64_t j = i + 1; j < fc_coff[c + 1]; ++j) cd_keep[j] = 0;
        break;
      }
    }
    uint32_t leaf = 0, split = 0;
    int32_t val = 0;
    if (nk == 0) {  // EMPTY
      if (desc) desc[fc_slot[c]] = make_desc(TAG_EMPTY, 0);
      atomicAdd(counters + 0, 1ull);
      val = -1;
      ne = 0;
    } else if (nk == 1 && first_full) {  // INTERIOR (keeps its one full candidate)
      if (desc) desc[fc_slot[c]] = make_desc(TAG_INTERIOR, (uint32_t)cd_poly[first]);
      atomicAdd(counters + 1, 1ull);
      val = cd_poly[first];
      ne = 0;
    } else {
      const long long side = 1ll << shift;
      // compact_early: every boundary cell splits until it is compact
      // (decided once its edges are known) or the deepest level is reached
      const bool want = compact_early || ne > leaf_edges || (size_ratio > 0 && side * size_ratio > min_ext) ||
                        (approx > 0 && side > approx);
      if (can_split && want) {
        split = 1;
      } else {
        leaf = 1;
      }
    }
    fc_nk[c] = nk;
    fc_ne[c] = ne;
    fc_leaf[c] = leaf;
    fc_split[c] = split;
    fc_val[c] = val;
  }
}

// Children of one split cell (frontier cells p*16 .. p*16+15): give each
// EMPTY / INTERIOR child a 2-bit code into the node's 4-entry palette. A
// child whose value does not fit the palette becomes a leaf instead (its
// one full candidate, or none, then answers through the crossing test), or,
// with compact leaves, a one-slot compact record holding that value
// (fcomp = 1 | COMP_CONST). Parent p's node is nodes[node_slot[p]].
constexpr uint32_t COMP_CONST = 0x100u;

__global__ void k_palette(int64_t n_parent, uint32_t* __restrict__ fc_leaf,
                          const uint32_t* __restrict__ fc_split, uint32_t* __restrict__ fc_comp,
                          const int32_t* __restrict__ fc_val, const uint32_t* __restrict__ node_slot,
                          TrieNode* __restrict__ nodes, unsigned long long* counters) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_parent;
       p += (int64_t)gridDim.x * blockDim.x) {
    uint32_t codes = 0;
    int32_t pal[4] = {-1, -1, -1, -1};
    int np = 0;
    for (int sub = 0; sub < NODE_FAN; ++sub) {
      const int64_t c = p * NODE_FAN + sub;
      if (fc_leaf[c] || fc_split[c] || (fc_comp && fc_comp[c])) continue;
      const int32_t v = fc_val[c];
      int j = 0;
      while (j < np && pal[j] != v) ++j;
      if (j == np) {
        if (np == 4) {
          if (fc_comp) fc_comp[c] = 1u | COMP_CONST;
          else fc_leaf[c] = 1;
          atomicAdd(counters + 2, 1ull);
          continue;
        }
        pal[np++] = v;
      }
      codes |= (uint32_t)j << (2 * sub);
    }
    TrieNode& nd = nodes[node_slot[p]];
    nd.codes = codes;
    for (int j = 0; j < 4; ++j) nd.pal[j] = pal[j];
  }
}

// Leaf / split masks and rank bases of each node (after the ranks exist).
// Compact children set both bits and add (slots - 1) as their code; split
// and compact children are numbered together from child_base (the first
// one's global slot), compact ones taking their record's slots.
__global__ void k_node_finish(int64_t n_parent, const uint32_t* __restrict__ fc_leaf,
                              const uint32_t* __restrict__ fc_split, const uint32_t* __restrict__ fc_comp,
                              const uint64_t* __restrict__ leaf_rank,
                              const uint64_t* __restrict__ slot_rank, uint32_t slot_base,
                              uint64_t level_base, const uint32_t* __restrict__ node_slot,
                              TrieNode* __restrict__ nodes) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_parent;
       p += (int64_t)gridDim.x * blockDim.x) {
    uint32_t lm = 0, cm = 0, ccodes = 0;
    int64_t first_leaf = -1, first_child = -1;
    for (int sub = 0; sub < NODE_FAN; ++sub) {
      const int64_t c = p * NODE_FAN + sub;
      const uint32_t comp = fc_comp ? (fc_comp[c] & 0xFFu) : 0u;
      if (fc_leaf[c]) {
        lm |= 1u << sub;
        if (first_leaf < 0) first_leaf = c;
      } else if (fc_split[c] || comp) {
        cm |= 1u << sub;
        if (comp) {
          lm |= 1u << sub;
          ccodes |= (comp - 1u) << (2 * sub);
        }
        if (first_child < 0) first_child = c;
      }
    }
    TrieNode& nd = nodes[node_slot[p]];
    nd.masks = lm | (cm << 16);
    nd.codes |= ccodes;
    nd.leaf_base = first_leaf >= 0 ? slot_base + (uint32_t)leaf_rank[first_leaf] : 0u;
    nd.child_base = first_child >= 0 ? (uint32_t)(level_base + slot_rank[first_child]) : 0u;
  }
}

// ---- 16-byte entries (an index without compact leaves) -------------------
// Codes of a 32-byte node's children in the 16-byte form. Of the polygons
// its EMPTY / INTERIOR children name, the two that most children name take
// codes 0 and 1 (a, b); empty children take code 2; split and leaf
// children, and children naming any other polygon, descend (code 3) to an
// entry of their own.
__device__ __forceinline__ void e16_codes(const TrieNode& nd, uint32_t& codes, int32_t& a, int32_t& b) {
  const uint32_t lm = nd.masks & 0xFFFFu, cm = nd.masks >> 16;
  int cnt[4] = {0, 0, 0, 0};
  for (int sub = 0; sub < NODE_FAN; ++sub)
    if (!((lm | cm) >> sub & 1u)) ++cnt[(nd.codes >> (2 * sub)) & 3u];
  int ia = -1, ib = -1;  // palette entries taking codes 0 and 1
  for (int j = 0; j < 4; ++j) {
    if (cnt[j] == 0 || nd.pal[j] < 0) continue;
    if (ia < 0 || cnt[j] > cnt[ia]) {
      ib = ia;
      ia = j;
    } else if (ib < 0 || cnt[j] > cnt[ib]) {
      ib = j;
    }
  }
  a = ia >= 0 ? nd.pal[ia] : -1;
  b = ib >= 0 ? nd.pal[ib] : -1;
  codes = 0;
  for (int sub = 0; sub < NODE_FAN; ++sub) {
    uint32_t c = E16_DESCEND;
    if (!((lm | cm) >> sub & 1u)) {
      const int j = (int)((nd.codes >> (2 * sub)) & 3u);
      c = nd.pal[j] < 0 ? E16_EMPTY : j == ia ? 0u : j == ib ? 1u : E16_DESCEND;
    }
    codes |= c << (2 * sub);
  }
}

__device__ __forceinline__ uint32_t e16_ndesc(uint32_t codes) {
  return __popc(codes & (codes >> 1) & 0x55555555u);
}

__device__ __forceinline__ uint4 e16_node(const TrieNode& nd, uint64_t base) {
  uint32_t codes;
  int32_t a, b;
  e16_codes(nd, codes, a, b);
  return make_uint4(codes, (uint32_t)base | (E16_NODE << 30), (uint32_t)a, (uint32_t)b);
}

// Descending children of each node.
__global__ void k_e16_count(int64_t n, const TrieNode* __restrict__ old, uint32_t* __restrict__ n_desc) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t codes;
    int32_t a, b;
    e16_codes(old[i], codes, a, b);
    n_desc[i] = e16_ndesc(codes);
  }
}

// Level-1 entries keep their nodes' indices (the top grid names them).
// rel: each node's first descending child, relative to the next level.
__global__ void k_e16_first(int64_t n1, const TrieNode* __restrict__ old, const uint64_t* __restrict__ rel,
                            uint64_t next_start, uint4* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n1; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = e16_node(old[i], next_start + rel[i]);
}

// The entries of the descending children of nodes [lo, lo + n) (one level):
// a split child's node, a leaf child's slot, or the polygon of a child
// outside its parent's two codes.
__global__ void k_e16_children(int64_t lo, int64_t n, const TrieNode* __restrict__ old,
                               const uint64_t* __restrict__ rel, uint64_t next_start, uint64_t next2_start,
                               uint4* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = lo + i;
    const TrieNode nd = old[p];
    uint32_t codes;
    int32_t a, b;
    e16_codes(nd, codes, a, b);
    const uint32_t lm = nd.masks & 0xFFFFu, cm = nd.masks >> 16;
    uint64_t e = next_start + rel[p];
    for (int sub = 0; sub < NODE_FAN; ++sub) {
      if (((codes >> (2 * sub)) & 3u) != E16_DESCEND) continue;
      const uint32_t bit = 1u << sub, below = bit - 1u;
      uint4 v;
      if (cm & bit) {
        const uint32_t oc = nd.child_base + __popc(cm & below);
        v = e16_node(old[oc], next2_start + rel[oc]);
      } else if (lm & bit) {
        v = make_uint4(nd.leaf_base + __popc(lm & below), E16_LEAF << 30, 0u, 0u);
      } else {
        v = make_uint4((uint32_t)nd.pal[(nd.codes >> (2 * sub)) & 3u], E16_ID << 30, 0u, 0u);
      }
      out[e++] = v;
    }
  }
}

__global__ void k_eff_nk(int64_t n, const uint32_t* __restrict__ fc_nk, const uint32_t* __restrict__ fc_leaf,
                         const uint32_t* __restrict__ fc_split, uint32_t* __restrict__ out) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x)
    out[c] = (fc_leaf[c] | fc_split[c]) ? fc_nk[c] : 0u;
}

// Boundary cells (leaf or split so far): compact their kept candidates
// (poly, base, kept count, source) in cell order.
__global__ void k_boundary_kc(int64_t n_cell, const uint64_t* __restrict__ fc_coff,
                              const uint8_t* __restrict__ cd_keep, const int32_t* __restrict__ cd_poly,
                              const uint8_t* __restrict__ cd_base, const uint32_t* __restrict__ cd_kept,
                              const uint64_t* __restrict__ cd_src, const uint32_t* __restrict__ cd_srcn,
                              const uint32_t* __restrict__ fc_leaf, const uint32_t* __restrict__ fc_split,
                              const uint64_t* __restrict__ kc_off, int32_t* __restrict__ kc_poly,
                              uint8_t* __restrict__ kc_base, uint32_t* __restrict__ kc_cnt,
                              uint64_t* __restrict__ kc_src, uint32_t* __restrict__ kc_srcn,
                              uint32_t* __restrict__ kc_cell) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cell;
       c += (int64_t)gridDim.x * blockDim.x) {
    if (!fc_leaf[c] && !fc_split[c]) continue;
    uint64_t w = kc_off[c];
    for (uint64_t i = fc_coff[c]; i < fc_coff[c + 1]; ++i) {
      if (!cd_keep[i]) continue;
      kc_poly[w] = cd_poly[i];
      kc_base[w] = cd_base[i];
      kc_cnt[w] = cd_kept[i];
      kc_src[w] = cd_src ? cd_src[i] : 0;
      kc_srcn[w] = cd_srcn ? cd_srcn[i] : 0;
      kc_cell[w] = (uint32_t)c;
      ++w;
    }
  }
}

// Descriptors of this level's boundary cells (top level only: deeper levels
// are described by their parents' nodes) and leaf -> cell for the blobs.
__global__ void k_boundary_desc(int64_t n_cell, const uint32_t* __restrict__ fc_slot,
                                const uint32_t* __restrict__ fc_leaf, const uint32_t* __restrict__ fc_split,
                                const uint32_t* __restrict__ fc_comp, const uint64_t* __restrict__ leaf_rank,
                                const uint64_t* __restrict__ slot_rank, uint32_t* __restrict__ desc,
                                uint32_t slot_base, uint64_t level_base, uint32_t* __restrict__ leaf_cell) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cell;
       c += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t comp = fc_comp ? (fc_comp[c] & 0xFFu) : 0u;
    if (fc_leaf[c]) {
      const uint64_t r = leaf_rank[c];
      if (desc) desc[fc_slot[c]] = make_desc(TAG_LEAF, slot_base + (uint32_t)r);
      leaf_cell[r] = (uint32_t)c;
    } else if (desc && fc_split[c]) {
      desc[fc_slot[c]] = make_desc(TAG_CHILD, (uint32_t)(level_base + slot_rank[c]));
    } else if (desc && comp) {
      desc[fc_slot[c]] = make_desc(TAG_CHILD, DESC_COMPACT | ((comp - 1u) << DESC_SLOTS_SHIFT) |
                                                  (uint32_t)(level_base + slot_rank[c]));
    }
  }
}

// Distinct non-horizontal kept edges of a boundary cell and each kept
// candidate's mask over them (horizontal edges never count, so they drop
// out). Candidates that are never inside (mask 0, base 0) are skipped, and
// one that is inside everywhere (mask 0, base 1) ends the list. Returns
// false when the cell does not fit a compact record (more than max_edges
// edges, more than COMPACT_MAX_CANDS candidates, or an id above 24 bits).
__device__ bool compact_gather(uint64_t k0, uint64_t k1, const int32_t* __restrict__ kc_poly,
                               const uint8_t* __restrict__ kc_base, const uint32_t* __restrict__ kc_cnt,
                               const uint64_t* __restrict__ kc_eoff, const int4* __restrict__ kedges,
                               int max_edges, int4 (&edge)[COMPACT_MAX_EDGES], uint32_t& ne,
                               uint32_t (&cand)[COMPACT_MAX_CANDS], uint32_t& nc) {
  ne = 0;
  nc = 0;
  for (uint64_t i = k0; i < k1; ++i) {
    uint32_t mask = 0;
    for (uint64_t e = kc_eoff[i]; e < kc_eoff[i] + kc_cnt[i]; ++e) {
      const int4 v = kedges[e];
      if (v.y == v.w) continue;
      uint32_t k = 0;
      while (k < ne && !(edge[k].x == v.x && edge[k].y == v.y && edge[k].z == v.z && edge[k].w == v.w)) ++k;
      if (k == ne) {
        if ((int)ne >= max_edges) return false;
        edge[ne++] = v;
      }
      mask ^= 1u << k;
    }
    const uint32_t base = kc_base[i] & 1u;
    if (mask == 0u && !base) continue;
    if (nc >= (uint32_t)COMPACT_MAX_CANDS || (uint32_t)kc_poly[i] > CAND_ID_MASK) return false;
    cand[nc++] = (uint32_t)kc_poly[i] | (mask << 24) | (base << 31);
    if (mask == 0u) break;
  }
  return true;
}

// Which boundary cells become compact leaves: fc_comp = record slots (0 =
// not compact); a compact cell is no longer a leaf or split. Without
// `early` only leaves are considered (the trie keeps its shape and compact
// records replace residual leaves); with it, a cell that would split stops
// as soon as it fits a record.
__global__ void k_compact_check(int64_t n_cell, int early, uint32_t* __restrict__ fc_leaf,
                                uint32_t* __restrict__ fc_split,
                                const uint64_t* __restrict__ kc_off, const int32_t* __restrict__ kc_poly,
                                const uint8_t* __restrict__ kc_base, const uint32_t* __restrict__ kc_cnt,
                                const uint64_t* __restrict__ kc_eoff, const int4* __restrict__ kedges,
                                int max_edges, uint32_t* __restrict__ fc_comp,
                                unsigned long long* counters) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cell;
       c += (int64_t)gridDim.x * blockDim.x) {
    fc_comp[c] = 0;
    if (!fc_leaf[c] && !(early && fc_split[c])) continue;
    int4 edge[COMPACT_MAX_EDGES];
    uint32_t cand[COMPACT_MAX_CANDS];
    uint32_t ne = 0, nc = 0;
    if (!compact_gather(kc_off[c], kc_off[c + 1], kc_poly, kc_base, kc_cnt, kc_eoff, kedges, max_edges,
                        edge, ne, cand, nc))
      continue;
    const uint32_t slots = compact_slots_for(ne);
    fc_comp[c] = slots;
    fc_leaf[c] = 0;
    fc_split[c] = 0;
    atomicAdd(counters + 3, 1ull);
    atomicAdd(counters + 4, (unsigned long long)slots);
    atomicAdd(counters + 5 + ne, 1ull);
  }
}

// Slots a frontier cell takes in its level's node array: a split cell one
// (its trie node), a compact cell its record's slots.
__global__ void k_slot_size(int64_t n_cell, const uint32_t* __restrict__ fc_split,
                            const uint32_t* __restrict__ fc_comp, uint32_t* __restrict__ out) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cell;
       c += (int64_t)gridDim.x * blockDim.x)
    out[c] = fc_split[c] ? 1u : (fc_comp ? (fc_comp[c] & 0xFFu) : 0u);
}

// Write the compact records of this level (level array `rec`, local slots).
__global__ void k_compact_fill(int64_t n_cell, const uint32_t* __restrict__ fc_comp,
                               const int32_t* __restrict__ fc_val, const uint64_t* __restrict__ slot_rank,
                               const uint64_t* __restrict__ kc_off, const int32_t* __restrict__ kc_poly,
                               const uint8_t* __restrict__ kc_base, const uint32_t* __restrict__ kc_cnt,
                               const uint64_t* __restrict__ kc_eoff, const int4* __restrict__ kedges,
                               int max_edges, uint32_t* __restrict__ rec) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cell;
       c += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t comp = fc_comp[c];
    if (!comp) continue;
    int4 edge[COMPACT_MAX_EDGES];
    uint32_t cand[COMPACT_MAX_CANDS];
    uint32_t ne = 0, nc = 0;
    if (comp & COMP_CONST) {  // a constant child that did not fit its parent's palette
      const int32_t v = fc_val[c];
      if (v >= 0) cand[nc++] = (uint32_t)v | (1u << 31);
    } else {
      compact_gather(kc_off[c], kc_off[c + 1], kc_poly, kc_base, kc_cnt, kc_eoff, kedges, max_edges, edge,
                     ne, cand, nc);
    }
    uint32_t* w = rec + 8 * slot_rank[c];
    const uint32_t nw = 8u * (comp & 0xFFu);
    for (uint32_t k = 0; k < nw; ++k) w[k] = 0u;
    w[0] = ne | (nc << 3);
    for (uint32_t i = 0; i < nc; ++i) w[1 + i] = cand[i];
    for (uint32_t k = 0; k < ne; ++k) {
      uint32_t* e = w + 4 + 4 * k;
      e[0] = (uint32_t)edge[k].x;
      e[1] = (uint32_t)edge[k].y;
      e[2] = (uint32_t)edge[k].z;
      e[3] = (uint32_t)edge[k].w;
    }
  }
}

// Children of split cells: count (ids == nullptr) or fill their candidates.
__global__ void k_children(int64_t n_child, int k, Grid g, int child_shift,
                           const uint32_t* __restrict__ split_cells, const uint32_t* __restrict__ fc_x,
                           const uint32_t* __restrict__ fc_y, const uint64_t* __restrict__ kc_off,
                           const int32_t* __restrict__ kc_poly, const uint8_t* __restrict__ kc_base,
                           const uint32_t* __restrict__ kc_cnt, const uint64_t* __restrict__ kc_eoff,
                           const int4* __restrict__ poly_box, uint32_t* __restrict__ ccount,
                           const uint64_t* __restrict__ coff, uint32_t* __restrict__ nx_,
                           uint32_t* __restrict__ ny_, uint32_t* __restrict__ nslot,
                           uint32_t* __restrict__ ncell, int32_t* __restrict__ npoly,
                           uint8_t* __restrict__ nbase, uint64_t* __restrict__ nsrc,
                           uint32_t* __restrict__ nsrcn) {
  const int fan = 1 << (2 * k);
  for (int64_t ch = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ch < n_child;
       ch += (int64_t)gridDim.x * blockDim.x) {
    const int64_t si = ch / fan;
    const uint32_t sub = (uint32_t)(ch % fan);
    const uint32_t parent = split_cells[si];
    const uint32_t cx = (fc_x[parent] << k) | (sub & ((1u << k) - 1u));
    const uint32_t cy = (fc_y[parent] << k) | (sub >> k);
    long long x0, y0, x1, y1;
    cell_rect(g, child_shift, cx, cy, x0, y0, x1, y1);
    uint32_t n = 0;
    uint64_t w = coff ? coff[ch] : 0;
    for (uint64_t i = kc_off[parent]; i < kc_off[parent + 1]; ++i) {
      if (!box_meets(poly_box[kc_poly[i]], x0, y0, x1 - 1, y1 - 1)) continue;
      if (coff) {
        ncell[w] = (uint32_t)ch;
        npoly[w] = kc_poly[i];
        nbase[w] = kc_base[i];
        nsrc[w] = kc_eoff[i];
        nsrcn[w] = kc_cnt[i];
        ++w;
      }
      ++n;
    }
    if (!coff) {
      ccount[ch] = n;
    } else {
      nx_[ch] = cx;
      ny_[ch] = cy;
      nslot[ch] = (uint32_t)(si * fan + sub);
    }
  }
}

// Record size of every leaf slot of this level (16-byte units): header
// (nc, candidates, edge ends) padded to 16 bytes, then the edges; padding
// slots past the level's leaves get an empty one-unit record.
__global__ void k_rec_size(int64_t n_slots, int64_t n_leaf, const uint32_t* __restrict__ leaf_cell,
                           const uint32_t* __restrict__ fc_nk, const uint32_t* __restrict__ fc_ne,
                           uint64_t* __restrict__ size16) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_slots;
       t += (int64_t)gridDim.x * blockDim.x) {
    if (t >= n_leaf) {
      size16[t] = 1;
      continue;
    }
    const uint32_t c = leaf_cell[t];
    size16[t] = (1ull + 2ull * fc_nk[c] + 3ull) / 4ull + fc_ne[c];
  }
}

// Largest superbin (32 consecutive records) in 16-byte units, for reports.
__global__ void k_superbin_max(int64_t n_sb, const uint64_t* __restrict__ off16, unsigned long long* out) {
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n_sb;
       b += (int64_t)gridDim.x * blockDim.x)
    atomicMax(out, (unsigned long long)(off16[(b + 1) * SB_SLOTS] - off16[b * SB_SLOTS]));
}

// Fill the leaf records and the slots' global offsets (a thread per slot:
// records are short; the rare long one is copied by its thread alone).
__global__ void k_rec_fill(int64_t n_slots, int64_t n_leaf, const uint32_t* __restrict__ leaf_cell,
                           const uint64_t* __restrict__ kc_off, const int32_t* __restrict__ kc_poly,
                           const uint8_t* __restrict__ kc_base, const uint32_t* __restrict__ kc_cnt,
                           const uint64_t* __restrict__ kc_eoff, const int4* __restrict__ kedges,
                           const uint64_t* __restrict__ off16, uint4* __restrict__ blobs,
                           uint32_t* __restrict__ slot_off, uint64_t base16) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_slots;
       t += (int64_t)gridDim.x * blockDim.x) {
    uint4* rec = blobs + off16[t];
    uint32_t* w = (uint32_t*)rec;
    slot_off[t] = (uint32_t)(base16 + off16[t]);
    if (t >= n_leaf) {
      rec[0] = make_uint4(0u, 0u, 0u, 0u);
      continue;
    }
    const uint32_t c = leaf_cell[t];
    const uint64_t k0 = kc_off[c];
    const uint32_t nc = (uint32_t)(kc_off[c + 1] - k0);
    const uint32_t head = (1u + 2u * nc + 3u) / 4u;
    w[0] = nc;
    uint32_t e = 0;
    for (uint32_t i = 0; i < nc; ++i) {
      w[1 + i] = (uint32_t)kc_poly[k0 + i] | ((uint32_t)kc_base[k0 + i] << 31);
      e += kc_cnt[k0 + i];
      w[1 + nc + i] = e;
    }
    for (uint32_t k = 1 + 2 * nc; k < 4 * head; ++k) w[k] = 0u;
    int4* edges = (int4*)(rec + head);
    uint32_t at = 0;
    for (uint32_t i = 0; i < nc; ++i) {
      const uint32_t cnt = kc_cnt[k0 + i];
      const int4* src = kedges + kc_eoff[k0 + i];
      for (uint32_t q = 0; q < cnt; ++q) edges[at + q] = src[q];
      at += cnt;
    }
  }
}

__global__ void k_compact_nonempty(int64_t n, const uint32_t* __restrict__ cnt,
                                   const uint64_t* __restrict__ rank, const uint64_t* __restrict__ coff,
                                   Grid g, uint32_t* __restrict__ fx, uint32_t* __restrict__ fy,
                                   uint32_t* __restrict__ fslot, uint64_t* __restrict__ fcoff) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    if (!cnt[c]) continue;
    const uint64_t r = rank[c];
    fx[r] = (uint32_t)(c % g.nx);
    fy[r] = (uint32_t)(c / g.nx);
    fslot[r] = (uint32_t)c;
    fcoff[r] = coff[c];
  }
}

__global__ void k_nonzero(const uint32_t* __restrict__ in, int64_t n, uint32_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i] ? 1u : 0u;
}

__global__ void k_expand_cell(int64_t n_cell, const uint64_t* __restrict__ coff,
                              uint32_t* __restrict__ cd_cell) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cell;
       c += (int64_t)gridDim.x * blockDim.x)
    for (uint64_t i = coff[c]; i < coff[c + 1]; ++i) cd_cell[i] = (uint32_t)c;
}

__global__ void k_gather_u32(const uint32_t* __restrict__ flags, const uint64_t* __restrict__ rank,
                             int64_t n, uint32_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (flags[i]) out[rank[i]] = (uint32_t)i;
}

// Local node slot of each split cell (split cells in rank order).
__global__ void k_split_slot(int64_t n_split, const uint32_t* __restrict__ split_cells,
                             const uint64_t* __restrict__ slot_rank, uint32_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_split;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (uint32_t)slot_rank[split_cells[i]];
}

__global__ void k_add_u32(uint2* p, int64_t n, uint32_t add) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i].x += add;
}

template <class T>
pip_status d2h(T* h, const T* d, size_t n, cudaStream_t s) {
  PIP_CUDA(cudaMemcpyAsync(h, d, n * sizeof(T), cudaMemcpyDeviceToHost, s));
  PIP_CUDA(cudaStreamSynchronize(s));
  return PIP_OK;
}

#define CHECK(st)                       \
  do {                                  \
    pip_status _st = (st);              \
    if (_st != PIP_OK) return _st;      \
  } while (0)

#define ALLOC(buf, n)                                                       \
  do {                                                                      \
    if (!(buf).alloc(al, (size_t)(n) + 1, s))                               \
      return fail(PIP_ENOMEM, "index build: device allocation failed");     \
  } while (0)

// Convert the trie's 32-byte nodes (levels concatenated: node_len[i] nodes
// for the split cells of level i) to 16-byte entries. *done stays false,
// and the nodes stay, when the entries would not fit their 30-bit indices.
pip_status to_entries16(Alloc* al, DBuf<uint4>& nodes, const std::vector<int64_t>& node_len,
                        int64_t* n_entries, bool* done, cudaStream_t s) {
  *done = false;
  *n_entries = 0;
  const size_t L = node_len.size();
  int64_t n_nodes = 0;
  for (int64_t l : node_len) n_nodes += l;
  DBuf<uint4> out;
  if (n_nodes == 0) {
    ALLOC(out, 0);
    PIP_CUDA(cudaMemsetAsync(out.p, 0, sizeof(uint4), s));
    nodes = std::move(out);
    *done = true;
    return PIP_OK;
  }
  const TrieNode* old = reinterpret_cast<const TrieNode*>(nodes.p);
  DBuf<uint32_t> nd;
  DBuf<uint64_t> rel, tot;
  ALLOC(nd, n_nodes);
  ALLOC(rel, n_nodes);
  ALLOC(tot, L);
  k_e16_count<<<blocks_for(n_nodes), TB, 0, s>>>(n_nodes, old, nd.p);
  PIP_CUDA(cudaGetLastError());
  int64_t lo = 0;
  for (size_t i = 0; i < L; ++i) {  // each node's first descending child within the next level
    CHECK(scan_u32_to_u64(*al, nd.p + lo, rel.p + lo, node_len[i], tot.p + i, s));
    lo += node_len[i];
  }
  std::vector<uint64_t> desc(L);
  CHECK(d2h(desc.data(), tot.p, L, s));
  // entries of level i + 1 (i = 0: the level-1 nodes) start at start[i]
  std::vector<uint64_t> start(L + 2, 0);
  start[1] = (uint64_t)node_len[0];
  for (size_t i = 0; i < L; ++i) start[i + 2] = start[i + 1] + desc[i];
  const uint64_t total = start[L + 1];
  if (total >= (1ull << 30)) return PIP_OK;
  ALLOC(out, total);
  k_e16_first<<<blocks_for(node_len[0]), TB, 0, s>>>(node_len[0], old, rel.p, start[1], out.p);
  PIP_CUDA(cudaGetLastError());
  lo = 0;
  for (size_t i = 0; i < L; ++i) {
    if (node_len[i] > 0) {
      k_e16_children<<<blocks_for(node_len[i]), TB, 0, s>>>(lo, node_len[i], old, rel.p, start[i + 1],
                                                            start[i + 2], out.p);
      PIP_CUDA(cudaGetLastError());
    }
    lo += node_len[i];
  }
  PIP_CUDA(cudaStreamSynchronize(s));
  nodes = std::move(out);
  *n_entries = (int64_t)total;
  *done = true;
  return PIP_OK;
}

}  // namespace

// Approximate mode: the centre lattice point of each leaf cell of a level,
// by leaf slot (slots past the level's leaves are padding with no candidates).
__global__ void k_leaf_centers(int64_t n_leaf, const uint32_t* __restrict__ leaf_cell,
                               const uint32_t* __restrict__ fc_x, const uint32_t* __restrict__ fc_y,
                               Grid g, int shift, int2* __restrict__ centre) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_leaf;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t c = leaf_cell[i];
    long long x0, y0, x1, y1;
    cell_rect(g, shift, fc_x[c], fc_y[c], x0, y0, x1, y1);
    const long long h = (1ll << shift) >> 1;
    centre[i] = make_int2((int32_t)(x0 + h), (int32_t)(y0 + h));
  }
}

// Approximate mode: the exact id of each leaf's centre, from the leaf's own
// record (its kept edges decide every point of the cell, Sec. III-A test).
__global__ void k_leaf_answer(int64_t n_slots, const int2* __restrict__ centre,
                              const uint4* __restrict__ blobs, const uint32_t* __restrict__ slot_off,
                              int32_t* __restrict__ answer) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_slots;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int2 p = centre[t];
    answer[t] = test_point(leaf_rec(blobs + slot_off[t]), p.x, p.y);  // padding slots: no candidates, -1
  }
}

// Resolve automatic options for a set.
static void resolve_opts(const pip_build_opts& in, int64_t n_poly, long long w, long long h,
                         pip_build_opts& o, int n_levels) {
  o = in;
  if (o.cell_log2 <= 0) {
    const double area = (double)std::max(1ll, w) * (double)std::max(1ll, h);
    const double target = std::min(std::max(32.0 * (double)n_poly, 4096.0), (double)(1 << 24));
    int s = (int)std::lround(std::log2(std::sqrt(area / target)));
    const double cells_cap = (double)(1 << 24);
    while (s < 30 && area / std::ldexp(1.0, 2 * s) > cells_cap) ++s;
    o.cell_log2 = std::max(4, std::min(30, s));
  }
  o.fanout_log2 = NODE_K;  // trie nodes hold 4 x 4 children
  if (o.approx_units < 0) o.approx_units = 0;
  if (o.approx_units == 1) o.approx_units = 2;  // the finest cells are 1 or 2 units wide
  if (o.max_depth == 0) o.max_depth = std::max(0, std::min(8, (o.cell_log2 - 6) / o.fanout_log2));
  else if (o.max_depth < 0) o.max_depth = 0;  // uniform grid
  if (o.approx_units > 0) {  // leaves no wider than approx_units: enough levels for that
    int need = 0;
    while ((1ll << std::max(0, o.cell_log2 - o.fanout_log2 * need)) > o.approx_units) ++need;
    o.max_depth = std::max(o.max_depth, need);
  }
  o.max_depth = std::min(o.max_depth, std::max(0, (o.cell_log2 - (o.approx_units > 0 ? 0 : 1)) / o.fanout_log2));
  if (o.leaf_edges <= 0) o.leaf_edges = 8;
  // measured on the state workload: a deeper trie costs K1 little (it walks
  // levels in bulk) and saves more in the residual kernels (128: 1.63 ms a
  // step against 1.74 at 48 and 1.69 at 64). With compact leaves every leaf
  // becomes a record in the node array, and ratio 128 overflows its 2^27
  // slots on the state set; the approximate mode splits leaves further by
  // its own bound. In both the automatic ratio stays 48.
  const bool compact_asked = o.compact_edges > 0 && o.approx_units <= 0;
  if (o.size_ratio == 0) o.size_ratio = (compact_asked || o.approx_units > 0) ? 48 : 128;
  if (o.pts_per_cta <= 0) o.pts_per_cta = 256;
  if (o.stage_depth == 0) o.stage_depth = -1;  // measured best when chunks span many superbins
  if (o.stage_depth < 0) o.stage_depth = -1;  // no shared-memory staging
  if (o.stage_depth > 2) o.stage_depth = 2;
  if (o.cand_mode <= 0) o.cand_mode = n_levels > 0 ? 1 : 2;
  // compact leaves: off unless asked for (compact_edges 1..7); also off in
  // approximate mode (whose leaves answer without a test) and when ids do
  // not fit a compact candidate word
  if (o.compact_edges == 0) o.compact_edges = -1;  // measured slower on the state workload: off
  if (o.compact_edges > COMPACT_MAX_EDGES) o.compact_edges = COMPACT_MAX_EDGES;
  if (o.approx_units > 0 || n_poly > (int64_t)CAND_ID_MASK + 1) o.compact_edges = -1;
  o.compact_early = (o.compact_edges > 0 && o.compact_early > 0) ? 1 : 0;
  o.bin_residual = o.bin_residual > 0 ? 1 : o.bin_residual < 0 ? -1 : 0;
}

// Build the hierarchy arrays on the device.
struct HierBufs {
  std::vector<DBuf<int4>> box;
  std::vector<DBuf<uint64_t>> coff;
  std::vector<DBuf<int32_t>> cids;
};

static pip_status build_hierarchy(pip_set_s* S, Alloc* al, cudaStream_t s, HierBufs& hb, Hier& h,
                                  DBuf<uint32_t>& err) {
  const int L = (int)S->parent.size();
  h.levels = L;
  hb.box.resize(L + 1);
  hb.coff.resize(L + 1);
  hb.cids.resize(L + 1);
  h.len[0] = S->n_poly;
  h.box[0] = S->poly_box.p;
  for (int l = 1; l <= L; ++l) {
    const int64_t n_par = S->level_len[l], n_ch = S->level_len[l - 1];
    h.len[l] = n_par;
    ALLOC(hb.box[l], n_par);
    ALLOC(hb.coff[l], n_par + 1);
    ALLOC(hb.cids[l], n_ch);
    DBuf<uint32_t> cnt, cur;
    ALLOC(cnt, n_par);
    ALLOC(cur, n_par);
    PIP_CUDA(cudaMemsetAsync(cnt.p, 0, (n_par + 1) * sizeof(uint32_t), s));
    PIP_CUDA(cudaMemsetAsync(cur.p, 0, (n_par + 1) * sizeof(uint32_t), s));
    k_fill_int4<<<blocks_for(n_par), TB, 0, s>>>(hb.box[l].p, n_par,
                                                 make_int4(INT32_MAX, INT32_MAX, INT32_MIN, INT32_MIN));
    k_count_children<<<blocks_for(n_ch), TB, 0, s>>>(S->parent[l - 1].p, n_ch, cnt.p, n_par, err.p);
    CHECK(scan_u32_to_u64(*al, cnt.p, hb.coff[l].p, n_par + 1, nullptr, s));
    k_fill_children<<<blocks_for(n_ch), TB, 0, s>>>(S->parent[l - 1].p, n_ch, hb.coff[l].p, cur.p,
                                                    hb.cids[l].p, hb.box[l].p, h.box[l - 1], n_par);
    PIP_CUDA(cudaGetLastError());
    h.box[l] = hb.box[l].p;
    h.coff[l] = hb.coff[l].p;
    h.cids[l] = hb.cids[l].p;
  }
  for (int l = L + 1; l < MAX_LEVELS; ++l) {
    h.len[l] = 0;
    h.box[l] = nullptr;
    h.coff[l] = nullptr;
    h.cids[l] = nullptr;
  }
  return PIP_OK;
}

// Candidate lists of the top cells (sorted ascending per cell).
static pip_status top_candidates(pip_set_s* S, Alloc* al, cudaStream_t s, const Hier& h,
                                 const Grid& g, int mode, DBuf<uint32_t>& cnt,
                                 DBuf<uint64_t>& coff, DBuf<int32_t>& ids, uint64_t& total) {
  const int64_t cells = (int64_t)g.nx * g.ny;
  ALLOC(cnt, cells);
  ALLOC(coff, cells + 1);
  PIP_CUDA(cudaMemsetAsync(cnt.p, 0, (cells + 1) * sizeof(uint32_t), s));
  if (mode == 1) {
    k_top_hier<<<blocks_for(cells, 128), 128, 0, s>>>(h, g, cnt.p, nullptr, nullptr);
  } else {
    k_top_raster<<<blocks_for(S->n_poly), TB, 0, s>>>(S->poly_box.p, S->n_poly, g, cnt.p, nullptr,
                                                      nullptr, nullptr);
  }
  PIP_CUDA(cudaGetLastError());
  DBuf<uint64_t> tot;
  ALLOC(tot, 1);
  CHECK(scan_u32_to_u64(*al, cnt.p, coff.p, cells + 1, tot.p, s));
  CHECK(d2h(&total, tot.p, 1, s));
  if (total >= (1ull << 32)) return fail(PIP_ERANGE, "index build: too many top-cell candidates");
  ALLOC(ids, total);
  if (mode == 1) {
    k_top_hier<<<blocks_for(cells, 128), 128, 0, s>>>(h, g, nullptr, coff.p, ids.p);
  } else {
    DBuf<uint32_t> cur;
    ALLOC(cur, cells);
    PIP_CUDA(cudaMemsetAsync(cur.p, 0, (cells + 1) * sizeof(uint32_t), s));
    k_top_raster<<<blocks_for(S->n_poly), TB, 0, s>>>(S->poly_box.p, S->n_poly, g, cnt.p, coff.p,
                                                      cur.p, ids.p);
  }
  PIP_CUDA(cudaGetLastError());
  k_sort_segments<<<blocks_for(cells, 128), 128, 0, s>>>(coff.p, cells, ids.p);
  PIP_CUDA(cudaGetLastError());
  return PIP_OK;
}

pip_status build_grid(pip_set_s* S, Grid& g, pip_build_opts& o, Alloc* al, cudaStream_t s) {
  DBuf<int> u;
  ALLOC(u, 4);
  const int init[4] = {INT32_MAX, INT32_MAX, INT32_MIN, INT32_MIN};
  PIP_CUDA(cudaMemcpyAsync(u.p, init, sizeof(init), cudaMemcpyHostToDevice, s));
  k_union_box<<<blocks_for(S->n_poly), TB, 0, s>>>(S->poly_box.p, S->n_poly, u.p);
  PIP_CUDA(cudaGetLastError());
  int b[4];
  CHECK(d2h(b, u.p, 4, s));
  if (b[0] > b[2]) {  // no vertices at all: one empty cell
    b[0] = b[1] = 0;
    b[2] = b[3] = 0;
  }
  resolve_opts(S->opts, S->n_poly, (long long)b[2] - b[0] + 1, (long long)b[3] - b[1] + 1, o,
               (int)S->parent.size());
  g.gx0 = b[0];
  g.gy0 = b[1];
  g.s0 = o.cell_log2;
  const long long nx = (((long long)b[2] - b[0]) >> g.s0) + 1;
  const long long ny = (((long long)b[3] - b[1]) >> g.s0) + 1;
  if (nx * ny > (1ll << 30)) return fail(PIP_ERANGE, "index build: top grid too large; raise cell_log2");
  g.nx = (uint32_t)nx;
  g.ny = (uint32_t)ny;
  return PIP_OK;
}

static pip_status build_index_shape(pip_set_s* S, cudaStream_t s);

// Build the set's index. With the split ratio left automatic, a ratio whose
// trie or leaves outgrow their 27 / 30-bit indices (a large set with coarse
// top cells, e.g. 800,000 blocks at ratio 128) falls back to 48, then 16.
pip_status build_index(pip_set_s* S, cudaStream_t s) {
  if (S->opts.size_ratio != 0) return build_index_shape(S, s);
  pip_status st = PIP_OK;
  for (int fallback : {0, 48, 16}) {
    S->opts.size_ratio = fallback;
    st = build_index_shape(S, s);
    if (st != PIP_ERANGE) break;
  }
  if (st != PIP_OK) S->opts.size_ratio = 0;  // leave the caller's automatic choice in place
  return st;
}

static pip_status build_index_shape(pip_set_s* S, cudaStream_t s) {
  Alloc* al = &S->alloc;
  cudaEvent_t ev0, ev1;
  PIP_CUDA(cudaEventCreate(&ev0));
  PIP_CUDA(cudaEventCreate(&ev1));
  PIP_CUDA(cudaEventRecord(ev0, s));
  DBuf<uint32_t> err;
  ALLOC(err, 1);
  PIP_CUDA(cudaMemsetAsync(err.p, 0, 2 * sizeof(uint32_t), s));

  Grid g;
  pip_build_opts o;
  CHECK(build_grid(S, g, o, al, s));
  const int k = NODE_K;
  const int fan = NODE_FAN;
  HierBufs hb;
  Hier h;
  CHECK(build_hierarchy(S, al, s, hb, h, err));
  uint32_t herr = 0;
  CHECK(d2h(&herr, err.p, 1, s));
  if (herr) return fail(PIP_EINVAL, "index build: parent id out of range");

  const int64_t top_cells = (int64_t)g.nx * g.ny;
  DBuf<uint32_t> top_cnt;
  DBuf<uint64_t> top_coff;
  DBuf<int32_t> top_ids;
  uint64_t top_total = 0;
  CHECK(top_candidates(S, al, s, h, g, o.cand_mode, top_cnt, top_coff, top_ids, top_total));

  unsigned long long* counters = nullptr;  // [0] empty, [1] interior, [2] palette overflows
  DBuf<unsigned long long> cnt_buf;
  ALLOC(cnt_buf, 13);  // [3] compact cells [4] compact slots [5 + E] compact cells by edge count
  PIP_CUDA(cudaMemsetAsync(cnt_buf.p, 0, 14 * sizeof(unsigned long long), s));
  counters = cnt_buf.p;

  // per-level outputs
  std::vector<DBuf<uint32_t>> desc_lv;   // descriptors of this level's table part
  std::vector<int64_t> desc_len;
  std::vector<DBuf<uint4>> blob_lv;
  std::vector<DBuf<uint32_t>> sbd_lv;  // per level: the leaf slots' record offsets
  std::vector<DBuf<int2>> cen_lv;  // approximate mode: leaf centres per level
  std::vector<int64_t> blob_len, sb_len;
  std::vector<DBuf<TrieNode>> node_lv;  // nodes of each level's split cells
  std::vector<int64_t> node_len;
  int64_t table_total = top_cells;
  desc_lv.emplace_back();
  ALLOC(desc_lv[0], top_cells);
  PIP_CUDA(cudaMemsetAsync(desc_lv[0].p, 0, (top_cells + 1) * sizeof(uint32_t), s));
  desc_len.push_back(top_cells);

  // frontier 0: non-empty top cells
  DBuf<uint32_t> fx, fy, fslot, cd_cell, cd_srcn;
  DBuf<uint64_t> fcoff, cd_src;
  DBuf<int32_t> cd_poly;
  DBuf<uint8_t> cd_base;
  int64_t n_cell = 0, n_cand = (int64_t)top_total;
  {
    DBuf<uint32_t> nz;
    DBuf<uint64_t> rank, tot;
    ALLOC(nz, top_cells);
    ALLOC(rank, top_cells + 1);
    ALLOC(tot, 1);
    k_nonzero<<<blocks_for(top_cells), TB, 0, s>>>(top_cnt.p, top_cells, nz.p);
    CHECK(scan_u32_to_u64(*al, nz.p, rank.p, top_cells, tot.p, s));
    uint64_t t = 0;
    CHECK(d2h(&t, tot.p, 1, s));
    n_cell = (int64_t)t;
    ALLOC(fx, n_cell);
    ALLOC(fy, n_cell);
    ALLOC(fslot, n_cell);
    ALLOC(fcoff, n_cell + 1);
    k_compact_nonempty<<<blocks_for(top_cells), TB, 0, s>>>(top_cells, top_cnt.p, rank.p, top_coff.p, g,
                                                           fx.p, fy.p, fslot.p, fcoff.p);
    PIP_CUDA(cudaMemcpyAsync(fcoff.p + n_cell, &top_total, sizeof(uint64_t), cudaMemcpyHostToDevice, s));
    PIP_CUDA(cudaStreamSynchronize(s));
    ALLOC(cd_cell, n_cand);
    ALLOC(cd_base, n_cand);
    PIP_CUDA(cudaMemsetAsync(cd_base.p, 0, n_cand + 1, s));
    k_expand_cell<<<blocks_for(n_cell), TB, 0, s>>>(n_cell, fcoff.p, cd_cell.p);
    PIP_CUDA(cudaGetLastError());
    cd_poly = std::move(top_ids);  // candidates stay in cell order
  }
  top_cnt.release();
  top_coff.release();

  DBuf<int4> src_edges;         // parent's kept edges (level > 0)
  DBuf<uint32_t> split_slot_prev;  // node slot of each split cell of the previous level
  uint32_t slot_base = 0;
  int64_t sb_total = 0, blob_total16 = 0, max_blob16 = 0, leaf_cands = 0, leaf_edges = 0;
  int64_t level_base = 0;  // global node-array slot of this level's first entry
  int depth_used = 0;
  const bool compact = o.compact_edges > 0;
  for (int lv = 0; n_cell > 0; ++lv) {
    depth_used = lv;
    const int shift = g.s0 - lv * k;
    const bool can_split = lv < o.max_depth;
    // clip: count kept edges and base parity per candidate
    DBuf<uint32_t> cd_kept;
    DBuf<uint8_t> cd_keep;
    ALLOC(cd_kept, n_cand);
    ALLOC(cd_keep, n_cand);
    if (lv == 0) {
      k_clip<true><<<blocks_for(n_cand, 128), 128, 0, s>>>(
          g, shift, n_cand, cd_cell.p, fx.p, fy.p, cd_poly.p, nullptr, nullptr, nullptr, S->vx.p,
          S->vy.p, S->ring_off.p, S->poly_ring_off.p, cd_kept.p, cd_base.p, nullptr, nullptr);
    } else {
      k_clip<false><<<blocks_for(n_cand, 128), 128, 0, s>>>(
          g, shift, n_cand, cd_cell.p, fx.p, fy.p, cd_poly.p, cd_src.p, cd_srcn.p, src_edges.p,
          nullptr, nullptr, nullptr, nullptr, cd_kept.p, cd_base.p, nullptr, nullptr);
    }
    PIP_CUDA(cudaGetLastError());
    // classify
    DBuf<uint32_t> fnk, fne, fleaf, fsplit, fnk_eff, fcomp, fsize;
    DBuf<int32_t> fval;
    ALLOC(fnk, n_cell);
    ALLOC(fne, n_cell);
    ALLOC(fleaf, n_cell);
    ALLOC(fsplit, n_cell);
    ALLOC(fval, n_cell);
    ALLOC(fnk_eff, n_cell);
    ALLOC(fcomp, n_cell);
    ALLOC(fsize, n_cell);
    PIP_CUDA(cudaMemsetAsync(fcomp.p, 0, (n_cell + 1) * sizeof(uint32_t), s));
    k_classify<<<blocks_for(n_cell), TB, 0, s>>>(n_cell, fcoff.p, cd_poly.p, cd_kept.p, cd_base.p,
                                                 cd_keep.p, S->poly_box.p, fslot.p,
                                                 lv == 0 ? desc_lv[0].p : nullptr, fnk.p, fne.p, fleaf.p,
                                                 fsplit.p, fval.p, shift, can_split ? 1 : 0,
                                                 (uint32_t)o.leaf_edges, o.size_ratio,
                                                 (long long)o.approx_units, compact ? o.compact_early : 0,
                                                 counters);
    PIP_CUDA(cudaGetLastError());
    const int64_t n_parent = lv == 0 ? 0 : n_cell / fan;
    if (lv > 0 && !compact) {  // palettes of the parents' nodes (may turn children into leaves)
      k_palette<<<blocks_for(n_parent), TB, 0, s>>>(n_parent, fleaf.p, fsplit.p, nullptr, fval.p,
                                                    split_slot_prev.p, node_lv.back().p, counters);
      PIP_CUDA(cudaGetLastError());
    }
    k_eff_nk<<<blocks_for(n_cell), TB, 0, s>>>(n_cell, fnk.p, fleaf.p, fsplit.p, fnk_eff.p);
    PIP_CUDA(cudaGetLastError());
    // kept candidates of the boundary cells, in cell order
    DBuf<uint64_t> kc_off;
    int64_t n_kc = 0;
    ALLOC(kc_off, n_cell + 1);
    {
      DBuf<uint64_t> tot;
      ALLOC(tot, 1);
      PIP_CUDA(cudaMemsetAsync(fnk_eff.p + n_cell, 0, sizeof(uint32_t), s));
      CHECK(scan_u32_to_u64(*al, fnk_eff.p, kc_off.p, n_cell + 1, tot.p, s));
      uint64_t t = 0;
      CHECK(d2h(&t, tot.p, 1, s));
      n_kc = (int64_t)t;
    }
    DBuf<uint32_t> kc_cnt, kc_srcn, kc_cell;
    DBuf<int32_t> kc_poly;
    DBuf<uint8_t> kc_base;
    DBuf<uint64_t> kc_src, kc_eoff;
    ALLOC(kc_cnt, n_kc);
    ALLOC(kc_srcn, n_kc);
    ALLOC(kc_cell, n_kc);
    ALLOC(kc_poly, n_kc);
    ALLOC(kc_base, n_kc);
    ALLOC(kc_src, n_kc);
    ALLOC(kc_eoff, n_kc + 1);
    k_boundary_kc<<<blocks_for(n_cell), TB, 0, s>>>(
        n_cell, fcoff.p, cd_keep.p, cd_poly.p, cd_base.p, cd_kept.p, lv ? cd_src.p : nullptr,
        lv ? cd_srcn.p : nullptr, fleaf.p, fsplit.p, kc_off.p, kc_poly.p, kc_base.p, kc_cnt.p, kc_src.p,
        kc_srcn.p, kc_cell.p);
    PIP_CUDA(cudaGetLastError());
    // kept edges of every kept candidate
    uint64_t n_ke = 0;
    {
      DBuf<uint64_t> tot;
      ALLOC(tot, 1);
      PIP_CUDA(cudaMemsetAsync(kc_cnt.p + n_kc, 0, sizeof(uint32_t), s));
      CHECK(scan_u32_to_u64(*al, kc_cnt.p, kc_eoff.p, n_kc + 1, tot.p, s));
      CHECK(d2h(&n_ke, tot.p, 1, s));
    }
    DBuf<int4> kedges;
    ALLOC(kedges, n_ke);
    if (n_kc > 0) {
      // re-walk the sources of the kept candidates to emit their edges
      DBuf<uint8_t> dummy_base;
      ALLOC(dummy_base, n_kc);
      PIP_CUDA(cudaMemsetAsync(dummy_base.p, 0, n_kc + 1, s));
      if (lv == 0) {
        k_clip<true><<<blocks_for(n_kc, 128), 128, 0, s>>>(
            g, shift, n_kc, kc_cell.p, fx.p, fy.p, kc_poly.p, nullptr, nullptr, nullptr, S->vx.p,
            S->vy.p, S->ring_off.p, S->poly_ring_off.p, nullptr, dummy_base.p, kc_eoff.p, kedges.p);
      } else {
        k_clip<false><<<blocks_for(n_kc, 128), 128, 0, s>>>(
            g, shift, n_kc, kc_cell.p, fx.p, fy.p, kc_poly.p, kc_src.p, kc_srcn.p, src_edges.p,
            nullptr, nullptr, nullptr, nullptr, nullptr, dummy_base.p, kc_eoff.p, kedges.p);
      }
      PIP_CUDA(cudaGetLastError());
    }
    if (compact) {  // compact leaves, then the parents' palettes (overflows become compact too)
      k_compact_check<<<blocks_for(n_cell), TB, 0, s>>>(n_cell, o.compact_early, fleaf.p, fsplit.p, kc_off.p, kc_poly.p,
                                                        kc_base.p, kc_cnt.p, kc_eoff.p, kedges.p,
                                                        o.compact_edges, fcomp.p, counters);
      PIP_CUDA(cudaGetLastError());
      if (lv > 0) {
        k_palette<<<blocks_for(n_parent), TB, 0, s>>>(n_parent, fleaf.p, fsplit.p, fcomp.p, fval.p,
                                                      split_slot_prev.p, node_lv.back().p, counters);
        PIP_CUDA(cudaGetLastError());
      }
    }
    // ranks: leaf slots, split cells, node-array slots (split nodes + compact records)
    k_slot_size<<<blocks_for(n_cell), TB, 0, s>>>(n_cell, fsplit.p, compact ? fcomp.p : nullptr, fsize.p);
    PIP_CUDA(cudaGetLastError());
    DBuf<uint64_t> leaf_rank, split_rank, slot_rank, tots;
    ALLOC(leaf_rank, n_cell + 1);
    ALLOC(split_rank, n_cell + 1);
    ALLOC(slot_rank, n_cell + 1);
    ALLOC(tots, 3);
    CHECK(scan_u32_to_u64(*al, fleaf.p, leaf_rank.p, n_cell, tots.p + 0, s));
    CHECK(scan_u32_to_u64(*al, fsplit.p, split_rank.p, n_cell, tots.p + 1, s));
    CHECK(scan_u32_to_u64(*al, fsize.p, slot_rank.p, n_cell, tots.p + 2, s));
    uint64_t t3[3];
    CHECK(d2h(t3, tots.p, 3, s));
    const int64_t n_leaf = (int64_t)t3[0], n_split = (int64_t)t3[1], n_slots_lv = (int64_t)t3[2];
    if ((uint64_t)level_base + (uint64_t)n_slots_lv >= (uint64_t)SLOT_MASK ||
        (uint64_t)slot_base + (uint64_t)n_leaf + SB_SLOTS >= (1ull << 30))
      return fail(PIP_ERANGE, "index build: trie or leaves exceed their 27 / 30-bit indices; raise cell_log2");
    if (lv > 0) {  // masks and bases of the parents' nodes
      k_node_finish<<<blocks_for(n_parent), TB, 0, s>>>(n_parent, fleaf.p, fsplit.p,
                                                        compact ? fcomp.p : nullptr, leaf_rank.p,
                                                        slot_rank.p, slot_base, (uint64_t)level_base,
                                                        split_slot_prev.p, node_lv.back().p);
      PIP_CUDA(cudaGetLastError());
    }
    // top-level descriptors of boundary cells, leaf -> cell
    DBuf<uint32_t> leaf_cell;
    ALLOC(leaf_cell, n_leaf);
    k_boundary_desc<<<blocks_for(n_cell), TB, 0, s>>>(n_cell, fslot.p, fleaf.p, fsplit.p,
                                                      compact ? fcomp.p : nullptr, leaf_rank.p, slot_rank.p,
                                                      lv == 0 ? desc_lv[0].p : nullptr, slot_base,
                                                      (uint64_t)level_base, leaf_cell.p);
    PIP_CUDA(cudaGetLastError());
    // this level's node array: the split cells' nodes (filled while their
    // children are classified at the next level) and the compact records
    node_lv.emplace_back();
    ALLOC(node_lv.back(), n_slots_lv);
    PIP_CUDA(cudaMemsetAsync(node_lv.back().p, 0, (n_slots_lv + 1) * sizeof(TrieNode), s));
    node_len.push_back(n_slots_lv);
    if (compact && n_slots_lv > 0) {
      k_compact_fill<<<blocks_for(n_cell), TB, 0, s>>>(n_cell, fcomp.p, fval.p, slot_rank.p, kc_off.p,
                                                       kc_poly.p, kc_base.p, kc_cnt.p, kc_eoff.p, kedges.p,
                                                       o.compact_edges, (uint32_t*)node_lv.back().p);
      PIP_CUDA(cudaGetLastError());
    }
    // leaves of this level -> one record per slot (superbins of 32 slots)
    const int64_t n_sb = (n_leaf + SB_SLOTS - 1) / SB_SLOTS;
    if (n_sb > 0) {
      const int64_t n_slots_sb = n_sb * SB_SLOTS;
      DBuf<uint64_t> rsize, roff, tot;
      DBuf<unsigned long long> sbmax;
      ALLOC(rsize, n_slots_sb);
      ALLOC(roff, n_slots_sb + 1);
      ALLOC(tot, 1);
      ALLOC(sbmax, 1);
      k_rec_size<<<blocks_for(n_slots_sb), TB, 0, s>>>(n_slots_sb, n_leaf, leaf_cell.p, fnk.p, fne.p, rsize.p);
      PIP_CUDA(cudaMemsetAsync(rsize.p + n_slots_sb, 0, sizeof(uint64_t), s));
      CHECK(scan_u64(*al, rsize.p, roff.p, n_slots_sb + 1, tot.p, s));
      uint64_t total16 = 0;
      CHECK(d2h(&total16, tot.p, 1, s));
      if ((uint64_t)blob_total16 + total16 >= (1ull << 32))
        return fail(PIP_ERANGE, "index build: leaf data exceeds 64 GB");
      blob_lv.emplace_back();
      sbd_lv.emplace_back();
      ALLOC(blob_lv.back(), total16);
      ALLOC(sbd_lv.back(), n_slots_sb);
      k_rec_fill<<<blocks_for(n_slots_sb), TB, 0, s>>>(n_slots_sb, n_leaf, leaf_cell.p, kc_off.p, kc_poly.p,
                                                           kc_base.p, kc_cnt.p, kc_eoff.p, kedges.p, roff.p,
                                                           blob_lv.back().p, sbd_lv.back().p,
                                                           (uint64_t)blob_total16);
      PIP_CUDA(cudaGetLastError());
      // stats: largest superbin
      PIP_CUDA(cudaMemsetAsync(sbmax.p, 0, sizeof(unsigned long long), s));
      k_superbin_max<<<blocks_for(n_sb), TB, 0, s>>>(n_sb, roff.p, sbmax.p);
      PIP_CUDA(cudaGetLastError());
      unsigned long long hmax = 0;
      CHECK(d2h(&hmax, sbmax.p, 1, s));
      max_blob16 = std::max<int64_t>(max_blob16, (int64_t)hmax);
      if (o.approx_units > 0) {
        cen_lv.emplace_back();
        ALLOC(cen_lv.back(), n_sb * SB_SLOTS);
        PIP_CUDA(cudaMemsetAsync(cen_lv.back().p, 0, n_sb * SB_SLOTS * sizeof(int2), s));
        k_leaf_centers<<<blocks_for(n_leaf), TB, 0, s>>>(n_leaf, leaf_cell.p, fx.p, fy.p, g, shift,
                                                         cen_lv.back().p);
        PIP_CUDA(cudaGetLastError());
      }
      blob_len.push_back((int64_t)total16);
      sb_len.push_back(n_sb);
      blob_total16 += (int64_t)total16;
      sb_total += n_sb;
    }
    slot_base += (uint32_t)(n_sb * SB_SLOTS);
    // next frontier from split cells
    if (n_split == 0) {
      level_base += n_slots_lv;
      break;
    }
    const int64_t n_child = n_split * fan;
    DBuf<uint32_t> split_cells, split_slot;
    ALLOC(split_cells, n_split);
    ALLOC(split_slot, n_split);
    k_gather_u32<<<blocks_for(n_cell), TB, 0, s>>>(fsplit.p, split_rank.p, n_cell, split_cells.p);
    k_split_slot<<<blocks_for(n_split), TB, 0, s>>>(n_split, split_cells.p, slot_rank.p, split_slot.p);
    PIP_CUDA(cudaGetLastError());
    DBuf<uint32_t> ccount;
    DBuf<uint64_t> coff, tot;
    ALLOC(ccount, n_child);
    ALLOC(coff, n_child + 1);
    ALLOC(tot, 1);
    const int child_shift = shift - k;
    k_children<<<blocks_for(n_child), TB, 0, s>>>(
        n_child, k, g, child_shift, split_cells.p, fx.p, fy.p, kc_off.p, kc_poly.p, kc_base.p, kc_cnt.p,
        kc_eoff.p, S->poly_box.p, ccount.p, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
        nullptr, nullptr, nullptr);
    PIP_CUDA(cudaGetLastError());
    PIP_CUDA(cudaMemsetAsync(ccount.p + n_child, 0, sizeof(uint32_t), s));
    CHECK(scan_u32_to_u64(*al, ccount.p, coff.p, n_child + 1, tot.p, s));
    uint64_t n_cc = 0;
    CHECK(d2h(&n_cc, tot.p, 1, s));
    if (n_cc >= (1ull << 32)) return fail(PIP_ERANGE, "index build: too many child candidates");
    DBuf<uint32_t> nfx, nfy, nslot, ncell, nsrcn;
    DBuf<int32_t> npoly;
    DBuf<uint8_t> nbase;
    DBuf<uint64_t> nsrc;
    ALLOC(nfx, n_child);
    ALLOC(nfy, n_child);
    ALLOC(nslot, n_child);
    ALLOC(ncell, n_cc);
    ALLOC(nsrcn, n_cc);
    ALLOC(npoly, n_cc);
    ALLOC(nbase, n_cc);
    ALLOC(nsrc, n_cc);
    k_children<<<blocks_for(n_child), TB, 0, s>>>(
        n_child, k, g, child_shift, split_cells.p, fx.p, fy.p, kc_off.p, kc_poly.p, kc_base.p, kc_cnt.p,
        kc_eoff.p, S->poly_box.p, nullptr, coff.p, nfx.p, nfy.p, nslot.p, ncell.p, npoly.p, nbase.p,
        nsrc.p, nsrcn.p);
    PIP_CUDA(cudaGetLastError());
    // advance
    fx = std::move(nfx);
    fy = std::move(nfy);
    fslot = std::move(nslot);
    fcoff = std::move(coff);
    cd_cell = std::move(ncell);
    cd_poly = std::move(npoly);
    cd_base = std::move(nbase);
    cd_src = std::move(nsrc);
    cd_srcn = std::move(nsrcn);
    src_edges = std::move(kedges);
    split_slot_prev = std::move(split_slot);
    n_cell = n_child;
    n_cand = (int64_t)n_cc;
    level_base += n_slots_lv;
    PIP_CUDA(cudaStreamSynchronize(s));
  }

  // concatenate the nodes and the blobs; the top grid is the table
  S->table.release();
  S->nodes.release();
  S->blobs.release();
  S->slot_off.release();
  S->table = std::move(desc_lv[0]);
  int64_t n_nodes = 0;
  for (int64_t l : node_len) n_nodes += l;
  if (!S->nodes.alloc(al, (size_t)(2 * n_nodes + 2), s)) return fail(PIP_ENOMEM, "index: nodes");
  {
    int64_t at = 0;
    for (size_t i = 0; i < node_lv.size(); ++i) {
      PIP_CUDA(cudaMemcpyAsync(S->nodes.p + 2 * at, node_lv[i].p, node_len[i] * sizeof(TrieNode),
                               cudaMemcpyDeviceToDevice, s));
      at += node_len[i];
    }
  }
  table_total = top_cells + 8 * n_nodes;
  // blobs padded by one 16-byte unit so bulk copies never read past the end
  if (!S->blobs.alloc(al, (size_t)blob_total16 + 1, s)) return fail(PIP_ENOMEM, "index: blobs");
  // record offsets of every slot, plus one past the last record
  if (!S->slot_off.alloc(al, (size_t)sb_total * SB_SLOTS + 1, s)) return fail(PIP_ENOMEM, "index: slot offsets");
  {
    int64_t at16 = 0, at_slot = 0;
    for (size_t i = 0; i < blob_lv.size(); ++i) {
      PIP_CUDA(cudaMemcpyAsync(S->blobs.p + at16, blob_lv[i].p, blob_len[i] * sizeof(uint4),
                               cudaMemcpyDeviceToDevice, s));
      PIP_CUDA(cudaMemcpyAsync(S->slot_off.p + at_slot, sbd_lv[i].p, sb_len[i] * SB_SLOTS * sizeof(uint32_t),
                               cudaMemcpyDeviceToDevice, s));
      at16 += blob_len[i];
      at_slot += sb_len[i] * SB_SLOTS;
    }
    const uint32_t end16 = (uint32_t)blob_total16;
    PIP_CUDA(cudaMemcpyAsync(S->slot_off.p + at_slot, &end16, sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    PIP_CUDA(cudaStreamSynchronize(s));
  }
  S->approx.release();
  if (o.approx_units > 0 && sb_total > 0) {  // approximate mode: answer of every leaf slot
    const int64_t n_slots = sb_total * SB_SLOTS;
    DBuf<int2> cen;
    ALLOC(cen, n_slots);
    int64_t at = 0;
    for (size_t i = 0; i < cen_lv.size(); ++i) {
      PIP_CUDA(cudaMemcpyAsync(cen.p + at, cen_lv[i].p, sb_len[i] * SB_SLOTS * sizeof(int2),
                               cudaMemcpyDeviceToDevice, s));
      at += sb_len[i] * SB_SLOTS;
    }
    if (!S->approx.alloc(al, (size_t)n_slots, s)) return fail(PIP_ENOMEM, "index: approximate answers");
    k_leaf_answer<<<blocks_for(n_slots), TB, 0, s>>>(n_slots, cen.p, S->blobs.p, S->slot_off.p, S->approx.p);
    PIP_CUDA(cudaGetLastError());
  }
  uint32_t e2 = 0;
  CHECK(d2h(&e2, err.p, 1, s));
  unsigned long long hc[13];
  CHECK(d2h(hc, counters, 13, s));
  // a trie without compact leaves is walked as 16-byte entries
  int64_t n_entries = 0;
  bool entries16 = false;
  if (hc[3] == 0) CHECK(to_entries16(al, S->nodes, node_len, &n_entries, &entries16, s));
  if (entries16) table_total = top_cells + 4 * n_entries;
  PIP_CUDA(cudaEventRecord(ev1, s));
  PIP_CUDA(cudaEventSynchronize(ev1));
  float ms = 0;
  cudaEventElapsedTime(&ms, ev0, ev1);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);

  IndexView& v = S->view;
  v.gx0 = (int32_t)g.gx0;
  v.gy0 = (int32_t)g.gy0;
  v.nx = g.nx;
  v.ny = g.ny;
  v.s0 = g.s0;
  v.depth = depth_used;
  v.n_sb = (uint32_t)sb_total;
  v.table = S->table.p;
  v.nodes = S->nodes.p;
  v.blobs = S->blobs.p;
  v.slot_off = S->slot_off.p;
  v.approx_id = S->approx.p;  // nullptr unless approximate
  v.compact = entries16 ? 0u : 1u;
  {  // L2-resident part of the trie: the top grid plus the first nodes (the
     // shallow levels come first) up to three quarters of the L2
    int dev = 0, l2 = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess || l2 <= 0) {
      cudaGetLastError();
      l2 = 64 << 20;
    }
    const int64_t budget = (int64_t)l2 * 3 / 4 - top_cells * 4;
    v.hot_nodes = (uint32_t)std::max<int64_t>(0, entries16 ? std::min<int64_t>(n_entries, budget / 16)
                                                            : std::min<int64_t>(n_nodes, budget / 32));
  }

  pip_set_info_t& I = S->info;
  I.n_poly = S->n_poly;
  I.n_ring = S->n_ring;
  I.n_vert = S->n_vert;
  I.n_levels = (int64_t)S->parent.size();
  I.top_cells = top_cells;
  I.table_entries = table_total;
  I.leaves = (int64_t)slot_base;
  I.empty_cells = (int64_t)hc[0];
  I.interior_cells = (int64_t)hc[1] - (int64_t)hc[2];  // palette overflows became leaves
  I.superbins = sb_total;
  I.leaf_cands = leaf_cands;
  I.leaf_edges = leaf_edges;
  I.index_bytes = top_cells * 4 + (entries16 ? n_entries * 16 : n_nodes * 32) + blob_total16 * 16 +
                  (sb_total * SB_SLOTS + 1) * 4;
  I.max_blob_bytes = max_blob16 * 16;
  I.compact_leaves = (int64_t)hc[3];
  I.compact_bytes = (int64_t)hc[4] * 32;
  for (int e = 0; e < 8; ++e) I.compact_by_edges[e] = (int64_t)hc[5 + e];
  I.size_ratio = o.size_ratio;
  I.compact_edges = o.compact_edges;
  for (size_t l = 0; l < 8; ++l) I.nodes_by_level[l] = l < node_len.size() ? node_len[l] : 0;
  I.cell_log2 = g.s0;
  I.fanout_log2 = k;
  I.depth = depth_used;
  I.cand_mode = o.cand_mode;
  I.pts_per_cta = o.pts_per_cta;
  I.stage_depth = o.stage_depth;
  I.grid_x0 = (int32_t)g.gx0;
  I.grid_y0 = (int32_t)g.gy0;
  I.grid_nx = g.nx;
  I.grid_ny = g.ny;
  I.build_ms = ms;
  S->opts = o;
  return PIP_OK;
}

// Top-cell candidate lists in a given mode (test hook for the equivalence of
// hierarchy descent and box rasterization).
pip_status top_candidates_export(pip_set_s* S, int mode, int64_t* off, int32_t* ids, int64_t cap,
                                 cudaStream_t s) {
  Alloc* al = &S->alloc;
  Grid g;
  g.gx0 = S->view.gx0;
  g.gy0 = S->view.gy0;
  g.nx = S->view.nx;
  g.ny = S->view.ny;
  g.s0 = S->view.s0;
  DBuf<uint32_t> err;
  ALLOC(err, 1);
  PIP_CUDA(cudaMemsetAsync(err.p, 0, 2 * sizeof(uint32_t), s));
  HierBufs hb;
  Hier h;
  CHECK(build_hierarchy(S, al, s, hb, h, err));
  if (mode == 1 && S->parent.empty()) h.levels = 0;
  DBuf<uint32_t> cnt;
  DBuf<uint64_t> coff;
  DBuf<int32_t> cids;
  uint64_t total = 0;
  CHECK(top_candidates(S, al, s, h, g, mode, cnt, coff, cids, total));
  const int64_t cells = (int64_t)g.nx * g.ny;
  std::vector<uint64_t> ho(cells + 1);
  CHECK(d2h(ho.data(), coff.p, cells + 1, s));
  for (int64_t i = 0; i <= cells; ++i) off[i] = (int64_t)ho[i];
  if ((int64_t)total > cap) return fail(PIP_EINVAL, "pip_set_top_candidates: cap too small");
  if (total) CHECK(d2h(ids, cids.p, total, s));
  return PIP_OK;
}

pip_status load_validate(pip_set_s* S, cudaStream_t s) {
  Alloc* al = &S->alloc;
  DBuf<uint32_t> err;
  ALLOC(err, 1);
  PIP_CUDA(cudaMemsetAsync(err.p, 0, 2 * sizeof(uint32_t), s));
  k_validate_csr<<<blocks_for(std::max(S->n_ring, S->n_poly) + 1), TB, 0, s>>>(
      S->ring_off.p, S->n_ring, S->poly_ring_off.p, S->n_poly, S->n_vert, err.p);
  PIP_CUDA(cudaGetLastError());
  uint32_t e = 0;
  CHECK(d2h(&e, err.p, 1, s));
  if (e) return fail(PIP_EINVAL, "pip_set_load: malformed ring_off / poly_ring_off");
  if (!S->poly_box.alloc(al, (size_t)S->n_poly + 1, s)) return fail(PIP_ENOMEM, "poly boxes");
  k_poly_box<<<blocks_for(S->n_poly * 32), TB, 0, s>>>(S->vx.p, S->vy.p, S->ring_off.p,
                                                       S->poly_ring_off.p, S->n_poly, S->poly_box.p, err.p);
  PIP_CUDA(cudaGetLastError());
  CHECK(d2h(&e, err.p, 1, s));
  if (e & 2u) return fail(PIP_ERANGE, "pip_set_load: an edge spans 2^31 lattice units or more");
  return PIP_OK;
}

pip_status quantize_vertices(const double* x, const double* y, int64_t n, int32_t* qx, int32_t* qy,
                             Alloc* al, cudaStream_t s) {
  DBuf<uint32_t> err;
  ALLOC(err, 1);
  PIP_CUDA(cudaMemsetAsync(err.p, 0, 2 * sizeof(uint32_t), s));
  k_f64_to_lattice<<<blocks_for(n), TB, 0, s>>>(x, y, n, qx, qy, err.p);
  PIP_CUDA(cudaGetLastError());
  uint32_t e = 0;
  CHECK(d2h(&e, err.p, 1, s));
  if (e) return fail(PIP_ERANGE, "pip_set_load_f64: a vertex coordinate is not finite or out of range");
  return PIP_OK;
}

}  // namespace pip
