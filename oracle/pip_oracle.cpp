// Plain CPU oracle for the census-block point-in-polygon join.
//
// TEST INFRASTRUCTURE ONLY. Nothing on the product path may call, link or
// load this file; only tests/, __graft_entry__.smoke() and bench.py's CPU
// baseline leg and reference arm use it. It shares no source with the CUDA
// library.
//
// What it computes (Kepner et al., "Fast Mapping onto Census Blocks"):
//   * Sec. II: points are IEEE doubles (x_pt = longitude, y_pt = latitude);
//     polygons are rings of vertices (x_poly, y_poly) with bounding boxes
//     [x_min x_max y_min y_max] arranged in a hierarchy.
//   * Sec. III-A: membership is the crossing-number test: cast a ray from the
//     point towards +x, count boundary crossings, odd = inside. Polygons may
//     be concave and multiply connected (holes are extra rings).
//   * Sec. III (Appendix A, findCensusBlock): bounding boxes, tested level by
//     level down the hierarchy, only pick which polygons get the crossing
//     test; the first polygon (lowest index) that contains a point claims it.
//
// Readings where the paper is silent (each one is listed with its reason in
// the design notes):
//   * Q(v): the coordinate lattice is 1e-7 degree. Q(v) is the integer
//     nearest to the exact real number v * 10^7, ties to even. v is valid iff
//     it is finite and |Q(v)| <= 2^31 - 1; an invalid coordinate gives id -1.
//   * Tie rule for points on edges and vertices: an edge a->b counts for the
//     point p iff (a.y > p.y) != (b.y > p.y) and the edge's crossing with the
//     horizontal line through p lies strictly right of p. This equals the
//     textbook even-odd test at p + (delta, eps) with 0 < eps << delta
//     infinitesimal, so polygons own their left and bottom boundary.
//   * Bounding boxes are closed and only filter; they never decide.
//   * Output: int32 polygon index, -1 when no polygon contains the point.
//
// Products are evaluated in 128-bit integers, so this oracle is exact for
// every int32 vertex and point, with no range precondition.

#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

typedef __int128 i128;
typedef unsigned __int128 u128;

// Q(v) = round-half-even(v * 10^7) computed exactly from the binary64
// encoding v = m * 2^e (Sec. II: points are IEEE doubles).
int quantize(double v, int32_t* q) {
  uint64_t bits;
  std::memcpy(&bits, &v, sizeof bits);
  const int negative = (int)(bits >> 63);
  const int biased = (int)((bits >> 52) & 0x7ff);
  const uint64_t frac = bits & ((1ull << 52) - 1);
  if (biased == 0x7ff) return 0;  // inf or NaN
  if (biased == 0 && frac == 0) {  // +0 or -0
    *q = 0;
    return 1;
  }
  const uint64_t m = biased ? (frac | (1ull << 52)) : frac;
  const int e = (biased ? biased : 1) - 1075;  // v = m * 2^e exactly
  if (e >= 0) return 0;                        // |v| >= 2^52: far out of range
  const u128 product = (u128)m * 10000000u;    // v * 10^7 = product * 2^e
  const int shift = -e;
  u128 whole, rest, half;
  if (shift >= 127) {
    whole = 0;
    rest = product;
    half = (u128)1 << 126;  // product < 2^77 < half: rounds to zero
  } else {
    whole = product >> shift;
    rest = product & (((u128)1 << shift) - 1);
    half = (u128)1 << (shift - 1);
  }
  if (rest > half || (rest == half && (whole & 1))) whole += 1;
  if (whole > (u128)INT32_MAX) return 0;
  *q = negative ? -(int32_t)whole : (int32_t)whole;
  return 1;
}

// Crossing-number contribution of the edge a->b for the point p (Sec. III-A)
// under the half-open rule stated above.
int edge_crossing(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t px,
                  int64_t py) {
  if ((ay > py) == (by > py)) return 0;   // edge does not straddle the ray
  if (std::max(ax, bx) <= px) return 0;   // edge wholly at or left of p
  if (std::min(ax, bx) > px) return 1;    // edge wholly right of p
  // Orientation of p against a->b; the crossing is right of p exactly when
  // this has the sign of (by - ay).
  const i128 s = (i128)(bx - ax) * (py - ay) - (i128)(by - ay) * (px - ax);
  if (s == 0) return 0;  // p on the edge: the crossing is not strictly right
  return (s > 0) == (by > ay);
}

struct PolySet {
  const int32_t* vx;
  const int32_t* vy;
  const int64_t* ring_off;       // ring r = vertices [ring_off[r], ring_off[r+1])
  const int64_t* poly_ring_off;  // polygon p = rings [poly_ring_off[p], ...[p+1])
  int64_t n_poly;
};

// inpolygon(): parity of crossings over every edge of every ring of polygon
// p; each ring is closed by its last->first edge (Appendix A, inpolygon2).
int inside(const PolySet& s, int64_t p, int32_t px, int32_t py) {
  int parity = 0;
  for (int64_t r = s.poly_ring_off[p]; r < s.poly_ring_off[p + 1]; ++r) {
    const int64_t first = s.ring_off[r], last = s.ring_off[r + 1] - 1;
    for (int64_t i = first; i <= last; ++i) {
      const int64_t j = (i == last) ? first : i + 1;
      parity ^= edge_crossing(s.vx[i], s.vy[i], s.vx[j], s.vy[j], px, py);
    }
  }
  return parity;
}

template <class F>
void parallel_for(int64_t n, int n_threads, F f) {
  if (n_threads <= 1 || n < 1024) {
    f(0, n);
    return;
  }
  std::vector<std::thread> pool;
  const int64_t step = (n + n_threads - 1) / n_threads;
  for (int t = 0; t < n_threads; ++t) {
    const int64_t a = t * step, b = std::min(n, a + step);
    if (a >= b) break;
    pool.emplace_back([=] { f(a, b); });
  }
  for (auto& th : pool) th.join();
}

// O0: every point against every polygon in ascending index order; no filter.
int32_t bruteforce_one(const PolySet& s, int32_t px, int32_t py) {
  for (int64_t p = 0; p < s.n_poly; ++p)
    if (inside(s, p, px, py)) return (int32_t)p;
  return -1;
}

// Bounding box [x_min x_max y_min y_max] of each node of the hierarchy.
struct Box {
  int32_t x_min, x_max, y_min, y_max;
  bool contains(int32_t px, int32_t py) const {  // closed box
    return x_min <= px && px <= x_max && y_min <= py && py <= y_max;
  }
};

// The region -> county -> tract -> block hierarchy of Sec. III: level 0 are
// the polygons, parent[l][i] is the level l+1 node that owns level-l node i.
// A parent's box is the union of its children's boxes, so the hierarchy only
// prunes and never changes an answer.
struct Hierarchy {
  int n_levels = 0;
  std::vector<std::vector<Box>> box;               // per level
  std::vector<std::vector<int64_t>> child_off;     // per level >= 1
  std::vector<std::vector<int64_t>> child;         // per level >= 1
  std::vector<int64_t> roots;                      // nodes of the top level
};

Box empty_box() { return Box{INT32_MAX, INT32_MIN, INT32_MAX, INT32_MIN}; }

void grow(Box& b, const Box& c) {
  b.x_min = std::min(b.x_min, c.x_min);
  b.x_max = std::max(b.x_max, c.x_max);
  b.y_min = std::min(b.y_min, c.y_min);
  b.y_max = std::max(b.y_max, c.y_max);
}

Hierarchy build_hierarchy(const PolySet& s, const int32_t* parent_flat,
                          const int64_t* level_len, int n_levels) {
  Hierarchy h;
  h.n_levels = n_levels;
  h.box.resize(n_levels + 1);
  h.child_off.resize(n_levels + 1);
  h.child.resize(n_levels + 1);
  h.box[0].assign(s.n_poly, empty_box());
  for (int64_t p = 0; p < s.n_poly; ++p) {
    Box& b = h.box[0][p];
    const int64_t v0 = s.ring_off[s.poly_ring_off[p]];
    const int64_t v1 = s.ring_off[s.poly_ring_off[p + 1]];
    for (int64_t v = v0; v < v1; ++v) {
      b.x_min = std::min(b.x_min, s.vx[v]);
      b.x_max = std::max(b.x_max, s.vx[v]);
      b.y_min = std::min(b.y_min, s.vy[v]);
      b.y_max = std::max(b.y_max, s.vy[v]);
    }
  }
  const int32_t* parent = parent_flat;
  for (int l = 0; l < n_levels; ++l) {
    const int64_t n_child = level_len[l];
    int64_t n_parent = 0;
    for (int64_t i = 0; i < n_child; ++i)
      n_parent = std::max<int64_t>(n_parent, (int64_t)parent[i] + 1);
    h.box[l + 1].assign(n_parent, empty_box());
    std::vector<int64_t> count(n_parent + 1, 0);
    for (int64_t i = 0; i < n_child; ++i) {
      grow(h.box[l + 1][parent[i]], h.box[l][i]);
      count[parent[i] + 1]++;
    }
    for (int64_t k = 0; k < n_parent; ++k) count[k + 1] += count[k];
    h.child_off[l + 1] = count;
    h.child[l + 1].assign(n_child, 0);
    std::vector<int64_t> fill(count.begin(), count.end() - 1);
    for (int64_t i = 0; i < n_child; ++i) h.child[l + 1][fill[parent[i]]++] = i;
    parent += n_child;
  }
  const int64_t n_top = (int64_t)h.box[n_levels].size();
  for (int64_t i = 0; i < n_top; ++i) h.roots.push_back(i);
  return h;
}

// O1: Sec. III made exact. Descend the box hierarchy to the polygons whose
// closed box holds the point, then run the crossing test on those, lowest
// index first (the first containing polygon claims the point).
int32_t hierarchical_one(const PolySet& s, const Hierarchy& h, int32_t px,
                         int32_t py, std::vector<int64_t>& cand,
                         std::vector<std::pair<int, int64_t>>& stack) {
  cand.clear();
  stack.clear();
  for (int64_t r : h.roots)
    if (h.box[h.n_levels][r].contains(px, py)) stack.push_back({h.n_levels, r});
  while (!stack.empty()) {
    const auto [level, node] = stack.back();
    stack.pop_back();
    if (level == 0) {
      cand.push_back(node);
      continue;
    }
    for (int64_t k = h.child_off[level][node]; k < h.child_off[level][node + 1]; ++k) {
      const int64_t c = h.child[level][k];
      if (h.box[level - 1][c].contains(px, py)) stack.push_back({level - 1, c});
    }
  }
  std::sort(cand.begin(), cand.end());
  for (int64_t p : cand)
    if (inside(s, p, px, py)) return (int32_t)p;
  return -1;
}

}  // namespace

extern "C" {

int orc_quantize(double v, int32_t* q) { return quantize(v, q); }

void orc_quantize_many(const double* v, int64_t n, int32_t* q, uint8_t* valid) {
  for (int64_t i = 0; i < n; ++i) {
    int32_t t = 0;
    valid[i] = (uint8_t)quantize(v[i], &t);
    q[i] = t;
  }
}

int orc_edge_crossing(int32_t ax, int32_t ay, int32_t bx, int32_t by, int32_t px,
                      int32_t py) {
  return edge_crossing(ax, ay, bx, by, px, py);
}

int orc_inside(const int32_t* vx, const int32_t* vy, const int64_t* ring_off,
               const int64_t* poly_ring_off, int64_t n_poly, int64_t poly,
               int32_t px, int32_t py) {
  PolySet s{vx, vy, ring_off, poly_ring_off, n_poly};
  return inside(s, poly, px, py);
}

// Number of polygons whose inside() holds at each lattice point (partition
// invariant checks).
void orc_count_owners_q(const int32_t* vx, const int32_t* vy, const int64_t* ring_off,
                        const int64_t* poly_ring_off, int64_t n_poly,
                        const int32_t* qx, const int32_t* qy, int64_t n,
                        int32_t* count, int n_threads) {
  PolySet s{vx, vy, ring_off, poly_ring_off, n_poly};
  parallel_for(n, n_threads, [&](int64_t a, int64_t b) {
    for (int64_t i = a; i < b; ++i) {
      int32_t c = 0;
      for (int64_t p = 0; p < n_poly; ++p) c += inside(s, p, qx[i], qy[i]);
      count[i] = c;
    }
  });
}

// O0 on lattice points.
void orc_join_bruteforce_q(const int32_t* vx, const int32_t* vy,
                           const int64_t* ring_off, const int64_t* poly_ring_off,
                           int64_t n_poly, const int32_t* qx, const int32_t* qy,
                           int64_t n, int32_t* out, int n_threads) {
  PolySet s{vx, vy, ring_off, poly_ring_off, n_poly};
  parallel_for(n, n_threads, [&](int64_t a, int64_t b) {
    for (int64_t i = a; i < b; ++i) out[i] = bruteforce_one(s, qx[i], qy[i]);
  });
}

// O0 on double coordinates (quantized by Q first; invalid -> -1).
void orc_join_bruteforce(const int32_t* vx, const int32_t* vy, const int64_t* ring_off,
                         const int64_t* poly_ring_off, int64_t n_poly,
                         const double* x_pt, const double* y_pt, int64_t n,
                         int32_t* out, int n_threads) {
  PolySet s{vx, vy, ring_off, poly_ring_off, n_poly};
  parallel_for(n, n_threads, [&](int64_t a, int64_t b) {
    for (int64_t i = a; i < b; ++i) {
      int32_t px, py;
      if (!quantize(x_pt[i], &px) || !quantize(y_pt[i], &py)) {
        out[i] = -1;
        continue;
      }
      out[i] = bruteforce_one(s, px, py);
    }
  });
}

// O1 with the hierarchy prepared once and reused across calls (a handle owns
// the boxes and child lists; the polygon arrays stay the caller's).
struct HierHandle {
  PolySet s;
  Hierarchy h;
};

void* orc_hier_create(const int32_t* vx, const int32_t* vy, const int64_t* ring_off,
                      const int64_t* poly_ring_off, int64_t n_poly, const int32_t* parent_flat,
                      const int64_t* level_len, int n_levels) {
  HierHandle* H = new HierHandle{PolySet{vx, vy, ring_off, poly_ring_off, n_poly}, Hierarchy{}};
  H->h = build_hierarchy(H->s, parent_flat, level_len, n_levels);
  return H;
}

void orc_hier_join(void* handle, const double* x_pt, const double* y_pt, int64_t n, int32_t* out,
                   int n_threads) {
  const HierHandle* H = (const HierHandle*)handle;
  parallel_for(n, n_threads, [&](int64_t a, int64_t b) {
    std::vector<int64_t> cand;
    std::vector<std::pair<int, int64_t>> stack;
    for (int64_t i = a; i < b; ++i) {
      int32_t px, py;
      if (!quantize(x_pt[i], &px) || !quantize(y_pt[i], &py)) {
        out[i] = -1;
        continue;
      }
      out[i] = hierarchical_one(H->s, H->h, px, py, cand, stack);
    }
  });
}

void orc_hier_free(void* handle) { delete (HierHandle*)handle; }

// O1 on double coordinates. parent_flat holds the parent arrays of levels
// 0..n_levels-1 back to back; level_len[l] is the length of level l's array
// (level_len[0] = n_poly). n_levels = 0 means a flat set.
void orc_join_hier(const int32_t* vx, const int32_t* vy, const int64_t* ring_off,
                   const int64_t* poly_ring_off, int64_t n_poly,
                   const int32_t* parent_flat, const int64_t* level_len,
                   int n_levels, const double* x_pt, const double* y_pt, int64_t n,
                   int32_t* out, int n_threads) {
  PolySet s{vx, vy, ring_off, poly_ring_off, n_poly};
  const Hierarchy h = build_hierarchy(s, parent_flat, level_len, n_levels);
  parallel_for(n, n_threads, [&](int64_t a, int64_t b) {
    std::vector<int64_t> cand;
    std::vector<std::pair<int, int64_t>> stack;
    for (int64_t i = a; i < b; ++i) {
      int32_t px, py;
      if (!quantize(x_pt[i], &px) || !quantize(y_pt[i], &py)) {
        out[i] = -1;
        continue;
      }
      out[i] = hierarchical_one(s, h, px, py, cand, stack);
    }
  });
}

}  // extern "C"
