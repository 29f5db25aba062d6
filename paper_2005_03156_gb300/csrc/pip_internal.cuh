// Internal definitions shared by the library's translation units.
//
// Layout of a loaded set in HBM (all device-resident, built by index.cu):
//   table  u32 descriptors of the top grid (row-major, nx * ny). A
//          descriptor is tag:2 | payload:30 with
//            TAG_EMPTY     no polygon contains any point of the cell  -> -1
//            TAG_INTERIOR  payload = polygon id answering every point
//            TAG_LEAF      payload = leaf slot: the crossing test decides
//            TAG_CHILD     payload = index of the cell's trie node
//   nodes  the trie, in one of two forms (IndexView::compact says which):
//          32-byte nodes (one DRAM sector) per split cell, describing its
//          4 x 4 children: a leaf mask and a child mask (children that are
//          boundary leaves / split again, numbered from leaf_base /
//          child_base in child order), and for the other children a 2-bit
//          code into a 4-entry palette of polygon ids (-1 = empty). An
//          index without compact leaves converts them, once built, to
//          16-byte entries (half the bytes per node, so twice the nodes per
//          L2 line; the walk reads one entry per level):
//            node  w0 = 2-bit code per child: 0 -> polygon w2, 1 -> polygon
//                  w3, 2 -> empty, 3 -> descend to entry (w1 & 2^30 - 1) +
//                  the child's rank among the node's code-3 children;
//                  w1 bits 30-31 = 0
//            leaf  w0 = leaf slot (a boundary leaf child); w1 bits 30-31 = 1
//            id    w0 = polygon id (a child whose polygon is neither w2 nor
//                  w3 of its parent); w1 bits 30-31 = 2
//          The top grid names a level-1 entry; the entries of each level
//          follow the previous level's, a node's descending children
//          contiguous in child order.
//   blobs  one 16-byte-aligned record per leaf slot, in slot order (so
//          the records of consecutive slots, e.g. a chunk of binned points,
//          are one contiguous range that one bulk copy can stage):
//            u32 nc                 kept candidates
//            u32 cand[nc]           polygon id | base_parity << 31
//            u32 edge_end[nc]       end of each candidate's edges (cumulative)
//            (pad to 16 bytes)
//            int4 edge[ne]          (ax, ay, bx, by) with ay <= by; an edge
//                                   with ay == by is horizontal and never
//                                   counts (kept only to mark the boundary)
//          Padding slots (past a level's leaves) hold an empty record.
//   slot_off u32 per leaf slot (+ one past the last): the record's offset
//          in 16-byte units. Slots are grouped by 32 into superbins, the
//          binning key of the residual points.
//
// Compact leaves. A boundary cell whose kept candidates (at most 3) share at
// most a few distinct non-horizontal edges is answered in the classify
// kernel itself from one record of 1..4 consecutive 32-byte slots of the
// node array (no residual queue, no binning):
//   w[0]      E (bits 0-2: distinct edges) | C << 3 (bits 3-4: candidates)
//   w[1..3]   candidate words: id (bits 0-23) | edge mask << 24 (bits 24-30:
//             which of the E edges belong to the candidate) | base << 31
//   w[4..]    the E edges as int4 (ax, ay, bx, by), ay < by: edge 0 in
//             slot 0 words 4-7, edges 1-2 in slot 1, 3-4 in slot 2, 5-6 in
//             slot 3.
// A point's answer is the first candidate whose base parity XOR the parity
// of its counted edges is odd (the candidate lists keep id order), else -1.
// A CHILD descriptor with DESC_COMPACT set names such a record: its slot in
// bits 0-26 and the record's slot count minus one in bits 27-28. Inside a
// trie node a compact child has both its leaf and its split bit set, takes
// its slots in the child numbering, and keeps slots - 1 in its 2-bit code.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/pip.h"

namespace pip {

constexpr uint32_t TAG_EMPTY = 0u;
constexpr uint32_t TAG_INTERIOR = 1u;
constexpr uint32_t TAG_LEAF = 2u;
constexpr uint32_t TAG_CHILD = 3u;
constexpr uint32_t PAYLOAD_MASK = 0x3FFFFFFFu;
constexpr int SB_LOG2 = 5;  // 32 leaf slots per superbin
constexpr int SB_SLOTS = 1 << SB_LOG2;
constexpr int MAX_LEVELS = 12;
constexpr uint32_t DESC_COMPACT = 1u << 29;
constexpr int DESC_SLOTS_SHIFT = 27;
constexpr uint32_t SLOT_MASK = (1u << 27) - 1u;  // node-array slots (32 bytes each)
constexpr int COMPACT_MAX_EDGES = 7;
constexpr int COMPACT_MAX_CANDS = 3;
constexpr uint32_t CAND_ID_MASK = (1u << 24) - 1u;

// Slots of a compact record with E distinct edges: edge 0 shares slot 0
// with the header and candidates, later edges take two per slot.
__host__ __device__ inline uint32_t compact_slots_for(uint32_t edges) {
  return edges <= 1u ? 1u : 1u + (edges) / 2u;
}

__host__ __device__ inline uint32_t make_desc(uint32_t tag, uint32_t payload) {
  return (tag << 30) | (payload & PAYLOAD_MASK);
}

constexpr int NODE_K = 2;  // a split cell has 2^NODE_K x 2^NODE_K children
constexpr int NODE_FAN = 1 << (2 * NODE_K);

struct __align__(32) TrieNode {
  uint32_t masks;       // bits 0-15: leaf children, bits 16-31: split children
  uint32_t codes;       // 2 bits per child: palette entry of the other children
  uint32_t leaf_base;   // leaf slot of the first leaf child
  uint32_t child_base;  // node index of the first split child
  int32_t pal[4];       // polygon id, or -1 for an empty child
};
static_assert(sizeof(TrieNode) == 32, "trie node must be one 32-byte sector");

// Device view of one set's index, passed to kernels by value.
struct IndexView {
  int32_t gx0, gy0;       // lattice origin of the grid
  uint32_t nx, ny;        // top cells per row / column
  int32_t s0;             // log2 side of a top cell
  int32_t depth;          // deepest level present (trie levels below the top grid)
  uint32_t n_sb;          // superbins
  uint32_t hot_nodes;     // nodes / entries [0, hot_nodes) (the shallow levels) are kept in L2
  uint32_t compact;       // 1: 32-byte nodes (which may hold compact leaves);
                          // 0: 16-byte entries
  const uint32_t* table;  // top-grid descriptors
  const uint4* nodes;     // trie nodes, two uint4 per node
  const uint4* blobs;     // superbin records (16-byte units)
  const uint32_t* slot_off;  // per leaf slot (+1): record offset in 16-byte units
  const int32_t* approx_id;  // approximate mode: id per leaf slot (nullptr when exact)
};

// L2 eviction policy for the index: keep it resident while the point stream
// (loaded and stored with evict-first .cs operations) passes through L2.
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// Policy for the deep trie levels: each node there serves few points, so it
// should not displace the top grid and the shallow levels, which every point
// or most points read.
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// Index loads do not allocate in L1: each top-grid cell or trie node a warp
// reads is seldom read again by the same SM soon, and leaving L1 to the
// loads in flight measured 8 % faster for the classify kernel.
__device__ __forceinline__ uint32_t ld_index_u32(const uint32_t* ptr, uint64_t pol) {
  uint32_t r;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(r) : "l"(ptr), "l"(pol));
  return r;
}

// A whole 32-byte node in one 256-bit load (one sector, one request).
struct NodeWords {
  uint32_t w[8];
};

__device__ __forceinline__ NodeWords ld_node(const uint4* nodes, uint32_t node, uint64_t pol) {
  NodeWords n;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8], %9;"
               : "=r"(n.w[0]), "=r"(n.w[1]), "=r"(n.w[2]), "=r"(n.w[3]), "=r"(n.w[4]), "=r"(n.w[5]),
                 "=r"(n.w[6]), "=r"(n.w[7])
               : "l"(nodes + 2 * (size_t)node), "l"(pol));
  return n;
}

// Bit j of a 16-bit mask to bits 2j and 2j+1.
__device__ __forceinline__ uint32_t spread2(uint32_t m) {
  m = (m | (m << 8)) & 0x00FF00FFu;
  m = (m | (m << 4)) & 0x0F0F0F0Fu;
  m = (m | (m << 2)) & 0x33333333u;
  m = (m | (m << 1)) & 0x55555555u;
  return m | (m << 1);
}

// One trie step: child `sub` of node n. Returns a descriptor; TAG_CHILD
// means descend into node `payload`, or, with DESC_COMPACT set, answer from
// the compact record at that slot. Split children and compact children
// share the child numbering; a compact child takes (its code + 1) slots.
// COMPACT = false is the same step for a trie without compact children.
template <bool COMPACT = true>
__device__ __forceinline__ uint32_t node_step(const NodeWords& n, uint32_t sub) {
  const uint32_t bit = 1u << sub, below = bit - 1u;
  const uint32_t lm = n.w[0] & 0xFFFFu, cm = n.w[0] >> 16;
  if (!COMPACT) {
    if (lm & bit) return make_desc(TAG_LEAF, n.w[2] + __popc(lm & below));
    if (cm & bit) return make_desc(TAG_CHILD, n.w[3] + __popc(cm & below));
  }
  const uint32_t both = lm & cm;
  if (COMPACT && ((lm | cm) & bit)) {
    if ((lm & bit) && !(cm & bit)) return make_desc(TAG_LEAF, n.w[2] + __popc(lm & ~cm & below));
    uint32_t slot = n.w[3] + __popc(cm & below);
    if (both & below) {  // compact children before this one take (code + 1) slots each
      const uint32_t v = n.w[1] & spread2(both & below);
      slot += __popc(v & 0x55555555u) + 2u * __popc(v & 0xAAAAAAAAu);
    }
    if (!(both & bit)) return make_desc(TAG_CHILD, slot);
    const uint32_t extra = (n.w[1] >> (2 * sub)) & 3u;
    return make_desc(TAG_CHILD, DESC_COMPACT | (extra << DESC_SLOTS_SHIFT) | slot);
  }
  const uint32_t code = (n.w[1] >> (2 * sub)) & 3u;
  const int32_t id = (int32_t)(code == 0 ? n.w[4] : code == 1 ? n.w[5] : code == 2 ? n.w[6] : n.w[7]);
  return id < 0 ? make_desc(TAG_EMPTY, 0) : make_desc(TAG_INTERIOR, (uint32_t)id);
}

// 16-byte trie entries (see the layout above).
constexpr uint32_t E16_NODE = 0u, E16_LEAF = 1u, E16_ID = 2u;  // w1 bits 30-31
constexpr uint32_t E16_EMPTY = 2u, E16_DESCEND = 3u;           // child codes
constexpr uint32_t E16_BASE_MASK = (1u << 30) - 1u;

__device__ __forceinline__ uint4 ld_entry(const uint4* nodes, uint32_t e, uint64_t pol) {
  uint4 r;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "l"(nodes + e), "l"(pol));
  return r;
}

// One trie step on a 16-byte entry: child `sub` of a node entry, or the
// answer a leaf / id entry holds (sub unused). Returns a descriptor as
// node_step does (TAG_CHILD: payload = entry index).
__device__ __forceinline__ uint32_t entry_step(const uint4& n, uint32_t sub) {
  const uint32_t kind = n.y >> 30;
  if (kind == E16_LEAF) return make_desc(TAG_LEAF, n.x);
  if (kind == E16_ID) return make_desc(TAG_INTERIOR, n.x);
  const uint32_t code = (n.x >> (2 * sub)) & 3u;
  if (code == E16_DESCEND) {
    const uint32_t desc = n.x & (n.x >> 1) & 0x55555555u;  // bit 2c: child c descends
    return make_desc(TAG_CHILD, (n.y & E16_BASE_MASK) + __popc(desc & ((1u << (2 * sub)) - 1u)));
  }
  if (code == E16_EMPTY) return make_desc(TAG_EMPTY, 0);
  return make_desc(TAG_INTERIOR, code ? n.w : n.z);
}

// Residual entry: a point that fell in a boundary leaf.
// x = qx, y = qy, z = index of the point within the call (or batch),
// w = leaf slot (superbin = slot >> 5).
typedef uint4 Residual;
// w of a queue entry that was reserved but never written (skipped by K2)
constexpr uint32_t RES_HOLE = 0xFFFFFFFFu;

// ---------------------------------------------------------------------------
// Q(v) on the device with integer instructions only (GB300's double rate is
// a small fraction of its integer rate). Q(v) is the integer nearest to the
// exact product v * 10^7 (ties to even); valid iff finite and |Q| <= 2^31-1.
//
// With v = m * 2^(e-1075) (m the 53-bit significand, e the biased exponent)
// and 10^7 = 78125 * 2^7, the exact product is P * 2^(e-1068), P = m * 78125
// < 2^70. For 1004 <= e <= 1030 (2^-19 <= |v| < 2^8) the product in 32.32
// fixed point is P >> (1036 - e), a shift of 6..32 bits, taken with two
// funnel shifts; the bits shifted out fold into a sticky bit for the
// round-half-even decision. Other exponents are rare and take an exact
// 128-bit path (tiny values) or are out of range.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool quantize_slow(uint32_t hi, uint32_t lo, int32_t& q) {
  const uint32_t e = (hi >> 20) & 0x7FFu;
  if (e >= 1031u) return false;  // |v| >= 2^8 (includes inf, NaN): |v*1e7| > 2^31
  const uint64_t frac = ((uint64_t)(hi & 0xFFFFFu) << 32) | lo;
  if (e == 0u && frac == 0u) {
    q = 0;
    return true;
  }
  // only |v| < 2^-19 reaches here (the fast path covers [2^-19, 2^8))
  const uint64_t m = e ? (frac | (1ull << 52)) : frac;
  const int sh = (int)(e ? 1075u - e : 1074u);  // v = m * 2^-sh, sh >= 52
  const unsigned __int128 prod = (unsigned __int128)m * 10000000u;  // < 2^77
  uint64_t whole;
  unsigned __int128 rest, half;
  if (sh >= 100) {  // prod < 2^77 < 2^99: rounds to zero
    whole = 0;
    rest = 0;
    half = 1;
  } else {
    whole = (uint64_t)(prod >> sh);
    rest = prod & ((((unsigned __int128)1) << sh) - 1);
    half = ((unsigned __int128)1) << (sh - 1);
  }
  if (rest > half || (rest == half && (whole & 1ull))) whole += 1;
  const int32_t w = (int32_t)whole;  // < 20 here
  q = (hi >> 31) ? -w : w;
  return true;
}

__device__ __forceinline__ bool quantize_bits(uint32_t hi, uint32_t lo, int32_t& q) {
  const uint32_t e = (hi >> 20) & 0x7FFu;
  const uint32_t sh = 1036u - e;  // wraps for e > 1036: fails the range test
  if (sh - 6u > 26u) return quantize_slow(hi, lo, q);
  const uint32_t mh = (hi & 0xFFFFFu) | 0x100000u;
  const uint64_t c = (uint64_t)lo * 78125u;                       // < 2^49
  const uint64_t a = (uint64_t)mh * 78125u + (uint32_t)(c >> 32);  // < 2^39
  const uint32_t p0 = (uint32_t)c, p1 = (uint32_t)a, p2 = (uint32_t)(a >> 32);
  const uint32_t t_lo = __funnelshift_rc(p0, p1, sh);  // 32.32 fixed point
  const uint32_t t_hi = __funnelshift_rc(p1, p2, sh);
  const uint32_t sticky = (p0 << (32u - sh)) != 0u;
  const uint32_t f = t_lo | sticky;
  const uint32_t mag = t_hi + (f > (0x80000000u - (t_hi & 1u)) ? 1u : 0u);
  if (mag > 0x7FFFFFFFu) return false;
  q = (hi >> 31) ? -(int32_t)mag : (int32_t)mag;
  return true;
}

__device__ __forceinline__ bool quantize_double(double v, int32_t& q) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return quantize_bits((uint32_t)(b >> 32), (uint32_t)b, q);
}

// ---------------------------------------------------------------------------
// Crossing-number contribution (Sec. III-A) of a stored edge for the lattice
// point (px, py). Stored edges have ay <= by (the even-odd parity does not
// depend on edge direction); horizontal ones (ay == by) never count.
// The edge counts iff ay <= py < by and its crossing with y = py lies
// strictly right of px: wholly right counts, wholly at-or-left does not, and
// otherwise the sign of (bx-ax)(py-ay) - (by-ay)(px-ax) decides (> 0 counts).
// The early-outs keep |px-ax| <= |bx-ax| < 2^31, so both products are exact
// 32x32->64 bit multiplies.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int32_t sub32(int32_t a, int32_t b) {
  return (int32_t)((uint32_t)a - (uint32_t)b);  // wraps; exact where it is used
}

__device__ __forceinline__ uint32_t edge_crosses(int4 e, int32_t px, int32_t py) {
  const bool in_y = (py >= e.y) & (py < e.w);
  const int32_t xmin = min(e.x, e.z), xmax = max(e.x, e.z);
  const bool right = px < xmin;
  const bool span = (px >= xmin) & (px < xmax);
  const long long l = (long long)sub32(e.z, e.x) * (long long)sub32(py, e.y);
  const long long r = (long long)sub32(e.w, e.y) * (long long)sub32(px, e.x);
  return (uint32_t)(in_y & (right | (span & (l > r))));
}

// Answer of a compact leaf for the lattice point (px, py): w0..w7 are the
// record's first slot (already loaded); the other slots, slot + 1 .. slot +
// nslots - 1, are loaded here. Edge k's crossing goes to bit k of a mask;
// candidate i is inside iff its base XOR the parity of (mask AND its own
// edge mask) is odd (Sec. III-A, restricted to the cell's kept edges).
__device__ __forceinline__ int32_t compact_answer_words(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3,
                                                     uint32_t w4, uint32_t w5, uint32_t w6, uint32_t w7,
                                                     const uint4* nodes, uint32_t slot, uint32_t nslots,
                                                     int32_t px, int32_t py, uint64_t pol) {
  const uint32_t ne = w0 & 7u, nc = (w0 >> 3) & 3u;
  uint32_t cross = 0;
  if (ne > 0u) cross = edge_crosses(make_int4((int)w4, (int)w5, (int)w6, (int)w7), px, py);
#pragma unroll 1
  for (uint32_t k = 1; k < nslots; ++k) {
    const NodeWords b = ld_node(nodes, slot + k, pol);
    if (2 * k - 1 < ne)
      cross |= edge_crosses(make_int4((int)b.w[0], (int)b.w[1], (int)b.w[2], (int)b.w[3]), px, py) << (2 * k - 1);
    if (2 * k < ne)
      cross |= edge_crosses(make_int4((int)b.w[4], (int)b.w[5], (int)b.w[6], (int)b.w[7]), px, py) << (2 * k);
  }
  int32_t id = -1;
  const uint32_t cw[3] = {w1, w2, w3};
#pragma unroll
  for (uint32_t i = 0; i < 3; ++i) {
    const uint32_t par = (cw[i] >> 31) ^ (__popc((cw[i] >> 24) & 0x7Fu & cross) & 1u);
    if (id < 0 && i < nc && par) id = (int32_t)(cw[i] & CAND_ID_MASK);
  }
  return id;
}

__device__ __forceinline__ int32_t compact_answer(const NodeWords& a, const uint4* nodes, uint32_t slot,
                                                  uint32_t nslots, int32_t px, int32_t py, uint64_t pol) {
  return compact_answer_words(a.w[0], a.w[1], a.w[2], a.w[3], a.w[4], a.w[5], a.w[6], a.w[7], nodes, slot,
                              nslots, px, py, pol);
}

// ---------------------------------------------------------------------------
// Host-side helpers
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
pip_status fail(pip_status st, const std::string& msg);
pip_status cuda_fail(cudaError_t e, const char* what);

#define PIP_CUDA(call)                                        \
  do {                                                        \
    cudaError_t _e = (call);                                  \
    if (_e != cudaSuccess) return ::pip::cuda_fail(_e, #call); \
  } while (0)

int num_sms();
void count_launches(int64_t n);
bool is_device_ptr(const void* p);

// Device memory with an optional user allocator (stream ordered).
struct Alloc {
  pip_allocator hook{};
  bool has_hook = false;
  void* get(size_t bytes, cudaStream_t s);
  void put(void* p, cudaStream_t s);
};

template <class T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  Alloc* a = nullptr;
  cudaStream_t s = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept { *this = std::move(o); }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p; n = o.n; a = o.a; s = o.s;
      o.p = nullptr; o.n = 0;
    }
    return *this;
  }
  ~DBuf() { release(); }
  bool alloc(Alloc* al, size_t count, cudaStream_t st) {
    release();
    a = al;
    s = st;
    n = count;
    if (count == 0) return true;
    p = (T*)a->get(count * sizeof(T), st);
    return p != nullptr;
  }
  void release() {
    if (p && a) a->put(p, s);
    p = nullptr;
    n = 0;
  }
};

// Exclusive scan of n u32 values into u64 outputs; returns the total via
// *total_dev (device) when not null. Stream ordered.
pip_status scan_u32_to_u64(Alloc& al, const uint32_t* in, uint64_t* out, int64_t n,
                           uint64_t* total_dev, cudaStream_t s);
pip_status scan_u64(Alloc& al, const uint64_t* in, uint64_t* out, int64_t n,
                    uint64_t* total_dev, cudaStream_t s);
pip_status scan_u32_to_u64_scratch(const uint32_t* in, uint64_t* out, int64_t n, uint64_t* tmp,
                                   int64_t tmp_len, cudaStream_t s);

}  // namespace pip

// The set as the library holds it.
namespace pip {
struct HostStage;  // host.cu
}

struct pip_set_s {
  int device = 0;
  pip::Alloc alloc;
  pip_build_opts opts{};
  // polygon data (device)
  pip::DBuf<int32_t> vx, vy;
  pip::DBuf<int64_t> ring_off, poly_ring_off;
  pip::DBuf<int4> poly_box;  // (xmin, ymin, xmax, ymax); empty polygon: xmin > xmax
  std::vector<pip::DBuf<int32_t>> parent;  // parent[l]: level-l node -> level-(l+1) node
  std::vector<int64_t> level_len;          // nodes per level (level 0 = polygons)
  int64_t n_vert = 0, n_ring = 0, n_poly = 0;
  // index
  pip::DBuf<uint32_t> table;
  pip::DBuf<uint4> nodes;
  pip::DBuf<uint4> blobs;
  pip::DBuf<uint32_t> slot_off;
  pip::DBuf<int32_t> approx;  // approximate mode: id per leaf slot
  pip::IndexView view{};
  pip_set_info_t info{};
  // error word for bounded device waits
  pip::DBuf<uint32_t> status;
  // per-stage profiling: 4 events per recorded call
  std::vector<cudaEvent_t> prof_ev;
  int32_t prof_cap = 0, prof_n = 0;
  // host-memory calls: a second stream, staging buffers and projection
  // scratch, reserved at the first call and reused (no allocation per call)
  pip::HostStage* host = nullptr;
  ~pip_set_s();
};

namespace pip {
// Scratch of device-resident projections of up to `cap` points: residual
// queue, binned residual (when binning), per-superbin counts and cursors,
// offsets, counters. The host-memory form reserves one per stream and
// reuses it for every chunk.
struct ProjScratch {
  DBuf<Residual> queue, binned;
  DBuf<uint32_t> hist;   // [n_sb] counts then [n_sb] cursors
  DBuf<uint64_t> off;    // [n_sb] exclusive scan of the counts
  DBuf<uint32_t> ctr;    // [0] queue count, [1] crossing work items, [2] residual count
  int64_t cap = 0;       // points
  int64_t n_sb = 0;      // superbins of the index it was sized for
  bool bin = false;      // holds the binned buffer
};
pip_status proj_scratch_alloc(pip_set_s* S, ProjScratch& w, int64_t n, cudaStream_t s);
bool proj_scratch_fits(const pip_set_s* S, const ProjScratch& w, int64_t n);
// Staging of the host-memory form, kept with the set (host.cu).
HostStage* host_stage_new();
void host_stage_free(HostStage* h);
pip_status project_device_with(pip_set_s* S, const double* lon, const double* lat, int64_t n, int32_t* out,
                               cudaStream_t s, pip_project_stats* stats, ProjScratch* pre);
}  // namespace pip
