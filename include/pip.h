/*
 * pip.h - C ABI of the GB300 census-block point-in-polygon join.
 *
 * The operation (Kepner et al., "Fast Mapping onto Census Blocks"):
 *   Sec. II    points are IEEE-double vectors x_pt (longitude) and y_pt
 *              (latitude); polygons are vertex rings with bounding boxes,
 *              organised in a hierarchy (state -> county -> block group).
 *   Sec. III   bounding boxes, level by level, choose which polygons get the
 *              crossing-number test (Sec. III-A: ray to +x, odd = inside;
 *              concave and multiply-connected polygons allowed); the first
 *              (lowest-index) containing polygon claims a point (Appendix A).
 *   Sec. IV    cells that lie wholly inside one polygon answer without any
 *              crossing test ("true hit filtering").
 * The call shape follows the paper's problem statement: load a polygon set
 * once, then map point vectors to block ids (Appendix A findCensusBlock is
 * the query, Appendix B buildCensusStruct the load).
 *
 * Exact semantics used by every entry point:
 *   Q(v)   the integer nearest to the real number v * 10^7 (ties to even);
 *          v is valid iff it is finite and |Q(v)| <= 2^31 - 1.
 *   edge   a->b counts for the lattice point p iff (a.y > p.y) != (b.y > p.y)
 *          and its crossing with the line y = p.y lies strictly right of p
 *          (decided with exact 64-bit integer orientation signs).
 *   inside the parity of counted edges over all rings of the polygon.
 *   id(p)  the smallest polygon index i with inside(P_i, p), else -1; an
 *          invalid coordinate also gives -1.
 * Polygons therefore own their left and bottom boundary: a point on a shared
 * edge or vertex belongs to exactly one block of a gap-free partition.
 *
 * Conventions:
 *   - No exceptions cross the ABI; every call returns a pip_status and
 *     leaves a thread-local message for pip_last_error().
 *   - `stream` arguments are cudaStream_t handles passed as void* (NULL =
 *     the legacy default stream). Calls documented as asynchronous enqueue
 *     work on that stream and return; the caller synchronises the stream.
 *   - Input pointers may be host or device memory (detected with
 *     cudaPointerGetAttributes); the library never keeps them after the
 *     call returns (asynchronous calls read them until the stream reaches
 *     the enqueued work). Output pointers are caller-owned.
 *   - n = 0 is a no-op returning PIP_OK; a NULL pointer with n > 0 is
 *     PIP_EINVAL.
 */
#ifndef PIP_H
#define PIP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pip_set_s* pip_set;         /* opaque; owns device memory */
typedef struct pip_server_s* pip_server;   /* opaque serving loop */
typedef struct pip_plan_s* pip_plan;       /* opaque batched launch plan */

typedef enum {
  PIP_OK = 0,
  PIP_EINVAL = 1,    /* bad argument (NULL, negative size, malformed CSR) */
  PIP_ENOMEM = 2,    /* device or host allocation failed */
  PIP_ECUDA = 3,     /* a CUDA runtime call failed (message has the name) */
  PIP_ERANGE = 4,    /* an edge spans >= 2^31 lattice units, or an extent overflows */
  PIP_ETIMEOUT = 5,  /* a bounded device or host wait ran out */
  PIP_EBUSY = 6      /* admission refused (serving) or resource in use */
} pip_status;

/* Optional allocator hook for device memory. alloc returns a device pointer
 * usable on `stream` (NULL on failure); free releases it in stream order.
 * When no hook is given the library uses the CUDA stream-ordered pool. */
typedef struct {
  void* (*alloc)(size_t bytes, void* stream, void* ctx);
  void (*free)(void* ptr, void* stream, void* ctx);
  void* ctx;
} pip_allocator;

/* Index build options (Sec. IV: cells of different sizes; interior cells
 * answer at once, boundary cells keep the crossing test). 0 = automatic. */
typedef struct {
  int32_t cell_log2;    /* log2 side of a top-level cell in lattice units (0 = auto) */
  int32_t max_depth;    /* subdivision levels below the top grid (0 = auto, < 0 = none:
                           a uniform grid) */
  int32_t fanout_log2;  /* reported only: a split cell always has 4 x 4 children, held
                           in one 16-byte trie entry (32-byte node with compact leaves) */
  int32_t leaf_edges;   /* split a boundary cell holding more kept edges than this (0 = auto) */
  int32_t size_ratio;   /* split while cell side * ratio > smallest candidate box side
                           (0 = auto: 128, or 48 with compact leaves or the approximate mode;
                           when the trie or leaves outgrow their 27 / 30-bit indices at that
                           ratio, the build falls back to 48, then 16; negative = off) */
  int32_t pts_per_cta;  /* residual points per crossing work item (0 = auto) */
  int32_t stage_depth;  /* shared-memory stages in the crossing kernel: 1 or 2, or
                           negative for none (records read through L1/L2); 0 = auto */
  int32_t cand_mode;    /* 0 = auto, 1 = descend the box hierarchy, 2 = rasterize block boxes */
  int32_t approx_units; /* 0 = exact. > 0: error-bounded approximate mode (Sec. IV): boundary
                           cells are split until their side is at most approx_units lattice
                           units (max_depth is raised as needed), and each such leaf answers
                           every point in it with the exact id of the leaf's centre lattice
                           point, computed at build time, so no crossing test runs at query
                           time. A returned id is then the exact id of a lattice point at
                           Chebyshev distance <= approx_units / 2 of the query point. Leaves
                           whose children overflow a trie node's palette stay exact. */
  int32_t compact_edges; /* compact leaves: a boundary leaf whose kept candidates (at most 3)
                           share at most this many distinct edges is answered in the classify
                           kernel by the exact crossing test (Sec. III-A) on those edges, read
                           from one 32..128-byte record, instead of going through the residual
                           queue and crossing kernel. 1..7 = on with at most that many edges;
                           0 = auto (off: on the state-scale workload the classify kernel's
                           extra work cost more than the residual kernels it saves); negative
                           = off. Always off in approximate mode and for sets of more than
                           2^24 polygons. */
  int32_t compact_early; /* 1: a boundary cell that fits a compact record stops splitting there
                           (a shallower trie; the other boundary cells split to max_depth);
                           0 = auto: the split rules above decide the trie's shape and compact
                           records replace only its leaves. Ignored when compact_edges is off. */
  int32_t bin_residual;  /* radix binning of the residual points by superbin before the
                           crossing test (Sec. III-A: points that share polygons tested
                           together): 1 = on; 0 = auto, or negative: off, the unstaged crossing
                           kernel reads the residual queue in arrival order (on the state
                           workload binning lost at every density measured, 0.4 to 75 residual
                           points per superbin: each point reads its own leaf record either
                           way). The staged crossing kernel (stage_depth 1, 2), the batched
                           form and the no-allocation entry point always bin. Results do not
                           depend on it. */
} pip_build_opts;

/* Facts about a loaded set's index (for tests, tuning and reports). */
typedef struct {
  int64_t n_poly, n_ring, n_vert, n_levels;
  int64_t top_cells;        /* cells of the top grid */
  int64_t table_entries;    /* descriptors: top grid + child tables */
  int64_t leaves;           /* boundary leaf cells (keep the crossing test) */
  int64_t interior_cells;   /* cells answered by one polygon id */
  int64_t empty_cells;      /* cells answered by -1 */
  int64_t superbins;        /* groups of 32 leaf slots, the binning key */
  int64_t leaf_cands;       /* candidate polygons over all leaves */
  int64_t leaf_edges;       /* clipped edges over all leaves */
  int64_t index_bytes;      /* device bytes of top grid, trie nodes, leaf records and their offsets */
  int64_t max_blob_bytes;   /* largest superbin: the records of 32 consecutive leaf slots */
  int32_t cell_log2, fanout_log2, depth, cand_mode;
  int32_t pts_per_cta, stage_depth;
  int32_t grid_x0, grid_y0; /* lattice origin of the grid */
  int64_t grid_nx, grid_ny;
  double build_ms;          /* device time of the last index build */
  int64_t compact_leaves;   /* boundary cells answered from compact records */
  int64_t compact_bytes;    /* bytes of those records (inside the trie-node array) */
  int64_t compact_by_edges[8]; /* compact leaves by number of distinct edges 0..7 */
  int32_t size_ratio;       /* the split ratio the index was built with (after any fallback) */
  int32_t compact_edges;    /* compact leaves' edge limit, or negative when off */
  int64_t nodes_by_level[8]; /* trie nodes (32 bytes each) of levels 1..8 below the top grid */
} pip_set_info_t;

/* Per-call counters of pip_project_ex (read after the stream is synchronised). */
typedef struct {
  int64_t n;          /* points projected */
  int64_t residual;   /* points that fell in boundary cells (crossing tests) */
  int64_t items;      /* crossing work items */
} pip_project_stats;

/* ---- Polygon sets (Sec. III-B data structure; Appendix B) -------------- */

/* Load a polygon set given on the 1e-7 degree lattice and build its index on
 * the device (synchronous: returns after the build finished on `stream`).
 *   vx, vy          [n_vert] int32 vertex coordinates (host or device)
 *   ring_off        [n_ring+1] int64: ring r is vertices [ring_off[r], ring_off[r+1]);
 *                   each ring is closed implicitly (last -> first); a repeated
 *                   closing vertex is allowed; orientation does not matter
 *   poly_ring_off   [n_poly+1] int64: polygon p is rings [poly_ring_off[p], ...[p+1]);
 *                   extra rings are holes or islands (even-odd rule)
 *   parent          n_levels pointers; parent[0][i] is the level-1 node (tract)
 *                   of polygon i, parent[l][j] the level-(l+1) node of level-l
 *                   node j (tract -> county -> region). NULL / 0 = flat set.
 *                   Parent boxes are unions of child boxes: the hierarchy only
 *                   prunes candidates and never changes an answer.
 *   opts, alloc     may be NULL (defaults).
 * Errors: PIP_EINVAL (NULL with n > 0, non-monotone offsets, n_poly >= 2^30),
 * PIP_ERANGE (an edge spans >= 2^31 units), PIP_ENOMEM, PIP_ECUDA. On error
 * *out is NULL and nothing is leaked. */
pip_status pip_set_load_i32(const int32_t* vx, const int32_t* vy, int64_t n_vert,
                            const int64_t* ring_off, int64_t n_ring,
                            const int64_t* poly_ring_off, int32_t n_poly,
                            const int32_t* const* parent, int32_t n_levels,
                            const pip_build_opts* opts, const pip_allocator* alloc,
                            void* stream, pip_set* out);

/* Same, with double vertex coordinates in degrees, quantized by Q on the
 * device (a vertex with an invalid coordinate is PIP_ERANGE). */
pip_status pip_set_load_f64(const double* vx, const double* vy, int64_t n_vert,
                            const int64_t* ring_off, int64_t n_ring,
                            const int64_t* poly_ring_off, int32_t n_poly,
                            const int32_t* const* parent, int32_t n_levels,
                            const pip_build_opts* opts, const pip_allocator* alloc,
                            void* stream, pip_set* out);

/* Rebuild the index of a loaded set with new options (synchronous). */
pip_status pip_set_rebuild(pip_set set, const pip_build_opts* opts, void* stream);

/* Index facts. */
pip_status pip_set_info(pip_set set, pip_set_info_t* info);

/* Free a set and its device memory (synchronises the device first). */
pip_status pip_set_free(pip_set set);

/* ---- Projection (Appendix A findCensusBlock; Sec. IV true-hit filter) --- */

/* out[i] = id((lon[i], lat[i])) for i < n. Asynchronous on `stream` when
 * lon, lat and out are device pointers. With host pointers the call streams
 * the points through the device in chunks (pinned host memory overlaps the
 * copies with compute) and returns after out[] is written. The set's first
 * host-memory call reserves its staging (a second stream, two 16M-point
 * chunk buffers and their scratch: about 1.2 GB of device memory, plus the
 * per-superbin counts), kept until pip_set_free; host-memory calls on one
 * set run one at a time.
 * out must not alias lon or lat. When device-resident, n must stay about
 * 1M below 2^32 per call (the residual queue is indexed with 32 bits and
 * holds n plus two reserved chunks per warp); larger n gives PIP_EINVAL. */
pip_status pip_project(pip_set set, const double* lon, const double* lat, int64_t n,
                       int32_t* out, void* stream);

/* pip_project plus counters; stats (host) is filled after stream sync and
 * may be NULL. */
pip_status pip_project_ex(pip_set set, const double* lon, const double* lat, int64_t n,
                          int32_t* out, void* stream, pip_project_stats* stats);

/* pip_project for callers that cannot allocate device memory during the
 * call. The paper has no counterpart: it is an addition for embedding the
 * join where an allocation is not allowed or not affordable at call time,
 * e.g. code recorded into a CUDA stream capture that must not allocate,
 * latency-critical serving paths where a pool miss or an out-of-memory
 * failure mid-request is unacceptable, and processes that reserve all their
 * device memory up front. lon, lat, out are device pointers; n <= 262144
 * points per call and the set may have at most 524288 superbins
 * (PIP_EINVAL otherwise). The scratch is one fixed device array of about
 * 16 MB inside the library: every GPU context that loads the library holds
 * it until the process exits, whether or not this call is used. The first
 * call on a device looks up that array's device address; make that first
 * call before any stream capture. All calls share the array and it keeps
 * the last call's contents (the call clears what must start at zero), so
 * calls that overlap on the GPU race: serialise them (one stream, or
 * synchronise between calls). Unlike pip_project, which switches to the
 * set's device itself, this call requires the set's device to be the
 * current device (PIP_EINVAL otherwise), so that it never changes devices
 * inside a capture. The looked-up address is kept for the life of the
 * process: after cudaDeviceReset, or any teardown of the device's primary
 * context, do not call it again in that process (the kept address would
 * belong to the old context). Asynchronous on `stream`; results are the
 * same as pip_project's. */
pip_status pip_project_noalloc(pip_set set, const double* lon, const double* lat, int64_t n,
                               int32_t* out, void* stream);

/* Hierarchical outputs (Appendix A assigns state and county codes before the
 * block code): out[i] = the level-`level` ancestor of block id ids[i] through
 * the parent arrays given at load (0 = the block itself, 1 = its tract,
 * 2 = county, 3 = region ...); -1 stays -1. Device pointers, asynchronous.
 * PIP_EINVAL if level exceeds the set's levels. */
pip_status pip_parent_ids(pip_set set, const int32_t* ids, int64_t n, int32_t level, int32_t* out,
                          void* stream);

/* Diagnostic of the failure path of bounded device waits: launches one CTA
 * that waits on an mbarrier nothing completes, giving up after limit_ns
 * (0 < limit_ns <= 1e10) nanoseconds of %globaltimer, as every wait in the
 * library does after 2 s. Returns PIP_ETIMEOUT when the wait ran out (the
 * expected outcome; the context stays usable), PIP_OK if it completed,
 * PIP_EINVAL for a bad limit, PIP_ECUDA on a CUDA error. Synchronises
 * `stream`. The paper has no counterpart. */
pip_status pip_selftest_bounded_wait(int64_t limit_ns, void* stream);

/* Device error word of the set (a bounded device wait that ran out sets it):
 * synchronises `stream`, returns PIP_OK or PIP_ETIMEOUT and clears it. */
pip_status pip_set_check(pip_set set, void* stream);

/* ---- Batched form: many queries over many sets in one launch ------------ */

typedef struct {
  pip_set set;
  const double* lon;   /* device pointers */
  const double* lat;
  int64_t n;
  int32_t* out;
} pip_query;

/* A plan holds the device buffers and a CUDA graph of one persistent,
 * work-stealing launch (classify, bin, crossing phases separated by
 * grid-wide barriers with bounded waits). max_points / max_queries bound
 * what one launch may carry. */
pip_status pip_plan_create(int64_t max_points, int32_t max_queries, void* stream,
                           pip_plan* out);
/* Run q[0..n_q) in one graph launch on `stream` (asynchronous). The same
 * results as n_q separate pip_project calls, bit for bit. */
pip_status pip_plan_run(pip_plan plan, const pip_query* q, int32_t n_q, void* stream);
/* Synchronise `stream` and report a device timeout of the last run. */
pip_status pip_plan_check(pip_plan plan, void* stream);
pip_status pip_plan_destroy(pip_plan plan);

/* Autotuner for a plan: time runs of q[0..n_q) with points per crossing
 * item in {128, 256, 512, 1024} and staging off / on, keep the fastest
 * (written to *pts_per_cta and *staged when not NULL). Synchronous. */
pip_status pip_plan_tune(pip_plan plan, const pip_query* q, int32_t n_q, void* stream,
                         int32_t* pts_per_cta, int32_t* staged);

/* One-shot convenience: create a plan, run, destroy (synchronous). */
pip_status pip_project_batch(const pip_query* q, int32_t n_q, void* stream);

/* Autotuner: time candidate index shapes (cell_log2 - 1 .. + 1, split ratio
 * 16 / 32 / 64 / 128, 4 or 8 kept edges per leaf), then compact leaves (3
 * edges) on the fastest shape, then crossing work items (pts_per_cta
 * 128 .. 1024, stage_depth none / 1 / 2), each on a sample of the set's
 * queries (device pointers), and rebuild the set with the fastest; the
 * chosen options are written to *chosen (may be NULL). Synchronous. Shapes
 * whose index fails to build (too large) are skipped. */
pip_status pip_set_tune(pip_set set, const double* lon, const double* lat, int64_t n_sample,
                        void* stream, pip_build_opts* chosen);

/* ---- Served form: continuous batching over resident sets ---------------- */

typedef struct {
  int32_t n_streams;          /* concurrent launches in flight (0 = 2) */
  int64_t mem_budget_bytes;   /* device bytes reserved at creation for in-flight requests
                                 (0 = 1/4 of the memory free at creation) */
  int64_t max_batch_points;   /* points coalesced into one launch (0 = 1<<24) */
  int32_t max_batch_queries;  /* requests coalesced into one launch (0 = 1024) */
  int32_t max_pending;        /* queued requests before submit says PIP_EBUSY (0 = 1<<20) */
} pip_server_opts;

typedef struct {
  int64_t submitted, completed, rejected, launches;
  int64_t points;
  double p50_us, p99_us, max_us, mean_batch_queries;
} pip_server_stats_t;

/* Start a serving loop over resident sets (the sets must outlive it). A
 * dispatcher thread admits requests into slots and collects finished
 * launches; while launches are in flight, and for 200 us after the last
 * activity, it polls (yielding the CPU between polls) instead of sleeping,
 * which keeps a small request's latency near the kernel time at the cost of
 * one busy host thread. Each slot's batched plan is sized for all the sets
 * and its launch graphs are captured here, so no request waits for an
 * allocation or a graph capture. */
pip_status pip_server_create(const pip_set* sets, int32_t n_sets, const pip_server_opts* opts,
                             pip_server* out);
/* Queue a request of any size n >= 0: lon/lat/out are host memory (pinned
 * is fastest) that stays valid until pip_server_wait reports it done. The
 * device memory for requests in flight is reserved once, at
 * pip_server_create, from mem_budget_bytes (default: a quarter of the memory
 * free at that moment) and split into n_streams slots of equal point
 * capacity; admission is then against a free slot and its capacity, not
 * against memory free at run time. A request that arrives while others run
 * joins the next launch whose slot frees up (continuous batching). A request
 * larger than one slot is queued as consecutive parts of at most a slot each
 * and its ticket completes when the last part is done; its results equal a
 * single pip_project call. PIP_EBUSY when the queue (in parts) would exceed
 * max_pending; PIP_EINVAL for a bad set, NULL buffers with n > 0 or a
 * stopping server. */
pip_status pip_server_submit(pip_server srv, int32_t set, const double* lon, const double* lat,
                             int64_t n, int32_t* out, uint64_t* ticket);
/* Wait up to timeout_us (< 0 = forever) for a ticket (polling for up to
 * 300 us before sleeping). PIP_ETIMEOUT if not done. One thread waits per
 * ticket; once a wait reports it done (PIP_OK or the launch's error), the
 * ticket is forgotten. */
pip_status pip_server_wait(pip_server srv, uint64_t ticket, int64_t timeout_us);
/* Latency percentiles of completed requests since creation or the last reset
 * (over the most recent 4,194,304 completions when there were more). */
pip_status pip_server_stats(pip_server srv, pip_server_stats_t* st, int32_t reset);
void pip_server_destroy(pip_server srv);

/* ---- Diagnostics --------------------------------------------------------- */

/* Q on the device for n doubles (device pointers): q[i], valid[i] (0/1).
 * Exposes the device quantizer so tests can compare it bit for bit. */
pip_status pip_quantize(const double* v, int64_t n, int32_t* q, uint8_t* valid, void* stream);

/* Candidate polygons per top-level cell, for checking that hierarchy
 * descent and box rasterization agree: fills off[top_cells+1] and
 * ids[cap] (host arrays); returns PIP_EINVAL if cap is too small
 * (off[top_cells] then holds the needed size). */
pip_status pip_set_top_candidates(pip_set set, int32_t cand_mode, int64_t* off, int32_t* ids,
                                  int64_t cap);

/* Per-stage device timing of pip_project on a set, taken with CUDA events
 * recorded on the call's stream around the stages (no synchronisation in
 * the calls themselves). enable = capacity in calls (0 disables and frees).
 * pip_profile_read synchronises the device and returns, for up to *n calls
 * recorded since enabling (or the last read), the milliseconds of
 * classify (K1), bin (K2: scan, scatter, work items) and cross (K3), each
 * array of length *n; *n is updated to the number returned. */
pip_status pip_profile_enable(pip_set set, int32_t capacity);
pip_status pip_profile_read(pip_set set, double* k1_ms, double* bin_ms, double* k3_ms, int32_t* n);

/* Which cell of the set's index answers each lattice point: code[i] for
 * the point (qx[i], qy[i]) (device pointers, asynchronous) is a kind in bits
 * 0-7 and the trie depth of the answering cell in bits 8-15 (0 = a top-grid
 * cell). Kinds: EMPTY and INTERIOR cells answer without a crossing test
 * (Sec. IV, true-hit filtering); COMPACT leaves answer with the test inside
 * the classify kernel; RESIDUAL leaves send the point to the crossing
 * kernel; OUTSIDE = beyond the grid (answered -1). For tests and tuning:
 * the projection never calls it. */
enum { PIP_LOC_EMPTY = 0, PIP_LOC_INTERIOR = 1, PIP_LOC_RESIDUAL = 2, PIP_LOC_COMPACT = 3,
       PIP_LOC_OUTSIDE = 4 };
pip_status pip_locate(pip_set set, const int32_t* qx, const int32_t* qy, int64_t n, uint32_t* code,
                      void* stream);

/* Kernel launches the library has issued in this process so far. */
int64_t pip_kernel_launches(void);

/* Thread-local message of the last failing call on this thread. */
const char* pip_last_error(void);

/* ABI version: major * 10000 + minor * 100 + patch. */
int32_t pip_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PIP_H */
