// Internal declarations of the GB300 DF Louvain library (sm_103a).
//
// Device data layout (all arrays in HBM, owned by the handle):
//   slack CSR of G^t   off[n] (u64 arc offset), deg[n] (u32, slots in use),
//                      cap[n], srt[n] (sorted prefix), ntomb[n] (deleted arcs
//                      kept as weight-0 tombstones), arcs[pool] as uint2
//                      {neighbour, weight}; every row starts on an even arc
//                      index (16-byte aligned)
//   state              K[n], Sigma[n] (int64), csize[n] (int32), C[n] (u32)
//   super-vertex CSR   two ping-pong graphs (off, deg, arcs) for passes >= 1
//   frontier           bitmaps (n/32 words) + per (sub-step class, degree bin)
//                      vertex lists, double-buffered (current / next)
//   control block      counters, error word and 128-bit sums, mirrored into
//                      pinned host memory once per iteration
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/dfl.h"

namespace dfl {

typedef __int128 i128;
typedef unsigned __int128 u128;

// ---------------------------------------------------------------------------
// Compile-time configuration
// ---------------------------------------------------------------------------
constexpr int kWarp = 32;
constexpr int kBins = 4;            // degree bins of the local-moving kernels
constexpr uint32_t kBinWarp = 32;   // deg <= 32: registers only (largest bin-0 limit)
constexpr uint32_t kBinWarpDefault = 8;  // default bin-0 limit: 8 lanes per vertex, 4 vertices a warp
constexpr uint32_t kBinWarpHash = 256;   // deg <= 256: one warp, shared-memory table
constexpr uint32_t kBinBlock = 4096;     // deg <= 4096: one block, shared-memory table
                                          // larger: one block, global-memory table
constexpr uint32_t kMaxSubsteps = 8;
constexpr uint32_t kEmpty = 0xFFFFFFFFu;  // empty hash-table key

// Error bits raised by kernels (ctrl.err)
enum : uint32_t {
  kErrInvalid = 1u,
  kErrNotFound = 2u,
  kErrOverflow = 4u,
  kErrInternal = 8u,  // a hash table overflowed or an index check failed
  kErrTimeout = 16u,  // a bounded wait of the persistent iteration kernel gave up
};

// ---------------------------------------------------------------------------
// Control block (device), mirrored to pinned host memory.
// ---------------------------------------------------------------------------
struct Ctrl {
  unsigned long long s_lo;           // sum of the low 32 bits of the movers' dQ numerators
  unsigned long long s_hi;           // sum of the high parts (value = s_hi * 2^32 + s_lo)
  unsigned long long processed;      // frontier vertices processed in the iteration
  unsigned long long moved;          // movers in the iteration
  unsigned long long move_bytes;     // algorithmic bytes of the decide kernels
  unsigned int movers;               // movers of the current sub-step (list length)
  unsigned int big_movers;           // ... of them listed for k_commit to mark the neighbours of
  unsigned int err;                  // kErr* bits
  unsigned int pad_err;
  unsigned int count[2][kMaxSubsteps][kBins];  // frontier list lengths [buffer][class][bin]
  // batch apply
  unsigned long long reloc_need;     // arc slots needed for relocated rows
  unsigned long long scratch_need;   // scratch slots for in-place merges
  long long m2_delta;                // change of 2m by the batch
  unsigned int max_deg;              // largest new degree of a touched row
  unsigned int rows;                 // touched rows
  long long arc_delta;               // change of the live arc count by the batch
  unsigned int rebuild_rows;         // rows rebuilt by the batch
  unsigned int pad2;
  unsigned long long skipped;        // frontier vertices without arcs (processed, not queued)
  unsigned long long ever_count;     // vertices newly added to the first-pass processed set
  // persistent iteration kernel: per sub-step parity, movers, listed
  // high-degree movers, work units taken, vertices left to the part blocks;
  // chunk items of each class; grid barrier
  unsigned int it_movers[2], it_nbig[2], it_work[2], it_bignd[2];
  unsigned int it_items[kMaxSubsteps];
  unsigned int bar_count, bar_gen;
  long long m2v;                     // 2m of the current local-moving call
  unsigned int npairs;               // distinct (u, v) pairs of the batch (hashed apply)
  unsigned int max_app;              // most new arcs of one rebuilt row
  unsigned long long extra_top;      // new arcs of rebuilt rows
  unsigned long long pool_top;       // first free arc slot of the pool
  unsigned long long scratch_top;
  // misc reductions
  unsigned long long red_a;
  unsigned long long red_b;
  unsigned long long red_c;
  unsigned int red_u;
  unsigned int apply_go;             // the batch apply's gate: the batch is written (1) or nothing is (0)
  unsigned int apply_defer;          // ... with rows to rebuild (by the multi-block rebuild kernel)
  unsigned int pad3;
};

// A CSR whose rows are addressed by (offset, degree): the slack CSR of G^t
// and the super-vertex graphs with holes (Alg. 6) share this view.
struct GraphView {
  const unsigned long long* off;
  const uint32_t* deg;
  const uint2* arcs;
  uint32_t nv;
};

struct SuperGraph {
  unsigned long long* off = nullptr;
  uint32_t* deg = nullptr;
  uint2* arcs = nullptr;
  uint64_t arc_cap = 0;
  uint32_t nv_cap = 0;
};

// Frontier list layout: segment (class s, bin b) starts at off[s*kBins+b]
// and holds at most the number of ids in [0, n) of class s.
struct Segs {
  uint32_t off[kMaxSubsteps * kBins];
  uint32_t cap[kMaxSubsteps * kBins];
  uint32_t hi[kBins - 1];  // largest degree of bins 0..2 (tuning; bin 3 takes the rest)
  // group: a vertex's sub-step class comes from its id within its own graph
  // (first vertex of each graph at the current level, device memory)
  const uint32_t* goff;
  uint32_t ng;
};

struct Handle {
  uint32_t n = 0;
  cudaStream_t stream = nullptr;
  dfl_options opt;
  std::string err;
  int device = 0;

  // slack CSR of G^t
  unsigned long long* off = nullptr;
  uint32_t* deg = nullptr;
  uint32_t* cap = nullptr;
  uint32_t* srt = nullptr;    // length of the sorted prefix of each row
  uint32_t* ntomb = nullptr;  // tombstones (weight-0 arcs) in each row
  uint2* arcs = nullptr;
  uint64_t pool_cap = 0;   // arc slots allocated
  uint64_t pool_top = 0;   // first free slot (host mirror)
  uint64_t num_arcs = 0;   // arcs in use
  uint32_t max_deg = 0;    // upper bound of the degrees of G^t

  // community state
  long long* K = nullptr;
  long long* Sigma = nullptr;
  int* csize = nullptr;
  uint32_t* C = nullptr;
  long long m2 = 0;
  bool have_communities = false;

  // pending batch arcs (sorted keys and weights of every dfl_apply_batch
  // since the last update)
  unsigned long long* pend_key = nullptr;
  uint32_t* pend_w = nullptr;
  uint64_t pend_count = 0, pend_cap = 0;
  uint32_t key_shift = 0;  // key = u << (key_shift + 1) | v << 1 | type
  uint32_t key_bits = 0;

  // Louvain work buffers (sized n)
  uint32_t* Ctop = nullptr;     // dendrogram: vertex of G^t -> vertex of G'
  uint32_t* Cs = nullptr;       // membership of the super-vertex graph
  long long* Ks = nullptr;
  long long* Ss = nullptr;
  int* sizes = nullptr;
  uint32_t* used = nullptr;     // n+1: flags, then exclusive scan = new ids
  uint32_t* cnt = nullptr;      // n+1: community vertex counts / offsets
  unsigned long long* tdeg = nullptr;  // n+1: community total degree / super offsets
  uint32_t* fillc = nullptr;    // n
  uint32_t* members = nullptr;  // n
  SuperGraph sg[2];

  // frontier
  uint32_t words = 0;           // bitmap words = ceil(n / 32)
  uint32_t* fbits[2] = {nullptr, nullptr};
  uint32_t* rbits = nullptr;    // affected range (DS first pass)
  uint32_t* ever = nullptr;     // ever processed in the first pass
  uint32_t* lists[2] = {nullptr, nullptr};  // kBins * n ids each, split by `segs`
  Segs segs;
  uint32_t segs_k = 0;          // sub-step count the layout was made for
  uint32_t* mv_i = nullptr;     // movers of a sub-step
  uint32_t* mv_c = nullptr;
  uint32_t* mv_d = nullptr;

  // DS marking scratch
  uint32_t* dsV = nullptr;
  uint32_t* dsE = nullptr;
  uint32_t* dsC = nullptr;

  // batch apply scratch (grown on demand)
  unsigned long long* b_key = nullptr;
  uint32_t* b_w = nullptr;
  unsigned long long* b_key2 = nullptr;
  uint32_t* b_w2 = nullptr;
  uint64_t b_cap = 0;
  uint32_t* b_rowlist = nullptr;   // row-head positions
  unsigned long long* b_pos = nullptr;  // per run head: position in row | found << 63
  uint32_t* b_wnew = nullptr;      // per run head: new weight
  uint32_t* b_flag = nullptr;      // per arc: run/row head flags (see batch.cu)
  long long* b_delta = nullptr;    // per run head: weight change of the arc
  uint32_t* b_newdeg = nullptr;    // per row head: degree after the batch
  uint32_t* b_newtomb = nullptr;   // per row head: tombstones after the batch
  uint32_t* b_cum = nullptr;       // per run head: appended runs before it in its row
  uint32_t* b_rebuild = nullptr;   // row heads of rebuilt rows
  dfl_edge* b_edges = nullptr;     // staging copy of the caller's edges
  uint64_t b_edges_cap = 0;
  uint2* scratch = nullptr;        // merge scratch
  uint64_t scratch_cap = 0;
  // hashed apply: pair table (capacity h_cap, a power of two), per-vertex
  // scratch counters (zero at rest), touched rows, new arcs of rebuilt rows
  unsigned long long* h_keys = nullptr;
  uint32_t* h_ndel = nullptr;
  uint32_t* h_wdel = nullptr;
  unsigned long long* h_wins = nullptr;
  uint32_t* h_slot = nullptr;
  uint32_t* h_wnew = nullptr;
  uint32_t* h_flag = nullptr;
  long long* h_delta = nullptr;
  uint32_t* h_pairs = nullptr;
  uint64_t h_cap = 0;
  uint32_t* r_app = nullptr;
  int* r_tomb = nullptr;
  int* r_live = nullptr;
  uint32_t* r_state = nullptr;
  uint32_t* r_reg = nullptr;
  uint32_t* h_rows = nullptr;
  uint2* h_extra = nullptr;
  uint64_t h_rows_cap = 0;

  // generic scratch
  void* tmp = nullptr;
  uint64_t tmp_cap = 0;
  uint2* gtable = nullptr;         // global hash tables of the largest bin
  uint64_t gtable_cap = 0;
  uint32_t* bigmv = nullptr;       // high-degree movers of a sub-step (marked by k_mark_big)
  uint64_t bigmv_cap = 0;
  uint2* aggq = nullptr;           // high-degree members of giant communities (aggregation)
  uint64_t aggq_cap = 0;
  // decisions of the largest bin: per list position its table and list
  // offsets, chunk prefix, occupied-slot count, finished part blocks and
  // weight to the own community (the last two zero at rest); per part
  // results; the global tables (empty at rest) and occupied-slot lists
  unsigned long long* g_toff = nullptr;
  unsigned long long* g_loff = nullptr;
  uint32_t* g_cpre = nullptr;
  uint32_t* g_ndist = nullptr;
  uint32_t* g_done = nullptr;
  unsigned long long* g_hd = nullptr;
  uint64_t g_items_cap = 0;
  void* g_res = nullptr;
  uint64_t g_res_cap = 0;
  uint32_t* g_tkeys = nullptr;
  uint32_t* g_tvals = nullptr;
  uint64_t g_tab_cap = 0;
  uint2* g_tlist = nullptr;
  uint64_t g_lst_cap = 0;

  // auxiliary streams for the concurrent degree bins of a sub-step
  cudaStream_t aux[kBins - 1] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[kBins - 1] = {nullptr, nullptr, nullptr};

  // control
  Ctrl* ctrl = nullptr;       // device
  Ctrl* hctrl = nullptr;      // pinned host mirror
  // control blocks of the hashed batch apply (validation results and gate),
  // two that alternate: an apply's last kernel clears the next one's, so an
  // apply starts without a memset.  They follow `ctrl` in one allocation
  // (actrl = ctrl + 1, hactrl = hctrl + 1), so that one copy reads the
  // local-moving control block and a pending apply's together.  Separate
  // from `ctrl`, so that a DF update can be enqueued behind the apply before
  // the host has read it.
  Ctrl* actrl = nullptr;
  Ctrl* hactrl = nullptr;
  int apar = 0;  // the block the next apply uses
  // a batch apply enqueued without a host wait (dfl_step): the first control
  // read of the update that follows settles it
  struct PendingApply {
    bool active = false;
    bool small = false;  // the single-block path
    int par = 0;         // its control block: actrl[par]
    uint64_t na = 0;     // arcs of the batch (2 per edge)
    int rc = 0;          // how it settled: DFL_OK, a DFL_ERR code or kApplyRetry*
  } papply;
  bool ever_clear = false;  // DF marking cleared `ever` for the update that follows

  // statistics
  dfl_stats_t stats;
  std::vector<uint64_t> trace;  // 4 per first-pass iteration
  uint64_t launches = 0;

  // profiling
  struct Ev {
    cudaEvent_t a, b;
    int cls;
  };
  std::vector<Ev> ev_pending;
  // captured local-moving iteration per list-buffer parity (base graph only)
  struct IterGraph {
    cudaGraphExec_t exec = nullptr;
    std::vector<char> key;
    std::vector<Ev> evs;
    uint64_t kernels = 0;
    uint64_t class_launches[DFL_PROF_CLASSES] = {0};
    uint64_t last_use = 0;
  };
  static constexpr int kGraphCache = 4;  // graphs kept per parity (DF, ND/static, DS, ...)
  IterGraph igraph[2][kGraphCache];
  uint64_t graph_use = 0;                 // LRU clock
  uint64_t graph_captures = 0;
  double graph_capture_ms = 0;
  std::vector<cudaEvent_t> ev_free;
  dfl_profile_t prof;

  // launch-shape tuning of local-moving (never changes results)
  dfl_tuning tune{kBinWarpDefault, kBinWarpHash, kBinBlock, 256};

  // group: ngraphs > 0 independent graphs held as one disjoint union
  uint32_t ngraphs = 0;
  std::vector<uint32_t> goff0;         // first vertex of each graph (ngraphs + 1)
  std::vector<long long> gm2;          // 2m of each graph
  std::vector<uint8_t> gfin;           // graph finished the current Louvain run
  std::vector<dfl_stats_t> gstats;
  uint32_t* d_goff0 = nullptr;         // device copy of goff0
  uint32_t* d_goff = nullptr;          // first vertex of each graph at the current level
  uint32_t* d_gnext = nullptr;         // the next level's offsets (gathered scan)
  long long* d_gm2 = nullptr;
  uint8_t* d_gdone = nullptr;          // graph skipped by local-moving
  uint8_t* d_gflag = nullptr;          // graphs to finalize
  unsigned long long* d_gS = nullptr;  // per graph S limbs (lo, hi) of the iteration
  unsigned long long* d_gsum = nullptr;  // per graph reduction slots (3 each)
  uint8_t* h_gdone = nullptr;          // pinned host mirrors
  unsigned long long* h_gS = nullptr;
  uint32_t* Cfin = nullptr;            // final labels of the graphs (union ids)
  dfl_edge* gb_edges = nullptr;        // staged group batch (union ids)
  uint64_t gb_cap = 0;
  uint64_t* d_eoff = nullptr;          // per graph edge offsets of a group batch (2 x (ngraphs + 1))
};

// ---------------------------------------------------------------------------
// Error handling
// ---------------------------------------------------------------------------
int set_error(Handle* h, int code, const std::string& msg);

#define DFL_CUDA(h, call)                                                          \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return ::dfl::set_error((h), e_ == cudaErrorMemoryAllocation ? DFL_ERR_NOMEM \
                                                                   : DFL_ERR_CUDA, \
                              std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define DFL_TRY(expr)        \
  do {                       \
    int r_ = (expr);         \
    if (r_ != DFL_OK) return r_; \
  } while (0)

// Every device allocation of the library goes through dev_malloc, so that a
// test can make allocations fail on the host (dfl_test_fail_allocations):
// after that many more successful allocations every further one returns
// cudaErrorMemoryAllocation without calling CUDA.
cudaError_t dev_malloc_bytes(void** p, size_t bytes);
template <typename T>
inline cudaError_t dev_malloc(T** p, size_t bytes) {
  return dev_malloc_bytes(reinterpret_cast<void**>(p), bytes);
}

// Launch bookkeeping: counts launches and, with DFL_FLAG_PROFILE, brackets
// the launch with CUDA events of class `cls`.
struct LaunchScope {
  Handle* h;
  int cls;
  cudaStream_t s;
  cudaEvent_t a = nullptr, b = nullptr;
  LaunchScope(Handle* h_, int cls_, cudaStream_t s_);
  LaunchScope(Handle* h_, int cls_) : LaunchScope(h_, cls_, h_->stream) {}
  ~LaunchScope();
};

int check_launch(Handle* h, const char* what);
cudaError_t record_timing_event(cudaEvent_t e, cudaStream_t s);
cudaEvent_t take_event(Handle* h);  // a timing event from the handle's pool (nullptr if none)

// Programmatic dependent launch (sm_90 and later) for chains of short
// dependent kernels on one stream: a kernel launched with launch_pdl may be
// scheduled while its predecessor is still running; pdl_wait() at its start
// waits until the predecessor has completed and its writes are visible, then
// allows its own successor to be scheduled.  The kernel gets past the
// launch latency that would otherwise separate the two (about 3.5 us between
// dependent stream launches on this GPU).  In a kernel launched the ordinary
// way both instructions return at once.
__device__ __forceinline__ void pdl_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// The wait alone, for kernels that share the GPU with concurrent work: their
// successor is then launched when they exit rather than when they start, so
// that its blocks do not wait on SM resources the concurrent kernels need.
__device__ __forceinline__ void pdl_wait_only() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint32_t substep_class(uint32_t i, uint32_t k) {
  return uint32_t((uint64_t(i * 0x9E3779B1u) * k) >> 32);
}

__host__ __device__ __forceinline__ uint32_t graph_of(const uint32_t* goff, uint32_t ng, uint32_t v) {
  uint32_t lo = 0, hi = ng;  // largest g with goff[g] <= v
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) >> 1;
    if (goff[mid] <= v) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Sub-step class of vertex v of the current graph (a group's vertices by
// their id within their own graph, so each graph gets its own schedule).
__device__ __forceinline__ uint32_t vertex_class(uint32_t v, uint32_t k, const Segs& s) {
  if (s.ng) v -= s.goff[graph_of(s.goff, s.ng, v)];
  return substep_class(v, k);
}

__host__ __device__ __forceinline__ uint32_t degree_bin(uint32_t d, const Segs& s) {
  return d <= s.hi[0] ? 0u : d <= s.hi[1] ? 1u : d <= s.hi[2] ? 2u : 3u;
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Home slot hashes of the open-addressing tables: the low bits of the id
// times an odd constant (a bijection on the low bits, so the dense ids of an
// aggregated graph land without collisions).  Aggregation and local-moving
// use different multipliers: aggregation writes a super-vertex's row in its
// table's slot order, and with the same multiplier a run of consecutive arcs
// would fill a narrow window of a local-moving table densely (R-MAT 2^22,
// second pass: probe runs of up to 1,000 slots in the 2,048-slot chunk
// tables of the largest-degree vertices).
__device__ __forceinline__ uint32_t hash32(uint32_t x) { return x * 0x9E3779B1u; }       // aggregation
__device__ __forceinline__ uint32_t hash_move(uint32_t x) { return x * 0x85EBCA6Bu; }    // local-moving

// Warp-wide maximum of (score, -c): larger score wins, ties to the smaller c.
// Lanes without a candidate pass have = false.
__device__ __forceinline__ void warp_argmax(bool& have, i128& score, uint32_t& c) {
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    unsigned long long lo = (unsigned long long)(u128)score;
    unsigned long long hi = (unsigned long long)((u128)score >> 64);
    unsigned long long olo = __shfl_xor_sync(0xFFFFFFFFu, lo, s);
    unsigned long long ohi = __shfl_xor_sync(0xFFFFFFFFu, hi, s);
    uint32_t oc = __shfl_xor_sync(0xFFFFFFFFu, c, s);
    bool oh = __shfl_xor_sync(0xFFFFFFFFu, have ? 1 : 0, s) != 0;
    i128 os = (i128)(((u128)ohi << 64) | (u128)olo);
    if (oh && (!have || os > score || (os == score && oc < c))) {
      have = true;
      score = os;
      c = oc;
    }
  }
}

// Bitmap helpers
__device__ __forceinline__ bool bit_test(const uint32_t* bits, uint32_t i) {
  return (bits[i >> 5] >> (i & 31u)) & 1u;
}
// Returns true if the bit was newly set.
__device__ __forceinline__ bool bit_set(uint32_t* bits, uint32_t i) {
  uint32_t m = 1u << (i & 31u);
  return (atomicOr(bits + (i >> 5), m) & m) == 0;
}

// Append vertex v (if valid) to frontier list `key` = class * kBins + bin of
// buffer `buf`; one atomic per distinct key in the warp (the distinct keys
// are visited one by one with ballots).  Every lane of the warp must call it.
__device__ __forceinline__ void append_vertex(uint32_t v, bool valid, uint32_t key,
                                              uint32_t* lists, const Segs& seg, Ctrl* ctrl,
                                              int buf) {
  const unsigned lane = threadIdx.x & 31u;
  unsigned act = __ballot_sync(0xFFFFFFFFu, valid);
  while (act) {
    const unsigned leader = __ffs(act) - 1;
    const uint32_t kl = __shfl_sync(0xFFFFFFFFu, key, leader);
    const unsigned grp = __ballot_sync(0xFFFFFFFFu, valid && key == kl);
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(&ctrl->count[buf][kl / kBins][kl % kBins], __popc(grp));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    if ((grp >> lane) & 1u) {
      const uint32_t r = base + __popc(grp & ((1u << lane) - 1u));
      if (r < seg.cap[kl]) lists[seg.off[kl] + r] = v;
      else atomicOr(&ctrl->err, kErrInternal);
    }
    act &= ~grp;
  }
}

// Frontier lists from a bitmap, one bitmap word per thread: a block counts
// its vertices per list key in shared memory, reserves each key's range with
// one global atomic, then writes (so a dense frontier does not funnel every
// vertex through the few global list counters).
__device__ __forceinline__ void lists_bits_body(const uint32_t* __restrict__ bits, uint32_t words,
                                                uint32_t nv, const uint32_t* __restrict__ deg,
                                                uint32_t* lists, const Segs& seg, Ctrl* ctrl, int buf,
                                                uint32_t k) {
  __shared__ uint32_t s_cnt[kMaxSubsteps * kBins];
  __shared__ uint32_t s_base[kMaxSubsteps * kBins];
  const uint32_t nkeys = k * kBins;
  for (uint64_t w0 = blockIdx.x * uint64_t(blockDim.x); w0 < words; w0 += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t w = w0 + threadIdx.x;
    const uint32_t word = w < words ? bits[w] : 0u;
    if (!__syncthreads_or(word != 0u)) continue;  // block-uniform: no vertex in this tile
    if (threadIdx.x < nkeys) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    for (uint32_t x = word; x; x &= x - 1) {
      const uint32_t v = uint32_t(w * 32 + __ffs(x) - 1);
      if (v >= nv) break;
      atomicAdd(&s_cnt[vertex_class(v, k, seg) * kBins + degree_bin(deg[v], seg)], 1u);
    }
    __syncthreads();
    if (threadIdx.x < nkeys) {
      const uint32_t c = s_cnt[threadIdx.x];
      s_base[threadIdx.x] = c ? atomicAdd(&ctrl->count[buf][threadIdx.x / kBins][threadIdx.x % kBins], c) : 0u;
      s_cnt[threadIdx.x] = 0;
    }
    __syncthreads();
    for (uint32_t x = word; x; x &= x - 1) {
      const uint32_t v = uint32_t(w * 32 + __ffs(x) - 1);
      if (v >= nv) break;
      const uint32_t key = vertex_class(v, k, seg) * kBins + degree_bin(deg[v], seg);
      const uint32_t r = s_base[key] + atomicAdd(&s_cnt[key], 1u);
      if (r < seg.cap[key]) lists[seg.off[key] + r] = v;
      else atomicOr(&ctrl->err, kErrInternal);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Host-side entry points of the other translation units
// ---------------------------------------------------------------------------
// prim.cu
void make_segs(Handle* h, uint32_t k);
int ensure_tmp(Handle* h, uint64_t bytes);
int scan_u32(Handle* h, const uint32_t* in, uint32_t* out, uint64_t n);  // exclusive, out[n] = total
int scan_u64(Handle* h, const unsigned long long* in, unsigned long long* out, uint64_t n);
int sort_pairs(Handle* h, unsigned long long* key, uint32_t* val, unsigned long long* key2,
               uint32_t* val2, uint64_t n, uint32_t bits);  // result in key/val
int fill_u32(Handle* h, uint32_t* p, uint32_t v, uint64_t n);
int iota_u32(Handle* h, uint32_t* p, uint64_t n);
int fill_i32(Handle* h, int* p, int v, uint64_t n);
int copy_i64(Handle* h, long long* dst, const long long* src, uint64_t n);
int lists_from_bits(Handle* h, const uint32_t* bits, uint32_t nv, const uint32_t* deg, int buf,
                    uint32_t substeps);
// (also zeroes clear[0, clear_words), a bitset no one else touches meanwhile)
__global__ void k_lists_bits(const uint32_t* __restrict__ bits, uint32_t words, uint32_t nv,
                             const uint32_t* __restrict__ deg, uint32_t* lists, Segs seg, Ctrl* ctrl,
                             int buf, uint32_t k, uint32_t* __restrict__ clear, uint32_t clear_words);
int lists_all(Handle* h, uint32_t nv, const uint32_t* deg, int buf, uint32_t substeps);
int bits_to_bytes(Handle* h, const uint32_t* bits, uint8_t* out, uint32_t n);
int bytes_to_bits(Handle* h, const uint8_t* in, uint32_t* bits, uint32_t n);
uint64_t popcount_bits(Handle* h, const uint32_t* bits, uint32_t words, int* rc);

// graph.cu
int graph_build(Handle* h, const unsigned long long* off_in, const uint32_t* idx_in,
                const uint32_t* w_in, uint64_t nnz);
int weighted_degrees(Handle* h);  // K from scratch, m2 on host
int compact_pool(Handle* h, uint64_t* before, uint64_t* after);  // dfl_compact
int recompute_aux(Handle* h);      // K, 2m, Sigma, sizes from scratch (DFL_FLAG_RECOMPUTE_AUX)
int modularity_parts(Handle* h, i128* num, i128* den);
int graph_export(Handle* h, uint64_t* off, uint32_t* idx, uint32_t* w, bool device_out);
int recompute_sigma_sizes(Handle* h, const uint32_t* C);

// batch.cu
// Results of settling a hashed batch apply besides DFL_OK and the DFL_ERR
// codes: nothing was written, and the batch must be enqueued again (its
// buffers grew) or take the sort-based path (a rebuilt row gains more new
// arcs than a block sorts in shared memory).
constexpr int kApplyRetryGrown = 1;
constexpr int kApplyRetrySorted = 2;
// Enqueue the batch's apply with no host wait; h->papply describes it.
int apply_batch_begin(Handle* h, const dfl_edge* del, uint64_t nd, const dfl_edge* ins, uint64_t ni,
                      int mem_kind);
// Copy the apply's control block to the host (ordered on the handle's
// stream, no wait) / settle it from that copy: on success the host mirrors
// (2m, the pending count, the pool top, the arc count, the largest degree)
// take the batch; otherwise the per-row scratch counters are cleared and the
// error or the retry is returned.
int copy_apply_ctrl(Handle* h);
int settle_apply(Handle* h);
// Upper bounds of the live arc count, the pool top and the largest degree
// while an enqueued apply has not settled (the exact values once it has).
uint64_t live_arcs_bound(const Handle* h);
uint64_t pool_top_bound(const Handle* h);
uint32_t max_deg_bound(const Handle* h);
int apply_batch(Handle* h, const dfl_edge* del, uint64_t nd, const dfl_edge* ins, uint64_t ni,
                int mem_kind);
int mark(Handle* h, int mode, bool* all, bool* use_range, uint64_t* initial);

// move.cu
struct MoveArgs {
  GraphView g;
  uint32_t* graph_iters = nullptr;  // group: iterations each graph ran (host, ngraphs)
  uint32_t* C;
  const long long* K;
  long long* Sigma;
  int* size;
  long long m2;
  uint32_t max_deg;  // upper bound of the degrees of g
  bool use_range;
  bool track_ever;
  bool prefer_host = false;  // launch from the host unless DFL_FLAG_GRAPH asks for replay
  // upper bound of the initial frontier's vertex count (DF: the pending
  // batch arcs); chooses launch shapes for a replayed first iteration
  uint64_t frontier_hint = ~0ull;
};
// A frontier list of a sub-step class shorter than this is decided by the
// per-vertex kernels of bin 0 (W lanes a vertex) instead of the
// thread-per-vertex kernel: with few vertices the latter leaves the SMs to
// the largest-degree chain less well (R-MAT 2^22, DF at 1e-3|E|: 0.44 vs
// 0.49-0.52 ms per batch), while on full frontiers it is the faster one.
constexpr uint64_t kSmallList = 32768;
// Below this many pending batch arcs a DF or DS update launches its
// iterations from the host even when graph replay is allowed: a frontier of
// a few vertices leaves most bins empty, and skipping them beats replaying
// a graph that launches every bin (R-MAT 2^22: 0.19 vs 0.23 ms at 3 edges,
// while replay won from about 300 edges up).  Groups prefer host launches
// too (64 graphs: 0.600 vs 0.607 ms per DF step, static 267 vs 296 ms).
constexpr uint64_t kGraphMinArcs = 512;
void destroy_iteration_graph(Handle::IterGraph& g);
int local_move(Handle* h, const MoveArgs& a, uint32_t pass, uint32_t* iterations,
               bool record_trace, uint64_t* initial = nullptr, uint64_t* ever = nullptr);
int time_decide(Handle* h, const MoveArgs& a, uint32_t reps, std::vector<float>* ms);

// aggregate.cu
int count_communities(Handle* h, const uint32_t* Cp, uint32_t nv, uint32_t* ncomm);
int renumber(Handle* h, uint32_t* Cp, uint32_t nv, bool first_level);
int aggregate(Handle* h, const GraphView& g, const uint32_t* Cp, uint32_t ncomm, int dst,
              long long* Knew);
int louvain(Handle* h, bool all, bool use_range, uint64_t initial);

// group.cu
int louvain_group(Handle* h, bool all, bool use_range, uint64_t initial);
int group_m2(Handle* h);  // 2m of every graph from K (checks each < 2^32)
// group_m2 without a wait: each graph's 2m from K into d_gm2 and into pinned
// host memory (h_gS[0, G)), queued on the handle's stream; group_m2_take
// checks and keeps them after the caller's wait.
int group_m2_enqueue(Handle* h);
int group_m2_take(Handle* h);
// A group's batch (staged in union ids, its checks queued into ctrl->err):
// the hashed apply gated on those checks too, every graph's 2m, one wait.
int group_apply(Handle* h, const dfl_edge* sd, uint64_t nd, const dfl_edge* si, uint64_t ni);
int group_modularity(Handle* h, uint32_t g, i128* num, i128* den);
int group_upload_flags(Handle* h, uint8_t* dev, const uint8_t* host);
int group_set_level(Handle* h, const uint32_t* dev_off);

// tune.cu
int check_tuning(const dfl_tuning& t);
int autotune(Handle* h, int mode, uint32_t reps, double* best_ms);


inline GraphView base_view(const Handle* h) {
  return GraphView{h->off, h->deg, h->arcs, h->n};
}

inline uint32_t grid_for(uint64_t items, uint32_t per_block, uint32_t cap = 152u * 16u) {
  uint64_t g = (items + per_block - 1) / per_block;
  if (g == 0) g = 1;
  if (g > cap) g = cap;
  return uint32_t(g);
}

}  // namespace dfl
