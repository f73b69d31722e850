// Local-moving phase (Alg. 5) with Dynamic Frontier expansion.
//
// One iteration visits the frontier in `substeps` hash classes.  For each
// class, the decide kernels (one per degree bin) evaluate every frontier
// vertex i against the membership C', totals Sigma' and sizes left by the
// previous class:
//   scanCommunities: H[c] = sum of w_ij over neighbours j != i with C'[j] = c
//   best c != d = C'[i] by score(c) = 2m*H[c] - K_i*Sigma_c (ties: smaller c)
//   move iff score(c*) > stay = 2m*H[d] - K_i*(Sigma_d - K_i)   (Eq. 2 > 0)
//   except a singleton moving into a singleton community with a larger id.
// A mover is recorded, its numerator score - stay is added to S, and its
// neighbours (in the affected range) are marked for the next iteration
// (Section 4.1: a mover makes its neighbours affected).  The commit kernel then
// applies the class's moves to C', Sigma' and the sizes.
#include <chrono>
#include <cstring>
#include <mutex>

#include "common.cuh"

namespace dfl {

namespace {

struct DecideArgs {
  GraphView g;
  const uint32_t* C;
  const long long* K;
  const long long* Sigma;
  const int* size;
  const long long* m2p;   // 2m, read from device memory so captured graphs stay valid
  const uint32_t* list;
  const unsigned int* count;
  uint32_t* fbits_next;
  uint32_t* next_lists;
  Segs seg;
  int next_buf;
  const uint32_t* rbits;  // affected range, nullptr = every vertex
  uint32_t* ever;         // first-pass processed set, nullptr = not tracked
  uint32_t* mv_i;
  uint32_t* mv_c;
  uint32_t* mv_d;
  Ctrl* ctrl;
  uint32_t k;
  uint2* gtable;          // bin 3: per-block global tables
  uint32_t gslots;        // slots per block (power of two)
  // group of graphs (ngraphs > 0): the vertex's graph gives its 2m, whether
  // it is still processed, and where its movers' dQ sum goes
  uint32_t ngraphs;
  const uint32_t* goff;   // first vertex of each graph at this level
  const long long* gm2;
  const uint8_t* gdone;
  unsigned long long* gS;
};

// Group lookup for vertex i: false if its graph is no longer processed;
// otherwise its graph and 2m.
__device__ __forceinline__ bool group_active(const DecideArgs& a, uint32_t i, long long* m2,
                                             uint32_t* gi) {
  if (!a.ngraphs) return true;
  const uint32_t g = graph_of(a.goff, a.ngraphs, i);
  if (a.gdone[g]) return false;
  *gi = g;
  *m2 = a.gm2[g];
  return true;
}

// Outcome of one vertex's decision, identical on every lane / thread.
__device__ __forceinline__ bool decide_move(const DecideArgs& a, long long m2, uint32_t i, uint32_t d,
                                            long long Ki, bool have, i128 best, uint32_t bc,
                                            unsigned long long Hd, i128* gain) {
  if (!have) return false;
  i128 stay = (i128)m2 * (i128)Hd - (i128)Ki * (i128)(a.Sigma[d] - Ki);
  if (!(best > stay)) return false;
  if (a.size[d] == 1 && a.size[bc] == 1 && bc > d) return false;  // singleton-swap guard
  *gain = best - stay;
  return true;
}

__device__ __forceinline__ void record_move(const DecideArgs& a, uint32_t i, uint32_t c, uint32_t d,
                                            i128 gain, uint32_t gi) {
  uint32_t slot = atomicAdd(&a.ctrl->movers, 1u);
  a.mv_i[slot] = i;
  a.mv_c[slot] = c;
  a.mv_d[slot] = d;
  add_s(a.ctrl, (u128)gain);
  if (a.ngraphs) {
    const u128 v = (u128)gain;
    const unsigned long long lo = (unsigned long long)(v & 0xFFFFFFFFull);
    const unsigned long long hi = (unsigned long long)(v >> 32);
    if (lo) atomicAdd(a.gS + 2 * gi, lo);
    if (hi) atomicAdd(a.gS + 2 * gi + 1, hi);
  }
}

// Mark neighbour j of a mover for the next iteration (warp-collective).
__device__ __forceinline__ void mark_next(const DecideArgs& a, uint32_t j, bool valid) {
  bool fresh = false;
  uint32_t key = 0;
  if (valid && (!a.rbits || bit_test(a.rbits, j)) && bit_set(a.fbits_next, j)) {
    fresh = true;
    key = vertex_class(j, a.k, a.seg) * kBins + degree_bin(a.g.deg[j], a.seg);
  }
  append_vertex(j, fresh, key, a.next_lists, a.seg, a.ctrl, a.next_buf);
}

// ---------------------------------------------------------------------------
// Bin 0: deg <= 32, one warp per vertex, one arc per lane, aggregation by
// community with match/reduce in registers.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_decide_warp(DecideArgs a) {
  const long long m2_one = *a.m2p;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t cnt = *a.count;
  uint64_t warp = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) >> 5;
  uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  unsigned long long bytes = 0, processed = 0, fresh_ever = 0;
  for (uint64_t t = warp; t < cnt; t += nwarps) {
    const uint32_t i = a.list[t];
    long long m2 = m2_one;
    uint32_t gi = 0;
    if (!group_active(a, i, &m2, &gi)) continue;
    if (a.ever && lane == 0 && bit_set(a.ever, i)) ++fresh_ever;
    ++processed;
    if (a.rbits && !bit_test(a.rbits, i)) continue;  // processed, not in the affected range
    const uint32_t d = a.C[i];
    const long long Ki = a.K[i];
    const unsigned long long o = a.g.off[i];
    const uint32_t dg = a.g.deg[i];
    uint2 arc = lane < dg ? a.g.arcs[o + lane] : make_uint2(i, 0u);
    bool valid = lane < dg && arc.x != i && arc.y != 0;  // weight 0 = deleted arc
    uint32_t c = valid ? a.C[arc.x] : kEmpty;
    unsigned peers = __match_any_sync(0xFFFFFFFFu, c);
    uint32_t hsum = __reduce_add_sync(peers, valid ? arc.y : 0u);
    bool leader = valid && lane == uint32_t(__ffs(peers) - 1);
    unsigned dm = __ballot_sync(0xFFFFFFFFu, leader && c == d);
    unsigned long long Hd = dm ? __shfl_sync(0xFFFFFFFFu, hsum, __ffs(dm) - 1) : 0u;
    bool cand = leader && c != d;
    unsigned cm = __ballot_sync(0xFFFFFFFFu, cand);
    i128 score = 0;
    if (cand) score = (i128)m2 * (i128)hsum - (i128)Ki * (i128)a.Sigma[c];
    bool have = cand;
    uint32_t bc = c;
    warp_argmax(have, score, bc);
    i128 gain = 0;
    bool mv = decide_move(a, m2, i, d, Ki, have, score, bc, Hd, &gain);
    bytes += 24 + 12ull * dg + 12ull * __popc(cm);
    if (mv) {
      if (lane == 0) record_move(a, i, bc, d, gain, gi);
      mark_next(a, arc.x, valid);
      bytes += 16 + 4ull * dg;
    }
  }
  if (lane == 0) {
    atomicAdd(&a.ctrl->move_bytes, bytes);
    if (processed) atomicAdd(&a.ctrl->processed, processed);
    if (fresh_ever) atomicAdd(&a.ctrl->ever_count, fresh_ever);
  }
}

// Open-addressing insert (linear probing) of weight w under key c; gives up
// after `limit` probes (the caller then falls back to a larger table).
__device__ __forceinline__ bool table_add(uint32_t* keys, uint32_t* vals, uint32_t mask, uint32_t c,
                                          uint32_t w, uint32_t limit) {
  uint32_t s = hash32(c) & mask;
  for (uint32_t probe = 0; probe < limit; ++probe) {
    uint32_t prev = keys[s];
    if (prev == kEmpty) prev = atomicCAS(&keys[s], kEmpty, c);
    if (prev == kEmpty || prev == c) {
      atomicAdd(&vals[s], w);
      return true;
    }
    s = (s + 1) & mask;
  }
  return false;
}

// scanCommunities over arcs [k0, dg) of row o, lanes striding by `step`:
// each 32-arc chunk is pre-aggregated per community inside the warp
// (match + reduce), so only one table update per distinct community and
// chunk is issued.  Loads of kUnroll chunks are issued before use.
template <int kUnroll>
__device__ __forceinline__ bool scan_row(const DecideArgs& a, uint32_t i, unsigned long long o,
                                         uint32_t dg, uint32_t k0, uint32_t step, uint32_t* keys,
                                         uint32_t* vals, uint32_t mask, uint32_t limit) {
  const uint32_t lane = threadIdx.x & 31u;
  bool ok = true;
  for (uint32_t base = k0; base < dg; base += step * kUnroll) {
    uint2 arc[kUnroll];
    uint32_t c[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      uint32_t k = base + u * step + lane;
      arc[u] = k < dg ? a.g.arcs[o + k] : make_uint2(i, 0u);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      bool valid = arc[u].x != i && arc[u].y != 0;  // skip self-loops and deleted arcs
      c[u] = valid ? a.C[arc[u].x] : kEmpty;
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      unsigned peers = __match_any_sync(0xFFFFFFFFu, c[u]);
      uint32_t hs = __reduce_add_sync(peers, c[u] != kEmpty ? arc[u].y : 0u);
      if (c[u] != kEmpty && lane == uint32_t(__ffs(peers) - 1))
        ok &= table_add(keys, vals, mask, c[u], hs, limit);
    }
  }
  return ok;
}

// ---------------------------------------------------------------------------
// Bin 1: 32 < deg <= 256, one warp per vertex with a shared table.
// ---------------------------------------------------------------------------
constexpr uint32_t kWarpSlots = 512;
constexpr int kWarpHashWarps = 8;

__global__ void __launch_bounds__(256) k_decide_warp_hash(DecideArgs a) {
  const long long m2_one = *a.m2p;
  __shared__ uint32_t skeys[kWarpHashWarps][kWarpSlots];
  __shared__ uint32_t svals[kWarpHashWarps][kWarpSlots];
  const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
  uint32_t* keys = skeys[wib];
  uint32_t* vals = svals[wib];
  const uint32_t cnt = *a.count;
  uint64_t warp = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) >> 5;
  uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  unsigned long long bytes = 0, processed = 0, fresh_ever = 0;
  for (uint64_t t = warp; t < cnt; t += nwarps) {
    const uint32_t i = a.list[t];
    long long m2 = m2_one;
    uint32_t gi = 0;
    if (!group_active(a, i, &m2, &gi)) continue;
    if (a.ever && lane == 0 && bit_set(a.ever, i)) ++fresh_ever;
    ++processed;
    if (a.rbits && !bit_test(a.rbits, i)) continue;
    const uint32_t d = a.C[i];
    const long long Ki = a.K[i];
    const unsigned long long o = a.g.off[i];
    const uint32_t dg = a.g.deg[i];
    uint32_t slots = 64;
    while (slots < 2 * dg && slots < kWarpSlots) slots <<= 1;
    const uint32_t mask = slots - 1;
    for (uint32_t s = lane; s < slots; s += 32) {
      keys[s] = kEmpty;
      vals[s] = 0;
    }
    __syncwarp();
    bool ok = scan_row<4>(a, i, o, dg, 0, 32, keys, vals, mask, slots);
    if (!__all_sync(0xFFFFFFFFu, ok) && lane == 0) atomicOr(&a.ctrl->err, kErrInternal);
    __syncwarp();
    bool have = false;
    i128 best = 0;
    uint32_t bc = 0;
    unsigned long long Hd = 0;
    uint32_t ncand = 0;
    for (uint32_t s = lane; s < slots; s += 32) {
      uint32_t c = keys[s];
      if (c == kEmpty) continue;
      if (c == d) {
        Hd = vals[s];
        continue;
      }
      ++ncand;
      i128 sc = (i128)m2 * (i128)vals[s] - (i128)Ki * (i128)a.Sigma[c];
      if (!have || sc > best || (sc == best && c < bc)) {
        have = true;
        best = sc;
        bc = c;
      }
    }
    for (int x = 16; x; x >>= 1) {
      Hd += __shfl_xor_sync(0xFFFFFFFFu, Hd, x);
      ncand += __shfl_xor_sync(0xFFFFFFFFu, ncand, x);
    }
    warp_argmax(have, best, bc);
    i128 gain = 0;
    bool mv = decide_move(a, m2, i, d, Ki, have, best, bc, Hd, &gain);
    bytes += 24 + 12ull * dg + 12ull * ncand;
    if (mv) {
      if (lane == 0) record_move(a, i, bc, d, gain, gi);
      for (uint32_t k0 = 0; k0 < dg; k0 += 32) {
        uint32_t k = k0 + lane;
        uint2 arc = k < dg ? a.g.arcs[o + k] : make_uint2(i, 0u);
        mark_next(a, arc.x, k < dg && arc.x != i && arc.y != 0);
      }
      bytes += 16 + 4ull * dg;
    }
    __syncwarp();
  }
  if (lane == 0) {
    atomicAdd(&a.ctrl->move_bytes, bytes);
    if (processed) atomicAdd(&a.ctrl->processed, processed);
    if (fresh_ever) atomicAdd(&a.ctrl->ever_count, fresh_ever);
  }
}

// ---------------------------------------------------------------------------
// Bins 2 and 3: one block per vertex with a shared table of kBlockSlots
// (bin 2 fits by construction; a bin-3 vertex has so many neighbours that the
// number of distinct neighbour communities, not the degree, sizes the table).
// If a bin-3 vertex overflows the shared table, it is redone with a table in
// a per-block slice of global memory sized from the maximum degree.
// ---------------------------------------------------------------------------
constexpr uint32_t kBlockSlots = 2 * kBinBlock;  // 8192 keys + 8192 values = 64 KB

template <int kThreads>
__global__ void __launch_bounds__(kThreads) k_decide_block(DecideArgs a) {
  const long long m2_one = *a.m2p;
  extern __shared__ uint32_t dyn[];
  __shared__ unsigned long long s_hd;
  __shared__ uint32_t s_ncand;
  __shared__ unsigned long long s_lo[kThreads / 32], s_hi[kThreads / 32];
  __shared__ uint32_t s_c[kThreads / 32];
  __shared__ int s_have[kThreads / 32];
  __shared__ int s_ok;
  const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5, nw = kThreads / 32;
  const uint32_t cnt = *a.count;
  unsigned long long bytes = 0, processed = 0, fresh_ever = 0;
  for (uint64_t t = blockIdx.x; t < cnt; t += gridDim.x) {
    const uint32_t i = a.list[t];
    long long m2 = m2_one;
    uint32_t gi = 0;
    if (!group_active(a, i, &m2, &gi)) continue;
    if (a.ever && threadIdx.x == 0 && bit_set(a.ever, i)) ++fresh_ever;
    ++processed;
    if (a.rbits && !bit_test(a.rbits, i)) continue;
    const uint32_t d = a.C[i];
    const long long Ki = a.K[i];
    const unsigned long long o = a.g.off[i];
    const uint32_t dg = a.g.deg[i];
    uint32_t slots = 1024;
    while (slots < 2 * dg && slots < kBlockSlots) slots <<= 1;
    uint32_t* keys = dyn;
    uint32_t* vals = dyn + slots;
    bool global = false;
    for (int attempt = 0; attempt < 2; ++attempt) {
      if (attempt == 1) {  // shared table overflowed: global slice of gslots
        global = true;
        slots = a.gslots;
        keys = reinterpret_cast<uint32_t*>(a.gtable + uint64_t(blockIdx.x) * a.gslots);
        vals = keys + a.gslots;
      }
      const uint32_t mask = slots - 1;
      for (uint32_t s = threadIdx.x; s < slots; s += kThreads) {
        keys[s] = kEmpty;
        vals[s] = 0;
      }
      if (threadIdx.x == 0) {
        s_hd = 0;
        s_ncand = 0;
        s_ok = 1;
      }
      __syncthreads();
      // a table of >= 2 * deg slots cannot overflow: probe it to the end;
      // a smaller shared table (bin 3) gives up early and falls back
      const uint32_t limit = (global || slots >= 2 * dg) ? slots : 64;
      bool ok = scan_row<4>(a, i, o, dg, wib * 32, kThreads, keys, vals, mask, limit);
      if (!ok) s_ok = 0;
      __syncthreads();
      const bool done = s_ok;
      __syncthreads();  // everyone has read s_ok before the retry resets it
      if (done) break;
      if (global || !a.gtable) {
        if (threadIdx.x == 0) atomicOr(&a.ctrl->err, kErrInternal);
        break;
      }
    }
    bool have = false;
    i128 best = 0;
    uint32_t bc = 0;
    uint32_t ncand = 0;
    for (uint32_t s = threadIdx.x; s < slots; s += kThreads) {
      uint32_t c = keys[s];
      if (c == kEmpty) continue;
      if (c == d) {
        s_hd = vals[s];  // exactly one slot holds d
        continue;
      }
      ++ncand;
      i128 sc = (i128)m2 * (i128)vals[s] - (i128)Ki * (i128)a.Sigma[c];
      if (!have || sc > best || (sc == best && c < bc)) {
        have = true;
        best = sc;
        bc = c;
      }
    }
    for (int x = 16; x; x >>= 1) ncand += __shfl_xor_sync(0xFFFFFFFFu, ncand, x);
    warp_argmax(have, best, bc);
    if (lane == 0) {
      s_lo[wib] = (unsigned long long)(u128)best;
      s_hi[wib] = (unsigned long long)((u128)best >> 64);
      s_c[wib] = bc;
      s_have[wib] = have;
      if (ncand) atomicAdd(&s_ncand, ncand);
    }
    __syncthreads();
    if (wib == 0) {
      have = lane < nw && s_have[lane];
      best = lane < nw ? (i128)(((u128)s_hi[lane] << 64) | (u128)s_lo[lane]) : 0;
      bc = lane < nw ? s_c[lane] : 0;
      warp_argmax(have, best, bc);
      if (lane == 0) {
        s_lo[0] = (unsigned long long)(u128)best;
        s_hi[0] = (unsigned long long)((u128)best >> 64);
        s_c[0] = bc;
        s_have[0] = have;
      }
    }
    __syncthreads();
    have = s_have[0];
    best = (i128)(((u128)s_hi[0] << 64) | (u128)s_lo[0]);
    bc = s_c[0];
    i128 gain = 0;
    bool mv = decide_move(a, m2, i, d, Ki, have, best, bc, s_hd, &gain);
    bytes += 24 + 12ull * dg + 12ull * s_ncand;
    if (mv) {
      if (threadIdx.x == 0) record_move(a, i, bc, d, gain, gi);
      for (uint32_t k0 = wib * 32; k0 < dg; k0 += kThreads) {
        uint32_t k = k0 + lane;
        uint2 arc = k < dg ? a.g.arcs[o + k] : make_uint2(i, 0u);
        mark_next(a, arc.x, k < dg && arc.x != i && arc.y != 0);
      }
      bytes += 16 + 4ull * dg;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicAdd(&a.ctrl->move_bytes, bytes);
    if (processed) atomicAdd(&a.ctrl->processed, processed);
    if (fresh_ever) atomicAdd(&a.ctrl->ever_count, fresh_ever);
  }
}

// ---------------------------------------------------------------------------
// Bin 3 (deg > 4096): a vertex is split into chunks of kGiantChunk arcs, one
// block per chunk.  A chunk block aggregates its arcs in shared memory and
// writes the distinct (community, weight) partial sums to the vertex's region
// of g_partial; the last chunk block of the vertex merges the partial sums
// (in hash-partitioned passes that each fit the shared table) and decides.
// If a pass still overflows, the last block redoes the vertex alone with a
// global table slice.
// ---------------------------------------------------------------------------
constexpr uint32_t kGiantChunk = 4096;
constexpr uint32_t kGiantSlots = 2 * kGiantChunk;  // 8192 keys + values = 64 KB
constexpr int kGiantThreads = 256;

struct GiantDecide {
  unsigned long long* poff;
  uint32_t* cpre;
  uint32_t* done;
  uint32_t* pcount;
  uint2* partial;
  unsigned int* nitems;
};

// One block: exclusive prefix over the bin-3 list of deg (partial regions)
// and of the chunk counts (work items).
__global__ void __launch_bounds__(1024) k_giant_prefix(DecideArgs a, GiantDecide gd) {
  __shared__ unsigned long long s_d[32];
  __shared__ uint32_t s_c[32];
  __shared__ unsigned long long s_base;
  __shared__ uint32_t s_cbase;
  const uint32_t cnt = *a.count;
  const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    s_base = 0;
    s_cbase = 0;
  }
  __syncthreads();
  for (uint32_t t0 = 0; t0 < cnt; t0 += blockDim.x) {
    uint32_t t = t0 + threadIdx.x;
    unsigned long long d = t < cnt ? a.g.deg[a.list[t]] : 0ull;
    if (d && a.ngraphs && a.gdone[graph_of(a.goff, a.ngraphs, a.list[t])]) d = 0;  // skipped
    uint32_t ch = uint32_t((d + kGiantChunk - 1) / kGiantChunk);
    unsigned long long xd = d;
    uint32_t xc = ch;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long yd = __shfl_up_sync(0xFFFFFFFFu, xd, o);
      uint32_t yc = __shfl_up_sync(0xFFFFFFFFu, xc, o);
      if (lane >= (uint32_t)o) {
        xd += yd;
        xc += yc;
      }
    }
    if (lane == 31) {
      s_d[w] = xd;
      s_c[w] = xc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long rd = s_base;
      uint32_t rc = s_cbase;
      for (uint32_t k = 0; k < blockDim.x / 32; ++k) {
        unsigned long long td = s_d[k];
        uint32_t tc = s_c[k];
        s_d[k] = rd;
        s_c[k] = rc;
        rd += td;
        rc += tc;
      }
      s_base = rd;
      s_cbase = rc;
    }
    __syncthreads();
    if (t < cnt) {
      gd.poff[t] = s_d[w] + xd - d;
      gd.cpre[t] = s_c[w] + xc - ch;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    gd.cpre[cnt] = s_cbase;
    *gd.nitems = s_cbase;
  }
}

__global__ void __launch_bounds__(kGiantThreads, 2) k_decide_giant(DecideArgs a, GiantDecide gd) {
  const long long m2_one = *a.m2p;
  extern __shared__ uint32_t dyn[];
  uint32_t* keys = dyn;
  uint32_t* vals = dyn + kGiantSlots;
  __shared__ int s_last, s_ok, s_have[kGiantThreads / 32];
  __shared__ unsigned long long s_hd, s_lo[kGiantThreads / 32], s_hi[kGiantThreads / 32];
  __shared__ uint32_t s_c[kGiantThreads / 32], s_ncand;
  const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5, nw = kGiantThreads / 32;
  const uint32_t cnt = *a.count;
  const uint32_t nitems = *gd.nitems;
  unsigned long long bytes = 0, processed = 0, fresh_ever = 0;
  for (uint32_t item = blockIdx.x; item < nitems; item += gridDim.x) {
    uint32_t lo = 0, hi = cnt;  // list position owning this chunk
    while (hi - lo > 1) {
      uint32_t mid = (lo + hi) >> 1;
      if (gd.cpre[mid] <= item) lo = mid;
      else hi = mid;
    }
    const uint32_t t = lo;
    const uint32_t chunk = item - gd.cpre[t];
    const uint32_t nch = gd.cpre[t + 1] - gd.cpre[t];
    const uint32_t i = a.list[t];
    long long m2 = m2_one;
    uint32_t gi = 0;
    group_active(a, i, &m2, &gi);  // its graph is active: the prefix gave it chunks
    if (chunk == 0) {
      if (a.ever && threadIdx.x == 0 && bit_set(a.ever, i)) ++fresh_ever;
      ++processed;
    }
    if (a.rbits && !bit_test(a.rbits, i)) continue;  // processed, not in the affected range
    const unsigned long long o = a.g.off[i];
    const uint32_t dg = a.g.deg[i];
    const uint32_t k0 = chunk * kGiantChunk;
    const uint32_t k1 = min(dg, k0 + kGiantChunk);
    // 1. this chunk's partial sums
    for (uint32_t s = threadIdx.x; s < kGiantSlots; s += kGiantThreads) {
      keys[s] = kEmpty;
      vals[s] = 0;
    }
    __syncthreads();
    // a table of 2x the chunk's arcs cannot overflow
    scan_row<4>(a, i, o, k1, k0 + wib * 32, kGiantThreads, keys, vals, kGiantSlots - 1, kGiantSlots);
    __syncthreads();
    for (uint32_t s0 = wib * 32; s0 < kGiantSlots; s0 += kGiantThreads) {
      uint32_t s = s0 + lane;
      uint32_t key = keys[s];
      unsigned m = __ballot_sync(0xFFFFFFFFu, key != kEmpty);
      uint32_t base = 0;
      if (lane == 0 && m) base = atomicAdd(&gd.pcount[t], __popc(m));
      base = __shfl_sync(0xFFFFFFFFu, base, 0);
      if (key != kEmpty) gd.partial[gd.poff[t] + base + __popc(m & ((1u << lane) - 1u))] = make_uint2(key, vals[s]);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&gd.done[t], 1u) == nch - 1;
    __syncthreads();
    if (!s_last) continue;
    __threadfence();
    // 2. last block of the vertex: merge the partial sums and decide
    const uint32_t d = a.C[i];
    const long long Ki = a.K[i];
    const uint32_t np = __ldcg(gd.pcount + t);
    const uint32_t passes = (np + kGiantChunk - 1) / kGiantChunk > 0 ? (np + kGiantChunk - 1) / kGiantChunk : 1;
    bool have = false;
    i128 best = 0;
    uint32_t bc = 0;
    uint32_t ncand = 0;
    unsigned long long hd_local = 0;
    if (threadIdx.x == 0) {
      s_ok = 1;
      s_hd = 0;
      s_ncand = 0;
    }
    for (uint32_t pass = 0; pass < passes; ++pass) {
      for (uint32_t s = threadIdx.x; s < kGiantSlots; s += kGiantThreads) {
        keys[s] = kEmpty;
        vals[s] = 0;
      }
      __syncthreads();
      bool ok = true;
      for (uint32_t e = threadIdx.x; e < np; e += kGiantThreads) {
        uint2 pe = __ldcg(gd.partial + gd.poff[t] + e);  // written by other blocks: bypass L1
        if (passes == 1 || hash32(pe.x ^ 0x5bd1e995u) % passes == pass)
          ok &= table_add(keys, vals, kGiantSlots - 1, pe.x, pe.y, kGiantSlots);
      }
      if (!ok) s_ok = 0;
      __syncthreads();
      for (uint32_t s = threadIdx.x; s < kGiantSlots; s += kGiantThreads) {
        uint32_t c = keys[s];
        if (c == kEmpty) continue;
        if (c == d) {
          hd_local = vals[s];
          continue;
        }
        ++ncand;
        i128 sc = (i128)m2 * (i128)vals[s] - (i128)Ki * (i128)a.Sigma[c];
        if (!have || sc > best || (sc == best && c < bc)) {
          have = true;
          best = sc;
          bc = c;
        }
      }
      __syncthreads();
    }
    const bool overflow = !s_ok;
    __syncthreads();
    if (overflow) {
      // rare: redo the whole vertex with this block's global table slice
      have = false;
      ncand = 0;
      hd_local = 0;
      uint32_t* gk = reinterpret_cast<uint32_t*>(a.gtable + uint64_t(blockIdx.x) * a.gslots);
      uint32_t* gv = gk + a.gslots;
      uint32_t slots = a.gslots;
      for (uint32_t s = threadIdx.x; s < slots; s += kGiantThreads) {
        gk[s] = kEmpty;
        gv[s] = 0;
      }
      __syncthreads();
      scan_row<4>(a, i, o, dg, wib * 32, kGiantThreads, gk, gv, slots - 1, slots);
      __syncthreads();
      for (uint32_t s = threadIdx.x; s < slots; s += kGiantThreads) {
        uint32_t c = gk[s];
        if (c == kEmpty) continue;
        if (c == d) {
          hd_local = gv[s];
          continue;
        }
        ++ncand;
        i128 sc = (i128)m2 * (i128)gv[s] - (i128)Ki * (i128)a.Sigma[c];
        if (!have || sc > best || (sc == best && c < bc)) {
          have = true;
          best = sc;
          bc = c;
        }
      }
    }
    for (int x = 16; x; x >>= 1) {
      ncand += __shfl_xor_sync(0xFFFFFFFFu, ncand, x);
      hd_local += __shfl_xor_sync(0xFFFFFFFFu, hd_local, x);
    }
    warp_argmax(have, best, bc);
    if (lane == 0) {
      s_lo[wib] = (unsigned long long)(u128)best;
      s_hi[wib] = (unsigned long long)((u128)best >> 64);
      s_c[wib] = bc;
      s_have[wib] = have;
      if (ncand) atomicAdd(&s_ncand, ncand);
      if (hd_local) atomicAdd(&s_hd, hd_local);
    }
    __syncthreads();
    if (wib == 0) {
      have = lane < nw && s_have[lane];
      best = lane < nw ? (i128)(((u128)s_hi[lane] << 64) | (u128)s_lo[lane]) : 0;
      bc = lane < nw ? s_c[lane] : 0;
      warp_argmax(have, best, bc);
      if (lane == 0) {
        s_lo[0] = (unsigned long long)(u128)best;
        s_hi[0] = (unsigned long long)((u128)best >> 64);
        s_c[0] = bc;
        s_have[0] = have;
      }
    }
    __syncthreads();
    have = s_have[0];
    best = (i128)(((u128)s_hi[0] << 64) | (u128)s_lo[0]);
    bc = s_c[0];
    i128 gain = 0;
    bool mv = decide_move(a, m2, i, d, Ki, have, best, bc, s_hd, &gain);
    bytes += 24 + 12ull * dg + 12ull * s_ncand;
    if (mv) {
      if (threadIdx.x == 0) record_move(a, i, bc, d, gain, gi);
      for (uint32_t q0 = wib * 32; q0 < dg; q0 += kGiantThreads) {
        uint32_t q = q0 + lane;
        uint2 arc = q < dg ? a.g.arcs[o + q] : make_uint2(i, 0u);
        mark_next(a, arc.x, q < dg && arc.x != i && arc.y != 0);
      }
      bytes += 16 + 4ull * dg;
    }
    if (threadIdx.x == 0) {  // ready for the next use of this list position
      gd.done[t] = 0;
      gd.pcount[t] = 0;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicAdd(&a.ctrl->move_bytes, bytes);
    if (processed) atomicAdd(&a.ctrl->processed, processed);
    if (fresh_ever) atomicAdd(&a.ctrl->ever_count, fresh_ever);
  }
}

// Apply the moves of one sub-step.
__global__ void k_commit(const uint32_t* __restrict__ mv_i, const uint32_t* __restrict__ mv_c,
                         const uint32_t* __restrict__ mv_d, uint32_t* __restrict__ C,
                         const long long* __restrict__ K, long long* __restrict__ Sigma,
                         int* __restrict__ size, Ctrl* ctrl) {
  const uint32_t m = ctrl->movers;
  if (blockIdx.x == 0 && threadIdx.x == 0 && m) atomicAdd(&ctrl->moved, (unsigned long long)m);
  for (uint64_t t = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; t < m;
       t += uint64_t(gridDim.x) * blockDim.x) {
    uint32_t i = mv_i[t], c = mv_c[t], d = mv_d[t];
    long long ki = K[i];
    C[i] = c;
    atomicAdd((unsigned long long*)&Sigma[d], (unsigned long long)(-ki));
    atomicAdd((unsigned long long*)&Sigma[c], (unsigned long long)ki);
    atomicSub(&size[d], 1);
    atomicAdd(&size[c], 1);
  }
}

int read_ctrl(Handle* h) {
  DFL_CUDA(h, cudaMemcpyAsync(h->hctrl, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
  DFL_CUDA(h, cudaStreamSynchronize(h->stream));
  return DFL_OK;
}

// floor(tau_num * m2^2 / (2 * tau_den * drop^pass)), the exact form of
// "sum of dQ <= tau" (Alg. 5) with S = sum of the movers' 2m^2 * dQ.
u128 tolerance_threshold(const dfl_options& o, long long m2, uint32_t pass) {
  u128 num = (u128)o.tau_num * (u128)(uint64_t)m2 * (u128)(uint64_t)m2;
  u128 den = (u128)2 * (u128)o.tau_den;
  for (uint32_t p = 0; p < pass; ++p) {
    if (den > num) return 0;
    den *= (u128)o.tolerance_drop;
  }
  if (den == 0) return ~(u128)0;
  return num / den;
}

uint32_t next_pow2(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return uint32_t(p);
}



__global__ void k_set_m2(Ctrl* ctrl, long long m2) { ctrl->m2v = m2; }

constexpr uint32_t kGiantBlocks = 2 * 152;

// Issue one local-moving iteration (all sub-steps) on h->stream.  With
// `counts` (host-known list lengths) empty bins are skipped and grids are
// sized to the work; without (graph capture) every bin is launched with a
// fixed grid and reads its length on the device.
int issue_iteration(Handle* h, DecideArgs a, int cur, const unsigned int (*counts)[kBins],
                    const GiantDecide& gd_base, bool decide_only = false) {
  const uint32_t k = a.k;
  const int nxt = cur ^ 1;
  // reset the iteration's sums and the next buffer's list lengths
  DFL_CUDA(h, cudaMemsetAsync(h->ctrl, 0, offsetof(Ctrl, move_bytes), h->stream));
  DFL_CUDA(h, cudaMemsetAsync(&h->ctrl->movers, 0, sizeof(unsigned int), h->stream));
  DFL_CUDA(h, cudaMemsetAsync(&h->ctrl->count[nxt][0][0], 0, sizeof(h->ctrl->count[0]), h->stream));
  if (a.ngraphs)
    DFL_CUDA(h, cudaMemsetAsync(a.gS, 0, sizeof(unsigned long long) * 2 * a.ngraphs, h->stream));
  a.fbits_next = h->fbits[nxt];
  a.next_lists = h->lists[nxt];
  a.next_buf = nxt;
  for (uint32_t s = 0; s < k; ++s) {
    // the degree bins of one class are independent: the larger ones run on
    // auxiliary streams, concurrently with the rest
    int nb = 0;
    for (int b = 0; b < kBins; ++b) nb += (!counts || counts[s][b]) ? 1 : 0;
    const bool any = nb > 0;
    cudaEvent_t pa = nullptr, pb = nullptr;  // wall time of the decide phase (profiling)
    if (any && (h->opt.flags & DFL_FLAG_PROFILE)) {
      cudaEventCreate(&pa);
      cudaEventCreate(&pb);
      record_timing_event(pa, h->stream);
    }
    const bool forked = nb > 1;
    if (forked) DFL_CUDA(h, cudaEventRecord(h->ev_fork, h->stream));
    bool joined[kBins - 1] = {false, false, false};
    for (int b = kBins - 1; b >= 0; --b) {
      const uint32_t c = counts ? counts[s][b] : 0u;
      if (counts && !c) continue;
      cudaStream_t st = h->stream;
      if (forked && b > 0) {
        st = h->aux[b - 1];
        DFL_CUDA(h, cudaStreamWaitEvent(st, h->ev_fork, 0));
        joined[b - 1] = true;
      }
      a.list = h->lists[cur] + h->segs.off[s * kBins + b];
      a.count = &h->ctrl->count[cur][s][b];
      LaunchScope ls(h, DFL_PROF_BIN0 + b, st);
      if (b == 0) {
        k_decide_warp<<<counts ? grid_for(uint64_t(c) * 32, 256, 152 * 64) : 152 * 8, 256, 0, st>>>(a);
      } else if (b == 1) {
        k_decide_warp_hash<<<counts ? grid_for(uint64_t(c) * 32, 256, 152 * 16) : 152 * 4, 256, 0, st>>>(a);
      } else if (b == 2) {
        const size_t smem = sizeof(uint32_t) * 2 * kBlockSlots;
        const uint32_t bt = h->tune.block_threads;
        const uint32_t per_sm = bt == 128 ? 3 : bt == 256 ? 3 : 2;  // 64 KB table each
        const uint32_t grid = counts ? grid_for(c, 1, 152 * per_sm) : 152 * per_sm;
        if (bt == 128) k_decide_block<128><<<grid, 128, smem, st>>>(a);
        else if (bt == 512) k_decide_block<512><<<grid, 512, smem, st>>>(a);
        else k_decide_block<256><<<grid, 256, smem, st>>>(a);
      } else {
        GiantDecide gd = gd_base;
        gd.nitems = &h->ctrl->giant_chunks[cur];
        k_giant_prefix<<<1, 1024, 0, st>>>(a, gd);
        DFL_TRY(check_launch(h, "giant prefix"));
        k_decide_giant<<<kGiantBlocks, kGiantThreads, sizeof(uint32_t) * 2 * kGiantSlots, st>>>(a, gd);
      }
      DFL_TRY(check_launch(h, "decide"));
    }
    for (int b = 0; b < kBins - 1; ++b)
      if (joined[b]) {
        DFL_CUDA(h, cudaEventRecord(h->ev_join[b], h->aux[b]));
        DFL_CUDA(h, cudaStreamWaitEvent(h->stream, h->ev_join[b], 0));
      }
    if (pa && pb) {
      record_timing_event(pb, h->stream);
      h->ev_pending.push_back(Handle::Ev{pa, pb, DFL_PROF_MOVE});
      h->prof.launches[DFL_PROF_MOVE]++;
    }
    if (any && decide_only) {
      DFL_CUDA(h, cudaMemsetAsync(&h->ctrl->movers, 0, sizeof(unsigned int), h->stream));
    } else if (any) {
      {
        LaunchScope ls(h, DFL_PROF_COMMIT);
        k_commit<<<152 * 2, 256, 0, h->stream>>>(h->mv_i, h->mv_c, h->mv_d, const_cast<uint32_t*>(a.C), a.K,
                                                 const_cast<long long*>(a.Sigma), const_cast<int*>(a.size),
                                                 h->ctrl);
        DFL_TRY(check_launch(h, "commit"));
      }
      DFL_CUDA(h, cudaMemsetAsync(&h->ctrl->movers, 0, sizeof(unsigned int), h->stream));
    }
  }
  // the processed frontier's bitmap becomes the next-next target
  DFL_CUDA(h, cudaMemsetAsync(h->fbits[cur], 0, sizeof(uint32_t) * h->words, h->stream));
  return DFL_OK;
}

// Everything an iteration graph bakes in; a different key means re-capture.
struct GraphKey {
  DecideArgs a;
  GiantDecide gd;
  int cur;
  uint32_t flags;
  void* stream;
  uint32_t block_threads;
};

// The cached graph for this iteration's key (captured on a miss, evicting
// the least recently used entry of this parity).
int ensure_iteration_graph(Handle* h, const DecideArgs& a, const GiantDecide& gd, int cur,
                           Handle::IterGraph** out) {
  GraphKey key;
  std::memset(&key, 0, sizeof(key));
  key.a = a;
  key.gd = gd;
  key.cur = cur;
  key.flags = h->opt.flags;
  key.stream = h->stream;
  key.block_threads = h->tune.block_threads;
  Handle::IterGraph* slot = nullptr;
  for (auto& e : h->igraph[cur])
    if (e.exec && e.key.size() == sizeof(key) && std::memcmp(e.key.data(), &key, sizeof(key)) == 0) {
      e.last_use = ++h->graph_use;
      *out = &e;
      return DFL_OK;
    }
  for (auto& e : h->igraph[cur])
    if (!slot || !e.exec || (slot->exec && e.last_use < slot->last_use)) slot = &e;
  Handle::IterGraph& g = *slot;
  destroy_iteration_graph(g);
  const auto t0 = std::chrono::steady_clock::now();
  const size_t ev0 = h->ev_pending.size();
  const uint64_t l0 = h->launches;
  uint64_t cl0[DFL_PROF_CLASSES];
  for (int q = 0; q < DFL_PROF_CLASSES; ++q) cl0[q] = h->prof.launches[q];
  DFL_CUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  int rc = issue_iteration(h, a, cur, nullptr, gd);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return set_error(h, DFL_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    g.exec = nullptr;
    return set_error(h, DFL_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  // events recorded inside the graph are harvested after every replay
  g.evs.assign(h->ev_pending.begin() + ev0, h->ev_pending.end());
  h->ev_pending.resize(ev0);
  g.kernels = h->launches - l0;
  h->launches = l0;
  for (int q = 0; q < DFL_PROF_CLASSES; ++q) {  // counted per replay instead
    g.class_launches[q] = h->prof.launches[q] - cl0[q];
    h->prof.launches[q] = cl0[q];
  }
  g.key.assign(reinterpret_cast<const char*>(&key), reinterpret_cast<const char*>(&key) + sizeof(key));
  g.last_use = ++h->graph_use;
  h->graph_captures++;
  h->graph_capture_ms +=
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = &g;
  return DFL_OK;
}

}  // namespace

void destroy_iteration_graph(Handle::IterGraph& g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  for (auto& ev : g.evs) {
    cudaEventDestroy(ev.a);
    cudaEventDestroy(ev.b);
  }
  g.evs.clear();
  g.key.clear();
  g.exec = nullptr;
  g.kernels = 0;
}

namespace {

// Buffers, streams and kernel attributes one local-moving run needs, and its
// decide arguments.
int prepare_move(Handle* h, const MoveArgs& ma, DecideArgs* out, GiantDecide* gdo) {
  const uint32_t k = h->opt.substeps;
  make_segs(h, k);
  // global tables for the largest bins: one slice of gslots keys + gslots
  // values per block, gslots >= 2 * (max degree of the current graph)
  const uint32_t gslots = next_pow2(2ull * (ma.max_deg > kBinBlock ? ma.max_deg : kBinBlock));
  if (ma.max_deg > kBinBlock && uint64_t(kGiantBlocks) * gslots > h->gtable_cap) {
    if (h->gtable) {
      cudaStreamSynchronize(h->stream);
      cudaFree(h->gtable);
      h->gtable = nullptr;
      h->gtable_cap = 0;
    }
    DFL_CUDA(h, cudaMalloc(&h->gtable, sizeof(uint2) * uint64_t(kGiantBlocks) * gslots));
    h->gtable_cap = uint64_t(kGiantBlocks) * gslots;
  }
  // once per process (handles may be driven from several host threads)
  static std::once_flag smem_once;
  static cudaError_t smem_rc = cudaSuccess;
  std::call_once(smem_once, [] {
    const int tb = int(sizeof(uint32_t) * 2 * kBlockSlots);
    smem_rc = cudaFuncSetAttribute(k_decide_block<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, tb);
    if (smem_rc == cudaSuccess)
      smem_rc = cudaFuncSetAttribute(k_decide_block<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, tb);
    if (smem_rc == cudaSuccess)
      smem_rc = cudaFuncSetAttribute(k_decide_block<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, tb);
    if (smem_rc == cudaSuccess)
      smem_rc = cudaFuncSetAttribute(k_decide_giant, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(sizeof(uint32_t) * 2 * kGiantSlots));
  });
  DFL_CUDA(h, smem_rc);
  // chunked bin-3 buffers: per list item offsets/counters (sized by the
  // largest bin-3 list: at most arcs / (bin_block + 1) vertices) and partial sums
  {
    uint64_t items = h->pool_top / (uint64_t(h->tune.bin_block) + 1) + 64;
    uint64_t parts = h->pool_top + 64;
    for (int q = 0; q < 2; ++q) parts = parts > h->sg[q].arc_cap ? parts : h->sg[q].arc_cap;
    if (items > h->g_items_cap) {
      cudaStreamSynchronize(h->stream);
      cudaFree(h->g_poff);
      cudaFree(h->g_cpre);
      cudaFree(h->g_done);
      cudaFree(h->g_pcount);
      h->g_poff = nullptr;
      h->g_cpre = h->g_done = h->g_pcount = nullptr;
      h->g_items_cap = 0;
      uint64_t want = items + items / 2;
      DFL_CUDA(h, cudaMalloc(&h->g_poff, sizeof(unsigned long long) * want));
      DFL_CUDA(h, cudaMalloc(&h->g_cpre, sizeof(uint32_t) * (want + 1)));
      DFL_CUDA(h, cudaMalloc(&h->g_done, sizeof(uint32_t) * want));
      DFL_CUDA(h, cudaMalloc(&h->g_pcount, sizeof(uint32_t) * want));
      DFL_CUDA(h, cudaMemsetAsync(h->g_done, 0, sizeof(uint32_t) * want, h->stream));
      DFL_CUDA(h, cudaMemsetAsync(h->g_pcount, 0, sizeof(uint32_t) * want, h->stream));
      h->g_items_cap = want;
    }
    if (ma.max_deg > h->tune.bin_block && parts > h->g_partial_cap) {
      cudaStreamSynchronize(h->stream);
      cudaFree(h->g_partial);
      h->g_partial = nullptr;
      h->g_partial_cap = 0;
      uint64_t want = parts + parts / 4;
      DFL_CUDA(h, cudaMalloc(&h->g_partial, sizeof(uint2) * want));
      h->g_partial_cap = want;
    }
  }
  if (!h->ev_fork) {
    DFL_CUDA(h, cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    for (int b = 0; b < kBins - 1; ++b) {
      DFL_CUDA(h, cudaStreamCreateWithFlags(&h->aux[b], cudaStreamNonBlocking));
      DFL_CUDA(h, cudaEventCreateWithFlags(&h->ev_join[b], cudaEventDisableTiming));
    }
  }
  DFL_CUDA(h, cudaMemsetAsync(&h->ctrl->move_bytes, 0, sizeof(unsigned long long), h->stream));
  DFL_CUDA(h, cudaMemsetAsync(&h->ctrl->ever_count, 0, sizeof(unsigned long long), h->stream));
  {
    LaunchScope ls(h, DFL_PROF_OTHER);
    k_set_m2<<<1, 1, 0, h->stream>>>(h->ctrl, ma.m2);
    DFL_TRY(check_launch(h, "set m2"));
  }
  DecideArgs& a = *out;
  std::memset(&a, 0, sizeof(a));
  a.g = ma.g;
  a.C = ma.C;
  a.K = ma.K;
  a.Sigma = ma.Sigma;
  a.size = ma.size;
  a.m2p = &h->ctrl->m2v;
  a.seg = h->segs;
  a.rbits = ma.use_range ? h->rbits : nullptr;
  a.ever = ma.track_ever ? h->ever : nullptr;
  a.mv_i = h->mv_i;
  a.mv_c = h->mv_c;
  a.mv_d = h->mv_d;
  a.ctrl = h->ctrl;
  a.k = k;
  a.gtable = h->gtable;
  a.gslots = gslots;
  if (h->ngraphs) {
    a.ngraphs = h->ngraphs;
    a.goff = h->d_goff;
    a.gm2 = h->d_gm2;
    a.gdone = h->d_gdone;
    a.gS = h->d_gS;
  }
  *gdo = GiantDecide{h->g_poff, h->g_cpre, h->g_done, h->g_pcount, h->g_partial, nullptr};
  return DFL_OK;
}

}  // namespace

int local_move(Handle* h, const MoveArgs& ma, uint32_t pass, uint32_t* iterations,
               bool record_trace, uint64_t* initial, uint64_t* ever) {
  const uint32_t G = h->ngraphs;
  const u128 threshold = tolerance_threshold(h->opt, ma.m2, pass);
  // a group tests each graph against its own threshold; graphs that have
  // finished (h->gfin) or converge stop being processed
  std::vector<u128> gthr(G);
  std::vector<uint8_t> gactive(G);
  uint32_t nactive = 0;
  for (uint32_t g = 0; g < G; ++g) {
    gthr[g] = tolerance_threshold(h->opt, h->gm2[g], pass);
    gactive[g] = !h->gfin[g];
    nactive += gactive[g];
    h->h_gdone[g] = !gactive[g];
    if (ma.graph_iters) ma.graph_iters[g] = 0;
  }
  if (G) DFL_TRY(group_upload_flags(h, h->d_gdone, h->h_gdone));
  // graph replay of the iterations needs stable buffers (the base graph) and
  // a capturable (non-default) stream
  const bool use_graph = ma.g.off == h->off && h->stream != nullptr &&
                         !(h->opt.flags & DFL_FLAG_NO_GRAPH);
  unsigned int cur_count[kMaxSubsteps][kBins];
  unsigned long long skipped = 0;
  bool have_counts = false;
  if (!use_graph) {
    DFL_TRY(read_ctrl(h));  // list lengths of the initial frontier (buffer 0)
    if (h->hctrl->err) return set_error(h, DFL_ERR_CUDA, "internal error in frontier marking");
    for (uint32_t s = 0; s < kMaxSubsteps; ++s)
      for (int b = 0; b < kBins; ++b) cur_count[s][b] = h->hctrl->count[0][s][b];
    skipped = h->hctrl->skipped;
    have_counts = true;
  }
  DecideArgs a;
  GiantDecide gd;
  DFL_TRY(prepare_move(h, ma, &a, &gd));
  int cur = 0;
  uint32_t it = 0;
  Handle::IterGraph* graph_used[2] = {nullptr, nullptr};
  while (it < h->opt.max_iterations && (!G || nactive)) {
    ++it;
    const int nxt = cur ^ 1;
    if (use_graph) {
      Handle::IterGraph* gp = nullptr;
      DFL_TRY(ensure_iteration_graph(h, a, gd, cur, &gp));
      const Handle::IterGraph& g = *gp;
      graph_used[cur] = gp;
      DFL_CUDA(h, cudaGraphLaunch(g.exec, h->stream));
      h->launches += g.kernels;
      for (int q = 0; q < DFL_PROF_CLASSES; ++q) h->prof.launches[q] += g.class_launches[q];
    } else {
      DFL_TRY(issue_iteration(h, a, cur, cur_count, gd));
    }
    if (G)
      DFL_CUDA(h, cudaMemcpyAsync(h->h_gS, h->d_gS, sizeof(unsigned long long) * 2 * G,
                                  cudaMemcpyDeviceToHost, h->stream));
    DFL_TRY(read_ctrl(h));
    const Ctrl& c = *h->hctrl;
    if (c.err) return set_error(h, DFL_ERR_CUDA, "internal error in local-moving (table overflow)");
    if (use_graph) {
      for (const auto& ev : graph_used[cur]->evs) {  // harvest this replay's timings
        float ms = 0;
        if (cudaEventElapsedTime(&ms, ev.a, ev.b) == cudaSuccess) h->prof.ms[ev.cls] += ms;
      }
      if (it == 1) {
        skipped = c.skipped;
        if (initial) {
          *initial = skipped;
          for (uint32_t s = 0; s < kMaxSubsteps; ++s)
            for (int b = 0; b < kBins; ++b) *initial += c.count[0][s][b];
        }
      }
    } else if (it == 1 && initial) {
      *initial = skipped;
      for (uint32_t s = 0; s < kMaxSubsteps; ++s)
        for (int b = 0; b < kBins; ++b) *initial += cur_count[s][b];
    }
    u128 S = ((u128)c.s_hi << 32) + (u128)c.s_lo;
    if (record_trace) {
      h->trace.push_back(c.processed + skipped);
      h->trace.push_back(c.moved);
      h->trace.push_back(uint64_t(S >> 64));
      h->trace.push_back(uint64_t(S));
    }
    if (have_counts)
      for (uint32_t s = 0; s < kMaxSubsteps; ++s)
        for (int b = 0; b < kBins; ++b) cur_count[s][b] = c.count[nxt][s][b];
    cur = nxt;
    skipped = 0;
    if (!G) {
      if (S <= threshold) break;  // locally converged
      continue;
    }
    bool changed = false;
    for (uint32_t g = 0; g < G; ++g) {
      if (!gactive[g]) continue;
      if (ma.graph_iters) ma.graph_iters[g] = it;
      const u128 Sg = ((u128)h->h_gS[2 * g + 1] << 32) + (u128)h->h_gS[2 * g];
      if (Sg <= gthr[g]) {  // this graph converged: skip its vertices from now on
        gactive[g] = 0;
        h->h_gdone[g] = 1;
        --nactive;
        changed = true;
      }
    }
    if (changed && nactive) DFL_TRY(group_upload_flags(h, h->d_gdone, h->h_gdone));
  }
  h->prof.bytes[DFL_PROF_MOVE] += h->hctrl->move_bytes;
  if (ever) *ever = h->hctrl->ever_count;
  // leave the unprocessed frontier behind: clear the other buffer's bitmap
  DFL_CUDA(h, cudaMemsetAsync(h->fbits[cur], 0, sizeof(uint32_t) * h->words, h->stream));
  *iterations = it;
  return DFL_OK;
}

// Decide phase of one local-moving iteration over the frontier in list
// buffer 0, without applying the moves: `reps` timed runs (the autotuner).
int time_decide(Handle* h, const MoveArgs& ma, uint32_t reps, std::vector<float>* ms) {
  DFL_TRY(read_ctrl(h));
  unsigned int counts[kMaxSubsteps][kBins];
  for (uint32_t s = 0; s < kMaxSubsteps; ++s)
    for (int b = 0; b < kBins; ++b) counts[s][b] = h->hctrl->count[0][s][b];
  if (h->ngraphs) {
    for (uint32_t g = 0; g < h->ngraphs; ++g) h->h_gdone[g] = 0;
    DFL_TRY(group_upload_flags(h, h->d_gdone, h->h_gdone));
  }
  DecideArgs a;
  GiantDecide gd;
  DFL_TRY(prepare_move(h, ma, &a, &gd));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  DFL_CUDA(h, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return set_error(h, DFL_ERR_CUDA, "event");
  }
  int rc = DFL_OK;
  ms->clear();
  for (uint32_t r = 0; r < reps && !rc; ++r) {
    if (cudaMemsetAsync(h->fbits[1], 0, sizeof(uint32_t) * h->words, h->stream) != cudaSuccess)
      rc = set_error(h, DFL_ERR_CUDA, "memset");
    if (!rc) rc = cudaEventRecord(e0, h->stream) == cudaSuccess ? DFL_OK : DFL_ERR_CUDA;
    if (!rc) rc = issue_iteration(h, a, 0, counts, gd, true);
    if (!rc) rc = cudaEventRecord(e1, h->stream) == cudaSuccess ? DFL_OK : DFL_ERR_CUDA;
    if (!rc) rc = read_ctrl(h);
    if (!rc && h->hctrl->err) rc = set_error(h, DFL_ERR_CUDA, "internal error in local-moving");
    float t = 0;
    if (!rc && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess) ms->push_back(t);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

}  // namespace dfl
