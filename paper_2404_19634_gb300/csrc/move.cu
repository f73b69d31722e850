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
#include <type_traits>

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
  uint32_t* bigmv;        // movers of degree > kMarkInline (neighbours marked by k_commit)
  unsigned int* movers;   // movers of the sub-step (slot counter into mv_i/mv_c/mv_d)
  unsigned int* nbig;     // ... of them in bigmv
  unsigned int* clear_movers;  // the next sub-step's two counters, zeroed by this sub-step's
  unsigned int* clear_nbig;    // commit (null: nothing to zero)
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

// m2 * h - k * sig, the numerator of a modularity gain (Eq. 2 scaled by
// 2m^2; a candidate's score or the stay term).  Every factor is below 2^32:
// 2m < 2^32 holds on every graph (dfl_create and dfl_apply_batch refuse
// more), and h, k and sig are sums of parts of 2m.  So each product is one
// 32 x 32 -> 64-bit multiply, and the difference is exact in 128 bits.
__device__ __forceinline__ i128 gain_num(long long m2, unsigned long long h, long long k, long long sig) {
  const unsigned long long p = (unsigned long long)(uint32_t)m2 * (uint32_t)h;
  const unsigned long long q = (unsigned long long)(uint32_t)k * (uint32_t)sig;
  return (i128)p - (i128)q;
}

// Outcome of one vertex's decision, identical on every lane / thread.
__device__ __forceinline__ bool decide_move(const DecideArgs& a, long long m2, uint32_t i, uint32_t d,
                                            long long Ki, bool have, i128 best, uint32_t bc,
                                            unsigned long long Hd, i128* gain) {
  if (!have) return false;
  const i128 stay = gain_num(m2, Hd, Ki, a.Sigma[d] - Ki);
  if (!(best > stay)) return false;
  if (a.size[d] == 1 && a.size[bc] == 1 && bc > d) return false;  // singleton-swap guard
  *gain = best - stay;
  return true;
}

// A decide kernel's counters: summed in registers by the thread that owns a
// vertex's outcome, then once per block (flush_sums).
struct MoveSums {
  unsigned long long bytes = 0, processed = 0, ever = 0, s_lo = 0, s_hi = 0;
};

__device__ __forceinline__ void record_move(const DecideArgs& a, uint32_t i, uint32_t c, uint32_t d,
                                            i128 gain, uint32_t gi, MoveSums& sums) {
  uint32_t slot = atomicAdd(a.movers, 1u);
  a.mv_i[slot] = i;
  a.mv_c[slot] = c;
  a.mv_d[slot] = d;
  sums.s_lo += (unsigned long long)((u128)gain & 0xFFFFFFFFull);
  sums.s_hi += (unsigned long long)((u128)gain >> 32);
  if (a.ngraphs) {
    const u128 v = (u128)gain;
    const unsigned long long lo = (unsigned long long)(v & 0xFFFFFFFFull);
    const unsigned long long hi = (unsigned long long)(v >> 32);
    if (lo) atomicAdd(a.gS + 2 * gi, lo);
    if (hi) atomicAdd(a.gS + 2 * gi + 1, hi);
  }
}

// Block-wide sums of the counters held by `holder` threads, one global
// atomic each per block.  Every thread of the block must call it.
__device__ __forceinline__ void flush_sums(const DecideArgs& a, const MoveSums& v, bool holder) {
  __shared__ unsigned long long sh[5];
  if (threadIdx.x < 5) sh[threadIdx.x] = 0;
  __syncthreads();
  if (holder) {
    if (v.bytes) atomicAdd(&sh[0], v.bytes);
    if (v.processed) atomicAdd(&sh[1], v.processed);
    if (v.ever) atomicAdd(&sh[2], v.ever);
    if (v.s_lo) atomicAdd(&sh[3], v.s_lo);
    if (v.s_hi) atomicAdd(&sh[4], v.s_hi);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (sh[0]) atomicAdd(&a.ctrl->move_bytes, sh[0]);
    if (sh[1]) atomicAdd(&a.ctrl->processed, sh[1]);
    if (sh[2]) atomicAdd(&a.ctrl->ever_count, sh[2]);
    if (sh[3]) atomicAdd(&a.ctrl->s_lo, sh[3]);
    if (sh[4]) atomicAdd(&a.ctrl->s_hi, sh[4]);
  }
}

// flush_sums for kernels where every thread holds counts: the warp sums
// them first, so the block's shared counters take one update per warp.
__device__ __forceinline__ void flush_sums_all(const DecideArgs& a, MoveSums v) {
#pragma unroll
  for (int x = 16; x; x >>= 1) {
    v.bytes += __shfl_xor_sync(0xFFFFFFFFu, v.bytes, x);
    v.s_lo += __shfl_xor_sync(0xFFFFFFFFu, v.s_lo, x);
    v.s_hi += __shfl_xor_sync(0xFFFFFFFFu, v.s_hi, x);
  }
  v.processed = __reduce_add_sync(0xFFFFFFFFu, uint32_t(v.processed));
  v.ever = __reduce_add_sync(0xFFFFFFFFu, uint32_t(v.ever));
  flush_sums(a, v, (threadIdx.x & 31u) == 0);
}

// A mover of more than kMarkInline arcs does not mark its neighbours itself
// (one block would walk them all while the rest of the GPU idles): it is
// listed, and k_commit spreads every listed mover's arcs over all blocks.
constexpr uint32_t kMarkInline = 512;
constexpr uint32_t kMarkChunk = 1024;

// Mark neighbour j of a mover for the next iteration: its bit in the next
// frontier's bitmap (the lists are built from the bitmap once, at the end of
// the iteration).  The bit is read first, so a vertex marked by many movers
// takes one atomic.
__device__ __forceinline__ void mark_next(const DecideArgs& a, uint32_t j, bool valid) {
  if (valid && (!a.rbits || bit_test(a.rbits, j)) && !bit_test(a.fbits_next, j)) bit_set(a.fbits_next, j);
}

// ---------------------------------------------------------------------------
// Bin 0: small degrees (at most W <= 32 arcs), W lanes per vertex, so one
// warp decides 32 / W vertices at once, one arc per lane; aggregation by
// community in registers inside each W-lane segment (W shuffles and
// compares).  A long bin-0 list instead takes a vertex per thread
// (k_decide_thread, below).
// ---------------------------------------------------------------------------

// Argmax of (score, -c) over the aligned W-lane segment of each lane.
template <int W>
__device__ __forceinline__ void segment_argmax(bool& have, i128& score, uint32_t& c) {
#pragma unroll
  for (int s = W / 2; s >= 1; s >>= 1) {
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

// One vertex per W-lane segment (`active` false: the segment idles).  Every
// lane of the warp must call it.  Returns the segment's move decision.
template <int W>
__device__ __forceinline__ bool decide_segment(const DecideArgs& a, bool active, uint32_t i, long long m2,
                                               uint32_t gi, MoveSums& sums) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t seg = lane / W, sl = lane % W;
  const unsigned segmask = W == 32 ? 0xFFFFFFFFu : (((1u << W) - 1u) << (seg * W));
  const uint32_t d = active ? a.C[i] : 0u;
  const long long Ki = active ? a.K[i] : 0;
  const unsigned long long o = active ? a.g.off[i] : 0ull;
  const uint32_t dg = active ? a.g.deg[i] : 0u;
  uint2 arc = sl < dg ? a.g.arcs[o + sl] : make_uint2(i, 0u);
  const bool valid = sl < dg && arc.x != i && arc.y != 0;  // weight 0 = deleted arc
  const uint32_t c = valid ? a.C[arc.x] : kEmpty;
  // weight of this lane's community within the segment, and whether this is
  // the community's first lane: W shuffles and compares (cheaper here than
  // match/reduce over many groups)
  uint32_t hsum = 0;
  bool leader = valid;
  const uint32_t wv = valid ? arc.y : 0u;
#pragma unroll
  for (int k = 0; k < W; ++k) {
    const uint32_t src = seg * W + k;
    const uint32_t ck = __shfl_sync(0xFFFFFFFFu, c, src);
    const uint32_t wk = __shfl_sync(0xFFFFFFFFu, wv, src);
    if (valid && ck == c) {
      hsum += wk;
      if (uint32_t(k) < sl) leader = false;
    }
  }
  const unsigned dm = __ballot_sync(0xFFFFFFFFu, leader && c == d) & segmask;
  // every lane shuffles (from its segment's holder of d, or from itself)
  const uint32_t hd_src = dm ? uint32_t(__ffs(dm) - 1) : lane;
  const uint32_t hd_val = __shfl_sync(0xFFFFFFFFu, hsum, hd_src);
  const unsigned long long Hd = dm ? hd_val : 0u;
  const bool cand = leader && c != d;
  const unsigned cm = __ballot_sync(0xFFFFFFFFu, cand) & segmask;
  i128 score = 0;
  if (cand) score = gain_num(m2, hsum, Ki, a.Sigma[c]);
  bool have = cand;
  uint32_t bc = c;
  segment_argmax<W>(have, score, bc);
  i128 gain = 0;
  const bool mv = active && decide_move(a, m2, i, d, Ki, have, score, bc, Hd, &gain);
  if (active && sl == 0) sums.bytes += 24 + 12ull * dg + 12ull * __popc(cm);
  if (mv) {
    if (sl == 0) {
      record_move(a, i, bc, d, gain, gi, sums);
      sums.bytes += 16 + 4ull * dg;
    }
  }
  mark_next(a, arc.x, mv && valid);
  return mv;
}

template <int W>
__global__ void __launch_bounds__(256, 5) k_decide_warp(DecideArgs a) {
  constexpr uint32_t kSegs = 32 / W;
  const long long m2_one = *a.m2p;
  const uint32_t lane = threadIdx.x & 31u, seg = lane / W, sl = lane % W;
  const uint32_t cnt = *a.count;
  const uint64_t warp = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) >> 5;
  const uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  MoveSums sums;
  for (uint64_t t0 = warp * kSegs; t0 < cnt; t0 += nwarps * kSegs) {
    const uint64_t t = t0 + seg;
    bool active = t < cnt;
    const uint32_t i = active ? a.list[t] : 0u;
    long long m2 = m2_one;
    uint32_t gi = 0;
    if (active && !group_active(a, i, &m2, &gi)) active = false;
    if (active && sl == 0) {
      if (a.ever && bit_set(a.ever, i)) ++sums.ever;
      ++sums.processed;
    }
    if (active && a.rbits && !bit_test(a.rbits, i)) active = false;  // processed, not in range
    decide_segment<W>(a, active, i, m2, gi, sums);
  }
  flush_sums(a, sums, sl == 0);
}

// Open-addressing insert (linear probing) of weight w under key c; gives up
// after `limit` probes (the caller then falls back to a larger table).
__device__ __forceinline__ bool table_add(uint32_t* keys, uint32_t* vals, uint32_t mask, uint32_t c,
                                          uint32_t w, uint32_t limit) {
  uint32_t s = hash_move(c) & mask;
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
// every lane adds its arc's weight under its neighbour's community (shared
// memory atomics).  Grouping equal communities inside the warp first was
// measured slower on this GPU both ways tried: match/reduce when a warp
// holds many communities, and ballot/shuffle rounds that sum the lanes of
// the first pending lane's community (even for hubs whose thousands of arcs
// lead to a few dozen communities, the DF decide phase on R-MAT 2^22 went
// from 0.219 to 0.246-0.296 ms with 2-8 such rounds).  Loads of kUnroll
// chunks are issued before use.
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
    for (int u = 0; u < kUnroll; ++u)
      if (c[u] != kEmpty) ok &= table_add(keys, vals, mask, c[u], arc[u].y, limit);
  }
  return ok;
}

// Best candidate of table slots start, start + step, ... below `slots`: U
// slots' keys and values, then their Sigma gathers, are issued before any is
// used, so a thread waits once per U occupied slots.  Returns (per thread)
// the weight to d if this thread met d's slot, and counts candidates.
template <int U>
__device__ __forceinline__ unsigned long long table_argmax(const DecideArgs& a, const uint32_t* keys,
                                                           const uint32_t* vals, uint32_t slots,
                                                           uint32_t start, uint32_t step, uint32_t d,
                                                           long long m2, long long Ki, bool& have,
                                                           i128& best, uint32_t& bc, uint32_t& ncand) {
  unsigned long long hd = 0;
  for (uint32_t s0 = start; s0 < slots; s0 += step * U) {
    uint32_t c[U], w[U];
    long long sg[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t sl = s0 + u * step;
      c[u] = sl < slots ? keys[sl] : kEmpty;
      w[u] = sl < slots ? vals[sl] : 0u;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) sg[u] = (c[u] != kEmpty && c[u] != d) ? a.Sigma[c[u]] : 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (c[u] == kEmpty) continue;
      if (c[u] == d) {
        hd = w[u];
        continue;
      }
      ++ncand;
      const i128 sc = gain_num(m2, w[u], Ki, sg[u]);
      if (!have || sc > best || (sc == best && c[u] < bc)) {
        have = true;
        best = sc;
        bc = c[u];
      }
    }
  }
  return hd;
}

// Reduce (have, score, c) of every thread of the block to thread 0 (larger
// score wins, ties to the smaller c); every thread calls it.
constexpr uint32_t kMaxBlockWarps = 16;  // blocks of up to 512 threads

__device__ __forceinline__ void block_argmax(bool& have, i128& best, uint32_t& bc) {
  __shared__ unsigned long long s_lo[kMaxBlockWarps], s_hi[kMaxBlockWarps];
  __shared__ uint32_t s_c[kMaxBlockWarps];
  __shared__ int s_have[kMaxBlockWarps];
  const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5, nw = blockDim.x / 32;
  warp_argmax(have, best, bc);
  __syncthreads();
  if (lane == 0) {
    s_lo[wib] = (unsigned long long)(u128)best;
    s_hi[wib] = (unsigned long long)((u128)best >> 64);
    s_c[wib] = bc;
    s_have[wib] = have;
  }
  __syncthreads();
  if (wib == 0) {
    have = lane < nw && s_have[lane];
    best = lane < nw ? (i128)(((u128)s_hi[lane] << 64) | (u128)s_lo[lane]) : 0;
    bc = lane < nw ? s_c[lane] : 0;
    warp_argmax(have, best, bc);
  }
}

// ---------------------------------------------------------------------------
// Bin 1: 32 < deg <= 256, one warp per vertex with a shared table.
// ---------------------------------------------------------------------------
constexpr uint32_t kWarpSlots = 512;
constexpr int kWarpHashWarps = 8;
static_assert(kBinWarpHash <= 8 * 32 && 2 * kBinWarpHash <= kWarpSlots, "a bin-1 vertex fits 8 arcs a lane and its table");

// One vertex of bin 1 by one warp (its degree up to kWarpSlots / 2): up to
// 32 arcs by the register path, else a shared table of the warp.  Every lane
// of the warp calls it.
__device__ __forceinline__ void warp_table_vertex(const DecideArgs& a, uint32_t i, long long m2, uint32_t gi,
                                                  uint32_t* keys, uint32_t* vals, MoveSums& sums) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t dg = a.g.deg[i];
  if (dg <= 32) {  // (when bin 0 takes fewer than 32 arcs) registers, not a table
    decide_segment<32>(a, true, i, m2, gi, sums);
    return;
  }
  const uint32_t d = a.C[i];
  const long long Ki = a.K[i];
  const unsigned long long o = a.g.off[i];
  uint32_t slots = 64;
  while (slots < 2 * dg && slots < kWarpSlots) slots <<= 1;
  const uint32_t mask = slots - 1;
  for (uint32_t s = lane; s < slots; s += 32) {
    keys[s] = kEmpty;
    vals[s] = 0;
  }
  __syncwarp();
  bool ok = scan_row<8>(a, i, o, dg, 0, 32, keys, vals, mask, slots);
  if (!__all_sync(0xFFFFFFFFu, ok) && lane == 0) atomicOr(&a.ctrl->err, kErrInternal);
  __syncwarp();
  bool have = false;
  i128 best = 0;
  uint32_t bc = 0;
  uint32_t ncand = 0;
  unsigned long long Hd = table_argmax<4>(a, keys, vals, slots, lane, 32, d, m2, Ki, have, best, bc, ncand);
  for (int x = 16; x; x >>= 1) {
    Hd += __shfl_xor_sync(0xFFFFFFFFu, Hd, x);
    ncand += __shfl_xor_sync(0xFFFFFFFFu, ncand, x);
  }
  warp_argmax(have, best, bc);
  i128 gain = 0;
  bool mv = decide_move(a, m2, i, d, Ki, have, best, bc, Hd, &gain);
  if (lane == 0) sums.bytes += 24 + 12ull * dg + 12ull * ncand;
  if (mv) {
    if (lane == 0) {
      record_move(a, i, bc, d, gain, gi, sums);
      sums.bytes += 16 + 4ull * dg;
    }
    for (uint32_t k0 = 0; k0 < dg; k0 += 32) {
      uint32_t k = k0 + lane;
      uint2 arc = k < dg ? a.g.arcs[o + k] : make_uint2(i, 0u);
      mark_next(a, arc.x, k < dg && arc.x != i && arc.y != 0);
    }
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// Vertex headers a warp at a time.  A vertex's decision is a chain of
// dependent loads: list entry -> its row offset, degree, community and K ->
// the Sigma and size of its community -> its arcs -> the neighbours'
// communities -> the candidates' Sigma.  The kernels below take the first
// links of that chain for up to 32 list positions at once (one lane each),
// so they wait for them once per batch of vertices instead of once per
// vertex.
// ---------------------------------------------------------------------------

// K_i, Sigma_d and 2m are below 2^32 (2m < 2^32 on every graph, and K_i and
// Sigma_d are parts of 2m), so they travel as 32-bit words.
struct VHdr {
  unsigned long long o;  // row offset
  uint32_t Ki, Sd, m2;   // K_i, Sigma of its community d, 2m of its graph
  uint32_t i, d, dg, gi;
  int szd;               // size of d
  bool act;              // processed and in the affected range: decide it
};

// Sigma_c as a 32-bit word (the low half of the int64: Sigma_c is in [0, 2m)).
__device__ __forceinline__ uint32_t sigma32(const long long* Sigma, uint32_t c) {
  return reinterpret_cast<const uint32_t*>(Sigma)[2ull * c];
}

// Exact 64-bit form of Eq. 2's comparisons.  Adding K_i * 2m to every score
// of vertex i shifts them all by the same amount:
//   score'(c) = 2m * H[c] + K_i * (2m - Sigma_c)           (a candidate c)
//   stay'     = 2m * H[d] + K_i * (2m - (Sigma_d - K_i))
// so the best candidate, the move test score > stay and the gain score - stay
// are unchanged.  Each is at most 2 * 2m * K_i (H[c] <= K_i and Sigma_c <= 2m),
// so it fits 64 bits whenever 2m * K_i < 2^63, which holds unless 2m and K_i
// both approach 2^32; those vertices take the 128-bit path.  A candidate's
// score' is at least 1 (H[c] >= 1).
__device__ __forceinline__ bool fits64(uint32_t m2, uint32_t Ki) {
  return (unsigned long long)m2 * Ki < (1ull << 63);
}
__device__ __forceinline__ unsigned long long score64(uint32_t m2, uint32_t h, uint32_t Ki, uint32_t sig) {
  return (unsigned long long)m2 * h + (unsigned long long)Ki * (m2 - sig);
}

// Warp-wide best (largest score', then smallest c) of the lanes with `have`,
// by three warp reductions; the result on every lane.
__device__ __forceinline__ void warp_best64(bool& have, unsigned long long& s, uint32_t& c) {
  const uint32_t hi = have ? uint32_t(s >> 32) : 0u, lo = have ? uint32_t(s) : 0u;
  const uint32_t mh = __reduce_max_sync(0xFFFFFFFFu, hi);
  const uint32_t ml = __reduce_max_sync(0xFFFFFFFFu, (have && hi == mh) ? lo : 0u);
  c = __reduce_min_sync(0xFFFFFFFFu, (have && hi == mh && lo == ml) ? c : kEmpty);
  s = ((unsigned long long)mh << 32) | ml;
  have = c != kEmpty;
}

// This lane's header of list position t (`valid`: t is in the list).  The
// vertex is counted as processed (and newly ever-processed) as in the
// per-vertex kernels.
__device__ __forceinline__ void load_header(const DecideArgs& a, uint64_t t, bool valid, long long m2_one,
                                            MoveSums& sums, VHdr& h) {
  h.i = valid ? a.list[t] : 0u;
  long long m2 = m2_one;
  h.gi = 0;
  if (valid && !group_active(a, h.i, &m2, &h.gi)) valid = false;
  h.m2 = uint32_t(m2);
  // the row and state loads are issued before the bookkeeping atomics
  h.d = valid ? a.C[h.i] : 0u;
  h.Ki = valid ? uint32_t(a.K[h.i]) : 0u;
  h.o = valid ? a.g.off[h.i] : 0ull;
  h.dg = valid ? a.g.deg[h.i] : 0u;
  bool inr = valid;
  if (valid) {
    if (a.ever && bit_set(a.ever, h.i)) ++sums.ever;
    ++sums.processed;
    if (a.rbits) inr = bit_test(a.rbits, h.i);
  }
  h.act = inr;
  h.Sd = inr ? sigma32(a.Sigma, h.d) : 0u;
  h.szd = inr ? a.size[h.d] : 0;
}

__device__ __forceinline__ VHdr shfl_header(const VHdr& h, int k) {
  VHdr v;
  v.o = __shfl_sync(0xFFFFFFFFu, h.o, k);
  v.Ki = __shfl_sync(0xFFFFFFFFu, h.Ki, k);
  v.Sd = __shfl_sync(0xFFFFFFFFu, h.Sd, k);
  v.m2 = __shfl_sync(0xFFFFFFFFu, h.m2, k);
  v.i = __shfl_sync(0xFFFFFFFFu, h.i, k);
  v.d = __shfl_sync(0xFFFFFFFFu, h.d, k);
  v.dg = __shfl_sync(0xFFFFFFFFu, h.dg, k);
  v.gi = __shfl_sync(0xFFFFFFFFu, h.gi, k);
  v.szd = __shfl_sync(0xFFFFFFFFu, h.szd, k);
  v.act = true;
  return v;
}

// The move decision of Eq. 2 from the best candidate (score' form), with the
// community's Sigma and size already loaded: the best candidate's size is
// read only when the singleton-swap guard needs it.
__device__ __forceinline__ bool decide64(const DecideArgs& a, const VHdr& v, bool have, unsigned long long best,
                                         uint32_t bc, uint32_t Hd, i128* gain) {
  if (!have) return false;
  const unsigned long long stay = score64(v.m2, Hd, v.Ki, v.Sd - v.Ki);
  if (!(best > stay)) return false;
  if (v.szd == 1 && bc > v.d && a.size[bc] == 1) return false;  // singleton-swap guard
  *gain = (i128)(best - stay);
  return true;
}

// The same in 128 bits (vertices whose 2m * K_i reaches 2^63).
__device__ __forceinline__ bool decide128(const DecideArgs& a, const VHdr& v, bool have, i128 best, uint32_t bc,
                                          uint32_t Hd, i128* gain) {
  if (!have) return false;
  const i128 stay = gain_num(v.m2, Hd, v.Ki, v.Sd - v.Ki);
  if (!(best > stay)) return false;
  if (v.szd == 1 && bc > v.d && a.size[bc] == 1) return false;
  *gain = best - stay;
  return true;
}

// record_move for every mover lane of the warp with one slot reservation.
// Every lane of the warp calls it.
__device__ __forceinline__ void record_moves_warp(const DecideArgs& a, bool mv, uint32_t i, uint32_t c,
                                                  uint32_t d, i128 gain, uint32_t gi, MoveSums& sums) {
  const unsigned m = __ballot_sync(0xFFFFFFFFu, mv);
  if (!m) return;
  const uint32_t lane = threadIdx.x & 31u;
  const int first = __ffs(m) - 1;
  uint32_t base = 0;
  if (int(lane) == first) base = atomicAdd(a.movers, uint32_t(__popc(m)));
  base = __shfl_sync(0xFFFFFFFFu, base, first);
  if (!mv) return;
  const uint32_t slot = base + __popc(m & ((1u << lane) - 1u));
  a.mv_i[slot] = i;
  a.mv_c[slot] = c;
  a.mv_d[slot] = d;
  const u128 v = (u128)gain;
  const unsigned long long lo = (unsigned long long)(v & 0xFFFFFFFFull);
  const unsigned long long hi = (unsigned long long)(v >> 32);
  sums.s_lo += lo;
  sums.s_hi += hi;
  if (a.ngraphs) {
    if (lo) atomicAdd(a.gS + 2 * gi, lo);
    if (hi) atomicAdd(a.gS + 2 * gi + 1, hi);
  }
}

// ---------------------------------------------------------------------------
// Bin 0: one thread per vertex (degree <= D), its arcs, their communities and
// the community weights in registers; the weight of a community is summed
// by its first arc over the others (D x D compares, no table, no shuffles).
// ---------------------------------------------------------------------------

// Best candidate over the thread's community weights (hw[k] > 0: arc k is the
// first of a candidate community c[k]) and the move decision.
template <int D, bool F64>
__device__ __forceinline__ bool thread_decide(const DecideArgs& a, const VHdr& h, const uint32_t* c,
                                              const uint32_t* hw, const uint32_t* sg, uint32_t Hd, uint32_t* bco,
                                              i128* gain) {
  bool have = false;
  uint32_t bc = 0;
  typename std::conditional<F64, unsigned long long, i128>::type best = 0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    if (!hw[k]) continue;
    decltype(best) sc;
    if constexpr (F64) sc = score64(h.m2, hw[k], h.Ki, sg[k]);
    else sc = gain_num(h.m2, hw[k], h.Ki, sg[k]);
    if (!have || sc > best || (sc == best && c[k] < bc)) {
      have = true;
      best = sc;
      bc = c[k];
    }
  }
  *bco = bc;
  if constexpr (F64) return decide64(a, h, have, best, bc, Hd, gain);
  else return decide128(a, h, have, best, bc, Hd, gain);
}

template <int D>
__global__ void __launch_bounds__(256, 3) k_decide_thread(DecideArgs a) {
  const long long m2_one = *a.m2p;
  const uint32_t cnt = *a.count;
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  MoveSums sums;
  for (uint64_t t0 = blockIdx.x * uint64_t(blockDim.x) + (threadIdx.x & ~31u); t0 < cnt; t0 += stride) {
    const uint64_t t = t0 + lane;  // warp-uniform loop: the movers are recorded per warp
    VHdr h;
    load_header(a, t, t < cnt, m2_one, sums, h);
    uint2 arc[D];
#pragma unroll
    for (int k = 0; k < D; ++k) arc[k] = (h.act && uint32_t(k) < h.dg) ? a.g.arcs[h.o + k] : make_uint2(h.i, 0u);
    uint32_t c[D];
#pragma unroll
    for (int k = 0; k < D; ++k) c[k] = (arc[k].x != h.i && arc[k].y != 0) ? a.C[arc[k].x] : kEmpty;
    // hw[k]: weight of candidate community c[k] if arc k is its first arc, else 0
    uint32_t hw[D];
    uint32_t Hd = 0, ncand = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      uint32_t sum = 0;
      bool lead = c[k] != kEmpty;
#pragma unroll
      for (int m = 0; m < D; ++m)
        if (c[m] == c[k]) {
          sum += arc[m].y;
          if (m < k) lead = false;
        }
      if (lead && c[k] == h.d) Hd = sum;
      hw[k] = lead && c[k] != h.d ? sum : 0u;  // a valid arc weighs at least 1
      ncand += hw[k] ? 1u : 0u;
    }
    uint32_t sg[D];
#pragma unroll
    for (int k = 0; k < D; ++k) sg[k] = hw[k] ? sigma32(a.Sigma, c[k]) : 0u;
    uint32_t bc = 0;
    i128 gain = 0;
    bool mv = false;
    if (h.act) {
      mv = fits64(h.m2, h.Ki) ? thread_decide<D, true>(a, h, c, hw, sg, Hd, &bc, &gain)
                              : thread_decide<D, false>(a, h, c, hw, sg, Hd, &bc, &gain);
      sums.bytes += 24 + 12ull * h.dg + 12ull * ncand;
    }
    record_moves_warp(a, mv, h.i, bc, h.d, gain, h.gi, sums);
    if (mv) {  // the arcs again (cached)
      sums.bytes += 16 + 4ull * h.dg;
      for (uint32_t k = 0; k < h.dg; ++k) {
        const uint2 e = a.g.arcs[h.o + k];
        mark_next(a, e.x, e.x != h.i && e.y != 0);
      }
    }
  }
  flush_sums_all(a, sums);
}

// ---------------------------------------------------------------------------
// Bin 1: one warp per vertex, vertices taken in batches of up to 32 headers.
// A vertex of at most 32 arcs is decided in registers (one arc per lane);
// a larger one in the warp's shared table.  The table is empty at rest: the
// lane that creates a community's slot loads that community's Sigma at once,
// and after the last arc is in, scores the slot and clears it, so the table
// is neither cleared nor scanned as a whole.  Vertices whose scores need
// 128 bits take the per-vertex path of the persistent kernel.
// ---------------------------------------------------------------------------

// Decision of vertex v (at most 32 arcs; `arc` = this lane's arc, lane < dg,
// else (i, 0)), identical on every lane; *ncand on every lane.
__device__ __forceinline__ bool reg_vertex(const DecideArgs& a, const VHdr& v, uint2 arc, uint32_t* bco,
                                           i128* gain, uint32_t* ncand) {
  const uint32_t lane = threadIdx.x & 31u;
  const bool valid = lane < v.dg && arc.x != v.i && arc.y != 0;
  const uint32_t c = valid ? a.C[arc.x] : kEmpty;
  const uint32_t wv = valid ? arc.y : 0u;
  uint32_t hsum = 0;
  bool leader = valid;
  for (uint32_t k = 0; k < v.dg; ++k) {  // warp-uniform bound
    const uint32_t ck = __shfl_sync(0xFFFFFFFFu, c, k);
    const uint32_t wk = __shfl_sync(0xFFFFFFFFu, wv, k);
    if (valid && ck == c) {
      hsum += wk;
      if (k < lane) leader = false;
    }
  }
  const uint32_t Hd = __reduce_add_sync(0xFFFFFFFFu, (leader && c == v.d) ? hsum : 0u);
  bool cand = leader && c != v.d;
  *ncand = __popc(__ballot_sync(0xFFFFFFFFu, cand));
  unsigned long long s = cand ? score64(v.m2, hsum, v.Ki, sigma32(a.Sigma, c)) : 0ull;
  uint32_t bc = c;
  warp_best64(cand, s, bc);
  *bco = bc;
  return decide64(a, v, cand, s, bc, Hd, gain);
}

// Decision of vertex v (32 < degree <= 32 U) in the warp's table (keys kEmpty
// and values 0 at rest, and left so).  `a0` is this lane's first arc,
// loaded ahead.  Returns the decision on every lane; a mover's arcs are read
// again to mark the next frontier.
template <int U>
__device__ __forceinline__ bool table_vertex(const DecideArgs& a, const VHdr& v, uint2 a0, uint32_t* keys,
                                             uint32_t* vals, uint32_t* bco, i128* gain, uint32_t* ncand) {
  const uint32_t lane = threadIdx.x & 31u;
  uint32_t slots = 64;
  while (slots < 2 * v.dg) slots <<= 1;  // at most 64 U: never full
  const uint32_t mask = slots - 1;
  uint2 arc[U];
  arc[0] = a0;
#pragma unroll
  for (int u = 1; u < U; ++u) {
    const uint32_t k = u * 32 + lane;
    arc[u] = k < v.dg ? a.g.arcs[v.o + k] : make_uint2(v.i, 0u);
  }
  uint32_t c[U];
#pragma unroll
  for (int u = 0; u < U; ++u) c[u] = (arc[u].x != v.i && arc[u].y != 0) ? a.C[arc[u].x] : kEmpty;
  uint32_t cs[U], sg[U];
  bool ok = true;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    cs[u] = kEmpty;
    sg[u] = 0;
    if (c[u] == kEmpty) continue;
    uint32_t s = hash_move(c[u]) & mask;
    bool placed = false;
    for (uint32_t probe = 0; probe < slots; ++probe) {
      uint32_t prev = keys[s];
      if (prev == kEmpty) prev = atomicCAS(&keys[s], kEmpty, c[u]);
      if (prev == kEmpty) {  // created: this lane scores the slot
        cs[u] = s;
        if (c[u] != v.d) sg[u] = sigma32(a.Sigma, c[u]);
      }
      if (prev == kEmpty || prev == c[u]) {
        atomicAdd(&vals[s], arc[u].y);
        placed = true;
        break;
      }
      s = (s + 1) & mask;
    }
    ok &= placed;
  }
  if (!__all_sync(0xFFFFFFFFu, ok) && lane == 0) atomicOr(&a.ctrl->err, kErrInternal);
  __syncwarp();  // every arc is in
  bool have = false;
  unsigned long long best = 0;
  uint32_t bc = 0, nc = 0, Hd = 0;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    if (cs[u] == kEmpty) continue;
    const uint32_t hw = vals[cs[u]];
    keys[cs[u]] = kEmpty;  // only this lane reads the slot it created
    vals[cs[u]] = 0;
    if (c[u] == v.d) {
      Hd = hw;
      continue;
    }
    ++nc;
    const unsigned long long sc = score64(v.m2, hw, v.Ki, sg[u]);
    if (!have || sc > best || (sc == best && c[u] < bc)) {
      have = true;
      best = sc;
      bc = c[u];
    }
  }
  __syncwarp();  // the table is empty again before the next vertex
  Hd = __reduce_add_sync(0xFFFFFFFFu, Hd);
  *ncand = __reduce_add_sync(0xFFFFFFFFu, nc);
  warp_best64(have, best, bc);
  *bco = bc;
  const bool mv = decide64(a, v, have, best, bc, Hd, gain);
  if (mv) {  // the arcs again (cached): holding them in registers costs occupancy
    for (uint32_t k = lane; k < v.dg; k += 32) {
      const uint2 e = a.g.arcs[v.o + k];
      mark_next(a, e.x, e.x != v.i && e.y != 0);
    }
  }
  return mv;
}

// The rare 128-bit vertices, out of line so that they do not cost the common
// path registers.
__device__ __noinline__ void warp_vertex_128(const DecideArgs& a, const VHdr& v, uint32_t* keys, uint32_t* vals,
                                             MoveSums& sums) {
  warp_table_vertex(a, v.i, v.m2, v.gi, keys, vals, sums);
}

__global__ void __launch_bounds__(256, 3) k_decide_warp_hash(DecideArgs a) {
  __shared__ uint32_t skeys[kWarpHashWarps][kWarpSlots];
  __shared__ uint32_t svals[kWarpHashWarps][kWarpSlots];
  const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
  uint32_t* keys = skeys[wib];
  uint32_t* vals = svals[wib];
  for (uint32_t s = lane; s < kWarpSlots; s += 32) {
    keys[s] = kEmpty;
    vals[s] = 0;
  }
  __syncwarp();
  const long long m2_one = *a.m2p;
  const uint32_t cnt = *a.count;
  const uint64_t warp = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) >> 5;
  const uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  // vertices per warp and round: up to 32, fewer when the list is short
  uint64_t B = (uint64_t(cnt) + nwarps - 1) / nwarps;
  B = B < 1 ? 1 : B > 32 ? 32 : B;
  MoveSums sums;
  for (uint64_t t0 = warp * B; t0 < cnt; t0 += nwarps * B) {
    VHdr h;
    load_header(a, t0 + lane, lane < B && t0 + lane < cnt, m2_one, sums, h);
    bool my_mv = false;
    uint32_t my_c = 0;
    i128 my_gain = 0;
    unsigned m = __ballot_sync(0xFFFFFFFFu, h.act);
    // each vertex's first 32 arcs are loaded while the one before is decided
    uint2 pre = make_uint2(0u, 0u);
    if (m) {
      const int k = __ffs(m) - 1;
      const unsigned long long o = __shfl_sync(0xFFFFFFFFu, h.o, k);
      const uint32_t dg = __shfl_sync(0xFFFFFFFFu, h.dg, k), i = __shfl_sync(0xFFFFFFFFu, h.i, k);
      pre = lane < dg ? a.g.arcs[o + lane] : make_uint2(i, 0u);
    }
    while (m) {
      const int k = __ffs(m) - 1;
      m &= m - 1;
      const VHdr v = shfl_header(h, k);
      const uint2 a0 = pre;
      if (m) {
        const int k1 = __ffs(m) - 1;
        const unsigned long long o = __shfl_sync(0xFFFFFFFFu, h.o, k1);
        const uint32_t dg = __shfl_sync(0xFFFFFFFFu, h.dg, k1), i = __shfl_sync(0xFFFFFFFFu, h.i, k1);
        pre = lane < dg ? a.g.arcs[o + lane] : make_uint2(i, 0u);
      }
      if (!fits64(v.m2, v.Ki)) {  // 128-bit scores: the per-vertex path, then the table emptied again
        warp_vertex_128(a, v, keys, vals, sums);
        for (uint32_t s = lane; s < kWarpSlots; s += 32) {
          keys[s] = kEmpty;
          vals[s] = 0;
        }
        __syncwarp();
        continue;
      }
      uint32_t bc = 0, ncand = 0;
      i128 gain = 0;
      bool mv;
      if (v.dg <= 32) {
        mv = reg_vertex(a, v, a0, &bc, &gain, &ncand);
        if (mv) mark_next(a, a0.x, lane < v.dg && a0.x != v.i && a0.y != 0);
      } else if (v.dg <= 64) {
        mv = table_vertex<2>(a, v, a0, keys, vals, &bc, &gain, &ncand);
      } else if (v.dg <= 128) {
        mv = table_vertex<4>(a, v, a0, keys, vals, &bc, &gain, &ncand);
      } else {
        mv = table_vertex<8>(a, v, a0, keys, vals, &bc, &gain, &ncand);
      }
      if (int(lane) == k) {
        sums.bytes += 24 + 12ull * v.dg + 12ull * ncand + (mv ? 16 + 4ull * v.dg : 0ull);
        my_mv = mv;
        my_c = bc;
        my_gain = gain;
      }
    }
    record_moves_warp(a, my_mv, h.i, my_c, h.d, my_gain, h.gi, sums);
  }
  flush_sums_all(a, sums);
}

// ---------------------------------------------------------------------------
// Bins 2 and 3: one block per vertex with a shared table of kBlockSlots
// (bin 2 fits by construction; a bin-3 vertex has so many neighbours that the
// number of distinct neighbour communities, not the degree, sizes the table).
// If a bin-3 vertex overflows the shared table, it is redone with a table in
// a per-block slice of global memory sized from the maximum degree.
// ---------------------------------------------------------------------------
constexpr uint32_t kBlockSlots = 2 * kBinBlock;  // 8192 keys + 8192 values = 64 KB

// Shared scalars of the block-level bodies.
struct BlockScratch {
  unsigned long long hd;
  uint32_t ncand, ne;
  int ok, last;
};

// One vertex by the whole block (up to 512 threads): a shared table of
// 2 x degree slots at `dyn` (at most kBlockSlots keys + values); a vertex of
// larger degree whose distinct communities overflow it is redone in the
// block's slice of the global table.  Every thread of the block calls it.
template <int kThreads>
__device__ __forceinline__ void block_vertex(const DecideArgs& a, uint32_t i, long long m2, uint32_t gi,
                                             uint32_t* dyn, BlockScratch& sc, MoveSums& sums) {
  const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
  constexpr uint32_t nthr = kThreads;  // compile-time strides
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
    for (uint32_t s = threadIdx.x; s < slots; s += nthr) {
      keys[s] = kEmpty;
      vals[s] = 0;
    }
    if (threadIdx.x == 0) {
      sc.hd = 0;
      sc.ncand = 0;
      sc.ok = 1;
    }
    __syncthreads();
    // a table of >= 2 * deg slots cannot overflow: probe it to the end;
    // a smaller shared table (bin 3) gives up early and falls back
    const uint32_t limit = (global || slots >= 2 * dg) ? slots : 64;
    bool ok = scan_row<8>(a, i, o, dg, wib * 32, nthr, keys, vals, mask, limit);
    if (!ok) sc.ok = 0;
    __syncthreads();
    const bool done = sc.ok;
    __syncthreads();  // everyone has read sc.ok before the retry resets it
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
  {
    const unsigned long long hd = table_argmax<4>(a, keys, vals, slots, threadIdx.x, nthr, d, m2, Ki,
                                                   have, best, bc, ncand);
    if (hd) sc.hd = hd;  // exactly one slot holds d
  }
  for (int x = 16; x; x >>= 1) ncand += __shfl_xor_sync(0xFFFFFFFFu, ncand, x);
  if (lane == 0 && ncand) atomicAdd(&sc.ncand, ncand);
  block_argmax(have, best, bc);
  if (threadIdx.x == 0) {
    i128 gain = 0;
    const bool mv = decide_move(a, m2, i, d, Ki, have, best, bc, sc.hd, &gain);
    sums.bytes += 24 + 12ull * dg + 12ull * sc.ncand;
    sc.last = mv;
    if (mv) {
      record_move(a, i, bc, d, gain, gi, sums);
      sums.bytes += 16 + 4ull * dg;
      if (dg > kMarkInline) a.bigmv[atomicAdd(a.nbig, 1u)] = i;
    }
  }
  __syncthreads();
  if (sc.last && dg <= kMarkInline) {
    for (uint32_t k0 = wib * 32; k0 < dg; k0 += nthr) {
      uint32_t k = k0 + lane;
      uint2 arc = k < dg ? a.g.arcs[o + k] : make_uint2(i, 0u);
      mark_next(a, arc.x, k < dg && arc.x != i && arc.y != 0);
    }
  }
  __syncthreads();
}

// Bin 2 (and bin-3 degrees when the tuning sends them here): one block per
// vertex.  Headers are loaded by warp 0 for up to 32 of the block's vertices
// at once.  The shared table (kBlockSlots keys + values) is empty at rest: a
// vertex uses the first power of two >= 2 x degree slots, and the scan that
// scores the occupied slots also clears them.  Two block barriers per
// vertex: after the inserts, and after the per-warp bests; warp 0 then
// decides while the other warps start the next vertex (the per-vertex
// scratch is double-buffered), the batch's movers are recorded together at
// its end, and their neighbours are marked by the commit kernel (the mover
// list it spreads over all blocks).  Vertices of degree above kBinBlock, or
// whose scores need 128 bits, take block_vertex (which may fall back to a
// global table) and the table is emptied after it.
template <int kThreads>
__device__ __noinline__ void block_vertex_slow(const DecideArgs& a, const VHdr& v, uint32_t* dyn, BlockScratch& sc,
                                               MoveSums& sums) {
  block_vertex<kThreads>(a, v.i, v.m2, v.gi, dyn, sc, sums);
}

template <int kThreads>
__global__ void __launch_bounds__(kThreads) k_decide_block(DecideArgs a) {
  extern __shared__ uint32_t dyn[];
  uint32_t* keys = dyn;
  uint32_t* vals = dyn + kBlockSlots;
  __shared__ BlockScratch sc;  // the 128-bit path's
  __shared__ VHdr s_hdr[32];
  __shared__ unsigned long long s_best[2][kMaxBlockWarps];
  __shared__ uint32_t s_bc[2][kMaxBlockWarps];
  __shared__ uint32_t s_hd[2], s_nc[2];
  __shared__ unsigned long long s_gain[32];
  __shared__ uint32_t s_mvc[32];
  __shared__ int s_mv[32];
  constexpr uint32_t nthr = kThreads;
  const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
  for (uint32_t s = threadIdx.x; s < kBlockSlots; s += nthr) {
    keys[s] = kEmpty;
    vals[s] = 0;
  }
  if (threadIdx.x < 2) {
    s_hd[threadIdx.x] = 0;
    s_nc[threadIdx.x] = 0;
  }
  const long long m2_one = *a.m2p;
  const uint32_t cnt = *a.count;
  const uint64_t G = gridDim.x;
  MoveSums sums;
  __syncthreads();
  for (uint64_t t0 = blockIdx.x; t0 < cnt; t0 += 32 * G) {
    if (wib == 0) {
      const uint64_t t = t0 + lane * G;
      VHdr h;
      load_header(a, t, t < cnt, m2_one, sums, h);
      s_hdr[lane] = h;
      s_mv[lane] = 0;
    }
    __syncthreads();
    const uint64_t left = (uint64_t(cnt) - t0 + G - 1) / G;
    const uint32_t nv = uint32_t(left < 32 ? left : 32);
    uint32_t p = 0;  // scratch buffer of the current vertex
    for (uint32_t k = 0; k < nv; ++k) {
      const VHdr v = s_hdr[k];
      if (!v.act) continue;  // block-uniform
      if (v.dg > kBinBlock || !fits64(v.m2, v.Ki)) {
        __syncthreads();  // warp 0 has finished the decisions before (it uses sc)
        block_vertex_slow<kThreads>(a, v, dyn, sc, sums);
        for (uint32_t s = threadIdx.x; s < kBlockSlots; s += nthr) {
          keys[s] = kEmpty;
          vals[s] = 0;
        }
        __syncthreads();
        continue;
      }
      uint32_t slots = 64;
      while (slots < 2 * v.dg) slots <<= 1;
      const uint32_t mask = slots - 1;
      // every arc's weight under its neighbour's community (a table of
      // >= 2 x degree slots cannot overflow)
      const bool ok = scan_row<8>(a, v.i, v.o, v.dg, wib * 32, nthr, keys, vals, mask, slots);
      if (!ok) atomicOr(&a.ctrl->err, kErrInternal);
      __syncthreads();
      // score the occupied slots and clear them; four slots' Sigma loads in flight
      bool have = false;
      unsigned long long best = 0;
      uint32_t bc = 0, nc = 0;
      for (uint32_t s0 = threadIdx.x; s0 < slots; s0 += nthr * 4) {
        uint32_t c[4], w[4], sg[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const uint32_t sl = s0 + u * nthr;
          c[u] = sl < slots ? keys[sl] : kEmpty;
          w[u] = c[u] != kEmpty ? vals[sl] : 0u;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) sg[u] = (c[u] != kEmpty && c[u] != v.d) ? sigma32(a.Sigma, c[u]) : 0u;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (c[u] == kEmpty) continue;
          const uint32_t sl = s0 + u * nthr;
          keys[sl] = kEmpty;
          vals[sl] = 0;
          if (c[u] == v.d) {
            s_hd[p] = w[u];  // exactly one slot holds d
            continue;
          }
          ++nc;
          const unsigned long long s = score64(v.m2, w[u], v.Ki, sg[u]);
          if (!have || s > best || (s == best && c[u] < bc)) {
            have = true;
            best = s;
            bc = c[u];
          }
        }
      }
      nc = __reduce_add_sync(0xFFFFFFFFu, nc);
      if (lane == 0 && nc) atomicAdd(&s_nc[p], nc);
      warp_best64(have, best, bc);
      if (lane == 0) {
        s_best[p][wib] = have ? best : 0ull;
        s_bc[p][wib] = bc;
      }
      __syncthreads();
      if (wib == 0) {  // the other warps go on to the next vertex
        have = lane < nthr / 32 && s_bc[p][lane] != kEmpty;
        best = have ? s_best[p][lane] : 0ull;
        bc = have ? s_bc[p][lane] : kEmpty;
        warp_best64(have, best, bc);
        if (lane == 0) {
          i128 gain = 0;
          const bool mv = decide64(a, v, have, best, bc, s_hd[p], &gain);
          sums.bytes += 24 + 12ull * v.dg + 12ull * s_nc[p] + (mv ? 16 + 4ull * v.dg : 0ull);
          s_mv[k] = mv;
          s_mvc[k] = bc;
          s_gain[k] = (unsigned long long)gain;  // a gain is positive and below 2^64
          s_hd[p] = 0;  // ready for the vertex after next
          s_nc[p] = 0;
        }
      }
      p ^= 1;
    }
    __syncthreads();  // every decision of the batch is made
    if (wib == 0) {  // the batch's movers: one slot reservation, then the mover list for marking
      const bool mv = lane < nv && s_mv[lane];
      const VHdr& v = s_hdr[lane];
      record_moves_warp(a, mv, v.i, s_mvc[lane], v.d, (i128)s_gain[lane], v.gi, sums);
      const unsigned m = __ballot_sync(0xFFFFFFFFu, mv);
      if (m) {
        uint32_t base = 0;
        if (lane == uint32_t(__ffs(m) - 1)) base = atomicAdd(a.nbig, uint32_t(__popc(m)));
        base = __shfl_sync(0xFFFFFFFFu, base, __ffs(m) - 1);
        if (mv) a.bigmv[base + __popc(m & ((1u << lane) - 1u))] = v.i;  // neighbours marked by k_commit
      }
    }
    __syncthreads();  // s_hdr and s_mv are rewritten by the next round
  }
  flush_sums_all(a, sums);
}

// ---------------------------------------------------------------------------
// Bin 3 (the largest degrees): three kernels, every step parallel and
// proportional to the vertex's arcs or its distinct neighbour communities.
//   k_giant_prefix  at the start of an iteration, for every sub-step class
//                   (one block each), lays out per listed vertex its chunks
//                   of kGiantChunk arcs, a global open-addressing table of a
//                   power of two >= 2 x degree slots (empty at rest) and a
//                   list of the table's occupied slots (capacity = degree);
//   k_giant_accum   one block per chunk: the chunk's arcs are aggregated by
//                   community in shared memory, then every distinct (community,
//                   weight) is added into the vertex's table; a new key's slot
//                   is appended to the vertex's occupied list;
//   k_giant_decide  one block per kGiantPart occupied slots of a vertex: those
//                   entries are read and cleared, the part's best candidate is
//                   kept (and the weight to the own community, when met); the
//                   vertex's last part block reduces the parts and decides.
// ---------------------------------------------------------------------------
constexpr uint32_t kGiantChunk = 1024;             // short per-block work: latency, not bandwidth, bounds it
constexpr uint32_t kGiantSlots = 2 * kGiantChunk;  // shared chunk table: 2048 keys + values = 16 KB
constexpr int kAccumThreads = 128;
constexpr uint32_t kGiantPart = 2048;               // occupied slots per decide block
constexpr int kGiantThreads = 256;
constexpr uint32_t kGiantListSmem = 2048;          // chunk prefix cached in shared memory

struct GiantRes {
  unsigned long long lo, hi;  // best score of the part
  uint32_t c;
  uint32_t have;
};

struct GiantDecide {
  unsigned long long* toff;   // per list position: first slot of its table
  unsigned long long* loff;   // ... first entry of its occupied-slot list
  uint32_t* cpre;             // exclusive prefix of chunk counts (+ total)
  uint32_t* ndist;            // occupied slots of its table (zeroed by k_giant_prefix)
  uint32_t* done;             // part blocks finished (zero at rest)
  unsigned long long* hd;     // weight to the own community (zero at rest)
  GiantRes* res;              // per part
  uint32_t* tkeys;            // tables (kEmpty at rest)
  uint32_t* tvals;            // (0 at rest)
  uint2* tlist;               // occupied-slot lists: (slot, community) per entry
  unsigned int* nitems;       // chunk total
  unsigned int* nbignd;       // vertices left to the part blocks (counted)
};

__device__ __forceinline__ uint32_t giant_deg(const DecideArgs& a, uint32_t t) {
  const uint32_t v = a.list[t];
  uint32_t d = a.g.deg[v];
  if (d && a.ngraphs && a.gdone[graph_of(a.goff, a.ngraphs, v)]) d = 0;  // finished graph: skipped
  return d;
}

// Table of a vertex of degree d: a power of two >= 2d (at least 64 slots).
__device__ __forceinline__ uint64_t giant_table_slots(uint32_t d) {
  if (!d) return 0;
  uint64_t p = 64;
  while (p < 2 * uint64_t(d)) p <<= 1;
  return p;
}

// One block: exclusive prefixes over the bin-3 list of chunks, table slots
// and list capacities.
__device__ __forceinline__ void giant_prefix_body(const DecideArgs& a, const GiantDecide& gd) {
  __shared__ unsigned long long s_t[32], s_l[32];
  __shared__ uint32_t s_c[32];
  __shared__ unsigned long long s_tbase, s_lbase;
  __shared__ uint32_t s_cbase;
  const uint32_t cnt = *a.count;
  const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    s_tbase = s_lbase = 0;
    s_cbase = 0;
  }
  __syncthreads();
  for (uint32_t t0 = 0; t0 < cnt; t0 += blockDim.x) {
    const uint32_t t = t0 + threadIdx.x;
    const uint32_t d = t < cnt ? giant_deg(a, t) : 0u;
    const uint32_t ch = (d + kGiantChunk - 1) / kGiantChunk;
    const unsigned long long ts = giant_table_slots(d);
    unsigned long long xt = ts, xl = d;
    uint32_t xc = ch;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long yt = __shfl_up_sync(0xFFFFFFFFu, xt, o);
      unsigned long long yl = __shfl_up_sync(0xFFFFFFFFu, xl, o);
      uint32_t yc = __shfl_up_sync(0xFFFFFFFFu, xc, o);
      if (lane >= (uint32_t)o) {
        xt += yt;
        xl += yl;
        xc += yc;
      }
    }
    if (lane == 31) {
      s_t[w] = xt;
      s_l[w] = xl;
      s_c[w] = xc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long rt = s_tbase, rl = s_lbase;
      uint32_t rc = s_cbase;
      for (uint32_t k = 0; k < blockDim.x / 32; ++k) {
        const unsigned long long tt = s_t[k], tl = s_l[k];
        const uint32_t tc = s_c[k];
        s_t[k] = rt;
        s_l[k] = rl;
        s_c[k] = rc;
        rt += tt;
        rl += tl;
        rc += tc;
      }
      s_tbase = rt;
      s_lbase = rl;
      s_cbase = rc;
    }
    __syncthreads();
    if (t < cnt) {
      gd.toff[t] = s_t[w] + xt - ts;
      gd.loff[t] = s_l[w] + xl - d;
      gd.cpre[t] = s_c[w] + xc - ch;
      gd.ndist[t] = 0;  // counted by k_giant_accum, read by every k_giant_decide block
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    gd.cpre[cnt] = s_cbase;
    *gd.nitems = s_cbase;
  }
}

// Class s's region of the bin-3 arrays: every sub-step class has its own
// layout (at s * gstride), so all of an iteration's layouts are made at once.
__host__ __device__ __forceinline__ GiantDecide giant_class(GiantDecide gd, uint32_t s, uint64_t gstride,
                                                          Ctrl* ctrl) {
  const uint64_t o = uint64_t(s) * gstride;
  gd.toff += o;
  gd.loff += o;
  gd.cpre += o;
  gd.ndist += o;
  gd.done += o;
  gd.hd += o;
  gd.nitems = &ctrl->it_items[s];
  return gd;
}

// The bin-3 layouts of every sub-step class (block s: class s), at the start
// of an iteration, when all classes' lists are final; each sub-step's chain
// of largest-degree kernels then starts with its chunks.
__global__ void __launch_bounds__(1024) k_giant_prefix(DecideArgs a, GiantDecide gd, uint64_t gstride,
                                                       const uint32_t* lists, int cur) {
  pdl_wait_only();
  const uint32_t s = blockIdx.x;
  a.list = lists + a.seg.off[s * kBins + 3];
  a.count = &a.ctrl->count[cur][s][3];
  giant_prefix_body(a, giant_class(gd, s, gstride, a.ctrl));
}

// Entries [e0, e1) of vertex t's occupied list: read and clear them, keep the
// best candidate of this thread (and the weight to d, in hd[t]); returns the
// number of candidates this thread saw.  Four entries' loads are in flight
// at a time (slot, then key and weight, then Sigma).
template <int U>
__device__ __forceinline__ uint32_t giant_scan_entries(const DecideArgs& a, const GiantDecide& gd, uint32_t t,
                                                       uint32_t e0, uint32_t e1, uint32_t d, long long m2,
                                                       long long Ki, bool& have, i128& best, uint32_t& bc) {
  uint32_t* gk = gd.tkeys + gd.toff[t];
  uint32_t* gv = gd.tvals + gd.toff[t];
  const uint2* gl = gd.tlist + gd.loff[t];
  uint32_t ncand = 0;
  for (uint32_t b = e0 + threadIdx.x; b < e1; b += blockDim.x * U) {
    uint2 en[U];  // (slot, community): the weight and Sigma loads go out together
    uint32_t h[U], sg[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t e = b + u * blockDim.x;
      en[u] = e < e1 ? __ldcg(gl + e) : make_uint2(kEmpty, kEmpty);  // written by other blocks of this kernel
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      h[u] = en[u].x != kEmpty ? __ldcg(gv + en[u].x) : 0u;
      sg[u] = (en[u].x != kEmpty && en[u].y != d) ? sigma32(a.Sigma, en[u].y) : 0u;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (en[u].x == kEmpty) continue;
      gk[en[u].x] = kEmpty;
      gv[en[u].x] = 0;
      if (en[u].y == d) {
        gd.hd[t] = h[u];  // exactly one entry of the table holds d
        continue;
      }
      ++ncand;
      const i128 sc = gain_num(m2, h[u], Ki, sg[u]);
      if (!have || sc > best || (sc == best && en[u].y < bc)) {
        have = true;
        best = sc;
        bc = en[u].y;
      }
    }
  }
  return ncand;
}

constexpr uint32_t kSmallDecide = 4096;  // occupied slots the last chunk block decides alone

// One chunk (arcs [chunk * kGiantChunk, +kGiantChunk)) of list position t
// by the whole block: aggregated in the shared table (keys, vals:
// kGiantSlots each), its distinct communities compacted (ek, ev: kGiantChunk
// each) and added into the vertex's global table; the vertex's last chunk
// block decides it when the table holds at most kSmallDecide communities.
// `nch` is the vertex's chunk count.  Every thread of the block calls it.
__device__ __forceinline__ void giant_chunk(const DecideArgs& a, const GiantDecide& gd, uint32_t t,
                                            uint32_t chunk, uint32_t nch, long long m2_one, uint32_t* keys,
                                            uint32_t* vals, uint32_t* ek, uint32_t* ev, BlockScratch& sc,
                                            MoveSums& sums) {
  const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5, nthr = blockDim.x;
  const uint32_t i = a.list[t];
  if (chunk == 0 && threadIdx.x == 0) {
    if (a.ever && bit_set(a.ever, i)) ++sums.ever;
    ++sums.processed;
  }
  if (a.rbits && !bit_test(a.rbits, i)) return;  // processed, not in the affected range
  const unsigned long long o = a.g.off[i];
  const uint32_t dg = a.g.deg[i];
  const uint32_t k0 = chunk * kGiantChunk;
  const uint32_t k1 = min(dg, k0 + kGiantChunk);
  for (uint32_t s = threadIdx.x; s < kGiantSlots; s += nthr) {
    keys[s] = kEmpty;
    vals[s] = 0;
  }
  if (threadIdx.x == 0) sc.ne = 0;
  __syncthreads();
  // a table of 2x the chunk's arcs cannot overflow
  scan_row<8>(a, i, o, k1, k0 + wib * 32, nthr, keys, vals, kGiantSlots - 1, kGiantSlots);
  __syncthreads();
  // the chunk's distinct communities: compacted in shared memory, then
  // added into the vertex's global table, four per thread in flight; new
  // keys' slots go onto its occupied list (one counter update per warp)
  for (uint32_t s0 = wib * 32; s0 < kGiantSlots; s0 += nthr) {
    const uint32_t c = keys[s0 + lane];
    const unsigned m = __ballot_sync(0xFFFFFFFFu, c != kEmpty);
    if (!m) continue;
    uint32_t base = 0;
    if (lane == uint32_t(__ffs(m) - 1)) base = atomicAdd(&sc.ne, uint32_t(__popc(m)));
    base = __shfl_sync(0xFFFFFFFFu, base, __ffs(m) - 1);
    if (c != kEmpty) {
      const uint32_t r = base + __popc(m & ((1u << lane) - 1u));
      ek[r] = c;
      ev[r] = vals[s0 + lane];
    }
  }
  __syncthreads();
  const uint32_t ne = sc.ne;
  const uint32_t tmask = uint32_t(giant_table_slots(dg) - 1);
  uint32_t* gk = gd.tkeys + gd.toff[t];
  uint32_t* gv = gd.tvals + gd.toff[t];
  uint2* gl = gd.tlist + gd.loff[t];
  constexpr int U = 4;
  for (uint32_t b0 = wib * 32 * U; b0 < ne; b0 += nthr * U) {  // warp-uniform
    uint32_t c[U], slot[U], prev[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t e = b0 + u * 32 + lane;
      c[u] = e < ne ? ek[e] : kEmpty;
      slot[u] = hash_move(c[u]) & tmask;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) prev[u] = c[u] != kEmpty ? atomicCAS(&gk[slot[u]], kEmpty, c[u]) : kEmpty;
    unsigned cm[U];  // lanes that created a slot, per group
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t e = b0 + u * 32 + lane;
      bool created = false;
      if (c[u] != kEmpty) {
        // load <= 1/2: the probe ends within the table
        for (uint32_t probe = 0; prev[u] != kEmpty && prev[u] != c[u] && probe < tmask; ++probe) {
          slot[u] = (slot[u] + 1) & tmask;
          prev[u] = atomicCAS(&gk[slot[u]], kEmpty, c[u]);
        }
        if (prev[u] != kEmpty && prev[u] != c[u]) {
          atomicOr(&a.ctrl->err, kErrInternal);  // (cannot happen: the table is never full)
        } else {
          created = prev[u] == kEmpty;
          atomicAdd(&gv[slot[u]], ev[e]);
        }
      }
      cm[u] = __ballot_sync(0xFFFFFFFFu, created);
    }
    // the new keys' slots onto the vertex's occupied list: one reservation for
    // all groups of the warp
    uint32_t total = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) total += __popc(cm[u]);
    if (total) {
      uint32_t base = 0;
      if (lane == 0) base = atomicAdd(&gd.ndist[t], total);
      base = __shfl_sync(0xFFFFFFFFu, base, 0);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if ((cm[u] >> lane) & 1u) gl[base + __popc(cm[u] & ((1u << lane) - 1u))] = make_uint2(slot[u], c[u]);
        base += __popc(cm[u]);
      }
    }
  }
  // the vertex's last chunk block decides it when its table holds few
  // communities; the part blocks take the rest
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) sc.last = atomicAdd(&gd.done[t], 1u) == nch - 1;
  __syncthreads();
  if (sc.last) {
    __threadfence();
    const uint32_t nd = __ldcg(gd.ndist + t);
    if (threadIdx.x == 0) {
      gd.done[t] = 0;  // the part blocks count from 0
      sc.ncand = 0;
    }
    if (nd > kSmallDecide && gd.nbignd && threadIdx.x == 0) atomicAdd(gd.nbignd, 1u);
    if (nd <= kSmallDecide) {
      long long m2 = m2_one;
      uint32_t gi = 0;
      group_active(a, i, &m2, &gi);
      const uint32_t d = a.C[i];
      const long long Ki = a.K[i];
      bool have = false;
      i128 best = 0;
      uint32_t bc = 0;
      uint32_t ncand = giant_scan_entries<4>(a, gd, t, 0, nd, d, m2, Ki, have, best, bc);
      for (int x = 16; x; x >>= 1) ncand += __shfl_xor_sync(0xFFFFFFFFu, ncand, x);
      __threadfence();
      __syncthreads();
      if (lane == 0 && ncand) atomicAdd(&sc.ncand, ncand);
      block_argmax(have, best, bc);
      if (threadIdx.x == 0) {
        const unsigned long long Hd = __ldcg(gd.hd + t);
        gd.hd[t] = 0;
        i128 gain = 0;
        const bool mv = decide_move(a, m2, i, d, Ki, have, best, bc, Hd, &gain);
        sums.bytes += 24 + 12ull * dg + 12ull * sc.ncand;
        if (mv) {
          record_move(a, i, bc, d, gain, gi, sums);
          a.bigmv[atomicAdd(a.nbig, 1u)] = i;  // neighbours marked by the commit
          sums.bytes += 16 + 4ull * dg;
        }
      }
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kAccumThreads, 8) k_giant_accum(DecideArgs a, GiantDecide gd) {
  pdl_wait_only();
  __shared__ uint32_t keys[kGiantSlots];
  __shared__ uint32_t vals[kGiantSlots];
  __shared__ uint32_t s_pre[kGiantListSmem];
  __shared__ uint32_t s_ek[kGiantChunk], s_ev[kGiantChunk];  // distinct communities of a chunk
  __shared__ BlockScratch sc;
  const long long m2_one = *a.m2p;
  const uint32_t cnt = *a.count;
  const uint32_t nitems = *gd.nitems;
  // the chunk prefix, cached in shared memory when it fits
  const uint32_t* cp = gd.cpre;
  if (cnt + 1 <= kGiantListSmem) {
    for (uint32_t k = threadIdx.x; k <= cnt; k += blockDim.x) s_pre[k] = gd.cpre[k];
    __syncthreads();
    cp = s_pre;
  }
  MoveSums sums;
  for (uint32_t item = blockIdx.x; item < nitems; item += gridDim.x) {
    uint32_t lo = 0, hi = cnt;  // list position owning this chunk
    while (hi - lo > 1) {
      uint32_t mid = (lo + hi) >> 1;
      if (cp[mid] <= item) lo = mid;
      else hi = mid;
    }
    giant_chunk(a, gd, lo, item - cp[lo], cp[lo + 1] - cp[lo], m2_one, keys, vals, s_ek, s_ev, sc, sums);
  }
  flush_sums(a, sums, threadIdx.x == 0);
}

// Vertices whose tables hold more than kSmallDecide communities: kGiantPart
// occupied slots per block (blocks of kGiantThreads threads), the vertex's
// last part block reduces.  The block sweeps the list in tiles to number
// the parts.  Every thread of the block calls it.
__device__ __forceinline__ void giant_parts(const DecideArgs& a, const GiantDecide& gd, long long m2_one,
                                            MoveSums& sums) {
  __shared__ uint32_t s_ipre[kGiantThreads + 1];  // part prefix of one tile of the list
  __shared__ uint32_t s_ncand;
  __shared__ int s_last;
  const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
  const uint32_t cnt = *a.count;
  // sweep the list in tiles of blockDim.x positions; part items of a tile
  // are numbered from `ibase` and dealt round-robin over the blocks
  uint32_t ibase = 0;
  for (uint32_t t0 = 0; t0 < cnt; t0 += kGiantThreads) {
    {
      const uint32_t t = t0 + threadIdx.x;
      const uint32_t nd = t < cnt ? gd.ndist[t] : 0u;
      const uint32_t np = nd > kSmallDecide ? (nd + kGiantPart - 1) / kGiantPart : 0u;  // else decided
      uint32_t x = np;
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= (uint32_t)o) x += y;
      }
      __shared__ uint32_t s_w[kGiantThreads / 32];
      if (lane == 31) s_w[wib] = x;
      __syncthreads();
      uint32_t wbase = 0;
      for (uint32_t k = 0; k < wib; ++k) wbase += s_w[k];
      s_ipre[threadIdx.x + 1] = wbase + x;
      if (threadIdx.x == 0) s_ipre[0] = 0;
      __syncthreads();
    }
    const uint32_t tile_items = s_ipre[kGiantThreads];
    const uint32_t first = (blockIdx.x + gridDim.x - ibase % gridDim.x) % gridDim.x;
    for (uint32_t it = first; it < tile_items; it += gridDim.x) {
      uint32_t lo = 0, hi = kGiantThreads;  // tile position owning part item `it`
      while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (s_ipre[mid] <= it) lo = mid;
        else hi = mid;
      }
      const uint32_t t = t0 + lo;
      const uint32_t part = it - s_ipre[lo];
      const uint32_t nparts = s_ipre[lo + 1] - s_ipre[lo];
      const uint32_t ridx = ibase + s_ipre[lo];  // results of this vertex start here
      const uint32_t nd = gd.ndist[t];
      const uint32_t i = a.list[t];
      long long m2 = m2_one;
      uint32_t gi = 0;
      group_active(a, i, &m2, &gi);  // its graph is active: it has entries
      const uint32_t d = a.C[i];
      const long long Ki = a.K[i];
      if (threadIdx.x == 0) s_ncand = 0;
      // 1. this part's entries: best candidate, weight to d; then clear them
      bool have = false;
      i128 best = 0;
      uint32_t bc = 0;
      uint32_t ncand = giant_scan_entries<4>(a, gd, t, part * kGiantPart, min(nd, (part + 1) * kGiantPart), d, m2,
                                          Ki, have, best, bc);
      for (int x = 16; x; x >>= 1) ncand += __shfl_xor_sync(0xFFFFFFFFu, ncand, x);
      __syncthreads();  // s_ncand reset seen
      if (lane == 0 && ncand) atomicAdd(&s_ncand, ncand);
      block_argmax(have, best, bc);
      __threadfence();  // hd[t] (from whichever thread met d) ...
      __syncthreads();  // ... before thread 0's done count
      if (threadIdx.x == 0) {
        GiantRes r;
        r.lo = (unsigned long long)(u128)best;
        r.hi = (unsigned long long)((u128)best >> 64);
        r.c = bc;
        r.have = have ? 1u : 0u;
        gd.res[ridx + part] = r;
        sums.bytes += 12ull * s_ncand;
        __threadfence();
        s_last = atomicAdd(&gd.done[t], 1u) == nparts - 1;
      }
      __syncthreads();
      if (s_last) {
        // 2. last part block of the vertex: reduce the parts and decide
        __threadfence();
        have = false;
        best = 0;
        bc = 0;
        for (uint32_t k = threadIdx.x; k < nparts; k += kGiantThreads) {
          const GiantRes* src = gd.res + ridx + k;
          const unsigned long long rlo = __ldcg(&src->lo), rhi = __ldcg(&src->hi);
          const uint32_t rc = __ldcg(&src->c), rh = __ldcg(&src->have);
          const i128 sc = (i128)(((u128)rhi << 64) | (u128)rlo);
          if (rh && (!have || sc > best || (sc == best && rc < bc))) {
            have = true;
            best = sc;
            bc = rc;
          }
        }
        block_argmax(have, best, bc);
        if (threadIdx.x == 0) {
          const unsigned long long Hd = __ldcg(gd.hd + t);
          gd.hd[t] = 0;  // zero at rest for the next use of this list position
          gd.done[t] = 0;
          const uint32_t dg = a.g.deg[i];
          i128 gain = 0;
          const bool mv = decide_move(a, m2, i, d, Ki, have, best, bc, Hd, &gain);
          sums.bytes += 24 + 12ull * dg;
          if (mv) {
            record_move(a, i, bc, d, gain, gi, sums);
            a.bigmv[atomicAdd(a.nbig, 1u)] = i;  // neighbours marked by k_commit
            sums.bytes += 16 + 4ull * dg;
          }
        }
      }
      __syncthreads();
    }
    ibase += tile_items;
    __syncthreads();  // s_ipre is rewritten for the next tile
  }
}

__global__ void __launch_bounds__(kGiantThreads) k_giant_decide(DecideArgs a, GiantDecide gd) {
  pdl_wait_only();
  MoveSums sums;
  giant_parts(a, gd, *a.m2p, sums);
  flush_sums(a, sums, threadIdx.x == 0);
}

constexpr int kCommitThreads = 256;

// Apply the moves of one sub-step, then mark the next frontier around the
// listed high-degree movers: their arcs in kMarkChunk pieces spread over the
// blocks.  The list is swept in tiles of one block's threads: a block-wide
// prefix numbers the pieces of a tile, which are dealt round-robin over the
// blocks, so a long list (the first iterations of a static run) costs every
// block one parallel pass per tile instead of one dependent walk per mover.
// Blocks of kCommitThreads threads.
__device__ __forceinline__ void commit_body(const DecideArgs& a, uint32_t m, uint32_t count) {
  if (blockIdx.x == 0 && threadIdx.x == 0 && m) atomicAdd(&a.ctrl->moved, (unsigned long long)m);
  uint32_t* C = const_cast<uint32_t*>(a.C);
  long long* Sigma = const_cast<long long*>(a.Sigma);
  int* size = const_cast<int*>(a.size);
  // warp-uniform loop; movers of one warp joining (or leaving) the same
  // community are summed first, so a popular community takes one update
  // per warp instead of one per mover
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t t0 = blockIdx.x * uint64_t(blockDim.x) + (threadIdx.x & ~31u); t0 < m; t0 += stride) {
    const uint64_t t = t0 + (threadIdx.x & 31u);
    const bool ok = t < m;
    const uint32_t i = ok ? a.mv_i[t] : 0u;
    const uint32_t c = ok ? a.mv_c[t] : kEmpty, d = ok ? a.mv_d[t] : kEmpty;
    const long long ki = ok ? a.K[i] : 0;
    if (ok) C[i] = c;
    const uint32_t lane = threadIdx.x & 31u;
    for (int side = 0; side < 2; ++side) {
      const uint32_t key = side ? d : c;
      long long sk = 0;
      int cnt = 0;
      bool first = ok;
      // sum over the lanes with the same community (32 shuffles)
      for (int k = 0; k < 32; ++k) {
        const uint32_t kk = __shfl_sync(0xFFFFFFFFu, key, k);
        const long long kv = __shfl_sync(0xFFFFFFFFu, ki, k);
        if (ok && kk == key) {
          sk += kv;
          ++cnt;
          if (uint32_t(k) < lane) first = false;
        }
      }
      if (first) {
        atomicAdd((unsigned long long*)&Sigma[key], (unsigned long long)(side ? -sk : sk));
        atomicAdd(&size[key], side ? -cnt : cnt);
      }
    }
  }
  const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
  __shared__ uint32_t s_pre[kCommitThreads + 1];
  __shared__ uint32_t s_w[kCommitThreads / 32];
  uint64_t ibase = 0;  // pieces of the earlier tiles
  for (uint32_t q0 = 0; q0 < count; q0 += kCommitThreads) {
    const uint32_t q = q0 + threadIdx.x;
    const uint32_t nch = q < count ? (a.g.deg[a.bigmv[q]] + kMarkChunk - 1) / kMarkChunk : 0u;
    uint32_t x = nch;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= uint32_t(o)) x += y;
    }
    if (lane == 31) s_w[wib] = x;
    __syncthreads();
    uint32_t wbase = 0;
    for (uint32_t k = 0; k < wib; ++k) wbase += s_w[k];
    s_pre[threadIdx.x + 1] = wbase + x;
    if (threadIdx.x == 0) s_pre[0] = 0;
    __syncthreads();
    const uint32_t tile_items = s_pre[kCommitThreads];
    // piece `it` of the tile is item ibase + it, handled by block (ibase + it) mod grid
    for (uint32_t it = uint32_t((blockIdx.x + gridDim.x - ibase % gridDim.x) % gridDim.x); it < tile_items;
         it += gridDim.x) {
      uint32_t lo = 0, hi = kCommitThreads;  // tile position owning piece `it`
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (s_pre[mid] <= it) lo = mid;
        else hi = mid;
      }
      const uint32_t i = a.bigmv[q0 + lo];
      const uint32_t c = it - s_pre[lo];
      const uint32_t dg = a.g.deg[i];
      const unsigned long long o = a.g.off[i];
      const uint32_t k1 = min(dg, (c + 1) * kMarkChunk);
      for (uint32_t k0 = c * kMarkChunk + wib * 32; k0 < k1; k0 += kCommitThreads) {
        const uint32_t k = k0 + lane;
        const uint2 arc = k < k1 ? a.g.arcs[o + k] : make_uint2(i, 0u);
        mark_next(a, arc.x, k < k1 && arc.x != i && arc.y != 0);
      }
    }
    ibase += tile_items;
    __syncthreads();  // s_pre and s_w are rewritten by the next tile
  }
}

__global__ void __launch_bounds__(kCommitThreads) k_commit(DecideArgs a) {
  pdl_wait_only();
  // the next sub-step counts into the other pair of counters, last used two
  // sub-steps ago: zeroed here, so no memset separates the sub-steps
  if (blockIdx.x == 0 && threadIdx.x == 0 && a.clear_movers) {
    *a.clear_movers = 0;
    *a.clear_nbig = 0;
  }
  commit_body(a, *a.movers, *a.nbig);
}

int read_ctrl(Handle* h) {
  DFL_CUDA(h, cudaMemcpyAsync(h->hctrl, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
  DFL_CUDA(h, cudaStreamSynchronize(h->stream));
  return DFL_OK;
}

// A control read of local-moving.  The first one after a batch apply that
// was enqueued without a host wait also settles that apply, in the same
// wait; if the batch was not written (an invalid batch, or buffers to grow
// first) the code is returned and local-moving stops -- its iteration ran on
// an empty frontier, since nothing was marked.
int read_move_ctrl(Handle* h, bool* settled) {
  const bool pend = h->papply.active;
  // (the apply's control blocks follow this one: one copy takes both)
  const size_t blocks = pend ? size_t(2 + h->papply.par) : 1;
  DFL_CUDA(h, cudaMemcpyAsync(h->hctrl, h->ctrl, blocks * sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
  DFL_CUDA(h, cudaStreamSynchronize(h->stream));
  *settled = pend;
  return pend ? settle_apply(h) : DFL_OK;
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




// ---------------------------------------------------------------------------
// Persistent iteration kernel: one cooperative launch runs a whole
// local-moving iteration.  Its blocks take work units of a sub-step from a
// shared counter (largest-degree chunks first, then block, warp and
// segment units), meet at grid barriers between deciding and committing,
// and build the next frontier's lists at the end.  It replaces the per
// sub-step launches, stream forks and joins of issue_iteration.
// ---------------------------------------------------------------------------
constexpr int kIterThreads = 256;
constexpr uint32_t kIterPreCache = kGiantListSmem;                   // chunk prefix cached in shared memory
constexpr uint32_t kIterDynWords = 2 * kBlockSlots + kIterPreCache;  // tables + chunk prefix cache
constexpr unsigned long long kBarrierPolls = 1ull << 22;             // x 256 ns: about a second
constexpr unsigned long long kTestBarrierPolls = 1ull << 14;         // a few ms (the timeout test hook)
// vertices per warp in one work unit of bins 1 and 0 (rounds of 1 and of
// 32 / W vertices); larger units save counter updates on big frontiers but
// measured slower on small DF frontiers, where they leave blocks idle
constexpr uint32_t kIterRounds1 = 1;
constexpr uint32_t kIterRounds0 = 1;

struct IterArgs {
  DecideArgs a;            // list/count/movers/nbig are set per bin and sub-step
  GiantDecide gd;          // class 0's arrays; class s at + s * gstride
  uint32_t gstride;
  uint32_t k;
  int cur;
  uint32_t seg_lanes;      // W: lanes per bin-0 vertex
  const uint32_t* lists_cur;
  uint32_t* fbits_cur;     // cleared at the end (the processed frontier)
  uint32_t words;
  // grid barriers: arrivals beyond the grid that complete one (0; 1 makes
  // every barrier unreachable, DFL_FLAG_TEST_UNREACHABLE_BARRIER) and polls
  // before a wait gives up
  uint32_t bar_extra;
  unsigned long long bar_polls;
};

// Grid-wide barrier with a bounded wait: false if it gave up (the error bit
// kErrTimeout is then set and the kernel must return).  Every thread calls it.
__device__ __forceinline__ bool grid_barrier(Ctrl* ctrl, uint32_t extra, unsigned long long max_polls) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* genp = &ctrl->bar_gen;
    const unsigned int gen = *genp;
    __threadfence();
    int ok = 1;
    if (atomicAdd(&ctrl->bar_count, 1u) == gridDim.x - 1 + extra) {
      ctrl->bar_count = 0;
      __threadfence();
      atomicAdd(&ctrl->bar_gen, 1u);
    } else {
      unsigned long long polls = 0;
      while (*genp == gen) {
        if (++polls > max_polls || (*((volatile unsigned int*)&ctrl->err) & kErrTimeout)) {
          ok = 0;
          atomicOr(&ctrl->err, kErrTimeout);
          break;
        }
        __nanosleep(256);
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  __threadfence();  // every thread: later reads see what other blocks wrote before the barrier
  return s_ok;
}

__device__ __forceinline__ DecideArgs bin_args(const IterArgs& ia, uint32_t s, int b) {
  DecideArgs a = ia.a;
  a.list = ia.lists_cur + a.seg.off[s * kBins + b];
  a.count = &a.ctrl->count[ia.cur][s][b];
  a.movers = &a.ctrl->it_movers[s & 1];
  a.nbig = &a.ctrl->it_nbig[s & 1];
  return a;
}

__device__ __forceinline__ GiantDecide class_giant(const IterArgs& ia, uint32_t s) {
  GiantDecide gd = giant_class(ia.gd, s, ia.gstride, ia.a.ctrl);
  gd.nbignd = &ia.a.ctrl->it_bignd[s & 1];
  return gd;
}

// Every lane of the warp calls it: bin-0 vertices of one warp (32 / W of them).
template <int W>
__device__ __forceinline__ void iter_segments(const DecideArgs& a, uint64_t first, uint32_t cnt, long long m2_one,
                                              MoveSums& sums) {
  const uint32_t lane = threadIdx.x & 31u, seg = lane / W, sl = lane % W;
  const uint64_t t = first + seg;
  bool active = t < cnt;
  const uint32_t i = active ? a.list[t] : 0u;
  long long m2 = m2_one;
  uint32_t gi = 0;
  if (active && !group_active(a, i, &m2, &gi)) active = false;
  if (active && sl == 0) {
    if (a.ever && bit_set(a.ever, i)) ++sums.ever;
    ++sums.processed;
  }
  if (active && a.rbits && !bit_test(a.rbits, i)) active = false;
  decide_segment<W>(a, active, i, m2, gi, sums);
}

static_assert(kIterThreads == kGiantThreads && kIterThreads == kCommitThreads,
              "the part blocks and the commit sweep their lists in tiles of one block");
static_assert(kIterDynWords >= 2 * kBlockSlots && 8 * 2 * kWarpSlots <= 2 * kBlockSlots &&
                  2 * kGiantSlots + 2 * kGiantChunk <= 2 * kBlockSlots,
              "the dynamic tables hold every unit kind");

// two blocks per SM: 128 registers a thread (three blocks, at 80 registers,
// spilled and measured slower)
__global__ void __launch_bounds__(kIterThreads, 2) k_iterate(IterArgs ia) {
  extern __shared__ uint32_t dyn[];
  __shared__ BlockScratch sc;
  __shared__ uint32_t s_unit;
  Ctrl* ctrl = ia.a.ctrl;
  const long long m2_one = *ia.a.m2p;
  const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
  uint32_t* pre_cache = dyn + 2 * kBlockSlots;
  MoveSums sums;
  // 1. the largest-degree lists of every class: chunk, table and list layouts
  if (blockIdx.x < ia.k) {
    const DecideArgs a3 = bin_args(ia, blockIdx.x, 3);
    giant_prefix_body(a3, class_giant(ia, blockIdx.x));
  }
  if (!grid_barrier(ctrl, ia.bar_extra, ia.bar_polls)) return;
  for (uint32_t s = 0; s < ia.k; ++s) {
    const uint32_t par = s & 1;
    if (blockIdx.x == 0 && threadIdx.x == 0 && s >= 1) {  // the other parity's counters are idle now
      ctrl->it_movers[par ^ 1] = 0;
      ctrl->it_nbig[par ^ 1] = 0;
      ctrl->it_work[par ^ 1] = 0;
      ctrl->it_bignd[par ^ 1] = 0;
    }
    const DecideArgs a0 = bin_args(ia, s, 0), a1 = bin_args(ia, s, 1), a2 = bin_args(ia, s, 2),
                     a3 = bin_args(ia, s, 3);
    const GiantDecide gd = class_giant(ia, s);
    const uint32_t n0 = *a0.count, n1 = *a1.count, n2 = *a2.count, n3 = *a3.count;
    const uint32_t G = *gd.nitems;
    // chunk prefix of the class, cached when it fits
    const uint32_t* cp = gd.cpre;
    if (n3 + 1 <= kIterPreCache) {
      for (uint32_t q = threadIdx.x; q <= n3; q += blockDim.x) pre_cache[q] = gd.cpre[q];
      __syncthreads();
      cp = pre_cache;
    }
    const uint32_t per_warp0 = 32 / ia.seg_lanes;
    const uint64_t U0 = (uint64_t(n0) + per_warp0 * 8 * kIterRounds0 - 1) / (per_warp0 * 8 * kIterRounds0);
    const uint64_t U1 = (uint64_t(n1) + 8 * kIterRounds1 - 1) / (8 * kIterRounds1);
    const uint64_t total = uint64_t(G) + n2 + U1 + U0;
    // 2. decide: work units from the shared counter
    for (;;) {
      if (threadIdx.x == 0) s_unit = atomicAdd(&ctrl->it_work[par], 1u);
      __syncthreads();
      const uint64_t u = s_unit;
      __syncthreads();
      if (u >= total) break;
      if (u < G) {
        uint32_t lo = 0, hi = n3;  // list position owning chunk u
        while (hi - lo > 1) {
          uint32_t mid = (lo + hi) >> 1;
          if (cp[mid] <= u) lo = mid;
          else hi = mid;
        }
        giant_chunk(a3, gd, lo, uint32_t(u) - cp[lo], cp[lo + 1] - cp[lo], m2_one, dyn, dyn + kGiantSlots,
                    dyn + 2 * kGiantSlots, dyn + 2 * kGiantSlots + kGiantChunk, sc, sums);
      } else if (u < uint64_t(G) + n2) {
        const uint32_t i = a2.list[u - G];
        long long m2 = m2_one;
        uint32_t gi = 0;
        if (!group_active(a2, i, &m2, &gi)) continue;
        if (threadIdx.x == 0) {
          if (a2.ever && bit_set(a2.ever, i)) ++sums.ever;
          ++sums.processed;
        }
        if (a2.rbits && !bit_test(a2.rbits, i)) continue;
        block_vertex<kIterThreads>(a2, i, m2, gi, dyn, sc, sums);
      } else if (u < uint64_t(G) + n2 + U1) {
        // one bin-1 vertex per warp and round, in the warp's own table
        for (uint32_t r = 0; r < kIterRounds1; ++r) {
          const uint64_t t = ((u - G - n2) * kIterRounds1 + r) * 8 + wib;
          if (t >= n1) break;
          const uint32_t i = a1.list[t];
          long long m2 = m2_one;
          uint32_t gi = 0;
          if (!group_active(a1, i, &m2, &gi)) continue;
          if (lane == 0) {
            if (a1.ever && bit_set(a1.ever, i)) ++sums.ever;
            ++sums.processed;
          }
          if (!a1.rbits || bit_test(a1.rbits, i))
            warp_table_vertex(a1, i, m2, gi, dyn + wib * 2 * kWarpSlots, dyn + wib * 2 * kWarpSlots + kWarpSlots,
                              sums);
        }
      } else {
        for (uint32_t r = 0; r < kIterRounds0; ++r) {
          const uint64_t first =
              ((u - G - n2 - U1) * kIterRounds0 + r) * (per_warp0 * 8) + uint64_t(wib) * per_warp0;
          if (first >= n0) break;  // warp-uniform
          switch (ia.seg_lanes) {
            case 4: iter_segments<4>(a0, first, n0, m2_one, sums); break;
            case 8: iter_segments<8>(a0, first, n0, m2_one, sums); break;
            case 16: iter_segments<16>(a0, first, n0, m2_one, sums); break;
            default: iter_segments<32>(a0, first, n0, m2_one, sums); break;
          }
        }
      }
    }
    if (!grid_barrier(ctrl, ia.bar_extra, ia.bar_polls)) return;
    // 3. vertices with many distinct communities: spread over part blocks
    if (*((volatile unsigned int*)&ctrl->it_bignd[par])) {
      giant_parts(a3, gd, m2_one, sums);
      if (!grid_barrier(ctrl, ia.bar_extra, ia.bar_polls)) return;
    }
    // 4. commit the sub-step's moves (and mark around high-degree movers)
    commit_body(a0, *((volatile unsigned int*)a0.movers), *((volatile unsigned int*)a0.nbig));
    if (!grid_barrier(ctrl, ia.bar_extra, ia.bar_polls)) return;
  }
  // 5. the next frontier's lists; clear the processed frontier's bitmap
  lists_bits_body(ia.a.fbits_next, ia.words, ia.a.g.nv, ia.a.g.deg, ia.a.next_lists, ia.a.seg, ctrl,
                  ia.a.next_buf, ia.k);
  for (uint64_t w = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; w < ia.words;
       w += uint64_t(gridDim.x) * blockDim.x)
    ia.fbits_cur[w] = 0;
  flush_sums_all(ia.a, sums);  // every thread holds counts (segment and warp leaders, block leaders)
}

// The start of an iteration: its sums (s_lo .. moved), both pairs of mover
// counters (sub-step s counts into pair s & 1) and the next list buffer's
// lengths are zeroed.
__global__ void k_iter_start(Ctrl* ctrl, int nxt) {
  pdl_wait();
  if (threadIdx.x == 0) {
    ctrl->s_lo = ctrl->s_hi = 0;
    ctrl->processed = ctrl->moved = 0;
  }
  if (threadIdx.x < 2) {
    ctrl->it_movers[threadIdx.x] = 0;
    ctrl->it_nbig[threadIdx.x] = 0;
  }
  unsigned int* c = &ctrl->count[nxt][0][0];
  for (uint32_t q = threadIdx.x; q < sizeof(ctrl->count[0]) / sizeof(unsigned int); q += blockDim.x) c[q] = 0u;
}

// 2m of this local-moving call; with a batch apply enqueued just before (ap),
// the batch's change of 2m if its gate opened
__global__ void k_set_m2(Ctrl* ctrl, long long m2, const Ctrl* ap) {
  pdl_wait();
  ctrl->m2v = m2 + (ap && ap->apply_go ? ap->m2_delta : 0ll);
  ctrl->move_bytes = 0;  // this call's counters
  ctrl->ever_count = 0;
}

// largest grid of the block-per-vertex kernel; each of its blocks owns one
// slice of the global overflow table
constexpr uint32_t kBlockGridMax = 3 * 152;

// Issue one local-moving iteration (all sub-steps) on h->stream.  With
// `counts` (host-known list lengths) empty bins are skipped and grids are
// sized to the work; without (graph capture) every bin is launched with a
// fixed grid and reads its length on the device.
int issue_iteration(Handle* h, DecideArgs a, int cur, const unsigned int (*counts)[kBins],
                    const GiantDecide& gd_base, bool decide_only = false, bool small_hint = false) {
  const uint32_t k = a.k;
  const int nxt = cur ^ 1;
  // reset the iteration's sums, both pairs of mover counters and the next
  // buffer's list lengths (one launch)
  {
    LaunchScope ls(h, DFL_PROF_OTHER);
    launch_pdl(k_iter_start, 1, 64, 0, h->stream, h->ctrl, nxt);
    DFL_TRY(check_launch(h, "iteration start"));
  }
  if (a.ngraphs)
    DFL_CUDA(h, cudaMemsetAsync(a.gS, 0, sizeof(unsigned long long) * 2 * a.ngraphs, h->stream));
  a.fbits_next = h->fbits[nxt];
  a.next_lists = h->lists[nxt];
  a.next_buf = nxt;
  const uint64_t gstride = h->g_items_cap / kMaxSubsteps;
  // The degree bins of a sub-step are independent and run concurrently.  The
  // chain that bounds a sub-step -- the largest-degree chunks, their
  // decisions, the commit -- runs on one stream (the spine, the highest-
  // priority auxiliary stream), so that each of its kernels is a dependent
  // launch of the one before; the spine forks the other bins (bin 0 on the
  // handle's stream, bins 1 and 2 on auxiliary streams) at the start of a
  // sub-step and joins them before the commit.  With DFL_FLAG_SERIAL_BINS
  // everything runs on the handle's stream.
  const bool par = !(h->opt.flags & DFL_FLAG_SERIAL_BINS);
  cudaStream_t spine = par ? h->aux[kBins - 2] : h->stream;
  cudaStream_t bst[kBins] = {h->stream, par ? h->aux[0] : h->stream, par ? h->aux[1] : h->stream, spine};
  if (par) {
    DFL_CUDA(h, cudaEventRecord(h->ev_fork, h->stream));
    DFL_CUDA(h, cudaStreamWaitEvent(spine, h->ev_fork, 0));
  }
  bool any3 = !counts;
  for (uint32_t s = 0; counts && s < k; ++s) any3 |= counts[s][3] != 0;
  if (any3) {  // the largest-degree layouts of all classes, once
    LaunchScope ls(h, DFL_PROF_BIN3, spine);
    launch_pdl(k_giant_prefix, k, 1024, 0, spine, a, gd_base, gstride, h->lists[cur], cur);
    DFL_TRY(check_launch(h, "giant prefix"));
  }
  for (uint32_t s = 0; s < k; ++s) {
    a.movers = &h->ctrl->it_movers[s & 1];
    a.nbig = &h->ctrl->it_nbig[s & 1];
    a.clear_movers = s + 1 < k ? &h->ctrl->it_movers[(s + 1) & 1] : nullptr;
    a.clear_nbig = s + 1 < k ? &h->ctrl->it_nbig[(s + 1) & 1] : nullptr;
    int nb = 0;
    for (int b = 0; b < kBins; ++b) nb += (!counts || counts[s][b]) ? 1 : 0;
    const bool any = nb > 0;
    cudaEvent_t pa = nullptr, pb = nullptr;  // wall time of the decide phase (profiling)
    if (any && (h->opt.flags & (DFL_FLAG_PROFILE | DFL_FLAG_PROFILE_MOVE))) {
      pa = take_event(h);
      pb = take_event(h);
      if (pa) record_timing_event(pa, spine);
    }
    // the fork point is this sub-step's start on the spine, before its own kernels
    bool fork = false;
    for (int b = 0; b < kBins; ++b) fork |= bst[b] != spine && (!counts || counts[s][b]);
    if (fork) DFL_CUDA(h, cudaEventRecord(h->ev_fork, spine));
    bool joined[kBins - 1] = {false, false, false};
    for (int b = kBins - 1; b >= 0; --b) {
      const uint32_t c = counts ? counts[s][b] : 0u;
      if (counts && !c) continue;
      cudaStream_t st = bst[b];
      if (st != spine) {
        DFL_CUDA(h, cudaStreamWaitEvent(st, h->ev_fork, 0));
        joined[b] = true;
      }
      a.list = h->lists[cur] + h->segs.off[s * kBins + b];
      a.count = &h->ctrl->count[cur][s][b];
      LaunchScope ls(h, DFL_PROF_BIN0 + b, st);
      if (b == 0) {
        const uint32_t lim = h->tune.bin_warp;
        const bool small = counts ? c < kSmallList : small_hint;
        if (lim <= 8 && small) {  // W = 4 or 8 lanes per vertex
          const uint32_t segs = lim <= 4 ? 8 : 4;
          const uint32_t grid = counts ? grid_for((uint64_t(c) + segs - 1) / segs * 32, 256, 152 * 64) : 152 * 8;
          if (segs == 8) k_decide_warp<4><<<grid, 256, 0, st>>>(a);
          else k_decide_warp<8><<<grid, 256, 0, st>>>(a);
        } else if (lim <= 8) {  // a thread per vertex, its arcs in registers
          const uint32_t grid = counts ? grid_for(c, 256, 152 * 16) : 152 * 4;
          if (lim <= 4) k_decide_thread<4><<<grid, 256, 0, st>>>(a);
          else k_decide_thread<8><<<grid, 256, 0, st>>>(a);
        } else {  // W = 16 or 32 lanes per vertex
          const uint32_t segs = lim <= 16 ? 2 : 1;
          const uint32_t grid = counts ? grid_for((uint64_t(c) + segs - 1) / segs * 32, 256, 152 * 64) : 152 * 8;
          if (segs == 2) k_decide_warp<16><<<grid, 256, 0, st>>>(a);
          else k_decide_warp<32><<<grid, 256, 0, st>>>(a);
        }
      } else if (b == 1) {
        // a warp per vertex, headers in batches of up to 32 (fewer when the list is short)
        k_decide_warp_hash<<<counts ? grid_for(uint64_t(c) * 32, 256, 152 * 6) : 152 * 3, 256, 0, st>>>(a);
      } else if (b == 2) {
        const size_t smem = sizeof(uint32_t) * 2 * kBlockSlots;
        const uint32_t bt = h->tune.block_threads;
        const uint32_t per_sm = bt == 512 ? 2 : 3;  // 64 KB table each; grid <= kBlockGridMax
        const uint32_t grid = counts ? grid_for(c, 1, 152 * per_sm) : 152 * per_sm;
        if (bt == 128) k_decide_block<128><<<grid, 128, smem, st>>>(a);
        else if (bt == 512) k_decide_block<512><<<grid, 512, smem, st>>>(a);
        else k_decide_block<256><<<grid, 256, smem, st>>>(a);
      } else {
        const GiantDecide gd = giant_class(gd_base, s, gstride, h->ctrl);  // laid out above
        launch_pdl(k_giant_accum, 152 * 8, kAccumThreads, 0, st, a, gd);
        DFL_TRY(check_launch(h, "giant accumulate"));
        launch_pdl(k_giant_decide, 152 * 4, kGiantThreads, 0, st, a, gd);
      }
      DFL_TRY(check_launch(h, "decide"));
    }
    for (int b = 0; b < kBins - 1; ++b)
      if (joined[b]) {
        DFL_CUDA(h, cudaEventRecord(h->ev_join[b], bst[b]));
        DFL_CUDA(h, cudaStreamWaitEvent(spine, h->ev_join[b], 0));
      }
    if (pa && pb) {
      record_timing_event(pb, spine);
      h->ev_pending.push_back(Handle::Ev{pa, pb, DFL_PROF_MOVE});
      h->prof.launches[DFL_PROF_MOVE]++;
    } else {
      if (pa) h->ev_free.push_back(pa);
      if (pb) h->ev_free.push_back(pb);
    }
    if (any && decide_only) {
      DFL_CUDA(h, cudaMemsetAsync(&h->ctrl->it_movers[0], 0, 4 * sizeof(unsigned int), spine));
    } else if (any) {
      LaunchScope ls(h, DFL_PROF_COMMIT, spine);
      launch_pdl(k_commit, 152 * 2, kCommitThreads, 0, spine, a);
      DFL_TRY(check_launch(h, "commit"));
    } else if (a.clear_movers) {  // no commit ran: zero the next sub-step's counters here
      DFL_CUDA(h, cudaMemsetAsync(a.clear_movers, 0, sizeof(unsigned int), spine));
      DFL_CUDA(h, cudaMemsetAsync(a.clear_nbig, 0, sizeof(unsigned int), spine));
    }
  }
  // the next frontier's lists, from its bitmap
  {
    const uint32_t words = (a.g.nv + 31) / 32;
    LaunchScope ls(h, DFL_PROF_MARK, spine);
    // (the processed frontier's bitmap, cleared alongside, becomes the next-next target)
    launch_pdl(k_lists_bits, grid_for(words, 256, 152 * 8), 256, 0, spine, a.fbits_next, words, a.g.nv,
               a.g.deg, a.next_lists, a.seg, h->ctrl, nxt, k, h->fbits[cur], h->words);
    DFL_TRY(check_launch(h, "next frontier lists"));
  }
  if (par) {  // the handle's stream continues after the spine
    DFL_CUDA(h, cudaEventRecord(h->ev_fork, spine));
    DFL_CUDA(h, cudaStreamWaitEvent(h->stream, h->ev_fork, 0));
  }
  return DFL_OK;
}

// Blocks of the cooperative iteration kernel that are resident at once
// (0: it cannot run); queried once per process.
uint32_t persistent_grid() {
  static std::once_flag once;
  static uint32_t grid = 0;
  std::call_once(once, [] {
    int dev = 0, sms = 0, per_sm = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return;
    if (cudaFuncSetAttribute(k_iterate, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(sizeof(uint32_t) * kIterDynWords)) != cudaSuccess)
      return;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_iterate, kIterThreads,
                                                      sizeof(uint32_t) * kIterDynWords) != cudaSuccess)
      return;
    uint64_t g = uint64_t(sms) * uint64_t(per_sm);
    // each block may own a slice of the block kernel's overflow table
    grid = uint32_t(g < kBlockGridMax ? g : kBlockGridMax);
  });
  return grid;
}

// One local-moving iteration as a single cooperative launch of k_iterate.
int issue_persistent(Handle* h, const DecideArgs& a_base, int cur, const GiantDecide& gd, uint32_t grid) {
  const int nxt = cur ^ 1;
  DFL_CUDA(h, cudaMemsetAsync(h->ctrl, 0, offsetof(Ctrl, move_bytes), h->stream));
  DFL_CUDA(h, cudaMemsetAsync(&h->ctrl->movers, 0, 2 * sizeof(unsigned int), h->stream));
  DFL_CUDA(h, cudaMemsetAsync(&h->ctrl->it_movers[0], 0,
                              offsetof(Ctrl, bar_gen) + sizeof(unsigned int) - offsetof(Ctrl, it_movers),
                              h->stream));
  DFL_CUDA(h, cudaMemsetAsync(&h->ctrl->count[nxt][0][0], 0, sizeof(h->ctrl->count[0]), h->stream));
  if (a_base.ngraphs)
    DFL_CUDA(h, cudaMemsetAsync(a_base.gS, 0, sizeof(unsigned long long) * 2 * a_base.ngraphs, h->stream));
  IterArgs ia;
  std::memset(&ia, 0, sizeof(ia));
  ia.a = a_base;
  ia.a.fbits_next = h->fbits[nxt];
  ia.a.next_lists = h->lists[nxt];
  ia.a.next_buf = nxt;
  ia.gd = gd;
  ia.gstride = uint32_t(h->g_items_cap / kMaxSubsteps);
  ia.k = a_base.k;
  ia.cur = cur;
  const uint32_t lim = h->tune.bin_warp;
  ia.seg_lanes = lim <= 4 ? 4 : lim <= 8 ? 8 : lim <= 16 ? 16 : 32;
  ia.lists_cur = h->lists[cur];
  ia.fbits_cur = h->fbits[cur];
  ia.words = h->words;
  const bool test_timeout = (h->opt.flags & DFL_FLAG_TEST_UNREACHABLE_BARRIER) != 0;
  ia.bar_extra = test_timeout ? 1u : 0u;
  ia.bar_polls = test_timeout ? kTestBarrierPolls : kBarrierPolls;
  void* args[] = {&ia};
  {
    LaunchScope ls(h, DFL_PROF_MOVE);
    DFL_CUDA(h, cudaLaunchCooperativeKernel((const void*)k_iterate, dim3(grid), dim3(kIterThreads), args,
                                            sizeof(uint32_t) * kIterDynWords, h->stream));
  }
  return DFL_OK;
}

// Everything an iteration graph bakes in; a different key means re-capture.
struct GraphKey {
  DecideArgs a;
  GiantDecide gd;
  int cur;
  int small;
  uint32_t flags;
  void* stream;
  uint32_t block_threads;
};

// The cached graph for this iteration's key (captured on a miss, evicting
// the least recently used entry of this parity).
int ensure_iteration_graph(Handle* h, const DecideArgs& a, const GiantDecide& gd, int cur, bool small,
                           Handle::IterGraph** out) {
  GraphKey key;
  std::memset(&key, 0, sizeof(key));
  key.a = a;
  key.gd = gd;
  key.cur = cur;
  key.small = small;
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
  int rc = issue_iteration(h, a, cur, nullptr, gd, false, small);
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
  // overflow tables of the block-per-vertex kernel, needed only when its bin
  // takes degrees beyond what its shared table always holds: one slice of
  // gslots keys + gslots values per block, gslots >= 2 * (largest degree it takes)
  const uint32_t blk_max = ma.max_deg < h->tune.bin_block ? ma.max_deg : h->tune.bin_block;
  const bool need_gtable = blk_max > kBinBlock;
  const uint32_t gslots = next_pow2(2ull * (need_gtable ? blk_max : kBinBlock));
  if (need_gtable && uint64_t(kBlockGridMax) * gslots > h->gtable_cap) {
    if (h->gtable) {
      cudaStreamSynchronize(h->stream);
      cudaFree(h->gtable);
      h->gtable = nullptr;
      h->gtable_cap = 0;
    }
    DFL_CUDA(h, dev_malloc(&h->gtable, sizeof(uint2) * uint64_t(kBlockGridMax) * gslots));
    h->gtable_cap = uint64_t(kBlockGridMax) * gslots;
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
      smem_rc = cudaFuncSetAttribute(k_iterate, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(sizeof(uint32_t) * kIterDynWords));

  });
  DFL_CUDA(h, smem_rc);
  // bin-3 buffers, sized by bounds: at most arcs / (bin_block + 1) listed
  // vertices; tables of at most 4 x degree (>= 64) slots each; occupied
  // lists of at most degree entries; at most arcs / kGiantPart + items parts
  {
    uint64_t arcs = live_arcs_bound(h);
    for (int q = 0; q < 2; ++q) arcs = arcs > h->sg[q].arc_cap ? arcs : h->sg[q].arc_cap;
    // (one region per sub-step class: the persistent kernel lays out all
    // classes at the start of an iteration)
    const uint64_t items = (arcs / (uint64_t(h->tune.bin_block) + 1) + 64 + 1) * kMaxSubsteps;
    const bool any = ma.max_deg > h->tune.bin_block;
    const uint64_t tab = any ? 4 * arcs + 64 * items : 0;
    const uint64_t lst = any ? arcs + 64 : 0;
    const uint64_t res = any ? arcs / kGiantPart + items : 0;
    auto regrow = [&](auto** p, uint64_t& cap, uint64_t need, size_t elem, int fill) -> int {
      if (need <= cap) return DFL_OK;
      cudaStreamSynchronize(h->stream);
      cudaFree(*p);
      *p = nullptr;
      cap = 0;
      const uint64_t want = need + need / 4;
      DFL_CUDA(h, dev_malloc(p, elem * want));
      if (fill >= 0) DFL_CUDA(h, cudaMemsetAsync(*p, fill, elem * want, h->stream));
      cap = want;
      return DFL_OK;
    };
    if (items > h->g_items_cap) {
      uint64_t c0 = h->g_items_cap, c1 = c0, c2 = c0, c3 = c0, c4 = c0, c5 = c0;
      DFL_TRY(regrow(&h->g_toff, c0, items, sizeof(unsigned long long), -1));
      DFL_TRY(regrow(&h->g_loff, c1, items, sizeof(unsigned long long), -1));
      DFL_TRY(regrow(&h->g_cpre, c2, items + 1, sizeof(uint32_t), -1));
      DFL_TRY(regrow(&h->g_ndist, c3, items, sizeof(uint32_t), 0));
      DFL_TRY(regrow(&h->g_done, c4, items, sizeof(uint32_t), 0));
      DFL_TRY(regrow(&h->g_hd, c5, items, sizeof(unsigned long long), 0));
      h->g_items_cap = c0 < c2 ? c0 : c2 - 1;
    }
    {
      uint64_t c = h->g_res_cap;
      GiantRes* r = static_cast<GiantRes*>(h->g_res);
      const int rc = regrow(&r, c, res, sizeof(GiantRes), -1);
      h->g_res = r;  // also when the allocation failed: the old buffer is gone
      h->g_res_cap = c;
      DFL_TRY(rc);
    }
    if (tab > h->g_tab_cap) {
      uint64_t c0 = h->g_tab_cap, c1 = c0;
      DFL_TRY(regrow(&h->g_tkeys, c0, tab, sizeof(uint32_t), 0xFF));  // kEmpty
      DFL_TRY(regrow(&h->g_tvals, c1, tab, sizeof(uint32_t), 0));
      h->g_tab_cap = c0;
    }
    DFL_TRY(regrow(&h->g_tlist, h->g_lst_cap, lst, sizeof(uint2), -1));
  }
  {  // movers whose neighbours k_commit marks: at most one per vertex of degree
     // > kMarkInline, or of the block-per-vertex bin (degree > bin_warp_hash)
    uint64_t arcs = pool_top_bound(h);
    for (int q = 0; q < 2; ++q) arcs = arcs > h->sg[q].arc_cap ? arcs : h->sg[q].arc_cap;
    const uint64_t lo = h->tune.bin_warp_hash < kMarkInline ? h->tune.bin_warp_hash : kMarkInline;
    uint64_t need = arcs / (lo + 1) + 64;
    if (need > uint64_t(h->n) + 64) need = uint64_t(h->n) + 64;
    if (need > h->bigmv_cap) {
      cudaStreamSynchronize(h->stream);
      cudaFree(h->bigmv);
      h->bigmv = nullptr;
      h->bigmv_cap = 0;
      DFL_CUDA(h, dev_malloc(&h->bigmv, sizeof(uint32_t) * (need + need / 2)));
      h->bigmv_cap = need + need / 2;
    }
  }
  if (!h->ev_fork) {  // (created last: a failure part-way is completed by the next call)
    // the largest degrees make the longest chains of a sub-step: their
    // stream gets the highest priority, the block-per-vertex bin the next
    int least = 0, greatest = 0;
    DFL_CUDA(h, cudaDeviceGetStreamPriorityRange(&least, &greatest));
    for (int b = 0; b < kBins - 1; ++b) {
      int prio = b == kBins - 2 ? greatest : b == kBins - 3 ? (greatest < least ? greatest + 1 : least) : least;
      if (!h->aux[b]) DFL_CUDA(h, cudaStreamCreateWithPriority(&h->aux[b], cudaStreamNonBlocking, prio));
      if (!h->ev_join[b]) DFL_CUDA(h, cudaEventCreateWithFlags(&h->ev_join[b], cudaEventDisableTiming));
    }
    DFL_CUDA(h, cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
  }
  {
    LaunchScope ls(h, DFL_PROF_OTHER);
    launch_pdl(k_set_m2, 1, 1, 0, h->stream, h->ctrl, ma.m2,
               h->papply.active ? h->actrl + h->papply.par : nullptr);
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
  a.gtable = need_gtable ? h->gtable : nullptr;
  a.gslots = gslots;
  a.bigmv = h->bigmv;
  a.movers = &h->ctrl->movers;
  a.nbig = &h->ctrl->big_movers;
  if (h->ngraphs) {
    a.ngraphs = h->ngraphs;
    a.goff = h->d_goff;
    a.gm2 = h->d_gm2;
    a.gdone = h->d_gdone;
    a.gS = h->d_gS;
  }
  *gdo = GiantDecide{h->g_toff, h->g_loff, h->g_cpre, h->g_ndist, h->g_done, h->g_hd,
                     static_cast<GiantRes*>(h->g_res), h->g_tkeys, h->g_tvals, h->g_tlist, nullptr,
                     nullptr};
  return DFL_OK;
}

}  // namespace

int local_move(Handle* h, const MoveArgs& ma, uint32_t pass, uint32_t* iterations,
               bool record_trace, uint64_t* initial, uint64_t* ever) {
  const uint32_t G = h->ngraphs;
  u128 threshold = tolerance_threshold(h->opt, ma.m2, pass);
  MoveArgs mv = ma;
  bool settled = false;  // a pending batch apply settled by a control read (2m changed)
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
  // the persistent kernel when asked for; else graph replay, which needs
  // stable buffers (the base graph) and a capturable (non-default) stream,
  // unless forbidden, or unless the caller prefers host launches (a small
  // update, a group) and replay was not asked for explicitly; else host
  // launches
  const uint32_t pgrid = (h->opt.flags & DFL_FLAG_PERSISTENT) ? persistent_grid() : 0u;
  const bool use_persistent = pgrid >= kMaxSubsteps;
  const uint32_t fl = h->opt.flags;
  const bool want_graph = !(fl & DFL_FLAG_NO_GRAPH) && ((fl & DFL_FLAG_GRAPH) || !ma.prefer_host);
  const bool use_graph = !use_persistent && want_graph && ma.g.off == h->off && h->stream != nullptr;
  unsigned int cur_count[kMaxSubsteps][kBins];
  unsigned long long skipped = 0;
  bool have_counts = false;
  if (!use_graph && !use_persistent) {
    DFL_TRY(read_move_ctrl(h, &settled));  // list lengths of the initial frontier (buffer 0)
    if (settled && !G) {
      threshold = tolerance_threshold(h->opt, h->m2, pass);
      mv.m2 = h->m2;  // the batch's 2m, for the decide kernels
    }
    if (h->hctrl->err) return set_error(h, DFL_ERR_CUDA, "internal error in frontier marking");
    for (uint32_t s = 0; s < kMaxSubsteps; ++s)
      for (int b = 0; b < kBins; ++b) cur_count[s][b] = h->hctrl->count[0][s][b];
    skipped = h->hctrl->skipped;
    have_counts = true;
  }
  DecideArgs a;
  GiantDecide gd;
  DFL_TRY(prepare_move(h, mv, &a, &gd));
  int cur = 0;
  uint32_t it = 0;
  uint64_t hint = ma.frontier_hint;  // upper bound of this iteration's frontier
  Handle::IterGraph* graph_used[2] = {nullptr, nullptr};
  while (it < h->opt.max_iterations && (!G || nactive)) {
    ++it;
    const int nxt = cur ^ 1;
    if (use_graph) {
      Handle::IterGraph* gp = nullptr;
      DFL_TRY(ensure_iteration_graph(h, a, gd, cur, hint / h->opt.substeps < kSmallList, &gp));
      const Handle::IterGraph& g = *gp;
      graph_used[cur] = gp;
      DFL_CUDA(h, cudaGraphLaunch(g.exec, h->stream));
      h->launches += g.kernels;
      for (int q = 0; q < DFL_PROF_CLASSES; ++q) h->prof.launches[q] += g.class_launches[q];
    } else if (use_persistent) {
      DFL_TRY(issue_persistent(h, a, cur, gd, pgrid));
    } else {
      DFL_TRY(issue_iteration(h, a, cur, cur_count, gd));
    }
    if (G)
      DFL_CUDA(h, cudaMemcpyAsync(h->h_gS, h->d_gS, sizeof(unsigned long long) * 2 * G,
                                  cudaMemcpyDeviceToHost, h->stream));
    DFL_TRY(read_move_ctrl(h, &settled));
    if (settled && !G) threshold = tolerance_threshold(h->opt, h->m2, pass);
    const Ctrl& c = *h->hctrl;
    if (c.err & kErrTimeout) return set_error(h, DFL_ERR_TIMEOUT, "grid barrier of the iteration kernel gave up");
    if (c.err) return set_error(h, DFL_ERR_CUDA, "internal error in local-moving (table overflow)");
    if (use_persistent) {
      if (it == 1) {
        skipped = c.skipped;
        if (initial) {
          *initial = skipped;
          for (uint32_t s = 0; s < kMaxSubsteps; ++s)
            for (int b = 0; b < kBins; ++b) *initial += c.count[0][s][b];
        }
      }
    } else if (use_graph) {
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
    hint = 0;
    for (uint32_t s = 0; s < kMaxSubsteps; ++s)
      for (int b = 0; b < kBins; ++b) hint += c.count[nxt][s][b];
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
