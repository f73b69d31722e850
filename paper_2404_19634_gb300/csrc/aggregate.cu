// Aggregation phase (Alg. 6): collapse each community of G' into one
// super-vertex of G''.
//   1. community vertex counts and total degrees (one pass over vertices),
//   2. exclusive scans: community-vertex CSR offsets, and super-vertex row
//      offsets from the total degree (an over-estimate, so rows have holes),
//   3. community-vertex CSR fill,
//   4. per community, a hash merge of its members' arcs keyed by the
//      neighbour's community, self-loops included (scanCommunities with
//      self = true); distinct keys are written as the super-vertex's row, and
//      its weight K'' = Sigma'' is the row sum (Alg. 4, weight reset).
// Communities are binned by total degree: one warp with a shared-memory
// table (<= 256), one block with a shared-memory table (<= 4096); a larger
// community is split into chunks of members, each chunk aggregated by one
// block in shared memory and merged into the community's global table, which
// is then emitted slot-parallel.  Every arc goes straight into a table with
// a shared-memory (or, for a giant community's overflow, global) atomic.
#include <mutex>
#include <vector>

#include "common.cuh"

namespace dfl {

namespace {

__global__ void k_agg_count(GraphView g, const uint32_t* __restrict__ Cp, uint32_t* __restrict__ cnt,
                            unsigned long long* __restrict__ tdeg) {
  for (uint64_t v = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; v < g.nv;
       v += uint64_t(gridDim.x) * blockDim.x) {
    uint32_t c = Cp[v];
    atomicAdd(&cnt[c], 1u);
    uint32_t d = g.deg[v];
    if (d) atomicAdd(&tdeg[c], (unsigned long long)d);
  }
}

// Round every community's total degree up to an even count (rows then start
// 16-byte aligned), track the maximum, and bin the community.
__global__ void k_agg_bins(uint32_t ncomm, unsigned long long* __restrict__ tdeg, uint32_t* lists,
                           Segs seg, Ctrl* ctrl) {
  uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t c0 = blockIdx.x * uint64_t(blockDim.x); c0 < ncomm; c0 += stride) {
    uint64_t c = c0 + threadIdx.x;
    bool valid = c < ncomm;
    uint32_t key = 0;
    if (valid) {
      unsigned long long t = tdeg[c];
      unsigned long long te = (t + 1) & ~1ull;
      tdeg[c] = te;
      uint32_t tc = t > 0xFFFFFFFFull ? 0xFFFFFFFFu : uint32_t(t);
      key = tc <= kBinWarpHash ? 0u : tc <= kBinBlock ? 1u : 2u;
      if (key == 2) atomicMax(&ctrl->red_u, tc);
    }
    append_vertex(uint32_t(c), valid, key, lists, seg, ctrl, 1);
  }
}

__global__ void k_agg_fill(uint32_t nv, const uint32_t* __restrict__ Cp, const uint32_t* __restrict__ coff,
                           uint32_t* __restrict__ fillc, uint32_t* __restrict__ members) {
  for (uint64_t v = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; v < nv;
       v += uint64_t(gridDim.x) * blockDim.x) {
    uint32_t c = Cp[v];
    members[coff[c] + atomicAdd(&fillc[c], 1u)] = uint32_t(v);
  }
}

struct AggArgs {
  GraphView g;
  const uint32_t* Cp;
  const uint32_t* coff;
  const uint32_t* members;
  const unsigned long long* soff;
  uint32_t* deg_out;
  uint2* arcs_out;
  long long* Knew;
  const uint32_t* list;
  const unsigned int* count;
  uint32_t ncomm;
  Ctrl* ctrl;
  uint2* gtable;
  uint32_t gslots;
  uint2* bigq;              // giant-community members of high degree: (member, giant index)
  unsigned int* nbig;       // their count
};

__device__ __forceinline__ bool agg_add(uint32_t* keys, uint32_t* vals, uint32_t mask, uint32_t c,
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

// Add arcs [0, d) of one vertex (warp-strided, two loads in flight per lane)
// to the table by neighbour community; deleted arcs (weight 0) skipped.
// Entries that do not fit are added to the fallback table if one is given.
__device__ __forceinline__ bool agg_row(const AggArgs& a, unsigned long long o, uint32_t d,
                                        uint32_t* keys, uint32_t* vals, uint32_t mask, uint32_t limit,
                                        uint32_t* fkeys, uint32_t* fvals, uint32_t fmask) {
  const uint32_t lane = threadIdx.x & 31u;
  bool ok = true;
  for (uint32_t k0 = 0; k0 < d; k0 += 64) {
    uint2 arc0 = k0 + lane < d ? a.g.arcs[o + k0 + lane] : make_uint2(0u, 0u);
    uint2 arc1 = k0 + 32 + lane < d ? a.g.arcs[o + k0 + 32 + lane] : make_uint2(0u, 0u);
    uint32_t c0 = arc0.y ? a.Cp[arc0.x] : kEmpty;
    uint32_t c1 = arc1.y ? a.Cp[arc1.x] : kEmpty;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      uint32_t c = u ? c1 : c0;
      uint32_t w = u ? arc1.y : arc0.y;
      if (c != kEmpty && !agg_add(keys, vals, mask, c, w, limit)) {
        if (fkeys) ok &= agg_add(fkeys, fvals, fmask, c, w, fmask + 1);
        else ok = false;
      }
    }
  }
  return ok;
}

constexpr uint32_t kAggWarpSlots = 512;
constexpr int kAggWarps = 8;
constexpr uint32_t kAggBlockSlots = 2 * kBinBlock;  // 8192 keys + values = 64 KB
constexpr uint32_t kChunkMembers = 256;             // members per block of a giant community
constexpr uint32_t kAggBigMember = 512;             // larger member rows go to k_agg_big ...
constexpr uint32_t kAggPiece = 2048;                // ... in pieces of this many arcs
constexpr uint32_t kGiantSlots = 4096;              // shared table of a giant-community block

// Write the table's entries as the row of super-vertex c (ballot order).
__device__ __forceinline__ void emit_warp(const AggArgs& a, uint32_t c, const uint32_t* keys,
                                          const uint32_t* vals, uint32_t slots, uint32_t* maxd) {
  const uint32_t lane = threadIdx.x & 31u;
  const unsigned long long base = a.soff[c];
  uint32_t pos = 0;
  unsigned long long ksum = 0;
  for (uint32_t s0 = 0; s0 < slots; s0 += 32) {
    uint32_t s = s0 + lane;
    uint32_t key = s < slots ? keys[s] : kEmpty;
    bool has = key != kEmpty;
    unsigned m = __ballot_sync(0xFFFFFFFFu, has);
    if (has) {
      uint32_t val = vals[s];
      a.arcs_out[base + pos + __popc(m & ((1u << lane) - 1u))] = make_uint2(key, val);
      ksum += val;
    }
    pos += __popc(m);
  }
  for (int x = 16; x; x >>= 1) ksum += __shfl_xor_sync(0xFFFFFFFFu, ksum, x);
  if (lane == 0) {
    a.deg_out[c] = pos;
    a.Knew[c] = (long long)ksum;
  }
  *maxd = max(*maxd, pos);
}

// Bin 0: one warp per community (total degree <= 256).
__global__ void __launch_bounds__(256) k_agg_warp(AggArgs a) {
  __shared__ uint32_t skeys[kAggWarps][kAggWarpSlots];
  __shared__ uint32_t svals[kAggWarps][kAggWarpSlots];
  const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
  uint32_t* keys = skeys[wib];
  uint32_t* vals = svals[wib];
  const uint32_t cnt = *a.count;
  uint64_t warp = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) >> 5;
  uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  uint32_t maxd = 0;
  for (uint64_t t = warp; t < cnt; t += nwarps) {
    const uint32_t c = a.list[t];
    const unsigned long long td = a.soff[c + 1] - a.soff[c];
    uint32_t slots = 32;
    while (slots < 2 * td && slots < kAggWarpSlots) slots <<= 1;
    for (uint32_t s = lane; s < slots; s += 32) {
      keys[s] = kEmpty;
      vals[s] = 0;
    }
    __syncwarp();
    bool ok = true;
    for (uint32_t m = a.coff[c]; m < a.coff[c + 1]; ++m) {
      uint32_t v = a.members[m];
      ok &= agg_row(a, a.g.off[v], a.g.deg[v], keys, vals, slots - 1, slots, nullptr, nullptr, 0);
    }
    if (!__all_sync(0xFFFFFFFFu, ok) && lane == 0) atomicOr(&a.ctrl->err, kErrInternal);
    __syncwarp();
    emit_warp(a, c, keys, vals, slots, &maxd);
    __syncwarp();
  }
  if (lane == 0 && maxd) atomicMax(&a.ctrl->max_deg, maxd);
}

// Bin 1: one block per community (total degree <= 4096); a warp per member.
__global__ void __launch_bounds__(256) k_agg_block(AggArgs a) {
  extern __shared__ uint32_t dyn[];
  __shared__ unsigned int s_pos;
  __shared__ unsigned long long s_sum;
  __shared__ int s_ok;
  const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint32_t cnt = *a.count;
  unsigned int maxd = 0;
  for (uint64_t t = blockIdx.x; t < cnt; t += gridDim.x) {
    const uint32_t c = a.list[t];
    const unsigned long long td = a.soff[c + 1] - a.soff[c];
    uint32_t slots = 1024;
    while (slots < 2 * td && slots < kAggBlockSlots) slots <<= 1;
    uint32_t* keys = dyn;
    uint32_t* vals = dyn + slots;
    for (uint32_t s = threadIdx.x; s < slots; s += blockDim.x) {
      keys[s] = kEmpty;
      vals[s] = 0;
    }
    if (threadIdx.x == 0) {
      s_pos = 0;
      s_sum = 0;
      s_ok = 1;
    }
    __syncthreads();
    bool ok = true;
    for (uint32_t m = a.coff[c] + wib; m < a.coff[c + 1]; m += nw) {
      uint32_t v = a.members[m];
      ok &= agg_row(a, a.g.off[v], a.g.deg[v], keys, vals, slots - 1, slots, nullptr, nullptr, 0);
    }
    if (!ok) s_ok = 0;
    __syncthreads();
    if (!s_ok && threadIdx.x == 0) atomicOr(&a.ctrl->err, kErrInternal);
    const unsigned long long base = a.soff[c];
    unsigned long long ksum = 0;
    for (uint32_t s0 = wib * 32; s0 < slots; s0 += blockDim.x) {
      uint32_t s = s0 + lane;
      uint32_t key = s < slots ? keys[s] : kEmpty;
      bool has = key != kEmpty;
      unsigned m = __ballot_sync(0xFFFFFFFFu, has);
      uint32_t wbase = 0;
      if (lane == 0 && m) wbase = atomicAdd(&s_pos, __popc(m));
      wbase = __shfl_sync(0xFFFFFFFFu, wbase, 0);
      if (has) {
        uint32_t val = vals[s];
        a.arcs_out[base + wbase + __popc(m & ((1u << lane) - 1u))] = make_uint2(key, val);
        ksum += val;
      }
    }
    for (int x = 16; x; x >>= 1) ksum += __shfl_xor_sync(0xFFFFFFFFu, ksum, x);
    if (lane == 0 && ksum) atomicAdd(&s_sum, ksum);
    __syncthreads();
    if (threadIdx.x == 0) {
      a.deg_out[c] = s_pos;
      a.Knew[c] = (long long)s_sum;
      maxd = max(maxd, s_pos);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && maxd) atomicMax(&a.ctrl->max_deg, maxd);
}

// Giant communities (bin 2).  giant[g] = community, gtab[g] = offset of its
// global table of gsize[g] slots (keys, then values, in uint2 units: the
// table of g occupies gtable[gtab[g] .. gtab[g] + gsize[g]) as keys|values).
struct GiantArgs {
  const uint32_t* giant;
  const unsigned long long* gtab;
  const uint32_t* gsize;
  const uint32_t* chunk0;  // first work item of each giant (exclusive scan of chunk counts)
  uint32_t ngiant;
  uint32_t nitems;         // total (giant, chunk) work items
};

// Block (g, chunk): aggregate members [chunk*256, +256) of giant g in shared
// memory (overflow goes straight to the global table), then merge the shared
// entries into the global table.
__global__ void __launch_bounds__(256) k_agg_giant_accum(AggArgs a, GiantArgs gi) {
  __shared__ uint32_t keys[kGiantSlots];
  __shared__ uint32_t vals[kGiantSlots];
  const uint32_t wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
  bool ok = true;
  for (uint32_t item = blockIdx.x; item < gi.nitems; item += gridDim.x) {
    // giant owning this work item
    uint32_t lo = 0, hi = gi.ngiant;
    while (hi - lo > 1) {
      uint32_t mid = (lo + hi) >> 1;
      if (gi.chunk0[mid] <= item) lo = mid;
      else hi = mid;
    }
    const uint32_t g = lo;
    const uint32_t chunk = item - gi.chunk0[g];
    const uint32_t c = gi.giant[g];
    const uint32_t gs = gi.gsize[g];
    uint32_t* gkeys = reinterpret_cast<uint32_t*>(a.gtable + gi.gtab[g]);
    uint32_t* gvals = gkeys + gs;
    const uint64_t m0 = a.coff[c] + uint64_t(chunk) * kChunkMembers;
    const uint64_t mend = m0 + kChunkMembers;
    const uint32_t m1 = a.coff[c + 1] < mend ? a.coff[c + 1] : uint32_t(mend);
    for (uint32_t s = threadIdx.x; s < kGiantSlots; s += blockDim.x) {
      keys[s] = kEmpty;
      vals[s] = 0;
    }
    __syncthreads();
    for (uint32_t m = uint32_t(m0) + wib; m < m1; m += nw) {
      const uint32_t v = a.members[m];
      const uint32_t dv = a.g.deg[v];
      if (dv > kAggBigMember) {  // spread over many blocks by k_agg_big
        if ((threadIdx.x & 31u) == 0) a.bigq[atomicAdd(a.nbig, 1u)] = make_uint2(v, g);
        continue;
      }
      ok &= agg_row(a, a.g.off[v], dv, keys, vals, kGiantSlots - 1, 32, gkeys, gvals, gs - 1);
    }
    __syncthreads();
    for (uint32_t s = threadIdx.x; s < kGiantSlots; s += blockDim.x) {
      uint32_t k = keys[s];
      if (k != kEmpty) ok &= agg_add(gkeys, gvals, gs - 1, k, vals[s], gs);
    }
    __syncthreads();
  }
  if (!ok) atomicOr(&a.ctrl->err, kErrInternal);
}

// The queued high-degree members of giant communities: their rows in pieces
// of kAggPiece arcs dealt over the blocks; a piece is aggregated in shared
// memory and added to the community's global table.  The queue is swept in
// tiles of one block's threads (a block-wide prefix numbers the pieces of a
// tile, dealt round-robin), so a long queue costs each block one parallel
// pass per tile rather than a dependent walk over every entry.
constexpr int kAggBigThreads = 256;

__global__ void __launch_bounds__(kAggBigThreads) k_agg_big(AggArgs a, GiantArgs gi) {
  __shared__ uint32_t keys[kGiantSlots];
  __shared__ uint32_t vals[kGiantSlots];
  __shared__ uint32_t s_pre[kAggBigThreads + 1];
  __shared__ uint32_t s_w[kAggBigThreads / 32];
  const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
  const uint32_t count = *a.nbig;
  bool ok = true;
  uint64_t ibase = 0;  // pieces of the earlier tiles
  for (uint32_t q0 = 0; q0 < count; q0 += kAggBigThreads) {
    const uint32_t q = q0 + threadIdx.x;
    const uint32_t npc = q < count ? (a.g.deg[a.bigq[q].x] + kAggPiece - 1) / kAggPiece : 0u;
    uint32_t x = npc;
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
    const uint32_t tile_items = s_pre[kAggBigThreads];
    // piece `it` of the tile is item ibase + it, handled by block (ibase + it) mod grid
    for (uint32_t it = uint32_t((blockIdx.x + gridDim.x - ibase % gridDim.x) % gridDim.x); it < tile_items;
         it += gridDim.x) {
      uint32_t lo = 0, hi = kAggBigThreads;  // tile position owning piece `it`
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (s_pre[mid] <= it) lo = mid;
        else hi = mid;
      }
      const uint2 e = a.bigq[q0 + lo];
      const uint32_t v = e.x, g = e.y;
      const uint32_t dv = a.g.deg[v];
      const unsigned long long o = a.g.off[v];
      const uint32_t gs = gi.gsize[g];
      uint32_t* gkeys = reinterpret_cast<uint32_t*>(a.gtable + gi.gtab[g]);
      uint32_t* gvals = gkeys + gs;
      const uint32_t k0 = (it - s_pre[lo]) * kAggPiece, k1 = min(dv, k0 + kAggPiece);
      for (uint32_t s = threadIdx.x; s < kGiantSlots; s += kAggBigThreads) {
        keys[s] = kEmpty;
        vals[s] = 0;
      }
      __syncthreads();
      for (uint32_t k = k0 + threadIdx.x; k < k1; k += kAggBigThreads) {
        const uint2 arc = a.g.arcs[o + k];
        if (!arc.y) continue;  // deleted arc
        const uint32_t c = a.Cp[arc.x];
        if (!agg_add(keys, vals, kGiantSlots - 1, c, arc.y, 32)) ok &= agg_add(gkeys, gvals, gs - 1, c, arc.y, gs);
      }
      __syncthreads();
      for (uint32_t s = threadIdx.x; s < kGiantSlots; s += kAggBigThreads) {
        const uint32_t c = keys[s];
        if (c != kEmpty) ok &= agg_add(gkeys, gvals, gs - 1, c, vals[s], gs);
      }
      __syncthreads();
    }
    ibase += tile_items;
    __syncthreads();  // s_pre and s_w are rewritten by the next tile
  }
  if (!ok) atomicOr(&a.ctrl->err, kErrInternal);
}

// Thread per global-table slot of every giant: emit the super arcs.
__global__ void k_agg_giant_emit(AggArgs a, GiantArgs gi, unsigned long long total) {
  uint32_t maxd = 0;
  for (unsigned long long t = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; t < total;
       t += uint64_t(gridDim.x) * blockDim.x) {
    // giant owning slot t (tables are laid out in giant order)
    uint32_t lo = 0, hi = gi.ngiant;
    while (hi - lo > 1) {
      uint32_t mid = (lo + hi) >> 1;
      if (gi.gtab[mid] <= t) lo = mid;
      else hi = mid;
    }
    const uint32_t g = lo;
    const unsigned long long s = t - gi.gtab[g];
    if (s >= gi.gsize[g]) continue;
    const uint32_t* gkeys = reinterpret_cast<const uint32_t*>(a.gtable + gi.gtab[g]);
    uint32_t key = gkeys[s];
    if (key == kEmpty) continue;
    uint32_t val = gkeys[gi.gsize[g] + s];
    uint32_t c = gi.giant[g];
    uint32_t pos = atomicAdd(&a.deg_out[c], 1u);
    a.arcs_out[a.soff[c] + pos] = make_uint2(key, val);
    atomicAdd((unsigned long long*)&a.Knew[c], (unsigned long long)val);
    maxd = max(maxd, pos + 1);
  }
  if (maxd) atomicMax(&a.ctrl->max_deg, maxd);
}

__global__ void k_giant_init(AggArgs a, GiantArgs gi, unsigned long long total) {
  for (unsigned long long t = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; t < total;
       t += uint64_t(gridDim.x) * blockDim.x) {
    uint32_t* w = reinterpret_cast<uint32_t*>(a.gtable);
    uint32_t lo = 0, hi = gi.ngiant;
    while (hi - lo > 1) {
      uint32_t mid = (lo + hi) >> 1;
      if (gi.gtab[mid] <= t) lo = mid;
      else hi = mid;
    }
    unsigned long long s = t - gi.gtab[lo];
    // keys (first gsize words of the table) empty, values zero
    w[2 * gi.gtab[lo] + s] = kEmpty;
    w[2 * gi.gtab[lo] + gi.gsize[lo] + s] = 0;
  }
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < gi.ngiant; g += gridDim.x * blockDim.x) {
    a.deg_out[gi.giant[g]] = 0;
    a.Knew[gi.giant[g]] = 0;
  }
}

int read_ctrl(Handle* h) {
  DFL_CUDA(h, cudaMemcpyAsync(h->hctrl, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
  DFL_CUDA(h, cudaStreamSynchronize(h->stream));
  return DFL_OK;
}

uint32_t next_pow2(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return uint32_t(p);
}

}  // namespace

// Aggregate g under the renumbered membership Cp (labels in [0, ncomm)) into
// super graph sg[dst]; Knew receives the super-vertex weights.  Returns the
// super graph's maximum degree in h->hctrl->max_deg.
int aggregate(Handle* h, const GraphView& g, const uint32_t* Cp, uint32_t ncomm, int dst,
              long long* Knew) {
  SuperGraph& sg = h->sg[dst];
  if (ncomm + 1 > sg.nv_cap) {
    cudaStreamSynchronize(h->stream);
    cudaFree(sg.off);
    cudaFree(sg.deg);
    sg.off = nullptr;
    sg.deg = nullptr;
    sg.nv_cap = 0;
    DFL_CUDA(h, dev_malloc(&sg.off, sizeof(unsigned long long) * (uint64_t(h->n) + 1)));
    DFL_CUDA(h, dev_malloc(&sg.deg, sizeof(uint32_t) * (uint64_t(h->n) + 1)));
    sg.nv_cap = h->n + 1;
  }
  DFL_CUDA(h, cudaMemsetAsync(h->ctrl, 0, sizeof(Ctrl), h->stream));
  DFL_CUDA(h, cudaMemsetAsync(h->cnt, 0, sizeof(uint32_t) * (uint64_t(ncomm) + 1), h->stream));
  DFL_CUDA(h, cudaMemsetAsync(h->fillc, 0, sizeof(uint32_t) * uint64_t(ncomm), h->stream));
  DFL_CUDA(h, cudaMemsetAsync(sg.off, 0, sizeof(unsigned long long) * (uint64_t(ncomm) + 1),
                              h->stream));
  {
    LaunchScope ls(h, DFL_PROF_AGG);
    k_agg_count<<<grid_for(g.nv, 256), 256, 0, h->stream>>>(g, Cp, h->cnt, sg.off);
    DFL_TRY(check_launch(h, "agg count"));
  }
  Segs seg;
  for (int b = 0; b < kMaxSubsteps * kBins; ++b) {
    seg.off[b] = b < 3 ? uint32_t(b) * h->n : 0;
    seg.cap[b] = b < 3 ? h->n : 0;
  }
  {
    LaunchScope ls(h, DFL_PROF_AGG);
    k_agg_bins<<<grid_for(ncomm, 256), 256, 0, h->stream>>>(ncomm, sg.off, h->lists[1], seg, h->ctrl);
    DFL_TRY(check_launch(h, "agg bins"));
  }
  DFL_TRY(scan_u32(h, h->cnt, h->cnt, ncomm));
  DFL_TRY(scan_u64(h, sg.off, sg.off, ncomm));
  {
    LaunchScope ls(h, DFL_PROF_AGG);
    k_agg_fill<<<grid_for(g.nv, 256), 256, 0, h->stream>>>(g.nv, Cp, h->cnt, h->fillc, h->members);
    DFL_TRY(check_launch(h, "agg fill"));
  }
  unsigned long long total = 0;
  DFL_CUDA(h, cudaMemcpyAsync(&total, sg.off + ncomm, sizeof(total), cudaMemcpyDeviceToHost, h->stream));
  DFL_TRY(read_ctrl(h));
  const Ctrl c = *h->hctrl;
  if (c.err) return set_error(h, DFL_ERR_CUDA, "internal error in aggregation lists");
  if (total > sg.arc_cap) {
    cudaFree(sg.arcs);
    sg.arcs = nullptr;
    sg.arc_cap = 0;
    uint64_t want = total + total / 8 + 1024;
    DFL_CUDA(h, dev_malloc(&sg.arcs, sizeof(uint2) * want));
    sg.arc_cap = want;
  }
  // once per process (handles may be driven from several host threads)
  static std::once_flag smem_once;
  static cudaError_t smem_rc = cudaSuccess;
  std::call_once(smem_once, [] {
    smem_rc = cudaFuncSetAttribute(k_agg_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   int(sizeof(uint32_t) * 2 * kAggBlockSlots));
  });
  DFL_CUDA(h, smem_rc);
  AggArgs a;
  a.g = g;
  a.Cp = Cp;
  a.coff = h->cnt;
  a.members = h->members;
  a.soff = sg.off;
  a.deg_out = sg.deg;
  a.arcs_out = sg.arcs;
  a.Knew = Knew;
  a.ncomm = ncomm;
  a.ctrl = h->ctrl;
  a.gtable = h->gtable;
  a.gslots = 0;
  for (int b = 0; b < 2; ++b) {
    uint32_t nc = c.count[1][0][b];
    if (!nc) continue;
    a.list = h->lists[1] + seg.off[b];
    a.count = &h->ctrl->count[1][0][b];
    LaunchScope ls(h, DFL_PROF_AGG);
    if (b == 0)
      k_agg_warp<<<grid_for(uint64_t(nc) * 32, 256, 152 * 16), 256, 0, h->stream>>>(a);
    else
      k_agg_block<<<grid_for(nc, 1, 152 * 3), 256, sizeof(uint32_t) * 2 * kAggBlockSlots,
                    h->stream>>>(a);
    DFL_TRY(check_launch(h, "aggregate"));
  }
  const uint32_t ngiant = c.count[1][0][2];
  if (ngiant) {
    // giant communities: their ids and sizes on the host to lay out the tables
    std::vector<uint32_t> giant(ngiant);
    DFL_CUDA(h, cudaMemcpy(giant.data(), h->lists[1] + seg.off[2], sizeof(uint32_t) * ngiant,
                           cudaMemcpyDeviceToHost));
    std::vector<unsigned long long> soff(ncomm + 1);
    DFL_CUDA(h, cudaMemcpy(soff.data(), sg.off, sizeof(unsigned long long) * (ncomm + 1),
                           cudaMemcpyDeviceToHost));
    std::vector<uint32_t> cntv(ncomm + 1);
    DFL_CUDA(h, cudaMemcpy(cntv.data(), h->cnt, sizeof(uint32_t) * (ncomm + 1), cudaMemcpyDeviceToHost));
    std::vector<unsigned long long> gtab(ngiant);
    std::vector<uint32_t> gsize(ngiant);
    unsigned long long total = 0;
    std::vector<uint32_t> chunk0(ngiant);
    uint32_t nitems = 0;
    for (uint32_t k = 0; k < ngiant; ++k) {
      uint32_t cc = giant[k];
      unsigned long long td = soff[cc + 1] - soff[cc];
      unsigned long long distinct = td < ncomm ? td : ncomm;
      gsize[k] = next_pow2(2 * distinct);
      gtab[k] = total;
      total += gsize[k];
      uint32_t members = cntv[cc + 1] - cntv[cc];
      chunk0[k] = nitems;
      nitems += (members + kChunkMembers - 1) / kChunkMembers;
    }
    if (total > h->gtable_cap) {
      cudaFree(h->gtable);
      h->gtable = nullptr;
      h->gtable_cap = 0;
      DFL_CUDA(h, dev_malloc(&h->gtable, sizeof(uint2) * total));
      h->gtable_cap = total;
    }
    // small device arrays for the giant layout (in the generic scratch)
    DFL_TRY(ensure_tmp(h, ngiant * (sizeof(uint32_t) * 3 + sizeof(unsigned long long)) + 64));
    unsigned long long* d_gtab = static_cast<unsigned long long*>(h->tmp);
    uint32_t* d_giant = reinterpret_cast<uint32_t*>(d_gtab + ngiant);
    uint32_t* d_gsize = d_giant + ngiant;
    uint32_t* d_chunk0 = d_gsize + ngiant;
    DFL_CUDA(h, cudaMemcpyAsync(d_chunk0, chunk0.data(), sizeof(uint32_t) * ngiant, cudaMemcpyHostToDevice,
                                h->stream));
    DFL_CUDA(h, cudaMemcpyAsync(d_gtab, gtab.data(), sizeof(unsigned long long) * ngiant,
                                cudaMemcpyHostToDevice, h->stream));
    DFL_CUDA(h, cudaMemcpyAsync(d_giant, giant.data(), sizeof(uint32_t) * ngiant, cudaMemcpyHostToDevice,
                                h->stream));
    DFL_CUDA(h, cudaMemcpyAsync(d_gsize, gsize.data(), sizeof(uint32_t) * ngiant, cudaMemcpyHostToDevice,
                                h->stream));
    a.gtable = h->gtable;
    {  // queue of high-degree members: at most one per vertex of degree > kAggBigMember
      uint64_t arcs = h->num_arcs;
      for (int q = 0; q < 2; ++q) arcs = arcs > h->sg[q].arc_cap ? arcs : h->sg[q].arc_cap;
      const uint64_t need = arcs / (kAggBigMember + 1) + 64;
      if (need > h->aggq_cap) {
        cudaStreamSynchronize(h->stream);
        cudaFree(h->aggq);
        h->aggq = nullptr;
        h->aggq_cap = 0;
        DFL_CUDA(h, dev_malloc(&h->aggq, sizeof(uint2) * need));
        h->aggq_cap = need;
      }
    }
    a.bigq = h->aggq;
    a.nbig = &h->ctrl->red_u;
    DFL_CUDA(h, cudaMemsetAsync(&h->ctrl->red_u, 0, sizeof(unsigned int), h->stream));
    GiantArgs gi{d_giant, d_gtab, d_gsize, d_chunk0, ngiant, nitems};
    {
      LaunchScope ls(h, DFL_PROF_AGG);
      k_giant_init<<<grid_for(total, 256), 256, 0, h->stream>>>(a, gi, total);
      DFL_TRY(check_launch(h, "giant init"));
    }
    {
      LaunchScope ls(h, DFL_PROF_AGG);
      k_agg_giant_accum<<<grid_for(nitems, 1, 152 * 8), 256, 0, h->stream>>>(a, gi);
      DFL_TRY(check_launch(h, "giant accum"));
    }
    {
      LaunchScope ls(h, DFL_PROF_AGG);
      k_agg_big<<<152 * 4, kAggBigThreads, 0, h->stream>>>(a, gi);
      DFL_TRY(check_launch(h, "giant members"));
    }
    {
      LaunchScope ls(h, DFL_PROF_AGG);
      k_agg_giant_emit<<<grid_for(total, 256), 256, 0, h->stream>>>(a, gi, total);
      DFL_TRY(check_launch(h, "giant emit"));
    }
    // the layout arrays live in h->tmp: finish before anyone reuses it
    DFL_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  DFL_TRY(read_ctrl(h));
  if (h->hctrl->err) return set_error(h, DFL_ERR_CUDA, "internal error in aggregation (table overflow)");
  return DFL_OK;
}

}  // namespace dfl
