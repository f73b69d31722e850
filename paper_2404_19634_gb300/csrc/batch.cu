// Batch update of the slack CSR (Section 3.4), incremental K and Sigma
// (Alg. 7), and marking of the initially affected vertices (Alg. 1 DF,
// Alg. 2 ND, Alg. 3 DS).
//
// Two paths.  The hashed path (the default): the batch's arcs go into a
// table of (u, v) pairs, each pair is validated against its row, and a gate
// evaluated on the device after validation lets the writes run or stops
// everything, so the host reads the result once, at the end (or, for
// dfl_step, after the update queued behind it).  The sort-based path (a
// rebuilt row gaining more arcs than a block sorts): the batch is expanded
// into directed arcs keyed u << (b+1) | v << 1 | type (type 0 = deletion,
// 1 = insertion; b = bits of n-1) and sorted, so the arcs of one row are
// contiguous, ordered by neighbour, deletions before insertions; a maximal
// run of equal (u, v) is one arc change, and everything is validated (one
// host read-back) before any state is touched.
#include "common.cuh"

namespace dfl {

int apply_batch_sorted(Handle* h, const dfl_edge* del, uint64_t nd, const dfl_edge* ins, uint64_t ni,
                       int mem_kind);

namespace {

// Slack-CSR row layout: arcs [0, srt) are sorted by neighbour, arcs
// [srt, deg) are an unsorted tail of at most kTailMax appended arcs, and a
// deleted arc stays as a tombstone (weight 0) until the row is rebuilt.  A
// neighbour id appears at most once in a row (a re-inserted edge revives its
// tombstone).  A row is rebuilt (sorted, tombstones dropped, relocated) when
// it would outgrow its capacity, its tail or its tombstone budget.
constexpr uint32_t kTailMax = 64;
constexpr uint32_t kTombMin = 8;

// b_flag bits
constexpr uint32_t kRunHead = 1u;     // first arc of a (u, v) run
constexpr uint32_t kFound = 2u;       // the row already has a slot for v
constexpr uint32_t kLiveBefore = 4u;  // ... holding weight > 0
constexpr uint32_t kLiveAfter = 8u;   // the arc has weight > 0 after the batch
constexpr uint32_t kAppend = 16u;     // a new slot is needed
constexpr uint32_t kRebuild = 32u;    // (every run of the row) the row is rebuilt

__host__ __device__ inline uint32_t grow_cap(uint32_t d) {
  uint64_t c = uint64_t(d) + d / 2 + 8;
  c = (c + 1) & ~uint64_t(1);
  return c > 0xFFFFFFFEull ? 0xFFFFFFFEu : uint32_t(c);
}

struct KeyFmt {
  uint32_t b;          // bits of a vertex id
  uint64_t vmask;
  __device__ uint32_t u(unsigned long long k) const { return uint32_t(k >> (b + 1)); }
  __device__ uint32_t v(unsigned long long k) const { return uint32_t((k >> 1) & vmask); }
  __device__ unsigned long long pair(unsigned long long k) const { return k >> 1; }
};

// Expand edges into both arcs; reject ids >= n, self-loops, zero insertions.
__global__ void k_expand(const dfl_edge* __restrict__ e, uint64_t nd, uint64_t ne, uint32_t n,
                         KeyFmt f, unsigned long long* __restrict__ key, uint32_t* __restrict__ w,
                         Ctrl* ctrl) {
  for (uint64_t t = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; t < ne;
       t += uint64_t(gridDim.x) * blockDim.x) {
    dfl_edge x = e[t];
    unsigned long long type = t >= nd ? 1ull : 0ull;
    bool bad = x.u >= n || x.v >= n || x.u == x.v || (type && x.w == 0);
    if (bad) {
      atomicOr(&ctrl->err, kErrInvalid);
      key[2 * t] = key[2 * t + 1] = 0;
      w[2 * t] = w[2 * t + 1] = 0;
      continue;
    }
    key[2 * t] = ((unsigned long long)x.u << (f.b + 1)) | ((unsigned long long)x.v << 1) | type;
    key[2 * t + 1] = ((unsigned long long)x.v << (f.b + 1)) | ((unsigned long long)x.u << 1) | type;
    w[2 * t] = w[2 * t + 1] = x.w;
  }
}

// Slot of neighbour v in row u: binary search of the sorted prefix, then a
// scan of the tail.  Returns kEmpty if absent.
__device__ __forceinline__ uint32_t find_slot(const uint2* __restrict__ row, uint32_t srt, uint32_t deg,
                                              uint32_t v) {
  // lower bound of v in the sorted prefix: nine-way splits with the eight
  // probe loads in flight together (a hub row takes ~6 rounds, not ~20)
  uint32_t lo = 0, hi = srt;
  while (hi - lo > 16) {
    const uint32_t step = (hi - lo) / 9;
    uint32_t key[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) key[j] = row[lo + (j + 1) * step].x;
    uint32_t nlo = lo, nhi = hi;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint32_t pos = lo + (j + 1) * step;
      if (key[j] < v) nlo = pos + 1;
      else if (pos < nhi) nhi = pos;
    }
    lo = nlo;
    hi = nhi;
  }
  {
    uint32_t key[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) key[j] = lo + j < hi ? row[lo + j].x : 0xFFFFFFFFu;
    uint32_t lb = hi;
#pragma unroll
    for (int j = 15; j >= 0; --j)
      if (lo + j < hi && key[j] >= v) lb = lo + j;
    lo = lb;
  }
  if (lo < srt && row[lo].x == v) return lo;
  // the unsorted tail (at most kTailMax arcs), eight loads in flight
  for (uint32_t q0 = srt; q0 < deg; q0 += 8) {
    uint32_t x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = q0 + u < deg ? row[q0 + u].x : ~v;
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (x[u] == v) return q0 + u;
  }
  return kEmpty;
}

// Thread per sorted arc: each run head evaluates its (u, v) change against
// the current row (validation happens here, before any state changes).
__global__ void k_runs(const unsigned long long* __restrict__ key, const uint32_t* __restrict__ w,
                       uint64_t na, KeyFmt f, uint32_t n, const unsigned long long* __restrict__ off,
                       const uint32_t* __restrict__ deg, const uint32_t* __restrict__ srt,
                       const uint2* __restrict__ arcs, unsigned long long* __restrict__ pos_out,
                       uint32_t* __restrict__ wnew_out, uint32_t* __restrict__ flag,
                       long long* __restrict__ delta_out, uint32_t* __restrict__ rowlist, Ctrl* ctrl) {
  for (uint64_t p = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; p < na;
       p += uint64_t(gridDim.x) * blockDim.x) {
    unsigned long long k = key[p];
    bool head = p == 0 || f.pair(key[p - 1]) != f.pair(k);
    if (!head) {
      flag[p] = 0;
      continue;
    }
    uint32_t u = f.u(k), v = f.v(k);
    if (p == 0 || f.u(key[p - 1]) != u) {
      uint32_t slot = atomicAdd(&ctrl->rows, 1u);
      rowlist[slot] = uint32_t(p);
    }
    uint32_t ndel = 0, wdel = 0;
    unsigned long long wins = 0;
    for (uint64_t q = p; q < na && f.pair(key[q]) == f.pair(k); ++q) {
      if (key[q] & 1ull) wins += w[q];
      else {
        ++ndel;
        wdel = w[q];
      }
    }
    if (u >= n || v >= n) {
      atomicOr(&ctrl->err, kErrInvalid);
      flag[p] = kRunHead;
      continue;
    }
    if (ndel > 1) atomicOr(&ctrl->err, kErrInvalid);  // the same edge deleted twice
    const uint2* row = arcs + off[u];
    uint32_t slot = find_slot(row, srt[u], deg[u], v);
    unsigned long long wold = slot != kEmpty ? row[slot].y : 0ull;
    unsigned long long weff = 0;
    if (ndel) {
      if (wold == 0 || wdel > wold) atomicOr(&ctrl->err, kErrNotFound);  // absent edge
      else weff = wdel ? wdel : wold;
    }
    unsigned long long wn = wold - weff + wins;
    if (wn > 0xFFFFFFFFull) atomicOr(&ctrl->err, kErrOverflow);
    uint32_t fl = kRunHead;
    if (slot != kEmpty) fl |= kFound;
    if (wold > 0) fl |= kLiveBefore;
    if (wn > 0) fl |= kLiveAfter;
    if (slot == kEmpty && wn > 0) fl |= kAppend;
    long long delta = (long long)wins - (long long)weff;
    pos_out[p] = slot;
    wnew_out[p] = uint32_t(wn);
    flag[p] = fl;
    delta_out[p] = delta;
    if (delta) atomicAdd((unsigned long long*)&ctrl->m2_delta, (unsigned long long)delta);
  }
}

// Thread per touched row: appends (ranked in run order), tombstone and live
// counts, and whether the row must be rebuilt.
__global__ void k_rows(const unsigned long long* __restrict__ key, uint64_t na, KeyFmt f,
                       const uint32_t* __restrict__ rowlist, const uint32_t* __restrict__ deg,
                       const uint32_t* __restrict__ cap, const uint32_t* __restrict__ srt,
                       const uint32_t* __restrict__ ntomb, unsigned long long* __restrict__ pos,
                       uint32_t* __restrict__ flag, uint32_t* __restrict__ cum,
                       uint32_t* __restrict__ newdeg, uint32_t* __restrict__ newtomb,
                       uint32_t* __restrict__ rebuild_list, Ctrl* ctrl) {
  const uint32_t rows = ctrl->rows;
  for (uint64_t t = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; t < rows;
       t += uint64_t(gridDim.x) * blockDim.x) {
    const uint32_t p = rowlist[t];
    const uint32_t u = f.u(key[p]);
    const uint32_t d = deg[u], s = srt[u], nt = ntomb[u];
    uint32_t appends = 0;
    long long tomb = nt, live = (long long)d - nt;
    uint64_t end = p;
    for (; end < na && f.u(key[end]) == u; ++end) {
      uint32_t fl = flag[end];
      if (!(fl & kRunHead)) continue;
      cum[end] = appends;
      if (fl & kAppend) pos[end] = appends++;
      bool before = fl & kLiveBefore, after = fl & kLiveAfter;
      live += (after ? 1 : 0) - (before ? 1 : 0);
      if ((fl & kFound) && before && !after) ++tomb;
      if ((fl & kFound) && !before && after) --tomb;
    }
    const uint32_t raw = d + appends;
    const uint32_t tail = d - s + appends;
    const uint32_t tomb_lim = raw / 4 > kTombMin ? raw / 4 : kTombMin;
    const bool rebuild = raw > cap[u] || tail > kTailMax || uint32_t(tomb) > tomb_lim;
    if (rebuild) {
      for (uint64_t q = p; q < end; ++q)
        if (flag[q] & kRunHead) flag[q] |= kRebuild;
      uint32_t slot = atomicAdd(&ctrl->rebuild_rows, 1u);
      rebuild_list[slot] = p;
      atomicAdd(&ctrl->reloc_need, (unsigned long long)grow_cap(uint32_t(live)));
      atomicAdd(&ctrl->scratch_need, (unsigned long long)s);
    }
    newdeg[p] = rebuild ? uint32_t(live) : raw;
    newtomb[p] = rebuild ? 0u : uint32_t(tomb);
    atomicMax(&ctrl->max_deg, rebuild ? uint32_t(live) : raw);
    long long dl = live - ((long long)d - nt);
    if (dl) atomicAdd((unsigned long long*)&ctrl->arc_delta, (unsigned long long)dl);
  }
}

// Thread per run: weight changes in place (also before a rebuild, which
// then reads the updated row), and appends to the tail of kept rows.
__global__ void k_write(const unsigned long long* __restrict__ key, uint64_t na, KeyFmt f,
                        const unsigned long long* __restrict__ off, const uint32_t* __restrict__ deg,
                        uint2* __restrict__ arcs, const unsigned long long* __restrict__ pos,
                        const uint32_t* __restrict__ wnew, const uint32_t* __restrict__ flag) {
  for (uint64_t p = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; p < na;
       p += uint64_t(gridDim.x) * blockDim.x) {
    uint32_t fl = flag[p];
    if (!(fl & kRunHead)) continue;
    uint32_t u = f.u(key[p]);
    uint2* row = arcs + off[u];
    if (fl & kFound) row[pos[p]].y = wnew[p];
    else if ((fl & kAppend) && !(fl & kRebuild)) row[deg[u] + pos[p]] = make_uint2(f.v(key[p]), wnew[p]);
  }
}

// Thread per touched row that is kept: new degree and tombstone count.
__global__ void k_finish(const unsigned long long* __restrict__ key, KeyFmt f,
                         const uint32_t* __restrict__ rowlist, const uint32_t* __restrict__ flag,
                         const uint32_t* __restrict__ newdeg, const uint32_t* __restrict__ newtomb,
                         uint32_t* __restrict__ deg, uint32_t* __restrict__ ntomb, Ctrl* ctrl) {
  const uint32_t rows = ctrl->rows;
  for (uint64_t t = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; t < rows;
       t += uint64_t(gridDim.x) * blockDim.x) {
    uint32_t p = rowlist[t];
    if (flag[p] & kRebuild) continue;
    uint32_t u = f.u(key[p]);
    deg[u] = newdeg[p];
    ntomb[u] = newtomb[p];
  }
}

// Number of appended runs of the row [p, end) with neighbour < v.
__device__ __forceinline__ uint32_t new_below(const unsigned long long* __restrict__ key, KeyFmt f,
                                              uint64_t p, uint64_t end, const uint32_t* __restrict__ cum,
                                              uint32_t total, uint32_t v) {
  uint64_t lo = p, hi = end;
  while (lo < hi) {
    uint64_t mid = (lo + hi) >> 1;
    if (f.v(key[mid]) < v) lo = mid + 1;
    else hi = mid;
  }
  return lo == end ? total : cum[lo];  // lo is a run head
}

__device__ __forceinline__ uint32_t count_below(const uint2* __restrict__ a, uint32_t len, uint32_t v) {
  uint32_t lo = 0, hi = len;
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (a[mid].x < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

constexpr int kRebuildThreads = 256;

// Block per rebuilt row: three-way merge of the live sorted prefix (first
// compacted into scratch), the live tail (sorted in shared memory) and the
// batch's new arcs (sorted by the batch sort) into a new, larger slot.
__global__ void __launch_bounds__(kRebuildThreads)
k_rebuild(const unsigned long long* __restrict__ key, uint64_t na, KeyFmt f,
          const uint32_t* __restrict__ rebuild_list, unsigned long long* __restrict__ off,
          uint32_t* __restrict__ deg, uint32_t* __restrict__ cap, uint32_t* __restrict__ srt,
          uint32_t* __restrict__ ntomb, uint2* __restrict__ arcs, const unsigned long long* __restrict__ pos,
          const uint32_t* __restrict__ wnew, const uint32_t* __restrict__ flag,
          const uint32_t* __restrict__ cum, const uint32_t* __restrict__ newdeg, uint2* __restrict__ scratch,
          unsigned long long pool_base, unsigned long long pool_cap, unsigned long long scratch_cap,
          Ctrl* ctrl) {
  __shared__ uint2 tail[kTailMax];
  __shared__ uint2 stail[kTailMax];
  __shared__ unsigned long long s_sbase, s_dst;
  __shared__ uint32_t s_nt, s_warp[kRebuildThreads / 32], s_total;
  const uint32_t nrows = ctrl->rebuild_rows;
  const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
  for (uint32_t r = blockIdx.x; r < nrows; r += gridDim.x) {
    const uint32_t p = rebuild_list[r];
    const uint32_t u = f.u(key[p]);
    const uint2* old = arcs + off[u];
    const uint32_t d = deg[u], s = srt[u], live = newdeg[p];
    uint64_t end = p;
    while (end < na && f.u(key[end]) == u) ++end;
    // appended runs of this row
    uint32_t nnew = 0;
    for (uint64_t q = end; q > p; --q)
      if (flag[q - 1] & kRunHead) {
        nnew = cum[q - 1] + ((flag[q - 1] & kAppend) ? 1u : 0u);
        break;
      }
    if (threadIdx.x == 0) {
      s_sbase = atomicAdd(&ctrl->scratch_top, (unsigned long long)s);
      uint32_t nc = grow_cap(live);
      s_dst = pool_base + atomicAdd(&ctrl->pool_top, (unsigned long long)nc);
      s_nt = 0;
      if (s_sbase + s > scratch_cap || s_dst + nc > pool_cap) atomicOr(&ctrl->err, kErrInternal);
    }
    __syncthreads();
    const unsigned long long sbase = s_sbase, dst = s_dst;
    const uint32_t nc = grow_cap(live);
    if (sbase + s > scratch_cap || dst + nc > pool_cap) {
      __syncthreads();
      continue;
    }
    uint2* A = scratch + sbase;
    // A: live prefix compacted in order
    uint32_t L = 0;
    for (uint32_t c0 = 0; c0 < s; c0 += blockDim.x) {
      uint32_t k = c0 + threadIdx.x;
      uint2 a = k < s ? old[k] : make_uint2(0, 0);
      bool lv = k < s && a.y > 0;
      unsigned m = __ballot_sync(0xFFFFFFFFu, lv);
      if (lane == 0) s_warp[wib] = __popc(m);
      __syncthreads();
      if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (uint32_t x = 0; x < blockDim.x / 32; ++x) {
          uint32_t t = s_warp[x];
          s_warp[x] = run;
          run += t;
        }
        s_total = run;
      }
      __syncthreads();
      if (lv) A[L + s_warp[wib] + __popc(m & ((1u << lane) - 1u))] = a;
      L += s_total;
      __syncthreads();
    }
    // T: live tail, sorted by rank
    for (uint32_t k = s + threadIdx.x; k < d; k += blockDim.x) {
      uint2 a = old[k];
      if (a.y > 0) tail[atomicAdd(&s_nt, 1u)] = a;
    }
    __syncthreads();
    const uint32_t nt = s_nt;
    for (uint32_t k = threadIdx.x; k < nt; k += blockDim.x) {
      uint32_t rk = 0;
      for (uint32_t x = 0; x < nt; ++x) rk += tail[x].x < tail[k].x;
      stail[rk] = tail[k];
    }
    __syncthreads();
    uint2* out = arcs + dst;
    for (uint32_t k = threadIdx.x; k < L; k += blockDim.x) {
      uint2 a = A[k];
      out[k + count_below(stail, nt, a.x) + new_below(key, f, p, end, cum, nnew, a.x)] = a;
    }
    for (uint32_t k = threadIdx.x; k < nt; k += blockDim.x) {
      uint2 a = stail[k];
      out[k + count_below(A, L, a.x) + new_below(key, f, p, end, cum, nnew, a.x)] = a;
    }
    for (uint64_t q = p + threadIdx.x; q < end; q += blockDim.x) {
      uint32_t fl = flag[q];
      if ((fl & kRunHead) && (fl & kAppend)) {
        uint32_t v = f.v(key[q]);
        out[pos[q] + count_below(A, L, v) + count_below(stail, nt, v)] = make_uint2(v, wnew[q]);
      }
    }
    if (threadIdx.x == 0) {
      if (L + nt + nnew != live) atomicOr(&ctrl->err, kErrInternal);
      off[u] = dst;
      deg[u] = live;
      srt[u] = live;
      cap[u] = nc;
      ntomb[u] = 0;
    }
    __syncthreads();
  }
}

// Alg. 7: K[i] and Sigma[C^{t-1}[i]] change by the net weight of each arc.
__global__ void k_update_weights(const unsigned long long* __restrict__ key, uint64_t na, KeyFmt f,
                                 const uint32_t* __restrict__ flag, const long long* __restrict__ delta,
                                 const uint32_t* __restrict__ C, long long* __restrict__ K,
                                 long long* __restrict__ Sigma) {
  for (uint64_t p = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; p < na;
       p += uint64_t(gridDim.x) * blockDim.x) {
    if (!(flag[p] & kRunHead)) continue;
    long long dl = delta[p];
    if (!dl) continue;
    uint32_t u = f.u(key[p]);
    atomicAdd((unsigned long long*)&K[u], (unsigned long long)dl);
    atomicAdd((unsigned long long*)&Sigma[C[u]], (unsigned long long)dl);
  }
}

// ---------------------------------------------------------------------------
// Marking
// ---------------------------------------------------------------------------

// Alg. 1: a deletion inside a community or an insertion across communities
// marks its source (both arcs are present, so both endpoints).
// One launch clears what an update starts from: local-moving's control block,
// the two frontier bitsets and (DF) the set of vertices processed in the
// first pass -- instead of one memset each.
__global__ void k_mark_clear(Ctrl* ctrl, uint32_t* __restrict__ f0, uint32_t* __restrict__ f1,
                             uint32_t* __restrict__ ever, uint32_t words) {
  pdl_wait();
  const uint64_t base = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x;
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  unsigned int* z = reinterpret_cast<unsigned int*>(ctrl);
  for (uint64_t q = base; q < sizeof(Ctrl) / sizeof(unsigned int); q += stride) z[q] = 0u;
  for (uint64_t q = base; q < words; q += stride) {
    f0[q] = 0u;
    f1[q] = 0u;
    if (ever) ever[q] = 0u;
  }
}

__global__ void k_mark_df(const unsigned long long* __restrict__ key, uint64_t na, KeyFmt f,
                          const uint32_t* __restrict__ C, const uint32_t* __restrict__ deg,
                          uint32_t* __restrict__ fbits, uint32_t* lists, Segs seg, Ctrl* ctrl,
                          uint32_t k, const unsigned int* go) {
  pdl_wait();
  if (go && *go == 0u) return;  // the batch enqueued before this update was not applied: mark nothing
  uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t p0 = blockIdx.x * uint64_t(blockDim.x); p0 < na; p0 += stride) {
    uint64_t p = p0 + threadIdx.x;
    bool valid = false;
    uint32_t u = 0, lk = 0;
    if (p < na) {
      unsigned long long kk = key[p];
      u = f.u(kk);
      uint32_t v = f.v(kk);
      bool ins = kk & 1ull;
      bool same = C[u] == C[v];
      if (ins != same && bit_set(fbits, u)) {
        valid = true;
        lk = vertex_class(u, k, seg) * kBins + degree_bin(deg[u], seg);
      }
    }
    append_vertex(u, valid, lk, lists, seg, ctrl, 0);
  }
}

// Alg. 3, deletions inside a community: dV[i], dE[i], dC[C[j]].
__global__ void k_ds_del(const unsigned long long* __restrict__ key, uint64_t na, KeyFmt f,
                         const uint32_t* __restrict__ C, uint32_t* dV, uint32_t* dE, uint32_t* dC) {
  for (uint64_t p = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; p < na;
       p += uint64_t(gridDim.x) * blockDim.x) {
    unsigned long long kk = key[p];
    if (kk & 1ull) continue;
    uint32_t u = f.u(kk), v = f.v(kk);
    if (C[u] == C[v]) {
      bit_set(dV, u);
      bit_set(dE, u);
      bit_set(dC, C[v]);
    }
  }
}

// Alg. 3, insertions across communities: collect (source, C[target]) keys.
__global__ void k_ds_keys(const unsigned long long* __restrict__ key, const uint32_t* __restrict__ w,
                          uint64_t na, KeyFmt f, const uint32_t* __restrict__ C,
                          unsigned long long* __restrict__ okey, uint32_t* __restrict__ ow,
                          Ctrl* ctrl) {
  for (uint64_t p = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; p < na;
       p += uint64_t(gridDim.x) * blockDim.x) {
    unsigned long long kk = key[p];
    if (!(kk & 1ull)) continue;
    uint32_t u = f.u(kk), v = f.v(kk);
    uint32_t cv = C[v];
    if (C[u] == cv) continue;
    unsigned long long slot = atomicAdd(&ctrl->red_a, 1ull);
    okey[slot] = ((unsigned long long)u << 32) | cv;
    ow[slot] = w[p];
  }
}

// Per source u (sorted keys u << 32 | c): H[c] = summed inserted weight;
// best c by 2m*H[c] - K_u*Sigma_c, ties to the smallest c.
__global__ void k_ds_best(const unsigned long long* __restrict__ key, const uint32_t* __restrict__ w,
                          uint64_t na, long long m2_one, uint32_t ngraphs, const uint32_t* __restrict__ goff,
                          const long long* __restrict__ gm2, const long long* __restrict__ K,
                          const long long* __restrict__ Sigma, uint32_t* dV, uint32_t* dE,
                          uint32_t* dC) {
  for (uint64_t p = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; p < na;
       p += uint64_t(gridDim.x) * blockDim.x) {
    uint32_t u = uint32_t(key[p] >> 32);
    if (p > 0 && uint32_t(key[p - 1] >> 32) == u) continue;
    const long long m2 = ngraphs ? gm2[graph_of(goff, ngraphs, u)] : m2_one;  // u's graph's 2m
    bool have = false;
    i128 best_s = 0;
    uint32_t best = 0;
    uint64_t q = p;
    while (q < na && uint32_t(key[q] >> 32) == u) {
      uint32_t c = uint32_t(key[q]);
      unsigned long long hsum = 0;
      while (q < na && key[q] == (((unsigned long long)u << 32) | c)) hsum += w[q++];
      i128 s = (i128)m2 * (i128)hsum - (i128)K[u] * (i128)Sigma[c];
      if (!have || s > best_s) {
        have = true;
        best_s = s;
        best = c;
      }
    }
    bit_set(dV, u);
    bit_set(dE, u);
    bit_set(dC, best);
  }
}

// Alg. 3: neighbours of dE vertices join dV (warp per bitmap word).
__global__ void k_ds_expand(const uint32_t* __restrict__ dE, uint32_t words, uint32_t n,
                            GraphView g, uint32_t* dV) {
  const uint32_t lane = threadIdx.x & 31u;
  uint64_t warp = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) >> 5;
  uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  for (uint64_t wd = warp; wd < words; wd += nwarps) {
    uint32_t x = dE[wd];
    while (x) {
      int b = __ffs(x) - 1;
      x &= x - 1;
      uint32_t i = uint32_t(wd * 32 + b);
      if (i >= n) break;
      unsigned long long o = g.off[i];
      uint32_t d = g.deg[i];
      for (uint32_t k = lane; k < d; k += 32) {
        uint2 a = g.arcs[o + k];
        if (a.y) bit_set(dV, a.x);  // weight 0 = deleted arc
      }
    }
  }
}

// Alg. 3: vertices of dC communities join dV.
__global__ void k_ds_comm(uint32_t n, const uint32_t* __restrict__ C, const uint32_t* __restrict__ dC,
                          uint32_t* dV) {
  uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i0 = blockIdx.x * uint64_t(blockDim.x); i0 < n; i0 += stride) {
    uint64_t i = i0 + threadIdx.x;
    bool set = i < n && bit_test(dC, C[i]);
    unsigned m = __ballot_sync(0xFFFFFFFFu, set);
    if ((threadIdx.x & 31u) == 0 && m) atomicOr(&dV[i >> 5], m);
  }
}

// ---------------------------------------------------------------------------
// Hashed batch apply.  Arcs are grouped by (u, v) in an open-addressing table
// (no sort); a new arc's tail position comes from a per-row counter (the tail
// is unsorted, so the order does not matter); only rebuilt rows need their
// new arcs sorted, which a block does in shared memory.  Per-vertex scratch
// counters are zero at rest and reset for the touched rows at the end.
// ---------------------------------------------------------------------------
constexpr uint32_t kExtraMax = 4096;   // new arcs of one rebuilt row sorted in shared memory
constexpr unsigned long long kNoKey = ~0ull;

struct HashApply {
  unsigned long long* keys;   // (u << 32 | v), kNoKey = empty
  uint32_t* ndel;             // deletions of the pair
  uint32_t* wdel;             // their weight (0 = whole edge)
  unsigned long long* wins;   // summed inserted weight
  uint32_t* slot;             // row slot of the pair (found) or append rank
  uint32_t* wnew;
  uint32_t* flag;
  long long* delta;
  uint32_t* pairs;            // occupied table slots, in claim order
  uint64_t mask;
  // per-vertex scratch
  uint32_t* r_app;            // appends of the row (then: rank counter)
  int* r_tomb;                // tombstone change
  int* r_live;                // live-arc change
  uint32_t* r_state;          // 0 untouched, 1 touched, 2 rebuilt
  uint32_t* r_reg;            // rebuilt row: offset of its new arcs in `extra`
  uint32_t* rows;             // touched rows, in touch order
  uint2* extra;               // new arcs of rebuilt rows
};

__device__ __forceinline__ unsigned long long hash64(unsigned long long k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

// Thread per edge: both arcs into the table; arcs also staged (key format of
// the pending list) for the frontier marking of the next update.
// Claim `n` consecutive entries of a shared counter for the lanes with `want`
// set (one atomic per warp); returns this lane's entry.  Every lane of the
// warp must call it.
__device__ __forceinline__ uint32_t warp_claim(unsigned int* counter, bool want) {
  const unsigned m = __ballot_sync(0xFFFFFFFFu, want);
  if (!m) return 0;
  const uint32_t lane = threadIdx.x & 31u, leader = __ffs(m) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(counter, uint32_t(__popc(m)));
  base = __shfl_sync(0xFFFFFFFFu, base, leader);
  return base + __popc(m & ((1u << lane) - 1u));
}

__device__ __forceinline__ long long warp_sum64(long long x) {
  for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
  return x;
}

// del: the nd deletions, ins: the ne - nd insertions
__device__ __forceinline__ void hash_insert_body(const dfl_edge* __restrict__ del, const dfl_edge* __restrict__ ins,
                              uint64_t nd, uint64_t ne, uint32_t n,
                              KeyFmt f, HashApply t, unsigned long long* __restrict__ key,
                              uint32_t* __restrict__ w, Ctrl* ctrl, uint64_t base, uint64_t stride) {
  // warp-uniform loop: the claims of new table slots are made per warp
  const uint32_t lane = threadIdx.x & 31u;
  for (uint64_t q0 = base + (threadIdx.x & ~31u); q0 < ne; q0 += stride) {
    const uint64_t q = q0 + lane;
    bool valid = q < ne;
    const bool is_ins = q >= nd;
    dfl_edge x = valid ? (is_ins ? ins[q - nd] : del[q]) : dfl_edge{0, 0, 0};
    if (valid && (x.u >= n || x.v >= n || x.u == x.v || (is_ins && x.w == 0))) {
      atomicOr(&ctrl->err, kErrInvalid);
      key[2 * q] = key[2 * q + 1] = 0;
      w[2 * q] = w[2 * q + 1] = 0;
      valid = false;
    }
    for (int dir = 0; dir < 2; ++dir) {
      bool claimed = false;
      uint32_t cs = 0;
      if (valid) {
        const uint32_t a = dir ? x.v : x.u, b = dir ? x.u : x.v;
        key[2 * q + dir] = ((unsigned long long)a << (f.b + 1)) | ((unsigned long long)b << 1) |
                           (is_ins ? 1ull : 0ull);
        w[2 * q + dir] = x.w;
        const unsigned long long k = ((unsigned long long)a << 32) | b;
        uint64_t s = hash64(k) & t.mask;
        for (uint64_t probe = 0; probe <= t.mask; ++probe) {
          unsigned long long prev = t.keys[s];
          if (prev == kNoKey) {
            prev = atomicCAS(&t.keys[s], kNoKey, k);
            if (prev == kNoKey) {
              claimed = true;
              cs = uint32_t(s);
              prev = k;
            }
          }
          if (prev == k) {
            if (is_ins) {
              atomicAdd(&t.wins[s], (unsigned long long)x.w);
            } else {
              atomicAdd(&t.ndel[s], 1u);
              t.wdel[s] = x.w;  // several deletions of one pair are an error anyway
            }
            break;
          }
          s = (s + 1) & t.mask;
        }
      }
      const uint32_t at = warp_claim(&ctrl->npairs, claimed);
      if (claimed) t.pairs[at] = cs;
    }
  }
}

__global__ void k_hash_insert(const dfl_edge* __restrict__ del, const dfl_edge* __restrict__ ins, uint64_t nd,
                              uint64_t ne, uint32_t n, KeyFmt f, HashApply t, unsigned long long* __restrict__ key,
                              uint32_t* __restrict__ w, Ctrl* ctrl) {
  pdl_wait();
  hash_insert_body(del, ins, nd, ne, n, f, t, key, w, ctrl, blockIdx.x * uint64_t(blockDim.x), uint64_t(gridDim.x) * blockDim.x);
}

// Thread per pair: validate against the row, weights after the batch, and
// per-row bookkeeping (append ranks, live and tombstone changes).
__device__ __forceinline__ void hash_pairs_body(HashApply t, uint32_t n, const unsigned long long* __restrict__ off,
                             const uint32_t* __restrict__ deg, const uint32_t* __restrict__ srt,
                             const uint2* __restrict__ arcs, Ctrl* ctrl, uint64_t base, uint64_t stride) {
  const uint32_t np = ctrl->npairs;
  const uint32_t lane = threadIdx.x & 31u;
  // warp-uniform loop: 2m and arc-count changes are summed, new rows claimed, per warp
  for (uint64_t p0 = base + (threadIdx.x & ~31u); p0 < np; p0 += stride) {
    const uint64_t p = p0 + lane;
    long long dm2 = 0, darcs = 0;
    bool new_row = false;
    uint32_t row_u = 0;
    if (p < np) {
      const uint32_t s = t.pairs[p];
      const unsigned long long k = t.keys[s];
      const uint32_t u = uint32_t(k >> 32), v = uint32_t(k);
      const uint32_t ndel = t.ndel[s], wdel = t.wdel[s];
      const unsigned long long wins = t.wins[s];
      if (ndel > 1) atomicOr(&ctrl->err, kErrInvalid);  // the same edge deleted twice
      const uint2* row = arcs + off[u];
      const uint32_t slot = find_slot(row, srt[u], deg[u], v);
      const unsigned long long wold = slot != kEmpty ? row[slot].y : 0ull;
      unsigned long long weff = 0;
      if (ndel) {
        if (wold == 0 || wdel > wold) atomicOr(&ctrl->err, kErrNotFound);
        else weff = wdel ? wdel : wold;
      }
      const unsigned long long wn = wold - weff + wins;
      if (wn > 0xFFFFFFFFull) atomicOr(&ctrl->err, kErrOverflow);
      uint32_t fl = kRunHead;
      if (slot != kEmpty) fl |= kFound;
      if (wold > 0) fl |= kLiveBefore;
      if (wn > 0) fl |= kLiveAfter;
      if (slot == kEmpty && wn > 0) fl |= kAppend;
      const long long dl = (long long)wins - (long long)weff;
      t.wnew[s] = uint32_t(wn);
      t.flag[s] = fl;
      t.delta[s] = dl;
      t.slot[s] = (fl & kAppend) ? atomicAdd(&t.r_app[u], 1u) : slot;
      dm2 = dl;
      const int live = (wn > 0 ? 1 : 0) - (wold > 0 ? 1 : 0);
      if (live) {
        atomicAdd(&t.r_live[u], live);
        darcs = live;
      }
      if ((fl & kFound) && wold > 0 && wn == 0) atomicAdd(&t.r_tomb[u], 1);
      if ((fl & kFound) && wold == 0 && wn > 0) atomicAdd(&t.r_tomb[u], -1);
      new_row = atomicCAS(&t.r_state[u], 0u, 1u) == 0u;
      row_u = u;
    }
    const uint32_t at = warp_claim(&ctrl->rows, new_row);
    if (new_row) t.rows[at] = row_u;
    dm2 = warp_sum64(dm2);
    darcs = warp_sum64(darcs);
    if (lane == 0) {
      if (dm2) atomicAdd((unsigned long long*)&ctrl->m2_delta, (unsigned long long)dm2);
      if (darcs) atomicAdd((unsigned long long*)&ctrl->arc_delta, (unsigned long long)darcs);
    }
  }
}

__global__ void k_hash_pairs(HashApply t, uint32_t n, const unsigned long long* __restrict__ off,
                             const uint32_t* __restrict__ deg, const uint32_t* __restrict__ srt,
                             const uint2* __restrict__ arcs, Ctrl* ctrl) {
  pdl_wait();
  hash_pairs_body(t, n, off, deg, srt, arcs, ctrl, blockIdx.x * uint64_t(blockDim.x), uint64_t(gridDim.x) * blockDim.x);
}

// Thread per touched row: keep (append in place) or rebuild.
__device__ __forceinline__ void hash_rows_body(HashApply t, const uint32_t* __restrict__ deg, const uint32_t* __restrict__ cap,
                            const uint32_t* __restrict__ srt, const uint32_t* __restrict__ ntomb, Ctrl* ctrl, uint64_t base, uint64_t stride) {
  const uint32_t nr = ctrl->rows;
  for (uint64_t q0 = base + (threadIdx.x & ~31u); q0 < nr; q0 += stride) {
    const uint64_t q = q0 + (threadIdx.x & 31u);
    uint32_t dmax = 0;
    if (q < nr) {
      const uint32_t u = t.rows[q];
      const uint32_t d = deg[u], s = srt[u], app = t.r_app[u];
      const long long tomb = (long long)ntomb[u] + t.r_tomb[u];
      const long long live = (long long)d - ntomb[u] + t.r_live[u];
      const uint32_t raw = d + app;
      const uint32_t tomb_lim = raw / 4 > kTombMin ? raw / 4 : kTombMin;
      const bool rebuild = raw > cap[u] || d - s + app > kTailMax || uint32_t(tomb) > tomb_lim;
      if (rebuild) {
        t.r_state[u] = 2u;
        t.r_reg[u] = uint32_t(atomicAdd(&ctrl->extra_top, (unsigned long long)app));
        atomicAdd(&ctrl->rebuild_rows, 1u);
        atomicAdd(&ctrl->reloc_need, (unsigned long long)grow_cap(uint32_t(live)));
        atomicAdd(&ctrl->scratch_need, (unsigned long long)s);
        atomicMax(&ctrl->max_app, app);
      }
      dmax = rebuild ? uint32_t(live) : raw;
    }
    dmax = __reduce_max_sync(0xFFFFFFFFu, dmax);  // one update per warp
    if ((threadIdx.x & 31u) == 0 && dmax) atomicMax(&ctrl->max_deg, dmax);
  }
}

__global__ void k_hash_rows(HashApply t, const uint32_t* __restrict__ deg, const uint32_t* __restrict__ cap,
                            const uint32_t* __restrict__ srt, const uint32_t* __restrict__ ntomb, Ctrl* ctrl) {
  pdl_wait();
  hash_rows_body(t, deg, cap, srt, ntomb, ctrl, blockIdx.x * uint64_t(blockDim.x), uint64_t(gridDim.x) * blockDim.x);
}

// Thread per pair: in-place weight changes; new arcs to the row's tail, or to
// the rebuilt row's region of `extra`.
__device__ __forceinline__ void hash_write_body(HashApply t, const unsigned long long* __restrict__ off,
                             const uint32_t* __restrict__ deg, uint2* __restrict__ arcs, Ctrl* ctrl, uint64_t base, uint64_t stride) {
  const uint32_t np = ctrl->npairs;
  for (uint64_t p = base + threadIdx.x; p < np;
       p += stride) {
    const uint32_t s = t.pairs[p];
    const uint32_t fl = t.flag[s];
    const unsigned long long k = t.keys[s];
    const uint32_t u = uint32_t(k >> 32), v = uint32_t(k);
    if (fl & kFound) {
      arcs[off[u] + t.slot[s]].y = t.wnew[s];
    } else if (fl & kAppend) {
      if (t.r_state[u] == 2u) t.extra[t.r_reg[u] + t.slot[s]] = make_uint2(v, t.wnew[s]);
      else arcs[off[u] + deg[u] + t.slot[s]] = make_uint2(v, t.wnew[s]);
    }
  }
}

// Whether a validated batch is written: no error, 2m stays below 2^32 (single
// graphs), every rebuilt row's new arcs fit a block's sort, and the arc pool
// and the merge scratch have the room the rebuilt rows need.  Every input is
// final once the row decisions are made, so every block that evaluates it
// agrees.
struct ApplyGate {
  unsigned long long pool_top, pool_cap, scratch_cap;
  long long m2;
  int check_m2;
  const unsigned int* pre_err;  // error bits of checks made before the apply (a group's staging), or null
};

__device__ __forceinline__ bool gate_open(const Ctrl& c, const ApplyGate& g) {
  if (c.err) return false;
  if (g.pre_err && *g.pre_err) return false;
  if (g.check_m2 && g.m2 + c.m2_delta >= (1ll << 32)) return false;
  if (c.max_app > kExtraMax) return false;
  return g.pool_top + c.reloc_need <= g.pool_cap && c.scratch_need <= g.scratch_cap;
}

// The gate of the multi-kernel path: decided here (block 0 publishes it in
// ctrl->apply_go / apply_defer for the kernels after this one and the host),
// and nothing is written if it is closed.
__global__ void k_hash_write(HashApply t, const unsigned long long* __restrict__ off,
                             const uint32_t* __restrict__ deg, uint2* __restrict__ arcs, Ctrl* ctrl,
                             ApplyGate g) {
  pdl_wait();
  const bool go = gate_open(*ctrl, g);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctrl->apply_go = go ? 1u : 0u;
    ctrl->apply_defer = go && ctrl->rebuild_rows ? 1u : 0u;
  }
  if (!go) return;
  hash_write_body(t, off, deg, arcs, ctrl, blockIdx.x * uint64_t(blockDim.x), uint64_t(gridDim.x) * blockDim.x);
}

constexpr int kHRebuildThreads = 256;

// Block per rebuilt row: merge of the live sorted prefix (compacted into
// scratch), the live tail and the row's new arcs (both sorted in shared
// memory) into a new slot of 1.5x the live degree.
__device__ __forceinline__ void hash_rebuild_body(HashApply t, unsigned long long* __restrict__ off, uint32_t* __restrict__ deg,
               uint32_t* __restrict__ cap, uint32_t* __restrict__ srt, uint32_t* __restrict__ ntomb,
               uint2* __restrict__ arcs, uint2* __restrict__ scratch, unsigned long long pool_base,
               unsigned long long pool_cap, unsigned long long scratch_cap, Ctrl* ctrl, uint32_t r0, uint32_t rstep) {
  __shared__ uint2 tail[kTailMax];
  __shared__ uint2 stail[kTailMax];
  __shared__ uint2 sn[kExtraMax];
  __shared__ unsigned long long s_sbase, s_dst;
  __shared__ uint32_t s_nt, s_warp[kHRebuildThreads / 32], s_total;
  const uint32_t nr = ctrl->rows;
  const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
  for (uint32_t r = r0; r < nr; r += rstep) {
    const uint32_t u = t.rows[r];
    if (t.r_state[u] != 2u) continue;
    const uint2* old = arcs + off[u];
    const uint32_t d = deg[u], s = srt[u], nnew = t.r_app[u];
    const uint32_t live = uint32_t((long long)d - ntomb[u] + t.r_live[u]);
    const uint32_t nc = grow_cap(live);
    if (threadIdx.x == 0) {
      s_sbase = atomicAdd(&ctrl->scratch_top, (unsigned long long)s);
      s_dst = pool_base + atomicAdd(&ctrl->pool_top, (unsigned long long)nc);
      s_nt = 0;
      if (s_sbase + s > scratch_cap || s_dst + nc > pool_cap || nnew > kExtraMax)
        atomicOr(&ctrl->err, kErrInternal);
    }
    __syncthreads();
    const unsigned long long sbase = s_sbase, dst = s_dst;
    if (sbase + s > scratch_cap || dst + nc > pool_cap || nnew > kExtraMax) {
      __syncthreads();
      continue;
    }
    uint2* A = scratch + sbase;
    uint32_t L = 0;
    for (uint32_t c0 = 0; c0 < s; c0 += blockDim.x) {
      uint32_t k = c0 + threadIdx.x;
      uint2 a = k < s ? old[k] : make_uint2(0, 0);
      bool lv = k < s && a.y > 0;
      unsigned m = __ballot_sync(0xFFFFFFFFu, lv);
      if (lane == 0) s_warp[wib] = __popc(m);
      __syncthreads();
      if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (uint32_t x = 0; x < blockDim.x / 32; ++x) {
          uint32_t tt = s_warp[x];
          s_warp[x] = run;
          run += tt;
        }
        s_total = run;
      }
      __syncthreads();
      if (lv) A[L + s_warp[wib] + __popc(m & ((1u << lane) - 1u))] = a;
      L += s_total;
      __syncthreads();
    }
    for (uint32_t k = s + threadIdx.x; k < d; k += blockDim.x) {
      uint2 a = old[k];
      if (a.y > 0) tail[atomicAdd(&s_nt, 1u)] = a;
    }
    // new arcs into shared memory, padded to a power of two for a bitonic sort
    uint32_t np2 = 1;
    while (np2 < nnew) np2 <<= 1;
    for (uint32_t k = threadIdx.x; k < np2; k += blockDim.x)
      sn[k] = k < nnew ? t.extra[t.r_reg[u] + k] : make_uint2(0xFFFFFFFFu, 0u);
    __syncthreads();
    const uint32_t nt = s_nt;
    for (uint32_t k = threadIdx.x; k < nt; k += blockDim.x) {
      uint32_t rk = 0;
      for (uint32_t x = 0; x < nt; ++x) rk += tail[x].x < tail[k].x;
      stail[rk] = tail[k];
    }
    for (uint32_t kk = 2; kk <= np2; kk <<= 1)
      for (uint32_t j = kk >> 1; j > 0; j >>= 1) {
        for (uint32_t i = threadIdx.x; i < np2; i += blockDim.x) {
          uint32_t ixj = i ^ j;
          if (ixj > i) {
            bool up = (i & kk) == 0;
            uint2 x = sn[i], y = sn[ixj];
            if ((x.x > y.x) == up) {
              sn[i] = y;
              sn[ixj] = x;
            }
          }
        }
        __syncthreads();
      }
    __syncthreads();
    uint2* out = arcs + dst;
    for (uint32_t k = threadIdx.x; k < L; k += blockDim.x) {
      uint2 a = A[k];
      out[k + count_below(stail, nt, a.x) + count_below(sn, nnew, a.x)] = a;
    }
    for (uint32_t k = threadIdx.x; k < nt; k += blockDim.x) {
      uint2 a = stail[k];
      out[k + count_below(A, L, a.x) + count_below(sn, nnew, a.x)] = a;
    }
    for (uint32_t k = threadIdx.x; k < nnew; k += blockDim.x) {
      uint2 a = sn[k];
      out[k + count_below(A, L, a.x) + count_below(stail, nt, a.x)] = a;
    }
    if (threadIdx.x == 0) {
      if (L + nt + nnew != live) atomicOr(&ctrl->err, kErrInternal);
      off[u] = dst;
      deg[u] = live;
      srt[u] = live;
      cap[u] = nc;
      ntomb[u] = 0;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kHRebuildThreads)
k_hash_rebuild(HashApply t, unsigned long long* __restrict__ off, uint32_t* __restrict__ deg,
               uint32_t* __restrict__ cap, uint32_t* __restrict__ srt, uint32_t* __restrict__ ntomb,
               uint2* __restrict__ arcs, uint2* __restrict__ scratch, unsigned long long pool_base,
               unsigned long long pool_cap, unsigned long long scratch_cap, Ctrl* ctrl) {
  pdl_wait();
  if (!ctrl->apply_go || !ctrl->apply_defer) return;  // closed gate, or no row to rebuild
  hash_rebuild_body(t, off, deg, cap, srt, ntomb, arcs, scratch, pool_base, pool_cap, scratch_cap, ctrl, blockIdx.x, gridDim.x);
}

// Thread per touched row: metadata of kept rows, then reset the scratch.
__device__ __forceinline__ void hash_finish_body(HashApply t, uint32_t* __restrict__ deg, uint32_t* __restrict__ ntomb,
                              Ctrl* ctrl, uint64_t base, uint64_t stride) {
  const uint32_t nr = ctrl->rows;
  for (uint64_t q = base + threadIdx.x; q < nr;
       q += stride) {
    const uint32_t u = t.rows[q];
    if (t.r_state[u] != 2u) {
      deg[u] += t.r_app[u];
      ntomb[u] = uint32_t((long long)ntomb[u] + t.r_tomb[u]);
    }
    t.r_app[u] = 0;
    t.r_tomb[u] = 0;
    t.r_live[u] = 0;
    t.r_state[u] = 0;
    t.r_reg[u] = 0;
  }
}

// need_defer: after the single-block path, which finished the rows itself
// unless it left rebuilds to the multi-block kernels
__global__ void k_hash_finish(HashApply t, uint32_t* __restrict__ deg, uint32_t* __restrict__ ntomb,
                              Ctrl* ctrl, int need_defer) {
  pdl_wait();
  if (!ctrl->apply_go || (need_defer && !ctrl->apply_defer)) return;
  hash_finish_body(t, deg, ntomb, ctrl, blockIdx.x * uint64_t(blockDim.x), uint64_t(gridDim.x) * blockDim.x);
}

// Alg. 7 per pair: K[u] and Sigma[C^{t-1}[u]] change by the net weight.
__device__ __forceinline__ void hash_weights_body(HashApply t, const uint32_t* __restrict__ C, long long* __restrict__ K,
                               long long* __restrict__ Sigma, Ctrl* ctrl, uint64_t base, uint64_t stride) {
  const uint32_t np = ctrl->npairs;
  const uint32_t lane = threadIdx.x & 31u;
  // warp-uniform loop: changes to one community's Sigma are summed in the
  // warp first (a large community takes one update per warp, not per arc)
  for (uint64_t p0 = base + (threadIdx.x & ~31u); p0 < np; p0 += stride) {
    const uint64_t p = p0 + lane;
    long long dl = 0;
    uint32_t c = kEmpty;
    if (p < np) {
      const uint32_t s = t.pairs[p];
      dl = t.delta[s];
      if (dl) {
        const uint32_t u = uint32_t(t.keys[s] >> 32);
        atomicAdd((unsigned long long*)&K[u], (unsigned long long)dl);
        c = C[u];
      }
    }
    long long sum = 0;
    bool first = c != kEmpty;
    for (int k = 0; k < 32; ++k) {
      const uint32_t ck = __shfl_sync(0xFFFFFFFFu, c, k);
      const long long dk = __shfl_sync(0xFFFFFFFFu, dl, k);
      if (c != kEmpty && ck == c) {
        sum += dk;
        if (uint32_t(k) < lane) first = false;
      }
    }
    if (first && sum) atomicAdd((unsigned long long*)&Sigma[c], (unsigned long long)sum);
  }
}

__global__ void k_hash_weights(HashApply t, const uint32_t* __restrict__ C, long long* __restrict__ K,
                               long long* __restrict__ Sigma, Ctrl* ctrl) {
  pdl_wait();
  if (!ctrl->apply_go) return;
  hash_weights_body(t, C, K, Sigma, ctrl, blockIdx.x * uint64_t(blockDim.x), uint64_t(gridDim.x) * blockDim.x);
}

// Reset the per-vertex scratch of the touched rows after a failed validation.
__device__ __forceinline__ void hash_reset_body(HashApply t, Ctrl* ctrl, uint64_t base, uint64_t stride) {
  const uint32_t nr = ctrl->rows;
  for (uint64_t q = base + threadIdx.x; q < nr;
       q += stride) {
    const uint32_t u = t.rows[q];
    t.r_app[u] = 0;
    t.r_tomb[u] = 0;
    t.r_live[u] = 0;
    t.r_state[u] = 0;
    t.r_reg[u] = 0;
  }
}

__global__ void k_hash_reset(HashApply t, Ctrl* ctrl) {
  hash_reset_body(t, ctrl, blockIdx.x * uint64_t(blockDim.x), uint64_t(gridDim.x) * blockDim.x);
}

// Every slot a batch claimed in the pair table is emptied again after its
// last reader, so the table is empty between batches and an apply needs no
// clear of the whole table; the next apply's control block is cleared too.
__device__ __forceinline__ void apply_rest(HashApply t, const Ctrl* ctrl, Ctrl* next, uint64_t base,
                                           uint64_t stride) {
  const uint32_t np = ctrl->npairs;
  for (uint64_t q = base; q < np; q += stride) {
    const uint32_t s = t.pairs[q];
    t.keys[s] = kNoKey;
    t.ndel[s] = 0;
    t.wins[s] = 0;
  }
  if (base < sizeof(Ctrl) / sizeof(unsigned int)) {
    unsigned int* z = reinterpret_cast<unsigned int*>(next);
    for (uint64_t q = base; q < sizeof(Ctrl) / sizeof(unsigned int); q += stride) z[q] = 0u;
  }
}

// Last kernel of the multi-kernel apply: the batch's arcs join the pending
// list of the next update if the batch was written; the table is emptied
// either way.
__global__ void k_apply_tail(const unsigned long long* __restrict__ key, const uint32_t* __restrict__ w,
                             uint64_t na, unsigned long long* __restrict__ pend_key,
                             uint32_t* __restrict__ pend_w, HashApply t, const Ctrl* ctrl, Ctrl* next) {
  pdl_wait();
  const uint64_t base = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x;
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  if (ctrl->apply_go)
    for (uint64_t q = base; q < na; q += stride) {
      pend_key[q] = key[q];
      pend_w[q] = w[q];
    }
  apply_rest(t, ctrl, next, base, stride);
}

// Small batches (at most kSmallApplyEdges edges, one arc per thread) in one
// block: the phases of the hashed apply above -- table insert, pair
// validation, row decisions, then, if the batch is valid and fits, in-place
// writes, K and Sigma, the pending list and the row metadata -- separated by
// block barriers, so that a batch of a few edges costs one launch instead of
// six kernels and three table clears.  The table is the first `t.mask + 1`
// slots of the pair table, cleared here.  Nothing is written if the gate
// (gate_open) is closed: the per-row scratch counters are cleared,
// ctrl->apply_go stays 0 and the host reports the error or redoes the batch.
// Rows to rebuild (rare for small batches) are left to the multi-block
// rebuild, one block per row, and the row metadata kernel after it, which
// are enqueued behind this kernel and run only when it sets
// ctrl->apply_defer.
constexpr uint64_t kSmallApplyEdges = 512;
constexpr int kSmallApplyThreads = 1024;

__global__ void __launch_bounds__(kSmallApplyThreads)
k_apply_small(const dfl_edge* __restrict__ del, const dfl_edge* __restrict__ ins, uint64_t nd, uint64_t ne,
              uint32_t n, KeyFmt f, HashApply t,
              unsigned long long* __restrict__ key, uint32_t* __restrict__ w, const unsigned long long* __restrict__ off,
              uint32_t* __restrict__ deg, const uint32_t* __restrict__ cap, const uint32_t* __restrict__ srt,
              uint32_t* __restrict__ ntomb, uint2* __restrict__ arcs, const uint32_t* __restrict__ C,
              long long* __restrict__ K, long long* __restrict__ Sigma, unsigned long long* __restrict__ pend_key,
              uint32_t* __restrict__ pend_w, ApplyGate g, Ctrl* ctrl, Ctrl* next) {
  pdl_wait();
  __shared__ int s_go;
  const uint64_t nt = blockDim.x;
  hash_insert_body(del, ins, nd, ne, n, f, t, key, w, ctrl, 0, nt);
  __syncthreads();
  hash_pairs_body(t, n, off, deg, srt, arcs, ctrl, 0, nt);
  __syncthreads();
  hash_rows_body(t, deg, cap, srt, ntomb, ctrl, 0, nt);
  __syncthreads();
  if (threadIdx.x == 0) {
    const Ctrl& c = *ctrl;
    const bool go = gate_open(c, g);
    const bool defer = c.rebuild_rows != 0;
    s_go = go ? (defer ? 2 : 1) : 0;
    ctrl->apply_go = go ? 1u : 0u;
    ctrl->apply_defer = go && defer ? 1u : 0u;
  }
  __syncthreads();
  if (!s_go) {
    hash_reset_body(t, ctrl, 0, nt);
  } else {
    hash_write_body(t, off, deg, arcs, ctrl, 0, nt);
    hash_weights_body(t, C, K, Sigma, ctrl, 0, nt);
    for (uint64_t q = threadIdx.x; q < 2 * ne; q += nt) {
      pend_key[q] = key[q];
      pend_w[q] = w[q];
    }
    if (s_go == 1) {  // (rows to rebuild: the rebuild and metadata kernels enqueued behind this one)
      __syncthreads();  // every write has read deg before the metadata changes it
      hash_finish_body(t, deg, ntomb, ctrl, 0, nt);
    }
  }
  __syncthreads();  // the table's last readers are done
  apply_rest(t, ctrl, next, threadIdx.x, nt);
}

int read_ctrl(Handle* h) {
  DFL_CUDA(h, cudaMemcpyAsync(h->hctrl, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
  DFL_CUDA(h, cudaStreamSynchronize(h->stream));
  return DFL_OK;
}

template <typename T>
int grow(Handle* h, T** p, uint64_t need, uint64_t* cap_out, uint64_t cap_now, bool keep = false,
         uint64_t keep_items = 0) {
  if (need <= cap_now) return DFL_OK;
  uint64_t want = need + need / 2 + 256;
  T* q = nullptr;
  DFL_CUDA(h, dev_malloc(&q, sizeof(T) * want));
  if (keep && *p && keep_items)
    DFL_CUDA(h, cudaMemcpyAsync(q, *p, sizeof(T) * keep_items, cudaMemcpyDeviceToDevice, h->stream));
  if (*p) {
    DFL_CUDA(h, cudaStreamSynchronize(h->stream));
    cudaFree(*p);
  }
  *p = q;
  if (cap_out) *cap_out = want;
  return DFL_OK;
}

int ensure_batch_scratch(Handle* h, uint64_t na) {
  if (na <= h->b_cap) return DFL_OK;
  uint64_t want = na + na / 2 + 256, c = 0;
  DFL_TRY(grow(h, &h->b_key, want, &c, 0));
  DFL_TRY(grow(h, &h->b_key2, want, &c, 0));
  DFL_TRY(grow(h, &h->b_w, want, &c, 0));
  DFL_TRY(grow(h, &h->b_w2, want, &c, 0));
  DFL_TRY(grow(h, &h->b_pos, want, &c, 0));
  DFL_TRY(grow(h, &h->b_wnew, want, &c, 0));
  DFL_TRY(grow(h, &h->b_flag, want, &c, 0));
  DFL_TRY(grow(h, &h->b_delta, want, &c, 0));
  DFL_TRY(grow(h, &h->b_rowlist, want, &c, 0));
  DFL_TRY(grow(h, &h->b_newdeg, want, &c, 0));
  DFL_TRY(grow(h, &h->b_newtomb, want, &c, 0));
  DFL_TRY(grow(h, &h->b_cum, want, &c, 0));
  DFL_TRY(grow(h, &h->b_rebuild, want, &c, 0));
  h->b_cap = c;
  return DFL_OK;
}

KeyFmt key_fmt(const Handle* h) {
  KeyFmt f;
  f.b = h->key_shift;
  f.vmask = (1ull << h->key_shift) - 1;
  return f;
}



int ensure_hash_buffers(Handle* h, uint64_t na) {
  uint64_t cap = 1024;
  while (cap < 2 * na) cap <<= 1;
  if (cap > h->h_cap) {
    cudaStreamSynchronize(h->stream);
    // freed and cleared together, so that an allocation failing below leaves
    // no member pointing at freed memory (destroy and the next growth free
    // every member)
    void** old[] = {(void**)&h->h_keys, (void**)&h->h_ndel, (void**)&h->h_wdel, (void**)&h->h_wins,
                    (void**)&h->h_slot, (void**)&h->h_wnew, (void**)&h->h_flag, (void**)&h->h_delta,
                    (void**)&h->h_pairs};
    for (void** q : old) {
      cudaFree(*q);
      *q = nullptr;
    }
    h->h_cap = 0;
    DFL_CUDA(h, dev_malloc(&h->h_keys, sizeof(unsigned long long) * cap));
    DFL_CUDA(h, dev_malloc(&h->h_ndel, sizeof(uint32_t) * cap));
    DFL_CUDA(h, dev_malloc(&h->h_wdel, sizeof(uint32_t) * cap));
    DFL_CUDA(h, dev_malloc(&h->h_wins, sizeof(unsigned long long) * cap));
    DFL_CUDA(h, dev_malloc(&h->h_slot, sizeof(uint32_t) * cap));
    DFL_CUDA(h, dev_malloc(&h->h_wnew, sizeof(uint32_t) * cap));
    DFL_CUDA(h, dev_malloc(&h->h_flag, sizeof(uint32_t) * cap));
    DFL_CUDA(h, dev_malloc(&h->h_delta, sizeof(long long) * cap));
    DFL_CUDA(h, dev_malloc(&h->h_pairs, sizeof(uint32_t) * cap));
    // empty; every apply empties the slots it claimed again
    DFL_CUDA(h, cudaMemsetAsync(h->h_keys, 0xFF, sizeof(unsigned long long) * cap, h->stream));
    DFL_CUDA(h, cudaMemsetAsync(h->h_ndel, 0, sizeof(uint32_t) * cap, h->stream));
    DFL_CUDA(h, cudaMemsetAsync(h->h_wins, 0, sizeof(unsigned long long) * cap, h->stream));
    h->h_cap = cap;
  }
  if (!h->r_app || !h->r_tomb || !h->r_live || !h->r_state || !h->r_reg) {
    // all five or none: what an earlier failed allocation left is freed first
    void** rs[] = {(void**)&h->r_app, (void**)&h->r_tomb, (void**)&h->r_live, (void**)&h->r_state,
                   (void**)&h->r_reg};
    for (void** q : rs) {
      cudaFree(*q);
      *q = nullptr;
    }
    const uint64_t n = h->n ? h->n : 1;
    DFL_CUDA(h, dev_malloc(&h->r_app, sizeof(uint32_t) * n));
    DFL_CUDA(h, dev_malloc(&h->r_tomb, sizeof(int) * n));
    DFL_CUDA(h, dev_malloc(&h->r_live, sizeof(int) * n));
    DFL_CUDA(h, dev_malloc(&h->r_state, sizeof(uint32_t) * n));
    DFL_CUDA(h, dev_malloc(&h->r_reg, sizeof(uint32_t) * n));
    DFL_CUDA(h, cudaMemsetAsync(h->r_app, 0, sizeof(uint32_t) * n, h->stream));
    DFL_CUDA(h, cudaMemsetAsync(h->r_tomb, 0, sizeof(int) * n, h->stream));
    DFL_CUDA(h, cudaMemsetAsync(h->r_live, 0, sizeof(int) * n, h->stream));
    DFL_CUDA(h, cudaMemsetAsync(h->r_state, 0, sizeof(uint32_t) * n, h->stream));
    DFL_CUDA(h, cudaMemsetAsync(h->r_reg, 0, sizeof(uint32_t) * n, h->stream));
  }
  if (na > h->h_rows_cap) {
    cudaStreamSynchronize(h->stream);
    cudaFree(h->h_rows);
    cudaFree(h->h_extra);
    h->h_rows = nullptr;
    h->h_extra = nullptr;
    h->h_rows_cap = 0;
    uint64_t want = na + na / 2 + 256;
    DFL_CUDA(h, dev_malloc(&h->h_rows, sizeof(uint32_t) * want));
    DFL_CUDA(h, dev_malloc(&h->h_extra, sizeof(uint2) * want));
    h->h_rows_cap = want;
  }
  return DFL_OK;
}

HashApply hash_args(const Handle* h) {
  HashApply t;
  t.keys = h->h_keys;
  t.ndel = h->h_ndel;
  t.wdel = h->h_wdel;
  t.wins = h->h_wins;
  t.slot = h->h_slot;
  t.wnew = h->h_wnew;
  t.flag = h->h_flag;
  t.delta = h->h_delta;
  t.pairs = h->h_pairs;
  t.mask = h->h_cap - 1;
  t.r_app = h->r_app;
  t.r_tomb = h->r_tomb;
  t.r_live = h->r_live;
  t.r_state = h->r_state;
  t.r_reg = h->r_reg;
  t.rows = h->h_rows;
  t.extra = h->h_extra;
  return t;
}


}  // namespace

// Batch apply (Section 3.4 and Alg. 7): validate, then change the graph, K,
// Sigma and 2m, and append the batch to the pending list.
namespace {

int hash_reset(Handle* h, const HashApply& t, Ctrl* c) {
  LaunchScope ls(h, DFL_PROF_APPLY);
  k_hash_reset<<<grid_for(h->h_rows_cap, 256), 256, 0, h->stream>>>(t, c);
  DFL_TRY(check_launch(h, "hash reset"));
  DFL_CUDA(h, cudaStreamSynchronize(h->stream));
  return DFL_OK;
}

ApplyGate apply_gate(const Handle* h, const unsigned int* pre_err) {
  return ApplyGate{h->pool_top, h->pool_cap, h->scratch_cap, h->m2, h->ngraphs ? 0 : 1, pre_err};
}

// Enqueue the hashed apply of a batch in device memory (nd deletions at
// del, then ne - nd insertions at ins): validation, the gate, and -- if it opens -- the
// writes, K and Sigma (Alg. 7), the row metadata and the pending list, all
// on the handle's stream with no host wait.  Its control block is h->actrl.
int enqueue_hashed(Handle* h, const dfl_edge* del, const dfl_edge* ins, uint64_t nd, uint64_t ne,
                   const unsigned int* pre_err = nullptr) {
  const uint64_t na = 2 * ne;
  // the pending list's room first: a failed growth leaves everything as it was
  if (h->pend_count + na > h->pend_cap) {
    uint64_t c2 = 0, c3 = 0, need = h->pend_count + na;
    DFL_TRY(grow(h, &h->pend_key, need, &c2, h->pend_cap, true, h->pend_count));
    DFL_TRY(grow(h, &h->pend_w, need, &c3, h->pend_cap, true, h->pend_count));
    h->pend_cap = c2 < c3 ? c2 : c3;
  }
  // this apply's control block was cleared by the previous apply (or at
  // creation); it clears the other one for the next
  const int par = h->apar;
  Ctrl* c = h->actrl + par;
  Ctrl* next = h->actrl + (par ^ 1);
  const ApplyGate gate = apply_gate(h, pre_err);
  const KeyFmt f = key_fmt(h);
  HashApply t = hash_args(h);
  const bool small = ne <= kSmallApplyEdges;
  if (small) {
    uint64_t sc = 64;
    while (sc < 2 * na) sc <<= 1;
    t.mask = (sc < h->h_cap ? sc : h->h_cap) - 1;
    LaunchScope ls(h, DFL_PROF_APPLY);
    launch_pdl(k_apply_small, 1, kSmallApplyThreads, 0, h->stream, del, ins, nd, ne, h->n, f, t, h->b_key, h->b_w, h->off, h->deg, h->cap, h->srt, h->ntomb, h->arcs,
        h->C, h->K, h->Sigma, h->pend_key + h->pend_count, h->pend_w + h->pend_count, gate, c, next);
    DFL_TRY(check_launch(h, "small batch apply"));
  } else {
    {
      LaunchScope ls(h, DFL_PROF_APPLY);
      launch_pdl(k_hash_insert, grid_for(ne, 256), 256, 0, h->stream, del, ins, nd, ne, h->n, f, t,
                 h->b_key, h->b_w, c);
      DFL_TRY(check_launch(h, "hash insert"));
    }
    {
      LaunchScope ls(h, DFL_PROF_APPLY);
      launch_pdl(k_hash_pairs, grid_for(na, 256), 256, 0, h->stream, t, h->n, h->off, h->deg, h->srt,
                 h->arcs, c);
      DFL_TRY(check_launch(h, "hash pairs"));
    }
    {
      LaunchScope ls(h, DFL_PROF_APPLY);
      launch_pdl(k_hash_rows, grid_for(na, 256), 256, 0, h->stream, t, h->deg, h->cap, h->srt, h->ntomb, c);
      DFL_TRY(check_launch(h, "hash rows"));
    }
    {
      LaunchScope ls(h, DFL_PROF_APPLY);
      launch_pdl(k_hash_write, grid_for(na, 256), 256, 0, h->stream, t, h->off, h->deg, h->arcs, c, gate);
      DFL_TRY(check_launch(h, "hash write"));
    }
  }
  // (the touched rows are at most the batch's arcs)
  {
    LaunchScope ls(h, DFL_PROF_APPLY);
    launch_pdl(k_hash_rebuild, grid_for(na, 1, 152 * 4), kHRebuildThreads, 0, h->stream, t, h->off, h->deg, h->cap, h->srt, h->ntomb, h->arcs, h->scratch, h->pool_top, h->pool_cap,
        h->scratch_cap, c);
    DFL_TRY(check_launch(h, "hash rebuild"));
  }
  if (!small) {
    LaunchScope ls(h, DFL_PROF_APPLY);
    launch_pdl(k_hash_weights, grid_for(na, 256), 256, 0, h->stream, t, h->C, h->K, h->Sigma, c);
    DFL_TRY(check_launch(h, "hash weights"));
  }
  {
    LaunchScope ls(h, DFL_PROF_APPLY);
    launch_pdl(k_hash_finish, grid_for(na, 256), 256, 0, h->stream, t, h->deg, h->ntomb, c,
               small ? 1 : 0);
    DFL_TRY(check_launch(h, "hash finish"));
  }
  if (!small) {
    LaunchScope ls(h, DFL_PROF_APPLY);
    launch_pdl(k_apply_tail, grid_for(na, 256), 256, 0, h->stream, h->b_key, h->b_w, na,
               h->pend_key + h->pend_count, h->pend_w + h->pend_count, t, c, next);
    DFL_TRY(check_launch(h, "pending list"));
  }
  h->apar = par ^ 1;
  h->papply.active = true;
  h->papply.par = par;
  h->papply.small = small;
  h->papply.na = na;
  h->papply.rc = DFL_OK;
  return DFL_OK;
}

// Enqueue the batch's apply.  Device batches are read in place (the call
// waits for the apply's kernels before it returns); host batches are copied
// into b_edges first.  The buffers grow before anything is enqueued, so a
// failure there leaves nothing enqueued.  *ddel / *dins: the device arrays
// the kernels read.
int begin_hashed(Handle* h, const dfl_edge* del, uint64_t nd, const dfl_edge* ins, uint64_t ni,
                 int mem_kind, const dfl_edge** ddel, const dfl_edge** dins,
                 const unsigned int* pre_err = nullptr) {
  const uint64_t ne = nd + ni;
  const uint64_t na = 2 * ne;
  if (mem_kind != DFL_MEM_DEVICE && ne > h->b_edges_cap) {
    uint64_t cap = 0;
    DFL_TRY(grow(h, &h->b_edges, ne, &cap, h->b_edges_cap));
    h->b_edges_cap = cap;
  }
  DFL_TRY(ensure_batch_scratch(h, na));
  DFL_TRY(ensure_hash_buffers(h, na));
  if (mem_kind == DFL_MEM_DEVICE) {
    *ddel = del;
    *dins = ins;
  } else {
    if (nd) DFL_CUDA(h, cudaMemcpyAsync(h->b_edges, del, sizeof(dfl_edge) * nd, cudaMemcpyHostToDevice, h->stream));
    if (ni) DFL_CUDA(h, cudaMemcpyAsync(h->b_edges + nd, ins, sizeof(dfl_edge) * ni, cudaMemcpyHostToDevice, h->stream));
    *ddel = h->b_edges;
    *dins = h->b_edges + nd;
  }
  return enqueue_hashed(h, *ddel, *dins, nd, ne, pre_err);
}

}  // namespace

int copy_apply_ctrl(Handle* h) {
  const int p = h->papply.par;
  DFL_CUDA(h, cudaMemcpyAsync(h->hactrl + p, h->actrl + p, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
  return DFL_OK;
}

int settle_apply(Handle* h) {
  if (!h->papply.active) return h->papply.rc;
  h->papply.active = false;
  const int par = h->papply.par;
  const Ctrl c = h->hactrl[par];
  const uint64_t na = h->papply.na;
  int rc = DFL_OK;
  if (c.apply_go) {
    h->pend_count += na;
    h->m2 += c.m2_delta;
    h->pool_top += c.reloc_need;
    h->num_arcs = uint64_t((long long)h->num_arcs + c.arc_delta);
    if (c.max_deg > h->max_deg) h->max_deg = c.max_deg;
    if (c.err) rc = set_error(h, DFL_ERR_CUDA, "internal error in batch apply");
    h->papply.rc = rc;
    return rc;
  }
  // nothing was written; the per-row scratch counters are cleared again
  rc = hash_reset(h, hash_args(h), h->actrl + par);
  if (!rc) {
    if (c.err & kErrInvalid) rc = set_error(h, DFL_ERR_INVALID, "invalid edge in batch");
    else if (c.err & kErrNotFound) rc = set_error(h, DFL_ERR_NOT_FOUND, "deleted edge not found");
    else if (c.err & kErrOverflow) rc = set_error(h, DFL_ERR_OVERFLOW, "edge weight overflow");
    else if (c.err) rc = set_error(h, DFL_ERR_CUDA, "internal error in batch validation");
    else if (!h->ngraphs && h->m2 + c.m2_delta >= (1ll << 32))
      rc = set_error(h, DFL_ERR_OVERFLOW, "2m would reach 2^32");
    else if (c.max_app > kExtraMax)
      rc = kApplyRetrySorted;  // a rebuilt row gains too many arcs to sort in shared memory
  }
  if (!rc) {
    // more room in the arc pool or the merge scratch: grown before the batch
    // is enqueued again (a grown buffer keeps its contents)
    if (h->pool_top + c.reloc_need > h->pool_cap) {
      uint64_t c2 = 0;
      uint64_t need = h->pool_top + c.reloc_need;
      need = need + need / 4 + 1024;
      rc = grow(h, &h->arcs, need, &c2, h->pool_cap, true, h->pool_top);
      if (!rc) h->pool_cap = c2;
    }
    if (!rc && c.scratch_need > h->scratch_cap) {
      uint64_t c2 = 0;
      rc = grow(h, &h->scratch, c.scratch_need, &c2, h->scratch_cap);
      if (!rc) h->scratch_cap = c2;
    }
    if (!rc) rc = kApplyRetryGrown;
  }
  h->papply.rc = rc;
  return rc;
}

uint64_t live_arcs_bound(const Handle* h) {
  return h->num_arcs + (h->papply.active ? h->papply.na : 0);
}

uint64_t pool_top_bound(const Handle* h) { return h->papply.active ? h->pool_cap : h->pool_top; }

uint32_t max_deg_bound(const Handle* h) {
  if (!h->papply.active) return h->max_deg;
  // a row gains at most one arc per edge of the batch
  const uint64_t b = uint64_t(h->max_deg) + h->papply.na / 2;
  return b < 0xFFFFFFFFull ? uint32_t(b) : 0xFFFFFFFFu;
}

int apply_batch_begin(Handle* h, const dfl_edge* del, uint64_t nd, const dfl_edge* ins, uint64_t ni,
                      int mem_kind) {
  if (!h->have_communities) return set_error(h, DFL_ERR_STATE, "dfl_apply_batch before dfl_static");
  if (nd + ni == 0) return DFL_OK;
  const dfl_edge *ddel = nullptr, *dins = nullptr;
  return begin_hashed(h, del, nd, ins, ni, mem_kind, &ddel, &dins);
}

int apply_batch(Handle* h, const dfl_edge* del, uint64_t nd, const dfl_edge* ins, uint64_t ni,
                int mem_kind) {
  if (!h->have_communities) return set_error(h, DFL_ERR_STATE, "dfl_apply_batch before dfl_static");
  if (nd + ni == 0) return DFL_OK;
  const dfl_edge *ddel = nullptr, *dins = nullptr;
  int rc = begin_hashed(h, del, nd, ins, ni, mem_kind, &ddel, &dins);
  for (int attempt = 0; !rc; ++attempt) {
    // one host wait, after the whole sequence
    rc = copy_apply_ctrl(h);
    if (!rc && cudaStreamSynchronize(h->stream) != cudaSuccess) rc = set_error(h, DFL_ERR_CUDA, "batch apply");
    if (rc) {
      h->papply.active = false;
      return rc;
    }
    rc = settle_apply(h);
    if (rc == kApplyRetryGrown && attempt == 0) {
      rc = enqueue_hashed(h, ddel, dins, nd, nd + ni);
      continue;
    }
    if (rc == kApplyRetrySorted) return apply_batch_sorted(h, del, nd, ins, ni, mem_kind);
    if (rc > 0) return set_error(h, DFL_ERR_CUDA, "batch apply did not settle");
    return rc;
  }
  return rc;
}

int group_apply(Handle* h, const dfl_edge* sd, uint64_t nd, const dfl_edge* si, uint64_t ni) {
  if (nd + ni == 0) return DFL_OK;
  const unsigned int* staging = &h->ctrl->err;  // the staging checks' bits, queued before this
  const dfl_edge *ddel = nullptr, *dins = nullptr;
  int rc = begin_hashed(h, sd, nd, si, ni, DFL_MEM_DEVICE, &ddel, &dins, staging);
  for (int attempt = 0; !rc; ++attempt) {
    // every graph's 2m from the new K, then one wait for the staging checks,
    // the apply's control block and the sums (the control blocks are adjacent)
    rc = group_m2_enqueue(h);
    if (!rc) {
      const size_t blocks = size_t(2 + h->papply.par);
      if (cudaMemcpyAsync(h->hctrl, h->ctrl, blocks * sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream) !=
              cudaSuccess ||
          cudaStreamSynchronize(h->stream) != cudaSuccess)
        rc = set_error(h, DFL_ERR_CUDA, "group batch apply");
    }
    if (rc) {
      h->papply.active = false;
      return rc;
    }
    const unsigned int err = h->hctrl->err;
    const int arc = settle_apply(h);  // (a closed gate: the row counters are cleared)
    if (err & kErrInvalid) return set_error(h, DFL_ERR_INVALID, "vertex id >= the graph's size");
    if (err & kErrOverflow) return set_error(h, DFL_ERR_OVERFLOW, "a graph's 2m could reach 2^32");
    rc = arc;
    if (rc == kApplyRetryGrown && attempt == 0) {
      rc = enqueue_hashed(h, ddel, dins, nd, nd + ni, staging);
      continue;
    }
    if (rc == kApplyRetrySorted) {
      rc = apply_batch_sorted(h, sd, nd, si, ni, DFL_MEM_DEVICE);
      return rc ? rc : group_m2(h);
    }
    if (rc > 0) return set_error(h, DFL_ERR_CUDA, "batch apply did not settle");
    return rc ? rc : group_m2_take(h);
  }
  return rc;
}

// Sort-based batch apply: used when a rebuilt row receives more new arcs
// in one batch than the hashed path sorts in shared memory.
int apply_batch_sorted(Handle* h, const dfl_edge* del, uint64_t nd, const dfl_edge* ins, uint64_t ni,
                       int mem_kind) {
  const uint64_t ne = nd + ni;
  if (ne == 0) return DFL_OK;
  const uint64_t na = 2 * ne;
  if (ne > h->b_edges_cap) {
    uint64_t cap = 0;
    DFL_TRY(grow(h, &h->b_edges, ne, &cap, h->b_edges_cap));
    h->b_edges_cap = cap;
  }
  DFL_TRY(ensure_batch_scratch(h, na));
  cudaMemcpyKind kind = mem_kind == DFL_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (nd) DFL_CUDA(h, cudaMemcpyAsync(h->b_edges, del, sizeof(dfl_edge) * nd, kind, h->stream));
  if (ni) DFL_CUDA(h, cudaMemcpyAsync(h->b_edges + nd, ins, sizeof(dfl_edge) * ni, kind, h->stream));
  DFL_CUDA(h, cudaMemsetAsync(h->ctrl, 0, sizeof(Ctrl), h->stream));
  const KeyFmt f = key_fmt(h);
  {
    LaunchScope ls(h, DFL_PROF_APPLY);
    k_expand<<<grid_for(ne, 256), 256, 0, h->stream>>>(h->b_edges, nd, ne, h->n, f, h->b_key, h->b_w,
                                                       h->ctrl);
    DFL_TRY(check_launch(h, "expand"));
  }
  DFL_TRY(sort_pairs(h, h->b_key, h->b_w, h->b_key2, h->b_w2, na, h->key_bits));
  {
    LaunchScope ls(h, DFL_PROF_APPLY);
    k_runs<<<grid_for(na, 256), 256, 0, h->stream>>>(h->b_key, h->b_w, na, f, h->n, h->off, h->deg,
                                                     h->srt, h->arcs, h->b_pos, h->b_wnew, h->b_flag,
                                                     h->b_delta, h->b_rowlist, h->ctrl);
    DFL_TRY(check_launch(h, "runs"));
  }
  {
    LaunchScope ls(h, DFL_PROF_APPLY);
    k_rows<<<grid_for(na, 256), 256, 0, h->stream>>>(h->b_key, na, f, h->b_rowlist, h->deg, h->cap,
                                                     h->srt, h->ntomb, h->b_pos, h->b_flag, h->b_cum,
                                                     h->b_newdeg, h->b_newtomb, h->b_rebuild, h->ctrl);
    DFL_TRY(check_launch(h, "rows"));
  }
  DFL_TRY(read_ctrl(h));
  const Ctrl c = *h->hctrl;
  if (c.err & kErrInvalid) return set_error(h, DFL_ERR_INVALID, "invalid edge in batch");
  if (c.err & kErrNotFound) return set_error(h, DFL_ERR_NOT_FOUND, "deleted edge not found");
  if (c.err & kErrOverflow) return set_error(h, DFL_ERR_OVERFLOW, "edge weight overflow");
  if (c.err) return set_error(h, DFL_ERR_CUDA, "internal error in batch validation");
  if (!h->ngraphs && h->m2 + c.m2_delta >= (1ll << 32))
    return set_error(h, DFL_ERR_OVERFLOW, "2m would reach 2^32");
  // every buffer the writes need, before the first write: a failed
  // allocation (DFL_ERR_NOMEM) leaves the graph, K, Sigma and the pending
  // list as they were (a grown buffer keeps its contents)
  {
    int grc = DFL_OK;
    if (h->pool_top + c.reloc_need > h->pool_cap) {
      uint64_t c2 = 0;
      uint64_t need = h->pool_top + c.reloc_need;
      need = need + need / 4 + 1024;
      grc = grow(h, &h->arcs, need, &c2, h->pool_cap, true, h->pool_top);
      if (!grc) h->pool_cap = c2;
    }
    if (!grc && c.scratch_need > h->scratch_cap) {
      uint64_t c2 = 0;
      grc = grow(h, &h->scratch, c.scratch_need, &c2, h->scratch_cap);
      if (!grc) h->scratch_cap = c2;
    }
    if (!grc && h->pend_count + na > h->pend_cap) {
      uint64_t c2 = 0, c3 = 0, need = h->pend_count + na;
      grc = grow(h, &h->pend_key, need, &c2, h->pend_cap, true, h->pend_count);
      if (!grc) grc = grow(h, &h->pend_w, need, &c3, h->pend_cap, true, h->pend_count);
      if (!grc) h->pend_cap = c2 < c3 ? c2 : c3;
    }
    if (grc) {
      return grc;
    }
  }
  // --- mutation starts here ---
  {
    LaunchScope ls(h, DFL_PROF_APPLY);
    k_write<<<grid_for(na, 256), 256, 0, h->stream>>>(h->b_key, na, f, h->off, h->deg, h->arcs, h->b_pos,
                                                      h->b_wnew, h->b_flag);
    DFL_TRY(check_launch(h, "write"));
  }
  if (c.rebuild_rows) {
    LaunchScope ls(h, DFL_PROF_APPLY);
    k_rebuild<<<grid_for(c.rebuild_rows, 1, 152 * 8), kRebuildThreads, 0, h->stream>>>(
        h->b_key, na, f, h->b_rebuild, h->off, h->deg, h->cap, h->srt, h->ntomb, h->arcs, h->b_pos,
        h->b_wnew, h->b_flag, h->b_cum, h->b_newdeg, h->scratch, h->pool_top, h->pool_cap,
        h->scratch_cap, h->ctrl);
    DFL_TRY(check_launch(h, "rebuild"));
  }
  {
    LaunchScope ls(h, DFL_PROF_APPLY);
    k_finish<<<grid_for(c.rows, 256), 256, 0, h->stream>>>(h->b_key, f, h->b_rowlist, h->b_flag,
                                                           h->b_newdeg, h->b_newtomb, h->deg,
                                                           h->ntomb, h->ctrl);
    DFL_TRY(check_launch(h, "finish"));
  }
  {
    LaunchScope ls(h, DFL_PROF_APPLY);
    k_update_weights<<<grid_for(na, 256), 256, 0, h->stream>>>(h->b_key, na, f, h->b_flag,
                                                               h->b_delta, h->C, h->K, h->Sigma);
    DFL_TRY(check_launch(h, "update weights"));
  }
  // pending arcs for the next dfl_update
  DFL_CUDA(h, cudaMemcpyAsync(h->pend_key + h->pend_count, h->b_key, sizeof(unsigned long long) * na,
                              cudaMemcpyDeviceToDevice, h->stream));
  DFL_CUDA(h, cudaMemcpyAsync(h->pend_w + h->pend_count, h->b_w, sizeof(uint32_t) * na,
                              cudaMemcpyDeviceToDevice, h->stream));
  h->pend_count += na;
  h->m2 += c.m2_delta;
  h->pool_top += c.reloc_need;
  h->num_arcs = uint64_t((long long)h->num_arcs + c.arc_delta);
  if (c.max_deg > h->max_deg) h->max_deg = c.max_deg;
  return DFL_OK;
}

// Initial frontier into list buffer 0 (and fbits[0]); `all` when every
// vertex is affected; `use_range` when the first pass is limited to rbits.
int mark(Handle* h, int mode, bool* all, bool* use_range, uint64_t* initial) {
  const uint32_t n = h->n;
  const uint32_t k = h->opt.substeps;
  make_segs(h, k);
  {
    // (a DF update's first pass also tracks the vertices it processed)
    LaunchScope ls(h, DFL_PROF_MARK);
    uint32_t* ever = mode == DFL_DF ? h->ever : nullptr;
    launch_pdl(k_mark_clear, grid_for(h->words, 256, 152 * 4), 256, 0, h->stream, h->ctrl, h->fbits[0],
               h->fbits[1], ever, h->words);
    DFL_TRY(check_launch(h, "mark clear"));
    h->ever_clear = ever != nullptr;
  }
  *all = false;
  *use_range = false;
  const KeyFmt f = key_fmt(h);
  if (mode == DFL_ND) {
    *all = true;
    DFL_TRY(lists_all(h, n, h->deg, 0, k));
    *initial = n;
    return DFL_OK;
  }
  if (mode == DFL_DF) {
    // a batch enqueued just before (and not yet settled) is marked if its
    // apply's gate opened; its arcs follow the pending list's
    const bool pending = h->papply.active;
    const uint64_t np = h->pend_count + (pending ? h->papply.na : 0);
    if (np) {
      LaunchScope ls(h, DFL_PROF_MARK);
      launch_pdl(k_mark_df, grid_for(np, 256), 256, 0, h->stream, h->pend_key, np, f, h->C, h->deg,
                 h->fbits[0], h->lists[0], h->segs, h->ctrl, k,
                 pending ? &h->actrl[h->papply.par].apply_go : nullptr);
      DFL_TRY(check_launch(h, "mark df"));
    }
    *initial = ~0ull;  // counted from the frontier lists when local-moving starts
    return DFL_OK;
  }
  if (mode != DFL_DS) return set_error(h, DFL_ERR_INVALID, "unknown mode");
  // Delta-screening
  const uint64_t na = h->pend_count;
  DFL_CUDA(h, cudaMemsetAsync(h->dsV, 0, sizeof(uint32_t) * h->words, h->stream));
  DFL_CUDA(h, cudaMemsetAsync(h->dsE, 0, sizeof(uint32_t) * h->words, h->stream));
  DFL_CUDA(h, cudaMemsetAsync(h->dsC, 0, sizeof(uint32_t) * h->words, h->stream));
  if (na) {
    DFL_TRY(ensure_batch_scratch(h, na));
    {
      LaunchScope ls(h, DFL_PROF_MARK);
      k_ds_del<<<grid_for(na, 256), 256, 0, h->stream>>>(h->pend_key, na, f, h->C, h->dsV, h->dsE,
                                                         h->dsC);
      DFL_TRY(check_launch(h, "ds del"));
    }
    {
      LaunchScope ls(h, DFL_PROF_MARK);
      k_ds_keys<<<grid_for(na, 256), 256, 0, h->stream>>>(h->pend_key, h->pend_w, na, f, h->C,
                                                          h->b_key, h->b_w, h->ctrl);
      DFL_TRY(check_launch(h, "ds keys"));
    }
    DFL_TRY(read_ctrl(h));
    uint64_t nk = h->hctrl->red_a;
    if (nk) {
      DFL_TRY(sort_pairs(h, h->b_key, h->b_w, h->b_key2, h->b_w2, nk, 32 + h->key_shift));
      LaunchScope ls(h, DFL_PROF_MARK);
      k_ds_best<<<grid_for(nk, 256), 256, 0, h->stream>>>(h->b_key, h->b_w, nk, h->m2, h->ngraphs,
                                                          h->d_goff0, h->d_gm2, h->K, h->Sigma,
                                                          h->dsV, h->dsE, h->dsC);
      DFL_TRY(check_launch(h, "ds best"));
    }
    {
      LaunchScope ls(h, DFL_PROF_MARK);
      k_ds_expand<<<grid_for(uint64_t(h->words) * 32, 256), 256, 0, h->stream>>>(
          h->dsE, h->words, n, base_view(h), h->dsV);
      DFL_TRY(check_launch(h, "ds expand"));
    }
    {
      LaunchScope ls(h, DFL_PROF_MARK);
      k_ds_comm<<<grid_for(n, 256), 256, 0, h->stream>>>(n, h->C, h->dsC, h->dsV);
      DFL_TRY(check_launch(h, "ds comm"));
    }
  }
  DFL_CUDA(h, cudaMemcpyAsync(h->rbits, h->dsV, sizeof(uint32_t) * h->words,
                              cudaMemcpyDeviceToDevice, h->stream));
  DFL_TRY(lists_from_bits(h, h->dsV, n, h->deg, 0, k));
  *use_range = true;
  int rc = DFL_OK;
  *initial = popcount_bits(h, h->dsV, h->words, &rc);
  return rc;
}

}  // namespace dfl
