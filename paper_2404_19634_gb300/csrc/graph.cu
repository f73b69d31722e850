// Graph storage: input validation, slack CSR build, weighted degrees,
// modularity (Eq. 1) and CSR export.
#include <algorithm>

#include "common.cuh"

namespace dfl {

namespace {

// Capacity of a row of degree d in the slack CSR: 25% headroom plus eight
// slots (so low-degree rows absorb a few insertions before a rebuild),
// rounded up to an even count so every row starts 16-byte aligned.
__host__ __device__ inline uint32_t slack_cap(uint32_t d) {
  uint64_t c = uint64_t(d) + d / 4 + 8;
  c = (c + 1) & ~uint64_t(1);
  return c > 0xFFFFFFFEull ? 0xFFFFFFFEu : uint32_t(c);
}

// Warp per row: checks of Section 3's graph (undirected: both arcs with equal
// weights), plus sorted rows, no self-loops, no duplicates, weights > 0.
__global__ void k_validate(uint32_t n, const unsigned long long* __restrict__ off,
                           const uint32_t* __restrict__ idx, const uint32_t* __restrict__ w,
                           uint64_t nnz, Ctrl* ctrl) {
  const uint32_t lane = threadIdx.x & 31u;
  uint64_t warp = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) >> 5;
  uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  if (warp == 0 && lane == 0 && (off[0] != 0 || off[n] != nnz)) atomicOr(&ctrl->err, kErrInvalid);
  unsigned long long wsum = 0;
  uint32_t dmax = 0;
  for (uint64_t i = warp; i < n; i += nwarps) {
    unsigned long long a = off[i], b = off[i + 1];
    if (b < a || b > nnz) {
      if (lane == 0) atomicOr(&ctrl->err, kErrInvalid);
      continue;
    }
    unsigned long long rd = b - a;
    dmax = max(dmax, rd > 0xFFFFFFFFull ? 0xFFFFFFFFu : uint32_t(rd));
    bool bad = false;
    for (unsigned long long k = a + lane; k < b; k += 32) {
      uint32_t j = idx[k], wt = w[k];
      wsum += wt;
      if (j >= n || j == uint32_t(i) || wt == 0) { bad = true; continue; }
      if (k > a && idx[k - 1] >= j) bad = true;
      // symmetric arc (j, i) with the same weight: binary search in row j
      unsigned long long lo = off[j], hi = off[j + 1];
      if (hi < lo || hi > nnz) { bad = true; continue; }
      while (lo < hi) {
        unsigned long long mid = (lo + hi) >> 1;
        if (idx[mid] < uint32_t(i)) lo = mid + 1;
        else hi = mid;
      }
      if (lo >= off[j + 1] || idx[lo] != uint32_t(i) || w[lo] != wt) bad = true;
    }
    if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) atomicOr(&ctrl->err, kErrInvalid);
  }
  for (int o = 16; o; o >>= 1) wsum += __shfl_xor_sync(0xFFFFFFFFu, wsum, o);
  if (lane == 0) {
    if (wsum) atomicAdd(&ctrl->red_a, wsum);
    atomicMax(&ctrl->max_deg, dmax);
  }
}

__global__ void k_caps(uint32_t n, const unsigned long long* __restrict__ off_in,
                       uint32_t* __restrict__ deg, uint32_t* __restrict__ cap,
                       uint32_t* __restrict__ srt, uint32_t* __restrict__ ntomb,
                       unsigned long long* __restrict__ capl) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n;
       i += uint64_t(gridDim.x) * blockDim.x) {
    uint32_t d = uint32_t(off_in[i + 1] - off_in[i]);
    deg[i] = d;
    srt[i] = d;
    ntomb[i] = 0;
    cap[i] = slack_cap(d);
    capl[i] = cap[i];
  }
}

// Warp per row: copy the input row into its slack-CSR slot.
__global__ void k_fill_rows(uint32_t n, const unsigned long long* __restrict__ off_in,
                            const uint32_t* __restrict__ idx, const uint32_t* __restrict__ w,
                            const unsigned long long* __restrict__ off, uint2* __restrict__ arcs) {
  const uint32_t lane = threadIdx.x & 31u;
  uint64_t warp = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) >> 5;
  uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  for (uint64_t i = warp; i < n; i += nwarps) {
    unsigned long long a = off_in[i], b = off_in[i + 1], o = off[i];
    for (unsigned long long k = a + lane; k < b; k += 32) arcs[o + (k - a)] = make_uint2(idx[k], w[k]);
  }
}

// K_i = sum_j w_ij (Section 3), warp per row; 2m accumulated in ctrl->red_a.
__global__ void k_weighted_degree(GraphView g, long long* __restrict__ K, Ctrl* ctrl) {
  const uint32_t lane = threadIdx.x & 31u;
  uint64_t warp = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) >> 5;
  uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  unsigned long long tot = 0;
  for (uint64_t i = warp; i < g.nv; i += nwarps) {
    unsigned long long s = 0;
    unsigned long long o = g.off[i];
    uint32_t d = g.deg[i];
    for (uint32_t k = lane; k < d; k += 32) s += g.arcs[o + k].y;
    for (int x = 16; x; x >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, x);
    if (lane == 0) K[i] = (long long)s;
    tot += s;
  }
  if (lane == 0 && tot) atomicAdd(&ctrl->red_a, tot);
}

// sigma = sum of arc weights with both ends in one community (red_a);
// sum_c Sigma_c^2 split into low (red_b) and high (red_c) 32-bit parts.
__global__ void k_modularity(GraphView g, const uint32_t* __restrict__ C,
                             const long long* __restrict__ Sigma, uint32_t n, Ctrl* ctrl) {
  const uint32_t lane = threadIdx.x & 31u;
  uint64_t warp = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) >> 5;
  uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  unsigned long long sig = 0;
  for (uint64_t i = warp; i < g.nv; i += nwarps) {
    uint32_t ci = C[i];
    unsigned long long o = g.off[i];
    uint32_t d = g.deg[i];
    for (uint32_t k = lane; k < d; k += 32) {
      uint2 a = g.arcs[o + k];
      if (C[a.x] == ci) sig += a.y;
    }
  }
  unsigned long long lo = 0, hi = 0;
  for (uint64_t c = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; c < n;
       c += uint64_t(gridDim.x) * blockDim.x) {
    unsigned long long s = (unsigned long long)Sigma[c];
    u128 sq = (u128)s * s;
    lo += (unsigned long long)(sq & 0xFFFFFFFFull);
    hi += (unsigned long long)(sq >> 32);
  }
  for (int x = 16; x; x >>= 1) {
    sig += __shfl_xor_sync(0xFFFFFFFFu, sig, x);
    lo += __shfl_xor_sync(0xFFFFFFFFu, lo, x);
    hi += __shfl_xor_sync(0xFFFFFFFFu, hi, x);
  }
  if (lane == 0) {
    if (sig) atomicAdd(&ctrl->red_a, sig);
    if (lo) atomicAdd(&ctrl->red_b, lo);
    if (hi) atomicAdd(&ctrl->red_c, hi);
  }
}

__global__ void k_sigma_sizes(uint32_t n, const uint32_t* __restrict__ C,
                              const long long* __restrict__ K, long long* __restrict__ Sigma,
                              int* __restrict__ size) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n;
       i += uint64_t(gridDim.x) * blockDim.x) {
    uint32_t c = C[i];
    atomicAdd((unsigned long long*)&Sigma[c], (unsigned long long)K[i]);
    atomicAdd(&size[c], 1);
  }
}

int read_ctrl(Handle* h) {
  DFL_CUDA(h, cudaMemcpyAsync(h->hctrl, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
  DFL_CUDA(h, cudaStreamSynchronize(h->stream));
  return DFL_OK;
}

}  // namespace

int graph_build(Handle* h, const unsigned long long* off_in, const uint32_t* idx_in,
                const uint32_t* w_in, uint64_t nnz) {
  const uint32_t n = h->n;
  DFL_CUDA(h, cudaMemsetAsync(h->ctrl, 0, sizeof(Ctrl), h->stream));
  {
    LaunchScope ls(h, DFL_PROF_OTHER);
    k_validate<<<grid_for(uint64_t(n) * 32, 256), 256, 0, h->stream>>>(n, off_in, idx_in, w_in,
                                                                         nnz, h->ctrl);
    DFL_TRY(check_launch(h, "validate"));
  }
  DFL_TRY(read_ctrl(h));
  if (h->hctrl->err) return set_error(h, DFL_ERR_INVALID, "input CSR is not a valid symmetric graph");
  // (a group checks the 2m of each of its graphs instead)
  if (!h->ngraphs && h->hctrl->red_a >= (1ull << 32)) return set_error(h, DFL_ERR_OVERFLOW, "2m >= 2^32");
  h->max_deg = h->hctrl->max_deg;
  h->num_arcs = nnz;
  // slack capacities and offsets
  unsigned long long* capl = nullptr;
  DFL_CUDA(h, dev_malloc(&capl, sizeof(unsigned long long) * (uint64_t(n) + 1)));
  int rc = DFL_OK;
  {
    LaunchScope ls(h, DFL_PROF_OTHER);
    k_caps<<<grid_for(n, 256), 256, 0, h->stream>>>(n, off_in, h->deg, h->cap, h->srt, h->ntomb,
                                                     capl);
    rc = check_launch(h, "caps");
  }
  if (!rc) rc = scan_u64(h, capl, h->off, n);  // off has n+1 entries during the build
  unsigned long long total = 0;
  if (!rc && cudaMemcpyAsync(&total, h->off + n, sizeof(total), cudaMemcpyDeviceToHost,
                             h->stream) != cudaSuccess)
    rc = set_error(h, DFL_ERR_CUDA, "copy total");
  if (!rc && cudaStreamSynchronize(h->stream) != cudaSuccess) rc = set_error(h, DFL_ERR_CUDA, "sync");
  cudaFree(capl);
  if (rc) return rc;
  uint64_t pool = total + total / 8 + 1024;
  pool = (pool + 1) & ~uint64_t(1);
  DFL_CUDA(h, dev_malloc(&h->arcs, sizeof(uint2) * pool));
  h->pool_cap = pool;
  h->pool_top = total;
  {
    LaunchScope ls(h, DFL_PROF_OTHER);
    k_fill_rows<<<grid_for(uint64_t(n) * 32, 256), 256, 0, h->stream>>>(n, off_in, idx_in, w_in,
                                                                         h->off, h->arcs);
    DFL_TRY(check_launch(h, "fill rows"));
  }
  return DFL_OK;
}

// K, 2m (and every graph's 2m in a group), Sigma and community sizes from
// scratch: the state a dynamic method without auxiliary information
// (Section 4.2) computes before each update.
int recompute_aux(Handle* h) {
  DFL_TRY(weighted_degrees(h));
  if (h->ngraphs) DFL_TRY(group_m2(h));
  return recompute_sigma_sizes(h, h->C);
}

int weighted_degrees(Handle* h) {
  DFL_CUDA(h, cudaMemsetAsync(&h->ctrl->red_a, 0, sizeof(unsigned long long), h->stream));
  {
    LaunchScope ls(h, DFL_PROF_OTHER);
    k_weighted_degree<<<grid_for(uint64_t(h->n) * 32, 256), 256, 0, h->stream>>>(base_view(h), h->K,
                                                                                  h->ctrl);
    DFL_TRY(check_launch(h, "weighted degree"));
  }
  DFL_TRY(read_ctrl(h));
  h->m2 = (long long)h->hctrl->red_a;
  return DFL_OK;
}

int modularity_parts(Handle* h, i128* num, i128* den) {
  DFL_CUDA(h, cudaMemsetAsync(&h->ctrl->red_a, 0, 3 * sizeof(unsigned long long), h->stream));
  {
    LaunchScope ls(h, DFL_PROF_OTHER);
    k_modularity<<<grid_for(uint64_t(h->n) * 32, 256), 256, 0, h->stream>>>(base_view(h), h->C,
                                                                             h->Sigma, h->n, h->ctrl);
    DFL_TRY(check_launch(h, "modularity"));
  }
  DFL_TRY(read_ctrl(h));
  i128 sig = (i128)h->hctrl->red_a;
  i128 sq = ((i128)h->hctrl->red_c << 32) + (i128)h->hctrl->red_b;
  *num = (i128)h->m2 * sig - sq;
  *den = (i128)h->m2 * (i128)h->m2;
  return DFL_OK;
}

// Pool compaction, pass 1, warp per row: the row's live arcs (weight > 0),
// counted, and the fresh slack capacity for them.
__global__ void k_compact_caps(uint32_t n, const uint2* __restrict__ arcs, const unsigned long long* __restrict__ off,
                               const uint32_t* __restrict__ deg, unsigned long long* __restrict__ capl) {
  const uint32_t lane = threadIdx.x & 31u;
  uint64_t warp = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) >> 5;
  const uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  for (; warp < n; warp += nwarps) {
    const unsigned long long o = off[warp];
    const uint32_t d = deg[warp];
    uint32_t live = 0;
    for (uint32_t k = lane; k < d; k += 32) live += arcs[o + k].y != 0;
    for (int x = 16; x; x >>= 1) live += __shfl_xor_sync(0xFFFFFFFFu, live, x);
    if (lane == 0) capl[warp] = slack_cap(live);
  }
}

// Pass 2, warp per row: the row's live arcs into its new slot in the same
// order -- the live part of the sorted prefix first (still sorted), then the
// live tail -- and the row's new length, sorted-prefix length, capacity and
// offset (each row's own entries are read before they are written).
__global__ void k_compact_rows(uint32_t n, const uint2* __restrict__ arcs, unsigned long long* __restrict__ off,
                               const unsigned long long* __restrict__ noff, uint32_t* __restrict__ deg,
                               uint32_t* __restrict__ cap, uint32_t* __restrict__ srt,
                               uint32_t* __restrict__ ntomb, uint2* __restrict__ out) {
  const uint32_t lane = threadIdx.x & 31u;
  uint64_t warp = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) >> 5;
  const uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  for (; warp < n; warp += nwarps) {
    const uint32_t i = uint32_t(warp);
    const unsigned long long o = off[i], no = noff[i];
    const uint32_t d = deg[i], sp = srt[i];
    uint32_t pos = 0, live_prefix = 0;
    for (uint32_t k0 = 0; k0 < d; k0 += 32) {
      const uint32_t k = k0 + lane;
      const uint2 a = k < d ? arcs[o + k] : make_uint2(0u, 0u);
      const bool live = k < d && a.y != 0;
      const unsigned m = __ballot_sync(0xFFFFFFFFu, live);
      if (live) out[no + pos + __popc(m & ((1u << lane) - 1u))] = a;
      // live arcs of the sorted prefix [0, sp) of this group of 32
      const unsigned pre = sp > k0 ? (sp - k0 >= 32 ? 0xFFFFFFFFu : ((1u << (sp - k0)) - 1u)) : 0u;
      live_prefix += __popc(m & pre);
      pos += __popc(m);
    }
    __syncwarp();
    if (lane == 0) {
      off[i] = no;
      deg[i] = pos;
      srt[i] = live_prefix;
      ntomb[i] = 0;
      cap[i] = slack_cap(pos);
    }
  }
}

int compact_pool(Handle* h, uint64_t* before, uint64_t* after) {
  const uint32_t n = h->n;
  if (before) *before = h->pool_cap;
  if (!n) {
    if (after) *after = h->pool_cap;
    return DFL_OK;
  }
  DFL_CUDA(h, cudaStreamSynchronize(h->stream));
  unsigned long long* capl = nullptr;
  DFL_CUDA(h, dev_malloc(&capl, sizeof(unsigned long long) * (uint64_t(n) + 1)));
  int rc = DFL_OK;
  {
    LaunchScope ls(h, DFL_PROF_OTHER);
    k_compact_caps<<<grid_for(uint64_t(n) * 32, 256), 256, 0, h->stream>>>(n, h->arcs, h->off, h->deg, capl);
    rc = check_launch(h, "compact caps");
  }
  if (!rc) rc = scan_u64(h, capl, capl, n);  // new offsets, capl[n] = total
  unsigned long long total = 0;
  if (!rc && cudaMemcpyAsync(&total, capl + n, sizeof(total), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
    rc = set_error(h, DFL_ERR_CUDA, "copy total");
  if (!rc && cudaStreamSynchronize(h->stream) != cudaSuccess) rc = set_error(h, DFL_ERR_CUDA, "sync");
  uint2* pool = nullptr;
  uint64_t cap = 0;
  if (!rc) {
    cap = (total + total / 8 + 1024 + 1) & ~uint64_t(1);
    if (dev_malloc(&pool, sizeof(uint2) * cap) != cudaSuccess) {
      cudaGetLastError();
      rc = set_error(h, DFL_ERR_NOMEM, "compacted arc pool");
    }
  }
  if (!rc) {
    LaunchScope ls(h, DFL_PROF_OTHER);
    k_compact_rows<<<grid_for(uint64_t(n) * 32, 256), 256, 0, h->stream>>>(n, h->arcs, h->off, capl, h->deg,
                                                                           h->cap, h->srt, h->ntomb, pool);
    rc = check_launch(h, "compact rows");
  }
  if (!rc && cudaStreamSynchronize(h->stream) != cudaSuccess) rc = set_error(h, DFL_ERR_CUDA, "sync");
  cudaFree(capl);
  if (rc) {
    if (pool) cudaFree(pool);
    return rc;
  }
  // captured iterations bake the old pool's address in
  for (auto& row : h->igraph)
    for (auto& g : row) destroy_iteration_graph(g);
  cudaFree(h->arcs);
  h->arcs = pool;
  h->pool_cap = cap;
  h->pool_top = total;
  if (after) *after = h->pool_cap;
  return DFL_OK;
}

// G^t as a compact CSR: live arcs only, rows sorted by neighbour.  The rows
// are read back and put in canonical order on the host (an inspection path).
int graph_export(Handle* h, uint64_t* off, uint32_t* idx, uint32_t* w, bool device_out) {
  const uint32_t n = h->n;
  std::vector<unsigned long long> hoff(n);
  std::vector<uint32_t> hdeg(n);
  std::vector<uint2> arcs(h->pool_top ? h->pool_top : 1);
  DFL_CUDA(h, cudaStreamSynchronize(h->stream));
  if (n) {
    DFL_CUDA(h, cudaMemcpy(hoff.data(), h->off, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost));
    DFL_CUDA(h, cudaMemcpy(hdeg.data(), h->deg, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost));
  }
  if (h->pool_top)
    DFL_CUDA(h, cudaMemcpy(arcs.data(), h->arcs, sizeof(uint2) * h->pool_top, cudaMemcpyDeviceToHost));
  std::vector<uint64_t> o(uint64_t(n) + 1, 0);
  std::vector<uint32_t> vi, vw;
  vi.reserve(h->num_arcs);
  vw.reserve(h->num_arcs);
  std::vector<uint2> row;
  for (uint32_t i = 0; i < n; ++i) {
    row.clear();
    for (uint32_t k = 0; k < hdeg[i]; ++k) {
      uint2 a = arcs[hoff[i] + k];
      if (a.y) row.push_back(a);
    }
    std::sort(row.begin(), row.end(), [](const uint2& x, const uint2& y) { return x.x < y.x; });
    for (const uint2& a : row) {
      vi.push_back(a.x);
      vw.push_back(a.y);
    }
    o[i + 1] = vi.size();
  }
  if (vi.size() != h->num_arcs) return set_error(h, DFL_ERR_CUDA, "live arc count mismatch");
  cudaMemcpyKind kd = device_out ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
  DFL_CUDA(h, cudaMemcpy(off, o.data(), sizeof(uint64_t) * o.size(), kd));
  if (!vi.empty()) {
    DFL_CUDA(h, cudaMemcpy(idx, vi.data(), sizeof(uint32_t) * vi.size(), kd));
    DFL_CUDA(h, cudaMemcpy(w, vw.data(), sizeof(uint32_t) * vw.size(), kd));
  }
  return DFL_OK;
}

int recompute_sigma_sizes(Handle* h, const uint32_t* C) {
  DFL_CUDA(h, cudaMemsetAsync(h->Sigma, 0, sizeof(long long) * h->n, h->stream));
  DFL_CUDA(h, cudaMemsetAsync(h->csize, 0, sizeof(int) * h->n, h->stream));
  LaunchScope ls(h, DFL_PROF_OTHER);
  k_sigma_sizes<<<grid_for(h->n, 256), 256, 0, h->stream>>>(h->n, C, h->K, h->Sigma, h->csize);
  return check_launch(h, "sigma sizes");
}

}  // namespace dfl
