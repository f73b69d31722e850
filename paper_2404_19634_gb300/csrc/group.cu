// Groups: many independent graphs in one handle, stored as their disjoint
// union so that each step of an update is one launch over every graph.
//
// Louvain (Alg. 4) runs on the union with the per-graph parts kept apart:
//   - local-moving scores a vertex with its own graph's 2m and sums its
//     movers' dQ per graph; a graph whose sum falls to its own tolerance
//     (Alg. 5) stops being processed while the others continue;
//   - after each pass a graph is finished if it ran at most one iteration or
//     its communities shrank too little (|Gamma| / |V'| > tau_agg), exactly
//     as a handle of its own would stop; its final labels are fixed then
//     (the current level's membership looked up through the dendrogram, put
//     back into the graph's own id range);
//   - the union is renumbered by ascending label and aggregated (Alg. 6):
//     every graph's labels lie in its own id range, so the super-vertex graph
//     is again a disjoint union, and the graphs' new vertex ranges are the
//     renumbering's prefix sums at the old range starts.  Finished graphs ride
//     along as frozen super-vertices that are never processed again.
#include "common.cuh"

namespace dfl {

namespace {

__global__ void k_group_ksum(uint32_t n, uint32_t ng, const uint32_t* __restrict__ goff,
                             const long long* __restrict__ K, unsigned long long* __restrict__ out) {
  // each thread sums a contiguous slice, flushing when the graph changes
  const uint64_t nth = uint64_t(gridDim.x) * blockDim.x;
  const uint64_t t = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x;
  const uint64_t per = (n + nth - 1) / nth;
  uint64_t v0 = t * per, v1 = v0 + per < n ? v0 + per : n;
  if (v0 >= v1) return;
  uint32_t g = graph_of(goff, ng, uint32_t(v0));
  unsigned long long acc = 0;
  for (uint64_t v = v0; v < v1; ++v) {
    while (v >= goff[g + 1]) {
      if (acc) atomicAdd(out + g, acc);
      acc = 0;
      ++g;
    }
    acc += (unsigned long long)K[v];
  }
  if (acc) atomicAdd(out + g, acc);
}

// d_gm2[g] = sum[g] (below 2^32: the batch's staging checked each graph's
// 2m against its insertions before the apply)
__global__ void k_group_m2_store(const unsigned long long* __restrict__ sum, long long* __restrict__ gm2,
                                 uint32_t ng) {
  for (uint64_t g = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; g < ng; g += uint64_t(gridDim.x) * blockDim.x)
    gm2[g] = (long long)sum[g];
}

// sigma (arcs inside communities) over rows [v0, v1) and sum of Sigma_c^2
// over labels [v0, v1): graph g's share of Eq. 1.
__global__ void k_range_modularity(GraphView g, const uint32_t* __restrict__ C,
                                   const long long* __restrict__ Sigma, uint32_t v0, uint32_t v1,
                                   Ctrl* ctrl) {
  const uint32_t lane = threadIdx.x & 31u;
  uint64_t warp = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) >> 5;
  uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  unsigned long long sig = 0;
  for (uint64_t i = v0 + warp; i < v1; i += nwarps) {
    const uint32_t ci = C[i];
    const unsigned long long o = g.off[i];
    const uint32_t dg = g.deg[i];
    for (uint32_t k = lane; k < dg; k += 32) {
      uint2 arc = g.arcs[o + k];
      if (arc.y && C[arc.x] == ci) sig += arc.y;
    }
  }
  unsigned long long lo = 0, hi = 0;
  for (uint64_t c = v0 + blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; c < v1;
       c += uint64_t(gridDim.x) * blockDim.x) {
    u128 sq = (u128)(unsigned long long)Sigma[c] * (unsigned long long)Sigma[c];
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

// next[g] = new id of the first label of graph g (the renumbering's
// exclusive scan at the range start).
__global__ void k_gather_starts(uint32_t ng, const uint32_t* __restrict__ goff,
                                const uint32_t* __restrict__ scan, uint32_t* __restrict__ next) {
  for (uint32_t g = threadIdx.x; g <= ng; g += blockDim.x) next[g] = scan[goff[g]];
}

// Final labels of the flagged graphs: the current level's label of each
// original vertex (through the dendrogram once aggregated), moved from the
// level's id range of the graph to its original one.
__global__ void k_finalize(uint32_t n, uint32_t ng, const uint32_t* __restrict__ goff0,
                           const uint32_t* __restrict__ goffL, const uint8_t* __restrict__ flag,
                           const uint32_t* __restrict__ Cp, const uint32_t* __restrict__ Ctop,
                           bool aggregated, uint32_t* __restrict__ Cfin) {
  for (uint64_t v = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; v < n;
       v += uint64_t(gridDim.x) * blockDim.x) {
    const uint32_t g = graph_of(goff0, ng, uint32_t(v));
    if (!flag[g]) continue;
    const uint32_t label = aggregated ? Cp[Ctop[v]] : Cp[v];
    Cfin[v] = goff0[g] + (label - goffL[g]);
  }
}

__global__ void k_copy_u32(uint64_t n, const uint32_t* __restrict__ src, uint32_t* __restrict__ dst) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n;
       i += uint64_t(gridDim.x) * blockDim.x)
    dst[i] = src[i];
}

}  // namespace

int group_upload_flags(Handle* h, uint8_t* dev, const uint8_t* host) {
  DFL_CUDA(h, cudaMemcpyAsync(dev, host, h->ngraphs, cudaMemcpyHostToDevice, h->stream));
  return DFL_OK;
}

int group_set_level(Handle* h, const uint32_t* dev_off) {
  if (dev_off == h->d_goff) return DFL_OK;
  DFL_CUDA(h, cudaMemcpyAsync(h->d_goff, dev_off, sizeof(uint32_t) * (h->ngraphs + 1),
                              cudaMemcpyDeviceToDevice, h->stream));
  return DFL_OK;
}

int group_m2(Handle* h) {
  const uint32_t G = h->ngraphs;
  DFL_CUDA(h, cudaMemsetAsync(h->d_gsum, 0, sizeof(unsigned long long) * G, h->stream));
  if (h->n) {
    LaunchScope ls(h, DFL_PROF_OTHER);
    k_group_ksum<<<grid_for(h->n, 256 * 64, 152 * 4), 256, 0, h->stream>>>(h->n, G, h->d_goff0, h->K,
                                                                           h->d_gsum);
    DFL_TRY(check_launch(h, "group 2m"));
  }
  std::vector<unsigned long long> m(G);
  DFL_CUDA(h, cudaMemcpyAsync(m.data(), h->d_gsum, sizeof(unsigned long long) * G,
                              cudaMemcpyDeviceToHost, h->stream));
  DFL_CUDA(h, cudaStreamSynchronize(h->stream));
  for (uint32_t g = 0; g < G; ++g) {
    if (m[g] >= (1ull << 32)) return set_error(h, DFL_ERR_OVERFLOW, "2m of a graph >= 2^32");
    h->gm2[g] = (long long)m[g];
  }
  DFL_CUDA(h, cudaMemcpyAsync(h->d_gm2, h->gm2.data(), sizeof(long long) * G,
                              cudaMemcpyHostToDevice, h->stream));
  DFL_CUDA(h, cudaStreamSynchronize(h->stream));
  return DFL_OK;
}

int group_m2_enqueue(Handle* h) {
  const uint32_t G = h->ngraphs;
  unsigned long long* sum = h->d_gsum + G;  // (the first G entries hold the staged insertion weights)
  DFL_CUDA(h, cudaMemsetAsync(sum, 0, sizeof(unsigned long long) * G, h->stream));
  if (h->n) {
    LaunchScope ls(h, DFL_PROF_OTHER);
    k_group_ksum<<<grid_for(h->n, 256 * 64, 152 * 4), 256, 0, h->stream>>>(h->n, G, h->d_goff0, h->K, sum);
    DFL_TRY(check_launch(h, "group 2m"));
  }
  {
    LaunchScope ls(h, DFL_PROF_OTHER);
    k_group_m2_store<<<grid_for(G, 256), 256, 0, h->stream>>>(sum, h->d_gm2, G);
    DFL_TRY(check_launch(h, "group 2m store"));
  }
  DFL_CUDA(h, cudaMemcpyAsync(h->h_gS, sum, sizeof(unsigned long long) * G, cudaMemcpyDeviceToHost, h->stream));
  return DFL_OK;
}

int group_m2_take(Handle* h) {
  for (uint32_t g = 0; g < h->ngraphs; ++g) {
    const unsigned long long m = h->h_gS[g];
    if (m >= (1ull << 32)) return set_error(h, DFL_ERR_OVERFLOW, "2m of a graph >= 2^32");
    h->gm2[g] = (long long)m;
  }
  return DFL_OK;
}

int group_modularity(Handle* h, uint32_t g, i128* num, i128* den) {
  const uint32_t v0 = h->goff0[g], v1 = h->goff0[g + 1];
  DFL_CUDA(h, cudaMemsetAsync(&h->ctrl->red_a, 0, 3 * sizeof(unsigned long long), h->stream));
  if (v1 > v0) {
    LaunchScope ls(h, DFL_PROF_OTHER);
    k_range_modularity<<<grid_for(uint64_t(v1 - v0) * 32, 256), 256, 0, h->stream>>>(
        base_view(h), h->C, h->Sigma, v0, v1, h->ctrl);
    DFL_TRY(check_launch(h, "group modularity"));
  }
  DFL_CUDA(h, cudaMemcpyAsync(h->hctrl, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
  DFL_CUDA(h, cudaStreamSynchronize(h->stream));
  const i128 m2 = (i128)h->gm2[g];
  const i128 sig = (i128)h->hctrl->red_a;
  const i128 sq = ((i128)h->hctrl->red_c << 32) + (i128)h->hctrl->red_b;
  *num = m2 * sig - sq;
  *den = m2 * m2;
  return DFL_OK;
}

int louvain_group(Handle* h, bool all, bool use_range, uint64_t initial) {
  const uint32_t n = h->n, G = h->ngraphs;
  h->trace.clear();
  dfl_stats_t& st = h->stats;
  st.passes = 0;
  for (int p = 0; p < 16; ++p) st.iterations[p] = 0;
  st.affected_initial = initial;
  for (auto& s : h->gstats) {
    s.passes = 0;
    for (int p = 0; p < 16; ++p) s.iterations[p] = 0;
    s.num_communities = 0;
  }
  if (!all) DFL_CUDA(h, cudaMemsetAsync(h->ever, 0, sizeof(uint32_t) * h->words, h->stream));
  for (uint32_t g = 0; g < G; ++g) h->gfin[g] = h->goff0[g + 1] == h->goff0[g];  // empty graphs
  DFL_TRY(group_set_level(h, h->d_goff0));

  GraphView gv = base_view(h);
  uint32_t nv = n;
  uint32_t* Cp = h->C;
  const long long* Kp = h->K;
  long long* Sp = h->Sigma;
  int* szp = h->csize;
  uint32_t maxdeg = h->max_deg;
  bool aggregated = false;
  int level = 0;
  std::vector<uint32_t> offL(h->goff0);  // graph ranges at the current level
  std::vector<uint32_t> git(G), noff(G + 1);
  std::vector<uint8_t> flag(G);

  // final labels of the graphs flagged in `flag` at the current level, into
  // Cfin (in the first pass they are C itself, which a later renumbering of
  // the union would overwrite)
  auto finalize = [&]() -> int {
    bool any = false;
    for (uint32_t g = 0; g < G; ++g) any |= flag[g] != 0;
    if (!any) return DFL_OK;
    DFL_TRY(group_upload_flags(h, h->d_gflag, flag.data()));
    LaunchScope ls(h, DFL_PROF_AGG);
    k_finalize<<<grid_for(n, 256), 256, 0, h->stream>>>(n, G, h->d_goff0, h->d_goff, h->d_gflag, Cp,
                                                        h->Ctop, aggregated, h->Cfin);
    return check_launch(h, "group finalize");
  };

  uint32_t pass = 0;
  for (; pass < h->opt.max_passes; ++pass) {
    if (pass > 0) {
      DFL_CUDA(h, cudaMemsetAsync(h->ctrl, 0, sizeof(Ctrl), h->stream));
      DFL_CUDA(h, cudaMemsetAsync(h->fbits[0], 0, sizeof(uint32_t) * h->words, h->stream));
      DFL_CUDA(h, cudaMemsetAsync(h->fbits[1], 0, sizeof(uint32_t) * h->words, h->stream));
      DFL_TRY(lists_all(h, nv, gv.deg, 0, h->opt.substeps));
    }
    MoveArgs a;
    a.g = gv;
    a.C = Cp;
    a.K = Kp;
    a.Sigma = Sp;
    a.size = szp;
    a.m2 = h->m2;
    a.max_deg = maxdeg;
    a.use_range = use_range && pass == 0;
    a.track_ever = pass == 0 && !all;
    a.prefer_host = true;
    a.graph_iters = git.data();
    uint32_t it = 0;
    uint64_t init0 = 0, ever0 = 0;
    DFL_TRY(local_move(h, a, pass, &it, false, &init0, &ever0));
    if (pass < 16) st.iterations[pass] = it;
    st.passes = pass + 1;
    if (pass == 0) {
      if (initial == ~0ull) st.affected_initial = init0;
      st.affected_ever = all ? n : ever0;
    }
    // graphs that converged globally (at most one iteration)
    uint32_t nactive = 0;
    for (uint32_t g = 0; g < G; ++g) {
      flag[g] = 0;
      if (h->gfin[g]) continue;
      if (pass < 16) h->gstats[g].iterations[pass] = git[g];
      h->gstats[g].passes = pass + 1;
      if (git[g] <= 1) flag[g] = 1;
      else ++nactive;
    }
    if (nactive) {
      uint32_t total = 0;
      DFL_TRY(count_communities(h, Cp, nv, &total));
      {
        LaunchScope ls(h, DFL_PROF_AGG);
        k_gather_starts<<<1, 256, 0, h->stream>>>(G, h->d_goff, h->used, h->d_gnext);
        DFL_TRY(check_launch(h, "group starts"));
      }
      DFL_CUDA(h, cudaMemcpyAsync(noff.data(), h->d_gnext, sizeof(uint32_t) * (G + 1),
                                  cudaMemcpyDeviceToHost, h->stream));
      DFL_CUDA(h, cudaStreamSynchronize(h->stream));
      for (uint32_t g = 0; g < G; ++g) {
        if (h->gfin[g] || flag[g]) continue;
        const uint32_t ncomm = noff[g + 1] - noff[g];
        if (pass == 0) h->gstats[g].num_communities = ncomm;
        const double ratio = double(ncomm) / double(offL[g + 1] - offL[g]);
        if (ratio > h->opt.tau_agg) {  // low shrink
          flag[g] = 1;
          --nactive;
        }
      }
    }
    DFL_TRY(finalize());
    for (uint32_t g = 0; g < G; ++g) h->gfin[g] |= flag[g];
    if (!nactive) break;
    // renumber and aggregate the whole union; finished graphs are frozen
    uint32_t ncomm = noff[G];
    DFL_TRY(renumber(h, Cp, nv, !aggregated));
    DFL_TRY(aggregate(h, gv, Cp, ncomm, level, h->Ks));
    maxdeg = h->hctrl->max_deg;
    SuperGraph& sg = h->sg[level];
    gv = GraphView{sg.off, sg.deg, sg.arcs, ncomm};
    nv = ncomm;
    Kp = h->Ks;
    Sp = h->Ss;
    szp = h->sizes;
    Cp = h->Cs;
    DFL_TRY(copy_i64(h, h->Ss, h->Ks, nv));
    DFL_TRY(fill_i32(h, h->sizes, 1, nv));
    DFL_TRY(iota_u32(h, h->Cs, nv));
    DFL_TRY(group_set_level(h, h->d_gnext));
    offL = noff;
    level ^= 1;
    aggregated = true;
  }
  // graphs still running when the passes ran out
  bool rest = false;
  for (uint32_t g = 0; g < G; ++g) {
    flag[g] = !h->gfin[g];
    rest |= flag[g] != 0;
  }
  if (rest) DFL_TRY(finalize());
  if (aggregated) {  // every graph's labels are in Cfin
    LaunchScope ls(h, DFL_PROF_AGG);
    k_copy_u32<<<grid_for(n, 256), 256, 0, h->stream>>>(n, h->Cfin, h->C);
    DFL_TRY(check_launch(h, "group labels"));
  }
  if (aggregated) DFL_TRY(recompute_sigma_sizes(h, h->C));
  st.num_communities = 0;
  return check_launch(h, "group louvain");  // (stream-ordered, as in louvain)
}

}  // namespace dfl
