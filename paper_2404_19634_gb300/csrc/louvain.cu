// Dynamic-supporting Louvain driver (Alg. 4): passes of local-moving and
// aggregation, renumbering, dendrogram lookup, threshold scaling.
//
// Pass 0 works in place on the handle's state (G^t, C, K, Sigma, sizes)
// starting from C^{t-1} and the marked frontier.  If it runs more than one
// iteration and the communities shrink enough (|Gamma| / |V'| <= tau_agg),
// communities are renumbered by ascending label, the top-level membership
// is looked up, and G' is aggregated; later passes run on the super-vertex
// graph with every vertex unprocessed, C' = identity, K' = Sigma' = row sums.
// The final membership is the last C' looked up through the dendrogram (not
// renumbered); after an aggregation Sigma and the sizes are recomputed.
#include "common.cuh"

namespace dfl {

namespace {

__global__ void k_used(uint32_t nv, const uint32_t* __restrict__ Cp, uint32_t* __restrict__ used) {
  for (uint64_t v = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; v < nv;
       v += uint64_t(gridDim.x) * blockDim.x)
    used[Cp[v]] = 1u;
}

__global__ void k_relabel(uint32_t nv, uint32_t* __restrict__ Cp, const uint32_t* __restrict__ newid) {
  for (uint64_t v = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; v < nv;
       v += uint64_t(gridDim.x) * blockDim.x)
    Cp[v] = newid[Cp[v]];
}

// Ctop[v] <- Cp[Ctop[v]] (first: Ctop[v] <- Cp[v]).
__global__ void k_lookup(uint32_t n, uint32_t* __restrict__ Ctop, const uint32_t* __restrict__ Cp,
                         bool first) {
  for (uint64_t v = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; v < n;
       v += uint64_t(gridDim.x) * blockDim.x)
    Ctop[v] = first ? Cp[v] : Cp[Ctop[v]];
}

__global__ void k_final(uint32_t n, uint32_t* __restrict__ C, const uint32_t* __restrict__ Ctop,
                        const uint32_t* __restrict__ Cp) {
  for (uint64_t v = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; v < n;
       v += uint64_t(gridDim.x) * blockDim.x)
    C[v] = Cp[Ctop[v]];
}

}  // namespace

// |Gamma|: distinct labels of Cp over [0, nv); leaves the exclusive scan of
// the used flags (= new ids by ascending label) in h->used.
int count_communities(Handle* h, const uint32_t* Cp, uint32_t nv, uint32_t* ncomm) {
  DFL_CUDA(h, cudaMemsetAsync(h->used, 0, sizeof(uint32_t) * (uint64_t(nv) + 1), h->stream));
  {
    LaunchScope ls(h, DFL_PROF_AGG);
    k_used<<<grid_for(nv, 256), 256, 0, h->stream>>>(nv, Cp, h->used);
    DFL_TRY(check_launch(h, "used"));
  }
  DFL_TRY(scan_u32(h, h->used, h->used, nv));
  uint32_t total = 0;
  DFL_CUDA(h, cudaMemcpyAsync(&total, h->used + nv, sizeof(total), cudaMemcpyDeviceToHost, h->stream));
  DFL_CUDA(h, cudaStreamSynchronize(h->stream));
  *ncomm = total;
  return DFL_OK;
}

// Renumber Cp with the ids left by count_communities, then update the
// top-level membership (dendrogram lookup).
int renumber(Handle* h, uint32_t* Cp, uint32_t nv, bool first_level) {
  {
    LaunchScope ls(h, DFL_PROF_AGG);
    k_relabel<<<grid_for(nv, 256), 256, 0, h->stream>>>(nv, Cp, h->used);
    DFL_TRY(check_launch(h, "relabel"));
  }
  LaunchScope ls(h, DFL_PROF_AGG);
  k_lookup<<<grid_for(h->n, 256), 256, 0, h->stream>>>(h->n, h->Ctop, Cp, first_level);
  return check_launch(h, "lookup");
}

int louvain(Handle* h, bool all, bool use_range, uint64_t initial) {
  const uint32_t n = h->n;
  h->trace.clear();
  dfl_stats_t& st = h->stats;
  st.passes = 0;
  for (int p = 0; p < 16; ++p) st.iterations[p] = 0;
  st.affected_initial = initial;
  if (!all && !h->ever_clear) DFL_CUDA(h, cudaMemsetAsync(h->ever, 0, sizeof(uint32_t) * h->words, h->stream));
  h->ever_clear = false;

  GraphView g = base_view(h);
  uint32_t nv = n;
  uint32_t* Cp = h->C;
  const long long* Kp = h->K;
  long long* Sp = h->Sigma;
  int* szp = h->csize;
  // (bounds while a batch apply enqueued before this update has not settled)
  uint32_t maxdeg = max_deg_bound(h);
  const uint64_t pend = h->pend_count + (h->papply.active ? h->papply.na : 0);
  bool aggregated = false;
  int level = 0;
  uint32_t last_comm = 0;

  for (uint32_t pass = 0; pass < h->opt.max_passes; ++pass) {
    if (pass > 0) {
      // every super-vertex unprocessed, in range
      DFL_CUDA(h, cudaMemsetAsync(h->ctrl, 0, sizeof(Ctrl), h->stream));
      DFL_CUDA(h, cudaMemsetAsync(h->fbits[0], 0, sizeof(uint32_t) * h->words, h->stream));
      DFL_CUDA(h, cudaMemsetAsync(h->fbits[1], 0, sizeof(uint32_t) * h->words, h->stream));
      DFL_TRY(lists_all(h, nv, g.deg, 0, h->opt.substeps));
    }
    MoveArgs a;
    a.g = g;
    a.C = Cp;
    a.K = Kp;
    a.Sigma = Sp;
    a.size = szp;
    a.m2 = h->m2;
    a.max_deg = maxdeg;
    a.use_range = use_range && pass == 0;
    a.track_ever = pass == 0 && !all;
    a.prefer_host = !all && pend < kGraphMinArcs;
    // DF marks at most one vertex per pending batch arc; ND, DS and later
    // passes may mark every vertex
    a.frontier_hint = (pass == 0 && !all && !use_range) ? pend : nv;
    uint32_t it = 0;
    uint64_t init0 = 0, ever0 = 0;
    DFL_TRY(local_move(h, a, pass, &it, pass == 0, &init0, &ever0));
    if (pass < 16) st.iterations[pass] = it;
    st.passes = pass + 1;
    if (pass == 0) {
      if (initial == ~0ull) st.affected_initial = init0;
      st.affected_ever = all ? n : ever0;
    }
    if (it <= 1) break;  // globally converged
    uint32_t ncomm = 0;
    DFL_TRY(count_communities(h, Cp, nv, &ncomm));
    if (pass == 0) last_comm = ncomm;
    if (double(ncomm) / double(nv) > h->opt.tau_agg) break;  // low shrink
    DFL_TRY(renumber(h, Cp, nv, !aggregated));
    DFL_TRY(aggregate(h, g, Cp, ncomm, level, h->Ks));
    maxdeg = h->hctrl->max_deg;
    SuperGraph& sg = h->sg[level];
    g = GraphView{sg.off, sg.deg, sg.arcs, ncomm};
    nv = ncomm;
    Kp = h->Ks;
    Sp = h->Ss;
    szp = h->sizes;
    Cp = h->Cs;
    DFL_TRY(copy_i64(h, h->Ss, h->Ks, nv));
    DFL_TRY(fill_i32(h, h->sizes, 1, nv));
    DFL_TRY(iota_u32(h, h->Cs, nv));
    level ^= 1;
    aggregated = true;
  }
  if (aggregated) {
    {
      LaunchScope ls(h, DFL_PROF_AGG);
      k_final<<<grid_for(n, 256), 256, 0, h->stream>>>(n, h->C, h->Ctop, Cp);
      DFL_TRY(check_launch(h, "final lookup"));
    }
    DFL_TRY(recompute_sigma_sizes(h, h->C));
  }
  st.num_communities = last_comm;
  // every host decision is made; what is left on the stream (clearing the
  // frontier, the final lookup) is ordered before the caller's next call
  return check_launch(h, "louvain");
}

}  // namespace dfl
