// Reference oracle for Dynamic Frontier (DF) Louvain -- TEST INFRASTRUCTURE.
//
// This file is a plain, slow, single-threaded statement of what the GPU path
// computes.  Only the test-suite, the package smoke check and the benchmark's
// CPU-baseline leg may load it.  It shares no code, header, table or helper
// with the CUDA library; the two only meet on the seeded synthetic inputs.
//
// It follows the paper (arXiv 2404.19634, "DF Louvain: Fast Incrementally
// Expanding Approach for Community Detection on Dynamic Graphs"):
//   Eq. 1  modularity           Q = sum_c [sigma_c/2m - (Sigma_c/2m)^2]
//   Eq. 2  delta-modularity     dQ_{i:d->c}
//   Alg. 1 Dynamic Frontier marking, Alg. 2 Naive-dynamic, Alg. 3 Delta-screening
//   Alg. 4 dynamic-supporting Louvain driver (passes)
//   Alg. 5 local-moving phase (louvainMove / scanCommunities)
//   Alg. 6 aggregation phase (louvainAggregate)
//   Alg. 7 updateWeights (incremental K and Sigma)
//
// The paper's local-moving is asynchronous; this oracle fixes a deterministic
// schedule instead, and the GPU path must reproduce it bit for bit:
//   * synchronous sub-steps: each local-moving iteration visits the frontier
//     in `substeps` classes (class of vertex i = top bits of the 32-bit
//     multiplicative hash i * 0x9E3779B1, Knuth TAOCP vol. 3, 6.4); within a
//     class every vertex decides against the membership C, community totals
//     Sigma and community sizes left by the previous sub-step, then all of
//     the class's moves are applied at once.  substeps = 1 is the plain
//     synchronous (Jacobi) schedule; the default 4 keeps the schedule
//     deterministic while damping the oscillation that plain synchronous
//     moves show from singleton starts;
//   * the best community is the neighbour community (other than the current
//     one) with the largest 2m*K_{i->c} - K_i*Sigma_c, ties to the smallest id;
//     a vertex moves only if that beats staying (dQ > 0 strictly);
//   * singleton-swap guard: a vertex alone in its community does not move
//     into another singleton community with a larger id (minimum-label rule
//     of Lu, Halappanavar and Kalyanaraman, Parallel Computing 2015);
//   * integer edge weights, int64 K/Sigma, exact 128-bit dQ arithmetic, and
//     the per-iteration tolerance test done exactly in integers.
//
// Parity status: Eq. 1, Eq. 2, Alg. 7, Alg. 6 and the marking rules of
// Alg. 1-3 are pinned by the CPU tests (closed forms, brute force on tiny
// graphs, invariants).  End-to-end memberships have no printed values in the
// paper: "parity unpinned" for the final communities beyond those invariants.

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <new>
#include <set>
#include <string>
#include <utility>
#include <vector>

typedef __int128 i128;
typedef unsigned __int128 u128;

namespace {

enum {
  OK = 0,
  E_INVALID = -1,
  E_NOT_FOUND = -2,
  E_OVERFLOW = -3,
  E_NOMEM = -4,
  E_STATE = -7,
};

enum { MODE_ND = 0, MODE_DS = 1, MODE_DF = 2 };

// One arc of a graph: neighbour j and weight w_ij.
struct Arc {
  uint32_t j;
  uint64_t w;
};
// Adjacency lists, each sorted by neighbour id.  Self-loops (j == i) appear
// once in the list of i (super-vertex graphs have them).
typedef std::vector<std::vector<Arc>> Graph;

// One directed arc of a batch update (both directions are stored).
struct BatchArc {
  uint32_t i, j;
  uint64_t w;
};

struct Options {
  uint32_t max_iterations = 20;  // MAX_ITERATIONS (Section 5.1.2)
  uint32_t max_passes = 10;      // MAX_PASSES
  uint64_t tau_num = 1;          // iteration tolerance tau = tau_num/tau_den = 1e-2
  uint64_t tau_den = 100;
  uint64_t tolerance_drop = 10;  // TOLERANCE_DROP (threshold scaling)
  double tau_agg = 0.8;          // aggregation tolerance
  uint32_t substeps = 4;         // synchronous sub-steps per iteration (1, 2, 4 or 8)
};

// Per-iteration record of the first pass (for trace parity).
struct IterRecord {
  uint64_t frontier;  // vertices processed (unprocessed at the start)
  uint64_t movers;
  u128 dq_sum;        // sum of the movers' 2m^2 * dQ numerators
};

struct Oracle {
  uint32_t n = 0;
  Graph G;                      // current graph G^t
  std::vector<int64_t> K;       // weighted degree of each vertex
  std::vector<int64_t> Sigma;   // total edge weight of each community (by label)
  int64_t m2 = 0;               // 2m = sum of all arc weights
  std::vector<uint32_t> C;      // community of each vertex
  bool have_communities = false;
  std::vector<BatchArc> pend_del, pend_ins;  // batch arcs since the last update
  Options opt;
  // statistics of the last louvain() call
  std::vector<uint32_t> pass_iterations;
  std::vector<IterRecord> trace;
  uint64_t affected_initial = 0;
  uint64_t affected_ever = 0;
  std::string err;
};

const uint64_t kWeightMax = 0xFFFFFFFFull;   // edge weights are u32
const int64_t kTwoMLimit = int64_t(1) << 32;  // 2m must stay below 2^32

// ---------------------------------------------------------------------------
// Graph helpers
// ---------------------------------------------------------------------------

// Index of neighbour j in the sorted list of i, or -1.
long find_arc(const std::vector<Arc>& row, uint32_t j) {
  auto it = std::lower_bound(row.begin(), row.end(), j,
                             [](const Arc& a, uint32_t x) { return a.j < x; });
  if (it == row.end() || it->j != j) return -1;
  return long(it - row.begin());
}

// K_i = sum_j w_ij (Section 3); a self-loop arc counts once.
std::vector<int64_t> weighted_degrees(const Graph& G) {
  std::vector<int64_t> K(G.size(), 0);
  for (size_t i = 0; i < G.size(); ++i)
    for (const Arc& a : G[i]) K[i] += int64_t(a.w);
  return K;
}

// Sigma_c = sum of K_i over the vertices of community c (Section 3.1).
std::vector<int64_t> community_totals(const std::vector<uint32_t>& C,
                                      const std::vector<int64_t>& K, size_t labels) {
  std::vector<int64_t> S(labels, 0);
  for (size_t i = 0; i < C.size(); ++i) S[C[i]] += K[i];
  return S;
}

std::vector<int64_t> community_sizes(const std::vector<uint32_t>& C, size_t labels) {
  std::vector<int64_t> s(labels, 0);
  for (uint32_t c : C) s[c] += 1;
  return s;
}

// ---------------------------------------------------------------------------
// scanCommunities (Alg. 5): H[C[j]] += w over the arcs of i, skipping the
// self-loop unless `self`.  H is a dense array indexed by community with the
// list of touched keys beside it (the paper's collision-free hashtable).
// ---------------------------------------------------------------------------
struct DenseTable {
  std::vector<uint64_t> val;
  std::vector<uint32_t> keys;
  std::vector<char> used;
  explicit DenseTable(size_t n) : val(n, 0), used(n, 0) {}
  void add(uint32_t c, uint64_t w) {
    if (!used[c]) {
      used[c] = 1;
      keys.push_back(c);
    }
    val[c] += w;
  }
  uint64_t get(uint32_t c) const { return used[c] ? val[c] : 0; }
  void clear() {
    for (uint32_t c : keys) {
      val[c] = 0;
      used[c] = 0;
    }
    keys.clear();
  }
};

void scan_communities(DenseTable& H, const Graph& G, const std::vector<uint32_t>& C,
                      uint32_t i, bool self) {
  for (const Arc& a : G[i])
    if (self || a.j != i) H.add(C[a.j], a.w);
}

// ---------------------------------------------------------------------------
// Eq. 2 in integers.  For vertex i in community d, with H = K_{i->*}:
//   2m^2 * dQ_{i:d->c} = 2m (K_{i->c} - K_{i->d}) - K_i (K_i + Sigma_c - Sigma_d)
// which equals score(c) - stay with
//   score(c) = 2m K_{i->c} - K_i Sigma_c,  stay = 2m K_{i->d} - K_i (Sigma_d - K_i).
// ---------------------------------------------------------------------------
i128 score_of(int64_t m2, uint64_t Hc, int64_t Ki, int64_t Sigma_c) {
  return i128(m2) * i128(Hc) - i128(Ki) * i128(Sigma_c);
}
i128 stay_of(int64_t m2, uint64_t Hd, int64_t Ki, int64_t Sigma_d) {
  return i128(m2) * i128(Hd) - i128(Ki) * i128(Sigma_d - Ki);
}

// Exact per-pass tolerance: stop when sum(dQ) <= tau_p, i.e. (in integers)
// S <= floor(tau_num * m2^2 / (2 * tau_den * drop^p)), S = sum of numerators.
// Sub-step class of vertex i among `k` classes (k a power of two).
uint32_t substep_class(uint32_t i, uint32_t k) {
  uint32_t h = i * 0x9E3779B1u;
  return uint32_t((uint64_t(h) * k) >> 32);
}

u128 tolerance_threshold(const Options& o, int64_t m2, uint32_t pass) {
  u128 num = u128(o.tau_num) * u128(uint64_t(m2)) * u128(uint64_t(m2));
  u128 den = u128(2) * u128(o.tau_den);
  for (uint32_t p = 0; p < pass; ++p) {
    if (den > num) return 0;
    den *= u128(o.tolerance_drop);
  }
  if (den == 0) return ~u128(0);
  return num / den;
}

// ---------------------------------------------------------------------------
// louvainMove (Alg. 5) under the synchronous schedule.
//   Gp, Cp, Kp, Sp, sizep: current graph G', membership C', K', Sigma', sizes
//   F: unprocessed flags (frontier), R: inAffectedRange flags
// Returns the number of iterations executed (>= 1).
// ---------------------------------------------------------------------------
uint32_t louvain_move(Oracle& o, const Graph& Gp, std::vector<uint32_t>& Cp,
                      const std::vector<int64_t>& Kp, std::vector<int64_t>& Sp,
                      std::vector<int64_t>& sizep, std::vector<char>& F,
                      const std::vector<char>& R, uint32_t pass,
                      std::vector<char>* ever) {
  const size_t nv = Gp.size();
  const u128 threshold = tolerance_threshold(o.opt, o.m2, pass);
  DenseTable H(Sp.size());
  struct Move {
    uint32_t i, d, c;
  };
  const uint32_t k = o.opt.substeps;
  uint32_t it = 0;
  while (it < o.opt.max_iterations) {
    ++it;
    std::vector<char> Fnext(nv, 0);  // neighbours of this iteration's movers
    u128 dq_sum = 0;
    uint64_t processed = 0, moved = 0;
    for (uint32_t sub = 0; sub < k; ++sub) {
      // snapshot of the state left by the previous sub-step
      const std::vector<uint32_t> Cold = Cp;
      const std::vector<int64_t> Sold = Sp;
      const std::vector<int64_t> sizeold = sizep;
      std::vector<Move> moves;
      for (uint32_t i = 0; i < nv; ++i) {
        if (!F[i] || substep_class(i, k) != sub) continue;
        F[i] = 0;  // mark i as processed (vertex pruning)
        ++processed;
        if (ever) (*ever)[i] = 1;
        if (!R[i]) continue;  // not in the affected range
        H.clear();
        scan_communities(H, Gp, Cold, i, false);
        const uint32_t d = Cold[i];
        bool have = false;
        uint32_t best = 0;
        i128 best_score = 0;
        for (uint32_t c : H.keys) {
          if (c == d) continue;
          i128 s = score_of(o.m2, H.get(c), Kp[i], Sold[c]);
          if (!have || s > best_score || (s == best_score && c < best)) {
            have = true;
            best = c;
            best_score = s;
          }
        }
        if (!have) continue;
        i128 stay = stay_of(o.m2, H.get(d), Kp[i], Sold[d]);
        if (!(best_score > stay)) continue;  // dQ > 0 strictly
        if (sizeold[d] == 1 && sizeold[best] == 1 && best > d) continue;  // swap guard
        moves.push_back({i, d, best});
        dq_sum += u128(best_score - stay);
      }
      // apply the sub-step's moves at once; neighbours of movers become
      // unprocessed for the next iteration
      for (const Move& mv : moves) {
        Cp[mv.i] = mv.c;
        Sp[mv.d] -= Kp[mv.i];
        Sp[mv.c] += Kp[mv.i];
        sizep[mv.d] -= 1;
        sizep[mv.c] += 1;
      }
      for (const Move& mv : moves)
        for (const Arc& a : Gp[mv.i])
          if (a.j != mv.i && R[a.j]) Fnext[a.j] = 1;
      moved += moves.size();
    }
    F.swap(Fnext);  // every vertex of F was processed, so F is empty here
    if (pass == 0) o.trace.push_back({processed, moved, dq_sum});
    if (dq_sum <= threshold) break;  // locally converged
  }
  return it;
}

// ---------------------------------------------------------------------------
// louvainAggregate (Alg. 6): super-vertex c gets one arc per neighbouring
// community d with the summed weight, self-loops included (self = true).
// Cp must already be renumbered to [0, ncomm).
// ---------------------------------------------------------------------------
Graph louvain_aggregate(const Graph& Gp, const std::vector<uint32_t>& Cp, uint32_t ncomm) {
  // community -> member vertices (G'_{C'})
  std::vector<std::vector<uint32_t>> members(ncomm);
  for (uint32_t i = 0; i < Gp.size(); ++i) members[Cp[i]].push_back(i);
  Graph Gs(ncomm);
  DenseTable H(ncomm);
  for (uint32_t c = 0; c < ncomm; ++c) {
    H.clear();
    for (uint32_t i : members[c]) scan_communities(H, Gp, Cp, i, true);
    std::vector<uint32_t> ks = H.keys;
    std::sort(ks.begin(), ks.end());
    for (uint32_t d : ks) Gs[c].push_back({d, H.get(d)});
  }
  return Gs;
}

// ---------------------------------------------------------------------------
// louvain (Alg. 4).  Cprev: starting membership of G^t; K, Sigma: current
// weights; F0: initially affected vertices; R0: affected range for pass 0.
// Returns C^t; Sigma is replaced by Sigma^t.
// ---------------------------------------------------------------------------
std::vector<uint32_t> louvain(Oracle& o, const std::vector<uint32_t>& Cprev,
                              std::vector<int64_t>& Sigma, std::vector<char> F0,
                              const std::vector<char>& R0) {
  const uint32_t n = o.n;
  o.pass_iterations.clear();
  o.trace.clear();
  std::vector<char> ever(n, 0);
  o.affected_initial = 0;
  for (char f : F0) o.affected_initial += f ? 1 : 0;

  std::vector<uint32_t> Ctop(n);  // C: top-level membership, identity at first
  for (uint32_t i = 0; i < n; ++i) Ctop[i] = i;
  const Graph* Gp = &o.G;
  Graph Gstore;
  std::vector<uint32_t> Cp = Cprev;
  std::vector<int64_t> Kp = o.K;
  std::vector<int64_t> Sp = Sigma;
  std::vector<int64_t> sizep = community_sizes(Cprev, n);
  std::vector<char> F = std::move(F0);
  std::vector<char> R = R0;
  bool aggregated = false;

  for (uint32_t pass = 0; pass < o.opt.max_passes; ++pass) {
    uint32_t li = louvain_move(o, *Gp, Cp, Kp, Sp, sizep, F, R, pass,
                               pass == 0 ? &ever : nullptr);
    o.pass_iterations.push_back(li);
    if (li <= 1) break;  // globally converged
    // number of communities in C' against the vertex count of G'
    const size_t nv = Gp->size();
    std::vector<char> used(Sp.size(), 0);
    for (uint32_t c : Cp) used[c] = 1;
    uint32_t ncomm = 0;
    for (char u : used) ncomm += u ? 1 : 0;
    if (double(ncomm) / double(nv) > o.opt.tau_agg) break;  // low shrink
    // renumber communities by ascending old label
    std::vector<uint32_t> newid(Sp.size(), 0);
    uint32_t next = 0;
    for (size_t c = 0; c < used.size(); ++c)
      if (used[c]) newid[c] = next++;
    for (uint32_t& c : Cp) c = newid[c];
    // dendrogram lookup C <- C'[C]
    for (uint32_t i = 0; i < n; ++i) Ctop[i] = Cp[Ctop[i]];
    // aggregate, reset weights, all vertices unprocessed, C' <- identity
    Gstore = louvain_aggregate(*Gp, Cp, ncomm);
    Gp = &Gstore;
    Kp = weighted_degrees(Gstore);
    Sp = Kp;
    sizep.assign(ncomm, 1);
    F.assign(ncomm, 1);
    R.assign(ncomm, 1);
    Cp.resize(ncomm);
    for (uint32_t c = 0; c < ncomm; ++c) Cp[c] = c;
    aggregated = true;
  }
  // final dendrogram lookup with the last C' (not renumbered)
  std::vector<uint32_t> Ct(n);
  for (uint32_t i = 0; i < n; ++i) Ct[i] = Cp[Ctop[i]];
  if (!aggregated) Sigma = Sp;
  else Sigma = community_totals(Ct, o.K, n);
  o.affected_ever = 0;
  for (char e : ever) o.affected_ever += e ? 1 : 0;
  return Ct;
}

// ---------------------------------------------------------------------------
// Marking of initially affected vertices.
// ---------------------------------------------------------------------------

// Alg. 1 (DF): endpoints of deletions inside a community and of insertions
// across communities; inAffectedRange = all.
void mark_dynamic_frontier(const Oracle& o, std::vector<char>& F, std::vector<char>& R) {
  F.assign(o.n, 0);
  R.assign(o.n, 1);
  for (const BatchArc& e : o.pend_del)
    if (o.C[e.i] == o.C[e.j]) F[e.i] = 1;
  for (const BatchArc& e : o.pend_ins)
    if (o.C[e.i] != o.C[e.j]) F[e.i] = 1;
}

// Alg. 2 (ND): everything affected, everything in range.
void mark_naive_dynamic(const Oracle& o, std::vector<char>& F, std::vector<char>& R) {
  F.assign(o.n, 1);
  R.assign(o.n, 1);
}

// Alg. 3 (DS): vertex / neighbour / community flags, then expand.
// The best community for an insertion source uses the current K, Sigma, 2m.
void mark_delta_screening(const Oracle& o, std::vector<char>& F, std::vector<char>& R) {
  std::vector<char> dV(o.n, 0), dE(o.n, 0), dC(o.n, 0);
  for (const BatchArc& e : o.pend_del)
    if (o.C[e.i] == o.C[e.j]) {
      dV[e.i] = 1;
      dE[e.i] = 1;
      dC[o.C[e.j]] = 1;
    }
  // group insertion arcs by source vertex
  std::map<uint32_t, std::map<uint32_t, uint64_t>> Hs;
  std::set<uint32_t> sources;
  for (const BatchArc& e : o.pend_ins) {
    sources.insert(e.i);
    if (o.C[e.i] != o.C[e.j]) Hs[e.i][o.C[e.j]] += e.w;
  }
  for (uint32_t i : sources) {
    auto it = Hs.find(i);
    if (it == Hs.end() || it->second.empty()) continue;  // no cross-community insertion
    bool have = false;
    uint32_t best = 0;
    i128 best_score = 0;
    for (const auto& kv : it->second) {  // ascending community id
      i128 s = score_of(o.m2, kv.second, o.K[i], o.Sigma[kv.first]);
      if (!have || s > best_score) {
        have = true;
        best = kv.first;
        best_score = s;
      }
    }
    dV[i] = 1;
    dE[i] = 1;
    dC[best] = 1;
  }
  for (uint32_t i = 0; i < o.n; ++i) {
    if (dE[i])
      for (const Arc& a : o.G[i]) dV[a.j] = 1;
  }
  for (uint32_t i = 0; i < o.n; ++i)
    if (dC[o.C[i]]) dV[i] = 1;
  F = dV;
  R = dV;
}

// ---------------------------------------------------------------------------
// Batch update: validate everything, then apply deletions before insertions
// to the graph and update K, Sigma, 2m with the current membership (Alg. 7).
// ---------------------------------------------------------------------------
int apply_batch(Oracle& o, const uint32_t* del, uint64_t nd, const uint32_t* ins, uint64_t ni) {
  if (!o.have_communities) {
    o.err = "apply_batch before static";
    return E_STATE;
  }
  int invalid = 0, notfound = 0, overflow = 0;
  std::set<std::pair<uint32_t, uint32_t>> seen_del;
  std::map<std::pair<uint32_t, uint32_t>, uint64_t> after;  // weight after the batch
  for (uint64_t k = 0; k < nd; ++k) {
    uint32_t u = del[3 * k], v = del[3 * k + 1], w = del[3 * k + 2];
    if (u >= o.n || v >= o.n || u == v) { invalid = 1; continue; }
    auto key = std::make_pair(std::min(u, v), std::max(u, v));
    if (!seen_del.insert(key).second) { invalid = 1; continue; }
    long p = find_arc(o.G[u], v);
    if (p < 0) { notfound = 1; continue; }
    uint64_t cur = o.G[u][p].w;
    if (w > cur) { notfound = 1; continue; }
    after[key] = cur - (w == 0 ? cur : w);
  }
  for (uint64_t k = 0; k < ni; ++k) {
    uint32_t u = ins[3 * k], v = ins[3 * k + 1], w = ins[3 * k + 2];
    if (u >= o.n || v >= o.n || u == v || w == 0) { invalid = 1; continue; }
  }
  if (invalid) { o.err = "invalid edge in batch"; return E_INVALID; }
  if (notfound) { o.err = "deleted edge not found"; return E_NOT_FOUND; }
  int64_t m2_new = o.m2;
  for (const auto& kv : after) {
    long p = find_arc(o.G[kv.first.first], kv.first.second);
    m2_new -= 2 * int64_t(o.G[kv.first.first][p].w - kv.second);
  }
  for (uint64_t k = 0; k < ni; ++k) {
    uint32_t u = ins[3 * k], v = ins[3 * k + 1], w = ins[3 * k + 2];
    auto key = std::make_pair(std::min(u, v), std::max(u, v));
    auto it = after.find(key);
    uint64_t base;
    if (it != after.end()) base = it->second;
    else {
      long p = find_arc(o.G[key.first], key.second);
      base = p < 0 ? 0 : o.G[key.first][p].w;
    }
    after[key] = base + w;
    if (base + w > kWeightMax) overflow = 1;
    m2_new += 2 * int64_t(w);
  }
  if (m2_new >= kTwoMLimit) overflow = 1;
  if (overflow) { o.err = "edge weight or 2m overflow"; return E_OVERFLOW; }

  // Apply (updateWeights, Alg. 7, plus the graph change itself).
  auto set_weight = [&](uint32_t u, uint32_t v, uint64_t w) {
    std::vector<Arc>& row = o.G[u];
    long p = find_arc(row, v);
    if (w == 0) {
      if (p >= 0) row.erase(row.begin() + p);
    } else if (p >= 0) {
      row[p].w = w;
    } else {
      auto it = std::lower_bound(row.begin(), row.end(), v,
                                 [](const Arc& a, uint32_t x) { return a.j < x; });
      row.insert(it, Arc{v, w});
    }
  };
  for (uint64_t k = 0; k < nd; ++k) {
    uint32_t u = del[3 * k], v = del[3 * k + 1], w = del[3 * k + 2];
    uint64_t cur = o.G[u][find_arc(o.G[u], v)].w;
    uint64_t weff = (w == 0) ? cur : w;
    for (int dir = 0; dir < 2; ++dir) {
      uint32_t a = dir ? v : u, b = dir ? u : v;
      o.K[a] -= int64_t(weff);
      o.Sigma[o.C[a]] -= int64_t(weff);
      o.pend_del.push_back({a, b, weff});
      set_weight(a, b, cur - weff);
    }
    o.m2 -= 2 * int64_t(weff);
  }
  for (uint64_t k = 0; k < ni; ++k) {
    uint32_t u = ins[3 * k], v = ins[3 * k + 1], w = ins[3 * k + 2];
    long p = find_arc(o.G[u], v);
    uint64_t cur = p < 0 ? 0 : o.G[u][p].w;
    for (int dir = 0; dir < 2; ++dir) {
      uint32_t a = dir ? v : u, b = dir ? u : v;
      o.K[a] += int64_t(w);
      o.Sigma[o.C[a]] += int64_t(w);
      o.pend_ins.push_back({a, b, uint64_t(w)});
      set_weight(a, b, cur + w);
    }
    o.m2 += 2 * int64_t(w);
  }
  return OK;
}

// Eq. 1, per-community form, as an exact integer numerator over 4m^2:
//   Q = (2m * sum_c sigma_c - sum_c Sigma_c^2) / (2m)^2
// sigma_c sums the arcs (i, j) with C_i = C_j = c (both directions of an edge).
void modularity_parts(const Graph& G, const std::vector<uint32_t>& C,
                      const std::vector<int64_t>& K, int64_t m2, i128* num, i128* den) {
  size_t labels = 0;
  for (uint32_t c : C) labels = std::max<size_t>(labels, size_t(c) + 1);
  std::vector<int64_t> sigma(labels, 0);
  std::vector<int64_t> Sig = community_totals(C, K, labels);
  for (size_t i = 0; i < G.size(); ++i)
    for (const Arc& a : G[i])
      if (C[i] == C[a.j]) sigma[C[i]] += int64_t(a.w);
  i128 s1 = 0, s2 = 0;
  for (size_t c = 0; c < labels; ++c) {
    s1 += sigma[c];
    s2 += i128(Sig[c]) * i128(Sig[c]);
  }
  *num = i128(m2) * s1 - s2;
  *den = i128(m2) * i128(m2);
}

void put_i128(i128 x, int64_t* out) {
  out[0] = int64_t(uint64_t(u128(x) >> 64));
  out[1] = int64_t(uint64_t(u128(x)));
}

}  // namespace

// ===========================================================================
// C ABI used by the Python test harness (ctypes).  Every call returns 0 or a
// negative error code; the state is unchanged on error.
// ===========================================================================
extern "C" {

// flags bit 0: accept self-loops (tests of super-vertex-like graphs only).
void* orc_create_ex(uint32_t n, const uint64_t* off, const uint32_t* idx, const uint32_t* w,
                    uint32_t flags, int* status) {
  *status = OK;
  Oracle* o = new (std::nothrow) Oracle();
  if (!o) { *status = E_NOMEM; return nullptr; }
  o->n = n;
  o->G.assign(n, {});
  int64_t total = 0;
  for (uint32_t i = 0; i < n; ++i) {
    if (off[i + 1] < off[i]) { *status = E_INVALID; break; }
    for (uint64_t k = off[i]; k < off[i + 1]; ++k) {
      uint32_t j = idx[k];
      if (j >= n || (j == i && !(flags & 1u)) || w[k] == 0) { *status = E_INVALID; break; }
      o->G[i].push_back({j, w[k]});
      total += w[k];
    }
    if (*status) break;
    std::sort(o->G[i].begin(), o->G[i].end(),
              [](const Arc& a, const Arc& b) { return a.j < b.j; });
    for (size_t k = 1; k < o->G[i].size(); ++k)
      if (o->G[i][k].j == o->G[i][k - 1].j) *status = E_INVALID;  // duplicate arc
  }
  if (!*status) {  // symmetric with equal weights
    for (uint32_t i = 0; i < n && !*status; ++i)
      for (const Arc& a : o->G[i]) {
        long p = find_arc(o->G[a.j], i);
        if (p < 0 || o->G[a.j][p].w != a.w) { *status = E_INVALID; break; }
      }
  }
  if (!*status && total >= kTwoMLimit) *status = E_OVERFLOW;
  if (*status) { delete o; return nullptr; }
  o->m2 = total;
  o->K = weighted_degrees(o->G);
  return o;
}

void* orc_create(uint32_t n, const uint64_t* off, const uint32_t* idx, const uint32_t* w,
                 int* status) {
  return orc_create_ex(n, off, idx, w, 0u, status);
}

void orc_destroy(void* h) { delete static_cast<Oracle*>(h); }

int orc_set_options(void* h, uint32_t max_iterations, uint32_t max_passes, uint64_t tau_num,
                    uint64_t tau_den, uint64_t tolerance_drop, double tau_agg,
                    uint32_t substeps) {
  Oracle* o = static_cast<Oracle*>(h);
  if (max_iterations == 0 || max_passes == 0 || tau_den == 0 || tolerance_drop == 0)
    return E_INVALID;
  if (substeps != 1 && substeps != 2 && substeps != 4 && substeps != 8) return E_INVALID;
  o->opt.substeps = substeps;
  o->opt.max_iterations = max_iterations;
  o->opt.max_passes = max_passes;
  o->opt.tau_num = tau_num;
  o->opt.tau_den = tau_den;
  o->opt.tolerance_drop = tolerance_drop;
  o->opt.tau_agg = tau_agg;
  return OK;
}

// Static Louvain: K from scratch, singleton communities, every vertex affected.
int orc_static(void* h) {
  Oracle* o = static_cast<Oracle*>(h);
  o->K = weighted_degrees(o->G);
  o->m2 = 0;
  for (int64_t k : o->K) o->m2 += k;
  std::vector<uint32_t> C0(o->n);
  for (uint32_t i = 0; i < o->n; ++i) C0[i] = i;
  o->Sigma = o->K;
  std::vector<char> F(o->n, 1), R(o->n, 1);
  o->C = louvain(*o, C0, o->Sigma, F, R);
  o->have_communities = true;
  o->pend_del.clear();
  o->pend_ins.clear();
  return OK;
}

int orc_apply_batch(void* h, const uint32_t* del, uint64_t nd, const uint32_t* ins, uint64_t ni) {
  return apply_batch(*static_cast<Oracle*>(h), del, nd, ins, ni);
}

int orc_update(void* h, int mode) {
  Oracle* o = static_cast<Oracle*>(h);
  if (!o->have_communities) return E_STATE;
  std::vector<char> F, R;
  if (mode == MODE_ND) mark_naive_dynamic(*o, F, R);
  else if (mode == MODE_DS) mark_delta_screening(*o, F, R);
  else if (mode == MODE_DF) mark_dynamic_frontier(*o, F, R);
  else return E_INVALID;
  std::vector<uint32_t> Cprev = o->C;
  o->C = louvain(*o, Cprev, o->Sigma, F, R);
  o->pend_del.clear();
  o->pend_ins.clear();
  return OK;
}

// Initial frontier of `mode` for the pending batch, without running Louvain.
int orc_mark(void* h, int mode, uint8_t* F_out, uint8_t* R_out) {
  Oracle* o = static_cast<Oracle*>(h);
  if (!o->have_communities) return E_STATE;
  std::vector<char> F, R;
  if (mode == MODE_ND) mark_naive_dynamic(*o, F, R);
  else if (mode == MODE_DS) mark_delta_screening(*o, F, R);
  else if (mode == MODE_DF) mark_dynamic_frontier(*o, F, R);
  else return E_INVALID;
  for (uint32_t i = 0; i < o->n; ++i) {
    F_out[i] = F[i] ? 1 : 0;
    R_out[i] = R[i] ? 1 : 0;
  }
  return OK;
}

// Replace the membership (tests only): K and Sigma recomputed from scratch,
// pending batch cleared.
int orc_set_membership(void* h, const uint32_t* C) {
  Oracle* o = static_cast<Oracle*>(h);
  for (uint32_t i = 0; i < o->n; ++i)
    if (C[i] >= o->n) return E_INVALID;
  o->C.assign(C, C + o->n);
  o->K = weighted_degrees(o->G);
  o->m2 = 0;
  for (int64_t k : o->K) o->m2 += k;
  o->Sigma = community_totals(o->C, o->K, o->n);
  o->have_communities = true;
  o->pend_del.clear();
  o->pend_ins.clear();
  return OK;
}

// Run Louvain from the current membership with an explicit initial frontier
// F0 and range R0 (tests only; e.g. DF with every vertex affected).
int orc_louvain_from(void* h, const uint8_t* F0, const uint8_t* R0) {
  Oracle* o = static_cast<Oracle*>(h);
  if (!o->have_communities) return E_STATE;
  std::vector<char> F(F0, F0 + o->n), R(R0, R0 + o->n);
  std::vector<uint32_t> Cprev = o->C;
  o->C = louvain(*o, Cprev, o->Sigma, F, R);
  o->pend_del.clear();
  o->pend_ins.clear();
  return OK;
}

// One local-moving iteration (all sub-steps) on G^t with the current membership,
// frontier F (in/out: becomes the next frontier) and range R.  Membership and
// Sigma are updated; `moved` gets 1 for each mover.  dq[2] = hi, lo of S.
int orc_move_iteration(void* h, uint8_t* F, const uint8_t* R, uint8_t* moved, int64_t* dq) {
  Oracle* o = static_cast<Oracle*>(h);
  if (!o->have_communities) return E_STATE;
  std::vector<char> Fv(F, F + o->n), Rv(R, R + o->n);
  std::vector<int64_t> sizes = community_sizes(o->C, o->n);
  std::vector<uint32_t> before = o->C;
  Options saved = o->opt;
  o->opt.max_iterations = 1;
  o->trace.clear();
  louvain_move(*o, o->G, o->C, o->K, o->Sigma, sizes, Fv, Rv, 0, nullptr);
  o->opt = saved;
  for (uint32_t i = 0; i < o->n; ++i) {
    F[i] = Fv[i] ? 1 : 0;
    moved[i] = (before[i] != o->C[i]) ? 1 : 0;
  }
  put_i128(i128(o->trace.empty() ? 0 : o->trace[0].dq_sum), dq);
  return OK;
}

// 2m^2 * dQ_{i:C_i->c} (Eq. 2) for the current state, as hi, lo int64.
int orc_delta_q_num(void* h, uint32_t i, uint32_t c, int64_t* out) {
  Oracle* o = static_cast<Oracle*>(h);
  if (!o->have_communities || i >= o->n || c >= o->n) return E_INVALID;
  DenseTable H(o->n);
  scan_communities(H, o->G, o->C, i, false);
  uint32_t d = o->C[i];
  i128 v = score_of(o->m2, H.get(c), o->K[i], o->Sigma[c]) -
           stay_of(o->m2, H.get(d), o->K[i], o->Sigma[d]);
  put_i128(v, out);
  return OK;
}

// Aggregate G^t with the current membership (renumbered ascending) and
// export the super-vertex graph as CSR.  Call with off == nullptr to get the
// sizes in *nv, *na.
int orc_aggregate(void* h, uint32_t* nv, uint64_t* na, uint64_t* off, uint32_t* idx,
                  uint64_t* w) {
  Oracle* o = static_cast<Oracle*>(h);
  if (!o->have_communities) return E_STATE;
  std::vector<char> used(o->n, 0);
  for (uint32_t c : o->C) used[c] = 1;
  std::vector<uint32_t> newid(o->n, 0);
  uint32_t ncomm = 0;
  for (uint32_t c = 0; c < o->n; ++c)
    if (used[c]) newid[c] = ncomm++;
  std::vector<uint32_t> Cr(o->n);
  for (uint32_t i = 0; i < o->n; ++i) Cr[i] = newid[o->C[i]];
  Graph Gs = louvain_aggregate(o->G, Cr, ncomm);
  uint64_t arcs = 0;
  for (const auto& r : Gs) arcs += r.size();
  *nv = ncomm;
  *na = arcs;
  if (!off) return OK;
  uint64_t k = 0;
  off[0] = 0;
  for (uint32_t c = 0; c < ncomm; ++c) {
    for (const Arc& a : Gs[c]) {
      idx[k] = a.j;
      w[k] = a.w;
      ++k;
    }
    off[c + 1] = k;
  }
  return OK;
}

uint64_t orc_num_arcs(void* h) {
  Oracle* o = static_cast<Oracle*>(h);
  uint64_t a = 0;
  for (const auto& r : o->G) a += r.size();
  return a;
}

// Current graph as CSR with sorted rows (off: n+1, idx/w: num_arcs).
int orc_graph(void* h, uint64_t* off, uint32_t* idx, uint32_t* w) {
  Oracle* o = static_cast<Oracle*>(h);
  uint64_t k = 0;
  off[0] = 0;
  for (uint32_t i = 0; i < o->n; ++i) {
    for (const Arc& a : o->G[i]) {
      idx[k] = a.j;
      w[k] = uint32_t(a.w);
      ++k;
    }
    off[i + 1] = k;
  }
  return OK;
}

int orc_membership(void* h, uint32_t* out) {
  Oracle* o = static_cast<Oracle*>(h);
  if (!o->have_communities) return E_STATE;
  std::memcpy(out, o->C.data(), sizeof(uint32_t) * o->n);
  return OK;
}

// K, Sigma (n each) and 2m.
int orc_weights(void* h, int64_t* K, int64_t* Sigma, int64_t* m2) {
  Oracle* o = static_cast<Oracle*>(h);
  if (!o->have_communities) return E_STATE;
  std::memcpy(K, o->K.data(), sizeof(int64_t) * o->n);
  std::memcpy(Sigma, o->Sigma.data(), sizeof(int64_t) * o->n);
  *m2 = o->m2;
  return OK;
}

// Modularity of the current membership (Eq. 1).  parts = {num_hi, num_lo,
// den_hi, den_lo}; *q = double(num) / double(den), 0 when 2m = 0.
int orc_modularity(void* h, double* q, int64_t* parts) {
  Oracle* o = static_cast<Oracle*>(h);
  if (!o->have_communities) return E_STATE;
  i128 num, den;
  modularity_parts(o->G, o->C, o->K, o->m2, &num, &den);
  put_i128(num, parts);
  put_i128(den, parts + 2);
  *q = den == 0 ? 0.0 : double(num) / double(den);
  return OK;
}

// Statistics of the last louvain() run.
//   out[0] passes, out[1] affected at start, out[2] affected ever (pass 0),
//   out[3] number of pass-0 iterations recorded, out[4..4+passes) iterations per pass.
int orc_stats(void* h, uint64_t* out, uint32_t cap) {
  Oracle* o = static_cast<Oracle*>(h);
  if (cap < 4) return E_INVALID;
  out[0] = o->pass_iterations.size();
  out[1] = o->affected_initial;
  out[2] = o->affected_ever;
  out[3] = o->trace.size();
  for (size_t p = 0; p < o->pass_iterations.size() && 4 + p < cap; ++p)
    out[4 + p] = o->pass_iterations[p];
  return OK;
}

// Pass-0 trace: per iteration {frontier, movers, S_hi, S_lo}.
int orc_trace(void* h, uint64_t* out, uint32_t cap_iters) {
  Oracle* o = static_cast<Oracle*>(h);
  for (size_t t = 0; t < o->trace.size() && t < cap_iters; ++t) {
    out[4 * t + 0] = o->trace[t].frontier;
    out[4 * t + 1] = o->trace[t].movers;
    out[4 * t + 2] = uint64_t(o->trace[t].dq_sum >> 64);
    out[4 * t + 3] = uint64_t(o->trace[t].dq_sum);
  }
  return OK;
}

const char* orc_last_error(void* h) { return static_cast<Oracle*>(h)->err.c_str(); }

}  // extern "C"
