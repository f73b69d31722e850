// C ABI of libdfl.so (declared in include/dfl.h): handle lifetime, argument
// checks, copies between caller buffers and the device, statistics and
// profiling.  The algorithmic work lives in the other translation units.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>

#include "common.cuh"

namespace dfl {

namespace {
std::atomic<long long> g_fail_after{-1};  // allocations left before they fail (-1: never)
}  // namespace

cudaError_t dev_malloc_bytes(void** p, size_t bytes) {
  long long k = g_fail_after.load();
  while (k >= 0) {
    if (k == 0) {
      *p = nullptr;
      return cudaErrorMemoryAllocation;
    }
    if (g_fail_after.compare_exchange_weak(k, k - 1)) break;
  }
  return cudaMalloc(p, bytes);
}

int set_error(Handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

int check_launch(Handle* h, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(h, DFL_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return DFL_OK;
}

// Record a timing event; inside a stream capture it must become an event
// record node of the graph (an external record), not a dependency marker.
cudaError_t record_timing_event(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) == cudaSuccess && st == cudaStreamCaptureStatusActive)
    return cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  return cudaEventRecord(e, s);
}

cudaEvent_t take_event(Handle* h) {
  cudaEvent_t e = nullptr;
  if (!h->ev_free.empty()) {
    e = h->ev_free.back();
    h->ev_free.pop_back();
  } else if (cudaEventCreate(&e) != cudaSuccess) {
    e = nullptr;
  }
  return e;
}

LaunchScope::LaunchScope(Handle* h_, int cls_, cudaStream_t s_) : h(h_), cls(cls_), s(s_) {
  h->launches++;
  h->prof.launches[cls]++;
  if ((h->opt.flags & DFL_FLAG_PROFILE) || ((h->opt.flags & DFL_FLAG_PROFILE_MOVE) && cls == DFL_PROF_MOVE)) {
    a = take_event(h);
    b = take_event(h);
    if (a) record_timing_event(a, s);
  }
}

LaunchScope::~LaunchScope() {
  if (a && b) {
    record_timing_event(b, s);
    h->ev_pending.push_back(Handle::Ev{a, b, cls});
  } else {
    if (a) h->ev_free.push_back(a);
    if (b) h->ev_free.push_back(b);
  }
}

namespace {

__global__ void k_check_labels(uint32_t n, const uint32_t* __restrict__ C, Ctrl* ctrl) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n;
       i += uint64_t(gridDim.x) * blockDim.x)
    if (C[i] >= n) atomicOr(&ctrl->err, kErrInvalid);
}

__global__ void k_lists_to_bytes(const uint32_t* __restrict__ lists, Segs seg, uint32_t k,
                                 const unsigned int* __restrict__ counts, uint8_t* __restrict__ out) {
  for (uint32_t key = 0; key < k * kBins; ++key) {
    uint32_t c = counts[key];
    const uint32_t* l = lists + seg.off[key];
    for (uint64_t t = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; t < c;
         t += uint64_t(gridDim.x) * blockDim.x)
      out[l[t]] = 1;
  }
}

__global__ void k_moved(uint32_t n, const uint32_t* __restrict__ a, const uint32_t* __restrict__ b,
                        uint8_t* __restrict__ out) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n;
       i += uint64_t(gridDim.x) * blockDim.x)
    out[i] = a[i] != b[i];
}

__global__ void k_relabel_copy(uint32_t n, const uint32_t* __restrict__ C, const uint32_t* __restrict__ newid,
                               uint32_t* __restrict__ out) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n;
       i += uint64_t(gridDim.x) * blockDim.x)
    out[i] = newid[C[i]];
}

template <typename T>
int alloc(Handle* h, T** p, uint64_t count) {
  if (count == 0) count = 1;
  DFL_CUDA(h, dev_malloc(p, sizeof(T) * count));
  return DFL_OK;
}

void free_all(Handle* h) {
  for (auto& row : h->igraph)
    for (auto& g : row) destroy_iteration_graph(g);
  void* ptrs[] = {h->off, h->deg, h->cap, h->srt, h->ntomb, h->b_newtomb, h->b_cum, h->b_rebuild, h->arcs, h->K, h->Sigma, h->csize, h->C, h->pend_key,
                  h->pend_w, h->Ctop, h->Cs, h->Ks, h->Ss, h->sizes, h->used, h->cnt, h->tdeg,
                  h->fillc, h->members, h->fbits[0], h->fbits[1], h->rbits, h->ever, h->lists[0],
                  h->lists[1], h->mv_i, h->mv_c, h->mv_d, h->dsV, h->dsE, h->dsC, h->b_key, h->b_w,
                  h->b_key2, h->b_w2, h->b_rowlist, h->b_pos, h->b_wnew, h->b_flag, h->b_delta,
                  h->b_newdeg, h->b_edges, h->scratch, h->tmp, h->gtable, h->ctrl,
                  h->g_toff, h->g_loff, h->g_cpre, h->g_ndist, h->g_done, h->g_hd, h->g_res,
                  h->g_tkeys, h->g_tvals, h->g_tlist,
                  h->h_keys, h->h_ndel, h->h_wdel, h->h_wins, h->h_slot, h->h_wnew, h->h_flag,
                  h->h_delta, h->h_pairs, h->r_app, h->r_tomb, h->r_live, h->r_state, h->r_reg,
                  h->h_rows, h->h_extra,
                  h->sg[0].off, h->sg[0].deg, h->sg[0].arcs, h->sg[1].off, h->sg[1].deg,
                  h->sg[1].arcs, h->d_goff0, h->d_goff, h->d_gnext, h->d_gm2, h->d_gdone,
                  h->d_gflag, h->d_gS, h->d_gsum, h->Cfin, h->gb_edges, h->d_eoff, h->bigmv,
                  h->aggq};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->hctrl) cudaFreeHost(h->hctrl);
  if (h->h_gdone) cudaFreeHost(h->h_gdone);
  if (h->h_gS) cudaFreeHost(h->h_gS);
  for (int k = 0; k < kBins - 1; ++k) {
    if (h->aux[k]) cudaStreamDestroy(h->aux[k]);
    if (h->ev_join[k]) cudaEventDestroy(h->ev_join[k]);
  }
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  for (auto& e : h->ev_pending) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  for (auto e : h->ev_free) cudaEventDestroy(e);
}

int check_options(const dfl_options* o) {
  if (o->max_iterations == 0 || o->max_passes == 0 || o->tau_den == 0 || o->tolerance_drop == 0)
    return DFL_ERR_INVALID;
  if (o->substeps != 1 && o->substeps != 2 && o->substeps != 4 && o->substeps != 8)
    return DFL_ERR_INVALID;
  if (!std::isfinite(o->tau_agg)) return DFL_ERR_INVALID;
  return DFL_OK;
}

int read_ctrl(Handle* h) {
  DFL_CUDA(h, cudaMemcpyAsync(h->hctrl, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
  DFL_CUDA(h, cudaStreamSynchronize(h->stream));
  return DFL_OK;
}

int copy_out(Handle* h, void* dst, const void* src, uint64_t bytes, int mem_kind) {
  if (!bytes) return DFL_OK;
  DFL_CUDA(h, cudaMemcpyAsync(dst, src, bytes,
                              mem_kind == DFL_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                                         : cudaMemcpyDeviceToHost,
                              h->stream));
  return DFL_OK;
}

int copy_in(Handle* h, void* dst, const void* src, uint64_t bytes, int mem_kind) {
  if (!bytes) return DFL_OK;
  DFL_CUDA(h, cudaMemcpyAsync(dst, src, bytes,
                              mem_kind == DFL_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                                         : cudaMemcpyHostToDevice,
                              h->stream));
  return DFL_OK;
}

// Frontier from a byte mask into list buffer 0 and the range into rbits.
int frontier_from_bytes(Handle* h, const uint8_t* F, const uint8_t* R, int mem_kind, uint64_t* initial) {
  const uint32_t n = h->n;
  uint8_t* tmpb = nullptr;
  DFL_TRY(alloc(h, &tmpb, n));
  int rc = copy_in(h, tmpb, F, n, mem_kind);
  DFL_CUDA(h, cudaMemsetAsync(h->ctrl, 0, sizeof(Ctrl), h->stream));
  DFL_CUDA(h, cudaMemsetAsync(h->fbits[0], 0, sizeof(uint32_t) * h->words, h->stream));
  DFL_CUDA(h, cudaMemsetAsync(h->fbits[1], 0, sizeof(uint32_t) * h->words, h->stream));
  if (!rc) rc = bytes_to_bits(h, tmpb, h->dsV, n);
  if (!rc) rc = copy_in(h, tmpb, R, n, mem_kind);
  if (!rc) rc = bytes_to_bits(h, tmpb, h->rbits, n);
  if (!rc) rc = lists_from_bits(h, h->dsV, n, h->deg, 0, h->opt.substeps);
  if (!rc) *initial = popcount_bits(h, h->dsV, h->words, &rc);
  cudaStreamSynchronize(h->stream);
  cudaFree(tmpb);
  return rc;
}

}  // namespace

}  // namespace dfl

using dfl::Handle;

struct dfl_handle : public Handle {};

extern "C" {

void dfl_default_options(dfl_options* o) {
  if (!o) return;
  o->max_iterations = 20;
  o->max_passes = 10;
  o->tau_num = 1;
  o->tau_den = 100;
  o->tolerance_drop = 10;
  o->tau_agg = 0.8;
  o->substeps = 4;
  o->flags = 0;
}

}  // extern "C"

namespace dfl {
namespace {

// Everything of dfl_create after the handle exists (a group sets its graph
// ranges first).  On failure the caller frees the handle.
int create_common(Handle* h, uint32_t n, const uint64_t* offsets, const uint32_t* indices,
                  const uint32_t* weights, uint64_t nnz, int mem_kind, const dfl_options* opt,
                  void* cuda_stream) {
  dfl_default_options(&h->opt);
  if (opt) {
    if (check_options(opt)) return DFL_ERR_INVALID;
    h->opt = *opt;
  }
  std::memset(&h->stats, 0, sizeof(h->stats));
  std::memset(&h->prof, 0, sizeof(h->prof));
  h->n = n;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaGetDevice(&h->device);
  h->words = (n + 31) / 32;
  uint32_t b = 1;
  while (b < 31 && (1u << b) < n) ++b;
  h->key_shift = b;
  h->key_bits = 2 * b + 1;
  int rc = DFL_OK;
  auto A = [&](auto** p, uint64_t cnt) {
    if (!rc) rc = alloc(h, p, cnt);
  };
  A(&h->off, uint64_t(n) + 1);
  A(&h->deg, n);
  A(&h->cap, n);
  A(&h->srt, n);
  A(&h->ntomb, n);
  A(&h->K, n);
  A(&h->Sigma, n);
  A(&h->csize, n);
  A(&h->C, n);
  A(&h->Ctop, n);
  A(&h->Cs, n);
  A(&h->Ks, n);
  A(&h->Ss, n);
  A(&h->sizes, n);
  A(&h->used, uint64_t(n) + 1);
  A(&h->cnt, uint64_t(n) + 1);
  A(&h->fillc, n);
  A(&h->members, n);
  A(&h->fbits[0], h->words);
  A(&h->fbits[1], h->words);
  A(&h->rbits, h->words);
  A(&h->ever, h->words);
  A(&h->dsV, h->words);
  A(&h->dsE, h->words);
  A(&h->dsC, h->words);
  A(&h->lists[0], uint64_t(kBins) * n);
  A(&h->lists[1], uint64_t(kBins) * n);
  A(&h->mv_i, n);
  A(&h->mv_c, n);
  A(&h->mv_d, n);
  A(&h->ctrl, 3);  // local-moving's, then the two of the batch apply
  if (!rc) {
    h->actrl = h->ctrl + 1;
    if (cudaMemsetAsync(h->ctrl, 0, 3 * sizeof(Ctrl), h->stream) != cudaSuccess)
      rc = set_error(h, DFL_ERR_CUDA, "control blocks");
  }
  if (!rc && cudaMallocHost(&h->hctrl, 3 * sizeof(Ctrl)) != cudaSuccess) {
    h->hctrl = nullptr;
    rc = set_error(h, DFL_ERR_NOMEM, "pinned control block");
  }
  if (!rc) h->hactrl = h->hctrl + 1;
  // input graph on the device
  unsigned long long* doff = nullptr;
  uint32_t *didx = nullptr, *dw = nullptr;
  if (!rc) {
    if (mem_kind == DFL_MEM_DEVICE) {
      doff = (unsigned long long*)offsets;
      didx = (uint32_t*)indices;
      dw = (uint32_t*)weights;
    } else {
      A(&doff, uint64_t(n) + 1);
      A(&didx, nnz);
      A(&dw, nnz);
      if (!rc) rc = copy_in(h, doff, offsets, sizeof(uint64_t) * (uint64_t(n) + 1), DFL_MEM_HOST);
      if (!rc) rc = copy_in(h, didx, indices, sizeof(uint32_t) * nnz, DFL_MEM_HOST);
      if (!rc) rc = copy_in(h, dw, weights, sizeof(uint32_t) * nnz, DFL_MEM_HOST);
    }
  }
  if (!rc) rc = graph_build(h, doff, didx, dw, nnz);
  if (mem_kind != DFL_MEM_DEVICE) {
    cudaStreamSynchronize(h->stream);
    cudaFree(doff);
    cudaFree(didx);
    cudaFree(dw);
  }
  if (!rc) rc = weighted_degrees(h);
  if (!rc) rc = (cudaStreamSynchronize(h->stream) == cudaSuccess) ? DFL_OK : DFL_ERR_CUDA;
  return rc;
}

// Group membership of graph g: labels moved to [0, n_g).
__global__ void k_local_labels(uint32_t v0, uint32_t cnt, const uint32_t* __restrict__ C,
                               uint32_t* __restrict__ out) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < cnt;
       i += uint64_t(gridDim.x) * blockDim.x)
    out[i] = C[v0 + i] - v0;
}

// A group batch in union ids: edge e of the staged array belongs to the
// graph whose range of eoff holds e; ids are checked against that graph's
// size and shifted to its range; inserted weight is summed per graph.
__global__ void k_group_edges(dfl_edge* __restrict__ e, uint64_t cnt, const uint64_t* __restrict__ eoff,
                              uint32_t ng, const uint32_t* __restrict__ goff0, bool ins,
                              unsigned long long* __restrict__ insw, Ctrl* ctrl) {
  for (uint64_t t = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; t < cnt;
       t += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t pos = eoff[0] + t;
    uint32_t lo = 0, hi = ng;  // largest g with eoff[g] <= pos
    while (hi - lo > 1) {
      uint32_t mid = (lo + hi) >> 1;
      if (eoff[mid] <= pos) lo = mid;
      else hi = mid;
    }
    const uint32_t g = lo, base = goff0[g], size = goff0[g + 1] - base;
    dfl_edge x = e[t];
    if (x.u >= size || x.v >= size) {
      atomicOr(&ctrl->err, kErrInvalid);
      continue;
    }
    x.u += base;
    x.v += base;
    e[t] = x;
    if (ins) atomicAdd(insw + g, (unsigned long long)x.w);
  }
}

// A graph whose 2m could reach 2^32 with the batch's insertions: the batch is refused.
__global__ void k_group_check(const unsigned long long* __restrict__ insw, const long long* __restrict__ gm2,
                              uint32_t ng, Ctrl* ctrl) {
  for (uint64_t g = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; g < ng; g += uint64_t(gridDim.x) * blockDim.x)
    if ((unsigned long long)gm2[g] + 2 * insw[g] >= (1ull << 32)) atomicOr(&ctrl->err, kErrOverflow);
}

}  // namespace
}  // namespace dfl

extern "C" {

int dfl_create(dfl_handle** out, uint32_t n, const uint64_t* offsets, const uint32_t* indices,
               const uint32_t* weights, uint64_t nnz, int mem_kind, const dfl_options* opt,
               void* cuda_stream) {
  using namespace dfl;
  if (!out || !offsets || (nnz && (!indices || !weights))) return DFL_ERR_INVALID;
  if (n >= (1u << 31)) return DFL_ERR_INVALID;
  if (mem_kind != DFL_MEM_HOST && mem_kind != DFL_MEM_DEVICE) return DFL_ERR_INVALID;
  *out = nullptr;
  dfl_handle* h = new (std::nothrow) dfl_handle();
  if (!h) return DFL_ERR_NOMEM;
  int rc = create_common(h, n, offsets, indices, weights, nnz, mem_kind, opt, cuda_stream);
  if (rc) {
    free_all(h);
    delete h;
    return rc;
  }
  *out = h;
  return DFL_OK;
}

void dfl_destroy(dfl_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  dfl::free_all(h);
  delete h;
}

int dfl_set_options(dfl_handle* h, const dfl_options* opt) {
  if (!h || !opt) return DFL_ERR_INVALID;
  if (dfl::check_options(opt)) return dfl::set_error(h, DFL_ERR_INVALID, "invalid options");
  h->opt = *opt;
  return DFL_OK;
}

int dfl_set_stream(dfl_handle* h, void* s) {
  if (!h) return DFL_ERR_INVALID;
  h->stream = static_cast<cudaStream_t>(s);
  return DFL_OK;
}

namespace {

// A Louvain run that fails part-way (an allocation, a bounded wait) leaves
// labels, Sigma and sizes of an unfinished pass: the handle keeps its graph
// and K but no communities until dfl_static or dfl_set_membership succeeds.
int louvain_result(dfl::Handle* h, int rc) {
  if (rc != DFL_OK) h->have_communities = false;
  return rc;
}

int static_body(dfl_handle* h) {
  using namespace dfl;
  DFL_TRY(weighted_degrees(h));
  DFL_TRY(iota_u32(h, h->C, h->n));
  DFL_TRY(copy_i64(h, h->Sigma, h->K, h->n));
  DFL_TRY(fill_i32(h, h->csize, 1, h->n));
  h->pend_count = 0;
  h->have_communities = true;
  make_segs(h, h->opt.substeps);
  DFL_CUDA(h, cudaMemsetAsync(h->ctrl, 0, sizeof(Ctrl), h->stream));
  DFL_CUDA(h, cudaMemsetAsync(h->fbits[0], 0, sizeof(uint32_t) * h->words, h->stream));
  DFL_CUDA(h, cudaMemsetAsync(h->fbits[1], 0, sizeof(uint32_t) * h->words, h->stream));
  DFL_TRY(lists_all(h, h->n, h->deg, 0, h->opt.substeps));
  return louvain(h, true, false, h->n);
}

}  // namespace

int dfl_static(dfl_handle* h) {
  if (!h) return DFL_ERR_INVALID;
  if (h->ngraphs) return dfl::set_error(h, DFL_ERR_STATE, "a group handle takes the dfl_group_* calls");
  return louvain_result(h, static_body(h));
}

int dfl_apply_batch(dfl_handle* h, const dfl_edge* del, uint64_t n_del, const dfl_edge* ins,
                    uint64_t n_ins, int mem_kind) {
  if (!h || (n_del && !del) || (n_ins && !ins)) return DFL_ERR_INVALID;
  if (mem_kind != DFL_MEM_HOST && mem_kind != DFL_MEM_DEVICE) return DFL_ERR_INVALID;
  if (h->ngraphs) return dfl::set_error(h, DFL_ERR_STATE, "a group handle takes the dfl_group_* calls");
  return dfl::apply_batch(h, del, n_del, ins, n_ins, mem_kind);
}

int dfl_update(dfl_handle* h, int mode) {
  using namespace dfl;
  if (!h) return DFL_ERR_INVALID;
  if (h->ngraphs) return dfl::set_error(h, DFL_ERR_STATE, "a group handle takes the dfl_group_* calls");
  if (!h->have_communities) return set_error(h, DFL_ERR_STATE, "dfl_update before dfl_static");
  if (mode != DFL_ND && mode != DFL_DS && mode != DFL_DF)
    return set_error(h, DFL_ERR_INVALID, "unknown mode");
  bool all = false, use_range = false;
  uint64_t initial = 0;
  int rc = DFL_OK;
  if (h->opt.flags & DFL_FLAG_RECOMPUTE_AUX) rc = recompute_aux(h);
  if (!rc) rc = mark(h, mode, &all, &use_range, &initial);
  if (!rc) rc = louvain(h, all, use_range, initial);
  h->pend_count = 0;
  return louvain_result(h, rc);
}

int dfl_step(dfl_handle* h, const dfl_edge* del, uint64_t n_del, const dfl_edge* ins, uint64_t n_ins,
             int mem_kind, int mode) {
  using namespace dfl;
  if (!h || (n_del && !del) || (n_ins && !ins)) return DFL_ERR_INVALID;
  if (mem_kind != DFL_MEM_HOST && mem_kind != DFL_MEM_DEVICE) return DFL_ERR_INVALID;
  if (h->ngraphs) return dfl::set_error(h, DFL_ERR_STATE, "a group handle takes the dfl_group_* calls");
  if (!h->have_communities) return set_error(h, DFL_ERR_STATE, "dfl_step before dfl_static");
  if (mode != DFL_ND && mode != DFL_DS && mode != DFL_DF)
    return set_error(h, DFL_ERR_INVALID, "unknown mode");
  // Only a DF update runs behind an apply that has not settled: it marks
  // vertices from the batch alone (nothing, if the batch is not written),
  // while ND and DS would process vertices whatever the batch, and the aux
  // recomputation reads 2m on the host
  if (mode != DFL_DF || (h->opt.flags & DFL_FLAG_RECOMPUTE_AUX) || n_del + n_ins == 0) {
    const int rc = apply_batch(h, del, n_del, ins, n_ins, mem_kind);
    if (rc) return rc;
    return dfl_update(h, mode);
  }
  DFL_TRY(apply_batch_begin(h, del, n_del, ins, n_ins, mem_kind));
  bool all = false, use_range = false;
  uint64_t initial = 0;
  int rc = mark(h, DFL_DF, &all, &use_range, &initial);
  if (!rc) rc = louvain(h, all, use_range, initial);  // its first control read settles the apply
  if (h->papply.active) {  // the update stopped before that read
    int c = copy_apply_ctrl(h);
    if (!c && cudaStreamSynchronize(h->stream) != cudaSuccess) c = set_error(h, DFL_ERR_CUDA, "batch apply");
    if (c) {
      h->papply.active = false;
      return louvain_result(h, c);
    }
    settle_apply(h);
  }
  const int arc = h->papply.rc;
  h->papply.rc = DFL_OK;
  if (arc == DFL_OK) {
    h->pend_count = 0;
    return louvain_result(h, rc);
  }
  if (rc != DFL_OK && rc != arc) return louvain_result(h, rc);
  // The batch was not written, so no vertex was marked and local-moving
  // moved nothing: the handle is as it was before the call.
  if (arc == kApplyRetryGrown || arc == kApplyRetrySorted) {
    // buffers grew, or the sort-based path takes the batch: apply, then update
    rc = apply_batch(h, del, n_del, ins, n_ins, mem_kind);
    if (rc) return rc;
    return dfl_update(h, DFL_DF);
  }
  return arc;  // the batch's error; earlier pending batches stay pending
}

int dfl_membership(const dfl_handle* hc, uint32_t* out, int mem_kind) {
  dfl_handle* h = const_cast<dfl_handle*>(hc);
  if (!h || !out) return DFL_ERR_INVALID;
  if (!h->have_communities) return dfl::set_error(h, DFL_ERR_STATE, "no communities yet");
  DFL_TRY(dfl::copy_out(h, out, h->C, sizeof(uint32_t) * h->n, mem_kind));
  DFL_CUDA(h, cudaStreamSynchronize(h->stream));
  return DFL_OK;
}

int dfl_modularity(dfl_handle* h, double* q, int64_t* parts) {
  using namespace dfl;
  if (!h || !q) return DFL_ERR_INVALID;
  if (h->ngraphs) return dfl::set_error(h, DFL_ERR_STATE, "a group handle takes the dfl_group_* calls");
  if (!h->have_communities) return set_error(h, DFL_ERR_STATE, "no communities yet");
  i128 num = 0, den = 0;
  DFL_TRY(modularity_parts(h, &num, &den));
  *q = den == 0 ? 0.0 : double(num) / double(den);
  if (parts) {
    parts[0] = int64_t(uint64_t((u128)num >> 64));
    parts[1] = int64_t(uint64_t((u128)num));
    parts[2] = int64_t(uint64_t((u128)den >> 64));
    parts[3] = int64_t(uint64_t((u128)den));
  }
  return DFL_OK;
}

int dfl_weights(dfl_handle* h, int64_t* K, int64_t* Sigma, int64_t* two_m, int mem_kind) {
  if (!h) return DFL_ERR_INVALID;
  if (K) DFL_TRY(dfl::copy_out(h, K, h->K, sizeof(int64_t) * h->n, mem_kind));
  if (Sigma) DFL_TRY(dfl::copy_out(h, Sigma, h->Sigma, sizeof(int64_t) * h->n, mem_kind));
  if (two_m) *two_m = h->m2;
  DFL_CUDA(h, cudaStreamSynchronize(h->stream));
  return DFL_OK;
}

int dfl_compact(dfl_handle* h, uint64_t* before, uint64_t* after) {
  if (!h) return DFL_ERR_INVALID;
  return dfl::compact_pool(h, before, after);
}

int dfl_num_arcs(dfl_handle* h, uint64_t* num_arcs) {
  if (!h || !num_arcs) return DFL_ERR_INVALID;
  *num_arcs = h->num_arcs;
  return DFL_OK;
}

int dfl_graph(dfl_handle* h, uint64_t* offsets, uint32_t* indices, uint32_t* weights, int mem_kind) {
  if (!h || !offsets || (h->num_arcs && (!indices || !weights))) return DFL_ERR_INVALID;
  return dfl::graph_export(h, offsets, indices, weights, mem_kind == DFL_MEM_DEVICE);
}

int dfl_stats(dfl_handle* h, dfl_stats_t* s) {
  if (!h || !s) return DFL_ERR_INVALID;
  *s = h->stats;
  s->kernel_launches = h->launches;
  s->num_arcs = h->num_arcs;
  s->arc_pool = h->pool_cap;
  s->max_degree = h->max_deg;
  s->graph_captures = h->graph_captures;
  s->graph_capture_ms = h->graph_capture_ms;
  return DFL_OK;
}

int dfl_profile(dfl_handle* h, dfl_profile_t* p, int reset) {
  if (!h || !p) return DFL_ERR_INVALID;
  for (auto& e : h->ev_pending) {
    float ms = 0;
    if (cudaEventSynchronize(e.b) == cudaSuccess && cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess)
      h->prof.ms[e.cls] += ms;
    h->ev_free.push_back(e.a);
    h->ev_free.push_back(e.b);
  }
  h->ev_pending.clear();
  *p = h->prof;
  if (reset) std::memset(&h->prof, 0, sizeof(h->prof));
  return DFL_OK;
}

int dfl_trace(dfl_handle* h, uint64_t* out, uint32_t cap, uint32_t* len) {
  if (!h || !len) return DFL_ERR_INVALID;
  uint32_t t = uint32_t(h->trace.size() / 4);
  *len = t;
  if (out)
    for (uint32_t k = 0; k < t && k < cap; ++k)
      for (int j = 0; j < 4; ++j) out[4 * k + j] = h->trace[4 * k + j];
  return DFL_OK;
}

const char* dfl_last_error(const dfl_handle* h) { return h ? h->err.c_str() : "null handle"; }

int dfl_set_membership(dfl_handle* h, const uint32_t* C, int mem_kind) {
  using namespace dfl;
  if (!h || !C) return DFL_ERR_INVALID;
  if (h->ngraphs) return dfl::set_error(h, DFL_ERR_STATE, "a group handle takes the dfl_group_* calls");
  DFL_TRY(copy_in(h, h->Cs, C, sizeof(uint32_t) * h->n, mem_kind));
  DFL_CUDA(h, cudaMemsetAsync(h->ctrl, 0, sizeof(Ctrl), h->stream));
  {
    LaunchScope ls(h, DFL_PROF_OTHER);
    k_check_labels<<<grid_for(h->n, 256), 256, 0, h->stream>>>(h->n, h->Cs, h->ctrl);
    DFL_TRY(check_launch(h, "check labels"));
  }
  DFL_TRY(read_ctrl(h));
  if (h->hctrl->err) return set_error(h, DFL_ERR_INVALID, "label >= n");
  DFL_CUDA(h, cudaMemcpyAsync(h->C, h->Cs, sizeof(uint32_t) * h->n, cudaMemcpyDeviceToDevice, h->stream));
  DFL_TRY(weighted_degrees(h));
  DFL_TRY(recompute_sigma_sizes(h, h->C));
  h->pend_count = 0;
  h->have_communities = true;
  DFL_CUDA(h, cudaStreamSynchronize(h->stream));
  return DFL_OK;
}

int dfl_mark(dfl_handle* h, int mode, uint8_t* F, uint8_t* R, int mem_kind) {
  using namespace dfl;
  if (!h || !F || !R) return DFL_ERR_INVALID;
  if (h->ngraphs) return dfl::set_error(h, DFL_ERR_STATE, "a group handle takes the dfl_group_* calls");
  if (!h->have_communities) return set_error(h, DFL_ERR_STATE, "no communities yet");
  if (mode != DFL_ND && mode != DFL_DS && mode != DFL_DF) return set_error(h, DFL_ERR_INVALID, "mode");
  bool all = false, use_range = false;
  uint64_t initial = 0;
  DFL_TRY(mark(h, mode, &all, &use_range, &initial));
  uint8_t* tmpb = nullptr;
  DFL_TRY(alloc(h, &tmpb, h->n));
  int rc = DFL_OK;
  if (all) {
    if (cudaMemsetAsync(tmpb, 1, h->n, h->stream) != cudaSuccess) rc = DFL_ERR_CUDA;
  } else {
    rc = bits_to_bytes(h, mode == DFL_DS ? h->dsV : h->fbits[0], tmpb, h->n);
  }
  if (!rc) rc = copy_out(h, F, tmpb, h->n, mem_kind);
  if (!rc) {
    if (use_range) rc = bits_to_bytes(h, h->rbits, tmpb, h->n);
    else if (cudaMemsetAsync(tmpb, 1, h->n, h->stream) != cudaSuccess) rc = DFL_ERR_CUDA;
  }
  if (!rc) rc = copy_out(h, R, tmpb, h->n, mem_kind);
  cudaStreamSynchronize(h->stream);
  cudaFree(tmpb);
  return rc;
}

int dfl_louvain_from(dfl_handle* h, const uint8_t* F0, const uint8_t* R0, int mem_kind) {
  using namespace dfl;
  if (!h || !F0 || !R0) return DFL_ERR_INVALID;
  if (h->ngraphs) return dfl::set_error(h, DFL_ERR_STATE, "a group handle takes the dfl_group_* calls");
  if (!h->have_communities) return set_error(h, DFL_ERR_STATE, "no communities yet");
  uint64_t initial = 0;
  DFL_TRY(frontier_from_bytes(h, F0, R0, mem_kind, &initial));
  int rc = louvain(h, false, true, initial);
  h->pend_count = 0;
  return rc;
}

int dfl_move_iteration(dfl_handle* h, uint8_t* F, const uint8_t* R, uint8_t* moved, int64_t* dq,
                       int mem_kind) {
  using namespace dfl;
  if (!h || !F || !R || !moved || !dq) return DFL_ERR_INVALID;
  if (h->ngraphs) return dfl::set_error(h, DFL_ERR_STATE, "a group handle takes the dfl_group_* calls");
  if (!h->have_communities) return set_error(h, DFL_ERR_STATE, "no communities yet");
  uint64_t initial = 0;
  DFL_TRY(frontier_from_bytes(h, F, R, mem_kind, &initial));
  DFL_CUDA(h, cudaMemcpyAsync(h->Ctop, h->C, sizeof(uint32_t) * h->n, cudaMemcpyDeviceToDevice, h->stream));
  MoveArgs a;
  a.g = base_view(h);
  a.C = h->C;
  a.K = h->K;
  a.Sigma = h->Sigma;
  a.size = h->csize;
  a.m2 = h->m2;
  a.max_deg = h->max_deg;
  a.use_range = true;
  a.track_ever = false;
  uint32_t saved = h->opt.max_iterations;
  h->opt.max_iterations = 1;
  h->trace.clear();
  uint32_t it = 0;
  int rc = local_move(h, a, 0, &it, true);
  h->opt.max_iterations = saved;
  if (rc) return rc;
  // the next frontier is in list buffer 1 (the last control read has its lengths)
  unsigned int counts[kMaxSubsteps * kBins];
  for (uint32_t s = 0; s < kMaxSubsteps; ++s)
    for (int b = 0; b < kBins; ++b) counts[s * kBins + b] = h->hctrl->count[1][s][b];
  unsigned int* dcounts = nullptr;
  uint8_t* tmpb = nullptr;
  DFL_TRY(alloc(h, &dcounts, kMaxSubsteps * kBins));
  if (alloc(h, &tmpb, h->n)) {
    cudaFree(dcounts);
    return DFL_ERR_NOMEM;
  }
  rc = copy_in(h, dcounts, counts, sizeof(counts), DFL_MEM_HOST);
  if (!rc && cudaMemsetAsync(tmpb, 0, h->n, h->stream) != cudaSuccess) rc = DFL_ERR_CUDA;
  if (!rc) {
    LaunchScope ls(h, DFL_PROF_OTHER);
    k_lists_to_bytes<<<grid_for(h->n, 256), 256, 0, h->stream>>>(h->lists[1], h->segs, h->opt.substeps,
                                                                 dcounts, tmpb);
    rc = check_launch(h, "lists to bytes");
  }
  if (!rc) rc = copy_out(h, F, tmpb, h->n, mem_kind);
  if (!rc) {
    LaunchScope ls(h, DFL_PROF_OTHER);
    k_moved<<<grid_for(h->n, 256), 256, 0, h->stream>>>(h->n, h->Ctop, h->C, tmpb);
    rc = check_launch(h, "moved");
  }
  if (!rc) rc = copy_out(h, moved, tmpb, h->n, mem_kind);
  cudaStreamSynchronize(h->stream);
  cudaFree(tmpb);
  cudaFree(dcounts);
  if (rc) return rc;
  dq[0] = h->trace.size() >= 4 ? int64_t(h->trace[2]) : 0;
  dq[1] = h->trace.size() >= 4 ? int64_t(h->trace[3]) : 0;
  return DFL_OK;
}

int dfl_aggregate(dfl_handle* h, uint32_t* nv, uint64_t* na, uint64_t* offsets, uint32_t* indices,
                  uint64_t* weights) {
  using namespace dfl;
  if (!h || !nv || !na) return DFL_ERR_INVALID;
  if (h->ngraphs) return dfl::set_error(h, DFL_ERR_STATE, "a group handle takes the dfl_group_* calls");
  if (!h->have_communities) return set_error(h, DFL_ERR_STATE, "no communities yet");
  uint32_t ncomm = 0;
  DFL_TRY(count_communities(h, h->C, h->n, &ncomm));
  {
    LaunchScope ls(h, DFL_PROF_OTHER);
    k_relabel_copy<<<grid_for(h->n, 256), 256, 0, h->stream>>>(h->n, h->C, h->used, h->Cs);
    DFL_TRY(check_launch(h, "relabel copy"));
  }
  DFL_TRY(aggregate(h, base_view(h), h->Cs, ncomm, 0, h->Ks));
  const SuperGraph& sg = h->sg[0];
  std::vector<unsigned long long> off(ncomm + 1);
  std::vector<uint32_t> deg(ncomm);
  DFL_CUDA(h, cudaMemcpyAsync(off.data(), sg.off, sizeof(unsigned long long) * (ncomm + 1),
                              cudaMemcpyDeviceToHost, h->stream));
  DFL_CUDA(h, cudaMemcpyAsync(deg.data(), sg.deg, sizeof(uint32_t) * ncomm, cudaMemcpyDeviceToHost,
                              h->stream));
  std::vector<uint2> arcs(off[ncomm] ? off[ncomm] : 1);
  DFL_CUDA(h, cudaStreamSynchronize(h->stream));
  DFL_CUDA(h, cudaMemcpy(arcs.data(), sg.arcs, sizeof(uint2) * off[ncomm], cudaMemcpyDeviceToHost));
  uint64_t total = 0;
  for (uint32_t c = 0; c < ncomm; ++c) total += deg[c];
  *nv = ncomm;
  *na = total;
  if (!offsets) return DFL_OK;
  if (total && (!indices || !weights)) return DFL_ERR_INVALID;
  // inspection output: rows sorted by neighbour on the host
  uint64_t k = 0;
  offsets[0] = 0;
  for (uint32_t c = 0; c < ncomm; ++c) {
    std::vector<uint2> row(arcs.begin() + off[c], arcs.begin() + off[c] + deg[c]);
    std::sort(row.begin(), row.end(), [](const uint2& x, const uint2& y) { return x.x < y.x; });
    for (const uint2& a : row) {
      indices[k] = a.x;
      weights[k] = a.y;
      ++k;
    }
    offsets[c + 1] = k;
  }
  return DFL_OK;
}

int dfl_get_tuning(const dfl_handle* h, dfl_tuning* t) {
  if (!h || !t) return DFL_ERR_INVALID;
  *t = h->tune;
  return DFL_OK;
}

int dfl_set_tuning(dfl_handle* h, const dfl_tuning* t) {
  if (!h || !t) return DFL_ERR_INVALID;
  if (dfl::check_tuning(*t)) return dfl::set_error(h, DFL_ERR_INVALID, "tuning out of range");
  h->tune = *t;
  return DFL_OK;
}

int dfl_autotune(dfl_handle* h, int mode, uint32_t reps, dfl_tuning* chosen, double* ms) {
  using namespace dfl;
  if (!h) return DFL_ERR_INVALID;
  if (!h->have_communities) return set_error(h, DFL_ERR_STATE, "no communities yet");
  if (mode != DFL_ND && mode != DFL_DS && mode != DFL_DF)
    return set_error(h, DFL_ERR_INVALID, "unknown mode");
  double t = 0;
  DFL_TRY(autotune(h, mode, reps, &t));
  if (chosen) *chosen = h->tune;
  if (ms) *ms = t;
  return DFL_OK;
}

int dfl_group_create(dfl_handle** out, uint32_t num_graphs, const uint32_t* n,
                     const uint64_t* const* offsets, const uint32_t* const* indices,
                     const uint32_t* const* weights, const dfl_options* opt, void* cuda_stream) {
  using namespace dfl;
  if (!out || !num_graphs || !n || !offsets || !indices || !weights) return DFL_ERR_INVALID;
  *out = nullptr;
  const uint32_t G = num_graphs;
  // the disjoint union on the host: graph g's vertices start at goff0[g]
  std::vector<uint32_t> goff0(G + 1, 0);
  uint64_t total = 0, nnz = 0;
  for (uint32_t g = 0; g < G; ++g) {
    if (!offsets[g] || (offsets[g][n[g]] && (!indices[g] || !weights[g]))) return DFL_ERR_INVALID;
    total += n[g];
    if (total >= (1ull << 31)) return DFL_ERR_INVALID;
    goff0[g + 1] = uint32_t(total);
    nnz += offsets[g][n[g]];
  }
  std::vector<uint64_t> off(total + 1);
  std::vector<uint32_t> idx(nnz ? nnz : 1), w(nnz ? nnz : 1);
  uint64_t e = 0;
  for (uint32_t g = 0; g < G; ++g) {
    const uint64_t* o = offsets[g];
    const uint64_t base = o[0];
    for (uint32_t i = 0; i < n[g]; ++i) off[goff0[g] + i] = e + (o[i] - base);
    const uint64_t cnt = o[n[g]] - base;
    for (uint64_t k = 0; k < cnt; ++k) {
      idx[e + k] = indices[g][base + k] + goff0[g];
      w[e + k] = weights[g][base + k];
    }
    e += cnt;
  }
  off[total] = e;
  dfl_handle* h = new (std::nothrow) dfl_handle();
  if (!h) return DFL_ERR_NOMEM;
  h->ngraphs = G;
  h->goff0 = goff0;
  h->gm2.assign(G, 0);
  h->gfin.assign(G, 0);
  dfl_stats_t z;
  std::memset(&z, 0, sizeof(z));
  h->gstats.assign(G, z);
  int rc = create_common(h, uint32_t(total), off.data(), idx.data(), w.data(), e, DFL_MEM_HOST, opt,
                         cuda_stream);
  auto A = [&](auto** p, uint64_t cnt) {
    if (!rc) rc = alloc(h, p, cnt);
  };
  A(&h->d_goff0, G + 1);
  A(&h->d_goff, G + 1);
  A(&h->d_gnext, G + 1);
  A(&h->d_gm2, G);
  A(&h->d_gdone, G);
  A(&h->d_gflag, G);
  A(&h->d_gS, 2 * uint64_t(G));
  A(&h->d_gsum, 3 * uint64_t(G));
  A(&h->d_eoff, 2 * (uint64_t(G) + 1));
  A(&h->Cfin, total);
  if (!rc && (cudaMallocHost(&h->h_gdone, G) != cudaSuccess ||
              cudaMallocHost(&h->h_gS, sizeof(unsigned long long) * 2 * G) != cudaSuccess))
    rc = set_error(h, DFL_ERR_NOMEM, "pinned group buffers");
  if (!rc) rc = copy_in(h, h->d_goff0, goff0.data(), sizeof(uint32_t) * (G + 1), DFL_MEM_HOST);
  if (!rc) rc = copy_in(h, h->d_goff, goff0.data(), sizeof(uint32_t) * (G + 1), DFL_MEM_HOST);
  if (!rc) rc = group_m2(h);
  if (rc) {
    free_all(h);
    delete h;
    return rc;
  }
  *out = h;
  return DFL_OK;
}

namespace {

int group_static_body(dfl_handle* h) {
  using namespace dfl;
  DFL_TRY(weighted_degrees(h));
  DFL_TRY(group_m2(h));
  DFL_TRY(iota_u32(h, h->C, h->n));
  DFL_TRY(copy_i64(h, h->Sigma, h->K, h->n));
  DFL_TRY(fill_i32(h, h->csize, 1, h->n));
  h->pend_count = 0;
  h->have_communities = true;
  DFL_TRY(group_set_level(h, h->d_goff0));  // classes of the base graphs' vertices
  make_segs(h, h->opt.substeps);
  DFL_CUDA(h, cudaMemsetAsync(h->ctrl, 0, sizeof(Ctrl), h->stream));
  DFL_CUDA(h, cudaMemsetAsync(h->fbits[0], 0, sizeof(uint32_t) * h->words, h->stream));
  DFL_CUDA(h, cudaMemsetAsync(h->fbits[1], 0, sizeof(uint32_t) * h->words, h->stream));
  DFL_TRY(lists_all(h, h->n, h->deg, 0, h->opt.substeps));
  return louvain_group(h, true, false, h->n);
}

}  // namespace

int dfl_group_static(dfl_handle* h) {
  if (!h) return DFL_ERR_INVALID;
  if (!h->ngraphs) return dfl::set_error(h, DFL_ERR_STATE, "not a group handle");
  return louvain_result(h, group_static_body(h));
}

int dfl_group_apply_batch(dfl_handle* h, const dfl_edge* del, const uint64_t* del_off,
                          const dfl_edge* ins, const uint64_t* ins_off, int mem_kind) {
  using namespace dfl;
  if (!h || !del_off || !ins_off) return DFL_ERR_INVALID;
  if (mem_kind != DFL_MEM_HOST && mem_kind != DFL_MEM_DEVICE) return DFL_ERR_INVALID;
  if (!h->ngraphs) return set_error(h, DFL_ERR_STATE, "not a group handle");
  if (!h->have_communities) return set_error(h, DFL_ERR_STATE, "dfl_group_apply_batch before dfl_group_static");
  const uint32_t G = h->ngraphs;
  for (uint32_t g = 0; g < G; ++g)
    if (del_off[g + 1] < del_off[g] || ins_off[g + 1] < ins_off[g])
      return set_error(h, DFL_ERR_INVALID, "batch offsets must not decrease");
  const uint64_t nd = del_off[G] - del_off[0], ni = ins_off[G] - ins_off[0];
  if ((nd && !del) || (ni && !ins)) return DFL_ERR_INVALID;
  // stage both lists on the device, in union ids
  if (nd + ni > h->gb_cap) {
    cudaStreamSynchronize(h->stream);
    cudaFree(h->gb_edges);
    h->gb_edges = nullptr;
    h->gb_cap = 0;
    const uint64_t want = (nd + ni) + (nd + ni) / 4 + 1024;
    DFL_CUDA(h, dev_malloc(&h->gb_edges, sizeof(dfl_edge) * want));
    h->gb_cap = want;
  }
  dfl_edge* sd = h->gb_edges;
  dfl_edge* si = h->gb_edges + nd;
  DFL_TRY(copy_in(h, sd, del + del_off[0], sizeof(dfl_edge) * nd, mem_kind));
  DFL_TRY(copy_in(h, si, ins + ins_off[0], sizeof(dfl_edge) * ni, mem_kind));
  DFL_TRY(copy_in(h, h->d_eoff, del_off, sizeof(uint64_t) * (G + 1), DFL_MEM_HOST));
  DFL_TRY(copy_in(h, h->d_eoff + G + 1, ins_off, sizeof(uint64_t) * (G + 1), DFL_MEM_HOST));
  DFL_CUDA(h, cudaMemsetAsync(h->ctrl, 0, sizeof(Ctrl), h->stream));
  DFL_CUDA(h, cudaMemsetAsync(h->d_gsum, 0, sizeof(unsigned long long) * G, h->stream));
  if (nd) {
    LaunchScope ls(h, DFL_PROF_APPLY);
    k_group_edges<<<grid_for(nd, 256), 256, 0, h->stream>>>(sd, nd, h->d_eoff, G, h->d_goff0, false,
                                                            h->d_gsum, h->ctrl);
    DFL_TRY(check_launch(h, "group batch"));
  }
  if (ni) {
    LaunchScope ls(h, DFL_PROF_APPLY);
    k_group_edges<<<grid_for(ni, 256), 256, 0, h->stream>>>(si, ni, h->d_eoff + G + 1, G, h->d_goff0,
                                                            true, h->d_gsum, h->ctrl);
    DFL_TRY(check_launch(h, "group batch"));
  }
  {
    LaunchScope ls(h, DFL_PROF_APPLY);
    k_group_check<<<grid_for(G, 256), 256, 0, h->stream>>>(h->d_gsum, h->d_gm2, G, h->ctrl);
    DFL_TRY(check_launch(h, "group batch"));
  }
  // the apply runs only if these checks passed; one wait for everything
  return group_apply(h, sd, nd, si, ni);
}

int dfl_group_update(dfl_handle* h, int mode) {
  using namespace dfl;
  if (!h) return DFL_ERR_INVALID;
  if (!h->ngraphs) return set_error(h, DFL_ERR_STATE, "not a group handle");
  if (!h->have_communities) return set_error(h, DFL_ERR_STATE, "dfl_group_update before dfl_group_static");
  if (mode != DFL_ND && mode != DFL_DS && mode != DFL_DF)
    return set_error(h, DFL_ERR_INVALID, "unknown mode");
  bool all = false, use_range = false;
  uint64_t initial = 0;
  int rc = group_set_level(h, h->d_goff0);  // classes of the base graphs' vertices
  if (!rc && (h->opt.flags & DFL_FLAG_RECOMPUTE_AUX)) rc = recompute_aux(h);
  if (!rc) rc = mark(h, mode, &all, &use_range, &initial);
  if (!rc) rc = louvain_group(h, all, use_range, initial);
  h->pend_count = 0;
  return louvain_result(h, rc);
}

int dfl_group_membership(dfl_handle* h, uint32_t g, uint32_t* out, int mem_kind) {
  using namespace dfl;
  if (!h || !out) return DFL_ERR_INVALID;
  if (!h->ngraphs || g >= h->ngraphs) return set_error(h, DFL_ERR_INVALID, "no such graph");
  if (!h->have_communities) return set_error(h, DFL_ERR_STATE, "no communities yet");
  const uint32_t v0 = h->goff0[g], cnt = h->goff0[g + 1] - v0;
  if (!cnt) return DFL_OK;
  {
    LaunchScope ls(h, DFL_PROF_OTHER);
    k_local_labels<<<grid_for(cnt, 256), 256, 0, h->stream>>>(v0, cnt, h->C, h->Cs);
    DFL_TRY(check_launch(h, "group labels"));
  }
  DFL_TRY(copy_out(h, out, h->Cs, sizeof(uint32_t) * cnt, mem_kind));
  DFL_CUDA(h, cudaStreamSynchronize(h->stream));
  return DFL_OK;
}

int dfl_group_modularity(dfl_handle* h, uint32_t g, double* q, int64_t* parts) {
  using namespace dfl;
  if (!h || !q) return DFL_ERR_INVALID;
  if (!h->ngraphs || g >= h->ngraphs) return set_error(h, DFL_ERR_INVALID, "no such graph");
  if (!h->have_communities) return set_error(h, DFL_ERR_STATE, "no communities yet");
  i128 num = 0, den = 0;
  DFL_TRY(group_modularity(h, g, &num, &den));
  *q = den == 0 ? 0.0 : double(num) / double(den);
  if (parts) {
    parts[0] = int64_t(uint64_t((u128)num >> 64));
    parts[1] = int64_t(uint64_t((u128)num));
    parts[2] = int64_t(uint64_t((u128)den >> 64));
    parts[3] = int64_t(uint64_t((u128)den));
  }
  return DFL_OK;
}

int dfl_group_stats(dfl_handle* h, uint32_t g, dfl_stats_t* s) {
  if (!h || !s) return DFL_ERR_INVALID;
  if (!h->ngraphs || g >= h->ngraphs) return dfl::set_error(h, DFL_ERR_INVALID, "no such graph");
  DFL_TRY(dfl_stats(h, s));
  const dfl_stats_t& q = h->gstats[g];
  s->passes = q.passes;
  for (int p = 0; p < 16; ++p) s->iterations[p] = q.iterations[p];
  s->num_communities = q.num_communities;
  return DFL_OK;
}

}  // extern "C"

extern "C" int dfl_test_fail_allocations(int64_t after) {
  dfl::g_fail_after.store(after < 0 ? -1 : (long long)after);
  return DFL_OK;
}
