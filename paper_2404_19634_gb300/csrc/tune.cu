// Launch-shape tuning of local-moving and its autotuner.
//
// A tuning decides which decide kernel handles a vertex (by degree) and the
// block size of the block-per-vertex kernel; the community table then lives
// in registers, shared memory or a global slice accordingly.  Every kernel
// computes the same exact integer decision, so a tuning changes time only.
//
// The autotuner times the decide phase of one local-moving iteration over
// the real initial frontier of the next update (the frontier dfl_update would
// mark for the pending batch), computing the decisions without applying
// them, and walks one coordinate at a time: block size, then the bin limits
// from the largest down.  A candidate replaces the best only when it is
// faster by more than the noise margin.
#include <algorithm>
#include <cstring>

#include "common.cuh"

namespace dfl {

int check_tuning(const dfl_tuning& t) {
  if (t.bin_warp > kBinWarp) return DFL_ERR_INVALID;
  if (t.bin_warp_hash < t.bin_warp || t.bin_warp_hash > kBinWarpHash) return DFL_ERR_INVALID;
  if (t.bin_block < t.bin_warp_hash) return DFL_ERR_INVALID;
  if (t.block_threads != 128 && t.block_threads != 256 && t.block_threads != 512)
    return DFL_ERR_INVALID;
  return DFL_OK;
}

int autotune(Handle* h, int mode, uint32_t reps, double* best_ms) {
  const uint32_t n = h->n, k = h->opt.substeps;
  if (reps == 0) reps = 1;
  bool all = false, use_range = false;
  uint64_t initial = 0;
  if (h->ngraphs) DFL_TRY(group_set_level(h, h->d_goff0));
  DFL_TRY(mark(h, mode, &all, &use_range, &initial));
  // keep the frontier as a bitmap (the lists are rebuilt for every
  // candidate, whose bin limits sort vertices differently); the first-pass
  // "ever processed" bitmap is free between updates
  if (!all) {
    const uint32_t* fb = mode == DFL_DS ? h->dsV : h->fbits[0];
    DFL_CUDA(h, cudaMemcpyAsync(h->ever, fb, sizeof(uint32_t) * h->words, cudaMemcpyDeviceToDevice,
                                h->stream));
  }
  MoveArgs ma;
  ma.g = base_view(h);
  ma.C = h->C;
  ma.K = h->K;
  ma.Sigma = h->Sigma;
  ma.size = h->csize;
  ma.m2 = h->m2;
  ma.max_deg = h->max_deg;
  ma.use_range = use_range;
  ma.track_ever = false;

  auto measure = [&](const dfl_tuning& t, double* med) -> int {
    h->tune = t;
    make_segs(h, k);
    DFL_CUDA(h, cudaMemsetAsync(h->ctrl, 0, sizeof(Ctrl), h->stream));
    DFL_CUDA(h, cudaMemsetAsync(h->fbits[1], 0, sizeof(uint32_t) * h->words, h->stream));
    if (all) DFL_TRY(lists_all(h, n, h->deg, 0, k));
    else DFL_TRY(lists_from_bits(h, h->ever, n, h->deg, 0, k));
    std::vector<float> ms;
    DFL_TRY(time_decide(h, ma, reps + 1, &ms));
    if (ms.size() > 1) ms.erase(ms.begin());  // the first run warms caches and allocations
    std::sort(ms.begin(), ms.end());
    *med = ms.empty() ? 0.0 : ms[ms.size() / 2];
    return DFL_OK;
  };

  const dfl_tuning start = h->tune;
  dfl_tuning best = start;
  double best_t = 0;
  int rc = measure(best, &best_t);
  const uint32_t threads[] = {128, 256, 512};
  const uint32_t blocks[] = {1024, 2048, 4096, 8192, 16384};
  const uint32_t hashes[] = {64, 128, 256};
  const uint32_t warps[] = {8, 16, 32};
  auto consider = [&](dfl_tuning c) {
    if (rc || check_tuning(c) || std::memcmp(&c, &best, sizeof(c)) == 0) return;
    double t = 0;
    rc = measure(c, &t);
    if (!rc && t < best_t * 0.97) {
      best = c;
      best_t = t;
    }
  };
  for (uint32_t v : threads) {
    dfl_tuning c = best;
    c.block_threads = v;
    consider(c);
  }
  for (uint32_t v : blocks) {
    dfl_tuning c = best;
    c.bin_block = v;
    consider(c);
  }
  for (uint32_t v : hashes) {
    dfl_tuning c = best;
    c.bin_warp_hash = v;
    consider(c);
  }
  for (uint32_t v : warps) {
    dfl_tuning c = best;
    c.bin_warp = v;
    consider(c);
  }
  h->tune = rc ? start : best;
  make_segs(h, k);
  // leave the frontier state as between updates (dfl_update marks again)
  DFL_CUDA(h, cudaMemsetAsync(h->ctrl, 0, sizeof(Ctrl), h->stream));
  DFL_CUDA(h, cudaMemsetAsync(h->fbits[0], 0, sizeof(uint32_t) * h->words, h->stream));
  DFL_CUDA(h, cudaMemsetAsync(h->fbits[1], 0, sizeof(uint32_t) * h->words, h->stream));
  DFL_CUDA(h, cudaMemsetAsync(h->ever, 0, sizeof(uint32_t) * h->words, h->stream));
  DFL_CUDA(h, cudaStreamSynchronize(h->stream));
  if (best_ms) *best_ms = best_t;
  return rc;
}

}  // namespace dfl
