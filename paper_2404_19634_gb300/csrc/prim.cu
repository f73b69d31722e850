// Primitives: exclusive scan, key/value sort, fills, frontier list builders.
#include "common.cuh"

namespace dfl {

namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ T block_exclusive_scan(T v, T* total) {
  __shared__ T warp_sums[kScanThreads / 32];
  const unsigned lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int s = 1; s < 32; s <<= 1) {
    T y = __shfl_up_sync(0xFFFFFFFFu, x, s);
    if (lane >= (unsigned)s) x += y;
  }
  if (lane == 31) warp_sums[w] = x;
  __syncthreads();
  if (w == 0) {
    T s0 = lane < kScanThreads / 32 ? warp_sums[lane] : T(0);
    T t = s0;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
      T y = __shfl_up_sync(0xFFFFFFFFu, t, s);
      if (lane >= (unsigned)s) t += y;
    }
    if (lane < kScanThreads / 32) warp_sums[lane] = t - s0;
    if (lane == kScanThreads / 32 - 1) *total = t;
  }
  __syncthreads();
  T r = x - v + warp_sums[w];
  __syncthreads();
  return r;
}

template <typename T>
__global__ void k_scan_reduce(const T* __restrict__ in, T* __restrict__ part, uint64_t n) {
  __shared__ T tot;
  uint64_t base = uint64_t(blockIdx.x) * kScanTile + threadIdx.x * kScanItems;
  T s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < n) s += in[base + k];
  block_exclusive_scan<T>(s, &tot);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// out[i] = exclusive prefix; out[n] = total when write_total.
template <typename T>
__global__ void k_scan_down(const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ part,
                            uint64_t n, bool write_total) {
  __shared__ T tot;
  uint64_t base = uint64_t(blockIdx.x) * kScanTile + threadIdx.x * kScanItems;
  T v[kScanItems];
  T s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < n) ? in[base + k] : T(0);
    s += v[k];
  }
  T off = block_exclusive_scan<T>(s, &tot);
  T carry = part ? part[blockIdx.x] : T(0);
  off += carry;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = off;
    off += v[k];
  }
  if (write_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = carry + tot;
}

template <typename T>
int scan_impl(Handle* h, const T* in, T* out, uint64_t n, T* scratch, uint64_t scratch_items) {
  if (n == 0) {
    DFL_CUDA(h, cudaMemsetAsync(out, 0, sizeof(T), h->stream));
    return DFL_OK;
  }
  uint64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles == 1) {
    LaunchScope ls(h, DFL_PROF_OTHER);
    k_scan_down<T><<<1, kScanThreads, 0, h->stream>>>(in, out, nullptr, n, true);
    return check_launch(h, "scan");
  }
  if (scratch_items < tiles * 2 + 2) return set_error(h, DFL_ERR_CUDA, "scan scratch too small");
  T* part = scratch;
  T* part_scan = scratch + tiles;
  {
    LaunchScope ls(h, DFL_PROF_OTHER);
    k_scan_reduce<T><<<(unsigned)tiles, kScanThreads, 0, h->stream>>>(in, part, n);
    DFL_TRY(check_launch(h, "scan reduce"));
  }
  DFL_TRY(scan_impl<T>(h, part, part_scan, tiles, scratch + 2 * tiles + 1,
                       scratch_items - 2 * tiles - 1));
  LaunchScope ls(h, DFL_PROF_OTHER);
  k_scan_down<T><<<(unsigned)tiles, kScanThreads, 0, h->stream>>>(in, out, part_scan, n, true);
  return check_launch(h, "scan down");
}

uint64_t scan_scratch_items(uint64_t n) {
  uint64_t total = 0;
  while (n > uint64_t(kScanTile)) {
    uint64_t tiles = (n + kScanTile - 1) / kScanTile;
    total += 2 * tiles + 2;
    n = tiles;
  }
  return total + 4;
}

// ---------------------------------------------------------------------------
// Sort of (u64 key, u32 value) pairs
// ---------------------------------------------------------------------------
constexpr int kSmallSort = 2048;

__global__ void k_bitonic(unsigned long long* key, uint32_t* val, uint32_t n) {
  __shared__ unsigned long long sk[kSmallSort];
  __shared__ uint32_t sv[kSmallSort];
  uint32_t np2 = 1;
  while (np2 < n) np2 <<= 1;
  for (uint32_t i = threadIdx.x; i < np2; i += blockDim.x) {
    sk[i] = i < n ? key[i] : ~0ull;
    sv[i] = i < n ? val[i] : 0u;
  }
  __syncthreads();
  for (uint32_t k = 2; k <= np2; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < np2; i += blockDim.x) {
        uint32_t ixj = i ^ j;
        if (ixj > i) {
          bool up = (i & k) == 0;
          unsigned long long a = sk[i], b = sk[ixj];
          if ((a > b) == up) {
            sk[i] = b;
            sk[ixj] = a;
            uint32_t t = sv[i];
            sv[i] = sv[ixj];
            sv[ixj] = t;
          }
        }
      }
      __syncthreads();
    }
  }
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
    key[i] = sk[i];
    val[i] = sv[i];
  }
}

constexpr int kRadixThreads = 256;
constexpr int kRadixItems = 8;  // per thread
constexpr int kRadixTile = kRadixThreads * kRadixItems;
constexpr int kRadixWarps = kRadixThreads / 32;

// Item position inside a tile: warp w owns [w*256, w*256+256); round r and
// lane l give position w*256 + r*32 + l, so rounds visit items in order.
__device__ __forceinline__ uint32_t radix_pos(uint32_t w, uint32_t r, uint32_t l) {
  return w * (32 * kRadixItems) + r * 32 + l;
}

__global__ void k_radix_hist(const unsigned long long* __restrict__ key, uint64_t n,
                             uint32_t shift, uint32_t* __restrict__ counts, uint32_t nblocks) {
  __shared__ uint32_t hist[256];
  for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[d] = 0;
  __syncthreads();
  uint64_t base = uint64_t(blockIdx.x) * kRadixTile;
  for (int k = threadIdx.x; k < kRadixTile; k += blockDim.x) {
    uint64_t p = base + k;
    if (p < n) atomicAdd(&hist[(key[p] >> shift) & 255u], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += blockDim.x) counts[uint64_t(d) * nblocks + blockIdx.x] = hist[d];
}

__global__ void k_radix_scatter(const unsigned long long* __restrict__ key,
                                const uint32_t* __restrict__ val, unsigned long long* __restrict__ okey,
                                uint32_t* __restrict__ oval, uint64_t n, uint32_t shift,
                                const uint32_t* __restrict__ offs, uint32_t nblocks) {
  __shared__ uint32_t wcnt[kRadixWarps][256];
  const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
  for (int d = lane; d < 256; d += 32) wcnt[w][d] = 0;
  __syncwarp();
  const uint64_t base = uint64_t(blockIdx.x) * kRadixTile;
  const uint32_t lt = (1u << lane) - 1u;
  unsigned long long k_[kRadixItems];
  uint32_t v_[kRadixItems], d_[kRadixItems], rank_[kRadixItems];
#pragma unroll
  for (int r = 0; r < kRadixItems; ++r) {
    uint64_t p = base + radix_pos(w, r, lane);
    bool valid = p < n;
    k_[r] = valid ? key[p] : 0ull;
    v_[r] = valid ? val[p] : 0u;
    uint32_t d = valid ? uint32_t((k_[r] >> shift) & 255u) : 256u;
    d_[r] = d;
    unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
    uint32_t before = valid ? wcnt[w][d] : 0u;
    __syncwarp();
    rank_[r] = before + __popc(peers & lt);
    if (valid && lane == uint32_t(__ffs(peers) - 1)) wcnt[w][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // exclusive prefix of the per-warp counts, per digit, in warp order
  for (int d = threadIdx.x; d < 256; d += blockDim.x) {
    uint32_t run = 0;
    for (int ww = 0; ww < kRadixWarps; ++ww) {
      uint32_t t = wcnt[ww][d];
      wcnt[ww][d] = run;
      run += t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kRadixItems; ++r) {
    if (d_[r] < 256u) {
      uint64_t dst = uint64_t(offs[uint64_t(d_[r]) * nblocks + blockIdx.x]) + wcnt[w][d_[r]] + rank_[r];
      okey[dst] = k_[r];
      oval[dst] = v_[r];
    }
  }
}

// ---------------------------------------------------------------------------
// Fills
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_fill(T* p, T v, uint64_t n) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n;
       i += uint64_t(gridDim.x) * blockDim.x)
    p[i] = v;
}

__global__ void k_iota(uint32_t* p, uint64_t n) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n;
       i += uint64_t(gridDim.x) * blockDim.x)
    p[i] = uint32_t(i);
}

__global__ void k_copy_i64(long long* d, const long long* s, uint64_t n) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n;
       i += uint64_t(gridDim.x) * blockDim.x)
    d[i] = s[i];
}

// ---------------------------------------------------------------------------
// Frontier lists
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_lists_all(uint32_t nv, const uint32_t* __restrict__ deg, uint32_t* lists,
                                                   Segs seg, Ctrl* ctrl, int buf, uint32_t k) {
  // every vertex with arcs, thread per vertex, counted per list key in shared
  // memory and reserved once per block and key
  __shared__ uint32_t s_cnt[kMaxSubsteps * kBins];
  __shared__ uint32_t s_base[kMaxSubsteps * kBins];
  const uint32_t nkeys = k * kBins;
  for (uint64_t i0 = blockIdx.x * uint64_t(blockDim.x); i0 < nv; i0 += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t i = i0 + threadIdx.x;
    // a vertex without arcs has no neighbour community: it is processed
    // (counted) but never queued
    const uint32_t d = i < nv ? deg[i] : 0u;
    const bool valid = i < nv && d > 0;
    const unsigned idle = __ballot_sync(0xFFFFFFFFu, i < nv && d == 0);
    if ((threadIdx.x & 31u) == 0 && idle) atomicAdd(&ctrl->skipped, (unsigned long long)__popc(idle));
    const uint32_t key = valid ? vertex_class(uint32_t(i), k, seg) * kBins + degree_bin(d, seg) : 0u;
    if (threadIdx.x < nkeys) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    if (valid) atomicAdd(&s_cnt[key], 1u);
    __syncthreads();
    if (threadIdx.x < nkeys) {
      const uint32_t c = s_cnt[threadIdx.x];
      s_base[threadIdx.x] = c ? atomicAdd(&ctrl->count[buf][threadIdx.x / kBins][threadIdx.x % kBins], c) : 0u;
      s_cnt[threadIdx.x] = 0;
    }
    __syncthreads();
    if (valid) {
      const uint32_t r = s_base[key] + atomicAdd(&s_cnt[key], 1u);
      if (r < seg.cap[key]) lists[seg.off[key] + r] = uint32_t(i);
      else atomicOr(&ctrl->err, kErrInternal);
    }
    __syncthreads();
  }
}

__global__ void k_bits_to_bytes(const uint32_t* bits, uint8_t* out, uint32_t n) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n;
       i += uint64_t(gridDim.x) * blockDim.x)
    out[i] = (bits[i >> 5] >> (i & 31)) & 1u;
}

__global__ void k_bytes_to_bits(const uint8_t* in, uint32_t* bits, uint32_t n, uint32_t words) {
  for (uint64_t w = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; w < words;
       w += uint64_t(gridDim.x) * blockDim.x) {
    uint32_t x = 0;
    for (int b = 0; b < 32; ++b) {
      uint64_t i = w * 32 + b;
      if (i < n && in[i]) x |= 1u << b;
    }
    bits[w] = x;
  }
}

__global__ void k_popcount(const uint32_t* bits, uint32_t words, unsigned long long* out) {
  unsigned long long s = 0;
  for (uint64_t w = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; w < words;
       w += uint64_t(gridDim.x) * blockDim.x)
    s += __popc(bits[w]);
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

}  // namespace

__global__ void __launch_bounds__(256) k_lists_bits(const uint32_t* __restrict__ bits, uint32_t words,
                                                    uint32_t nv, const uint32_t* __restrict__ deg,
                                                    uint32_t* lists, Segs seg, Ctrl* ctrl, int buf,
                                                    uint32_t k, uint32_t* __restrict__ clear,
                                                    uint32_t clear_words) {
  pdl_wait_only();
  for (uint64_t q = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; q < clear_words;
       q += uint64_t(gridDim.x) * blockDim.x)
    clear[q] = 0u;
  lists_bits_body(bits, words, nv, deg, lists, seg, ctrl, buf, k);
}

// Segment layout for k sub-step classes: class s gets kBins segments, each
// as large as the number of ids in [0, n) of class s (a vertex is in at most
// one segment of a buffer, and a super-vertex graph has ids in [0, nv) with
// nv <= n).
void make_segs(Handle* h, uint32_t k) {
  h->segs.hi[0] = h->tune.bin_warp;
  h->segs.hi[1] = h->tune.bin_warp_hash;
  h->segs.hi[2] = h->tune.bin_block;
  h->segs.goff = h->ngraphs ? h->d_goff : nullptr;
  h->segs.ng = h->ngraphs;
  if (h->segs_k == k) return;
  // a segment holds every vertex of its class; a group's classes come from
  // ids within each graph, and later levels only have fewer vertices per graph
  uint64_t counts[kMaxSubsteps] = {0};
  if (h->ngraphs) {
    for (uint32_t g = 0; g < h->ngraphs; ++g)
      for (uint32_t i = 0; i < h->goff0[g + 1] - h->goff0[g]; ++i) counts[substep_class(i, k)]++;
  } else {
    for (uint32_t i = 0; i < h->n; ++i) counts[substep_class(i, k)]++;
  }
  uint64_t off = 0;
  for (uint32_t c = 0; c < kMaxSubsteps; ++c)
    for (int b = 0; b < kBins; ++b) {
      h->segs.off[c * kBins + b] = uint32_t(off);
      h->segs.cap[c * kBins + b] = c < k ? uint32_t(counts[c]) : 0u;
      off += c < k ? counts[c] : 0;
    }
  h->segs_k = k;
}

int ensure_tmp(Handle* h, uint64_t bytes) {
  if (bytes <= h->tmp_cap) return DFL_OK;
  if (h->tmp) cudaFree(h->tmp);
  h->tmp = nullptr;
  h->tmp_cap = 0;
  uint64_t want = bytes + bytes / 4 + 4096;
  DFL_CUDA(h, dev_malloc(&h->tmp, want));
  h->tmp_cap = want;
  return DFL_OK;
}

int scan_u32(Handle* h, const uint32_t* in, uint32_t* out, uint64_t n) {
  uint64_t items = scan_scratch_items(n);
  DFL_TRY(ensure_tmp(h, items * sizeof(uint32_t)));
  return scan_impl<uint32_t>(h, in, out, n, static_cast<uint32_t*>(h->tmp), items);
}

int scan_u64(Handle* h, const unsigned long long* in, unsigned long long* out, uint64_t n) {
  uint64_t items = scan_scratch_items(n);
  DFL_TRY(ensure_tmp(h, items * sizeof(unsigned long long)));
  return scan_impl<unsigned long long>(h, in, out, n, static_cast<unsigned long long*>(h->tmp),
                                       items);
}

int sort_pairs(Handle* h, unsigned long long* key, uint32_t* val, unsigned long long* key2,
               uint32_t* val2, uint64_t n, uint32_t bits) {
  if (n <= 1) return DFL_OK;
  if (n <= uint64_t(kSmallSort)) {
    LaunchScope ls(h, DFL_PROF_APPLY);
    k_bitonic<<<1, 1024, 0, h->stream>>>(key, val, uint32_t(n));
    return check_launch(h, "bitonic sort");
  }
  uint32_t nblocks = uint32_t((n + kRadixTile - 1) / kRadixTile);
  uint64_t ncounts = uint64_t(nblocks) * 256;
  uint64_t items = scan_scratch_items(ncounts);
  DFL_TRY(ensure_tmp(h, (2 * ncounts + 1 + items) * sizeof(uint32_t)));
  uint32_t* counts = static_cast<uint32_t*>(h->tmp);
  uint32_t* offs = counts + ncounts;
  uint32_t* sscratch = offs + ncounts + 1;
  unsigned long long *ka = key, *kb = key2;
  uint32_t *va = val, *vb = val2;
  uint32_t passes = (bits + 7) / 8;
  for (uint32_t p = 0; p < passes; ++p) {
    uint32_t shift = p * 8;
    {
      LaunchScope ls(h, DFL_PROF_APPLY);
      k_radix_hist<<<nblocks, kRadixThreads, 0, h->stream>>>(ka, n, shift, counts, nblocks);
      DFL_TRY(check_launch(h, "radix hist"));
    }
    DFL_TRY(scan_impl<uint32_t>(h, counts, offs, ncounts, sscratch, items));
    {
      LaunchScope ls(h, DFL_PROF_APPLY);
      k_radix_scatter<<<nblocks, kRadixThreads, 0, h->stream>>>(ka, va, kb, vb, n, shift, offs,
                                                                 nblocks);
      DFL_TRY(check_launch(h, "radix scatter"));
    }
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (ka != key) {
    DFL_CUDA(h, cudaMemcpyAsync(key, ka, n * sizeof(unsigned long long), cudaMemcpyDeviceToDevice,
                                h->stream));
    DFL_CUDA(h, cudaMemcpyAsync(val, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, h->stream));
  }
  return DFL_OK;
}

int fill_u32(Handle* h, uint32_t* p, uint32_t v, uint64_t n) {
  if (!n) return DFL_OK;
  LaunchScope ls(h, DFL_PROF_OTHER);
  k_fill<uint32_t><<<grid_for(n, 256), 256, 0, h->stream>>>(p, v, n);
  return check_launch(h, "fill");
}

int fill_i32(Handle* h, int* p, int v, uint64_t n) {
  if (!n) return DFL_OK;
  LaunchScope ls(h, DFL_PROF_OTHER);
  k_fill<int><<<grid_for(n, 256), 256, 0, h->stream>>>(p, v, n);
  return check_launch(h, "fill");
}

int iota_u32(Handle* h, uint32_t* p, uint64_t n) {
  if (!n) return DFL_OK;
  LaunchScope ls(h, DFL_PROF_OTHER);
  k_iota<<<grid_for(n, 256), 256, 0, h->stream>>>(p, n);
  return check_launch(h, "iota");
}

int copy_i64(Handle* h, long long* dst, const long long* src, uint64_t n) {
  if (!n) return DFL_OK;
  LaunchScope ls(h, DFL_PROF_OTHER);
  k_copy_i64<<<grid_for(n, 256), 256, 0, h->stream>>>(dst, src, n);
  return check_launch(h, "copy");
}

int lists_all(Handle* h, uint32_t nv, const uint32_t* deg, int buf, uint32_t k) {
  make_segs(h, k);
  const Segs& seg = h->segs;
  LaunchScope ls(h, DFL_PROF_MARK);
  k_lists_all<<<grid_for(nv, 256, 152 * 8), 256, 0, h->stream>>>(nv, deg, h->lists[buf], seg, h->ctrl, buf,
                                                        k);
  return check_launch(h, "lists_all");
}

int lists_from_bits(Handle* h, const uint32_t* bits, uint32_t nv, const uint32_t* deg, int buf,
                    uint32_t k) {
  make_segs(h, k);
  const Segs& seg = h->segs;
  uint32_t words = (nv + 31) / 32;
  LaunchScope ls(h, DFL_PROF_MARK);
  k_lists_bits<<<grid_for(words, 256, 152 * 8), 256, 0, h->stream>>>(bits, words, nv, deg, h->lists[buf],
                                                                     seg, h->ctrl, buf, k, nullptr, 0u);
  return check_launch(h, "lists_from_bits");
}

int bits_to_bytes(Handle* h, const uint32_t* bits, uint8_t* out, uint32_t n) {
  if (!n) return DFL_OK;
  LaunchScope ls(h, DFL_PROF_OTHER);
  k_bits_to_bytes<<<grid_for(n, 256), 256, 0, h->stream>>>(bits, out, n);
  return check_launch(h, "bits_to_bytes");
}

int bytes_to_bits(Handle* h, const uint8_t* in, uint32_t* bits, uint32_t n) {
  uint32_t words = (n + 31) / 32;
  if (!words) return DFL_OK;
  LaunchScope ls(h, DFL_PROF_OTHER);
  k_bytes_to_bits<<<grid_for(words, 256), 256, 0, h->stream>>>(in, bits, n, words);
  return check_launch(h, "bytes_to_bits");
}

uint64_t popcount_bits(Handle* h, const uint32_t* bits, uint32_t words, int* rc) {
  *rc = DFL_OK;
  if (!words) return 0;
  cudaError_t e = cudaMemsetAsync(&h->ctrl->red_a, 0, sizeof(unsigned long long), h->stream);
  if (e != cudaSuccess) {
    *rc = set_error(h, DFL_ERR_CUDA, cudaGetErrorString(e));
    return 0;
  }
  {
    LaunchScope ls(h, DFL_PROF_OTHER);
    k_popcount<<<grid_for(words, 256), 256, 0, h->stream>>>(bits, words, &h->ctrl->red_a);
    *rc = check_launch(h, "popcount");
    if (*rc) return 0;
  }
  unsigned long long v = 0;
  e = cudaMemcpyAsync(&v, &h->ctrl->red_a, sizeof(v), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) *rc = set_error(h, DFL_ERR_CUDA, cudaGetErrorString(e));
  return v;
}

}  // namespace dfl
