// dfl_modularity_csr_noalloc: modularity of a caller-supplied graph and
// membership that allocates no memory at all.
//
// Some callers cannot allocate device memory while they run this code: a
// service whose device memory is owned by another allocator (a framework's
// caching allocator, or a fixed budget reserved at start-up), or a
// latency-critical path where cudaMalloc/cudaFree would block or synchronize
// the device.  This entry point therefore takes every input and output from
// the caller and keeps its own scratch -- the per-community totals Sigma_c and
// a few reduction words -- in file-scope __device__ arrays of fixed size.
//
// Limits and sharing:
//   - at most kNoAllocMaxVertices vertices (labels < n), i.e. 8 MiB of
//     scratch that every GPU which loads the library holds until the process
//     exits;
//   - all calls share that scratch: every call clears what it uses before it
//     starts, but calls whose GPU work overlaps (two streams, two threads)
//     race on it and must be serialized by the caller;
//   - the first call on a device looks up the scratch's device address
//     (cudaGetSymbolAddress) with that device current, then reuses it for
//     the life of the process (keyed by device ordinal: after a
//     cudaDeviceReset of that device the remembered address is stale, so the
//     entry point must not be used after a reset).  With CUDA's lazy module
//     loading that first call also loads the library's device code, which
//     allocates the fixed array and may synchronize; it belongs outside any
//     stream capture and any latency-critical path (one warm-up call);
//   - offsets must be non-decreasing and offsets[n] is the arc count that
//     indices and weights hold; a row whose offsets decrease is reported as
//     DFL_ERR_INVALID, but offsets past the end of the caller's arrays
//     cannot be detected (the call does not know their length).
#include <mutex>

#include "common.cuh"

namespace dfl {

namespace {

constexpr uint32_t kNoAllocMaxVertices = 1u << 20;
constexpr int kMaxDevices = 64;

// Per-community totals Sigma_c, indexed by label.
static __device__ __align__(256) long long g_na_sigma[kNoAllocMaxVertices];
// [0] sum of arc weights (2m), [1] sum of arcs inside communities (sigma),
// [2] low and [3] high 32-bit parts of sum Sigma_c^2, [4] error flags.
static __device__ __align__(256) unsigned long long g_na_acc[8];

struct DevPtrs {
  long long* sigma = nullptr;
  unsigned long long* acc = nullptr;
  bool ready = false;
};
DevPtrs g_ptrs[kMaxDevices];
std::mutex g_mu;

// Host code sees only stand-ins for the __device__ arrays: their device
// addresses come from the runtime, once per device, with that device current.
int device_scratch(DevPtrs* out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DFL_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  DevPtrs& p = g_ptrs[dev];
  if (!p.ready) {
    void* s = nullptr;
    void* a = nullptr;
    if (cudaGetSymbolAddress(&s, g_na_sigma) != cudaSuccess) return DFL_ERR_CUDA;
    if (cudaGetSymbolAddress(&a, g_na_acc) != cudaSuccess) return DFL_ERR_CUDA;
    p.sigma = static_cast<long long*>(s);
    p.acc = static_cast<unsigned long long*>(a);
    p.ready = true;
  }
  *out = p;
  return DFL_OK;
}

__global__ void k_na_clear(uint32_t n, long long* __restrict__ sigma, unsigned long long* __restrict__ acc) {
  for (uint64_t c = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; c < n;
       c += uint64_t(gridDim.x) * blockDim.x)
    sigma[c] = 0;
  if (blockIdx.x == 0 && threadIdx.x < 8) acc[threadIdx.x] = 0;
}

// Warp per row: K_i, Sigma_{C_i} += K_i, arcs inside the community, 2m.
__global__ void k_na_rows(uint32_t n, const unsigned long long* __restrict__ off,
                          const uint32_t* __restrict__ idx, const uint32_t* __restrict__ w,
                          const uint32_t* __restrict__ C, long long* __restrict__ sigma,
                          unsigned long long* __restrict__ acc) {
  const uint32_t lane = threadIdx.x & 31u;
  uint64_t warp = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) >> 5;
  uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  unsigned long long tot = 0, inside = 0;
  bool bad = false;
  for (uint64_t i = warp; i < n; i += nwarps) {
    const uint32_t ci = C[i];
    bad |= ci >= n;
    const unsigned long long o0 = off[i], o1 = off[i + 1];
    bad |= o1 < o0;  // decreasing offsets: the row is skipped and the call fails
    unsigned long long k = 0;
    for (unsigned long long q = o0 + lane; q < o1; q += 32) {
      uint32_t j = idx[q];
      if (j >= n) {
        bad = true;
        continue;
      }
      k += w[q];
      if (C[j] == ci) inside += w[q];
    }
    for (int x = 16; x; x >>= 1) k += __shfl_xor_sync(0xFFFFFFFFu, k, x);
    if (lane == 0 && ci < n && k) atomicAdd((unsigned long long*)&sigma[ci], k);
    tot += k;
  }
  for (int x = 16; x; x >>= 1) inside += __shfl_xor_sync(0xFFFFFFFFu, inside, x);
  if (lane == 0) {
    if (tot) atomicAdd(&acc[0], tot);
    if (inside) atomicAdd(&acc[1], inside);
  }
  if (bad) atomicOr(&acc[4], 1ull);
}

__global__ void k_na_squares(uint32_t n, const long long* __restrict__ sigma,
                             unsigned long long* __restrict__ acc) {
  unsigned long long lo = 0, hi = 0;
  for (uint64_t c = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; c < n;
       c += uint64_t(gridDim.x) * blockDim.x) {
    unsigned long long s = (unsigned long long)sigma[c];
    u128 sq = (u128)s * s;
    lo += (unsigned long long)(sq & 0xFFFFFFFFull);
    hi += (unsigned long long)(sq >> 32);
  }
  for (int x = 16; x; x >>= 1) {
    lo += __shfl_xor_sync(0xFFFFFFFFu, lo, x);
    hi += __shfl_xor_sync(0xFFFFFFFFu, hi, x);
  }
  if ((threadIdx.x & 31u) == 0) {
    if (lo) atomicAdd(&acc[2], lo);
    if (hi) atomicAdd(&acc[3], hi);
  }
}

}  // namespace

}  // namespace dfl

extern "C" int dfl_modularity_csr_noalloc(uint32_t n, const uint64_t* offsets, const uint32_t* indices,
                                          const uint32_t* weights, const uint32_t* membership,
                                          double* q, int64_t* parts, void* cuda_stream) {
  using namespace dfl;
  if (n > kNoAllocMaxVertices) return DFL_ERR_INVALID;  // beyond the fixed scratch
  if (!offsets || !membership || !q || (n && (!indices || !weights))) return DFL_ERR_INVALID;
  DevPtrs p;
  int rc = device_scratch(&p);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const auto* off = reinterpret_cast<const unsigned long long*>(offsets);
  k_na_clear<<<grid_for(n ? n : 1, 256, 152 * 8), 256, 0, s>>>(n, p.sigma, p.acc);
  if (n) {
    k_na_rows<<<grid_for(uint64_t(n) * 32, 256), 256, 0, s>>>(n, off, indices, weights, membership,
                                                                p.sigma, p.acc);
    k_na_squares<<<grid_for(n, 256, 152 * 8), 256, 0, s>>>(n, p.sigma, p.acc);
  }
  if (cudaGetLastError() != cudaSuccess) return DFL_ERR_CUDA;
  unsigned long long acc[8];
  if (cudaMemcpyAsync(acc, p.acc, sizeof(acc), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return DFL_ERR_CUDA;
  if (acc[4]) return DFL_ERR_INVALID;              // a label or neighbour id >= n, or decreasing offsets
  if (acc[0] >= (1ull << 32)) return DFL_ERR_OVERFLOW;  // 2m must stay below 2^32
  const i128 m2 = (i128)acc[0];
  const i128 num = m2 * (i128)acc[1] - (((i128)acc[3] << 32) + (i128)acc[2]);
  const i128 den = m2 * m2;
  *q = den == 0 ? 0.0 : double(num) / double(den);
  if (parts) {
    parts[0] = int64_t(uint64_t((u128)num >> 64));
    parts[1] = int64_t(uint64_t((u128)num));
    parts[2] = int64_t(uint64_t((u128)den >> 64));
    parts[3] = int64_t(uint64_t((u128)den));
  }
  return DFL_OK;
}
