// Work orders of the persistent evaluation kernels: a permutation of boxes
// (or leaves) by descending work, ties in ascending index order, built on
// the device by a stable least-significant-digit radix sort (four passes of
// 8-bit digits over 32-bit keys; per pass a tile histogram, a scan of the
// digit-major tile counts and a stable scatter).  The order only balances
// the persistent kernels' load; results never depend on it.
#include <algorithm>

#include "common.cuh"

namespace fmm {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 4;
constexpr int kSortTile = kSortThreads * kSortItems;

// descending key order = ascending order of the complemented, clamped key
__global__ void sort_keys_kernel(const int64_t* __restrict__ key, int64_t n, uint32_t* __restrict__ k32,
                                 int32_t* __restrict__ idx) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = key[i] < 0 ? 0 : (key[i] > 0xffffffffll ? 0xffffffffll : key[i]);
    k32[i] = 0xffffffffu - (uint32_t)k;
    idx[i] = (int32_t)i;
  }
}

__global__ void __launch_bounds__(kSortThreads) sort_hist_kernel(const uint32_t* __restrict__ k, int64_t n, int shift,
                                                                 int64_t nblk, int64_t* __restrict__ hist) {
  __shared__ unsigned cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t t0 = (int64_t)blockIdx.x * kSortTile;
  for (int j = 0; j < kSortItems; j++) {
    const int64_t i = t0 + (int64_t)j * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(k[i] >> shift) & 0xffu], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter of one tile: items are ranked chunk by chunk (256 at a
// time, in index order), inside a chunk by warp and by lane.
__global__ void __launch_bounds__(kSortThreads) sort_scatter_kernel(const uint32_t* __restrict__ k,
                                                                    const int32_t* __restrict__ v, int64_t n,
                                                                    int shift, int64_t nblk,
                                                                    const int64_t* __restrict__ pref,
                                                                    uint32_t* __restrict__ ko,
                                                                    int32_t* __restrict__ vo) {
  constexpr int W = kSortThreads / 32;
  __shared__ unsigned wcnt[W][256];
  __shared__ int64_t base[256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  base[threadIdx.x] = pref[(int64_t)threadIdx.x * nblk + blockIdx.x];
  const int64_t t0 = (int64_t)blockIdx.x * kSortTile;
  for (int j = 0; j < kSortItems; j++) {
    for (int w = 0; w < W; w++) wcnt[w][threadIdx.x] = 0;
    __syncthreads();
    const int64_t i = t0 + (int64_t)j * kSortThreads + threadIdx.x;
    const bool valid = i < n;
    const uint32_t key = valid ? k[i] : 0u;
    const unsigned d = (key >> shift) & 0xffu;
    const unsigned act = __ballot_sync(0xffffffffu, valid);
    const unsigned peers = __match_any_sync(0xffffffffu, valid ? d : 0x100u) & act;
    const unsigned lower = __popc(peers & ((1u << lane) - 1u));
    if (valid && lower == 0) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      int64_t off = base[d] + lower;
      for (int w = 0; w < warp; w++) off += wcnt[w][d];
      ko[off] = key;
      vo[off] = v[i];
    }
    __syncthreads();
    unsigned tot = 0;
    for (int w = 0; w < W; w++) tot += wcnt[w][threadIdx.x];
    base[threadIdx.x] += tot;
    __syncthreads();
  }
}

}  // namespace

void order_desc(const int64_t* key, int64_t n, int32_t* perm, cudaStream_t st) {
  if (n <= 0) return;
  const int64_t nblk = (n + kSortTile - 1) / kSortTile;
  uint32_t* ka = scratch_alloc<uint32_t>(n);
  uint32_t* kb = scratch_alloc<uint32_t>(n);
  int32_t* va = scratch_alloc<int32_t>(n);
  int32_t* vb = scratch_alloc<int32_t>(n);
  int64_t* hist = scratch_alloc<int64_t>(256 * nblk);
  int64_t* pref = scratch_alloc<int64_t>(256 * nblk);
  int64_t* total = scratch_alloc<int64_t>(2);  // total, error word of the scans
  FMM_CUDA_TRY(cudaMemsetAsync(total + 1, 0, sizeof(int64_t), st));
  sort_keys_kernel<<<grid_for(n, 256), 256, 0, st>>>(key, n, ka, va);
  FMM_LAUNCH_CHECK();
  for (int pass = 0; pass < 4; pass++) {
    const int shift = 8 * pass;
    sort_hist_kernel<<<(unsigned)nblk, kSortThreads, 0, st>>>(ka, n, shift, nblk, hist);
    FMM_LAUNCH_CHECK();
    exclusive_scan_async(hist, pref, 256 * nblk, total, reinterpret_cast<int*>(total + 1), st);
    const bool last = pass == 3;
    sort_scatter_kernel<<<(unsigned)nblk, kSortThreads, 0, st>>>(ka, va, n, shift, nblk, pref, kb,
                                                                 last ? perm : vb);
    FMM_LAUNCH_CHECK();
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  int64_t err = 0;
  FMM_CUDA_TRY(cudaMemcpyAsync(&err, total + 1, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  FMM_CUDA_TRY(cudaStreamSynchronize(st));
  dev_free(ka), dev_free(kb), dev_free(va), dev_free(vb), dev_free(hist), dev_free(pref), dev_free(total);
  if (err) {
    set_error("a bounded device-side wait gave up (prefix sum look-back)");
    throw Fail{FMM_ERR_TIMEOUT};
  }
}

}  // namespace fmm
