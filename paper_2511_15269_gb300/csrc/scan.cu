// Exclusive prefix sums of int64 arrays on the device (reduce-then-scan:
// per-block scans, a recursive scan of the block totals, then a fix-up).
#include "common.cuh"

namespace fmm {
namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ int64_t block_exclusive(int64_t v, int64_t* total) {
  __shared__ int64_t warp_sums[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t w = (lane < kScanThreads / 32) ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kScanThreads / 32) warp_sums[lane] = w;
  }
  __syncthreads();
  int64_t before = (warp > 0) ? warp_sums[warp - 1] : 0;
  *total = warp_sums[kScanThreads / 32 - 1];
  __syncthreads();
  return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads) scan_tiles(const int64_t* in, int64_t* out, int64_t n,
                                                           int64_t* tile_sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    v[k] = (base + k < n) ? in[base + k] : 0;
    s += v[k];
  }
  int64_t total;
  int64_t run = block_exclusive(s, &total);
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void add_tile_offsets(int64_t* out, int64_t n, const int64_t* tile_off) {
  const int64_t i = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
  const int64_t add = tile_off[blockIdx.x];
  for (int k = 0; k < kScanItems; k++) {
    int64_t j = i + (int64_t)k * kScanThreads;
    if (j < n) out[j] += add;
  }
}

__global__ void write_total(const int64_t* in_last, const int64_t* out_last, int64_t* total) {
  *total = *in_last + *out_last;
}

void scan_rec(const int64_t* in, int64_t* out, int64_t n, cudaStream_t st, int64_t* total_dev) {
  if (n <= 0) {
    FMM_CUDA_TRY(cudaMemsetAsync(total_dev, 0, sizeof(int64_t), st));
    return;
  }
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  int64_t* sums = scratch_alloc<int64_t>((size_t)tiles + 1);
  // keep the last input before an in-place scan overwrites it
  int64_t* last_in = scratch_alloc<int64_t>(1);
  FMM_CUDA_TRY(cudaMemcpyAsync(last_in, in + n - 1, sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
  scan_tiles<<<(unsigned)tiles, kScanThreads, 0, st>>>(in, out, n, sums);
  FMM_LAUNCH_CHECK();
  if (tiles > 1) {
    int64_t* dummy = scratch_alloc<int64_t>(1);
    scan_rec(sums, sums, tiles, st, dummy);
    add_tile_offsets<<<(unsigned)tiles, kScanThreads, 0, st>>>(out, n, sums);
    FMM_LAUNCH_CHECK();
    FMM_CUDA_TRY(cudaStreamSynchronize(st));
    dev_free(dummy);
  }
  write_total<<<1, 1, 0, st>>>(last_in, out + n - 1, total_dev);
  FMM_LAUNCH_CHECK();
  FMM_CUDA_TRY(cudaStreamSynchronize(st));
  dev_free(sums);
  dev_free(last_in);
}

}  // namespace

void exclusive_scan_async(const int64_t* in, int64_t* out, int64_t n, int64_t* total_dev,
                          cudaStream_t st) {
  scan_rec(in, out, n, st, total_dev);
}

int64_t exclusive_scan(const int64_t* in, int64_t* out, int64_t n, cudaStream_t st) {
  int64_t* tot = scratch_alloc<int64_t>(1);
  scan_rec(in, out, n, st, tot);
  int64_t h = 0;
  FMM_CUDA_TRY(cudaMemcpyAsync(&h, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  FMM_CUDA_TRY(cudaStreamSynchronize(st));
  dev_free(tot);
  return h;
}

}  // namespace fmm
