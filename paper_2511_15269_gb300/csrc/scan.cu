// Exclusive prefix sums of int64 arrays on the device: one launch, single
// pass with decoupled look-back (Merrill & Garland, "Single-pass Parallel
// Prefix Scan with Decoupled Look-back", 2016).  Blocks take tiles in the
// order they start (a ticket counter), so a tile only ever waits for tiles
// whose blocks are already running; every tile publishes its own sum at
// once and its inclusive prefix as soon as it is known, and a tile's look-back
// (one warp, 32 predecessors per step) adds its predecessors' sums until it
// meets a published prefix.  The wait
// for a predecessor is bounded (a clock limit, then an error word), so a
// fault elsewhere cannot leave the scan spinning.
#include "common.cuh"

namespace fmm {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr long long kScanWaitCycles = 2000000000ll;  // about a second at 2 GHz

// Per-tile look-back record: the tile's own sum (flag 1) and its inclusive
// prefix (flag 2), written before the flag that announces them.
struct __align__(16) TileState {
  int64_t agg;
  int64_t incl;
  int flag;
  int pad;
};

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

// ws: tiles TileStates, then the ticket counter (zeroed before the launch).
// total: the sum of all n inputs; err: set when a look-back wait gave up.
__global__ void __launch_bounds__(kScanThreads) scan_kernel(const int64_t* in, int64_t* out, int64_t n,
                                                            TileState* ws, unsigned* ticket, int64_t* total,
                                                            int* err) {
  __shared__ unsigned tile_sh;
  __shared__ int64_t prefix_sh;
  if (threadIdx.x == 0) tile_sh = atomicAdd(ticket, 1u);
  __syncthreads();
  const int64_t tile = tile_sh;
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  const int64_t base = tile * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    v[k] = (base + k < n) ? in[base + k] : 0;
    s += v[k];
  }
  int64_t agg;
  int64_t run = block_exclusive(s, &agg);
  // warp 0 publishes this tile's sum and looks back over windows of 32
  // predecessors at once: each lane waits for its predecessor's record, the
  // nearest one with a published prefix ends the look-back
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    volatile TileState* me = ws + tile;
    if (lane == 0) {
      if (tile == 0) {
        me->incl = agg;
      } else {
        me->agg = agg;
      }
      __threadfence();
      me->flag = tile == 0 ? 2 : 1;
    }
    int64_t excl = 0;
    if (tile > 0) {
      const long long t0 = clock64();
      int64_t j = tile - 1;  // top of the window
      for (;;) {
        const int64_t jj = j - lane;
        int f = 2;
        int64_t val = 0;
        bool late = false;
        if (jj >= 0) {
          volatile TileState* pj = ws + jj;
          f = pj->flag;
          while (f == 0) {
            if (clock64() - t0 > kScanWaitCycles) {
              late = true;
              break;
            }
            f = pj->flag;
          }
          __threadfence();
          if (f == 2) val = pj->incl;
          else if (f == 1) val = pj->agg;
        }
        if (__any_sync(0xffffffffu, late)) {
          if (lane == 0) atomicExch(err, 1);
          break;
        }
        const unsigned done = __ballot_sync(0xffffffffu, f == 2);
        const int k = done ? __ffs(done) - 1 : 32;  // nearest predecessor with a prefix
        int64_t c = lane <= k ? val : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        excl += c;
        if (done) break;
        j -= 32;
      }
      if (lane == 0) {
        me->incl = excl + agg;
        __threadfence();
        me->flag = 2;
      }
    }
    if (lane == 0) {
      prefix_sh = excl;
      if (tile == tiles - 1) *total = excl + agg;
    }
  }
  __syncthreads();
  run += prefix_sh;
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
}

// Launches the scan; total_dev and err_dev receive the sum and the error word.
void scan_launch(const int64_t* in, int64_t* out, int64_t n, int64_t* total_dev, int* err_dev, cudaStream_t st) {
  if (n <= 0) {
    FMM_CUDA_TRY(cudaMemsetAsync(total_dev, 0, sizeof(int64_t), st));
    return;
  }
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  require(tiles < ((int64_t)1 << 31), "scan too long");
  const size_t ws_bytes = sizeof(TileState) * (size_t)tiles + 16;
  unsigned char* ws = scratch_alloc<unsigned char>(ws_bytes);
  FMM_CUDA_TRY(cudaMemsetAsync(ws, 0, ws_bytes, st));
  scan_kernel<<<(unsigned)tiles, kScanThreads, 0, st>>>(in, out, n, reinterpret_cast<TileState*>(ws),
                                                        reinterpret_cast<unsigned*>(ws + sizeof(TileState) * tiles),
                                                        total_dev, err_dev);
  FMM_LAUNCH_CHECK();
  dev_free(ws);  // stream-ordered: reused only after the scan has run
}

}  // namespace

void exclusive_scan_async(const int64_t* in, int64_t* out, int64_t n, int64_t* total_dev, int* err_dev,
                          cudaStream_t st) {
  scan_launch(in, out, n, total_dev, err_dev, st);
}

int64_t exclusive_scan(const int64_t* in, int64_t* out, int64_t n, cudaStream_t st) {
  int64_t* res = scratch_alloc<int64_t>(2);  // total, error word
  FMM_CUDA_TRY(cudaMemsetAsync(res, 0, 2 * sizeof(int64_t), st));
  scan_launch(in, out, n, res, reinterpret_cast<int*>(res + 1), st);
  int64_t h[2] = {0, 0};
  FMM_CUDA_TRY(cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, st));
  FMM_CUDA_TRY(cudaStreamSynchronize(st));
  dev_free(res);
  if (h[1]) {
    set_error("a bounded device-side wait gave up (prefix sum look-back)");
    throw Fail{FMM_ERR_TIMEOUT};
  }
  return h[0];
}

}  // namespace fmm
