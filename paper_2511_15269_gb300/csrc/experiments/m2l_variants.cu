// M2L kernel variants timed on a synthetic interaction list shaped like the
// 2^20-point uniform cube at p = 8 (21,845 boxes, about 4.0 M interactions,
// 120-250 interactions per target, random sources; multipoles and rotation
// records random but well formed).  A measurement program, not part of the
// library: it includes the library's expansion algebra and compares
//   base     the library's M2L kernel itself (a lane per interaction, the
//            7-field rotation record, angle multiples in the kernel,
//            shared-memory accumulation rows, 3 blocks per SM by registers)
//   occ4     the same code capped at 128 registers (4 blocks per SM; spills)
//   pf_rec   the next work item's rotation records prefetched into shared
//            memory by cp.async while the current one is computed
//   pf_all   the records and the source multipoles prefetched (2 blocks per
//            SM: the shared memory of the prefetch buffers)
//   tc_path  the data path a tensor-core form of the quarter-turn products
//            (Y(+-pi/2) with the turns, Sec. II.D / App. B.2) needs in place
//            of those products: each degree's coefficients split into tf32
//            hi + lo, both stored to a shared operand tile and the result read
//            back, with no product formed (a lower bound on the time of any
//            such restructuring, whatever the speed of the products)
// Build and run (one GPU):
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 --expt-relaxed-constexpr \
//        -I include -o m2l_variants paper_2511_15269_gb300/csrc/experiments/m2l_variants.cu
//   ./m2l_variants
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "../common.cuh"
namespace fmm {
using real = float;
}
#include "../eval_impl.cuh"

namespace fmm {
namespace {
Ptrs ptrs(const fmm_tree*) { return Ptrs{}; }  // the library's host pipeline is not used here
}  // namespace
void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vfprintf(stderr, fmt, ap);
  va_end(ap);
}
const char* last_error() { return ""; }
}  // namespace fmm
using namespace fmm;

#define CK(x)                                                                                       \
  do {                                                                                              \
    cudaError_t e_ = (x);                                                                           \
    if (e_ != cudaSuccess) {                                                                        \
      fprintf(stderr, "CUDA error %s at line %d: %s\n", #x, __LINE__, cudaGetErrorString(e_));      \
      exit(1);                                                                                      \
    }                                                                                               \
  } while (0)

namespace m2lx {
constexpr int kP = 8;
constexpr int kNF = 7;  // rotation record: 1/r, rho_S/r, rho_T/r, cos phi, sin phi, cos theta, sin theta

template <int P>
constexpr int chunks() {
  return ((ncoef(P) + 3) / 4) | 1;
}

__device__ __forceinline__ void two_sum(float& s, float& e, float b) {
  const float a = s, t = a + b, bb = t - a;
  e += (a - (t - bb)) + (b - bb);
  s = t;
}

template <int P>
__device__ __forceinline__ void acc_add(float* row, const float (&v)[ncoef(P)]) {
  constexpr int NC = ncoef(P);
  sfor<0, chunks<P>()>([&](auto kk) {
    constexpr int k = decltype(kk)::value;
    constexpr int i = 4 * k;
    if constexpr (i < NC) {
      float4* p4 = reinterpret_cast<float4*>(row) + k;
      float4 a = *p4;
      a.x += v[i];
      if constexpr (i + 1 < NC) a.y += v[i + 1];
      if constexpr (i + 2 < NC) a.z += v[i + 2];
      if constexpr (i + 3 < NC) a.w += v[i + 3];
      *p4 = a;
    }
  });
}

// the warp's 32 rows summed per coefficient in lane order (whole warp)
template <int P>
__device__ __forceinline__ void reduce_rows(const float* rows, float* out, int lane) {
  constexpr int NC = ncoef(P), NCP = ncoef_pad(P), ROW = chunks<P>() * 4;
  for (int c = lane; c < NCP; c += 32) {
    float s = 0.f, err = 0.f;
    if (c < NC)
      for (int j = 0; j < 32; j++) two_sum(s, err, rows[j * ROW + c]);
    out[c] = s + err;
  }
}

template <int P>
__device__ __forceinline__ void load_row(const float* src, float (&v)[ncoef(P)]) {
  constexpr int NC = ncoef(P);
#pragma unroll
  for (int c = 0; c < (NC + 3) / 4; c++) {
    const float4 x = reinterpret_cast<const float4*>(src)[c];
    v[4 * c] = x.x;
    if (4 * c + 1 < NC) v[4 * c + 1] = x.y;
    if (4 * c + 2 < NC) v[4 * c + 2] = x.z;
    if (4 * c + 3 < NC) v[4 * c + 3] = x.w;
  }
}

// ---- occ4: the library kernel's code with a register cap ---------------------------
template <int P, int MINB>
__global__ void __launch_bounds__(128, MINB) m2l_capped(int64_t n_items, const M2LItem* __restrict__ items,
                                                        const int32_t* __restrict__ src, const float* __restrict__ geo,
                                                        int64_t nm, const float* __restrict__ M,
                                                        float* __restrict__ Lam, float* __restrict__ /*partial*/,
                                                        int* __restrict__ counter) {
  constexpr int NC = ncoef(P), NCP = ncoef_pad(P), ROW = m2l_chunks<P>() * 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = lane_id(), warp = threadIdx.x >> 5;
  float* rows = reinterpret_cast<float*>(smem_raw) + (size_t)warp * 32 * ROW;
  float* mine = rows + lane * ROW;
  for (;;) {
    int t = 0;
    if (lane == 0) t = atomicAdd(counter, 1);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= n_items) break;
    const M2LItem it = items[t];
#pragma unroll
    for (int c = 0; c < ROW; c++) mine[c] = 0.f;
    for (int64_t i = it.b + lane; i < it.e; i += 32) {
      float v[NC];
      load_coef<P>(M + (int64_t)src[i] * NCP, v);
      const float rinv = geo[i], uS = geo[nm + i], uT = geo[2 * nm + i];
      float cp[P], sp[P], ct[P], st[P];
      trig_multiples<P>(geo[3 * nm + i], geo[4 * nm + i], cp, sp);
      trig_multiples<P>(geo[5 * nm + i], geo[6 * nm + i], ct, st);
      translate_rotated<P>(v, cp, sp, ct, st, [&](float (&w)[ncoef(P)]) { axial_m2l<P>(w, uS, uT, rinv); });
      m2l_acc_add<P>(mine, v);
    }
    __syncwarp();
    reduce_rows<P>(rows, Lam + (int64_t)it.g * NCP, lane);
    __syncwarp();
  }
}

// ---- pf_rec / pf_all: the next work item's data by cp.async ------------------------
__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp4(void* dst, const void* s) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(saddr(dst)), "l"(s) : "memory");
}
__device__ __forceinline__ void cp16(void* dst, const void* s) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr(dst)), "l"(s) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Warps walk a stream of items (target, first interaction of a chunk of 32);
// while one item is computed the next one's records (and, PFM, source rows)
// land in this lane's shared-memory slots.  Each lane reads only its own
// slots; every warp-wide step is reached by the whole warp.
template <int P, int MINB, bool PFM>
__global__ void __launch_bounds__(128, MINB) m2l_pf(int64_t n_targets, const int32_t* __restrict__ order,
                                                    const int64_t* __restrict__ off, const int32_t* __restrict__ src,
                                                    const float* __restrict__ geo, int64_t nm,
                                                    const float* __restrict__ M, float* __restrict__ Lam,
                                                    int* __restrict__ counter) {
  constexpr int NC = ncoef(P), NCP = ncoef_pad(P), ROW = chunks<P>() * 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* base = reinterpret_cast<float*>(smem_raw);
  float* rows = base + (size_t)warp * 32 * ROW;
  float* mine = rows + lane * ROW;
  float* gb = base + 4 * 32 * ROW + (size_t)warp * kNF * 32;
  float* mb = base + 4 * 32 * ROW + 4 * kNF * 32 + ((size_t)warp * 32 + lane) * NCP;
  auto grab = [&](int64_t& g, int64_t& b, int64_t& e) -> bool {
    for (;;) {
      int t = 0;
      if (lane == 0) t = atomicAdd(counter, 1);
      t = __shfl_sync(0xffffffffu, t, 0);
      if (t >= n_targets) return false;
      g = order[t];
      b = off[g];
      e = off[g + 1];
      if (e > b) return true;
      for (int c = lane; c < NCP; c += 32) Lam[g * NCP + c] = 0.f;
    }
  };
  auto issue_rec = [&](int64_t j) {
    if (j >= 0)
      for (int f = 0; f < kNF; f++) cp4(gb + f * 32 + lane, geo + (int64_t)f * nm + j);
  };
  auto issue_row = [&](int64_t s) {
    if (s >= 0)
      for (int c = 0; c < NCP / 4; c++) cp16(mb + 4 * c, M + s * NCP + 4 * c);
  };
  int64_t g = 0, b = 0, e = 0;
  bool have = grab(g, b, e);
  int64_t i = b;
  if (have) {
    const int64_t j = i + lane < e ? i + lane : -1;
    issue_rec(j);
    if (PFM) issue_row(j >= 0 ? (int64_t)src[j] : -1);
    cp_commit();
  }
  for (int c = 0; c < ROW; c++) mine[c] = 0.f;
  while (have) {
    const int64_t j = i + lane;
    const bool act = j < e;
    cp_wait_all();
    float v[NC];
    float c1p = 1.f, s1p = 0.f, c1t = 1.f, s1t = 0.f, rinv = 0.f, uS = 0.f, uT = 0.f;
    if (act) {
      if (PFM) load_row<P>(mb, v);
      else load_row<P>(M + (int64_t)src[j] * NCP, v);
      rinv = gb[lane];
      uS = gb[32 + lane];
      uT = gb[64 + lane];
      c1p = gb[96 + lane];
      s1p = gb[128 + lane];
      c1t = gb[160 + lane];
      s1t = gb[192 + lane];
    }
    __syncwarp();
    int64_t g2 = g, b2 = b, e2 = e, i2 = i + 32;
    const bool last = i2 >= e;
    bool have2 = true;
    if (last) {
      have2 = grab(g2, b2, e2);
      i2 = b2;
    }
    const int64_t jn = (have2 && i2 + lane < e2) ? i2 + lane : -1;
    int64_t sn = -1;
    if (have2) {
      issue_rec(jn);
      if (PFM && jn >= 0) sn = src[jn];
      if (!PFM) cp_commit();
    }
    if (act) {
      float cp[P], sp[P], ct[P], st[P];
      trig_multiples<P>(c1p, s1p, cp, sp);
      trig_multiples<P>(c1t, s1t, ct, st);
      translate_rotated<P>(v, cp, sp, ct, st, [&](float (&w)[ncoef(P)]) {
        if (PFM && have2) {
          issue_row(sn);
          cp_commit();
        }
        axial_m2l<P>(w, uS, uT, rinv);
      });
      acc_add<P>(mine, v);
    } else if (PFM && have2) {
      issue_row(sn);
      cp_commit();
    }
    if (last) {
      __syncwarp();
      reduce_rows<P>(rows, Lam + g * NCP, lane);
      __syncwarp();
      for (int c = 0; c < ROW; c++) mine[c] = 0.f;
    }
    g = g2;
    b = b2;
    e = e2;
    i = i2;
    have = have2;
  }
  cp_wait_all();
}

// ---- tc_path ------------------------------------------------------------------------
__device__ __forceinline__ float tf32_rna(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
// per degree: the 2n + 1 coefficients split into tf32 hi + lo and stored to
// this lane's operand slots, then 2n + 1 results read back (the lane's own
// slots only: lanes leave the interaction loop at different times)
template <int P>
__device__ __forceinline__ void tc_datapath(float (&v)[ncoef(P)], float* tile) {
  sfor<1, P + 1>([&](auto nn) {
    constexpr int n = decltype(nn)::value;
    constexpr int w = 2 * n + 1;
#pragma unroll
    for (int i = 0; i < w; i++) {
      const float x = v[n * n + i];
      const float h = tf32_rna(x);
      tile[i] = h;
      tile[17 + i] = x - h;
    }
#pragma unroll
    for (int i = 0; i < w; i++) v[n * n + i] += tile[34 + i];
  });
}
template <int P>
__global__ void __launch_bounds__(128) m2l_tcpath(int64_t n_items, const M2LItem* __restrict__ items,
                                                  const int32_t* __restrict__ src, const float* __restrict__ geo,
                                                  int64_t nm, const float* __restrict__ M, float* __restrict__ Lam,
                                                  float* __restrict__ /*partial*/, int* __restrict__ counter) {
  constexpr int NC = ncoef(P), NCP = ncoef_pad(P), ROW = m2l_chunks<P>() * 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = lane_id(), warp = threadIdx.x >> 5;
  float* rows = reinterpret_cast<float*>(smem_raw) + (size_t)warp * 32 * ROW;
  float* mine = rows + lane * ROW;
  float* tile = reinterpret_cast<float*>(smem_raw) + 4 * 32 * ROW + ((size_t)warp * 32 + lane) * 53;
  for (;;) {
    int t = 0;
    if (lane == 0) t = atomicAdd(counter, 1);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= n_items) break;
    const M2LItem it = items[t];
#pragma unroll
    for (int c = 0; c < ROW; c++) mine[c] = 0.f;
    for (int64_t i = it.b + lane; i < it.e; i += 32) {
      float v[NC];
      load_coef<P>(M + (int64_t)src[i] * NCP, v);
      const float rinv = geo[i], uS = geo[nm + i], uT = geo[2 * nm + i];
      float cp[P], sp[P], ct[P], st[P], s2[P];
      trig_multiples<P>(geo[3 * nm + i], geo[4 * nm + i], cp, sp);
      trig_multiples<P>(geo[5 * nm + i], geo[6 * nm + i], ct, st);
#pragma unroll
      for (int m = 0; m < P; m++) s2[m] = st[m];
      rot_z<P, false>(v, cp, sp);
#pragma unroll 1
      for (int pass = 0; pass < 2; pass++) {
        if (pass == 1) axial_m2l<P>(v, uS, uT, rinv);
        tc_datapath<P>(v, tile);
        rot_z<P, false>(v, ct, s2);
        tc_datapath<P>(v, tile);
#pragma unroll
        for (int m = 0; m < P; m++) s2[m] = -s2[m];
      }
      rot_z<P, true>(v, cp, sp);
      m2l_acc_add<P>(mine, v);
    }
    __syncwarp();
    reduce_rows<P>(rows, Lam + (int64_t)it.g * NCP, lane);
    __syncwarp();
  }
}

// item-based kernels (the library's m2l_kernel and the variants above)
template <class K>
float timed_items(const char* name, K kern, size_t smem, int nsm, int64_t ni, const M2LItem* items,
                  const int32_t* src, const float* geo, int64_t nm, const float* M, float* Lam, float* part,
                  int* ctr) {
  CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 128, smem));
  const int blocks = nsm * std::max(occ, 1);
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  float best = 1e30f;
  for (int r = 0; r < 6; r++) {
    CK(cudaMemset(ctr, 0, sizeof(int)));
    CK(cudaEventRecord(a));
    kern<<<blocks, 128, smem>>>(ni, items, src, geo, nm, M, Lam, part, ctr);
    CK(cudaEventRecord(b));
    CK(cudaEventSynchronize(b));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, a, b));
    if (r > 0) best = std::min(best, ms);
  }
  CK(cudaGetLastError());
  printf("%-8s %3d blocks/SM  %6zu B shared  %8.1f us  %6.2f TFLOP/s (3510 flops per interaction)\n", name, occ, smem,
         best * 1e3, 2.0 * 1755.0 * nm / (best * 1e-3) / 1e12);
  return best;
}

template <class K>
float timed(const char* name, K kern, size_t smem, int nsm, int64_t nb, const int32_t* order, const int64_t* off,
            const int32_t* src, const float* geo, int64_t nm, const float* M, float* Lam, int* ctr) {
  CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 128, smem));
  const int blocks = nsm * std::max(occ, 1);
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  float best = 1e30f;
  for (int r = 0; r < 6; r++) {
    CK(cudaMemset(ctr, 0, sizeof(int)));
    CK(cudaEventRecord(a));
    kern<<<blocks, 128, smem>>>(nb, order, off, src, geo, nm, M, Lam, ctr);
    CK(cudaEventRecord(b));
    CK(cudaEventSynchronize(b));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, a, b));
    if (r > 0) best = std::min(best, ms);
  }
  CK(cudaGetLastError());
  printf("%-8s %3d blocks/SM  %6zu B shared  %8.1f us  %6.2f TFLOP/s (3510 flops per interaction)\n", name, occ, smem,
         best * 1e3, 2.0 * 1755.0 * nm / (best * 1e-3) / 1e12);
  return best;
}
}  // namespace m2lx
using namespace m2lx;

int main() {
  constexpr int P = kP;
  const int64_t nb = 21845;
  const int NCP = ncoef_pad(P);
  std::mt19937_64 rng(1);
  std::uniform_real_distribution<double> U(0.0, 1.0);
  std::vector<int64_t> off(nb + 1, 0);
  std::vector<int32_t> srcv;
  for (int64_t g = 0; g < nb; g++) {
    const int len = g < 5 ? 0 : 120 + (int)(rng() % 131);
    for (int k = 0; k < len; k++) srcv.push_back((int32_t)(rng() % nb));
    off[g + 1] = (int64_t)srcv.size();
  }
  const int64_t nm = (int64_t)srcv.size();
  std::vector<int32_t> order(nb);
  for (int64_t g = 0; g < nb; g++) order[g] = (int32_t)g;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return off[a + 1] - off[a] > off[b + 1] - off[b]; });
  std::vector<float> geo((size_t)kNF * nm), M((size_t)nb * NCP, 0.f);
  for (int64_t i = 0; i < nm; i++) {
    const double ph = 6.283185307179586 * U(rng), th = 3.141592653589793 * U(rng);
    geo[i] = 1.0f;
    geo[nm + i] = (float)(0.2 + 0.2 * U(rng));
    geo[2 * nm + i] = (float)(0.2 + 0.2 * U(rng));
    geo[3 * nm + i] = (float)cos(ph);
    geo[4 * nm + i] = (float)sin(ph);
    geo[5 * nm + i] = (float)cos(th);
    geo[6 * nm + i] = (float)sin(th);
  }
  for (int64_t g = 0; g < nb; g++)
    for (int c = 0; c < ncoef(P); c++) M[g * NCP + c] = (float)(U(rng) - 0.5);
  std::vector<M2LItem> items(nb);
  for (int64_t k = 0; k < nb; k++) {
    const int32_t g = order[k];
    items[k] = M2LItem{off[g], off[g + 1], g, -1};
  }
  M2LItem* d_items = nullptr;
  float* d_part = nullptr;
  CK(cudaMalloc(&d_items, sizeof(M2LItem) * nb));
  CK(cudaMalloc(&d_part, sizeof(float) * NCP));
  CK(cudaMemcpy(d_items, items.data(), sizeof(M2LItem) * nb, cudaMemcpyHostToDevice));
  int32_t *d_order = nullptr, *d_src = nullptr;
  int64_t* d_off = nullptr;
  float *d_geo = nullptr, *d_M = nullptr, *d_L = nullptr;
  int* d_ctr = nullptr;
  CK(cudaMalloc(&d_order, sizeof(int32_t) * nb));
  CK(cudaMalloc(&d_src, sizeof(int32_t) * nm));
  CK(cudaMalloc(&d_off, sizeof(int64_t) * (nb + 1)));
  CK(cudaMalloc(&d_geo, sizeof(float) * geo.size()));
  CK(cudaMalloc(&d_M, sizeof(float) * M.size()));
  CK(cudaMalloc(&d_L, sizeof(float) * M.size()));
  CK(cudaMalloc(&d_ctr, sizeof(int)));
  CK(cudaMemcpy(d_order, order.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d_src, srcv.data(), sizeof(int32_t) * nm, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d_off, off.data(), sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d_geo, geo.data(), sizeof(float) * geo.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d_M, M.data(), sizeof(float) * M.size(), cudaMemcpyHostToDevice));
  int dev = 0, nsm = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  printf("synthetic M2L list: %lld targets, %lld interactions, p = %d\n", (long long)nb, (long long)nm, P);
  const size_t rows = (size_t)4 * 32 * chunks<P>() * 16;
  const size_t pf_rec = rows + (size_t)4 * kNF * 32 * 4;
  const size_t pf_all = pf_rec + (size_t)4 * 32 * NCP * 4;
  const size_t tc = rows + (size_t)4 * 32 * 53 * 4;
  std::vector<float> ref(M.size()), got(M.size());
  auto compare = [&](const char* name) {
    CK(cudaMemcpy(got.data(), d_L, sizeof(float) * M.size(), cudaMemcpyDeviceToHost));
    double md = 0, mx = 0;
    for (size_t k = 0; k < ref.size(); k++) {
      md = std::max(md, (double)std::fabs(got[k] - ref[k]));
      mx = std::max(mx, (double)std::fabs(ref[k]));
    }
    printf("         %s: max |difference| / max |base| = %.2e\n", name, md / mx);
  };
  const float t0 = timed_items("base", m2l_kernel<P>, rows, nsm, nb, d_items, d_src, d_geo, nm, d_M, d_L, d_part,
                               d_ctr);
  CK(cudaMemcpy(ref.data(), d_L, sizeof(float) * M.size(), cudaMemcpyDeviceToHost));
  timed_items("occ4", m2l_capped<P, 4>, rows, nsm, nb, d_items, d_src, d_geo, nm, d_M, d_L, d_part, d_ctr);
  compare("occ4");
  timed("pf_rec", m2l_pf<P, 3, false>, pf_rec, nsm, nb, d_order, d_off, d_src, d_geo, nm, d_M, d_L, d_ctr);
  compare("pf_rec");
  timed("pf_all", m2l_pf<P, 2, true>, pf_all, nsm, nb, d_order, d_off, d_src, d_geo, nm, d_M, d_L, d_ctr);
  compare("pf_all");
  const float t9 =
      timed_items("tc_path", m2l_tcpath<P>, tc, nsm, nb, d_items, d_src, d_geo, nm, d_M, d_L, d_part, d_ctr);
  printf("tc_path / base = %.2f (the tensor-core data path alone, without any product)\n", t9 / t0);
  return 0;
}
