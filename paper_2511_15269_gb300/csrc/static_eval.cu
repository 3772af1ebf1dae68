// fmm_eval_potential_static: the potential evaluation of fmm_eval_potential
// with its per-call scratch (tree-ordered point records, near-field sums,
// multipole and local expansions, work counters) in one file-scope device
// array instead of the tree's own workspace.  It exists for callers that must
// not allocate device memory at evaluation time: code running while another
// allocator owns the device memory budget (a framework's caching pool), code
// on latency-critical paths where cudaMalloc's implicit synchronisation is not
// acceptable, and plug-ins that are only allowed to allocate at start-up.
//
// The evaluation itself runs the same kernels on a shallow copy of the tree
// whose workspace pointers point into the array; the tree's hierarchy,
// geometry and rotation coefficients are read as usual.
#include <mutex>

#include "common.cuh"

namespace fmm {
namespace {

constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
constexpr int64_t kMaxPts = FMM_STATIC_MAX_POINTS;
constexpr int64_t kMaxBoxes = FMM_STATIC_MAX_BOXES;
constexpr size_t kExpBytes = align256((size_t)kMaxBoxes * ncoef_pad(kMaxP) * sizeof(double));
constexpr size_t kOffSrc32 = 0;
constexpr size_t kOffDup = kOffSrc32 + align256(kMaxPts * sizeof(float4));
constexpr size_t kOffSrc64 = kOffDup + align256(kMaxPts * sizeof(DupRec));
constexpr size_t kOffNear = kOffSrc64 + align256(kMaxPts * sizeof(dvec4));
constexpr size_t kOffM = kOffNear + align256(kMaxPts * sizeof(double));
constexpr size_t kOffLam = kOffM + kExpBytes;
constexpr size_t kOffCtr = kOffLam + kExpBytes;
constexpr size_t kBytes = kOffCtr + 256;
static_assert(kBytes == FMM_STATIC_SCRATCH_BYTES, "FMM_STATIC_SCRATCH_BYTES must match the layout");

// Shared by every call on a device; holds the last call's contents.
static __device__ __align__(256) unsigned char g_scratch[kBytes];

std::mutex g_mu;
unsigned char* g_scratch_dev[64] = {};

// Device address of g_scratch on the current device (first call per device
// looks it up with that device current).
unsigned char* scratch_address() {
  int dev = 0;
  FMM_CUDA_TRY(cudaGetDevice(&dev));
  require(dev >= 0 && dev < 64, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    FMM_CUDA_TRY(cudaGetSymbolAddress(&p, g_scratch));
    g_scratch_dev[dev] = static_cast<unsigned char*>(p);
  }
  return g_scratch_dev[dev];
}

}  // namespace
}  // namespace fmm

extern "C" int fmm_eval_potential_static(const fmm_tree* tree, const double* q, double* u, void* stream) {
  using namespace fmm;
  try {
    require(tree != nullptr && q != nullptr && u != nullptr, "NULL argument");
    require(!tree->two_trees, "fmm_eval_potential_static takes trees of one point set");
    if (tree->n > kMaxPts || tree->n_boxes > kMaxBoxes) {
      set_error("fmm_eval_potential_static: tree with %lld points and %lld boxes exceeds the static scratch "
                "capacity of %lld points and %lld boxes",
                (long long)tree->n, (long long)tree->n_boxes, (long long)kMaxPts, (long long)kMaxBoxes);
      return FMM_ERR_CAPACITY;
    }
    unsigned char* base = scratch_address();
    fmm_tree view = *tree;  // shallow copy: same hierarchy, redirected workspace
    view.src32 = reinterpret_cast<float4*>(base + kOffSrc32);
    view.src_dup = reinterpret_cast<DupRec*>(base + kOffDup);
    view.src64 = reinterpret_cast<dvec4*>(base + kOffSrc64);
    view.near_u = base + kOffNear;
    view.near_f = nullptr;  // potential only
    view.M32 = reinterpret_cast<float*>(base + kOffM);
    view.M64 = reinterpret_cast<double*>(base + kOffM);
    view.Lam32 = reinterpret_cast<float*>(base + kOffLam);
    view.Lam64 = reinterpret_cast<double*>(base + kOffLam);
    view.counters = reinterpret_cast<int*>(base + kOffCtr);  // zeroed before every use
    view.m2m_ready = nullptr;  // M2M one launch per round (no readiness flags in the array)
    view.sym = 0;  // the symmetric near field's slots are tree workspace; the one-sided kernel needs none
    view.prof_on = 0;
    view.prof_ev = nullptr;
    view.level_avg_host = nullptr;
    const int64_t before = view.launches;
    cudaStream_t st = (cudaStream_t)stream;
    if (view.prm.precision == FMM_FP32C) eval_fp32(&view, q, u, nullptr, st);
    else eval_fp64(&view, q, u, nullptr, st);
    tree->launches += view.launches - before;
    return FMM_OK;
  } catch (const Fail& e) {
    return e.code;
  } catch (...) {
    set_error("unexpected C++ exception");
    return FMM_ERR_CUDA;
  }
}
