// FP64 evaluation path (FMM_FP64): every stage in FP64.
#include "common.cuh"
namespace fmm {
using real = double;
}
#include "eval_impl.cuh"

namespace fmm {
namespace {
Ptrs ptrs(const fmm_tree* t) {
  return Ptrs{t->pos64, t->src64, t->inv_rho64, t->geo64, t->m2m64, t->l2d64, t->M64, t->Lam64};
}
}  // namespace
void eval_fp64(const fmm_tree* t, const double* q, double* u, double* field, cudaStream_t st) {
  // the FP64 data are made when an FP64 precision is selected (ensure_fp64)
  require(t->geo64 && t->m2m64 && t->l2d64 && t->M64 && t->Lam64 && t->src64 && (!t->sym || t->sym_partial_f64),
          "the tree's FP64 data are missing (select FMM_FP64 or FMM_FP64DF with fmm_tree_set_precision)");
  eval_impl(t, q, u, field, st);
}
void init_tables_fp64() { upload_tables(); }
}  // namespace fmm
