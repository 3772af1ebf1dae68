// FP32 evaluation path (FMM_FP32C): expansions and near-field sums in FP32
// on radius-scaled coefficients, FP32 offsets from leaf centres, two-sum
// compensated leaf and local accumulation, FP64 rotation coefficients rounded
// once, FP64 near + far combination.
#include "common.cuh"
namespace fmm {
using real = float;
}
#include "eval_impl.cuh"

namespace fmm {
namespace {
Ptrs ptrs(const fmm_tree* t) {
  return Ptrs{t->pos_local, t->src32, t->inv_rho32, t->geo32, t->m2m32, t->l2d32, t->M32, t->Lam32};
}
}  // namespace
void eval_fp32(const fmm_tree* t, const double* q, double* u, double* field, cudaStream_t st) {
  eval_impl(t, q, u, field, st);
}
void backward_fp32(const fmm_tree* t, const double* q, const double* g, double* ug, double* fq, double* fg,
                   cudaStream_t st) {
  backward_impl(t, q, g, ug, fq, fg, st);
}
void backward_sym_fp32(const fmm_tree* t, const double* q, const double* g, double* grad_q, double* grad_pos,
                       cudaStream_t st) {
  backward_sym_impl(t, q, g, grad_q, grad_pos, st);
}
void init_tables_fp32() { upload_tables(); }
}  // namespace fmm
