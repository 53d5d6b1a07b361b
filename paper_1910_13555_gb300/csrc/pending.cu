// Entry points whose kernels are added in later files; they report UNSUPPORTED.
#include "bst_internal.h"

namespace bst {
void execute_emu_bf16(bst_plan *, const NumArgs &, cudaStream_t) {
  throw Error{BST_ERR_UNSUPPORTED, "emulated FP64 not built yet"};
}
void execute_tf32x3(bst_plan *, const NumArgs &, cudaStream_t) {
  throw Error{BST_ERR_UNSUPPORTED, "3xTF32 not built yet"};
}
}  // namespace bst

extern "C" {
bst_status bst_plan_adjoint(bst_plan *, const double *, double *, double *, double *, double, double,
                            void *) {
  bst::set_error("adjoint not built yet");
  return BST_ERR_UNSUPPORTED;
}
bst_status bst_tensor_create(bst_ctx *, bst_tensor **, int32_t, const int32_t *, const int32_t *,
                             int64_t, const int32_t *, double *, void *) {
  return BST_ERR_UNSUPPORTED;
}
bst_status bst_tensor_info(const bst_tensor *, int32_t *, int64_t *, int64_t *) { return BST_ERR_UNSUPPORTED; }
bst_status bst_tensor_get_index(const bst_tensor *, int32_t *, int64_t *) { return BST_ERR_UNSUPPORTED; }
bst_status bst_tensor_bind_data(bst_tensor *, double *) { return BST_ERR_UNSUPPORTED; }
bst_status bst_tensor_destroy(bst_tensor *) { return BST_ERR_UNSUPPORTED; }
bst_status bst_contract_plan(bst_ctx *, const bst_tensor *, const bst_tensor *, int32_t, const int32_t *,
                             const int32_t *, int32_t, const int32_t *, int32_t, const int32_t *,
                             const int32_t *, const bst_tensor *, double, void *, bst_plan **) {
  return BST_ERR_UNSUPPORTED;
}
bst_status bst_plan_result_tensor(bst_plan *, bst_tensor **) { return BST_ERR_UNSUPPORTED; }
bst_status bst_batch_create(bst_ctx *, int32_t, bst_plan *const *, bst_batch **) { return BST_ERR_UNSUPPORTED; }
bst_status bst_batch_execute(bst_batch *, const double *, const double *, int32_t, void *) {
  return BST_ERR_UNSUPPORTED;
}
bst_status bst_batch_destroy(bst_batch *) { return BST_ERR_UNSUPPORTED; }
}
