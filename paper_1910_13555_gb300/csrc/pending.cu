// Entry points whose kernels are added in later files; they report UNSUPPORTED.
#include "bst_internal.h"



extern "C" {
bst_status bst_batch_create(bst_ctx *, int32_t, bst_plan *const *, bst_batch **) { return BST_ERR_UNSUPPORTED; }
bst_status bst_batch_execute(bst_batch *, const double *, const double *, int32_t, void *) {
  return BST_ERR_UNSUPPORTED;
}
bst_status bst_batch_destroy(bst_batch *) { return BST_ERR_UNSUPPORTED; }
}
