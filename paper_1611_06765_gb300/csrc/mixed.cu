// mixed.cu -- mixed-precision iteration body (filled in with the tcgen05 pp ladder).
#include "pnm_context.cuh"

void pnm_prepare_mixed(pnm_ctx*) {
  throw PnmError{PNM_EINVAL, "mixed precision is not available in this build"};
}

void pnm_enqueue_body_mixed(pnm_ctx*, int, cudaGraphConditionalHandle) {
  throw PnmError{PNM_EINVAL, "mixed precision is not available in this build"};
}

void pnm_free_mixed(pnm_ctx*) {}
