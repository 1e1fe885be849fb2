#include "fe_tc.cuh"
namespace rchfsi {
void fe_tc_product(cudaStream_t, FeOp&, int, const float*, float*, int, float, int) {
  throw Error(RCHFSI_ERR_UNSUPPORTED, "tensor-core FE product not built");
}
}  // namespace rchfsi
