// dense.cu — dense tensor-core path (filled in below).
#include "internal.h"

namespace isg {
cudaError_t launch_dense(ising_handle *, const ising_search_params *, int32_t, cudaStream_t) {
  return cudaErrorNotSupported;
}
bool dense_supported(const ising_handle *, int32_t) { return false; }
void dense_free(ising_handle *) {}
}  // namespace isg
