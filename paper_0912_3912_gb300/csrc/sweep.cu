// sweep.cu — large-instance sweeps (filled in below).
#include "internal.h"

namespace isg {
cudaError_t launch_sweep(ising_handle *, const ising_search_params *, int32_t, cudaStream_t) {
  return cudaErrorNotSupported;
}
void sweep_free(ising_handle *) {}
}  // namespace isg
