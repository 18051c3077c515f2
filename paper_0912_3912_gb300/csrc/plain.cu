// plain.cu — plain comparator kernel family (filled in below).
#include "internal.h"

namespace isg {
cudaError_t launch_plain(ising_handle *, const ising_search_params *, int32_t, cudaStream_t) {
  return cudaErrorNotSupported;
}
void plain_free(ising_handle *) {}
}  // namespace isg
