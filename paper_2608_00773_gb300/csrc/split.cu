// Split-precision batch products on tcgen05 tensor cores (in progress).
#include "internal.h"

namespace q4c {

q4c_status integrate_split(const q4c_tables*, const q4c_grid*, const double*, const q4c_matrices*, cudaStream_t) {
  set_error("q4c_integrate: the split-precision path is not built yet");
  return Q4C_EUNSUPPORTED;
}

}  // namespace q4c
