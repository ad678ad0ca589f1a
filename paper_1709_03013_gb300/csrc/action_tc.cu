// Tensor-core form of the interval counts (placeholder until the tcgen05 kernel lands).
#include "csg_internal.cuh"

namespace csg {

int action_tc(const SetDesc *, int, cudaStream_t) {
    set_error("tensor-core action is not available in this build");
    return CSG_E_INVAL;
}

}  // namespace csg
