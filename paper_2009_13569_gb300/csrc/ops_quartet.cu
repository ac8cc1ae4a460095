// ops_quartet.cu -- kernel instantiations for the quartet element type.
#include "ops_impl.cuh"

namespace ipsgpu {
const TypeOps ops_quartet = OpsImpl<TQuartet>::make();
}  // namespace ipsgpu
