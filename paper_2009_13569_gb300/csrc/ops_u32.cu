// ops_u32.cu -- kernel instantiations for the u32 element type.
#include "ops_impl.cuh"

namespace ipsgpu {
const TypeOps ops_u32 = OpsImpl<TU32>::make();
}  // namespace ipsgpu
