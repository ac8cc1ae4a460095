// ops_u64.cu -- kernel instantiations for the u64 element type.
#include "ops_impl.cuh"

namespace ipsgpu {
const TypeOps ops_u64 = OpsImpl<TU64>::make();
}  // namespace ipsgpu
