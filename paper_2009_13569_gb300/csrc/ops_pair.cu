// ops_pair.cu -- kernel instantiations for the pair element type.
#include "ops_impl.cuh"

namespace ipsgpu {
const TypeOps ops_pair = OpsImpl<TPair>::make();
}  // namespace ipsgpu
