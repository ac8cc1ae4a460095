// ops_rec100.cu -- kernel instantiations for the rec100 element type.
#include "ops_impl.cuh"

namespace ipsgpu {
const TypeOps ops_rec100 = OpsImpl<TRec100>::make();
}  // namespace ipsgpu
