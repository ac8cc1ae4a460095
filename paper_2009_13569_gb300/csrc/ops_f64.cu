// ops_f64.cu -- kernel instantiations for the f64 element type.
#include "ops_impl.cuh"

namespace ipsgpu {
const TypeOps ops_f64 = OpsImpl<TF64>::make();
}  // namespace ipsgpu
