// Compile-time plane-transform plans for N' = 2048 (see transforms_impl.cuh).
#include "transforms_impl.cuh"

namespace ws {
namespace tf {
const Ops &ops_2048() {
    static const Ops o = ops_of<2048>();
    return o;
}
}  // namespace tf
}  // namespace ws
