// Compile-time plane-transform plans for N' = 4096 (see transforms_impl.cuh).
#include "transforms_impl.cuh"

namespace ws {
namespace tf {
const Ops &ops_4096() {
    static const Ops o = ops_of<4096>();
    return o;
}
}  // namespace tf
}  // namespace ws
