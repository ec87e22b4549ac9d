// Compile-time plane-transform plans for N' = 512, 1024 (see transforms_impl.cuh).
#include "transforms_impl.cuh"

namespace ws {
namespace tf {
const Ops &ops_512() {
    static const Ops o = ops_of<512>();
    return o;
}
const Ops &ops_1024() {
    static const Ops o = ops_of<1024>();
    return o;
}
}  // namespace tf
}  // namespace ws
