// Algorithm 1 kernels for uint8 guides: every variant of the tuning table.
#include "common.cuh"

namespace glu {
GLU_DEFINE_STATUS(search_u8)
}  // namespace glu

#include "search_kernel.cuh"

namespace glu {
int search_launch_u8(int v, const SearchArgs* items, int n, cudaStream_t st) {
    return search_dispatch<uint8_t>(v, items, n, st);
}
}  // namespace glu
