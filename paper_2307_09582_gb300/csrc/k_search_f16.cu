// Algorithm 1 kernels for float16 guides: every variant of the tuning table.
#include "common.cuh"

namespace glu {
GLU_DEFINE_STATUS(search_f16)
}  // namespace glu

#include "search_kernel.cuh"

namespace glu {
int search_launch_f16(int v, const SearchArgs* items, int n, cudaStream_t st) {
    return search_dispatch<__half>(v, items, n, st);
}
}  // namespace glu
