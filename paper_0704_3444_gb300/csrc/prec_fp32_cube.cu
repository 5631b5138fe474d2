// prec_fp32_cube.cu -- the D3Q19 kernels, float storage.
#include "table_impl.cuh"

namespace mclb {

void fill_fp32_cube(KernelTable& t) { fill_cube<float>(t); }

}  // namespace mclb
