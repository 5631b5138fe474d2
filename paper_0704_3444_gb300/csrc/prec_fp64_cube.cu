// prec_fp64_cube.cu -- the D3Q19 kernels, double storage.
#include "table_impl.cuh"

namespace mclb {

void fill_fp64_cube(KernelTable& t) { fill_cube<double>(t); }

}  // namespace mclb
