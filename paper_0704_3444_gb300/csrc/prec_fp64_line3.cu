// prec_fp64_line3.cu -- the D1Q3 kernels, double storage.
#include "table_impl.cuh"

namespace mclb {

void fill_fp64_line3(KernelTable& t) { fill_line3<double>(t); }

}  // namespace mclb
