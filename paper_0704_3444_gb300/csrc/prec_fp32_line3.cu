// prec_fp32_line3.cu -- the D1Q3 kernels, float storage.
#include "table_impl.cuh"

namespace mclb {

void fill_fp32_line3(KernelTable& t) { fill_line3<float>(t); }

}  // namespace mclb
