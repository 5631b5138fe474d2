// prec_fp32_march.cu -- the single-pass kernel on D2Q9, float storage.
#include "table_impl.cuh"

namespace mclb {

void fill_fp32_march(KernelTable& t) { fill_march<float>(t); }

}  // namespace mclb
