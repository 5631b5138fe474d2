// prec_fp32_staged.cu -- the staged schedule and the diagnostics on D2Q9, float storage.
#include "table_impl.cuh"

namespace mclb {

void fill_fp32_staged(KernelTable& t) { fill_staged<float>(t); }

}  // namespace mclb
