// prec_fp16_staged.cu -- the staged schedule and the diagnostics on D2Q9, __half storage.
#include "table_impl.cuh"

namespace mclb {

void fill_fp16_staged(KernelTable& t) { fill_staged<__half>(t); }

}  // namespace mclb
