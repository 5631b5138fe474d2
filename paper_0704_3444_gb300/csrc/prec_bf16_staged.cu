// prec_bf16_staged.cu -- the staged schedule and the diagnostics on D2Q9, __nv_bfloat16 storage.
#include "table_impl.cuh"

namespace mclb {

void fill_bf16_staged(KernelTable& t) { fill_staged<__nv_bfloat16>(t); }

}  // namespace mclb
