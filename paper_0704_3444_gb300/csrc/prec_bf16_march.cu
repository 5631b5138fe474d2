// prec_bf16_march.cu -- the single-pass kernel on D2Q9, __nv_bfloat16 storage.
#include "table_impl.cuh"

namespace mclb {

void fill_bf16_march(KernelTable& t) { fill_march<__nv_bfloat16>(t); }

}  // namespace mclb
