// prec_bf16_batch.cu -- the batched march and staged batch, __nv_bfloat16 storage.
#include "table_impl.cuh"

namespace mclb {

void fill_bf16_batch(KernelTable& t) { fill_batch<__nv_bfloat16>(t); }

}  // namespace mclb
