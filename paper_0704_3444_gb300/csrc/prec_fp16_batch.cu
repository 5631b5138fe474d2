// prec_fp16_batch.cu -- the batched march and staged batch, __half storage.
#include "table_impl.cuh"

namespace mclb {

void fill_fp16_batch(KernelTable& t) { fill_batch<__half>(t); }

}  // namespace mclb
