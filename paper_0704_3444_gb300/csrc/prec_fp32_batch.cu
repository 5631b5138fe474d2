// prec_fp32_batch.cu -- the batched march and staged batch, float storage.
#include "table_impl.cuh"

namespace mclb {

void fill_fp32_batch(KernelTable& t) { fill_batch<float>(t); }

}  // namespace mclb
