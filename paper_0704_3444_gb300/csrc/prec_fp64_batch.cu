// prec_fp64_batch.cu -- the batched march and staged batch, double storage.
#include "table_impl.cuh"

namespace mclb {

void fill_fp64_batch(KernelTable& t) { fill_batch<double>(t); }

}  // namespace mclb
