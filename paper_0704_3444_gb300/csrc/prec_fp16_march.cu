// prec_fp16_march.cu -- the single-pass kernel on D2Q9, __half storage.
#include "table_impl.cuh"

namespace mclb {

void fill_fp16_march(KernelTable& t) { fill_march<__half>(t); }

}  // namespace mclb
