// prec_fp64_march.cu -- the single-pass kernel on D2Q9, double storage.
#include "table_impl.cuh"

namespace mclb {

void fill_fp64_march(KernelTable& t) { fill_march<double>(t); }

}  // namespace mclb
