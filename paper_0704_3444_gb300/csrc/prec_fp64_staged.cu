// prec_fp64_staged.cu -- the staged schedule and the diagnostics on D2Q9, double storage.
#include "table_impl.cuh"

namespace mclb {

void fill_fp64_staged(KernelTable& t) { fill_staged<double>(t); }

}  // namespace mclb
