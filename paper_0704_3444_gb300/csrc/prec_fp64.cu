// prec_fp64.cu -- kernels and launchers for double distribution storage.
#include "table_impl.cuh"

namespace mclb {

const KernelTable& table_fp64()
{
    static const KernelTable t = make_table<double>(CU_TENSOR_MAP_DATA_TYPE_FLOAT64);
    return t;
}

}  // namespace mclb
