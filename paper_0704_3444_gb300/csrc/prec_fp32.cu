// prec_fp32.cu -- kernels and launchers for float distribution storage.
#include "table_impl.cuh"

namespace mclb {

const KernelTable& table_fp32()
{
    static const KernelTable t = make_table<float>(CU_TENSOR_MAP_DATA_TYPE_FLOAT32);
    return t;
}

}  // namespace mclb
