// prec_bf16.cu -- kernels and launchers for __nv_bfloat16 distribution storage.
#include "table_impl.cuh"

namespace mclb {

const KernelTable& table_bf16()
{
    static const KernelTable t = make_table<__nv_bfloat16>(CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
    return t;
}

}  // namespace mclb
