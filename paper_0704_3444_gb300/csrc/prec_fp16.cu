// prec_fp16.cu -- kernels and launchers for __half distribution storage.
#include "table_impl.cuh"

namespace mclb {

const KernelTable& table_fp16()
{
    static const KernelTable t = make_table<__half>(CU_TENSOR_MAP_DATA_TYPE_FLOAT16);
    return t;
}

}  // namespace mclb
