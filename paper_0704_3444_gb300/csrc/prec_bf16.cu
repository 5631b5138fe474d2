// prec_bf16.cu -- the kernel table for __nv_bfloat16 distribution storage, assembled from the
// parts compiled in prec_bf16_*.cu.
#include "table_impl.cuh"

namespace mclb {

void fill_bf16_march(KernelTable& t);   // prec_bf16_march.cu
void fill_bf16_staged(KernelTable& t);   // prec_bf16_staged.cu
void fill_bf16_batch(KernelTable& t);   // prec_bf16_batch.cu

const KernelTable& table_bf16()
{
    static const KernelTable t = [] {
        KernelTable x{};
        table_base<__nv_bfloat16>(x, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
        fill_bf16_march(x);
        fill_bf16_staged(x);
        fill_bf16_batch(x);
        return x;
    }();
    return t;
}

}  // namespace mclb
