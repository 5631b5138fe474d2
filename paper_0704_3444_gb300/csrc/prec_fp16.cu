// prec_fp16.cu -- the kernel table for __half distribution storage, assembled from the
// parts compiled in prec_fp16_*.cu.
#include "table_impl.cuh"

namespace mclb {

void fill_fp16_march(KernelTable& t);   // prec_fp16_march.cu
void fill_fp16_staged(KernelTable& t);   // prec_fp16_staged.cu
void fill_fp16_batch(KernelTable& t);   // prec_fp16_batch.cu

const KernelTable& table_fp16()
{
    static const KernelTable t = [] {
        KernelTable x{};
        table_base<__half>(x, CU_TENSOR_MAP_DATA_TYPE_FLOAT16);
        fill_fp16_march(x);
        fill_fp16_staged(x);
        fill_fp16_batch(x);
        return x;
    }();
    return t;
}

}  // namespace mclb
