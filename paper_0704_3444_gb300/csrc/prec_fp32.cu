// prec_fp32.cu -- the kernel table for float distribution storage, assembled from the
// parts compiled in prec_fp32_*.cu.
#include "table_impl.cuh"

namespace mclb {

void fill_fp32_march(KernelTable& t);   // prec_fp32_march.cu
void fill_fp32_staged(KernelTable& t);   // prec_fp32_staged.cu
void fill_fp32_batch(KernelTable& t);   // prec_fp32_batch.cu
void fill_fp32_line3(KernelTable& t);   // prec_fp32_line3.cu
void fill_fp32_cube(KernelTable& t);   // prec_fp32_cube.cu

const KernelTable& table_fp32()
{
    static const KernelTable t = [] {
        KernelTable x{};
        table_base<float>(x, CU_TENSOR_MAP_DATA_TYPE_FLOAT32);
        fill_fp32_march(x);
        fill_fp32_staged(x);
        fill_fp32_batch(x);
        fill_fp32_line3(x);
        fill_fp32_cube(x);
        return x;
    }();
    return t;
}

}  // namespace mclb
