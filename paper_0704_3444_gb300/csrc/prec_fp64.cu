// prec_fp64.cu -- the kernel table for double distribution storage, assembled from the
// parts compiled in prec_fp64_*.cu.
#include "table_impl.cuh"

namespace mclb {

void fill_fp64_march(KernelTable& t);   // prec_fp64_march.cu
void fill_fp64_staged(KernelTable& t);   // prec_fp64_staged.cu
void fill_fp64_batch(KernelTable& t);   // prec_fp64_batch.cu
void fill_fp64_line3(KernelTable& t);   // prec_fp64_line3.cu
void fill_fp64_cube(KernelTable& t);   // prec_fp64_cube.cu

const KernelTable& table_fp64()
{
    static const KernelTable t = [] {
        KernelTable x{};
        table_base<double>(x, CU_TENSOR_MAP_DATA_TYPE_FLOAT64);
        fill_fp64_march(x);
        fill_fp64_staged(x);
        fill_fp64_batch(x);
        fill_fp64_line3(x);
        fill_fp64_cube(x);
        return x;
    }();
    return t;
}

}  // namespace mclb
