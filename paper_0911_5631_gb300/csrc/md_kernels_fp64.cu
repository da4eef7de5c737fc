// Kernels of the FP64 form (all arithmetic in double precision).
#include "md_kernels.cuh"

namespace md {
template KernelTable<F64> make_kernel_table<F64>();
}
