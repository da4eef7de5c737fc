// Kernels of the mixed precision form (FP32 pair arithmetic, FP64
// positions, int64 fixed-point force sums).
#include "md_kernels.cuh"

namespace md {
template KernelTable<Mixed> make_kernel_table<Mixed>();
}
