// Instantiation of the row-pass kernels for block width 8 (FP64 and complex64).
#include "blcoc_rowpass.cuh"
namespace blcoc {
template const KernelSet& kernel_set<8, double>();
template const KernelSet& kernel_set<8, float>();
}
namespace blcoc {
template const KernelSet& kernel_set_tc<8>();
}
