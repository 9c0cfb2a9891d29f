// Instantiation of the row-pass kernels for block width 16 (FP64 and complex64).
#include "blcoc_rowpass.cuh"
namespace blcoc {
template const KernelSet& kernel_set<16, double>();
template const KernelSet& kernel_set<16, float>();
}
namespace blcoc {
template const KernelSet& kernel_set_tc<16>();
}
