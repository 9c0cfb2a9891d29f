// Instantiation of the row-pass kernels for block width 32 (FP64 and complex64).
#include "blcoc_rowpass.cuh"
namespace blcoc {
template const KernelSet& kernel_set<32, double>();
template const KernelSet& kernel_set<32, float>();
}
namespace blcoc {
template const KernelSet& kernel_set_tc<32>();
}
