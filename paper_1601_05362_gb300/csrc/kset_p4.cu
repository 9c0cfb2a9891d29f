// Instantiation of the row-pass kernels for block width 4.
#include "blcoc_rowpass.cuh"
namespace blcoc {
template const KernelSet& kernel_set<4>();
}
