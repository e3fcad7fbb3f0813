// Meta-mesh kernels, FP64 arithmetic (FP64 lattices).
#include "lm_mm_impl.cuh"
namespace lm {
template cudaError_t launch_metamesh<double>(int, bool, const MMLaunch<double>&, int, int, cudaStream_t, int*);
template cudaError_t launch_mm_gather<double>(const MMLaunch<double>&, cudaStream_t);
}
