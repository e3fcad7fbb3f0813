// Meta-mesh kernels, FP64 arithmetic (FP64 lattices).
#include "lm_mm_impl.cuh"
namespace lm {
template cudaError_t launch_metamesh<double>(bool, const MMLaunch<double>&, const MMBuckets&, int, cudaStream_t, int*);
template int metamesh_ctas_per_sm<double>();
template cudaError_t launch_mm_gather<double>(const MMLaunch<double>&, cudaStream_t);
}
