// Meta-mesh kernels, FP32 arithmetic with FP64 stability steps.
#include "lm_mm_impl.cuh"
namespace lm {
template cudaError_t launch_metamesh<float>(bool, const MMLaunch<float>&, const MMBuckets&, int, cudaStream_t, int*);
template int metamesh_ctas_per_sm<float>();
template cudaError_t launch_mm_gather<float>(const MMLaunch<float>&, cudaStream_t);
}
