// Triangulation kernels, FP64 arithmetic (FP64 lattices).
#include "lm_tri_impl.cuh"
namespace lm {
template cudaError_t launch_tri_count<double>(const TriLaunch<double>&, cudaStream_t);
template cudaError_t launch_tri_emit<double>(const TriLaunch<double>&, cudaStream_t);
}
