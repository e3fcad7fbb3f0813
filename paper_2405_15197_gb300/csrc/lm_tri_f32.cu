// Triangulation kernels, FP32 arithmetic with FP64 stability steps.
#include "lm_tri_impl.cuh"
namespace lm {
template cudaError_t launch_tri_count<float>(const TriLaunch<float>&, cudaStream_t);
template cudaError_t launch_tri_emit<float>(const TriLaunch<float>&, cudaStream_t);
size_t node64_bytes() { return sizeof(Node64); }
int64_t tri_scratch_warps() { return 152 * 64 * 2; }
cudaError_t launch_chunk_begin(int64_t* cursor, int64_t stride, int64_t chunk, int64_t i0, int64_t i1, int64_t* range,
                               cudaStream_t st) {
  count_launch();
  k_chunk_begin<<<1, 32, 0, st>>>(cursor, stride, chunk, i0, i1, range);
  return cudaGetLastError();
}
}
