// qft_k_node.cu -- the NODE and SLICE kernels of the large-row path (they do
// not depend on the transform's IO), compiled once for every launcher.
#define QFT_NODE_TU 1
#include "qft_large.cuh"

cudaError_t qft_large_node_prepare(int nt, size_t smem) {
  return nt == 256 ? cudaFuncSetAttribute(k_large_node<qft_lib::kL1, 256>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                   : cudaFuncSetAttribute(k_large_node<qft_lib::kL1, 512>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t qft_large_node_launch(const LargeArgs& a, dim3 grid, int nt, size_t smem, cudaStream_t st) {
  if (nt == 256) k_large_node<qft_lib::kL1, 256><<<grid, 256, smem, st>>>(a);
  else k_large_node<qft_lib::kL1, 512><<<grid, 512, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t qft_large_slice_launch(const LargeArgs& a, int phase, dim3 grid, cudaStream_t st) {
  k_large_slice<<<grid, kLargeNT, 0, st>>>(a, phase);
  return cudaGetLastError();
}
