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

// Persistent NODE launch: as many CTAs as fit on the GPU at once (at most one
// per item); each loops over its items.
cudaError_t qft_large_node_launch(const LargeArgs& a, int64_t rows, int64_t items, int nt, size_t smem,
                                  cudaStream_t st) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = nt == 256 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_large_node<qft_lib::kL1, 256>, 256, smem)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_large_node<qft_lib::kL1, 512>, 512, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)per_sm * sms;
  if (grid > items) grid = items;
  if (grid < 1) grid = 1;
  if (nt == 256) k_large_node<qft_lib::kL1, 256><<<(unsigned)grid, 256, smem, st>>>(a, rows);
  else k_large_node<qft_lib::kL1, 512><<<(unsigned)grid, 512, smem, st>>>(a, rows);
  return cudaGetLastError();
}

cudaError_t qft_large_tab_launch(const LargeArgs& a, int64_t rows, int LF, cudaStream_t st) {
  k_large_tab<<<(unsigned)rows, 256, 0, st>>>(a, LF);
  return cudaGetLastError();
}

cudaError_t qft_large_slice_launch(const LargeArgs& a, int phase, dim3 grid, cudaStream_t st) {
  k_large_slice<<<grid, kLargeNT, 0, st>>>(a, phase);
  return cudaGetLastError();
}
