// qft_k_node.cu -- the NODE and SLICE kernels of the large-row path (they do
// not depend on the transform's IO), compiled once for every launcher, with
// and without the compensated segments.
#define QFT_NODE_TU 1
#include "qft_large.cuh"

template <int NT, bool COMP>
static cudaError_t node_attr(size_t smem) {
  return cudaFuncSetAttribute(k_large_node<qft_lib::kL1, NT, COMP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem);
}

cudaError_t qft_large_node_prepare(int nt, size_t smem, int comp) {
  if (comp) return nt == 256 ? node_attr<256, true>(smem) : node_attr<512, true>(smem);
  return nt == 256 ? node_attr<256, false>(smem) : node_attr<512, false>(smem);
}

// Persistent NODE launch: as many CTAs as fit on the GPU at once (at most one
// per item); each loops over its items.
template <int NT, bool COMP>
static cudaError_t node_launch(const LargeArgs& a, int64_t rows, int64_t items, size_t smem, cudaStream_t st) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_large_node<qft_lib::kL1, NT, COMP>, NT, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)per_sm * sms;
  if (grid > items) grid = items;
  if (grid < 1) grid = 1;
  k_large_node<qft_lib::kL1, NT, COMP><<<(unsigned)grid, NT, smem, st>>>(a, rows);
  return cudaGetLastError();
}

cudaError_t qft_large_node_launch(const LargeArgs& a, int64_t rows, int64_t items, int nt, size_t smem,
                                  cudaStream_t st, int comp) {
  if (comp) return nt == 256 ? node_launch<256, true>(a, rows, items, smem, st)
                             : node_launch<512, true>(a, rows, items, smem, st);
  return nt == 256 ? node_launch<256, false>(a, rows, items, smem, st)
                   : node_launch<512, false>(a, rows, items, smem, st);
}

// Threads per row: 256 from 2048 rows on, 512 from 512, else 1024.  Measured
// on the batched workload (2^28 elements; 4096, 1024 and 256 rows at 2^16,
// 2^18 and 2^20): 256 threads were best at 2^16, 512 at 2^18, 1024 at 2^20.
cudaError_t qft_large_tab_launch(const LargeArgs& a, int64_t rows, int LF, cudaStream_t st) {
  if (rows >= 2048) k_large_tab<256><<<(unsigned)rows, 256, 0, st>>>(a, LF);
  else if (rows >= 512) k_large_tab<512><<<(unsigned)rows, 512, 0, st>>>(a, LF);
  else k_large_tab<1024><<<(unsigned)rows, 1024, 0, st>>>(a, LF);
  return cudaGetLastError();
}

cudaError_t qft_large_slice_launch(const LargeArgs& a, int phase, dim3 grid, cudaStream_t st, int comp) {
  if (comp) k_large_slice<true><<<grid, kLargeNT, 0, st>>>(a, phase);
  else k_large_slice<false><<<grid, kLargeNT, 0, st>>>(a, phase);
  return cudaGetLastError();
}

cudaError_t qft_large_slice_ip_launch(const LargeArgs& a, int phase, int nblk, int64_t rows, cudaStream_t st,
                                      int comp) {
  if (nblk > 1) {   // block edges 1 .. nblk-1
    const dim3 hg((unsigned)((nblk - 1 + 255) / 256), (unsigned)rows);
    if (comp) k_large_halo<true><<<hg, 256, 0, st>>>(a, phase, nblk);
    else k_large_halo<false><<<hg, 256, 0, st>>>(a, phase, nblk);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const dim3 g((unsigned)nblk, (unsigned)rows);
  if (comp) k_large_slice_ip<true><<<g, QFT_IP_TASKS, 0, st>>>(a, phase);
  else k_large_slice_ip<false><<<g, QFT_IP_TASKS, 0, st>>>(a, phase);
  return cudaGetLastError();
}
