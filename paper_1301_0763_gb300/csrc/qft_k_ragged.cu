// qft_k_ragged.cu -- the row kernels of one length class of a ragged plan.
#include "qft_large.cuh"

int qft_launch_ragged_class(qft_plan sub, const QftIoArgs* d_args, const int64_t* d_offsets,
                            const int32_t* d_rows, cudaStream_t st) {
  return exec_ragged_class(sub, d_args, d_offsets, d_rows, st);
}
