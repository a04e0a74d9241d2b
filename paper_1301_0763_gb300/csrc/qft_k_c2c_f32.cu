// qft_k_c2c_f32.cu -- C2C row-engine kernels, StC64 storage.
#include "qft_large.cuh"

int qft_launch_c2c_f32(qft_plan p, int op, const void* in, void* out, cudaStream_t st) {
  return exec_c2c<StC64>(p, op, in, out, st);
}

int qft_launch_ragged_class(qft_plan sub, const QftIoArgs* d_args, const int64_t* d_offsets,
                            const int32_t* d_rows, cudaStream_t st) {
  return exec_ragged_class(sub, d_args, d_offsets, d_rows, st);
}
