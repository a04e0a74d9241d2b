// qft_k_c2c_bf16.cu -- C2C row-engine kernels, StBF16 storage.
#include "qft_large.cuh"

int qft_launch_c2c_bf16(qft_plan p, int op, const void* in, void* out, cudaStream_t st) {
  return exec_c2c<StBF16>(p, op, in, out, st);
}
