// qft_k_c2c_f32.cu -- C2C row-engine kernels, StC64 storage.
#include "qft_large.cuh"

int qft_launch_c2c_f32(qft_plan p, int op, const void* in, void* out, cudaStream_t st) {
  return exec_c2c<StC64>(p, op, in, out, st);
}
