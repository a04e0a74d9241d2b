// qft_k_real.cu -- R2C / C2R row-engine kernels (two real rows per CTA pass).
#include "qft_large.cuh"

int qft_launch_real(qft_plan p, int op, const void* in, void* out, cudaStream_t st) {
  return exec_r2c(p, op, in, out, st);
}
