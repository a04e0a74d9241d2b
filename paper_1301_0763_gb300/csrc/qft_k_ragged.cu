// qft_k_ragged.cu -- the row kernels of one length class of a ragged plan.
#include "qft_large.cuh"

// N = 2 rows of a ragged plan
__global__ void k_ragged_n2(FacRaggedC2C<StC64> fac, int64_t rows) {
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= rows) return;
  const auto io = fac.make(row);
  const qc a = io.ld(0), b = io.ld(1);
  io.st(0, cadd(a, b));
  io.st(1, csub(a, b));
}

static inline int exec_ragged_class(qft_plan sub, const QftIoArgs* d_args, const int64_t* d_offsets,
                                    const int32_t* d_rows, cudaStream_t st) {
  FacRaggedC2C<StC64> f;
  f.args = d_args; f.offsets = d_offsets; f.rows = d_rows; f.N = (int)sub->n;
  if (sub->r == 1) {
    const int64_t blocks = (sub->batch + 127) / 128;
    k_ragged_n2<<<(unsigned)blocks, 128, 0, st>>>(f, sub->batch);
    return qft_set_cuda(sub, cudaGetLastError());
  }
  return launch_any<FacRaggedC2C<StC64>>(sub, f, sub->batch, st);
}

int qft_launch_ragged_class(qft_plan sub, const QftIoArgs* d_args, const int64_t* d_offsets,
                            const int32_t* d_rows, cudaStream_t st) {
  return exec_ragged_class(sub, d_args, d_offsets, d_rows, st);
}
