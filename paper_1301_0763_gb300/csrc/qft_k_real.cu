// qft_k_real.cu -- R2C / C2R row-engine kernels (two real rows per CTA pass).
#include "qft_large.cuh"

static inline int exec_r2c(qft_plan p, int op, const void* in, void* out, cudaStream_t st) {
  const int64_t items = (p->batch + 1) / 2;
  const int N = (int)p->n;
  if (op == QFT_OP_FORWARD || op == QFT_OP_INVERSE_ADJOINT) {
    FacR2C<StC64> f;
    f.in = static_cast<const float*>(in);
    f.out = static_cast<qc*>(out);
    f.rows = p->batch; f.N = N;
    f.wscale = op == QFT_OP_FORWARD ? 0.f : 1.f / (float)N;
    return launch_any<FacR2C<StC64>>(p, f, items, st, (size_t)2 * N * sizeof(float), ((uintptr_t)in % 16) == 0);
  }
  if (op == QFT_OP_INVERSE || op == QFT_OP_FORWARD_ADJOINT) {
    FacC2R<StC64> f;
    f.in = static_cast<const qc*>(in);
    f.out = static_cast<float*>(out);
    f.rows = p->batch; f.N = N;
    if (op == QFT_OP_INVERSE) { f.wmid = 2.f; f.scale = 1.f / (float)N; }
    else { f.wmid = 1.f; f.scale = 1.f; }
    return launch_any<FacC2R<StC64>>(p, f, items, st);
  }
  return QFT_ERR_INVALID_ARG;
}

int qft_launch_real(qft_plan p, int op, const void* in, void* out, cudaStream_t st) {
  return exec_r2c(p, op, in, out, st);
}
