// qft_k_r2r.cu -- standalone DCT-0 / DST-0 kernels (eqs qft_0B, qft_0C): the
// dct and dst recursions of Sec. 5 on their own, two real rows per CTA pass.
#include "qft_large.cuh"

template <bool DST>
static int exec_r2r(qft_plan p, const void* in, void* out, cudaStream_t st) {
  FacR2R<DST> f;
  f.in = static_cast<const float*>(in);
  f.out = static_cast<float*>(out);
  f.rows = p->batch;
  f.N = (int)p->n;
  return launch_any<FacR2R<DST>>(p, f, (p->batch + 1) / 2, st);
}

int qft_launch_r2r(qft_plan p, const void* in, void* out, cudaStream_t st) {
  return p->kind == QFT_KIND_DST0 ? exec_r2r<true>(p, in, out, st) : exec_r2r<false>(p, in, out, st);
}
