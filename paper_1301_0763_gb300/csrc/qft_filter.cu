// qft_filter.cu -- the spectral-filter layer y = irfft(W (.) rfft(x)) on
// real rows x[B][C][N] with complex weights W[C][N/2+1], forward and backward,
// each a single pass of fused row-engine transforms per pair of rows.
//
// forward  (per row pair (b, c), (b+1, c)):  X = rfft(x) -> shared memory,
//          y = irfft(W (.) X).
// backward (per channel c, a slice of its row pairs):
//          G = irfft^H(gy) = (w_k/N) rfft(gy) -> shared memory,
//          X = rfft(x) (recomputed; nothing is saved by the forward),
//          acc += G (.) conj(X)  (the partial weight gradient, in shared memory),
//          gx = rfft^H(conj(W) (.) G);
//          the partials of a channel are summed in a fixed order afterwards, so
//          gW is deterministic.
#include "qft_large.cuh"

namespace {

constexpr int kFiltNT = 256;
constexpr int kFiltParts = 16;  // row-pair slices per channel in the backward pass (CTAs = channels x 16)

struct FiltLayout {
  size_t spec_off, spec_cells, acc_off, total;
};

__host__ __device__ inline FiltLayout filt_layout(int N, int LF, bool backward) {
  FiltLayout L;
  L.spec_off = (qft_lib::row_smem_bytes(N, LF) + 15) & ~(size_t)15;
  L.spec_cells = (size_t)N / 2 + 1;
  const size_t spec_bytes = qft_lib::align16(8 * L.spec_cells);
  L.acc_off = L.spec_off + 2 * spec_bytes;
  L.total = L.acc_off + (backward ? spec_bytes : 0);
  return L;
}

struct FiltArgs {
  const QftRowPlan* plan;
  const float* gsec;
  const float* x;
  const qc* W;
  const float* gy;
  float* y;      // forward output / backward gx
  qc* gwpart;    // [C][kFiltParts][N/2+1]
  int B, C, N;
};

__device__ __forceinline__ Eng filt_setup(unsigned char* smem, const FiltArgs& a) {
  QftRowPlan& P = *reinterpret_cast<QftRowPlan*>(smem);
  {
    const int* src = reinterpret_cast<const int*>(a.plan);
    int* dst = reinterpret_cast<int*>(smem);
    for (int i = threadIdx.x; i < (int)(sizeof(QftRowPlan) / 4); i += kFiltNT) dst[i] = src[i];
  }
  __syncthreads();
  const int N = 1 << P.r;
  float* sec = reinterpret_cast<float*>(smem + qft_lib::off_sec());
  for (int m = threadIdx.x; m <= N / 4; m += kFiltNT) sec[m] = a.gsec[m];
  __syncthreads();
  Eng e;
  e.side0 = reinterpret_cast<qc*>(smem + qft_lib::off_side0(N));
  e.side1 = reinterpret_cast<qc*>(smem + qft_lib::off_side0(N) + qft_lib::side_bytes(N));
  e.sec = sec; e.r = P.r; e.N = N;
  e.tabC = reinterpret_cast<qc*>(smem + qft_lib::off_tab(N));
  e.tabS = e.tabC + (N >> P.LF) / 2 + 1;
  e.lo0 = nullptr;
  e.lo1 = nullptr;
  return e;
}

#ifndef QFT_FILTER_BACKWARD_TU
__global__ void __launch_bounds__(kFiltNT, 2) k_filter_fwd(FiltArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Eng e = filt_setup(smem, a);
  const QftRowPlan& P = *reinterpret_cast<const QftRowPlan*>(smem);
  const int N = a.N, C = a.C;
  const FiltLayout L = filt_layout(N, P.LF, false);
  qc* spa = reinterpret_cast<qc*>(smem + L.spec_off);
  qc* spb = spa + qft_lib::align16(8 * L.spec_cells) / 8;
  const int64_t pairs = (int64_t)((a.B + 1) / 2) * C;
  for (int64_t item = blockIdx.x; item < pairs; item += gridDim.x) {
    const int c = (int)(item % C);
    const int b0 = 2 * (int)(item / C);
    const int64_t ra = (int64_t)b0 * C + c;
    const bool hasb = b0 + 1 < a.B;
    const int64_t rb = ra + C;
    IoR2CSpec f;
    f.ina = a.x + ra * N; f.inb = hasb ? a.x + rb * N : nullptr;
    f.spa = spa; f.spb = spb; f.N = N; f.wscale = 0.f;
    run_row_phases<qft_lib::kL1, kFiltNT>(P, e, f, 0);
    IoC2RFilt g;
    g.spa = spa; g.spb = hasb ? spb : nullptr;
    g.w = a.W + (int64_t)c * (N / 2 + 1); g.conjw = false;
    g.outa = a.y + ra * N; g.outb = hasb ? a.y + rb * N : nullptr;
    g.N = N; g.wmid = 2.f; g.scale = 1.f / (float)N;
    run_row_phases<qft_lib::kL1, kFiltNT>(P, e, g, 0);
  }
}

#else
// blockIdx.x = c * kFiltParts + part
__global__ void __launch_bounds__(kFiltNT, 1) k_filter_bwd(FiltArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Eng e = filt_setup(smem, a);
  const QftRowPlan& P = *reinterpret_cast<const QftRowPlan*>(smem);
  const int N = a.N, C = a.C, H = N / 2 + 1;
  const FiltLayout L = filt_layout(N, P.LF, true);
  qc* ga = reinterpret_cast<qc*>(smem + L.spec_off);
  qc* gb = ga + qft_lib::align16(8 * L.spec_cells) / 8;
  qc* acc = reinterpret_cast<qc*>(smem + L.acc_off);
  const int c = blockIdx.x / kFiltParts;
  const int part = blockIdx.x % kFiltParts;
  const int npairs = (a.B + 1) / 2;
  const int p0 = (int)((int64_t)npairs * part / kFiltParts);
  const int p1 = (int)((int64_t)npairs * (part + 1) / kFiltParts);
  for (int k = threadIdx.x; k < H; k += kFiltNT) acc[k] = mkc(0.f, 0.f);
  __syncthreads();
  for (int pr = p0; pr < p1; ++pr) {
    const int b0 = 2 * pr;
    const int64_t ra = (int64_t)b0 * C + c;
    const bool hasb = b0 + 1 < a.B;
    const int64_t rb = ra + C;
    IoR2CSpec f;                      // G = (w_k / N) rfft(gy)
    f.ina = a.gy + ra * N; f.inb = hasb ? a.gy + rb * N : nullptr;
    f.spa = ga; f.spb = gb; f.N = N; f.wscale = 1.f / (float)N;
    run_row_phases<qft_lib::kL1, kFiltNT>(P, e, f, 0);
    IoR2CAccum h;                     // acc += G conj(rfft(x))
    h.ina = a.x + ra * N; h.inb = hasb ? a.x + rb * N : nullptr;
    h.ga = ga; h.gb = gb; h.acc = acc; h.N = N;
    run_row_phases<qft_lib::kL1, kFiltNT>(P, e, h, 0);
    IoC2RFilt g;                      // gx = rfft^H(conj(W) G)
    g.spa = ga; g.spb = hasb ? gb : nullptr;
    g.w = a.W + (int64_t)c * H; g.conjw = true;
    g.outa = a.y + ra * N; g.outb = hasb ? a.y + rb * N : nullptr;
    g.N = N; g.wmid = 1.f; g.scale = 1.f;
    run_row_phases<qft_lib::kL1, kFiltNT>(P, e, g, 0);
  }
  qc* dst = a.gwpart + ((int64_t)c * kFiltParts + part) * H;
  for (int k = threadIdx.x; k < H; k += kFiltNT) dst[k] = acc[k];
}

// gW[c][k] = sum over parts in order
__global__ void k_filter_reduce(const qc* __restrict__ gwpart, qc* __restrict__ gw, int C, int H) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)C * H) return;
  const int c = (int)(i / H), k = (int)(i % H);
  qc s = gwpart[((int64_t)c * kFiltParts) * H + k];
  for (int p = 1; p < kFiltParts; ++p) s = cadd(s, gwpart[((int64_t)c * kFiltParts + p) * H + k]);
  gw[i] = s;
}
#endif  // QFT_FILTER_BACKWARD_TU

FiltArgs filt_args(qft_plan p, const float* x, const void* W, const float* gy, float* out) {
  FiltArgs a;
  a.plan = p->d_plan; a.gsec = p->d_sec; a.x = x; a.W = static_cast<const qc*>(W); a.gy = gy; a.y = out;
  a.gwpart = reinterpret_cast<qc*>(p->scratch);
  a.B = (int)p->batch; a.C = (int)p->channels; a.N = (int)p->n;
  return a;
}

}  // namespace

// The backward kernels are compiled in their own translation unit
// (qft_filter_bwd.cu), in parallel with the forward one.
int qft_launch_filter_bwd(qft_plan p, const float* x, const void* W, const float* gy, float* gx, void* gW,
                          cudaStream_t st);

#ifdef QFT_FILTER_BACKWARD_TU
int qft_launch_filter_bwd(qft_plan p, const float* x, const void* W, const float* gy, float* gx, void* gW,
                          cudaStream_t st) {
  const FiltArgs a = filt_args(p, x, W, gy, gx);
  const int smem = (int)filt_layout(a.N, p->host_plan.LF, true).total;
  cudaError_t e = cudaFuncSetAttribute(k_filter_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return qft_set_cuda(p, e);
  k_filter_bwd<<<(unsigned)(a.C * kFiltParts), kFiltNT, smem, st>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return qft_set_cuda(p, e);
  const int H = a.N / 2 + 1;
  const int64_t n = (int64_t)a.C * H;
  k_filter_reduce<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a.gwpart, static_cast<qc*>(gW), a.C, H);
  return qft_set_cuda(p, cudaGetLastError());
}
#else

#ifndef QFT_FILTER_BACKWARD_TU
int qft_filter_smem(int N, int LF, int backward) { return (int)filt_layout(N, LF, backward != 0).total; }
int qft_filter_parts() { return kFiltParts; }
#endif

int qft_launch_filter(qft_plan p, int backward, const float* x, const void* W, const float* gy, float* out,
                      void* gW, cudaStream_t st) {
  if (backward) return qft_launch_filter_bwd(p, x, W, gy, out, gW, st);
  const FiltArgs a = filt_args(p, x, W, gy, out);
  const int smem = qft_filter_smem(a.N, p->host_plan.LF, backward);
  {
    cudaError_t e = cudaFuncSetAttribute(k_filter_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return qft_set_cuda(p, e);
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_filter_fwd, kFiltNT, smem);
    if (per_sm < 1) per_sm = 1;
    const int64_t pairs = (int64_t)((a.B + 1) / 2) * a.C;
    int64_t grid = (int64_t)per_sm * p->sms;
    if (grid > pairs) grid = pairs;
    if (grid < 1) grid = 1;
    k_filter_fwd<<<(unsigned)grid, kFiltNT, smem, st>>>(a);
    return qft_set_cuda(p, cudaGetLastError());
  }
}
#endif  // QFT_FILTER_BACKWARD_TU
