// qft_k_fixed.cu -- the fixed-point variant's kernel (qft_fixed.cuh) and its
// launcher.
//
// One CTA transforms G rows at a time in shared memory (persistent grid over
// the rows; G > 1 for rows up to 2^9).  A row is a sequence of steps -- fold,
// the forward depths of the class trees, the backward heights (tree nodes
// and the class chain), the CDFT combine -- and every step has two phases
// separated by a CTA barrier: each thread evaluates its items (values kept in
// registers) and takes their block maxima (butterfly shuffles within a warp
// for blocks of fewer than 32 items, which are aligned runs of lanes; one
// shared-memory atomicMax per warp for larger blocks); after the barrier it
// stores them, shifted, in place (every read of the step came before it).
#include "qft_internal.h"
#include "qft_fixed.cuh"

static_assert(qfx::kMaxLog2 == qft_lib::kFixedMaxLog2, "fixed-point row limit");

namespace {
using namespace qfx;

// Maximum of `k` over the aligned block of `seg` consecutive items holding
// item w (seg a power of two; 0 for a lane without work).  Blocks of 32 items
// or more fill whole warps: one warp reduction, and one shared-memory
// atomicMax per warp into slot[first item / 32].  Smaller blocks sit inside a
// warp and reduce with xor shuffles.
__device__ __forceinline__ int block_max(int k, int seg, int* slot, int w) {
  if (__all_sync(0xffffffffu, seg >= 32)) {
    k = (int)__reduce_max_sync(0xffffffffu, (unsigned)k);
    if ((threadIdx.x & 31) == 0) atomicMax(slot + ((w & ~(seg - 1)) >> 5), k);
    return k;
  }
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_xor_sync(0xffffffffu, k, o);
    if (o < seg) k = max(k, t);
  }
  return k;
}
__device__ __forceinline__ int block_get(int k, int seg, const int* slot, int w) {
  return seg >= 32 ? slot[(w & ~(seg - 1)) >> 5] : k;
}

// One step over `items` items of the CTA's rows, NI items per thread: ev(w,
// v) evaluates an item (its values stay in registers), st(w, v, max1, max2)
// stores it after the barrier.  TWO: the step has a second key.
template <int NT, int NI, bool TWO, class EV, class ST>
__device__ __forceinline__ void fx_step(int* slots, int NS, int items, EV ev, ST st) {
  Val v[NI];
#pragma unroll
  for (int kk = 0; kk < NI; ++kk) {
    const int w = threadIdx.x + kk * NT;
    if (w < items) ev(w, v[kk]);
    else val_none(v[kk]);
    v[kk].k1 = block_max(v[kk].k1, v[kk].seg, slots, w);
    if (TWO) v[kk].k2 = block_max(v[kk].k2, v[kk].seg, slots + NS, w);
  }
  __syncthreads();
#pragma unroll
  for (int kk = 0; kk < NI; ++kk) {
    const int w = threadIdx.x + kk * NT;
    if (v[kk].seg)
      st(w, v[kk], block_get(v[kk].k1, v[kk].seg, slots, w), TWO ? block_get(v[kk].k2, v[kk].seg, slots + NS, w) : 0);
  }
}

// NT threads and G = 2^lgG rows per CTA pass, K NT = G N: the fold, backward
// and final steps have K/2 items per thread, the forward steps K/4.
// 64 registers a thread (1024 resident threads per SM): measured faster than
// the unbounded allocation (110-120 registers) at every length, spills included
template <int NT, int K>
__global__ void __launch_bounds__(NT, 1024 / NT) k_fixed(const uint32_t* __restrict__ z, Cell* __restrict__ out,
                                              int* __restrict__ eout, const Sec* __restrict__ sec, int r,
                                              int64_t batch, int lgG) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int N = 1 << r, G = 1 << lgG, tid = threadIdx.x;
  if (N == 2) {   // one row per thread
    for (int64_t row = (int64_t)blockIdx.x * NT + tid; row < batch; row += (int64_t)gridDim.x * NT)
      row_n2(z + 2 * row, out + 2 * row, eout + row);
    return;
  }
  const int rbytes = (int)row_bytes(N);
  const int NS = slot_count(G * N);
  int* slot_base = reinterpret_cast<int*>(sm + G * rbytes);   // [2 alternates][2 keys][NS]
  const auto row_of = [&](int g) { return make_row(sm + g * rbytes, r, sec); };
  for (int64_t r0 = (int64_t)blockIdx.x * G; r0 < batch; r0 += (int64_t)gridDim.x * G) {
    const int gv = batch - r0 < G ? (int)(batch - r0) : G;
    for (int i = tid; i < gv * N; i += NT)     // stage the rows' input (coalesced)
      staged(row_of(i >> r))[i & (N - 1)] = z[(r0 + (i >> r)) * N + (i & (N - 1))];
    for (int i = tid; i < 4 * NS; i += NT) slot_base[i] = 0;
    __syncthreads();
    int cur = 0;
    const auto end_step = [&]() {
      int* nx = slot_base + (cur ^ 1) * 2 * NS;   // cleared for the next step while this one stores
      for (int i = tid; i < 2 * NS; i += NT) nx[i] = 0;
      __syncthreads();
      cur ^= 1;
    };
    for (int g = tid; g < gv; g += NT) fold_base(row_of(g), staged(row_of(g)));
    fx_step<NT, K / 2, false>(
        slot_base + cur * 2 * NS, NS, gv * (N / 2),
        [&](int w, Val& v) { const Row R = row_of(w >> (r - 1)); fold_eval(R, staged(R), w & (N / 2 - 1), v); },
        [&](int w, const Val& v, int m1, int) { fold_store(row_of(w >> (r - 1)), w & (N / 2 - 1), v, m1); });
    end_step();
    for (int dep = 0; dep <= r - 3; ++dep) {   // mirror butterflies and secant products
      fx_step<NT, (K / 4 > 0 ? K / 4 : 1), true>(
          slot_base + cur * 2 * NS, NS, gv * (N / 4),
          [&](int w, Val& v) { fwd_eval(row_of(w >> (r - 2)), dep, w & (N / 4 - 1), v); },
          [&](int w, const Val& v, int m1, int m2) { fwd_store(row_of(w >> (r - 2)), dep, w & (N / 4 - 1), v, m1, m2); });
      end_step();
    }
    for (int h = 1; h <= r - 1; ++h) {         // node outputs (two cells an item) and the class chain
      fx_step<NT, K / 2, false>(
          slot_base + cur * 2 * NS, NS, gv * (N / 2),
          [&](int w, Val& v) { bwd_eval(row_of(w >> (r - 1)), h, w & (N / 2 - 1), v); },
          [&](int w, const Val& v, int m1, int) { bwd_store(row_of(w >> (r - 1)), h, w & (N / 2 - 1), v, m1); });
      end_step();
    }
    fx_step<NT, K / 2, false>(                   // CDFT combine, one block per row
        slot_base + cur * 2 * NS, NS, gv * (N / 2),
        [&](int w, Val& v) { fin_eval(row_of(w >> (r - 1)), w & (N / 2 - 1), v); },
        [&](int w, const Val& v, int m1, int) {
          const int g = w >> (r - 1);
          fin_store(row_of(g), w & (N / 2 - 1), v, m1, out + (r0 + g) * N, eout + r0 + g);
        });
    end_step();   // the next pass restages the rows
  }
}

struct FxCfg {
  int nt, k, lgG;
};
// threads, items per thread and rows per CTA pass for rows of length 2^r:
// 256 threads and up to 1024 items (at most 48 KB of rows) per CTA up to 2^10,
// then one row per CTA (1024 threads from 2^12; 192 KB of shared memory at 2^14)
inline FxCfg fx_cfg(int r) {
  if (r <= 1) return {256, 4, 0};
  if (r == 11) return {512, 4, 0};
  if (r == 12) return {1024, 4, 0};
  if (r == 13) return {1024, 8, 0};
  if (r == 14) return {1024, 16, 0};
  const int N = 1 << r;
  int G = 1024 >> r;
  while (G > 1 && (size_t)G * row_bytes(N) > 49152) G >>= 1;
  int lg = 0;
  while ((1 << lg) < G) ++lg;
  return {256, G * N / 256, lg};
}

template <int NT, int K>
cudaError_t launch_k(const qft_plan p, const FxCfg& c, const uint32_t* z, Cell* out, int* eout, cudaStream_t st) {
  const int N = (int)p->n, G = 1 << c.lgG;
  const size_t smem = N == 2 ? 0 : G * row_bytes(N) + sizeof(int) * 4 * (size_t)slot_count(G * N);
  cudaError_t e = cudaFuncSetAttribute(k_fixed<NT, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fixed<NT, K>, NT, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int64_t per_cta = N == 2 ? NT : G;
  int64_t grid = (int64_t)per_sm * p->sms;
  const int64_t need = (p->batch + per_cta - 1) / per_cta;
  if (grid > need) grid = need;
  k_fixed<NT, K><<<(unsigned)grid, NT, smem, st>>>(z, out, eout, reinterpret_cast<const Sec*>(p->d_fx), p->r,
                                                  p->batch, c.lgG);
  return cudaGetLastError();
}

}  // namespace

int qft_fixed_prepare(qft_plan p) {
  const int N = (int)p->n;
  const int ne = N >= 8 ? N / 4 - 1 : 1;
  Sec* h = (Sec*)calloc((size_t)ne, sizeof(Sec));
  if (!h) return QFT_ERR_CUDA;
  fill_consts(N, h);
  cudaError_t e = cudaMalloc(&p->d_fx, sizeof(Sec) * (size_t)ne);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_fx, h, sizeof(Sec) * (size_t)ne, cudaMemcpyHostToDevice);
  free(h);
  if (e != cudaSuccess) return qft_set_cuda(p, e);
  const FxCfg c = fx_cfg(p->r);
  p->threads = c.nt;
  p->smem = N == 2 ? 0 : (size_t)(1 << c.lgG) * row_bytes(N) + sizeof(int) * 4 * (size_t)slot_count((1 << c.lgG) * N);
  return QFT_OK;
}

int qft_launch_fixed(qft_plan p, const void* in, void* out, int32_t* exps, cudaStream_t st) {
  const uint32_t* z = static_cast<const uint32_t*>(in);
  Cell* o = static_cast<Cell*>(out);
  int* eo = reinterpret_cast<int*>(exps);
  const FxCfg c = fx_cfg(p->r);
  cudaError_t (*launch)(const qft_plan, const FxCfg&, const uint32_t*, Cell*, int*, cudaStream_t) = nullptr;
  if (c.nt == 256 && c.k == 2) launch = launch_k<256, 2>;
  else if (c.nt == 256 && c.k == 4) launch = launch_k<256, 4>;
  else if (c.nt == 512 && c.k == 4) launch = launch_k<512, 4>;
  else if (c.nt == 1024 && c.k == 4) launch = launch_k<1024, 4>;
  else if (c.nt == 1024 && c.k == 8) launch = launch_k<1024, 8>;
  else if (c.nt == 1024 && c.k == 16) launch = launch_k<1024, 16>;
  if (!launch) return QFT_ERR_INVALID_N;
  qft_time_begin(p, st, QFT_KERNEL_ROWS);
  const cudaError_t e = launch(p, c, z, o, eo, st);
  qft_time_end(p, st);
  return qft_set_cuda(p, e);
}
