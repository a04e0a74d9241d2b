// qft_k_fixed.cu -- the fixed-point variant's kernel (qft_fixed.cuh) and its
// launcher.
//
// One CTA transforms one row at a time in shared memory (persistent grid over
// the rows).  A row is a sequence of steps -- fold, the forward depths of the
// class trees, the backward heights (tree nodes and the class chain), the
// CDFT combine -- and every step has two phases separated by a CTA barrier:
// each thread computes its items (register values and block keys) and takes
// the block maxima (butterfly shuffles within a warp for blocks of fewer than
// 32 items, which are aligned runs of lanes; one shared-memory atomicMax per
// warp for larger blocks), then, after the barrier, shifts and stores.
#include "qft_internal.h"
#include "qft_fixed.cuh"

static_assert(qfx::kMaxLog2 == qft_lib::kFixedMaxLog2, "fixed-point row limit");

namespace {
using namespace qfx;

// Maximum of `k` over the aligned block of `seg` consecutive items holding
// item w (seg a power of two; 0 for a lane without work).  Blocks of 32 items
// or more also fold their warp's maximum into slot[first item / 32].
__device__ __forceinline__ int block_max(int k, int seg, int* slot, int w) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_xor_sync(0xffffffffu, k, o);
    if (o < seg) k = max(k, t);
  }
  if (seg >= 32 && (threadIdx.x & 31) == 0) atomicMax(slot + ((w & ~(seg - 1)) >> 5), k);
  return k;
}
__device__ __forceinline__ int block_get(int k, int seg, const int* slot, int w) {
  return seg >= 32 ? slot[(w & ~(seg - 1)) >> 5] : k;
}

// NT threads, K items per thread per step (K * NT >= N).
template <int NT, int K>
__global__ void __launch_bounds__(NT) k_fixed(const uint32_t* __restrict__ z, Cell* __restrict__ out,
                                              int* __restrict__ eout, const Sec* __restrict__ sec, int r,
                                              int64_t batch) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int N = 1 << r, H = N / 2, NS = slot_count(N);
  Row R;
  R.V0 = reinterpret_cast<Cell*>(sm);
  R.V1 = R.V0 + (H + 2);
  R.X0 = reinterpret_cast<int16_t*>(R.V1 + (H + 2));
  R.X1 = R.X0 + N;
  int* slots = reinterpret_cast<int*>(R.X1 + N);   // [2 alternates][2 keys][NS]
  R.ch = slots + 4 * NS;
  R.sec = sec;
  R.r = r;
  R.N = N;
  const int tid = threadIdx.x;
  for (int64_t row = blockIdx.x; row < batch; row += gridDim.x) {
    const uint32_t* zr = z + row * N;
    Cell* orow = out + row * N;
    if (N == 2) {
      if (tid == 0) row_n2(zr, orow, eout + row);
      continue;
    }
    for (int i = tid; i < 4 * NS; i += NT) slots[i] = 0;
    __syncthreads();
    int cur = 0;
    // the slots of the next step are cleared while this step stores
    const auto clear_next = [&]() {
      int* nx = slots + (cur ^ 1) * 2 * NS;
      for (int i = tid; i < 2 * NS; i += NT) nx[i] = 0;
    };
    {  // fold (Sec. 4.2 on complex data) and the class blocks
      Item it[K];
      if (tid == 0) fold_base(R, zr);
#pragma unroll
      for (int kk = 0; kk < K; ++kk) {
        const int w = tid + kk * NT;
        if (w < N) fold_compute(R, zr, w, it[kk]);
        else item_none(it[kk]);
        it[kk].k1 = block_max(it[kk].k1, it[kk].seg, slots + cur * 2 * NS, w);
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < K; ++kk) {
        const int w = tid + kk * NT;
        if (it[kk].seg) fold_write(R, w, it[kk], block_get(it[kk].k1, it[kk].seg, slots + cur * 2 * NS, w));
      }
      clear_next();
      __syncthreads();
      cur ^= 1;
    }
    for (int dep = 0; dep <= r - 3; ++dep) {   // mirror butterflies and secant products
      Item it[K / 2 > 0 ? K / 2 : 1];
#pragma unroll
      for (int kk = 0; kk < (K / 2 > 0 ? K / 2 : 1); ++kk) {
        const int w = tid + kk * NT;
        if (w < H) fwd_compute(R, dep, w, it[kk]);
        else item_none(it[kk]);
        it[kk].k1 = block_max(it[kk].k1, it[kk].seg, slots + cur * 2 * NS, w);
        it[kk].k2 = block_max(it[kk].k2, it[kk].seg, slots + cur * 2 * NS + NS, w);
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < (K / 2 > 0 ? K / 2 : 1); ++kk) {
        const int w = tid + kk * NT;
        if (it[kk].seg)
          fwd_write(R, dep, w, it[kk], block_get(it[kk].k1, it[kk].seg, slots + cur * 2 * NS, w),
                    block_get(it[kk].k2, it[kk].seg, slots + cur * 2 * NS + NS, w));
      }
      clear_next();
      __syncthreads();
      cur ^= 1;
    }
    for (int h = 1; h <= r - 1; ++h) {         // node outputs and the class chain
      Item it[K];
#pragma unroll
      for (int kk = 0; kk < K; ++kk) {
        const int w = tid + kk * NT;
        if (w < N) bwd_compute(R, h, w, it[kk]);
        else item_none(it[kk]);
        it[kk].k1 = block_max(it[kk].k1, it[kk].seg, slots + cur * 2 * NS, w);
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < K; ++kk) {
        const int w = tid + kk * NT;
        if (it[kk].seg) bwd_write(R, h, w, it[kk], block_get(it[kk].k1, it[kk].seg, slots + cur * 2 * NS, w));
      }
      clear_next();
      __syncthreads();
      cur ^= 1;
    }
    {  // CDFT combine, one block: the row exponent
      int kf[K / 2 > 0 ? K / 2 : 1], sg[K / 2 > 0 ? K / 2 : 1];
#pragma unroll
      for (int kk = 0; kk < (K / 2 > 0 ? K / 2 : 1); ++kk) {
        const int w = tid + kk * NT;
        Item it;
        if (w < H) fin_compute(R, w, it);
        else item_none(it);
        kf[kk] = block_max(it.k1, it.seg, slots + cur * 2 * NS, w);
        sg[kk] = it.seg;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < (K / 2 > 0 ? K / 2 : 1); ++kk) {
        const int w = tid + kk * NT;
        if (sg[kk]) fin_write(R, w, block_get(kf[kk], sg[kk], slots + cur * 2 * NS, w), orow, eout + row);
      }
      __syncthreads();   // the next row reuses the shared memory
    }
  }
}

struct FxCfg {
  int nt, k;
};
// threads and items per thread of a row of length 2^r
inline FxCfg fx_cfg(int r) {
  const int N = 1 << r;
  if (N <= 128) return {32, 4};
  if (N <= 2048) return {N / 4, 4};
  return {N / 8, 8};
}

template <int NT, int K>
cudaError_t launch_k(const qft_plan p, const uint32_t* z, Cell* out, int* eout, cudaStream_t st) {
  const size_t smem = smem_bytes((int)p->n);
  cudaError_t e = cudaFuncSetAttribute(k_fixed<NT, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fixed<NT, K>, NT, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int64_t grid = (int64_t)per_sm * p->sms;
  if (grid > p->batch) grid = p->batch;
  k_fixed<NT, K><<<(unsigned)grid, NT, smem, st>>>(z, out, eout, reinterpret_cast<const Sec*>(p->d_fx), p->r,
                                                  p->batch);
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
  p->smem = smem_bytes(N);
  return QFT_OK;
}

int qft_launch_fixed(qft_plan p, const void* in, void* out, int32_t* exps, cudaStream_t st) {
  const uint32_t* z = static_cast<const uint32_t*>(in);
  Cell* o = static_cast<Cell*>(out);
  int* eo = reinterpret_cast<int*>(exps);
  cudaError_t e;
  qft_time_begin(p, st, QFT_KERNEL_ROWS);
  switch (p->r) {
  case 1: case 2: case 3: case 4: case 5: case 6: case 7: e = launch_k<32, 4>(p, z, o, eo, st); break;
  case 8: e = launch_k<64, 4>(p, z, o, eo, st); break;
  case 9: e = launch_k<128, 4>(p, z, o, eo, st); break;
  case 10: e = launch_k<256, 4>(p, z, o, eo, st); break;
  case 11: e = launch_k<512, 4>(p, z, o, eo, st); break;
  case 12: e = launch_k<512, 8>(p, z, o, eo, st); break;
  case 13: e = launch_k<1024, 8>(p, z, o, eo, st); break;
  default: return QFT_ERR_INVALID_N;
  }
  qft_time_end(p, st);
  return qft_set_cuda(p, e);
}
