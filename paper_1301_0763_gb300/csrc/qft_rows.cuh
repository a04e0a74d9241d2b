// qft_rows.cuh -- the row-engine kernel (one CTA per row or pair of real rows,
// persistent over the batch) and its launch helpers.
#pragma once
#include "qft_internal.h"
#include "qft_io.cuh"

using namespace qft;

namespace {

// ------------------------------------------------------------ factories
template <class ST>
struct FacC2C {
  const typename ST::elem* in;
  typename ST::elem* out;
  int N;
  int in_op, out_op;
  float scale;
  int scaled;
  __device__ __forceinline__ IoC2C<ST> make(int64_t row) const {
    IoC2C<ST> io;
    io.in = in + row * (int64_t)N;
    io.out = out + row * (int64_t)N;
    io.N = N; io.in_op = in_op; io.out_op = out_op; io.scale = scale; io.scaled = scaled != 0;
    return io;
  }
  // staging of the input row in shared memory by one bulk copy
  static constexpr bool kCanStage = true;
  __device__ __forceinline__ int stage_src(int64_t row, const void** src, uint32_t* bytes) const {
    src[0] = in + row * (int64_t)N;
    bytes[0] = (uint32_t)(N * sizeof(typename ST::elem));
    return 1;
  }
  __device__ __forceinline__ IoC2C<ST> make_staged(int64_t row, const void* stage) const {
    IoC2C<ST> io = make(row);
    io.in = static_cast<const typename ST::elem*>(stage);
    return io;
  }
};

// Ragged C2C: item i is row rows[i] of a packed buffer, at complex offset
// offsets[row]; pointers and lane operations come from device memory.
template <class ST>
struct FacRaggedC2C {
  const QftIoArgs* args;
  const int64_t* offsets;
  const int32_t* rows;
  int N;
  __device__ __forceinline__ IoC2C<ST> make(int64_t item) const {
    IoC2C<ST> io;
    const int64_t off = offsets[rows[item]];
    io.in = static_cast<const typename ST::elem*>(args->in) + off;
    io.out = static_cast<typename ST::elem*>(args->out) + off;
    // scaled == 2: scale by 1/N of this row's own length (inverse-type ops)
    io.N = N; io.in_op = args->in_op; io.out_op = args->out_op;
    io.scale = args->scaled == 2 ? 1.f / (float)N : args->scale;
    io.scaled = args->scaled != 0;
    return io;
  }
  static constexpr bool kCanStage = false;
  __device__ int stage_src(int64_t, const void**, uint32_t*) const { return 0; }
  __device__ IoC2C<ST> make_staged(int64_t item, const void*) const { return make(item); }
};

template <class ST>
struct FacR2C {
  const float* in;
  typename ST::elem* out;
  int64_t rows;
  int N;
  float wscale;
  __device__ __forceinline__ IoR2C<ST> make(int64_t item) const {
    IoR2C<ST> io;
    const int64_t a = 2 * item, b = 2 * item + 1;
    const int64_t H = N / 2 + 1;
    io.ina = in + a * (int64_t)N;
    io.inb = b < rows ? in + b * (int64_t)N : nullptr;
    io.outa = out + a * H;
    io.outb = b < rows ? out + b * H : nullptr;
    io.N = N; io.wscale = wscale;
    return io;
  }
  static constexpr bool kCanStage = true;
  __device__ __forceinline__ int stage_src(int64_t item, const void** src, uint32_t* bytes) const {
    const int64_t a = 2 * item, b = 2 * item + 1;
    src[0] = in + a * (int64_t)N;
    bytes[0] = (uint32_t)(N * sizeof(float));
    if (b < rows) { src[1] = in + b * (int64_t)N; bytes[1] = bytes[0]; return 2; }
    return 1;
  }
  __device__ __forceinline__ IoR2C<ST> make_staged(int64_t item, const void* stage) const {
    IoR2C<ST> io = make(item);
    io.ina = static_cast<const float*>(stage);
    if (io.inb) io.inb = static_cast<const float*>(stage) + N;
    return io;
  }
};

template <class ST>
struct FacC2R {
  const typename ST::elem* in;
  float* out;
  int64_t rows;
  int N;
  float wmid, scale;
  __device__ __forceinline__ IoC2R<ST> make(int64_t item) const {
    IoC2R<ST> io;
    const int64_t a = 2 * item, b = 2 * item + 1;
    const int64_t H = N / 2 + 1;
    io.ina = in + a * H;
    io.inb = b < rows ? in + b * H : nullptr;
    io.outa = out + a * (int64_t)N;
    io.outb = b < rows ? out + b * (int64_t)N : nullptr;
    io.N = N; io.wmid = wmid; io.scale = scale;
    return io;
  }
  static constexpr bool kCanStage = false;
  __device__ int stage_src(int64_t, const void**, uint32_t*) const { return 0; }
  __device__ IoC2R<ST> make_staged(int64_t item, const void*) const { return make(item); }
};

// DCT-0 / DST-0 of periodization N: item i = real rows 2i and 2i+1 of
// length N/2+1 (DCT) or N/2-1 (DST).
template <bool DST>
struct FacR2R {
  const float* in;
  float* out;
  int64_t rows;
  int N;
  __device__ __forceinline__ IoR2R<DST> make(int64_t item) const {
    IoR2R<DST> io;
    const int64_t L = DST ? N / 2 - 1 : N / 2 + 1;
    const int64_t a = 2 * item, b = 2 * item + 1;
    io.ina = in + a * L;
    io.inb = b < rows ? in + b * L : nullptr;
    io.outa = out + a * L;
    io.outb = b < rows ? out + b * L : nullptr;
    io.N = N;
    return io;
  }
  static constexpr bool kCanStage = false;
  __device__ int stage_src(int64_t, const void**, uint32_t*) const { return 0; }
  __device__ IoR2R<DST> make_staged(int64_t item, const void*) const { return make(item); }
};

// ------------------------------------------------------------ row kernel
using qft_lib::off_sec;
using qft_lib::off_side0;
using qft_lib::side_bytes;

// ------------------------------------------------------ bulk-copy staging
// The input of the next row is copied into shared memory by one TMA bulk copy
// (cp.async.bulk, completion on an mbarrier) while the current row computes;
// the F1 phase then reads shared memory instead of waiting on HBM.
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint32_t mb, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint32_t mb, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mb) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(mb) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t mb, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
               "selp.u32 %0, 1, 0, p;\n}" : "=r"(ok) : "r"(mb), "r"(parity) : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s: a bulk copy never takes that long

// Limit of the wait for an item's staged copy (the plan's, 2 s by default) and
// the plan's one-shot test of that path: with `withhold` set, every CTA arms
// its first item's barrier without issuing the copy, so that wait runs out and
// the kernel reports QFT_ERR_TIMEOUT with no copy in flight.
struct QftWait {
  uint64_t ns;
  int withhold;
};

// Bulk prefetch of a global range into L2 (no shared memory, no completion to
// wait for); used for the next row when it cannot be staged in shared memory.
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

struct NoHook {
  __device__ __forceinline__ void operator()() const {}
};

// All phases of a QftRowPlan on the cells behind `e` (shared memory), by the
// NT threads of one CTA.  `g` offsets every task index by g * count (the node
// groups of the large-row path); 0 for whole rows.  Plain phases end with a
// barrier; SLICE phases run in rounds of NT tasks, all reads of a round before
// any of its writes (the plan guarantees a node's tasks never straddle rounds).
template <int L1, int NT, class IO, class HOOK = NoHook, bool COMP = false>
__device__ __forceinline__ void run_row_phases(const QftRowPlan& P, const Eng& e, const IO& io, int g,
                                               const HOOK& after_f1 = HOOK()) {
  const int tid = threadIdx.x;
  for (int p = 0; p < P.nphase; ++p) {
    const int nt = P.phase_ntasks[p];
    const int kind = P.phase_is_slice[p];
    // tasks are visited in increasing order, so the segment is found by
    // advancing from the previous one (amortised O(1) per task)
    int sgi = P.phase_seg0[p];
    const int sge = P.phase_seg0[p + 1];
    if (kind != 1) {
      // plain tasks (kind 0) and the phase's own tasks of the table phase (kind
      // 2: warps 0 and 1 build the C_Mt / S_Mt tables, the other warps run the
      // special FINAL tasks, which read no table).  One task loop: the task
      // code is inlined once per kernel.
      int t0 = tid, stride = NT;
      if (kind == 2) {
        const int warp = tid >> 5, lane = tid & 31;
        const int mt = P.r - P.LF;
        if (warp == 0) {
          for (int m = 1; m <= mt; ++m) { tab_level_c(e, m, lane, 32); __syncwarp(); }
        } else if (warp == 1) {
          for (int m = 2; m <= mt; ++m) { tab_level_s(e, m, lane, 32); __syncwarp(); }
        }
        t0 = tid < 64 ? nt : tid - 64;
        stride = NT - 64;
      }
      for (int tau = t0; tau < nt; tau += stride) {
        while (sgi + 1 < sge && P.segs[sgi + 1].begin <= tau) ++sgi;
        const QftSeg& sg = P.segs[sgi];
        run_plain_task<L1, IO, COMP>(P.LF, sg, e, io, g * sg.count + tau - sg.begin);
      }
      __syncthreads();
      if (p == P.in_last_phase) after_f1();
    } else {
      for (int rb = 0; rb < nt; rb += NT) {
        const int tau = rb + tid;
        const bool act = tau < nt;
        if constexpr (COMP) {
          // compensated segments keep the l parts as well (pad[2] of the segment)
          SliceRegsC s;
          bool cs = false;
          if (act) {
            while (sgi + 1 < sge && P.segs[sgi + 1].begin <= tau) ++sgi;
            cs = P.segs[sgi].pad[2] != 0;
            const int loc = g * P.segs[sgi].count + tau - P.segs[sgi].begin;
            if (cs) run_slice_read_c<QFT_COMP_NODE_LB>(P.segs[sgi], e, loc, s);
            else run_slice_read(P.segs[sgi], e, loc, s.p);
          }
          __syncthreads();
          if (act) {
            if (cs) run_slice_write_c<QFT_COMP_NODE_LB>(P.segs[sgi], e, s);
            else run_slice_write(P.segs[sgi], e, s.p);
          }
          __syncthreads();
        } else {
          SliceRegs s;
          if (act) {
            while (sgi + 1 < sge && P.segs[sgi + 1].begin <= tau) ++sgi;
            run_slice_read(P.segs[sgi], e, g * P.segs[sgi].count + tau - P.segs[sgi].begin, s);
          }
          __syncthreads();
          if (act) run_slice_write(P.segs[sgi], e, s);
          __syncthreads();
        }
      }
    }
  }
}

// NT threads per CTA; the register budget allows 512 threads per SM
// (2 CTAs of 256 or 1 of 512), i.e. at most 128 registers per thread.
template <class FAC, int L1, int NT>
__global__ void __launch_bounds__(NT, 512 / NT)
k_rows(const QftRowPlan* __restrict__ gplan, const float* __restrict__ gsec, int sec_stride,
       int64_t nitems, FAC fac, int stage_off, int* status, QftWait wait) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar;
  QftRowPlan& P = *reinterpret_cast<QftRowPlan*>(smem);
  {
    const int* src = reinterpret_cast<const int*>(gplan);
    int* dst = reinterpret_cast<int*>(smem);
    for (int i = threadIdx.x; i < (int)(sizeof(QftRowPlan) / 4); i += NT) dst[i] = src[i];
  }
  const bool staged = FAC::kCanStage && stage_off > 0;
  const uint32_t mb = smem_u32(&mbar);
  unsigned char* stage = smem + (staged ? stage_off : 0);
  const uint32_t stage_s = smem_u32(stage);
  const auto issue = [&](int64_t item) {          // thread 0 only
    const void* src[2];
    uint32_t bytes[2];
    const int np = fac.stage_src(item, src, bytes);
    uint32_t total = 0;
    for (int k = 0; k < np; ++k) total += bytes[k];
    mbar_expect_tx(mb, total);
    uint32_t off = 0;
    for (int k = 0; k < np; ++k) { bulk_g2s(stage_s + off, src[k], bytes[k], mb); off += bytes[k]; }
  };
  if (staged && threadIdx.x == 0) {
    mbar_init(mb, 1);
    fence_mbar_init();
  }
  __syncthreads();
  // a withheld copy is never issued: nothing is in flight when its wait runs out
  bool withheld = staged && wait.withhold != 0;
  if (staged && threadIdx.x == 0 && (int64_t)blockIdx.x < nitems && !withheld) issue(blockIdx.x);
  const int r = P.r;
  const int N = 1 << r;
  float* sec = reinterpret_cast<float*>(smem + off_sec());
  qc* side0 = reinterpret_cast<qc*>(smem + off_side0(N));
  qc* side1 = reinterpret_cast<qc*>(smem + off_side0(N) + side_bytes(N));
  for (int m = threadIdx.x; m <= N / 4; m += NT) sec[m] = gsec[(int64_t)m * sec_stride];
  __syncthreads();
  Eng e;
  e.side0 = side0; e.side1 = side1; e.sec = sec; e.r = r; e.N = N;
  e.tabC = reinterpret_cast<qc*>(smem + qft_lib::off_tab(N));
  e.tabS = e.tabC + (N >> P.LF) / 2 + 1;
  e.lo0 = nullptr;
  e.lo1 = nullptr;
  uint32_t parity = 0;
  for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
    if (staged) {
      // every thread waits for the bulk copy of this item (bounded)
      const uint64_t t0 = global_ns();
      bool ok = true;
      while (!mbar_try_wait(mb, parity)) {
        if (global_ns() - t0 > wait.ns) { ok = false; break; }
      }
      if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) {
          atomicExch(status, QFT_ERR_TIMEOUT);
          // the copy in flight writes this CTA's shared memory: give it a
          // second bounded wait (the long limit) before the CTA leaves
          const uint64_t t1 = global_ns();
          while (!withheld && !mbar_try_wait(mb, parity) && global_ns() - t1 < kWaitLimitNs) {
          }
        }
        __syncthreads();
        return;
      }
      withheld = false;
      parity ^= 1;
      const auto io = fac.make_staged(item, stage);
      const int64_t next = item + gridDim.x;
      run_row_phases<L1, NT>(P, e, io, 0, [&]() {
        // F1 has read the staged row: the buffer may take the next one
        if (threadIdx.x == 0 && next < nitems) {
          fence_proxy_async_smem();
          issue(next);
        }
      });
    } else {
      if constexpr (FAC::kCanStage) {
        // the next row of this CTA goes to L2 while this one is transformed
        const int64_t next = item + gridDim.x;
        if (threadIdx.x == 0 && next < nitems) {
          const void* src[2];
          uint32_t bytes[2];
          const int np = fac.stage_src(next, src, bytes);
          for (int k = 0; k < np; ++k)
            if (((uintptr_t)src[k] & 15) == 0 && (bytes[k] & 15) == 0) prefetch_l2(src[k], bytes[k]);
        }
      }
      const auto io = fac.make(item);
      run_row_phases<L1, NT>(P, e, io, 0);
    }
  }
}

// N = 2: the CDFT definition (Sec. 4.1), one thread per row.
template <class ST>
__global__ void k_c2c_n2(FacC2C<ST> fac, int64_t rows) {
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= rows) return;
  const auto io = fac.make(row);
  const qc a = io.ld(0), b = io.ld(1);
  io.st(0, cadd(a, b));
  io.st(1, csub(a, b));
}

}  // namespace


template <class K>
static int occupancy_grid(qft_plan p, K kernel, int nt, int64_t items) {
  int per_sm = 0;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem);
  if (e != cudaSuccess) return qft_set_cuda(p, e);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, nt, p->smem);
  if (e != cudaSuccess) return qft_set_cuda(p, e);
  if (per_sm < 1) per_sm = 1;
  int64_t g = (int64_t)per_sm * p->sms;
  if (g > items) g = items;
  if (g < 1) g = 1;
  p->grid = (int)g;
  return QFT_OK;
}

// ------------------------------------------------------------ launchers
template <class FAC, int L1, int NT>
static inline int launch_rows_nt(qft_plan p, FAC fac, int64_t items, size_t stage_bytes, bool stage_ok,
                                 cudaStream_t st) {
  auto kern = k_rows<FAC, L1, NT>;
  // stage the input rows in shared memory when the staging buffer keeps two CTAs per SM
  int stage_off = 0;
  size_t smem = p->smem;
  if (FAC::kCanStage && stage_ok && stage_bytes > 0 && !p->no_stage) {
    const size_t off = (p->smem + 127) & ~(size_t)127;
    if (NT == 256 && off + stage_bytes <= (size_t)(227 * 1024) / 2) { stage_off = (int)off; smem = off + stage_bytes; }
  }
  const size_t keep = p->smem;
  p->smem = smem;
  int rc = occupancy_grid(p, kern, NT, items);
  p->smem = keep;
  if (rc != QFT_OK) return rc;
  qft_time_begin(p, st, QFT_KERNEL_ROWS);
  QftWait w;
  w.ns = p->wait_ns > 0 ? (uint64_t)p->wait_ns : kWaitLimitNs;
  w.withhold = p->withhold_copy;
  kern<<<p->grid, NT, smem, st>>>(p->d_plan, p->d_sec, 1, items, fac, stage_off, p->d_status, w);
  qft_time_end(p, st);
  return qft_set_cuda(p, cudaGetLastError());
}

template <class FAC>
static inline int launch_rows(qft_plan p, FAC fac, int64_t items, cudaStream_t st, size_t stage_bytes = 0,
                              bool stage_ok = false) {
  if (p->threads == 512) return launch_rows_nt<FAC, qft_lib::kL1, 512>(p, fac, items, 0, false, st);
  return launch_rows_nt<FAC, qft_lib::kL1, 256>(p, fac, items, stage_bytes, stage_ok, st);
}

