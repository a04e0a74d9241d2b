// qft_lib.cu -- sm_103a kernels of the improved-QFT row engine and the C ABI
// declared in include/qft_gb300.h.
//
// One CTA transforms one row (C2C) or one pair of real rows (R2C / C2R) at a
// time, entirely in shared memory, and loops over rows (persistent grid).
// The phases of a row are listed in a QftRowPlan built on the host at plan
// creation (qft_planner.h) and copied to shared memory by every CTA.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <new>

#include "qft_consts.h"
#include "qft_io.cuh"
#include "qft_planner.h"
#include "../../include/qft_gb300.h"

using namespace qft;

namespace {

constexpr int kThreads = 256;
constexpr int kMaxRowLog2 = 14;   // largest row that fits one CTA's shared memory

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
};

// ------------------------------------------------------------ row kernel
__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline size_t row_smem_bytes(int N) {
  return align16(sizeof(QftRowPlan)) + align16(sizeof(float) * (size_t)(N / 4 + 1)) +
         2 * align16(sizeof(qc) * (size_t)qft_side_len(N));
}

template <class FAC, int L1>
__global__ void __launch_bounds__(kThreads)
k_rows(const QftRowPlan* __restrict__ gplan, const float* __restrict__ gsec, int sec_stride,
       int64_t nitems, FAC fac) {
  extern __shared__ __align__(16) unsigned char smem[];
  QftRowPlan& P = *reinterpret_cast<QftRowPlan*>(smem);
  {
    const int* src = reinterpret_cast<const int*>(gplan);
    int* dst = reinterpret_cast<int*>(smem);
    for (int i = threadIdx.x; i < (int)(sizeof(QftRowPlan) / 4); i += kThreads) dst[i] = src[i];
  }
  __syncthreads();
  const int r = P.r;
  const int N = 1 << r;
  float* sec = reinterpret_cast<float*>(smem + align16(sizeof(QftRowPlan)));
  qc* side0 = reinterpret_cast<qc*>(smem + align16(sizeof(QftRowPlan)) + align16(sizeof(float) * (N / 4 + 1)));
  qc* side1 = side0 + align16(sizeof(qc) * qft_side_len(N)) / sizeof(qc);
  for (int m = threadIdx.x; m <= N / 4; m += kThreads) sec[m] = gsec[(int64_t)m * sec_stride];
  __syncthreads();
  Eng e;
  e.side0 = side0; e.side1 = side1; e.sec = sec; e.r = r; e.N = N;
  const int tid = threadIdx.x;
  for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
    const auto io = fac.make(item);
    for (int p = 0; p < P.nphase; ++p) {
      const int nt = P.phase_ntasks[p];
      if (!P.phase_is_slice[p]) {
        for (int tau = tid; tau < nt; tau += kThreads) {
          const QftSeg& sg = find_seg(P, p, tau);
          run_plain_task<L1>(P, sg, e, io, tau - sg.begin);
        }
        __syncthreads();
      } else {
        for (int rb = 0; rb < nt; rb += kThreads) {
          const int tau = rb + tid;
          SliceRegs s;
          int segi = -1;
          if (tau < nt) {
            const QftSeg& sg = find_seg(P, p, tau);
            segi = (int)(&sg - P.segs);
            run_slice_read(sg, e, tau - sg.begin, s);
          }
          __syncthreads();
          if (segi >= 0) run_slice_write(P.segs[segi], e, s);
          __syncthreads();
        }
      }
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

// ================================================================ plans
struct qft_plan_s {
  uint32_t magic;
  int kind, dtype;
  int64_t n, batch;
  int r;
  QftTune tune;
  QftRowPlan host_plan;
  QftRowPlan* d_plan;
  float* d_sec;
  int grid;
  size_t smem;
  int device;
  int sms;
  cudaError_t last_cuda;
  cudaStream_t last_stream;
};

static const uint32_t kMagic = 0x51465447u;   // "QFTG"
static const uint32_t kDead = 0xdeadbeefu;

static int set_cuda(qft_plan p, cudaError_t e) {
  if (e == cudaSuccess) return QFT_OK;
  if (p) p->last_cuda = e;
  return QFT_ERR_CUDA;
}

static int plan_check(qft_plan p) {
  if (!p) return QFT_ERR_NULLPTR;
  if (p->magic == kDead) return QFT_ERR_DESTROYED;
  if (p->magic != kMagic) return QFT_ERR_INVALID_ARG;
  return QFT_OK;
}

template <class K>
static int occupancy_grid(qft_plan p, K kernel, int64_t items) {
  int per_sm = 0;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem);
  if (e != cudaSuccess) return set_cuda(p, e);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, p->smem);
  if (e != cudaSuccess) return set_cuda(p, e);
  if (per_sm < 1) per_sm = 1;
  int64_t g = (int64_t)per_sm * p->sms;
  if (g > items) g = items;
  if (g < 1) g = 1;
  p->grid = (int)g;
  return QFT_OK;
}

extern "C" int qft_plan_create(qft_plan* out, int64_t n, int64_t batch, int kind, int dtype, unsigned flags) {
  if (!out) return QFT_ERR_NULLPTR;
  *out = nullptr;
  if (flags != 0) return QFT_ERR_INVALID_ARG;
  if (kind != QFT_KIND_C2C && kind != QFT_KIND_R2C) return QFT_ERR_DTYPE;
  if (dtype != QFT_DTYPE_F32 && dtype != QFT_DTYPE_F16 && dtype != QFT_DTYPE_BF16) return QFT_ERR_DTYPE;
  if (kind == QFT_KIND_R2C && dtype != QFT_DTYPE_F32) return QFT_ERR_DTYPE;
  if (n < 2 || (n & (n - 1)) != 0) return QFT_ERR_INVALID_N;
  if (kind == QFT_KIND_R2C && n < 4) return QFT_ERR_INVALID_N;
  int r = 0;
  while ((int64_t(1) << r) < n) ++r;
  if (r > kMaxRowLog2) return QFT_ERR_INVALID_N;
  if (batch < 0 || batch > (int64_t(1) << 40)) return QFT_ERR_INVALID_BATCH;

  qft_plan p = new (std::nothrow) qft_plan_s();
  if (!p) return QFT_ERR_CUDA;
  p->magic = kMagic; p->kind = kind; p->dtype = dtype; p->n = n; p->batch = batch; p->r = r;
  p->d_plan = nullptr; p->d_sec = nullptr; p->last_cuda = cudaSuccess; p->last_stream = nullptr;
  cudaError_t e = cudaGetDevice(&p->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device);
  if (e != cudaSuccess) { int rc = set_cuda(p, e); delete p; return rc; }
  if (r >= 2) {
    p->tune = qft_default_tune(r);
    if (qft_build_row_plan(r, p->tune, &p->host_plan) != 0 || p->host_plan.max_slice_nodes > kThreads) {
      delete p;
      return QFT_ERR_INVALID_N;
    }
    const int N = 1 << r;
    float* hsec = (float*)malloc(sizeof(float) * (N / 4 + 1));
    if (!hsec) { delete p; return QFT_ERR_CUDA; }
    qft_fill_secants(N, hsec);
    e = cudaMalloc(&p->d_sec, sizeof(float) * (N / 4 + 1));
    if (e == cudaSuccess) e = cudaMemcpy(p->d_sec, hsec, sizeof(float) * (N / 4 + 1), cudaMemcpyHostToDevice);
    free(hsec);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_plan, sizeof(QftRowPlan));
    if (e == cudaSuccess) e = cudaMemcpy(p->d_plan, &p->host_plan, sizeof(QftRowPlan), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      int rc = set_cuda(p, e);
      cudaFree(p->d_sec); cudaFree(p->d_plan); delete p;
      return rc;
    }
    p->smem = row_smem_bytes(N);
  } else {
    p->smem = 0;
  }
  *out = p;
  return QFT_OK;
}

extern "C" int qft_plan_create_ragged(qft_plan* out, const int64_t* offsets_host, const int32_t* log2n_host,
                                      int64_t count, int kind, int dtype, unsigned flags) {
  (void)offsets_host; (void)log2n_host; (void)count; (void)kind; (void)dtype; (void)flags;
  if (out) *out = nullptr;
  return QFT_ERR_INVALID_ARG;
}

extern "C" int qft_plan_destroy(qft_plan p) {
  if (!p) return QFT_OK;
  int rc = plan_check(p);
  if (rc != QFT_OK) return rc;
  cudaFree(p->d_plan);
  cudaFree(p->d_sec);
  p->magic = kDead;
  delete p;
  return QFT_OK;
}

// ------------------------------------------------------------ launchers
template <class FAC, int L1>
static int launch_rows(qft_plan p, FAC fac, int64_t items, cudaStream_t st) {
  auto kern = k_rows<FAC, L1>;
  int rc = occupancy_grid(p, kern, items);
  if (rc != QFT_OK) return rc;
  kern<<<p->grid, kThreads, p->smem, st>>>(p->d_plan, p->d_sec, 1, items, fac);
  return set_cuda(p, cudaGetLastError());
}

template <class ST>
static int exec_c2c(qft_plan p, int op, const void* in, void* out, cudaStream_t st) {
  FacC2C<ST> f;
  f.in = static_cast<const typename ST::elem*>(in);
  f.out = static_cast<typename ST::elem*>(out);
  f.N = (int)p->n;
  f.scale = 1.f; f.scaled = 0;
  switch (op) {
  case QFT_OP_FORWARD: f.in_op = QFT_LANE_ID; f.out_op = QFT_LANE_ID; break;
  case QFT_OP_INVERSE: f.in_op = QFT_LANE_SWAP; f.out_op = QFT_LANE_SWAP; f.scale = 1.f / (float)p->n; f.scaled = 1; break;
  case QFT_OP_FORWARD_ADJOINT: f.in_op = QFT_LANE_CONJ; f.out_op = QFT_LANE_CONJ; break;
  case QFT_OP_INVERSE_ADJOINT: f.in_op = QFT_LANE_ID; f.out_op = QFT_LANE_ID; f.scale = 1.f / (float)p->n; f.scaled = 1; break;
  default: return QFT_ERR_INVALID_ARG;
  }
  if (p->r == 1) {
    const int64_t blocks = (p->batch + 127) / 128;
    k_c2c_n2<ST><<<(unsigned)blocks, 128, 0, st>>>(f, p->batch);
    return set_cuda(p, cudaGetLastError());
  }
  return launch_rows<FacC2C<ST>, 4>(p, f, p->batch, st);
}

static int exec_r2c(qft_plan p, int op, const void* in, void* out, cudaStream_t st) {
  const int64_t items = (p->batch + 1) / 2;
  const int N = (int)p->n;
  if (op == QFT_OP_FORWARD || op == QFT_OP_INVERSE_ADJOINT) {
    FacR2C<StC64> f;
    f.in = static_cast<const float*>(in);
    f.out = static_cast<qc*>(out);
    f.rows = p->batch; f.N = N;
    f.wscale = op == QFT_OP_FORWARD ? 0.f : 1.f / (float)N;
    return launch_rows<FacR2C<StC64>, 4>(p, f, items, st);
  }
  if (op == QFT_OP_INVERSE || op == QFT_OP_FORWARD_ADJOINT) {
    FacC2R<StC64> f;
    f.in = static_cast<const qc*>(in);
    f.out = static_cast<float*>(out);
    f.rows = p->batch; f.N = N;
    if (op == QFT_OP_INVERSE) { f.wmid = 2.f; f.scale = 1.f / (float)N; }
    else { f.wmid = 1.f; f.scale = 1.f; }
    return launch_rows<FacC2R<StC64>, 4>(p, f, items, st);
  }
  return QFT_ERR_INVALID_ARG;
}

extern "C" int qft_execute(qft_plan p, int op, const void* in, void* out, void* stream) {
  int rc = plan_check(p);
  if (rc != QFT_OK) return rc;
  if (op < QFT_OP_FORWARD || op > QFT_OP_INVERSE_ADJOINT) return QFT_ERR_INVALID_ARG;
  if (p->batch == 0) return QFT_OK;
  if (!in || !out) return QFT_ERR_NULLPTR;
  const size_t al_c = p->dtype == QFT_DTYPE_F32 ? 8 : 4;
  if (p->kind == QFT_KIND_C2C) {
    if (((uintptr_t)in % al_c) || ((uintptr_t)out % al_c)) return QFT_ERR_ALIGN;
  } else {
    const bool real_in = (op == QFT_OP_FORWARD || op == QFT_OP_INVERSE_ADJOINT);
    if (((uintptr_t)in % (real_in ? 4 : 8)) || ((uintptr_t)out % (real_in ? 8 : 4))) return QFT_ERR_ALIGN;
    if (in == out) return QFT_ERR_INPLACE;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  p->last_stream = st;
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return set_cuda(p, e);
  if (cur != p->device) return QFT_ERR_INVALID_ARG;
  if (p->kind == QFT_KIND_R2C) return exec_r2c(p, op, in, out, st);
  switch (p->dtype) {
  case QFT_DTYPE_F32: return exec_c2c<StC64>(p, op, in, out, st);
  case QFT_DTYPE_F16: return exec_c2c<StC16>(p, op, in, out, st);
  case QFT_DTYPE_BF16: return exec_c2c<StBF16>(p, op, in, out, st);
  default: return QFT_ERR_DTYPE;
  }
}

extern "C" int qft_execute_forward(qft_plan p, const void* in, void* out, void* stream) {
  return qft_execute(p, QFT_OP_FORWARD, in, out, stream);
}
extern "C" int qft_execute_inverse(qft_plan p, const void* in, void* out, void* stream) {
  return qft_execute(p, QFT_OP_INVERSE, in, out, stream);
}
extern "C" int qft_execute_backward(qft_plan p, const void* grad_out, void* grad_in, void* stream) {
  return qft_execute(p, QFT_OP_FORWARD_ADJOINT, grad_out, grad_in, stream);
}

extern "C" int qft_plan_sync_status(qft_plan p) {
  int rc = plan_check(p);
  if (rc != QFT_OK) return rc;
  return set_cuda(p, cudaStreamSynchronize(p->last_stream));
}

extern "C" int qft_plan_last_cuda_error(qft_plan p) {
  if (plan_check(p) != QFT_OK) return 0;
  return (int)p->last_cuda;
}

extern "C" int qft_plan_info(qft_plan p, int* threads, int* ctas, int* smem_bytes, int* launches) {
  int rc = plan_check(p);
  if (rc != QFT_OK) return rc;
  if (threads) *threads = kThreads;
  if (ctas) *ctas = p->grid;
  if (smem_bytes) *smem_bytes = (int)p->smem;
  if (launches) *launches = 1;
  return QFT_OK;
}

extern "C" const char* qft_status_string(int s) {
  switch (s) {
  case QFT_OK: return "ok";
  case QFT_ERR_INVALID_N: return "invalid transform length";
  case QFT_ERR_INVALID_BATCH: return "invalid batch";
  case QFT_ERR_DTYPE: return "unsupported kind/dtype";
  case QFT_ERR_ALIGN: return "misaligned data pointer";
  case QFT_ERR_NULLPTR: return "null pointer";
  case QFT_ERR_CUDA: return "CUDA runtime error";
  case QFT_ERR_TIMEOUT: return "device-side wait timed out";
  case QFT_ERR_DESTROYED: return "plan was destroyed";
  case QFT_ERR_INVALID_ARG: return "invalid argument";
  case QFT_ERR_INPLACE: return "in-place execution not supported for this transform";
  default: return "unknown status";
  }
}
