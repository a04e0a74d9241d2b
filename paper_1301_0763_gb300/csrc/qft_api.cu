// qft_api.cu -- the C ABI declared in include/qft_gb300.h: plan creation
// (schedule, constant table), validation and dispatch to the kernels.
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
#include <mutex>
#include <unordered_set>

#include "qft_consts.h"
#include "qft_engine.cuh"
#include "qft_internal.h"

using namespace qft;
using qft_lib::kMaxRowLog2;

static const uint32_t kMagic = 0x51465447u;   // "QFTG"
static const uint32_t kDead = 0xdeadbeefu;

// Live and destroyed handles, so that a destroyed plan is reported instead of
// being dereferenced (an address reused by a later plan is live again).
static std::mutex g_plans_mu;
static std::unordered_set<const void*> g_live, g_dead;

static void register_plan(qft_plan p) {
  std::lock_guard<std::mutex> g(g_plans_mu);
  g_dead.erase(p);
  g_live.insert(p);
}

static int plan_check(qft_plan p) {
  if (!p) return QFT_ERR_NULLPTR;
  std::lock_guard<std::mutex> g(g_plans_mu);
  if (g_live.count(p)) return p->magic == kMagic ? QFT_OK : QFT_ERR_INVALID_ARG;
  return g_dead.count(p) ? QFT_ERR_DESTROYED : QFT_ERR_INVALID_ARG;
}

static void free_resources(qft_plan p) {
  cudaFree(p->d_plan);
  cudaFree(p->d_sec);
  cudaFree(p->d_large);
  cudaFree(p->scratch);
  free(p->large_host);
  p->d_plan = nullptr; p->d_sec = nullptr; p->d_large = nullptr; p->scratch = nullptr; p->large_host = nullptr;
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
  if (r > qft_lib::kMaxLog2) return QFT_ERR_INVALID_N;
  if (batch < 0 || batch > (int64_t(1) << 40)) return QFT_ERR_INVALID_BATCH;

  qft_plan p = new (std::nothrow) qft_plan_s();
  if (!p) return QFT_ERR_CUDA;
  p->magic = kMagic; p->kind = kind; p->dtype = dtype; p->n = n; p->batch = batch; p->r = r;
  p->d_plan = nullptr; p->d_sec = nullptr; p->last_cuda = cudaSuccess; p->last_stream = nullptr;
  p->large_host = nullptr; p->d_large = nullptr; p->scratch = nullptr; p->scratch_rows = 0; p->side_len = 0;
  p->grid = 0; p->threads = 0; p->smem = 0;
  cudaError_t e = cudaGetDevice(&p->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device);
  if (e != cudaSuccess) { int rc = qft_set_cuda(p, e); delete p; return rc; }
  if (r >= 2) {
    p->tune = qft_default_tune(r);
    p->tune.L1 = qft_lib::kL1;
    p->tune.LB = qft_lib::kLB;
    const int64_t N = int64_t(1) << r;
    // FP32 secant table (Sec. 6.1), Gray order of the butterflies
    const size_t nsec = (size_t)N / 4 + 1;
    float* hsec = (float*)calloc(nsec, sizeof(float));
    if (!hsec) { delete p; return QFT_ERR_CUDA; }
    qft_fill_gray_secants(r, hsec);
    e = cudaMalloc(&p->d_sec, sizeof(float) * nsec);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_sec, hsec, sizeof(float) * nsec, cudaMemcpyHostToDevice);
    free(hsec);
    if (e != cudaSuccess) { int rc = qft_set_cuda(p, e); free_resources(p); delete p; return rc; }
    if (r <= qft_lib::kMaxRowLog2) {
      p->threads = qft_default_threads(r);
      if (qft_build_row_plan(r, p->tune, &p->host_plan) != 0 || p->host_plan.max_slice_nodes > p->threads) {
        free_resources(p); delete p;
        return QFT_ERR_INVALID_N;
      }
      e = cudaMalloc(&p->d_plan, sizeof(QftRowPlan));
      if (e == cudaSuccess) e = cudaMemcpy(p->d_plan, &p->host_plan, sizeof(QftRowPlan), cudaMemcpyHostToDevice);
      p->smem = qft_lib::row_smem_bytes((int)N, p->host_plan.LF);
    } else {
      p->large_host = (QftLargePlan*)malloc(sizeof(QftLargePlan));
      if (!p->large_host ||
          qft_build_large_plan(r, p->tune, qft_lib::kNodeLog2, qft_lib::kNodeThreads, p->large_host) != 0) {
        free_resources(p); delete p;
        return QFT_ERR_INVALID_N;
      }
      e = cudaMalloc(&p->d_large, sizeof(QftLargePlan));
      if (e == cudaSuccess) e = cudaMemcpy(p->d_large, p->large_host, sizeof(QftLargePlan), cudaMemcpyHostToDevice);
      p->side_len = qft_side_len((int)N);
      const int64_t items = kind == QFT_KIND_R2C ? (batch + 1) / 2 : batch;
      const int64_t per_row = 2 * 2 * (int64_t)p->side_len * 8;
      int64_t rows = qft_lib::kScratchBudget / per_row;
      if (rows > items) rows = items;
      if (rows > 65535) rows = 65535;
      if (rows < 1) rows = 1;
      p->scratch_rows = rows;
      p->threads = 256;
      if (e == cudaSuccess && items > 0) e = cudaMalloc(&p->scratch, (size_t)(rows * per_row));
    }
    if (e != cudaSuccess) { int rc = qft_set_cuda(p, e); free_resources(p); delete p; return rc; }
  }
  register_plan(p);
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
  {
    std::lock_guard<std::mutex> g(g_plans_mu);
    g_live.erase(p);
    g_dead.insert(p);
  }
  free_resources(p);
  p->magic = kDead;
  delete p;
  return QFT_OK;
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
  if (e != cudaSuccess) return qft_set_cuda(p, e);
  if (cur != p->device) return QFT_ERR_INVALID_ARG;
  if (p->kind == QFT_KIND_R2C) return qft_launch_real(p, op, in, out, st);
  switch (p->dtype) {
  case QFT_DTYPE_F32: return qft_launch_c2c_f32(p, op, in, out, st);
  case QFT_DTYPE_F16: return qft_launch_c2c_f16(p, op, in, out, st);
  case QFT_DTYPE_BF16: return qft_launch_c2c_bf16(p, op, in, out, st);
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
  return qft_set_cuda(p, cudaStreamSynchronize(p->last_stream));
}

extern "C" int qft_plan_last_cuda_error(qft_plan p) {
  if (plan_check(p) != QFT_OK) return 0;
  return (int)p->last_cuda;
}

extern "C" int qft_plan_info(qft_plan p, int* threads, int* ctas, int* smem_bytes, int* launches) {
  int rc = plan_check(p);
  if (rc != QFT_OK) return rc;
  if (threads) *threads = p->threads;
  if (ctas) *ctas = p->grid;
  if (smem_bytes) *smem_bytes = (int)p->smem;
  if (launches) *launches = p->large_host ? p->large_host->nphase : 1;
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
