// qft_static.cu -- qft_execute_static_scratch: the large-row C2C FP32 launch
// sequence (qft_large.cuh) run on storage that is part of the library image
// instead of storage a plan allocates.
//
// Who needs it: a caller that cannot allocate device memory where it wants a
// transform.  A regular plan reserves its scratch copies (up to 8 GiB) and its
// tables with cudaMalloc when it is created; that fails when another allocator
// already holds the device's free memory, and cudaMalloc / cudaFree may
// synchronise the whole device, which a latency-bound loop cannot afford.  This
// entry point takes no plan and never calls cudaMalloc, cudaFree or any other
// routine that allocates, neither here nor through torch.
//
// Storage (file-scope device arrays, reserved when the module loads):
//   g_static_scratch  64 MiB: scratch copies A and B, the FINAL tasks' C/S
//                     tables and, for n >= 2^16, the lo parts of both copies
//                     (the compensated classes, as a plan of that length
//                     evaluates them), for as many rows as fit (2 or 4 copies
//                     x 2 sides x side_len cells plus N/8 + 4 table cells, 8
//                     bytes each, per row); rows beyond that are done in
//                     successive chunks.
//   g_static_sec      Gray-ordered FP32 secants of Sec. 6.1 for N = 2^20; the
//                     table for a shorter N is its prefix of N/4 entries.
//   g_static_plans    the launch schedules for N = 2^15 ... 2^20.
//   g_static_status   the device status word of the NODE kernel's bounded
//                     waits (QFT_OK or QFT_ERR_TIMEOUT), read and cleared by
//                     qft_static_scratch_sync_status.
// Every call shares these arrays.  No scratch cell has to start at zero: each
// call writes every scratch cell it reads before reading it, so nothing is
// cleared.  The status word starts at zero when the module loads and is
// cleared by every status read.  Two calls whose executions overlap (different
// streams, or different host threads without ordering) race on the scratch and
// give wrong results.
//
// Set-up: the first call on a device looks up the arrays' device addresses
// with cudaGetSymbolAddress (checked) and fills the secant table and the
// schedules with blocking cudaMemcpyToSymbol copies; make that first call
// before any stream capture begins.  Later calls only launch kernels.  The
// set-up is not repeated after cudaDeviceReset (which discards the arrays'
// contents): do not use the entry point across a device reset.
#include <string.h>

#include <mutex>

#include "qft_consts.h"
#include "qft_large.cuh"

namespace {

constexpr int kStaticMinLog2 = qft_lib::kMaxRowLog2 + 1;   // 2^15: the first large-row length
constexpr int kStaticMaxLog2 = 20;
constexpr int kStaticPlans = kStaticMaxLog2 - kStaticMinLog2 + 1;
constexpr size_t kStaticScratchBytes = (size_t)64 << 20;
constexpr size_t kStaticSecEntries = ((size_t)1 << kStaticMaxLog2) / 4 + 1;
constexpr int kStaticMaxDevices = 64;

static __device__ __align__(256) qc_storage g_static_scratch[kStaticScratchBytes / sizeof(qc_storage)];
static __device__ __align__(256) float g_static_sec[kStaticSecEntries];
static __device__ __align__(256) QftLargePlan g_static_plans[kStaticPlans];
static __device__ __align__(256) int g_static_status;

// host copies (device independent), built once
static float g_host_sec[kStaticSecEntries];
static QftLargePlan g_host_plans[kStaticPlans];
static QftTune g_host_tunes[kStaticPlans];
static bool g_host_ready = false;

struct StaticDev {
  bool ready;
  qc_storage* scratch;
  float* sec;
  QftLargePlan* plans;
  int* status;
};
static StaticDev g_dev[kStaticMaxDevices];
static std::mutex g_static_mu;

static int host_setup() {
  if (g_host_ready) return QFT_OK;
  qft_fill_gray_secants(kStaticMaxLog2, g_host_sec);
  g_host_sec[kStaticSecEntries - 1] = 0.f;
  for (int i = 0; i < kStaticPlans; ++i) {
    const int r = kStaticMinLog2 + i;
    QftTune t = qft_default_tune(r);
    t.L1 = qft_lib::kL1;
    t.LB = qft_lib::kLB;
    g_host_tunes[i] = t;
    // the same precision as a plan of this length (compensated largest classes)
    if (qft_build_large_plan(r, t, qft_lib::kNodeLog2, qft_lib::kNodeThreads, &g_host_plans[i],
                             qft_comp_classes(r)) != 0)
      return QFT_ERR_INVALID_N;
  }
  g_host_ready = true;
  return QFT_OK;
}

static int device_setup(int dev, StaticDev* out) {
  StaticDev& d = g_dev[dev];
  if (!d.ready) {
    int rc = host_setup();
    if (rc != QFT_OK) return rc;
    if (cudaGetSymbolAddress((void**)&d.scratch, g_static_scratch) != cudaSuccess) return QFT_ERR_CUDA;
    if (cudaGetSymbolAddress((void**)&d.sec, g_static_sec) != cudaSuccess) return QFT_ERR_CUDA;
    if (cudaGetSymbolAddress((void**)&d.plans, g_static_plans) != cudaSuccess) return QFT_ERR_CUDA;
    if (cudaGetSymbolAddress((void**)&d.status, g_static_status) != cudaSuccess) return QFT_ERR_CUDA;
    if (cudaMemcpyToSymbol(g_static_sec, g_host_sec, sizeof(g_host_sec)) != cudaSuccess) return QFT_ERR_CUDA;
    if (cudaMemcpyToSymbol(g_static_plans, g_host_plans, sizeof(g_host_plans)) != cudaSuccess) return QFT_ERR_CUDA;
    d.ready = true;
  }
  *out = d;
  return QFT_OK;
}

}  // namespace

extern "C" int qft_execute_static_scratch(int64_t n, int64_t batch, int op, const void* in, void* out,
                                          void* stream) {
  if (n < ((int64_t)1 << kStaticMinLog2) || n > ((int64_t)1 << kStaticMaxLog2) || (n & (n - 1)) != 0)
    return QFT_ERR_INVALID_N;
  if (batch < 0) return QFT_ERR_INVALID_BATCH;
  if (op < QFT_OP_FORWARD || op > QFT_OP_INVERSE_ADJOINT) return QFT_ERR_INVALID_ARG;
  if (batch == 0) return QFT_OK;
  if (!in || !out) return QFT_ERR_NULLPTR;
  if (((uintptr_t)in % 8) || ((uintptr_t)out % 8)) return QFT_ERR_ALIGN;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return QFT_ERR_CUDA;
  if (dev < 0 || dev >= kStaticMaxDevices) return QFT_ERR_INVALID_ARG;
  StaticDev d;
  {
    std::lock_guard<std::mutex> g(g_static_mu);
    const int rc = device_setup(dev, &d);
    if (rc != QFT_OK) return rc;
  }
  int r = 0;
  while (((int64_t)1 << r) < n) ++r;
  const int idx = r - kStaticMinLog2;

  // A plan descriptor on the stack that points at the static storage; the
  // launch sequence reads only the fields set here.
  qft_plan_s p;
  memset(&p, 0, sizeof(p));
  p.kind = QFT_KIND_C2C;
  p.dtype = QFT_DTYPE_F32;
  p.n = n;
  p.batch = batch;
  p.r = r;
  p.tune = g_host_tunes[idx];
  p.d_sec = d.sec;
  p.device = dev;
  p.large_host = &g_host_plans[idx];
  p.d_large = d.plans + idx;
  p.scratch = d.scratch;
  p.d_status = d.status;
  p.side_len = qft_side_len((int)n);
  p.comp_j = g_host_plans[idx].comp_classes;
  // two scratch copies (four with the lo parts of a compensated length) and the tables
  const int64_t per_row = (p.comp_j > 0 ? 4 : 2) * 2 * (int64_t)p.side_len * (int64_t)sizeof(qc_storage) +
                          (int64_t)qft_lib::large_tab_cells((int)n, qft_lib::kLargeMinLF) * (int64_t)sizeof(qc_storage);
  int64_t rows = (int64_t)kStaticScratchBytes / per_row;
  if (rows > batch) rows = batch;
  if (rows > 65535) rows = 65535;
  p.scratch_rows = rows;
  // the FINAL tasks read per-row C/S tables when a chunk holds enough rows (the
  // same rule as a plan's); either way the result is the same bits
  p.large_tab = rows >= 64 ? 1 : 0;
  return exec_c2c<StC64>(&p, op, in, out, static_cast<cudaStream_t>(stream));
}

extern "C" int qft_static_scratch_sync_status(void* stream) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return QFT_ERR_CUDA;
  if (dev < 0 || dev >= kStaticMaxDevices) return QFT_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> g(g_static_mu);
    if (!g_dev[dev].ready) return QFT_OK;   // no call has run on this device
  }
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return QFT_ERR_CUDA;
  int st = 0;
  const int zero = 0;
  if (cudaMemcpyFromSymbol(&st, g_static_status, sizeof(int)) != cudaSuccess) return QFT_ERR_CUDA;
  if (cudaMemcpyToSymbol(g_static_status, &zero, sizeof(int)) != cudaSuccess) return QFT_ERR_CUDA;
  return st;
}
