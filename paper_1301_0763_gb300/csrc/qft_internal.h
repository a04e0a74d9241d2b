// qft_internal.h -- definitions shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "qft_plan.h"
#include "qft_planner.h"
#include "../../include/qft_gb300.h"

// Execute-time arguments of a ragged plan, read by its kernels from device
// memory so that the captured CUDA graph stays valid across executes.
struct QftIoArgs {
  const void* in;
  void* out;
  int in_op, out_op;
  float scale;
  int scaled;
};

struct qft_plan_s;
struct QftRaggedClass {
  int r;                 // log2 N of the rows of this class
  int64_t count;         // rows
  int32_t* d_rows;       // row indices (device)
  qft_plan_s* sub;       // plan of `count` rows of length 2^r (not registered)
};

// complex cell storage of the scratch copies (layout of qft::qc)
struct __align__(8) qc_storage { float x, y; };

namespace qft_lib {
constexpr int kMaxRowLog2 = 14;   // largest row one CTA transforms in shared memory
constexpr int kMaxLog2 = 24;      // largest transform length
constexpr int kFixedMaxLog2 = 14; // largest row of the fixed-point variant (one CTA, shared memory)
constexpr int kNodeLog2 = 12;     // largest node group of the large-row path (cells)
constexpr int kNodeThreads = 512;
constexpr int64_t kScratchBudget = (int64_t)16 << 30;  // bytes of scratch per plan
constexpr int kL1 = 3;            // mirror levels per F1 task (register tile 2^kL1 per side)
constexpr int kLB = 3;            // backward levels per SLICE task (QFT_MAX_LB)

// Shared-memory layout of the row engine: plan | secant table | DCT side | DST side.
__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }
__host__ __device__ inline size_t side_bytes(int N) { return align16(8 * (size_t)((N / 2) + ((N / 2) >> 4) + 1)); }
__host__ __device__ inline size_t off_sec() { return align16(sizeof(QftRowPlan)); }
__host__ __device__ inline size_t off_side0(int N) { return off_sec() + align16(sizeof(float) * (size_t)(N / 4 + 1)); }
__host__ __device__ inline size_t off_tab(int N) { return off_side0(N) + 2 * side_bytes(N); }
__host__ __device__ inline size_t tab_cells(int N, int LF) { return (size_t)(N >> LF) + 2; }
__host__ __device__ inline size_t row_smem_bytes(int N, int LF) { return off_tab(N) + align16(8 * tab_cells(N, LF)); }
// large-row path: cells per row of the C/S tables in scratch (Mt = N / 2^LF), even;
// the scratch is sized for LF >= kLargeMinLF
constexpr int kLargeMinLF = 3;
__host__ __device__ inline int large_tab_cells(int N, int LF) { return ((N >> LF) + 2 + 1) & ~1; }
}

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
  int threads;
  int no_stage;               // 1: never stage input rows in shared memory
  int node_log2, node_nt;     // large-row path: largest node group (log2 cells), NODE kernel threads
  int* d_status;              // device status word (QFT_OK or QFT_ERR_TIMEOUT)
  int64_t wait_ns;            // limit of the kernels' waits for staged copies (ns; 0: 2 s)
  int withhold_copy;          // one-shot test: the next execute withholds each CTA's first staged copy
  int64_t channels;           // spectral-filter plans: C (batch holds B)
  void* d_fx;                 // fixed-point plans (QFT_DTYPE_I16): the secant constants (qfx::Sec)
  // large-row path (N > 2^kMaxRowLog2): schedule, scratch copies A and B
  QftLargePlan* large_host;
  QftLargePlan* d_large;
  qc_storage* scratch;
  int64_t scratch_rows;       // rows the scratch copies hold
  int64_t scratch_bytes;      // bytes of `scratch`
  int64_t chunk_rows;         // rows per launch sequence (0: scratch_rows); fewer keep a chunk's copies in L2
  int large_tab;              // 1: TAB launch + FINAL from C/S tables; 0: FINAL walks the class recursion
  int comp_j;                 // classes (per side) whose trees run on compensated pairs (large rows only)
  int inplace;                // large rows: one scratch copy, in-place SLICE levels (QFT_PLAN_IN_PLACE)
  int side_len;
  // ragged plans (qft_plan_create_ragged)
  int nclasses;
  QftRaggedClass* classes;
  int64_t* d_offsets;
  QftIoArgs* d_args;
  QftIoArgs* h_args;          // pinned host staging of the arguments
  cudaGraph_t graph;
  cudaGraphExec_t gexec;
  int graph_kernels;
  size_t smem;
  int device;
  int sms;
  cudaError_t last_cuda;
  cudaStream_t last_stream;
  // launch timing (qft_plan_time_launches): an event pair around each launch
  int timing;
  int tev_n, tev_cap;
  cudaEvent_t* tev;           // 2 per recorded launch
  int* tev_kind;              // QFT_KERNEL_* of each recorded launch
};

// Kernel kinds reported by qft_plan_launch_times.
enum { QFT_KERNEL_ROWS = 0, QFT_KERNEL_GLOBAL = 1, QFT_KERNEL_NODE = 2, QFT_KERNEL_SLICE = 3, QFT_KERNEL_KINDS = 4 };

// Records the start event of a launch of kind `kind` on `st` when timing is on.
static inline void qft_time_begin(qft_plan p, cudaStream_t st, int kind) {
  if (!p->timing) return;
  if (p->tev_n == p->tev_cap) {
    const int cap = p->tev_cap ? 2 * p->tev_cap : 64;
    cudaEvent_t* ev = (cudaEvent_t*)realloc(p->tev, sizeof(cudaEvent_t) * 2 * (size_t)cap);
    if (!ev) return;
    p->tev = ev;
    int* k = (int*)realloc(p->tev_kind, sizeof(int) * (size_t)cap);
    if (!k) return;
    p->tev_kind = k;
    for (int i = 2 * p->tev_cap; i < 2 * cap; ++i) p->tev[i] = nullptr;
    p->tev_cap = cap;
  }
  cudaEvent_t* pair = p->tev + 2 * p->tev_n;
  if (!pair[0] && cudaEventCreate(&pair[0]) != cudaSuccess) return;
  if (!pair[1] && cudaEventCreate(&pair[1]) != cudaSuccess) return;
  p->tev_kind[p->tev_n] = kind;
  cudaEventRecord(pair[0], st);
}

// Records the end event of the launch started by qft_time_begin.
static inline void qft_time_end(qft_plan p, cudaStream_t st) {
  if (!p->timing || p->tev_n >= p->tev_cap || !p->tev[2 * p->tev_n + 1]) return;
  cudaEventRecord(p->tev[2 * p->tev_n + 1], st);
  p->tev_n++;
}


static inline int qft_set_cuda(qft_plan p, cudaError_t e) {
  if (e == cudaSuccess) return QFT_OK;
  if (p) p->last_cuda = e;
  return QFT_ERR_CUDA;
}

// Launchers, one translation unit each (compiled in parallel).
int qft_launch_c2c_f32(qft_plan p, int op, const void* in, void* out, cudaStream_t st);
int qft_launch_c2c_f16(qft_plan p, int op, const void* in, void* out, cudaStream_t st);
int qft_launch_c2c_bf16(qft_plan p, int op, const void* in, void* out, cudaStream_t st);
int qft_launch_real(qft_plan p, int op, const void* in, void* out, cudaStream_t st);
int qft_launch_r2r(qft_plan p, const void* in, void* out, cudaStream_t st);
int qft_launch_filter(qft_plan p, int backward, const float* x, const void* W, const float* gy, float* out,
                      void* gW, cudaStream_t st);
int qft_filter_smem(int N, int LF, int backward);
int qft_filter_parts();
int qft_fixed_prepare(qft_plan p);
int qft_launch_fixed(qft_plan p, const void* in, void* out, int32_t* exps, cudaStream_t st);
int qft_launch_ragged_class(qft_plan sub, const QftIoArgs* d_args, const int64_t* d_offsets,
                            const int32_t* d_rows, cudaStream_t st);
