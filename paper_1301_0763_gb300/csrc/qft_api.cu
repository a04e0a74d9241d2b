// qft_api.cu -- the C ABI declared in include/qft_gb300.h: plan creation
// (schedule, constant table, scratch), validation and dispatch to the kernels.
//
// Rows up to 2^14: one CTA transforms one row (C2C) or one pair of real rows
// (R2C / C2R) at a time, entirely in shared memory, and loops over rows
// (persistent grid); its phases are the QftRowPlan built at plan creation.
// Longer rows: the launch sequence of qft_large.cuh over scratch copies.
// Ragged plans: one sub-plan per row length, all captured in one CUDA graph.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <new>
#include <mutex>
#include <unordered_set>

#include "qft_consts.h"
#include "qft_io.cuh"
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

static void free_timing(qft_plan p) {
  for (int i = 0; i < 2 * p->tev_cap; ++i)
    if (p->tev[i]) cudaEventDestroy(p->tev[i]);
  free(p->tev);
  free(p->tev_kind);
  p->tev = nullptr; p->tev_kind = nullptr; p->tev_n = 0; p->tev_cap = 0; p->timing = 0;
}

static void free_resources(qft_plan p) {
  free_timing(p);
  cudaFree(p->d_status);
  p->d_status = nullptr;
  cudaFree(p->d_plan);
  cudaFree(p->d_sec);
  cudaFree(p->d_large);
  cudaFree(p->scratch);
  cudaFree(p->d_fx);
  p->d_fx = nullptr;
  free(p->large_host);
  p->d_plan = nullptr; p->d_sec = nullptr; p->d_large = nullptr; p->scratch = nullptr; p->large_host = nullptr;
  p->scratch_bytes = 0;
}

// (Re)builds the schedule of a plan of length 2^r >= 4 for the given tile
// sizes, threads per CTA (row engine) and node size / NODE threads (large-row
// path), and copies it to the device.  Returns QFT_ERR_INVALID_N if the
// planner rejects the combination; the plan's previous schedule is then kept.
static int plan_schedule(qft_plan p, QftTune t, int threads, int node_log2, int node_nt) {
  const int r = p->r;
  cudaError_t e = cudaSuccess;
  if (r <= qft_lib::kMaxRowLog2) {
    QftRowPlan hp;
    if (qft_build_row_plan(r, t, &hp, threads) != 0 || hp.max_slice_nodes > threads) return QFT_ERR_INVALID_N;
    const size_t smem = qft_lib::row_smem_bytes((int)p->n, hp.LF);
    if (smem > (size_t)227 * 1024) return QFT_ERR_INVALID_N;
    if (!p->d_plan) e = cudaMalloc(&p->d_plan, sizeof(QftRowPlan));
    if (e == cudaSuccess) e = cudaMemcpy(p->d_plan, &hp, sizeof(QftRowPlan), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return qft_set_cuda(p, e);
    p->host_plan = hp;
    p->smem = smem;
    p->threads = threads;
  } else {
    if (t.LF < qft_lib::kLargeMinLF) return QFT_ERR_INVALID_N;   // the scratch holds tables for LF >= 3
    QftLargePlan* lp = (QftLargePlan*)malloc(sizeof(QftLargePlan));
    if (!lp) return QFT_ERR_CUDA;
    if (qft_build_large_plan(r, t, node_log2, node_nt, lp, p->comp_j, p->inplace) != 0) {
      free(lp);
      return QFT_ERR_INVALID_N;
    }
    if (!p->d_large) e = cudaMalloc(&p->d_large, sizeof(QftLargePlan));
    if (e == cudaSuccess) e = cudaMemcpy(p->d_large, lp, sizeof(QftLargePlan), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { free(lp); return qft_set_cuda(p, e); }
    memcpy(p->large_host, lp, sizeof(QftLargePlan));
    free(lp);
    p->node_log2 = node_log2;
    p->node_nt = node_nt;
  }
  p->tune = t;
  return QFT_OK;
}

// Fills a freshly allocated plan for `batch` rows of length 2^r: schedule,
// constant table and scratch.  On failure everything it allocated is freed.
static int plan_init(qft_plan p, int r, int64_t batch, int kind, int dtype, int plain = 0, int inplace = 0) {
  p->magic = kMagic; p->kind = kind; p->dtype = dtype; p->n = int64_t(1) << r; p->batch = batch; p->r = r;
  p->d_plan = nullptr; p->d_sec = nullptr; p->last_cuda = cudaSuccess; p->last_stream = nullptr;
  p->large_host = nullptr; p->d_large = nullptr; p->scratch = nullptr; p->scratch_rows = 0; p->side_len = 0;
  p->scratch_bytes = 0;
  p->chunk_rows = 0;
  p->large_tab = 0;
  p->comp_j = 0;
  p->inplace = inplace && r > qft_lib::kMaxRowLog2 ? 1 : 0;
  p->grid = 0; p->threads = 0; p->smem = 0;
  p->nclasses = 0; p->classes = nullptr; p->d_offsets = nullptr; p->d_args = nullptr; p->h_args = nullptr;
  p->graph = nullptr; p->gexec = nullptr; p->graph_kernels = 0;
  p->d_status = nullptr;
  p->wait_ns = 0;
  p->withhold_copy = 0;
  p->channels = 0;
  p->d_fx = nullptr;
  p->timing = 0; p->tev_n = 0; p->tev_cap = 0; p->tev = nullptr; p->tev_kind = nullptr;
  cudaError_t e = cudaGetDevice(&p->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(p->d_status, 0, sizeof(int));
  if (e != cudaSuccess) { int rc = qft_set_cuda(p, e); free_resources(p); return rc; }
  p->no_stage = 0;
  p->node_log2 = qft_lib::kNodeLog2;
  p->node_nt = qft_lib::kNodeThreads;
  if (r >= 2) {
    p->tune = qft_default_tune(r);
    p->tune.L1 = qft_lib::kL1;
    p->tune.LB = qft_lib::kLB;
    const int64_t N = int64_t(1) << r;
    // FP32 secant table (Sec. 6.1), Gray order of the butterflies
    const size_t nsec = (size_t)N / 4 + 1;
    float* hsec = (float*)calloc(nsec, sizeof(float));
    if (!hsec) return QFT_ERR_CUDA;
    qft_fill_gray_secants(r, hsec);
    e = cudaMalloc(&p->d_sec, sizeof(float) * nsec);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_sec, hsec, sizeof(float) * nsec, cudaMemcpyHostToDevice);
    free(hsec);
    if (e != cudaSuccess) { int rc = qft_set_cuda(p, e); free_resources(p); return rc; }
    if (r <= qft_lib::kMaxRowLog2) {
      p->threads = qft_default_threads(r);
    } else {
      p->large_host = (QftLargePlan*)malloc(sizeof(QftLargePlan));
      if (!p->large_host) { free_resources(p); return QFT_ERR_CUDA; }
      p->side_len = qft_side_len((int)N);
      // the largest classes run on compensated pairs unless the plan asks for plain FP32
      p->comp_j = plain ? 0 : qft_comp_classes(r);
      const int64_t items = kind == QFT_KIND_C2C ? batch : (batch + 1) / 2;   // real kinds: row pairs
      // two copies of the class data (one for in-place plans, plus the halo
      // copies of the SLICE block edges) plus the FINAL tasks' C/S tables,
      // plus the lo parts of the copies and halos for compensated plans
      const int64_t lo = p->comp_j > 0 ? 2 : 1;
      const int64_t per_row = (p->inplace ? lo : 2 * lo) * 2 * (int64_t)p->side_len * 8 +
                              (int64_t)qft_lib::large_tab_cells((int)N, qft_lib::kLargeMinLF) * 8 +
                              (p->inplace ? lo * (int64_t)QFT_IP_EDGES(r) * QFT_IP_HALO * 8 : 0);
      int64_t rows = qft_lib::kScratchBudget / per_row;
      if (rows > items) rows = items;
      if (rows > 65535) rows = 65535;
      if (rows < 1) rows = 1;
      p->scratch_rows = rows;
      p->threads = 256;
      p->large_tab = (r <= 20 && rows >= 64) ? 1 : 0;
      if (items > 0) e = cudaMalloc(&p->scratch, (size_t)(rows * per_row));
      if (items > 0 && e == cudaSuccess) p->scratch_bytes = rows * per_row;
      if (e != cudaSuccess) { int rc = qft_set_cuda(p, e); free_resources(p); return rc; }
    }
    // large rows: the NODE kernel at 256 threads (two CTAs per SM) where the
    // planner accepts it (nodes of at most 2^11 cells), else 512
    int rc = QFT_ERR_INVALID_N;
    if (p->large_host) rc = plan_schedule(p, p->tune, p->threads, p->node_log2, 256);
    if (rc != QFT_OK) rc = plan_schedule(p, p->tune, p->threads, p->node_log2, p->node_nt);
    if (rc != QFT_OK) { free_resources(p); return rc; }
  }
  return QFT_OK;
}

// The kernels of one execute of a single-size plan (arguments already checked).
static int launch_plain(qft_plan p, int op, const void* in, void* out, cudaStream_t st) {
  if (p->kind == QFT_KIND_R2C) return qft_launch_real(p, op, in, out, st);
  if (p->kind == QFT_KIND_DCT0 || p->kind == QFT_KIND_DST0) return qft_launch_r2r(p, in, out, st);
  switch (p->dtype) {
  case QFT_DTYPE_F32: return qft_launch_c2c_f32(p, op, in, out, st);
  case QFT_DTYPE_F16: return qft_launch_c2c_f16(p, op, in, out, st);
  case QFT_DTYPE_BF16: return qft_launch_c2c_bf16(p, op, in, out, st);
  default: return QFT_ERR_DTYPE;
  }
}

// ------------------------------------------------------------------ autotuner
// The schedule knobs (tile sizes of the phases, threads per CTA, input staging,
// node size and NODE threads of the large-row path) change how the work is cut,
// never an arithmetic operation or its operands, so every schedule gives the
// same bits.  The tuner times the forward execute of candidate schedules on
// the plan's own row count (capped so that a candidate moves ~256 MB) and keeps
// the fastest, by coordinate descent from the default: one knob at a time over
// its values, two sweeps.  Results are cached per (length, kind, dtype, rows,
// device) for the life of the process.
struct QftSched {
  QftTune t;
  int threads, no_stage, node_log2, node_nt;
  int64_t chunk_rows;
};

static std::mutex g_tune_mu;
struct TuneKey {
  int r, kind, dtype, dev, comp;
  int64_t rows;
  bool operator==(const TuneKey& o) const {
    return r == o.r && kind == o.kind && dtype == o.dtype && dev == o.dev && comp == o.comp && rows == o.rows;
  }
};
static TuneKey g_tune_keys[256];
static QftSched g_tune_vals[256];
static int g_tune_n = 0;

static bool sched_same(const QftSched& a, const QftSched& b) {
  return a.t.L1 == b.t.L1 && a.t.LS == b.t.LS && a.t.LL == b.t.LL && a.t.LB == b.t.LB && a.t.LF == b.t.LF &&
         a.threads == b.threads && a.no_stage == b.no_stage && a.node_log2 == b.node_log2 &&
         a.node_nt == b.node_nt && a.chunk_rows == b.chunk_rows;
}

static QftSched sched_of(qft_plan p) {
  QftSched c;
  c.t = p->tune; c.threads = p->threads; c.no_stage = p->no_stage;
  c.node_log2 = p->node_log2; c.node_nt = p->node_nt;
  c.chunk_rows = p->chunk_rows;
  return c;
}

static int sched_apply(qft_plan p, const QftSched& c) {
  const int rc = plan_schedule(p, c.t, c.threads, c.node_log2, c.node_nt);
  if (rc == QFT_OK) { p->no_stage = c.no_stage; p->chunk_rows = c.chunk_rows; }
  return rc;
}

// Mean milliseconds of one forward execute on `rows` rows (or -1 if the
// schedule cannot launch).
static float tune_time(qft_plan p, const void* din, void* dout, int64_t rows, cudaStream_t st, cudaEvent_t e0,
                       cudaEvent_t e1) {
  const int64_t keep = p->batch;
  p->batch = rows;
  float ms = -1.f;
  int rc = QFT_OK;
  for (int w = 0; w < 2 && rc == QFT_OK; ++w) rc = launch_plain(p, QFT_OP_FORWARD, din, dout, st);
  const int reps = 3;
  if (rc == QFT_OK) {
    cudaEventRecord(e0, st);
    for (int k = 0; k < reps && rc == QFT_OK; ++k) rc = launch_plain(p, QFT_OP_FORWARD, din, dout, st);
    cudaEventRecord(e1, st);
  }
  if (cudaStreamSynchronize(st) == cudaSuccess && rc == QFT_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
    ms /= reps;
  else
    ms = -1.f;
  cudaGetLastError();   // a schedule that cannot launch leaves no error behind
  p->batch = keep;
  p->last_cuda = cudaSuccess;
  return ms;
}

static int autotune(qft_plan p) {
  if (p->r < 3 || p->batch == 0) return QFT_OK;
  const int64_t N = p->n;
  const int64_t items = p->kind == QFT_KIND_C2C ? p->batch : (p->batch + 1) / 2;
  const int64_t row_bytes = p->kind == QFT_KIND_R2C ? 4 * N + 8 * (N / 2 + 1)
                            : p->kind == QFT_KIND_C2C ? (p->dtype == QFT_DTYPE_F32 ? 16 : 8) * N
                                                      : 4 * N;   // DCT-0 / DST-0: N/2 reals in and out
  int64_t cap = ((int64_t)256 << 20) / row_bytes;
  if (cap < 1) cap = 1;
  const int64_t rows = p->batch < cap ? p->batch : cap;
  const TuneKey key{p->r, p->kind, p->dtype, p->device, p->comp_j, rows};
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    for (int i = 0; i < g_tune_n; ++i)
      if (g_tune_keys[i] == key) return sched_apply(p, g_tune_vals[i]);
  }
  (void)items;
  void* din = nullptr;
  void* dout = nullptr;
  const size_t bytes = (size_t)rows * (size_t)N * 8 + 64;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&din, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&dout, bytes);
  if (e == cudaSuccess) e = cudaMemset(din, 0, bytes);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  int rc = qft_set_cuda(p, e);
  QftSched best = sched_of(p);
  if (rc == QFT_OK) {
    float best_ms = tune_time(p, din, dout, rows, st, e0, e1);
    const bool large = p->r > qft_lib::kMaxRowLog2;
    static const int kThreads[] = {256, 512};
    static const int kLS[] = {2, 3, 4};
    static const int kLL[] = {0, 2, 3, 4};
    static const int kLB[] = {2, 3};
    static const int kLF[] = {1, 2, 3};
    static const int kStage[] = {0, 1};
    // node size and NODE threads are tried together: 256 threads need smaller
    // nodes at large N, which one knob at a time would never reach
    static const int kNode[] = {(12 << 16) | 512, (12 << 16) | 256, (11 << 16) | 256, (11 << 16) | 512,
                                (10 << 16) | 256, (10 << 16) | 512};
    for (int sweep = 0; sweep < 2; ++sweep) {
      for (int knob = 0; knob < 8; ++knob) {
        const int* vals = nullptr;
        int nv = 0;
        switch (knob) {
        case 0: if (!large) { vals = kThreads; nv = 2; } break;
        case 1: vals = kLS; nv = 3; break;
        case 2: vals = kLL; nv = 4; break;
        case 3: vals = kLB; nv = 2; break;
        case 4: if (!large) { vals = kLF; nv = 3; } break;
        case 5: if (!large) { vals = kStage; nv = 2; } break;
        case 6: if (large) { vals = kNode; nv = 6; } break;   // (node size, NODE threads) pairs

        }
        for (int v = 0; v < nv; ++v) {
          QftSched c = best;
          switch (knob) {
          case 0: c.threads = vals[v]; break;
          case 1: c.t.LS = vals[v]; break;
          case 2: c.t.LL = vals[v]; break;
          case 3: c.t.LB = vals[v]; break;
          case 4: c.t.LF = vals[v]; break;
          case 5: c.no_stage = vals[v]; break;
          case 6: c.node_log2 = vals[v] >> 16; c.node_nt = vals[v] & 0xffff; break;
          }
          if (sched_same(c, best)) continue;
          if (sched_apply(p, c) != QFT_OK) continue;
          const float ms = tune_time(p, din, dout, rows, st, e0, e1);
          if (ms > 0.f && (best_ms < 0.f || ms < 0.98f * best_ms)) { best = c; best_ms = ms; }
        }
        sched_apply(p, best);
      }
    }
    std::lock_guard<std::mutex> g(g_tune_mu);
    if (g_tune_n < 256) { g_tune_keys[g_tune_n] = key; g_tune_vals[g_tune_n] = best; ++g_tune_n; }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaFree(din);
  cudaFree(dout);
  if (rc == QFT_OK) rc = sched_apply(p, best);
  return rc;
}

// Fixed-point plans (QFT_DTYPE_I16, C2C forward only): the constant table and
// the kernel configuration; no schedule, no scratch.
static int plan_create_fixed(qft_plan* out, int64_t n, int64_t batch, int kind, unsigned flags) {
  if (kind != QFT_KIND_C2C) return QFT_ERR_DTYPE;
  if (flags != 0) return QFT_ERR_INVALID_ARG;
  if (n < 2 || (n & (n - 1)) != 0 || n > ((int64_t)1 << qft_lib::kFixedMaxLog2)) return QFT_ERR_INVALID_N;
  if (batch < 0 || batch > (int64_t(1) << 40)) return QFT_ERR_INVALID_BATCH;
  int r = 0;
  while ((int64_t(1) << r) < n) ++r;
  qft_plan p = new (std::nothrow) qft_plan_s();
  if (!p) return QFT_ERR_CUDA;
  int rc = plan_init(p, 1, batch, kind, QFT_DTYPE_I16);   // common fields and the status word only
  if (rc != QFT_OK) { delete p; return rc; }
  p->n = n;
  p->r = r;
  rc = qft_fixed_prepare(p);
  if (rc != QFT_OK) { free_resources(p); delete p; return rc; }
  register_plan(p);
  *out = p;
  return QFT_OK;
}

extern "C" int qft_plan_create(qft_plan* out, int64_t n, int64_t batch, int kind, int dtype, unsigned flags) {
  if (!out) return QFT_ERR_NULLPTR;
  *out = nullptr;
  if ((flags & ~(QFT_PLAN_AUTOTUNE | QFT_PLAN_FP32_PLAIN | QFT_PLAN_IN_PLACE)) != 0) return QFT_ERR_INVALID_ARG;
  if (kind != QFT_KIND_C2C && kind != QFT_KIND_R2C && kind != QFT_KIND_DCT0 && kind != QFT_KIND_DST0)
    return QFT_ERR_DTYPE;
  if (dtype == QFT_DTYPE_I16) return plan_create_fixed(out, n, batch, kind, flags);
  if (dtype != QFT_DTYPE_F32 && dtype != QFT_DTYPE_F16 && dtype != QFT_DTYPE_BF16) return QFT_ERR_DTYPE;
  if (kind != QFT_KIND_C2C && dtype != QFT_DTYPE_F32) return QFT_ERR_DTYPE;
  if (n < 2 || (n & (n - 1)) != 0) return QFT_ERR_INVALID_N;
  if (kind != QFT_KIND_C2C && n < 4) return QFT_ERR_INVALID_N;
  int r = 0;
  while ((int64_t(1) << r) < n) ++r;
  if (r > qft_lib::kMaxLog2) return QFT_ERR_INVALID_N;
  if (batch < 0 || batch > (int64_t(1) << 40)) return QFT_ERR_INVALID_BATCH;

  qft_plan p = new (std::nothrow) qft_plan_s();
  if (!p) return QFT_ERR_CUDA;
  int rc = plan_init(p, r, batch, kind, dtype, (flags & QFT_PLAN_FP32_PLAIN) ? 1 : 0,
                     (flags & QFT_PLAN_IN_PLACE) ? 1 : 0);
  if (rc != QFT_OK) { delete p; return rc; }
  if (flags & QFT_PLAN_AUTOTUNE) {
    rc = autotune(p);
    if (rc != QFT_OK) { free_resources(p); delete p; return rc; }
  }
  register_plan(p);
  *out = p;
  return QFT_OK;
}

// Ragged plans: rows grouped by length, one (unregistered) sub-plan per length
// class, and the class launches captured once into a CUDA graph that reads the
// execute-time pointers from d_args.
static void free_ragged(qft_plan p) {
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  if (p->graph) cudaGraphDestroy(p->graph);
  for (int c = 0; c < p->nclasses; ++c) {
    if (p->classes[c].sub) { free_resources(p->classes[c].sub); delete p->classes[c].sub; }
    cudaFree(p->classes[c].d_rows);
  }
  free(p->classes);
  cudaFree(p->d_offsets);
  cudaFree(p->d_args);
  p->classes = nullptr; p->nclasses = 0; p->d_offsets = nullptr; p->d_args = nullptr;
  p->graph = nullptr; p->gexec = nullptr;
}

__global__ void k_set_args(QftIoArgs* d, QftIoArgs v) { *d = v; }

static int ragged_launch_all(qft_plan p, cudaStream_t st) {
  for (int c = 0; c < p->nclasses; ++c) {
    const int rc = qft_launch_ragged_class(p->classes[c].sub, p->d_args, p->d_offsets, p->classes[c].d_rows, st);
    if (rc != QFT_OK) { p->last_cuda = p->classes[c].sub->last_cuda; return rc; }
  }
  return QFT_OK;
}

// The same launches on one forked stream per length class (ss[c], created by
// the caller before the capture), joined back into `st` through the events
// ev[0..n] (used while capturing the graph): the classes share nothing but the
// argument block, which they only read, so their launches may overlap, and
// the small classes fill the SMs the large ones leave idle at their tails.
static int ragged_launch_forked(qft_plan p, cudaStream_t st, cudaStream_t* ss, cudaEvent_t* ev) {
  const int n = p->nclasses;
  cudaError_t e = cudaEventRecord(ev[n], st);
  int rc = QFT_OK;
  for (int c = 0; c < n && e == cudaSuccess && rc == QFT_OK; ++c) {
    e = cudaStreamWaitEvent(ss[c], ev[n], 0);
    if (e != cudaSuccess) break;
    rc = qft_launch_ragged_class(p->classes[c].sub, p->d_args, p->d_offsets, p->classes[c].d_rows, ss[c]);
    if (rc != QFT_OK) { p->last_cuda = p->classes[c].sub->last_cuda; break; }
    e = cudaEventRecord(ev[c], ss[c]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev[c], 0);
  }
  if (rc == QFT_OK && e != cudaSuccess) rc = qft_set_cuda(p, e);
  return rc;
}

extern "C" int qft_plan_create_ragged(qft_plan* out, const int64_t* offsets_host, const int32_t* log2n_host,
                                      int64_t count, int kind, int dtype, unsigned flags) {
  if (!out) return QFT_ERR_NULLPTR;
  *out = nullptr;
  if ((flags & ~(QFT_PLAN_AUTOTUNE | QFT_PLAN_FP32_PLAIN | QFT_PLAN_IN_PLACE)) != 0) return QFT_ERR_INVALID_ARG;
  if (kind != QFT_KIND_C2C || dtype != QFT_DTYPE_F32) return QFT_ERR_DTYPE;
  if (count < 0 || count > (int64_t(1) << 31)) return QFT_ERR_INVALID_BATCH;
  if (count > 0 && (!offsets_host || !log2n_host)) return QFT_ERR_NULLPTR;
  if (count > 0 && offsets_host[0] != 0) return QFT_ERR_INVALID_ARG;
  int64_t per_r[32] = {0};
  for (int64_t i = 0; i < count; ++i) {
    const int r = log2n_host[i];
    if (r < 1 || r > qft_lib::kMaxLog2) return QFT_ERR_INVALID_N;
    if (offsets_host[i + 1] - offsets_host[i] != (int64_t(1) << r)) return QFT_ERR_INVALID_ARG;
    per_r[r]++;
  }
  qft_plan p = new (std::nothrow) qft_plan_s();
  if (!p) return QFT_ERR_CUDA;
  int rc = plan_init(p, 1, 0, kind, dtype);   // the container itself holds no kernels' resources
  if (rc != QFT_OK) { delete p; return rc; }
  p->n = 0; p->batch = count; p->r = 0;
  int ncls = 0;
  for (int r = 1; r <= qft_lib::kMaxLog2; ++r) ncls += per_r[r] > 0;
  p->classes = (QftRaggedClass*)calloc(ncls > 0 ? ncls : 1, sizeof(QftRaggedClass));
  if (!p->classes) { delete p; return QFT_ERR_CUDA; }
  cudaError_t e = cudaSuccess;
  // largest rows first: their launches are the longest
  for (int r = qft_lib::kMaxLog2; r >= 1 && rc == QFT_OK; --r) {
    if (!per_r[r]) continue;
    QftRaggedClass& C = p->classes[p->nclasses++];
    C.r = r; C.count = per_r[r]; C.d_rows = nullptr;
    C.sub = new (std::nothrow) qft_plan_s();
    if (!C.sub) { rc = QFT_ERR_CUDA; break; }
    rc = plan_init(C.sub, r, C.count, kind, dtype, (flags & QFT_PLAN_FP32_PLAIN) ? 1 : 0,
                   (flags & QFT_PLAN_IN_PLACE) ? 1 : 0);
    if (rc != QFT_OK) { delete C.sub; C.sub = nullptr; break; }
    if (flags & QFT_PLAN_AUTOTUNE) {
      rc = autotune(C.sub);
      if (rc != QFT_OK) break;
    }
    int32_t* rows = (int32_t*)malloc(sizeof(int32_t) * (size_t)C.count);
    if (!rows) { rc = QFT_ERR_CUDA; break; }
    int64_t k = 0;
    for (int64_t i = 0; i < count; ++i) if (log2n_host[i] == r) rows[k++] = (int32_t)i;
    e = cudaMalloc(&C.d_rows, sizeof(int32_t) * (size_t)C.count);
    if (e == cudaSuccess) e = cudaMemcpy(C.d_rows, rows, sizeof(int32_t) * (size_t)C.count, cudaMemcpyHostToDevice);
    free(rows);
    if (e != cudaSuccess) rc = qft_set_cuda(p, e);
  }
  if (rc == QFT_OK) {
    e = cudaMalloc(&p->d_offsets, sizeof(int64_t) * (size_t)(count + 1));
    if (e == cudaSuccess && count > 0)
      e = cudaMemcpy(p->d_offsets, offsets_host, sizeof(int64_t) * (size_t)(count + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_args, sizeof(QftIoArgs));
    if (e != cudaSuccess) rc = qft_set_cuda(p, e);
  }
  if (rc == QFT_OK && p->nclasses > 0) {
    // capture every class launch once; executes replay the graph
    cudaStream_t cs = nullptr;
    const int nc = p->nclasses;
    cudaStream_t* fs = (cudaStream_t*)calloc((size_t)nc, sizeof(cudaStream_t));
    cudaEvent_t* fe = (cudaEvent_t*)calloc((size_t)nc + 1, sizeof(cudaEvent_t));
    e = (fs && fe) ? cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) : cudaErrorMemoryAllocation;
    for (int c = 0; c < nc && e == cudaSuccess; ++c) e = cudaStreamCreateWithFlags(&fs[c], cudaStreamNonBlocking);
    for (int c = 0; c <= nc && e == cudaSuccess; ++c) e = cudaEventCreateWithFlags(&fe[c], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const int lrc = ragged_launch_forked(p, cs, fs, fe);
      cudaGraph_t g = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
      if (lrc == QFT_OK && e2 == cudaSuccess) {
        p->graph = g;
        e = cudaGraphInstantiate(&p->gexec, g, 0);
        size_t nn = 0;
        if (e == cudaSuccess) e = cudaGraphGetNodes(g, nullptr, &nn);
        p->graph_kernels = (int)nn;
      } else {
        if (g) cudaGraphDestroy(g);
        e = e2 != cudaSuccess ? e2 : cudaErrorUnknown;
      }
    }
    if (cs) cudaStreamDestroy(cs);
    for (int c = 0; fs && c < nc; ++c) if (fs[c]) cudaStreamDestroy(fs[c]);
    for (int c = 0; fe && c <= nc; ++c) if (fe[c]) cudaEventDestroy(fe[c]);
    free(fs);
    free(fe);
    if (e != cudaSuccess) {   // no graph: executes launch the classes directly
      if (p->graph) { cudaGraphDestroy(p->graph); p->graph = nullptr; }
      p->gexec = nullptr;
      cudaGetLastError();
    }
  }
  if (rc != QFT_OK) { free_ragged(p); free_resources(p); delete p; return rc; }
  register_plan(p);
  *out = p;
  return QFT_OK;
}

static int exec_ragged(qft_plan p, int op, const void* in, void* out, cudaStream_t st) {
  QftIoArgs a;
  a.in = in; a.out = out; a.scale = 1.f; a.scaled = 0;
  switch (op) {
  case QFT_OP_FORWARD: a.in_op = QFT_LANE_ID; a.out_op = QFT_LANE_ID; break;
  case QFT_OP_INVERSE: a.in_op = QFT_LANE_SWAP; a.out_op = QFT_LANE_SWAP; a.scaled = 2; break;
  case QFT_OP_FORWARD_ADJOINT: a.in_op = QFT_LANE_CONJ; a.out_op = QFT_LANE_CONJ; break;
  case QFT_OP_INVERSE_ADJOINT: a.in_op = QFT_LANE_ID; a.out_op = QFT_LANE_ID; a.scaled = 2; break;
  default: return QFT_ERR_INVALID_ARG;
  }
  k_set_args<<<1, 1, 0, st>>>(p->d_args, a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return qft_set_cuda(p, e);
  if (p->gexec) return qft_set_cuda(p, cudaGraphLaunch(p->gexec, st));
  return ragged_launch_all(p, st);
}

// ---------------------------------------------------------- spectral filter
static const int kKindFilter = 100;   // internal kind of filter plans (not a QFT_KIND_*)

extern "C" int qft_filter_create(qft_plan* out, int64_t n, int64_t batch, int64_t channels, unsigned flags) {
  if (!out) return QFT_ERR_NULLPTR;
  *out = nullptr;
  if (flags != 0) return QFT_ERR_INVALID_ARG;
  if (n < 4 || (n & (n - 1)) != 0 || n > (int64_t(1) << 13)) return QFT_ERR_INVALID_N;
  if (batch < 1 || channels < 1 || batch > (int64_t(1) << 24) || channels > (int64_t(1) << 20))
    return QFT_ERR_INVALID_BATCH;
  int r = 0;
  while ((int64_t(1) << r) < n) ++r;
  qft_plan p = new (std::nothrow) qft_plan_s();
  if (!p) return QFT_ERR_CUDA;
  int rc = plan_init(p, r, batch, QFT_KIND_R2C, QFT_DTYPE_F32);
  if (rc != QFT_OK) { delete p; return rc; }
  p->kind = kKindFilter;
  p->channels = channels;
  // partial weight gradients [C][parts][n/2+1] (complex)
  const size_t bytes = (size_t)channels * qft_filter_parts() * (size_t)(n / 2 + 1) * 8;
  cudaError_t e = cudaMalloc(&p->scratch, bytes);
  if (e != cudaSuccess) { rc = qft_set_cuda(p, e); free_resources(p); delete p; return rc; }
  p->scratch_bytes = (int64_t)bytes;
  register_plan(p);
  *out = p;
  return QFT_OK;
}

static int filter_check(qft_plan p, const void* a, const void* b, const void* c) {
  int rc = plan_check(p);
  if (rc != QFT_OK) return rc;
  if (p->kind != kKindFilter) return QFT_ERR_INVALID_ARG;
  if (!a || !b || !c) return QFT_ERR_NULLPTR;
  return QFT_OK;
}

extern "C" int qft_filter_forward(qft_plan p, const float* x, const void* W, float* y, void* stream) {
  int rc = filter_check(p, x, W, y);
  if (rc != QFT_OK) return rc;
  if (((uintptr_t)x % 4) || ((uintptr_t)y % 4) || ((uintptr_t)W % 8)) return QFT_ERR_ALIGN;
  if ((const void*)x == (const void*)y) return QFT_ERR_INPLACE;
  p->last_stream = static_cast<cudaStream_t>(stream);
  return qft_launch_filter(p, 0, x, W, nullptr, y, nullptr, p->last_stream);
}

extern "C" int qft_filter_backward(qft_plan p, const float* x, const void* W, const float* gy, float* gx, void* gW,
                                   void* stream) {
  int rc = filter_check(p, x, W, gy);
  if (rc != QFT_OK) return rc;
  if (!gx || !gW) return QFT_ERR_NULLPTR;
  if (((uintptr_t)x % 4) || ((uintptr_t)gy % 4) || ((uintptr_t)gx % 4) || ((uintptr_t)W % 8) ||
      ((uintptr_t)gW % 8))
    return QFT_ERR_ALIGN;
  if ((const void*)gx == (const void*)gy || (const void*)gx == (const void*)x) return QFT_ERR_INPLACE;
  p->last_stream = static_cast<cudaStream_t>(stream);
  return qft_launch_filter(p, 1, x, W, gy, gx, gW, p->last_stream);
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
  free_ragged(p);
  free_resources(p);
  p->magic = kDead;
  delete p;
  return QFT_OK;
}

extern "C" int qft_execute(qft_plan p, int op, const void* in, void* out, void* stream) {
  int rc = plan_check(p);
  if (rc != QFT_OK) return rc;
  if (op < QFT_OP_FORWARD || op > QFT_OP_INVERSE_ADJOINT) return QFT_ERR_INVALID_ARG;
  if (p->dtype == QFT_DTYPE_I16) return QFT_ERR_DTYPE;   // qft_execute_fixed
  if (p->batch == 0) return QFT_OK;
  if (!in || !out) return QFT_ERR_NULLPTR;
  const size_t al_c = p->dtype == QFT_DTYPE_F32 ? 8 : 4;
  if (p->kind == QFT_KIND_C2C) {
    if (((uintptr_t)in % al_c) || ((uintptr_t)out % al_c)) return QFT_ERR_ALIGN;
  } else if (p->kind == QFT_KIND_DCT0 || p->kind == QFT_KIND_DST0) {
    // symmetric matrices: the adjoint is the transform itself; no inverse op
    if (op != QFT_OP_FORWARD && op != QFT_OP_FORWARD_ADJOINT) return QFT_ERR_INVALID_ARG;
    if (((uintptr_t)in % 4) || ((uintptr_t)out % 4)) return QFT_ERR_ALIGN;
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
  if (p->kind == kKindFilter) return QFT_ERR_INVALID_ARG;
  if (p->classes) return exec_ragged(p, op, in, out, st);
  rc = launch_plain(p, op, in, out, st);
  p->withhold_copy = 0;   // the test of the timeout path is one-shot
  return rc;
}

extern "C" int qft_execute_fixed(qft_plan p, const void* in, void* out, int32_t* exponents, void* stream) {
  int rc = plan_check(p);
  if (rc != QFT_OK) return rc;
  if (p->dtype != QFT_DTYPE_I16) return QFT_ERR_DTYPE;
  if (p->batch == 0) return QFT_OK;
  if (!in || !out || !exponents) return QFT_ERR_NULLPTR;
  if (((uintptr_t)in % 4) || ((uintptr_t)out % 8) || ((uintptr_t)exponents % 4)) return QFT_ERR_ALIGN;
  if (in == out || (const void*)exponents == in || (void*)exponents == out) return QFT_ERR_INPLACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  p->last_stream = st;
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return qft_set_cuda(p, e);
  if (cur != p->device) return QFT_ERR_INVALID_ARG;
  return qft_launch_fixed(p, in, out, exponents, st);
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
  rc = qft_set_cuda(p, cudaStreamSynchronize(p->last_stream));
  if (rc != QFT_OK) return rc;
  // the plan's own status word and those of its sub-plans (ragged)
  int st = 0;
  rc = qft_set_cuda(p, cudaMemcpy(&st, p->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (rc != QFT_OK) return rc;
  cudaMemset(p->d_status, 0, sizeof(int));
  for (int c = 0; c < p->nclasses && st == 0; ++c) {
    int sc = 0;
    if (cudaMemcpy(&sc, p->classes[c].sub->d_status, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && sc) {
      st = sc;
      cudaMemset(p->classes[c].sub->d_status, 0, sizeof(int));
    }
  }
  return st;
}

extern "C" int qft_plan_scratch_bytes(qft_plan p, int64_t* bytes) {
  int rc = plan_check(p);
  if (rc != QFT_OK) return rc;
  int64_t b = p->scratch_bytes;
  for (int c = 0; c < p->nclasses; ++c) b += p->classes[c].sub->scratch_bytes;
  if (bytes) *bytes = b;
  return QFT_OK;
}

extern "C" int qft_plan_comp_classes(qft_plan p) {
  int rc = plan_check(p);
  if (rc != QFT_OK) return rc;
  if (p->classes) {   // ragged: the largest of its length classes
    int j = 0;
    for (int c = 0; c < p->nclasses; ++c) j = p->classes[c].sub->comp_j > j ? p->classes[c].sub->comp_j : j;
    return j;
  }
  return p->comp_j;
}

extern "C" int qft_plan_set_wait_limit(qft_plan p, int64_t ns) {
  int rc = plan_check(p);
  if (rc != QFT_OK) return rc;
  if (p->classes || p->kind == kKindFilter || p->dtype == QFT_DTYPE_I16 || ns < 0) return QFT_ERR_INVALID_ARG;
  p->wait_ns = ns;
  return QFT_OK;
}

extern "C" int qft_plan_withhold_next_copy(qft_plan p) {
  int rc = plan_check(p);
  if (rc != QFT_OK) return rc;
  if (p->classes || p->kind == kKindFilter || p->dtype == QFT_DTYPE_I16) return QFT_ERR_INVALID_ARG;
  p->withhold_copy = 1;
  return QFT_OK;
}

extern "C" int qft_plan_last_cuda_error(qft_plan p) {
  if (plan_check(p) != QFT_OK) return 0;
  return (int)p->last_cuda;
}

extern "C" int qft_plan_info(qft_plan p, int* threads, int* ctas, int* smem_bytes, int* launches) {
  int rc = plan_check(p);
  if (rc != QFT_OK) return rc;
  if (threads) *threads = p->threads;
  // large-row plans: the NODE launch's CTAs and every launch of every scratch chunk
  const int64_t items = p->kind == QFT_KIND_C2C ? p->batch : (p->batch + 1) / 2;
  const int64_t crow = p->chunk_rows > 0 && p->chunk_rows < p->scratch_rows ? p->chunk_rows : p->scratch_rows;
  const int64_t chunks = crow > 0 ? (items + crow - 1) / crow : 0;
  if (ctas) *ctas = p->large_host ? (int)(p->large_host->node_ctas * (crow < items ? crow : items))
                                  : p->grid;
  if (smem_bytes) *smem_bytes = (int)p->smem;
  int per_chunk = p->large_host ? p->large_host->nphase : 0;
  if (p->large_host && p->large_host->inplace)   // the halo copy before each in-place SLICE level of several blocks
    for (int i = 0; i < p->large_host->nphase; ++i)
      per_chunk += p->large_host->phases[i].kind == QFT_LPH_SLICE && p->large_host->phases[i].ntasks > QFT_IP_TASKS;
  if (launches) *launches = p->classes ? 1 + p->graph_kernels : (p->large_host ? (int)(per_chunk * chunks) : 1);
  return QFT_OK;
}

extern "C" int qft_plan_time_launches(qft_plan p, int enable) {
  int rc = plan_check(p);
  if (rc != QFT_OK) return rc;
  if (p->classes) return QFT_ERR_INVALID_ARG;
  p->timing = enable ? 1 : 0;
  p->tev_n = 0;
  return QFT_OK;
}

extern "C" int qft_plan_launch_times(qft_plan p, float* ms, int* launches) {
  int rc = plan_check(p);
  if (rc != QFT_OK) return rc;
  if (!ms || !launches) return QFT_ERR_NULLPTR;
  for (int k = 0; k < QFT_KERNEL_KINDS; ++k) { ms[k] = 0.f; launches[k] = 0; }
  for (int i = 0; i < p->tev_n; ++i) {
    cudaError_t e = cudaEventSynchronize(p->tev[2 * i + 1]);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, p->tev[2 * i], p->tev[2 * i + 1]);
    if (e != cudaSuccess) return qft_set_cuda(p, e);
    ms[p->tev_kind[i]] += t;
    launches[p->tev_kind[i]] += 1;
  }
  p->tev_n = 0;
  return QFT_OK;
}

extern "C" int qft_plan_schedule(qft_plan p, int* v) {
  int rc = plan_check(p);
  if (rc != QFT_OK) return rc;
  if (!v) return QFT_ERR_NULLPTR;
  v[0] = p->threads; v[1] = p->tune.L1; v[2] = p->tune.LS; v[3] = p->tune.LL; v[4] = p->tune.LB;
  v[5] = p->tune.LF; v[6] = p->no_stage ? 0 : 1; v[7] = p->large_host ? p->node_log2 : 0;
  v[8] = p->large_host ? p->node_nt : 0;
  v[9] = p->large_host ? (int)(p->chunk_rows > 0 && p->chunk_rows < p->scratch_rows ? p->chunk_rows : p->scratch_rows) : 0;
  return QFT_OK;
}

extern "C" int qft_plan_set_schedule(qft_plan p, const int* v) {
  int rc = plan_check(p);
  if (rc != QFT_OK) return rc;
  if (!v) return QFT_ERR_NULLPTR;
  if (p->classes || p->kind == kKindFilter || p->r < 2 || p->dtype == QFT_DTYPE_I16) return QFT_ERR_INVALID_ARG;
  QftSched c = sched_of(p);
  c.threads = p->large_host ? p->threads : v[0];
  if (!p->large_host && c.threads != 256 && c.threads != 512) return QFT_ERR_INVALID_ARG;
  if (v[1] != qft_lib::kL1) return QFT_ERR_INVALID_ARG;
  c.t.LS = v[2]; c.t.LL = v[3]; c.t.LB = v[4]; c.t.LF = v[5];
  if (c.t.LB > qft_lib::kLB) return QFT_ERR_INVALID_ARG;
  c.no_stage = v[6] ? 0 : 1;
  if (p->large_host) {
    if (v[8] != 256 && v[8] != 512) return QFT_ERR_INVALID_ARG;
    if (v[9] < 0) return QFT_ERR_INVALID_ARG;
    c.node_log2 = v[7]; c.node_nt = v[8];
    c.chunk_rows = v[9] >= p->scratch_rows ? 0 : v[9];
  }
  return sched_apply(p, c);
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
