/*
 * qft_gb300.h -- C ABI of the GB300 (sm_103a) improved-QFT library.
 *
 * The library computes batched power-of-two DFTs by the improved Quick
 * Fourier Transform of L. Pasquini, "Improved QFT algorithm for power-of-two
 * FFT" (arXiv 1301.0763):
 *   - forward:  X(k) = sum_n x(n) e^{-2 pi i n k / N}  (eq qft_0A, unscaled),
 *     computed by the recursion of Sec. 5 (cdft -> rdft -> dct/dst ->
 *     dct_ot/dct_oo/dst_ot/dst_oo) with the constants of Sec. 6.1;
 *   - inverse:  x = swap(DFT(swap(X))) / N (swap exchanges re and im); the
 *     paper is silent on the inverse, this is the reading the library takes;
 *   - backward: the exact adjoint of the forward map (the transform is linear,
 *     so a backward pass stores nothing);
 *   - inverse backward: the exact adjoint of the inverse map.
 *
 * Conventions shared by every entry point
 *   - All data pointers are DEVICE pointers owned by the caller.  Rows are
 *     contiguous and row-major: [batch][N] complex (interleaved re, im) for
 *     QFT_KIND_C2C; [batch][N] real and [batch][N/2+1] complex for
 *     QFT_KIND_R2C.  Outputs are in natural frequency (or time) order.
 *   - Storage dtype (QFT_DTYPE_*): FP32 (complex64 / float32), FP16 or BF16
 *     pairs (C2C only).  Arithmetic is always FP32 with round-to-nearest.
 *   - Pointers must be aligned to their element size (8 bytes for complex64,
 *     4 bytes otherwise); misaligned pointers return QFT_ERR_ALIGN.
 *   - Execution is asynchronous and ordered on the CUDA stream passed as
 *     `stream` (a cudaStream_t; NULL means the legacy default stream).  No
 *     call synchronises the host except qft_plan_sync_status.
 *   - C2C, DCT-0 and DST-0 transforms may run in place (in == out); R2C may not.
 *   - Every call returns QFT_OK (0) or a negative QFT_ERR_* code and never
 *     throws.  CUDA errors are reported as QFT_ERR_CUDA; the CUDA error code is
 *     kept in the plan (qft_plan_last_cuda_error).
 *   - Plans are not thread-safe: one plan must not be executed concurrently
 *     from several host threads.  Different plans are independent.
 */
#ifndef QFT_GB300_H
#define QFT_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qft_plan_s* qft_plan;

/* transform kinds */
#define QFT_KIND_C2C 0 /* complex -> complex, length N */
#define QFT_KIND_R2C 1 /* forward: real N -> complex N/2+1 (Hermitian-pruned, rdft of Sec. 4.2);
                          inverse: complex N/2+1 -> real N (1/N scaled)                      */
#define QFT_KIND_DCT0 2 /* DCT-0 of periodization N (eq qft_0B, the dct recursion of Sec. 5):
                           real c(n), n in [0, N/2] -> C(k) = sum_n c(n) cos(2 pi n k/N), k in [0, N/2] */
#define QFT_KIND_DST0 3 /* DST-0 of periodization N (eq qft_0C, the dst recursion of Sec. 5):
                           real d(n), n in [1, N/2-1] -> S(k) = sum_n d(n) sin(2 pi n k/N), k in [1, N/2-1] */

/* storage dtypes */
#define QFT_DTYPE_F32 0  /* complex64 (C2C) / float32 real + complex64 spectrum (R2C) */
#define QFT_DTYPE_F16 1  /* complex stored as two IEEE half values (C2C only)          */
#define QFT_DTYPE_BF16 2 /* complex stored as two bfloat16 values (C2C only)           */
#define QFT_DTYPE_I16 3  /* fixed-point variant (C2C forward only, qft_execute_fixed):
                            complex int16 Q15 in, int32 block-floating-point out       */

/* operations for qft_execute */
#define QFT_OP_FORWARD 0
#define QFT_OP_INVERSE 1
#define QFT_OP_FORWARD_ADJOINT 2 /* = backward of the forward transform */
#define QFT_OP_INVERSE_ADJOINT 3 /* = backward of the inverse transform */

/* plan creation flags */
#define QFT_PLAN_AUTOTUNE 1u   /* time candidate schedules at creation and keep the fastest */
#define QFT_PLAN_FP32_PLAIN 2u /* n >= 2^16: evaluate every class tree in plain FP32 (see below)  */
#define QFT_PLAN_IN_PLACE 4u   /* n > 2^14: one scratch copy of the class data (in-place backward levels) */

/* status codes */
#define QFT_OK 0
#define QFT_ERR_INVALID_N (-1)     /* N not a power of two, or outside the supported range */
#define QFT_ERR_INVALID_BATCH (-2) /* batch < 0 or too large                                */
#define QFT_ERR_DTYPE (-3)         /* unknown kind/dtype or unsupported combination          */
#define QFT_ERR_ALIGN (-4)         /* data pointer not aligned to its element size           */
#define QFT_ERR_NULLPTR (-5)       /* null plan, output handle or data pointer               */
#define QFT_ERR_CUDA (-6)          /* a CUDA runtime call failed                             */
#define QFT_ERR_TIMEOUT (-7)       /* a bounded device-side wait expired                     */
#define QFT_ERR_DESTROYED (-8)     /* the plan was destroyed                                 */
#define QFT_ERR_INVALID_ARG (-9)   /* other invalid argument (op code, ragged table, ...)    */
#define QFT_ERR_INPLACE (-10)      /* in == out where not allowed                            */

/*
 * qft_plan_create -- plan `batch` transforms of length n (eq qft_0A with N = n).
 *   out    receives the plan handle (owned by the caller, release with
 *          qft_plan_destroy).
 *   n      transform length (periodization for DCT-0 / DST-0), a power of two,
 *          2 <= n <= 2^24 (C2C) or 4 <= n <= 2^24 (the real kinds).
 *   batch  number of rows (>= 0; 0 makes every execute a no-op).
 *   kind   QFT_KIND_C2C or QFT_KIND_R2C; dtype QFT_DTYPE_*.
 *   flags  0, QFT_PLAN_AUTOTUNE and/or QFT_PLAN_FP32_PLAIN.  With
 *          QFT_PLAN_AUTOTUNE the plan times the
 *          forward transform under candidate schedules (tile sizes of the
 *          phases, threads per CTA, input staging, node size and node threads
 *          for n > 2^14) on up to ~256 MB of its own rows, on a private stream,
 *          and keeps the fastest.  The schedule never changes the result: every
 *          schedule performs the same FP32 operations on the same operands.
 *          Results are cached per (n, kind, dtype, rows, device) in the process.
 *   Precision: the FP32 error of the improved QFT grows like ~3.5e-8 sqrt(n)
 *          (relative L2; it comes from the secant conversion of eq qft_38A,
 *          whose factors reach n/(4 pi)).  For n >= 2^16 the plan therefore
 *          evaluates the dct_ot / dst_ot trees of its J = floor((log2 n - 14)/2)
 *          largest classes on compensated pairs of FP32 numbers (TwoSum adds,
 *          exact FMA product errors, one rounding per class output), which
 *          keeps the error near 5e-6 for every n up to 2^24 at a cost in
 *          throughput; qft_plan_comp_classes reports J.  QFT_PLAN_FP32_PLAIN
 *          turns this off (J = 0: the plain FP32 evaluation of the recursion).
 *   In place (QFT_PLAN_IN_PLACE, Sec. 6.1: every function of the improved QFT
 *          returns as many values as it takes (eqs qft_42/43), which makes an
 *          in-place evaluation possible).  For n > 2^14 the plan keeps one
 *          scratch copy of each row's class data instead of two: the backward
 *          levels above the node depth overwrite the cells they read, leaving
 *          the class outputs in a bit-reversed order that the final combine
 *          reads, and the only extra memory is a halo copy of 8 cells per 256
 *          tasks of a level (plus the C/S tables); qft_plan_scratch_bytes
 *          reports the size.  Same results, bit for bit, as without the flag.
 *          For n <= 2^14 the flag changes nothing: each row is transformed in
 *          place in shared memory.
 * The plan owns the FP32 secant table (Sec. 6.1, N/4 entries) and every
 * scratch buffer; it allocates them here, on the current CUDA device, and
 * frees them in qft_plan_destroy.  Executions must run on that device.
 */
int qft_plan_create(qft_plan* out, int64_t n, int64_t batch, int kind, int dtype, unsigned flags);

/*
 * qft_plan_create_ragged -- plan many independent C2C transforms of uneven
 * power-of-two lengths.  Rows are grouped by length at plan creation (one
 * schedule per length); every execute replays one CUDA graph holding the
 * launches of all length classes (it reads the data pointers from device
 * memory, so the graph is captured once, here).
 *   offsets_host  count+1 int64 entries (host memory): row i occupies complex
 *                 elements [offsets[i], offsets[i+1]) of the packed buffer;
 *                 offsets[0] == 0 and offsets[i+1]-offsets[i] == 2^log2n[i].
 *   log2n_host    count int32 entries (host memory), each in [1, 24].
 *   flags         0, QFT_PLAN_AUTOTUNE (each length class is tuned on its own
 *                 row count before the graph is captured), QFT_PLAN_FP32_PLAIN
 *                 and QFT_PLAN_IN_PLACE (as for qft_plan_create).
 * Data layout: one packed complex buffer for input and one for output.
 * Supported: QFT_KIND_C2C, QFT_DTYPE_F32.
 */
int qft_plan_create_ragged(qft_plan* out, const int64_t* offsets_host, const int32_t* log2n_host,
                           int64_t count, int kind, int dtype, unsigned flags);

/*
 * qft_execute -- run operation `op` (QFT_OP_*) of the plan on `in`, writing `out`.
 * Shapes per op for QFT_KIND_R2C:
 *   FORWARD:          in real [batch][N]      -> out complex [batch][N/2+1]
 *   INVERSE:          in complex [batch][N/2+1] -> out real [batch][N] (1/N scaled;
 *                     the imaginary parts of bins 0 and N/2 are ignored)
 *   FORWARD_ADJOINT:  in complex [batch][N/2+1] -> out real [batch][N]
 *                     (g_x(n) = sum_k Re g_k cos(2 pi n k/N) - Im g_k sin(2 pi n k/N))
 *   INVERSE_ADJOINT:  in real [batch][N] -> out complex [batch][N/2+1]
 *                     (w_k/N times the forward, w = 1 at k = 0, N/2 and 2 elsewhere,
 *                     imaginary parts at k = 0, N/2 set to zero)
 * For QFT_KIND_C2C every op maps [batch][N] complex to [batch][N] complex:
 *   FORWARD = F, INVERSE = F^-1, FORWARD_ADJOINT = F^H, INVERSE_ADJOINT = F / N.
 * For QFT_KIND_DCT0 (rows of N/2+1 floats) and QFT_KIND_DST0 (rows of N/2-1
 * floats, d(1..N/2-1) -> S(1..N/2-1)): FORWARD, or FORWARD_ADJOINT, which is
 * the same map (both matrices are symmetric); other ops return
 * QFT_ERR_INVALID_ARG.  FP32 only, 4-byte aligned, in place allowed.
 */
int qft_execute(qft_plan plan, int op, const void* in, void* out, void* stream);

/* Named forms of qft_execute (same arguments, same errors). */
int qft_execute_forward(qft_plan plan, const void* in, void* out, void* stream);
int qft_execute_inverse(qft_plan plan, const void* in, void* out, void* stream);
int qft_execute_backward(qft_plan plan, const void* grad_out, void* grad_in, void* stream);

/*
 * qft_execute_fixed -- forward DFT (eq qft_0A) of every row of a
 * QFT_DTYPE_I16 plan by the fixed-point variant of the improved QFT: the
 * recursion of Sec. 5 (fold, class split, mirror butterflies, secant
 * conversion eq qft_38A, neighbour adds eqs qft_38B/C, combines eqs
 * qft_5C-6, the CDFT combine of Sec. 4.1) with every value an int32 mantissa
 * of a block floating-point block.  The paper names fixed point as its target
 * (Sec. 1, 7) without a scaling rule; the library's rule: each block
 * (fold output per class, each child of a mirror butterfly, each node and
 * chain output, the output row) is normalized so that its largest mantissa
 * has 29 significant bits, right shifts rounded half up; adds are exact;
 * secants are 31-bit mantissas with their own exponents and the 64-bit
 * products are normalized once per node.
 *   plan       created with kind QFT_KIND_C2C, dtype QFT_DTYPE_I16, flags 0,
 *              2 <= n <= 2^14 (QFT_ERR_INVALID_N otherwise).
 *   in         device, [batch][n] complex int16 pairs (re, im): value q 2^-15;
 *              4-byte aligned.
 *   out        device, [batch][n] complex int32 mantissa pairs; 8-byte aligned.
 *   exponents  device, [batch] int32: X(k) = out(k) * 2^exponents[row]
 *              (0 for a row of zeros); 4-byte aligned.
 *   Outputs are normalized: the largest |mantissa| of a nonzero row lies in
 *   [2^28, 2^29].  The buffers may not overlap (QFT_ERR_INPLACE).  The result
 *   depends on nothing but the input: it is the same bits on every run.
 * Stream-ordered; qft_execute on such a plan returns QFT_ERR_DTYPE.
 */
int qft_execute_fixed(qft_plan plan, const void* in, void* out, int32_t* exponents, void* stream);

/*
 * Spectral-filter layer y = irfft(W (.) rfft(x)) on real rows: rfft is the
 * rdft of Sec. 4.2, irfft the real inverse x(n) = (A(n) - B(n))/N,
 * x(N-n) = (A(n) + B(n))/N with A, B the DCT-0 / DST-0 (eqs qft_0B, qft_0C)
 * of the weighted real and imaginary parts; W is applied bin by bin.
 *   qft_filter_create: plan for x, y of shape [batch][channels][n] (float32,
 *     device, contiguous) and weights W of shape [channels][n/2+1] (complex64).
 *     4 <= n <= 2^13 power of two; batch, channels >= 1.  The plan owns a
 *     scratch of channels * 16 * (n/2+1) complex partial gradients.
 *   qft_filter_forward:  y = irfft(W[c] (.) rfft(x[b][c])) for every b, c.
 *   qft_filter_backward: given x, W and gy = dL/dy, writes
 *     gx = dL/dx = rfft^H(conj(W) (.) irfft^H(gy))  (shape of x) and
 *     gW = dL/dW = sum_b irfft^H(gy[b]) (.) conj(rfft(x[b]))  ([channels][n/2+1]),
 *     with the complex-gradient convention dL/dRe + i dL/dIm; the batch sum
 *     is done in a fixed order (deterministic).  Nothing from the forward
 *     pass is needed.
 * Pointers: x, y, gy, gx 4-byte aligned; W, gW 8-byte aligned; y (gx) must not
 * alias x or gy.  Same status codes as qft_execute.
 */
int qft_filter_create(qft_plan* out, int64_t n, int64_t batch, int64_t channels, unsigned flags);
int qft_filter_forward(qft_plan plan, const float* x, const void* W, float* y, void* stream);
int qft_filter_backward(qft_plan plan, const float* x, const void* W, const float* gy, float* gx, void* gW,
                        void* stream);

/*
 * qft_execute_static_scratch -- run op (QFT_OP_*) on `batch` C2C FP32 rows of
 * length n, 2^15 <= n <= 2^20, like qft_execute on a QFT_KIND_C2C /
 * QFT_DTYPE_F32 plan (the same bits), but without a plan and without
 * allocating.  The paper has no counterpart: this is a service entry point
 * for callers that cannot allocate device memory at the point of use (all
 * free memory held by another allocator, or a latency-bound loop where
 * cudaMalloc / cudaFree would synchronise the device).  It calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *   in, out  device pointers, [batch][n] complex64, 8-byte aligned; in == out
 *            is allowed.  stream as in qft_execute.
 * Storage: a 64 MiB scratch array, the secant table, the schedules and a
 * status word are file-scope device arrays of the library, reserved when its
 * module loads and shared by every call.  Nothing in the scratch has to start
 * at zero (each call writes every scratch cell before reading it).  Calls
 * whose executions overlap (two streams, or host threads without ordering)
 * race on the scratch: serialise them.  Batches larger than the rows the
 * scratch holds (113 rows at n = 2^15, 29 at 2^16, 7 at 2^18, 1 at 2^20, where the
 * compensated classes also keep their lo parts) run in successive chunks.
 * Set-up: the first call on each device (with that device current) looks up the
 * arrays with cudaGetSymbolAddress and fills the tables with blocking copies;
 * make that first call before any stream capture begins.  The set-up is not
 * repeated after cudaDeviceReset: do not use the entry point across a reset.
 * Errors: QFT_ERR_INVALID_N for n not a power of two or outside [2^15, 2^20]
 * (the limit the static scratch sets); QFT_ERR_INVALID_BATCH, _INVALID_ARG (op,
 * device ordinal >= 64), _NULLPTR, _ALIGN, _CUDA as for qft_execute.  A bounded
 * device-side wait that expired is reported by qft_static_scratch_sync_status.
 */
int qft_execute_static_scratch(int64_t n, int64_t batch, int op, const void* in, void* out, void* stream);

/* Host-blocking status read of qft_execute_static_scratch on the current
 * device: synchronises `stream` and returns the static status word (QFT_OK, or
 * QFT_ERR_TIMEOUT if a bounded wait of a call expired and that call's output is
 * incomplete), then clears it.  Allocates nothing (blocking copies to and from
 * the word); QFT_OK if no call has run on the device.  Paper counterpart: none
 * (the status of the entry point above). */
int qft_static_scratch_sync_status(void* stream);

/* Releases every resource of the plan.  Safe on NULL.  A destroyed plan must
 * not be used again; the library detects most such uses (QFT_ERR_DESTROYED). */
int qft_plan_destroy(qft_plan plan);

/* Host-blocking: synchronises the plan's last stream and returns the plan's
 * device status word (QFT_OK or QFT_ERR_TIMEOUT), then clears it. */
int qft_plan_sync_status(qft_plan plan);

/* Number of classes (per side) whose trees the plan evaluates on compensated
 * FP32 pairs (0 for n < 2^16 or with QFT_PLAN_FP32_PLAIN; ragged plans: the
 * largest over their lengths), or a negative QFT_ERR_* code. */
int qft_plan_comp_classes(qft_plan plan);

/* Limit, in nanoseconds, of the kernels' bounded waits for the input copies they
 * stage in shared memory (default 0 = 2 s).  When a wait expires the kernel
 * records QFT_ERR_TIMEOUT in the plan's status word (qft_plan_sync_status),
 * waits once more with the 2 s limit for its copy in flight and returns; that
 * execute's output is then incomplete.  Single-size plans only
 * (QFT_ERR_INVALID_ARG otherwise, or for ns < 0). */
int qft_plan_set_wait_limit(qft_plan plan, int64_t ns);

/* Test of that failure path (diagnostics, single-size plans): the next execute
 * of the plan arms each CTA's first staging barrier without issuing its copy,
 * so that wait runs out after the wait limit with nothing in flight, the kernel
 * returns early and the status word reads QFT_ERR_TIMEOUT.  Applies to the
 * row kernel when it stages rows and to the NODE kernel of n > 2^14; one shot
 * (cleared by that execute). */
int qft_plan_withhold_next_copy(qft_plan plan);

/* Last CUDA error recorded by the plan (a cudaError_t value, 0 if none). */
int qft_plan_last_cuda_error(qft_plan plan);

/* Bytes of device scratch the plan holds for its transforms (the large-row
 * path's class-data copies, lo parts, C/S tables and halo copies; ragged plans:
 * the sum over their lengths; 0 for n <= 2^14), or a negative QFT_ERR_* code
 * (bytes may be null).  The secant table and the plan's small descriptors are
 * not counted. */
int qft_plan_scratch_bytes(qft_plan plan, int64_t* bytes);

/* Launch geometry chosen for the plan: threads per CTA, CTAs, dynamic shared
 * memory bytes, and the number of kernel launches one execute issues. */
int qft_plan_info(qft_plan plan, int* threads, int* ctas, int* smem_bytes, int* launches);

/* Schedule of a single-size plan (the default, or the one QFT_PLAN_AUTOTUNE
 * chose).  values receives 10 ints: threads per CTA, L1 (levels done while
 * loading), LS (levels per in-place forward phase), LL (forward levels of the
 * leaf tasks, 0 = per class), LB (backward levels per slice phase), LF
 * (class-combine levels per final task), staging allowed (1/0), and for
 * n > 2^14 the node size log2, the node kernel's threads and the rows per
 * launch sequence (fewer rows keep a chunk's scratch copies in L2) (else 0). */
int qft_plan_schedule(qft_plan plan, int* values);

/* Sets the schedule of a single-size plan from the same 10 values (L1 must be
 * the library's 3, LB at most 3; threads and node threads 256 or 512).  Every
 * schedule gives the same results; QFT_ERR_INVALID_N if the planner rejects the
 * combination for this n (the previous schedule is kept), QFT_ERR_INVALID_ARG
 * for ragged or filter plans or out-of-range values. */
int qft_plan_set_schedule(qft_plan plan, const int* values);

/*
 * Launch timing (diagnostics, single-size plans).  qft_plan_time_launches(plan,
 * 1) makes every following execute record a CUDA event pair around each of its
 * kernel launches, on the execute's stream; 0 stops it.  Events are created on
 * demand and owned by the plan.  qft_plan_launch_times synchronises with the
 * recorded events and writes, per kernel kind, the summed milliseconds
 * ms[4] and the number of launches launches[4] since timing was enabled (or
 * since the previous read), then starts a new count.  Kinds: 0 the row kernel
 * (n <= 2^14), 1 the large-row F1 / forward / final kernel, 2 the NODE kernel,
 * 3 the SLICE kernel.  Ragged plans return QFT_ERR_INVALID_ARG.
 */
int qft_plan_time_launches(qft_plan plan, int enable);
int qft_plan_launch_times(qft_plan plan, float* ms, int* launches);

/* Human-readable text of a status code (static storage). */
const char* qft_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* QFT_GB300_H */
