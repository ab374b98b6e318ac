/*
 * fftgb — batched single-precision complex-to-complex FFT for GB300 (sm_103a).
 *
 * C ABI of libfftgb.so.  Plain pointers and sizes only; no C++ or framework
 * types cross this boundary.
 *
 * The transform (paper Sec. II-A): for each of `batch` transforms of length N,
 *     forward  X[k] = sum_{n=0}^{N-1} x[n] W_N^{n k},   W_N = exp(-2 pi i / N),
 *              unnormalised;
 *     inverse  x[n] = (1/N) sum_k X[k] exp(+2 pi i n k / N)
 *              (the paper defines only the forward transform; the inverse is
 *               scaled by 1/N unless FFT_FLAG_UNNORMALIZED_INVERSE is given).
 * It is computed as a Stockham autosort factorisation (Sec. II-B) with
 * register-resident radix-8/16 DIT butterflies and radix-4/2 tails
 * (Sec. V-A, V-B), shared-memory exchange between passes, precomputed
 * twiddle tables, and a four-step decomposition (Sec. IV-B, Eq. 3) for large N.
 *
 * Data layout (all entry points unless stated otherwise): interleaved complex
 * float32 (`float2`: re, im), transform-major: element n of transform b is at
 * index b*N + n.  Device buffers are owned by the caller, must be 16-byte
 * aligned, and must not overlap partially; in == out (in place) is allowed.
 *
 * Asynchrony: every exec call enqueues work on the caller's CUDA stream
 * (`stream` is a cudaStream_t; NULL means the legacy default stream) and
 * returns without synchronising.  Errors detected on the host are returned
 * immediately; errors raised by kernels are recorded in a per-plan device
 * status word read by fft_last_device_status() after a synchronisation.
 *
 * Thread safety: a plan may be executed from one host thread at a time;
 * different plans are independent.
 */
#ifndef FFTGB_H_
#define FFTGB_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fft_plan_s *fft_plan_t;

/* The value is the sign of the exponent of the transform kernel. */
typedef enum { FFT_FORWARD = -1, FFT_INVERSE = 1 } fft_direction_t;

typedef enum {
    FFT_PREC_FP32 = 0,    /* FP32 data and arithmetic (the plain path)        */
    FFT_PREC_FP16X2 = 1,  /* tensor-core radix-16 DFT, FP16 hi+lo operands     */
    FFT_PREC_BF16X2 = 2,  /* tensor-core radix-16 DFT, BF16 hi+lo operands     */
    FFT_PREC_FP16_STORAGE = 3, /* data in HBM as FP16 (re, im) pairs, 4 bytes per
                               point; FP32 arithmetic; output rounded to FP16
                               (overflow to infinity: the caller keeps
                               |X| below 65504).  N in [256, 16384].          */
    FFT_PREC_BF16_STORAGE = 4  /* data in HBM as BF16 (re, im) pairs, 4 bytes per
                               point; FP32 arithmetic; output rounded to BF16
                               (FP32 range, 8 significant bits).
                               N in [256, 16384].                             */
} fft_precision_t;

typedef enum {
    FFT_OK = 0,
    FFT_ERR_INVALID_SIZE = 1,   /* N not a supported power of two, batch < 0   */
    FFT_ERR_INVALID_VALUE = 2,  /* bad handle, direction, flag or overlap      */
    FFT_ERR_MISALIGNED = 3,     /* a pointer is not 16-byte aligned            */
    FFT_ERR_ALLOC = 4,          /* device or host allocation failed            */
    FFT_ERR_CUDA = 5,           /* a CUDA runtime call failed                  */
    FFT_ERR_TIMEOUT = 6,        /* a bounded device-side wait ran out          */
    FFT_ERR_NOT_SUPPORTED = 7   /* valid request the library does not implement */
} fft_status_t;

/* Plan flags (bitwise OR). */
#define FFT_FLAG_UNNORMALIZED_INVERSE 0x1 /* inverse without the 1/N factor    */
#define FFT_FLAG_FORCE_SINGLE_CTA 0x2     /* whole transform inside one CTA    */
#define FFT_FLAG_FORCE_FOURSTEP 0x4       /* two-phase four-step through L2/HBM */
#define FFT_FLAG_NO_AUTOTUNE_CACHE 0x8    /* ignore the autotuner's choices     */
/* Plan the ADJOINT of the `direction` transform instead of the transform:
 * adjoint(forward F) = F^H, the unnormalised conjugate-sign transform;
 * adjoint(inverse G = F^H / N) = F / N.  The backward pass of a layer that
 * applies F (or G) applies this plan to the incoming gradient. */
#define FFT_FLAG_ADJOINT 0x10
/* fft_ragged_plan only: time every compiled routine of each class (N,
 * direction) of the batch on that class's rows and use the fastest; the
 * choices are kept in a process-wide cache that later ragged plans use
 * (unless they pass FFT_FLAG_NO_AUTOTUNE_CACHE). */
#define FFT_FLAG_RAGGED_AUTOTUNE 0x20

/* Execution paths reported by fft_plan_info(). */
#define FFT_PATH_SINGLE_CTA 1  /* Stockham, every pass inside one CTA        */
#define FFT_PATH_FOURSTEP 2    /* column FFTs + twiddle, then row FFTs        */
#define FFT_PATH_RAGGED 3      /* ragged batch: one persistent launch         */
#define FFT_PATH_TENSORCORE 4  /* split-precision tensor-core radix-16 DFT    */
#define FFT_PATH_FILTER 5      /* fused spectral filter (fft_filter_plan)     */
#define FFT_PATH_COLUMNS 6     /* strided column transforms (fft_plan_columns) */
#define FFT_PATH_TMEM_HALVES 7 /* N = 32768 in one HBM pass: a radix-2 split into
                                  two 16384-point halves on one SM, one half held
                                  in tensor memory while the other transforms    */

/* What a plan chose; filled by fft_plan_info(). */
typedef struct {
    int N;            /* transform length (0 for a ragged plan)                */
    int64_t batch;    /* transforms per exec (count for a ragged plan)         */
    int direction;    /* FFT_FORWARD / FFT_INVERSE (0 = mixed, ragged)         */
    int precision;    /* fft_precision_t                                       */
    int path;         /* FFT_PATH_*                                            */
    int points_per_thread;  /* registers of complex data per thread per pass  */
    int transforms_per_cta; /* transforms sharing one CTA (single-CTA path)   */
    int threads_per_cta;
    int num_passes;         /* exchange passes of the (first) kernel          */
    int radix[8];           /* radix of each pass, first pass first           */
    int n1, n2;             /* four-step split N = n1 * n2, or a column plan's
                               two-launch split L = n1 * n2 (0 otherwise)     */
    int64_t scratch_bytes;  /* device scratch owned by the plan               */
    int twiddle_mode;       /* as in fft_config_t                              */
    int grid_ctas;          /* CTAs launched per exec (0 = one per tile)      */
    int tma_slabs;          /* as in fft_config_t                              */
    int cluster_split;      /* as in fft_config_t                              */
    int l2_chunk_rows;      /* as in fft_config_t                              */
} fft_plan_info_t;

/* One compiled execution configuration (see fft_list_configs). */
typedef struct {
    int path;               /* FFT_PATH_SINGLE_CTA, FFT_PATH_FOURSTEP or
                               FFT_PATH_TMEM_HALVES (N = 32768)                 */
    int points_per_thread;  /* complex points each thread keeps in registers    */
    int transforms_per_cta; /* rows per CTA (single-CTA path)                    */
    int threads_per_cta;
    int num_passes;
    int radix[8];           /* radix schedule of the (first) kernel              */
    int n1;                 /* four-step: N = n1 * (N / n1); 0 otherwise         */
    int twiddle_mode;       /* 0: every twiddle read from its table; 1: W^k and
                               W^{4k} (W^{16k}) read, the rest formed as products */
    int ctas_per_sm;        /* 0: one CTA per tile; -1: persistent grid at full
                               occupancy with L2 prefetch of the next tile;
                               k > 0: persistent with k CTAs per SM             */
    int tma_slabs;          /* > 0: TMA-staged persistent kernel keeping this many
                               slabs of the next row in a shared-memory ring;
                               0: pass 0 loads straight from global memory      */
    int cluster_split;      /* K = 2, 4, 8: each row on a cluster of K CTAs, each
                               transforming an N/K-point part, combined through
                               distributed shared memory (persistent clusters,
                               one HBM pass; N up to 131072); 0: one CTA per row */
    int l2_chunk_rows;      /* four-step with n1 == n2 only.  > 0: both phases in
                               one persistent launch; rows are cut into chunks of
                               this many rows whose intermediate stays in a ring
                               of L2-sized scratch slots (HBM traffic 16 N B per
                               row instead of 32 N B); 0: two launches through
                               a scratch copy of the whole batch               */
} fft_config_t;

/* Human-readable name of a status code (static string, never NULL).
 * Paper: Sec. II-A (the problem statement whose calls these codes report on;
 * the paper defines no error reporting). */
const char *fft_status_string(fft_status_t status);

/*
 * fft_plan — plan `batch` transforms of length N in one direction.
 * N: power of two, 2 <= N <= 2^20.  Up to 16384 a row fits one CTA.  At
 * 32768 a row still crosses HBM once (path FFT_PATH_TMEM_HALVES: a radix-2
 * decimation-in-frequency split into two 16384-point halves on one SM, one
 * half held in tensor memory while the other transforms; one persistent
 * 512-thread CTA per SM).  Above that the two-phase four-step runs
 * (N = n1 * n2 with a phase-1 length n2 of 256 up to 2^17 and 512 above,
 * and a phase-2 length n1 <= 4096; its intermediate doubles the HBM
 * traffic).  Rows on
 * thread-block clusters (cluster_split in fft_config_t, N = 8192 .. 65536)
 * and the four-step at 32768 are selectable through fft_plan_config.
 * batch >= 0 (0 makes a valid plan whose
 * exec does nothing).  direction: FFT_FORWARD or FFT_INVERSE.
 * Allocates and fills the plan's twiddle tables on the current device
 * (generated in FP64 on the GPU, rounded to FP32) and synchronises once.
 * On success *out holds a plan to free with fft_destroy(); on failure *out is
 * set to NULL.
 * Paper: Sec. II-A (the batched transform, fft_plan(N, batch, direction));
 * Sec. IV-D (synthesis rules) decides the factorisation; the radix schedule
 * follows Sec. V-B/V-D.
 */
fft_status_t fft_plan(fft_plan_t *out, int N, int64_t batch, int direction);

/* As fft_plan with a precision (fft_precision_t) and FFT_FLAG_* flags
 * (N > 16384: FP32 only, FFT_FLAG_FORCE_SINGLE_CTA is FFT_ERR_NOT_SUPPORTED).
 * The tensor-core precisions support N in {256, 4096, 16384} only
 * (FFT_ERR_NOT_SUPPORTED otherwise).
 * Paper: Sec. II-A (the transform); Sec. V-C, Eqs. 5-6 (the DFT block as a
 * real matrix product: FFT_PREC_FP16X2 / BF16X2); Sec. IX-A (mixed precision
 * for radar data: the 16-bit storage precisions); Sec. IV-B, Eq. 3
 * (FFT_FLAG_FORCE_FOURSTEP). */
fft_status_t fft_plan_ex(fft_plan_t *out, int N, int64_t batch, int direction,
                         int precision, int flags);

/*
 * fft_list_configs — enumerate the FP32 execution configurations compiled
 * into this library for length N: every single-CTA Stockham variant (radix
 * schedule, points per thread, transforms per CTA), every cluster
 * configuration (cluster_split K, N = 8192 .. 65536), the tensor-memory
 * halves at 32768 (path FFT_PATH_TMEM_HALVES; radix: the 16384-point
 * schedule of each half) and every four-step split.
 * Writes min(count, capacity) entries to out (out may be NULL) and returns
 * the total count (0 for an unsupported N).
 * Paper: Sec. IV-C (radix selection) and Sec. V-D (the per-size kernel
 * configurations, Table of multi-size kernels) -- the space the autotuner
 * searches.
 */
int fft_list_configs(int N, fft_config_t *out, int capacity);

/*
 * fft_plan_config — plan with one explicit configuration from
 * fft_list_configs (used by the autotuner and by tests that cover every
 * configuration).  flags as in fft_plan_ex, except the FORCE_* flags.
 * FFT_ERR_NOT_SUPPORTED if the configuration is not compiled in.
 * Paper: Sec. V-D (one explicit kernel configuration per size).
 */
fft_status_t fft_plan_config(fft_plan_t *out, int N, int64_t batch, int direction,
                             int flags, const fft_config_t *config);

/*
 * fft_exec — run the plan on device buffers.
 * in, out: device pointers to batch*N float2 each (see layout above; batch*N
 * FP16 or BF16 pairs, 4 bytes each, for FFT_PREC_FP16_STORAGE or
 * FFT_PREC_BF16_STORAGE), 16-byte
 * aligned; in == out is allowed, partial overlap is FFT_ERR_INVALID_VALUE.
 * For a ragged plan, in and out are the packed base pointers the plan's
 * offsets index.  stream: cudaStream_t or NULL.  Asynchronous.
 * Stream order holds as for any launch: the single-CTA, filter and
 * (up to 2048-point) column kernels use programmatic dependent launch, so
 * their CTAs may become resident while the previous kernel of the stream
 * finishes, but they read and write nothing before it has completed.
 * Paper: Sec. II-A (fft_exec(plan, in, out, stream) over the DFT defined
 * there); Sec. II-B (Stockham autosort: natural-order output).
 */
fft_status_t fft_exec(fft_plan_t plan, const void *in, void *out, void *stream);

/*
 * fft_exec_host — the same transform on HOST buffers: the library copies the
 * input to device memory it owns, runs the plan and copies the result back,
 * pipelining the copies with the transforms in chunks.  Blocks until the
 * result is in host_out.  Page-locked (pinned) host memory gives full copy
 * bandwidth; pageable memory works but is slower.  Not for ragged plans.
 * Paper: Sec. II-A (the same transform; the host copies stand in for the
 * unified memory of Sec. III-A, which a discrete GPU does not have).
 */
fft_status_t fft_exec_host(fft_plan_t plan, const void *host_in, void *host_out,
                           void *stream);

/* Free a plan and all device memory it owns.  NULL is accepted.
 * Paper: Sec. II-A (the plan of the problem statement). */
fft_status_t fft_destroy(fft_plan_t plan);

/* Describe what a plan chose (path, radix schedule, threads, split).
 * Paper: Sec. IV-D (synthesis rules) and Sec. V-D (kernel configurations):
 * what the planner chose for the problem of Sec. II-A. */
fft_status_t fft_plan_info(fft_plan_t plan, fft_plan_info_t *info);

/*
 * Read and clear the plan's device status word.  Synchronises the device.
 * Returns FFT_OK, or the first error a kernel recorded (FFT_ERR_TIMEOUT for a
 * bounded wait that ran out).
 * Paper: Sec. II-A (reports on the execution of the problem statement's
 * transform; the paper defines no device error reporting).
 */
fft_status_t fft_last_device_status(fft_plan_t plan);

/*
 * fft_twiddle_table — copy the plan's FP32 twiddle table to host memory
 * (for inspection and tests).  *count receives the number of complex entries;
 * if host_out is non-NULL, min(*count, capacity) entries are copied.
 * Each entry is W_M^e = exp(-2 pi i e / M) for the (M, e) that
 * fft_twiddle_index() reports for the same position.
 * Paper: Sec. V-A and V-B (the twiddle factors W of each pass; here
 * precomputed in FP64 and rounded to FP32 instead of sincos chains).
 */
fft_status_t fft_twiddle_table(fft_plan_t plan, void *host_out, int64_t capacity,
                               int64_t *count);
/* Position -> (M, e) of the twiddle table entry.
 * Paper: Sec. V-A and V-B (as fft_twiddle_table). */
fft_status_t fft_twiddle_index(fft_plan_t plan, int64_t pos, int64_t *M, int64_t *e);

/*
 * fft_ragged_plan — a batch of `count` transforms of mixed lengths and
 * directions, executed in ONE persistent launch: one 512-thread CTA per SM
 * claims work units longest N first through a device counter; a unit fills
 * the CTA (512 P / N rows of one (N, direction), N / P threads each, P = 16
 * or 32 points per thread).
 * N[i]: power of two in [16, 16384] (2..8 give FFT_ERR_NOT_SUPPORTED);
 * direction[i]: -1 or +1;
 * in_offset[i], out_offset[i]: start of transform i, in complex elements,
 * inside the packed buffers passed to fft_exec(); every offset must be a
 * multiple of 2 (16-byte alignment).  Host arrays are copied; the caller keeps
 * ownership.  flags: FFT_FLAG_UNNORMALIZED_INVERSE; FFT_FLAG_RAGGED_AUTOTUNE
 * (time the compiled routines of each class on its rows now and use the
 * fastest, remembered for later ragged plans); FFT_FLAG_NO_AUTOTUNE_CACHE
 * (ignore remembered choices: built-in routines).  fft_ragged_class_config
 * reports each class's routine.  fft_exec replays a CUDA graph (counter
 * reset + the one kernel) captured for the (in, out) pair; a new pair
 * re-captures.
 * Paper: Sec. II-D (batched radar FFTs; here with mixed lengths).
 */
fft_status_t fft_ragged_plan(fft_plan_t *out, int count, const int *N,
                             const int *direction, const int64_t *in_offset,
                             const int64_t *out_offset, int flags);

/* The routine a ragged plan runs for its class (N, direction): points per
 * thread, radix schedule, twiddle mode, rows per unit (transforms_per_cta),
 * threads_per_cta (512) and path FFT_PATH_RAGGED.  FFT_ERR_INVALID_VALUE if
 * the plan is not ragged or holds no transform of that class.
 * Paper: Sec. IV-C (radix selection) and Sec. V-D (per-size kernel
 * configuration), per class of the Sec. II-D batch. */
fft_status_t fft_ragged_class_config(fft_plan_t plan, int N, int direction,
                                     fft_config_t *config);

/* The routines compiled for class N of a ragged batch (path
 * FFT_PATH_RAGGED), as fft_list_configs does for plain plans; returns the
 * total count and writes min(count, capacity) entries to out (may be NULL).
 * Paper: Sec. IV-C (radix selection) and Sec. V-D (per-size kernel
 * configurations). */
int fft_ragged_list_configs(int N, fft_config_t *out, int capacity);
/* Make `config` (one of fft_ragged_list_configs(N)) the remembered routine
 * for class (N, direction) of later ragged plans, as the autotuner would;
 * fft_autotune_clear forgets it.  FFT_ERR_NOT_SUPPORTED if not compiled in.
 * Paper: Sec. V-D (one explicit kernel configuration per size). */
fft_status_t fft_ragged_choose(int N, int direction, const fft_config_t *config);

/*
 * fft_autotune — time the candidate configurations (points per thread, radix
 * schedule, transforms per CTA, single-CTA vs four-step) for (N, direction,
 * precision) on the current device with a batch of `batch` transforms, and
 * store the fastest in the process-wide cache used by later plans.  If
 * cache_path is non-NULL the whole cache is also written there as JSON
 * (keyed by GPU name, N, direction, precision).  Allocates its own buffers.
 * Paper: Sec. IV-C (radix selection) and Sec. V-D (the kernel-selection
 * table per size), chosen here by measurement on the current GPU.
 */
fft_status_t fft_autotune(int N, int direction, int precision, int64_t batch,
                          const char *cache_path);
/* Load a JSON cache written by fft_autotune (entries for other GPUs are
 * ignored).  A missing file is FFT_ERR_INVALID_VALUE.
 * Paper: Sec. V-D (as fft_autotune). */
fft_status_t fft_autotune_load(const char *cache_path);
/* Forget every autotuned choice, plain and ragged (plans fall back to the
 * built-in table).
 * Paper: Sec. V-D (as fft_autotune). */
fft_status_t fft_autotune_clear(void);

/*
 * Spectral-filter building blocks (SAR range compression, paper Sec. II-D and
 * the fused pipeline of Sec. IX-A), for y = IFFT(FFT(x) * H).
 *
 * fft_filter_apply: Z[b][k] = X[b][k] * H[k] (conj_h = 0) or
 *   X[b][k] * conj(H[k]) (conj_h = 1), elementwise, for batch rows of N
 *   points; Z may alias X.  scale multiplies the result (exact for powers of 2).
 * fft_filter_grad_h: grad_H[k] = sum_b conj(X[b][k]) * G[b][k], accumulated in
 *   FP32 in 32-row chunks and a fixed-order pairwise tree (bitwise
 *   reproducible); `work` must hold fft_filter_grad_h_workspace(N, batch)
 *   bytes.
 * All pointers are device pointers, 16-byte aligned (8 for grad_h); all
 * calls are asynchronous on stream.
 * Paper: Sec. II-D (range compression as a matched filter in the frequency
 * domain) and Sec. IX-A (the fused FFT / matched-filter pipeline).
 */
fft_status_t fft_filter_apply(const void *X, const void *H, void *Z, int N,
                              int64_t batch, int conj_h, float scale, void *stream);
int64_t fft_filter_grad_h_workspace(int N, int64_t batch);
fft_status_t fft_filter_grad_h(const void *X, const void *G, void *grad_H, int N,
                               int64_t batch, void *work, void *stream);

/*
 * Fused spectral filter: the forward FFT, the multiplication by H and the
 * inverse FFT of a row run in ONE kernel with the row in registers (after a
 * Stockham transform each thread already holds the points the next
 * transform's first pass reads), so a row crosses HBM once each way.
 *
 * fft_filter_plan: plan for `batch` rows of N points, N power of two in
 *   [256, 16384] (FFT_ERR_NOT_SUPPORTED otherwise).  Owns the twiddle tables
 *   and the backward pass's grad_H workspace (one row of sums per 32 rows).
 *   Free with fft_destroy.
 * fft_filter_forward: y = IFFT(FFT(x) * H) (conj_h = 1: * conj(H)), inverse
 *   scaled by 1/N; if X_save is non-NULL it also receives FFT(x) (needed by
 *   the backward).  x, y, X_save: batch*N float2; H: N float2.  y may equal
 *   x; X_save may not overlap x or y (FFT_ERR_INVALID_VALUE).  One kernel,
 *   one HBM read and one write per point of y (plus X_save).
 * fft_filter_backward: with g_y = dL/dy (PyTorch convention),
 *   grad_x = IFFT(FFT(g_y) * conj(H)) = F^H(conj(H) * g_z), g_z = FFT(g_y)/N,
 *   grad_H = sum_rows conj(X_saved) * g_z  (per-block sums over fixed row
 *   sets in row order, then a fixed-order pairwise tree: bitwise
 *   reproducible on a given GPU).  N >= 8192: one kernel (its grad_H partial
 *   sums in tensor memory) and the tree; N <= 4096: three kernels (g_z into
 *   grad_x's buffer, the grad_H reduction over 32-row chunks, then grad_x in
 *   place).  grad_x may not overlap g_y or X_saved
 *   (FFT_ERR_INVALID_VALUE).
 * Device pointers, 16-byte aligned; asynchronous on stream.
 * Paper: Sec. IX-A (FFT fused with matched filtering in one kernel) and
 * Sec. II-D (SAR range compression).
 */
fft_status_t fft_filter_plan(fft_plan_t *out, int N, int64_t batch);
fft_status_t fft_filter_forward(fft_plan_t plan, const void *x, const void *H, void *y,
                                void *X_save, int conj_h, void *stream);
fft_status_t fft_filter_backward(fft_plan_t plan, const void *g_y, const void *H,
                                 const void *X_saved, void *grad_x, void *grad_H,
                                 void *stream);

/*
 * fft_filter_step: one training step of the spectral filter under the
 * masked-energy loss L = sum_{rows, k} mask * |y|^2 (mask real, one float per
 * point), forward and backward fused.  One persistent kernel computes, per
 * row: X = FFT(x); y = IFFT(X * H); the row's share of L; g_y = 2 mask y;
 * g_z = FFT(g_y) / N; the grad_H partial sums conj(X) * g_z (in tensor
 * memory); grad_x = F^H (conj(H) * g_z).  X and g_y never leave the SM, so
 * a row moves 28 bytes per point (read x and mask, write y and grad_x).
 * Then grad_H is summed over the CTAs by the same fixed-order tree as the
 * backward's, and L over the CTAs in a fixed order in FP64 (both bitwise
 * reproducible on a given GPU).
 * plan: from fft_filter_plan (N = 256..16384; below 8192 the kernel takes
 *   TB = 4096 / N rows per CTA and adds its rows' sums before the tree).
 *   x, y, grad_x: batch*N float2; mask: batch*N float; H,
 *   grad_H: N float2; loss: one float.  y may be NULL (not stored).  y and
 *   grad_x may each equal x (a row is read before it is written) but may not
 *   overlap anything else; mask, H, grad_H and loss may not overlap y or
 *   grad_x (FFT_ERR_INVALID_VALUE).  Device pointers, 16-byte aligned (loss:
 *   4-byte); asynchronous on stream.  batch 0: grad_H and loss are zeroed.
 * The same results as fft_filter_forward, g_y = 2 mask y computed apart,
 * and fft_filter_backward (to rounding).
 * Paper: Sec. IX-A (FFT fused with matched filtering in one kernel) and
 * Sec. II-D (SAR range compression); the loss and the backward pass have no
 * counterpart in the paper.
 */
fft_status_t fft_filter_step(fft_plan_t plan, const void *x, const void *H, const float *mask,
                             void *y, void *grad_x, void *grad_H, float *loss, void *stream);

/*
 * fft_plan_columns — transforms down the columns of strided matrices without
 * a transpose: the azimuth pass (corner turn) of SAR processing over a
 * [azimuth, range] matrix stored range-contiguous (paper Sec. II-D, range and
 * azimuth compression as batched 1-D FFTs; Sec. IX-A).  Element (m, r, c) of
 * matrix m, row r (the transform index, 0 <= r < L) and column c (0 <= c <
 * ncols) is at complex offset m * mat_stride + r * row_stride + c from the
 * buffer pointer, for input and output alike; each of the nmat * ncols
 * columns gets an L-point transform (W_L = e^{-2 pi i / L}, forward
 * unnormalised, inverse scaled by 1/L unless FFT_FLAG_UNNORMALIZED_INVERSE).
 * L: power of two in [16, 2^21].  ncols: a multiple of the kernel's column
 * tile (16 for L <= 512 and for L > 4096, 8 for 1024 and 2048, 4 for 4096),
 * else FFT_ERR_INVALID_SIZE.
 * row_stride >= ncols and < 2^31; mat_stride >= (L - 1) * row_stride + ncols
 * (matrices do not overlap); nmat >= 0 (0: exec does nothing).  Execute with
 * fft_exec(plan, in, out, stream): device pointers, 8-byte aligned, in == out
 * allowed, any other overlap of the two extents is FFT_ERR_INVALID_VALUE;
 * fft_exec_host is FFT_ERR_NOT_SUPPORTED.  Up to L = 2048 a column is one
 * tile in one CTA, read whole before it is written, so the in-place
 * transform is safe.  L = 4096 runs as the two launches below when ncols is a
 * multiple of 16, else as one launch of 4-column tiles.  flags may add
 * FFT_FLAG_FORCE_SINGLE_CTA (one launch; L <= 4096) or FFT_FLAG_FORCE_FOURSTEP
 * (two launches; L >= 2048), else FFT_ERR_NOT_SUPPORTED.
 * L > 4096 (a long aperture): the four-step factorisation of paper Sec. IV-B
 * (Eq. 3) down the column, L = n1 n2 with n2 = min(512, 2^ceil(log2(L)/2)):
 * one launch of n2-point column FFTs over the n1 interleaved sub-matrices
 * (rows j, j + n1, ...), each output row k2 times W_L^{j k2}, into a
 * plan-owned scratch, then one launch of n1-point column FFTs from the
 * scratch to the output, row k2 + n2 k1.  n1 * max(row_stride, ncols) and
 * n2 * row_stride must stay below 2^31 (else FFT_ERR_INVALID_SIZE).  The
 * scratch holds min(nmat, max(1, 2^30 / (8 L ncols))) matrices
 * (fft_plan_info: scratch_bytes, n1, n2); more matrices run as several such
 * pairs of launches.  in == out stays allowed (the input is read whole before
 * the output is written); executions of one plan may not overlap in time.
 * Paper: Sec. II-D (azimuth compression as batched 1-D FFTs over the other
 * matrix dimension) and Sec. IX-A (the corner turn).
 */
fft_status_t fft_plan_columns(fft_plan_t *out, int L, int64_t ncols, int64_t nmat,
                              int64_t row_stride, int64_t mat_stride, int direction,
                              int flags);

/*
 * fft_fourstep_noalloc — the two-phase four-step transform (same kernels,
 * tables and results, bit for bit, as a plan made with
 * FFT_FLAG_FORCE_FOURSTEP) for callers that must not allocate device memory.  The paper has no counterpart: this entry
 * point exists for users of the library whose code may not call cudaMalloc
 * while it runs, e.g. a real-time pipeline whose memory is fixed at start-up
 * or code that hands the device heap to its own allocator.  It takes no plan
 * (making a plan allocates) and allocates nothing: its intermediate lives in
 * a fixed file-scope device array of FFT_NOALLOC_MAX_POINTS complex values
 * (16 MiB) and its twiddle tables in another (512 KiB); both are reserved on
 * every GPU that loads the library until the process exits.
 * in, out: device pointers to batch*N float2 (layout as above), 16-byte
 * aligned; in == out allowed.  N: power of two in [256, 16384].
 * N * batch above FFT_NOALLOC_MAX_POINTS is FFT_ERR_INVALID_SIZE (split
 * larger batches into several calls).  direction: FFT_FORWARD or
 * FFT_INVERSE (inverse scaled by 1/N).  Asynchronous on `stream`.
 * The first call on a device sets that device up (resolves the arrays'
 * addresses, fills the tables, synchronises the device): make it before any
 * stream capture.  The set-up belongs to the device's context: after
 * cudaDeviceReset the next call sets the device up again (same rule).  All calls share the one scratch array, which keeps the
 * last call's contents; calls whose work overlaps on the GPU race with each
 * other, so serialise them (e.g. one stream).
 */
#define FFT_NOALLOC_MAX_POINTS 2097152
fft_status_t fft_fourstep_noalloc(const void *in, void *out, int N, int64_t batch,
                                  int direction, void *stream);

/*
 * Failure injection, for tests of the library's error paths (no GPU fault,
 * trap or hang is ever made).  The paper has no counterpart: the paper
 * reports no error handling; these calls let a test reach the failures that
 * a healthy GPU never produces.
 *
 * fft_debug_fail_alloc — the next `after` device allocations the library
 * makes succeed and the one after them fails as an out-of-memory cudaMalloc
 * would (nothing is allocated, no sticky CUDA error is left); the call that
 * made it returns FFT_ERR_ALLOC and frees what it had allocated.  after < 0
 * disarms.  Process-wide (all threads and devices); not for production use.
 */
void fft_debug_fail_alloc(int after);

/*
 * fft_debug_bounded_wait — run one of the kernels' bounded device waits on
 * something that never arrives, with a limit of limit_us microseconds
 * (1 .. 1000000): kind 0 the mbarrier wait of the bulk-copy kernels (a
 * barrier expecting one arrival), kind 1 the counter wait of the
 * single-launch four-step (a counter nobody increments).  The waiting thread
 * gives up after the limit, records FFT_ERR_TIMEOUT in a device status word
 * and returns; the call synchronises `stream` and returns that status
 * (FFT_ERR_TIMEOUT), after which the context stays usable.  Allocates and
 * frees 8 bytes.  FFT_ERR_INVALID_VALUE for another kind or limit.  The
 * paper has no counterpart (failure injection, as above).
 */
fft_status_t fft_debug_bounded_wait(int kind, int limit_us, void *stream);

/*
 * Bounds-checking debug build (the library compiled with FFTGB_BOUNDS_CHECK,
 * e.g. build.build(debug=True)); the product build has no checks.  In the
 * single-CTA Stockham kernels every global load and store (row in the batch,
 * index in the row), pass-table read and exchange-buffer access checks its
 * index; a check that fails records a site number and skips its access, so a
 * wrong index is reported, never faulted on.  The paper has no counterpart
 * (it is the library's substitute for a memory checker).
 * fft_debug_bounds_status — synchronises the device and returns the first
 * failed site since the last call (0: none; the record is cleared), -1 in
 * the product build, -2 on a CUDA error.
 * fft_debug_bounds_selftest — fails one check on purpose (site 99; nothing
 * is accessed) on `stream` and synchronises; FFT_ERR_NOT_SUPPORTED in the
 * product build.  The paper has no counterpart.
 */
int fft_debug_bounds_status(void);
fft_status_t fft_debug_bounds_selftest(void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FFTGB_H_ */
