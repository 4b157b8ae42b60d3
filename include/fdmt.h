/*
 * fdmt.h -- C ABI of the GB300 (sm_103a) Fast Dispersion Measure Transform.
 *
 * The transform is the FDMT of Zackay & Ofek, "An accurate and efficient
 * algorithm for detection of radio bursts with an unknown dispersion measure"
 * (arXiv:1411.5373), section 4 and Algorithm 1.  Given an intensity matrix
 * I[f][t] (Nf channels, Nt samples, channel 0 at the lowest frequency f_min,
 * t contiguous in memory -- section 4.2 "Memory access") it returns
 *
 *     A[d][t] = sum over the discretised dispersion curve of total delay d
 *               (samples across the whole band) that reaches f_min at t
 *                                                 (section 4, Eq. parametrization)
 *
 * for d = 0 .. Nd-1 and t = 0 .. Nt-1, with samples before t = 0 taken as
 * zero (the paper's copy rule).  The curve is fixed by the paper's addition
 * rule: each band [f0, f2] splits at its border frequency f1 and the lower
 * half takes row dl = floor(C * Dt + 1/2) with C from Eq. (C_{f2,f0}); the
 * upper half takes row Dt - dl, dl samples earlier.  Channels are intervals
 * [f_min + k df, f_min + (k+1) df], df = (f_max - f_min) / Nf (section 4).
 *
 * Conventions for every function below:
 *   - Every call returns an int status (enum fdmt_status); FDMT_OK is 0.
 *   - "device pointer" means memory the calling process allocated on the
 *     current CUDA device (cudaMalloc / torch); the library never frees it.
 *   - "stream" is a cudaStream_t passed as void*; NULL means the legacy
 *     default stream.  All device work of a call is enqueued on it; calls
 *     return without waiting unless stated.
 *   - Nothing allocates device memory except fdmt_plan (its delay tables).
 *     Execution needs a caller-owned workspace (fdmt_workspace_bytes).
 *   - A plan is immutable after creation and may be used from several
 *     streams at once if each call has its own workspace.
 *   - Asynchronous kernel failures surface as FDMT_ERR_CUDA on the next call
 *     that checks the CUDA error state.
 */
#ifndef FDMT_GB300_H
#define FDMT_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fdmt_plan_s *fdmt_plan_t;

enum fdmt_status {
  FDMT_OK = 0,
  FDMT_ERR_INVALID_ARG = -1,   /* a value, pointer, alignment or size is wrong */
  FDMT_ERR_UNSUPPORTED = -2,   /* valid request outside this build (e.g. a shape no fused cone fits) */
  FDMT_ERR_CUDA = -3,          /* a CUDA runtime call or launch failed */
  FDMT_ERR_NO_MEMORY = -4,     /* fdmt_plan could not allocate its tables */
  FDMT_ERR_TIMEOUT = -5,       /* a bounded device wait gave up */
  FDMT_ERR_WORKSPACE = -6      /* workspace missing or smaller than required */
};

/* Element types: input -> intermediate state -> output. */
enum fdmt_dtype {
  FDMT_U8_I32 = 0,        /* uint8 in, int32 state and out: exact integer sums */
  FDMT_F32_F32 = 1,       /* float32 in, state and out; fixed association:
                             init row j = row j-1 + I[t-j], one add per merge */
  FDMT_F32_F16STATE = 2   /* float32 in and out; every stored intermediate state
                             is rounded to IEEE fp16, every add is fp32 */
};

/* Plan flags (bitwise or). */
enum fdmt_flags {
  FDMT_PLAN_HOST_ONLY = 1u << 0,  /* build the tables on the host only: no device
                                     memory, no CUDA call; execute is refused.
                                     For inspecting tables without a GPU. */
  FDMT_SCHED_PLAIN = 0u,          /* schedule: one launch per level (default) */
  FDMT_SCHED_FUSED = 1u << 4      /* schedule: several merge levels per launch; each
                                     block stages the level-lb rows of one cone (a
                                     band's row range and its sub-bands' windows)
                                     for one time tile in shared memory by TMA and
                                     computes the levels above it there; the level
                                     grouping and tile are chosen at plan time */
};

/*
 * fdmt_plan -- build the delay tables for one transform shape
 * (Algorithm 1: C_{f2,f0} and Dt_max per band are fixed before the
 * computation, section 4 "this decision can be made prior to the computation").
 *
 *   f_min, f_max  band edges, any unit (only ratios of f^-2 enter, Eq. DtD);
 *                 need 0 < f_min < f_max, both finite.
 *   nf            channels, >= 2.  Not a power of two: the unequal split of
 *                 section 4.2 (band b of level l spans channels
 *                 [b 2^l, min((b+1) 2^l, nf)), split at the border after
 *                 2^(l-1) channels; a band with nothing above that border is
 *                 passed up unchanged), in every schedule and batch mode.
 *   nt            samples per channel, 1 <= nd <= nt, and nt * (input
 *                 element size) and nt * (state element size) multiples of
 *                 16 bytes (vector loads; else FDMT_ERR_INVALID_ARG).
 *   nd            output delay rows (the paper's N_Delta), >= 1.
 *   dtype         enum fdmt_dtype.
 *   flags         enum fdmt_flags.
 *   out           receives the plan handle (NULL on failure).
 *
 * Allocates and uploads the device tables unless FDMT_PLAN_HOST_ONLY.
 * Tables are FP64 arithmetic rounded to int32; the GPU never sees a float
 * delay.  Errors: INVALID_ARG, UNSUPPORTED, NO_MEMORY, CUDA.
 */
int fdmt_plan(double f_min, double f_max, int32_t nf, int64_t nt, int32_t nd,
              int32_t dtype, uint32_t flags, fdmt_plan_t *out);

/* Schedule parameters for fdmt_plan_ex (fused schedule only). */
typedef struct fdmt_schedule_params {
  int32_t tile;         /* time-tile width in samples, a multiple of 64; 0 = chosen */
  int32_t smem_budget;  /* shared memory per block in bytes (<= 227 KiB); 0 = 112 KiB */
  int32_t n_bounds;     /* 0 = level grouping chosen; else the number of entries of */
  int32_t bounds[32];   /* level boundaries 0 = b0 < b1 < ... < b_{n-1} = log2(nf) */
  int32_t group_tile[32];    /* with bounds: tile of launch i (levels b_i..b_{i+1}); 0 = tile */
  int32_t group_budget[32];  /* with bounds: shared memory of launch i; 0 = smem_budget */
  int32_t staging;      /* how staged rows are copied: 0 = row blocks where nt allows
                           (nt a multiple of 128 bytes' worth of samples; 64 samples for
                           uint8), else row boxes; 1 = row boxes; 2 = row blocks only */
  int32_t state16;      /* uint8 input: 0 = levels stored between launches as uint16 where
                           their sums fit (255 (2^l + rows - 1) <= 65535), exact; 1 = int32 */
  int32_t search_widths; /* 0 = none; K = 1 .. 9: the last launch also runs the boxcar search
                            of widths 1, 2, .., 2^(K-1) (fdmt_execute_search) on its top level
                            while it is in shared memory; its time tiles carry 2^(K-1) - 1
                            samples of history (rounded up to 16).  uint8 plans need
                            255 (nf + nd - 1) 2^(K-1) <= 2^31 - 1 (else UNSUPPORTED) */
  /* Which adjoint fdmt_adjoint runs for a fused float plan: the plain one (one
     or two transposed levels per launch) or the fused one (pull cones of
     several transposed levels per launch, the last ending with the transpose
     of the Option-1 initialisation, level 0 never written): */
  int32_t adjoint_schedule;    /* 0 = fused for fused float plans (the faster on GB300), 1 = plain,
                                  2 = fused (fused float plans only) */
  int32_t adjoint_tile;        /* time tile, a multiple of 64; 0 = 512 */
  int32_t adjoint_smem_budget; /* shared memory per block; 0 = 112 KiB */
  int32_t adjoint_n_bounds;    /* 0 = chosen; else entries of adjoint_bounds, */
  int32_t adjoint_bounds[32];  /* 0 = b0 < ... < b_{n-1} = log2(nf): launch k (from the top)
                                  covers the transposed levels b_{n-1-k} -> b_{n-2-k} */
  int32_t adjoint_group_tile[32];    /* with adjoint_bounds: tile of the launch over levels
                                        b_{i+1} -> b_i (index i as bounds); 0 = adjoint_tile */
  int32_t adjoint_group_budget[32];  /* with adjoint_bounds: its shared memory; 0 = the budget */
} fdmt_schedule_params;

/*
 * fdmt_plan_ex -- fdmt_plan with explicit fused-schedule parameters (for
 * autotuning: each launch computes the merge levels (b_i, b_{i+1}] of the
 * addition rule, section 4).  params may be NULL (= fdmt_plan).  Parameters
 * that cannot fit the shared-memory budget give FDMT_ERR_UNSUPPORTED.
 */
int fdmt_plan_ex(double f_min, double f_max, int32_t nf, int64_t nt, int32_t nd,
                 int32_t dtype, uint32_t flags, const fdmt_schedule_params *params,
                 fdmt_plan_t *out);

/* The family of curves a plan sums along (section 4.2, "Applying FDMT for
 * other functional forms"): the delay across the band follows
 * Dt(f) ~ f^gamma, which enters only the merge coefficients
 * C = (f0^gamma - f1^gamma) / (f0^gamma - f2^gamma). */
typedef struct fdmt_curve_params {
  double gamma;        /* -2 = cold-plasma dispersion (what fdmt_plan uses); any finite nonzero value */
  int32_t d_min;       /* delay of output row 0 in samples, 0 .. 2^30 (section 4.2: the input
                          is pre-shifted by the delay of d_min, so row d follows delay
                          d_min + d): channel k (lower edge e_k) is delayed by
                          s_k = floor(d_min r(e_k) + 1/2) samples, r(f) = (f_min^gamma -
                          f^gamma) / (f_min^gamma - f_max^gamma), zeros shifted in */
  int32_t descending;  /* 1: input row j holds channel nf - 1 - j (f_max first); 0: row k is
                          channel k (f_min first).  Weights and weight gradients stay indexed
                          by channel (ascending frequency) either way. */
} fdmt_curve_params;

/*
 * fdmt_plan_curve -- fdmt_plan_ex for another curve family, a d_min offset
 * or descending channel order.  curve may be NULL (gamma = -2, d_min = 0,
 * ascending).  With d_min > 0 or descending input, execute first writes the
 * mapped input into the workspace (one extra pass over the input; the
 * workspace grows by nf * nt input elements, the adjoint's by two float
 * planes) and the adjoint maps its gradient back; fdmt_execute_static
 * refuses such plans (UNSUPPORTED).  Errors as fdmt_plan_ex; a gamma that is
 * zero or not finite, d_min outside 0..2^30 or descending not 0/1 give
 * INVALID_ARG.
 */
int fdmt_plan_curve(double f_min, double f_max, int32_t nf, int64_t nt, int32_t nd, int32_t dtype,
                    uint32_t flags, const fdmt_curve_params *curve, const fdmt_schedule_params *params,
                    fdmt_plan_t *out);

/* Release a plan and its device tables.  NULL is a no-op.  The caller must
 * make sure no work using the plan is still queued on any stream. */
void fdmt_destroy(fdmt_plan_t plan);

/* Bytes of device workspace fdmt_execute needs for this plan (intermediate
 * level states).  Errors: INVALID_ARG (NULL plan or bytes). */
int fdmt_workspace_bytes(fdmt_plan_t plan, size_t *bytes);

/* Bytes of device workspace fdmt_adjoint needs for this plan. */
int fdmt_adjoint_workspace_bytes(fdmt_plan_t plan, size_t *bytes);

/*
 * fdmt_execute -- the forward transform A = FDMT(w .* I) (section 4,
 * Algorithm 1): Option-1 initialisation, then log2(Nf) merge iterations.
 *
 *   in         device pointer, [nf][nt] row-major, element per dtype
 *              (uint8 or float32), 16-byte aligned.
 *   weights    device pointer to nf float32 per-channel weights applied to
 *              the input before the transform (x * w[k], one fp32 multiply),
 *              or NULL for none.  Must be NULL for FDMT_U8_I32.
 *   out        device pointer, [nd][nt] row-major, int32 (FDMT_U8_I32) or
 *              float32, 16-byte aligned; must not overlap in or workspace.
 *   workspace  device pointer, >= fdmt_workspace_bytes, 256-byte aligned.
 *   ws_bytes   its size.
 *   stream     cudaStream_t as void*.
 *
 * Errors: INVALID_ARG (NULL or misaligned pointers, host-only plan,
 * weights with FDMT_U8_I32), WORKSPACE, CUDA.  Asynchronous.
 */
int fdmt_execute(fdmt_plan_t plan, const void *in, const float *weights, void *out,
                 void *workspace, size_t ws_bytes, void *stream);

/*
 * fdmt_execute_static -- fdmt_execute without a caller workspace and without
 * allocating anything.  The paper has no counterpart; this is for callers
 * that cannot allocate device memory when they run the transform, such as a
 * real-time pipeline that must not allocate once data is flowing, or a host
 * framework that owns the whole device memory pool.  They create the plan
 * once beforehand (fdmt_plan allocates its delay tables) and then use this.
 *
 * The scratch is a fixed array of FDMT_STATIC_SCRATCH_BYTES inside the
 * library, present on every GPU that loads it until the process exits.  This
 * call always runs the plain schedule (one launch per level), also for plans
 * made with the fused schedule.  Its scratch is the plain schedule's
 * workspace: the level states of two consecutive levels, i.e. the
 * fdmt_workspace_bytes of a plan of the same shape made with the plain
 * schedule, which can differ from this plan's own fdmt_workspace_bytes when
 * it is fused.  Plans whose plain-schedule scratch is larger get
 * FDMT_ERR_WORKSPACE and nothing runs; e.g. Nf = Nd = 1024 fits up to
 * Nt = 2048 in float32.  Every call looks up the array's device address in
 * the current device's context (cudaGetSymbolAddress); the first call on a
 * device may load the library's module, so make that first call before any
 * stream capture.  All calls share the array: calls that overlap on the GPU
 * (several streams or host threads at once) race and give wrong results.
 * Arguments, result and other errors as fdmt_execute (plain schedule).
 */
#define FDMT_STATIC_SCRATCH_BYTES (32u << 20)
int fdmt_execute_static(fdmt_plan_t plan, const void *in, const float *weights, void *out,
                        void *stream);

/*
 * fdmt_execute_search -- the transform of fdmt_execute followed by the
 * boxcar search of fdmt_search on its output (section 4.2, pulse profile:
 * a uniform profile convolved with the time axis commutes with the
 * transform): for row d and width 2^k, k < n_widths, peak[d][k] is the
 * largest boxcar sum over t and time[d][k] the first t reaching it (types
 * and sums as fdmt_search; out receives A).  When the plan was made with
 * search_widths == n_widths (fused schedule) the search of each tile runs
 * in the last launch while the top level is still in shared memory,
 * leaving per-tile (value, region) partials in the workspace that one small
 * launch resolves to times from A; otherwise the standalone search runs
 * after the transform.  The results are the same either way.
 *   workspace  fdmt_execute_search_workspace_bytes(plan, n_widths) bytes.
 * Errors as fdmt_execute and fdmt_search.
 */
int fdmt_execute_search(fdmt_plan_t plan, const void *in, const float *weights, void *out, int32_t n_widths,
                        void *peak, int32_t *time, void *workspace, size_t ws_bytes, void *stream);
int fdmt_execute_search_workspace_bytes(fdmt_plan_t plan, int32_t n_widths, size_t *bytes);

/*
 * fdmt_execute_host -- fdmt_execute on host buffers: copies host_in to
 * dev_in, transforms into dev_out, copies dev_out back to host_out, and
 * waits for the stream.  Host buffers should be page-locked for full copy
 * speed.  host_weights (nf floats, host) may be NULL; when given, dev_weights
 * (nf floats, device) receives them.  Same errors as fdmt_execute.
 */
int fdmt_execute_host(fdmt_plan_t plan, const void *host_in, const float *host_weights,
                      void *host_out, void *dev_in, float *dev_weights, void *dev_out,
                      void *workspace, size_t ws_bytes, void *stream);

/*
 * fdmt_adjoint -- the transposed transform (not in the paper: the exact
 * transpose of the addition rule and of the Option-1 initialisation, in
 * gather form so no atomics are needed), plus the gradients of the
 * per-channel weights of fdmt_execute.  With g = FDMT^T(grad_out):
 *
 *     grad_in[k][s]   = w[k] * g[k][s]               (w = 1 if weights is NULL)
 *     grad_weights[k] = sum_s in[k][s] * g[k][s]     (if grad_weights != NULL)
 *
 *   grad_out      device float32 [nd][nt], 16-byte aligned.
 *   in            device float32 [nf][nt]: the input the forward call saw;
 *                 read only when grad_weights != NULL (else may be NULL).
 *   weights       device float32 [nf] or NULL.
 *   grad_in       device float32 [nf][nt], 16-byte aligned.
 *   grad_weights  device float32 [nf] or NULL.
 *   workspace     device, >= fdmt_adjoint_workspace_bytes, 256-byte aligned.
 *
 * Only float plans (FDMT_F32_F32, FDMT_F32_F16STATE; the adjoint always
 * computes in float32; FDMT_U8_I32 gives FDMT_ERR_UNSUPPORTED).  A plan made
 * with FDMT_SCHED_FUSED runs the fused adjoint (several transposed levels
 * per launch, level 0 never written; adjoint_schedule in
 * fdmt_schedule_params), other plans one or two transposed levels per
 * launch; the two agree to float32 rounding order.  Shapes whose one-row
 * cone cannot fit (2^k + 1 channels over a wide band: the lone upper
 * channel's row reads hundreds of parent rows) keep the plain adjoint.
 * Errors as
 * fdmt_execute.  Asynchronous.
 */
int fdmt_adjoint(fdmt_plan_t plan, const float *grad_out, const float *in, const float *weights,
                 float *grad_in, float *grad_weights, void *workspace, size_t ws_bytes,
                 void *stream);

/* ---- boxcar search of a transform output ---- */

/*
 * fdmt_search -- the pulse-width search of section 4.2 ("Pulse profile"):
 * convolving the time axis with a uniform (boxcar) profile commutes with the
 * transform, so widths are tested on its output.  For k < n_widths,
 * w = 2^k and every row d:
 *
 *     B_w[d][t] = sum_{i=0}^{w-1} A[d][t-i]     (A = 0 before t = 0)
 *     peak[d][k] = max_{0 <= t < nt} B_w[d][t]
 *     time[d][k] = the first t with B_w[d][t] == peak[d][k]
 *
 * summed as the binary tree B_1 = A, B_2w[t] = B_w[t] + B_w[t-w]: exactly
 * for an integer output, in float32 for a float output (that order of
 * additions, so the result is reproducible bit for bit).
 *
 *   A           device, [nd][nt] row-major: int32 when dtype is FDMT_U8_I32
 *               (the output of a uint8 plan), else float32.  Any alignment
 *               (16-byte aligned rows with nt % 4 == 0 read faster).
 *               Finite values (a NaN is never a maximum).
 *   dtype       the plan dtype that produced A (FDMT_F32_F16STATE = float).
 *   nd          rows, >= 1.
 *   nt          samples per row, 1 <= nt <= 2^31 - 2^14 (else UNSUPPORTED).
 *   n_widths    K, 1..13 (widths 1 .. 4096 samples).
 *   value_bound integer A only: 0 (unknown) or a bound the caller
 *               guarantees, |A[d][t]| <= value_bound everywhere (for a uint8
 *               plan, 255 * (nf + nd - 1): no output cell sums more input
 *               samples).  When value_bound * 2^(K-1) <= 2^31 - 1 the sums
 *               run in int32, else in int64; both are exact under the
 *               guarantee.  Negative: INVALID_ARG.
 *   peak        device, [nd][K]: int64 for FDMT_U8_I32, else float32.
 *   time        device, [nd][K] int32.
 *   workspace   device, >= fdmt_search_workspace_bytes, 16-byte aligned
 *               (else WORKSPACE).
 *   stream      cudaStream_t (NULL = legacy default stream).
 *
 * Two launches; nothing is allocated.  Errors: INVALID_ARG, UNSUPPORTED,
 * WORKSPACE, CUDA.  Asynchronous.
 */
int fdmt_search(const void *A, int32_t dtype, int32_t nd, int64_t nt, int32_t n_widths, int64_t value_bound,
                void *peak, int32_t *time, void *workspace, size_t ws_bytes, void *stream);

/* Bytes of device workspace fdmt_search needs (INVALID_ARG outside the
 * ranges above). */
int fdmt_search_workspace_bytes(int32_t nd, int64_t nt, int32_t n_widths, size_t *bytes);

/* ---- pipelined host execution ---- */

typedef struct fdmt_pipeline_s *fdmt_pipeline_t;

/*
 * fdmt_pipeline_create -- transforms of host-resident data, overlapped.
 * Each push copies a host input to the device, runs fdmt_execute and copies
 * the output back; the input copy of the next push and the output copy of
 * the previous one run on their own CUDA streams while a push computes (two
 * device slots take turns), so a push costs about the larger of its copies,
 * not their sum.  The plan is borrowed (destroy the pipeline first); no
 * weights.  The pipeline owns its device buffers (2 inputs, 2 outputs, one
 * workspace), streams and events, allocated here.
 * Errors: INVALID_ARG, NO_MEMORY, CUDA.
 */
int fdmt_pipeline_create(fdmt_plan_t plan, fdmt_pipeline_t *out);

/*
 * fdmt_pipeline_push -- queue one transform: host_in [nf][nt] (uint8 or
 * float32, page-locked for the copies to be asynchronous) to host_out
 * [nd][nt] (int32 or float32, page-locked).  Returns at once; host_in may
 * be reused and host_out read only after fdmt_pipeline_wait.  Errors:
 * INVALID_ARG, CUDA, and those of fdmt_execute.
 */
int fdmt_pipeline_push(fdmt_pipeline_t p, const void *host_in, void *host_out);

/* Block until every queued push has finished (outputs in host memory). */
int fdmt_pipeline_wait(fdmt_pipeline_t p);

/* Waits, then frees the pipeline; NULL-safe. */
void fdmt_pipeline_destroy(fdmt_pipeline_t p);

/* ---- STFT filterbank in front of the transform ---- */

/*
 * fdmt_filterbank -- the front end of section 2: the voltage series is cut
 * into blocks of nf samples, each block is Fourier transformed (STFT) and
 * the squared magnitude at each frequency kept, with the footnote's
 * optional binning of nbin consecutive spectra:
 *
 *     out[c][t] = sum_{b < nbin} |sum_{m < nf} v[(t nbin + b) nf + m]
 *                                 exp(-2 pi i k m / nf)|^2,  k = (c + nf/2) mod nf
 *
 * Channel c is in ascending frequency (negative offsets first): for complex
 * baseband voltages sampled at rate B around f_c, channel c is centred on
 * f_c - B/2 + c B/nf, so a plan with f_min = f_c - B/2 - B/(2 nf) and
 * f_max = f_min + B puts each channel's interval on its response.
 *
 *   volts   device, n complex64 values (interleaved re, im), 16-byte aligned.
 *   nf      channels = samples per block: a power of two, 2..4096.
 *   nbin    spectra summed per output sample, 1..1024; nbin nf (up to 8192
 *           samples per output time) must fit shared memory, else
 *           UNSUPPORTED.
 *   out     device float32 [nf][nt], row stride nt, 4-byte aligned.
 *   nt      output samples, 1 <= nt <= n / (nf nbin) (later samples of v
 *           are not read).
 *   stream  cudaStream_t.
 * Float32 Stockham FFT (radix 16): each value within about 8 eps log2(nf)
 * of the spectrum's total power of the float64 result.  Errors: INVALID_ARG,
 * UNSUPPORTED, CUDA.  Asynchronous.
 */
int fdmt_filterbank(const void *volts, int64_t n, int32_t nf, int32_t nbin, float *out, int64_t nt, void *stream);

/* ---- FFT-FDMT (section 5, Algorithm 2) ---- */

/*
 * The transform computed in the Fourier domain of the time axis: each shifted
 * row addition of Algorithm 1 becomes a product with the shift vector
 * exp(-2 pi i k s / N), so every addition stays within one Fourier bin.  The
 * result is the direct transform's (fdmt_execute), up to float32 FFT
 * rounding:
 *
 *     out[d][t] = sum over the curve of row d of in[k][t - o],  zero before t = 0
 *
 * Shifts are cyclic within an FFT block (the zero-padding paragraph of
 * section 5), so the time axis is cut into overlapping blocks of N samples:
 * block j covers input samples [j S - (Nd-1), j S - (Nd-1) + N) and gives
 * output columns [j S, j S + S), hop S = N - (Nd - 1).  Two consecutive blocks
 * share one complex FFT, one in the real and one in the imaginary part (the
 * machine-word paragraph's packing).  Tables, channel edges and rounding are
 * those of fdmt_plan (power law -2, ascending channels, no d_min).
 *
 *   dtype   FDMT_F32_F32 (float32 input) or FDMT_U8_I32 (uint8 input); the
 *           output is float32 either way.
 *   block   FFT length N: 0 picks the smallest power of two >= 4 (Nd - 1)
 *           within [256, 4096]; else a power of two in [256, 4096].
 *           N <= Nd - 1 is UNSUPPORTED.
 *   bins    Fourier bins per merge block: 0 (pick: 2 when four blocks fit
 *           an SM, else 4 when two do, else what fits), 1, 2, 4 or 8; the
 *           merge state (rows of two consecutive levels, the shift vectors
 *           of the block's bins) must fit 200 KB of shared memory, else
 *           UNSUPPORTED.
 *   flags   0 or FDMT_PLAN_HOST_ONLY (shape and workspace only; no device
 *           allocation; execute then fails with INVALID_ARG).
 *   out     receives the plan (NULL on failure).  The plan owns its device
 *           tables (row ops, the N roots of unity) on the current device,
 *           allocated here and freed by fdmt_fft_destroy; it is bound to
 *           that device.
 * Limits: 2 <= nf <= 65535, 1 <= nd <= 65535, nt >= 1.
 * Errors: INVALID_ARG (arguments, table builder), UNSUPPORTED, NO_MEMORY, CUDA.
 */
typedef struct fdmt_fft_s *fdmt_fft_t;
int fdmt_fft_plan(double f_min, double f_max, int32_t nf, int64_t nt, int32_t nd, int32_t dtype, int32_t block,
                  int32_t bins, uint32_t flags, fdmt_fft_t *out);
void fdmt_fft_destroy(fdmt_fft_t plan); /* NULL is a no-op */

/* Workspace of fdmt_fft_execute: max(nf, nd) rows of pairs * N complex64
 * Fourier bins (the transformed input, then the top level over it). */
int fdmt_fft_workspace_bytes(fdmt_fft_t plan, size_t *bytes);

/* Block length N, hop S, block pairs (complex FFTs per row) and bins per
 * merge block of a plan; any pointer may be NULL. */
int fdmt_fft_info(fdmt_fft_t plan, int32_t *block, int64_t *hop, int64_t *pairs, int32_t *bins);

/*
 * fdmt_fft_execute -- three launches on `stream`: forward FFTs of the input
 * blocks, the merges of all levels per Fourier bin, inverse FFTs into `out`.
 *   in         device [nf][nt] (float32 4-byte aligned, or uint8).
 *   out        device float32 [nd][nt], 4-byte aligned.
 *   workspace  device, >= fdmt_fft_workspace_bytes, 16-byte aligned; its
 *              contents are overwritten.
 * Float32 arithmetic: each output row within about 1e-5 of its RMS of the
 * float64 result for the sizes of the tests (FFT rounding, growing with
 * log2 N and the number of levels).  Asynchronous.  Errors: INVALID_ARG
 * (pointers, alignment, workspace size, host-only plan, other device),
 * UNSUPPORTED, CUDA.
 */
int fdmt_fft_execute(fdmt_fft_t plan, const void *in, float *out, void *workspace, size_t ws_bytes, void *stream);

/* Per-launch timing of an FFT-FDMT plan, as fdmt_profile_enable /
 * fdmt_profile_read: a ring of `capacity` event pairs around each of the
 * three launches (0 turns it off; kernel ids named by fdmt_kernel_name:
 * "fft_forward", "fft_merge", "fft_inverse").  Read returns up to n
 * (kernel id, ms) of the latest launches, oldest first, waits for them, and
 * resets the count; *launches receives the launches recorded since enable
 * or the last read.  Errors: INVALID_ARG (NULL plan, host-only plan), CUDA. */
int fdmt_fft_profile_enable(fdmt_fft_t plan, int32_t capacity);
int fdmt_fft_profile_read(fdmt_fft_t plan, int32_t *kernel_ids, float *ms, int32_t n, int64_t *launches);

/* ---- overlap-save streaming ---- */

typedef struct fdmt_stream_s *fdmt_stream_t;

/*
 * fdmt_stream_create -- transform a continuous stream chunk by chunk.
 * Output column t depends only on input columns [t - nd + 1, t] (the
 * recursion looks back in time only, Algorithm 1, with the copy rule of
 * section 4 for samples before the first), so each chunk is appended to the
 * last carry = ceil16(nd - 1) input columns of the stream and the window of
 * carry + chunk columns is transformed; the output of a push equals
 * columns [T, T + chunk) of a transform of the whole stream so far (T = the
 * samples pushed before), bit for bit.
 *
 *   f_min, f_max, nf, nd, dtype, flags   as fdmt_plan (the plan is built for
 *                 nt = carry + chunk; FDMT_PLAN_HOST_ONLY is refused).
 *   chunk         samples per push, a multiple of 16, >= 16.
 *   out           receives the stream handle (NULL on failure).
 *
 * The stream owns its device memory (two input windows, one window output,
 * the plan's workspace), allocated here and freed by fdmt_stream_destroy.
 * Errors: as fdmt_plan (the shape is checked before any allocation),
 * NO_MEMORY, CUDA.
 */
int fdmt_stream_create(double f_min, double f_max, int32_t nf, int64_t chunk, int32_t nd, int32_t dtype,
                       uint32_t flags, fdmt_stream_t *out);

/*
 * fdmt_stream_push -- transform the next chunk.
 *   in      device, [nf][chunk] (uint8 or float32 as the dtype), 16-byte aligned.
 *   out     device, [nd][chunk] (int32 or float32), 16-byte aligned.
 *   stream  cudaStream_t; every push of one stream object must be ordered
 *           (same CUDA stream, or synchronised), as they share the windows.
 * Asynchronous (copies and launches only).  Errors: INVALID_ARG, CUDA, and
 * those of fdmt_execute.
 */
int fdmt_stream_push(fdmt_stream_t s, const void *in, void *out, void *stream);

/* Forget the history: the next push starts a new stream (zero carry). */
int fdmt_stream_reset(fdmt_stream_t s, void *stream);

/* carry (input columns kept between pushes) and window (= carry + chunk). */
int fdmt_stream_info(fdmt_stream_t s, int64_t *carry, int64_t *window);

/* Frees the stream and its device memory; NULL-safe. */
void fdmt_stream_destroy(fdmt_stream_t s);

/* ---- batches of independent beams ---- */

typedef struct fdmt_batch_s *fdmt_batch_t;

/* One beam of a batch: its own band, channels, samples and delay rows
 * (same rules as fdmt_plan; all beams of a batch share one dtype). */
typedef struct fdmt_beam_desc {
  double f_min, f_max;
  int32_t nf;
  int32_t nd;
  int64_t nt;
} fdmt_beam_desc;

/* Work-item shape of the batch kernel (0 = default). */
typedef struct fdmt_batch_params {
  int32_t rows_per_item;   /* level schedule: delay rows of one work item (default 16) */
  int32_t tile;            /* level schedule: samples of one work item, multiple of 1024 (default 2048) */
  int32_t blocks_per_sm;   /* resident blocks per SM (default: as many as fit) */
  int32_t wait_ms;         /* limit of one dependency wait in ms (default 2000) */
  int32_t schedule;        /* 0 = one merge level per work item; 1 = fused: every beam's
                              cone programme of the fused schedule (fdmt_plan_ex), uint8 and
                              float32 only; 2 = launches: one fused plan per beam, the beams' launches spread
                              over 4 streams forked from the caller's stream, largest beam
                              first (no dependency waits; drop_level: UNSUPPORTED) */
  int32_t fused_tile;      /* fused: time tile, multiple of 64 (0 = chosen per level group) */
  int32_t smem_budget;     /* fused: shared memory per block in bytes (0 = 72 KiB) */
} fdmt_batch_params;

/*
 * fdmt_plan_batch -- plan the transforms of n independent beams (each the
 * FDMT of section 4 / Algorithm 1 with its own band and sizes) as ONE
 * persistent kernel launch: the blocks take work items from a global
 * counter, and an item waits (bounded) until its producers are done.  Level
 * schedule (params->schedule = 0): items (beam, level, block of delay rows,
 * time tile) in level-major order; an item of level l needs every item of
 * level l-1 of its beam.  Fused schedule (1): items (beam, level group,
 * cone, time tile) of every beam's fused programme in group-major order; an
 * item of group g needs every item of group g-1 of its beam.  Because items
 * are handed out in that order, waits happen only between items and every
 * block is resident, every wait ends unless a producer is missing; a wait
 * that exceeds wait_ms makes the launch stop and report FDMT_ERR_TIMEOUT.
 * Allocates the device tables and the work counters; params may be NULL.
 * Errors: INVALID_ARG, UNSUPPORTED, NO_MEMORY, CUDA.
 */
int fdmt_plan_batch(int32_t n, const fdmt_beam_desc *beams, int32_t dtype, uint32_t flags,
                    const fdmt_batch_params *params, fdmt_batch_t *out);

/* Release a batch plan (NULL is a no-op). */
void fdmt_destroy_batch(fdmt_batch_t batch);

/* Workspace bytes of fdmt_execute_batch (all beams' intermediate levels). */
int fdmt_batch_workspace_bytes(fdmt_batch_t batch, size_t *bytes);

/*
 * fdmt_execute_batch -- transform every beam: in[i] / out[i] are device
 * pointers (host arrays of n pointers) laid out as for fdmt_execute.  The
 * first call with a given set of pointers records the launch (counter
 * reset + kernel) as a CUDA graph; later calls with the same pointers
 * replay it.  Waits for `stream` before returning and reports
 * FDMT_ERR_TIMEOUT if a dependency wait gave up.  Errors: INVALID_ARG,
 * WORKSPACE, CUDA, TIMEOUT.
 */
int fdmt_execute_batch(fdmt_batch_t batch, const void *const *in, void *const *out,
                       void *workspace, size_t ws_bytes, void *stream);

/*
 * fdmt_batch_drop_level -- test hook for failure detection: remove the
 * work items of (beam, level) -- of (beam, level group) for the fused
 * schedule -- from the work list so that the next level (group) of that
 * beam waits for producers that never run.  The next fdmt_execute_batch
 * must then return FDMT_ERR_TIMEOUT within about wait_ms, with no device
 * fault.  level >= 0; -1 restores the full list.
 */
int fdmt_batch_drop_level(fdmt_batch_t batch, int32_t beam, int32_t level);

/*
 * fdmt_batch_levels -- the level boundaries beam `beam` is computed in:
 * *groups = work-item kinds of that beam (level groups for the fused
 * schedule, levels + 1 for the level schedule), bounds[0 .. groups] their
 * boundaries (level schedule: 0, 0, 1, ..., L, the first entry the
 * initialisation), sizes[0 .. groups] the bytes per sample stored at each
 * boundary (sizes[0]: the input).  bounds / sizes may be NULL, else
 * n >= groups + 1.  Host only.  Errors: INVALID_ARG.
 */
int fdmt_batch_levels(fdmt_batch_t batch, int32_t beam, int32_t *groups, int32_t *bounds, int32_t *sizes,
                      int32_t n);

/* ---- launch profiler (per-kernel device time, for benchmarks) ---- */

/*
 * fdmt_profile_enable -- record a pair of CUDA events around every kernel
 * launch this plan makes from now on, in a ring of `capacity` slots (the
 * oldest are overwritten).  capacity 0 turns recording off.  Creates events,
 * allocates no device memory.  Not for concurrent use of one plan from
 * several host threads.  Errors: INVALID_ARG, CUDA.
 */
int fdmt_profile_enable(fdmt_plan_t plan, int32_t capacity);

/*
 * fdmt_profile_read -- wait for the recorded launches and report them oldest
 * first: kernel id (see fdmt_kernel_name), level (merge level, 0 for init) and
 * device time in ms, at most n entries; *launches receives the number of
 * launches recorded since enable or the last read (which may exceed the
 * ring).  Resets the count.  Errors: INVALID_ARG, CUDA.
 */
int fdmt_profile_read(fdmt_plan_t plan, int32_t *kernel_ids, int32_t *levels, float *ms,
                      int32_t n, int64_t *launches);

/* Name of a kernel id reported by fdmt_profile_read (static string). */
const char *fdmt_kernel_name(int32_t kernel_id);

/*
 * fdmt_device_status -- wait for `stream`, then report whether any kernel of
 * this plan gave up a bounded wait since the last check (the fused kernels
 * wait on their shared-memory copies with an iteration limit instead of
 * hanging): FDMT_ERR_TIMEOUT if so (and the word is cleared), FDMT_OK if
 * not.  Errors: INVALID_ARG, CUDA.
 */
int fdmt_device_status(fdmt_plan_t plan, void *stream);

/*
 * fdmt_schedule_info -- the fused schedule chosen at plan time: *groups =
 * launches per transform (0 for the plain schedule), bounds[0..groups] = the
 * level boundaries (0 = b0 < ... < b_groups = L; may be NULL, else n >=
 * groups + 1), *tile = time-tile width in samples.
 */
int fdmt_schedule_info(fdmt_plan_t plan, int32_t *groups, int32_t *bounds, int32_t n, int32_t *tile);

/*
 * fdmt_fused_tables -- copy one table of the fused schedule (host copy, for
 * inspection and tests) as int32 values: kind 0 groups (16 per group: lb,
 * lt, from_input, first template, templates, shared bytes, tiles, tile
 * width, end of the staged-row region, end of the first compute region,
 * row-box width in elements (0 for row blocks), row-block chunk in
 * elements (0 for row boxes), chunks per row block, log2 of the largest
 * row block, bytes per staged sample, bytes per written sample), 1
 * templates (8 each: first load, loads, first walk, walks, first stage
 * word, stages, TMA bytes, shared bytes), 2 loads (4: row, shared offset,
 * column offset from the tile start, boxes per row for row boxes or log2 of
 * the rows copied for row blocks), 3 walks (12 each, level 1 of a band of
 * two channels straight from the staged input: destination, destination
 * row bytes, lower and upper channel sample offsets, width, first column,
 * first row, last row, first lower row, row-step bits, lower channel, 0),
 * 4 ops (8 each: destination, four source offsets, width, reuse flags,
 * first column), 5 stages (10 words per stage: kind 0 walk / 1 one level /
 * 2 two levels, then the first walk or op of each of the 8 warps and the
 * end),
 * 6 constants (tile, state size, input size, acc size, bytes of over-read
 * slack that end a block's shared memory, bytes of the warps' descriptor
 * slots before it), 7 the planner's cost
 * model per group (6 each: HBM KiB, shared-memory pipe kilo-slots, work
 * items, thousands of ops, resident blocks, modelled microseconds).  The
 * fused adjoint (empty unless the plan has one): kind 10 launches in launch
 * order (15 each: top level lt, bottom level lb, 1 if the launch ends with
 * the transpose of the initialisation, tile, row-box width (0 for row
 * blocks), first template, templates, shared bytes, end of the staged-row
 * region, end of the first compute region, tiles, modelled HBM KiB,
 * row-block chunk (0 for row boxes), chunks per staged row, log2 of the
 * largest row block), 11 templates (as kind 1), 12 loads (as kind 2), 13 ops (8 each: destination, first source byte
 * offset, source stride in bytes, terms, the piece within the tile (the
 * initialisation transposes; else 0), width, flags (the folded
 * transpose: bit 0 upper half, then 4 bits per level-0 row with the length
 * of its run of level-1 rows; else 0), first column relative to the tile
 * start), 14 stages (10 words: kind 1 gather / 2 initialisation transpose
 * / 3 initialisation transpose with the level 1 -> 0 gather folded in,
 * the first op of each warp, the end).  *count
 * receives the number of values; dst may be NULL to query.
 */
int fdmt_fused_tables(fdmt_plan_t plan, int32_t kind, int32_t *dst, int64_t n, int64_t *count);

/* Human-readable name of a status code (static string, never NULL). */
const char *fdmt_error_string(int status);

/* ---- table inspection (host-side; used to cross-check the delay tables) ---- */

/* Number of merge levels L = ceil(log2(nf)). */
int fdmt_num_levels(fdmt_plan_t plan, int32_t *levels);

/* Rows held by each band of level l (0 <= l <= L): writes ceil(nf / 2^l) values.
 * Level 0 bands are single channels (rows = max intra-channel sweep + 1);
 * level L is the whole band (rows = nd).  n = capacity of rows_out. */
int fdmt_band_rows(fdmt_plan_t plan, int32_t level, int32_t *rows_out, int32_t n);

/* The plan's shape: channels, samples, delay rows, dtype (NULL pointers are
 * skipped). */
int fdmt_plan_shape(fdmt_plan_t plan, int32_t *nf, int64_t *nt, int32_t *nd, int32_t *dtype);

/* The plan's input mapping: shift[k] = s_k of channel k (n >= nf; all zero
 * without d_min) and *descending (either pointer may be NULL). */
int fdmt_input_map(fdmt_plan_t plan, int32_t *shift, int32_t n, int32_t *descending);

/* Lower-half rows dl[Dt] of band b at level l >= 1 (one per row Dt of that
 * band; the upper half is read at row Dt - dl, shifted by dl samples). */
int fdmt_band_dl(fdmt_plan_t plan, int32_t level, int32_t band, int32_t *dl_out, int32_t n);

#ifdef __cplusplus
}
#endif

#endif /* FDMT_GB300_H */
