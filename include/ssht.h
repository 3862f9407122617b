/*
 * ssht.h -- C ABI of libssht, a GB300 (sm_103a) implementation of the exact spin
 * spherical harmonic transform of J. D. McEwen, "Fast, exact (but unstable) spin
 * spherical harmonic transforms" (arXiv:0807.4494).
 *
 * The transform maps spin-s coefficients sf_lm, 0 <= l < L, |m| <= l, to samples of
 *   f(theta, phi) = sum_{l,m} sf_lm sY_lm(theta, phi)                (eqn ssht_inv, Sec. 2.3)
 * on the paper's equiangular grid (eqns nodes_theta / nodes_phi, Sec. 3.4.1) and back.
 * Through eqn wigner_sum_reln (Sec. 2.2) the harmonics become Fourier series on the
 * torus whose coefficients are eqn fourier_coeff (Sec. 3.1):
 *   F_{m m'} = (-1)^s i^{-(m+s)} sum_l sqrt((2l+1)/4pi) Delta^l_{m'm} Delta^l_{m',-s} sf_lm,
 * with Delta^l_{m'm} = d^l_{m'm}(pi/2) made in FP64 by a three-term recursion within each degree
 * (from J_x Delta^l = Delta^l J_z and the closed-form first row), or by the paper's Risbo
 * recursion (Sec. 2.2) with SSHT_FLAG_RISBO.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - L is the EXCLUSIVE band-limit (coefficients with l < L).  The paper's inclusive
 *    band-limit is L-1; its torus has N = 2L-1 samples per axis.
 *  - Coefficients: flm[b][l*l + l + m], complex interleaved (re, im), batch outermost,
 *    b = 0 .. batch-1.  Entries with l < |s| do not exist: inputs there are ignored,
 *    outputs there are written as 0.
 *  - Sphere samples: f[b][t][p], complex interleaved, t = 0..L-1 (theta_t = pi(2t+1)/(2L-1),
 *    the last ring is theta = pi), p = 0..2L-2 (phi_p = pi(2p+1)/(2L-1)).
 *  - Element type: plans of precision SSHT_FP64 take and return double pairs
 *    (16 bytes per complex value); every other precision takes and returns float pairs
 *    (8 bytes per complex value).
 *  - Data pointers may be device memory or host memory (pinned or pageable); host
 *    buffers are staged through plan-owned device memory.  The caller owns all data
 *    buffers.  Calls are asynchronous on `stream` (a cudaStream_t; NULL is the legacy
 *    default stream) when all pointers are device pointers; with host pointers a call
 *    returns once its host output has been written.
 *  - Errors: every entry point returns 0 on success or a negative SSHT_E* code and
 *    records a message retrievable with ssht_last_error() (per host thread).  Nothing
 *    aborts the process.  Kernel-side failures (a grid barrier that exceeded its spin
 *    limit) are latched in the plan and reported by ssht_plan_check().
 *  - A plan is bound to the CUDA device that was current when it was created and must
 *    be used with that device current.  One plan must not be used concurrently from
 *    two host threads or on two streams at once (it owns one workspace).
 */
#ifndef SSHT_H
#define SSHT_H

#include <stddef.h>

#if defined(__GNUC__)
#define SSHT_API __attribute__((visibility("default")))
#else
#define SSHT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define SSHT_OK 0
#define SSHT_EINVAL (-1)       /* bad argument (band-limit, spin, batch, null pointer, ...) */
#define SSHT_ENOMEM (-2)       /* device or host allocation failed */
#define SSHT_ECUDA (-3)        /* a CUDA runtime or cuFFT call failed */
#define SSHT_ETIMEOUT (-4)     /* a device-side wait hit its iteration limit */
#define SSHT_EUNSUPPORTED (-5) /* valid request that this build does not implement */

/* Arithmetic of the O(L^3) contraction.  The Delta recursion is FP64 in every mode. */
typedef enum {
  SSHT_FP64 = 0,   /* FP64 everywhere (CUDA cores); double I/O                          */
  SSHT_FP32 = 1,   /* FP32 contraction on CUDA cores with FP64 Delta; float I/O          */
  SSHT_TF32X3 = 2, /* contraction on tcgen05 tensor cores, 3xTF32 split products         */
  SSHT_BF16X6 = 3  /* contraction on tcgen05 tensor cores, 3-way BF16 split, 6 products  */
} ssht_precision;

/* Where the Delta^l table lives. */
typedef enum {
  SSHT_DELTA_RECOMPUTE = 0, /* the recursion runs inside every transform call            */
  SSHT_DELTA_CACHE = 1      /* the recursion runs once at plan creation; calls reuse it  */
} ssht_delta_mode;

/* Plan flags. */
#define SSHT_FLAG_REAL 1 /* real fields of spin 0: f real, sf_{l,-m} = (-1)^m conj(sf_lm) (the
                          * conjugate symmetry of Sec. 3.3).  batch counts real fields; two ride in
                          * one complex transform (half the work).  Samples f are real arrays
                          * [batch][L][2L-1] (double or float); coefficients stay complex and the
                          * inverse reads them as given (they must have the symmetry). */
#define SSHT_FLAG_RISBO 2 /* make the Delta^l table with the Risbo recursion (the recursion the paper
                           * uses, Sec. 2.2: degree l+1 from degree l by two half-integer steps)
                           * instead of the default three-term relation in the first index m'
                           * (Delta_{m'-1,m} from Delta_{m'm} and Delta_{m'+1,m} within one degree,
                           * from the closed-form first row Delta_{l m}).  Both give Delta^l to
                           * rounding; the default needs no hand-off between degrees and 2 FP64
                           * instructions an entry against about 9. */
#define SSHT_FLAG_TUNE 4  /* tensor-core plans: at creation, time the contraction's shape candidates
                           * (fields per GEMM launch 64/32/16, pipeline depth 2-4, work order) on the
                           * plan's own operands and keep the fastest; with the environment variable
                           * SSHT_TUNE_CACHE naming a file, choices are read from it (no timing) and
                           * appended to it after tuning, one JSON object per line keyed by
                           * "L=.. s=.. B=.. precision".  Ignored by the other precisions. */
#define SSHT_FLAG_SPIN_PAIR 8 /* each field comes with its conjugate, the pair of spins s and -s
                               * the paper writes f_s* = f_{-s} (Sec. 3.3; for s = 0 and real f the
                               * reality condition).  Coefficients are [batch][2][L*L]: spin s, then
                               * spin -s of the conjugate field, tied by _{-s}f_{l,-m} =
                               * (-1)^{s+m} conj(_s f_lm).  forward / adjoint compute both sets with
                               * one spin-s transform (half the work of two transforms); inverse
                               * reads the spin-s half only and returns f.  Not with SSHT_FLAG_REAL. */

typedef struct {
  int L;          /* exclusive band-limit, 1 <= L <= 2048                      */
  int s;          /* spin, |s| < L                                              */
  int batch;      /* number of fields per call, 1 <= batch <= 65535            */
  int precision;  /* ssht_precision                                            */
  int delta_mode; /* ssht_delta_mode                                           */
  int flags;      /* 0 or SSHT_FLAG_* (REAL, RISBO, TUNE, SPIN_PAIR)            */
} ssht_plan_desc;

typedef struct ssht_plan_s* ssht_plan_t;

/* Create an FP64 plan with the Delta recursion run in every call.
 * out: receives the plan; L, s, batch as in ssht_plan_desc.
 * Allocates the plan's device workspace (see ssht_plan_workspace_bytes) and cuFFT plans. */
SSHT_API int ssht_plan(ssht_plan_t* out, int L, int s, int batch);

/* Create a plan from a descriptor (precision and Delta mode).  With SSHT_DELTA_CACHE the
 * recursion runs here, synchronously, and its table stays resident in device memory.
 * The tensor-core precisions (SSHT_TF32X3, SSHT_BF16X6) take any batch: the contraction runs the
 * fields in slices of at most 64 (one GEMM launch each, all reading the same A operand). */
SSHT_API int ssht_plan_ex(ssht_plan_t* out, const ssht_plan_desc* desc);

/* Release every resource of a plan (NULL is accepted).  Synchronises the device. */
SSHT_API int ssht_plan_destroy(ssht_plan_t plan);

/* Device bytes owned by the plan (workspace, Delta table, cuFFT work areas). */
SSHT_API int ssht_plan_workspace_bytes(ssht_plan_t plan, size_t* bytes);

/* Inverse transform, eqn ssht_inv (Sec. 3.4.3 of the paper): for each field, F_{m m'}
 * for m' >= 0 by eqn fourier_coeff, F_{m,-m'} = (-1)^{m+s} F_{m m'} (eqn Ffourier_sym),
 * then the torus samples by eqn idft_spatial, keeping the L rings with theta <= pi.
 * flm: [batch][L*L] complex in; f: [batch][L][2L-1] complex out. */
SSHT_API int ssht_inverse(ssht_plan_t plan, const void* flm, void* f, void* stream);

/* Forward transform, eqn ssht_fwd, by exact quadrature on the torus: per-m parity
 * extension of the samples to theta in [0, 2pi) (Sec. 3.2), the torus DFT (eqn
 * dft_spatial), the sin(theta) weight convolution G_{mm'} = 2pi sum_{m''} F_{mm''} w(m''-m'),
 * w(p) = int_0^pi sin(t) e^{ipt} dt, and the projection
 *   sf_lm = (-1)^s i^{m+s} sqrt((2l+1)/4pi) sum_{|m'|<=l} Delta^l_{m'm} Delta^l_{m',-s} G_{mm'}.
 * Exact (up to rounding) for band-limited f; the paper's own forward (a triangular solve,
 * eqn matrix_fwd) is unstable beyond L ~ 32 and is not used here.
 * f: [batch][L][2L-1] complex in; flm: [batch][L*L] complex out. */
SSHT_API int ssht_forward(ssht_plan_t plan, const void* f, void* flm, void* stream);

/* Adjoint of ssht_inverse: flm = A^H g where A is the linear map of ssht_inverse
 * (sum over the L x (2L-1) samples of g times conj(sY_lm); no quadrature weight).
 * g: [batch][L][2L-1] complex in; flm: [batch][L*L] complex out. */
SSHT_API int ssht_adjoint(ssht_plan_t plan, const void* g, void* flm, void* stream);

/* The paper's own forward transform (Sec. 3.4.2, eqn matrix_fwd): F_{m m'} (m' >= 0) of the
 * extended signal (the torus stage of ssht_forward without the weight convolution), then for each
 * m the upper triangular system in l solved by back substitution.  Exact in exact arithmetic for
 * band-limited f, but it loses accuracy as L grows (the instability the paper reports); it is
 * here to reproduce that behaviour next to ssht_forward.  FP64 plans only (SSHT_EUNSUPPORTED
 * otherwise).  f: [batch][L][2L-1] complex in; flm: [batch][L*L] complex out. */
SSHT_API int ssht_forward_triangular(ssht_plan_t plan, const void* f, void* flm, void* stream);

/* The table of Delta^l_{m'm} = d^l_{m'm}(pi/2) (Sec. 2.2; the plan's recursion) for
 * 0 <= l < L and 0 <= m', m <= l (the non-negative quadrant the paper precomputes, Sec. 4.1),
 * FP64, entry (l, m', m) at offset(l) + m'(l+1) + m with offset(l) = l(l+1)(2l+1)/6.
 * out: device or host buffer of L(L+1)(2L+1)/6 doubles. */
SSHT_API int ssht_wigner_delta(ssht_plan_t plan, double* out, void* stream);

/* The same Delta table as ssht_wigner_delta, for 1 <= L <= 512, computed without allocating
 * any device memory (the paper has no counterpart; this is a service for callers that cannot
 * allocate -- e.g. a host application that has reserved nearly all device memory for its own
 * pool, or a latency-critical loop that must not pay for cudaMalloc and the synchronisation it
 * can cause).  Needs no plan.  The recursion's scratch lives in a fixed array of about 2.1 MB
 * that every GPU loading this library holds until the process exits.
 * out: device buffer of L(L+1)(2L+1)/6 doubles, layout as in ssht_wigner_delta; the caller owns
 * it.  L outside [1, 512] or a NULL out returns SSHT_EINVAL before any device work.
 * The first call on a device sets that device up (looks up the address of the array, fills its
 * square-root table and waits for that fill on `stream`); made during stream capture it returns
 * SSHT_EINVAL and sets nothing up, so make it before any capture.  Later calls are asynchronous
 * on `stream`.  All calls share the one array: calls whose work overlaps on the GPU (on different
 * streams or devices' shared contexts) race and must be serialised by the caller.  If a grid
 * barrier inside the recursion exceeds its one-second spin limit the table is left incomplete
 * and out[0] (normally Delta^0_00 = 1) is set to NaN. */
SSHT_API int ssht_wigner_delta_noalloc(int L, double* out, void* stream);

/* Wait for the plan's outstanding work and report a latched kernel-side failure
 * (SSHT_ETIMEOUT) or a CUDA error; clears the latched status. */
SSHT_API int ssht_plan_check(ssht_plan_t plan);

/* Stages of a transform, for ssht_plan_profile_read. */
#define SSHT_STAGE_DELTA 0      /* recursion of Delta^l (and the spin column); for plans  */
                                /* whose recursion writes the A tiles, the forward's      */
#define SSHT_STAGE_INVERSE 1    /* inverse contraction (eqn fourier_coeff)                */
#define SSHT_STAGE_PROJECT 2    /* forward / adjoint contraction (harmonic projection)    */
#define SSHT_STAGE_FFT 3        /* torus DFTs: fused torus passes (FP32 plans) or cuFFT   */
#define SSHT_STAGE_TORUS 4      /* extension, phase, transpose and weight-product kernels */
#define SSHT_STAGE_PACK 5       /* operand packing for the tensor-core contraction        */
#define SSHT_STAGE_DELTA_INVERSE 6 /* the recursion writing the inverse's A tiles (3xTF32) */
#define SSHT_NUM_STAGES 7

/* Enable (1) or disable (0) per-stage timing: each stage of each later call is bracketed by
 * CUDA events recorded on the call's stream.  Enabling resets the accumulated times. */
SSHT_API int ssht_plan_profile(ssht_plan_t plan, int enable);

/* Accumulated per-stage device time in milliseconds (ms[i], i < nstages <= SSHT_NUM_STAGES)
 * and number of stage executions (count[i]) since profiling was enabled; synchronises the
 * device.  launches (may be NULL) receives the number of kernels this library launched for
 * the plan since it was created (cuFFT's kernels are not counted). */
SSHT_API int ssht_plan_profile_read(ssht_plan_t plan, double* ms, long long* count, int nstages,
                                    long long* launches);

/* The stage brackets recorded since profiling was enabled or last read (a timeline; the paper
 * has no counterpart), in recording order, at most cap of them: *n receives the number written.
 * stage[i] is an SSHT_STAGE_* id, lane[i] 0 for the caller's stream and 1 for the plan's second
 * stream (the recursion and the A-operand packing), t0[i] / t1[i] the bracket's start and end
 * in milliseconds after the earliest bracket's start.  A bracket starts when its stream reaches it,
 * which can precede the first kernel's start when that kernel waits for room on the GPU.  The
 * brackets are then folded into the totals of ssht_plan_profile_read.  Synchronises the device.
 * At most the last 8192 brackets are kept between reads. */
SSHT_API int ssht_plan_profile_trace(ssht_plan_t plan, int* stage, int* lane, double* t0, double* t1, int cap,
                                     int* n);

/* ---------------------------------------------------------------------------------------
 * Groups: many fields of uneven band-limit and spin in one call.  This extends the paper's
 * single-field transform (which has no batching) to a heterogeneous batch.
 * --------------------------------------------------------------------------------------- */
typedef struct ssht_group_s* ssht_group_t;

/* Create a group of n fields with band-limits L[i] (1..2048) and spins s[i] (|s[i]| < L[i]).
 * Fields are bucketed by (L, s) and each bucket is transformed by one plan of the given
 * precision and Delta mode; buckets of the same L share one Delta table (recompute mode: one
 * recursion per distinct L per call; cache mode: made here).  tune != 0 (FP32-class
 * precisions only) times the FP32, 3xTF32 and split-BF16 contractions on each bucket, the
 * tensor-core forms each with their own tuned shape (SSHT_FLAG_TUNE, SSHT_TUNE_CACHE), and keeps
 * the fastest.  Synchronises the device. */
SSHT_API int ssht_group_create(ssht_group_t* out, int n, const int* L, const int* s, int precision,
                               int delta_mode, int tune);
SSHT_API int ssht_group_destroy(ssht_group_t group);

/* Group order of the fields and their offsets in the flat buffers of the group calls:
 * order[k] (n entries) = caller's index of the k-th field; coeff_offset[k], grid_offset[k]
 * (n + 1 entries, the last = total) = complex-element offsets of field k's coefficients
 * [L^2] and samples [L][2L-1].  Any pointer may be NULL. */
SSHT_API int ssht_group_layout(ssht_group_t group, int* order, long long* coeff_offset, long long* grid_offset);

/* Buckets: on entry *nbuckets = capacity of the arrays (may be 0); on return the number of
 * buckets, and for the first min(capacity, number) buckets their L, s, field count and the
 * precision their plan uses (after tuning).  Array pointers may be NULL. */
SSHT_API int ssht_group_buckets(ssht_group_t group, int* nbuckets, int* L, int* s, int* count, int* precision);

/* Transforms of every field of the group; flat DEVICE buffers in group order (ssht_group_layout),
 * complex float (FP32-class precisions) or double (SSHT_FP64).  Buckets run concurrently on
 * group-owned streams forked from and joined back to `stream`. */
SSHT_API int ssht_group_inverse(ssht_group_t group, const void* flm, void* f, void* stream);
SSHT_API int ssht_group_forward(ssht_group_t group, const void* f, void* flm, void* stream);
SSHT_API int ssht_group_adjoint(ssht_group_t group, const void* f, void* flm, void* stream);

/* Capture inverse (flm -> f) followed by forward (f -> flm_out) of the whole group into one
 * CUDA graph (replacing a previous capture); ssht_group_replay launches it on `stream`.  The
 * buffers are bound at capture time.  Capturing launches nothing: it records on a private stream
 * and does not use its `stream` argument. */
SSHT_API int ssht_group_capture(ssht_group_t group, const void* flm, void* f, void* flm_out, void* stream);
SSHT_API int ssht_group_replay(ssht_group_t group, void* stream);

/* ssht_plan_tile_config of bucket `bucket` (in the order of ssht_group_buckets). */
SSHT_API int ssht_group_bucket_tile_config(ssht_group_t group, int bucket, int* cfg);

/* Wait for the group's work and report a latched kernel-side timeout (SSHT_ETIMEOUT). */
SSHT_API int ssht_group_check(ssht_group_t group);

/* Test hook (the paper has no counterpart): the n-th device allocation this library makes from
 * now on, in any call on any thread, fails as if the device were out of memory (cudaMalloc
 * returning cudaErrorMemoryAllocation); n = 0 disables it.  Plan and group creation then return
 * SSHT_ENOMEM after releasing what they had allocated.  n < 0 returns SSHT_EINVAL. */
SSHT_API int ssht_debug_fail_allocation(int n);

/* Test hook (the paper has no counterpart): the spin limit, in nanoseconds, of the waits of the
 * recursion that ssht_wigner_delta_noalloc launches from now on (it takes no plan, so
 * ssht_plan_set_wait_limit cannot reach it); 0 restores the default of one second.  A wait that
 * runs out makes the call's table start with a NaN (out[0]).  ns < 0 returns SSHT_EINVAL. */
SSHT_API int ssht_debug_noalloc_wait_limit(long long ns);

/* Index checks of the bounds-checked build (the paper has no counterpart; the library compiled
 * with -DSSHT_DEBUG, `python -m paper_0807_4494_gb300.build --debug`): in that build every checked
 * global access of the kernels (torus passes, packing, tensor-core contraction, recursions writing
 * the tiles, real-field and spin-pair kernels, SIMT contractions) tests its index against the extent
 * of its buffer and skips it when it lies outside.  *count receives the number of such accesses
 * since the last call, *site / *index / *extent the first one's site (an internal number), index
 * and extent (null pointers are skipped); the record is then cleared.  Synchronises the device.
 * Release builds check nothing: SSHT_EUNSUPPORTED. */
SSHT_API int ssht_debug_bounds(long long* count, int* site, long long* index, long long* extent);

/* The tensor-core contraction's shape (the paper has no counterpart): cfg[0] fields per GEMM
 * launch, cfg[1] pipeline stages, cfg[2] inverse work order (0 grouped by m, 1 longest first),
 * cfg[3] forward work order (0 grouped by m, 1 longest first).  SSHT_EUNSUPPORTED for plans
 * without tensor-core contraction. */
SSHT_API int ssht_plan_tile_config(ssht_plan_t plan, int* cfg);

/* Spin limit of the plan's device-side waits, in nanoseconds of the device clock (default 10^9, one
 * second): the Risbo recursion's hand-offs between CTAs (SSHT_FLAG_RISBO plans) and the
 * tensor-core contraction's pipeline waits.  A wait that exceeds it latches SSHT_ETIMEOUT in the
 * plan (read by ssht_plan_check), makes the kernel's other CTAs leave at their next wait, and leaves
 * the outputs of that call incomplete; copies and tensor-core operations already issued are waited
 * for before a CTA leaves, with the default limit.  A tiny limit makes the waits give up at once
 * (how the tests exercise this path).  ns <= 0 restores the default. */
SSHT_API int ssht_plan_set_wait_limit(ssht_plan_t plan, long long ns);

/* Message describing the last error on the calling host thread ("" if none). */
SSHT_API const char* ssht_last_error(void);

/* Library version as major*10000 + minor*100 + patch. */
SSHT_API int ssht_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SSHT_H */
