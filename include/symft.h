/*
 * symft.h -- C ABI of the B300 SymFT per-shot sampling engine.
 *
 * The engine samples noisy, adaptive, Clifford-dominated circuits with Pauli
 * rotations exactly, following SymFT (arxiv 2607.28600):
 *   - symft_compile runs the one-time compile step on the host: symbolic
 *     Clifford-Pauli frame factorization (Sec. 3, Eqs. factorization-invariant
 *     and factorized-circuit), adaptive stabilizer-coordinate planning over the
 *     stabilizer-destabilizer tableau (Sec. 4, seven instruction kinds), and
 *     lowering of the affine sign expressions into a flat device plan (Sec. 6,
 *     precompiled instruction descriptors).
 *   - symft_sample runs the per-shot sampler (Sec. 5, single-shot algorithm)
 *     on the GPU for many shots at once: counter-based noise and random bits,
 *     bit-packed sign evaluation (64 shots per word), and the dense
 *     active-state executor for PromoteRot / ActiveDiagRot / ActivePairRot /
 *     ActiveDiagMeas / ActivePairMeas.
 *
 * Output layout (every column output): column j occupies words
 * out[j*W .. j*W + W-1] with W = ceil(shots / 64); bit (r & 63) of word r >> 6
 * is shot r (relative to shot_offset).  Padding bits past `shots` are 0.
 * Columns: meas_out has one column per recorded measurement (record order),
 * det_out one per DETECTOR, obs_out one per observable index, discard_out a
 * single column.
 *
 * Randomness: shot r (absolute index shot_offset + r) of seed s draws from a
 * fixed Philox4x32-10 stream keyed by (s, channel ordinal, measurement
 * ordinal, shot block), so outputs do not depend on launch shapes, on how
 * shots are split across calls, or on the precision of the dense executor
 * (up to outcome flips where an FP32 branch probability sits within rounding
 * of the measurement uniform).
 *
 * Errors: every int-returning call returns SYMFT_OK (0) or a negative
 * symft_status; symft_last_error() returns a message for the calling thread.
 * Device code never traps: errors it detects are written to a status word
 * that symft_sample_ex reads back when args->check is set.
 */
#ifndef SYMFT_H
#define SYMFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SYMFT_OK = 0,
  SYMFT_E_PARSE = -1,        /* malformed circuit text */
  SYMFT_E_UNSUPPORTED = -2,  /* instruction outside the supported model */
  SYMFT_E_ARG = -3,          /* invalid argument (null plan, bad sizes, ...) */
  SYMFT_E_CAPACITY = -4,     /* plan exceeds a build limit (active width, ...) */
  SYMFT_E_NOMEM = -5,        /* host or device allocation failed */
  SYMFT_E_CUDA = -6,         /* CUDA runtime error */
  SYMFT_E_TIMEOUT = -7,      /* a bounded device wait expired */
  SYMFT_E_DEVICE = -8        /* device-side check failed (status word) */
} symft_status;

/* Shot offsets (symft_sample_args.shot_offset) are multiples of this: the
 * noise block of the random-stream specification.  Shards of one sample set
 * over several calls or GPUs start on such boundaries. */
#define SYMFT_SHOT_ALIGN 512

enum { SYMFT_POSTSELECT_NONE = 0, SYMFT_POSTSELECT_ALL = 1, SYMFT_POSTSELECT_LISTED = 2 };
enum { SYMFT_FP32 = 0, SYMFT_FP64 = 1 };
enum { SYMFT_OUT_DEVICE = 0, SYMFT_OUT_HOST = 1 };
/* Comparison forms of the paper's own GPU design (Sec. 6, GPU acceleration):
 * one CTA per shot with the shot's vector in shared memory, either sampling
 * the exogenous variables and evaluating every affine sign inside the shot's
 * CTA (IN_KERNEL), or reading them from packed columns that a separate
 * device-side pass computed for all shots (PREPASS: the bit-packed sign
 * kernel).  OFF is this library's batched executor choice. */
enum { SYMFT_PLAIN_OFF = 0, SYMFT_PLAIN_IN_KERNEL = 1, SYMFT_PLAIN_PREPASS = 2 };

typedef struct symft_plan symft_plan;   /* opaque; immutable after compile */

typedef struct {
  int postselect;          /* SYMFT_POSTSELECT_*: reject a shot at the first
                              fired postselected detector (Sec. 6, detector
                              postselection): NONE, ALL detectors, or the
                              LISTED ones */
  uint32_t n_post_dets;    /* LISTED: number of entries of post_dets */
  const uint32_t* post_dets;   /* LISTED: detector indices (annotation order,
                              0-based, duplicates allowed); caller-owned, read
                              only during symft_compile_ex; an index >= the
                              number of detectors is SYMFT_E_ARG */
  int no_simplify;         /* non-zero: skip the commutation-aware
                              simplification before planning (Sec. 6): same
                              output distribution, possibly a wider active
                              state and more dense instructions */
  int no_product_components;  /* non-zero: never use the product-component
                              representation (Sec. 6); by default it is used
                              when its cost model predicts a clear benefit */
  int executor;            /* dense executor preference, the numbering of
                              symft_info.dense_executor (1 register, 2 warp,
                              3 CTA, 4 wide, 5 / 6 product components on a warp
                              / a CTA); used when it can run the plan, else the
                              automatic choice; 0 = automatic.  symft_autotune
                              replaces it with its own pick */
  int wide_tile_bits;      /* wide executor: amplitudes per fused-window tile
                              as a power of two, 10..13 (FP32) or 10..12 (FP64;
                              larger values are clamped); 0 = the default (12 /
                              11).  symft_autotune replaces it with its own pick */
} symft_options;

/* Counts of a compiled plan (Sec. 5, sampling complexity). */
typedef struct {
  uint32_t n_qubits;
  uint32_t n_meas_events;     /* all measurements, recorded and hidden (resets) */
  uint32_t n_records;         /* recorded measurements: columns of meas_out */
  uint32_t n_dets;            /* columns of det_out */
  uint32_t n_obs;             /* columns of obs_out */
  uint32_t n_channels;        /* stochastic Pauli noise locations n_e */
  uint32_t k_max;             /* peak active width k_max^S */
  uint32_t n_instr[7];        /* PromoteRot, ActiveDiagRot, ActivePairRot,
                                 RandomMeas, DetMeas, ActiveDiagMeas,
                                 ActivePairMeas */
  uint32_t max_expr_weight;   /* d - 1 = max weight of an evaluated sign */
  uint32_t n_noise_components;/* symplectic noise bits carried by the plan */
  uint32_t n_targets;         /* bit-packed outputs the sign kernel computes */
  uint32_t n_causal;          /* active-measurement outcomes (m3 symbols) */
  uint64_t sign_xor_terms;    /* total (symbol, target) incidences */
  float tuned_ns_per_shot[2]; /* GPU time per shot of the autotuned shape
                                 (FP32, FP64); 0 until symft_autotune ran */
  uint64_t dense_amp_traffic;  /* amplitudes read + written per shot by the dense
                                  instructions as streaming passes (rotation 2 * 2^k,
                                  PromoteRot 3 * 2^k, measurement 2^k + 1.5 * 2^k);
                                  times 8 B (FP32) or 16 B (FP64) = vector bytes
                                  per shot when vectors live in HBM */
  uint64_t dense_flops;       /* floating-point operations per shot of the dense
                                 instructions (per amplitude: PromoteRot 4,
                                 ActiveDiagRot 6, ActivePairRot 10,
                                 ActiveDiagMeas 5, ActivePairMeas 13) */
  uint64_t wide_amp_traffic[2];/* amplitudes one shot moves through HBM when its
                                 vector lives there (the wide executor: runs of
                                 rotations fused into one pass per shared-memory
                                 tile, one pass per other rotation, sums and
                                 compaction per measurement), for FP32 and FP64
                                 tiles; times 8 B or 16 B = HBM bytes per shot */
  uint32_t dense_executor[2]; /* dense executor a call at FP32 / FP64 uses: 1
                                 register-resident warp per shot (k <= 5), 2 warp
                                 per shot with the vector in shared memory, 3 CTA
                                 per shot with the vector in shared memory, 4 wide
                                 (vectors in HBM, instruction-major passes), 5
                                 warp per shot on the product-component program,
                                 6 CTA per shot on it (workspace in shared memory);
                                 the product components when selected, else the
                                 smallest that fits, unless symft_autotune chose
                                 another; 0 without dense instructions */
  uint32_t pc_capacity;       /* product-component representation (Sec. 6):
                                 workspace amplitudes per shot */
  uint32_t pc_selected;       /* 1 when its cost model selected it (at most half
                                 the monolithic vector work, k_max > 5) */
  uint64_t pc_work[2];        /* amplitudes touched per shot: [0] product
                                 components (merges included), [1] monolithic */
  double sign_model[3];       /* algorithmic integer work of the bit-packed sign
                                 path per noise block of SYMFT_SHOT_ALIGN shots:
                                 [0] Philox4x32-10 blocks (head draws, the tail
                                 draws of the expected fires, random-measurement
                                 words), [1] expected noise fires, [2] 32-bit XOR
                                 operations (fired targets, random-measurement
                                 sources, record parents and output gathers) */
  uint32_t simplified[3];     /* commutation-aware simplification (Sec. 6):
                                 rotations merged into an earlier same-body
                                 rotation, merged rotations removed (angle a
                                 multiple of 2 pi), rotations removed as the
                                 branch phase of a later same-body measurement */
  uint32_t wide_tile_bits[2]; /* wide executor: amplitudes per fused-window
                                 tile, as a power of two, at FP32 / FP64 (the
                                 default, or the one symft_autotune chose) */
} symft_info;

/* One sampling request.  All pointers may be NULL to skip that output. */
typedef struct {
  uint64_t shots;          /* number of shots (>= 1) */
  uint64_t seed;           /* Philox key */
  uint64_t shot_offset;    /* absolute index of the first shot; a multiple of
                              SYMFT_SHOT_ALIGN */
  uint64_t* meas_out;      /* n_records * W words */
  uint64_t* det_out;       /* n_dets * W words */
  uint64_t* obs_out;       /* n_obs * W words */
  uint64_t* discard_out;   /* W words: 1 = shot rejected by postselection */
  int precision;           /* SYMFT_FP32 (default) or SYMFT_FP64 dense vectors */
  int out_location;        /* SYMFT_OUT_DEVICE (default) or SYMFT_OUT_HOST */
  int check;               /* non-zero: synchronise and read the device status */
  int plain;               /* SYMFT_PLAIN_*: the paper's GPU design, kept for
                              comparison (same bits): IN_KERNEL = per-shot
                              unpacked evaluation, one CTA per shot; PREPASS =
                              packed exogenous columns, then one CTA per shot;
                              a vector beyond shared memory is SYMFT_E_CAPACITY */
  void* stream;            /* cudaStream_t (NULL: legacy default stream) */
  double* prob_out;        /* n_causal * shots doubles, [j * shots + r]: Pr(m = 0)
                              of active measurement j (plan order) in shot r as
                              the executor computed it (Sec. 4, Eqs. of
                              ActiveDiagMeas / ActivePairMeas), rounded from
                              FP32 when precision = FP32; for checking branch
                              probabilities against an FP64 reference.  Under
                              postselection a rejected shot may stop its dense
                              work early: entries of measurements it never
                              reached are left unwritten */
  uint64_t* counts_out;    /* 2 + n_obs words: [0] kept shots, [1] discarded
                              shots, [2 + j] kept shots whose observable j is 1 */
} symft_sample_args;

/* One job of a batched request (symft_sample_batch). */
typedef struct {
  uint32_t plan;           /* index into the plans[] array of the call */
  uint32_t reserved0;
  uint64_t shots, seed, shot_offset;              /* as in symft_sample_args */
  uint64_t* meas_out;      /* DEVICE outputs (NULL skips), layout as above */
  uint64_t* det_out;
  uint64_t* obs_out;
  uint64_t* discard_out;
  int precision;           /* SYMFT_FP32 / SYMFT_FP64 */
  int plain;               /* SYMFT_PLAIN_* comparison form */
  uint64_t* counts_out;    /* DEVICE, 2 + n_obs words as in symft_sample_args */
} symft_job;

/* Compile circuit text (grammar below) with default options.
 * circuit_text: NUL-terminated, caller-owned, only read during the call.
 * *out receives a plan owned by the library; free with symft_plan_free.
 * Returns SYMFT_E_PARSE / SYMFT_E_UNSUPPORTED / SYMFT_E_CAPACITY on bad input.
 *
 * Grammar (Stim-like, one instruction per line, '#' comments):
 *   H S S_DAG SQRT_X SQRT_X_DAG X Y Z I  q...        single-qubit Cliffords
 *   CX|CNOT CY CZ SWAP  a b ...                      two-qubit Cliffords
 *   CX|CY|CZ rec[-k] q                               record-controlled Pauli
 *   R_X(t) R_Y(t) R_Z(t) T T_DAG q...; R_PAULI(t) X0*Z3*...  rotations
 *       R_P(t) = exp(-i t P / 2)  (Sec. 2)
 *   M MX MY MR MRX R RX q...; MPP X0*Z1 ...          Pauli measurements
 *       (R = hidden Z measurement + X feedback, RX likewise in X)
 *   X_ERROR(p) Y_ERROR(p) Z_ERROR(p) DEPOLARIZE1(p) DEPOLARIZE2(p)
 *   PAULI_CHANNEL_1(px,py,pz)                        stochastic Pauli noise
 *   DETECTOR rec[-k]...  OBSERVABLE_INCLUDE(i) rec[-k]...  REPEAT n { }
 *   TICK QUBIT_COORDS SHIFT_COORDS                    ignored
 */
int symft_compile(const char* circuit_text, symft_plan** out);

/* As symft_compile with options (NULL = defaults). */
int symft_compile_ex(const char* circuit_text, const symft_options* opt, symft_plan** out);

/* Fill *info with the plan's counts.  Host only, no GPU needed. */
int symft_plan_info(const symft_plan* plan, symft_info* info);

/* Measurement ordinals (0-based, every measurement event in circuit order,
 * resets included) of the plan's active measurements -- the ActiveDiagMeas /
 * ActivePairMeas instructions of Sec. 4, whose outcomes are the causal m3
 * symbols -- in plan order: entry j is the measurement whose branch
 * probability prob_out row j holds.  Writes min(capacity, n_causal) entries
 * to t_out (caller-owned host memory; NULL with capacity 0 only queries) and
 * returns n_causal, or a negative status.  Host only. */
int symft_plan_active_meas(const symft_plan* plan, uint32_t* t_out, uint32_t capacity);

/* Release a plan and its device workspace.  NULL is a no-op.  The caller must
 * make sure no sampling call on the plan is still running. */
void symft_plan_free(symft_plan* plan);

/* Sample `shots` shots with seed `seed` into caller-owned DEVICE buffers
 * (layout above), asynchronously on `cuda_stream` (a cudaStream_t or NULL).
 * Results are valid once the stream has been synchronised.  The first call
 * on a plan uploads it and allocates its workspace (cudaMalloc); later calls
 * reuse both.  Calls on one plan must not overlap (one stream at a time). */
int symft_sample(const symft_plan* plan, uint64_t shots, uint64_t seed,
                 uint64_t* meas_out, uint64_t* det_out, uint64_t* obs_out,
                 void* cuda_stream);

/* General form: shot offset, discard column, precision, host outputs
 * (out_location = SYMFT_OUT_HOST: the pointers are host memory, preferably
 * pinned; the call copies results back and returns after the copy). */
int symft_sample_ex(const symft_plan* plan, const symft_sample_args* args);

/* Pick the plan's launch shapes for one precision by timing candidates
 * (the dense executor kind among those that fit, resident sign-kernel CTAs
 * per SM, executor grid sizes, warps per CTA) on
 * `shots` shots with throw-away outputs; later calls on the plan use the
 * winner.  Runs synchronously on `cuda_stream`; allocates probe buffers. */
int symft_autotune(symft_plan* plan, uint64_t shots, int precision, void* cuda_stream);

/* Run many jobs (possibly of different plans) as ONE CUDA graph launch on
 * `cuda_stream`: every job's kernels are captured into a graph whose branches
 * (one per plan) run concurrently; jobs of the same plan run in order on its
 * branch (they share its workspace).  The graph is cached per thread and
 * updated in place when only parameters change.  Asynchronous; outputs are
 * device buffers.  Plans must not be used by another call meanwhile. */
int symft_sample_batch(const symft_plan* const* plans, int n_plans, const symft_job* jobs,
                       int n_jobs, void* cuda_stream);

/* Message describing the last error on the calling thread ("" if none). */
const char* symft_last_error(void);

/* Number of kernel launches the last sampling call on this thread issued. */
int symft_last_launch_count(void);

/* Sampling without any device allocation (the paper has no counterpart; this
 * is an integration aid).  Some callers cannot let a library call cudaMalloc:
 * frameworks whose caching allocator owns the device heap, or services with a
 * fixed memory budget.
 * This call runs the sampler's sign, warp-executor and finalize kernels on
 * caller-owned DEVICE outputs (same layout and results as symft_sample_ex,
 * up to the rare FP32 outcome flips the executors allow), and takes every
 * other byte it needs --
 * the plan copy, dense-sign and active-outcome columns, the status word, any
 * global active vectors -- from one fixed 32 MiB __device__ array that the
 * library holds on every GPU that loads it until the process exits.
 *   - Limit: a request whose scratch (plan image + (n_dense + n_active) * W
 *     words + detector scratch when postselecting without det_out) exceeds
 *     32 MiB returns SYMFT_E_CAPACITY before any GPU work; sample fewer shots
 *     per call.
 *   - Set-up: the first call made with a device current looks up the array's
 *     device address (cudaGetSymbolAddress) and the device's SM count.  Every
 *     call copies the plan image from host memory into the array
 *     (cudaMemcpyAsync on `cuda_stream`), so the plan must stay alive until
 *     the call's work on the stream is done.
 *   - Sharing: all calls share the array and it keeps the last call's
 *     contents; the call clears what must start at zero.  Calls that overlap
 *     on the GPU (other streams, other threads) race on it: serialise them.
 *   - No host outputs, no status readback; errors are reported by
 *     symft_noalloc_last_error().  Asynchronous on `cuda_stream`. */
int symft_sample_noalloc(const symft_plan* plan, uint64_t shots, uint64_t seed,
                         uint64_t shot_offset, uint64_t* meas_out, uint64_t* det_out,
                         uint64_t* obs_out, uint64_t* discard_out, int precision,
                         void* cuda_stream);

/* Message describing the last symft_sample_noalloc error on this thread. */
const char* symft_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SYMFT_H */
