/*
 * qsim.h -- C ABI of a GB300 (sm_103a) state-vector simulator for deep, fused
 * gate streams with mid-circuit measurement.
 *
 * The method is the one of "Deep Quantum Circuit Simulations of Low-energy
 * Nuclear States" (arXiv 2310.17739):
 *   - state vector of 2^n complex amplitudes, qubit q = bit q of the index
 *     (Section "State-Vector Simulation");
 *   - gates applied by Eq. (1q-op) (2x2 on amplitude pairs) and Eq. (2q-op)
 *     (4x4 on amplitude quadruples), the matrices need not be unitary;
 *   - gate fusion (Section "Gate Fusion"): 1q+1q -> C1, 2q absorbs 1q forward
 *     and backward -> C2, operand order canonicalised (first qubit lower),
 *     2q+2q on one pair -> C2;
 *   - mid-circuit measurement and its assertion variant (Section "Mid-Circuit
 *     Measurement Assertion"): Born probability, outcome, collapse,
 *     renormalisation; in assertion mode outcome 0 is asserted while P(0) > thr
 *     and the product of the asserted P(0) is tracked.
 *
 * Conventions for every function:
 *   - All functions return qsim_status; nothing throws or aborts across the ABI.
 *   - A context is single-threaded: calls on one context must not overlap.
 *     Different contexts may be used from different threads.
 *   - Work is enqueued on the context's CUDA stream in call order.  Functions
 *     that return results to host memory synchronise that stream; the others
 *     return without waiting.  Errors raised by device work that was enqueued
 *     earlier (a failed assertion, a CUDA fault) are reported by the next call
 *     that synchronises.
 *   - On an argument error (QSIM_E_INVAL) nothing is enqueued and the state is
 *     unchanged.  A failed assertion (QSIM_E_ZEROPROB) leaves the state as it
 *     was before that measurement and every later operation on the context is
 *     skipped until qsim_reset_state or qsim_set_state.
 *   - Pointers passed in are borrowed: gate, matrix and term arrays are fully
 *     consumed (copied) before the call returns, so the caller may free or
 *     reuse them immediately.
 *   - qsim_last_error returns a message for the most recent failure.
 */
#ifndef QSIM_H
#define QSIM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define QSIM_API __attribute__((visibility("default")))
#else
#define QSIM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qsim_ctx qsim_ctx;
typedef struct qsim_program qsim_program;

typedef enum {
    QSIM_C64 = 0,   /* complex64 amplitudes (float2), FP32 gate arithmetic,
                       FP64 probability / norm / expectation / renormalisation */
    QSIM_C128 = 1   /* complex128 amplitudes (double2), FP64 throughout */
} qsim_dtype;

typedef enum {
    QSIM_OK = 0,
    QSIM_E_INVAL = 1,     /* bad argument or malformed gate record */
    QSIM_E_OOM = 2,       /* device or host allocation failed */
    QSIM_E_CUDA = 3,      /* CUDA runtime error (message in qsim_last_error) */
    QSIM_E_ZEROPROB = 4,  /* assertion-mode measurement with P(0) <= threshold */
    QSIM_E_TIMEOUT = 5,   /* a bounded wait (qsim_sync_timeout) expired; the work goes on */
    QSIM_E_STATE = 6,     /* context unusable after an earlier failure */
    QSIM_E_CANCELED = 7   /* a served request cancelled before admission (qsim_server_cancel) */
} qsim_status;

/* ---------------------------------------------------------------- records --
 * One gate record (40 bytes).  q0 is the first operand: the control of
 * controlled gates.  For 2-qubit matrices the local basis index is
 * l = b_q0 + 2*b_q1 (row-major 4x4, rows = output).  C1 and C2 carry a general
 * (not necessarily unitary) 2x2 / 4x4 complex matrix at mats[mat ...]:
 * 8 / 32 doubles, interleaved (re, im), row-major.  Angles are in p[].
 * Gate definitions: the OpenQASM gate table of the paper (Table "Gates defined
 * in IBM OpenQASM") with RX/RY/RZ(t) = exp(-i t {X,Y,Z}/2), U1(l) = diag(1, e^{il}),
 * U2(p,l) = U3(pi/2,p,l), U3(t,p,l) = [[cos t/2, -e^{il} sin t/2],
 * [e^{ip} sin t/2, e^{i(p+l)} cos t/2]], CU1/CU3/CRX/CRY/CRZ/CY/CH controlled
 * versions, RXX/RZZ(t) = exp(-i t XX/2), exp(-i t ZZ/2).
 * MEASURE q0: flags bit 0 set = assertion mode (outcome 0 asserted).
 * RESET q0: a drawn measurement, then the |1> half moved onto |0>.
 * BARRIER: no effect on the state; stops fusion and reordering across it.
 */
typedef struct {
    uint16_t op;
    uint16_t flags;
    uint32_t q0;
    uint32_t q1;
    uint32_t mat;
    double p[3];
} qsim_gate;

enum {
    QSIM_OP_ID = 0, QSIM_OP_X = 1, QSIM_OP_Y = 2, QSIM_OP_Z = 3, QSIM_OP_H = 4,
    QSIM_OP_S = 5, QSIM_OP_SDG = 6, QSIM_OP_T = 7, QSIM_OP_TDG = 8,
    QSIM_OP_RX = 9, QSIM_OP_RY = 10, QSIM_OP_RZ = 11, QSIM_OP_U1 = 12,
    QSIM_OP_U2 = 13, QSIM_OP_U3 = 14, QSIM_OP_C1 = 15,
    QSIM_OP_CX = 32, QSIM_OP_CY = 33, QSIM_OP_CZ = 34, QSIM_OP_CH = 35,
    QSIM_OP_SWAP = 36, QSIM_OP_CRX = 37, QSIM_OP_CRY = 38, QSIM_OP_CRZ = 39,
    QSIM_OP_CU1 = 40, QSIM_OP_CU3 = 41, QSIM_OP_RXX = 42, QSIM_OP_RZZ = 43,
    QSIM_OP_C2 = 44,
    QSIM_OP_MEASURE = 64, QSIM_OP_RESET = 65, QSIM_OP_BARRIER = 66
};

#define QSIM_MEAS_ASSERT 1u

/* Pauli string: bit q of x_mask = X or Y on qubit q, bit q of z_mask = Z or Y. */
typedef struct {
    uint64_t x_mask;
    uint64_t z_mask;
    double coef;
} qsim_pauli_term;

/* ------------------------------------------------------------- compiling --
 * fusion   0: no fusion (one C1/C2 op per gate, still tiled into passes);
 *          1: the paper's four fusion stages (C1/C2 only);
 *          2: stages 1-4 plus Pauli-gadget recognition: a basis change, a CX
 *          network computing a parity, RZ, the network reversed and the
 *          basis undone become one rotation exp(-i theta P), kept with a
 *          Pauli frame (rotations with |cos| < |sin| are split, their Pauli
 *          factor folded into the frame, which is applied before every
 *          measurement or reset and at the end of the stream).
 * k_max    2: the paper's C1/C2 ops; 3..5: fused ops of a pass are further
 *          merged into dense 2^k x 2^k blocks of up to k_max qubits when the
 *          cost model says it is cheaper.
 * tile_bits m: dimension of a pass's tile (see qsim_schedule); 0 picks by
 *          dtype and n.  States with n <= tile limit run resident in one block.
 * threads  threads per block of the generic tile pass (256 or 512); 0 = auto,
 *          which also lets complex64 rotation passes run as register segments
 *          (2^(m-5) threads of 32 amplitudes).
 * chunk_gates  qsim_apply compiles and launches the stream in chunks of this
 *          many gates, overlapping host compilation with device work; 0 = a
 *          first chunk of 2^16 gates, each next one twice as long up to 2^20
 *          (the device starts sooner).  Every chunk ends with a Pauli-frame
 *          flush, so chunking changes rounding only.
 * lookahead  how many fused ops the pass scheduler may scan past an op that
 *          does not fit, pulling later ops on disjoint qubits forward; 0 = 64.
 * compile_threads  host threads compiling chunks ahead of the launcher; 0 = auto.
 * persistent  1: register-segment rotation passes (m <= 13) run as resident
 *          blocks that take tiles from a device counter and prefetch the next
 *          tile while computing the current one; 0: one block per tile.
 * graphs   CUDA-graph launches of tile passes.  qsim_run: 0 = each run of
 *          tile passes between two measurements of a compiled program is
 *          captured once as a CUDA graph when the program is run for the
 *          second time (programs of up to 2^21 tile passes; ~2.7 KB of device
 *          memory per pass) and replayed as one graph launch from then on;
 *          1 = captured at the first run.  qsim_apply (0 or 1): a chunk of
 *          >= 256 tile passes is captured and launched as graphs, which are
 *          destroyed once their launches have completed.  2 = never (every
 *          pass launched from the host).  Graphs are rebuilt after
 *          qsim_set_config; persistent = 1 never uses them.  The server
 *          launches its requests' passes from the host.
 * forced_low  low qubits kept in every tile so that tile rows are contiguous
 *          (0 = 4 for complex64, 3 for complex128: 128-byte rows; 1..8 any
 *          other count, raised to m - 10 when below).  Fewer forced qubits
 *          leave more tile dimensions for rotations (fewer passes) at the cost
 *          of shorter contiguous rows.  Resident-block passes (persistent = 1)
 *          need 4 and fall back to one block per tile below that.  At most
 *          4 for complex64 and 3 for complex128 (the longest contiguous row
 *          the tile kernels use); larger values are rejected.
 * struct_size  must equal sizeof(qsim_config) (qsim_config_init sets it):
 *          every call that reads a qsim_config refuses one whose size field
 *          differs (QSIM_E_INVAL), so a caller built against another layout
 *          of this struct is told so instead of having memory past its struct
 *          read or written.
 */
typedef struct {
    uint32_t struct_size;
    int32_t fusion;
    int32_t k_max;
    int32_t tile_bits;
    int32_t threads;
    int32_t chunk_gates;
    int32_t lookahead;
    int32_t compile_threads;
    int32_t persistent;
    int32_t graphs;
    int32_t forced_low;
} qsim_config;

/* The defaults (the paper's fusion, k_max 2, every other field 0 = automatic)
 * with struct_size set.  Start every qsim_config from this. */
QSIM_API void qsim_config_init(qsim_config *cfg);

typedef struct {
    uint64_t gates;          /* input records */
    uint64_t fused_ops;      /* dense ops after fusion (C1/C2/k-blocks) */
    uint64_t passes;         /* full-state sweeps of dense ops */
    uint64_t measurements;   /* MEASURE and RESET records */
    uint64_t device_bytes;   /* device memory held by a compiled program */
    uint64_t op_hist[8];     /* fused ops by qubit count k (index k) */
} qsim_program_info;

/* Allocator hook: alloc(bytes, stream, user) -> device pointer or NULL;
 * free(ptr, bytes, stream, user).  Frees are stream-ordered on `stream`. */
typedef void *(*qsim_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*qsim_free_fn)(void *ptr, size_t bytes, void *stream, void *user);

/* ------------------------------------------------------------- lifecycle -- */

/* New context holding a 2^n-amplitude state |0...0> on the current CUDA
 * device, enqueued on `stream` (NULL = legacy default stream).  Device memory
 * comes from alloc/free when given (both or neither), else cudaMallocAsync.
 * 1 <= n_qubits <= 34.  QSIM_E_OOM when the state does not fit. */
QSIM_API qsim_status qsim_create(int n_qubits, qsim_dtype dtype, void *stream,
                        qsim_alloc_fn alloc, qsim_free_fn free_fn, void *user,
                        qsim_ctx **out);
/* Releases the state and every buffer of the context (stream-ordered),
 * including the device memory of programs compiled on it that are still
 * alive; those programs can no longer be run but must still be passed to
 * qsim_program_free (which then only releases their host memory). */
QSIM_API qsim_status qsim_destroy(qsim_ctx *ctx);
QSIM_API qsim_status qsim_set_stream(qsim_ctx *ctx, void *stream);
QSIM_API qsim_status qsim_set_config(qsim_ctx *ctx, const qsim_config *cfg);
QSIM_API qsim_status qsim_get_config(const qsim_ctx *ctx, qsim_config *cfg);
/* Seed of the draws of in-stream MEASURE/RESET records (default 0). */
QSIM_API qsim_status qsim_set_seed(qsim_ctx *ctx, uint64_t seed);
/* Assertion-mode threshold: fail when P(0) <= thr (default 0, as in the paper). */
QSIM_API qsim_status qsim_set_assert_threshold(qsim_ctx *ctx, double thr);

/* ------------------------------------------------------- gate application --
 * Eq. (1q-op)/(2q-op) over a gate stream, after the fusion of Section "Gate
 * Fusion" and tiling into shared-memory passes.  Asynchronous.  Each MEASURE /
 * RESET record consumes the next draw ordinal k of the context and draws
 * u(seed, k) with the context seed. */
QSIM_API qsim_status qsim_apply(qsim_ctx *ctx, const qsim_gate *gates, size_t n_gates,
                       const double *mats, size_t n_mats);
/* Compile once into a device-resident program; run it any number of times.
 * The program belongs to the context that compiled it (same n and dtype). */
QSIM_API qsim_status qsim_compile(qsim_ctx *ctx, const qsim_gate *gates, size_t n_gates,
                         const double *mats, size_t n_mats, qsim_program **out);
/* Enqueue the program on the context's stream (asynchronous).  The first run
 * with graphs != 2 in the config may capture the program's runs of tile passes
 * as CUDA graphs on the host before enqueueing (see qsim_config.graphs). */
QSIM_API qsim_status qsim_run(qsim_ctx *ctx, const qsim_program *prog);
QSIM_API qsim_status qsim_program_get_info(const qsim_program *prog, qsim_program_info *info);
/* Releases the program's device memory (stream-ordered) and host memory; a
 * program holding CUDA graphs first synchronises the context's stream. */
QSIM_API qsim_status qsim_program_free(qsim_program *prog);

/* ------------------------------------------------------------ measurement --
 * Section "Mid-Circuit Measurement Assertion".  p0 = sum |a_i|^2 over bit q = 0,
 * p1 likewise (FP64).  mode 0: outcome 0 iff u(seed, k) < p0/(p0+p1), with
 * u(seed, k) = (word 0 of Philox4x64-10, counter (k,0,0,0), key (seed,0)) >> 11
 * times 2^-53 and k the context's next draw ordinal.  mode 1 (assertion):
 * outcome 0 when p0/(p0+p1) > thr, else QSIM_E_ZEROPROB with the state kept.
 * Then amplitudes with bit q != outcome are zeroed and the rest scaled by
 * 1/sqrt(p_outcome) (FP64 scale).  *prob = p_outcome/(p0+p1).  When outcome
 * is non-NULL the call synchronises and returns the result; when it is NULL
 * the measurement stays asynchronous (read it later with qsim_outcomes). */
QSIM_API qsim_status qsim_measure(qsim_ctx *ctx, int qubit, uint64_t seed, int mode,
                         int *outcome, double *prob);
/* Born probabilities of one qubit without collapsing (synchronises). */
QSIM_API qsim_status qsim_prob(qsim_ctx *ctx, int qubit, double *p0, double *p1);
/* Outcome log of every measurement since the last reset, in order:
 * outcomes[i] in {0, 1} (-1 = failed assertion), probs[i] = probability of the
 * recorded outcome.  Synchronises.  *n_total = records available. */
QSIM_API qsim_status qsim_outcomes(qsim_ctx *ctx, int32_t *outcomes, double *probs, size_t cap,
                          size_t *n_total);
/* Product of the asserted P(0) since the last reset (1 if none).  Synchronises. */
QSIM_API qsim_status qsim_success_prob(qsim_ctx *ctx, double *p);

/* ------------------------------------------------------------ expectation --
 * out[t] = coef_t * Re <psi| P_t |psi> with P_t |j> = i^{#Y} (-1)^{popcount(j & z)}
 * |j ^ x>, FP64 accumulation, for t < n_terms.  Synchronises. */
QSIM_API qsim_status qsim_expect(qsim_ctx *ctx, const qsim_pauli_term *terms, size_t n_terms,
                        double *out);

/* ------------------------------------------------------------------ state --
 * Copy the 2^n amplitudes out / in (bytes must equal 2^n * 8 for C64 or
 * 2^n * 16 for C128; interleaved re, im).  dst/src may be device or host.
 * qsim_state synchronises.  qsim_reset_state restores |0...0> and clears the
 * draw ordinal, the outcome log, the success product and a failed-assertion
 * mark. */
/* Final-state shots (the register read-out `measure q -> c` of Listing "Block
 * structure ...", taken `shots` times from the current state without collapse;
 * the counterpart of the measurement assertion's repeated runs, Section
 * "Mid-Circuit Measurement Assertion").  Shot s draws v = (word 0 of the
 * Philox4x64-10 block with counter (s, 1, 0, 0) and key (seed, 0)) >> 11 times
 * 2^-53 and takes the smallest index x with v * total < sum_{i <= x} |a_i|^2
 * (total = sum of all |a_i|^2; FP64 sums of FP64 squares); out[s] (host memory,
 * `shots` entries) receives the bits of x selected by qubit_mask packed in
 * ascending order.  The state is not changed and the measurement ordinal does
 * not advance.  QSIM_E_INVAL: mask beyond n qubits, out NULL with shots > 0,
 * or shots > 2^40; QSIM_E_OOM: no device memory for the 2^n / 512 partial sums
 * and the shots; synchronises. */
QSIM_API qsim_status qsim_sample(qsim_ctx *ctx, uint64_t qubit_mask, uint64_t shots, uint64_t seed,
                                 uint64_t *out);
QSIM_API qsim_status qsim_state(qsim_ctx *ctx, void *dst, size_t bytes, int dst_is_device);
QSIM_API qsim_status qsim_set_state(qsim_ctx *ctx, const void *src, size_t bytes, int src_is_device);
QSIM_API qsim_status qsim_reset_state(qsim_ctx *ctx);
/* Checkpoint / resume.  The draw of the k-th measurement depends only on
 * (seed, k) (see qsim_measure), so a run resumes exactly from a saved state
 * (qsim_state), the seed and the ordinal of the next draw: a context given
 * that state (qsim_set_state), seed (qsim_set_seed) and ordinal draws what the
 * original context would have drawn next.  get: the ordinal the next MEASURE /
 * RESET record or qsim_measure call will use (the number of draws since the
 * last qsim_reset_state, unless set); set: make the next draw use ordinal k.
 * Neither synchronises; set applies to work enqueued after it. */
QSIM_API qsim_status qsim_get_draw_ordinal(const qsim_ctx *ctx, uint64_t *k);
QSIM_API qsim_status qsim_set_draw_ordinal(qsim_ctx *ctx, uint64_t k);
/* Device pointer of the state (valid until qsim_destroy) and its size. */
QSIM_API qsim_status qsim_state_ptr(qsim_ctx *ctx, void **dptr, size_t *bytes);
/* ---------------------------------------------------------------- timing --
 * Sampled device timing of the tile passes (the gate-application sweep of
 * Eq. (1q-op)/(2q-op) over tiles).  After qsim_profile_start with every > 0, a
 * window of min(every, 16) consecutive tile-pass launches starting at every
 * every-th launch is bracketed by CUDA events recorded on the context stream
 * (dependent launches inside a window keep overlapping; a window closes early
 * at a measurement; at most 8192 windows; every = 0 stops).
 * qsim_profile_read synchronises and returns, for the sampled launches, the
 * summed device time of the windows (ms), the number of launches in them,
 * their algorithmic flops (8 * 2^k real flops per amplitude per dense k-qubit
 * op, 8 per rotation) and algorithmic bytes (one read and one write of the
 * state per launch), and the number of tile-pass launches since the start. */
QSIM_API qsim_status qsim_profile_start(qsim_ctx *ctx, int every);
QSIM_API qsim_status qsim_profile_read(qsim_ctx *ctx, double *sampled_ms, uint64_t *n_sampled,
                                       double *sampled_flops, double *sampled_bytes,
                                       uint64_t *n_launches);

/* Wait for all enqueued work; report deferred device errors. */
QSIM_API qsim_status qsim_sync(qsim_ctx *ctx);
/* qsim_sync with a bound on the host's wait: polls an event recorded behind
 * the work enqueued so far and returns QSIM_E_TIMEOUT if it has not completed
 * after `seconds` (>= 0).  On timeout nothing is cancelled: the work keeps
 * running, the context stays usable, and a later qsim_sync or
 * qsim_sync_timeout reports its outcome.  Otherwise as qsim_sync. */
QSIM_API qsim_status qsim_sync_timeout(qsim_ctx *ctx, double seconds);
QSIM_API const char *qsim_last_error(const qsim_ctx *ctx);
QSIM_API const char *qsim_status_string(qsim_status s);

/* ---------------------------------------------------------------- batches --
 * Many independent state vectors (for example one circuit structure with many
 * parameter sets, or circuits of uneven width) advanced together.  Each
 * instance i has n_qubits[i] qubits and its own compiled program (fused as in
 * Section "Gate Fusion", passes as for qsim_apply), seed and measurement log.
 * qsim_batch_run resets every state to |0...0> and runs every program: all
 * instances whose state fits one block's shared memory (n <= 14 for C64,
 * n <= 13 for C128, unless tile_bits forces tiling) run in ONE kernel launch,
 * one block per instance, with their measurements inside the kernel; larger
 * instances advance in lockstep, pass k of every one of them in a single
 * multi-state tile launch (their measurements as launches between steps).
 * Everything is enqueued on the batch stream.  Asynchronous.  The first run
 * after a compile, reconfiguration or reseeding is enqueued eagerly (and makes
 * every allocation); the second is captured into a CUDA graph that it and all
 * later runs launch with one call.  Each run restarts every state from
 * |0...0>, so runs are identical.
 * Memory: as for qsim_create (alloc/free hooks or cudaMallocAsync).  Argument
 * errors return QSIM_E_INVAL with nothing enqueued. */
typedef struct qsim_batch qsim_batch;
QSIM_API qsim_status qsim_batch_create(int count, const int32_t *n_qubits, qsim_dtype dtype,
                                       void *stream, qsim_alloc_fn alloc, qsim_free_fn free_fn,
                                       void *user, qsim_batch **out);
QSIM_API qsim_status qsim_batch_destroy(qsim_batch *b);
QSIM_API qsim_status qsim_batch_set_config(qsim_batch *b, const qsim_config *cfg);
/* The configuration of instance `index` alone (for example one tuned for its
 * width); it applies to that instance's next qsim_batch_compile.  Instances
 * run resident keep tile_bits = their n. */
QSIM_API qsim_status qsim_batch_set_instance_config(qsim_batch *b, int index, const qsim_config *cfg);
/* seeds[i]: draw seed of instance i (default 0). */
QSIM_API qsim_status qsim_batch_set_seeds(qsim_batch *b, const uint64_t *seeds);
/* Compile gates for instance `index` (host compiler) and upload the program,
 * replacing any earlier one.  Synchronous on the host compile only. */
QSIM_API qsim_status qsim_batch_compile(qsim_batch *b, int index, const qsim_gate *gates,
                                        size_t n_gates, const double *mats, size_t n_mats);
/* qsim_batch_compile for `count` instances at once: instance indices[k] gets
 * gates[k][0, n_gates[k]) (mats NULL, or mats[k] / n_mats[k] as in
 * qsim_batch_compile).  Every record is validated first (nothing changes on an
 * invalid one); the host compiles the programs on `threads` threads (0 =
 * auto), then uploads them in order, so the result equals count calls of
 * qsim_batch_compile.  The caller's arrays may be freed after the call. */
QSIM_API qsim_status qsim_batch_compile_many(qsim_batch *b, int count, const int32_t *indices,
                                             const qsim_gate *const *gates, const size_t *n_gates,
                                             const double *const *mats, const size_t *n_mats,
                                             int threads);
QSIM_API qsim_status qsim_batch_run(qsim_batch *b);
/* Expectation values for every instance: instance i uses terms
 * [term_offsets[i], term_offsets[i+1]) and writes out[t] = coef_t * Re <psi_i|P_t|psi_i>
 * for those t (FP64 accumulation, definition as qsim_expect).  Synchronises. */
QSIM_API qsim_status qsim_batch_expect(qsim_batch *b, const qsim_pauli_term *terms,
                                       const uint64_t *term_offsets, double *out);
/* State of instance `index` (bytes = 2^n * element size).  Synchronises. */
QSIM_API qsim_status qsim_batch_state(qsim_batch *b, int index, void *dst, size_t bytes,
                                      int dst_is_device);
/* Outcome log of instance `index` since the last qsim_batch_run (as
 * qsim_outcomes).  Synchronises; returns QSIM_E_ZEROPROB if that instance's
 * assertion failed. */
QSIM_API qsim_status qsim_batch_outcomes(qsim_batch *b, int index, int32_t *outcomes, double *probs,
                                         size_t cap, size_t *n_total);
/* Number of instances run resident (one block each, one launch) by qsim_batch_run. */
QSIM_API qsim_status qsim_batch_resident_count(const qsim_batch *b, int *count);

/* ---------------------------------------------------------------- serving --
 * A request loop with continuous admission.  qsim_server_submit copies a
 * request (its gate records) into a pending queue and returns at once; host
 * worker threads compile pending requests (fusion of Section "Gate Fusion",
 * passes as for qsim_apply); a native scheduler thread admits compiled
 * requests in arrival order whenever one of `slots` CUDA streams is idle and
 * the request's device memory (state + program) fits the remaining budget,
 * then enqueues the whole request on that slot's stream: state |0...0>, every
 * pass and measurement (draws with the request's seed), <Z_q> of every qubit,
 * and the read-back.  Requests on different slots overlap on the GPU; a
 * request's state stays resident until its result is read back, then its
 * memory returns to the budget and the next request is admitted.
 * Results are delivered through qsim_server_poll in completion order.
 * Times are host steady-clock seconds since the server was created. */
typedef struct qsim_server qsim_server;
typedef struct {
    uint64_t id;              /* as returned by qsim_server_submit */
    int32_t status;           /* QSIM_OK, QSIM_E_ZEROPROB, ... */
    int32_t n_qubits;
    int32_t n_meas;           /* MEASURE/RESET records in the request */
    int32_t pad;
    uint64_t outcomes;        /* bit i = outcome of the i-th of the first 64 measurements */
    double success;           /* product of asserted P(0) (1 if none) */
    double z[32];             /* <Z_q> for q < min(n, 32) */
    double t_submit, t_admit, t_done;
} qsim_result;
/* slots: concurrent requests (1..64); mem_budget: device bytes for states and
 * programs (0 = 80% of the free device memory at creation). */
QSIM_API qsim_status qsim_server_create(int slots, size_t mem_budget, qsim_dtype dtype,
                                        const qsim_config *cfg, int compile_threads,
                                        qsim_server **out);
QSIM_API qsim_status qsim_server_destroy(qsim_server *s);
/* t_submit < 0: use the current time; else the request's arrival time (s). */
QSIM_API qsim_status qsim_server_submit(qsim_server *s, int n_qubits, const qsim_gate *gates,
                                        size_t n_gates, const double *mats, size_t n_mats,
                                        uint64_t seed, double t_submit, uint64_t *id);
/* Move up to cap finished results into out; *n_out = how many. */
QSIM_API qsim_status qsim_server_poll(qsim_server *s, qsim_result *out, size_t cap, size_t *n_out);
/* Cancel a request that has not been admitted yet (still compiling, or
 * waiting for a slot or memory): its result is delivered at once with status
 * QSIM_E_CANCELED, t_admit = -1, and it never runs; the requests behind it
 * keep their order.  QSIM_E_INVAL if `id` is not waiting (unknown, already
 * admitted, finished or cancelled). */
QSIM_API qsim_status qsim_server_cancel(qsim_server *s, uint64_t id);
/* Counters: submitted, admitted, completed (results produced, cancelled ones
 * included), pending (neither admitted nor cancelled), running. */
QSIM_API qsim_status qsim_server_counts(const qsim_server *s, uint64_t *submitted, uint64_t *admitted,
                                        uint64_t *completed, uint64_t *pending, uint64_t *running);
QSIM_API double qsim_server_now(const qsim_server *s);

/* ------------------------------------------------ no-allocation variant --
 * The paper has no counterpart to this entry point; it serves callers that
 * own a state vector in device memory but may not allocate device memory
 * themselves or through the library (for example a plug-in whose host
 * framework hands out all device memory from its own fixed pool, or a
 * latency-critical loop where cudaMalloc/cudaFree, which can synchronise the
 * device, are not allowed).
 *
 * qsim_prob_noalloc: p0 = sum |a_i|^2 over bit `qubit` = 0 and p1 likewise
 * (FP64 accumulation, the same reduction as qsim_prob) of the caller's state
 * d_state (device pointer, 2^n_qubits interleaved amplitudes of `dtype`),
 * enqueued on `stream` (NULL = legacy default stream) and synchronised; the
 * results are written to the host doubles *p0, *p1.  It allocates nothing: the
 * reduction's scratch is a fixed 16.25 KiB array in the library's device
 * memory, present on every GPU that loads the library until the process
 * exits.  Limits: 1 <= n_qubits <= 34 and 0 <= qubit < n_qubits, otherwise
 * QSIM_E_INVAL with nothing enqueued; d_state and stream must belong to the
 * current CUDA device (QSIM_E_INVAL otherwise: the scratch used is that
 * device's copy); QSIM_E_CUDA on a CUDA error.  The first
 * call on each device looks up the scratch array's address
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture.  Every call on a device shares the scratch array, which
 * keeps the last call's contents (each call clears what must start at zero);
 * calls that may overlap on the GPU (different streams or threads) race on it
 * and must be ordered by the caller. */
QSIM_API qsim_status qsim_prob_noalloc(const void *d_state, int n_qubits, qsim_dtype dtype, int qubit,
                                       void *stream, double *p0, double *p1);

/* ------------------------------------------------------ OpenQASM 2.0 text --
 * qsim_parse_qasm: the gate records of an OpenQASM 2.0 program (the paper's
 * circuits are QASM files; Section "Simulator Framework", Table "Gates defined
 * in IBM OpenQASM").  Read: OPENQASM 2.x; include (qelib1 is built in);
 * qreg/creg (qubits numbered by declaration order, up to 64); the qelib1 gates
 * id x y z h s sdg t tdg rx ry rz u1 p u2 u3 u U cx CX cy cz ch swap crx cry crz
 * cu1 cp cu3 rxx rzz sx sxdg ccx cswap c3x c4x c3sqrtx rccx rc3x, applied to
 * qubits or broadcast over whole registers of one size; parameter expressions
 * (numbers, pi, + - * / ^,
 * unary minus, sin cos tan exp ln sqrt); `gate` definitions (expanded in
 * place); measure (-> a declared creg), reset, barrier (a full barrier).  Not
 * read: opaque, if.  ccx, cswap, rccx and rc3x become 1- and 2-qubit gates
 * (rccx / rc3x with the relative phases of the OpenQASM 2.0 standard header),
 * c3x, c4x and c3sqrtx exact controlled-X^t C2 records (X^(1/2) = the matrix of
 * sx), sx and sxdg C1 records; gate matrices and global phases are the
 * library's (see the record definitions above).  Writes gates[0..*n_gates),
 * mats[0..*n_mats) (doubles, for the C1 / C2 records) and *n_qubits.  Two-call use: with capacities too small
 * it returns QSIM_E_INVAL after setting *n_gates and *n_mats.  Errors: a
 * message "line L: ..." in err (err_cap bytes, NUL-terminated), QSIM_E_INVAL;
 * QSIM_E_OOM when host memory runs out.  Host only. */
QSIM_API qsim_status qsim_parse_qasm(const char *text, size_t len, qsim_gate *gates, size_t cap_gates,
                                     size_t *n_gates, double *mats, size_t cap_mats, size_t *n_mats,
                                     int *n_qubits, char *err, size_t err_cap);

/* ------------------------------------------- host-only compiler inspection --
 * These run the host compiler only (no GPU needed).
 *
 * qsim_fuse: the fusion stages of Section "Gate Fusion", the pass schedule
 * and (for k_max > 2) the k-qubit merge over gates[0..n_gates), exactly as
 * qsim_apply compiles one chunk.  Writes the fused ops in execution order:
 * out_k[i] = qubit count (1..5) or 0 for a MEASURE/RESET record
 * (then out_q[6i] = qubit, out_q[6i+1] = op code, out_q[6i+2] = flags);
 * out_q[6i .. 6i+k) = qubits, with bit j of the local matrix index = qubit
 * out_q[6i+j]; the 2^k x 2^k row-major complex matrix (interleaved doubles)
 * starts at out_mats[out_mat[i]].  out_k[i] = 7: a Pauli rotation
 * i^g exp(-i theta P), P = i^{|x & z|} X^x Z^z, with x = out_q[6i] |
 * out_q[6i+1] << 32, z = out_q[6i+2] | out_q[6i+3] << 32, g = out_q[6i+4] & 3,
 * (cos theta, sin theta) at out_mats[out_mat[i]]; out_q[6i+4] bit 2 marks a
 * Pauli-frame flush (theta = pi/2), which fusion level 2 emits before each
 * measurement or reset and at the end of the stream.  Returns QSIM_E_INVAL when a capacity is too
 * small (*n_ops / *n_mat_doubles then give the sizes needed). */
QSIM_API qsim_status qsim_fuse(int n_qubits, qsim_dtype dtype, const qsim_gate *gates, size_t n_gates,
                      const double *mats, size_t n_mats, const qsim_config *cfg,
                      uint8_t *out_k, uint32_t *out_q, uint64_t *out_mat, size_t cap_ops,
                      double *out_mats, size_t cap_mat_doubles,
                      size_t *n_ops, size_t *n_mat_doubles);
/* qsim_schedule: the pass schedule of the same compile.  A pass's tile is a
 * coset of an m-dimensional subspace V of the amplitude-index space GF(2)^n:
 * tile element t is amplitude x0 ^ (XOR of basis[j] over the set bits j of
 * t), the tile origin x0 ranging over the indices that are zero at every
 * pivot of V.  A dense op needs the unit vector of each of its qubits in V; a
 * Pauli rotation needs only its X mask in V.  With dense ops only, V is
 * spanned by unit vectors and the tile is the classic set of m qubits.
 * For pass i: out_tile[i] = the pivot positions of V (its qubits when V is
 * spanned by unit vectors; 0 for a measurement pass); out_first[i],
 * out_count[i] = its range in the op order qsim_fuse returns; if out_basis is
 * not NULL, out_basis[16 i + j] = basis vector j (j < m; the rest 0). */
QSIM_API qsim_status qsim_schedule(int n_qubits, qsim_dtype dtype, const qsim_gate *gates, size_t n_gates,
                          const double *mats, size_t n_mats, const qsim_config *cfg,
                          uint64_t *out_tile, uint64_t *out_first, uint32_t *out_count,
                          uint64_t *out_basis, size_t cap, size_t *n_passes);

#ifdef __cplusplus
}
#endif
#endif /* QSIM_H */
