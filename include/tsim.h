/*
 * tsim.h -- C ABI of the GB300 per-shot sampler for noisy Clifford+T circuits.
 *
 * The library implements the compile-once / sample-many pipeline of Tsim
 * (Haenel, Luo, Zhao, "Tsim: Fast Universal Simulator for Quantum Error
 * Correction", arXiv 2604.01059):
 *
 *   tsim_compile   Sec. "Simulation pipeline" and Appendices "Pauli noise
 *                  channels", "Channel reduction", "Stabilizer decompositions",
 *                  "Parameterized evaluation of Clifford ZX diagrams": the
 *                  circuit becomes a doubled, parameterised diagram, Clifford
 *                  rewriting separates detectors (Eq. detector_sampling,
 *                  f = T e mod 2) from the observable part, and every marginal
 *                  of Algorithm 1 becomes a sum of stabilizer terms
 *                  P = sum_t c^t prod_k h(alpha_k^t, beta_k^t; a_k, b_k)
 *                  (Eqs. parities, phase_pair, scalar_product).
 *   tsim_sample    Sec. "Complexity", paragraph "Sampling", Eq. detector_sampling
 *                  and Algorithm 1: per shot, sample error mechanisms, compute
 *                  f, evaluate the marginals exactly and draw the outputs; on
 *                  one GPU, in hand-written sm_103a kernels.
 *
 * Conventions for every entry point:
 *   - Status codes only; no C++ exception crosses this boundary.  On failure
 *     tsim_last_error() returns a thread-local message.
 *   - Programs are opaque, owned by the library, freed with tsim_program_free.
 *   - Device buffers are caller-owned (e.g. torch tensors); the library never
 *     frees them.  Host buffers likewise.
 *   - Records are row-major [shot][word] uint64, record bit b of a row is bit
 *     (b & 63) of word (b >> 6); unused high bits are zero.
 *   - Output is a pure function of (program, seed, global shot index): the
 *     Philox4x32-10 counter of shot s is (s lo, s hi, stream, block) with key
 *     (seed lo, seed hi); stream 0 drives noise channel c (word c%4 of block
 *     c/4) or, in geometric-gap noise sampling, stream 2 gives the noise
 *     words in the order they are used (word j = word j%4 of block j/4);
 *     stream 1 drives autoregressive output i (word i%4 of block i/4).
 */
#ifndef TSIM_H
#define TSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TSIM_OK = 0,
  TSIM_ERR_PARSE = 1,            /* malformed circuit or program text */
  TSIM_ERR_UNSUPPORTED_GATE = 2, /* instruction outside the supported set */
  TSIM_ERR_CHI_BUDGET = 3,       /* stabilizer terms exceed chi_budget */
  TSIM_ERR_OVERFLOW_BOUND = 4,   /* exact accumulation would not fit the kernel's integers */
  TSIM_ERR_CUDA = 5,             /* a CUDA call failed (message names it) */
  TSIM_ERR_OOM = 6,              /* host or device allocation failed */
  TSIM_ERR_ARG = 7,              /* invalid argument (NULL, size, mode mismatch) */
  TSIM_ERR_ZERO_PROB = 8,        /* a sampled prefix had P_prev = 0 (compiler bug guard) */
  TSIM_ERR_TIMEOUT = 9,          /* a bounded device wait gave up */
  TSIM_ERR_INTERNAL = 10         /* internal invariant violated */
} tsim_status;

typedef struct tsim_program tsim_program;

enum { TSIM_MODE_DETECTORS = 0, TSIM_MODE_MEASUREMENTS = 1 };
enum { TSIM_DECOMP_HEURISTIC = 0, TSIM_DECOMP_LEARNED = 1, TSIM_DECOMP_SINGLE_T = 2, TSIM_DECOMP_PAIRS = 3,
       TSIM_DECOMP_CAT5 = 4 };

typedef struct {
  int mode;              /* TSIM_MODE_DETECTORS: records are detector + observable bits
                            (Sec. "Sampling detectors and observables"); TSIM_MODE_MEASUREMENTS:
                            records are the measurement outcomes (plus detectors /
                            observables computed from them by Eq. xor). */
  int decomp;            /* stabilizer decomposition policy (Appendix "Stabilizer
                            decompositions"), non-Clifford vertices in ascending order:
                            CAT5 = the partial Cat5 decomposition (Eq. cat5) on groups
                            of five (3 terms per group, each keeping one non-Clifford
                            vertex: alpha = log2(3)/4), BSS pairs (2 terms, alpha = 0.5)
                            when two to four remain, a T-state cut for the last one;
                            HEURISTIC (default) = as CAT5, except that the first two are
                            split as a BSS pair while two consecutive vertices have
                            phases that cancel (a T gate's ket and bra copies, which
                            the pair split removes together); PAIRS = BSS pairs only;
                            SINGLE_T = one T-state cut at a time; LEARNED = the three
                            cut units the cut-order network ranks best split first,
                            each followed by the heuristic order, and every unit in the
                            network's order, against the heuristic itself (kept only
                            with strictly fewer terms). */
  uint64_t chi_budget;   /* maximum stabilizer terms per marginal; 0 = 1<<20 */
  int channel_reduction; /* 1 = apply the four steps of Appendix "Channel reduction" */
  uint64_t total_budget; /* maximum stabilizer terms summed over all marginals; 0 = none.
                            Both budgets fail with TSIM_ERR_CHI_BUDGET as soon as they
                            are exceeded. */
} tsim_compile_opts;

typedef struct {
  int mode;
  int num_qubits;
  int num_measurements;   /* N_m */
  int num_detectors;      /* N_d */
  int num_observables;    /* N_o */
  int num_error_bits;     /* raw error bits e (Appendix "Pauli noise channels") */
  int num_channels;       /* reduced noise channels sampled per shot */
  int num_f;              /* f variables after GF(2) elimination (Eq. detector_sampling) */
  int num_random;         /* outputs drawn by Algorithm 1 */
  int num_outputs;        /* all outputs in autoregressive order */
  int num_chains;         /* independent autoregressive chains (connected components) */
  int num_tables;         /* marginal tables (chain normalisations included) */
  int x_words;            /* 64-bit words of the per-shot vector X = (f, random outputs) */
  uint64_t total_terms;   /* sum over tables of stabilizer terms chi_j */
  uint64_t max_terms;     /* largest chi_j */
  int max_factors;        /* largest number of factors m in one term */
  int meas_words, det_words, obs_words; /* record row widths in uint64 words */
  uint64_t device_classes;  /* terms left after merging terms with equal factor lists
                               (exact: their c^t are summed in Z[w]) */
  uint64_t device_parities; /* distinct factor parities over all tables */
  int device_status;        /* TSIM_OK if the program can run on the GPU */
} tsim_program_info_t;

/* Compile a Stim-format circuit (text, len bytes; the Clifford+T subset: I X Y Z
 * H S S_DAG SQRT_X SQRT_X_DAG T T_DAG CX CY CZ SWAP (and CX/CY/CZ with a rec[-k]
 * control), R RX M MX MR MRX (optional flip probability), X_ERROR Y_ERROR
 * Z_ERROR DEPOLARIZE1 DEPOLARIZE2 PAULI_CHANNEL_1 PAULI_CHANNEL_2, DETECTOR,
 * OBSERVABLE_INCLUDE, REPEAT, TICK, QUBIT_COORDS, SHIFT_COORDS, and the
 * rotations R_X(t) R_Y(t) R_Z(t) U3(a, b, c) with angles in units of pi,
 * Sec. "Methods") into a program.  Rotations by multiples of pi/4 stay in the
 * exact ring; other angles make their chain's tables floating point: the
 * marginals are then computed in complex double, and Algorithm 1 rounds each
 * ratio P_1 / P_prev to the nearest FP32 value q and draws 1 iff U < q 2^32.
 * opts may be NULL (detector mode, heuristic, default budget, reduction on).
 * On success *out owns a new program. */
tsim_status tsim_compile(const char* text, size_t len, const tsim_compile_opts* opts,
                         tsim_program** out);

/* Fill *out with the program's sizes (used to size the record buffers). */
tsim_status tsim_program_info(const tsim_program* prog, tsim_program_info_t* out);

/* Number of stabilizer terms of marginal table t (0 <= t < num_tables). */
tsim_status tsim_program_table_terms(const tsim_program* prog, int t, uint64_t* terms);

/* Terms and total factors (sum over terms of m_t) of marginal table t. */
tsim_status tsim_program_table_stats(const tsim_program* prog, int t, uint64_t* terms, uint64_t* factors);

/* Sample shots [shot_offset, shot_offset + shots) on the current CUDA device,
 * asynchronously on cuda_stream (a cudaStream_t; NULL = legacy default stream).
 * Outputs are DEVICE pointers, caller-owned, each may be NULL when not wanted:
 *   d_meas   [shots][meas_words]  measurement records (measurement mode only,
 *                                 must be NULL in detector mode -> TSIM_ERR_ARG)
 *   d_det    [shots][det_words]   detector bits
 *   d_obs    [shots][obs_words]   observable bits
 *   d_accept [shots]              1 iff every detector bit of the shot is 0
 * The first call for a program uploads its tables (synchronously).  Errors
 * detected on the device are reported by the next tsim_sync/tsim_sample. */
tsim_status tsim_sample(const tsim_program* prog, uint64_t shots, uint64_t seed,
                        uint64_t shot_offset, uint64_t* d_meas, uint64_t* d_det,
                        uint64_t* d_obs, uint8_t* d_accept, void* cuda_stream);

/* End-to-end variant with HOST buffers (same layout as tsim_sample): samples
 * into device staging buffers, copies the records back and synchronises.
 * Launches of more than 2^19 shots run in up to 8 chunks, the copies of one
 * chunk (on a stream of the library's own) overlapping the sampling of the
 * next; the records are the same.  The staging buffers, copy stream and
 * events are kept per host thread and device (until the process exits);
 * page-locked host buffers make the copies fastest. */
tsim_status tsim_sample_host(const tsim_program* prog, uint64_t shots, uint64_t seed,
                             uint64_t shot_offset, uint64_t* h_meas, uint64_t* h_det,
                             uint64_t* h_obs, uint8_t* h_accept, void* cuda_stream);

/* Batched launch: n programs, each with its own shots / seed / offset and its
 * own output pointers (arrays of n device pointers; entries may be NULL), in
 * persistent launches over (program, shot-block) work items: one for the
 * programs without bit-sliced tables and one for those with (each with its
 * own register budget).  Every record equals what tsim_sample gives for the
 * same program, seed and shot.  Synchronises cuda_stream before returning (the
 * plan it builds is freed). */
tsim_status tsim_sample_batch(const tsim_program* const* progs, int n, const uint64_t* shots,
                              const uint64_t* seeds, const uint64_t* shot_offsets,
                              uint64_t* const* d_meas, uint64_t* const* d_det,
                              uint64_t* const* d_obs, uint8_t* const* d_accept,
                              void* cuda_stream);

/* Same arguments, layout and records as tsim_sample, for callers that cannot
 * allocate device memory (for example code running inside an allocator or
 * memory pool it does not own, or a host that has carved up device memory in
 * advance).  The paper has no counterpart: this is an interface of this
 * library only.  The call allocates nothing, host or device: the program's
 * device tables, which tsim_sample keeps in memory it allocates once per
 * program, are packed into a fixed 4 MiB array in the library's device
 * memory (every GPU that loads the library holds it until the process exits)
 * and copied there on cuda_stream before the kernel runs.  The array's first
 * 256 bytes hold the call's device status word; the tables follow.
 *   - Programs whose packed tables exceed 4 MiB - 256 bytes are rejected with
 *     TSIM_ERR_ARG before anything is written; tsim_sample has no such limit.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current); make that first call
 *     before any stream capture.  Every later call outside a stream capture
 *     looks the address up again, so a cudaDeviceReset of the device (which
 *     moves the array) is picked up by the next such call.
 *   - Every call reuses the same array and rewrites all of it that the kernel
 *     reads.  Calls whose work overlaps on the GPU (different streams without
 *     ordering between them) race on the array and must not be issued; calls
 *     on one stream are ordered and safe.  Host threads are serialised.
 * Device-side errors are reported by tsim_sync, as for tsim_sample (which
 * clears the status word after reading it). */
tsim_status tsim_sample_noalloc(const tsim_program* prog, uint64_t shots, uint64_t seed,
                                uint64_t shot_offset, uint64_t* d_meas, uint64_t* d_det,
                                uint64_t* d_obs, uint8_t* d_accept, void* cuda_stream);

/* Validation form of tsim_sample (Appendix "Validation": probabilities of bit
 * strings; Eqs. parities, phase_pair, scalar_product): the same kernel, grid
 * and records as tsim_sample, and in addition, for the n_dump shots whose
 * indices within the launch are dump_shots[0..n_dump) (host array, distinct,
 * each < shots), an exact copy of every marginal table the kernel evaluated
 * for that shot.  h_dump (host, caller-owned) receives, per dumped shot in the
 * order given, per evaluation (each chain's normalisation in chain order,
 * then the table of each random output in output order: num_chains +
 * num_random evaluations), 6 + x_words int64 values: the table index, the
 * four Z[w] coefficients c0..c3 and the sqrt2 exponent k of the kernel's
 * value (c0 + c1 w + c2 w^2 + c3 w^3) sqrt2^k, then the words of X at which
 * the kernel evaluated it.  For a floating-point table (arbitrary rotations)
 * c0 and c1 hold the IEEE-754 bits of the real and imaginary parts of its
 * complex value, c2 = c3 = 0, and k = INT32_MIN.  Allocates and frees device scratch, and
 * synchronises cuda_stream.  At most 2^31 shots. */
tsim_status tsim_debug_sample(const tsim_program* prog, uint64_t shots, uint64_t seed, uint64_t shot_offset,
                              uint64_t* d_meas, uint64_t* d_det, uint64_t* d_obs, uint8_t* d_accept,
                              const uint64_t* dump_shots, int n_dump, int64_t* h_dump, void* cuda_stream);

/* How the error mechanisms of a shot are drawn (Sec. "Detectors"):
 *   0  one Philox word per reduced channel (stream 0, word c of the shot);
 *   1  geometric gaps: the channels, sorted by firing probability, are cut
 *      into groups (runs chosen to minimise the expected words per shot);
 *      a group's Q is its most likely channel's outcome-0 threshold, so its
 *      largest firing probability is 1 - Q/2^32; candidates are
 *      Bernoulli(1 - Q/2^32) trials along a
 *      group, each gap drawn from one word U as the largest k (up to the
 *      channels left) with U < T_k, T_0 = 2^32, T_k = floor(T_{k-1} Q / 2^32);
 *      a candidate's word V, mapped onto [Q, 2^32) by Q + floor(V (2^32 - Q)
 *      / 2^32), picks its outcome by the channel's own thresholds.  All words
 *      come from stream 2 in the order they are used.  Cost per shot: one
 *      word per group plus two per candidate, against one word per channel.
 *  -1  whichever of the two is expected to draw fewer words (the default at
 *      compile and load time: a program file records the mode it was saved
 *      with).
 * Re-packs the device tables (keeping their layout settings); the records
 * change with the mode (both sample the same distribution, within 2^-32 per
 * channel and gap step).  Must not be called while a launch of the program
 * is in flight or while a batch created from it exists. */
tsim_status tsim_program_set_noise_sampling(tsim_program* prog, int mode);

/* Bytes of the program's packed device tables (what tsim_sample uploads once
 * per program and tsim_sample_noalloc copies on every call). */
tsim_status tsim_program_device_bytes(const tsim_program* prog, uint64_t* bytes);

/* out[0] = noise sampling mode (0 or 1), out[1] = groups (mode 1), out[2] =
 * random words per shot of mode 0 (channels that can fire), out[3] = expected
 * random words per shot of mode 1 (an upper bound: one per group plus two per
 * expected candidate). */
tsim_status tsim_program_noise_info(const tsim_program* prog, double out[4]);

/* Reusable batched launch (Appendix "Additional benchmarks": batched sampling;
 * here heterogeneous programs share persistent kernels).  tsim_batch_create
 * uploads every program, lays out the (program, shot-block) work items,
 * (autotune = 1) autotunes the shots per work item (32, 128 or 512; 128
 * without autotuning; each item is taken by one warp) and the resident
 * blocks per SM (4, 8, 16) by timing each candidate on the real batch,
 * then times the other launch form (each program's own sampling kernel, one
 * after another) and keeps the faster form, and captures the launch
 * ("reset the work counter + persistent launch" for each group of programs
 * with equal padded X width and with or without bit-sliced tables, or the
 * programs' launches) in a CUDA graph.  Both forms write the same records.  tsim_batch_launch
 * replays that graph on cuda_stream (asynchronous); the output pointers
 * given at creation are written on every launch.  The batch owns a small
 * device allocation (descriptors, work counter) freed by tsim_batch_free,
 * which must not be called while a launch is in flight.
 * tsim_batch_info: out[0] shots per work item, out[1] blocks per SM,
 * out[2] work items, out[3] 1 if a graph is captured, out[4] words of the
 * widest X,
 * out[5] autotuned launch time in microseconds (0 without autotuning),
 * out[6] launch form (0 persistent, 1 one launch per program).
 * autotune = 0 keeps the persistent form with its defaults; autotune = 2
 * takes the one-launch-per-program form without timing anything. */
typedef struct tsim_batch tsim_batch;
tsim_status tsim_batch_create(const tsim_program* const* progs, int n, const uint64_t* shots,
                              const uint64_t* seeds, const uint64_t* shot_offsets,
                              uint64_t* const* d_meas, uint64_t* const* d_det,
                              uint64_t* const* d_obs, uint8_t* const* d_accept, int autotune,
                              tsim_batch** out);
tsim_status tsim_batch_launch(tsim_batch* batch, void* cuda_stream);
tsim_status tsim_batch_info(const tsim_batch* batch, int64_t out[7]);
void tsim_batch_free(tsim_batch* batch);

/* Wait for cuda_stream and report any device-side error status. */
tsim_status tsim_sync(void* cuda_stream);

/* Exact value of marginal table t at the per-shot vector X (x_words uint64,
 * host memory): P = sum_t c^t prod_k h(...) returned as
 * (c0 + c1 w + c2 w^2 + c3 w^3) * sqrt2^(*sqrt2_exp), w = e^{i pi/4}.
 * Used to validate compiled marginals against exact probabilities
 * (Appendix "Validation"). */
tsim_status tsim_eval_table(const tsim_program* prog, int t, const uint64_t* x,
                            int64_t out_zw[4], int32_t* sqrt2_exp);

/* Value of marginal table t at X in complex double, for every table and in
 * particular for those of circuits with arbitrary rotations (R_X, R_Y, R_Z,
 * U3 at angles that are not multiples of pi/4), whose terms carry phases
 * e^(i pi t) outside Z[w]: out[0] + i out[1].  tsim_eval_table refuses such
 * tables with TSIM_ERR_ARG. */
tsim_status tsim_eval_table_float(const tsim_program* prog, int t, const uint64_t* x, double out[2]);

/* Map raw error bits e (num_error_bits bytes, 0/1) to X = (T e) in the
 * program's X layout (x_words words), Eq. detector_sampling. */
tsim_status tsim_raw_to_x(const tsim_program* prog, const uint8_t* e, uint64_t* x);

/* Serialise / restore a program (text format documented in the program
 * writer; both directions are exact). */
tsim_status tsim_program_save(const tsim_program* prog, const char* path);
tsim_status tsim_program_load(const char* path, tsim_program** out);

void tsim_program_free(tsim_program* prog);

/* Thread-local description of the last failure on this thread. */
const char* tsim_last_error(void);

/* Integer-issue microbenchmark of the current GPU (the paper has no
 * counterpart; it states the ALU roofline of the sampling kernel): op 0 =
 * 32-bit three-input logic, 1 = 32-bit multiply-add, 2 = 32x32->64 multiply
 * (Philox's product), 3 = popcount.  *ops_per_s receives results per second
 * of that instruction class over the whole GPU.  Allocates 4 bytes. */
tsim_status tsim_measure_int_peak(int op, double* ops_per_s);

/* Per-table statistics of the packed device tables of table t:
 * out[0] = classes (terms after merging equal factor lists), out[1] = factors
 * over those classes, out[2] = distinct factor parities. */
tsim_status tsim_program_device_table_stats(const tsim_program* prog, int t, uint64_t out[3]);

/* Device table layout.  Every marginal table is packed for the GPU in one
 * of three layouts: 0 = SCALAR (one thread per shot; the table's distinct
 * factor parities (Eq. parities) are evaluated once per shot and indexed per
 * factor), 1 = BASIS (as SCALAR, with parities given by their coordinates in
 * a GF(2) basis of their span, for tables with many distinct parities),
 * 2 = SLICED (warp-cooperative and bit-sliced: a warp evaluates 32 shots at
 * once, bit s of a 32-bit word belonging to shot s; lane l of the warp carries
 * term l of a batch of 32 terms, and each factor of Table "Types of
 * parameterized phase terms" acts as one or two word operations on the term's
 * phase exponent J mod 8 and its vanishing flag).  SLICED applies to tables
 * whose terms are monomials of shot-independent magnitude (Node, phase and
 * pi-pair factors at Clifford angles).  All layouts give identical records.
 *
 * tsim_program_set_table_layout re-packs the program: tables with at least
 * sliced_min_terms terms (after merging terms with equal factor lists) use
 * SLICED when they qualify; sliced_min_terms < 0 disables SLICED.  A SLICED
 * table whose batches have at most stage_rows operation rows each is read
 * through shared memory (each warp bulk-copies the next batch's rows while
 * it evaluates the current one); 0 reads rows from global memory through
 * L1, < 0 takes the default (0).  A SLICED table is split into segments of
 * consecutive terms whose distinct parities fit segment_parities 32-bit words
 * of shared memory per warp (each segment forms its own parity words; fewer
 * words let more warps reside per SM); <= 0 takes the default (1536).  The
 * defaults at compile / load time are 4, 0 and 1536.
 * It frees the program's uploaded
 * device copy, so it must not be called while a launch of the program is in
 * flight or while a batch created from it (tsim_batch_create) exists.
 *
 * tsim_program_device_table_layout: out[0] = layout of table t, out[1] =
 * batches of 32 terms (over all segments), out[2] = padded operation rows,
 * out[3] = operations before padding (lane-rows of real factors), out[4] =
 * integer lane-operations one warp executes on the table for its 32 shots,
 * out[5] = the same count without padding (each term's own rows, one batch
 * epilogue per term) (out[1..5] are 0 unless SLICED). */
tsim_status tsim_program_set_table_layout(tsim_program* prog, int64_t sliced_min_terms, int32_t stage_rows,
                                          int32_t segment_parities);
tsim_status tsim_program_device_table_layout(const tsim_program* prog, int t, uint64_t out[6]);

/* Output entries of the packed program: out[0] = entries the kernel walks
 * per shot, out[1] = runs (in detector mode, consecutive single-bit
 * deterministic outputs without a constant that read consecutive bits of X,
 * Eq. detector_sampling, copied into the record by word shifts), out[2] =
 * outputs covered by runs. */
tsim_status tsim_program_device_output_stats(const tsim_program* prog, uint64_t out[3]);

/* Self-check of the bit-sliced layout (host only, no GPU): every SLICED table
 * of the packed program is evaluated by a host emulation of the
 * warp-cooperative kernel, reading the packed segments, batches and rows
 * exactly as the kernel does, for rounds x 32 seeded random per-shot vectors
 * X, and compared exactly with the table's value from its term list (Eqs.
 * parities, scalar_product).  TSIM_ERR_INTERNAL names the first table that
 * differs. */
tsim_status tsim_selftest_sliced(const tsim_program* prog, uint64_t seed, int rounds);

/* Self-check of the compiler's rewrite rules against brute-force summation on
 * random small parameterised graphs (no GPU).  Returns TSIM_OK when all pass. */
tsim_status tsim_selftest_rules(uint64_t seed, int iterations);


/* ---- Learned cut order (compile time).  The paper names better cutting
 * decompositions as open work (Sec. "Discussion"); any cut order yields the
 * same sum of stabilizer terms (Appendix "Stabilizer decompositions"), so a
 * learned order changes table sizes only.  The network: node features
 * [non-Clifford, Pauli, proper Clifford, phase one-hot (8), log(1 + degree),
 * parameter-dependent phase, fraction of non-Clifford neighbours]
 * (TSIM_CUT_FEATURES), H0 = relu(X W_in + b_in), three layers
 * H' = relu(H Ws + mean_nbrs(H) Wn + b) of width 64, score s = H3 w_o + b_o.
 * Weights are applied in BF16 (round to nearest even of the FP32 master
 * copy), products accumulate in FP32.  Parameter vector layout (FP32):
 * [W_in (14 x 64 row-major), b_in (64)], 3 x [Ws (64x64), Wn (64x64), b (64)],
 * [w_o (64), b_o (1)].  Graph arguments are host arrays: x [n][14] row-major,
 * CSR rowptr [n + 1], col [rowptr[n]] (neighbour ids; symmetric for the
 * gradient), graph_off [n_graphs + 1] node offsets, y [n] labels (NaN = no
 * label).  Entry points that compute run on the current CUDA device and
 * allocate their own device memory; they return TSIM_ERR_ARG on inconsistent
 * arrays and TSIM_ERR_CUDA when the device fails. */
#define TSIM_CUT_FEATURES 14
int tsim_cut_num_params(void);

/* He-uniform weights, zero biases, from a splitmix64 stream of seed (host). */
tsim_status tsim_cut_init_params(uint64_t seed, float* params);

/* Training graphs: n_graphs marginal diagrams of seeded random Clifford+T
 * circuits with t_min..t_max T/T_DAG gates, reduced by the Clifford rewrites;
 * up to max_candidates cut units per graph (a cancelling ket/bra pair of one
 * T gate, or a single non-Clifford spider) are labelled, on their members,
 * with log2 of the exact number of stabilizer terms the decomposition
 * produces when that unit is split first and the rest follow the heuristic
 * (log2(2 budget) when it exceeds budget).  Written to path in a binary
 * format read by tsim_cut_train (host only, multithreaded). */
tsim_status tsim_cut_dataset(uint64_t seed, int n_graphs, int t_min, int t_max, uint64_t budget,
                             int max_candidates, const char* path);

/* Scores of all nodes of a graph batch. */
tsim_status tsim_cut_forward(const float* params, int n_nodes, const float* x, const int* rowptr,
                             const int* col, float* scores);

/* Loss (centred squared error per graph, averaged over graphs with two or
 * more labels) and its gradient with respect to the BF16 weights, written in
 * the parameter layout. */
tsim_status tsim_cut_loss_grad(const float* params, int n_nodes, const float* x, const int* rowptr,
                               const int* col, const float* y, int n_graphs, const int* graph_off,
                               float* loss, float* grad);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8; step >= 1 counts from 1)
 * on host arrays of tsim_cut_num_params() floats, updated in place. */
tsim_status tsim_cut_adam_step(float* params, const float* grad, float* m, float* v, int step, float lr);

/* Adam training on a dataset file over minibatches of batch_graphs
 * consecutive graphs, visited in a seeded order each epoch; params holds the
 * initial values and receives the trained ones; loss_per_epoch (may be NULL)
 * receives each epoch's mean minibatch loss. */
tsim_status tsim_cut_train(const char* dataset_path, int epochs, int batch_graphs, float lr, uint64_t seed,
                           float* params, float* loss_per_epoch);

/* Register (params != NULL) the network used by TSIM_DECOMP_LEARNED on the
 * current device, or remove it (NULL).  Without a model, or when scoring
 * fails, LEARNED compiles with the heuristic order.  With a model the
 * compiler decomposes each marginal in the heuristic order, with each of the
 * three cut units the network ranks best split first (a unit is a
 * cancelling ket/bra pair of one T gate, or a single spider; the rest in the
 * heuristic order), and with every unit in the network's order (each bounded
 * by the fewest terms so far), and keeps a learned order only when it has
 * strictly fewer terms. */
tsim_status tsim_cut_model_set(const float* params);

/* Held-out comparison of cut orders, against the heuristic that judges them:
 * n_graphs graphs drawn as tsim_cut_dataset draws them (seed, t_min..t_max),
 * and per graph g, out[5 g + 0..4] = non-Clifford spiders, terms in the
 * heuristic order, terms with TSIM_DECOMP_LEARNED (the registered network;
 * the heuristic when none is registered), the geometric mean of the terms
 * when one cut unit (a cancelling ket/bra pair, or a single non-Clifford
 * spider) is split first and the rest follow the heuristic (up to 16 units:
 * a random first unit), and the fewest of those and the heuristic's.
 * Counts above budget read 2 budget.  Host and the current device (for
 * scoring). */
tsim_status tsim_cut_evaluate(uint64_t seed, int n_graphs, int t_min, int t_max, uint64_t budget, double* out);

/* out[0] = scorer calls, out[1] = calls that produced scores, out[2] =
 * marginals where a learned first cut had strictly fewer terms, out[3] =
 * marginals that kept the heuristic order (counts since the library was
 * loaded). */
tsim_status tsim_cut_policy_stats(uint64_t out[4]);

#ifdef __cplusplus
}
#endif
#endif /* TSIM_H */
