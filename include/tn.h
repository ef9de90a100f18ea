/*
 * tn.h - C ABI of the GB300 sliced tensor-network contraction engine (libtn.so).
 *
 * The engine computes amplitudes of a quantum circuit by contracting its tensor network
 * (Sec. 2.1 of "Efficient Quantum Circuit Simulation by Tensor Network Methods on Modern GPUs")
 * in pairwise steps along a given path (Sec. 3.1), each step being the einsum of Sec. 2.4,
 * Eq. (chap2_einsum), run as a (permuted) complex GEMM on the GPU (Sec. 4.1).  The network may
 * be cut on a set of bonds (slicing, Sec. 3.2); every slice is an independent sub-task and the
 * amplitudes are the sum of the slice results.  Two further entry points: path annealing with
 * dynamic slicing on the host (tn_path_optimize, Sec. 3.2) and the sparse-state contraction for
 * a list of sampled bitstrings (tn_sparse_plan / tn_sparse_contract, Sec. 3.3).
 *
 * Conventions for every entry point:
 *   - Every call returns a tn_status; nothing is thrown across the ABI.  On failure a message is
 *     kept per thread and can be read with tn_last_error_detail().
 *   - Host pointers are read during the call only; the caller keeps ownership.
 *   - Device pointers are raw CUDA device addresses on the device current at tn_plan() time.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream); all device
 *     work of a call is ordered on it.
 *   - Tensors are row-major over their label list (the last label varies fastest).  Every
 *     label has dimension 2 (qubit bonds); other dimensions give TN_ERR_UNSUPPORTED.
 *   - Complex numbers are interleaved (re, im) doubles on the host and in the amplitude buffer.
 */
#ifndef TN_H_
#define TN_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TN_OK = 0,
    TN_ERR_INVALID_ARG = 1,  /* NULL pointer, negative size, out-of-range id or label      */
    TN_ERR_SHAPE = 2,        /* a label used with inconsistent dims, a dangling label       */
    TN_ERR_PATH = 3,         /* path reuses a retired id or does not reduce to the output   */
    TN_ERR_OOM = 4,          /* device memory (or the workspace limit) exhausted            */
    TN_ERR_CUDA = 5,         /* a CUDA runtime/driver call failed; see the detail message   */
    TN_ERR_TIMEOUT = 6,      /* a bounded device-side wait gave up                          */
    TN_ERR_UNSUPPORTED = 7,  /* valid input this build does not handle (e.g. dim != 2)     */
    TN_ERR_NUMERIC = 8       /* reserved: scaled storage overflow (bounded exponents rule it out) */
} tn_status;

/* Arithmetic of the contraction steps (Sec. 4.2-4.3).  Storage between steps is complex64
 * unless a step runs on the tensor cores, whose operands are then stored as planar numbers
 * (16-bit, or FP32 rounded to TF32) with one power-of-two exponent per tensor and slice.
 * Accumulation is FP32 in every mode; the cross-slice sum and the readout are FP64. */
typedef enum {
    TN_PREC_C64 = 0,          /* complex64 storage, FP32 FMA arithmetic on CUDA cores        */
    TN_PREC_TF32 = 1,         /* dense steps: TF32 tensor cores (kind::tf32), operands
                                 rounded to nearest TF32 (Sec. 4.2, Table 2's TF32)         */
    TN_PREC_SPLIT_TF32 = 2,   /* dense steps: 3xTF32 compensated products (Sec. 4.2):
                                 hi = TF32(x), lo = TF32(x - hi), three products            */
    TN_PREC_FP16_SCALED = 3,  /* dense steps: FP16 tensor cores, per-tensor 2^e scaling     */
    TN_PREC_BF16_SCALED = 4,  /* dense steps: BF16 tensor cores, per-tensor 2^e scaling; the
                                 largest-T_cc dense steps run single-pass BF16, as many as the
                                 error model allows within eps_budget (5e-3 when 0), the
                                 others compensated 3xBF16 (Sec. 4.3's top-k policy)         */
    TN_PREC_SPLIT_BF16 = 5,   /* dense steps: compensated BF16 products (3xBF16, Sec. 4.2)   */
    TN_PREC_SPLIT_FP16 = 6,   /* dense steps: compensated FP16 products (3xFP16, Sec. 4.2):
                                 x = hi + lo, xy ~ hi hi + hi lo + lo hi, near-FP32 accuracy  */
    TN_PREC_MIXED = 7         /* Sec. 4.3: the mixed_topk largest-T_cc dense steps single-pass
                                 FP16, the other dense steps compensated FP16                */
} tn_precision;

/* Precision policy of the dense (tensor-core) steps, Sec. 4.3 / Table 3.  The dense steps are
 * ranked by T_cc; the first k run single-pass in the mode's type, the rest as compensated hi/lo
 * products of the same type (3 products, near-FP32 accuracy).  k is
 *   - every dense step for TN_PREC_FP16_SCALED and TN_PREC_TF32, mixed_topk for
 *     TN_PREC_MIXED (1 when 0), at most mixed_topk (when > 0) for the other single-pass modes;
 *   - then lowered until the predicted amplitude error fits the budget, when there is one
 *     (eps_budget > 0, or TN_PREC_BF16_SCALED's default of 5e-3).
 * Error model (predicted relative L2 error of the amplitudes against exact arithmetic):
 *   eps^2 = k (c u)^2 + (dense steps compensated) d_split^2 + d_floor^2,
 * with u the unit roundoff of the single-pass type (2^-11 FP16 and TF32, 2^-8 BF16),
 * c = 1.5 sqrt(2/7) (two operands rounded to nearest; sqrt(1/7) is the relative Frobenius
 * error of round-to-nearest for significands uniform in [1, 2); 1.5 is a safety factor over the
 * ~1.15 measured on the 30-qubit 14-cycle circuit), d_split = 4e-6 (a compensated step with
 * accumulator promotion, measured) and d_floor = 1e-5 (the complex64 storage of the leaves and
 * the FP32 steps).  Errors of independent steps add in quadrature.  A budget on the amplitude
 * error r also bounds the paper's eps_L2^2 (Eq. l2_squared_error): eps_L2^2 <= 2r + r^2. */

/* Complex GEMM form for the tensor-core steps: 4M = four real products, 3M = three. */
typedef enum { TN_GEMM_AUTO = 0, TN_GEMM_4M = 1, TN_GEMM_3M = 2 } tn_gemm_form;

typedef struct tn_network tn_network_t;
typedef struct tn_plan tn_plan_t;

typedef struct {
    int64_t max_slices_in_flight;  /* slices contracted together per launch; 0 = as many as
                                      the workspace limit allows                            */
    int64_t workspace_limit;       /* bytes of device workspace the plan may use; 0 = 60% of
                                      the free device memory at tn_plan() time               */
    void *workspace;               /* optional caller-owned device buffer of workspace_limit
                                      bytes, 256-byte aligned (else TN_ERR_INVALID_ARG); NULL =
                                      the plan allocates (cudaMalloc) and frees              */
    int32_t gemm_form;             /* tn_gemm_form                                           */
    int32_t sync_each_call;        /* 1 = tn_contract synchronises its stream and reports
                                      asynchronous errors itself                             */
    int32_t use_graph;             /* 1 = replay the step sequence as a captured CUDA graph  */
    int32_t profile;               /* 1 = time every step with CUDA events on the contraction
                                      stream (read by tn_plan_get_step_info after the stream is
                                      synchronised)                                           */
    int32_t tc_bk;                 /* tensor-core shared-memory row preference, in 16-bit
                                      elements: 0 = automatic, 32 (64-byte rows) or 64
                                      (128-byte rows); a preference selects the one-tile-per-CTA
                                      kernels instead of the persistent short-K kernel        */
    int32_t tc_bn;                 /* tensor-core N tile preference: 0 = automatic, 128, 256  */
    int32_t autotune;              /* 1 = during the first full batch, time every applicable
                                      tensor-core kernel variant (tile shape, 4M / 3M) per step
                                      and keep the fastest                                    */
    int32_t mixed_topk;            /* how many tensor-core steps, largest T_cc first, run
                                      single-pass (TN_PREC_MIXED: exactly that many, 0 = 1;
                                      FP16/BF16-scaled and TF32: at most that many, 0 = all);
                                      the others use compensated hi/lo products              */
    int32_t thin_tc;               /* streaming (thin-operand) steps with 4-16 columns and
                                      4-16 terms on the tensor cores (compensated TF32,
                                      FP32-level accuracy) in the tensor-core modes: 0 =
                                      those with 16 terms or with 16 columns and 8 terms, 1 =
                                      all of them, -1 = none (CUDA cores)                     */
    double eps_budget;             /* > 0: largest predicted amplitude relative L2 error the
                                      precision policy may reach (error model above); 0 = none,
                                      except TN_PREC_BF16_SCALED (5e-3)                      */
    int32_t reserved[2];
} tn_plan_options;

typedef struct {
    int64_t num_steps;             /* pairwise steps of the path                             */
    int64_t num_slices;            /* 2^(number of sliced labels)                            */
    int64_t slices_in_flight;      /* slices per launch chosen by the plan                   */
    int64_t workspace_bytes;       /* device workspace used                                  */
    int32_t num_open;              /* open labels = log2(number of amplitudes)               */
    int32_t max_log2_size;         /* largest intermediate (log2 elements, per slice)        */
    double tcc_per_slice;          /* sum of T_cc (Eq. T_cc, 8 flops per complex MAC) of the
                                      slice-dependent steps, per slice                        */
    double tcc_invariant;          /* T_cc of the slice-independent steps (run once per call) */
    double tmc_per_slice;          /* sum of T_mc (Eq. T_mc) of the slice-dependent steps,
                                      in bytes of complex64                                  */
    int32_t num_tc_steps;          /* steps routed to the tcgen05 GEMM                       */
    int32_t num_gemm_steps;        /* steps routed to the CUDA-core GEMM                     */
    int32_t num_stream_steps;      /* steps routed to the streaming (thin-operand) kernel    */
    int32_t num_generic_steps;     /* steps routed to the element-wise kernel                */
    int64_t kernel_launches;       /* kernels this plan has launched so far (all calls)      */
    double bind_ms;                /* profile mode: summed CUDA-event time of the leaf binding
                                      (slice fixing + permutation into plan order + complex64
                                      conversion, Sec. 3.2 / 4.1)                            */
    int64_t bind_launches;         /* profile mode: binding passes timed                     */
    int32_t num_single_pass;       /* tensor-core steps run single-pass (the policy's k)      */
    int32_t num_compensated;       /* tensor-core steps run with compensated hi/lo products   */
    double eps_predicted;          /* the error model's amplitude relative L2 error of the
                                      plan (precision policy above)                          */
    int32_t num_open_sliced;       /* sliced labels that are open: amplitude batches of
                                      2^(num_open - num_open_sliced) amplitudes              */
    int32_t reserved[3];
} tn_plan_info;

typedef struct {
    int32_t kernel;                /* 0 generic, 1 stream, 2 CUDA-core GEMM, 3 tcgen05 GEMM,
                                      4 stream on the tensor cores (opts.thin_tc)           */
    int32_t slice_dependent;       /* 0 = computed once per call and shared by all slices    */
    int32_t log2_m, log2_n, log2_k, log2_batch;  /* GEMM extents of the step (Sec. A.2)    */
    int32_t log2_a, log2_b, log2_c;              /* operand and result sizes               */
    int32_t gemm_form;             /* 1 = 4M, 2 = 3M, 3 = 4M with compensated hi/lo planes   */
    double tcc;                    /* Eq. T_cc of one slice of this step                     */
    double time_ms;                /* profile mode: summed CUDA-event time of its main kernel */
    int64_t launches;              /* profile mode: launches timed                           */
    double prep_ms;                /* profile mode: time of its operand conversions (tensor-
                                      core steps: amax + planar 16-bit copies)               */
    int32_t tc_variant;            /* tensor-core kernel variant in use (-1 otherwise):
                                      0-5 4M / 3M 16-bit one tile per CTA (128 x 128 or
                                      128 x 256), 6 compensated 16-bit, 7-10 the TF32
                                      counterparts of 0-3, 11 3xTF32, 12-16 the persistent
                                      short-K kernel (16-bit rows of 64 / 16 / 32 bytes: 12,
                                      14, 15; TF32 rows of 64 / 32 bytes: 13, 16), 17-22 the
                                      128 x 64 tile for results 64 wide (4M 16-bit / TF32,
                                      compensated 16-bit / TF32, 3M 16-bit / TF32), 23-28 the
                                      128 x 32 tile for results 32 wide (same order), 29-33 /
                                      34-38 the persistent kernel's variants of 12-16 with 64- /
                                      32-column tiles, 39-53 the compensated (hi / lo) forms of
                                      12-16, 29-33 and 34-38                                 */
    int32_t store_run_log2;        /* GEMM kernels: log2 of the longest run of consecutive
                                      result elements one staged chunk writes (its bits that
                                      are also the result's lowest positions)                */
    double tmc_bytes;              /* algorithmic bytes of one slice of the step in its storage
                                      formats: operands read once (complex64, or the planar
                                      copies a tensor-core step reads), the result written once
                                      (complex64, or planar when written directly)           */
} tn_step_info;

/*
 * Load a tensor network (Sec. 2.1; D1 of the paper's pipeline).
 *   num_tensors       number of tensors (>= 1)
 *   ranks[i]          rank of tensor i (0..62)
 *   labels[i][r]      label of axis r of tensor i; labels are ints in [0, 2^20)
 *   dims[i][r]        dimension of that axis; must be 2
 *   data[i]           2 * prod(dims) doubles: interleaved complex128, row-major
 *   num_open          number of open (output) labels
 *   open_labels[j]    output order: open_labels[0] is the most significant bit of the
 *                     amplitude index
 * A label must appear on exactly two tensors, or on one tensor and in open_labels; a label on
 * three or more tensors is a hyperedge (allowed; it becomes a batch index where two of its
 * tensors meet).  The data are copied to the device; the caller may free them on return.
 * Errors: TN_ERR_INVALID_ARG, TN_ERR_SHAPE, TN_ERR_UNSUPPORTED (dim != 2), TN_ERR_CUDA.
 */
tn_status tn_network_load(int32_t num_tensors, const int32_t *ranks,
                          const int32_t *const *labels, const int64_t *const *dims,
                          const double *const *data, int32_t num_open,
                          const int32_t *open_labels, tn_network_t **out);

/*
 * Replace the numbers of a loaded network (same structure), e.g. new gate parameters.
 * data[i] as in tn_network_load.  Synchronous with respect to the host buffers.
 */
tn_status tn_network_set_data(tn_network_t *net, const double *const *data);

/*
 * Build an execution plan.
 *   path              path_len = num_tensors - 1 pairs (a, b): tensor a becomes the
 *                     contraction of a and b and id b is retired (Sec. 3.1)
 *   sliced_labels     bonds cut by slicing (Sec. 3.2); bit j of a slice id fixes
 *                     sliced_labels[j].  An open label may be sliced too: it then splits the
 *                     amplitudes into batches instead of a sum (open-qubit amplitude batches run
 *                     in the same launches as the slices): a slice's result is added to the
 *                     block of amps whose index bits for those labels equal the slice id's
 *                     bits for them, and the intermediates no longer carry those labels
 *   mode              tn_precision
 *   opts              may be NULL (defaults)
 * The plan decides the memory order of every intermediate so that each dense step reads its
 * operands as GEMM matrices and each producer writes in its consumer's order (Sec. 4.1), routes
 * every step to a kernel, and sizes its device workspace.  The network must outlive the plan.
 * Errors: TN_ERR_INVALID_ARG, TN_ERR_PATH, TN_ERR_OOM, TN_ERR_UNSUPPORTED, TN_ERR_CUDA.
 */
tn_status tn_plan(const tn_network_t *net, int32_t path_len, const int32_t *path,
                  int32_t num_sliced, const int32_t *sliced_labels, tn_precision mode,
                  const tn_plan_options *opts, tn_plan_t **out);

/* Plan statistics (host memory out). */
tn_status tn_plan_get_info(const tn_plan_t *plan, tn_plan_info *out);

/* Per-step statistics, step in [0, num_steps) in path order (host memory out).  In profile
 * mode this waits for the step's recorded events; synchronise the stream first. */
tn_status tn_plan_get_step_info(const tn_plan_t *plan, int64_t step, tn_step_info *out);

/*
 * Contract slices [slice_begin, slice_end) and ADD their sum into amps_dev (Sec. 3.2: the
 * answer is the sum of the sub-task results).
 *   amps_dev          device buffer of 2^num_open complex128 (interleaved doubles), caller
 *                     owned and caller zeroed; results are accumulated (+=) in FP64, slices in
 *                     increasing order.  Splitting a range into sub-ranges gives the same sum
 *                     up to FP64 rounding.
 * Device work is asynchronous on `stream`; an asynchronous failure is reported by this call
 * when opts.sync_each_call was set, otherwise by the next call on the plan.
 * Errors: TN_ERR_INVALID_ARG (range), TN_ERR_CUDA, TN_ERR_TIMEOUT.  (TN_ERR_NUMERIC is not
 * returned: every power-of-two exponent of the scaled 16-bit storage comes from a bound on
 * measured max-abs values, so that storage cannot overflow for finite inputs; non-finite inputs
 * propagate into the amplitudes.)
 */
tn_status tn_contract(tn_plan_t *plan, int64_t slice_begin, int64_t slice_end, void *amps_dev,
                      void *stream);

/*
 * Host-buffer convenience: zero a device accumulator, contract [slice_begin, slice_end), copy
 * the 2^num_open complex128 amplitudes to amps_host and synchronise `stream`.
 */
tn_status tn_contract_host(tn_plan_t *plan, int64_t slice_begin, int64_t slice_end,
                           double *amps_host, void *stream);

/*
 * FP64 readout of m = 2^num_open amplitudes on the device (Eq. lxeb_2, Eq. lxeb_as_l2):
 *   out[0] = sum |a|^2, out[1] = sum |a|^4, out[2] = F_l = 2^n_qubits * out[0] / m - 1,
 *   out[3] = 2^n_qubits * out[1] / out[0] - 1  (XEB of ideal samples from these amplitudes).
 * out is host memory; the call synchronises `stream`.
 */
tn_status tn_readout(const tn_plan_t *plan, const void *amps_dev, int32_t n_qubits,
                     double out[4], void *stream);

/*
 * FP64 readout of `num_amps` complex128 amplitudes at amps_dev, with no plan and no device
 * allocation; out[0..3] as in tn_readout with m = num_amps.  The paper has no counterpart: this
 * is for callers that cannot allocate device memory, such as a process whose GPU memory is held
 * by another allocator (a caching allocator keeps freed blocks reserved, so a cudaMalloc from
 * this library can fail although the caller has memory to spare) or one that runs under a fixed
 * budget where every allocation must come from its own pool.
 *   - Scratch: a fixed 64 KiB device array inside libtn.so (on every GPU that loads the library,
 *     until the process exits); the call allocates and frees nothing.
 *   - Limit: num_amps <= 2^28 (4096 block sums of 65536 amplitudes); larger -> TN_ERR_INVALID_ARG.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress);
 *     make that first call before any stream capture.
 *   - All calls share the array, which keeps the last call's partial sums; calls whose work
 *     overlaps on the GPU (e.g. on two streams) race.  The call synchronises `stream`.
 * Errors: TN_ERR_INVALID_ARG, TN_ERR_CUDA.
 */
tn_status tn_readout_noalloc(const void *amps_dev, int64_t num_amps, int32_t n_qubits,
                             double out[4], void *stream);

/*
 * Failure-detection self-test of the tensor-core kernel's bounded waits: launches one CTA whose
 * producer issues no copies, so its MMA warp's wait gives up after limit_ms (1..10000); the CTA
 * records the timeout, frees its tensor memory and exits without writing results.  Returns
 * TN_ERR_TIMEOUT when the wait ran out as designed (the CUDA context stays usable), TN_OK if it
 * did not, TN_ERR_UNSUPPORTED without a tcgen05 device.  Synchronises `stream`.
 */
tn_status tn_selftest_wait_timeout(int32_t limit_ms, void *stream);

/*
 * Contraction-path optimisation (host only; no device is used).
 *
 * Simulated annealing over the contraction tree (Sec. 3.2): the score
 *     log2(T_cc + alpha * T_mc) + beta * log2(T_sc)
 * (T_cc: multiply-adds of all pairwise steps, T_mc: elements read and written by them, T_sc: the
 * largest intermediate, all per slice, plus log2 of the slice count) is lowered by local updates
 * that exchange the three nearest descendants of a vertex (X = (A, (B, C)) becomes ((A, C), B)
 * or ((A, B), C)), one per internal vertex in each sweep from the root to the leaves, accepted
 * by the Metropolis rule; the temperature falls geometrically from t_start to t_end over the
 * sweeps.  Dynamic slicing (Sec. 3.2): with max_log2_size > 0, while the largest intermediate
 * exceeds 2^max_log2_size, the bond whose slicing gives the lowest score is sliced and the tree
 * is re-tuned by sweeps_per_slice further sweeps.  `chains` independent chains (one host thread
 * each, seeds derived from `seed`) run; the lowest final score wins.  Results are deterministic
 * for given inputs and options.
 */
typedef struct {
    uint64_t seed;
    int32_t sweeps;            /* sweeps before slicing (< 0: default 200)                   */
    int32_t sweeps_per_slice;  /* re-tuning sweeps after each sliced bond (< 0: default 40)  */
    int32_t sweeps_final;      /* sweeps after slicing (< 0: default 200)                    */
    int32_t max_log2_size;     /* dynamic slicing target in log2 elements; 0 = no slicing    */
    int32_t max_sliced;        /* most bonds to slice (<= 0: 64; capped by sliced_capacity)  */
    int32_t chains;            /* independent chains (<= 0: 1; at most 256)                  */
    double t_start, t_end;     /* temperatures in score units (<= 0: defaults 0.05, 0.001)   */
    double alpha;              /* weight of T_mc (>= 0)                                       */
    double beta;               /* weight of log2(T_sc) (>= 0)                                 */
    int32_t greedy_trials;     /* > 0: each chain first builds this many random greedy trees
                                  (cost log2 size(out) - g log2(size(a) + size(b)), g and the
                                  noise temperature drawn per tree) and anneals from the best
                                  of them and path_in                                         */
    int32_t balance_log2;      /* balanced indices (App. A.2): > 0 counts the multiply-adds of
                                  every unbalanced step 2^balance_log2 times in T_cc (a step is
                                  unbalanced when, as a GEMM, k < 64 or min(m, n) < 32); the
                                  reported T_cc stays the plain count.  0 = off              */
    int32_t reserved[6];
} tn_path_options;

typedef struct {
    double log2_tcc;               /* log2 of T_cc per slice (real flops, 8 per multiply-add) */
    double log2_tcc_total;         /* log2 of T_cc over all slices                            */
    double log2_tmc;               /* log2 of T_mc per slice (elements)                       */
    double score;                  /* final score of the returned tree                        */
    double initial_log2_tcc;       /* the same for the input path, unsliced                   */
    int32_t initial_max_log2_size;
    int32_t max_log2_size;         /* largest intermediate per slice, log2 elements           */
    int32_t num_sliced;            /* bonds written to sliced_out                             */
    int32_t reserved0;
    int64_t moves_tried, moves_accepted;
    int64_t reserved[4];
} tn_path_info;

/*
 * Improve a contraction path (and choose sliced bonds).
 *   num_tensors, ranks, labels, num_open, open_labels   the network's structure, as in
 *                     tn_network_load (host memory); every dimension is taken as 2
 *   path_in           the starting path: num_tensors - 1 pairs (a, b), result in a (Sec. 3.1)
 *   opts              may be NULL (defaults)
 *   path_out          num_tensors - 1 pairs, the optimised path in the same format (may alias
 *                     path_in only if the caller no longer needs the input)
 *   sliced_out        up to sliced_capacity labels: the sliced bonds, in label order
 *   info              costs before and after (host memory out)
 * Every label must lie on exactly two tensors, or on one tensor and in open_labels; labels on
 * three or more tensors (hyperedges) give TN_ERR_UNSUPPORTED.  Open labels are never sliced.
 * Errors: TN_ERR_INVALID_ARG, TN_ERR_SHAPE (dangling or repeated label), TN_ERR_PATH (invalid
 * path_in), TN_ERR_UNSUPPORTED.
 */
tn_status tn_path_optimize(int32_t num_tensors, const int32_t *ranks,
                           const int32_t *const *labels, int32_t num_open,
                           const int32_t *open_labels, const int32_t *path_in,
                           const tn_path_options *opts, int32_t *path_out, int32_t *sliced_out,
                           int32_t sliced_capacity, tn_path_info *info);

/*
 * Sparse-state contraction (Sec. 3.3): the amplitudes of a list of sampled bitstrings.
 *
 * Every tensor keeps, for the open labels it carries, only the configurations of those labels
 * that occur among the samples (its merged sparse bond), each with a complex64 array over its
 * other labels.  A pairwise step (path format of Sec. 3.1) forms the configurations of the union
 * of its operands' open labels that occur among the samples, pairs each with its projections
 * onto the operands (gather tables built at plan time) and contracts the other labels per
 * configuration on the CUDA cores (FP32 arithmetic: result configurations that share an entry of
 * one operand form one 64 x 64-tiled GEMM over the stacked entries of the other (grouped GEMM)
 * when at least 8 elements are contracted and the tiles are at least a quarter full; else a
 * tiled GEMM per configuration, a thread per row for at most 16 columns, or one thread per
 * output); the root holds one value per distinct sample.  No slicing; every non-open label must lie on exactly two tensors.
 */
typedef struct tn_sparse_plan tn_sparse_plan_t;

typedef struct {
    int64_t num_steps;
    int64_t num_samples;
    int64_t distinct_samples;     /* distinct bitstrings among the samples                    */
    int64_t total_configs;        /* sum over all tensors of their sampled configurations     */
    int64_t arena_bytes;          /* device storage of all tensors (no reuse)                 */
    double tcc;                   /* real flops of all steps (8 per complex multiply-add)     */
    int64_t kernel_launches;      /* kernels launched by this plan so far                     */
    int32_t max_log2_dense;       /* largest dense part of a tensor, log2 elements            */
    int32_t gemm_steps;           /* steps run as a tiled GEMM per configuration              */
    int64_t dense_subtrees;       /* subtrees without open labels run by ordinary plans       */
    int64_t dense_subtree_steps;  /* steps inside them                                        */
    int64_t thin_steps;           /* steps run as thread-per-row thin kernels (<= 16 columns) */
    int64_t grouped_steps;        /* steps run as grouped GEMMs over shared operand entries   */
} tn_sparse_info;

/*
 * Plan a sparse-state contraction of `net` along `path` (num_tensors - 1 pairs).
 *   samples           num_samples x num_open bytes, row i = sample i, byte j = value (0 or 1) of
 *                     the network's open label j (host memory, copied)
 *   mode              precision of the dense subtrees: every maximal subtree of the path with no
 *                     open label below it (and at least 2^28 flops) is contracted by an ordinary
 *                     plan in this mode (layout pass, tensor cores in the low-precision modes)
 *                     and its result joins the sparse steps, which always run in FP32
 * Errors: TN_ERR_INVALID_ARG (sizes, a byte other than 0/1), TN_ERR_PATH, TN_ERR_UNSUPPORTED
 * (more than 64 open labels, a hyperedge, a tensor too large), TN_ERR_OOM, TN_ERR_CUDA.
 */
tn_status tn_sparse_plan(const tn_network_t *net, int32_t path_len, const int32_t *path,
                         int64_t num_samples, const uint8_t *samples, tn_precision mode,
                         tn_sparse_plan_t **out);

/*
 * ADD the amplitudes of the samples into amps_dev (device complex128[num_samples], caller-owned
 * and caller-zeroed, entry i = sample i, repeated samples get the same value); all work on
 * `stream`.  Errors: TN_ERR_INVALID_ARG, TN_ERR_CUDA.
 */
tn_status tn_sparse_contract(tn_sparse_plan_t *plan, void *amps_dev, void *stream);

/* Statistics of a sparse-state plan (host memory out). */
tn_status tn_sparse_get_info(const tn_sparse_plan_t *plan, tn_sparse_info *out);

/* Free a network, a plan or a sparse-state plan (NULL is a no-op).  Destroy plans before their
 * network. */
void tn_destroy(void *handle);

/* Static description of a status code. */
const char *tn_status_string(tn_status s);

/* Copy this thread's last error message into buf (always NUL-terminated when len > 0). */
tn_status tn_last_error_detail(char *buf, size_t len);

#ifdef __cplusplus
}
#endif

#endif /* TN_H_ */
