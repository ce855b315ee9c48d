/*
 * tn.h -- C ABI of the GB300 tensor-network contraction engine.
 *
 * The engine executes a FIXED pairwise contraction path (Sec. II-B of "Parallelizing
 * Large-Scale Tensor Network Contraction on Multiple GPUs") on one GPU:
 *   - every step A x B -> C is run as a GEMM A_MK x B_KN -> C_MN (Sec. II-B), with the
 *     mode orders of all tensors chosen ahead of time by the GEMM-oriented backward
 *     pass of Sec. IV-A so that no step needs a runtime transpose;
 *   - sliced labels (Sec. II-C) become an on-device batch dimension, and the slice
 *     results are summed in FP64 with compensated (Neumaier) summation.
 *
 * Conventions shared by every entry point:
 *   - Row-major storage; the leftmost mode is outermost (Sec. IV-B, prefix distribution).
 *   - Complex tensors are complex64 (interleaved re, im float32) on input; real
 *     tensors are float32. Results are complex128 / float64.
 *   - The caller owns every input and output buffer; the library never frees them.
 *   - Every function returns a tn_status; no C++ exception and no device trap crosses
 *     the ABI. tn_last_error() gives a thread-local message for the last failure.
 *   - Device work is asynchronous on the caller's stream unless stated otherwise.
 */
#ifndef TN_GB300_H
#define TN_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TN_OK = 0,
  TN_ERR_INVALID = 1,      /* malformed network/path/arguments */
  TN_ERR_UNSUPPORTED = 2,  /* valid input the engine does not handle (hyper-edge, ...) */
  TN_ERR_OOM = 3,          /* device memory for the plan workspace not available */
  TN_ERR_CUDA = 4,         /* a CUDA call failed; message has the CUDA error string */
  TN_ERR_BUSY = 5,         /* serve queue full */
  TN_ERR_TIMEOUT = 6,      /* bounded wait expired (serve poll, device-side spin) */
  TN_ERR_NOT_READY = 7     /* serve ticket still in flight */
} tn_status;

/* Arithmetic form of the pairwise GEMMs. C64_* take complex64 inputs, R32_* float32.
 *   FP32_SIMT : FP32 FMA on the CUDA cores (the plain form).
 *   TF32      : tcgen05 tensor cores, operands read as TF32, FP32 accumulation.
 *   3XTF32    : tcgen05, each operand split hi + lo, three TF32 products, FP32 accum.
 *   BF16X3    : tcgen05 kind::f16, each operand split hi + lo in BF16 (rounded to
 *               nearest) by the kernel that produces it, three products hi.hi +
 *               hi.lo + lo.hi (complex only; relative error per product <= ~3 * 2^-16),
 *               FP32 accumulation.
 * Steps too small or too thin for a tensor-core tile run on the FP32 SIMT kernels
 * whatever the form (tn_plan_step reports each step's kernel). Real networks take the
 * TF32 and 3XTF32 forms on 128 x 256 tiles; R32_BF16X3 is not built. Exponent scaling
 * runs in every form but the 3M product (the tensor-core kernels apply the operands' exact
 * power-of-two scales to the accumulated result, the same values as scaling the operands
 * on load; scaled BF16X3 steps keep one SM per tile). tn_plan returns TN_ERR_UNSUPPORTED
 * for R32_BF16X3 and for the 3M product with exponent scaling rather than running another
 * form. */
typedef enum {
  TN_C64_FP32_SIMT = 0,
  TN_C64_TF32 = 1,
  TN_C64_3XTF32 = 2,
  TN_C64_BF16X3 = 3,
  TN_R32_FP32_SIMT = 4,
  TN_R32_TF32 = 5,
  TN_R32_3XTF32 = 6,
  TN_R32_BF16X3 = 7
} tn_precision;

/* The semiring the network is contracted over (Sec. III-C: counting and optimisation
 * problems as contractions of local-constraint tensors).
 *   STANDARD : (+, x), every form above.
 *   MAXPLUS  : (max, +), the tropical semiring: a step computes
 *              C[i, j] = max_k (A[i, k] + B[j, k]) and slices combine by maximum. Only
 *              with TN_R32_FP32_SIMT and no exponent scaling (TN_ERR_UNSUPPORTED
 *              otherwise); FP32 max and add, exact while the values are integers below
 *              2^24; -inf is the semiring's zero (an excluded configuration). */
typedef enum { TN_SEMIRING_STANDARD = 0, TN_SEMIRING_MAXPLUS = 1 } tn_semiring;

/* Plan flags. */
#define TN_PLAN_HOST_ONLY 1u     /* plan and query only: no device memory, no contract */
#define TN_PLAN_SINGLE_SM_TILES 2u /* BF16x3 4M steps keep one SM per output tile (by default
                                      a step with m >= 256 and k > 256 runs 256 x 128 tiles
                                      on pairs of SMs); the results are the same bits */

typedef struct {
  int32_t prec;            /* tn_precision */
  int32_t complex_mult;    /* 4 (4M); 3 (3M, Gauss) with TN_C64_BF16X3 only, else rejected */
  int32_t exp_scaling;     /* 1: per-intermediate power-of-two scaling, log scale in FP64
                              (every form but the 3M product) */
  int32_t max_slice_batch; /* slices per device pass; 0 = as many as fit in free HBM */
  uint32_t flags;          /* TN_PLAN_* */
  int32_t semiring;        /* tn_semiring */
  int32_t reserved[2];
} tn_dtype_policy;

/* A network: tensor t has rank[t] modes modes[t][0..rank[t]-1] (labels in
 * 0..n_labels-1, leftmost outermost). extent[label] is the label's dimension. A closed
 * label appears in exactly two tensors; an open label in exactly one and in
 * open_modes, which fixes the result's mode order (Sec. IV-A: the root order is given
 * by the problem). */
typedef struct {
  int32_t n_tensors;
  const int32_t* rank;
  const int32_t* const* modes;
  int32_t n_labels;
  const int64_t* extent;
  int32_t n_open;
  const int32_t* open_modes;
} tn_network;

/* A contraction path in SSA form: leaves are 0..n_tensors-1 and step s contracts
 * pair[2s], pair[2s+1] into tensor n_tensors+s. Must form one binary tree
 * (n_steps = n_tensors - 1, every id consumed once). */
typedef struct {
  int32_t n_steps;
  const int32_t* pair; /* 2*n_steps ids */
} tn_path;

typedef struct tn_plan_s* tn_plan_t;

/* Kernel class chosen for a step (Sec. IV-C cost model t = max(D_rw/B, FLOPs/F)). */
typedef enum {
  TN_CLASS_SIMT = 0,   /* tiled FP32 GEMM on the CUDA cores (any shape; when its tiles
                          cannot fill the GPU and k >= 2048, k is split across CTAs and
                          the parts combined in order) */
  TN_CLASS_STREAM = 1, /* big x small: one pass over the big operand */
  TN_CLASS_TC = 2,     /* tcgen05 tensor-core GEMM (rows >= 128, columns >= 16, k >= 8; a
                          persistent variant for k <= 256 in the 4M BF16X3 form) */
  TN_CLASS_SPLITK = 3, /* few outputs, long k: split-K partials in FP64, fixed-order sum */
  TN_CLASS_PERM = 4    /* not a step class: leaf staging (a leaf permuted from its declared
                          order into its planned order); in tn_profile only */
} tn_step_class;
#define TN_N_CLASSES 5

typedef struct {
  int64_t n_steps, n_leaves, n_slices, slice_batch, n_passes;
  double flops;            /* algorithmic: sum 8mnk (complex) or 2mnk (real), all slices */
  double bytes;            /* algorithmic: sum e(mk+kn+mn) + leaf staging, all slices */
  double Ct, Cm, Cs;       /* Sec. II-B Eqs. 1-3 for one slice (element counts) */
  int64_t peak_elems;      /* largest tensor of one slice, elements */
  int64_t workspace_bytes; /* device bytes the plan holds */
  int64_t steps_per_class[TN_N_CLASSES];
  double flops_per_class[TN_N_CLASSES];
  int64_t leaf_permutes;   /* leaves whose planned order differs from the declared one
                              (permuted once while staging; no step permutes) */
} tn_plan_stats;

typedef struct {
  int64_t m, n, k;         /* GEMM view of the step */
  int32_t a_id, b_id;      /* SSA ids of the operands in the A (rows) and B (cols) roles */
  int32_t cls;             /* tn_step_class */
  int32_t batched;         /* 1 if the step depends on a sliced label */
  /* Output placement: row index r (mixed radix over row_ext, last fastest) lands at
   * sum_d digit_d * row_stride[d] elements, columns likewise; C[r, c] is stored at
   * rows(r) + cols(c) of the output's planned layout. */
  int32_t n_row_dims, n_col_dims;
  int64_t row_ext[12], row_stride[12], col_ext[12], col_stride[12];
  int32_t ksplit;          /* SIMT steps: k cut in this many parts (then two launches) */
  int32_t single_sm;       /* tensor-core steps: 1 if kept on one SM per tile (tn_plan_autotune) */
  int32_t chain;           /* -1, or the step chain the step runs in: a run of consecutive tiny
                              CUDA-core steps executed by one CTA in one launch (the profile
                              attributes the chain's time to its first step) */
  int32_t reserved;
} tn_step_info;

/* How a tensor's copies are stored in the workspace. PLANAR: FP32 (complex: the real
 * plane, then the imaginary plane). SPLIT_BF16 (complex, BF16X3 plans only): the
 * operands of tensor-core steps are written by their producers as four BF16 planes
 * [re_hi | im_hi | re_lo | im_lo] with hi = RN_bf16(v), lo = RN_bf16(v - hi); same
 * bytes per element as PLANAR. */
typedef enum { TN_FORMAT_PLANAR = 0, TN_FORMAT_SPLIT_BF16 = 1 } tn_storage_format;

/* Where a tensor lives in the plan's workspace (introspection). */
typedef struct {
  int64_t size;            /* elements of one slice copy (sliced labels removed) */
  int64_t offset;          /* byte offset from the workspace base */
  int64_t bytes;           /* bytes reserved, all batch copies */
  int32_t batched;         /* one copy per slice of a pass (else one copy) */
  int32_t pinned;          /* made in the first pass, kept for every pass */
  int32_t producer;        /* step index, -1 for a leaf */
  int32_t consumer;        /* step index, -1 for the root */
  int32_t format;          /* tn_storage_format of the tensor's copies */
  int32_t tiled;           /* leaves: staged by the tiled permutation kernel (one launch per
                              pass that stages it) rather than the per-leaf kernel: 1 its
                              general form, 2 its pipelined form (each index group one 32-wide
                              chunk, 16-byte loads; used when the source is 16-byte aligned) */
} tn_tensor_info;

/* Rates of the kernel choice, the roofline cost model of Sec. IV-C Eq. 6: a step's time
 * under a kernel family is max(bytes / hbm_bytes_per_s, flops / F) with F that family's
 * peak in algorithmic flops (8 per complex MAC, 2 per real MAC). Process-wide; plans built
 * after tn_cost_model_set use the new rates. Defaults: 6.8e12 B/s, FP32 FMA 152 SMs x 128
 * lanes x 2 x 1.9 GHz, and from a sustained dense BF16 rate of 1.7e15 flop/s: TF32 at
 * 1.1/2.25 of it, 3xTF32 a third of TF32, BF16x3 a third of BF16. */
typedef struct {
  double hbm_bytes_per_s;  /* B */
  double simt_flops;       /* F of the CUDA-core kernels (FP32 FMA) */
  double tc_flops[3];      /* F of the tensor-core forms: [TF32, 3XTF32, BF16X3] */
} tn_cost_model;

/* Replace the rates (every field > 0, else TN_ERR_INVALID). Not thread-safe against
 * concurrent tn_plan calls. */
tn_status tn_cost_model_set(const tn_cost_model* m);
tn_status tn_cost_model_get(tn_cost_model* out);

/* Measure the FP32 FMA peak of the current device (the paper has no counterpart; it is the
 * denominator of the CUDA-core kernels' roofline): a kernel whose every thread runs
 * `iters` rounds of 8 independent FMA chains, 4 CTAs of 256 threads per SM, timed with CUDA
 * events on `stream`. Writes the rate in flop/s (2 per FMA) and the elapsed milliseconds.
 * Synchronous; 0 < iters <= 2^24. */
tn_status tn_measure_ffma(int64_t iters, double* flops_per_s, double* ms, void* stream);

/* The same probe in FP64 (double FMA chains): this GPU's FP64 rate, which the cross-slice
 * sum runs at. Synchronous; 0 < iters <= 2^24. */
tn_status tn_measure_dfma(int64_t iters, double* flops_per_s, double* ms, void* stream);

/* Build a plan: validate, analyse each step (Sec. II-B), run the backward mode
 * reordering pass (Sec. IV-A), choose a kernel per step, assign every tensor a
 * place in one workspace by liveness, and (unless TN_PLAN_HOST_ONLY) allocate that
 * workspace on the current CUDA device. sliced_modes lists the labels to slice
 * (Sec. II-C); n_sliced may be 0. Returns TN_ERR_INVALID / TN_ERR_UNSUPPORTED for bad
 * input and TN_ERR_OOM if the workspace does not fit. *out is set only on TN_OK. */
tn_status tn_plan(const tn_network* net, const tn_path* path, const int32_t* sliced_modes,
                  int32_t n_sliced, tn_dtype_policy policy, tn_plan_t* out);

/* Plan statistics (host only). */
tn_status tn_plan_info(tn_plan_t plan, tn_plan_stats* out);

/* Host-side check of the tiled leaf staging (no device work; the paper has no
 * counterpart): replays the index arithmetic of the tiled permutation kernel for every
 * large leaf and up to max_slices slice ids, and checks that every source index lies in
 * the declared tensor and is the element the declared order places at each staged
 * position, that every staged element is written exactly once, and that the paired
 * 16-byte loads read adjacent elements. TN_OK, or TN_ERR_INVALID naming the first
 * mismatch. */
tn_status tn_plan_check_staging(tn_plan_t plan, int64_t max_slices);

/* Planned mode order of tensor `id` (SSA id; leaves and intermediates, sliced labels
 * removed). modes_out must hold at least the tensor's rank; *rank_out gets the rank.
 * This is the layout the backward pass of Sec. IV-A assigns. */
tn_status tn_plan_layout(tn_plan_t plan, int32_t id, int32_t* modes_out, int32_t* rank_out);

/* The number of kernel launches one tn_contract_slices call over slice_count slices makes
 * (the same for any first slice): staging, every step (two for split-k steps, several for a
 * deep step on paired SMs, launched in bands of tiles), and the slice sum, per pass. */
tn_status tn_plan_launches(tn_plan_t plan, int64_t slice_count, int64_t* out);

/* Description of step s (host only). */
tn_status tn_plan_step(tn_plan_t plan, int32_t s, tn_step_info* out);

/* Workspace placement of tensor `id` (SSA id) for the plan's slice batch (host only).
 * Complex tensors are planar: copy b of a batched tensor holds its real plane at
 * offset + 8*b*size bytes and its imaginary plane right after (size floats later). */
tn_status tn_plan_tensor(tn_plan_t plan, int32_t id, tn_tensor_info* out);

/* Contract all slices. inputs[t] is a DEVICE pointer to leaf t in its declared mode
 * order (complex64 or float32, per the plan's precision). output is a DEVICE pointer
 * to the result in open_modes order: complex128 (complex plans) or float64 (real).
 * out_log_scale: DEVICE pointer to one double or NULL; when exp_scaling is on the
 * result is output * exp(*out_log_scale). Asynchronous on `stream` (a cudaStream_t;
 * NULL = legacy default stream). Calls on one plan must not overlap in time. */
tn_status tn_contract(tn_plan_t plan, const void* const* inputs, void* output,
                      double* out_log_scale, void* stream);

/* Choose, per BF16x3 (4M) tensor-core step that the paired-SM kernels take, between paired
 * SMs and one SM per tile by timing both: two runs of the plan's first pass (its first
 * slice_batch slices) in each form, per-step CUDA-event times, the faster kept for later
 * calls. Both forms give the same bits, so results do not change. Writes into output (the
 * caller's, sized as for tn_contract) as a side effect; the caller's per-step profile is set
 * aside and restored. Synchronous. A no-op for other forms or with TN_PLAN_SINGLE_SM_TILES. */
tn_status tn_plan_autotune(tn_plan_t plan, const void* const* inputs, void* output, void* stream);

/* As tn_contract (all slices, device buffers), with the call's launches replayed from a
 * CUDA graph: the first call with a given set of input pointers, output, log_scale and
 * stream runs the contraction as tn_contract does and then captures the same call on a
 * private stream; later calls with the same pointers and stream launch the captured graph
 * (one launch instead of one per step and pass), with the same results bit for bit. A call
 * with other pointers or another stream re-captures (after the previous graph's last launch
 * has finished). The first call allocates the graph and a pinned copy of the leaf
 * descriptors; tn_plan_destroy frees them. The inputs are read at launch time, so new values
 * in the same buffers are contracted by a replay. TN_ERR_INVALID while per-step profiling is
 * on (tn_plan_profile) or for a host-only plan; TN_ERR_CUDA if capture fails. */
tn_status tn_contract_graph(tn_plan_t plan, const void* const* inputs, void* output, double* out_log_scale,
                            void* stream);

/* As tn_contract, summing only slices [slice_begin, slice_begin + slice_count). With
 * slice_count = 1 the output is that slice's partial result (Sec. V-A projection: time
 * per slice). */
tn_status tn_contract_slices(tn_plan_t plan, const void* const* inputs, int64_t slice_begin,
                             int64_t slice_count, void* output, double* out_log_scale,
                             void* stream);

/* End-to-end form: inputs and output in HOST memory. Copies the leaves into the
 * plan's device staging area, contracts all slices, copies the result back, and
 * returns after the stream has finished. out_log_scale is a host pointer or NULL. */
tn_status tn_contract_host(tn_plan_t plan, const void* const* host_inputs, void* host_output,
                           double* out_log_scale, void* stream);

/* End-to-end form of tn_contract_slices: host inputs and host output as in
 * tn_contract_host, summing only slices [slice_begin, slice_begin + slice_count). */
tn_status tn_contract_slices_host(tn_plan_t plan, const void* const* host_inputs, int64_t slice_begin,
                                  int64_t slice_count, void* host_output, double* out_log_scale,
                                  void* stream);

/* Free the plan and its device workspace (after any contract on it has finished). */
tn_status tn_plan_destroy(tn_plan_t plan);

/* ---- per-kernel-class timing (the roofline evidence) ------------------------------ */

/* Per kernel class (index tn_step_class): launches, device milliseconds measured with
 * CUDA events recorded on the contract's stream around each step launch, and the
 * algorithmic flops (8mnk complex, 2mnk real) and bytes (e(mk+kn+mn), each operand
 * and the output counted once per batch entry that reads or writes it). Entry
 * TN_CLASS_PERM covers the leaf staging of each pass: no flops, bytes = the staged
 * leaves read and written once per copy (2 e |leaf| per copy). */
typedef struct {
  int64_t launches[TN_N_CLASSES];
  double ms[TN_N_CLASSES];
  double flops[TN_N_CLASSES];
  double bytes[TN_N_CLASSES];
} tn_profile;

/* enable != 0: later contract calls on this plan record events around every step
 * launch (a few microseconds per launch). enable == 0 stops recording. */
tn_status tn_plan_profile(tn_plan_t plan, int32_t enable);

/* Wait for the recorded events and write the totals accumulated since the last reset
 * to *out; reset != 0 clears the totals after reading. */
tn_status tn_plan_profile_read(tn_plan_t plan, tn_profile* out, int32_t reset);

/* Self-test of the device-side failure path (the paper has no counterpart). Every
 * mbarrier wait in the tensor-core kernels is bounded; on expiry the kernel writes a
 * code to the plan's error word, releases what it holds and returns, and the
 * synchronising calls report TN_ERR_TIMEOUT. This runs that same bounded wait in a
 * one-thread kernel on a barrier that is completed only if `arrive` != 0, with a limit of
 * limit_us microseconds (<= 10 s). Synchronous. Returns TN_OK when the barrier completed,
 * TN_ERR_TIMEOUT when the wait ran out; the CUDA context stays usable either way. */
tn_status tn_selftest_bounded_wait(tn_plan_t plan, int32_t arrive, int64_t limit_us, void* stream);

/* Device milliseconds per step accumulated by the same events (ms_out holds n_steps
 * doubles), for the recordings folded in by tn_plan_profile_read since its last reset. A
 * step chain (tn_step_info.chain) is one launch: its time is reported at its first step and
 * 0 at the others. */
tn_status tn_plan_profile_steps(tn_plan_t plan, double* ms_out, int32_t n_steps);

/* ---- serving: continuous batching of contraction requests ------------------------ */

typedef struct {
  int32_t max_inflight;      /* launches on the GPU at once (slots; a pack takes one) */
  int32_t n_streams;         /* CUDA streams work is spread over */
  int64_t hbm_budget_bytes;  /* limit on the device memory the server holds in request
                                workspaces (resident plan instances, busy or idle; 0 = no
                                limit): idle instances are freed, least recently used first,
                                before a request waits for running ones to finish */
  int32_t queue_capacity;    /* pending requests beyond which submit returns TN_ERR_BUSY */
  int32_t pack_max;          /* > 0: queued requests on small closed unsliced plans without
                                tensor-core steps (the same arithmetic kind: complex, real with
                                or without scaling, max-plus) are packed, up to pack_max per
                                launch, into one launch of the batched small-network kernel (one
                                CTA per request); 0: every request runs its own plan launch */
  int32_t reserved[2];
} tn_serve_config;

typedef struct tn_server_s* tn_server_t;

/* Start a server with its scheduler thread on the current device. */
tn_status tn_serve_create(const tn_serve_config* cfg, tn_server_t* out);

/* Submit a request: contract `plan` (all slices) on HOST inputs. The server copies the
 * inputs before returning, so the caller may reuse its buffers. Admission waits until a
 * slot and the plan's workspace fit the HBM budget. Returns TN_ERR_BUSY when the queue
 * is full. The plan must stay alive until the ticket is polled to completion. Requests on
 * one plan run on separate resident instances of it (or packed together, see pack_max).
 * A packed request's result comes from the batched kernel: identical whatever else is in
 * its pack (one CTA computes it, in a fixed order), and within rounding of the plan's own
 * kernels. */
tn_status tn_serve_submit(tn_server_t srv, tn_plan_t plan, const void* const* host_inputs,
                          uint64_t* ticket);

/* Submit n requests at once: request j contracts plans[j] on host_inputs[j] (one host
 * pointer per leaf of that plan, as for tn_serve_submit); its ticket goes to tickets[j].
 * All are queued together, in order, under one acquisition of the server's queue, so the
 * scheduler sees them side by side and can pack compatible ones into one launch (a burst
 * submitted one by one may be admitted request by request). All or nothing: on an error
 * (TN_ERR_INVALID for a null argument, TN_ERR_BUSY when the queue cannot take all n) no
 * request is queued. */
tn_status tn_serve_submit_batch(tn_server_t srv, int32_t n, const tn_plan_t* plans,
                                const void* const* const* host_inputs, uint64_t* tickets);

/* Wait up to timeout_us (0 = do not wait, <0 = forever) for a ticket. On TN_OK writes
 * the result (complex128 or float64, |open| elements) to host `result`, the log scale
 * to *log_scale if non-NULL, and retires the ticket. TN_ERR_NOT_READY if still in
 * flight after the wait; TN_ERR_INVALID for an unknown ticket. */
tn_status tn_serve_poll(tn_server_t srv, uint64_t ticket, void* result, double* log_scale,
                        int32_t timeout_us);

/* Counters of a server since its creation (the paper has no counterpart). */
typedef struct {
  int64_t completed;        /* requests retired (any status) */
  int64_t plan_launches;    /* requests run as their own plan launch */
  int64_t packs;            /* packed launches of the batched kernel */
  int64_t packed_requests;  /* requests run inside packed launches */
  int64_t max_pack;         /* largest pack so far */
  int64_t hbm_in_use;       /* device bytes held by resident instances and pack buffers */
} tn_serve_stats;

tn_status tn_serve_stats_get(tn_server_t srv, tn_serve_stats* out);

/* Stop the scheduler (finishing admitted work) and free the server. */
tn_status tn_serve_destroy(tn_server_t srv);

/* ---- many small independent networks in one launch -------------------------------- */

typedef struct tn_batch_s* tn_batch_t;

/* Plan n_nets independent CLOSED networks (each with its own path; no slicing) for one
 * persistent launch: every network gets the same analysis and mode reordering as
 * tn_plan (Sec. II-B, Sec. IV-A) and its own arena; one CTA contracts one network at a
 * time, taking networks from an atomic queue. policy.prec must be TN_C64_FP32_SIMT or
 * TN_R32_FP32_SIMT; policy.exp_scaling renormalises every tensor by an exact power of two
 * as it is made and sums the exponents per network in an int64; policy.semiring may be
 * TN_SEMIRING_MAXPLUS with R32 and no scaling (each value is then the network's max-plus
 * value, log scale 0). With
 * TN_PLAN_HOST_ONLY no device memory is taken (tables only, for tn_batch_info). */
tn_status tn_batch_plan(int32_t n_nets, const tn_network* nets, const tn_path* paths, tn_dtype_policy policy,
                        tn_batch_t* out);

/* leaf_offsets (total leaves + 1 int64, or NULL): element offset of every leaf in the
 * packed input buffer (network 0's leaves in order, then network 1's, ...; each leaf in
 * its declared order, row-major); the last entry is the buffer's length in elements.
 * flops (or NULL): algorithmic flops of one launch. threads / ctas_per_sm / nets_per_cta
 * (or NULL): the launch shape currently chosen (see tn_batch_autotune) -- threads per
 * network, resident CTAs per SM, networks per CTA (1: a CTA per network with block
 * barriers between steps; > 1: a warp per network, warp-synchronous steps), and the
 * shared-memory arena per network slot in floats (0: every arena in global memory; a
 * network whose arena is larger keeps its global arena). */
tn_status tn_batch_info(tn_batch_t b, int64_t* leaf_offsets, double* flops, int32_t* threads,
                        int32_t* ctas_per_sm, int32_t* nets_per_cta, int32_t* smem_arena);

/* Contract every network. packed_inputs: DEVICE buffer laid out as tn_batch_info says
 * (complex64 or float32). values: DEVICE, 2 doubles per network (real, imaginary; 0 for
 * real networks); log_scales: DEVICE, 1 double per network; result = value * exp(log).
 * Asynchronous on `stream`; calls on one batch must not overlap. */
tn_status tn_batch_contract(tn_batch_t b, const void* packed_inputs, double* values, double* log_scales,
                            void* stream);

/* As tn_batch_contract, replayed from a CUDA graph (queue reset + kernel) captured on
 * the first call and re-captured when any pointer or the stream changes. */
tn_status tn_batch_contract_graph(tn_batch_t b, const void* packed_inputs, double* values, double* log_scales,
                                  void* stream);

/* Time the batch under candidate launch shapes -- a CTA per network at 32-256 threads, or
 * a warp per network at 4 or 8 per CTA, each at 2-16 CTAs per SM, with every arena in
 * global memory or the arenas up to the largest size the shape leaves room for in shared
 * memory -- and keep the fastest for later calls. Writes results into values/log_scales as a side effect. Synchronous. */
tn_status tn_batch_autotune(tn_batch_t b, const void* packed_inputs, double* values, double* log_scales,
                            void* stream);

/* Set the launch shape by hand: threads per network (a multiple of 32, <= 1024), CTAs per
 * SM, networks per CTA (> 1 needs threads = 32: a warp per network), and smem_arena (the
 * shared-memory arena per network slot in floats, 0 for none: smem_arena x 4 bytes x
 * networks per CTA must fit a CTA's shared memory, and ctas_per_sm of those an SM's;
 * networks whose arena is larger run in global memory); at most 2048 threads per SM.
 * TN_ERR_INVALID otherwise. */
tn_status tn_batch_set_shape(tn_batch_t b, int32_t threads, int32_t ctas_per_sm, int32_t nets_per_cta,
                             int32_t smem_arena);

tn_status tn_batch_destroy(tn_batch_t b);

/* ---- allocation-free batched dot products ----------------------------------------- */

/* The paper has no counterpart to this call. It exists for callers that must not
 * allocate device memory on this path -- a host process whose device memory is already
 * handed out by another allocator, or a latency-critical loop where cudaMalloc (which
 * may synchronize the device) is not acceptable. It computes a reduction of the same
 * shape as the engine's split-K step (few outputs, long contracted index: k cut in
 * chunks of 4096, FP64 partial sums, chunks added in a fixed order), with its own pair
 * of kernels, on interleaved complex64 inputs, without exponent scaling or the max-plus
 * semiring. Its FP64 partial sums live in a fixed file-scope device array of 2^18
 * complex doubles (4 MiB) that every device using the library holds until the process
 * exits.
 *
 *   out[b][i][j] = sum_t a[b][i][t] * b[b][j][t]      (no conjugation)
 *
 * a: DEVICE complex64, [batch][m][k] row-major; b: DEVICE complex64, [batch][n][k];
 * out: DEVICE complex128, [batch][m][n]. All three are owned by the caller.
 * Limits: m*n <= 16, batch <= 65535, batch * ceil(k/4096) * m*n <= 2^18; larger sizes
 * (m and n are checked one at a time before their product) return TN_ERR_INVALID with a
 * message. Allocates nothing (no cudaMalloc/cudaFree, no allocating library call).
 * Asynchronous on `stream` (a cudaStream_t; NULL = legacy default stream). The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture. The address is kept
 * per device together with the id of the context it belongs to: after a device reset
 * (cudaDeviceReset) the next call sees a new context and looks the address up again,
 * so that call too belongs outside stream capture. All calls share the array: each call
 * overwrites every partial it reads, so calls in sequence need no clearing, but calls
 * that overlap on the GPU race. */
tn_status tn_dot_noalloc(const void* a, const void* b, int64_t batch, int64_t m, int64_t n, int64_t k,
                         void* out, void* stream);

/* ---- offline distribution planning (Sec. IV-B), host only ------------------------- */
/* For a built plan and a device count P, decide which steps run distributed over P
 * devices, which modes of each distributed intermediate are split across them, and where
 * along each use-chain to redistribute or gather; report the simulated time of one slice
 * under the cost model of Sec. IV-B. Nothing is executed and no device memory is used
 * (this library runs one GPU; the plan is the schedule a multi-GPU executor would follow).
 *
 *  * A step is large (Sec. IV-B) if an operand or its output holds >= large_bytes.
 *  * The first large step of a lineage activates distribution of its output: the modes
 *    split are the shortest leading prefix of the output's planned order (Sec. IV-A puts
 *    the longest-lived modes first) whose extents multiply to >= P (Eq. 4), skipping any
 *    mode the next step contracts.
 *  * Distribution follows the output into its consumer while the output holds >=
 *    gather_bytes; where two distributed tensors meet, the larger one carries on and the
 *    other is gathered (replicated). Each step of a use-chain keeps the modes it
 *    inherits (no communication) or redistributes its output to a fresh prefix (an
 *    all-to-all); keeping is not allowed when an inherited mode is contracted by the next
 *    step (a forced redistribution). A chain ends with a gather of its last output.
 *  * Step time (Eq. 6): t_gemm = max(bytes read and written per device / dev_bw,
 *    flops per device / dev_flops); a chain step splits its distributed operand, its
 *    output and its flops P ways and holds the other operand whole; other steps run
 *    whole on every device.
 *  * Redistribution of output C (Eq. 7): |C| (P-1) / (P net_bw) + n_blk max(latency,
 *    block_bytes / net_bw), where n_blk = |C| / (P * run) and run is the contiguous run of
 *    C's row-major layout below the innermost mode split before or after the shuffle
 *    (block_bytes: the base block size). A gather costs the same with nothing split after.
 *  * The keep/redistribute choices of each chain minimise its summed step and
 *    communication times by dynamic programming over the set of split modes (Sec. IV-B),
 *    with the gather added at the end; backtracking gives the redistribution points. */
typedef struct {
  int32_t n_gpus;        /* P >= 1 (P = 1: nothing is distributed) */
  int32_t reserved0;
  double large_bytes;    /* s of Sec. IV-B (8 GiB there) */
  double gather_bytes;   /* distributed outputs below this size are gathered; 0 = large_bytes */
  double dev_bw;         /* B_dev, bytes/s per device */
  double dev_flops;      /* F_dev, algorithmic flops/s per device (8 per complex MAC) */
  double net_bw;         /* B_net, bytes/s per device */
  double latency;        /* lambda, seconds per message */
  double block_bytes;    /* s_blk, base block size in bytes */
} tn_dist_config;

typedef enum {
  TN_DIST_NONE = 0,          /* runs whole on every device */
  TN_DIST_ACTIVATE = 1,      /* first step of a use-chain: its output is split (Eq. 4) */
  TN_DIST_KEEP = 2,          /* output inherits the split modes, no communication */
  TN_DIST_REDISTRIBUTE = 3,  /* output shuffled to fresh split modes (all-to-all) */
  TN_DIST_GATHER = 4         /* last step of a use-chain: output replicated */
} tn_dist_state;

#define TN_DIST_MAX_MODES 16

typedef struct {
  int32_t state;             /* tn_dist_state */
  int32_t forced;            /* REDISTRIBUTE only: 1 if keeping was not allowed */
  int32_t chain;             /* use-chain index, -1 if the step is not on one */
  int32_t n_dist;            /* modes of the output split across devices after the step */
  int32_t dist_modes[TN_DIST_MAX_MODES]; /* their labels, in the output's planned order */
  double t_gemm;             /* Eq. 6, seconds */
  double t_comm;             /* Eq. 7 redistribution or gather after the step, seconds */
  double out_bytes;          /* |C| of one slice */
  int64_t n_blk;             /* blocks per device of that redistribution or gather */
} tn_dist_step;

typedef struct {
  int32_t n_chains, n_redistributions, n_forced, n_gathers;
  int64_t n_large_steps;
  int64_t dp_states;         /* DP state evaluations over all chains */
  double t_total;            /* simulated seconds for one slice on P devices */
  double t_single;           /* the same path on one device (sum of Eq. 6) */
  double t_comm_total;       /* communication part of t_total */
  double bytes_redistributed;/* sum of |C| over redistributions and gathers */
  double speedup;            /* S_P = t_single / t_total (Eq. 9 with the path fixed) */
  double extra_speedup;      /* E_P = S_P / P (Eq. 10) */
  double projected_total;    /* T_P^proj = t_total * n_slices (Eq. 8) */
} tn_dist_report;

/* Plan the distribution of `plan` (any plan, host-only ones included) under `cfg`.
 * steps: NULL, or an array of the plan's n_steps entries to receive the per-step
 * schedule. TN_ERR_INVALID for a null plan/config, P < 1 or non-positive rates;
 * TN_ERR_UNSUPPORTED if a chain cannot be split P ways (a tensor with too few modes). */
tn_status tn_plan_distribute(tn_plan_t plan, const tn_dist_config* cfg, tn_dist_report* report,
                             tn_dist_step* steps);

/* Thread-local message for the last non-OK status on this thread. */
const char* tn_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TN_GB300_H */
