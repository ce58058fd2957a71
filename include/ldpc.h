/*
 * ldpc.h -- C ABI of the GB300 (sm_103a) syndrome-based sum-product LDPC
 * decoder with early termination.
 *
 * The operation (arXiv 2507.03509, section "Early Termination"): belief
 * propagation on the Tanner graph of a parity-check matrix H, at most D_max
 * iterations, each iteration a variable-node update, a check-node update
 * (tanh/atanh rule, sign flipped by the check's syndrome bit), a hard
 * decision with a parity check (PCE-ET: stop once H x^ = s), and the
 * variable-node-reliability test (VNR-ET: with q^(k) the sum over variable
 * nodes of degree > 1 of the a-posteriori LLR magnitude after iteration k,
 * stop once q^(k) < q^(k-1)).  Its throughput K = N R (1 - FER) / D_mean
 * (Eq. 2) is what early termination raises.
 *
 * Conventions used everywhere below:
 *   - H is m x n: rows are check nodes, columns variable nodes.
 *   - LLR L = ln P(x=0)/P(x=1); hard decision x^ = 1 iff L < 0.
 *   - The decoded word satisfies H x^ = s (mod 2) on success.
 *   - All sizes are element counts.  All arrays are dense and row-major.
 *
 * Errors: every call returns an ldpc_status; nothing aborts, traps or
 * prints.  Argument and graph errors are found on the host before any GPU
 * work is queued; errors found on the GPU (a syndrome byte not 0/1, a
 * synchronisation wait that ran out) come back from the same call.
 *
 * Threads: graph objects may be shared between threads for reading, but
 * one graph runs one decode at a time (its workspace is reused).
 */
#ifndef LDPC_GB300_LDPC_H
#define LDPC_GB300_LDPC_H

#include <stdint.h>

/* Symbols of the shared library are exported explicitly; everything else in
 * it is hidden. */
#if defined(__GNUC__)
#define LDPC_API __attribute__((visibility("default")))
#else
#define LDPC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ldpc_status {
    LDPC_OK = 0,
    LDPC_ERR_INVALID_ARG = 1,   /* null pointer, bad size, bad option, syndrome byte not 0/1 */
    LDPC_ERR_INVALID_GRAPH = 2, /* malformed CSR / QC description */
    LDPC_ERR_OOM = 3,           /* device or pinned-host allocation failed */
    LDPC_ERR_CUDA = 4,          /* a CUDA runtime call failed (no device, launch error, ...) */
    LDPC_ERR_TIMEOUT = 5,       /* a grid-wide wait inside the decoder ran out; results invalid */
    LDPC_ERR_TOO_LARGE = 6,     /* the problem does not fit ldpc_decode_qc_noalloc's fixed scratch */
    LDPC_ERR_BOUNDS = 7         /* debug aids: the index-checking build found an index outside its
                                   array, or a guard word around the decoder's arrays was overwritten */
} ldpc_status;

/* Termination rule (paper section "Early Termination"; the baselines of
 * section "Simulations" keep PCE-ET on and vary D_max). */
typedef enum ldpc_term_rule {
    LDPC_TERM_NONE = 0,    /* run exactly max_iter iterations; success = (H x^ = s) at the end */
    LDPC_TERM_PCE = 1,     /* stop with success once H x^ = s                                   */
    LDPC_TERM_PCE_VNR = 2  /* PCE-ET, then VNR-ET: abort once q^(k) < q^(k-1)                   */
} ldpc_term_rule;

/* Output flag bits, one byte per frame. */
#define LDPC_FLAG_SUCCESS 1u /* the final hard decision satisfies H x^ = s */
#define LDPC_FLAG_ABORTED 2u /* VNR-ET stopped the frame                   */

/* Opaque decoder graph: library-owned, device-resident, with a cached
 * workspace that grows on demand.  Bound to the CUDA device that was current
 * when it was created. */
typedef struct ldpc_graph ldpc_graph;

/* Optional statistics of one decode call (host struct, filled on return). */
typedef struct ldpc_decode_stats {
    float kernel_ms;          /* device time of the persistent decode kernel (CUDA events) */
    float total_ms;           /* device time of everything the call queued                  */
    int32_t kernel_launches;  /* kernels this call launched                                 */
    int32_t grid_ctas;        /* CTAs of the persistent kernel                              */
    int32_t threads_per_cta;
    int32_t active_frames;    /* frames decoded concurrently (slots)                        */
    int64_t frame_iterations; /* sum over frames of iterations run (the D of each frame)    */
} ldpc_decode_stats;

/* Decode options.  Always start from ldpc_decode_opts_init(). */
typedef struct ldpc_decode_opts {
    int32_t vnr_first_iter;    /* first k at which VNR-ET compares q^(k) < q^(k-1); default 2.
                                  1 compares q^(1) with q^(0) = sum over V of |Lch|.  >= 1.   */
    float clamp;               /* message limit LMAX: v2c and c2v are clamped to [-LMAX, LMAX];
                                  default 25.  Must be finite and > 0.                         */
    int32_t fp64;              /* 0: FP32 messages (default).  1: FP64 debug mode, which takes
                                  the tanh/atanh rule literally (slow on GB300's FP64 units).  */
    int32_t max_active_frames; /* frames decoded concurrently (slots), 0 = automatic: about
                                  192 MB of algorithmic traffic (8E + 12n bytes per frame and
                                  iteration) per CTA group and step, so 48 frames at n = 10^6
                                  with 8 groups, at most all frames and 1024.  Others wait in a
                                  queue and start as running frames terminate.  Rounded up to
                                  a multiple of the group count.                              */
    int32_t grid_ctas;         /* CTAs of the persistent kernel, 0 = all that fit on the GPU;
                                  rounded down to a multiple of the group count.              */
    int32_t trace_iters;       /* record messages of iterations 1..trace_iters (0 = off)      */
    void* trace_c2v;           /* device [trace_iters][frames][E] check-to-variable messages,
                                  edges in row-major order of H (CSR order; for QC codes the
                                  lifted matrix's, columns ascending in each row).  float when
                                  fp64 = 0, double when fp64 = 1.  May be NULL.                 */
    void* trace_app;           /* device [trace_iters][frames][n] a-posteriori LLRs; float or
                                  double as above.  May be NULL.                               */
    double* trace_q;           /* device [trace_iters][frames] q^(k).  May be NULL.           */
    ldpc_decode_stats* stats;  /* host; filled when not NULL                                   */
    int32_t barrier_timeout_ms; /* limit of one barrier wait inside the decoder; 0 = 10000.
                                   A wait that runs out ends the call with LDPC_ERR_TIMEOUT.   */
    int32_t test_unreachable_barrier; /* failure-injection hook for tests only: nonzero makes
                                   the first grid-wide wait expect one CTA more than the grid
                                   has, so the waits run out after barrier_timeout_ms and the
                                   call returns LDPC_ERR_TIMEOUT.  Leave 0.                    */
    int32_t groups;            /* independent CTA groups, 0 = automatic (two groups per
                                  resident CTA per SM, at most one group per running frame).  Each group
                                  advances its own frames in lock-step between its own
                                  barriers, and frames that stop are replaced from one shared
                                  queue.  Results are bit-identical for any value.             */
    int32_t schedule;          /* LDPC_SCHEDULE_*: how the persistent kernel orders its work.
                                  0 = automatic (frame per CTA pair or per CTA where it
                                  applies, lock-step otherwise).  Results are bit-identical
                                  for every schedule.                                          */
    int32_t flow_lag;          /* dataflow schedule only: how many slot-steps after a frame's
                                  check pass its variable pass is scheduled (0 = 2; at most the
                                  number of frames in flight).                                */
    int32_t debug_guards;      /* debug aid: nonzero places a 256-byte guard region before and
                                  after each of the decoder's workspace arrays and fills it
                                  before the decode; ldpc_graph_check_guards /
                                  ldpc_batch_check_guards then tell whether the decode wrote
                                  outside its arrays.  Default 0 (no guards).                 */
} ldpc_decode_opts;

/* Values of ldpc_decode_opts.schedule.  Automatic selection takes frame per
 * CTA pair (when every frame gets its own pair at once) or frame per CTA for
 * one small CSR code in FP32 (on GB300 at n = 4096 with 64 frames they ran
 * 2-3x faster than lock-step, the pair 3-4 % faster than one CTA) and
 * lock-step otherwise: at n = 10^6
 * with 32 frames the dataflow schedule measured half the lock-step rate (its
 * items wait on each frame's decision, a join over all of the frame's check
 * items, every iteration). */
#define LDPC_SCHEDULE_AUTO 0
/* Lock-step: CTA groups advance their frames between grid-wide barriers
 * (check pass of every frame in flight, barrier, decisions, variable pass,
 * barrier).  Any code, FP32 or FP64. */
#define LDPC_SCHEDULE_LOCKSTEP 1
/* Dataflow (QC codes only): no grid barriers.  Every CTA takes a fixed share
 * of one endless list of work items -- the variable pass of one frame and the
 * check pass of another, slot by slot -- and starts an item as soon as the
 * items of the previous pass that it reads are done (per-item completion
 * words), so one frame's new check messages are read back while still in L2. */
#define LDPC_SCHEDULE_DATAFLOW 2
/* Frame per CTA (one CSR code in FP32 whose frame and index lists fit a CTA's
 * shared memory: 16-bit indices, so n, m and E below 65536, and about
 * 8 E + 12 n + 4 m bytes up to 220 KB): each 1024-thread CTA takes whole frames
 * from the queue and decodes each in shared memory with CTA barriers only.
 * max_active_frames and groups do not apply.  Asking for it where it does not
 * apply returns LDPC_ERR_INVALID_ARG. */
#define LDPC_SCHEDULE_FRAME 3
/* Frame per cluster (where frame per CTA applies): a thread-block cluster of
 * two CTAs on two SMs decodes each frame, each CTA running half of the checks
 * and variables and storing the messages and APP values the other one reads
 * into its shared memory (distributed shared memory), with cluster barriers
 * between the passes.  grid_ctas counts CTAs (two per frame in flight).
 * Automatic selection takes it over frame per CTA when every frame gets its
 * own pair at once.  Asking for it where it does not apply returns
 * LDPC_ERR_INVALID_ARG. */
#define LDPC_SCHEDULE_FRAME_PAIR 4

/* Fill *opts with the defaults (vnr_first_iter 2, clamp 25, FP32, automatic
 * concurrency and grid, no trace, no stats).  NULL is ignored. */
LDPC_API void ldpc_decode_opts_init(ldpc_decode_opts* opts);

/* Build a decoder graph from a binary H in check-major CSR form: the Tanner
 * graph on which the paper's decoder passes messages (section "Early
 * Termination") has one check node per row of H and one variable node per
 * column, joined wherever H holds a 1.
 *   m, n     : checks, variables (m >= 1, n >= 1)
 *   row_ptr  : host int32 [m+1], row_ptr[0] = 0, non-decreasing
 *   col_idx  : host int32 [row_ptr[m]], each row strictly increasing, in [0, n)
 *   out      : receives the new graph (set to NULL on error)
 * Inputs are copied; the caller keeps ownership.  Limits: check degree
 * <= 64, edges < 2^31.  Rows of degree 0 are allowed (always satisfied).
 * Returns LDPC_ERR_INVALID_GRAPH for a malformed matrix. */
LDPC_API ldpc_status ldpc_graph_create_csr(int32_t m, int32_t n, const int32_t* row_ptr,
                                  const int32_t* col_idx, ldpc_graph** out);

/* Build a decoder graph for a quasi-cyclic H given by an mb x nb base matrix
 * of circulant shifts (host int32, row-major).  shifts[i*nb + j] = -1 is an
 * all-zero Z x Z block; s in [0, Z) connects check i*Z + t to variable
 * j*Z + (t + s) mod Z.  Limits: row weight <= 64, mb*Z, nb*Z and the edge
 * count < 2^31.  Copied; the caller keeps ownership. */
LDPC_API ldpc_status ldpc_graph_create_qc(int32_t mb, int32_t nb, int32_t Z, const int32_t* shifts,
                                 ldpc_graph** out);

/* Free a graph and its device workspace.  NULL is ignored.  Call it only when
 * no decode on the graph is in flight. */
LDPC_API void ldpc_graph_destroy(ldpc_graph* graph);

/* Report m, n and the edge count (nonzeros of H).  Any output may be NULL. */
LDPC_API ldpc_status ldpc_graph_info(const ldpc_graph* graph, int32_t* m, int32_t* n, int64_t* edges);

/* Decode `frames` frames with flooding sum-product BP and the chosen
 * termination rule (paper section "Early Termination").
 *   llr       : device float [frames][n] channel LLRs (finite values)
 *   syndrome  : device uint8 [frames][m], each byte 0 or 1
 *   max_iter  : D_max >= 1
 *   rule      : ldpc_term_rule
 *   bits_out  : device uint8 [frames][n], the final hard decision (0/1)
 *   flags_out : device uint8 [frames], LDPC_FLAG_* bits
 *   iters_out : device int32 [frames], iterations run (the frame's D)
 *   opts      : NULL for the defaults
 *   cuda_stream : cudaStream_t to queue on (NULL = legacy default stream)
 * All device buffers are caller-owned and must not overlap.  The work is
 * stream-ordered; the call returns after the stream has reached its end
 * (it reads one status word back), so outputs are ready on return.
 * frames = 0 returns LDPC_OK without GPU work. */
LDPC_API ldpc_status ldpc_decode(const ldpc_graph* graph, int32_t frames, const float* llr,
                        const uint8_t* syndrome, int32_t max_iter, ldpc_term_rule rule,
                        uint8_t* bits_out, uint8_t* flags_out, int32_t* iters_out,
                        const ldpc_decode_opts* opts, void* cuda_stream);

/* ldpc_decode with HOST buffers (same shapes and meaning): copies the inputs
 * to library-owned device staging, decodes, copies the outputs back, and
 * returns when they are in host memory.  Pinned host memory makes the copies
 * asynchronous and faster; pageable memory works too.  trace_* options must
 * be NULL here. */
LDPC_API ldpc_status ldpc_decode_host(const ldpc_graph* graph, int32_t frames, const float* llr,
                             const uint8_t* syndrome, int32_t max_iter, ldpc_term_rule rule,
                             uint8_t* bits_out, uint8_t* flags_out, int32_t* iters_out,
                             const ldpc_decode_opts* opts, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Batches of frames of several codes (different lengths, rates and noise
 * levels) decoded by one persistent kernel: frames that stop early are
 * replaced by waiting ones, whatever their code.  Not in the paper, whose
 * decoder design is not given; built for streams of reconciliation frames.
 * ------------------------------------------------------------------------- */
typedef struct ldpc_batch ldpc_batch;

/* Plan a batch: frame f is decoded with graphs[frame_graph[f]].
 *   graphs      : 1..4 graphs of one kind (all QC or all CSR), same device
 *   frame_graph : host int32 [frames], values in [0, n_graphs)
 * The frames' values sit back to back in the batch buffers: frame f's LLRs
 * and decided bits start at the sum of n over frames 0..f-1, its syndrome
 * bytes at the sum of m (ldpc_batch_info gives the totals).  The plan copies
 * these tables to the device and owns a workspace; the graphs must outlive
 * it.  One decode at a time per plan. */
LDPC_API ldpc_status ldpc_batch_create(const ldpc_graph* const* graphs, int32_t n_graphs, int32_t frames,
                                       const int32_t* frame_graph, ldpc_batch** out);
LDPC_API void ldpc_batch_destroy(ldpc_batch* batch);
/* frames, and the lengths of the concatenated LLR (= bits) and syndrome buffers. */
LDPC_API ldpc_status ldpc_batch_info(const ldpc_batch* batch, int32_t* frames, int64_t* llr_len,
                                     int64_t* syndrome_len);
/* As ldpc_decode, on the batch's buffers: llr float / bits_out uint8 [llr_len],
 * syndrome uint8 [syndrome_len], flags_out uint8 / iters_out int32 [frames].
 * Traces are not available for batches.  Returns when the results are ready. */
LDPC_API ldpc_status ldpc_batch_decode(ldpc_batch* batch, const float* llr, const uint8_t* syndrome,
                                       int32_t max_iter, ldpc_term_rule rule, uint8_t* bits_out,
                                       uint8_t* flags_out, int32_t* iters_out, const ldpc_decode_opts* opts,
                                       void* cuda_stream);
/* The same, stream-ordered and without waiting for the GPU: the outcome is
 * written to the device int32 *status_out as an ldpc_status code when the
 * stream reaches it.  Nothing in it synchronises with the host, so it can be
 * captured in a CUDA graph and replayed; run it (or ldpc_batch_decode) once
 * with the same options before capturing, so that the workspace exists
 * (LDPC_ERR_INVALID_ARG otherwise).  opts->stats is ignored. */
LDPC_API ldpc_status ldpc_batch_decode_async(ldpc_batch* batch, const float* llr, const uint8_t* syndrome,
                                             int32_t max_iter, ldpc_term_rule rule, uint8_t* bits_out,
                                             uint8_t* flags_out, int32_t* iters_out, int32_t* status_out,
                                             const ldpc_decode_opts* opts, void* cuda_stream);
/* Autotuner: decodes the given inputs once per candidate block schedule (CTA
 * groups 1, 2, 4, 8 x frames in flight: all, 8 per group, 2 per group) and
 * keeps the fastest by kernel time; then, for QC codes, it tunes each code's
 * item sizes (checks of a base row per item: 512-4096; variables of a base
 * column: 1024-8192) one code and side at a time from the built-in model's
 * pick.  The plan uses the result for its later decodes whose opts leave
 * groups / max_active_frames at 0.  Results do not depend on any of these
 * choices; the outputs hold the last candidate's results.  best_groups /
 * best_slots may be NULL. */
LDPC_API ldpc_status ldpc_batch_autotune(ldpc_batch* batch, const float* llr, const uint8_t* syndrome,
                                         int32_t max_iter, ldpc_term_rule rule, uint8_t* bits_out,
                                         uint8_t* flags_out, int32_t* iters_out, void* cuda_stream,
                                         int32_t* best_groups, int32_t* best_slots);

/* Device scratch that ldpc_decode_qc_noalloc works in: one fixed array of this
 * many bytes, reserved on every GPU that loads the library, for as long as the
 * library stays loaded. */
#define LDPC_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)

/* ldpc_graph_create_qc + ldpc_decode in one call that allocates nothing.
 * The paper has no counterpart: this is a service for callers that must not
 * allocate device memory themselves -- real-time reconciliation loops whose
 * latency budget cannot absorb cudaMalloc/cudaFree (both can synchronise the
 * device and take unbounded time), and host processes whose memory manager
 * reserves the GPU's memory up front and forbids allocations outside it.
 *
 * Arguments: the QC base matrix as in ldpc_graph_create_qc (host int32
 * mb x nb, -1 = zero block), then the inputs and outputs as in ldpc_decode
 * (device buffers, caller-owned).  The decode uses the default options (FP32,
 * vnr_first_iter 2, clamp 25).  The graph tables and all decoder state live in
 * one file-scope device array of LDPC_NOALLOC_SCRATCH_BYTES; as many frames as
 * fit are decoded at once and the rest wait in the queue.
 * Schedule: one CTA group over the whole grid and the default item sizes
 * (2048 checks, 4096 variables), whatever ldpc_decode would pick; results are
 * bit-identical to ldpc_decode's, only the speed differs.
 *
 * Limits: the packed syndrome of all frames plus the state of one frame
 * (about 14 bytes per edge plus 8 bytes per variable) must fit the scratch,
 * else LDPC_ERR_TOO_LARGE is returned before any GPU work.
 *
 * Set-up: the first call on each device looks up that device's address of the
 * scratch array (with that device current); later calls reuse it.
 * Sharing: every call on a device uses the same scratch, which keeps whatever
 * the previous call left (the call clears what has to start at zero).  Calls
 * whose GPU work overlaps -- on two streams, or from two threads -- race on it,
 * so callers must order them.  The call returns after its stream has drained. */
LDPC_API ldpc_status ldpc_decode_qc_noalloc(int32_t mb, int32_t nb, int32_t Z, const int32_t* shifts,
                                            int32_t frames, const float* llr, const uint8_t* syndrome,
                                            int32_t max_iter, ldpc_term_rule rule, uint8_t* bits_out,
                                            uint8_t* flags_out, int32_t* iters_out, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Weighted belief propagation (trainable decoder)
 *
 * The sum-product decoder of ldpc_decode (paper, section "Early Termination":
 * tanh/atanh check rule with the syndrome sign, l_out the a-posteriori value)
 * unrolled for exactly `iters` flooding iterations, without early
 * termination, with one weight per (iteration k, edge class cl) that scales
 * every check-to-variable message of that class:
 *     c2v_e^(k) = w[k][class(e)] * clamp((1 - 2 s_c) * boxplus of the other
 *                 clamped v2c messages of check c, +-25)
 * (a degree-1 check sends (1 - 2 s_c) * 25).  The calls below run it forward,
 * evaluate a binary cross-entropy loss on its soft output, run its adjoint
 * (the exact reverse-mode gradient w.r.t. the weights and the channel LLRs)
 * with recomputation from checkpoints, and take a plain gradient step.
 *
 * Element type: the plan's arithmetic type -- float, or double when the plan
 * is created with fp64 = 1.  Every buffer typed `void*` below holds that type.
 * All buffers are device buffers owned by the caller; the plan owns its
 * workspace (allocated at creation).  No call allocates or waits for the GPU:
 * each is stream-ordered and can be captured in a CUDA graph.  Calls on one
 * plan share its workspace, so their GPU work must not overlap (order them on
 * one stream).  Syndrome and bit bytes count as 1 when nonzero.
 * ------------------------------------------------------------------------- */
typedef struct ldpc_wbp ldpc_wbp;

/* Plan for `frames` frames of `graph`, `iters` iterations, `n_classes` weight
 * classes.  edge_class (host, copied): for a QC graph one class per nonzero
 * base block, in row-major block order (length = nonzero blocks); for a CSR
 * graph one class per edge in CSR order (length = edges); values in
 * [0, n_classes).  checkpoint_every (>= 1): the forward pass keeps the
 * messages of every checkpoint_every-th iteration, and the backward pass
 * recomputes the iterations in between.  The iterations of the last segment
 * (after the last checkpoint) are kept whole by the forward pass, since the
 * backward pass needs them first (1 = keep all; >= iters = keep all but the
 * last).  FP32 QC plans own a second CUDA stream, on which the backward pass
 * recomputes one segment while the adjoint of the next runs on the caller's
 * stream; it joins the caller's stream before the call's work ends.
 * The graph must outlive the plan.  LDPC_ERR_INVALID_ARG on bad sizes or
 * classes. */
LDPC_API ldpc_status ldpc_wbp_create(const ldpc_graph* graph, int32_t frames, int32_t iters, int32_t n_classes,
                                     const int32_t* edge_class, int32_t checkpoint_every, int32_t fp64,
                                     ldpc_wbp** out);
LDPC_API void ldpc_wbp_destroy(ldpc_wbp* plan);
/* Forward pass: llr float [frames][n], syndrome uint8 [frames][m], weights
 * [iters][n_classes]; writes app_out [frames][n] = APP after the last
 * iteration.  With save_for_backward the checkpoints a later ldpc_wbp_backward
 * needs are kept in the plan (the next forward with it set replaces them). */
LDPC_API ldpc_status ldpc_wbp_forward(ldpc_wbp* plan, const float* llr, const uint8_t* syndrome,
                                      const void* weights, void* app_out, int32_t save_for_backward,
                                      void* cuda_stream);
/* Loss: loss_out[0] = mean over frames*n bits of softplus(-(1 - 2 x) APP),
 * the binary cross-entropy of P(x = 1) = 1 / (1 + e^APP) against x uint8
 * [frames][n]; if grad_app is not NULL it receives dloss/dAPP [frames][n]. */
LDPC_API ldpc_status ldpc_wbp_loss(ldpc_wbp* plan, const void* app, const uint8_t* x, void* loss_out,
                                   void* grad_app, void* cuda_stream);
/* Backward pass for the last forward with save_for_backward (same llr,
 * syndrome and weights, unchanged since): from grad_app = dloss/dAPP
 * [frames][n] writes grad_weights [iters][n_classes] and, if not NULL,
 * grad_llr [frames][n] = dloss/dLch.  LDPC_ERR_INVALID_ARG if the plan keeps
 * iterations and no forward has saved them. */
LDPC_API ldpc_status ldpc_wbp_backward(ldpc_wbp* plan, const float* llr, const uint8_t* syndrome,
                                       const void* weights, const void* grad_app, void* grad_weights,
                                       void* grad_llr, void* cuda_stream);
/* Early-terminating decode (as ldpc_decode, same arguments and options) with
 * the plan's learned weights: in iteration k every check-to-variable message
 * of class cl is scaled by weights[min(k, iters) - 1][cl] (iterations past the
 * plan's last keep its weights).  weights: device float [iters][n_classes]
 * (float whatever the plan's type; opts->fp64 selects the decoder's
 * arithmetic).  The plan's graph and class map are used; `frames` is
 * independent of the plan's frame count.  Traces are available as in
 * ldpc_decode.  Returns when the results are ready. */
LDPC_API ldpc_status ldpc_wbp_decode(const ldpc_wbp* plan, int32_t frames, const float* llr, const uint8_t* syndrome,
                                     const float* weights, int32_t max_iter, ldpc_term_rule rule, uint8_t* bits_out,
                                     uint8_t* flags_out, int32_t* iters_out, const ldpc_decode_opts* opts,
                                     void* cuda_stream);
/* weights -= lr * grad over [iters][n_classes] (a plain gradient step). */
LDPC_API ldpc_status ldpc_wbp_sgd_step(ldpc_wbp* plan, void* weights, const void* grad, double lr,
                                       void* cuda_stream);

/* Debug aids.  After a decode (ldpc_decode, ldpc_decode_host, ldpc_wbp_decode
 * on the graph's workspace; ldpc_batch_* on the batch's) run with
 * opts->debug_guards set, report whether every guard region around the
 * workspace's arrays still holds its fill: LDPC_OK, LDPC_ERR_BOUNDS if any
 * byte changed, LDPC_ERR_INVALID_ARG if the last decode placed no guards.
 * Waits for the device to finish.
 *
 * A library built with -DLDPC_BOUNDS_CHECK (the binding builds and loads one,
 * libldpc_gb300_checked.so, when the environment sets LDPC_GB300_CHECKED=1)
 * tests every index its decode kernels compute against the array it indexes;
 * the first index outside ends the decode with LDPC_ERR_BOUNDS (the access
 * itself is redirected to element 0, so nothing outside is touched). */
LDPC_API ldpc_status ldpc_graph_check_guards(const ldpc_graph* graph);
LDPC_API ldpc_status ldpc_batch_check_guards(const ldpc_batch* batch);

/* Static, human-readable name of a status code. */
LDPC_API const char* ldpc_status_str(ldpc_status status);

#ifdef __cplusplus
}
#endif

#endif /* LDPC_GB300_LDPC_H */
