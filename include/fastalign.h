/*
 * fastalign.h -- C ABI of the GB300 (sm_103a) implementation of the
 * per-outer-iteration transport-plan update of FastAlign's OT-based network
 * alignment ("Scalable Optimal Transport Algorithm for Network Alignment",
 * Algorithm 1, Eq. 1-4).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every call returns fa_status and never aborts or throws.  On failure
 *   fa_last_error_string() (per thread) describes the cause.
 * - "host" pointers are read before the call returns.  "device" pointers
 *   are CUDA device memory owned by the caller; the library never frees
 *   them.  The library owns only what it allocates inside a handle
 *   (fa_graph, fa_ctx, fa_gnn) and frees it in the matching *_destroy.
 * - Calls that take a cudaStream_t enqueue their work on that stream and
 *   return without synchronising, except where they return a host scalar
 *   (fa_sinkhorn, fa_plan_change), which synchronises that stream only.
 * - One fa_ctx serves one host thread and one stream at a time.
 * - Dense n1 x n2 matrices are row-major with a padded leading dimension
 *   ld = fa_ctx_ld(ctx) >= n2 (a multiple of 128 elements).  Padding columns
 *   of the Gibbs kernel K are written as 0 and must stay 0.
 * - The transport plan is held implicitly as
 *       T_ij = exp(log_u_i) * K_ij * exp(log_v_j)
 *   with K the row-stabilised Gibbs kernel (float32 or bfloat16 storage),
 *   log_u (n1) and log_v (n2) float32 log-scalings.  These are the
 *   exponentiated dual potentials of Eq. 3/Eq. 4 (b_i/eps and a_j/eps) up
 *   to the stabilising row offsets folded into K.
 */
#ifndef FASTALIGN_H
#define FASTALIGN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* cudaStream_t without pulling in the CUDA headers. */
typedef struct CUstream_st* fa_stream_t;

typedef enum {
  FA_OK = 0,
  FA_ERR_ARG = 1,            /* invalid argument (sizes, null pointers, bad graph) */
  FA_ERR_OOM = 2,            /* a device allocation inside a handle failed */
  FA_ERR_CUDA = 3,           /* a CUDA runtime call or kernel launch failed */
  FA_ERR_NOT_CONVERGED = 4,  /* fa_sinkhorn hit max_iter with err > tol */
  FA_ERR_NUMERIC = 5,        /* NaN/Inf or an all-zero row/column was met */
  FA_ERR_UNSUPPORTED = 6,    /* size or mode outside what the kernels support */
  FA_ERR_TIMEOUT = 7         /* a bounded device-side wait gave up */
} fa_status;

typedef enum { FA_F32 = 0, FA_BF16 = 1 } fa_dtype;

/* GEMM engine for the node-similarity cost (Algorithm 1, node cost). */
typedef enum {
  FA_GEMM_AUTO = 0,      /* tcgen05: bf16 operands for FA_BF16, 3xTF32 split for FA_F32 */
  FA_GEMM_TCGEN05 = 1,   /* same as AUTO */
  FA_GEMM_SIMT = 2       /* plain FP32 CUDA-core GEMM (cross-check path) */
} fa_gemm_mode;

/* Hyper-parameters of Algorithm 1 (named in the paper, values unstated). */
typedef struct {
  int32_t dtype;              /* fa_dtype: storage type of the Gibbs kernel K */
  float eps;                  /* entropic regulariser (Eq. 1, Eq. 3) */
  float eps_anc;              /* eps inside C_anc = -log(eps_anc + OneHot(L)) (Algorithm 1, anchor cost) */
  float alpha;                /* node-cost mix (Algorithm 1, node cost) */
  float beta;                 /* RWR restart probability (Algorithm 1, RWR) */
  int32_t k_rwr;              /* RWR iterations (Algorithm 1, RWR) */
  int32_t k_prop;             /* C_node propagation steps A1bar C A2bar^T (Algorithm 1) */
  float lam_e, lam_n, lam_a;  /* cost weights (Eq. 2) */
  float lam_p;                /* proximal weight: C_eff = C - lam_p log T_prev */
  float delta;                /* clamp inside -log(max(., delta)) of C_nbr */
  int32_t normalize_features; /* 1: unit-L2 attribute rows before X1 X2^T */
  int32_t gemm_mode;          /* fa_gemm_mode */
} fa_params;

/* Fills *p with the library defaults (eps = eps_anc = lam_p = 0.05,
 * alpha = 0.5, beta = 0.15, k_rwr = 10, k_prop = 1, lam_e = 1,
 * lam_n = lam_a = 0.05, delta = 1e-30, normalize_features = 1, FA_F32). */
void fa_params_default(fa_params* p);

typedef struct fa_graph fa_graph;
typedef struct fa_ctx fa_ctx;

/* ----------------------------------------------------------------------
 * fa_build_graph -- Algorithm 1, row normalisation (Section 3.3 sparse form).
 * n: node count (>= 1).  src, dst: host int32 arrays of n_edges undirected
 * edges; self-loops and duplicates are dropped, node ids must lie in
 * [0, n) (FA_ERR_ARG otherwise).  Builds on the current device the CSR of
 * the symmetric adjacency A (int32 row_ptr/col, columns sorted) with the
 * values of Abar = D^-1 A and of Abar^T; degree-0 rows are empty.
 * *out receives a handle freed by fa_graph_destroy.  Synchronous.
 * -------------------------------------------------------------------- */
fa_status fa_build_graph(int32_t n, int64_t n_edges, const int32_t* src,
                         const int32_t* dst, fa_graph** out);

/* ----------------------------------------------------------------------
 * fa_graph_csr_host -- the host half of fa_build_graph (Algorithm 1, row normalisation), with
 * no device work: the same CSR, returned in caller-owned host arrays.
 * Call once with row_ptr = col = val_row = val_col = NULL to get *nnz_out;
 * then with row_ptr of n + 1 entries and col, val_row (1/deg_i, Abar) and
 * val_col (1/deg_k, Abar^T) of cap >= *nnz_out entries (FA_ERR_ARG
 * otherwise).  Same argument checks and errors as fa_build_graph.
 * -------------------------------------------------------------------- */
fa_status fa_graph_csr_host(int32_t n, int64_t n_edges, const int32_t* src,
                            const int32_t* dst, int64_t* nnz_out, int32_t* row_ptr,
                            int32_t* col, float* val_row, float* val_col, int64_t cap);

fa_status fa_graph_destroy(fa_graph* g);
/* n and nnz (= 2 x unique undirected edges) of a built graph. */
fa_status fa_graph_info(const fa_graph* g, int32_t* n, int64_t* nnz);

/* ----------------------------------------------------------------------
 * fa_ctx_create -- an alignment context for the pair (g1, g2).  Copies
 * *params, allocates the device workspaces of the outer iteration (the
 * transposed left-product buffer, the log-kernel scratch, partial sums).
 * The graphs must outlive the context.  fa_ctx_ld gives the padded leading
 * dimension ld of every n1 x n2 matrix passed to the other calls;
 * fa_ctx_workspace_bytes the device bytes the context holds.
 * -------------------------------------------------------------------- */
fa_status fa_ctx_create(const fa_graph* g1, const fa_graph* g2,
                        const fa_params* params, fa_ctx** out);
fa_status fa_ctx_destroy(fa_ctx* ctx);
int64_t fa_ctx_ld(const fa_ctx* ctx);
int64_t fa_ctx_workspace_bytes(const fa_ctx* ctx);

/* ----------------------------------------------------------------------
 * fa_node_cost -- Phase 1 of Algorithm 1:
 *   R_g  <- k_rwr steps of (1-beta) Abar_g R_g + beta R_g^(0)     (RWR)
 *   C_node = alpha exp(-R1 R2^T) + (1-alpha) exp(-X1h X2h^T)      (node cost)
 *   C_node <- k_prop steps of A1bar C_node A2bar^T                 (propagation)
 *   C1 = (R1 R1^T) .* A1bar,  C2 = (R2 R2^T) .* A2bar^T  (SDDMM)    (intra-graph costs)
 * X1 (n1 x d), X2 (n2 x d): device float32 row-major attributes (d >= 1,
 * may be NULL with d = 0 to drop the attribute term's variation: exp(0)).
 * anchors: host int32 [n_anchor][2] pairs (i, j); 0 <= n_anchor.
 * C_node: device float32 n1 x ld output (padding columns set to 0).
 * C1/C2 values and the anchor list stay in ctx for fa_align_iter.
 * The GEMM runs on tcgen05 tensor cores (see fa_gemm_mode).
 * -------------------------------------------------------------------- */
fa_status fa_node_cost(fa_ctx* ctx, const float* X1, const float* X2,
                       int32_t d, const int32_t* anchors, int32_t n_anchor,
                       float* C_node, fa_stream_t stream);

/* ----------------------------------------------------------------------
 * fa_plan_init -- the independent coupling T0 = mu nu^T (mu = 1/n1,
 * nu = 1/n2, Section 2.1): K = 1 (0 in padding), log_u = log mu,
 * log_v = log nu.  K: device n1 x ld of params.dtype; log_u (n1), log_v
 * (n2): device float32.
 * -------------------------------------------------------------------- */
fa_status fa_plan_init(fa_ctx* ctx, void* K, float* log_u, float* log_v,
                       fa_stream_t stream);

/* ----------------------------------------------------------------------
 * fa_align_iter -- Phase 2 of one outer iteration (Algorithm 1) and
 * the Gibbs kernel of the proximal step:
 *   W   = P1 T_prev           P1 in {C1, A1bar^T}        (left SpMMs)
 *   Z   = W P2^T              P2 in {C2, A2bar^T}         (right SpMMs)
 *   C   = C_node + lam_e Z_e - lam_n log max(Z_n, delta) + lam_a C_anc
 *   log K_new = -C/eps + (lam_p/eps) log T_prev,  row-max stabilised
 * then the first Sinkhorn column update a_1 (Eq. 3, Algorithm 1 Phase 3) from the
 * row-stabilised start b0.
 * In:  K (T_prev's kernel), log_u, log_v, C_node (from fa_node_cost).
 * Out: K overwritten in place by the new row-stabilised kernel (row max 1),
 *      log_u = 0, log_v = a_1 / eps.
 * -------------------------------------------------------------------- */
fa_status fa_align_iter(fa_ctx* ctx, void* K, float* log_u, float* log_v,
                        const float* C_node, fa_stream_t stream);

/* ----------------------------------------------------------------------
 * fa_sinkhorn -- Phase 3 of Algorithm 1 (Eq. 3) on a fixed kernel K.
 * One fused sweep per iteration reads K once: the row update
 * u_i = mu_i / sum_j K_ij v_j (b update) and, in the same pass, the column
 * sums sum_i K_ij u_i for the next column update (a update).  The L1
 * marginal error |T^T 1 - nu|_1 of the plan after each b update is
 * computed in FP64 on the device.
 * In: log_v holds the current column scaling (a_1 from fa_align_iter) unless
 *     warm_log_v (device n2 float32, nullable) is given, which replaces it.
 * Runs until err <= tol at a checked iteration (every check_every
 * iterations; tol < 0 disables the check) or max_iter iterations.
 * Out: log_u, log_v of the last completed iteration (a_t, b_t); *iters_out,
 *      *err_out (host, nullable) its count and error.
 * Returns FA_ERR_NOT_CONVERGED (state still valid) when tol >= 0 and the
 * cap was hit, FA_ERR_NUMERIC on NaN/Inf or an all-zero row or column,
 * FA_ERR_TIMEOUT when a bounded device-side wait gave up (results invalid;
 * the context stays usable).  Both conditions are status bits kept in the
 * context: a bit set by an earlier asynchronous call on it (fa_node_cost,
 * fa_align_iter) is reported here too, and every bit is cleared once
 * reported.  FA_ERR_TIMEOUT takes precedence.  FA_ERR_UNSUPPORTED when no
 * sweep shape fits a row of ld columns (ld > 196608; see fa_sweep_plan).
 * Synchronises the stream when it reads the error back.
 * -------------------------------------------------------------------- */
fa_status fa_sinkhorn(fa_ctx* ctx, const void* K, float* log_u, float* log_v,
                      const float* warm_log_v, int32_t max_iter, double tol,
                      int32_t check_every, int32_t* iters_out, double* err_out,
                      fa_stream_t stream);

/* ----------------------------------------------------------------------
 * fa_topk -- alignment read-out (Eq. 4, Section 4.1.1): per row i the k
 * columns with the largest T_ij (ties to the lower j).  1 <= k <= 32.
 * idx: device int32 n1 x k; score: device float32 n1 x k (T_ij / u_i,
 * i.e. K_ij v_j), nullable.
 * -------------------------------------------------------------------- */
fa_status fa_topk(fa_ctx* ctx, const void* K, const float* log_v, int32_t k,
                  int32_t* idx, float* score, fa_stream_t stream);

/* ----------------------------------------------------------------------
 * fa_rank -- 1-based rank of column cols[t] in row rows[t] under the same
 * order as fa_topk: 1 + #{j: T_ij > T_ic} + #{j < c: T_ij == T_ic}
 * (Section 4.1.1, Hits@K and MRR).  rows, cols, rank_out: device int32
 * arrays of n_query entries.
 * -------------------------------------------------------------------- */
fa_status fa_rank(fa_ctx* ctx, const void* K, const float* log_v,
                  int32_t n_query, const int32_t* rows, const int32_t* cols,
                  int32_t* rank_out, fa_stream_t stream);

/* ----------------------------------------------------------------------
 * Kernel-level timing of the last fa_sinkhorn call: average device time of
 * one fused sweep (ms), measured with CUDA events on the call's stream
 * when enabled by fa_ctx_set_timing(ctx, 1).
 * -------------------------------------------------------------------- */
fa_status fa_ctx_set_timing(fa_ctx* ctx, int32_t on);
fa_status fa_ctx_last_sweep_ms(const fa_ctx* ctx, double* ms, int32_t* n);

/* ======================================================================
 * Learned warm start of the Sinkhorn solves.  The paper has no learned
 * component: this is a small 2-layer graph network on the column graph
 * G2 (hidden width 64, BF16 weights, FP32 accumulation) that predicts the
 * change of the correction y = log v* - log v1 between the converged
 * column scaling of a solve and its cold first column update, so that
 * fa_sinkhorn can start from warm_log_v = log v1 + c_prev + prediction.
 *
 *   AF = Abar F,  A1 = AF W1 + b1,  H = relu(A1),  z2 = H w2,
 *   a  = Abar z2 + c,
 *   L  = 1/n sum_j ((a_j - mean a) - (y_j - mean y))^2   (gauge invariant)
 *
 * Parameters (FP32 master copy, FA_GNN_NPARAMS floats): W1 [6 x 64,
 * row-major] | b1 [64] | w2 [64] | c.  The forward pass reads BF16 copies
 * of W1 and w2 refreshed by fa_gnn_set_params and fa_gnn_adam_step.
 * ====================================================================== */
#define FA_GNN_FIN 6
#define FA_GNN_HIDDEN 64
#define FA_GNN_NPARAMS (FA_GNN_FIN * FA_GNN_HIDDEN + 2 * FA_GNN_HIDDEN + 1)

typedef struct fa_gnn fa_gnn;

/* A model with all parameters and the Adam state set to zero. */
fa_status fa_gnn_create(fa_gnn** out);
fa_status fa_gnn_destroy(fa_gnn* g);
/* host_theta: FA_GNN_NPARAMS floats (host).  Resets the Adam state.
 * Synchronous. */
fa_status fa_gnn_set_params(fa_gnn* g, const float* host_theta);
fa_status fa_gnn_get_params(const fa_gnn* g, float* host_theta);
/* Floats of caller-owned device workspace the calls below need for a
 * graph of n nodes (activations kept for the backward pass, partial sums);
 * -1 if n < 1. */
int64_t fa_gnn_workspace_floats(int32_t n);

/* Per-node inputs F (device, n x FA_GNN_FIN row-major) of the column graph
 * g2, column j:
 *   0  log_v1_j - mean log_v1        (the solve's cold first column update)
 *   1  corr_prev_j - mean corr_prev  (the previous solve's correction)
 *   2  log(1 + deg_j)
 *   3  pot_prev_j - mean pot_prev    (the previous solve's converged log v)
 *   4  anchor_mask_j                 (1 if column j is an anchor's partner)
 *   5  log(1 + outer_index)          (outer iterations done before this one)
 * Potentials are defined up to a constant, so they are centred.  corr_prev,
 * pot_prev and anchor_mask are device vectors of n floats, each nullable
 * (= zeros, as for the first solve); outer_index >= 0 (FA_ERR_ARG
 * otherwise).  ws: workspace of fa_gnn_workspace_floats(n). */
fa_status fa_gnn_features(const fa_graph* g2, const float* log_v1,
                          const float* corr_prev, const float* pot_prev,
                          const float* anchor_mask, int32_t outer_index, float* F,
                          float* ws, fa_stream_t stream);
/* a_out (device, n) = model(F) on graph g; keeps activations in ws. */
fa_status fa_gnn_forward(fa_gnn* m, const fa_graph* g, const float* F,
                         float* ws, float* a_out, fa_stream_t stream);
/* Gradient of L for the forward pass whose activations ws holds.
 * grad: device, FA_GNN_NPARAMS floats (overwritten); loss: device scalar
 * (nullable). */
fa_status fa_gnn_backward(fa_gnn* m, const fa_graph* g, const float* ws,
                          const float* a_pred, const float* target,
                          float* grad, float* loss, fa_stream_t stream);
/* One Adam step (bias-corrected) of the FP32 master parameters with the
 * device gradient grad; refreshes the BF16 copies. */
fa_status fa_gnn_adam_step(fa_gnn* m, const float* grad, float lr,
                           float beta1, float beta2, float eps,
                           fa_stream_t stream);
/* The warm start handed to fa_sinkhorn:
 *   out = log_v1 + scale * clamp(pred, -max_abs, max_abs)
 * (device vectors of n floats; scale: device scalar, nullable = 1); a
 * non-finite prediction leaves that column at its cold value.  Bounding
 * the correction keeps the FP32 column scaling finite whatever the model
 * predicts. */
fa_status fa_gnn_warm_start(int32_t n, const float* log_v1, const float* pred,
                            float max_abs, const float* scale, float* out,
                            fa_stream_t stream);
/* The least-squares scale of a prediction against the change it was meant
 * to predict, clipped to [0, 1]:
 *   p = clamp(pred, -max_abs, max_abs) (non-finite -> 0),
 *   a = clip( sum_j (p_j - mean p)(y_j - mean y) / sum_j (p_j - mean p)^2, 0, 1 )
 * (0 when p is constant).  shrink selects a further factor from rho, the
 * correlation of p and y, so that a prediction that explains little of y
 * is trusted little: 1 -> a rho^2, 2 -> a |rho|, anything else -> a.
 * Centred because potentials are defined up to a constant.  pred, y: device vectors of n floats; scale: device scalar.
 * Fixed-order FP64 sums.  Used after each solve to damp the next solve's
 * prediction by how well the last one matched (0: the previous-correction
 * start, 1: the network's own prediction). */
fa_status fa_gnn_fit_scale(int32_t n, const float* pred, const float* y, float max_abs,
                           int32_t shrink, float* scale, fa_stream_t stream);
/* out = a x + b y on device vectors of n floats (y nullable = 0). */
fa_status fa_vec_axpby(int32_t n, float a, const float* x, float b,
                       const float* y, float* out, fa_stream_t stream);

/*
 * fa_plan_change -- how far the plan moved between two outer iterations,
 * the convergence test of Algorithm 1's outer loop (repeat until the plan converges;
 * reading: the L1 distance of the plans):
 *     *l1_out = sum_ij | T_a,ij - T_b,ij |,
 *     T = diag(exp(log_u)) K diag(exp(log_v)).
 * K_a, K_b: device, n1 x ld in the context's storage type (padding columns
 * ignored); log_u_* (n1), log_v_* (n2): device float32.  Each element's two
 * plan values are formed in float32 and their differences summed in
 * float64 in a fixed order.  l1_out: host; synchronises `stream`.
 * FA_ERR_NUMERIC if the sum is not finite.
 */
fa_status fa_plan_change(fa_ctx* ctx, const void* K_a, const float* log_u_a,
                         const float* log_v_a, const void* K_b, const float* log_u_b,
                         const float* log_v_b, double* l1_out, fa_stream_t stream);

/* ----------------------------------------------------------------------
 * fa_sinkhorn_step_static -- one fused Sinkhorn iteration that allocates
 * no device memory.  The paper has no counterpart: this entry serves
 * callers that cannot allocate device memory while they run, for example a
 * serving process whose memory budget is fixed at start-up (another
 * framework owns the device memory pool and forbids raw allocations), or a
 * latency-critical loop that cannot afford cudaMalloc's cost and implicit
 * synchronisation.  It needs no fa_ctx (creating one allocates).
 *
 * Computes, with the arithmetic of one fa_sinkhorn iteration: u_i = mu_i /
 * sum_j K_ij v_j (log_u, n1), the next column scaling from the column sums
 * sum_i K_ij u_i (log_v_next, n2) and the L1 column-marginal error of the
 * plan (log_u, log_v) into *err (device double), with mu = 1/n1 and
 * nu = 1/n2.  The partial column sums may be grouped over fewer row groups
 * than fa_sinkhorn uses (the static array bounds them), so results agree
 * with fa_sinkhorn up to FP32 summation order, not bit for bit.
 * K: device, n1 x ld, FA_F32 or FA_BF16 (dtype), 16-byte aligned, padding
 * columns 0; log_v, log_u, log_v_next, err: device.
 * status (device int32, nullable) receives the kernels' status bits
 * (1: NaN/Inf or an all-zero row or column, 2: a bounded wait gave up);
 * the call itself returns before the kernels run, so it cannot report
 * them.  With status == NULL the bits go to a static word nobody reads:
 * they are lost, and a NaN or a timed-out wait goes unnoticed -- pass a
 * status word to learn of them.
 * The launch shape is planned on the first call for each (device, n1, ld,
 * dtype) and reused by later calls (the FA_SWEEP_* tuning variables are
 * read at that first call only).
 *
 * Scratch: file-scope static device arrays reserved when the library is
 * loaded (8 MiB of partial column sums plus small counters) and held by
 * every GPU that loads the library until the process exits.  Limit: ld <=
 * 65536 columns (FA_ERR_UNSUPPORTED beyond); ld must be a multiple of 128.
 * The first call on a device looks the arrays' device addresses up
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Every call shares the same scratch: calls that can overlap on the GPU
 * (other streams, other host threads) race and must be serialised by the
 * caller.  Asynchronous on `stream`.
 * -------------------------------------------------------------------- */
fa_status fa_sinkhorn_step_static(const void* K, int32_t dtype, int32_t n1,
                                  int32_t n2, int64_t ld, const float* log_v,
                                  float* log_u, float* log_v_next, double* err,
                                  int32_t* status, fa_stream_t stream);

/* ----------------------------------------------------------------------
 * Column-sharded Sinkhorn iteration (Algorithm 1, Phase 3; Eq. 3) -- the
 * data path of a sweep whose columns of K are split over devices, each
 * owning a column range [j0, j1).  One iteration is three calls instead of
 * the fused pass of fa_sinkhorn:
 *
 *   fa_sinkhorn_shard_rows     partial row sums sum_{j in block b} K_ij v_j
 *                              for every column block b of the range
 *   fa_sinkhorn_shard_combine  u_i = mu_i / sum_b (partials), all blocks of
 *                              all ranges added in block order (with
 *                              several devices the blocks are gathered
 *                              first: n1 floats per block)
 *   fa_sinkhorn_shard_cols     column sums sum_i K_ij u_i of the range and
 *                              the next column scaling v_j = nu_j / (.)
 *
 * Column blocks are FA_SHARD_BLOCK columns wide and fixed by ld alone, and
 * every sum runs in a fixed order, so any split into ranges whose bounds
 * are multiples of FA_SHARD_BLOCK (or ld) gives bit-identical results.
 * A range's columns of K are read twice per iteration.
 *
 * j0 must be a multiple of FA_SHARD_BLOCK, j1 a multiple of it or ld,
 * 0 <= j0 < j1 <= ld (FA_ERR_ARG otherwise).  row_partials: device float,
 * fa_shard_blocks(ld) x n1 (block-major); shard_rows writes the range's
 * blocks, shard_combine reads all of them.  log_v: device n2 (the current
 * column scaling); log_u: device n1.  shard_cols reads log_u, writes
 * log_v_next[j] for j in [j0, min(j1, n2)) and, when err is not NULL, the
 * L1 error sum_{j in range} |v_j (sum_i K_ij u_i) - nu_j| of the plan
 * (log_u, log_v) into *err (device double).  FA_ERR_NUMERIC bits (an
 * all-zero row) stay in the context's status and are reported by the next
 * fa_sinkhorn.  Asynchronous on `stream`.
 * -------------------------------------------------------------------- */
#define FA_SHARD_BLOCK 2048
int64_t fa_shard_blocks(int64_t ld);
fa_status fa_sinkhorn_shard_rows(fa_ctx* ctx, const void* K, const float* log_v, int64_t j0,
                                 int64_t j1, float* row_partials, fa_stream_t stream);
fa_status fa_sinkhorn_shard_combine(fa_ctx* ctx, const float* row_partials, float* log_u,
                                    fa_stream_t stream);
fa_status fa_sinkhorn_shard_cols(fa_ctx* ctx, const void* K, const float* log_u,
                                 const float* log_v, int64_t j0, int64_t j1,
                                 float* log_v_next, double* err, fa_stream_t stream);

/* ----------------------------------------------------------------------
 * fa_sweep_plan -- the launch shape fa_sinkhorn would use for the fused
 * sweep (Algorithm 1, Phase 3) on n1 rows of ld columns (ld a positive multiple
 * of 128) in storage type dtype, from host logic only (no device query;
 * the FA_SWEEP_* tuning variables apply).  out (host int32[8]) receives:
 * cluster size Q, the widest slab W (elements; the row's 16-byte units are
 * split over the Q CTAs as evenly as possible, so slabs differ by at most
 * one unit), 16-byte vectors per thread per row S, rows per step R, ring
 * stages NS, threads per CTA NT, kind (0 CTA-synchronous, 1 warp-
 * specialised, 2 tensor-core row pass), and the cluster count G before the
 * device's occupancy limit is applied.
 * FA_ERR_UNSUPPORTED when no shape fits a row that wide.
 * -------------------------------------------------------------------- */
fa_status fa_sweep_plan(int32_t n1, int64_t ld, int32_t dtype, int32_t* out);

/* ----------------------------------------------------------------------
 * fa_ctx_selftest_wait -- failure-detection self-test (no counterpart in
 * the paper).  Launches one kernel whose bounded wait, the one every
 * mbarrier wait of the sweep uses, waits on a phase that nothing completes;
 * it gives up after its limit (about 2 s), records the timeout bit in the
 * context's status and returns normally.  Nothing is faulted.  The next
 * fa_sinkhorn on the context then returns FA_ERR_TIMEOUT and clears the
 * bit.  Asynchronous on `stream`.
 * -------------------------------------------------------------------- */
fa_status fa_ctx_selftest_wait(fa_ctx* ctx, fa_stream_t stream);

/* Per-thread description of the last error. */
const char* fa_last_error_string(void);

/* Number of kernels this library launched since load (all entry points). */
int64_t fa_kernel_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* FASTALIGN_H */
