// Internal declarations shared by the translation units of libfastalign.
// Nothing here is part of the C ABI (include/fastalign.h is).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <atomic>
#include <vector>

#include "fastalign.h"

namespace fa {

// ------------------------------------------------------------ errors
void set_error(const char* fmt, ...);
extern std::atomic<int64_t> g_launches;

#define FA_CUDA(call)                                                        \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      fa::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),  \
                    __FILE__, __LINE__);                                     \
      return FA_ERR_CUDA;                                                    \
    }                                                                        \
  } while (0)

// After every kernel launch: count it and surface launch errors.
#define FA_LAUNCHED(name)                                                    \
  do {                                                                       \
    fa::g_launches.fetch_add(1, std::memory_order_relaxed);                  \
    cudaError_t e_ = cudaGetLastError();                                     \
    if (e_ != cudaSuccess) {                                                 \
      fa::set_error("launch of %s failed: %s", name, cudaGetErrorString(e_)); \
      return FA_ERR_CUDA;                                                    \
    }                                                                        \
  } while (0)

#define FA_TRY(expr)                 \
  do {                               \
    fa_status s_ = (expr);           \
    if (s_ != FA_OK) return s_;      \
  } while (0)

// status word bits written by kernels
enum : int { ST_NUMERIC = 1, ST_TIMEOUT = 2 };

// ------------------------------------------------------------ sizes
// Leading-dimension padding (elements): a multiple of 128 keeps every column
// slab of a 16-CTA cluster a multiple of 16 bytes (TMA bulk copies).
constexpr int64_t kLdAlign = 128;
inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// ------------------------------------------------------------ device graph
struct DevGraph {
  int32_t n = 0;
  int64_t nnz = 0;
  int32_t* row_ptr = nullptr;   // n+1
  int32_t* col = nullptr;       // nnz, sorted per row
  float* val_row = nullptr;     // Abar[i,k]   = 1/deg(i)
  float* val_col = nullptr;     // Abar^T[i,k] = 1/deg(k)
  int32_t max_deg = 0;
};

// ------------------------------------------------------------ kernel launchers
// (each returns FA_OK or FA_ERR_CUDA and counts its launches)

// Phase 1
fa_status launch_rwr_step(const DevGraph& g, int L, int64_t ldr, float beta,
                          const float* Rin, float* Rout, cudaStream_t s);
fa_status launch_add_onehot(int L, int64_t ldr, const int32_t* nodes,
                            float value, float* R, cudaStream_t s);
fa_status launch_onehot(int n, int L, int64_t ldr, const int32_t* nodes,
                        float* R, cudaStream_t s);
fa_status launch_sddmm(const DevGraph& g, int L, int64_t ldr, const float* R,
                       bool weight_by_col, float* out, cudaStream_t s);
fa_status launch_normalize_rows(int n, int d, const float* X, int64_t ldx,
                                bool normalize, float* Xh, cudaStream_t s);
fa_status launch_node_cost_simt(int n1, int n2, int L, int64_t ldr,
                                const float* R1, const float* R2, int d,
                                int64_t ldx, const float* X1h,
                                const float* X2h, float alpha, float* C,
                                int64_t ldc, cudaStream_t s);
// tcgen05 GEMM: operands converted into K-major bf16 / tf32 tiles first.
fa_status launch_node_cost_tc(int n1, int n2, int L, int64_t ldr,
                              const float* R1, const float* R2, int d,
                              int64_t ldx, const float* X1h, const float* X2h,
                              float alpha, bool bf16, float* C, int64_t ldc,
                              void* ws, size_t ws_bytes, int* status,
                              cudaStream_t s);
size_t node_cost_tc_workspace(int n1, int n2, int L, int d, bool bf16);
bool tc_gemm_available();

// Sparse x dense products (Section 3.3/3.4): left product stored transposed,
// right product with a fused epilogue.
struct CostEpi {
  const float* C_node;      // n1 x ldo
  const void* K_prev;       // n1 x ldo, dtype per bf16 flag
  const float* log_u;       // n1
  const float* log_v;       // n2
  const int32_t* anc_ptr;   // n1+1, anchors of row i: anc_col[anc_ptr[i]..]
  const int32_t* anc_col;
  float eps, eps_anc, lam_e, lam_n, lam_a, lam_p, delta;
  float* X;                 // out: log of the unnormalised new kernel, n1 x ldo
  float* rowmax_part;       // out: [n2/64 tiles][n1] partial row maxima
};
fa_status launch_spmm_left_T(const DevGraph& g1, int n2, int64_t ldd,
                             int64_t ldw, const float* va, const float* vb,
                             const float* scale, const void* D, bool d_bf16,
                             float* Wt, cudaStream_t s);
fa_status launch_spmm_right_prop(const DevGraph& g2, int n1, int64_t ldw,
                                 const float* qa, const float* Wt, float* C,
                                 int64_t ldc, cudaStream_t s);
fa_status launch_spmm_right_cost(const DevGraph& g2, int n1, int64_t ldw,
                                 int64_t ldo, const float* qa, const float* qb,
                                 const float* scale, const float* Wt,
                                 const CostEpi& ep, bool k_bf16,
                                 cudaStream_t s);
fa_status launch_rowmax_reduce(int n1, int ntiles, const float* part,
                               float* rowmax, int* status, cudaStream_t s);
fa_status launch_exp_vec(int n, const float* x, float* y, cudaStream_t s);
fa_status launch_fill(float* p, int64_t n, float v, cudaStream_t s);

// Sinkhorn (Phase 3)
fa_status launch_wait_selftest(int* status, cudaStream_t s);
fa_status launch_plan_init(int n1, int n2, int64_t ld, void* K, bool bf16,
                           float* log_u, float* log_v, cudaStream_t s);
fa_status launch_normalize_kernel(int n1, int n2, int64_t ld, const float* X,
                                  const float* rowmax, void* K, bool bf16,
                                  float* colpart, int G, cudaStream_t s);
struct SweepPlan {
  int Q = 1;         // cluster size (column slabs per row)
  int W = 0;         // slab width in elements (ld / Q)
  int S = 1;         // 16-byte vectors per thread per row
  int R = 1;         // rows per step
  int NS = 2;        // shared-memory ring stages
  int NT = 512;      // threads per CTA (256: two CTAs per SM)
  int G = 1;         // clusters (= rows of the partial column-sum buffer)
  int kind = 0;      // 0: CTA-synchronous sweep, 1: warp-specialised sweep,
                     // 2: tensor-core row pass (BF16 storage only)
  int L = 1;         // warp-specialised: steps the column pass lags the row pass
  int MB = 1;        // tensor-core sweep: CTAs per SM its shape is sized for
};
SweepPlan plan_sweep(int n1, int64_t ld, bool bf16, int max_G);
fa_status launch_sweep(const SweepPlan& sp, int n1, int n2, int64_t ld,
                       const void* K, bool bf16, const float* log_v,
                       float* log_u, float mu, float* colpart, int* status,
                       cudaStream_t s);
int sweep_max_active_clusters(const SweepPlan& sp, bool bf16);
fa_status launch_col_finalize(int n2, int64_t ld, int G, const float* colpart,
                              const float* log_v_cur, float nu,
                              float* log_v_next, double* err_part,
                              unsigned* ticket, double* err_out, int* status,
                              cudaStream_t s);

// Column-sharded sweep (k_shard.cu)
constexpr int kShardBlock = FA_SHARD_BLOCK;
fa_status launch_shard_rows(int n1, int n2, int64_t ld, int64_t j0, int64_t j1, const void* K,
                            bool bf16, const float* v, float* rowpart, cudaStream_t s);
fa_status launch_shard_combine(int n1, int nblocks, const float* rowpart, float mu, float* u,
                               float* log_u, int* status, cudaStream_t s);
int shard_col_groups(int n1);
fa_status launch_shard_cols(int n1, int64_t ld, int64_t j0, int64_t j1, const void* K, bool bf16,
                            const float* u, float* colpart, cudaStream_t s);

// Read-out
fa_status launch_topk(int n1, int n2, int64_t ld, const void* K, bool bf16,
                      const float* log_v, int k, int32_t* idx, float* score,
                      cudaStream_t s);
constexpr int kPlanDiffBlocks = 1024;
fa_status launch_plan_l1diff(int n1, int n2, int64_t ld, bool bf16, const void* Ka,
                             const float* lua, const float* lva, const void* Kb,
                             const float* lub, const float* lvb, double* part, int nblocks,
                             double* out, cudaStream_t s);
fa_status launch_rank(int n2, int64_t ld, const void* K, bool bf16,
                      const float* log_v, int nq, const int32_t* rows,
                      const int32_t* cols, int32_t* rank, cudaStream_t s);

}  // namespace fa

// ------------------------------------------------------------ handles
struct fa_graph {
  fa::DevGraph d;
};

struct fa_ctx {
  const fa_graph* g1 = nullptr;
  const fa_graph* g2 = nullptr;
  fa_params p{};
  int32_t n1 = 0, n2 = 0;
  int64_t ld = 0;       // padded n2 (leading dimension of n1 x n2 matrices)
  int64_t ld1 = 0;      // padded n1 (leading dimension of the transposed buffer)
  int device = 0;
  // workspaces (owned)
  float* Wt = nullptr;            // n2 x ld1 x 2 floats
  float* X = nullptr;             // n1 x ld floats
  float* rowmax_part = nullptr;   // (ld/64) x n1
  float* rowmax = nullptr;        // n1
  float* colpart = nullptr;       // maxG x ld
  int maxG = 0;
  float* u_scale = nullptr;       // n1
  float* v_scale = nullptr;       // n2
  float* logv_buf[2] = {nullptr, nullptr};   // n2 each
  float* intra1 = nullptr;        // nnz1: C1 values
  float* intra2 = nullptr;        // nnz2: C2 values
  int32_t* anc_ptr = nullptr;     // n1+1
  int32_t* anc_col = nullptr;     // n_anchor (>= 1 slot)
  int32_t n_anchor = 0;
  double* err_part = nullptr;     // per finalize block
  unsigned* ticket = nullptr;
  double* err = nullptr;          // device scalar
  double* diff = nullptr;         // plan-change block sums + result
  int* status = nullptr;          // device status word
  int64_t ws_bytes = 0;
  // timing
  int G_sweep = 1;                // co-resident clusters of the sweep
  int anc_cap = 1;                // capacity of anc_col
  double host_err = 0.0;
  int host_status = 0;
  // timing
  int timing = 0;
  double last_sweep_ms = 0.0;
  int last_sweep_n = 0;
  std::vector<cudaEvent_t> sweep_events;
};
