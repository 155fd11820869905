// Host side of the C ABI (include/fastalign.h): argument checking, handle
// and workspace management, and the order of kernel launches for each entry
// point.  All arithmetic of the method runs in the kernels.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "fa_internal.cuh"

namespace fa {

std::atomic<int64_t> g_launches{0};
static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}

template <typename T>
static fa_status dalloc(T** p, size_t count, int64_t* acc = nullptr) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc of %zu bytes failed: %s", count * sizeof(T),
              cudaGetErrorString(e));
    return FA_ERR_OOM;
  }
  if (acc) *acc += (int64_t)(count * sizeof(T));
  return FA_OK;
}

static void dfree(void* p) {
  if (p) cudaFree(p);
}

static bool is_bf16(const fa_ctx* c) { return c->p.dtype == FA_BF16; }

// rows of the partial column-sum buffer used by the normalise pass
static int normalize_groups(int n1) { return std::min(n1, 128); }

}  // namespace fa

using namespace fa;

extern "C" {

const char* fa_last_error_string(void) { return fa::g_err; }
int64_t fa_kernel_launch_count(void) { return fa::g_launches.load(); }

void fa_params_default(fa_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->dtype = FA_F32;
  p->eps = 0.05f;
  p->eps_anc = 0.05f;
  p->alpha = 0.5f;
  p->beta = 0.15f;
  p->k_rwr = 10;
  p->k_prop = 1;
  p->lam_e = 1.0f;
  p->lam_n = 0.05f;
  p->lam_a = 0.05f;
  p->lam_p = 0.05f;
  p->delta = 1e-30f;
  p->normalize_features = 1;
  p->gemm_mode = FA_GEMM_AUTO;
}

// ------------------------------------------------------------ graphs
}  // extern "C"

namespace fa {

// Host half of fa_build_graph (Algorithm 1, row normalisation): CSR of the symmetric adjacency
// with columns ascending, values 1/deg_i (Abar) and 1/deg_k (Abar^T).
struct HostCSR {
  std::vector<int32_t> rp, col;
  std::vector<float> vr, vc;
  int32_t max_deg = 0;
  int64_t nnz = 0;
};

static fa_status csr_from_edges(const char* who, int32_t n, int64_t n_edges,
                                const int32_t* src, const int32_t* dst, HostCSR& h) {
  if (n < 1) { set_error("%s: n=%d < 1", who, n); return FA_ERR_ARG; }
  if (n_edges < 0 || (n_edges > 0 && (!src || !dst))) {
    set_error("%s: bad edge arrays", who);
    return FA_ERR_ARG;
  }
  std::vector<int64_t> keys;
  keys.reserve((size_t)n_edges);
  for (int64_t e = 0; e < n_edges; ++e) {
    const int32_t a = src[e], b = dst[e];
    if (a < 0 || a >= n || b < 0 || b >= n) {
      set_error("%s: edge %lld = (%d, %d) outside [0, %d)", who, (long long)e, a, b, n);
      return FA_ERR_ARG;
    }
    if (a == b) continue;
    const int64_t u = std::min(a, b), v = std::max(a, b);
    keys.push_back(u * (int64_t)n + v);
  }
  std::sort(keys.begin(), keys.end());
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  std::vector<int32_t> deg(n, 0);
  for (int64_t k : keys) {
    deg[k / n]++;
    deg[k % n]++;
  }
  const int64_t nnz = 2 * (int64_t)keys.size();
  if (nnz > INT32_MAX) { set_error("%s: too many edges", who); return FA_ERR_UNSUPPORTED; }
  h.nnz = nnz;
  h.rp.assign(n + 1, 0);
  h.col.resize(nnz);
  std::vector<int32_t> pos(n);
  for (int i = 0; i < n; ++i) h.rp[i + 1] = h.rp[i] + deg[i];
  for (int i = 0; i < n; ++i) pos[i] = h.rp[i];
  // keys are sorted by (u, v): every row receives its smaller neighbours
  // (as v) before its larger ones (as u), each group ascending.
  for (int64_t k : keys) {
    const int32_t u = (int32_t)(k / n), v = (int32_t)(k % n);
    h.col[pos[u]++] = v;
    h.col[pos[v]++] = u;
  }
  h.vr.resize(nnz);
  h.vc.resize(nnz);
  h.max_deg = 0;
  for (int i = 0; i < n; ++i) {
    h.max_deg = std::max(h.max_deg, deg[i]);
    for (int32_t e = h.rp[i]; e < h.rp[i + 1]; ++e) {
      h.vr[e] = 1.0f / (float)deg[i];
      h.vc[e] = 1.0f / (float)deg[h.col[e]];
    }
  }
  return FA_OK;
}

}  // namespace fa

extern "C" {

fa_status fa_build_graph(int32_t n, int64_t n_edges, const int32_t* src,
                         const int32_t* dst, fa_graph** out) {
  if (!out) { set_error("fa_build_graph: out is NULL"); return FA_ERR_ARG; }
  *out = nullptr;
  HostCSR h;
  FA_TRY(csr_from_edges("fa_build_graph", n, n_edges, src, dst, h));
  const int64_t nnz = h.nnz;
  fa_graph* g = new fa_graph();
  g->d.n = n;
  g->d.nnz = nnz;
  g->d.max_deg = h.max_deg;
  fa_status st;
  if ((st = dalloc(&g->d.row_ptr, n + 1)) != FA_OK ||
      (st = dalloc(&g->d.col, nnz)) != FA_OK ||
      (st = dalloc(&g->d.val_row, nnz)) != FA_OK ||
      (st = dalloc(&g->d.val_col, nnz)) != FA_OK) {
    fa_graph_destroy(g);
    return st;
  }
  cudaError_t e1 = cudaMemcpy(g->d.row_ptr, h.rp.data(), (n + 1) * sizeof(int32_t), cudaMemcpyHostToDevice);
  cudaError_t e2 = nnz ? cudaMemcpy(g->d.col, h.col.data(), nnz * sizeof(int32_t), cudaMemcpyHostToDevice) : cudaSuccess;
  cudaError_t e3 = nnz ? cudaMemcpy(g->d.val_row, h.vr.data(), nnz * sizeof(float), cudaMemcpyHostToDevice) : cudaSuccess;
  cudaError_t e4 = nnz ? cudaMemcpy(g->d.val_col, h.vc.data(), nnz * sizeof(float), cudaMemcpyHostToDevice) : cudaSuccess;
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || e4 != cudaSuccess) {
    set_error("fa_build_graph: upload failed: %s",
              cudaGetErrorString(e1 != cudaSuccess ? e1 : e2 != cudaSuccess ? e2 : e3 != cudaSuccess ? e3 : e4));
    fa_graph_destroy(g);
    return FA_ERR_CUDA;
  }
  *out = g;
  return FA_OK;
}

fa_status fa_graph_csr_host(int32_t n, int64_t n_edges, const int32_t* src,
                            const int32_t* dst, int64_t* nnz_out, int32_t* row_ptr,
                            int32_t* col, float* val_row, float* val_col, int64_t cap) {
  if (!nnz_out) { set_error("fa_graph_csr_host: nnz_out is NULL"); return FA_ERR_ARG; }
  HostCSR h;
  FA_TRY(csr_from_edges("fa_graph_csr_host", n, n_edges, src, dst, h));
  *nnz_out = h.nnz;
  if (!row_ptr && !col && !val_row && !val_col) return FA_OK;   // size query
  if (!row_ptr || !col || !val_row || !val_col || cap < h.nnz) {
    set_error("fa_graph_csr_host: need four arrays with room for %lld entries",
              (long long)h.nnz);
    return FA_ERR_ARG;
  }
  std::copy(h.rp.begin(), h.rp.end(), row_ptr);
  std::copy(h.col.begin(), h.col.end(), col);
  std::copy(h.vr.begin(), h.vr.end(), val_row);
  std::copy(h.vc.begin(), h.vc.end(), val_col);
  return FA_OK;
}

fa_status fa_graph_destroy(fa_graph* g) {
  if (!g) return FA_OK;
  dfree(g->d.row_ptr);
  dfree(g->d.col);
  dfree(g->d.val_row);
  dfree(g->d.val_col);
  delete g;
  return FA_OK;
}

fa_status fa_graph_info(const fa_graph* g, int32_t* n, int64_t* nnz) {
  if (!g) { set_error("fa_graph_info: NULL graph"); return FA_ERR_ARG; }
  if (n) *n = g->d.n;
  if (nnz) *nnz = g->d.nnz;
  return FA_OK;
}

// ------------------------------------------------------------ context
fa_status fa_ctx_destroy(fa_ctx* c) {
  if (!c) return FA_OK;
  dfree(c->Wt); dfree(c->X); dfree(c->rowmax_part); dfree(c->rowmax);
  dfree(c->colpart); dfree(c->u_scale); dfree(c->v_scale);
  dfree(c->logv_buf[0]); dfree(c->logv_buf[1]);
  dfree(c->intra1); dfree(c->intra2); dfree(c->anc_ptr); dfree(c->anc_col);
  dfree(c->err_part); dfree(c->ticket); dfree(c->err); dfree(c->status);
  dfree(c->diff);
  for (auto& ev : c->sweep_events) cudaEventDestroy(ev);
  delete c;
  return FA_OK;
}

static fa_status check_params(const fa_params* p) {
  if (!p) { set_error("params is NULL"); return FA_ERR_ARG; }
  if (p->dtype != FA_F32 && p->dtype != FA_BF16) { set_error("bad dtype %d", p->dtype); return FA_ERR_ARG; }
  if (!(p->eps > 0.f) || !(p->eps_anc > 0.f) || !(p->delta > 0.f)) {
    set_error("eps, eps_anc and delta must be > 0");
    return FA_ERR_ARG;
  }
  if (p->k_rwr < 0 || p->k_prop < 0) { set_error("k_rwr, k_prop must be >= 0"); return FA_ERR_ARG; }
  if (p->lam_p < 0.f) { set_error("lam_p must be >= 0"); return FA_ERR_ARG; }
  if (p->gemm_mode < 0 || p->gemm_mode > 2) { set_error("bad gemm_mode %d", p->gemm_mode); return FA_ERR_ARG; }
  return FA_OK;
}

fa_status fa_ctx_create(const fa_graph* g1, const fa_graph* g2,
                        const fa_params* params, fa_ctx** out) {
  if (!out) { set_error("fa_ctx_create: out is NULL"); return FA_ERR_ARG; }
  *out = nullptr;
  if (!g1 || !g2) { set_error("fa_ctx_create: NULL graph"); return FA_ERR_ARG; }
  FA_TRY(check_params(params));
  fa_ctx* c = new fa_ctx();
  c->g1 = g1;
  c->g2 = g2;
  c->p = *params;
  c->n1 = g1->d.n;
  c->n2 = g2->d.n;
  c->ld = round_up(c->n2, kLdAlign);
  c->ld1 = round_up(c->n1, kLdAlign);
  cudaGetDevice(&c->device);
  const bool bf16 = is_bf16(c);
  // sweep shape and the number of co-resident clusters
  SweepPlan sp = plan_sweep(c->n1, c->ld, bf16, 1 << 20);
  int maxact = sp.Q >= 1 ? sweep_max_active_clusters(sp, bf16) : 0;
  c->G_sweep = std::max(1, maxact);
  c->maxG = std::max(c->G_sweep, normalize_groups(c->n1));
  const int64_t n1 = c->n1, n2 = c->n2, ld = c->ld, ld1 = c->ld1;
  fa_status st;
  int64_t* acc = &c->ws_bytes;
  if ((st = dalloc(&c->Wt, (size_t)(n2 * ld1 * 2), acc)) != FA_OK ||
      (st = dalloc(&c->X, (size_t)(n1 * ld), acc)) != FA_OK ||
      (st = dalloc(&c->rowmax_part, (size_t)((ld / 64) * n1), acc)) != FA_OK ||
      (st = dalloc(&c->rowmax, (size_t)n1, acc)) != FA_OK ||
      (st = dalloc(&c->colpart, (size_t)(c->maxG * ld), acc)) != FA_OK ||
      (st = dalloc(&c->u_scale, (size_t)n1, acc)) != FA_OK ||
      (st = dalloc(&c->v_scale, (size_t)n2, acc)) != FA_OK ||
      (st = dalloc(&c->logv_buf[0], (size_t)n2, acc)) != FA_OK ||
      (st = dalloc(&c->logv_buf[1], (size_t)n2, acc)) != FA_OK ||
      (st = dalloc(&c->intra1, (size_t)g1->d.nnz, acc)) != FA_OK ||
      (st = dalloc(&c->intra2, (size_t)g2->d.nnz, acc)) != FA_OK ||
      (st = dalloc(&c->anc_ptr, (size_t)(n1 + 1), acc)) != FA_OK ||
      (st = dalloc(&c->anc_col, 1, acc)) != FA_OK ||
      (st = dalloc(&c->err_part, (size_t)((n2 + 255) / 256), acc)) != FA_OK ||
      (st = dalloc(&c->ticket, 1, acc)) != FA_OK ||
      (st = dalloc(&c->err, 1, acc)) != FA_OK ||
      (st = dalloc(&c->diff, (size_t)kPlanDiffBlocks + 1, acc)) != FA_OK ||
      (st = dalloc(&c->status, 1, acc)) != FA_OK) {
    fa_ctx_destroy(c);
    return st;
  }
  if (cudaMemset(c->ticket, 0, sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(c->status, 0, sizeof(int)) != cudaSuccess ||
      cudaMemset(c->anc_ptr, 0, (n1 + 1) * sizeof(int32_t)) != cudaSuccess ||
      cudaMemset(c->intra1, 0, std::max<int64_t>(1, g1->d.nnz) * sizeof(float)) != cudaSuccess ||
      cudaMemset(c->intra2, 0, std::max<int64_t>(1, g2->d.nnz) * sizeof(float)) != cudaSuccess) {
    set_error("fa_ctx_create: memset failed");
    fa_ctx_destroy(c);
    return FA_ERR_CUDA;
  }
  *out = c;
  return FA_OK;
}

int64_t fa_ctx_ld(const fa_ctx* c) { return c ? c->ld : -1; }
int64_t fa_ctx_workspace_bytes(const fa_ctx* c) { return c ? c->ws_bytes : -1; }

fa_status fa_ctx_set_timing(fa_ctx* c, int32_t on) {
  if (!c) { set_error("NULL ctx"); return FA_ERR_ARG; }
  c->timing = on ? 1 : 0;
  return FA_OK;
}

fa_status fa_ctx_last_sweep_ms(const fa_ctx* c, double* ms, int32_t* n) {
  if (!c) { set_error("NULL ctx"); return FA_ERR_ARG; }
  if (ms) *ms = c->last_sweep_ms;
  if (n) *n = c->last_sweep_n;
  return FA_OK;
}

// ------------------------------------------------------------ Phase 1
fa_status fa_node_cost(fa_ctx* c, const float* X1, const float* X2, int32_t d,
                       const int32_t* anchors, int32_t n_anchor, float* C_node,
                       fa_stream_t stream) {
  if (!c || !C_node) { set_error("fa_node_cost: NULL ctx or C_node"); return FA_ERR_ARG; }
  if (d < 0 || (d > 0 && (!X1 || !X2))) { set_error("fa_node_cost: bad attributes"); return FA_ERR_ARG; }
  if (n_anchor < 0 || (n_anchor > 0 && !anchors)) { set_error("fa_node_cost: bad anchors"); return FA_ERR_ARG; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int n1 = c->n1, n2 = c->n2;
  const int L = n_anchor;
  // anchors: host checks, per-graph node lists and the row-sorted list
  std::vector<int32_t> a1(std::max(L, 1)), a2(std::max(L, 1));
  std::vector<std::pair<int32_t, int32_t>> byrow(L);
  for (int l = 0; l < L; ++l) {
    const int32_t i = anchors[2 * l], j = anchors[2 * l + 1];
    if (i < 0 || i >= n1 || j < 0 || j >= n2) {
      set_error("fa_node_cost: anchor %d = (%d, %d) out of range", l, i, j);
      return FA_ERR_ARG;
    }
    a1[l] = i;
    a2[l] = j;
    byrow[l] = {i, j};
  }
  std::sort(byrow.begin(), byrow.end());
  std::vector<int32_t> aptr(n1 + 1, 0), acol(std::max(L, 1));
  for (int l = 0; l < L; ++l) { aptr[byrow[l].first + 1]++; acol[l] = byrow[l].second; }
  for (int i = 0; i < n1; ++i) aptr[i + 1] += aptr[i];
  if (L + 1 > c->anc_cap) {
    dfree(c->anc_col);
    c->anc_col = nullptr;
    FA_TRY(dalloc(&c->anc_col, (size_t)(L + 1)));
    c->anc_cap = L + 1;
  }
  FA_CUDA(cudaMemcpyAsync(c->anc_ptr, aptr.data(), (n1 + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  FA_CUDA(cudaMemcpyAsync(c->anc_col, acol.data(), std::max(L, 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  c->n_anchor = L;

  const int64_t ldr = round_up(std::max(L, 1), 64);
  const int64_t ldx = round_up(std::max(d, 1), 64);
  float *R1a = nullptr, *R1b = nullptr, *R2a = nullptr, *R2b = nullptr;
  float *X1h = nullptr, *X2h = nullptr;
  int32_t *da1 = nullptr, *da2 = nullptr;
  auto freeall = [&]() {
    if (R1a) cudaFreeAsync(R1a, s);
    if (R1b) cudaFreeAsync(R1b, s);
    if (R2a) cudaFreeAsync(R2a, s);
    if (R2b) cudaFreeAsync(R2b, s);
    if (X1h) cudaFreeAsync(X1h, s);
    if (X2h) cudaFreeAsync(X2h, s);
    if (da1) cudaFreeAsync(da1, s);
    if (da2) cudaFreeAsync(da2, s);
  };
  auto amalloc = [&](void** p, size_t bytes) -> fa_status {
    cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("fa_node_cost: cudaMallocAsync(%zu) failed: %s", bytes, cudaGetErrorString(e));
      return FA_ERR_OOM;
    }
    return FA_OK;
  };
  fa_status st = FA_OK;
#define FA_STEP(expr) do { st = (expr); if (st != FA_OK) { freeall(); return st; } } while (0)
  FA_STEP(amalloc((void**)&R1a, (size_t)n1 * ldr * 4));
  FA_STEP(amalloc((void**)&R1b, (size_t)n1 * ldr * 4));
  FA_STEP(amalloc((void**)&R2a, (size_t)n2 * ldr * 4));
  FA_STEP(amalloc((void**)&R2b, (size_t)n2 * ldr * 4));
  FA_STEP(amalloc((void**)&X1h, (size_t)n1 * ldx * 4));
  FA_STEP(amalloc((void**)&X2h, (size_t)n2 * ldx * 4));
  FA_STEP(amalloc((void**)&da1, (size_t)std::max(L, 1) * 4));
  FA_STEP(amalloc((void**)&da2, (size_t)std::max(L, 1) * 4));
  if (cudaMemcpyAsync(da1, a1.data(), std::max(L, 1) * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(da2, a2.data(), std::max(L, 1) * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) {
    set_error("fa_node_cost: anchor upload failed");
    freeall();
    return FA_ERR_CUDA;
  }
  // Algorithm 1, RWR: R <- (1-beta) Abar R + beta R^(0), k_rwr times
  const float beta = c->p.beta;
  FA_STEP(launch_onehot(n1, L, ldr, da1, R1a, s));
  FA_STEP(launch_onehot(n2, L, ldr, da2, R2a, s));
  for (int t = 0; t < c->p.k_rwr; ++t) {
    FA_STEP(launch_rwr_step(c->g1->d, L, ldr, beta, R1a, R1b, s));
    FA_STEP(launch_add_onehot(L, ldr, da1, beta, R1b, s));
    std::swap(R1a, R1b);
    FA_STEP(launch_rwr_step(c->g2->d, L, ldr, beta, R2a, R2b, s));
    FA_STEP(launch_add_onehot(L, ldr, da2, beta, R2b, s));
    std::swap(R2a, R2b);
  }
  // Algorithm 1, intra-graph costs: SDDMM for C1 (1/deg i) and C2 (1/deg l)
  FA_STEP(launch_sddmm(c->g1->d, L, ldr, R1a, false, c->intra1, s));
  FA_STEP(launch_sddmm(c->g2->d, L, ldr, R2a, true, c->intra2, s));
  // attributes
  if (d > 0) {
    FA_STEP(launch_normalize_rows(n1, d, X1, ldx, c->p.normalize_features != 0, X1h, s));
    FA_STEP(launch_normalize_rows(n2, d, X2, ldx, c->p.normalize_features != 0, X2h, s));
  } else {
    FA_STEP(launch_fill(X1h, (int64_t)n1 * ldx, 0.f, s));
    FA_STEP(launch_fill(X2h, (int64_t)n2 * ldx, 0.f, s));
  }
  // Algorithm 1, node cost: the node-similarity GEMMs with the exp epilogue
  const bool use_tc = c->p.gemm_mode != FA_GEMM_SIMT && tc_gemm_available();
  if (use_tc) {
    const bool bf16 = is_bf16(c);
    size_t wsb = node_cost_tc_workspace(n1, n2, L, d, bf16);
    void* ws = nullptr;
    FA_STEP(amalloc(&ws, wsb));
    st = launch_node_cost_tc(n1, n2, L, ldr, R1a, R2a, d, ldx, X1h, X2h,
                             c->p.alpha, bf16, C_node, c->ld, ws, wsb, c->status, s);
    cudaFreeAsync(ws, s);
    if (st != FA_OK) { freeall(); return st; }
  } else {
    FA_STEP(launch_node_cost_simt(n1, n2, L, ldr, R1a, R2a, d, ldx, X1h, X2h,
                                  c->p.alpha, C_node, c->ld, s));
  }
  // Algorithm 1, propagation (reading: A1bar C A2bar^T), k_prop times, as two SpMMs
  for (int t = 0; t < c->p.k_prop; ++t) {
    FA_STEP(launch_spmm_left_T(c->g1->d, n2, c->ld, c->ld1, c->g1->d.val_row,
                               nullptr, nullptr, C_node, false, c->Wt, s));
    FA_STEP(launch_spmm_right_prop(c->g2->d, n1, c->ld1, c->g2->d.val_row,
                                   c->Wt, C_node, c->ld, s));
  }
#undef FA_STEP
  freeall();
  return FA_OK;
}

fa_status fa_plan_init(fa_ctx* c, void* K, float* log_u, float* log_v,
                       fa_stream_t stream) {
  if (!c || !K || !log_u || !log_v) { set_error("fa_plan_init: NULL argument"); return FA_ERR_ARG; }
  return launch_plan_init(c->n1, c->n2, c->ld, K, is_bf16(c), log_u, log_v,
                          reinterpret_cast<cudaStream_t>(stream));
}

// ------------------------------------------------------------ Phase 2
fa_status fa_align_iter(fa_ctx* c, void* K, float* log_u, float* log_v,
                        const float* C_node, fa_stream_t stream) {
  if (!c || !K || !log_u || !log_v || !C_node) { set_error("fa_align_iter: NULL argument"); return FA_ERR_ARG; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const bool bf16 = is_bf16(c);
  const int n1 = c->n1, n2 = c->n2;
  FA_TRY(launch_exp_vec(n1, log_u, c->u_scale, s));
  FA_TRY(launch_exp_vec(n2, log_v, c->v_scale, s));
  // W = P1 T_prev for P1 in {C1, A1bar^T}; T_prev = diag(u) K diag(v): u is
  // folded into P1's column scale here and v into P2's below.
  FA_TRY(launch_spmm_left_T(c->g1->d, n2, c->ld, c->ld1, c->intra1,
                            c->g1->d.val_col, c->u_scale, K, bf16, c->Wt, s));
  CostEpi ep;
  ep.C_node = C_node;
  ep.K_prev = K;
  ep.log_u = log_u;
  ep.log_v = log_v;
  ep.anc_ptr = c->anc_ptr;
  ep.anc_col = c->anc_col;
  ep.eps = c->p.eps;
  ep.eps_anc = c->p.eps_anc;
  ep.lam_e = c->p.lam_e;
  ep.lam_n = c->p.lam_n;
  ep.lam_a = c->p.lam_a;
  ep.lam_p = c->p.lam_p;
  ep.delta = c->p.delta;
  ep.X = c->X;
  ep.rowmax_part = c->rowmax_part;
  // Z = W P2^T for P2 in {C2, A2bar^T}, cost assembly and log Gibbs kernel
  FA_TRY(launch_spmm_right_cost(c->g2->d, n1, c->ld1, c->ld, c->intra2,
                                c->g2->d.val_col, c->v_scale, c->Wt, ep, bf16, s));
  FA_TRY(launch_rowmax_reduce(n1, (int)(c->ld / 64), c->rowmax_part, c->rowmax, c->status, s));
  // row-stabilised kernel and the first column update a_1 (u = 1)
  const int Gn = normalize_groups(n1);
  FA_TRY(launch_normalize_kernel(n1, n2, c->ld, c->X, c->rowmax, K, bf16, c->colpart, Gn, s));
  FA_TRY(launch_col_finalize(n2, c->ld, Gn, c->colpart, nullptr, 1.0f / (float)n2,
                             log_v, c->err_part, c->ticket, c->err, c->status, s));
  FA_TRY(launch_fill(log_u, n1, 0.f, s));
  return FA_OK;
}

// ------------------------------------------------------------ Phase 3
fa_status fa_sinkhorn(fa_ctx* c, const void* K, float* log_u, float* log_v,
                      const float* warm_log_v, int32_t max_iter, double tol,
                      int32_t check_every, int32_t* iters_out, double* err_out,
                      fa_stream_t stream) {
  if (!c || !K || !log_u || !log_v) { set_error("fa_sinkhorn: NULL argument"); return FA_ERR_ARG; }
  if (max_iter < 1) { set_error("fa_sinkhorn: max_iter=%d < 1", max_iter); return FA_ERR_ARG; }
  if (check_every < 1) check_every = 1;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const bool bf16 = is_bf16(c);
  const int n1 = c->n1, n2 = c->n2;
  SweepPlan sp = plan_sweep(n1, c->ld, bf16, c->G_sweep);
  if (warm_log_v)
    FA_CUDA(cudaMemcpyAsync(log_v, warm_log_v, n2 * sizeof(float), cudaMemcpyDeviceToDevice, s));
  // c->status is not cleared here: bits set by earlier asynchronous calls on
  // this context (a bounded wait in the node-cost GEMM, a non-finite row in
  // Pass B) are reported by this call, which clears them once read.
  const float mu = 1.0f / (float)n1, nu = 1.0f / (float)n2;
  float* bufs[3] = {log_v, c->logv_buf[0], c->logv_buf[1]};
  int cur = 0;
  double err = -1.0;
  int it = 0;
  bool converged = false;
  if (c->timing && (int)c->sweep_events.size() < 2 * max_iter) {
    while ((int)c->sweep_events.size() < 2 * max_iter) {
      cudaEvent_t ev;
      FA_CUDA(cudaEventCreate(&ev));
      c->sweep_events.push_back(ev);
    }
  }
  for (it = 1; it <= max_iter; ++it) {
    // the next column scaling never goes into the caller's buffer (index 0)
    const int next = (cur == 1) ? 2 : 1;
    if (c->timing) FA_CUDA(cudaEventRecord(c->sweep_events[2 * (it - 1)], s));
    FA_TRY(launch_sweep(sp, n1, n2, c->ld, K, bf16, bufs[cur], log_u, mu, c->colpart, c->status, s));
    if (c->timing) FA_CUDA(cudaEventRecord(c->sweep_events[2 * (it - 1) + 1], s));
    FA_TRY(launch_col_finalize(n2, c->ld, sp.G, c->colpart, bufs[cur], nu,
                               bufs[next], c->err_part, c->ticket, c->err, c->status, s));
    const bool check = tol >= 0.0 && (it % check_every == 0 || it == max_iter);
    if (check) {
      FA_CUDA(cudaMemcpyAsync(&c->host_err, c->err, sizeof(double), cudaMemcpyDeviceToHost, s));
      FA_CUDA(cudaStreamSynchronize(s));
      err = c->host_err;
      if (err <= tol) { converged = true; break; }
    }
    if (it == max_iter) break;   // state = (a_t in bufs[cur], b_t in log_u)
    cur = next;
  }
  if (it > max_iter) it = max_iter;
  if (cur != 0)
    FA_CUDA(cudaMemcpyAsync(log_v, bufs[cur], n2 * sizeof(float), cudaMemcpyDeviceToDevice, s));
  int host_status = 0;
  FA_CUDA(cudaMemcpyAsync(&c->host_err, c->err, sizeof(double), cudaMemcpyDeviceToHost, s));
  FA_CUDA(cudaMemcpyAsync(&c->host_status, c->status, sizeof(int), cudaMemcpyDeviceToHost, s));
  FA_CUDA(cudaStreamSynchronize(s));
  err = c->host_err;
  host_status = c->host_status;
  if (host_status != 0) FA_CUDA(cudaMemsetAsync(c->status, 0, sizeof(int), s));
  if (c->timing) {
    double tot = 0.0;
    for (int t = 0; t < it; ++t) {
      float ms = 0.f;
      FA_CUDA(cudaEventElapsedTime(&ms, c->sweep_events[2 * t], c->sweep_events[2 * t + 1]));
      tot += ms;
    }
    c->last_sweep_ms = tot / std::max(1, it);
    c->last_sweep_n = it;
  }
  if (iters_out) *iters_out = it;
  if (err_out) *err_out = err;
  if (host_status & ST_TIMEOUT) {
    set_error("fa_sinkhorn: a bounded device-side wait gave up (this call or an "
              "earlier asynchronous call on the context); results are not valid");
    return FA_ERR_TIMEOUT;
  }
  if (host_status & ST_NUMERIC) {
    set_error("fa_sinkhorn: NaN/Inf or an all-zero row or column");
    return FA_ERR_NUMERIC;
  }
  if (tol >= 0.0 && !converged) {
    set_error("fa_sinkhorn: err %.3e > tol %.3e after %d iterations", err, tol, it);
    return FA_ERR_NOT_CONVERGED;
  }
  return FA_OK;
}

// ------------------------------------------------------------ read-out
fa_status fa_topk(fa_ctx* c, const void* K, const float* log_v, int32_t k,
                  int32_t* idx, float* score, fa_stream_t stream) {
  if (!c || !K || !log_v || !idx) { set_error("fa_topk: NULL argument"); return FA_ERR_ARG; }
  if (k < 1 || k > 32) { set_error("fa_topk: k=%d outside [1, 32]", k); return FA_ERR_ARG; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  FA_TRY(launch_exp_vec(c->n2, log_v, c->v_scale, s));
  return launch_topk(c->n1, c->n2, c->ld, K, is_bf16(c), c->v_scale, k, idx, score, s);
}

fa_status fa_rank(fa_ctx* c, const void* K, const float* log_v, int32_t n_query,
                  const int32_t* rows, const int32_t* cols, int32_t* rank_out,
                  fa_stream_t stream) {
  if (!c || !K || !log_v || (n_query > 0 && (!rows || !cols || !rank_out))) {
    set_error("fa_rank: NULL argument");
    return FA_ERR_ARG;
  }
  if (n_query < 0) { set_error("fa_rank: n_query < 0"); return FA_ERR_ARG; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  FA_TRY(launch_exp_vec(c->n2, log_v, c->v_scale, s));
  return launch_rank(c->n2, c->ld, K, is_bf16(c), c->v_scale, n_query, rows, cols, rank_out, s);
}

// ------------------------------------------------------------ column-sharded sweep
int64_t fa_shard_blocks(int64_t ld) { return ld < 1 ? -1 : (ld + kShardBlock - 1) / kShardBlock; }

static fa_status check_range(const fa_ctx* c, int64_t j0, int64_t j1, const char* who) {
  if (j0 < 0 || j1 > c->ld || j0 >= j1 || j0 % kShardBlock != 0 ||
      (j1 != c->ld && j1 % kShardBlock != 0)) {
    set_error("%s: column range [%lld, %lld) must satisfy 0 <= j0 < j1 <= ld = %lld with j0 "
              "a multiple of %d and j1 a multiple of it or ld",
              who, (long long)j0, (long long)j1, (long long)c->ld, kShardBlock);
    return FA_ERR_ARG;
  }
  return FA_OK;
}

fa_status fa_sinkhorn_shard_rows(fa_ctx* c, const void* K, const float* log_v, int64_t j0,
                                 int64_t j1, float* row_partials, fa_stream_t stream) {
  if (!c || !K || !log_v || !row_partials) { set_error("fa_sinkhorn_shard_rows: NULL argument"); return FA_ERR_ARG; }
  FA_TRY(check_range(c, j0, j1, "fa_sinkhorn_shard_rows"));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  FA_TRY(launch_exp_vec(c->n2, log_v, c->v_scale, s));
  return launch_shard_rows(c->n1, c->n2, c->ld, j0, j1, K, is_bf16(c), c->v_scale, row_partials, s);
}

fa_status fa_sinkhorn_shard_combine(fa_ctx* c, const float* row_partials, float* log_u,
                                    fa_stream_t stream) {
  if (!c || !row_partials || !log_u) { set_error("fa_sinkhorn_shard_combine: NULL argument"); return FA_ERR_ARG; }
  return launch_shard_combine(c->n1, (int)fa_shard_blocks(c->ld), row_partials,
                              1.0f / (float)c->n1, c->u_scale, log_u, c->status,
                              reinterpret_cast<cudaStream_t>(stream));
}

fa_status fa_sinkhorn_shard_cols(fa_ctx* c, const void* K, const float* log_u, const float* log_v,
                                 int64_t j0, int64_t j1, float* log_v_next, double* err,
                                 fa_stream_t stream) {
  if (!c || !K || !log_u || !log_v || !log_v_next) { set_error("fa_sinkhorn_shard_cols: NULL argument"); return FA_ERR_ARG; }
  FA_TRY(check_range(c, j0, j1, "fa_sinkhorn_shard_cols"));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  FA_TRY(launch_exp_vec(c->n1, log_u, c->u_scale, s));
  FA_TRY(launch_shard_cols(c->n1, c->ld, j0, j1, K, is_bf16(c), c->u_scale, c->colpart, s));
  const int64_t jend = std::min<int64_t>(j1, c->n2);
  if (jend <= j0) return FA_OK;          // a range of padding columns only
  return launch_col_finalize((int)(jend - j0), c->ld, shard_col_groups(c->n1), c->colpart + j0,
                             log_v + j0, 1.0f / (float)c->n2, log_v_next + j0, c->err_part,
                             c->ticket, err ? err : c->err, c->status, s);
}

// ------------------------------------------------------------ sweep plan
fa_status fa_sweep_plan(int32_t n1, int64_t ld, int32_t dtype, int32_t* out) {
  if (!out) { set_error("fa_sweep_plan: out is NULL"); return FA_ERR_ARG; }
  if (n1 < 1 || ld < 128 || ld % 128 != 0) {
    set_error("fa_sweep_plan: n1=%d, ld=%lld (need n1 >= 1, ld a positive multiple of 128)",
              n1, (long long)ld);
    return FA_ERR_ARG;
  }
  if (dtype != FA_F32 && dtype != FA_BF16) { set_error("fa_sweep_plan: bad dtype %d", dtype); return FA_ERR_ARG; }
  const SweepPlan sp = plan_sweep(n1, ld, dtype == FA_BF16, 1 << 20);
  if (sp.Q < 1) {
    set_error("fa_sweep_plan: no cluster shape fits a row of %lld elements", (long long)ld);
    return FA_ERR_UNSUPPORTED;
  }
  const int32_t v[8] = {sp.Q, sp.W, sp.S, sp.R, sp.NS, sp.NT, sp.kind, sp.G};
  std::copy(v, v + 8, out);
  return FA_OK;
}

// ------------------------------------------------------------ self-test
fa_status fa_ctx_selftest_wait(fa_ctx* c, fa_stream_t stream) {
  if (!c) { set_error("fa_ctx_selftest_wait: NULL ctx"); return FA_ERR_ARG; }
  return launch_wait_selftest(c->status, reinterpret_cast<cudaStream_t>(stream));
}

// ------------------------------------------------------------ plan change
fa_status fa_plan_change(fa_ctx* c, const void* K_a, const float* log_u_a,
                         const float* log_v_a, const void* K_b, const float* log_u_b,
                         const float* log_v_b, double* l1_out, fa_stream_t stream) {
  if (!c || !K_a || !log_u_a || !log_v_a || !K_b || !log_u_b || !log_v_b || !l1_out) {
    set_error("fa_plan_change: NULL argument");
    return FA_ERR_ARG;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  double* out = c->diff + kPlanDiffBlocks;
  FA_TRY(launch_plan_l1diff(c->n1, c->n2, c->ld, is_bf16(c), K_a, log_u_a, log_v_a, K_b,
                            log_u_b, log_v_b, c->diff, kPlanDiffBlocks, out, s));
  FA_CUDA(cudaMemcpyAsync(&c->host_err, out, sizeof(double), cudaMemcpyDeviceToHost, s));
  FA_CUDA(cudaStreamSynchronize(s));
  *l1_out = c->host_err;
  if (!std::isfinite(*l1_out)) {
    set_error("fa_plan_change: non-finite plan entries");
    return FA_ERR_NUMERIC;
  }
  return FA_OK;
}

}  // extern "C"
