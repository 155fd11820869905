// fa_sinkhorn_step_static: one fused Sinkhorn iteration that allocates no
// device memory.  The scratch the sweep and its finalisation need (partial
// column sums, per-block error partials, a block counter and a status word)
// lives in file-scope static device arrays of fixed size, reserved when the
// library is loaded and held by every GPU that loads it until the process
// exits.  Host code reaches them only through cudaGetSymbolAddress: the
// array names seen by host code are host-side stand-ins, not device
// addresses.
#include <algorithm>
#include <mutex>
#include <utility>
#include <vector>

#include "fa_internal.cuh"

namespace fa {

constexpr int64_t kStaticMaxLd = 65536;            // padded columns
constexpr int64_t kStaticColpart = int64_t(1) << 21;  // floats: 8 MiB
constexpr int kStaticMaxBlocks = (int)((kStaticMaxLd + 255) / 256);

// Partial column sums, one row of ld floats per row group of the sweep: at
// most kStaticColpart / ld groups (32 at the largest ld), plus small counters.
static __device__ __align__(256) float g_static_colpart[kStaticColpart];
static __device__ __align__(256) double g_static_err_part[kStaticMaxBlocks];
static __device__ __align__(256) unsigned g_static_ticket[1];
static __device__ __align__(256) int g_static_status[1];

struct StaticScratch {
  float* colpart = nullptr;
  double* err_part = nullptr;
  unsigned* ticket = nullptr;
  int* status = nullptr;
};

constexpr int kMaxDevices = 128;
static std::mutex g_static_mu;
static bool g_static_ready[kMaxDevices] = {};
static StaticScratch g_static_ptrs[kMaxDevices];

// Sweep shapes already planned, per (device, n1, ld, storage type): the
// entry is meant for loops of many calls, so the host-side planning and
// the occupancy query run once per shape, not on every call.
struct PlanKey {
  int dev;
  int32_t n1;
  int64_t ld;
  bool bf16;
};
static std::vector<std::pair<PlanKey, SweepPlan>> g_static_plans;

// Device addresses of the static scratch on the current device, looked up
// once per device (the first call on a device does it).
static fa_status static_scratch(StaticScratch* out) {
  int dev = 0;
  FA_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("fa_sinkhorn_step_static: device ordinal %d not supported", dev);
    return FA_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ready[dev]) {
    StaticScratch p;
    FA_CUDA(cudaGetSymbolAddress(reinterpret_cast<void**>(&p.colpart), g_static_colpart));
    FA_CUDA(cudaGetSymbolAddress(reinterpret_cast<void**>(&p.err_part), g_static_err_part));
    FA_CUDA(cudaGetSymbolAddress(reinterpret_cast<void**>(&p.ticket), g_static_ticket));
    FA_CUDA(cudaGetSymbolAddress(reinterpret_cast<void**>(&p.status), g_static_status));
    g_static_ptrs[dev] = p;
    g_static_ready[dev] = true;
  }
  *out = g_static_ptrs[dev];
  return FA_OK;
}

}  // namespace fa

using namespace fa;

extern "C" fa_status fa_sinkhorn_step_static(const void* K, int32_t dtype, int32_t n1,
                                             int32_t n2, int64_t ld, const float* log_v,
                                             float* log_u, float* log_v_next, double* err,
                                             int32_t* status, fa_stream_t stream) {
  if (!K || !log_v || !log_u || !log_v_next || !err) {
    set_error("fa_sinkhorn_step_static: NULL argument");
    return FA_ERR_ARG;
  }
  if (dtype != FA_F32 && dtype != FA_BF16) {
    set_error("fa_sinkhorn_step_static: bad dtype %d", dtype);
    return FA_ERR_ARG;
  }
  if (n1 < 1 || n2 < 1 || ld < n2 || ld % kLdAlign != 0) {
    set_error("fa_sinkhorn_step_static: need n1, n2 >= 1 and ld >= n2 a multiple of %lld",
              (long long)kLdAlign);
    return FA_ERR_ARG;
  }
  if (ld > kStaticMaxLd) {
    set_error("fa_sinkhorn_step_static: ld = %lld exceeds the static scratch maximum of %lld "
              "columns; use fa_sinkhorn with a context",
              (long long)ld, (long long)kStaticMaxLd);
    return FA_ERR_UNSUPPORTED;
  }
  if ((reinterpret_cast<uintptr_t>(K) & 15u) != 0) {
    set_error("fa_sinkhorn_step_static: K must be 16-byte aligned");
    return FA_ERR_ARG;
  }
  StaticScratch P;
  FA_TRY(static_scratch(&P));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int* st = status ? status : P.status;
  // the block counter of the error reduction and the status word start at 0
  FA_CUDA(cudaMemsetAsync(P.ticket, 0, sizeof(unsigned), s));
  FA_CUDA(cudaMemsetAsync(st, 0, sizeof(int), s));
  const bool bf16 = dtype == FA_BF16;
  int dev = 0;
  FA_CUDA(cudaGetDevice(&dev));
  SweepPlan sp;
  bool have = false;
  {
    std::lock_guard<std::mutex> lock(g_static_mu);
    for (const auto& e : g_static_plans)
      if (e.first.dev == dev && e.first.n1 == n1 && e.first.ld == ld && e.first.bf16 == bf16) {
        sp = e.second;
        have = true;
        break;
      }
  }
  if (!have) {
    // as many row groups as clusters fit on the device at once, bounded by
    // the rows of partial column sums the static array holds
    sp = plan_sweep(n1, ld, bf16, 1 << 20);
    const int resident = sp.Q >= 1 ? sweep_max_active_clusters(sp, bf16) : 0;
    const int max_G = (int)std::min<int64_t>(std::max(1, resident), kStaticColpart / ld);
    sp = plan_sweep(n1, ld, bf16, max_G);
    std::lock_guard<std::mutex> lock(g_static_mu);
    g_static_plans.push_back({PlanKey{dev, n1, ld, bf16}, sp});
  }
  FA_TRY(launch_sweep(sp, n1, n2, ld, K, bf16, log_v, log_u, 1.0f / (float)n1, P.colpart, st, s));
  FA_TRY(launch_col_finalize(n2, ld, sp.G, P.colpart, log_v, 1.0f / (float)n2, log_v_next,
                             P.err_part, P.ticket, err, st, s));
  return FA_OK;
}
