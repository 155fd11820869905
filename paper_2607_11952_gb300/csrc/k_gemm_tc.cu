// placeholder until the tcgen05 kernel lands
#include "fa_internal.cuh"
namespace fa {
bool tc_gemm_available() { return false; }
size_t node_cost_tc_workspace(int, int, int, int, bool) { return 0; }
fa_status launch_node_cost_tc(int, int, int, int64_t, const float*, const float*, int, int64_t,
                              const float*, const float*, float, bool, float*, int64_t, void*,
                              size_t, int*, cudaStream_t) {
  set_error("tcgen05 GEMM not built");
  return FA_ERR_UNSUPPORTED;
}
}  // namespace fa
