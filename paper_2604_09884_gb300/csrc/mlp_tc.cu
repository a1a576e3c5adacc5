// placeholder: BF16 tensor-core path not built yet
#include "mlp.cuh"
namespace inrct {
bool tc_supported(const Net&, char* why, size_t n) { snprintf(why, n, "not built"); return false; }
size_t tc_eval_ws_bytes(const Net&) { return 0; }
int tc_eval(const Net&, const float*, int, int64_t, float*, void*, size_t, cudaStream_t) { return INRCT_ERR_UNSUPPORTED; }
size_t tc_vjp_ws_bytes(const Net&, int64_t) { return 0; }
int tc_vjp(const Net&, const float*, int, const int32_t*, int64_t, const float*, double, double*, float*, void*, size_t, cudaStream_t) { return INRCT_ERR_UNSUPPORTED; }
}
