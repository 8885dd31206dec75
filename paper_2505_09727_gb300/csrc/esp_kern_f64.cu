// FP64 plain-mode instantiations of the ESP kernels (P = 4 ... 16).
#define ESP_REAL double
#define ESP_P_MIN 4
#define ESP_NEAR_SHORT 24
#define ESP_P_MAX 16
// P = 4 ... 7 here, 8 ... 16 in esp_kern_f64_rest.cu (compiled in parallel)
#define ESP_P_CASES(FN, ...)                                              \
  ESP_P_CASE(4, FN, __VA_ARGS__) ESP_P_CASE(5, FN, __VA_ARGS__)           \
  ESP_P_CASE(6, FN, __VA_ARGS__) ESP_P_CASE(7, FN, __VA_ARGS__)
#include "esp_kern_impl.cuh"

namespace espk {

// The cluster form of the local part is FP32 only; FP64 plans use k_near.
template <>
cudaError_t Launch<double>::near_clusters(const SysDesc*, int, long long, const uint32_t*, const void*,
                                          void*, const NearCoef<double>&, int, uint32_t*, uint32_t*,
                                          uint32_t*, int2*, int2*, long long, bool, long long, int, int*,
                                          cudaStream_t, double*, bool) {
  return cudaErrorNotSupported;
}

}  // namespace espk
