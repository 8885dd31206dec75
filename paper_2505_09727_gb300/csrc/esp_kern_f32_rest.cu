// FP32 spread and gather instantiations for P = 8 ... 12 (the rest of the
// stencil widths of esp_kern_f32.cu, compiled in parallel with it).
#define ESP_REAL float
#define ESP_P_MIN 4
#define ESP_NEAR_SHORT 10
#define ESP_P_MAX 12
#define ESP_IMPL_REST
#define ESP_P_CASES(FN, ...)                                              \
  ESP_P_CASE(8, FN, __VA_ARGS__) ESP_P_CASE(9, FN, __VA_ARGS__)           \
  ESP_P_CASE(10, FN, __VA_ARGS__) ESP_P_CASE(11, FN, __VA_ARGS__)         \
  ESP_P_CASE(12, FN, __VA_ARGS__)
#include "esp_kern_impl.cuh"
