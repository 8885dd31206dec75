// FP64 spread and gather instantiations for P = 8 ... 16 (the rest of the
// stencil widths of esp_kern_f64.cu, compiled in parallel with it).
#define ESP_REAL double
#define ESP_P_MIN 4
#define ESP_NEAR_SHORT 24
#define ESP_P_MAX 16
#define ESP_IMPL_REST
#define ESP_P_CASES(FN, ...)                                              \
  ESP_P_CASE(8, FN, __VA_ARGS__) ESP_P_CASE(9, FN, __VA_ARGS__)           \
  ESP_P_CASE(10, FN, __VA_ARGS__) ESP_P_CASE(11, FN, __VA_ARGS__)         \
  ESP_P_CASE(12, FN, __VA_ARGS__) ESP_P_CASE(13, FN, __VA_ARGS__)         \
  ESP_P_CASE(14, FN, __VA_ARGS__) ESP_P_CASE(15, FN, __VA_ARGS__)         \
  ESP_P_CASE(16, FN, __VA_ARGS__)
#include "esp_kern_impl.cuh"
