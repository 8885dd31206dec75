// Throughput microbenchmarks that give the roofline denominators of the
// arithmetic kernels on the GPU at hand, at its current clocks:
//  * FP32 fused multiply-add, scalar (FFMA) and packed two-wide (the
//    f32x2 instructions of sm_100-class GPUs): many independent chains per
//    thread, every SM filled;
//  * shared memory: float atomicAdd and plain read-add-write to
//    conflict-free addresses (lane l uses bank l), the two ways a spread
//    tile can accumulate.
// Each launch is timed with CUDA events on a private stream after a
// warm-up launch; the best of `reps` launches is reported. Results are
// operations per second over the whole GPU (a multiply-add counts 2 flop).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;        // independent accumulators per thread (scalar)
constexpr int kIters = 4096;

__global__ void __launch_bounds__(kThreads) k_ffma(float* out, float a, float b) {
  float v[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) v[k] = (float)(threadIdx.x + k);
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) v[k] = fmaf(v[k], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += v[k];
  if (s == 12345.678f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains live
}

__global__ void __launch_bounds__(kThreads) k_ffma2(float* out, float a, float b) {
  float2 v[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) v[k] = make_float2((float)(threadIdx.x + k), (float)(threadIdx.x - k));
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) v[k] = __ffma2_rn(v[k], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += v[k].x + v[k].y;
  if (s == 12345.678f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Shared accumulation: every lane owns bank (lane) of rows of 32 floats;
// each warp works on its own rows, 8 rows per warp, updated in turn.
constexpr int kRows = 8;
constexpr int kSharedIters = 2048;

template <bool ATOMIC>
__global__ void __launch_bounds__(kThreads) k_shared(float* out, float x) {
  __shared__ float tile[kThreads / 32][kRows][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int r = 0; r < kRows; ++r) tile[w][r][lane] = 0.f;
  __syncwarp();
  for (int it = 0; it < kSharedIters; ++it) {
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      if (ATOMIC) {
        atomicAdd(&tile[w][r][lane], x);
      } else {
        volatile float* p = &tile[w][r][lane];    // a real load and store every time
        *p = *p + x;
      }
    }
  }
  __syncwarp();
  float s = 0.f;
#pragma unroll
  for (int r = 0; r < kRows; ++r) s += tile[w][r][lane];
  if (s == 12345.678f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename F>
int best_ms(F launch, int reps, cudaStream_t st, float* best) {
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return 1;
  launch();                                       // warm-up
  *best = 1e30f;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(a, st);
    launch();
    cudaEventRecord(b, st);
    if (cudaEventSynchronize(b) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    *best = std::min(*best, ms);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return cudaGetLastError() != cudaSuccess;
}

}  // namespace

extern "C" {

// out[0] FP32 FFMA flop/s, out[1] FP32 packed FFMA2 flop/s, out[2] shared
// float atomicAdd/s, out[3] shared read-add-write/s, out[4] SM count,
// out[5] FP32 lanes assumed per SM for the scalar rate check (128).
// Returns 0 on success, 1 on a CUDA error.
int esp_measure_peaks(int device, int reps, double* out) {
  if (!out || reps < 1) return 1;
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return 1;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaStream_t st;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return 1;
  float* d_out = nullptr;
  const int blocks = sms * 8;                     // 8 resident blocks of 256 threads per SM
  int rc = cudaMalloc(&d_out, (size_t)blocks * kThreads * sizeof(float)) != cudaSuccess;
  float ms = 0.f;
  const double threads = (double)blocks * kThreads;
  if (!rc) {
    rc |= best_ms([&] { k_ffma<<<blocks, kThreads, 0, st>>>(d_out, 0.999f, 1e-3f); }, reps, st, &ms);
    out[0] = threads * kChains * kIters * 2.0 / (ms * 1e-3);
    rc |= best_ms([&] { k_ffma2<<<blocks, kThreads, 0, st>>>(d_out, 0.999f, 1e-3f); }, reps, st, &ms);
    out[1] = threads * kChains * kIters * 4.0 / (ms * 1e-3);
    rc |= best_ms([&] { k_shared<true><<<blocks, kThreads, 0, st>>>(d_out, 1e-3f); }, reps, st, &ms);
    out[2] = threads * kRows * kSharedIters / (ms * 1e-3);
    rc |= best_ms([&] { k_shared<false><<<blocks, kThreads, 0, st>>>(d_out, 1e-3f); }, reps, st, &ms);
    out[3] = threads * kRows * kSharedIters / (ms * 1e-3);
    out[4] = sms;
    out[5] = 128;
  }
  if (d_out) cudaFree(d_out);
  cudaStreamDestroy(st);
  cudaSetDevice(prev);
  return rc;
}

}  // extern "C"
