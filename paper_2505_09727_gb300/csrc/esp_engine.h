// Internal interface of the execution engine for the request server: one
// whole step of a plan enqueued without any host wait.
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "../../include/esp.h"

namespace espe {

// Enqueue on the plan's stream: host->device copy of xyz (FP64, N x 3, pinned
// host memory), ingest + bin sort, the whole compute, device->host copies of
// forces (N x 3), potential (N) and the energy into pinned host buffers, the
// kernels' error flag into *err_host (cleared on the device afterwards), and
// a record of `done`. The plan's charges must be set. Buffers must stay
// valid until `done` has completed.
esp_status plan_enqueue_step(esp_plan_t p, const double* xyz, double* forces, double* potential,
                             double* energy, int* err_host, cudaEvent_t done);

// Device bytes the plan holds (allocations and cuFFT work areas).
size_t plan_device_bytes(esp_plan_t p);

// Device ordinal of the plan.
int plan_device(esp_plan_t p);

// The stream the plan's work runs on.
cudaStream_t plan_stream(esp_plan_t p);

// Message reported by esp_last_error() for the calling thread.
void set_last_error(const std::string& msg);

}  // namespace espe
