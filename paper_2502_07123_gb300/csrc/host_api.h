// Host-side internals of the C ABI shared between api.cu and engine.cu.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "item.h"
#include "mlmc.h"

struct mlmc_plan;

namespace mlmc_host {

// Status-returning wrapper of a CUDA call.
#define MLMC_CK(call)                                 \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return MLMC_ECUDA;         \
  } while (0)

struct Arena;

// Initialise (once per device) the library's context on the current device.
mlmc_status ensure_ctx();
// The context's internal stream.
cudaStream_t ctx_stream();
// Relative cost per fine path-step of an estimator kind (mlmc_cost_model).
double cost_of_variant(int variant);
bool params_ok(const mlmc_params *p);

// Plans: create (borrowing the context arena when `transient`), launch on a
// stream, read results, release.  plan_out_device gives the device array of
// one mlmc::DevSums (undiscounted) per work item of the last launch;
// plan_item_scale gives the factors the host applies to them.
mlmc_status plan_create_transient(mlmc_plan **out, const mlmc_work *work, int n_work, uint64_t seed,
                                  const mlmc_tuning *tuning);
mlmc_status plan_launch_on(mlmc_plan *pl, cudaStream_t st);
const mlmc::DevSums *plan_out_device(const mlmc_plan *pl);
void plan_item_scale(const mlmc_plan *pl, int i, double *disc, int *unit, int *exact_int);
void plan_release(mlmc_plan *pl);

}  // namespace mlmc_host
