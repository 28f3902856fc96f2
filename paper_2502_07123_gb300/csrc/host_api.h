// Host-side internals of the C ABI shared between api.cu and engine.cu.
#pragma once
#include <cuda_runtime.h>

#include <mutex>
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

// The library's context (streams, tables, caches, staging buffers, tuning
// table) is shared by every call: the public entry points hold this lock, so
// calls from several host threads are serialised.
std::recursive_mutex &api_mutex();
#define MLMC_API_LOCK() std::lock_guard<std::recursive_mutex> mlmc_api_lock_(mlmc_host::api_mutex())

// Initialise (once per device) the library's context on the current device.
mlmc_status ensure_ctx();
// The context's internal stream.
cudaStream_t ctx_stream();
// The context's SM count.
int ctx_num_sms();
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

// A work item with its constants and tables resolved (build_item), before
// chunking (chunk_built).
struct BuiltItem {
  mlmc::ItemDesc it;
  int family, scheme, pc;
  size_t smem;
  int kp;               // samples per pack
  double cost_step;     // model cost per fine path-step
  double chunk_cost;    // model cost of one chunk (set by chunk_built)
};
mlmc_status build_item(const mlmc_work &w, int out_index, void *dump, BuiltItem &b, double &disc, int &unit,
                       int &exact_int);
mlmc_status chunk_built(BuiltItem &b, int threads, int spt);
// Launch shape (CTA threads, fine path-steps per thread) of a kernel class.
void tuning_for(int family, int scheme, int pc, int level, int *threads, int *spt);
void make_round_keys(uint64_t seed, mlmc::RoundKeys &rk);
// Launch one level kernel of a family (or, with occ, query the resident CTAs
// per SM of its device-scheduled kernel).
cudaError_t launch_by_family(int fam, int scheme, int pc, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                             const mlmc::LaunchArgs &a, int *occ);

}  // namespace mlmc_host
