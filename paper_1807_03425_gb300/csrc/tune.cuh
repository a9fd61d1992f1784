// tune.cuh -- the launch-parameter autotuner (tune.cu) and its cache.
#pragma once

#include "sap_internal.cuh"
#include "../../include/sap.h"

namespace sap {

// What a tuning is valid for: the shape of the problem and the settings that
// change the work of an iteration.
struct TuneKey {
    long long N = 0;
    int n = 0, k = 0, dt = 0, path = 0, split = 0;
    unsigned long long eps_bits = 0;
    bool operator<(const TuneKey &o) const;
    bool operator==(const TuneKey &o) const { return !(*this < o) && !(o < *this); }
};

// Engine hooks (capi.cu).
TuneKey handle_tune_key(sap_handle h);
bool handle_path_restructured(sap_handle h);
double *handle_u64(sap_handle h);
int handle_profiling(sap_handle h);
bool &handle_tuning_flag(sap_handle h);
// The key the handle's parameters were last looked up or set for: cached
// parameters are applied only when the handle reaches a new key, so
// parameters set by hand stay until the problem's shape changes.
TuneKey &handle_applied_key(sap_handle h);
void handle_drop_graphs(sap_handle h);

// Whether two parameter sets launch the same kernels the same way.
bool tune_same_launch(const TuneParams &a, const TuneParams &b);
// Apply a parameter set to the handle (re-classifies the near list when the
// pass bound changes; drops captured graphs when anything changes).
sap_status tune_apply(sap_handle h, const TuneParams &p);
// Apply the cached parameters for the handle's current key, if any.
sap_status tune_lookup(sap_handle h);
// Time candidate parameter sets on the handle's current basis and keep the
// fastest (see sap_autotune in sap.h).
sap_status tune_handle(sap_handle h, double alpha, int iters);

} // namespace sap
