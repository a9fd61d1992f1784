// sweep.cuh -- the dimension-estimation sweep (Sec. VI-A): SAP for every
// k = 1..k_max over one dataset, all bases advancing together.
#pragma once

#include <cuda.h>
#include <vector>

#include "sap_internal.cuh"
#include "../../include/sap.h"

namespace sap {

struct SweepBasis {
    int k = 0, KP = 0, KY = 0, off = 0;  // width, FP32 stride, Y stride, first component in the sweep's Y
    double *U64 = nullptr;               // n x k column-major
    float *Ydh = nullptr, *Ydl = nullptr;  // double-float Y of the refine tier, KY x Npad
    float *U32 = nullptr, *U32lo = nullptr;
    double *work = nullptr;
    ProbState *st = nullptr;
    int2 *cand1 = nullptr, *cand2 = nullptr;
    Partial *partials = nullptr;
    double *hist = nullptr;
    int2 *am = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
};

struct SweepState {
    int kmax = 0;
    int hist_cap = 0;
    int last_iters = -1;
    long long cap = 0;
    std::vector<SweepBasis> b;
    void *Uhi = nullptr, *Ulo = nullptr;  // all bases' split operands, KPG x NP 16-bit
    int KPG = 0;
    CUtensorMap mhi, mlo;
    float *Y = nullptr;                   // KY x Npad, all bases' components
    float *Yd = nullptr;                  // doubled row-side copy for the pass (2 KY x Npad)
    int KY = 0;
    float *Ypart = nullptr;
    int ksplit = 1;
    ProbState *gst = nullptr;             // status word of the product
    cudaEvent_t fork = nullptr;
    // captured chunks, reused while the handle's buffers and settings stay
    struct Graph {
        cudaGraphExec_t exec;
        double alpha;
        int eval_only, chunk, n_near;
        long long gen, launches;
    };
    std::vector<Graph> graphs;
};

sap_status sweep_run(sap_handle h, const double *U0, int kmax, int iters, double alpha, double threshold,
                     int *k_out, double *ratios_out);
sap_status sweep_history(sap_handle h, int k, double *hist, int64_t *argmins, int capacity);
sap_status sweep_basis(sap_handle h, int k, double *U_out, int out_is_device);
void sweep_free(SweepState *&s);

// Engine accessors (capi.cu).
SweepState *&sweep_state(sap_handle h);
long long handle_graph_gen(sap_handle h);
int handle_mode(sap_handle h);
Cert handle_seed_cert(int n, int k);
sap_status handle_check_status(sap_handle h, ProbState *st);

} // namespace sap
