// softmin.cuh -- buffers and entry points of the soft-min objective (a
// differentiable surrogate of the SAP minimum; the paper has no counterpart),
// used by the engine in capi.cu.
#pragma once

#include "sap_internal.cuh"
#include "../../include/sap.h"

namespace sap {

// Device scalars of the soft-min kernels.
struct SoftDev {
    double L;               // latest forward value
    double gnorm;           // ||G_R||_F of the latest ascent step
    int status;             // StatusBits
    unsigned int ticket;    // blocks of the forward pass that finished
    int step;               // ascent steps taken (history index)
    int hist_cap;
};

// Per-block partial of the shifted exponential sum: sum exp((M - r)/tau).
struct SoftPart {
    double S;
    float M;
    int pad;
};

struct SoftState {
    int k = 0;                  // basis width the buffers were made for
    float *Yh = nullptr, *Yl = nullptr;  // Y = X U as hi + lo FP32 pairs, k x Npad
    SoftPart *part = nullptr;   // forward partials: far-pass blocks, then near blocks
    int part_cap = 0;
    float *P = nullptr;         // backward tile partials: ntiles x 2 x k x 128
    float2 *GP = nullptr;       // gradient partials (hi, lo): (nb + near blocks) x k x n
    int gp_cap = 0;
    double *G = nullptr;        // k x n (the n x k column-major gradient)
    SoftDev *dev = nullptr;
    double *hist = nullptr;
    int hist_cap = 0;
    int grid_far = 0;           // persistent pass grid
    int near_blocks = 0;        // blocks of the near-pair kernels
    int n_near = -1;            // near count the grids were sized for
};

sap_status softmin_forward(sap_handle h, double tau, double *L_out);
sap_status softmin_backward(sap_handle h, double tau, double L, double *G_out, int out_is_device);
sap_status softmin_ascent(sap_handle h, double tau, double eta, int steps, double *hist);
void softmin_free(sap_handle h);

// Engine accessors (capi.cu) beyond those of restructured.cuh.
SoftState &soft_state(sap_handle h);
double *handle_u64(sap_handle h);
float *handle_u32_mut(sap_handle h);
sap_status handle_reset_state(sap_handle h);
int handle_profiling(sap_handle h);
long long handle_launches(sap_handle h);
void handle_add_launches(sap_handle h, long long delta);

} // namespace sap
