// restructured.cuh -- buffers and entry points of the restructured form
// (Y = X U on tensor cores, then an all-pairs pass over stored inverse squared
// lengths), used by the engine in capi.cu.
#pragma once

#include "sap_internal.cuh"
#include "gemm_tc.cuh"
#include "../../include/sap.h"

namespace sap {

struct RestrState {
    // centred, scaled, split copy of X: Npad x NP 16-bit, hi and lo parts
    void *Xhi = nullptr, *Xlo = nullptr;
    int Npad = 0;         // N rounded up to the tile (128)
    int NP = 0;           // n rounded up to the GEMM k-block (64)
    float xscale = 1.f;   // power of two applied to (x - mean) before splitting
    float *center = nullptr;  // column means (n), FP32
    float *nu = nullptr;  // ||fl(x_i - mean)||, rounded up (Npad)
    // inverse squared lengths, tile-major upper triangle (kTile x kTile tiles);
    // NaN marks a pair the pass skips (invalid, excluded, or near)
    float *w = nullptr;
    // the same tiles as BF16 w_ij (raw bits), the form the pass streams
    // (2 bytes per pair); NaN where w is NaN
    uint16_t *wb = nullptr;
    int2 *wtiles = nullptr;   // (I, J) per tile, I <= J
    int nwtiles = 0;
    long long tile0 = 0;      // global index of the first stored tile (a shard's range starts there)
    int2 *near = nullptr;     // pairs the pass skips, evaluated by the refine tier
    float *near_w = nullptr;  // their 1/d^2 (FP32; +inf when too short for FP32)
    unsigned int near_cap = 0;
    float *xn = nullptr;      // ||x_i|| (not centred), rounded up (Npad)
    unsigned int *counters = nullptr;  // [0] near count, [1..2] excluded (u64)
    int n_near = 0;
    long long n_excluded = 0;
    int k_cls = 0;            // k the near classification was made for
    double y_eps = 0.0;       // bound on |y~ - y| per unit ||x - mean||
    double b_cap = 5e-4;      // absolute ratio bound of the all-pairs pass
    // basis operands
    void *Uhi = nullptr, *Ulo = nullptr;  // KPG x NP 16-bit
    int KPG = 0;              // k rounded up to the MMA N granule (16)
    float *Y = nullptr;       // block-major [Npad/128][KY][128]
    float *Yd = nullptr;      // doubled row-side copy of Y for the pass: [Npad/128][KY][256]
    float *Ydh = nullptr, *Ydl = nullptr;  // double-float Y of the refine tier, KY x Npad each
    int KY = 0;               // k rounded up to 4
    int ksplit = 1;           // K slices of the product (shorter accumulation chains)
    float *Ypart = nullptr;   // ksplit x KY x Npad slice results (ksplit > 1)
    GemmArgs gemm;            // tensor maps and shapes of the product
    bool maps_x = false, maps_u = false;
};

// Engine accessors (capi.cu).
RestrState &restr_state(sap_handle h);
cudaStream_t handle_stream(sap_handle h);
int handle_sms(sap_handle h);
ProbState *handle_state(sap_handle h);
const float *handle_x32(sap_handle h);
const float *handle_u32(sap_handle h);
int restructured_pass_grid(sap_handle h);  // blocks of the all-pairs pass
Partial *handle_partials(sap_handle h);
double *handle_u64(sap_handle h);
const float *handle_u32lo(sap_handle h);
int2 *handle_cand1(sap_handle h);
int2 *handle_cand2(sap_handle h);
long long handle_cap(sap_handle h);
int handle_k(sap_handle h);
int handle_kp(sap_handle h);
int64_t handle_n_points(sap_handle h);
int handle_n_dim(sap_handle h);
int handle_split_bf16(sap_handle h);
double handle_eps2(sap_handle h);
float handle_eps2_lo(sap_handle h);
float handle_eps2_hi(sap_handle h);
void handle_count_launch(sap_handle h, int cls, cudaEvent_t *a, cudaEvent_t *b);
void handle_push_timing(sap_handle h, int cls, cudaEvent_t a, cudaEvent_t b);
sap_status handle_fail(sap_handle h, sap_status s, const char *msg);
TuneParams &handle_tune(sap_handle h);
void handle_shard(sap_handle h, long long *t0, long long *t1);  // stored tile range (all tiles: 0, -1)

// One basis of the restructured form: the handle's own, or one of the bases
// of a dimension sweep that share the handle's dataset, lengths and near list.
struct BasisView {
    int k, KP, KY;            // width, FP32 basis stride, Y stride (components)
    const float *U32, *U32lo; // n x KP FP32 basis and its low part
    float *Y;                 // this basis's first component in block 0 of a block-major Y
    float *Yd;                // the same in the doubled row-side copy (block stride Ykt * 256)
    int Ykt;                  // components per 128-point block of that Y buffer
    float *Ydh, *Ydl;         // double-float Y (refine tier), KY x Npad each
    ProbState *st;
    int2 *cand1, *cand2;      // candidate lists of the pass and of the explicit tier
    long long cap;            // capacity of each list
    const double *U64;        // n x k FP64 basis, column-major (tiers inside the pass)
    Partial *partials;        // per-block best pairs (tiers inside the pass)
};

// Restructured-form entry points (restructured.cu).
// seeds: the product also evaluates the next pass's seed bound (one basis
// per handle; the update then leaves the seeds to it)
sap_status restructured_enqueue_product(sap_handle h, const CUtensorMap *mhi, const CUtensorMap *mlo, int KPG,
                                        float *Y, float *Yd, int KY, float *Ypart, ProbState *st, cudaStream_t s,
                                        bool seeds = false);
sap_status restructured_enqueue_basis(sap_handle h, const BasisView &b, cudaStream_t s); // pass + explicit tier
bool restructured_u_maps(sap_handle h, void *Uhi, void *Ulo, int KPG, CUtensorMap *mhi, CUtensorMap *mlo);
void restructured_split_host(sap_handle h, const double *U, int k, uint16_t *hi, uint16_t *lo); // k rows of NP
sap_status restructured_classify(sap_handle h, int k);  // near list for width k (valid for every k' <= k)
sap_status restructured_prepare(sap_handle h);          // X split, norms, lengths, near list
sap_status restructured_basis_alloc(sap_handle h);      // U operands and Y for k
sap_status restructured_upload_basis(sap_handle h, const double *U); // n x k col-major
sap_status restructured_enqueue(sap_handle h, double alpha);
int restructured_kernels_per_iteration(sap_handle h);
// Second tier of the restructured form: 0 explicit differences (own
// launch), 1 double-float Y + refine, 2 explicit differences fused into the
// FP64 recheck (tuning value 2; only where the plain FP32 explicit tier
// applies, n <= 256, else 0), 3 explicit differences in extended precision
// fused into the FP64 recheck on the tier's grid (tuning value 3; k <= 8,
// else 0), 4 explicit differences in extended precision in their own
// launch, whose list carries each pair's ratio so that the FP64 recheck
// evaluates only the pairs within the final bound (tuning value 4).
int restructured_tier(sap_handle h);
int restructured_tier_for(sap_handle h, int k);
bool restructured_uses_refine(sap_handle h);
// Fills the fused-tier fields of the FP64 recheck of basis b (fused = 0
// unless the tier is 2 or 3; then list/which name the pass's candidates,
// and for tier 3 the grid is the tier's).
void restructured_fuse_args(sap_handle h, const BasisView &b, SelectUpdateArgs &u);
void restructured_free(sap_handle h);
void restructured_stats(sap_handle h, sap_stats *out);
sap_status restructured_set_bound(sap_handle h, double b_cap);
sap_status restructured_project(sap_handle h, float *Y_out, int out_is_device);
sap_status restructured_project_df(sap_handle h, float *Yh_out, float *Yl_out, int out_is_device);

} // namespace sap
