// gemm_tc.cuh -- launcher interface of the tensor-core product Y = X U.
#pragma once

#include <cuda.h>
#include "sap_internal.cuh"

namespace sap {

struct GemmArgs {
    CUtensorMap ta_hi, ta_lo;   // X split parts: Npad x NP, 16-bit, box 64 x 128
    CUtensorMap tb_hi, tb_lo;   // U split parts: KPG x NP, 16-bit, box 64 x KPG
    float *Y;                   // FP32, block-major: [Npad/128][KY][128]
    // optional second copy for the row side of the all-pairs pass: per
    // block and component 256 floats, row a = 16 r + g at g * 16 + (r / 2) * 4
    // + (r % 2) * 2, written twice ({y, y} pairs)
    float *Yd;
    int KY;                     // components written (multiple of 4, <= KPG)
    int Npad;                   // rows (multiple of 128)
    int nkb;                    // K blocks of 64
    int KPG;                    // MMA N: multiple of 16, 16..256
    int ab_bf16;                // operand type: 1 BF16, 0 FP16
    int stages;                 // shared-memory ring depth
    float lo_scale;             // 2^-s: weight of the low-part accumulator
    float out_scale;            // 1/scale of X
    ProbState *st;              // receives ST_TIMEOUT if a wait gives up
    int ksplit;                 // K slices (grid.y); > 1: raw slices go to Ypart
    float *Ypart;               // ksplit x KY x Npad FP32 (ksplit > 1)
    int pdl;                    // programmatic launch (see sap_internal.cuh)
    // Seeds of the next all-pairs pass, computed by idle warps of every CTA
    // (single-basis handles; null seed_st: none): the recent argmin pairs'
    // ratios under the basis this product uses, in extended precision from
    // explicit differences, as certified upper bounds merged into
    // seed_st->seed_ub by an atomic minimum (the update that changed the
    // basis reset it to +inf; an unchanged basis keeps its valid bound).
    const float *seed_X = nullptr;   // N x n row-major FP32 points
    const float *seed_U = nullptr;   // the basis, FP32 n x KP row-major ...
    const float *seed_Ulo = nullptr; // ... and its FP32 residual
    ProbState *seed_st = nullptr;
    int seed_N = 0, seed_n = 0, seed_k = 0, seed_KP = 0;
};

size_t gemm_smem_bytes(int KPG, int stages);
int gemm_pick_stages(int KPG, int nkb);
cudaError_t gemm_configure();
// Y = X U; with ksplit > 1 each K slice accumulates separately (shorter FP32
// chains) and a second kernel sums the slices into Y.
cudaError_t launch_gemm_y(const GemmArgs &a, cudaStream_t s);

} // namespace sap
