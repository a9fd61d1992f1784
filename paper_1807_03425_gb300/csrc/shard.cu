// shard.cu -- the multi-GPU split of the all-pairs step and the exchange that
// merges the ranks' results (host code; no device needed).
//
// Algorithm 1's argmin step (Sec. IV of Kvinge et al., arXiv:1807.03425)
// takes the minimum over all N(N-1)/2 unit secants.  The pairs split into
// disjoint sets with no dependence between them, so each GPU can own a set
// and find its exact minimum on its own; the global minimum is the minimum
// of the ranks' minima.  The split: the upper triangle of 128 x 128 pair
// tiles (I <= J), in row-major order over the tile grid, is cut into `world`
// contiguous ranges of nearly equal pair count (row bands; a band may begin
// or end inside a tile row).  Each rank keeps the points and the basis in
// full but stores and streams only its own tiles' lengths.
//
// Exchange per iteration: every rank contributes one record, its exact
// (FP64) minimum as (q = r^2, i, j) -- 16 bytes -- and all records are
// gathered to every rank; each rank then takes the same FP64 update from the
// same winning pair, so the bases stay identical without further traffic.
#include "sap_internal.cuh"
#include "../../include/sap.h"

#include <algorithm>
#include <cstdint>

namespace {

constexpr int64_t kShardTile = 128;

// Pairs i < j inside tile (I, J) of an N-point set.
int64_t tile_pairs(int64_t N, int64_t I, int64_t J)
{
    const int64_t rI = std::min<int64_t>(kShardTile, N - I * kShardTile);
    const int64_t rJ = std::min<int64_t>(kShardTile, N - J * kShardTile);
    return I == J ? rI * (rI - 1) / 2 : rI * rJ;
}

} // namespace

extern "C" sap_status sap_shard_range(int64_t N, int32_t world, int32_t rank, int64_t *t0, int64_t *t1,
                                      int64_t *pairs)
{
    if (N < 2 || N > 92681 || world < 1 || world > 4096 || rank < 0 || rank >= world) return SAP_E_ARG;
    const int64_t nb = (N + kShardTile - 1) / kShardTile;
    const int64_t P = N * (N - 1) / 2;
    // rank r starts at the first tile whose preceding pairs reach r P / world
    const int64_t lo_target = P * rank / world, hi_target = P * (rank + 1) / world;
    int64_t t = 0, before = 0, first = -1, last = -1, own = 0;
    for (int64_t I = 0; I < nb; ++I)
        for (int64_t J = I; J < nb; ++J, ++t) {
            if (first < 0 && before >= lo_target) first = t;
            if (last < 0 && before >= hi_target && rank + 1 < world) last = t;
            const int64_t p = tile_pairs(N, I, J);
            if (first >= 0 && last < 0) own += p;
            before += p;
        }
    if (first < 0) first = t;
    if (last < 0) last = t;
    if (t0) *t0 = first;
    if (t1) *t1 = last;
    if (pairs) *pairs = own;
    return SAP_OK;
}

extern "C" sap_status sap_merge_records(const sap_record *recs, int32_t count, sap_record *out)
{
    if (!recs || count < 0 || !out) return SAP_E_ARG;
    sap_record best = {0.0, -1, -1};
    for (int32_t e = 0; e < count; ++e) {
        const sap_record &r = recs[e];
        if (r.i < 0) continue;
        // lexicographic (q, i, j): ties go to the smallest pair index
        if (best.i < 0 || r.q < best.q || (r.q == best.q && (r.i < best.i || (r.i == best.i && r.j < best.j))))
            best = r;
    }
    *out = best;
    return best.i < 0 ? SAP_E_NO_SECANT : SAP_OK;
}
