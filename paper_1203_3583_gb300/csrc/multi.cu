// Sum of several surfaces' fields at one destination (the CGH use the paper's
// conclusion names: an object made of many polygons or surfaces).  The sum
// is linear, so surfaces that share the destination sampling, wavelength,
// distance, oversampling, kernel and source pitch -- hence the fine grid and
// the deconvolution / chirp tables -- are spread into ONE fine grid (the
// default spreading path accumulates with atomic adds) and transformed by one
// row pass and one column pass over the union of their bands.  Each surface
// keeps its own height map, size and position (asfd_params offset_x/y).
#include <algorithm>
#include <cmath>
#include <vector>

#include "asfd_impl.cuh"

namespace asfd {

namespace {

bool same(double a, double b) { return a == b || std::fabs(a - b) <= 1e-12 * std::fabs(a); }

}  // namespace

asfd_status multi_execute(asfd_plan_s* const* plans, const float2* const* u1, int count,
                          float2* u2, cudaStream_t st)
{
    asfd_plan_s* P0 = plans[0];
    const asfd_params& a = P0->prm;
    int ty0 = P0->band_ty0, ty1 = P0->band_ty1, tx0 = P0->band_tx0, tx1 = P0->band_tx1;
    for (int i = 0; i < count; ++i) {
        asfd_plan_s* P = plans[i];
        const asfd_params& b = P->prm;
        if (!u1[i]) return fail(ASFD_ERR_ARG, "u1 pointer is NULL");
        if (P->device != P0->device) return fail(ASFD_ERR_ARG, "plans live on different devices");
        if (!P->dense)
            return fail(ASFD_ERR_UNSUPPORTED,
                        "a multi-surface sum needs the default spread (widths up to 7, "
                        "deterministic = 0, a monotone map without wrap)");
        if (P->nfx != P0->nfx || P->nfy != P0->nfy || b.m2x != a.m2x || b.m2y != a.m2y ||
            !same(b.p2x, a.p2x) || !same(b.p2y, a.p2y) || !same(b.lambda, a.lambda) ||
            !same(b.z0, a.z0) || P->w != P0->w || !same(P->beta, P0->beta) ||
            !same(b.p1x * b.p1y, a.p1x * a.p1y) || P->learned != P0->learned)
            return fail(ASFD_ERR_ARG,
                        "surfaces of one sum must share m2, p2, wavelength, z0, sigma, kernel "
                        "width, beta and the source sample area p1x*p1y");
        ty0 = std::min(ty0, P->band_ty0);
        ty1 = std::max(ty1, P->band_ty1);
        tx0 = std::min(tx0, P->band_tx0);
        tx1 = std::max(tx1, P->band_tx1);
    }
    // clear the union band of the shared grid, spread every surface into it
    const size_t pitch = sizeof(float2) * (size_t)P0->nfx;
    ASFD_CUDA(cudaMemset2DAsync(P0->grid + (size_t)ty0 * kTileY * P0->nfx + (size_t)tx0 * kTileX,
                                pitch, 0, sizeof(float2) * (size_t)(tx1 - tx0) * kTileX,
                                (size_t)(ty1 - ty0) * kTileY, st));
    P0->band_clean = false;
    for (int i = 0; i < count; ++i) {
        const asfd_status s = launch_spread_into(plans[i], u1[i], P0->grid, st);
        if (s != ASFD_OK) return s;
    }
    asfd_status s = launch_fft_rows_band(P0, ty0, ty1, tx0, tx1, st);
    if (s != ASFD_OK) return s;
    return launch_fft_cols_band(P0, ty0, ty1, u2, st);
}

}  // namespace asfd
