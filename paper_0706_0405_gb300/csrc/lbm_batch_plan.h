// lbm_batch_plan.h -- host-side planning of the batch kernel's step order
// (plain C++, no CUDA): for each CTA of a launch, the other CTAs whose tiles
// border one of its own, so that a CTA can start step s + 1 as soon as those
// have finished step s.
#pragma once

#include <vector>

namespace lbm {

// Tile t of the batch is tile (ix, iy) of problem p, whose tiles form a
// tiles_x[p] x tiles_y[p] grid numbered from base[p] in row order.  Two tiles
// border each other if they are next to each other in x or y, or if they are
// the first and last tile of a row (column) of a problem with a periodic x
// (y) side.  owner(t) is the CTA that walks tile t.  out receives max_nbr
// entries per CTA, -1 padded; returns false if some CTA borders more than
// max_nbr others (the caller then orders the steps by a grid barrier).
template <class Owner>
bool batch_plan_neighbours(int ntiles, const int* tile_p, const int* tile_ix, const int* tile_iy,
                           const int* tiles_x, const int* tiles_y, const int* base,
                           const unsigned char* periodic_x, const unsigned char* periodic_y, int grid,
                           Owner owner, int max_nbr, std::vector<int>& out) {
    out.assign((size_t)grid * (size_t)max_nbr, -1);
    std::vector<int> cnt((size_t)grid, 0);
    auto add = [&](int c, int n) {
        if (n == c) return true;
        for (int j = 0; j < cnt[(size_t)c]; ++j)
            if (out[(size_t)c * max_nbr + j] == n) return true;
        if (cnt[(size_t)c] == max_nbr) return false;
        out[(size_t)c * max_nbr + cnt[(size_t)c]++] = n;
        return true;
    };
    for (int t = 0; t < ntiles; ++t) {
        const int p = tile_p[t], tx = tiles_x[p], ty = tiles_y[p];
        const int ix = tile_ix[t], iy = tile_iy[t], c = owner(t);
        const int nb[4][2] = {{ix - 1, iy}, {ix + 1, iy}, {ix, iy - 1}, {ix, iy + 1}};
        for (const auto& q : nb) {
            int jx = q[0], jy = q[1];
            if (jx < 0 || jx >= tx) {
                if (!periodic_x[p]) continue;
                jx = (jx + tx) % tx;
            }
            if (jy < 0 || jy >= ty) {
                if (!periodic_y[p]) continue;
                jy = (jy + ty) % ty;
            }
            if (!add(c, owner(base[p] + jy * tx + jx))) return false;
        }
    }
    return true;
}

}  // namespace lbm
