// lbm_geometry.cpp -- host-side geometry preparation: per-node link mask and
// the 16x16 tile map with its neighbour-tile table.
//
// Sec. 3 (boundary paragraph) stores a node-type field with a bitmask of the
// neighbours that are present; here one byte per node holds which of the 8
// moving links bounce back (half-way bounce-back).  Sec. 4.2.2 stores only the
// 16^2-node tiles that hold data ("pointer tile"); here the kept tiles are
// numbered densely and a table of 9 neighbour-tile numbers replaces pointers.
#include <vector>

#include "lbm_internal.h"

namespace lbm {
namespace {

const int kCx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
const int kCy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

// Source of link i of node (x, y): true and the node index when x - c_i is a
// lattice node (periodic axes wrapped); false when it lies beyond a wall
// (the y side is examined first).
bool pull_source(const lbm_params &p, int x, int y, int i, long long *src) {
    int sx = x - kCx[i], sy = y - kCy[i];
    if (sy < 0 || sy >= p.ny) {
        if (!p.south.periodic) return false;
        sy = (sy + p.ny) % p.ny;
    }
    if (sx < 0 || sx >= p.nx) {
        if (!p.west.periodic) return false;
        sx = (sx + p.nx) % p.nx;
    }
    *src = (long long)sy * p.nx + sx;
    return true;
}

} // namespace

long long build_link_mask(const lbm_params &p, uint8_t *mask) {
    long long fluid = 0;
    for (int y = 0; y < p.ny; ++y) {
        for (int x = 0; x < p.nx; ++x) {
            const long long n = (long long)y * p.nx + x;
            if (p.solid && p.solid[n]) {
                mask[n] = 0xFF;
                continue;
            }
            unsigned bits = 0;
            for (int i = 1; i < 9; ++i) {
                long long s = 0;
                if (!pull_source(p, x, y, i, &s) || (p.solid && p.solid[s]))
                    bits |= 1u << (i - 1);
            }
            mask[n] = (uint8_t)bits;
            if (bits != 0xFF) ++fluid;
        }
    }
    return fluid;
}

int build_tile_map(const lbm_params &p, const uint8_t *mask, int32_t *tile_id,
                   int32_t *nbr, int32_t *tile_xy) {
    const int ntx = (p.nx + TILE - 1) / TILE, nty = (p.ny + TILE - 1) / TILE;
    int count = 0;
    for (int ty = 0; ty < nty; ++ty)
        for (int tx = 0; tx < ntx; ++tx) {
            bool keep = false;
            const int y1 = ty * TILE + TILE < p.ny ? ty * TILE + TILE : p.ny;
            const int x1 = tx * TILE + TILE < p.nx ? tx * TILE + TILE : p.nx;
            for (int y = ty * TILE; y < y1 && !keep; ++y)
                for (int x = tx * TILE; x < x1; ++x)
                    if (mask[(long long)y * p.nx + x] != 0xFF) { keep = true; break; }
            tile_id[ty * ntx + tx] = keep ? count : -1;
            if (keep) {
                if (tile_xy) tile_xy[count] = (ty << 16) | tx;
                ++count;
            }
        }
    if (nbr) {
        for (int ty = 0; ty < nty; ++ty)
            for (int tx = 0; tx < ntx; ++tx) {
                const int t = tile_id[ty * ntx + tx];
                if (t < 0) continue;
                for (int i = 0; i < 9; ++i) {
                    int ux = tx + kCx[i], uy = ty + kCy[i];
                    bool ok = true;
                    if (ux < 0 || ux >= ntx) {
                        if (p.west.periodic) ux = (ux + ntx) % ntx; else ok = false;
                    }
                    if (uy < 0 || uy >= nty) {
                        if (p.south.periodic) uy = (uy + nty) % nty; else ok = false;
                    }
                    nbr[9 * t + i] = ok ? tile_id[uy * ntx + ux] : -1;
                }
            }
    }
    return count;
}

void build_tile_masks(const lbm_params &p, const uint8_t *mask, const int32_t *tile_xy,
                      int ntiles, uint8_t *tile_mask) {
    for (int t = 0; t < ntiles; ++t) {
        const int tx = tile_xy[t] & 0xFFFF, ty = tile_xy[t] >> 16;
        for (int ly = 0; ly < TILE; ++ly)
            for (int lx = 0; lx < TILE; ++lx) {
                const int x = tx * TILE + lx, y = ty * TILE + ly;
                tile_mask[(long long)t * TILE_N + ly * TILE + lx] =
                    (x < p.nx && y < p.ny) ? mask[(long long)y * p.nx + x] : 0xFF;
            }
    }
}

} // namespace lbm
