// inc_plan.cuh -- the copy plan of one offspring of the incremental
// Gram-delta mode (a7): which 16-byte units of its parents' stored half-Grams
// (H = G / 2 as int8 in 8 x 8 tiles, common.cuh) an offspring cut at column c
// copies, and the ring slot each lands in.  Host and device, so that the
// plan's coverage can be checked exhaustively on the CPU.
#pragma once

#include <cstdint>

#include "common.cuh"

namespace hadga {

// Copies of one offspring cut at c, in 16-byte groups (16-byte units of a
// Gram buffer):
//  [0, nG)              phase 1: the H[:c, :c] tiles of Pt (4 nTL groups,
//                       the triangle of side J0 = c / 8), then the H[c:, c:]
//                       tiles of Pb (from tile tBR on);
//  [nG, nG + n4g)       when 8 does not divide c: Pt's rows i < c of tile
//                       column J0 (row pairs 2q, 2q + 1), read by phase 2;
//  [.., total)          and Pb's rows i >= c of tile row I0 = c / 8 (row
//                       pairs from r0 & ~1 on, g3 per tile), copied to O.
struct IncCopyPlan {
    int nTL, J0, nb, tBR, nG, n4g, n3g, g3, r0, total;
    __host__ __device__ IncCopyPlan(int m, int c)
    {
        nb = gram_tiles_nb(m);
        const int nt = nb * (nb + 1) / 2, I1 = (c + 7) >> 3;
        J0 = c >> 3;
        nTL = J0 * (J0 + 1) / 2;
        tBR = I1 * nb - (I1 * (I1 - 1)) / 2;
        nG = 4 * (nTL + (nt - tBR));
        r0 = c & 7;
        g3 = r0 ? 4 - (r0 >> 1) : 0;
        n4g = r0 ? (c + 1) >> 1 : 0;
        n3g = g3 * (nb - J0);
        total = nG + n4g + n3g;
    }
    __host__ __device__ __forceinline__ uint32_t tile(int I, int J) const
    {
        return (uint32_t)(I * nb - (I * (I - 1)) / 2 + (J - I));
    }
    // unit of extra group x in [0, n4g + n3g) and whether it comes from Pt
    __host__ __device__ __forceinline__ uint32_t extra_unit(int x, bool &from_pt) const
    {
        if (x < n4g) {
            const int i = 2 * x;
            from_pt = true;
            return tile(i >> 3, J0) * 4u + (uint32_t)((i & 7) >> 1);
        }
        x -= n4g;
        from_pt = false;
        const int J = J0 + x / g3, q = (r0 >> 1) + x % g3;
        return tile(J0, J) * 4u + (uint32_t)q;
    }
};

// A lane's phase-1 groups e = e0, e0 + 32, ...: the H[:c, :c] tile (I, J) is
// stepped through the triangle of side J0 (8 tiles per step), no root taken
// per group.
struct IncGroupIter {
    int e, I, J;
    __host__ __device__ __forceinline__ IncGroupIter(const IncCopyPlan &pl, int e0) : e(e0), I(0), J(0)
    {
        if (e0 < 4 * pl.nTL)
            tile_coords(e0 >> 2, pl.J0, I, J);
    }
    __host__ __device__ __forceinline__ bool from_pt(const IncCopyPlan &pl) const { return e < 4 * pl.nTL; }
    __host__ __device__ __forceinline__ uint32_t unit(const IncCopyPlan &pl) const
    {
        return from_pt(pl) ? pl.tile(I, J) * 4u + (uint32_t)(e & 3) : (uint32_t)(pl.tBR * 4 + (e - 4 * pl.nTL));
    }
    __host__ __device__ __forceinline__ void next(const IncCopyPlan &pl)
    {
        e += 32;
        if (e < 4 * pl.nTL) {
            J += 8;
            while (J >= pl.J0 && I < pl.J0 - 1) {
                J = J - pl.J0 + I + 1;
                ++I;
            }
        }
    }
};

} // namespace hadga
