// Exhaustive host-side check of the incremental mode's copy plan
// (inc_plan.cuh): for every order m = 36, 40, ..., 128 and every cut
// c = 1 .. m-1, the ring slots 0 .. total-1 are each filled exactly once, and
// the 16-byte units copied are exactly
//   - every unit of the H[:c, :c] tiles (tile column J < c/8) from the top
//     parent Pt,
//   - every unit of the tiles of tile rows I >= ceil(c/8) from the bottom
//     parent Pb,
//   - when 8 does not divide c: Pt's row pairs of tile column c/8 holding the
//     rows i < c, and Pb's row pairs of tile row c/8 holding the rows i >= c,
// with no unit twice.  Phase-1 groups are enumerated as the kernel's lanes
// do (IncGroupIter from lane, stepping by 32).  Prints "ok" and exits 0 on
// success, else the first failure and exits 1.
#include <cstdio>
#include <set>
#include <utility>
#include <vector>

#include "inc_plan.cuh"

using hadga::IncCopyPlan;
using hadga::IncGroupIter;

static int fail(int m, int c, const char *what)
{
    std::printf("m=%d c=%d: %s\n", m, c, what);
    return 1;
}

int main()
{
    long checked = 0;
    for (int m = 36; m <= 128; m += 4) {
        for (int c = 1; c < m; ++c) {
            const IncCopyPlan pl(m, c);
            const int nb = pl.nb, J0 = c >> 3, I1 = (c + 7) >> 3, r0 = c & 7;
            // expected (from Pt?, unit) pairs
            std::set<std::pair<int, uint32_t>> want;
            for (int I = 0; I < nb; ++I)
                for (int J = I; J < nb; ++J) {
                    const bool tl = J < J0, br = I >= I1;
                    for (uint32_t q = 0; q < 4; ++q) {
                        if (tl)
                            want.insert({1, pl.tile(I, J) * 4u + q});
                        if (br)
                            want.insert({0, pl.tile(I, J) * 4u + q});
                    }
                }
            if (r0) {
                for (int i = 0; i < c; i += 2)  // Pt's row pairs with rows i < c in tile column J0
                    want.insert({1, pl.tile(i >> 3, J0) * 4u + (uint32_t)((i & 7) >> 1)});
                for (int J = J0; J < nb; ++J)  // Pb's row pairs with rows i >= c in tile row J0
                    for (int q = r0 >> 1; q < 4; ++q)
                        want.insert({0, pl.tile(J0, J) * 4u + (uint32_t)q});
            }
            std::vector<int> slot_hits((size_t)pl.total, 0);
            std::set<std::pair<int, uint32_t>> got;
            size_t copies = 0;
            for (int lane = 0; lane < 32; ++lane)
                for (IncGroupIter it(pl, lane); it.e < pl.nG; it.next(pl)) {
                    if (it.e < 0 || it.e >= pl.total)
                        return fail(m, c, "phase-1 slot out of range");
                    ++slot_hits[(size_t)it.e];
                    got.insert({it.from_pt(pl) ? 1 : 0, it.unit(pl)});
                    ++copies;
                }
            for (int x = 0; x < pl.n4g + pl.n3g; ++x) {
                bool pt = false;
                const uint32_t u = pl.extra_unit(x, pt);
                ++slot_hits[(size_t)(pl.nG + x)];
                got.insert({pt ? 1 : 0, u});
                ++copies;
            }
            for (int sl = 0; sl < pl.total; ++sl)
                if (slot_hits[(size_t)sl] != 1)
                    return fail(m, c, "a ring slot is not filled exactly once");
            if (copies != got.size())
                return fail(m, c, "a unit is copied twice");
            if (got != want)
                return fail(m, c, "copied units differ from the plan's definition");
            const uint32_t units = (uint32_t)(nb * (nb + 1) / 2) * 4u;
            for (const auto &g : got)
                if (g.second >= units)
                    return fail(m, c, "unit outside the Gram buffer");
            ++checked;
        }
    }
    std::printf("ok: %ld (m, c) plans\n", checked);
    return 0;
}
