// Host check of the band kernel's triangle items (tri_range in
// ozaki_common.cuh): for every geometry, the compact enumeration through the
// cumulative table and a binary search yields exactly the tiles the raster
// keeps when it skips the tiles outside the triangle, in the same order.
// Prints "cases N bad B".
#include <cstdio>
#include <vector>

#include "ozaki_common.cuh"

using namespace mpdd;

// The raster of the band kernel: groups of group_n tile columns, rows
// within a group, columns within a row.
static void raster(int tile, int units, int tiles_n, int group_n, int &u, int &tn) {
    const int group = tile / (units * group_n), first = group * group_n;
    const int gn = tiles_n - first < group_n ? tiles_n - first : group_n;
    const int local = tile - group * units * group_n;
    tn = first + local % gn;
    u = local / gn;
}

int main() {
    const int TM = 128;
    int bad = 0, cases = 0;
    for (int tri = 1; tri <= 2; ++tri)
        for (int pair = 0; pair <= 1; ++pair)
            for (int TN : {128, 256})
                for (int tiles_m = 1; tiles_m <= 40; ++tiles_m)
                    for (int tiles_n = 1; tiles_n <= 24; ++tiles_n) {
                        if (pair && (TN != 256 || tiles_m % 2)) continue;
                        const int units = pair ? tiles_m / 2 : tiles_m, R = pair ? 2 * TM : TM;
                        std::vector<int> ru, rt;
                        for (int t = 0; t < units * tiles_n; ++t) {
                            int u, tn;
                            raster(t, units, tiles_n, 4, u, tn);
                            const long long r0 = (long long)u * R, c0 = (long long)tn * TN;
                            const bool skip = (tri == 1 && r0 > c0 + TN - 1) ||
                                              (tri == 2 && r0 + R - 1 < c0);
                            if (!skip) {
                                ru.push_back(u);
                                rt.push_back(tn);
                            }
                        }
                        const TriGeom g{tri, R, TN, tiles_n, 4};
                        const int rows = ((tiles_n + 3) / 4) * units;
                        std::vector<int> cum(rows + 1);
                        int run = 0;
                        for (int x = 0; x < rows; ++x) {
                            cum[x] = run;
                            int lo, hi;
                            tri_range(g, x / units, x % units, lo, hi);
                            run += hi >= lo ? hi - lo + 1 : 0;
                        }
                        cum[rows] = run;
                        ++cases;
                        if (run != (int)ru.size()) {
                            ++bad;
                            continue;
                        }
                        for (int tile = 0; tile < run; ++tile) {
                            int lo = 0, hi = rows;
                            while (hi - lo > 1) {
                                const int mid = (lo + hi) >> 1;
                                if (cum[mid] <= tile) lo = mid;
                                else hi = mid;
                            }
                            const int grp = lo / units, u = lo - grp * units;
                            int clo, chi;
                            tri_range(g, grp, u, clo, chi);
                            if (u != ru[tile] || clo + (tile - cum[lo]) != rt[tile]) {
                                ++bad;
                                break;
                            }
                        }
                    }
    printf("cases %d bad %d\n", cases, bad);
    return bad != 0;
}
