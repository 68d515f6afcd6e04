// Host-side check of the force-region tile enumeration (for_each_tile in
// csrc/internal.cuh): for every node box of width 1..7 on small periodic and
// bounded lattices and every tile shape, the visited tiles must be exactly
// the tiles that hold a node of the box (brute force over the wrapped
// nodes). Built and run by tests/test_tiles.py; prints "ok" or the first
// mismatch.
#include <cstdio>
#include <set>

#include "../paper_2003_03130_gb300/csrc/internal.cuh"

using namespace cf;

int main() {
    const int shapes[4][3] = {{4, 2, 2}, {5, 2, 1}, {5, 1, 2}, {3, 3, 2}};
    const int sizes[] = {1, 3, 8, 17, 20, 40};
    long long cases = 0;
    for (const auto &sh : shapes)
        for (int nx : sizes)
            for (int ny : sizes)
                for (int nz : {1, 9}) {
                    LbmParams p{};
                    p.nx = nx;
                    p.ny = ny;
                    p.nz = nz;
                    p.tlx = sh[0];
                    p.tly = sh[1];
                    p.tlz = sh[2];
                    p.ntx = (nx + (1 << p.tlx) - 1) >> p.tlx;
                    p.nty = (ny + (1 << p.tly) - 1) >> p.tly;
                    p.ntz = (nz + (1 << p.tlz) - 1) >> p.tlz;
                    for (int w = 1; w <= 7; ++w)
                        for (int x0 = -9; x0 <= nx + 2; ++x0)
                            for (int y0 = 0; y0 < ny; ++y0)
                                for (int z0 = -3; z0 <= nz; z0 += 2) {
                                    const int x1 = x0 + w - 1, z1 = z0 + w - 1;
                                    const int y1 = y0 + w - 1 < ny ? y0 + w - 1 : ny - 1;
                                    std::set<int> want, got;
                                    for (int z = z0; z <= z1; ++z)
                                        for (int y = y0; y <= y1; ++y)
                                            for (int x = x0; x <= x1; ++x)
                                                want.insert(tile_index(p, wrapi(x, nx) >> p.tlx, y >> p.tly,
                                                                       wrapi(z, nz) >> p.tlz));
                                    bool in_range = true;
                                    for_each_tile(p, x0, x1, y0, y1, z0, z1, [&](int t) {
                                        if (t < 0 || t >= p.ntx * p.nty * p.ntz) in_range = false;
                                        got.insert(t);
                                    });
                                    ++cases;
                                    if (!in_range || want != got) {
                                        std::printf("mismatch: n=%d,%d,%d tile=%d,%d,%d box x[%d,%d] y[%d,%d] z[%d,%d]\n",
                                                    nx, ny, nz, sh[0], sh[1], sh[2], x0, x1, y0, y1, z0, z1);
                                        return 1;
                                    }
                                }
                }
    std::printf("ok %lld\n", cases);
    return 0;
}
