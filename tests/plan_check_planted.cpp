// Planted mistakes for the schedule check: a plan built by the host analysis passes, and each
// corruption below (an index out of its buffer, two items writing the same block, an index map
// entry outside the parent front, a tile outside its item, a diagonal block wider than its
// kernel) is reported.  Prints one line per
// case; exits non-zero if a corruption goes unnoticed or the clean plan fails.
#include <algorithm>
#include <cstdio>
#include <string>
#include <vector>

#include "plan.hpp"

namespace ndsi {
void set_last_error(const std::string&) {}
}  // namespace ndsi

int main() {
    // a 2D sheet of 10 x 8 atoms, 2 orbitals each, nearest and next-nearest neighbours
    const int nx = 10, ny = 8, o = 2, na = nx * ny, n = na * o;
    std::vector<std::vector<int>> nbr(na);
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int x2 = x + dx, y2 = y + dy;
                    if (x2 >= 0 && x2 < nx && y2 >= 0 && y2 < ny) nbr[x + nx * y].push_back(x2 + nx * y2);
                }
    std::vector<int64_t> rowptr(1, 0);
    std::vector<int32_t> col;
    for (int i = 0; i < n; ++i) {
        std::vector<int> cs;
        for (int b : nbr[i / o])
            for (int q = 0; q < o; ++q) cs.push_back(b * o + q);
        std::sort(cs.begin(), cs.end());
        for (int c : cs) col.push_back(c);
        rowptr.push_back(static_cast<int64_t>(col.size()));
    }
    std::vector<double> centers(3 * na, 0.0);
    for (int a = 0; a < na; ++a) {
        centers[3 * a] = a % nx;
        centers[3 * a + 1] = a / nx;
    }
    std::vector<int32_t> aob(n);
    for (int i = 0; i < n; ++i) aob[i] = i / o;
    ndsi_pattern pat{n, rowptr.data(), col.data()};
    ndsi_options opt{};
    opt.leaf_atoms = 6;
    opt.block = 16;
    opt.outer_block = 32;
    opt.m0_radius = 1e7;
    ndsi::Plan P;
    std::string err;
    if (ndsi::analyze(&pat, na, centers.data(), aob.data(), opt, P, err)) {
        std::printf("analyze failed: %s\n", err.c_str());
        return 2;
    }
    int bad = 0;
    auto expect = [&](const char* what, bool want_ok) {
        std::string e;
        const bool ok = ndsi::check_plan(P, e) == NDSI_OK;
        std::printf("%-40s %s %s\n", what, ok ? "passes" : "rejected:", e.c_str());
        if (ok != want_ok) ++bad;
    };
    expect("clean plan", true);
    // 1. a GEMM result beyond the end of its buffer
    const int64_t save_off = P.gemm_items[0].c_off;
    P.gemm_items[0].c_off = 1LL << 40;
    expect("GEMM result out of its buffer", false);
    P.gemm_items[0].c_off = save_off;
    // 2. two items of one GEMM launch writing the same block: two items of equal shape, the
    // second made to write where the first writes (every bound still holds)
    bool planted = false;
    for (const ndsi::Launch& l : P.launches) {
        if (l.kind != ndsi::L_GEMM || planted) continue;
        for (int64_t i = l.first; i < l.first + l.count && !planted; ++i)
            for (int64_t k = i + 1; k < l.first + l.count && !planted; ++k) {
                ndsi::GemmItem& a = P.gemm_items[i];
                ndsi::GemmItem& b = P.gemm_items[k];
                if (a.M != b.M || a.N != b.N || a.K != b.K || a.ldc != b.ldc || a.c_off == b.c_off) continue;
                const int64_t keep = b.c_off;
                b.c_off = a.c_off;
                expect("two items writing one block", false);
                b.c_off = keep;
                planted = true;
            }
    }
    if (!planted) ++bad;
    expect("clean plan again", true);
    // 3. an index-map entry outside the parent's front
    for (int32_t j = 0; j < P.n_nodes; ++j) {
        if (P.parent[j] < 0 || P.r[j] == 0) continue;
        const int32_t keep = P.rel_map[P.nodes[j].rel_off];
        P.rel_map[P.nodes[j].rel_off] = P.f[P.parent[j]];
        expect("rel_map entry outside the parent", false);
        P.rel_map[P.nodes[j].rel_off] = keep;
        break;
    }
    // 4. a GEMM tile outside its item
    {
        const int32_t keep = P.gemm_tiles[0].m0;
        P.gemm_tiles[0].m0 = 1 << 20;
        expect("GEMM tile outside its item", false);
        P.gemm_tiles[0].m0 = keep;
    }
    // 5. a diagonal block wider than the kernel its launch selects
    planted = false;
    for (const ndsi::Launch& l : P.launches) {
        if (l.kind != ndsi::L_DIAGINV || planted) continue;
        ndsi::DiagItem& d = P.diag_items[l.first];
        const int32_t keep = d.nb;
        d.nb = l.tile + 1;
        expect("diagonal block wider than its kernel", false);
        d.nb = keep;
        planted = true;
    }
    if (!planted) ++bad;
    expect("clean plan at the end", true);
    return bad ? 1 : 0;
}
