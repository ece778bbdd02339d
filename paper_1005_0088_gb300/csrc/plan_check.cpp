// Host-side check of a plan's schedule: every index a kernel will follow stays inside its buffer,
// and no two work items of one launch write overlapping memory (nor does an item write what it
// reads in the same buffer).  The kernels index the fronts and the scratch only through these
// tables, so a plan that passes cannot make them read or write out of bounds or race inside a
// launch.  Cost: linear in the schedule size.
#include <algorithm>
#include <string>
#include <vector>

#include "plan.hpp"

namespace ndsi {

namespace {

// A block of a column-major matrix: rows [r0, r1) x cols [c0, c1) of node `node`'s front (node
// >= 0), or the linear range [r0, r1) of a buffer without node structure (node < 0).
struct Region {
    int32_t node;
    int64_t r0, r1, c0, c1;
};

bool overlap(const Region& a, const Region& b) {
    if (a.node != b.node) return false;
    if (a.node < 0) return a.r0 < b.r1 && b.r0 < a.r1;
    return a.r0 < b.r1 && b.r0 < a.r1 && a.c0 < b.c1 && b.c0 < a.c1;
}

struct Checker {
    const Plan& P;
    std::string& err;
    std::vector<std::pair<int64_t, int32_t>> starts;  // (front_off, node), sorted

    Checker(const Plan& p, std::string& e) : P(p), err(e) {
        for (int32_t j = 0; j < P.n_nodes; ++j) starts.emplace_back(P.front_off[j], j);
        std::sort(starts.begin(), starts.end());
    }

    bool fail(const std::string& msg) {
        err = "plan check: " + msg;
        return false;
    }

    int64_t size_of(int32_t buf) const { return buf == BUF_FRONT ? P.front_total : P.scr_total; }

    // The region an operand of `rows` x `cols` memory elements at `off` with leading dimension
    // `ld` covers in buffer `buf`; false when it leaves the buffer or, in the fronts, its node.
    bool region(int32_t buf, int64_t off, int64_t ld, int64_t rows, int64_t cols, Region& out, const char* what) {
        if (rows <= 0 || cols <= 0) {
            out = Region{-2, 0, 0, 0, 0};
            return true;
        }
        if (off < 0 || ld < rows || off + (rows - 1) + (cols - 1) * ld >= size_of(buf))
            return fail(std::string(what) + " leaves its buffer");
        if (buf != BUF_FRONT) {
            out = Region{-1, off, off + (rows - 1) + (cols - 1) * ld + 1, 0, 0};
            return true;
        }
        auto it = std::upper_bound(starts.begin(), starts.end(), std::make_pair(off, INT32_MAX));
        if (it == starts.begin()) return fail(std::string(what) + " before the first front");
        const int32_t j = std::prev(it)->second;
        const int64_t base = P.front_off[j], f = P.f[j];
        if (ld != f) return fail(std::string(what) + " has a leading dimension other than its front's");
        const int64_t r0 = (off - base) % f, c0 = (off - base) / f;
        if (r0 + rows > f || c0 + cols > f) return fail(std::string(what) + " leaves its front");
        out = Region{j, r0, r0 + rows, c0, c0 + cols};
        return true;
    }

    // Memory extent of op(X) with logical rows x cols.
    static void extent(int32_t op, int64_t rows, int64_t cols, int64_t& mr, int64_t& mc) {
        if (op == OP_N) {
            mr = rows;
            mc = cols;
        } else if (op == OP_T) {
            mr = cols;
            mc = rows;
        } else {  // symmetric, lower triangle: X(r, c) = X[max + min * ld]
            mr = std::max(rows, cols);
            mc = std::min(rows, cols);
        }
    }

    // Writes of one launch: regions in the fronts grouped by node (a launch has at most a few
    // items per node), linear scratch ranges sorted.  They must be pairwise disjoint.
    struct Writes {
        std::vector<std::pair<int32_t, int>> by_node;   // (node, item), sorted
        std::vector<std::pair<Region, int>> linear;     // sorted by start
        const std::vector<Region>* regs = nullptr;
    };

    bool build_writes(const std::vector<Region>& regs, Writes& W, const std::string& what) {
        W.regs = &regs;
        for (int i = 0; i < static_cast<int>(regs.size()); ++i) {
            if (regs[i].node >= 0) W.by_node.emplace_back(regs[i].node, i);
            else if (regs[i].node == -1) W.linear.emplace_back(regs[i], i);
        }
        std::sort(W.by_node.begin(), W.by_node.end());
        std::sort(W.linear.begin(), W.linear.end(),
                  [](const std::pair<Region, int>& a, const std::pair<Region, int>& b) { return a.first.r0 < b.first.r0; });
        for (size_t a = 0; a < W.by_node.size(); ++a)
            for (size_t b = a + 1; b < W.by_node.size() && W.by_node[b].first == W.by_node[a].first; ++b)
                if (overlap(regs[W.by_node[a].second], regs[W.by_node[b].second]))
                    return fail(what + ": two items write overlapping memory");
        for (size_t a = 1; a < W.linear.size(); ++a)
            if (W.linear[a].first.r0 < W.linear[a - 1].first.r1)
                return fail(what + ": two items write overlapping memory");
        return true;
    }

    // Does `r` (read by item `self`) meet a write of another item?
    bool meets(const Writes& W, const Region& r, int self) const {
        if (r.node >= 0) {
            auto it = std::lower_bound(W.by_node.begin(), W.by_node.end(), std::make_pair(r.node, -1));
            for (; it != W.by_node.end() && it->first == r.node; ++it)
                if (it->second != self && overlap(r, (*W.regs)[it->second])) return true;
            return false;
        }
        if (r.node != -1) return false;
        // writes are disjoint and sorted, so their ends are sorted too
        auto it = std::lower_bound(W.linear.begin(), W.linear.end(), r.r0,
                                   [](const std::pair<Region, int>& w, int64_t v) { return w.first.r1 <= v; });
        for (; it != W.linear.end() && it->first.r0 < r.r1; ++it)
            if (it->second != self) return true;
        return false;
    }

    bool run() {
        // node records and index maps
        for (int32_t j = 0; j < P.n_nodes; ++j) {
            const NodeDev& d = P.nodes[j];
            if (d.f != d.s + d.r || d.front_off != P.front_off[j] ||
                d.front_off + static_cast<int64_t>(d.f) * d.f > P.front_total)
                return fail("node " + std::to_string(j) + " front out of range");
            if (d.parent >= 0) {
                const int32_t pf = P.f[d.parent];
                for (int32_t i = 0; i < d.r; ++i) {
                    const int32_t v = P.rel_map[d.rel_off + i];
                    if (v < 0 || v >= pf) return fail("rel_map entry of node " + std::to_string(j) + " out of range");
                }
            }
            for (int t = 0; t < d.nchild; ++t) {
                const int32_t cr = P.r[d.child[t]];
                for (int32_t i = 0; i < d.f; ++i) {
                    const int32_t v = P.inv_map[d.inv_off[t] + i];
                    if (v < -1 || v >= cr) return fail("inv_map entry of node " + std::to_string(j) + " out of range");
                }
            }
        }
        for (int64_t k = 0; k < P.nnz; ++k) {
            if (P.out_map[k] < 0 || P.out_map[k] >= P.front_total) return fail("out_map entry out of range");
            if (P.asm_map[k] < -1 || P.asm_map[k] >= P.front_total) return fail("asm_map entry out of range");
        }
        for (const Launch& l : P.launches) {
            const std::string tag = "launch tag " + std::to_string(l.tag) + " level " + std::to_string(l.level);
            std::vector<Region> writes;
            if (l.kind == L_GEMM) {
                std::vector<Region> As, Bs;
                for (int64_t i = l.first; i < l.first + l.count; ++i) {
                    const GemmItem& g = P.gemm_items[i];
                    int64_t ar, ac, br, bc;
                    extent(l.opA, g.M, g.K, ar, ac);
                    extent(l.opB, g.K, g.N, br, bc);
                    Region A, B, C;
                    if (!region(l.bufA, g.a_off, g.lda, ar, ac, A, "GEMM operand A") ||
                        !region(l.bufB, g.b_off, g.ldb, br, bc, B, "GEMM operand B") ||
                        !region(l.bufC, g.c_off, g.ldc, g.M, g.N, C, "GEMM result"))
                        return fail(err.substr(12) + " (" + tag + ")");
                    if ((l.bufA == l.bufC && overlap(A, C)) || (l.bufB == l.bufC && overlap(B, C)))
                        return fail("a GEMM item writes memory it reads (" + tag + ")");
                    writes.push_back(C);
                    As.push_back(A);
                    Bs.push_back(B);
                }
                for (int64_t t = l.tfirst; t < l.tfirst + l.tcount; ++t) {
                    const GemmTile& gt = P.gemm_tiles[t];
                    if (gt.item < 0 || gt.item >= l.count) return fail("GEMM tile names no item (" + tag + ")");
                    const GemmItem& g = P.gemm_items[l.first + gt.item];
                    if (gt.m0 < 0 || gt.m0 >= g.M || gt.n0 < 0 || gt.n0 >= g.N)
                        return fail("GEMM tile outside its item (" + tag + ")");
                }
                Writes W;
                if (!build_writes(writes, W, tag)) return false;
                for (int i = 0; i < static_cast<int>(writes.size()); ++i)
                    if ((l.bufA == l.bufC && meets(W, As[i], i)) || (l.bufB == l.bufC && meets(W, Bs[i], i)))
                        return fail("a GEMM item reads what another item of the launch writes (" + tag + ")");
            } else if (l.kind == L_COPY) {
                for (int64_t i = l.first; i < l.first + l.count; ++i) {
                    const CopyItem& c = P.copy_items[i];
                    if (static_cast<int64_t>(c.rows) * c.cols >= (int64_t{1} << 31))
                        return fail("copy block of 2^31 or more elements (" + tag + ")");
                    Region S, D;
                    if (!region(BUF_SCR, c.src_off, c.lds, c.rows, c.cols, S, "copy source") ||
                        !region(BUF_FRONT, c.dst_off, c.ldd, c.rows, c.cols, D, "copy destination"))
                        return fail(err.substr(12) + " (" + tag + ")");
                    writes.push_back(D);
                }
                Writes W;
                if (!build_writes(writes, W, tag)) return false;
            } else if (l.kind == L_DIAGINV) {
                // widest block the launch's kernel inverts: warp sweeps of 16 or 32, else the
                // shared-memory kernel of 64
                const int32_t cap = P.block <= 32 ? (l.tile == 16 ? 16 : 32) : 64;
                for (int64_t i = l.first; i < l.first + l.count; ++i) {
                    const DiagItem& d = P.diag_items[i];
                    Region D;
                    if (d.nb <= 0 || d.nb > cap || !region(BUF_FRONT, d.off, d.ld, d.nb, d.nb, D, "pivot block"))
                        return fail("pivot block out of range (" + tag + ")");
                    writes.push_back(D);
                }
                Writes W;
                if (!build_writes(writes, W, tag)) return false;
            } else if (l.kind == L_ASSEMBLE || l.kind == L_GATHER) {
                for (int64_t i = l.first; i < l.first + l.count; ++i) {
                    const NodeTile& t = P.node_tiles[i];
                    if (t.node < 0 || t.node >= P.n_nodes) return fail("node tile names no node (" + tag + ")");
                    const int32_t lim = l.kind == L_ASSEMBLE ? P.f[t.node] : P.r[t.node];
                    if (t.i0 < 0 || t.i0 >= lim || t.j0 < 0 || t.j0 > t.i0)
                        return fail("node tile outside its front (" + tag + ")");
                    if (l.kind == L_GATHER && P.parent[t.node] < 0) return fail("gather tile of the root (" + tag + ")");
                }
            } else if (l.kind == L_SCATTER) {
                for (int64_t i = l.first; i < l.first + l.count; ++i) {
                    const int64_t k = P.scatter_idx[i];
                    if (k < 0 || k >= P.nnz || P.asm_map[k] < 0) return fail("scatter entry out of range (" + tag + ")");
                }
            }
        }
        return true;
    }
};

}  // namespace

int check_plan(const Plan& P, std::string& err) {
    Checker c(P, err);
    return c.run() ? NDSI_OK : NDSI_ERR_INVALID;
}

}  // namespace ndsi
