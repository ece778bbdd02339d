// Host analysis: geometric nested dissection (Sec. II.C.1), the supernodal structure and every
// index table of the numeric phase (the "table function" of Sec. II.C.2), the per-level launch
// schedule, and the continued-fraction poles of Eq. 7.  Integer work only (plus the poles).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <numeric>
#include <utility>

#include "plan.hpp"

namespace ndsi {

namespace {

struct Dissector {
    int32_t na;
    const double* centers;
    const std::vector<std::vector<int32_t>>& adj;
    int32_t leaf_atoms;
    double cell[3];               // periodic cell length per axis (0 = open)
    std::vector<int32_t> ord_of;  // atom -> ordering number in the current domain (0 = outside)
    std::vector<double> xw;       // coordinate along the current axis, wrapped into [0, L)
    // output tree (postorder)
    std::vector<std::vector<int32_t>> nodes;
    std::vector<int32_t> child0, child1;

    Dissector(int32_t n, const double* c, const std::vector<std::vector<int32_t>>& a, int32_t leaf,
              const double* cell_len)
        : na(n), centers(c), adj(a), leaf_atoms(leaf), ord_of(n, 0), xw(n, 0.0) {
        for (int k = 0; k < 3; ++k) cell[k] = cell_len[k] > 0 ? cell_len[k] : 0.0;
    }

    // Best split of D (steps i, iii, iv, v).  Returns false for a leaf.
    bool split(const std::vector<int32_t>& D, std::vector<int32_t>& sub0, std::vector<int32_t>& sub1,
               std::vector<int32_t>& sep) {
        const int32_t Nd = static_cast<int32_t>(D.size());
        if (Nd <= leaf_atoms) return false;
        bool have = false;
        int64_t best_meas = 0, best_ns = 0;
        int32_t b_mmin = 0, b_mmax = 0, b_nmin = 0, b_nmax = 0;
        std::vector<int32_t> best_order, order(D);
        for (int axis = 0; axis < 3; ++axis) {
            // (i) ordering numbers along the axis: (coordinate, atom index); on a periodic axis the
            // coordinate is wrapped into the central cell [0, L)
            const double L = cell[axis];
            for (int32_t a : D) {
                const double c = centers[3 * static_cast<int64_t>(a) + axis];
                xw[a] = L > 0 ? c - L * std::floor(c / L) : c;
            }
            order = D;
            std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
                if (xw[a] != xw[b]) return xw[a] < xw[b];
                return a < b;
            });
            for (int32_t i = 0; i < Nd; ++i) ord_of[order[i]] = i + 1;
            // (iii) nucleus: fewest adjacent atoms inside the domain, then lowest ordering number
            int32_t nucleus = -1, nbest = 0;
            for (int32_t i = 0; i < Nd; ++i) {
                const int32_t a = order[i];
                int32_t cnt = 0;
                for (int32_t b : adj[a]) cnt += ord_of[b] > 0;
                if (nucleus < 0 || cnt < nbest) {
                    nucleus = a;
                    nbest = cnt;
                }
            }
            // ordering numbers of the neighbours; on a periodic axis the neighbour's image nearest
            // the atom, l = -floor(dx/L + 1/2) cells away, has ordering number ord + l*Nd
            auto span = [&](int32_t atom, int32_t& lo, int32_t& hi) {
                for (int32_t b : adj[atom]) {
                    int32_t o = ord_of[b];
                    if (o > 0) {
                        if (L > 0) o -= static_cast<int32_t>(std::floor((xw[b] - xw[atom]) / L + 0.5)) * Nd;
                        lo = std::min(lo, o);
                        hi = std::max(hi, o);
                    }
                }
            };
            const int32_t q = ord_of[nucleus];
            int32_t m_min = q, m_max = q, n_min = q, n_max = q;
            span(nucleus, n_min, n_max);
            bool ahave = false;
            int64_t a_meas = 0, a_ns = 0;
            int32_t a_mmin = 0, a_mmax = 0, a_nmin = 0, a_nmax = 0;
            auto consider = [&]() {
                const int64_t N0 = m_max - m_min + 1;
                const int64_t Ns = n_max - n_min + 1 - N0;
                const int64_t N1 = Nd - N0 - Ns;
                if (N1 >= 1) {
                    const int64_t meas = std::llabs(N0 - N1) + Ns;
                    if (!ahave || meas < a_meas || (meas == a_meas && Ns <= a_ns)) {
                        ahave = true;
                        a_meas = meas;
                        a_ns = Ns;
                        a_mmin = m_min; a_mmax = m_max; a_nmin = n_min; a_nmax = n_max;
                    }
                }
            };
            consider();
            // (iv) growth of the nucleus
            while (m_max - m_min + 1 < Nd) {
                bool has_up = false, has_dn = false;
                int64_t up_meas = 0, dn_meas = 0;
                int32_t up_lo = 0, up_hi = 0, dn_lo = 0, dn_hi = 0;
                const int64_t N0 = m_max - m_min + 2;
                if (m_max < Nd) {
                    up_lo = std::min(n_min, m_max + 1);
                    up_hi = std::max(n_max, m_max + 1);
                    span(order[m_max], up_lo, up_hi);
                    const int64_t Ns = up_hi - up_lo + 1 - N0;
                    up_meas = std::llabs(N0 - (Nd - N0 - Ns)) + Ns;
                    has_up = true;
                }
                if (m_min > 1) {
                    dn_lo = std::min(n_min, m_min - 1);
                    dn_hi = std::max(n_max, m_min - 1);
                    span(order[m_min - 2], dn_lo, dn_hi);
                    const int64_t Ns = dn_hi - dn_lo + 1 - N0;
                    dn_meas = std::llabs(N0 - (Nd - N0 - Ns)) + Ns;
                    has_dn = true;
                }
                if (has_up && (!has_dn || up_meas <= dn_meas)) {
                    m_max += 1;
                    n_min = up_lo;
                    n_max = up_hi;
                } else {
                    m_min -= 1;
                    n_min = dn_lo;
                    n_max = dn_hi;
                }
                consider();
            }
            for (int32_t i = 0; i < Nd; ++i) ord_of[order[i]] = 0;
            // (v) axis choice: smallest (measure, Ns), ties to the lowest axis
            if (ahave && (!have || a_meas < best_meas || (a_meas == best_meas && a_ns < best_ns))) {
                have = true;
                best_meas = a_meas;
                best_ns = a_ns;
                b_mmin = a_mmin; b_mmax = a_mmax; b_nmin = a_nmin; b_nmax = a_nmax;
                best_order = order;
            }
        }
        if (!have) return false;
        // subdomain 0 = [m_min, m_max]; separator = [n_min, n_max] minus subdomain 0, modulo Nd
        // (periodic axes can reach below 1 and above Nd); subdomain 1 = the rest
        std::vector<char> role(Nd, 1);
        for (int32_t x = b_mmin; x <= b_mmax; ++x) role[x - 1] = 0;
        for (int32_t x = b_nmin; x <= b_nmax; ++x)
            if (x < b_mmin || x > b_mmax) role[((x - 1) % Nd + Nd) % Nd] = 2;
        sub0.clear();
        sub1.clear();
        sep.clear();
        for (int32_t i = 0; i < Nd; ++i) (role[i] == 0 ? sub0 : role[i] == 1 ? sub1 : sep).push_back(best_order[i]);
        std::sort(sub0.begin(), sub0.end());
        std::sort(sub1.begin(), sub1.end());
        std::sort(sep.begin(), sep.end());
        return true;
    }

    // `extra` (the screened long-tail atoms, root only) joins the domain's separator, or the
    // domain itself when it is a leaf
    int32_t rec(std::vector<int32_t> D, const std::vector<int32_t>& extra = {}) {
        std::vector<int32_t> s0, s1, sp;
        if (!split(D, s0, s1, sp)) {
            D.insert(D.end(), extra.begin(), extra.end());
            std::sort(D.begin(), D.end());
            nodes.push_back(std::move(D));
            child0.push_back(-1);
            child1.push_back(-1);
            return static_cast<int32_t>(nodes.size()) - 1;
        }
        D.clear();
        D.shrink_to_fit();
        const int32_t c0 = rec(std::move(s0));
        const int32_t c1 = rec(std::move(s1));
        sp.insert(sp.end(), extra.begin(), extra.end());
        std::sort(sp.begin(), sp.end());
        nodes.push_back(std::move(sp));
        child0.push_back(c0);
        child1.push_back(c1);
        return static_cast<int32_t>(nodes.size()) - 1;
    }
};

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

int analyze(const ndsi_pattern* pat, int32_t n_atoms, const double* centers,
            const int32_t* atom_of_basis, const ndsi_options& opt, Plan& P, std::string& err) {
    if (!pat || !pat->rowptr || !pat->col || !centers || !atom_of_basis || pat->n <= 0 ||
        n_atoms <= 0) {
        err = "ndsi_analyze: null pointer or empty problem";
        return NDSI_ERR_INVALID;
    }
    if (pat->n > (int64_t(1) << 31) - 1) {
        err = "ndsi_analyze: n exceeds int32 indexing";
        return NDSI_ERR_INVALID;
    }
    const int64_t n = pat->n;
    const int64_t nnz = pat->rowptr[n];
    if (pat->rowptr[0] != 0 || nnz <= 0) {
        err = "ndsi_analyze: rowptr[0] must be 0 and nnz > 0";
        return NDSI_ERR_INVALID;
    }
    P.n = n;
    P.nnz = nnz;
    P.n_atoms = n_atoms;
    P.opt = opt;
    P.block = opt.block > 0 ? opt.block : 16;
    if (P.block != 16 && P.block != 32 && P.block != 64) {
        err = "ndsi_analyze: block must be 16, 32 or 64";
        return NDSI_ERR_INVALID;
    }
    P.outer = opt.outer_block > 0 ? opt.outer_block : 128;
    if (P.outer % P.block != 0 || P.outer > 4096) {
        err = "ndsi_analyze: outer_block must be a multiple of block, at most 4096";
        return NDSI_ERR_INVALID;
    }
    P.rowptr.assign(pat->rowptr, pat->rowptr + n + 1);
    P.col.assign(pat->col, pat->col + nnz);
    // ---- pattern checks: monotone rows, sorted columns, diagonal present, symmetric
    for (int64_t i = 0; i < n; ++i) {
        const int64_t a = P.rowptr[i], b = P.rowptr[i + 1];
        if (b < a) {
            err = "ndsi_analyze: rowptr not monotone";
            return NDSI_ERR_INVALID;
        }
        bool diag = false;
        for (int64_t k = a; k < b; ++k) {
            const int32_t j = P.col[k];
            if (j < 0 || j >= n || (k > a && P.col[k - 1] >= j)) {
                err = "ndsi_analyze: column index out of range or unsorted in row " + std::to_string(i);
                return NDSI_ERR_INVALID;
            }
            diag |= (j == i);
        }
        if (!diag) {
            err = "ndsi_analyze: missing diagonal in row " + std::to_string(i);
            return NDSI_ERR_INVALID;
        }
    }
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t k = P.rowptr[i]; k < P.rowptr[i + 1]; ++k) {
            const int32_t j = P.col[k];
            const int32_t* b = P.col.data() + P.rowptr[j];
            const int32_t* e = P.col.data() + P.rowptr[j + 1];
            if (!std::binary_search(b, e, static_cast<int32_t>(i))) {
                err = "ndsi_analyze: pattern is not symmetric at (" + std::to_string(i) + "," +
                      std::to_string(j) + ")";
                return NDSI_ERR_INVALID;
            }
        }
    }
    // ---- atoms: basis lists and adjacency
    std::vector<std::vector<int32_t>> atom_basis(n_atoms);
    for (int64_t i = 0; i < n; ++i) {
        const int32_t a = atom_of_basis[i];
        if (a < 0 || a >= n_atoms) {
            err = "ndsi_analyze: atom_of_basis out of range";
            return NDSI_ERR_INVALID;
        }
        atom_basis[a].push_back(static_cast<int32_t>(i));
    }
    for (int32_t a = 0; a < n_atoms; ++a) {
        if (atom_basis[a].empty()) {
            err = "ndsi_analyze: atom " + std::to_string(a) + " owns no basis function";
            return NDSI_ERR_INVALID;
        }
    }
    std::vector<std::vector<int32_t>> adj(n_atoms);
    {
        std::vector<int32_t> stamp(n_atoms, -1);
        for (int32_t a = 0; a < n_atoms; ++a) {
            for (int32_t i : atom_basis[a]) {
                for (int64_t k = P.rowptr[i]; k < P.rowptr[i + 1]; ++k) {
                    const int32_t b = atom_of_basis[P.col[k]];
                    if (b != a && stamp[b] != a) {
                        stamp[b] = a;
                        adj[a].push_back(b);
                    }
                }
            }
            std::sort(adj[a].begin(), adj[a].end());
        }
    }
    // ---- nested dissection
    const int32_t leaf = opt.leaf_atoms > 0 ? opt.leaf_atoms : 20;
    for (int k = 0; k < 3; ++k)
        if (!(opt.cell[k] >= 0) || !std::isfinite(opt.cell[k])) {
            err = "ndsi_analyze: cell lengths must be finite and >= 0";
            return NDSI_ERR_INVALID;
        }
    if (opt.screen_degree < 0) {
        err = "ndsi_analyze: screen_degree must be >= 0";
        return NDSI_ERR_INVALID;
    }
    Dissector dis(n_atoms, centers, adj, leaf, opt.cell);
    {
        // (ii) long-tail screening: atoms adjacent to more than screen_degree atoms go to the
        // root separator and take no part in the dissection
        std::vector<int32_t> kept, screened;
        for (int32_t a = 0; a < n_atoms; ++a)
            (opt.screen_degree > 0 && static_cast<int32_t>(adj[a].size()) > opt.screen_degree ? screened : kept)
                .push_back(a);
        dis.rec(std::move(kept), screened);
    }
    const int32_t nn = static_cast<int32_t>(dis.nodes.size());
    P.n_nodes = nn;
    P.child0 = dis.child0;
    P.child1 = dis.child1;
    P.parent.assign(nn, -1);
    P.nchild.assign(nn, 0);
    for (int32_t j = 0; j < nn; ++j) {
        if (P.child0[j] >= 0) {
            P.parent[P.child0[j]] = j;
            P.parent[P.child1[j]] = j;
            P.nchild[j] = 2;
        }
    }
    P.node_atom_first.assign(nn + 1, 0);
    P.perm_atoms.clear();
    for (int32_t j = 0; j < nn; ++j) {
        P.node_atom_first[j] = static_cast<int32_t>(P.perm_atoms.size());
        P.perm_atoms.insert(P.perm_atoms.end(), dis.nodes[j].begin(), dis.nodes[j].end());
    }
    P.node_atom_first[nn] = n_atoms;
    std::vector<int32_t> apos(n_atoms);
    for (int32_t k = 0; k < n_atoms; ++k) apos[P.perm_atoms[k]] = k;
    // basis order: atoms in structured order, basis functions of an atom ascending
    P.perm_basis.clear();
    P.node_first.assign(nn + 1, 0);
    for (int32_t j = 0; j < nn; ++j) {
        P.node_first[j] = static_cast<int32_t>(P.perm_basis.size());
        for (int32_t t = P.node_atom_first[j]; t < P.node_atom_first[j + 1]; ++t) {
            const auto& bl = atom_basis[P.perm_atoms[t]];
            P.perm_basis.insert(P.perm_basis.end(), bl.begin(), bl.end());
        }
    }
    P.node_first[nn] = static_cast<int32_t>(n);
    P.ipos_basis.assign(n, 0);
    for (int64_t k = 0; k < n; ++k) P.ipos_basis[P.perm_basis[k]] = static_cast<int32_t>(k);
    std::vector<int32_t> atom_first_pos(n_atoms);  // first structured basis position of an atom
    {
        int32_t pos = 0;
        for (int32_t k = 0; k < n_atoms; ++k) {
            atom_first_pos[P.perm_atoms[k]] = pos;
            pos += static_cast<int32_t>(atom_basis[P.perm_atoms[k]].size());
        }
    }
    // ---- symbolic structure (atoms): struct(J) = (adj(J) U struct(children)) beyond J
    {
        std::vector<std::vector<int32_t>> st(nn);
        std::vector<int32_t> stamp(n_atoms, -1);
        for (int32_t j = 0; j < nn; ++j) {
            std::vector<int32_t>& tmp = st[j];
            const int32_t last = P.node_atom_first[j + 1] - 1;
            auto add = [&](int32_t b) {
                if (apos[b] > last && stamp[b] != j) {
                    stamp[b] = j;
                    tmp.push_back(b);
                }
            };
            for (int32_t t = P.node_atom_first[j]; t <= last; ++t)
                for (int32_t b : adj[P.perm_atoms[t]]) add(b);
            for (int32_t c : {P.child0[j], P.child1[j]}) {
                if (c < 0) continue;
                for (int32_t b : st[c]) add(b);
            }
            std::sort(tmp.begin(), tmp.end(), [&](int32_t a, int32_t b) { return apos[a] < apos[b]; });
        }
        P.struct_ptr.assign(nn + 1, 0);
        P.struct_atoms.clear();
        for (int32_t j = 0; j < nn; ++j) {
            P.struct_ptr[j] = static_cast<int64_t>(P.struct_atoms.size());
            P.struct_atoms.insert(P.struct_atoms.end(), st[j].begin(), st[j].end());
        }
        P.struct_ptr[nn] = static_cast<int64_t>(P.struct_atoms.size());
    }
    // struct in basis positions
    P.sstruct_ptr.assign(nn + 1, 0);
    P.struct_basis.clear();
    for (int32_t j = 0; j < nn; ++j) {
        P.sstruct_ptr[j] = static_cast<int64_t>(P.struct_basis.size());
        for (int64_t q = P.struct_ptr[j]; q < P.struct_ptr[j + 1]; ++q) {
            const int32_t a = P.struct_atoms[q];
            const int32_t p0 = atom_first_pos[a];
            for (size_t t = 0; t < atom_basis[a].size(); ++t)
                P.struct_basis.push_back(p0 + static_cast<int32_t>(t));
        }
    }
    P.sstruct_ptr[nn] = static_cast<int64_t>(P.struct_basis.size());
    // ---- levels, fronts
    P.level.assign(nn, 0);
    for (int32_t j = 0; j < nn; ++j) {
        if (P.child0[j] >= 0) P.level[j] = 1 + std::max(P.level[P.child0[j]], P.level[P.child1[j]]);
    }
    P.n_levels = 1 + *std::max_element(P.level.begin(), P.level.end());
    P.level_nodes.assign(P.n_levels, {});
    for (int32_t j = 0; j < nn; ++j) P.level_nodes[P.level[j]].push_back(j);
    P.f.assign(nn, 0);
    P.s.assign(nn, 0);
    P.r.assign(nn, 0);
    P.front_off.assign(nn, 0);
    int64_t off = 0;
    P.max_front = 0;
    for (int32_t j = 0; j < nn; ++j) {
        P.s[j] = P.node_first[j + 1] - P.node_first[j];
        P.r[j] = static_cast<int32_t>(P.sstruct_ptr[j + 1] - P.sstruct_ptr[j]);
        P.f[j] = P.s[j] + P.r[j];
        P.front_off[j] = off;
        off += static_cast<int64_t>(P.f[j]) * P.f[j];
        P.max_front = std::max(P.max_front, P.f[j]);
    }
    P.front_total = std::max<int64_t>(off, 1);
    compute_scratch(P);
    // ---- rel / inv maps
    std::vector<int32_t> node_of_pos(n);
    for (int32_t j = 0; j < nn; ++j)
        for (int32_t p = P.node_first[j]; p < P.node_first[j + 1]; ++p) node_of_pos[p] = j;
    auto struct_index = [&](int32_t j, int32_t g) -> int32_t {
        const int32_t* bgn = P.struct_basis.data() + P.sstruct_ptr[j];
        const int32_t* end = P.struct_basis.data() + P.sstruct_ptr[j + 1];
        const int32_t* it = std::lower_bound(bgn, end, g);
        if (it == end || *it != g) return -1;
        return static_cast<int32_t>(it - bgn);
    };
    P.rel_map.clear();
    P.inv_map.clear();
    P.nodes.assign(nn, NodeDev{});
    std::vector<int64_t> rel_off(nn, -1);
    for (int32_t j = 0; j < nn; ++j) {
        const int32_t p = P.parent[j];
        if (p < 0) continue;
        rel_off[j] = static_cast<int64_t>(P.rel_map.size());
        for (int64_t q = P.sstruct_ptr[j]; q < P.sstruct_ptr[j + 1]; ++q) {
            const int32_t g = P.struct_basis[q];
            int32_t loc;
            if (g >= P.node_first[p] && g < P.node_first[p + 1]) {
                loc = g - P.node_first[p];
            } else {
                const int32_t t = struct_index(p, g);
                if (t < 0) {
                    err = "ndsi_analyze: elimination-tree containment violated";
                    return NDSI_ERR_INVALID;
                }
                loc = P.s[p] + t;
            }
            P.rel_map.push_back(loc);
        }
    }
    for (int32_t j = 0; j < nn; ++j) {
        NodeDev& d = P.nodes[j];
        d.front_off = P.front_off[j];
        d.f = P.f[j];
        d.s = P.s[j];
        d.r = P.r[j];
        d.nchild = P.nchild[j];
        d.child[0] = P.child0[j];
        d.child[1] = P.child1[j];
        d.parent = P.parent[j];
        d.level = P.level[j];
        d.rel_off = rel_off[j];
        d.inv_off[0] = d.inv_off[1] = -1;
        for (int t = 0; t < d.nchild; ++t) {
            const int32_t c = d.child[t];
            d.inv_off[t] = static_cast<int64_t>(P.inv_map.size());
            P.inv_map.resize(P.inv_map.size() + P.f[j], -1);
            int32_t* inv = P.inv_map.data() + d.inv_off[t];
            for (int32_t i = 0; i < P.r[c]; ++i) inv[P.rel_map[rel_off[c] + i]] = i;
        }
    }
    if (P.rel_map.empty()) P.rel_map.push_back(0);
    if (P.inv_map.empty()) P.inv_map.push_back(-1);
    // ---- assembly and output maps
    P.asm_map.assign(nnz, -1);
    P.out_map.assign(nnz, -1);
    P.level_entries.assign(P.n_levels, {});
    auto& lvl_entries = P.level_entries;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t k = P.rowptr[i]; k < P.rowptr[i + 1]; ++k) {
            const int32_t gi = P.ipos_basis[i];
            const int32_t gj = P.ipos_basis[P.col[k]];
            const int32_t I = node_of_pos[gi], J = node_of_pos[gj];
            auto lower_off = [&](int32_t node, int32_t row, int32_t colx) {
                return P.front_off[node] + row + static_cast<int64_t>(colx) * P.f[node];
            };
            if (I == J) {
                const int32_t a = std::max(gi, gj) - P.node_first[J];
                const int32_t c = std::min(gi, gj) - P.node_first[J];
                P.out_map[k] = lower_off(J, a, c);
                if (gi >= gj) P.asm_map[k] = P.out_map[k];
            } else if (gi > gj) {
                const int32_t t = struct_index(J, gi);
                if (t < 0) {
                    err = "ndsi_analyze: pattern entry outside struct (separator property violated)";
                    return NDSI_ERR_INVALID;
                }
                P.out_map[k] = lower_off(J, P.s[J] + t, gj - P.node_first[J]);
                P.asm_map[k] = P.out_map[k];
            } else {
                const int32_t t = struct_index(I, gj);
                if (t < 0) {
                    err = "ndsi_analyze: pattern entry outside struct (separator property violated)";
                    return NDSI_ERR_INVALID;
                }
                P.out_map[k] = lower_off(I, P.s[I] + t, gi - P.node_first[I]);
            }
            if (P.asm_map[k] >= 0) lvl_entries[P.level[J]].push_back(k);
        }
    }
    P.n_systems = 1;
    P.sys_nnz_first = {0, nnz};
    P.sys_n_first = {0, n};
    P.entry_sys.assign(nnz, 0);
    build_schedule(P);
    return NDSI_OK;
}

void compute_scratch(Plan& P) {
    const int32_t b = P.block;
    P.scr_off.assign(P.n_nodes, 0);
    P.scr_total = 1;
    for (int32_t L = 0; L < P.n_levels; ++L) {
        int64_t acc = 0;
        for (int32_t j : P.level_nodes[L]) {
            P.scr_off[j] = acc;
            const int64_t need = std::max<int64_t>(static_cast<int64_t>(P.s[j]) * std::max(b, std::min(P.outer, P.s[j])),
                                                   static_cast<int64_t>(P.r[j]) * P.s[j]);
            acc += need;
        }
        P.scr_total = std::max(P.scr_total, acc);
    }
}

// Per-level launch schedule of the factor (bottom-up) and the selected inversion (top-down),
// from the node structure of a plan (one system or several merged level by level).
void build_schedule(Plan& P) {
    const int32_t b = P.block;
    const auto& lvl_entries = P.level_entries;
    P.launches.clear();
    P.gemm_items.clear();
    P.gemm_tiles.clear();
    P.copy_items.clear();
    P.diag_items.clear();
    P.node_tiles.clear();
    P.scatter_idx.clear();
    P.flops_per_pole = 0;
    P.bytes_per_pole = 0;
    auto new_launch = [&](int32_t kind, int32_t L, int32_t phase, int32_t tag) {
        Launch l{};
        l.kind = kind;
        l.level = L;
        l.phase = phase;
        l.tag = tag;
        return l;
    };
    struct GSpec {
        int64_t a_off, b_off, c_off;
        int32_t lda, ldb, ldc, M, N, K;
    };
    auto emit_gemm = [&](int32_t L, int32_t phase, int32_t tag, int32_t opA, int32_t opB,
                         int32_t bufA, int32_t bufB, int32_t bufC, double alpha, double beta,
                         bool lower, const std::vector<GSpec>& specs, bool exact = false) {
        if (specs.empty()) return;
        Launch l = new_launch(L_GEMM, L, phase, tag);
        l.exact = exact ? 1 : 0;
        l.opA = opA; l.opB = opB; l.bufA = bufA; l.bufB = bufB; l.bufC = bufC;
        l.alpha = alpha; l.beta = beta; l.lower = lower ? 1 : 0;
        l.first = static_cast<int64_t>(P.gemm_items.size());
        l.tfirst = static_cast<int64_t>(P.gemm_tiles.size());
        // Output tile edge: the small tile when the large one would spend more than 10% of the
        // launch's multiply-adds on padding (ragged edges of small fronts).
        auto padded = [&](int32_t T) {
            double e = 0;
            for (const GSpec& g : specs) {
                if (g.M <= 0 || g.N <= 0 || g.K <= 0) continue;
                double nt = 0;
                for (int32_t m0 = 0; m0 < g.M; m0 += T)
                    for (int32_t n0 = 0; n0 < g.N; n0 += T)
                        if (!(lower && n0 > m0 + T - 1)) nt += 1;
                e += nt * T * T * g.K;
            }
            return e;
        };
        l.tile = padded(kGemmTile) > 1.1 * padded(kGemmTileSmall) ? kGemmTileSmall : kGemmTile;
        double fl = 0;
        for (const GSpec& g : specs) {
            if (g.M <= 0 || g.N <= 0 || g.K <= 0) continue;
            const int32_t it = static_cast<int32_t>(P.gemm_items.size() - l.first);
            P.gemm_items.push_back(GemmItem{g.a_off, g.b_off, g.c_off, g.lda, g.ldb, g.ldc, g.M, g.N, g.K, 0});
            for (int32_t m0 = 0; m0 < g.M; m0 += l.tile)
                for (int32_t n0 = 0; n0 < g.N; n0 += l.tile) {
                    if (lower && n0 > m0 + l.tile - 1) continue;
                    P.gemm_tiles.push_back(GemmTile{it, m0, n0, 0});
                }
            const double mn = lower ? 0.5 * g.M * (g.M + 1.0) : static_cast<double>(g.M) * g.N;
            fl += 8.0 * mn * g.K;
            l.bytes += 16.0 * (static_cast<double>(g.M) * g.K + static_cast<double>(g.N) * g.K +
                               mn * (beta != 0.0 ? 2.0 : 1.0));
        }
        l.count = static_cast<int64_t>(P.gemm_items.size()) - l.first;
        l.tcount = static_cast<int64_t>(P.gemm_tiles.size()) - l.tfirst;
        l.flops = fl;
        if (l.count > 0) {
            P.flops_per_pole += fl;
            P.launches.push_back(l);
        }
    };
    auto emit_copy = [&](int32_t L, int32_t phase, int32_t tag, double scale,
                         const std::vector<CopyItem>& items) {
        if (items.empty()) return;
        Launch l = new_launch(L_COPY, L, phase, tag);
        l.alpha = scale;
        l.first = static_cast<int64_t>(P.copy_items.size());
        for (const CopyItem& c : items) P.copy_items.push_back(c);
        l.count = static_cast<int64_t>(items.size());
        for (const CopyItem& c : items) l.bytes += 32.0 * c.rows * c.cols;
        P.launches.push_back(l);
    };
    for (int32_t L = 0; L < P.n_levels; ++L) {
        const auto& nodesL = P.level_nodes[L];
        // assembly tiles
        {
            Launch l = new_launch(L_ASSEMBLE, L, 0, T_ASSEMBLE);
            l.first = static_cast<int64_t>(P.node_tiles.size());
            for (int32_t j : nodesL) {
                for (int32_t i0 = 0; i0 < P.f[j]; i0 += kNodeTile)
                    for (int32_t j0 = 0; j0 <= i0; j0 += kNodeTile) P.node_tiles.push_back(NodeTile{j, i0, j0, 0});
                l.bytes += 16.0 * 0.5 * P.f[j] * (P.f[j] + 1.0);
                for (int t = 0; t < P.nchild[j]; ++t) {
                    const int32_t c = t == 0 ? P.child0[j] : P.child1[j];
                    l.bytes += 16.0 * 0.5 * P.r[c] * (P.r[c] + 1.0);
                }
            }
            P.bytes_per_pole += l.bytes;
            l.count = static_cast<int64_t>(P.node_tiles.size()) - l.first;
            if (l.count > 0) P.launches.push_back(l);
        }
        // scatter of z*S - H
        {
            Launch l = new_launch(L_SCATTER, L, 0, T_SCATTER);
            l.first = static_cast<int64_t>(P.scatter_idx.size());
            P.scatter_idx.insert(P.scatter_idx.end(), lvl_entries[L].begin(), lvl_entries[L].end());
            l.count = static_cast<int64_t>(lvl_entries[L].size());
            l.bytes = 48.0 * static_cast<double>(l.count);  // index, map, H, S, front read+write
            P.bytes_per_pole += l.bytes;
            if (l.count > 0) P.launches.push_back(l);
        }
        // F2/F3: block LDL^T of A_J (Eqs. 18-20) and its inverse (Eqs. 38-39 inside the block), in
        // two levels.  A_J is cut into diagonal blocks of `outer` columns; each block, once its
        // trailing update has arrived, is factored in b x b pivot blocks and inverted in place
        // (FP64, marked exact), then the panel below it is scaled by that inverse and the
        // trailing matrix updated with inner dimension `outer`.  The inverse of A_J is assembled
        // block by block from the last one backwards.  The outer GEMMs are few and large, which
        // is what split mode needs; the pivot-level work stays in FP64.
        const int32_t Bo = P.outer;
        int32_t nob = 0;
        for (int32_t j : nodesL) nob = std::max<int32_t>(nob, static_cast<int32_t>(ceil_div(P.s[j], Bo)));
        for (int32_t T = 0; T < nob; ++T) {
            // (i) block LDL^T of diagonal block T in pivot blocks of b
            for (int32_t t = 0; t < Bo / b; ++t) {
                Launch ld = new_launch(L_DIAGINV, L, 0, T_DINV);
                ld.first = static_cast<int64_t>(P.diag_items.size());
                std::vector<GSpec> panel, update;
                std::vector<CopyItem> copies;
                for (int32_t j : nodesL) {
                    const int32_t s = P.s[j], f = P.f[j];
                    const int32_t K0 = T * Bo;
                    if (K0 >= s) continue;
                    const int32_t K1 = std::min(K0 + Bo, s);
                    const int32_t k0 = K0 + t * b;
                    if (k0 >= K1) continue;
                    const int32_t nb = std::min(b, K1 - k0);
                    const int32_t k1 = k0 + nb;
                    const int64_t fo = P.front_off[j];
                    P.diag_items.push_back(DiagItem{fo + k0 + static_cast<int64_t>(k0) * f, f, nb});
                    ld.flops += 8.0 * nb * nb * nb;
                    ld.bytes += 16.0 * nb * (nb + 1.0);
                    if (k1 < K1) {
                        const int32_t m = K1 - k1;
                        panel.push_back(GSpec{fo + k1 + static_cast<int64_t>(k0) * f, fo + k0 + static_cast<int64_t>(k0) * f,
                                              P.scr_off[j], f, f, m, m, nb, nb});
                        update.push_back(GSpec{P.scr_off[j], fo + k1 + static_cast<int64_t>(k0) * f,
                                               fo + k1 + static_cast<int64_t>(k1) * f, m, f, f, m, m, nb});
                        copies.push_back(CopyItem{P.scr_off[j], fo + k1 + static_cast<int64_t>(k0) * f, m, f, m, nb});
                    }
                }
                ld.count = static_cast<int64_t>(P.diag_items.size()) - ld.first;
                // pivot-sweep variant: 16 when every block of the launch is at most 16 wide
                ld.tile = 16;
                for (int64_t i = ld.first; i < ld.first + ld.count; ++i)
                    if (P.diag_items[i].nb > 16) ld.tile = 32;
                if (ld.count > 0) {
                    P.flops_per_pole += ld.flops;
                    P.launches.push_back(ld);
                }
                emit_gemm(L, 0, T_PANEL, OP_N, OP_S, BUF_FRONT, BUF_FRONT, BUF_SCR, 1.0, 0.0, false, panel, true);
                emit_gemm(L, 0, T_UPDATE, OP_N, OP_T, BUF_SCR, BUF_FRONT, BUF_FRONT, -1.0, 1.0, true, update, true);
                emit_copy(L, 0, T_PCOPY, 1.0, copies);
            }
            // (ii) inverse of diagonal block T in place, from its pivot blocks backwards
            for (int32_t t = Bo / b - 1; t >= 0; --t) {
                std::vector<GSpec> tg, dg;
                std::vector<CopyItem> copies;
                for (int32_t j : nodesL) {
                    const int32_t s = P.s[j], f = P.f[j];
                    const int32_t K0 = T * Bo;
                    if (K0 >= s) continue;
                    const int32_t K1 = std::min(K0 + Bo, s);
                    const int32_t k0 = K0 + t * b;
                    if (k0 >= K1) continue;
                    const int32_t nb = std::min(b, K1 - k0);
                    const int32_t k1 = k0 + nb;
                    if (k1 >= K1) continue;
                    const int32_t m = K1 - k1;
                    const int64_t fo = P.front_off[j];
                    tg.push_back(GSpec{fo + k1 + static_cast<int64_t>(k1) * f, fo + k1 + static_cast<int64_t>(k0) * f,
                                       P.scr_off[j], f, f, m, m, nb, m});
                    dg.push_back(GSpec{fo + k1 + static_cast<int64_t>(k0) * f, P.scr_off[j],
                                       fo + k0 + static_cast<int64_t>(k0) * f, f, m, f, nb, nb, m});
                    copies.push_back(CopyItem{P.scr_off[j], fo + k1 + static_cast<int64_t>(k0) * f, m, f, m, nb});
                }
                emit_gemm(L, 0, T_AINV_T, OP_S, OP_N, BUF_FRONT, BUF_FRONT, BUF_SCR, 1.0, 0.0, false, tg, true);
                emit_gemm(L, 0, T_AINV_D, OP_T, OP_N, BUF_FRONT, BUF_SCR, BUF_FRONT, 1.0, 1.0, true, dg, true);
                emit_copy(L, 0, T_AINV_COPY, -1.0, copies);
            }
            // (iii) panel below the block scaled by its inverse, trailing update, store the panel
            {
                std::vector<GSpec> panel, update;
                std::vector<CopyItem> copies;
                for (int32_t j : nodesL) {
                    const int32_t s = P.s[j], f = P.f[j];
                    const int32_t K0 = T * Bo;
                    if (K0 >= s) continue;
                    const int32_t K1 = std::min(K0 + Bo, s);
                    if (K1 >= s) continue;
                    const int32_t m = s - K1, w = K1 - K0;
                    const int64_t fo = P.front_off[j];
                    panel.push_back(GSpec{fo + K1 + static_cast<int64_t>(K0) * f, fo + K0 + static_cast<int64_t>(K0) * f,
                                          P.scr_off[j], f, f, m, m, w, w});
                    update.push_back(GSpec{P.scr_off[j], fo + K1 + static_cast<int64_t>(K0) * f,
                                           fo + K1 + static_cast<int64_t>(K1) * f, m, f, f, m, m, w});
                    copies.push_back(CopyItem{P.scr_off[j], fo + K1 + static_cast<int64_t>(K0) * f, m, f, m, w});
                }
                emit_gemm(L, 0, T_OPANEL, OP_N, OP_S, BUF_FRONT, BUF_FRONT, BUF_SCR, 1.0, 0.0, false, panel);
                emit_gemm(L, 0, T_OUPDATE, OP_N, OP_T, BUF_SCR, BUF_FRONT, BUF_FRONT, -1.0, 1.0, true, update);
                emit_copy(L, 0, T_OPCOPY, 1.0, copies);
            }
        }
        // inverse of A_J assembled from the diagonal-block inverses, last block first
        for (int32_t T = nob - 1; T >= 0; --T) {
            std::vector<GSpec> tg, dg;
            std::vector<CopyItem> copies;
            for (int32_t j : nodesL) {
                const int32_t s = P.s[j], f = P.f[j];
                const int32_t K0 = T * Bo;
                if (K0 >= s) continue;
                const int32_t K1 = std::min(K0 + Bo, s);
                if (K1 >= s) continue;
                const int32_t m = s - K1, w = K1 - K0;
                const int64_t fo = P.front_off[j];
                tg.push_back(GSpec{fo + K1 + static_cast<int64_t>(K1) * f, fo + K1 + static_cast<int64_t>(K0) * f,
                                   P.scr_off[j], f, f, m, m, w, m});
                dg.push_back(GSpec{fo + K1 + static_cast<int64_t>(K0) * f, P.scr_off[j],
                                   fo + K0 + static_cast<int64_t>(K0) * f, f, m, f, w, w, m});
                copies.push_back(CopyItem{P.scr_off[j], fo + K1 + static_cast<int64_t>(K0) * f, m, f, m, w});
            }
            emit_gemm(L, 0, T_OAINV_T, OP_S, OP_N, BUF_FRONT, BUF_FRONT, BUF_SCR, 1.0, 0.0, false, tg);
            emit_gemm(L, 0, T_OAINV_D, OP_T, OP_N, BUF_FRONT, BUF_SCR, BUF_FRONT, 1.0, 1.0, true, dg);
            emit_copy(L, 0, T_OAINV_COPY, -1.0, copies);
        }
        // F4-F6: L_RJ = B A_J^{-1}; Schur update of the separator front (Eq. 32); store L
        {
            std::vector<GSpec> lrj, schur;
            std::vector<CopyItem> copies;
            for (int32_t j : nodesL) {
                const int32_t s = P.s[j], r = P.r[j], f = P.f[j];
                if (s == 0 || r == 0) continue;
                const int64_t fo = P.front_off[j];
                lrj.push_back(GSpec{fo + s, fo, P.scr_off[j], f, f, r, r, s, s});
                schur.push_back(GSpec{P.scr_off[j], fo + s, fo + s + static_cast<int64_t>(s) * f, r, f, f, r, r, s});
                copies.push_back(CopyItem{P.scr_off[j], fo + s, r, f, r, s});
            }
            emit_gemm(L, 0, T_LRJ, OP_N, OP_S, BUF_FRONT, BUF_FRONT, BUF_SCR, 1.0, 0.0, false, lrj);
            emit_gemm(L, 0, T_SCHUR, OP_N, OP_T, BUF_SCR, BUF_FRONT, BUF_FRONT, -1.0, 1.0, true, schur);
            emit_copy(L, 0, T_LCOPY, 1.0, copies);
        }
    }
    // selected inversion, top-down
    for (int32_t L = P.n_levels - 1; L >= 0; --L) {
        const auto& nodesL = P.level_nodes[L];
        {
            Launch l = new_launch(L_GATHER, L, 1, T_GATHER);
            l.first = static_cast<int64_t>(P.node_tiles.size());
            for (int32_t j : nodesL) {
                if (P.parent[j] < 0) continue;
                for (int32_t i0 = 0; i0 < P.r[j]; i0 += kNodeTile)
                    for (int32_t j0 = 0; j0 <= i0; j0 += kNodeTile) P.node_tiles.push_back(NodeTile{j, i0, j0, 0});
                l.bytes += 2.0 * 16.0 * 0.5 * P.r[j] * (P.r[j] + 1.0);
            }
            P.bytes_per_pole += l.bytes;
            l.count = static_cast<int64_t>(P.node_tiles.size()) - l.first;
            if (l.count > 0) P.launches.push_back(l);
        }
        std::vector<GSpec> tg, dg;
        std::vector<CopyItem> copies;
        for (int32_t j : nodesL) {
            const int32_t s = P.s[j], r = P.r[j], f = P.f[j];
            if (s == 0 || r == 0) continue;
            const int64_t fo = P.front_off[j];
            tg.push_back(GSpec{fo + s + static_cast<int64_t>(s) * f, fo + s, P.scr_off[j], f, f, r, r, s, r});
            dg.push_back(GSpec{fo + s, P.scr_off[j], fo, f, r, f, s, s, r});
            copies.push_back(CopyItem{P.scr_off[j], fo + s, r, f, r, s});
        }
        emit_gemm(L, 1, T_SEL_T, OP_S, OP_N, BUF_FRONT, BUF_FRONT, BUF_SCR, 1.0, 0.0, false, tg);
        emit_gemm(L, 1, T_SEL_D, OP_T, OP_N, BUF_FRONT, BUF_SCR, BUF_FRONT, 1.0, 1.0, true, dg);
        emit_copy(L, 1, T_SEL_COPY, -1.0, copies);
    }
    // the accumulation reads each pattern value of G once per pole
    P.bytes_per_pole += 16.0 * static_cast<double>(P.nnz);
}

// Merge per-system plans into one: nodes, fronts and index tables are concatenated with
// offsets, tree levels are aligned (level = height above the innermost domains), and one
// schedule covers every system, so each launch processes a level of all systems at once.
int merge_plans(std::vector<Plan>& parts, Plan& M, std::string& err) {
    if (parts.empty()) {
        err = "ndsi_analyze_batched: no systems";
        return NDSI_ERR_INVALID;
    }
    M = Plan{};
    M.opt = parts[0].opt;
    M.block = parts[0].block;
    M.outer = parts[0].outer;
    M.n_systems = static_cast<int32_t>(parts.size());
    M.sys_nnz_first.assign(parts.size() + 1, 0);
    M.sys_n_first.assign(parts.size() + 1, 0);
    int32_t node_base = 0;
    int64_t front_base = 0, nnz_base = 0, n_base = 0, inv_base = 0, rel_base = 0;
    for (const Plan& Q : parts) M.n_levels = std::max(M.n_levels, Q.n_levels);
    M.level_entries.assign(M.n_levels, {});
    M.level_nodes.assign(M.n_levels, {});
    M.rowptr.assign(1, 0);
    for (size_t si = 0; si < parts.size(); ++si) {
        const Plan& Q = parts[si];
        M.sys_nnz_first[si] = nnz_base;
        M.sys_n_first[si] = n_base;
        for (int32_t j = 0; j < Q.n_nodes; ++j) {
            NodeDev d = Q.nodes[j];
            d.front_off += front_base;
            for (int t = 0; t < 2; ++t) {
                if (d.inv_off[t] >= 0) d.inv_off[t] += inv_base;
                if (d.child[t] >= 0) d.child[t] += node_base;
            }
            if (d.rel_off >= 0) d.rel_off += rel_base;
            if (d.parent >= 0) d.parent += node_base;
            M.nodes.push_back(d);
            M.f.push_back(Q.f[j]);
            M.s.push_back(Q.s[j]);
            M.r.push_back(Q.r[j]);
            M.front_off.push_back(Q.front_off[j] + front_base);
            M.parent.push_back(Q.parent[j] >= 0 ? Q.parent[j] + node_base : -1);
            M.child0.push_back(Q.child0[j] >= 0 ? Q.child0[j] + node_base : -1);
            M.child1.push_back(Q.child1[j] >= 0 ? Q.child1[j] + node_base : -1);
            M.nchild.push_back(Q.nchild[j]);
            M.level.push_back(Q.level[j]);
            M.level_nodes[Q.level[j]].push_back(node_base + j);
            M.max_front = std::max(M.max_front, Q.f[j]);
        }
        for (int64_t k = 0; k < Q.nnz; ++k) {
            M.asm_map.push_back(Q.asm_map[k] >= 0 ? Q.asm_map[k] + front_base : -1);
            M.out_map.push_back(Q.out_map[k] + front_base);
            M.entry_sys.push_back(static_cast<int32_t>(si));
        }
        for (int32_t L = 0; L < Q.n_levels; ++L)
            for (int64_t k : Q.level_entries[L]) M.level_entries[L].push_back(k + nnz_base);
        for (int32_t v : Q.inv_map) M.inv_map.push_back(v);
        for (int32_t v : Q.rel_map) M.rel_map.push_back(v);
        for (int64_t i = 0; i < Q.n; ++i) M.rowptr.push_back(Q.rowptr[i + 1] + nnz_base);
        for (int32_t c : Q.col) M.col.push_back(static_cast<int32_t>(c + n_base));
        node_base += Q.n_nodes;
        front_base += Q.front_total;
        nnz_base += Q.nnz;
        n_base += Q.n;
        inv_base += static_cast<int64_t>(Q.inv_map.size());
        rel_base += static_cast<int64_t>(Q.rel_map.size());
        M.n_atoms += Q.n_atoms;
    }
    M.sys_nnz_first[parts.size()] = nnz_base;
    M.sys_n_first[parts.size()] = n_base;
    M.n_nodes = node_base;
    M.front_total = std::max<int64_t>(front_base, 1);
    M.nnz = nnz_base;
    M.n = n_base;
    // per-node level lists must follow the merged ids in ascending order
    for (auto& v : M.level_nodes) std::sort(v.begin(), v.end());
    compute_scratch(M);
    build_schedule(M);
    return NDSI_OK;
}

// ---------------------------------------------------------------------------------------------
// Continued-fraction poles (Eq. 7).  The fraction 1/2 - (x/4)/(1 + (x/2)^2/(3 + ...)) truncated
// after the denominator 4M-1 equals 1/2 + sum_p R_p/(x - i z_p) + R_p/(x + i z_p), where
// lambda_p = 2/z_p are the positive eigenvalues of the 2M x 2M symmetric tridiagonal matrix with
// zero diagonal and off-diagonal 1/sqrt((2k-1)(2k+1)), and R_p = -v1_p^2/lambda_p^2 with v1_p the
// first component of the unit eigenvector.  The eigenproblem is solved by implicit symmetric QR
// steps with Wilkinson shifts and deflation, accumulating only the first row of the orthogonal
// factor.
int cf_poles(int32_t M, double* z, double* R, std::string& err) {
    if (M < 1 || !z || !R) {
        err = "ndsi_poles: M must be >= 1 and outputs non-NULL";
        return NDSI_ERR_INVALID;
    }
    const int K = 2 * M;
    std::vector<double> d(K, 0.0), e(K, 0.0), q(K, 0.0);
    for (int k = 1; k < K; ++k) e[k - 1] = 1.0 / std::sqrt((2.0 * k - 1.0) * (2.0 * k + 1.0));
    q[0] = 1.0;
    const double eps = std::ldexp(1.0, -53);
    int hi = K - 1;
    int64_t iters = 0;
    const int64_t max_iters = 60LL * K;
    while (hi > 0) {
        if (std::fabs(e[hi - 1]) <= eps * (std::fabs(d[hi - 1]) + std::fabs(d[hi])) ||
            std::fabs(e[hi - 1]) < 1e-300) {
            e[hi - 1] = 0.0;
            --hi;
            continue;
        }
        int lo = hi - 1;
        while (lo > 0 && !(std::fabs(e[lo - 1]) <= eps * (std::fabs(d[lo - 1]) + std::fabs(d[lo])) ||
                           std::fabs(e[lo - 1]) < 1e-300))
            --lo;
        if (++iters > max_iters) {
            err = "ndsi_poles: eigenvalue iteration did not converge";
            return NDSI_ERR_INVALID;
        }
        // Wilkinson shift from the trailing 2 x 2 block
        const double delta = 0.5 * (d[hi - 1] - d[hi]);
        const double bb = e[hi - 1];
        const double sg = delta >= 0 ? 1.0 : -1.0;
        const double mu = d[hi] - bb * bb / (delta + sg * std::hypot(delta, bb));
        double x = d[lo] - mu, zz = e[lo];
        double bulge = 0.0;
        for (int k = lo; k < hi; ++k) {
            const double rr = std::hypot(x, zz);
            double c = 1.0, s = 0.0;
            if (rr > 0) {
                c = x / rr;
                s = -zz / rr;
            }
            if (k > lo) e[k - 1] = c * x - s * zz;  // bulge annihilated
            const double a = d[k], bk = e[k], dd = d[k + 1];
            d[k] = c * c * a - 2.0 * c * s * bk + s * s * dd;
            d[k + 1] = s * s * a + 2.0 * c * s * bk + c * c * dd;
            e[k] = c * s * a + (c * c - s * s) * bk - c * s * dd;
            if (k + 1 < hi) {
                bulge = -s * e[k + 1];
                e[k + 1] = c * e[k + 1];
            }
            const double qk = q[k], qk1 = q[k + 1];
            q[k] = c * qk - s * qk1;
            q[k + 1] = s * qk + c * qk1;
            x = e[k];
            zz = bulge;
        }
    }
    std::vector<std::pair<double, double>> out;
    for (int k = 0; k < K; ++k) {
        if (d[k] > 0) out.emplace_back(2.0 / d[k], -(q[k] * q[k]) / (d[k] * d[k]));
    }
    if (static_cast<int>(out.size()) != M) {
        err = "ndsi_poles: unexpected eigenvalue signs";
        return NDSI_ERR_INVALID;
    }
    std::sort(out.begin(), out.end());
    for (int p = 0; p < M; ++p) {
        z[p] = out[p].first;
        R[p] = out[p].second;
    }
    return NDSI_OK;
}

}  // namespace ndsi
