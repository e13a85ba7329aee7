// TEST INFRASTRUCTURE ONLY -- the CPU oracle for the Morse-Smale complex 1-skeleton.
//
// A plain, slow, single-threaded restatement of what the method computes, used only to
// check the CUDA path. Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline
// (and --impl reference) legs may load it. It shares no code, header, table or helper
// with the CUDA library, and neither side includes the other.
//
// What it follows (sections of arXiv:2009.03707, Subhash/Pandey/Natarajan):
//   * Sec. 2.2 (Discrete Morse theory): gradient pairs, discrete vector field, V-paths,
//     critical cells.  The gradient rule itself is deferred by the paper (Sec. 3 and
//     Sec. 3.5, "Gradient pairs and critical points") to the locally independent
//     lower-star rules it cites in Sec. 1.1 (Robins, Wood, Sheppard 2011); this file
//     restates that rule, ProcessLowerStars, in the order of their algorithm.
//   * Sec. 3.4 / Sec. 3.5 "Saddle-Extrema arcs": saddle-extremum arcs and the
//     destination extremum of every cell, here as plain memoised walks.
//   * Sec. 3.2 / Sec. 3.5 "Saddle-Saddle reachability": the DAG of 1-2 gradient pairs
//     (Fig. "msc-max-min-dag" (d)) and the set of its nodes reachable from 1-saddles.
//   * Sec. 3.3 / Sec. 3.5 "Gradient path counting": junction nodes and the DAG minor
//     (matrices A, B, B*, D), and the saddle-saddle path counts D*, here computed by the
//     plain definition -- per 1-saddle, a topological-order count of paths in the DAG --
//     rather than by the paper's iterated sparse products.
//   * Sec. 3.4 and Sec. 3.5 "Data structure": the cells along each saddle-extremum arc and
//     along each saddle-saddle arc of multiplicity 1 (its single V-path), as plain walks.
//
// Readings where the paper is silent (each one is also listed in the design notes):
//   R1 vertex order: v < w iff (f(v), index(v)) < (f(w), index(w)); IEEE compare, so
//      -0 == +0 and +-Inf order normally; NaN input is rejected (status 2).
//   R2 key of a cell in the lower star of x: its vertices sorted in decreasing vertex
//      order, compared lexicographically; a proper prefix is smaller.
//   R3 the two priority queues are sets; a popped cell that is already classified is
//      skipped.  "Unclassified" = neither paired nor critical.
//   R4 a walk from a 2-saddle towards a maximum that leaves through a boundary quad
//      (a quad with a single cofacet cube) ends at NONE.
//   R5 junction = a reachable 1-cell that is not a 1-saddle and has DAG out-degree > 1.
//   R6 path counts are exact uint64; an overflowing add is an error (status 6).
//
// Cells live on the refined grid R = (2nx-1) x (2ny-1) x (2nz-1): cell (cx,cy,cz) has
// dimension = number of odd coordinates and id cx + (2nx-1)*(cy + (2ny-1)*cz).  Vertex
// (x,y,z) is cell (2x,2y,2z) and has index x + nx*(y + ny*z).

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <set>
#include <unordered_map>
#include <unordered_set>
#include <tuple>
#include <vector>

namespace {

constexpr uint32_t NONE = 0xFFFFFFFFu;   // critical / no partner / no label
constexpr uint32_t UNSET = 0xFFFFFFFEu;  // not yet classified (must not survive)

enum Status { OK = 0, ERR_ARG = 1, ERR_NAN = 2, ERR_TOO_LARGE = 4, ERR_OVERFLOW = 6, ERR_INTERNAL = 9 };

struct Grid {
    int64_t nx, ny, nz;  // vertex counts
    int64_t rx, ry, rz;  // refined grid extents
    const float* f;      // may be null when only the combinatorics is needed

    Grid(const int64_t* d, const float* field)
        : nx(d[0]), ny(d[1]), nz(d[2]), rx(2 * d[0] - 1), ry(2 * d[1] - 1), rz(2 * d[2] - 1), f(field) {}

    int64_t nverts() const { return nx * ny * nz; }
    int64_t ncells() const { return rx * ry * rz; }
    bool inside(int64_t cx, int64_t cy, int64_t cz) const {
        return cx >= 0 && cy >= 0 && cz >= 0 && cx < rx && cy < ry && cz < rz;
    }
    int64_t cell(int64_t cx, int64_t cy, int64_t cz) const { return cx + rx * (cy + ry * cz); }
    void coords(int64_t c, int64_t& cx, int64_t& cy, int64_t& cz) const {
        cx = c % rx;
        cy = (c / rx) % ry;
        cz = c / (rx * ry);
    }
    int dim(int64_t c) const {
        int64_t cx, cy, cz;
        coords(c, cx, cy, cz);
        return int(cx & 1) + int(cy & 1) + int(cz & 1);
    }
    int64_t vertex(int64_t x, int64_t y, int64_t z) const { return x + nx * (y + ny * z); }
    int64_t vertex_cell(int64_t v) const {
        int64_t x = v % nx, y = (v / nx) % ny, z = v / (nx * ny);
        return cell(2 * x, 2 * y, 2 * z);
    }
    int64_t cell_to_vertex(int64_t c) const {
        int64_t cx, cy, cz;
        coords(c, cx, cy, cz);
        return vertex(cx / 2, cy / 2, cz / 2);
    }
    // R1: the total order on vertices.
    bool vless(int64_t a, int64_t b) const {
        if (f[a] < f[b]) return true;
        if (f[b] < f[a]) return false;
        return a < b;
    }
    // Vertices of a cell: along every odd coordinate both neighbours, along even ones itself.
    // Writes up to 8 vertex ids into out[] and returns how many.
    int vertices(int64_t c, int64_t* out) const {
        int64_t cc[3];
        coords(c, cc[0], cc[1], cc[2]);
        int64_t lo[3], hi[3];
        for (int i = 0; i < 3; ++i) {
            lo[i] = cc[i] / 2;
            hi[i] = (cc[i] & 1) ? lo[i] + 1 : lo[i];
        }
        int n = 0;
        for (int64_t z = lo[2]; z <= hi[2]; ++z)
            for (int64_t y = lo[1]; y <= hi[1]; ++y)
                for (int64_t x = lo[0]; x <= hi[0]; ++x) out[n++] = vertex(x, y, z);
        return n;
    }
    std::vector<int64_t> vertices(int64_t c) const {
        int64_t buf[8];
        int n = vertices(c, buf);
        return std::vector<int64_t>(buf, buf + n);
    }
    // Facets: move one odd coordinate by +-1.  Cofacets: move one even coordinate by +-1 inside R.
    std::vector<int64_t> facets(int64_t c) const {
        int64_t cc[3];
        coords(c, cc[0], cc[1], cc[2]);
        std::vector<int64_t> out;
        for (int i = 0; i < 3; ++i) {
            if (!(cc[i] & 1)) continue;
            for (int s = -1; s <= 1; s += 2) {
                int64_t d[3] = {cc[0], cc[1], cc[2]};
                d[i] += s;
                out.push_back(cell(d[0], d[1], d[2]));
            }
        }
        return out;
    }
    std::vector<int64_t> cofacets(int64_t c) const {
        int64_t cc[3];
        coords(c, cc[0], cc[1], cc[2]);
        std::vector<int64_t> out;
        for (int i = 0; i < 3; ++i) {
            if (cc[i] & 1) continue;
            for (int s = -1; s <= 1; s += 2) {
                int64_t d[3] = {cc[0], cc[1], cc[2]};
                d[i] += s;
                if (inside(d[0], d[1], d[2])) out.push_back(cell(d[0], d[1], d[2]));
            }
        }
        return out;
    }
    int64_t max_vertex(int64_t c) const {
        std::vector<int64_t> vs = vertices(c);
        int64_t m = vs[0];
        for (int64_t v : vs)
            if (vless(m, v)) m = v;
        return m;
    }
};

bool check_dims(const int64_t* d) {
    if (!d) return false;
    for (int i = 0; i < 3; ++i)
        if (d[i] < 2) return false;
    return true;
}

bool ids_fit_u32(const Grid& g) { return g.ncells() < int64_t(UNSET); }

bool has_nan(const Grid& g) {
    for (int64_t v = 0; v < g.nverts(); ++v)
        if (std::isnan(g.f[v])) return true;
    return false;
}

// ---------------------------------------------------------------------------------
// ProcessLowerStars (Robins, Wood, Sheppard 2011) for one vertex x.
// The lower star L(x) is the set of cells whose maximal vertex (under R1) is x.
// Cells of L(x) are paired among themselves or declared critical; the result is
// written into `pair_of` (partner id, or NONE for critical) for those cells only.
// ---------------------------------------------------------------------------------
struct LowerStar {
    const Grid& g;
    struct Cell {
        int64_t id;
        int dim;
        std::vector<int64_t> key;   // R2: vertices in decreasing vertex order
        std::vector<int> facets;    // local indices of the facets that lie in L(x)
        std::vector<int> cofacets;  // local indices of the cofacets that lie in L(x)
        int state;                  // 0 unclassified, 1 paired, 2 critical
    };
    std::vector<Cell> cells;

    LowerStar(const Grid& grid, int64_t x) : g(grid) {
        int64_t cx, cy, cz;
        g.coords(g.vertex_cell(x), cx, cy, cz);
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    if (!g.inside(cx + dx, cy + dy, cz + dz)) continue;
                    int64_t c = g.cell(cx + dx, cy + dy, cz + dz);
                    int64_t vs[8];
                    int nv = g.vertices(c, vs);
                    bool x_is_max = true;
                    for (int i = 0; i < nv; ++i)
                        if (g.vless(x, vs[i])) x_is_max = false;
                    if (!x_is_max) continue;  // c belongs to the lower star of another vertex
                    Cell cell;
                    cell.key.assign(vs, vs + nv);
                    std::sort(cell.key.begin(), cell.key.end(),
                              [&](int64_t a, int64_t b) { return g.vless(b, a); });
                    cell.id = c;
                    cell.dim = g.dim(c);
                    cell.state = 0;
                    cells.push_back(cell);
                }
        for (Cell& cell : cells) {
            for (int64_t fc : g.facets(cell.id)) {
                int i = index_of(fc);
                if (i >= 0) cell.facets.push_back(i);
            }
            for (int64_t cf : g.cofacets(cell.id)) {
                int i = index_of(cf);
                if (i >= 0) cell.cofacets.push_back(i);
            }
        }
    }

    int index_of(int64_t id) const {
        for (size_t i = 0; i < cells.size(); ++i)
            if (cells[i].id == id) return int(i);
        return -1;
    }
    // R2: lexicographic comparison of keys; a proper prefix is smaller.
    bool key_less(int a, int b) const {
        const std::vector<int64_t>& ka = cells[a].key;
        const std::vector<int64_t>& kb = cells[b].key;
        size_t n = std::min(ka.size(), kb.size());
        for (size_t i = 0; i < n; ++i)
            if (ka[i] != kb[i]) return g.vless(ka[i], kb[i]);
        return ka.size() < kb.size();
    }
    const std::vector<int>& facets_in_L(int a) const { return cells[a].facets; }
    const std::vector<int>& cofacets_in_L(int a) const { return cells[a].cofacets; }
    int num_unclassified_facets(int a) const {
        int n = 0;
        for (int i : facets_in_L(a))
            if (cells[i].state == 0) ++n;
        return n;
    }
    int unclassified_facet(int a) const {
        for (int i : facets_in_L(a))
            if (cells[i].state == 0) return i;
        return -1;
    }
};

struct KeyOrder {
    const LowerStar* ls;
    bool operator()(int a, int b) const { return ls->key_less(a, b); }
};

// Returns false if the procedure left a cell of L(x) unclassified (cannot happen for a
// correct restatement; reported as an internal error).
bool process_lower_star(const Grid& g, int64_t x, std::map<int64_t, uint32_t>& out) {
    LowerStar ls(g, x);
    auto pair_cells = [&](int lo, int hi) {
        ls.cells[lo].state = 1;
        ls.cells[hi].state = 1;
        out[ls.cells[lo].id] = uint32_t(ls.cells[hi].id);
        out[ls.cells[hi].id] = uint32_t(ls.cells[lo].id);
    };
    auto make_critical = [&](int a) {
        ls.cells[a].state = 2;
        out[ls.cells[a].id] = NONE;
    };
    const int vx = ls.index_of(g.vertex_cell(x));

    if (ls.cells.size() == 1) {  // L(x) = {x}: x is a minimum
        make_critical(vx);
        return true;
    }
    // x is paired with the edge of least key (the steepest descending edge).
    int delta = -1;
    for (int i = 0; i < int(ls.cells.size()); ++i)
        if (ls.cells[i].dim == 1 && (delta < 0 || ls.key_less(i, delta))) delta = i;
    pair_cells(vx, delta);

    std::set<int, KeyOrder> pq_zero(KeyOrder{&ls}), pq_one(KeyOrder{&ls});
    for (int i = 0; i < int(ls.cells.size()); ++i)
        if (ls.cells[i].dim == 1 && i != delta) pq_zero.insert(i);
    for (int b : ls.cofacets_in_L(delta))
        if (ls.cells[b].state == 0 && ls.num_unclassified_facets(b) == 1) pq_one.insert(b);

    while (!pq_one.empty() || !pq_zero.empty()) {
        while (!pq_one.empty()) {
            int a = *pq_one.begin();
            pq_one.erase(pq_one.begin());
            if (ls.cells[a].state != 0) continue;  // R3
            if (ls.num_unclassified_facets(a) == 0) {
                pq_zero.insert(a);
                continue;
            }
            int p = ls.unclassified_facet(a);
            pair_cells(p, a);
            pq_zero.erase(p);
            std::vector<int> nb = ls.cofacets_in_L(a);
            const std::vector<int>& nb2 = ls.cofacets_in_L(p);
            nb.insert(nb.end(), nb2.begin(), nb2.end());
            for (int b : nb)
                if (ls.cells[b].state == 0 && ls.num_unclassified_facets(b) == 1) pq_one.insert(b);
        }
        if (!pq_zero.empty()) {
            int c = *pq_zero.begin();
            pq_zero.erase(pq_zero.begin());
            if (ls.cells[c].state != 0) continue;  // R3
            make_critical(c);
            for (int b : ls.cofacets_in_L(c))
                if (ls.cells[b].state == 0 && ls.num_unclassified_facets(b) == 1) pq_one.insert(b);
        }
    }
    for (const auto& c : ls.cells)
        if (c.state == 0) return false;
    return true;
}

// ---------------------------------------------------------------------------------
// Packed per-vertex gradient word (the library's exchange format).
// Vertex (x,y,z) owns the 8 cells (2x+a, 2y+b, 2z+c), a,b,c in {0,1}; slot s = a + 2b + 4c
// holds a 3-bit code in bits [3s, 3s+3): 0 = critical, 1..6 = partner at -x,+x,-y,+y,-z,+z,
// 7 = the cell lies outside the refined grid.
// ---------------------------------------------------------------------------------
uint32_t direction_code(const Grid& g, int64_t c, uint32_t partner) {
    if (partner == NONE) return 0;
    int64_t ax, ay, az, bx, by, bz;
    g.coords(c, ax, ay, az);
    g.coords(int64_t(partner), bx, by, bz);
    if (bx == ax - 1) return 1;
    if (bx == ax + 1) return 2;
    if (by == ay - 1) return 3;
    if (by == ay + 1) return 4;
    if (bz == az - 1) return 5;
    return 6;
}

uint32_t packed_word(const Grid& g, int64_t v, const std::map<int64_t, uint32_t>& pairs) {
    int64_t x = v % g.nx, y = (v / g.nx) % g.ny, z = v / (g.nx * g.ny);
    uint32_t w = 0;
    for (int s = 0; s < 8; ++s) {
        int a = s & 1, b = (s >> 1) & 1, c = (s >> 2) & 1;
        uint32_t code = 7;
        if (g.inside(2 * x + a, 2 * y + b, 2 * z + c)) {
            int64_t id = g.cell(2 * x + a, 2 * y + b, 2 * z + c);
            code = direction_code(g, id, pairs.at(id));
        }
        w |= code << (3 * s);
    }
    return w;
}

// ---------------------------------------------------------------------------------
// DAG of 1-2 gradient pairs (Sec. 3.2, Fig. "msc-max-min-dag" (d)).
// Nodes: 1-saddles, 1-cells paired with a 2-cell, and 2-saddles.  For a 1-cell node e,
// each cofacet quad q of e other than e's own partner gives an out-edge: to q if q is
// critical (a 2-saddle), to the 1-cell paired with q if q is paired downwards, and none
// if q is paired with a cube.  Following an out-edge walks a V-path backwards, i.e. the
// traversal runs against the discrete gradient (Sec. 3.5).
// ---------------------------------------------------------------------------------
// The pairing is read through an accessor P with `uint32_t operator()(int64_t cell)`: a full
// array for whole-volume runs, or LazyPairs (below) for sampled queries on large volumes.
template <class P>
std::vector<int64_t> dag_out_p(const Grid& g, P& pair, int64_t e) {
    std::vector<int64_t> out;
    const uint32_t own = pair(e);
    for (int64_t q : g.cofacets(e)) {
        if (uint32_t(q) == own) continue;
        uint32_t p = pair(q);
        if (p == NONE) {
            out.push_back(q);
        } else if (g.dim(int64_t(p)) == 1) {
            out.push_back(int64_t(p));
        }
    }
    return out;
}

struct ArrayPairs {
    const uint32_t* a;
    uint32_t operator()(int64_t c) const { return a[c]; }
};

std::vector<int64_t> dag_out(const Grid& g, const uint32_t* pair_of, int64_t e) {
    ArrayPairs ap{pair_of};
    return dag_out_p(g, ap, e);
}

bool is_dag_node_1cell(const Grid& g, const uint32_t* pair_of, int64_t e) {
    if (g.dim(e) != 1) return false;
    uint32_t p = pair_of[e];
    return p == NONE || g.dim(int64_t(p)) == 2;
}

std::vector<int64_t> critical_list(const Grid& g, const uint32_t* pair_of, int dim) {
    std::vector<int64_t> out;
    for (int64_t c = 0; c < g.ncells(); ++c)
        if (pair_of[c] == NONE && g.dim(c) == dim) out.push_back(c);
    return out;
}

// Bit `axis` of visited[v] marks the 1-cell owned by vertex v along that axis.
int64_t one_cell_slot(const Grid& g, int64_t e, int& axis) {
    int64_t cx, cy, cz;
    g.coords(e, cx, cy, cz);
    axis = (cx & 1) ? 0 : ((cy & 1) ? 1 : 2);
    return g.vertex(cx / 2, cy / 2, cz / 2);
}

bool visited_get(const Grid& g, const uint8_t* visited, int64_t e) {
    int axis;
    int64_t v = one_cell_slot(g, e, axis);
    return (visited[v] >> axis) & 1;
}

struct Minor {
    // (row rank, col rank) -> multiplicity, for A (1s x j), B (j x j), B* (j x 2s), D (1s x 2s)
    std::map<std::pair<int64_t, int64_t>, uint64_t> m[4];
    int status = OK;
};

int64_t rank_in(const std::vector<int64_t>& sorted, int64_t id) {
    auto it = std::lower_bound(sorted.begin(), sorted.end(), id);
    if (it == sorted.end() || *it != id) return -1;
    return int64_t(it - sorted.begin());
}


// ---------------------------------------------------------------------------------
// Sampled queries on large volumes.  The lower-star rule is local: the pair of a cell is
// decided inside the lower star of its maximal vertex alone.  LazyPairs runs
// ProcessLowerStars for a vertex the first time one of its cells is asked for, and keeps the
// result; the walks and counts below are the same definitions as the whole-volume ones.
// ---------------------------------------------------------------------------------
struct LazyPairs {
    const Grid& g;
    std::unordered_map<int64_t, uint32_t> pair;
    int status = OK;
    explicit LazyPairs(const Grid& grid) : g(grid) {}
    uint32_t operator()(int64_t c) {
        auto it = pair.find(c);
        if (it != pair.end()) return it->second;
        std::map<int64_t, uint32_t> local;
        for (int64_t w : g.vertices(c))
            if (std::isnan(g.f[w])) status = ERR_NAN;
        if (!process_lower_star(g, g.max_vertex(c), local)) status = ERR_INTERNAL;
        for (const auto& kv : local) pair[kv.first] = kv.second;
        it = pair.find(c);
        return it == pair.end() ? NONE : it->second;
    }
};
}  // namespace

// =====================================================================================
// C entry points (ctypes).  dims = {nx, ny, nz}; field layout f[x + nx*(y + ny*z)].
// =====================================================================================
extern "C" {

int ora_version() { return 1; }

// Full discrete gradient: pair_of[c] = partner id or 0xFFFFFFFF (critical), for every cell.
int ora_gradient(const int64_t* dims, const float* f, uint32_t* pair_of) {
    if (!check_dims(dims) || !f || !pair_of) return ERR_ARG;
    Grid g(dims, f);
    if (!ids_fit_u32(g)) return ERR_TOO_LARGE;
    if (has_nan(g)) return ERR_NAN;
    for (int64_t c = 0; c < g.ncells(); ++c) pair_of[c] = UNSET;
    std::map<int64_t, uint32_t> local;
    for (int64_t x = 0; x < g.nverts(); ++x) {
        local.clear();
        if (!process_lower_star(g, x, local)) return ERR_INTERNAL;
        for (const auto& kv : local) {
            if (pair_of[kv.first] != UNSET) return ERR_INTERNAL;  // classified twice
            pair_of[kv.first] = kv.second;
        }
    }
    for (int64_t c = 0; c < g.ncells(); ++c)
        if (pair_of[c] == UNSET) return ERR_INTERNAL;
    return OK;
}

// Pairing restricted to the lower star of each listed vertex: writes the packed words of
// the listed vertices (computing every lower star those 8 cells fall into).
int ora_packed_at(const int64_t* dims, const float* f, int64_t n, const int64_t* verts, uint32_t* words) {
    if (!check_dims(dims) || !f || (n > 0 && (!verts || !words))) return ERR_ARG;
    Grid g(dims, f);
    if (!ids_fit_u32(g)) return ERR_TOO_LARGE;
    std::map<int64_t, uint32_t> pairs;
    for (int64_t i = 0; i < n; ++i) {
        int64_t v = verts[i];
        if (v < 0 || v >= g.nverts()) return ERR_ARG;
        int64_t x = v % g.nx, y = (v / g.nx) % g.ny, z = v / (g.nx * g.ny);
        pairs.clear();
        for (int c = 0; c < 2; ++c)
            for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a) {
                    if (!g.inside(2 * x + a, 2 * y + b, 2 * z + c)) continue;
                    int64_t id = g.cell(2 * x + a, 2 * y + b, 2 * z + c);
                    if (pairs.count(id)) continue;
                    for (int64_t w : g.vertices(id))
                        if (std::isnan(g.f[w])) return ERR_NAN;
                    if (!process_lower_star(g, g.max_vertex(id), pairs)) return ERR_INTERNAL;
                }
        words[i] = packed_word(g, v, pairs);
    }
    return OK;
}

// Packed words of all vertices from a full pairing.
int ora_pack(const int64_t* dims, const uint32_t* pair_of, uint32_t* words) {
    if (!check_dims(dims) || !pair_of || !words) return ERR_ARG;
    Grid g(dims, nullptr);
    for (int64_t v = 0; v < g.nverts(); ++v) {
        int64_t x = v % g.nx, y = (v / g.nx) % g.ny, z = v / (g.nx * g.ny);
        uint32_t w = 0;
        for (int s = 0; s < 8; ++s) {
            int a = s & 1, b = (s >> 1) & 1, c = (s >> 2) & 1;
            uint32_t code = 7;
            if (g.inside(2 * x + a, 2 * y + b, 2 * z + c)) {
                int64_t id = g.cell(2 * x + a, 2 * y + b, 2 * z + c);
                code = direction_code(g, id, pair_of[id]);
            }
            w |= code << (3 * s);
        }
        words[v] = w;
    }
    return OK;
}

// Critical cells: counts per dimension, and the list of one dimension in cell-id order.
int ora_critical_counts(const int64_t* dims, const uint32_t* pair_of, int64_t* counts) {
    if (!check_dims(dims) || !pair_of || !counts) return ERR_ARG;
    Grid g(dims, nullptr);
    for (int k = 0; k < 4; ++k) counts[k] = 0;
    for (int64_t c = 0; c < g.ncells(); ++c)
        if (pair_of[c] == NONE) counts[g.dim(c)]++;
    return OK;
}

int ora_critical_list(const int64_t* dims, const uint32_t* pair_of, int dim, uint32_t* out) {
    if (!check_dims(dims) || !pair_of || !out || dim < 0 || dim > 3) return ERR_ARG;
    Grid g(dims, nullptr);
    int64_t n = 0;
    for (int64_t c = 0; c < g.ncells(); ++c)
        if (pair_of[c] == NONE && g.dim(c) == dim) out[n++] = uint32_t(c);
    return OK;
}

// Destination extrema (Sec. 3.4): vertex_min[v] = cell id of the minimum that the
// descending walk from v reaches; cube_max[v] = cell id of the maximum that the ascending
// walk from cube (2x+1,2y+1,2z+1) reaches, NONE if it leaves the domain (R4) or if v has
// no such cube (x = nx-1, y = ny-1 or z = nz-1).
int ora_extremum_labels(const int64_t* dims, const uint32_t* pair_of, uint32_t* vertex_min, uint32_t* cube_max) {
    if (!check_dims(dims) || !pair_of || !vertex_min || !cube_max) return ERR_ARG;
    Grid g(dims, nullptr);
    const int64_t nv = g.nverts();
    // Vertices: v paired with edge (v,w) steps to w; an unpaired vertex is a minimum.
    for (int64_t v = 0; v < nv; ++v) vertex_min[v] = UNSET;
    std::vector<int64_t> stack;
    for (int64_t v0 = 0; v0 < nv; ++v0) {
        int64_t v = v0;
        stack.clear();
        uint32_t label = UNSET;
        while (true) {
            if (vertex_min[v] != UNSET) { label = vertex_min[v]; break; }
            stack.push_back(v);
            int64_t vc = g.vertex_cell(v);
            uint32_t e = pair_of[vc];
            if (e == NONE) { label = uint32_t(vc); break; }
            int64_t other = -1;
            for (int64_t w : g.vertices(int64_t(e)))
                if (w != v) other = w;
            v = other;
            if (int64_t(stack.size()) > nv) return ERR_INTERNAL;  // a cycle
        }
        for (int64_t s : stack) vertex_min[s] = label;
    }
    // Cubes: a cube paired with quad p steps to the other cofacet cube of p (NONE if p is on
    // the boundary); an unpaired cube is a maximum.
    for (int64_t v = 0; v < nv; ++v) cube_max[v] = UNSET;
    auto cube_slot = [&](int64_t c) { return g.cell_to_vertex(c); };
    for (int64_t v0 = 0; v0 < nv; ++v0) {
        int64_t x = v0 % g.nx, y = (v0 / g.nx) % g.ny, z = v0 / (g.nx * g.ny);
        if (x == g.nx - 1 || y == g.ny - 1 || z == g.nz - 1) { cube_max[v0] = NONE; continue; }
        int64_t c = g.cell(2 * x + 1, 2 * y + 1, 2 * z + 1);
        stack.clear();
        uint32_t label = UNSET;
        while (true) {
            int64_t slot = cube_slot(c);
            if (cube_max[slot] != UNSET) { label = cube_max[slot]; break; }
            stack.push_back(slot);
            uint32_t p = pair_of[c];
            if (p == NONE) { label = uint32_t(c); break; }
            int64_t cx, cy, cz, px, py, pz;
            g.coords(c, cx, cy, cz);
            g.coords(int64_t(p), px, py, pz);
            int64_t nxc = 2 * px - cx, nyc = 2 * py - cy, nzc = 2 * pz - cz;  // across the quad
            if (!g.inside(nxc, nyc, nzc)) { label = NONE; break; }
            c = g.cell(nxc, nyc, nzc);
            if (int64_t(stack.size()) > nv) return ERR_INTERNAL;
        }
        for (int64_t s : stack) cube_max[s] = label;
    }
    return OK;
}

// Saddle-extremum arcs.  1-saddle edge: labels of its lower-coordinate then upper-coordinate
// vertex.  2-saddle quad: labels of its cofacet cube on the - side then the + side of the
// quad's even axis (NONE where the cube does not exist).
int ora_min_arcs(const int64_t* dims, const uint32_t* vertex_min, int64_t n1, const uint32_t* s1, uint32_t* out) {
    if (!check_dims(dims) || !vertex_min || (n1 > 0 && (!s1 || !out))) return ERR_ARG;
    Grid g(dims, nullptr);
    for (int64_t i = 0; i < n1; ++i) {
        std::vector<int64_t> vs = g.vertices(int64_t(s1[i]));
        if (vs.size() != 2) return ERR_ARG;
        out[2 * i] = vertex_min[std::min(vs[0], vs[1])];
        out[2 * i + 1] = vertex_min[std::max(vs[0], vs[1])];
    }
    return OK;
}

int ora_max_arcs(const int64_t* dims, const uint32_t* cube_max, int64_t n2, const uint32_t* s2, uint32_t* out) {
    if (!check_dims(dims) || !cube_max || (n2 > 0 && (!s2 || !out))) return ERR_ARG;
    Grid g(dims, nullptr);
    for (int64_t i = 0; i < n2; ++i) {
        int64_t cc[3];
        g.coords(int64_t(s2[i]), cc[0], cc[1], cc[2]);
        int axis = !(cc[0] & 1) ? 0 : (!(cc[1] & 1) ? 1 : 2);
        for (int side = 0; side < 2; ++side) {
            int64_t d[3] = {cc[0], cc[1], cc[2]};
            d[axis] += side ? 1 : -1;
            out[2 * i + side] = g.inside(d[0], d[1], d[2]) ? cube_max[g.cell_to_vertex(g.cell(d[0], d[1], d[2]))] : NONE;
        }
    }
    return OK;
}

// Cells along the saddle-extremum arcs (Sec. 3.4 and Sec. 3.5 "Data structure"): the V-path
// (Sec. 2.2) that each arc follows, walked from its saddle.  Arcs come in the order of the arc
// lists: two per 1-saddle (its lower-coordinate vertex, then its upper one), then two per
// 2-saddle (its cofacet cube on the - side, then the + side, of the quad's even axis).
//   Descending: the 1-saddle, its vertex v, then alternately the edge v is paired with and that
//   edge's other vertex, until a vertex that is not paired (a minimum).
//   Ascending: the 2-saddle, its cofacet cube c, then alternately the quad c is paired with and
//   the cube across that quad, until a cube that is not paired (a maximum); a quad with no cube
//   across it ends the path there (R4: it leaves the domain); the 2-saddle alone when the cube
//   on that side does not exist.
struct ArcCells {
    std::vector<int64_t> offsets;
    std::vector<uint32_t> cells;
    int status = OK;
};

void* ora_arc_cells(const int64_t* dims, const uint32_t* pair_of, int64_t n1, const uint32_t* s1, int64_t n2,
                    const uint32_t* s2) {
    ArcCells* res = new ArcCells();
    if (!check_dims(dims) || !pair_of || (n1 > 0 && !s1) || (n2 > 0 && !s2)) {
        res->status = ERR_ARG;
        return res;
    }
    Grid g(dims, nullptr);
    const int64_t limit = g.ncells();  // a longer walk would have to repeat a cell
    res->offsets.push_back(0);
    for (int64_t i = 0; i < n1; ++i) {
        std::vector<int64_t> vs = g.vertices(int64_t(s1[i]));
        if (vs.size() != 2) { res->status = ERR_ARG; return res; }
        for (int side = 0; side < 2; ++side) {
            int64_t v = side ? std::max(vs[0], vs[1]) : std::min(vs[0], vs[1]);
            res->cells.push_back(s1[i]);
            res->cells.push_back(uint32_t(g.vertex_cell(v)));
            for (int64_t steps = 0;; ++steps) {
                uint32_t e = pair_of[g.vertex_cell(v)];
                if (e == NONE) break;  // a minimum
                if (steps > limit) { res->status = ERR_INTERNAL; return res; }
                int64_t w = -1;
                for (int64_t u : g.vertices(int64_t(e)))
                    if (u != v) w = u;
                res->cells.push_back(e);
                res->cells.push_back(uint32_t(g.vertex_cell(w)));
                v = w;
            }
            res->offsets.push_back(int64_t(res->cells.size()));
        }
    }
    for (int64_t i = 0; i < n2; ++i) {
        int64_t cc[3];
        g.coords(int64_t(s2[i]), cc[0], cc[1], cc[2]);
        int axis = !(cc[0] & 1) ? 0 : (!(cc[1] & 1) ? 1 : 2);
        for (int side = 0; side < 2; ++side) {
            res->cells.push_back(s2[i]);
            int64_t d[3] = {cc[0], cc[1], cc[2]};
            d[axis] += side ? 1 : -1;
            if (g.inside(d[0], d[1], d[2])) {
                int64_t c = g.cell(d[0], d[1], d[2]);
                res->cells.push_back(uint32_t(c));
                for (int64_t steps = 0;; ++steps) {
                    uint32_t q = pair_of[c];
                    if (q == NONE) break;  // a maximum
                    if (steps > limit) { res->status = ERR_INTERNAL; return res; }
                    res->cells.push_back(q);
                    int64_t cx, cy, cz, qx, qy, qz;
                    g.coords(c, cx, cy, cz);
                    g.coords(int64_t(q), qx, qy, qz);
                    int64_t ax = 2 * qx - cx, ay = 2 * qy - cy, az = 2 * qz - cz;  // across the quad
                    if (!g.inside(ax, ay, az)) break;  // R4: the path leaves the domain here
                    c = g.cell(ax, ay, az);
                    res->cells.push_back(uint32_t(c));
                }
            }
            res->offsets.push_back(int64_t(res->cells.size()));
        }
    }
    return res;
}

// Cells along the saddle-saddle arcs of multiplicity 1 (Sec. 3.3 and Sec. 3.5 "Data structure").
// A D* entry (s, t) with count 1 is a single V-path from the 2-saddle t down to the 1-saddle s, so
// it has one cell sequence; an entry with a larger count stands for several paths and gets none.
// The path is walked from s along the DAG (Sec. 3.2), at each node taking the one successor from
// which t can still be reached; the cells are s, then for each step to a 1-cell e' the quad paired
// with e' followed by e', and finally t.  The paths from a node to t are counted by a memoised
// depth-first search over the DAG (saturating at 2: only "none", "one" and "several" matter).
// Entries come as the D* CSR (rowptr over 1-saddle ranks, 2-saddle rank columns, counts) and the
// offsets follow its entry order.
void* ora_ss_arc_cells(const int64_t* dims, const uint32_t* pair_of, int64_t n1, const uint32_t* s1, int64_t n2,
                       const uint32_t* s2, const int64_t* rowptr, const uint32_t* col, const uint64_t* cnt) {
    ArcCells* res = new ArcCells();
    if (!check_dims(dims) || !pair_of || n1 < 0 || n2 < 0 || (n1 > 0 && (!s1 || !rowptr)) || (n2 > 0 && !s2)) {
        res->status = ERR_ARG;
        return res;
    }
    Grid g(dims, nullptr);
    const int64_t limit = g.ncells();
    res->offsets.push_back(0);
    for (int64_t i = 0; i < n1; ++i) {
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            if (cnt[k] == 1) {
                if (int64_t(col[k]) >= n2) { res->status = ERR_ARG; return res; }
                const int64_t s = int64_t(s1[i]), t = int64_t(s2[col[k]]);
                std::map<int64_t, uint64_t> memo;  // node -> paths to t, capped at 2
                bool bad = false;
                // the count of a node that needs no search: t itself, another 2-saddle, or memoised
                auto known = [&](int64_t y, uint64_t& v) {
                    if (y == t) { v = 1; return true; }
                    if (g.dim(y) != 1) { v = 0; return true; }
                    auto it = memo.find(y);
                    if (it == memo.end()) return false;
                    v = it->second;
                    return true;
                };
                auto paths_to_t = [&](int64_t start) -> uint64_t {
                    uint64_t v;
                    if (known(start, v)) return v;
                    struct Frame { int64_t x; std::vector<int64_t> out; size_t next; uint64_t n; };
                    std::vector<Frame> st;
                    st.push_back(Frame{start, dag_out(g, pair_of, start), 0, 0});
                    for (int64_t steps = 0; !st.empty(); ++steps) {
                        if (steps > 8 * limit) { bad = true; return 0; }  // a cycle: cannot happen
                        if (st.back().next < st.back().out.size()) {
                            const int64_t y = st.back().out[st.back().next];
                            if (known(y, v)) {
                                st.back().n = std::min<uint64_t>(2, st.back().n + v);
                                ++st.back().next;
                            } else {
                                st.push_back(Frame{y, dag_out(g, pair_of, y), 0, 0});
                            }
                        } else {
                            const uint64_t done = st.back().n;
                            memo[st.back().x] = done;
                            st.pop_back();
                            if (!st.empty()) {
                                st.back().n = std::min<uint64_t>(2, st.back().n + done);
                                ++st.back().next;
                            }
                        }
                    }
                    return memo[start];
                };
                if (paths_to_t(s) != 1 || bad) { res->status = ERR_INTERNAL; return res; }
                res->cells.push_back(uint32_t(s));
                int64_t e = s;
                for (int64_t steps = 0;; ++steps) {
                    if (steps > limit) { res->status = ERR_INTERNAL; return res; }
                    int64_t next = -1;
                    int found = 0;
                    for (int64_t y : dag_out(g, pair_of, e))
                        if (paths_to_t(y) > 0) { next = y; ++found; }
                    if (found != 1 || bad) { res->status = ERR_INTERNAL; return res; }
                    if (next == t) { res->cells.push_back(uint32_t(t)); break; }
                    res->cells.push_back(pair_of[next]);  // the quad between e and next
                    res->cells.push_back(uint32_t(next));
                    e = next;
                }
            }
            res->offsets.push_back(int64_t(res->cells.size()));
        }
    }
    return res;
}

int ora_arc_status(void* h) { return static_cast<ArcCells*>(h)->status; }
int64_t ora_arc_count(void* h) { return int64_t(static_cast<ArcCells*>(h)->offsets.size()) - 1; }
int64_t ora_arc_cells_size(void* h) { return int64_t(static_cast<ArcCells*>(h)->cells.size()); }
void ora_arc_copy(void* h, int64_t* offsets, uint32_t* cells) {
    ArcCells* r = static_cast<ArcCells*>(h);
    std::copy(r->offsets.begin(), r->offsets.end(), offsets);
    std::copy(r->cells.begin(), r->cells.end(), cells);
}
void ora_arc_free(void* h) { delete static_cast<ArcCells*>(h); }

// Saddle-saddle reachability (Sec. 3.2): multi-source BFS over the DAG from all 1-saddles.
// visited[v] bit a (a = 0,1,2) marks the 1-cell of vertex v along axis a as reachable
// (the 1-saddles themselves included).  Returns the number of non-empty BFS levels
// (level 0 = the 1-saddles), or -status on error.
int64_t ora_reachable(const int64_t* dims, const uint32_t* pair_of, uint8_t* visited) {
    if (!check_dims(dims) || !pair_of || !visited) return -ERR_ARG;
    Grid g(dims, nullptr);
    std::memset(visited, 0, size_t(g.nverts()));
    std::vector<int64_t> frontier = critical_list(g, pair_of, 1), next;
    for (int64_t e : frontier) {
        int axis;
        int64_t v = one_cell_slot(g, e, axis);
        visited[v] |= uint8_t(1u << axis);
    }
    int64_t levels = 0;
    while (!frontier.empty()) {
        ++levels;
        next.clear();
        for (int64_t e : frontier)
            for (int64_t t : dag_out(g, pair_of, e)) {
                if (g.dim(t) != 1) continue;
                int axis;
                int64_t v = one_cell_slot(g, t, axis);
                if ((visited[v] >> axis) & 1) continue;
                visited[v] |= uint8_t(1u << axis);
                next.push_back(t);
            }
        frontier.swap(next);
    }
    return levels;
}

// Junction nodes (R5), in cell-id order.  Returns the count; out may be null.
int64_t ora_junctions(const int64_t* dims, const uint32_t* pair_of, const uint8_t* visited, uint32_t* out) {
    if (!check_dims(dims) || !pair_of || !visited) return -ERR_ARG;
    Grid g(dims, nullptr);
    int64_t n = 0;
    for (int64_t c = 0; c < g.ncells(); ++c) {
        if (g.dim(c) != 1 || pair_of[c] == NONE) continue;
        if (!visited_get(g, visited, c)) continue;
        if (dag_out(g, pair_of, c).size() > 1) {
            if (out) out[n] = uint32_t(c);
            ++n;
        }
    }
    return n;
}

// DAG minor (Sec. 3.3 "DAG minor construction"): from every out-edge of every 1-saddle and
// junction, follow the unique successor while the node is neither a junction nor a
// 2-saddle; a node without successors ends a dead path, which is dropped.  Each traced
// path adds 1 to the multiplicity of its (source, destination) entry in A (1s->j),
// B (j->j), B* (j->2s) or D (1s->2s).  The four matrices are kept behind a handle; each
// is read back sorted by (row, col).
void* ora_minor(const int64_t* dims, const uint32_t* pair_of, int64_t n1, const uint32_t* s1, int64_t nj,
                const uint32_t* junc, int64_t n2, const uint32_t* s2) {
    Minor* mn = new Minor();
    if (!check_dims(dims) || !pair_of) {
        mn->status = ERR_ARG;
        return mn;
    }
    Grid g(dims, nullptr);
    std::vector<int64_t> L1(s1, s1 + n1), LJ(junc, junc + nj), L2(s2, s2 + n2);
    std::unordered_set<int64_t> jset(LJ.begin(), LJ.end());
    auto trace_from = [&](int64_t u, bool u_is_saddle) {
        int64_t urank = u_is_saddle ? rank_in(L1, u) : rank_in(LJ, u);
        for (int64_t w : dag_out(g, pair_of, u)) {
            for (int64_t steps = 0;; ++steps) {
                if (steps > g.ncells()) {  // longer than any simple path: the DAG has a cycle
                    mn->status = ERR_INTERNAL;
                    return;
                }
                if (g.dim(w) == 2) {  // a 2-saddle
                    mn->m[u_is_saddle ? 3 : 2][{urank, rank_in(L2, w)}] += 1;
                    break;
                }
                if (jset.count(w)) {
                    mn->m[u_is_saddle ? 0 : 1][{urank, rank_in(LJ, w)}] += 1;
                    break;
                }
                std::vector<int64_t> nxt = dag_out(g, pair_of, w);
                if (nxt.empty()) break;  // dead path
                w = nxt[0];
            }
        }
    };
    for (int64_t u : L1) trace_from(u, true);
    for (int64_t u : LJ) trace_from(u, false);
    return mn;
}

int ora_minor_status(void* h) { return static_cast<Minor*>(h)->status; }

int64_t ora_minor_size(void* h, int which) { return int64_t(static_cast<Minor*>(h)->m[which].size()); }

void ora_minor_copy(void* h, int which, uint32_t* rows, uint32_t* cols, uint64_t* mult) {
    int64_t i = 0;
    for (const auto& kv : static_cast<Minor*>(h)->m[which]) {
        rows[i] = uint32_t(kv.first.first);
        cols[i] = uint32_t(kv.first.second);
        mult[i] = kv.second;
        ++i;
    }
}

void ora_minor_free(void* h) { delete static_cast<Minor*>(h); }

// Saddle-saddle path counts D* (O5): for each requested 1-saddle s (by rank in s1), collect
// the DAG nodes reachable from s, visit them in topological order (Kahn) with cnt[s] = 1
// and cnt[w] += cnt[v] along every edge, and emit (rank(s), rank(t), cnt[t]) for every
// 2-saddle t with cnt > 0.  Results are kept behind a handle, sorted by (row, col).
struct PathCounts {
    std::vector<uint32_t> rows, cols;
    std::vector<uint64_t> counts;
    int status = OK;
};

void* ora_path_counts(const int64_t* dims, const uint32_t* pair_of, int64_t n1, const uint32_t* s1, int64_t n2,
                      const uint32_t* s2, int64_t nsrc, const int64_t* src_ranks) {
    PathCounts* res = new PathCounts();
    if (!check_dims(dims) || !pair_of) { res->status = ERR_ARG; return res; }
    Grid g(dims, nullptr);
    std::vector<int64_t> L2(s2, s2 + n2);
    std::vector<int64_t> order;
    if (src_ranks) order.assign(src_ranks, src_ranks + nsrc);
    else for (int64_t i = 0; i < n1; ++i) order.push_back(i);
    std::sort(order.begin(), order.end());
    std::vector<int64_t> stack;
    for (int64_t r : order) {
        if (r < 0 || r >= n1) { res->status = ERR_ARG; return res; }
        int64_t s = int64_t(s1[r]);
        // reachable set R(s) and in-degrees within it
        std::unordered_map<int64_t, int64_t> indeg;
        std::unordered_set<int64_t> seen{s};
        stack.assign(1, s);
        while (!stack.empty()) {
            int64_t v = stack.back();
            stack.pop_back();
            if (g.dim(v) != 1) continue;  // 2-saddles are sinks
            for (int64_t w : dag_out(g, pair_of, v)) {
                indeg[w] += 1;
                if (seen.insert(w).second) stack.push_back(w);
            }
        }
        // Kahn's order from s
        std::unordered_map<int64_t, uint64_t> cnt;
        cnt[s] = 1;
        std::vector<int64_t> queue{s};
        std::map<int64_t, uint64_t> row;  // 2-saddle rank -> count
        for (size_t qi = 0; qi < queue.size(); ++qi) {
            int64_t v = queue[qi];
            uint64_t cv = cnt[v];
            if (g.dim(v) == 2) {
                if (cv > 0) row[rank_in(L2, v)] = cv;
                continue;
            }
            for (int64_t w : dag_out(g, pair_of, v)) {
                uint64_t before = cnt[w];
                uint64_t after = before + cv;
                if (after < before) { res->status = ERR_OVERFLOW; return res; }  // R6
                cnt[w] = after;
                if (--indeg[w] == 0) queue.push_back(w);
            }
        }
        for (const auto& kv : row) {
            res->rows.push_back(uint32_t(r));
            res->cols.push_back(uint32_t(kv.first));
            res->counts.push_back(kv.second);
        }
    }
    return res;
}

int ora_result_status(void* h) { return static_cast<PathCounts*>(h)->status; }
int64_t ora_result_size(void* h) { return int64_t(static_cast<PathCounts*>(h)->rows.size()); }
void ora_result_copy(void* h, uint32_t* rows, uint32_t* cols, uint64_t* counts) {
    PathCounts* r = static_cast<PathCounts*>(h);
    std::copy(r->rows.begin(), r->rows.end(), rows);
    std::copy(r->cols.begin(), r->cols.end(), cols);
    std::copy(r->counts.begin(), r->counts.end(), counts);
}
void ora_result_free(void* h) { delete static_cast<PathCounts*>(h); }

// Number of non-zero iterates A_k = A B^k (k >= 0) of the paper's product loop: the length,
// in minor edges, of the longest minor path that starts with an A edge and stays among
// junctions.  Computed by longest-path DP over the B edges, given A and B as COO lists.
int64_t ora_n_iter(int64_t nj, int64_t nnzA, const uint32_t* Acols, int64_t nnzB, const uint32_t* Brows,
                   const uint32_t* Bcols) {
    std::vector<std::vector<int64_t>> succ(static_cast<size_t>(nj));
    std::vector<int64_t> indeg(static_cast<size_t>(nj), 0), depth(static_cast<size_t>(nj), 0);
    for (int64_t i = 0; i < nnzB; ++i) {
        succ[Brows[i]].push_back(Bcols[i]);
        indeg[Bcols[i]]++;
    }
    for (int64_t i = 0; i < nnzA; ++i) depth[Acols[i]] = 1;
    std::vector<int64_t> queue;
    for (int64_t j = 0; j < nj; ++j)
        if (indeg[j] == 0) queue.push_back(j);
    int64_t best = 0;
    for (size_t qi = 0; qi < queue.size(); ++qi) {
        int64_t j = queue[qi];
        best = std::max(best, depth[j]);
        for (int64_t k : succ[j]) {
            if (depth[j] > 0) depth[k] = std::max(depth[k], depth[j] + 1);
            if (--indeg[k] == 0) queue.push_back(k);
        }
    }
    return best;
}


// ---- sampled queries (LazyPairs) ------------------------------------------------------
// For each listed cell: the partner id (0xFFFFFFFF = critical).
int ora_lazy_pairs(const int64_t* dims, const float* f, int64_t n, const uint32_t* cells, uint32_t* out) {
    if (!check_dims(dims) || !f || (n > 0 && (!cells || !out))) return ERR_ARG;
    Grid g(dims, f);
    if (!ids_fit_u32(g)) return ERR_TOO_LARGE;
    LazyPairs lp(g);
    for (int64_t i = 0; i < n; ++i) {
        if (int64_t(cells[i]) >= g.ncells()) return ERR_ARG;
        out[i] = lp(int64_t(cells[i]));
    }
    return lp.status;
}

// Destination minimum (cell id) of each listed vertex: the descending walk of Sec. 3.4.
int ora_lazy_vertex_min(const int64_t* dims, const float* f, int64_t n, const int64_t* verts, uint32_t* out) {
    if (!check_dims(dims) || !f || (n > 0 && (!verts || !out))) return ERR_ARG;
    Grid g(dims, f);
    LazyPairs lp(g);
    for (int64_t i = 0; i < n; ++i) {
        int64_t v = verts[i];
        for (int64_t steps = 0;; ++steps) {
            if (steps > g.nverts()) return ERR_INTERNAL;
            const int64_t vc = g.vertex_cell(v);
            const uint32_t e = lp(vc);
            if (e == NONE) {
                out[i] = uint32_t(vc);
                break;
            }
            int64_t other = -1;
            for (int64_t w : g.vertices(int64_t(e)))
                if (w != v) other = w;
            v = other;
        }
    }
    return lp.status;
}

// Destination maximum (cell id, NONE if the walk leaves the domain) of the cube owned by each
// listed vertex (NONE where the vertex owns no cube): the ascending walk of Sec. 3.4.
int ora_lazy_cube_max(const int64_t* dims, const float* f, int64_t n, const int64_t* verts, uint32_t* out) {
    if (!check_dims(dims) || !f || (n > 0 && (!verts || !out))) return ERR_ARG;
    Grid g(dims, f);
    LazyPairs lp(g);
    for (int64_t i = 0; i < n; ++i) {
        const int64_t v = verts[i];
        const int64_t x = v % g.nx, y = (v / g.nx) % g.ny, z = v / (g.nx * g.ny);
        if (x == g.nx - 1 || y == g.ny - 1 || z == g.nz - 1) {
            out[i] = NONE;
            continue;
        }
        int64_t c = g.cell(2 * x + 1, 2 * y + 1, 2 * z + 1);
        for (int64_t steps = 0;; ++steps) {
            if (steps > g.nverts()) return ERR_INTERNAL;
            const uint32_t p = lp(c);
            if (p == NONE) {
                out[i] = uint32_t(c);
                break;
            }
            int64_t cx, cy, cz, px, py, pz;
            g.coords(c, cx, cy, cz);
            g.coords(int64_t(p), px, py, pz);
            const int64_t nxc = 2 * px - cx, nyc = 2 * py - cy, nzc = 2 * pz - cz;
            if (!g.inside(nxc, nyc, nzc)) {
                out[i] = NONE;
                break;
            }
            c = g.cell(nxc, nyc, nzc);
        }
    }
    return lp.status;
}

// DAG facts of each listed 1-cell: out[3i] = 1 if it is a DAG node (critical or paired with a
// quad), out[3i+1] = 1 if it is critical, out[3i+2] = its out-degree (0 if not a node).
int ora_lazy_nodes(const int64_t* dims, const float* f, int64_t n, const uint32_t* cells, int32_t* out) {
    if (!check_dims(dims) || !f || (n > 0 && (!cells || !out))) return ERR_ARG;
    Grid g(dims, f);
    LazyPairs lp(g);
    for (int64_t i = 0; i < n; ++i) {
        const int64_t e = cells[i];
        if (g.dim(e) != 1) return ERR_ARG;
        const uint32_t p = lp(e);
        const bool node = p == NONE || g.dim(int64_t(p)) == 2;
        out[3 * i] = node;
        out[3 * i + 1] = p == NONE;
        out[3 * i + 2] = node ? int32_t(dag_out_p(g, lp, e).size()) : 0;
    }
    return lp.status;
}

// D* rows of listed 1-saddles (O5 on the lazily paired DAG): entries (sample index, 2-saddle
// cell id, count), sorted by (sample, cell id).  Kept behind a handle like ora_path_counts.
void* ora_lazy_dstar_rows(const int64_t* dims, const float* f, int64_t n, const uint32_t* s1_cells) {
    PathCounts* res = new PathCounts();
    if (!check_dims(dims) || !f || (n > 0 && !s1_cells)) {
        res->status = ERR_ARG;
        return res;
    }
    Grid g(dims, f);
    LazyPairs lp(g);
    for (int64_t r = 0; r < n; ++r) {
        const int64_t s = s1_cells[r];
        if (g.dim(s) != 1 || lp(s) != NONE) {
            res->status = ERR_ARG;  // not a 1-saddle
            return res;
        }
        std::unordered_map<int64_t, int64_t> indeg;
        std::unordered_set<int64_t> seen{s};
        std::vector<int64_t> stack{s};
        while (!stack.empty()) {
            const int64_t v = stack.back();
            stack.pop_back();
            if (g.dim(v) != 1) continue;
            for (int64_t w : dag_out_p(g, lp, v)) {
                indeg[w] += 1;
                if (seen.insert(w).second) stack.push_back(w);
            }
        }
        std::unordered_map<int64_t, uint64_t> cnt;
        cnt[s] = 1;
        std::vector<int64_t> queue{s};
        std::map<int64_t, uint64_t> row;
        for (size_t qi = 0; qi < queue.size(); ++qi) {
            const int64_t v = queue[qi];
            const uint64_t cv = cnt[v];
            if (g.dim(v) == 2) {
                if (cv > 0) row[v] = cv;
                continue;
            }
            for (int64_t w : dag_out_p(g, lp, v)) {
                const uint64_t before = cnt[w], after = before + cv;
                if (after < before) {
                    res->status = ERR_OVERFLOW;
                    return res;
                }
                cnt[w] = after;
                if (--indeg[w] == 0) queue.push_back(w);
            }
        }
        for (const auto& kv : row) {
            res->rows.push_back(uint32_t(r));
            res->cols.push_back(uint32_t(kv.first));
            res->counts.push_back(kv.second);
        }
    }
    if (lp.status) res->status = lp.status;
    return res;
}

// ---------------------------------------------------------------------------------
// Persistence-ordered simplification of the 1-skeleton (Sec. 4 "Parallel Simplification",
// "Grid subdivision": the cancellation it performs in each subgrid, here serially over the whole
// complex).  Nodes are critical cells with their index (dimension) and value; an arc joins
// nodes of consecutive index and carries a multiplicity (the number of gradient paths).
//   S1 value of a critical cell = the value of its highest vertex (the vertex whose lower star
//      holds it); persistence of an arc = value(upper) - value(lower), never negative for an arc
//      of the complex, taken as an absolute difference here.
//   S2 a pair (p, q), index(p) = index(q) + 1, may be cancelled iff both are alive and exactly one
//      arc joins them (several arcs: a strangulation, Sec. 4).
//   S3 order: the least valid arc by (persistence, cell id of its upper node, cell id of its lower
//      node) is cancelled next, while its persistence <= threshold.
//   S4 cancelling (p, q): every node a joined to p by m_pa arcs (a != q, index(q)) and every node
//      b joined to q by m_qb arcs (b != p, index(p)) gain m_pa * m_qb arcs between b and a (the
//      descending arcs of p rerouted to the ends of the ascending arcs of q); then p, q and all
//      their arcs are removed.  Multiplicities are exact uint64 (an overflow is status 6).
// A multiplicity only grows while its arc lives, so an arc that is not valid when it is the least
// one never becomes valid later: a key-ordered set with lazy deletion gives exactly "repeatedly
// cancel the least valid arc".
struct Simplified {
    std::vector<uint32_t> log_upper, log_lower;  // cancelled pairs, in order (node indices)
    std::vector<double> log_persistence;
    std::vector<uint32_t> arc_u, arc_v;          // surviving arcs, u < v (node indices)
    std::vector<uint64_t> arc_mult;
    std::vector<uint8_t> alive;
    int status = OK;
};

void* ora_simplify(int64_t n_nodes, const int32_t* index, const double* value, const uint32_t* cell,
                   int64_t n_arcs, const uint32_t* arc_u, const uint32_t* arc_v, const uint64_t* arc_mult,
                   double threshold) {
    Simplified* res = new Simplified();
    if (n_nodes < 0 || n_arcs < 0 || (n_nodes > 0 && (!index || !value || !cell)) ||
        (n_arcs > 0 && (!arc_u || !arc_v || !arc_mult))) {
        res->status = ERR_ARG;
        return res;
    }
    std::vector<std::map<int64_t, uint64_t>> adj(static_cast<size_t>(n_nodes));
    for (int64_t i = 0; i < n_arcs; ++i) {
        const int64_t u = arc_u[i], v = arc_v[i];
        if (u < 0 || v < 0 || u >= n_nodes || v >= n_nodes || u == v || std::abs(index[u] - index[v]) != 1) {
            res->status = ERR_ARG;
            return res;
        }
        adj[size_t(u)][v] += arc_mult[i];
        adj[size_t(v)][u] += arc_mult[i];
    }
    std::vector<uint8_t> alive(size_t(n_nodes), 1);
    // key: (persistence, upper cell, lower cell) -> (upper node, lower node)
    using Key = std::tuple<double, uint32_t, uint32_t, int64_t, int64_t>;
    auto key_of = [&](int64_t a, int64_t b) {
        const int64_t up = index[a] > index[b] ? a : b, lo = up == a ? b : a;
        return Key(std::fabs(value[up] - value[lo]), cell[up], cell[lo], up, lo);
    };
    std::set<Key> queue;
    for (int64_t u = 0; u < n_nodes; ++u)
        for (const auto& kv : adj[size_t(u)])
            if (u < kv.first) queue.insert(key_of(u, kv.first));
    while (!queue.empty()) {
        const Key k = *queue.begin();
        queue.erase(queue.begin());
        if (std::get<0>(k) > threshold) break;
        const int64_t p = std::get<3>(k), q = std::get<4>(k);
        if (!alive[size_t(p)] || !alive[size_t(q)]) continue;
        auto it = adj[size_t(p)].find(q);
        if (it == adj[size_t(p)].end() || it->second != 1) continue;  // S2
        std::vector<std::pair<int64_t, uint64_t>> down, up;
        for (const auto& kv : adj[size_t(p)])
            if (kv.first != q && index[kv.first] == index[q]) down.push_back(kv);
        for (const auto& kv : adj[size_t(q)])
            if (kv.first != p && index[kv.first] == index[p]) up.push_back(kv);
        for (const auto& a : down)
            for (const auto& b : up) {
                const uint64_t add = a.second * b.second;
                if (b.second != 0 && add / b.second != a.second) { res->status = ERR_OVERFLOW; return res; }
                uint64_t& m = adj[size_t(b.first)][a.first];
                if (m + add < m) { res->status = ERR_OVERFLOW; return res; }
                m += add;
                adj[size_t(a.first)][b.first] = m;
                queue.insert(key_of(b.first, a.first));
            }
        for (int64_t x : {p, q}) {
            for (const auto& kv : adj[size_t(x)]) adj[size_t(kv.first)].erase(x);
            adj[size_t(x)].clear();
            alive[size_t(x)] = 0;
        }
        res->log_upper.push_back(uint32_t(p));
        res->log_lower.push_back(uint32_t(q));
        res->log_persistence.push_back(std::get<0>(k));
    }
    for (int64_t u = 0; u < n_nodes; ++u)
        for (const auto& kv : adj[size_t(u)])
            if (u < kv.first) {
                res->arc_u.push_back(uint32_t(u));
                res->arc_v.push_back(uint32_t(kv.first));
                res->arc_mult.push_back(kv.second);
            }
    res->alive = alive;
    return res;
}

int ora_simplify_status(void* h) { return static_cast<Simplified*>(h)->status; }
int64_t ora_simplify_cancelled(void* h) { return int64_t(static_cast<Simplified*>(h)->log_upper.size()); }
int64_t ora_simplify_arcs(void* h) { return int64_t(static_cast<Simplified*>(h)->arc_u.size()); }
void ora_simplify_copy(void* h, uint32_t* log_upper, uint32_t* log_lower, double* log_persistence, uint8_t* alive,
                       uint32_t* arc_u, uint32_t* arc_v, uint64_t* arc_mult) {
    Simplified* r = static_cast<Simplified*>(h);
    std::copy(r->log_upper.begin(), r->log_upper.end(), log_upper);
    std::copy(r->log_lower.begin(), r->log_lower.end(), log_lower);
    std::copy(r->log_persistence.begin(), r->log_persistence.end(), log_persistence);
    std::copy(r->alive.begin(), r->alive.end(), alive);
    std::copy(r->arc_u.begin(), r->arc_u.end(), arc_u);
    std::copy(r->arc_v.begin(), r->arc_v.end(), arc_v);
    std::copy(r->arc_mult.begin(), r->arc_mult.end(), arc_mult);
}
void ora_simplify_free(void* h) { delete static_cast<Simplified*>(h); }

// ---------------------------------------------------------------------------------
// Simplification in rounds of independent cancellations (the data-parallel scheme Sec. 4
// "Discussion" describes: an independent set of arcs under the 3-link neighbourhood, cancelled
// together).  Same keys (S3), validity (S2) and cancellation (S4) as ora_simplify; the order is:
//   S5 a round cancels every valid arc (persistence <= threshold) whose key is the least among the
//      valid arcs that have an endpoint within two links of one of its endpoints; rounds repeat
//      until no valid arc is left.
// Two arcs selected in one round are more than two links apart, so the nodes whose arcs each
// cancellation changes (the two ends and their neighbours) are disjoint and the round's
// cancellations do not depend on their order; the globally least valid arc is always selected.
// The round structure is kept: round_of_log[i] is the round of the i-th cancellation.
struct Rounds : Simplified {
    std::vector<uint32_t> round_of_log;
    int64_t rounds = 0;
};

void* ora_simplify_rounds(int64_t n_nodes, const int32_t* index, const double* value, const uint32_t* cell,
                          int64_t n_arcs, const uint32_t* arc_u, const uint32_t* arc_v, const uint64_t* arc_mult,
                          double threshold) {
    Rounds* res = new Rounds();
    if (n_nodes < 0 || n_arcs < 0 || (n_nodes > 0 && (!index || !value || !cell)) ||
        (n_arcs > 0 && (!arc_u || !arc_v || !arc_mult))) {
        res->status = ERR_ARG;
        return res;
    }
    std::vector<std::map<int64_t, uint64_t>> adj(static_cast<size_t>(n_nodes));
    for (int64_t i = 0; i < n_arcs; ++i) {
        const int64_t u = arc_u[i], v = arc_v[i];
        if (u < 0 || v < 0 || u >= n_nodes || v >= n_nodes || u == v || std::abs(index[u] - index[v]) != 1) {
            res->status = ERR_ARG;
            return res;
        }
        adj[size_t(u)][v] += arc_mult[i];
        adj[size_t(v)][u] += arc_mult[i];
    }
    std::vector<uint8_t> alive(size_t(n_nodes), 1);
    using Key = std::tuple<double, uint32_t, uint32_t>;
    const Key NO_KEY(HUGE_VAL, 0xFFFFFFFFu, 0xFFFFFFFFu);
    while (true) {
        // the valid arcs and, per node, the least key of the valid arcs incident on it
        std::vector<std::tuple<Key, int64_t, int64_t>> valid;
        std::vector<Key> m0(size_t(n_nodes), NO_KEY);
        for (int64_t p = 0; p < n_nodes; ++p) {
            if (!alive[size_t(p)]) continue;
            for (const auto& kv : adj[size_t(p)]) {
                const int64_t q = kv.first;
                if (!alive[size_t(q)] || index[p] != index[q] + 1 || kv.second != 1) continue;
                const double pers = std::fabs(value[p] - value[q]);
                if (pers > threshold) continue;
                const Key k(pers, cell[p], cell[q]);
                valid.emplace_back(k, p, q);
                m0[size_t(p)] = std::min(m0[size_t(p)], k);
                m0[size_t(q)] = std::min(m0[size_t(q)], k);
            }
        }
        if (valid.empty()) break;
        // least key within one, then two links (closed neighbourhoods)
        std::vector<Key> m1 = m0, m2;
        for (int64_t u = 0; u < n_nodes; ++u)
            for (const auto& kv : adj[size_t(u)]) m1[size_t(u)] = std::min(m1[size_t(u)], m0[size_t(kv.first)]);
        m2 = m1;
        for (int64_t u = 0; u < n_nodes; ++u)
            for (const auto& kv : adj[size_t(u)]) m2[size_t(u)] = std::min(m2[size_t(u)], m1[size_t(kv.first)]);
        std::vector<std::pair<int64_t, int64_t>> picked;
        std::vector<std::tuple<Key, int64_t, int64_t>> chosen;
        for (const auto& t : valid) {
            const int64_t p = std::get<1>(t), q = std::get<2>(t);
            if (std::get<0>(t) == std::min(m2[size_t(p)], m2[size_t(q)])) chosen.push_back(t);
        }
        // the footprints (both ends and their neighbours) must be disjoint
        std::vector<uint8_t> touched(size_t(n_nodes), 0);
        for (const auto& t : chosen) {
            const int64_t p = std::get<1>(t), q = std::get<2>(t);
            std::set<int64_t> fp{p, q};
            for (const auto& kv : adj[size_t(p)]) fp.insert(kv.first);
            for (const auto& kv : adj[size_t(q)]) fp.insert(kv.first);
            for (int64_t x : fp) {
                if (touched[size_t(x)]) { res->status = ERR_INTERNAL; return res; }
                touched[size_t(x)] = 1;
            }
        }
        for (const auto& t : chosen) {
            const int64_t p = std::get<1>(t), q = std::get<2>(t);
            std::vector<std::pair<int64_t, uint64_t>> down, up;
            for (const auto& kv : adj[size_t(p)])
                if (kv.first != q && index[kv.first] == index[q]) down.push_back(kv);
            for (const auto& kv : adj[size_t(q)])
                if (kv.first != p && index[kv.first] == index[p]) up.push_back(kv);
            for (const auto& a : down)
                for (const auto& b : up) {
                    const uint64_t add = a.second * b.second;
                    if (b.second != 0 && add / b.second != a.second) { res->status = ERR_OVERFLOW; return res; }
                    uint64_t& m = adj[size_t(b.first)][a.first];
                    if (m + add < m) { res->status = ERR_OVERFLOW; return res; }
                    m += add;
                    adj[size_t(a.first)][b.first] = m;
                }
            for (int64_t x : {p, q}) {
                for (const auto& kv : adj[size_t(x)]) adj[size_t(kv.first)].erase(x);
                adj[size_t(x)].clear();
                alive[size_t(x)] = 0;
            }
            res->log_upper.push_back(uint32_t(p));
            res->log_lower.push_back(uint32_t(q));
            res->log_persistence.push_back(std::get<0>(std::get<0>(t)));
            res->round_of_log.push_back(uint32_t(res->rounds));
        }
        ++res->rounds;
    }
    for (int64_t u = 0; u < n_nodes; ++u)
        for (const auto& kv : adj[size_t(u)])
            if (u < kv.first) {
                res->arc_u.push_back(uint32_t(u));
                res->arc_v.push_back(uint32_t(kv.first));
                res->arc_mult.push_back(kv.second);
            }
    res->alive = alive;
    return res;
}

int64_t ora_simplify_rounds_count(void* h) { return static_cast<Rounds*>(h)->rounds; }
void ora_simplify_rounds_of(void* h, uint32_t* round_of_log) {
    Rounds* r = static_cast<Rounds*>(h);
    std::copy(r->round_of_log.begin(), r->round_of_log.end(), round_of_log);
}

}  // extern "C"
