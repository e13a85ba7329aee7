// The DAG of 1-2 gradient pairs (Sec. 3.2, Fig. "msc-max-min-dag" (d)), read straight from
// the packed gradient words.
//
// Nodes are 1-cells (1-saddles and 1-cells paired with a quad) and 2-saddles.  For a 1-cell e,
// each cofacet quad q other than e's own partner gives an out-edge: to q itself if q is
// critical (a 2-saddle), to the 1-cell that q is paired with if q is paired with a facet, and
// nothing if q is paired with a cube.  Following an out-edge walks a V-path backwards, so
// traversals move against the gradient (Sec. 3.5).  Out-degree <= 4 (Sec. 3.2).
//
// A 1-cell is named by its owner vertex and axis: handle = (vertex index << 2) | axis, where
// the cell is (2x+1,2y,2z), (2x,2y+1,2z) or (2x,2y,2z+1) for axis 0, 1, 2.  A 2-saddle target
// is named by its owner vertex and slot.  All index arithmetic is 32-bit: a plan's cell ids
// fit in 32 bits, so its vertex count is below 2^29.
#pragma once

#include "geom.cuh"

namespace msc {

struct DagTarget {
    uint32_t v;    // owner vertex index
    int x, y, z;   // owner vertex coordinates
    uint8_t kind;  // 1 = 1-cell (then `sub` is its axis), 2 = 2-saddle (then `sub` is its slot)
    uint8_t sub;
};

__host__ __device__ __forceinline__ uint32_t edge_handle(uint32_t v, int axis) { return (v << 2) | uint32_t(axis); }

struct Vtx {
    int x, y, z;
};

__host__ __device__ __forceinline__ Vtx vtx_of(const Geom& g, uint32_t v) {
    Vtx r;
    const uint32_t q = g.div_nx.div(v);
    r.x = int(v - q * uint32_t(g.nx));
    r.z = int(g.div_ny.div(q));
    r.y = int(q - uint32_t(r.z) * uint32_t(g.ny));
    return r;
}

__host__ __device__ __forceinline__ uint32_t vid32(const Geom& g, int x, int y, int z) {
    return uint32_t(x) + uint32_t(g.nx) * (uint32_t(y) + uint32_t(g.ny) * uint32_t(z));
}

// Slot of the 1-cell along `axis` in its owner's word: a=1 (slot 1), b=1 (slot 2), c=1 (slot 4).
__host__ __device__ __forceinline__ int edge_slot(int axis) { return 1 << axis; }

// Word index of a 1-cell in the 1-cell row bitmap layout (see Geom::edge_word); bit x & 31.
__host__ __device__ __forceinline__ int64_t edge_bitmap_word(const Geom& g, int x, int y, int z, int axis) {
    return g.edge_word(z, axis == 2, y, axis == 1, x >> 5);
}

// Out-edges of the 1-cell of vertex (x,y,z) along `axis`, one slot per cofacet quad: the quads
// are e +- u_b for the two axes b != axis (slots 0,1 for the first such b, 2,3 for the second);
// the quad on the + side of b shares e's owner, the one on the - side is owned by the vertex
// one step back along b.  A slot without an edge has kind 0.  Returns the number of edges.
// (Fixed slots keep the targets in registers.)
__host__ __device__ __forceinline__ int pick3(int i, int a0, int a1, int a2) { return i == 0 ? a0 : i == 1 ? a1 : a2; }

__host__ __device__ __forceinline__ int dag_out(const Geom& g, const uint32_t* __restrict__ words, int x, int y, int z,
                                                int axis, DagTarget out[4]) {
    const uint32_t v = vid32(g, x, y, z);
    const uint32_t sy = uint32_t(g.nx), sz = uint32_t(g.nx) * uint32_t(g.ny);
    const uint32_t own = slot_code(words[v], edge_slot(axis));
    int cnt = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int b = axis + 1 + (i >> 1) - (axis + 1 + (i >> 1) >= 3 ? 3 : 0);  // the two axes other than `axis`
        const bool plus = i & 1;
        const int other = 3 - axis - b;  // the quad's even axis
        out[i].kind = 0;
        const int cb = pick3(b, x, y, z), nb = pick3(b, g.nx, g.ny, g.nz);
        if (plus ? cb >= nb - 1 : cb == 0) continue;               // no quad on that side
        if (own == uint32_t(1 + 2 * b + (plus ? 1 : 0))) continue;  // q is e's own partner
        // owner of q: e's owner, or one step back along b
        const int back = plus ? 0 : 1;
        int ox = x - (b == 0 ? back : 0), oy = y - (b == 1 ? back : 0), oz = z - (b == 2 ? back : 0);
        uint32_t ov = v - (plus ? 0u : (b == 0 ? 1u : b == 1 ? sy : sz));
        const int slot = (1 << axis) | (1 << b);
        const uint32_t qc = slot_code(words[ov], slot);
        if (qc == 0) {
            out[i] = DagTarget{ov, ox, oy, oz, 2, uint8_t(slot)};
            ++cnt;
            continue;
        }
        const int k = int(qc - 1) >> 1;
        if (k == other) continue;  // paired with a cube: no edge
        if (!(qc & 1u)) {          // partner on the + side along k: owner one step forward
            ox += k == 0;
            oy += k == 1;
            oz += k == 2;
            ov += k == 0 ? 1u : k == 1 ? sy : sz;
        }
        out[i] = DagTarget{ov, ox, oy, oz, 1, uint8_t(k == axis ? b : axis)};
        ++cnt;
    }
    return cnt;
}

// Per-node record of every reachable 1-cell that is not a 1-saddle: whether the node is a dead
// end, a branch point (out-degree > 1), or else its one successor.  A 1-cell successor is its
// handle; a 2-saddle successor has bit 31 set and (owner << 2 | even axis).  Records are stored
// one plane per axis (info_index), so a row of cells writes a contiguous run.
constexpr uint32_t INFO_DEAD = 0xFFFFFFFFu;
__host__ __device__ __forceinline__ uint32_t info_index(const Geom& g, uint32_t handle) {
    return (handle & 3u) * uint32_t(g.nverts) + (handle >> 2);
}
constexpr uint32_t INFO_BRANCH = 0xFFFFFFFEu;

}  // namespace msc
