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
// is named by its owner vertex and slot.
#pragma once

#include "geom.cuh"

namespace msc {

struct DagTarget {
    uint32_t v;     // owner vertex index
    uint8_t kind;   // 1 = 1-cell (then `sub` is its axis), 2 = 2-saddle (then `sub` is its slot)
    uint8_t sub;
};

__host__ __device__ __forceinline__ uint32_t edge_handle(uint32_t v, int axis) { return (v << 2) | uint32_t(axis); }

struct Vtx {
    int x, y, z;
};

__host__ __device__ __forceinline__ Vtx vtx_of(const Geom& g, uint32_t v) {
    Vtx r;
    r.x = int(v % uint32_t(g.nx));
    uint32_t q = v / uint32_t(g.nx);
    r.y = int(q % uint32_t(g.ny));
    r.z = int(q / uint32_t(g.ny));
    return r;
}

// Slot of the 1-cell along `axis` in its owner's word: a=1 (slot 1), b=1 (slot 2), c=1 (slot 4).
__host__ __device__ __forceinline__ int edge_slot(int axis) { return 1 << axis; }

// Word index and bit of a 1-cell in the 1-cell row bitmap layout (see Geom::edge_word).
__host__ __device__ __forceinline__ int64_t edge_bitmap_word(const Geom& g, int x, int y, int z, int axis) {
    return g.edge_word(z, axis == 2, y, axis == 1, x >> 5);
}

// Out-edges of the 1-cell (x,y,z,axis); returns how many were written to out[0..3].
__host__ __device__ __forceinline__ int dag_out(const Geom& g, const uint32_t* __restrict__ words, int x, int y, int z,
                                       int axis, DagTarget out[4]) {
    int c[3] = {2 * x, 2 * y, 2 * z};
    c[axis] += 1;
    const int ext[3] = {2 * g.nx - 1, 2 * g.ny - 1, 2 * g.nz - 1};
    const uint32_t own = slot_code(words[g.vid(x, y, z)], edge_slot(axis));
    int n = 0;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        if (b == axis) continue;
#pragma unroll
        for (int sgn = -1; sgn <= 1; sgn += 2) {
            int q[3] = {c[0], c[1], c[2]};
            q[b] += sgn;
            if (q[b] < 0 || q[b] >= ext[b]) continue;
            if (own == uint32_t(1 + 2 * b + (sgn > 0))) continue;  // q is e's own partner
            const int ox = q[0] >> 1, oy = q[1] >> 1, oz = q[2] >> 1;
            const int slot = (q[0] & 1) | ((q[1] & 1) << 1) | ((q[2] & 1) << 2);
            const uint32_t ov = uint32_t(g.vid(ox, oy, oz));
            const uint32_t qc = slot_code(words[ov], slot);
            if (qc == 0) {
                out[n++] = DagTarget{ov, 2, uint8_t(slot)};
                continue;
            }
            const int k = int(qc - 1) >> 1;
            if (k != axis && k != b) continue;  // paired with a cube: no edge
            const int s2 = (qc & 1) ? -1 : 1;
            int e[3] = {q[0], q[1], q[2]};
            e[k] += s2;
            const int eaxis = (k == axis) ? b : axis;  // the odd coordinate that remains
            out[n++] = DagTarget{uint32_t(g.vid(e[0] >> 1, e[1] >> 1, e[2] >> 1)), 1, uint8_t(eaxis)};
        }
    }
    return n;
}

}  // namespace msc
