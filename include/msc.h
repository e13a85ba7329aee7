/*
 * msc.h -- C ABI of libmsc: the Morse-Smale complex 1-skeleton of a float32 scalar field
 * on a 3D structured grid, computed on one GPU (arXiv:2009.03707, Subhash, Pandey,
 * Natarajan, "A GPU Parallel Algorithm for Computing Morse-Smale Complexes").
 *
 * Conventions used by every call
 * ------------------------------
 * Grid:   dims = {nx, ny, nz} vertex counts (each >= 2).  The field is float32, vertex
 *         (x,y,z) at index x + nx*(y + ny*z) (a C-contiguous [nz][ny][nx] array).
 * Cells:  the cubical complex of the grid lives on the refined grid
 *         R = (2nx-1) x (2ny-1) x (2nz-1) (Sec. 2.2): cell (cx,cy,cz) has dimension =
 *         number of odd coordinates, and cell id = cx + (2nx-1)*(cy + (2ny-1)*cz), a
 *         uint32 (grids whose cell count does not fit return MSC_ERR_TOO_LARGE).
 * Order:  vertices are ordered by (value, index); IEEE comparison (-0 == +0, +-Inf are
 *         ordered); a NaN anywhere in the field is MSC_ERR_NAN.
 * NONE:   0xFFFFFFFF marks "no cell" in arcs and labels.
 * Memory: pointers named d_* are device pointers.  Buffers returned through `const T**`
 *         are owned by the plan and stay valid until the next msc_gradient on the same
 *         plan or msc_plan_destroy.  Host buffers are caller-owned.
 * Streams: every call enqueues its work on `stream` (a cudaStream_t).  Calls that return
 *         counts on the host synchronise that stream before returning.  One plan must not
 *         be used from two host threads at once.
 * Errors: every call returns an msc_status; msc_last_error_string(plan) describes the
 *         last failure of that plan.  After MSC_ERR_CUDA the plan should be destroyed.
 */
#ifndef MSC_H_
#define MSC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st* msc_stream_t; /* identical to cudaStream_t */

typedef enum msc_status {
    MSC_OK = 0,
    MSC_ERR_ARG = 1,        /* a null pointer, a dimension < 2, an out-of-range selector */
    MSC_ERR_NAN = 2,        /* the field holds a NaN */
    MSC_ERR_OOM = 3,        /* a device allocation failed */
    MSC_ERR_TOO_LARGE = 4,  /* cell ids would not fit in 32 bits */
    MSC_ERR_OVERFLOW = 6,   /* a saddle-saddle path count exceeds 2^64 - 1 */
    MSC_ERR_ITER_LIMIT = 7, /* an iterative stage exceeded its iteration cap */
    MSC_ERR_TIMEOUT = 8,    /* a bounded device wait gave up */
    MSC_ERR_CUDA = 9,       /* a CUDA runtime error (message in msc_last_error_string) */
    MSC_NOT_READY = 10,     /* msc_poll: the ticket has not finished yet */
    MSC_ERR_STATE = 11,     /* a stage was requested before msc_gradient */
    MSC_ERR_CAPACITY = 12,  /* a caller-provided output buffer is too small (counts are still reported) */
    MSC_ERR_INTERNAL = 13   /* a device-side invariant failed (a lower-star cell left unclassified, a
                               bounds check): a defect of the library, not of the input */
} msc_status;

typedef struct msc_plan_s* msc_plan_t;

/* msc_opts.flags: run every msc_compute with host synchronisation between the stages, never as a
 * replayed CUDA graph (the results are identical; tests use it to compare the two paths). */
#define MSC_FLAG_NO_GRAPH 1
/* msc_opts.flags: replay the pass as one chain of kernels.  By default a replayed pass runs the
 * saddle-extremum stage (a3) as a branch of its own beside the critical path (reachability, the
 * minor, the path counts), its kernels at the device's lowest stream priority and those of the
 * critical path at the highest, which shortens the pass on an otherwise idle device.  When
 * several passes are kept in flight (msc_compute_async on several plans, or a batch), they already
 * fill the device, and one chain per pass at the launching stream's priority gives more
 * throughput.  The results are identical. */
#define MSC_FLAG_SERIAL_PASS 2

/* Plan options (all fields may be zero for defaults). */
typedef struct msc_opts {
    int64_t max_iterations;  /* cap on every iterative stage; 0 = 1<<20 */
    int32_t flags;           /* MSC_FLAG_* bits; other bits must be 0 */
    int32_t path_count_tier; /* first tier of the row-wise path count: 0 = per-thread registers
                                (default), 1 = per-warp shared-memory tables, 2 = per-CTA global
                                tables.  Results are identical; tests use it to cover every tier. */
    int32_t gradient_tile;   /* 0 = autotuned (the lower-star tile variant that runs fastest for the
                                grid shape on this device, timed once per shape on the first
                                synchronised run); 1..9 = force variant (TY,TZ,threads) =
                                (8,8,512), (8,4,256), (4,8,256), (8,16,512), (16,8,512),
                                (16,8,1024), (16,16,512), (8,8,256), (16,8,256); a tile row
                                is 32 vertices.  Results are identical. */
    int32_t path_count_method; /* 1 = the paper's iteration A <- A B, row by row (path_count_tier
                                  picks its first tier); 2 = junction waves: J = B* + B J once per
                                  junction in topological order of the minor, then D* = D + A J;
                                  0 = automatic (default): the plan's first run uses the waves and
                                  later runs use the row-wise products if the minor is at most 64
                                  levels deep (their work grows with the depth).  The counts are
                                  identical. */
} msc_opts;

/* Per-stage diagnostics (Sec. 4.2 "performance analysis" quantities). Times are the
 * device time of the last run of each stage, from CUDA events recorded on the stream (inside
 * the graph when msc_compute replays one); they are read by msc_get_stats. */
typedef struct msc_stats {
    int64_t counts[4];        /* critical cells by index: min, 1-saddle, 2-saddle, max */
    int64_t n_reachable;      /* 1-cells reachable from 1-saddles (1-saddles included) */
    int64_t n_bfs_levels;     /* non-empty BFS levels, level 0 = the 1-saddles */
    int64_t n_junctions;      /* junction nodes of the DAG minor */
    int64_t nnz_A, nnz_B, nnz_Bstar, nnz_D, nnz_Dstar;
    int64_t n_iter;           /* non-zero iterates A B^k (junction waves: the same number, 1 + the
                                 longest chain of junctions) */
    int64_t n_pointer_jumps;  /* pointer-jumping rounds of the extremum forests */
    uint64_t max_path_count;  /* largest entry of D* */
    int64_t peak_device_bytes;
    int64_t n_launches;       /* kernels this plan launched since the last msc_gradient */
    float ms_gradient, ms_critical, ms_extremum, ms_reachability, ms_minor, ms_path_count;
                              /* per stage, CUDA events; in a replayed pass the extremum stage runs
                                 beside the reachability, minor and path-count stages, so the six
                                 may add up to more than the pass */
    float ms_rows_kernel;      /* the product kernels: the junction waves and D* rows, or the
                                  row-wise tier 0 (CUDA events) */
    float ms_trace_kernel;     /* the simple-path tracing kernel alone, CUDA events */
    int64_t n_frontier_entries; /* row-wise method: sum over 1-saddles and iterations of the frontier
                                   sizes; junction waves: J-row entries merged (pool slots) */
    int64_t gradient_tile;      /* the lower-star tile used: TY | TZ << 8 | threads << 16 */
    int64_t path_count_method;  /* the path-count method of the last run: 1 row-wise, 2 waves */
    float ms_gradient_kernel;   /* the lower-star kernel alone (CUDA events) */
    float reserved_f;
} msc_stats;

/* ---- plan ----------------------------------------------------------------------------
 * Sec. 3.5 (implementation): the pipeline keeps the gradient, the critical cells, the
 * reachability and the matrices of Sec. 3.3 in device arrays sized from the grid and from the
 * counts of earlier stages.  A plan holds those arrays for one grid shape on the current CUDA
 * device; they are grown on demand and reused across runs (a time series on one shape
 * allocates once).
 * dims: host array {nx, ny, nz}, each >= 2.  opts: nullable.  *out receives the plan. */
msc_status msc_plan(const int64_t dims[3], const msc_opts* opts, msc_plan_t* out);
msc_status msc_plan_destroy(msc_plan_t plan);
const char* msc_last_error_string(msc_plan_t plan);

/* ---- (a1) discrete gradient ----------------------------------------------------------
 * Sec. 3 / Sec. 3.5 "Gradient pairs and critical points": every cell of the grid is paired
 * with a facet or cofacet, or left critical, by the lower-star rule (Robins, Wood, Sheppard
 * 2011, cited in Sec. 1.1): the cells whose maximal vertex is x are processed together.
 * d_field: caller-owned device float32 field, valid until `stream` reaches this call.
 * Result (plan-owned, read with msc_gradient_words): one uint32 word per vertex; vertex
 * (x,y,z) owns the 8 cells (2x+a, 2y+b, 2z+c), a,b,c in {0,1}; slot s = a + 2b + 4c holds
 * a 3-bit code in bits [3s, 3s+3): 0 = critical, 1..6 = paired with the neighbouring cell
 * at -x,+x,-y,+y,-z,+z on the refined grid, 7 = no such cell (beyond the far boundary).
 * Returns MSC_ERR_NAN (checked when the next call synchronises) if the field has a NaN. */
msc_status msc_gradient(msc_plan_t plan, const float* d_field, msc_stream_t stream);
msc_status msc_gradient_words(msc_plan_t plan, const uint32_t** d_words);

/* ---- (a2) critical cells -------------------------------------------------------------
 * Sec. 3.5 "Gradient pairs and critical points": critical cells are counted and
 * stream-compacted.  counts: host int64[4], filled after a stream synchronisation.
 * d_cells[k]: plan-owned device list of the critical k-cells' ids in increasing cell-id
 * order (counts[k] entries).  d_cells may be null when only the counts are wanted. */
msc_status msc_critical(msc_plan_t plan, msc_stream_t stream, int64_t counts[4], const uint32_t* d_cells[4]);

/* ---- (a3) saddle-extremum arcs and manifold labels -----------------------------------
 * Sec. 3.4 and Sec. 3.5 "Saddle-Extrema arcs": gradient paths from every cell are followed
 * to their extremum by pointer jumping.
 * d_vertex_min_label: [nz][ny][nx] uint32, the cell id of the minimum that the descending
 *   path from each vertex reaches.
 * d_cube_max_label:   [nz][ny][nx] uint32, entry (x,y,z) for the cube (2x+1,2y+1,2z+1): the
 *   cell id of the maximum its ascending path reaches, NONE if the path leaves the domain
 *   through a boundary quad, NONE where x = nx-1, y = ny-1 or z = nz-1.
 * d_min_arcs: 2 per 1-saddle (in d_cells[1] order): the minima of its lower-coordinate and
 *   upper-coordinate vertex.
 * d_max_arcs: 2 per 2-saddle (in d_cells[2] order): the maxima of its cofacet cube on the
 *   - side and + side of the quad's even axis (NONE if the cube does not exist or the
 *   path leaves the domain).
 * Any output pointer may be null. */
msc_status msc_extremum_arcs(msc_plan_t plan, msc_stream_t stream, const uint32_t** d_min_arcs,
                             const uint32_t** d_max_arcs, const uint32_t** d_vertex_min_label,
                             const uint32_t** d_cube_max_label);

/* ---- (a4) saddle-saddle reachability ---------------------------------------------------
 * Sec. 3.2 and Sec. 3.5 "Saddle-Saddle reachability": a frontier BFS from all 1-saddles
 * over the DAG of 1-2 gradient pairs (Fig. "msc-max-min-dag" (d)), moving against the
 * gradient: a 1-cell e leads to the 1-cell paired with each cofacet quad q != pair(e)
 * (when q is paired with a facet) or to q itself (when q is a 2-saddle).
 * d_visited: plan-owned bitmap in the 1-cell row layout: word index
 *   (((z*2 + c)*ny + y)*2 + b)*W + w, W = ceil(nx/32), bit (x & 31) with w = x >> 5, for
 *   the 1-cell (2x+a, 2y+b, 2z+c), a = 1-b-c (rows with b = c = 1 are unused).
 * n_words: number of words in d_visited.  n_levels: host, non-empty BFS levels. */
msc_status msc_reachability(msc_plan_t plan, msc_stream_t stream, const uint32_t** d_visited, int64_t* n_words,
                            int64_t* n_levels);

/* ---- (a5) junction nodes and the DAG minor ---------------------------------------------
 * Sec. 3.3 "DAG minor construction" and Sec. 3.5 "Gradient path counting": a junction is a
 * reachable 1-cell, not a 1-saddle, with DAG out-degree > 1; simple paths from every
 * 1-saddle and junction are traced to the first junction or 2-saddle (dead ends dropped).
 * msc_junctions: d_cells = junction ids in increasing cell-id order, n = count (host).
 * msc_minor: which = 0 A (1-saddle x junction), 1 B (junction x junction), 2 B* (junction x
 *   2-saddle), 3 D (1-saddle x 2-saddle); CSR with rows/cols by rank in the d_cells[1],
 *   junction and d_cells[2] lists, columns increasing within a row, uint32 multiplicities.
 *   rowptr has rows+1 entries; nnz and rows are returned on the host. */
msc_status msc_junctions(msc_plan_t plan, msc_stream_t stream, const uint32_t** d_cells, int64_t* n);
msc_status msc_minor(msc_plan_t plan, msc_stream_t stream, int which, int64_t* rows, int64_t* nnz,
                     const int64_t** d_rowptr, const uint32_t** d_col, const uint32_t** d_mult);

/* ---- (a6) saddle-saddle arcs with multiplicity -----------------------------------------
 * Sec. 3.3 "Path counting via matrix operations": D* = D + sum_{k>=0} A B^k B*, iterating
 * A <- A B while the product is non-zero; every entry is the exact number of gradient paths
 * between a 1-saddle and a 2-saddle, in uint64 (MSC_ERR_OVERFLOW if one exceeds 2^64-1).
 * CSR over 1-saddle ranks (rows = counts[1], rowptr has rows+1 int64 entries), columns are
 * 2-saddle ranks increasing within a row.  nnz: host. */
msc_status msc_saddle_arcs(msc_plan_t plan, msc_stream_t stream, int64_t* nnz, const int64_t** d_rowptr,
                           const uint32_t** d_col, const uint64_t** d_count);

/* ---- the same arcs by 2-saddle -------------------------------------------------------
 * Sec. 3.5 "Data structure": the complex keeps every arc in both directions, so that the arcs
 * reaching a critical point can be queried as well as those leaving it.  This is D* in
 * compressed sparse column form: for each 2-saddle (by rank in d_cells[2]; colptr has
 * counts[2]+1 int64 entries) the 1-saddles (by rank in d_cells[1]) with a gradient path to it,
 * increasing within a column, and the same uint64 path counts as msc_saddle_arcs.  Built on the
 * first call after a pass (host-synchronised; a stable radix sort of the CSR's entries by
 * column) and kept until the next pass.  Plan-owned, valid until the next pass or
 * msc_plan_destroy.  nnz: host.  MSC_ERR_TOO_LARGE if D* has 2^32 or more entries. */
msc_status msc_saddle_arcs_csc(msc_plan_t plan, msc_stream_t stream, int64_t* nnz, const int64_t** d_colptr,
                               const uint32_t** d_row, const uint64_t** d_count);

/* ---- the 1-skeleton as one adjacency, exported to the host -----------------------------
 * Sec. 3.5 "Data structure": the complex as its critical points, each with the arcs incident on
 * it in both directions (every arc stored at both ends).  Nodes are the critical cells numbered
 * minima, then 1-saddles, 2-saddles, maxima, each group in its d_cells order (node id = rank +
 * the counts of the groups before it).  Node u's neighbours are h_adj[h_nodeptr[u] ..
 * h_nodeptr[u+1]), increasing, with h_mult the number of arcs between the two: the D* path
 * count for a pair of saddles; 1 or 2 for a saddle and an extremum (2 when both of the saddle's
 * arcs reach it).  Arcs that leave the domain (max arcs with NONE) are left out.
 * Size query: *n_adj on entry is the room in h_adj / h_mult; on return *n_nodes and *n_adj are
 * set, and with h_nodeptr null nothing is copied.  Otherwise h_nodeptr (n_nodes + 1 int64),
 * h_adj (uint32) and h_mult (uint64) are caller-owned host buffers, filled after a stream
 * synchronisation; MSC_ERR_CAPACITY (nothing copied) if the room is smaller than *n_adj.
 * Built on the device on the first call after a pass (host-synchronised) and kept until the next
 * pass.  MSC_ERR_TOO_LARGE if there are 2^32 or more critical cells. */
msc_status msc_complex_graph(msc_plan_t plan, msc_stream_t stream, int64_t* n_nodes, int64_t* n_adj,
                             int64_t* h_nodeptr, uint32_t* h_adj, uint64_t* h_mult);

/* ---- the cells along the saddle-extremum arcs (on request) -----------------------------
 * Sec. 3.4 and Sec. 3.5 "Data structure": besides its end points, each saddle-extremum arc has a
 * geometry, the V-path (Sec. 2.2) it follows from its saddle.  Arcs are numbered as the arc lists:
 * arc 2i and 2i+1 (i < counts[1]) start at the 1-saddle of rank i, from its lower-coordinate and
 * upper-coordinate vertex (as d_min_arcs); arc 2*counts[1] + 2j + s starts at the 2-saddle of rank j,
 * into its cofacet cube on the - (s = 0) or + (s = 1) side of its even axis (as d_max_arcs).
 *   Descending arc: the 1-saddle, its vertex, then alternately the edge that vertex is paired with
 *     and that edge's other vertex, ending at the minimum.
 *   Ascending arc: the 2-saddle, the cube, then alternately the quad the cube is paired with and the
 *     cube across that quad, ending at the maximum -- or at the quad through which the path leaves
 *     the domain (the arc's maximum is NONE), or at the 2-saddle alone when that side has no cube.
 * Arc a's cells are d_cells[d_offsets[a] .. d_offsets[a+1]) (cell ids).  *n_arcs = 2*(counts[1] +
 * counts[2]); d_offsets has n_arcs+1 int64 entries; *n_cells = d_offsets[n_arcs].  Built on the
 * first call after a pass (host-synchronised: a thread per arc walks the gradient words to count,
 * a scan, a second walk to write) and kept until the next pass.  Plan-owned.  Any output pointer may
 * be null. */
msc_status msc_arc_geometry(msc_plan_t plan, msc_stream_t stream, int64_t* n_arcs, int64_t* n_cells,
                            const int64_t** d_offsets, const uint32_t** d_cells);

/* ---- the cells along the saddle-saddle arcs of multiplicity 1 (on request) -----------------
 * Sec. 3.3 and Sec. 3.5 "Data structure": a saddle-saddle arc (s, t) of D* with count 1 is a single
 * V-path (Sec. 2.2) from the 2-saddle t down to the 1-saddle s, so it has one geometry; an entry with
 * a larger count stands for several paths and gets none.  Entry k of the D* CSR (msc_saddle_arcs
 * order: by 1-saddle rank, columns increasing) has the cells d_cells[d_offsets[k] .. d_offsets[k+1]),
 * read from s against the gradient: s, then for each step the quad and the 1-cell paired with it,
 * then t.  Empty for a count other than 1.  *n_entries = nnz of D*; d_offsets has nnz+1 int64
 * entries; *n_cells = d_offsets[nnz].  Built on the first call after a pass (host-synchronised): the
 * path is chosen at each junction by the junction-to-2-saddle path counts J of the junction waves
 * (which run once more for this, giving the same D*, when the pass counted paths row by row; the
 * pass's statistics are kept), then walked through the gradient words.  MSC_ERR_INTERNAL if the
 * minor and the gradient disagree (cannot happen).  Plan-owned until the next pass; any output pointer
 * may be null. */
msc_status msc_saddle_arc_geometry(msc_plan_t plan, msc_stream_t stream, int64_t* n_entries, int64_t* n_cells,
                                   const int64_t** d_offsets, const uint32_t** d_cells);

/* ---- simplification of the 1-skeleton (on request) --------------------------------------
 * Sec. 4 "Parallel Simplification": critical-point pairs of consecutive index joined by exactly one
 * arc are cancelled in order of persistence; a cancellation reroutes the upper point's descending
 * arcs to the end points of the lower point's ascending arcs (multiplicities multiply) and deletes
 * both points.  Pairs joined by several arcs are never cancelled (strangulations).  This runs the
 * paper's data-parallel form on the GPU, in rounds: a round cancels every valid arc whose key
 * (persistence, cell id of the upper point, cell id of the lower point) is the least among the valid
 * arcs with an end within two links of one of its ends; those arcs are independent (their
 * cancellations touch disjoint points), and rounds repeat until no arc with persistence <= threshold
 * can be cancelled.  The value of a critical cell is the field's value at its highest vertex;
 * persistence = |value(upper) - value(lower)|.
 * d_field: the field of the plan's last pass (caller-owned; its values are read).  threshold >= 0
 *   (absolute, in the field's units).
 * The complex starts as msc_complex_graph's (built if needed; same node numbering) and is left
 * unchanged there; the result is plan-owned until the next pass or simplification:
 *   d_alive[n_nodes] (1 = survives), d_nodeptr[n_nodes+1] / d_adj[n_adj] / d_mult[n_adj] (CSR, every
 *   arc in both rows, neighbours increasing), counts[4] (points left by index), d_log (3 uint32 per
 *   cancellation in order: upper node, lower node, round).  Host-synchronised once per round.
 *   MSC_ERR_OVERFLOW if a multiplicity exceeds 2^64 - 1; MSC_ERR_ITER_LIMIT after max_iterations
 *   rounds. */
typedef struct msc_simplified {
    int64_t n_nodes, n_rounds, n_cancelled, n_adj;
    int64_t counts[4];
    const uint8_t* d_alive;
    const int64_t* d_nodeptr;
    const uint32_t* d_adj;
    const uint64_t* d_mult;
    const uint32_t* d_log;
} msc_simplified;
msc_status msc_simplify(msc_plan_t plan, msc_stream_t stream, const float* d_field, double threshold,
                        msc_simplified* out);

/* ---- outputs into host memory --------------------------------------------------------
 * Sec. 3.5 "Data structure": the complex is assembled on the host from the arrays the GPU
 * stages produce.  This copies one of those arrays into caller-owned host memory, computing the stage if
 * it has not run yet (as the accessor above would).  `what` selects the array and its element type:
 *   MSC_OUT_CELLS0..3      critical k-cell ids (uint32, counts[k])
 *   MSC_OUT_MIN_ARCS       2 minima per 1-saddle (uint32)       MSC_OUT_MAX_ARCS  2 maxima per 2-saddle (uint32)
 *   MSC_OUT_VERTEX_MIN     minimum of every vertex (uint32)     MSC_OUT_CUBE_MAX  maximum of every cube (uint32)
 *   MSC_OUT_DSTAR_ROWPTR   D* row pointers (int64, counts[1]+1) MSC_OUT_DSTAR_COL columns (uint32, nnz)
 *   MSC_OUT_DSTAR_COUNT    path counts (uint64, nnz)
 *   MSC_OUT_ARC_OFFSETS    arc geometry offsets (int64, n_arcs+1)  MSC_OUT_ARC_CELLS  cells along the arcs (uint32)
 *   MSC_OUT_SS_ARC_OFFSETS saddle-saddle arc offsets (int64, nnz+1) MSC_OUT_SS_ARC_CELLS their cells (uint32)
 * Size query: *bytes on entry is the room in h_out; on return it is the output's size in bytes.
 * With h_out null nothing is copied.  Otherwise the copy is made and the stream synchronised;
 * MSC_ERR_CAPACITY (nothing copied) if the room is smaller.  MSC_ERR_ARG for an unknown `what`. */
enum {
    MSC_OUT_CELLS0 = 0,
    MSC_OUT_CELLS1 = 1,
    MSC_OUT_CELLS2 = 2,
    MSC_OUT_CELLS3 = 3,
    MSC_OUT_MIN_ARCS = 4,
    MSC_OUT_MAX_ARCS = 5,
    MSC_OUT_VERTEX_MIN = 6,
    MSC_OUT_CUBE_MAX = 7,
    MSC_OUT_DSTAR_ROWPTR = 8,
    MSC_OUT_DSTAR_COL = 9,
    MSC_OUT_DSTAR_COUNT = 10,
    MSC_OUT_ARC_OFFSETS = 11,
    MSC_OUT_ARC_CELLS = 12,
    MSC_OUT_SS_ARC_OFFSETS = 13,
    MSC_OUT_SS_ARC_CELLS = 14
};
msc_status msc_copy_to_host(msc_plan_t plan, msc_stream_t stream, int what, void* h_out, int64_t* bytes);

/* ---- the whole pass without waiting ----------------------------------------------------
 * msc_compute_async enqueues a pass on `stream` and returns without waiting for it, so that one
 * thread can keep several plans' passes (on their own streams) in flight -- e.g. upload the next
 * field and read back the previous results while a pass runs.  It does so when the plan replays a
 * captured graph (from its second msc_compute on the same grid shape, graphs enabled); otherwise
 * it runs the pass synchronised, exactly as msc_compute.  msc_compute_wait waits for the pass and
 * returns its status; a pass that outgrew the capacities of the captured graph is then run again
 * synchronised (so the wait can take as long as a synchronised pass).  A plan holds one pass in
 * flight: every other entry point on the plan (msc_get_stats included) waits for it first, and
 * reports its error if it failed.  The field must stay valid and unchanged until the wait.  The
 * outputs are those of the pass only once it has been waited for. */
msc_status msc_compute_async(msc_plan_t plan, const float* d_field, msc_stream_t stream);
msc_status msc_compute_wait(msc_plan_t plan);

/* Runs every stage (a1..a6) on `stream` for one field; equivalent to the calls above in
 * order.  Results are read afterwards with the getters (they do no further work, except that
 * msc_minor builds the CSR of A, B, B*, D on its first call for a field).
 * The first call on a plan runs the stages with host synchronisation between them and so learns
 * the sizes of the field's products.  Later calls replay the whole pipeline as one CUDA graph,
 * captured on a plan-private stream with buffers sized from those sizes plus headroom; the
 * iterative stages are conditional WHILE nodes, so a replay needs no host round trip until it
 * ends.  The call returns after one synchronisation of `stream` at the end of the pass.  If a
 * field needs more room than the graph was captured with, the kernels say so, the pass is run
 * again synchronised (same results), and the next call captures a larger graph.  d_field must
 * stay valid while the call runs; a new pointer is captured anew.  MSC_FLAG_NO_GRAPH disables
 * the replay. */
msc_status msc_compute(msc_plan_t plan, const float* d_field, msc_stream_t stream);

msc_status msc_get_stats(msc_plan_t plan, msc_stats* out);

/* ---- batching and serving ------------------------------------------------------------------
 * Many volumes of uneven size, processed concurrently (the time-varying, interactive use that
 * motivates the paper, Sec. 1, where every time step must be analysed quickly).  A batch owns a pool of
 * host worker threads, each driving its own CUDA stream on the batch's device; submitted
 * volumes are queued and started as workers and device memory free up (continuous batching):
 * a volume is admitted while the summed working-set estimates of the volumes in flight stay
 * within hbm_budget_bytes (one volume is always admitted when nothing else runs).  The
 * estimate is the plan's measured peak from earlier runs, else 128 bytes per voxel.
 *
 * msc_batch_create: n_workers >= 1 host threads (0 = 4); hbm_budget_bytes <= 0 = no limit.
 * msc_batch_submit: vols[i].d_field is a caller-owned device field (valid until the volume
 *   completes); vols[i].plan is an existing plan of the same dims to reuse (a time series keeps
 *   its state on the device) or NULL, in which case a plan is created and returned in
 *   vols[i].plan; the caller owns it and destroys it with msc_plan_destroy after the ticket is
 *   done.  Work on one plan is never run concurrently: later submissions on a plan wait for the
 *   earlier ones.  Every volume's work is ordered after the work already queued on `stream` at
 *   submission.  Returns immediately; *ticket names the submission.
 * msc_poll: never blocks; *done = 1 once every volume of the ticket has finished, *status =
 *   the first non-OK status among them (MSC_OK otherwise).  Results are read from each
 *   volume's plan with the getters above (they do no further work).
 * msc_batch_wait: blocks until the ticket is done, then reports like msc_poll.
 * msc_batch_destroy: waits for all queued work, then stops the workers. */
typedef struct msc_batch_s* msc_batch_t;
typedef struct msc_volume {
    int64_t dims[3];
    const float* d_field;
    msc_plan_t plan; /* in: plan to reuse, or NULL; out: the plan holding this volume's results */
} msc_volume;

msc_status msc_batch_create(int n_workers, int64_t hbm_budget_bytes, msc_batch_t* out);
msc_status msc_batch_destroy(msc_batch_t batch);
msc_status msc_batch_submit(msc_batch_t batch, msc_volume* vols, int n, msc_stream_t stream, uint64_t* ticket);
msc_status msc_poll(msc_batch_t batch, uint64_t ticket, int* done, int* status);
msc_status msc_batch_wait(msc_batch_t batch, uint64_t ticket, int* status);

/* ---- (a1)+(a2) without any device allocation ---------------------------------------------
 * The paper has no counterpart: this is a convenience for callers that cannot allocate device
 * memory -- a host program that has already reserved the whole GPU for its own memory pool, or
 * code running in a callback or a deadline-bound loop where a cudaMalloc (which may synchronise
 * the device, and may fail) is not allowed.  It computes the same packed gradient and critical
 * lists as msc_gradient + msc_critical, but needs no plan: all of its scratch (critical-cell
 * bitmaps, their word prefixes, scan block sums and a status word) lives in one static device
 * array of MSC_STATIC_SCRATCH_BYTES.  It calls no cudaMalloc, cudaFree or allocating library
 * routine.
 *
 * dims: host {nx, ny, nz}.  d_field: caller-owned float32 field (as msc_gradient).
 * d_words: caller-owned output, nx*ny*nz uint32 in the msc_gradient word layout.
 * d_cells[k], capacity[k]: caller-owned output lists of the critical k-cells (increasing cell
 *   id) and their capacities in entries.  counts: host int64[4], filled before returning.
 * Size limit: the scratch holds 64 * nz * ny * ceil(nx/32) bytes of bitmaps and prefixes, the
 *   scan's block sums and 512 bytes of status; it must fit in MSC_STATIC_SCRATCH_BYTES.  Cubes up
 *   to 193^3 fit; 194^3 and larger return MSC_ERR_TOO_LARGE before any GPU work.  If a count
 *   exceeds its capacity the lists are not written, counts are still filled, and
 *   MSC_ERR_CAPACITY is returned.  MSC_ERR_INTERNAL if the gradient kernel reports a broken
 *   invariant.
 * Loading: CUDA loads the library's device code, and so creates the array, lazily -- when a
 *   device first needs it.  msc_static_prepare(device) does that for one device (and looks up
 *   the array's address) without running anything; call it while device memory is still free,
 *   before the caller reserves the rest of the GPU.  The first msc_gradient_critical_static on a
 *   device not prepared does the same itself.
 * Streams: the call synchronises `stream` once (to read the counts) and so cannot be recorded
 *   into a CUDA graph; the lists are complete when `stream` reaches the end of the call.  All
 *   calls share the one array, which keeps the last call's contents: calls that overlap on the
 *   GPU (two streams, or two host threads) race on it and must be serialised by the caller.
 *   The array's address is remembered per device for the life of the process; do not use the
 *   entry point on a device after cudaDeviceReset. */
#define MSC_STATIC_SCRATCH_BYTES (16u << 20)
msc_status msc_static_prepare(int device);
msc_status msc_gradient_critical_static(const int64_t dims[3], const float* d_field, uint32_t* d_words,
                                        uint32_t* const d_cells[4], const int64_t capacity[4], int64_t counts[4],
                                        msc_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* MSC_H_ */
