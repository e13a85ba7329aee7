// (a1) Lower-star discrete gradient + (a2, first half) critical-cell bitmaps.
//
// Sec. 3 / Sec. 3.5 "Gradient pairs and critical points" of arXiv:2009.03707: every cell is
// paired with a facet or cofacet or left critical.  The rule is the lower-star pairing of
// Robins, Wood and Sheppard (2011, cited in Sec. 1.1): the cells whose maximal vertex is x
// (the lower star L(x)) are paired among themselves, so every vertex is independent work.
//
// GB300 design (not the paper's texture-object kernel):
//  * One CTA owns a 32 x TY x TZ tile of vertices (a tuned choice) and computes exactly their lower
//    stars.  The field tile plus a one-vertex halo is staged in shared memory as order-preserving
//    uint32 keys.
//  * A cell's 3-bit code lives in the word of its lowest corner vertex (its owner) but is decided
//    by its highest vertex, so a tile's stars write the words of the tile and of a one-vertex
//    layer on its - sides.  All of them are OR-ed into shared words; at the end the layer's words
//    go to global memory with atomicOr, as do the tile's words on its + faces (which receive the
//    next tiles' layers), into words a small kernel zeroes beforehand (about a quarter of all
//    words, mostly whole rows and planes).  Every other word is a plain coalesced store.
//  * A lower star is handled as 27-bit masks over the offsets d in {-1,0,1}^3 (lower_star.cuh),
//    with the per-position masks tabulated in shared memory and the vertex keys read straight
//    from the staged tile.  Large stars rank their vertices once with a sorting network and keep
//    their cells' integer keys in a per-thread column of shared memory.  Stars differ widely in
//    size (1..27 cells) and a warp runs as long as its largest, so the CTA first sizes every star
//    and counting-sorts its vertices by size; warps then claim 32 consecutive stars at a time,
//    largest first.
//  * A second, bandwidth-bound kernel turns the finished words into per-slot critical bitmaps:
//    one warp ballot per slot gives 32 vertices' bits -- the input of the ordered compaction.
#include <map>
#include <mutex>
#include <tuple>

#include "lower_star.cuh"
#include "msc_internal.cuh"

namespace msc {

namespace {

constexpr int TX = 32;  // a tile row is one warp wide
constexpr uint32_t OUTSIDE_KEY = 0xFFFFFFFFu;

using star::pdx;
using star::pdy;
using star::pdz;

// Monotone map float -> uint32 (IEEE order; -0 and +0 map to the same key).
__device__ __forceinline__ uint32_t order_key(float f) {
    uint32_t u = __float_as_uint(f);
    if ((u & 0x7fffffffu) == 0) u = 0;
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// The owned tile is TX x TY x TZ vertices, run by THREADS threads (a tuning choice: every
// variant computes the same words).
template <int TY, int TZ, int THREADS>
struct Shared {
    static constexpr int FX = TX + 2, FY = TY + 2, FZ = TZ + 2;  // field keys staged (x0-1 .. x0+TX)
    static constexpr int FXP = TX + 4;                            // their row pitch: 16-byte rows
    static constexpr int NOWN = TX * TY * TZ;
    static constexpr int WX = TX + 1, WY = TY + 1, WZ = TZ + 1;  // words kept (x0-1 .. x0+TX-1)
    uint32_t fkey[FZ][FY][FXP];  // order keys of the field tile (OUTSIDE_KEY off-grid); columns >= FX unused
    uint32_t words[WZ][WY][WX];  // packed codes of the owned tile and its - layer
    uint32_t inl[NOWN];          // lower-star mask of every owned vertex (0: off-grid)
    uint16_t order[NOWN];        // non-minimal vertices, largest stars first
    uint32_t ckey[27][THREADS];  // per-thread cell keys of the star in hand (ranked path)
    int bin[28];                 // counting-sort bins by star size
    int next;                    // next unclaimed entry of `order`
    star::Tables tab;            // per-position masks; key offsets within fkey
    // per position p: the bit offset of the cell's slot in its owner's word (bits 0-4) and the
    // owner's distance back in `words` (bits 8+)
    uint32_t emit_info[27];
};

template <int TY, int TZ, int THREADS>
__global__ void __launch_bounds__(THREADS, 65536 / (64 * THREADS)) gradient_kernel(Geom g, const float* __restrict__ field,
                                                           uint32_t* __restrict__ words_out,
                                                           uint32_t* __restrict__ status) {
    using S = Shared<TY, TZ, THREADS>;
    constexpr int FX = S::FX, FXP = S::FXP, FY = S::FY, FZ = S::FZ, NOWN = S::NOWN;
    constexpr int WX = S::WX, WY = S::WY, WZ = S::WZ;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S& sh = *reinterpret_cast<S*>(smem_raw);
    const int t = threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;

    // stage the field tile with its one-vertex halo as order keys: every load of the thread is
    // issued first (their latencies overlap, and the shared initialisation runs under them), then
    // the values are converted and stored
    constexpr int NST = FX * FY * FZ, ST_IT = (NST + THREADS - 1) / THREADS;
    float v[ST_IT];
#pragma unroll
    for (int k = 0; k < ST_IT; ++k) {
        const int i = t + k * THREADS;
        const int fx = i % FX, fy = (i / FX) % FY, fz = i / (FX * FY);
        const int gx = x0 - 1 + fx, gy = y0 - 1 + fy, gz = z0 - 1 + fz;
        const bool in = i < NST && gx >= 0 && gy >= 0 && gz >= 0 && gx < g.nx && gy < g.ny && gz < g.nz;
        v[k] = in ? __ldg(field + g.vid(gx, gy, gz)) : __uint_as_float(0x7FFFFFFFu);
    }
    for (int i = t; i < WX * WY * WZ; i += THREADS) (&sh.words[0][0][0])[i] = 0;
    if (t < 28) sh.bin[t] = 0;
    if (t == 0) sh.next = 0;
    if (t < 27) {
        star::fill_tables(sh.tab, t, FXP, FXP * FY);
        const uint32_t xn = (star::XN >> t) & 1, yn = (star::YN >> t) & 1, zn = (star::ZN >> t) & 1;
        const uint32_t slot = (pdx(t) != 0) | ((pdy(t) != 0) << 1) | ((pdz(t) != 0) << 2);
        sh.emit_info[t] = (3 * slot) | ((xn + yn * WX + zn * WX * WY) << 8);
    }
    bool saw_nan = false;
    const int lane = t & 31, warp = t >> 5;
#pragma unroll
    for (int k = 0; k < ST_IT; ++k) {
        const int i = t + k * THREADS;
        if (i >= NST) break;
        const int fx = i % FX, fy = (i / FX) % FY, fz = i / (FX * FY);
        const int gx = x0 - 1 + fx, gy = y0 - 1 + fy, gz = z0 - 1 + fz;
        const bool in = gx >= 0 && gy >= 0 && gz >= 0 && gx < g.nx && gy < g.ny && gz < g.nz;
        saw_nan |= in && isnan(v[k]);
        sh.fkey[fz][fy][fx] = in ? order_key(v[k]) : OUTSIDE_KEY;
    }
    if (saw_nan) atomicOr(status, ST_NAN);
    __syncthreads();

    // size every star (cheap mask arithmetic) and counting-sort the non-minimal ones by size, one shared
    // atomic per vertex (a ballot-based warp histogram measured slower).  A thread takes four
    // consecutive vertices of a row: the six keys of each of their nine neighbour rows come in one
    // 16-byte and one 8-byte shared load.
    for (int i4 = t; i4 < NOWN / 4; i4 += THREADS) {
        const int lx0 = (i4 % (TX / 4)) * 4, ly = (i4 / (TX / 4)) % TY, lz = i4 / ((TX / 4) * TY);
        uint32_t lower[4], kc[4];
        {
            const uint32_t* c = &sh.fkey[lz + 1][ly + 1][lx0];
            const uint4 a = *reinterpret_cast<const uint4*>(c);
            const uint2 b = *reinterpret_cast<const uint2*>(c + 4);
            kc[0] = a.y;
            kc[1] = a.z;
            kc[2] = a.w;
            kc[3] = b.x;
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) lower[v] = 1u << star::CENTER;
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
                const uint32_t* row = &sh.fkey[lz + 1 + dz][ly + 1 + dy][lx0];
                const uint4 a = *reinterpret_cast<const uint4*>(row);
                const uint2 b = *reinterpret_cast<const uint2*>(row + 4);
                const uint32_t r[6] = {a.x, a.y, a.z, a.w, b.x, b.y};
#pragma unroll
                for (int v = 0; v < 4; ++v)
#pragma unroll
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int p = 9 * (dz + 1) + 3 * (dy + 1) + (dx + 1);
                        if (p == star::CENTER) continue;
                        const uint32_t kp = r[v + 1 + dx];  // lower: smaller key, or equal and earlier
                        const bool lo = p < star::CENTER ? kp <= kc[v] : kp < kc[v];
                        lower[v] |= uint32_t(lo) << p;
                    }
            }
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int lx = lx0 + v, i = lx + TX * (ly + TY * lz);
            uint32_t inL = 0;
            if (x0 + lx < g.nx && y0 + ly < g.ny && z0 + lz < g.nz) {
                inL = star::lower_star_mask(lower[v]);
                const int m = __popc(inL) - 1;
                if (m > 0) atomicAdd(&sh.bin[m], 1);
            }
            sh.inl[i] = inL;
        }
    }
    __syncthreads();
    if (t == 0) {
        int acc = 0;
        for (int m = 26; m >= 1; --m) {
            const int c = sh.bin[m];
            sh.bin[m] = acc;
            acc += c;
        }
        sh.bin[0] = acc;  // number of non-minimal vertices
    }
    __syncthreads();
    for (int i = t; i < NOWN; i += THREADS) {
        const int m = __popc(sh.inl[i]) - 1;
        if (m > 0) sh.order[atomicAdd(&sh.bin[m], 1)] = uint16_t(i);
    }
    __syncthreads();
    const int n_items = sh.bin[0];

    // warps claim 32 consecutive stars at a time, largest first, so the CTA's stars are
    // spread over its warps by longest-processing-time order
    bool ok = true;
    for (;;) {
        int base = 0;
        if (lane == 0) base = atomicAdd(&sh.next, 32);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if (base >= n_items) break;
        if (base + lane < n_items) {
        const int i = sh.order[base + lane];
        const int lx = i % TX, ly = (i / TX) % TY, lz = i / (TX * TY);
        const uint32_t inL = sh.inl[i];
        const star::Star st{&sh.fkey[lz + 1][ly + 1][lx + 1], &sh.tab};
        uint32_t* const wx = &sh.words[lz + 1][ly + 1][lx + 1];
        // a cell is owned by its lowest corner vertex: OR its code into that vertex's word
        auto emit = [&](int p, uint32_t code) {
            const uint32_t e = sh.emit_info[p];
            atomicOr(wx - int(e >> 8), code << (e & 31u));
        };
        // the scratch word of position p of this thread, in its own bank column
        auto ckey = [&](int p) -> uint32_t& { return sh.ckey[p][t]; };
        ok &= star::pair_lower_star<FXP, FXP * FY>(inL, st, ckey, emit);
        }
    }
    if (!ok) atomicOr(status, ST_INTERNAL);
    __syncthreads();

    // epilogue, a warp per row of kept words: the tile's words get their far-boundary codes and a
    // plain store -- or atomicOr on the tile's + faces, whose words also receive codes from the
    // neighbouring tiles; the - layer's words (the previous tiles' + faces) get atomicOr where
    // they received a code (code 7 in the slots with a = 1, b = 1 or c = 1 of a vertex on the last
    // x, y or z layer)
    constexpr uint32_t OUT_X = 0xE38E38u, OUT_Y = 0xFC0FC0u, OUT_Z = 0xFFF000u;
    const int gx = x0 + lane;
    for (int r = warp; r < WY * WZ; r += THREADS / 32) {
        const int ey = r % WY, ez = r / WY;
        const int gy = y0 - 1 + ey, gz = z0 - 1 + ez;
        if (gy < 0 || gz < 0 || gy >= g.ny || gz >= g.nz) continue;  // warp-uniform
        if (lane == 0 && x0 > 0) {
            const uint32_t w = sh.words[ez][ey][0];
            if (w) atomicOr(words_out + g.vid(x0 - 1, gy, gz), w);
        }
        if (gx >= g.nx) continue;
        uint32_t* dst = words_out + g.vid(gx, gy, gz);
        const uint32_t w = sh.words[ez][ey][lane + 1];
        if (ey == 0 || ez == 0) {  // the - layer
            if (w) atomicOr(dst, w);
            continue;
        }
        const uint32_t wf = w | (gx == g.nx - 1 ? OUT_X : 0u) | (gy == g.ny - 1 ? OUT_Y : 0u) |
                            (gz == g.nz - 1 ? OUT_Z : 0u);
        if (lane == TX - 1 || ey == TY || ez == TZ) atomicOr(dst, wf);
        else *dst = wf;
    }
}

// Per-slot critical bitmaps from finished words: one warp per CB_WORDS row words of 32 vertices,
// their loads issued together.
constexpr int CB_WORDS = 4;
__global__ void __launch_bounds__(256) critical_bitmaps(Geom g, const uint32_t* __restrict__ words,
                                                        uint32_t* __restrict__ crit_bits) {
    const uint32_t nrw = uint32_t(g.nz) * uint32_t(g.ny) * uint32_t(g.W);  // < 2^28 row words
    const uint32_t w0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * CB_WORDS;
    const int lane = threadIdx.x & 31;
    if (w0 >= nrw) return;  // warp-uniform
    uint32_t word[CB_WORDS];
    int w[CB_WORDS], y[CB_WORDS], z[CB_WORDS];
#pragma unroll
    for (int u = 0; u < CB_WORDS; ++u) {
        const uint32_t wid = min(w0 + u, nrw - 1);
        const uint32_t q = g.div_W.div(wid);
        w[u] = int(wid - q * uint32_t(g.W));
        z[u] = int(g.div_ny.div(q));
        y[u] = int(q - uint32_t(z[u]) * uint32_t(g.ny));
        const int x = w[u] * 32 + lane;
        word[u] = x < g.nx ? words[uint32_t(x) + uint32_t(g.nx) * (uint32_t(y[u]) + uint32_t(g.ny) * uint32_t(z[u]))]
                           : 0x00FFFFFFu;  // all codes 7: no cell
    }
#pragma unroll
    for (int u = 0; u < CB_WORDS; ++u) {
        if (w0 + u >= nrw) break;  // warp-uniform
        uint32_t mine = 0;
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const uint32_t bits = __ballot_sync(0xFFFFFFFFu, slot_code(word[u], s) == 0);
            if (lane == s) mine = bits;
        }
        if (lane < 8) crit_bits[g.slot_word(lane, z[u], y[u], w[u])] = mine;
    }
}

// Zeroes the words that the lower-star kernel finishes with atomicOr: those on the + faces of its
// tiles (x = 31 mod 32, y = TY-1 mod TY, z = TZ-1 mod TZ), which receive codes from the next tiles'
// stars.  Every other word gets one plain store, so it needs no zeroing.  A warp per (y, z) row:
// a row on a y or z face is cleared whole, any other row only at x = 31 mod 32.
__global__ void __launch_bounds__(256) zero_face_words(Geom g, uint32_t* __restrict__ words, int ty, int tz) {
    const uint32_t row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;  // ny * nz < 2^31
    const int lane = threadIdx.x & 31;
    if (row >= uint32_t(g.ny) * uint32_t(g.nz)) return;  // warp-uniform
    const uint32_t z = g.div_ny.div(row), y = row - z * uint32_t(g.ny);
    uint32_t* w = words + int64_t(row) * g.nx;
    if (int(y) % ty == ty - 1 || int(z) % tz == tz - 1) {
        for (int x = lane; x < g.nx; x += 32) w[x] = 0;
    } else {
        for (int x = 32 * lane + 31; x < g.nx; x += 32 * 32) w[x] = 0;
    }
}

// Tile variants the autotuner chooses from: (TY, TZ, threads).
struct Variant {
    int ty, tz, threads;
};
constexpr Variant VARIANTS[] = {{8, 8, 512},   {8, 4, 256},  {4, 8, 256},  {8, 16, 512}, {16, 8, 512},
                                {16, 8, 1024}, {16, 16, 512}, {8, 8, 256}, {16, 8, 256}};
constexpr int N_VARIANTS = int(sizeof(VARIANTS) / sizeof(VARIANTS[0]));

template <int TY, int TZ, int THREADS>
cudaError_t launch_tile(const Geom& g, const float* d_field, uint32_t* words, uint32_t* status, cudaStream_t s) {
    const size_t smem = sizeof(Shared<TY, TZ, THREADS>);
    // set on every call: the attribute is per device, and plans may live on several devices
    cudaError_t e =
        cudaFuncSetAttribute(gradient_kernel<TY, TZ, THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, (g.nz + TZ - 1) / TZ);
    gradient_kernel<TY, TZ, THREADS><<<grid, THREADS, smem, s>>>(g, d_field, words, status);
    return cudaGetLastError();
}

cudaError_t launch_zero_faces(int v, const Geom& g, uint32_t* words, cudaStream_t s) {
    if (v < 0 || v >= N_VARIANTS) v = 0;
    const int64_t rows = int64_t(g.ny) * g.nz;
    zero_face_words<<<unsigned((rows * 32 + 255) / 256), 256, 0, s>>>(g, words, VARIANTS[v].ty, VARIANTS[v].tz);
    return cudaGetLastError();
}

// The words of a whole grid with tile variant v: zero the face words, then the lower-star kernel.
cudaError_t launch_words(int v, const Geom& g, const float* d_field, uint32_t* words, uint32_t* status,
                         cudaStream_t s) {
    const cudaError_t e = launch_zero_faces(v, g, words, s);
    if (e != cudaSuccess) return e;
    switch (v) {
        case 1: return launch_tile<8, 4, 256>(g, d_field, words, status, s);
        case 2: return launch_tile<4, 8, 256>(g, d_field, words, status, s);
        case 3: return launch_tile<8, 16, 512>(g, d_field, words, status, s);
        case 4: return launch_tile<16, 8, 512>(g, d_field, words, status, s);
        case 5: return launch_tile<16, 8, 1024>(g, d_field, words, status, s);
        case 6: return launch_tile<16, 16, 512>(g, d_field, words, status, s);
        case 7: return launch_tile<8, 8, 256>(g, d_field, words, status, s);
        case 8: return launch_tile<16, 8, 256>(g, d_field, words, status, s);
        default: return launch_tile<8, 8, 512>(g, d_field, words, status, s);
    }
}

cudaError_t launch_gradient(int v, const Geom& g, const float* d_field, uint32_t* words, uint32_t* crit_bits,
                            uint32_t* status, cudaStream_t s, const Plan* p = nullptr) {
    cudaError_t e = launch_zero_faces(v, g, words, s);
    if (e != cudaSuccess) return e;
    if (p) record_event(p, p->gev0, s);  // the lower-star kernel alone is timed
    switch (v) {
        case 1: e = launch_tile<8, 4, 256>(g, d_field, words, status, s); break;
        case 2: e = launch_tile<4, 8, 256>(g, d_field, words, status, s); break;
        case 3: e = launch_tile<8, 16, 512>(g, d_field, words, status, s); break;
        case 4: e = launch_tile<16, 8, 512>(g, d_field, words, status, s); break;
        case 5: e = launch_tile<16, 8, 1024>(g, d_field, words, status, s); break;
        case 6: e = launch_tile<16, 16, 512>(g, d_field, words, status, s); break;
        case 7: e = launch_tile<8, 8, 256>(g, d_field, words, status, s); break;
        case 8: e = launch_tile<16, 8, 256>(g, d_field, words, status, s); break;
        default: e = launch_tile<8, 8, 512>(g, d_field, words, status, s); break;
    }
    if (p) record_event(p, p->gev1, s);
    if (e != cudaSuccess) return e;
    const int64_t warps = (int64_t(g.nz) * g.ny * g.W + CB_WORDS - 1) / CB_WORDS;
    critical_bitmaps<<<int((warps * 32 + 255) / 256), 256, 0, s>>>(g, words, crit_bits);
    return cudaGetLastError();
}

// Autotuning: the tile variant that computes this grid's words fastest on this device, timed on
// the field at hand (every variant gives the same words) and remembered per device and shape.
std::mutex tune_mu;
std::map<std::tuple<int, int, int, int>, int> tune_cache;

int tune_variant(Plan* p, const float* d_field, cudaStream_t s) {
    const Geom& g = p->g;
    const auto key = std::make_tuple(p->device, g.nx, g.ny, g.nz);
    {
        std::lock_guard<std::mutex> lk(tune_mu);
        auto it = tune_cache.find(key);
        if (it != tune_cache.end()) return it->second;
    }
    auto* words = static_cast<uint32_t*>(p->words.ptr);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return 0;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return 0;
    }
    // a warm-up launch of every variant, then three rounds over all of them (so that a clock
    // still ramping up, or a neighbour's burst, does not favour one variant); each variant's
    // best round counts
    float best_of[N_VARIANTS];
    int nv = N_VARIANTS;
    for (int v = 0; v < nv; ++v) {
        best_of[v] = 1e30f;
        if (launch_words(v, g, d_field, words, p->status_word(), s) != cudaSuccess) nv = v;
    }
    for (int r = 0; r < 3; ++r)
        for (int v = 0; v < nv; ++v) {
            cudaEventRecord(e0, s);
            launch_words(v, g, d_field, words, p->status_word(), s);
            cudaEventRecord(e1, s);
            float t = 0;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) t = 1e30f;
            best_of[v] = std::min(best_of[v], t);
        }
    int best = 0;
    for (int v = 1; v < nv; ++v)
        if (best_of[v] < best_of[best]) best = v;
    cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lk(tune_mu);
    tune_cache[key] = best;
    return best;
}

}  // namespace

msc_status run_gradient(Plan* p, const float* d_field, cudaStream_t s) {
    const Geom& g = p->g;
    msc_status st;
    if ((st = ensure(p, p->words, sizeof(uint32_t) * size_t(g.nverts)))) return st;
    if ((st = ensure(p, p->crit_bits, sizeof(uint32_t) * size_t(g.slot_words())))) return st;
    // the tile variant: forced by the plan's options, else tuned on the first synchronised run
    if (p->opts.gradient_tile > 0) p->grad_variant = std::min(int(p->opts.gradient_tile), N_VARIANTS) - 1;
    else if (p->grad_variant < 0 && !p->capturing) p->grad_variant = tune_variant(p, d_field, s);
    const int v = std::max(0, p->grad_variant);
    p->stats.gradient_tile = VARIANTS[v].ty | (VARIANTS[v].tz << 8) | (int64_t(VARIANTS[v].threads) << 16);
    launched(p, 3);
    return check_cuda(p,
                      launch_gradient(v, g, d_field, static_cast<uint32_t*>(p->words.ptr),
                                      static_cast<uint32_t*>(p->crit_bits.ptr), p->status_word(), s, p),
                      "gradient launch");
}

// Loads the kernels of launch_gradient_raw on the current device now (under lazy module loading
// CUDA would load them, and take device memory for their code, at their first launch) and sets
// the lower-star kernel's shared-memory limit there.
cudaError_t load_gradient_raw() {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, zero_face_words);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, gradient_kernel<8, 8, 512>);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gradient_kernel<8, 8, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(sizeof(Shared<8, 8, 512>)));
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, critical_bitmaps);
    return e;
}

// The same launches on caller-supplied buffers, with no plan and no allocation (used by the
// no-allocation entry point, static_entry.cu).
cudaError_t launch_gradient_raw(const Geom& g, const float* d_field, uint32_t* words, uint32_t* crit_bits,
                                uint32_t* status, cudaStream_t s) {
    return launch_gradient(0, g, d_field, words, crit_bits, status, s);
}

}  // namespace msc
