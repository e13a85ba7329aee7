// msc_gradient_critical_static: stages (a1)+(a2) for callers that cannot allocate device memory.
//
// The paper has no counterpart.  Some host programs reserve the whole GPU for their own memory
// pool, and some run this step inside a callback or a deadline-bound loop where cudaMalloc --
// which may synchronise the device and may fail -- is not allowed.  This entry point runs the
// same gradient kernel and ordered compaction as msc_gradient + msc_critical, but takes every
// output from the caller and keeps all scratch (critical bitmaps, word prefixes, scan sums, the
// status word) in one file-scope device array of MSC_STATIC_SCRATCH_BYTES.
//
// In host code the array's name is only a host-side stand-in, not a device address, so the
// address is looked up once per device with cudaGetSymbolAddress (with that device current)
// and passed to the kernels.  Under lazy module loading that lookup is also what loads the
// library's device code on the device and creates the array, which is why msc_static_prepare
// exists: a caller runs it before reserving the rest of the GPU.  Every call shares the array
// and overwrites it; overlapping calls race, which the header documents.
#include <mutex>

#include "scan.cuh"

namespace msc {

cudaError_t launch_gradient_raw(const Geom& g, const float* d_field, uint32_t* words, uint32_t* crit_bits,
                                uint32_t* status, cudaStream_t s);
cudaError_t load_gradient_raw();

namespace {

static __device__ __align__(256) unsigned char g_static_scratch[MSC_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on `dev` (looked up on the first call per device).
cudaError_t scratch_address(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_scratch_addr[dev]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = ptr;
    }
    *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
    return cudaSuccess;
}

size_t round_up(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace
}  // namespace msc

extern "C" msc_status msc_static_prepare(int device) {
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess) {
        cudaGetLastError();
        return MSC_ERR_CUDA;
    }
    if (device < 0 || device >= n) return MSC_ERR_ARG;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return MSC_ERR_CUDA;
    }
    unsigned char* base = nullptr;
    cudaError_t e = msc::scratch_address(device, &base);
    // load every kernel the entry point launches, so none is loaded lazily later
    cudaFuncAttributes a;
    if (e == cudaSuccess) e = msc::load_gradient_raw();
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, msc::scan_reduce_kernel<msc::CritSource>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, msc::scan_top_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, msc::scan_emit_kernel<msc::CritSource>);
    cudaSetDevice(prev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return MSC_ERR_CUDA;
    }
    return MSC_OK;
}

extern "C" msc_status msc_gradient_critical_static(const int64_t dims[3], const float* d_field, uint32_t* d_words,
                                                   uint32_t* const d_cells[4], const int64_t capacity[4],
                                                   int64_t counts[4], msc_stream_t stream) {
    using namespace msc;
    if (!dims || !d_field || !d_words || !d_cells || !capacity || !counts) return MSC_ERR_ARG;
    for (int i = 0; i < 3; ++i)
        if (dims[i] < 2 || dims[i] > (int64_t(1) << 30)) return MSC_ERR_ARG;
    for (int k = 0; k < 4; ++k)
        if (capacity[k] < 0 || (capacity[k] > 0 && !d_cells[k])) return MSC_ERR_ARG;
    const int64_t rx = 2 * dims[0] - 1, ry = 2 * dims[1] - 1, rz = 2 * dims[2] - 1;
    if (double(rx) * double(ry) * double(rz) >= 4294967295.0) return MSC_ERR_TOO_LARGE;
    Geom g;
    g.nx = int(dims[0]);
    g.ny = int(dims[1]);
    g.nz = int(dims[2]);
    g.finish();

    // scratch layout: status | bitmaps | prefixes | scan block sums | totals
    const int64_t len = seq_length(g);
    const int bps = int((len + SCAN_CHUNK - 1) / SCAN_CHUNK);
    const size_t off_bits = 256;
    const size_t off_prefix = off_bits + round_up(sizeof(uint32_t) * size_t(g.slot_words()));
    const size_t off_sums = off_prefix + round_up(sizeof(uint32_t) * size_t(g.slot_words()));
    const size_t off_totals = off_sums + round_up(sizeof(unsigned long long) * size_t(bps) * 4);
    const size_t need = off_totals + 256;
    if (need > MSC_STATIC_SCRATCH_BYTES) return MSC_ERR_TOO_LARGE;

    int dev = 0;
    unsigned char* base = nullptr;
    if (cudaGetDevice(&dev) != cudaSuccess || scratch_address(dev, &base) != cudaSuccess) {
        cudaGetLastError();
        return MSC_ERR_CUDA;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    uint32_t* status = reinterpret_cast<uint32_t*>(base);
    uint32_t* bits = reinterpret_cast<uint32_t*>(base + off_bits);
    uint32_t* prefix = reinterpret_cast<uint32_t*>(base + off_prefix);
    auto* sums = reinterpret_cast<unsigned long long*>(base + off_sums);
    auto* totals = reinterpret_cast<unsigned long long*>(base + off_totals);

    // the status word must start at zero; every other region is fully overwritten
    if (cudaMemsetAsync(status, 0, sizeof(uint32_t), s) != cudaSuccess) return MSC_ERR_CUDA;
    if (launch_gradient_raw(g, d_field, d_words, bits, status, s) != cudaSuccess) return MSC_ERR_CUDA;

    CritSource src{};
    src.g = g;
    src.bits = bits;
    src.prefix = prefix;
    src.status = status;
    scan_reduce_kernel<CritSource><<<bps * 4, SCAN_THREADS, 0, s>>>(src, len, bps, sums);
    scan_top_kernel<<<4, 1024, 0, s>>>(sums, bps, totals);
    unsigned long long tot[4] = {0, 0, 0, 0};
    uint32_t word = 0;
    if (cudaMemcpyAsync(tot, totals, sizeof(tot), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&word, status, sizeof(word), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return MSC_ERR_CUDA;
    }
    if (word & ST_NAN) return MSC_ERR_NAN;
    if (word) return MSC_ERR_INTERNAL;  // a lower-star cell left unclassified or a bounds check
    bool fits = true;
    for (int k = 0; k < 4; ++k) {
        counts[k] = int64_t(tot[k]);
        fits = fits && counts[k] <= capacity[k];
        src.out[k] = d_cells[k];
        src.cap[k] = uint64_t(capacity[k]);
    }
    if (!fits) return MSC_ERR_CAPACITY;
    scan_emit_kernel<CritSource><<<bps * 4, SCAN_THREADS, 0, s>>>(src, len, bps, sums);
    return cudaGetLastError() == cudaSuccess ? MSC_OK : MSC_ERR_CUDA;
}
