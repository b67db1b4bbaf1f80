// vs_noalloc.cu -- vortex check without any allocation.
//
// vs_vortex_check needs scratch memory (a plane of current labels and a few
// counters), which a field allocates when it is created.  This entry point
// runs the same two kernels on buffers the caller already owns and keeps the
// scratch in a fixed, file-scope device array instead, so it never calls
// cudaMalloc, cudaFree or an allocating library routine.
#include <cstring>
#include <mutex>

#include "vs_api_internal.h"

using namespace vs;

// Scratch shared by every call: the current-label plane (one byte per link)
// and eight 64-bit counters.  Every GPU that loads the library holds it until
// the process exits.
static __device__ __align__(256) int8_t g_noalloc_labels[VS_NOALLOC_MAX_LINKS];
static __device__ __align__(256) unsigned long long g_noalloc_counts[8];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
int8_t *g_labels_addr[kMaxDevices];
unsigned long long *g_counts_addr[kMaxDevices];
bool g_ready[kMaxDevices];

// Device addresses of the scratch arrays on the current device, looked up once
// per device (host code cannot use the arrays' names as device pointers).
vs_status scratch_of_current_device(int8_t **labels, unsigned long long **counts) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "vs_vortex_check_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices)
        return fail(VS_EUNSUPPORTED, "vs_vortex_check_noalloc: device %d beyond %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_ready[dev]) {
        void *pl = nullptr, *pc = nullptr;
        e = cudaGetSymbolAddress(&pl, g_noalloc_labels);
        if (e != cudaSuccess) return cuda_fail(e, "vs_vortex_check_noalloc: cudaGetSymbolAddress(labels)");
        e = cudaGetSymbolAddress(&pc, g_noalloc_counts);
        if (e != cudaSuccess) return cuda_fail(e, "vs_vortex_check_noalloc: cudaGetSymbolAddress(counters)");
        g_labels_addr[dev] = static_cast<int8_t *>(pl);
        g_counts_addr[dev] = static_cast<unsigned long long *>(pc);
        g_ready[dev] = true;
    }
    *labels = g_labels_addr[dev];
    *counts = g_counts_addr[dev];
    return VS_OK;
}

}  // namespace

extern "C" vs_status vs_vortex_check_noalloc(const void *links, const int8_t *ref_labels,
                                             const int32_t dims[4], int32_t precision,
                                             int32_t storage, void *stream, vs_vortex_report *out) {
    if (!links || !ref_labels || !dims || !out)
        return fail(VS_EINVAL, "vs_vortex_check_noalloc: NULL argument");
    if (precision != VS_FP64 && precision != VS_FP32)
        return fail(VS_EINVAL, "vs_vortex_check_noalloc: bad precision");
    if (storage != VS_LINK18 && storage != VS_LINK12)
        return fail(VS_EINVAL, "vs_vortex_check_noalloc: bad storage");
    if (precision == VS_FP64 && storage == VS_LINK12)
        return fail(VS_EUNSUPPORTED, "vs_vortex_check_noalloc: 12-real storage is FP32 only");
    long long V = 1;
    for (int k = 0; k < 4; ++k) {
        if (dims[k] < 4 || dims[k] % 4)
            return fail(VS_EINVAL, "vs_vortex_check_noalloc: extents must be positive multiples of 4");
        V *= dims[k];
    }
    if (4 * V > (long long)VS_NOALLOC_MAX_LINKS)
        return fail(VS_EINVAL,
                    "vs_vortex_check_noalloc: %lld links exceed the fixed scratch of %lld links "
                    "(at most %lld sites); use vs_vortex_check for larger lattices",
                    4 * V, (long long)VS_NOALLOC_MAX_LINKS, (long long)VS_NOALLOC_MAX_LINKS / 4);
    int8_t *cur = nullptr;
    unsigned long long *cnt = nullptr;
    vs_status st = scratch_of_current_device(&cur, &cnt);
    if (st) return st;
    Geo g;
    for (int k = 0; k < 4; ++k) g.L[k] = dims[k];
    g.Q = dims[0] / 4;
    g.V = (int)V;
    g.P = V;
    cudaStream_t s = (cudaStream_t)stream;
    // counters start at zero, the minimum margin at a huge value; the label
    // plane needs no clearing (every link's entry is written before it is read)
    cudaError_t e = cudaMemsetAsync(cnt, 0, 3 * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt + 3, 0x7f, sizeof(unsigned long long), s);
    if (e == cudaSuccess)
        e = launch_vortex(precision == VS_FP32, storage == VS_LINK12 ? 12 : 18, g, links, ref_labels, cur,
                          cnt, cnt + 3, s);
    unsigned long long h[4] = {0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, cnt, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "vs_vortex_check_noalloc");
    out->n_links = 4 * V;
    out->n_label_diff = (int64_t)h[0];
    out->n_charge_diff = (int64_t)h[1];
    out->n_near_boundary = (int64_t)h[2];
    double m;
    memcpy(&m, &h[3], sizeof m);
    out->min_margin = m;
    return VS_OK;
}
