// vs_noalloc.cu -- vortex check without device allocation.
//
// vs_vortex_check needs scratch memory (a plane of current labels and a few
// counters), which a field allocates when it is created.  This entry point
// runs the same two kernels on buffers the caller already owns and keeps the
// scratch in a fixed, file-scope device array instead, so it never allocates
// device memory: no cudaMalloc, cudaFree or allocating library routine.  The
// one allocation it ever makes is on the host: a 64-byte pinned, mapped block
// per device, made once by vs_noalloc_prepare (which vs_create calls for its
// device) or else by the first call on that device.  It also makes no
// synchronising CUDA call, so it stays usable while another stream of the
// thread captures a graph in the global capture mode: a last one-thread
// kernel publishes the counters and a sequence number into the mapped host
// block, and the host waits for that number (with a time limit).
#include <atomic>
#include <chrono>
#include <cstring>
#include <mutex>
#include <thread>

#include "vs_api_internal.h"

using namespace vs;

// Scratch shared by every call: the current-label plane (one byte per link)
// and eight 64-bit counters.  Every GPU that loads the library holds it until
// the process exits.
static __device__ __align__(256) int8_t g_noalloc_labels[VS_NOALLOC_MAX_LINKS];
static __device__ __align__(256) unsigned long long g_noalloc_counts[8];

// Copy the four report words to the mapped host block, then the sequence
// number: the host reads the words once it sees the number.
__global__ void k_noalloc_publish(const unsigned long long *cnt, volatile unsigned long long *host,
                                  unsigned long long seq) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        for (int k = 0; k < 4; ++k) host[k] = cnt[k];
        __threadfence_system();
        host[4] = seq;
    }
}

namespace {

constexpr int kMaxDevices = 64;
constexpr double kWaitLimitMs = 30000.0;   // the check takes milliseconds; a GPU that stalls this long is lost

struct DeviceScratch {
    std::mutex mu;                          // one call at a time per device: the scratch is shared
    bool ready = false;
    int8_t *labels = nullptr;
    unsigned long long *counts = nullptr;
    volatile unsigned long long *host = nullptr;   // mapped pinned block: 4 report words + sequence
    unsigned long long *host_dev = nullptr;        // its device address
    unsigned long long seq = 0;
    // sequence number of a call that gave up waiting: its kernels may still
    // use the scratch, so calls are refused until its result is published
    unsigned long long stale = 0;
};
DeviceScratch g_dev[kMaxDevices];

// Once per device, with that device current: the device addresses of the
// scratch arrays (host code cannot use the arrays' names as device
// pointers), the mapped host block, and the kernels this file launches
// loaded now (with lazy module loading a first launch loads them).  The
// thread's capture mode is relaxed meanwhile, so that a first call made
// while another stream of the thread captures a graph neither fails nor
// invalidates that capture.  Called with the device's mutex held.
vs_status setup(DeviceScratch &d) {
    if (d.ready) return VS_OK;
    cudaStreamCaptureMode mode = cudaStreamCaptureModeRelaxed;
    cudaError_t e = cudaThreadExchangeStreamCaptureMode(&mode);
    if (e != cudaSuccess) return cuda_fail(e, "vs_vortex_check_noalloc: cudaThreadExchangeStreamCaptureMode");
    void *pl = nullptr, *pc = nullptr, *ph = nullptr, *phd = nullptr;
    const char *what = "cudaGetSymbolAddress";
    e = cudaGetSymbolAddress(&pl, g_noalloc_labels);
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&pc, g_noalloc_counts);
    if (e == cudaSuccess) {
        cudaFuncAttributes fa;
        what = "kernel loading";
        e = cudaFuncGetAttributes(&fa, k_noalloc_publish);
        if (e == cudaSuccess) e = preload_vortex_kernels();
    }
    if (e == cudaSuccess) {
        what = "cudaHostAlloc";
        e = cudaHostAlloc(&ph, 8 * sizeof(unsigned long long), cudaHostAllocMapped | cudaHostAllocPortable);
    }
    if (e == cudaSuccess) {
        what = "cudaHostGetDevicePointer";
        e = cudaHostGetDevicePointer(&phd, ph, 0);
        if (e != cudaSuccess) cudaFreeHost(ph);
    }
    cudaStreamCaptureMode back = mode;
    cudaThreadExchangeStreamCaptureMode(&back);
    if (e != cudaSuccess) return cuda_fail(e, what);
    memset(ph, 0, 8 * sizeof(unsigned long long));
    d.labels = static_cast<int8_t *>(pl);
    d.counts = static_cast<unsigned long long *>(pc);
    d.host = static_cast<volatile unsigned long long *>(ph);
    d.host_dev = static_cast<unsigned long long *>(phd);
    d.ready = true;
    return VS_OK;
}

}  // namespace

extern "C" vs_status vs_noalloc_prepare(int32_t device) {
    if (device < 0 || device >= kMaxDevices)
        return fail(VS_EUNSUPPORTED, "vs_noalloc_prepare: device %d beyond %d", device, kMaxDevices);
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return cuda_fail(e, "vs_noalloc_prepare: cudaGetDevice");
    if (cur != device && (e = cudaSetDevice(device)) != cudaSuccess) return cuda_fail(e, "vs_noalloc_prepare");
    vs_status st;
    {
        std::lock_guard<std::mutex> lock(g_dev[device].mu);
        st = setup(g_dev[device]);
    }
    if (cur != device) cudaSetDevice(cur);
    return st;
}

extern "C" vs_status vs_vortex_check_noalloc(const void *links, const int8_t *ref_labels, const void *gauge,
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
    for (int k = 0; k < 4; ++k)
        if (dims[k] < 4 || dims[k] % 4)
            return fail(VS_EINVAL, "vs_vortex_check_noalloc: extents must be positive multiples of 4");
    // the scratch label plane is indexed like the field's: 4 x plane stride
    // positions (the sites, plus the layout's unused positions when Lx/4 is
    // 5, 6 or 7)
    const Geo g = make_geo(dims);
    if (4 * g.P > (long long)VS_NOALLOC_MAX_LINKS)
        return fail(VS_EINVAL,
                    "vs_vortex_check_noalloc: %lld link positions exceed the fixed scratch of %lld "
                    "(at most %lld sites, e.g. 32^3 x 64); use vs_vortex_check for larger lattices",
                    4 * g.P, (long long)VS_NOALLOC_MAX_LINKS, (long long)VS_NOALLOC_MAX_LINKS / 4);
    const long long V = g.V;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "vs_vortex_check_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices)
        return fail(VS_EUNSUPPORTED, "vs_vortex_check_noalloc: device %d beyond %d", dev, kMaxDevices);
    DeviceScratch &d = g_dev[dev];
    std::lock_guard<std::mutex> lock(d.mu);
    vs_status st = setup(d);
    if (st) return st;
    if (d.stale) {
        if (d.host[4] != d.stale)
            return fail(VS_EBUSY,
                        "vs_vortex_check_noalloc: an earlier call on device %d gave up waiting and its kernels "
                        "have not finished; the shared scratch stays in use until they do", dev);
        d.stale = 0;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned long long seq = ++d.seq;
    // counters start at zero, the minimum margin at a huge value; the label
    // plane needs no clearing (every link's entry is written before it is read)
    unsigned long long *cnt = d.counts;
    e = cudaMemsetAsync(cnt, 0, 3 * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt + 3, 0x7f, sizeof(unsigned long long), s);
    if (e == cudaSuccess)
        e = launch_vortex(precision == VS_FP32, storage == VS_LINK12 ? 12 : 18, g, links, ref_labels, d.labels,
                          cnt, cnt + 3, s, gauge);
    if (e == cudaSuccess) {
        k_noalloc_publish<<<1, 32, 0, s>>>(cnt, d.host_dev, seq);
        count_launches(1);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_fail(e, "vs_vortex_check_noalloc");
    // wait for the sequence number: spin briefly, then sleep between looks
    const auto t0 = std::chrono::steady_clock::now();
    for (long n = 0; d.host[4] != seq; ++n) {
        if (n > 1000) std::this_thread::sleep_for(std::chrono::microseconds(20));
        if ((n & 255) == 0 &&
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count() > kWaitLimitMs) {
            d.stale = seq;
            return fail(VS_EDEVICE, "vs_vortex_check_noalloc: no result from the GPU after %.0f ms", kWaitLimitMs);
        }
    }
    std::atomic_thread_fence(std::memory_order_acquire);
    unsigned long long h[4];
    for (int k = 0; k < 4; ++k) h[k] = d.host[k];
    out->n_links = 4 * V;
    out->n_label_diff = (int64_t)h[0];
    out->n_charge_diff = (int64_t)h[1];
    out->n_near_boundary = (int64_t)h[2];
    double m;
    memcpy(&m, &h[3], sizeof m);
    out->min_margin = m;
    return VS_OK;
}
