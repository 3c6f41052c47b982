// sbt_sample_noalloc: the weighted draw of sbt_sample for callers that must
// not allocate device memory during the call.
//
// Some callers cannot allocate at call time: a serving process that hands the
// whole device to its own memory pool at start-up, or a latency-critical loop
// in which a cudaMalloc (which may synchronise the device) is not allowed.
// This entry point takes its scratch (the 128-bit sampling keys and the status
// word) from one fixed array in the library's device memory instead.  The
// array is SBT_SAMPLE_NOALLOC_MAX_N * 16 + 256 bytes (about 4 MiB); every GPU
// that loads the library holds it until the process exits.
//
// Host code cannot hand the array's name to a kernel: on the host that name
// is only a stand-in for the symbol, not a device address.  The first call on
// each device therefore looks the address up with cudaGetSymbolAddress (with
// that device current) and caches it; that first call should come before any
// stream capture.  Later calls outside a capture look it up again, so the
// cache never outlives a device reset.  All calls share the array and it keeps the last call's
// contents, so the status word is cleared before every launch; calls that
// overlap on the GPU (unordered streams or threads) race on the array.
#include "sambaten.h"
#include "sbt_internal.cuh"

#include <cstring>
#include <mutex>
#include <string>

namespace {

constexpr size_t kKeyBytes = (size_t)SBT_SAMPLE_NOALLOC_MAX_N * 16;
constexpr size_t kScratchBytes = kKeyBytes + 256;

static __device__ __align__(256) unsigned char g_sample_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  Outside stream
// capture it is looked up again on every call (cheap once the module is
// loaded), so a context that was reset and recreated, with the array at a new
// address, is never handed a stale pointer; inside a capture the address
// cached by an earlier call is used.
cudaError_t scratch_address(cudaStream_t st, unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev] || cs == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_sample_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" sbt_status sbt_sample_noalloc(const uint64_t *w, int64_t N, int64_t n, uint64_t seed,
                                         uint32_t stream_id, int32_t mode, int32_t rep, uint32_t batch,
                                         int32_t *out, void *stream) {
    if (!w || !out || N < 1 || n < 0 || n > N) {
        sbt::set_last_error("sbt_sample_noalloc: bad arguments");
        return SBT_E_INVALID;
    }
    if (N > SBT_SAMPLE_NOALLOC_MAX_N) {
        sbt::set_last_error("sbt_sample_noalloc: N = " + std::to_string(N) + " exceeds SBT_SAMPLE_NOALLOC_MAX_N = " +
                        std::to_string(SBT_SAMPLE_NOALLOC_MAX_N) + " (use sbt_sample)");
        return SBT_E_INVALID;
    }
    if (mode < 0 || mode > 15 || rep < 0) {
        sbt::set_last_error("sbt_sample_noalloc: mode or rep out of range");
        return SBT_E_INVALID;
    }
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *base = nullptr;
    cudaError_t e = scratch_address(st, &base);
    if (e != cudaSuccess) {
        sbt::set_last_error(std::string("sbt_sample_noalloc: scratch address: ") + cudaGetErrorString(e));
        return SBT_E_CUDA;
    }
    sbt::DevStatus *ds = reinterpret_cast<sbt::DevStatus *>(base + kKeyBytes);
    e = cudaMemsetAsync(ds, 0, sizeof(sbt::DevStatus), st);
    sbt::SampleParams sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.w[0] = (const unsigned long long *)w;
    sp.N[0] = (int)N;
    sp.n[0] = (int)n;
    sp.mode_id[0] = mode;
    sp.nmodes = 1;
    sp.nrep = 1;
    sp.rep0 = rep;
    sp.out = out;
    sp.out_stride = n;
    sp.khi = reinterpret_cast<unsigned long long *>(base);
    sp.klo = reinterpret_cast<unsigned long long *>(base) + N;
    sp.key_stride = N;
    sp.seed = seed;
    sp.stream_id = stream_id;
    sp.batch = batch;
    sp.status = ds;
    if (e == cudaSuccess) e = sbt::launch_sample(sp, st);
    unsigned herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, &ds->err, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        sbt::set_last_error(std::string("sbt_sample_noalloc: ") + cudaGetErrorString(e));
        return SBT_E_CUDA;
    }
    if (herr & sbt::ERR_SAMPLE) {
        sbt::set_last_error("sbt_sample_noalloc: sample size above the number of positive weights");
        return SBT_E_INVALID;
    }
    return SBT_OK;
}

