// scan_noalloc.cu -- the exclusive prefix sum of the scan entry points, for
// callers that must not allocate device memory.
//
// spr_exclusive_scan_u32 takes its look-back scratch (one status word per
// tile, a ticket, a flag word) from the device allocator on every call.
// Some callers cannot do that: a caller that runs while device memory is
// exhausted (for instance to compact a work list while recovering from an
// out-of-memory error), a caller inside an allocator hook, where allocating
// would re-enter the allocator, and a latency-bound loop that shares the GPU
// with other streams, where cudaMalloc and cudaFree may synchronise the whole
// device.  spr_exclusive_scan_u32_noalloc serves them: its scratch is one
// file-scope device array, sized for at most kNoAllocMaxN elements, whose
// address is resolved once per device.  The paper has no counterpart of this
// entry point; the scan itself is the same kernel (scan.cuh).
//
// Because the array is a single object per device, two calls in flight on
// one device at the same time (on different streams, or from different host
// threads without ordering between them) share it and corrupt each other's
// results; callers order their calls, e.g. by issuing them on one stream.

#include <algorithm>
#include <mutex>

#include "scan.cuh"
#include "spr_common.cuh"

namespace spr {
namespace {

// Largest n accepted: 2^26 elements, i.e. 32768 tiles of kScanTile.
constexpr int64_t kNoAllocMaxN = int64_t(1) << 26;
constexpr int64_t kNoAllocTiles = kNoAllocMaxN / kScanTile;
static_assert(kNoAllocMaxN % kScanTile == 0, "whole tiles");

// Layout of the scratch, in 64-bit words: [0, kNoAllocTiles) tile status
// words; words kTicketWord.. hold the ticket, done and epoch counters (three
// uint32); word kFlagsWord the flag word.  The control words sit in their
// own 128-byte lines.  All of these must be zero when the kernel starts;
// every call clears the status words of the tiles it uses and the control
// words on its stream before the launch.
constexpr int64_t kTicketWord = kNoAllocTiles;
constexpr int64_t kFlagsWord = kNoAllocTiles + 16;
constexpr int64_t kNoAllocWords = kNoAllocTiles + 32;  // 256 KiB + 256 B

static __device__ __align__(256) unsigned long long g_noalloc_scan_scratch[kNoAllocWords];

struct NoAllocCount {
    const uint32_t *a;
    __device__ bool enabled() const { return true; }
    __device__ uint32_t operator()(int64_t i) const { return a[i]; }
};

struct NoAllocEmit {
    uint32_t *out;
    __device__ void operator()(int64_t i, uint32_t pre, uint32_t) const { out[i] = pre; }
};

// Per-device set-up: the scratch address (cudaGetSymbolAddress with the
// device current), the SM count that sizes the persistent grid, and the
// kernel itself.  Under CUDA's lazy module loading the module holding the
// array and the kernel's code are placed in device memory the first time
// they are used; resolving the symbol and querying the kernel's attributes
// here makes both happen in this first call, not in a later one (which may
// then run when device memory is exhausted).
constexpr int kMaxDevices = 64;
struct DeviceSetup {
    unsigned long long *scratch = nullptr;
    int sms = 0;
};
std::mutex g_setup_mu;
DeviceSetup g_setup[kMaxDevices];

int setup_for_current_device(DeviceSetup &out)
{
    int dev = 0;
    SPR_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices)
        return set_error(SPR_ERR_INVALID_ARG, "device ordinal %d beyond the %d supported", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_setup_mu);
    DeviceSetup &d = g_setup[dev];
    if (!d.scratch) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scan_scratch);
        if (e != cudaSuccess || !p)
            return set_error(SPR_ERR_CUDA, "cudaGetSymbolAddress of the scan scratch failed: %s",
                             cudaGetErrorString(e));
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess)
            return set_error(SPR_ERR_CUDA, "cudaDeviceGetAttribute failed: %s", cudaGetErrorString(e));
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, compact_kernel<NoAllocCount, NoAllocEmit>);
        if (e != cudaSuccess)
            return set_error(SPR_ERR_CUDA, "loading the scan kernel failed: %s", cudaGetErrorString(e));
        d.sms = sms > 0 ? sms : 1;
        d.scratch = static_cast<unsigned long long *>(p);
    }
    out = d;
    return SPR_OK;
}

}  // namespace
}  // namespace spr

using namespace spr;

extern "C" int spr_exclusive_scan_u32_noalloc(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total,
                                              spr_stream stream)
{
    clear_error();
    if (n < 0 || (n > 0 && (!in || !out))) return set_error(SPR_ERR_INVALID_ARG, "bad scan arguments");
    if (n > kNoAllocMaxN)
        return set_error(SPR_ERR_INVALID_ARG,
                         "scan of %lld elements exceeds the static scratch limit of %lld elements",
                         (long long)n, (long long)kNoAllocMaxN);
    DeviceSetup d;
    SPR_TRY(setup_for_current_device(d));
    cudaStream_t s = as_stream(stream);
    const int64_t tiles = std::max<int64_t>(1, scan_tiles(n));
    unsigned long long *status = d.scratch;
    unsigned int *ticket = reinterpret_cast<unsigned int *>(d.scratch + kTicketWord);
    unsigned int *flags = reinterpret_cast<unsigned int *>(d.scratch + kFlagsWord);
    // what must start at zero: the used status words, the ticket, the flags
    SPR_CUDA_TRY(cudaMemsetAsync(status, 0, (size_t)tiles * sizeof(unsigned long long), s));
    SPR_CUDA_TRY(cudaMemsetAsync(d.scratch + kTicketWord, 0,
                                 (size_t)(kNoAllocWords - kTicketWord) * sizeof(unsigned long long), s));
    ScanCtl ctl{status, tiles, ticket, flags, kDefaultSpinLimit, -1, nullptr, 0u};
    const int64_t grid = std::min<int64_t>(tiles, (int64_t)d.sms * 4);
    compact_kernel<NoAllocCount, NoAllocEmit>
        <<<(unsigned)grid, kScanThreads, 0, s>>>(n, nullptr, ctl, NoAllocCount{in}, NoAllocEmit{out}, total);
    SPR_CUDA_TRY(cudaGetLastError());
    uint32_t f = 0;
    SPR_CUDA_TRY(cudaMemcpyAsync(&f, flags, sizeof(f), cudaMemcpyDeviceToHost, s));
    SPR_CUDA_TRY(cudaStreamSynchronize(s));
    if (f) return set_error(SPR_ERR_DEVICE_TIMEOUT, "a look-back wait gave up after its poll limit");
    return SPR_OK;
}
