// noalloc.cu -- cwthf_deposit_noalloc: the CIC deposit on a fixed scratch
// area that lives in the library image, for callers that cannot allocate
// device memory.
//
// Who needs it: code that must not call cudaMalloc at all -- work recorded
// while a stream is being captured into a CUDA graph (allocation calls are
// not capturable), hosts whose device memory is owned by another allocator
// or pool and where a stray cudaMalloc would break its accounting, and
// latency-critical loops where cudaMalloc / cudaFree would synchronise the
// device.  They pass only inputs and outputs; the binning scratch the
// deposit needs (bin counts and offsets, the packed particle records, the
// scan's block sums, the status word) is the array below.
//
// Limits: ng <= kNoAllocMaxNg and np <= kNoAllocMaxNp (3.3 MB of scratch).
// Larger calls are rejected with CWTHF_E_SCRATCH_LIMIT before anything is
// queued.  The array is loaded with the library on every GPU that uses it
// and stays allocated until the process exits.
//
// Sharing: every call, from any thread or stream, uses the same array and
// leaves its contents behind; each call clears what must start at zero.
// Two calls whose GPU work overlaps (different streams, or different host
// threads on one device) race on the array and give wrong results: order
// them on one stream.
//
// Set-up: every call made outside a stream capture looks the array's device
// address up with cudaGetSymbolAddress (with the device current); a call made
// during a capture reuses the address of the last such call on its device, so
// make one call on each device before capturing.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "internal.cuh"

namespace cwthf {

int check_ng(int ng);

namespace {

constexpr int kNoAllocMaxNg = 128;
constexpr int64_t kNoAllocMaxNp = 262144;
constexpr int64_t kMaxKeys = int64_t((kNoAllocMaxNg + kDepTX - 1) / kDepTX) * ((kNoAllocMaxNg + kDepTY - 1) / kDepTY) *
                             ((kNoAllocMaxNg + kDepTZ - 1) / kDepTZ) * kDepClasses;
constexpr size_t kScanWords = size_t(kMaxKeys / 4096) + 8;

constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kOffStatus = 0;
constexpr size_t kOffMtot = align256(kOffStatus + 16);
constexpr size_t kOffCount = align256(kOffMtot + 16);
constexpr size_t kOffOff = align256(kOffCount + size_t(kMaxKeys + 2) * 4);
constexpr size_t kOffCursor = align256(kOffOff + size_t(kMaxKeys + 2) * 4);
constexpr size_t kOffScan = align256(kOffCursor + size_t(kMaxKeys + 2) * 4);
constexpr size_t kOffRec = align256(kOffScan + kScanWords * 4);
constexpr size_t kOffMq = align256(kOffRec + size_t(kNoAllocMaxNp) * 8);
constexpr size_t kScratchBytes = align256(kOffMq + size_t(kNoAllocMaxNp) * 4);

// The fixed scratch.  In host code this name is only a host-side stand-in:
// its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_deposit_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

// Device address of the scratch on the current device, or nullptr on failure.
// Looked up on every call made outside a stream capture (so a module reloaded
// after cudaDeviceReset is seen); a call made while `s` is being captured
// uses the address of the last uncaptured call on this device.  Failures are
// not cleared from the runtime's error state, so the caller still sees them.
void* scratch_address(int dev, cudaStream_t s, int* sms) {
    if (dev < 0 || dev >= kMaxDevices) return nullptr;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> g(g_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        int n = 0;
        if (cudaGetSymbolAddress(&p, g_deposit_scratch) != cudaSuccess || !p ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            return nullptr;
        g_sms[dev] = n;
        g_addr[dev] = p;
    }
    *sms = g_sms[dev];
    return g_addr[dev];
}

}  // namespace
}  // namespace cwthf

using namespace cwthf;

extern "C" int cwthf_deposit_noalloc(const float* pos, const float* mass, double mass_unit, int64_t np, double L,
                                     int ng, int64_t* grid, int64_t* mtot, int* status, void* stream) {
    if (check_ng(ng)) return CWTHF_E_UNSUPPORTED_SIZE;
    if (ng > kNoAllocMaxNg || np > kNoAllocMaxNp) return CWTHF_E_SCRATCH_LIMIT;
    if (np < 0 || (np > 0 && !pos) || !grid || !(L > 0) || !std::isfinite(L) || !(mass_unit > 0) ||
        !std::isfinite(mass_unit))
        return CWTHF_E_INVALID_ARG;
    int dev = -1, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CWTHF_E_CUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned char* base = static_cast<unsigned char*>(scratch_address(dev, s, &sms));
    if (!base) return CWTHF_E_CUDA;
    DepositScratch sc;
    sc.status = reinterpret_cast<int*>(base + kOffStatus);
    sc.mtot = reinterpret_cast<unsigned long long*>(base + kOffMtot);
    sc.count = reinterpret_cast<uint32_t*>(base + kOffCount);
    sc.off = reinterpret_cast<uint32_t*>(base + kOffOff);
    sc.cursor = reinterpret_cast<uint32_t*>(base + kOffCursor);
    sc.scan_tmp = reinterpret_cast<uint32_t*>(base + kOffScan);
    sc.scan_cap = kScanWords;
    sc.rec = reinterpret_cast<unsigned long long*>(base + kOffRec);
    sc.mq = reinterpret_cast<uint32_t*>(base + kOffMq);
    sc.sm_count = sms;
    // the status word keeps the previous call's value: start from zero
    cudaError_t e = cudaMemsetAsync(sc.status, 0, sizeof(int), s);
    if (e != cudaSuccess) return CWTHF_E_CUDA;
    int rc = deposit_into_scratch(sc, pos, mass, mass_unit, np, L, ng, grid, s);
    if (rc) return rc;
    if (mtot && cudaMemcpyAsync(mtot, sc.mtot, 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return CWTHF_E_CUDA;
    if (status && cudaMemcpyAsync(status, sc.status, sizeof(int), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return CWTHF_E_CUDA;
    return CWTHF_OK;
}
