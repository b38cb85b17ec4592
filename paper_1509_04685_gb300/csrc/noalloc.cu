// cola_density_noalloc: the density call of cola_density, for callers that
// cannot hand the library any scratch memory.  Examples are a host application
// that has already given all device memory to its own pool allocator and
// forbids allocations from outside it, and an in-situ analysis step inside a
// running simulation whose device memory is fully reserved.  The fixed-point
// CIC mesh that the deposit accumulates into lives in a file-scope device
// array of fixed size instead of a caller workspace; no allocation happens
// anywhere on this path.
#include <mutex>

#include "cola_common.cuh"

namespace cola {

// Largest mesh side this entry point accepts: 128^3 cells of 8-byte counts
// (16 MiB), plus one status word.  Every GPU that loads the library holds the
// array until the process exits.
constexpr int kNoAllocMaxNg = 128;
constexpr size_t kNoAllocCells = (size_t)kNoAllocMaxNg * kNoAllocMaxNg * kNoAllocMaxNg;

static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoAllocCells + 32];

constexpr int kMaxDevices = 64;
static unsigned long long* g_scratch_ptr[kMaxDevices];
static std::mutex g_scratch_mutex;

// Device address of the array on the current device.  The symbol name is only
// a host-side stand-in: it must not be handed to a kernel; cudaGetSymbolAddress
// gives the real device address.  Outside stream capture the address is looked
// up on every call, so a device reset (after which the module is loaded again
// and the array may move) never leaves a stale address behind.  While `s` is
// being captured the lookup is not made (it is not a capturable call): the
// address cached by the last uncaptured call on this device is used, and with
// none cached the call fails with COLA_EINVAL.
static int scratch_for_current_device(cudaStream_t s, unsigned long long** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return COLA_ECUDA;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return COLA_ECUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return COLA_ECUDA;
        g_scratch_ptr[dev] = static_cast<unsigned long long*>(p);
    } else if (!g_scratch_ptr[dev]) {
        return COLA_EINVAL;
    }
    *out = g_scratch_ptr[dev];
    return COLA_OK;
}

// If the deposit met a non-finite or absurd displacement, poison the output
// with NaN: this entry point has no status word the caller can read.  The
// flag itself is cleared at the start of the next call.
__global__ void k_noalloc_poison(float* delta, long long n3, const int* status) {
    if (!*status) return;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (long long)gridDim.x * blockDim.x)
        delta[i] = __int_as_float(0x7fc00000);
}

}  // namespace cola

using namespace cola;

extern "C" int cola_density_noalloc(const cola_config* cfg, const cola_state* st, float* delta, void* stream) {
    if (!cfg || !st || !st->d || !delta) return COLA_EINVAL;
    if (!(cfg->box > 0.0)) return COLA_EINVAL;
    // the sizes cola_density accepts, and no more cells than the array holds
    if (!mesh_ok(cfg->nq) || !mesh_ok(cfg->ng) || cfg->ng > kNoAllocMaxNg) return COLA_EUNSUPPORTED_SIZE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned long long* scratch = nullptr;
    int rc = scratch_for_current_device(s, &scratch);
    if (rc) return rc;
    const size_t n3 = (size_t)cfg->ng * cfg->ng * cfg->ng;
    int* status = reinterpret_cast<int*>(scratch + kNoAllocCells);
    // The fix-up kernel clears every count it reads, and device arrays start at
    // zero, so after a completed call the counts are already zero.  The clear
    // guards against a previous call that stopped between its deposit and its
    // fix-up (a failed launch) and leaves the array dirty; it costs about as
    // much as one read of n3 counts.  The poison flag is cleared the same way.
    if (cudaMemsetAsync(scratch, 0, n3 * sizeof(unsigned long long), s) != cudaSuccess) return COLA_ECUDA;
    if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) return COLA_ECUDA;
    if ((rc = launch_deposit_ex(st->d, nullptr, nullptr, nullptr, scratch, cfg->nq, cfg->ng, cfg->box, nullptr, status,
                                s)))
        return rc;
    const double ratio = (double)cfg->ng / (double)cfg->nq;
    if ((rc = launch_fix_to_delta(scratch, delta, cfg->ng, (float)(ratio * ratio * ratio / 1099511627776.0), s)))
        return rc;
    k_noalloc_poison<<<64, 256, 0, s>>>(delta, (long long)n3, status);
    return check_launch();
}
