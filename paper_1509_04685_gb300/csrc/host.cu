// cola_step_host: one PM step (Sec. 2.2, Eqs. 1-2, exactly as cola_step) of a
// particle state held in host memory.  The copies are spread over the
// caller's stream and three side streams, so that several copy engines share
// the host link: the three position components come in first, one per
// stream, and the force computation starts on the caller's stream as soon as
// they have landed (it reads nothing else); v, psi1 and psi2 follow, one per
// side stream, while the forces are computed, and the kick waits for them.
// The updated positions and velocities go back on two streams at once, and
// the call returns when they have landed.  Pinned host memory makes the copies
// asynchronous DMA at the link's rate; pageable memory works too, through
// CUDA's own staging copies.
#include "cola_common.cuh"

namespace {

constexpr int kSide = 3;

struct SideStreams {
    cudaStream_t s[kSide] = {};
    cudaEvent_t ev[kSide] = {};
    cudaEvent_t start = nullptr, kicked = nullptr, in_done = nullptr;
    ~SideStreams() {
        for (int i = 0; i < kSide; ++i) {
            if (ev[i]) cudaEventDestroy(ev[i]);
            if (s[i]) cudaStreamDestroy(s[i]);
        }
        if (start) cudaEventDestroy(start);
        if (kicked) cudaEventDestroy(kicked);
        if (in_done) cudaEventDestroy(in_done);
    }
    bool create() {
        const unsigned f = cudaEventDisableTiming;
        for (int i = 0; i < kSide; ++i)
            if (cudaStreamCreateWithFlags(&s[i], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&ev[i], f) != cudaSuccess)
                return false;
        return cudaEventCreateWithFlags(&start, f) == cudaSuccess &&
               cudaEventCreateWithFlags(&kicked, f) == cudaSuccess &&
               cudaEventCreateWithFlags(&in_done, f) == cudaSuccess;
    }
    void drain() {
        for (int i = 0; i < kSide; ++i) cudaStreamSynchronize(s[i]);
    }
};

}  // namespace

extern "C" {

int cola_step_host(const cola_config* cfg, const cola_state* host, cola_state* dev, int32_t step, void* ws,
                   size_t ws_bytes, void* stream) {
    if (!cfg || !host || !dev) return COLA_EINVAL;
    size_t need = 0;
    int rc = cola_workspace_size(cfg, &need);
    if (rc) return rc;
    if (!ws) return COLA_EINVAL;
    if (ws_bytes < need) return COLA_EWORKSPACE;
    if (step < 0 || step >= cfg->n_steps) return COLA_EINVAL;
    float* const hs[4] = {host->d, host->v, host->psi1, host->psi2};
    float* const ds[4] = {dev->d, dev->v, dev->psi1, dev->psi2};
    for (int a = 0; a < 4; ++a)
        if (!hs[a] || !ds[a]) return COLA_EINVAL;
    const size_t np = (size_t)cfg->nq * cfg->nq * cfg->nq;
    const size_t comp = np * sizeof(float), bytes = 3 * comp;  // one component, one array
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    SideStreams side;
    if (!side.create()) return COLA_ECUDA;
    auto fail = [&]() {
        side.drain();
        return COLA_ECUDA;
    };
    // the side streams start after everything already queued on s
    if (cudaEventRecord(side.start, s) != cudaSuccess) return fail();
    for (int i = 0; i < kSide; ++i)
        if (cudaStreamWaitEvent(side.s[i], side.start, 0) != cudaSuccess) return fail();
    // positions: x on s, y and z on two side streams; s waits for both
    if (cudaMemcpyAsync(ds[0], hs[0], comp, cudaMemcpyHostToDevice, s) != cudaSuccess) return fail();
    for (int c = 1; c < 3; ++c) {
        cudaStream_t q = side.s[c - 1];
        if (cudaMemcpyAsync(ds[0] + c * np, hs[0] + c * np, comp, cudaMemcpyHostToDevice, q) != cudaSuccess ||
            cudaEventRecord(side.ev[c - 1], q) != cudaSuccess || cudaStreamWaitEvent(s, side.ev[c - 1], 0) != cudaSuccess)
            return fail();
    }
    // v, psi1, psi2: one per side stream, gathered on the last one for the kick
    for (int a = 1; a < 4; ++a)
        if (cudaMemcpyAsync(ds[a], hs[a], bytes, cudaMemcpyHostToDevice, side.s[a - 1]) != cudaSuccess) return fail();
    for (int i = 0; i < kSide - 1; ++i)
        if (cudaEventRecord(side.ev[i], side.s[i]) != cudaSuccess ||
            cudaStreamWaitEvent(side.s[kSide - 1], side.ev[i], 0) != cudaSuccess)
            return fail();
    if (cudaEventRecord(side.in_done, side.s[kSide - 1]) != cudaSuccess) return fail();
    if ((rc = cola::step_node(cfg, dev, step, ws, ws_bytes, s, side.in_done))) {
        side.drain();
        return rc;
    }
    // d back on s, v on a side stream that waits for the kick
    if (cudaEventRecord(side.kicked, s) != cudaSuccess || cudaStreamWaitEvent(side.s[0], side.kicked, 0) != cudaSuccess)
        return fail();
    if (cudaMemcpyAsync(hs[0], ds[0], bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(hs[1], ds[1], bytes, cudaMemcpyDeviceToHost, side.s[0]) != cudaSuccess)
        return fail();
    const bool ok = cudaStreamSynchronize(side.s[0]) == cudaSuccess;
    side.drain();
    return ok && cudaStreamSynchronize(s) == cudaSuccess ? COLA_OK : COLA_ECUDA;
}

}  // extern "C"
