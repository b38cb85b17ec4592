// cola_step_host: one PM step (Sec. 2.2, Eqs. 1-2, exactly as cola_step) of a
// particle state held in host memory.  The positions go to the device first
// on the caller's stream, where the force computation starts at once (it
// reads nothing else); v, psi1 and psi2 follow on a second stream meanwhile,
// and the fused gather + kick + drift waits for them.  The updated positions
// and velocities then come back on the caller's stream, and the call returns
// once they have landed.  Pinned host memory makes the copies asynchronous DMA
// at the link's rate; pageable memory works too, through CUDA's own staging
// copies.
#include "cola_common.cuh"

namespace {

struct SideStream {
    cudaStream_t s = nullptr;
    cudaEvent_t start = nullptr, done = nullptr;
    ~SideStream() {
        if (done) cudaEventDestroy(done);
        if (start) cudaEventDestroy(start);
        if (s) cudaStreamDestroy(s);
    }
    bool create() {
        return cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
               cudaEventCreateWithFlags(&start, cudaEventDisableTiming) == cudaSuccess &&
               cudaEventCreateWithFlags(&done, cudaEventDisableTiming) == cudaSuccess;
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
    const size_t bytes = (size_t)3 * cfg->nq * cfg->nq * cfg->nq * sizeof(float);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    SideStream side;
    if (!side.create()) return COLA_ECUDA;
    // the side stream starts after everything already queued on s
    if (cudaEventRecord(side.start, s) != cudaSuccess || cudaStreamWaitEvent(side.s, side.start, 0) != cudaSuccess)
        return COLA_ECUDA;
    if (cudaMemcpyAsync(ds[0], hs[0], bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return COLA_ECUDA;
    for (int a = 1; a < 4; ++a)
        if (cudaMemcpyAsync(ds[a], hs[a], bytes, cudaMemcpyHostToDevice, side.s) != cudaSuccess) return COLA_ECUDA;
    if (cudaEventRecord(side.done, side.s) != cudaSuccess) return COLA_ECUDA;
    if ((rc = cola::step_node(cfg, dev, step, ws, ws_bytes, s, side.done))) {
        cudaStreamSynchronize(side.s);
        return rc;
    }
    for (int a = 0; a < 2; ++a)
        if (cudaMemcpyAsync(hs[a], ds[a], bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return COLA_ECUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? COLA_OK : COLA_ECUDA;
}

}  // extern "C"
