// Ensembles of independent realisations (the paper's motive for cheap runs:
// many mocks, e.g. the 48 realisations of Sec. 6) advanced by one CUDA-graph
// launch, and the FFT tile autotuner.
//
// The graph is captured once: every member's 2LPT set-up and PM steps are
// recorded on one of several streams forked from the capture stream, members
// assigned largest-cost-first to the least loaded stream so that small
// meshes run side by side and fill the GPU.  Launching the graph replays the
// whole ensemble with a single host call.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "fft_static.cuh"

struct cola_ensemble {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int n = 0;
};

namespace cola {

// measured best column width per line length (0: not tuned)
int g_tile_choice[kMaxFft + 1] = {0};

}  // namespace cola

using namespace cola;

extern "C" {

int cola_ensemble_create(int32_t n, const cola_config* cfgs, const uint64_t* seeds, const cola_state* states,
                         void* const* ws, const size_t* ws_bytes, int32_t nstreams, int32_t step_from,
                         int32_t step_to, cola_ensemble** out) {
    if (n < 1 || !cfgs || !states || !ws || !ws_bytes || !out || nstreams < 1 || nstreams > 64) return COLA_EINVAL;
    if (step_from < 0 || step_to < step_from) return COLA_EINVAL;
    for (int i = 0; i < n; ++i) {
        size_t need = 0;
        int rc = cola_workspace_size(&cfgs[i], &need);
        if (rc) return rc;
        if (ws_bytes[i] < need) return COLA_EWORKSPACE;
        if (step_to > cfgs[i].n_steps) return COLA_EINVAL;
        if (step_from == 0 && !seeds) return COLA_EINVAL;
    }
    // cost ~ mesh cells * log cells per step, largest first to the least loaded stream
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    auto cost = [&](int i) {
        const double c = (double)cfgs[i].ng * cfgs[i].ng * cfgs[i].ng;
        return c * std::log2(c) + 40.0 * cfgs[i].nq * cfgs[i].nq * cfgs[i].nq;
    };
    std::sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
    std::vector<double> load(nstreams, 0.0);
    std::vector<std::vector<int>> lanes(nstreams);
    for (int i : order) {
        const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[l] += cost(i);
        lanes[l].push_back(i);
    }
    cudaStream_t origin = nullptr;
    std::vector<cudaStream_t> st(nstreams, nullptr);
    std::vector<cudaEvent_t> ev(nstreams + 1, nullptr);
    int rc = COLA_OK;
    auto fail = [&](int code) {
        rc = code;
        return code;
    };
    if (cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking) != cudaSuccess) return COLA_ECUDA;
    for (int l = 0; l < nstreams; ++l)
        if (cudaStreamCreateWithFlags(&st[l], cudaStreamNonBlocking) != cudaSuccess) fail(COLA_ECUDA);
    for (auto& e : ev)
        if (!rc && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) fail(COLA_ECUDA);
    cola_ensemble* E = nullptr;
    if (!rc && cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess) fail(COLA_ECUDA);
    if (!rc) {
        cudaEventRecord(ev[nstreams], origin);
        for (int l = 0; l < nstreams && !rc; ++l) {
            cudaStreamWaitEvent(st[l], ev[nstreams], 0);
            for (int i : lanes[l]) {
                cola_state s = states[i];
                // a member's own error code is passed on
                const int r = step_from == 0 ? cola_ic_2lpt(&cfgs[i], seeds[i], &s, ws[i], ws_bytes[i], st[l])
                                             : cola_init(&cfgs[i], ws[i], ws_bytes[i], st[l]);
                if (r) {
                    fail(r);
                    break;
                }
                for (int j = step_from; j < step_to && !rc; ++j)
                    if (const int rs = cola_step(&cfgs[i], &s, j, ws[i], ws_bytes[i], st[l])) fail(rs);
            }
            cudaEventRecord(ev[l], st[l]);
            cudaStreamWaitEvent(origin, ev[l], 0);
        }
        cudaGraph_t graph = nullptr;
        if (cudaStreamEndCapture(origin, &graph) != cudaSuccess) fail(COLA_ECUDA);
        if (!rc) {
            E = new cola_ensemble;
            E->graph = graph;
            E->n = n;
            if (cudaGraphInstantiate(&E->exec, graph, 0) != cudaSuccess) fail(COLA_ECUDA);
        } else if (graph) {
            cudaGraphDestroy(graph);
        }
    }
    for (auto e : ev)
        if (e) cudaEventDestroy(e);
    for (auto s : st)
        if (s) cudaStreamDestroy(s);
    cudaStreamDestroy(origin);
    if (rc) {
        if (E) {
            if (E->exec) cudaGraphExecDestroy(E->exec);
            if (E->graph) cudaGraphDestroy(E->graph);
            delete E;
        }
        cudaGetLastError();
        return rc;
    }
    *out = E;
    return COLA_OK;
}

int cola_ensemble_launch(cola_ensemble* e, void* stream) {
    if (!e || !e->exec) return COLA_EINVAL;
    g_launches++;
    return cudaGraphLaunch(e->exec, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess ? COLA_OK : COLA_ECUDA;
}

void cola_ensemble_destroy(cola_ensemble* e) {
    if (!e) return;
    if (e->exec) cudaGraphExecDestroy(e->exec);
    if (e->graph) cudaGraphDestroy(e->graph);
    delete e;
}

int cola_fft_set_tile(int32_t n, int32_t B) {
    if (n < 2 || n > kMaxFft) return COLA_EINVAL;
    if (B != 0 && B != 2 && B != 4 && B != 8 && B != 16) return COLA_EINVAL;
    if (B && !static_tile_ok(n, B) && (size_t)(3 * spad(n) * B + n) * 8 > 220 * 1024) return COLA_EINVAL;
    g_tile_choice[n] = B;
    return COLA_OK;
}

int cola_particle_set_traversal(int32_t edge, int32_t brick_k) { return set_particle_traversal(edge, brick_k); }

// Time the y pass of an n^3 mesh for every admissible column width and keep
// the fastest for this n (used by every later strided pass of that size).
int cola_fft_autotune(int32_t n, float* mesh, void* ws, size_t ws_bytes, void* stream, int32_t* best) {
    if (n < 4 || n > kMaxFft || (n & 1) || !mesh || !ws || ws_bytes < kHdrBytes) return COLA_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    float2* tw = twiddle_ptr(ws, kTwScratch);
    int rc = launch_twiddles(tw, n, s);
    if (rc) return rc;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return COLA_ECUDA;
    float best_ms = 1e30f;
    int best_b = 0;
    for (int B : {2, 4, 8, 16}) {
        // the specialised passes (two tile buffers) or the runtime ones (three)
        // must fit in shared memory
        if (!static_tile_ok(n, B) && (size_t)(3 * spad(n) * B + n) * 8 > 220 * 1024) continue;
        g_tile_choice[n] = B;
        float ms = 0.f;
        for (int rep = 0; rep < 3 && !rc; ++rep) {
            cudaEventRecord(e0, s);
            rc = fft_strided(reinterpret_cast<float2*>(mesh), n, 1, -1, tw, s);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0) ms += t;
        }
        if (rc) break;
        if (ms < best_ms) {
            best_ms = ms;
            best_b = B;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    g_tile_choice[n] = rc ? 0 : best_b;
    if (best) *best = best_b;
    return rc;
}

}  // extern "C"
