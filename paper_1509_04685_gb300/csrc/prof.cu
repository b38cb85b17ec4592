// Per-kernel timing with CUDA events recorded on the launching stream around
// every launch of the library while profiling is on (the tracing subsystem).
#include <vector>

#include "cola_common.cuh"

namespace cola {

namespace {
struct Rec {
    int id;
    cudaEvent_t start, stop;
};
bool g_on = false;
std::vector<Rec> g_recs;
size_t g_used = 0;
const char* kNames[kNumKernelIds] = {"deposit",     "fft_z_r2c_fix", "fft_z_r2c", "fft_y_fwd",  "fft_x_fwd",
                                     "fft_x_green", "fft_y_inv",     "fft_x_inv", "fft_z_c2r",  "gather_kick_drift",
                                     "gather",      "fix_to_delta",  "pk_shells", "pk_reduce",  "ic",
                                     "setup",       "learned",       "bins",      "dep_r2c",    "c2r_gather",
                                     "kick_drift"};
}  // namespace

ProfScope::ProfScope(int id, cudaStream_t s) : rec_(-1), s_(s) {
    if (!g_on || id < 0 || g_used >= g_recs.size()) return;
    rec_ = (int)g_used++;
    g_recs[rec_].id = id;
    cudaEventRecord(g_recs[rec_].start, s);
}

ProfScope::~ProfScope() {
    if (rec_ >= 0) cudaEventRecord(g_recs[rec_].stop, s_);
}

}  // namespace cola

using namespace cola;

extern "C" {

int cola_profile_start(int32_t max_records) {
    if (max_records < 1) return COLA_EINVAL;
    for (size_t i = g_recs.size(); i < (size_t)max_records; ++i) {
        Rec r{0, nullptr, nullptr};
        if (cudaEventCreate(&r.start) != cudaSuccess || cudaEventCreate(&r.stop) != cudaSuccess) return COLA_ECUDA;
        g_recs.push_back(r);
    }
    g_used = 0;
    g_on = true;
    return COLA_OK;
}

int cola_profile_stop(double* ms, int64_t* launches, int32_t nkernels) {
    g_on = false;
    if (!ms || !launches || nkernels < kNumKernelIds) return COLA_EINVAL;
    for (int i = 0; i < nkernels; ++i) {
        ms[i] = 0.0;
        launches[i] = 0;
    }
    for (size_t i = 0; i < g_used; ++i) {
        float t = 0.f;
        if (cudaEventSynchronize(g_recs[i].stop) != cudaSuccess) return COLA_ECUDA;
        if (cudaEventElapsedTime(&t, g_recs[i].start, g_recs[i].stop) != cudaSuccess) return COLA_ECUDA;
        ms[g_recs[i].id] += t;
        launches[g_recs[i].id] += 1;
    }
    g_used = 0;
    return COLA_OK;
}

const char* cola_kernel_name(int32_t id) { return (id >= 0 && id < kNumKernelIds) ? kNames[id] : "?"; }

int32_t cola_num_kernel_ids(void) { return kNumKernelIds; }

}  // extern "C"
