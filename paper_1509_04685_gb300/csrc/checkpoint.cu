// Checkpoint and resume of a COLA run (not in the paper, whose runs restart
// from the initial-condition seed).  A checkpoint is one host buffer: a fixed
// header that identifies the run and the next time node, then the four
// particle arrays d, v, psi1, psi2 as they are on the device.  The workspace
// needs no saving: cola_init rebuilds its tables and twiddles bit for bit from
// the configuration, and the fixed-point deposit mesh is all-zero between
// calls, so a run resumed from a checkpoint continues bit-identically.
#include <cstring>

#include "cola_common.cuh"

namespace {

constexpr char kMagic[8] = {'C', 'O', 'L', 'A', 'C', 'K', 'P', '1'};
constexpr uint32_t kVersion = 1;
constexpr size_t kHeaderBytes = 256;

// Header fields in a fixed order (little-endian as the host writes them; the
// buffer is meant to be read back on a machine of the same byte order).
struct CkptHeader {
    char magic[8];
    uint32_t version;
    int32_t node;  // next time node to run
    int32_t nq, ng, n_steps, sampling;
    uint32_t flags, pad;
    double box, a_init, a_final, sampling_p;
    double omega_m, omega_l, omega_b, h, sigma8, n_s, t_cmb;
    uint64_t array_bytes;  // bytes of each of the four arrays
};
static_assert(sizeof(CkptHeader) <= kHeaderBytes, "header must fit its slot");

size_t array_bytes(const cola_config* cfg) { return (size_t)3 * cfg->nq * cfg->nq * cfg->nq * sizeof(float); }

CkptHeader header_of(const cola_config* cfg, int32_t node) {
    CkptHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kMagic, sizeof(kMagic));
    h.version = kVersion;
    h.node = node;
    h.nq = cfg->nq;
    h.ng = cfg->ng;
    h.n_steps = cfg->n_steps;
    h.sampling = cfg->sampling;
    h.flags = cfg->flags;
    h.box = cfg->box;
    h.a_init = cfg->a_init;
    h.a_final = cfg->a_final;
    h.sampling_p = cfg->sampling_p;
    h.omega_m = cfg->cosmo.omega_m;
    h.omega_l = cfg->cosmo.omega_l;
    h.omega_b = cfg->cosmo.omega_b;
    h.h = cfg->cosmo.h;
    h.sigma8 = cfg->cosmo.sigma8;
    h.n_s = cfg->cosmo.n_s;
    h.t_cmb = cfg->cosmo.t_cmb;
    h.array_bytes = array_bytes(cfg);
    return h;
}

bool cfg_ok(const cola_config* cfg) {
    size_t ws = 0;
    return cfg && cola_workspace_size(cfg, &ws) == COLA_OK;
}

}  // namespace

extern "C" {

int cola_checkpoint_bytes(const cola_config* cfg, size_t* bytes) {
    if (!bytes || !cfg_ok(cfg)) return COLA_EINVAL;
    *bytes = kHeaderBytes + 4 * array_bytes(cfg);
    return COLA_OK;
}

int cola_checkpoint_save(const cola_config* cfg, const cola_state* st, int32_t node, void* host, size_t host_bytes,
                         void* stream) {
    if (!cfg_ok(cfg)) return COLA_EINVAL;
    if (!st || !st->d || !st->v || !st->psi1 || !st->psi2 || !host) return COLA_EINVAL;
    if (node < 0 || node >= cfg->n_steps) return COLA_EINVAL;
    if (host_bytes < kHeaderBytes + 4 * array_bytes(cfg)) return COLA_EINVAL;
    const CkptHeader h = header_of(cfg, node);
    unsigned char* out = static_cast<unsigned char*>(host);
    std::memset(out, 0, kHeaderBytes);
    std::memcpy(out, &h, sizeof(h));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t n = array_bytes(cfg);
    const float* src[4] = {st->d, st->v, st->psi1, st->psi2};
    for (int a = 0; a < 4; ++a)
        if (cudaMemcpyAsync(out + kHeaderBytes + a * n, src[a], n, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return COLA_ECUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? COLA_OK : COLA_ECUDA;
}

int cola_checkpoint_load(const cola_config* cfg, const void* host, size_t host_bytes, cola_state* st, int32_t* node,
                         void* stream) {
    if (!cfg_ok(cfg)) return COLA_EINVAL;
    if (!host || !st || !st->d || !st->v || !st->psi1 || !st->psi2 || !node) return COLA_EINVAL;
    if (host_bytes < kHeaderBytes + 4 * array_bytes(cfg)) return COLA_EINVAL;
    CkptHeader got;
    std::memcpy(&got, host, sizeof(got));
    // the stored run must be this configuration's, field for field
    CkptHeader want = header_of(cfg, got.node);
    if (std::memcmp(&got, &want, sizeof(got)) != 0) return COLA_EINVAL;
    if (got.node < 0 || got.node >= cfg->n_steps) return COLA_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t n = array_bytes(cfg);
    const unsigned char* in = static_cast<const unsigned char*>(host);
    float* dst[4] = {st->d, st->v, st->psi1, st->psi2};
    for (int a = 0; a < 4; ++a)
        if (cudaMemcpyAsync(dst[a], in + kHeaderBytes + a * n, n, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return COLA_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return COLA_ECUDA;
    *node = got.node;
    return COLA_OK;
}

}  // extern "C"
