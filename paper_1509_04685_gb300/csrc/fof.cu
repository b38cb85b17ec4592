// Friends-of-friends halo finder (Sec. 2.1: FoF, linking length b = 0.2 mean
// inter-particle spacings; Sec. 2.5: halos of more than 100
// particles, Warren et al. 2006 masses M = m_p N (1 - N^-0.6)) and the halo
// mass function.
//
// Positions are taken in units of the mean spacing, u = q + d nq / L wrapped
// into [0, nq), in FP32 with every operation rounded once (the __f*_rn
// intrinsics are never contracted), so the friendship test r^2 <= b^2 gives
// the same answer bit for bit wherever it is evaluated.
//
// Cell list: one cell per mean spacing (nq^3 cells, cell = floor(u); b < 1/2
// keeps every friend in the 27 cells around a particle), built by counting
// sort: a histogram, an exclusive scan, and a scatter of (u, p) into cell
// order.
//
// Linking: one thread per particle, in cell order, visits the neighbour cells
// its position can reach within b and tests their particles; a pair is taken
// by the thread with the smaller sorted slot.  Friends are united in a
// lock-free union-find whose roots only ever hook under smaller indices, so
// every tree's root is its smallest member whatever order the unions land in:
// the labels are deterministic.
#include "cola_common.cuh"

namespace cola {
namespace {

constexpr int kUnionCap = 1 << 20;  // default bound on the retries of one find or union
int g_union_cap = kUnionCap;        // the bound in use (cola_fof_set_retry_cap)
constexpr double kRhoCrit = 2.77536627e11;  // 3 H0^2 / (8 pi G) in h^2 Msun Mpc^-3

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct FofLayout {
    size_t status, sorted, start, cursor, sums, total;
};

FofLayout fof_layout(long long np) {
    FofLayout L;
    size_t o = 0;
    L.status = o;
    o += 256;
    L.sorted = o;
    o = align256(o + (size_t)np * sizeof(float4));
    L.start = o;
    o = align256(o + (size_t)(np + 1) * sizeof(int));
    L.cursor = o;
    o = align256(o + (size_t)np * sizeof(int));
    L.sums = o;
    o = align256(o + scan_sums_bytes(np + 1));
    L.total = o;
    return L;
}

template <class T>
T* at(void* ws, size_t off) {
    return reinterpret_cast<T*>(static_cast<char*>(ws) + off);
}

// position along one axis in units of the mean spacing, wrapped into [0, nq)
__device__ __forceinline__ float wrap_pos(float q, float d, float inv, float nqf) {
    float u = __fadd_rn(q, __fmul_rn(d, inv));
    u = __fsub_rn(u, __fmul_rn(nqf, floorf(__fdiv_rn(u, nqf))));
    if (u < 0.f) u = __fadd_rn(u, nqf);
    if (u >= nqf) u = __fsub_rn(u, nqf);
    return u;
}

// u of particle p and its cell; false (cell 0, u NaN) for non-finite input
__device__ __forceinline__ bool particle_pos(const float* __restrict__ d, long long np, int nq, float inv, long long p,
                                             float u[3], int* cell) {
    const unsigned nqu = (unsigned)nq, pu = (unsigned)p;
    const unsigned q[3] = {pu / (nqu * nqu), (pu / nqu) % nqu, pu % nqu};
    const float nqf = (float)nq;
    bool ok = true;
    int c = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        u[a] = wrap_pos((float)q[a], d[a * np + p], inv, nqf);
        ok = ok && (u[a] >= 0.f && u[a] < nqf);  // false for NaN
        int ca = (int)u[a];
        if (ca > nq - 1) ca = nq - 1;
        c = c * nq + ca;
    }
    if (!ok) {
        u[0] = u[1] = u[2] = __int_as_float(0x7fc00000);
        c = 0;
    }
    *cell = c;
    return ok;
}

__global__ void k_fof_count(const float* __restrict__ d, long long np, int nq, float inv, int* count, int* status) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    float u[3];
    int c;
    if (!particle_pos(d, np, nq, inv, p, u, &c)) set_status(status, COLA_ENONFINITE);
    atomicAdd(count + c, 1);
}

__global__ void k_fof_scatter(const float* __restrict__ d, long long np, int nq, float inv, int* cursor,
                              float4* sorted) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    float u[3];
    int c;
    particle_pos(d, np, nq, inv, p, u, &c);
    const int slot = atomicAdd(cursor + c, 1);
    sorted[slot] = make_float4(u[0], u[1], u[2], __int_as_float((int)p));
}


// ---------------------------------------------------------------------------
// union-find over particle indices; parent[x] <= x always holds
// ---------------------------------------------------------------------------
__device__ __forceinline__ int fof_find(int* parent, int x, int* status, int cap) {
    for (int it = 0; it < cap; ++it) {
        const int px = __ldcg(parent + x);
        if (px == x) return x;
        const int gp = __ldcg(parent + px);
        if (gp != px) parent[x] = gp;  // path halving: gp is an ancestor of x, so gp <= px
        x = gp;
    }
    set_status(status, COLA_ETIMEOUT);
    return x;
}

__device__ __forceinline__ void fof_unite(int* parent, int a, int b, int* status, int cap) {
    for (int it = 0; it < cap; ++it) {
        a = fof_find(parent, a, status, cap);
        b = fof_find(parent, b, status, cap);
        if (a == b) return;
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        if (atomicCAS(parent + b, b, a) == b) return;  // the larger root hooks under the smaller
    }
    set_status(status, COLA_ETIMEOUT);
}

__device__ __forceinline__ float min_image(float x, float nqf, float half) {
    if (x > half) x = __fsub_rn(x, nqf);
    if (x < -half) x = __fadd_rn(x, nqf);
    return x;
}

__global__ void k_fof_init(int* parent, long long np) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < np) parent[p] = (int)p;
}

// A friend pair (k, j), k < j in sorted order, is taken by thread k.  Thread
// k's candidate cells are the neighbour cells its position reaches within
// `reach`; any superset also works (the distance test decides).  When all 32
// lanes of a warp lie in one cell (the dense regions, where the work is), the
// warp walks the union of its lanes' cells in step: every lane reads the same
// candidate (one broadcast load) and the loop bounds are the same for all.
__device__ __forceinline__ int wrap_cell(int c, int nq) { return c < 0 ? c + nq : (c >= nq ? c - nq : c); }

__device__ __forceinline__ void link_candidate(const float4& a, const float4& o, float nqf, float half, float b2,
                                               int* parent, int* status, int cap) {
    const float dx = min_image(__fsub_rn(a.x, o.x), nqf, half);
    const float dy = min_image(__fsub_rn(a.y, o.y), nqf, half);
    const float dz = min_image(__fsub_rn(a.z, o.z), nqf, half);
    const float r2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    if (r2 <= b2) fof_unite(parent, __float_as_int(a.w), __float_as_int(o.w), status, cap);
}

__global__ void k_fof_link(const float4* __restrict__ sorted, const int* __restrict__ start, long long np, int nq,
                           float b2, float reach, int* parent, int* status, int cap) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = k < np;
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
    if (active) a = sorted[k];
    const bool finite = active && a.x == a.x && a.y == a.y && a.z == a.z;  // non-finite input links to nothing
    const float nqf = (float)nq, half = (float)(nq / 2.0);
    const float pos[3] = {a.x, a.y, a.z};
    int c[3], lo[3], hi[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        c[e] = finite ? (int)pos[e] : 0;
        if (c[e] > nq - 1) c[e] = nq - 1;
        const float f = pos[e] - (float)c[e];  // exact
        lo[e] = f <= reach ? -1 : 0;
        hi[e] = 1.f - f <= reach ? 1 : 0;
    }
    const int cid = finite ? (c[0] * nq + c[1]) * nq + c[2] : -1;
    const unsigned full = 0xffffffffu;
    const int cid0 = __shfl_sync(full, cid, 0);
    if (__all_sync(full, cid == cid0 && cid >= 0)) {
        unsigned mine = 0;  // this lane's cells as bits o = (ox + 1) 9 + (oy + 1) 3 + (oz + 1)
        for (int ox = lo[0]; ox <= hi[0]; ++ox)
            for (int oy = lo[1]; oy <= hi[1]; ++oy)
                for (int oz = lo[2]; oz <= hi[2]; ++oz) mine |= 1u << ((ox + 1) * 9 + (oy + 1) * 3 + (oz + 1));
        const unsigned cells = __reduce_or_sync(full, mine);
        for (int o = 0; o < 27; ++o) {
            if (!((cells >> o) & 1u)) continue;
            const int cell = (wrap_cell(c[0] + o / 9 - 1, nq) * nq + wrap_cell(c[1] + (o / 3) % 3 - 1, nq)) * nq +
                             wrap_cell(c[2] + o % 3 - 1, nq);
            const int j1 = start[cell + 1];
            for (int j = start[cell]; j < j1; ++j) {
                const float4 q = sorted[j];
                if (j > k) link_candidate(a, q, nqf, half, b2, parent, status, cap);
            }
        }
        return;
    }
    if (!finite) return;
    for (int ox = lo[0]; ox <= hi[0]; ++ox) {
        const int cx = wrap_cell(c[0] + ox, nq);
        for (int oy = lo[1]; oy <= hi[1]; ++oy) {
            const int cy = wrap_cell(c[1] + oy, nq);
            for (int oz = lo[2]; oz <= hi[2]; ++oz) {
                const int cell = (cx * nq + cy) * nq + wrap_cell(c[2] + oz, nq);
                const int j1 = start[cell + 1];
                for (int j = start[cell] > k + 1 ? start[cell] : (int)k + 1; j < j1; ++j)
                    link_candidate(a, sorted[j], nqf, half, b2, parent, status, cap);
            }
        }
    }
}

// every label becomes its root, the smallest member of its group
__global__ void k_fof_flatten(int* parent, long long np, int* status, int cap) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    int x = (int)p;
    for (int it = 0; it < cap; ++it) {
        const int px = __ldcg(parent + x);
        if (px == x) {
            parent[p] = x;
            return;
        }
        x = px;
    }
    set_status(status, COLA_ETIMEOUT);
}

__global__ void k_fof_sizes(const int* __restrict__ group, long long np, int* size) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < np) atomicAdd(size + group[p], 1);
}

__global__ void k_fof_flags(const int* __restrict__ group, const int* __restrict__ size, long long np, int nmin,
                            int* flag) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < np) flag[p] = (group[p] == (int)p && size[p] >= nmin) ? 1 : 0;
}

// off: exclusive scan of the flags (np + 1 entries, off[np] = halo count)
__global__ void k_fof_emit(const int* __restrict__ off, const int* __restrict__ size, long long np, int* halo_root,
                           int* halo_size, long long* n_halos) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0) *n_halos = off[np];
    if (p >= np) return;
    const int o = off[p];
    if (off[p + 1] != o) {
        halo_root[o] = (int)p;
        halo_size[o] = size[p];
    }
}

__global__ void k_mass_function(const int* __restrict__ halo_size, const long long* __restrict__ n_halos,
                                long long max_halos, double m_p, double lo, double dlog, int nbins,
                                unsigned long long* counts) {
    const long long n = min(*n_halos, max_halos);
    for (long long h = (long long)blockIdx.x * blockDim.x + threadIdx.x; h < n; h += (long long)gridDim.x * blockDim.x) {
        const double N = (double)halo_size[h];
        const double lm = log10(m_p * N * (1.0 - pow(N, -0.6)));
        const double t = floor((lm - lo) / dlog);
        if (t >= 0.0 && t < (double)nbins) atomicAdd(counts + (int)t, 1ull);
    }
}

unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

int check_fof_args(const cola_config* cfg, long long* np) {
    size_t ignored = 0;
    if (!cfg) return COLA_EINVAL;
    if (int rc = cola_workspace_size(cfg, &ignored)) return rc;
    const long long n = (long long)cfg->nq * cfg->nq * cfg->nq;
    if (n + 1 > 0x7fffffffll) return COLA_EUNSUPPORTED_SIZE;  // int32 particle indices and scans
    *np = n;
    return COLA_OK;
}

int read_status(const int* dev_status, cudaStream_t s) {
    int h = 0;
    if (cudaMemcpyAsync(&h, dev_status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return COLA_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return COLA_ECUDA;
    return h;
}

}  // namespace
}  // namespace cola

extern "C" {

int cola_fof_set_retry_cap(int32_t cap) {
    if (cap < 0 || cap > (1 << 30)) return COLA_EINVAL;
    cola::g_union_cap = cap ? cap : cola::kUnionCap;
    return COLA_OK;
}

int cola_fof_workspace_size(const cola_config* cfg, size_t* bytes) {
    long long np = 0;
    if (!bytes) return COLA_EINVAL;
    if (int rc = cola::check_fof_args(cfg, &np)) return rc;
    *bytes = cola::fof_layout(np).total;
    return COLA_OK;
}

int cola_fof(const cola_config* cfg, const cola_state* st, double b, int32_t* group, void* fws, size_t fws_bytes,
             void* stream) {
    using namespace cola;
    long long np = 0;
    if (int rc = check_fof_args(cfg, &np)) return rc;
    if (!st || !st->d || !group || !fws || !(b > 0.0 && b < 0.5)) return COLA_EINVAL;
    const FofLayout L = fof_layout(np);
    if (fws_bytes < L.total) return COLA_EWORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int* status = at<int>(fws, L.status);
    int* start = at<int>(fws, L.start);
    int* cursor = at<int>(fws, L.cursor);
    float4* sorted = at<float4>(fws, L.sorted);
    const float inv = (float)((double)cfg->nq / cfg->box);
    const int T = 256;
    const unsigned nb = blocks_for(np, T);
    if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess ||
        cudaMemsetAsync(start, 0, (size_t)(np + 1) * sizeof(int), s) != cudaSuccess)
        return COLA_ECUDA;
    k_fof_count<<<nb, T, 0, s>>>(st->d, np, cfg->nq, inv, start, status);
    if (int rc = check_launch()) return rc;
    if (int rc = exclusive_scan(start, np, at<int>(fws, L.sums), s)) return rc;
    if (cudaMemcpyAsync(cursor, start, (size_t)np * sizeof(int), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return COLA_ECUDA;
    k_fof_scatter<<<nb, T, 0, s>>>(st->d, np, cfg->nq, inv, cursor, sorted);
    k_fof_init<<<nb, T, 0, s>>>(group, np);
    // cells wider than the linking length by a margin far above FP32 rounding
    k_fof_link<<<nb, T, 0, s>>>(sorted, start, np, cfg->nq, (float)(b * b), (float)b + 0.01f, group, status,
                                  g_union_cap);
    k_fof_flatten<<<nb, T, 0, s>>>(group, np, status, g_union_cap);
    if (int rc = check_launch()) return rc;
    return read_status(status, s);
}

int cola_fof_halos(const cola_config* cfg, const int32_t* group, int32_t min_members, int32_t* halo_root,
                   int32_t* halo_size, int64_t* n_halos, void* fws, size_t fws_bytes, void* stream) {
    using namespace cola;
    long long np = 0;
    if (int rc = check_fof_args(cfg, &np)) return rc;
    if (!group || !halo_root || !halo_size || !n_halos || !fws || min_members < 1) return COLA_EINVAL;
    const FofLayout L = fof_layout(np);
    if (fws_bytes < L.total) return COLA_EWORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int* size = at<int>(fws, L.cursor);
    int* off = at<int>(fws, L.start);
    const int T = 256;
    const unsigned nb = blocks_for(np, T);
    if (cudaMemsetAsync(size, 0, (size_t)np * sizeof(int), s) != cudaSuccess) return COLA_ECUDA;
    k_fof_sizes<<<nb, T, 0, s>>>(group, np, size);
    k_fof_flags<<<nb, T, 0, s>>>(group, size, np, min_members, off);
    if (int rc = check_launch()) return rc;
    if (int rc = exclusive_scan(off, np, at<int>(fws, L.sums), s)) return rc;
    k_fof_emit<<<nb, T, 0, s>>>(off, size, np, halo_root, halo_size, reinterpret_cast<long long*>(n_halos));
    return check_launch();
}

int cola_mass_function(const cola_config* cfg, const int32_t* halo_size, const int64_t* n_halos, int64_t max_halos,
                       double log10m_lo, double dlog10m, int32_t nbins, int64_t* counts, void* stream) {
    using namespace cola;
    long long np = 0;
    if (int rc = check_fof_args(cfg, &np)) return rc;
    if (!halo_size || !n_halos || !counts || max_halos < 0 || nbins < 1 || !(dlog10m > 0.0)) return COLA_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(counts, 0, (size_t)nbins * sizeof(int64_t), s) != cudaSuccess) return COLA_ECUDA;
    if (max_halos == 0) return COLA_OK;
    const double m_p = kRhoCrit * cfg->cosmo.omega_m * std::pow(cfg->box / cfg->nq, 3);
    const int T = 256;
    long long blocks = (max_halos + T - 1) / T;
    if (blocks > 4096) blocks = 4096;
    k_mass_function<<<(unsigned)blocks, T, 0, s>>>(halo_size, reinterpret_cast<const long long*>(n_halos), max_halos,
                                                   m_p, log10m_lo, dlog10m, nbins,
                                                   reinterpret_cast<unsigned long long*>(counts));
    return check_launch();
}

}  // extern "C"
