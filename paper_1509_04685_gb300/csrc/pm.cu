// Particle side of the PM step (Sec. 2.2): the row binning of the particles,
// the CIC deposit onto a global fixed-point mesh (outputs and the density
// call), the CIC gather, and the COLA kick + drift in the frame comoving with
// the 2LPT trajectories (Eqs. 1-2), either fused with a gather from the force
// mesh or from the per-particle partial sums the fused c2r pass leaves.
// Particle positions, CIC corners and deposit weights: particles.cuh.
#include "particles.cuh"

namespace cola {

// --------------------------------------------------------------------------
// Traversal order of the particle kernels.  A block of kTravThreads threads
// takes a brick of I (i) x J (j) x K (k) lattice sites, K a power of two in
// 8..256, J = min(8, 256 / K), I = 256 / (J K) (a warp covers consecutive k, so
// every SoA read is whole 32-byte sectors); bricks are grouped into cubic
// tiles of E^3 sites (E a power of two), bricks in raster order inside a tile,
// tiles in raster order over the lattice (k fastest).  The launch grid is
// (tiles along k x bricks per tile, tiles along j, tiles along i), so blocks
// are dispatched in that order and each thread finds its site with shifts
// alone; the padding sites of ragged tiles or bricks exit at once.  Every
// site is visited exactly once for any K and E: only the order of the memory
// traffic changes, never a result (the gather is per particle and the deposit
// adds integers).  Once particles have moved several cells, Lagrangian raster
// order has the blocks in flight read mesh planes from several i-slabs at
// once, far more than L2 holds; in tiles the blocks in flight touch a compact
// region of the mesh and only the tile faces are fetched twice.
// --------------------------------------------------------------------------
constexpr int kTravThreads = 256;
constexpr int kTileEdgeDefault = 256;
constexpr int kBrickKDefault = 16;
static int g_tile_edge = kTileEdgeDefault;
static int g_brick_k = kBrickKDefault;

struct Trav {
    int nq;
    int lb;            // log2 of the bricks per tile
    int lt[3];         // log2 of the tile extent in bricks along i, j, k
    int lbr[3];        // log2 of the brick extent in sites along i, j, k
    unsigned grid[3];  // launch grid (x, y, z)
};

static int ilog2(long long x) {
    int l = 0;
    while ((1ll << (l + 1)) <= x) ++l;
    return l;
}

// The tile edge actually used for an nq^3 lattice: the largest power of two
// not above the requested edge (and not below the brick) whose padded lattice
// is at most 5% larger than nq^3; else the one that pads least.
static int trav_edge(int nq, int want, int minE) {
    int best = 0;
    double best_pad = 1e300;
    for (int E = want; E >= minE; E >>= 1) {
        const double n = (double)((nq + E - 1) / E) * E / nq;
        const double pad = n * n * n;
        if (pad <= 1.05) return E;
        if (pad < best_pad) {
            best_pad = pad;
            best = E;
        }
    }
    return best;
}

static Trav make_trav(int nq) {
    const int K = g_brick_k, J = kTravThreads / K < 8 ? kTravThreads / K : 8, I = kTravThreads / (J * K);
    const int minE = K > 32 ? K : 32;
    int want = g_tile_edge > minE ? g_tile_edge : minE;
    while (want > minE && want / 2 >= nq) want >>= 1;  // no tile larger than the lattice needs
    const int E = trav_edge(nq, want, minE);
    Trav t;
    t.nq = nq;
    t.lbr[0] = ilog2(I);
    t.lbr[1] = ilog2(J);
    t.lbr[2] = ilog2(K);
    for (int a = 0; a < 3; ++a) t.lt[a] = ilog2(E) - t.lbr[a];
    t.lb = t.lt[0] + t.lt[1] + t.lt[2];
    const unsigned ntile = (unsigned)((nq + E - 1) / E);
    t.grid[0] = ntile << t.lb;
    t.grid[1] = ntile;
    t.grid[2] = ntile;
    return t;
}

static dim3 trav_grid(const Trav& t) { return dim3(t.grid[0], t.grid[1], t.grid[2]); }

// Lattice site (i, j, k) of this thread; false for padding sites.
__device__ __forceinline__ bool trav_site(const Trav& t, int idx[3]) {
    const unsigned x = blockIdx.x;
    const unsigned tk = x >> t.lb, l = x & ((1u << t.lb) - 1u);
    const unsigned bk = l & ((1u << t.lt[2]) - 1u);
    const unsigned bj = (l >> t.lt[2]) & ((1u << t.lt[1]) - 1u);
    const unsigned bi = l >> (t.lt[2] + t.lt[1]);
    const unsigned tid = threadIdx.x;
    idx[0] = (int)((((blockIdx.z << t.lt[0]) + bi) << t.lbr[0]) + (tid >> (t.lbr[2] + t.lbr[1])));
    idx[1] = (int)((((blockIdx.y << t.lt[1]) + bj) << t.lbr[1]) + ((tid >> t.lbr[2]) & ((1u << t.lbr[1]) - 1u)));
    idx[2] = (int)((((tk << t.lt[2]) + bk) << t.lbr[2]) + (tid & ((1u << t.lbr[2]) - 1u)));
    return idx[0] < t.nq && idx[1] < t.nq && idx[2] < t.nq;
}

__device__ __forceinline__ long long site_index(const int idx[3], int nq) {
    return ((long long)idx[0] * nq + idx[1]) * nq + idx[2];
}

// --------------------------------------------------------------------------
// deposit (optionally drifting to an output time on the fly:
// d_out = d + dr v + dD1 psi1 + dD2 psi2, coefficients in snap[0..2])
// --------------------------------------------------------------------------
// RSD (with SNAP): then shift along z into redshift space,
// dz += cv v_z + c1 psi1_z + c2 psi2_z (coefficients in snap[3..5])
template <bool SNAP, bool RSD = false>
__global__ void k_deposit(const float* __restrict__ d, const float* __restrict__ v, const float* __restrict__ psi1,
                          const float* __restrict__ psi2, unsigned long long* __restrict__ dep, int nq, int ng,
                          float inv_cell, long long np, const double* __restrict__ snap, int* status, Trav tv) {
    int idx[3];
    if (!trav_site(tv, idx)) return;
    const long long p = site_index(idx, nq);
    float dx[3];
    float dr = 0.f, d1 = 0.f, d2 = 0.f;
    if (SNAP) {
        dr = (float)snap[0];
        d1 = (float)snap[1];
        d2 = (float)snap[2];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        dx[a] = d[a * np + p];
        if (SNAP) dx[a] += dr * v[a * np + p] + d1 * psi1[a * np + p] + d2 * psi2[a * np + p];
    }
    if (RSD) dx[2] += (float)snap[3] * v[2 * np + p] + (float)snap[4] * psi1[2 * np + p] + (float)snap[5] * psi2[2 * np + p];
    Cic c;
    if (!particle_cic(idx, nq, ng, inv_cell, dx, c)) {
        set_status(status, COLA_ENONFINITE);
        return;
    }
    unsigned long long w[8];
    cic_fix_weights(c, w);
    const int ix[2] = {c.c0[0], c.c1[0]};
    const int iy[2] = {c.c0[1], c.c1[1]};
    const int iz[2] = {c.c0[2], c.c1[2]};
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int e = 0; e < 2; ++e)
                atomicAdd(dep + ((long long)ix[a] * ng + iy[b]) * ng + iz[e], w[4 * a + 2 * b + e]);
}

int launch_deposit_ex(const float* d, const float* v, const float* psi1, const float* psi2, unsigned long long* dep,
                      int nq, int ng, double box, const double* snap, int* status, cudaStream_t s, bool rsd) {
    const long long np = (long long)nq * nq * nq;
    const Trav tv = make_trav(nq);
    const dim3 grid = trav_grid(tv);
    const int T = kTravThreads;
    const float inv_cell = (float)((double)ng / box);
    ProfScope ps(kKDeposit, s);
    if (snap && rsd)
        k_deposit<true, true><<<grid, T, 0, s>>>(d, v, psi1, psi2, dep, nq, ng, inv_cell, np, snap, status, tv);
    else if (snap)
        k_deposit<true><<<grid, T, 0, s>>>(d, v, psi1, psi2, dep, nq, ng, inv_cell, np, snap, status, tv);
    else
        k_deposit<false><<<grid, T, 0, s>>>(d, v, psi1, psi2, dep, nq, ng, inv_cell, np, nullptr, status, tv);
    return check_launch();
}

// --------------------------------------------------------------------------
// CIC interpolation of the three force components from the interleaved,
// x-blocked force mesh (real view): component j of cell (ix, iy, z) at
// frow(ix, iy, j) P2 + z, P2 = 2P floats, so the three components of a cell
// are P2 apart.
// --------------------------------------------------------------------------
__device__ __forceinline__ void gather3(const float* __restrict__ Fm, int ng, long long P2, const Cic& c,
                                        float F[3]) {
    const FRow fr = force_rows(ng);
    F[0] = F[1] = F[2] = 0.f;
    const int ix[2] = {c.c0[0], c.c1[0]};
    const int iy[2] = {c.c0[1], c.c1[1]};
    const int iz[2] = {c.c0[2], c.c1[2]};
    const float wx[2] = {1.f - c.f[0], c.f[0]};
    const float wy[2] = {1.f - c.f[1], c.f[1]};
    const float wz[2] = {1.f - c.f[2], c.f[2]};
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const long long row = frow(ix[a], iy[b], 0, fr) * P2;
            const float wab = wx[a] * wy[b];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const float w = wab * wz[e];
                const long long q = row + iz[e];
                F[0] += w * __ldg(Fm + q);
                F[1] += w * __ldg(Fm + q + P2);
                F[2] += w * __ldg(Fm + q + 2 * P2);
            }
        }
}

__global__ void k_gather(const float* __restrict__ Fm, const float* __restrict__ d, float* __restrict__ out, int nq,
                         int ng, long long P2, float inv_cell, long long np, Trav tv) {
    int idx[3];
    if (!trav_site(tv, idx)) return;
    const long long p = site_index(idx, nq);
    float dx[3] = {d[p], d[np + p], d[2 * np + p]};
    Cic c;
    if (!particle_cic(idx, nq, ng, inv_cell, dx, c)) {
        out[p] = out[np + p] = out[2 * np + p] = __int_as_float(0x7fc00000);
        return;
    }
    float F[3];
    gather3(Fm, ng, P2, c, F);
    out[p] = F[0];
    out[np + p] = F[1];
    out[2 * np + p] = F[2];
}

int launch_gather(const float2* Fm, const float* d, float* out, int nq, int ng, double box, cudaStream_t s) {
    const long long np = (long long)nq * nq * nq;
    const Trav tv = make_trav(nq);
    ProfScope ps(kKGather, s);
    k_gather<<<trav_grid(tv), kTravThreads, 0, s>>>((const float*)Fm, d, out, nq, ng, 2ll * fft_pitch(ng),
                                                       (float)((double)ng / box), np, tv);
    return check_launch();
}

// --------------------------------------------------------------------------
// fused gather + kick + drift of node j.  row = FP64 table row:
// (a, green, c1, c2, kick, drift, dD1, dD2, ...), each rounded once to FP32.
//   A = F - c1 psi1 - c2 psi2;  v += kick A;  (not last) d += drift v + dD1 psi1 + dD2 psi2
// PM-only (App. B): A = F, d += drift v.
// --------------------------------------------------------------------------
__global__ void k_gather_kick_drift(const float* __restrict__ Fm, float* __restrict__ d, float* __restrict__ v,
                                    const float* __restrict__ psi1, const float* __restrict__ psi2,
                                    const double* __restrict__ row, int nq, int ng, long long P2, float inv_cell,
                                    long long np, int last, int pm_only, int* status, Trav tv) {
    int idx[3];
    if (!trav_site(tv, idx)) return;
    const long long p = site_index(idx, nq);
    const float c1 = (float)row[2], c2 = (float)row[3], kick = (float)row[4];
    const float drift = (float)row[5], dD1 = (float)row[6], dD2 = (float)row[7];
    float dx[3] = {d[p], d[np + p], d[2 * np + p]};
    Cic c;
    if (!particle_cic(idx, nq, ng, inv_cell, dx, c)) {
        set_status(status, COLA_ENONFINITE);
        return;
    }
    float F[3];
    gather3(Fm, ng, P2, c, F);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const long long q = a * np + p;
        const float s1 = psi1[q], s2 = psi2[q];
        const float acc = pm_only ? F[a] : F[a] - c1 * s1 - c2 * s2;
        const float vn = v[q] + kick * acc;
        v[q] = vn;
        if (!last) d[q] = dx[a] + (pm_only ? drift * vn : drift * vn + dD1 * s1 + dD2 * s2);
    }
}

int launch_gather_kick_drift(const float2* Fm, cola_state st, const double* row, int nq, int ng, double box, int last,
                             int pm_only, int* status, cudaStream_t s) {
    const long long np = (long long)nq * nq * nq;
    const Trav tv = make_trav(nq);
    ProfScope ps(kKGatherKD, s);
    k_gather_kick_drift<<<trav_grid(tv), kTravThreads, 0, s>>>(
        (const float*)Fm, st.d, st.v, st.psi1, st.psi2, row, nq, ng,
        2ll * fft_pitch(ng), (float)((double)ng / box), np, last, pm_only, status, tv);
    return check_launch();
}

// --------------------------------------------------------------------------
// fixed-point mesh -> delta (unpadded float ng^3); clears the fixed-point mesh
// --------------------------------------------------------------------------
__global__ void k_fix_to_delta(unsigned long long* dep, float* delta, long long n3, float scale, int clear) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n3) return;
    delta[i] = (float)dep[i] * scale - 1.0f;
    if (clear) dep[i] = 0ull;
}

int launch_fix_to_delta(unsigned long long* dep, float* delta, int ng, float scale, cudaStream_t s, bool clear) {
    const long long n3 = (long long)ng * ng * ng;
    ProfScope ps(kKFixToDelta, s);
    k_fix_to_delta<<<(unsigned)((n3 + 255) / 256), 256, 0, s>>>(dep, delta, n3, scale, clear ? 1 : 0);
    return check_launch();
}

// --------------------------------------------------------------------------
// adjoint of the CIC gather: deposit per-particle vectors res (SoA 3 x Np)
// with the gather's weights into three signed fixed-point meshes (2^30 per
// unit, two's complement in uint64 atomics: order-independent)
// --------------------------------------------------------------------------
__global__ void k_adjoint_deposit(const float* __restrict__ d, const float* __restrict__ res,
                                  unsigned long long* __restrict__ fix3, int nq, int ng, float inv_cell, long long np,
                                  Trav tv) {
    int idx[3];
    if (!trav_site(tv, idx)) return;
    const long long p = site_index(idx, nq);
    float dx[3] = {d[p], d[np + p], d[2 * np + p]};
    Cic c;
    if (!particle_cic(idx, nq, ng, inv_cell, dx, c)) return;
    const long long n3 = (long long)ng * ng * ng;
    const float wx[2] = {1.f - c.f[0], c.f[0]};
    const float wy[2] = {1.f - c.f[1], c.f[1]};
    const float wz[2] = {1.f - c.f[2], c.f[2]};
    const int ix[2] = {c.c0[0], c.c1[0]};
    const int iy[2] = {c.c0[1], c.c1[1]};
    const int iz[2] = {c.c0[2], c.c1[2]};
    const float r[3] = {res[p], res[np + p], res[2 * np + p]};
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const float w = wx[a] * wy[b] * wz[e];
                const long long cell = ((long long)ix[a] * ng + iy[b]) * ng + iz[e];
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const long long q = __float2ll_rn(w * r[j] * 1073741824.0f);  // 2^30
                    atomicAdd(fix3 + j * n3 + cell, (unsigned long long)q);
                }
            }
}

int launch_adjoint_deposit(const float* d, const float* res, unsigned long long* fix3, int nq, int ng, double box,
                           cudaStream_t s) {
    const long long np = (long long)nq * nq * nq;
    const Trav tv = make_trav(nq);
    ProfScope ps(kKDeposit, s);
    k_adjoint_deposit<<<trav_grid(tv), kTravThreads, 0, s>>>(d, res, fix3, nq, ng, (float)((double)ng / box), np,
                                                                tv);
    return check_launch();
}

// --------------------------------------------------------------------------
// Row binning of the PM step: a counting sort of the particle indices by the
// (x, y) mesh row of their lower CIC corner, key x ng + y.  k_bin_count takes
// each particle's rank inside its bin with an atomic (counts start at zero),
// exclusive_scan turns the counts into offsets, k_bin_scatter writes
// sorted[start[key] + rank] = p and, at the same place, the particle's CIC
// fractions and lower z cell (its x and y cells are the bin's), so that the
// fused passes read one contiguous 16-byte record per particle visit; rank[p]
// is then replaced by that sorted position (-1 for a particle left out).  The order inside a bin depends on the atomics
// and changes no result: the fused deposit adds integers, and every particle's
// partial force sums are its own.  A non-finite position latches
// COLA_ENONFINITE and leaves the particle out of every bin.
// --------------------------------------------------------------------------
__global__ void k_bin_count(const float* __restrict__ d, int nq, int ng, float inv_cell, long long np,
                            int* __restrict__ count, int* __restrict__ key, int* __restrict__ rank, int* status,
                            Trav tv) {
    int idx[3];
    if (!trav_site(tv, idx)) return;
    const long long p = site_index(idx, nq);
    const float dx[3] = {d[p], d[np + p], d[2 * np + p]};
    Cic c;
    if (!particle_cic(idx, nq, ng, inv_cell, dx, c)) {
        set_status(status, COLA_ENONFINITE);
        key[p] = -1;
        return;
    }
    const int k = c.c0[0] * ng + c.c0[1];
    if (!bounds_ok(status, (unsigned)k < (unsigned)(ng * ng))) {
        key[p] = -1;
        return;
    }
    key[p] = k;
    rank[p] = atomicAdd(count + k, 1);
}

__global__ void k_bin_scatter(const float* __restrict__ d, int nq, int ng, float inv_cell, long long np,
                              const int* __restrict__ key, int* __restrict__ rank, const int* __restrict__ start,
                              int* __restrict__ sorted, float4* __restrict__ cic, int* status, Trav tv) {
    int idx[3];
    if (!trav_site(tv, idx)) return;
    const long long p = site_index(idx, nq);
    const int k = key[p];
    if (k < 0) {
        rank[p] = -1;
        return;
    }
    const float dx[3] = {d[p], d[np + p], d[2 * np + p]};
    Cic c;
    particle_cic(idx, nq, ng, inv_cell, dx, c);  // finite: k_bin_count binned it
    const int pos = start[k] + rank[p];
    if (!bounds_ok(status, pos >= 0 && pos < np)) {
        rank[p] = -1;
        return;
    }
    sorted[pos] = (int)p;
    cic[pos] = make_float4(c.f[0], c.f[1], c.f[2], __int_as_float(c.c0[2]));
    rank[p] = pos;
}

int launch_bins(const float* d, int nq, int ng, double box, const BinBufs& b, int* status, cudaStream_t s) {
    const long long np = (long long)nq * nq * nq;
    const long long nb = (long long)ng * ng;
    ProfScope ps(kKBins, s);
    if (cudaMemsetAsync(b.start, 0, (size_t)(nb + 1) * sizeof(int), s) != cudaSuccess) return COLA_ECUDA;
    const Trav tv = make_trav(nq);
    k_bin_count<<<trav_grid(tv), kTravThreads, 0, s>>>(d, nq, ng, (float)((double)ng / box), np, b.start, b.key,
                                                        b.rank, status, tv);
    int rc = check_launch();
    if (rc) return rc;
    if ((rc = exclusive_scan(b.start, nb, b.sums, s))) return rc;
    k_bin_scatter<<<trav_grid(tv), kTravThreads, 0, s>>>(d, nq, ng, (float)((double)ng / box), np, b.key, b.rank,
                                                          b.start, b.sorted, b.cic, status, tv);
    return check_launch();
}

// --------------------------------------------------------------------------
// Kick + drift of node j from the partial force sums the fused c2r pass left
// (record layout: fft_fused.cuh).  The record of particle p is at its sorted
// position pos[p]: 12 floats S(dy, xs)[c] at 6 dy + 3 xs + c, every one of them
// written in each step (zeros where a tile held both x rows), summed in one
// fixed order:  F = (S(0,0) + S(0,1)) + (S(1,0) + S(1,1)),
// then exactly the arithmetic of k_gather_kick_drift.  A particle the binning
// left out (non-finite position, pos = -1) latches COLA_ENONFINITE and keeps its
// state.
// --------------------------------------------------------------------------
__device__ __forceinline__ void record_force(const float4* __restrict__ rec, float F[3]) {
    const float4 a = __ldg(rec), b = __ldg(rec + 1), c = __ldg(rec + 2);
    // a = S00 x y z, S01 x | b = S01 y z, S10 x y | c = S10 z, S11 x y z
    F[0] = (a.x + a.w) + (b.z + c.y);
    F[1] = (a.y + b.x) + (b.w + c.z);
    F[2] = (a.z + b.y) + (c.x + c.w);
}

__global__ void k_slot_kick_drift(const float* __restrict__ slots, const int* __restrict__ pos,
                                  float* __restrict__ d, float* __restrict__ v, const float* __restrict__ psi1,
                                  const float* __restrict__ psi2, const double* __restrict__ row, int nq,
                                  long long np, int last, int pm_only, int* status, Trav tv) {
    int idx[3];
    if (!trav_site(tv, idx)) return;
    const long long p = site_index(idx, nq);
    const int at = pos[p];
    if (at < 0) {
        set_status(status, COLA_ENONFINITE);
        return;
    }
    if (!bounds_ok(status, at < np)) return;
    const float c1 = (float)row[2], c2 = (float)row[3], kick = (float)row[4];
    const float drift = (float)row[5], dD1 = (float)row[6], dD2 = (float)row[7];
    float F[3];
    record_force(reinterpret_cast<const float4*>(slots) + 3ll * at, F);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const long long q = a * np + p;
        const float s1 = psi1[q], s2 = psi2[q];
        const float acc = pm_only ? F[a] : F[a] - c1 * s1 - c2 * s2;
        const float vn = v[q] + kick * acc;
        v[q] = vn;
        if (!last) d[q] = d[q] + (pm_only ? drift * vn : drift * vn + dD1 * s1 + dD2 * s2);
    }
}

int launch_slot_kick_drift(const float* slots, const int* pos, cola_state st, const double* row, int nq, int last,
                           int pm_only, int* status, cudaStream_t s) {
    const long long np = (long long)nq * nq * nq;
    const Trav tv = make_trav(nq);
    ProfScope ps(kKKickDrift, s);
    k_slot_kick_drift<<<trav_grid(tv), kTravThreads, 0, s>>>(slots, pos, st.d, st.v, st.psi1, st.psi2, row, nq, np,
                                                              last, pm_only, status, tv);
    return check_launch();
}

// the force alone (cola_pm_force), NaN for a particle the binning left out
__global__ void k_slot_force(const float* __restrict__ slots, const int* __restrict__ pos, float* __restrict__ out,
                             int nq, long long np, Trav tv) {
    int idx[3];
    if (!trav_site(tv, idx)) return;
    const long long p = site_index(idx, nq);
    const int at = pos[p];
    if (at < 0) {
        out[p] = out[np + p] = out[2 * np + p] = __int_as_float(0x7fc00000);
        return;
    }
    float F[3];
    record_force(reinterpret_cast<const float4*>(slots) + 3ll * at, F);
    out[p] = F[0];
    out[np + p] = F[1];
    out[2 * np + p] = F[2];
}

int launch_slot_force(const float* slots, const int* pos, float* out, int nq, cudaStream_t s) {
    const long long np = (long long)nq * nq * nq;
    const Trav tv = make_trav(nq);
    ProfScope ps(kKGather, s);
    k_slot_force<<<trav_grid(tv), kTravThreads, 0, s>>>(slots, pos, out, nq, np, tv);
    return check_launch();
}

int mark_dep_dirty(void* ws, cudaStream_t s) {
    return cudaMemsetAsync(wsp(ws, kHdrDepState), 0, sizeof(int), s) == cudaSuccess ? COLA_OK : COLA_ECUDA;
}

int mark_dep_clean(void* ws, cudaStream_t s) {
    return cudaMemsetAsync(wsp(ws, kHdrDepState), kDepClean & 0xff, sizeof(int), s) == cudaSuccess ? COLA_OK
                                                                                                   : COLA_ECUDA;
}

// zero count[0 .. n) (n even) unless the state word says it is already zero
__global__ void k_clear_if_dirty(ulonglong2* __restrict__ c, long long n2, const int* state) {
    if (*state == kDepClean) return;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n2; e += (long long)gridDim.x * blockDim.x)
        c[e] = make_ulonglong2(0ull, 0ull);
}

int clear_dep_if_dirty(void* ws, unsigned long long* dep, size_t count, cudaStream_t s) {
    k_clear_if_dirty<<<num_sms() * 4, 512, 0, s>>>(reinterpret_cast<ulonglong2*>(dep), (long long)(count / 2),
                                                         reinterpret_cast<const int*>(wsp(ws, kHdrDepState)));
    return check_launch();
}

// one thread: the bounds check of index < n, then the write it guards
__global__ void k_checks_probe(int* area, int index, int n, int* status) {
    if (bounds_ok(status, index < n)) area[index] = index;
}

int launch_checks_probe(int* area, int index, int n, int* status, cudaStream_t s) {
    k_checks_probe<<<1, 1, 0, s>>>(area, index, n, status);
    return check_launch();
}

int set_particle_traversal(int edge, int brick_k) {
    if (edge == 0) edge = kTileEdgeDefault;
    if (brick_k == 0) brick_k = kBrickKDefault;
    if (brick_k < 8 || brick_k > kTravThreads || (brick_k & (brick_k - 1))) return COLA_EINVAL;
    if (edge < 32 || edge > 4096 || (edge & (edge - 1)) || edge < brick_k) return COLA_EINVAL;
    g_tile_edge = edge;
    g_brick_k = brick_k;
    return COLA_OK;
}

}  // namespace cola
