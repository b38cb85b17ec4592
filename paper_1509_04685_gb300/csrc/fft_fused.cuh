// Fused z passes of the PM step (Sec. 2.2): the CIC deposit moved into the
// forward r2c pass along z, and the CIC gather moved into the inverse c2r
// pass, so that neither the density nor the real force field ever goes
// through global memory.  The particles reach the tiles through the row bins
// (pm.cu: particles sorted by the (x, y) mesh row of their lower CIC corner).
//
// r2c + deposit.  A tile is TY consecutive mesh rows (x, y0 .. y0 + TY - 1) of
// one x (TY divides ng).  The particles that can reach it sit in the bins
// x0 in {x - 1, x}, y0' in [y0 - 1, y0 + TY - 1] (periodic): 2 (TY + 1) bins.
// Each adds its 2^40 fixed-point weights (the integers the global deposit
// adds, cic_fix_weights) of the corners inside the tile to 64-bit counts in
// shared memory: integer sums, so the rows are bit-identical to the global
// fixed-point mesh, whatever the order.  The rows then go through the r2c
// transform of the fixed-point z pass and its post-processing, and the
// half-complex rows are written to component 0 of the force mesh.
//
// c2r + gather.  A tile is the three force components of TX consecutive x rows
// (x_first .. x_first + TX - 1, TX dividing the x-block of the force layout) of
// one y: 3 TX consecutive rows of the force mesh.  After the c2r transform the
// real rows stay in shared memory.  The particles whose CIC stencil reaches
// them sit in the bins x0 in [x_first - 1, x_first + TX - 1], y0 in {y - 1, y}:
// 2 (TX + 1) bins.  A particle's four (x, y) rows are (x0, y0), (x1, y0),
// (x0, y1), (x1, y1) with x1 = x0 + 1, y1 = y0 + 1 (periodic).  This tile holds
// either both x rows of one y (x0 inside the tile, or x0 and x1 both) or only
// x1.  The partial sum over the rows it holds,
//   S = sum_a (wx_a wy_dy) (wz_0 F(a, z0) + wz_1 F(a, z1))   (a in x order),
// goes to slot (dy, xs) of the particle: dy = y - y0 (0 or 1), xs = 0 if the
// tile holds x0, 1 if it holds only x1.  The slots of a particle form one
// record of 12 floats at its sorted position pos (where its CIC record is), so
// that a tile's writes are contiguous: component c of slot (dy, xs) at
// slots[12 pos + 6 dy + 3 xs + c].  A tile that holds both x rows writes the
// sum to (dy, 0) and zeros to (dy, 1); a particle whose x0 and x1 fall into
// different tiles gets (dy, 0) and (dy, 1) from one each.  Every float of the
// record is written once per step, and the kick sums the four slots in one
// fixed order (pm.cu), so the force is deterministic.
#pragma once

#include "fft_static.cuh"
#include "particles.cuh"

namespace cola {

constexpr int kMaxTileBins = 2 * (64 + 1);  // row tiles of at most 64 rows

// Bin list of a tile in shared memory: bin b is mesh row (x0, y0) =
// (bxy[b] >> 16, bxy[b] & 0xffff) (coord_of(b) packs them), it starts at beg[b]
// in the sorted arrays, and pre[b] is the number of particles in the bins
// before it.  Returns the total.  Ends synchronised.
// The group is threads tid < nthr (whole warps) synchronised by `sync`.
template <class CoordOf, class Sync>
__device__ __forceinline__ int tile_bins_g(const RowBins& bins, int nb, int ng, const CoordOf& coord_of, int* beg,
                                           int* pre, int* bxy, int tid, int nthr, const Sync& sync) {
    for (int b = tid; b < nb; b += nthr) {
        const int xy = coord_of(b);
        const int k = (xy >> 16) * ng + (xy & 0xffff);
        const int s0 = __ldg(bins.start + k), s1 = __ldg(bins.start + k + 1);
        beg[b] = s0;
        pre[b + 1] = s1 - s0;
        bxy[b] = xy;
    }
    sync();
    if (tid < 32) {
        const unsigned full = 0xffffffffu;
        const int lane = tid;
        int carry = 0;
        for (int base = 0; base < nb; base += 32) {
            const int b = base + lane;
            int v = b < nb ? pre[b + 1] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(full, v, o);
                if (lane >= o) v += y;
            }
            if (b < nb) pre[b + 1] = carry + v;
            carry += __shfl_sync(full, v, 31);
        }
        if (lane == 0) pre[0] = 0;
    }
    sync();
    return pre[nb];
}
// the whole block as the group
template <class CoordOf>
__device__ __forceinline__ int tile_bins(const RowBins& bins, int nb, int ng, const CoordOf& coord_of, int* beg,
                                         int* pre, int* bxy) {
    return tile_bins_g(bins, nb, ng, coord_of, beg, pre, bxy, (int)threadIdx.x, (int)blockDim.x,
                       [] { __syncthreads(); });
}

// the bin holding flat index e (pre[b] <= e < pre[b + 1])
__device__ __forceinline__ int tile_find(const int* pre, int nb, int e) {
    int lo = 0, hi = nb;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= e)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// A particle of a tile as read from the bins: its index (p < 0: none), its
// CIC record (fractions, lower z cell) and the tile's bin it came from.  The
// compile-time forms read each tile's particles into registers one tile ahead,
// so that the latency of these loads overlaps the FFT passes instead of
// stalling the block.
struct TilePart {
    int p, b, pos;
    float4 q;
};

__device__ __forceinline__ TilePart tile_load(int e, int total, const RowBins& bins, const int* beg, const int* pre,
                                              int nb) {
    TilePart t;
    t.p = -1;
    t.b = 0;
    t.pos = 0;
    t.q = make_float4(0.f, 0.f, 0.f, 0.f);
    if (e < total) {
        const int b = tile_find(pre, nb, e);
        const int pos = beg[b] + (e - pre[b]);
        if (!bounds_ok(bins.status, pos >= 0 && pos < bins.np)) return t;
        t.p = __ldg(bins.sorted + pos);
        t.q = __ldg(bins.cic + pos);
        t.b = b;
        t.pos = pos;
        if (kChecks && !bounds_ok(bins.status, (unsigned)__float_as_int(t.q.w) < (unsigned)bins.ng)) t.p = -1;
    }
    return t;
}

// the particle's CIC corners: x0, y0 from its bin, z0 and the fractions from its record
__device__ __forceinline__ bool part_cic(const TilePart& t, const int* bxy, int ng, Cic& c) {
    if (t.p < 0) return false;
    const int xy = bxy[t.b];
    c.c0[0] = xy >> 16;
    c.c0[1] = xy & 0xffff;
    c.c0[2] = __float_as_int(t.q.w);
#pragma unroll
    for (int a = 0; a < 3; ++a) c.c1[a] = c.c0[a] + 1 == ng ? 0 : c.c0[a] + 1;
    c.f[0] = t.q.x;
    c.f[1] = t.q.y;
    c.f[2] = t.q.z;
    return true;
}

// Deposit of one particle's corners inside rows (x, y0 + l), l < ty, into cnt[l ng + z].
__device__ __forceinline__ void deposit_one(const TilePart& t, const int* bxy, int ng, int x, int y0, int ty,
                                            unsigned long long* cnt) {
    Cic c;
    if (!part_cic(t, bxy, ng, c)) return;
    unsigned long long w[8];
    cic_fix_weights(c, w);
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        if ((a ? c.c1[0] : c.c0[0]) != x) continue;
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int l = (b ? c.c1[1] : c.c0[1]) - y0;
            if (l < 0 || l >= ty) continue;
            atomicAdd(cnt + l * ng + c.c0[2], w[4 * a + 2 * b]);
            atomicAdd(cnt + l * ng + c.c1[2], w[4 * a + 2 * b + 1]);
        }
    }
}

// Deposit of all the tile's particles (loaded here).
__device__ __forceinline__ void tile_deposit(const RowBins& bins, const int* beg, const int* pre, const int* bxy,
                                             int nb, int total, int ng, int x, int y0, int ty,
                                             unsigned long long* cnt) {
    for (int e = threadIdx.x; e < total; e += blockDim.x)
        deposit_one(tile_load(e, total, bins, beg, pre, nb), bxy, ng, x, y0, ty, cnt);
}

// real value z of row l of a c2r result in shared memory (complex pairs,
// element m of row l at l lstr + spad(m))
__device__ __forceinline__ float row_value(const float2* Z, int lstr, int l, int z) {
    return reinterpret_cast<const float*>(Z + l * lstr + spad(z >> 1))[z & 1];
}

// Partial CIC sums of one particle from rows l = 3 xi + c (component c of mesh
// row (x_first + xi, y)), written to its slot.
__device__ __forceinline__ void gather_one(const TilePart& t, const int* bxy, long long np, int ng, int x_first,
                                           int tx, int y, const float2* Z, int lstr, float* __restrict__ slots) {
    Cic c;
    if (!part_cic(t, bxy, ng, c)) return;
    const int dy = c.c0[1] == y ? 0 : 1;
    const int i0 = c.c0[0] - x_first, i1 = c.c1[0] - x_first;
    const bool in0 = i0 >= 0 && i0 < tx, in1 = i1 >= 0 && i1 < tx;
    if ((!in0 && !in1) || (dy && c.c1[1] != y)) return;  // never for a particle of the tile's bins
    const float wy = dy ? c.f[1] : 1.f - c.f[1];
    const float wz0 = 1.f - c.f[2], wz1 = c.f[2];
    const float w0 = (1.f - c.f[0]) * wy, w1 = c.f[0] * wy;
    float acc[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (in0) {
            const int l = 3 * i0 + k;
            acc[k] = w0 * (wz0 * row_value(Z, lstr, l, c.c0[2]) + wz1 * row_value(Z, lstr, l, c.c1[2]));
            if (in1) {
                const int l1 = 3 * i1 + k;
                acc[k] += w1 * (wz0 * row_value(Z, lstr, l1, c.c0[2]) + wz1 * row_value(Z, lstr, l1, c.c1[2]));
            }
        } else {
            const int l1 = 3 * i1 + k;
            acc[k] = w1 * (wz0 * row_value(Z, lstr, l1, c.c0[2]) + wz1 * row_value(Z, lstr, l1, c.c1[2]));
        }
    }
    float* r = slots + 12ll * t.pos + 6 * dy;  // 8-byte aligned
    if (in0 && in1) {
        float2* r2 = reinterpret_cast<float2*>(r);
        __stcs(r2, make_float2(acc[0], acc[1]));
        __stcs(r2 + 1, make_float2(acc[2], 0.f));
        __stcs(r2 + 2, make_float2(0.f, 0.f));
    } else {
        if (!in0) r += 3;
#pragma unroll
        for (int k = 0; k < 3; ++k) __stcs(r + k, acc[k]);
    }
}

// Partial sums of all the tile's particles (loaded here).
__device__ __forceinline__ void tile_gather(const RowBins& bins, const int* beg, const int* pre, const int* bxy,
                                            int nb, int total, long long np, int ng, int x_first, int tx, int y,
                                            const float2* Z, int lstr, float* __restrict__ slots) {
    for (int e = threadIdx.x; e < total; e += blockDim.x)
        gather_one(tile_load(e, total, bins, beg, pre, nb), bxy, np, ng, x_first, tx, y, Z, lstr, slots);
}

// ---------------------------------------------------------------------------
// compile-time forms (the runtime forms are in fft.cu)
// ---------------------------------------------------------------------------
template <int N, int NR, int T>
constexpr size_t z_r2c_dep_smem() {
    return ((size_t)NR * N + 2 * (size_t)NR * (spad(N / 2) + 1) + ordered_tw_size(N / 2) + N / 2 + 1) * 8;
}

// particles per thread read one tile ahead (more go through the direct path)
constexpr int kDepAhead = 3;
constexpr int kGatherAhead = 2;

// r2c + deposit: tiles of TY = NR rows of one x, t = x (N / NR) + y0 / NR.
// Per tile: clear the counts, deposit the particles read during the previous
// tile's transform, list the next tile's bins and read its particles, then the
// r2c transform and its post-processing.
template <int N, int NR, int T, int MB>
__global__ void __launch_bounds__(T, MB)
    k_fft_z_r2c_dep_s(const float* __restrict__ d, int nq, long long np, float inv_cell, RowBins bins, float2* out,
                      long long rs, int ntiles, float scale, const float2* __restrict__ tw, FRow fr,
                      float* __restrict__ delta_out) {
    static_assert(NR + 1 <= N && 2 * (NR + 1) <= kMaxTileBins, "tile bins must be distinct");
    constexpr int M = N / 2;
    constexpr int TPX = N / NR;  // tiles per x
    constexpr int NB = 2 * (NR + 1);
    using Geo = RowTile<M, NR>;
    extern __shared__ float2 sm[];
    __shared__ long long obase[NR];
    __shared__ int beg[NB], pre[NB + 1], bxy[NB];
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(sm);
    float2* A = sm + NR * N;
    float2* Bf = A + NR * Geo::LSTR;
    float2* tws = Bf + NR * Geo::LSTR;       // pass-ordered twiddles of the M-point transform
    float2* twh = tws + ordered_tw_size(M);  // W_N^k, k <= M, for the r2c post-processing
    ordered_twiddles<M, T, 2>(tws, tw);
    for (int q = threadIdx.x; q <= M; q += T) twh[q] = __ldg(tw + q);
    // bins x0 in {x - 1, x}, y0' in [y0 - 1, y0 + NR - 1] of tile t
    auto list = [&](int t) {
        const int x = t / TPX, y0 = (t - x * TPX) * NR;
        return tile_bins(
            bins, NB, N,
            [&](int b) { return (wrap(x - 1 + b / (NR + 1), N) << 16) | wrap(y0 - 1 + b % (NR + 1), N); }, beg, pre,
            bxy);
    };
    TilePart ahead[kDepAhead];
    int total = 0;
    int t = blockIdx.x;
    if (t < ntiles) {
        total = list(t);
#pragma unroll
        for (int k = 0; k < kDepAhead; ++k) ahead[k] = tile_load(threadIdx.x + k * T, total, bins, beg, pre, NB);
    }
    for (; t < ntiles; t += gridDim.x) {
        const int x = t / TPX, y0 = (t - x * TPX) * NR;
        ulonglong2* c2 = reinterpret_cast<ulonglong2*>(cnt);
        for (int e = threadIdx.x; e < NR * N / 2; e += T) c2[e] = make_ulonglong2(0ull, 0ull);
        if (threadIdx.x < NR) obase[threadIdx.x] = frow(x, y0 + threadIdx.x, 0, fr) * rs;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kDepAhead; ++k) deposit_one(ahead[k], bxy, N, x, y0, NR, cnt);
        for (int e = threadIdx.x + kDepAhead * T; e < total; e += T)
            deposit_one(tile_load(e, total, bins, beg, pre, NB), bxy, N, x, y0, NR, cnt);
        __syncthreads();
        const int tn = t + gridDim.x;
        if (tn < ntiles) {
            total = list(tn);
#pragma unroll
            for (int k = 0; k < kDepAhead; ++k) ahead[k] = tile_load(threadIdx.x + k * T, total, bins, beg, pre, NB);
        }
        if (delta_out) {
            float* o = delta_out + ((long long)x * N + y0) * N;
            for (int e = threadIdx.x; e < NR * N; e += T) o[e] = (float)cnt[e] * scale - 1.0f;
        }
        const float2* Z = srun_smem<M, T, Geo, -1>(FixStage<N>{cnt, scale}, A, Bf, tws, NoHook());
        // X[k] = E[k] + W^k O[k], E = (Z[k] + conj Z[M-k]) / 2, O = (Z[k] - conj Z[M-k]) / (2i)
#pragma unroll 2
        for (int e = threadIdx.x; e < NR * (M + 1); e += T) {
            const int l = e / (M + 1), k = e - l * (M + 1);
            const float2 a = Z[l * Geo::LSTR + spad(k == M ? 0 : k)];
            const float2 b = cconj(Z[l * Geo::LSTR + spad(k == 0 ? 0 : M - k)]);
            const float2 E = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y + b.y));
            const float2 D = csub(a, b);
            const float2 O = make_float2(0.5f * D.y, -0.5f * D.x);
            __stcs(out + obase[l] + k, cadd(E, cmul(twh[k], O)));
        }
        __syncthreads();  // obase and the counts are reused by the next tile
    }
}

template <int N, int TX>
constexpr size_t z_c2r_gather_smem() {
    return ((size_t)3 * TX * (N / 2 + 2) + 2 * (size_t)3 * TX * (spad(N / 2) + 1) + ordered_tw_size(N / 2) + N / 2 +
            1) *
           8;
}

// c2r + gather: tiles of the 3 TX force rows of x_first .. x_first + TX - 1 at
// one y, t = (x_first / TX) N + y.  The rows are staged with cp.async (the next
// tile's while this one is transformed and gathered) and the particles of the
// next tile are read into registers after this one's gather.
template <int N, int TX, int T, int MB>
__global__ void __launch_bounds__(T, MB)
    k_fft_z_c2r_gather_s(const float2* __restrict__ data, long long rs, int ntiles, const float2* __restrict__ tw,
                         FRow fr, const float* __restrict__ d, int nq, long long np, float inv_cell, RowBins bins,
                         float* __restrict__ slots) {
    constexpr int NR = 3 * TX;
    constexpr int M = N / 2;
    constexpr int NB = 2 * (TX + 1);
    static_assert(TX + 1 <= N, "tile bins must be distinct");
    using Geo = RowTile<M, NR>;
    constexpr int SP = M + 2;  // staged row: X[0..M], whole 16-byte chunks
    constexpr int HS = SP / 2;
    extern __shared__ float2 sm[];
    __shared__ int beg[NB], pre[NB + 1], bxy[NB];
    float2* stg = sm;
    float2* A = stg + NR * SP;
    float2* Bf = A + NR * Geo::LSTR;
    float2* tws = Bf + NR * Geo::LSTR;
    float2* twh = tws + ordered_tw_size(M);
    ordered_twiddles<M, T, 2>(tws, tw);
    for (int q = threadIdx.x; q <= M; q += T) twh[q] = __ldg(tw + q);
    auto prefetch = [&](int t) {
        const int xg = t / N, y = t - xg * N;
        const long long row0 = frow(xg * TX, y, 0, fr);
#pragma unroll 4
        for (int e = threadIdx.x; e < NR * HS; e += T) {
            const int l = e / HS, c = (e - l * HS) * 2;
            cp_async16(stg + l * SP + c, data + (row0 + l) * rs + c);
        }
        cp_async_commit();
    };
    // bins x0 in [x_first - 1, x_first + TX - 1], y0 in {y - 1, y} of tile t
    auto list = [&](int t) {
        const int xg = t / N, y = t - xg * N, x_first = xg * TX;
        return tile_bins(
            bins, NB, N,
            [&](int b) { return (wrap(x_first - 1 + b % (TX + 1), N) << 16) | wrap(y - 1 + b / (TX + 1), N); }, beg,
            pre, bxy);
    };
    TilePart ahead[kGatherAhead];
    int total = 0;
    int t = blockIdx.x;
    if (t < ntiles) {
        prefetch(t);
        total = list(t);
#pragma unroll
        for (int k = 0; k < kGatherAhead; ++k) ahead[k] = tile_load(threadIdx.x + k * T, total, bins, beg, pre, NB);
    }
    for (; t < ntiles; t += gridDim.x) {
        const int xg = t / N, y = t - xg * N, x_first = xg * TX;
        cp_async_wait_all();
        __syncthreads();
        const int tn = t + gridDim.x;
        auto next = [&]() {
            if (tn < ntiles) prefetch(tn);
        };
        const float2* Z = srun_smem<M, T, Geo, +1>(C2rStage<M, SP>{stg, twh}, A, Bf, tws, next);
#pragma unroll
        for (int k = 0; k < kGatherAhead; ++k) gather_one(ahead[k], bxy, np, N, x_first, TX, y, Z, Geo::LSTR, slots);
        for (int e = threadIdx.x + kGatherAhead * T; e < total; e += T)
            gather_one(tile_load(e, total, bins, beg, pre, NB), bxy, np, N, x_first, TX, y, Z, Geo::LSTR, slots);
        __syncthreads();  // Z and the bin list are reused by the next tile
        if (tn < ntiles) {
            total = list(tn);
#pragma unroll
            for (int k = 0; k < kGatherAhead; ++k)
                ahead[k] = tile_load(threadIdx.x + k * T, total, bins, beg, pre, NB);
        }
    }
}

// c2r + gather with warp-owned rows: G groups of 3 TX warps per block; group g
// takes tiles t = blockIdx.x G + g, then every gridDim.x G-th (tile t is the
// three force components of the x rows x_first .. x_first + TX - 1 at one y,
// t = (x_first / TX) N + y: 3 TX consecutive rows of the force mesh).  Warp w of
// a group transforms row w of the tile: the first pass reads the row from
// global memory, the others run in place in the warp's row buffer, separated
// by __syncwarp only.  The group's named barrier (id g + 1, 96 TX threads) then
// lets its threads list the tile's bins and gather; no block-wide barrier
// follows the start-up.
template <int N, int TX, int G>
constexpr size_t z_c2r_gather_w_smem() {
    return ((size_t)ordered_tw_size(N / 2) + N / 2 + 1 + (size_t)G * 3 * TX * (spad(N / 2) + 1)) * 8;
}

template <int N, int TX, int G, int MB>
__global__ void __launch_bounds__(96 * TX * G, MB)
    k_fft_z_c2r_gather_w(const float2* __restrict__ data, long long rs, int ntiles, const float2* __restrict__ tw,
                         FRow fr, long long np, RowBins bins, float* __restrict__ slots) {
    static_assert(G >= 1 && G <= 15 && 96 * TX * G <= 1024, "named barriers 1 .. G, at most 1024 threads");
    constexpr int M = N / 2;
    constexpr int NB = 2 * (TX + 1);
    constexpr int GT = 96 * TX;  // threads of a group
    using Geo = WarpRow<M>;
    extern __shared__ float2 sm[];
    __shared__ int beg[G][NB], pre[G][NB + 1], bxy[G][NB];
    float2* tws = sm;                        // pass-ordered twiddles of the M-point transform
    float2* twh = tws + ordered_tw_size(M);  // W_N^k, k <= M, for the c2r pre-processing
    float2* rows = twh + (M + 1);
    ordered_twiddles<M, GT * G, 2>(tws, tw);
    for (int q = threadIdx.x; q <= M; q += GT * G) twh[q] = __ldg(tw + q);
    __syncthreads();
    const int g = threadIdx.x / GT, gl = threadIdx.x - g * GT, w = gl >> 5;
    float2* Z = rows + (size_t)g * 3 * TX * Geo::LSTR;
    float2* mine = Z + w * Geo::LSTR;
    const auto gsync = [g] { asm volatile("bar.sync %0, %1;\n" ::"r"(g + 1), "n"(GT) : "memory"); };
    for (int t = blockIdx.x * G + g; t < ntiles; t += gridDim.x * G) {
        const int xg = t / N, y = t - xg * N, x_first = xg * TX;
        sip_run<M, 32, Geo, +1, false, true>(C2rGlobal<M>{data + (frow(x_first, y, 0, fr) + w) * rs, twh},
                                             SSmem<Geo>{mine}, mine, tws, NoHook());
        // bins x0 in [x_first - 1, x_first + TX - 1], y0 in {y - 1, y}; its barriers
        // also publish the rows
        const int total = tile_bins_g(
            bins, NB, N,
            [&](int b) { return (wrap(x_first - 1 + b % (TX + 1), N) << 16) | wrap(y - 1 + b / (TX + 1), N); },
            beg[g], pre[g], bxy[g], gl, GT, gsync);
        for (int e = gl; e < total; e += GT)
            gather_one(tile_load(e, total, bins, beg[g], pre[g], NB), bxy[g], np, N, x_first, TX, y, Z, Geo::LSTR,
                       slots);
        gsync();  // the rows and the bin list are reused by the group's next tile
    }
}

// r2c + deposit with warp-owned rows: G groups of NR warps per block; group g
// takes tiles t = blockIdx.x G + g, then every gridDim.x G-th (tile t is rows
// (x, y0 .. y0 + NR - 1), t = x (N / NR) + y0 / NR, as in k_fft_z_r2c_dep_s).
// Per tile the group clears its NR count rows and deposits the particles of
// the tile's 2 (NR + 1) bins (integer atomics in shared memory); then warp l
// transforms count row l in place (the first pass loads all its inputs before
// it stores, so the complex row can overwrite the counts it came from),
// post-processes it and writes delta_k row (x, y0 + l).  Only the group's named
// barriers (id g + 1) separate the phases.
template <int N, int NR, int G>
constexpr int z_r2c_dep_w_tw() {  // float2 entries before the counts (16-byte aligned)
    return (ordered_tw_size(N / 2) + N / 2 + 1 + 1) & ~1;
}
template <int N, int NR, int G>
constexpr size_t z_r2c_dep_w_smem() {
    return (size_t)z_r2c_dep_w_tw<N, NR, G>() * 8 + (size_t)G * NR * N * 8;
}

template <int N, int NR, int G, int MB>
__global__ void __launch_bounds__(32 * NR * G, MB)
    k_fft_z_r2c_dep_w(RowBins bins, float2* out, long long rs, int ntiles, float scale,
                      const float2* __restrict__ tw, FRow fr, float* __restrict__ delta_out) {
    constexpr int M = N / 2;
    constexpr int TPX = N / NR;
    constexpr int NB = 2 * (NR + 1);
    constexpr int GT = 32 * NR;  // threads of a group
    static_assert(NR + 1 <= N && NB <= kMaxTileBins && G * NR <= 32, "tile bins, threads per block");
    using Geo = WarpRow<M>;
    static_assert(Geo::LSTR <= N, "a complex row fits in its count row");
    extern __shared__ float2 sm[];
    __shared__ int beg[G][NB], pre[G][NB + 1], bxy[G][NB];
    float2* tws = sm;                        // pass-ordered twiddles of the M-point transform
    float2* twh = tws + ordered_tw_size(M);  // W_N^k, k <= M, for the r2c post-processing
    unsigned long long* cnt_all = reinterpret_cast<unsigned long long*>(sm + z_r2c_dep_w_tw<N, NR, G>());
    ordered_twiddles<M, GT * G, 2>(tws, tw);
    for (int q = threadIdx.x; q <= M; q += GT * G) twh[q] = __ldg(tw + q);
    __syncthreads();
    const int g = threadIdx.x / GT, gl = threadIdx.x - g * GT, l = gl >> 5, lane = gl & 31;
    unsigned long long* cnt = cnt_all + (size_t)g * NR * N;
    unsigned long long* myc = cnt + (size_t)l * N;
    float2* Z = reinterpret_cast<float2*>(myc);
    const auto gsync = [g] { asm volatile("bar.sync %0, %1;\n" ::"r"(g + 1), "n"(GT) : "memory"); };
    for (int t = blockIdx.x * G + g; t < ntiles; t += gridDim.x * G) {
        const int x = t / TPX, y0 = (t - x * TPX) * NR;
        ulonglong2* c2 = reinterpret_cast<ulonglong2*>(cnt);
        for (int e = gl; e < NR * N / 2; e += GT) c2[e] = make_ulonglong2(0ull, 0ull);
        // bins x0 in {x - 1, x}, y0' in [y0 - 1, y0 + NR - 1]; its first barrier orders the clear
        const int total = tile_bins_g(
            bins, NB, N,
            [&](int b) { return (wrap(x - 1 + b / (NR + 1), N) << 16) | wrap(y0 - 1 + b % (NR + 1), N); }, beg[g],
            pre[g], bxy[g], gl, GT, gsync);
        for (int e = gl; e < total; e += GT)
            deposit_one(tile_load(e, total, bins, beg[g], pre[g], NB), bxy[g], N, x, y0, NR, cnt);
        gsync();
        if (delta_out) {
            float* o = delta_out + ((long long)x * N + y0 + l) * N;
            for (int e = lane; e < N; e += 32) o[e] = (float)myc[e] * scale - 1.0f;
        }
        sip_run<M, 32, Geo, -1, true, true>(FixStage<N>{myc, scale}, SSmem<Geo>{Z}, Z, tws, NoHook());
        // X[k] = E[k] + W^k O[k], E = (Z[k] + conj Z[M-k]) / 2, O = (Z[k] - conj Z[M-k]) / (2i)
        float2* orow = out + frow(x, y0 + l, 0, fr) * rs;
        for (int k = lane; k <= M; k += 32) {
            const float2 a = Z[spad(k == M ? 0 : k)];
            const float2 b = cconj(Z[spad(k == 0 ? 0 : M - k)]);
            const float2 E = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y + b.y));
            const float2 D = csub(a, b);
            const float2 O = make_float2(0.5f * D.y, -0.5f * D.x);
            __stcs(orow + k, cadd(E, cmul(twh[k], O)));
        }
        gsync();  // the counts and the bin list are reused by the group's next tile
    }
}

template <int N, int NR, int G, int MB>
inline int run_z_r2c_dep_w(const RowBins& bins, float2* out, long long rs, float scale, const float2* tw, FRow fr,
                           float* delta_out, cudaStream_t s) {
    constexpr size_t smem = z_r2c_dep_w_smem<N, NR, G>();
    static_assert((smem + 12 * (2 * (NR + 1)) * G + 4 * G + 1024) * MB <= 227 * 1024, "MB blocks must fit");
    const int nt = N * (N / NR);
    if (!set_smem((const void*)k_fft_z_r2c_dep_w<N, NR, G, MB>, smem)) return COLA_ECUDA;
    k_fft_z_r2c_dep_w<N, NR, G, MB><<<persistent_grid(smem, (nt + G - 1) / G, MB), 32 * NR * G, smem, s>>>(
        bins, out, rs, nt, scale, tw, fr, delta_out);
    return check_launch();
}

template <int N, int TX, int G, int MB>
inline int run_z_c2r_gather_w(float2* data, long long rs, const float2* tw, FRow fr, int nq, const RowBins& bins,
                              float* slots, cudaStream_t s) {
    constexpr size_t smem = z_c2r_gather_w_smem<N, TX, G>();
    static_assert((smem + 12 * (2 * TX + 3) * G + 1024) * MB <= 227 * 1024, "MB blocks must fit");
    const long long np = (long long)nq * nq * nq;
    const int nt = (N / TX) * N;
    if (!set_smem((const void*)k_fft_z_c2r_gather_w<N, TX, G, MB>, smem)) return COLA_ECUDA;
    k_fft_z_c2r_gather_w<N, TX, G, MB><<<persistent_grid(smem, (nt + G - 1) / G, MB), 96 * TX * G, smem, s>>>(
        data, rs, nt, tw, fr, np, bins, slots);
    return check_launch();
}

template <int N, int NR, int T, int MB>
inline int run_z_r2c_dep(const float* d, int nq, float inv_cell, const RowBins& bins, float2* out, long long rs,
                         float scale, const float2* tw, FRow fr, float* delta_out, cudaStream_t s) {
    constexpr size_t smem = z_r2c_dep_smem<N, NR, T>();
    static_assert((smem + 16 * NR + 8 * kMaxTileBins + 1024) * MB <= 227 * 1024, "MB blocks must fit");
    const long long np = (long long)nq * nq * nq;
    const int nt = N * (N / NR);
    if (!set_smem((const void*)k_fft_z_r2c_dep_s<N, NR, T, MB>, smem)) return COLA_ECUDA;
    k_fft_z_r2c_dep_s<N, NR, T, MB><<<persistent_grid(smem, nt, MB), T, smem, s>>>(d, nq, np, inv_cell, bins, out, rs,
                                                                                   nt, scale, tw, fr, delta_out);
    return check_launch();
}

template <int N, int TX, int T, int MB>
inline int run_z_c2r_gather(float2* data, long long rs, const float2* tw, FRow fr, const float* d, int nq,
                            float inv_cell, const RowBins& bins, float* slots, cudaStream_t s) {
    constexpr size_t smem = z_c2r_gather_smem<N, TX>();
    static_assert((smem + 8 * kMaxTileBins + 1024) * MB <= 227 * 1024, "MB blocks must fit");
    const long long np = (long long)nq * nq * nq;
    const int nt = (N / TX) * N;
    if (!set_smem((const void*)k_fft_z_c2r_gather_s<N, TX, T, MB>, smem)) return COLA_ECUDA;
    k_fft_z_c2r_gather_s<N, TX, T, MB><<<persistent_grid(smem, nt, MB), T, smem, s>>>(data, rs, nt, tw, fr, d, nq,
                                                                                      np, inv_cell, bins, slots);
    return check_launch();
}

// launchers of the specialised fused passes (fft_spec_large.cu); false when
// n has no specialisation, without launching
bool launch_z_r2c_dep_static(const float* d, int nq, float inv_cell, const RowBins& bins, float2* out, int n,
                             long long rs, float scale, const float2* tw, FRow fr, float* delta_out, cudaStream_t s,
                             int* rc);
bool launch_z_c2r_gather_static(float2* data, int n, long long rs, const float2* tw, FRow fr, const float* d, int nq,
                                float inv_cell, const RowBins& bins, float* slots, int* tx, cudaStream_t s, int* rc);

}  // namespace cola
