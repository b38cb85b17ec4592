// Compile-time specialised line transforms for the mesh sizes the library
// runs most.  Same algorithm as the runtime engine in cola_common.cuh (Stockham
// passes over the radices of static_plan, the same twiddle table, the same
// padded line-interleaved shared-memory layout l + spad(i) B), but with the
// line length N, the tile width B and the block size T known to the compiler:
// index divisions become shifts or multiply-highs, and a pass's R loads and R
// stores become one base address plus constant offsets whenever the padding is
// linear over the stride (stride a multiple of 16, or a unit stride over an
// aligned group of R | 16 elements).
#pragma once

#include "cola_common.cuh"

namespace cola {

// Shape of a tile in shared memory: NL lines, element (l, i) at
// l LSTR + spad(i) ES; LF: butterflies run over the lines first (consecutive
// threads take adjacent lines; NL a power of two), else along a line.  TWM is
// the twiddle table's stride: the table holds N TWM entries exp(-2 pi i q / (N TWM)).
// TWO: the passes read a pass-ordered twiddle table (see ordered_twiddles)
// instead of that table: with butterflies along a line, neighbouring threads
// have consecutive k, and W^{r k} read at stride r k N / (LS R) would hit the
// same shared-memory banks.  WARP: the tile belongs to one warp (thread index
// = lane, passes separated by __syncwarp), so warps transform their own lines
// without waiting for the rest of the block.
template <int NL_, bool LF_, int LSTR_, int ES_, int TWM_, bool TWO_ = false, bool WARP_ = false>
struct TileGeo {
    static constexpr int NL = NL_;
    static constexpr bool LF = LF_;
    static constexpr int LSTR = LSTR_;
    static constexpr int ES = ES_;
    static constexpr int TWM = TWM_;
    static constexpr bool TWO = TWO_;
    static constexpr bool WARP = WARP_;
};
// the thread's index in the group that owns a tile, and that group's barrier
template <class Geo>
__device__ __forceinline__ unsigned geo_tid() {
    if constexpr (Geo::WARP)
        return threadIdx.x & 31u;
    else
        return threadIdx.x;
}
template <class Geo>
__device__ __forceinline__ void geo_sync() {
    if constexpr (Geo::WARP)
        __syncwarp();
    else
        __syncthreads();
}
// B interleaved columns (strided y/x passes)
template <int B>
using ColTile = TileGeo<B, true, 1, B, 1>;
// NR rows of the half-length complex transform of real rows of 2M values (z passes)
template <int M, int NR>
using RowTile = TileGeo<NR, false, spad(M) + 1, 1, 2, true>;
// one such row owned by one warp
template <int M>
using WarpRow = TileGeo<1, false, spad(M) + 1, 1, 2, true, true>;

// Pass-ordered twiddles: pass s (LS = product of the earlier radices, radix R)
// reads W_{LS R}^{r k} at offset tw_offset(P, s) + (r - 1) LS + k, so that
// consecutive k are consecutive entries.
__host__ __device__ constexpr int tw_offset(const StaticPlan& p, int s) {
    int off = 0, ls = p.r[0];
    for (int q = 1; q < s; ++q) {
        off += (p.r[q] - 1) * ls;
        ls *= p.r[q];
    }
    return off;
}
__host__ __device__ constexpr bool same_plan(const StaticPlan& a, const StaticPlan& b) {
    if (a.nr != b.nr) return false;
    for (int i = 0; i < a.nr; ++i)
        if (a.r[i] != b.r[i]) return false;
    return true;
}
// Fill the pass-ordered table of an N-point plan in shared memory from the
// table tw of N TWM entries exp(-2 pi i q / (N TWM)) (the same values).
template <int N, int T, int TWM>
__device__ __forceinline__ void ordered_twiddles(float2* out, const float2* __restrict__ tw) {
    constexpr StaticPlan P = static_plan(N);
    int ls = P.r[0], off = 0;
    for (int s = 1; s < P.nr; ++s) {
        const int R = P.r[s], tws = N / (ls * R) * TWM;
        for (int q = threadIdx.x; q < (R - 1) * ls; q += T) {
            const int r = q / ls + 1, k = q - (r - 1) * ls;
            out[off + q] = __ldg(tw + r * k * tws);
        }
        off += (R - 1) * ls;
        ls *= R;
    }
}

template <class Geo>
struct SSmem {
    float2* p;
    template <int R, int D>
    __device__ __forceinline__ void load(int l, int i0, float2* v) const {
        if constexpr (D % 16 == 0) {
            const float2* q = p + l * Geo::LSTR + spad(i0) * Geo::ES;
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = q[r * spad(D) * Geo::ES];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = p[l * Geo::LSTR + spad(i0 + r * D) * Geo::ES];
        }
    }
    // stores come from butterflies with i0 = jq LS R + k: for LS = D = 1 the
    // group i0 .. i0 + R - 1 starts at a multiple of R, which with R | 16 never
    // crosses a padding slot
    template <int R, int D>
    __device__ __forceinline__ void store(int l, int i0, const float2* v) const {
        if constexpr (D % 16 == 0 || (D == 1 && 16 % R == 0)) {
            float2* q = p + l * Geo::LSTR + spad(i0) * Geo::ES;
#pragma unroll
            for (int r = 0; r < R; ++r) q[r * spad(D) * Geo::ES] = v[r];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) p[l * Geo::LSTR + spad(i0 + r * D) * Geo::ES] = v[r];
        }
    }
};

// One Stockham pass of radix R over a tile of Geo::NL lines of length N (see
// fft_pass for the index map): butterfly b = (j, l), j < N / R, k = j mod LS,
//   v_r = in(l, j + r N/R) W_{LS R}^{r k},  v = DFT_R(v),  out(l, (j / LS) LS R + k + r LS) = v_r.
template <int N, int T, class Geo, int R, int LS, int SIGN, class In, class Out>
__device__ __forceinline__ void spass(const In& in, const Out& out, const float2* __restrict__ tw) {
    constexpr int NBL = N / R;
    constexpr int NB = NBL * Geo::NL;
    constexpr int IT = (NB + T - 1) / T;
    constexpr int TWS = N / (LS * R) * Geo::TWM;
#pragma unroll
    for (int it = 0; it < IT; ++it) {
        const unsigned b = geo_tid<Geo>() + (unsigned)(it * T);
        if (NB % T != 0 && it == IT - 1 && b >= (unsigned)NB) break;
        int l, j;
        if constexpr (Geo::LF) {
            l = (int)(b % Geo::NL);
            j = (int)(b / Geo::NL);
        } else {
            l = (int)(b / NBL);
            j = (int)(b - (unsigned)l * NBL);
        }
        const int jq = (int)((unsigned)j / LS);
        const int k = j - jq * LS;
        float2 v[R];
        in.template load<R, NBL>(l, j, v);
        if constexpr (LS > 1) {
            const int step = k * TWS;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = Geo::TWO ? tw[(r - 1) * LS + k] : tw[r * step];
                if (SIGN > 0) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        SmallDft<R>::run(v, SIGN);
        out.template store<R, LS>(l, jq * LS * R + k, v);
    }
}

// passes S .. nr-1: S reads a; the last pass writes `out`
template <int N, int T, class Geo, int SIGN, int S, class Out>
__device__ __forceinline__ void srun_tail(float2* a, float2* b, const Out& out, const float2* __restrict__ tw) {
    constexpr StaticPlan P = static_plan(N);
    constexpr int R = P.r[S];
    constexpr int LS = plan_ls(P, S);
    const float2* twp = Geo::TWO ? tw + tw_offset(P, S) : tw;
    if constexpr (S == P.nr - 1) {
        spass<N, T, Geo, R, LS, SIGN>(SSmem<Geo>{a}, out, twp);
        geo_sync<Geo>();
    } else {
        spass<N, T, Geo, R, LS, SIGN>(SSmem<Geo>{a}, SSmem<Geo>{b}, twp);
        geo_sync<Geo>();
        srun_tail<N, T, Geo, SIGN, S + 1>(b, a, out, tw);
    }
}

// Transform reading `in` in the first pass (into a), then `hook` (uniform:
// the input is no longer needed), the middle passes ping-pong a/b, the last
// pass writes `out`.  Needs at least two passes.  Returns synchronised.
template <int N, int T, class Geo, int SIGN, class In, class Out, class Hook>
__device__ __forceinline__ void srun_out(const In& in, const Out& out, float2* a, float2* b,
                                         const float2* __restrict__ tw, const Hook& hook) {
    constexpr StaticPlan P = static_plan(N);
    static_assert(P.ok && P.nr >= 2, "specialised transforms need two or more passes");
    spass<N, T, Geo, P.r[0], 1, SIGN>(in, SSmem<Geo>{a}, tw);
    geo_sync<Geo>();
    hook();
    srun_tail<N, T, Geo, SIGN, 1>(a, b, out, tw);
}

// Same, with the result left in shared memory; returns the buffer holding it.
template <int N, int T, class Geo, int SIGN, class In, class Hook>
__device__ __forceinline__ float2* srun_smem(const In& in, float2* a, float2* b, const float2* __restrict__ tw,
                                             const Hook& hook) {
    constexpr StaticPlan P = static_plan(N);
    float2* res = ((P.nr - 1) % 2 == 1) ? b : a;
    srun_out<N, T, Geo, SIGN>(in, SSmem<Geo>{res}, a, b, tw, hook);
    return res;
}

// Radix order of a transform: the default plan of N, or three given radices.
// Any order computes the same transform (the Stockham passes accumulate LS);
// orders are chosen so that the in-place passes hold few values per thread.
template <int N, int R0 = 0, int R1 = 0, int R2 = 0>
struct PlanOf {
    static constexpr StaticPlan P = R0 ? StaticPlan{true, 3, {R0, R1, R2}} : static_plan(N);
    static_assert(R0 == 0 || R0 * R1 * R2 == N, "radices must multiply to N");
};

// In-place pass: every butterfly of the thread is loaded into registers, the
// block synchronises, then the butterflies are computed and stored over the
// same buffer.  A tile then needs one working buffer instead of a ping-pong
// pair; the registers hold N NL / T values per thread.
template <int N, int T, class Geo, int R, int LS, int SIGN, class In, class Out>
__device__ __forceinline__ void spass_ip(const In& in, const Out& out, const float2* __restrict__ tw) {
    constexpr int NBL = N / R;
    constexpr int NB = NBL * Geo::NL;
    constexpr int IT = (NB + T - 1) / T;
    constexpr int TWS = N / (LS * R) * Geo::TWM;
    float2 v[IT][R];
    auto coords = [](unsigned b, int& l, int& j) {
        if constexpr (Geo::LF) {
            l = (int)(b % Geo::NL);
            j = (int)(b / Geo::NL);
        } else {
            l = (int)(b / NBL);
            j = (int)(b - (unsigned)l * NBL);
        }
    };
#pragma unroll
    for (int it = 0; it < IT; ++it) {
        const unsigned b = geo_tid<Geo>() + (unsigned)(it * T);
        if (NB % T == 0 || it < IT - 1 || b < (unsigned)NB) {
            int l, j;
            coords(b, l, j);
            in.template load<R, NBL>(l, j, v[it]);
        }
    }
    geo_sync<Geo>();
#pragma unroll
    for (int it = 0; it < IT; ++it) {
        const unsigned b = geo_tid<Geo>() + (unsigned)(it * T);
        if (NB % T != 0 && it == IT - 1 && b >= (unsigned)NB) break;
        int l, j;
        coords(b, l, j);
        const int jq = (int)((unsigned)j / LS);
        const int k = j - jq * LS;
        if constexpr (LS > 1) {
            const int step = k * TWS;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = Geo::TWO ? tw[(r - 1) * LS + k] : tw[r * step];
                if (SIGN > 0) w.y = -w.y;
                v[it][r] = cmul(v[it][r], w);
            }
        }
        SmallDft<R>::run(v[it], SIGN);
        out.template store<R, LS>(l, jq * LS * R + k, v[it]);
    }
}

// passes S .. nr-1 in the single buffer a: in place, the last one into `out`
// (in place as well when LAST_IP, i.e. `out` is a itself)
template <int N, int T, class Geo, int SIGN, int S, bool LAST_IP, class PL, class Out>
__device__ __forceinline__ void sip_tail(float2* a, const Out& out, const float2* __restrict__ tw) {
    constexpr StaticPlan P = PL::P;
    constexpr int R = P.r[S];
    constexpr int LS = plan_ls(P, S);
    static_assert(!Geo::TWO || same_plan(P, static_plan(N)), "pass-ordered twiddles are laid out for the default plan");
    const float2* twp = Geo::TWO ? tw + tw_offset(P, S) : tw;
    if constexpr (S == P.nr - 1) {
        if constexpr (LAST_IP)
            spass_ip<N, T, Geo, R, LS, SIGN>(SSmem<Geo>{a}, out, twp);
        else
            spass<N, T, Geo, R, LS, SIGN>(SSmem<Geo>{a}, out, twp);
        geo_sync<Geo>();
    } else {
        spass_ip<N, T, Geo, R, LS, SIGN>(SSmem<Geo>{a}, SSmem<Geo>{a}, twp);
        geo_sync<Geo>();
        sip_tail<N, T, Geo, SIGN, S + 1, LAST_IP, PL>(a, out, tw);
    }
}

// Transform with one working buffer a: the first pass reads `in` (another
// buffer, or a itself when FIRST_IP) into a, then `hook`, the other passes run
// in place and the last writes `out` (a itself when LAST_IP).  Returns
// synchronised.
template <int N, int T, class Geo, int SIGN, bool FIRST_IP, bool LAST_IP, class PL = PlanOf<N>, class In, class Out,
          class Hook>
__device__ __forceinline__ void sip_run(const In& in, const Out& out, float2* a, const float2* __restrict__ tw,
                                        const Hook& hook) {
    constexpr StaticPlan P = PL::P;
    static_assert(P.ok && P.nr >= 2, "specialised transforms need two or more passes");
    if constexpr (FIRST_IP)
        spass_ip<N, T, Geo, P.r[0], 1, SIGN>(in, SSmem<Geo>{a}, tw);
    else
        spass<N, T, Geo, P.r[0], 1, SIGN>(in, SSmem<Geo>{a}, tw);
    geo_sync<Geo>();
    hook();
    sip_tail<N, T, Geo, SIGN, 1, LAST_IP, PL>(a, out, tw);
}

// Stage an N x B tile (row i at g + i S, B adjacent complex columns) into the
// padded layout, 16 bytes per cp.async.
template <int N, int B, int T, class Off>
__device__ __forceinline__ void stile_prefetch(float2* stg, const float2* g, const Off& off) {
    constexpr int HB = B / 2;
    constexpr int NE = N * HB;
#pragma unroll 4
    for (int e = threadIdx.x; e < NE; e += T) {
        const int i = e / HB, c = (e % HB) * 2;
        cp_async16(stg + c + spad(i) * B, g + off(i) + c);
    }
    cp_async_commit();
}

// global column tile: element i of line l at g + i S + l
struct SCol {
    float2* g;
    long long S;
    __device__ __forceinline__ long long operator()(int i) const { return (long long)i * S; }
    template <int R, int D>
    __device__ __forceinline__ void store(int l, int i0, const float2* v) const {
        float2* q = g + (long long)i0 * S + l;
        const long long st = (long long)D * S;
#pragma unroll
        for (int r = 0; r < R; ++r) __stcs(q + r * st, v[r]);
    }
};

// Geometry of the interleaved, x-blocked force mesh of an N^3 grid: rows
// ((x / XB) N + y) XB + x mod XB of 3 component rows of P complex each.
template <int N>
struct XGeom {
    static constexpr int P = fft_pitch(N);
    static constexpr int XBS = xblock_shift(N);
    static constexpr int XB = 1 << XBS;
    static constexpr long long SB = 3ll * XB * N * P;  // between x blocks
    static constexpr long long SI = 3ll * P;           // within an x block
    static constexpr long long RS = 3ll * XB * P;      // between y rows
    __device__ __forceinline__ static long long off(int i) {
        return (long long)(i >> XBS) * SB + (long long)(i & (XB - 1)) * SI;
    }
};

template <int N>
struct XOff {
    __device__ __forceinline__ long long operator()(int i) const { return XGeom<N>::off(i); }
};

// x line of one component: element i of line l at g + off(i) + l
template <int N>
struct SXIO {
    float2* g;
    template <int R, int D>
    __device__ __forceinline__ void store(int l, int i0, const float2* v) const {
        using G = XGeom<N>;
        if constexpr (D % G::XB == 0) {
            float2* q = g + G::off(i0) + l;
#pragma unroll
            for (int r = 0; r < R; ++r) __stcs(q + (long long)r * (D / G::XB) * G::SB, v[r]);
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) __stcs(g + G::off(i0 + r * D) + l, v[r]);
        }
    }
};

// i k times a spectrum tile read from shared memory, k the wave number of the
// line index (0 on the Nyquist index): the x component of the force in the x
// pass (i k_x phi), the y component in the y pass (i k_y Psi)
template <int N, class Geo>
struct IkxLoad {
    float2* p;
    float kf;
    template <int R, int D>
    __device__ __forceinline__ void load(int l, int i0, float2* v) const {
        SSmem<Geo>{p}.template load<R, D>(l, i0, v);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = i0 + r * D;
            const float kx = (i == N / 2) ? 0.f : kf * (float)(i < N / 2 ? i : i - N);
            v[r] = make_float2(-kx * v[r].y, kx * v[r].x);
        }
    }
};

// Radix orders of the two-buffer fused pass's transforms (forward, F_x, Psi).
// In-place passes may hold at most N B / T values per thread; a radix whose
// butterflies do not spread evenly over the threads goes where its pass is out
// of place (the forward's and F_x's first pass, Psi's last).
template <int N>
struct GreenPlans {
    using F = PlanOf<N>;
    using I1 = PlanOf<N>;
    using I2 = PlanOf<N>;
};
template <>
struct GreenPlans<1536> {
    using F = PlanOf<1536, 12, 8, 16>;
    using I1 = PlanOf<1536, 12, 8, 16>;
    using I2 = PlanOf<1536, 16, 8, 12>;
};
template <>
struct GreenPlans<768> {
    using F = PlanOf<768, 12, 4, 16>;
    using I1 = PlanOf<768, 12, 4, 16>;
    using I2 = PlanOf<768, 16, 4, 12>;
};

// strided complex pass (y: S = row stride, outer = x; or x on a plain mesh):
// persistent blocks; the first pass reads the staged tile into the working
// buffer, after which the next tile is staged with cp.async while the other
// passes run in place
template <int N, int B, int T, int SIGN>
__global__ void __launch_bounds__(T, 1) k_fft_strided_s(float2* data, LineGeom lg, int nct, int ntiles,
                                                      const float2* __restrict__ tw) {
    using Geo = ColTile<B>;
    constexpr int TSZ = spad(N) * B;
    extern __shared__ float2 sm[];
    float2* stg = sm;
    float2* A = sm + TSZ;
    float2* tws = A + TSZ;
    for (int q = threadIdx.x; q < N; q += T) tws[q] = __ldg(tw + q);
    const SCol rows{nullptr, lg.S};
    auto tile_base = [&](int t) {
        const int o = t / nct;
        const int ct = t - o * nct;
        const int o1 = o / lg.o2n, o2 = o - o1 * lg.o2n;
        return data + o1 * lg.s1 + o2 * lg.s2 + ct * B;
    };
    int t = blockIdx.x;
    if (t < ntiles) stile_prefetch<N, B, T>(stg, tile_base(t), rows);
    for (; t < ntiles; t += gridDim.x) {
        cp_async_wait_all();
        __syncthreads();
        const int tn = t + gridDim.x;
        auto next = [&]() {
            if (tn < ntiles) stile_prefetch<N, B, T>(stg, tile_base(tn), rows);
        };
        sip_run<N, T, Geo, SIGN, false, false>(SSmem<Geo>{stg}, SCol{tile_base(t), lg.S}, A, tws, next);
    }
}

// x pass fused with the Poisson solve and the ik gradient on the interleaved,
// x-blocked force mesh (the runtime form is k_fft_x_green): forward x FFT of
// delta_k (component 0) from the staged tile into A, phi = gscale delta_k / k^2
// (times the radial filter if given) in place, F_x = IFFT_x(i k_x phi) worked
// in the staging buffer, then (the next tile staged meanwhile) Psi =
// IFFT_x(phi) in place in A, stored as F_y = i k_y Psi and F_z = i k_z Psi.
template <int N, int B, int T>
__global__ void __launch_bounds__(T, 1) k_fft_x_green_s(float2* F, int nct, int ntiles, const float2* __restrict__ tw,
                                                      float gscale, float kf, const float* __restrict__ filt,
                                                      int nfilt, float fstep) {
    using G = XGeom<N>;
    using Geo = ColTile<B>;
    constexpr int TSZ = spad(N) * B;
    constexpr int TB = T / B;    // line-element stride between a thread's spectrum values
    constexpr int EPT = N / TB;  // spectrum values per thread
    static_assert(T % B == 0 && N % TB == 0, "tile must split evenly over the block");
    constexpr int half = N / 2;
    extern __shared__ float2 sm[];
    float2* stg = sm;
    float2* A = sm + TSZ;
    float2* tws = A + TSZ;
    for (int q = threadIdx.x; q < N; q += T) tws[q] = __ldg(tw + q);
    const int c = threadIdx.x % B;   // this thread's column in the Green phase
    const int i0 = threadIdx.x / B;  // and its first line element: i = i0 + q TB
    auto elem = [&](float2* base, int q) -> float2& {
        if constexpr (TB % 16 == 0)
            return base[c + spad(i0) * B + q * spad(TB) * B];
        else
            return base[c + spad(i0 + q * TB) * B];
    };
    auto tile_off = [&](int t) {
        const int iy = t / nct;
        return (long long)iy * G::RS + (long long)(t - iy * nct) * B;
    };
    const XOff<N> xo{};
    int t = blockIdx.x;
    if (t < ntiles) stile_prefetch<N, B, T>(stg, F + tile_off(t), xo);
    for (; t < ntiles; t += gridDim.x) {
        const int iy = t / nct;
        const int col0 = (t - iy * nct) * B;
        const long long off = (long long)iy * G::RS + col0;
        cp_async_wait_all();
        __syncthreads();
        sip_run<N, T, Geo, -1, false, true, typename GreenPlans<N>::F>(SSmem<Geo>{stg}, SSmem<Geo>{A}, A, tws,
                                                                      NoHook{});
        const float ky = kf * (float)(iy < half ? iy : iy - N);
        const float kz = kf * (float)(col0 + c);
        const float kyz2 = ky * ky + kz * kz;
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            const int i = i0 + q * TB;
            const float kx = kf * (float)(i < half ? i : i - N);
            const float k2 = kx * kx + kyz2;
            float gk = k2 > 0.f ? gscale / k2 : 0.f;
            if (filt) {
                // radial transfer T(|k|), piecewise linear on nodes b * fstep
                const float u = sqrtf(k2) / fstep;
                int b = (int)u;
                if (b > nfilt - 2) b = nfilt - 2;
                const float f = fminf(u - (float)b, 1.f);
                gk *= (1.f - f) * filt[b] + f * filt[b + 1];
            }
            float2& x = elem(A, q);
            x = cscale(x, gk);
        }
        __syncthreads();
        sip_run<N, T, Geo, +1, false, false, typename GreenPlans<N>::I1>(IkxLoad<N, Geo>{A, kf}, SXIO<N>{F + off}, stg,
                                                                         tws, NoHook{});
        const int tn = t + gridDim.x;
        if (tn < ntiles) stile_prefetch<N, B, T>(stg, F + tile_off(tn), xo);
        sip_run<N, T, Geo, +1, true, false, typename GreenPlans<N>::I2>(SSmem<Geo>{A}, SXIO<N>{F + off + G::P}, A,
                                                                        tws, NoHook{});
    }
}

// The same fused pass with three tile buffers (staging + ping-pong) and phi
// kept in registers: the next tile is staged during all three transforms, at
// the cost of half the columns per tile of the two-buffer form.
template <int N, int B, int T>
__global__ void __launch_bounds__(T, 1) k_fft_x_green3_s(float2* F, int nct, int ntiles, const float2* __restrict__ tw,
                                                      float gscale, float kf, const float* __restrict__ filt,
                                                      int nfilt, float fstep) {
    using G = XGeom<N>;
    constexpr int TSZ = spad(N) * B;
    constexpr int TB = T / B;    // line-element stride between a thread's spectrum values
    constexpr int EPT = N / TB;  // spectrum values per thread
    static_assert(T % B == 0 && N % TB == 0, "tile must split evenly over the block");
    constexpr int half = N / 2;
    extern __shared__ float2 sm[];
    float2* stg = sm;
    float2* A = sm + TSZ;
    float2* W = A + TSZ;
    float2* tws = W + TSZ;
    for (int q = threadIdx.x; q < N; q += T) tws[q] = __ldg(tw + q);
    const int c = threadIdx.x % B;   // this thread's column in the Green phase
    const int i0 = threadIdx.x / B;  // and its first line element: i = i0 + q TB
    auto elem = [&](float2* base, int q) -> float2& {
        if constexpr (TB % 16 == 0)
            return base[c + spad(i0) * B + q * spad(TB) * B];
        else
            return base[c + spad(i0 + q * TB) * B];
    };
    auto tile_off = [&](int t) {
        const int iy = t / nct;
        return (long long)iy * G::RS + (long long)(t - iy * nct) * B;
    };
    const XOff<N> xo{};
    int t = blockIdx.x;
    if (t < ntiles) stile_prefetch<N, B, T>(stg, F + tile_off(t), xo);
    for (; t < ntiles; t += gridDim.x) {
        const int iy = t / nct;
        const int col0 = (t - iy * nct) * B;
        const long long off = (long long)iy * G::RS + col0;
        cp_async_wait_all();
        __syncthreads();
        const int tn = t + gridDim.x;
        auto next = [&]() {
            if (tn < ntiles) stile_prefetch<N, B, T>(stg, F + tile_off(tn), xo);
        };
        float2* X = srun_smem<N, T, ColTile<B>, -1>(SSmem<ColTile<B>>{stg}, A, W, tws, next);
        const float ky = kf * (float)(iy < half ? iy : iy - N);
        const float kz = kf * (float)(col0 + c);
        const float kyz2 = ky * ky + kz * kz;
        float2 phi[EPT];
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            const int i = i0 + q * TB;
            const float kx = kf * (float)(i < half ? i : i - N);
            const float k2 = kx * kx + kyz2;
            float gk = k2 > 0.f ? gscale / k2 : 0.f;
            if (filt) {
                // radial transfer T(|k|), piecewise linear on nodes b * fstep
                const float u = sqrtf(k2) / fstep;
                int b = (int)u;
                if (b > nfilt - 2) b = nfilt - 2;
                const float f = fminf(u - (float)b, 1.f);
                gk *= (1.f - f) * filt[b] + f * filt[b + 1];
            }
            phi[q] = cscale(elem(X, q), gk);
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            const int i = i0 + q * TB;
            const float kx = (i == half) ? 0.f : kf * (float)(i < half ? i : i - N);
            elem(A, q) = make_float2(-kx * phi[q].y, kx * phi[q].x);  // i k_x phi
        }
        __syncthreads();
        srun_out<N, T, ColTile<B>, +1>(SSmem<ColTile<B>>{A}, SXIO<N>{F + off}, W, A, tws, NoHook{});
#pragma unroll
        for (int q = 0; q < EPT; ++q) elem(A, q) = phi[q];
        __syncthreads();
        srun_out<N, T, ColTile<B>, +1>(SSmem<ColTile<B>>{A}, SXIO<N>{F + off + G::P}, W, A, tws, NoHook{});
    }
}

// global column tile written as i k_z times the values, k_z the wave number of
// the tile's column (0 on the Nyquist column n/2)
struct SColIkz {
    float2* g;
    long long S;
    float kf;
    int col0, half;
    template <int R, int D>
    __device__ __forceinline__ void store(int l, int i0, const float2* v) const {
        const float kz = (col0 + l == half) ? 0.f : kf * (float)(col0 + l);
        float2* q = g + (long long)i0 * S + l;
        const long long st = (long long)D * S;
#pragma unroll
        for (int r = 0; r < R; ++r) __stcs(q + r * st, make_float2(-kz * v[r].y, kz * v[r].x));
    }
};

// Inverse y pass of the force mesh's second component, which the fused x pass
// leaves as Psi = IFFT_x(phi) (the x transform of the potential): one staged
// tile of Psi gives F_y = IFFT_y(i k_y Psi) (k_y varies along the y line) into
// component 1 and F_z = i k_z IFFT_y(Psi) (k_z is the column's, constant along
// the line) into component 2.  lg addresses component 1; component 2 follows
// at + comp2.
template <int N, int B, int T>
__global__ void __launch_bounds__(T, 1) k_fft_y_psi_s(float2* data, LineGeom lg, long long comp2, int nct, int ntiles,
                                                       const float2* __restrict__ tw, float kf) {
    using Geo = ColTile<B>;
    constexpr int TSZ = spad(N) * B;
    extern __shared__ float2 sm[];
    float2* stg = sm;
    float2* A = sm + TSZ;
    float2* tws = A + TSZ;
    for (int q = threadIdx.x; q < N; q += T) tws[q] = __ldg(tw + q);
    const SCol rows{nullptr, lg.S};
    auto tile_base = [&](int t) {
        const int o = t / nct;
        const int ct = t - o * nct;
        const int o1 = o / lg.o2n, o2 = o - o1 * lg.o2n;
        return data + o1 * lg.s1 + o2 * lg.s2 + ct * B;
    };
    int t = blockIdx.x;
    if (t < ntiles) stile_prefetch<N, B, T>(stg, tile_base(t), rows);
    for (; t < ntiles; t += gridDim.x) {
        cp_async_wait_all();
        __syncthreads();
        float2* base = tile_base(t);
        const int col0 = (t - (t / nct) * nct) * B;
        sip_run<N, T, Geo, +1, false, false>(IkxLoad<N, Geo>{stg, kf}, SCol{base, lg.S}, A, tws, NoHook{});
        const int tn = t + gridDim.x;
        auto next = [&]() {
            if (tn < ntiles) stile_prefetch<N, B, T>(stg, tile_base(tn), rows);
        };
        sip_run<N, T, Geo, +1, false, false>(SSmem<Geo>{stg}, SColIkz{base + comp2, lg.S, kf, col0, N / 2}, A, tws,
                                             next);
    }
}

// ---------------------------------------------------------------------------
// Column tiles with two lines per thread.  The tile is the ColTile layout (B
// interleaved lines, element (l, i) at l + spad(i) B); a butterfly is taken for
// the adjacent lines 2 l2 and 2 l2 + 1 at once: one 16-byte shared-memory
// access per element pair and one twiddle for both, so a pass issues about
// half the memory, twiddle and index instructions of the one-line form for
// the same arithmetic.
// ---------------------------------------------------------------------------
template <int B>
struct S2Smem {
    float2* p;
    __device__ __forceinline__ float4* at(int l2, int i) const {
        return reinterpret_cast<float4*>(p + 2 * l2 + spad(i) * B);
    }
    template <int R, int D>
    __device__ __forceinline__ void load(int l2, int i0, float2* v0, float2* v1) const {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float4 q = (D % 16 == 0) ? at(l2, i0)[r * (spad(D) * B / 2)] : *at(l2, i0 + r * D);
            v0[r] = make_float2(q.x, q.y);
            v1[r] = make_float2(q.z, q.w);
        }
    }
    template <int R, int D>
    __device__ __forceinline__ void store(int l2, int i0, const float2* v0, const float2* v1) const {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float4 q = make_float4(v0[r].x, v0[r].y, v1[r].x, v1[r].y);
            if constexpr (D % 16 == 0 || (D == 1 && 16 % R == 0))
                at(l2, i0)[r * (spad(D) * B / 2)] = q;
            else
                *at(l2, i0 + r * D) = q;
        }
    }
};

// global column tile, two lines at a time: element i of line l at g + i S + l
struct SCol2 {
    float2* g;
    long long S;
    template <int R, int D>
    __device__ __forceinline__ void store(int l2, int i0, const float2* v0, const float2* v1) const {
        float2* q = g + (long long)i0 * S + 2 * l2;
        const long long st = (long long)D * S;
#pragma unroll
        for (int r = 0; r < R; ++r)
            __stcs(reinterpret_cast<float4*>(q + r * st), make_float4(v0[r].x, v0[r].y, v1[r].x, v1[r].y));
    }
};

// One Stockham pass of radix R over the line pairs of a B-line tile (see
// spass); butterfly b = (j, l2), consecutive threads take adjacent pairs.
template <int N, int T, int B, int R, int LS, int SIGN, bool IP, class In, class Out>
__device__ __forceinline__ void spass2(const In& in, const Out& out, const float2* __restrict__ tw) {
    constexpr int NP = B / 2;
    constexpr int NBL = N / R;
    constexpr int NB = NBL * NP;
    constexpr int IT = (NB + T - 1) / T;
    constexpr int TWS = N / (LS * R);
    constexpr int ITL = IP ? IT : 1;  // butterflies held at once
    float2 v0[ITL][R], v1[ITL][R];
    if constexpr (IP) {
#pragma unroll
        for (int it = 0; it < IT; ++it) {
            const unsigned b = threadIdx.x + (unsigned)(it * T);
            if (NB % T == 0 || it < IT - 1 || b < (unsigned)NB)
                in.template load<R, NBL>((int)(b % NP), (int)(b / NP), v0[it], v1[it]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int it = 0; it < IT; ++it) {
        const unsigned b = threadIdx.x + (unsigned)(it * T);
        if (NB % T != 0 && it == IT - 1 && b >= (unsigned)NB) break;
        const int l2 = (int)(b % NP), j = (int)(b / NP);
        const int jq = (int)((unsigned)j / LS);
        const int k = j - jq * LS;
        float2* a0 = v0[IP ? it : 0];
        float2* a1 = v1[IP ? it : 0];
        if constexpr (!IP) in.template load<R, NBL>(l2, j, a0, a1);
        if constexpr (LS > 1) {
            const int step = k * TWS;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = tw[r * step];
                if (SIGN > 0) w.y = -w.y;
                a0[r] = cmul(a0[r], w);
                a1[r] = cmul(a1[r], w);
            }
        }
        SmallDft<R>::run(a0, SIGN);
        SmallDft<R>::run(a1, SIGN);
        out.template store<R, LS>(l2, jq * LS * R + k, a0, a1);
    }
}

// passes S .. nr-1 in buffer a: in place, the last one into `out` (in place
// as well when LAST_IP, i.e. `out` is a itself)
template <int N, int T, int B, int SIGN, int S, bool LAST_IP, class PL, class Out>
__device__ __forceinline__ void sip2_tail(float2* a, const Out& out, const float2* __restrict__ tw) {
    constexpr StaticPlan P = PL::P;
    constexpr int R = P.r[S];
    constexpr int LS = plan_ls(P, S);
    if constexpr (S == P.nr - 1) {
        spass2<N, T, B, R, LS, SIGN, LAST_IP>(S2Smem<B>{a}, out, tw);
        __syncthreads();
    } else {
        spass2<N, T, B, R, LS, SIGN, true>(S2Smem<B>{a}, S2Smem<B>{a}, tw);
        __syncthreads();
        sip2_tail<N, T, B, SIGN, S + 1, LAST_IP, PL>(a, out, tw);
    }
}

// Transform of a B-line tile two lines per thread: the first pass reads `in`
// (another buffer, or a itself when FIRST_IP) into a, then `hook`, the middle
// passes run in place, the last writes `out` (a itself when LAST_IP).
// Returns synchronised.
template <int N, int T, int B, int SIGN, bool FIRST_IP = false, bool LAST_IP = false, class PL = PlanOf<N>, class In,
          class Out, class Hook>
__device__ __forceinline__ void sip2_run(const In& in, const Out& out, float2* a, const float2* __restrict__ tw,
                                         const Hook& hook) {
    constexpr StaticPlan P = PL::P;
    static_assert(P.ok && P.nr >= 2 && B % 2 == 0, "two or more passes, line pairs");
    spass2<N, T, B, P.r[0], 1, SIGN, FIRST_IP>(in, S2Smem<B>{a}, tw);
    __syncthreads();
    hook();
    sip2_tail<N, T, B, SIGN, 1, LAST_IP, PL>(a, out, tw);
}

// the two-lines-per-thread forms of IkxLoad and SColIkz
template <int N, int B>
struct Ikx2Load {
    float2* p;
    float kf;
    template <int R, int D>
    __device__ __forceinline__ void load(int l2, int i0, float2* v0, float2* v1) const {
        S2Smem<B>{p}.template load<R, D>(l2, i0, v0, v1);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = i0 + r * D;
            const float kx = (i == N / 2) ? 0.f : kf * (float)(i < N / 2 ? i : i - N);
            v0[r] = make_float2(-kx * v0[r].y, kx * v0[r].x);
            v1[r] = make_float2(-kx * v1[r].y, kx * v1[r].x);
        }
    }
};

struct SCol2Ikz {
    float2* g;
    long long S;
    float kf;
    int col0, half;
    template <int R, int D>
    __device__ __forceinline__ void store(int l2, int i0, const float2* v0, const float2* v1) const {
        const int c = col0 + 2 * l2;
        const float k0 = (c == half) ? 0.f : kf * (float)c;
        const float k1 = (c + 1 == half) ? 0.f : kf * (float)(c + 1);
        float2* q = g + (long long)i0 * S + 2 * l2;
        const long long st = (long long)D * S;
#pragma unroll
        for (int r = 0; r < R; ++r)
            __stcs(reinterpret_cast<float4*>(q + r * st),
                   make_float4(-k0 * v0[r].y, k0 * v0[r].x, -k1 * v1[r].y, k1 * v1[r].x));
    }
};

// k_fft_y_psi_s with two lines per thread
template <int N, int B, int T>
__global__ void __launch_bounds__(T, 1) k_fft_y_psi2_s(float2* data, LineGeom lg, long long comp2, int nct,
                                                        int ntiles, const float2* __restrict__ tw, float kf) {
    constexpr int TSZ = spad(N) * B;
    extern __shared__ float2 sm[];
    float2* stg = sm;
    float2* A = sm + TSZ;
    float2* tws = A + TSZ;
    for (int q = threadIdx.x; q < N; q += T) tws[q] = __ldg(tw + q);
    const SCol rows{nullptr, lg.S};
    auto tile_base = [&](int t) {
        const int o = t / nct;
        const int ct = t - o * nct;
        const int o1 = o / lg.o2n, o2 = o - o1 * lg.o2n;
        return data + o1 * lg.s1 + o2 * lg.s2 + ct * B;
    };
    int t = blockIdx.x;
    if (t < ntiles) stile_prefetch<N, B, T>(stg, tile_base(t), rows);
    for (; t < ntiles; t += gridDim.x) {
        cp_async_wait_all();
        __syncthreads();
        float2* base = tile_base(t);
        const int col0 = (t - (t / nct) * nct) * B;
        sip2_run<N, T, B, +1>(Ikx2Load<N, B>{stg, kf}, SCol2{base, lg.S}, A, tws, NoHook{});
        const int tn = t + gridDim.x;
        auto next = [&]() {
            if (tn < ntiles) stile_prefetch<N, B, T>(stg, tile_base(tn), rows);
        };
        sip2_run<N, T, B, +1>(S2Smem<B>{stg}, SCol2Ikz{base + comp2, lg.S, kf, col0, N / 2}, A, tws, next);
    }
}

template <int N, int B, int T>
inline int run_y_psi2(float2* data, LineGeom lg, long long comp2, int nct, int ntiles, const float2* tw, float kf,
                      cudaStream_t s) {
    const size_t smem = ((size_t)2 * spad(N) * B + N) * 8;
    if (!set_smem((const void*)k_fft_y_psi2_s<N, B, T>, smem)) return COLA_ECUDA;
    k_fft_y_psi2_s<N, B, T><<<persistent_grid(smem, ntiles, 1), T, smem, s>>>(data, lg, comp2, nct, ntiles, tw, kf);
    return check_launch();
}

template <int N, int B, int T>
inline int run_y_psi(float2* data, LineGeom lg, long long comp2, int nct, int ntiles, const float2* tw, float kf,
                     cudaStream_t s) {
    const size_t smem = ((size_t)2 * spad(N) * B + N) * 8;
    if (!set_smem((const void*)k_fft_y_psi_s<N, B, T>, smem)) return COLA_ECUDA;
    k_fft_y_psi_s<N, B, T><<<persistent_grid(smem, ntiles), T, smem, s>>>(data, lg, comp2, nct, ntiles, tw, kf);
    return check_launch();
}

template <int N, int B, int T>
constexpr size_t line_pass_smem() {
    return ((size_t)2 * spad(N) * B + N) * 8;
}

template <int N, int B, int T>
inline int run_strided(float2* data, int sign, LineGeom lg, int nct, int ntiles, const float2* tw, cudaStream_t s) {
    constexpr size_t smem = line_pass_smem<N, B, T>();
    auto kern = sign < 0 ? k_fft_strided_s<N, B, T, -1> : k_fft_strided_s<N, B, T, +1>;
    if (!set_smem((const void*)kern, smem)) return COLA_ECUDA;
    kern<<<persistent_grid(smem, ntiles), T, smem, s>>>(data, lg, nct, ntiles, tw);
    return check_launch();
}

// k_fft_strided_s with two lines per thread
template <int N, int B, int T, int SIGN>
__global__ void __launch_bounds__(T, 1) k_fft_strided2_s(float2* data, LineGeom lg, int nct, int ntiles,
                                                       const float2* __restrict__ tw) {
    constexpr int TSZ = spad(N) * B;
    extern __shared__ float2 sm[];
    float2* stg = sm;
    float2* A = sm + TSZ;
    float2* tws = A + TSZ;
    for (int q = threadIdx.x; q < N; q += T) tws[q] = __ldg(tw + q);
    const SCol rows{nullptr, lg.S};
    auto tile_base = [&](int t) {
        const int o = t / nct;
        const int ct = t - o * nct;
        const int o1 = o / lg.o2n, o2 = o - o1 * lg.o2n;
        return data + o1 * lg.s1 + o2 * lg.s2 + ct * B;
    };
    int t = blockIdx.x;
    if (t < ntiles) stile_prefetch<N, B, T>(stg, tile_base(t), rows);
    for (; t < ntiles; t += gridDim.x) {
        cp_async_wait_all();
        __syncthreads();
        const int tn = t + gridDim.x;
        auto next = [&]() {
            if (tn < ntiles) stile_prefetch<N, B, T>(stg, tile_base(tn), rows);
        };
        sip2_run<N, T, B, SIGN>(S2Smem<B>{stg}, SCol2{tile_base(t), lg.S}, A, tws, next);
    }
}

template <int N, int B, int T>
inline int run_strided2(float2* data, int sign, LineGeom lg, int nct, int ntiles, const float2* tw, cudaStream_t s) {
    constexpr size_t smem = line_pass_smem<N, B, T>();
    auto kern = sign < 0 ? k_fft_strided2_s<N, B, T, -1> : k_fft_strided2_s<N, B, T, +1>;
    if (!set_smem((const void*)kern, smem)) return COLA_ECUDA;
    kern<<<persistent_grid(smem, ntiles, 1), T, smem, s>>>(data, lg, nct, ntiles, tw);
    return check_launch();
}

// x line of one component, two lines at a time (SXIO)
template <int N>
struct SX2IO {
    float2* g;
    template <int R, int D>
    __device__ __forceinline__ void store(int l2, int i0, const float2* v0, const float2* v1) const {
        using G = XGeom<N>;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const long long o = (D % G::XB == 0) ? G::off(i0) + (long long)r * (D / G::XB) * G::SB : G::off(i0 + r * D);
            __stcs(reinterpret_cast<float4*>(g + o + 2 * l2), make_float4(v0[r].x, v0[r].y, v1[r].x, v1[r].y));
        }
    }
};

// k_fft_x_green_s with two lines per thread in its transforms
template <int N, int B, int T>
__global__ void __launch_bounds__(T, 1) k_fft_x_green2_s(float2* F, int nct, int ntiles, const float2* __restrict__ tw,
                                                       float gscale, float kf, const float* __restrict__ filt,
                                                       int nfilt, float fstep) {
    using G = XGeom<N>;
    constexpr int TSZ = spad(N) * B;
    constexpr int TB = T / B;    // line-element stride between a thread's spectrum values
    constexpr int EPT = N / TB;  // spectrum values per thread
    static_assert(T % B == 0 && N % TB == 0, "tile must split evenly over the block");
    constexpr int half = N / 2;
    extern __shared__ float2 sm[];
    float2* stg = sm;
    float2* A = sm + TSZ;
    float2* tws = A + TSZ;
    for (int q = threadIdx.x; q < N; q += T) tws[q] = __ldg(tw + q);
    const int c = threadIdx.x % B;   // this thread's column in the Green phase
    const int i0 = threadIdx.x / B;  // and its first line element: i = i0 + q TB
    auto elem = [&](float2* base, int q) -> float2& {
        if constexpr (TB % 16 == 0)
            return base[c + spad(i0) * B + q * spad(TB) * B];
        else
            return base[c + spad(i0 + q * TB) * B];
    };
    auto tile_off = [&](int t) {
        const int iy = t / nct;
        return (long long)iy * G::RS + (long long)(t - iy * nct) * B;
    };
    const XOff<N> xo{};
    int t = blockIdx.x;
    if (t < ntiles) stile_prefetch<N, B, T>(stg, F + tile_off(t), xo);
    for (; t < ntiles; t += gridDim.x) {
        const int iy = t / nct;
        const int col0 = (t - iy * nct) * B;
        const long long off = (long long)iy * G::RS + col0;
        cp_async_wait_all();
        __syncthreads();
        sip2_run<N, T, B, -1, false, true, typename GreenPlans<N>::F>(S2Smem<B>{stg}, S2Smem<B>{A}, A, tws, NoHook{});
        const float ky = kf * (float)(iy < half ? iy : iy - N);
        const float kz = kf * (float)(col0 + c);
        const float kyz2 = ky * ky + kz * kz;
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            const int i = i0 + q * TB;
            const float kx = kf * (float)(i < half ? i : i - N);
            const float k2 = kx * kx + kyz2;
            float gk = k2 > 0.f ? gscale / k2 : 0.f;
            if (filt) {
                // radial transfer T(|k|), piecewise linear on nodes b * fstep
                const float u = sqrtf(k2) / fstep;
                int b = (int)u;
                if (b > nfilt - 2) b = nfilt - 2;
                const float f = fminf(u - (float)b, 1.f);
                gk *= (1.f - f) * filt[b] + f * filt[b + 1];
            }
            float2& x = elem(A, q);
            x = cscale(x, gk);
        }
        __syncthreads();
        sip2_run<N, T, B, +1, false, false, typename GreenPlans<N>::I1>(Ikx2Load<N, B>{A, kf}, SX2IO<N>{F + off}, stg,
                                                                        tws, NoHook{});
        const int tn = t + gridDim.x;
        if (tn < ntiles) stile_prefetch<N, B, T>(stg, F + tile_off(tn), xo);
        sip2_run<N, T, B, +1, true, false, typename GreenPlans<N>::I2>(S2Smem<B>{A}, SX2IO<N>{F + off + G::P}, A,
                                                                       tws, NoHook{});
    }
}

template <int N, int B, int T>
inline int run_x_green2(float2* F, int nct, int ntiles, const float2* tw, float gscale, float kf, const float* filt,
                        int nfilt, float fstep, cudaStream_t s) {
    constexpr size_t smem = ((size_t)2 * spad(N) * B + N) * 8;
    if (!set_smem((const void*)k_fft_x_green2_s<N, B, T>, smem)) return COLA_ECUDA;
    k_fft_x_green2_s<N, B, T><<<persistent_grid(smem, ntiles, 1), T, smem, s>>>(F, nct, ntiles, tw, gscale, kf, filt,
                                                                               nfilt, fstep);
    return check_launch();
}

// NBUF = 2: k_fft_x_green_s (in-place passes), 3: k_fft_x_green3_s
template <int N, int B, int T, int NBUF>
inline int run_x_green(float2* F, int nct, int ntiles, const float2* tw, float gscale, float kf, const float* filt,
                       int nfilt, float fstep, cudaStream_t s) {
    constexpr size_t smem = ((size_t)NBUF * spad(N) * B + N) * 8;
    auto kern = [] {
        if constexpr (NBUF == 2)
            return k_fft_x_green_s<N, B, T>;
        else
            return k_fft_x_green3_s<N, B, T>;
    }();
    if (!set_smem((const void*)kern, smem)) return COLA_ECUDA;
    kern<<<persistent_grid(smem, ntiles), T, smem, s>>>(F, nct, ntiles, tw, gscale, kf, filt, nfilt, fstep);
    return check_launch();
}

// ---------------------------------------------------------------------------
// z passes (rows of the mesh, real <-> half-complex): persistent blocks over
// tiles of NR rows; the next tile's rows are staged into shared memory with
// cp.async while this one is transformed.
// ---------------------------------------------------------------------------
// c2r pre-processing from a staged row X[0..M]:
// Z[k] = (X[k] + conj X[M-k]) + i (X[k] - conj X[M-k]) W_2M^-k, Im X[0], Im X[M] ignored
template <int M, int SP>
struct C2rStage {
    const float2* stg;
    const float2* tw;  // W_2M^k = exp(-2 pi i k / 2M) for k <= M (shared memory)
    template <int R, int D>
    __device__ __forceinline__ void load(int l, int i0, float2* v) const {
        const float2* x = stg + l * SP;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int k = i0 + r * D;
            float2 a = x[k], bb = x[M - k];
            if (k == 0) {
                a.y = 0.f;
                bb.y = 0.f;
            }
            const float2 b = cconj(bb);
            float2 w = tw[k];
            w.y = -w.y;
            const float2 d = cmul(csub(a, b), w);
            v[r] = make_float2(a.x + b.x - d.y, a.y + b.y + d.x);
        }
    }
};

// row output (in place): z[m] as the float pair (2m, 2m+1) of row row0 + l
struct SRowStore {
    float2* data;
    long long rs, row0, nrows;
    template <int R, int D>
    __device__ __forceinline__ void store(int l, int i0, const float2* v) const {
        const long long row = row0 + l;
        if (row >= nrows) return;
        float2* q = data + row * rs + i0;
#pragma unroll
        for (int r = 0; r < R; ++r) __stcs(q + r * D, v[r]);
    }
};

// fixed-point CIC counts (2^40 per particle, staged rows of N) -> packed
// complex pairs of delta = count scale - 1
template <int N>
struct FixStage {
    const unsigned long long* stg;
    float scale;
    template <int R, int D>
    __device__ __forceinline__ void load(int l, int i0, float2* v) const {
        const ulonglong2* x = reinterpret_cast<const ulonglong2*>(stg + (size_t)l * N);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const ulonglong2 c = x[i0 + r * D];
            v[r] = make_float2((float)c.x * scale - 1.0f, (float)c.y * scale - 1.0f);
        }
    }
};

// entries of the pass-ordered twiddle table of an M-point plan
constexpr int ordered_tw_size(int M) { return tw_offset(static_plan(M), static_plan(M).nr); }

// c2r pre-processing read straight from a row X[0..M] in global memory (the
// same arithmetic as C2rStage)
template <int M>
struct C2rGlobal {
    const float2* __restrict__ x;
    const float2* tw;  // W_2M^k, k <= M (shared memory)
    template <int R, int D>
    __device__ __forceinline__ void load(int, int i0, float2* v) const {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int k = i0 + r * D;
            float2 a = __ldg(x + k), bb = __ldg(x + M - k);
            if (k == 0) {
                a.y = 0.f;
                bb.y = 0.f;
            }
            const float2 b = cconj(bb);
            float2 w = tw[k];
            w.y = -w.y;
            const float2 d = cmul(csub(a, b), w);
            v[r] = make_float2(a.x + b.x - d.y, a.y + b.y + d.x);
        }
    }
};

// counts read straight from a row of the fixed-point mesh in global memory
// and cleared as they are read (each pair is read once, by the first pass):
// packed complex pairs of delta = count scale - 1, as FixStage
template <int N>
struct FixGlobal {
    unsigned long long* row;
    float scale;
    template <int R, int D>
    __device__ __forceinline__ void load(int, int i0, float2* v) const {
        ulonglong2* x = reinterpret_cast<ulonglong2*>(row);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const ulonglong2 c = __ldcs(x + i0 + r * D);
            __stcs(x + i0 + r * D, make_ulonglong2(0ull, 0ull));
            v[r] = make_float2((float)c.x * scale - 1.0f, (float)c.y * scale - 1.0f);
        }
    }
};

// Plain z pass with warp-owned rows (the separate path's r2c of the counts):
// W warps per block, warp w of block b takes rows b W + w, then every
// gridDim.x W-th; the first pass reads the row from global memory, the others
// run in place in the warp's row buffer with __syncwarp between them; no block
// barrier after the start-up.
template <int N, int W>
constexpr size_t z_warp_smem() {
    return ((size_t)ordered_tw_size(N / 2) + N / 2 + 1 + (size_t)W * (spad(N / 2) + 1)) * 8;
}

// forward r2c along z of the fixed-point counts (cleared as they are read):
// input row r = x N + y, output row frow(x, y, 0, fr)
template <int N, int W, int MB>
__global__ void __launch_bounds__(32 * W, MB) k_fft_z_r2c_fix_w(unsigned long long* __restrict__ dep, float2* out,
                                                               long long rs, long long nrows, float scale,
                                                               const float2* __restrict__ tw, FRow fr) {
    constexpr int M = N / 2;
    using Geo = WarpRow<M>;
    extern __shared__ float2 sm[];
    float2* tws = sm;
    float2* twh = tws + ordered_tw_size(M);
    float2* rows = twh + (M + 1);
    ordered_twiddles<M, 32 * W, 2>(tws, tw);
    for (int q = threadIdx.x; q <= M; q += 32 * W) twh[q] = __ldg(tw + q);
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* Z = rows + w * Geo::LSTR;
    for (long long r = (long long)blockIdx.x * W + w; r < nrows; r += (long long)gridDim.x * W) {
        const int x = (int)(r / N), y = (int)(r - (long long)x * N);
        sip_run<M, 32, Geo, -1, false, true>(FixGlobal<N>{dep + r * N, scale}, SSmem<Geo>{Z}, Z, tws, NoHook());
        // X[k] = E[k] + W^k O[k], E = (Z[k] + conj Z[M-k]) / 2, O = (Z[k] - conj Z[M-k]) / (2i)
        float2* orow = out + frow(x, y, 0, fr) * rs;
        for (int k = lane; k <= M; k += 32) {
            const float2 a = Z[spad(k == M ? 0 : k)];
            const float2 b = cconj(Z[spad(k == 0 ? 0 : M - k)]);
            const float2 E = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y + b.y));
            const float2 D = csub(a, b);
            const float2 O = make_float2(0.5f * D.y, -0.5f * D.x);
            __stcs(orow + k, cadd(E, cmul(twh[k], O)));
        }
        __syncwarp();  // the row buffer is reused by the next row
    }
}

template <int N, int NR, int T>
constexpr size_t z_c2r_smem() {
    return ((size_t)NR * (N / 2 + 2) + 2 * (size_t)NR * (spad(N / 2) + 1) + ordered_tw_size(N / 2) + N / 2 + 1) * 8;
}
template <int N, int NR, int T>
constexpr size_t z_r2c_smem() {
    return ((size_t)NR * N + 2 * (size_t)NR * (spad(N / 2) + 1) + ordered_tw_size(N / 2) + N / 2 + 1) * 8;
}

// inverse c2r along z, in place on rows of rs complex (the runtime form is
// k_fft_z_c2r<false>): tiles of NR rows staged with cp.async; the first pass
// pre-processes the staged rows, after which the next tile is staged while the
// other passes ping-pong between two buffers
template <int N, int NR, int T, int MB>
__global__ void __launch_bounds__(T, MB) k_fft_z_c2r_s(float2* data, long long rs, long long nrows, int ntiles,
                                                        const float2* __restrict__ tw) {
    constexpr int M = N / 2;
    using Geo = RowTile<M, NR>;
    constexpr int SP = M + 2;  // staged row: X[0..M], whole 16-byte chunks
    constexpr int HS = SP / 2;
    extern __shared__ float2 sm[];
    float2* stg = sm;
    float2* A = stg + NR * SP;
    float2* Bf = A + NR * Geo::LSTR;
    float2* tws = Bf + NR * Geo::LSTR;  // pass-ordered twiddles of the M-point transform
    float2* twh = tws + ordered_tw_size(M);  // W_N^k, k <= M, for the c2r pre-processing
    ordered_twiddles<M, T, 2>(tws, tw);
    for (int q = threadIdx.x; q <= M; q += T) twh[q] = __ldg(tw + q);
    auto prefetch = [&](int t) {
        const long long row0 = (long long)t * NR;
#pragma unroll 4
        for (int e = threadIdx.x; e < NR * HS; e += T) {
            const int l = e / HS, c = (e - l * HS) * 2;
            if (row0 + l < nrows) cp_async16(stg + l * SP + c, data + (row0 + l) * rs + c);
        }
        cp_async_commit();
    };
    int t = blockIdx.x;
    if (t < ntiles) prefetch(t);
    for (; t < ntiles; t += gridDim.x) {
        cp_async_wait_all();
        __syncthreads();
        const int tn = t + gridDim.x;
        auto next = [&]() {
            if (tn < ntiles) prefetch(tn);
        };
        srun_out<M, T, Geo, +1>(C2rStage<M, SP>{stg, twh}, SRowStore{data, rs, (long long)t * NR, nrows}, A, Bf, tws,
                                next);
    }
}

// forward r2c along z of the fixed-point CIC mesh (rows of N counts), which
// is cleared as it is consumed; output row r = x n + y to frow(x, y, 0, fr)
// (the runtime form is k_fft_z_r2c<true>)
template <int N, int NR, int T, int MB>
__global__ void __launch_bounds__(T, MB) k_fft_z_r2c_fix_s(unsigned long long* __restrict__ dep, float2* out,
                                                            long long rs, long long nrows, int ntiles, float scale,
                                                            const float2* __restrict__ tw, FRow fr) {
    constexpr int M = N / 2;
    using Geo = RowTile<M, NR>;
    constexpr int HN = N / 2;  // 16-byte chunks per count row
    extern __shared__ float2 sm[];
    __shared__ long long obase[NR];
    unsigned long long* stg = reinterpret_cast<unsigned long long*>(sm);
    float2* A = sm + NR * N;
    float2* Bf = A + NR * Geo::LSTR;
    float2* tws = Bf + NR * Geo::LSTR;  // pass-ordered twiddles of the M-point transform
    float2* twh = tws + ordered_tw_size(M);  // W_N^k, k <= M, for the r2c post-processing
    ordered_twiddles<M, T, 2>(tws, tw);
    for (int q = threadIdx.x; q <= M; q += T) twh[q] = __ldg(tw + q);
    auto prefetch = [&](int t) {
        const long long row0 = (long long)t * NR;
#pragma unroll 4
        for (int e = threadIdx.x; e < NR * HN; e += T) {
            const int l = e / HN, c = (e - l * HN) * 2;
            if (row0 + l < nrows) cp_async16(stg + (size_t)l * N + c, dep + (row0 + l) * N + c);
        }
        cp_async_commit();
    };
    int t = blockIdx.x;
    if (t < ntiles) prefetch(t);
    for (; t < ntiles; t += gridDim.x) {
        const long long row0 = (long long)t * NR;
        cp_async_wait_all();
        __syncthreads();
        // the counts of this tile are in shared memory: clear them in the mesh
#pragma unroll 4
        for (int e = threadIdx.x; e < NR * HN; e += T) {
            const int l = e / HN, c = (e - l * HN) * 2;
            if (row0 + l < nrows)
                __stcs(reinterpret_cast<ulonglong2*>(dep + (row0 + l) * N + c), make_ulonglong2(0ull, 0ull));
        }
        if (threadIdx.x < NR) {
            const long long r = row0 + threadIdx.x;
            const int x = (int)(r / N), y = (int)(r - (long long)x * N);
            obase[threadIdx.x] = frow(x, y, 0, fr) * rs;
        }
        const int tn = t + gridDim.x;
        auto next = [&]() {
            if (tn < ntiles) prefetch(tn);
        };
        const float2* Z = srun_smem<M, T, Geo, -1>(FixStage<N>{stg, scale}, A, Bf, tws, next);
        // X[k] = E[k] + W^k O[k], E = (Z[k] + conj Z[M-k]) / 2, O = (Z[k] - conj Z[M-k]) / (2i)
#pragma unroll 2
        for (int e = threadIdx.x; e < NR * (M + 1); e += T) {
            const int l = e / (M + 1), k = e - l * (M + 1);
            if (row0 + l >= nrows) continue;
            const float2 a = Z[l * Geo::LSTR + spad(k == M ? 0 : k)];
            const float2 b = cconj(Z[l * Geo::LSTR + spad(k == 0 ? 0 : M - k)]);
            const float2 E = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y + b.y));
            const float2 D = csub(a, b);
            const float2 O = make_float2(0.5f * D.y, -0.5f * D.x);
            __stcs(out + obase[l] + k, cadd(E, cmul(twh[k], O)));
        }
    }
}

// MB: resident blocks per SM the kernel is compiled for (registers per thread
// at most 65536 / (MB T)); shared memory must allow as many
template <int N, int NR, int T, int MB>
inline int run_z_c2r(float2* data, long long rs, long long nrows, const float2* tw, cudaStream_t s) {
    static_assert(fft_pitch(N) >= N / 2 + 2, "staged rows must fit the row pitch");
    constexpr size_t smem = z_c2r_smem<N, NR, T>();
    static_assert((smem + 1024) * MB <= 227 * 1024, "MB blocks must fit in shared memory");
    const long long nt = (nrows + NR - 1) / NR;
    if (nt > 0x7fffffff) return COLA_EUNSUPPORTED_SIZE;
    if (!set_smem((const void*)k_fft_z_c2r_s<N, NR, T, MB>, smem)) return COLA_ECUDA;
    k_fft_z_c2r_s<N, NR, T, MB><<<persistent_grid(smem, (int)nt, MB), T, smem, s>>>(data, rs, nrows, (int)nt, tw);
    return check_launch();
}

template <int N, int NR, int T, int MB>
inline int run_z_r2c_fix(unsigned long long* dep, float2* out, long long rs, long long nrows, float scale,
                         const float2* tw, FRow fr, cudaStream_t s) {
    constexpr size_t smem = z_r2c_smem<N, NR, T>();
    static_assert((smem + 64 * NR + 1024) * MB <= 227 * 1024, "MB blocks must fit in shared memory");
    const long long nt = (nrows + NR - 1) / NR;
    if (nt > 0x7fffffff) return COLA_EUNSUPPORTED_SIZE;
    if (!set_smem((const void*)k_fft_z_r2c_fix_s<N, NR, T, MB>, smem)) return COLA_ECUDA;
    k_fft_z_r2c_fix_s<N, NR, T, MB><<<persistent_grid(smem, (int)nt, MB), T, smem, s>>>(dep, out, rs, nrows, (int)nt,
                                                                                     scale, tw, fr);
    return check_launch();
}

// launchers for the specialised kernels (fft_spec_*.cu); return false when
// (n, B) has no specialisation, without launching
bool launch_strided_static(float2* data, int n, int B, int sign, LineGeom lg, int nct, int ntiles,
                           const float2* tw, cudaStream_t s, int* rc);
bool launch_x_green_static(float2* F, int n, int B, int nct, int ntiles, const float2* tw, float gscale, float kf,
                           const float* filt, int nfilt, float fstep, cudaStream_t s, int* rc);
// z passes of the step: the in-place c2r of the force rows and the r2c of the
// fixed-point counts (fft_spec_large.cu)
bool launch_z_c2r_static(float2* data, int n, long long rs, long long nrows, const float2* tw, cudaStream_t s,
                         int* rc);
bool launch_z_r2c_fix_static(unsigned long long* dep, float2* out, int n, long long rs, long long nrows,
                             float scale, const float2* tw, FRow fr, cudaStream_t s, int* rc);
// default column width of the specialised line passes for n (0: none)
int static_tile(int n);
// whether (n, B) has specialised line passes
bool static_tile_ok(int n, int B);
// default column width of the specialised fused x/Green pass for n (0: the
// strided passes' width)
int static_green_tile(int n);
int launch_static_green_tile_small(int n);
// inverse y pass of the Psi component (k_fft_y_psi_s) for (n, B); false when
// there is no specialisation, without launching
bool launch_y_psi_static(float2* data, int n, int B, LineGeom lg, long long comp2, int nct, int ntiles,
                         const float2* tw, float kf, cudaStream_t s, int* rc);
bool launch_y_psi_static_small(float2* data, int n, int B, LineGeom lg, long long comp2, int nct, int ntiles,
                               const float2* tw, float kf, cudaStream_t s, int* rc);
// the mesh sizes below 512 (batched ensembles, tests), in fft_spec_small.cu
bool launch_strided_static_small(float2* data, int n, int B, int sign, LineGeom lg, int nct, int ntiles,
                                 const float2* tw, cudaStream_t s, int* rc);
bool launch_x_green_static_small(float2* F, int n, int B, int nct, int ntiles, const float2* tw, float gscale,
                                 float kf, const float* filt, int nfilt, float fstep, cudaStream_t s, int* rc);

}  // namespace cola
