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

// padded line-interleaved tile in shared memory: element i of line l at l + spad(i) B
template <int B>
struct SSmem {
    float2* p;
    template <int R, int D>
    __device__ __forceinline__ void load(int l, int i0, float2* v) const {
        if constexpr (D % 16 == 0) {
            const float2* q = p + l + spad(i0) * B;
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = q[r * spad(D) * B];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = p[l + spad(i0 + r * D) * B];
        }
    }
    // stores come from butterflies with i0 = jq LS R + k: for LS = D = 1 the
    // group i0 .. i0 + R - 1 starts at a multiple of R, which with R | 16 never
    // crosses a padding slot
    template <int R, int D>
    __device__ __forceinline__ void store(int l, int i0, const float2* v) const {
        if constexpr (D % 16 == 0 || (D == 1 && 16 % R == 0)) {
            float2* q = p + l + spad(i0) * B;
#pragma unroll
            for (int r = 0; r < R; ++r) q[r * spad(D) * B] = v[r];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) p[l + spad(i0 + r * D) * B] = v[r];
        }
    }
};

// One Stockham pass of radix R over a tile of B lines (see fft_pass for the
// index map): butterfly b = (j, l), j < N / R, k = j mod LS,
//   v_r = in(l, j + r N/R) W_{LS R}^{r k},  v = DFT_R(v),  out(l, (j / LS) LS R + k + r LS) = v_r.
template <int N, int B, int T, int R, int LS, int SIGN, class In, class Out>
__device__ __forceinline__ void spass(const In& in, const Out& out, const float2* __restrict__ tw) {
    constexpr int NBL = N / R;
    constexpr int NB = NBL * B;
    constexpr int IT = (NB + T - 1) / T;
    constexpr int TWS = N / (LS * R);
#pragma unroll
    for (int it = 0; it < IT; ++it) {
        const unsigned b = threadIdx.x + (unsigned)(it * T);
        if (NB % T != 0 && it == IT - 1 && b >= (unsigned)NB) break;
        const int l = (int)(b % B);
        const int j = (int)(b / B);
        const int jq = (int)((unsigned)j / LS);
        const int k = j - jq * LS;
        float2 v[R];
        in.template load<R, NBL>(l, j, v);
        if constexpr (LS > 1) {
            const float2* tq = tw;
            const int step = k * TWS;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = tq[r * step];
                if (SIGN > 0) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        SmallDft<R>::run(v, SIGN);
        out.template store<R, LS>(l, jq * LS * R + k, v);
    }
}

// passes S .. nr-1: S reads a; the last pass writes `out`
template <int N, int B, int T, int SIGN, int S, class Out>
__device__ __forceinline__ void srun_tail(float2* a, float2* b, const Out& out, const float2* __restrict__ tw) {
    constexpr StaticPlan P = static_plan(N);
    constexpr int R = P.r[S];
    constexpr int LS = plan_ls(P, S);
    if constexpr (S == P.nr - 1) {
        spass<N, B, T, R, LS, SIGN>(SSmem<B>{a}, out, tw);
        __syncthreads();
    } else {
        spass<N, B, T, R, LS, SIGN>(SSmem<B>{a}, SSmem<B>{b}, tw);
        __syncthreads();
        srun_tail<N, B, T, SIGN, S + 1>(b, a, out, tw);
    }
}

// Transform reading `in` in the first pass (into a), then `hook` (uniform:
// the input is no longer needed), the middle passes ping-pong a/b, the last
// pass writes `out`.  Needs at least two passes.  Returns synchronised.
template <int N, int B, int T, int SIGN, class In, class Out, class Hook>
__device__ __forceinline__ void srun_out(const In& in, const Out& out, float2* a, float2* b,
                                         const float2* __restrict__ tw, const Hook& hook) {
    constexpr StaticPlan P = static_plan(N);
    static_assert(P.ok && P.nr >= 2, "specialised transforms need two or more passes");
    spass<N, B, T, P.r[0], 1, SIGN>(in, SSmem<B>{a}, tw);
    __syncthreads();
    hook();
    srun_tail<N, B, T, SIGN, 1>(a, b, out, tw);
}

// Same, with the result left in shared memory; returns the buffer holding it.
template <int N, int B, int T, int SIGN, class In, class Hook>
__device__ __forceinline__ float2* srun_smem(const In& in, float2* a, float2* b, const float2* __restrict__ tw,
                                             const Hook& hook) {
    constexpr StaticPlan P = static_plan(N);
    float2* res = ((P.nr - 1) % 2 == 1) ? b : a;
    srun_out<N, B, T, SIGN>(in, SSmem<B>{res}, a, b, tw, hook);
    return res;
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

// Psi = IFFT_x(phi) written as F_y = i k_y Psi and F_z = i k_z Psi (both
// constant along an x line)
template <int N>
struct SYZStore {
    float2* fy;
    float2* fz;
    float ky, kf;
    int col0;
    template <int R, int D>
    __device__ __forceinline__ void store(int l, int i0, const float2* v) const {
        using G = XGeom<N>;
        const float kz = (col0 + l == N / 2) ? 0.f : kf * (float)(col0 + l);
        if constexpr (D % G::XB == 0) {
            const long long q0 = G::off(i0) + l;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const long long q = q0 + (long long)r * (D / G::XB) * G::SB;
                __stcs(fy + q, make_float2(-ky * v[r].y, ky * v[r].x));
                __stcs(fz + q, make_float2(-kz * v[r].y, kz * v[r].x));
            }
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const long long q = G::off(i0 + r * D) + l;
                __stcs(fy + q, make_float2(-ky * v[r].y, ky * v[r].x));
                __stcs(fz + q, make_float2(-kz * v[r].y, kz * v[r].x));
            }
        }
    }
};

// strided complex pass (y: S = row stride, outer = x; or x on a plain mesh):
// persistent blocks, cp.async prefetch of the next tile during this one
template <int N, int B, int T, int SIGN>
__global__ void __launch_bounds__(T) k_fft_strided_s(float2* data, LineGeom lg, int nct, int ntiles,
                                                      const float2* __restrict__ tw) {
    constexpr int TSZ = spad(N) * B;
    extern __shared__ float2 sm[];
    float2* stg = sm;
    float2* A = sm + TSZ;
    float2* Bf = A + TSZ;
    float2* tws = Bf + TSZ;
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
        srun_out<N, B, T, SIGN>(SSmem<B>{stg}, SCol{tile_base(t), lg.S}, A, Bf, tws, next);
    }
}

// x pass fused with the Poisson solve and the ik gradient on the interleaved,
// x-blocked force mesh (the runtime form is k_fft_x_green): forward x FFT of
// delta_k (component 0), phi = gscale delta_k / k^2 (times the radial filter
// if given), F_x = IFFT_x(i k_x phi) and Psi = IFFT_x(phi) stored as
// F_y = i k_y Psi, F_z = i k_z Psi.
template <int N, int B, int T>
__global__ void __launch_bounds__(T) k_fft_x_green_s(float2* F, int nct, int ntiles, const float2* __restrict__ tw,
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
        float2* X = srun_smem<N, B, T, -1>(SSmem<B>{stg}, A, W, tws, next);
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
        const float ky_eff = (iy == half) ? 0.f : ky;
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            const int i = i0 + q * TB;
            const float kx = (i == half) ? 0.f : kf * (float)(i < half ? i : i - N);
            elem(A, q) = make_float2(-kx * phi[q].y, kx * phi[q].x);  // i k_x phi
        }
        __syncthreads();
        srun_out<N, B, T, +1>(SSmem<B>{A}, SXIO<N>{F + off}, W, A, tws, NoHook{});
#pragma unroll
        for (int q = 0; q < EPT; ++q) elem(A, q) = phi[q];
        __syncthreads();
        srun_out<N, B, T, +1>(SSmem<B>{A}, SYZStore<N>{F + off + G::P, F + off + 2 * G::P, ky_eff, kf, col0}, W, A,
                              tws, NoHook{});
    }
}

template <int N, int B, int T>
inline int run_strided(float2* data, int sign, LineGeom lg, int nct, int ntiles, const float2* tw, cudaStream_t s) {
    const size_t smem = ((size_t)3 * spad(N) * B + N) * 8;
    auto kern = sign < 0 ? k_fft_strided_s<N, B, T, -1> : k_fft_strided_s<N, B, T, +1>;
    if (!set_smem((const void*)kern, smem)) return COLA_ECUDA;
    kern<<<persistent_grid(smem, ntiles), T, smem, s>>>(data, lg, nct, ntiles, tw);
    return check_launch();
}

template <int N, int B, int T>
inline int run_x_green(float2* F, int nct, int ntiles, const float2* tw, float gscale, float kf, const float* filt,
                       int nfilt, float fstep, cudaStream_t s) {
    const size_t smem = ((size_t)3 * spad(N) * B + N) * 8;
    if (!set_smem((const void*)k_fft_x_green_s<N, B, T>, smem)) return COLA_ECUDA;
    k_fft_x_green_s<N, B, T><<<persistent_grid(smem, ntiles), T, smem, s>>>(F, nct, ntiles, tw, gscale, kf, filt,
                                                                             nfilt, fstep);
    return check_launch();
}

// launchers for the specialised kernels (fft_spec_*.cu); return false when
// (n, B) has no specialisation, without launching
bool launch_strided_static(float2* data, int n, int B, int sign, LineGeom lg, int nct, int ntiles,
                           const float2* tw, cudaStream_t s, int* rc);
bool launch_x_green_static(float2* F, int n, int B, int nct, int ntiles, const float2* tw, float gscale, float kf,
                           const float* filt, int nfilt, float fstep, cudaStream_t s, int* rc);
// the mesh sizes below 512 (batched ensembles, tests), in fft_spec_small.cu
bool launch_strided_static_small(float2* data, int n, int B, int sign, LineGeom lg, int nct, int ntiles,
                                 const float2* tw, cudaStream_t s, int* rc);
bool launch_x_green_static_small(float2* F, int n, int B, int nct, int ntiles, const float2* tw, float gscale,
                                 float kf, const float* filt, int nfilt, float fstep, cudaStream_t s, int* rc);

}  // namespace cola
