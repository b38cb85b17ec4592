// Internal definitions shared by the translation units of the COLA library:
// complex helpers, the shared-memory mixed-radix FFT engine, the workspace
// layout and the host-side launch helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cola.h"

namespace cola {

// Row bins of the PM step: particles sorted by the (x, y) mesh row of their
// lower CIC corner, bin x ng + y holding sorted[start[b] .. start[b + 1]).
struct RowBins {
    const int* start;     // ng^2 + 1 offsets
    const int* sorted;    // particle indices
    const float4* cic;    // per sorted particle: CIC fractions (fx, fy, fz) and the lower z cell (int bits in w)
    int* status;          // the workspace's status word (bounds checks of a COLA_CHECKS build)
    long long np;         // particles (sorted positions are < np)
    int ng;               // mesh side (z cells are < ng)
};

// ---------------------------------------------------------------------------
// complex helpers (float2 = complex64)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// multiply by i*sign (sign = +1 or -1)
__device__ __forceinline__ float2 cmul_isign(float2 a, int sign) {
    return sign > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// ---------------------------------------------------------------------------
// small DFTs: X_k = sum_r v_r exp(sign 2 pi i r k / R), in registers
// ---------------------------------------------------------------------------
template <int R>
struct SmallDft;

template <>
struct SmallDft<2> {
    __device__ __forceinline__ static void run(float2* v, int) {
        float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <>
struct SmallDft<3> {
    __device__ __forceinline__ static void run(float2* v, int sign) {
        const float h = 0.86602540378443864676f;  // sin(2 pi / 3)
        float2 t = cadd(v[1], v[2]);
        float2 m = make_float2(v[0].x - 0.5f * t.x, v[0].y - 0.5f * t.y);
        float2 s = cmul_isign(cscale(csub(v[1], v[2]), h), sign);
        v[0] = cadd(v[0], t);
        v[1] = cadd(m, s);
        v[2] = csub(m, s);
    }
};

template <>
struct SmallDft<4> {
    __device__ __forceinline__ static void run(float2* v, int sign) {
        float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        float2 t2 = cadd(v[1], v[3]), t3 = cmul_isign(csub(v[1], v[3]), sign);
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    }
};

template <>
struct SmallDft<5> {
    __device__ __forceinline__ static void run(float2* v, int sign) {
        const float c1 = 0.30901699437494742410f;   // cos(2 pi/5)
        const float c2 = -0.80901699437494742410f;  // cos(4 pi/5)
        const float s1 = 0.95105651629515357212f;   // sin(2 pi/5)
        const float s2 = 0.58778525229247312917f;   // sin(4 pi/5)
        float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
        float2 d1 = csub(v[1], v[4]), d2 = csub(v[2], v[3]);
        float2 a1 = make_float2(v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y);
        float2 a2 = make_float2(v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y);
        float2 b1 = cmul_isign(make_float2(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y), sign);
        float2 b2 = cmul_isign(make_float2(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y), sign);
        v[0] = cadd(v[0], cadd(t1, t2));
        v[1] = cadd(a1, b1);
        v[4] = csub(a1, b1);
        v[2] = cadd(a2, b2);
        v[3] = csub(a2, b2);
    }
};

template <>
struct SmallDft<8> {
    // radix-2 decimation in frequency on top of two 4-point DFTs
    __device__ __forceinline__ static void run(float2* v, int sign) {
        const float r = 0.70710678118654752440f;
        float2 a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            a[i] = cadd(v[i], v[i + 4]);
            b[i] = csub(v[i], v[i + 4]);
        }
        // b_i *= exp(sign 2 pi i i/8)
        b[1] = make_float2(r * (b[1].x - sign * b[1].y), r * (b[1].y + sign * b[1].x));
        b[2] = cmul_isign(b[2], sign);
        b[3] = make_float2(r * (-b[3].x - sign * b[3].y), r * (-b[3].y + sign * b[3].x));
        SmallDft<4>::run(a, sign);
        SmallDft<4>::run(b, sign);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            v[2 * i] = a[i];
            v[2 * i + 1] = b[i];
        }
    }
};

template <>
struct SmallDft<16> {
    // 4 x 4: DFT4 over stride-4 groups, twiddle by W16^(a b), DFT4 again
    __device__ __forceinline__ static void run(float2* v, int sign) {
        const float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f, r = 0.70710678118654752440f;
        float2 g[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
#pragma unroll
            for (int q = 0; q < 4; ++q) g[a][q] = v[a + 4 * q];
            SmallDft<4>::run(g[a], sign);  // g[a][b] = sum_q v[a+4q] W4^(qb)
        }
        // twiddle W16^(a b) = exp(sign 2 pi i a b / 16)
        const float2 w1 = make_float2(c1, sign * s1), w2 = make_float2(r, sign * r), w3 = make_float2(s1, sign * c1);
        const float2 w6 = make_float2(-r, sign * r), w9 = make_float2(-c1, -sign * s1);
        g[1][1] = cmul(g[1][1], w1);
        g[1][2] = cmul(g[1][2], w2);
        g[1][3] = cmul(g[1][3], w3);
        g[2][1] = cmul(g[2][1], w2);
        g[2][2] = cmul_isign(g[2][2], sign);
        g[2][3] = cmul(g[2][3], w6);
        g[3][1] = cmul(g[3][1], w3);
        g[3][2] = cmul(g[3][2], w6);
        g[3][3] = cmul(g[3][3], w9);
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            float2 t[4] = {g[0][b], g[1][b], g[2][b], g[3][b]};
            SmallDft<4>::run(t, sign);  // X[b + 4c] = sum_a t[a] W4^(ac)
#pragma unroll
            for (int c = 0; c < 4; ++c) v[b + 4 * c] = t[c];
        }
    }
};

// Radix P*Q (coprime P, Q, Good-Thomas index map): 6 = 2 x 3, 12 = 4 x 3.
template <int P, int Q>
__device__ __forceinline__ void pfa_dft(float2* v, int sign) {
    constexpr int N = P * Q;
    float2 g[Q][P];
    // input n = (P a + Q b) mod N -> g[a'][b] with a' indexing Q, b indexing P
#pragma unroll
    for (int a = 0; a < Q; ++a)
#pragma unroll
        for (int b = 0; b < P; ++b) g[a][b] = v[(P * a + Q * b) % N];
#pragma unroll
    for (int a = 0; a < Q; ++a) SmallDft<P>::run(g[a], sign);
#pragma unroll
    for (int b = 0; b < P; ++b) {
        float2 t[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) t[a] = g[a][b];
        SmallDft<Q>::run(t, sign);
#pragma unroll
        for (int a = 0; a < Q; ++a) g[a][b] = t[a];
    }
    // output k with k = c1 (mod P), k = c2 (mod Q): CRT
#pragma unroll
    for (int c2 = 0; c2 < Q; ++c2)
#pragma unroll
        for (int c1 = 0; c1 < P; ++c1) {
            int k = 0;
#pragma unroll
            for (int t = 0; t < N; ++t)
                if (t % P == c1 && t % Q == c2) k = t;
            v[k] = g[c2][c1];
        }
}

template <>
struct SmallDft<6> {
    __device__ __forceinline__ static void run(float2* v, int sign) { pfa_dft<2, 3>(v, sign); }
};
template <>
struct SmallDft<12> {
    __device__ __forceinline__ static void run(float2* v, int sign) { pfa_dft<4, 3>(v, sign); }
};

// ---------------------------------------------------------------------------
// FFT plan: n = product of radices (applied in order), n <= kMaxFft
// ---------------------------------------------------------------------------
constexpr int kMaxFft = 4096;   // largest line length

// n has no prime factor other than 2, 3 and 5
inline bool factorable(int n) {
    if (n < 1) return false;
    for (int p : {2, 3, 5})
        while (n % p == 0) n /= p;
    return n == 1;
}
// a mesh or lattice side every transform of the library can run: even, at
// least 4, at most kMaxFft, and n and n/2 factorable (the real transforms run
// n/2-point complex ones)
inline bool mesh_ok(int n) { return n >= 4 && n % 2 == 0 && n <= kMaxFft && factorable(n) && factorable(n / 2); }
constexpr int kMaxRadices = 16;

// Exact division by a runtime constant d for numerators n with n * d < 2^32:
// q = umulhi(n, ceil(2^32 / d)) (d = 1 handled apart).
struct FastDiv {
    unsigned d, m;
};
inline FastDiv make_fastdiv(unsigned d) {
    return FastDiv{d, d <= 1 ? 0u : (unsigned)(((1ull << 32) + d - 1) / d)};
}
__device__ __forceinline__ unsigned fdiv(unsigned n, FastDiv f) { return f.d <= 1 ? n : __umulhi(n, f.m); }

struct FftPlan {
    int n;
    int nr;
    int radix[kMaxRadices];
    FastDiv ls_div[kMaxRadices];   // division by Ls (product of the radices before pass s)
    FastDiv nbl_div[kMaxRadices];  // division by n / radix[s]
};

// Radix list of a length-n transform: threes are paired with spare factors of
// two (12 = 4*3, 6 = 2*3), the remaining twos go in 16s, then 8/4/2, then the
// leftover 3s and 5s; sorted largest first (the first pass reads global memory
// and needs no twiddles).  ok = false if n has another prime factor.
struct StaticPlan {
    bool ok;
    int nr;
    int r[kMaxRadices];
};
__host__ __device__ constexpr StaticPlan static_plan(int n) {
    StaticPlan p{false, 0, {}};
    if (n < 1 || n > kMaxFft) return p;
    int m = n, a = 0, b = 0, c = 0;
    while (m % 2 == 0) { m /= 2; ++a; }
    while (m % 3 == 0) { m /= 3; ++b; }
    while (m % 5 == 0) { m /= 5; ++c; }
    if (m != 1) return p;
    int nr = 0;
    const int pairs = b < a / 2 ? b : a / 2;
    for (int i = 0; i < pairs; ++i) p.r[nr++] = 12;
    a -= 2 * pairs;
    b -= pairs;
    if (b > 0 && a > 0) { p.r[nr++] = 6; --a; --b; }
    while (a >= 4) { p.r[nr++] = 16; a -= 4; }
    if (a == 3) p.r[nr++] = 8;
    if (a == 2) p.r[nr++] = 4;
    if (a == 1) p.r[nr++] = 2;
    while (b-- > 0) p.r[nr++] = 3;
    while (c-- > 0) p.r[nr++] = 5;
    for (int i = 0; i < nr; ++i)
        for (int j = i + 1; j < nr; ++j)
            if (p.r[j] > p.r[i]) { const int t = p.r[i]; p.r[i] = p.r[j]; p.r[j] = t; }
    p.nr = nr;
    p.ok = true;
    return p;
}
// product of the radices before pass s
__host__ __device__ constexpr int plan_ls(const StaticPlan& p, int s) {
    int ls = 1;
    for (int i = 0; i < s; ++i) ls *= p.r[i];
    return ls;
}

// Runtime plan of static_plan(n).  Returns false if n is unsupported.
bool make_plan(int n, FftPlan* p);

// ---------------------------------------------------------------------------
// Stockham autosort passes (Govindaraju et al. 2008, "expand" form) over nl
// lines of length n, reading through an input accessor and writing through an
// output accessor.  Butterfly j of line l (0 <= j < n/R), k = j mod Ls:
//   v_r = in(l, j + r n/R) * W_{Ls R}^{r k},  v = DFT_R(v),
//   out(l, (j / Ls) Ls R + k + r Ls) = v_r
// with Ls the product of the radices already applied and
// tw[q * twmul] = exp(-2 pi i q / n).  Accessors give load<R>(l, i0, di, v)
// (v_r = x(l, i0 + r di)) and store<R>(l, i0, di, v).
// The first pass of a transform reads global memory directly and the last
// one may write it directly, so a transform of p passes moves its data
// through shared memory only p - 1 times.
// ---------------------------------------------------------------------------
// Shared-memory element i of a line sits at i + i/16: one pad slot per 16
// elements keeps the stride-R accesses of a Stockham pass off a single bank.
__host__ __device__ constexpr int spad(int i) { return i + (i >> 4); }

struct SmemIO {
    float2* p;
    int ls, es;
    template <int R>
    __device__ __forceinline__ void load(int l, int i0, int di, float2* v) const {
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = p[l * ls + spad(i0 + r * di) * es];
    }
    template <int R>
    __device__ __forceinline__ void store(int l, int i0, int di, const float2* v) const {
#pragma unroll
        for (int r = 0; r < R; ++r) p[l * ls + spad(i0 + r * di) * es] = v[r];
    }
};

template <int R, int SIGN, bool LF, class In, class Out>
__device__ __forceinline__ void fft_pass(const In& in, const Out& out, int n, int nl, int nl_shift, int Ls,
                                         FastDiv lsd, FastDiv nbld, const float2* __restrict__ tw, int twmul) {
    constexpr int sign = SIGN;
    constexpr bool line_fast = LF;
    const int nbl = n / R;
    const int nb = nbl * nl;
    const int twstep = (n / (Ls * R)) * twmul;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        int l, j;
        if (line_fast) {
            l = b & (nl - 1);
            j = b >> nl_shift;
        } else {
            l = (int)fdiv((unsigned)b, nbld);
            j = b - l * nbl;
        }
        const int jq = (int)fdiv((unsigned)j, lsd);
        const int k = j - jq * Ls;
        float2 v[R];
        in.template load<R>(l, j, nbl, v);
        if (Ls > 1) {
            const int step = k * twstep;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = tw[r * step];
                if (sign > 0) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        SmallDft<R>::run(v, sign);
        out.template store<R>(l, jq * Ls * R + k, Ls, v);
    }
}

template <int SIGN, bool LF, class In, class Out>
__device__ __forceinline__ void fft_pass_any(int R, const In& in, const Out& out, int n, int nl, int nl_shift, int Ls,
                                             FastDiv lsd, FastDiv nbld, const float2* __restrict__ tw, int twmul) {
    switch (R) {
        case 16: fft_pass<16, SIGN, LF>(in, out, n, nl, nl_shift, Ls, lsd, nbld, tw, twmul); break;
        case 12: fft_pass<12, SIGN, LF>(in, out, n, nl, nl_shift, Ls, lsd, nbld, tw, twmul); break;
        case 8: fft_pass<8, SIGN, LF>(in, out, n, nl, nl_shift, Ls, lsd, nbld, tw, twmul); break;
        case 6: fft_pass<6, SIGN, LF>(in, out, n, nl, nl_shift, Ls, lsd, nbld, tw, twmul); break;
        case 5: fft_pass<5, SIGN, LF>(in, out, n, nl, nl_shift, Ls, lsd, nbld, tw, twmul); break;
        case 4: fft_pass<4, SIGN, LF>(in, out, n, nl, nl_shift, Ls, lsd, nbld, tw, twmul); break;
        case 3: fft_pass<3, SIGN, LF>(in, out, n, nl, nl_shift, Ls, lsd, nbld, tw, twmul); break;
        default: fft_pass<2, SIGN, LF>(in, out, n, nl, nl_shift, Ls, lsd, nbld, tw, twmul); break;
    }
}

// Force-mesh row of (x, y, component c): x is blocked by XB = 2^xbs so that a
// line along x (stride n XB comps P between blocks) touches n / XB memory
// pages instead of n, while a line along y spans XB times more; rows
// ((x / XB) n + y) XB + x mod XB, each holding `comps` component rows.
struct FRow {
    int n, xbs, comps;
};
__host__ __device__ __forceinline__ long long frow(int x, int y, int c, const FRow& f) {
    return ((((long long)(x >> f.xbs) * f.n + y) << f.xbs) + (x & ((1 << f.xbs) - 1))) * f.comps + c;
}
__host__ __device__ constexpr int xblock_shift(int n) {
    return n % 8 == 0 ? 3 : (n % 4 == 0 ? 2 : (n % 2 == 0 ? 1 : 0));
}

struct LineGeom {
    long long S;   // element stride along the transformed axis
    int nouter;    // number of outer indices
    int o2n;       // outer index o = o1 * o2n + o2
    long long s1, s2;
};

struct FftGeom {
    int nl;          // lines per block
    int ls, es;      // shared-memory layout: element i of line l at l*ls + i*es
    bool line_fast;  // butterfly index runs over lines first (needs nl = 2^nl_shift)
    int nl_shift;
    int twmul;       // table stride: tw is the table of n*twmul
};

// Transform reading `in`, all intermediate passes in shared memory (ping-pong
// a/b), last pass written through `out`.  Returns synchronised.
struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};

// `hook` runs (uniformly, by every thread) right after the first pass, when
// the input accessor's memory is no longer needed.
template <int SIGN, bool LF, class In, class Out, class Hook = NoHook>
__device__ __forceinline__ void fft_run_out(const In& in, const Out& out, float2* a, float2* b, const FftPlan& plan,
                                            const FftGeom& g, const float2* __restrict__ tw,
                                            const Hook& hook = Hook()) {
    int Ls = 1;
    if (plan.nr == 1) {
        // single pass: go through shared memory so that in-place callers never
        // store an element another thread has still to load
        fft_pass_any<SIGN, LF>(plan.radix[0], in, SmemIO{a, g.ls, g.es}, plan.n, g.nl, g.nl_shift, 1, plan.ls_div[0],
                           plan.nbl_div[0], tw, g.twmul);
        __syncthreads();
        hook();
        for (int e = threadIdx.x; e < plan.n * g.nl; e += blockDim.x) {
            const int l = LF ? (e & (g.nl - 1)) : e / plan.n;
            const int i = LF ? (e >> g.nl_shift) : e - l * plan.n;
            const float2 v = a[l * g.ls + spad(i) * g.es];
            out.template store<1>(l, i, 1, &v);
        }
        __syncthreads();
        return;
    }
    fft_pass_any<SIGN, LF>(plan.radix[0], in, SmemIO{a, g.ls, g.es}, plan.n, g.nl, g.nl_shift, 1, plan.ls_div[0],
                           plan.nbl_div[0], tw, g.twmul);
    __syncthreads();
    hook();
    Ls = plan.radix[0];
    for (int s = 1; s + 1 < plan.nr; ++s) {
        fft_pass_any<SIGN, LF>(plan.radix[s], SmemIO{a, g.ls, g.es}, SmemIO{b, g.ls, g.es}, plan.n, g.nl,
                               g.nl_shift, Ls, plan.ls_div[s], plan.nbl_div[s], tw, g.twmul);
        __syncthreads();
        float2* t = a;
        a = b;
        b = t;
        Ls *= plan.radix[s];
    }
    const int s = plan.nr - 1;
    fft_pass_any<SIGN, LF>(plan.radix[s], SmemIO{a, g.ls, g.es}, out, plan.n, g.nl, g.nl_shift, Ls, plan.ls_div[s],
                           plan.nbl_div[s], tw, g.twmul);
    __syncthreads();
}

// Same, with the result left in shared memory; returns the buffer holding it.
template <int SIGN, bool LF, class In, class Hook = NoHook>
__device__ __forceinline__ float2* fft_run_smem(const In& in, float2* a, float2* b, const FftPlan& plan,
                                                const FftGeom& g, const float2* __restrict__ tw,
                                                const Hook& hook = Hook()) {
    fft_pass_any<SIGN, LF>(plan.radix[0], in, SmemIO{a, g.ls, g.es}, plan.n, g.nl, g.nl_shift, 1, plan.ls_div[0],
                           plan.nbl_div[0], tw, g.twmul);
    __syncthreads();
    hook();
    int Ls = plan.radix[0];
    for (int s = 1; s < plan.nr; ++s) {
        fft_pass_any<SIGN, LF>(plan.radix[s], SmemIO{a, g.ls, g.es}, SmemIO{b, g.ls, g.es}, plan.n, g.nl,
                               g.nl_shift, Ls, plan.ls_div[s], plan.nbl_div[s], tw, g.twmul);
        __syncthreads();
        float2* t = a;
        a = b;
        b = t;
        Ls *= plan.radix[s];
    }
    return a;
}

// ---------------------------------------------------------------------------
// workspace layout
// ---------------------------------------------------------------------------
constexpr int kMaxSteps = 2048;
constexpr int kTableCols = 12;
constexpr size_t kHdrStatus = 0;          // int: latched device status
constexpr size_t kHdrSigmaAmp = 64;       // double: P(k) amplitude A (sigma8 normalisation)
constexpr size_t kHdrSnap = 128;          // 6 doubles: snapshot drift (dr, dD1, dD2), redshift-space (cv, c1, c2)
constexpr size_t kHdrProbe = 512;         // 64 ints written by cola_checks_probe
constexpr int kProbeInts = 64;
constexpr size_t kHdrDepState = 768;      // int: kDepClean while the fixed-point region holds zero counts
constexpr int kDepClean = 0x5a5a5a5a;     // (a byte pattern, so cudaMemsetAsync can write it)
constexpr size_t kHdrFilter = 1024;       // radial filter basis table (<= 64 floats)
constexpr size_t kHdrTable = 4096;        // kMaxSteps x kTableCols doubles
constexpr size_t kHdrTwiddle = 262144;    // 3 slots of kMaxFft float2
constexpr size_t kHdrBytes = 524288;

enum TwSlot { kTwMesh = 0, kTwLagr = 1, kTwScratch = 2 };

struct Layout {
    size_t dep;        // uint64 fixed-point CIC mesh, ng^3 (outputs and the density call; cleared by its user)
    // the PM step's row bins and partial force sums, aliasing the region of dep
    size_t bstart, bsums, bkey, brank, bsorted, bcic, slots;
    size_t F;          // interleaved force mesh: ng x ng x 3 rows of P complex (delta_k in component 0)
    size_t ic;         // 2LPT scratch: 7 complex meshes of nq x nq x Pq (aliases dep..)
    size_t pk_part;    // P(k) per-block partial sums (after the first two thirds of F)
    size_t lrn;        // learned-correction buffers (COLA_FLAG_LEARNED), 0 otherwise
    size_t total;
};

__host__ __device__ constexpr int fft_pitch(int n) { return (n / 2 + 1 + 15) / 16 * 16; }
inline size_t mesh_bytes(int n) { return (size_t)n * n * fft_pitch(n) * 8; }
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
bool layout_for(const cola_config* cfg, Layout* L);

inline char* wsp(void* ws, size_t off) { return static_cast<char*>(ws) + off; }
inline int* status_ptr(void* ws) { return reinterpret_cast<int*>(wsp(ws, kHdrStatus)); }
inline double* table_ptr(void* ws) { return reinterpret_cast<double*>(wsp(ws, kHdrTable)); }
inline float2* twiddle_ptr(void* ws, int slot) {
    return reinterpret_cast<float2*>(wsp(ws, kHdrTwiddle + (size_t)slot * kMaxFft * 8));
}

// ---------------------------------------------------------------------------
// asynchronous global -> shared copies (16 bytes, L2 only) for tile prefetch
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
// wait until at most N of this thread's committed groups are still in flight
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Stage an n x B tile (rows i at stride S, B adjacent complex columns) into
// shared memory with the padded line layout (l + spad(i) B), 16 bytes at a time.
__device__ __forceinline__ void tile_prefetch(float2* stg, const float2* g, int n, int B, long long S) {
    const int hb = B >> 1;
    const int hs = __ffs(hb) - 1;
    for (int e = threadIdx.x; e < n * hb; e += blockDim.x) {
        const int i = e >> hs, c = (e & (hb - 1)) << 1;
        cp_async16(stg + c + spad(i) * B, g + (long long)i * S + c);
    }
    cp_async_commit();
}

// device status latch
__device__ __forceinline__ void set_status(int* status, int code) { atomicCAS(status, 0, code); }

// Bounds check of a data-dependent index (a sorted position from the bin scan,
// a z cell read back from a CIC record, a bin key).  In a build with
// COLA_CHECKS defined a failed check latches COLA_EBOUNDS and the caller skips
// the access; in the normal build the check is constant true and compiles away.
#ifdef COLA_CHECKS
constexpr bool kChecks = true;
__device__ __forceinline__ bool bounds_ok(int* status, bool ok) {
    if (!ok) set_status(status, COLA_EBOUNDS);
    return ok;
}
#else
constexpr bool kChecks = false;
__device__ __forceinline__ bool bounds_ok(int*, bool) { return true; }
#endif

// ---------------------------------------------------------------------------
// per-kernel event timing (prof.cu): a ProfScope around each launch
// ---------------------------------------------------------------------------
enum KernelId {
    kKDeposit = 0, kKZr2cFix, kKZr2c, kKYFwd, kKXFwd, kKXGreen, kKYInv, kKXInv, kKZc2r, kKGatherKD, kKGather,
    kKFixToDelta, kKPkShells, kKPkReduce, kKIc, kKSetup, kKLearned, kKBins, kKDepR2c, kKC2rGather, kKKickDrift,
    kNumKernelIds
};
// a ProfScope with id < 0 records nothing (launches inside an enclosing scope)
class ProfScope {
  public:
    ProfScope(int id, cudaStream_t s);
    ~ProfScope();
  private:
    int rec_;
    cudaStream_t s_;
};

// ---------------------------------------------------------------------------
// host-side launch helpers (defined in the .cu files)
// ---------------------------------------------------------------------------
extern unsigned long long g_launches;
extern int g_last_cuda_error;  // the CUDA error behind the last COLA_ECUDA of a launch (cola_last_cuda_error)
inline int check_launch() {
    g_launches++;
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) return COLA_OK;
    g_last_cuda_error = (int)e;
    return COLA_ECUDA;
}

int launch_twiddles(float2* tw, int n, cudaStream_t s);
// raise a kernel's dynamic shared-memory limit (cached per kernel and size)
bool set_smem(const void* fn, size_t bytes);
// persistent grid: blocks per SM from the shared-memory budget, at most ntiles
int num_sms();  // of the current device (cached)
int persistent_grid(size_t smem, int ntiles);
// the same with at most max_per_sm blocks per SM (the launch bounds' count, when
// registers or threads limit residency before shared memory does)
int persistent_grid(size_t smem, int ntiles, int max_per_sm);
// z passes: row r at base + r*rs (complex units), nrows rows
// r2c: input row r = x n + y goes to output row frow(x, y, 0, fr) (fr = {n, 0, 1}: in place, same row)
int fft_z_r2c(unsigned long long* dep, float2* out, int n, float scale, const float2* tw, cudaStream_t s,
              long long rs, long long nrows, FRow fr);
int fft_z_c2r(float2* data, int n, const float2* tw, cudaStream_t s, float* out, long long opitch, float oscale,
              long long rs, long long nrows);
// line passes: tile of outer index o starts at (o / o2n) s1 + (o % o2n) s2, element stride S
int fft_lines(float2* data, int n, int sign, const float2* tw, cudaStream_t s, LineGeom lg, int kid);
// plain n x n x P mesh, axis 1 = y, 0 = x
int fft_strided(float2* data, int n, int axis, int sign, const float2* tw, cudaStream_t s);
// interleaved force mesh (rows (ix, iy, c)): delta_k in c = 0 -> F_x, F_y, F_z in c = 0, 1, 2
// filt: optional radial transfer function T(|k|) on nodes b * fstep, b < nfilt (nullptr: none)
int fft_x_green(float2* F, int n, float gscale, float kf, const float2* tw, cudaStream_t s,
                const float* filt = nullptr, int nfilt = 0, float fstep = 1.f, bool* psi = nullptr);
// inverse y pass of the force mesh after fft_x_green: three component lines, or,
// if the x pass left Psi in component 1 (psi), F_y = IFFT_y(i k_y Psi) and
// F_z = i k_z IFFT_y(Psi) from it (kf = 2 pi / L)
int fft_y_inverse_force(float2* F, int n, const float2* tw, cudaStream_t s, bool psi, float kf);
__host__ __device__ __forceinline__ FRow force_rows(int ng) { return FRow{ng, xblock_shift(ng), 3}; }

// snap (optional): drift to an output time; rsd: also shift along z into redshift space (snap[3..5])
int launch_deposit_ex(const float* d, const float* v, const float* psi1, const float* psi2, unsigned long long* dep,
                      int nq, int ng, double box, const double* snap, int* status, cudaStream_t s, bool rsd = false);
// F: interleaved force mesh, real view, component c of (ix, iy) at ((ix n + iy) 3 + c) 2P floats
int launch_gather(const float2* F, const float* d, float* out, int nq, int ng, double box, cudaStream_t s);
int launch_gather_kick_drift(const float2* F, cola_state st, const double* row, int nq, int ng, double box, int last,
                             int pm_only, int* status, cudaStream_t s);
int launch_fix_to_delta(unsigned long long* dep, float* delta, int ng, float scale, cudaStream_t s,
                        bool clear = true);
int launch_adjoint_deposit(const float* d, const float* res, unsigned long long* fix3, int nq, int ng, double box,
                           cudaStream_t s);
int set_particle_traversal(int edge, int brick_k);  // traversal order of the particle kernels (pm.cu)

// Row bins of the PM step (pm.cu): start[ng^2 + 1] (counts, then offsets),
// sums (exclusive_scan scratch), key/rank/sorted[Np], cic[Np] (RowBins::cic).
struct BinBufs {
    int *start, *sums, *key, *rank, *sorted;
    float4* cic;
};
int launch_bins(const float* d, int nq, int ng, double box, const BinBufs& b, int* status, cudaStream_t s);
// kick + drift (and the force alone) from the partial-sum records of the
// fused c2r pass: slots float[Np][12] by sorted position, pos[p] (the bins'
// rank array after the scatter) the sorted position of particle p
int launch_slot_kick_drift(const float* slots, const int* pos, cola_state st, const double* row, int nq, int last,
                           int pm_only, int* status, cudaStream_t s);
int launch_slot_force(const float* slots, const int* pos, float* out, int nq, cudaStream_t s);
// The separate-kernel PM path deposits into the fixed-point region and its z
// r2c pass clears the counts as it reads them, so the region stays zero from
// one such step to the next.  Everything else that writes the region (the
// fused path's bins, the 2LPT scratch, the P(k) and density calls) marks it
// dirty first; clear_dep_if_dirty zeroes it only when marked.
int mark_dep_dirty(void* ws, cudaStream_t s);
int mark_dep_clean(void* ws, cudaStream_t s);
int clear_dep_if_dirty(void* ws, unsigned long long* dep, size_t count, cudaStream_t s);
// cola_checks_probe's kernel: area[index] = index if the bounds check index < n passes
int launch_checks_probe(int* area, int index, int n, int* status, cudaStream_t s);

// Fused z passes of the PM step (fft.cu, fft_fused.cuh):
// fft_z_r2c_deposit: CIC deposit of the binned particles into shared memory,
// row tile by row tile, and the r2c along z of those rows, written to
// component 0 of the force mesh (rows frow(x, y, 0)); with delta_out, delta is
// also written there unpadded (float[ng^3], C order).
int fft_z_r2c_deposit(const float* d, int nq, const RowBins& bins, float2* F, int ng, double box, float scale,
                      const float2* tw, float* delta_out, cudaStream_t s);
// fft_z_c2r_gather: c2r along z of all three force components, row tile by
// row tile in shared memory, and each binned particle's partial CIC sums from
// those rows into slots; *tx receives the tile's x rows for the kick.
int fft_z_c2r_gather(float2* F, int ng, const float* d, int nq, const RowBins& bins, float* slots, double box,
                     const float2* tw, int* tx, cudaStream_t s);
// true when both fused z passes of an n^3 mesh have warp-row forms (fft_spec_large.cu)
bool fused_passes_warp_rows(int n);
// exclusive scan of a[0..n) in place, a[n] = total; sums holds scan_sums_bytes(n) (scan.cu)
int exclusive_scan(int* a, long long n, int* sums, cudaStream_t s);
size_t scan_sums_bytes(long long n);
// one COLA node; the kick waits for before_kick when given (api.cu)
int step_node(const cola_config* cfg, cola_state* st, int32_t step, void* ws, size_t ws_bytes, cudaStream_t s,
              cudaEvent_t before_kick);

int launch_tables(const cola_config* cfg, double* table, cudaStream_t s);
int launch_snapshot_coeffs(const cola_config* cfg, double a_node, double a_out, double* snap, cudaStream_t s);
int launch_ic(const cola_config* cfg, uint64_t seed, cola_state st, void* ws, const Layout& L, cudaStream_t s);
// p2, p4 (optional, both or neither): quadrupole and hexadecapole about the z axis
int launch_power(const float2* mk, int ng, long long rs, double box, int flags, double* part, double* k, double* pk,
                 double* nmodes, int nbins, cudaStream_t s, double* p2 = nullptr, double* p4 = nullptr);
size_t power_partial_bytes(int nbins);

// learned coarse-mesh correction (learned.cu)
size_t learned_bytes(int ng, int nq);
int net_pack(const cola_net* net, cudaStream_t s);
int net_forward(const cola_net* net, char* lbase, int ng, int nq, float green, float2* F, cudaStream_t s);
int net_backward(const cola_net* net, char* lbase, int ng, int nq, double box, float green, const float2* F,
                 const float* d, const float* target, float* grad, double* loss, cudaStream_t s);
int launch_adam(float* p, const float* g, float* m, float* v, int n, int t, float lr, float b1, float b2, float eps,
                cudaStream_t s);
int launch_lsq_accumulate(const float* A, const float* y, long long len, int nb, double* ATA, double* ATy,
                          cudaStream_t s);
int launch_lsq_solve(const double* ATA, const double* ATy, int nb, double ridge, float* T, cudaStream_t s);
int launch_basis_table(float* T, int nb, int b, cudaStream_t s);

}  // namespace cola
