// Internal definitions shared by the translation units of the COLA library:
// complex helpers, the shared-memory mixed-radix FFT engine, the workspace
// layout and the host-side launch helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cola.h"

namespace cola {

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

// ---------------------------------------------------------------------------
// FFT plan: n = product of radices (applied in order), n <= kMaxFft
// ---------------------------------------------------------------------------
constexpr int kMaxFft = 4096;   // largest line length
constexpr int kMaxRadices = 16;

struct FftPlan {
    int n;
    int nr;
    int radix[kMaxRadices];
};

// Factor n into radices 8, 4, 2, 3, 5 (largest powers of two first).
// Returns false if n has another prime factor or is out of range.
bool make_plan(int n, FftPlan* p);

// One Stockham autosort pass (Govindaraju et al. 2008 "expand" form) over nl
// lines of length n held in shared memory, from src to dst: element i of line
// l at buf[l*ls + i*es].  Ls = product of the radices already applied;
// tw[q * twmul] = exp(-2 pi i q / n) for q < n.
//   butterfly j (0 <= j < n/R), k = j mod Ls:
//   v_r = src[j + r n/R] * W_{Ls R}^{r k},  v = DFT_R(v),
//   dst[(j / Ls) Ls R + k + r Ls] = v_r.
template <int R>
__device__ __forceinline__ void stockham_pass(const float2* __restrict__ src, float2* __restrict__ dst, int n, int nl,
                                              int ls, int es, bool line_fast, int Ls, const float2* __restrict__ tw,
                                              int twmul, int sign) {
    const int nbl = n / R;
    const int nb = nbl * nl;
    const int twstep = (n / (Ls * R)) * twmul;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        int l, j;
        if (line_fast) {
            l = b % nl;
            j = b / nl;
        } else {
            j = b % nbl;
            l = b / nbl;
        }
        const int k = j % Ls;
        const float2* s = src + l * ls;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = s[(j + r * nbl) * es];
        if (Ls > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = __ldg(&tw[r * k * twstep]);
                if (sign > 0) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        SmallDft<R>::run(v, sign);
        float2* d = dst + l * ls + ((j / Ls) * Ls * R + k) * es;
#pragma unroll
        for (int r = 0; r < R; ++r) d[r * Ls * es] = v[r];
    }
    __syncthreads();
}

// Full FFT of nl lines in shared memory, ping-ponging between a and b (the
// caller has synchronised after filling a).  Returns the buffer holding the
// result; returns synchronised.
__device__ __forceinline__ float2* fft_smem(float2* a, float2* b, const FftPlan& plan, int nl, int ls, int es,
                                            bool line_fast, const float2* __restrict__ tw, int twmul, int sign) {
    int Ls = 1;
    for (int s = 0; s < plan.nr; ++s) {
        const int R = plan.radix[s];
        switch (R) {
            case 8: stockham_pass<8>(a, b, plan.n, nl, ls, es, line_fast, Ls, tw, twmul, sign); break;
            case 4: stockham_pass<4>(a, b, plan.n, nl, ls, es, line_fast, Ls, tw, twmul, sign); break;
            case 2: stockham_pass<2>(a, b, plan.n, nl, ls, es, line_fast, Ls, tw, twmul, sign); break;
            case 3: stockham_pass<3>(a, b, plan.n, nl, ls, es, line_fast, Ls, tw, twmul, sign); break;
            default: stockham_pass<5>(a, b, plan.n, nl, ls, es, line_fast, Ls, tw, twmul, sign); break;
        }
        float2* t = a;
        a = b;
        b = t;
        Ls *= R;
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
constexpr size_t kHdrSnap = 128;          // 3 doubles: snapshot drift coefficients (dr, dD1, dD2)
constexpr size_t kHdrGrowthScratch = 256; // small FP64 scratch for the snapshot growth call
constexpr size_t kHdrTable = 4096;        // kMaxSteps x kTableCols doubles
constexpr size_t kHdrTwiddle = 262144;    // 3 slots of kMaxFft float2
constexpr size_t kHdrBytes = 524288;

enum TwSlot { kTwMesh = 0, kTwLagr = 1, kTwScratch = 2 };

struct Layout {
    size_t dep;        // uint64 fixed-point CIC mesh, ng^3 (zero between calls)
    size_t mk;         // complex mesh ng x ng x P
    size_t force[3];   // three complex/real meshes ng x ng x P
    size_t ic;         // 2LPT scratch: 7 complex meshes of nq x nq x Pq (aliases dep..)
    size_t pk_part;    // P(k) per-block partial sums (aliases force[0])
    size_t total;
};

inline int fft_pitch(int n) {
    int h = n / 2 + 1;
    return (h + 15) / 16 * 16;
}
inline size_t mesh_bytes(int n) { return (size_t)n * n * fft_pitch(n) * 8; }
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
bool layout_for(const cola_config* cfg, Layout* L);

inline char* wsp(void* ws, size_t off) { return static_cast<char*>(ws) + off; }
inline int* status_ptr(void* ws) { return reinterpret_cast<int*>(wsp(ws, kHdrStatus)); }
inline double* table_ptr(void* ws) { return reinterpret_cast<double*>(wsp(ws, kHdrTable)); }
inline float2* twiddle_ptr(void* ws, int slot) {
    return reinterpret_cast<float2*>(wsp(ws, kHdrTwiddle + (size_t)slot * kMaxFft * 8));
}

// device status latch
__device__ __forceinline__ void set_status(int* status, int code) { atomicCAS(status, 0, code); }

// ---------------------------------------------------------------------------
// per-kernel event timing (prof.cu): a ProfScope around each launch
// ---------------------------------------------------------------------------
enum KernelId {
    kKDeposit = 0, kKZr2cFix, kKZr2c, kKYFwd, kKXFwd, kKXGreen, kKYInv, kKXInv, kKZc2r, kKGatherKD, kKGather,
    kKFixToDelta, kKPkShells, kKPkReduce, kKIc, kKSetup, kNumKernelIds
};
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
inline int check_launch() {
    g_launches++;
    return cudaGetLastError() == cudaSuccess ? COLA_OK : COLA_ECUDA;
}

int launch_twiddles(float2* tw, int n, cudaStream_t s);
int fft_z_r2c(unsigned long long* dep, float2* out, int n, float scale, const float2* tw, cudaStream_t s);
int fft_z_c2r(float2* data, int n, const float2* tw, cudaStream_t s, float* out, long long opitch, float oscale);
int fft_strided(float2* data, int n, int axis, int sign, const float2* tw, cudaStream_t s);
int fft_x_green(const float2* mk, float2* f0, float2* f1, float2* f2, int n, float gscale, float kf,
                const float2* tw, cudaStream_t s);

int launch_deposit_ex(const float* d, const float* v, const float* psi1, const float* psi2, unsigned long long* dep,
                      int nq, int ng, double box, const double* snap, int* status, cudaStream_t s);
int launch_gather(const float2* f0, const float2* f1, const float2* f2, const float* d, float* out, int nq, int ng,
                  double box, cudaStream_t s);
int launch_gather_kick_drift(const float2* f0, const float2* f1, const float2* f2, cola_state st, const double* row,
                             int nq, int ng, double box, int last, int pm_only, int* status, cudaStream_t s);
int launch_fix_to_delta(unsigned long long* dep, float* delta, int ng, float scale, cudaStream_t s);

int launch_tables(const cola_config* cfg, double* table, cudaStream_t s);
int launch_snapshot_coeffs(const cola_config* cfg, double a_node, double a_out, double* snap, cudaStream_t s);
int launch_ic(const cola_config* cfg, uint64_t seed, cola_state st, void* ws, const Layout& L, cudaStream_t s);
int launch_power(const float2* mk, int ng, double box, int flags, double* part, double* k, double* pk,
                 double* nmodes, int nbins, cudaStream_t s);
size_t power_partial_bytes(int nbins);

}  // namespace cola
