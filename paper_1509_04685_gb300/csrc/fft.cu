// Mixed-radix (2, 3, 4, 5, 8) 3D FFTs on the padded half-complex mesh layout,
// the pieces of the PM force of Sec. 2.2 (one forward r2c, three c2r inverses
// per step), with the Poisson solve and ik gradient fused into the x pass.
//
// Mesh layout: n x n x P complex64, P = fft_pitch(n) >= n/2 + 1 (multiple of
// 16), index (ix, iy, kz) at (ix*n + iy)*P + kz.  The real view of the same
// buffer has rows of 2P floats, real value (ix, iy, z) at (ix*n + iy)*2P + z.
// Forward passes run z (r2c), y, x; inverse passes x, y, z (c2r).
#include <cmath>

#include "cola_common.cuh"

namespace cola {

unsigned long long g_launches = 0;

bool make_plan(int n, FftPlan* p) {
    if (n < 1 || n > kMaxFft) return false;
    p->n = n;
    p->nr = 0;
    int m = n;
    const int order[5] = {8, 4, 2, 3, 5};
    for (int r : order) {
        while (m % r == 0) {
            if (p->nr >= kMaxRadices) return false;
            p->radix[p->nr++] = r;
            m /= r;
        }
    }
    return m == 1;
}

// about twelve complex elements per thread, 64 .. 512 threads (two blocks of
// ~48-register threads fit on an SM)
static int round_threads(long elems) {
    long t = (elems + 11) / 12;
    t = (t + 31) / 32 * 32;
    if (t < 64) t = 64;
    if (t > 512) t = 512;
    return (int)t;
}

// ---------------------------------------------------------------------------
// twiddles: tw[q] = exp(-2 pi i q / n), FP64 sincospi rounded once to FP32
// ---------------------------------------------------------------------------
__global__ void k_twiddles(float2* tw, int n) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    double s, c;
    sincospi(-2.0 * (double)q / (double)n, &s, &c);
    tw[q] = make_float2((float)c, (float)s);
}

int launch_twiddles(float2* tw, int n, cudaStream_t s) {
    ProfScope ps(kKSetup, s);
    k_twiddles<<<(n + 255) / 256, 256, 0, s>>>(tw, n);
    return check_launch();
}

// ---------------------------------------------------------------------------
// z pass, forward r2c.  FIX: input is the uint64 fixed-point CIC mesh (rows of
// n counts, 2^40 per particle), converted to delta = count*scale - 1 and
// cleared after reading; otherwise the input is the real view of `out`.
// A real row is packed as n/2 complex values, transformed, and unpacked with
// X[k] = E[k] + W^k O[k], E = (Z[k] + conj Z[M-k])/2, O = (Z[k] - conj Z[M-k])/(2i).
// ---------------------------------------------------------------------------
template <bool FIX>
__global__ void k_fft_z_r2c(unsigned long long* __restrict__ dep, float2* out, int n, int P, long long nrows,
                            int NR, float scale, FftPlan plan, const float2* __restrict__ tw) {
    extern __shared__ float2 sm[];
    const int M = n / 2;
    const int ls = M + 1;
    float2* sb = sm + NR * ls;
    const long long row0 = (long long)blockIdx.x * NR;
    const int T = blockDim.x;
    for (int e = threadIdx.x; e < NR * M; e += T) {
        const int l = e / M, m = e - l * M;
        const long long row = row0 + l;
        float2 v = make_float2(0.f, 0.f);
        if (row < nrows) {
            if (FIX) {
                ulonglong2* p = reinterpret_cast<ulonglong2*>(dep + row * n) + m;
                ulonglong2 c = *p;
                v = make_float2((float)c.x * scale - 1.0f, (float)c.y * scale - 1.0f);
                *p = make_ulonglong2(0ull, 0ull);
            } else {
                v = out[row * P + m];
            }
        }
        sm[l * ls + m] = v;
    }
    __syncthreads();
    const float2* Z = fft_smem(sm, sb, plan, NR, ls, 1, false, tw, 2, -1);
    for (int e = threadIdx.x; e < NR * (M + 1); e += T) {
        const int l = e / (M + 1), k = e - l * (M + 1);
        const long long row = row0 + l;
        if (row >= nrows) continue;
        const float2 a = Z[l * ls + (k == M ? 0 : k)];
        const float2 b = cconj(Z[l * ls + (k == 0 ? 0 : M - k)]);
        const float2 E = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y + b.y));
        const float2 D = csub(a, b);
        const float2 O = make_float2(0.5f * D.y, -0.5f * D.x);  // (a-b)/(2i)
        out[row * P + k] = cadd(E, cmul(__ldg(&tw[k]), O));
    }
}

// ---------------------------------------------------------------------------
// z pass, inverse c2r (unnormalised).  Z[k] = (X[k] + conj X[M-k]) +
// i (X[k] - conj X[M-k]) W^-k, z = IFFT_M(Z), x[2m] = Re z[m], x[2m+1] = Im z[m].
// Im X[0] and Im X[M] are ignored (as for a Hermitian spectrum).  Output goes
// to the real view of `data` (GENERIC = false) or to out[row*opitch + z]*oscale.
// ---------------------------------------------------------------------------
template <bool GENERIC>
__global__ void k_fft_z_c2r(float2* data, int n, int P, long long nrows, int NR, FftPlan plan,
                            const float2* __restrict__ tw, float* out, long long opitch, float oscale) {
    extern __shared__ float2 sm[];
    const int M = n / 2;
    const int ls = M + 2;
    float2* sb = sm + NR * ls;
    const long long row0 = (long long)blockIdx.x * NR;
    const int T = blockDim.x;
    for (int e = threadIdx.x; e < NR * (M + 1); e += T) {
        const int l = e / (M + 1), k = e - l * (M + 1);
        const long long row = row0 + l;
        float2 v = make_float2(0.f, 0.f);
        if (row < nrows) v = data[row * P + k];
        if (k == 0 || k == M) v.y = 0.f;
        sm[l * ls + k] = v;
    }
    __syncthreads();
    const int H = M / 2 + 1;  // pairs (k, M-k) for k = 0 .. M/2
    for (int e = threadIdx.x; e < NR * H; e += T) {
        const int l = e / H, k = e - l * H;
        float2* s = sm + l * ls;
        if (k == 0) {
            const float2 x0 = s[0], xm = s[M];
            s[0] = make_float2(x0.x + xm.x, x0.x - xm.x);
        } else {
            const float2 xk = s[k], xmk = s[M - k];
            float2 w = __ldg(&tw[k]);
            w.y = -w.y;  // W^-k
            {
                const float2 a = xk, b = cconj(xmk);
                const float2 d = cmul(csub(a, b), w);
                s[k] = make_float2(a.x + b.x - d.y, a.y + b.y + d.x);
            }
            if (M - k != k) {
                float2 w2 = __ldg(&tw[M - k]);
                w2.y = -w2.y;
                const float2 a = xmk, b = cconj(xk);
                const float2 d = cmul(csub(a, b), w2);
                s[M - k] = make_float2(a.x + b.x - d.y, a.y + b.y + d.x);
            }
        }
    }
    __syncthreads();
    const float2* Zr = fft_smem(sm, sb, plan, NR, ls, 1, false, tw, 2, +1);
    for (int e = threadIdx.x; e < NR * M; e += T) {
        const int l = e / M, m = e - l * M;
        const long long row = row0 + l;
        if (row >= nrows) continue;
        const float2 z = Zr[l * ls + m];
        if (GENERIC) {
            out[row * opitch + 2 * m] = z.x * oscale;
            out[row * opitch + 2 * m + 1] = z.y * oscale;
        } else {
            data[row * P + m] = z;
        }
    }
}

// ---------------------------------------------------------------------------
// strided complex pass along y (S = P, outer = ix) or x (S = n P, outer = iy):
// a block transforms B adjacent kz columns of one outer index.
// ---------------------------------------------------------------------------
__global__ void k_fft_strided(float2* data, int n, long long S, long long outer_stride, int ncols, int B, int nct,
                              FftPlan plan, const float2* __restrict__ tw, int sign) {
    extern __shared__ float2 sm[];
    const long long o = blockIdx.x / nct;
    const int ct = blockIdx.x - (int)(o * nct);
    const int col0 = ct * B;
    float2* base = data + o * outer_stride + col0;
    const int T = blockDim.x;
    for (int e = threadIdx.x; e < n * B; e += T) {
        const int i = e / B, c = e - i * B;
        sm[e] = (col0 + c < ncols) ? base[i * S + c] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const float2* R = fft_smem(sm, sm + n * B, plan, B, 1, B, true, tw, 1, sign);
    for (int e = threadIdx.x; e < n * B; e += T) {
        const int i = e / B, c = e - i * B;
        if (col0 + c < ncols) base[i * S + c] = R[e];
    }
}

// ---------------------------------------------------------------------------
// x pass fused with the Poisson solve and gradient (Sec. 2.2; Eq. 2 force):
// forward x FFT of delta_k, Phi_k = -green delta_k / k^2 (0 at k = 0), then for
// each component F_j,k = -i k_j Phi_k (k_j = 0 on axis j's Nyquist plane) and
// its inverse x FFT.  gscale = green / n^3 carries the c2r normalisation.
// ---------------------------------------------------------------------------
constexpr int kGreenEpt = 8;  // spectrum values each thread keeps in registers

__global__ void __launch_bounds__(768) k_fft_x_green(const float2* __restrict__ mk, float2* f0, float2* f1, float2* f2, int n, int P,
                              int B, int nct, FftPlan plan, const float2* __restrict__ tw, float gscale, float kf) {
    extern __shared__ float2 sm[];
    float2* A = sm;
    float2* W = sm + n * B;
    const int iy = blockIdx.x / nct;
    const int ct = blockIdx.x - iy * nct;
    const int col0 = ct * B;
    const int ncols = n / 2 + 1;
    const long long S = (long long)n * P;
    const long long off = (long long)iy * P + col0;
    const int T = blockDim.x;
    for (int e = threadIdx.x; e < n * B; e += T) {
        const int i = e / B, c = e - i * B;
        A[e] = (col0 + c < ncols) ? mk[off + i * S + c] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const float2* X = fft_smem(A, W, plan, B, 1, B, true, tw, 1, -1);
    // phi_e = green delta_k / (n^3 k^2) kept in registers: F_j,k = -i k_j Phi_k = i k_j phi
    const int half = n / 2;
    const float ky = kf * (float)(iy < half ? iy : iy - n);
    float2 phi[kGreenEpt];
#pragma unroll
    for (int q = 0; q < kGreenEpt; ++q) {
        const int e = threadIdx.x + q * T;
        phi[q] = make_float2(0.f, 0.f);
        if (e < n * B) {
            const int i = e / B, c = e - i * B;
            const float kx = kf * (float)(i < half ? i : i - n);
            const float kz = kf * (float)(col0 + c);
            const float k2 = kx * kx + ky * ky + kz * kz;
            phi[q] = cscale(X[e], k2 > 0.f ? gscale / k2 : 0.f);
        }
    }
    __syncthreads();
    for (int j = 0; j < 3; ++j) {
#pragma unroll
        for (int q = 0; q < kGreenEpt; ++q) {
            const int e = threadIdx.x + q * T;
            if (e < n * B) {
                const int i = e / B, c = e - i * B;
                float kj;
                if (j == 0)
                    kj = (i == half) ? 0.f : kf * (float)(i < half ? i : i - n);
                else if (j == 1)
                    kj = (iy == half) ? 0.f : ky;
                else
                    kj = (col0 + c == half) ? 0.f : kf * (float)(col0 + c);
                A[e] = make_float2(-kj * phi[q].y, kj * phi[q].x);  // i k_j phi
            }
        }
        __syncthreads();
        const float2* R = fft_smem(A, W, plan, B, 1, B, true, tw, 1, +1);
        float2* dst = (j == 0 ? f0 : (j == 1 ? f1 : f2)) + off;
        for (int e = threadIdx.x; e < n * B; e += T) {
            const int i = e / B, c = e - i * B;
            if (col0 + c < ncols) dst[i * S + c] = R[e];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// host drivers
// ---------------------------------------------------------------------------
static int z_rows_per_block(int M) {
    int nr = 4096 / M;
    if (nr < 1) nr = 1;
    if (nr > 64) nr = 64;
    return nr;
}

static bool set_smem(const void* fn, size_t bytes) {
    if (bytes <= 48 * 1024) return true;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess;
}

int fft_z_r2c(unsigned long long* dep, float2* out, int n, float scale, const float2* tw, cudaStream_t s) {
    FftPlan plan;
    if (!make_plan(n / 2, &plan)) return COLA_EUNSUPPORTED_SIZE;
    const int M = n / 2, P = fft_pitch(n);
    const int NR = z_rows_per_block(M);
    const long long nrows = (long long)n * n;
    const int T = round_threads((long)NR * M);
    const size_t smem = (size_t)2 * NR * (M + 1) * 8;
    const long long grid = (nrows + NR - 1) / NR;
    ProfScope ps(dep ? kKZr2cFix : kKZr2c, s);
    if (dep) {
        if (!set_smem((const void*)k_fft_z_r2c<true>, smem)) return COLA_ECUDA;
        k_fft_z_r2c<true><<<(unsigned)grid, T, smem, s>>>(dep, out, n, P, nrows, NR, scale, plan, tw);
    } else {
        if (!set_smem((const void*)k_fft_z_r2c<false>, smem)) return COLA_ECUDA;
        k_fft_z_r2c<false><<<(unsigned)grid, T, smem, s>>>(nullptr, out, n, P, nrows, NR, 0.f, plan, tw);
    }
    return check_launch();
}

int fft_z_c2r(float2* data, int n, const float2* tw, cudaStream_t s, float* out, long long opitch, float oscale) {
    FftPlan plan;
    if (!make_plan(n / 2, &plan)) return COLA_EUNSUPPORTED_SIZE;
    const int M = n / 2, P = fft_pitch(n);
    const int NR = z_rows_per_block(M);
    const long long nrows = (long long)n * n;
    const int T = round_threads((long)NR * M);
    const size_t smem = (size_t)2 * NR * (M + 2) * 8;
    const long long grid = (nrows + NR - 1) / NR;
    ProfScope ps(kKZc2r, s);
    if (out) {
        if (!set_smem((const void*)k_fft_z_c2r<true>, smem)) return COLA_ECUDA;
        k_fft_z_c2r<true><<<(unsigned)grid, T, smem, s>>>(data, n, P, nrows, NR, plan, tw, out, opitch, oscale);
    } else {
        if (!set_smem((const void*)k_fft_z_c2r<false>, smem)) return COLA_ECUDA;
        k_fft_z_c2r<false><<<(unsigned)grid, T, smem, s>>>(data, n, P, nrows, NR, plan, tw, nullptr, 0, 1.f);
    }
    return check_launch();
}

// adjacent kz columns per block: two ping-pong buffers of n*B complex each
static int strided_cols(int n) { return n <= 256 ? 16 : (n <= 768 ? 8 : (n <= 2048 ? 4 : 2)); }

int fft_strided(float2* data, int n, int axis, int sign, const float2* tw, cudaStream_t s) {
    FftPlan plan;
    if (!make_plan(n, &plan)) return COLA_EUNSUPPORTED_SIZE;
    const int P = fft_pitch(n);
    const int B = strided_cols(n);
    const int ncols = n / 2 + 1;
    const int nct = (ncols + B - 1) / B;
    const long long S = axis == 1 ? P : (long long)n * P;
    const long long outer_stride = axis == 1 ? (long long)n * P : P;
    const int T = round_threads((long)n * B);
    const size_t smem = (size_t)2 * n * B * 8;
    if (!set_smem((const void*)k_fft_strided, smem)) return COLA_ECUDA;
    ProfScope ps(axis == 1 ? (sign < 0 ? kKYFwd : kKYInv) : (sign < 0 ? kKXFwd : kKXInv), s);
    k_fft_strided<<<(unsigned)(n * nct), T, smem, s>>>(data, n, S, outer_stride, ncols, B, nct, plan, tw, sign);
    return check_launch();
}

int fft_x_green(const float2* mk, float2* f0, float2* f1, float2* f2, int n, float gscale, float kf,
                const float2* tw, cudaStream_t s) {
    FftPlan plan;
    if (!make_plan(n, &plan)) return COLA_EUNSUPPORTED_SIZE;
    const int P = fft_pitch(n);
    int B = strided_cols(n);
    while (B > 1 && n * B > 768 * kGreenEpt) B /= 2;
    const int ncols = n / 2 + 1;
    const int nct = (ncols + B - 1) / B;
    int T = ((n * B + kGreenEpt - 1) / kGreenEpt + 31) / 32 * 32;
    if (T < 64) T = 64;
    if (T > 768) return COLA_EUNSUPPORTED_SIZE;
    const size_t smem = (size_t)2 * n * B * 8;
    if (!set_smem((const void*)k_fft_x_green, smem)) return COLA_ECUDA;
    ProfScope ps(kKXGreen, s);
    k_fft_x_green<<<(unsigned)(n * nct), T, smem, s>>>(mk, f0, f1, f2, n, P, B, nct, plan, tw, gscale, kf);
    return check_launch();
}

}  // namespace cola
