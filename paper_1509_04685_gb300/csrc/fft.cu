// Mixed-radix (2, 3, 4, 5, 8) 3D FFTs on the padded half-complex mesh layout,
// the pieces of the PM force of Sec. 2.2 (one forward r2c, three c2r inverses
// per step), with the Poisson solve and ik gradient fused into the x pass.
//
// Mesh layout: n x n x P complex64, P = fft_pitch(n) >= n/2 + 1 (multiple of
// 16), index (ix, iy, kz) at (ix*n + iy)*P + kz.  The real view of the same
// buffer has rows of 2P floats, real value (ix, iy, z) at (ix*n + iy)*2P + z.
// Forward passes run z (r2c), y, x; inverse passes x, y, z (c2r).
#include <algorithm>
#include <cmath>

#include "fft_fused.cuh"

namespace cola {

unsigned long long g_launches = 0;
int g_last_cuda_error = 0;

bool make_plan(int n, FftPlan* p) {
    const StaticPlan sp = static_plan(n);
    if (!sp.ok) return false;
    p->n = n;
    p->nr = sp.nr;
    for (int s = 0; s < sp.nr; ++s) {
        p->radix[s] = sp.r[s];
        p->ls_div[s] = make_fastdiv(plan_ls(sp, s));
        p->nbl_div[s] = make_fastdiv(n / sp.r[s]);
    }
    return true;
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
// accessors for the z (row) passes.  Line l of a block is mesh row row0 + l.
// ---------------------------------------------------------------------------
// fixed-point CIC counts (2^40 per particle) -> delta = count*scale - 1, packed
// as complex pairs; every count is cleared after it is read.
struct FixRowLoader {
    unsigned long long* dep;
    int n;
    long long row0, nrows;
    float scale;
    template <int R>
    __device__ __forceinline__ void load(int l, int i0, int di, float2* v) const {
        const long long row = row0 + l;
        if (row >= nrows) {
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = make_float2(0.f, 0.f);
            return;
        }
        ulonglong2* p = reinterpret_cast<ulonglong2*>(dep + row * n);
        ulonglong2 c[R];
#pragma unroll
        for (int r = 0; r < R; ++r) c[r] = __ldcs(p + i0 + r * di);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            v[r] = make_float2((float)c[r].x * scale - 1.0f, (float)c[r].y * scale - 1.0f);
            __stcs(p + i0 + r * di, make_ulonglong2(0ull, 0ull));
        }
    }
};

// real rows (row pitch P complex) packed as complex pairs
struct RowLoader {
    const float2* data;
    long long rs;  // row stride (complex)
    long long row0, nrows;
    template <int R>
    __device__ __forceinline__ void load(int l, int i0, int di, float2* v) const {
        const long long row = row0 + l;
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = row < nrows ? data[row * rs + i0 + r * di] : make_float2(0.f, 0.f);
    }
};

// c2r pre-processing: Z[k] = (X[k] + conj X[M-k]) + i (X[k] - conj X[M-k]) W_n^-k,
// with Im X[0] and Im X[M] ignored.
struct C2rLoader {
    const float2* data;
    long long rs;
    int M;
    long long row0, nrows;
    const float2* tw;
    template <int R>
    __device__ __forceinline__ void load(int l, int i0, int di, float2* v) const {
        const long long row = row0 + l;
        if (row >= nrows) {
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = make_float2(0.f, 0.f);
            return;
        }
        const float2* x = data + row * rs;
        float2 a[R], bb[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int k = i0 + r * di;
            a[r] = x[k];
            bb[r] = x[M - k];
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int k = i0 + r * di;
            if (k == 0) {
                a[r].y = 0.f;
                bb[r].y = 0.f;
            }
            const float2 b = cconj(bb[r]);
            float2 w = __ldg(tw + k);
            w.y = -w.y;
            const float2 d = cmul(csub(a[r], b), w);
            v[r] = make_float2(a[r].x + b.x - d.y, a[r].y + b.y + d.x);
        }
    }
};

// z[m] written as the float pair (2m, 2m+1) of real row row0 + l
struct RowStore {
    float2* data;
    long long rs;
    long long row0, nrows;
    template <int R>
    __device__ __forceinline__ void store(int l, int i0, int di, const float2* v) const {
        const long long row = row0 + l;
        if (row >= nrows) return;
#pragma unroll
        for (int r = 0; r < R; ++r) data[row * rs + i0 + r * di] = v[r];
    }
};

// same, scaled, into a plain float array with row pitch opitch
struct RowStoreGeneric {
    float* out;
    long long opitch;
    float scale;
    long long row0, nrows;
    template <int R>
    __device__ __forceinline__ void store(int l, int i0, int di, const float2* v) const {
        const long long row = row0 + l;
        if (row >= nrows) return;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const long long q = row * opitch + 2 * (i0 + r * di);
            out[q] = v[r].x * scale;
            out[q + 1] = v[r].y * scale;
        }
    }
};

// strided tile (y or x pass): line l = column col0 + l, element i at row stride S
struct ColIO {
    float2* g;
    long long S;
    template <int R>
    __device__ __forceinline__ void load(int l, int i0, int di, float2* v) const {
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = __ldcs(g + (long long)(i0 + r * di) * S + l);
    }
    template <int R>
    __device__ __forceinline__ void store(int l, int i0, int di, const float2* v) const {
#pragma unroll
        for (int r = 0; r < R; ++r) __stcs(g + (long long)(i0 + r * di) * S + l, v[r]);
    }
};

// Psi = IFFT_x(phi) stored twice: F_y = i k_y Psi and F_z = i k_z Psi.  Along
// an x line k_y (fixed row iy) and k_z (fixed column) are constants, so they
// commute with the inverse x transform: one transform serves both components.
// x-line addressing of the blocked force mesh: element i at
// (i >> xbs) Sb + (i & (XB - 1)) Si
struct XLine {
    long long Sb, Si;
    int xbs;
    __device__ __forceinline__ long long off(int i) const {
        return (long long)(i >> xbs) * Sb + (long long)(i & ((1 << xbs) - 1)) * Si;
    }
};

struct XIO {
    float2* g;
    XLine xl;
    template <int R>
    __device__ __forceinline__ void load(int l, int i0, int di, float2* v) const {
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = __ldcs(g + xl.off(i0 + r * di) + l);
    }
    template <int R>
    __device__ __forceinline__ void store(int l, int i0, int di, const float2* v) const {
#pragma unroll
        for (int r = 0; r < R; ++r) __stcs(g + xl.off(i0 + r * di) + l, v[r]);
    }
};

struct YZStore {
    float2* fy;
    float2* fz;
    XLine xl;
    float ky;             // 0 on the y Nyquist plane
    float kf;
    int col0, half;
    template <int R>
    __device__ __forceinline__ void store(int l, int i0, int di, const float2* v) const {
        const float kz = (col0 + l == half) ? 0.f : kf * (float)(col0 + l);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const long long q = xl.off(i0 + r * di) + l;
            __stcs(fy + q, make_float2(-ky * v[r].y, ky * v[r].x));
            __stcs(fz + q, make_float2(-kz * v[r].y, kz * v[r].x));
        }
    }
};

// ---------------------------------------------------------------------------
// z pass, forward r2c.  FIX: input is the uint64 fixed-point CIC mesh (rows of
// n counts, 2^40 per particle), converted to delta = count*scale - 1 and
// cleared after reading; otherwise the input is the real view of `out`.
// A real row is packed as n/2 complex values, transformed, and unpacked with
// X[k] = E[k] + W^k O[k], E = (Z[k] + conj Z[M-k])/2, O = (Z[k] - conj Z[M-k])/(2i).
// ---------------------------------------------------------------------------
template <bool FIX>
__global__ void k_fft_z_r2c(unsigned long long* __restrict__ dep, float2* out, int n, long long rs, long long nrows,
                            int NR, float scale, FftPlan plan, const float2* __restrict__ tw, FastDiv m1div, FRow fr) {
    extern __shared__ float2 sm[];
    __shared__ long long obase[64];  // output row offsets of this block's lines
    const int M = n / 2;
    const int ls = spad(M) + 1;
    float2* sb = sm + NR * ls;
    const long long row0 = (long long)blockIdx.x * NR;
    if (threadIdx.x < NR) {
        const long long r = row0 + threadIdx.x;
        const int x = (int)(r / n), y = (int)(r - (long long)x * n);
        obase[threadIdx.x] = frow(x, y, 0, fr) * rs;
    }
    const FftGeom g{NR, ls, 1, false, 0, 2};
    const float2* Z;
    if (FIX)
        Z = fft_run_smem<-1, false>(FixRowLoader{dep, n, row0, nrows, scale}, sm, sb, plan, g, tw);
    else
        Z = fft_run_smem<-1, false>(RowLoader{out, rs, row0, nrows}, sm, sb, plan, g, tw);
    for (int e = threadIdx.x; e < NR * (M + 1); e += blockDim.x) {
        const int l = (int)fdiv((unsigned)e, m1div), k = e - l * (M + 1);
        const long long row = row0 + l;
        if (row >= nrows) continue;
        const float2 a = Z[l * ls + spad(k == M ? 0 : k)];
        const float2 b = cconj(Z[l * ls + spad(k == 0 ? 0 : M - k)]);
        const float2 E = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y + b.y));
        const float2 D = csub(a, b);
        const float2 O = make_float2(0.5f * D.y, -0.5f * D.x);  // (a-b)/(2i)
        out[obase[l] + k] = cadd(E, cmul(__ldg(&tw[k]), O));
    }
}

// ---------------------------------------------------------------------------
// z pass, inverse c2r (unnormalised): the pre-processing runs inside the first
// pass's loads and the last pass writes the real row.
// ---------------------------------------------------------------------------
template <bool GENERIC>
__global__ void k_fft_z_c2r(float2* data, int n, long long rs, long long nrows, int NR, FftPlan plan,
                            const float2* __restrict__ tw, float* out, long long opitch, float oscale) {
    extern __shared__ float2 sm[];
    const int M = n / 2;
    const int ls = spad(M) + 1;
    float2* sb = sm + NR * ls;
    const long long row0 = (long long)blockIdx.x * NR;
    const FftGeom g{NR, ls, 1, false, 0, 2};
    const C2rLoader in{data, rs, M, row0, nrows, tw};
    if (GENERIC)
        fft_run_out<+1, false>(in, RowStoreGeneric{out, opitch, oscale, row0, nrows}, sm, sb, plan, g, tw);
    else
        fft_run_out<+1, false>(in, RowStore{data, rs, row0, nrows}, sm, sb, plan, g, tw);
}

// ---------------------------------------------------------------------------
// strided complex pass along y (S = P, outer = ix) or x (S = n P, outer = iy):
// a block transforms B adjacent kz columns of one outer index, reading and
// writing global memory in its first and last passes.  Tiles never cross the
// padded row pitch P (a multiple of 16), so pad columns past n/2+1 are
// transformed too: no kernel reads them as data.
// ---------------------------------------------------------------------------
template <int SIGN>
__global__ void k_fft_strided(float2* data, int n, LineGeom lg, int B, int nct, int ntiles, FftPlan plan,
                              const float2* __restrict__ tw) {
    const long long S = lg.S;
    extern __shared__ float2 sm[];
    const int tsz = spad(n) * B;
    float2* stg = sm;  // prefetched raw tile
    float2* A = sm + tsz;
    float2* Bf = A + tsz;
    float2* tws = Bf + tsz;  // twiddle table, copied once per persistent block
    for (int q = threadIdx.x; q < n; q += blockDim.x) tws[q] = __ldg(tw + q);
    const FftGeom g{B, 1, B, true, __ffs(B) - 1, 1};
    auto tile_base = [&](int t) {
        const int o = t / nct;
        const int ct = t - o * nct;
        const int o1 = o / lg.o2n, o2 = o - o1 * lg.o2n;
        return data + o1 * lg.s1 + o2 * lg.s2 + ct * B;
    };
    int t = blockIdx.x;
    if (t < ntiles) tile_prefetch(stg, tile_base(t), n, B, S);
    for (; t < ntiles; t += gridDim.x) {
        cp_async_wait_all();
        __syncthreads();
        const int tn = t + gridDim.x;
        auto prefetch_next = [&]() {
            if (tn < ntiles) tile_prefetch(stg, tile_base(tn), n, B, S);
        };
        fft_run_out<SIGN, true>(SmemIO{stg, 1, B}, ColIO{tile_base(t), S}, A, Bf, plan, g, tws, prefetch_next);
    }
}

// ---------------------------------------------------------------------------
// x pass fused with the Poisson solve and gradient (Sec. 2.2; Eq. 2 force):
// forward x FFT of delta_k, Phi_k = -green delta_k / k^2 (0 at k = 0), and the
// force components F_j,k = -i k_j Phi_k (k_j = 0 on axis j's Nyquist plane)
// brought back along x.  gscale = green / n^3 carries the c2r normalisation,
// so with phi = gscale delta_k / k^2 (kept in registers), F_j = i k_j phi.
// Two inverse transforms per tile: i k_x phi for the x component, and phi
// itself, whose transform is scaled by i k_y and i k_z on the way out.  The
// next tile's delta_k is prefetched with cp.async while this one is computed.
// ---------------------------------------------------------------------------
constexpr int kGreenEpt = 12;  // spectrum values each thread keeps in registers

__global__ void __launch_bounds__(512) k_fft_x_green(const float2* mk, float2* f0, float2* f1, float2* f2,
                                                     int n, long long RS, XLine xl, int B, int nct, int ntiles,
                                                     FftPlan plan, const float2* __restrict__ tw, float gscale,
                                                     float kf, const float* __restrict__ filt, int nfilt,
                                                     float fstep) {
    extern __shared__ float2 sm[];
    const int tsz = spad(n) * B;
    float2* stg = sm;
    float2* A = sm + tsz;
    float2* W = A + tsz;
    float2* tws = W + tsz;  // twiddle table, copied once per persistent block
    for (int q = threadIdx.x; q < n; q += blockDim.x) tws[q] = __ldg(tw + q);
    const int T = blockDim.x;
    const int bs = __ffs(B) - 1;
    const int half = n / 2;
    const FftGeom g{B, 1, B, true, bs, 1};
    // RS: offset of one y row (the x lines of the tile start at iy RS)
    auto tile_off = [&](int t) {
        const int iy = t / nct;
        const int ct = t - iy * nct;
        return (long long)iy * RS + ct * B;
    };
    auto prefetch = [&](const float2* g0) {
        const int hb = B >> 1;
        const int hs = __ffs(hb) - 1;
        for (int e = threadIdx.x; e < n * hb; e += blockDim.x) {
            const int i = e >> hs, c = (e & (hb - 1)) << 1;
            cp_async16(stg + c + spad(i) * B, g0 + xl.off(i) + c);
        }
        cp_async_commit();
    };
    int t = blockIdx.x;
    if (t < ntiles) prefetch(mk + tile_off(t));
    for (; t < ntiles; t += gridDim.x) {
        const int iy = t / nct;
        const int col0 = (t - iy * nct) * B;
        const long long off = (long long)iy * RS + col0;
        cp_async_wait_all();
        __syncthreads();
        const int tn = t + gridDim.x;
        auto prefetch_next = [&]() {
            if (tn < ntiles) prefetch(mk + tile_off(tn));
        };
        const float2* X = fft_run_smem<-1, true>(SmemIO{stg, 1, B}, A, W, plan, g, tws, prefetch_next);
        const float ky = kf * (float)(iy < half ? iy : iy - n);
        float2 phi[kGreenEpt];
#pragma unroll
        for (int q = 0; q < kGreenEpt; ++q) {
            const int e = threadIdx.x + q * T;
            phi[q] = make_float2(0.f, 0.f);
            if (e < n * B) {
                const int i = e >> bs, c = e & (B - 1);
                const float kx = kf * (float)(i < half ? i : i - n);
                const float kz = kf * (float)(col0 + c);
                const float k2 = kx * kx + ky * ky + kz * kz;
                float gk = k2 > 0.f ? gscale / k2 : 0.f;
                if (filt) {
                    // learned radial transfer T(|k|), piecewise linear on nodes b * fstep
                    const float u = sqrtf(k2) / fstep;
                    int b = (int)u;
                    if (b > nfilt - 2) b = nfilt - 2;
                    const float f = fminf(u - (float)b, 1.f);
                    gk *= (1.f - f) * filt[b] + f * filt[b + 1];
                }
                phi[q] = cscale(X[c + spad(i) * B], gk);
            }
        }
        __syncthreads();
        const float ky_eff = (iy == half) ? 0.f : ky;
        for (int j = 0; j < 2; ++j) {
            // j = 0: x component, IFFT_x(i k_x phi); j = 1: Psi = IFFT_x(phi) for y and z
#pragma unroll
            for (int q = 0; q < kGreenEpt; ++q) {
                const int e = threadIdx.x + q * T;
                if (e < n * B) {
                    const int i = e >> bs, c = e & (B - 1);
                    if (j == 0) {
                        const float kx = (i == half) ? 0.f : kf * (float)(i < half ? i : i - n);
                        A[c + spad(i) * B] = make_float2(-kx * phi[q].y, kx * phi[q].x);  // i k_x phi
                    } else {
                        A[c + spad(i) * B] = phi[q];
                    }
                }
            }
            __syncthreads();
            if (j == 0)
                fft_run_out<+1, true>(SmemIO{A, 1, B}, XIO{f0 + off, xl}, W, A, plan, g, tws);
            else
                fft_run_out<+1, true>(SmemIO{A, 1, B}, YZStore{f1 + off, f2 + off, xl, ky_eff, kf, col0, half}, W,
                                      A, plan, g, tws);
        }
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

// Raise a kernel's dynamic shared-memory limit once per size (also keeps the
// attribute call out of stream captures after the first, uncaptured use).
bool set_smem(const void* fn, size_t bytes) {
    // the 48 KB a launch may take without the attribute covers static and
    // dynamic shared memory together; the kernels' static arrays stay far below 8 KB
    if (bytes + 8 * 1024 <= 48 * 1024) return true;
    static const void* fns[64];
    static size_t done[64];
    static int nf = 0;
    for (int i = 0; i < nf; ++i)
        if (fns[i] == fn && done[i] >= bytes) return true;
    const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) {
        g_last_cuda_error = (int)e;
        cudaGetLastError();
        return false;
    }
    for (int i = 0; i < nf; ++i)
        if (fns[i] == fn) {
            done[i] = bytes;
            return true;
        }
    if (nf < 64) {
        fns[nf] = fn;
        done[nf++] = bytes;
    }
    return true;
}

// threads: about one butterfly of the first (largest-radix) pass per thread
static int pass_threads(const FftPlan& plan, long lines) {
    long t = plan.n / plan.radix[0] * lines;
    t = (t + 31) / 32 * 32;
    if (t < 128) t = 128;
    if (t > 256) t = 256;
    return (int)t;
}

int fft_z_r2c(unsigned long long* dep, float2* out, int n, float scale, const float2* tw, cudaStream_t s,
              long long rs, long long nrows, FRow fr) {
    FftPlan plan;
    if (!make_plan(n / 2, &plan)) return COLA_EUNSUPPORTED_SIZE;
    const int M = n / 2;
    const int NR = z_rows_per_block(M);
    const int T = pass_threads(plan, NR);
    const size_t smem = (size_t)2 * NR * (spad(M) + 1) * 8;
    const long long grid = (nrows + NR - 1) / NR;
    ProfScope ps(dep ? kKZr2cFix : kKZr2c, s);
    int rc = COLA_OK;
    if (dep && launch_z_r2c_fix_static(dep, out, n, rs, nrows, scale, tw, fr, s, &rc)) return rc;
    if (dep) {
        if (!set_smem((const void*)k_fft_z_r2c<true>, smem)) return COLA_ECUDA;
        k_fft_z_r2c<true><<<(unsigned)grid, T, smem, s>>>(dep, out, n, rs, nrows, NR, scale, plan, tw,
                                                           make_fastdiv(M + 1), fr);
    } else {
        if (!set_smem((const void*)k_fft_z_r2c<false>, smem)) return COLA_ECUDA;
        k_fft_z_r2c<false><<<(unsigned)grid, T, smem, s>>>(nullptr, out, n, rs, nrows, NR, 0.f, plan, tw,
                                                            make_fastdiv(M + 1), fr);
    }
    return check_launch();
}

int fft_z_c2r(float2* data, int n, const float2* tw, cudaStream_t s, float* out, long long opitch, float oscale,
              long long rs, long long nrows) {
    FftPlan plan;
    if (!make_plan(n / 2, &plan)) return COLA_EUNSUPPORTED_SIZE;
    const int M = n / 2;
    const int NR = z_rows_per_block(M);
    const int T = pass_threads(plan, NR);
    const size_t smem = (size_t)2 * NR * (spad(M) + 1) * 8;
    const long long grid = (nrows + NR - 1) / NR;
    ProfScope ps(kKZc2r, s);
    int rc = COLA_OK;
    if (!out && launch_z_c2r_static(data, n, rs, nrows, tw, s, &rc)) return rc;
    if (out) {
        if (!set_smem((const void*)k_fft_z_c2r<true>, smem)) return COLA_ECUDA;
        k_fft_z_c2r<true><<<(unsigned)grid, T, smem, s>>>(data, n, rs, nrows, NR, plan, tw, out, opitch, oscale);
    } else {
        if (!set_smem((const void*)k_fft_z_c2r<false>, smem)) return COLA_ECUDA;
        k_fft_z_c2r<false><<<(unsigned)grid, T, smem, s>>>(data, n, rs, nrows, NR, plan, tw, nullptr, 0, 1.f);
    }
    return check_launch();
}

// ---------------------------------------------------------------------------
// fused z passes of the PM step, runtime forms (fft_fused.cuh has the layout
// of the tiles and slots and the compile-time forms)
// ---------------------------------------------------------------------------
// fixed-point counts staged in shared memory (rows of n) -> packed complex
// pairs of delta = count scale - 1
struct SmemFixLoader {
    const unsigned long long* cnt;
    int n;
    float scale;
    template <int R>
    __device__ __forceinline__ void load(int l, int i0, int di, float2* v) const {
        const ulonglong2* x = reinterpret_cast<const ulonglong2*>(cnt + (size_t)l * n);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const ulonglong2 c = x[i0 + r * di];
            v[r] = make_float2((float)c.x * scale - 1.0f, (float)c.y * scale - 1.0f);
        }
    }
};

// one tile of ty rows (x, y0 .. y0 + ty - 1) per block
__global__ void k_fft_z_r2c_dep(const float* __restrict__ d, int nq, long long np, float inv_cell, RowBins bins,
                                float2* out, int n, long long rs, int ty, float scale, FftPlan plan,
                                const float2* __restrict__ tw, FastDiv m1div, FRow fr, float* __restrict__ delta_out) {
    extern __shared__ float2 sm[];
    __shared__ long long obase[64];
    __shared__ int beg[kMaxTileBins], pre[kMaxTileBins + 1], bxy[kMaxTileBins];
    const int M = n / 2;
    const int ls = spad(M) + 1;
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(sm);
    float2* a = sm + ty * n;
    float2* b = a + ty * ls;
    const int tpx = n / ty;
    const int x = blockIdx.x / tpx, y0 = (blockIdx.x - x * tpx) * ty;
    for (int e = threadIdx.x; e < ty * n; e += blockDim.x) cnt[e] = 0ull;
    if (threadIdx.x < ty) obase[threadIdx.x] = frow(x, y0 + threadIdx.x, 0, fr) * rs;
    const int nb = 2 * (ty + 1);
    const int total = tile_bins(
        bins, nb, n, [&](int bb) { return (wrap(x - 1 + bb / (ty + 1), n) << 16) | wrap(y0 - 1 + bb % (ty + 1), n); },
        beg, pre, bxy);
    tile_deposit(bins, beg, pre, bxy, nb, total, n, x, y0, ty, cnt);
    __syncthreads();
    if (delta_out) {
        float* o = delta_out + ((long long)x * n + y0) * n;
        for (int e = threadIdx.x; e < ty * n; e += blockDim.x) o[e] = (float)cnt[e] * scale - 1.0f;
    }
    const FftGeom g{ty, ls, 1, false, 0, 2};
    const float2* Z = fft_run_smem<-1, false>(SmemFixLoader{cnt, n, scale}, a, b, plan, g, tw);
    for (int e = threadIdx.x; e < ty * (M + 1); e += blockDim.x) {
        const int l = (int)fdiv((unsigned)e, m1div), k = e - l * (M + 1);
        const float2 za = Z[l * ls + spad(k == M ? 0 : k)];
        const float2 zb = cconj(Z[l * ls + spad(k == 0 ? 0 : M - k)]);
        const float2 E = make_float2(0.5f * (za.x + zb.x), 0.5f * (za.y + zb.y));
        const float2 D = csub(za, zb);
        const float2 O = make_float2(0.5f * D.y, -0.5f * D.x);
        out[obase[l] + k] = cadd(E, cmul(__ldg(&tw[k]), O));
    }
}

// one tile of the 3 tx force rows of x_first .. x_first + tx - 1 at one y per block
__global__ void k_fft_z_c2r_gather(const float2* __restrict__ data, int n, long long rs, int tx, FftPlan plan,
                                   const float2* __restrict__ tw, FRow fr, const float* __restrict__ d, int nq,
                                   long long np, float inv_cell, RowBins bins, float* __restrict__ slots) {
    extern __shared__ float2 sm[];
    __shared__ int beg[kMaxTileBins], pre[kMaxTileBins + 1], bxy[kMaxTileBins];
    const int M = n / 2;
    const int ls = spad(M) + 1;
    const int nr = 3 * tx;
    float2* sb = sm + nr * ls;
    const int xg = blockIdx.x / n, y = blockIdx.x - xg * n, x_first = xg * tx;
    const long long row0 = frow(x_first, y, 0, fr);
    const int nb = 2 * (tx + 1);
    const int total = tile_bins(
        bins, nb, n,
        [&](int bb) { return (wrap(x_first - 1 + bb % (tx + 1), n) << 16) | wrap(y - 1 + bb / (tx + 1), n); }, beg,
        pre, bxy);
    const FftGeom g{nr, ls, 1, false, 0, 2};
    const float2* Z = fft_run_smem<+1, false>(C2rLoader{data, rs, M, row0, row0 + nr, tw}, sm, sb, plan, g, tw);
    tile_gather(bins, beg, pre, bxy, nb, total, np, n, x_first, tx, y, Z, ls, slots);
}

int fft_z_r2c_deposit(const float* d, int nq, const RowBins& bins, float2* F, int ng, double box, float scale,
                      const float2* tw, float* delta_out, cudaStream_t s) {
    FftPlan plan;
    if (!make_plan(ng / 2, &plan)) return COLA_EUNSUPPORTED_SIZE;
    const FRow fr = force_rows(ng);
    const long long P = fft_pitch(ng);
    const float inv_cell = (float)((double)ng / box);
    ProfScope ps(kKDepR2c, s);
    int rc = COLA_OK;
    if (launch_z_r2c_dep_static(d, nq, inv_cell, bins, F, ng, P, scale, tw, fr, delta_out, s, &rc)) return rc;
    const int M = ng / 2;
    // rows per tile: a power of two dividing ng, at most the runtime z pass's
    // rows per block and ng / 2 (the tile's 2 (ty + 1) bins stay distinct)
    const int want = std::min(std::min(z_rows_per_block(M), 64), ng / 2);
    int ty = 1;
    while (2 * ty <= want && ng % (2 * ty) == 0) ty *= 2;
    const size_t smem = (size_t)ty * ng * 8 + (size_t)2 * ty * (spad(M) + 1) * 8;
    const int T = pass_threads(plan, ty);
    const long long grid = (long long)ng * (ng / ty);
    if (!set_smem((const void*)k_fft_z_r2c_dep, smem)) return COLA_ECUDA;
    k_fft_z_r2c_dep<<<(unsigned)grid, T, smem, s>>>(d, nq, (long long)nq * nq * nq, inv_cell, bins, F, ng, P, ty,
                                                     scale, plan, tw, make_fastdiv(M + 1), fr, delta_out);
    return check_launch();
}

int fft_z_c2r_gather(float2* F, int ng, const float* d, int nq, const RowBins& bins, float* slots, double box,
                     const float2* tw, int* tx, cudaStream_t s) {
    FftPlan plan;
    if (!make_plan(ng / 2, &plan)) return COLA_EUNSUPPORTED_SIZE;
    const FRow fr = force_rows(ng);
    const long long P = fft_pitch(ng);
    const float inv_cell = (float)((double)ng / box);
    ProfScope ps(kKC2rGather, s);
    int rc = COLA_OK;
    if (launch_z_c2r_gather_static(F, ng, P, tw, fr, d, nq, inv_cell, bins, slots, tx, s, &rc)) return rc;
    // x rows per tile: divides the x-block of the force layout, at most 4 and ng / 2
    int t = std::min(std::min(1 << fr.xbs, 4), ng / 2);
    *tx = t;
    const int M = ng / 2;
    const size_t smem = (size_t)2 * 3 * t * (spad(M) + 1) * 8;
    const int T = pass_threads(plan, 3 * t);
    const long long grid = (long long)(ng / t) * ng;
    if (!set_smem((const void*)k_fft_z_c2r_gather, smem)) return COLA_ECUDA;
    k_fft_z_c2r_gather<<<(unsigned)grid, T, smem, s>>>(F, ng, P, t, plan, tw, fr, d, nq, (long long)nq * nq * nq,
                                                        inv_cell, bins, slots);
    return check_launch();
}

// adjacent kz columns per block: the autotuned width if cola_fft_autotune ran
// for this size, else a default that keeps the three tile buffers near 100 KB
extern int g_tile_choice[kMaxFft + 1];
static int strided_cols(int n) {
    if (n <= kMaxFft && g_tile_choice[n]) return g_tile_choice[n];
    if (const int b = static_tile(n)) return b;
    return n <= 256 ? 16 : (n <= 768 ? 8 : (n <= 2048 ? 4 : 2));
}

// a column width the runtime engine (three tile buffers) can run
static bool runtime_tile_fits(int n, int B) { return (size_t)(3 * spad(n) * B + n) * 8 <= 220 * 1024; }

static int g_num_sms = 0;
int num_sms() {
    if (!g_num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) g_num_sms = 132;
    }
    return g_num_sms;
}

// Persistent blocks: three tile buffers (prefetch + ping-pong), blocks per SM
// from the shared-memory budget.
int persistent_grid(size_t smem, int ntiles) { return persistent_grid(smem, ntiles, 1 << 20); }

int persistent_grid(size_t smem, int ntiles, int max_per_sm) {
    int per_sm = (int)((227 * 1024) / (smem + 1024));
    if (per_sm > max_per_sm) per_sm = max_per_sm;
    if (per_sm < 1) per_sm = 1;
    int grid = num_sms() * per_sm;
    return grid < ntiles ? grid : ntiles;
}

int fft_lines(float2* data, int n, int sign, const float2* tw, cudaStream_t s, LineGeom lg, int kid) {
    FftPlan plan;
    if (!make_plan(n, &plan)) return COLA_EUNSUPPORTED_SIZE;
    const int B = strided_cols(n);
    const int nct = (n / 2 + 1 + B - 1) / B;
    const long long ntl = (long long)lg.nouter * nct;
    if (ntl > 0x7fffffff) return COLA_EUNSUPPORTED_SIZE;
    const int ntiles = (int)ntl;
    ProfScope ps(kid, s);
    int rc = COLA_OK;
    if (launch_strided_static(data, n, B, sign, lg, nct, ntiles, tw, s, &rc)) return rc;
    if (!runtime_tile_fits(n, B)) return COLA_EUNSUPPORTED_SIZE;
    int T = pass_threads(plan, B) * 2;
    const size_t smem = ((size_t)3 * spad(n) * B + n) * 8;
    auto kern = sign < 0 ? k_fft_strided<-1> : k_fft_strided<+1>;
    if (!set_smem((const void*)kern, smem)) return COLA_ECUDA;
    kern<<<persistent_grid(smem, ntiles), T, smem, s>>>(data, n, lg, B, nct, ntiles, plan, tw);
    return check_launch();
}

int fft_strided(float2* data, int n, int axis, int sign, const float2* tw, cudaStream_t s) {
    const long long P = fft_pitch(n);
    const LineGeom lg = axis == 1 ? LineGeom{P, n, 1, (long long)n * P, 0} : LineGeom{(long long)n * P, n, 1, P, 0};
    return fft_lines(data, n, sign, tw, s, lg,
                     axis == 1 ? (sign < 0 ? kKYFwd : kKYInv) : (sign < 0 ? kKXFwd : kKXInv));
}

int fft_x_green(float2* F, int n, float gscale, float kf, const float2* tw, cudaStream_t s, const float* filt,
                int nfilt, float fstep, bool* psi) {
    if (psi) *psi = false;
    FftPlan plan;
    if (!make_plan(n, &plan)) return COLA_EUNSUPPORTED_SIZE;
    const long long P = fft_pitch(n);
    const int bg = static_green_tile(n);
    int B = (n <= kMaxFft && g_tile_choice[n]) || !bg ? strided_cols(n) : bg;
    ProfScope ps(kKXGreen, s);
    int rc = COLA_OK;
    {
        const int nct = (n / 2 + 1 + B - 1) / B;
        if (launch_x_green_static(F, n, B, nct, n * nct, tw, gscale, kf, filt, nfilt, fstep, s, &rc)) {
            if (psi) *psi = true;  // the specialised passes leave Psi in component 1
            return rc;
        }
    }
    while (B > 2 && (n * B > 512 * kGreenEpt || !runtime_tile_fits(n, B))) B /= 2;
    const int nct = (n / 2 + 1 + B - 1) / B;
    const int ntiles = n * nct;
    int T = ((n * B + kGreenEpt - 1) / kGreenEpt + 31) / 32 * 32;
    if (T < 64) T = 64;
    if (T > 512) return COLA_EUNSUPPORTED_SIZE;
    const size_t smem = ((size_t)3 * spad(n) * B + n) * 8;
    if (!set_smem((const void*)k_fft_x_green, smem)) return COLA_ECUDA;
    // interleaved, x-blocked force mesh: rows frow(x, y, c) of P complex, delta_k in c = 0
    const FRow fr = force_rows(n);
    const int XB = 1 << fr.xbs;
    const XLine xl{3ll * XB * n * P, 3 * P, fr.xbs};
    k_fft_x_green<<<persistent_grid(smem, ntiles), T, smem, s>>>(F, F, F + P, F + 2 * P, n, 3ll * XB * P, xl, B, nct,
                                                                  ntiles, plan, tw, gscale, kf, filt, nfilt, fstep);
    return check_launch();
}

// F_y = i k_y Psi and F_z = i k_z Psi from Psi in component 1, for tile widths
// without a specialised Psi y pass
__global__ void k_expand_psi(float2* F, int n, int P, int xbs, float kf) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n2 = (long long)n * n;
    if (e >= n2 * (n / 2 + 1)) return;
    const int kz = (int)(e % (n / 2 + 1));
    const long long r = e / (n / 2 + 1);
    const int x = (int)(r / n), y = (int)(r - (long long)x * n);
    const FRow fr{n, xbs, 3};
    float2* f1 = F + frow(x, y, 1, fr) * P + kz;
    float2* f2 = F + frow(x, y, 2, fr) * P + kz;
    const float ky = (y == n / 2) ? 0.f : kf * (float)(y < n / 2 ? y : y - n);
    const float kzf = (kz == n / 2) ? 0.f : kf * (float)kz;
    const float2 v = *f1;
    *f1 = make_float2(-ky * v.y, ky * v.x);
    *f2 = make_float2(-kzf * v.y, kzf * v.x);
}

int fft_y_inverse_force(float2* F, int n, const float2* tw, cudaStream_t s, bool psi, float kf) {
    ProfScope ps(kKYInv, s);
    const long long P = fft_pitch(n);
    const FRow fr = force_rows(n);
    const long long XB = 1ll << fr.xbs;
    const LineGeom all3{3 * XB * P, 3 * n, (int)(3 * XB), 3 * XB * n * P, P};
    if (!psi) return fft_lines(F, n, +1, tw, s, all3, -1);
    FftPlan plan;
    if (!make_plan(n, &plan)) return COLA_EUNSUPPORTED_SIZE;
    const int B = strided_cols(n);
    const int nct = (n / 2 + 1 + B - 1) / B;
    // lines of one component: outer x = xb XB + xi
    const LineGeom one{3 * XB * P, n, (int)XB, 3 * XB * n * P, 3 * P};
    int rc = COLA_OK;
    if ((long long)n * nct <= 0x7fffffff &&
        launch_y_psi_static(F + P, n, B, one, P, nct, n * nct, tw, kf, s, &rc)) {
        if (rc) return rc;
        return fft_lines(F, n, +1, tw, s, one, -1);
    }
    const long long ne = (long long)n * n * (n / 2 + 1);
    k_expand_psi<<<(unsigned)((ne + 255) / 256), 256, 0, s>>>(F, n, (int)P, fr.xbs, kf);
    if ((rc = check_launch())) return rc;
    return fft_lines(F, n, +1, tw, s, all3, -1);
}

}  // namespace cola
