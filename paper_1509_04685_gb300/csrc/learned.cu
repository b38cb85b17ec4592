// Learned coarse-mesh force correction (not in the paper): a 3-layer circular
// 3x3x3 convolution net on the PM_grid = 1 mesh, input channels
// (delta, F_x/g, F_y/g, F_z/g) with g = 3/2 Om/a, output the residual force
// / g added to the force mesh.  BF16 weights and activations, FP32 accumulation
// on tensor cores (mma.sync m16n8k16): each tap of the stencil is one K = C_in
// slice of an implicit GEMM over voxels.
//
// Layouts: activations channels-last bf16 [v][C], v = (x N + y) N + z;
// forward weights bf16 [tap][co][ci] (ci contiguous), tap = 9 tx + 3 ty + tz,
// the stencil reading x[v + t - 1] (cross-correlation, periodic).
#include <cuda_bf16.h>

#include "cola_common.cuh"

namespace cola {

typedef __nv_bfloat16 bf16;

// brick of output voxels per block: 4 (x) x 8 (y) x 16 (z) = 32 warp tiles of 16 voxels
constexpr int kBx = 4, kBy = 8, kBz = 16;
constexpr int kHx = kBx + 2, kHy = kBy + 2, kHz = kBz + 2;
constexpr int kConvWarps = 8;

__device__ __forceinline__ void mma_bf16_16816(float* c, const unsigned* a, const unsigned* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

enum ConvEpi { kEpiBiasRelu = 0, kEpiAddForce = 1, kEpiMask = 2 };

// Forward stencil conv (also the data gradient, with flipped/transposed
// weights).  CIN = 16 (inputs padded with zero channels), NT = number of 8-wide
// output channel tiles (COUT = 8 NT).
//   kEpiBiasRelu: out[v][co] = bf16(relu(acc + bias))
//   kEpiAddForce: F[((x N + y) 3 + c) P2 + z] += scale (acc + bias), c < 3 (force-mesh real view)
//   kEpiMask:     out[v][co] = bf16(acc * (mask[v][co] > 0))
template <int NT, int EPI>
__global__ void __launch_bounds__(kConvWarps * 32) k_conv(const bf16* __restrict__ x, const bf16* __restrict__ w,
                                                          const float* __restrict__ bias, int N, bf16* out,
                                                          const bf16* __restrict__ mask, float* F, long long P2,
                                                          float scale) {
    constexpr int CIN = 16, COUT = 8 * NT;
    __shared__ __align__(16) bf16 sx[kHx * kHy * kHz * CIN];
    __shared__ __align__(16) bf16 sw[27 * COUT * CIN];
    const int nbz = N / kBz, nby = N / kBy;
    int b = blockIdx.x;
    const int bz = b % nbz;
    b /= nbz;
    const int by = b % nby;
    const int bx = b / nby;
    const int x0 = bx * kBx - 1, y0 = by * kBy - 1, z0 = bz * kBz - 1;
    // halo brick: 16-byte chunks of 8 channels
    for (int e = threadIdx.x; e < kHx * kHy * kHz * 2; e += blockDim.x) {
        const int half = e & 1;
        const int hv = e >> 1;
        const int hz = hv % kHz, hy = (hv / kHz) % kHy, hx = hv / (kHz * kHy);
        const long long v = ((long long)wrap(x0 + hx, N) * N + wrap(y0 + hy, N)) * N + wrap(z0 + hz, N);
        reinterpret_cast<uint4*>(sx)[e] = reinterpret_cast<const uint4*>(x + v * CIN)[half];
    }
    for (int e = threadIdx.x; e < 27 * COUT * CIN / 8; e += blockDim.x)
        reinterpret_cast<uint4*>(sw)[e] = reinterpret_cast<const uint4*>(w)[e];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, tg = lane & 3;
    for (int tile = warp; tile < kBx * kBy; tile += kConvWarps) {
        const int lx = tile / kBy, ly = tile % kBy;  // one z-row of 16 voxels
        float acc[NT][4];
#pragma unroll
        for (int n = 0; n < NT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
#pragma unroll 3
        for (int t = 0; t < 27; ++t) {
            const int tx = t / 9, ty = (t / 3) % 3, tz = t % 3;
            const int hbase = ((lx + tx) * kHy + (ly + ty)) * kHz + tz;
            const unsigned* r0 = reinterpret_cast<const unsigned*>(sx + (hbase + g) * CIN);
            const unsigned* r1 = reinterpret_cast<const unsigned*>(sx + (hbase + g + 8) * CIN);
            unsigned a[4] = {r0[tg], r1[tg], r0[tg + 4], r1[tg + 4]};
#pragma unroll
            for (int n = 0; n < NT; ++n) {
                const unsigned* wb = reinterpret_cast<const unsigned*>(sw + (t * COUT + n * 8 + g) * CIN);
                unsigned bb[2] = {wb[tg], wb[tg + 4]};
                mma_bf16_16816(acc[n], a, bb);
            }
        }
        // epilogue: rows g and g+8 of the tile are voxels z = g, g+8; columns co = 2 tg, 2 tg + 1
        const int vx = bx * kBx + lx, vy = by * kBy + ly;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int vz = bz * kBz + g + 8 * h;
            const long long v = ((long long)vx * N + vy) * N + vz;
#pragma unroll
            for (int n = 0; n < NT; ++n) {
                const int co = n * 8 + 2 * tg;
                float r0 = acc[n][2 * h], r1 = acc[n][2 * h + 1];
                if (EPI == kEpiBiasRelu) {
                    r0 = fmaxf(r0 + bias[co], 0.f);
                    r1 = fmaxf(r1 + bias[co + 1], 0.f);
                    *reinterpret_cast<__nv_bfloat162*>(out + v * COUT + co) = __floats2bfloat162_rn(r0, r1);
                } else if (EPI == kEpiMask) {
                    const __nv_bfloat162 m = *reinterpret_cast<const __nv_bfloat162*>(mask + v * COUT + co);
                    r0 = __bfloat162float(m.x) > 0.f ? r0 : 0.f;
                    r1 = __bfloat162float(m.y) > 0.f ? r1 : 0.f;
                    *reinterpret_cast<__nv_bfloat162*>(out + v * COUT + co) = __floats2bfloat162_rn(r0, r1);
                } else {
                    const FRow fr = force_rows(N);
                    const long long row = frow(vx, vy, 0, fr);
                    if (co < 3) F[(row + co) * P2 + vz] += scale * (r0 + bias[co]);
                    if (co + 1 < 3) F[(row + co + 1) * P2 + vz] += scale * (r1 + bias[co + 1]);
                }
            }
        }
    }
}

// Weight gradient partials: dW[t][co][ci] = sum_v dy[v][co] x[v + t - 1][ci]
// (16 channels each; padded channels are zero).  A = dy^T (co x voxels),
// B = shifted x (voxels x ci); each warp owns three taps, blocks are
// persistent over bricks and write one partial per block (fixed-order
// reduction afterwards keeps the result deterministic).
constexpr size_t kDwSmem = (size_t)(kHx * kHy * kHz + kBx * kBy * kBz) * 16 * sizeof(bf16);

__global__ void __launch_bounds__(288) k_conv_dw(const bf16* __restrict__ x, const bf16* __restrict__ dy, int N,
                                                 float* __restrict__ part) {
    constexpr int CIN = 16, COUT = 16;
    extern __shared__ __align__(16) unsigned char dsm[];
    bf16* sx = reinterpret_cast<bf16*>(dsm);
    bf16* sd = sx + kHx * kHy * kHz * CIN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, tg = lane & 3;
    // accumulators: 3 taps x (co tiles: NT... M = 16 rows of co) -> use M = co (16, padded), N = ci (2 x 8)
    float acc[3][2][4];
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int n = 0; n < 2; ++n) acc[q][n][0] = acc[q][n][1] = acc[q][n][2] = acc[q][n][3] = 0.f;
    const int nbz = N / kBz, nby = N / kBy, nbx = N / kBx;
    const int nbricks = nbx * nby * nbz;
    for (int b0 = blockIdx.x; b0 < nbricks; b0 += gridDim.x) {
        int b = b0;
        const int bz = b % nbz;
        b /= nbz;
        const int by = b % nby;
        const int bx = b / nby;
        const int x0 = bx * kBx - 1, y0 = by * kBy - 1, z0 = bz * kBz - 1;
        __syncthreads();
        for (int e = threadIdx.x; e < kHx * kHy * kHz * 2; e += blockDim.x) {
            const int half = e & 1;
            const int hv = e >> 1;
            const int hz = hv % kHz, hy = (hv / kHz) % kHy, hx = hv / (kHz * kHy);
            const long long v = ((long long)wrap(x0 + hx, N) * N + wrap(y0 + hy, N)) * N + wrap(z0 + hz, N);
            reinterpret_cast<uint4*>(sx)[e] = reinterpret_cast<const uint4*>(x + v * CIN)[half];
        }
        for (int e = threadIdx.x; e < kBx * kBy * kBz * COUT / 8; e += blockDim.x) {
            const int per = COUT / 8;
            const int bv = e / per, part8 = e % per;
            const int lz = bv % kBz, ly = (bv / kBz) % kBy, lx = bv / (kBz * kBy);
            const long long v = ((long long)(bx * kBx + lx) * N + (by * kBy + ly)) * N + (bz * kBz + lz);
            reinterpret_cast<uint4*>(sd)[e] = reinterpret_cast<const uint4*>(dy + v * COUT)[part8];
        }
        __syncthreads();
        if (warp < 9) {
            // K loop over the brick's voxels, 16 at a time (one z-row)
            for (int row = 0; row < kBx * kBy; ++row) {
                const int lx = row / kBy, ly = row % kBy;
                // A fragment: A[co][v], co = g / g+8, v = 2tg, 2tg+1 / +8, +9 (z offsets in the row)
                unsigned a[4];
                {
                    const bf16* d0 = sd + ((lx * kBy + ly) * kBz) * COUT;
                    auto pk = [&](int co, int vz) -> unsigned {
                        const bf16 lo = co < COUT ? d0[vz * COUT + co] : __float2bfloat16(0.f);
                        const bf16 hi = co < COUT ? d0[(vz + 1) * COUT + co] : __float2bfloat16(0.f);
                        return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
                    };
                    a[0] = pk(g, 2 * tg);
                    a[1] = pk(g + 8, 2 * tg);
                    a[2] = pk(g, 2 * tg + 8);
                    a[3] = pk(g + 8, 2 * tg + 8);
                }
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const int t = warp * 3 + q;
                    const int tx = t / 9, ty = (t / 3) % 3, tz = t % 3;
                    const bf16* xs = sx + (((lx + tx) * kHy + (ly + ty)) * kHz + tz) * CIN;
#pragma unroll
                    for (int n = 0; n < 2; ++n) {
                        // B fragment: B[v][ci], v = 2tg, 2tg+1 (reg 0) / +8, +9 (reg 1), ci = n*8 + g
                        const int ci = n * 8 + g;
                        auto pb = [&](int vz) -> unsigned {
                            return (unsigned)__bfloat16_as_ushort(xs[vz * CIN + ci]) |
                                   ((unsigned)__bfloat16_as_ushort(xs[(vz + 1) * CIN + ci]) << 16);
                        };
                        unsigned bb[2] = {pb(2 * tg), pb(2 * tg + 8)};
                        mma_bf16_16816(acc[q][n], a, bb);
                    }
                }
            }
        }
    }
    if (warp < 9) {
        float* o = part + (size_t)blockIdx.x * 27 * COUT * CIN;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int t = warp * 3 + q;
#pragma unroll
            for (int n = 0; n < 2; ++n) {
                const int ci = n * 8 + 2 * tg;
                if (g < COUT) {
                    o[(t * COUT + g) * CIN + ci] = acc[q][n][0];
                    o[(t * COUT + g) * CIN + ci + 1] = acc[q][n][1];
                }
                if (g + 8 < COUT) {
                    o[(t * COUT + g + 8) * CIN + ci] = acc[q][n][2];
                    o[(t * COUT + g + 8) * CIN + ci + 1] = acc[q][n][3];
                }
            }
        }
    }
}

// fixed-order sum of per-block partials: out[i] = sum_b part[b][i]
__global__ void k_sum_partials(const float* __restrict__ part, int nblocks, int len, float* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    float s = 0.f;
    for (int b = 0; b < nblocks; ++b) s += part[(size_t)b * len + i];
    out[i] = s;
}

// bias gradient partials: db[co] = sum_v dy[v][co] (dy with 16 channels)
__global__ void k_bias_grad(const bf16* __restrict__ dy, long long nv, int cout, float* __restrict__ part) {
    __shared__ float red[256][16];
    float s[16];
    for (int c = 0; c < 16; ++c) s[c] = 0.f;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (long long)gridDim.x * blockDim.x)
        for (int c = 0; c < cout; ++c) s[c] += __bfloat162float(dy[v * 16 + c]);
    for (int c = 0; c < 16; ++c) red[threadIdx.x][c] = s[c];
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st)
            for (int c = 0; c < 16; ++c) red[threadIdx.x][c] += red[threadIdx.x + st][c];
        __syncthreads();
    }
    if (threadIdx.x < cout) part[blockIdx.x * cout + threadIdx.x] = red[0][threadIdx.x];
}

// network input: channels (delta, F_x/g, F_y/g, F_z/g, 0...) as bf16 [v][16]
// from delta (float [v]) and the interleaved force mesh real view
__global__ void k_pack_input(const float* __restrict__ delta, const float* __restrict__ F, int N, long long P2,
                             float inv_g, bf16* __restrict__ x) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n3 = (long long)N * N * N;
    if (v >= n3) return;
    const long long row = v / N;
    const int z = (int)(v - row * N);
    const int ix = (int)(row / N), iy = (int)(row - (long long)ix * N);
    const FRow fr = force_rows(N);
    const long long fb = frow(ix, iy, 0, fr) * P2 + z;
    float c[16];
    c[0] = delta[v];
    for (int j = 0; j < 3; ++j) c[1 + j] = F[fb + j * P2] * inv_g;
    for (int j = 4; j < 16; ++j) c[j] = 0.f;
    uint4* o = reinterpret_cast<uint4*>(x + v * 16);
    for (int q = 0; q < 2; ++q) {
        __nv_bfloat162 h[4];
        for (int r = 0; r < 4; ++r) h[r] = __floats2bfloat162_rn(c[q * 8 + 2 * r], c[q * 8 + 2 * r + 1]);
        o[q] = *reinterpret_cast<uint4*>(h);
    }
}

// upstream gradient of the last layer: dy[v][c] = g * dL/dF_c(v) (c < 3), 0 above
__global__ void k_pack_grad(const float* __restrict__ dF, int N, float gsc, bf16* __restrict__ dy) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n3 = (long long)N * N * N;
    if (v >= n3) return;
    __nv_bfloat162 h[8];
    h[0] = __floats2bfloat162_rn(gsc * dF[v], gsc * dF[n3 + v]);
    h[1] = __floats2bfloat162_rn(gsc * dF[2 * n3 + v], 0.f);
    for (int q = 2; q < 8; ++q) h[q] = __floats2bfloat162_rn(0.f, 0.f);
    reinterpret_cast<uint4*>(dy + v * 16)[0] = reinterpret_cast<uint4*>(h)[0];
    reinterpret_cast<uint4*>(dy + v * 16)[1] = reinterpret_cast<uint4*>(h)[1];
}

// Weight packing from FP32 master [co][ci][27] (true sizes co_n x ci_n):
// forward layout [t][COUT][16] and data-gradient layout [t'][16][COUT'] with
// t' = 26 - t (flipped stencil) and the channel roles swapped.
__global__ void k_pack_weights(const float* __restrict__ W, int co_n, int ci_n, int cout_pad, bf16* __restrict__ wf,
                               bf16* __restrict__ wd, int cin_pad_d) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    // forward: 27 x cout_pad x 16
    if (e < 27 * cout_pad * 16) {
        const int ci = e % 16, co = (e / 16) % cout_pad, t = e / (16 * cout_pad);
        const float val = (co < co_n && ci < ci_n) ? W[(co * ci_n + ci) * 27 + t] : 0.f;
        wf[e] = __float2bfloat16(val);
    }
    // data gradient: output channels = ci (padded to 16 -> two n tiles), input channels = co padded to 16
    if (wd && e < 27 * 16 * cin_pad_d) {
        const int c_in = e % cin_pad_d;   // original co
        const int c_out = (e / cin_pad_d) % 16;  // original ci
        const int tp = e / (cin_pad_d * 16);
        const int t = 26 - tp;
        const float val = (c_in < co_n && c_out < ci_n) ? W[(c_in * ci_n + c_out) * 27 + t] : 0.f;
        wd[e] = __float2bfloat16(val);
    }
}

// Adam on a flat FP32 parameter vector
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ gsum, float* __restrict__ m,
                       float* __restrict__ v2, int n, float lr, float b1, float b2, float eps, float c1, float c2,
                       float gscale) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = gsum[i] * gscale;
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v2[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v2[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// --------------------------------------------------------------------------
// particle side of the training loss
// L = 1/(2 Np) sum_p |F_pred(p) - F_target(p)|^2; residual r = F_pred - F_target
// --------------------------------------------------------------------------
__global__ void k_residual(const float* __restrict__ pred, const float* __restrict__ target, float* __restrict__ res,
                           long long n3p, double* __restrict__ part) {
    __shared__ double red[256];
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n3p; i += (long long)gridDim.x * blockDim.x) {
        const float r = pred[i] - target[i];
        res[i] = r;
        acc += (double)r * r;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_sum_double(const double* __restrict__ part, int n, double scale, double* out) {
    if (threadIdx.x || blockIdx.x) return;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[i];
    *out = s * scale;
}

// Normal equations of the k-space filter fit: with basis force columns
// A_b (3 Np values each, b < nb) and target y, accumulate ATA[b][c] += A_b . A_c
// and ATy[b] += A_b . y in FP64 (one block per (b, c) pair, fixed order).
__global__ void k_lsq_accumulate(const float* __restrict__ A, const float* __restrict__ y, long long len, int nb,
                                 double* ATA, double* ATy) {
    __shared__ double red[256];
    const int b = blockIdx.x / (nb + 1), c = blockIdx.x % (nb + 1);
    if (c < b && c < nb) return;
    const float* ab = A + (size_t)b * len;
    const float* ac = c < nb ? A + (size_t)c * len : y;
    double acc = 0.0;
    for (long long i = threadIdx.x; i < len; i += blockDim.x) acc += (double)ab[i] * ac[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (c < nb) {
            ATA[b * nb + c] += red[0];
            if (c != b) ATA[c * nb + b] += red[0];
        } else {
            ATy[b] += red[0];
        }
    }
}

// (ATA + ridge tr(ATA)/nb I) T = ATy by Cholesky in FP64 (one thread; nb <= 64)
__global__ void k_lsq_solve(const double* ATA, const double* ATy, int nb, double ridge, float* T) {
    if (threadIdx.x || blockIdx.x) return;
    double L[64 * 64], z[64];
    double tr = 0.0;
    for (int i = 0; i < nb; ++i) tr += ATA[i * nb + i];
    const double lam = ridge * tr / nb;
    for (int i = 0; i < nb; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = ATA[i * nb + j] + (i == j ? lam : 0.0);
            for (int k = 0; k < j; ++k) s -= L[i * 64 + k] * L[j * 64 + k];
            L[i * 64 + j] = (i == j) ? sqrt(s > 0 ? s : 1e-300) : s / L[j * 64 + j];
        }
    for (int i = 0; i < nb; ++i) {
        double s = ATy[i];
        for (int k = 0; k < i; ++k) s -= L[i * 64 + k] * z[k];
        z[i] = s / L[i * 64 + i];
    }
    for (int i = nb - 1; i >= 0; --i) {
        double s = z[i];
        for (int k = i + 1; k < nb; ++k) s -= L[k * 64 + i] * z[k];
        z[i] = s / L[i * 64 + i];
    }
    for (int i = 0; i < nb; ++i) T[i] = (float)z[i];
}

}  // namespace cola

namespace cola {

// --------------------------------------------------------------------------
// host side
// --------------------------------------------------------------------------
constexpr int kDwBlocks = 608;  // persistent blocks of the weight-gradient kernel (4 per SM)
constexpr int kBiasBlocks = 304;
constexpr int kLossBlocks = 304;

// parameter / packed-weight offsets (include/cola.h)
constexpr int kW1 = 0, kB1 = 1728, kW2 = 1744, kB2 = 8656, kW3 = 8672, kB3 = 9968;
constexpr int kPf1 = 0, kPf2 = 6912, kPf3 = 13824, kPd2 = 17280, kPd3 = 24192;

struct LearnedBufs {
    float* delta;
    bf16 *x0, *h1, *h2, *g1, *g2;
    float* dF;
    unsigned long long* fix3;
    float *pred, *res, *dwpart, *dwsum, *bpart;
    double* lpart;
};

static size_t a256(size_t x) { return (x + 255) / 256 * 256; }

size_t learned_bytes(int ng, int nq) {
    const size_t n3 = (size_t)ng * ng * ng, np = (size_t)nq * nq * nq;
    return a256(4 * n3) + 5 * a256(32 * n3) + a256(12 * n3) + a256(24 * n3) + 2 * a256(12 * np) +
           a256((size_t)kDwBlocks * 27 * 256 * 4) + a256(27 * 256 * 4) + a256((size_t)kBiasBlocks * 16 * 4) +
           a256((size_t)kLossBlocks * 8);
}

static LearnedBufs learned_bufs(char* base, int ng, int nq) {
    const size_t n3 = (size_t)ng * ng * ng, np = (size_t)nq * nq * nq;
    LearnedBufs B;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        char* p = base + o;
        o += a256(bytes);
        return p;
    };
    B.delta = (float*)take(4 * n3);
    B.x0 = (bf16*)take(32 * n3);
    B.h1 = (bf16*)take(32 * n3);
    B.h2 = (bf16*)take(32 * n3);
    B.g1 = (bf16*)take(32 * n3);
    B.g2 = (bf16*)take(32 * n3);
    B.dF = (float*)take(12 * n3);
    B.fix3 = (unsigned long long*)take(24 * n3);
    B.pred = (float*)take(12 * np);
    B.res = (float*)take(12 * np);
    B.dwpart = (float*)take((size_t)kDwBlocks * 27 * 256 * 4);
    B.dwsum = (float*)take(27 * 256 * 4);
    B.bpart = (float*)take((size_t)kBiasBlocks * 16 * 4);
    B.lpart = (double*)take((size_t)kLossBlocks * 8);
    return B;
}

int net_pack(const cola_net* net, cudaStream_t s) {
    if (!net || !net->params || !net->wpack) return COLA_EINVAL;
    bf16* wp = (bf16*)net->wpack;
    const float* P = net->params;
    ProfScope ps(kKSetup, s);
    k_pack_weights<<<(27 * 16 * 16 + 255) / 256, 256, 0, s>>>(P + kW1, 16, 4, 16, wp + kPf1, nullptr, 16);
    k_pack_weights<<<(27 * 16 * 16 + 255) / 256, 256, 0, s>>>(P + kW2, 16, 16, 16, wp + kPf2, wp + kPd2, 16);
    k_pack_weights<<<(27 * 16 * 16 + 255) / 256, 256, 0, s>>>(P + kW3, 3, 16, 8, wp + kPf3, wp + kPd3, 16);
    return check_launch();
}

static unsigned conv_grid(int N) { return (unsigned)((N / kBx) * (N / kBy) * (N / kBz)); }

// input packing and the three convolutions; adds g * net to the force mesh
int net_forward(const cola_net* net, char* lbase, int ng, int nq, float green, float2* F, cudaStream_t s) {
    LearnedBufs B = learned_bufs(lbase, ng, nq);
    const bf16* wp = (const bf16*)net->wpack;
    const float* P = net->params;
    const long long n3 = (long long)ng * ng * ng;
    const long long P2 = 2ll * fft_pitch(ng);
    ProfScope ps(kKLearned, s);
    k_pack_input<<<(unsigned)((n3 + 255) / 256), 256, 0, s>>>(B.delta, (const float*)F, ng, P2, 1.f / green, B.x0);
    k_conv<2, kEpiBiasRelu><<<conv_grid(ng), kConvWarps * 32, 0, s>>>(B.x0, wp + kPf1, P + kB1, ng, B.h1, nullptr,
                                                                        nullptr, 0, 0.f);
    k_conv<2, kEpiBiasRelu><<<conv_grid(ng), kConvWarps * 32, 0, s>>>(B.h1, wp + kPf2, P + kB2, ng, B.h2, nullptr,
                                                                        nullptr, 0, 0.f);
    k_conv<1, kEpiAddForce><<<conv_grid(ng), kConvWarps * 32, 0, s>>>(B.h2, wp + kPf3, P + kB3, ng, nullptr, nullptr,
                                                                        (float*)F, P2, green);
    g_launches += 3;
    return check_launch();
}

// transposed weight-gradient sum [27][16][16] -> master layout [co][ci][27]
__global__ void k_unpack_dw(const float* __restrict__ dwt, int co_n, int ci_n, float* __restrict__ out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= co_n * ci_n * 27) return;
    const int t = e % 27, ci = (e / 27) % ci_n, co = e / (27 * ci_n);
    out[e] = dwt[(t * 16 + co) * 16 + ci];
}

__global__ void k_fix3_to_float(const unsigned long long* __restrict__ fix3, float* __restrict__ dF, long long n,
                                float scale) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    dF[i] = (float)(long long)fix3[i] * scale;
}

static int layer_grads(const bf16* x, const bf16* dy, int ng, int co_n, int ci_n, float* gW, float* gb,
                       const LearnedBufs& B, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_conv_dw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDwSmem) != cudaSuccess)
            return COLA_ECUDA;
        attr = true;
    }
    const long long n3 = (long long)ng * ng * ng;
    k_conv_dw<<<kDwBlocks, 288, kDwSmem, s>>>(x, dy, ng, B.dwpart);
    k_sum_partials<<<(27 * 256 + 255) / 256, 256, 0, s>>>(B.dwpart, kDwBlocks, 27 * 256, B.dwsum);
    k_unpack_dw<<<(co_n * ci_n * 27 + 255) / 256, 256, 0, s>>>(B.dwsum, co_n, ci_n, gW);
    k_bias_grad<<<kBiasBlocks, 256, 0, s>>>(dy, n3, co_n, B.bpart);
    k_sum_partials<<<1, 32, 0, s>>>(B.bpart, kBiasBlocks, co_n, gb);
    g_launches += 5;
    return check_launch();
}

// loss and gradient, after net_forward has left x0, h1, h2 and the force mesh F
int net_backward(const cola_net* net, char* lbase, int ng, int nq, double box, float green, const float2* F,
                 const float* d, const float* target, float* grad, double* loss, cudaStream_t s) {
    LearnedBufs B = learned_bufs(lbase, ng, nq);
    const bf16* wp = (const bf16*)net->wpack;
    const long long n3 = (long long)ng * ng * ng, np = (long long)nq * nq * nq;
    int rc;
    if ((rc = launch_gather(F, d, B.pred, nq, ng, box, s))) return rc;
    ProfScope ps(kKLearned, s);
    k_residual<<<kLossBlocks, 256, 0, s>>>(B.pred, target, B.res, 3 * np, B.lpart);
    k_sum_double<<<1, 32, 0, s>>>(B.lpart, kLossBlocks, 0.5 / (double)np, loss);
    if (cudaMemsetAsync(B.fix3, 0, 24 * (size_t)n3, s) != cudaSuccess) return COLA_ECUDA;
    if ((rc = launch_adjoint_deposit(d, B.res, B.fix3, nq, ng, box, s))) return rc;
    // dL/dF_mesh = deposit / Np (2^-30 fixed point)
    k_fix3_to_float<<<(unsigned)((3 * n3 + 255) / 256), 256, 0, s>>>(B.fix3, B.dF, 3 * n3,
                                                                     (float)(1.0 / 1073741824.0 / (double)np));
    // last layer: F += g out  ->  dL/dout = g dL/dF
    k_pack_grad<<<(unsigned)((n3 + 255) / 256), 256, 0, s>>>(B.dF, ng, green, B.g1);
    g_launches += 4;
    if ((rc = layer_grads(B.h2, B.g1, ng, 3, 16, grad + kW3, grad + kB3, B, s))) return rc;
    k_conv<2, kEpiMask><<<conv_grid(ng), kConvWarps * 32, 0, s>>>(B.g1, wp + kPd3, nullptr, ng, B.g2, B.h2, nullptr,
                                                                  0, 0.f);
    if ((rc = layer_grads(B.h1, B.g2, ng, 16, 16, grad + kW2, grad + kB2, B, s))) return rc;
    k_conv<2, kEpiMask><<<conv_grid(ng), kConvWarps * 32, 0, s>>>(B.g2, wp + kPd2, nullptr, ng, B.g1, B.h1, nullptr,
                                                                  0, 0.f);
    if ((rc = layer_grads(B.x0, B.g1, ng, 16, 4, grad + kW1, grad + kB1, B, s))) return rc;
    g_launches += 2;
    return check_launch();
}

int launch_adam(float* p, const float* g, float* m, float* v, int n, int t, float lr, float b1, float b2, float eps,
                cudaStream_t s) {
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    ProfScope ps(kKLearned, s);
    k_adam<<<(n + 255) / 256, 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2, 1.f);
    return check_launch();
}

int launch_lsq_accumulate(const float* A, const float* y, long long len, int nb, double* ATA, double* ATy,
                          cudaStream_t s) {
    ProfScope ps(kKLearned, s);
    k_lsq_accumulate<<<nb * (nb + 1), 256, 0, s>>>(A, y, len, nb, ATA, ATy);
    return check_launch();
}

int launch_lsq_solve(const double* ATA, const double* ATy, int nb, double ridge, float* T, cudaStream_t s) {
    ProfScope ps(kKLearned, s);
    k_lsq_solve<<<1, 32, 0, s>>>(ATA, ATy, nb, ridge, T);
    return check_launch();
}

__global__ void k_basis_table(float* T, int nb, int b) {
    const int i = threadIdx.x;
    if (i < nb) T[i] = (i == b) ? 1.f : 0.f;
}

int launch_basis_table(float* T, int nb, int b, cudaStream_t s) {
    k_basis_table<<<1, 64, 0, s>>>(T, nb, b);
    return check_launch();
}

}  // namespace cola
