// Matter power spectrum shells (Sec. 2.5): P(k) = <|delta_k|^2> over the modes
// of each k-bin, with optional CIC deconvolution and the Jing (2005) CIC
// aliasing correction, closed form or iterated.
//
// Bin i (1 .. ng/2) holds the modes with (i - 1/2)^2 < |n|^2 < (i + 1/2)^2,
// decided in integer arithmetic.  Half-spectrum modes count twice except on
// the kz = 0 and kz = Nyquist planes.  P(k_n) = |delta_k|^2 L^3 / ng^6.
// A fixed grid of blocks each accumulates its share of the modes into FP32
// shared-memory bins; the per-block partials are then summed in FP64 in a
// fixed block order.  With MULTI the bins also take P L_2(mu) and P L_4(mu),
// mu = n_z / |n| (line of sight z): the redshift-space multipoles
// P_l = (2l + 1) <P L_l(mu)> of the paper's RSD study (Eq. 5).
#include "cola_common.cuh"

namespace cola {

constexpr int kPkBlocks = 608;  // 4 blocks per SM on a 152-SM GB300
constexpr int kPkThreads = 256;

// Iterated Jing (2005) correction of one mode m (flag COLA_PK_ALIAS_ITER): the
// raw power over C(m) = sum over the images |n_i| <= kJingImages of
// W^2(m + ng n) (|m + ng n| / |m|)^n_eff, W the CIC window, P taken as a power
// law of index n_eff (this mode's bin) around |m|.  sin(pi (m + ng n) / ng) =
// +-sin(pi m / ng), so each image's window factor is, per axis,
// sin^4(pi m / ng) / (pi (m + ng n) / ng)^4 (1 for m = n = 0, 0 for m = 0 != n).
constexpr int kJingImages = 2;
constexpr int kJingIterations = 3;
constexpr double kNeffClamp = 4.0;

__device__ __forceinline__ float jing_alias_sum(const int nn[3], int ng, float n_eff) {
    constexpr int NI = 2 * kJingImages + 1;
    const float inv_ng = 1.0f / (float)ng;
    float fa[3][NI], x[3][NI];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float s = sinpif((float)nn[a] * inv_ng);
        const float s4 = (s * s) * (s * s);
#pragma unroll
        for (int j = 0; j < NI; ++j) {
            const int n = j - kJingImages;
            x[a][j] = (float)(nn[a] + ng * n);
            if (nn[a] == 0) {
                fa[a][j] = n == 0 ? 1.f : 0.f;
            } else {
                const float t = 3.14159265358979f * x[a][j] * inv_ng;
                fa[a][j] = s4 / ((t * t) * (t * t));
            }
        }
    }
    const float lm2 = log2f((float)((long long)nn[0] * nn[0] + (long long)nn[1] * nn[1] + (long long)nn[2] * nn[2]));
    const float h = 0.5f * n_eff;
    float C = 0.f;
#pragma unroll
    for (int i = 0; i < NI; ++i) {
        if (fa[0][i] == 0.f) continue;
#pragma unroll
        for (int j = 0; j < NI; ++j) {
            const float wxy = fa[0][i] * fa[1][j];
            if (wxy == 0.f) continue;
            const float rxy = x[0][i] * x[0][i] + x[1][j] * x[1][j];
#pragma unroll
            for (int l = 0; l < NI; ++l) {
                const float w = wxy * fa[2][l];
                if (w != 0.f) C += w * exp2f(h * (log2f(rxy + x[2][l] * x[2][l]) - lm2));
            }
        }
    }
    return C;
}

template <bool MULTI>
__global__ void k_pk_shells(const float2* __restrict__ mk, int ng, long long P, float amp_scale, float kf, int flags,
                            int nbins, double* __restrict__ part, const double* __restrict__ neff) {
    constexpr int NA = MULTI ? 5 : 3;  // sum w, sum w k, sum w P [, sum w P L2, sum w P L4]
    extern __shared__ float bins[];
    for (int i = threadIdx.x; i < NA * nbins; i += blockDim.x) bins[i] = 0.f;
    __syncthreads();
    const int H = ng / 2 + 1;
    const long long total = (long long)ng * ng * H;
    const int half = ng / 2;
    const float inv_ng = 1.0f / (float)ng;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long row = e / H;
        const int kz = (int)(e - row * H);
        const int ix = (int)(row / ng), iy = (int)(row - (long long)ix * ng);
        const int nx = ix < half ? ix : ix - ng;
        const int ny = iy < half ? iy : iy - ng;
        const long long n2 = (long long)nx * nx + (long long)ny * ny + (long long)kz * kz;
        if (n2 == 0) continue;
        int i = (int)(sqrtf((float)n2) + 0.5f);
        while ((long long)i * i + i < n2) ++i;
        while ((long long)i * i - i + 1 > n2) --i;
        if (i < 1 || i > nbins) continue;
        const float2 d = mk[row * P + kz];
        const float dr = d.x * amp_scale, di = d.y * amp_scale;
        float p = dr * dr + di * di;
        if (flags & COLA_PK_ALIAS_ITER) {
            const int nn[3] = {nx, ny, kz};
            p /= jing_alias_sum(nn, ng, (float)neff[i - 1]);
        }
        if (flags & COLA_PK_DECONV_CIC) {
            float W = 1.f;
            const int nn[3] = {nx, ny, kz};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (nn[a] != 0) {
                    const float x = (float)nn[a] * inv_ng;
                    const float sc = sinpif(x) / (3.14159265358979f * x);
                    W *= sc * sc;
                }
            }
            p /= W * W;
        }
        if (flags & COLA_PK_ALIAS_JING) {
            float C = 1.f;
            const int nn[3] = {nx, ny, kz};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float s = sinpif((float)nn[a] * inv_ng);
                C *= 1.f - 2.f / 3.f * s * s;
            }
            p /= C;
        }
        const float w = (kz == 0 || kz == half) ? 1.f : 2.f;
        const float kmag = kf * sqrtf((float)n2);
        atomicAdd(&bins[i - 1], w);
        atomicAdd(&bins[nbins + i - 1], w * kmag);
        atomicAdd(&bins[2 * nbins + i - 1], w * p);
        if (MULTI) {
            const float mu2 = (float)((double)kz * kz / (double)n2);
            const float l2 = 1.5f * mu2 - 0.5f;
            const float l4 = (35.f * mu2 * mu2 - 30.f * mu2 + 3.f) * 0.125f;
            atomicAdd(&bins[3 * nbins + i - 1], w * p * l2);
            atomicAdd(&bins[4 * nbins + i - 1], w * p * l4);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NA * nbins; i += blockDim.x)
        part[(size_t)blockIdx.x * NA * nbins + i] = (double)bins[i];
}

__global__ void k_pk_reduce(const double* __restrict__ part, int nblocks, int nbins, double* k, double* pk,
                            double* nmodes, double* p2, double* p4) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nbins) return;
    const int NA = p2 ? 5 : 3;
    double w = 0.0, wk = 0.0, wp = 0.0, w2 = 0.0, w4 = 0.0;
    for (int b = 0; b < nblocks; ++b) {
        const double* q = part + (size_t)b * NA * nbins;
        w += q[i];
        wk += q[nbins + i];
        wp += q[2 * nbins + i];
        if (p2) {
            w2 += q[3 * nbins + i];
            w4 += q[4 * nbins + i];
        }
    }
    nmodes[i] = w;
    k[i] = w > 0.0 ? wk / w : 0.0;
    pk[i] = w > 0.0 ? wp / w : 0.0;
    if (p2) {
        p2[i] = w > 0.0 ? 5.0 * w2 / w : 0.0;
        p4[i] = w > 0.0 ? 9.0 * w4 / w : 0.0;
    }
}

// n_eff per bin for the next Jing iteration: d ln P / d ln k over the
// neighbouring bins (one-sided at the ends; 0 where a power is not positive),
// clamped to [-kNeffClamp, kNeffClamp]
__global__ void k_pk_slopes(const double* __restrict__ k, const double* __restrict__ pk, int nbins, double* neff) {
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
        const int lo = b > 0 ? b - 1 : 0, hi = b + 1 < nbins ? b + 1 : nbins - 1;
        double n = 0.0;
        if (hi != lo && pk[lo] > 0.0 && pk[hi] > 0.0 && k[hi] > k[lo] && k[lo] > 0.0)
            n = fmin(fmax(log(pk[hi] / pk[lo]) / log(k[hi] / k[lo]), -kNeffClamp), kNeffClamp);
        neff[b] = n;
    }
}

int launch_power(const float2* mk, int ng, long long rs, double box, int flags, double* part, double* k, double* pk,
                 double* nmodes, int nbins, cudaStream_t s, double* p2, double* p4) {
    if (flags & COLA_PK_ALIAS_ITER) {
        // closed-form start, then kJingIterations passes with slopes from the last estimate
        int rc = launch_power(mk, ng, rs, box, COLA_PK_DECONV_CIC | COLA_PK_ALIAS_JING, part, k, pk, nmodes, nbins, s,
                              nullptr, nullptr);
        double* neff = part + (size_t)kPkBlocks * 5 * nbins;
        for (int it = 0; it < kJingIterations && !rc; ++it) {
            k_pk_slopes<<<1, 256, 0, s>>>(k, pk, nbins, neff);
            if ((rc = check_launch())) break;
            const double ng3 = (double)ng * ng * ng;
            const float amp_scale = (float)(box * sqrt(box) / ng3);
            const float kf = (float)(2.0 * 3.14159265358979323846 / box);
            const size_t smem = (size_t)3 * nbins * sizeof(float);
            if (smem > 48 * 1024 && cudaFuncSetAttribute(k_pk_shells<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                         (int)smem) != cudaSuccess)
                return COLA_ECUDA;
            {
                ProfScope ps(kKPkShells, s);
                k_pk_shells<false><<<kPkBlocks, kPkThreads, smem, s>>>(mk, ng, rs, amp_scale, kf, COLA_PK_ALIAS_ITER,
                                                                     nbins, part, neff);
            }
            if ((rc = check_launch())) break;
            ProfScope ps(kKPkReduce, s);
            k_pk_reduce<<<(nbins + 127) / 128, 128, 0, s>>>(part, kPkBlocks, nbins, k, pk, nmodes, nullptr, nullptr);
            rc = check_launch();
        }
        return rc;
    }
    const double ng3 = (double)ng * ng * ng;
    const float amp_scale = (float)(box * sqrt(box) / ng3);  // sqrt(L^3 / ng^6)
    const float kf = (float)(2.0 * 3.14159265358979323846 / box);
    const bool multi = p2 && p4;
    const size_t smem = (size_t)(multi ? 5 : 3) * nbins * sizeof(float);
    auto kern = multi ? k_pk_shells<true> : k_pk_shells<false>;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return COLA_ECUDA;
    {
        ProfScope ps(kKPkShells, s);
        kern<<<kPkBlocks, kPkThreads, smem, s>>>(mk, ng, rs, amp_scale, kf, flags, nbins, part, nullptr);
    }
    int rc = check_launch();
    if (rc) return rc;
    ProfScope ps(kKPkReduce, s);
    k_pk_reduce<<<(nbins + 127) / 128, 128, 0, s>>>(part, kPkBlocks, nbins, k, pk, nmodes, multi ? p2 : nullptr,
                                                      multi ? p4 : nullptr);
    return check_launch();
}

// per-block partial sums, then the n_eff table of the iterated Jing correction
size_t power_partial_bytes(int nbins) { return ((size_t)kPkBlocks * 5 + 1) * nbins * sizeof(double); }

}  // namespace cola
