// Particle-side helpers shared by the particle kernels (pm.cu) and the fused
// mesh kernels that deposit or gather inside an FFT pass (fft_fused.cuh):
// the CIC corners and fractions of a particle (Sec. 2.2), its fixed-point
// deposit weights, and the row bins of the PM step.
//
// Particle p = (i*nq + j)*nq + k sits at mesh coordinate
//   u = (i, j, k) * ng/nq + 1/2 + d * ng/L      (periodic)
// The Lagrangian part is formed exactly in integers, (i*2ng + nq)/(2nq), and
// only the small displacement term is FP32, so the CIC fraction keeps FP32
// precision for any mesh size.
//
// Deposit determinism: each particle's eight CIC weights are turned into
// unsigned 64-bit fixed point with 2^40 per particle (the largest corner takes
// the remainder so the eight sum to exactly 2^40) and added with integer
// atomics, which commute: the mesh is bit-identical whatever the order.
#pragma once

#include "cola_common.cuh"

namespace cola {

constexpr float kFix = 1099511627776.0f;  // 2^40
constexpr unsigned long long kFixU = 1ull << 40;

struct Cic {
    int c0[3];    // lower corner cell (wrapped)
    int c1[3];    // upper corner cell (wrapped)
    float f[3];   // fraction towards the upper corner
};

// Lattice site of particle index p (p < 2^31: nq^3 <= 4096^3 / 8 in practice;
// every lattice the library accepts has nq^3 < 2^31 particles addressed by int)
__device__ __forceinline__ void lattice_site(long long p, int nq, int idx[3]) {
    const unsigned q = (unsigned)p, n = (unsigned)nq;
    const unsigned ij = q / n;
    idx[2] = (int)(q - ij * n);
    idx[0] = (int)(ij / n);
    idx[1] = (int)(ij - (unsigned)idx[0] * n);
}

__device__ __forceinline__ bool particle_cic(const int idx[3], int nq, int ng, float inv_cell, const float dx[3],
                                             Cic& c) {
    // the Lagrangian part (i 2 ng + nq) / (2 nq) in integers: for ng a multiple
    // of nq it is i m + 1/2 exactly; otherwise one 32-bit division
    // (i 2 ng + nq < 2^26 for the sizes the library accepts)
    const int m = ng / nq;
    const bool whole = m * nq == ng;
    const int den = 2 * nq;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int base;
        float frac0;
        if (whole) {
            base = idx[a] * m;
            frac0 = 0.5f;
        } else {
            const int num = idx[a] * 2 * ng + nq;
            base = num / den;
            frac0 = (float)(num - base * den) / (float)den;
        }
        // rounded explicitly (no contraction into an FMA): the binning, the
        // fused passes and the kick, in different translation units, must find
        // the same corner for the same particle
        const float t = __fadd_rn(frac0, __fmul_rn(dx[a], inv_cell));
        if (!(fabsf(t) < 1.0e7f)) return false;  // NaN, Inf or absurd displacement
        const float fl = floorf(t);
        c.f[a] = t - fl;
        int cell = base + (int)fl;  // |cell| < 1e7 + 4096
        if ((unsigned)cell >= (unsigned)ng) {
            cell %= ng;
            if (cell < 0) cell += ng;
        }
        c.c0[a] = cell;
        c.c1[a] = (cell + 1 == ng) ? 0 : cell + 1;
    }
    return true;
}

// The eight fixed-point weights w[4a + 2b + e] of corner (c_a x, c_b y, c_e z):
// each rounded from the FP32 product, the corner of the largest weight along
// every axis taking the remainder of 2^40.
__device__ __forceinline__ void cic_fix_weights(const Cic& c, unsigned long long w[8]) {
    const float wx[2] = {1.f - c.f[0], c.f[0]};
    const float wy[2] = {1.f - c.f[1], c.f[1]};
    const float wz[2] = {1.f - c.f[2], c.f[2]};
    const int m = 4 * (c.f[0] >= 0.5f) + 2 * (c.f[1] >= 0.5f) + (c.f[2] >= 0.5f);
    unsigned long long sum = 0;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int i = 4 * a + 2 * b + e;
                const unsigned long long v = i == m ? 0ull : __float2ull_rn(wx[a] * wy[b] * wz[e] * kFix);
                sum += v;
                w[i] = v;
            }
    // integer sums: the remainder is exact whatever the order of the others
#pragma unroll
    for (int i = 0; i < 8; ++i) w[i] = i == m ? kFixU - sum : w[i];
}

}  // namespace cola
