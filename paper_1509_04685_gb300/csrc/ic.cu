// Initial conditions and FP64 time tables.
//
// * Growth factors and the COLA kick/drift integrals (Eqs. 2-3) are computed
//   in FP64 on the device by one thread: RK4 in ln a on
//   (D1, dD1/dlna, D2, dD2/dlna, K, Dr) with
//     D1'' + (2 + dlnE/dlna) D1' = 3/2 Om(a) D1,
//     D2'' + (2 + dlnE/dlna) D2' = 3/2 Om(a) (D2 - D1^2),
//     dK/dlna = 1/E,  dDr/dlna = 1/(a^2 E),
//   started on the Einstein-de Sitter growing modes (D1 = a, D2 = -3/7 a^2)
//   at a = 1e-5 and normalised to D1(1) = 1.
// * 2LPT initial conditions (Sec. 2.2: Gaussian field + 2LPT): Philox-4x32-10
//   white noise (Salmon et al. 2011) with a 53-bit Box-Muller draw in FP64,
//   the Eisenstein & Hu (1998) no-wiggle spectrum normalised to sigma8, and
//   Psi1_k = i k delta_k/k^2, delta2 = sum_{i<j} phi_ii phi_jj - phi_ij^2,
//   Psi2_k = -i k delta2_k / k^2 (Crocce et al. 2006 convention).
#include <cmath>

#include "cola_common.cuh"

namespace cola {


struct CosmoD {
    double om, ol, ok, ob, h, s8, ns, tcmb;
};

static CosmoD cosmo_of(const cola_config* cfg) {
    const cola_cosmology& c = cfg->cosmo;
    return CosmoD{c.omega_m, c.omega_l, 1.0 - c.omega_m - c.omega_l, c.omega_b, c.h, c.sigma8, c.n_s, c.t_cmb};
}

__device__ double E_of(double a, const CosmoD& c) {
    return sqrt(c.om / (a * a * a) + c.ok / (a * a) + c.ol);
}

// Growth ODEs in y = ln a for D1 = a u and D2 = a^2 w (Sec. 2.2's 2LPT growth
// factors; the same equations as D1'' + (2 + dlnE/dy) D1' = 3/2 Om(a) D1 and
// D2'' + (2 + dlnE/dy) D2' = 3/2 Om(a) (D2 - D1^2)): u and w are constant in the
// matter era, so RK4 in these variables is accurate with far fewer steps than
// in D1, D2 themselves, which grow like a and a^2.  State s = (u, u', w, w',
// K, Dr) with K = int dy / E and Dr = int dy a^kn / (a^2 E) over the current
// segment (kn = 0: the standard drift; kn = n_LPT: the modified drift's integral).
__device__ void growth_rhs(double y, const double* s, double* ds, const CosmoD& c, double kn) {
    const double a = exp(y);
    const double a2 = a * a, a3 = a2 * a;
    const double E2 = c.om / a3 + c.ok / a2 + c.ol;
    const double E = sqrt(E2);
    const double oma = c.om / a3 / E2;
    const double fr = 2.0 + (-3.0 * c.om / a3 - 2.0 * c.ok / a2) / (2.0 * E2);
    ds[0] = s[1];
    ds[1] = -(2.0 + fr) * s[1] - (1.0 + fr - 1.5 * oma) * s[0];
    ds[2] = s[3];
    ds[3] = -(4.0 + fr) * s[3] - (4.0 + 2.0 * fr - 1.5 * oma) * s[2] - 1.5 * oma * s[0] * s[0];
    ds[4] = 1.0 / E;
    ds[5] = (kn != 0.0 ? exp(kn * y) : 1.0) / (a2 * E);
}

// step bounds in y: from the start to the first output, and between outputs
constexpr double kHEarly = 1.0 / 64.0;
constexpr double kHSeg = 1.0 / 256.0;

// Advance s from y0 to y1 with RK4 steps of at most hmax.
__device__ void rk4_to(double* s, double y0, double y1, const CosmoD& c, double hmax, double kn = 0.0) {
    const double span = y1 - y0;
    if (span <= 0.0) return;
    const int nstep = (int)ceil(span / hmax);
    const double h = span / nstep;
    double k1[6], k2[6], k3[6], k4[6], t[6];
    double y = y0;
    for (int i = 0; i < nstep; ++i) {
        growth_rhs(y, s, k1, c, kn);
        for (int q = 0; q < 6; ++q) t[q] = s[q] + 0.5 * h * k1[q];
        growth_rhs(y + 0.5 * h, t, k2, c, kn);
        for (int q = 0; q < 6; ++q) t[q] = s[q] + 0.5 * h * k2[q];
        growth_rhs(y + 0.5 * h, t, k3, c, kn);
        for (int q = 0; q < 6; ++q) t[q] = s[q] + h * k3[q];
        growth_rhs(y + h, t, k4, c, kn);
        for (int q = 0; q < 6; ++q) s[q] += h / 6.0 * (k1[q] + 2.0 * k2[q] + 2.0 * k3[q] + k4[q]);
        y = (i + 1 == nstep) ? y1 : y + h;
    }
}

constexpr double kAEarly = 1e-5;
constexpr double kNLpt = -2.5;  // n_LPT of the modified kick and drift (Tassev et al. 2013)

// the Einstein-de Sitter modes at a = kAEarly: D1 = a, D2 = -3/7 a^2
__device__ void growth_init(double* s) {
    s[0] = 1.0;
    s[1] = 0.0;
    s[2] = -3.0 / 7.0;
    s[3] = 0.0;
    s[4] = s[5] = 0.0;
}

__device__ double node_a(int j, int n, double ai, double af, int sampling, double p) {
    const double t = (double)j / (double)(n - 1);
    if (sampling == COLA_SAMPLING_LOG) return exp(log(ai) + t * (log(af) - log(ai)));
    if (sampling == COLA_SAMPLING_POW) return pow(pow(ai, p) + t * (pow(af, p) - pow(ai, p)), 1.0 / p);
    return ai + t * (af - ai);
}

// Table row j (12 doubles): a, green, c1, c2, kick, drift, dD1, dD2, D1, D2, dD1/da, dD2/da.
// kn = 0: the standard kick and drift factors, kick = int da / (a E) over
// [a_{j-1/2}, a_{j+1/2}] and drift = int da / (a^3 E) over [a_j, a_{j+1}].
// kn = n_LPT: the modified factors of Tassev et al. (2013), the residual
// momentum varying as a power a^n of the scale factor about the reference time:
// kick = (a_{j+1/2}^n - a_{j-1/2}^n) / (n a_j^n E(a_j)) (force at the node),
// drift = a_{j+1/2}^-n int da a^n / (a^3 E) over [a_j, a_{j+1}] (momentum at the midpoint).
__global__ void k_tables(double* tab, int n, double ai, double af, int sampling, double sp, CosmoD c, int pm_only,
                         double kn) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s[6];
    growth_init(s);
    double y = log(kAEarly);
    for (int j = 0; j < n; ++j) {
        const double aj = node_a(j, n, ai, af, sampling, sp);
        const double yj = log(aj);
        rk4_to(s, y, yj, c, j == 0 ? kHEarly : kHSeg, kn);
        y = yj;
        double* r = tab + (size_t)j * kTableCols;
        r[0] = aj;
        r[1] = 1.5 * c.om / aj;
        r[8] = aj * s[0];  // raw D1 (normalised below)
        r[9] = aj * aj * s[2];
        r[10] = s[0] + s[1];                  // dD1/da
        r[11] = aj * (2.0 * s[2] + s[3]);     // dD2/da
        r[4] = (j > 0) ? s[4] : 0.0;  // segment mid_{j-1} -> a_j
        double drift = (j > 0) ? s[5] : 0.0;
        if (j > 0) tab[(size_t)(j - 1) * kTableCols + 5] += drift;
        s[4] = s[5] = 0.0;
        if (j + 1 < n) {
            const double an = node_a(j + 1, n, ai, af, sampling, sp);
            const double ym = log(0.5 * (aj + an));
            rk4_to(s, y, ym, c, kHSeg, kn);
            y = ym;
            r[4] += s[4];  // a_j -> mid_j
            r[5] = s[5];
            s[4] = s[5] = 0.0;
        } else {
            r[5] = 0.0;
        }
    }
    // normalisation D1(1) = 1 (at a = 1, D1 = u)
    if (y < 0.0) rk4_to(s, y, 0.0, c, kHSeg);
    const double norm = (y <= 0.0) ? s[0] : 0.0;
    double nrm = norm;
    if (y > 0.0) {
        // a_final beyond 1: integrate again from the start to a = 1
        double t[6];
        growth_init(t);
        rk4_to(t, log(kAEarly), log(ai), c, kHEarly);
        rk4_to(t, log(ai), 0.0, c, kHSeg);
        nrm = t[0];
    }
    for (int j = 0; j < n; ++j) {
        double* r = tab + (size_t)j * kTableCols;
        r[8] /= nrm;
        r[9] /= nrm * nrm;
        r[10] /= nrm;
        r[11] /= nrm * nrm;
    }
    for (int j = 0; j < n; ++j) {
        double* r = tab + (size_t)j * kTableCols;
        const double D1 = r[8], D2 = r[9];
        r[2] = r[1] * D1;
        r[3] = r[1] * (D2 - D1 * D1);
        if (j + 1 < n) {
            const double* rn = r + kTableCols;
            r[6] = rn[8] - D1;
            r[7] = rn[9] - D2;
        } else {
            r[6] = r[7] = 0.0;
        }
        if (pm_only) r[2] = r[3] = r[6] = r[7] = 0.0;
    }
    if (kn != 0.0) {
        for (int j = 0; j < n; ++j) {
            double* r = tab + (size_t)j * kTableCols;
            const double aj = r[0];
            const double ajn = pow(aj, kn);
            double k = 0.0;
            if (j > 0) k += ajn - pow(0.5 * (tab[(size_t)(j - 1) * kTableCols] + aj), kn);
            if (j + 1 < n) {
                const double am = 0.5 * (aj + tab[(size_t)(j + 1) * kTableCols]);
                k += pow(am, kn) - ajn;
                r[5] /= pow(am, kn);
            }
            r[4] = k / (kn * ajn * E_of(aj, c));
        }
    }
}

int launch_tables(const cola_config* cfg, double* table, cudaStream_t s) {
    ProfScope ps(kKSetup, s);
    k_tables<<<1, 32, 0, s>>>(table, cfg->n_steps, cfg->a_init, cfg->a_final, cfg->sampling, cfg->sampling_p,
                              cosmo_of(cfg), (cfg->flags & COLA_FLAG_PM_ONLY) ? 1 : 0,
                              (cfg->flags & COLA_FLAG_MODIFIED_KDK) ? kNLpt : 0.0);
    return check_launch();
}

// Snapshot drift from a_node to a_out: (Dr(a_node, a_out), D1(a_out)-D1(a_node), D2(a_out)-D2(a_node)),
// then the redshift-space coefficients at a_out (1 / (a^2 E), a D1'(a), a D2'(a)).
__global__ void k_snapshot(double* snap, double a_node, double a_out, CosmoD c, int pm_only) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double lo = fmin(a_node, a_out), hi = fmax(a_node, a_out);
    double s[6];
    growth_init(s);
    rk4_to(s, log(kAEarly), log(lo), c, kHEarly);
    const double D1lo = lo * s[0], D2lo = lo * lo * s[2];
    s[4] = s[5] = 0.0;
    double t[6];
    for (int q = 0; q < 6; ++q) t[q] = s[q];
    rk4_to(s, log(lo), log(hi), c, kHSeg);
    const double D1hi = hi * s[0], D2hi = hi * hi * s[2], dr = s[5];
    // D1(1) for the normalisation (continue from lo; from the start if lo > 1)
    if (lo > 1.0) {
        growth_init(t);
        rk4_to(t, log(kAEarly), 0.0, c, kHEarly);
    } else {
        rk4_to(t, log(lo), 0.0, c, kHSeg);
    }
    const double nrm = t[0];
    const double sign = (a_out >= a_node) ? 1.0 : -1.0;
    snap[0] = sign * dr;
    snap[1] = pm_only ? 0.0 : sign * (D1hi - D1lo) / nrm;
    snap[2] = pm_only ? 0.0 : sign * (D2hi - D2lo) / (nrm * nrm);
    // redshift-space shift along the line of sight at a_out: p_z / (a^2 E) with the full
    // momentum p = v + a^3 E (D1' Psi1 + D2' Psi2), i.e. v_z / (a^2 E) + a (D1' Psi1_z + D2' Psi2_z)
    double u[6];
    growth_init(u);
    rk4_to(u, log(kAEarly), log(a_out), c, kHEarly);
    const double dD1 = (u[0] + u[1]) / nrm;                // dD1/da at a_out
    const double dD2 = a_out * (2.0 * u[2] + u[3]) / (nrm * nrm);  // dD2/da at a_out
    snap[3] = 1.0 / (a_out * a_out * E_of(a_out, c));
    snap[4] = pm_only ? 0.0 : a_out * dD1;
    snap[5] = pm_only ? 0.0 : a_out * dD2;
}

int launch_snapshot_coeffs(const cola_config* cfg, double a_node, double a_out, double* snap, cudaStream_t s) {
    ProfScope ps(kKSetup, s);
    k_snapshot<<<1, 32, 0, s>>>(snap, a_node, a_out, cosmo_of(cfg), (cfg->flags & COLA_FLAG_PM_ONLY) ? 1 : 0);
    return check_launch();
}

// ---------------------------------------------------------------------------
// Eisenstein & Hu (1998) no-wiggle transfer function (their Eqs. 26, 28-31)
// ---------------------------------------------------------------------------
__device__ double eh_nowiggle(double k, const CosmoD& c) {
    const double omh2 = c.om * c.h * c.h;
    const double obh2 = c.ob * c.h * c.h;
    const double fb = c.ob / c.om;
    const double th = c.tcmb / 2.7;
    const double sh = 44.5 * log(9.83 / omh2) / sqrt(1.0 + 10.0 * pow(obh2, 0.75));
    const double al = 1.0 - 0.328 * log(431.0 * omh2) * fb + 0.38 * log(22.3 * omh2) * fb * fb;
    const double x = 0.43 * k * c.h * sh;
    const double x2 = x * x;
    const double geff = c.om * c.h * (al + (1.0 - al) / (1.0 + x2 * x2));
    const double q = k * th * th / geff;
    const double L0 = log(2.0 * 2.718281828459045235 + 1.8 * q);
    const double C0 = 14.2 + 731.0 / (1.0 + 62.5 * q);
    return L0 / (L0 + C0 * q * q);
}

__device__ double tophat(double x) {
    if (fabs(x) < 0.1) {
        const double x2 = x * x;
        return 1.0 - x2 / 10.0 + x2 * x2 / 280.0 - x2 * x2 * x2 / 15120.0;
    }
    return 3.0 * (sin(x) - x * cos(x)) / (x * x * x);
}

// A = sigma8^2 / sigma_8,unnormalised^2 by composite Simpson in ln k over
// [1e-7, 250] h/Mpc with 2^17 intervals; fixed-order block reduction.
__global__ void __launch_bounds__(256) k_sigma8(double* amp, CosmoD c) {
    __shared__ double red[256];
    const int N = 1 << 17;
    const double lo = log(1e-7), hi = log(2e3 / 8.0);
    const double h = (hi - lo) / N;
    double acc = 0.0;
    for (int i = threadIdx.x; i <= N; i += blockDim.x) {
        const double k = exp(lo + i * h);
        const double T = eh_nowiggle(k, c);
        const double W = tophat(8.0 * k);
        const double f = k * k * k * pow(k, c.ns) * T * T * W * W;
        const double w = (i == 0 || i == N) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
        acc += w * f;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double s2 = red[0] * h / 3.0 / (2.0 * 3.14159265358979323846 * 3.14159265358979323846);
        amp[0] = c.s8 * c.s8 / s2;
    }
}

// ---------------------------------------------------------------------------
// Philox-4x32-10 (Salmon et al. 2011) and the white-noise field
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 ctr, uint2 key) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            key.x += 0x9E3779B9u;
            key.y += 0xBB67AE85u;
        }
        const unsigned lo0 = 0xD2511F53u * ctr.x, hi0 = __umulhi(0xD2511F53u, ctr.x);
        const unsigned lo1 = 0xCD9E8D57u * ctr.z, hi1 = __umulhi(0xCD9E8D57u, ctr.z);
        ctr = make_uint4(hi1 ^ ctr.y ^ key.x, lo1, hi0 ^ ctr.w ^ key.y, lo0);
    }
    return ctr;
}

__device__ __forceinline__ double uniform53(unsigned a, unsigned b) {
    const unsigned long long m = ((unsigned long long)(a >> 5) << 26) + (unsigned long long)(b >> 6) + 1ull;
    return (double)m * 1.1102230246251565404e-16;  // 2^-53
}

// noise of Lagrangian cell (i, j, k) -> real view of an nq mesh (row pitch 2P floats)
__global__ void k_noise(float* mesh, int nq, long long P2, unsigned long long seed) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n3 = (long long)nq * nq * nq;
    if (n >= n3) return;
    const uint4 w = philox4x32_10(make_uint4((unsigned)n, (unsigned)(n >> 32), 0u, 0u),
                                  make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
    const double u1 = uniform53(w.x, w.y);
    const double u2 = uniform53(w.z, w.w);
    const double g = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
    const long long row = n / nq;
    const int k = (int)(n - row * nq);
    mesh[row * P2 + k] = (float)g;
}

// ---------------------------------------------------------------------------
// spectral operations on the nq half-complex mesh
// ---------------------------------------------------------------------------
enum IcMode { kDelta = 0, kPsi1 = 1, kPhi = 2, kPsi2 = 3 };

__device__ __forceinline__ int signed_index(int i, int n) { return i < n / 2 ? i : i - n; }

// mode kDelta: in place delta_k = w_k sqrt(A k^ns T^2 / dq^3) (FP64 per mode)
// mode kPsi1:  dst = i k_a src / k^2 * norm
// mode kPhi:   dst = k_a k_b src / k^2 * norm
// mode kPsi2:  dst = -i k_a src / k^2 * norm
// k = 0 and every mode with an index on a Nyquist plane are set to zero.
__global__ void k_ic_spectral(const float2* src, float2* dst, int nq, int P, int mode, int ca, int cb, float kf,
                              float norm, const double* amp, CosmoD c, double dq3) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int H = nq / 2 + 1;
    const long long total = (long long)nq * nq * H;
    if (e >= total) return;
    const long long row = e / H;
    const int kz = (int)(e - row * H);
    const int ix = (int)(row / nq), iy = (int)(row - (long long)ix * nq);
    const long long q = row * P + kz;
    const int half = nq / 2;
    if (ix == half || iy == half || kz == half || (ix == 0 && iy == 0 && kz == 0)) {
        dst[q] = make_float2(0.f, 0.f);
        return;
    }
    const int nv[3] = {signed_index(ix, nq), signed_index(iy, nq), kz};
    if (mode == kDelta) {
        const double kfd = (double)kf;
        const double k2 = (double)nv[0] * nv[0] + (double)nv[1] * nv[1] + (double)nv[2] * nv[2];
        const double kk = kfd * sqrt(k2);
        const double T = eh_nowiggle(kk, c);
        const double pk = amp[0] * pow(kk, c.ns) * T * T;
        const float f = (float)sqrt(pk / dq3);
        dst[q] = cscale(src[q], f);
        return;
    }
    const float ka = kf * nv[ca];
    const float k2 = kf * kf * (float)(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
    const float2 a = src[q];
    if (mode == kPhi) {
        const float kb = kf * nv[cb];
        dst[q] = cscale(a, ka * kb / k2 * norm);
    } else {
        const float f = (mode == kPsi1 ? 1.f : -1.f) * ka / k2 * norm;
        dst[q] = make_float2(-f * a.y, f * a.x);  // i f a
    }
}

// delta2 = phi00 phi11 + phi00 phi22 + phi11 phi22 - phi01^2 - phi02^2 - phi12^2 (real views)
__global__ void k_ic_delta2(float* b00, const float* b11, const float* b22, const float* b01, const float* b02,
                            const float* b12, int nq, long long P2) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n3 = (long long)nq * nq * nq;
    if (n >= n3) return;
    const long long row = n / nq;
    const long long q = row * P2 + (n - row * nq);
    const float p00 = b00[q], p11 = b11[q], p22 = b22[q], p01 = b01[q], p02 = b02[q], p12 = b12[q];
    b00[q] = p00 * p11 + p00 * p22 + p11 * p22 - p01 * p01 - p02 * p02 - p12 * p12;
}

// d = D1 psi1 + D2 psi2; v = 0 (COLA) or the LPT momentum a^3 E (D1' psi1 + D2' psi2) (PM only)
__global__ void k_ic_finish(cola_state st, long long np3, const double* row0, CosmoD c, int pm_only) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= np3) return;
    const float D1 = (float)row0[8], D2 = (float)row0[9];
    const float s1 = st.psi1[q], s2 = st.psi2[q];
    st.d[q] = D1 * s1 + D2 * s2;
    if (pm_only) {
        const double a = row0[0];
        const double pref = a * a * a * E_of(a, c);
        st.v[q] = (float)(pref * row0[10]) * s1 + (float)(pref * row0[11]) * s2;
    } else {
        st.v[q] = 0.f;
    }
}

int launch_ic(const cola_config* cfg, uint64_t seed, cola_state st, void* ws, const Layout& L, cudaStream_t s) {
    const int nq = cfg->nq;
    const int P = fft_pitch(nq);
    const size_t Mq = mesh_bytes(nq);
    float2* b[7];
    for (int i = 0; i < 7; ++i) b[i] = reinterpret_cast<float2*>(wsp(ws, L.ic + i * Mq));
    const float2* tw = twiddle_ptr(ws, kTwLagr);
    const CosmoD c = cosmo_of(cfg);
    double* amp = reinterpret_cast<double*>(wsp(ws, kHdrSigmaAmp));
    const long long n3 = (long long)nq * nq * nq;
    const long long modes = (long long)nq * nq * (nq / 2 + 1);
    const float kf = (float)(2.0 * 3.14159265358979323846 / cfg->box);
    const double dq = cfg->box / nq;
    const float norm = (float)(1.0 / ((double)n3));
    const unsigned gm = (unsigned)((modes + 255) / 256), gr = (unsigned)((n3 + 255) / 256);
    int rc;

    {

        ProfScope ps(kKIc, s);

        k_sigma8<<<1, 256, 0, s>>>(amp, c);

    }
    if ((rc = check_launch())) return rc;
    // white noise -> delta_k
    {
        ProfScope ps(kKIc, s);
        k_noise<<<gr, 256, 0, s>>>(reinterpret_cast<float*>(b[0]), nq, 2ll * P, seed);
    }
    if ((rc = check_launch())) return rc;
    const long long nrows = (long long)nq * nq;
    if ((rc = fft_z_r2c(nullptr, b[0], nq, 0.f, tw, s, P, nrows, FRow{nq, 0, 1}))) return rc;
    if ((rc = fft_strided(b[0], nq, 1, -1, tw, s))) return rc;
    if ((rc = fft_strided(b[0], nq, 0, -1, tw, s))) return rc;
    {
        ProfScope ps(kKIc, s);
        k_ic_spectral<<<gm, 256, 0, s>>>(b[0], b[0], nq, P, kDelta, 0, 0, kf, 1.f, amp, c, dq * dq * dq);
    }
    if ((rc = check_launch())) return rc;

    auto inverse_to = [&](float2* buf, float* out) -> int {
        int r;
        if ((r = fft_strided(buf, nq, 0, +1, tw, s))) return r;
        if ((r = fft_strided(buf, nq, 1, +1, tw, s))) return r;
        if (out) return fft_z_c2r(buf, nq, tw, s, out, nq, 1.f, P, nrows);
        return fft_z_c2r(buf, nq, tw, s, nullptr, 0, 1.f, P, nrows);
    };
    // Psi1
    for (int a = 0; a < 3; ++a) {
        {
            ProfScope ps(kKIc, s);
            k_ic_spectral<<<gm, 256, 0, s>>>(b[0], b[1], nq, P, kPsi1, a, 0, kf, norm, amp, c, 0.0);
        }
        if ((rc = check_launch())) return rc;
        if ((rc = inverse_to(b[1], st.psi1 + a * n3))) return rc;
    }
    // phi_ij -> delta2
    const int pairs[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
    for (int t = 0; t < 6; ++t) {
        {
            ProfScope ps(kKIc, s);
            k_ic_spectral<<<gm, 256, 0, s>>>(b[0], b[1 + t], nq, P, kPhi, pairs[t][0], pairs[t][1], kf, norm, amp, c,
                                             0.0);
        }
        if ((rc = check_launch())) return rc;
        if ((rc = inverse_to(b[1 + t], nullptr))) return rc;
    }
    {
        ProfScope ps(kKIc, s);
        k_ic_delta2<<<gr, 256, 0, s>>>((float*)b[1], (const float*)b[2], (const float*)b[3], (const float*)b[4],
                                       (const float*)b[5], (const float*)b[6], nq, 2ll * P);
    }
    if ((rc = check_launch())) return rc;
    if ((rc = fft_z_r2c(nullptr, b[1], nq, 0.f, tw, s, P, nrows, FRow{nq, 0, 1}))) return rc;
    if ((rc = fft_strided(b[1], nq, 1, -1, tw, s))) return rc;
    if ((rc = fft_strided(b[1], nq, 0, -1, tw, s))) return rc;
    for (int a = 0; a < 3; ++a) {
        {
            ProfScope ps(kKIc, s);
            k_ic_spectral<<<gm, 256, 0, s>>>(b[1], b[2], nq, P, kPsi2, a, 0, kf, norm, amp, c, 0.0);
        }
        if ((rc = check_launch())) return rc;
        if ((rc = inverse_to(b[2], st.psi2 + a * n3))) return rc;
    }
    {
        ProfScope ps(kKIc, s);
        k_ic_finish<<<(unsigned)((3 * n3 + 255) / 256), 256, 0, s>>>(st, 3 * n3, table_ptr(ws), c,
                                                                       (cfg->flags & COLA_FLAG_PM_ONLY) ? 1 : 0);
    }
    return check_launch();
}

}  // namespace cola
