// Specialised strided and fused x/Green passes (fft_static.cuh) for the large
// meshes: 768^3, 1152^3, 1536^3 and 2304^3, the tile-width tables and the
// specialised z passes.
#include "fft_fused.cuh"

namespace cola {

// (n, B, threads) of every specialisation: B adjacent columns per tile, two
// tile buffers of spad(n) B complex in shared memory
#define COLA_STRIDED_SPECS(X) \
    X(768, 16, 1024) \
    X(768, 8, 512) \
    X(1152, 8, 1024) \
    X(1536, 8, 1024) \
    X(2304, 4, 1024)

#define COLA_XGREEN_SPECS(X) \
    X(768, 16, 768, 2)       \
    X(768, 8, 1024, 3)       \
    X(1152, 8, 768, 2)       \
    X(1152, 4, 768, 3)       \
    X(1536, 8, 768, 2)       \
    X(1536, 4, 1024, 3)      \
    X(2304, 4, 768, 2)       \
    X(2304, 2, 768, 3)

// (n, B, threads) of the strided passes with two lines per thread; they take precedence
#define COLA_STRIDED2_SPECS(X) \
    X(768, 16, 512)             \
    X(1152, 8, 384)             \
    X(1536, 8, 384)             \
    X(2304, 4, 384)
#define COLA_YPSI2_SPECS(X) \
    X(768, 16, 512)          \
    X(1152, 8, 384)          \
    X(1536, 8, 512)          \
    X(2304, 4, 384)
#define COLA_XGREEN2_SPECS(X) \
    X(768, 16, 384)            \
    X(1152, 8, 384)            \
    X(1536, 8, 384)            \
    X(2304, 4, 384)

bool launch_strided_static(float2* data, int n, int B, int sign, LineGeom lg, int nct, int ntiles,
                           const float2* tw, cudaStream_t s, int* rc) {
#define COLA_CASE(NN, BB, TT)                                                \
    if (n == NN && B == BB) {                                                \
        *rc = run_strided2<NN, BB, TT>(data, sign, lg, nct, ntiles, tw, s); \
        return true;                                                         \
    }
    COLA_STRIDED2_SPECS(COLA_CASE)
#undef COLA_CASE
#define COLA_CASE(NN, BB, TT)                                               \
    if (n == NN && B == BB) {                                               \
        *rc = run_strided<NN, BB, TT>(data, sign, lg, nct, ntiles, tw, s); \
        return true;                                                        \
    }
    COLA_STRIDED_SPECS(COLA_CASE)
#undef COLA_CASE
    return launch_strided_static_small(data, n, B, sign, lg, nct, ntiles, tw, s, rc);
}

bool launch_x_green_static(float2* F, int n, int B, int nct, int ntiles, const float2* tw, float gscale,
                           float kf, const float* filt, int nfilt, float fstep, cudaStream_t s, int* rc) {
#define COLA_CASE(NN, BB, TT)                                                                      \
    if (n == NN && B == BB) {                                                                      \
        *rc = run_x_green2<NN, BB, TT>(F, nct, ntiles, tw, gscale, kf, filt, nfilt, fstep, s);   \
        return true;                                                                               \
    }
    COLA_XGREEN2_SPECS(COLA_CASE)
#undef COLA_CASE
#define COLA_CASE(NN, BB, TT, NBUF)                                                                  \
    if (n == NN && B == BB) {                                                                        \
        *rc = run_x_green<NN, BB, TT, NBUF>(F, nct, ntiles, tw, gscale, kf, filt, nfilt, fstep, s); \
        return true;                                                                                 \
    }
    COLA_XGREEN_SPECS(COLA_CASE)
#undef COLA_CASE
    return launch_x_green_static_small(F, n, B, nct, ntiles, tw, gscale, kf, filt, nfilt, fstep, s, rc);
}

// default column width of the specialised line passes of each size
static const int kStaticTiles[][2] = {{96, 16}, {128, 16}, {160, 16}, {192, 16}, {256, 16}, {288, 16}, {320, 16}, {384, 16}, {480, 16}, {768, 16}, {1152, 8}, {1536, 8}, {2304, 4}};
static const int kStaticSpecs[][2] = {{96, 16}, {128, 16}, {160, 16}, {192, 16}, {256, 16}, {256, 8}, {288, 16}, {320, 16}, {384, 16}, {384, 8}, {480, 16}, {480, 8}, {768, 16}, {768, 8}, {1152, 8}, {1536, 8}, {2304, 4}};

// default column width of the specialised fused x/Green pass of each size
static const int kGreenTiles[][2] = {{768, 8}, {1152, 8}, {1536, 8}, {2304, 4}};

int static_green_tile(int n) {
    for (const auto& e : kGreenTiles)
        if (e[0] == n) return e[1];
    return launch_static_green_tile_small(n);
}

int static_tile(int n) {
    for (const auto& e : kStaticTiles)
        if (e[0] == n) return e[1];
    return 0;
}

bool static_tile_ok(int n, int B) {
    for (const auto& e : kStaticSpecs)
        if (e[0] == n && e[1] == B) return true;
    return false;
}

// (n, rows per tile, threads, blocks per SM) of the z-pass specialisations
#define COLA_ZC2R_SPECS(X)   \
    X(256, 16, 256, 1)       \
    X(384, 8, 128, 1)        \
    X(768, 8, 256, 2)        \
    X(1152, 4, 256, 2)       \
    X(1536, 4, 256, 2)       \
    X(2304, 2, 256, 2)

#define COLA_ZR2C_SPECS(X)   \
    X(256, 16, 256, 1)       \
    X(384, 8, 128, 1)        \
    X(768, 8, 256, 2)        \
    X(1152, 4, 256, 2)       \
    X(1536, 4, 256, 2)       \
    X(2304, 2, 256, 2)

// (n, warps per block, blocks per SM) of the warp-row r2c of the fixed-point
// counts; it takes precedence.  (At 1152 it was slower than the block tile,
// 6.6 ms against 5.8 ms, and a warp-row plain c2r was slower at 2304, 74 ms
// against 64 ms.)
#define COLA_ZWARP_SPECS(X) \
    X(2304, 16, 1)

template <int N, int W, int MB>
static int run_z_r2c_fix_w(unsigned long long* dep, float2* out, long long rs, long long nrows, float scale,
                           const float2* tw, FRow fr, cudaStream_t s) {
    constexpr size_t smem = z_warp_smem<N, W>();
    static_assert((smem + 1024) * MB <= 227 * 1024, "MB blocks must fit");
    if (!set_smem((const void*)k_fft_z_r2c_fix_w<N, W, MB>, smem)) return COLA_ECUDA;
    const long long units = (nrows + W - 1) / W;
    k_fft_z_r2c_fix_w<N, W, MB><<<persistent_grid(smem, (int)(units < 0x7fffffff ? units : 0x7fffffff), MB),
                                  32 * W, smem, s>>>(dep, out, rs, nrows, scale, tw, fr);
    return check_launch();
}

bool launch_z_c2r_static(float2* data, int n, long long rs, long long nrows, const float2* tw, cudaStream_t s,
                         int* rc) {

#define COLA_CASE(NN, RR, TT, MB)                                \
    if (n == NN) {                                               \
        *rc = run_z_c2r<NN, RR, TT, MB>(data, rs, nrows, tw, s); \
        return true;                                             \
    }
    COLA_ZC2R_SPECS(COLA_CASE)
#undef COLA_CASE
    return false;
}

bool launch_z_r2c_fix_static(unsigned long long* dep, float2* out, int n, long long rs, long long nrows,
                             float scale, const float2* tw, FRow fr, cudaStream_t s, int* rc) {
#define COLA_CASE(NN, WW, MB)                                                               \
    if (n == NN && nrows == (long long)NN * NN) {                                          \
        *rc = run_z_r2c_fix_w<NN, WW, MB>(dep, out, rs, nrows, scale, tw, fr, s);           \
        return true;                                                                        \
    }
    COLA_ZWARP_SPECS(COLA_CASE)
#undef COLA_CASE
#define COLA_CASE(NN, RR, TT, MB)                                                   \
    if (n == NN) {                                                                  \
        *rc = run_z_r2c_fix<NN, RR, TT, MB>(dep, out, rs, nrows, scale, tw, fr, s); \
        return true;                                                                \
    }
    COLA_ZR2C_SPECS(COLA_CASE)
#undef COLA_CASE
    return false;
}



// (n, rows per tile, threads, blocks per SM) of the fused r2c + deposit pass
#define COLA_ZR2CD_SPECS(X) \
    X(256, 16, 256, 1)      \
    X(384, 8, 128, 1)       \
    X(768, 8, 256, 2)       \
    X(1152, 4, 256, 2)      \
    X(1536, 4, 256, 2)      \
    X(2304, 2, 256, 2)

// (n, x rows per tile, threads, blocks per SM) of the fused c2r + gather pass
#define COLA_ZC2RG_SPECS(X) \
    X(256, 2, 128, 4)       \
    X(384, 2, 128, 4)       \
    X(768, 1, 256, 3)       \
    X(1152, 1, 256, 3)      \
    X(1536, 1, 256, 3)      \
    X(2304, 1, 256, 2)

// (n, rows per tile, groups of such tiles per block, blocks per SM) of the
// warp-row form of the fused r2c + deposit pass; it takes precedence
#define COLA_ZR2CDW_SPECS(X) \
    X(768, 4, 6, 1)          \
    X(1536, 4, 4, 1)

// (n, x rows per tile, groups of such tiles per block, blocks per SM) of the
// warp-row form of the fused c2r + gather pass; it takes precedence
#define COLA_ZC2RGW_SPECS(X) \
    X(768, 1, 8, 1)          \
    X(1536, 1, 8, 1)

bool fused_passes_warp_rows(int n) {
    bool r2c = false, c2r = false;
#define COLA_CASE(NN, ...) r2c = r2c || n == NN;
    COLA_ZR2CDW_SPECS(COLA_CASE)
#undef COLA_CASE
#define COLA_CASE(NN, ...) c2r = c2r || n == NN;
    COLA_ZC2RGW_SPECS(COLA_CASE)
#undef COLA_CASE
    return r2c && c2r;
}

bool launch_z_r2c_dep_static(const float* d, int nq, float inv_cell, const RowBins& bins, float2* out, int n,
                             long long rs, float scale, const float2* tw, FRow fr, float* delta_out, cudaStream_t s,
                             int* rc) {
#define COLA_CASE(NN, RR, GG, MB)                                                       \
    if (n == NN) {                                                                      \
        *rc = run_z_r2c_dep_w<NN, RR, GG, MB>(bins, out, rs, scale, tw, fr, delta_out, s); \
        return true;                                                                    \
    }
    COLA_ZR2CDW_SPECS(COLA_CASE)
#undef COLA_CASE
#define COLA_CASE(NN, RR, TT, MB)                                                                          \
    if (n == NN) {                                                                                         \
        *rc = run_z_r2c_dep<NN, RR, TT, MB>(d, nq, inv_cell, bins, out, rs, scale, tw, fr, delta_out, s); \
        return true;                                                                                       \
    }
    COLA_ZR2CD_SPECS(COLA_CASE)
#undef COLA_CASE
    return false;
}

bool launch_z_c2r_gather_static(float2* data, int n, long long rs, const float2* tw, FRow fr, const float* d, int nq,
                                float inv_cell, const RowBins& bins, float* slots, int* tx, cudaStream_t s, int* rc) {
#define COLA_CASE(NN, TX, GG, MB)                                                   \
    if (n == NN) {                                                                  \
        *tx = TX;                                                                   \
        *rc = run_z_c2r_gather_w<NN, TX, GG, MB>(data, rs, tw, fr, nq, bins, slots, s); \
        return true;                                                                \
    }
    COLA_ZC2RGW_SPECS(COLA_CASE)
#undef COLA_CASE
#define COLA_CASE(NN, TX, TT, MB)                                                                       \
    if (n == NN) {                                                                                      \
        *tx = TX;                                                                                       \
        *rc = run_z_c2r_gather<NN, TX, TT, MB>(data, rs, tw, fr, d, nq, inv_cell, bins, slots, s);     \
        return true;                                                                                    \
    }
    COLA_ZC2RG_SPECS(COLA_CASE)
#undef COLA_CASE
    return false;
}

bool launch_y_psi_static(float2* data, int n, int B, LineGeom lg, long long comp2, int nct, int ntiles,
                         const float2* tw, float kf, cudaStream_t s, int* rc) {
#define COLA_CASE(NN, BB, TT)                                                     \
    if (n == NN && B == BB) {                                                     \
        *rc = run_y_psi2<NN, BB, TT>(data, lg, comp2, nct, ntiles, tw, kf, s);   \
        return true;                                                              \
    }
    COLA_YPSI2_SPECS(COLA_CASE)
#undef COLA_CASE
#define COLA_CASE(NN, BB, TT)                                                   \
    if (n == NN && B == BB) {                                                   \
        *rc = run_y_psi<NN, BB, TT>(data, lg, comp2, nct, ntiles, tw, kf, s); \
        return true;                                                            \
    }
    COLA_STRIDED_SPECS(COLA_CASE)
#undef COLA_CASE
    return launch_y_psi_static_small(data, n, B, lg, comp2, nct, ntiles, tw, kf, s, rc);
}

}  // namespace cola
