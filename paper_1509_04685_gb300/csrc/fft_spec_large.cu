// Specialised strided and fused x/Green passes (fft_static.cuh) for the large
// meshes: 768^3, 1152^3, 1536^3 and 2304^3.
#include "fft_static.cuh"

namespace cola {

// (n, B, threads) of every specialisation; B is a tile width the runtime
// engine or the tile autotuner picks for n, so a specialisation replaces
// exactly the runtime kernel's launch for that (n, B)
#define COLA_STRIDED_SPECS(X) \
    X(768, 8, 512) \
    X(1152, 4, 512) \
    X(1536, 4, 512) \
    X(2304, 2, 512)

#define COLA_XGREEN_SPECS(X) \
    X(768, 8, 512) \
    X(1152, 4, 384) \
    X(1536, 4, 512) \
    X(2304, 2, 384)

bool launch_strided_static(float2* data, int n, int B, int sign, LineGeom lg, int nct, int ntiles,
                           const float2* tw, cudaStream_t s, int* rc) {
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
#define COLA_CASE(NN, BB, TT)                                                                  \
    if (n == NN && B == BB) {                                                                  \
        *rc = run_x_green<NN, BB, TT>(F, nct, ntiles, tw, gscale, kf, filt, nfilt, fstep, s); \
        return true;                                                                           \
    }
    COLA_XGREEN_SPECS(COLA_CASE)
#undef COLA_CASE
    return launch_x_green_static_small(F, n, B, nct, ntiles, tw, gscale, kf, filt, nfilt, fstep, s, rc);
}

}  // namespace cola
