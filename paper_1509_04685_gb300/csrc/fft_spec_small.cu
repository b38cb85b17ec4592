// Specialised strided and fused x/Green passes (fft_static.cuh) for the mesh
// sizes below 512: the batched-ensemble members and the parity-test meshes.
#include "fft_static.cuh"

namespace cola {

// (n, B, threads) of every specialisation: B adjacent columns per tile, two
// tile buffers of spad(n) B complex in shared memory
#define COLA_STRIDED_SPECS(X) \
    X(96, 16, 256) \
    X(128, 16, 256) \
    X(160, 16, 320) \
    X(192, 16, 384) \
    X(256, 16, 512) \
    X(256, 8, 256) \
    X(288, 16, 512) \
    X(320, 16, 512) \
    X(384, 16, 512) \
    X(384, 8, 384) \
    X(480, 16, 512) \
    X(480, 8, 512)

#define COLA_XGREEN_SPECS(X) \
    X(96, 16, 128, 2) \
    X(128, 16, 256, 2) \
    X(160, 16, 256, 2) \
    X(192, 16, 256, 2) \
    X(256, 16, 512, 2) \
    X(256, 8, 256, 2) \
    X(288, 16, 384, 2) \
    X(320, 16, 512, 2) \
    X(384, 16, 512, 2) \
    X(384, 8, 256, 2) \
    X(480, 16, 640, 2) \
    X(480, 8, 320, 2)

bool launch_strided_static_small(float2* data, int n, int B, int sign, LineGeom lg, int nct, int ntiles,
                           const float2* tw, cudaStream_t s, int* rc) {
#define COLA_CASE(NN, BB, TT)                                               \
    if (n == NN && B == BB) {                                               \
        *rc = run_strided<NN, BB, TT>(data, sign, lg, nct, ntiles, tw, s); \
        return true;                                                        \
    }
    COLA_STRIDED_SPECS(COLA_CASE)
#undef COLA_CASE
    return false;
}

bool launch_x_green_static_small(float2* F, int n, int B, int nct, int ntiles, const float2* tw, float gscale,
                           float kf, const float* filt, int nfilt, float fstep, cudaStream_t s, int* rc) {
#define COLA_CASE(NN, BB, TT, NBUF)                                                                  \
    if (n == NN && B == BB) {                                                                        \
        *rc = run_x_green<NN, BB, TT, NBUF>(F, nct, ntiles, tw, gscale, kf, filt, nfilt, fstep, s); \
        return true;                                                                                 \
    }
    COLA_XGREEN_SPECS(COLA_CASE)
#undef COLA_CASE
    return false;
}

// the small meshes run the fused pass at the strided passes' width
int launch_static_green_tile_small(int) { return 0; }


bool launch_y_psi_static_small(float2* data, int n, int B, LineGeom lg, long long comp2, int nct, int ntiles,
                         const float2* tw, float kf, cudaStream_t s, int* rc) {
#define COLA_CASE(NN, BB, TT)                                                   \
    if (n == NN && B == BB) {                                                   \
        *rc = run_y_psi<NN, BB, TT>(data, lg, comp2, nct, ntiles, tw, kf, s); \
        return true;                                                            \
    }
    COLA_STRIDED_SPECS(COLA_CASE)
#undef COLA_CASE
    return false;
}

}  // namespace cola
