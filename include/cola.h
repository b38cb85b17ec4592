/*
 * cola.h -- C ABI of the GB300 COLA particle-mesh library.
 *
 * The library advances N-body particles with the COLA method studied in
 * Izard, Crocce & Fosalba, "ICE-COLA" (arXiv:1509.04685): particles move in the
 * frame comoving with their 2LPT trajectories (Eq. 1), and only the residual
 * displacement is integrated in time with particle-mesh forces (Eq. 2), on the
 * time nodes of Eq. 3.  Sec. 2.2 describes the force as a PM solve on a mesh
 * PM_grid times finer than the particle grid with one forward and three
 * inverse FFTs per step; Sec. 2.5 the CIC power-spectrum estimator.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Units: lengths in Mpc/h, time in 1/H0; momenta p = a^2 dx/dt.
 * Particles: Np = nq^3, index p = (i*nq + j)*nq + k (Lagrangian C order, z
 *   fastest).  Particle fields are SoA float arrays of 3*Np values: component c
 *   of particle p at [c*Np + p].  Lagrangian position q = (i,j,k)*L/nq + L/(2 ng)
 *   (the lattice sits at force-mesh cell midpoints); position x = q + d.
 * Memory: every pointer argument is a DEVICE pointer unless stated otherwise.
 *   All memory is owned by the caller: the library never allocates.  The
 *   workspace (size from cola_workspace_size) holds the FP64 step tables, the
 *   FFT twiddles and every mesh; its contents between calls are private.
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Every call only enqueues work and returns; results are ready when
 *   the stream is.  Calls on one workspace must not overlap in time.
 * Errors: host-side argument errors are returned immediately (negative codes,
 *   see cola_strerror).  Errors a kernel detects (non-finite input, a bounded
 *   wait that gave up) are latched in a status word inside the workspace and
 *   returned by cola_status.
 */
#ifndef COLA_GB300_H
#define COLA_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define COLA_OK 0
#define COLA_EINVAL (-1)            /* bad argument (NULL pointer, size, range) */
#define COLA_EWORKSPACE (-2)        /* workspace smaller than cola_workspace_size */
#define COLA_EUNSUPPORTED_SIZE (-3) /* a mesh side with a prime factor > 5, odd, or too large */
#define COLA_ECUDA (-4)             /* a CUDA launch or runtime call failed */
#define COLA_ETIMEOUT (-5)          /* a bounded device-side wait gave up */
#define COLA_ENONFINITE (-6)        /* a kernel met a NaN/Inf in its input */
#define COLA_EBOUNDS (-7)           /* a device bounds check failed (COLA_CHECKS builds only) */

#define COLA_SAMPLING_LINEAR 0 /* Eq. 3 with f(a) = a (the paper's choice, Sec. 4.2) */
#define COLA_SAMPLING_LOG 1    /* f(a) = ln a */
#define COLA_SAMPLING_POW 2    /* f(a) = a^p, p = sampling_p */

#define COLA_FLAG_PM_ONLY 1u /* App. B: plain PM, no LPT frame (v holds the full momentum) */
#define COLA_FLAG_LEARNED 2u /* force = filtered coarse PM force + conv-net residual (cfg->net) */
/* The modified kick and drift factors of Tassev, Zaldarriaga & Eisenstein (2013),
 * the COLA paper Sec. 1 cites for Eq. 2, in place of the standard ones: the
 * residual momentum is taken to vary as a^n, n = n_LPT = -2.5, about the time
 * the force (kick: the node a_j) or the momentum (drift: the midpoint
 * a_{j+1/2}) is known:  kick_j = (a_{j+1/2}^n - a_{j-1/2}^n) / (n a_j^n E(a_j)),
 * drift_j = a_{j+1/2}^-n int_{a_j}^{a_{j+1}} a^n da / (a^3 E).  Snapshots between
 * nodes (cola_power_spectrum's a_out) keep the standard drift. */
#define COLA_FLAG_MODIFIED_KDK 4u

#define COLA_PK_DECONV_CIC 1 /* divide each mode by W_CIC(k)^2 (Sec. 2.5) */
#define COLA_PK_ALIAS_JING 2 /* divide by prod_i [1 - 2/3 sin^2(pi n_i/ng)] (Jing 2005, Sec. 2.5) */
/* The full Jing (2005) correction, iterated (Sec. 2.5): divide each mode by
 * C(m) = sum over images |n_i| <= 2 of W_CIC^2(m + ng n) (|m + ng n|/|m|)^n_eff,
 * n_eff per bin the log-slope of the previous estimate between neighbouring
 * bins (clamped to [-4, 4]); start from flags 1 | 2, three iterations.  Use
 * alone (not with 1 or 2), and with cola_power_spectrum only. */
#define COLA_PK_ALIAS_ITER 4

/* Flat LCDM parameters (Sec. 2.1, MICE-GC: 0.25, 0.75, 0.044, 0.7, 0.8, 0.95). */
typedef struct cola_cosmology {
    double omega_m, omega_l, omega_b, h, sigma8, n_s;
    double t_cmb; /* K, used by the Eisenstein & Hu no-wiggle transfer function */
} cola_cosmology;

/* Learned coarse-mesh force correction (not in the paper; used with
 * COLA_FLAG_LEARNED, typically on a PM_grid = 1 mesh).  The force mesh is
 *   F = IFFT(T(|k|) F_k) + g net(delta, F/g),   g = 3/2 Om/a,
 * with T a radial transfer function (piecewise linear on nfilter nodes
 * k_b = b sqrt(3) pi ng / (L (nfilter - 1)); NULL means T = 1).  With
 * nfilter_a > 1 the filter holds nfilter_a rows of nfilter values, row r for
 * a_r = a_init + r (a_final - a_init) / (nfilter_a - 1), and a force at scale
 * factor a uses the nearest row (nfilter_a <= 1: one row for all a).  With
 * params = wpack = NULL the correction is the filter alone: no net, no net
 * buffers in the workspace and no mesh-size condition (the form for meshes
 * whose net activations would not fit).  net is three
 * circular 3x3x3 convolutions 4 -> 16 -> 16 -> 3 with ReLU, BF16 weights and
 * activations, FP32 accumulation.  params (device, FP32, COLA_NET_NPARAMS):
 *   W1 [16][4][27] @0, b1 [16] @1728, W2 [16][16][27] @1744, b2 [16] @8656,
 *   W3 [3][16][27] @8672, b3 [3] @9968   (tap t = 9 tx + 3 ty + tz reads x[v + t - 1]).
 * wpack (device, COLA_NET_NPACK bf16 values) holds the packed weights that
 * cola_net_pack writes from params; call it after every change of params. */
#define COLA_NET_NPARAMS 9971
#define COLA_NET_NPACK 31104
typedef struct cola_net {
    float* params;
    void* wpack;
    const float* filter;
    int32_t nfilter;
    int32_t nfilter_a;
} cola_net;

/* One simulation (Table 1's code parameters). */
typedef struct cola_config {
    int32_t nq;         /* particles per side (even) */
    int32_t ng;         /* force mesh cells per side: PM_grid * nq (Sec. 2.2); even, 2^a 3^b 5^c */
    double box;         /* L in Mpc/h */
    double a_init;      /* a_i = 1/(1+z_i) (Sec. 4.3) */
    double a_final;     /* a_f (1 in the paper) */
    int32_t n_steps;    /* number of time nodes n of Eq. 3 = force evaluations */
    int32_t sampling;   /* COLA_SAMPLING_* */
    double sampling_p;  /* exponent for COLA_SAMPLING_POW */
    uint32_t flags;     /* COLA_FLAG_* */
    cola_cosmology cosmo;
    const cola_net* net; /* host pointer, required with COLA_FLAG_LEARNED (ng a multiple of 16 with a net) */
} cola_config;

/* Particle state: four SoA float[3*Np] device arrays.
 * d: displacement x - q;  v: residual momentum p - p_LPT (Eq. 1);
 * psi1, psi2: first- and second-order LPT displacements at D1 = 1. */
typedef struct cola_state {
    float* d;
    float* v;
    float* psi1;
    float* psi2;
} cola_state;

/* Bytes of workspace that every call with this configuration needs (the
 * largest of the step, the 2LPT set-up and a P(k) on a mesh of side <= ng). */
int cola_workspace_size(const cola_config* cfg, size_t* bytes);

/* Fill the workspace's FP64 tables: growth factors D1, D2 (growth ODEs), the
 * per-node kick/drift integrals of the KDK scheme for Eq. 2 and the FFT
 * twiddles.  Required once per workspace before cola_step / cola_pm_force;
 * cola_ic_2lpt calls it itself.  Also clears the status word. */
int cola_init(const cola_config* cfg, void* ws, size_t ws_bytes, void* stream);

/* 2LPT initial conditions (Sec. 2.2: Gaussian random field + 2LPT).  White
 * noise from Philox-4x32-10 keyed by `seed` (the same field for every run with
 * that seed, Sec. 2.3), scaled by the Eisenstein-Hu no-wiggle P(k) normalised
 * to sigma8; writes psi1, psi2, d = D1(a_i) psi1 + D2(a_i) psi2 and v = 0.
 * Runs cola_init first. */
int cola_ic_2lpt(const cola_config* cfg, uint64_t seed, cola_state* st, void* ws, size_t ws_bytes,
                 void* stream);

/* Particle-mesh force at scale factor `a` (Eq. 2 right-hand side, -grad Phi
 * with lap Phi = 3/2 Om/a delta): CIC deposit, r2c FFT, Green's function and
 * ik gradient, three c2r FFTs, CIC gather.  `force` is SoA float[3*Np]. */
int cola_pm_force(const cola_config* cfg, const cola_state* st, double a, float* force, void* ws,
                  size_t ws_bytes, void* stream);

/* One COLA node j (0 <= j < n_steps): force at a_j, kick of the residual
 * momentum by the LPT-frame acceleration F - c1 psi1 - c2 psi2, then (j < n-1)
 * drift of d by the residual momentum plus the D1/D2 increments.  After node
 * j < n-1 the positions are at a_{j+1}; after the last node v is at a_f. */
int cola_step(const cola_config* cfg, cola_state* st, int32_t step, void* ws, size_t ws_bytes,
              void* stream);

/* End-to-end form of cola_step for a state held in HOST memory: copies
 * host->d, v, psi1, psi2 (each 3 Nq^3 float32, SoA, HOST pointers; pinned memory
 * gives asynchronous DMA) into the device state dev (DEVICE pointers, same
 * layout), runs node `step` exactly as cola_step does, and copies dev->d and
 * dev->v back into host->d and host->v.  The positions are copied on `stream`,
 * where the force computation starts at once; v, psi1 and psi2 are copied on
 * an internal stream meanwhile (it starts after the work already queued on
 * `stream`), and the kick waits for them.  The copies back are on `stream`;
 * the call returns after they have completed, so the host arrays hold the new
 * state on return.  Arguments are validated before any copy
 * (COLA_EINVAL, COLA_EWORKSPACE, or a config error); if the step itself fails,
 * dev holds the copied-in state and host is unchanged.  COLA_ECUDA on a failed
 * copy or synchronisation. */
int cola_step_host(const cola_config* cfg, const cola_state* host, cola_state* dev, int32_t step, void* ws,
                   size_t ws_bytes, void* stream);

/* Checkpoint and resume of a run (the paper has no counterpart: its runs
 * restart from the initial-condition seed).  A checkpoint is one HOST buffer
 * of cola_checkpoint_bytes: a 256-byte header (magic "COLACKP1", format
 * version, every field of cfg except the net pointer, the next time node to
 * run, the array size) followed by d, v, psi1, psi2 (each 3 Nq^3 float32, SoA,
 * as on the device).  The workspace is not part of it: cola_init rebuilds the
 * tables and twiddles bit for bit and the deposit mesh is all-zero between
 * calls, so after cola_init on a fresh workspace and cola_checkpoint_load,
 * cola_step(node), cola_step(node + 1), ... continue the run bit-identically.
 * cola_checkpoint_save copies st (DEVICE) into `host` and returns once the
 * copies have landed; node in [0, n_steps).  cola_checkpoint_load checks that
 * the header is this configuration's, field for field (COLA_EINVAL if not, or
 * if host_bytes is short, before any copy), copies the arrays into st and
 * returns the stored node in *node (HOST int32) once they have landed.  The
 * buffer is read back on a host of the same byte order.  COLA_ECUDA on a
 * failed copy. */
int cola_checkpoint_bytes(const cola_config* cfg, size_t* bytes);
int cola_checkpoint_save(const cola_config* cfg, const cola_state* st, int32_t node, void* host, size_t host_bytes,
                         void* stream);
int cola_checkpoint_load(const cola_config* cfg, const void* host, size_t host_bytes, cola_state* st, int32_t* node,
                         void* stream);

/* Matter power spectrum (Sec. 2.5) of the state on a CIC mesh of side ng_pk
 * (2 <= ng_pk <= ng, even, 2^a 3^b 5^c).  `node` is the time node the
 * positions sit at; if a_out differs from a_node the positions are first
 * drifted to a_out on the fly with the state's momentum (no force
 * evaluation).  k, pk, nmodes are DEVICE float64 arrays of nbins = ng_pk/2:
 * bin i holds modes with (i+1/2)^2 > |n|^2 > (i-1/2)^2 (i = 1..ng_pk/2). */
int cola_power_spectrum(const cola_config* cfg, const cola_state* st, int32_t node, double a_out,
                        int32_t ng_pk, int32_t flags, double* k, double* pk, double* nmodes,
                        int32_t nbins, void* ws, size_t ws_bytes, void* stream);

/* Redshift-space multipoles about the z axis (the paper's RSD study, Eq. 5;
 * a plane-parallel line of sight along z): as cola_power_spectrum, but each
 * particle is first moved along z by its peculiar velocity,
 *   s_z = x_z + p_z / (a^2 E(a)),  p = v + a^3 E(a) (D1'(a) Psi1 + D2'(a) Psi2)
 * (p = v with COLA_FLAG_PM_ONLY), at a = a_out, and the shells accumulate
 *   P_l(k) = (2l + 1) <P L_l(mu)>, mu = k_z / |k|, l = 0, 2, 4
 * into p0, p2, p4 (DEVICE float64[nbins]).  Needs the full state (v, psi1,
 * psi2).  Same bins, flags, workspace and errors as cola_power_spectrum. */
int cola_power_multipoles(const cola_config* cfg, const cola_state* st, int32_t node, double a_out,
                          int32_t ng_pk, int32_t flags, double* k, double* p0, double* p2, double* p4,
                          double* nmodes, int32_t nbins, void* ws, size_t ws_bytes, void* stream);

/* Density contrast delta = rho (ng/nq)^3 - 1 of the state on the force mesh,
 * written unpadded as float[ng^3] (C order).  The deposit is deterministic
 * (fixed-point, 2^40 per particle). */
int cola_density(const cola_config* cfg, const cola_state* st, float* delta, void* ws,
                 size_t ws_bytes, void* stream);

/* FP64 step table as computed on the device: n_steps rows of 12 doubles
 * (a, green, c1, c2, kick, drift, dD1, dD2, D1, D2, dD1/da, dD2/da), copied
 * to the DEVICE array `out`. */
int cola_step_table(const cola_config* cfg, double* out, void* ws, size_t ws_bytes, void* stream);

/* In-place 3D FFTs of an n^3 mesh stored with half-complex row pitch
 * cola_fft_pitch(n) complex values (real rows padded to 2*pitch floats).
 * r2c is unnormalised (exp(-i k x)); c2r is the unnormalised inverse (the
 * caller divides by n^3). Uses the workspace of any config with ng >= n. */
int32_t cola_fft_pitch(int32_t n);
int cola_fft3d_r2c(int32_t n, float* data, void* ws, size_t ws_bytes, void* stream);
int cola_fft3d_c2r(int32_t n, float* data, void* ws, size_t ws_bytes, void* stream);

/* Synchronise `stream`, return the latched device status (COLA_OK or a
 * negative code) and clear it. */
int cola_status(void* ws, size_t ws_bytes, void* stream);

/* Number of kernels this library launched since load (a counter the host
 * side increments per launch). */
uint64_t cola_launch_count(void);

/* Write the packed BF16 weights of `net` from its FP32 parameters. */
int cola_net_pack(const cola_net* net, void* stream);

/* Gradient of the particle loss of the learned force (COLA_FLAG_LEARNED):
 *   L = 1/(2 Np) sum_p |F(p) - target(p)|^2
 * at scale factor a, through the CIC gather adjoint (a deposit of the
 * residuals) and the three convolutions.  target: device SoA float[3*Np];
 * grad: device float[COLA_NET_NPARAMS] (overwritten, W and b of all layers);
 * loss: device double[1]. */
int cola_net_grad(const cola_config* cfg, const cola_state* st, double a, const float* target, float* grad,
                  double* loss, void* ws, size_t ws_bytes, void* stream);

/* Adam step on n device floats: m, v moments, step t >= 1 (bias correction). */
int cola_adam(float* params, const float* grad, float* m, float* v, int32_t n, int32_t t, float lr, float beta1,
              float beta2, float eps, void* stream);

/* Normal equations of the radial filter fit (linear least squares: the
 * gathered force is linear in T).  For each hat basis function b < nb the
 * filtered coarse force G(IFFT(e_b(|k|) F_k)) at the particles forms column b;
 * ATA (nb*nb) and ATy (nb), device float64, are accumulated (not cleared) with
 * y = target.  basis: device scratch of nb*3*Np floats. */
int cola_filter_accumulate(const cola_config* cfg, const cola_state* st, double a, const float* target, int32_t nb,
                           float* basis, double* ATA, double* ATy, void* ws, size_t ws_bytes, void* stream);

/* Solve (ATA + ridge tr(ATA)/nb I) T = ATy (FP64 Cholesky on the device), T float[nb]. */
int cola_filter_solve(const double* ATA, const double* ATy, int32_t nb, double ridge, float* T, void* stream);

/* cola_density without any caller workspace, for callers that cannot hand the
 * library scratch memory: e.g. a host application whose device memory is all
 * owned by its own pool allocator, or an in-situ analysis inside a simulation
 * that has reserved the whole device.  The paper has no counterpart; this is
 * an integration convenience.  Same output as cola_density (delta as float[ng^3],
 * deterministic).  The fixed-point deposit mesh lives in one file-scope device
 * array of 128^3 cells (16 MiB per GPU that loads the library, held until the
 * process exits): ng > 128 returns COLA_EUNSUPPORTED_SIZE, and so do the
 * sizes cola_density rejects.  Nothing is allocated.  Outside stream capture
 * every call looks up the array's device address on the current device (so a
 * device reset needs nothing special); a call on a stream being captured
 * uses the address found by the last uncaptured call on that device, so make
 * one uncaptured call on each device first, and again after a device reset
 * (otherwise the captured call returns COLA_EINVAL).  There is one array per
 * device: calls that overlap in time on the same device (different streams
 * or host threads) share it and race; calls on different devices do not.
 * Each call clears the cells it uses first.  Non-finite particle data turns
 * the whole output into NaN; the next clean call is unaffected. */
int cola_density_noalloc(const cola_config* cfg, const cola_state* st, float* delta, void* stream);

/* Ensembles of independent realisations (Sec. 6 uses 48 realisations to beat
 * down sampling variance).  cola_ensemble_create captures, once, every
 * member's work (2LPT set-up when step_from == 0, then nodes
 * step_from .. step_to-1) into one CUDA graph: members are spread over
 * nstreams concurrent streams, largest first onto the least loaded stream.
 * cfgs, seeds, states, ws, ws_bytes are arrays of n (host arrays of device
 * pointers); sizes may differ between members.  cola_ensemble_launch replays
 * the whole ensemble with one graph launch on `stream`. */
typedef struct cola_ensemble cola_ensemble;
int cola_ensemble_create(int32_t n, const cola_config* cfgs, const uint64_t* seeds, const cola_state* states,
                         void* const* ws, const size_t* ws_bytes, int32_t nstreams, int32_t step_from,
                         int32_t step_to, cola_ensemble** out);
int cola_ensemble_launch(cola_ensemble* e, void* stream);
void cola_ensemble_destroy(cola_ensemble* e);

/* Friends-of-friends halos (Sec. 2.1: FoF, linking length 0.2 of the mean
 * inter-particle spacing; Sec. 2.5: halos of more than 100 particles with Warren
 * masses M = m_p N (1 - N^-0.6)).  Positions are q + d nq / L in units of the
 * mean spacing, periodic; two particles are friends when their minimum-image
 * separation is at most b (decided in FP32, each operation rounded once);
 * groups are the connected components.  Needs nq^3 < 2^31 and 0 < b < 1/2.
 *
 * cola_fof_workspace_size: bytes of the FoF workspace `fws` (device memory,
 * caller-owned, about 24 bytes per particle; separate from the step's).
 * cola_fof: group[p] (DEVICE int32[nq^3]) = the smallest particle index in
 * p's group, from st->d (only d is read).  Deterministic.  Synchronises
 * `stream` before returning, to report COLA_ENONFINITE (a non-finite position;
 * that particle is left alone) or COLA_ETIMEOUT (a bounded union-find retry
 * loop gave up).
 * cola_fof_halos: the groups of at least min_members particles (the paper's
 * samples: min_members = 101, "more than 100"), ordered by
 * root: halo_root[h], halo_size[h] (DEVICE int32 arrays with room for
 * nq^3 / min_members entries) and *n_halos (DEVICE int64).  Uses fws.
 * cola_mass_function: counts[i] (DEVICE int64[nbins]) = halos with
 * log10(M / (Msun/h)) in [lo + i dlog, lo + (i+1) dlog), M the Warren mass
 * with m_p = rho_c Omega_m (L / nq)^3, rho_c = 2.77536627e11 h^2 Msun Mpc^-3;
 * reads the first min(*n_halos, max_halos) entries of halo_size. */
int cola_fof_workspace_size(const cola_config* cfg, size_t* bytes);
int cola_fof(const cola_config* cfg, const cola_state* st, double b, int32_t* group, void* fws, size_t fws_bytes,
             void* stream);
/* Bound on the retries of each union-find find, union and flattening loop of
 * cola_fof (default 2^20, far above any real chain: 0 restores it; 1 <= cap
 * <= 2^30).  A loop that reaches it stops and cola_fof returns COLA_ETIMEOUT
 * (the labels are then not valid).  A hook for testing that error path
 * without any wait running long; process-wide, not thread-safe against
 * concurrent cola_fof calls. */
int cola_fof_set_retry_cap(int32_t cap);

int cola_fof_halos(const cola_config* cfg, const int32_t* group, int32_t min_members, int32_t* halo_root,
                   int32_t* halo_size, int64_t* n_halos, void* fws, size_t fws_bytes, void* stream);
int cola_mass_function(const cola_config* cfg, const int32_t* halo_size, const int64_t* n_halos, int64_t max_halos,
                       double log10m_lo, double dlog10m, int32_t nbins, int64_t* counts, void* stream);

/* FFT tile autotuner: times the y pass of an n^3 mesh (device buffer of
 * n*n*2*cola_fft_pitch(n) floats, contents destroyed) for each admissible
 * column width and keeps the fastest for all later passes of that size in this
 * process; *best receives it (may be NULL). */
int cola_fft_autotune(int32_t n, float* mesh, void* ws, size_t ws_bytes, void* stream, int32_t* best);

/* Set the column width B (2, 4, 8 or 16 adjacent columns per tile) of every
 * later strided pass of line length n in this process, as the autotuner does;
 * B = 0 restores the built-in default.  Results do not depend on B (same
 * arithmetic per line).  Returns COLA_EINVAL for n outside 2..4096, another B,
 * or a B whose tile buffers exceed the shared memory of one block. */
int cola_fft_set_tile(int32_t n, int32_t B);

/* PM path of every later force computation and step in this process (Sec. 2.2;
 * the same force either way, up to FP32 rounding order):
 *   1: fused passes: particles binned by mesh row, the CIC deposit inside the
 *      z r2c pass (shared-memory counts), the CIC gather inside the z c2r pass
 *      (partial sums per particle), then the kick;
 *   2: separate kernels: global fixed-point deposit, z r2c of the counts, the
 *      real force mesh written by the z c2r pass, then gather + kick;
 *   0: automatic (the default): fused where the library has warp-row forms
 *      of both fused z passes (ng = 768, 1536) and the particles per (x, y)
 *      mesh row, nq^3 / ng^2, are at most COLA_FUSED_MAX_PER_ROW; separate
 *      otherwise.  The fused passes visit each particle in four tiles; with
 *      many particles per row that costs more than the mesh traffic it saves,
 *      and the other mesh sizes' fused forms are slower than the separate
 *      kernels (measured on GB300: 512^3 on 1536^3, 57 per row, 84 ms fused
 *      against 87 ms separate; 768^3 on 1152^3, 341 per row, 117 ms against
 *      66 ms; 768^3 on 2304^3 376 ms against 364 ms).
 * The learned convolution net always takes the fused deposit (it needs delta
 * in real space from it) and the real force mesh.  Returns COLA_EINVAL for
 * another mode. */
#define COLA_FUSED_MAX_PER_ROW 96
int cola_pm_set_path(int32_t mode);

/* The PM path the next force computation or step of cfg takes under the
 * current mode: 1 (fused passes) or 2 (separate kernels); COLA_EINVAL (or a
 * config error) if cfg is invalid.  Host only: no launch, no device access. */
int cola_pm_path(const cola_config* cfg);

/* Set the traversal order of the particle kernels (deposit, gather, fused
 * gather + kick + drift, adjoint deposit) for later launches in this process:
 * each 256-thread block takes a brick of I x J x brick_k Lagrangian sites
 * (i, j, k; J = min(8, 256 / brick_k), I = 256 / (J brick_k)), bricks are
 * grouped in cubic tiles of edge^3 sites, tiles in raster order.  For a lattice
 * of nq^3 sites the tile edge used is the largest power of two not above
 * `edge` whose padded lattice is within 5% of nq^3 (else the one that pads
 * least).  The order only shapes the mesh traffic (locality in L2 once
 * particles have left their lattice sites): every particle is visited once and
 * the results are bit-identical for any choice.  brick_k is a power of two in
 * 8..256, edge a power of two in 32..4096 and >= brick_k; 0 restores the
 * built-in value of either.  Returns COLA_EINVAL for anything else. */
int cola_particle_set_traversal(int32_t edge, int32_t brick_k);

/* Per-kernel timing (tracing): between cola_profile_start and
 * cola_profile_stop every kernel launch of the library is bracketed by CUDA
 * events on its own stream (at most max_records launches are recorded).
 * cola_profile_stop synchronises on the events and returns, per kernel id,
 * the summed milliseconds and the launch count (arrays of at least
 * cola_num_kernel_ids() entries, HOST memory). */
int cola_profile_start(int32_t max_records);
int cola_profile_stop(double* ms, int64_t* launches, int32_t nkernels);
int32_t cola_num_kernel_ids(void);
const char* cola_kernel_name(int32_t id);

const char* cola_strerror(int code);

/* The CUDA runtime's description of the error behind the most recent
 * COLA_ECUDA that a kernel launch or a shared-memory attribute call returned
 * (process-wide; "no error" if there was none).  A diagnostic aid only. */
const char* cola_last_cuda_error(void);

/* 1 if this library was built with COLA_CHECKS defined, else 0.  In that build
 * every data-dependent index of the PM step (the bin key of a particle's CIC
 * row, its sorted position from the bin scan as the scatter, the fused z
 * passes and the kick use it, the z cell stored in its CIC record) is checked
 * before the access it guards; a failed check skips the access and latches
 * COLA_EBOUNDS in the workspace's status word (read by cola_status).  The
 * checks replace a memory checker where none can run; results are
 * bit-identical to the normal build's. */
int cola_checks_enabled(void);

/* Test hook of the bounds checks: one device thread checks index < n and, if
 * the check passes, writes one int at position `index` of a 64-int probe area
 * in the workspace header.  COLA_EINVAL unless 1 <= n <= 64 and
 * 0 <= index < 64 (so the write always stays inside the probe area).  In a
 * COLA_CHECKS build an index >= n is caught on the device (the write is
 * skipped, COLA_EBOUNDS latched); in the normal build it is refused on the
 * host with COLA_EINVAL.  Asynchronous on `stream`; read the result with
 * cola_status. */
int cola_checks_probe(int32_t index, int32_t n, void* ws, size_t ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* COLA_GB300_H */
