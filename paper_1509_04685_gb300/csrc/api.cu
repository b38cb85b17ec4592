// C ABI entry points (include/cola.h): argument checking, workspace layout and
// the sequencing of the kernels of each call.  No allocation happens here:
// every buffer lives in the caller's workspace or state arrays.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "cola_common.cuh"

namespace cola {

static int check_config(const cola_config* c) {
    if (!c) return COLA_EINVAL;
    if (!mesh_ok(c->nq) || !mesh_ok(c->ng)) return COLA_EUNSUPPORTED_SIZE;
    if (!(c->box > 0.0) || !(c->a_init > 0.0) || !(c->a_final > c->a_init) || !(c->a_final <= 1.0))
        return COLA_EINVAL;
    if (c->n_steps < 2 || c->n_steps > kMaxSteps) return COLA_EINVAL;
    if (c->sampling < COLA_SAMPLING_LINEAR || c->sampling > COLA_SAMPLING_POW) return COLA_EINVAL;
    if (c->sampling == COLA_SAMPLING_POW && !(c->sampling_p > 0.0)) return COLA_EINVAL;
    const cola_cosmology& k = c->cosmo;
    if (!(k.omega_m > 0.0) || !(k.h > 0.0) || !(k.sigma8 > 0.0) || !(k.omega_b >= 0.0) || !(k.t_cmb > 0.0))
        return COLA_EINVAL;
    if (c->flags & COLA_FLAG_LEARNED) {
        if (!c->net) return COLA_EINVAL;
        const bool has_net = c->net->params && c->net->wpack;
        if (!has_net && (c->net->params || c->net->wpack || !c->net->filter)) return COLA_EINVAL;
        if (has_net && c->ng % 16) return COLA_EUNSUPPORTED_SIZE;  // conv bricks of 4 x 8 x 16 voxels
        if (c->net->filter && (c->net->nfilter < 2 || c->net->nfilter > 64)) return COLA_EINVAL;
        if (c->net->filter && (c->net->nfilter_a < 0 || c->net->nfilter_a > kMaxSteps)) return COLA_EINVAL;
    }
    return COLA_OK;
}

// the learned correction includes the convolution net (not the filter alone)
static bool net_on(const cola_config* c) {
    return (c->flags & COLA_FLAG_LEARNED) && c->net && c->net->params && c->net->wpack;
}

bool layout_for(const cola_config* cfg, Layout* L) {
    const int ng = cfg->ng, nq = cfg->nq;
    const size_t Mg = mesh_bytes(ng), Mq = mesh_bytes(nq);
    const size_t np = (size_t)nq * nq * nq, nb = (size_t)ng * ng;
    L->dep = align_up(kHdrBytes, 4096);
    // the step's bins and slots share the fixed-point region (never in use at the same time)
    size_t o = L->dep;
    L->bstart = o;
    o = align_up(o + (nb + 1) * 4, 256);
    L->bsums = o;
    o = align_up(o + scan_sums_bytes((long long)nb) + 4, 256);
    L->bkey = o;
    o = align_up(o + np * 4, 256);
    L->brank = o;
    o = align_up(o + np * 4, 256);
    L->bsorted = o;
    o = align_up(o + np * 4, 256);
    L->bcic = o;
    o = align_up(o + np * 16, 256);
    L->slots = o;
    o = align_up(o + 12 * np * 4, 256);
    const size_t dep_end = std::max(L->dep + (size_t)ng * ng * ng * 8, o);
    L->F = align_up(dep_end, 4096);
    L->ic = L->dep;
    L->pk_part = align_up(L->F + 2 * Mg, 4096);
    size_t end = L->F + 3 * Mg;
    L->lrn = 0;
    if (net_on(cfg)) {
        L->lrn = align_up(end, 4096);
        end = L->lrn + learned_bytes(ng, nq);
    }
    size_t ic_end = L->ic + 7 * Mq;
    size_t pk_end = L->pk_part + power_partial_bytes(ng / 2);
    if (ic_end > end) end = ic_end;
    if (pk_end > end) end = pk_end;
    L->total = align_up(end, 4096);
    return true;
}

static int check_ws(const cola_config* cfg, void* ws, size_t ws_bytes, Layout* L) {
    int rc = check_config(cfg);
    if (rc) return rc;
    layout_for(cfg, L);
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255)) return COLA_EINVAL;
    if (ws_bytes < L->total) return COLA_EWORKSPACE;
    return COLA_OK;
}

static bool state_ok(const cola_state* st, bool need_all) {
    if (!st || !st->d) return false;
    if (need_all && (!st->v || !st->psi1 || !st->psi2)) return false;
    return true;
}

static double host_node_a(const cola_config* c, int j) {
    const double t = (double)j / (double)(c->n_steps - 1);
    const double ai = c->a_init, af = c->a_final;
    if (c->sampling == COLA_SAMPLING_LOG) return std::exp(std::log(ai) + t * (std::log(af) - std::log(ai)));
    if (c->sampling == COLA_SAMPLING_POW) {
        const double p = c->sampling_p;
        return std::pow(std::pow(ai, p) + t * (std::pow(af, p) - std::pow(ai, p)), 1.0 / p);
    }
    return ai + t * (af - ai);
}

static inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

static BinBufs bin_bufs(void* ws, const Layout& L) {
    return BinBufs{reinterpret_cast<int*>(wsp(ws, L.bstart)), reinterpret_cast<int*>(wsp(ws, L.bsums)),
                   reinterpret_cast<int*>(wsp(ws, L.bkey)),   reinterpret_cast<int*>(wsp(ws, L.brank)),
                   reinterpret_cast<int*>(wsp(ws, L.bsorted)), reinterpret_cast<float4*>(wsp(ws, L.bcic))};
}
static float* slots_ptr(void* ws, const Layout& L) { return reinterpret_cast<float*>(wsp(ws, L.slots)); }

// the PM path (cola_pm_set_path): 0 automatic, 1 fused passes, 2 separate kernels
static int g_pm_path = 0;
static bool fused_path(const cola_config* cfg) {
    if (g_pm_path) return g_pm_path == 1;
    const double per_row = (double)cfg->nq * cfg->nq * cfg->nq / ((double)cfg->ng * cfg->ng);
    return fused_passes_warp_rows(cfg->ng) && per_row <= COLA_FUSED_MAX_PER_ROW;
}

// The PM force of Sec. 2.2 on the interleaved force mesh F (rows (ix, iy, c)
// of P complex): the particles are binned by mesh row; the r2c pass along z
// deposits them row tile by row tile in shared memory and transforms the rows
// (delta_k in component 0); y pass; the fused x pass (Green's function,
// gradient) replaces delta_k by F_x and Psi; the inverse y pass gives the three
// components.  The inverse z pass then either gathers the particles' partial
// CIC sums into the slots (to_slots; *tx receives its tile width) or writes the
// real force mesh (the learned net and the least-squares filter read it).
static int pm_mesh_forces(const cola_config* cfg, const cola_state* st, double green, void* ws, const Layout& L,
                          cudaStream_t s, const float* filt, int nfilt, bool learned, bool to_slots, int* tx) {
    const int ng = cfg->ng, nq = cfg->nq;
    float2* F = reinterpret_cast<float2*>(wsp(ws, L.F));
    const float2* tw = twiddle_ptr(ws, kTwMesh);
    const double ratio = (double)ng / (double)nq;
    const float scale = (float)(ratio * ratio * ratio / 1099511627776.0);
    const double ng3 = (double)ng * ng * ng;
    const long long P = fft_pitch(ng), n2 = (long long)ng * ng;
    const BinBufs bb = bin_bufs(ws, L);
    const RowBins bins{bb.start, bb.sorted, bb.cic, status_ptr(ws), (long long)nq * nq * nq, ng};
    const FRow fr = force_rows(ng);
    const bool fused = learned || fused_path(cfg);
    int rc;
    if (fused) {
        if ((rc = mark_dep_dirty(ws, s))) return rc;  // the bins overwrite the fixed-point region
        if ((rc = launch_bins(st->d, nq, ng, cfg->box, bb, status_ptr(ws), s))) return rc;
        // the net's input keeps delta in real space (first buffer of the learned region)
        if ((rc = fft_z_r2c_deposit(st->d, nq, bins, F, ng, cfg->box, scale, tw,
                                    learned ? reinterpret_cast<float*>(wsp(ws, L.lrn)) : nullptr, s)))
            return rc;
    } else {
        // zero counts to start from (the region is shared with the bins and the
        // 2LPT scratch); the r2c pass leaves them zero again, and only then is
        // the region marked clean
        unsigned long long* dep = reinterpret_cast<unsigned long long*>(wsp(ws, L.dep));
        if ((rc = clear_dep_if_dirty(ws, dep, (size_t)ng * ng * ng, s))) return rc;
        if ((rc = mark_dep_dirty(ws, s))) return rc;
        if ((rc = launch_deposit_ex(st->d, nullptr, nullptr, nullptr, dep, nq, ng, cfg->box, nullptr, status_ptr(ws),
                                    s, false)))
            return rc;
        if ((rc = fft_z_r2c(dep, F, ng, scale, tw, s, P, n2, fr))) return rc;
        if ((rc = mark_dep_clean(ws, s))) return rc;
    }
    const long long XB = 1ll << fr.xbs;
    // y lines of component 0 (outer x = xb XB + xi), then of all three components (outer 3 x + c)
    if ((rc = fft_lines(F, ng, -1, tw, s, LineGeom{3 * XB * P, ng, (int)XB, 3 * XB * ng * P, 3 * P}, kKYFwd)))
        return rc;
    const double kmax = std::sqrt(3.0) * 3.14159265358979323846 * ng / cfg->box;
    const float kf = (float)(2.0 * 3.14159265358979323846 / cfg->box);
    bool psi = false;
    if ((rc = fft_x_green(F, ng, (float)(green / ng3), kf, tw, s, filt, nfilt,
                          nfilt > 1 ? (float)(kmax / (nfilt - 1)) : 1.f, &psi)))
        return rc;
    if ((rc = fft_y_inverse_force(F, ng, tw, s, psi, kf))) return rc;
    if (to_slots && fused) return fft_z_c2r_gather(F, ng, st->d, nq, bins, slots_ptr(ws, L), cfg->box, tw, tx, s);
    if ((rc = fft_z_c2r(F, ng, tw, s, nullptr, 0, 1.f, P, 3 * n2))) return rc;
    if (learned) return net_forward(cfg->net, wsp(ws, L.lrn), ng, nq, (float)green, F, s);
    return COLA_OK;
}

// filter row of the learned correction for scale factor a: the nearest of the
// nfilter_a rows spaced linearly from a_init to a_final
static const float* filter_row(const cola_config* cfg, double a) {
    const cola_net* n = cfg->net;
    if (!n->filter || n->nfilter_a <= 1) return n->filter;
    const double u = (a - cfg->a_init) / (cfg->a_final - cfg->a_init) * (n->nfilter_a - 1);
    int r = (int)std::floor(u + 0.5);
    r = r < 0 ? 0 : (r > n->nfilter_a - 1 ? n->nfilter_a - 1 : r);
    return n->filter + (size_t)r * n->nfilter;
}

// The force of the configuration (plain, or with the learned filter and net).
// With to_slots and no net, the forces end as partial sums in the slots
// (*tx set); otherwise as the real force mesh (*tx = 0).
static int pm_forces_for(const cola_config* cfg, const cola_state* st, double green, void* ws, const Layout& L,
                         cudaStream_t s, bool to_slots, int* tx) {
    const bool net = net_on(cfg);
    to_slots = to_slots && !net;
    *tx = 0;
    if (cfg->flags & COLA_FLAG_LEARNED) {
        const double a = 1.5 * cfg->cosmo.omega_m / green;
        return pm_mesh_forces(cfg, st, green, ws, L, s, filter_row(cfg, a), cfg->net->filter ? cfg->net->nfilter : 0,
                              net, to_slots, tx);
    }
    return pm_mesh_forces(cfg, st, green, ws, L, s, nullptr, 0, false, to_slots, tx);
}

static const float2* twiddles_for(int n, const cola_config* cfg, void* ws, cudaStream_t s, int* rc) {
    if (cfg && n == cfg->ng) return twiddle_ptr(ws, kTwMesh);
    if (cfg && n == cfg->nq) return twiddle_ptr(ws, kTwLagr);
    float2* tw = twiddle_ptr(ws, kTwScratch);
    *rc = launch_twiddles(tw, n, s);
    return tw;
}

// One node (Eqs. 1-2): the PM forces from the positions, then the fused
// gather + kick + drift, the only kernel that reads v, psi1 and psi2.  With
// before_kick, stream s waits for that event first (cola_step_host brings
// those arrays in meanwhile).
int step_node(const cola_config* cfg, cola_state* st, int32_t step, void* ws, size_t ws_bytes, cudaStream_t s,
              cudaEvent_t before_kick) {
    Layout L;
    int rc = check_ws(cfg, ws, ws_bytes, &L);
    if (rc) return rc;
    if (!state_ok(st, true) || step < 0 || step >= cfg->n_steps) return COLA_EINVAL;
    const double green = 1.5 * cfg->cosmo.omega_m / host_node_a(cfg, step);
    int tx = 0;
    if ((rc = pm_forces_for(cfg, st, green, ws, L, s, true, &tx))) return rc;
    if (before_kick && cudaStreamWaitEvent(s, before_kick, 0) != cudaSuccess) return COLA_ECUDA;
    const double* row = table_ptr(ws) + (size_t)step * kTableCols;
    const int last = step == cfg->n_steps - 1, pm_only = (cfg->flags & COLA_FLAG_PM_ONLY) ? 1 : 0;
    if (tx)
        return launch_slot_kick_drift(slots_ptr(ws, L), bin_bufs(ws, L).rank, *st, row, cfg->nq, last, pm_only,
                                      status_ptr(ws), s);
    return launch_gather_kick_drift(reinterpret_cast<float2*>(wsp(ws, L.F)), *st, row, cfg->nq, cfg->ng, cfg->box,
                                    last, pm_only, status_ptr(ws), s);
}

}  // namespace cola

using namespace cola;

extern "C" {

int cola_workspace_size(const cola_config* cfg, size_t* bytes) {
    if (!bytes) return COLA_EINVAL;
    int rc = check_config(cfg);
    if (rc) return rc;
    Layout L;
    layout_for(cfg, &L);
    *bytes = L.total;
    return COLA_OK;
}

int cola_init(const cola_config* cfg, void* ws, size_t ws_bytes, void* stream) {
    Layout L;
    int rc = check_ws(cfg, ws, ws_bytes, &L);
    if (rc) return rc;
    cudaStream_t s = S(stream);
    if (cudaMemsetAsync(ws, 0, kHdrBytes, s) != cudaSuccess) return COLA_ECUDA;
    if ((rc = launch_twiddles(twiddle_ptr(ws, kTwMesh), cfg->ng, s))) return rc;
    if ((rc = launch_twiddles(twiddle_ptr(ws, kTwLagr), cfg->nq, s))) return rc;
    return launch_tables(cfg, table_ptr(ws), s);
}

int cola_ic_2lpt(const cola_config* cfg, uint64_t seed, cola_state* st, void* ws, size_t ws_bytes, void* stream) {
    Layout L;
    int rc = check_ws(cfg, ws, ws_bytes, &L);
    if (rc) return rc;
    if (!state_ok(st, true)) return COLA_EINVAL;
    if ((rc = cola_init(cfg, ws, ws_bytes, stream))) return rc;
    cudaStream_t s = S(stream);
    return launch_ic(cfg, seed, *st, ws, L, s);
}

int cola_pm_force(const cola_config* cfg, const cola_state* st, double a, float* force, void* ws, size_t ws_bytes,
                  void* stream) {
    Layout L;
    int rc = check_ws(cfg, ws, ws_bytes, &L);
    if (rc) return rc;
    if (!state_ok(st, false) || !force || !(a > 0.0)) return COLA_EINVAL;
    cudaStream_t s = S(stream);
    const double green = 1.5 * cfg->cosmo.omega_m / a;
    int tx = 0;
    if ((rc = pm_forces_for(cfg, st, green, ws, L, s, true, &tx))) return rc;
    if (tx) return launch_slot_force(slots_ptr(ws, L), bin_bufs(ws, L).rank, force, cfg->nq, s);
    return launch_gather(reinterpret_cast<float2*>(wsp(ws, L.F)), st->d, force, cfg->nq, cfg->ng, cfg->box, s);
}

int cola_step(const cola_config* cfg, cola_state* st, int32_t step, void* ws, size_t ws_bytes, void* stream) {
    return cola::step_node(cfg, st, step, ws, ws_bytes, S(stream), nullptr);
}

}  // extern "C"

// P(k) (or, with p2/p4, the redshift-space multipoles) of the state at node,
// drifted to a_out if a_out differs from the node's scale factor
static int power_common(const cola_config* cfg, const cola_state* st, int32_t node, double a_out, int32_t ng_pk,
                        int32_t flags, double* k, double* pk, double* nmodes, int32_t nbins, void* ws,
                        size_t ws_bytes, cudaStream_t s, double* p2, double* p4) {
    Layout L;
    int rc = check_ws(cfg, ws, ws_bytes, &L);
    if (rc) return rc;
    const bool rsd = p2 && p4;
    if (!state_ok(st, rsd) || !k || !pk || !nmodes) return COLA_EINVAL;
    if (!mesh_ok(ng_pk) || ng_pk > cfg->ng) return COLA_EUNSUPPORTED_SIZE;
    if (nbins != ng_pk / 2 || node < 0 || node >= cfg->n_steps || (flags & ~7)) return COLA_EINVAL;
    if ((flags & COLA_PK_ALIAS_ITER) && ((flags & 3) || rsd)) return COLA_EINVAL;
    const double a_node = host_node_a(cfg, node);
    const double* snap = nullptr;
    if (rsd || std::fabs(a_out - a_node) > 1e-12 * a_node) {
        if (!(a_out > 0.0) || !state_ok(st, true)) return COLA_EINVAL;
        double* sp = reinterpret_cast<double*>(wsp(ws, kHdrSnap));
        if ((rc = launch_snapshot_coeffs(cfg, a_node, a_out, sp, s))) return rc;
        snap = sp;
    }
    if ((rc = mark_dep_dirty(ws, s))) return rc;
    unsigned long long* dep = reinterpret_cast<unsigned long long*>(wsp(ws, L.dep));
    float2* mk = reinterpret_cast<float2*>(wsp(ws, L.F));  // plain ng_pk mesh in the force-mesh region
    const float2* tw = twiddles_for(ng_pk, cfg, ws, s, &rc);
    if (rc) return rc;
    const double ratio = (double)ng_pk / (double)cfg->nq;
    // the region is shared with the step's bins: start from zero counts (the z pass clears them again)
    if (cudaMemsetAsync(dep, 0, (size_t)ng_pk * ng_pk * ng_pk * 8, s) != cudaSuccess) return COLA_ECUDA;
    if ((rc = launch_deposit_ex(st->d, st->v, st->psi1, st->psi2, dep, cfg->nq, ng_pk, cfg->box, snap,
                                status_ptr(ws), s, rsd)))
        return rc;
    const long long Ppk = fft_pitch(ng_pk);
    if ((rc = fft_z_r2c(dep, mk, ng_pk, (float)(ratio * ratio * ratio / 1099511627776.0), tw, s, Ppk,
                        (long long)ng_pk * ng_pk, FRow{ng_pk, 0, 1})))
        return rc;
    if ((rc = fft_strided(mk, ng_pk, 1, -1, tw, s))) return rc;
    if ((rc = fft_strided(mk, ng_pk, 0, -1, tw, s))) return rc;
    return launch_power(mk, ng_pk, Ppk, cfg->box, flags, reinterpret_cast<double*>(wsp(ws, L.pk_part)), k, pk, nmodes,
                        nbins, s, p2, p4);
}

extern "C" {

int cola_power_spectrum(const cola_config* cfg, const cola_state* st, int32_t node, double a_out, int32_t ng_pk,
                        int32_t flags, double* k, double* pk, double* nmodes, int32_t nbins, void* ws,
                        size_t ws_bytes, void* stream) {
    return power_common(cfg, st, node, a_out, ng_pk, flags, k, pk, nmodes, nbins, ws, ws_bytes, S(stream), nullptr,
                        nullptr);
}

int cola_power_multipoles(const cola_config* cfg, const cola_state* st, int32_t node, double a_out, int32_t ng_pk,
                          int32_t flags, double* k, double* p0, double* p2, double* p4, double* nmodes, int32_t nbins,
                          void* ws, size_t ws_bytes, void* stream) {
    if (!p2 || !p4) return COLA_EINVAL;
    return power_common(cfg, st, node, a_out, ng_pk, flags, k, p0, nmodes, nbins, ws, ws_bytes, S(stream), p2, p4);
}

int cola_density(const cola_config* cfg, const cola_state* st, float* delta, void* ws, size_t ws_bytes,
                 void* stream) {
    Layout L;
    int rc = check_ws(cfg, ws, ws_bytes, &L);
    if (rc) return rc;
    if (!state_ok(st, false) || !delta) return COLA_EINVAL;
    cudaStream_t s = S(stream);
    unsigned long long* dep = reinterpret_cast<unsigned long long*>(wsp(ws, L.dep));
    if ((rc = mark_dep_dirty(ws, s))) return rc;
    if (cudaMemsetAsync(dep, 0, (size_t)cfg->ng * cfg->ng * cfg->ng * 8, s) != cudaSuccess) return COLA_ECUDA;
    if ((rc = launch_deposit_ex(st->d, nullptr, nullptr, nullptr, dep, cfg->nq, cfg->ng, cfg->box, nullptr,
                                status_ptr(ws), s)))
        return rc;
    const double ratio = (double)cfg->ng / (double)cfg->nq;
    return launch_fix_to_delta(dep, delta, cfg->ng, (float)(ratio * ratio * ratio / 1099511627776.0), s);
}

int cola_step_table(const cola_config* cfg, double* out, void* ws, size_t ws_bytes, void* stream) {
    Layout L;
    int rc = check_ws(cfg, ws, ws_bytes, &L);
    if (rc) return rc;
    if (!out) return COLA_EINVAL;
    return cudaMemcpyAsync(out, table_ptr(ws), (size_t)cfg->n_steps * kTableCols * sizeof(double),
                           cudaMemcpyDeviceToDevice, S(stream)) == cudaSuccess
               ? COLA_OK
               : COLA_ECUDA;
}

int32_t cola_fft_pitch(int32_t n) { return n > 0 ? fft_pitch(n) : 0; }

static int fft3d_common(int32_t n, float* data, void* ws, size_t ws_bytes) {
    if (!mesh_ok(n)) return COLA_EUNSUPPORTED_SIZE;
    if (!data || !ws || ws_bytes < kHdrBytes || (reinterpret_cast<uintptr_t>(ws) & 255) ||
        (reinterpret_cast<uintptr_t>(data) & 15))
        return COLA_EINVAL;
    return COLA_OK;
}

int cola_fft3d_r2c(int32_t n, float* data, void* ws, size_t ws_bytes, void* stream) {
    int rc = fft3d_common(n, data, ws, ws_bytes);
    if (rc) return rc;
    cudaStream_t s = S(stream);
    const float2* tw = twiddles_for(n, nullptr, ws, s, &rc);
    if (rc) return rc;
    float2* c = reinterpret_cast<float2*>(data);
    if ((rc = fft_z_r2c(nullptr, c, n, 0.f, tw, s, fft_pitch(n), (long long)n * n, FRow{n, 0, 1}))) return rc;
    if ((rc = fft_strided(c, n, 1, -1, tw, s))) return rc;
    return fft_strided(c, n, 0, -1, tw, s);
}

int cola_fft3d_c2r(int32_t n, float* data, void* ws, size_t ws_bytes, void* stream) {
    int rc = fft3d_common(n, data, ws, ws_bytes);
    if (rc) return rc;
    cudaStream_t s = S(stream);
    const float2* tw = twiddles_for(n, nullptr, ws, s, &rc);
    if (rc) return rc;
    float2* c = reinterpret_cast<float2*>(data);
    if ((rc = fft_strided(c, n, 0, +1, tw, s))) return rc;
    if ((rc = fft_strided(c, n, 1, +1, tw, s))) return rc;
    return fft_z_c2r(c, n, tw, s, nullptr, 0, 1.f, fft_pitch(n), (long long)n * n);
}

int cola_net_pack(const cola_net* net, void* stream) { return net_pack(net, S(stream)); }

int cola_net_grad(const cola_config* cfg, const cola_state* st, double a, const float* target, float* grad,
                  double* loss, void* ws, size_t ws_bytes, void* stream) {
    Layout L;
    int rc = check_ws(cfg, ws, ws_bytes, &L);
    if (rc) return rc;
    if (!net_on(cfg) || !state_ok(st, false) || !target || !grad || !loss || !(a > 0.0)) return COLA_EINVAL;
    cudaStream_t s = S(stream);
    const double green = 1.5 * cfg->cosmo.omega_m / a;
    int tx = 0;
    if ((rc = pm_forces_for(cfg, st, green, ws, L, s, false, &tx))) return rc;
    return net_backward(cfg->net, wsp(ws, L.lrn), cfg->ng, cfg->nq, cfg->box, (float)green,
                        reinterpret_cast<float2*>(wsp(ws, L.F)), st->d, target, grad, loss, s);
}

int cola_adam(float* params, const float* grad, float* m, float* v, int32_t n, int32_t t, float lr, float beta1,
              float beta2, float eps, void* stream) {
    if (!params || !grad || !m || !v || n <= 0 || t < 1) return COLA_EINVAL;
    return launch_adam(params, grad, m, v, n, t, lr, beta1, beta2, eps, S(stream));
}

int cola_filter_accumulate(const cola_config* cfg, const cola_state* st, double a, const float* target, int32_t nb,
                           float* basis, double* ATA, double* ATy, void* ws, size_t ws_bytes, void* stream) {
    Layout L;
    int rc = check_ws(cfg, ws, ws_bytes, &L);
    if (rc) return rc;
    if (!state_ok(st, false) || !target || !basis || !ATA || !ATy || nb < 2 || nb > 64 || !(a > 0.0))
        return COLA_EINVAL;
    cudaStream_t s = S(stream);
    const double green = 1.5 * cfg->cosmo.omega_m / a;
    const long long np3 = 3ll * cfg->nq * cfg->nq * cfg->nq;
    float* table = reinterpret_cast<float*>(wsp(ws, kHdrFilter));
    for (int b = 0; b < nb; ++b) {
        if ((rc = launch_basis_table(table, nb, b, s))) return rc;
        int tx = 0;
        if ((rc = pm_mesh_forces(cfg, st, green, ws, L, s, table, nb, false, false, &tx))) return rc;
        if ((rc = launch_gather(reinterpret_cast<float2*>(wsp(ws, L.F)), st->d, basis + (size_t)b * np3, cfg->nq,
                                cfg->ng, cfg->box, s)))
            return rc;
    }
    return launch_lsq_accumulate(basis, target, np3, nb, ATA, ATy, s);
}

int cola_filter_solve(const double* ATA, const double* ATy, int32_t nb, double ridge, float* T, void* stream) {
    if (!ATA || !ATy || !T || nb < 2 || nb > 64 || !(ridge >= 0.0)) return COLA_EINVAL;
    return launch_lsq_solve(ATA, ATy, nb, ridge, T, S(stream));
}

int cola_status(void* ws, size_t ws_bytes, void* stream) {
    if (!ws || ws_bytes < kHdrBytes) return COLA_EINVAL;
    cudaStream_t s = S(stream);
    int host = 0;
    if (cudaMemcpyAsync(&host, status_ptr(ws), sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return COLA_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return COLA_ECUDA;
    if (host != 0 && cudaMemsetAsync(status_ptr(ws), 0, sizeof(int), s) != cudaSuccess) return COLA_ECUDA;
    return host;
}

uint64_t cola_launch_count(void) { return g_launches; }

int cola_checks_enabled(void) { return kChecks ? 1 : 0; }

int cola_pm_set_path(int32_t mode) {
    if (mode < 0 || mode > 2) return COLA_EINVAL;
    g_pm_path = mode;
    return COLA_OK;
}

int cola_pm_path(const cola_config* cfg) {
    size_t need = 0;
    const int rc = cola_workspace_size(cfg, &need);  // validates cfg
    if (rc) return rc;
    return (net_on(cfg) || fused_path(cfg)) ? 1 : 2;
}

int cola_checks_probe(int32_t index, int32_t n, void* ws, size_t ws_bytes, void* stream) {
    if (!ws || ws_bytes < kHdrBytes || n < 1 || n > kProbeInts || index < 0 || index >= kProbeInts)
        return COLA_EINVAL;
    // without the device checks an index >= n is refused here; the write stays
    // inside the probe area of the header in either build
    if (!kChecks && index >= n) return COLA_EINVAL;
    return launch_checks_probe(reinterpret_cast<int*>(wsp(ws, kHdrProbe)), index, n, status_ptr(ws), S(stream));
}

const char* cola_last_cuda_error(void) {
    return g_last_cuda_error ? cudaGetErrorString((cudaError_t)g_last_cuda_error) : "no error";
}

const char* cola_strerror(int code) {
    switch (code) {
        case COLA_OK: return "ok";
        case COLA_EINVAL: return "invalid argument";
        case COLA_EWORKSPACE: return "workspace too small";
        case COLA_EUNSUPPORTED_SIZE: return "unsupported mesh size (must be even, <= 4096, factors 2, 3, 5)";
        case COLA_ECUDA: return "CUDA launch or runtime error";
        case COLA_ETIMEOUT: return "a bounded device wait gave up";
        case COLA_ENONFINITE: return "non-finite or out-of-range particle data";
        case COLA_EBOUNDS: return "an index failed its bounds check (COLA_CHECKS build)";
        default: return "unknown error";
    }
}

}  // extern "C"
