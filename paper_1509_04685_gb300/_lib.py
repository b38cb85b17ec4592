"""ctypes binding of libcola_gb300.so (include/cola.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  Tensors are passed by device pointer (``tensor.data_ptr()``); the
stream is the caller's current torch stream unless given.  There is no CPU
fallback: if the library is missing or fails to load, importing this module
raises.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
# COLA_GB300_CHECKS=1 loads the build with device bounds checks (build(checks=True))
CHECKS = os.environ.get("COLA_GB300_CHECKS", "0") == "1"
LIB_PATH = (os.path.join(_HERE, "_build_checks", "libcola_gb300_checks.so") if CHECKS else
            os.path.join(_HERE, "_build", "libcola_gb300.so"))

COLA_OK = 0
ERRORS = {-1: "COLA_EINVAL", -2: "COLA_EWORKSPACE", -3: "COLA_EUNSUPPORTED_SIZE", -4: "COLA_ECUDA",
          -5: "COLA_ETIMEOUT", -6: "COLA_ENONFINITE", -7: "COLA_EBOUNDS"}
SAMPLING_LINEAR, SAMPLING_LOG, SAMPLING_POW = 0, 1, 2
FLAG_PM_ONLY = 1
FLAG_LEARNED = 2
FLAG_MODIFIED_KDK = 4
NET_NPARAMS = 9971
NET_NPACK = 31104
NET_OFFSETS = {"W1": (0, (16, 4, 27)), "b1": (1728, (16,)), "W2": (1744, (16, 16, 27)), "b2": (8656, (16,)),
               "W3": (8672, (3, 16, 27)), "b3": (9968, (3,))}
PK_DECONV_CIC, PK_ALIAS_JING, PK_ALIAS_ITER = 1, 2, 4
TABLE_COLUMNS = ("a", "green", "c1", "c2", "kick", "drift", "dD1", "dD2", "D1", "D2", "dD1da", "dD2da")


class cola_cosmology(ctypes.Structure):
    _fields_ = [("omega_m", ctypes.c_double), ("omega_l", ctypes.c_double), ("omega_b", ctypes.c_double),
                ("h", ctypes.c_double), ("sigma8", ctypes.c_double), ("n_s", ctypes.c_double),
                ("t_cmb", ctypes.c_double)]


class cola_net(ctypes.Structure):
    _fields_ = [("params", ctypes.c_void_p), ("wpack", ctypes.c_void_p), ("filter", ctypes.c_void_p),
                ("nfilter", ctypes.c_int32), ("nfilter_a", ctypes.c_int32)]


class cola_config(ctypes.Structure):
    _fields_ = [("nq", ctypes.c_int32), ("ng", ctypes.c_int32), ("box", ctypes.c_double),
                ("a_init", ctypes.c_double), ("a_final", ctypes.c_double), ("n_steps", ctypes.c_int32),
                ("sampling", ctypes.c_int32), ("sampling_p", ctypes.c_double), ("flags", ctypes.c_uint32),
                ("cosmo", cola_cosmology), ("net", ctypes.POINTER(cola_net))]


class cola_state(ctypes.Structure):
    _fields_ = [("d", ctypes.c_void_p), ("v", ctypes.c_void_p), ("psi1", ctypes.c_void_p),
                ("psi2", ctypes.c_void_p)]


class ColaError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        detail = f"; CUDA: {LIB.cola_last_cuda_error().decode()}" if code == -4 else ""
        super().__init__(f"{what}: {ERRORS.get(code, code)} ({_strerror(code)}{detail})")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"COLA CUDA library not built ({LIB_PATH}); run paper_1509_04685_gb300.build.build"
                          f"({'checks=True' if CHECKS else ''})")
    lib = ctypes.CDLL(LIB_PATH)
    vp, sz, i32, dbl = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32, ctypes.c_double
    cfgp, stp = ctypes.POINTER(cola_config), ctypes.POINTER(cola_state)
    sigs = {
        "cola_workspace_size": ([cfgp, ctypes.POINTER(sz)], ctypes.c_int),
        "cola_init": ([cfgp, vp, sz, vp], ctypes.c_int),
        "cola_ic_2lpt": ([cfgp, ctypes.c_uint64, stp, vp, sz, vp], ctypes.c_int),
        "cola_pm_force": ([cfgp, stp, dbl, vp, vp, sz, vp], ctypes.c_int),
        "cola_step": ([cfgp, stp, i32, vp, sz, vp], ctypes.c_int),
        "cola_step_host": ([cfgp, stp, stp, i32, vp, sz, vp], ctypes.c_int),
        "cola_fof_workspace_size": ([cfgp, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
        "cola_fof": ([cfgp, stp, ctypes.c_double, vp, vp, sz, vp], ctypes.c_int),
        "cola_fof_halos": ([cfgp, vp, i32, vp, vp, vp, vp, sz, vp], ctypes.c_int),
        "cola_mass_function": ([cfgp, vp, vp, ctypes.c_int64, ctypes.c_double, ctypes.c_double, i32, vp, vp],
                               ctypes.c_int),
        "cola_power_spectrum": ([cfgp, stp, i32, dbl, i32, i32, vp, vp, vp, i32, vp, sz, vp], ctypes.c_int),
        "cola_density": ([cfgp, stp, vp, vp, sz, vp], ctypes.c_int),
        "cola_step_table": ([cfgp, vp, vp, sz, vp], ctypes.c_int),
        "cola_fft_pitch": ([i32], i32),
        "cola_fft3d_r2c": ([i32, vp, vp, sz, vp], ctypes.c_int),
        "cola_fft3d_c2r": ([i32, vp, vp, sz, vp], ctypes.c_int),
        "cola_status": ([vp, sz, vp], ctypes.c_int),
        "cola_launch_count": ([], ctypes.c_uint64),
        "cola_strerror": ([ctypes.c_int], ctypes.c_char_p),
        "cola_net_pack": ([ctypes.POINTER(cola_net), vp], ctypes.c_int),
        "cola_net_grad": ([cfgp, stp, dbl, vp, vp, vp, vp, sz, vp], ctypes.c_int),
        "cola_adam": ([vp, vp, vp, vp, i32, i32, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, vp],
                      ctypes.c_int),
        "cola_filter_accumulate": ([cfgp, stp, dbl, vp, i32, vp, vp, vp, vp, sz, vp], ctypes.c_int),
        "cola_filter_solve": ([vp, vp, i32, dbl, vp, vp], ctypes.c_int),
        "cola_ensemble_create": ([i32, cfgp, vp, stp, vp, vp, i32, i32, i32, ctypes.POINTER(vp)], ctypes.c_int),
        "cola_ensemble_launch": ([vp, vp], ctypes.c_int),
        "cola_ensemble_destroy": ([vp], None),
        "cola_fft_autotune": ([i32, vp, vp, sz, vp, ctypes.POINTER(i32)], ctypes.c_int),
        "cola_fft_set_tile": ([i32, i32], ctypes.c_int),
        "cola_particle_set_traversal": ([i32, i32], ctypes.c_int),
        "cola_power_multipoles": ([cfgp, stp, i32, dbl, i32, i32, vp, vp, vp, vp, vp, i32, vp, sz, vp], ctypes.c_int),
        "cola_profile_start": ([i32], ctypes.c_int),
        "cola_profile_stop": ([vp, vp, i32], ctypes.c_int),
        "cola_num_kernel_ids": ([], i32),
        "cola_kernel_name": ([i32], ctypes.c_char_p),
        "cola_fof_set_retry_cap": ([i32], ctypes.c_int),
        "cola_last_cuda_error": ([], ctypes.c_char_p),
        "cola_checkpoint_bytes": ([cfgp, ctypes.POINTER(sz)], ctypes.c_int),
        "cola_checkpoint_save": ([cfgp, stp, i32, vp, sz, vp], ctypes.c_int),
        "cola_checkpoint_load": ([cfgp, vp, sz, stp, ctypes.POINTER(i32), vp], ctypes.c_int),
        "cola_checks_enabled": ([], ctypes.c_int),
        "cola_checks_probe": ([i32, i32, vp, sz, vp], ctypes.c_int),
        "cola_pm_set_path": ([i32], ctypes.c_int),
        "cola_pm_path": ([cfgp], ctypes.c_int),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


LIB = _load()


def _strerror(code: int) -> str:
    return LIB.cola_strerror(code).decode()


def _check(rc: int, what: str):
    if rc != COLA_OK:
        raise ColaError(rc, what)


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    import torch
    return torch.cuda.current_stream().cuda_stream


def make_config(nq: int, ng: int, box: float, a_init: float, a_final: float = 1.0, n_steps: int = 40,
                sampling: int = SAMPLING_LINEAR, sampling_p: float = 1.0, flags: int = 0,
                omega_m=0.25, omega_l=0.75, omega_b=0.044, h=0.7, sigma8=0.8, n_s=0.95, t_cmb=2.7255, net=None):
    cosmo = cola_cosmology(omega_m, omega_l, omega_b, h, sigma8, n_s, t_cmb)
    cfg = cola_config(nq, ng, box, a_init, a_final, n_steps, sampling, sampling_p, flags, cosmo,
                      ctypes.pointer(net) if net is not None else None)
    cfg._net_ref = net  # keep the descriptor alive with the config
    return cfg


def make_net(params, wpack, filt=None) -> cola_net:
    """Descriptor of a learned correction: params (device float[NET_NPARAMS]),
    wpack (device bf16[NET_NPACK] storage), optional filter table: device
    float[nfilter], or float[nfilter_a, nfilter] with one row per scale-factor
    node (rows spaced linearly from a_init to a_final of the config)."""
    if filt is None:
        net = cola_net(_ptr(params), _ptr(wpack), None, 0, 0)
    elif filt.dim() == 2:
        net = cola_net(_ptr(params), _ptr(wpack), _ptr(filt), int(filt.shape[1]), int(filt.shape[0]))
    else:
        net = cola_net(_ptr(params), _ptr(wpack), _ptr(filt), int(filt.numel()), 1)
    net._tensors = (params, wpack, filt)  # the descriptor holds raw device pointers: keep the tensors alive
    return net


def cola_net_pack(net: cola_net, stream=None):
    _check(LIB.cola_net_pack(ctypes.byref(net), _stream(stream)), "cola_net_pack")


def cola_net_grad(cfg, st: cola_state, a: float, target, grad, loss, ws, stream=None):
    _check(LIB.cola_net_grad(ctypes.byref(cfg), ctypes.byref(st), a, _ptr(target), _ptr(grad), _ptr(loss), _ptr(ws),
                             ws.numel() * ws.element_size(), _stream(stream)), "cola_net_grad")


def cola_adam(params, grad, m, v, n: int, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(LIB.cola_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), n, t, lr, beta1, beta2, eps, _stream(stream)),
           "cola_adam")


def cola_filter_accumulate(cfg, st: cola_state, a: float, target, nb: int, basis, ATA, ATy, ws, stream=None):
    _check(LIB.cola_filter_accumulate(ctypes.byref(cfg), ctypes.byref(st), a, _ptr(target), nb, _ptr(basis), _ptr(ATA),
                                      _ptr(ATy), _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)),
           "cola_filter_accumulate")


def cola_filter_solve(ATA, ATy, nb: int, ridge: float, T, stream=None):
    _check(LIB.cola_filter_solve(_ptr(ATA), _ptr(ATy), nb, ridge, _ptr(T), _stream(stream)), "cola_filter_solve")


class Ensemble:
    """One CUDA graph replaying the 2LPT set-up and nodes [step_from, step_to)
    of every member (cola_ensemble_create); members are (cfg, seed, state, ws)."""

    def __init__(self, cfgs, seeds, states, workspaces, nstreams=8, step_from=0, step_to=None):
        n = len(cfgs)
        self._cfgs = (cola_config * n)(*cfgs)
        self._seeds = (ctypes.c_uint64 * n)(*seeds)
        self._states = (cola_state * n)(*states)
        self._ws = (ctypes.c_void_p * n)(*[_ptr(w) for w in workspaces])
        self._wsb = (ctypes.c_size_t * n)(*[w.numel() * w.element_size() for w in workspaces])
        self._keep = (cfgs, states, workspaces)
        st_to = cfgs[0].n_steps if step_to is None else step_to
        h = ctypes.c_void_p()
        _check(LIB.cola_ensemble_create(n, self._cfgs, self._seeds, self._states, self._ws, self._wsb, nstreams,
                                        step_from, st_to, ctypes.byref(h)), "cola_ensemble_create")
        self.handle = h

    def launch(self, stream=None):
        _check(LIB.cola_ensemble_launch(self.handle, _stream(stream)), "cola_ensemble_launch")

    def __del__(self):
        if getattr(self, "handle", None):
            LIB.cola_ensemble_destroy(self.handle)
            self.handle = None


def cola_fft_autotune(n: int, mesh, ws, stream=None) -> int:
    best = ctypes.c_int32(0)
    _check(LIB.cola_fft_autotune(n, _ptr(mesh), _ptr(ws), ws.numel() * ws.element_size(), _stream(stream),
                                 ctypes.byref(best)), "cola_fft_autotune")
    return best.value


def cola_fft_set_tile(n: int, B: int) -> None:
    _check(LIB.cola_fft_set_tile(n, B), "cola_fft_set_tile")


def cola_particle_set_traversal(edge: int, brick_k: int = 0) -> None:
    _check(LIB.cola_particle_set_traversal(edge, brick_k), "cola_particle_set_traversal")


def make_state(d, v=None, psi1=None, psi2=None) -> cola_state:
    return cola_state(_ptr(d), _ptr(v), _ptr(psi1), _ptr(psi2))


def cola_workspace_size(cfg: cola_config) -> int:
    out = ctypes.c_size_t(0)
    _check(LIB.cola_workspace_size(ctypes.byref(cfg), ctypes.byref(out)), "cola_workspace_size")
    return out.value


def cola_init(cfg, ws, stream=None):
    _check(LIB.cola_init(ctypes.byref(cfg), _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)), "cola_init")


def cola_ic_2lpt(cfg, seed: int, st: cola_state, ws, stream=None):
    _check(LIB.cola_ic_2lpt(ctypes.byref(cfg), seed, ctypes.byref(st), _ptr(ws), ws.numel() * ws.element_size(),
                            _stream(stream)), "cola_ic_2lpt")


def cola_pm_force(cfg, st: cola_state, a: float, force, ws, stream=None):
    _check(LIB.cola_pm_force(ctypes.byref(cfg), ctypes.byref(st), a, _ptr(force), _ptr(ws),
                             ws.numel() * ws.element_size(), _stream(stream)), "cola_pm_force")


def cola_step(cfg, st: cola_state, step: int, ws, stream=None):
    _check(LIB.cola_step(ctypes.byref(cfg), ctypes.byref(st), step, _ptr(ws), ws.numel() * ws.element_size(),
                         _stream(stream)), "cola_step")


def cola_step_host(cfg, host: cola_state, dev: cola_state, step: int, ws, stream=None):
    """cola_step on a state in host memory: host holds HOST pointers (copied in,
    d and v copied back before return), dev the device state."""
    _check(LIB.cola_step_host(ctypes.byref(cfg), ctypes.byref(host), ctypes.byref(dev), step, _ptr(ws),
                              ws.numel() * ws.element_size(), _stream(stream)), "cola_step_host")


def cola_fof_set_retry_cap(cap: int):
    _check(LIB.cola_fof_set_retry_cap(cap), "cola_fof_set_retry_cap")


def cola_fof_workspace_size(cfg) -> int:
    out = ctypes.c_size_t(0)
    _check(LIB.cola_fof_workspace_size(ctypes.byref(cfg), ctypes.byref(out)), "cola_fof_workspace_size")
    return out.value


def cola_fof(cfg, st: cola_state, b: float, group, fws, stream=None):
    _check(LIB.cola_fof(ctypes.byref(cfg), ctypes.byref(st), b, _ptr(group), _ptr(fws),
                        fws.numel() * fws.element_size(), _stream(stream)), "cola_fof")


def cola_fof_halos(cfg, group, min_members: int, halo_root, halo_size, n_halos, fws, stream=None):
    _check(LIB.cola_fof_halos(ctypes.byref(cfg), _ptr(group), min_members, _ptr(halo_root), _ptr(halo_size),
                              _ptr(n_halos), _ptr(fws), fws.numel() * fws.element_size(), _stream(stream)),
           "cola_fof_halos")


def cola_mass_function(cfg, halo_size, n_halos, max_halos: int, lo: float, dlog: float, nbins: int, counts,
                       stream=None):
    _check(LIB.cola_mass_function(ctypes.byref(cfg), _ptr(halo_size), _ptr(n_halos), max_halos, lo, dlog, nbins,
                                  _ptr(counts), _stream(stream)), "cola_mass_function")


def cola_power_spectrum(cfg, st: cola_state, node: int, a_out: float, ng_pk: int, flags: int, k, pk, nmodes, ws,
                        stream=None):
    _check(LIB.cola_power_spectrum(ctypes.byref(cfg), ctypes.byref(st), node, a_out, ng_pk, flags, _ptr(k), _ptr(pk),
                                   _ptr(nmodes), ng_pk // 2, _ptr(ws), ws.numel() * ws.element_size(),
                                   _stream(stream)), "cola_power_spectrum")


def cola_power_multipoles(cfg, st: cola_state, node: int, a_out: float, ng_pk: int, flags: int, k, p0, p2, p4,
                          nmodes, ws, stream=None):
    _check(LIB.cola_power_multipoles(ctypes.byref(cfg), ctypes.byref(st), node, a_out, ng_pk, flags, _ptr(k),
                                     _ptr(p0), _ptr(p2), _ptr(p4), _ptr(nmodes), k.numel(), _ptr(ws),
                                     ws.numel() * ws.element_size(), _stream(stream)), "cola_power_multipoles")


def cola_checkpoint_bytes(cfg) -> int:
    out = ctypes.c_size_t(0)
    _check(LIB.cola_checkpoint_bytes(ctypes.byref(cfg), ctypes.byref(out)), "cola_checkpoint_bytes")
    return out.value


def cola_checkpoint_save(cfg, st: cola_state, node: int, host, stream=None):
    """host: a HOST uint8 tensor (pinned for DMA) of cola_checkpoint_bytes."""
    _check(LIB.cola_checkpoint_save(ctypes.byref(cfg), ctypes.byref(st), node, _ptr(host),
                                    host.numel() * host.element_size(), _stream(stream)), "cola_checkpoint_save")


def cola_checkpoint_load(cfg, host, st: cola_state, stream=None) -> int:
    node = ctypes.c_int32(-1)
    _check(LIB.cola_checkpoint_load(ctypes.byref(cfg), _ptr(host), host.numel() * host.element_size(),
                                    ctypes.byref(st), ctypes.byref(node), _stream(stream)), "cola_checkpoint_load")
    return node.value


def cola_density(cfg, st: cola_state, delta, ws, stream=None):
    _check(LIB.cola_density(ctypes.byref(cfg), ctypes.byref(st), _ptr(delta), _ptr(ws),
                            ws.numel() * ws.element_size(), _stream(stream)), "cola_density")


def cola_step_table(cfg, out, ws, stream=None):
    _check(LIB.cola_step_table(ctypes.byref(cfg), _ptr(out), _ptr(ws), ws.numel() * ws.element_size(),
                               _stream(stream)), "cola_step_table")


def cola_fft_pitch(n: int) -> int:
    return LIB.cola_fft_pitch(n)


def cola_fft3d_r2c(n: int, data, ws, stream=None):
    _check(LIB.cola_fft3d_r2c(n, _ptr(data), _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)),
           "cola_fft3d_r2c")


def cola_fft3d_c2r(n: int, data, ws, stream=None):
    _check(LIB.cola_fft3d_c2r(n, _ptr(data), _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)),
           "cola_fft3d_c2r")


def cola_status(ws, stream=None) -> int:
    return LIB.cola_status(_ptr(ws), ws.numel() * ws.element_size(), _stream(stream))


def cola_launch_count() -> int:
    return LIB.cola_launch_count()


def cola_strerror(code: int) -> str:
    return _strerror(code)
