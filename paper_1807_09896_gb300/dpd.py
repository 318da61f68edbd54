"""Thin ctypes binding of the C ABI in ``include/dpd.h`` (same names, argument marshalling only).

Every step of the time-stepping path runs in the CUDA library ``libdpd.so``; this
module converts numpy arrays (host memory) or torch CUDA tensors (device memory)
into pointers and turns negative return codes into :class:`DPDError`.  There is no
CPU fallback: if the library is missing or the machine has no GPU, calls fail.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libdpd.so")

DPD_OK, DPD_EINVAL, DPD_ENOMEM, DPD_ECUDA, DPD_ESTATE = 0, -1, -2, -3, -4
DPD_ELOST, DPD_EBAND, DPD_ETIMEOUT, DPD_ENAN, DPD_EOVERFLOW = -5, -6, -7, -8, -9
DPD_HOST, DPD_DEVICE = 0, 1

ERROR_NAMES = {
    DPD_EINVAL: "DPD_EINVAL", DPD_ENOMEM: "DPD_ENOMEM", DPD_ECUDA: "DPD_ECUDA",
    DPD_ESTATE: "DPD_ESTATE", DPD_ELOST: "DPD_ELOST", DPD_EBAND: "DPD_EBAND",
    DPD_ETIMEOUT: "DPD_ETIMEOUT", DPD_ENAN: "DPD_ENAN", DPD_EOVERFLOW: "DPD_EOVERFLOW",
}

# Every entry point of include/dpd.h: name -> (restype, argtypes)
_vp = ctypes.c_void_p
_d = ctypes.c_double
_i = ctypes.c_int
_SIGS = {
    "dpd_create": (_i, [ctypes.POINTER(_vp), _vp, _d, _vp, _d, _d, _d, _d, _vp]),
    "dpd_set_phase_field": (_i, [_vp, _vp, _vp, _d]),
    "dpd_set_particles": (_i, [_vp, _i, _vp, _vp, _vp, _vp, _i]),
    "dpd_step": (_i, [_vp, _i]),
    "dpd_time_phases": (_i, [_vp, _i, _vp]),
    "dpd_autotune": (_i, [_vp, _i, _vp, ctypes.POINTER(_i)]),
    "dpd_get_state": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _i]),
    "dpd_adjoint_window": (_i, [_vp, _i, _i, _i, _d, _d, _i, _d, _vp, _i, _vp, _vp]),
    "dpd_adjoint_window_record": (_i, [_vp, _i, _i, _i, _d, _d, _i, _d, _vp, _i, _vp, _vp, _vp, _vp,
                                       _vp, _vp, _vp]),
    "dpd_velocity_profile": (_i, [_vp, _i, _i, _d, _d, _vp, _i]),
    "dpd_velocity_profile_noalloc": (_i, [_vp, _vp, _vp, _i, _i, _i, _d, _d, _vp, _i, _vp]),
    "dpd_relax_phase_field": (_i, [_vp, _vp, _d, _d, _i, _d, _i, _vp]),
    "dpd_init_particles": (_i, [_vp, ctypes.c_uint64, _d]),
    "dpd_get_stats": (_i, [_vp, _vp]),
    "dpd_set_option": (_i, [_vp, ctypes.c_char_p, _d]),
    "dpd_get_option": (_i, [_vp, ctypes.c_char_p, ctypes.POINTER(_d)]),
    "dpd_num_particles": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "dpd_set_stream": (_i, [_vp, _vp]),
    "dpd_destroy": (_i, [_vp]),
    "dpd_last_error": (ctypes.c_char_p, [_vp]),
    "dpd_batch_create": (_i, [ctypes.POINTER(_vp), _i, _vp]),
    "dpd_batch_step": (_i, [_vp, _i]),
    "dpd_batch_time_phases": (_i, [_vp, _i, _vp]),
    "dpd_batch_autotune": (_i, [_vp, _i, _vp, ctypes.POINTER(_i)]),
    "dpd_batch_get_state": (_i, [_vp, _i, _vp, _vp, _vp, _vp, _vp, _i]),
    "dpd_batch_get_stats": (_i, [_vp, _i, _vp]),
    "dpd_batch_set_option": (_i, [_vp, ctypes.c_char_p, _d]),
    "dpd_batch_get_option": (_i, [_vp, ctypes.c_char_p, ctypes.POINTER(_d)]),
    "dpd_batch_num_particles": (_i, [_vp, _i, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "dpd_batch_set_stream": (_i, [_vp, _vp]),
    "dpd_batch_destroy": (_i, [_vp]),
    "dpd_batch_last_error": (ctypes.c_char_p, [_vp]),
}

_lib = None


class DPDError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Load ``libdpd.so`` (built by ``paper_1807_09896_gb300._build``); fails loudly if absent."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library {p} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(p)
    for name, (res, args) in _SIGS.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = L
    return L


def _ptr(a, dtype=None):
    """Pointer of a numpy array (host) or a torch tensor (its data_ptr)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    if dtype is not None:
        assert a.dtype == dtype and a.flags["C_CONTIGUOUS"], (a.dtype, dtype)
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(h, rc):
    if rc != DPD_OK:
        raise DPDError(rc, dpd_last_error(h))
    return rc


def dpd_last_error(h) -> str:
    return load_library().dpd_last_error(h).decode(errors="replace")


def dpd_create(box, rho, a_ij, gamma, sigma, kBT, dt, body_force):
    L = load_library()
    h = ctypes.c_void_p()
    b = np.ascontiguousarray(box, np.float64)
    a = np.ascontiguousarray(a_ij, np.float64)
    g = np.ascontiguousarray(body_force, np.float64)
    assert b.shape == (3,) and a.shape == (4,) and g.shape == (3,)
    rc = L.dpd_create(ctypes.byref(h), _ptr(b), rho, _ptr(a), gamma, sigma, kBT, dt, _ptr(g))
    if rc != DPD_OK:
        raise DPDError(rc, L.dpd_last_error(None).decode(errors="replace"))
    return h


def dpd_set_phase_field(h, grid, spacing):
    """grid: float32 array shaped (nz, ny, nx) (x fastest), host memory."""
    g = np.ascontiguousarray(grid, np.float32)
    nz, ny, nx = g.shape
    dims = np.asarray([nx, ny, nz], np.int32)
    return _check(h, load_library().dpd_set_phase_field(h, _ptr(g), _ptr(dims), spacing))


def dpd_set_particles(h, pos4, vel4, ids, types, where=DPD_HOST):
    n = len(ids)
    if where == DPD_HOST:
        pos4 = np.ascontiguousarray(pos4, np.float32)
        vel4 = np.ascontiguousarray(vel4, np.float32)
        ids = np.ascontiguousarray(ids, np.int32)
        types = np.ascontiguousarray(types, np.uint8)
        assert pos4.shape == (n, 4) and vel4.shape == (n, 4) and types.shape == (n,)
    return _check(h, load_library().dpd_set_particles(h, n, _ptr(pos4), _ptr(vel4), _ptr(ids),
                                                      _ptr(types), where))


def dpd_step(h, nsteps: int):
    return _check(h, load_library().dpd_step(h, int(nsteps)))


PHASES = ("integrate", "scan", "scatter", "cell_sort", "gather", "force_pairs", "force_finish")


def dpd_time_phases(h, nsteps: int) -> dict:
    """Mean duration (ms) of each phase of a step over nsteps event-timed steps."""
    ms = np.zeros(len(PHASES), np.float64)
    _check(h, load_library().dpd_time_phases(h, int(nsteps), _ptr(ms)))
    return dict(zip(PHASES, ms.tolist()))


def dpd_autotune(h, nsteps: int = 5):
    """Time every launch shape of the force kernel; keep the fastest.  Returns
    (chosen index, list of mean force ms per shape)."""
    nv = int(dpd_get_option(h, "force_variants"))
    ms = np.zeros(nv, np.float64)
    chosen = ctypes.c_int()
    _check(h, load_library().dpd_autotune(h, int(nsteps), _ptr(ms), ctypes.byref(chosen)))
    return chosen.value, ms.tolist()


def dpd_adjoint_window(h, nsteps, ckpt_every, axis, wall_lo, wall_hi, target, bin_width,
                       tie_sigma=True):
    """Loss and gradient (dL/da_fs, dL/dgamma, dL/dg_x) of the near-wall profile loss
    over a window of nsteps steps (see include/dpd.h)."""
    t = np.ascontiguousarray(target, np.float64)
    grad = np.zeros(3, np.float64)
    loss = np.zeros(1, np.float64)
    _check(h, load_library().dpd_adjoint_window(h, int(nsteps), int(ckpt_every), int(axis),
                                                float(wall_lo), float(wall_hi), len(t),
                                                float(bin_width), _ptr(t), int(bool(tie_sigma)),
                                                _ptr(loss), _ptr(grad)))
    return float(loss[0]), grad


def dpd_adjoint_window_record(h, nsteps, ckpt_every, axis, wall_lo, wall_hi, target, bin_width,
                              tie_sigma=True):
    """As dpd_adjoint_window, plus the record of include/dpd.h: a dict with ckpt and
    adj ((nseg + 1, n, 3, 4) float32, id order), seg_grad (nseg, 3), coef (nbins,)
    and seg_step (nseg + 1,)."""
    t = np.ascontiguousarray(target, np.float64)
    n = dpd_num_particles(h)[0]
    nseg = int(nsteps) // int(ckpt_every)
    rec = {"ckpt": np.zeros((nseg + 1, n, 3, 4), np.float32),
           "adj": np.zeros((nseg + 1, n, 3, 4), np.float32),
           "seg_grad": np.zeros((nseg, 3), np.float64), "coef": np.zeros(len(t), np.float32),
           "seg_step": np.zeros(nseg + 1, np.uint32)}
    grad = np.zeros(3, np.float64)
    loss = np.zeros(1, np.float64)
    _check(h, load_library().dpd_adjoint_window_record(
        h, int(nsteps), int(ckpt_every), int(axis), float(wall_lo), float(wall_hi), len(t),
        float(bin_width), _ptr(t), int(bool(tie_sigma)), _ptr(loss), _ptr(grad), _ptr(rec["ckpt"]),
        _ptr(rec["adj"]), _ptr(rec["seg_grad"]), _ptr(rec["coef"]), _ptr(rec["seg_step"])))
    return float(loss[0]), grad, rec


def dpd_num_particles(h):
    n, nf = ctypes.c_int(), ctypes.c_int()
    _check(h, load_library().dpd_num_particles(h, ctypes.byref(n), ctypes.byref(nf)))
    return n.value, nf.value


def dpd_get_state(h, pos4=None, vel4=None, force4=None, ids=None, types=None, where=DPD_HOST):
    """Read the state in id order.  With where=DPD_HOST and no buffers given, returns
    new numpy arrays (pos4, vel4, force4, ids, types)."""
    if where == DPD_HOST and all(x is None for x in (pos4, vel4, force4, ids, types)):
        n, _ = dpd_num_particles(h)
        pos4 = np.zeros((n, 4), np.float32)
        vel4 = np.zeros((n, 4), np.float32)
        force4 = np.zeros((n, 4), np.float32)
        ids = np.zeros(n, np.int32)
        types = np.zeros(n, np.uint8)
    _check(h, load_library().dpd_get_state(h, _ptr(pos4), _ptr(vel4), _ptr(force4), _ptr(ids),
                                           _ptr(types), where))
    return pos4, vel4, force4, ids, types


def dpd_velocity_profile(h, axis: int, nbins: int, lo: float, hi: float, mode: int = 0,
                         out=None):
    """Per bin {count, sum vx, sum vy, sum vz, sum |v|^2} (FP64, accumulated)."""
    if out is None and mode != 3:
        out = np.zeros((nbins, 5), np.float64)
    _check(h, load_library().dpd_velocity_profile(h, axis, nbins, lo, hi, _ptr(out), mode))
    return out


def dpd_init_particles(h, seed, solid_layer=1.0):
    """Random fluid at rho over the box, classified by the phase field (Sec. II.C)."""
    return _check(h, load_library().dpd_init_particles(h, int(seed), float(solid_layer)))


def dpd_relax_phase_field(phi, spacing, eps, iters, dtau, curvature=True):
    """Relax a phase field (float32 array (nz, ny, nx)) by Eq. 15 (curvature=True) or
    Eq. 13; returns (new array, mean ms per step)."""
    a = np.ascontiguousarray(phi, np.float32).copy()
    nz, ny, nx = a.shape
    dims = np.asarray([nx, ny, nz], np.int32)
    ms = np.zeros(1, np.float64)
    rc = load_library().dpd_relax_phase_field(_ptr(a), _ptr(dims), float(spacing), float(eps),
                                              int(iters), float(dtau), int(bool(curvature)),
                                              _ptr(ms))
    if rc != DPD_OK:
        raise DPDError(rc, dpd_last_error(None))
    return a, float(ms[0])


NOALLOC_MAX_BINS = 4096


def dpd_velocity_profile_noalloc(pos4, vel4, types, n, axis, nbins, lo, hi, out, where=DPD_HOST,
                                 stream=None):
    """Allocation-free profile sums of caller-owned device arrays (torch CUDA tensors
    or raw device pointers) into `out` (numpy array for DPD_HOST, CUDA tensor for
    DPD_DEVICE).  See include/dpd.h."""
    s = getattr(stream, "cuda_stream", stream)
    rc = load_library().dpd_velocity_profile_noalloc(
        _ptr(pos4) if hasattr(pos4, "data_ptr") else pos4,
        _ptr(vel4) if hasattr(vel4, "data_ptr") else vel4,
        _ptr(types) if hasattr(types, "data_ptr") else types, int(n), int(axis), int(nbins),
        float(lo), float(hi), _ptr(out), int(where), ctypes.c_void_p(s) if s else None)
    if rc != DPD_OK:
        raise DPDError(rc, dpd_last_error(None))
    return out


def dpd_get_stats(h) -> np.ndarray:
    out = np.zeros(8, np.float64)
    _check(h, load_library().dpd_get_stats(h, _ptr(out)))
    return out


def dpd_set_option(h, key: str, value: float):
    return _check(h, load_library().dpd_set_option(h, key.encode(), float(value)))


def dpd_get_option(h, key: str) -> float:
    v = ctypes.c_double()
    _check(h, load_library().dpd_get_option(h, key.encode(), ctypes.byref(v)))
    return v.value


def dpd_set_stream(h, stream):
    """stream: a torch.cuda.Stream, an integer cudaStream_t, or None (own stream)."""
    s = getattr(stream, "cuda_stream", stream)
    return _check(h, load_library().dpd_set_stream(h, ctypes.c_void_p(s) if s else None))


def dpd_destroy(h):
    if h:
        load_library().dpd_destroy(h)


class System:
    """Owns one handle; built from a workload description (box, phase field, particles)."""

    def __init__(self, box, a_ff=25.0, a_fs=25.0, gamma=4.5, sigma=3.0, kBT=1.0, dt=0.01,
                 g=(0.0, 0.0, 0.0), rho=3.0, **options):
        self.h = dpd_create(box, rho, (a_ff, a_fs, a_fs, 0.0), gamma, sigma, kBT, dt, g)
        for k, v in options.items():
            dpd_set_option(self.h, k, v)

    @classmethod
    def from_workload(cls, w, set_particles=True, **kw):
        s = cls(w.box, **kw)
        dpd_set_phase_field(s.h, w.phi, w.h)
        if set_particles:
            s.set_particles(w.pos4(), w.vel4(), w.id, w.type)
        return s

    def init_particles(self, seed, solid_layer=1.0):
        return dpd_init_particles(self.h, seed, solid_layer)

    def set_particles(self, pos4, vel4, ids, types, where=DPD_HOST):
        return dpd_set_particles(self.h, pos4, vel4, ids, types, where)

    def step(self, n=1):
        return dpd_step(self.h, n)

    def state(self):
        return dpd_get_state(self.h)

    def profile(self, axis, nbins, lo, hi, mode=0):
        return dpd_velocity_profile(self.h, axis, nbins, lo, hi, mode)

    def stats(self):
        return dpd_get_stats(self.h)

    def set_option(self, k, v):
        return dpd_set_option(self.h, k, v)

    def get_option(self, k):
        return dpd_get_option(self.h, k)

    def close(self):
        if self.h:
            dpd_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- batches -------------------------------------------------------------------

def dpd_batch_last_error(hb) -> str:
    return load_library().dpd_batch_last_error(hb).decode(errors="replace")


def _bcheck(hb, rc):
    if rc != DPD_OK:
        raise DPDError(rc, dpd_batch_last_error(hb))
    return rc


def dpd_batch_create(handles):
    """Batch of loaded systems (a list of dpd handles)."""
    L = load_library()
    arr = (ctypes.c_void_p * len(handles))(*[h.value if isinstance(h, ctypes.c_void_p) else h
                                             for h in handles])
    hb = ctypes.c_void_p()
    rc = L.dpd_batch_create(ctypes.byref(hb), len(handles), ctypes.cast(arr, ctypes.c_void_p))
    if rc != DPD_OK:
        raise DPDError(rc, L.dpd_batch_last_error(None).decode(errors="replace"))
    return hb


def dpd_batch_step(hb, nsteps: int):
    return _bcheck(hb, load_library().dpd_batch_step(hb, int(nsteps)))


def dpd_batch_time_phases(hb, nsteps: int) -> dict:
    ms = np.zeros(len(PHASES), np.float64)
    _bcheck(hb, load_library().dpd_batch_time_phases(hb, int(nsteps), _ptr(ms)))
    return dict(zip(PHASES, ms.tolist()))


def dpd_batch_autotune(hb, nsteps: int = 5):
    nv = int(dpd_batch_get_option(hb, "force_variants"))
    ms = np.zeros(nv, np.float64)
    chosen = ctypes.c_int()
    _bcheck(hb, load_library().dpd_batch_autotune(hb, int(nsteps), _ptr(ms), ctypes.byref(chosen)))
    return chosen.value, ms.tolist()


def dpd_batch_num_particles(hb, k: int):
    n, nf = ctypes.c_int(), ctypes.c_int()
    _bcheck(hb, load_library().dpd_batch_num_particles(hb, int(k), ctypes.byref(n), ctypes.byref(nf)))
    return n.value, nf.value


def dpd_batch_get_state(hb, k: int, pos4=None, vel4=None, force4=None, ids=None, types=None,
                        where=DPD_HOST):
    if where == DPD_HOST and all(x is None for x in (pos4, vel4, force4, ids, types)):
        n, _ = dpd_batch_num_particles(hb, k)
        pos4 = np.zeros((n, 4), np.float32)
        vel4 = np.zeros((n, 4), np.float32)
        force4 = np.zeros((n, 4), np.float32)
        ids = np.zeros(n, np.int32)
        types = np.zeros(n, np.uint8)
    _bcheck(hb, load_library().dpd_batch_get_state(hb, int(k), _ptr(pos4), _ptr(vel4), _ptr(force4),
                                                   _ptr(ids), _ptr(types), where))
    return pos4, vel4, force4, ids, types


def dpd_batch_get_stats(hb, k: int) -> np.ndarray:
    out = np.zeros(8, np.float64)
    _bcheck(hb, load_library().dpd_batch_get_stats(hb, int(k), _ptr(out)))
    return out


def dpd_batch_set_option(hb, key: str, value: float):
    return _bcheck(hb, load_library().dpd_batch_set_option(hb, key.encode(), float(value)))


def dpd_batch_get_option(hb, key: str) -> float:
    v = ctypes.c_double()
    _bcheck(hb, load_library().dpd_batch_get_option(hb, key.encode(), ctypes.byref(v)))
    return v.value


def dpd_batch_set_stream(hb, stream):
    s = getattr(stream, "cuda_stream", stream)
    return _bcheck(hb, load_library().dpd_batch_set_stream(hb, ctypes.c_void_p(s) if s else None))


def dpd_batch_destroy(hb):
    if hb:
        load_library().dpd_batch_destroy(hb)


class Batch:
    """Owns one batch handle built from loaded Systems (which must outlive it)."""

    def __init__(self, systems, **options):
        self.systems = list(systems)
        self.hb = dpd_batch_create([s.h for s in self.systems])
        for k, v in options.items():
            dpd_batch_set_option(self.hb, k, v)

    def step(self, n=1):
        return dpd_batch_step(self.hb, n)

    def state(self, k):
        return dpd_batch_get_state(self.hb, k)

    def stats(self, k):
        return dpd_batch_get_stats(self.hb, k)

    def close(self):
        if self.hb:
            dpd_batch_destroy(self.hb)
            self.hb = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
