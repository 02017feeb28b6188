"""Thin ctypes binding of libdg (include/dg.h): argument marshalling only.

Every step of the computation runs inside libdg (host setup in C++, the
right-hand side, LSRK stages and energy in CUDA kernels).  Importing this
module raises if libdg.so has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdg.so")
if not os.path.exists(LIB_PATH):
    raise ImportError(f"libdg.so not built ({LIB_PATH}); run paper_1507_02557_b300/build.py")
_lib = C.CDLL(LIB_PATH)

HEX, WEDGE, PYR, TET = 0, 1, 2, 3
EXPORTS = ("dg_mesh_create", "dg_mesh_destroy", "dg_host_check", "dg_layout", "dg_ndof", "dg_level_counts",
           "dg_set_state", "dg_get_state", "dg_rhs", "dg_timestep", "dg_step", "dg_state_ptr",
           "dg_energy", "dg_energy_noalloc", "dg_profile", "dg_watchdog_selftest", "dg_adjoint_step",
           "dg_batch_create", "dg_batch_step", "dg_batch_stats", "dg_batch_set_packing", "dg_batch_autotune",
           "dg_batch_destroy",
           "dg_set_source", "dg_set_receivers", "dg_sample_receivers", "dg_autotune",
           "dg_status_string", "dg_last_error")


class Desc(C.Structure):
    _fields_ = [("nverts", C.c_int64), ("xyz", C.POINTER(C.c_double)),
                ("nelem", C.c_int64 * 4), ("conn", C.POINTER(C.c_int32) * 4),
                ("c2", C.POINTER(C.c_double) * 4), ("N", C.c_int), ("hex_basis", C.c_int),
                ("pyr_form", C.c_int), ("tau_scale", C.c_double), ("nlevels", C.c_int),
                ("cfl", C.c_double), ("precision", C.c_int), ("integrator", C.c_int)]


_vp = C.c_void_p
_lib.dg_mesh_create.argtypes = [C.POINTER(Desc), _vp, C.POINTER(_vp)]
_lib.dg_mesh_destroy.argtypes = [_vp]
_lib.dg_mesh_destroy.restype = None
_lib.dg_host_check.argtypes = [C.POINTER(Desc), C.POINTER(C.c_double), C.POINTER(C.c_double), _vp]
_lib.dg_layout.argtypes = [_vp, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int)]
_lib.dg_ndof.argtypes = [_vp, C.POINTER(C.c_int64)]
_lib.dg_level_counts.argtypes = [_vp, C.c_int, C.POINTER(C.c_int64)]
_lib.dg_set_state.argtypes = [_vp, _vp, C.c_int]
_lib.dg_get_state.argtypes = [_vp, _vp, C.c_int]
_lib.dg_rhs.argtypes = [_vp, _vp, _vp, C.c_double]
_lib.dg_timestep.argtypes = [_vp, C.POINTER(C.c_double), _vp]
_lib.dg_step.argtypes = [_vp, C.c_int, C.c_double, C.POINTER(C.c_double)]
_lib.dg_state_ptr.argtypes = [_vp, C.POINTER(_vp)]
_lib.dg_energy.argtypes = [_vp, _vp, C.POINTER(C.c_double)]
_lib.dg_energy_noalloc.argtypes = [_vp, _vp, C.POINTER(C.c_double)]
_lib.dg_watchdog_selftest.argtypes = [_vp, C.c_int64]
_lib.dg_adjoint_step.argtypes = [_vp, C.c_int, C.c_double, C.c_double, _vp, _vp, _vp, _vp]
_lib.dg_autotune.argtypes = [_vp, C.c_int, C.POINTER(C.c_int)]
_lib.dg_set_source.argtypes = [_vp, C.POINTER(C.c_double), C.c_double, C.c_double, C.c_double]
_lib.dg_set_receivers.argtypes = [_vp, C.c_int, C.POINTER(C.c_double)]
_lib.dg_sample_receivers.argtypes = [_vp, _vp, _vp]
_lib.dg_profile.argtypes = [_vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int64)]
_lib.dg_batch_create.argtypes = [C.POINTER(_vp), C.c_int, _vp, C.POINTER(_vp)]
_lib.dg_batch_step.argtypes = [_vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
_lib.dg_batch_stats.argtypes = [_vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
_lib.dg_batch_set_packing.argtypes = [_vp, C.c_int]
_lib.dg_batch_autotune.argtypes = [_vp, C.c_int, C.POINTER(C.c_int)]
_lib.dg_batch_destroy.argtypes = [_vp]
_lib.dg_batch_destroy.restype = None
BATCH_CHUNK = 3   # DG_BATCH_CHUNK
_lib.dg_status_string.restype = C.c_char_p
_lib.dg_status_string.argtypes = [C.c_int]
_lib.dg_last_error.restype = C.c_char_p


class DGError(RuntimeError):
    pass


def _check(st):
    if st != 0:
        msg = _lib.dg_status_string(st).decode()
        detail = _lib.dg_last_error().decode()
        raise DGError(f"{msg} ({st}): {detail}")


def _ptr(x):
    """Raw pointer of a torch tensor or numpy array."""
    if hasattr(x, "data_ptr"):
        return _vp(x.data_ptr())
    return x.ctypes.data_as(_vp)


def _desc(mesh, N, tau_scale, pyr_form, cfl, keep, nlevels=1, hex_basis=0, precision=0, integrator=0):
    d = Desc()
    xyz = np.ascontiguousarray(mesh.xyz, dtype=np.float64)
    keep.append(xyz)
    d.nverts = xyz.shape[0]
    d.xyz = xyz.ctypes.data_as(C.POINTER(C.c_double))
    for t in range(4):
        cn = np.ascontiguousarray(mesh.conn[t], dtype=np.int32)
        c2 = np.ascontiguousarray(mesh.c2[t], dtype=np.float64)
        keep += [cn, c2]
        d.nelem[t] = cn.shape[0]
        d.conn[t] = cn.ctypes.data_as(C.POINTER(C.c_int32))
        d.c2[t] = c2.ctypes.data_as(C.POINTER(C.c_double))
    d.N, d.hex_basis, d.pyr_form = N, hex_basis, pyr_form
    d.tau_scale, d.nlevels, d.cfl, d.precision = tau_scale, nlevels, cfl, precision
    d.integrator = integrator
    return d


def host_check(mesh, N, tau_scale=1.0, pyr_form=0, cfl=0.5, nlevels=1, levels=False, hex_basis=0):
    """dg_host_check: (dt_min, [C_T hex, wedge, pyr, tet][, level counts]) from the host setup alone.
    hex_basis 1 = SEM hexahedra (GLL nodes, GLL points on every quadrilateral face)."""
    keep = []
    d = _desc(mesh, N, tau_scale, pyr_form, cfl, keep, nlevels, hex_basis)
    dt = C.c_double()
    ct = (C.c_double * 4)()
    lc = (C.c_int64 * 2)()
    _check(_lib.dg_host_check(C.byref(d), C.byref(dt), ct, C.cast(lc, _vp)))
    if levels:
        return dt.value, list(ct), list(lc)[:nlevels]
    return dt.value, list(ct)


class Mesh:
    """A dg_mesh on the current CUDA device (see include/dg.h)."""

    def __init__(self, mesh, N, tau_scale=1.0, pyr_form=0, cfl=0.5, stream=None, nlevels=1, hex_basis=0,
                 precision=0, integrator=0):
        """precision: 0 = FP32 products; 1 = BF16 x 3, 2 = FP16 x 3 split products on the tensor cores
        for the tet and pyramid volume terms.  integrator (nlevels = 2): 0 = multi-rate AB3,
        1 = multi-rate LSRK(5,4)."""
        keep = []
        d = _desc(mesh, N, tau_scale, pyr_form, cfl, keep, nlevels, hex_basis, precision, integrator)
        h = _vp()
        _check(_lib.dg_mesh_create(C.byref(d), _vp(stream or 0), C.byref(h)))
        self._h = h
        self.N = N
        self.nlevels = nlevels
        self.precision = precision
        n = C.c_int64()
        _check(_lib.dg_ndof(h, C.byref(n)))
        self.ndof = n.value

    def close(self):
        if getattr(self, "_h", None):
            _lib.dg_mesh_destroy(self._h)
            self._h = None

    __del__ = close

    def layout(self, t):
        o, k, npn = C.c_int64(), C.c_int64(), C.c_int()
        _check(_lib.dg_layout(self._h, t, C.byref(o), C.byref(k), C.byref(npn)))
        return o.value, k.value, npn.value

    def set_state(self, q, on_device):
        _check(_lib.dg_set_state(self._h, _ptr(q), int(on_device)))

    def get_state(self, out, on_device):
        _check(_lib.dg_get_state(self._h, _ptr(out), int(on_device)))
        return out

    def state_ptr(self):
        p = _vp()
        _check(_lib.dg_state_ptr(self._h, C.byref(p)))
        return p.value

    def rhs(self, q_dev, rhs_dev, t=0.0):
        _check(_lib.dg_rhs(self._h, _ptr(q_dev), _ptr(rhs_dev), float(t)))

    def timestep(self):
        dt = C.c_double()
        _check(_lib.dg_timestep(self._h, C.byref(dt), None))
        return dt.value

    def level_type_counts(self, level):
        """Elements per type (hex, wedge, pyramid, tet) in time-step level 1..nlevels."""
        c = (C.c_int64 * 4)()
        _check(_lib.dg_level_counts(self._h, int(level), c))
        return list(c)

    def mr_s_counts(self):
        """Multi-rate LSRK: elements per type of S (fine + coarse elements next to fine ones)."""
        c = (C.c_int64 * 4)()
        _check(_lib.dg_level_counts(self._h, 0, c))
        return list(c)

    def level_counts(self):
        """Element counts of the time-step levels (coarse first)."""
        dt = C.c_double()
        lc = (C.c_int64 * 2)()
        _check(_lib.dg_timestep(self._h, C.byref(dt), lc))
        return list(lc)[: self.nlevels]

    def step(self, nsteps, dt=0.0, t=0.0):
        tt = C.c_double(t)
        _check(_lib.dg_step(self._h, int(nsteps), float(dt), C.byref(tt)))
        return tt.value

    def energy_noalloc(self, q_dev=None):
        """dg_energy_noalloc: the energy with no device allocation (static scratch)."""
        E = C.c_double()
        _check(_lib.dg_energy_noalloc(self._h, _ptr(q_dev) if q_dev is not None else None, C.byref(E)))
        return E.value

    def adjoint_step(self, nsteps, lam_dev, grad_c2_dev=None, dt=0.0, t0=0.0, resid_dev=None, grad_amp_dev=None):
        """dg_adjoint_step: lam_dev (device [4][ndof] float32) from dL/dq_n to dL/dq_0 for nsteps
        LSRK steps from the current state at time t0; resid_dev (device [nsteps][nrec] float32)
        receiver forcing; grad_c2_dev (device float64, one per element) += dL/dc^2;
        grad_amp_dev (device float64 [1]) += dL/damp."""
        opt = lambda x: _ptr(x) if x is not None else None
        _check(_lib.dg_adjoint_step(self._h, int(nsteps), float(dt), float(t0), _ptr(lam_dev), opt(resid_dev),
                                    opt(grad_c2_dev), opt(grad_amp_dev)))

    CHOICES = ("hex_tma", "tet_tensor_cores", "type_streams")

    def autotune(self, nsteps=2):
        """dg_autotune: {"hex_tma", "tet_tensor_cores", "type_streams"} chosen for this mesh."""
        c = (C.c_int * 3)()
        _check(_lib.dg_autotune(self._h, int(nsteps), c))
        return dict(zip(self.CHOICES, (bool(v) for v in c)))

    def set_choices(self, hex_tma=True, tet_tensor_cores=True, type_streams=True):
        """dg_autotune with nsteps = 0: apply kernel choices; returns those in effect."""
        c = (C.c_int * 3)(int(hex_tma), int(tet_tensor_cores), int(type_streams))
        _check(_lib.dg_autotune(self._h, 0, c))
        return dict(zip(self.CHOICES, (bool(v) for v in c)))

    def set_source(self, x, amp, f0, t0):
        """dg_set_source: Ricker point source amp ricker(t; f0, t0) at x (inside a hexahedron)."""
        xs = (C.c_double * 3)(*[float(v) for v in x])
        _check(_lib.dg_set_source(self._h, xs, float(amp), float(f0), float(t0)))

    def set_receivers(self, xyz):
        """dg_set_receivers: receivers at the rows of xyz (n, 3)."""
        a = np.ascontiguousarray(np.asarray(xyz, dtype=np.float64).reshape(-1, 3))
        self.nrec = a.shape[0]
        _check(_lib.dg_set_receivers(self._h, a.shape[0], a.ctypes.data_as(C.POINTER(C.c_double))))

    def sample_receivers(self, out_dev, q_dev=None):
        """dg_sample_receivers: p at the receivers into out_dev (device float32 [nrec])."""
        _check(_lib.dg_sample_receivers(self._h, _ptr(q_dev) if q_dev is not None else None, _ptr(out_dev)))
        return out_dev

    def watchdog_selftest(self, limit_cycles):
        """dg_watchdog_selftest: the status (an int) a bounded device wait that runs out reports."""
        return int(_lib.dg_watchdog_selftest(self._h, int(limit_cycles)))

    def profile(self, enable):
        """Per-type kernel ms and launch counts since the last call; then (re)arm timing."""
        ms = (C.c_double * 4)()
        n = (C.c_int64 * 4)()
        _check(_lib.dg_profile(self._h, int(enable), ms, n))
        return list(ms), list(n)

    def energy(self, q_dev=None):
        E = C.c_double()
        _check(_lib.dg_energy(self._h, _ptr(q_dev) if q_dev is not None else None, C.byref(E)))
        return E.value


class Batch:
    """A dg_batch: several Mesh objects stepped through one captured CUDA graph (include/dg.h).
    The meshes must outlive the batch."""

    def __init__(self, meshes, stream=None):
        self.meshes = list(meshes)
        arr = (_vp * len(self.meshes))(*[g._h for g in self.meshes])
        h = _vp()
        _check(_lib.dg_batch_create(arr, len(self.meshes), _vp(stream or 0), C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib.dg_batch_destroy(self._h)
            self._h = None

    __del__ = close

    def step(self, nsteps, dt=None, t=None):
        """dg_batch_step; dt, t: per-mesh sequences (None = each mesh's dt_min / not reported).
        Returns the updated times."""
        n = len(self.meshes)
        dta = (C.c_double * n)(*(dt if dt is not None else [0.0] * n))
        ta = (C.c_double * n)(*(t if t is not None else [0.0] * n))
        _check(_lib.dg_batch_step(self._h, int(nsteps), dta, ta))
        return list(ta)

    def set_packing(self, packed):
        """dg_batch_set_packing: 1 = same-kind meshes through their combined meshes, 0 = mesh by mesh."""
        _check(_lib.dg_batch_set_packing(self._h, int(packed)))

    def autotune(self, nsteps=3):
        """dg_batch_autotune: keeps the faster of packed / unpacked stepping; returns 1 if packed."""
        p = C.c_int()
        _check(_lib.dg_batch_autotune(self._h, int(nsteps), C.byref(p)))
        return p.value

    def stats(self):
        """(graph replays, graph captures) since creation."""
        r, c = C.c_int64(), C.c_int64()
        _check(_lib.dg_batch_stats(self._h, C.byref(r), C.byref(c)))
        return r.value, c.value
