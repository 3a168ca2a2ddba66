"""Thin Python binding of ``include/colatus.h`` (ctypes over libcolatus.so).

Functions keep the C names and argument order; they only marshal arguments
(NumPy arrays or PyTorch tensors, host or CUDA) into pointers and turn a
non-OK status into ``ColatusError``.  Every step of the computation runs in the
library's CUDA kernels: there is no CPU fallback, and importing the library
fails loudly when ``libcolatus.so`` has not been built.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# COLATUS_LIBRARY may point at another build of the same library
LIB_PATH = os.environ.get("COLATUS_LIBRARY") or os.path.join(HERE, "libcolatus.so")

# enums of colatus.h
OK, E_ARG, E_CUDA, E_NONFINITE, E_FRIEDMANN, E_STATE, E_OOM, E_TIMEOUT = range(8)
FP32, FP32_COMP, FP64 = 0, 1, 2
DKD, KDK, KDK_CANONICAL = 0, 1, 2
F32, F64 = 0, 1
NDIAG = 16
STATUS_NAMES = {0: "COLATUS_OK", 1: "COLATUS_E_ARG", 2: "COLATUS_E_CUDA",
                3: "COLATUS_E_NONFINITE", 4: "COLATUS_E_FRIEDMANN", 5: "COLATUS_E_STATE",
                6: "COLATUS_E_OOM", 7: "COLATUS_E_TIMEOUT"}

# every symbol the header declares
EXPORTS = ("colatus_init", "colatus_set_config", "colatus_set_masses", "colatus_set_state",
           "colatus_get_state", "colatus_forces", "colatus_step", "colatus_synchronize",
           "colatus_record_tracers", "colatus_read_tracers", "colatus_diagnostics",
           "colatus_last_error", "colatus_stats", "colatus_profile_forces",
           "colatus_profile_read", "colatus_force_vjp", "colatus_adjoint_forward",
           "colatus_adjoint_backward", "colatus_forces_noalloc", "colatus_destroy",
           "colatus_ensemble_init", "colatus_ensemble_set_state", "colatus_ensemble_get_state",
           "colatus_ensemble_forces", "colatus_ensemble_step", "colatus_ensemble_synchronize",
           "colatus_ensemble_record_tracers", "colatus_ensemble_read_tracers",
           "colatus_ensemble_set_scheme",
           "colatus_ensemble_stats", "colatus_ensemble_last_error", "colatus_ensemble_destroy",
           "colatus_tangent_init", "colatus_tangent_step", "colatus_tangent_read",
           "colatus_autotune", "colatus_set_tuning", "colatus_probe_pipes",
           "colatus_set_deformation", "colatus_velocity_spectrum", "colatus_tracer_spectrum",
           "colatus_set_periodic", "colatus_periodic_params", "colatus_get_state_async",
           "colatus_wait_state", "colatus_selftest_wait", "colatus_profile_read_kinds",
           "colatus_ensemble_autotune", "colatus_ensemble_set_tuning", "colatus_force_plan",
           "colatus_vjp_plan", "colatus_selftest_sym_tables", "colatus_selftest_ens_sym_tables")


class ColatusError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None
_vp, _i64, _dbl, _int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int


def lib():
    """Load libcolatus.so (built by ``python -m paper_1208_3444_b300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: the CUDA library must be built "
                           "(python -m paper_1208_3444_b300.build); there is no fallback")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "colatus_init": [ctypes.POINTER(_vp), _i64, _vp, _dbl, _dbl, _dbl, _dbl, _dbl, _dbl, _dbl],
        "colatus_set_config": [_vp, _int, _int, _dbl, _vp],
        "colatus_set_masses": [_vp, _vp, _int, _int],
        "colatus_set_state": [_vp, _vp, _vp, _int, _int],
        "colatus_get_state": [_vp, _vp, _vp, _int, _int, _vp, _vp],
        "colatus_forces": [_vp, _vp, _int, _int],
        "colatus_step": [_vp, _dbl, _i64],
        "colatus_synchronize": [_vp],
        "colatus_record_tracers": [_vp, _vp, _int, _i64],
        "colatus_read_tracers": [_vp, _vp, _vp],
        "colatus_diagnostics": [_vp, _vp],
        "colatus_stats": [_vp, _vp],
        "colatus_profile_forces": [_vp, _int],
        "colatus_profile_read": [_vp, _vp],
        "colatus_profile_read_kinds": [_vp, _vp],
        "colatus_ensemble_autotune": [_vp, _int, _vp, _vp],
        "colatus_ensemble_set_tuning": [_vp, _int],
        "colatus_forces_noalloc": [_vp, _i64, _dbl, _dbl, _dbl, _vp, _vp],
        "colatus_force_plan": [_vp, _vp],
        "colatus_vjp_plan": [_vp, _vp],
        "colatus_force_vjp": [_vp, _vp, _vp, _vp, _int, _int],
        "colatus_adjoint_forward": [_vp, _dbl, _i64, _i64],
        "colatus_adjoint_backward": [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _int, _int],
        "colatus_ensemble_init": [ctypes.POINTER(_vp), _int, _vp, _vp, _vp, _dbl, _dbl, _dbl, _dbl,
                                  _dbl, _dbl, _dbl, _vp],
        "colatus_ensemble_set_state": [_vp, _vp, _vp, _int, _int],
        "colatus_ensemble_get_state": [_vp, _vp, _vp, _int, _int, _vp, _vp],
        "colatus_ensemble_forces": [_vp, _vp, _int, _int],
        "colatus_ensemble_step": [_vp, _dbl, _i64],
        "colatus_ensemble_synchronize": [_vp],
        "colatus_ensemble_record_tracers": [_vp, _vp, _int, _i64],
        "colatus_ensemble_set_scheme": [_vp, _int],
        "colatus_ensemble_read_tracers": [_vp, _vp, _vp],
        "colatus_ensemble_stats": [_vp, _int, _vp],
        "colatus_tangent_init": [_vp, _vp, _int, _vp, _i64],
        "colatus_autotune": [_vp, _int, _vp, _vp],
        "colatus_set_tuning": [_vp, _int],
        "colatus_probe_pipes": [_vp],
        "colatus_set_deformation": [_vp, _dbl, _vp],
        "colatus_velocity_spectrum": [_vp, _int, _int, _i64, _i64, _i64, _dbl, _int, _int, _vp,
                                      _int, _vp],
        "colatus_tracer_spectrum": [_vp, _dbl, _int, _int, _vp, _vp],
        "colatus_set_periodic": [_vp, _dbl, _dbl, _int],
        "colatus_get_state_async": [_vp, _vp, _vp, _int],
        "colatus_wait_state": [_vp],
        "colatus_selftest_wait": [_vp, _i64],
        "colatus_periodic_params": [_vp, _vp, _vp, _vp],
        "colatus_tangent_step": [_vp, _dbl, _i64],
        "colatus_tangent_read": [_vp, _vp, _vp],
        "colatus_selftest_sym_tables": [_i64, _int, _int, _int, _int, _int, _vp],
        "colatus_selftest_ens_sym_tables": [_int, _vp, _int, _int, _int, _vp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = _int
    L.colatus_last_error.argtypes = [_vp]
    L.colatus_last_error.restype = ctypes.c_char_p
    L.colatus_destroy.argtypes = [_vp]
    L.colatus_destroy.restype = None
    L.colatus_ensemble_last_error.argtypes = [_vp]
    L.colatus_ensemble_last_error.restype = ctypes.c_char_p
    L.colatus_ensemble_destroy.argtypes = [_vp]
    L.colatus_ensemble_destroy.restype = None
    _lib = L
    return L


def _check(status, handle=None):
    if status != OK:
        msg = lib().colatus_last_error(handle)
        raise ColatusError(status, msg.decode() if msg else "")


def _buf(a, ncols=None):
    """(pointer, on_device, dtype, keep-alive) for a NumPy array or tensor."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype not in (torch.float32, torch.float64):
                raise TypeError("tensors must be float32 or float64")
            if not a.is_contiguous():
                raise ValueError("tensor must be contiguous")
            return a.data_ptr(), int(a.is_cuda), F64 if a.dtype == torch.float64 else F32, a
    except ImportError:
        pass
    arr = np.asarray(a)
    if arr.dtype not in (np.float32, np.float64):
        arr = arr.astype(np.float64)
    arr = np.ascontiguousarray(arr)
    return arr.ctypes.data, 0, F64 if arr.dtype == np.float64 else F32, arr


# ------------------------------------------------------------- C entry points
def colatus_init(N, masses, eps, Omega_R, Omega_M, Omega_K, Omega_L, H0, a_start):
    m = np.ascontiguousarray(np.asarray(masses, dtype=np.float64).reshape(-1))
    if m.size != N:
        raise ValueError("masses must have N entries")
    h = _vp()
    st = lib().colatus_init(ctypes.byref(h), int(N), m.ctypes.data, float(eps), float(Omega_R),
                            float(Omega_M), float(Omega_K), float(Omega_L), float(H0),
                            float(a_start))
    _check(st, None)
    return h


def colatus_set_config(h, prec, scheme, G=1.0, stream=None):
    _check(lib().colatus_set_config(h, int(prec), int(scheme), float(G),
                                    None if stream is None else int(stream)), h)


def colatus_set_masses(h, m):
    p, dev, dt, keep = _buf(m)
    _check(lib().colatus_set_masses(h, p, dt, dev), h)


def colatus_set_state(h, x, v=None):
    px, dev, dt, kx = _buf(x)
    if v is not None:
        pv, dev2, dt2, kv = _buf(v)
        if dev2 != dev or dt2 != dt:
            raise ValueError("x and v must share device and dtype")
    else:
        pv = None
    _check(lib().colatus_set_state(h, px, pv, dt, dev), h)


def colatus_get_state(h, x=None, v=None):
    """Fill x and/or v (N x 3 arrays or tensors, same device and dtype) and
    return (t, a)."""
    t, a = _dbl(), _dbl()
    px = pv = None
    dev, dt = 0, F64
    keep = []
    if x is not None:
        px, dev, dt, k = _buf(x)
        keep.append(k)
    if v is not None:
        pv, dev2, dt2, k = _buf(v)
        if x is not None and (dev2 != dev or dt2 != dt):
            raise ValueError("x and v must share device and dtype")
        dev, dt = dev2, dt2
        keep.append(k)
    _check(lib().colatus_get_state(h, px, pv, dt, dev, ctypes.byref(t), ctypes.byref(a)), h)
    return t.value, a.value


def colatus_forces(h, out):
    p, dev, dt, keep = _buf(out)
    _check(lib().colatus_forces(h, p, dt, dev), h)
    return out


def colatus_step(h, dt, nsteps):
    _check(lib().colatus_step(h, float(dt), int(nsteps)), h)


def colatus_synchronize(h):
    _check(lib().colatus_synchronize(h), h)


def colatus_record_tracers(h, idx, capacity_steps):
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64).reshape(-1))
    _check(lib().colatus_record_tracers(h, idx.ctypes.data if idx.size else None, int(idx.size),
                                        int(capacity_steps)), h)


def colatus_read_tracers(h, ntr):
    n = ctypes.c_int64()
    _check(lib().colatus_read_tracers(h, None, ctypes.byref(n)), h)
    out = np.empty((n.value, ntr, 6), dtype=np.float32)
    if n.value:
        _check(lib().colatus_read_tracers(h, out.ctypes.data, ctypes.byref(n)), h)
    return out


def colatus_diagnostics(h):
    out = np.zeros(NDIAG)
    _check(lib().colatus_diagnostics(h, out.ctypes.data), h)
    return out


def colatus_stats(h):
    out = np.zeros(4)
    _check(lib().colatus_stats(h, out.ctypes.data), h)
    return out


def colatus_profile_forces(h, on):
    _check(lib().colatus_profile_forces(h, int(on)), h)


def colatus_profile_read(h, vjp=False):
    """(milliseconds, launches) of the force kernel (or of the VJP kernel with
    vjp=True) since the last read; a read resets both totals."""
    out = np.zeros(4)
    _check(lib().colatus_profile_read(h, out.ctypes.data), h)
    k = 2 if vjp else 0
    return float(out[k]), int(out[k + 1])


def colatus_profile_read_all(h):
    """{'force': (ms, launches), 'vjp': (ms, launches), 'adjoint_update': (ms,
    launches)} since the last read."""
    out = np.zeros(6)
    _check(lib().colatus_profile_read_kinds(h, out.ctypes.data), h)
    return {"force": (float(out[0]), int(out[1])), "vjp": (float(out[2]), int(out[3])),
            "adjoint_update": (float(out[4]), int(out[5]))}


def _same(*arrs):
    bufs = [_buf(a) for a in arrs if a is not None]
    if not bufs:
        return 0, F64, []
    devs = {b[1] for b in bufs}
    dts = {b[2] for b in bufs}
    if len(devs) != 1 or len(dts) != 1:
        raise ValueError("arrays must share device and dtype")
    return bufs[0][1], bufs[0][2], bufs


def _ptr_or_none(a, bufs, k):
    return None if a is None else bufs[k][0]


def colatus_force_vjp(h, w, gx=None, gm=None):
    dev, dt, bufs = _same(w, gx, gm)
    ptrs = iter(b[0] for b in bufs)
    pw = next(ptrs)
    pgx = next(ptrs) if gx is not None else None
    pgm = next(ptrs) if gm is not None else None
    _check(lib().colatus_force_vjp(h, pw, pgx, pgm, dt, dev), h)


def colatus_adjoint_forward(h, dt, nsteps, checkpoint_every):
    _check(lib().colatus_adjoint_forward(h, float(dt), int(nsteps), int(checkpoint_every)), h)


def colatus_adjoint_backward(h, gx_T=None, gv_T=None, gm_T=None, gx_0=None, gv_0=None, gm=None):
    arrs = (gx_T, gv_T, gm_T, gx_0, gv_0, gm)
    dev, dt, bufs = _same(*arrs)
    it = iter(b[0] for b in bufs)
    ptrs = [None if a is None else next(it) for a in arrs]
    _check(lib().colatus_adjoint_backward(h, *ptrs, dt, dev), h)


def colatus_forces_noalloc(pos, eps, G, a, acc_out, stream=None):
    """Allocation-free force (see colatus.h): pos is a CUDA float32 tensor of
    N x 4 (x, y, z, m), acc_out a CUDA float32 tensor of N x 3."""
    import torch
    for t, cols in ((pos, 4), (acc_out, 3)):
        p, dev, dt, keep = _buf(t)
        if not dev or dt != F32 or tuple(t.shape[1:]) != (cols,):
            raise ValueError(f"expected a contiguous CUDA float32 tensor of N x {cols}")
    if pos.device != acc_out.device:
        raise ValueError("pos and acc_out must be on the same GPU")
    if acc_out.shape[0] != pos.shape[0]:
        raise ValueError("pos and acc_out must have the same number of rows")
    # the C call runs on the current device; make it the tensors' device
    with torch.cuda.device(pos.device):
        st = lib().colatus_forces_noalloc(pos.data_ptr(), int(pos.shape[0]), float(eps), float(G),
                                          float(a), acc_out.data_ptr(),
                                          None if stream is None else int(stream))
    if st != OK:
        raise ColatusError(st, "colatus_forces_noalloc")


def colatus_probe_pipes():
    """Measured lane-ops per SM per clock: {'ffma', 'ffma2', 'mufu_rsq', 'sms'}."""
    out = np.zeros(6)
    _check(lib().colatus_probe_pipes(out.ctypes.data), None)
    return {"ffma": float(out[0]), "ffma2": float(out[1]), "mufu_rsq": float(out[2]),
            "sms": int(out[3])}


WINDOWS = {"rect": 0, "hann": 1}


def colatus_velocity_spectrum(v, dt, window="rect", detrend=True, out=None, stream=None,
                              offset=0):
    """Energy spectrum of a [T, ntr, stride] velocity series, host or CUDA,
    whose components sit at [offset, offset + 3) of each stride (a tracer
    record [T, ntr, 6] has offset 3); returns E [ntr, T//2 + 1] float64
    (``out`` if given, which may be a CUDA float64 tensor)."""
    ptr, on_dev, dtype, keep = _buf(v)
    shape = tuple(v.shape)
    if len(shape) != 3 or offset < 0 or shape[2] < offset + 3:
        raise ValueError("v must be [T, ntr, stride >= offset + 3]")
    T, ntr, stride = shape
    ptr += offset * (8 if dtype == F64 else 4)
    nf = T // 2 + 1
    if out is None:
        out = np.empty((ntr, nf), dtype=np.float64)
    optr, out_dev, odt, okeep = _buf(out)
    if odt != F64 or tuple(out.shape) != (ntr, nf):
        raise ValueError("out must be float64 [ntr, T//2 + 1]")
    sp = 0 if stream is None else int(getattr(stream, "cuda_stream", stream))
    _check(lib().colatus_velocity_spectrum(ptr, dtype, on_dev, T, ntr, stride, float(dt),
                                           WINDOWS[window], int(bool(detrend)), optr, out_dev,
                                           sp or None), None)
    return out


def colatus_tracer_spectrum(h, ntr, dt, window="rect", detrend=True):
    n = ctypes.c_int64()
    _check(lib().colatus_tracer_spectrum(h, float(dt), WINDOWS[window], int(bool(detrend)), None,
                                         ctypes.byref(n)), h)
    out = np.empty((ntr, n.value // 2 + 1), dtype=np.float64)
    _check(lib().colatus_tracer_spectrum(h, float(dt), WINDOWS[window], int(bool(detrend)),
                                         out.ctypes.data, ctypes.byref(n)), h)
    return out


def colatus_get_state_async(h, x, v):
    """Start a read-back of the state into host arrays/tensors x, v (N x 3,
    float32 or float64, the same dtype; pinned tensors let it overlap later
    steps).  They must stay alive until colatus_wait_state."""
    px, dx, tx, kx = _buf(x) if x is not None else (None, 0, None, None)
    pv, dv, tv, kv = _buf(v) if v is not None else (None, 0, None, None)
    if dx or dv:
        raise ValueError("colatus_get_state_async writes host memory")
    # the copy lands after this call returns: the caller's own buffers only,
    # never a converted temporary
    if (x is not None and kx is not x) or (v is not None and kv is not v):
        raise ValueError("x and v must be C-contiguous float32/float64 arrays or tensors")
    if x is not None and v is not None and tx != tv:
        raise ValueError("x and v must have the same dtype")
    _check(lib().colatus_get_state_async(h, px, pv, tx if x is not None else tv), h)


def colatus_wait_state(h):
    _check(lib().colatus_wait_state(h), h)


def colatus_selftest_wait(h, limit_cycles):
    """Run the bounded-wait self-test; raises ColatusError (COLATUS_E_TIMEOUT)
    when the failure path works."""
    _check(lib().colatus_selftest_wait(h, int(limit_cycles)), h)


def colatus_selftest_sym_tables(n_pad, T, NW, G, cost_diag, cost_sym):
    """Host-only replay of the pair-once kernels' walk over their tables;
    returns {tiles, tile_pairs, ctas, row_segments, column_slots} or raises
    ColatusError (COLATUS_E_STATE names the first failure)."""
    out = np.zeros(5, dtype=np.int64)
    _check(lib().colatus_selftest_sym_tables(int(n_pad), int(T), int(NW), int(G), int(cost_diag),
                                             int(cost_sym), out.ctypes.data), None)
    return dict(zip(("tiles", "tile_pairs", "ctas", "row_segments", "column_slots"), map(int, out)))


def colatus_selftest_ens_sym_tables(n_bodies, G, cost_diag, cost_sym):
    """The same for the ensemble's tables of realisations of n_bodies[r] bodies."""
    nb = np.ascontiguousarray(n_bodies, dtype=np.int64)
    out = np.zeros(5, dtype=np.int64)
    _check(lib().colatus_selftest_ens_sym_tables(len(nb), nb.ctypes.data, int(G), int(cost_diag),
                                                 int(cost_sym), out.ctypes.data), None)
    return dict(zip(("tiles", "tile_pairs", "ctas", "row_segments", "column_slots"), map(int, out)))


def colatus_last_error(h=None):
    s = lib().colatus_last_error(h)
    return s.decode() if s else ""


def colatus_destroy(h):
    if h:
        lib().colatus_destroy(h)


# ------------------------------------------------------------ convenience
DIAG_NAMES = ("K", "W", "Px", "Py", "Pz", "Lx", "Ly", "Lz", "Cx", "Cy", "Cz", "a", "t", "H",
              "Wx", "step")


class Simulation:
    """Owns one colatus context; methods map one-to-one onto the C calls."""

    def __init__(self, masses, eps, cosmo, a_start, prec=FP32, scheme=KDK, G=1.0, stream=None):
        m = np.asarray(masses, dtype=np.float64).reshape(-1)
        self.N = m.size
        c = dict(cosmo)
        self.h = colatus_init(self.N, m, eps, c["Omega_R"], c["Omega_M"], c["Omega_K"],
                              c["Omega_L"], c["H0"], a_start)
        self.prec, self.scheme, self.G = prec, scheme, G
        colatus_set_config(self.h, prec, scheme, G, stream)

    def configure(self, prec=None, scheme=None, G=None, stream=None):
        self.prec = self.prec if prec is None else prec
        self.scheme = self.scheme if scheme is None else scheme
        self.G = self.G if G is None else G
        colatus_set_config(self.h, self.prec, self.scheme, self.G, stream)

    def set_state(self, x, v=None):
        colatus_set_state(self.h, x, v)

    def set_masses(self, m):
        colatus_set_masses(self.h, m)

    def set_periodic(self, L, alpha=0.0, nk=0):
        """Periodic boundaries in a cube of side L (0: isolated); alpha, nk <= 0
        choose the Ewald parameters from the precision."""
        _check(lib().colatus_set_periodic(self.h, float(L), float(alpha), int(nk)), self.h)

    def periodic_params(self):
        a, nk, nkv = ctypes.c_double(), ctypes.c_int(), ctypes.c_int()
        _check(lib().colatus_periodic_params(self.h, ctypes.byref(a), ctypes.byref(nk),
                                             ctypes.byref(nkv)), self.h)
        return dict(alpha=a.value, nk=nk.value, nkv=nkv.value)

    def set_deformation(self, Cpsi, x_psi=(0.0, 0.0, 0.0)):
        xp = np.ascontiguousarray(np.asarray(x_psi, dtype=np.float64))
        _check(lib().colatus_set_deformation(self.h, float(Cpsi), xp.ctypes.data), self.h)

    def state(self, dtype=np.float64):
        x = np.empty((self.N, 3), dtype=dtype)
        v = np.empty((self.N, 3), dtype=dtype)
        t, a = colatus_get_state(self.h, x, v)
        return x, v, t, a

    def forces(self, out=None):
        if out is None:
            out = np.empty((self.N, 3), dtype=np.float64)
        return colatus_forces(self.h, out)

    def step(self, dt, nsteps=1):
        colatus_step(self.h, dt, nsteps)

    def synchronize(self):
        colatus_synchronize(self.h)

    def record_tracers(self, idx, capacity_steps):
        self.ntr = len(idx)
        colatus_record_tracers(self.h, idx, capacity_steps)

    def read_tracers(self):
        return colatus_read_tracers(self.h, getattr(self, "ntr", 0))

    def tracer_spectrum(self, dt, window="rect", detrend=True):
        """Energy spectrum [ntr, nrec//2 + 1] of the recorded tracer velocities."""
        return colatus_tracer_spectrum(self.h, getattr(self, "ntr", 0), dt, window, detrend)

    def diagnostics(self):
        return dict(zip(DIAG_NAMES, colatus_diagnostics(self.h)))

    def stats(self):
        s = colatus_stats(self.h)
        return dict(launches=int(s[0]), interactions=float(s[1]), steps=int(s[2]), N=int(s[3]))

    def force_plan(self):
        """The force kernel launched for the current configuration (colatus_force_plan)."""
        out = np.zeros(9, dtype=np.int64)
        _check(lib().colatus_force_plan(self.h, out.ctypes.data), self.h)
        kinds = ("force_f32", "force_f64", "ewald_f32", "ewald_f64", "force_sym_f32", "ewald_sym_f32")
        return dict(kind=kinds[int(out[0])], threads=int(out[1]), ipt=int(out[2]), jt=int(out[3]),
                    comp=bool(out[4]), eqm=bool(out[5]), grid=int(out[6]), units=int(out[7]),
                    nrcp=int(out[8]))

    def vjp_plan(self):
        """The VJP kernel the adjoint's backward pass launches (colatus_vjp_plan)."""
        out = np.zeros(6, dtype=np.int64)
        _check(lib().colatus_vjp_plan(self.h, out.ctypes.data), self.h)
        kinds = ("vjp_f32", "vjp_f64", "ewald_vjp_f32", "ewald_vjp_f64", "vjp_eqm_f32", "vjp_sym_eqm_f32",
                 "vjp_sym_f32", "ewald_vjp_sym_f32")
        return dict(kind=kinds[int(out[0])], threads=int(out[1]), ipt=int(out[2]), jt=int(out[3]),
                    grid=int(out[4]), units=int(out[5]))

    def profile_forces(self, on=True):
        colatus_profile_forces(self.h, on)

    def profile_read(self, vjp=False):
        return colatus_profile_read(self.h, vjp)

    def profile_read_all(self):
        return colatus_profile_read_all(self.h)

    def force_vjp(self, w, dtype=np.float64):
        gx = np.empty((self.N, 3), dtype=dtype)
        gm = np.empty(self.N, dtype=dtype)
        colatus_force_vjp(self.h, np.asarray(w, dtype=dtype), gx, gm)
        return gx, gm

    def adjoint_forward(self, dt, nsteps, checkpoint_every):
        colatus_adjoint_forward(self.h, dt, nsteps, checkpoint_every)

    def adjoint_backward(self, gx_T=None, gv_T=None, gm_T=None, dtype=np.float64):
        gx = np.empty((self.N, 3), dtype=dtype)
        gv = np.empty((self.N, 3), dtype=dtype)
        gm = np.empty(self.N, dtype=dtype)
        cast = (lambda a: None if a is None else np.ascontiguousarray(a, dtype=dtype))
        colatus_adjoint_backward(self.h, cast(gx_T), cast(gv_T), cast(gm_T), gx, gv, gm)
        return gx, gv, gm

    def autotune(self, reps=3):
        """Time the FP32 force shapes on the current state; keep the fastest.
        Returns (chosen shape, [ms per launch of shapes 0, 1, 2, 3])."""
        ms = np.zeros(4)
        ch = ctypes.c_int()
        _check(lib().colatus_autotune(self.h, int(reps), ms.ctypes.data, ctypes.byref(ch)), self.h)
        return int(ch.value), ms.tolist()

    def set_tuning(self, shape):
        _check(lib().colatus_set_tuning(self.h, int(shape)), self.h)

    def tangent_init(self, seeds, capacity_steps, direction=(1.0, 0.0, 0.0)):
        sd = np.ascontiguousarray(np.asarray(seeds, dtype=np.int64).reshape(-1))
        d = np.ascontiguousarray(np.asarray(direction, dtype=np.float64))
        self.ntan = sd.size
        _check(lib().colatus_tangent_init(self.h, sd.ctypes.data, int(sd.size), d.ctypes.data,
                                          int(capacity_steps)), self.h)

    def tangent_step(self, dt, nsteps=1):
        _check(lib().colatus_tangent_step(self.h, float(dt), int(nsteps)), self.h)

    def tangent_growth(self):
        """[nrec, B] norms |(dx, dv)| of each tangent's seed body after each step."""
        n = ctypes.c_int64()
        _check(lib().colatus_tangent_read(self.h, None, ctypes.byref(n)), self.h)
        out = np.empty((n.value, self.ntan), dtype=np.float32)
        if n.value:
            _check(lib().colatus_tangent_read(self.h, out.ctypes.data, ctypes.byref(n)), self.h)
        return out

    def close(self):
        if self.h:
            colatus_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ ensembles
def _echeck(status, handle):
    if status != OK:
        msg = lib().colatus_ensemble_last_error(handle)
        raise ColatusError(status, msg.decode() if msg else "")


class Ensemble:
    """R independent realisations stepped together (colatus_ensemble_*).
    Arrays are dense concatenations of the realisations (N_tot rows)."""

    def __init__(self, Ns, masses, eps_r, cosmo, a_start, G=1.0, stream=None, scheme=KDK):
        Ns = np.ascontiguousarray(np.asarray(Ns, dtype=np.int64))
        m = np.ascontiguousarray(np.asarray(masses, dtype=np.float64).reshape(-1))
        e = np.ascontiguousarray(np.asarray(eps_r, dtype=np.float64).reshape(-1))
        if m.size != Ns.sum() or e.size != Ns.size:
            raise ValueError("masses must have sum(Ns) entries and eps_r len(Ns)")
        self.Ns, self.Ntot = Ns, int(Ns.sum())
        c = dict(cosmo)
        h = _vp()
        st = lib().colatus_ensemble_init(ctypes.byref(h), int(Ns.size), Ns.ctypes.data, m.ctypes.data,
                                         e.ctypes.data, c["Omega_R"], c["Omega_M"], c["Omega_K"],
                                         c["Omega_L"], c["H0"], float(a_start), float(G),
                                         None if stream is None else int(stream))
        _echeck(st, None)
        self.h = h
        if scheme != KDK:
            self.set_scheme(scheme)

    def set_state(self, x, v=None):
        dev, dt, bufs = _same(x, v)
        _echeck(lib().colatus_ensemble_set_state(self.h, bufs[0][0],
                                                 bufs[1][0] if v is not None else None, dt, dev), self.h)

    def state(self, dtype=np.float64):
        x = np.empty((self.Ntot, 3), dtype=dtype)
        v = np.empty((self.Ntot, 3), dtype=dtype)
        t, a = _dbl(), _dbl()
        dt = F64 if dtype == np.float64 else F32
        _echeck(lib().colatus_ensemble_get_state(self.h, x.ctypes.data, v.ctypes.data, dt, 0,
                                                 ctypes.byref(t), ctypes.byref(a)), self.h)
        return x, v, t.value, a.value

    def forces(self, out=None):
        if out is None:
            out = np.empty((self.Ntot, 3), dtype=np.float64)
        p, dev, dt, keep = _buf(out)
        _echeck(lib().colatus_ensemble_forces(self.h, p, dt, dev), self.h)
        return out

    def step(self, dt, nsteps=1):
        _echeck(lib().colatus_ensemble_step(self.h, float(dt), int(nsteps)), self.h)

    def synchronize(self):
        _echeck(lib().colatus_ensemble_synchronize(self.h), self.h)

    def set_scheme(self, scheme):
        """DKD, KDK or KDK_CANONICAL for the following steps."""
        _echeck(lib().colatus_ensemble_set_scheme(self.h, int(scheme)), self.h)

    def record_tracers(self, idx, capacity_steps):
        """Record (x, v) of bodies idx (dense row indices) after every step."""
        idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64).reshape(-1))
        _echeck(lib().colatus_ensemble_record_tracers(self.h, idx.ctypes.data if idx.size else None,
                                                      int(idx.size), int(capacity_steps)), self.h)
        self.ntr = int(idx.size)

    def read_tracers(self):
        """Recorded tracers, oldest first: [nrec, ntr, 6] (x, y, z, vx, vy, vz)."""
        n = ctypes.c_int64()
        _echeck(lib().colatus_ensemble_read_tracers(self.h, None, ctypes.byref(n)), self.h)
        out = np.empty((n.value, getattr(self, "ntr", 0), 6), dtype=np.float32)
        if n.value and out.size:
            _echeck(lib().colatus_ensemble_read_tracers(self.h, out.ctypes.data, ctypes.byref(n)), self.h)
        return out

    def autotune(self, reps=3):
        """Time the force kernel's CTA shapes at the current state and keep
        the fastest: (milliseconds per evaluation of each shape, chosen)."""
        ms = np.zeros(4)
        ch = ctypes.c_int(-1)
        _echeck(lib().colatus_ensemble_autotune(self.h, int(reps), ms.ctypes.data, ctypes.byref(ch)),
                self.h)
        return ms, ch.value

    def set_tuning(self, shape):
        _echeck(lib().colatus_ensemble_set_tuning(self.h, int(shape)), self.h)

    def stats(self, profile_on=False):
        out = np.zeros(6)
        _echeck(lib().colatus_ensemble_stats(self.h, int(profile_on), out.ctypes.data), self.h)
        return dict(launches=int(out[0]), interactions=float(out[1]), steps=int(out[2]),
                    pairs_per_step=float(out[3]), force_ms=float(out[4]), force_launches=int(out[5]))

    def close(self):
        if self.h:
            lib().colatus_ensemble_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
