"""Thin ctypes binding of liblbem.so (include/lbem.h).

Each lbem_* function here has the name of the C entry point it calls and only
marshals arguments: torch tensors (CUDA or CPU) and numpy arrays are passed as
raw pointers, status codes become LbemError.  All computation happens in the
CUDA library; there is no fallback: if liblbem.so is missing or cannot be
loaded, load() raises.
"""
import ctypes as C
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbem.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "lbem.h")

F32, F16, BF16, I16B = 0, 1, 2, 3
STORAGE = {"f32": F32, "f16": F16, "bf16": BF16, "i16b": I16B}
STATUS = {0: "LBEM_OK", 1: "LBEM_ERR_ARG", 2: "LBEM_ERR_CUDA", 3: "LBEM_ERR_MEDIUM", 4: "LBEM_ERR_UNSTABLE",
          5: "LBEM_ERR_TIMEOUT", 6: "LBEM_ERR_STATE", 7: "LBEM_ERR_NOMEM"}


class LbemError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Desc(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("storage", C.c_int),
                ("c_ref2", C.c_double), ("stream", C.c_void_p)]


_lib = None
_VP, _I, _LL, _D = C.c_void_p, C.c_int, C.c_longlong, C.c_double
_SIGS = {
    "lbem_create": [C.POINTER(Desc), C.POINTER(_VP)],
    "lbem_destroy": [_VP],
    "lbem_set_stream": [_VP, _VP],
    "lbem_sync": [_VP],
    "lbem_last_error": [],
    "lbem_set_wait_limit": [_D],
    "lbem_info": [_VP, C.POINTER(_LL), C.POINTER(C.c_size_t)],
    "lbem_set_medium": [_VP, _VP, _VP],
    "lbem_set_fields": [_VP, _VP, _VP],
    "lbem_set_sources": [_VP, _I, _VP, _VP, _VP, _I],
    "lbem_set_receivers": [_VP, _I, _VP, _VP, _I],
    "lbem_step": [_VP, _I],
    "lbem_set_graphs": [_VP, _I],
    "lbem_set_temporal_blocking": [_VP, _I, _I],
    "lbem_get_temporal_blocking": [_VP, C.POINTER(_I), C.POINTER(_I), C.POINTER(_I)],
    "lbem_set_watchdog": [_VP, _I, _D],
    "lbem_set_boundaries": [_VP, C.POINTER(_I), _I, _D],
    "lbem_set_dispersion": [_VP, _VP, _VP, _VP],
    "lbem_set_medium_aniso": [_VP, _VP, _D, _D],
    "lbem_rows": [_VP, _I, _I, _I, _VP, _I],
    "lbem_get_boundaries": [_VP, C.POINTER(_I), C.POINTER(_I), C.POINTER(_D)],
    "lbem_time": [_VP, C.POINTER(_LL)],
    "lbem_fields": [_VP, _VP, _VP],
    "lbem_traces": [_VP, _VP, C.POINTER(_I)],
    "lbem_energy_flux": [_VP, _VP, _VP],
    "lbem_diagnostics": [_VP, C.POINTER(_D)],
    "lbem_diagnostics_static": [_I, _I, _I, _I, _VP, _VP, _VP, _D, _VP, _VP],
    "lbem_halo_out": [_VP, _I, _VP, _VP],
    "lbem_halo_in": [_VP, _I, _VP, _VP],
    "lbem_save_state": [_VP, _VP],
    "lbem_check_guards": [_VP],
    "lbem_load_state": [_VP, _VP, _LL],
    "lbem_forward_record": [_VP, _I, _I],
    "lbem_adjoint": [_VP, _VP, _VP, _VP],
    "lbem_autotune": [_VP, _I, C.POINTER(_I)],
    "lbem_set_variant": [_VP, _I],
    "lbem_get_variant": [_VP, C.POINTER(_I), C.POINTER(_I)],
    "lbem_batch_create": [_I, C.POINTER(_VP), _VP, C.POINTER(_VP)],
    "lbem_batch_step": [_VP, _I],
    "lbem_batch_autotune": [_VP, _I, C.POINTER(_I)],
    "lbem_batch_destroy": [_VP],
    "lbem_batch_set_variant": [_VP, _I],
    "lbem_batch_get_variant": [_VP, C.POINTER(_I), C.POINTER(_I)],
}


def header_symbols():
    """Names of the functions include/lbem.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbem_[a-z0-9_]+)\s*\(", text)))


def load(path=None):
    """Load liblbem.so (raises OSError if it is missing: build it with __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise OSError(f"{path} not found: the CUDA library is not built (run __graft_entry__.build())")
    lib = C.CDLL(path)
    for name, args in _SIGS.items():
        f = getattr(lib, name)
        f.argtypes = args
        if name == "lbem_last_error":
            f.restype = C.c_char_p
        elif name in ("lbem_destroy", "lbem_batch_destroy"):
            f.restype = None
        else:
            f.restype = C.c_int
    _lib = lib
    return lib


def _check(status, what=""):
    if status != 0:
        msg = load().lbem_last_error().decode()
        raise LbemError(status, msg or what)


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a, dtype=np.float32, count=None, writable=False):
    """Raw pointer of a contiguous torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if _is_torch(a):
        import torch

        tdt = {np.float32: torch.float32, np.float64: torch.float64, np.int64: torch.int64, np.int32: torch.int32,
               np.uint8: torch.uint8}[dtype]
        if a.dtype != tdt or not a.is_contiguous():
            raise TypeError(f"expected a contiguous {tdt} tensor")
        if count is not None and a.numel() < count:
            raise ValueError(f"tensor has {a.numel()} elements, need {count}")
        return a.data_ptr()
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags.c_contiguous:
        raise TypeError(f"expected a C-contiguous numpy array of {np.dtype(dtype)}")
    if writable and not a.flags.writeable:
        raise ValueError("output array is read-only")
    if count is not None and a.size < count:
        raise ValueError(f"array has {a.size} elements, need {count}")
    return a.ctypes.data


# --------------------------------------------------------------------------- C entry points


def lbem_create(dim, nx, ny, nz=1, storage=F32, c_ref2=0.0, stream=None):
    d = Desc(dim, nx, ny, nz, storage, c_ref2, stream)
    h = _VP()
    _check(load().lbem_create(C.byref(d), C.byref(h)), "lbem_create")
    return h


def lbem_destroy(h):
    load().lbem_destroy(h)


def lbem_last_error():
    return load().lbem_last_error().decode()


def lbem_set_wait_limit(seconds):
    _check(load().lbem_set_wait_limit(float(seconds)))


def lbem_set_stream(h, stream):
    _check(load().lbem_set_stream(h, stream))


def lbem_sync(h):
    _check(load().lbem_sync(h))


def lbem_info(h):
    n, b = _LL(), C.c_size_t()
    _check(load().lbem_info(h, C.byref(n), C.byref(b)))
    return n.value, b.value


def lbem_set_medium(h, eps_r, mu_r=None):
    n = lbem_info(h)[0]
    _check(load().lbem_set_medium(h, _ptr(eps_r, count=n), _ptr(mu_r, count=n)))


def lbem_set_fields(h, E=None, B=None):
    n = lbem_info(h)[0]
    _check(load().lbem_set_fields(h, _ptr(E, count=3 * n), _ptr(B, count=3 * n)))


def lbem_set_sources(h, site, comp, amp):
    site = np.ascontiguousarray(site, dtype=np.int64).ravel()
    comp = np.ascontiguousarray(comp, dtype=np.int32).ravel()
    amp = np.ascontiguousarray(amp, dtype=np.float32)
    if amp.ndim == 1:
        amp = amp[None, :]
    n = site.size
    nt = amp.shape[1] if n else 1
    _check(load().lbem_set_sources(h, n, _ptr(site, np.int64), _ptr(comp, np.int32), _ptr(amp), nt))


def lbem_set_receivers(h, site, comp, capacity):
    site = np.ascontiguousarray(site, dtype=np.int64).ravel()
    comp = np.ascontiguousarray(comp, dtype=np.int32).ravel()
    _check(load().lbem_set_receivers(h, site.size, _ptr(site, np.int64), _ptr(comp, np.int32), int(capacity)))


def lbem_step(h, nsteps):
    _check(load().lbem_step(h, int(nsteps)))


def lbem_set_watchdog(h, every, max_growth=1e6):
    _check(load().lbem_set_watchdog(h, int(every), float(max_growth)))


BC_PERIODIC, BC_PEC, BC_PMC = 0, 1, 2


def lbem_set_boundaries(h, kind, layer=0, gamma_max=0.0):
    """kind: boundary per axis (x, y[, z]): BC_PERIODIC, BC_PEC or BC_PMC."""
    k = (_I * 3)(*(list(kind) + [0] * (3 - len(kind))))
    _check(load().lbem_set_boundaries(h, k, int(layer), float(gamma_max)))


def lbem_rows(h, plane, row0, nrows, buf, to_state):
    """Copy nrows rows of one population plane of the current state to (to_state False) or from (True) buf."""
    _check(load().lbem_rows(h, int(plane), int(row0), int(nrows), _ptr(buf, writable=not to_state),
                            1 if to_state else 0))


def lbem_set_medium_aniso(h, eps_r, mu_xx, mu_yy):
    """eps_r per site ([nsite], host or device) and a uniform permeability tensor diag(mu_xx, mu_yy) (2D)."""
    n = lbem_info(h)[0]
    _check(load().lbem_set_medium_aniso(h, _ptr(eps_r, count=n), float(mu_xx), float(mu_yy)))


def lbem_set_dispersion(h, wp2, wr2=None, gamma=None):
    """One Drude-Lorentz pole per site ([nsite] arrays, host or device; wp2 None removes it)."""
    n = lbem_info(h)[0]
    _check(load().lbem_set_dispersion(h, _ptr(wp2, count=n), _ptr(wr2, count=n), _ptr(gamma, count=n)))


def lbem_get_boundaries(h):
    """((kind_x, kind_y, kind_z), layer, gamma_max)."""
    k, L, g = (_I * 3)(), _I(), _D()
    _check(load().lbem_get_boundaries(h, k, C.byref(L), C.byref(g)))
    return tuple(k), L.value, g.value


def lbem_set_temporal_blocking(h, steps_per_pass, tile_shape=-1):
    _check(load().lbem_set_temporal_blocking(h, int(steps_per_pass), int(tile_shape)))


def lbem_get_temporal_blocking(h):
    """(steps_per_pass, tile_shape, number of tile shapes)."""
    a, b, c = _I(), _I(), _I()
    _check(load().lbem_get_temporal_blocking(h, C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def lbem_set_graphs(h, on):
    _check(load().lbem_set_graphs(h, 1 if on else 0))


def lbem_time(h):
    t = _LL()
    _check(load().lbem_time(h, C.byref(t)))
    return t.value


def lbem_fields(h, E=None, B=None):
    n = lbem_info(h)[0]
    _check(load().lbem_fields(h, _ptr(E, count=3 * n, writable=True), _ptr(B, count=3 * n, writable=True)))


def lbem_energy_flux(h, u=None, P=None):
    n = lbem_info(h)[0]
    _check(load().lbem_energy_flux(h, _ptr(u, count=n, writable=True), _ptr(P, count=3 * n, writable=True)))


def lbem_traces(h, out=None):
    k = _I()
    _check(load().lbem_traces(h, _ptr(out, writable=True), C.byref(k)))
    return k.value


def lbem_diagnostics(h):
    out = (_D * 3)()
    _check(load().lbem_diagnostics(h, out))
    return float(out[0]), float(out[1]), float(out[2])


def lbem_diagnostics_static(dim, nx, ny, nz, state, eps_r, mu_r, c_ref2, out, stream=None):
    _check(load().lbem_diagnostics_static(int(dim), int(nx), int(ny), int(nz), _ptr(state, np.uint8), _ptr(eps_r),
                                          _ptr(mu_r), float(c_ref2), _ptr(out, np.float64, 3, writable=True), stream))


def lbem_check_guards(h):
    _check(load().lbem_check_guards(h))


def lbem_halo_out(h, halo, up, down):
    _check(load().lbem_halo_out(h, int(halo), _ptr(up, writable=True), _ptr(down, writable=True)))


def lbem_halo_in(h, halo, from_below, from_above):
    _check(load().lbem_halo_in(h, int(halo), _ptr(from_below), _ptr(from_above)))


def lbem_save_state(h, dst):
    _check(load().lbem_save_state(h, _ptr(dst, np.uint8, writable=True)))


def lbem_load_state(h, src, t_at_save):
    _check(load().lbem_load_state(h, _ptr(src, np.uint8), int(t_at_save)))


def lbem_forward_record(h, nsteps, checkpoint_every):
    _check(load().lbem_forward_record(h, int(nsteps), int(checkpoint_every)))


def lbem_adjoint(h, trace_cot, grad_eps, grad_cL2=None):
    _check(load().lbem_adjoint(h, _ptr(trace_cot), _ptr(grad_eps, writable=True),
                               _ptr(grad_cL2, np.float64, writable=True)))


def lbem_autotune(h, trial_steps):
    b = _I()
    _check(load().lbem_autotune(h, int(trial_steps), C.byref(b)))
    return b.value


def lbem_set_variant(h, v):
    _check(load().lbem_set_variant(h, int(v)))


def lbem_get_variant(h):
    v, n = _I(), _I()
    _check(load().lbem_get_variant(h, C.byref(v), C.byref(n)))
    return v.value, n.value


def lbem_batch_create(members, stream=None):
    arr = (_VP * len(members))(*[m.value if isinstance(m, _VP) else m for m in members])
    b = _VP()
    _check(load().lbem_batch_create(len(members), arr, stream, C.byref(b)))
    return b


def lbem_batch_step(b, nsteps):
    _check(load().lbem_batch_step(b, int(nsteps)))


def lbem_batch_autotune(b, trial_steps):
    k = _I()
    _check(load().lbem_batch_autotune(b, int(trial_steps), C.byref(k)))
    return k.value


def lbem_batch_set_variant(b, v):
    _check(load().lbem_batch_set_variant(b, int(v)))


def lbem_batch_get_variant(b):
    v, n = _I(), _I()
    _check(load().lbem_batch_get_variant(b, C.byref(v), C.byref(n)))
    return v.value, n.value


def lbem_batch_destroy(b):
    load().lbem_batch_destroy(b)


# --------------------------------------------------------------------------- convenience wrapper


class Solver:
    """Owns one lbem handle on the current CUDA device and torch stream."""

    def __init__(self, shape, storage="f32", c_ref2=0.0, stream=None):
        import torch

        self.shape = tuple(shape)
        self.dim = len(shape)
        if self.dim == 2:
            ny, nx = shape
            nz = 1
        else:
            nz, ny, nx = shape
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        st = STORAGE[storage] if isinstance(storage, str) else storage
        self.h = lbem_create(self.dim, nx, ny, nz, st, c_ref2, stream)
        self.nsite = lbem_info(self.h)[0]

    def close(self):
        if self.h:
            lbem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_problem(self, p, device="cuda"):
        """Upload a workloads.Problem: medium, sources, receivers, initial fields (t = 0)."""
        import torch

        eps = torch.as_tensor(np.ascontiguousarray(p.eps_r, np.float32).ravel(), device=device)
        mu = None if p.mu_r is None else torch.as_tensor(np.ascontiguousarray(p.mu_r, np.float32).ravel(), device=device)
        if getattr(p, "aniso", None) is not None:
            lbem_set_medium_aniso(self.h, eps, *p.aniso)
        else:
            lbem_set_medium(self.h, eps, mu)
        if getattr(p, "wp2", None) is not None:
            dev = lambda a: None if a is None else torch.as_tensor(
                np.ascontiguousarray(np.broadcast_to(a, p.shape), np.float32).ravel(), device=device)
            lbem_set_dispersion(self.h, dev(p.wp2), dev(p.wr2), dev(p.gamma))
        bc = tuple(getattr(p, "bc", (0, 0, 0)))
        if any(bc) or any(lbem_get_boundaries(self.h)[0]):
            lbem_set_boundaries(self.h, bc, getattr(p, "layer", 0), getattr(p, "gamma_max", 0.0))
        if p.src_site.size:
            lbem_set_sources(self.h, p.src_site, p.src_comp, p.src_amp)
        else:
            lbem_set_sources(self.h, [], [], np.zeros((0, 1), np.float32))
        lbem_set_receivers(self.h, p.rec_site, p.rec_comp, p.nsteps)
        E = None if p.E0 is None else torch.as_tensor(np.ascontiguousarray(np.moveaxis(p.E0, -1, 0), np.float32).ravel(), device=device)
        B = None if p.B0 is None else torch.as_tensor(np.ascontiguousarray(np.moveaxis(p.B0, -1, 0), np.float32).ravel(), device=device)
        lbem_set_fields(self.h, E, B)

    def step(self, n):
        lbem_step(self.h, n)

    def fields(self):
        """(E, B) as torch CUDA tensors of shape (3,) + grid."""
        import torch

        E = torch.empty(3 * self.nsite, dtype=torch.float32, device="cuda")
        B = torch.empty_like(E)
        lbem_fields(self.h, E, B)
        return E.view((3,) + self.shape), B.view((3,) + self.shape)

    def traces(self, nrec):
        import torch

        n = lbem_traces(self.h, None)
        out = torch.empty(max(nrec * n, 1), dtype=torch.float32, device="cuda")
        if nrec and n:
            lbem_traces(self.h, out)
        return out[: nrec * n].view(nrec, n)

    def diagnostics(self):
        return lbem_diagnostics(self.h)
