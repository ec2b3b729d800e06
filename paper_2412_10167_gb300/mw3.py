"""Python binding of libmw3 (ctypes). Argument marshalling only.

Every entry point of ``include/mw3.h`` is exposed under the same name; every step
of the propagation runs in the library's CUDA kernels. There is no CPU fallback:
importing this module fails if ``libmw3.so`` is missing, and creating a device
context fails if no CUDA device is present.

``Propagator`` builds a context from a workload dictionary (bohr, eV, amu, as in
the ``workloads`` module) and converts units at this edge: energies to hartree,
masses to electron masses.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libmw3.so")

HARTREE_EV = 27.211386245988
AMU_ME = 1822.888486

MW3_FP64, MW3_MIXED = 0, 1
STATUS = {0: "MW3_OK", -1: "MW3_ERR_BAD_ARG", -2: "MW3_ERR_OOM", -3: "MW3_ERR_CUDA",
          -4: "MW3_ERR_DIVERGED", -5: "MW3_ERR_SPECTRUM", -6: "MW3_ERR_TIMEOUT",
          -7: "MW3_ERR_STATE", -8: "MW3_ERR_IO", -9: "MW3_ERR_NAN"}


class mw3_grid_desc(C.Structure):
    _fields_ = [("NR", C.c_int), ("Rmin", C.c_double), ("Rmax", C.c_double),
                ("nr", C.c_int), ("rmin", C.c_double), ("rmax", C.c_double),
                ("ngamma", C.c_int), ("masses", C.c_double * 3), ("nJ", C.c_int),
                ("J", C.POINTER(C.c_int)), ("omega_max", C.c_int), ("nelec", C.c_int)]


class mw3_packet_desc(C.Structure):
    _fields_ = [("R0", C.c_double), ("Gamma", C.c_double), ("Ecol", C.c_double),
                ("v0", C.c_int), ("j0", C.c_int), ("omega0", C.c_int), ("elec0", C.c_int)]


class mw3_pcb_desc(C.Structure):
    _fields_ = [("arrangement", C.c_int), ("rmin", C.c_double), ("rmax", C.c_double),
                ("nr", C.c_int)]


class mw3_analysis_desc(C.Structure):
    _fields_ = [("rstar", C.c_double), ("E_lo", C.c_double), ("E_hi", C.c_double),
                ("nE", C.c_int), ("Rinf", C.c_double), ("vmax", C.c_int), ("jmax", C.c_int),
                ("kmin", C.c_long)]


class mw3_products_desc(C.Structure):
    _fields_ = [("arrangement", C.c_int), ("Rinf", C.c_double), ("nr", C.c_int),
                ("rmin", C.c_double), ("rmax", C.c_double), ("ngamma", C.c_int),
                ("vmax", C.c_int), ("jmax", C.c_int)]


ARRANGEMENTS = {"AC+B": 1, "AB+C": 2}
PCB_ARRANGEMENTS = {"A+BC": 0, "AC+B": 1, "AB+C": 2}


class mw3_leps_params(C.Structure):
    _fields_ = [("D", C.c_double), ("beta", C.c_double), ("re", C.c_double),
                ("delta", C.c_double), ("masses", C.c_double * 3), ("two_state", C.c_int),
                ("bump", C.c_double), ("bump_r0", C.c_double), ("bump_w2", C.c_double),
                ("coup", C.c_double), ("coup_R0", C.c_double), ("coup_r0", C.c_double),
                ("coup_w2", C.c_double)]


POT_FN = C.CFUNCTYPE(C.c_int, C.c_double, C.c_double, C.c_double, C.POINTER(C.c_double),
                     C.c_void_p)
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

# name -> (restype, argtypes)
_SIGS = {
    "mw3_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int]),
    "mw3_destroy": (None, [C.c_void_p]),
    "mw3_last_error": (C.c_char_p, [C.c_void_p]),
    "mw3_status_string": (C.c_char_p, [C.c_int]),
    "mw3_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mw3_set_allocator": (C.c_int, [C.c_void_p, ALLOC_FN, FREE_FN, C.c_void_p]),
    "mw3_grid": (C.c_int, [C.c_void_p, C.POINTER(mw3_grid_desc)]),
    "mw3_load_potential": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_double,
                                     C.c_double]),
    "mw3_load_potential_grid": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_double,
                                          C.c_double, C.c_double]),
    "mw3_pes_leps": (C.c_int, [C.c_double, C.c_double, C.c_double, C.POINTER(C.c_double),
                               C.c_void_p]),
    "mw3_init_packet": (C.c_int, [C.c_void_p, C.POINTER(mw3_packet_desc)]),
    "mw3_init_packet_pcb": (C.c_int, [C.c_void_p, C.POINTER(mw3_packet_desc),
                                      C.POINTER(mw3_pcb_desc)]),
    "mw3_set_absorber": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_int, C.c_double,
                                   C.c_double, C.c_int]),
    "mw3_set_analysis": (C.c_int, [C.c_void_p, C.POINTER(mw3_analysis_desc)]),
    "mw3_set_products": (C.c_int, [C.c_void_p, C.POINTER(mw3_products_desc)]),
    "mw3_product_probabilities": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "mw3_propagate": (C.c_int, [C.c_void_p, C.c_long]),
    "mw3_iteration": (C.c_long, [C.c_void_p]),
    "mw3_flux_probabilities": (C.c_int, [C.c_void_p, C.POINTER(C.c_double),
                                         C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "mw3_get_state": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "mw3_set_state": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "mw3_set_state_f32": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_float)]),
    "mw3_apply_hs": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "mw3_norm_trace": (C.c_long, [C.c_void_p, C.POINTER(C.c_double), C.c_long]),
    "mw3_enable_autocorrelation": (C.c_int, [C.c_void_p]),
    "mw3_incoming_amplitude": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "mw3_lanczos": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_int,
                              C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "mw3_bound_states": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_int, C.c_double,
                                   C.c_double, C.c_int, C.POINTER(C.c_double),
                                   C.POINTER(C.c_int)]),
    "mw3_bound_state_vector": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_int, C.c_int,
                                         C.c_double, C.POINTER(C.c_double)]),
    "mw3_enable_time_packets": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double)]),
    "mw3_time_packets": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_long)]),
    "mw3_autocorrelation": (C.c_long, [C.c_void_p, C.POINTER(C.c_double), C.c_long]),
    "mw3_photo_spectrum": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_int,
                                     C.POINTER(C.c_double)]),
    "mw3_sizes": (C.c_int, [C.c_void_p, C.POINTER(C.c_long), C.POINTER(C.c_long)]),
    "mw3_spectral_range": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "mw3_reference_energy": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "mw3_checkpoint_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "mw3_checkpoint_load": (C.c_int, [C.c_void_p, C.c_char_p]),
    "mw3_measure_peak": (C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_double)]),
    "mw3_norms_noalloc": (C.c_int, [C.c_void_p, C.c_long, C.c_int, C.c_void_p, C.c_void_p]),
    "mw3_mlp_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_int, C.c_int,
                                 C.c_ulonglong]),
    "mw3_mlp_destroy": (None, [C.c_void_p]),
    "mw3_mlp_last_error": (C.c_char_p, [C.c_void_p]),
    "mw3_mlp_num_params": (C.c_long, [C.c_void_p]),
    "mw3_mlp_set_params": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "mw3_mlp_get_params": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "mw3_mlp_forward": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.c_long,
                                  C.POINTER(C.c_float)]),
    "mw3_mlp_loss_grad": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_float),
                                    C.c_long, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "mw3_mlp_train": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_long,
                                C.c_int, C.c_int, C.c_double, C.c_double, C.c_ulonglong,
                                C.POINTER(C.c_double)]),
    "mw3_set_tuning": (C.c_int, [C.c_void_p, C.c_char_p, C.c_long]),
    "mw3_get_tuning": (C.c_long, [C.c_void_p, C.c_char_p]),
    "mw3_kernel_times": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_char_p),
                                   C.POINTER(C.c_double), C.POINTER(C.c_long),
                                   C.POINTER(C.c_int)]),
}


def load_library(path: str = _LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libmw3.so not built at {path}; run __graft_entry__.build()")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = load_library()
EXPORTED = tuple(_SIGS)


class MW3Error(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _check(ctx, code):
    if code != 0:
        raise MW3Error(code, lib.mw3_last_error(ctx).decode())
    return code


# ----------------------------------------------------------- same-name wrappers

def mw3_create(device: int, precision: int):
    h = C.c_void_p()
    code = lib.mw3_create(C.byref(h), device, precision)
    if code != 0:
        raise MW3Error(code, lib.mw3_last_error(None).decode())
    return h


def mw3_destroy(ctx):
    lib.mw3_destroy(ctx)


def mw3_grid(ctx, NR, Rmin, Rmax, nr, rmin, rmax, ngamma, masses, J, omega_max, nelec):
    Jarr = (C.c_int * len(J))(*J)
    d = mw3_grid_desc(NR, Rmin, Rmax, nr, rmin, rmax, ngamma, (C.c_double * 3)(*masses),
                      len(J), Jarr, omega_max, nelec)
    return _check(ctx, lib.mw3_grid(ctx, C.byref(d)))


def mw3_load_potential(ctx, fn, user, vcut, tcut_rad, ecut_rot):
    return _check(ctx, lib.mw3_load_potential(ctx, fn, user, vcut, tcut_rad, ecut_rot))


def mw3_load_potential_grid(ctx, V, vcut, tcut_rad, ecut_rot):
    V = np.ascontiguousarray(V, dtype=np.float64)
    return _check(ctx, lib.mw3_load_potential_grid(ctx, _dp(V), vcut, tcut_rad, ecut_rot))


def mw3_init_packet(ctx, R0, Gamma, Ecol, v0, j0, omega0, elec0):
    d = mw3_packet_desc(R0, Gamma, Ecol, v0, j0, omega0, elec0)
    return _check(ctx, lib.mw3_init_packet(ctx, C.byref(d)))


def mw3_set_absorber(ctx, RI, AR, nR, rI, Ar, nr):
    return _check(ctx, lib.mw3_set_absorber(ctx, RI, AR, nR, rI, Ar, nr))


def mw3_set_analysis(ctx, rstar, E_lo, E_hi, nE, Rinf, vmax, jmax, kmin):
    d = mw3_analysis_desc(rstar, E_lo, E_hi, nE, Rinf, vmax, jmax, kmin)
    return _check(ctx, lib.mw3_set_analysis(ctx, C.byref(d)))


def mw3_propagate(ctx, nsteps):
    return _check(ctx, lib.mw3_propagate(ctx, int(nsteps)))


def mw3_iteration(ctx):
    return lib.mw3_iteration(ctx)


def mw3_norms_noalloc(x_ptr: int, seg_len: int, nseg: int, out_ptr: int, stream: int = 0) -> int:
    """Allocation-free per-segment sums of squares on device pointers (no cudaMalloc)."""
    code = lib.mw3_norms_noalloc(C.c_void_p(x_ptr), seg_len, nseg, C.c_void_p(out_ptr),
                                 C.c_void_p(stream))
    if code != 0:
        raise MW3Error(code, "mw3_norms_noalloc failed")
    return code


def mw3_measure_peak(device: int, kind: int) -> float:
    v = C.c_double()
    code = lib.mw3_measure_peak(device, kind, C.byref(v))
    if code != 0:
        raise MW3Error(code, "peak probe failed")
    return v.value


# ------------------------------------------------------------ workload driver

class Propagator:
    """One libmw3 context configured from a workload dictionary."""

    def __init__(self, cfg: dict, device: int = 0, precision: str | None = None,
                 torch_memory: bool = True, analysis: bool = True, tuning: dict | None = None):
        self.cfg = cfg
        prec = precision or cfg.get("precision", "fp64")
        self.precision = MW3_FP64 if prec == "fp64" else MW3_MIXED
        self.ctx = mw3_create(device, self.precision)
        self._keep = []
        self._stream = None
        if device >= 0 and torch_memory:
            self._use_torch(device)
        if tuning == "auto":
            from . import tune as _tune
            tuning = _tune.tune(cfg, "fp64" if self.precision == MW3_FP64 else "mixed",
                                device=device)
        for key, val in (tuning or {}).items():
            _check(self.ctx, lib.mw3_set_tuning(self.ctx, key.encode(), int(val)))
        g = cfg["grid"]
        self.masses = tuple(m * AMU_ME for m in cfg["masses_u"])
        mw3_grid(self.ctx, g["NR"], g["Rmin"], g["Rmax"], g["nr"], g["rmin"], g["rmax"],
                 g["ngamma"], self.masses, cfg["J"], cfg["omega_max"], cfg["nelec"])
        caps = cfg["caps"]
        pes = cfg["pes"]
        if pes.get("kind", "leps") == "leps":
            p = mw3_leps_params()
            p.D = pes["D_eV"] / HARTREE_EV
            p.beta, p.re, p.delta = pes["beta"], pes["re"], pes["delta"]
            p.masses = (C.c_double * 3)(*self.masses)
            ts = pes.get("two_state")
            if ts:
                p.two_state = 1
                p.bump, p.bump_r0, p.bump_w2 = ts["bump_eV"] / HARTREE_EV, ts["bump_r0"], ts["bump_w2"]
                p.coup, p.coup_R0 = ts["coup_eV"] / HARTREE_EV, ts["coup_R0"]
                p.coup_r0, p.coup_w2 = ts["coup_r0"], ts["coup_w2"]
            self._keep.append(p)
            fn = C.cast(lib.mw3_pes_leps, C.c_void_p)
            mw3_load_potential(self.ctx, fn, C.cast(C.pointer(p), C.c_void_p),
                               caps["vcut_eV"] / HARTREE_EV, caps["tcut_eV"] / HARTREE_EV,
                               caps["erot_eV"] / HARTREE_EV)
        else:
            raise ValueError("use load_potential_grid() for non-LEPS surfaces")
        self.init_packet()
        a = cfg["absorber"]
        mw3_set_absorber(self.ctx, a["RI"], a["AR"], a["nR"], a["rI"], a["Ar"], a["nr"])
        if analysis:
            self.set_analysis()

    def _use_torch(self, device):
        import torch
        torch.cuda.set_device(device)
        self._stream = torch.cuda.Stream(device=device)
        stream = self._stream

        def _alloc(nbytes, user):
            return torch.cuda.caching_allocator_alloc(int(nbytes), device, stream)

        def _free(ptr, user):
            torch.cuda.caching_allocator_delete(ptr)

        fa, ff = ALLOC_FN(_alloc), FREE_FN(_free)
        self._keep += [fa, ff]
        _check(self.ctx, lib.mw3_set_stream(self.ctx, C.c_void_p(stream.cuda_stream)))
        _check(self.ctx, lib.mw3_set_allocator(self.ctx, fa, ff, None))

    def init_packet(self):
        pk = self.cfg["packet"]
        src = self.cfg.get("pcb")
        if src:   # products-coordinate-based start: the grid is the product arrangement
            d = mw3_packet_desc(pk["R0"], pk["Gamma"], pk["Ecol_eV"] / HARTREE_EV, pk["v0"],
                                pk["j0"], pk["omega0"], pk["elec0"])
            s = mw3_pcb_desc(PCB_ARRANGEMENTS[src["arrangement"]], src["rmin"], src["rmax"],
                             src["nr"])
            _check(self.ctx, lib.mw3_init_packet_pcb(self.ctx, C.byref(d), C.byref(s)))
            return
        mw3_init_packet(self.ctx, pk["R0"], pk["Gamma"], pk["Ecol_eV"] / HARTREE_EV, pk["v0"],
                        pk["j0"], pk["omega0"], pk["elec0"])

    def set_analysis(self):
        an = self.cfg["analysis"]
        pd = an.get("products")
        if pd:
            d = mw3_products_desc(ARRANGEMENTS[pd["arrangement"]], pd["Rinf"], pd["nr"], pd["rmin"],
                                  pd["rmax"], pd["ngamma"], pd["vmax"], pd["jmax"])
            _check(self.ctx, lib.mw3_set_products(self.ctx, C.byref(d)))
        mw3_set_analysis(self.ctx, an["rstar"], an["E_lo_eV"] / HARTREE_EV,
                         an["E_hi_eV"] / HARTREE_EV, an["nE"], an["Rinf"], an.get("vmax", -1),
                         an.get("jmax", 0), an.get("kmin", 0))

    # -------------------------------------------------------------- queries
    @property
    def stream(self):
        """The torch stream the library's kernels are launched on (None without torch memory)."""
        return self._stream

    @property
    def shape(self):
        nb, npb = C.c_long(), C.c_long()
        _check(self.ctx, lib.mw3_sizes(self.ctx, C.byref(nb), C.byref(npb)))
        g = self.cfg["grid"]
        return (nb.value, g["ngamma"], g["nr"], g["NR"])

    def propagate(self, n):
        return mw3_propagate(self.ctx, n)

    @property
    def iteration(self):
        return lib.mw3_iteration(self.ctx)

    def state(self):
        q = np.zeros(self.shape)
        qp = np.zeros(self.shape)
        _check(self.ctx, lib.mw3_get_state(self.ctx, _dp(q), _dp(qp)))
        return q, qp

    def set_state(self, q, qprev=None):
        q = np.ascontiguousarray(q, dtype=np.float64)
        qp = None if qprev is None else np.ascontiguousarray(qprev, dtype=np.float64)
        _check(self.ctx, lib.mw3_set_state(self.ctx, _dp(q), None if qp is None else _dp(qp)))

    def set_state_f32(self, q, qprev=None):
        q = np.ascontiguousarray(q, dtype=np.float32)
        qp = None if qprev is None else np.ascontiguousarray(qprev, dtype=np.float32)
        _check(self.ctx, lib.mw3_set_state_f32(self.ctx, _fp(q), None if qp is None else _fp(qp)))

    def apply_hs(self, q):
        q = np.ascontiguousarray(q, dtype=np.float64)
        out = np.zeros_like(q)
        _check(self.ctx, lib.mw3_apply_hs(self.ctx, _dp(q), _dp(out)))
        return out

    def spectral_range(self):
        n = len(self.cfg["J"])
        E0, dE = np.zeros(n), np.zeros(n)
        _check(self.ctx, lib.mw3_spectral_range(self.ctx, _dp(E0), _dp(dE)))
        return E0, dE

    def reference_energy(self):
        e = C.c_double()
        _check(self.ctx, lib.mw3_reference_energy(self.ctx, C.byref(e)))
        return e.value

    def probabilities(self):
        an = self.cfg["analysis"]
        nJ, nE = len(self.cfg["J"]), an["nE"]
        E = np.zeros(nE)
        P = np.zeros((nJ, nE))
        vmax = an.get("vmax", -1)
        Pin = None
        if vmax >= 0:
            Pin = np.zeros((nJ, self.cfg["nelec"], vmax + 1, an["jmax"] + 1, nE))
        _check(self.ctx, lib.mw3_flux_probabilities(self.ctx, _dp(E), _dp(P),
                                                    None if Pin is None else _dp(Pin)))
        return E, P, Pin

    def product_probabilities(self):
        """|S|^2 of the product channels summed over Omega': [nJ, nelec, v', j', nE]."""
        pd = self.cfg["analysis"]["products"]
        P = np.zeros((len(self.cfg["J"]), self.cfg["nelec"], pd["vmax"] + 1, pd["jmax"] + 1,
                      self.cfg["analysis"]["nE"]))
        _check(self.ctx, lib.mw3_product_probabilities(self.ctx, _dp(P)))
        return P

    def norm_trace(self, n=None):
        nJ = len(self.cfg["J"])
        n = self.iteration if n is None else n
        out = np.zeros((max(n, 0), nJ))
        cnt = lib.mw3_norm_trace(self.ctx, _dp(out), n)
        return out[:cnt]

    def lanczos(self, v0, m):
        """(alpha[m, nJ], beta[m, nJ]) of m non-orthogonal Lanczos steps from grid values v0."""
        v0 = np.ascontiguousarray(np.asarray(v0, dtype=np.float64).reshape(self.shape))
        nJ = len(self.cfg["J"])
        a, b = np.zeros((m, nJ)), np.zeros((m, nJ))
        _check(self.ctx, lib.mw3_lanczos(self.ctx, _dp(v0), m, _dp(a), _dp(b)))
        return a, b

    def bound_states(self, v0, m, emin=-1e300, emax=1e300, maxev=4096):
        """Accepted Lanczos eigenvalues (hartree) per J inside [emin, emax]: list of arrays."""
        v0 = np.ascontiguousarray(np.asarray(v0, dtype=np.float64).reshape(self.shape))
        nJ = len(self.cfg["J"])
        E = np.zeros((nJ, maxev))
        cnt = np.zeros(nJ, dtype=np.int32)
        _check(self.ctx, lib.mw3_bound_states(self.ctx, _dp(v0), m, emin, emax, maxev, _dp(E),
                                              cnt.ctypes.data_as(C.POINTER(C.c_int))))
        return [E[i, :cnt[i]].copy() for i in range(nJ)]

    def bound_state_vector(self, v0, m, E, iJ=0):
        """Normalised Ritz vector (grid values) of J index iJ for the eigenvalue E."""
        v0 = np.ascontiguousarray(np.asarray(v0, dtype=np.float64).reshape(self.shape))
        out = np.zeros(self.shape)
        _check(self.ctx, lib.mw3_bound_state_vector(self.ctx, _dp(v0), m, iJ, E, _dp(out)))
        return out

    def incoming_amplitude(self):
        """|a(E)|^2 of the packet's incoming part at the analysis energies."""
        out = np.zeros(self.cfg["analysis"]["nE"])
        _check(self.ctx, lib.mw3_incoming_amplitude(self.ctx, _dp(out)))
        return out

    def enable_autocorrelation(self):
        """Keep the current state as Psi(k=0) and record C_k = <Psi(0)|Psi(k)> per J."""
        _check(self.ctx, lib.mw3_enable_autocorrelation(self.ctx))

    def enable_time_packets(self, times):
        """Accumulate Psi(t) = sum_k f_k(t) q_k for the given times (atomic units) from k = 0."""
        t = np.ascontiguousarray(np.asarray(times, dtype=np.float64))
        self._tp_nt = len(t)
        _check(self.ctx, lib.mw3_enable_time_packets(self.ctx, len(t), _dp(t)))

    def time_packets(self):
        """(Psi(t_j) as complex grid values [nt, nblocks, ngamma, nr, NR], K)."""
        out = np.zeros((self._tp_nt, 2, int(np.prod(self.shape))))
        K = C.c_long(0)
        _check(self.ctx, lib.mw3_time_packets(self.ctx, _dp(out), C.byref(K)))
        psi = out[:, 0] + 1j * out[:, 1]
        return psi.reshape((self._tp_nt,) + self.shape), K.value

    def autocorrelation(self):
        """C[k, iJ] for the recorded iterations k = 0 .. iteration - 1."""
        nJ = len(self.cfg["J"])
        n = self.iteration
        out = np.zeros((max(n, 0), nJ))
        cnt = lib.mw3_autocorrelation(self.ctx, _dp(out), n)
        if cnt < 0:
            _check(self.ctx, int(cnt))
        return out[:cnt]

    def photo_spectrum(self, E):
        """a0(E) per J (Eq. chebyshev-transform) at total energies E (hartree)."""
        E = np.ascontiguousarray(np.asarray(E, dtype=np.float64))
        out = np.zeros((len(self.cfg["J"]), len(E)))
        _check(self.ctx, lib.mw3_photo_spectrum(self.ctx, _dp(E), len(E), _dp(out)))
        return out

    def set_tuning(self, key, value):
        _check(self.ctx, lib.mw3_set_tuning(self.ctx, key.encode(), int(value)))

    def get_tuning(self, key):
        return lib.mw3_get_tuning(self.ctx, key.encode())

    def kernel_times(self, enable=None):
        cnt = C.c_int(16)
        names = (C.c_char_p * 16)()
        ms = (C.c_double * 16)()
        nl = (C.c_long * 16)()
        en = -1 if enable is None else int(bool(enable))
        _check(self.ctx, lib.mw3_kernel_times(self.ctx, en, names, ms, nl, C.byref(cnt)))
        return {names[i].decode(): (ms[i], nl[i]) for i in range(cnt.value)}

    def checkpoint_save(self, path):
        _check(self.ctx, lib.mw3_checkpoint_save(self.ctx, path.encode()))

    def checkpoint_load(self, path):
        _check(self.ctx, lib.mw3_checkpoint_load(self.ctx, path.encode()))

    def close(self):
        if self.ctx:
            mw3_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------ surrogate network

def _fp(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


class MLP:
    """The J-interpolation surrogate network (hand-written CUDA training/inference)."""

    def __init__(self, n_in=4, width=256, depth=3, seed=10167, device=0):
        h = C.c_void_p()
        code = lib.mw3_mlp_create(C.byref(h), device, n_in, width, depth, seed)
        if code != 0:
            raise MW3Error(code, "mw3_mlp_create failed")
        self.h = h
        self.n_in = n_in
        self.sizes = [n_in] + [width] * depth + [1]

    def _chk(self, code):
        if code != 0:
            raise MW3Error(code, lib.mw3_mlp_last_error(self.h).decode())

    @property
    def num_params(self):
        return lib.mw3_mlp_num_params(self.h)

    def get_params(self):
        p = np.zeros(self.num_params)
        self._chk(lib.mw3_mlp_get_params(self.h, _dp(p)))
        return p

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float64)
        self._chk(lib.mw3_mlp_set_params(self.h, _dp(flat)))

    def forward(self, X):
        X = np.ascontiguousarray(X, dtype=np.float32)
        y = np.zeros(X.shape[0], dtype=np.float32)
        self._chk(lib.mw3_mlp_forward(self.h, _fp(X), X.shape[0], _fp(y)))
        return y

    def loss_grad(self, X, y):
        X = np.ascontiguousarray(X, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.float32)
        loss = C.c_double()
        g = np.zeros(self.num_params)
        self._chk(lib.mw3_mlp_loss_grad(self.h, _fp(X), _fp(y), X.shape[0], C.byref(loss), _dp(g)))
        return loss.value, g

    def train(self, X, y, epochs, batch=4096, lr=1e-3, wd=0.0, seed=10167):
        X = np.ascontiguousarray(X, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.float32)
        loss = C.c_double()
        self._chk(lib.mw3_mlp_train(self.h, _fp(X), _fp(y), X.shape[0], epochs, batch, lr, wd,
                                    seed, C.byref(loss)))
        return loss.value

    def unflatten(self, flat):
        """[(W, b), ...] views of a flat parameter vector (library order)."""
        out, o = [], 0
        for a, b in zip(self.sizes[:-1], self.sizes[1:]):
            W = flat[o:o + a * b].reshape(b, a)
            o += a * b
            bb = flat[o:o + b]
            o += b
            out.append([W, bb])
        return out

    def close(self):
        if self.h:
            lib.mw3_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
