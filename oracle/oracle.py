"""ctypes wrapper of the plain-C FP64 oracle (test infrastructure only).

Only the test-suite, the smoke check and the CPU-baseline leg of the benchmark import this
module.  It marshals a problem description (the plain dict produced by the seeded input
generators) into the oracle's own parameter struct; it shares no code with the CUDA path.
"""
import ctypes
import os

import numpy as np

from . import build_oracle

_c_int = ctypes.c_int
_c_double = ctypes.c_double

BC = {"periodic": 0, "outflow": 1, "reflect": 2, "dirichlet": 3}
EXCHANGE = {"full": 0, "absorb": 1, "equilibrium": 2, "frozen_t": 3, "linear": 4}
LIMITER = {"minmod": 0, "mc": 1, "none": 2}
CLOSURE = {"m1": 0, "p1": 1}
SPEEDS = {"m1": 0, "fixed": 1}


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("n", _c_int * 3),
        ("dx", _c_double * 3),
        ("bc_lo", _c_int * 3),
        ("bc_hi", _c_int * 3),
        ("dirichlet_lo", (_c_double * 4) * 3),
        ("dirichlet_hi", (_c_double * 4) * 3),
        ("c", _c_double),
        ("a_rad", _c_double),
        ("gamma", _c_double),
        ("mu_over_kB", _c_double),
        ("theta_F", _c_double),
        ("theta_E", _c_double),
        ("E_floor", _c_double),
        ("exchange", _c_int),
        ("beta_tau", _c_int),
        ("limiter", _c_int),
        ("closure", _c_int),
        ("speeds", _c_int),
        ("kappa_P", _c_double),
        ("kappa_F", _c_double),
        ("kappa_rho_pow", _c_int),
        ("linear_eps", _c_double),
    ]


class OrcStats(ctypes.Structure):
    _fields_ = [
        ("n_realizability_fix", ctypes.c_longlong),
        ("n_face_fallback", ctypes.c_longlong),
        ("n_theta_fallback", ctypes.c_longlong),
        ("n_nonfinite", ctypes.c_longlong),
        ("boundary_E_out", _c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build_oracle.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(_c_double)
        L.orc_chi.restype = _c_double
        L.orc_chi.argtypes = [_c_double]
        L.orc_eddington_tensor.argtypes = [_c_double, dp, _c_int, dp]
        L.orc_flux.argtypes = [dp, _c_int, _c_double, _c_int, dp]
        L.orc_wave_speeds.argtypes = [dp, _c_int, _c_double, _c_int, dp, dp]
        L.orc_hll.argtypes = [dp, dp, _c_int, _c_double, _c_int, _c_int, dp]
        L.orc_theta_factor.restype = _c_double
        L.orc_theta_factor.argtypes = [_c_double, _c_double]
        L.orc_limited_slope.restype = _c_double
        L.orc_limited_slope.argtypes = [_c_double, _c_double, _c_int]
        L.orc_quartic_root.restype = _c_double
        L.orc_quartic_root.argtypes = [_c_double, _c_double, _c_double]
        L.orc_exchange_full.restype = _c_int
        L.orc_exchange_full.argtypes = [ctypes.POINTER(OrcParams), _c_double, _c_double, _c_double,
                                        _c_double, dp, dp]
        L.orc_exchange_linear.restype = None
        L.orc_exchange_linear.argtypes = [ctypes.POINTER(OrcParams), _c_double, _c_double, _c_double, dp, dp]
        args = [ctypes.POINTER(OrcParams), _c_int, _c_double, _c_double] + [dp] * 5 + [dp] * 7 + [
            ctypes.POINTER(OrcStats)]
        L.orc_subcycles.restype = _c_int
        L.orc_subcycles.argtypes = args
        L.orc_subcycle_box.restype = _c_int
        L.orc_subcycle_box.argtypes = [ctypes.POINTER(OrcParams), _c_double, _c_double,
                                       ctypes.POINTER(_c_int), ctypes.POINTER(_c_int)] + [dp] * 5 + [
            dp] * 7 + [ctypes.POINTER(OrcStats)]
        L.orc_num_threads.restype = _c_int
        _lib = L
    return _lib


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(_c_double))


def params(desc) -> OrcParams:
    p = OrcParams()
    n = desc["n"]
    for d in range(3):
        p.n[d] = int(n[d])
        p.dx[d] = float(desc["dx"][d])
        p.bc_lo[d] = BC[desc["bc_lo"][d]]
        p.bc_hi[d] = BC[desc["bc_hi"][d]]
        lo = desc.get("dirichlet_lo", [[0.0] * 4] * 3)[d]
        hi = desc.get("dirichlet_hi", [[0.0] * 4] * 3)[d]
        for q in range(4):
            p.dirichlet_lo[d][q] = float(lo[q])
            p.dirichlet_hi[d][q] = float(hi[q])
    p.c = desc["c"]
    p.a_rad = desc["a_rad"]
    p.gamma = desc["gamma"]
    p.mu_over_kB = desc["mu_over_kB"]
    p.theta_F = desc["theta_F"]
    p.theta_E = desc["theta_E"]
    p.E_floor = desc["E_floor"]
    p.exchange = EXCHANGE[desc["exchange"]]
    p.beta_tau = int(bool(desc["beta_tau"]))
    p.limiter = LIMITER[desc["limiter"]]
    p.closure = CLOSURE[desc["closure"]]
    p.speeds = SPEEDS[desc["speeds"]]
    p.kappa_P = desc["kappa_P"]
    p.kappa_F = desc["kappa_F"]
    p.kappa_rho_pow = int(desc["kappa_rho_pow"])
    p.linear_eps = float(desc.get("linear_eps", 1.0))
    return p


# ----------------------------------------------------------------------------- point functions

def chi(f):
    return lib().orc_chi(float(f))


def eddington_tensor(E, G, closure="m1"):
    G = np.ascontiguousarray(G, dtype=np.float64)
    T = np.zeros(9)
    lib().orc_eddington_tensor(float(E), _dp(G), CLOSURE[closure], _dp(T))
    return T.reshape(3, 3)


def flux(U, d, chat, closure="m1"):
    U = np.ascontiguousarray(U, dtype=np.float64)
    out = np.zeros(4)
    lib().orc_flux(_dp(U), int(d), float(chat), CLOSURE[closure], _dp(out))
    return out


def wave_speeds(U, d, chat, speeds="m1"):
    U = np.ascontiguousarray(U, dtype=np.float64)
    l1 = np.zeros(1)
    l3 = np.zeros(1)
    lib().orc_wave_speeds(_dp(U), int(d), float(chat), SPEEDS[speeds], _dp(l1), _dp(l3))
    return float(l1[0]), float(l3[0])


def hll(UL, UR, d, chat, closure="m1", speeds="m1"):
    UL = np.ascontiguousarray(UL, dtype=np.float64)
    UR = np.ascontiguousarray(UR, dtype=np.float64)
    out = np.zeros(4)
    lib().orc_hll(_dp(UL), _dp(UR), int(d), float(chat), CLOSURE[closure], SPEEDS[speeds], _dp(out))
    return out


def theta_factor(theta, x):
    return lib().orc_theta_factor(float(theta), float(x))


def limited_slope(dl, dr, limiter):
    """The oracle's limited slope of a cell from its left / right differences (minmod, mc, none)."""
    return lib().orc_limited_slope(float(dl), float(dr), LIMITER[limiter])


def quartic_root(c4, c1, c0):
    return lib().orc_quartic_root(float(c4), float(c1), float(c0))


def exchange_full(desc, chat, dt, rho, kP, E, T):
    p = params(desc)
    e = np.array([E], dtype=np.float64)
    t = np.array([T], dtype=np.float64)
    fb = lib().orc_exchange_full(ctypes.byref(p), float(chat), float(dt), float(rho), float(kP), _dp(e), _dp(t))
    return float(e[0]), float(t[0]), int(fb)


def exchange_linear(desc, chat, dt, kP, E, T):
    """One linear (Pomraning material) exchange of a single cell; returns (E, T)."""
    p = params(desc)
    e = np.array([E], dtype=np.float64)
    t = np.array([T], dtype=np.float64)
    lib().orc_exchange_linear(ctypes.byref(p), float(chat), float(dt), float(kP), _dp(e), _dp(t))
    return float(e[0]), float(t[0])


# ----------------------------------------------------------------------------- grid functions

_GAS = ("rho", "vx", "vy", "vz", "kP", "kF", "j")


def _prep(case):
    desc = case["desc"]
    f = case["fields"]
    state = {}
    for k in ("E", "Fx", "Fy", "Fz", "T"):
        a = f.get(k)
        state[k] = None if a is None else np.array(a, dtype=np.float64, order="C", copy=True)
    gas = {}
    for k in _GAS:
        a = f.get(k)
        gas[k] = None if a is None else np.ascontiguousarray(a, dtype=np.float64)
    if state["T"] is None:
        state["T"] = np.ones_like(state["E"])
    return desc, state, gas


def subcycles(case, n_sub=None, chat=None, dt=None):
    """Run n_sub subcycles of the oracle on a copy of case['fields']; returns (state dict, stats dict)."""
    desc, state, gas = _prep(case)
    n_sub = case["n_sub"] if n_sub is None else n_sub
    chat = case["chat"] if chat is None else chat
    dt = case["dt"] if dt is None else dt
    p = params(desc)
    st = OrcStats()
    rc = lib().orc_subcycles(ctypes.byref(p), int(n_sub), float(chat), float(dt),
                             _dp(state["E"]), _dp(state["Fx"]), _dp(state["Fy"]), _dp(state["Fz"]),
                             _dp(state["T"]), *[_dp(gas[k]) for k in _GAS], ctypes.byref(st))
    if rc != 0:
        raise RuntimeError(f"orc_subcycles failed with {rc}")
    return state, st.as_dict()


def subcycle_box(case, lo, hi, chat=None, dt=None):
    """One subcycle of the oracle restricted to the interior box [lo, hi) (x, y, z order)."""
    desc, state, gas = _prep(case)
    chat = case["chat"] if chat is None else chat
    dt = case["dt"] if dt is None else dt
    p = params(desc)
    st = OrcStats()
    lo_a = (_c_int * 3)(*[int(v) for v in lo])
    hi_a = (_c_int * 3)(*[int(v) for v in hi])
    rc = lib().orc_subcycle_box(ctypes.byref(p), float(chat), float(dt), lo_a, hi_a,
                                _dp(state["E"]), _dp(state["Fx"]), _dp(state["Fy"]), _dp(state["Fz"]),
                                _dp(state["T"]), *[_dp(gas[k]) for k in _GAS], ctypes.byref(st))
    if rc != 0:
        raise RuntimeError(f"orc_subcycle_box failed with {rc}")
    return state, st.as_dict()


def num_threads():
    return lib().orc_num_threads()
