"""ctypes binding of librhd.so (argument marshalling only; every step of the radiation subcycle runs
in the library's CUDA kernels).

The functions keep the C names (rhd_init_grid, rhd_set_gas_state, rhd_radiation_subcycle, ...)
through `lib()`, and the classes Grid and Ensemble wrap a context.  Arrays may be numpy float64
arrays or torch tensors: CUDA tensors are passed as device pointers (on_device = 1), CPU tensors
(pinned or not) as host pointers.  There is no CPU fallback: if the library is missing the import
of a context raises.
"""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librhd.so")
# the same library with bounds-checked kernels (rhd_bounds_checked() = 1); pass it to lib() first
DEBUG_LIB_PATH = os.path.join(_HERE, "librhd_debug.so")

OK, ERR_ARG, ERR_STATE, ERR_CUDA, ERR_OOM, ERR_CFL, ERR_NONFINITE, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_BOUNDS = range(10)
STATUS_NAMES = {0: "RHD_OK", 1: "RHD_ERR_ARG", 2: "RHD_ERR_STATE", 3: "RHD_ERR_CUDA", 4: "RHD_ERR_OOM",
                5: "RHD_ERR_CFL", 6: "RHD_ERR_NONFINITE", 7: "RHD_ERR_TIMEOUT", 8: "RHD_ERR_UNSUPPORTED",
                9: "RHD_ERR_BOUNDS"}
BC = {"periodic": 0, "outflow": 1, "reflect": 2, "dirichlet": 3}
EXCHANGE = {"full": 0, "absorb": 1, "equilibrium": 2, "frozen_t": 3, "linear": 4}
LIMITER = {"minmod": 0, "mc": 1, "none": 2}
CLOSURE = {"m1": 0, "p1": 1}
SPEEDS = {"m1": 0, "fixed": 1}
PRECISION = {"fp64": 0, "split": 1}
FLAG_NO_GRAPH = 1
FLAG_SPLIT_FUSED = 2
FLAG_AUTOTUNE = 4
FLAG_EXCHANGE_ON_GAS_STEP = 8
VARIANT = {"fused": 0, "twopass": 1}
STAGING = {"cpasync": 0, "tma": 1}


class RhdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class GridDesc(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int * 3),
        ("dx", ctypes.c_double * 3),
        ("bc_lo", ctypes.c_int * 3),
        ("bc_hi", ctypes.c_int * 3),
        ("c", ctypes.c_double),
        ("a_rad", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("mu_over_kB", ctypes.c_double),
        ("theta_F", ctypes.c_double),
        ("theta_E", ctypes.c_double),
        ("E_floor", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("exchange", ctypes.c_int),
        ("beta_tau", ctypes.c_int),
        ("limiter", ctypes.c_int),
        ("closure", ctypes.c_int),
        ("speeds", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("flags", ctypes.c_int),
        ("z_chunk", ctypes.c_int),
        ("kappa_P", ctypes.c_double),
        ("kappa_F", ctypes.c_double),
        ("kappa_rho_pow", ctypes.c_int),
        ("cuda_stream", ctypes.c_void_p),
        ("linear_eps", ctypes.c_double),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("n_subcycles", ctypes.c_int64),
        ("n_realizability_fix", ctypes.c_int64),
        ("n_face_fallback", ctypes.c_int64),
        ("n_theta_fallback", ctypes.c_int64),
        ("n_newton_fallback", ctypes.c_int64),
        ("n_nonfinite", ctypes.c_int64),
        ("newton_iter_max", ctypes.c_int32),
        ("wait_timeouts", ctypes.c_int32),
        ("sum_E", ctypes.c_double),
        ("sum_F", ctypes.c_double * 3),
        ("max_f", ctypes.c_double),
        ("bounds_violations", ctypes.c_int64),
        ("gas_energy_floors", ctypes.c_int64),
        ("gas_nonfinite", ctypes.c_int64),
    ]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "sum_F"}
        d["sum_F"] = tuple(self.sum_F)
        return d


class LaunchConfig(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int),
                ("z_chunk", ctypes.c_int), ("staging", ctypes.c_int), ("ms_per_subcycle", ctypes.c_double)]

    def as_dict(self):
        inv_v = {v: k for k, v in VARIANT.items()}
        inv_s = {v: k for k, v in STAGING.items()}
        return {"variant": inv_v.get(self.variant, self.variant), "tile": (self.tile_x, self.tile_y),
                "z_chunk": self.z_chunk, "staging": inv_s.get(self.staging, self.staging),
                "ms_per_subcycle": self.ms_per_subcycle}

    @classmethod
    def from_dict(cls, d):
        return cls(VARIANT[d["variant"]] if isinstance(d["variant"], str) else int(d["variant"]),
                   int(d["tile"][0]), int(d["tile"][1]), int(d["z_chunk"]),
                   STAGING[d["staging"]] if isinstance(d["staging"], str) else int(d["staging"]), -1.0)


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double),
                ("alg_bytes_per_launch", ctypes.c_double)]


_TUNE_CAP = 64


def _kernel_times(ctx):
    out = (KernelTime * 16)()
    n = ctypes.c_int(0)
    _check(ctx, lib().rhd_get_kernel_times(ctx, out, 16, ctypes.byref(n)))
    return {out[i].name.decode(): {"launches": int(out[i].launches), "total_ms": float(out[i].total_ms),
                                   "alg_bytes_per_launch": float(out[i].alg_bytes_per_launch)}
            for i in range(min(n.value, 16))}


def _tune_result(fn, *args):
    table = (LaunchConfig * _TUNE_CAP)()
    n = ctypes.c_int(0)
    chosen = LaunchConfig()
    st = fn(*args, table, _TUNE_CAP, ctypes.byref(n), ctypes.byref(chosen))
    return st, chosen.as_dict(), [table[i].as_dict() for i in range(min(n.value, _TUNE_CAP))]


# the entry points declared in include/rhd.h, with their ctypes signatures
_P = ctypes.c_void_p
_CTXP = ctypes.POINTER(ctypes.c_void_p)
_SIGS = {
    "rhd_init_grid": (ctypes.c_int, [_CTXP, ctypes.POINTER(GridDesc)]),
    "rhd_set_gas_state": (ctypes.c_int, [_P] + [_P] * 8 + [ctypes.c_int]),
    "rhd_set_moments": (ctypes.c_int, [_P] + [_P] * 4 + [ctypes.c_int]),
    "rhd_set_dirichlet": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "rhd_radiation_subcycle": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, ctypes.c_double]),
    "rhd_gas_step": (ctypes.c_int, [_P, ctypes.c_double]),
    "rhd_gas_correct": (ctypes.c_int, [_P]),
    "rhd_gas_exchange": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_double]),
    "rhd_set_wait_limit": (ctypes.c_int, [_P, ctypes.c_longlong]),
    "rhd_get_gas": (ctypes.c_int, [_P] + [_P] * 5 + [ctypes.c_int]),
    "rhd_get_moments": (ctypes.c_int, [_P] + [_P] * 4 + [ctypes.c_int]),
    "rhd_set_conserved": (ctypes.c_int, [_P] + [_P] * 4 + [ctypes.c_int]),
    "rhd_get_conserved": (ctypes.c_int, [_P] + [_P] * 4 + [ctypes.c_int]),
    "rhd_get_gas_state": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "rhd_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(Stats)]),
    "rhd_reset_stats": (ctypes.c_int, [_P]),
    "rhd_synchronize": (ctypes.c_int, [_P, ctypes.c_int]),
    "rhd_last_error": (ctypes.c_char_p, [_P]),
    "rhd_destroy": (ctypes.c_int, [_P]),
    "rhd_ensemble_create": (ctypes.c_int, [_CTXP, ctypes.c_int, ctypes.POINTER(GridDesc)]),
    "rhd_ensemble_set_gas_state": (ctypes.c_int, [_P, ctypes.c_int] + [_P] * 8 + [ctypes.c_int]),
    "rhd_ensemble_set_moments": (ctypes.c_int, [_P, ctypes.c_int] + [_P] * 4 + [ctypes.c_int]),
    "rhd_ensemble_get_moments": (ctypes.c_int, [_P, ctypes.c_int] + [_P] * 4 + [ctypes.c_int]),
    "rhd_ensemble_get_gas_state": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int]),
    "rhd_ensemble_subcycle": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
    "rhd_subcycle_noalloc": (ctypes.c_int, [ctypes.POINTER(GridDesc), ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                            ctypes.c_double, ctypes.c_double] + [_P] * 17 + [ctypes.POINTER(Stats)]),
    "rhd_autotune": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.POINTER(LaunchConfig),
                                    ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(LaunchConfig)]),
    "rhd_ensemble_autotune": (ctypes.c_int, [_P, ctypes.c_double, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                             ctypes.POINTER(LaunchConfig), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                             ctypes.POINTER(LaunchConfig)]),
    "rhd_get_launch_config": (ctypes.c_int, [_P, ctypes.POINTER(LaunchConfig)]),
    "rhd_set_launch_config": (ctypes.c_int, [_P, ctypes.POINTER(LaunchConfig)]),
    "rhd_set_kernel_timing": (ctypes.c_int, [_P, ctypes.c_int]),
    "rhd_get_kernel_times": (ctypes.c_int, [_P, ctypes.POINTER(KernelTime), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "rhd_max_signal_speed": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "rhd_max_optical_depth": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "rhd_suggest_chat": (ctypes.c_int, [ctypes.c_double] * 4 + [ctypes.POINTER(ctypes.c_double)]),
    "rhd_time_steps": (ctypes.c_int, [ctypes.c_double] * 4 + [ctypes.POINTER(ctypes.c_double)] * 2
                       + [ctypes.POINTER(ctypes.c_int)]),
    "rhd_subcycle_steps": (ctypes.c_int, [ctypes.c_double] * 4 + [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]),
    "rhd_bounds_checked": (ctypes.c_int, []),
    "rhd_marshak_boundary": (ctypes.c_int, [ctypes.c_double] * 4 + [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "rhd_marshak_advance": (ctypes.c_int, [_P, ctypes.c_int] + [ctypes.c_double] * 6 + [ctypes.c_int]),
    "rhd_abi_version": (ctypes.c_int, []),
    "rhd_built_arch": (ctypes.c_int, []),
}

_lib = None


def lib(path: str | None = None):
    """Load librhd.so (built in-tree by paper_1306_0010_gb300.build); raises if it is missing."""
    global _lib
    if _lib is None:
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"librhd.so not found at {p}: build it with paper_1306_0010_gb300.build.build()")
        L = ctypes.CDLL(p)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(ctx, st):
    if st != OK:
        msg = lib().rhd_last_error(ctx)
        raise RhdError(st, msg.decode() if msg else "")


def desc_struct(d: dict, stream=None) -> GridDesc:
    s = GridDesc()
    for k in range(3):
        s.n[k] = int(d["n"][k])
        s.dx[k] = float(d["dx"][k])
        s.bc_lo[k] = BC[d["bc_lo"][k]]
        s.bc_hi[k] = BC[d["bc_hi"][k]]
    s.c = d["c"]
    s.a_rad = d["a_rad"]
    s.gamma = d["gamma"]
    s.mu_over_kB = d["mu_over_kB"]
    s.theta_F = d["theta_F"]
    s.theta_E = d["theta_E"]
    s.E_floor = d["E_floor"]
    s.cfl = d.get("cfl", 0.4)
    s.exchange = EXCHANGE[d["exchange"]]
    s.beta_tau = int(bool(d["beta_tau"]))
    s.limiter = LIMITER[d["limiter"]]
    s.closure = CLOSURE[d["closure"]]
    s.speeds = SPEEDS[d["speeds"]]
    s.precision = PRECISION[d.get("precision", "fp64")]
    s.flags = int(d.get("flags", 0))
    s.z_chunk = int(d.get("z_chunk", 0))
    s.kappa_P = d["kappa_P"]
    s.kappa_F = d["kappa_F"]
    s.kappa_rho_pow = int(d["kappa_rho_pow"])
    s.cuda_stream = stream
    s.linear_eps = float(d.get("linear_eps", 1.0))
    return s


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x, n, writable=False):
    """(pointer, on_device) of an FP64 array of n elements; None -> NULL."""
    if x is None:
        return None, 0
    if _is_torch(x):
        import torch

        if x.dtype != torch.float64 or not x.is_contiguous() or x.numel() != n:
            raise ValueError("tensors must be contiguous float64 with one value per cell")
        return ctypes.c_void_p(x.data_ptr()), int(x.is_cuda)
    if not isinstance(x, np.ndarray) or x.dtype != np.float64 or not x.flags["C_CONTIGUOUS"] or x.size != n:
        raise ValueError("arrays must be C-contiguous float64 with one value per cell")
    if writable and not x.flags["WRITEABLE"]:
        raise ValueError("output array is read-only")
    return ctypes.c_void_p(x.ctypes.data), 0


def _same_residency(ptrs):
    flags = {od for p, od in ptrs if p is not None}
    if len(flags) > 1:
        raise ValueError("mix of host and device arrays in one call")
    return flags.pop() if flags else 0


class Grid:
    """One grid: rhd_init_grid ... rhd_destroy."""

    def __init__(self, desc: dict, stream=None):
        self.desc = dict(desc)
        self.n = tuple(int(v) for v in desc["n"])
        self.ncell = self.n[0] * self.n[1] * self.n[2]
        self._ctx = ctypes.c_void_p()
        self._desc = desc_struct(desc, stream)
        st = lib().rhd_init_grid(ctypes.byref(self._ctx), ctypes.byref(self._desc))
        _check(None, st)

    @property
    def shape(self):
        return (self.n[2], self.n[1], self.n[0])

    def close(self):
        if self._ctx:
            lib().rhd_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    _GAS_KEYS = ("rho", "T", "vx", "vy", "vz", "kP", "kF", "j")

    def set_gas_state(self, rho, T, vx=None, vy=None, vz=None, kP=None, kF=None, j=None):
        # references to the frozen gas inputs, for checkpoint() (T evolves and is read back from the device)
        self._gas_in = dict(zip(self._GAS_KEYS, (rho, T, vx, vy, vz, kP, kF, j)))
        self._set_gas_state(rho, T, vx, vy, vz, kP, kF, j)
        self._gas_stepped = self._gas_pending = False

    def _set_gas_state(self, rho, T, vx=None, vy=None, vz=None, kP=None, kF=None, j=None):
        ps = [_ptr(a, self.ncell) for a in (rho, T, vx, vy, vz, kP, kF, j)]
        od = _same_residency(ps)
        _check(self._ctx, lib().rhd_set_gas_state(self._ctx, *[p for p, _ in ps], od))

    def set_moments(self, E, Fx, Fy, Fz):
        ps = [_ptr(a, self.ncell) for a in (E, Fx, Fy, Fz)]
        od = _same_residency(ps)
        _check(self._ctx, lib().rhd_set_moments(self._ctx, *[p for p, _ in ps], od))

    def set_dirichlet(self, face, state):
        arr = (ctypes.c_double * 4)(*[float(v) for v in state])
        _check(self._ctx, lib().rhd_set_dirichlet(self._ctx, int(face), arr))

    def radiation_subcycle(self, n_sub, chat, dt):
        _check(self._ctx, lib().rhd_radiation_subcycle(self._ctx, int(n_sub), float(chat), float(dt)))

    def gas_step(self, dt_gas):
        """The gas half of a cycle (Section 3.1 step 3): one van Leer step of the gas with the explicit gas
        sources, the radiation held at its current state; leaves the source correction pending."""
        _check(self._ctx, lib().rhd_gas_step(self._ctx, float(dt_gas)))
        self._gas_stepped = self._gas_pending = True

    def gas_exchange(self, dt_gas, chat):
        """Section 3.1 step 2 with the paper's placement of the stiff exchange (grids with
        FLAG_EXCHANGE_ON_GAS_STEP): the FULL energy exchange integrated once over dt_gas in every cell."""
        _check(self._ctx, lib().rhd_gas_exchange(self._ctx, float(dt_gas), float(chat)))

    def gas_correct(self):
        """Section 3.1 step 6: the pending gas step's sources corrected with the current radiation."""
        _check(self._ctx, lib().rhd_gas_correct(self._ctx))
        self._gas_pending = False

    def gas_cycle(self, chat, cfl=None, ratio=None, dt_gas=None):
        """One whole cycle of Section 3.1: time steps (unless dt_gas is given: then the subcycles are
        the fewest of length <= cfl min(dx) / chat spanning it), on grids with FLAG_EXCHANGE_ON_GAS_STEP
        the energy exchange over dt_gas (step 2), the gas step, the radiation subcycles over dt_gas, the
        source correction.  Returns (dt_gas, n_sub)."""
        cfl = self.desc.get("cfl", 0.4) if cfl is None else cfl
        dxm = min(self.desc["dx"][d] for d in range(3) if self.desc["n"][d] > 1)
        if dt_gas is None:
            dt_gas, dt_rad, n_sub = time_steps(cfl, dxm, self.max_signal_speed(), chat)
        else:
            dt_rad, n_sub = subcycle_steps(cfl, dxm, chat, dt_gas)
        if int(self.desc.get("flags", 0)) & FLAG_EXCHANGE_ON_GAS_STEP:
            self.gas_exchange(dt_gas, chat)
        self.gas_step(dt_gas)
        self.radiation_subcycle(n_sub, chat, dt_rad)
        self.gas_correct()
        return dt_gas, n_sub

    def get_gas(self):
        """The gas state: dict rho, vx, vy, vz, T (NumPy)."""
        out = {k: np.empty(self.shape) for k in ("rho", "vx", "vy", "vz", "T")}
        ps = [_ptr(out[k], self.ncell, writable=True)[0] for k in ("rho", "vx", "vy", "vz", "T")]
        _check(self._ctx, lib().rhd_get_gas(self._ctx, *ps, 0))
        return out

    def get_moments(self, E=None, Fx=None, Fy=None, Fz=None):
        if E is None:
            E, Fx, Fy, Fz = (np.empty(self.shape) for _ in range(4))
        ps = [_ptr(a, self.ncell, writable=True) for a in (E, Fx, Fy, Fz)]
        od = _same_residency(ps)
        _check(self._ctx, lib().rhd_get_moments(self._ctx, *[p for p, _ in ps], od))
        return {"E": E, "Fx": Fx, "Fy": Fy, "Fz": Fz}

    def marshak_advance(self, n_sub, chat, dt, t0, marshak, n_quad=1024):
        """n_sub subcycles of the non-equilibrium Marshak wave from time t0, the low x face's state set on
        the device before each from the Su & Olson surface value at the subcycle's midpoint tau."""
        _check(self._ctx, lib().rhd_marshak_advance(self._ctx, int(n_sub), float(chat), float(dt), float(t0),
                                                    float(marshak["tau_rate"]), float(marshak["eps"]),
                                                    float(marshak["F_inc"]), int(n_quad)))

    def max_signal_speed(self):
        """v_max = max(|v| + c_eff) over the grid (Eq. algorithm:ceff), from the gas state and current E."""
        out = ctypes.c_double()
        _check(self._ctx, lib().rhd_max_signal_speed(self._ctx, ctypes.byref(out)))
        return out.value

    def max_optical_depth(self):
        """The largest optical depth sum(k_F dx) along any grid line parallel to an active axis."""
        out = ctypes.c_double()
        _check(self._ctx, lib().rhd_max_optical_depth(self._ctx, ctypes.byref(out)))
        return out.value

    def set_conserved(self, E, Gx, Gy, Gz):
        """Set the solver's own variables E and G = F/c (no conversion; see get_conserved)."""
        ps = [_ptr(a, self.ncell) for a in (E, Gx, Gy, Gz)]
        od = _same_residency(ps)
        _check(self._ctx, lib().rhd_set_conserved(self._ctx, *[p for p, _ in ps], od))

    def get_conserved(self, E=None, Gx=None, Gy=None, Gz=None):
        """The solver's own variables E and G = F/c, copied without arithmetic (bitwise restartable)."""
        if E is None:
            E, Gx, Gy, Gz = (np.empty(self.shape) for _ in range(4))
        ps = [_ptr(a, self.ncell, writable=True) for a in (E, Gx, Gy, Gz)]
        od = _same_residency(ps)
        _check(self._ctx, lib().rhd_get_conserved(self._ctx, *[p for p, _ in ps], od))
        return {"E": E, "Gx": Gx, "Gy": Gy, "Gz": Gz}

    def get_gas_state(self, T=None):
        if T is None:
            T = np.empty(self.shape)
        p, od = _ptr(T, self.ncell, writable=True)
        _check(self._ctx, lib().rhd_get_gas_state(self._ctx, p, od))
        return T

    def get_stats(self, allow_nonfinite=False):
        s = Stats()
        st = lib().rhd_get_stats(self._ctx, ctypes.byref(s))
        if not (allow_nonfinite and st == ERR_NONFINITE):
            _check(self._ctx, st)
        return s.as_dict()

    def reset_stats(self):
        _check(self._ctx, lib().rhd_reset_stats(self._ctx))

    def synchronize(self, timeout_ms=-1):
        _check(self._ctx, lib().rhd_synchronize(self._ctx, int(timeout_ms)))

    def autotune(self, chat, dt, reps=3):
        """Time every candidate launch configuration on the current state and keep the fastest;
        returns (chosen, table) as dicts (see rhd_autotune)."""
        st, chosen, table = _tune_result(lib().rhd_autotune, self._ctx, float(chat), float(dt), int(reps))
        _check(self._ctx, st)
        return chosen, table

    def launch_config(self):
        c = LaunchConfig()
        _check(self._ctx, lib().rhd_get_launch_config(self._ctx, ctypes.byref(c)))
        return c.as_dict()

    def set_kernel_timing(self, enable=True):
        """Bracket every kernel with CUDA events (plain launches while on); see kernel_times()."""
        _check(self._ctx, lib().rhd_set_kernel_timing(self._ctx, int(bool(enable))))

    def kernel_times(self):
        """{kernel name: {launches, total_ms, alg_bytes_per_launch}} since the timer was enabled or last read."""
        return _kernel_times(self._ctx)

    def set_wait_limit(self, polls):
        """Poll limit of the two-pass corrector's TMA plane waits (polls < 0: the default; 0: give up at
        once, for tests of the timeout path)."""
        _check(self._ctx, lib().rhd_set_wait_limit(self._ctx, int(polls)))

    def set_launch_config(self, cfg: dict):
        c = LaunchConfig.from_dict(cfg)
        _check(self._ctx, lib().rhd_set_launch_config(self._ctx, ctypes.byref(c)))

    def checkpoint(self, path):
        """Save the evolving state (E, G = F/c, T), the descriptor, the launch configuration and the frozen
        gas inputs last given to set_gas_state (as they are at this call) to an .npz file;
        Grid.restore(path) continues bit for bit."""
        if getattr(self, "_gas_pending", False):
            raise RhdError(ERR_STATE, "a gas step waits for its source correction: checkpoint after gas_correct")
        out = self.get_conserved()
        out["T_state"] = self.get_gas_state()
        for k, v in getattr(self, "_gas_in", {}).items():
            if v is not None and k != "T":
                out["gas_" + k] = v.detach().cpu().numpy() if _is_torch(v) else np.asarray(v)
        if getattr(self, "_gas_stepped", False):
            # the gas steps moved rho and v away from the inputs: save the current state
            gas = self.get_gas()
            for k in ("rho", "vx", "vy", "vz"):
                out["gas_" + k] = gas[k]
        cfg = self.launch_config()
        np.savez(path, desc=np.array(json.dumps(self.desc, default=float)),
                 launch=np.array(json.dumps(dict(cfg, tile=list(cfg["tile"])))), **out)

    @classmethod
    def restore(cls, path, stream=None):
        """A new Grid in the state a checkpoint() saved (same launch configuration)."""
        z = np.load(path)
        desc = json.loads(str(z["desc"]))
        g = cls(desc, stream=stream)
        cfg = json.loads(str(z["launch"]))
        g.set_launch_config(dict(cfg, tile=tuple(cfg["tile"])))
        gas = {k: (np.ascontiguousarray(z["gas_" + k]) if "gas_" + k in z else None) for k in cls._GAS_KEYS}
        gas["T"] = np.ascontiguousarray(z["T_state"])
        g.set_gas_state(*(gas[k] for k in cls._GAS_KEYS))
        g.set_conserved(*(np.ascontiguousarray(z[k]) for k in ("E", "Gx", "Gy", "Gz")))
        g._set_dirichlet_from_desc(desc)
        return g

    def _set_dirichlet_from_desc(self, d):
        for face in range(6):
            dd, side = face // 2, face % 2
            if (d["bc_hi"] if side else d["bc_lo"])[dd] == "dirichlet":
                self.set_dirichlet(face, (d["dirichlet_hi"] if side else d["dirichlet_lo"])[dd])

    def load_case(self, case):
        """Set the gas state and moments of a case dict (see workloads.py)."""
        f = case["fields"]
        self.set_gas_state(*(None if f.get(k) is None else np.ascontiguousarray(f[k], dtype=np.float64)
                             for k in ("rho", "T", "vx", "vy", "vz", "kP", "kF", "j")))
        self.set_moments(*(np.ascontiguousarray(f[k], dtype=np.float64) for k in ("E", "Fx", "Fy", "Fz")))
        self._set_dirichlet_from_desc(case["desc"])


class Ensemble:
    """Many independent grids advanced by one persistent launch per subcycle."""

    def __init__(self, descs, stream=None):
        self.descs = [dict(d) for d in descs]
        self.shapes = [(int(d["n"][2]), int(d["n"][1]), int(d["n"][0])) for d in descs]
        arr = (GridDesc * len(descs))(*[desc_struct(d, stream) for d in descs])
        self._keep = arr
        self._ctx = ctypes.c_void_p()
        _check(None, lib().rhd_ensemble_create(ctypes.byref(self._ctx), len(descs), arr))

    def close(self):
        if self._ctx:
            lib().rhd_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _n(self, g):
        s = self.shapes[g]
        return s[0] * s[1] * s[2]

    def set_gas_state(self, g, rho, T, vx=None, vy=None, vz=None, kP=None, kF=None, j=None):
        ps = [_ptr(a, self._n(g)) for a in (rho, T, vx, vy, vz, kP, kF, j)]
        od = _same_residency(ps)
        _check(self._ctx, lib().rhd_ensemble_set_gas_state(self._ctx, int(g), *[p for p, _ in ps], od))

    def set_moments(self, g, E, Fx, Fy, Fz):
        ps = [_ptr(a, self._n(g)) for a in (E, Fx, Fy, Fz)]
        od = _same_residency(ps)
        _check(self._ctx, lib().rhd_ensemble_set_moments(self._ctx, int(g), *[p for p, _ in ps], od))

    def get_moments(self, g, E=None, Fx=None, Fy=None, Fz=None):
        if E is None:
            E, Fx, Fy, Fz = (np.empty(self.shapes[g]) for _ in range(4))
        ps = [_ptr(a, self._n(g), writable=True) for a in (E, Fx, Fy, Fz)]
        od = _same_residency(ps)
        _check(self._ctx, lib().rhd_ensemble_get_moments(self._ctx, int(g), *[p for p, _ in ps], od))
        return {"E": E, "Fx": Fx, "Fy": Fy, "Fz": Fz}

    def get_gas_state(self, g, T=None):
        if T is None:
            T = np.empty(self.shapes[g])
        p, od = _ptr(T, self._n(g), writable=True)
        _check(self._ctx, lib().rhd_ensemble_get_gas_state(self._ctx, int(g), p, od))
        return T

    def subcycle(self, n_sub, chat, dts):
        arr = (ctypes.c_double * len(dts))(*[float(v) for v in dts])
        _check(self._ctx, lib().rhd_ensemble_subcycle(self._ctx, int(n_sub), float(chat), arr))

    def autotune(self, chat, dts, reps=3):
        arr = (ctypes.c_double * len(dts))(*[float(v) for v in dts])
        st, chosen, table = _tune_result(lib().rhd_ensemble_autotune, self._ctx, float(chat), arr, int(reps))
        _check(self._ctx, st)
        return chosen, table

    def launch_config(self):
        c = LaunchConfig()
        _check(self._ctx, lib().rhd_get_launch_config(self._ctx, ctypes.byref(c)))
        return c.as_dict()

    def set_kernel_timing(self, enable=True):
        _check(self._ctx, lib().rhd_set_kernel_timing(self._ctx, int(bool(enable))))

    def kernel_times(self):
        return _kernel_times(self._ctx)

    def get_stats(self, allow_nonfinite=False):
        s = Stats()
        st = lib().rhd_get_stats(self._ctx, ctypes.byref(s))
        if not (allow_nonfinite and st == ERR_NONFINITE):
            _check(self._ctx, st)
        return s.as_dict()

    def reset_stats(self):
        _check(self._ctx, lib().rhd_reset_stats(self._ctx))

    def synchronize(self, timeout_ms=-1):
        _check(self._ctx, lib().rhd_synchronize(self._ctx, int(timeout_ms)))

    def load_case(self, g, case):
        f = case["fields"]
        self.set_gas_state(g, *(None if f.get(k) is None else np.ascontiguousarray(f[k], dtype=np.float64)
                                for k in ("rho", "T", "vx", "vy", "vz", "kP", "kF", "j")))
        self.set_moments(g, *(np.ascontiguousarray(f[k], dtype=np.float64) for k in ("E", "Fx", "Fy", "Fz")))


NOALLOC_MAX_CELLS = 1048576


def subcycle_noalloc(desc: dict, n_sub, chat, dt, E, Fx, Fy, Fz, rho, T, E_out, Fx_out, Fy_out, Fz_out, T_out,
                     vx=None, vy=None, vz=None, kP=None, kF=None, j=None, stream=None, want_stats=True):
    """rhd_subcycle_noalloc: n_sub FP64 subcycles on caller-owned device arrays (torch CUDA tensors)
    with no device allocation by the library (for callers that cannot allocate)."""
    n = int(desc["n"][0]) * int(desc["n"][1]) * int(desc["n"][2])
    ins = [E, Fx, Fy, Fz, rho, T, vx, vy, vz, kP, kF, j, E_out, Fx_out, Fy_out, Fz_out, T_out]
    ps = [_ptr(a, n, writable=(i >= 12)) for i, a in enumerate(ins)]
    if any(p is not None and not od for p, od in ps):
        raise ValueError("rhd_subcycle_noalloc takes device arrays only")
    d = desc_struct(desc, stream)
    dirs = None
    if any(b == "dirichlet" for b in list(desc["bc_lo"]) + list(desc["bc_hi"])):
        vals = []
        for f in range(6):
            dd, side = f // 2, f % 2
            vals += [float(v) for v in (desc["dirichlet_hi"] if side else desc["dirichlet_lo"])[dd]]
        dirs = (ctypes.c_double * 24)(*vals)
    st = Stats()
    status = lib().rhd_subcycle_noalloc(ctypes.byref(d), dirs, int(n_sub), float(chat), float(dt),
                                        *[p for p, _ in ps], ctypes.byref(st) if want_stats else None)
    _check(None, status)
    return st.as_dict() if want_stats else None


def suggest_chat(c, v_max, tau_max, ratio=10.0):
    """chat = min(c, ratio v_max max(1, tau_max)) (Eq. rsla:staticdiffreq with 'much greater' as ratio)."""
    out = ctypes.c_double()
    _check(None, lib().rhd_suggest_chat(float(c), float(v_max), float(tau_max), float(ratio), ctypes.byref(out)))
    return out.value


def time_steps(cfl, dx_min, v_max, chat):
    """(dt_gas, dt_rad, n_sub) of one gas cycle (Eqs. algorithm:gastimestep and algorithm:radtimestep)."""
    dg, dr, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    _check(None, lib().rhd_time_steps(float(cfl), float(dx_min), float(v_max), float(chat), ctypes.byref(dg),
                                      ctypes.byref(dr), ctypes.byref(n)))
    return dg.value, dr.value, n.value


def subcycle_steps(cfl, dx_min, chat, dt_gas):
    """(dt_rad, n_sub): the fewest subcycles of length <= cfl dx_min / chat spanning dt_gas (Eq.
    algorithm:radtimestep)."""
    dr, n = ctypes.c_double(), ctypes.c_int()
    _check(None, lib().rhd_subcycle_steps(float(cfl), float(dx_min), float(chat), float(dt_gas), ctypes.byref(dr),
                                          ctypes.byref(n)))
    return dr.value, n.value


def marshak_boundary(tau, eps, F_inc, c, n_quad=4096):
    """(E, Fx, 0, 0) of the low x face of the Marshak wave at tau (Eqs. marshak:suolson, marshak:bc_ix1)."""
    out = (ctypes.c_double * 4)()
    _check(None, lib().rhd_marshak_boundary(float(tau), float(eps), float(F_inc), float(c), int(n_quad), out))
    return tuple(out)
