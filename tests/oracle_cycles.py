"""Whole Section 3.1 cycles on the oracle (test infrastructure): the gas step (oracle/gas.py), the
radiation subcycles that span it (oracle/rhd_oracle.c) with the new gas, and the source correction."""
import math

import numpy as np

from oracle import gas as ogas
from oracle import oracle as orc


def gas_time_step(desc, gas, cfl):
    """Delta t_gas = cfl min(dx) / max(|v| + a) (Eq. algorithm:gastimestep without the radiation term)."""
    dxm = min(desc["dx"][d] for d in range(3) if desc["n"][d] > 1)
    a = np.sqrt(desc["gamma"] * gas["T"] / desc["mu_over_kB"])
    speed = np.sqrt(gas["vx"] ** 2 + gas["vy"] ** 2 + gas["vz"] ** 2) + a
    return cfl * dxm / float(np.max(speed))


def run_cycles(case, t_end, cfl=0.4, exchange_on_gas_step=False, dt_fixed=None):
    """Advance case["fields"] to t_end by cycles of Delta t_gas (last one shortened; dt_fixed: that
    length instead of the Courant step), each with the fewest subcycles of length <= cfl min(dx) / chat.
    exchange_on_gas_step: the FULL exchange runs once per cycle over Delta t_gas before the gas step
    (Section 3.1 step 2) and not in the subcycles.  Returns (gas dict, radiation dict, number of
    cycles)."""
    desc, chat = case["desc"], case["chat"]
    sub_desc = dict(desc, exchange="equilibrium") if exchange_on_gas_step else desc
    f = case["fields"]
    gas = {k: f[k] for k in ("rho", "vx", "vy", "vz", "T", "kF")}
    rad = {k: f[k] for k in ("E", "Fx", "Fy", "Fz")}
    dxm = min(desc["dx"][d] for d in range(3) if desc["n"][d] > 1)
    t, n = 0.0, 0
    while t < t_end * (1 - 1e-12):
        dt = min(gas_time_step(desc, gas, cfl) if dt_fixed is None else dt_fixed, t_end - t)
        n_sub = max(1, math.ceil(dt / (cfl * dxm / chat) * (1 - 1e-12)))
        if exchange_on_gas_step:
            gas, rad, _ = ogas.gas_exchange(desc, dict(gas, kP=f.get("kP")), rad, dt, chat)
        g1, pend, _ = ogas.gas_step(desc, gas, rad, dt)
        fields = dict(rad, T=g1["T"], rho=g1["rho"], vx=g1["vx"], vy=g1["vy"], vz=g1["vz"], kP=f.get("kP"),
                      kF=f.get("kF"), j=f.get("j"))
        r1, _ = orc.subcycles({"desc": sub_desc, "fields": fields, "chat": chat, "dt": dt / n_sub, "n_sub": n_sub})
        rad = {k: r1[k] for k in ("E", "Fx", "Fy", "Fz")}
        gas, _ = ogas.gas_correct(desc, dict(g1, T=r1["T"], kF=f.get("kF")), pend, rad)
        gas["kF"] = f.get("kF")
        t += dt
        n += 1
    return gas, rad, n
