"""Error bound of the split path against the FP64 oracle, derived from the split path's arithmetic.

What is FP32 on the split path.  Per subcycle a cell's update is U^{m+1} = S(U^m + d): d is the FP32
increment of the transport (reconstruction, closure, wave speeds, HLL, flux divergence) and of the
explicit sources (O(beta tau) terms, emissivity); S is the stiff part (theta updates of F and E, the
energy exchange), evaluated in FP64 on the FP64 state U^m + d.  The FP32 copies of the gas inputs are
exact in the cases that use this bound for stiff gas (rounded to FP32 by the input recipe), and are
the path's own input rounding (relative 2^-23) otherwise.

Transport.  A face flux is a chain of FP32 operations on values of the flux's own size (at most
chat max E per component): the truncated FP32 copy of the state, the limited slope and face value, the
closure (|G|^2, f^2, s = sqrt(4 - 3 f^2), the coefficients of P = a I + b G G^T), the wave speeds, the
HLL combination.  C_F = 32 counts those roundings, each of at most u = 2^-24 relative, with the MUFU
square root and reciprocal (about 2 ulp each) counted twice.  The divergence weighs each of the 2 D
faces of a D-dimensional cell by dt/dx, i.e. by CFL / chat with CFL = chat dt / min(dx).  The explicit
sources and the final rounding of d add C_S = 8 roundings of values of size at most max|U| (the
O(beta tau) terms are small by the paper's assumption beta tau << 1, Sec. 3.4).  So per subcycle
|delta d| <= (2 D CFL C_F + C_S) u max|E| (and c max|E| for F).

Stiff part.  The theta factors of F and E are FP64 (1 - (1 - theta) x)/(1 + theta x) <= 1 and the
exchange is a contraction in E: E^{n+1} = E + x (a_R M - E)/(1 + theta x) at its root, so
|dE^{n+1}/dE_in| <= 1 and the transport error is not amplified.  In particular it is not amplified by
the gas-to-radiation energy ratio K = e / ((c/chat) E): an exchange solved in FP32 for e^{n+1} and
then E = (chat/c)(Ebar - e^{n+1}) (Eq. source:eradupdate) would lose about K u in E per subcycle, while
the FP64 Newton step from the FP32 seed leaves at most 6 (s/T)^2 a_R T^4 + 12 u^2 max(E, a_R T^4) with
|s| <= 2^-22 T (its stopping rule), i.e. C_X u^2 with C_X = 128 per subcycle, independent of K.

Errors add over subcycles: the theta factors and the exchange are contractions, and the transport is
stable at CFL <= 0.4, so an error made in one subcycle is carried by the later ones, not amplified (an
assumption of the bound for the limited second-order scheme, whose L-infinity stability is not proved
for unsplit 3D updates).  After n_sub subcycles
the normwise L-infinity error of E (by max|E|), F (by c max|E|) and T (by max|T|, through
dT = dE / (4 a_R T^3) near radiative equilibrium) is at most

    n_sub ((2 D CFL C_F + C_S) u + C_X u^2).

This is a worst-case bound; the measured errors are one to two orders of magnitude below it, because
the rounding errors are not all of one sign and most intermediate values are below the flux scale.
"""
U32 = 2.0 ** -24
C_F = 32
C_S = 8
C_X = 128


def active_dims(desc):
    return sum(1 for d in range(3) if desc["n"][d] > 1)


def cfl(case):
    desc = case["desc"]
    dxs = [desc["dx"][d] for d in range(3) if desc["n"][d] > 1] or [1.0]
    return case["chat"] * case["dt"] / min(dxs)


def per_subcycle(case):
    D = max(active_dims(case["desc"]), 1)
    return (2 * D * cfl(case) * C_F + C_S) * U32 + C_X * U32 ** 2


def split_bound(case, n_sub):
    """Normwise L-infinity bound of the split path against the oracle after n_sub subcycles."""
    return n_sub * per_subcycle(case)


def gas_energy_ratio(case):
    """K = e / ((c / chat) E), largest over the cells (the exchange's gas-to-radiation energy ratio)."""
    f, d = case["fields"], case["desc"]
    e = f["rho"] * f["T"] / ((d["gamma"] - 1.0) * d["mu_over_kB"])
    return float((e / ((d["c"] / case["chat"]) * f["E"])).max())
