"""High-precision solution of case 4 of Theorem 3 (projection onto D K_exp), for pinning
the oracle.  The plain formulas of eqs. h_rho, sp_rd and vpvd_defn are evaluated in
mpmath at about 32 significant digits (more when an interval end is far from 0, so that
offsets of e^-|a| from it stay visible); rho = anchor + dir e^L is located by bisection
on L over the interval of eq. lrho_urho until L is settled to ~26 digits.  It shares
nothing with the oracle but the paper's definitions.  Module-level so that worker
processes (spawn) can import it."""
import numpy as np


def exp_case4(v, d, dps=32):
    import mpmath as mp
    f = [float(x) for x in v]
    g = [float(x) for x in d]
    span = 1.0
    if f[1] > 0:
        span = max(span, abs(f[0] * g[1] / (f[1] * g[0])))
    if f[0] > 0:
        span = max(span, abs(1.0 - f[1] * g[1] / (f[0] * g[0])))
    mp.mp.dps = int(dps + 1.3 * span)
    r0, s0, t0 = [mp.mpf(x) for x in f]
    dr, ds, dt = [mp.mpf(x) for x in g]
    tau2 = ds ** 2 / dr ** 2

    def parts(rho):
        den = tau2 + rho * (rho - 1)
        return ((s0 * ds / dr ** 2 - r0 * (1 - rho) / dr) / den,
                (ds ** 2 / dr * (r0 - dr / ds * rho * s0)) / den)

    def h(rho):
        sp, rd = parts(rho)
        return dt * mp.exp(rho) * sp - mp.exp(-rho) * rd / dt - t0

    a3 = r0 * ds / (s0 * dr) if s0 > 0 else None
    a4 = 1 - s0 * ds / (r0 * dr) if r0 > 0 else None
    if r0 > 0:
        anchor, direction = a4, (mp.sign(a3 - a4) if s0 > 0 else 1)
    else:
        anchor, direction = a3, -1

    def rho_of(L):
        return anchor + direction * mp.exp(L)

    if r0 > 0 and s0 > 0:
        hiL = mp.log(abs(a3 - a4)) - mp.mpf(10) ** -(mp.mp.dps - 5)
    else:
        hiL = mp.mpf(0)
        s_anchor = -1 if r0 > 0 else 1
        while mp.sign(h(rho_of(hiL))) == s_anchor:
            hiL = 2 * hiL + 1
    loL = -mp.mpf(3 * mp.mp.dps + 50)  # e^loL is below the working precision of rho
    s_lo = mp.sign(h(rho_of(loL)))
    tol = mp.mpf(10) ** -(dps - 6)
    while hiL - loL > tol:
        mid = (loL + hiL) / 2
        if mp.sign(h(rho_of(mid))) == s_lo:
            loL = mid
        else:
            hiL = mid
    rho = rho_of((loL + hiL) / 2)
    sp, _ = parts(rho)
    return np.array([float(dr * rho * sp), float(ds * sp), float(dt * mp.exp(rho) * sp)])


def exp_case4_rows(rows):
    """exp_case4 over a list of (v, d) pairs (one worker's share)."""
    return [exp_case4(v, d) for v, d in rows]
