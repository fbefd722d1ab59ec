"""High-precision (mpmath) statements of the paper's plain definitions, used by the CPU tests
to pin the oracle: prim->cons (Eq. primitive_to_conserved), the flux (Eq. srhd_flux) and
the two enthalpies (Sec. 2.2).  These are definitions evaluated exactly, not the oracle's
rearranged double-precision forms."""
import mpmath as mp

mp.mp.dps = 40


def enthalpy(eos, gamma_ad, rho, P):
    rho, P = mp.mpf(rho), mp.mpf(P)
    th = P / rho
    if eos == "ideal":
        g = mp.mpf(gamma_ad)
        return 1 + g / (g - 1) * th
    return mp.mpf(5) / 2 * th + mp.mpf(3) / 2 * mp.sqrt(th * th + mp.mpf(4) / 9)


def prim2cons(eos, gamma_ad, W):
    """W = (rho, vx, vy, vz, P) -> (D, Sx, Sy, Sz, tau) with tau = gamma^2 rho h - P - D."""
    rho, vx, vy, vz, P = (mp.mpf(float(x)) for x in W)
    lor = 1 / mp.sqrt(1 - (vx * vx + vy * vy + vz * vz))
    h = enthalpy(eos, gamma_ad, rho, P)
    D = lor * rho
    w = lor * lor * rho * h
    return [D, w * vx, w * vy, w * vz, w - P - D]


def flux(eos, gamma_ad, W, d):
    """Eq. srhd_flux along axis d in the variables (D, S, tau): (rho u_d, rho h u_d u + P e_d,
    gamma rho h u_d - rho u_d), u = gamma v."""
    rho, vx, vy, vz, P = (mp.mpf(float(x)) for x in W)
    v = [vx, vy, vz]
    lor = 1 / mp.sqrt(1 - (vx * vx + vy * vy + vz * vz))
    u = [lor * c for c in v]
    h = enthalpy(eos, gamma_ad, rho, P)
    F = [rho * u[d]]
    for k in range(3):
        F.append(rho * h * u[d] * u[k] + (P if k == d else 0))
    F.append(lor * rho * h * u[d] - rho * u[d])
    return F
