"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the benchmark.

This module holds problem descriptions (mesh, equation of state, boundary
conditions, time integrator) and initial primitive fields as functions of the
node coordinates.  It holds none of the method's arithmetic: no
prim->cons map, no con2prim, no flux, no basis.  Each side computes its own
node coordinates and its own conserved state from the primitive fields given
here.

A problem description is a plain dict:
  dim, degree, n_elem, lo, hi, eos ('ideal' | 'tm'), gamma_ad,
  c2p ('analytic' | 'iterative' | 'default'), c2p_max_iter, flux ('llf' | 'hll' | 'hllc'),
  rk_stages, bc [(lo, hi) per dim: 'periodic' | 'dirichlet' | 'outflow' | 'reflect'],
  bc_state [[(rho, vx, vy, vz, P) low, high] per dim], enforce, cfl.

The workloads follow the problems of the paper:
  blast_wave      -- 1D relativistic blast wave (Sec. 4.2, problem 1)
  riemann_1d      -- 1D Riemann problems 2-5 of Sec. 4.2 (problem 5: a reflecting wall)
  riemann_2d      -- the three 2D Riemann problems of Sec. 4.4 (four quadrants)
  advected_wave   -- 2D smooth density wave, periodic (smooth convergence case)
  kh2d            -- 2D relativistic Kelvin-Helmholtz, double shear layer (Sec. 4.5 set-up
                     recast as periodic with two layers), Taub-Matthews EOS
  kh3d            -- 3D high-Lorentz-factor Kelvin-Helmholtz, Taub-Matthews EOS
  kh_single       -- the paper's own Kelvin-Helmholtz set-up (Sec. 4.5): one shear layer,
                     ideal EOS, outflow in y
  linear_wave     -- linear waves of Sec. 4.1 in grid-aligned and oblique periodic boxes
  e2_grid         -- the 25 x 25 (gamma, P) grid of the con2prim accuracy study (Sec. 3.3)
"""
from __future__ import annotations

import math

import numpy as np

KH3D_SEED = 2205000950


# --------------------------------------------------------------------------
# Problem descriptions
# --------------------------------------------------------------------------

def blast_wave(n: int = 128, degree: int = 1, p_left: float = 13.33, p_right: float = 1e-6,
               flux: str = "llf") -> dict:
    """1D blast wave on [0, 1], interface x = 0.5, Gamma = 5/3, Dirichlet ends, SSPRK2,
    CFL 0.2, to t = 0.4 (Sec. 4.2 problem 1 with pressures 13.33 and 1e-6)."""
    left = (10.0, 0.0, 0.0, 0.0, p_left)
    right = (1.0, 0.0, 0.0, 0.0, p_right)
    return dict(name="blast_wave_1d", dim=1, degree=degree, n_elem=[n], lo=[0.0], hi=[1.0],
                eos="ideal", gamma_ad=5.0 / 3.0, c2p="iterative", flux=flux, rk_stages=2,
                bc=[("dirichlet", "dirichlet")], bc_state=[[left, right]], enforce=True,
                cfl=0.2, t_final=0.4, left=left, right=right)


# The paper's 1D Riemann problems 2-5 (Sec. 4.2): primitive (rho, vx, vy, vz, P) left and
# right of x = 0.5, adiabatic index, final time, right-hand boundary.  Problem 5 is a uniform
# flow into a reflecting wall at x = 1.  (Problem 1 is `blast_wave`.)
RIEMANN_1D = {
    2: dict(left=(1.0, 0.0, 0.0, 0.0, 1e3), right=(1.0, 0.0, 0.0, 0.0, 1e-2), gamma_ad=5.0 / 3.0,
            t_final=0.4, right_bc="dirichlet"),
    3: dict(left=(1.0, 0.0, 0.0, 0.0, 1e3), right=(1.0, 0.0, 0.99, 0.0, 1e-2), gamma_ad=5.0 / 3.0,
            t_final=0.4, right_bc="dirichlet"),
    4: dict(left=(1.0, 0.01, 0.0, 0.0, 1.0), right=(0.125, 0.01, 0.0, 0.0, 0.1), gamma_ad=4.0 / 3.0,
            t_final=0.4, right_bc="dirichlet"),
    5: dict(left=(1.0, 0.99999, 0.0, 0.0, 0.01), right=(1.0, 0.99999, 0.0, 0.0, 0.01),
            gamma_ad=4.0 / 3.0, t_final=1.5, right_bc="reflect"),
}


# The paper's 2D Riemann problems (Sec. 4.4): primitive (rho, vx, vy, P) in the quadrants
# Q1 = [0,1]x[0,1], Q2 = [-1,0]x[0,1], Q3 = [-1,0]x[-1,0], Q4 = [0,1]x[-1,0].
RIEMANN_2D = {
    1: [(0.035145216124503, 0.0, 0.0, 0.162931056509027), (0.1, 0.7, 0.0, 1.0),
        (0.5, 0.0, 0.0, 1.0), (0.1, 0.0, 0.7, 1.0)],
    2: [(0.5, 0.5, -0.5, 5.0), (1.0, 0.5, 0.5, 5.0), (3.0, -0.5, 0.5, 5.0), (1.5, -0.5, -0.5, 5.0)],
    3: [(1.0, 0.0, 0.0, 1.0), (0.5771, -0.3529, 0.0, 0.4), (1.0, -0.3529, -0.3529, 1.0),
        (0.5771, 0.0, -0.3529, 0.4)],
}


def riemann_2d(test: int, n: int = 128, degree: int = 1, flux: str = "hllc",
               limiter: bool = True) -> dict:
    """2D Riemann problem `test` (1-3) of Sec. 4.4 on [-1,1]^2: ideal EOS Gamma = 5/3 with the
    iterative con2prim, transmissive (outflow) boundaries, HLLC and the limiter, to t = 0.8."""
    return dict(name="riemann_2d", test=test, dim=2, degree=degree, n_elem=[n, n],
                lo=[-1.0, -1.0], hi=[1.0, 1.0], eos="ideal", gamma_ad=5.0 / 3.0, c2p="iterative",
                flux=flux, rk_stages=min(degree + 1, 3), bc=[("outflow", "outflow")] * 2,
                enforce=True, limiter=limiter, cfl=0.2, t_final=0.8,
                quadrants=RIEMANN_2D[test])


def riemann_2d_ic(spec: dict, X):
    xp = _xp(X)
    x, y = X[0], X[1]
    Q = spec["quadrants"]
    right, top = x >= 0.0, y >= 0.0
    out = []
    for v in range(4):
        q1, q2, q3, q4 = (_const(x, Q[k][v]) for k in range(4))
        out.append(xp.where(top, xp.where(right, q1, q2), xp.where(right, q4, q3)))
    rho, vx, vy, P = out
    return xp.stack([rho, vx, vy, _const(x, 0.0), P])


def riemann_1d(problem: int, n: int = 128, degree: int = 1, flux: str = "hllc") -> dict:
    """1D Riemann problem `problem` (2-5) of Sec. 4.2 on [0, 1]: ideal EOS with the iterative
    con2prim, Dirichlet ends (problem 5: a reflecting wall at x = 1), SSP-RK with p + 1 stages
    (at most 3), CFL 0.2."""
    P = RIEMANN_1D[problem]
    left, right = P["left"], P["right"]
    return dict(name="riemann_1d", problem=problem, dim=1, degree=degree, n_elem=[n], lo=[0.0],
                hi=[1.0], eos="ideal", gamma_ad=P["gamma_ad"], c2p="iterative", flux=flux,
                rk_stages=min(degree + 1, 3), bc=[("dirichlet", P["right_bc"])],
                bc_state=[[left, right]], enforce=True, cfl=0.2, t_final=P["t_final"],
                left=left, right=right)


# The blast wave with relativistic temperature on the left and a non-relativistic one on the
# right (Sec. 4.3, the Taub-Matthews test): primitive (rho, vx, vy, vz, P), transverse velocity
# on both sides, evolved to t = 0.7 with the Taub-Matthews EOS and the ideal EOS at 4/3 and 5/3.
TM_BLAST = dict(left=(1.0, 0.0, 0.9, 0.0, 1e3), right=(1.0, 0.0, 0.99, 0.0, 1e-2), t_final=0.7)


def tm_blast(eos: str = "tm", gamma_ad: float = 4.0 / 3.0, n: int = 128, degree: int = 1,
             flux: str = "hllc") -> dict:
    """The Taub-Matthews blast wave of Sec. 4.3 on [0, 1] with the interface at x = 0.5 and
    Dirichlet ends; `eos` "tm" (gamma_ad unused) or "ideal" (4/3 or 5/3 in the paper); the
    iterative con2prim, SSP-RK with p + 1 stages (at most 3), CFL 0.2."""
    left, right = TM_BLAST["left"], TM_BLAST["right"]
    return dict(name="riemann_1d", problem="tm_blast", dim=1, degree=degree, n_elem=[n],
                lo=[0.0], hi=[1.0], eos=eos, gamma_ad=gamma_ad, c2p="iterative", flux=flux,
                rk_stages=min(degree + 1, 3), bc=[("dirichlet", "dirichlet")],
                bc_state=[[left, right]], enforce=True, cfl=0.2, t_final=TM_BLAST["t_final"],
                left=left, right=right)


def advected_wave(n: int = 512, degree: int = 3, flux: str = "llf", c2p: str = "default") -> dict:
    """2D advected density wave on the periodic unit square, Gamma = 4/3, SSPRK3."""
    return dict(name="advected_wave_2d", dim=2, degree=degree, n_elem=[n, n], lo=[0.0, 0.0],
                hi=[1.0, 1.0], eos="ideal", gamma_ad=4.0 / 3.0, c2p=c2p, flux=flux,
                rk_stages=3, bc=[("periodic", "periodic")] * 2, enforce=True, cfl=0.2)


def kh2d(nx: int = 256, ny: int = 512, degree: int = 3, flux: str = "hll",
         c2p: str = "default") -> dict:
    """2D relativistic Kelvin-Helmholtz, Taub-Matthews EOS, [-0.5,0.5] x [-1,1], periodic."""
    return dict(name="kh_2d", dim=2, degree=degree, n_elem=[nx, ny], lo=[-0.5, -1.0],
                hi=[0.5, 1.0], eos="tm", gamma_ad=4.0 / 3.0, c2p=c2p, flux=flux, rk_stages=3,
                bc=[("periodic", "periodic")] * 2, enforce=True, cfl=0.2, amplitude=0.01)


def kh_single(nx: int = 256, ny: int = 512, degree: int = 1, flux: str = "hll",
              c2p: str = "iterative") -> dict:
    """The paper's Kelvin-Helmholtz set-up (Sec. 4.5): [-0.5,0.5] x [-1,1], one shear layer at
    y = 0 of thickness a = 0.01 with shear velocity 0.25 (c = 1), rho0 = 1, P0 = 1, ideal EOS
    Gamma = 4/3 with the iterative con2prim, perturbation amplitude A = 0.05 at k = 2 pi;
    periodic in x, outflow in y; SSP-RK with p + 1 stages (at most 3)."""
    return dict(name="kh_single", dim=2, degree=degree, n_elem=[nx, ny], lo=[-0.5, -1.0],
                hi=[0.5, 1.0], eos="ideal", gamma_ad=4.0 / 3.0, c2p=c2p, flux=flux,
                rk_stages=min(degree + 1, 3),
                bc=[("periodic", "periodic"), ("outflow", "outflow")], enforce=True, cfl=0.2,
                shear=0.25, amplitude=0.05, layer=0.01, sigma=0.1)


# Linear waves (Sec. 4.1): wave frames.  Table 1 of that section gives (N wavelengths, n-th
# acceptable angle) per test type; tan(theta) = sqrt(N / (N - n) - 1).  The 3D rotation is
# about a = (0, -1, 1)/sqrt(2); in 2D the wave vector is turned by theta within the x-y plane.
LINEAR_WAVE_FRAMES = {
    "1d": (1, 1, 0), "2d": (2, 1, 0), "2d_oblique": (2, 2, 1), "3d": (3, 1, 0), "3d_oblique": (3, 3, 2),
}


def _rotation(axis, theta):
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0.0, -a[2], a[1]], [a[2], 0.0, -a[0]], [-a[1], a[0], 0.0]])
    return math.cos(theta) * np.eye(3) + (1.0 - math.cos(theta)) * np.outer(a, a) + math.sin(theta) * K


def linear_wave(frame: str, degree: int, n_base: int, refine: int, eigvec, eigval: float,
                rho0: float = 1.0, P0: float = 1.0, gamma_ad: float = 5.0 / 3.0,
                amplitude: float = 1e-6, t_final: float = 0.5, flux: str = "llf") -> dict:
    """A linear wave of unit wavelength (Sec. 4.1) on a periodic box aligned with its wave frame
    (`frame` in LINEAR_WAVE_FRAMES), base state (rho0, v = 0, P0), ideal EOS.  eigvec is the
    right eigenvector (rho, v_par, v_perp1, v_perp2, P) in the wave frame and eigval its
    eigenvalue (the caller computes both: they need the sound speed).  Elements per axis:
    n_base 2^refine times the box length; SSP-RK with p + 1 stages (RK1, SSPRK2, SSPRK3)."""
    dim, N, n = LINEAR_WAVE_FRAMES[frame]
    theta = math.atan(math.sqrt(N / (N - n) - 1.0)) if n else 0.0
    R = _rotation((0.0, -1.0, 1.0) if dim == 3 else (0.0, 0.0, 1.0), theta)
    khat = R[:, 0]
    # box: N khat per axis (N |khat_d| is a whole number of wave periods along axis d); one
    # unit along the axes the wave does not vary on
    L = [float(N * abs(khat[d])) if abs(khat[d]) > 1e-12 else 1.0 for d in range(dim)]
    ne = [max(1, int(round(n_base * 2 ** refine * L[d]))) for d in range(dim)]
    return dict(name="linear_wave", frame=frame, dim=dim, degree=degree, n_elem=ne,
                lo=[0.0] * dim, hi=L, eos="ideal", gamma_ad=gamma_ad, c2p="iterative",
                flux=flux, rk_stages=min(degree + 1, 3), bc=[("periodic", "periodic")] * dim,
                enforce=True, cfl=0.2, t_final=t_final, rho0=rho0, P0=P0, amplitude=amplitude,
                eigvec=tuple(float(v) for v in eigvec), eigval=float(eigval),
                khat=tuple(float(v) for v in khat), e1=tuple(float(v) for v in R[:, 1]),
                e2=tuple(float(v) for v in R[:, 2]))


def kh3d(n: int = 128, degree: int = 3, flux: str = "hll", c2p: str = "default") -> dict:
    """3D high-Lorentz-factor Kelvin-Helmholtz on the periodic unit cube, Taub-Matthews EOS."""
    return dict(name="kh_3d", dim=3, degree=degree, n_elem=[n, n, n], lo=[0.0] * 3,
                hi=[1.0] * 3, eos="tm", gamma_ad=4.0 / 3.0, c2p=c2p, flux=flux, rk_stages=3,
                bc=[("periodic", "periodic")] * 3, enforce=True, cfl=0.2, seed=KH3D_SEED)


def shape(spec: dict):
    """(total elements, nodes per element)."""
    dim = int(spec["dim"])
    return int(np.prod([int(v) for v in spec["n_elem"][:dim]])), (int(spec["degree"]) + 1) ** dim


# --------------------------------------------------------------------------
# Initial primitive fields W = (rho, vx, vy, vz, P) at given coordinates.
# X is a numpy array or a torch tensor (then the field is evaluated where X lives, e.g. on
# the GPU); the result has the same type, shape (5,) + X.shape[1:].
# --------------------------------------------------------------------------

def _xp(X):
    """numpy or torch, whichever holds X (only functions both provide are used)."""
    if isinstance(X, np.ndarray):
        return np
    import torch
    if isinstance(X, torch.Tensor):
        return torch
    raise TypeError(f"coordinates must be a numpy array or a torch tensor, not {type(X)}")


def _const(x, c):
    return x * 0.0 + c


def blast_wave_ic(spec: dict, X) -> np.ndarray:
    xp = _xp(X)
    x = X[0]
    left, right = spec["left"], spec["right"]
    return xp.stack([xp.where(x < 0.5, _const(x, left[v]), _const(x, right[v])) for v in range(5)])


def advected_wave_ic(spec: dict, X, t: float = 0.0):
    """rho = 1 + 0.5 sin(2 pi (x + y - (vx + vy) t)), v = (0.5, 0.5)/sqrt(2), P = 1."""
    xp = _xp(X)
    x, y = X[0], X[1]
    vx = vy = 0.5 / math.sqrt(2.0)
    rho = 1.0 + 0.5 * xp.sin(2.0 * np.pi * (x + y - (vx + vy) * t))
    return xp.stack([rho, _const(x, vx), _const(x, vy), _const(x, 0.0), _const(x, 1.0)])


def _double_layer(xp, y, a=0.01):
    """+1 inside 0 < y < 1, -1 inside -1 < y < 0 (period 2), tanh layers of width a."""
    return xp.tanh(y / a) - xp.tanh((y - 1.0) / a) - xp.tanh((y + 1.0) / a)


def linear_wave_ic(spec: dict, X, t: float = 0.0):
    """W = W0 + A r sin(2 pi (khat . x) - omega t), omega = 2 pi eigval, with the velocity
    part of r turned from the wave frame: v = r_par khat + r_perp1 e1 + r_perp2 e2."""
    xp = _xp(X)
    dim = int(spec["dim"])
    x = X[0]
    phase = _const(x, 0.0)
    for d in range(dim):
        phase = phase + spec["khat"][d] * X[d]
    s = xp.sin(2.0 * np.pi * (phase - spec["eigval"] * t))
    A, r = spec["amplitude"], spec["eigvec"]
    v = [A * (r[1] * spec["khat"][c] + r[2] * spec["e1"][c] + r[3] * spec["e2"][c]) * s
         for c in range(3)]
    return xp.stack([spec["rho0"] + A * r[0] * s, v[0], v[1], v[2], spec["P0"] + A * r[4] * s])


def kh_single_ic(spec: dict, X):
    """v_x = v0 tanh(y / a), v_y = A sin(2 pi x) exp(-y^2 / sigma^2), rho = 1, P = 1."""
    xp = _xp(X)
    x, y = X[0], X[1]
    vx = spec["shear"] * xp.tanh(y / spec["layer"])
    vy = spec["amplitude"] * xp.sin(2.0 * np.pi * x) * xp.exp(-(y * y) / spec["sigma"] ** 2)
    return xp.stack([_const(x, 1.0), vx, vy, _const(x, 0.0), _const(x, 1.0)])


def kh2d_ic(spec: dict, X, amplitude: float | None = None):
    """v_x = 0.5 f(y), rho = 0.55 + 0.45 f(y) (1 and 0.1), P = 1,
    v_y = A sin(2 pi x) exp(-y^2 / 0.01)."""
    xp = _xp(X)
    A = spec.get("amplitude", 0.01) if amplitude is None else amplitude
    x, y = X[0], X[1]
    f = _double_layer(xp, y)
    return xp.stack([0.55 + 0.45 * f, 0.5 * f, A * xp.sin(2.0 * np.pi * x) * xp.exp(-y * y / 0.01),
                     _const(x, 0.0), _const(x, 1.0)])


def _modes(rng, kmax2):
    ks = [(i, j, k) for i in range(-2, 3) for j in range(-2, 3) for k in range(-2, 3)
          if 0 < i * i + j * j + k * k <= kmax2]
    phases = rng.uniform(0.0, 2.0 * np.pi, size=len(ks))
    return np.array(ks, dtype=np.float64), phases


def _mode_sum(xp, ks, phases, x, y, z):
    s = x * 0.0
    for (kx, ky, kz), ph in zip(ks, phases):
        s = s + xp.sin(2.0 * np.pi * (kx * x + ky * y + kz * z) + ph)
    return s / len(ks)


def _kh3d_fields(xp, kp, php, kq, phq, kb, phb, x, y, z):
    f = xp.tanh((y - 0.25) / 0.01) - xp.tanh((y - 0.75) / 0.01) - 1.0
    ux = 0.9 / math.sqrt(1.0 - 0.81) * f
    uy = 1e-3 * _mode_sum(xp, kp, php, x, y, z)
    uz0 = 1e-3 * _mode_sum(xp, kq, phq, x, y, z)
    g = _mode_sum(xp, kb, phb, x, y, z)
    return f, ux, uy, uz0, g


def kh3d_ic(spec: dict, X):
    """Shear v_x = +-0.9 between layers at y = 0.25 and 0.75, a seeded perturbation of
    amplitude 1e-3 in (v_y, v_z), and a seeded smooth bulk boost in the 4-velocity u_z
    scaled so that the largest Lorentz factor on a fixed 64^3 sample grid is 10.
    Built in the 4-velocity u so that every state is subluminal."""
    rng = np.random.default_rng(spec.get("seed", KH3D_SEED))
    kp, php = _modes(rng, 4)
    kq, phq = _modes(rng, 4)
    kb, phb = _modes(rng, 2)
    g1 = (np.arange(64) + 0.5) / 64.0
    gx, gy, gz = np.meshgrid(g1, g1, g1, indexing="ij")
    _, ux_s, uy_s, uz0_s, g_s = _kh3d_fields(np, kp, php, kq, phq, kb, phb, gx, gy, gz)
    base = 1.0 + ux_s * ux_s + uy_s * uy_s

    def max_gamma(boost):
        uz = uz0_s + boost * g_s
        return float(np.sqrt(base + uz * uz).max())

    lo, hi = 0.0, 100.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if max_gamma(mid) < 10.0:
            lo = mid
        else:
            hi = mid
    boost = 0.5 * (lo + hi)
    xp = _xp(X)
    f, ux, uy, uz0, g = _kh3d_fields(xp, kp, php, kq, phq, kb, phb, X[0], X[1], X[2])
    uz = uz0 + boost * g
    lor = xp.sqrt(1.0 + ux * ux + uy * uy + uz * uz)
    return xp.stack([0.55 + 0.45 * f, ux / lor, uy / lor, uz / lor, _const(f, 1.0)])


def initial_primitive(spec: dict, X):
    name = spec["name"]
    if name in ("blast_wave_1d", "riemann_1d"):
        return blast_wave_ic(spec, X)
    if name == "advected_wave_2d":
        return advected_wave_ic(spec, X)
    if name == "kh_2d":
        return kh2d_ic(spec, X)
    if name == "kh_3d":
        return kh3d_ic(spec, X)
    if name == "kh_single":
        return kh_single_ic(spec, X)
    if name == "linear_wave":
        return linear_wave_ic(spec, X)
    if name == "riemann_2d":
        return riemann_2d_ic(spec, X)
    if name == "smooth_random":
        return smooth_random_ic(spec, X)
    raise KeyError(name)


# --------------------------------------------------------------------------
# Seeded random inputs for parity tests
# --------------------------------------------------------------------------

def smooth_random(dim: int, n_elem, degree: int, eos: str = "ideal", seed: int = 0,
                  flux: str = "llf", c2p: str = "default", vmax: float = 0.6,
                  bc=None, rk_stages: int = 3) -> dict:
    """A periodic box with a seeded smooth random primitive field (a few Fourier modes):
    rho in about [0.3, 1.7], |v| up to vmax, P in about [0.2, 1.8]."""
    bc = bc or [("periodic", "periodic")] * dim
    return dict(name="smooth_random", dim=dim, degree=degree, n_elem=list(n_elem),
                lo=[0.0] * dim, hi=[1.0] * dim, eos=eos, gamma_ad=5.0 / 3.0 if eos == "ideal" else 4.0 / 3.0,
                c2p=c2p, flux=flux, rk_stages=rk_stages, bc=bc, enforce=True, cfl=0.2, seed=seed,
                vmax=vmax, bc_state=[[(1.0, 0.1, 0.0, 0.0, 1.0), (0.5, -0.1, 0.0, 0.0, 0.5)]] * dim)


def smooth_random_ic(spec: dict, X):
    xp = _xp(X)
    rng = np.random.default_rng(spec.get("seed", 0))
    dim = X.shape[0]
    coords = [X[d] for d in range(dim)]

    def field():
        s = coords[0] * 0.0
        for _ in range(3):
            k = rng.integers(-2, 3, size=dim)
            if not np.any(k):
                k[0] = 1
            ph = rng.uniform(0, 2 * np.pi)
            amp = rng.uniform(0.3, 1.0)
            s = s + amp * xp.sin(2 * np.pi * sum(float(k[d]) * coords[d] for d in range(dim)) + ph)
        return s / 3.0

    rho = 1.0 + 0.7 * field()
    vx, vy, vz = field(), field(), field()
    vmag = xp.sqrt(vx * vx + vy * vy + vz * vz)
    scale = spec.get("vmax", 0.6) / max(float(vmag.max()), 1e-30)
    P = 1.0 + 0.8 * field()
    return xp.stack([rho, vx * scale, vy * scale, vz * scale, P])


def random_primitive_states(n: int, seed: int = 0, gamma_max: float = 10.0,
                            theta_range=(1e-3, 1e3), rho_range=(1e-3, 1e3)) -> np.ndarray:
    """n seeded primitive states (rho, vx, vy, vz, P): log-uniform rho, Theta = P/rho and
    gamma in [1, gamma_max], isotropic velocity direction."""
    rng = np.random.default_rng(seed)
    rho = 10.0 ** rng.uniform(np.log10(rho_range[0]), np.log10(rho_range[1]), n)
    th = 10.0 ** rng.uniform(np.log10(theta_range[0]), np.log10(theta_range[1]), n)
    lor = 10.0 ** rng.uniform(0.0, np.log10(gamma_max), n)
    beta = np.sqrt(1.0 - 1.0 / (lor * lor))
    d = rng.normal(size=(3, n))
    d /= np.linalg.norm(d, axis=0)
    W = np.empty((5, n))
    W[0] = rho
    W[1:4] = beta * d
    W[4] = rho * th
    return W


def e2_grid():
    """The (gamma, P) grid of the con2prim accuracy study: 25 log-spaced Lorentz factors
    in [1, 100] and 25 log-spaced pressures in [1e5, 1e10] N/m^2 with D = 1 kg/m^3 and
    c = 3e8 m/s (Sec. 3.3), in units c = 1: P -> P/c^2, rho = D/gamma, v along x.
    Returns (W (5, 25, 25), gamma (25,), P_si (25,)) indexed [pressure, gamma]."""
    c = 3e8
    lor = np.logspace(0.0, 2.0, 25)
    P_si = np.logspace(5.0, 10.0, 25)
    G, P = np.meshgrid(lor, P_si / (c * c))
    W = np.zeros((5, 25, 25))
    W[0] = 1.0 / G
    W[1] = np.sqrt(1.0 - 1.0 / (G * G))
    W[4] = P
    return W, lor, P_si


def random_conserved_cells(n_cells: int, nodes: int, seed: int = 0, bad_fraction: float = 0.3,
                           bad_mean_fraction: float = 0.05):
    """Seeded conserved nodal states U (5, n_cells, nodes) built directly in (D, S, tau):
    each cell is a random mean plus nodal deviations large enough that roughly
    `bad_fraction` of the cells hold nodes outside the admissible set; about
    `bad_mean_fraction` of the cells are centred outside it.  Used to exercise the
    physicality operator."""
    rng = np.random.default_rng(seed)
    U = np.empty((5, n_cells, nodes))
    D0 = rng.uniform(0.5, 2.0, (n_cells, 1))
    S0 = rng.normal(0.0, 0.5, (3, n_cells, 1)) * D0
    margin0 = rng.uniform(0.2, 1.0, (n_cells, 1)) * D0
    centred_out = rng.uniform(size=(n_cells, 1)) < bad_mean_fraction
    margin0 = np.where(centred_out, -rng.uniform(0.05, 0.3, (n_cells, 1)) * D0, margin0)
    bad = rng.uniform(size=(n_cells, 1)) < bad_fraction
    amp = np.where(bad, 1.5, 0.05)
    U[0] = D0 + amp * rng.normal(0.0, 0.6, (n_cells, nodes)) * D0
    U[1:4] = S0 + amp * rng.normal(0.0, 0.6, (3, n_cells, nodes)) * D0
    # tau so that E = tau + D sits near sqrt(D^2 + S^2) + margin
    Smag = np.sqrt(U[1] ** 2 + U[2] ** 2 + U[3] ** 2)
    U[4] = np.sqrt(U[0] ** 2 + Smag ** 2) - U[0] + margin0 + amp * rng.normal(0.0, 0.8, (n_cells, nodes)) * D0
    return U
