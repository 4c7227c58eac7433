"""Seeded synthetic initial conditions for the direct PP N-body workloads.

This module is shared by the FP64 oracle tests and the GPU library tests and
benchmark; it holds none of the method's arithmetic (no pairwise force sum,
no integrator, no diagnostics).  Every generator takes an explicit seed and
returns float64 numpy arrays: pos (n, 3), vel (n, 3), mass (n,).

The paper's own galaxy model comes from an iterative equilibrium procedure
(section 1, Eq. 3-4 and the works it cites) that is not reproduced here; the
generators below stand in for it with the same shapes and sizes:

* plummer          -- Plummer sphere sampled with the Aarseth, Henon & Wielen
                      (1974) recipe: radius from the inverted cumulative mass,
                      speed from the isotropic distribution function by
                      von Neumann rejection.
* uniform_sphere   -- positions uniform in a ball.
* lognormal_masses -- masses exp(sigma * N(0,1)), normalised to a total.
* disk_halo        -- exponential stellar disk (surface density exp(-R/Rd),
                      truncated), sech^2 vertical profile, Toomre-Q velocity
                      dispersions, asymmetric-drift corrected rotation, and a
                      live Plummer halo.  The circular speed comes from the
                      analytic potentials of a thin exponential disk (Freeman
                      1970, modified Bessel functions) and a Plummer sphere,
                      not from the N-body sum.

Seeds: workload k of the benchmark uses numpy PCG64 with seed 20180111 + k.
"""
import numpy as np

SEED_BASE = 20180111


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _iso_dirs(g, n):
    """n isotropic unit vectors."""
    z = g.uniform(-1.0, 1.0, n)
    phi = g.uniform(0.0, 2.0 * np.pi, n)
    s = np.sqrt(1.0 - z * z)
    return np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)


def _centre(pos, vel, mass):
    m = mass[:, None]
    pos = pos - (m * pos).sum(0) / mass.sum()
    vel = vel - (m * vel).sum(0) / mass.sum()
    return pos, vel


def plummer(n, seed, a=1.0, M=1.0, G=1.0, centre=True):
    """Plummer sphere of total mass M and scale radius a, equal masses.
    Untruncated: only the draw X = 1 (infinite radius) is rejected."""
    g = rng(seed)
    X = g.uniform(0.0, 1.0, n)
    while True:
        bad = (X <= 0.0) | (X >= 1.0)
        if not bad.any():
            break
        X[bad] = g.uniform(0.0, 1.0, int(bad.sum()))
    r = a / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
    pos = r[:, None] * _iso_dirs(g, n)
    # speed: q = v / v_esc with density g(q) = q^2 (1 - q^2)^{7/2}, max < 0.1
    q = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        x = g.uniform(0.0, 1.0, todo.size)
        y = g.uniform(0.0, 0.1, todo.size)
        ok = y < x * x * (1.0 - x * x) ** 3.5
        q[todo[ok]] = x[ok]
        todo = todo[~ok]
    vesc = np.sqrt(2.0 * G * M / a) * (1.0 + (r / a) ** 2) ** -0.25
    vel = (q * vesc)[:, None] * _iso_dirs(g, n)
    mass = np.full(n, M / n)
    if centre:
        pos, vel = _centre(pos, vel, mass)
    return pos, vel, mass


def uniform_sphere(n, seed, R=1.0):
    """Positions uniform in a ball of radius R; zero velocities; equal masses summing to 1."""
    g = rng(seed)
    r = R * g.uniform(0.0, 1.0, n) ** (1.0 / 3.0)
    pos = r[:, None] * _iso_dirs(g, n)
    return pos, np.zeros((n, 3)), np.full(n, 1.0 / n)


def lognormal_masses(n, seed, sigma=0.5, total=1.0):
    """Masses exp(sigma * N(0,1)), scaled so that they sum to `total`."""
    m = np.exp(sigma * rng(seed).standard_normal(n))
    return m * (total / m.sum())


def _bessel():
    from scipy import special
    return special.i0, special.i1, special.k0, special.k1


def disk_vc2(R, Md=1.0, Rd=1.0, Rmax=5.0, G=1.0):
    """Circular speed squared in the plane of a razor-thin exponential disk
    (Freeman 1970): v^2 = 4 pi G S0 Rd y^2 [I0 K0 - I1 K1](y), y = R / (2 Rd),
    with S0 chosen so that the disk truncated at Rmax holds mass Md."""
    i0, i1, k0, k1 = _bessel()
    frac = 1.0 - (1.0 + Rmax / Rd) * np.exp(-Rmax / Rd)
    S0 = Md / (2.0 * np.pi * Rd * Rd * frac)
    y = np.maximum(R, 1e-8) / (2.0 * Rd)
    return 4.0 * np.pi * G * S0 * Rd * y * y * (i0(y) * k0(y) - i1(y) * k1(y))


def plummer_vc2(R, M=1.0, a=1.0, G=1.0):
    return G * M * R * R / (R * R + a * a) ** 1.5


def disk_halo(n, seed, Rd=1.0, Rmax=5.0, h=0.05, Q=1.2, Md=1.0, Mh=1.0, ah=3.0, G=1.0,
              disk_fraction=0.5, centre=True):
    """Exponential disk + live Plummer halo (disk:halo particle ratio set by
    disk_fraction, 1:1 by default; equal disk and halo masses give equal
    particle masses).  Disk particles come first, then halo particles."""
    g = rng(seed)
    nd = int(round(n * disk_fraction))
    nh = n - nd
    # --- disk radii: inverse of the truncated cumulative mass 1 - (1 + x) e^{-x}
    u = g.uniform(0.0, 1.0, nd)
    xmax = Rmax / Rd
    target = u * (1.0 - (1.0 + xmax) * np.exp(-xmax))
    lo = np.zeros(nd)
    hi = np.full(nd, xmax)
    for _ in range(60):                       # bisection, monotone CDF
        mid = 0.5 * (lo + hi)
        f = 1.0 - (1.0 + mid) * np.exp(-mid)
        lo = np.where(f < target, mid, lo)
        hi = np.where(f < target, hi, mid)
    R = Rd * 0.5 * (lo + hi)
    phi = g.uniform(0.0, 2.0 * np.pi, nd)
    uz = g.uniform(0.0, 1.0, nd)
    uz = np.clip(uz, 1e-12, 1.0 - 1e-12)
    z = h * np.arctanh(2.0 * uz - 1.0)
    # --- kinematics from the analytic rotation curve of disk + halo
    Rs = np.maximum(R, 1e-3)
    vc2 = lambda x: disk_vc2(x, Md, Rd, Rmax, G) + plummer_vc2(x, Mh, ah, G)
    dR = 1e-4
    v2 = vc2(Rs)
    Omega = np.sqrt(v2) / Rs
    # kappa^2 = R^-3 d(R^2 v_c^2)/dR
    d_r2v2 = ((Rs + dR) ** 2 * vc2(Rs + dR) - (Rs - dR) ** 2 * vc2(Rs - dR)) / (2 * dR)
    kappa = np.sqrt(np.maximum(d_r2v2 / Rs ** 3, 1e-12))
    frac = 1.0 - (1.0 + xmax) * np.exp(-xmax)
    Sigma = Md / (2.0 * np.pi * Rd * Rd * frac) * np.exp(-Rs / Rd)
    sR = Q * 3.36 * G * Sigma / kappa
    sphi = sR * kappa / (2.0 * Omega)
    sz = np.sqrt(np.pi * G * Sigma * h)
    # asymmetric drift: vphi^2 = vc^2 + sR^2 (1 - sphi^2/sR^2 + dln(Sigma sR^2)/dlnR)
    def lnSs(x):
        xs = np.maximum(x, 1e-3)
        kk = np.sqrt(np.maximum(((xs + dR) ** 2 * vc2(xs + dR) - (xs - dR) ** 2 * vc2(xs - dR)) / (2 * dR) / xs ** 3, 1e-12))
        S = np.exp(-xs / Rd)
        return np.log(S * (Q * 3.36 * G * S / kk) ** 2)
    eps_l = 1e-3
    dlnSs = (lnSs(Rs * (1 + eps_l)) - lnSs(Rs * (1 - eps_l))) / (np.log1p(eps_l) - np.log1p(-eps_l))
    vphi2 = v2 + sR ** 2 * (1.0 - (sphi / sR) ** 2 + dlnSs)
    vphi = np.sqrt(np.maximum(vphi2, 0.0))
    vR = sR * g.standard_normal(nd)
    vp = vphi + sphi * g.standard_normal(nd)
    vz = sz * g.standard_normal(nd)
    c, s = np.cos(phi), np.sin(phi)
    dpos = np.stack([R * c, R * s, z], axis=1)
    dvel = np.stack([vR * c - vp * s, vR * s + vp * c, vz], axis=1)
    # --- halo: Plummer sphere with its own isotropic distribution function
    hseed = int(g.integers(0, 2 ** 62))
    hpos, hvel, _ = plummer(nh, hseed, a=ah, M=Mh, G=G, centre=False) if nh > 0 else (np.zeros((0, 3)),) * 3
    pos = np.concatenate([dpos, hpos])
    vel = np.concatenate([dvel, hvel])
    mass = np.concatenate([np.full(nd, Md / max(nd, 1)), np.full(nh, Mh / max(nh, 1))])
    if centre:
        pos, vel = _centre(pos, vel, mass)
    return pos, vel, mass


def workload(name, n=None, seed=None):
    """Named synthetic workloads (sizes of the benchmark configurations).

    plummer4096   : Plummer a=1, G=M=1, N=4096, eps=0.01         (seed base+0)
    disk_halo_2^17: disk + halo, N=2^17, eps=0.02                (seed base+1)
    disk_halo_2^20: disk + halo, N=2^20, eps=0.02                (seed base+2)
    sweep_*       : uniform sphere / Plummer with lognormal masses (seed base+3)
    Returns dict(pos, vel, mass, eps, G)."""
    if name == "plummer":
        n = 4096 if n is None else n
        s = SEED_BASE + 0 if seed is None else seed
        p, v, m = plummer(n, s)
        return dict(pos=p, vel=v, mass=m, eps=0.01, G=1.0)
    if name == "disk_halo":
        n = 2 ** 17 if n is None else n
        s = (SEED_BASE + (2 if n >= 2 ** 20 else 1)) if seed is None else seed
        p, v, m = disk_halo(n, s)
        return dict(pos=p, vel=v, mass=m, eps=0.02, G=1.0)
    if name in ("sweep_uniform", "sweep_plummer"):
        n = 2 ** 16 if n is None else n
        s = SEED_BASE + 3 if seed is None else seed
        if name == "sweep_uniform":
            p, v, _ = uniform_sphere(n, s)
        else:
            p, v, _ = plummer(n, s)
        m = lognormal_masses(n, s + 1)
        return dict(pos=p, vel=v, mass=m, eps=1e-2, G=1.0)
    raise KeyError(name)
