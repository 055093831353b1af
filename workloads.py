"""Seeded synthetic workloads shaped like the cases of Zhang et al. (arXiv 1502.01159).

This module holds input generation only -- lattice sizes, physical parameters,
wall settings, particle placement, marker placement -- and none of the
method's arithmetic.  Both the CUDA library's binding and the CPU oracle are
fed from these dicts, so the two sides always see bit-identical inputs.

Case dict keys
--------------
dim, shape=(nx, ny, nz), Ra, Pr, U_c, L_c, T_ref, T_init, buoyancy,
gravity_axis, body_force[3], g_particle[3], dem_substeps, kappa_T, cell_size,
nu_dT, pibm, flow_q (0 default; 15 selects D3Q15 in 3-D), particle_model
("resolved" or "point"), walls = 2*dim entries (kind, thermal, T_w) ordered
x-lo, x-hi, y-lo, y-hi, z-lo, z-hi (kind 0 periodic / 1 wall; thermal 0
adiabatic / 1 isothermal), contact = contact-law dict, particles = dict of
arrays (X n*3, U, W, R, rho_p, T_p, heat_cap, fixed) or None, markers =
dict (X n*3, A, T) or None.

Recipes (units: lattice units, h = dt = 1)
------------------------------------------
cavity   : square cavity with concentric isothermal cylinder (paper's
           natural-convection case): four cold walls T = 0, cylinder of
           radius L/(2 Ar) built from static points of diameter h/2 on a
           square sub-lattice of spacing h/2 (area pi/16 each), T = 1;
           fluid starts at 0.5; Ra, Pr, U_c = 0.25, L_c = L.
sed2d    : 2-D sedimentation of heated disks: n_p disks placed by random
           sequential addition (gap >= 1 to each other and to the walls) in
           the upper half; density ratio 1.5; T_p = 1; walls T = 0; fluid 0.5;
           linear spring-dashpot contacts; 10 DEM substeps.
sed3d    : 3-D sedimentation of heated spheres: random sequential addition in
           the upper 3/5; density ratio 1.2; Hertz / Mindlin-Deresiewicz.
ensemble : batched thermosensitive 3-D sedimentation: cubic boxes with edge
           drawn from {64, 72, ..., 128}, Ra log-uniform in [1e3, 1e5],
           sphere count uniform in [50, 400] (capped at a 12% solid fraction
           so random sequential addition over the whole box succeeds),
           d = 8, T_p(0) uniform in [0, 1], heat capacity rho_p V_p, Hertz.
points   : sub-grid particles (the paper's own regime, d_p <= h): the sed2d /
           sed3d recipes with d = 0.5, density ratio 4, particle_model "point".
poiseuille, conduction, periodic_box : closed-form and invariant checks.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 1502011590

D2Q9_E = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (-1, 0, 0), (0, -1, 0),
          (1, 1, 0), (-1, 1, 0), (-1, -1, 0), (1, -1, 0)]
D3Q19_E = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
           (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1),
           (1, 0, -1), (-1, 0, 1), (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]


def rng(config_index: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + config_index))


def _base(dim, shape, **kw):
    case = dict(dim=dim, shape=tuple(int(v) for v in shape), Ra=1e4, Pr=0.71, U_c=0.1,
                L_c=float(shape[dim - 1]), T_ref=0.5, T_init=0.5, buoyancy=True,
                gravity_axis=dim - 1, body_force=[0.0, 0.0, 0.0], g_particle=[0.0, 0.0, 0.0],
                dem_substeps=10, kappa_T=1.0, cell_size=0.0, nu_dT=1.0, pibm=True,
                walls=[(1, 1, 0.0)] * (2 * dim), contact=None, particles=None, markers=None,
                storage="f32")
    case.update(kw)
    return case


def spring_dashpot(kn=100.0, kt=28.6, gamma_n=5.15, gamma_t=0.0, mu=0.3):
    return dict(law=0, E=0.0, poisson=0.0, mu=mu, kn=kn, kt=kt, gamma_n=gamma_n, gamma_t=gamma_t)


def hertz(E=2000.0, poisson=0.33, mu=0.3, gamma_n=0.0, gamma_t=0.0):
    return dict(law=1, E=E, poisson=poisson, mu=mu, kn=0.0, kt=0.0, gamma_n=gamma_n, gamma_t=gamma_t)


def rsa_positions(gen, n, radius, lo, hi, gap=1.0, max_tries=200000):
    """Random sequential addition of n equal spheres/disks with centres drawn
    uniformly in the box [lo, hi] (per-axis arrays), rejecting any candidate
    closer than 2*radius + gap to an accepted one."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    dim = len(lo)
    cell = 2 * radius + gap
    grid: dict = {}
    out = []
    tries = 0
    while len(out) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError(f"random sequential addition placed only {len(out)} of {n}")
        c = lo + gen.random(dim) * (hi - lo)
        key = tuple((c // cell).astype(int))
        ok = True
        for off in np.ndindex(*([3] * dim)):
            nb = tuple(k + o - 1 for k, o in zip(key, off))
            for q in grid.get(nb, ()):
                if np.sum((out[q] - c) ** 2) < cell * cell:
                    ok = False
                    break
            if not ok:
                break
        if ok:
            grid.setdefault(key, []).append(len(out))
            out.append(c)
    X = np.zeros((n, 3))
    if n:
        X[:, :dim] = np.array(out)
    return X


def cavity(n=128, Ra=1e4, Pr=0.71, Ar=2.5, U_c=0.25, storage="f64"):
    """Natural convection in a square cavity with a concentric cylinder built
    from static points of diameter h/2 (the paper's cavity case)."""
    R = n / (2.0 * Ar)
    c = (n - 1) / 2.0
    k = np.arange(-int(2 * R) - 2, int(2 * R) + 3)
    off = (k + 0.5) * 0.5
    xs, ys = np.meshgrid(c + off, c + off, indexing="xy")
    inside = (xs - c) ** 2 + (ys - c) ** 2 < R * R
    X = np.zeros((int(inside.sum()), 3))
    X[:, 0] = xs[inside]
    X[:, 1] = ys[inside]
    m = X.shape[0]
    markers = dict(X=X, A=np.full(m, np.pi / 16.0), T=np.ones(m))
    return _base(2, (n, n, 1), Ra=Ra, Pr=Pr, U_c=U_c, L_c=float(n), markers=markers,
                 dem_substeps=1, storage=storage, name=f"cavity{n}_Ra{Ra:g}_Ar{Ar:g}")


def sed2d(nx=512, ny=1024, n_p=500, d=10.0, rho_ratio=1.5, g=1e-4, config_index=1, storage="f32",
          T_p=1.0):
    gen = rng(config_index)
    R = d / 2
    X = rsa_positions(gen, n_p, R, [R + 1.0, ny / 2 + R + 1.0], [nx - 1.5 - R - 1.0, ny - 1.5 - R - 1.0])
    parts = dict(X=X, R=np.full(n_p, R), rho_p=np.full(n_p, rho_ratio), T_p=np.full(n_p, T_p))
    return _base(2, (nx, ny, 1), particles=parts, contact=spring_dashpot(),
                 g_particle=[0.0, -g, 0.0], storage=storage, name=f"sed2d_{nx}x{ny}_{n_p}p")


def sed3d(nx=256, ny=256, nz=512, n_p=2000, d=8.0, rho_ratio=1.2, g=1e-4, config_index=2,
          storage="f32", T_p=1.0, heat_cap=None, T_p_random=False):
    gen = rng(config_index)
    R = d / 2
    lo = [R + 1.0, R + 1.0, nz * 2.0 / 5.0 + R]
    hi = [nx - 1.5 - R - 1.0, ny - 1.5 - R - 1.0, nz - 1.5 - R - 1.0]
    X = rsa_positions(gen, n_p, R, lo, hi)
    Tp = gen.random(n_p) if T_p_random else np.full(n_p, T_p)
    parts = dict(X=X, R=np.full(n_p, R), rho_p=np.full(n_p, rho_ratio), T_p=Tp)
    if heat_cap is not None:
        parts["heat_cap"] = np.full(n_p, heat_cap)
    return _base(3, (nx, ny, nz), particles=parts, contact=hertz(),
                 g_particle=[0.0, 0.0, -g], storage=storage, name=f"sed3d_{nx}x{ny}x{nz}_{n_p}p")


def ensemble(n_boxes=32, edges=tuple(range(64, 129, 8)), n_range=(50, 400), Ra_range=(1e3, 1e5), d=8.0,
             rho_ratio=1.2, g=1e-4, config_index=3, storage="f32"):
    """Uneven boxes of thermosensitive sphere sedimentation, one dict per box."""
    gen = rng(config_index)
    R = d / 2
    v_sphere = 4.0 / 3.0 * np.pi * R ** 3
    cases = []
    for b in range(n_boxes):
        n = int(gen.choice(edges))
        Ra = float(10.0 ** gen.uniform(np.log10(Ra_range[0]), np.log10(Ra_range[1])))
        n_p = int(gen.integers(n_range[0], n_range[1] + 1))
        n_p = min(n_p, int(0.12 * n ** 3 / v_sphere))
        lo = [R + 1.0] * 3
        hi = [n - 1.5 - R - 1.0] * 3
        X = rsa_positions(gen, n_p, R, lo, hi)
        Tp = gen.random(n_p)
        parts = dict(X=X, R=np.full(n_p, R), rho_p=np.full(n_p, rho_ratio), T_p=Tp,
                     heat_cap=np.full(n_p, rho_ratio * v_sphere))
        cases.append(_base(3, (n, n, n), Ra=Ra, particles=parts, contact=hertz(), g_particle=[0.0, 0.0, -g],
                           storage=storage, name=f"ens{b}_{n}^3_{n_p}p_Ra{Ra:.3g}"))
    return cases


def points(dim=2, shape=(96, 128, 1), n_p=200, d=0.5, rho_ratio=4.0, g=2e-4, config_index=5, storage="f32"):
    """Sub-grid point particles: the sedimentation recipe of the dimension with
    d <= 1 and particle_model "point" (one PIBM point per particle).  The
    explicit point coupling (A_p = pi d^2 / 4 against the mass) is stable for
    dense enough particles: in 3-D it needs about rho_p R > 3/4 (d = 0.5 at a
    density ratio of 1.5 blows up), hence the default ratio of 4."""
    if dim == 2:
        case = sed2d(nx=shape[0], ny=shape[1], n_p=n_p, d=d, rho_ratio=rho_ratio, g=g, config_index=config_index,
                     storage=storage)
    else:
        case = sed3d(nx=shape[0], ny=shape[1], nz=shape[2], n_p=n_p, d=d, rho_ratio=rho_ratio, g=g,
                     config_index=config_index, storage=storage)
    case["particle_model"] = "point"
    case["name"] = f"points{dim}d_{n_p}p"
    return case


def poiseuille(ny=16, nx=4, nu=np.sqrt(3.0 / 16.0) / 3.0, F=1e-6, dim=2, nz=1):
    """Channel periodic in x (and z), no-slip walls in y, constant body force along x."""
    walls = [(0, 0, 0.0), (0, 0, 0.0), (1, 0, 0.0), (1, 0, 0.0)]
    if dim == 3:
        walls += [(0, 0, 0.0), (0, 0, 0.0)]
    return _base(dim, (nx, ny, nz), Ra=1.0, Pr=1.0, U_c=nu, L_c=1.0, buoyancy=False,
                 body_force=[F, 0.0, 0.0], walls=walls, pibm=False, name="poiseuille")


def conduction(ny=16, nx=4, alpha=0.1, T_lo=1.0, T_hi=0.0, dim=2, nz=1):
    """Periodic in x (and z), isothermal walls in y, fluid at rest."""
    walls = [(0, 0, 0.0), (0, 0, 0.0), (1, 1, T_lo), (1, 1, T_hi)]
    if dim == 3:
        walls += [(0, 0, 0.0), (0, 0, 0.0)]
    nu = alpha  # Pr = 1
    return _base(dim, (nx, ny, nz), Ra=1.0, Pr=1.0, U_c=nu, L_c=1.0, buoyancy=False, T_init=0.5,
                 walls=walls, pibm=False, name="conduction")


def periodic_box(shape=(16, 12, 1), dim=2, buoyancy=True, body=(0.0, 0.0, 0.0)):
    walls = [(0, 0, 0.0)] * (2 * dim)
    return _base(dim, shape, U_c=0.05, L_c=float(shape[dim - 1]), buoyancy=buoyancy,
                 body_force=list(body), walls=walls, pibm=False, name="periodic")


def random_populations(case, config_index=7, amp=0.01):
    """Positive populations near rest equilibrium with seeded perturbations
    (for invariant tests): returns (f, g) in the [q][z][y][x] layout."""
    gen = rng(config_index)
    dim = case["dim"]
    nx, ny, nz = case["shape"]
    if dim == 2:
        w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
        wg = np.array([1 / 3] + [1 / 6] * 4)
    elif case.get("flow_q", 0) == 15:
        w = np.array([2 / 9] + [1 / 9] * 6 + [1 / 72] * 8)
        wg = np.array([1 / 4] + [1 / 8] * 6)
    else:
        w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
        wg = np.array([1 / 4] + [1 / 8] * 6)
    f = w[:, None, None, None] * (1.0 + amp * (gen.random((len(w), nz, ny, nx)) - 0.5))
    g = wg[:, None, None, None] * (0.5 + amp * (gen.random((len(wg), nz, ny, nx)) - 0.5))
    return f, g


def dense_pile(seed=71, law=1, mu=0.3):
    """DEM only: 7 x 7 x 6 spheres on a square lattice of spacing 4.98 resting on
    the floor of a 36 x 36 x 40 walled box, diameters 4.94 .. 5.02 (neighbours
    overlap by up to 0.04 or sit up to 0.04 apart), small random velocities and
    spins; Hertz E = 200, nu = 0.33, normal and tangential damping; gravity 1e-3
    along -z; no fluid coupling."""
    gen = rng(seed)
    nxs, nys, nzs, s, L = 7, 7, 6, 4.98, 36
    idx = np.array([(i, j, k) for k in range(nzs) for j in range(nys) for i in range(nxs)], dtype=float)
    n = len(idx)
    X = np.zeros((n, 3))
    X[:, 0] = (L - 1) / 2.0 + (idx[:, 0] - (nxs - 1) / 2.0) * s + 0.02 * (gen.random(n) - 0.5)
    X[:, 1] = (L - 1) / 2.0 + (idx[:, 1] - (nys - 1) / 2.0) * s + 0.02 * (gen.random(n) - 0.5)
    X[:, 2] = 2.0 + idx[:, 2] * s + 0.02 * (gen.random(n) - 0.5)
    U = gen.normal(size=(n, 3)) * 2e-3
    Wv = gen.normal(size=(n, 3)) * 1e-3
    R = 2.47 + 0.04 * rng(seed + 1).random(n)
    case = periodic_box(shape=(L, L, 40), dim=3, buoyancy=False)
    case.update(walls=[(1, 1, 0.0)] * 6, pibm=False, g_particle=[0.0, 0.0, -1e-3],
                contact=dict(hertz(E=200.0, poisson=0.33, mu=mu, gamma_n=10.0, gamma_t=2.0), law=law),
                particles=dict(X=X, U=U, W=Wv, R=R, rho_p=np.full(n, 1.5), T_p=np.zeros(n)),
                name=f"pile294_law{law}")
    return case


def colliding_gas(seed=5, n_p=160, L=56, speed=2e-2, law=2, mu=0.3):
    """DEM only: n_p spheres of radius 2.4 .. 2.5 placed at random (centres at
    least 5.3 apart) in an L^3 walled box, Gaussian velocities of scale `speed`
    and spins of scale 0.3 speed, no gravity, no fluid coupling: binary
    collisions with the wall and pair contacts of Hertz E = 200, nu = 0.33,
    normal and tangential damping."""
    gen = rng(seed)
    X = []
    while len(X) < n_p:
        x = 4 + (L - 9) * gen.random(3)
        if all(np.linalg.norm(x - y) > 5.3 for y in X):
            X.append(x)
    X = np.array(X)
    U = gen.normal(size=(n_p, 3)) * speed
    Wv = gen.normal(size=(n_p, 3)) * speed * 0.3
    R = 2.4 + 0.1 * gen.random(n_p)
    case = periodic_box(shape=(L, L, L), dim=3, buoyancy=False)
    case.update(walls=[(1, 1, 0.0)] * 6, pibm=False, g_particle=[0.0, 0.0, 0.0],
                contact=dict(hertz(E=200.0, poisson=0.33, mu=mu, gamma_n=10.0, gamma_t=2.0), law=law),
                particles=dict(X=X, U=U, W=Wv, R=R, rho_p=np.full(n_p, 1.5), T_p=np.zeros(n_p)),
                name=f"gas{n_p}_law{law}")
    return case
