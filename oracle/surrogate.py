"""Learned coupling surrogate: plain FP64 reference of everything the GPU
surrogate computes -- the per-particle feature map, the MLP (forward, loss,
backward, Adam), the BF16 inference arithmetic, the secant Jacobian used in
the DEM substeps, and the gate that falls back to the plain PIBM load.

TEST INFRASTRUCTURE ONLY: used by the tests and by nothing on the product
path; it shares no code with the CUDA library.

The surrogate is not in the paper.  It serves the momentum balance of Eq
demgov: the hydrodynamic force, torque and heat flux of a particle (Eq lbm13
and its torque / heat analogues) are computed once per lattice step by the
PIBM coupling and are held fixed over the DEM substeps; the surrogate
predicts how they change with the particle's own velocity and spin inside
the step.  The coupling acts on the fluid the particle covers (Eqs lbm7,
lbm8: F_f = 2 (rho U_l - j) on every covered node), so the velocity
features are taken against that fluid.  Definitions (lattice units):

  region S_p  the nodes particle p owns in the coupling: r inside the lattice
              with epsilon_p(r) = min(R_p + 1/2 - |r - X_p|, 1) > 0, and no
              other particle with a larger epsilon there (equal: the lower
              index owns it)
  raw fields  the moments before the coupling's correction, u = j / rho with
              rho = sum f, j = sum e f, and T0 = sum g (see raw_fields): the
              coupling acts on exactly these (F_f = 2 (rho U_l - j))
  V_s, Om_s   rigid-motion fit of the raw fluid velocity over S_p about X_p,
              weighted as the coupling weighs each node, w = epsilon rho:
              minimise sum w |u(r) - V - Om x d|^2, d = r - X_p; with m =
              sum w, D = sum w d, M = sum w (|d|^2 I - d d^T) the normal
              equations are
                  m V - D x Om = sum w u,   D x V + M Om = sum w d x u
              (w u = epsilon j; 2-D: unknowns V_x, V_y, Om_z); exact for any
              rigid field.  With these weights the coupling's load at a frozen
              fluid state is exactly linear in the velocity features:
                  F = -2 m (U_p - V_s) - 2 (omega_p - Om_s) x D,
                  tau = -2 D x (U_p - V_s) - 2 M (omega_p - Om_s)
  T_s         raw fluid temperature T0 averaged over S_p with weights
              epsilon; then H = 2 kappa_T (sum epsilon) (T_p - T_s)
  features    U_p - V_s (3), omega_p - Om_s (3), T_p - T_s (1),
              phi_p = sum_{q != p, |X_q - X_p| < 4 R_p} (R_q / 4 R_p)^D (1),
              the four smallest surface gaps |X_q - X_p| - R_p - R_q, each
              capped at 2 R_p and padded with 2 R_p (4)
  targets     the PIBM coupling's force (3), torque (3) and heat flux (1) of
              the state (Eq lbm13 and its analogues)
  network     12 -> 64 -> 64 -> 64 -> 7, tanh on the hidden layers, plus a
              linear path from the inputs to the outputs (y = W4 a3 + b4 +
              Ws x); inputs and outputs standardised with the training set's
              mean and standard deviation (a standard deviation below 1e-12
              counts as 1)
  training    the linear path and the output bias first by least squares
              over the training set (ridge 1e-8 per row), the hidden layers'
              output weights W4 zero; then every parameter by Adam on the
              mean squared standardised error
  Jacobian    secant over delta standard deviations of each of the six
              velocity / spin features and of the temperature feature (in the
              BF16 inference, delta is widened to two BF16 spacings of the
              feature and the secant divides by the BF16 inputs' difference):
              J_FU[a][b] = dF_a / dU_b, J_TW[a][b] = dtau_a / domega_b of the
              coupling and J_HT = dH / dT_p; the DEM holds the mean of the
              couplings of t and t-1 and a change of the particle's state
              enters only the newer one, so it applies half of each
              (applied_jacobian); a block that cannot be physical for an
              explicit substep is zeroed (admissible); 19 values per particle
  gate        e = sum_p |F_mlp,p - F_pibm,p| / sum_p |F_pibm,p|; the
              Jacobian is applied in the next step only when e <= bound
"""
from __future__ import annotations

import numpy as np

N_FEAT, N_OUT, WIDTH = 12, 7, 64
SIZES = [(N_FEAT, WIDTH), (WIDTH, WIDTH), (WIDTH, WIDTH), (WIDTH, N_OUT)]


# ------------------------------------------------------------------ features
_E2 = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (-1, 0, 0), (0, -1, 0), (1, 1, 0), (-1, 1, 0), (-1, -1, 0), (1, -1, 0)]
_E3 = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
       (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1),
       (1, 0, -1), (-1, 0, 1), (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]


def raw_fields(f, g, dim):
    """rho = sum f, u = (sum e f) / rho, T = sum g from full populations
    f [q][z][y][x] (D2Q9 / D3Q19 in the oracle's direction order) and g."""
    E = np.asarray(_E2 if dim == 2 else _E3, dtype=np.float64)
    rho = f.sum(axis=0)
    j = np.einsum("qa,q...->a...", E, f)
    return {"rho": rho, "ux": j[0] / rho, "uy": j[1] / rho, "uz": j[2] / rho, "T": g.sum(axis=0)}


def region(X, R, shape_xyz, dim):
    """Integer node coordinates (k, 3) of the covered nodes |r - X| < R + 1/2."""
    lo = np.floor(np.asarray(X[:dim]) - R - 1).astype(int)
    hi = np.ceil(np.asarray(X[:dim]) + R + 1).astype(int)
    axes = [np.arange(max(lo[a], 0), min(hi[a], shape_xyz[a] - 1) + 1) for a in range(dim)]
    grid = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, dim)
    d = grid - np.asarray(X[:dim])[None, :]
    r = np.sqrt(np.sum(d * d, axis=1))
    sel = r < R + 0.5
    out = np.zeros((int(sel.sum()), 3), dtype=np.int64)
    out[:, :dim] = grid[sel]
    return out


def _eps(nodes, Xq, Rq, dim):
    d = nodes[:, :dim].astype(np.float64) - np.asarray(Xq[:dim])[None, :]
    e = (Rq + 0.5) - np.sqrt(np.sum(d * d, axis=1))
    return np.minimum(e, 1.0)


def owned(nodes, p, X, R, dim):
    """The rows of nodes (covered by p) that p owns against the other particles."""
    ep = _eps(nodes, X[p], R[p], dim)
    keep = ep > 0
    for q in range(len(R)):
        if q == p or np.linalg.norm(np.asarray(X[q][:dim]) - np.asarray(X[p][:dim])) >= R[p] + R[q] + 2:
            continue
        eq = _eps(nodes, X[q], R[q], dim)
        keep &= ~((eq > ep) | ((eq == ep) & (q < p)))
    return nodes[keep]


def features(fields, X, U, W, R, Tp, dim):
    """fields: dict with rho, ux, uy, uz (3-D), T as (nz, ny, nx) arrays."""
    n = len(R)
    nz, ny, nx = fields["T"].shape
    out = np.zeros((n, N_FEAT))
    uz = fields.get("uz", np.zeros_like(fields["T"]))
    for p in range(n):
        nodes = owned(region(X[p], R[p], (nx, ny, nz), dim), p, X, R, dim)
        x, y, z = nodes[:, 0], nodes[:, 1], nodes[:, 2]
        eps = np.minimum(_eps(nodes, X[p], R[p], dim), 1.0)
        w = eps * fields["rho"][z, y, x]
        u = np.stack([fields["ux"][z, y, x], fields["uy"][z, y, x], uz[z, y, x]], axis=1)
        Ts = np.sum(eps * fields["T"][z, y, x]) / np.sum(eps)
        d = nodes.astype(np.float64) - np.asarray(X[p])[None, :]
        if dim == 2:
            d[:, 2] = 0.0
        m = np.sum(w)
        D = (w[:, None] * d).sum(axis=0)
        su = (w[:, None] * u).sum(axis=0)
        sdu = (w[:, None] * np.cross(d, u)).sum(axis=0)
        if dim == 3:
            M = np.sum(w * np.sum(d * d, axis=1)) * np.eye(3) - (w[:, None] * d).T @ d
            Dx = np.array([[0, -D[2], D[1]], [D[2], 0, -D[0]], [-D[1], D[0], 0]])
            A = np.block([[m * np.eye(3), -Dx], [Dx, M]])
            sol = np.linalg.solve(A, np.concatenate([su, sdu]))
            V, Om = sol[:3], sol[3:]
        else:
            A = np.array([[m, 0.0, -D[1]], [0.0, m, D[0]], [-D[1], D[0], np.sum(w * np.sum(d * d, axis=1))]])
            sol = np.linalg.solve(A, np.array([su[0], su[1], sdu[2]]))
            V, Om = np.array([sol[0], sol[1], 0.0]), np.array([0.0, 0.0, sol[2]])
        out[p, 0:3] = np.asarray(U[p]) - V
        out[p, 3:6] = np.asarray(W[p]) - Om
        out[p, 6] = Tp[p] - Ts
        dist = np.sqrt(np.sum((np.asarray(X) - np.asarray(X[p])[None, :]) ** 2, axis=1))
        others = np.arange(n) != p
        near = others & (dist < 4 * R[p])
        out[p, 7] = np.sum((np.asarray(R)[near] / (4 * R[p])) ** dim)
        gaps = np.sort(dist[others] - R[p] - np.asarray(R)[others])
        cap = 2 * R[p]
        g4 = np.full(4, cap)
        k = min(4, len(gaps))
        g4[:k] = np.minimum(gaps[:k], cap)
        out[p, 8:12] = g4
    return out


def targets(F, T, H):
    return np.concatenate([np.asarray(F), np.asarray(T), np.asarray(H)[:, None]], axis=1)


# ---------------------------------------------------------------- the network
# params: [(W1, b1), (W2, b2), (W3, b3), (W4, b4), (Ws, [])] with W[out][in];
# Ws (7 x 12) is the linear path from the inputs to the outputs
def init_params(seed):
    """Glorot-uniform weights, zero biases, zero linear path."""
    gen = np.random.Generator(np.random.PCG64(seed))
    params = []
    for fi, fo in SIZES:
        lim = np.sqrt(6.0 / (fi + fo))
        params.append((gen.uniform(-lim, lim, size=(fo, fi)), np.zeros(fo)))
    params.append((np.zeros((N_OUT, N_FEAT)), np.zeros(0)))
    return params


def flatten(params):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params])


def unflatten(vec):
    params, k = [], 0
    for fi, fo in SIZES:
        W = np.asarray(vec[k:k + fo * fi], dtype=np.float64).reshape(fo, fi)
        k += fo * fi
        b = np.asarray(vec[k:k + fo], dtype=np.float64)
        k += fo
        params.append((W, b))
    params.append((np.asarray(vec[k:k + N_OUT * N_FEAT], dtype=np.float64).reshape(N_OUT, N_FEAT), np.zeros(0)))
    return params


N_PARAMS = sum(fo * fi + fo for fi, fo in SIZES) + N_OUT * N_FEAT


def standardise(A):
    mu = A.mean(axis=0)
    sd = A.std(axis=0)
    sd = np.where(sd < 1e-12, 1.0, sd)
    return mu, sd


def forward(params, Xn):
    """Returns the list of layer outputs [x, a1, a2, a3, y] (FP64)."""
    acts = [Xn]
    a = Xn
    for l in range(3):
        W, b = params[l]
        a = np.tanh(a @ W.T + b)
        acts.append(a)
    W4, b4 = params[3]
    Ws = params[4][0]
    acts.append(a @ W4.T + b4 + Xn @ Ws.T)
    return acts


def loss_and_grads(params, Xn, Yn):
    """Mean squared standardised error and its gradient (backpropagation)."""
    acts = forward(params, Xn)
    B = Xn.shape[0]
    diff = acts[-1] - Yn
    loss = float(np.mean(diff * diff))
    delta = 2.0 * diff / (B * Yn.shape[1])          # dL/dy
    grads = [None] * 5
    grads[4] = (delta.T @ Xn, np.zeros(0))           # the linear path
    for l in range(3, -1, -1):
        W, _ = params[l]
        grads[l] = (delta.T @ acts[l], delta.sum(axis=0))
        if l > 0:
            delta = (delta @ W) * (1.0 - acts[l] ** 2)  # through tanh of layer l-1's output
    return loss, grads


def linear_fit(params, Xn, Yn, ridge=1e-8):
    """The linear path and output bias by least squares over the rows, the
    output weights W4 zero: minimise |[Xn 1] C - Yn|^2 + ridge B |C|^2."""
    B = Xn.shape[0]
    A = np.concatenate([Xn, np.ones((B, 1))], axis=1)
    C = np.linalg.solve(A.T @ A + ridge * B * np.eye(N_FEAT + 1), A.T @ Yn)
    out = [(W.copy(), b.copy()) for W, b in params[:3]]
    out.append((np.zeros_like(params[3][0]), C[N_FEAT].copy()))
    out.append((C[:N_FEAT].T.copy(), np.zeros(0)))
    return out


def adam(params, grads, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns new params, m, v."""
    out_p, out_m, out_v = [], [], []
    for (W, b), (gW, gb), (mW, mb), (vW, vb) in zip(params, grads, m, v):
        new = []
        for x, g, mm, vv in ((W, gW, mW, vW), (b, gb, mb, vb)):
            mm = b1 * mm + (1 - b1) * g
            vv = b2 * vv + (1 - b2) * g * g
            mh = mm / (1 - b1 ** t)
            vh = vv / (1 - b2 ** t)
            new.append((x - lr * mh / (np.sqrt(vh) + eps), mm, vv))
        out_p.append((new[0][0], new[1][0]))
        out_m.append((new[0][1], new[1][1]))
        out_v.append((new[0][2], new[1][2]))
    return out_p, out_m, out_v


# ------------------------------------------------------- BF16 inference model
def to_bf16(a):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    a32 = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    bits = a32.view(np.uint32).astype(np.uint64)
    bits = (bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(params, Xn):
    """The tensor-core inference arithmetic: BF16 inputs, weights and hidden
    activations, wide accumulation, FP32 bias and tanh, FP32 output."""
    x = to_bf16(Xn)
    a = x
    for l in range(3):
        W, b = params[l]
        a = to_bf16(np.tanh(a @ to_bf16(W).T + np.asarray(b, dtype=np.float32).astype(np.float64)))
    W4, b4 = params[3]
    return a @ to_bf16(W4).T + x @ to_bf16(params[4][0]).T + np.asarray(b4, dtype=np.float32).astype(np.float64)


ROWS = 8  # rows per particle in the Jacobian: the state, six velocity / spin and one temperature perturbation


def secant_steps(Xn, delta):
    """The secant step of each standardised feature: delta, widened to two BF16
    spacings of the feature's value where that is larger (the network takes its
    inputs in BF16, and a smaller step would vanish for features far out in the
    tails).  Computed in FP32, as the device does."""
    x = np.asarray(Xn, dtype=np.float32)
    _, e = np.frexp(x)                                   # |x| in [2^(e-1), 2^e)
    two_spacings = np.ldexp(np.float32(1.0), e - 7).astype(np.float32)
    return np.where(x == 0, np.float32(delta), np.maximum(np.float32(delta), two_spacings)).astype(np.float32)


def jacobian(params, xmu, xsd, ymu, ysd, Xraw, delta=0.25, infer=forward):
    """Secant Jacobian of (F, tau) in (U, omega) and of H in T_p, and the value
    row.  Returns (Y (n, 7) de-standardised, J (n, 19): J_FU row-major, J_TW
    row-major, J_HT).  With infer=forward_bf16 (the tensor-core arithmetic) the
    rows are formed in FP32, the steps widened by secant_steps, and each secant
    divided by the difference of its two BF16 inputs, as on the device."""
    bf16 = infer is forward_bf16
    Xn = (Xraw - xmu) / xsd
    if bf16:
        Xn = Xn.astype(np.float32)
    n = Xn.shape[0]
    rows = np.repeat(Xn, ROWS, axis=0)
    step = secant_steps(Xn, delta) if bf16 else np.full(Xn.shape, delta)
    for j in range(7):
        rows[j + 1::ROWS, j] = (rows[j + 1::ROWS, j] + step[:, j]).astype(rows.dtype)
    Yn = infer(params, rows.astype(np.float64)) if infer is not forward else forward(params, rows)[-1]
    Y = Yn * ysd + ymu
    Y = Y.reshape(n, ROWS, N_OUT)
    base = Y[:, 0, :]
    if bf16:
        x32 = Xn[:, :7].astype(np.float32)
        dq = (to_bf16((x32 + step[:, :7]).astype(np.float32)) - to_bf16(x32)) * np.asarray(xsd[:7])
    else:
        dq = np.broadcast_to(delta * np.asarray(xsd[:7]), (n, 7))
    J = np.zeros((n, 19))
    for b in range(3):
        J[:, b:9:3] = (Y[:, 1 + b, 0:3] - base[:, 0:3]) / dq[:, b:b + 1]
        J[:, 9 + b:18:3] = (Y[:, 4 + b, 3:6] - base[:, 3:6]) / dq[:, 3 + b:4 + b]
    J[:, 18] = (Y[:, 7, 6] - base[:, 6]) / dq[:, 6]
    return base, J


def admissible(J, mass, inertia, h, dim):
    """Zero each Jacobian block (J_FU, J_TW; the axes that can move: x, y for
    J_FU and z for J_TW in 2-D) that cannot be physical for an explicit substep:
    a diagonal entry above 0, a row not diagonally dominant (then an eigenvalue
    could have a positive real part), or |J_aa| h >= 2 m, m the mass (or the
    moment of inertia), beyond which the substep kick is unstable."""
    J = np.array(J, dtype=np.float64)
    for p in range(J.shape[0]):
        for off, lo, hi, m in ((0, 0, 2 if dim == 3 else 1, mass[p]), (9, 0 if dim == 3 else 2, 2, inertia[p])):
            B = J[p, off:off + 9].reshape(3, 3)
            ok = True
            for a in range(lo, hi + 1):
                d = B[a, a]
                rest = sum(abs(B[a, b]) for b in range(lo, hi + 1) if b != a)
                if not (d <= 0) or not (rest <= -d) or not (-d * h < 2 * m):
                    ok = False
            if not ok:
                J[p, off:off + 9] = 0.0
    return J


def applied_jacobian(J):
    """The Jacobian the DEM applies to the held load (half the coupling's)."""
    return 0.5 * np.asarray(J)


def gate_error(F_mlp, F_pibm):
    num = np.sum(np.sqrt(np.sum((F_mlp - F_pibm) ** 2, axis=1)))
    den = np.sum(np.sqrt(np.sum(F_pibm ** 2, axis=1)))
    return float(num / den) if den > 0 else float("inf")
