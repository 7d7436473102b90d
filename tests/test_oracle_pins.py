"""Pins for the CPU oracle against facts that do not come from the oracle itself:
linear elasticity at rest, frame invariance, finite differences, brute-force
distance minimisation, closed-form special cases, Coulomb's law, and
closed-form motion (free fall, static rest, inclined plane)."""
import math

import numpy as np
import pytest

from oracle import ipc
from paper_2609_25653_b300 import scenes
from tests.conftest import random_rotation

E_Y, NU = 1e5, 0.45
MU = E_Y / (2 * (1 + NU))
LAME = E_Y * NU / ((1 + NU) * (1 - 2 * NU))   # first Lame parameter
LAM = ipc.snh_params(E_Y, NU)[1]              # model parameter of the Neo-Hookean form


def fd_grad(f, x, h):
    g = np.zeros_like(x)
    for i in range(x.size):
        e = np.zeros_like(x); e[i] = h
        g[i] = (f(x + e) - f(x - e)) / (2 * h)
    return g


def fd_jac(f, x, h):
    cols = []
    for i in range(x.size):
        e = np.zeros_like(x); e[i] = h
        cols.append((f(x + e) - f(x - e)) / (2 * h))
    return np.stack(cols, axis=1)


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


# --------------------------------------------------------------------------
# Stable Neo-Hookean (§III-C.1)
# --------------------------------------------------------------------------

def test_snh_rest_and_rotations_are_stress_free(gen):
    for F in [np.eye(3)] + [random_rotation(gen) for _ in range(5)]:
        psi, P, _ = ipc.snh(F, MU, LAM)
        assert abs(psi) < 1e-9 * MU
        assert np.max(np.abs(P)) < 1e-9 * MU


def test_snh_hessian_at_rest_is_linear_elasticity():
    """At F = I the tangent must be the isotropic tensor mu(d_ik d_jl + d_il d_jk) + lam d_ij d_kl."""
    _, _, H = ipc.snh(np.eye(3), MU, LAM)
    Cten = np.zeros((9, 9))
    for i in range(3):
        for j in range(3):
            for k in range(3):
                for l in range(3):
                    v = MU * ((i == k) * (j == l) + (i == l) * (j == k)) + LAME * (i == j) * (k == l)
                    Cten[3 * j + i, 3 * l + k] = v
    assert rel(H, Cten) < 1e-12


def test_snh_uniaxial_small_strain_recovers_young_and_poisson():
    """Small uniaxial stretch with free lateral faces: P_xx / eps -> E and -eps_lat / eps -> nu."""
    eps = 1e-7
    def lateral_stress(d):
        return ipc.snh(np.diag([1 + eps, 1 + d, 1 + d]), MU, LAM)[1][1, 1]
    lo, hi = -2 * eps, 0.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if lateral_stress(mid) > 0:
            hi = mid
        else:
            lo = mid
    d = 0.5 * (lo + hi)
    Pxx = ipc.snh(np.diag([1 + eps, 1 + d, 1 + d]), MU, LAM)[1][0, 0]
    assert abs(-d / eps - NU) < 1e-5
    assert abs(Pxx / eps - E_Y) / E_Y < 1e-5


def test_snh_frame_invariance(gen):
    F = np.eye(3) + 0.3 * gen.normal(size=(3, 3))
    R = random_rotation(gen)
    a = ipc.snh(F, MU, LAM)[0]
    b = ipc.snh(R @ F, MU, LAM)[0]
    assert abs(a - b) < 1e-10 * abs(a)


def test_snh_fd(gen):
    for _ in range(5):
        F = np.eye(3) + 0.4 * gen.normal(size=(3, 3))
        vecF = F.T.reshape(-1)  # column-major vec
        f = lambda v: ipc.snh(v.reshape(3, 3).T, MU, LAM)[0]
        P = lambda v: ipc.snh(v.reshape(3, 3).T, MU, LAM)[1].T.reshape(-1)
        _, Pa, Ha = ipc.snh(F, MU, LAM)
        assert rel(fd_grad(f, vecF, 1e-6), Pa.T.reshape(-1)) < 1e-7
        assert rel(fd_jac(P, vecF, 1e-6), Ha) < 1e-7


def test_snh_inverted_is_defined():
    psi, P, H = ipc.snh(np.diag([1.0, 1.0, -0.5]), MU, LAM)
    assert np.isfinite(psi) and np.all(np.isfinite(P)) and np.all(np.isfinite(H))


def _random_tet(gen, scale=1e-3):
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]]) * scale + 0.1 * scale * gen.normal(size=(4, 3))
    Dm = np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], axis=1)
    if np.linalg.det(Dm) < 0:
        X[[1, 2]] = X[[2, 1]]
        Dm = np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], axis=1)
    return X, np.linalg.inv(Dm), np.linalg.det(Dm) / 6


def test_tet_rest_rigid_and_momentum(gen):
    X, B, V = _random_tet(gen)
    for _ in range(3):
        R = random_rotation(gen)
        x = X @ R.T + gen.normal(size=3)
        E, g, _ = ipc.tet(x, B, V, MU, LAM)
        assert abs(E) < 1e-12 * MU * V and np.max(np.abs(g)) < 1e-8 * MU * V / 1e-3
    x = X + 2e-4 * gen.normal(size=(4, 3))
    E, g, _ = ipc.tet(x, B, V, MU, LAM)
    g4 = g.reshape(4, 3)
    scale = np.abs(g4).max()
    assert np.abs(g4.sum(0)).max() < 1e-10 * scale                    # translation invariance
    assert np.abs(np.cross(x, g4).sum(0)).max() < 1e-10 * scale * 1e-3  # rotation invariance


def test_tet_fd(gen):
    X, B, V = _random_tet(gen)
    x = (X + 2e-4 * gen.normal(size=(4, 3))).reshape(-1)
    E, g, H = ipc.tet(x, B, V, MU, LAM)
    assert rel(fd_grad(lambda y: ipc.tet(y, B, V, MU, LAM)[0], x, 1e-8), g) < 1e-6
    assert rel(fd_jac(lambda y: ipc.tet(y, B, V, MU, LAM)[1], x, 1e-8), H) < 1e-6


def test_psd_projection(gen):
    for n in (9, 12):
        A = gen.normal(size=(n, n)); A = A + A.T
        P = ipc.project_psd(A)
        w, V = np.linalg.eigh(A)
        ref = (V * np.maximum(w, 0)) @ V.T        # independent eigen-solver
        assert rel(P, ref) < 1e-12
        assert np.linalg.eigvalsh(P).min() > -1e-12 * np.abs(A).max()
        B = A @ A.T                                # already PSD: unchanged
        assert rel(ipc.project_psd(B), B) < 1e-12
    X, Bm, V = _random_tet(gen)
    _, _, H = ipc.tet(X, Bm, V, MU, LAM, project=False)
    _, _, Hp = ipc.tet(X, Bm, V, MU, LAM, project=True)
    assert rel(Hp, H) < 1e-10  # at rest the Hessian is PSD


# --------------------------------------------------------------------------
# distances
# --------------------------------------------------------------------------

def brute_pt(x, n=200):
    p, a, b, c = x.reshape(4, 3)
    best = math.inf
    u = np.linspace(0, 1, n + 1)
    U, W = np.meshgrid(u, u, indexing="ij")
    m = U + W <= 1
    pts = a + U[m, None] * (b - a) + W[m, None] * (c - a)
    best = np.min(np.sum((pts - p) ** 2, axis=1))
    for e0, e1 in ((a, b), (b, c), (c, a)):
        t = np.clip(np.dot(p - e0, e1 - e0) / np.dot(e1 - e0, e1 - e0), 0, 1)
        best = min(best, np.sum((e0 + t * (e1 - e0) - p) ** 2))
    return best


def brute_ee(x, n=400):
    a0, a1, b0, b1 = x.reshape(4, 3)
    u = np.linspace(0, 1, n + 1)
    A = a0 + u[:, None] * (a1 - a0)
    Bp = b0 + u[:, None] * (b1 - b0)
    return np.min(np.sum((A[:, None, :] - Bp[None, :, :]) ** 2, axis=2))


def test_pt_classify_matches_brute_force(gen):
    for _ in range(60):
        x = gen.normal(size=12)
        t, s, w = ipc.classify(0, x)
        sb = brute_pt(x)
        assert s <= sb * (1 + 1e-9) + 1e-15
        assert s >= sb - 1e-3 * sb - 1e-4  # grid resolution
        # weights reproduce the closest-point difference
        d = (w[:, None] * x.reshape(4, 3)).sum(0)
        assert abs(d @ d - s) < 1e-9 * max(s, 1e-12)


def test_ee_classify_matches_brute_force(gen):
    for _ in range(60):
        x = gen.normal(size=12)
        t, s, w = ipc.classify(1, x)
        sb = brute_ee(x)
        assert s <= sb * (1 + 1e-9) + 1e-15
        assert s >= sb - 2e-2 * sb - 1e-4
        d = (w[:, None] * x.reshape(4, 3)).sum(0)
        assert abs(d @ d - s) < 1e-9 * max(s, 1e-12)


def test_distance_special_cases():
    # point above the interior of a triangle: squared height
    x = np.array([0.2, 0.3, 0.7, 0, 0, 0, 1, 0, 0, 0, 1, 0.0])
    t, s, _ = ipc.classify(0, x)
    assert t == 6 and abs(s - 0.49) < 1e-15
    # crossing edges at height h: line-line distance
    x = np.array([-1, 0, 0.25, 1, 0, 0.25, 0, -1, 0, 0, 1, 0.0])
    t, s, _ = ipc.classify(1, x)
    assert t == 8 and abs(s - 0.0625) < 1e-15
    # parallel overlapping edges: distance between the lines, endpoint type
    x = np.array([0, 0, 0, 2, 0, 0, 1, 0.5, 0, 3, 0.5, 0.0])
    t, s, _ = ipc.classify(1, x)
    assert t != 8 and abs(s - 0.25) < 1e-15


@pytest.mark.parametrize("kind,ntypes", [(0, 7), (1, 9)])
def test_distance_fd_all_types(gen, kind, ntypes):
    f = ipc.pt_dist if kind == 0 else ipc.ee_dist
    for t in range(ntypes):
        x = gen.normal(size=12)
        s, g, H = f(x, t)
        assert rel(fd_grad(lambda y: f(y, t)[0], x, 1e-6), g) < 1e-7
        assert rel(fd_jac(lambda y: f(y, t)[1], x, 1e-6), H) < 1e-6


# --------------------------------------------------------------------------
# barrier, mollifier, pair energy
# --------------------------------------------------------------------------

def test_barrier_shape():
    sh = 1e-6
    b, b1, b2 = ipc.barrier(sh, sh)
    assert b == 0 and b1 == 0
    b, b1, b2 = ipc.barrier(sh * (1 - 1e-9), sh)
    assert abs(b) < 1e-25 and abs(b1) < 1e-14
    assert ipc.barrier(1e-20, sh)[0] > ipc.barrier(1e-12, sh)[0] > ipc.barrier(1e-8, sh)[0] > 0
    for s in (1e-9, 3e-7, 9e-7):
        h = s * 1e-6
        assert abs((ipc.barrier(s + h, sh)[0] - ipc.barrier(s - h, sh)[0]) / (2 * h) - ipc.barrier(s, sh)[1]) < 1e-6 * abs(ipc.barrier(s, sh)[1])
        assert abs((ipc.barrier(s + h, sh)[1] - ipc.barrier(s - h, sh)[1]) / (2 * h) - ipc.barrier(s, sh)[2]) < 1e-5 * abs(ipc.barrier(s, sh)[2])
        assert ipc.barrier(s, sh)[2] > 0  # convex in s


def test_mollifier(gen):
    x = gen.normal(size=12)
    a = x[3:6] - x[0:3]; b = x[9:12] - x[6:9]
    c = np.sum(np.cross(a, b) ** 2)
    assert ipc.ee_mollifier(x, 0.5 * c)[0] == 1.0
    m, g, H = ipc.ee_mollifier(x, 2 * c)
    assert abs(m - 0.75) < 1e-12  # -r^2 + 2r at r = 1/2
    assert rel(fd_grad(lambda y: ipc.ee_mollifier(y, 2 * c)[0], x, 1e-6), g) < 1e-7
    assert rel(fd_jac(lambda y: ipc.ee_mollifier(y, 2 * c)[1], x, 1e-6), H) < 1e-6
    # C1 at the threshold: slope of m(c) is 0 at c = eps
    m_lo = ipc.ee_mollifier(x, c * (1 + 1e-7))[0]
    assert abs(m_lo - 1.0) < 1e-12


def test_pair_fd(gen):
    sh = 1.0
    for kind in (0, 1):
        for trial in range(6):
            while True:
                x = 0.4 * gen.normal(size=12)
                t, s, _ = ipc.classify(kind, x)
                if 0.05 < s < 0.8:
                    break
            a = x[3:6] - x[0:3]; b = x[9:12] - x[6:9]
            epsx = 2.0 * np.sum(np.cross(a, b) ** 2) if kind == 1 else 1.0
            E, g, H = ipc.pair(kind, t, x, sh, 3.0, epsx)
            f = lambda y: ipc.pair(kind, t, y, sh, 3.0, epsx)[0]
            gf = lambda y: ipc.pair(kind, t, y, sh, 3.0, epsx)[1]
            assert rel(fd_grad(f, x, 1e-6), g) < 1e-6
            assert rel(fd_jac(gf, x, 1e-6), H) < 1e-5
            _, _, Hp = ipc.pair(kind, t, x, sh, 3.0, epsx, project=True)
            assert np.linalg.eigvalsh(Hp).min() > -1e-10 * np.abs(Hp).max()


# --------------------------------------------------------------------------
# friction (Coulomb's law and smoothness)
# --------------------------------------------------------------------------

def test_friction_coulomb_and_fd(gen):
    n = np.array([0, 0, 1.0])
    w = np.array([1.0, -0.2, -0.3, -0.5])
    xt = gen.normal(size=12)
    lam, mu, eps = 2.0, 0.4, 1e-3
    # sliding: tangential force magnitude mu * lam, normal component zero
    x = xt.copy(); x[0:3] += [0.01, 0.02, 0.05]
    E, g, H = ipc.friction(w, n, lam, mu, eps, x, xt)
    fp = g[0:3]
    assert abs(np.linalg.norm(fp) - mu * lam) < 1e-12 and abs(fp[2]) < 1e-15
    for du in ([3e-4, -2e-4, 1e-4], [0.02, 0.01, -0.3]):
        x = xt.copy(); x[0:3] += du
        E, g, H = ipc.friction(w, n, lam, mu, eps, x, xt)
        assert rel(fd_grad(lambda y: ipc.friction(w, n, lam, mu, eps, y, xt)[0], x, 1e-8), g) < 1e-6
        assert rel(fd_jac(lambda y: ipc.friction(w, n, lam, mu, eps, y, xt)[1], x, 1e-8), H) < 1e-5
        assert np.linalg.eigvalsh(H).min() > -1e-10 * np.abs(H).max()


# --------------------------------------------------------------------------
# additive CCD
# --------------------------------------------------------------------------

def test_accd_point_toward_plane():
    x = np.array([0.2, 0.3, 1.0, 0, 0, 0, 1, 0, 0, 0, 1, 0.0])
    p = np.zeros(12); p[2] = -4.0          # analytic contact at t* = 0.25
    t = ipc.accd(0, x, p, 0.1, 1.0)
    assert 0 < t <= 0.25 * 0.9 + 1e-15      # stops before the 10 % separation
    assert 1.0 - 4.0 * t >= 0.1 * 1.0 - 1e-12
    assert t >= 0.25 * 0.5                 # and reaches a useful fraction
    p[2] = -0.5                            # contact beyond the step: full step
    assert ipc.accd(0, x, p, 0.1, 1.0) == 1.0


def test_accd_conservative_random(gen):
    for kind in (0, 1):
        for _ in range(40):
            x = gen.normal(size=12)
            p = 3 * gen.normal(size=12)
            t = ipc.accd(kind, x, p, 0.1, 1.0)
            s0 = ipc.classify(kind, x)[1]
            ts = np.linspace(0, t, 200)
            dmin = min(math.sqrt(ipc.classify(kind, x + tt * p)[1]) for tt in ts)
            assert dmin >= 0.1 * math.sqrt(s0) * (1 - 1e-9) - 1e-12


# --------------------------------------------------------------------------
# ABD (§III-C.1, "affine body dynamics with a stiff orthogonality energy")
# --------------------------------------------------------------------------

def test_abd_moments_of_box():
    X, T = scenes.box_surface((-1.0, -2.0, -0.5), (3.0, 1.0, 2.5))
    vol, first, second = ipc.closed_mesh_moments(X, T)
    lx, ly, lz = 4.0, 3.0, 3.0
    c = np.array([1.0, -0.5, 1.0])
    assert abs(vol - lx * ly * lz) < 1e-12
    assert np.allclose(first, vol * c, rtol=0, atol=1e-12)
    cov = np.diag([lx ** 2, ly ** 2, lz ** 2]) * vol / 12.0 + vol * np.outer(c, c)
    assert np.allclose(second, cov, rtol=0, atol=1e-11)


def test_abd_orthogonality(gen):
    R = random_rotation(gen)
    a = R.T.reshape(-1)  # columns of R
    E, g, _ = ipc.abd_orth(a, 5.0)
    assert abs(E) < 1e-24 and np.max(np.abs(g)) < 1e-12
    a = a + 0.1 * gen.normal(size=9)
    E, g, H = ipc.abd_orth(a, 5.0)
    assert rel(fd_grad(lambda y: ipc.abd_orth(y, 5.0)[0], a, 1e-6), g) < 1e-7
    assert rel(fd_jac(lambda y: ipc.abd_orth(y, 5.0)[1], a, 1e-6), H) < 1e-7


# --------------------------------------------------------------------------
# whole steps
# --------------------------------------------------------------------------

def test_free_fall_is_exact():
    sc = scenes.free_block(n_steps=4, v0=(0.1, -0.2, 0.3))
    o = ipc.Oracle(sc, tol=1e-12)
    X0 = o.x().copy()
    dt = sc["params"]["dt"]
    v = np.array([0.1, -0.2, 0.3])
    x = X0.copy()
    for _ in range(4):
        o.step()
        v = v + dt * sc["gravity"]
        x = x + dt * v
        assert np.max(np.abs(o.x() - x)) < 1e-14
        assert np.max(np.abs(o.zd.reshape(-1, 3) - v)) < 1e-11


def test_abd_free_fall_is_exact():
    X, T = scenes.box_surface((-1e-3, -1e-3, -1e-3), (1e-3, 1e-3, 1e-3))
    R = random_rotation(np.random.default_rng(3))
    q0 = np.concatenate([[0.0, 0.0, 0.5], R[:, 0], R[:, 1], R[:, 2]])
    sc = scenes.free_block(n_steps=3)
    sc["abd"] = [dict(X=X, tris=T, rho=1000.0, q0=q0)]
    o = ipc.Oracle(sc, tol=1e-12)
    dt = sc["params"]["dt"]
    for k in range(3):
        o.step()
    nf = o.S.n_fem_dof
    q = o.z[nf:nf + 12]
    t = 3 * dt
    # p(t) = p0 + g dt^2 (1 + 2 + 3) for implicit Euler from rest; A unchanged
    p_exp = q0[:3] + sc["gravity"] * dt * dt * 6
    assert np.max(np.abs(q[:3] - p_exp)) < 1e-14
    assert np.max(np.abs(q[3:] - q0[3:])) < 1e-12


@pytest.mark.slow
def test_rest_on_plane_supports_weight():
    sc = scenes.block_on_plane(n_steps=40, tilt=0.0, mu=0.0)
    o = ipc.Oracle(sc, tol=1e-10)
    for _ in range(40):
        o.step()
    v = o.zd.reshape(-1, 3)[:o.S.nf]
    assert np.max(np.abs(v)) < 2e-3
    # contact force balances gravity: the barrier gradient sums to m g
    x = o.x().reshape(-1)
    rec, s = o.S.active_pairs(x)
    assert len(rec) > 0 and s.min() > 0
    F = np.zeros(3)
    for k in range(len(rec)):
        kind, _, _, t = (int(c) for c in rec[k, :4])
        ids = rec[k, 4:8]
        _, g, _ = ipc.pair(kind, t, o.x()[ids], o.S.sh, o.S.kappa, o.S.eps_x(rec[k:k + 1])[0])
        for j, vid in enumerate(ids):
            if vid < o.S.nf:
                F -= g[3 * j:3 * j + 3]
    m = o.S.mass_v.sum()
    assert abs(F[2] - m * 9.81) < 0.02 * m * 9.81
    assert abs(F[0]) < 1e-3 * m * 9.81 and abs(F[1]) < 1e-3 * m * 9.81


@pytest.mark.slow
@pytest.mark.parametrize("mu,expect_slide", [(0.6, False), (0.1, True)])
def test_inclined_plane_friction(mu, expect_slide):
    theta = math.atan(0.3)  # tan(theta) = 0.3
    n_steps = 30
    sc = scenes.block_on_plane(n_steps=n_steps, tilt=theta, mu=mu)
    o = ipc.Oracle(sc, tol=1e-9)
    com = []
    for _ in range(n_steps):
        o.step()
        com.append(o.x()[:o.S.nf].mean(0))
    com = np.array(com)
    down = np.array([math.cos(theta), 0.0, -math.sin(theta)])  # downhill direction of the tilted plane
    s = (com - com[0]) @ down
    dt = sc["params"]["dt"]
    T = (n_steps - 1) * dt
    if expect_slide:
        a_exp = 9.81 * (math.sin(theta) - mu * math.cos(theta))
        # fit s = s0 + v0 t + a t^2 / 2 over the second half (after contact settles)
        t = np.arange(n_steps) * dt
        h = n_steps // 2
        A = np.stack([np.ones(n_steps - h), t[h:], 0.5 * t[h:] ** 2], axis=1)
        a_fit = np.linalg.lstsq(A, s[h:], rcond=None)[0][2]
        assert abs(a_fit - a_exp) < 0.1 * a_exp
    else:
        creep = sc["params"]["eps_v"] * T
        assert abs(s[-1]) < 3 * creep


def test_press_scene_invariants():
    """Every iterate keeps positive distance; accepted line-search steps never raise the energy."""
    sc = scenes.fingertip_press(0, n_steps=3)
    o = ipc.Oracle(sc)
    for _ in range(3):
        st = o.step()
        for r in st:
            assert r["min_s"] > 0
            if "E_new" in r:
                assert r["E_new"] <= r["E"] + 1e-13 * abs(r["E"])


def test_converged_step_is_stationary():
    """First-order optimality at the converged positions: free-DOF gradient ~ 0."""
    sc = scenes.fingertip_press(0, n_steps=2)
    o = ipc.Oracle(sc, tol=1e-11)
    z_t, zd_t = o.z.copy(), o.zd.copy()
    o.step()
    S = o.S
    x_t = S.positions(z_t)
    ctx = dict(z_tilde=z_t + S.dt * zd_t + S.dt ** 2 * S.grav_acc, x_t=x_t,
               lag=S.friction_lag(x_t.reshape(-1)), stitch_hat=S.stitch_targets(1))
    _, g, _, _ = S.evaluate(o.z, ctx, want_hess=False)
    _, g0, _, _ = S.evaluate(z_t, ctx, want_hess=False)
    gF = g[:S.n_free]
    scale = np.max(np.abs(g0[:S.n_free]))  # residual force at the start of the step
    assert np.max(np.abs(gF)) < 1e-7 * scale
