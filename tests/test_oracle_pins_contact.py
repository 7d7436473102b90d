"""Pins for the parts of the CPU oracle that decide which primitive pairs exist at all (the exclusion
rules of the active set, the swept-box filter in front of the additive CCD) and for the stitch springs of
Eq. 2.  Each expected value is counted or derived by hand from the configuration, not computed by the
oracle: pair sets of hand-built triangles whose distances are known, a triangle that sweeps through a
point in a known time, and the closed-form stretch of a block hanging from N stitch springs."""
import math

import numpy as np
import pytest

from oracle import ipc
from paper_2609_25653_b300 import scenes

FEM, ABD, KIN = 0, 1, 2


class Surf:
    """An OrcSurf over hand-given arrays (kept alive by this object)."""

    def __init__(self, x, tris, vbody, bkind, sv=None):
        self.x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
        self.tris = np.ascontiguousarray(tris, dtype=np.int32)
        self.edges = ipc.tri_edges(self.tris)
        self.sv = np.ascontiguousarray(np.unique(self.tris) if sv is None else sv, dtype=np.int32)
        self.vbody = np.ascontiguousarray(vbody, dtype=np.int32)
        self.bkind = np.ascontiguousarray(bkind, dtype=np.int32)
        self.s = ipc.OrcSurf(len(self.sv), len(self.tris), len(self.edges), ipc._i(self.sv), ipc._i(self.tris),
                             ipc._i(self.edges), ipc._i(self.vbody), ipc._i(self.bkind))

    def pairs(self, sh):
        import ctypes as C
        cap = 256
        rec = np.zeros((cap, 8), np.int32)
        s = np.zeros(cap)
        n = ipc.lib().orc_active_pairs(C.byref(self.s), ipc._d(self.x), sh, cap, ipc._i(rec), ipc._d(s))
        assert n <= cap
        return rec[:n], s[:n]

    def ccd(self, p, s_frac=0.1):
        import ctypes as C
        nc = C.c_int()
        p = np.ascontiguousarray(p, dtype=np.float64).reshape(-1)
        a = ipc.lib().orc_ccd_alpha(C.byref(self.s), ipc._d(self.x), ipc._d(p), s_frac, ipc.ACCD_MAX_ITER,
                                    C.byref(nc))
        return a, nc.value


DHAT = 1e-3
H = 0.4e-3  # gap between the two parallel triangles (below dhat)


def two_parallel_triangles():
    """T1 = (0, 1, 2) in z = 0 and T2 = (3, 4, 5) the same triangle lifted by H.  Every vertex of one lies
    right above / below a vertex of the other and every edge of T2 shares a projected endpoint with every
    edge of T1, so all 3 + 3 point-triangle and 3 x 3 edge-edge pairs between them are at distance H."""
    a = 2e-3
    base = np.array([[0.0, 0.0, 0.0], [a, 0.0, 0.0], [0.0, a, 0.0]])
    x = np.concatenate([base, base + np.array([0.0, 0.0, H])])
    return x, np.array([[0, 1, 2], [3, 4, 5]])


@pytest.mark.parametrize("kinds,bodies,expect", [
    # (body kind of T1, of T2), (body id of T1, of T2), expected number of pairs
    ((FEM, FEM), (0, 0), 15),   # FEM self-contact is included
    ((FEM, FEM), (0, 1), 15),
    ((FEM, KIN), (0, 1), 15),
    ((FEM, ABD), (0, 1), 15),
    ((ABD, KIN), (0, 1), 15),
    ((ABD, ABD), (0, 1), 15),   # two affine bodies
    ((ABD, ABD), (0, 0), 0),    # one rigid body never touches itself
    ((KIN, KIN), (0, 0), 0),
    ((KIN, KIN), (0, 1), 0),    # both kinematic: nothing free to move
])
def test_exclusion_rules_decide_the_pair_set(kinds, bodies, expect):
    x, tris = two_parallel_triangles()
    nb = max(bodies) + 1
    bkind = [0] * nb
    for k, b in zip(kinds, bodies):
        bkind[b] = k
    vbody = [bodies[0]] * 3 + [bodies[1]] * 3
    S = Surf(x, tris, vbody, bkind)
    rec, s = S.pairs(DHAT * DHAT)
    assert len(rec) == expect
    if expect:
        assert int((rec[:, 0] == 0).sum()) == 6 and int((rec[:, 0] == 1).sum()) == 9
        # every pair joins one primitive of each triangle, at distance H
        for r in rec:
            ids = r[4:8]
            assert len(set(ids) & {0, 1, 2}) >= 1 and len(set(ids) & {3, 4, 5}) >= 1
        assert np.allclose(s, H * H, rtol=1e-12)


def test_shared_vertex_exclusion_on_a_flat_quad():
    """Quad (0, 1, 2, 3) split along 0-2 on one FEM body, side 0.1 dhat: every primitive is within dhat of
    every other, so only the shared-vertex rule removes pairs.  Left: vertex 3 with triangle (0, 1, 2),
    vertex 1 with (0, 2, 3), and the two pairs of opposite quad sides (0-1 | 2-3, 0-3 | 1-2)."""
    a = 0.1 * DHAT
    x = np.array([[0.0, 0.0, 0.0], [a, 0.0, 0.0], [a, a, 0.0], [0.0, a, 0.0]])
    S = Surf(x, np.array([[0, 1, 2], [0, 2, 3]]), [0, 0, 0, 0], [FEM])
    rec, s = S.pairs(DHAT * DHAT)
    got = sorted((int(r[0]), tuple(int(v) for v in r[4:8])) for r in rec)
    assert got == [(0, (1, 0, 2, 3)), (0, (3, 0, 1, 2)), (1, (0, 1, 2, 3)), (1, (0, 3, 1, 2))]
    # a lone triangle: every pair shares a vertex although all distances are zero
    S1 = Surf(x[:3], np.array([[0, 1, 2]]), [0, 0, 0], [FEM])
    assert len(S1.pairs(DHAT * DHAT)[0]) == 0


def point_and_triangle(point, tri_pts):
    """Vertex 0 (a FEM point, surface vertex) and a kinematic triangle (1, 2, 3)."""
    x = np.concatenate([np.asarray(point, float).reshape(1, 3), np.asarray(tri_pts, float)])
    return Surf(x, np.array([[1, 2, 3]]), [0, 1, 1, 1], [FEM, KIN], sv=np.array([0, 1, 2, 3]))


TRI = np.array([[-1e-3, -1e-3, 0.0], [2e-3, -1e-3, 0.0], [-1e-3, 2e-3, 0.0]])


def test_ccd_filter_finds_a_triangle_sweeping_through_a_point():
    """The triangle starts 1 mm above a static point and moves 2 mm down: the point is swept at t = 1/2.
    Only the swept box (start and end vertex positions) overlaps the point; the start box does not."""
    S = point_and_triangle([0.0, 0.0, 0.0], TRI + np.array([0.0, 0.0, 1e-3]))
    p = np.zeros((4, 3))
    p[1:, 2] = -2e-3
    alpha, nc = S.ccd(p)
    assert nc == 1
    t_contact = 0.5
    # additive CCD stops before the distance falls below s_frac of its start value: t <= 0.9 t_contact,
    # and it advances to within one conservative step of that time
    assert 0.85 * t_contact < alpha <= 0.9 * t_contact
    assert alpha == ipc.accd(0, S.x.reshape(-1, 3)[[0, 1, 2, 3]], p[[0, 1, 2, 3]], 0.1, 1.0, ipc.ACCD_MAX_ITER)


def test_ccd_filter_uses_the_moving_point_end_position():
    """The point moves through the static triangle (start 1 mm above, end 1 mm below): found through the
    point's swept box only."""
    S = point_and_triangle([0.0, 0.0, 1e-3], TRI)
    p = np.zeros((4, 3))
    p[0, 2] = -2e-3
    alpha, nc = S.ccd(p)
    assert nc == 1 and 0.85 * 0.5 < alpha <= 0.9 * 0.5


def test_ccd_filter_rejects_separated_sweeps():
    """The triangle slides sideways 1 mm above the point: swept boxes never overlap, no candidate, alpha 1.
    A diagonal sweep that starts far to the side and ends below the point is a candidate again."""
    S = point_and_triangle([0.0, 0.0, 0.0], TRI + np.array([0.0, 0.0, 1e-3]))
    p = np.zeros((4, 3))
    p[1:, 0] = 5e-3
    assert S.ccd(p) == (1.0, 0)
    S2 = point_and_triangle([0.0, 0.0, 0.0], TRI + np.array([6e-3, 0.0, 1e-3]))
    p2 = np.zeros((4, 3))
    p2[1:] = [-6e-3, 0.0, -2e-3]
    a2, n2 = S2.ccd(p2)
    # straight-line motion: the triangle's plane reaches z = 0 at t = 1/2, when the triangle (shifted by
    # -3 mm in x) still lies to the side of the point ([2, 5] mm in x at y = 0): no contact, the full step
    # is safe, but the boxes overlap, so the pair is tested
    assert n2 == 1 and a2 == 1.0


def test_stitch_springs_hold_a_hanging_block_at_the_closed_form_stretch():
    """A stiff block hanging from N stitch springs (Eq. 2) at fixed anchors, one implicit step with a very
    long time step (the inertia term vanishes, leaving the static balance): the block translates rigidly by
    u = m g / (N k_c) downwards."""
    k_c = 0.2
    sc = scenes.stitched_block(n_steps=2, dt=10.0, k_c=k_c, newton_tol=1e-12, pcg_rtol=1e-14, mu=0.0)
    sc["fem_logE"] = np.full(len(sc["fem_tets"]), math.log(1e9))
    sc["kin_T"] = np.tile(scenes.translation((0.0, 0.0, 0.0)), (3, 1, 1, 1))
    o = ipc.Oracle(sc)
    S = o.S
    N = len(S.stitch_v)
    m = float(S.mass_v.sum())
    x0 = o.x()[:S.nf].copy()
    o.step()
    u = o.x()[:S.nf] - x0
    u_expect = m * 9.81 / (N * k_c)
    assert N == 9
    assert abs(-u[:, 2].mean() - u_expect) <= 1e-4 * u_expect
    assert np.max(np.abs(u[:, 2] - u[:, 2].mean())) <= 1e-4 * u_expect
    assert np.max(np.abs(u[:, :2])) <= 1e-6 * u_expect


def test_incremental_potential_fd_with_stitch_springs():
    """Gradient and Hessian of the whole incremental potential (inertia, elasticity, stitch) against
    central differences of its energy, on the swinging stitched block away from contact."""
    sc = scenes.stitched_block(n_steps=2, mu=0.0)
    S = ipc.Scene(sc)
    r = np.random.default_rng(3)
    z_t = S.z0.copy()
    ctx = ipc.step_context(S, z_t, S.zd0, 1)
    z = z_t.copy()
    z[:S.n_fem_dof] += 1e-4 * r.normal(size=S.n_fem_dof)
    E, g, Hm, info = S.evaluate(z, ctx, project=False)
    assert info["E_stitch"] > 0 and info["n_pairs"] == 0
    F = S.n_free
    h = 1e-7
    idx = r.choice(F, 12, replace=False)
    Hd = Hm.toarray()
    for i in idx:
        e = np.zeros_like(z)
        e[i] = h
        gi = (S.energy(z + e, ctx) - S.energy(z - e, ctx)) / (2 * h)
        assert abs(gi - g[i]) <= 1e-6 * np.max(np.abs(g[:F]))
        _, gp, _, _ = S.evaluate(z + e, ctx, want_hess=False)
        _, gm, _, _ = S.evaluate(z - e, ctx, want_hess=False)
        col = (gp - gm)[:F] / (2 * h)
        assert np.max(np.abs(col - Hd[:F, i])) <= 1e-6 * np.max(np.abs(Hd[:F, :F]))


def test_pair_loops_do_not_depend_on_the_thread_count():
    """The brute-force pair loops run on OpenMP threads in chunks: pairs, their order, the squared
    distances, the CCD bound and the candidate count equal those of one thread."""
    import ctypes as C
    sc = scenes.fingertip_press(2)
    S = ipc.Scene(sc)
    r = np.random.default_rng(7)
    x = S.positions(S.z0).copy()
    x[:S.nf, 2] = 0.5e-3 + (x[:S.nf, 2] - 0.5e-3) * 0.96 - 0.35e-3
    x[:S.nf] += 5e-5 * r.normal(size=(S.nf, 3))
    x[S.nf + S.na_v + 8:] += np.array([0, 0, -0.45e-3])
    p = np.zeros_like(x)
    p[:S.nf] = 1e-3 * r.normal(size=(S.nf, 3)) + np.array([0, 0, -1.5e-3])
    xf, pf = np.ascontiguousarray(x.reshape(-1)), np.ascontiguousarray(p.reshape(-1))
    out = []
    for nth in (1, 5):
        ipc.set_threads(nth)
        try:
            rec, s = S.active_pairs(xf)
            nc = C.c_int()
            a = ipc.lib().orc_ccd_alpha(C.byref(S.surf), ipc._d(xf), ipc._d(pf), S.s_ccd, ipc.ACCD_MAX_ITER,
                                        C.byref(nc))
        finally:
            ipc.set_threads(0)
        out.append((rec, s, a, nc.value))
    assert len(out[0][0]) > 20
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2] and out[0][3] == out[1][3]
