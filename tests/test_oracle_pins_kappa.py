"""Pins of the oracle's barrier stiffness against the static force balance of a resting body.

A 10 mm affine cube rests on a large ground triangle with its four bottom corners in point-triangle
contact (no other pair is within dhat).  At rest the barrier forces carry the weight:
4 kappa (-db/dd)(d) = m g with b(d) = -(d^2 - dhat^2)^2 ln(d^2 / dhat^2), so the resting height d of the
corners is the root of that equation for the kappa in use.  With the adaptive stiffness on, kappa doubles
while the closest distance stays below kappa_dmin * dhat, so it ends at the first power-of-two multiple of
the initial kappa whose resting height clears that distance."""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

from oracle import ipc
from paper_2609_25653_b300 import scenes

MM = 1e-3
H = 5 * MM          # half edge of the cube
RHO = 1000.0
DHAT = 1e-3
KAPPA0 = 2452.0     # rests near 2e-6 m, below 1e-2 dhat
G = 9.81


def corner_force(d, kappa):
    """Barrier force on one corner at height d: -kappa d/dd of b(d^2)."""
    s, sh = d * d, DHAT * DHAT
    db_ds = -2.0 * (s - sh) * math.log(s / sh) - (s - sh) ** 2 / s
    return -kappa * db_ds * 2.0 * d


def rest_height(kappa):
    m = RHO * (2 * H) ** 3
    return brentq(lambda d: 4.0 * corner_force(d, kappa) - m * G, 1e-12, DHAT * (1 - 1e-12), xtol=1e-18, rtol=1e-15)


def _scene(adaptive, n_steps=30, d_start=2e-5):
    X, T = scenes.subdivided_box((-H, -H, -H), (H, H, H), 1)
    q0 = np.concatenate([[0.0, 0.0, H + d_start], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])
    gX = np.array([[-1.0, -1.0, 0.0], [2.0, -1.0, 0.0], [-1.0, 2.0, 0.0]])
    p = scenes.default_params(dt=1e-2, dhat=DHAT, mu=0.0, kappa=KAPPA0, n_steps=n_steps, newton_tol=1e-10,
                              pcg_rtol=1e-12, max_newton=300)
    p.update(kappa_adaptive=int(adaptive), kappa_dmin=1e-2, kappa_max_factor=100.0)
    return dict(name="resting_cube", fem_X=np.zeros((0, 3)), fem_tets=np.zeros((0, 4), np.int32),
                fem_logE=np.zeros(0), fem_nu=np.zeros(0), fem_rho=np.zeros(0), fem_body=np.zeros(0, np.int32),
                kin=[dict(X=gX, tris=np.array([[0, 1, 2]], np.int32))],
                kin_T=np.tile(scenes.translation((0.0, 0.0, 0.0)), (n_steps + 1, 1, 1, 1)),
                abd=[dict(X=X, tris=T, rho=RHO, q0=q0)],
                stitch_v=np.zeros(0, np.int32), stitch_b=np.zeros(0, np.int32), stitch_X=np.zeros((0, 3)),
                gravity=np.array([0.0, 0.0, -G]), params=p)


def _run(adaptive):
    sc = _scene(adaptive)
    o = ipc.Oracle(sc)
    for _ in range(sc["params"]["n_steps"]):
        o.step()
    x = o.S.positions(o.z).reshape(-1, 3)
    nf = o.S.nf
    corners = x[nf:nf + 8]
    d = corners[:, 2].min()
    return o, d, corners


def test_resting_cube_fixed_kappa_balances_weight():
    o, d, corners = _run(False)
    assert o.S.kappa == KAPPA0
    bottom = np.sort(corners[:, 2])[:4]
    assert np.ptp(bottom) < 1e-12           # the four corners share the load
    d_star = rest_height(KAPPA0)
    assert d_star < 1e-2 * DHAT
    assert abs(d - d_star) <= 1e-6 * d_star
    assert np.abs(o.zd).max() < 1e-8


def test_adaptive_kappa_doubles_until_the_rest_height_clears_the_threshold():
    o, d, _ = _run(True)
    ratio = o.S.kappa / KAPPA0
    k = round(math.log2(ratio))
    assert k >= 1 and ratio == 2.0 ** k     # doublings only
    assert abs(d - rest_height(o.S.kappa)) <= 1e-6 * d
    assert d >= 1e-2 * DHAT                  # the growth stopped because the distance cleared the threshold
    assert rest_height(o.S.kappa / 2) < 1e-2 * DHAT   # ... and not earlier


def test_adaptive_kappa_is_capped():
    sc = _scene(True)
    sc["params"]["kappa_max_factor"] = 3.0
    o = ipc.Oracle(sc)
    for _ in range(20):
        o.step()
    assert o.S.kappa == 3.0 * KAPPA0
