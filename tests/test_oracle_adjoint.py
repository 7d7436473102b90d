"""The oracle's implicit adjoint against central finite differences of the oracle's own step."""
import numpy as np
import pytest

from oracle import ipc
from paper_2609_25653_b300 import scenes

TOL = 1e-11


def _run(mu, logE=None, z0=None, zd0=None):
    sc = scenes.fingertip_press(0, n_steps=2, mu=mu, max_newton=300)
    o = ipc.Oracle(sc, tol=TOL)
    if logE is not None:
        ipc.set_material(o, logE=logE)
    if z0 is not None:
        o.z, o.zd = z0.copy(), zd0.copy()
    o.step()
    return o


@pytest.mark.slow
@pytest.mark.parametrize("mu", [0.0, 0.5])
def test_adjoint_matches_central_differences(mu):
    r = np.random.default_rng(11)
    o = _run(mu)
    S = o.S
    nF = S.n_free
    z_t, zd_t = S.z0.copy(), S.zd0.copy()
    target = o.z + 1e-4 * r.normal(size=o.z.shape)
    wv = r.normal(size=o.z.shape)

    def loss(oo):
        return 0.5 * float(np.sum((oo.z[:nF] - target[:nF]) ** 2)) + 1e-4 * float(wv[:nF] @ oo.zd[:nF])

    gz = np.zeros(S.ndof); gz[:nF] = (o.z - target)[:nF]
    gzd = np.zeros(S.ndof); gzd[:nF] = 1e-4 * wv[:nF]
    gz_t, gzd_t, dlogE, dmu = ipc.adjoint_step(o, z_t, zd_t, o.z, 1, gz, gzd)
    logE0 = S.logE.copy()
    for _ in range(2):
        d = r.normal(size=logE0.shape)
        h = 1e-5
        fd = (loss(_run(mu, logE0 + h * d)) - loss(_run(mu, logE0 - h * d))) / (2 * h)
        assert abs(fd - dlogE @ d) <= 1e-4 * abs(fd)
    if mu > 0:
        h = 1e-6
        fd = (loss(_run(mu + h)) - loss(_run(mu - h))) / (2 * h)
        assert abs(fd - dmu) <= 1e-4 * abs(fd)
    # initial position and velocity (with friction, through the lagged normal forces, normals and
    # closest points at x_t as well)
    for _ in range(2):
        d = r.normal(size=z_t.shape); d[nF:] = 0
        h = 1e-9
        fd = (loss(_run(mu, None, z_t + h * d, zd_t)) - loss(_run(mu, None, z_t - h * d, zd_t))) / (2 * h)
        assert abs(fd - gz_t @ d) <= 1e-4 * abs(fd), (fd, gz_t @ d)
        h = 1e-7
        fd = (loss(_run(mu, None, z_t, zd_t + h * d)) - loss(_run(mu, None, z_t, zd_t - h * d))) / (2 * h)
        assert abs(fd - gzd_t @ d) <= 1e-4 * abs(fd), (fd, gzd_t @ d)
