"""Implicit adjoint on the GPU: parity with the oracle's dense adjoint and
central finite differences of the GPU forward on 16 random directions."""
import numpy as np
import pytest

from oracle import ipc as orc
from paper_2609_25653_b300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TIGHT = dict(newton_tol=1e-10, pcg_rtol=1e-13, max_newton=300)


def _sim(sc, **kw):
    from paper_2609_25653_b300 import ipcsim
    return ipcsim.Simulator(sc, **kw)


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


@pytest.mark.parametrize("mu", [0.0, 0.5])
def test_adjoint_matches_oracle_dense(mu):
    sc = scenes.fingertip_press(0, n_steps=3, mu=mu, **TIGHT)
    o = orc.Oracle(sc)
    o.S.max_newton = 300
    o.step()
    z_t, zd_t = o.S.z0.copy(), o.S.zd0.copy()
    r = np.random.default_rng(3)
    nF = o.S.n_free
    gz = np.zeros(o.S.ndof); gz[:nF] = r.normal(size=nF)
    gzd = np.zeros(o.S.ndof); gzd[:nF] = 1e-2 * r.normal(size=nF)
    gz_t, gzd_t, dlogE, dmu = orc.adjoint_step(o, z_t, zd_t, o.z, 1, gz, gzd)
    sim = _sim(sc)
    T = sc["kin_T"]
    g_z, g_zd, g_logE, g_mu = sim.adjoint(_dev(z_t[:nF]), _dev(zd_t[:nF]), _dev(o.z[:nF]), T[0], T[1],
                                          _dev(gz[:nF]), _dev(gzd[:nF]))
    def rel(a, b):
        return np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(g_z.cpu().numpy(), gz_t[:nF]) < 1e-6
    assert rel(g_zd.cpu().numpy(), gzd_t[:nF]) < 1e-6
    assert rel(g_logE.cpu().numpy(), dlogE) < 1e-6
    if mu > 0:
        assert abs(g_mu - dmu) <= 1e-6 * abs(dmu)


def test_adjoint_fd_16_directions():
    """dL/dlogE over a 2-step rollout (mu = 0: exact) against central differences of the GPU forward."""
    from paper_2609_25653_b300 import autograd
    sc = scenes.fingertip_press(0, n_steps=3, mu=0.0, **TIGHT)
    sim = _sim(sc)
    z0, zd0 = sim.get_dofs()
    logE0 = torch.tensor(sc["fem_logE"], dtype=torch.float64)
    r = np.random.default_rng(7)
    target = None

    def loss(logE, keep=False):
        traj = autograd.rollout(sim, logE, 0.0, 2, z0, zd0)
        nonlocal target
        if target is None:
            target = (traj[-1] + 1e-4 * torch.as_tensor(r.normal(size=traj[-1].shape), device="cuda")).detach()
        return 0.5 * torch.sum((traj[-1] - target) ** 2)

    logE = logE0.clone().requires_grad_(True)
    L = loss(logE)
    L.backward()
    g = logE.grad.numpy()
    worst = 0.0
    for k in range(16):
        d = r.normal(size=g.shape)
        h = 1e-4
        with torch.no_grad():
            Lp = loss(logE0 + h * torch.as_tensor(d)).item()
            Lm = loss(logE0 - h * torch.as_tensor(d)).item()
        fd = (Lp - Lm) / (2 * h)
        ad = float(g @ d)
        worst = max(worst, abs(fd - ad) / max(abs(fd), 1e-30))
    assert worst < 1e-4, worst


def test_adjoint_rollout_fd_with_friction():
    """A 3-step rollout with friction (mu = 0.5): gradients with respect to the initial positions (which
    move the lagged normal forces, normals and closest points of every step), the friction coefficient and
    ln E against central differences of the GPU forward."""
    from paper_2609_25653_b300 import autograd
    sc = scenes.fingertip_press(0, n_steps=4, mu=0.5, **TIGHT)
    sim = _sim(sc)
    z0, zd0 = sim.get_dofs()
    logE0 = torch.tensor(sc["fem_logE"], dtype=torch.float64)
    r = np.random.default_rng(5)
    target = {}

    def loss(logE, mu, z_init):
        traj = autograd.rollout(sim, logE, mu, 3, z_init, zd0)
        if "t" not in target:
            target["t"] = (traj[-1] + 1e-4 * torch.as_tensor(r.normal(size=traj[-1].shape), device="cuda")).detach()
        return 0.5 * torch.sum((traj[-1] - target["t"]) ** 2)

    logE = logE0.clone().requires_grad_(True)
    mu = torch.tensor(0.5, dtype=torch.float64, requires_grad=True)
    zi = z0.clone().requires_grad_(True)
    L = loss(logE, mu, zi)
    L.backward()
    g_logE, g_mu, g_z = logE.grad.numpy(), mu.grad.item(), zi.grad.cpu().numpy()
    worst = 0.0
    with torch.no_grad():
        for k in range(3):
            d = r.normal(size=g_z.shape)
            d[3 * sim.nf:] = 0.0
            h = 1e-9
            dz = torch.as_tensor(h * d, device="cuda")
            fd = (loss(logE0, 0.5, z0 + dz).item() - loss(logE0, 0.5, z0 - dz).item()) / (2 * h)
            worst = max(worst, abs(fd - g_z @ d) / max(abs(fd), 1e-30))
        h = 1e-6
        fd = (loss(logE0, 0.5 + h, z0).item() - loss(logE0, 0.5 - h, z0).item()) / (2 * h)
        worst = max(worst, abs(fd - g_mu) / abs(fd))
        for k in range(4):
            d = r.normal(size=g_logE.shape)
            h = 1e-4
            dl = torch.as_tensor(h * d)
            fd = (loss(logE0 + dl, 0.5, z0).item() - loss(logE0 - dl, 0.5, z0).item()) / (2 * h)
            worst = max(worst, abs(fd - g_logE @ d) / max(abs(fd), 1e-30))
    assert worst < 1e-4, worst
