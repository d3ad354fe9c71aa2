"""The learned warm start (GPU required): trained on steady states the
lattice-Boltzmann / FENE-P step produces, the network's prediction of
held-out steady fields is much closer than the cold-start fields it starts
from, and a warm lattice built from it is a valid starting state (masses of
the set-up, SPD conformation, stable steps)."""
import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_network_prediction_beats_cold_start():
    import torch
    from paper_1406_2686_gb300 import nn, vefd, warmstart as ws
    N = 32
    train = ws.sample_setups(32, seed=11, N=N)
    held = ws.sample_setups(3, seed=29, N=N)
    X, Y, rec = ws.make_dataset(train, tol=1e-5, max_steps=30000)
    assert all(r["converged"] for r in rec)
    net = nn.UNet(ws.N_IN, ws.N_OUT, c=8, seed=0)
    losses = ws.train(net, X, Y, epochs=60, lr=1e-3)
    assert losses[-1] < losses[0] / 3
    Xh, Yh, _ = ws.make_dataset(held, tol=1e-5, max_steps=30000)
    err_net, err_cold = [], []
    for i in range(len(held)):
        out = net.forward(torch.from_numpy(Xh[i:i + 1]).cuda().contiguous())[0].cpu().numpy()
        err_net.append(float(np.mean((out[..., :ws.N_FIELDS] - Yh[i, ..., :ws.N_FIELDS]) ** 2)))
        # the cold start is the zero increment from the initial fields
        err_cold.append(float(np.mean(Yh[i, ..., :ws.N_FIELDS] ** 2)))
    assert np.mean(err_net) < 0.5 * np.mean(err_cold), (err_net, err_cold)
    # a warm lattice: masses of the set-up, SPD C, and it steps stably
    s = held[0]
    cold = s.cold(seed=7)
    phi0 = cold.read(vefd.PHI, device=True).clone()
    m_cold = cold.diagnostics()[:2]
    warm = ws.warm_lattice(net, s, phi0)
    m_warm = warm.diagnostics()[:2]
    assert np.allclose(m_warm, m_cold, rtol=1e-5)
    C = warm.read(vefd.C).reshape(6, -1).T.astype(np.float64)
    M = np.stack([C[:, [0, 1, 2]], C[:, [1, 3, 4]], C[:, [2, 4, 5]]], axis=1)
    assert np.linalg.eigvalsh(M).min() > 0
    warm.step(500)
    assert warm.status() == 0 and net.status() == 0
