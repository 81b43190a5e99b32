"""What the trained surrogate gains over the method without it.

A small surrogate (C = 16, K = 8, L = 2) is trained by the library's own
forward/backward kernels and Adam on 64-step windows of LBM trajectories of
a 64 x 128 closed box with gas plumes (the surrogate2d recipe at reduced
size), then judged by the LBM on a held-out trajectory: its predicted states must
be closer to the LBM's than the persistence baseline (the state 64 steps
earlier), and its alpha_g increment error below 100 %.  The speed gain (one
call against the 64 LBM steps it replaces) is measured on the full
256 x 1024 workload by `python -m paper_2409_10399_gb300.surrogate`.
"""
import pytest

pytestmark = pytest.mark.gpu


def test_trained_surrogate_beats_persistence():
    import torch

    from paper_2409_10399_gb300 import Surrogate
    from paper_2409_10399_gb300 import surrogate as S

    nx, ny, C, K, L = 64, 128, 16, 8, 2
    data = S.trajectories(3, 500, nx, ny, 64 * 8, recipe="plume")  # 3 trajectories, 9 snapshots each
    train, test = data[:2], data[2:]
    m = Surrogate(nx, ny, C, K, L)
    m.set_stream(torch.cuda.current_stream())
    m.set_params(S.init_params(C, K, L, seed=1))
    m.set_norm(*S.fit_norm(train))
    hist = S.train(m, train, epochs=40, batch=4, lr=3e-3, seed=1)
    assert hist[-1] < 0.5 * hist[0], hist
    ev = S.evaluate(m, test, max_drift=1e-4, rollout=2)
    assert ev["state_rel_l2"] < ev["persistence_rel_l2"], ev
    assert ev["increment_rel_l2"]["alpha_g"] < 1.0, ev
    m.close()
