"""The learned extension end to end at small scale (GPU): the surrogate is
trained on late-time diagnostics of batched PIC runs, predicts held-out PIC
runs, and guides the backflow-transition search with fewer PIC
particle-steps than plain batched bisection, reaching the same answers."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trained():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_07083_gb300 import build as B
    B.build()
    from paper_2605_07083_gb300 import surrogate as S
    _, Xtr, Ytr, _ = S.build_dataset(512, 11, n_flight=4.0e3, transits=4.0)
    _, Xte, Yte, _ = S.build_dataset(96, 12, n_flight=4.0e3, transits=4.0)
    model = S.Surrogate(3)
    hist = model.fit(Xtr, Ytr, steps=1500)
    return S, model, hist, Xte, Yte


def test_training_loss_falls_and_held_out_error_is_small(trained):
    S, model, hist, Xte, Yte = trained
    assert hist[-1][1] < 0.2 * hist[0][1]
    P = model.predict(Xte)
    err = np.abs(P - Yte)
    # PIC at 4e3 macro-electrons in flight is itself noisy at the percent level
    assert err[:, 0].mean() < 0.06
    assert np.median(err[:, 0]) < 0.04
    # net efficiency is one minus the backflow ratio in the data
    np.testing.assert_allclose(Yte[:, 1], 1.0 - Yte[:, 0], atol=1e-6)


def test_guided_search_needs_fewer_pic_particle_steps_and_rounds(trained):
    S, model, _, _, _ = trained
    from paper_2605_07083_gb300 import workloads as W
    settings = W.random_settings(24, 13)
    kw = dict(n_flight=4.0e3, transits=4.0)
    est_p, cost_p = S.plain_search(settings, **kw)
    # this small network (512 noisy samples) is judged with a wider band than
    # the 0.02 the full-size pipeline uses
    est_g, cost_g = S.guided_search(model, settings, max_err=0.1, **kw)
    # the guided search spends fewer PIC particle-steps and fewer launch rounds
    # (its fall-back k-section buys rounds with extra runs, so the margin in
    # particle-steps is smaller than in rounds)
    assert cost_g["particle_steps"] < cost_p["particle_steps"]
    assert cost_g["rounds"] < cost_p["rounds"]
    same = np.isnan(est_p) == np.isnan(est_g)
    assert same.mean() >= 0.75
    both = ~np.isnan(est_p) & ~np.isnan(est_g)
    if both.any():
        diff = np.abs(est_p[both] - est_g[both])
        assert np.mean(diff <= 4 * S.TOL) >= 0.7
