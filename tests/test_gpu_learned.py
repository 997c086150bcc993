"""The learned proposal: end to end at a small size (256x192, f = 210, T = 4:
plain-EM labels, training with the library's kernels, the learned
initialisation against the plain one on held-out windows), and the committed
weights at the benchmark's size (1242x375, T = 8) on the held-out windows the
benchmark line evaluates."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SIZE = dict(W=256, H=192, f=210.0, T=4)
# The small training run is a smoke test of the whole chain; its held-out
# medians after 3+ iterations sit within a few percent of each other, where the
# exact crossing point depends on the trained network's last bits.
N_TRAIN, TRAIN_STEPS, N_HELD = 256, 4000, 48


@pytest.fixture(scope="module")
def trained():
    from paper_2104_06789_gb300 import build, learned, voldor
    build.build()
    workers = max(1, min(8, (os.cpu_count() or 2) - 1))
    ds = learned.build_dataset([learned.TRAIN_SEED0 + i for i in range(N_TRAIN)], S=1024, label_iters=5,
                               workers=workers, **SIZE)
    net = voldor.Net(SIZE["T"], learned.init_weights(SIZE["T"], seed=0))
    losses = learned.train(net, ds, TRAIN_STEPS, batch=4, lr=2e-3)
    held = learned.build_dataset([learned.HELDOUT_SEED0 + i for i in range(N_HELD)], label_iters=0, workers=workers,
                                 **SIZE)
    res = learned.compare(net, held, S=1024, max_iters=6, plain_iters=5,
                          K=(SIZE["f"], SIZE["f"], (SIZE["W"] - 1) / 2.0, (SIZE["H"] - 1) / 2.0))
    yield losses, res
    net.destroy()


def test_labels_and_training(trained):
    losses, _ = trained
    assert np.all(np.isfinite(losses))
    assert losses[-50:].mean() < 0.8 * losses[:20].mean()


def test_learned_initialisation_runs_the_em(trained):
    _, res = trained
    e = res["init_depth_log_err"]
    assert np.isfinite(e["learned"]) and e["learned"] < 1.0, e
    for k in ("plain_err_m", "learned_err_m"):
        assert np.all(np.isfinite(res[k]))


def test_learned_rigidness_prior_improves_the_first_iterations(trained):
    """The gain of the learned proposal at this size, in the variant that has
    one: its rigidness output replaces the bootstrap's W = 1 (the depth is the
    triangulation's). Over the held-out windows the median translation error
    after 1 and 2 EM iterations is at least 5 % below the plain EM's, and the
    learned start costs less than one iteration. (Whether it reaches the plain
    EM's 5-iteration error an iteration earlier is decided near the error floor
    at this size: repeated trainings gave 3, 3, 4 and 6 iterations. That claim
    is tested on the committed weights at the benchmark's size below.)"""
    _, res = trained
    pl, lw = np.asarray(res["plain_median_err_m"]), np.asarray(res["learned_w_median_err_m"])
    print("median error per iteration: plain", np.round(pl, 5), "learned rigidness", np.round(lw, 5),
          "learned depth + rigidness", np.round(res["learned_median_err_m"], 5))
    assert lw[1] < 0.95 * pl[1] and lw[2] < 0.95 * pl[2], (pl, lw)
    boot = res["bootstrap_ms"]
    assert boot["learned_w"] < boot["plain"] + res["iteration_ms"], (boot, res["iteration_ms"])


def test_committed_weights_reach_the_plain_error_in_fewer_iterations():
    """The committed proposal weights (trained on 2000 windows at 1242x375,
    T = 8) on the 16 held-out windows the benchmark line evaluates (scene seeds
    from learned.HELDOUT_SEED0, S = 4096): started from the learned rigidness
    prior, the median translation error reaches the plain EM's median after 5
    iterations (within 1 %) in strictly fewer iterations, and in less time
    (bootstrap included). Training is bit-reproducible and the EM
    deterministic, so the outcome is fixed by the weights."""
    from paper_2104_06789_gb300 import build, learned, voldor
    build.build()
    weights = os.path.join(os.path.dirname(os.path.abspath(learned.__file__)), "weights",
                           "proposal_handheld_1242x375_T8.npy")
    net = voldor.Net(learned.SCENE["T"], np.load(weights))
    held = learned.build_dataset([learned.HELDOUT_SEED0 + i for i in range(16)], S=4096, label_iters=0,
                                 workers=max(1, min(8, (os.cpu_count() or 2) - 1)))
    res = learned.compare(net, held, S=4096, max_iters=6, plain_iters=5)
    net.destroy()
    k = res["learned_w_median_iters_to_target"]
    print("median error per iteration: plain", np.round(res["plain_median_err_m"], 5), "learned rigidness",
          np.round(res["learned_w_median_err_m"], 5))
    assert k is not None and k < 5, (k, res["learned_w_median_err_m"], res["median_target_err_m"])
    assert res["learned_w_median_ms"] < res["plain_ms"]
