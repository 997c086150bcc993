"""The learned proposal end to end at a small size: plain-EM labels, training
with the library's kernels, and the learned bootstrap's depth against the
triangulation bootstrap's on held-out windows."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SIZE = dict(W=256, H=192, f=210.0, T=4)


@pytest.fixture(scope="module")
def trained():
    from paper_2104_06789_gb300 import build, learned, voldor
    build.build()
    ds = learned.build_dataset([learned.TRAIN_SEED0 + i for i in range(48)], S=1024, label_iters=5, **SIZE)
    net = voldor.Net(SIZE["T"], learned.init_weights(SIZE["T"], seed=0))
    losses = learned.train(net, ds, 800, batch=4, lr=2e-3)
    held = learned.build_dataset([learned.HELDOUT_SEED0 + i for i in range(4)], label_iters=0, **SIZE)
    res = learned.compare(net, held, S=1024, max_iters=5, plain_iters=5,
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
