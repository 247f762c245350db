"""The cost model's training kernels on the GPU: the loss gradient equals the FP64
reference's, training is deterministic and fits a smooth synthetic cost."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import mlp  # noqa: E402
from paper_1509_04394_gb300 import build as kbuild  # noqa: E402
from paper_1509_04394_gb300 import kfuse as K  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kbuild.build()
    c = K.kf_create(0)
    yield c
    K.kf_destroy(c)


@pytest.mark.parametrize("n", [1, 63, 64, 200])
def test_gradient_matches_the_reference(ctx, n):
    rng = np.random.default_rng(n)
    p = rng.normal(scale=0.3, size=K.KF_MLP_NPARAMS)
    x, y = rng.normal(size=(n, K.KF_NFEAT)), rng.normal(size=n)
    L, g = K.kf_costmodel_grad(ctx, p, x, y)
    L_ref, g_ref = mlp.grad(p.astype(np.float32).astype(np.float64), x.astype(np.float32).astype(np.float64),
                            y.astype(np.float32).astype(np.float64))
    assert L == pytest.approx(L_ref, rel=1e-4)
    scale = np.max(np.abs(g_ref))
    assert np.max(np.abs(g - g_ref)) <= 1e-4 * scale


def test_training_is_deterministic_and_fits(ctx):
    rng = np.random.default_rng(7)
    n = 3000
    feats = rng.uniform(0, 30, size=(n, K.KF_NFEAT)).astype(np.float32)
    ms = (0.05 + 0.01 * feats[:, 0] * feats[:, 3] / 30 + 0.2 * np.sqrt(feats[:, 8])).astype(np.float32)
    l1 = K.kf_costmodel_train(ctx, feats, ms, steps=1500, lr=3e-3, seed=3)
    p1, _ = K.kf_costmodel_get(ctx)
    l2 = K.kf_costmodel_train(ctx, feats, ms, steps=1500, lr=3e-3, seed=3)
    p2, _ = K.kf_costmodel_get(ctx)
    assert l1 == l2 and np.array_equal(p1, p2)
    assert l1 < 0.02  # standardised log-runtime MSE (a constant predictor scores 1.0)
    pred = K.kf_costmodel_predict(ctx, feats[:200])
    assert np.median(np.abs(pred / ms[:200] - 1)) < 0.05


def test_the_learned_model_plans_better_than_the_traffic_model(ctx):
    """Trained on measured groups of 40 random DAGs, the MLP's partitions of 12 held-out
    DAGs cost less (measured) than those the analytic traffic model picks."""
    from paper_1509_04394_gb300 import costmodel as cm
    from synth import dags as sd
    from synth import video as sv
    W, H, T = 512, 256, 2
    fr, _ = sv.generate(sv.VideoSpec(T=T, H=H, W=W, seed=8), pitch=W)
    f = torch.from_numpy(fr).to("cuda:0")
    meas = [cm.measure(ctx, sd.to_array(sd.random_dag(900 + s)), f, W, 900 + s, reps=3) for s in range(52)]
    X, y = cm.dataset(meas[:40])
    K.kf_costmodel_train(ctx, X, y, steps=3000, lr=3e-3, seed=1)
    ev = cm.evaluate(ctx, meas[40:])
    assert ev["mlp_mean_regret"] < ev["traffic_mean_regret"]
    assert ev["mlp_better_or_equal"] >= 8
