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


def forward_error_bound(p, x):
    """Per-sample bound of |FP32 forward - FP64 forward|: each layer's dot products of
    m terms (with the bias) round within gamma_m of the sum of their magnitudes
    (Higham, Sec. 3.1), and the next layer carries the errors of its inputs through the
    magnitudes of its weights (ReLU is 1-Lipschitz)."""
    u = 2.0 ** -24
    g = lambda m: m * u / (1 - m * u)  # noqa: E731
    W1, b1, W2, b2, w3, b3 = mlp.unpack(p, x.shape[1])
    h1 = np.maximum(x @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    e1 = g(x.shape[1] + 1) * (np.abs(x) @ np.abs(W1).T + np.abs(b1))
    e2 = e1 @ np.abs(W2).T + g(65) * ((h1 + e1) @ np.abs(W2).T + np.abs(b2))
    return e2 @ np.abs(w3) + g(65) * ((h2 + e2) @ np.abs(w3) + abs(b3))


@pytest.mark.parametrize("n", [1, 127, 128, 1000])
def test_inference_kernel_matches_the_reference_forward(ctx, n):
    """The inference kernel's raw outputs against the FP64 network of the oracle, within
    the FP32 rounding bound of its dot products, and 1e-5 normwise."""
    rng = np.random.default_rng(100 + n)
    p = rng.normal(scale=0.3, size=K.KF_MLP_NPARAMS).astype(np.float32)
    x = rng.normal(size=(n, K.KF_NFEAT)).astype(np.float32)
    y = K.kf_costmodel_forward(ctx, p, x).astype(np.float64)
    p64, x64 = p.astype(np.float64), x.astype(np.float64)
    ref = mlp.forward(p64, x64)
    bound = forward_error_bound(p64, x64)
    assert np.all(np.abs(y - ref) <= bound)
    assert np.max(np.abs(y - ref)) <= 1e-5 * np.max(np.abs(ref))


def test_predictions_are_the_standardised_network(ctx):
    """kf_costmodel_predict on the GPU: log1p features standardised by the stored means
    and deviations, the network, then exp(y * ystd + ymean) -- against the same steps in
    FP64 on the oracle's network (relative error within 1e-4: the output's FP32 error
    times ystd, plus the rounding of the standardisation and of exp)."""
    rng = np.random.default_rng(5)
    F = K.KF_NFEAT
    p = rng.normal(scale=0.2, size=K.KF_MLP_NPARAMS).astype(np.float32)
    fmean, fstd = rng.uniform(0, 2, F).astype(np.float32), rng.uniform(0.5, 2, F).astype(np.float32)
    norm = np.concatenate([fmean, fstd, np.array([-1.5, 0.8], dtype=np.float32)])
    K.kf_costmodel_set(ctx, p, norm)
    feats = rng.uniform(0, 50, size=(500, F)).astype(np.float32)
    ms = K.kf_costmodel_predict(ctx, feats).astype(np.float64)
    xs = (np.log1p(feats.astype(np.float64)) - fmean) / fstd
    ref = np.exp(mlp.forward(p.astype(np.float64), xs) * float(norm[-1]) + float(norm[-2]))
    assert np.max(np.abs(ms / ref - 1.0)) <= 1e-4
