"""The cost model on the host (CPU only): parameters round-trip, and host inference is the
numpy reference network applied to standardised log1p(features), mapped back to ms."""
import numpy as np
import pytest

from oracle import mlp
from paper_1509_04394_gb300 import build as kbuild
from paper_1509_04394_gb300 import kfuse as K


@pytest.fixture(scope="module", autouse=True)
def _built():
    kbuild.build()


def test_predict_is_the_reference_network():
    ctx = K.kf_create(-1)
    rng = np.random.default_rng(4)
    p = rng.normal(scale=0.2, size=K.KF_MLP_NPARAMS).astype(np.float32)
    norm = np.concatenate([rng.normal(size=K.KF_NFEAT), rng.uniform(0.5, 2.0, K.KF_NFEAT), [0.3], [1.7]]).astype(np.float32)
    with pytest.raises(K.KfuseError):
        K.kf_costmodel_predict(ctx, np.zeros((1, K.KF_NFEAT)))
    K.kf_costmodel_set(ctx, p, norm)
    p2, n2 = K.kf_costmodel_get(ctx)
    np.testing.assert_array_equal(p2, p)
    np.testing.assert_array_equal(n2, norm)
    feats = rng.uniform(0, 50, size=(9, K.KF_NFEAT)).astype(np.float32)
    got = K.kf_costmodel_predict(ctx, feats)
    x = (np.log1p(feats.astype(np.float64)) - norm[:K.KF_NFEAT]) / norm[K.KF_NFEAT:2 * K.KF_NFEAT]
    exp = np.exp(mlp.forward(p.astype(np.float64), x) * norm[-1] + norm[-2])
    np.testing.assert_allclose(got, exp, rtol=2e-5)
    bad = norm.copy()
    bad[K.KF_NFEAT] = 0
    with pytest.raises(K.KfuseError):
        K.kf_costmodel_set(ctx, p, bad)
    K.kf_destroy(ctx)
