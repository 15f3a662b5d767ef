"""The geometry prior feeding the initializer and training (Sec. III: G -> I -> T) on a synthetic
keyframe ring: the fused MVS cloud seeds the paper's initializer and trains to a higher held-out
PSNR than the same budget seeded uniformly in the cloud's bounding box."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_mvs_prior_seeds_training_better_than_a_box():
    from paper_2601_17354_gb300 import evaluate as E
    out = E.prior_experiment(seed=3, iters=300)
    assert out["cloud_points"] > 200000
    assert out["mvs_prior"] > out["bounding_box"] + 1.0, out
