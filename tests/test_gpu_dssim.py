"""L1 + D-SSIM loss kernels (through the C ABI) against the SSIM oracle: loss, mean SSIM and the
image gradient, on ragged and tiny images and on a render against its target."""
import numpy as np
import pytest

from oracle import ssim as O
from paper_2601_17354_gb300 import synthetic as S
from tests._parity import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_2601_17354_gb300 import rasterizer
    return rasterizer


@pytest.mark.parametrize("lam", [0.2, 1.0])
@pytest.mark.parametrize("shape", [(45, 70), (96, 128), (5, 7)])
def test_dssim_matches_oracle(R, shape, lam):
    H, W = shape
    x = S.random_image(31, W, H, 0.0, 1.0)
    y = np.clip(x + np.random.default_rng(32).normal(0, 0.1, x.shape), 0, 1).astype(np.float32)
    rast = R.Rasterizer()
    dl, out = rast.loss_dssim(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), lam)
    torch.cuda.synchronize()
    loss, ssim, g = O.loss_and_grad(x, y, lam)
    o = out.cpu().numpy()
    assert abs(o[0] - loss) <= 1e-5 * abs(loss) + 1e-7
    assert abs(o[1] - ssim) <= 1e-5
    assert rel_l2(dl.cpu().numpy(), g) < 1e-4


def test_dssim_of_a_render_and_a_training_step(R):
    sc = S.surface_scene(5, 20000, 1, 160, 120, 140.0, n_cameras=6)
    gt = R.GaussianBuffer.from_arrays(sc.gt)
    rast = R.Rasterizer()
    target = rast.render(gt, sc.cameras[2]).clone()
    params = R.GaussianBuffer.from_arrays(sc.init)
    img = rast.render(params, sc.cameras[2])
    dl, out = rast.loss_dssim(img, target, 0.2)
    torch.cuda.synchronize()
    loss, ssim, g = O.loss_and_grad(img.cpu().numpy(), target.cpu().numpy(), 0.2)
    assert abs(out[0].item() - loss) <= 1e-5 * loss and abs(out[1].item() - ssim) <= 1e-5
    assert rel_l2(dl.cpu().numpy(), g) < 1e-4
    tr = R.Trainer(params, R.Rasterizer(), dssim=0.2)
    first = float(tr.step(sc.cameras[2], target)[0])
    for _ in range(30):
        last = float(tr.step(sc.cameras[2], target)[0])
    assert np.isfinite(last) and last < first
