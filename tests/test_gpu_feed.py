"""Training from pinned host images through ImageFeed (copies on their own stream, one step
ahead) gives the same parameters as training from device-resident targets."""
import numpy as np
import pytest

from paper_2601_17354_gb300 import synthetic as S
from tests._parity import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_image_feed_matches_device_targets():
    from paper_2601_17354_gb300 import rasterizer as R
    sc = S.surface_scene(3, 20000, 1, 160, 120, 140.0, n_cameras=6)
    targets = [torch.from_numpy(S.random_image(50 + k, 160, 120, 0.0, 1.0)).cuda() for k in range(6)]
    runs = []
    for use_feed in (False, True):
        p = R.GaussianBuffer.from_arrays(sc.init)
        rast = R.Rasterizer()
        tr = R.Trainer(p, rast)
        losses = []
        if use_feed:
            host = [t.cpu().pin_memory() for t in targets]
            feed = R.ImageFeed(targets[0].shape)
            feed.put(0, host[0])
        for k in range(6):
            if use_feed:
                if k + 1 < 6:
                    feed.put(k + 1, host[k + 1])
                tgt = feed.take(k, rast.stream)
            else:
                tgt = targets[k]
            losses.append(float(tr.step(sc.cameras[k], tgt)[0]))
            if use_feed:
                feed.release(k, rast.stream)
        torch.cuda.synchronize()
        assert rast.status()[0] == 0
        runs.append((p.data.cpu().numpy(), np.array(losses)))
    assert rel_l2(runs[1][0], runs[0][0]) < 1e-5
    assert np.allclose(runs[1][1], runs[0][1], rtol=1e-5)
