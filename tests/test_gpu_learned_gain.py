"""What the trained initializer gains: fitted on converged Gaussians of plain 500-iteration runs,
it starts held-out scenes better than the paper's initializer (held-out-view PSNR after 100, 250
and 500 iterations), and the batched learned-init form reaches the plain form's 500-iteration
PSNR in at most half its GPU time."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_learned_init_beats_paper_init_on_held_out_scenes():
    from paper_2601_17354_gb300 import evaluate as E
    res = E.compare_initializers(train_seeds=[101, 102, 103, 104, 105, 106], eval_seeds=[201, 202],
                                 n=30000, width=320, height=240, focal=250.0, fit_steps=600)
    paper, learned = res.mean("paper"), res.mean("learned")
    assert res.fallbacks == 0
    for b in (100, 250, 500):
        assert learned[b] > paper[b], (b, learned, paper)


def test_batched_learned_form_halves_the_time_to_the_plain_psnr():
    from paper_2601_17354_gb300 import evaluate as E
    from paper_2601_17354_gb300.initializer import Initializer, LearnedInit
    init = Initializer()
    feats, targs = [], []
    for seed in range(300, 306):
        sd = E.make_scene(seed, 30000, 320, 240, 250.0)
        pi = init.paper_init(sd.points, 3)
        p = E.with_colour(pi.paper.clone())
        E.train_plain(p, sd, 500, seed=seed)
        feats.append(pi.features_bf16)
        targs.append(init.make_targets(pi, p))
    li = LearnedInit(init, seed=1)
    li.fit(feats, targs, steps=600)
    r = E.time_to_target([401, 402, 403], 30000, 320, 240, 250.0, views_per_step=1, learned=li)
    assert r["all_reached"] and r["ratio"] <= 0.5, r
