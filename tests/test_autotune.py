"""Autotuner search logic on a synthetic cost model (no GPU), and on the GPU:
a tuned schedule gives the same depth and parent as the defaults."""
import numpy as np
import pytest

from paper_1803_03922_gb300 import autotune


def _cost(opts):
    # separable bowl with its minimum at alpha 30, beta 36, 3 CTAs/SM
    c = (np.log(opts.get("alpha", 15) / 30.0)) ** 2 + (np.log(opts.get("beta", 18) / 36.0)) ** 2
    c += 0.0 if opts.get("blocks_per_sm", 2) == 3 else 0.1
    if opts.get("schedule") == autotune.PAPER:
        c += 1.0  # the paper rule is worse in this model
    if opts.get("schedule") == autotune.MASK:
        m = opts["schedule_mask"]
        c += 0.05 * bin(m ^ 0b0110).count("1") - 0.2  # best per-level schedule: levels 1,2 backward
    return 1.0 + c


def test_coordinate_descent_finds_the_bowl_minimum():
    best, t = autotune.coordinate_descent(_cost, {"alpha": 15, "beta": 18, "blocks_per_sm": 2},
                                          autotune.RUN_SPACE)
    assert best == {"alpha": 30, "beta": 36, "blocks_per_sm": 3}
    assert t == pytest.approx(1.0)


def test_greedy_mask_flips_towards_the_best_schedule():
    best, t = autotune.greedy_mask(_cost, {"alpha": 30}, [0, 0, 1, 1, 0])  # heuristic took 0b01100
    assert best["schedule"] == autotune.MASK and best["schedule_mask"] == 0b0110


def test_tune_picks_threshold_and_reports_speedup():
    def ev_for(th):
        return lambda o: _cost(o) + (0.0 if th == 128 else 0.5)

    res = autotune.tune(ev_for, lambda th, o: [0, 1, 1, 0], ths=(32, 64, 128))
    assert res.th == 128
    assert res.options["alpha"] == 30 and res.options["beta"] == 36
    assert res.speedup > 1.0 and len(res.trials) > 10


@pytest.mark.gpu
def test_tuned_schedule_is_bit_exact():
    from tests.gpu_util import need_cuda

    torch = need_cuda()
    import graphgen
    import oracle

    scale = 14
    n = 1 << scale
    hs, hd = graphgen.rmat_host(scale, seed=14)
    og = oracle.Graph(n, hs, hd)
    mask = graphgen.nonisolated_mask_host(n, hs, hd)
    sources = graphgen.sample_sources(mask, 8, seed=3)
    src = torch.from_numpy(hs).cuda()
    dst = torch.from_numpy(hd).cuda()
    res, g = autotune.device_tuner(src, dst, n, sources, runs=1, ths=(16, 64))
    assert res.th in (16, 64) and res.seconds > 0
    for s in sources:
        d, p = g.run(int(s))
        want_d, want_p = og.bfs(int(s))
        assert np.array_equal(d.cpu().numpy(), want_d) and np.array_equal(p.cpu().numpy(), want_p)


def test_th_rule_per_scale():
    """Sec. VI-B: about sqrt(2) per scale, 64 at scale 30 and 128 at scale 32."""
    from paper_1803_03922_gb300.autotune import th_for_scale, th_goals, th_space_for_scale

    assert th_for_scale(30) == 64 and th_for_scale(32) == 128 and th_for_scale(28) == 32
    assert [th_for_scale(s) for s in (22, 24, 26)] == [4, 8, 16]
    for s in range(10, 40):
        assert th_for_scale(s + 2) in (2 * th_for_scale(s), 2 * th_for_scale(s) - 1, 2 * th_for_scale(s) + 1) \
            or th_for_scale(s) == 1
    assert 16 in th_space_for_scale(26) and 8 in th_space_for_scale(26) and 32 in th_space_for_scale(26)
    row = {"delegates": 10, "nn_pct": 12.0}
    assert th_goals(row, 100) == {"delegates_under_4n_over_p": True, "nn_under_10pct": False}


@pytest.mark.gpu
def test_batch_alpha_tuning_keeps_results():
    """The batched form's schedule search (alpha of the union frontier) leaves the
    graph at the best alpha; every query still gets the oracle's result."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import numpy as np

    import graphgen
    import oracle
    import paper_1803_03922_gb300 as bfs
    from paper_1803_03922_gb300.autotune import tune_batch_alpha

    scale = 13
    n = 1 << scale
    src, dst = graphgen.rmat_host(scale, seed=413)
    og = oracle.Graph(n, src, dst)
    g = bfs.Graph(np.ascontiguousarray(src), np.ascontiguousarray(dst), n, th=32)
    mask = (np.diff(og.csr()[0]) > 0).astype(np.uint8)
    sources = graphgen.sample_sources(mask, 128, seed=4131)
    best, times = tune_batch_alpha(g, sources, alphas=(2, 15, 120), batches=2)
    assert best in times and g.opt.alpha == best and len(times) == 3
    b = bfs.Batch(g)
    d, p = b.run(sources[:64])
    want_d, want_p = og.bfs_batch_u8(sources[:64])
    assert np.array_equal(d.cpu().numpy(), want_d) and np.array_equal(p.cpu().numpy(), want_p)
    b.close()
    g.close()
