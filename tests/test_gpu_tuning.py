"""Kernel variants of the grid-wide rounds (block size x points per thread),
the cutover range and the autotuner: every setting gives the oracle's hull and
per-generation live counts."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

VARIANTS = [(256, 16), (256, 8), (128, 16), (128, 8)]


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("name", ["square", "disk", "circle", "degenerate"])
@pytest.mark.parametrize("mode", ["quad", "chord"])
def test_variants_match_oracle(qh, name, mode):
    p = synth.make(name, 300_000, seed=5)
    want, live = oracle.quickhull(p, mode)
    d = _dev(p)
    plan = qh.Plan(len(p), 1, mode=qh.MODE_QUAD if mode == "quad" else qh.MODE_CHORD)
    for threads, ipt in VARIANTS:
        plan.set_block(threads)
        plan.set_items_per_thread(ipt)
        t = plan.tuning()
        assert t["threads_per_block"] == threads and t["items_per_thread"] == ipt
        for cut in sorted({threads * ipt, 3072, 4096}):
            if cut < threads * ipt:
                continue
            plan.set_tuning(cut)
            got = qh.hull2d(d, plan).cpu().numpy()
            st = plan.stats()
            assert np.array_equal(got, want), (threads, ipt, cut)
            assert st["device_status"] == 0
            assert st["live"] == live.tolist(), (threads, ipt, cut)
    plan.close()


def test_cutover_range_follows_tile(qh):
    plan = qh.Plan(10_000, 1)
    t = plan.tuning()
    assert (t["threads_per_block"], t["items_per_thread"]) == (256, 16)
    with pytest.raises(qh.QhError):
        plan.set_tuning(2048)  # below the 4096-point tile of 256 threads x 16 points
    plan.set_items_per_thread(8)
    plan.set_tuning(2048)
    assert plan.tuning()["cutover"] == 2048
    plan.set_block(128)
    plan.set_tuning(1024)
    assert plan.tuning()["cutover"] == 1024
    plan.set_items_per_thread(16)  # raises the cutover to the 2048-point tile
    assert plan.tuning()["cutover"] == 2048
    with pytest.raises(qh.QhError):
        plan.set_tuning(4097)
    with pytest.raises(qh.QhError):
        plan.set_block(192)
    with pytest.raises(qh.QhError):
        plan.set_items_per_thread(4)
    plan.close()


def test_autotune_single_set(qh):
    p = synth.disk(500_000, seed=6)
    plan = qh.Plan(len(p), 1)
    d = _dev(p)
    t = plan.autotune(d, reps=2)
    assert (t["threads_per_block"], t["items_per_thread"]) in VARIANTS
    assert t["threads_per_block"] * t["items_per_thread"] <= t["cutover"] <= 4096
    assert t["grid_ctas_per_sm"] >= 1
    assert np.array_equal(qh.hull2d(d, plan).cpu().numpy(), oracle.hull2d(p))
    plan.close()


def test_autotune_cache_and_reuse(qh, tmp_path):
    """A tuning stored under the GPU, build and configuration is applied by a later plan without timing."""
    p = synth.circle(400_000, seed=12)
    want = oracle.hull2d(p)
    d = _dev(p)
    path = str(tmp_path / "tune.json")
    plan = qh.Plan(len(p), 1)
    t = plan.autotune(d, reps=1, cache=path)
    assert t["cached"] is False
    assert np.array_equal(qh.hull2d(d, plan).cpu().numpy(), want)
    stored = qh.tune_cache_load(path)
    assert len(stored) == 1
    plan.close()
    plan2 = qh.Plan(len(p), 1)
    t2 = plan2.autotune(d, reps=1, cache=path)
    assert t2["cached"] is True
    assert {k: t2[k] for k in stored[next(iter(stored))]} == stored[next(iter(stored))]
    assert np.array_equal(qh.hull2d(d, plan2).cpu().numpy(), want)
    t3 = plan2.autotune(d[:300_000], reps=1, cache=path)  # another configuration: tuned, then stored
    assert t3["cached"] is False and len(qh.tune_cache_load(path)) == 2
    assert np.array_equal(qh.hull2d(d[:300_000], plan2).cpu().numpy(), oracle.hull2d(p[:300_000]))
    plan2.close()


def test_autotune_batched(qh):
    import torch

    p, off = synth.batched(200, seed=7, min_size=16, max_size=60_000)
    plan = qh.Plan(len(p), 200)
    d, doff = _dev(p), torch.from_numpy(off).cuda()
    t = plan.autotune(d, doff, reps=1)
    assert (t["threads_per_block"], t["items_per_thread"]) in VARIANTS
    out, counts = qh.hull2d_batched(d, doff, plan)
    out, counts = out.cpu().numpy(), counts.cpu().numpy()
    want_out, want_counts = oracle.hull2d_batched(p, off)
    assert np.array_equal(counts, want_counts)
    for s in range(len(counts)):
        a = int(off[s])
        assert np.array_equal(out[a:a + counts[s]], want_out[a:a + counts[s]]), s
    plan.close()
