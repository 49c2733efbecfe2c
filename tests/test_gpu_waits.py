"""Bounded device waits that run out on purpose.

The ordered coloring (static Random order, first fit; Sec. III-B) lets a vertex
wait for an earlier neighbour still undecided at a color it needs.  Every such
wait polls at most cfg.wait_polls times; then the kernel reports it and
returns.  The per-round path recolors the round with the sweep kernel, the
small-round engine hands the round back to the per-round path.  With one poll
per wait those recovery paths run in every round that has a real wait, and
the colors must still be the oracle's.  Nothing here can hang or fault: the
limit is a poll count, and the kernels return when it is reached.
"""
import numpy as np
import pytest
import torch

from paper_2401_06713_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pc():
    from paper_2401_06713_b300 import build, picasso

    build.build()
    assert torch.cuda.is_available()
    return picasso


def _xz(pc, chars):
    return pc.pack(torch.from_numpy(np.ascontiguousarray(chars)).cuda())


def _run(pc, chars, seed, palette, alpha, **kw):
    with pc.Picasso(_xz(pc, chars), chars.shape[1], seed=seed, palette=palette, alpha=alpha, **kw) as p:
        colors, rounds = p.run()
        return colors.cpu().numpy(), rounds, p.stats()


def test_per_round_waits_run_out(pc, orc):
    # the n = 1M law at n = 20,000, every round on the per-round path
    chars = synth.pauli_weighted(20_000, 64, 0.25, seed=3)
    ref, rounds, _ = orc.run(chars, 0, 1, 16, 1.5)
    got, r, st = _run(pc, chars, 0, (1, 16), 1.5, small="off", wait_polls=1)
    assert st["ordered_fallbacks"] > 0
    assert r == rounds and np.array_equal(got, ref)
    # the default limit is never reached on the same workload
    got2, _, st2 = _run(pc, chars, 0, (1, 16), 1.5, small="off")
    assert st2["ordered_fallbacks"] == 0 and np.array_equal(got2, ref)


def test_engine_waits_run_out(pc, orc):
    # every round fits the small-round engine; each round it starts hands
    # back after a wait runs out, and the per-round path finishes that round
    chars = synth.pauli_weighted(8000, 64, 0.25, seed=5)
    ref, rounds, _ = orc.run(chars, 2, 1, 16, 1.5)
    got, r, st = _run(pc, chars, 2, (1, 16), 1.5, wait_polls=1)
    assert st["small_stops"] > 0
    assert r == rounds and np.array_equal(got, ref)
    got2, _, st2 = _run(pc, chars, 2, (1, 16), 1.5)
    assert st2["small_stops"] == 0 and st2["small_rounds"] > 0 and np.array_equal(got2, ref)


def test_batch_waits_run_out(pc, orc):
    # a batch of three sets: per-set colors stay the oracle's
    sets = [synth.pauli_weighted(n, 48, 0.25, seed=n) for n in (3000, 7000, 1200)]
    chars = np.concatenate(sets)
    offs = np.concatenate([[0], np.cumsum([len(x) for x in sets])])
    with pc.Picasso(_xz(pc, chars), 48, seed=10, palette=(1, 8), alpha=2.0, set_offsets=offs,
                    wait_polls=1) as p:
        got, _ = p.run()
        got = got.cpu().numpy()
        st = p.stats()
    assert st["small_stops"] + st["ordered_fallbacks"] > 0
    for k, x in enumerate(sets):
        ref, _, _ = orc.run(x, 10 + k, 1, 8, 2.0)
        assert np.array_equal(got[offs[k]:offs[k + 1]], ref)


def test_wait_polls_validated(pc):
    chars = synth.pauli_uniform(100, 10, seed=1)
    for bad in (-1, (1 << 30) + 1):
        with pytest.raises(pc.PicassoError) as e:
            pc.Picasso(_xz(pc, chars), 10, wait_polls=bad)
        assert e.value.status == pc.ERR_INVALID_ARG
