"""Checkpoint / resume between rounds: a context that loads a saved state
colors exactly as the uninterrupted run (and as the oracle)."""
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


@pytest.mark.parametrize("stop", [0, 1, 3])
def test_resume_single_set(pc, orc, stop):
    chars = synth.pauli_weighted(3000, 40, 0.3, seed=31)
    xz = pc.pack(torch.from_numpy(chars).cuda())
    ref, rounds_ref, _ = orc.run(chars, 17, 1, 16, 1.5)
    with pc.Picasso(xz, 40, seed=17, palette=(1, 16), alpha=1.5) as p:
        for _ in range(stop):
            p.round()
        blob = p.save_state()
        a, ra = p.run()
        a = a.cpu().numpy()
    with pc.Picasso(xz, 40, seed=17, palette=(1, 16), alpha=1.5) as p2:
        p2.load_state(blob)
        b, rb = p2.run()
        b = b.cpu().numpy()
    assert np.array_equal(a, ref) and np.array_equal(b, ref)
    assert ra == rb == rounds_ref


def test_resume_batch(pc, orc):
    specs = [(800, 16, 0.3), (1500, 64, 0.25), (5, 24, 0.5), (1200, 48, 0.4)]
    sets = [synth.pauli_weighted(n, q, p, seed=9, stream=i) for i, (n, q, p) in enumerate(specs)]
    q = 64
    offs = [0]
    for c in sets:
        offs.append(offs[-1] + len(c))
    pad = np.zeros((offs[-1], q), dtype=np.uint8)
    for k, c in enumerate(sets):
        pad[offs[k]:offs[k + 1], :c.shape[1]] = c
    xz = pc.pack(torch.from_numpy(pad).cuda())
    seeds = [70 + k for k in range(len(sets))]
    kw = dict(palette=(1, 8), alpha=2.0, set_offsets=offs, seeds=seeds)
    with pc.Picasso(xz, q, **kw) as p:
        p.round()
        p.round()
        blob = p.save_state()
        stats_a = p.set_stats()
    with pc.Picasso(xz, q, **kw) as p2:
        p2.load_state(blob)
        assert p2.set_stats() == stats_a
        b, _ = p2.run()
        b = b.cpu().numpy()
    for k, c in enumerate(sets):
        ref, _, _ = orc.run(c, seeds[k], 1, 8, 2.0)
        assert np.array_equal(b[offs[k]:offs[k + 1]], ref), k


def test_state_errors(pc):
    chars = synth.pauli_weighted(1000, 20, 0.3, seed=1)
    xz = pc.pack(torch.from_numpy(chars).cuda())
    with pc.Picasso(xz, 20, seed=1) as p:
        p.round()
        blob = p.save_state()
        P, L, base = p.round_params()
        p.assign_lists(P, L, base)
        with pytest.raises(pc.PicassoError) as e:
            p.save_state()
        assert e.value.status == pc.ERR_STATE
    with pc.Picasso(xz, 20, seed=2) as p:  # another seed: another run
        with pytest.raises(pc.PicassoError) as e:
            p.load_state(blob)
        assert e.value.status == pc.ERR_INVALID_ARG
    with pc.Picasso(xz, 20, seed=1) as p:
        with pytest.raises(pc.PicassoError):
            p.load_state(blob[:-4])
        bad = bytearray(blob)
        bad[0] ^= 1
        with pytest.raises(pc.PicassoError):
            p.load_state(bytes(bad))
        p.load_state(blob)  # the context is unchanged by the failed loads
        c, _ = p.run()
        assert (c >= 0).all()
