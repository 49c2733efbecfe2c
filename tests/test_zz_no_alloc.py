"""The allocation-free whole-run entry point (picasso_run_small_static).

It is meant for callers that cannot allocate device memory while they work,
for example services whose fixed memory pool owns the GPU, or hosts that
forbid cudaMalloc on their hot path.  It must give exactly the colors of the
ordinary entry points (init + run), call after call, although all of its
temporaries live in one shared static device array.  This file is collected
last so that a run stopping at the first failure has run everything else.
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


def _regular(pc, xz, q, seed, palette, alpha, color="auto"):
    with pc.Picasso(xz, q, seed=seed, palette=palette, alpha=alpha, color=color) as p:
        colors, rounds = p.run()
        return colors.cpu().numpy(), rounds


CASES = [
    (synth.pauli_uniform(2000, 20, seed=0), 20, 0, (1, 8), 2.0),
    (synth.pauli_weighted(1800, 64, 0.25, seed=5), 64, 3, (1, 16), 1.5),
]


def test_static_entry_matches_run_on_two_calls_in_a_row(pc, orc):
    prepared = []
    for chars, q, seed, pal, alpha in CASES:
        xz = _xz(pc, chars)
        prepared.append((xz, q, seed, pal, alpha, _regular(pc, xz, q, seed, pal, alpha)))
        # the ordinary entry points agree with the oracle's whole run
        ref, ref_rounds, _ = orc.run(chars, seed, pal[0], pal[1], alpha)
        assert prepared[-1][-1][1] == ref_rounds and np.array_equal(prepared[-1][-1][0], ref)
    outs = [torch.full((x[0].shape[0],), 7, dtype=torch.int32, device="cuda") for x in prepared]
    torch.cuda.synchronize()
    requests0 = pc.memory_requests()
    free = []
    for (xz, q, seed, pal, alpha, (want, want_rounds)), out in zip(prepared, outs):
        got, rounds = pc.run_small_static(xz, q, seed=seed, palette=pal, alpha=alpha, out=out)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        assert rounds == want_rounds
        assert np.array_equal(got.cpu().numpy(), want)
    # the library made no memory request during either call, the first one
    # included, and the second call found everything it needed in place
    assert pc.memory_requests() == requests0
    assert free[1] == free[0]


def test_static_entry_sweep_and_exhausted_waits(pc, orc):
    # SWEEP colors with the dependency sweeps alone, and one poll per bounded
    # wait sends a round with a real wait to the same sweeps: both give the
    # colors of the ordinary entry points and of the oracle
    chars, q, seed, pal, alpha = CASES[1]
    xz = _xz(pc, chars)
    want, want_rounds = _regular(pc, xz, q, seed, pal, alpha, color="sweep")
    ref, _, _ = orc.run(chars, seed, pal[0], pal[1], alpha)
    assert np.array_equal(want, ref)
    for kw in ({"color": "sweep"}, {"wait_polls": 1}):
        got, rounds = pc.run_small_static(xz, q, seed=seed, palette=pal, alpha=alpha, **kw)
        assert rounds == want_rounds and np.array_equal(got.cpu().numpy(), ref)


def test_static_entry_config_checks(pc):
    chars, q, seed, pal, alpha = CASES[0]
    xz = _xz(pc, chars)
    with pytest.raises(pc.PicassoError) as e:  # Alg. 2's dynamic order is not built here
        pc.run_small_static(xz, q, seed=seed, color="dynamic")
    assert e.value.status == pc.ERR_UNSUPPORTED
    with pytest.raises(pc.PicassoError) as e:  # round 1's CSR alone passes 100 KB
        pc.run_small_static(xz, q, seed=seed, palette=pal, alpha=alpha, byte_budget=100_000)
    assert e.value.status == pc.ERR_BUDGET
    with pc.Picasso(xz, q, seed=seed, palette=pal, alpha=alpha, byte_budget=100_000) as p:
        with pytest.raises(pc.PicassoError) as e2:
            p.run()
        assert e2.value.status == pc.ERR_BUDGET


def test_static_entry_rejects_sizes_beyond_its_limits(pc):
    chars = synth.pauli_uniform(2049, 10, seed=1)
    xz = _xz(pc, chars)
    with pytest.raises(pc.PicassoError) as e:
        pc.run_small_static(xz, 10)
    assert e.value.status == pc.ERR_UNSUPPORTED
    small = _xz(pc, synth.pauli_uniform(100, 10, seed=2))
    with pytest.raises(pc.PicassoError) as e:  # L = ceil(30 ln 100) = 139 > 32
        pc.run_small_static(small, 10, palette=(1, 1), alpha=30.0)
    assert e.value.status == pc.ERR_UNSUPPORTED
