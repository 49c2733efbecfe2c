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


def _regular(pc, xz, q, seed, palette, alpha):
    with pc.Picasso(xz, q, seed=seed, palette=palette, alpha=alpha) as p:
        colors, rounds = p.run()
        return colors.cpu().numpy(), rounds


def test_static_entry_matches_run_on_two_calls_in_a_row(pc):
    cases = [
        (synth.pauli_uniform(2000, 20, seed=0), 20, 0, (1, 8), 2.0),
        (synth.pauli_weighted(1800, 64, 0.25, seed=5), 64, 3, (1, 16), 1.5),
    ]
    prepared = []
    for chars, q, seed, pal, alpha in cases:
        xz = _xz(pc, chars)
        prepared.append((xz, q, seed, pal, alpha, _regular(pc, xz, q, seed, pal, alpha)))
    outs = [torch.full((x[0].shape[0],), 7, dtype=torch.int32, device="cuda") for x in prepared]
    torch.cuda.synchronize()
    free = []
    for (xz, q, seed, pal, alpha, (want, want_rounds)), out in zip(prepared, outs):
        got, rounds = pc.run_small_static(xz, q, seed=seed, palette=pal, alpha=alpha, out=out)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        assert rounds == want_rounds
        assert np.array_equal(got.cpu().numpy(), want)
    # the second call found everything it needed in place: no device memory moved
    assert free[1] == free[0]


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
