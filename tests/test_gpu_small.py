"""The small-round engine (one cooperative launch for every round of at most
16384 vertices) against the CPU oracle and against the per-round path.

Integer work, so every comparison is bit-exact: whole runs of Alg. 1 (colors,
rounds, colors used), runs that start above the engine's size and hand over to
it, stops at the round limit and the byte budget, and a checkpoint taken where
the engine stopped."""
import numpy as np
import pytest
import torch

from paper_2401_06713_b300 import synth

pytestmark = pytest.mark.gpu

ENGINE_MAX = 16384


@pytest.fixture(scope="module")
def pc():
    from paper_2401_06713_b300 import build, picasso

    build.build()
    assert torch.cuda.is_available()
    return picasso


def _xz(pc, chars):
    return pc.pack(torch.from_numpy(np.ascontiguousarray(chars)).cuda())


def _run(pc, chars, seed, num, den, alpha, small, **kw):
    with pc.Picasso(_xz(pc, chars), chars.shape[1], seed=seed, palette=(num, den), alpha=alpha, small=small,
                    **kw) as p:
        got, r = p.run()
        st = p.stats()
        st["set_stats"] = p.set_stats()
        return got.cpu().numpy(), r, st


@pytest.mark.parametrize("n,q,pw,num,den,alpha,seed", [
    (ENGINE_MAX, 64, 0.25, 1, 16, 1.5, 0),   # the engine's largest round, the n=1M law
    (9001, 48, 0.3, 1, 8, 2.0, 4),           # ragged, the default palette
    (3000, 20, 0.5, 1, 4, 3.0, 7),           # P = n/4, long lists
    (777, 6, 0.5, 1, 8, 2.0, 1),             # few distinct strings (q = 6): duplicates
])
def test_engine_matches_oracle(pc, orc, n, q, pw, num, den, alpha, seed):
    chars = synth.pauli_weighted(n, q, pw, seed=seed)
    ref, rounds, ostats = orc.run(chars, seed, num, den, alpha)
    got, r, st = _run(pc, chars, seed, num, den, alpha, "auto")
    assert r == rounds
    assert np.array_equal(got, ref)
    assert st["colors_used"] == int(ostats[:, 1].sum())
    assert st["small_rounds"] == rounds and st["small_stops"] == 0
    assert st["rounds_done"] == rounds
    # the engine's CSR accounting matches the oracle's rows: each pair once,
    # at its later endpoint
    assert st["nnz_total"] == int(ostats[:, 4].sum()) // 2
    assert st["logical_pairs"] == int(sum(m * (m - 1) // 2 for m in ostats[:, 0]))


def test_handover_from_per_round_path(pc, orc):
    # round 1 (n > 16384) runs per round, the rest in the engine
    chars = synth.pauli_weighted(24000, 64, 0.25, seed=11)
    ref, rounds, ostats = orc.run(chars, 3, 1, 16, 1.5)
    got, r, st = _run(pc, chars, 3, 1, 16, 1.5, "auto")
    assert r == rounds and np.array_equal(got, ref)
    big = int((ostats[:, 0] > ENGINE_MAX).sum())
    assert big >= 1 and st["small_rounds"] == rounds - big


def test_engine_equals_per_round_path(pc):
    chars = synth.pauli_weighted(12000, 64, 0.25, seed=5)
    a, ra, sa = _run(pc, chars, 9, 1, 16, 1.5, "auto")
    b, rb, sb = _run(pc, chars, 9, 1, 16, 1.5, "off")
    assert ra == rb and np.array_equal(a, b)
    assert sa["colors_used"] == sb["colors_used"]
    assert sa["nnz_total"] == sb["nnz_total"] and sa["logical_pairs"] == sb["logical_pairs"]
    assert sb["small_rounds"] == 0 and sa["small_rounds"] == ra
    # colors used, largest CSR bytes of a round, nothing left
    assert sa["set_stats"] == sb["set_stats"]


def test_engine_launch_count(pc):
    chars = synth.pauli_weighted(8000, 64, 0.25, seed=2)
    xz = _xz(pc, chars)
    with pc.Picasso(xz, 64, seed=1, palette=(1, 16), alpha=1.5) as p:
        k0 = pc.kernel_launches()
        _, r = p.run()
        torch.cuda.synchronize()
        k = pc.kernel_launches() - k0
    # iota of V_1, the engine's three stages (grid, cluster, block), the
    # gather of the result (none: all colored)
    assert r > 5 and k <= 5, (r, k)


@pytest.mark.parametrize("stop_after", [1, 4])
def test_round_limit_and_resume(pc, orc, stop_after):
    chars = synth.pauli_weighted(5000, 40, 0.3, seed=21)
    ref, rounds, _ = orc.run(chars, 6, 1, 8, 2.0)
    xz = _xz(pc, chars)
    states = {}
    for small in ("auto", "off"):
        with pc.Picasso(xz, 40, seed=6, palette=(1, 8), alpha=2.0, max_rounds=stop_after, small=small) as p:
            with pytest.raises(pc.PicassoError) as e:
                p.run()
            assert e.value.status == pc.ERR_INTERNAL
            st = p.stats()
            states[small] = (p.colors().cpu().numpy(), st["round"], st["colors_used"], st["n_round"],
                             p.vertices().cpu().numpy(), p.save_state())
    ca, ra, ua, na, ga, blob = states["auto"]
    cb, rb, ub, nb, gb, _ = states["off"]
    assert ra == rb == stop_after + 1 and ua == ub and na == nb
    assert np.array_equal(ca, cb) and np.array_equal(ga, gb)
    # where the engine stopped, a checkpoint resumes to the oracle's colors
    with pc.Picasso(xz, 40, seed=6, palette=(1, 8), alpha=2.0) as p2:
        p2.load_state(blob)
        got, r = p2.run()
        assert r == rounds and np.array_equal(got.cpu().numpy(), ref)


def test_byte_budget_stop(pc):
    chars = synth.pauli_weighted(6000, 64, 0.25, seed=13)
    xz = _xz(pc, chars)
    # enough for the first round's CSR only if it were a quarter of its size
    full = _run(pc, chars, 2, 1, 16, 1.5, "off")[2]
    budget = 8 * 6001 + 4 * 1000
    assert full["nnz_total"] > 1000
    out = {}
    for small in ("auto", "off"):
        with pc.Picasso(xz, 64, seed=2, palette=(1, 16), alpha=1.5, byte_budget=budget, small=small) as p:
            with pytest.raises(pc.PicassoError) as e:
                p.run()
            assert e.value.status == pc.ERR_BUDGET
            st = p.stats()
            out[small] = (st["round"], st["n_round"], st["colors_used"], p.colors().cpu().numpy())
    assert out["auto"][:3] == out["off"][:3]
    assert np.array_equal(out["auto"][3], out["off"][3])


def test_engine_not_used_off_default_paths(pc, orc):
    # explicit conflict or coloring algorithms and the FULL form keep the
    # per-round path; the colors are the same
    chars = synth.pauli_weighted(2500, 32, 0.3, seed=3)
    ref, rounds, _ = orc.run(chars, 1, 1, 8, 2.0)
    for kw in (dict(algo="bucket"), dict(color="sweep"), dict(csr="full")):
        got, r, st = _run(pc, chars, 1, 1, 8, 2.0, "auto", **kw)
        assert r == rounds and np.array_equal(got, ref), kw
        assert st["small_rounds"] == 0, kw
