"""Rounds over the byte budget, colored in chunks of coloring order
(budget_mode="chunk") or with their columns in host memory (budget_mode=
"host", Alg. 3's fallback), against the CPU oracle.

Integer work, bit-exact: either way a run colors exactly as the oracle's
unrestricted run; no chunk's CSR passes the budget, and the host CSR equals
the device one."""
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


def _round1_bytes(ostats):
    # EARLIER CSR of round 1: 8 (n + 1) + 4 nnz, nnz half the oracle's two-sided rows
    n, nnz = int(ostats[0, 0]), int(ostats[0, 4]) // 2
    return 8 * (n + 1) + 4 * nnz


@pytest.mark.parametrize("n,q,pw,num,den,alpha,seed,parts", [
    (5000, 40, 0.3, 1, 8, 2.0, 6, 3),      # about three chunks in round 1
    (12000, 64, 0.25, 1, 16, 1.5, 2, 7),   # the n=1M law at a smaller size, many chunks
    (3000, 24, 0.5, 1, 4, 3.0, 9, 2),      # long lists
])
def test_chunked_run_matches_oracle(pc, orc, n, q, pw, num, den, alpha, seed, parts):
    chars = synth.pauli_weighted(n, q, pw, seed=seed)
    ref, rounds, ostats = orc.run(chars, seed, num, den, alpha)
    budget = _round1_bytes(ostats) // parts
    with pc.Picasso(_xz(pc, chars), q, seed=seed, palette=(num, den), alpha=alpha, byte_budget=budget,
                    budget_mode="chunk") as p:
        got, r = p.run()
        st = p.stats()
        used, peak, left = p.set_stats()
    assert r == rounds and np.array_equal(got.cpu().numpy(), ref)
    assert st["colors_used"] == int(ostats[:, 1].sum())
    assert st["round_chunks"] >= parts
    assert 0 < peak[0] <= budget and left == [0]


def test_fail_mode_and_single_row_limit(pc, orc):
    chars = synth.pauli_weighted(4000, 40, 0.3, seed=3)
    _, _, ostats = orc.run(chars, 3, 1, 8, 2.0)
    budget = _round1_bytes(ostats) // 3
    xz = _xz(pc, chars)
    # FAIL (the default): the first round over budget stops the run
    with pc.Picasso(xz, 40, seed=3, byte_budget=budget) as p:
        with pytest.raises(pc.PicassoError) as e:
            p.run()
        assert e.value.status == pc.ERR_BUDGET
    # CHUNK with a budget below one vertex's rows: nothing to cut
    with pc.Picasso(xz, 40, seed=3, byte_budget=64, budget_mode="chunk") as p:
        with pytest.raises(pc.PicassoError) as e:
            p.run()
        assert e.value.status == pc.ERR_BUDGET


def test_chunked_round_steps_equal_unchunked(pc):
    # one round through picasso_round: same colors and uncolored set as the
    # unchunked round
    chars = synth.pauli_weighted(20000, 64, 0.25, seed=4)
    xz = _xz(pc, chars)
    out = {}
    for mode, budget in (("fail", 0), ("chunk", 2_000_000)):
        with pc.Picasso(xz, 64, seed=4, palette=(1, 16), alpha=1.5, byte_budget=budget, budget_mode=mode) as p:
            left = p.round()
            st = p.stats()
            out[mode] = (left, p.colors().cpu().numpy(), p.vertices().cpu().numpy(), st["round_chunks"])
    assert out["chunk"][0] == out["fail"][0]
    assert np.array_equal(out["chunk"][1], out["fail"][1]) and np.array_equal(out["chunk"][2], out["fail"][2])
    assert out["chunk"][3] > 1 and out["fail"][3] == 0


@pytest.mark.parametrize("n,q,pw,num,den,alpha,seed,parts", [
    (5000, 40, 0.3, 1, 8, 2.0, 6, 3),
    (12000, 64, 0.25, 1, 16, 1.5, 2, 7),
])
def test_host_csr_run_matches_oracle(pc, orc, n, q, pw, num, den, alpha, seed, parts):
    # Alg. 3's fallback: rounds over the budget keep their columns in host
    # memory; the colors are those of the device rounds
    chars = synth.pauli_weighted(n, q, pw, seed=seed)
    ref, rounds, ostats = orc.run(chars, seed, num, den, alpha)
    budget = _round1_bytes(ostats) // parts
    with pc.Picasso(_xz(pc, chars), q, seed=seed, palette=(num, den), alpha=alpha, byte_budget=budget,
                    budget_mode="host") as p:
        got, r = p.run()
        st = p.stats()
    assert r == rounds and np.array_equal(got.cpu().numpy(), ref)
    assert st["colors_used"] == int(ostats[:, 1].sum())
    assert st["host_csr_rounds"] >= 1 and st["round_chunks"] == 0


@pytest.mark.parametrize("form", ["earlier", "full"])
def test_host_csr_equals_device_csr(pc, form):
    chars = synth.pauli_weighted(8000, 48, 0.25, seed=7)
    xz = _xz(pc, chars)
    out = {}
    for mode, budget in (("fail", 0), ("host", 100_000)):
        with pc.Picasso(xz, 48, seed=7, palette=(1, 8), alpha=2.0, csr=form, byte_budget=budget,
                        budget_mode=mode) as p:
            p.assign_lists(*p.round_params())
            p.build_conflicts()
            off, col = p.csr()
            k = p.color()
            out[mode] = (off.cpu().numpy(), col.cpu().numpy(), k, p.colors().cpu().numpy(),
                         p.stats()["host_csr_rounds"])
    assert np.array_equal(out["host"][0], out["fail"][0]) and np.array_equal(out["host"][1], out["fail"][1])
    assert out["host"][2] == out["fail"][2] and np.array_equal(out["host"][3], out["fail"][3])
    assert out["host"][4] == 1 and out["fail"][4] == 0


def test_host_csr_dynamic_order(pc, orc):
    chars = synth.pauli_weighted(4000, 48, 0.3, seed=12)
    ref, rounds, ostats = orc.run(chars, 4, 1, 8, 2.0, colorer="dynamic_par")
    budget = 8 * 4001 + 4 * int(ostats[0, 4]) // 4
    with pc.Picasso(_xz(pc, chars), 48, seed=4, palette=(1, 8), alpha=2.0, color="dynamic", byte_budget=budget,
                    budget_mode="host") as p:
        got, r = p.run()
        assert p.stats()["host_csr_rounds"] >= 1
    assert r == rounds and np.array_equal(got.cpu().numpy(), ref)


def test_host_csr_batch(pc, orc):
    # a batch context: rounds whose combined CSR passes the budget keep their
    # columns in host memory; every set colors as the oracle's own run
    specs = [(3000, 40, 0.3), (2500, 48, 0.25), (60, 24, 0.5)]
    sets = [synth.pauli_weighted(n, q, p, seed=3, stream=i) for i, (n, q, p) in enumerate(specs)]
    offs = [0]
    for c in sets:
        offs.append(offs[-1] + len(c))
    pad = np.zeros((offs[-1], 48), dtype=np.uint8)
    for k, c in enumerate(sets):
        pad[offs[k]:offs[k + 1], :c.shape[1]] = c
    seeds = [41, 42, 43]
    with pc.Picasso(_xz(pc, pad), 48, set_offsets=offs, seeds=seeds, byte_budget=200_000,
                    budget_mode="host") as p:
        got, _ = p.run()
        got = got.cpu().numpy()
        assert p.stats()["host_csr_rounds"] >= 1
    for k, c in enumerate(sets):
        ref, _, _ = orc.run(c, seeds[k], 1, 8, 2.0)
        assert np.array_equal(got[offs[k]:offs[k + 1]], ref), k
