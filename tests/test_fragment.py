"""Fragment meta-heuristic (Sec. II; App. A, Fig. 5) with SA fragment anneals: the oracle
pinned on CPU, the GPU path bit-exact against it."""
import numpy as np
import pytest

from oracle import oracle as o
from paper_2501_17267_gb300 import workloads as wl


def _class(L, l, i):
    x, y, z = i % L, (i // L) % L, i // (L * L)
    return (x % l) + l * ((y % l) + l * (z % l))


@pytest.mark.parametrize("S", [0, 1, 4])
def test_single_site_fragments_follow_the_draws(S):
    """l = 1: a fragment is its own site with no bond inside it, so every attempt is
    accepted (x = 0) and the spin flips every sweep; all reads have energy 0, read 0
    decides: s_i = (-1)^S times read 0's initial value, bit 31 of word 0 of the block at
    counter (i, 0xFFFFFFFF, 0, 5)."""
    L, seed, iid = 4, 77, 3
    J3, _, _ = o.generate(L, 5, (1 / 3, 1 / 3, 1 / 3), True)
    spins, E = o.fragment_run(L, J3, 1, S, 0.5, 4.0, seed, iid)
    k0, k1 = seed & 0xFFFFFFFF, (seed >> 32) ^ iid
    for i in range(L ** 3):
        w = int(o.philox([i, 0xFFFFFFFF, 0, 5], [k0, k1])[0])
        assert spins[i] == (-1 if w >> 31 else 1) * (-1) ** S
    assert E == o.energy(L, J3, spins)


@pytest.mark.parametrize("L,l", [(6, 3), (10, 5)])
def test_last_wave_spins_are_locally_stable(L, l):
    """A spin fixed in the last wave sees all six neighbours fixed inside its fragment;
    at a cold end of the schedule every read leaves it aligned with its field, so
    s_i h_i <= 0 there (h_i even: a wrong spin would need a move of cost >= 4 at beta 8)."""
    J3, _, egs = o.generate(L, 9 + L, (0, 0, 1), True)
    spins, E = o.fragment_run(L, J3, l, 6, 0.5, 8.0, 1, 0)
    assert set(np.unique(spins)) <= {-1, 1}
    assert E == o.energy(L, J3, spins) and E >= egs
    last = l ** 3 - 1
    checked = 0
    for i in range(L ** 3):
        if _class(L, l, i) == last:
            assert spins[i] * o.local_field(L, J3, spins, i) <= 0
            checked += 1
    assert checked == (L // l) ** 3


def test_second_to_last_wave_takes_the_fragment_optimum():
    """l = 3: at wave 25 a fragment has two free spins, its centre c and c + x (class 26),
    whose own +x bond leaves the cube and is dropped.  All other cube sites are fixed
    (their final values).  Over the four states of the pair, the lowest cube energy
    (brute force) fixes c whenever the optimal states agree on it: the best of 32 cold
    reads must have found it."""
    L, l = 6, 3
    J3, _, _ = o.generate(L, 44, (0, 0, 1), True)
    spins, _ = o.fragment_run(L, J3, l, 8, 0.5, 8.0, 2, 0)
    site = lambda x, y, z: o.site(L, x, y, z)
    decided = 0
    for i in range(L ** 3):
        if _class(L, l, i) != 25:
            continue
        x, y, z = i % L, (i // L) % L, i // (L * L)
        lo = (x - 1, y - 1, z - 1)
        cube = {site(lo[0] + a, lo[1] + b, lo[2] + c): (a, b, c) for a in range(3) for b in range(3)
                for c in range(3)}
        n = site(x + 1, y, z)
        best = {}
        for sc in (-1, 1):
            for sn in (-1, 1):
                s = spins.copy()
                s[i], s[n] = sc, sn
                e = 0
                for j, (a, b, c) in cube.items():  # bonds inside the cube, each once
                    for d, off in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
                        if (a, b, c)[d] + 1 < 3:
                            k = site(lo[0] + a + off[0], lo[1] + b + off[1], lo[2] + c + off[2])
                            e += int(J3[j, d]) * int(s[j]) * int(s[k])
                best[(sc, sn)] = e
        emin = min(best.values())
        opt_c = {sc for (sc, sn), e in best.items() if e == emin}
        if len(opt_c) == 1:
            assert spins[i] == opt_c.pop()
            decided += 1
    assert decided >= 4


def test_bad_parameters_are_rejected():
    J3, _, _ = o.generate(6, 1, (1 / 3, 1 / 3, 1 / 3), True)
    for l in (2, 4, 6, 5):  # even, or not dividing L, or not below L
        with pytest.raises(ValueError):
            o.fragment_run(6, J3, l, 2, 0.5, 3.0)


# --------------------------------------------------------------------------- GPU

@pytest.fixture(scope="module")
def sg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2501_17267_gb300 import build
    build.build()
    from paper_2501_17267_gb300 import sg as mod
    return mod


@pytest.mark.gpu
@pytest.mark.parametrize("L,l,S", [(6, 3, 10), (10, 5, 3), (12, 3, 5), (2, 1, 3), (14, 7, 1)])
def test_fragment_run_matches_oracle(sg, L, l, S):
    inst = sg.Instance.create(L, 3100 + L, (0, 0, 1), True)
    J3, _, egs = inst.get()
    res = sg.fragment_run(inst, l, S, 0.5, 6.0, seed=5, instance_id=2, spins="host")
    ospins, oE = o.fragment_run(L, J3, l, S, 0.5, 6.0, 5, 2)
    assert np.array_equal(res["spins"], ospins)
    assert res["E"] == oE
    assert res["eps"] == o.epsilon(oE, egs)


@pytest.mark.gpu
def test_fragment_run_general_couplings(sg):
    """|J| = 2 and zero couplings (the fragment fields take any even value up to 12)."""
    L, l = 6, 3
    J3 = wl.random_couplings(41, L, jmax=2)
    inst = sg.Instance.from_couplings(L, J3)
    res = sg.fragment_run(inst, l, 6, 0.3, 3.0, seed=8, spins="host")
    ospins, oE = o.fragment_run(L, J3, l, 6, 0.3, 3.0, 8, 0)
    assert np.array_equal(res["spins"], ospins) and res["E"] == oE


@pytest.mark.gpu
def test_fragment_batch_equals_separate_runs(sg):
    insts = [sg.Instance.create(10, 3200 + k, (0, 0, 1), True) for k in range(3)]
    params = [dict(l=5, sweeps=4, beta0=0.5, beta1=6.0, seed=1, instance_id=k) for k in range(3)]
    batch = sg.fragment_run_batch(insts, params, spins="host")
    for inst, p, b in zip(insts, params, batch):
        one = sg.fragment_run(inst, spins="host", **p)
        assert np.array_equal(one["spins"], b["spins"]) and one["E"] == b["E"]
    with pytest.raises(sg.SGError):
        sg.fragment_run(insts[0], 3, 4, 0.5, 6.0)  # 3 does not divide 10


def test_fit_inverse_L_recovers_the_asymptote():
    from paper_2501_17267_gb300 import fragments
    Ls = [10, 20, 30, 40, 50]
    a, b = fragments.fit_inverse_L(Ls, [0.4 / L + 0.031 for L in Ls])
    assert a == pytest.approx(0.4) and b == pytest.approx(0.031)


def test_gallus_families_mix_the_stated_classes():
    from paper_2501_17267_gb300 import fragments
    assert fragments.gallus_class_prob("gallus_26", 0.8) == pytest.approx((0.2, 0.0, 0.8))
    assert fragments.gallus_class_prob("gallus_46", 0.8) == pytest.approx((0.0, 0.2, 0.8))
    assert fragments.gallus_class_prob("gallus_26", 1.0) == fragments.gallus_class_prob("gallus_46", 1.0)
    with pytest.raises(ValueError):
        fragments.gallus_class_prob("gallus_22", 0.5)


# --------------------------------------------------------------------------- tropical

def test_enumerated_minima_equal_plain_brute_force():
    """The Gray-code enumeration of or_fragment_min_energies against a direct sum over
    every state, on random fields and couplings (|J| <= 2, zeros included)."""
    import itertools
    rng = np.random.default_rng(0)
    for F in (1, 2, 5, 9, 11):
        for _ in range(4):
            h = rng.integers(-6, 7, F)
            J = np.zeros((F, F), dtype=np.int8)
            for k in range(F):
                for j in range(k + 1, F):
                    J[k, j] = J[j, k] = rng.integers(-2, 3)
            c = int(rng.integers(0, F))
            best = {1: None, -1: None}
            for st in itertools.product((1, -1), repeat=F):
                s = np.array(st)
                e = int(h @ s) + sum(int(J[k, j]) * s[k] * s[j] for k in range(F) for j in range(k + 1, F))
                if best[s[c]] is None or e < best[s[c]]:
                    best[s[c]] = e
            assert o.fragment_min_energies(h, J, c) == (best[1], best[-1])


def test_tropical_single_site_fragments_choose_plus_one():
    """l = 1: no bond inside a cube, both values have energy 0, the tie gives +1."""
    J3, _, _ = o.generate(4, 3, (1 / 3, 1 / 3, 1 / 3), True)
    spins, E = o.fragment_tropical(4, J3, 1)
    assert (spins == 1).all() and E == int(J3.astype(np.int64).sum())


def test_tropical_last_wave_spins_follow_their_field_exactly():
    """l = 3: a last-wave spin is its cube's only free spin, all six neighbours fixed
    inside the cube: it is +1 exactly when its local field is <= 0."""
    L = 6
    J3, _, egs = o.generate(L, 44, (0, 0, 1), True)
    spins, E = o.fragment_tropical(L, J3, 3)
    assert E == o.energy(L, J3, spins) and E >= egs
    for i in range(L ** 3):
        if _class(L, 3, i) == 26:
            h = o.local_field(L, J3, spins, i)
            assert spins[i] == (1 if h <= 0 else -1)


@pytest.mark.gpu
@pytest.mark.parametrize("L,l", [(6, 3), (4, 1)])
def test_tropical_fragments_match_oracle(sg, L, l):
    inst = sg.Instance.create(L, 44 if L == 6 else 3, (0, 0, 1), True)
    J3, _, egs = inst.get()
    res = sg.fragment_tropical_run(inst, l, spins="host")
    ospins, oE = o.fragment_tropical(L, J3, l)
    assert np.array_equal(res["spins"], ospins) and res["E"] == oE
