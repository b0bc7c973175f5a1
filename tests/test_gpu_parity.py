"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

All couplings and spins are integers and every accept decision is an integer
compare of the same Philox word against the same threshold, so the bar is
bit-exact: spins, energies, eps, PT permutations, swap counts and minimum
energies must be identical.
"""
import numpy as np
import pytest

from oracle import oracle as o
from paper_2501_17267_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2501_17267_gb300 import build
    build.build()
    from paper_2501_17267_gb300 import sg as mod
    return mod


def _sa_compare(sg, inst, J3, egs, R, S, b0, b1, geometric=False, seed=0, iid=0, reps=None):
    res = sg.sa_run(inst, R, S, b0, b1, "geometric" if geometric else "linear", seed, iid,
                    spins="host")
    reps = list(range(R)) if reps is None else reps
    ospins, oE = o.sa_run(inst.L, J3, seed, iid, S, b0, b1, geometric, reps=reps)
    assert np.array_equal(res["spins"][reps], ospins)
    assert np.array_equal(res["E"][reps], oE)
    for n, r in enumerate(reps):
        assert res["eps"][r] == o.epsilon(int(oE[n]), egs)
    return res


def test_sa_L4_R8_S1000_full(sg):
    """Workload: L=4, 8 replicas, 1000 sweeps, beta linear 0.1 -> 3.0, seed 0 -- all outputs."""
    w = wl.SA_L4
    inst = sg.Instance.create(w.L, w.instance_seed(0), w.class_prob, True)
    J3, _, egs = inst.get()
    res = _sa_compare(sg, inst, J3, egs, w.replicas, w.sweeps, w.beta0, w.beta1, seed=w.run_seed)
    assert (res["E"] >= egs).all()


def test_sa_L16_R1024_S1000_sampled(sg):
    """Workload: L=16, 1024 replicas, 1000 sweeps -- full run on the GPU, replicas sampled
    across bit positions of several 32-replica words and both ends checked against the oracle."""
    w = wl.SA_L16
    inst = sg.Instance.create(w.L, w.instance_seed(0), w.class_prob, True)
    J3, _, egs = inst.get()
    reps = [0, 1, 31, 32, 257, 514, 771, 1020, 1021, 1022, 1023]
    res = _sa_compare(sg, inst, J3, egs, w.replicas, w.sweeps, w.beta0, w.beta1, reps=reps)
    assert (res["E"] >= egs).all()
    # every replica's reported energy equals a recompute of its spins
    assert np.array_equal(sg.energy(inst, res["spins"]), res["E"])


@pytest.mark.parametrize("L,R,S,geo", [(2, 5, 40, False), (6, 13, 30, True), (10, 7, 25, False),
                                       (12, 4, 20, True), (8, 1, 60, False)])
def test_sa_ragged_shapes(sg, L, R, S, geo):
    """Ragged replica counts (R not a multiple of 32), L=2 multi-edges, several row blocks."""
    inst = sg.Instance.create(L, 1000 + L, wl.UNIFORM, True)
    J3, _, egs = inst.get()
    _sa_compare(sg, inst, J3, egs, R, S, 0.2, 2.5, geometric=geo, seed=77 + L, iid=L)


def test_sa_zero_sweeps_is_initial_state(sg):
    inst = sg.Instance.create(6, 5)
    J3, _, egs = inst.get()
    _sa_compare(sg, inst, J3, egs, 9, 0, 0.5, 1.0, seed=3)


@pytest.mark.parametrize("cls", [(1, 0, 0), (0, 1, 0), (0, 0, 1)])
def test_sa_single_class_instances(sg, cls):
    inst = sg.Instance.create(8, 42, cls, True)
    J3, _, egs = inst.get()
    _sa_compare(sg, inst, J3, egs, 8, 40, 0.3, 3.0, geometric=True, seed=9)


def test_sa_general_couplings(sg):
    """|J| in {0, 1, 2}: exercises the magnitude path of the kernel."""
    L = 6
    J3 = wl.random_couplings(21, L, jmax=2, allow_zero=True)
    inst = sg.Instance.from_couplings(L, J3, e_gs=-1)
    _sa_compare(sg, inst, J3, -1, 12, 30, 0.1, 2.0, seed=5)


def test_sa_batch_equals_separate(sg):
    insts = [sg.Instance.create(L, 70 + L) for L in (4, 6, 4)]
    params = [dict(replicas=8, sweeps=30, beta0=0.1, beta1=3.0, schedule="linear", seed=1,
                   instance_id=k) for k in range(3)]
    batch = sg.sa_run_batch(insts, params, spins="host")
    for inst, p, b in zip(insts, params, batch):
        single = sg.sa_run(inst, spins="host", **p)
        assert np.array_equal(single["spins"], b["spins"])
        assert np.array_equal(single["E"], b["E"])


def test_sa_device_spins_output(sg):
    import torch
    inst = sg.Instance.create(8, 3)
    a = sg.sa_run(inst, 12, 20, 0.2, 2.0, spins="host", seed=4)
    b = sg.sa_run(inst, 12, 20, 0.2, 2.0, spins="device", seed=4)
    assert isinstance(b["spins"], torch.Tensor)
    assert np.array_equal(a["spins"], b["spins"].cpu().numpy())


def _pt_compare(sg, inst, J3, egs, K, S, bmin, bmax, seed=0, iid=0, res=None):
    if res is None:
        res = sg.pt_run(inst, K, S, bmin, bmax, seed, iid, spins="host")
    ref = o.pt_run(inst.L, J3, seed, iid, K, S, bmin, bmax)
    assert np.array_equal(res["spins"], ref["spins"])
    assert np.array_equal(res["E"], ref["E"])
    assert np.array_equal(res["perm"], ref["perm"])
    assert np.array_equal(res["accepts"], ref["accepts"])
    assert res["minE"] == ref["minE"]
    assert res["min_eps"] == o.epsilon(ref["minE"], egs)
    return res


@pytest.mark.parametrize("L,K,S", [(4, 5, 60), (8, 8, 40), (6, 1, 20), (2, 3, 30), (10, 11, 15)])
def test_pt_small(sg, L, K, S):
    inst = sg.Instance.create(L, 500 + L, wl.UNIFORM, True)
    J3, _, egs = inst.get()
    _pt_compare(sg, inst, J3, egs, K, S, 0.2, 3.0, seed=11, iid=L)


def test_pt_equal_rungs(sg):
    inst = sg.Instance.create(4, 9)
    J3, _, egs = inst.get()
    res = _pt_compare(sg, inst, J3, egs, 4, 30, 1.3, 1.3, seed=2)
    assert list(res["accepts"]) == [15, 15, 15]


def test_pt_L64_K32_truncated(sg):
    """Workload geometry (L=64, 32 temperatures, beta 0.2 -> 3.0), first 3 sweeps, one
    instance, checked in full against the oracle."""
    w = wl.PT_L64
    inst = sg.Instance.create(w.L, w.instance_seed(0), w.class_prob, True)
    J3, _, egs = inst.get()
    _pt_compare(sg, inst, J3, egs, w.temps, 3, w.beta_min, w.beta_max, seed=w.run_seed, iid=0)


def test_pt_batch_equals_separate_and_oracle(sg):
    """16 instances at L=16 in one batch: identical to separate runs; two checked
    against the oracle."""
    insts = [sg.Instance.create(16, 2 ** 33 + k) for k in range(16)]
    params = [dict(temps=12, sweeps=8, beta_min=0.2, beta_max=3.0, seed=3, instance_id=k)
              for k in range(16)]
    batch = sg.pt_run_batch(insts, params, spins="host")
    for k in (0, 11):
        J3, _, egs = insts[k].get()
        _pt_compare(sg, insts[k], J3, egs, 12, 8, 0.2, 3.0, seed=3, iid=k, res=batch[k])
    for k in (5, 15):
        single = sg.pt_run(insts[k], spins="host", **params[k])
        assert np.array_equal(single["spins"], batch[k]["spins"])
        assert single["minE"] == batch[k]["minE"]


def test_energy_parity(sg):
    for L, jmax in [(2, 2), (4, 1), (6, 2), (10, 2)]:
        J3 = wl.random_couplings(L, L, jmax=jmax)
        inst = sg.Instance.from_couplings(L, J3)
        spins = wl.random_spins(L + 1, (7, L ** 3))
        E = sg.energy(inst, spins)
        assert [o.energy(L, J3, s) for s in spins] == list(E)


def test_energy_device_input_and_validation(sg):
    import torch
    inst = sg.Instance.create(6, 1)
    J3, tau, egs = inst.get()
    s = torch.from_numpy(np.stack([tau, -tau, np.ones_like(tau)])).cuda()
    E = sg.energy(inst, s)
    assert E[0] == egs and E[1] == egs  # global flip leaves E unchanged
    bad = np.zeros((1, 216), dtype=np.int8)
    with pytest.raises(sg.SGError) as e:
        sg.energy(inst, bad)
    assert e.value.code == sg.SG_EINVAL


@pytest.mark.parametrize("L,R", [(16, 32), (32, 64), (48, 8), (8, 31), (8, 33), (6, 65), (10, 100)])
def test_sa_word_shapes(sg, L, R):
    """Replica counts below, at and above whole 32-replica words (ragged last words)."""
    inst = sg.Instance.create(L, 40 + L)
    J3, _, egs = inst.get()
    reps = sorted({0, 5 % R, R // 2, R - 1})
    _sa_compare(sg, inst, J3, egs, R, 12, 0.1, 3.0, seed=6, reps=reps)


@pytest.mark.parametrize("L,K,S", [(8, 40, 6), (6, 64, 8), (10, 100, 4), (4, 33, 12)])
def test_pt_several_words(sg, L, K, S):
    """Temperature ladders spanning two to four spin words, ragged and whole."""
    inst = sg.Instance.create(L, 7400 + L)
    J3, _, egs = inst.get()
    _pt_compare(sg, inst, J3, egs, K, S, 0.2, 3.0, seed=13, iid=1)


def test_largest_lattice_side(sg):
    """L = 256, the largest side the kernels accept (16.8 M sites, 65536 rows of 128 sites
    per colour; each thread walks about a hundred rows): SA with one replica for two
    sweeps and PT with two temperatures for one sweep, every spin checked."""
    inst = sg.Instance.create(256, 9100)
    J3, _, egs = inst.get()
    _sa_compare(sg, inst, J3, egs, 1, 2, 0.1, 3.0, seed=3, iid=1)
    _pt_compare(sg, inst, J3, egs, 2, 1, 0.2, 3.0, seed=3, iid=1)
    with pytest.raises(sg.SGError):
        sg.Instance.create(258, 1)


def test_sa_rows_wider_than_a_block(sg):
    """L = 58 with 288 replicas: a colour half row holds 29 sites x 9 words, more than
    one 256-thread block row, so threads walk several sites per row (no prefetch)."""
    inst = sg.Instance.create(58, 7700)
    J3, _, egs = inst.get()
    _sa_compare(sg, inst, J3, egs, 288, 3, 0.1, 3.0, seed=23, iid=1, reps=[0, 31, 200, 287])


@pytest.mark.parametrize("L,R,S", [(16, 1024, 30), (8, 64, 40), (6, 40, 25), (2, 12, 20), (64, 32, 3),
                                   (10, 100, 17), (4, 33, 60)])
def test_sa_cluster_kernel_equals_row_kernel_and_oracle(sg, monkeypatch, L, R, S):
    """Small lattices run every sweep in one launch, a word of 32 replicas per thread-block
    cluster whose blocks hold z-slabs (neighbour slabs read through distributed shared
    memory): identical to the row kernel, and to the oracle on sampled replicas.  Slabs
    of one z-plane (L = 8, C = 8), six blocks (L = 6), L = 2 (both z neighbours in the
    other block), ragged last words."""
    inst = sg.Instance.create(L, 8000 + L)
    J3, _, egs = inst.get()
    monkeypatch.setenv("SG_SA_CLUSTER", "1")
    a = sg.sa_run(inst, R, S, 0.1, 3.0, "geometric", 37, 2, spins="host")
    monkeypatch.setenv("SG_SA_CLUSTER", "0")
    b = sg.sa_run(inst, R, S, 0.1, 3.0, "geometric", 37, 2, spins="host")
    assert np.array_equal(a["spins"], b["spins"]) and np.array_equal(a["E"], b["E"])
    reps = sorted({0, R // 3, R - 1})
    ospins, oE = o.sa_run(L, J3, 37, 2, S, 0.1, 3.0, True, reps=reps)
    assert np.array_equal(a["spins"][reps], ospins)
    assert np.array_equal(a["E"][reps], oE)


@pytest.mark.parametrize("L,R,S", [(16, 1024, 25), (8, 64, 30), (12, 100, 20), (32, 64, 6), (4, 8, 40)])
def test_sa_cluster_block_sizes_agree(sg, monkeypatch, L, R, S):
    """The single-run cluster kernel with 256 and with 512 threads a block (each with the
    largest cluster size that fits one wave; the library picks one of the two by the
    items a thread updates and the blocks an SM runs) and the row kernel give the same
    spins and energies."""
    inst = sg.Instance.create(L, 8100 + L)
    monkeypatch.setenv("SG_SA_CLUSTER", "1")
    runs = []
    for t in ("256", "512"):
        monkeypatch.setenv("SG_SA_CLUSTER_THREADS", t)
        runs.append(sg.sa_run(inst, R, S, 0.1, 3.0, "linear", 41, 3, spins="host"))
    monkeypatch.delenv("SG_SA_CLUSTER_THREADS")
    runs.append(sg.sa_run(inst, R, S, 0.1, 3.0, "linear", 41, 3, spins="host"))
    monkeypatch.setenv("SG_SA_CLUSTER", "0")
    runs.append(sg.sa_run(inst, R, S, 0.1, 3.0, "linear", 41, 3, spins="host"))
    for other in runs[1:]:
        assert np.array_equal(runs[0]["spins"], other["spins"]) and np.array_equal(runs[0]["E"], other["E"])


def test_runs_longer_than_one_graph_chunk(sg):
    """Runs of 16 or more sweeps go through CUDA graphs of up to 100 sweeps with the
    sweep index on the device: 230 and 251 sweeps end in a shorter last chunk."""
    inst = sg.Instance.create(4, 7600)
    J3, _, egs = inst.get()
    _pt_compare(sg, inst, J3, egs, 8, 230, 0.2, 3.0, seed=17, iid=5)
    inst6 = sg.Instance.create(6, 7601)
    J3b, _, egsb = inst6.get()
    _sa_compare(sg, inst6, J3b, egsb, 40, 251, 0.1, 3.0, geometric=True, seed=19, iid=2)


@pytest.mark.parametrize("L,K,S", [(32, 64, 16), (16, 128, 20)])
def test_pt_graph_runs_with_one_warp_per_row(sg, L, K, S):
    """Graph-captured runs (16 or more sweeps) of shapes where a warp is exactly one row
    of threads: two words per site at L = 32, four at L = 16."""
    inst = sg.Instance.create(L, 7800 + L)
    J3, _, egs = inst.get()
    _pt_compare(sg, inst, J3, egs, K, S, 0.2, 3.0, seed=29, iid=6)


def test_sa_graph_run_with_one_warp_per_row(sg):
    inst = sg.Instance.create(32, 7900)
    J3, _, egs = inst.get()
    _sa_compare(sg, inst, J3, egs, 64, 17, 0.1, 3.0, seed=31, iid=3, reps=[0, 33, 63])


def test_pt_general_couplings(sg):
    """Couplings with |J| = 2 and zeros take the replica-by-replica path, energies included."""
    L = 6
    J3 = wl.random_couplings(21, L, jmax=2)
    inst = sg.Instance.from_couplings(L, J3)
    res = sg.pt_run(inst, 12, 10, 0.2, 1.5, seed=7, instance_id=2, spins="host")
    ref = o.pt_run(L, J3, 7, 2, 12, 10, 0.2, 1.5)
    assert np.array_equal(res["spins"], ref["spins"])
    assert np.array_equal(res["E"], ref["E"])
    assert np.array_equal(res["perm"], ref["perm"])
    assert np.array_equal(res["accepts"], ref["accepts"])
    assert res["minE"] == ref["minE"]


def test_pt_long_thread_runs_fold_energy_counters(sg, monkeypatch):
    """Every thread walks 400 rows (more sites than its energy counters hold before a
    fold), so the colour-1 energy sums fold mid-run and at the end."""
    monkeypatch.setenv("SG_ROWS_RPT", "400")
    inst = sg.Instance.create(32, 7500)
    J3, _, egs = inst.get()
    _pt_compare(sg, inst, J3, egs, 32, 3, 0.2, 3.0, seed=5, iid=4)


# --------------------------------------------------------------------------- uneven batches

def _uneven_batch(sg, seed=0):
    shapes = [(4, 8, 30), (6, 64, 12), (8, 16, 25), (12, 8, 7), (6, 8, 40), (16, 12, 5), (10, 4, 9)]
    insts, params = [], []
    for k, (L, R, S) in enumerate(shapes):
        insts.append(sg.Instance.create(L, 3 * 2 ** 32 + 100 * seed + k))
        params.append(dict(replicas=R, sweeps=S, beta0=0.1, beta1=3.0,
                           schedule="geometric" if k % 2 else "linear", seed=seed + 5, instance_id=k))
    return insts, params


def test_uneven_batch_equals_separate_runs_and_oracle(sg, monkeypatch, tmp_path):
    """Instances of several sizes in one persistent launch: byte-identical to separate
    runs; two instances also against the oracle."""
    monkeypatch.setenv("SG_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    insts, params = _uneven_batch(sg)
    batch = sg.sa_run_batch(insts, params, spins="host")
    for inst, p, b in zip(insts, params, batch):
        single = sg.sa_run(inst, spins="host", **p)
        assert np.array_equal(single["spins"], b["spins"])
        assert np.array_equal(single["E"], b["E"])
        assert np.array_equal(single["eps"], b["eps"])
    for k in (1, 3):
        J3, _, egs = insts[k].get()
        p = params[k]
        reps = [0, p["replicas"] - 1]
        ospins, oE = o.sa_run(insts[k].L, J3, p["seed"], p["instance_id"], p["sweeps"], p["beta0"],
                              p["beta1"], p["schedule"] == "geometric", reps=reps)
        assert np.array_equal(batch[k]["spins"][reps], ospins)
        assert np.array_equal(batch[k]["E"][reps], oE)


def test_batch_autotuner_records_and_reuses_choice(sg, monkeypatch, tmp_path):
    """With several plane widths possible the autotuner measures them, stores its choice,
    and a second run with the same mix reuses it; results do not depend on it."""
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("SG_AUTOTUNE_CACHE", str(cache))
    insts = [sg.Instance.create(L, 500 + L) for L in (8, 12, 16)]
    params = [dict(replicas=128, sweeps=10, beta0=0.1, beta1=3.0, schedule="linear", seed=1,
                   instance_id=k) for k in range(3)]  # four words: plane widths 4, 2, 1
    first = sg.sa_run_batch(insts, params, spins="host")
    assert cache.exists()
    text = cache.read_text()
    assert "8x128x10x1" in text and "16x128x10x1" in text
    second = sg.sa_run_batch(insts, params, spins="host")
    assert cache.read_text() == text
    for a, b in zip(first, second):
        assert np.array_equal(a["spins"], b["spins"])


@pytest.mark.parametrize("wg,graph", [("1", "1"), ("2", "0"), ("4", "1"), ("0", "1"), ("0", "0")])
def test_uneven_batch_any_plane_width(sg, monkeypatch, wg, graph):
    """Every words-per-plane choice, the thread-block-cluster form ("0": one-word planes,
    each split into z-slabs across a cluster; here C = 2 for L = 4, 8, 6) and graph
    capture on or off give the same bytes (R = 100 spans four words, the last ragged)."""
    insts = [sg.Instance.create(L, 77 + L) for L in (4, 8, 6)]
    params = [dict(replicas=100, sweeps=S, beta0=0.2, beta1=2.5, schedule="linear", seed=3,
                   instance_id=k) for k, S in enumerate((20, 9, 14))]
    monkeypatch.setenv("SG_BATCH_PLANES", "0")
    ref = sg.sa_run_batch(insts, params, spins="host")
    monkeypatch.setenv("SG_BATCH_PLANES", "1")
    monkeypatch.setenv("SG_BATCH_WG", wg)
    monkeypatch.setenv("SG_BATCH_GRAPH", graph)
    got = sg.sa_run_batch(insts, params, spins="device")
    for a, b in zip(ref, got):
        assert np.array_equal(a["spins"], b["spins"].cpu().numpy())
        assert np.array_equal(a["E"], b["E"])


# --------------------------------------------------------------------------- wide shapes

# Shapes from one word of replicas on a large lattice to eight words on a small one.
@pytest.mark.parametrize("L,K,S", [(64, 16, 2), (32, 64, 2), (16, 128, 3), (8, 256, 4)])
def test_pt_wide_shapes_match_oracle(sg, L, K, S):
    inst = sg.Instance.create(L, 7000 + L)
    J3, _, egs = inst.get()
    _pt_compare(sg, inst, J3, egs, K, S, 0.2, 3.0, seed=21, iid=3)


@pytest.mark.parametrize("L,R,S", [(64, 32, 2), (32, 64, 3), (16, 128, 4), (8, 256, 5), (2, 1024, 6)])
def test_sa_wide_shapes_match_oracle(sg, L, R, S):
    inst = sg.Instance.create(L, 7100 + L)
    J3, _, egs = inst.get()
    _sa_compare(sg, inst, J3, egs, R, S, 0.1, 3.0, seed=5, iid=1)


@pytest.mark.parametrize("L,R,S", [(16, 256, 20), (8, 64, 30), (24, 16, 10), (2, 12, 25), (2, 5, 40)])
def test_planes_in_shared_memory_equal_global(sg, monkeypatch, L, R, S):
    """Small lattices run with every plane held in shared memory for the whole run; the
    same run with planes in global memory, the row kernels and the oracle agree."""
    inst = sg.Instance.create(L, 7300 + L)
    J3, _, egs = inst.get()
    monkeypatch.setenv("SG_BATCH_PLANES", "1")
    smem = sg.sa_run(inst, R, S, 0.1, 3.0, seed=4, spins="host")
    monkeypatch.setenv("SG_PLANES_SMEM_KB", "0")
    glob = sg.sa_run(inst, R, S, 0.1, 3.0, seed=4, spins="host")
    monkeypatch.setenv("SG_BATCH_PLANES", "0")
    rows = sg.sa_run(inst, R, S, 0.1, 3.0, seed=4, spins="host")
    for other in (glob, rows):
        assert np.array_equal(smem["spins"], other["spins"]) and np.array_equal(smem["E"], other["E"])
    _sa_compare(sg, inst, J3, egs, R, S, 0.1, 3.0, seed=4, reps=[0, R // 2, R - 1])


# --------------------------------------------------------------------------- PT on clusters

@pytest.mark.parametrize("L,K,S,I", [(2, 3, 10, 1), (4, 5, 30, 2), (6, 32, 7, 1), (8, 8, 20, 1),
                                     (12, 17, 10, 1), (16, 32, 15, 3), (64, 32, 5, 2), (4, 1, 12, 2),
                                     (8, 2, 16, 3)])
def test_pt_cluster_kernel_equals_row_kernels_and_oracle(sg, monkeypatch, L, K, S, I):
    """PT with every sweep of a chunk in one launch, one thread-block cluster per instance
    holding the lattice in shared memory (exchange decided in every block from the
    cluster's energy sums): identical to the row kernels and to the oracle.  One z-plane
    per block (L = 2, 6), uneven half rows (L = 12), several instances, ragged K, one rung
    (no exchange pair) and two."""
    insts = [sg.Instance.create(L, 8800 + 10 * L + k) for k in range(I)]
    params = [dict(temps=K, sweeps=S, beta_min=0.2, beta_max=3.0, seed=41, instance_id=k) for k in range(I)]
    monkeypatch.setenv("SG_PT_CLUSTER", "1")
    a = sg.pt_run_batch(insts, params, spins="host")
    monkeypatch.setenv("SG_PT_CLUSTER", "0")
    b = sg.pt_run_batch(insts, params, spins="host")
    for x, y in zip(a, b):
        for k in ("spins", "E", "perm", "accepts"):
            assert np.array_equal(x[k], y[k]), k
        assert x["minE"] == y["minE"]
    J3, _, egs = insts[-1].get()
    _pt_compare(sg, insts[-1], J3, egs, K, S, 0.2, 3.0, seed=41, iid=I - 1, res=a[-1])


def test_pt_cluster_kernel_chunks(sg, monkeypatch):
    """A run longer than one cluster launch (chunks of 2000 sweeps, the state carried in
    device memory between them) equals the row kernels."""
    inst = sg.Instance.create(4, 8899)
    monkeypatch.setenv("SG_PT_CLUSTER", "1")
    a = sg.pt_run(inst, 6, 4100, 0.2, 3.0, seed=5, spins="host")
    monkeypatch.setenv("SG_PT_CLUSTER", "0")
    b = sg.pt_run(inst, 6, 4100, 0.2, 3.0, seed=5, spins="host")
    for k in ("spins", "E", "perm", "accepts"):
        assert np.array_equal(a[k], b[k]), k
    assert a["minE"] == b["minE"]


@pytest.mark.parametrize("L,I,K,S", [(64, 16, 32, 30), (64, 17, 17, 20), (48, 16, 32, 25), (64, 16, 32, 2100),
                                     (64, 16, 1, 20)])
def test_pt_split_between_clusters_and_rows_equals_row_kernels(sg, monkeypatch, L, I, K, S):
    """More instances than this GPU keeps clusters of 8 resident at once: the first ones
    run on clusters while the row kernels run the others beside them on a second stream
    (every per-instance array of the second part offset by the first part's size).
    Identical to the row kernels alone; the launch statistics show both kinds ran.  Slabs
    of 8 planes (L = 64) and 6 (L = 48), a ragged K, and a run of two cluster launches
    (chunks of 2000 sweeps) beside 21 row-kernel graphs."""
    insts = [sg.Instance.create(L, 9100 + 100 * L + k) for k in range(I)]
    params = [dict(temps=K, sweeps=S, beta_min=0.2, beta_max=3.0, seed=47, instance_id=k) for k in range(I)]
    for knob in ("SG_PT_CLUSTER", "SG_PT_HYBRID", "SG_PT_COOP"):
        monkeypatch.delenv(knob, raising=False)
    sg.stats_read(reset=True)
    a = sg.pt_run_batch(insts, params, spins="host")
    st = sg.stats_read(reset=True)
    on_clusters = st["sweep_chunk"]["units"] / (I * K * L ** 3 * S)
    assert st["sweep"]["launches"] > 0 and 0.5 < on_clusters < 1.0, st
    monkeypatch.setenv("SG_PT_CLUSTER", "0")
    b = sg.pt_run_batch(insts, params, spins="host")
    for x, y in zip(a, b):
        for k in ("spins", "E", "perm", "accepts"):
            assert np.array_equal(x[k], y[k]), k
        assert x["minE"] == y["minE"]


# --------------------------------------------------------------------------- PT on one cooperative grid

@pytest.mark.parametrize("L,K,S,I", [(8, 8, 20, 1), (16, 32, 12, 3), (32, 17, 10, 4), (48, 32, 4, 8),
                                     (64, 32, 3, 1), (64, 32, 5, 16)])
def test_pt_coop_kernel_equals_row_kernels_and_oracle(sg, monkeypatch, L, K, S, I):
    """PT with every sweep of a chunk in one cooperative launch, each instance's rows split
    into row blocks held in shared memory with one-plane halos exchanged through device
    memory (flags between neighbouring blocks, a per-instance barrier before the
    exchange): identical to the row kernels and to the oracle.  One block of 8 rows per
    plane pair (L = 8), ragged K, the 16 x L = 64 batch on all SMs (9 or 10 blocks per
    instance), one instance on 64 blocks."""
    insts = [sg.Instance.create(L, 8900 + 10 * L + k) for k in range(I)]
    params = [dict(temps=K, sweeps=S, beta_min=0.2, beta_max=3.0, seed=43, instance_id=k) for k in range(I)]
    monkeypatch.setenv("SG_PT_COOP", "1")
    a = sg.pt_run_batch(insts, params, spins="host")
    monkeypatch.setenv("SG_PT_COOP", "0")
    monkeypatch.setenv("SG_PT_CLUSTER", "0")
    b = sg.pt_run_batch(insts, params, spins="host")
    for x, y in zip(a, b):
        for k in ("spins", "E", "perm", "accepts"):
            assert np.array_equal(x[k], y[k]), k
        assert x["minE"] == y["minE"]
    J3, _, egs = insts[-1].get()
    _pt_compare(sg, insts[-1], J3, egs, K, S, 0.2, 3.0, seed=43, iid=I - 1, res=a[-1])


def test_pt_coop_kernel_chunks(sg, monkeypatch):
    """A run longer than one cooperative launch (chunks of 2000 sweeps) equals the row kernels."""
    inst = sg.Instance.create(8, 8998)
    monkeypatch.setenv("SG_PT_COOP", "1")
    a = sg.pt_run(inst, 6, 4100, 0.2, 3.0, seed=5, spins="host")
    monkeypatch.setenv("SG_PT_COOP", "0")
    monkeypatch.setenv("SG_PT_CLUSTER", "0")
    b = sg.pt_run(inst, 6, 4100, 0.2, 3.0, seed=5, spins="host")
    for k in ("spins", "E", "perm", "accepts"):
        assert np.array_equal(a[k], b[k]), k
    assert a["minE"] == b["minE"]


def test_pt_coop_wait_that_gives_up_reports_timeout(sg, monkeypatch):
    """Every wait of the cooperative kernel is bounded: with the poll limit set to 0 a wait
    gives up at once, the blocks stop, and the call returns SG_ETIMEOUT; the context stays
    usable and the next run (normal limit) is correct."""
    insts = [sg.Instance.create(64, 8990 + k) for k in range(16)]
    params = [dict(temps=32, sweeps=20, beta_min=0.2, beta_max=3.0, seed=3, instance_id=k) for k in range(16)]
    monkeypatch.setenv("SG_PT_COOP", "1")
    monkeypatch.setenv("SG_WAIT_LIMIT", "0")
    with pytest.raises(sg.SGError) as e:
        sg.pt_run_batch(insts, params)
    assert e.value.code == sg.SG_ETIMEOUT
    monkeypatch.delenv("SG_WAIT_LIMIT")
    a = sg.pt_run_batch(insts, params)
    monkeypatch.setenv("SG_PT_COOP", "0")
    b = sg.pt_run_batch(insts, params)
    for x, y in zip(a, b):
        assert np.array_equal(x["E"], y["E"]) and x["minE"] == y["minE"]
