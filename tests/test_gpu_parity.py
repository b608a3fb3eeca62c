"""GPU path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Bars: histograms bit-exact; MC trial coordinates bit-exact and dU within 1e-5 of the
condition scale C = sum |u(r') - u(r)| (FP32 against FP64; decisions may differ only
inside that band and are then replayed with the GPU's choice, after which final
coordinates are bit-exact); g(r) to FP32 rounding; S(Q) within 1e-4 barn.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1904_08756_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1904_08756_gb300 import epsr  # noqa: E402

DEV = torch.device("cuda:0")
DU_REL = 1e-5          # of the condition scale C
DU_ABS = 1e-4          # kJ/mol floor for moves whose C is tiny


def gpu_hist(box: epsr.Box, n_repeat: int = 1):
    H = torch.zeros(box.hist_len, dtype=torch.int64, device=DEV)
    for _ in range(n_repeat):
        box.epsr_partial_gr(H)
    torch.cuda.synchronize()
    return H.cpu().numpy().astype(np.uint64)


# --------------------------------------------------------------------------------------
# pair histograms: bit-exact
# --------------------------------------------------------------------------------------

def test_histogram_bit_exact_small_water(small_water):
    box = epsr.Box(small_water)
    H = gpu_hist(box).reshape(3, small_water.n_bins)
    ref = oracle.Box(small_water).histogram()
    assert np.array_equal(H, ref)


@pytest.mark.parametrize("n,L,types", [(1, 5.0, 1), (2, 5.0, 2), (1023, 14.0, 2),
                                       (1025, 14.0, 3), (2500, 19.0, 2), (3073, 20.0, 4)])
def test_histogram_bit_exact_ragged_tiles(n, L, types):
    s = synth.uniform_gas(n, L, seed=n, n_types=types)
    s.bin_p, s.bin_q, s.n_bins = 1, 25, 200      # 0.04 A bins to 8 A (beyond L/2 for some)
    H = gpu_hist(epsr.Box(s)).reshape(-1, 200)
    assert np.array_equal(H, oracle.Box(s).histogram(threads=8))


def test_histogram_lattice_closed_form():
    S = 1 << 20
    s = synth.lattice_box(8, S, n_bins=80, bin_p=1, bin_q=20)
    H = gpu_hist(epsr.Box(s))
    assert np.array_equal(H, oracle.Box(s).histogram()[0])


def test_histogram_accumulates_and_translation_invariant(small_water):
    box = epsr.Box(small_water)
    H2 = gpu_hist(box, n_repeat=2)
    shift = np.array([7777777, 1, small_water.L_fx - 3])
    s2 = synth.System(**{**small_water.__dict__,
                         "xyz": ((small_water.xyz.astype(np.int64) + shift) % small_water.L_fx)
                         .astype(np.int32)})
    H1 = gpu_hist(epsr.Box(s2))
    assert np.array_equal(H2, 2 * H1)


def test_histogram_tile_ranges_sum_to_full():
    s = synth.water_box(1100, seed=41, L_A=32.0)
    box = epsr.Box(s)
    nt = box.epsr_partial_gr_tiles()
    H = torch.zeros(box.hist_len, dtype=torch.int64, device=DEV)
    cut = nt // 2
    box.epsr_partial_gr_range(0, cut, H)
    box.epsr_partial_gr_range(cut, nt, H)
    torch.cuda.synchronize()
    assert np.array_equal(H.cpu().numpy().astype(np.uint64), gpu_hist(epsr.Box(s)))


@pytest.mark.parametrize("which", ["water", "silica"])
def test_histogram_bit_exact_paper_size(which):
    s = synth.paper_water() if which == "water" else synth.paper_silica()
    box = epsr.Box(s)
    H = gpu_hist(box).reshape(3, s.n_bins)
    ref = oracle.Box(s).histogram(threads=0)
    assert np.array_equal(H, ref)
    Hc = torch.zeros(box.hist_len, dtype=torch.int64, device=DEV)
    box.epsr_partial_gr_cells(Hc)
    torch.cuda.synchronize()
    assert np.array_equal(Hc.cpu().numpy().astype(np.uint64).reshape(3, s.n_bins), ref)


@pytest.mark.parametrize("n,L,cut_bins", [(3000, 44.8, 333), (2000, 31.0, 200), (5000, 40.0, 100)])
def test_cell_list_histogram_bit_exact(n, L, cut_bins):
    """Cell lists of 4, 3 and 9 cells per side (water; a gas with 0.04 A bins to 8 A; a gas
    with a 4 A range): the same integer counts as the oracle."""
    if n == 3000:
        s = synth.water_box(1000, seed=71, L_A=L)
    else:
        s = synth.uniform_gas(n, L, seed=n, n_types=3)
        s.bin_p, s.bin_q, s.n_bins = 1, 25, cut_bins
    box = epsr.Box(s)
    H = torch.zeros(box.hist_len, dtype=torch.int64, device=DEV)
    box.epsr_partial_gr_cells(H)
    torch.cuda.synchronize()
    ref = oracle.Box(s).histogram(threads=8)
    assert np.array_equal(H.cpu().numpy().astype(np.uint64).reshape(ref.shape), ref)


def test_cell_list_histogram_batch_with_small_boxes():
    """A handle mixing boxes with cell lists and boxes too small for three cells (counted
    by the all-pairs kernel): identical to epsr_partial_gr on the whole handle."""
    systems = [synth.water_box(300, seed=72, L_A=20.8), synth.water_box(3000, seed=73),
               synth.silica_box(600, seed=74), synth.silica_box(4000, seed=75)]
    box = epsr.Box(systems)
    H1 = gpu_hist(box)
    H2 = torch.zeros(box.hist_len, dtype=torch.int64, device=DEV)
    box.epsr_partial_gr_cells(H2)
    torch.cuda.synchronize()
    assert np.array_equal(H1, H2.cpu().numpy().astype(np.uint64))


def test_g_normalisation(small_water):
    box = epsr.Box(small_water)
    H = torch.zeros(box.hist_len, dtype=torch.int64, device=DEV)
    g = torch.zeros(box.hist_len, dtype=torch.float32, device=DEV)
    box.epsr_partial_gr(H, g, 1)
    box.epsr_partial_gr(H, g, 2)
    torch.cuda.synchronize()
    ob = oracle.Box(small_water)
    ref = ob.normalize_g(H.cpu().numpy().astype(np.uint64).reshape(3, -1), 2)
    assert np.allclose(g.cpu().numpy().reshape(3, -1), ref, rtol=2e-7, atol=0)


# --------------------------------------------------------------------------------------
# energies and MC replay
# --------------------------------------------------------------------------------------

def test_total_energy(small_water):
    box = epsr.Box(small_water)
    U = box.epsr_box_total_energy()[0]
    ref = oracle.Box(small_water).total_energy()
    assert abs(U - ref) <= 1e-5 * abs(ref)


def run_logged(box: epsr.Box, n_moves: int, seed: int, move0: int = 0):
    log = torch.zeros((box.n_boxes * n_moves * 128,), dtype=torch.uint8, device=DEV)
    stats = box.epsr_mc_sweep(n_moves, seed, move0, log=log)
    torch.cuda.synchronize()
    return stats, log.cpu().numpy().view(epsr.MOVE_LOG_DTYPE).reshape(box.n_boxes, n_moves)


def replay(system, start_xyz, log, seed, move0=0, box_index=0, check_every=1, ep=None):
    """Replay a GPU move log on the oracle. Returns (n_checked, max_err_over_C, flips)."""
    ob = oracle.Box(system, xyz=start_xyz, ep=ep)
    kT = oracle.gas_constant() * system.temperature
    worst, flips, checked = 0.0, 0, 0
    for t, e in enumerate(log):
        mol, trial, u = ob.propose(seed, move0 + t, box_index)
        m = len(trial)
        assert e["mol"] == mol and e["n_atoms"] == m, (t, e["mol"], mol)
        assert np.array_equal(e["trial"][:m], trial), (t, e["trial"][:m], trial)
        assert e["u_acc"] == u
        if t % check_every == 0:
            dU, C = ob.delta_u(mol, trial)
            err = abs(float(e["dU"]) - dU)
            tol = DU_REL * C + DU_ABS
            assert err <= tol, (t, float(e["dU"]), dU, C)
            worst = max(worst, err / max(C, 1e-30))
            checked += 1
            ref_acc = oracle.accept(dU, u, system.temperature)
            if bool(e["accepted"]) != ref_acc:
                flips += 1
                assert abs(dU + kT * math.log(u)) <= tol, (t, dU, u)
        if e["accepted"]:
            ob.apply(mol, trial)
    return ob, checked, worst, flips


@pytest.mark.parametrize("batch", [32, 16, 5, 1])
def test_mc_replay_small_water(small_water, batch):
    box = epsr.Box(small_water)
    box.epsr_mc_set_batch(batch)
    stats, log = run_logged(box, 2000, seed=12345)
    att, acc, nonfin, sdu = stats[0]
    assert att == 2000 and nonfin == 0 and 0 < acc < 2000
    ob, checked, worst, flips = replay(small_water, small_water.xyz, log[0], 12345)
    assert np.array_equal(box.epsr_box_get_coords(), ob.xyz)
    assert flips <= 2
    assert abs(sdu - float(log[0]["dU"][log[0]["accepted"] == 1].astype(np.float64).sum())) < 1e-6 * max(1, abs(sdu))


@pytest.mark.parametrize("batch", [64, 48])
def test_mc_replay_small_water_wide_batches(small_water, batch):
    """Batches above 32 moves (16 CTAs for the 900-atom box): the same sequential chain."""
    box = epsr.Box(small_water)
    box.epsr_mc_set_ctas(16)
    box.epsr_mc_set_batch(batch)
    stats, log = run_logged(box, 2000, seed=777)
    att, acc, nonfin, sdu = stats[0]
    assert att == 2000 and nonfin == 0 and 0 < acc < 2000
    ob, checked, worst, flips = replay(small_water, small_water.xyz, log[0], 777)
    assert np.array_equal(box.epsr_box_get_coords(), ob.xyz)
    assert flips <= 2


@pytest.mark.parametrize("batch", [0, 16, 1])
def test_mc_replay_flexible_water(batch):
    """Flexible water (Sec. 3.1): molecule translations, rotations and single-atom moves,
    springs between every two atoms of a molecule; trial coordinates bit-exact, dU within
    tolerance (the spring change is FP64 on both sides), final coordinates bit-exact."""
    s = synth.flexible_water_box(300, seed=5, L_A=20.8)
    box = epsr.Box(s)
    box.epsr_mc_set_batch(batch)
    U0 = box.epsr_box_total_energy()[0]
    stats, log = run_logged(box, 2000, seed=4242)
    att, acc, nonfin, sdu = stats[0]
    assert att == 2000 and nonfin == 0 and 0 < acc < 2000
    ob, checked, worst, flips = replay(s, s.xyz, log[0], 4242)
    assert np.array_equal(box.epsr_box_get_coords(), ob.xyz)
    assert flips <= 2
    U1 = box.epsr_box_total_energy()[0]
    assert abs(U1 - ob.total_energy()) <= 1e-5 * abs(U1) + 1e-3
    assert abs((U1 - U0) - sdu) <= 1e-4 * abs(U0) + 1.0


def test_mc_replay_flexible_paper_size_sampled():
    s = synth.flexible_water_box(33333, seed=6)
    box = epsr.Box(s)
    stats, log = run_logged(box, 3000, seed=77)
    ob, checked, worst, flips = replay(s, s.xyz, log[0], 77, check_every=30)
    assert np.array_equal(box.epsr_box_get_coords(), ob.xyz)


def test_mc_replay_multi_cta_water():
    """A box split over several CTAs exercises the grid barrier and the gathered sums."""
    s = synth.water_box(3000, seed=42, density=0.1)
    box = epsr.Box(s)
    box.epsr_mc_set_ctas(12)
    stats, log = run_logged(box, 3000, seed=777, move0=100)
    ob, checked, worst, flips = replay(s, s.xyz, log[0], 777, move0=100, check_every=3)
    assert np.array_equal(box.epsr_box_get_coords(), ob.xyz)


def test_mc_replay_silica_atom_moves_with_ep():
    s = synth.silica_box(700, seed=43)
    rng = np.random.default_rng(1)
    ep = (rng.normal(size=(3, s.n_bins)) * 0.3).astype(np.float32)
    box = epsr.Box(s)
    box.epsr_box_set_ep(0, ep)
    box.epsr_mc_set_ctas(4)
    stats, log = run_logged(box, 3000, seed=99)
    ob, checked, worst, flips = replay(s, s.xyz, log[0], 99, ep=ep.astype(np.float64))
    assert np.array_equal(box.epsr_box_get_coords(), ob.xyz)


@pytest.mark.parametrize("cells,check_every", [(None, 1), ((0, 256), 40), ((0, 4), 40), ((0, 0), 40)],
                         ids=["default-every-move", "margin0", "escapee-overflow", "no-cells"])
def test_mc_replay_paper_water_sampled(cells, check_every):
    """99,999-atom water on the full grid of CTAs: trial coordinates of every move
    bit-exact, dU (and the decision) checked against the oracle on every move for the
    default configuration and on every 40th for the cell-query variants, final coordinates
    bit-exact. With a zero cell margin every partner that leaves its cell becomes an escapee;
    a list of 4 overflows and the CTAs fall back to full scans; capacity 0 turns cell queries
    off."""
    s = synth.paper_water()
    box = epsr.Box(s)
    if cells is not None:
        box.epsr_mc_set_cells(*cells)
    n = 4000
    stats, log = run_logged(box, n, seed=2024)
    ob, checked, worst, flips = replay(s, s.xyz, log[0], 2024, check_every=check_every)
    assert checked == n // check_every
    assert flips <= 2
    assert np.array_equal(box.epsr_box_get_coords(), ob.xyz)


def test_mc_replay_paper_silica_every_move():
    """The 99,000-atom silica box as benchmarked (default CTAs, 64 moves per barrier,
    single-atom moves, Lennard-Jones on every type pair) with a random empirical potential on
    its 600 bins: dU and the decision of every one of 3,000 moves against the FP64 oracle,
    final coordinates bit-exact."""
    s = synth.paper_silica()
    rng = np.random.default_rng(21)
    ep = (rng.normal(size=(3, s.n_bins)) * 0.3).astype(np.float32)
    box = epsr.Box(s)
    box.epsr_box_set_ep(0, ep)
    n = 3000
    stats, log = run_logged(box, n, seed=606)
    att, acc, nonfin, sdu = stats[0]
    assert att == n and nonfin == 0 and 0 < acc < n
    ob, checked, worst, flips = replay(s, s.xyz, log[0], 606, ep=ep.astype(np.float64))
    assert checked == n and flips <= 2
    assert np.array_equal(box.epsr_box_get_coords(), ob.xyz)


@pytest.mark.parametrize("which", ["water", "silica"])
def test_mc_replay_lj_cutoff_paper_size(which):
    """The cutoff form of dU (Lennard-Jones truncated at 9 A, every row answered by cell
    queries) on the paper-scale boxes: trial coordinates, dU and the decision of every one of
    2,000 moves against the oracle's truncated pair energy, final coordinates bit-exact."""
    s = synth.paper_water() if which == "water" else synth.paper_silica()
    s.r_lj = 9.0
    box = epsr.Box(s)
    n = 2000
    stats, log = run_logged(box, n, seed=515)
    att, acc, nonfin, sdu = stats[0]
    assert att == n and nonfin == 0 and 0 < acc < n
    ob, checked, worst, flips = replay(s, s.xyz, log[0], 515)
    assert checked == n and flips <= 2
    assert np.array_equal(box.epsr_box_get_coords(), ob.xyz)


@pytest.mark.parametrize("batch", [0, 1])
def test_mc_replay_lj_cutoff_small_water(batch):
    """900-atom water with LJ cut at 6 A (cutoff below half the box, so partners on both
    sides): replay parity of 2,000 moves and the total energy against the oracle."""
    s = synth.water_box(300, seed=16, L_A=20.8)
    s.r_lj = 6.0
    box = epsr.Box(s)
    box.epsr_mc_set_batch(batch)
    U0 = box.epsr_box_total_energy()[0]
    assert abs(U0 - oracle.Box(s).total_energy()) <= 1e-5 * abs(U0)
    stats, log = run_logged(box, 2000, seed=616)
    ob, checked, worst, flips = replay(s, s.xyz, log[0], 616)
    assert flips <= 2
    assert np.array_equal(box.epsr_box_get_coords(), ob.xyz)
    U1 = box.epsr_box_total_energy()[0]
    assert abs(U1 - ob.total_energy()) <= 1e-5 * abs(U1)
    assert abs((U1 - U0) - stats[0][3]) <= 1e-4 * abs(U0) + 1.0


def test_mc_replay_mixed_cutoff_batch_with_ep():
    """One handle mixing boxes with and without the LJ cutoff (the cut instantiation reads each
    box's setting) and an empirical potential on a cut box: replay parity of every box."""
    a = synth.water_box(400, seed=24, L_A=23.0)
    a.r_lj = 6.5
    b = synth.silica_box(500, seed=25)
    c = synth.silica_box(700, seed=26)
    c.r_lj = 5.0
    systems = [a, b, c]
    rng = np.random.default_rng(27)
    ep = (rng.normal(size=(3, c.n_bins)) * 0.3).astype(np.float32)
    box = epsr.Box(systems)
    box.epsr_box_set_ep(2, ep)
    stats, log = run_logged(box, 1500, seed=28)
    xyz = box.epsr_box_get_coords()
    for k, s in enumerate(systems):
        _, a0 = box.epsr_box_offsets(k)
        ob, checked, _, flips = replay(s, s.xyz, log[k], 28, box_index=k,
                                       ep=ep.astype(np.float64) if k == 2 else None)
        assert flips <= 2
        assert np.array_equal(xyz[a0:a0 + s.n_atoms], ob.xyz), k


def test_mc_replay_global_memory_slices():
    """Slices too large for shared memory (8 CTAs for 99,999 atoms) run the global-memory
    variant of the sweep: same bit-exact trial coordinates and final state."""
    s = synth.paper_water()
    box = epsr.Box(s)
    box.epsr_mc_set_ctas(8)
    stats, log = run_logged(box, 1500, seed=31)
    ob, checked, worst, flips = replay(s, s.xyz, log[0], 31, check_every=30)
    assert np.array_equal(box.epsr_box_get_coords(), ob.xyz)


def test_mc_replay_lattice_1_5m_atoms():
    """1.5 million atoms (lattice water) on the full grid: global-memory slices, cell
    queries over 8^3 cells of 59 A."""
    s = synth.water_lattice(500_000, seed=12)
    box = epsr.Box(s)
    stats, log = run_logged(box, 1000, seed=32)
    ob, checked, worst, flips = replay(s, s.xyz, log[0], 32, check_every=50)
    assert np.array_equal(box.epsr_box_get_coords(), ob.xyz)


def test_mc_batched_replicas_replay():
    systems = [synth.water_box(400, seed=61), synth.silica_box(500, seed=62),
               synth.water_box(900, seed=63, n_bins=600, bin_p=2, bin_q=100)]
    box = epsr.Box(systems)
    stats, log = run_logged(box, 1500, seed=5)
    xyz = box.epsr_box_get_coords()
    for b, s in enumerate(systems):
        _, a0 = box.epsr_box_offsets(b)
        ob, _, _, _ = replay(s, s.xyz, log[b], 5, box_index=b, check_every=5)
        assert np.array_equal(xyz[a0:a0 + s.n_atoms], ob.xyz)


def test_replicas_64_boxes_graph_step_against_oracle():
    """The 64-box replica handle at its real shape (atom counts log-uniform on 2k-60k from
    seed 3, half water, half silica, 1.04 M atoms; boxes of 1-3 CTAs, so the small-batch and
    one-CTA paths run): one step captured as a CUDA graph -- 256 logged moves per box, the
    pair histograms with g, and S(Q) of all 192 columns in the BF16x3 tensor-core mode.
    Every box's moves are replayed on the oracle (trial coordinates of every move, dU on
    every fourth), final coordinates bit-exact; the histograms of eight boxes bit-exact; S(Q)
    within 1e-4 barn of the oracle's Eq. (1) on the GPU's own g."""
    systems = synth.replica_batch()
    nb = len(systems)
    n_moves, seed = 256, 3
    box = epsr.Box(systems)
    ws = np.concatenate([box.epsr_sq_weights(b)[0] for b in range(nb)])
    flats = np.array([box.epsr_sq_weights(b)[1] for b in range(nb)])
    Q = systems[0].Q
    plan = epsr.SqPlan(Q, 600, 0.02, epsr.SQ_BF16X3, max_cols=3 * nb)
    H = torch.zeros(box.hist_len, dtype=torch.int64, device=DEV)
    g = torch.zeros(box.hist_len, dtype=torch.float32, device=DEV)
    S = torch.zeros((nb, len(Q)), dtype=torch.float32, device=DEV)
    log = torch.zeros((nb * n_moves * 128,), dtype=torch.uint8, device=DEV)
    st = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=st):
        cs = torch.cuda.current_stream().cuda_stream
        box.epsr_mc_sweep_async(n_moves, seed, 0, log=log, stream=cs)
        H.zero_()
        box.epsr_partial_gr(H, g, 1, stream=cs)
        plan.epsr_sq_exec(g.view(-1, 600), ws, 3, flats, None, S, stream=cs)
    graph.replay()
    torch.cuda.synchronize()
    assert box.epsr_mc_status() == epsr.EPSR_OK
    assert plan.epsr_sq_plan_status() == epsr.EPSR_OK
    lg = log.cpu().numpy().view(epsr.MOVE_LOG_DTYPE).reshape(nb, n_moves)
    xyz = box.epsr_box_get_coords()
    Hn = H.cpu().numpy().astype(np.uint64)
    finals = []
    for b, s in enumerate(systems):
        h0, a0 = box.epsr_box_offsets(b)
        ob, checked, _, flips = replay(s, s.xyz, lg[b], seed, box_index=b, check_every=4)
        assert checked == n_moves // 4 and flips <= 2
        assert np.array_equal(xyz[a0:a0 + s.n_atoms], ob.xyz), b
        finals.append((ob, h0))
    order = np.argsort([s.n_atoms for s in systems])
    for b in list(order[:4]) + list(order[-4:]):
        ob, h0 = finals[b]
        ref = ob.histogram(threads=0)
        assert np.array_equal(Hn[h0:h0 + ref.size].reshape(ref.shape), ref), b
    gh = g.cpu().numpy().astype(np.float64).reshape(-1, 600)
    _, St_ref = oracle.sq(gh, 0.02, Q.astype(np.float32).astype(np.float64), ws, 3, flats)
    err = np.abs(S.cpu().numpy() - St_ref).max()
    print(f"64 replicas: BF16x3 S(Q) max |dS| {err:.3e} barn")
    assert err <= 1e-4


def test_autotune_keeps_state_and_results():
    """The autotuner times launch shapes on the handle itself and restores its state: the
    coordinates and running statistics are unchanged by tuning, the chain run with the tuned
    settings replays against the oracle, the tuned histogram equals the oracle's bit for bit,
    and a second handle of the same shape takes the cached choice without timing."""
    systems = [synth.water_box(700, seed=91), synth.silica_box(600, seed=92),
               synth.water_box(1500, seed=93)]
    box = epsr.Box(systems)
    box.epsr_mc_sweep(300, seed=40)
    xyz0 = box.epsr_box_get_coords()
    st0 = box.epsr_mc_stats_get()
    t = box.epsr_autotune(probe_moves=512)
    print("tuning:", t)
    assert t["from_cache"] == 0 and t["mc_batch"] in (16, 32, 64) and t["gr_ctas_per_sm"] in (2, 3, 4)
    assert box.epsr_box_get_launch() == {"mc_batch": t["mc_batch"], "mc_ctas": t["mc_ctas"],
                                         "gr_ctas_per_sm": t["gr_ctas_per_sm"]}
    assert np.array_equal(box.epsr_box_get_coords(), xyz0)
    assert box.epsr_mc_stats_get() == st0
    stats, log = run_logged(box, 1000, seed=41, move0=300)
    xyz = box.epsr_box_get_coords()
    Hg = gpu_hist(box)
    for b, s in enumerate(systems):
        h0, a0 = box.epsr_box_offsets(b)
        ob, checked, _, flips = replay(s, xyz0[a0:a0 + s.n_atoms], log[b], 41, move0=300, box_index=b,
                                       check_every=2)
        assert flips <= 2
        assert np.array_equal(xyz[a0:a0 + s.n_atoms], ob.xyz), b
        ref = ob.histogram()
        assert np.array_equal(Hg[h0:h0 + ref.size].reshape(ref.shape), ref), b
    second = epsr.Box(systems)
    t2 = second.epsr_autotune()
    assert t2["from_cache"] == 1
    assert (t2["mc_batch"], t2["mc_ctas"], t2["gr_ctas_per_sm"]) == (t["mc_batch"], t["mc_ctas"], t["gr_ctas_per_sm"])


def test_mc_energy_drift(small_water):
    box = epsr.Box(small_water)
    U0 = box.epsr_box_total_energy()[0]
    stats = box.epsr_mc_sweep(5000, seed=3, move0=0)
    U1 = box.epsr_box_total_energy()[0]
    assert abs((U1 - U0) - stats[0][3]) < 1e-4 * abs(U0) + 1.0


def test_mc_deterministic(small_water):
    a = epsr.Box(small_water)
    b = epsr.Box(small_water)
    a.epsr_mc_sweep(1000, seed=8)
    b.epsr_mc_sweep(600, seed=8)
    b.epsr_mc_sweep(400, seed=8, move0=600)
    assert np.array_equal(a.epsr_box_get_coords(), b.epsr_box_get_coords())


def test_barrier_timeout_is_reported_and_context_survives():
    s = synth.water_box(2000, seed=44)
    box = epsr.Box(s)
    box.epsr_mc_set_ctas(4)
    box.epsr_debug_barrier_fault(2, 200.0)
    with pytest.raises(epsr.EpsrError) as ei:
        box.epsr_mc_sweep(100, seed=1)
    assert ei.value.status == epsr.EPSR_ETIMEOUT
    box.epsr_debug_barrier_fault(-1, 2000.0)
    # the context is still usable
    H = gpu_hist(epsr.Box(synth.small_water()))
    assert H.sum() > 0


# --------------------------------------------------------------------------------------
# S(Q)
# --------------------------------------------------------------------------------------

def test_sq_fp32_against_oracle(small_water):
    box = epsr.Box(small_water)
    H = torch.zeros(box.hist_len, dtype=torch.int64, device=DEV)
    g = torch.zeros(box.hist_len, dtype=torch.float32, device=DEV)
    box.epsr_partial_gr(H, g, 1)
    w, flat = box.epsr_sq_weights(0)
    S_p = torch.zeros((3, len(small_water.Q)), dtype=torch.float32, device=DEV)
    S_t = torch.zeros((1, len(small_water.Q)), dtype=torch.float32, device=DEV)
    epsr.epsr_sq(g.view(3, -1), small_water.dr, small_water.Q, w, 3, np.array([flat]), S_p, S_t)
    torch.cuda.synchronize()
    ob = oracle.Box(small_water)
    gref = ob.normalize_g(H.cpu().numpy().astype(np.uint64).reshape(3, -1))
    Sp_ref, St_ref = oracle.sq_of_box(ob, gref, Q=small_water.Q.astype(np.float32).astype(np.float64))
    W, fl = oracle.eq1_weights(small_water)
    assert abs(fl - flat) < 1e-15
    assert np.abs(S_t.cpu().numpy()[0] - St_ref).max() < 1e-4
    assert np.abs(S_p.cpu().numpy() - Sp_ref).max() < 1e-4


def test_sq_flat_background_gpu():
    Q = 0.3 + np.arange(2000) * (39.7 / 1999)
    g = torch.ones((6, 600), dtype=torch.float32, device=DEV)
    S_t = torch.zeros((2, 2000), dtype=torch.float32, device=DEV)
    epsr.epsr_sq(g, 0.02, Q, np.ones(6), 3, np.array([0.25, 0.5]), None, S_t)
    torch.cuda.synchronize()
    assert torch.all(S_t[0] == 0.25) and torch.all(S_t[1] == 0.5)


# --------------------------------------------------------------------------------------
# batched replicas under a captured CUDA graph
# --------------------------------------------------------------------------------------

def _replica_systems():
    Q = 0.3 + np.arange(2000) * (39.7 / 1999)
    return [synth.water_box(700, seed=81, n_bins=600, bin_p=2, bin_q=100, Q=Q),
            synth.silica_box(500, seed=82, n_bins=600, bin_p=2, bin_q=100, Q=Q),
            synth.water_box(1500, seed=83, n_bins=600, bin_p=2, bin_q=100, Q=Q),
            synth.silica_box(900, seed=84, n_bins=600, bin_p=2, bin_q=100, Q=Q)]


def _replica_step(box, plan, H, g, S, w, flat, n_moves, seed, move0, stream):
    box.epsr_mc_sweep_async(n_moves, seed, move0, stream=stream)
    box.epsr_partial_gr(H, g, 1, stream=stream)
    plan.epsr_sq_exec(g.view(-1, 600), w, 3, flat, None, S, stream=stream)


def test_replicas_step_captured_in_cuda_graph():
    systems = _replica_systems()
    nb = len(systems)
    boxes = [epsr.Box(systems), epsr.Box(systems)]
    ws = np.concatenate([boxes[0].epsr_sq_weights(b)[0] for b in range(nb)])
    flats = np.array([boxes[0].epsr_sq_weights(b)[1] for b in range(nb)])
    plan = epsr.SqPlan(systems[0].Q, 600, 0.02, epsr.SQ_FP32, max_cols=3 * nb)
    bufs = []
    for bx in boxes:
        bufs.append((torch.zeros(bx.hist_len, dtype=torch.int64, device=DEV),
                     torch.zeros(bx.hist_len, dtype=torch.float32, device=DEV),
                     torch.zeros((nb, 2000), dtype=torch.float32, device=DEV)))
    # eager reference: two steps
    s0 = torch.cuda.Stream()
    with torch.cuda.stream(s0):
        for k in range(2):
            bufs[0][0].zero_()
            _replica_step(boxes[0], plan, *bufs[0], ws, flats, 400, 11, 400 * k, s0.cuda_stream)
    s0.synchronize()
    # captured: one graph per step (the move indices are baked into the graph)
    s1 = torch.cuda.Stream()
    graphs = []
    for k in range(2):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s1):
            bufs[1][0].zero_()
            _replica_step(boxes[1], plan, *bufs[1], ws, flats, 400, 11, 400 * k,
                          torch.cuda.current_stream().cuda_stream)
        graphs.append(g)
    # capture ran nothing; start from the same coordinates and replay
    boxes[1].epsr_box_set_coords(np.concatenate([s.xyz for s in systems]))
    for g in graphs:
        g.replay()
    torch.cuda.synchronize()
    assert boxes[1].epsr_mc_status() == epsr.EPSR_OK
    assert np.array_equal(boxes[0].epsr_box_get_coords(), boxes[1].epsr_box_get_coords())
    for a, b in zip(bufs[0], bufs[1]):
        assert torch.equal(a, b)


# --------------------------------------------------------------------------------------
# empirical-potential update
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("n_data,gamma", [(3, 0.0), (1, 1.0)])
def test_ep_update_against_oracle(small_water, n_data, gamma):
    s = small_water
    box = epsr.Box(s)
    rng = np.random.default_rng(12)
    Q = s.Q
    rho = s.n_atoms / s.L ** 3
    F = oracle.ep_basis_matrix(20, 0.5, Q, rho)
    C_true = rng.normal(size=(3, 20)) * 0.01
    w = rng.uniform(0.05, 0.3, (n_data, 3))
    dS32 = (w @ (C_true @ F.T)).astype(np.float32)
    dS = torch.from_numpy(dS32).to(DEV)
    C_gpu = box.epsr_ep_update(0, dS, w, Q, n_basis=20, s_basis=0.5, gamma=gamma, alpha=1.0)
    table = box.epsr_box_get_ep(0, (3, s.n_bins)).astype(np.float64)
    Qf = Q.astype(np.float32).astype(np.float64)
    Ff = oracle.ep_basis_matrix(20, 0.5, Qf, rho)
    dSp = oracle.pair_resolve(dS32.astype(np.float64), w, gamma)
    C_ref = oracle.ep_fit(dSp, Ff)
    kT = oracle.gas_constant() * s.temperature
    ref = oracle.ep_table(C_ref, 0.5, s.n_bins, s.dr, 1.0, kT)
    # the fitted Delta S is well determined; the coefficients carry the basis's conditioning
    assert np.abs(C_gpu @ Ff.T - C_ref @ Ff.T).max() <= 1e-8 * np.abs(dSp).max()
    assert np.abs(C_gpu - C_ref).max() <= 1e-3 * np.abs(C_ref).max()
    assert np.abs(table - ref).max() <= 1e-4 * np.abs(ref).max() + 1e-6
    # the update is additive: a second call adds the same increment
    box.epsr_ep_update(0, dS, w, Q, n_basis=20, s_basis=0.5, gamma=gamma, alpha=1.0)
    t2 = box.epsr_box_get_ep(0, (3, s.n_bins)).astype(np.float64)
    assert np.abs(t2 - 2 * ref).max() <= 2e-4 * np.abs(ref).max() + 1e-6


# --------------------------------------------------------------------------------------
# the refinement loop (Sec. 2.2 items III-VI; Eq. 2)
# --------------------------------------------------------------------------------------

def test_refine_pass_against_oracle():
    """Two passes of the GPU refiner (2,000 logged moves each, histograms accumulated) against
    the oracle's pass on the same inputs: the oracle replays each pass's moves with the GPU's
    table as it was, then computes the pass itself. Histograms bit-exact; S(Q) and Delta S
    within 1e-4 barn; the fitted pair-resolved Delta S and the table update within the
    tolerance the FP32 Delta S allows."""
    s = synth.lj_fluid(10, seed=61)
    Q = s.Q.astype(np.float32).astype(np.float64)
    W, flat = oracle.eq1_weights(s)
    rng = np.random.default_rng(3)
    target64 = flat + 0.05 * np.sin(Q * 1.3) * np.exp(-Q / 8) + rng.normal(size=len(Q)) * 0.002
    target = torch.tensor(target64[None, :], dtype=torch.float32, device=DEV)
    box = epsr.Box(s)
    plan = epsr.SqPlan(s.Q, s.n_bins, s.dr, epsr.SQ_FP32, max_cols=1)
    ref = epsr.Refiner(box, plan, target, W[None, :], np.array([flat]), s.Q, moves_per_pass=2000, seed=17,
                       accumulate=True, n_basis=20, s_basis=0.5, gamma=0.0, alpha=1.0)
    ob = oracle.Box(s)
    tgt = target.cpu().numpy().astype(np.float64)
    H_acc, n_cfg = None, 0
    rho = s.n_atoms / s.L ** 3
    F = oracle.ep_basis_matrix(20, 0.5, Q, rho)
    for it in range(2):
        ep_before = box.epsr_box_get_ep(0, (1, s.n_bins)).astype(np.float64)
        log = torch.zeros((2000 * 128,), dtype=torch.uint8, device=DEV)
        res = ref.step(log=log)
        lg = log.cpu().numpy().view(epsr.MOVE_LOG_DTYPE)
        ob.set_ep(ep_before if it else None)
        ob2, checked, _, flips = replay(s, ob.xyz, lg, 17, move0=2000 * it, ep=ob.ep)
        assert flips <= 2
        ob.xyz[:] = ob2.xyz
        r = oracle.refine_pass(ob, tgt, W[None, :], np.array([flat]), Q, 20, 0.5, 0.0, 1.0, H_acc=H_acc, n_cfg=n_cfg)
        H_acc, n_cfg = r["H"], r["n_cfg"]
        Hg = torch.zeros(s.n_bins, dtype=torch.int64, device=DEV)
        Sg = torch.zeros((1, len(Q)), dtype=torch.float32, device=DEV)
        dSg = torch.zeros((1, len(Q)), dtype=torch.float32, device=DEV)
        C_gpu = ref.get(hist=Hg, S=Sg, dS=dSg)
        assert np.array_equal(Hg.cpu().numpy().astype(np.uint64), r["H"][0])
        assert res["n_configs"] == it + 1 and res["iteration"] == it + 1
        assert np.abs(Sg.cpu().numpy() - r["S"]).max() <= 1e-4
        assert np.abs(dSg.cpu().numpy() - r["dS"]).max() <= 1e-4
        assert abs(res["chi2"] - r["chi2"]) <= 1e-3 * r["chi2"] + 1e-6
        fit_gpu, fit_ref = C_gpu @ F.T, r["C"] @ F.T
        assert np.abs(fit_gpu - fit_ref).max() <= 1e-3 * np.abs(fit_ref).max() + 1e-4
        ep_gpu = box.epsr_box_get_ep(0, (1, s.n_bins)).astype(np.float64)
        inc_ref = r["ep"] - (ep_before if it else 0.0)
        assert np.abs((ep_gpu - ep_before) - inc_ref).max() <= 1e-3 * np.abs(inc_ref).max() + 1e-4
        ob.set_ep(ep_gpu)


def test_refine_pass_three_isotopic_datasets():
    """The paper's water case: three datasets of the same box that differ only in the hydrogen
    scattering length (H2O, D2O and an HDO-like 50:50 mixture), so the 3 x 3 weight matrix is
    square and Eq. (2) inverts it (gamma = 0). One pass of 1,000 logged moves: the oracle replays
    the moves and computes the pass; histograms bit-exact, S(Q) of every dataset and Delta S
    within 1e-4 barn, fitted pair-resolved Delta S and table increment within the FP32 tolerance."""
    s = synth.water_box(300, seed=18, L_A=20.8)
    b_H, b_D = -3.739, 6.671
    ws, flats = [], []
    for bh in (b_H, b_D, 0.5 * (b_H + b_D)):
        sd = synth.System(**{**s.__dict__, "b": [s.b[0], bh]})
        W, fl = oracle.eq1_weights(sd)
        ws.append(W)
        flats.append(fl)
    w = np.array(ws)
    flat = np.array(flats)
    assert abs(np.linalg.det(w)) > 1e-6            # three independent datasets
    Q = s.Q.astype(np.float32).astype(np.float64)
    tgt64 = flat[:, None] + 0.03 * np.sin(np.outer([1.0, 1.3, 0.8], Q)) * np.exp(-Q / 6)
    target = torch.tensor(tgt64, dtype=torch.float32, device=DEV)
    box = epsr.Box(s)
    plan = epsr.SqPlan(s.Q, s.n_bins, s.dr, epsr.SQ_FP32, max_cols=9)
    ref = epsr.Refiner(box, plan, target, w, flat, s.Q, moves_per_pass=1000, seed=23, accumulate=True,
                       n_basis=20, s_basis=0.5, gamma=0.0, alpha=1.0)
    log = torch.zeros((1000 * 128,), dtype=torch.uint8, device=DEV)
    res = ref.step(log=log)
    lg = log.cpu().numpy().view(epsr.MOVE_LOG_DTYPE)
    ob, _, _, flips = replay(s, s.xyz, lg, 23)
    assert flips <= 2
    r = oracle.refine_pass(ob, target.cpu().numpy().astype(np.float64), w, flat, Q, 20, 0.5, 0.0, 1.0)
    Hg = torch.zeros(box.hist_len, dtype=torch.int64, device=DEV)
    Sg = torch.zeros((3, len(Q)), dtype=torch.float32, device=DEV)
    dSg = torch.zeros((3, len(Q)), dtype=torch.float32, device=DEV)
    C_gpu = ref.get(hist=Hg, S=Sg, dS=dSg)
    assert np.array_equal(Hg.cpu().numpy().astype(np.uint64).reshape(3, -1), r["H"])
    assert np.abs(Sg.cpu().numpy() - r["S"]).max() <= 1e-4
    assert np.abs(dSg.cpu().numpy() - r["dS"]).max() <= 1e-4
    assert abs(res["chi2"] - r["chi2"]) <= 1e-3 * r["chi2"]
    F = oracle.ep_basis_matrix(20, 0.5, Q, s.n_atoms / s.L ** 3)
    fit_gpu, fit_ref = C_gpu @ F.T, r["C"] @ F.T
    assert np.abs(fit_gpu - fit_ref).max() <= 1e-3 * np.abs(fit_ref).max() + 1e-4
    ep_gpu = box.epsr_box_get_ep(0, (3, s.n_bins)).astype(np.float64)
    assert np.abs(ep_gpu - r["ep"]).max() <= 1e-3 * np.abs(r["ep"]).max() + 1e-4


def test_refine_loop_reduces_chi2_on_the_gpu():
    """The GPU refiner against a target the oracle simulated with a planted repulsive bump
    (1.5 kJ/mol at 4.5 A) in an argon-like liquid: chi^2 falls to under half its first value
    within eight passes of 20,000 moves and the learned potential is repulsive at the bump
    (above a fifth of the planted height there)."""
    s0 = synth.lj_fluid(10, seed=52)
    r = (np.arange(s0.n_bins) + 0.5) * s0.dr
    bump = 1.5 * np.exp(-((r - 4.5) / 0.4) ** 2)
    o = oracle.Box(s0, ep=bump[None, :])
    o.mc_sweep(20000, seed=52)
    H = None
    for k in range(8):
        o.mc_sweep(2000, seed=52, move0=20000 + 2000 * k)
        h = o.histogram()
        H = h if H is None else H + h
    W, flat = oracle.eq1_weights(s0)
    rho = oracle.number_density(s0)
    Q64 = s0.Q.astype(np.float32).astype(np.float64)
    _, St = oracle.sq(o.normalize_g(H, 8), s0.dr, Q64, 4.0 * math.pi * rho * W, 1, np.array([flat]))
    target = torch.tensor(St, dtype=torch.float32, device=DEV)
    s = synth.lj_fluid(12, seed=53)
    box = epsr.Box(s)
    box.epsr_mc_sweep(40000, seed=53)
    plan = epsr.SqPlan(s.Q, s.n_bins, s.dr, epsr.SQ_FP32, max_cols=1)
    ref = epsr.Refiner(box, plan, target, W[None, :], np.array([flat]), s.Q, moves_per_pass=20000, seed=54,
                       move0=10**6, accumulate=False, n_basis=20, s_basis=0.5, gamma=0.0, alpha=1.0)
    chi = [ref.step()["chi2"] for _ in range(8)]
    print("chi2 per pass:", ["%.2e" % c for c in chi])
    ep = box.epsr_box_get_ep(0, (1, s.n_bins))[0]
    k = int(4.5 / s.dr)
    assert min(chi[-3:]) < 0.5 * chi[0], chi
    assert ep[k] > 0.2 * bump[k], ep[k]


# --------------------------------------------------------------------------------------
# differentiable form: smeared g(r), chi^2 and its adjoint
# --------------------------------------------------------------------------------------

def _diff_setup(s, target_seed, sigma, n_basis=4, noise=0.005):
    box = epsr.Box(s)
    W, flat = oracle.eq1_weights(s)
    rho = s.n_atoms / s.L ** 3
    w_cols = 4 * math.pi * rho * W
    Q = s.Q.astype(np.float32).astype(np.float64)
    plan = epsr.SqPlan(s.Q, s.n_bins, s.dr, epsr.SQ_FP32, max_cols=3)
    rng = np.random.default_rng(target_seed)
    target = flat + rng.normal(size=len(Q)) * noise
    C_ = rng.normal(size=(3, n_basis)) * 0.01
    return box, plan, W, flat, rho, w_cols, Q, target, C_


def test_smeared_chi2_and_gradients_small_box():
    s = synth.water_box(300, seed=41, L_A=20.8)
    sigma = 0.05
    box, plan, W, flat, rho, w_cols, Q, target, C_ = _diff_setup(s, 5, sigma)
    F = epsr.smeared_chi2_function()
    pos = torch.zeros((s.n_atoms, 3), dtype=torch.float32, device=DEV, requires_grad=True)
    Ct = torch.tensor(C_, dtype=torch.float64, device=DEV, requires_grad=True)
    tgt = torch.tensor(target, dtype=torch.float32, device=DEV)
    chi2 = F.apply(pos, Ct, box, plan, sigma, W, w_cols, flat, tgt, 0.5, rho)
    chi2.backward()
    ob = oracle.Box(s)
    tgt64 = tgt.cpu().numpy().astype(np.float64)
    c_ref, dC_ref, gx_ref, S_ref, _ = oracle.chi2_and_grads(ob, sigma, Q, tgt64, C_, 0.5)
    assert abs(chi2.item() - c_ref) <= 1e-4 * abs(c_ref)
    assert np.abs(Ct.grad.cpu().numpy() - dC_ref).max() <= 1e-4 * np.abs(dC_ref).max()
    g = pos.grad.cpu().numpy()
    rel = np.linalg.norm(g - gx_ref) / np.linalg.norm(gx_ref)
    assert rel <= 1e-4, rel


@pytest.mark.parametrize("n_mol,L", [(400, 23.0), (3000, 44.8)], ids=["tiles", "cell-lists"])
def test_smeared_histogram_matches_oracle(n_mol, L):
    """The 23 A box has no cell list (all-pairs tiles); the 44.8 A box has 4 cells per side."""
    s = synth.water_box(n_mol, seed=42, L_A=L)
    box = epsr.Box(s)
    Ht = torch.zeros(box.hist_len, dtype=torch.float64, device=DEV)
    box.epsr_gr_smeared_fwd(0.05, Ht)
    torch.cuda.synchronize()
    ref = oracle.Box(s).smeared_hist(0.05)
    got = Ht.cpu().numpy().reshape(ref.shape)
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()


def test_smeared_gradient_cell_lists_medium_box():
    """chi^2 gradients through the cell-list form (9,000 atoms, 4 cells per side) against
    the oracle for every atom."""
    s = synth.water_box(3000, seed=43, L_A=44.8)
    sigma = 0.05
    box, plan, W, flat, rho, w_cols, Q, target, C_ = _diff_setup(s, 5, sigma)
    F = epsr.smeared_chi2_function()
    pos = torch.zeros((s.n_atoms, 3), dtype=torch.float32, device=DEV, requires_grad=True)
    Ct = torch.tensor(C_, dtype=torch.float64, device=DEV, requires_grad=True)
    tgt = torch.tensor(target, dtype=torch.float32, device=DEV)
    chi2 = F.apply(pos, Ct, box, plan, sigma, W, w_cols, flat, tgt, 0.5, rho)
    chi2.backward()
    ob = oracle.Box(s)
    tgt64 = tgt.cpu().numpy().astype(np.float64)
    c_ref, dC_ref, gx_ref, _, _ = oracle.chi2_and_grads(ob, sigma, Q, tgt64, C_, 0.5)
    assert abs(chi2.item() - c_ref) <= 1e-4 * abs(c_ref)
    g = pos.grad.cpu().numpy()
    assert np.linalg.norm(g - gx_ref) <= 1e-4 * np.linalg.norm(gx_ref)


def test_smeared_gradient_paper_size_sampled():
    """99,999-atom water (seed 4), target from a seed-5 box plus N(0, 0.005^2) noise: the
    GPU gradient of chi^2 against the FP64 oracle on 64 sampled atoms."""
    s = synth.paper_water(seed=4)
    t = synth.paper_water(seed=5)
    sigma = 0.05
    box = epsr.Box(s)
    W, flat = oracle.eq1_weights(s)
    rho = s.n_atoms / s.L ** 3
    w_cols = 4 * math.pi * rho * W
    Q = s.Q.astype(np.float32).astype(np.float64)
    plan = epsr.SqPlan(s.Q, s.n_bins, s.dr, epsr.SQ_FP32, max_cols=3)
    ot = oracle.Box(t)
    _, St = oracle.sq_of_box(ot, ot.normalize_g(ot.histogram(threads=0)), Q=Q)
    target = St + np.random.default_rng(5).normal(size=len(Q)) * 0.005
    C_ = np.random.default_rng(6).normal(size=(3, 20)) * 0.001
    F = epsr.smeared_chi2_function()
    pos = torch.zeros((s.n_atoms, 3), dtype=torch.float32, device=DEV, requires_grad=True)
    Ct = torch.tensor(C_, dtype=torch.float64, device=DEV, requires_grad=True)
    tgt = torch.tensor(target, dtype=torch.float32, device=DEV)
    chi2 = F.apply(pos, Ct, box, plan, sigma, W, w_cols, flat, tgt, 0.5, rho)
    chi2.backward()
    ob = oracle.Box(s)
    idx = np.random.default_rng(7).choice(s.n_atoms, 64, replace=False)
    tgt64 = tgt.cpu().numpy().astype(np.float64)
    c_ref, dC_ref, gx_ref, _, _ = oracle.chi2_and_grads(ob, sigma, Q, tgt64, C_, 0.5, grad_atoms=idx)
    assert abs(chi2.item() - c_ref) <= 1e-4 * abs(c_ref)
    g = pos.grad.cpu().numpy()[idx]
    assert np.linalg.norm(g - gx_ref) <= 1e-4 * np.linalg.norm(gx_ref)


# --------------------------------------------------------------------------------------
# S(Q) on tensor cores (tcgen05) with split precision
# --------------------------------------------------------------------------------------

def _synthetic_g(n_cols, n_bins, dr, seed):
    """g-like columns: excluded core, oscillating shells, a sharp intramolecular spike."""
    rng = np.random.default_rng(seed)
    r = (np.arange(n_bins) + 0.5) * dr
    g = np.ones((n_cols, n_bins))
    for c in range(n_cols):
        r0 = rng.uniform(2.4, 3.2)
        g[c] = 1 + 1.5 * np.exp(-((r - r0) / 0.25) ** 2) - np.exp(-(r / 1.8) ** 8) \
            + 0.3 * np.sin(2 * np.pi * r / r0) * np.exp(-r / 4) + rng.normal(size=n_bins) * 0.01
        k = int(rng.uniform(0.95, 1.6) / dr)
        g[c, k] += rng.uniform(10, 80)
    return g.astype(np.float32)


@pytest.mark.parametrize("mode,tol", [(epsr.SQ_TF32X3, 1e-4), (epsr.SQ_BF16X6, 1e-4),
                                      (epsr.SQ_BF16X3, 1e-4), (epsr.SQ_FP32, 1e-4)])
@pytest.mark.parametrize("n_cols", [3, 192])
def test_sq_modes_against_oracle(mode, tol, n_cols):
    n_bins, dr = 600, 0.02
    Q = 0.3 + np.arange(2000) * (39.7 / 1999)
    g = _synthetic_g(n_cols, n_bins, dr, seed=n_cols)
    rng = np.random.default_rng(3)
    w = rng.uniform(0.05, 0.4, n_cols)
    flat = rng.uniform(0.2, 0.6, n_cols // 3)
    plan = epsr.SqPlan(Q, n_bins, dr, mode, max_cols=n_cols)
    gd = torch.from_numpy(g).to(DEV)
    Sp = torch.zeros((n_cols, 2000), dtype=torch.float32, device=DEV)
    St = torch.zeros((n_cols // 3, 2000), dtype=torch.float32, device=DEV)
    plan.epsr_sq_exec(gd, w, 3, flat, Sp, St)
    torch.cuda.synchronize()
    Sp_ref, St_ref = oracle.sq(g.astype(np.float64), dr, Q.astype(np.float32).astype(np.float64),
                               w, 3, flat)
    err_p = np.abs(Sp.cpu().numpy() - Sp_ref).max()
    err_t = np.abs(St.cpu().numpy() - St_ref).max()
    print(f"mode {mode} cols {n_cols}: max |dS_partial| {err_p:.3e}, max |dS_total| {err_t:.3e}")
    assert err_t <= tol and err_p <= tol
    assert plan.epsr_sq_plan_status() == epsr.EPSR_OK


@pytest.mark.parametrize("mode", [epsr.SQ_BF16X3, epsr.SQ_TF32X3, epsr.SQ_BF16X6])
def test_sq_tensor_core_tilings_against_oracle(mode):
    """Every tiling of the clustered tensor-core contraction -- columns per CTA with the set
    totals in the same launch (48, 96) or in a separate pass (16, 64), and 1 to 8 CTAs per
    output tile along the bins -- gives S(Q) within 1e-4 barn of the oracle, and repeated
    calls are bit-identical (the K-split partials are added in a fixed order)."""
    n_bins, dr, n_cols = 600, 0.02, 192
    Q = 0.3 + np.arange(2000) * (39.7 / 1999)
    g = _synthetic_g(n_cols, n_bins, dr, seed=5)
    rng = np.random.default_rng(4)
    w = rng.uniform(0.05, 0.4, n_cols)
    flat = rng.uniform(0.2, 0.6, n_cols // 3)
    Sp_ref, St_ref = oracle.sq(g.astype(np.float64), dr, Q.astype(np.float32).astype(np.float64), w, 3, flat)
    plan = epsr.SqPlan(Q, n_bins, dr, mode, max_cols=n_cols)
    gd = torch.from_numpy(g).to(DEV)
    for n_chunk, k_split in ((48, 1), (48, 5), (96, 8), (16, 3), (64, 2), (0, 0)):
        plan.epsr_sq_plan_set_tiles(n_chunk, k_split)
        outs = []
        for _ in range(2):
            Sp = torch.zeros((n_cols, 2000), dtype=torch.float32, device=DEV)
            St = torch.zeros((n_cols // 3, 2000), dtype=torch.float32, device=DEV)
            plan.epsr_sq_exec(gd, w, 3, flat, Sp, St)
            torch.cuda.synchronize()
            outs.append((Sp.cpu().numpy(), St.cpu().numpy()))
        assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
        err = max(np.abs(outs[0][0] - Sp_ref).max(), np.abs(outs[0][1] - St_ref).max())
        print(f"mode {mode} tiling ({n_chunk}, {k_split}): max |dS| {err:.3e}")
        assert err <= 1e-4, (n_chunk, k_split, err)
        # totals alone (no partial output requested)
        St2 = torch.zeros((n_cols // 3, 2000), dtype=torch.float32, device=DEV)
        plan.epsr_sq_exec(gd, w, 3, flat, None, St2)
        torch.cuda.synchronize()
        assert np.array_equal(St2.cpu().numpy(), outs[0][1])
    assert plan.epsr_sq_plan_status() == epsr.EPSR_OK
    with pytest.raises(epsr.EpsrError):
        plan.epsr_sq_plan_set_tiles(40, 1)          # not a multiple of 16
    with pytest.raises(epsr.EpsrError):
        plan.epsr_sq_plan_set_tiles(48, 9)          # more than one portable cluster


def test_sq_autotune_picks_a_tiling_that_matches_the_oracle():
    n_bins, dr, n_cols = 600, 0.02, 192
    Q = 0.3 + np.arange(2000) * (39.7 / 1999)
    g = _synthetic_g(n_cols, n_bins, dr, seed=7)
    rng = np.random.default_rng(8)
    w = rng.uniform(0.05, 0.4, n_cols)
    flat = rng.uniform(0.2, 0.6, n_cols // 3)
    _, St_ref = oracle.sq(g.astype(np.float64), dr, Q.astype(np.float32).astype(np.float64), w, 3, flat)
    plan = epsr.SqPlan(Q, n_bins, dr, epsr.SQ_BF16X3, max_cols=n_cols)
    gd = torch.from_numpy(g).to(DEV)
    St = torch.zeros((n_cols // 3, 2000), dtype=torch.float32, device=DEV)
    r = plan.epsr_sq_plan_autotune(gd, w, 3, flat, None, St)
    print("sq tuning:", r)
    assert r["cols_per_cta"] in (16, 32, 48, 64, 96) and r["k_split"] in (1, 2, 4, 8) and r["us"] > 0
    assert plan.epsr_sq_plan_get_tiles(n_cols, 3) == (r["cols_per_cta"], r["k_split"])
    St.zero_()
    plan.epsr_sq_exec(gd, w, 3, flat, None, St)
    torch.cuda.synchronize()
    assert np.abs(St.cpu().numpy() - St_ref).max() <= 1e-4
    plan2 = epsr.SqPlan(Q, n_bins, dr, epsr.SQ_BF16X3, max_cols=n_cols)
    assert plan2.epsr_sq_plan_autotune(gd, w, 3, flat, None, St)["cols_per_cta"] == r["cols_per_cta"]


def test_checkpoint_resume_is_bit_exact():
    s = synth.silica_box(800, seed=91)
    ep = (np.random.default_rng(2).normal(size=(3, s.n_bins)) * 0.2).astype(np.float32)
    a = epsr.Box(s)
    a.epsr_box_set_ep(0, ep)
    a.epsr_mc_sweep(2000, seed=17, move0=0)
    b = epsr.Box(s)
    b.epsr_box_set_ep(0, ep)
    b.epsr_mc_sweep(1000, seed=17, move0=0)
    ck = b.epsr_checkpoint_save()
    c = epsr.Box(synth.silica_box(800, seed=91))      # a fresh handle, zero EP table
    c.epsr_checkpoint_load(ck)
    c.epsr_mc_sweep(1000, seed=17, move0=1000)
    assert np.array_equal(a.epsr_box_get_coords(), c.epsr_box_get_coords())
    assert a.epsr_mc_stats_get()[0][:3] == c.epsr_mc_stats_get()[0][:3]
    assert np.array_equal(c.epsr_box_get_ep(0, ep.shape), ep)
    bad = bytearray(ck)
    bad[0] ^= 1
    with pytest.raises(epsr.EpsrError):
        c.epsr_checkpoint_load(bytes(bad))


def test_measurement_kernels():
    """The grid-barrier floor and the issue-rate kernels run, return finite rates and stay
    below the nominal ceilings (152 SMs x 128 lanes x 2.07 GHz)."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ns = epsr.epsr_bench_barrier_floor(sms, 500)
    assert 100.0 < ns < 1e6
    for kind in (0, 1):
        r = epsr.epsr_bench_alu_rate(kind)
        assert 1e12 < r < 1.2 * sms * 128 * 2.1e9
    with pytest.raises(epsr.EpsrError):
        epsr.epsr_bench_barrier_floor(100000, 10)
