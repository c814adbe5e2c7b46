"""Serving: the request loop over MOFF_SERVED plans (continuous batching with
admission by pool memory).

Each block's result must be the same alone and in the mix: the same served
plans fed the same blocks one at a time (one slot) and interleaved across
plans with several slots must give bit-identical images, and one of them is
checked against the FP64 oracle at the FP32 bar (1e-5).
"""
import time

import numpy as np
import pytest

import oracle
import paper_0812_3669_gb300 as moff
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    moff.build()
    yield


def c64(x):
    return np.asarray(x).astype(np.complex64).astype(np.complex128)


def subarray(seed, A, N, K, P, C, spread):
    """Seeded sub-array: positions in a spread x spread box at the grid centre."""
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, spread, size=(A, 2)) + (N - spread) / 2
    taps = c64(rng.normal(size=(A, P, K, K)) + 1j * rng.normal(size=(A, P, K, K)))
    gains = c64(synth.gains_random(rng, C, A, P))
    return pos, taps, gains


def blocks(seed, T_list, C, A, P):
    rng = np.random.default_rng(seed)
    out = []
    for T in T_list:
        re = np.clip(np.rint(rng.normal(0, 2.5, size=(T, C, A, P))), -7, 7).astype(int)
        im = np.clip(np.rint(rng.normal(0, 2.5, size=(T, C, A, P))), -7, 7).astype(int)
        out.append(synth.pack_4bit(re, im))
    return out


# three sub-arrays of uneven antenna count and grid size
ARRAYS = [
    dict(seed=11, A=256, N=64, K=5, P=2, C=6, spread=30, T=[40, 25, 33]),
    dict(seed=12, A=700, N=128, K=7, P=2, C=3, spread=90, T=[20, 31]),
    dict(seed=13, A=150, N=256, K=3, P=1, C=4, spread=120, T=[17, 9, 12, 5]),
]


def served_plans():
    plans, data = [], []
    for a in ARRAYS:
        pos, taps, gains = subarray(a["seed"], a["A"], a["N"], a["K"], a["P"], a["C"], a["spread"])
        pl = moff.Plan(pos, taps, a["N"], a["C"], a["P"], served=True)
        pl.set_gains(gains)
        plans.append(pl)
        data.append((pos, taps, gains, blocks(a["seed"] + 100, a["T"], a["C"], a["A"], a["P"])))
    return plans, data


def images(plans):
    out = []
    for pl in plans:
        img, n = pl.read_image()
        out.append((img, n))
    return out


def test_served_plan_takes_blocks_only_through_the_server():
    pos, taps, gains = subarray(1, 20, 32, 3, 1, 2, 20)
    with moff.Plan(pos, taps, 32, 2, 1, served=True) as pl:
        with pytest.raises(moff.MoffError) as e:
            pl.submit(blocks(2, [3], 2, 20, 1)[0])
        assert e.value.status == -4 and "MOFF_SERVED" in str(e.value)
    # a plan without the flag is refused by the server
    with moff.Server(1 << 26, 2) as srv, moff.Plan(pos, taps, 32, 2, 1) as pl:
        with pytest.raises(moff.MoffError) as e:
            srv.submit(pl, blocks(2, [3], 2, 20, 1)[0])
        assert e.value.status == -4


def test_mix_equals_alone_and_matches_oracle():
    # alone: one slot, each plan's blocks in order, one plan after the other
    plans_a, data = served_plans()
    with moff.Server(8 << 30, 1) as srv:
        for pl, (_, _, _, blks) in zip(plans_a, data):
            for b in blks:
                srv.submit(pl, b)
            srv.wait(0, 120000)
    alone = images(plans_a)
    # mix: several slots, blocks interleaved across plans, host and device inputs
    plans_m, _ = served_plans()
    dev_blocks = [[torch.from_numpy(b).cuda() for b in d[3]] for d in data]
    torch.cuda.synchronize()
    with moff.Server(8 << 30, 3) as srv:
        tickets = []
        for r in range(max(len(d[3]) for d in data)):
            for i, pl in enumerate(plans_m):
                if r < len(data[i][3]):
                    src = dev_blocks[i][r] if (r + i) % 2 else data[i][3][r]
                    tickets.append(srv.submit(pl, src))
        srv.wait(0, 120000)
        for t in tickets:
            st, ms = srv.poll(t)
            assert st == 2 and ms > 0.0
        stats = srv.stats()
    mix = images(plans_m)
    for (ia, na), (im, nm), d in zip(alone, mix, data):
        assert na == nm == sum(b.shape[0] for b in d[3])
        assert np.array_equal(ia, im)
    assert stats["completed"] == len(tickets)
    assert 0.0 < stats["p50_ms"] <= stats["p99_ms"] and stats["throughput"] > 0.0
    # the N = 128 dual-pol sub-array against the FP64 oracle
    pos, taps, gains, blks = data[1]
    a = ARRAYS[1]
    ref = oracle.moff_image(np.concatenate(blks), gains, pos, taps, a["N"], a["P"])
    err = oracle.max_norm_err(mix[1][0], ref)
    print("served N=128 dual-pol: max-normalised error", float(err.max()))
    assert err.max() <= TOL32
    for pl in plans_a + plans_m:
        pl.close()


def test_admission_by_pool_memory():
    """A pool that holds one block's scratch runs the blocks of two plans one at
    a time; a pool that holds two runs them together."""
    pos, taps, gains = subarray(21, 1024, 128, 7, 2, 64, 100)
    plans = [moff.Plan(pos, taps, 128, 64, 2, served=True) for _ in range(2)]
    for pl in plans:
        pl.set_gains(gains)
    rng = np.random.default_rng(22)   # 4000 samples x 64 channels: tens of ms per block
    volt = torch.from_numpy(rng.integers(0, 256, size=(4000, 64, 1024, 2), dtype=np.uint8)).cuda()
    torch.cuda.synchronize()
    info = plans[0].info()
    need = info["time_chunk"] * info["chan_chunk"] * 2 * 128 * 128 * 8   # FP32 row-field scratch
    for n_fit, overlap_expected in [(1, False), (2, True)]:
        with moff.Server(n_fit * need + 4096, 2) as srv:
            t1 = srv.submit(plans[0], volt)
            t2 = srv.submit(plans[1], volt)
            seen_overlap = False
            t0 = time.time()
            while time.time() - t0 < 60:
                s2 = srv.poll(t2)[0]
                s1 = srv.poll(t1)[0]
                if s2 >= 1 and s1 == 1:
                    seen_overlap = True
                if not overlap_expected:
                    # the second block's scratch only frees up when the first retires
                    assert s2 == 0 or s1 == 2
                if s1 == 2 and s2 == 2:
                    break
            srv.wait(0, 120000)
            assert srv.poll(t1)[0] == 2 and srv.poll(t2)[0] == 2
            if overlap_expected:
                assert seen_overlap
    for pl in plans:
        pl.close()


def test_block_larger_than_pool_is_refused_and_destroy_cancels_queue():
    pos, taps, gains = subarray(31, 64, 64, 3, 1, 8, 40)
    with moff.Plan(pos, taps, 64, 8, 1, served=True) as pl:
        b = blocks(32, [10], 8, 64, 1)[0]
        with moff.Server(1 << 12, 1) as srv:
            with pytest.raises(moff.MoffError) as e:
                srv.submit(pl, b)
            assert e.value.status == -2
        srv = moff.Server(1 << 28, 1)
        for _ in range(50):
            srv.submit(pl, b)
        srv.close()                                            # cancels what has not started
        img, n = pl.read_image()
        assert 0 <= n <= 500 and n % 10 == 0
        assert np.isfinite(img).all()


def test_served_tensor_core_plan_equals_unserved():
    """A MOFF_SERVED plan on the FP16 tensor-core path borrows its field scratch and
    voltage planes from the pool per block (tensor maps encoded per block): its
    image equals the same plan's unserved image bit for bit."""
    pos, taps, gains = subarray(41, 400, 128, 7, 2, 5, 90)
    blks = blocks(42, [70, 33], 5, 400, 2)
    with moff.Plan(pos, taps, 128, 5, 2, fp16tc=True) as pu:
        pu.set_gains(gains)
        for b in blks:
            pu.submit(b)
        ref, nr = pu.read_image()
    with moff.Plan(pos, taps, 128, 5, 2, fp16tc=True, served=True) as ps, moff.Server(8 << 30, 2) as srv:
        ps.set_gains(gains)
        for b in blks:
            srv.submit(ps, b)
        srv.wait(0, 120000)
        img, n = ps.read_image()
    assert n == nr == 103
    assert np.array_equal(img, ref)


def test_served_large_dense_array_equals_unserved():
    """A served plan on the tensor-core gridding route for an array large enough for the row plane kernel
    (6400 dual-pol antennas: 12 800 code bytes per channel-sample) borrows its planes from the pool per block,
    with their load and store tensor maps encoded per block: its image equals the unserved plan's bit for
    bit, over two blocks (one ragged), and is within the reduced-precision bar of the oracle."""
    rng = np.random.default_rng(4242)
    side, N, K, P, C = 80, 256, 5, 2, 2
    pos = synth.positions_lattice(rng, side, side, 1.0, 0.05, (N / 2 - side, N / 2 - side))
    A = len(pos)
    taps = c64(synth.taps_gaussian(rng, pos, K, 1.2, n_pol=P))
    gains = c64(synth.gains_random(rng, C, A, P))
    blks = blocks(4243, [29, 11], C, A, P)
    with moff.Plan(pos, taps, N, C, P, fp16tc=True) as pu:
        assert pu.route() == "fp16_tcgrid"
        pu.set_gains(gains)
        for b in blks:
            pu.submit(b)
        ref, nr = pu.read_image()
    with moff.Plan(pos, taps, N, C, P, fp16tc=True, served=True) as ps, moff.Server(8 << 30, 2) as srv:
        ps.set_gains(gains)
        for b in blks:
            srv.submit(ps, b)
        srv.wait(0, 120000)
        img, n = ps.read_image()
    assert n == nr == 40
    assert np.array_equal(img, ref)
    err = oracle.max_norm_err(img, oracle.moff_image(np.concatenate(blks), gains, pos, taps, N, P))
    print(f"served large dense array: max-normalised error {float(err.max()):.2e}")
    assert err.max() <= 3e-3


def test_served_fp16_routes_mix_equals_alone_and_match_oracle():
    """The FP16 stream of the serving pattern: a dense 48 x 48 lattice on the 256
    grid (tensor-core gridding and factored DFT) and a sparse array (row-spectrum
    contraction) served beside an FP32 plan.  Each image is bit-identical alone
    and in the mix, and within the reduced-precision bar (3e-3) of the oracle."""
    rng = np.random.default_rng(91)
    side, N, K, C = 48, 256, 7, 3
    dpos = synth.positions_lattice(rng, side, side, 1.0, 0.05, (N / 2 - side, N / 2 - side))
    dtaps = c64(synth.taps_gaussian(rng, dpos, K, 1.2, n_pol=2))
    dgains = c64(synth.gains_random(rng, C, dpos.shape[0], 2))
    spos, staps, sgains = subarray(92, 300, 128, 7, 2, 4, 100)
    fpos, ftaps, fgains = subarray(93, 200, 64, 5, 2, 2, 40)
    cases = [(dpos, dtaps, dgains, N, C, True, "fp16_tcgrid", blocks(94, [37, 20], C, dpos.shape[0], 2)),
             (spos, staps, sgains, 128, 4, True, "fp16_rowspec", blocks(95, [30, 11], 4, 300, 2)),
             (fpos, ftaps, fgains, 64, 2, False, "fp32", blocks(96, [25, 16], 2, 200, 2))]

    def make():
        out = []
        for pos, taps, gains, n, c, tc, route, _ in cases:
            pl = moff.Plan(pos, taps, n, c, 2, served=True, fp16tc=tc)
            assert pl.route() == route, pl.route()
            pl.set_gains(gains)
            out.append(pl)
        return out

    plans_a = make()
    with moff.Server(8 << 30, 1) as srv:
        for pl, case in zip(plans_a, cases):
            for b in case[7]:
                srv.submit(pl, b)
            srv.wait(0, 120000)
    alone = images(plans_a)
    plans_m = make()
    with moff.Server(8 << 30, 3) as srv:
        for r in range(2):
            for pl, case in zip(plans_m, cases):
                srv.submit(pl, case[7][r])
        srv.wait(0, 120000)
    mix = images(plans_m)
    for (ia, na), (im, nm), case in zip(alone, mix, cases):
        assert na == nm == sum(b.shape[0] for b in case[7])
        assert np.array_equal(ia, im), case[6]
    for (img, _), (pos, taps, gains, n, _, tc, route, blks) in zip(mix, cases):
        ref = oracle.moff_image(np.concatenate(blks), gains, pos, taps, n, 2)
        err = oracle.max_norm_err(img, ref)
        print(f"served {route}: max-normalised error {float(err.max()):.2e}")
        assert err.max() <= (3e-3 if tc else TOL32)
    for pl in plans_a + plans_m:
        pl.close()
