"""GPU parity of the batched path: one persistent launch over many images of mixed
size, pixel type, operator and connectivity must give, image by image, exactly the
oracle's result, under any schedule (tile order, per-tile sweep counts)."""
import numpy as np
import pytest

from paper_1605_00930_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def iw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_00930_gb300 import build
    build.build()
    from paper_1605_00930_gb300 import iwpp
    iwpp.lib()
    return iwpp


def _mixed_cases(seed, n, max_side=300):
    rng = np.random.default_rng(seed)
    cases = []
    for i in range(n):
        H, W = int(rng.integers(1, max_side)), int(rng.integers(1, max_side))
        is16 = bool(rng.integers(0, 2))
        field = synth.blob_field_u8(H, W, max(1, H * W // 3000), rng)
        mask = synth.to_u16(field) if is16 else field
        conn = int(rng.choice([4, 8]))
        if rng.random() < 0.5:
            h = int(rng.integers(5, 60)) * (257 if is16 else 1)
            cases.append(synth.Case(synth.hdome_marker(mask, h), mask, conn, "dilate"))
        else:
            cases.append(synth.Case(synth.fillholes_marker(mask), mask, conn, "erode"))
    return cases


def _run_batch(iw, cases, plan=None, schedule=None):
    items = [(torch.from_numpy(c.marker).cuda(), torch.from_numpy(c.mask).cuda(), c.conn, c.op) for c in cases]
    B = iw.Batch(items, plan)
    sched = schedule(B.ntiles) if schedule else {}
    rc = B(**sched)
    assert rc == 0, iw.STATUS.get(rc)
    st = B.status()
    assert st == 0, iw.STATUS.get(st)
    return [m.cpu().numpy() for m, _, _, _ in items], B, sched


def _check(oracle_lib, cases, outs):
    for i, (c, got) in enumerate(zip(cases, outs)):
        exp = oracle_lib.reconstruct(c.marker, c.mask, c.conn, c.op)
        if not np.array_equal(got, exp):
            bad = np.argwhere(got != exp)
            raise AssertionError(f"image {i} {c.mask.shape} {c.mask.dtype} conn {c.conn} {c.op}: "
                                 f"{len(bad)} mismatches, first at {tuple(bad[0])}")


@pytest.mark.parametrize("tile,solver,bps", [((32, 32), 0, 0), ((32, 64), 0, 0), ((64, 64), 0, 0),
                                             ((16, 32), 0, 0), ((16, 64), 0, 0), ((16, 64), 1, 0),
                                             ((16, 64), 1, 6), ((64, 64), 2, 0), ((64, 64), 2, 3)])
def test_mixed_batch_static(iw, oracle_lib, tile, solver, bps):
    cases = _mixed_cases(5, 24)
    p = iw.iwpp_default_batch_plan()
    p.tile_h, p.tile_w = tile
    p.local_solver = solver
    p.blocks_per_sm = bps
    outs, _, _ = _run_batch(iw, cases, p)
    _check(oracle_lib, cases, outs)


@pytest.mark.parametrize("solver,bps", [(0, 0), (1, 0), (1, 6), (2, 0), (2, 2)])
def test_uniform_batch_each_kind(iw, oracle_lib, solver, bps):
    """Batches whose images share pixel type and connectivity use the specialised kernels
    (the cooperative solver among them)."""
    p = iw.iwpp_default_batch_plan()
    p.tile_h, p.tile_w = {0: (32, 32), 1: (16, 64), 2: (64, 64)}[solver]
    p.local_solver = solver
    p.blocks_per_sm = bps
    for k, (dtype, conn) in enumerate([(np.uint8, 4), (np.uint16, 4), (np.uint8, 8), (np.uint16, 8)]):
        cases = []
        for i, (H, W) in enumerate([(77, 301), (256, 64), (19, 1000)]):
            field = synth.blob_field_u8(H, W, 6, synth.rng_for(95, 10 * k + i))
            mask = field if dtype == np.uint8 else synth.to_u16(field)
            if i % 2:
                cases.append(synth.Case(synth.fillholes_marker(mask), mask, conn, "erode"))
            else:
                cases.append(synth.Case(synth.hdome_marker(mask, 20 if dtype == np.uint8 else 5000), mask, conn,
                                        "dilate"))
        outs, _, _ = _run_batch(iw, cases, p)
        _check(oracle_lib, cases, outs)


def test_mixed_batch_random_schedule(iw, oracle_lib):
    cases = _mixed_cases(6, 30)

    def schedule(nt):
        g = torch.Generator().manual_seed(3)
        order = torch.randperm(nt, generator=g).to(torch.int32)
        order[: nt // 10] = order[nt // 10: 2 * (nt // 10)]          # repeated ids, some missing
        sweeps = torch.randint(0, 5, (nt,), generator=g, dtype=torch.uint8)
        work = torch.zeros(2 * nt, dtype=torch.int32)
        return {"order": order.cuda(), "sweeps": sweeps.cuda(), "work": work.cuda()}

    outs, B, sched = _run_batch(iw, cases, None, schedule)
    _check(oracle_lib, cases, outs)
    work = sched["work"].cpu().numpy().view(np.uint32)
    assert work[B.ntiles:].sum() > 0   # cycles recorded for the tiles


def test_coop_batch_with_schedule(iw, oracle_lib):
    """A uniform batch under the cooperative solver with an explicit tile order (repeated and
    missing ids) and per-tile sweep counts 0..4 (run by the cooperative scan kernel on whole
    64 x 64 tiles)."""
    cases = [synth.sparse_seed_case(700, 1100, nblobs=30, nseeds=6, image_idx=i) for i in range(3)]
    p = iw.iwpp_default_batch_plan()
    p.tile_h, p.tile_w, p.local_solver = 64, 64, 2

    def schedule(nt):
        g = torch.Generator().manual_seed(5)
        order = torch.randperm(nt, generator=g).to(torch.int32)
        order[: nt // 8] = order[nt // 8: 2 * (nt // 8)]
        sweeps = torch.randint(0, 5, (nt,), generator=g, dtype=torch.uint8)
        return {"order": order.cuda(), "sweeps": sweeps.cuda()}

    outs, _, _ = _run_batch(iw, cases, p, schedule)
    _check(oracle_lib, cases, outs)


def test_batch_rejects_value_levels(iw):
    """Value-ordered tile queues are a single-image option: a batch call refuses the plan."""
    cases = _mixed_cases(8, 2, max_side=300)
    p = iw.iwpp_default_batch_plan()
    p.value_levels = 4
    items = [(torch.from_numpy(c.marker).cuda(), torch.from_numpy(c.mask).cuda(), c.conn, c.op) for c in cases]
    B = iw.Batch(items)
    import ctypes
    assert iw.iwpp_reconstruct_batch(B.descs, p, ctypes.c_void_p(B.ws.data_ptr()), B.ws.numel(), None) == 1


def test_batch_of_one_matches_single(iw, oracle_lib):
    c = synth.tissue_case(700, 900, nblobs=40)
    outs, _, _ = _run_batch(iw, [c])
    _check(oracle_lib, [c], outs)


def test_batch_small_queue_overflow(iw, oracle_lib):
    cases = _mixed_cases(7, 8, max_side=400)
    p = iw.iwpp_default_batch_plan()
    p.smem_queue_cap = 16
    outs, _, _ = _run_batch(iw, cases, p)
    _check(oracle_lib, cases, outs)


def test_batch_precondition_reported(iw):
    mask = np.full((50, 70), 10, np.uint8)
    bad = np.zeros_like(mask)
    bad[3, 4] = 11
    good = synth.tissue_case(64, 64, nblobs=2)
    items = [(torch.from_numpy(good.marker).cuda(), torch.from_numpy(good.mask).cuda(), 8, "dilate"),
             (torch.from_numpy(bad).cuda(), torch.from_numpy(mask).cuda(), 8, "dilate")]
    B = iw.Batch(items)
    assert B() == 0
    assert B.status() == 2


def test_mixed_batch_full_size(iw, oracle_lib):
    """The 256-image uneven batch (log-uniform sides 256-4096, u8/u16, h-dome and
    fill-holes), checked image by image against the oracle."""
    cases = synth.mixed_batch()
    outs, _, _ = _run_batch(iw, cases)
    exps = oracle_lib.reconstruct_many([(c.marker, c.mask, c.conn, c.op) for c in cases])
    for i, (got, exp) in enumerate(zip(outs, exps)):
        assert np.array_equal(got, exp), f"image {i} differs"


def test_batch_graph_replays_bit_exact(iw, oracle_lib):
    cases = _mixed_cases(11, 16)
    items = [(torch.from_numpy(c.marker).cuda(), torch.from_numpy(c.mask).cuda(), c.conn, c.op) for c in cases]
    init = [m.clone() for m, _, _, _ in items]
    B = iw.Batch(items)
    g = B.graph()
    for _ in range(2):
        for (m, _, _, _), m0 in zip(items, init):
            m.copy_(m0)
        assert g.launch() == 0
        assert B.status() == 0
        _check(oracle_lib, cases, [m.cpu().numpy() for m, _, _, _ in items])


def test_batch_call_captures_in_torch_graph(iw, oracle_lib):
    cases = _mixed_cases(12, 6)
    items = [(torch.from_numpy(c.marker).cuda(), torch.from_numpy(c.mask).cuda(), c.conn, c.op) for c in cases]
    init = [m.clone() for m, _, _, _ in items]
    B = iw.Batch(items)
    assert B() == 0 and B.status() == 0          # warm-up outside capture
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            assert B(stream=s) == 0
    for (m, _, _, _), m0 in zip(items, init):
        m.copy_(m0)
    graph.replay()
    torch.cuda.synchronize()
    assert B.status() == 0
    _check(oracle_lib, cases, [m.cpu().numpy() for m, _, _, _ in items])


def test_autotune_restores_markers_and_caches(iw, oracle_lib, tmp_path):
    cases = _mixed_cases(13, 10, max_side=500)
    items = [(torch.from_numpy(c.marker).cuda(), torch.from_numpy(c.mask).cuda(), c.conn, c.op) for c in cases]
    B = iw.Batch(items)
    cache = str(tmp_path / "tune.txt")
    plan, ms = B.autotune(reps=1, cache_path=cache)
    assert ms > 0 and iw.iwpp_tile_shape_supported(plan.tile_h, plan.tile_w)
    for (m, _, _, _), c in zip(items, cases):
        assert np.array_equal(m.cpu().numpy(), c.marker)       # untouched by tuning
    assert B() == 0 and B.status() == 0
    _check(oracle_lib, cases, [m.cpu().numpy() for m, _, _, _ in items])
    # a second tuning of the same batch signature is a cache hit
    plan2, ms2 = iw.iwpp_autotune_batch(B.descs, iw.iwpp_default_batch_plan(), 1, cache)
    assert ms2 == 0.0 and plan2.as_dict()["tile_h"] == plan.tile_h and plan2.sweeps == plan.sweeps
