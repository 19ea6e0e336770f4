"""GPU parity of the learned schedule: feature kernel and MLP kernels against the
float64 oracle; schedule validity; and the learned-scheduled batch bit-exact."""
import numpy as np
import pytest

from oracle import features as ofeat
from oracle import mlp as omlp
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


def _cases(seed, n, side=260):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        H, W = int(rng.integers(1, side)), int(rng.integers(1, side))
        is16 = bool(rng.integers(0, 2))
        f = synth.blob_field_u8(H, W, max(1, H * W // 2500), rng)
        mask = synth.to_u16(f) if is16 else f
        if i % 2 == 0:
            out.append(synth.Case(synth.hdome_marker(mask, int(rng.integers(5, 50)) * (257 if is16 else 1)), mask,
                                  8, "dilate"))
        else:
            out.append(synth.Case(synth.fillholes_marker(mask), mask, 4, "erode"))
    return out


def _items(cases):
    return [(torch.from_numpy(c.marker).cuda(), torch.from_numpy(c.mask).cuda(), c.conn, c.op) for c in cases]


def test_features_match_oracle(iw):
    from paper_1605_00930_gb300 import learned
    cases = _cases(21, 9)
    got = learned.features(_items(cases)).cpu().numpy()
    exp = ofeat.batch_features(cases)
    assert got.shape == exp.shape
    # counts are exact integers; moments are rounded once to float32
    np.testing.assert_allclose(got, exp, rtol=1e-6, atol=1e-7)


@pytest.mark.parametrize("shape", [(128, 192), (130, 256), (64, 80), (200, 320)])
@pytest.mark.parametrize("is16", [False, True])
def test_features_vector_path_matches_oracle(iw, shape, is16):
    """Whole 64 x 64 blocks with 16-byte row pitch take the vectorised path; ragged edge
    blocks (and rows that are not 16-byte multiples) the scalar one. Both are exact."""
    from paper_1605_00930_gb300 import learned
    rng = synth.rng_for(97, shape[0] * 1000 + shape[1] + is16)
    f = synth.blob_field_u8(*shape, 12, rng)
    mask = synth.to_u16(f) if is16 else f
    cases = [synth.Case(synth.hdome_marker(mask, 20 * (257 if is16 else 1)), mask, 8, "dilate"),
             synth.Case(synth.fillholes_marker(mask), mask, 8, "erode")]
    got = learned.features(_items(cases)).cpu().numpy()
    exp = ofeat.batch_features(cases)
    np.testing.assert_allclose(got, exp, rtol=1e-6, atol=1e-7)


def test_mlp_forward_matches_oracle(iw):
    rng = np.random.default_rng(2)
    p = omlp.init_params(4).astype(np.float32)
    X = rng.random((1000, 16)).astype(np.float32)
    Y = torch.empty((1000, 2), dtype=torch.float32, device="cuda")
    iw.iwpp_mlp_forward(torch.from_numpy(p).cuda(), torch.from_numpy(X).cuda(), Y)
    exp = omlp.forward(p.astype(np.float64), X.astype(np.float64))
    # fp32 sums of <= 64 products of O(1) terms
    np.testing.assert_allclose(Y.cpu().numpy(), exp, rtol=1e-4, atol=1e-4)


def test_mlp_gradient_matches_oracle(iw):
    """One full-batch Adam step with lr = 0 leaves m = (1 - beta1) * gradient."""
    rng = np.random.default_rng(3)
    p = omlp.init_params(5).astype(np.float32)
    X = rng.random((700, 16)).astype(np.float32)
    T = rng.normal(size=(700, 2)).astype(np.float32)
    dp = torch.from_numpy(p).cuda()
    m = torch.zeros(iw.MLP_PARAMS, device="cuda")
    v = torch.zeros_like(m)
    g = torch.zeros_like(m)
    iw.iwpp_mlp_train(dp, m, v, g, torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(), 1, 700, 0.0, 1.0, 0.5)
    got = m.cpu().numpy() / 0.1
    exp = omlp.grad(p.astype(np.float64), X.astype(np.float64), T.astype(np.float64), (1.0, 0.5))
    np.testing.assert_allclose(got, exp, rtol=2e-3, atol=2e-5 * np.abs(exp).max())
    assert np.array_equal(dp.cpu().numpy(), p)          # lr = 0: parameters unchanged
    assert np.all(g.cpu().numpy() == 0)                  # gradient consumed


def test_training_reduces_loss(iw):
    rng = np.random.default_rng(4)
    X = rng.random((4000, 16)).astype(np.float32)
    T = np.stack([3 * X[:, 0] + X[:, 5], np.round(4 * X[:, 2])], 1).astype(np.float32)
    from paper_1605_00930_gb300 import learned
    s = learned.LearnedScheduler(learned.init_params(1))
    p0 = s.params.cpu().numpy().astype(np.float64)
    s.train(X, T, epochs=20, batch=256, lr=3e-3, w=(1.0, 1.0))
    p1 = s.params.cpu().numpy().astype(np.float64)
    assert omlp.loss(p1, X, T) < 0.2 * omlp.loss(p0, X, T)


def test_schedule_is_a_largest_first_permutation(iw):
    cases = _cases(22, 7)
    items = _items(cases)
    B = iw.Batch(items)
    nb = iw.iwpp_batch_block_count(B.descs)
    rng = np.random.default_rng(9)
    preds = np.stack([rng.uniform(0, 12, nb), rng.uniform(-2, 11, nb)], 1).astype(np.float32)
    sws = iw.alloc_workspace(iw.iwpp_sched_workspace_bytes(B.descs))
    order = torch.empty(B.ntiles, dtype=torch.int32, device="cuda")
    sweeps = torch.empty(B.ntiles, dtype=torch.uint8, device="cuda")
    iw.iwpp_schedule_from_predictions(B.descs, None, torch.from_numpy(preds).cuda(), order, sweeps, sws)
    o = order.cpu().numpy()
    assert np.array_equal(np.sort(o), np.arange(B.ntiles))
    # tile -> block map (the default batch plan's tiles inside 64 x 64 blocks), image by image
    plan = iw.iwpp_default_batch_plan()
    th, tw = plan.tile_h, plan.tile_w
    blk = []
    bbase = 0
    for c in cases:
        H, W = c.mask.shape
        tx, ty = (W + tw - 1) // tw, (H + th - 1) // th
        nbx = (W + 63) // 64
        for t in range(tx * ty):
            blk.append(bbase + ((t // tx) * th) // 64 * nbx + ((t % tx) * tw) // 64)
        bbase += nbx * ((H + 63) // 64)
    blk = np.array(blk)
    keys = np.clip((preds[blk, 0] * 64).astype(np.int64), 0, 1023)
    assert np.all(np.diff(keys[o]) <= 0)
    np.testing.assert_array_equal(sweeps.cpu().numpy(), np.clip(np.rint(preds[blk, 1]), 0, 8))


def test_learned_batch_is_bit_exact(iw, oracle_lib):
    from paper_1605_00930_gb300 import learned
    cases = _cases(23, 12, side=400)
    items = _items(cases)
    sch = learned.LearnedScheduler(learned.init_params(3))
    B = iw.Batch(items)
    order, sweeps = sch.schedule(B)
    assert B(order=order, sweeps=sweeps) == 0
    assert B.status() == 0
    for c, (m, _, _, _) in zip(cases, items):
        assert np.array_equal(m.cpu().numpy(), oracle_lib.reconstruct(c.marker, c.mask, c.conn, c.op))


def test_block_labels_and_roundtrip(iw, tmp_path):
    from paper_1605_00930_gb300 import learned
    cases = _cases(24, 4, side=300)
    items = _items(cases)
    lw, best, cyc = learned.block_labels(items)
    assert lw.shape == best.shape and np.all(lw >= 0) and set(np.unique(best)) <= set(learned.SWEEP_OPTIONS)
    for (m, _, _, _), c in zip(items, cases):
        assert np.array_equal(m.cpu().numpy(), c.marker)   # markers restored
    s = learned.LearnedScheduler(learned.init_params(2), meta={"note": "t"})
    s.save(str(tmp_path / "w.bin"))
    s2 = learned.LearnedScheduler.load(str(tmp_path / "w.bin"))
    assert s2 is not None and torch.equal(s.params, s2.params)
    (tmp_path / "w.bin").write_bytes(b"junk")
    assert learned.LearnedScheduler.load(str(tmp_path / "w.bin")) is None


def _mixed8_cases(seed, n, side=300):
    """u8 and u16 images of one connectivity (8): the batch kernel that reads the pixel size per
    image; h-dome dilations and fill-holes; ragged sizes (partial 64 x 64 tiles)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        H, W = int(rng.integers(1, side)), int(rng.integers(1, side))
        is16 = bool(rng.integers(0, 2))
        f = synth.blob_field_u8(H, W, max(1, H * W // 2500), rng)
        mask = synth.to_u16(f) if is16 else f
        if i % 2 == 0:
            out.append(synth.Case(synth.hdome_marker(mask, int(rng.integers(5, 50)) * (257 if is16 else 1)), mask,
                                  8, "dilate"))
        else:
            out.append(synth.Case(synth.fillholes_marker(mask), mask, 8, "erode"))
    return out


def _strip_edge_cases():
    """Heights that end a tile after one, two or three 16-row strips (whole strips at the
    image's bottom edge) and widths that are multiples of 64, u8 and u16, both operators."""
    out = []
    for i, (H, W) in enumerate([(80, 128), (144, 192), (16, 64), (48, 320), (112, 64), (96, 256)]):
        f = synth.blob_field_u8(H, W, 4, synth.rng_for(97, i))
        mask = synth.to_u16(f) if i % 2 else f
        if i % 3 == 2:
            out.append(synth.Case(synth.fillholes_marker(mask), mask, 8, "erode"))
        else:
            out.append(synth.Case(synth.hdome_marker(mask, 3000 if i % 2 else 12), mask, 8, "dilate"))
    return out


@pytest.mark.parametrize("kind", ["mixed8", "mixed_conn", "u8", "strip_edges"])
def test_learned_batch_call_bit_exact_and_features(iw, oracle_lib, kind):
    """iwpp_reconstruct_batch_learned: the schedule made inside the call (features from the scan
    kernel for one connectivity; a features pass first when connectivities are mixed) gives
    the oracle's result image by image, and the features it wrote equal the float64 oracle's."""
    from paper_1605_00930_gb300 import learned
    if kind == "mixed8":
        cases = _mixed8_cases(41, 14)
    elif kind == "mixed_conn":
        cases = _cases(42, 10, side=300)
    elif kind == "u8":
        cases = [synth.tissue_case(200 + 37 * i, 150 + 53 * i, nblobs=8, image_idx=i) for i in range(5)]
    else:
        cases = _strip_edge_cases()
    items = _items(cases)
    sch = learned.LearnedScheduler(learned.init_params(5))
    B = iw.Batch(items)
    assert sch.reconstruct(B) == 0
    assert B.status() == 0
    for i, (c, (m, _, _, _)) in enumerate(zip(cases, items)):
        assert np.array_equal(m.cpu().numpy(), oracle_lib.reconstruct(c.marker, c.mask, c.conn, c.op)), i
    got = sch.features_of(B).cpu().numpy()
    np.testing.assert_allclose(got, ofeat.batch_features(cases), rtol=1e-6, atol=1e-7)
    o = B._order.cpu().numpy()
    assert np.array_equal(np.sort(o), np.arange(B.ntiles))


def test_learned_batch_call_phases_and_sweeps(iw, oracle_lib):
    """The call split into its two phases (prepare + scan + schedule, then the drain) gives the
    whole call's result; with an MLP whose sweep output is large every tile runs sweep pairs in
    the sweeps-only pass, bit-exact as well."""
    from paper_1605_00930_gb300 import learned
    cases = _mixed8_cases(43, 10)
    p = learned.init_params(6)
    n1 = 16 * 64 + 64 + 64 * 64 + 64        # offset of the last layer's weights [64][2]
    p[n1 + 1:n1 + 128:2] = 0.0              # output 1 (sweep count) ignores the hidden layer ...
    p[-1] = 3.0                             # ... and is 3 pairs for every tile
    sch = learned.LearnedScheduler(p)
    items = _items(cases)
    B = iw.Batch(items)
    assert sch.reconstruct(B, phases=1) == 0
    assert sch.reconstruct(B, phases=2) == 0
    assert B.status() == 0
    assert np.all(B._sweeps.cpu().numpy() == 3)
    for i, (c, (m, _, _, _)) in enumerate(zip(cases, items)):
        assert np.array_equal(m.cpu().numpy(), oracle_lib.reconstruct(c.marker, c.mask, c.conn, c.op)), i


def test_full_512_image_learned_batch_matches_oracle(iw):
    """The 512-image uneven batch (the learned schedule's test batch: sides log-uniform in
    256..4096, u8/u16, h-dome dilations and fill-holes) reconstructed with a schedule from an
    estimator trained on labels of the 512^2, 4096^2 (conn 8 and 4) and 16384^2 workloads,
    then checked image by image against the oracle on the host's cores."""
    import os
    import oracle
    from paper_1605_00930_gb300 import learned
    oracle.build()
    cores = len(os.sched_getaffinity(0))
    c2 = synth.tissue_case()
    sets = [[synth.noise_blur_case()], [c2], [synth.Case(c2.marker, c2.mask, 4, "dilate")],
            [synth.sparse_seed_case()]]
    sch, report = learned.train_from_workloads([_items(s) for s in sets], n_samples=50000, epochs=60)
    assert report["mae_logwork"] <= report["mae_logwork_const"]
    del sets
    cases = synth.mixed_batch(512, workload_id=5, workers=min(16, cores))
    items = _items(cases)
    B = iw.Batch(items)
    order, sweeps = sch.schedule(B)
    assert B(order=order, sweeps=sweeps) == 0
    assert B.status() == 0
    outs = [m.cpu().numpy() for m, _, _, _ in items]
    del items, B
    exps = oracle.reconstruct_many([(c.marker, c.mask, c.conn, c.op) for c in cases], threads=cores)
    for i, (got, exp) in enumerate(zip(outs, exps)):
        assert np.array_equal(got, exp), f"image {i} {cases[i].mask.shape} {cases[i].mask.dtype} {cases[i].op} differs"
