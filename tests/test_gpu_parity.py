"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, bit-exact.

Reconstruction output is integer; the only acceptable difference is none. Sizes
span several tiles with ragged tails, every tile shape and plan knob, both dtypes,
both operators and both connectivities, plus the full-size workloads."""
import ctypes

import numpy as np
import pytest

from paper_1605_00930_gb300 import synth
from tests._golden import load_hand_cases

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


def _tdtype(np_dtype):
    return torch.uint8 if np.dtype(np_dtype) == np.uint8 else torch.uint16


def gpu_run(iw, marker, mask, conn, op, plan=None, expect_status=0):
    dt = _tdtype(marker.dtype)
    m = torch.from_numpy(np.ascontiguousarray(marker)).cuda()
    I = torch.from_numpy(np.ascontiguousarray(mask)).cuda()
    R = iw.Reconstructor(marker.shape[0], marker.shape[1], dt, plan)
    rc = R(m, I, conn, op)
    assert rc == 0, iw.STATUS.get(rc)
    st = R.status()
    assert st == expect_status, iw.STATUS.get(st)
    return m.cpu().numpy(), R


def check(iw, oracle_lib, marker, mask, conn, op, plan=None):
    exp = oracle_lib.reconstruct(marker, mask, conn, op)
    got, _ = gpu_run(iw, marker, mask, conn, op, plan)
    if not np.array_equal(got, exp):
        bad = np.argwhere(got != exp)
        y, x = bad[0]
        raise AssertionError(f"{len(bad)} mismatches, first at {(y, x)}: got {got[y, x]} "
                             f"expected {exp[y, x]} (shape {mask.shape}, conn {conn}, op {op})")


def _plan(iw, **kw):
    p = iw.iwpp_default_plan()
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _random_pair(rng, H, W, dtype, op, vmax):
    top = synth.maxval(dtype)
    mask = rng.integers(0, vmax + 1, size=(H, W)).astype(dtype)
    if op == "dilate":
        marker = (mask.astype(np.int64) * (rng.random((H, W)) < 0.05)).astype(dtype)
    else:
        marker = synth.fillholes_marker(mask)
    return marker, mask


SHAPES = [(1, 1), (1, 700), (700, 1), (32, 32), (64, 64), (65, 130), (129, 65), (200, 333), (257, 513)]


# The local solvers of the persistent kernel, each on a tile shape it supports.
SOLVERS = {"queue": dict(local_solver=0, tile_h=32, tile_w=32),
           "register": dict(local_solver=1, tile_h=16, tile_w=64),
           "coop": dict(local_solver=2, tile_h=64, tile_w=64)}


@pytest.mark.parametrize("solver", sorted(SOLVERS))
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
@pytest.mark.parametrize("op", ["dilate", "erode"])
@pytest.mark.parametrize("conn", [4, 8])
def test_random_small(iw, oracle_lib, shape, dtype, op, conn, solver):
    rng = np.random.default_rng([101, shape[0], shape[1], conn, op == "erode"])
    p = _plan(iw, **SOLVERS[solver])
    for vmax in (7, synth.maxval(dtype)):
        marker, mask = _random_pair(rng, *shape, dtype, op, vmax)
        check(iw, oracle_lib, marker, mask, conn, op, p)


# Widths around the 64-column register tiles and strips and their 2-pixel pairs (odd widths read the
# rows that start on an odd element as shifted pairs recombined across lanes; the narrowest widths
# and partial tiles mask columns), heights around its 16 rows.
EDGE_SHAPES = [(15, 63), (16, 64), (17, 65), (33, 127), (31, 128), (16, 129), (2, 2), (3, 1), (1, 3),
               (130, 5), (18, 3), (67, 191), (100, 255), (49, 257)]


@pytest.mark.parametrize("solver", ["register", "coop"])
@pytest.mark.parametrize("shape", EDGE_SHAPES + [(63, 65), (64, 64), (65, 130), (129, 63)])
@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
@pytest.mark.parametrize("op", ["dilate", "erode"])
def test_strip_solver_edges(iw, oracle_lib, shape, dtype, op, solver):
    rng = np.random.default_rng([102, shape[0], shape[1], op == "erode"])
    p = _plan(iw, **SOLVERS[solver])
    for conn in (4, 8):
        for vmax in (3, synth.maxval(dtype)):
            marker, mask = _random_pair(rng, *shape, dtype, op, vmax)
            check(iw, oracle_lib, marker, mask, conn, op, p)


@pytest.mark.parametrize("case", load_hand_cases(), ids=lambda c: c["name"])
def test_hand_cases_gpu(iw, case):
    for conn in case["conn"]:
        got, _ = gpu_run(iw, case["marker"], case["mask"], conn, case["op"])
        np.testing.assert_array_equal(got, case["expected"])


@pytest.mark.parametrize("tile", [(32, 32), (32, 64), (64, 64), (16, 32), (16, 64)])
@pytest.mark.parametrize("sweeps", [0, 1, 3])
@pytest.mark.parametrize("qcap", [16, 1024])
def test_plans_tissue(iw, oracle_lib, tile, sweeps, qcap):
    c = synth.tissue_case(301, 517, nblobs=30)
    p = _plan(iw, tile_h=tile[0], tile_w=tile[1], sweeps=sweeps, smem_queue_cap=min(qcap, tile[0] * tile[1]),
              local_solver=0)
    for conn in (4, 8):
        check(iw, oracle_lib, c.marker, c.mask, conn, "dilate", p)


@pytest.mark.parametrize("sweeps", [0, 1, 3])
@pytest.mark.parametrize("bps", [0, 1, 5, 6])
def test_plans_tissue_register(iw, oracle_lib, sweeps, bps):
    c = synth.tissue_case(301, 517, nblobs=30)
    p = _plan(iw, sweeps=sweeps, blocks_per_sm=bps, **SOLVERS["register"])
    for conn in (4, 8):
        check(iw, oracle_lib, c.marker, c.mask, conn, "dilate", p)


@pytest.mark.parametrize("levels", [2, 8, 16])
@pytest.mark.parametrize("bps", [0, 6])
def test_value_ordered_queue(iw, oracle_lib, levels, bps):
    """Tile queues by value level (highest level first) reach the same fixed point."""
    p = _plan(iw, value_levels=levels, blocks_per_sm=bps, **SOLVERS["register"])
    c = synth.tissue_case(517, 700, nblobs=40)
    for conn in (4, 8):
        check(iw, oracle_lib, c.marker, c.mask, conn, "dilate", p)
    field = synth.blob_field_u8(300, 451, 20, synth.rng_for(91, levels))
    mask = synth.to_u16(field)
    check(iw, oracle_lib, synth.fillholes_marker(mask), mask, 8, "erode", p)
    check(iw, oracle_lib, synth.fillholes_marker(field), field, 4, "erode", p)
    s = synth.sparse_seed_case(1024, 1536, nblobs=60, nseeds=12)
    check(iw, oracle_lib, s.marker, s.mask, 8, "dilate", p)


@pytest.mark.parametrize("solver", ["queue", "register"])
@pytest.mark.parametrize("revisit", [0, 2])
@pytest.mark.parametrize("bps", [0, 1])
def test_plans_fill_holes_u16(iw, oracle_lib, revisit, bps, solver):
    field = synth.blob_field_u8(390, 271, 25, synth.rng_for(90))
    mask = synth.to_u16(field)
    p = _plan(iw, revisit_sweeps=revisit, blocks_per_sm=bps, sweeps=0, **SOLVERS[solver])
    check(iw, oracle_lib, synth.fillholes_marker(mask), mask, 8, "erode", p)


def test_noise_blur_512(iw, oracle_lib):
    c = synth.noise_blur_case()
    check(iw, oracle_lib, c.marker, c.mask, c.conn, c.op)


@pytest.mark.parametrize("solver", [None, "queue", "register", "coop"])
@pytest.mark.parametrize("conn", [4, 8])
def test_tissue_4096(iw, oracle_lib, conn, solver):
    c = synth.tissue_case(conn=conn)
    p = _plan(iw, **SOLVERS[solver]) if solver else None
    check(iw, oracle_lib, c.marker, c.mask, conn, "dilate", p)


@pytest.mark.parametrize("solver", [None, "coop"])
def test_sparse_seeds_16384(iw, oracle_lib, solver):
    c = synth.sparse_seed_case()
    check(iw, oracle_lib, c.marker, c.mask, 8, "dilate", _plan(iw, **SOLVERS[solver]) if solver else None)


@pytest.mark.parametrize("bps", [0, 1, 3])
def test_coop_fill_holes_u16(iw, oracle_lib, bps):
    """The cooperative solver on the critical-path-bound workload: u16 fill-holes."""
    field = synth.blob_field_u8(1000, 1300, 80, synth.rng_for(94))
    mask = synth.to_u16(field)
    p = _plan(iw, blocks_per_sm=bps, **SOLVERS["coop"])
    for conn in (4, 8):
        check(iw, oracle_lib, synth.fillholes_marker(mask), mask, conn, "erode", p)


@pytest.mark.parametrize("conn", [8])
def test_image_beyond_2_32_pixels(iw, oracle_lib, conn):
    """A 65664 x 65664 u8 image (4.3 G pixels, more than 2^32): 128 x 128 copies of a
    tissue crop, each followed by a zero-mask gutter row and column, so no value can cross
    from one copy to another and the result must be the oracle's result for one copy,
    repeated. Exercises 64-bit pixel offsets everywhere on the path."""
    c = synth.tissue_case(512, 512, nblobs=8)
    mk = np.zeros((513, 513), np.uint8)
    ms = np.zeros((513, 513), np.uint8)
    mk[:512, :512] = c.marker
    ms[:512, :512] = c.mask
    exp = oracle_lib.reconstruct(mk, ms, conn, "dilate")
    reps = 128
    M = torch.from_numpy(mk).cuda().repeat(reps, reps)
    I = torch.from_numpy(ms).cuda().repeat(reps, reps)
    H, W = M.shape
    assert H * W > 2 ** 32
    R = iw.Reconstructor(H, W, torch.uint8)
    assert R(M, I, conn, "dilate") == 0
    assert R.status() == 0
    del I, R
    E = torch.from_numpy(exp).cuda()
    assert torch.equal(M.view(reps, 513, reps, 513), E[None, :, None, :].expand(reps, 513, reps, 513))


def test_repeatable_output(iw, oracle_lib):
    c = synth.tissue_case(777, 1031, nblobs=60)
    exp = oracle_lib.reconstruct(c.marker, c.mask, 8, "dilate")
    for _ in range(10):
        got, _ = gpu_run(iw, c.marker, c.mask, 8, "dilate")
        np.testing.assert_array_equal(got, exp)


@pytest.mark.parametrize("solver", sorted(SOLVERS))
def test_precondition_violation_reported(iw, solver):
    p = _plan(iw, **SOLVERS[solver])
    mask = np.full((70, 90), 10, np.uint8)
    marker = np.zeros_like(mask)
    marker[33, 44] = 11
    gpu_run(iw, marker, mask, 8, "dilate", p, expect_status=2)
    up = np.full_like(mask, 10)
    up[5, 6] = 9
    gpu_run(iw, up, mask, 8, "erode", p, expect_status=2)


def test_workspace_too_small(iw):
    m = torch.zeros((100, 100), dtype=torch.uint8, device="cuda")
    need = iw.iwpp_workspace_bytes(100, 100, 0)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    P = ctypes.c_void_p
    assert iw.iwpp_reconstruct(P(m.data_ptr()), P(m.data_ptr()), 100, 100, 8, 0, 0, P(ws.data_ptr()),
                               need - 1, s) == 3
    assert iw.iwpp_reconstruct(P(m.data_ptr()), P(m.data_ptr()), 100, 100, 8, 0, 0, P(ws.data_ptr()),
                               need, s) == 0
    assert iw.iwpp_sync_status(P(ws.data_ptr()), s) == 0


@pytest.mark.parametrize("solver", ["register", "queue", "coop"])
def test_watchdog_timeout_returns_and_workspace_recovers(iw, oracle_lib, solver):
    """A 1 ns watchdog makes an idle CTA's wait for work run out: the kernel records
    IWPP_ERR_TIMEOUT and returns (no hang, no trap); the same workspace then serves a
    normal call. Both local solvers share the queue protocol; both are exercised."""
    c = synth.tissue_case(256, 1024, nblobs=40)
    p = _plan(iw, watchdog_ns=1, sweeps=0, blocks_per_sm=1, **SOLVERS[solver])
    dt = torch.uint8
    seen = set()
    R = iw.Reconstructor(256, 1024, dt, p)
    R.plan = p
    for _ in range(5):
        m = torch.from_numpy(c.marker).cuda()
        I = torch.from_numpy(c.mask).cuda()
        assert R(m, I, 8, "dilate") == 0
        seen.add(R.status())
        if 5 in seen:
            break
    assert 5 in seen, seen
    torch.cuda.synchronize()
    R.plan = _plan(iw, **SOLVERS[solver])
    m = torch.from_numpy(c.marker).cuda()
    I = torch.from_numpy(c.mask).cuda()
    assert R(m, I, 8, "dilate") == 0
    assert R.status() == 0
    np.testing.assert_array_equal(m.cpu().numpy(), oracle_lib.reconstruct(c.marker, c.mask, 8, "dilate"))


def test_work_counters(iw):
    c = synth.tissue_case(512, 512, nblobs=20)
    _, R = gpu_run(iw, c.marker, c.mask, 8, "dilate")
    cnt = R.counters()
    assert cnt["visits"] >= 1 and cnt["pops"] >= cnt["seeds"] >= 0


def test_coop_drain_counters(iw):
    """The cooperative drain's counters (kept per CTA in shared memory, flushed at the end):
    each counted visit starts with its four strips unsettled, and an unsettled strip runs a
    down and an up pass, so the passes summed over the strips are at least 8 per visit; the
    processing time is positive and the waiting time not negative."""
    assert iw.iwpp_default_plan().local_solver == iw.IWPP_SOLVER_COOP
    c = synth.tissue_case(512, 512, nblobs=20)
    _, R = gpu_run(iw, c.marker, c.mask, 8, "dilate")
    cnt = R.counters()
    assert cnt["visits"] >= 1
    assert cnt["waves"] >= 8 * cnt["visits"], cnt
    assert cnt["busy_ns"] > 0 and cnt["idle_ns"] >= 0, cnt
