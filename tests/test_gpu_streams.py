"""Batch calls on concurrent streams, pipelined the way a caller streaming batches runs them
(and as the benchmark's end-to-end form does): each round copies the markers in from pinned
host memory on one stream, runs two independent batch calls (one with the learned schedule,
one static) on two other streams, and copies the results out on a fourth. The header's rule:
calls on different streams are safe when their workspaces and images differ. Every round's
output must be the oracle's, image by image."""
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


def _cases(seed, n, conns, max_side=300):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        H, W = int(rng.integers(1, max_side)), int(rng.integers(1, max_side))
        is16 = bool(rng.integers(0, 2))
        field = synth.blob_field_u8(H, W, max(1, H * W // 3000), rng)
        mask = synth.to_u16(field) if is16 else field
        conn = int(rng.choice(conns))
        if i % 2 == 0:
            h = int(rng.integers(5, 60)) * (257 if is16 else 1)
            out.append(synth.Case(synth.hdome_marker(mask, h), mask, conn, "dilate"))
        else:
            out.append(synth.Case(synth.fillholes_marker(mask), mask, conn, "erode"))
    return out


def test_batches_on_concurrent_streams_pipelined(iw, oracle_lib):
    from paper_1605_00930_gb300 import learned
    dev = torch.device("cuda", torch.cuda.current_device())
    # set 0: one connectivity (the learned call takes its features from the scan kernel);
    # set 1: both connectivities (the static call's mixed-kind kernels)
    sets = [_cases(31, 10, [8]), _cases(32, 9, [4, 8])]
    expected = [[oracle_lib.reconstruct(c.marker, c.mask, c.conn, c.op) for c in cs] for cs in sets]
    items = [[(torch.from_numpy(c.marker).to(dev), torch.from_numpy(c.mask).to(dev), c.conn, c.op) for c in cs]
             for cs in sets]
    host_in = [[torch.from_numpy(c.marker).pin_memory() for c in cs] for cs in sets]
    batches = [iw.Batch(items[0]), iw.Batch(items[1])]
    sch = learned.LearnedScheduler(learned.init_params(11), dev)
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    s_run = [torch.cuda.Stream(dev), torch.cuda.Stream(dev)]
    rounds = 3
    host_out = [[[torch.empty_like(h).pin_memory() for h in host_in[k]] for k in range(2)] for _ in range(rounds)]
    read_out = [None, None]   # per set: its last result copy has been issued (the next input copy waits)
    torch.cuda.synchronize()
    for r in range(rounds):
        for k in range(2):
            with torch.cuda.stream(s_in):
                if read_out[k] is not None:
                    s_in.wait_event(read_out[k])
                for (m, _, _, _), h in zip(items[k], host_in[k]):
                    m.copy_(h, non_blocking=True)
                loaded = torch.cuda.Event()
                loaded.record(s_in)
            s_run[k].wait_event(loaded)
            rc = sch.reconstruct(batches[k], s_run[k]) if k == 0 else batches[k](stream=s_run[k])
            assert rc == 0, iw.STATUS.get(rc)
            done = torch.cuda.Event()
            done.record(s_run[k])
            with torch.cuda.stream(s_out):
                s_out.wait_event(done)
                for (m, _, _, _), h in zip(items[k], host_out[r][k]):
                    h.copy_(m, non_blocking=True)
                read_out[k] = torch.cuda.Event()
                read_out[k].record(s_out)
    torch.cuda.synchronize()
    for k in range(2):
        st = batches[k].status(s_run[k])
        assert st == 0, iw.STATUS.get(st)
    for r in range(rounds):
        for k in range(2):
            for i, (got, exp) in enumerate(zip(host_out[r][k], expected[k])):
                assert np.array_equal(got.numpy(), exp), f"round {r} set {k} image {i}"
