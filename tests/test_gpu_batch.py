"""Batched and served imaging on the GPU: the same volume alone, in a batch,
from a replayed CUDA graph and from the continuous-batching server."""
import numpy as np
import pytest

import synth
from oracle import rma

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def small_mix(n=6):
    """Uneven scans shaped like the batched mix, scaled down for the test."""
    out = []
    for i in range(n):
        rng = np.random.default_rng(100 + i)
        npx, npy = int(rng.choice([6, 8, 10, 12])), int(rng.choice([6, 9, 12]))
        nk = int(rng.choice([16, 32, 48]))
        nx = 1 << int(np.ceil(np.log2(2 * npx + 8)))
        out.append(synth.custom(nx_pos=npx, ny_pos=npy, nk=nk, layout="awr1443", nx=nx, ny=nx, nz=8 + 2 * i,
                                seed=100 + i, serp=True, jitter=(1e-3, 2e-3), n_points=3))
    return out


def test_batch_equals_single(dev):
    from paper_2305_02064_gb300.batch import ScanJob, image_batch
    scans = small_mix()
    single = []
    for s in scans:
        j = ScanJob(s, dev)
        j.image()
        single.append(j.vol.cpu().numpy())
    jobs = [ScanJob(s, dev) for s in scans]
    streams = [torch.cuda.Stream(device=dev) for _ in range(3)]
    for st in streams:
        st.wait_stream(torch.cuda.current_stream())
    image_batch(jobs, streams)
    torch.cuda.synchronize()
    for j, ref, s in zip(jobs, single, scans):
        got = j.vol.cpu().numpy()
        assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
        assert rma.nmse(got, rma.rma_exact(rma.setup_from(s))) <= 2e-5


def test_fused_batch_equals_single(dev):
    """One fused launch per stage and kernel shape reproduces every scan's
    own image bit for bit: uneven shapes, FP32 and FP16 echoes, different
    gridding launch shapes and the grouped form in one batch."""
    from paper_2305_02064_gb300.batch import ScanJob, image_batch_fused
    scans = small_mix(8)
    jobs = [ScanJob(s, dev, dtype="f16" if i % 3 == 2 else "c64") for i, s in enumerate(scans)]
    shapes = [(2, 4, 0, 2), (1, 8, 0), (2, 8, 1), (2, 4, 0, 5), (4, 4, 0), (2, 4, 0, 3), (4, 8, 0)]
    for i, j in enumerate(jobs):
        j.plan.set_tiles(*shapes[i % len(shapes)])
    single = []
    for j in jobs:
        j.image()
        single.append(j.vol.cpu().numpy())
        j.vol.fill_(0)
    n = image_batch_fused(jobs)
    torch.cuda.synchronize()
    assert 0 < n < 10 * len(jobs)
    for j, ref in zip(jobs, single):
        assert np.array_equal(j.vol.cpu().numpy().view(np.uint32), ref.view(np.uint32))
        j.plan.poll_error(j.ws)


def test_fused_batch_beyond_one_table(dev):
    """More scans than one fused launch takes (32): the groups split into
    several launches, the images stay bit-identical."""
    from paper_2305_02064_gb300.batch import ScanJob, image_batch_fused
    scans = [small_mix(1)[0]] * 20 + small_mix(20)
    jobs = [ScanJob(s, dev) for s in scans]
    single = []
    for j in jobs:
        j.image()
        single.append(j.vol.cpu().numpy())
        j.vol.fill_(0)
    image_batch_fused(jobs)
    torch.cuda.synchronize()
    for j, ref in zip(jobs, single):
        assert np.array_equal(j.vol.cpu().numpy().view(np.uint32), ref.view(np.uint32))


def test_fused_batch_with_empty_and_single_sample_scans(dev):
    """A scan without samples gets a zero volume (and no fused launch), a
    one-position scan its own image, next to ordinary scans in one batch."""
    from paper_2305_02064_gb300.batch import ScanJob, image_batch_fused
    empty = synth.custom(nx_pos=0, ny_pos=0, nk=8, nx=8, ny=8, nz=4, seed=1)
    single = synth.custom(nx_pos=1, ny_pos=1, nk=16, layout="tiny", nx=16, ny=16, nz=8, seed=2,
                          scatterers=[[0.0, 0.0, 0.28, 1.0]])
    scans = [empty, single] + small_mix(3)
    jobs = [ScanJob(s, dev) for s in scans]
    ref = []
    for j in jobs:
        j.image()
        ref.append(j.vol.cpu().numpy())
        j.vol.fill_(1.0)
    image_batch_fused(jobs)
    torch.cuda.synchronize()
    assert np.all(jobs[0].vol.cpu().numpy() == 0)
    for j, r in zip(jobs[1:], ref[1:]):
        assert np.array_equal(j.vol.cpu().numpy().view(np.uint32), r.view(np.uint32))


def test_fused_graph_replay_equals_eager(dev):
    from paper_2305_02064_gb300.batch import BatchGraph, ScanJob
    scans = small_mix(5)
    jobs = [ScanJob(s, dev) for s in scans]
    g = BatchGraph(jobs, fused=True)
    eager = [j.vol.clone() for j in jobs]
    for j in jobs:
        j.vol.fill_(0)
    g.replay()
    torch.cuda.synchronize()
    assert 0 < g.launches < 10 * len(jobs)
    for j, e in zip(jobs, eager):
        assert torch.equal(j.vol.view(torch.float32), e.view(torch.float32))


def test_graph_replay_equals_eager(dev):
    from paper_2305_02064_gb300.batch import BatchGraph, ScanJob
    scans = small_mix(4)
    jobs = [ScanJob(s, dev) for s in scans]
    g = BatchGraph(jobs, n_streams=2)
    eager = [j.vol.clone() for j in jobs]
    for j in jobs:
        j.vol.fill_(0)
    g.replay()
    torch.cuda.synchronize()
    for j, e in zip(jobs, eager):
        assert torch.equal(j.vol.view(torch.float32), e.view(torch.float32))


@pytest.mark.parametrize("dtype", ["c64", "f16"])
def test_server_alone_and_in_the_mix(dev, dtype):
    """Served requests give the same volume alone and in the mix.  The
    device arena holds fewer requests than there are slots (the cap is under
    slots x the largest footprint), so admission queues on memory; nothing
    is allocated on the device while serving."""
    from paper_2305_02064_gb300.serve import GpuExecutor, Scheduler, ServeRequest, latency_summary
    scans = small_mix(8)
    probe = GpuExecutor(dev, dtype=dtype, n_streams=1, mem_cap=1 << 20)
    biggest = max(probe.footprint(s) for s in scans)
    del probe
    ex_alone = GpuExecutor(dev, dtype=dtype, n_streams=1, keep_results=True, mem_cap=biggest)
    alone = {}
    for i, s in enumerate(scans):
        r = ServeRequest(i, s, 0.0, footprint=ex_alone.footprint(s))
        Scheduler(ex_alone, slots=1, mem_cap=biggest).run([r])
        alone[i] = r.result.numpy()
    cap = 2 * biggest + biggest // 2
    ex = GpuExecutor(dev, dtype=dtype, n_streams=4, keep_results=True, mem_cap=cap)
    reqs = [ServeRequest(i, s, 0.0, footprint=ex.footprint(s)) for i, s in enumerate(scans)]
    for r in reqs:
        ex.pin(r)
    torch.cuda.synchronize()
    alloc0 = torch.cuda.memory_allocated()
    torch.cuda.reset_peak_memory_stats()
    sch = Scheduler(ex, slots=4, mem_cap=cap)
    done = sch.run(reqs)
    torch.cuda.synchronize()
    assert torch.cuda.max_memory_allocated() == alloc0   # the arena predates serving
    assert len(done) == len(scans) and ex.arena.peak <= cap and ex.arena.in_use == 0
    assert sch.max_concurrent < 4                        # memory, not slots, limited concurrency
    for r in done:
        assert np.array_equal(r.result.numpy().view(np.uint32), alone[r.rid].view(np.uint32))
        if dtype == "c64":
            assert rma.nmse(r.result.numpy(), rma.rma_exact(rma.setup_from(scans[r.rid]))) <= 2e-5
    s = latency_summary(done)
    assert s["p99_ms"] >= s["p50_ms"] > 0
