"""Multi-rank host logic on CPU (gloo, world size 2): the timing reduction
(max over ranks), barriers and the reference arm's rank-0-only rule (the
bench's data path has no collective: ranks image independent scans); and the
data flow a single scan split over ranks would take -- frequency slabs through
the spectrum, one all-to-all to k_x slabs, Stolt per column -- run with the
oracle's steps on CPU ranks."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import bench
d = bench.Dist(want_cuda=False)
r = d.rank
out = {{"rank": r, "world": d.world, "max": d.max(10.0 + r), "sum": d.sum(1.0 + r)}}
d.barrier()
print(json.dumps(out))
d.close()
"""


def _launch(code_or_args, world=2, timeout=120):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(world), LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS="2")
        cmd = [sys.executable, "-c", code_or_args] if isinstance(code_or_args, str) else [sys.executable] + code_or_args
        procs.append(subprocess.Popen(cmd, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                                      cwd=ROOT))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=timeout)
        assert p.returncode == 0, e
        outs.append(o)
    return outs


SHARDED = r"""
import os, sys, json, dataclasses
sys.path.insert(0, {root!r})
import numpy as np
import torch
import torch.distributed as dist
import synth
from oracle import rma
dist.init_process_group("gloo")
r, W = dist.get_rank(), dist.get_world_size()
scan = synth.custom(nx_pos=6, ny_pos=5, nk={nk}, layout="awr1443", nx=16, ny=12, nz=8, seed=7,
                    jitter=(0.7e-3, 3e-3))
su = rma.setup_from(scan)
nk, Mx = su.n_k, su.Mx
kb = [nk * j // W for j in range(W + 1)]      # frequency slab of each rank (uneven when W does not divide nk)
mb = [Mx * j // W for j in range(W + 1)]      # k_x slab of each rank
# compensation (Eq. 11) and the transform over the aperture (FT_2D of Eq. 16)
# are independent per frequency: this rank's slab only
sub = dataclasses.replace(su, echo=su.echo[..., kb[r]:kb[r + 1]], f0=su.f0 + kb[r] * su.df)
S = rma.spectrum_exact(sub)                   # [Mx, My, nk_r]
# one all-to-all: k_x slab j of this rank's frequencies to rank j
flat = lambda a: torch.view_as_real(torch.from_numpy(np.ascontiguousarray(a))).reshape(-1)
send = torch.cat([flat(S[mb[j]:mb[j + 1]]) for j in range(W)])
insz = [(mb[j + 1] - mb[j]) * su.My * (kb[r + 1] - kb[r]) * 2 for j in range(W)]
outsz = [(mb[r + 1] - mb[r]) * su.My * (kb[j + 1] - kb[j]) * 2 for j in range(W)]
recv = torch.empty(sum(outsz), dtype=torch.float64)
dist.all_to_all_single(recv, send, outsz, insz)
parts = torch.split(recv, outsz)
cols = np.concatenate([torch.view_as_complex(parts[j].reshape(-1, 2)).numpy().reshape(
    mb[r + 1] - mb[r], su.My, kb[j + 1] - kb[j]) for j in range(W)], axis=2)   # every frequency of my columns
# Eq. 15 and the transform over k_z need every frequency of a column: local now
kx, ky = rma.spectral_axes(su)
Z = rma.stolt_exact(su, cols, kx=kx[mb[r]:mb[r + 1]], ky=ky)   # [m_r, My, nz]
# the inverse transform over (k_x, k_y): gather the slabs
sizes = [torch.tensor([mb[j + 1] - mb[j]]) for j in range(W)]
mine = flat(Z)
n_max = max(mb[j + 1] - mb[j] for j in range(W)) * su.My * su.nz * 2
pad = torch.zeros(n_max, dtype=torch.float64)
pad[:mine.numel()] = mine
got = [torch.empty(n_max, dtype=torch.float64) for _ in range(W)]
dist.all_gather(got, pad)
if r == 0:
    Zall = np.concatenate([torch.view_as_complex(got[j][:(mb[j + 1] - mb[j]) * su.My * su.nz * 2].reshape(-1, 2))
                           .numpy().reshape(mb[j + 1] - mb[j], su.My, su.nz) for j in range(W)], axis=0)
    vol = rma.image_from_Z(su, Zall)
    ref = rma.rma_exact(su)
    print(json.dumps({{"nmse": rma.nmse(vol, ref), "same_peak": rma.peak_index(vol) == rma.peak_index(ref),
                      "bit_identical": bool(np.array_equal(vol, ref))}}))
dist.barrier()
dist.destroy_process_group()
"""


@pytest.mark.parametrize("nk", [16, 11])
def test_frequency_sharded_scan_matches_one_rank(nk):
    """A single scan split over two ranks by frequency (spectrum per slab,
    all-to-all to k_x slabs, Stolt and the k_z transform per column, gather)
    gives the one-rank oracle's image; 11 frequencies make the slabs uneven."""
    outs = _launch(SHARDED.format(root=ROOT, nk=nk), timeout=300)
    rows = [json.loads(o.strip().splitlines()[-1]) for o in outs if o.strip()]
    assert len(rows) == 1
    assert rows[0]["nmse"] < 1e-24 and rows[0]["same_peak"]


def test_max_and_sum_over_two_ranks():
    outs = _launch(WORKER.format(root=ROOT))
    rows = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    assert sorted(r["rank"] for r in rows) == [0, 1]
    for r in rows:
        assert r["world"] == 2 and r["max"] == 11.0 and r["sum"] == 3.0


def test_reference_arm_prints_once_on_rank_zero():
    outs = _launch(["bench.py", "--impl", "reference", "--workload", "tiny", "--steps", "1", "--warmup", "0",
                    "--gpus", "2"], timeout=300)
    lines = [o.strip() for o in outs if o.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0].splitlines()[-1])
    assert d["impl"] == "reference" and d["value"] > 0 and d["n_gpus"] == 2
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_reference_arm_single_process():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "tiny", "--steps", "2",
                          "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=300,
                         env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
    assert out.returncode == 0, out.stderr
    d = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is True
