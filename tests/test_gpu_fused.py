"""GPU parity of the fused passes (two tree levels per HBM pass, selected with PS_FUSED=1)
against the CPU oracle: same bit-exact output as the binary passes, on shapes that exercise
nodes with two, three and four input ranges, chunk boundaries, ragged tails, key types and
segments.  The mode is read once per process, so the checks run in a child process."""
import os
import subprocess
import sys

import pytest

from conftest import ROOT

pytestmark = pytest.mark.gpu

CHILD = r"""
import numpy as np, torch
import oracle, workloads
import paper_1805_04154_gb300 as ps
from paper_1805_04154_gb300 import _build
_build.build(); ps.load()

def dev(a):
    if a.dtype == np.uint32: return torch.from_numpy(a.view(np.int32)).cuda()
    if a.dtype == np.uint64: return torch.from_numpy(a.view(np.int64)).cuda()
    return torch.from_numpy(a).cuda()

def check(keys, vals, kt_name, kt):
    ref = oracle.powersort(keys, vals, kt=kt_name)
    dk, dv = dev(keys), dev(vals)
    ps.ps_sort(dk, dv, key_type=kt)
    assert ps.ps_stream_status() == 0
    assert np.array_equal(dk.cpu().numpy().view(keys.dtype), ref.keys), (kt_name, keys.size)
    assert np.array_equal(dv.cpu().numpy().view(np.uint32), ref.vals), (kt_name, keys.size)

for n, ml in [(300001, 5000), (1 << 20, 20000), (2000003, 700), (1 << 21, 3)]:
    k, v = workloads.runs_i32(n, seed=n, max_len=ml)
    check(k, v, "i32", 0)
k, v = workloads.perm_i32(1 << 20, seed=9)
check(k, v, "i32", 0)
k, v = workloads.runs_i32(1 << 20, seed=4, signed=False)
check(k, v, "u32", 1)
k, v = workloads.pareto_u64(1 << 21, seed=5, distinct=1000)
check(k, v, "u64", 2)
k, v = workloads.pareto_f32(1 << 20, seed=6)
check(k, v, "f32", 3)
k, v = workloads.random_runs_i32(3 * 10 ** 6, seed=2, mean_len=3000)
check(k, v, "i32", 0)
keys, vals, off = workloads.segmented_i32(400, seed=8, lo_exp=4, hi_exp=17)
ref = oracle.sort_segmented(keys, vals, off)
dk, dv = dev(keys), dev(vals)
ps.ps_sort_segmented(dk, dv, torch.from_numpy(off).cuda(), key_type=0)
assert ps.ps_stream_status() == 0
assert np.array_equal(dk.cpu().numpy(), ref[0]) and np.array_equal(dv.cpu().numpy().view(np.uint32), ref[1])
print("fused ok")
"""


def test_fused_passes_match_oracle():
    env = dict(os.environ, PS_FUSED="1")
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "fused ok" in r.stdout
