"""The bounds-checked build (kernels compiled with -DPS_DEBUG: every guarded data-derived index
is compared with its array's extent, out-of-range accesses are skipped and counted).  A child
process loads libpowersort_debug.so, sorts the workloads of the parity tests through every
entry point (plain, segmented, peeksort tree, minimal run length, device-driven) and checks each
result against the CPU oracle and that no access was out of range."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, ROOT)
sys.path.insert(0, ROOT + "/tests")
import oracle, workloads
import paper_1805_04154_gb300 as ps
assert ps.lib_path.endswith("libpowersort_debug.so"), ps.lib_path
ps.load()
def dev(a):
    if a.dtype == np.uint32: return torch.from_numpy(a.view(np.int32)).cuda()
    if a.dtype == np.uint64: return torch.from_numpy(a.view(np.int64)).cuda()
    return torch.from_numpy(a).cuda()
out = {}
def check(name, keys, vals, kt, ktn, how="plain", w=1):
    ref = oracle.powersort(keys, vals, kt=ktn, min_run=w)
    dk, dv = dev(keys), dev(vals)
    ws = torch.empty(ps.ps_workspace_size(kt, True, keys.size, False, 1 if how == "peek" else 0), dtype=torch.uint8, device="cuda")
    if how == "plain": ps.ps_sort_ws(dk, dv, ws, key_type=kt)
    elif how == "peek": ps.ps_sort_tree_ws(dk, dv, ws, 1, key_type=kt)
    elif how == "minrun": ps.ps_sort_minrun_ws(dk, dv, ws, w, key_type=kt)
    elif how == "async": ps.ps_sort_async_ws(dk, dv, ws, key_type=kt)
    st = ps.ps_stream_status()
    torch.cuda.synchronize()
    ok = st == 0 and np.array_equal(dk.cpu().numpy().view(keys.dtype), ref.keys) and \
        np.array_equal(dv.cpu().numpy().view(np.uint32), ref.vals)
    out[name] = bool(ok)
k, v = workloads.runs_i32(300001, seed=1, max_len=1000); check("runs_i32", k, v, 0, "i32")
check("runs_i32_peek", k, v, 0, "i32", "peek")
check("runs_i32_async", k, v, 0, "i32", "async")
k, v = workloads.perm_i32(200003, seed=2); check("perm_i32", k, v, 0, "i32")
check("perm_minrun24", k, v, 0, "i32", "minrun", 24)
k, v = workloads.pareto_u64(150000, seed=3, alpha=1.2, distinct=40, max_len=20000); check("pareto_u64", k, v, 2, "u64")
check("pareto_u64_minrun7", k, v, 2, "u64", "minrun", 7)
k, v = workloads.pareto_f32(120000, seed=4); check("pareto_f32", k, v, 3, "f32")
keys, vals, off = workloads.segmented_i32(200, seed=6, lo_exp=0, hi_exp=14)
ref = oracle.sort_segmented(keys, vals, off)
dk, dv = dev(keys), dev(vals)
ps.ps_sort_segmented(dk, dv, torch.from_numpy(off).cuda(), key_type=0)
st = ps.ps_stream_status()
out["segmented"] = bool(st == 0 and np.array_equal(dk.cpu().numpy(), ref[0]) and np.array_equal(dv.cpu().numpy().view(np.uint32), ref[1]))
torch.cuda.synchronize()
out["bounds_hits"] = ps.ps_debug_bounds()
print(json.dumps(out))
"""


def test_bounds_checked_build():
    from paper_1805_04154_gb300 import _build
    _build.build(debug=True)
    env = dict(os.environ, PS_DEBUG="1")
    res = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CHILD], env=env, capture_output=True,
                         text=True, timeout=900)
    assert res.returncode == 0, res.stderr[-3000:]
    out = json.loads(res.stdout.strip().splitlines()[-1])
    assert out.pop("bounds_hits") == 0
    assert all(out.values()), out
