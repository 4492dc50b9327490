"""Programmatic dependent launches change no result.

The small kernels of the block loop (panel, reductions, stop tests, Omega)
and the tensor-core products are launched with programmatic stream
serialisation; each waits for its predecessor before touching global memory,
so the arithmetic is the same as with ordinary launches.  The same seeded
factorizations run in two child processes, one with RQB_PDL=0 (ordinary
launches; the switch is read once per process) and one with the default, and
their Q, B and k must agree bit for bit on every handle: FP64, plain FP32
(blocked Cholesky at b = 256), split-TF32 and BF16 storage.  A second run
with the default launches checks that the factorization is deterministic.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import inputs
from paper_1503_07157_gb300 import rqb
out = {}
cases = [
    ("fp64", torch.float64, rqb.RQB_PREC_NATIVE, 1500, 900, 50, 1e-4),
    ("fp32", torch.float32, rqb.RQB_PREC_NATIVE, 3000, 2000, 256, 1e-3),
    ("tf32x3", torch.float32, rqb.RQB_PREC_TF32X3, 4096, 2048, 256, 1e-3),
    ("bf16", torch.bfloat16, rqb.RQB_PREC_BF16, 4096, 2048, 256, 1e-2),
]
for name, dt, prec, m, n, b, er in cases:
    s = inputs.spectrum_mixed_config(min(m, n), knee=600)
    A32 = inputs.usv_torch(m, n, s, 7, device="cuda", dtype=torch.float64 if dt == torch.float64 else torch.float32)
    if dt == torch.bfloat16:
        A = torch.empty(n, m, dtype=torch.bfloat16, device="cuda").t()
        A.copy_(A32)
    else:
        A = A32
    eps = er * float(np.sqrt(np.sum(s ** 2)))
    with rqb.Handle(dt, prec=prec) as h:
        Q, B, k, rc = h.rqb_factor(A, eps, b, 3, check=False)
        torch.cuda.synchronize()
        out[name + "_Q"] = Q.float().cpu().numpy() if dt == torch.bfloat16 else Q.cpu().numpy()
        out[name + "_B"] = B.cpu().numpy()
        out[name + "_k"] = np.array([k, rc])
np.savez(sys.argv[2], **out)
"""


def _run(tmp_path, tag, pdl):
    path = str(tmp_path / f"{tag}.npz")
    env = dict(os.environ)
    if pdl is not None:
        env["RQB_PDL"] = pdl
    else:
        env.pop("RQB_PDL", None)
    r = subprocess.run([sys.executable, "-c", _CHILD, ROOT, path], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return dict(np.load(path))


def _same(x, y):
    assert set(x) == set(y)
    bad = []
    for key in sorted(x):
        a, b = x[key], y[key]
        assert a.shape == b.shape, key
        a8, b8 = np.ascontiguousarray(a).view(np.uint8), np.ascontiguousarray(b).view(np.uint8)
        if not np.array_equal(a8, b8):
            bad.append(key)
    return bad


def test_pdl_launches_are_bitwise_neutral(rqb_lib, tmp_path):
    """Two runs with programmatic launches and one with ordinary launches:
    the factorization is deterministic (no order-dependent sums, no racing
    stores) and the launch mode does not change it."""
    on = _run(tmp_path, "on", None)
    on2 = _run(tmp_path, "on2", None)
    off = _run(tmp_path, "off", "0")
    for key in on:
        if key.endswith("_k"):
            assert on[key][1] == rqb_lib.RQB_OK, key
    assert _same(on, on2) == [], "repeat runs differ"
    assert _same(on, off) == [], "launch modes differ"
