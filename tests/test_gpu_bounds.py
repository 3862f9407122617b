"""The bounds-checked build, the stand-in for a memory checker: the library compiled with
-DSSHT_DEBUG tests the index of every checked global access of its kernels (torus passes, data and
operand packing, the tensor-core contraction's copies and outputs, the recursions writing the A
tiles, the real-field and spin-pair kernels, the SIMT contractions) against the extent of the
buffer it touches, records the ones outside and skips them.  Small cases of every path -- each
precision, ragged sizes, batches over one GEMM slice, real fields, spin pairs, the cache mode, a
group of uneven band-limits -- run in a child process on that library; no access may fall outside
its buffer, and the results still match the oracle."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent(r"""
    import numpy as np
    import torch
    from oracle import transforms as T
    from paper_0807_4494_gb300 import inputs, ssht

    TOL = {"fp64": 1e-11, "fp32": 3e-6, "tf32x3": 1e-6, "bf16x6": 1e-6}

    def rel(a, b):
        return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())

    def clean(what):
        n, site, idx, ext = ssht.ssht_debug_bounds()
        assert n == 0, "%s: %d accesses outside their buffers, first at site %d: index %d of %d" % (what, n, site, idx, ext)

    clean("start")
    cases = [(2, 0, 1, "tf32x3"), (33, 2, 3, "tf32x3"), (96, -1, 5, "tf32x3"), (129, 3, 2, "tf32x3"),
             (40, 1, 65, "tf32x3"), (33, 2, 3, "bf16x6"), (129, -2, 4, "bf16x6"), (33, 2, 3, "fp32"),
             (96, 0, 2, "fp32"), (17, 2, 2, "fp64"), (33, -3, 3, "fp64")]
    for L, s, B, prec in cases:
        dt = torch.complex128 if prec == "fp64" else torch.complex64
        flm = inputs.coeffs(L, s, B, seed=L + B)
        plan = ssht.Plan(L, s, B, precision=prec)
        f = plan.inverse(torch.from_numpy(flm).to(dt).cuda())
        back = plan.forward(f)
        adj = plan.adjoint(f)
        plan.check()
        clean("L=%d s=%d B=%d %s" % (L, s, B, prec))
        fo, bo, ao = f.cpu().numpy(), back.cpu().numpy(), adj.cpu().numpy()
        for b in sorted({0, B - 1}):
            g = fo[b].astype(np.complex128)
            assert rel(fo[b], T.inverse(flm[b], L, s)) < TOL[prec], (L, s, B, prec, "inverse", b)
            assert rel(bo[b], T.forward(g, L, s)) < TOL[prec], (L, s, B, prec, "forward", b)
            assert rel(ao[b], T.adjoint(g, L, s)) < TOL[prec], (L, s, B, prec, "adjoint", b)
        plan.close()

    # cache mode, the paper's recursion, real fields (odd count), spin pairs
    for kw in ({"delta_mode": "cache"}, {"recursion": "risbo"}):
        plan = ssht.Plan(48, 2, 3, precision="tf32x3", **kw)
        flm = inputs.coeffs(48, 2, 3, seed=5)
        for _ in range(2):
            back = plan.forward(plan.inverse(torch.from_numpy(flm).to(torch.complex64).cuda()))
        plan.check()
        clean(str(kw))
        assert rel(back.cpu().numpy(), flm) < 2e-6
        plan.close()
    for prec in ("fp32", "tf32x3", "fp64"):
        flm = inputs.coeffs(37, 0, 3, seed=9, real=True)
        plan = ssht.Plan(37, 0, 3, precision=prec, real=True)
        x = torch.from_numpy(flm).to(plan.dtype).cuda()
        f = plan.inverse(x)
        back, adj = plan.forward(f), plan.adjoint(f)
        plan.check()
        clean("real %s" % prec)
        assert rel(back.cpu().numpy(), flm) < 2 * TOL[prec]
        plan.close()
    for prec in ("tf32x3", "fp64"):
        dt = torch.complex128 if prec == "fp64" else torch.complex64
        flm = inputs.coeffs(33, 2, 2, seed=11)
        f = np.ascontiguousarray(T.inverse(flm, 33, 2))
        plan = ssht.Plan(33, 2, 2, precision=prec, spin_pair=True)
        fwd = plan.forward(torch.from_numpy(f).to(dt).cuda()).cpu().numpy()
        plan.adjoint(torch.from_numpy(f).to(dt).cuda())
        plan.inverse(torch.from_numpy(np.stack([flm, np.zeros_like(flm)], axis=1)).to(dt).cuda())
        plan.check()
        clean("spin pair %s" % prec)
        assert rel(fwd[1, 1], T.forward(np.conj(f[1]), 33, -2)) < TOL[prec]
        plan.close()

    # a group of uneven band-limits and spins (shared tables, per-bucket plans)
    Ls, ss = [16, 33, 33, 64, 16, 64], [0, 2, -1, 1, 2, 0]
    grp = ssht.Group(Ls, ss, precision="tf32x3", tune=False)
    flms = [inputs.coeffs(L, s, 1, seed=20 + k)[0] for k, (L, s) in enumerate(zip(Ls, ss))]
    x = grp.pack_coeffs([torch.from_numpy(a).to(torch.complex64).cuda() for a in flms])
    back = grp.forward(grp.inverse(x))
    grp.check()
    clean("group")
    for k, a in enumerate(grp.unpack_coeffs(back)):
        assert rel(a.cpu().numpy(), flms[k]) < 2e-6, k
    print("bounds-checked build: clean")
""")


def test_bounds_checked_build_finds_no_access_outside_its_buffer():
    from paper_0807_4494_gb300 import build
    lib = build.build(debug=True)
    env = dict(os.environ, SSHT_LIBRARY=lib, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-4000:]
    assert "bounds-checked build: clean" in r.stdout
