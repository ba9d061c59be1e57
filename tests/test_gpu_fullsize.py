"""Every coefficient of the benchmark's launch configuration against the FP64
oracle, and the synthesis / adjoint element by element at N = 256 and 512.

Forward, N = 256, 64 functions, complex64, both contraction paths (the FP32
FMA kernels and the split-BF16 tensor-core kernel), launched exactly as the
benchmark launches them (one plan over the whole batch).  Two base grids:

* the N = 256 precision workload's own input: coefficients CN(0, (1+l)^-1)
  up to l = 127.5, seed 2, synthesised by the oracle in FP64 (Sec. 3
  expansion) and rounded to complex64;
* a white-noise grid (seed 2), not band-limited.

The oracle analyses the rounded grids in FP64 (Sec. 4 quadrature sum in the
separated form).  Batch slot b holds base[b % 2] times alpha_b = 2^e i^r with
(e, r) different for every slot of a base; such a factor is exact in
complex64, so the exact answer of slot b is alpha_b times the oracle's, and a
kernel that mixed up functions within a 64-function tile would fail.  Every
coefficient of every slot is compared: rel = max |gpu - ref| / max |ref| over
the C(N) coefficients of a slot (then the max over slots), tolerance 1e-5.

Synthesis and adjoint: complete beta planes (all N^2 points of 8 beta nodes,
the poles included) of su2_inverse / su2_backward against the oracle's
synthesis and adjoint sums, at N = 256 (2 functions) and N = 512 (1).
"""
import numpy as np
import pytest

import su2inputs as I
from oracle import pool as OP

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5
N, B = 256, 64


@pytest.fixture(scope="module")
def su2():
    import paper_2605_23923_gb300 as m
    from paper_2605_23923_gb300 import build
    build.build()
    return m


def slot_factor(b):
    """alpha_b = 2^e i^r, distinct for the 32 slots of each base (b % 2)."""
    h = b // 2
    return (2.0 ** (h % 8 - 4)) * (1j ** (h // 8))


@pytest.fixture(scope="module")
def bases():
    c = I.draw_coeffs(N, np.random.default_rng(2), "inv1")
    g0 = OP.synthesis_planes(c[None], N, range(N))["synthesis"][0]      # [j1, k, j2]
    g1 = I.draw_grid_gaussian((N, N, N), np.random.default_rng(2))
    grids = np.stack([g0, g1]).astype(np.complex64)
    ref = OP.forward_all(grids.astype(np.complex128))                   # [2, C]
    return grids, ref


@pytest.mark.parametrize("algo", ["tc_bf16x3", "fp32"])
def test_forward_every_coefficient_n256_b64(su2, bases, algo):
    grids, ref = bases
    C = I.num_coeffs(N)
    plan = su2.Plan(N=N, batch=B, dtype="c64", algo=algo)
    x = torch.empty(B * N ** 3, dtype=torch.complex64, device="cuda")
    g_dev = [torch.from_numpy(g.reshape(-1)).cuda() for g in grids]
    for b in range(B):
        x[b * N ** 3:(b + 1) * N ** 3].copy_(g_dev[b % 2] * slot_factor(b))   # exact in complex64
    del g_dev
    out = plan.forward(x)
    plan.sync_status()
    del x
    ref_dev = [torch.from_numpy(r).cuda() for r in ref]
    worst = []
    for b in range(B):
        r = ref_dev[b % 2] * slot_factor(b)
        got = out[b * C:(b + 1) * C].to(torch.complex128)
        worst.append(((got - r).abs().max() / r.abs().max()).item())
    plan.close()
    assert max(worst) < TOL, (algo, int(np.argmax(worst)), max(worst))


PLANES = {256: [0, 1, 37, 127, 128, 200, 254, 255], 512: [0, 1, 63, 255, 256, 400, 510, 511]}


@pytest.mark.parametrize("Nb,Bb", [(256, 2), (512, 1)])
def test_inverse_and_adjoint_planes(su2, Nb, Bb):
    ks = PLANES[Nb]
    rng = np.random.default_rng(40 + Nb)
    cs = np.stack([I.draw_coeffs(Nb, rng, "inv1") for _ in range(Bb)]).astype(np.complex64)
    plan = su2.Plan(N=Nb, batch=Bb, dtype="c64")
    c_dev = torch.from_numpy(cs.reshape(-1)).cuda()
    syn = plan.inverse(c_dev)
    adj = plan.backward(c_dev)
    plan.sync_status()
    kt = torch.tensor(ks, device="cuda")
    got = {name: t.reshape(Bb, Nb, Nb, Nb)[:, :, kt, :].cpu().numpy().astype(np.complex128)
           for name, t in (("syn", syn), ("adj", adj))}
    del syn, adj
    plan.close()
    refs = OP.synthesis_planes(cs.astype(np.complex128), Nb, ks, modes=("synthesis", "adjoint"))
    for name, mode in (("syn", "synthesis"), ("adj", "adjoint")):
        ref = refs[mode]                                                     # [B, j1, len(ks), j2]
        for b in range(Bb):
            d = np.max(np.abs(got[name][b] - ref[b])) / np.max(np.abs(ref[b]))
            assert d < TOL, (name, Nb, b, d)
