"""The sharded forward transform's host logic on two gloo ranks (CPU): the
partition of the beta nodes and of the (s, m) rows, the all-to-all of the
exchange layout, and the gather of the coefficients by ownership.  The GPU
stages are replaced by stand-ins built from the FP64 oracle that read and
write the same exchange layout the library's kernels use (the GPU test checks
those kernels bit for bit against the unsharded transform); the gathered
coefficients must equal the oracle's forward transform of the whole grids."""
import os
import socket
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

N, B, WORLD = 16, 2, 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _grids():
    import su2inputs as I
    rng = np.random.default_rng(77)
    return np.stack([I.draw_grid_gaussian((N, N, N), rng) for _ in range(B)])


def _stage1(kb, nk, slab):
    """Planes F2_s[k][m][n] = w_k/(2N^2) sum f e^{i(n alpha + m gamma)} of the slab's
    nodes, in the exchange layout [2N][nfunc][N/4][nk][4] (row s N + mi)."""
    import torch
    from oracle import grid as G, quadrature as Q, transform as T
    fs = slab.numpy().reshape(B, N, nk, N)
    al, ga, w = G.alpha_nodes(N), G.gamma_nodes(N), Q.weights(N, "cc")
    x = np.zeros((2 * N, B, N // 4, nk, 4), dtype=np.complex128)
    for s, sector in ((0, "int"), (1, "half")):
        idx = T.sector_indices(N, sector)
        pos = (idx - s) // 2 + N // 2                 # mi (or ni) of each doubled index
        for f in range(B):
            F = T.torus_dft(fs[f], idx, idx, al, ga)   # [kk, n, m]
            for kk in range(nk):
                F2 = F[kk] * w[kb + kk] / (2.0 * N * N)
                for a, ni in enumerate(pos):
                    for c, mi in enumerate(pos):
                        x[s * N + mi, f, ni // 4, kk, ni % 4] = F2[a, c]
    return torch.from_numpy(x.reshape(-1))


def _stage2(r0, nr, nk, xrecv, coeffs):
    """Coefficients of rows [r0, r0 + nr) from the received exchange layout."""
    from oracle import basis, grid as G
    x = xrecv.numpy().reshape(N // nk, nr, B, N // 4, nk, 4)
    be = G.beta_nodes(N)
    C = G.num_coeffs(N)
    out = coeffs.numpy()
    for lr in range(nr):
        row = r0 + lr
        s, mi = divmod(row, N)
        if s == 0 and mi == 0:
            continue
        m2 = 2 * (mi - N // 2) + s
        for ni in range(N):
            if s == 0 and ni == 0:
                continue
            n2 = 2 * (ni - N // 2) + s
            j0, D = basis.wigner_d_column(n2, m2, be, N - 2 + s)
            for f in range(B):
                v = x[:, lr, f, ni // 4, :, ni % 4].reshape(N)       # all beta nodes, in order
                vals = basis.i_pow((n2 - m2) // 2) * (D @ v)
                for i, val in enumerate(vals):
                    out[f * C + G.coeff_index(j0 + 2 * i, m2, n2)] = val


def _worker(rank, port, q):
    import torch
    import torch.distributed as dist
    from paper_2605_23923_gb300.sharded import ShardedForward
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)

    class _Plan:                       # what ShardedForward reads from a plan
        Ns, batch = [N], B
        coeff_elems = B * (N * (N + 1) * (2 * N + 1) // 6)

    sf = ShardedForward(_Plan(), rank, WORLD, stage1=_stage1, stage2=_stage2)
    fs = _grids()
    slab = torch.from_numpy(np.ascontiguousarray(fs[:, :, sf.k_base:sf.k_base + sf.nk, :]).reshape(-1))
    coeffs = torch.zeros(_Plan.coeff_elems, dtype=torch.complex128)
    sf.forward(slab, coeffs)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, (sf.k_base, sf.nk, sf.row0, sf.nrows), coeffs.numpy()))


def test_two_gloo_ranks_gather_the_whole_transform():
    import torch.multiprocessing as mp
    from oracle import transform as T
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [(0, 8, 0, 16), (8, 8, 16, 16)]
    fs = _grids()
    ref = np.concatenate([T.forward_separable(f) for f in fs])
    for _, _, c in res:                               # every rank holds all coefficients
        assert np.max(np.abs(c - ref)) < 1e-13 * np.max(np.abs(ref))


def test_partition_covers_everything_once():
    from paper_2605_23923_gb300.sharded import partition
    for Nn, R in ((64, 2), (256, 4), (512, 8), (128, 1)):
        ks, rows = [], []
        for r in range(R):
            kb, nk, r0, nr = partition(Nn, R, r)
            ks += list(range(kb, kb + nk))
            rows += list(range(r0, r0 + nr))
        assert ks == list(range(Nn)) and rows == list(range(2 * Nn))
