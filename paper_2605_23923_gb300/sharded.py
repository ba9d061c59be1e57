"""Forward transform of functions split over several GPUs (one process each).

The paper's Sec. 6 first-stage Proposition makes stage 1 (the 2-D DFT over
alpha, gamma) independent per beta node, and the second-stage Proposition makes
stage 2 (the beta contraction) independent per (m, n) pair.  So a transform
too large for one GPU splits as:

  1. rank r holds the grids at its beta nodes k in [k_base, k_base + nk) and runs
     stage 1 for them (su2_forward_stage1_slab), writing the planes in the
     exchange layout [2N rows][nfunc][N/4][nk][4], row = s N + mi;
  2. one all-to-all: rank r sends each rank q the contiguous range of rows q
     owns, and receives from every source its nk beta nodes of r's own rows;
  3. rank r runs stage 2 for its rows (su2_forward_stage2_rows) and writes the
     coefficients (l, m, n) of those rows into a zeroed coefficient buffer;
  4. a sum over ranks gives every coefficient (each is owned by exactly one
     rank, so the sum is exact).

With R ranks: nk = N / R beta nodes and 2N / R rows per rank (nk a multiple of
16 for the tensor-core stage 2), so each rank holds 1/R of the grids, of the
planes and of the stage-2 work; the exchange moves (R - 1)/R of the planes.
Stage functions can be replaced (the CPU tests of the partition and the
exchange use stand-ins on CPU tensors); by default they are the library's.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def partition(N: int, world: int, rank: int):
    """(k_base, nk, row0, nrows) of `rank`: equal contiguous blocks of the N beta
    nodes and of the 2N rows."""
    if world < 1 or N % world or (2 * N) % world:
        raise ValueError(f"N = {N} does not split over {world} ranks")
    nk, nr = N // world, 2 * N // world
    return rank * nk, nk, rank * nr, nr


class ShardedForward:
    """The forward transform of one plan's batch split over the ranks of `group`.

    plan: a Plan with one bandwidth N (tensor-core algorithm) on this rank's GPU;
    stage1(k_base, nk, grid_slab) -> exchange-layout planes (flat),
    stage2(row0, nrows, nk, xrecv, coeffs) -> writes the rows' coefficients.
    """

    def __init__(self, plan, rank: int, world: int, group=None, stage1=None, stage2=None):
        self.plan, self.rank, self.world, self.group = plan, rank, world, group
        self.N = plan.Ns[0]
        self.nfunc = plan.batch
        self.k_base, self.nk, self.row0, self.nrows = partition(self.N, world, rank)
        self.stage1 = stage1 or (lambda kb, nk, g: plan.forward_stage1_slab(kb, nk, g))
        self.stage2 = stage2 or (lambda r0, nr, nk, x, c: plan.forward_stage2_rows(r0, nr, nk, x, out=c))

    def row_elems(self) -> int:
        """Complex elements of one row of the exchange layout (all functions, nk nodes)."""
        return self.nfunc * self.N * self.nk

    def exchange(self, xsend: torch.Tensor) -> torch.Tensor:
        """All-to-all of the exchange layout: rank q gets rows [q 2N/R, (q+1) 2N/R) of every
        rank's planes, stacked by source: [R][nrows][nfunc][N/4][nk][4]."""
        per = self.nrows * self.row_elems()
        xrecv = torch.empty(self.world * per, dtype=xsend.dtype, device=xsend.device)
        if self.world == 1:
            xrecv.copy_(xsend)
            return xrecv
        dist.all_to_all_single(torch.view_as_real(xrecv), torch.view_as_real(xsend), group=self.group)
        return xrecv

    def forward(self, grid_slab: torch.Tensor, coeffs: torch.Tensor | None = None) -> torch.Tensor:
        """Coefficients of the whole batch (every rank gets all of them)."""
        xsend = self.stage1(self.k_base, self.nk, grid_slab)
        xrecv = self.exchange(xsend)
        if coeffs is None:
            coeffs = torch.zeros(self.plan.coeff_elems, dtype=xsend.dtype, device=xsend.device)
        else:
            coeffs.zero_()
        self.stage2(self.row0, self.nrows, self.nk, xrecv, coeffs)
        if self.world > 1:
            dist.all_reduce(torch.view_as_real(coeffs), op=dist.ReduceOp.SUM, group=self.group)
        return coeffs
