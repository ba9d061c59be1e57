"""GB300-native Fourier transform on SU(2) (Delgado & Umana): Python binding.

Thin layer over the C ABI of libsu2fft.so (include/su2fft.h).  PyTorch
provides device memory and streams; every step of the transform runs in the
library's CUDA kernels (stage 1: 2-D DFT over alpha, gamma per beta node;
stage 2: beta contraction with the Wigner-d recurrence fused in).

    plan = Plan(N=64, batch=1, dtype="c64")
    coeffs = plan.forward(grid)          # grid: complex64 CUDA tensor, shape (B, N, N, N)
    grid2  = plan.inverse(coeffs)
    g      = plan.backward(grad_coeffs)  # adjoint of forward

Layouts: the grid of function f is f[j1, k, j2] (alpha, beta, gamma indices,
j2 fastest); coefficients are packed per function in blocks j = 2l, each the
(2l+1)x(2l+1) matrix f^(l)_{mn} row-major (row m+l, column n+l).
"""
from __future__ import annotations

import ctypes

import torch

from . import _abi
from ._abi import SU2Error, load  # noqa: F401

__all__ = ["Plan", "SU2FFT", "num_coeffs", "SU2Error", "load"]


def num_coeffs(N: int) -> int:
    return int(load().su2_num_coeffs(int(N)))


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class Plan:
    """A transform plan for a batch of functions (uniform or ragged bandwidths)."""

    def __init__(self, N=None, batch: int = 1, dtype: str = "c64", algo: str = "auto",
                 weights: str = "cc", device: int | None = None, Ns=None, graph: bool = False,
                 autotune: bool = False, full_group: bool = False, literal: bool = False,
                 persistent: bool = False):
        self._lib = load()
        if Ns is not None:
            Ns = [int(n) for n in Ns]
            batch = len(Ns)
        elif N is None:
            raise ValueError("give N (uniform) or Ns (ragged)")
        self.Ns = Ns if Ns is not None else [int(N)] * int(batch)
        self.batch = len(self.Ns)
        self.dtype = dtype
        self.algo = algo
        self.device = torch.cuda.current_device() if device is None else int(device)
        desc = _abi.PlanDesc()
        desc.num_functions = self.batch
        if Ns is not None:
            self._narr = (ctypes.c_int * self.batch)(*self.Ns)
            desc.N = ctypes.cast(self._narr, ctypes.POINTER(ctypes.c_int))
        else:
            desc.N = None
        desc.N_uniform = self.Ns[0]
        desc.dtype = _abi.DTYPES[dtype]
        desc.algo = _abi.ALGOS[algo]
        desc.weights = _abi.WEIGHTS[weights]
        desc.flags = ((_abi.FLAG_CUDA_GRAPH if graph else 0) | (_abi.FLAG_AUTOTUNE if autotune else 0) |
                      (_abi.FLAG_FULL_GROUP if full_group else 0) | (_abi.FLAG_LITERAL_GRID if literal else 0) |
                      (_abi.FLAG_PERSISTENT if persistent else 0))
        self.full_group = full_group
        self.literal = literal
        desc.device = self.device
        h = ctypes.c_void_p()
        _abi.check("su2_plan", self._lib.su2_plan(ctypes.byref(h), ctypes.byref(desc)))
        self._h = h
        sz = ctypes.c_size_t()
        _abi.check("su2_workspace_size", self._lib.su2_workspace_size(h, ctypes.byref(sz)))
        self.workspace_bytes = int(sz.value)
        used = ctypes.c_int()
        _abi.check("su2_plan_persistent", self._lib.su2_plan_persistent(h, ctypes.byref(used)))
        self.persistent = bool(used.value)      # su2_forward runs the one-launch path
        ge, ce = ctypes.c_size_t(), ctypes.c_size_t()
        _abi.check("su2_grid_elems", self._lib.su2_grid_elems(h, ctypes.byref(ge)))
        _abi.check("su2_coeff_elems", self._lib.su2_coeff_elems(h, ctypes.byref(ce)))
        self.grid_elems, self.coeff_elems = int(ge.value), int(ce.value)
        self.grid_offsets, self.coeff_offsets, self.plane_offsets = [], [], []
        for f in range(self.batch):
            o = ctypes.c_size_t()
            _abi.check("su2_grid_offset", self._lib.su2_grid_offset(h, f, ctypes.byref(o)))
            self.grid_offsets.append(int(o.value))
            _abi.check("su2_coeff_offset", self._lib.su2_coeff_offset(h, f, ctypes.byref(o)))
            self.coeff_offsets.append(int(o.value))
            _abi.check("su2_plane_offset", self._lib.su2_plane_offset(h, f, ctypes.byref(o)))
            self.plane_offsets.append(int(o.value))
        self._ws = None

    # ------------------------------------------------------------------
    @property
    def torch_dtype(self):
        return torch.complex128 if self.dtype == "c128" else torch.complex64

    def workspace(self) -> torch.Tensor:
        """A cached device workspace of the size the library asks for."""
        if self._ws is None:
            self._ws = torch.empty(max(self.workspace_bytes, 16), dtype=torch.uint8,
                                   device=f"cuda:{self.device}")
        return self._ws

    def _check_tensor(self, t: torch.Tensor, elems: int, what: str):
        if not t.is_cuda or t.dtype != self.torch_dtype or not t.is_contiguous():
            raise ValueError(f"{what}: need a contiguous {self.torch_dtype} CUDA tensor")
        if t.numel() != elems:
            raise ValueError(f"{what}: expected {elems} elements, got {t.numel()}")

    def forward(self, grid: torch.Tensor, out: torch.Tensor | None = None, ws: torch.Tensor | None = None,
                stream=None) -> torch.Tensor:
        self._check_tensor(grid, self.grid_elems, "grid")
        if out is None:
            out = torch.empty(self.coeff_elems, dtype=self.torch_dtype, device=grid.device)
        self._check_tensor(out, self.coeff_elems, "coeffs")
        ws = self.workspace() if ws is None else ws
        _abi.check("su2_forward", self._lib.su2_forward(self._h, grid.data_ptr(), out.data_ptr(),
                                                        ws.data_ptr(), _stream_ptr(stream)))
        return out

    def forward_stage1(self, grid: torch.Tensor, ws: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Stage 1 only (2-D DFT per beta node) into the workspace; returns the workspace."""
        self._check_tensor(grid, self.grid_elems, "grid")
        ws = self.workspace() if ws is None else ws
        _abi.check("su2_forward_stage1", self._lib.su2_forward_stage1(self._h, grid.data_ptr(), ws.data_ptr(),
                                                                      _stream_ptr(stream)))
        return ws

    def forward_stage2(self, out: torch.Tensor | None = None, ws: torch.Tensor | None = None,
                       stream=None) -> torch.Tensor:
        """Stage 2 only (beta contraction) from the workspace planes into coefficients."""
        ws = self.workspace() if ws is None else ws
        if out is None:
            out = torch.empty(self.coeff_elems, dtype=self.torch_dtype, device=ws.device)
        self._check_tensor(out, self.coeff_elems, "coeffs")
        _abi.check("su2_forward_stage2", self._lib.su2_forward_stage2(self._h, ws.data_ptr(), out.data_ptr(),
                                                                      _stream_ptr(stream)))
        return out

    def forward_pipelined(self, host_grid: torch.Tensor, host_out: torch.Tensor | None = None,
                          dev_grid: torch.Tensor | None = None, dev_out: torch.Tensor | None = None,
                          ws: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Forward transform of grids in host memory (pinned for overlap) into host
        coefficients, streamed through the device; returns host_out (complete once
        the stream has passed the call)."""
        if host_grid.device.type != "cpu" or not host_grid.is_contiguous() or host_grid.dtype != self.torch_dtype \
                or host_grid.numel() != self.grid_elems:
            raise ValueError("host_grid: contiguous CPU tensor of the plan's dtype and grid_elems elements")
        dev = torch.device(f"cuda:{self.device}")
        if host_out is None:
            host_out = torch.empty(self.coeff_elems, dtype=self.torch_dtype, pin_memory=True)
        if host_out.device.type != "cpu" or not host_out.is_contiguous() or host_out.dtype != self.torch_dtype \
                or host_out.numel() != self.coeff_elems:
            raise ValueError("host_out: contiguous CPU tensor of the plan's dtype and coeff_elems elements")
        dev_grid = torch.empty(self.grid_elems, dtype=self.torch_dtype, device=dev) if dev_grid is None else dev_grid
        dev_out = torch.empty(self.coeff_elems, dtype=self.torch_dtype, device=dev) if dev_out is None else dev_out
        self._check_tensor(dev_grid, self.grid_elems, "dev_grid")
        self._check_tensor(dev_out, self.coeff_elems, "dev_out")
        ws = self.workspace() if ws is None else ws
        _abi.check("su2_forward_pipelined",
                   self._lib.su2_forward_pipelined(self._h, host_grid.data_ptr(), host_out.data_ptr(),
                                                   dev_grid.data_ptr(), dev_out.data_ptr(), ws.data_ptr(),
                                                   _stream_ptr(stream)))
        return host_out

    def forward_stage2_depth(self, depth: int, out: torch.Tensor | None = None, ws: torch.Tensor | None = None,
                             stream=None) -> torch.Tensor:
        """Stage 2 by the depth-k divide-and-conquer projection (complex128 plans)."""
        ws = self.workspace() if ws is None else ws
        if out is None:
            out = torch.empty(self.coeff_elems, dtype=self.torch_dtype, device=ws.device)
        self._check_tensor(out, self.coeff_elems, "coeffs")
        _abi.check("su2_forward_stage2_depth",
                   self._lib.su2_forward_stage2_depth(self._h, int(depth), ws.data_ptr(), out.data_ptr(),
                                                      _stream_ptr(stream)))
        return out

    def forward_stage1_slab(self, k_base: int, nk: int, grid_slab: torch.Tensor, out: torch.Tensor | None = None,
                            ws: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Stage 1 for beta nodes [k_base, k_base + nk) (su2_forward_stage1_slab): grid_slab
        [nfunc][N][nk][N] -> exchange layout [2N][nfunc][N/4][nk][4] (flat)."""
        N = self.Ns[0]
        elems = self.batch * N * nk * N
        self._check_tensor(grid_slab, elems, "grid_slab")
        if out is None:
            out = torch.empty(2 * elems, dtype=self.torch_dtype, device=grid_slab.device)
        self._check_tensor(out, 2 * elems, "xplanes")
        ws = self.workspace() if ws is None else ws
        _abi.check("su2_forward_stage1_slab",
                   self._lib.su2_forward_stage1_slab(self._h, int(k_base), int(nk), grid_slab.data_ptr(),
                                                     out.data_ptr(), ws.data_ptr(), _stream_ptr(stream)))
        return out

    def forward_stage2_rows(self, row0: int, nrows: int, nk: int, xrecv: torch.Tensor,
                            out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Stage 2 for rows [row0, row0 + nrows) (su2_forward_stage2_rows) from the received
        exchange layout [N/nk][nrows][nfunc][N/4][nk][4]; writes only those rows' coefficients."""
        N = self.Ns[0]
        self._check_tensor(xrecv, nrows * self.batch * N * N, "xrecv")
        if out is None:
            out = torch.zeros(self.coeff_elems, dtype=self.torch_dtype, device=xrecv.device)
        self._check_tensor(out, self.coeff_elems, "coeffs")
        _abi.check("su2_forward_stage2_rows",
                   self._lib.su2_forward_stage2_rows(self._h, int(row0), int(nrows), int(nk), xrecv.data_ptr(),
                                                     out.data_ptr(), _stream_ptr(stream)))
        return out

    def inverse(self, coeffs: torch.Tensor, out: torch.Tensor | None = None, ws: torch.Tensor | None = None,
                stream=None) -> torch.Tensor:
        self._check_tensor(coeffs, self.coeff_elems, "coeffs")
        if out is None:
            out = torch.empty(self.grid_elems, dtype=self.torch_dtype, device=coeffs.device)
        self._check_tensor(out, self.grid_elems, "grid")
        ws = self.workspace() if ws is None else ws
        _abi.check("su2_inverse", self._lib.su2_inverse(self._h, coeffs.data_ptr(), out.data_ptr(),
                                                        ws.data_ptr(), _stream_ptr(stream)))
        return out

    def backward(self, grad_coeffs: torch.Tensor, out: torch.Tensor | None = None,
                 ws: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        self._check_tensor(grad_coeffs, self.coeff_elems, "grad_coeffs")
        if out is None:
            out = torch.empty(self.grid_elems, dtype=self.torch_dtype, device=grad_coeffs.device)
        self._check_tensor(out, self.grid_elems, "grad_grid")
        ws = self.workspace() if ws is None else ws
        _abi.check("su2_backward", self._lib.su2_backward(self._h, grad_coeffs.data_ptr(), out.data_ptr(),
                                                          ws.data_ptr(), _stream_ptr(stream)))
        return out

    def selftest_bounded_wait(self, kind: int, stream=None):
        """Enqueue a kernel whose bounded wait never completes (0: counter,
        1: mbarrier); the next sync_status raises SU2Error with SU2_ERR_TIMEOUT."""
        _abi.check("su2_selftest_bounded_wait",
                   self._lib.su2_selftest_bounded_wait(self._h, int(kind), _stream_ptr(stream)))

    def sync_status(self, stream=None):
        _abi.check("su2_sync_status", self._lib.su2_sync_status(self._h, _stream_ptr(stream)))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.su2_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SU2FFT(torch.autograd.Function):
    """Differentiable forward transform: coeffs = SU2FFT.apply(grid, plan).

    The map is linear, so the backward pass is the library's adjoint
    (su2_backward): grad_grid = A^H grad_coeffs, the conjugate-Wirtinger
    convention PyTorch uses for complex inputs.  The Wigner-d values are
    regenerated inside the adjoint kernel; nothing is saved for backward.
    """

    @staticmethod
    def forward(ctx, grid, plan):
        ctx.plan = plan
        return plan.forward(grid.contiguous().reshape(-1))

    @staticmethod
    def backward(ctx, grad):
        g = ctx.plan.backward(grad.contiguous())
        return g, None
