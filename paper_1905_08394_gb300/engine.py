"""Convenience wrapper over the C ABI: one context plus a device workspace.

PyTorch provides the device memory (a uint8 CUDA tensor used as the
workspace) and the stream; all work is done by the library's kernels.
"""
from __future__ import annotations

import numpy as np

from . import binding as B


class Simulator:
    def __init__(self, R: int, C: int, device: int = 0):
        import torch  # device memory and streams only

        self._torch = torch
        self.R, self.C = R, C
        self.device = torch.device("cuda", device)
        self.h = B.peps_create(R, C)
        self._ws = None

    def close(self) -> None:
        if self.h is not None:
            B.peps_destroy(self.h)
            self.h = None
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- circuit -------------------------------------------------------------
    def apply_1q(self, r: int, c: int, U) -> None:
        B.peps_apply_1q(self.h, r, c, U)

    def apply_cz(self, r0: int, c0: int, r1: int, c1: int) -> None:
        B.peps_apply_cz(self.h, r0, c0, r1, c1)

    def apply_circuit(self, circuit) -> None:
        """Queue the gates of an rqc_inputs.Circuit (same lattice)."""
        assert (circuit.R, circuit.C) == (self.R, self.C)
        C = self.C
        for g in circuit.gates:
            if g.kind == "1q":
                q = g.qubits[0]
                self.apply_1q(q // C, q % C, g.U)
            elif g.kind == "2q":
                a, b = g.qubits
                B.peps_apply_2q(self.h, a // C, a % C, b // C, b % C, g.U)
            else:
                a, b = g.qubits
                self.apply_cz(a // C, a % C, b // C, b % C)

    def bond_dim(self, r0, c0, r1, c1) -> int:
        return B.peps_bond_dim(self.h, r0, c0, r1, c1)

    def cz_count(self) -> int:
        return B.peps_cz_count(self.h)

    # -- workspace -----------------------------------------------------------
    def workspace(self, n: int, opts) -> tuple[int, int]:
        need = B.peps_workspace_bytes(self.h, n, opts)
        if self._ws is None or self._ws.numel() < need:
            self._ws = None
            self._ws = self._torch.empty(need, dtype=self._torch.uint8, device=self.device)
        return self._ws.data_ptr(), self._ws.numel()

    def _stream(self, stream) -> int:
        if stream is None:
            stream = self._torch.cuda.current_stream(self.device)
        return stream.cuda_stream

    # -- amplitudes ------------------------------------------------------------
    def amplitudes(self, bitstrings, stream=None, **kw) -> np.ndarray:
        """Host bitstrings in, host complex128 amplitudes out (blocking)."""
        bits = np.ascontiguousarray(bitstrings, dtype=np.uint64)
        opts, keep = B.make_opts(**kw)
        ws, nbytes = self.workspace(len(bits), opts)
        out = B.peps_amplitudes(self.h, bits, opts, ws, nbytes, self._stream(stream))
        del keep
        return out

    def amplitudes_device(self, d_bits, d_out=None, stream=None, **kw):
        """Device bitstrings (int64/uint64 CUDA tensor) in, complex128 CUDA
        tensor out; enqueued on the stream."""
        torch = self._torch
        n = d_bits.numel()
        if d_out is None:
            d_out = torch.empty(n, dtype=torch.complex128, device=self.device)
        opts, keep = B.make_opts(**kw)
        ws, nbytes = self.workspace(n, opts)
        B.peps_amplitudes_device(self.h, d_bits.data_ptr(), n, d_out.data_ptr(), opts, ws,
                                 nbytes, self._stream(stream))
        del keep
        return d_out

    def plan_info(self, n: int, **kw) -> dict:
        opts, keep = B.make_opts(**kw)
        info = B.peps_plan_info_get(self.h, n, opts)
        del keep
        return info

    def stats(self) -> dict:
        return B.peps_get_stats(self.h)
