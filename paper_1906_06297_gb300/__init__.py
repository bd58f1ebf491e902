"""GB300 checkerboard Metropolis sweeps of the 2D Ising model.

A thin Python binding over ``libising.so`` (CUDA kernels for sm_103a behind
the C ABI declared in ``include/ising.h``).  The functions carry the C names;
they only marshal arguments: device memory is PyTorch tensors, the stream is
PyTorch's current stream, and every step of the sweep runs in the library's
kernels.  There is no CPU fallback: if the library is missing or cannot be
loaded, every call raises.

Method: Romero, Bisson, Fatica, Bernaschi, "A Performance study of the 2D
Ising model on GPUs" (arXiv:1906.06297), Sec. 2 (model, Metropolis rule,
checkerboard), Sec. 3.1 (colour planes), Sec. 3.3 (multi-spin coding).
"""
from __future__ import annotations

import ctypes
import os
import threading

from ._build import LIB as _LIB_PATH
from ._build import build  # noqa: F401  (re-exported for build scripts)

ISING_OK, ISING_EINVAL, ISING_ECUDA, ISING_ETIMEOUT = 0, 1, 2, 3
ISING_INT8, ISING_MSC4 = 0, 1
ISING_INIT_RANDOM, ISING_INIT_UP, ISING_INIT_DOWN = 0, 1, 2
LAYOUTS = {"int8": ISING_INT8, "msc4": ISING_MSC4}


class IsingError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: {detail} (status {status})")
        self.status = status


class ising_lattice_t(ctypes.Structure):
    _fields_ = [
        ("black", ctypes.c_void_p),
        ("white", ctypes.c_void_p),
        ("L", ctypes.c_int64),
        ("layout", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("row_stride_bytes", ctypes.c_int64),
    ]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"libising.so is not built ({_LIB_PATH}); run __graft_entry__.build()")
        lib = ctypes.CDLL(_LIB_PATH)
        P, i32, i64, u32, u64, dbl = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                      ctypes.c_uint64, ctypes.c_double)
        LP = ctypes.POINTER(ising_lattice_t)
        sig = {
            "ising_lattice_bytes": [i64, i32, P, P],
            "ising_thresholds": [dbl, P],
            "ising_init_lattice": [LP, i32, u64, P],
            "ising_half_sweep": [LP, dbl, i32, u64, u64, P, P],
            "ising_sweep": [LP, dbl, i64, u64, u64, P, P],
            "ising_sweep_host": [LP, P, P, dbl, i64, u64, u64, P, P, P],
            "ising_observables": [LP, P, P],
            "ising_pack": [LP, LP, P],
            "ising_unpack": [LP, LP, P],
            "ising_rng_probe": [u64, u64, u64, i32, u32, P, P],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        lib.ising_strerror.argtypes = [ctypes.c_int]
        lib.ising_strerror.restype = ctypes.c_char_p
        lib.ising_last_error.argtypes = []
        lib.ising_last_error.restype = ctypes.c_char_p
        _lib = lib
        return lib


def _check(rc: int, where: str):
    if rc != ISING_OK:
        lib = _load()
        raise IsingError(rc, where, lib.ising_last_error().decode() or lib.ising_strerror(rc).decode())


def _stream(stream):
    """A raw cudaStream_t: an int handle, a torch.cuda.Stream, or None for the
    current PyTorch stream."""
    if stream is None:
        import torch

        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _addr(t) -> ctypes.c_void_p:
    if t is None:
        return ctypes.c_void_p(0)
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    if hasattr(t, "data_ptr"):
        return ctypes.c_void_p(t.data_ptr())
    return ctypes.c_void_p(t.ctypes.data)  # numpy (host buffers)


# ---------------------------------------------------------------------------
# C entry points, same names
# ---------------------------------------------------------------------------
def ising_strerror(status: int) -> str:
    return _load().ising_strerror(status).decode()


def ising_lattice_bytes(L: int, layout: int):
    row = ctypes.c_size_t()
    plane = ctypes.c_size_t()
    _check(_load().ising_lattice_bytes(L, layout, ctypes.byref(row), ctypes.byref(plane)), "ising_lattice_bytes")
    return row.value, plane.value


def ising_thresholds(beta: float):
    T = (ctypes.c_uint64 * 5)()
    _check(_load().ising_thresholds(float(beta), T), "ising_thresholds")
    return [int(x) for x in T]


def ising_init_lattice(lat, init: int = ISING_INIT_RANDOM, seed: int = 0, stream=None):
    _check(_load().ising_init_lattice(ctypes.byref(_struct(lat)), init, seed, _stream(stream)), "ising_init_lattice")


def ising_half_sweep(lat, beta: float, colour: int, seed: int, t: int, obs=None, stream=None):
    _check(_load().ising_half_sweep(ctypes.byref(_struct(lat)), float(beta), colour, seed, t, _addr(obs),
                                    _stream(stream)), "ising_half_sweep")


def ising_sweep(lat, beta: float, n_sweeps: int, seed: int, sweep_offset: int = 0, trace=None, stream=None):
    _check(_load().ising_sweep(ctypes.byref(_struct(lat)), float(beta), n_sweeps, seed, sweep_offset, _addr(trace),
                               _stream(stream)), "ising_sweep")


def ising_sweep_host(dev_lat, black_host, white_host, beta: float, n_sweeps: int, seed: int, sweep_offset: int = 0,
                     trace_dev=None, trace_host=None, stream=None):
    _check(_load().ising_sweep_host(ctypes.byref(_struct(dev_lat)), _addr(black_host), _addr(white_host),
                                    float(beta), n_sweeps, seed, sweep_offset, _addr(trace_dev), _addr(trace_host),
                                    _stream(stream)), "ising_sweep_host")


def ising_observables(lat, out, stream=None):
    _check(_load().ising_observables(ctypes.byref(_struct(lat)), _addr(out), _stream(stream)), "ising_observables")


def ising_pack(int8_src, msc4_dst, stream=None):
    _check(_load().ising_pack(ctypes.byref(_struct(int8_src)), ctypes.byref(_struct(msc4_dst)), _stream(stream)),
           "ising_pack")


def ising_unpack(msc4_src, int8_dst, stream=None):
    _check(_load().ising_unpack(ctypes.byref(_struct(msc4_src)), ctypes.byref(_struct(int8_dst)), _stream(stream)),
           "ising_unpack")


def ising_rng_probe(n_blocks: int, seed: int, t: int, colour: int, T3: int, count, stream=None):
    _check(_load().ising_rng_probe(n_blocks, seed, t, colour, T3, _addr(count), _stream(stream)), "ising_rng_probe")


# ---------------------------------------------------------------------------
# Lattice storage (PyTorch owns the device memory)
# ---------------------------------------------------------------------------
class Lattice:
    """Two colour planes in device memory, laid out as ``include/ising.h``
    describes.  ``row_stride_bytes`` may pad rows (MSC4: multiple of 16)."""

    def __init__(self, L: int, layout: str = "msc4", device="cuda", row_stride_bytes: int | None = None):
        import torch

        self.L = int(L)
        self.layout_name = layout
        self.layout = LAYOUTS[layout]
        row, _ = ising_lattice_bytes(self.L, self.layout)
        self.row_bytes = row
        self.row_stride_bytes = int(row_stride_bytes or row)
        dtype = torch.int8 if self.layout == ISING_INT8 else torch.uint8
        self.black = torch.empty((self.L, self.row_stride_bytes), dtype=dtype, device=device)
        self.white = torch.empty((self.L, self.row_stride_bytes), dtype=dtype, device=device)

    def struct(self) -> ising_lattice_t:
        return ising_lattice_t(self.black.data_ptr(), self.white.data_ptr(), self.L, self.layout, 0,
                               self.row_stride_bytes)

    def planes_numpy(self):
        """Host copies of the planes (rows trimmed to the row size): int8
        arrays for INT8, uint64 word arrays for MSC4."""
        import numpy as np

        b = self.black[:, : self.row_bytes].cpu().numpy()
        w = self.white[:, : self.row_bytes].cpu().numpy()
        if self.layout == ISING_MSC4:
            b = np.ascontiguousarray(b).view(np.uint64)
            w = np.ascontiguousarray(w).view(np.uint64)
        return np.ascontiguousarray(b), np.ascontiguousarray(w)

    def load_numpy(self, black, white):
        """Copy host planes (as returned by planes_numpy) into the device planes."""
        import numpy as np
        import torch

        for dst, src in ((self.black, black), (self.white, white)):
            a = np.ascontiguousarray(src)
            if self.layout == ISING_MSC4:
                a = a.view(np.uint8)
            dst[:, : self.row_bytes].copy_(torch.from_numpy(a.reshape(self.L, self.row_bytes)))


def _struct(lat) -> ising_lattice_t:
    if isinstance(lat, ising_lattice_t):
        return lat
    return lat.struct()
