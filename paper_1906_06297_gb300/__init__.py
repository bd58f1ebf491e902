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


class ising_slab_t(ctypes.Structure):
    _fields_ = [
        ("black", ctypes.c_void_p),
        ("white", ctypes.c_void_p),
        ("L", ctypes.c_int64),
        ("row0", ctypes.c_int64),
        ("rows", ctypes.c_int64),
        ("layout", ctypes.c_int32),
        ("spare_sms", ctypes.c_int32),
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
        SP = ctypes.POINTER(ising_slab_t)
        sig = {
            "ising_lattice_bytes": [i64, i32, P, P],
            "ising_thresholds": [dbl, P],
            "ising_init_lattice": [LP, i32, u64, P],
            "ising_half_sweep": [LP, dbl, i32, u64, u64, P, P],
            "ising_sweep": [LP, dbl, i64, u64, u64, P, P],
            "ising_sweep_host": [LP, P, P, dbl, i64, u64, u64, P, P, P],
            "ising_bits_bytes": [i64, P],
            "ising_msc4_to_bits": [LP, P, P, P],
            "ising_bits_to_msc4": [P, P, LP, P],
            "ising_sweep_host_bits": [LP, P, P, P, dbl, i64, u64, u64, P, P, P],
            "ising_observables": [LP, P, P],
            "ising_pack": [LP, LP, P],
            "ising_unpack": [LP, LP, P],
            "ising_rng_probe": [u64, u64, u64, i32, u32, P, P],
            "ising_mulwide_probe": [i32, u32, P, P, P],
            "ising_slab_bytes": [i64, i64, i32, P, P],
            "ising_slab_init": [SP, i32, u64, P],
            "ising_slab_half_sweep": [SP, dbl, i32, u64, u64, P, P],
            "ising_slab_exchange": [SP, i32, i32, P],
            "ising_slab_sweep": [SP, i32, dbl, i64, u64, u64, P, P],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        BP = ctypes.c_void_p  # opaque ising_batch_t *
        bsig = {
            "ising_batch_bytes": [i64, P, i32, P, P],
            "ising_batch_create": [i64, P, i32, P, P, ctypes.c_size_t, P],
            "ising_batch_destroy": [BP],
            "ising_batch_init": [BP, i32, u64, P],
            "ising_batch_run": [BP, i64, u64, u64, i32, i32, P, i32, P],
            "ising_batch_check": [BP, P],
            "ising_batch_planes": [BP, P, P, P],
            "ising_batch_state": [BP, P, P],
            "ising_batch_config": [BP, i32, i32],
            "ising_batch_get_config": [BP, P, P],
            "ising_batch_autotune": [BP, i64, P],
            "ising_batch_barrier_selftest": [BP, i64, P],
            "ising_batch_run_noalloc": [i64, P, i32, P, P, P, P, P, i64, u64, u64, i32, i32, P, P],
            "ising_net_workspace_bytes": [i64, i64, i32, P],
            "ising_net_forward": [i64, i64, P, P, P, P, P, P, ctypes.c_size_t, i32, P],
            "ising_net_forward_flipped": [i64, i64, P, P, P, P, P, P, P, ctypes.c_size_t, P],
            "ising_net_check": [P],
            "ising_net_wait_selftest": [i64, i64, P, P, P, P, P, ctypes.c_size_t, P],
            "ising_net_backward": [i64, i64, P, P, P, P, P, P, ctypes.c_size_t, P],
            "ising_net_targets_loss": [i64, i64, P, P, dbl, P, P, P, P, P],
            "ising_net_adam": [P, P, P, P, i64, ctypes.c_float, P],
            "ising_block_propose": [i64, i64, P, u64, u64, P, P],
            "ising_block_accept": [i64, i64, P, P, dbl, P, P, P, u64, u64, P, P, P],
        }
        for name, args in bsig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        lib.ising_net_param_count.argtypes = []
        lib.ising_net_param_count.restype = ctypes.c_int
        lib.ising_net_last_error.argtypes = []
        lib.ising_net_last_error.restype = ctypes.c_char_p
        lib.ising_batch_last_error.argtypes = []
        lib.ising_batch_last_error.restype = ctypes.c_char_p
        lib.ising_strerror.argtypes = [ctypes.c_int]
        lib.ising_strerror.restype = ctypes.c_char_p
        lib.ising_last_error.argtypes = []
        lib.ising_last_error.restype = ctypes.c_char_p
        _lib = lib
        return lib


def _check(rc: int, where: str):
    if rc != ISING_OK:
        lib = _load()
        msg = lib.ising_batch_last_error().decode() if where.startswith("ising_batch") else ""
        if where.startswith("ising_net") or where.startswith("ising_block"):
            msg = lib.ising_net_last_error().decode()
        raise IsingError(rc, where, msg or lib.ising_last_error().decode() or lib.ising_strerror(rc).decode())


def _stream(stream):
    """A raw cudaStream_t: an int handle, a torch.cuda.Stream, or None for the
    current PyTorch stream."""
    if stream is None:
        import torch

        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _on_stream(stream):
    """Context that makes `stream` PyTorch's current stream (a torch.cuda.Stream
    or a raw int handle; None keeps the current one), so that the PyTorch ops
    of a helper that sequences several calls (copies, fills, collectives) are
    ordered with the library calls it queues on `stream`."""
    import contextlib

    import torch

    if stream is None:
        return contextlib.nullcontext()
    if not hasattr(stream, "cuda_stream"):
        stream = torch.cuda.ExternalStream(int(stream))
    return torch.cuda.stream(stream)


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


def ising_bits_bytes(L: int) -> int:
    n = ctypes.c_size_t()
    _check(_load().ising_bits_bytes(L, ctypes.byref(n)), "ising_bits_bytes")
    return n.value


def ising_msc4_to_bits(msc4, black_bits, white_bits, stream=None):
    _check(_load().ising_msc4_to_bits(ctypes.byref(_struct(msc4)), _addr(black_bits), _addr(white_bits),
                                      _stream(stream)), "ising_msc4_to_bits")


def ising_bits_to_msc4(black_bits, white_bits, msc4, stream=None):
    _check(_load().ising_bits_to_msc4(_addr(black_bits), _addr(white_bits), ctypes.byref(_struct(msc4)),
                                      _stream(stream)), "ising_bits_to_msc4")


def ising_sweep_host_bits(dev_lat, black_host, white_host, stage_dev, beta: float, n_sweeps: int, seed: int,
                          sweep_offset: int = 0, trace_dev=None, trace_host=None, stream=None):
    _check(_load().ising_sweep_host_bits(ctypes.byref(_struct(dev_lat)), _addr(black_host), _addr(white_host),
                                         _addr(stage_dev), float(beta), n_sweeps, seed, sweep_offset,
                                         _addr(trace_dev), _addr(trace_host), _stream(stream)),
           "ising_sweep_host_bits")


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


def ising_mulwide_probe(form: int, iters: int, sink, stream=None) -> int:
    """Launches the wide-multiply throughput probe (form 0: as a Philox round
    issues it; form 1: with a 64-bit addend); returns the number of
    32 x 32 -> 64-bit multiplies the launch performs."""
    n = ctypes.c_uint64()
    _check(_load().ising_mulwide_probe(form, iters, _addr(sink), ctypes.byref(n), _stream(stream)),
           "ising_mulwide_probe")
    return n.value


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


# ---------------------------------------------------------------------------
# Horizontal slabs with halo rows (Sec. 4)
# ---------------------------------------------------------------------------
def ising_slab_bytes(L: int, rows: int, layout: int = ISING_MSC4):
    row = ctypes.c_size_t()
    plane = ctypes.c_size_t()
    _check(_load().ising_slab_bytes(L, rows, layout, ctypes.byref(row), ctypes.byref(plane)), "ising_slab_bytes")
    return row.value, plane.value


def _slab_struct(sl) -> ising_slab_t:
    return sl if isinstance(sl, ising_slab_t) else sl.struct()


def _slab_array(slabs):
    arr = (ising_slab_t * len(slabs))(*[_slab_struct(x) for x in slabs])
    return arr, len(slabs)


def ising_slab_init(slab, init: int = ISING_INIT_RANDOM, seed: int = 0, stream=None):
    _check(_load().ising_slab_init(ctypes.byref(_slab_struct(slab)), init, seed, _stream(stream)), "ising_slab_init")


def ising_slab_half_sweep(slab, beta: float, colour: int, seed: int, t: int, obs=None, stream=None):
    _check(_load().ising_slab_half_sweep(ctypes.byref(_slab_struct(slab)), float(beta), colour, seed, t, _addr(obs),
                                         _stream(stream)), "ising_slab_half_sweep")


def ising_slab_exchange(slabs, colour: int, stream=None):
    arr, n = _slab_array(slabs)
    _check(_load().ising_slab_exchange(arr, n, colour, _stream(stream)), "ising_slab_exchange")


def ising_slab_sweep(slabs, beta: float, n_sweeps: int, seed: int, sweep_offset: int = 0, trace=None, stream=None):
    arr, n = _slab_array(slabs)
    _check(_load().ising_slab_sweep(arr, n, float(beta), n_sweeps, seed, sweep_offset, _addr(trace),
                                    _stream(stream)), "ising_slab_sweep")


def slab_partition(L: int, n: int):
    """(row0, rows) of n horizontal slabs of an L x L lattice, sizes differing
    by at most one row, in order from row 0."""
    if n < 1 or n > L:
        raise ValueError(f"cannot cut {L} rows into {n} slabs")
    out, r0 = [], 0
    for k in range(n):
        rows = L // n + (1 if k < L % n else 0)
        out.append((r0, rows))
        r0 += rows
    return out


class Slab:
    """Rows row0 .. row0+rows-1 of an L x L MSC4 lattice with one halo row
    above and one below in each colour plane (plane row 0 and rows + 1), as
    ``ising_slab_t`` describes.  The planes are uint8 tensors of shape
    (rows + 2, row_bytes); ``device`` may be a CUDA device or, for the halo
    exchange alone, the CPU."""

    def __init__(self, L: int, row0: int, rows: int, device="cuda"):
        import torch

        self.L, self.row0, self.rows = int(L), int(row0), int(rows)
        self.row_bytes, _ = ising_slab_bytes(self.L, self.rows)
        self.black = torch.zeros((self.rows + 2, self.row_bytes), dtype=torch.uint8, device=device)
        self.white = torch.zeros((self.rows + 2, self.row_bytes), dtype=torch.uint8, device=device)
        self.spare_sms = 0

    def struct(self) -> ising_slab_t:
        return ising_slab_t(self.black.data_ptr(), self.white.data_ptr(), self.L, self.row0, self.rows, ISING_MSC4,
                            self.spare_sms, self.row_bytes)

    def view(self, first: int, count: int, spare_sms: int = 0) -> "Slab":
        """Own rows first .. first+count-1 as a slab of their own, sharing this
        slab's storage: its halo rows are the rows next to them (own rows of
        this slab, or this slab's halos at its ends).  A half-sweep of the
        view updates exactly those rows as the half-sweep of the whole slab
        does (the random numbers are keyed by the global row)."""
        if not (0 <= first and count >= 1 and first + count <= self.rows):
            raise ValueError(f"rows {first}..{first + count - 1} are not own rows of a {self.rows}-row slab")
        v = Slab.__new__(Slab)
        v.L, v.row0, v.rows, v.row_bytes = self.L, self.row0 + first, int(count), self.row_bytes
        v.black = self.black[first:first + count + 2]
        v.white = self.white[first:first + count + 2]
        v.spare_sms = int(spare_sms)
        return v

    def plane(self, colour: int):
        return self.black if colour == 0 else self.white

    def own_numpy(self):
        """Host copies of the own rows of both planes as uint64 words (rows x L/32)."""
        import numpy as np

        return tuple(np.ascontiguousarray(p[1:self.rows + 1].cpu().numpy()).view(np.uint64)
                     for p in (self.black, self.white))

    def load_own_numpy(self, black, white):
        """Copy host words (rows x L/32 uint64) into the own rows of both planes."""
        import numpy as np
        import torch

        for dst, src in ((self.black, black), (self.white, white)):
            a = np.ascontiguousarray(src, dtype=np.uint64).view(np.uint8).reshape(self.rows, self.row_bytes)
            dst[1:self.rows + 1].copy_(torch.from_numpy(a))


def _world(group):
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return 0, 1
    return dist.get_rank(group), dist.get_world_size(group)


def _post_halos(slab: Slab, colour: int, group=None, stream=None):
    """Start making the colour-`colour` halo rows of this rank's slab current
    and return what to wait for (a list of torch.distributed works, empty when
    the exchange was queued on `stream` itself)."""
    import torch.distributed as dist

    rank, world = _world(group)
    if world == 1:
        ising_slab_exchange([slab], colour, stream)
        return []
    p = slab.plane(colour)
    up, down = (rank - 1) % world, (rank + 1) % world
    peer = (lambda r: dist.get_global_rank(group, r)) if group is not None else (lambda r: r)
    ops = [
        dist.P2POp(dist.isend, p[slab.rows], peer(down), group, tag=0),  # my last row: halo above `down`
        dist.P2POp(dist.isend, p[1], peer(up), group, tag=1),            # my first row: halo below `up`
        dist.P2POp(dist.irecv, p[0], peer(up), group, tag=0),
        dist.P2POp(dist.irecv, p[slab.rows + 1], peer(down), group, tag=1),
    ]
    with _on_stream(stream):  # messages ordered after the half-sweeps queued on `stream`
        return dist.batch_isend_irecv(ops)


def _wait_halos(works, stream=None):
    with _on_stream(stream):  # NCCL: `stream` waits for the messages; gloo: the host does
        for w in works:
            w.wait()


def exchange_halos(slab: Slab, colour: int, group=None, stream=None):
    """Make the colour-`colour` halo rows of this rank's slab current.  Rank r
    holds the r-th slab of the lattice (ranks in row order, periodic): its
    halo above receives the last own row of rank r-1, its halo below the first
    own row of rank r+1.  One process: the library's copy (the slab is its own
    neighbour).  Several: point-to-point messages of one row each through
    torch.distributed (NCCL between GPUs), tagged 0 for rows travelling down
    and 1 for rows travelling up; with two ranks both messages between the
    pair are posted in the same order on both sides, so they also match where
    tags are ignored."""
    _wait_halos(_post_halos(slab, colour, group, stream), stream)


def slab_sweep(slab: Slab, beta: float, n_sweeps: int, seed: int, sweep_offset: int = 0, trace=None, group=None,
               half_sweep=None, stream=None, overlap: bool = True):
    """n_sweeps sweeps of a lattice distributed as one slab per rank (Sec. 4).
    `trace` (n_sweeps x 2 int64, on the slab's device) ends with the
    whole-lattice sums {sum of spins, sum over bonds} after each sweep.  The
    lattice equals ising_sweep of the whole lattice bit for bit.

    Order without overlap, per sweep: white halos, black half-sweep, black
    halos, white half-sweep.  With overlap (slabs of 3 rows or more), each
    half-sweep first updates the slab's first and last own rows, then posts
    those rows' messages to the neighbours and updates the interior rows
    while the messages travel; the next half-sweep waits for them before it
    starts.  The interior update leaves `slab.spare_sms` (at least one when
    there are several ranks) SMs free, so that the messages' kernels can run
    beside it.  Both orders give the same lattice: a half-sweep reads only the
    other colour's rows, and the boundary rows it sends are final once updated.

    ``half_sweep(slab, beta, colour, seed, t, obs)`` does the update of one
    colour of a slab's own rows; the default is the library's
    ising_slab_half_sweep.  Replacing it lets the exchange and ordering logic
    run against another implementation of the same rule."""
    import torch.distributed as dist

    hs = half_sweep or (lambda sl, b, c, sd, t, obs: ising_slab_half_sweep(sl, b, c, sd, t, obs, stream))
    _, world = _world(group)
    rows = slab.rows
    with _on_stream(stream):  # the fill, the messages and the half-sweeps in one stream order
        if trace is not None:
            trace.zero_()
        if not overlap or rows < 3:
            for k in range(n_sweeps):
                t = sweep_offset + k
                exchange_halos(slab, 1, group, stream)
                hs(slab, beta, 0, seed, t, None)
                exchange_halos(slab, 0, group, stream)
                hs(slab, beta, 1, seed, t, trace[k] if trace is not None else None)
        else:
            first, last = slab.view(0, 1), slab.view(rows - 1, 1)
            interior = slab.view(1, rows - 2, spare_sms=max(slab.spare_sms, 1 if world > 1 else 0))
            if n_sweeps > 0:
                exchange_halos(slab, 1, group, stream)
            for k in range(n_sweeps):
                t = sweep_offset + k
                for colour in (0, 1):
                    obs = trace[k] if (trace is not None and colour == 1) else None
                    hs(first, beta, colour, seed, t, obs)
                    hs(last, beta, colour, seed, t, obs)
                    works = _post_halos(slab, colour, group, stream)
                    hs(interior, beta, colour, seed, t, obs)
                    _wait_halos(works, stream)
        if trace is not None and world > 1:
            dist.all_reduce(trace, group=group)


# ---------------------------------------------------------------------------
# Batches with replica exchange
# ---------------------------------------------------------------------------
def ising_batch_bytes(L, ladder_size: int, beta) -> int:
    import numpy as np

    Ls = np.ascontiguousarray(L, dtype=np.int64)
    b = np.ascontiguousarray(beta, dtype=np.float64)
    out = ctypes.c_size_t()
    _check(_load().ising_batch_bytes(Ls.size, Ls.ctypes.data, ladder_size, b.ctypes.data, ctypes.byref(out)),
           "ising_batch_bytes")
    return out.value


class Batch:
    """n lattices (sides L[i]) in one device workspace owned by PyTorch; the
    ladders are S consecutive lattices over the S inverse temperatures `beta`."""

    def __init__(self, L, ladder_size: int, beta, device="cuda"):
        import numpy as np
        import torch

        self.L = np.ascontiguousarray(L, dtype=np.int64)
        self.n = int(self.L.size)
        self.S = int(ladder_size)
        self.beta = np.ascontiguousarray(beta, dtype=np.float64)
        nbytes = ising_batch_bytes(self.L, self.S, self.beta)
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=device)
        h = ctypes.c_void_p()
        _check(_load().ising_batch_create(self.n, self.L.ctypes.data, self.S, self.beta.ctypes.data,
                                          self.ws.data_ptr(), nbytes, ctypes.byref(h)), "ising_batch_create")
        self.handle = h
        black, white = ctypes.c_void_p(), ctypes.c_void_p()
        self.word_off = np.zeros(self.n + 1, dtype=np.int64)
        _check(_load().ising_batch_planes(h, ctypes.byref(black), ctypes.byref(white), self.word_off.ctypes.data),
               "ising_batch_planes")
        self._black_off = black.value - self.ws.data_ptr()
        self._white_off = white.value - self.ws.data_ptr()
        slot, at = ctypes.c_void_p(), ctypes.c_void_p()
        _check(_load().ising_batch_state(h, ctypes.byref(slot), ctypes.byref(at)), "ising_batch_state")
        self._slot_off = slot.value - self.ws.data_ptr()
        self._at_off = at.value - self.ws.data_ptr()

    def close(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.ising_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, init: int = ISING_INIT_RANDOM, seed: int = 0, stream=None):
        _check(_load().ising_batch_init(self.handle, init, seed, _stream(stream)), "ising_batch_init")

    def run(self, n_sweeps: int, seed: int, offset: int = 0, record_every: int = 0, swaps: bool = False,
            trace=None, use_graph: bool = True, stream=None):
        _check(_load().ising_batch_run(self.handle, n_sweeps, seed, offset, record_every, int(bool(swaps)),
                                       _addr(trace), int(bool(use_graph)), _stream(stream)), "ising_batch_run")

    def check(self, stream=None):
        _check(_load().ising_batch_check(self.handle, _stream(stream)), "ising_batch_check")

    def config(self, threads: int, words_per_thread: int):
        _check(_load().ising_batch_config(self.handle, threads, words_per_thread), "ising_batch_config")

    def get_config(self):
        a, b = ctypes.c_int32(), ctypes.c_int32()
        _check(_load().ising_batch_get_config(self.handle, ctypes.byref(a), ctypes.byref(b)), "ising_batch_get_config")
        return a.value, b.value

    def autotune(self, n_sweeps: int = 3, stream=None):
        _check(_load().ising_batch_autotune(self.handle, n_sweeps, _stream(stream)), "ising_batch_autotune")
        return self.get_config()

    def barrier_selftest(self, timeout_cycles: int, stream=None) -> int:
        """Runs the bounded-barrier self-test; returns its status code."""
        return int(_load().ising_batch_barrier_selftest(self.handle, timeout_cycles, _stream(stream)))

    def n_events(self, n_sweeps: int, offset: int, record_every: int) -> int:
        if record_every <= 0:
            return 0
        return (offset + n_sweeps) // record_every - offset // record_every

    def planes_numpy(self, i: int):
        """Host copies of lattice i's black and white planes (uint64 words)."""
        import numpy as np

        words = int(self.word_off[i + 1] - self.word_off[i])
        out = []
        for off in (self._black_off, self._white_off):
            a = off + 8 * int(self.word_off[i])
            out.append(np.ascontiguousarray(self.ws[a:a + 8 * words].cpu().numpy()).view(np.uint64)
                       .reshape(int(self.L[i]), int(self.L[i]) // 32))
        return out

    def state_numpy(self):
        import numpy as np

        slot = np.ascontiguousarray(self.ws[self._slot_off:self._slot_off + 4 * self.n].cpu().numpy()).view(np.int32)
        at = np.ascontiguousarray(self.ws[self._at_off:self._at_off + 4 * self.n].cpu().numpy()).view(np.int32)
        return slot.copy(), at.copy()


def ising_batch_run_noalloc(L, ladder_size: int, beta, black, white, slot_of, lattice_at, n_sweeps: int, seed: int,
                            sweep_offset: int = 0, record_every: int = 0, swaps: bool = False, trace=None,
                            stream=None):
    """Allocation-free batched run (see include/ising.h): the caller passes the
    planes, the slot state and the trace; the library's fixed scratch array
    holds everything else.  Synchronous."""
    import numpy as np

    Ls = np.ascontiguousarray(L, dtype=np.int64)
    b = np.ascontiguousarray(beta, dtype=np.float64)
    _check(_load().ising_batch_run_noalloc(Ls.size, Ls.ctypes.data, ladder_size, b.ctypes.data, _addr(black),
                                           _addr(white), _addr(slot_of), _addr(lattice_at), n_sweeps, seed,
                                           sweep_offset, record_every, int(bool(swaps)), _addr(trace),
                                           _stream(stream)), "ising_batch_run_noalloc")


# ---------------------------------------------------------------------------
# Learned block proposals
# ---------------------------------------------------------------------------
def ising_net_param_count() -> int:
    return int(_load().ising_net_param_count())


def ising_net_workspace_bytes(L: int, C: int, train: bool) -> int:
    out = ctypes.c_size_t()
    _check(_load().ising_net_workspace_bytes(L, C, int(bool(train)), ctypes.byref(out)), "ising_net_workspace_bytes")
    return out.value


def ising_net_forward(L, C, black, white, flip_block, params, logits, work, train=False, stream=None):
    _check(_load().ising_net_forward(L, C, _addr(black), _addr(white), _addr(flip_block), _addr(params),
                                     _addr(logits), _addr(work), work.numel() * work.element_size(),
                                     int(bool(train)), _stream(stream)), "ising_net_forward")


def ising_net_forward_flipped(L, C, black, white, flip_block, params, logits_x, logits, work, stream=None):
    _check(_load().ising_net_forward_flipped(L, C, _addr(black), _addr(white), _addr(flip_block), _addr(params),
                                             _addr(logits_x), _addr(logits), _addr(work),
                                             work.numel() * work.element_size(), _stream(stream)),
           "ising_net_forward_flipped")


def ising_net_check(stream=None):
    _check(_load().ising_net_check(_stream(stream)), "ising_net_check")


def ising_net_wait_selftest(L, C, black, white, params, logits, work, stream=None):
    _check(_load().ising_net_wait_selftest(L, C, _addr(black), _addr(white), _addr(params), _addr(logits),
                                           _addr(work), work.numel() * work.element_size(), _stream(stream)),
           "ising_net_wait_selftest")


def ising_net_backward(L, C, black, white, params, dlogits, grad, work, stream=None):
    _check(_load().ising_net_backward(L, C, _addr(black), _addr(white), _addr(params), _addr(dlogits), _addr(grad),
                                      _addr(work), work.numel() * work.element_size(), _stream(stream)),
           "ising_net_backward")


def ising_net_targets_loss(L, C, black, white, beta, logits, dlogits, chain_sq, loss, stream=None):
    _check(_load().ising_net_targets_loss(L, C, _addr(black), _addr(white), float(beta), _addr(logits),
                                          _addr(dlogits), _addr(chain_sq), _addr(loss), _stream(stream)),
           "ising_net_targets_loss")


def ising_net_adam(params, grad, m, v, step: int, lr: float, stream=None):
    _check(_load().ising_net_adam(_addr(params), _addr(grad), _addr(m), _addr(v), step, float(lr), _stream(stream)),
           "ising_net_adam")


def ising_block_propose(L, C, logits, seed: int, t: int, block, stream=None):
    _check(_load().ising_block_propose(L, C, _addr(logits), seed, t, _addr(block), _stream(stream)),
           "ising_block_propose")


def ising_block_accept(L, C, black, white, beta, logits_x, logits_xp, block, seed: int, t: int, accepted, dE=None,
                       stream=None):
    _check(_load().ising_block_accept(L, C, _addr(black), _addr(white), float(beta), _addr(logits_x),
                                      _addr(logits_xp), _addr(block), seed, t, _addr(accepted), _addr(dE),
                                      _stream(stream)), "ising_block_accept")


class BlockMove:
    """C chains of side L, kept in a Batch of equal sides at one beta (plain
    sweeps through the batch kernel), with a network-proposed (or uniform)
    Metropolis-Hastings block move after each sweep."""

    def __init__(self, L: int, C: int, beta: float, device="cuda"):
        import torch

        self.L, self.C, self.beta = int(L), int(C), float(beta)
        self.nb = (self.L // 8) ** 2
        self.batch = Batch([self.L] * self.C, 1, [self.beta], device=device)
        words = int(self.batch.word_off[-1])
        ws = self.batch.ws
        self.black = ws[self.batch._black_off:self.batch._black_off + 8 * words]
        self.white = ws[self.batch._white_off:self.batch._white_off + 8 * words]
        self.work = torch.empty(ising_net_workspace_bytes(self.L, self.C, False), dtype=torch.uint8, device=device)
        self.lx = torch.zeros((self.C, self.nb), dtype=torch.float32, device=device)
        self.lxp = torch.zeros_like(self.lx)
        self.block = torch.zeros(self.C, dtype=torch.int32, device=device)
        self.accepted = torch.zeros(self.C, dtype=torch.int32, device=device)
        self.dE = torch.zeros(self.C, dtype=torch.int64, device=device)
        torch.cuda.synchronize(device)  # the fills above precede moves queued on any stream

    def move(self, params, seed: int, t: int, stream=None):
        """One block move of every chain; params None proposes uniformly."""
        if params is None:
            ising_block_propose(self.L, self.C, None, seed, t, self.block, stream)
            ising_block_accept(self.L, self.C, self.black, self.white, self.beta, None, None, self.block, seed, t,
                               self.accepted, self.dE, stream)
            return
        ising_net_forward(self.L, self.C, self.black, self.white, None, params, self.lx, self.work, False, stream)
        ising_block_propose(self.L, self.C, self.lx, seed, t, self.block, stream)
        ising_net_forward_flipped(self.L, self.C, self.black, self.white, self.block, params, self.lx, self.lxp,
                                  self.work, stream)
        ising_block_accept(self.L, self.C, self.black, self.white, self.beta, self.lx, self.lxp, self.block, seed, t,
                           self.accepted, self.dE, stream)


def train_block_proposer(L: int, beta: float, n_configs: int = 100_000, batch: int = 64, steps: int = 2000,
                         lr: float = 1e-3, seed: int = 0, sweeps_between: int = 10, equilibrate: int = 200,
                         log_every: int = 10, device="cuda", stream=None):
    """Train the proposal network on the GPU with the library's kernels.

    Training data: n_configs configurations of side L from plain sweeps at
    beta (up to 1024 chains, snapshots `sweeps_between` sweeps apart after
    `equilibrate` sweeps).  Each step takes a minibatch of `batch` consecutive
    configurations, regresses the block logits on min(0, -beta dE_b) and takes
    an Adam step.  This function only sequences library calls; every
    arithmetic step runs in the kernels.  Returns {"params", "loss", "steps"}.
    """
    import numpy as np
    import torch

    # every copy, fill and read of this function in the stream order of the library calls
    with _on_stream(stream):
        n_chains = min(n_configs, 1024)
        gen = Batch([L] * n_chains, 1, [beta], device=device)
        gen.init(ISING_INIT_RANDOM, seed, stream)
        gen.run(equilibrate, seed, 0, 0, False, None, True, stream)
        words = L * L // 32
        data_b = torch.empty((n_configs, words * 8), dtype=torch.uint8, device=device)
        data_w = torch.empty_like(data_b)
        t, got = equilibrate, 0
        while got < n_configs:
            take = min(n_chains, n_configs - got)
            nbytes = 8 * words * take
            data_b[got:got + take].copy_(gen.ws[gen._black_off:gen._black_off + nbytes].view(take, words * 8))
            data_w[got:got + take].copy_(gen.ws[gen._white_off:gen._white_off + nbytes].view(take, words * 8))
            got += take
            gen.run(sweeps_between, seed, t, 0, False, None, True, stream)
            t += sweeps_between
        del gen
        rng = np.random.default_rng(seed)
        n_par = ising_net_param_count()
        theta = np.zeros(n_par, dtype=np.float32)
        o = 0
        for size, fan_in, is_w in ((32 * 9, 9, True), (32, 0, False), (32 * 32 * 9, 288, True), (32, 0, False),
                                   (32 * 32 * 9, 288, True), (32, 0, False), (32 * 9, 288, True), (1, 0, False)):
            if is_w:
                theta[o:o + size] = rng.normal(0.0, np.sqrt(2.0 / fan_in), size)
            o += size
        params = torch.from_numpy(theta).to(device)
        m = torch.zeros_like(params)
        v = torch.zeros_like(params)
        grad = torch.zeros_like(params)
        nb = (L // 8) ** 2
        work = torch.empty(ising_net_workspace_bytes(L, batch, True), dtype=torch.uint8, device=device)
        logits = torch.zeros((batch, nb), dtype=torch.float32, device=device)
        dlogits = torch.zeros_like(logits)
        chain_sq = torch.zeros(batch, dtype=torch.float32, device=device)
        loss = torch.zeros(1, dtype=torch.float32, device=device)
        n_mb = n_configs // batch
        order = rng.permutation(n_mb)
        history = []
        for step in range(1, steps + 1):
            i0 = int(order[(step - 1) % n_mb]) * batch
            blk, wht = data_b[i0:i0 + batch], data_w[i0:i0 + batch]
            ising_net_forward(L, batch, blk, wht, None, params, logits, work, True, stream)
            ising_net_targets_loss(L, batch, blk, wht, beta, logits, dlogits, chain_sq, loss, stream)
            ising_net_backward(L, batch, blk, wht, params, dlogits, grad, work, stream)
            ising_net_adam(params, grad, m, v, step, lr, stream)
            if step == 1 or step % log_every == 0 or step == steps:
                history.append(float(loss.item()))
        return {"params": params, "loss": history, "steps": steps}
