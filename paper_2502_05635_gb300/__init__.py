"""Python binding of the GB300 TD-aGW library (libtdagw.so, C ABI in include/tdagw.h).

Argument marshalling only: every computation runs in the library's CUDA kernels.  The
module-level functions carry the C names one-to-one; ``Context`` is a small convenience
wrapper over them.  Host arrays are numpy (complex128 / float64, C-contiguous); device
arrays are torch CUDA tensors (passed by data pointer).  There is no fallback: if the
library is missing, importing the names works but every call raises ``TdagwError``.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtdagw.so")

OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_NOT_BUILT, ERR_NO_FACTORS, ERR_TIMEOUT, \
    ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7
C64, C128 = 0, 1
FULL, LOWRANK, CHANNEL = 0, 1, 2
FIELD_GAUSS_COS, FIELD_CONST, FIELD_SIN2_SIN, FIELD_TABLE = 0, 1, 2, 3
FLAG_RESET, FLAG_NO_GRAPH, FLAG_NO_KAHAN, FLAG_STAGEWISE, FLAG_TEST_TIMEOUT, FLAG_CHECKPOINT, \
    FLAG_SPLIT_F16 = 1, 2, 4, 8, 16, 32, 64


class TdagwError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"tdagw error {code}: {msg}")
        self.code = code


class ModelDesc(ct.Structure):
    _fields_ = [("L", ct.c_int), ("nb_copies", ct.c_int), ("offsets", ct.c_double * 4),
                ("Delta", ct.c_double), ("t", ct.c_double), ("m", ct.c_double),
                ("a", ct.c_double), ("r0", ct.c_double), ("dtype", ct.c_int),
                ("exchange", ct.c_double)]


class Field(ct.Structure):
    _fields_ = [("kind", ct.c_int), ("E0", ct.c_double), ("omega", ct.c_double),
                ("t0", ct.c_double), ("sigma", ct.c_double), ("T_pulse", ct.c_double),
                ("dir_x", ct.c_double), ("dir_y", ct.c_double),
                ("table", ct.POINTER(ct.c_double))]


_P = ct.c_void_p
_D = ct.POINTER(ct.c_double)
_I64 = ct.POINTER(ct.c_int64)
_SIGS = {
    "tdagw_create": [ct.POINTER(ModelDesc), _P, ct.POINTER(_P)],
    "tdagw_build_kernel": [_P],
    "tdagw_model_info": [_P, _I64, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int)],
    "tdagw_get_model": [_P, _D, _D, _D, _D, _D],
    "tdagw_get_kernel_entries": [_P, _I64, _I64, ct.c_int64, _D],
    "tdagw_compress_svd": [_P, ct.c_int, ct.c_int, ct.c_int, ct.c_uint64, ct.c_int],
    "tdagw_set_factors": [_P, ct.c_int, _D, _D, _D, _D],
    "tdagw_get_factors": [_P, ct.POINTER(ct.c_int), _D, _D, _D, _D],
    "tdagw_set_kdiag_blocks": [_P, ct.c_int],
    "tdagw_compress_channels": [_P, ct.c_int, ct.c_int, ct.c_int, ct.c_uint64, ct.c_double],
    "tdagw_set_channel_factors": [_P, ct.c_int, ct.POINTER(ct.c_int), _D, _D, _D, _D],
    "tdagw_get_channel_factors": [_P, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int), _D, _D, _D, _D],
    "tdagw_apply": [_P, ct.c_int, _P, _P],
    "tdagw_propagate": [_P, ct.POINTER(Field), ct.c_int, ct.POINTER(ct.c_int), ct.c_double,
                        ct.c_int, ct.c_int],
    "tdagw_observables": [_P, _D, ct.c_int64, _I64, ct.c_int],
    "tdagw_get_state": [_P, _D, _D, _I64],
    "tdagw_set_state": [_P, _D, _D, ct.c_int64],
    "tdagw_sync": [_P],
    "tdagw_apply_lowrank_noalloc": [_P, _P, ct.c_int64, _P, _P, ct.c_int64, ct.c_int, _P, _P, _P],
    "tdagw_adjoint": [_P, _D, _D, _D],
    "tdagw_hhg_spectrum": [_D, ct.c_int64, ct.c_int64, ct.c_int, ct.POINTER(ct.c_int), ct.c_double, _D,
                           ct.c_int, _D, _P],
}
EXPORTED = sorted(list(_SIGS) + ["tdagw_last_error", "tdagw_destroy"])

_lib = None


def lib() -> ct.CDLL:
    """Load libtdagw.so (built by build.py / __graft_entry__.build()); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise TdagwError(ERR_UNSUPPORTED, f"{LIB_PATH} not built; run build.py")
        L = ct.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ct.c_int
        L.tdagw_last_error.argtypes = []
        L.tdagw_last_error.restype = ct.c_char_p
        L.tdagw_destroy.argtypes = [_P]
        L.tdagw_destroy.restype = None
        _lib = L
    return _lib


def _check(rc: int):
    if rc != OK:
        raise TdagwError(rc, lib().tdagw_last_error().decode())


def _dptr(a):
    """double* of a C-contiguous numpy float64/complex128 array (or None)."""
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"] and a.dtype in (np.float64, np.complex128)
    return a.ctypes.data_as(_D)


def _devptr(t) -> int:
    if not t.is_cuda:
        raise TdagwError(ERR_INVALID_ARG, "expected a CUDA tensor")
    return t.data_ptr()


def _need(cond: bool, msg: str):
    """Argument check of the binding: the C side cannot see the extent of a host or device
    array, so shapes are checked here before any pointer is passed."""
    if not cond:
        raise TdagwError(ERR_INVALID_ARG, msg)


def _dev_vec(t, n: int, dtype, name: str):
    """A contiguous CUDA-or-host tensor of n elements of dtype (device checked last)."""
    _need(t.dtype == dtype, f"{name} must be {dtype}")
    _need(t.is_contiguous() and t.numel() == n, f"{name} must be contiguous with {n} elements")


# per-handle facts the binding needs for its checks: dtype, K^diag reading, last batch size
_CTX_INFO: dict[int, dict] = {}


# ---------------------------------------------------------------- one-to-one names ------

def tdagw_create(desc: ModelDesc, stream: int | None = None) -> int:
    """New context for one model (no device memory yet); returns the handle.  stream: a
    cudaStream_t as an int (None: the legacy default stream)."""
    h = _P()
    _check(lib().tdagw_create(ct.byref(desc), _P(stream or 0), ct.byref(h)))
    _CTX_INFO[h.value] = {"dtype": int(desc.dtype), "kdiag": 0, "B": 1}
    return h.value


def tdagw_build_kernel(ctx: int):
    """Builds the model on the host and the dense kernel K on the device (Eq. bse-direct-def,
    plus the exchange term when the model has one)."""
    _check(lib().tdagw_build_kernel(_P(ctx)))


def tdagw_model_info(ctx: int):
    """(N, Nb, Nk) of the context's model (no GPU needed)."""
    n, nb, nk = ct.c_int64(), ct.c_int(), ct.c_int()
    _check(lib().tdagw_model_info(_P(ctx), ct.byref(n), ct.byref(nb), ct.byref(nk)))
    return n.value, nb.value, nk.value


def tdagw_get_model(ctx: int):
    """Host copies of the built model: eps (Nk, Nb), dx, dy, vx and U (Nk, Nb, Nb)."""
    N, Nb, Nk = tdagw_model_info(ctx)
    eps = np.empty(Nk * Nb)
    dx, dy, vx, U = (np.empty(Nk * Nb * Nb, np.complex128) for _ in range(4))
    _check(lib().tdagw_get_model(_P(ctx), _dptr(eps), _dptr(dx), _dptr(dy), _dptr(vx), _dptr(U)))
    sh = (Nk, Nb, Nb)
    return dict(eps=eps.reshape(Nk, Nb), dx=dx.reshape(sh), dy=dy.reshape(sh),
                vx=vx.reshape(sh), U=U.reshape(sh))


def tdagw_get_kernel_entries(ctx: int, rows, cols) -> np.ndarray:
    """K[rows[i], cols[i]] from the device kernel, complex128."""
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    out = np.empty(rows.size, np.complex128)
    _check(lib().tdagw_get_kernel_entries(_P(ctx), rows.ctypes.data_as(_I64),
                                          cols.ctypes.data_as(_I64), rows.size, _dptr(out)))
    return out


def tdagw_compress_svd(ctx: int, rank: int, oversample: int = 64, power_iters: int = 2,
                       seed: int = 1, precision: int = 0):
    """Randomised truncated SVD of K^off on the device (Eq. svd_diag_offdiag); precision 1
    also emits split-FP16 factors for TDAGW_FLAG_SPLIT_F16."""
    _check(lib().tdagw_compress_svd(_P(ctx), rank, oversample, power_iters, seed, precision))


def tdagw_set_factors(ctx: int, U, S, V, diag=None):
    """U, V: (N, rank) complex; S: (rank,); diag: (N,), or (Nk, P, P) with the k-block
    reading of K^diag, or None (taken from the built kernel)."""
    U = np.ascontiguousarray(U, np.complex128)
    V = np.ascontiguousarray(V, np.complex128)
    S = np.ascontiguousarray(S, np.float64)
    d = None if diag is None else np.ascontiguousarray(diag, np.complex128)
    N, Nb, Nk = tdagw_model_info(ctx)
    _need(U.ndim == 2 and U.shape[0] == N, f"U must be (N = {N}, rank)")
    _need(V.shape == U.shape, "V must have the shape of U")
    _need(S.shape == (U.shape[1],), "S must be (rank,)")
    if d is not None:
        nd = Nk * Nb ** 4 if _CTX_INFO.get(ctx, {}).get("kdiag") else N
        _need(d.size == nd, f"diag must have {nd} entries")
    _check(lib().tdagw_set_factors(_P(ctx), U.shape[1], _dptr(U), _dptr(S), _dptr(V), _dptr(d)))


def tdagw_set_kdiag_blocks(ctx: int, on: int):
    """Selects the reading of K^diag: 0 the strict diagonal, 1 the k = k' blocks (removes
    installed low-rank factors when it changes)."""
    _check(lib().tdagw_set_kdiag_blocks(_P(ctx), int(on)))
    _CTX_INFO.setdefault(ctx, {})["kdiag"] = int(on)


def tdagw_get_factors(ctx: int, kblocks: bool = False):
    """(U, S, V, diag); with kblocks (the k-block reading of K^diag is on) diag is the
    (Nk, P, P) array of k = k' blocks."""
    N, Nb, Nk = tdagw_model_info(ctx)
    r = ct.c_int()
    _check(lib().tdagw_get_factors(_P(ctx), ct.byref(r), None, None, None, None))
    r = r.value
    U = np.empty((N, r), np.complex128)
    V = np.empty((N, r), np.complex128)
    S = np.empty(r)
    d = np.empty((Nk, Nb * Nb, Nb * Nb) if kblocks else N, np.complex128)
    _check(lib().tdagw_get_factors(_P(ctx), None, _dptr(U), _dptr(S), _dptr(V), _dptr(d)))
    return U, S, V, d


def tdagw_compress_channels(ctx: int, rank: int, oversample: int = 64, power_iters: int = 2,
                            seed: int = 1, rel_tol: float = 0.0):
    """Channel-wise compression (Eq. svd-channel-wise): a randomised SVD of every off-diagonal
    channel, rank <= `rank`, dropping singular values below rel_tol of the channel's largest."""
    _check(lib().tdagw_compress_channels(_P(ctx), rank, oversample, power_iters, seed, rel_tol))


def tdagw_set_channel_factors(ctx: int, U, S, V, D=None, ranks=None):
    """U, V: (P, P, Nk, r) complex; S: (P, P, r); D: (P, Nk, Nk) or None; ranks: (P, P)
    ints or None (every off-diagonal channel rank r)."""
    U = np.ascontiguousarray(U, np.complex128)
    V = np.ascontiguousarray(V, np.complex128)
    S = np.ascontiguousarray(S, np.float64)
    d = None if D is None else np.ascontiguousarray(D, np.complex128)
    _, Nb, Nk = tdagw_model_info(ctx)
    P = Nb * Nb
    _need(U.ndim == 4 and U.shape[:3] == (P, P, Nk), f"U must be (P, P, Nk, rank) = ({P}, {P}, {Nk}, rank)")
    _need(V.shape == U.shape, "V must have the shape of U")
    _need(S.shape == (P, P, U.shape[3]), "S must be (P, P, rank)")
    _need(d is None or d.shape == (P, Nk, Nk), f"D must be (P, Nk, Nk) = ({P}, {Nk}, {Nk})")
    rk = None
    if ranks is not None:
        ra = np.ascontiguousarray(ranks, np.int32)
        _need(ra.shape == (P, P), f"ranks must be (P, P) = ({P}, {P})")
        rk = ra.ctypes.data_as(ct.POINTER(ct.c_int))
    _check(lib().tdagw_set_channel_factors(_P(ctx), U.shape[-1], rk, _dptr(U), _dptr(S), _dptr(V),
                                           _dptr(d)))


def tdagw_get_channel_factors(ctx: int, arrays: bool = True):
    """(ranks (P, P), U, S, V, D) in the layout of tdagw_set_channel_factors; with
    arrays=False only the ranks."""
    _, Nb, Nk = tdagw_model_info(ctx)
    P = Nb * Nb
    r = ct.c_int()
    ranks = np.zeros((P, P), np.int32)
    if not arrays:
        _check(lib().tdagw_get_channel_factors(_P(ctx), ct.byref(r), ranks.ctypes.data_as(ct.POINTER(ct.c_int)),
                                               None, None, None, None))
        return ranks
    _check(lib().tdagw_get_channel_factors(_P(ctx), ct.byref(r), None, None, None, None, None))
    r = r.value
    U = np.empty((P, P, Nk, r), np.complex128)
    V = np.empty((P, P, Nk, r), np.complex128)
    S = np.empty((P, P, r))
    D = np.empty((P, Nk, Nk), np.complex128)
    _check(lib().tdagw_get_channel_factors(_P(ctx), None, ranks.ctypes.data_as(ct.POINTER(ct.c_int)),
                                           _dptr(U), _dptr(S), _dptr(V), _dptr(D)))
    return ranks, U, S, V, D


def tdagw_apply(ctx: int, mode: int, x, y):
    """y = K x on the device: x, y contiguous CUDA tensors of N complex64 (C64 context) or
    complex128 (C128) entries."""
    import torch
    N = tdagw_model_info(ctx)[0]
    dt = torch.complex128 if _CTX_INFO.get(ctx, {}).get("dtype") == C128 else torch.complex64
    _dev_vec(x, N, dt, "x")
    _dev_vec(y, N, dt, "y")
    _check(lib().tdagw_apply(_P(ctx), mode, _P(_devptr(x)), _P(_devptr(y))))


def make_field(pulse, table=None) -> Field:
    """Field struct from an object with E0, omega, t0, sigma, T_pulse, dir_x, dir_y, kind."""
    f = Field(kind=int(pulse.kind), E0=pulse.E0, omega=pulse.omega, t0=pulse.t0,
              sigma=pulse.sigma, T_pulse=pulse.T_pulse, dir_x=pulse.dir_x, dir_y=pulse.dir_y)
    if table is not None:
        table = np.ascontiguousarray(table, np.float64)
        f.kind = FIELD_TABLE
        f.table = _dptr(table)
        f._table = table  # keeps the samples alive and lets tdagw_propagate check their count
    return f


def tdagw_propagate(ctx: int, fields, steps, dt: float, mode: int, flags: int = FLAG_RESET):
    """B = len(fields) trajectories of steps[b] RK4 steps; a table field (make_field with a
    table) needs E(j dt / 2) for j = 0 .. 2 steps[b]."""
    fields, steps = list(fields), list(steps)
    _need(len(steps) == len(fields), "one step count per field")
    for f, n in zip(fields, steps):
        tab = getattr(f, "_table", None)
        if f.kind == FIELD_TABLE and tab is not None:
            _need(tab.size >= 2 * int(n) + 1, "a table field needs 2 steps + 1 samples")
    arr = (Field * len(fields))(*fields)
    st = (ct.c_int * len(steps))(*[int(s) for s in steps])
    _check(lib().tdagw_propagate(_P(ctx), arr, len(fields), st, float(dt), mode, flags))
    _CTX_INFO.setdefault(ctx, {})["B"] = len(fields)


def tdagw_observables(ctx: int, out=None, B: int = 1) -> np.ndarray:
    """Observables of the last propagate: (rows, 3) for one trajectory, (rows, B, 3) for B."""
    rows = ct.c_int64()
    _check(lib().tdagw_observables(_P(ctx), None, 0, ct.byref(rows), 1))
    if out is None:
        out = np.empty((rows.value, 3) if B == 1 else (rows.value, B, 3))
    last_B = _CTX_INFO.get(ctx, {}).get("B", B)
    _need(out.dtype == np.float64 and out.flags["C_CONTIGUOUS"], "out must be C-contiguous float64")
    _need(out.size >= min(out.shape[0], rows.value) * last_B * 3,
          f"out rows must hold the {last_B} x 3 observables of the last propagate")
    _check(lib().tdagw_observables(_P(ctx), _dptr(out), out.shape[0], ct.byref(rows), 1))
    return out


def tdagw_get_state(ctx: int):
    """(drho, Kahan carry, step) of the single-trajectory state, complex128 host arrays."""
    N = tdagw_model_info(ctx)[0]
    drho = np.empty(N, np.complex128)
    carry = np.empty(N, np.complex128)
    step = ct.c_int64()
    _check(lib().tdagw_get_state(_P(ctx), _dptr(drho), _dptr(carry), ct.byref(step)))
    return drho, carry, step.value


def tdagw_set_state(ctx: int, drho, carry=None, step: int = 0):
    """Installs a single-trajectory state (to resume a run); carry None means zero."""
    drho = np.ascontiguousarray(drho, np.complex128)
    c = None if carry is None else np.ascontiguousarray(carry, np.complex128)
    N = tdagw_model_info(ctx)[0]
    _need(drho.size == N and (c is None or c.size == N), f"drho and carry must have N = {N} entries")
    _check(lib().tdagw_set_state(_P(ctx), _dptr(drho), _dptr(c), int(step)))


def tdagw_apply_lowrank_noalloc(U, V, S, diag, x, y, stream: int | None = None):
    """Allocation-free low-rank contraction on caller-owned CUDA tensors: U, V complex64
    (N, ld) with ld even, S float32 (rank,), diag/x/y complex64 (N,); rank = len(S)."""
    import torch
    _need(U.dim() == 2 and U.dtype == torch.complex64 and U.is_contiguous(), "U must be contiguous complex64 (N, ld)")
    N, ld = U.shape
    _need(V.shape == U.shape and V.dtype == torch.complex64 and V.is_contiguous(), "V must match U")
    _need(S.dim() == 1 and S.dtype == torch.float32 and S.is_contiguous() and S.shape[0] <= ld,
          "S must be contiguous float32 (rank,) with rank <= ld")
    for t, name in ((diag, "diag"), (x, "x"), (y, "y")):
        _dev_vec(t, N, torch.complex64, name)
    ptrs = [_devptr(t) for t in (U, V, S, diag, x, y)]          # CUDA tensors only
    devs = {t.device for t in (U, V, S, diag, x, y)}
    _need(len(devs) == 1, "all tensors must be on one device")
    # the library launches on the current device: make it the tensors' device
    with torch.cuda.device(U.device):
        _check(lib().tdagw_apply_lowrank_noalloc(
            _P(ptrs[0]), _P(ptrs[1]), ld, _P(ptrs[2]), _P(ptrs[3]), N, S.shape[0],
            _P(ptrs[4]), _P(ptrs[5]), _P(stream or 0)))


def tdagw_adjoint(ctx: int, dJdobs, steps_max: int, B: int):
    """Gradients through the last checkpointed propagate: returns (dJ/dE_j of shape
    (2 steps_max + 1, B), dJ/d(E0, omega, t0, sigma) of shape (B, 4))."""
    rows = ct.c_int64()
    _check(lib().tdagw_observables(_P(ctx), None, 0, ct.byref(rows), 1))
    _need(steps_max + 1 == rows.value and B == _CTX_INFO.get(ctx, {}).get("B", B),
          "steps_max and B must be those of the last checkpointed propagate")
    d = np.ascontiguousarray(dJdobs, np.float64).reshape(steps_max + 1, B, 3)
    gE = np.empty((2 * steps_max + 1, B))
    gp = np.empty((B, 4))
    _check(lib().tdagw_adjoint(_P(ctx), _dptr(d), _dptr(gE), _dptr(gp)))
    return gE, gp


def tdagw_hhg_spectrum(J, steps, dt: float, omega, component: int | None = None,
                       stream: int | None = None) -> np.ndarray:
    """HHG spectra of B currents: J is (rows, B) or, with `component`, the (rows, B, 3)
    observables array (component 1 = J).  Returns (nfreq, B)."""
    J = np.ascontiguousarray(J, np.float64)
    _need(J.ndim == (2 if component is None else 3), "J must be (rows, B), or (rows, B, 3) with a component")
    rows, B = J.shape[0], J.shape[1]
    _need(component is None or 0 <= int(component) < J.shape[2], "component out of range")
    stride, off = (1, 0) if component is None else (J.shape[2], int(component))
    flat = J.reshape(-1)[off:]
    flat = np.ascontiguousarray(flat) if off else flat
    st = np.ascontiguousarray(steps, np.int32)
    _need(st.shape == (B,), "one step count per current")
    w = np.ascontiguousarray(omega, np.float64)
    out = np.empty((w.size, B))
    _check(lib().tdagw_hhg_spectrum(_dptr(flat), rows, stride, B, st.ctypes.data_as(ct.POINTER(ct.c_int)),
                                    float(dt), _dptr(w), w.size, _dptr(out), _P(stream or 0)))
    return out


def tdagw_sync(ctx: int):
    """Waits for the context's stream; raises TDAGW_ERR_TIMEOUT if a bounded device wait
    of the last propagation gave up."""
    _check(lib().tdagw_sync(_P(ctx)))


def tdagw_last_error() -> str:
    """Message of the last failing call on this thread."""
    return lib().tdagw_last_error().decode()


def tdagw_destroy(ctx: int):
    """Frees the context and everything it allocated."""
    lib().tdagw_destroy(_P(ctx))
    _CTX_INFO.pop(ctx, None)


# ---------------------------------------------------------------- convenience -----------

def model_desc(p, dtype: int = C64) -> ModelDesc:
    """ModelDesc from an object with L, nb_copies, offsets, Delta, t, m, a, r0 (and
    optionally exchange)."""
    offs = list(p.offsets) + [0.0] * (4 - len(p.offsets))
    return ModelDesc(L=p.L, nb_copies=p.nb_copies, offsets=(ct.c_double * 4)(*offs[:4]),
                     Delta=p.Delta, t=p.t, m=p.m, a=p.a, r0=p.r0, dtype=dtype,
                     exchange=float(getattr(p, "exchange", 0.0)))


def propagate_autograd(context: "Context", params, pulses, steps, dt: float, mode: int = 1):
    """P_x(t) of B trajectories as a differentiable function of their Gaussian * cos pulse
    parameters params (B x 4 torch float64: E0, omega, t0, sigma).  Forward: one batched
    checkpointed propagation; backward: the library's discrete adjoint.  Returns a
    (max steps + 1, B) float64 tensor (NaN after each trajectory's end)."""
    import dataclasses

    import torch

    class _Fn(torch.autograd.Function):
        @staticmethod
        def forward(fctx, p):
            pv = p.detach().cpu().numpy()
            ps = [dataclasses.replace(pl, E0=float(v[0]), omega=float(v[1]), t0=float(v[2]),
                                      sigma=float(v[3]), kind=FIELD_GAUSS_COS)
                  for pl, v in zip(pulses, pv)]
            tdagw_propagate(context.h, [make_field(q) for q in ps], list(steps), dt, mode,
                            FLAG_RESET | FLAG_CHECKPOINT)
            obs = tdagw_observables(context.h, B=len(ps))
            return torch.from_numpy(obs[:, :, 0].copy())

        @staticmethod
        def backward(fctx, gP):
            g = gP.detach().cpu().numpy()
            d = np.zeros(g.shape + (3,))
            d[:, :, 0] = np.nan_to_num(g)
            _, gp = tdagw_adjoint(context.h, d, g.shape[0] - 1, g.shape[1])
            return torch.from_numpy(gp)

    return _Fn.apply(params)


class Context:
    """Owns one library context; methods forward to the tdagw_* functions."""

    def __init__(self, params, dtype: int = C64, stream: int | None = None, build: bool = True):
        self.h = tdagw_create(model_desc(params, dtype), stream)
        self.dtype = dtype
        if build:
            tdagw_build_kernel(self.h)
        self.N, self.Nb, self.Nk = tdagw_model_info(self.h)

    def close(self):
        if self.h:
            tdagw_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def propagate(self, pulse, steps: int, dt: float, mode: int = FULL, flags: int = FLAG_RESET,
                  table=None) -> np.ndarray:
        tdagw_propagate(self.h, [make_field(pulse, table)], [steps], dt, mode, flags)
        return tdagw_observables(self.h)

    def propagate_batch(self, pulses, steps, dt: float, mode: int = LOWRANK,
                        flags: int = FLAG_RESET) -> np.ndarray:
        """B trajectories in one launch; returns (max steps + 1, B, 3), NaN after the end."""
        tdagw_propagate(self.h, [make_field(p) for p in pulses], list(steps), dt, mode, flags)
        return tdagw_observables(self.h, B=len(pulses))
