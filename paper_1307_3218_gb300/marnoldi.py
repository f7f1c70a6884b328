"""Python binding of libmarnoldi (include/marnoldi.h): argument marshalling only.

Every function keeps the C name and forwards to the library through ctypes;
the work runs in the library's CUDA kernels.  There is no fallback: if the
library is not built or cannot be loaded, the first call raises.

PyTorch is used only as plumbing: the CUDA stream the library issues its work
on (``torch.cuda.current_stream()`` unless one is given) and, through
``marnoldi_set_allocator``, the caching allocator that backs the library's
device memory.
"""

from __future__ import annotations

import atexit
import ctypes as C
import os
import weakref

import numpy as np

from . import build as _build

MARNOLDI_OK = 0
MARNOLDI_EINVAL = -1
MARNOLDI_ENOTSPD = -2
MARNOLDI_ENOMEM = -3
MARNOLDI_ECUDA = -4
MARNOLDI_ETIMEOUT = -5
MARNOLDI_ESTATE = -6
MARNOLDI_ENOCONV = -7
MARNOLDI_EPENDING = -8
MARNOLDI_FP64 = 0
MARNOLDI_MIXED = 1
MARNOLDI_COUNT_NOALLOC_MAX_LEVELS = 16777216   # include/marnoldi.h

STATUS_NAMES = {0: "OK", -1: "EINVAL", -2: "ENOTSPD", -3: "ENOMEM", -4: "ECUDA", -5: "ETIMEOUT",
                -6: "ESTATE", -7: "ENOCONV", -8: "EPENDING"}

_LIB = None
_ALLOC_CB = None     # keep the ctypes callbacks alive
_FREE_CB = None
_KEEP_ALIVE: list = []

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class MarnoldiError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {message}")
        self.code = code


def library_path() -> str:
    """The library load() opens: $MARNOLDI_LIB if set (another build of the same sources, such as
    the index-check variant), else the default build."""
    return os.environ.get("MARNOLDI_LIB") or _build.lib_path()


def load(path: str | None = None):
    """Load libmarnoldi (building it first when MARNOLDI_BUILD=1)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    p = path or library_path()
    if not os.path.exists(p):
        if os.environ.get("MARNOLDI_BUILD", "0") == "1":
            p = _build.build()
        else:
            raise RuntimeError(
                f"libmarnoldi is not built ({p} missing); run paper_1307_3218_gb300.build.build() "
                "or __graft_entry__.build()")
    L = C.CDLL(p)
    P, i64, i32, d = C.c_void_p, C.c_int64, C.c_int, C.c_double
    sig = {
        "marnoldi_set_allocator": (i32, [ALLOC_FN, FREE_FN, P]),
        "marnoldi_setup": (i32, [C.POINTER(P), i64, P, P, P, P, P, P, P, i32, P]),
        "marnoldi_solve": (i32, [P, P, i64, i32, i32, d, d, P]),
        "marnoldi_density": (i32, [P, P, P]),
        "marnoldi_density_device": (i32, [P, P, P]),
        "marnoldi_energy": (i32, [P, P, P, P]),
        "marnoldi_level_range": (i32, [P, P, P]),
        "marnoldi_fermi_at": (i32, [P, d, d, P, P]),
        "marnoldi_green": (i32, [P, P, i32, P]),
        "marnoldi_column_stats": (i32, [P, P, P, P]),
        "marnoldi_solved_shape": (i32, [P, P, P]),
        "marnoldi_set_batch": (i32, [P, i64]),
        "marnoldi_set_profiling": (i32, [P, i32]),
        "marnoldi_set_krylov_graph": (i32, [P, i32]),
        "marnoldi_krylov_graph_launches": (i32, [P, P]),
        "marnoldi_kernel_kinds": (i32, []),
        "marnoldi_kernel_stats": (i32, [P, i32, C.POINTER(C.c_char_p), C.POINTER(i64),
                                        C.POINTER(d), i32]),
        "marnoldi_count_noalloc": (i32, [P, P, P, i64, i32, d, d, P, P]),
        "marnoldi_forces": (i32, [P, P, P, P]),
        "marnoldi_eigenstate": (i32, [P, i64, d, P, P, P]),
        "marnoldi_set_members": (i32, [P, i32, P, P]),
        "marnoldi_member_energy": (i32, [P, i32, P, P, P]),
        "marnoldi_set_member_temperatures": (i32, [P, i32, P]),
        "marnoldi_set_autotune": (i32, [i32]),
        "marnoldi_gs_shape": (i32, [P, P, P]),
        "marnoldi_check_status": (i32, [P, P, P]),
        "marnoldi_device_bytes": (i32, [P, P, P]),
        "marnoldi_footprint": (i32, [i64, P, P, P, i32, i32, i32, i64, P, P]),
        "marnoldi_server_create": (i32, [C.POINTER(P), i32, C.c_size_t]),
        "marnoldi_server_submit": (i32, [P, i64, P, P, P, P, P, P, P, i32, i32, i32, d, d, i64, P, P,
                                         P]),
        "marnoldi_server_wait": (i32, [P, i64, d, P, P, P, C.c_size_t]),
        "marnoldi_server_stats": (i32, [P, P]),
        "marnoldi_server_set_group_limit": (i32, [P, i32]),
        "marnoldi_server_last_error": (C.c_char_p, []),
        "marnoldi_server_destroy": (None, [P]),
        "marnoldi_last_error": (C.c_char_p, [P]),
        "marnoldi_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _LIB = L
    return L


def _check(rc: int, ctx=None):
    if rc != MARNOLDI_OK:
        msg = load().marnoldi_last_error(ctx.handle if ctx is not None else None)
        raise MarnoldiError(rc, msg.decode() if msg else "")


def _ptr(a) -> C.c_void_p:
    if a is None:
        return None
    if isinstance(a, int):
        return C.c_void_p(a)
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return 0


_LIVE = weakref.WeakSet()


class Context:
    """Owns one ``marnoldi_ctx``; destroyed with the object or by marnoldi_destroy."""

    def __init__(self, handle: int, nnzb: int, n_block_rows: int, stream: int):
        self.handle = C.c_void_p(handle)
        self.nnzb = nnzb
        self.n_block_rows = n_block_rows
        self.stream = stream
        _LIVE.add(self)

    def __del__(self):
        try:
            marnoldi_destroy(self)
        except Exception:
            pass


@atexit.register
def _destroy_all():
    # free device memory while PyTorch (which may back it) is still alive
    for ctx in list(_LIVE):
        try:
            marnoldi_destroy(ctx)
        except Exception:
            pass


def marnoldi_set_allocator(alloc=None, free=None, user=None) -> None:
    """Install a device allocator (Python callables) or restore the default (None, None)."""
    global _ALLOC_CB, _FREE_CB
    L = load()
    if alloc is None:
        _ALLOC_CB = ALLOC_FN()
        _FREE_CB = FREE_FN()
        _check(L.marnoldi_set_allocator(C.cast(None, ALLOC_FN), C.cast(None, FREE_FN), None))
        return
    _ALLOC_CB = ALLOC_FN(alloc)
    _FREE_CB = FREE_FN(free)
    # contexts keep the hooks they were created with: never let a callback die
    _KEEP_ALIVE.append((_ALLOC_CB, _FREE_CB))
    _check(L.marnoldi_set_allocator(_ALLOC_CB, _FREE_CB, user))


def use_torch_allocator() -> None:
    """Back the library's device memory with PyTorch's caching allocator."""
    import torch

    def _alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      int(stream or 0))
        except Exception:
            return None

    def _free(ptr, nbytes, stream, user):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass

    marnoldi_set_allocator(_alloc, _free)


_ALLOCATOR_CHOSEN = False


def _default_allocator():
    """On first setup, route device memory through PyTorch's caching allocator
    (MARNOLDI_ALLOCATOR=native keeps the library's cudaMallocAsync pool)."""
    global _ALLOCATOR_CHOSEN
    if _ALLOCATOR_CHOSEN:
        return
    _ALLOCATOR_CHOSEN = True
    if os.environ.get("MARNOLDI_ALLOCATOR", "torch") == "native":
        return
    try:
        import torch
        ok = torch.cuda.is_available()
    except Exception:
        ok = False
    if ok:
        use_torch_allocator()


def marnoldi_setup(n_block_rows: int, row_ptr, col_idx, H_vals, S_vals, orbital_mask=None,
                   positions=None, box=None, precision: int = MARNOLDI_FP64,
                   stream: int | None = None) -> Context:
    L = load()
    _default_allocator()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    H = np.ascontiguousarray(H_vals, dtype=np.float64)
    S = np.ascontiguousarray(S_vals, dtype=np.float64)
    mask = None if orbital_mask is None else np.ascontiguousarray(orbital_mask, dtype=np.uint8)
    pos = None if positions is None else np.ascontiguousarray(positions, dtype=np.float64)
    bx = None if box is None else np.ascontiguousarray(box, dtype=np.float64)
    if rp.size != n_block_rows + 1:
        raise MarnoldiError(MARNOLDI_EINVAL, "row_ptr must have n_block_rows + 1 entries")
    nnzb = int(rp[-1])
    if ci.size != nnzb or H.size != 16 * nnzb or S.size != 16 * nnzb:
        raise MarnoldiError(MARNOLDI_EINVAL, "col_idx / H_vals / S_vals sizes do not match row_ptr")
    if mask is not None and mask.size != 4 * n_block_rows:
        raise MarnoldiError(MARNOLDI_EINVAL, "orbital_mask must have 4 n_block_rows entries")
    st = _current_stream() if stream is None else int(stream)
    out = C.c_void_p()
    rc = L.marnoldi_setup(C.byref(out), int(n_block_rows), _ptr(rp), _ptr(ci), _ptr(H), _ptr(S),
                          _ptr(mask), _ptr(pos), _ptr(bx), int(precision), C.c_void_p(st))
    _check(rc)
    return Context(out.value, nnzb, int(n_block_rows), st)


def setup_system(sysm, precision: int = MARNOLDI_FP64, stream: int | None = None) -> Context:
    """marnoldi_setup for a tbsynth.TBSystem-like object."""
    s = getattr(sysm, "structure", None)
    return marnoldi_setup(sysm.n_block_rows, sysm.row_ptr, sysm.col_idx, sysm.H, sysm.S,
                          sysm.orbital_mask, None if s is None else s.positions,
                          None if s is None else s.box, precision, stream)


def marnoldi_solve(ctx: Context, columns=None, nu: int = 30, region_atoms: int = 0,
                   electron_count: float = 0.0, kT: float = 0.1, mu_fixed: float | None = None):
    L = load()
    if columns is None:
        cp, nc = None, -1
        cols = None
    else:
        cols = np.ascontiguousarray(columns, dtype=np.int64)
        cp, nc = _ptr(cols), cols.size
    mu = None if mu_fixed is None else C.byref(C.c_double(float(mu_fixed)))
    _check(L.marnoldi_solve(ctx.handle, cp, nc, int(nu), int(region_atoms), float(electron_count),
                            float(kT), mu), ctx)


def marnoldi_density(ctx: Context) -> tuple[np.ndarray, np.ndarray]:
    rho = np.empty((ctx.nnzb, 4, 4))
    rhoE = np.empty((ctx.nnzb, 4, 4))
    _check(load().marnoldi_density(ctx.handle, _ptr(rho), _ptr(rhoE)), ctx)
    return rho, rhoE


def marnoldi_density_device(ctx: Context, rho_device, rhoE_device) -> None:
    _check(load().marnoldi_density_device(ctx.handle, _ptr(rho_device), _ptr(rhoE_device)), ctx)


def marnoldi_energy(ctx: Context) -> tuple[float, float, float]:
    E, mu, N = C.c_double(), C.c_double(), C.c_double()
    _check(load().marnoldi_energy(ctx.handle, C.byref(E), C.byref(mu), C.byref(N)), ctx)
    return E.value, mu.value, N.value


def marnoldi_level_range(ctx: Context) -> tuple[float, float]:
    lo, hi = C.c_double(), C.c_double()
    _check(load().marnoldi_level_range(ctx.handle, C.byref(lo), C.byref(hi)), ctx)
    return lo.value, hi.value


def marnoldi_fermi_at(ctx: Context, mu: float, kT: float) -> tuple[float, float]:
    N, E = C.c_double(), C.c_double()
    _check(load().marnoldi_fermi_at(ctx.handle, float(mu), float(kT), C.byref(N), C.byref(E)), ctx)
    return N.value, E.value


def marnoldi_green(ctx: Context, zs) -> np.ndarray:
    z = np.asarray(zs, dtype=np.complex128).reshape(-1)
    zri = np.ascontiguousarray(np.stack([z.real, z.imag], axis=1).reshape(-1))
    G = np.empty((z.size, ctx.nnzb, 4, 4), np.complex128)
    _check(load().marnoldi_green(ctx.handle, _ptr(zri), int(z.size), _ptr(G)), ctx)
    return G


def marnoldi_set_members(ctx: Context, atom_offsets, electron_counts) -> None:
    """Declare the context's structure a block-diagonal union of members (see the C header)."""
    off = np.ascontiguousarray(atom_offsets, dtype=np.int64)
    ne = np.ascontiguousarray(electron_counts, dtype=np.float64)
    n = off.size - 1 if off.size else 0
    if n and ne.size != n:
        raise MarnoldiError(MARNOLDI_EINVAL, "one electron count per member")
    _check(load().marnoldi_set_members(ctx.handle, int(n), _ptr(off) if n else None,
                                       _ptr(ne) if n else None), ctx)


def marnoldi_set_member_temperatures(ctx: Context, kT) -> None:
    """Each member's own kT for its Fermi level, density and energy (see the C header)."""
    t = np.ascontiguousarray(kT, dtype=np.float64)
    _check(load().marnoldi_set_member_temperatures(ctx.handle, int(t.size), _ptr(t)), ctx)


def marnoldi_member_energy(ctx: Context, member: int) -> tuple[float, float, float]:
    E, mu, N = C.c_double(), C.c_double(), C.c_double()
    _check(load().marnoldi_member_energy(ctx.handle, int(member), C.byref(E), C.byref(mu), C.byref(N)), ctx)
    return E.value, mu.value, N.value


def union_of(systems, pad_to: int = 8):
    """Block-diagonal union of TBSystem-like structures, each starting at a multiple of
    `pad_to` atoms (padding atoms carry four padding orbitals: H = 0, S = I, no coupling).

    Returns (n_block_rows, row_ptr, col_idx, H, S, orbital_mask, atom_offsets, block_offsets),
    block_offsets[q] being the first block of member q (its blocks are contiguous).
    """
    rps, cis, Hs, Ss, masks, offs, boffs = [], [], [], [], [], [0], []
    nb_total = 0
    atom = 0
    for q, t in enumerate(systems):
        boffs.append(nb_total)
        n = int(t.n_block_rows)
        nnzb = int(t.row_ptr[-1])
        rps.append(np.asarray(t.row_ptr[1:], dtype=np.int64) + nb_total)
        cis.append(np.asarray(t.col_idx, dtype=np.int64) + atom)
        Hs.append(np.asarray(t.H, dtype=np.float64).reshape(nnzb, 4, 4))
        Ss.append(np.asarray(t.S, dtype=np.float64).reshape(nnzb, 4, 4))
        masks.append(np.asarray(t.orbital_mask, dtype=np.uint8).reshape(-1)
                     if t.orbital_mask is not None else np.ones(4 * n, np.uint8))
        atom += n
        nb_total += nnzb
        pad = (-atom) % pad_to if q + 1 < len(systems) else 0
        if pad:
            rps.append(nb_total + 1 + np.arange(pad, dtype=np.int64))
            cis.append(atom + np.arange(pad, dtype=np.int64))
            Hs.append(np.zeros((pad, 4, 4)))
            Ss.append(np.broadcast_to(np.eye(4), (pad, 4, 4)).copy())
            masks.append(np.zeros(4 * pad, np.uint8))
            atom += pad
            nb_total += pad
        offs.append(atom)
    row_ptr = np.concatenate([[0]] + rps).astype(np.int64)
    return (atom, row_ptr, np.concatenate(cis).astype(np.int32), np.concatenate(Hs), np.concatenate(Ss),
            np.concatenate(masks), np.array(offs, dtype=np.int64), np.array(boffs, dtype=np.int64))


def marnoldi_eigenstate(ctx: Context, k: int, sigma: float) -> tuple[float, np.ndarray, tuple[float, float]]:
    """(eps_k, phi_k over the M orbitals, (eta(k-1), eta(k))) from the last solve (see the C header)."""
    ek = C.c_double()
    phi = np.empty(4 * ctx.n_block_rows)
    eb = np.empty(2)
    _check(load().marnoldi_eigenstate(ctx.handle, int(k), float(sigma), C.byref(ek), _ptr(phi), _ptr(eb)), ctx)
    return ek.value, phi, (float(eb[0]), float(eb[1]))


def marnoldi_forces(ctx: Context, dH_dd, dS_dd) -> np.ndarray:
    """Forces (n_block_rows, 3) from the last solve; dH_dd, dS_dd of shape (3, nnzb, 4, 4)."""
    dH = np.ascontiguousarray(dH_dd, dtype=np.float64)
    dS = np.ascontiguousarray(dS_dd, dtype=np.float64)
    if dH.size != 3 * 16 * ctx.nnzb or dS.size != 3 * 16 * ctx.nnzb:
        raise MarnoldiError(MARNOLDI_EINVAL, "dH_dd and dS_dd must hold 3 x nnzb x 16 values")
    F = np.empty((ctx.n_block_rows, 3))
    _check(load().marnoldi_forces(ctx.handle, _ptr(dH), _ptr(dS), _ptr(F)), ctx)
    return F


def marnoldi_solved_shape(ctx: Context) -> tuple[int, int]:
    n, nu = C.c_int64(), C.c_int()
    _check(load().marnoldi_solved_shape(ctx.handle, C.byref(n), C.byref(nu)), ctx)
    return n.value, nu.value


def marnoldi_column_stats(ctx: Context) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    n, nu = marnoldi_solved_shape(ctx)
    nue = np.empty(n, np.int32)
    eps = np.empty((n, nu))
    w = np.empty((n, nu))
    _check(load().marnoldi_column_stats(ctx.handle, _ptr(nue), _ptr(eps), _ptr(w)), ctx)
    return nue, eps, w


def marnoldi_set_batch(ctx: Context, batch_columns: int) -> None:
    _check(load().marnoldi_set_batch(ctx.handle, int(batch_columns)), ctx)


def marnoldi_set_krylov_graph(ctx: Context, enable: bool) -> None:
    _check(load().marnoldi_set_krylov_graph(ctx.handle, int(bool(enable))), ctx)


def marnoldi_krylov_graph_launches(ctx: Context) -> int:
    n = C.c_int64()
    _check(load().marnoldi_krylov_graph_launches(ctx.handle, C.byref(n)), ctx)
    return n.value


def marnoldi_set_profiling(ctx: Context, enable: bool) -> None:
    _check(load().marnoldi_set_profiling(ctx.handle, int(bool(enable))), ctx)


def marnoldi_kernel_kinds() -> int:
    return int(load().marnoldi_kernel_kinds())


def marnoldi_kernel_stats(ctx: Context, reset: bool = False) -> dict:
    L = load()
    out = {}
    for k in range(L.marnoldi_kernel_kinds()):
        name, n, ms = C.c_char_p(), C.c_int64(), C.c_double()
        _check(L.marnoldi_kernel_stats(ctx.handle, k, C.byref(name), C.byref(n), C.byref(ms),
                                       int(bool(reset))), ctx)
        out[name.value.decode()] = (n.value, ms.value)
    return out


def marnoldi_count_noalloc(eps_device, w_device, nu_eff_device, ncols: int, nu: int, mu: float,
                           kT: float, out_device, stream: int | None = None) -> None:
    """N(mu) and E(mu) over device-resident levels into out_device[0:2], allocating nothing.

    For callers that cannot allocate device memory; the reduction's scratch is a
    fixed array inside the library (at most 16,777,216 levels per call).  eps_device
    and w_device: float64 CUDA tensors of at least ncols*nu elements; nu_eff_device:
    int32, at least ncols, or None; out_device: float64, at least 2; all contiguous
    and on the current device (else MarnoldiError(EINVAL) before any call).
    """
    ncols, nu = int(ncols), int(nu)
    if ncols >= 1 and nu >= 1 and ncols * nu > MARNOLDI_COUNT_NOALLOC_MAX_LEVELS:
        raise MarnoldiError(MARNOLDI_EINVAL, f"count_noalloc: ncols * nu exceeds the maximum of "
                            f"{MARNOLDI_COUNT_NOALLOC_MAX_LEVELS} levels of the fixed scratch")
    need = max(ncols, 0) * max(nu, 0)
    _device_tensor("eps_device", eps_device, "float64", need)
    _device_tensor("w_device", w_device, "float64", need)
    if nu_eff_device is not None:
        _device_tensor("nu_eff_device", nu_eff_device, "int32", max(ncols, 0))
    _device_tensor("out_device", out_device, "float64", 2)
    st = _current_stream() if stream is None else int(stream)
    _check(load().marnoldi_count_noalloc(_ptr(eps_device), _ptr(w_device), _ptr(nu_eff_device),
                                         ncols, nu, float(mu), float(kT),
                                         _ptr(out_device), C.c_void_p(st)))


def _device_tensor(name: str, a, dtype: str, min_len: int) -> None:
    """Raise MarnoldiError(EINVAL) unless `a` is a contiguous torch CUDA tensor of `dtype` on the
    current device with at least min_len elements (the C entry point cannot check any of this)."""
    import torch
    if not isinstance(a, torch.Tensor) or not a.is_cuda:
        raise MarnoldiError(MARNOLDI_EINVAL, f"count_noalloc: {name} must be a torch CUDA tensor")
    if a.device.index != torch.cuda.current_device():
        raise MarnoldiError(MARNOLDI_EINVAL, f"count_noalloc: {name} is on cuda:{a.device.index}, "
                            f"not the current device cuda:{torch.cuda.current_device()}")
    if a.dtype != getattr(torch, dtype):
        raise MarnoldiError(MARNOLDI_EINVAL, f"count_noalloc: {name} must be {dtype}, not {a.dtype}")
    if not a.is_contiguous():
        raise MarnoldiError(MARNOLDI_EINVAL, f"count_noalloc: {name} must be contiguous")
    if a.numel() < min_len:
        raise MarnoldiError(MARNOLDI_EINVAL, f"count_noalloc: {name} holds {a.numel()} elements, "
                            f"fewer than the {min_len} needed")


def marnoldi_check_status() -> tuple[bool, int, int]:
    """(built with index checks, first failed check site or 0, its index); clears the records."""
    comp, site, idx = C.c_int(), C.c_int(), C.c_int64()
    _check(load().marnoldi_check_status(C.byref(comp), C.byref(site), C.byref(idx)))
    return bool(comp.value), site.value, idx.value


def marnoldi_last_error(ctx: Context | None = None) -> str:
    r = load().marnoldi_last_error(None if ctx is None else ctx.handle)
    return r.decode() if r else ""


def marnoldi_destroy(ctx: Context) -> None:
    if ctx is not None and ctx.handle is not None and ctx.handle.value:
        load().marnoldi_destroy(ctx.handle)
        ctx.handle = C.c_void_p(None)


def marnoldi_set_autotune(mode: int) -> None:
    """0 = fixed launch-shape rule, 1 = time the Gram-Schmidt shapes on first use (process-wide)."""
    _check(load().marnoldi_set_autotune(int(mode)))


def marnoldi_gs_shape(ctx: Context) -> tuple[int, int]:
    """(values per thread, threads per CTA) of the Gram-Schmidt kernel in the last solve."""
    v, t = C.c_int(), C.c_int()
    _check(load().marnoldi_gs_shape(ctx.handle, C.byref(v), C.byref(t)), ctx)
    return v.value, t.value


def marnoldi_device_bytes(ctx: Context) -> tuple[int, int]:
    """(bytes held now, most bytes held since setup) of a context's device memory."""
    cur, peak = C.c_size_t(), C.c_size_t()
    _check(load().marnoldi_device_bytes(ctx.handle, C.byref(cur), C.byref(peak)), ctx)
    return cur.value, peak.value


def marnoldi_footprint(n_block_rows: int, row_ptr, orbital_mask=None, box=None,
                       precision: int = MARNOLDI_FP64, nu: int = 30, region_atoms: int = 0,
                       batch_columns: int = 1 << 40) -> tuple[int, int]:
    """(peak device bytes, batch used) of setup + solve of every real orbital + density."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    if rp.size != n_block_rows + 1:
        raise MarnoldiError(MARNOLDI_EINVAL, "row_ptr must have n_block_rows + 1 entries")
    mask = None if orbital_mask is None else np.ascontiguousarray(orbital_mask, dtype=np.uint8)
    bx = None if box is None else np.ascontiguousarray(box, dtype=np.float64)
    nbytes, used = C.c_size_t(), C.c_int64()
    _check(load().marnoldi_footprint(int(n_block_rows), _ptr(rp), _ptr(mask), _ptr(bx), int(precision),
                                     int(nu), int(region_atoms), int(batch_columns), C.byref(nbytes),
                                     C.byref(used)))
    return nbytes.value, used.value


class ServerError(MarnoldiError):
    pass


def _server_check(rc: int):
    if rc != MARNOLDI_OK:
        msg = load().marnoldi_server_last_error()
        raise ServerError(rc, msg.decode() if msg else "")


class Server:
    """``marnoldi_server``: whole calculations queued and run concurrently on the current GPU.

    ``submit`` returns a request id at once; ``wait`` returns its result.  The
    arrays of a request are kept referenced here until it has been waited for,
    as the C API requires.
    """

    def __init__(self, workers: int = 4, hbm_budget_bytes: int = 32 << 30):
        L = load()
        out = C.c_void_p()
        _server_check(L.marnoldi_server_create(C.byref(out), int(workers), int(hbm_budget_bytes)))
        self.handle = out
        self._held: dict[int, tuple] = {}

    def submit(self, n_block_rows: int, row_ptr, col_idx, H_vals, S_vals, orbital_mask=None,
               positions=None, box=None, precision: int = MARNOLDI_FP64, nu: int = 30,
               region_atoms: int = 0, electron_count: float = 0.0, kT: float = 0.1,
               batch_columns: int = 0, density: bool = True) -> int:
        rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
        ci = np.ascontiguousarray(col_idx, dtype=np.int32)
        H = np.ascontiguousarray(H_vals, dtype=np.float64)
        S = np.ascontiguousarray(S_vals, dtype=np.float64)
        mask = None if orbital_mask is None else np.ascontiguousarray(orbital_mask, dtype=np.uint8)
        pos = None if positions is None else np.ascontiguousarray(positions, dtype=np.float64)
        bx = None if box is None else np.ascontiguousarray(box, dtype=np.float64)
        if rp.size != n_block_rows + 1:
            raise ServerError(MARNOLDI_EINVAL, "row_ptr must have n_block_rows + 1 entries")
        nnzb = int(rp[-1])
        if ci.size != nnzb or H.size != 16 * nnzb or S.size != 16 * nnzb:
            raise ServerError(MARNOLDI_EINVAL, "col_idx / H_vals / S_vals sizes do not match row_ptr")
        if mask is not None and mask.size != 4 * n_block_rows:
            raise ServerError(MARNOLDI_EINVAL, "orbital_mask must have 4 n_block_rows entries")
        rho = np.empty((nnzb, 4, 4)) if density else None
        rhoE = np.empty((nnzb, 4, 4)) if density else None
        rid = C.c_int64()
        _server_check(load().marnoldi_server_submit(
            self.handle, int(n_block_rows), _ptr(rp), _ptr(ci), _ptr(H), _ptr(S), _ptr(mask), _ptr(pos),
            _ptr(bx), int(precision), int(nu), int(region_atoms), float(electron_count), float(kT),
            int(batch_columns), _ptr(rho), _ptr(rhoE), C.byref(rid)))
        self._held[rid.value] = (rp, ci, H, S, mask, pos, bx, rho, rhoE)
        return rid.value

    def submit_system(self, sysm, precision: int = MARNOLDI_FP64, nu: int = 30, region_atoms: int = 0,
                      electron_count: float | None = None, kT: float = 0.1, batch_columns: int = 0,
                      density: bool = True) -> int:
        """submit for a tbsynth.TBSystem-like object (N_e defaults to its n_electrons)."""
        s = getattr(sysm, "structure", None)
        if electron_count is None:
            electron_count = sysm.n_electrons
        return self.submit(sysm.n_block_rows, sysm.row_ptr, sysm.col_idx, sysm.H, sysm.S,
                           sysm.orbital_mask, None if s is None else s.positions,
                           None if s is None else s.box, precision, nu, region_atoms,
                           electron_count, kT, batch_columns, density)

    def wait(self, request_id: int, timeout_s: float = -1.0) -> dict | None:
        """The request's result, or None while it is still pending after timeout_s.

        Raises MarnoldiError with the request's own status if it failed.
        """
        st = C.c_int()
        res = np.zeros(8)
        msg = C.create_string_buffer(512)
        rc = load().marnoldi_server_wait(self.handle, int(request_id), float(timeout_s), C.byref(st),
                                         _ptr(res), msg, 512)
        if rc == MARNOLDI_EPENDING:
            return None
        _server_check(rc)
        held = self._held.pop(int(request_id))
        if st.value != MARNOLDI_OK:
            raise MarnoldiError(st.value, msg.value.decode())
        return {"band_energy": res[0], "mu": res[1], "N": res[2], "t_submit": res[3],
                "t_start": res[4], "t_end": res[5], "latency_s": res[5] - res[3],
                "footprint_bytes": int(res[6]), "batch": int(res[7]), "rho": held[7], "rhoE": held[8]}

    def set_group_limit(self, max_members: int) -> None:
        """Most requests run as members of one launch group (1 = no grouping)."""
        _server_check(load().marnoldi_server_set_group_limit(self.handle, int(max_members)))

    def stats(self) -> dict:
        v = np.zeros(9, np.int64)
        _server_check(load().marnoldi_server_stats(self.handle, _ptr(v)))
        keys = ("queued", "running", "completed", "bytes_in_use", "peak_bytes", "peak_running",
                "pool_reserved_high", "groups", "largest_group")
        return {k: int(x) for k, x in zip(keys, v)}

    def close(self) -> None:
        if self.handle is not None and self.handle.value:
            load().marnoldi_server_destroy(self.handle)
            self.handle = C.c_void_p(None)
            self._held.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
