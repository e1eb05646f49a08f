"""ctypes binding of the BlockBP C ABI (include/bbp.h): argument marshalling only.

Each ``bbp_*`` function here has the name and meaning of the C entry point;
NumPy arrays are passed as host pointers, torch tensors (or integers) as
device pointers.  Every non-OK status raises ``BBPError`` carrying the
library's message.  Loading fails loudly when the library is missing: there
is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB

STATUS = {
    0: "BBP_OK", 1: "BBP_ERR_ARG", 2: "BBP_ERR_OOM", 3: "BBP_ERR_CUDA", 4: "BBP_ERR_TILING",
    5: "BBP_ERR_NUMERIC", 6: "BBP_NOT_CONVERGED", 7: "BBP_ERR_TIMEOUT", 8: "BBP_ERR_STATE",
}
SQUARE, KAGOME = 0, 1
FP64, TF32, BF16, FP32 = 0, 1, 2, 3
BOTTOM, RIGHT, TOP, LEFT = 0, 1, 2, 3

EXPORTS = [
    "bbp_set_allocator", "bbp_create_peps", "bbp_partition_blocks", "bbp_set_options", "bbp_init_messages",
    "bbp_iterate", "bbp_expect_local", "bbp_block_rdm", "bbp_energy_per_site", "bbp_norm", "bbp_get_message", "bbp_core_pmps", "bbp_core_plan_debug", "bbp_core_expect", "bbp_ite_bond", "bbp_ite",
    "bbp_footprint_bytes", "bbp_info", "bbp_stats", "bbp_last_error", "bbp_destroy", "bbp_k_fuse",
    "bbp_k_svd_work_bytes", "bbp_k_svd_trunc", "bbp_k_svd_trunc_noalloc", "bbp_k_svd_stats", "bbp_k_qr", "bbp_k_panel_cluster", "bbp_k_panel_qr", "bbp_k_svd_work_bytes_rand", "bbp_k_svd_trunc_rand", "bbp_k_fma_peak", "bbp_set_hermitise", "bbp_expect_product", "bbp_bond_energies", "bbp_k_tc_gemm", "bbp_set_execution", "bbp_set_power_iters",
    "bbp_batch_iterate", "bbp_server_create", "bbp_job_footprint_bytes", "bbp_server_submit", "bbp_server_step",
    "bbp_server_poll", "bbp_server_take", "bbp_server_destroy", "bbp_ktimer_select", "bbp_ktimer_read",
    "bbp_k_tc_absorb_bytes", "bbp_k_tc_absorb", "bbp_plan_debug", "bbp_k_tc_gemm_tile", "bbp_autotune_record",
    "bbp_autotune_run", "bbp_autotune_load", "bbp_autotune_info", "bbp_autotune_clear", "bbp_batch_single_launch",
    "bbp_set_fuse_cache", "bbp_share_workers",
]


class BBPError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None
_keep = []   # ctypes callbacks kept alive

_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_ALLOC = ctypes.CFUNCTYPE(_vp, ctypes.c_size_t, _vp, _vp)
_FREE = ctypes.CFUNCTYPE(None, _vp, _vp, _vp)

_PROTOS = {
    "bbp_set_allocator": (None, [_ALLOC, _FREE, _vp]),
    "bbp_create_peps": (_i, [ctypes.POINTER(_vp), _i, _i, _i, _i, _i, _i, _vp, _i, _vp]),
    "bbp_partition_blocks": (_i, [_vp, _i, _i]),
    "bbp_set_options": (_i, [_vp, _i, _i, _d, ctypes.c_uint64]),
    "bbp_init_messages": (_i, [_vp, _dp]),
    "bbp_iterate": (_i, [_vp, _d, _i, _ip, _dp]),
    "bbp_expect_local": (_i, [_vp, _dp, _i, _ip, _dp, _dp]),
    "bbp_block_rdm": (_i, [_vp, _i, _ip, _i, _dp]),
    "bbp_energy_per_site": (_i, [_vp, _dp]),
    "bbp_norm": (_i, [_vp, _dp]),
    "bbp_get_message": (_i, [_vp, _i, _i, _ip, _ip, _dp, ctypes.c_size_t]),
    "bbp_core_pmps": (_i, [_vp, _i, _ip, _i, _i, _ip, _ip, _ip, _dp, ctypes.c_size_t, _dp]),
    "bbp_core_plan_debug": (_i, [_i, _i, _i, _i, _i, _i, _i, _ip, _i, _ip, _i, _ip, _ip, _i]),
    "bbp_core_expect": (_i, [_vp, _i, _ip, _i, _dp, _i, _dp, _dp]),
    "bbp_ite_bond": (_i, [_vp, _i, _i, _dp, _i, _d, _dp, _i, _ip]),
    "bbp_ite": (_i, [_vp, _dp, _i, _ip, _i, _d, _i, _i, _dp]),
    "bbp_footprint_bytes": (ctypes.c_size_t, [_i, _i, _i, _i, _i, _i, _i]),
    "bbp_info": (_i, [_vp, _ip, _ip, _ip]),
    "bbp_stats": (_i, [_vp, ctypes.POINTER(ctypes.c_longlong), _dp]),
    "bbp_last_error": (ctypes.c_char_p, [_vp]),
    "bbp_destroy": (None, [_vp]),
    "bbp_k_fuse": (_i, [_vp, _i, _i, _ip, _vp, _ip, _vp, _vp]),
    "bbp_k_svd_work_bytes": (ctypes.c_size_t, [_i, _i]),
    "bbp_k_svd_trunc": (_i, [_vp, _i, _i, _i, _vp, _vp, _vp, _vp, _vp]),
    "bbp_k_svd_trunc_noalloc": (_i, [_vp, _i, _i, _i, _vp, _vp, _vp, _vp]),
    "bbp_k_svd_stats": (_i, [_vp, _i, _i, _ip, ctypes.POINTER(ctypes.c_longlong), _vp]),
    "bbp_k_qr": (_i, [_vp, _i, _i, _vp, _vp, _vp, _vp]),
    "bbp_k_panel_cluster": (_i, [_i, _i, _i]),
    "bbp_k_panel_qr": (_i, [_i, _vp, _i, _i, _vp, _vp, _i, _i, _vp]),
    "bbp_k_svd_work_bytes_rand": (ctypes.c_size_t, [_i, _i, _i, _i, _i]),
    "bbp_k_fma_peak": (_i, [_i, _i, _i, _vp, _dp, _vp]),
    "bbp_set_hermitise": (_i, [_vp, _i]),
    "bbp_expect_product": (_i, [_vp, _dp, _dp, _i, _i, _dp, _dp]),
    "bbp_bond_energies": (_i, [_vp, _ip, _i, _dp]),
    "bbp_k_svd_trunc_rand": (_i, [_i, _vp, _i, _i, _i, _vp, _vp, _vp, _vp, _i, _i, _vp, _vp]),
    "bbp_set_execution": (_i, [_vp, _i, _i]),
    "bbp_set_power_iters": (_i, [_vp, _i]),
    "bbp_batch_iterate": (_i, [ctypes.POINTER(_vp), _i, ctypes.c_double, _i, _ip, ctypes.POINTER(ctypes.c_double), _ip]),
    "bbp_server_create": (_i, [ctypes.POINTER(_vp), ctypes.c_size_t, _i]),
    "bbp_job_footprint_bytes": (ctypes.c_size_t, [_vp]),
    "bbp_server_submit": (_i, [_vp, _vp, ctypes.POINTER(ctypes.c_longlong)]),
    "bbp_server_step": (_i, [_vp, ctypes.c_double, _ip, _ip, _ip]),
    "bbp_server_poll": (_i, [_vp, ctypes.POINTER(ctypes.c_longlong), _ip, _ip, ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), _i, _ip]),
    "bbp_server_take": (_i, [_vp, ctypes.c_longlong, ctypes.POINTER(_vp)]),
    "bbp_server_destroy": (None, [_vp]),
    "bbp_ktimer_select": (None, [_i]),
    "bbp_ktimer_read": (_i, [ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_double)]),
    "bbp_k_tc_gemm_tile": (_i, [_i, _vp, ctypes.c_longlong, _vp, ctypes.c_longlong, _vp, ctypes.c_longlong, _i, _i,
                                _i, ctypes.c_float, _i, _i, _vp, _vp]),
    "bbp_autotune_record": (_i, [_i]),
    "bbp_batch_single_launch": (_i, [_i]),
    "bbp_set_fuse_cache": (_i, [_vp, ctypes.c_size_t]),
    "bbp_share_workers": (_i, [_vp, _i, _i]),
    "bbp_autotune_run": (_i, [ctypes.c_char_p, _ip]),
    "bbp_autotune_load": (_i, [ctypes.c_char_p, _ip]),
    "bbp_autotune_info": (_i, [_ip, _ip, ctypes.POINTER(ctypes.c_ulonglong)]),
    "bbp_autotune_clear": (_i, []),
    "bbp_k_tc_gemm": (_i, [_i, _vp, ctypes.c_longlong, _vp, ctypes.c_longlong, _vp, ctypes.c_longlong, _i, _i, _i,
                           ctypes.c_float, _vp, _vp]),
    "bbp_k_tc_absorb_bytes": (ctypes.c_size_t, [_i, _i, _i, _i, _i]),
    "bbp_k_tc_absorb": (_i, [_i, _i, _vp, _i, _i, _vp, _i, _i, _vp, _vp, _vp, _vp]),
    "bbp_plan_debug": (_i, [_i, _i, _i, _i, _i, _i, _i, _i, _ip, _i, _ip]),
}


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"BlockBP CUDA library not built ({LIB}); call paper_2603_13304_gb300.build.build()")
        L = ctypes.CDLL(LIB)
        for name, (res, args) in _PROTOS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int, ctx=None):
    if status != 0:
        msg = lib().bbp_last_error(ctx).decode()
        raise BBPError(status, msg)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(_ip)


def _devptr(x) -> int:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def use_torch_allocator():
    """Route the library's device allocations through PyTorch's caching allocator."""
    import torch

    def _alloc(size, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(size), torch.cuda.current_device(), stream or 0)
        except Exception:
            return None

    def _free(ptr, stream, user):
        torch.cuda.caching_allocator_delete(ptr)

    a, f = _ALLOC(_alloc), _FREE(_free)
    _keep.extend([a, f])
    lib().bbp_set_allocator(a, f, None)


def use_default_allocator():
    lib().bbp_set_allocator(_ALLOC(0), _FREE(0), None)


def _c128(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a.view(np.float64)


# ------------------------------------------------------------ context calls

def bbp_create_peps(lattice: int, Lx: int, Ly: int, periodic: int, d: int, D: int, tensors, stream=None):
    """tensors: complex128, or complex64 (passed as such, dtype 1)."""
    if np.asarray(tensors).dtype == np.complex64:
        t = np.ascontiguousarray(tensors, dtype=np.complex64).view(np.float32)
        ptr, dtype = t.ctypes.data_as(ctypes.c_void_p), 1
    else:
        t = _c128(tensors)
        ptr, dtype = t.ctypes.data_as(ctypes.c_void_p), 0
    ctx = _vp()
    _check(lib().bbp_create_peps(ctypes.byref(ctx), lattice, Lx, Ly, int(periodic), d, D, ptr, dtype, _stream(stream)))
    return ctx


def bbp_partition_blocks(ctx, bx: int, by: int):
    _check(lib().bbp_partition_blocks(ctx, bx, by), ctx)


def bbp_set_options(ctx, chi: int, precision: int = FP64, alpha: float = 1.0, seed: int = 0):
    _check(lib().bbp_set_options(ctx, chi, precision, alpha, seed), ctx)


def bbp_init_messages(ctx, edge_mats):
    e = _c128(edge_mats)
    _check(lib().bbp_init_messages(ctx, _dptr(e)), ctx)


def bbp_iterate(ctx, tol: float, max_iter: int, allow_not_converged: bool = True):
    it = ctypes.c_int(0)
    err = ctypes.c_double(0.0)
    st = lib().bbp_iterate(ctx, tol, max_iter, ctypes.byref(it), ctypes.byref(err))
    if st == 6 and allow_not_converged:
        return it.value, err.value, False
    _check(st, ctx)
    return it.value, err.value, True


def bbp_expect_local(ctx, op, sites):
    o = _c128(op)
    s = np.ascontiguousarray(sites, dtype=np.int32)
    ns = len(s)   # [site] or [site, slot of the bond]
    re, im = ctypes.c_double(), ctypes.c_double()
    _check(lib().bbp_expect_local(ctx, _dptr(o), ns, _iptr(s), ctypes.byref(re), ctypes.byref(im)), ctx)
    return complex(re.value, im.value)


def bbp_expect_product(ctx, op1, op2, site: int, slot: int):
    a, b = _c128(op1), _c128(op2)
    re, im = ctypes.c_double(), ctypes.c_double()
    _check(lib().bbp_expect_product(ctx, _dptr(a), _dptr(b), site, slot, ctypes.byref(re), ctypes.byref(im)), ctx)
    return complex(re.value, im.value)


def bbp_bond_energies(ctx, bonds) -> np.ndarray:
    """<S_i . S_j> of every bond (site, slot) in `bonds`."""
    b = np.ascontiguousarray([(int(x[0]), int(x[1])) for x in bonds], dtype=np.int32).reshape(-1)
    out = np.zeros(len(bonds), dtype=np.float64)
    _check(lib().bbp_bond_energies(ctx, _iptr(b), len(bonds), _dptr(out)), ctx)
    return out


def bbp_block_rdm(ctx, block: int, sites, d: int = 2):
    s = np.ascontiguousarray(sites, dtype=np.int32)
    dim = d ** len(s)
    out = np.zeros((dim, dim), dtype=np.complex128)
    _check(lib().bbp_block_rdm(ctx, block, _iptr(s), len(s), _dptr(out.view(np.float64))), ctx)
    return out


def bbp_energy_per_site(ctx) -> float:
    e = ctypes.c_double()
    _check(lib().bbp_energy_per_site(ctx, ctypes.byref(e)), ctx)
    return e.value


def bbp_norm(ctx) -> float:
    v = ctypes.c_double()
    _check(lib().bbp_norm(ctx, ctypes.byref(v)), ctx)
    return v.value


def bbp_get_message(ctx, block: int, face: int, cap: int = 1 << 22):
    k = ctypes.c_int()
    shapes = np.zeros(3 * 64, dtype=np.int32)
    data = np.zeros(cap, dtype=np.float64)
    _check(lib().bbp_get_message(ctx, block, face, ctypes.byref(k), _iptr(shapes), _dptr(data), cap), ctx)
    out, off = [], 0
    for q in range(k.value):
        l, p, r = shapes[3 * q:3 * q + 3]
        n = int(l * p * r)
        out.append(data[off:off + 2 * n].view(np.complex128).reshape(l, p, r).copy())
        off += 2 * n
    return out


def bbp_core_pmps(ctx, block: int, core_sites, cap: int = 1 << 24, cap_len: int = 64):
    """The pMPS around core sites (global ids) of a block: (tensors (l, p, r)
    in cyclic order, [(position in core_sites, slot)] per tensor, logscale)."""
    s = np.ascontiguousarray(core_sites, dtype=np.int32)
    n = ctypes.c_int()
    shapes = np.zeros(3 * cap_len, dtype=np.int32)
    legs = np.zeros(2 * cap_len, dtype=np.int32)
    data = np.zeros(cap, dtype=np.float64)
    ls = ctypes.c_double()
    _check(lib().bbp_core_pmps(ctx, block, _iptr(s), len(s), cap_len, ctypes.byref(n), _iptr(shapes), _iptr(legs),
                               _dptr(data), cap, ctypes.byref(ls)), ctx)
    out, off = [], 0
    for q in range(n.value):
        l, p, r = shapes[3 * q:3 * q + 3]
        k = int(l * p * r)
        out.append(data[off:off + 2 * k].view(np.complex128).reshape(l, p, r).copy())
        off += 2 * k
    return out, [(int(legs[2 * q]), int(legs[2 * q + 1])) for q in range(n.value)], ls.value


def bbp_core_expect(ctx, block: int, core_sites, ops):
    """<O_k> for operator sets ops[k] = [O_site0, (O_site1)] (d x d each) on a
    core of one site or of a bond's two ends; returns a complex array."""
    s = np.ascontiguousarray(core_sites, dtype=np.int32)
    nops = len(ops)
    o = _c128(np.asarray(ops, dtype=np.complex128).reshape(nops, len(s), -1) if nops
              else np.zeros(1, dtype=np.complex128))
    re = np.zeros(max(nops, 1))
    im = np.zeros(max(nops, 1))
    _check(lib().bbp_core_expect(ctx, block, _iptr(s), len(s), _dptr(o), nops, _dptr(re), _dptr(im)), ctx)
    return (re + 1j * im)[:nops]


def bbp_ite_bond(ctx, site: int, slot: int, gate, max_sweeps: int = 50, tol: float = 1e-13):
    """One ITE bond update; returns the Phi history (start, every half-step)."""
    g = _c128(gate)
    phi = np.zeros(2 * max_sweeps + 1)
    n = ctypes.c_int()
    _check(lib().bbp_ite_bond(ctx, site, slot, _dptr(g), max_sweeps, tol, _dptr(phi), phi.size, ctypes.byref(n)), ctx)
    return phi[:n.value].copy()


def bbp_ite(ctx, gates, bonds, bp_tol: float = 1e-10, bp_max_iter: int = 40, als_sweeps: int = 50):
    """Full ITE over the gate list; bonds: (site, slot) pairs; returns the
    energy per site after each gate."""
    g = _c128(np.asarray(gates, dtype=np.complex128))
    b = np.ascontiguousarray(np.asarray(bonds, dtype=np.int32).reshape(-1))
    out = np.zeros(len(gates))
    _check(lib().bbp_ite(ctx, _dptr(g), len(gates), _iptr(b), len(b) // 2, bp_tol, bp_max_iter, als_sweeps,
                         _dptr(out)), ctx)
    return out


def bbp_footprint_bytes(lattice, n_sites, D, chi, bx, by, precision=FP64) -> int:
    return int(lib().bbp_footprint_bytes(lattice, n_sites, D, chi, bx, by, precision))


def bbp_info(ctx):
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().bbp_info(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), ctx)
    return a.value, b.value, c.value


def bbp_stats(ctx):
    n = ctypes.c_longlong()
    f = ctypes.c_double()
    _check(lib().bbp_stats(ctx, ctypes.byref(n), ctypes.byref(f)), ctx)
    return n.value, f.value


def bbp_last_error(ctx=None) -> str:
    return lib().bbp_last_error(ctx).decode()


def bbp_destroy(ctx):
    lib().bbp_destroy(ctx)


# ------------------------------------------------------------ kernel calls

def bbp_k_fuse(t, d: int, D: int, n, op, perm, T, stream=None):
    nn = np.ascontiguousarray(n, dtype=np.int32)
    pp = np.ascontiguousarray(perm, dtype=np.int32)
    _check(lib().bbp_k_fuse(_devptr(t), d, D, _iptr(nn), _devptr(op), _iptr(pp), _devptr(T), _stream(stream)))


def bbp_k_svd_work_bytes(m: int, n: int) -> int:
    return int(lib().bbp_k_svd_work_bytes(m, n))


def bbp_k_svd_trunc(Z, m: int, n: int, chi: int, U, Rem, work, status, stream=None):
    _check(lib().bbp_k_svd_trunc(_devptr(Z), m, n, chi, _devptr(U), _devptr(Rem), _devptr(work), _devptr(status),
                                 _stream(stream)))


def bbp_k_svd_trunc_noalloc(Z, m: int, n: int, chi: int, U, Rem, status, stream=None):
    _check(lib().bbp_k_svd_trunc_noalloc(_devptr(Z), m, n, chi, _devptr(U), _devptr(Rem), _devptr(status),
                                         _stream(stream)))


def bbp_k_svd_stats(work, m: int, n: int, stream=None):
    sw = ctypes.c_int()
    rot = ctypes.c_longlong()
    _check(lib().bbp_k_svd_stats(_devptr(work), m, n, ctypes.byref(sw), ctypes.byref(rot), _stream(stream)))
    return sw.value, rot.value


def bbp_k_qr(A, m: int, n: int, Q, R, tau, stream=None):
    _check(lib().bbp_k_qr(_devptr(A), m, n, _devptr(Q), _devptr(R), _devptr(tau), _stream(stream)))


def bbp_k_panel_cluster(c64: bool, m: int, n: int) -> int:
    return int(lib().bbp_k_panel_cluster(int(c64), m, n))


def bbp_k_panel_qr(c64: bool, A, m: int, n: int, Q, R, batch: int = 1, cluster: int = 0, stream=None):
    _check(lib().bbp_k_panel_qr(int(c64), _devptr(A), m, n, _devptr(Q), _devptr(R), batch, cluster,
                                _stream(stream)))


def bbp_k_svd_work_bytes_rand(c64: bool, m: int, n: int, chi: int, tensor_cores: bool = False) -> int:
    return int(lib().bbp_k_svd_work_bytes_rand(int(c64), m, n, chi, int(tensor_cores)))


def bbp_k_svd_trunc_rand(c64: bool, Z, m: int, n: int, chi: int, U, Rem, work, status, power_iters: int,
                         tensor_cores: bool = False, err=None, stream=None):
    _check(lib().bbp_k_svd_trunc_rand(int(c64), _devptr(Z), m, n, chi, _devptr(U), _devptr(Rem), _devptr(work),
                                      _devptr(status), power_iters, int(tensor_cores), _devptr(err), _stream(stream)))


def bbp_k_fma_peak(fp64: bool, blocks: int, iters: int, out, stream=None) -> float:
    fl = ctypes.c_double()
    _check(lib().bbp_k_fma_peak(int(fp64), blocks, iters, _devptr(out), ctypes.byref(fl), _stream(stream)))
    return fl.value


def bbp_set_hermitise(ctx, on: bool = True):
    _check(lib().bbp_set_hermitise(ctx, int(on)), ctx)


def bbp_set_execution(ctx, use_graphs: bool = True, max_streams: int = 16):
    _check(lib().bbp_set_execution(ctx, int(use_graphs), int(max_streams)), ctx)


def bbp_set_power_iters(ctx, power_iters: int):
    _check(lib().bbp_set_power_iters(ctx, int(power_iters)), ctx)


KT_JACOBI, KT_ORTH, KT_QR, KT_TC, KT_ABSORB, KT_GEMM = 1, 2, 3, 4, 5, 6


def bbp_ktimer_select(kernel_class: int):
    lib().bbp_ktimer_select(int(kernel_class))


def bbp_ktimer_read():
    n = ctypes.c_longlong()
    ms = ctypes.c_double()
    fl = ctypes.c_double()
    _check(lib().bbp_ktimer_read(ctypes.byref(n), ctypes.byref(ms), ctypes.byref(fl)))
    return n.value, ms.value, fl.value


def bbp_k_tc_gemm(bf16: bool, A, lda: int, Bt, ldb: int, C, ldc: int, M: int, N: int, K: int, alpha: float, err,
                  stream=None):
    _check(lib().bbp_k_tc_gemm(int(bf16), _devptr(A), lda, _devptr(Bt), ldb, _devptr(C), ldc, M, N, K, alpha,
                               _devptr(err), _stream(stream)))


def bbp_k_tc_gemm_tile(bf16: bool, A, lda: int, Bt, ldb: int, C, ldc: int, M: int, N: int, K: int, alpha: float,
                       bn: int, group_m: int, err, stream=None):
    _check(lib().bbp_k_tc_gemm_tile(int(bf16), _devptr(A), lda, _devptr(Bt), ldb, _devptr(C), ldc, M, N, K, alpha,
                                    bn, group_m, _devptr(err), _stream(stream)))


def bbp_set_fuse_cache(ctx, max_bytes: int):
    _check(lib().bbp_set_fuse_cache(ctx, int(max_bytes)), ctx)


def bbp_share_workers(ctxs, groups: int):
    n = len(ctxs)
    arr = (_vp * n)(*[c.value if isinstance(c, ctypes.c_void_p) else c for c in ctxs])
    _check(lib().bbp_share_workers(arr, n, int(groups)))


def bbp_batch_single_launch(on: bool):
    _check(lib().bbp_batch_single_launch(int(on)))


def bbp_autotune_record(on: bool):
    _check(lib().bbp_autotune_record(int(on)))


def bbp_autotune_run(cache_path: str = None) -> int:
    """Tunes the recorded tensor-core GEMM shapes; returns how many."""
    n = ctypes.c_int(0)
    _check(lib().bbp_autotune_run(cache_path.encode() if cache_path else None, ctypes.byref(n)))
    return n.value


def bbp_autotune_load(cache_path: str) -> int:
    n = ctypes.c_int(0)
    _check(lib().bbp_autotune_load(cache_path.encode(), ctypes.byref(n)))
    return n.value


def bbp_autotune_info():
    """(table entries, recorded shapes not yet tuned, generation)"""
    e, p, g = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_ulonglong(0)
    _check(lib().bbp_autotune_info(ctypes.byref(e), ctypes.byref(p), ctypes.byref(g)))
    return e.value, p.value, g.value


def bbp_autotune_clear():
    _check(lib().bbp_autotune_clear())


def bbp_k_tc_absorb_bytes(bf16: bool, P: int, Q: int, l: int, r: int) -> int:
    return int(lib().bbp_k_tc_absorb_bytes(int(bf16), P, Q, l, r))


def bbp_k_tc_absorb(bf16: bool, c64: bool, X, P: int, Q: int, S, l: int, r: int, R, work, err, stream=None):
    _check(lib().bbp_k_tc_absorb(int(bf16), int(c64), _devptr(X), P, Q, _devptr(S), l, r, _devptr(R), _devptr(work),
                                 _devptr(err), _stream(stream)))


def bbp_plan_debug(lattice, Lx, Ly, periodic, bx, by, block, face):
    out = np.zeros(4 * 4096, dtype=np.int32)
    n = ctypes.c_int()
    _check(lib().bbp_plan_debug(lattice, Lx, Ly, int(periodic), bx, by, block, face, _iptr(out), out.size,
                                ctypes.byref(n)))
    return out[:4 * n.value].reshape(-1, 4)

def bbp_core_plan_debug(lattice, Lx, Ly, periodic, bx, by, block, core_sites):
    """(bottom steps, top steps, (n, m, a, c, L), legs) of a core extraction's host plan."""
    s = np.ascontiguousarray(core_sites, dtype=np.int32)
    out = np.zeros(4 * 8192, dtype=np.int32)
    info = np.zeros(7, dtype=np.int32)
    legs = np.zeros(2 * 256, dtype=np.int32)
    _check(lib().bbp_core_plan_debug(lattice, Lx, Ly, int(periodic), bx, by, block, _iptr(s), len(s), _iptr(out),
                                     out.size, _iptr(info), _iptr(legs), 256))
    nb, nt = int(info[0]), int(info[1])
    steps = out[:4 * (nb + nt)].reshape(-1, 4)
    L = int(info[6])
    return (steps[:nb], steps[nb:], tuple(int(x) for x in info[2:7]),
            [(int(legs[2 * q]), int(legs[2 * q + 1])) for q in range(L)])

# ------------------------------------------------------- many problems

def bbp_batch_iterate(ctxs, tol: float, max_iter: int):
    """Iterate several contexts together; returns (status, iters, errs, statuses)."""
    n = len(ctxs)
    arr = (_vp * n)(*[c.value if isinstance(c, ctypes.c_void_p) else c for c in ctxs])
    iters = np.zeros(n, dtype=np.int32)
    errs = np.zeros(n, dtype=np.float64)
    st = np.zeros(n, dtype=np.int32)
    rc = lib().bbp_batch_iterate(arr, n, tol, max_iter, _iptr(iters),
                                 errs.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _iptr(st))
    return int(rc), iters, errs, st


class bbp_job(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int) for k in ("lattice", "Lx", "Ly", "periodic", "d", "D", "bx", "by", "chi",
                                            "precision")] + \
               [("tol", ctypes.c_double)] + [(k, ctypes.c_int) for k in ("max_iter", "streams", "power_iters")] + \
               [("host_tensors", _vp), ("edge_mats", _vp), ("tensor_dtype", ctypes.c_int)]


def make_job(lattice, Lx, Ly, periodic, d, D, bx, by, chi, precision, tensors, edge_mats, tol, max_iter,
             streams=4, power_iters=1):
    """A job description; keeps references to the host arrays until submitted."""
    c64 = np.asarray(tensors).dtype == np.complex64
    t = np.ascontiguousarray(tensors, dtype=np.complex64 if c64 else np.complex128)
    e = np.ascontiguousarray(edge_mats, dtype=np.complex128)
    j = bbp_job(lattice, Lx, Ly, int(periodic), d, D, bx, by, chi, precision, tol, max_iter, streams, power_iters,
                t.ctypes.data, e.ctypes.data, 1 if c64 else 0)
    j._keep = (t, e)
    return j


def bbp_job_footprint_bytes(job) -> int:
    return int(lib().bbp_job_footprint_bytes(ctypes.byref(job)))


def bbp_server_create(hbm_budget_bytes: int, max_active: int):
    s = _vp()
    _check(lib().bbp_server_create(ctypes.byref(s), int(hbm_budget_bytes), int(max_active)))
    return s


def bbp_server_submit(server, job) -> int:
    jid = ctypes.c_longlong()
    _check(lib().bbp_server_submit(server, ctypes.byref(job), ctypes.byref(jid)))
    return jid.value


def bbp_server_step(server, timeout_ms: float = 50.0):
    q, a, f = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().bbp_server_step(server, float(timeout_ms), ctypes.byref(q), ctypes.byref(a), ctypes.byref(f)))
    return q.value, a.value, f.value


def bbp_server_poll(server, cap: int = 4096):
    ids = np.zeros(cap, dtype=np.int64)
    st = np.zeros(cap, dtype=np.int32)
    it = np.zeros(cap, dtype=np.int32)
    err, wait, lat = (np.zeros(cap, dtype=np.float64) for _ in range(3))
    n = ctypes.c_int()
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa: E731
    _check(lib().bbp_server_poll(server, ids.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), _iptr(st), _iptr(it),
                                 dp(err), dp(wait), dp(lat), cap, ctypes.byref(n)))
    k = n.value
    return [dict(id=int(ids[i]), status=int(st[i]), iters=int(it[i]), err=float(err[i]), wait_s=float(wait[i]),
                 latency_s=float(lat[i])) for i in range(k)]


def bbp_server_take(server, job_id: int, keep_context: bool = False):
    c = _vp()
    _check(lib().bbp_server_take(server, int(job_id), ctypes.byref(c) if keep_context else None))
    return c if keep_context else None


def bbp_server_destroy(server):
    lib().bbp_server_destroy(server)
