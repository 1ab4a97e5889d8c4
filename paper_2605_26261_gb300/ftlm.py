"""Python binding of libftlm (include/ftlm.h): argument marshalling only.

Every ftlm_* function here calls the C entry point of the same name; the compute
runs in the CUDA kernels of libftlm.so.  torch supplies device memory and the
current CUDA stream.  There is no fallback: if the library is missing, every call
raises.

Convenience layer (also marshalling only): ``Basis`` owns a sector handle,
``lanczos``/``thermo`` allocate outputs and workspace with torch, and
``run_ftlm`` queues a whole FTLM job (all S^z >= 0 sectors, R chains each, then the
thermodynamic sums) through the same entry points.
"""
import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# FTLM_LIBRARY selects another build of the library (e.g. one compiled with other
# -D options); by default the in-tree libftlm.so next to this file.
LIB_PATH = os.environ.get("FTLM_LIBRARY") or os.path.join(_HERE, "libftlm.so")

FTLM_OK, FTLM_EINVAL, FTLM_ENOMEM, FTLM_EUNSUPPORTED, FTLM_ECUDA, FTLM_ETIMEOUT, FTLM_ENOCONV = range(7)
RANK_AUTO, RANK_CLT, RANK_CR = 0, 1, 2
HV_AUTO, HV_ONE_WALK, HV_SPLIT = 0, 1, 2
F64, F32 = 0, 1
GAUSS, RADEMACHER = 0, 1
MAX_SITES, MAX_BONDS, MAX_LANCZOS, MAX_SECTORS = 36, 256, 1024, 64

_lib = None


class BatchItem(ctypes.Structure):
    """ftlm_batch_item of include/ftlm.h."""
    _fields_ = [("basis", ctypes.c_void_p), ("R", ctypes.c_int), ("first_chain", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("theta_dev", ctypes.c_void_p), ("weight_dev", ctypes.c_void_p),
                ("m_eff_dev", ctypes.c_void_p)]


class BatchPlan(ctypes.Structure):
    """ftlm_batch_plan of include/ftlm.h."""
    _fields_ = [("block", ctypes.c_int), ("streams", ctypes.c_int), ("tile_rows", ctypes.c_int),
                ("stream_rows", ctypes.c_int)]

    def as_tuple(self):
        return (self.block, self.streams, self.tile_rows, self.stream_rows)


class FtlmError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{_status_name(status)}: {message}")
        self.status = status


def _status_name(s):
    return {0: "FTLM_OK", 1: "FTLM_EINVAL", 2: "FTLM_ENOMEM", 3: "FTLM_EUNSUPPORTED",
            4: "FTLM_ECUDA", 5: "FTLM_ETIMEOUT", 6: "FTLM_ENOCONV"}.get(s, f"status {s}")


def lib():
    """The loaded libftlm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing; build it with __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    P, I, U64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_double
    PU64 = ctypes.POINTER(ctypes.c_uint64)
    PD = ctypes.POINTER(ctypes.c_double)
    sig = {
        "ftlm_basis_create": [I, I, I, P, P, P, I, P, ctypes.POINTER(P)],
        "ftlm_basis_create_spin": [I, I, I, I, P, P, P, P, ctypes.POINTER(P)],
        "ftlm_basis_create_sectors": [I, I, I, P, I, P, P, P, I, I, P, P],
        "ftlm_basis_dim": [P, PU64],
        "ftlm_basis_bytes": [P, PU64],
        "ftlm_basis_mode": [P, ctypes.POINTER(I)],
        "ftlm_basis_set_schedule": [P, I, I],
        "ftlm_basis_hv_schedule": [P, I, I, ctypes.POINTER(I)],
        "ftlm_basis_updates": [P, PU64],
        "ftlm_basis_labels": [P, U64, U64, P, P],
        "ftlm_basis_rank": [P, U64, P, P, P],
        "ftlm_basis_clt": [P, P, P, P],
        "ftlm_hv": [P, I, P, P, P],
        "ftlm_hv_block": [P, I, I, P, P, P],
        "ftlm_lanczos_workspace_bytes": [P, I, I, I, PU64],
        "ftlm_lanczos": [P, I, I, U64, I, I, P, U64, P, P, P, P, P, P],
        "ftlm_lanczos_from": [P, I, I, P, I, P, U64, P, P, P, P, P, P],
        "ftlm_lanczos_noalloc": [P, I, I, U64, I, I, P, P, P, P, P, P],
        "ftlm_ritz": [I, I, P, P, P, P, P, P],
        "ftlm_ritz_status": [P, PU64],
        "ftlm_ritz_set_max_sweeps": [I],
        "ftlm_thermo": [I, P, P, I, I, P, P, P, I, D, D, I, P, P, P, P, P, P],
        "ftlm_batch_create": [I, P, I, I, I, I, I, P, ctypes.POINTER(P)],
        "ftlm_lanczos_set_block": [I],
        "ftlm_batch_autotune": [I, P, I, I, I, P, ctypes.POINTER(I), ctypes.POINTER(I), P],
        "ftlm_batch_workspace_bytes": [P, PU64],
        "ftlm_batch_create_plan": [I, P, I, I, I, P, P, ctypes.POINTER(P)],
        "ftlm_batch_autotune_plan": [I, P, I, I, I, P, P, P, P, I, ctypes.POINTER(I)],
        "ftlm_batch_run": [P, P, U64, P],
        "ftlm_basis_destroy_async": [P, P],
        "ftlm_batch_destroy_async": [P, P],
        "ftlm_profile_enable": [I],
        "ftlm_launch_count": [PU64],
        "ftlm_partition": [I, P, P, I, I, P, P, P, I, D, I, P, P, P, P],
        "ftlm_ghosts": [I, I, P, P, P, P, P, D, D, P, P, P, P, P, P],
        "ftlm_sigma_emp": [I, I, P, P, P, P],
        "ftlm_profile_read": [PU64, PU64, PD, PU64, PD],
        "ftlm_probe_read_bandwidth": [P, U64, I, P, PD],
        "ftlm_probe_gather_bandwidth": [P, U64, I, I, P, PD],
        "ftlm_flow_create": [I, I, I, I, I, P, U64, P, ctypes.POINTER(P)],
        "ftlm_flow_unit_bytes": [P, I, I, PU64],
        "ftlm_flow_add": [P, P, ctypes.POINTER(I)],
        "ftlm_flow_step": [P, I, P],
        "ftlm_flow_done": [P, P, I, ctypes.POINTER(I)],
        "ftlm_flow_wait_outputs": [P, P],
        "ftlm_flow_set_streams": [P, I],
        "ftlm_flow_status": [P, ctypes.POINTER(I), ctypes.POINTER(I), PU64],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.ftlm_basis_destroy.argtypes = [P]
    L.ftlm_basis_destroy.restype = None
    L.ftlm_batch_destroy.argtypes = [P]
    L.ftlm_batch_destroy.restype = None
    L.ftlm_flow_destroy.argtypes = [P]
    L.ftlm_flow_destroy.restype = None
    L.ftlm_status_string.argtypes = [ctypes.c_int]
    L.ftlm_status_string.restype = ctypes.c_char_p
    L.ftlm_last_error.argtypes = []
    L.ftlm_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(status):
    if status != FTLM_OK:
        raise FtlmError(status, lib().ftlm_last_error().decode())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dtype_code(dt):
    if dt in (torch.float32, F32, "f32", "float32"):
        return F32
    if dt in (torch.float64, F64, "f64", "float64"):
        return F64
    raise ValueError(f"unsupported dtype {dt}")


def torch_dtype(code):
    return torch.float32 if _dtype_code(code) == F32 else torch.float64


# ------------------------------------------------------------ raw entry points
def ftlm_status_string(status):
    return lib().ftlm_status_string(status).decode()


def ftlm_last_error():
    return lib().ftlm_last_error().decode()


def ftlm_basis_create(N, two_sz, bi, bj, J, mode=RANK_AUTO, stream=None):
    bi = np.ascontiguousarray(bi, dtype=np.int32)
    bj = np.ascontiguousarray(bj, dtype=np.int32)
    J = np.ascontiguousarray(J, dtype=np.float64)
    if not (len(bi) == len(bj) == len(J)):
        raise ValueError("bond arrays differ in length")
    out = ctypes.c_void_p()
    _check(lib().ftlm_basis_create(int(N), int(two_sz), len(J), bi.ctypes.data, bj.ctypes.data,
                                   J.ctypes.data, int(mode), _stream(stream), ctypes.byref(out)))
    return out


def ftlm_basis_create_spin(N, two_s, two_sz, bi, bj, J, stream=None):
    bi = np.ascontiguousarray(bi, dtype=np.int32)
    bj = np.ascontiguousarray(bj, dtype=np.int32)
    J = np.ascontiguousarray(J, dtype=np.float64)
    if not (len(bi) == len(bj) == len(J)):
        raise ValueError("bond arrays differ in length")
    out = ctypes.c_void_p()
    _check(lib().ftlm_basis_create_spin(int(N), int(two_s), int(two_sz), len(J), bi.ctypes.data, bj.ctypes.data,
                                        J.ctypes.data, _stream(stream), ctypes.byref(out)))
    return out


def ftlm_basis_destroy(handle):
    lib().ftlm_basis_destroy(handle)


def ftlm_basis_destroy_async(handle, stream=None):
    _check(lib().ftlm_basis_destroy_async(handle, _stream(stream)))


def _u64_query(fn, handle):
    v = ctypes.c_uint64()
    _check(fn(handle, ctypes.byref(v)))
    return v.value


def ftlm_basis_dim(handle):
    return _u64_query(lib().ftlm_basis_dim, handle)


def ftlm_basis_bytes(handle):
    return _u64_query(lib().ftlm_basis_bytes, handle)


def ftlm_basis_updates(handle):
    return _u64_query(lib().ftlm_basis_updates, handle)


def ftlm_basis_mode(handle):
    v = ctypes.c_int()
    _check(lib().ftlm_basis_mode(handle, ctypes.byref(v)))
    return v.value


def ftlm_basis_set_schedule(handle, schedule, rows_per_tile=0):
    _check(lib().ftlm_basis_set_schedule(handle, int(schedule), int(rows_per_tile)))


def ftlm_basis_hv_schedule(handle, B, dtype):
    v = ctypes.c_int()
    _check(lib().ftlm_basis_hv_schedule(handle, int(B), _dtype_code(dtype), ctypes.byref(v)))
    return v.value


def ftlm_basis_labels(handle, first, count, labels, stream=None):
    """labels: int64 device tensor (labels < 2^36 fit), length >= count."""
    _check(lib().ftlm_basis_labels(handle, int(first), int(count), _ptr(labels), _stream(stream)))


def ftlm_basis_rank(handle, labels, index, stream=None):
    """labels: int64 device tensor; index: int64 device tensor of the same length."""
    _check(lib().ftlm_basis_rank(handle, labels.numel(), _ptr(labels), _ptr(index), _stream(stream)))


def ftlm_basis_clt(handle, mask, prefix, stream=None):
    _check(lib().ftlm_basis_clt(handle, _ptr(mask), _ptr(prefix), _stream(stream)))


def ftlm_hv(handle, x, y, stream=None):
    """y = H x; x, y contiguous device tensors of equal float dtype and length D."""
    if x.dtype != y.dtype or not x.is_contiguous() or not y.is_contiguous():
        raise ValueError("x and y must be contiguous and of one dtype")
    _check(lib().ftlm_hv(handle, _dtype_code(x.dtype), _ptr(x), _ptr(y), _stream(stream)))


def ftlm_hv_block(handle, B, x, y, stream=None):
    """Y = H X for B interleaved vectors: x, y contiguous device tensors of D * B
    elements (e.g. shape (D, B)), entry (t, r) at t * B + r."""
    if x.dtype != y.dtype or not x.is_contiguous() or not y.is_contiguous():
        raise ValueError("x and y must be contiguous and of one dtype")
    _check(lib().ftlm_hv_block(handle, _dtype_code(x.dtype), int(B), _ptr(x), _ptr(y), _stream(stream)))


def ftlm_lanczos_workspace_bytes(handle, R, M, dtype):
    v = ctypes.c_uint64()
    _check(lib().ftlm_lanczos_workspace_bytes(handle, int(R), int(M), _dtype_code(dtype), ctypes.byref(v)))
    return v.value


def ftlm_lanczos(handle, R, M, seed, dist, dtype, work, theta, weight, m_eff, alpha=None, beta=None,
                 stream=None):
    _check(lib().ftlm_lanczos(handle, int(R), int(M), int(seed) & (2**64 - 1), int(dist),
                              _dtype_code(dtype), _ptr(work), work.numel() * work.element_size(),
                              _ptr(theta), _ptr(weight), _ptr(m_eff), _ptr(alpha), _ptr(beta),
                              _stream(stream)))


def ftlm_lanczos_from(handle, R, M, start, dtype, work, theta, weight, m_eff, alpha=None, beta=None,
                      stream=None):
    if start.dtype != torch.float64 or not start.is_contiguous():
        raise ValueError("start vectors must be a contiguous float64 tensor")
    _check(lib().ftlm_lanczos_from(handle, int(R), int(M), _ptr(start), _dtype_code(dtype), _ptr(work),
                                   work.numel() * work.element_size(), _ptr(theta), _ptr(weight),
                                   _ptr(m_eff), _ptr(alpha), _ptr(beta), _stream(stream)))


def ftlm_lanczos_noalloc(handle, R, M, seed, dist, dtype, theta, weight, m_eff, alpha=None, beta=None,
                         stream=None):
    """ftlm_lanczos with the library's static scratch instead of a workspace (for
    callers that cannot allocate device memory); outputs as for ftlm_lanczos."""
    _check(lib().ftlm_lanczos_noalloc(handle, int(R), int(M), int(seed) & (2**64 - 1), int(dist),
                                      _dtype_code(dtype), _ptr(theta), _ptr(weight), _ptr(m_eff),
                                      _ptr(alpha), _ptr(beta), _stream(stream)))


def ftlm_lanczos_set_block(width):
    _check(lib().ftlm_lanczos_set_block(int(width)))


def ftlm_ritz(n, M, alpha, beta, m, theta, weight, stream=None):
    _check(lib().ftlm_ritz(int(n), int(M), _ptr(alpha), _ptr(beta), _ptr(m), _ptr(theta),
                           _ptr(weight), _stream(stream)))


def ftlm_ritz_status(stream=None):
    """Waits for the stream; returns the number of tridiagonal eigenproblems that did
    not converge since the last call (raises FtlmError FTLM_ENOCONV when non-zero,
    with the count in .unconverged)."""
    v = ctypes.c_uint64()
    st = lib().ftlm_ritz_status(_stream(stream), ctypes.byref(v))
    if st == FTLM_ENOCONV:
        err = FtlmError(st, lib().ftlm_last_error().decode())
        err.unconverged = v.value
        raise err
    _check(st)
    return v.value


def ftlm_ritz_set_max_sweeps(sweeps):
    _check(lib().ftlm_ritz_set_max_sweeps(int(sweeps)))


def ftlm_thermo(two_sz, dims, R, M, thetas, weights, m_effs, mirror_neg, g, h, T, E, C, chi, mag=None,
                stream=None):
    n = len(two_sz)
    tz = (ctypes.c_int * n)(*[int(v) for v in two_sz])
    dm = (ctypes.c_uint64 * n)(*[int(v) for v in dims])
    th = (ctypes.c_void_p * n)(*[t.data_ptr() for t in thetas])
    wt = (ctypes.c_void_p * n)(*[t.data_ptr() for t in weights])
    me = (ctypes.c_void_p * n)(*[t.data_ptr() for t in m_effs])
    _check(lib().ftlm_thermo(n, tz, dm, int(R), int(M), th, wt, me, int(bool(mirror_neg)), float(g),
                             float(h), T.numel(), _ptr(T), _ptr(E), _ptr(C), _ptr(chi), _ptr(mag),
                             _stream(stream)))


def ftlm_partition(two_sz, dims, R, M, thetas, weights, m_effs, mirror_neg, h, T, Z, E0=None, stream=None):
    n = len(two_sz)
    tz = (ctypes.c_int * n)(*[int(v) for v in two_sz])
    dm = (ctypes.c_uint64 * n)(*[int(v) for v in dims])
    th = (ctypes.c_void_p * n)(*[t.data_ptr() for t in thetas])
    wt = (ctypes.c_void_p * n)(*[t.data_ptr() for t in weights])
    me = (ctypes.c_void_p * n)(*[t.data_ptr() for t in m_effs])
    _check(lib().ftlm_partition(n, tz, dm, int(R), int(M), th, wt, me, int(bool(mirror_neg)), float(h), T.numel(),
                                _ptr(T), _ptr(Z), _ptr(E0), _stream(stream)))


def ftlm_ghosts(n, M, alpha, beta, m, theta, weight, c_tau, u, ell, cluster, cweight, flags, count, stream=None):
    _check(lib().ftlm_ghosts(int(n), int(M), _ptr(alpha), _ptr(beta), _ptr(m), _ptr(theta), _ptr(weight),
                             float(c_tau), float(u), _ptr(ell), _ptr(cluster), _ptr(cweight), _ptr(flags),
                             _ptr(count), _stream(stream)))


def ftlm_sigma_emp(obs, mean, sigma, stream=None):
    """obs: (N_s, nT) contiguous float64 device tensor."""
    _check(lib().ftlm_sigma_emp(int(obs.shape[0]), int(obs.shape[1]), _ptr(obs), _ptr(mean), _ptr(sigma),
                                _stream(stream)))


def ghosts(res, c_tau=1.0, u=2.0**-24, stream=None):
    """Cullum-Willoughby diagnostic of the chains of a lanczos(..., keep_coeffs=True)
    result: dict of device tensors ell, cluster, cweight, flags (R x M) and count (R)."""
    R, M = res["alpha"].shape
    dev = res["alpha"].device
    out = {"ell": torch.empty((R, M), dtype=torch.float64, device=dev),
           "cluster": torch.empty((R, M), dtype=torch.int32, device=dev),
           "cweight": torch.empty((R, M), dtype=torch.float64, device=dev),
           "flags": torch.empty((R, M), dtype=torch.int32, device=dev),
           "count": torch.empty(R, dtype=torch.int32, device=dev)}
    ftlm_ghosts(R, M, res["alpha"], res["beta"], res["m_eff"], res["theta"], res["weight"], c_tau, u,
                out["ell"], out["cluster"], out["cweight"], out["flags"], out["count"], stream)
    return out


def ftlm_batch_create(items, M, dist, dtype, block=0, streams=0, stream=None):
    """items: sequence of BatchItem; returns the batch handle."""
    arr = (BatchItem * len(items))(*items)
    out = ctypes.c_void_p()
    _check(lib().ftlm_batch_create(len(items), arr, int(M), int(dist), _dtype_code(dtype), int(block),
                                   int(streams), _stream(stream), ctypes.byref(out)))
    return out


def ftlm_batch_autotune(items, M, dist, dtype, stream=None):
    """Returns (block, streams, times) with times[(block, streams)] = ms of the
    timed run of each candidate."""
    arr = (BatchItem * len(items))(*items)
    b, s = ctypes.c_int(), ctypes.c_int()
    ms = (ctypes.c_float * 12)(*([-1.0] * 12))
    _check(lib().ftlm_batch_autotune(len(items), arr, int(M), int(dist), _dtype_code(dtype), _stream(stream),
                                     ctypes.byref(b), ctypes.byref(s), ms))
    times = {(blk, st): ms[i * 4 + j] for i, blk in enumerate((4, 8, 16)) for j, st in enumerate((1, 2, 4, 8))
             if ms[i * 4 + j] >= 0}
    return b.value, s.value, times


def ftlm_batch_create_plan(items, M, dist, dtype, plan, stream=None):
    arr = (BatchItem * len(items))(*items)
    out = ctypes.c_void_p()
    _check(lib().ftlm_batch_create_plan(len(items), arr, int(M), int(dist), _dtype_code(dtype), ctypes.byref(plan),
                                        _stream(stream), ctypes.byref(out)))
    return out


def ftlm_batch_autotune_plan(items, M, dist, dtype, stream=None):
    """Returns (best plan, [(plan tuple, ms) of every timed candidate])."""
    arr = (BatchItem * len(items))(*items)
    best = BatchPlan()
    tried = (BatchPlan * 32)()
    ms = (ctypes.c_float * 32)()
    n = ctypes.c_int()
    _check(lib().ftlm_batch_autotune_plan(len(items), arr, int(M), int(dist), _dtype_code(dtype), _stream(stream),
                                          ctypes.byref(best), tried, ms, 32, ctypes.byref(n)))
    return best, [(tried[i].as_tuple(), ms[i]) for i in range(min(n.value, 32))]


def ftlm_batch_workspace_bytes(handle):
    return _u64_query(lib().ftlm_batch_workspace_bytes, handle)


def ftlm_batch_run(handle, work, stream=None):
    _check(lib().ftlm_batch_run(handle, _ptr(work), work.numel() * work.element_size(), _stream(stream)))


def ftlm_batch_destroy(handle):
    lib().ftlm_batch_destroy(handle)


def ftlm_batch_destroy_async(handle, stream=None):
    _check(lib().ftlm_batch_destroy_async(handle, _stream(stream)))


def ftlm_launch_count():
    return _u64_query(lambda h, p: lib().ftlm_launch_count(p), None)


def ftlm_probe_read_bandwidth(buf, reps, stream=None):
    """GB/s of `reps` coalesced passes over the device tensor buf (L2-resident when it
    fits in L2)."""
    v = ctypes.c_double()
    _check(lib().ftlm_probe_read_bandwidth(_ptr(buf), buf.numel() * buf.element_size(), int(reps), _stream(stream),
                                           ctypes.byref(v)))
    return v.value


def ftlm_probe_gather_bandwidth(buf, run, reps, stream=None):
    """GB/s of `reps` passes over the 32-byte rows of the device tensor buf in an order
    scrambled by blocks of `run` rows (1: scattered rows; 32: 1 KB runs per warp)."""
    v = ctypes.c_double()
    _check(lib().ftlm_probe_gather_bandwidth(_ptr(buf), buf.numel() * buf.element_size(), int(run), int(reps),
                                             _stream(stream), ctypes.byref(v)))
    return v.value


def ftlm_profile_enable(on=True):
    _check(lib().ftlm_profile_enable(int(bool(on))))


def ftlm_profile_read():
    """(hv_launches, hv_vectors, hv_ms, update_launches, update_ms) since the last read."""
    a, v, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    b, d = ctypes.c_double(), ctypes.c_double()
    _check(lib().ftlm_profile_read(ctypes.byref(a), ctypes.byref(v), ctypes.byref(b), ctypes.byref(c),
                                   ctypes.byref(d)))
    return a.value, v.value, b.value, c.value, d.value


# --------------------------------------------------------------- convenience
def ftlm_basis_create_sectors(N, two_s, two_sz, bi, bj, J, mode=RANK_AUTO, wait=True, stream=None):
    """Handles of the sectors two_sz (a list) of one cluster: one wait for all
    tables, or (wait=False) none: uses on other streams must follow `stream`."""
    bi = np.ascontiguousarray(bi, dtype=np.int32)
    bj = np.ascontiguousarray(bj, dtype=np.int32)
    J = np.ascontiguousarray(J, dtype=np.float64)
    if not (len(bi) == len(bj) == len(J)):
        raise ValueError("bond arrays differ in length")
    tz = np.ascontiguousarray(two_sz, dtype=np.int32)
    out = (ctypes.c_void_p * len(tz))()
    _check(lib().ftlm_basis_create_sectors(int(N), int(two_s), len(tz), tz.ctypes.data, len(J), bi.ctypes.data,
                                           bj.ctypes.data, J.ctypes.data, int(mode), int(bool(wait)),
                                           _stream(stream), out))
    return [ctypes.c_void_p(out[k]) for k in range(len(tz))]


class Basis:
    """One S^z sector of a cluster on the current CUDA device (owns the handle).
    Basis.sectors builds several sectors of one cluster with one wait."""

    def __init__(self, N, two_sz, bonds, mode=RANK_AUTO, stream=None, two_s=1, handle=None):
        bi, bj, J = bonds
        self.N, self.two_sz, self.two_s = int(N), int(two_sz), int(two_s)
        self.K = (self.N * self.two_s + self.two_sz) // 2  # digit sum (up spins at s = 1/2)
        if handle is not None:
            self.handle = handle
        elif self.two_s == 1:
            self.handle = ftlm_basis_create(N, two_sz, bi, bj, J, mode, stream)
        else:
            self.handle = ftlm_basis_create_spin(N, two_s, two_sz, bi, bj, J, stream)
        self.dim = ftlm_basis_dim(self.handle)
        self.table_bytes = ftlm_basis_bytes(self.handle)
        self.mode = ftlm_basis_mode(self.handle)
        self.updates = ftlm_basis_updates(self.handle)

    @classmethod
    def sectors(cls, N, two_sz, bonds, mode=RANK_AUTO, stream=None, two_s=1, wait=True):
        """The sectors two_sz (a list) of one cluster (ftlm_basis_create_sectors)."""
        hs = ftlm_basis_create_sectors(N, two_s, two_sz, *bonds, mode=mode, wait=wait, stream=stream)
        return [cls(N, tz, bonds, mode, two_s=two_s, handle=h) for tz, h in zip(two_sz, hs)]

    def set_schedule(self, schedule, rows_per_tile=0):
        """ftlm_basis_set_schedule: walks of the Lanczos H.v launches of this sector."""
        ftlm_basis_set_schedule(self.handle, schedule, rows_per_tile)
        return self

    def close(self):
        if self.handle is not None:
            ftlm_basis_destroy(self.handle)
            self.handle = None

    def release(self, stream=None):
        """Release without waiting: the tables return to the library's pool in the
        order of `stream` (all work that reads them must precede that point)."""
        if self.handle is not None:
            h, self.handle = self.handle, None
            ftlm_basis_destroy_async(h, stream)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lanczos(basis, R, M, seed=1, dist=GAUSS, dtype=torch.float32, start=None, work=None,
            keep_coeffs=False, stream=None):
    """Run R chains on one sector; returns dict of device tensors theta, weight
    (R x M), m_eff (R), and alpha, beta when keep_coeffs."""
    dev = torch.device("cuda", torch.cuda.current_device())
    code = _dtype_code(dtype)
    nbytes = ftlm_lanczos_workspace_bytes(basis.handle, R, M, code)
    if work is None or work.numel() * work.element_size() < nbytes:
        work = torch.empty((nbytes + 255) // 256 * 256, dtype=torch.uint8, device=dev)
    out = {
        "theta": torch.empty((R, M), dtype=torch.float64, device=dev),
        "weight": torch.empty((R, M), dtype=torch.float64, device=dev),
        "m_eff": torch.empty(R, dtype=torch.int32, device=dev),
    }
    if keep_coeffs:
        out["alpha"] = torch.empty((R, M), dtype=torch.float64, device=dev)
        out["beta"] = torch.empty((R, M), dtype=torch.float64, device=dev)
    args = (work, out["theta"], out["weight"], out["m_eff"], out.get("alpha"), out.get("beta"))
    if start is None:
        ftlm_lanczos(basis.handle, R, M, seed, dist, code, *args, stream=stream)
    else:
        ftlm_lanczos_from(basis.handle, R, M, start, code, *args, stream=stream)
    return out


def thermo(sectors, T, R, M, g=2.0, h=0.0, mirror=True, stream=None):
    """sectors: list of (two_sz, dim, result-dict-of-lanczos); T: device float64."""
    dev = T.device
    out = {k: torch.empty_like(T) for k in ("E", "C", "chi", "mag")}
    ftlm_thermo([s[0] for s in sectors], [s[1] for s in sectors], R, M,
                [s[2]["theta"] for s in sectors], [s[2]["weight"] for s in sectors],
                [s[2]["m_eff"] for s in sectors], mirror, g, h, T, out["E"], out["C"], out["chi"],
                out["mag"], stream=stream)
    return out


def _batch_items(entries, M, dev):
    results, items = [], []
    for basis, R, seed, first_chain in entries:
        out = {"theta": torch.zeros((R, M), dtype=torch.float64, device=dev),
               "weight": torch.zeros((R, M), dtype=torch.float64, device=dev),
               "m_eff": torch.zeros(R, dtype=torch.int32, device=dev)}
        results.append(out)
        items.append(BatchItem(basis.handle.value, int(R), int(first_chain), int(seed) & (2**64 - 1),
                               out["theta"].data_ptr(), out["weight"].data_ptr(), out["m_eff"].data_ptr()))
    return results, items


def autotune_plan(entries, M, dist=GAUSS, dtype=torch.float32, stream=None):
    """ftlm_batch_autotune_plan on the (basis, R, seed, first_chain) entries (outputs
    in scratch tensors); returns (best BatchPlan, timed candidates)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    results, items = _batch_items(entries, M, dev)
    out = ftlm_batch_autotune_plan(items, M, dist, dtype, stream)
    del results
    return out


def autotune(entries, M, dist=GAUSS, dtype=torch.float32, stream=None):
    """ftlm_batch_autotune on the (basis, R, seed, first_chain) entries (outputs in
    scratch tensors); returns (block, streams, times)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    results, items = _batch_items(entries, M, dev)
    out = ftlm_batch_autotune(items, M, dist, dtype, stream)
    del results
    return out


class Batch:
    """Many sectors in one batch (ftlm_batch_*): chains of every (basis, R, seed,
    first_chain) entry; outputs per entry as device tensors theta, weight (R x M)
    and m_eff (R)."""

    def __init__(self, entries, M, dist=GAUSS, dtype=torch.float32, block=0, streams=0, stream=None, lazy=False,
                 plan=None):
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self.M = int(M)
        self.results, items = _batch_items(entries, M, self.dev)
        if plan is not None:
            self.handle = ftlm_batch_create_plan(items, M, dist, dtype, plan, stream)
        else:
            self.handle = ftlm_batch_create(items, M, dist, dtype, block, streams, stream)
        self.workspace_bytes = (ftlm_batch_workspace_bytes(self.handle) + 255) // 256 * 256
        self.work = None
        if not lazy:
            self.alloc()

    def alloc(self):
        """The workspace (torch memory on the current stream), allocated on first use."""
        if self.work is None:
            self.work = torch.empty(self.workspace_bytes, dtype=torch.uint8, device=self.dev)
        return self.work

    def run(self, stream=None):
        ftlm_batch_run(self.handle, self.alloc(), stream)
        return self.results

    def close(self):
        if self.handle is not None:
            ftlm_batch_destroy(self.handle)
            self.handle = None

    def release(self, stream=None):
        """Release without waiting, in the order of `stream` (see Basis.release)."""
        if self.handle is not None:
            h, self.handle = self.handle, None
            ftlm_batch_destroy_async(h, stream)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Flow:
    """Continuous Lanczos flow (ftlm_flow_*): sectors join and leave at Lanczos-step
    boundaries.  The workspace is a torch tensor of work_bytes (default: 60 % of the
    free device memory); add() returns a ticket, or None when the sector does not
    fit now; streams: wave streams (1..4, default 4); done(stream) returns
    (ticket, outputs, owner) of finished sectors and
    makes `stream` (default: the current stream) wait until their outputs are
    written (their Ritz step runs on the flow's own stream)."""

    def __init__(self, M, dist=GAUSS, dtype=torch.float32, block=8, max_units=512, work_bytes=None, stream=None,
                 streams=None):
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self.M, self.block = int(M), int(block)
        if work_bytes is None:
            free, _ = torch.cuda.mem_get_info(self.dev)
            work_bytes = int(0.6 * free)
        self.work = torch.empty((int(work_bytes) + 255) // 256 * 256, dtype=torch.uint8, device=self.dev)
        out = ctypes.c_void_p()
        _check(lib().ftlm_flow_create(_dtype_code(dtype), self.block, self.M, int(dist), int(max_units),
                                      _ptr(self.work), self.work.numel(), _stream(stream), ctypes.byref(out)))
        self.handle = out
        self.outputs = {}  # ticket -> (outputs dict, owner)
        if streams is not None:
            _check(lib().ftlm_flow_set_streams(self.handle, int(streams)))

    def add(self, basis, R, seed, first_chain=0, owner=None):
        # no fill kernel: the Ritz launch writes every entry, on the flow's own stream,
        # which is not ordered after the caller's current stream
        out = {"theta": torch.empty((R, self.M), dtype=torch.float64, device=self.dev),
               "weight": torch.empty((R, self.M), dtype=torch.float64, device=self.dev),
               "m_eff": torch.empty(R, dtype=torch.int32, device=self.dev)}
        item = BatchItem(basis.handle.value, int(R), int(first_chain), int(seed) & (2**64 - 1),
                         out["theta"].data_ptr(), out["weight"].data_ptr(), out["m_eff"].data_ptr())
        t = ctypes.c_int()
        st = lib().ftlm_flow_add(self.handle, ctypes.byref(item), ctypes.byref(t))
        if st == FTLM_ENOMEM:
            return None
        _check(st)
        self.outputs[t.value] = (out, owner)
        return t.value

    def step(self, steps=1, stream=None):
        _check(lib().ftlm_flow_step(self.handle, int(steps), _stream(stream)))

    def done(self, stream=None):
        buf = (ctypes.c_int * 256)()
        n = ctypes.c_int()
        res = []
        while True:
            _check(lib().ftlm_flow_done(self.handle, buf, 256, ctypes.byref(n)))
            for i in range(n.value):
                out, owner = self.outputs.pop(buf[i])
                res.append((buf[i], out, owner))
            if n.value < 256:
                break
        if res:
            _check(lib().ftlm_flow_wait_outputs(self.handle, _stream(stream)))
        return res

    def status(self):
        u, s_, f = ctypes.c_int(), ctypes.c_int(), ctypes.c_uint64()
        _check(lib().ftlm_flow_status(self.handle, ctypes.byref(u), ctypes.byref(s_), ctypes.byref(f)))
        return {"units": u.value, "sectors": s_.value, "free_bytes": f.value}

    def close(self):
        if self.handle is not None:
            lib().ftlm_flow_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ftlm_flow_unit_bytes(handle, dtype, block):
    v = ctypes.c_uint64()
    _check(lib().ftlm_flow_unit_bytes(handle, _dtype_code(dtype), int(block), ctypes.byref(v)))
    return v.value


def computed_two_sz(N, two_s=1):
    """2 S^z of the sectors with S^z >= 0 (local spin two_s / 2)."""
    top = N * two_s
    return list(range(top % 2, top + 1, 2))


def run_ftlm(N, bonds, R, M, T, seed=1, dist=GAUSS, dtype=torch.float32, g=2.0, h=0.0,
             sectors=None, mode=RANK_AUTO, keep_coeffs=False, stream=None):
    """A whole FTLM job on the device: for each sector (default: every S^z >= 0,
    mirrored), R chains of M steps, then E, C, chi, mag on the grid T."""
    dev = torch.device("cuda", torch.cuda.current_device())
    if not torch.is_tensor(T):
        T = torch.as_tensor(np.asarray(T, dtype=np.float64), device=dev)
    two = computed_two_sz(N) if sectors is None else list(sectors)
    res, work = [], None
    for tz in two:
        with Basis(N, tz, bonds, mode, stream) as b:
            r = lanczos(b, R, M, seed, dist, dtype, work=work, keep_coeffs=keep_coeffs, stream=stream)
            res.append((tz, b.dim, r))
    obs = thermo(res, T, R, M, g, h, mirror=sectors is None, stream=stream)
    obs["sectors"] = res
    return obs
