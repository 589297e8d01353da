"""Thin ctypes binding of the hefx C ABI (include/hefx.h).

Argument marshalling only: every transform, product and conversion runs in libhefx.so's
CUDA kernels.  Device buffers are passed as raw pointers (torch tensors are accepted and
their data_ptr() used); streams as cudaStream_t handles (torch streams accepted).  There
is no CPU fallback: loading fails loudly when the library is missing or does not load.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhefx.so")

HEFX_OK, HEFX_EINVAL, HEFX_EUNSUPPORTED, HEFX_ENOMEM, HEFX_EBUDGET, HEFX_ECUDA, HEFX_ETIMEOUT = range(7)
STATUS_NAMES = ["HEFX_OK", "HEFX_EINVAL", "HEFX_EUNSUPPORTED", "HEFX_ENOMEM", "HEFX_EBUDGET", "HEFX_ECUDA",
                "HEFX_ETIMEOUT"]
HEFX_PATH_AUTO, HEFX_PATH_CUDACORE, HEFX_PATH_TENSOR = 0, 1, 2
PATHS = {"auto": HEFX_PATH_AUTO, "cudacore": HEFX_PATH_CUDACORE, "tensor": HEFX_PATH_TENSOR}
REDUCTIONS = {"shoup": 0, "montgomery": 1, "barrett": 2, "bat_lazy": 3}
CC_SCHEDULES = {"auto": 0, "cluster": 1, "two_pass": 2}

# Every symbol include/hefx.h declares, with its ctypes signature.
_vp, _u32, _sz, _i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_size_t, ctypes.c_int
_u32p = ctypes.POINTER(ctypes.c_uint32)
SIGNATURES = {
    "hefx_create": (_i32, [ctypes.POINTER(_vp), _i32]),
    "hefx_destroy": (None, [_vp]),
    "hefx_last_error": (ctypes.c_char_p, [_vp]),
    "hefx_version": (ctypes.c_char_p, []),
    "hefx_params_create": (_i32, [_vp, _u32, _u32p, _u32, ctypes.POINTER(_vp)]),
    "hefx_params_destroy": (None, [_vp]),
    "hefx_params_set_auto_path": (_i32, [_vp, _i32]),
    "hefx_params_set_reduction": (_i32, [_vp, _i32, _i32]),
    "hefx_params_set_tensor_config": (_i32, [_vp, _u32, _u32, _u32]),
    "hefx_params_set_cc_schedule": (_i32, [_vp, _i32]),
    "hefx_ntt_fwd": (_i32, [_vp, _vp, _vp, _sz, _i32, _vp]),
    "hefx_ntt_inv": (_i32, [_vp, _vp, _vp, _sz, _i32, _vp]),
    "hefx_poly_mul": (_i32, [_vp, _vp, _vp, _vp, _vp, _sz, _i32, _vp]),
    "hefx_poly_mul_noalloc": (_i32, [_vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "hefx_bconv_plan_create": (_i32, [_vp, _u32, _u32p, _u32, _u32p, _u32, ctypes.POINTER(_vp)]),
    "hefx_bconv_plan_destroy": (None, [_vp]),
    "hefx_basis_convert": (_i32, [_vp, _vp, _vp, _vp, _sz, _i32, _vp]),
    "hefx_stream_check": (_i32, [_vp, _vp, _vp]),
    "hefx_wait_check": (_i32, [_vp, _vp, ctypes.c_uint64, _i32, _vp]),
    "hefx_vec_mod_mul": (_i32, [_vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "hefx_tensor_product": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "hefx_vec_mod_add": (_i32, [_vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "hefx_basis_convert_exact": (_i32, [_vp, _vp, _vp, _vp, _sz, _vp]),
    "hefx_bconv_check": (_i32, [_vp, _vp, _vp]),
    "hefx_key_inner_product": (_i32, [_vp, _vp, _vp, _vp, _vp, _u32, _sz, _vp]),
    "hefx_mod_down": (_i32, [_vp, _vp, _vp, _vp, _sz, _vp]),
    "hefx_modup_plan_create": (_i32, [_vp, _u32, _u32p, _u32, _u32p, _u32, _u32, ctypes.POINTER(_vp)]),
    "hefx_modup_plan_destroy": (None, [_vp]),
    "hefx_modup_plan_dnum": (_u32, [_vp]),
    "hefx_mod_up": (_i32, [_vp, _vp, _vp, _vp, _sz, _vp]),
    "hefx_rescale": (_i32, [_vp, _vp, _vp, _vp, _sz, _vp]),
    "hefx_rescale_ntt": (_i32, [_vp, _vp, _vp, _vp, _sz, _vp]),
    "hefx_ntt_inv_hadamard": (_i32, [_vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "hefx_mult_plan_create": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(_vp)]),
    "hefx_mult_plan_destroy": (None, [_vp]),
    "hefx_mult_front": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "hefx_mult_front_host": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "hefx_mult_batch_create": (_i32, [_vp, _u32, _u32, ctypes.POINTER(_vp)]),
    "hefx_mult_batch_destroy": (None, [_vp]),
    "hefx_mult_front_batch_host": (_i32, [_vp, _vp, _vp, _u32, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "hefx_mult_front_batch": (_i32, [_vp, _vp, _vp, _u32, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "hefx_serve_run": (_i32, [_vp, _vp, _vp, _sz, _vp, _vp]),
    "hefx_batch_plan_create": (_i32, [_vp, _vp, _sz, _i32, ctypes.POINTER(_vp)]),
    "hefx_batch_plan_destroy": (None, [_vp]),
    "hefx_batch_polymul": (_i32, [_vp, _vp, _vp]),
    "hefx_batch_plan_launches": (_u32, [_vp]),
}


class hefx_job(ctypes.Structure):
    _fields_ = [("params", ctypes.c_void_p), ("nlimbs", ctypes.c_uint32), ("d_a", ctypes.c_void_p),
                ("d_b", ctypes.c_void_p), ("d_c", ctypes.c_void_p)]

_lib = None


def load(path: str = LIB_PATH):
    """Loads libhefx.so (building it first if absent) and binds every declared symbol."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            from . import build as _build
            _build.build()
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class HefxError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


def _ptr(x) -> int:
    if x is None:
        return 0
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return int(x)


def _stream(s) -> int:
    if s is None:
        return 0
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream
    return int(s)


def _path(p) -> int:
    return PATHS[p] if isinstance(p, str) else int(p)


def _u32_array(vals):
    arr = (ctypes.c_uint32 * len(vals))(*[int(v) for v in vals])
    return arr


# ----------------------------------------------------------------------------- raw C ABI

def hefx_create(device: int = 0) -> int:
    h = _vp()
    st = load().hefx_create(ctypes.byref(h), device)
    if st != HEFX_OK:
        raise HefxError(st, f"hefx_create(device={device}) failed")
    return h.value


def hefx_destroy(ctx: int) -> None:
    load().hefx_destroy(ctx)


def hefx_last_error(ctx: int) -> str:
    return (load().hefx_last_error(ctx) or b"").decode()


def hefx_version() -> str:
    return load().hefx_version().decode()


def _check(ctx: int, st: int):
    if st != HEFX_OK:
        raise HefxError(st, hefx_last_error(ctx))


def hefx_params_create(ctx: int, log2n: int, primes) -> int:
    h = _vp()
    arr = _u32_array(primes)
    _check(ctx, load().hefx_params_create(ctx, log2n, arr, len(primes), ctypes.byref(h)))
    return h.value


def hefx_params_destroy(params: int) -> None:
    load().hefx_params_destroy(params)


def hefx_params_set_auto_path(params: int, path) -> int:
    return load().hefx_params_set_auto_path(params, _path(path))


def hefx_params_set_reduction(ctx, params: int, ntt_red="shoup", vec_red="montgomery") -> None:
    """Reduction of the CUDA-core NTT twiddle products and of VecModMul (the paper's ablation)."""
    _check(ctx, load().hefx_params_set_reduction(params, REDUCTIONS[ntt_red], REDUCTIONS[vec_red]))


def hefx_params_set_cc_schedule(ctx, params: int, schedule="auto") -> None:
    """Schedule of the contiguous CUDA-core transforms: "cluster" (one launch, 8-CTA clusters),
    "two_pass" (N = 2^16: column pass + block pass through L2) or "auto"."""
    _check(ctx, load().hefx_params_set_cc_schedule(params, CC_SCHEDULES[schedule]))


def hefx_params_set_tensor_config(ctx, params: int, log2r: int = 0, tile_outputs: int = 64, log2r2: int = 0) -> None:
    """Tensor-path split (N = 2^log2r x rest, or with log2r2 > 0 the three factors 2^log2r x
    2^log2r2 x rest; log2r = 0: the square two-factor split) and GEMM tile width."""
    _check(ctx, load().hefx_params_set_tensor_config(params, int(log2r), int(log2r2), int(tile_outputs)))


def hefx_ntt_fwd(ctx, params, data, batch, path="cudacore", stream=None) -> None:
    _check(ctx, load().hefx_ntt_fwd(ctx, params, _ptr(data), batch, _path(path), _stream(stream)))


def hefx_ntt_inv(ctx, params, data, batch, path="cudacore", stream=None) -> None:
    _check(ctx, load().hefx_ntt_inv(ctx, params, _ptr(data), batch, _path(path), _stream(stream)))


def hefx_poly_mul(ctx, params, a, b, c, batch, path="cudacore", stream=None) -> None:
    _check(ctx, load().hefx_poly_mul(ctx, params, _ptr(a), _ptr(b), _ptr(c), batch, _path(path), _stream(stream)))


def hefx_poly_mul_noalloc(ctx, params, a, b, c, batch, stream=None) -> None:
    """Tensor-path product whose workspace is a fixed array inside the library (no device
    allocation); see include/hefx.h for the size limit and the sharing rules."""
    _check(ctx, load().hefx_poly_mul_noalloc(ctx, params, _ptr(a), _ptr(b), _ptr(c), batch, _stream(stream)))


def hefx_bconv_plan_create(ctx: int, log2n: int, src, dst) -> int:
    h = _vp()
    _check(ctx, load().hefx_bconv_plan_create(ctx, log2n, _u32_array(src), len(src), _u32_array(dst), len(dst),
                                             ctypes.byref(h)))
    return h.value


def hefx_bconv_plan_destroy(plan: int) -> None:
    load().hefx_bconv_plan_destroy(plan)


def hefx_basis_convert(ctx, plan, d_in, d_out, batch, path="auto", stream=None) -> None:
    _check(ctx, load().hefx_basis_convert(ctx, plan, _ptr(d_in), _ptr(d_out), batch, _path(path), _stream(stream)))


def hefx_stream_check(ctx, params, stream=None) -> None:
    _check(ctx, load().hefx_stream_check(ctx, params, _stream(stream)))


def hefx_wait_check(ctx, params, limit_ns: int, arrive: bool, stream=None) -> None:
    _check(ctx, load().hefx_wait_check(ctx, params, int(limit_ns), int(bool(arrive)), _stream(stream)))


def hefx_vec_mod_mul(ctx, params, x, y, z, batch, stream=None) -> None:
    _check(ctx, load().hefx_vec_mod_mul(ctx, params, _ptr(x), _ptr(y), _ptr(z), batch, _stream(stream)))


def hefx_tensor_product(ctx, params, a0, a1, b0, b1, d0, d1, d2, batch, stream=None) -> None:
    _check(ctx, load().hefx_tensor_product(ctx, params, _ptr(a0), _ptr(a1), _ptr(b0), _ptr(b1), _ptr(d0), _ptr(d1),
                                           _ptr(d2), batch, _stream(stream)))


def hefx_vec_mod_add(ctx, params, x, y, z, batch, stream=None) -> None:
    _check(ctx, load().hefx_vec_mod_add(ctx, params, _ptr(x), _ptr(y), _ptr(z), batch, _stream(stream)))


def hefx_key_inner_product(ctx, params, digits, evk, out, dnum, batch, stream=None) -> None:
    _check(ctx, load().hefx_key_inner_product(ctx, params, _ptr(digits), _ptr(evk), _ptr(out), dnum, batch,
                                              _stream(stream)))


def hefx_bconv_check(ctx, plan, stream=None) -> None:
    """Raises HefxError(ETIMEOUT) if a bounded wait of a conversion launched with `plan` expired."""
    _check(ctx, load().hefx_bconv_check(ctx, plan, _stream(stream)))


def hefx_basis_convert_exact(ctx, plan, x, out, batch, stream=None) -> None:
    _check(ctx, load().hefx_basis_convert_exact(ctx, plan, _ptr(x), _ptr(out), batch, _stream(stream)))


def hefx_mod_down(ctx, plan, x, out, batch, stream=None) -> None:
    _check(ctx, load().hefx_mod_down(ctx, plan, _ptr(x), _ptr(out), batch, _stream(stream)))


def hefx_modup_plan_create(ctx: int, log2n: int, q, p, alpha: int) -> int:
    h = _vp()
    _check(ctx, load().hefx_modup_plan_create(ctx, log2n, _u32_array(q), len(q), _u32_array(p), len(p), alpha,
                                             ctypes.byref(h)))
    return h.value


def hefx_modup_plan_destroy(plan: int) -> None:
    load().hefx_modup_plan_destroy(plan)


def hefx_modup_plan_dnum(plan: int) -> int:
    return int(load().hefx_modup_plan_dnum(plan))


def hefx_mod_up(ctx, plan, c, U, batch, stream=None) -> None:
    _check(ctx, load().hefx_mod_up(ctx, plan, _ptr(c), _ptr(U), batch, _stream(stream)))


def hefx_rescale(ctx, params, x, out, batch, stream=None) -> None:
    _check(ctx, load().hefx_rescale(ctx, params, _ptr(x), _ptr(out), batch, _stream(stream)))



def hefx_ntt_inv_hadamard(ctx, params, x, y, out, batch, stream=None) -> None:
    _check(ctx, load().hefx_ntt_inv_hadamard(ctx, params, _ptr(x), _ptr(y), _ptr(out), batch, _stream(stream)))


def hefx_rescale_ntt(ctx, params, x, out, batch, stream=None) -> None:
    _check(ctx, load().hefx_rescale_ntt(ctx, params, _ptr(x), _ptr(out), batch, _stream(stream)))

def hefx_mult_plan_create(ctx, pq, pp, bc, kq0, kq1, kp0, kp1) -> int:
    h = _vp()
    _check(ctx, load().hefx_mult_plan_create(ctx, pq, pp, bc, _ptr(kq0), _ptr(kq1), _ptr(kp0), _ptr(kp1),
                                             ctypes.byref(h)))
    return h.value


def hefx_mult_plan_destroy(plan) -> None:
    load().hefx_mult_plan_destroy(plan)


def hefx_mult_front(ctx, plan, d_in, d_out, d_work, stream=None) -> None:
    _check(ctx, load().hefx_mult_front(ctx, plan, _ptr(d_in), _ptr(d_out), _ptr(d_work), _stream(stream)))


def hefx_mult_front_host(ctx, plan, h_a0, h_a1, h_b0, h_b1, h_out, d_buf, stream=None) -> None:
    _check(ctx, load().hefx_mult_front_host(ctx, plan, _ptr(h_a0), _ptr(h_a1), _ptr(h_b0), _ptr(h_b1), _ptr(h_out),
                                            _ptr(d_buf), _stream(stream)))


def hefx_batch_plan_create(ctx, jobs, path="auto") -> int:
    """jobs: iterable of (params, nlimbs, a, b, c) with device buffers or pointers."""
    jobs = list(jobs)
    arr = (hefx_job * max(1, len(jobs)))()
    for i, (params, nl, a, b, c) in enumerate(jobs):
        arr[i] = hefx_job(params, nl, _ptr(a), _ptr(b), _ptr(c))
    h = _vp()
    _check(ctx, load().hefx_batch_plan_create(ctx, ctypes.cast(arr, _vp), len(jobs), _path(path), ctypes.byref(h)))
    return h.value


def hefx_batch_plan_destroy(plan) -> None:
    load().hefx_batch_plan_destroy(plan)


def hefx_batch_polymul(ctx, plan, stream=None) -> None:
    _check(ctx, load().hefx_batch_polymul(ctx, plan, _stream(stream)))


def raw_status(fn_name: str, *args) -> int:
    """Calls a C entry point and returns its status code without raising (for error tests)."""
    return getattr(load(), fn_name)(*args)


def hefx_batch_plan_launches(plan) -> int:
    """Kernel launches one hefx_batch_polymul of the plan makes (1 for the fused form)."""
    return int(load().hefx_batch_plan_launches(plan))


def hefx_mult_batch_create(ctx, max_requests: int, max_limbs: int) -> int:
    """Descriptor slots for batched serving requests (hefx_mult_front_batch(_host))."""
    out = _vp()
    _check(ctx, load().hefx_mult_batch_create(ctx, int(max_requests), int(max_limbs), ctypes.byref(out)))
    return out.value


def hefx_mult_batch_destroy(batch) -> None:
    load().hefx_mult_batch_destroy(batch)


def _ptr_array(items):
    return (_vp * len(items))(*[_ptr(x) for x in items])


def hefx_mult_front_batch_host(ctx, batch, plans, h_a0, h_a1, h_b0, h_b1, h_out, d_buf, stream=None) -> None:
    """Several serving requests of one ring degree in shared launches (lists of per-request
    plans and buffers, as in hefx_mult_front_host)."""
    n = len(plans)
    assert all(len(x) == n for x in (h_a0, h_a1, h_b0, h_b1, h_out, d_buf))
    arrs = [_ptr_array(x) for x in (plans, h_a0, h_a1, h_b0, h_b1, h_out, d_buf)]
    _check(ctx, load().hefx_mult_front_batch_host(ctx, batch, arrs[0], n, arrs[1], arrs[2], arrs[3], arrs[4],
                                                  arrs[5], arrs[6], _stream(stream)))


def hefx_mult_front_batch(ctx, batch, plans, d_a0, d_a1, d_b0, d_b1, d_out, d_work, stream=None) -> None:
    """The batched front half on device-resident operands (lists of per-request plans and device
    buffers, as in hefx_mult_front)."""
    n = len(plans)
    assert all(len(x) == n for x in (d_a0, d_a1, d_b0, d_b1, d_out, d_work))
    arrs = [_ptr_array(x) for x in (plans, d_a0, d_a1, d_b0, d_b1, d_out, d_work)]
    _check(ctx, load().hefx_mult_front_batch(ctx, batch, arrs[0], n, arrs[1], arrs[2], arrs[3], arrs[4],
                                             arrs[5], arrs[6], _stream(stream)))


class ServeRequest(ctypes.Structure):
    _fields_ = [("arrival_s", ctypes.c_double), ("plan", _vp), ("d_a0", _vp), ("d_a1", _vp), ("d_b0", _vp),
                ("d_b1", _vp), ("bytes", ctypes.c_uint64)]


class ServeResult(ctypes.Structure):
    _fields_ = [("admitted_s", ctypes.c_double), ("completed_s", ctypes.c_double), ("status", ctypes.c_int32),
                ("slot", ctypes.c_uint32)]


class ServeStats(ctypes.Structure):
    _fields_ = [("max_active", ctypes.c_uint64), ("memory_high_water_bytes", ctypes.c_uint64),
                ("groups", ctypes.c_uint64)]


class ServeConfig(ctypes.Structure):
    _fields_ = [("nstreams", ctypes.c_uint32), ("streams", ctypes.POINTER(_vp)), ("nslots", ctypes.c_uint32),
                ("slot_out", ctypes.POINTER(_vp)), ("slot_work", ctypes.POINTER(_vp)),
                ("budget_bytes", ctypes.c_uint64), ("max_group", ctypes.c_uint32),
                ("stats", ctypes.POINTER(ServeStats))]


SERVE_PENDING, SERVE_RUNNING, SERVE_DONE, SERVE_REJECTED = 0, 1, 2, 3


def hefx_serve_run(ctx, batch, requests, streams, slot_out, slot_work, budget_bytes: int, max_group: int):
    """Native serving loop.  requests: (arrival_s, plan, d_a0, d_a1, d_b0, d_b1, bytes) tuples
    sorted by arrival; streams: CUDA streams (objects with .cuda_stream or handles); slot_out /
    slot_work: the result slots' device buffers.  Returns (results, stats) as ctypes arrays."""
    n = len(requests)
    reqs = (ServeRequest * max(n, 1))()
    for i, (t, plan, a0, a1, b0, b1, nbytes) in enumerate(requests):
        reqs[i] = ServeRequest(float(t), plan, _ptr(a0), _ptr(a1), _ptr(b0), _ptr(b1), int(nbytes))
    res = (ServeResult * max(n, 1))()
    stats = ServeStats()
    st_arr = (_vp * len(streams))(*[_stream(x) for x in streams])
    so = _ptr_array(slot_out)
    sw = _ptr_array(slot_work)
    pv = ctypes.POINTER(_vp)
    cfg = ServeConfig(len(streams), ctypes.cast(st_arr, pv), len(slot_out), ctypes.cast(so, pv), ctypes.cast(sw, pv),
                      int(budget_bytes), int(max_group), ctypes.pointer(stats))
    _check(ctx, load().hefx_serve_run(ctx, batch, ctypes.cast(reqs, _vp), n, ctypes.byref(cfg), ctypes.cast(res, _vp)))
    return res, stats

