"""Python binding of libdino (the C ABI in include/dino.h).

Thin marshalling only: every function below converts numpy arrays to
pointers, calls the C entry point of the same name, checks the status and
copies results into numpy arrays.  All computation happens in the CUDA
library; if `_build/libdino.so` is missing, every call raises.

    import paper_2403_08220_gb300 as dino
    ctx = dino.dino_init()
    sid = dino.dino_load_surrogate(ctx, n_grid=33, prior_gamma=0.1, ...)
"""
from __future__ import annotations

import ctypes as ct
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libdino.so")

DINO_OK = 0
DINO_PENDING = 1
DINO_EINVAL = -1
DINO_ENOMEM = -2
DINO_ECUDA = -3
DINO_EBUSY = -4
DINO_ETIMEOUT = -5
DINO_ENOTFOUND = -6
DINO_ENUMERIC = -7
DINO_ESTATE = -8

DINO_ACT_IDENTITY, DINO_ACT_TANH, DINO_ACT_GELU = 0, 1, 2
DINO_BASIS_KLE, DINO_BASIS_DIS, DINO_BASIS_EXPLICIT = 0, 1, 2
DINO_PREC_FP64, DINO_PREC_BF16 = 0, 1
DINO_NOISE_AUTO, DINO_NOISE_CHOLESKY, DINO_NOISE_PERTURBATION, DINO_NOISE_EIGEN = 0, 1, 2, 3
NOISE_MAP_NAMES = {DINO_NOISE_CHOLESKY: "cholesky", DINO_NOISE_PERTURBATION: "perturbation",
                   DINO_NOISE_EIGEN: "eigen"}
DINO_DIAG_REDUCED, DINO_DIAG_FIELD = 0, 1
DINO_FLAG_TIMING = 1
DINO_FLAG_NO_DIRECT_HOST = 2

_ERRNAMES = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "EBUSY", -5: "ETIMEOUT",
             -6: "ENOTFOUND", -7: "ENUMERIC", -8: "ESTATE"}


class DinoError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"dino error {code} ({_ERRNAMES.get(code, '?')}): {msg}")
        self.code = code


class _Desc(ct.Structure):
    _fields_ = [("n_grid", ct.c_int), ("prior_gamma", ct.c_double), ("prior_delta", ct.c_double),
                ("r", ct.c_int), ("n_layers", ct.c_int), ("widths", ct.POINTER(ct.c_int)),
                ("activation", ct.c_int), ("W", ct.POINTER(ct.POINTER(ct.c_double))),
                ("b", ct.POINTER(ct.POINTER(ct.c_double))), ("basis_kind", ct.c_int),
                ("basis_gauss", ct.POINTER(ct.c_double)), ("E", ct.POINTER(ct.c_double)),
                ("D", ct.POINTER(ct.c_double)), ("y", ct.POINTER(ct.c_double)),
                ("noise_var", ct.c_double), ("precision", ct.c_int), ("fwd_slices", ct.c_int),
                ("jac_slices", ct.c_int), ("noise_map", ct.c_int)]


class _Info(ct.Structure):
    _fields_ = [("N", ct.c_int), ("r", ct.c_int), ("d_y", ct.c_int), ("n_layers", ct.c_int),
                ("precision", ct.c_int), ("noise_map", ct.c_int),
                ("gram_on_tensor_cores", ct.c_int), ("fwd_slices", ct.c_int),
                ("jac_slices", ct.c_int), ("true_model_rank", ct.c_int),
                ("jac_forward", ct.c_int)]


class _DiagResult(ct.Structure):
    _fields_ = [("n_samples", ct.c_int), ("ess_median", ct.c_double), ("msj", ct.c_double),
                ("mpsrf_w", ct.c_double), ("trace_w", ct.c_double), ("trace_v", ct.c_double),
                ("jacobi_sweeps", ct.c_int)]


class _Stats(ct.Structure):
    _fields_ = [("proposals", ct.c_uint64), ("accepts", ct.c_uint64),
                ("nan_rejects", ct.c_uint64), ("sum_alpha", ct.c_double),
                ("stage1_accepts", ct.c_uint64)]


class _TrueDesc(ct.Structure):
    _fields_ = [("r_t", ct.c_int), ("E_t", ct.POINTER(ct.c_double)), ("n_layers", ct.c_int),
                ("widths", ct.POINTER(ct.c_int)), ("activation", ct.c_int),
                ("W", ct.POINTER(ct.POINTER(ct.c_double))),
                ("b", ct.POINTER(ct.POINTER(ct.c_double)))]


class _Request(ct.Structure):
    _fields_ = [("surrogate_id", ct.c_int), ("n_chains", ct.c_int), ("n_steps", ct.c_int),
                ("dt", ct.c_double), ("seed", ct.c_uint64), ("chain_id_base", ct.c_uint64),
                ("m0", ct.POINTER(ct.c_double)), ("m_r_out", ct.POINTER(ct.c_double)),
                ("phi_out", ct.POINTER(ct.c_double)), ("accepts_out", ct.POINTER(ct.c_uint64)),
                ("m_out", ct.POINTER(ct.c_double))]


class _Result(ct.Structure):
    _fields_ = [("stats", _Stats), ("queue_s", ct.c_double), ("latency_s", ct.c_double)]


_lib = None
_P = ct.c_void_p
_D = ct.POINTER(ct.c_double)
_I = ct.c_int

_SIGNATURES = {
    "dino_version": ([], ct.c_int),
    "dino_init": ([ct.POINTER(_P), _I, ct.c_size_t, _P, ct.c_uint], _I),
    "dino_destroy": ([_P], _I),
    "dino_last_error": ([_P], ct.c_char_p),
    "dino_sync": ([_P], _I),
    "dino_load_surrogate": ([_P, ct.POINTER(_Desc), ct.POINTER(_I)], _I),
    "dino_set_data": ([_P, _I, _D, ct.c_double], _I),
    "dino_unload_surrogate": ([_P, _I], _I),
    "dino_read_basis": ([_P, _I, _D, _D], _I),
    "dino_surrogate_eval": ([_P, _I, _I, _D, _D, _D, _D, _D, _D, _D], _I),
    "dino_chains_create": ([_P, _I, _I, ct.c_double, ct.c_uint64, ct.c_uint64, _D,
                            ct.POINTER(_I)], _I),
    "dino_chains_step": ([_P, _I, _I, ct.POINTER(_Stats)], _I),
    "dino_chains_read": ([_P, _I, _D, _D, _D, ct.POINTER(ct.c_uint64)], _I),
    "dino_chains_read_last": ([_P, _I, _D, _D, _D, _D, ct.POINTER(_I)], _I),
    "dino_chains_destroy": ([_P, _I], _I),
    "dino_surrogate_query": ([_P, _I, ct.POINTER(_Info)], _I),
    "dino_chains_set_noise": ([_P, _I, _D, _D, _D, _D, _D], _I),
    "dino_set_true_model": ([_P, _I, ct.POINTER(_TrueDesc)], _I),
    "dino_chains_read_da": ([_P, _I, _D, _D, _D, ct.POINTER(_I)], _I),
    "dino_chains_step_many": ([_P, _I, ct.POINTER(_I), _I], _I),
    "dino_measure_fp32_peak": ([_P, _D], _I),
    "dino_dis_from_surrogate": ([_P, _I, _I, ct.c_uint64, _I, _D, _D, _D, _D], _I),
    "dino_diag_create": ([_P, _I, _I, _I, ct.POINTER(_I)], _I),
    "dino_diag_record": ([_P, _I, _I, _I, _I], _I),
    "dino_diag_push": ([_P, _I, _D], _I),
    "dino_diag_compute": ([_P, _I, _I, _D, ct.POINTER(_DiagResult)], _I),
    "dino_diag_destroy": ([_P, _I], _I),
    "dino_launch_count": ([_P], ct.c_uint64),
    "dino_kernel_times": ([_P, ct.c_char_p, _D, ct.POINTER(ct.c_uint64), _I, ct.POINTER(_I), _I],
                          _I),
    "dino_serve_config": ([_P, _I, _I, _I], _I),
    "dino_serve_submit": ([_P, ct.POINTER(_Request), ct.POINTER(ct.c_uint64)], _I),
    "dino_serve_poll": ([_P, ct.c_uint64, ct.POINTER(_Result)], _I),
    "dino_serve_wait": ([_P, ct.c_uint64, ct.c_double, ct.POINTER(_Result)], _I),
    "dino_serve_status": ([_P, ct.POINTER(_I), ct.POINTER(_I), ct.POINTER(_I),
                           ct.POINTER(ct.c_size_t), ct.POINTER(ct.c_size_t)], _I),
    "dino_surrogate_jacobian_noalloc": ([_I, _I, ct.POINTER(_I), _I, ct.POINTER(_P),
                                         ct.POINTER(_P), _P, _P, _P, _P], _I),
}


def lib():
    """The loaded libdino (raises if the CUDA library has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libdino.so not found at {LIB_PATH}; run "
                              "`python -m paper_2403_08220_gb300.build` (needs nvcc)")
        L = ct.CDLL(LIB_PATH)
        for name, (args, res) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGNATURES)


class Ctx:
    """Handle of a dino_ctx; `close()` (or garbage collection) destroys it."""

    def __init__(self, ptr):
        self.ptr = ptr

    def close(self):
        if self.ptr:
            lib().dino_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _check(ctx: Optional[Ctx], code: int):
    if code != DINO_OK and code != DINO_PENDING:
        msg = lib().dino_last_error(ctx.ptr).decode() if ctx is not None and ctx.ptr else ""
        raise DinoError(code, msg)
    return code


def _dptr(a):
    return None if a is None else a.ctypes.data_as(_D)


def _f64(a, shape=None):
    x = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None and x.shape != tuple(shape):
        x = x.reshape(shape)
    return x


def dino_version() -> int:
    return lib().dino_version()


def dino_init(device: int = 0, hbm_budget_bytes: int = 0, stream=None, flags: int = 0) -> Ctx:
    p = _P()
    code = lib().dino_init(ct.byref(p), device, hbm_budget_bytes,
                           _P(stream) if stream else None, flags)
    _check(None, code)
    return Ctx(p)


def dino_destroy(ctx: Ctx):
    ctx.close()


def dino_last_error(ctx: Ctx) -> str:
    return lib().dino_last_error(ctx.ptr).decode()


def dino_sync(ctx: Ctx):
    _check(ctx, lib().dino_sync(ctx.ptr))


def dino_load_surrogate(ctx: Ctx, *, n_grid, prior_gamma, prior_delta, r, widths, activation,
                        W, b, basis_kind, basis_gauss=None, E=None, D=None, y=None,
                        noise_var=0.0, precision=DINO_PREC_FP64, fwd_slices=0,
                        jac_slices=0, noise_map=DINO_NOISE_AUTO) -> int:
    L = len(W)
    wid = (ct.c_int * (L + 1))(*[int(x) for x in widths])
    Ws = [_f64(w) for w in W]
    bs = [_f64(x) for x in b]
    Wp = (ct.POINTER(ct.c_double) * L)(*[_dptr(w) for w in Ws])
    bp = (ct.POINTER(ct.c_double) * L)(*[_dptr(x) for x in bs])
    G = _f64(basis_gauss) if basis_gauss is not None else None
    Ea = _f64(E) if E is not None else None
    Da = _f64(D) if D is not None else None
    ya = _f64(y) if y is not None else None
    d = _Desc(n_grid, prior_gamma, prior_delta, r, L, wid, activation, Wp, bp, basis_kind,
              _dptr(G), _dptr(Ea), _dptr(Da), _dptr(ya), float(noise_var), precision,
              fwd_slices, jac_slices, int(noise_map))
    sid = _I()
    _check(ctx, lib().dino_load_surrogate(ctx.ptr, ct.byref(d), ct.byref(sid)))
    return sid.value


def dino_set_data(ctx: Ctx, sid: int, y, noise_var: float):
    ya = _f64(y)
    _check(ctx, lib().dino_set_data(ctx.ptr, sid, _dptr(ya), float(noise_var)))


def dino_unload_surrogate(ctx: Ctx, sid: int):
    _check(ctx, lib().dino_unload_surrogate(ctx.ptr, sid))


def dino_read_basis(ctx: Ctx, sid: int, r: int, N: int):
    E = np.empty((r, N))
    D = np.empty((N, r))
    _check(ctx, lib().dino_read_basis(ctx.ptr, sid, _dptr(E), _dptr(D)))
    return E, D


def dino_surrogate_eval(ctx: Ctx, sid: int, m_r, d_y: int, want_L: bool = True) -> dict:
    x = _f64(m_r)
    if x.ndim == 1:
        x = x[None, :]
    n, r = x.shape
    out = dict(f=np.empty((n, d_y)), J=np.empty((n, d_y, r)), phi=np.empty(n),
               g=np.empty((n, r)), L=np.empty((n, r, r)) if want_L else None, hld=np.empty(n))
    _check(ctx, lib().dino_surrogate_eval(ctx.ptr, sid, n, _dptr(x), _dptr(out["f"]),
                                          _dptr(out["J"]), _dptr(out["phi"]), _dptr(out["g"]),
                                          _dptr(out["L"]), _dptr(out["hld"])))
    return out


def dino_chains_create(ctx: Ctx, sid: int, n_chains: int, dt: float, seed: int,
                       chain_id_base: int = 0, m0=None) -> int:
    m = _f64(m0) if m0 is not None else None
    pid = _I()
    _check(ctx, lib().dino_chains_create(ctx.ptr, sid, n_chains, float(dt), int(seed),
                                         int(chain_id_base), _dptr(m), ct.byref(pid)))
    return pid.value


def dino_chains_step(ctx: Ctx, pool: int, n_steps: int, stats: bool = True):
    st = _Stats()
    _check(ctx, lib().dino_chains_step(ctx.ptr, pool, n_steps, ct.byref(st) if stats else None))
    if not stats:
        return None
    return dict(proposals=st.proposals, accepts=st.accepts, nan_rejects=st.nan_rejects,
                sum_alpha=st.sum_alpha, stage1_accepts=st.stage1_accepts)


def dino_chains_read(ctx: Ctx, pool: int, C: int, r: int, N: int, field: bool = True) -> dict:
    out = dict(m=np.empty((C, N)) if field else None, m_r=np.empty((C, r)), phi=np.empty(C),
               accepts=np.empty(C, dtype=np.uint64))
    _check(ctx, lib().dino_chains_read(ctx.ptr, pool, _dptr(out["m"]), _dptr(out["m_r"]),
                                       _dptr(out["phi"]),
                                       out["accepts"].ctypes.data_as(ct.POINTER(ct.c_uint64))))
    return out


def dino_chains_read_last(ctx: Ctx, pool: int, C: int, r: int) -> dict:
    out = dict(b=np.empty((C, r)), mu=np.empty((C, r)), log_rho=np.empty(C),
               log_u=np.empty(C), accepted=np.empty(C, dtype=np.int32))
    _check(ctx, lib().dino_chains_read_last(ctx.ptr, pool, _dptr(out["b"]), _dptr(out["mu"]),
                                            _dptr(out["log_rho"]), _dptr(out["log_u"]),
                                            out["accepted"].ctypes.data_as(ct.POINTER(_I))))
    out["accepted"] = out["accepted"].astype(bool)
    return out


def dino_chains_destroy(ctx: Ctx, pool: int):
    _check(ctx, lib().dino_chains_destroy(ctx.ptr, pool))


def dino_surrogate_query(ctx: Ctx, sid: int) -> dict:
    """Sizes, precision, noise map ("cholesky" / "perturbation") and paths of a surrogate."""
    info = _Info()
    _check(ctx, lib().dino_surrogate_query(ctx.ptr, sid, ct.byref(info)))
    out = {k: getattr(info, k) for k, _ in _Info._fields_}
    out["noise_map"] = NOISE_MAP_NAMES[info.noise_map]
    return out


def dino_chains_set_noise(ctx: Ctx, pool: int, xi=None, xi2=None, z=None, log_u=None,
                          log_u2=None):
    """Caller noise for the pool's next transition (None keeps Philox for that stream)."""
    arrs = [None if a is None else _f64(a) for a in (xi, xi2, z, log_u, log_u2)]
    _check(ctx, lib().dino_chains_set_noise(ctx.ptr, pool, *[_dptr(a) for a in arrs]))


def dino_set_true_model(ctx: Ctx, sid: int, E_t=None, W=None, b=None, activation=0):
    """Attach the true map G(m) = f_t(E_t m) of delayed acceptance (E_t None detaches)."""
    if E_t is None:
        _check(ctx, lib().dino_set_true_model(ctx.ptr, sid, None))
        return
    Et = _f64(E_t)
    Ws = [_f64(w) for w in W]
    bs = [_f64(x) for x in b]
    L = len(Ws)
    widths = [Et.shape[0]] + [w.shape[0] for w in Ws]
    wid = (ct.c_int * (L + 1))(*widths)
    Wp = (ct.POINTER(ct.c_double) * L)(*[_dptr(w) for w in Ws])
    bp = (ct.POINTER(ct.c_double) * L)(*[_dptr(x) for x in bs])
    d = _TrueDesc(Et.shape[0], _dptr(Et), L, wid, int(activation), Wp, bp)
    _check(ctx, lib().dino_set_true_model(ctx.ptr, sid, ct.byref(d)))


def dino_chains_read_da(ctx: Ctx, pool: int, C: int) -> dict:
    out = dict(phi_true=np.empty(C), log_rho2=np.empty(C), log_u2=np.empty(C),
               stage1=np.empty(C, dtype=np.int32))
    _check(ctx, lib().dino_chains_read_da(ctx.ptr, pool, _dptr(out["phi_true"]),
                                          _dptr(out["log_rho2"]), _dptr(out["log_u2"]),
                                          out["stage1"].ctypes.data_as(ct.POINTER(_I))))
    out["stage1"] = out["stage1"].astype(bool)
    return out


def dino_dis_from_surrogate(ctx: Ctx, sid: int, n_samples: int, seed: int, r_new: int, r: int,
                            N: int) -> dict:
    out = dict(eigvals=np.empty(r), P=np.empty((r, r_new)), E=np.empty((r_new, N)),
               D=np.empty((N, r_new)))
    _check(ctx, lib().dino_dis_from_surrogate(ctx.ptr, sid, n_samples, int(seed), r_new,
                                              _dptr(out["eigvals"]), _dptr(out["P"]),
                                              _dptr(out["E"]), _dptr(out["D"])))
    return out


def dino_diag_create(ctx: Ctx, n_chains: int, n_dof: int, max_samples: int) -> int:
    i = _I()
    _check(ctx, lib().dino_diag_create(ctx.ptr, n_chains, n_dof, max_samples, ct.byref(i)))
    return i.value


def dino_diag_record(ctx: Ctx, diag: int, pool: int, what: int = DINO_DIAG_REDUCED,
                     chain0: int = 0):
    _check(ctx, lib().dino_diag_record(ctx.ptr, diag, pool, what, chain0))


def dino_diag_push(ctx: Ctx, diag: int, sample):
    x = _f64(sample)
    _check(ctx, lib().dino_diag_push(ctx.ptr, diag, _dptr(x)))


def dino_diag_compute(ctx: Ctx, diag: int, n_dof: int, mpsrf: bool = True) -> dict:
    ess = np.empty(n_dof)
    r = _DiagResult()
    _check(ctx, lib().dino_diag_compute(ctx.ptr, diag, 1 if mpsrf else 0, _dptr(ess),
                                        ct.byref(r)))
    out = {k: getattr(r, k) for k, _ in _DiagResult._fields_}
    out["ess"] = ess
    return out


def dino_diag_destroy(ctx: Ctx, diag: int):
    _check(ctx, lib().dino_diag_destroy(ctx.ptr, diag))


def dino_chains_step_many(ctx: Ctx, pools, n_steps: int):
    ids = (_I * len(pools))(*[int(p) for p in pools])
    _check(ctx, lib().dino_chains_step_many(ctx.ptr, len(pools), ids, n_steps))


def dino_measure_fp32_peak(ctx: Ctx) -> float:
    t = ct.c_double()
    _check(ctx, lib().dino_measure_fp32_peak(ctx.ptr, ct.byref(t)))
    return t.value


def dino_launch_count(ctx: Ctx) -> int:
    return int(lib().dino_launch_count(ctx.ptr))


def dino_kernel_times(ctx: Ctx, reset: bool = False) -> dict:
    cap = 64
    names = ct.create_string_buffer(48 * cap)
    ms = np.zeros(cap)
    cnt = np.zeros(cap, dtype=np.uint64)
    n = _I()
    _check(ctx, lib().dino_kernel_times(ctx.ptr, names, _dptr(ms),
                                        cnt.ctypes.data_as(ct.POINTER(ct.c_uint64)), cap,
                                        ct.byref(n), 1 if reset else 0))
    out = {}
    raw = names.raw
    for k in range(min(n.value, cap)):
        nm = raw[48 * k:48 * (k + 1)].split(b"\0", 1)[0].decode()
        out[nm] = (float(ms[k]), int(cnt[k]))
    return out


def dino_surrogate_jacobian_noalloc(n: int, widths, activation: int, W_ptrs, b_ptrs, x_ptr: int,
                                    f_ptr: int, J_ptr: int, stream: int = 0) -> None:
    """f and J at n points from caller-owned device buffers, with no device allocation.

    W_ptrs / b_ptrs are device addresses (ints) of the layer weights and biases;
    x_ptr, f_ptr, J_ptr device addresses of the n x r inputs and the n x d_y and
    n x d_y x r outputs (float64, row-major).  The library's fixed scratch array
    is shared by all calls, so calls that may overlap on the GPU must be ordered
    on one stream.
    """
    L = len(W_ptrs)
    wid = (ct.c_int * (L + 1))(*[int(x) for x in widths])
    Wp = (_P * L)(*[int(p) for p in W_ptrs])
    bp = (_P * L)(*[int(p) for p in b_ptrs])
    code = lib().dino_surrogate_jacobian_noalloc(n, L, wid, activation, Wp, bp, _P(x_ptr),
                                                  _P(f_ptr), _P(J_ptr),
                                                  _P(stream) if stream else None)
    if code != DINO_OK:
        raise DinoError(code, "dino_surrogate_jacobian_noalloc rejected the request")


# ---- serving -------------------------------------------------------------

_SERVE_OUT = {}   # (ctx address, ticket) -> numpy outputs kept alive until completion


def dino_serve_config(ctx: Ctx, n_streams: int = 4, steps_per_round: int = 8,
                      max_active: int = 32):
    _check(ctx, lib().dino_serve_config(ctx.ptr, n_streams, steps_per_round, max_active))


def dino_serve_submit(ctx: Ctx, sid: int, n_chains: int, n_steps: int, dt: float, seed: int,
                      r: int, N: int, chain_id_base: int = 0, m0=None,
                      want_field: bool = False) -> int:
    """Queue a request; returns its ticket.  Outputs are filled on completion."""
    out = dict(m_r=np.empty((n_chains, r)), phi=np.empty(n_chains),
               accepts=np.empty(n_chains, dtype=np.uint64),
               m=np.empty((n_chains, N)) if want_field else None)
    m = _f64(m0) if m0 is not None else None
    req = _Request(sid, n_chains, n_steps, float(dt), int(seed), int(chain_id_base), _dptr(m),
                   _dptr(out["m_r"]), _dptr(out["phi"]),
                   out["accepts"].ctypes.data_as(ct.POINTER(ct.c_uint64)), _dptr(out["m"]))
    t = ct.c_uint64()
    _check(ctx, lib().dino_serve_submit(ctx.ptr, ct.byref(req), ct.byref(t)))
    _SERVE_OUT[(ctx.ptr.value, t.value)] = out
    return t.value


def _result(ctx, ticket, res):
    out = _SERVE_OUT.pop((ctx.ptr.value, ticket))
    out.update(stats=dict(proposals=res.stats.proposals, accepts=res.stats.accepts,
                          nan_rejects=res.stats.nan_rejects, sum_alpha=res.stats.sum_alpha,
                          stage1_accepts=res.stats.stage1_accepts),
               queue_s=res.queue_s, latency_s=res.latency_s)
    return out


def dino_serve_poll(ctx: Ctx, ticket: int):
    """None while the request is queued or running, else its outputs."""
    res = _Result()
    code = lib().dino_serve_poll(ctx.ptr, ticket, ct.byref(res))
    if code == DINO_PENDING:
        return None
    _check(ctx, code)
    return _result(ctx, ticket, res)


def dino_serve_wait(ctx: Ctx, ticket: int, timeout_s: float = 600.0):
    res = _Result()
    _check(ctx, lib().dino_serve_wait(ctx.ptr, ticket, float(timeout_s), ct.byref(res)))
    return _result(ctx, ticket, res)


def dino_serve_status(ctx: Ctx) -> dict:
    q, a, pa = _I(), _I(), _I()
    u, pu = ct.c_size_t(), ct.c_size_t()
    _check(ctx, lib().dino_serve_status(ctx.ptr, ct.byref(q), ct.byref(a), ct.byref(pa),
                                        ct.byref(u), ct.byref(pu)))
    return dict(queued=q.value, active=a.value, peak_active=pa.value, hbm_used=u.value,
                peak_hbm_used=pu.value)
