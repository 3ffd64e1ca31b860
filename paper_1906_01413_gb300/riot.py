"""Python binding of the RIOT C ABI (include/riot.h): argument marshalling only.

Every function here has the name of the C entry point it calls and passes
device pointers of torch tensors (torch is used for device memory and
streams only).  There is no fallback: if libriot.so is missing or fails to
load, ``load()`` raises.
"""
import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int32, c_int64, c_uint64, c_void_p

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libriot.so")

RIOT_OK = 0
RIOT_MODEL_L96 = 1
RIOT_MODEL_ADVDIFF = 2
RIOT_B_GAUSS_RING = 1
RIOT_B_EXP_SEPARABLE = 2
RIOT_PREC_MIXED = 0
RIOT_PREC_FP64 = 1
RIOT_EIG_TRIDIAG = 0
RIOT_EIG_JACOBI = 1
STATUS = {0: "RIOT_OK", -1: "RIOT_EINVAL", -2: "RIOT_ENOMEM", -3: "RIOT_ECUDA", -4: "RIOT_ENOTSPD",
          -5: "RIOT_ETIMEOUT", -6: "RIOT_ESTATE", -7: "RIOT_ENOCONV", -8: "RIOT_ENONFINITE"}


class AdvDiffDesc(ctypes.Structure):
    _fields_ = [("nx", c_int32), ("ny", c_int32), ("nz", c_int32), ("nblocks", c_int32),
                ("dx", c_double), ("dy", c_double), ("dz", c_double),
                ("u", POINTER(c_double)), ("v", POINTER(c_double)), ("amp", POINTER(c_double)),
                ("kz", POINTER(c_double)), ("emis_b", POINTER(c_double))]


class ModelDesc(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("T", c_int32), ("n", c_int64), ("dt", c_double), ("F", c_double),
                ("advdiff", POINTER(AdvDiffDesc))]


class ObsDesc(ctypes.Structure):
    _fields_ = [("p", c_int64), ("step", POINTER(c_int32)), ("idx", POINTER(c_int32)),
                ("y", POINTER(c_double)), ("sigma", POINTER(c_double)), ("pos", POINTER(c_double))]


class BcovDesc(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("reserved", c_int32), ("length", c_double), ("sigma_b", c_double),
                ("sigma_vec", POINTER(c_double))]


DEV_ALLOC_FN = ctypes.CFUNCTYPE(c_void_p, ctypes.c_size_t, c_void_p, c_void_p)
DEV_FREE_FN = ctypes.CFUNCTYPE(None, c_void_p, ctypes.c_size_t, c_void_p, c_void_p)


class Options(ctypes.Structure):
    _fields_ = [("precision", c_int32), ("kmax", c_int32), ("exact_rr", c_int32), ("eig_method", c_int32),
                ("seed", c_uint64), ("dev_alloc", DEV_ALLOC_FN), ("dev_free", DEV_FREE_FN),
                ("alloc_user", c_void_p)]


def _torch_alloc(nbytes, stream, user):
    """riot_dev_alloc_fn through PyTorch's caching allocator on the current device."""
    try:
        import torch
        return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), int(stream or 0))
    except Exception:   # out of memory: the library reports RIOT_ENOMEM
        return None


def _torch_free(ptr, nbytes, stream, user):
    try:
        import torch
        torch.cuda.caching_allocator_delete(int(ptr))
    except Exception:
        pass


# One pair of callbacks for every context; each Context also keeps a reference, so the
# C thunks outlive every context that may call them.
TORCH_ALLOC = DEV_ALLOC_FN(_torch_alloc)
TORCH_FREE = DEV_FREE_FN(_torch_free)


def _options(precision, kmax, exact_rr, eig_method, seed, torch_allocator):
    if torch_allocator:
        return Options(int(precision), int(kmax), int(bool(exact_rr)), int(eig_method), int(seed), TORCH_ALLOC,
                       TORCH_FREE, None)
    return Options(int(precision), int(kmax), int(bool(exact_rr)), int(eig_method), int(seed),
                   DEV_ALLOC_FN(), DEV_FREE_FN(), None)


class RiotError(RuntimeError):
    def __init__(self, fn, status, msg):
        super().__init__("%s returned %s: %s" % (fn, STATUS.get(status, status), msg))
        self.status = status


_lib = None


def load():
    """Load libriot.so (built in-tree by ``build()``); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libriot.so is not built (%s); run __graft_entry__.build() or "
                           "python -m paper_1906_01413_gb300.build" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    vp = c_void_p
    L.riot_setup.argtypes = [POINTER(vp), POINTER(ModelDesc), POINTER(ObsDesc), POINTER(BcovDesc),
                             POINTER(Options), vp]
    L.riot_outer_begin.argtypes = [vp, vp, vp, POINTER(c_double)]
    L.riot_hessian_apply.argtypes = [vp, vp, vp, c_int64, c_int32, c_int32]
    L.riot_hessian_apply_noalloc.argtypes = [vp, vp, vp, c_int64, c_int32, c_int32]
    L.riot_rsvd.argtypes = [vp, c_int32, c_int32, c_int64, vp, POINTER(c_double)]
    L.riot_increment.argtypes = [vp, vp, POINTER(c_int32)]
    L.riot_analysis_cov_lowrank.argtypes = [vp, c_int32, vp, POINTER(c_double), POINTER(c_int32)]
    L.riot_bsqrt_apply.argtypes = [vp, vp, vp, c_int32, c_int32]
    L.riot_get_state.argtypes = [vp, vp, vp, vp, vp, vp]
    L.riot_get_innovation.argtypes = [vp, vp]
    L.riot_draw_normal.argtypes = [c_uint64, c_int64, c_int64, c_int32, c_int64, c_int32, vp, vp]
    L.riot_l96_forecast.argtypes = [c_int64, c_int32, c_double, c_double, vp, vp, c_int32, vp]
    L.riot_rsvd_timings.argtypes = [vp, POINTER(c_double)]
    L.riot_symm_eig.argtypes = [vp, c_int32, vp, vp, c_int32, vp]
    L.riot_last_error.argtypes = [vp]
    L.riot_last_error.restype = c_char_p
    L.riot_status_string.argtypes = [c_int32]
    L.riot_status_string.restype = c_char_p
    L.riot_set_hvp_config.argtypes = [vp, c_int32, c_int32]
    L.riot_set_hvp_config.restype = c_int32
    L.riot_set_hvp_kernel.argtypes = [vp, c_int32]
    L.riot_set_hvp_kernel.restype = c_int32
    L.riot_set_wait_limit.argtypes = [vp, c_int32]
    L.riot_set_wait_limit.restype = c_int32
    L.riot_quadratic_cost.argtypes = [vp, vp, POINTER(c_double)]
    L.riot_quadratic_cost.restype = c_int32
    L.riot_rsvd_deflated.argtypes = [vp, c_int32, POINTER(c_int32), c_int32, c_double, c_int64, POINTER(c_double),
                                     POINTER(c_int32)]
    L.riot_rsvd_deflated.restype = c_int32
    L.riot_increment_pairs.argtypes = [vp, POINTER(c_int32)]
    L.riot_increment_pairs.restype = c_int32
    L.riot_rsvd_sweeps.argtypes = [vp]
    L.riot_rsvd_sweeps.restype = c_int32
    L.riot_kernel_launches.argtypes = []
    L.riot_kernel_launches.restype = c_uint64
    L.riot_measure_peaks.argtypes = [c_int32, POINTER(c_double), c_int32]
    L.riot_measure_peaks.restype = c_int32
    L.riot_destroy.argtypes = [vp]
    L.riot_destroy.restype = None
    L.riot_batch_create.argtypes = [POINTER(vp), POINTER(vp), c_int32, POINTER(c_int32), c_int32, vp]
    L.riot_batch_autotune.argtypes = [vp, POINTER(c_int32), POINTER(c_int32), POINTER(c_double)]
    L.riot_batch_set_config.argtypes = [vp, c_int32, c_int32]
    L.riot_batch_hessian_apply.argtypes = [vp]
    L.riot_batch_run.argtypes = [vp, c_int64, c_int32, POINTER(c_int32)]
    L.riot_batch_last_error.argtypes = [vp]
    L.riot_batch_last_error.restype = c_char_p
    L.riot_batch_destroy.argtypes = [vp]
    L.riot_batch_destroy.restype = None
    L.riot_get_trajectory.argtypes = [vp, vp]
    L.riot_tc_sgemm.argtypes = [ctypes.c_char, ctypes.c_char, c_int32, c_int32, c_int32, ctypes.c_float, vp, c_int64,
                                vp, c_int64, ctypes.c_float, vp, c_int64, vp]
    L.riot_tc_sgemm.restype = c_int32
    L.riot_varcg.argtypes = [vp, c_int32, vp, POINTER(c_double), POINTER(c_int32)]
    L.riot_varcg.restype = c_int32
    L.riot_tc_gram.argtypes = [c_int32, c_int32, vp, c_int64, vp, c_int64, vp]
    L.riot_tc_gram.restype = c_int32
    L.riot_psas.argtypes = [vp, c_int32, c_int32, c_int64, vp, POINTER(c_double), vp, POINTER(c_int32)]
    L.riot_psas.restype = c_int32
    L.riot_varbl.argtypes = [vp, c_int32, c_int32, vp, vp, POINTER(c_double), POINTER(c_int32)]
    L.riot_varbl.restype = c_int32
    L.riot_precond_enable.argtypes = [vp, c_int32, c_int32]
    L.riot_precond_enable.restype = c_int32
    L.riot_precond_push.argtypes = [vp, c_int32]
    L.riot_precond_push.restype = c_int32
    L.riot_precond_push_pairs.argtypes = [vp, vp, POINTER(c_double), c_int32]
    L.riot_precond_push_pairs.restype = c_int32
    L.riot_precond_apply.argtypes = [vp, vp, vp, c_int32, c_int32]
    L.riot_precond_apply.restype = c_int32
    L.riot_precond_count.argtypes = [vp]
    L.riot_precond_count.restype = c_int32
    L.riot_sketchnet_create.argtypes = [POINTER(vp), c_int32, c_int32, c_int32, c_int32, c_int32, c_int32, c_int32,
                                        c_int32, vp]
    L.riot_sketchnet_num_params.argtypes = [vp]
    L.riot_sketchnet_num_params.restype = c_int64
    L.riot_sketchnet_set_params.argtypes = [vp, vp]
    L.riot_sketchnet_get_params.argtypes = [vp, vp]
    L.riot_sketchnet_forward.argtypes = [vp, vp, c_int32, c_int32, vp, c_int32]
    L.riot_sketchnet_loss_grad.argtypes = [vp, vp, vp, c_int32, c_int32, c_int32, c_double, vp, POINTER(c_double)]
    L.riot_sketchnet_train_step.argtypes = [vp, vp, vp, c_int32, c_int32, c_int32, c_double, ctypes.c_float,
                                            POINTER(c_double)]
    L.riot_sketchnet_input.argtypes = [vp, c_int32, c_int64, c_int32, vp, vp]
    L.riot_sketchnet_destroy.argtypes = [vp]
    L.riot_sketchnet_destroy.restype = None
    L.riot_rsvd_proposal.argtypes = [vp, c_int32, c_int32, c_int64, vp, c_int32, c_double, POINTER(c_double),
                                     POINTER(c_double), POINTER(c_int32)]
    for name in ("riot_setup", "riot_outer_begin", "riot_hessian_apply", "riot_hessian_apply_noalloc",
                 "riot_rsvd", "riot_increment",
                 "riot_analysis_cov_lowrank", "riot_bsqrt_apply", "riot_get_state", "riot_draw_normal",
                 "riot_l96_forecast", "riot_rsvd_timings", "riot_symm_eig", "riot_get_innovation",
                 "riot_batch_create", "riot_batch_autotune", "riot_batch_set_config", "riot_batch_hessian_apply",
                 "riot_batch_run", "riot_get_trajectory", "riot_sketchnet_create", "riot_sketchnet_set_params",
                 "riot_sketchnet_get_params", "riot_sketchnet_forward", "riot_sketchnet_loss_grad",
                 "riot_sketchnet_train_step", "riot_sketchnet_input", "riot_rsvd_proposal"):
        getattr(L, name).restype = c_int32
    _lib = L
    return L


def _ptr(t):
    return None if t is None else c_void_p(t.data_ptr())


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return c_void_p(s.cuda_stream)


def _check(ctx, fn, status):
    if status != RIOT_OK:
        msg = load().riot_last_error(ctx).decode() if ctx else load().riot_status_string(status).decode()
        raise RiotError(fn, status, msg)


# ---- C entry points ------------------------------------------------------------------

def riot_setup(n, T, dt, F, obs_step, obs_idx, obs_y, obs_sigma, length, sigma_b=1.0, sigma_vec=None,
               precision=RIOT_PREC_MIXED, kmax=64, exact_rr=False, seed=0, stream=None,
               eig_method=RIOT_EIG_TRIDIAG, torch_allocator=True):
    """Create a context (host numpy arrays for the observations); returns the handle."""
    L = load()
    st = np.ascontiguousarray(obs_step, dtype=np.int32)
    ix = np.ascontiguousarray(obs_idx, dtype=np.int32)
    yy = np.ascontiguousarray(obs_y, dtype=np.float64)
    sg = np.ascontiguousarray(obs_sigma, dtype=np.float64)
    md = ModelDesc(RIOT_MODEL_L96, int(T), int(n), float(dt), float(F), None)
    od = ObsDesc(int(st.size), st.ctypes.data_as(POINTER(c_int32)), ix.ctypes.data_as(POINTER(c_int32)),
                 yy.ctypes.data_as(POINTER(c_double)), sg.ctypes.data_as(POINTER(c_double)), None)
    sv = None if sigma_vec is None else np.ascontiguousarray(sigma_vec, dtype=np.float64)
    bd = BcovDesc(RIOT_B_GAUSS_RING, 0, float(length), float(sigma_b),
                  None if sv is None else sv.ctypes.data_as(POINTER(c_double)))
    op = _options(precision, kmax, exact_rr, eig_method, seed, torch_allocator)
    h = c_void_p()
    status = L.riot_setup(ctypes.byref(h), ctypes.byref(md), ctypes.byref(od), ctypes.byref(bd),
                          ctypes.byref(op), _stream_handle(stream))
    _check(None, "riot_setup", status)
    return h


def _dp(a):
    return a.ctypes.data_as(POINTER(c_double))


def riot_setup_advdiff(nx, ny, nz, nblocks, T, dt, dx, dy, dz, u, v, amp, kz, emis_b, obs_step, obs_pos, obs_y,
                       obs_sigma, length, sigma_b, precision=RIOT_PREC_MIXED, kmax=64, exact_rr=False, seed=0,
                       stream=None, eig_method=RIOT_EIG_TRIDIAG, torch_allocator=True):
    """riot_setup for the tracer model (RIOT_MODEL_ADVDIFF with RIOT_B_EXP_SEPARABLE)."""
    L = load()
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (u, v, amp, kz, emis_b)]
    ad = AdvDiffDesc(int(nx), int(ny), int(nz), int(nblocks), float(dx), float(dy), float(dz),
                     *[_dp(a) for a in arrs])
    n = int(nblocks) * int(ny) * int(nx)
    md = ModelDesc(RIOT_MODEL_ADVDIFF, int(T), n, float(dt), 0.0, ctypes.pointer(ad))
    st = np.ascontiguousarray(obs_step, dtype=np.int32)
    pos = np.ascontiguousarray(obs_pos, dtype=np.float64).reshape(-1)
    yy = np.ascontiguousarray(obs_y, dtype=np.float64)
    sg = np.ascontiguousarray(obs_sigma, dtype=np.float64)
    od = ObsDesc(int(st.size), st.ctypes.data_as(POINTER(c_int32)), None, _dp(yy), _dp(sg), _dp(pos))
    bd = BcovDesc(RIOT_B_EXP_SEPARABLE, 0, float(length), float(sigma_b), None)
    op = _options(precision, kmax, exact_rr, eig_method, seed, torch_allocator)
    h = c_void_p()
    status = L.riot_setup(ctypes.byref(h), ctypes.byref(md), ctypes.byref(od), ctypes.byref(bd),
                          ctypes.byref(op), _stream_handle(stream))
    _check(None, "riot_setup", status)
    return h


RIOT_HVP_CTA_BARRIER = 0
RIOT_HVP_WARP_PAIRS = 1
RIOT_HVP_WARP_SHUFFLE = 2
RIOT_HVP_CTA_TWO_PER_SM = 3


def riot_set_hvp_kernel(ctx, kernel):
    """FP32 Hessian kernel of a mixed-precision Lorenz-96 context (RIOT_HVP_*)."""
    _check(ctx, "riot_set_hvp_kernel", load().riot_set_hvp_kernel(ctx, int(kernel)))


def riot_set_wait_limit(ctx, polls):
    """Poll bound of the Hessian kernel's waits (< 0: the default); tests of the timeout report."""
    _check(ctx, "riot_set_wait_limit", load().riot_set_wait_limit(ctx, int(polls)))


def riot_quadratic_cost(ctx, dv=None):
    """J~(dv) of Eq. 3 at the last riot_outer_begin's linearisation (FP64); dv None gives J~(0)."""
    J = c_double(0.0)
    _check(ctx, "riot_quadratic_cost", load().riot_quadratic_cost(ctx, _ptr(dv), ctypes.byref(J)))
    return J.value


def riot_rsvd_deflated(ctx, kcols, q=1, rel_floor=0.0, sketch_stream=0, kmax=4096):
    """Deflated multi-level eigendecomposition (mixed precision), kcols columns per level;
    returns the m eigenvalues kept."""
    kc = (c_int32 * len(kcols))(*[int(k) for k in kcols])
    lam = (c_double * kmax)()
    m = c_int32(0)
    _check(ctx, "riot_rsvd_deflated", load().riot_rsvd_deflated(ctx, len(kcols), kc, int(q), float(rel_floor),
                                                                 int(sketch_stream), lam, ctypes.byref(m)))
    return np.array(lam[:m.value])


def riot_increment_pairs(ctx):
    """Number of eigenpairs the last riot_increment retained."""
    m = c_int32(0)
    _check(ctx, "riot_increment_pairs", load().riot_increment_pairs(ctx, ctypes.byref(m)))
    return m.value


def riot_get_innovation(ctx, d):
    _check(ctx, "riot_get_innovation", load().riot_get_innovation(ctx, _ptr(d)))


def riot_outer_begin(ctx, x=None, v=None):
    J = c_double(0.0)
    _check(ctx, "riot_outer_begin", load().riot_outer_begin(ctx, _ptr(x), _ptr(v), ctypes.byref(J)))
    return J.value


def riot_hessian_apply(ctx, W, Y, ncols=None, add_identity=False):
    """Y[:, j] = A W[:, j] (+ W) for column blocks stored as (ncols, n) row-major tensors."""
    ncols = W.shape[0] if ncols is None else ncols
    ld = W.stride(0)
    assert Y.stride(0) == ld and W.is_contiguous() and Y.is_contiguous()
    _check(ctx, "riot_hessian_apply",
           load().riot_hessian_apply(ctx, _ptr(W), _ptr(Y), int(ld), int(ncols), int(bool(add_identity))))


def riot_hessian_apply_noalloc(ctx, W, Y, ncols=None, add_identity=False):
    """As riot_hessian_apply, with the residual scratch in the library's static
    device array (no allocation by the library at call time)."""
    ncols = W.shape[0] if ncols is None else ncols
    ld = W.stride(0)
    assert Y.stride(0) == ld and W.is_contiguous() and Y.is_contiguous()
    _check(ctx, "riot_hessian_apply_noalloc",
           load().riot_hessian_apply_noalloc(ctx, _ptr(W), _ptr(Y), int(ld), int(ncols), int(bool(add_identity))))


def riot_rsvd(ctx, k, q=0, sketch_stream=0, Omega=None):
    lam = (c_double * k)()
    _check(ctx, "riot_rsvd", load().riot_rsvd(ctx, int(k), int(q), int(sketch_stream), _ptr(Omega), lam))
    return np.array(lam[:])


def riot_increment(ctx, dv=None):
    mode = c_int32(-1)
    _check(ctx, "riot_increment", load().riot_increment(ctx, _ptr(dv), ctypes.byref(mode)))
    return mode.value


def riot_analysis_cov_lowrank(ctx, m, LU=None):
    coef = (c_double * m)()
    mode = c_int32(-1)
    _check(ctx, "riot_analysis_cov_lowrank",
           load().riot_analysis_cov_lowrank(ctx, int(m), _ptr(LU), coef, ctypes.byref(mode)))
    return np.array(coef[:]), mode.value


def riot_bsqrt_apply(ctx, x_in, x_out, transpose=False, ncols=1):
    _check(ctx, "riot_bsqrt_apply",
           load().riot_bsqrt_apply(ctx, _ptr(x_in), _ptr(x_out), int(bool(transpose)), int(ncols)))


def riot_get_state(ctx, x=None, v=None, g=None, U=None, lam=None):
    _check(ctx, "riot_get_state", load().riot_get_state(ctx, _ptr(x), _ptr(v), _ptr(g), _ptr(U), _ptr(lam)))


def riot_draw_normal(seed, stream_id, n, ncols, out, ld=None, stream=None):
    import torch
    is_double = int(out.dtype == torch.float64)
    ld = n if ld is None else ld
    status = load().riot_draw_normal(int(seed), int(stream_id), int(n), int(ncols), int(ld), is_double,
                                     _ptr(out), _stream_handle(stream))
    _check(None, "riot_draw_normal", status)


def riot_l96_forecast(n, T, dt, F, x0, out, store_all=True, stream=None):
    status = load().riot_l96_forecast(int(n), int(T), float(dt), float(F), _ptr(x0), _ptr(out),
                                      int(bool(store_all)), _stream_handle(stream))
    _check(None, "riot_l96_forecast", status)


def riot_symm_eig(K, lam, Z, method=RIOT_EIG_TRIDIAG, stream=None):
    """K (k, k) float64 device tensor (symmetric); lam (k,), Z (k, k) outputs (Z column-major)."""
    k = K.shape[0]
    _check(None, "riot_symm_eig",
           load().riot_symm_eig(_ptr(K), int(k), _ptr(lam), _ptr(Z), int(method), _stream_handle(stream)))


def riot_rsvd_timings(ctx):
    ms = (c_double * 6)()
    _check(ctx, "riot_rsvd_timings", load().riot_rsvd_timings(ctx, ms))
    return dict(zip(["hvp", "orth", "kmat", "eig", "ritz", "total"], ms[:]))


def riot_set_hvp_config(ctx, probes_per_cta=0, ring_depth=0):
    _check(ctx, "riot_set_hvp_config", load().riot_set_hvp_config(ctx, int(probes_per_cta), int(ring_depth)))


def riot_rsvd_sweeps(ctx):
    return int(load().riot_rsvd_sweeps(ctx))


def riot_kernel_launches():
    return int(load().riot_kernel_launches())


def riot_measure_peaks(device=0):
    """Measured FP64 / FP32 FMA throughput (TFLOP/s), FP64 FMA, rsqrt, division and refined
    reciprocal latencies (SM cycles) of a GPU and the refined reciprocal's largest error (ulps),
    as a dict."""
    out = (c_double * 7)()
    _check(None, "riot_measure_peaks", load().riot_measure_peaks(int(device), out, 7))
    keys = ("fp64_tflops", "fp32_tflops", "fp64_fma_cycles", "fp64_rsqrt_cycles", "fp64_div_cycles",
            "fp64_rcp_fast_cycles", "fp64_rcp_fast_max_ulps")
    return dict(zip(keys, (float(v) for v in out)))


def riot_destroy(ctx):
    if ctx:
        load().riot_destroy(ctx)


def _bcheck(b, fn, status):
    if status != RIOT_OK:
        msg = load().riot_batch_last_error(b).decode() if b else load().riot_status_string(status).decode()
        raise RiotError(fn, status, msg)


def riot_batch_create(ctxs, k, q, stream=None):
    """Batch of contexts (handles), k per window; returns the batch handle."""
    n = len(ctxs)
    arr = (c_void_p * n)(*[c.value if isinstance(c, c_void_p) else c for c in ctxs])
    ks = (c_int32 * n)(*[int(x) for x in k])
    h = c_void_p()
    _bcheck(None, "riot_batch_create", load().riot_batch_create(ctypes.byref(h), arr, n, ks, int(q),
                                                                 _stream_handle(stream)))
    return h


def riot_batch_autotune(b):
    P, S, ms = c_int32(0), c_int32(0), c_double(0.0)
    _bcheck(b, "riot_batch_autotune", load().riot_batch_autotune(b, ctypes.byref(P), ctypes.byref(S), ctypes.byref(ms)))
    return P.value, S.value, ms.value


def riot_batch_set_config(b, probes_cap=0, ring_depth=0):
    _bcheck(b, "riot_batch_set_config", load().riot_batch_set_config(b, int(probes_cap), int(ring_depth)))


def riot_batch_hessian_apply(b):
    _bcheck(b, "riot_batch_hessian_apply", load().riot_batch_hessian_apply(b))


def riot_batch_run(b, nwin, sketch_stream=0, use_graph=True, check=True):
    """One inner loop of every window; returns the per-window statuses (raises
    on the first failure unless check is False)."""
    st = (c_int32 * nwin)()
    status = load().riot_batch_run(b, int(sketch_stream), int(bool(use_graph)), st)
    if check:
        _bcheck(b, "riot_batch_run", status)
    return list(st)


def riot_batch_destroy(b):
    if b:
        load().riot_batch_destroy(b)


def _need_contiguous(*ts):
    for t in ts:
        if t is not None and not t.is_contiguous():
            raise ValueError("tensor arguments must be contiguous (the C ABI takes plain pointers)")


def riot_varcg(ctx, m, dv=None):
    """Algorithm 1 (VarCG, Lanczos form): returns (theta (Ritz values, decreasing), steps used);
    the increment goes to dv (n float64 device tensor) when given."""
    theta = (c_double * int(m))()
    used = c_int32(0)
    _check(ctx, "riot_varcg", load().riot_varcg(ctx, int(m), _ptr(dv), theta, ctypes.byref(used)))
    return np.array(theta[:used.value]), used.value


def riot_tc_sgemm(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, stream=None):
    """Column-major FP32 GEMM on the tensor cores (pointers of device tensors)."""
    _check(None, "riot_tc_sgemm",
           load().riot_tc_sgemm(ta.encode(), tb.encode(), int(m), int(n), int(k), float(alpha), _ptr(A), int(lda),
                                _ptr(B), int(ldb), float(beta), _ptr(C), int(ldc), _stream_handle(stream)))


def riot_tc_gram(n, k, Y, ldy, G, ldg, stream=None):
    """Lower triangle of G = Y^T Y (column-major FP32 Y, FP64 G) on the tensor cores."""
    _check(None, "riot_tc_gram",
           load().riot_tc_gram(int(n), int(k), _ptr(Y), int(ldy), _ptr(G), int(ldg), _stream_handle(stream)))


def riot_get_trajectory(ctx, traj):
    _check(ctx, "riot_get_trajectory", load().riot_get_trajectory(ctx, _ptr(traj)))


def riot_sketchnet_create(c_in, width, m_out, depth=4, ksize=5, n_max=4096, batch_max=8, r_max=None, stream=None):
    h = c_void_p()
    r_max = m_out if r_max is None else r_max
    _check(None, "riot_sketchnet_create",
           load().riot_sketchnet_create(ctypes.byref(h), int(c_in), int(width), int(m_out), int(depth), int(ksize),
                                        int(n_max), int(batch_max), int(r_max), _stream_handle(stream)))
    return h


def riot_sketchnet_num_params(net):
    return int(load().riot_sketchnet_num_params(net))


def riot_sketchnet_set_params(net, params):
    _check(None, "riot_sketchnet_set_params", load().riot_sketchnet_set_params(net, _ptr(params)))


def riot_sketchnet_get_params(net, params):
    _check(None, "riot_sketchnet_get_params", load().riot_sketchnet_get_params(net, _ptr(params)))


def riot_sketchnet_forward(net, x, Z, bf16=False):
    """x: (B, c_in, n) float32, Z: (B, m, n) float32 (device tensors)."""
    _need_contiguous(x, Z)
    B, _, n = x.shape
    _check(None, "riot_sketchnet_forward", load().riot_sketchnet_forward(net, _ptr(x), int(n), int(B), _ptr(Z),
                                                                          int(bool(bf16))))


def riot_sketchnet_loss_grad(net, x, U, mu, grad=None):
    """U: (B, r, n) float32 orthonormal targets; returns the mean loss."""
    _need_contiguous(x, U, grad)
    B, _, n = x.shape
    L = c_double(0.0)
    _check(None, "riot_sketchnet_loss_grad",
           load().riot_sketchnet_loss_grad(net, _ptr(x), _ptr(U), int(U.shape[1]), int(n), int(B), float(mu),
                                           _ptr(grad), ctypes.byref(L)))
    return L.value


def riot_sketchnet_train_step(net, x, U, mu, lr):
    _need_contiguous(x, U)
    B, _, n = x.shape
    L = c_double(0.0)
    _check(None, "riot_sketchnet_train_step",
           load().riot_sketchnet_train_step(net, _ptr(x), _ptr(U), int(U.shape[1]), int(n), int(B), float(mu),
                                            float(lr), ctypes.byref(L)))
    return L.value


def riot_sketchnet_input(traj, T, n, c_in, x, stream=None):
    _check(None, "riot_sketchnet_input", load().riot_sketchnet_input(_ptr(traj), int(T), int(n), int(c_in), _ptr(x),
                                                                      _stream_handle(stream)))


def riot_sketchnet_destroy(net):
    if net:
        load().riot_sketchnet_destroy(net)


def riot_rsvd_proposal(ctx, k, q, P, m, rho_max=1e-2, sketch_stream=0):
    """riot_rsvd with the proposal P (m, n) float32; returns (lam, rho, used)."""
    _need_contiguous(P)
    lam = (c_double * k)()
    rho = c_double(-1.0)
    used = c_int32(0)
    _check(ctx, "riot_rsvd_proposal",
           load().riot_rsvd_proposal(ctx, int(k), int(q), int(sketch_stream), _ptr(P), int(m), float(rho_max), lam,
                                     ctypes.byref(rho), ctypes.byref(used)))
    return np.array(lam[:]), rho.value, used.value


def riot_psas(ctx, m, q=0, sketch_stream=0, Omega=None, dv=None):
    """One RIOT-PSAS cycle; Omega (m, p) row-major FP64 device tensor (row j = sketch column j)
    or None.  Returns (eigenvalues of the dual Hessian descending, mode)."""
    _need_contiguous(Omega, dv)
    lam = (c_double * m)()
    mode = c_int32(-1)
    _check(ctx, "riot_psas", load().riot_psas(ctx, int(m), int(q), int(sketch_stream), _ptr(Omega), lam, _ptr(dv),
                                              ctypes.byref(mode)))
    return np.array(lam[:]), mode.value


def riot_varbl(ctx, l, m, B0, dv=None):
    """Algorithm 2 from the gradient samples B0, an (l, n) row-major FP64 device tensor (row j =
    sample j).  Returns (Ritz values descending, blocks used)."""
    _need_contiguous(B0, dv)
    theta = (c_double * (l * m))()
    nb = c_int32(0)
    _check(ctx, "riot_varbl", load().riot_varbl(ctx, int(l), int(m), _ptr(B0), _ptr(dv), theta, ctypes.byref(nb)))
    return np.array(theta[: l * nb.value]), nb.value


def riot_precond_enable(ctx, max_cols, rotation=True):
    _check(ctx, "riot_precond_enable", load().riot_precond_enable(ctx, int(max_cols), int(bool(rotation))))


def riot_precond_push(ctx, m):
    _check(ctx, "riot_precond_push", load().riot_precond_push(ctx, int(m)))


def riot_precond_push_pairs(ctx, V, lam):
    """Factor from given pairs: V (m, n) row-major FP64 device tensor (row j = eigenvector j), lam (m,)."""
    _need_contiguous(V)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    m = int(lam.size)
    _check(ctx, "riot_precond_push_pairs",
           load().riot_precond_push_pairs(ctx, _ptr(V), lam.ctypes.data_as(POINTER(c_double)), m))


PRECOND_P, PRECOND_PT, PRECOND_PINV = 0, 1, 2


def riot_precond_apply(ctx, X, Y, op=PRECOND_P):
    """Y = op(P_k) X for (ncols, n) row-major FP64 tensors (column j of the operator = row j)."""
    _need_contiguous(X)
    _need_contiguous(Y)
    ncols = X.shape[0] if X.dim() == 2 else 1
    _check(ctx, "riot_precond_apply", load().riot_precond_apply(ctx, _ptr(X), _ptr(Y), int(ncols), int(op)))


def riot_precond_count(ctx):
    return int(load().riot_precond_count(ctx))


class Context:
    """Owning wrapper: ``with Context(...) as c: riot_rsvd(c.h, ...)``."""

    def __init__(self, **kw):
        self._callbacks = (TORCH_ALLOC, TORCH_FREE)   # alive for as long as this context
        if "nx" in kw:
            self.n = int(kw["nblocks"]) * int(kw["ny"]) * int(kw["nx"])
            self.h = riot_setup_advdiff(**kw)
        else:
            self.n = int(kw["n"])
            self.h = riot_setup(**kw)

    def close(self):
        if self.h:
            riot_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
