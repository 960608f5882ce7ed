"""ctypes binding of include/thc_sigma.h (argument marshalling only).

Every function has the name of the C entry point it calls.  Array arguments
may be torch tensors (device or pinned host, float64, contiguous) or numpy
float64 arrays (host); ``None`` passes NULL.  A non-zero return code raises
ThcError with the library's message.  Loading fails loudly when the library
has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

THC_OK = 0
THC_EINVAL = -1
THC_ENOMEM = -2
THC_ECUDA = -3
THC_ETIMEOUT = -4
THC_ENOTSUP = -5

THC_FP64 = 0
THC_BF16X3 = 1
THC_TF32 = 2      # not built: thc_sigma_init returns THC_ENOTSUP

THC_DIRECT = 1
THC_SOX = 2
THC_KCLASS_SOX_BCD = 11   # index of sox_BCD among the kernel classes (profiler and autotune table)
THC_GW = 4        # screened direct term (scGW / scGWSOX); needs thc_sigma_set_bosonic

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libthcsigma.so")

_lib = None


class ThcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"thc error {code}: {msg}")
        self.code = code


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Load libthcsigma.so and declare the signatures of include/thc_sigma.h."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with `python -m paper_2404_17744_gb300.build`")
    lib = ctypes.CDLL(p)
    vp, dp, i, d = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.thc_sigma_init.argtypes = [ctypes.POINTER(vp), i, i, i, d, dp, dp, dp, i, i, vp]
    lib.thc_sigma_init.restype = i
    lib.thc_sigma_eval.argtypes = [vp, dp, dp, dp]
    lib.thc_sigma_eval.restype = i
    lib.thc_sigma_set_bosonic.argtypes = [vp, i, dp, dp]
    lib.thc_sigma_set_bosonic.restype = i
    lib.thc_sigma_eval_uhf.argtypes = [vp, dp, dp, dp, dp, dp, dp]
    lib.thc_sigma_eval_uhf.restype = i
    lib.thc_sigma_eval_host.argtypes = [vp, dp, dp, dp]
    lib.thc_sigma_eval_host.restype = i
    lib.thc_energy.argtypes = [vp, dp, dp, dp, dp, ctypes.POINTER(d)]
    lib.thc_energy.restype = i
    lib.thc_set_stream.argtypes = [vp, vp]
    lib.thc_set_stream.restype = i
    lib.thc_sigma_flops.argtypes = [vp, ctypes.POINTER(d)]
    lib.thc_sigma_flops.restype = d
    lib.thc_profile.argtypes = [vp, i]
    lib.thc_profile.restype = i
    lib.thc_profile_get.argtypes = [vp, i, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_longlong),
                                    ctypes.POINTER(d), ctypes.POINTER(d)]
    lib.thc_profile_get.restype = i
    lib.thc_launch_count.argtypes = [vp]
    lib.thc_launch_count.restype = ctypes.c_longlong
    lib.thc_energy_static.argtypes = [i, i, dp, dp, dp, dp, ctypes.POINTER(d), vp]
    lib.thc_energy_static.restype = i
    lib.thc_sync.argtypes = [vp]
    lib.thc_sync.restype = i
    lib.thc_wait_selftest.argtypes = [ctypes.c_longlong, vp]
    lib.thc_wait_selftest.restype = i
    lib.thc_fp64_dfma_rate.argtypes = [ctypes.c_longlong, ctypes.POINTER(d), ctypes.POINTER(d), vp]
    lib.thc_fp64_dfma_rate.restype = i
    ll = ctypes.c_longlong
    lib.thc_gemm_bf16x3.argtypes = [i, i, i, i, dp, ll, dp, ll, dp, ll, vp]
    lib.thc_gemm_bf16x3.restype = i
    lib.thc_destroy.argtypes = [vp]
    lib.thc_destroy.restype = None
    # self-consistency loop (include/thc_dyson.h)
    lib.thc_dyson_init.argtypes = [ctypes.POINTER(vp), i, i, i, i, d, dp, dp, dp, dp, dp, dp, dp, dp, dp, vp]
    lib.thc_dyson_init.restype = i
    lib.thc_dyson_solve.argtypes = [vp, dp, d, ctypes.POINTER(d), d, dp]
    lib.thc_dyson_solve.restype = i
    lib.thc_dyson_energy.argtypes = [vp, dp, dp, ctypes.POINTER(d), ctypes.POINTER(d), ctypes.POINTER(d)]
    lib.thc_dyson_energy.restype = i
    lib.thc_dyson_evals.argtypes = [vp]
    lib.thc_dyson_evals.restype = i
    lib.thc_dyson_count.argtypes = [vp, dp, d, ctypes.POINTER(d), ctypes.POINTER(d)]
    lib.thc_dyson_count.restype = i
    lib.thc_dyson_commutator.argtypes = [vp, dp, dp]
    lib.thc_dyson_commutator.restype = i
    lib.thc_dyson_last_error.argtypes = [vp]
    lib.thc_dyson_last_error.restype = ctypes.c_char_p
    lib.thc_dyson_destroy.argtypes = [vp]
    lib.thc_dyson_destroy.restype = None
    lib.thc_vec_dot.argtypes = [ctypes.c_longlong, dp, dp, dp, ctypes.POINTER(d), vp]
    lib.thc_vec_dot.restype = i
    lib.thc_vec_lincomb.argtypes = [i, ctypes.POINTER(d), ctypes.POINTER(vp), ctypes.c_longlong, dp, vp]
    lib.thc_vec_lincomb.restype = i
    # learned proposals (include/thc_learned.h)
    fp = ctypes.c_void_p
    lib.thc_mlp_init.argtypes = [ctypes.POINTER(vp), i, i, i, i, fp, fp, fp, fp, vp]
    lib.thc_mlp_init.restype = i
    lib.thc_mlp_forward.argtypes = [vp, i, fp, fp]
    lib.thc_mlp_forward.restype = i
    lib.thc_mlp_gradients.argtypes = [vp, i, fp, fp, ctypes.POINTER(d), fp, fp, fp, fp]
    lib.thc_mlp_gradients.restype = i
    lib.thc_mlp_train.argtypes = [vp, i, fp, fp, i, i, d, ctypes.POINTER(d)]
    lib.thc_mlp_train.restype = i
    lib.thc_mlp_get_weights.argtypes = [vp, fp, fp, fp, fp]
    lib.thc_mlp_get_weights.restype = i
    lib.thc_mlp_destroy.argtypes = [vp]
    lib.thc_mlp_destroy.restype = None
    lib.thc_proposer_init.argtypes = [ctypes.POINTER(vp), i, i, i, dp, dp, i, i, fp, fp, fp, fp, vp]
    lib.thc_proposer_init.restype = i
    lib.thc_proposer_observe.argtypes = [vp, dp]
    lib.thc_proposer_observe.restype = i
    lib.thc_proposer_count.argtypes = [vp]
    lib.thc_proposer_count.restype = i
    lib.thc_proposer_reset.argtypes = [vp]
    lib.thc_proposer_reset.restype = i
    lib.thc_proposer_train.argtypes = [vp, i, i, d, ctypes.POINTER(d)]
    lib.thc_proposer_train.restype = i
    lib.thc_proposer_propose.argtypes = [vp, dp]
    lib.thc_proposer_propose.restype = i
    lib.thc_proposer_state_size.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    lib.thc_proposer_state_size.restype = i
    lib.thc_proposer_save_state.argtypes = [vp, vp, ctypes.c_size_t]
    lib.thc_proposer_save_state.restype = i
    lib.thc_proposer_load_state.argtypes = [vp, vp, ctypes.c_size_t]
    lib.thc_proposer_load_state.restype = i
    lib.thc_proposer_last_error.argtypes = [vp]
    lib.thc_proposer_last_error.restype = ctypes.c_char_p
    lib.thc_proposer_destroy.argtypes = [vp]
    lib.thc_proposer_destroy.restype = None
    # batched evaluation (include/thc_batch.h) and the autotuner
    PP = ctypes.POINTER(ctypes.c_void_p)
    IP = ctypes.POINTER(ctypes.c_int)
    lib.thc_batch_init.argtypes = [ctypes.POINTER(vp), i, IP, IP, i, d, PP, PP, dp, i, i, ctypes.c_ulonglong, i, vp]
    lib.thc_batch_init.restype = i
    lib.thc_batch_eval.argtypes = [vp, PP, PP]
    lib.thc_batch_eval.restype = i
    lib.thc_batch_graph_info.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
    lib.thc_batch_graph_info.restype = i
    lib.thc_batch_flops.argtypes = [vp]
    lib.thc_batch_flops.restype = d
    lib.thc_batch_last_error.argtypes = [vp]
    lib.thc_batch_last_error.restype = ctypes.c_char_p
    lib.thc_batch_destroy.argtypes = [vp]
    lib.thc_batch_destroy.restype = None
    lib.thc_sigma_tune.argtypes = [vp, dp, dp]
    lib.thc_sigma_tune.restype = i
    lib.thc_autotune_save.argtypes = [ctypes.c_char_p]
    lib.thc_autotune_save.restype = i
    lib.thc_autotune_load.argtypes = [ctypes.c_char_p]
    lib.thc_autotune_load.restype = i
    lib.thc_autotune_entries.argtypes = []
    lib.thc_autotune_entries.restype = i
    lib.thc_last_error.argtypes = [vp]
    lib.thc_last_error.restype = ctypes.c_char_p
    if path is None:
        _lib = lib
    return lib


def _ptr(a, dtype="float64"):
    """Raw pointer of a contiguous tensor/array of `dtype`, or NULL for None."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):  # torch.Tensor
        if str(a.dtype) != "torch." + dtype or not a.is_contiguous():
            raise TypeError(f"expected a contiguous {dtype} tensor")
        return ctypes.c_void_p(a.data_ptr())
    if hasattr(a, "ctypes"):  # numpy.ndarray
        if a.dtype.name != dtype or not a.flags["C_CONTIGUOUS"]:
            raise TypeError(f"expected a C-contiguous {dtype} array")
        return ctypes.c_void_p(a.ctypes.data)
    if isinstance(a, int):
        return ctypes.c_void_p(a)
    raise TypeError(f"cannot pass {type(a)} as a pointer")


def _check(rc: int, ctx=None):
    if rc != THC_OK:
        raise ThcError(rc, thc_last_error(ctx))


def thc_last_error(ctx=None) -> str:
    return load_library().thc_last_error(ctx).decode()


def thc_sigma_init(n_ao, n_thc, n_tau, beta, X, V, tau, precision=THC_FP64,
                   terms=THC_DIRECT | THC_SOX, stream=None):
    """Returns the opaque context handle (ctypes.c_void_p)."""
    lib = load_library()
    ctx = ctypes.c_void_p()
    s = None if stream is None else ctypes.c_void_p(int(stream))
    rc = lib.thc_sigma_init(ctypes.byref(ctx), int(n_ao), int(n_thc), int(n_tau), float(beta),
                            _ptr(X), _ptr(V), _ptr(tau), int(precision), int(terms), s)
    _check(rc, None)
    return ctx


def thc_sigma_eval(ctx, G_tau, G_bmt, Sigma_tau):
    _check(load_library().thc_sigma_eval(ctx, _ptr(G_tau), _ptr(G_bmt), _ptr(Sigma_tau)), ctx)


def thc_sigma_set_bosonic(ctx, to_iw, to_tau):
    """Bosonic transforms (n_omega x n_tau and n_tau x n_omega, host float64) for THC_GW."""
    import numpy as np
    a = np.ascontiguousarray(to_iw, dtype=np.float64)
    b = np.ascontiguousarray(to_tau, dtype=np.float64)
    _check(load_library().thc_sigma_set_bosonic(ctx, int(a.shape[0]), _ptr(a), _ptr(b)), ctx)


def thc_sigma_eval_uhf(ctx, G_tau_a, G_bmt_a, G_tau_b, G_bmt_b, Sigma_a, Sigma_b):
    _check(load_library().thc_sigma_eval_uhf(ctx, _ptr(G_tau_a), _ptr(G_bmt_a), _ptr(G_tau_b), _ptr(G_bmt_b),
                                             _ptr(Sigma_a), _ptr(Sigma_b)), ctx)


def thc_sigma_eval_host(ctx, G_tau, G_bmt, Sigma_tau):
    _check(load_library().thc_sigma_eval_host(ctx, _ptr(G_tau), _ptr(G_bmt), _ptr(Sigma_tau)), ctx)


def thc_energy(ctx, G_tau, G_bmt, Sigma_tau, tau_weights) -> float:
    e = ctypes.c_double()
    _check(load_library().thc_energy(ctx, _ptr(G_tau), _ptr(G_bmt), _ptr(Sigma_tau), _ptr(tau_weights),
                                     ctypes.byref(e)), ctx)
    return e.value


def thc_set_stream(ctx, stream):
    _check(load_library().thc_set_stream(ctx, None if stream is None else ctypes.c_void_p(int(stream))), ctx)


def thc_sigma_flops(ctx) -> tuple[float, float]:
    u = ctypes.c_double()
    f = load_library().thc_sigma_flops(ctx, ctypes.byref(u))
    return f, u.value


def thc_profile(ctx, enable: bool):
    _check(load_library().thc_profile(ctx, int(bool(enable))), ctx)


def thc_profile_get(ctx, kclass: int):
    """(name, launches, ms, flops) of kernel class kclass, or None past the last class."""
    name = ctypes.c_char_p()
    launches = ctypes.c_longlong()
    ms = ctypes.c_double()
    fl = ctypes.c_double()
    rc = load_library().thc_profile_get(ctx, int(kclass), ctypes.byref(name), ctypes.byref(launches),
                                        ctypes.byref(ms), ctypes.byref(fl))
    if rc == THC_EINVAL and kclass >= 0:
        return None
    _check(rc, ctx)
    return name.value.decode(), launches.value, ms.value, fl.value


def thc_launch_count(ctx) -> int:
    return int(load_library().thc_launch_count(ctx))


def thc_energy_static(n_ao, n_tau, G_tau, G_bmt, Sigma_tau, tau_weights, stream=None) -> float:
    """E_dyn without a context or any device allocation (fixed static scratch)."""
    e = ctypes.c_double()
    s = None if stream is None else ctypes.c_void_p(int(stream))
    _check(load_library().thc_energy_static(int(n_ao), int(n_tau), _ptr(G_tau), _ptr(G_bmt), _ptr(Sigma_tau),
                                            _ptr(tau_weights), ctypes.byref(e), s), None)
    return e.value


def thc_sync(ctx):
    _check(load_library().thc_sync(ctx), ctx)


def thc_fp64_dfma_rate(iters=50_000, stream=None):
    """(TFLOP/s, ms) of the FP64 FMA micro-benchmark on the current device."""
    t, ms = ctypes.c_double(), ctypes.c_double()
    s = None if stream is None else ctypes.c_void_p(int(stream))
    _check(load_library().thc_fp64_dfma_rate(int(iters), ctypes.byref(t), ctypes.byref(ms), s), None)
    return t.value, ms.value


def thc_wait_selftest(limit_ns, stream=None):
    """Runs the bounded-wait failure path once; raises ThcError (THC_ETIMEOUT expected)."""
    s = None if stream is None else ctypes.c_void_p(int(stream))
    _check(load_library().thc_wait_selftest(int(limit_ns), s), None)


def thc_gemm_bf16x3(batch, M, N, K, A, strideA, B, strideB, C, strideC, stream=None):
    s = None if stream is None else ctypes.c_void_p(int(stream))
    _check(load_library().thc_gemm_bf16x3(int(batch), int(M), int(N), int(K), _ptr(A), int(strideA), _ptr(B),
                                          int(strideB), _ptr(C), int(strideC), s), None)


def thc_destroy(ctx):
    load_library().thc_destroy(ctx)


# ---------------------------------------------------------------- loop ABI
def _interleaved(z):
    """complex128 array -> contiguous float64 (re, im) interleaving, as the ABI expects."""
    import numpy as np
    return np.ascontiguousarray(np.asarray(z, dtype=np.complex128)).view(np.float64)


def _stream(stream):
    return None if stream is None else ctypes.c_void_p(int(stream))


def _dcheck(rc, d):
    if rc != THC_OK:
        msg = load_library().thc_dyson_last_error(d).decode() if d else thc_last_error(None)
        raise ThcError(rc, msg)


def thc_dyson_init(n_ao, n_tau, n_iw, n_l, beta, S, F, U_tau, fit_tau, U_iw, fit_iw, iw, u_beta, u_zero,
                   stream=None):
    import numpy as np
    d = ctypes.c_void_p()
    keep = [np.ascontiguousarray(x, dtype=np.float64) for x in (U_tau, fit_tau, iw, u_beta, u_zero)]
    ziw, zfit = _interleaved(U_iw), _interleaved(fit_iw)
    rc = load_library().thc_dyson_init(ctypes.byref(d), int(n_ao), int(n_tau), int(n_iw), int(n_l), float(beta),
                                       _ptr(S), _ptr(F), _ptr(keep[0]), _ptr(keep[1]), _ptr(ziw), _ptr(zfit),
                                       _ptr(keep[2]), _ptr(keep[3]), _ptr(keep[4]), _stream(stream))
    _dcheck(rc, None)
    return d


def thc_dyson_solve(d, Sigma_tau, n_elec, mu, tol, G_tau) -> float:
    m = ctypes.c_double(mu)
    _dcheck(load_library().thc_dyson_solve(d, _ptr(Sigma_tau), float(n_elec), ctypes.byref(m), float(tol),
                                           _ptr(G_tau)), d)
    return m.value


def thc_dyson_energy(d, G_tau, Sigma_tau):
    """(E_dyn, Tr[gamma F], Tr[gamma S])."""
    e, f, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _dcheck(load_library().thc_dyson_energy(d, _ptr(G_tau), _ptr(Sigma_tau), ctypes.byref(e), ctypes.byref(f),
                                            ctypes.byref(n)), d)
    return e.value, f.value, n.value


def thc_dyson_count(d, Sigma_tau, mu):
    """(N(mu), dN/dmu) per spin at fixed Sigma."""
    n, dn = ctypes.c_double(), ctypes.c_double()
    _dcheck(load_library().thc_dyson_count(d, _ptr(Sigma_tau), float(mu), ctypes.byref(n), ctypes.byref(dn)), d)
    return n.value, dn.value


def thc_dyson_commutator(d, Sigma_out_tau, E_iw):
    """E_iw (dev, n_iw x n x n x 2 float64) <- H G S - S G H with H = F + Sigma_out(i w)."""
    _dcheck(load_library().thc_dyson_commutator(d, _ptr(Sigma_out_tau), _ptr(E_iw)), d)


def thc_dyson_evals(d) -> int:
    return int(load_library().thc_dyson_evals(d))


def thc_dyson_destroy(d):
    load_library().thc_dyson_destroy(d)


def thc_vec_dot(length, x, y, scratch, stream=None) -> float:
    out = ctypes.c_double()
    _check(load_library().thc_vec_dot(int(length), _ptr(x), _ptr(y), _ptr(scratch), ctypes.byref(out),
                                      _stream(stream)), None)
    return out.value


def thc_vec_lincomb(coeffs, vecs, length, out, stream=None):
    k = len(coeffs)
    c = (ctypes.c_double * k)(*[float(x) for x in coeffs])
    ptrs = (ctypes.c_void_p * k)(*[_ptr(v).value for v in vecs])
    _check(load_library().thc_vec_lincomb(k, c, ptrs, int(length), _ptr(out), _stream(stream)), None)


# ------------------------------------------------------ learned proposals ABI
def _f32(a):
    return _ptr(a, "float32")


def _lcheck(rc, fn, h):
    if rc != THC_OK:
        msg = fn(h).decode() if h else thc_last_error(None)
        raise ThcError(rc, msg or thc_last_error(None))


def thc_mlp_init(d_in, hidden, d_out, max_batch, W1, b1, W2, b2, stream=None):
    m = ctypes.c_void_p()
    rc = load_library().thc_mlp_init(ctypes.byref(m), int(d_in), int(hidden), int(d_out), int(max_batch), _f32(W1),
                                     _f32(b1), _f32(W2), _f32(b2), _stream(stream))
    _check(rc, None)
    return m


def thc_mlp_forward(m, batch, X, Y):
    _check(load_library().thc_mlp_forward(m, int(batch), _f32(X), _f32(Y)), None)


def thc_mlp_gradients(m, batch, X, T, gW1=None, gb1=None, gW2=None, gb2=None) -> float:
    loss = ctypes.c_double()
    _check(load_library().thc_mlp_gradients(m, int(batch), _f32(X), _f32(T), ctypes.byref(loss), _f32(gW1), _f32(gb1),
                                            _f32(gW2), _f32(gb2)), None)
    return loss.value


def thc_mlp_train(m, n_samples, X, T, steps, batch, lr) -> float:
    loss = ctypes.c_double()
    _check(load_library().thc_mlp_train(m, int(n_samples), _f32(X), _f32(T), int(steps), int(batch), float(lr),
                                        ctypes.byref(loss)), None)
    return loss.value


def thc_mlp_get_weights(m, W1=None, b1=None, W2=None, b2=None):
    _check(load_library().thc_mlp_get_weights(m, _f32(W1), _f32(b1), _f32(W2), _f32(b2)), None)


def thc_mlp_destroy(m):
    load_library().thc_mlp_destroy(m)


def thc_proposer_init(n_ao, n_tau, n_l, U_tau, fit_tau, hidden, max_hist, W1, b1, W2, b2, stream=None):
    import numpy as np
    p = ctypes.c_void_p()
    Ut, Ft = np.ascontiguousarray(U_tau, dtype=np.float64), np.ascontiguousarray(fit_tau, dtype=np.float64)
    lib = load_library()
    rc = lib.thc_proposer_init(ctypes.byref(p), int(n_ao), int(n_tau), int(n_l), _ptr(Ut), _ptr(Ft), int(hidden),
                               int(max_hist), _f32(W1), _f32(b1), _f32(W2), _f32(b2), _stream(stream))
    _lcheck(rc, lib.thc_proposer_last_error, None)
    return p


def thc_proposer_observe(p, Sigma_tau):
    lib = load_library()
    _lcheck(lib.thc_proposer_observe(p, _ptr(Sigma_tau)), lib.thc_proposer_last_error, p)


def thc_proposer_count(p) -> int:
    return int(load_library().thc_proposer_count(p))


def thc_proposer_reset(p):
    lib = load_library()
    _lcheck(lib.thc_proposer_reset(p), lib.thc_proposer_last_error, p)


def thc_proposer_train(p, steps, batch, lr) -> float:
    lib = load_library()
    loss = ctypes.c_double()
    _lcheck(lib.thc_proposer_train(p, int(steps), int(batch), float(lr), ctypes.byref(loss)),
            lib.thc_proposer_last_error, p)
    return loss.value


def thc_proposer_propose(p, Sigma_tau):
    lib = load_library()
    _lcheck(lib.thc_proposer_propose(p, _ptr(Sigma_tau)), lib.thc_proposer_last_error, p)


def thc_proposer_save_state(p):
    """The proposer's resumable state as a host uint8 array."""
    import numpy as np
    lib = load_library()
    size = ctypes.c_size_t()
    _lcheck(lib.thc_proposer_state_size(p, ctypes.byref(size)), lib.thc_proposer_last_error, p)
    buf = np.empty(size.value, dtype=np.uint8)
    _lcheck(lib.thc_proposer_save_state(p, buf.ctypes.data_as(ctypes.c_void_p), buf.nbytes),
            lib.thc_proposer_last_error, p)
    return buf


def thc_proposer_load_state(p, buf):
    import numpy as np
    lib = load_library()
    b = np.ascontiguousarray(buf, dtype=np.uint8)
    _lcheck(lib.thc_proposer_load_state(p, b.ctypes.data_as(ctypes.c_void_p), b.nbytes),
            lib.thc_proposer_last_error, p)


def thc_proposer_destroy(p):
    load_library().thc_proposer_destroy(p)


# --------------------------------------------------------- batched ABI
def _ptr_array(xs):
    return (ctypes.c_void_p * len(xs))(*[_ptr(x).value for x in xs])


def thc_batch_init(n_ao, n_thc, n_tau, beta, X, V, tau, precision=THC_BF16X3, n_streams=4, budget_per_molecule=0,
                   tune=True, stream=None):
    import numpy as np
    b = ctypes.c_void_p()
    k = len(n_ao)
    na = (ctypes.c_int * k)(*[int(x) for x in n_ao])
    nt = (ctypes.c_int * k)(*[int(x) for x in n_thc])
    t = np.ascontiguousarray(tau, dtype=np.float64)
    lib = load_library()
    rc = lib.thc_batch_init(ctypes.byref(b), k, na, nt, int(n_tau), float(beta), _ptr_array(X), _ptr_array(V),
                            _ptr(t), int(precision), int(n_streams), int(budget_per_molecule), int(bool(tune)),
                            _stream(stream))
    _lcheck(rc, lib.thc_batch_last_error, None)
    return b


def thc_batch_eval(b, G_tau, Sigma_tau):
    lib = load_library()
    _lcheck(lib.thc_batch_eval(b, _ptr_array(G_tau), _ptr_array(Sigma_tau)), lib.thc_batch_last_error, b)


def thc_batch_graph_info(b):
    k, n = ctypes.c_longlong(), ctypes.c_longlong()
    _check(load_library().thc_batch_graph_info(b, ctypes.byref(k), ctypes.byref(n)), None)
    return k.value, n.value


def thc_batch_flops(b) -> float:
    return float(load_library().thc_batch_flops(b))


def thc_batch_destroy(b):
    load_library().thc_batch_destroy(b)


def thc_sigma_tune(ctx, G_tau, G_bmt=None):
    _check(load_library().thc_sigma_tune(ctx, _ptr(G_tau), _ptr(G_bmt)), ctx)


def thc_autotune_save(path):
    _check(load_library().thc_autotune_save(str(path).encode()), None)


def thc_autotune_load(path):
    _check(load_library().thc_autotune_load(str(path).encode()), None)


def thc_autotune_entries() -> int:
    return int(load_library().thc_autotune_entries())
