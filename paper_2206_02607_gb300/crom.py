"""Thin ctypes binding of the C ABI in include/crom.h.

Every function here only marshals arguments (torch CUDA tensors -> device
pointers, the current torch stream -> cudaStream_t) and raises on a non-zero
status.  All arithmetic of the latent step runs in libcrom.so's CUDA kernels;
there is no fallback: importing this module fails when the library is missing.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libcrom.so")

CROM_OK = 0
CROM_ERR_INVALID_ARG = 1
CROM_ERR_CUDA = 2
CROM_ERR_SINGULAR = 3
CROM_ERR_NONFINITE = 4
CROM_ERR_TIMEOUT = 5
CROM_ERR_UNSUPPORTED = 6

CROM_PREC_FP32 = 0
CROM_PREC_F16X2 = 1
CROM_PREC_F16 = 2
CROM_PREC_BF16_MIXED = 4
CROM_PREC_BF16X2 = CROM_PREC_F16X2   # earlier names of the same values
CROM_PREC_BF16 = CROM_PREC_F16

CROM_PDE_HEAT = 0
CROM_PDE_ADVDIFF = 1

CROM_WANT_VAL = 1
CROM_WANT_DX = 2
CROM_WANT_DXX = 4
CROM_WANT_LAP = 8
CROM_WANT_DQ = 16

# Every symbol include/crom.h declares.
CROM_FOM_HEAT1D_DIRICHLET = 0
CROM_FOM_HEAT2D_NEUMANN = 1
CROM_FOM_ADVDIFF2D_PERIODIC = 2
CROM_ACT_ELU = 0
CROM_ACT_SIREN = 1
CROM_FOM_HEAT1D_DIRICHLET_FIELD = 3
CROM_FOM_HEAT2D_NEUMANN_FIELD = 4
CROM_FOM_ADVDIFF2D_PERIODIC_CENTRAL = 5

EXPORTED = ("crom_version", "crom_last_error", "crom_create", "crom_destroy", "crom_set_weights",
            "crom_decode", "crom_step", "crom_step_host", "crom_rollout", "crom_step_noalloc", "crom_fom_step",
            "crom_trainer_create",
            "crom_trainer_destroy", "crom_trainer_param_count", "crom_trainer_set_params",
            "crom_trainer_get_params", "crom_trainer_get_grads", "crom_train_step", "crom_encode",
            "crom_reconstruct", "crom_robust_samples", "crom_tangent_velocity", "crom_trainer_set_precision",
            "crom_set_step_tiles", "crom_get_step_tiles", "crom_autotune", "crom_decode_tc", "crom_device_flags",
            "crom_trainer_save", "crom_trainer_load", "crom_crc32", "crom_stream_wait")


class CromError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"crom status {code}: {msg}")
        self.code = code


class crom_decoder_desc(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("r", ctypes.c_int), ("width", ctypes.c_int), ("hidden", ctypes.c_int),
                ("activation", ctypes.c_int), ("omega0", ctypes.c_float)]


class crom_step_desc(ctypes.Structure):
    _fields_ = [("pde", ctypes.c_int), ("gn_iters", ctypes.c_int), ("dt", ctypes.c_double),
                ("coef_per_sample", ctypes.c_int), ("line_search", ctypes.c_int)]


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with __graft_entry__.build() "
                          "(nvcc for sm_103a); there is no CPU fallback")
    lib = ctypes.CDLL(path)
    vp, i, u, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint, ctypes.c_double, ctypes.c_size_t
    lib.crom_version.restype = i
    lib.crom_last_error.restype = ctypes.c_char_p
    lib.crom_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(crom_decoder_desc), i]
    lib.crom_destroy.argtypes = [vp]
    lib.crom_set_weights.argtypes = [vp, vp, sz, i, vp]
    lib.crom_decode.argtypes = [vp, i, vp, vp, vp, i, u, vp, vp]
    lib.crom_decode_tc.argtypes = [vp, i, i, vp, vp, vp, i, u, vp, vp]
    lib.crom_device_flags.argtypes = [vp, ctypes.POINTER(i), vp]
    lib.crom_trainer_save.argtypes = [vp, ctypes.c_char_p]
    lib.crom_trainer_load.argtypes = [vp, ctypes.c_char_p]
    lib.crom_crc32.argtypes = [vp, ctypes.c_size_t]
    lib.crom_crc32.restype = ctypes.c_uint
    lib.crom_stream_wait.argtypes = [vp, d]
    lib.crom_step.argtypes = [vp, ctypes.POINTER(crom_step_desc), i, i, vp, vp, vp, vp, vp, i, i, vp, vp]
    lib.crom_step_noalloc.argtypes = [vp, ctypes.POINTER(crom_step_desc), i, vp, vp, vp, vp, vp, i, i, vp, vp]
    lib.crom_step_host.argtypes = [vp, ctypes.POINTER(crom_step_desc), i, i, vp, vp, vp, vp, vp, i, i, vp, vp]
    lib.crom_rollout.argtypes = [vp, ctypes.POINTER(crom_step_desc), i, i, i, vp, vp, vp, vp, vp, i, i, vp, vp]
    lib.crom_fom_step.argtypes = [i, i, i, i, vp, vp, vp, d, i, vp, vp, vp]
    lib.crom_trainer_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(crom_decoder_desc), i, i, i, i]
    lib.crom_trainer_destroy.argtypes = [vp]
    lib.crom_trainer_param_count.argtypes = [vp, ctypes.POINTER(sz)]
    lib.crom_trainer_set_precision.argtypes = [vp, i]
    for name in ("crom_trainer_set_params", "crom_trainer_get_params", "crom_trainer_get_grads"):
        getattr(lib, name).argtypes = [vp, vp, sz, i, vp]
    lib.crom_train_step.argtypes = [vp, vp, vp, vp, ctypes.c_float, vp, vp]
    lib.crom_encode.argtypes = [vp, i, vp, vp, vp]
    lib.crom_reconstruct.argtypes = [vp, i, i, vp, i, vp, vp, vp]
    lib.crom_tangent_velocity.argtypes = [vp, i, vp, vp, d, vp, vp, i, vp, vp]
    lib.crom_set_step_tiles.argtypes = [vp, i, i]
    lib.crom_get_step_tiles.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(ctypes.c_float)]
    lib.crom_autotune.argtypes = [vp, ctypes.POINTER(crom_step_desc), i, vp, vp, vp, vp, vp, i, i, vp, vp]
    lib.crom_robust_samples.argtypes = [vp, ctypes.POINTER(crom_step_desc), i, i, vp, vp, i, i, vp, vp, i, vp, i,
                                        d, i, vp, vp, vp, vp]
    for name in EXPORTED:
        if name not in ("crom_version", "crom_last_error", "crom_crc32"):
            getattr(lib, name).restype = i
    return lib


_LIB = load_library()


def lib() -> ctypes.CDLL:
    return _LIB


def _check(code: int):
    if code != CROM_OK:
        raise CromError(code, _LIB.crom_last_error().decode())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _need(t, dtype, name):
    import torch
    if t is None:
        return
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor of {dtype}")


def crom_version() -> int:
    return _LIB.crom_version()


class CromContext:
    """Owns a crom_ctx (decoder shape + weights on one device)."""

    def __init__(self, m: int, r: int, width: int, hidden: int, device: int = 0, activation: int = 0,
                 omega0: float = 30.0):
        self.desc = crom_decoder_desc(m, r, width, hidden, activation, omega0 if activation else 0.0)
        self.handle = ctypes.c_void_p()
        _check(_LIB.crom_create(ctypes.byref(self.handle), ctypes.byref(self.desc), device))
        self.device = device

    def close(self):
        if self.handle:
            _LIB.crom_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def crom_create(m, r, width, hidden, device=0, activation=0, omega0=30.0) -> CromContext:
    return CromContext(m, r, width, hidden, device, activation, omega0)


def crom_destroy(ctx: CromContext):
    ctx.close()


def crom_set_weights(ctx: CromContext, params, stream=None):
    """params: packed float32 image (numpy array on the host, or a CUDA tensor)."""
    import numpy as np
    if hasattr(params, "is_cuda") and params.is_cuda:
        _need(params, params.dtype, "params")
        _check(_LIB.crom_set_weights(ctx.handle, _ptr(params), params.numel(), 1, _stream(stream)))
    else:
        a = np.ascontiguousarray(params, dtype=np.float32)
        _check(_LIB.crom_set_weights(ctx.handle, a.ctypes.data_as(ctypes.c_void_p), a.size, 0,
                                     _stream(stream)))


def crom_decode(ctx: CromContext, q, pt_off, x, want: int, out, stream=None):
    import torch
    _need(q, torch.float64, "q"); _need(pt_off, torch.int32, "pt_off")
    _need(x, torch.float32, "x"); _need(out, torch.float32, "out")
    _check(_LIB.crom_decode(ctx.handle, q.shape[0], _ptr(q), _ptr(pt_off), _ptr(x), x.shape[0], want,
                            _ptr(out), _stream(stream)))


def crom_decode_tc(ctx: CromContext, q, pt_off, x, want: int, out, precision: int = CROM_PREC_F16X2, stream=None):
    """Step 1 on the tensor cores (want: VAL, DX, LAP, DQ; no DXX)."""
    import torch
    _need(q, torch.float64, "q"); _need(pt_off, torch.int32, "pt_off")
    _need(x, torch.float32, "x"); _need(out, torch.float32, "out")
    _check(_LIB.crom_decode_tc(ctx.handle, precision, q.shape[0], _ptr(q), _ptr(pt_off), _ptr(x), x.shape[0], want,
                               _ptr(out), _stream(stream)))


def crom_trainer_save(tr, path: str):
    _check(_LIB.crom_trainer_save(tr.handle, str(path).encode()))


def crom_trainer_load(tr, path: str):
    _check(_LIB.crom_trainer_load(tr.handle, str(path).encode()))


def crom_crc32(data: bytes) -> int:
    buf = ctypes.create_string_buffer(bytes(data), len(data))
    return int(_LIB.crom_crc32(buf, len(data)))


def crom_stream_wait(timeout_ms: float, stream=None):
    """Raises CromError(CROM_ERR_TIMEOUT) if the stream's work is not done in time."""
    _check(_LIB.crom_stream_wait(_stream(stream), float(timeout_ms)))


def crom_device_flags(ctx: CromContext, stream=None) -> int:
    """Bit 0: the last tensor-core step / decode launch gave up on a bounded wait;
    bit 1: a tensor-core reconstruction did since the last call."""
    f = ctypes.c_int(0)
    _check(_LIB.crom_device_flags(ctx.handle, ctypes.byref(f), _stream(stream)))
    return f.value


def crom_step(ctx: CromContext, q, alpha, s_off, samples, status, *, dt: float, gn_iters: int,
              max_samples: int, pde: int = CROM_PDE_HEAT, vel=None, precision: int = CROM_PREC_FP32,
              coef_per_sample: bool = False, line_search: int = 0, stream=None):
    import torch
    _need(q, torch.float64, "q"); _need(alpha, torch.float32, "alpha"); _need(s_off, torch.int32, "s_off")
    _need(samples, torch.float32, "samples"); _need(status, torch.int32, "status"); _need(vel, torch.float32, "vel")
    desc = crom_step_desc(pde, gn_iters, dt, int(bool(coef_per_sample)), int(line_search))
    _check(_LIB.crom_step(ctx.handle, ctypes.byref(desc), precision, q.shape[0], _ptr(q), _ptr(alpha),
                          _ptr(vel), _ptr(s_off), _ptr(samples), samples.shape[0], max_samples, _ptr(status),
                          _stream(stream)))


def _need_host(t, dtype, name):
    import torch
    if t is None:
        return
    if t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous host (CPU) tensor of {dtype}")


def crom_step_host(ctx: CromContext, q, alpha, s_off, samples, status, *, dt: float, gn_iters: int,
                   max_samples: int, pde: int = CROM_PDE_HEAT, vel=None, precision: int = CROM_PREC_FP32,
                   coef_per_sample: bool = False, line_search: int = 0, stream=None):
    """crom_step on host (CPU, preferably pinned) tensors; q and status are updated in
    place when the call returns (the library stages the copies and synchronises)."""
    import torch
    _need_host(q, torch.float64, "q"); _need_host(alpha, torch.float32, "alpha")
    _need_host(s_off, torch.int32, "s_off"); _need_host(samples, torch.float32, "samples")
    _need_host(status, torch.int32, "status"); _need_host(vel, torch.float32, "vel")
    desc = crom_step_desc(pde, gn_iters, dt, int(bool(coef_per_sample)), int(line_search))
    _check(_LIB.crom_step_host(ctx.handle, ctypes.byref(desc), precision, q.shape[0], _ptr(q), _ptr(alpha),
                               _ptr(vel), _ptr(s_off), _ptr(samples), samples.shape[0], max_samples, _ptr(status),
                               _stream(stream)))


def crom_rollout(ctx: CromContext, q, alpha, s_off, samples, status, *, n_steps: int, dt: float, gn_iters: int,
                 max_samples: int, pde: int = CROM_PDE_HEAT, vel=None, precision: int = CROM_PREC_FP32,
                 coef_per_sample: bool = False, line_search: int = 0, stream=None):
    """n_steps latent steps replayed from a CUDA graph cached in the context."""
    import torch
    _need(q, torch.float64, "q"); _need(alpha, torch.float32, "alpha"); _need(s_off, torch.int32, "s_off")
    _need(samples, torch.float32, "samples"); _need(status, torch.int32, "status"); _need(vel, torch.float32, "vel")
    desc = crom_step_desc(pde, gn_iters, dt, int(bool(coef_per_sample)), int(line_search))
    _check(_LIB.crom_rollout(ctx.handle, ctypes.byref(desc), precision, n_steps, q.shape[0], _ptr(q), _ptr(alpha),
                             _ptr(vel), _ptr(s_off), _ptr(samples), samples.shape[0], max_samples, _ptr(status),
                             _stream(stream)))


def crom_step_noalloc(ctx: CromContext, q, alpha, s_off, samples, status, *, dt: float, gn_iters: int,
                      max_samples: int, pde: int = CROM_PDE_HEAT, vel=None, coef_per_sample: bool = False,
                      stream=None):
    """The FP32 step with its scratch in the library's fixed device array: for
    callers that must not allocate device memory while stepping (see crom.h)."""
    import torch
    _need(q, torch.float64, "q"); _need(alpha, torch.float32, "alpha"); _need(s_off, torch.int32, "s_off")
    _need(samples, torch.float32, "samples"); _need(status, torch.int32, "status"); _need(vel, torch.float32, "vel")
    desc = crom_step_desc(pde, gn_iters, dt, int(bool(coef_per_sample)), 0)
    _check(_LIB.crom_step_noalloc(ctx.handle, ctypes.byref(desc), q.shape[0], _ptr(q), _ptr(alpha), _ptr(vel),
                                  _ptr(s_off), _ptr(samples), samples.shape[0], max_samples, _ptr(status),
                                  _stream(stream)))


def crom_fom_step(kind: int, u, tmp, coef, *, dt: float, n_steps: int, ax=None, ay=None, stream=None):
    """u: [n_batch, nx] (1D) or [n_batch, nx, nx] (2D) float32 CUDA tensor, advanced in place."""
    import torch
    for t, name in ((u, "u"), (tmp, "tmp"), (coef, "coef"), (ax, "ax"), (ay, "ay")):
        _need(t, torch.float32, name)
    nb, nx = u.shape[0], u.shape[1]
    ny = 1 if u.dim() == 2 else u.shape[2]
    _check(_LIB.crom_fom_step(kind, nb, nx, ny, _ptr(coef), _ptr(ax), _ptr(ay), dt, n_steps, _ptr(u), _ptr(tmp),
                              _stream(stream)))


class CromTrainer:
    """Owns a crom_trainer (encoder + decoder parameters, Adam state, activations)."""

    def __init__(self, m, r, width, hidden, P, B, S, device=0):
        self.desc = crom_decoder_desc(m, r, width, hidden)
        self.handle = ctypes.c_void_p()
        _check(_LIB.crom_trainer_create(ctypes.byref(self.handle), ctypes.byref(self.desc), P, B, S, device))
        n = ctypes.c_size_t()
        _check(_LIB.crom_trainer_param_count(self.handle, ctypes.byref(n)))
        self.n_params = n.value
        self.B, self.S, self.P = B, S, P

    def _io(self, fn, arr, stream):
        import numpy as np
        if hasattr(arr, "is_cuda") and arr.is_cuda:
            _check(fn(self.handle, _ptr(arr), arr.numel(), 1, _stream(stream)))
        else:
            _check(fn(self.handle, arr.ctypes.data_as(ctypes.c_void_p), arr.size, 0, _stream(stream)))

    def set_precision(self, precision: int):
        """CROM_PREC_FP32 (default) or CROM_PREC_BF16_MIXED for the decoder pass."""
        _check(_LIB.crom_trainer_set_precision(self.handle, precision))

    def set_params(self, params, stream=None):
        import numpy as np
        if not (hasattr(params, "is_cuda") and params.is_cuda):
            params = np.ascontiguousarray(params, dtype=np.float32)
        self._io(_LIB.crom_trainer_set_params, params, stream)

    def get_params(self, stream=None):
        import numpy as np
        out = np.empty(self.n_params, np.float32)
        self._io(_LIB.crom_trainer_get_params, out, stream)
        return out

    def get_grads(self, stream=None):
        import numpy as np
        out = np.empty(self.n_params, np.float32)
        self._io(_LIB.crom_trainer_get_grads, out, stream)
        return out

    def close(self):
        if self.handle:
            _LIB.crom_trainer_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def crom_train_step(tr: CromTrainer, snaps, pt_idx, coords, lr: float, loss_out=None, stream=None):
    import torch
    _need(snaps, torch.float32, "snaps"); _need(pt_idx, torch.int32, "pt_idx"); _need(coords, torch.float32, "coords")
    _need(loss_out, torch.float64, "loss_out")
    _check(_LIB.crom_train_step(tr.handle, _ptr(snaps), _ptr(pt_idx), _ptr(coords), lr, _ptr(loss_out),
                                _stream(stream)))


def crom_encode(tr: CromTrainer, snaps, q_out, stream=None):
    import torch
    _need(snaps, torch.float32, "snaps"); _need(q_out, torch.float32, "q_out")
    _check(_LIB.crom_encode(tr.handle, snaps.shape[0], _ptr(snaps), _ptr(q_out), _stream(stream)))


def crom_reconstruct(ctx: CromContext, q, x, out, precision: int = CROM_PREC_FP32, stream=None):
    import torch
    _need(q, torch.float64, "q"); _need(x, torch.float32, "x"); _need(out, torch.float32, "out")
    _check(_LIB.crom_reconstruct(ctx.handle, precision, q.shape[0], _ptr(q), x.shape[0], _ptr(x), _ptr(out),
                                 _stream(stream)))


def crom_set_step_tiles(ctx: CromContext, s0: int, s1: int):
    _check(_LIB.crom_set_step_tiles(ctx.handle, s0, s1))


def crom_get_step_tiles(ctx: CromContext):
    """(s0, s1, [ms for the large s1, ms for the small s1]) of the context's tensor-core step."""
    a, b = ctypes.c_int(), ctypes.c_int()
    ms = (ctypes.c_float * 2)()
    _check(_LIB.crom_get_step_tiles(ctx.handle, ctypes.byref(a), ctypes.byref(b), ms))
    return a.value, b.value, [ms[0], ms[1]]


def crom_autotune(ctx: CromContext, q, alpha, s_off, samples, status, *, dt: float, gn_iters: int,
                  max_samples: int, pde: int = CROM_PDE_HEAT, vel=None, coef_per_sample: bool = False,
                  line_search: int = 0, stream=None):
    """Measure the tensor-core step's tile shapes on this batch and keep the fastest."""
    import torch
    _need(q, torch.float64, "q"); _need(alpha, torch.float32, "alpha"); _need(s_off, torch.int32, "s_off")
    _need(samples, torch.float32, "samples"); _need(status, torch.int32, "status"); _need(vel, torch.float32, "vel")
    desc = crom_step_desc(pde, gn_iters, dt, int(bool(coef_per_sample)), int(line_search))
    _check(_LIB.crom_autotune(ctx.handle, ctypes.byref(desc), q.shape[0], _ptr(q), _ptr(alpha), _ptr(vel),
                              _ptr(s_off), _ptr(samples), samples.shape[0], max_samples, _ptr(status),
                              _stream(stream)))
    return crom_get_step_tiles(ctx)


def crom_tangent_velocity(ctx: CromContext, q, q_prev, pt_off, x, out, *, dt: float, stream=None):
    """v(x_p) = dg/dq(x_p, q_i) . (q_i - q_prev_i) / dt (see crom.h)."""
    import torch
    _need(q, torch.float64, "q"); _need(q_prev, torch.float64, "q_prev"); _need(pt_off, torch.int32, "pt_off")
    _need(x, torch.float32, "x"); _need(out, torch.float32, "out")
    _check(_LIB.crom_tangent_velocity(ctx.handle, q.shape[0], _ptr(q), _ptr(q_prev), dt, _ptr(pt_off), _ptr(x),
                                      x.shape[0], _ptr(out), _stream(stream)))


def crom_robust_samples(ctx: CromContext, q0, coef, nodes, fom_final, init_idx, *, dt: float, gn_iters: int,
                        n_steps: int, n_try: int, target: float, max_samples: int,
                        precision: int = CROM_PREC_FP32, coef_per_sample: bool = False, line_search: int = 0,
                        stream=None):
    """Greedy robust sample selection (see crom.h).  q0 [n_params, r] float64,
    coef [n_params] or [n_params, n_nodes] float32, nodes [n_nodes, m] float32,
    fom_final [n_params, n_nodes] float32 (CUDA tensors); init_idx: host ints.
    Returns (indices, metric)."""
    import torch
    _need(q0, torch.float64, "q0"); _need(coef, torch.float32, "coef"); _need(nodes, torch.float32, "nodes")
    _need(fom_final, torch.float32, "fom_final")
    init = (ctypes.c_int * max(len(init_idx), 1))(*[int(i) for i in init_idx])
    out = (ctypes.c_int * max_samples)()
    count = ctypes.c_int()
    met = ctypes.c_double()
    desc = crom_step_desc(CROM_PDE_HEAT, gn_iters, dt, int(bool(coef_per_sample)), int(line_search))
    _check(_LIB.crom_robust_samples(ctx.handle, ctypes.byref(desc), precision, q0.shape[0], _ptr(q0), _ptr(coef),
                                    n_steps, nodes.shape[0], _ptr(nodes), _ptr(fom_final), len(init_idx), init,
                                    n_try, float(target), max_samples, out, ctypes.byref(count),
                                    ctypes.byref(met), _stream(stream)))
    return [out[k] for k in range(count.value)], met.value


def raw_call(name: str, *args) -> int:
    """Direct access to a C entry point (used by tests that feed host pointers or
    invalid arguments); returns the status code."""
    return getattr(_LIB, name)(*args)


def last_error() -> str:
    return _LIB.crom_last_error().decode()
