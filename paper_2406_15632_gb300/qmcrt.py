"""Python binding of the qmcrt C ABI (include/qmcrt.h).

Argument marshalling only: every step of the tracer runs in the CUDA library
libqmcrt.so, built in-tree by build.py.  The functions named qmcrt_* mirror the C
entry points one to one; the helpers below them turn a scene description and torch
device tensors into those calls.  PyTorch provides device memory and streams.

There is no CPU fallback: if the library is missing or no GPU is present, the calls
raise.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading

from . import scenes

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libqmcrt.so")

OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_CUDA, ERR_DEVICE_TIMEOUT = 0, -1, -2, -3, -4
KINDS = {"sobol": 0, "sobol_owen": 1, "halton": 2, "hammersley": 3, "philox": 4, "niederreiter": 5, "faure": 6}
FORMATS = {"u32": 0, "f32": 1, "f64": 2}
MEDIUM_GRID, MEDIUM_SPHERE = 0, 1
SOURCE_POINT, SOURCE_SPHERE = 0, 1
ORDER_DIRECT, ORDER_INVERSE = 0, 1
SPLAT = {"nearest": 0, "bilinear": 1}
ACCUM = {"i64": 0, "f64": 1}
PREC = {"f32": 0, "f64": 1}
FORCE = {"all": 0, "first": 1}
MAX_DIMS = 256
MIN_PAD = 8
SKY_M = 64  # fewest texels per cube-face edge of the bound map of rays from a point source
# optical depth a peel-off walk with a tail map may leave out: in FP32 about one rounding of
# e^{-tau_obs} (2^-24), in FP64 far below the 1e-10 agreement with the oracle
TAIL_EPS = {"f32": 2.0 ** -24, "f64": 1e-13}


class QmcrtError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"qmcrt error {code}: {message}")
        self.code = code


class qmcrt_points_desc(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("kind", C.c_int32), ("dims", C.c_uint32), ("format", C.c_int32),
                ("first_index", C.c_uint64), ("count", C.c_uint64), ("total_n", C.c_uint64), ("seed", C.c_uint64)]


class qmcrt_medium(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("kind", C.c_int32), ("d_k", C.c_void_p), ("nx", C.c_int32),
                ("ny", C.c_int32), ("nz", C.c_int32), ("pad", C.c_int32), ("lo", C.c_double * 3),
                ("hi", C.c_double * 3), ("kscale", C.c_double), ("sphere_r", C.c_double), ("sphere_k", C.c_double),
                ("d_sky", C.c_void_p), ("sky_m", C.c_int32), ("sky_reserved", C.c_int32), ("sky_r", C.c_double)]


class qmcrt_source(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("kind", C.c_int32), ("radius", C.c_double), ("limb_u", C.c_double),
                ("order", C.c_int32), ("reserved", C.c_int32)]


class qmcrt_dust(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("reserved", C.c_int32), ("albedo", C.c_double), ("g", C.c_double),
                ("p_l", C.c_double)]


class qmcrt_observer(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("splat", C.c_int32), ("theta", C.c_double), ("phi", C.c_double),
                ("half_width", C.c_double), ("nx", C.c_int32), ("ny", C.c_int32), ("d_tail", C.c_void_p)]


class qmcrt_image(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("accum", C.c_int32), ("d_accum", C.c_void_p), ("n_images", C.c_int32),
                ("frac_bits", C.c_int32)]


class qmcrt_trace_opts(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("precision", C.c_int32), ("tau_min", C.c_double),
                ("max_orders", C.c_int32), ("force_mode", C.c_int32), ("rr_threshold", C.c_double),
                ("rr_survival", C.c_double), ("per_order", C.c_int32), ("block_size", C.c_int32),
                ("tail_eps", C.c_double)]


class qmcrt_instance(C.Structure):
    _fields_ = [("theta", C.c_double), ("phi", C.c_double), ("albedo", C.c_double), ("g", C.c_double),
                ("p_l", C.c_double), ("kscale", C.c_double), ("first_index", C.c_uint64), ("count", C.c_uint64),
                ("d_tail", C.c_void_p)]


class qmcrt_batch_config(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("chunk_log2", C.c_int32), ("block_size", C.c_int32),
                ("ctas_per_sm", C.c_int32), ("packets_per_thread", C.c_int32), ("reserved", C.c_int32)]


class qmcrt_gemm_epilogue(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("relu", C.c_int32), ("d_bias", C.c_void_p), ("d_mask", C.c_void_p),
                ("d_out_f32", C.c_void_p), ("d_out_bf16", C.c_void_p), ("d_out_bf16_t", C.c_void_p),
                ("ldt", C.c_int32), ("k_splits", C.c_int32), ("d_error", C.c_void_p)]


class qmcrt_warp(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("uniform_mix", C.c_float), ("d_params", C.c_void_p),
                ("d_weights", C.c_void_p), ("d_weights_t", C.c_void_p), ("d_error", C.c_void_p)]


class qmcrt_adam(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("step", C.c_int32), ("lr", C.c_double), ("beta1", C.c_double),
                ("beta2", C.c_double), ("eps", C.c_double)]


class qmcrt_host_io(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("reserved", C.c_int32), ("h_k", C.c_void_p), ("d_k", C.c_void_p),
                ("d_accum", C.c_void_p), ("d_image", C.c_void_p), ("h_image", C.c_void_p), ("d_sky_ws", C.c_void_p),
                ("sky_ws_bytes", C.c_uint64), ("d_tail_ws", C.c_void_p), ("tail_ws_bytes", C.c_uint64)]


def _new(cls, **kw):
    s = cls()
    s.struct_size = C.sizeof(cls)
    for k, v in kw.items():
        setattr(s, k, v)
    return s


_lock = threading.Lock()
_lib = None

# every C entry point: (name, restype, argtypes)
_P = C.POINTER
_SIGS = [
    ("qmcrt_abi_version", C.c_int, []),
    ("qmcrt_last_error", C.c_char_p, []),
    ("qmcrt_generate_points", C.c_int, [_P(qmcrt_points_desc), C.c_void_p, C.c_void_p]),
    ("qmcrt_trace_single", C.c_int, [_P(qmcrt_medium), _P(qmcrt_source), _P(qmcrt_dust), _P(qmcrt_observer),
                                     _P(qmcrt_points_desc), _P(qmcrt_trace_opts), _P(qmcrt_image), C.c_void_p,
                                     C.c_void_p]),
    ("qmcrt_trace_multiple", C.c_int, [_P(qmcrt_medium), _P(qmcrt_source), _P(qmcrt_dust), _P(qmcrt_observer),
                                       _P(qmcrt_points_desc), _P(qmcrt_trace_opts), _P(qmcrt_image), C.c_void_p]),
    ("qmcrt_image_reduce", C.c_int, [_P(qmcrt_image), C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_void_p,
                                     C.c_void_p]),
    ("qmcrt_trace_multiple_warped", C.c_int, [_P(qmcrt_medium), _P(qmcrt_source), _P(qmcrt_dust),
                                              _P(qmcrt_observer), _P(qmcrt_points_desc), _P(qmcrt_trace_opts),
                                              C.c_void_p, C.c_void_p, _P(qmcrt_image), C.c_void_p, C.c_void_p]),
    ("qmcrt_trace_observers", C.c_int, [_P(qmcrt_medium), _P(qmcrt_source), _P(qmcrt_dust), _P(qmcrt_observer),
                                        C.c_int32, _P(qmcrt_points_desc), _P(qmcrt_trace_opts), _P(qmcrt_image),
                                        C.c_void_p]),
    ("qmcrt_direct_light", C.c_int, [_P(qmcrt_medium), _P(qmcrt_source), _P(qmcrt_observer), C.c_int32, C.c_double,
                                     _P(qmcrt_trace_opts), _P(qmcrt_image), C.c_void_p]),
    ("qmcrt_wavefront_workspace_bytes", C.c_uint64, [C.c_uint64, C.c_int32]),
    ("qmcrt_trace_multiple_wavefront", C.c_int, [_P(qmcrt_medium), _P(qmcrt_source), _P(qmcrt_dust),
                                                 _P(qmcrt_observer), _P(qmcrt_points_desc), _P(qmcrt_trace_opts),
                                                 C.c_void_p, C.c_void_p, _P(qmcrt_image), C.c_void_p, C.c_void_p,
                                                 C.c_uint64, C.c_void_p]),
    ("qmcrt_batch_workspace_bytes", C.c_uint64, [C.c_int32]),
    ("qmcrt_trace_batch", C.c_int, [_P(qmcrt_medium), _P(qmcrt_source), _P(qmcrt_observer), _P(qmcrt_points_desc),
                                    _P(qmcrt_trace_opts), C.c_void_p, C.c_int32, _P(qmcrt_batch_config), C.c_void_p,
                                    C.c_uint64, _P(qmcrt_image), C.c_void_p]),
    ("qmcrt_batch_reduce", C.c_int, [_P(qmcrt_image), C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p,
                                     C.c_void_p]),
    ("qmcrt_gemm_bf16", C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32,
                                  _P(qmcrt_gemm_epilogue), C.c_void_p]),
    ("qmcrt_warp_workspace_bytes", C.c_uint64, [C.c_uint64]),
    ("qmcrt_warp_sync", C.c_int, [_P(qmcrt_warp), C.c_void_p]),
    ("qmcrt_warp_forward", C.c_int, [_P(qmcrt_warp), C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p,
                                     C.c_uint64, C.c_void_p]),
    ("qmcrt_warp_grad", C.c_int, [_P(qmcrt_warp), C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_uint64, C.c_void_p]),
    ("qmcrt_warp_adam", C.c_int, [_P(qmcrt_warp), C.c_void_p, C.c_void_p, C.c_void_p, _P(qmcrt_adam), C.c_void_p]),
    ("qmcrt_pad_grid", C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p]),
    ("qmcrt_sky_workspace_bytes", C.c_uint64, [C.c_int32, C.c_int32, C.c_int32, _P(C.c_double), _P(C.c_double),
                                               C.c_double]),
    ("qmcrt_sky_bound", C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, _P(C.c_double), _P(C.c_double),
                                  C.c_double, C.c_int32, C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p]),
    ("qmcrt_tail_map_bytes", C.c_uint64, [C.c_int32, C.c_int32, C.c_int32, C.c_int32]),
    ("qmcrt_tail_workspace_bytes", C.c_uint64, [C.c_int32, C.c_int32, C.c_int32]),
    ("qmcrt_tail_map", C.c_int, [_P(qmcrt_medium), _P(qmcrt_observer), C.c_void_p, C.c_void_p, C.c_uint64,
                                 C.c_void_p]),
    ("qmcrt_trace_single_noalloc", C.c_int, [_P(qmcrt_medium), _P(qmcrt_source), _P(qmcrt_dust),
                                             _P(qmcrt_observer), _P(qmcrt_points_desc), _P(qmcrt_trace_opts),
                                             C.c_int32, C.c_double, C.c_void_p, C.c_void_p]),
    ("qmcrt_contribution_bound", C.c_int, [_P(qmcrt_source), _P(qmcrt_dust), _P(qmcrt_trace_opts), C.c_int32,
                                           _P(C.c_double)]),
    ("qmcrt_default_frac_bits", C.c_int, [_P(qmcrt_source), _P(qmcrt_dust), _P(qmcrt_trace_opts), C.c_int32,
                                          C.c_uint64, C.c_double, _P(C.c_int32)]),
    ("qmcrt_render_single_host", C.c_int, [_P(qmcrt_medium), _P(qmcrt_source), _P(qmcrt_dust),
                                           _P(qmcrt_observer), _P(qmcrt_points_desc), _P(qmcrt_trace_opts),
                                           _P(qmcrt_host_io), C.c_int32, C.c_double, C.c_void_p]),
]
EXPORTED = [s[0] for s in _SIGS]


def load(path: str = LIB_PATH):
    """Load libqmcrt.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise QmcrtError(ERR_UNSUPPORTED, f"{path} missing: build the CUDA library first (build.py)")
            L = C.CDLL(path)
            for name, res, args in _SIGS:
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            if L.qmcrt_abi_version() != 3:
                raise QmcrtError(ERR_UNSUPPORTED, "ABI version mismatch")
            _lib = L
    return _lib


def last_error() -> str:
    return load().qmcrt_last_error().decode()


def _check(rc: int):
    if rc != OK:
        raise QmcrtError(rc, last_error())


# --- the C entry points, one to one ----------------------------------------------------

def qmcrt_generate_points(desc: qmcrt_points_desc, d_out: int, stream: int = 0) -> None:
    _check(load().qmcrt_generate_points(C.byref(desc), C.c_void_p(d_out), C.c_void_p(stream)))


def qmcrt_trace_single(medium, source, dust, obs, pts, opts, image, d_log: int = 0, stream: int = 0) -> None:
    _check(load().qmcrt_trace_single(C.byref(medium), C.byref(source), C.byref(dust), C.byref(obs), C.byref(pts),
                                     C.byref(opts), C.byref(image), C.c_void_p(d_log or None), C.c_void_p(stream)))


def qmcrt_trace_multiple(medium, source, dust, obs, pts, opts, image, stream: int = 0) -> None:
    _check(load().qmcrt_trace_multiple(C.byref(medium), C.byref(source), C.byref(dust), C.byref(obs), C.byref(pts),
                                       C.byref(opts), C.byref(image), C.c_void_p(stream)))


def qmcrt_batch_workspace_bytes(n_instances: int) -> int:
    return int(load().qmcrt_batch_workspace_bytes(n_instances))


def qmcrt_trace_batch(medium, source, obs, pts, opts, d_instances: int, n_instances: int, config, d_workspace: int,
                      workspace_bytes: int, image, stream: int = 0) -> None:
    _check(load().qmcrt_trace_batch(C.byref(medium), C.byref(source), C.byref(obs), C.byref(pts), C.byref(opts),
                                    C.c_void_p(d_instances), n_instances, C.byref(config), C.c_void_p(d_workspace),
                                    workspace_bytes, C.byref(image), C.c_void_p(stream)))


def qmcrt_batch_reduce(image, d_instances: int, n_instances: int, nx: int, ny: int, d_out: int,
                       stream: int = 0) -> None:
    _check(load().qmcrt_batch_reduce(C.byref(image), C.c_void_p(d_instances), n_instances, nx, ny, C.c_void_p(d_out),
                                     C.c_void_p(stream)))


def qmcrt_gemm_bf16(d_A: int, d_B: int, M: int, N: int, K: int, epilogue, stream: int = 0) -> None:
    _check(load().qmcrt_gemm_bf16(C.c_void_p(d_A), C.c_void_p(d_B), M, N, K, C.byref(epilogue), C.c_void_p(stream)))


def gemm(A, B, *, bias=None, relu=False, mask=None, out_f32=None, out_bf16=None, out_bf16_t=None, k_splits=1,
         error=None, stream=None):
    """Device tensors: A [M][K] and B [N][K] bf16 -> epilogue outputs (see qmcrt_gemm_bf16)."""
    M, K = A.shape
    N = B.shape[0]
    ptr = lambda t: t.data_ptr() if t is not None else None
    ep = _new(qmcrt_gemm_epilogue, relu=1 if relu else 0, d_bias=ptr(bias), d_mask=ptr(mask), d_out_f32=ptr(out_f32),
              d_out_bf16=ptr(out_bf16), d_out_bf16_t=ptr(out_bf16_t),
              ldt=out_bf16_t.shape[1] if out_bf16_t is not None else 0, k_splits=k_splits, d_error=ptr(error))
    qmcrt_gemm_bf16(A.data_ptr(), B.data_ptr(), M, N, K, ep, _stream(stream))


WARP_BINS, WARP_WIDTH, WARP_PARAMS, WARP_BF16_WEIGHTS = 32, 128, 107360, 106496


def qmcrt_warp_workspace_bytes(rows: int) -> int:
    return int(load().qmcrt_warp_workspace_bytes(rows))


def qmcrt_warp_sync(warp, stream: int = 0) -> None:
    _check(load().qmcrt_warp_sync(C.byref(warp), C.c_void_p(stream)))


def qmcrt_warp_forward(warp, d_u: int, d_x: int, d_logj: int, n: int, d_ws: int, ws_bytes: int,
                       stream: int = 0) -> None:
    _check(load().qmcrt_warp_forward(C.byref(warp), C.c_void_p(d_u), C.c_void_p(d_x), C.c_void_p(d_logj), n,
                                     C.c_void_p(d_ws), ws_bytes, C.c_void_p(stream)))


def qmcrt_warp_grad(warp, d_x: int, d_w: int, n: int, d_grad: int, d_loss: int, d_ws: int, ws_bytes: int,
                    stream: int = 0) -> None:
    _check(load().qmcrt_warp_grad(C.byref(warp), C.c_void_p(d_x), C.c_void_p(d_w), n, C.c_void_p(d_grad),
                                  C.c_void_p(d_loss), C.c_void_p(d_ws), ws_bytes, C.c_void_p(stream)))


def qmcrt_warp_adam(warp, d_grad: int, d_m: int, d_v: int, opt, stream: int = 0) -> None:
    _check(load().qmcrt_warp_adam(C.byref(warp), C.c_void_p(d_grad), C.c_void_p(d_m), C.c_void_p(d_v),
                                  C.byref(opt), C.c_void_p(stream)))


class Warp:
    """Device state of the learned warp: FP32 parameters, their bf16 copies, Adam
    moments, a workspace for `rows` samples per pass, and an error word."""

    def __init__(self, params=None, *, rows: int = 1 << 16, seed: int = 0, uniform_mix: float = 0.0):
        torch = _torch()
        if params is None:
            params = self.initial(seed)
        self.params = torch.as_tensor(params, dtype=torch.float32).to("cuda").contiguous()
        assert self.params.numel() == WARP_PARAMS
        self.wb = torch.zeros(WARP_BF16_WEIGHTS, dtype=torch.bfloat16, device="cuda")
        self.wt = torch.zeros(WARP_BF16_WEIGHTS, dtype=torch.bfloat16, device="cuda")
        self.error = torch.zeros(1, dtype=torch.int32, device="cuda")
        self.desc = _new(qmcrt_warp, d_params=self.params.data_ptr(), d_weights=self.wb.data_ptr(),
                         d_weights_t=self.wt.data_ptr(), d_error=self.error.data_ptr(), uniform_mix=uniform_mix)
        self.ws_bytes = qmcrt_warp_workspace_bytes(rows)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device="cuda")
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        self.step = 0
        qmcrt_warp_sync(self.desc, _stream(None))

    @staticmethod
    def initial(seed: int = 0):
        """He-initialised hidden layers, small output layers, uniform x0 density: the
        initial warp is close to the identity."""
        torch = _torch()
        g = torch.Generator().manual_seed(seed)
        parts = [torch.zeros(WARP_BINS)]
        for m in range(2):
            for l, (o, i) in enumerate([(128, 128), (128, 128), (128, 128), (32, 128)]):
                std = (2.0 / i) ** 0.5 * (0.1 if l == 3 else 1.0)
                parts += [torch.randn((o, i), generator=g).reshape(-1) * std, torch.zeros(o)]
        return torch.cat(parts)

    def forward(self, u, stream=None):
        """x = T(u), log|dx/du| for u [n][3] float32 on the device."""
        torch = _torch()
        n = u.shape[0]
        x = torch.empty((n, 3), dtype=torch.float32, device="cuda")
        lj = torch.empty(n, dtype=torch.float32, device="cuda")
        return self.forward_into(u, x, lj, stream)

    def forward_into(self, u, x, lj, stream=None):
        qmcrt_warp_forward(self.desc, u.data_ptr(), x.data_ptr(), lj.data_ptr(), u.shape[0], self.ws.data_ptr(),
                           self.ws_bytes, _stream(stream))
        return x, lj

    def gradient(self, x, w, stream=None):
        """(loss, gradient) of the cross-entropy on samples x [n][3] with weights w [n]."""
        self.grad.zero_()
        self.loss.zero_()
        qmcrt_warp_grad(self.desc, x.data_ptr(), w.data_ptr(), x.shape[0], self.grad.data_ptr(), self.loss.data_ptr(),
                        self.ws.data_ptr(), self.ws_bytes, _stream(stream))
        return self.loss, self.grad

    def adam_step(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None) -> None:
        self.step += 1
        opt = _new(qmcrt_adam, step=self.step, lr=lr, beta1=beta1, beta2=beta2, eps=eps)
        qmcrt_warp_adam(self.desc, self.grad.data_ptr(), self.m.data_ptr(), self.v.data_ptr(), opt, _stream(stream))

    def train(self, x, w, *, epochs: int = 4, batch: int = 1 << 16, lr: float = 2e-3):
        """Minibatch Adam over the logged samples; returns the loss per step.

        Minibatches are contiguous slices of the log.  A log written in point order by
        a low-discrepancy set needs no shuffle: every aligned block of 2^m consecutive
        Sobol points is itself a net, so each minibatch already covers the cube evenly.
        Epoch e starts at slice e (mod the slice count)."""
        torch = _torch()
        n = x.shape[0]
        nb = n // batch
        losses = []
        for e in range(epochs):
            for k in range(nb):
                b0 = ((e + k) % nb) * batch
                loss, _ = self.gradient(x[b0:b0 + batch], w[b0:b0 + batch])
                losses.append(loss.clone())
                self.adam_step(lr=lr)
        return torch.cat(losses).cpu().tolist() if losses else []


def qmcrt_pad_grid(d_k: int, nx: int, ny: int, nz: int, pad: int, d_padded: int, stream: int = 0) -> None:
    _check(load().qmcrt_pad_grid(C.c_void_p(d_k), nx, ny, nz, pad, C.c_void_p(d_padded), C.c_void_p(stream)))


MAX_OBSERVERS = 16


def qmcrt_sky_workspace_bytes(nx: int, ny: int, nz: int, lo, hi, radius: float) -> int:
    return load().qmcrt_sky_workspace_bytes(nx, ny, nz, (C.c_double * 3)(*lo), (C.c_double * 3)(*hi), float(radius))


def qmcrt_sky_bound(d_k: int, nx: int, ny: int, nz: int, lo, hi, radius: float, m: int, d_map: int, d_ws: int,
                    ws_bytes: int, stream: int = 0) -> None:
    _check(load().qmcrt_sky_bound(C.c_void_p(d_k), nx, ny, nz, (C.c_double * 3)(*lo), (C.c_double * 3)(*hi),
                                  float(radius), m, C.c_void_p(d_map), C.c_void_p(d_ws), ws_bytes,
                                  C.c_void_p(stream)))


def qmcrt_tail_map_bytes(nx: int, ny: int, nz: int, pad: int) -> int:
    return int(load().qmcrt_tail_map_bytes(nx, ny, nz, pad))


def qmcrt_tail_workspace_bytes(nx: int, ny: int, nz: int) -> int:
    return int(load().qmcrt_tail_workspace_bytes(nx, ny, nz))


def qmcrt_tail_map(medium, obs, d_map: int, d_ws: int, ws_bytes: int, stream: int = 0) -> None:
    _check(load().qmcrt_tail_map(C.byref(medium), C.byref(obs), C.c_void_p(d_map), C.c_void_p(d_ws), ws_bytes,
                                 C.c_void_p(stream)))


def qmcrt_wavefront_workspace_bytes(max_packets: int, precision: str = "f32") -> int:
    return int(load().qmcrt_wavefront_workspace_bytes(max_packets, PREC[precision]))


def qmcrt_trace_multiple_wavefront(medium, source, dust, obs, pts, opts, d_x: int, d_logj: int, image,
                                   d_train_log: int, d_workspace: int, workspace_bytes: int, stream: int = 0) -> None:
    _check(load().qmcrt_trace_multiple_wavefront(C.byref(medium), C.byref(source), C.byref(dust), C.byref(obs),
                                                 C.byref(pts), C.byref(opts), C.c_void_p(d_x or None),
                                                 C.c_void_p(d_logj or None), C.byref(image),
                                                 C.c_void_p(d_train_log or None), C.c_void_p(d_workspace),
                                                 workspace_bytes, C.c_void_p(stream)))


def qmcrt_direct_light(medium, source, obs, subsamples: int, weight: float, opts, image, stream: int = 0) -> None:
    _check(load().qmcrt_direct_light(C.byref(medium), C.byref(source), C.byref(obs), subsamples, weight,
                                     C.byref(opts), C.byref(image), C.c_void_p(stream)))


def qmcrt_trace_observers(medium, source, dust, obs_array, n_obs: int, pts, opts, image, stream: int = 0) -> None:
    _check(load().qmcrt_trace_observers(C.byref(medium), C.byref(source), C.byref(dust), obs_array, n_obs, C.byref(pts),
                                        C.byref(opts), C.byref(image), C.c_void_p(stream)))


def qmcrt_trace_multiple_warped(medium, source, dust, obs, pts, opts, d_x: int, d_logj: int, image,
                                d_train_log: int = 0, stream: int = 0) -> None:
    _check(load().qmcrt_trace_multiple_warped(C.byref(medium), C.byref(source), C.byref(dust), C.byref(obs),
                                              C.byref(pts), C.byref(opts), C.c_void_p(d_x or None),
                                              C.c_void_p(d_logj or None), C.byref(image),
                                              C.c_void_p(d_train_log or None), C.c_void_p(stream)))


def qmcrt_image_reduce(image, nx: int, ny: int, n_replicas: int, scale: float, d_out: int, stream: int = 0) -> None:
    _check(load().qmcrt_image_reduce(C.byref(image), nx, ny, n_replicas, scale, C.c_void_p(d_out),
                                     C.c_void_p(stream)))


def qmcrt_trace_single_noalloc(medium, source, dust, obs, pts, opts, frac_bits: int, scale: float, d_image: int,
                               stream: int = 0) -> None:
    """Single scattering into the FP64 image at d_image ([3][ny][nx]) with the library's
    own accumulation scratch: for callers that cannot allocate device memory.  Calls
    share that scratch, so calls that overlap on the GPU must be avoided."""
    _check(load().qmcrt_trace_single_noalloc(C.byref(medium), C.byref(source), C.byref(dust), C.byref(obs),
                                             C.byref(pts), C.byref(opts), frac_bits, scale, C.c_void_p(d_image),
                                             C.c_void_p(stream)))


def qmcrt_contribution_bound(source, dust, opts, multiple: bool) -> float:
    out = C.c_double(0.0)
    _check(load().qmcrt_contribution_bound(C.byref(source), C.byref(dust), C.byref(opts), int(bool(multiple)),
                                           C.byref(out)))
    return out.value


def qmcrt_default_frac_bits(source, dust, opts, multiple: bool, n_packets: int, weight_bound: float = 1.0) -> int:
    out = C.c_int32(0)
    _check(load().qmcrt_default_frac_bits(C.byref(source), C.byref(dust), C.byref(opts), int(bool(multiple)),
                                          int(n_packets), float(weight_bound), C.byref(out)))
    return out.value


def qmcrt_render_single_host(medium, source, dust, obs, pts, opts, io, frac_bits: int, scale: float,
                             stream: int = 0) -> None:
    _check(load().qmcrt_render_single_host(C.byref(medium), C.byref(source), C.byref(dust), C.byref(obs),
                                           C.byref(pts), C.byref(opts), C.byref(io), frac_bits, scale,
                                           C.c_void_p(stream)))


# --- marshalling helpers ------------------------------------------------------------------

def _torch():
    import torch

    return torch


def _stream(stream) -> int:
    torch = _torch()
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def points_desc(kind: str, dims: int, first: int, count: int, fmt: str = "f64", seed: int = 0,
                total_n: int = 0) -> qmcrt_points_desc:
    return _new(qmcrt_points_desc, kind=KINDS[kind], dims=dims, format=FORMATS[fmt], first_index=first, count=count,
                total_n=total_n, seed=seed)


def generate_points(kind: str, dims: int, first: int, count: int, fmt: str = "f64", seed: int = 0,
                    total_n: int = 0, out=None, stream=None):
    """Device tensor [count][dims] of points first..first+count-1."""
    torch = _torch()
    dt = {"u32": torch.int32, "f32": torch.float32, "f64": torch.float64}[fmt]
    if out is None:
        out = torch.empty((count, dims), dtype=dt, device="cuda")
    qmcrt_generate_points(points_desc(kind, dims, first, count, fmt, seed, total_n), out.data_ptr(), _stream(stream))
    return out


def _bound_structs(prob: scenes.Problem):
    """The source, dust and options descriptors of a problem (no device memory)."""
    source = _new(qmcrt_source, kind=SOURCE_POINT if prob.source == "point" else SOURCE_SPHERE, radius=prob.star_r,
                  limb_u=prob.limb_u, order=ORDER_DIRECT if prob.emit_order == "direct" else ORDER_INVERSE)
    dust = _new(qmcrt_dust, albedo=prob.albedo, g=prob.g, p_l=prob.p_l)
    opts = _new(qmcrt_trace_opts, precision=0, tau_min=prob.tau_min, max_orders=max(prob.max_orders, 1),
                force_mode=FORCE[prob.force], rr_threshold=prob.rr_threshold, rr_survival=prob.rr_survival,
                per_order=1 if prob.per_order else 0)
    return source, dust, opts


def contribution_bound(prob: scenes.Problem) -> float:
    """Upper bound on |I|, |Q|, |U| of one peel-off contribution of the problem
    (qmcrt_contribution_bound; multiple scattering when max_orders > 1)."""
    return qmcrt_contribution_bound(*_bound_structs(prob), prob.max_orders > 1)


def default_frac_bits(prob: scenes.Problem, n_contributions: int, weight_bound: float = 1.0) -> int:
    """Largest fixed-point scale that cannot overflow for n packets of the problem
    (qmcrt_default_frac_bits); weight_bound multiplies every weight (mix^-3 for a warp
    with a uniform mixture)."""
    return qmcrt_default_frac_bits(*_bound_structs(prob), prob.max_orders > 1, n_contributions, weight_bound)


class Scene:
    """The descriptor structs of one problem, with its grid resident on the device: the
    sentinel-padded copy the fast walk reads (pad > 0) and the bound map of rays from the
    source (qmcrt_sky_bound over the source's radius, sky texels per cube-face edge; 0:
    none; None: for a point source 1.25 per cell of the longest axis, rounded up to a multiple
    of 8 and at least SKY_M; none for a finite star), and for a padded grid
    the tail map of the observer's direction (qmcrt_tail_map; None: for single scattering
    only), with which peel-off walks stop once what is left of their optical depth is
    below TAIL_EPS."""

    def __init__(self, prob: scenes.Problem, grid_device=None, device="cuda", pad: int = MIN_PAD,
                 sky: int | None = None, tail: bool | None = None):
        torch = _torch()
        self.prob = prob
        self.pad = pad
        self.padded = None
        self.sky = None
        self.tail = None
        self._tails = {}
        if prob.grid is not None:
            if grid_device is None:
                grid_device = torch.as_tensor(prob.grid, dtype=torch.float32).to(device).contiguous()
            self.grid = grid_device
            nz, ny, nx = self.grid.shape
            d_k = self.grid.data_ptr()
            if pad:
                self.padded = torch.empty((nz + 2 * pad, ny + 2 * pad, nx + 2 * pad), dtype=torch.float32,
                                          device=device)
                d_k = self.padded.data_ptr()
            self.medium = _new(qmcrt_medium, kind=MEDIUM_GRID, d_k=d_k, nx=nx, ny=ny, nz=nz, pad=pad,
                               kscale=prob.kscale)
            if sky is None:
                # by default a point source only (over a finite star's ball the bound is loose:
                # steep rays from its edge reach the disk's dense inner rim), with at least
                # 1.25 texels per cell along a face so that a texel's cone stays within a cell
                # (256^3 disk: 320 texels built in 1.2 ms, the same rays certified as by 512
                # in 2.0 ms; 256 leave a third of the texels without a bound)
                sky = max(SKY_M, 8 * math.ceil(1.25 * max(nx, ny, nz) / 8)) if prob.source == "point" else 0
                sky = min(sky, 4096)
            if sky:
                r = prob.star_r if prob.source == "sphere" else 0.0
                self.sky = torch.empty((6, sky, sky), dtype=torch.float64, device=device)
                self.sky_ws_bytes = qmcrt_sky_workspace_bytes(nx, ny, nz, prob.lo, prob.hi, r)
                self.sky_ws = torch.empty(self.sky_ws_bytes // 8 + 32, dtype=torch.float64, device=device)
                self.medium.d_sky = self.sky.data_ptr()
                self.medium.sky_m = sky
                self.medium.sky_r = r
        else:
            self.grid = None
            self.medium = _new(qmcrt_medium, kind=MEDIUM_SPHERE, d_k=None, kscale=prob.kscale,
                               sphere_r=prob.sphere_r, sphere_k=prob.sphere_k)
        for a in range(3):
            self.medium.lo[a] = prob.lo[a]
            self.medium.hi[a] = prob.hi[a]
        self.source = _new(qmcrt_source, kind=SOURCE_POINT if prob.source == "point" else SOURCE_SPHERE,
                           radius=prob.star_r, limb_u=prob.limb_u,
                           order=ORDER_DIRECT if prob.emit_order == "direct" else ORDER_INVERSE)
        self.dust = _new(qmcrt_dust, albedo=prob.albedo, g=prob.g, p_l=prob.p_l)
        self.obs = _new(qmcrt_observer, splat=SPLAT[prob.splat], theta=prob.theta_obs, phi=prob.phi_obs,
                        half_width=prob.half_width, nx=prob.nx, ny=prob.ny)
        if tail is None:
            # by default for single scattering: on the 256^3 disk the peel-off walks drop from
            # 13.1 to 10.3 ms per 2^26 packets; in the clumpy envelope, which fills its box's
            # inscribed ball, the map seldom ends a walk and the 2^24-packet wavefront takes
            # 80.7 ms with it against 77.3 without
            tail = prob.max_orders == 1
        if tail and self.padded is not None:
            nz, ny, nx = self.grid.shape
            self.tail = torch.empty(qmcrt_tail_map_bytes(nx, ny, nz, pad), dtype=torch.uint8, device=device)
            self.tail_ws_bytes = qmcrt_tail_workspace_bytes(nx, ny, nz)
            self.tail_ws = torch.empty(self.tail_ws_bytes // 8 + 32, dtype=torch.float64, device=device)
            self.obs.d_tail = self.tail.data_ptr()
        self.repad()

    def repad(self, stream=None) -> None:
        """Refresh the padded copy, the bound map and the tail map after the grid changed."""
        if self.grid is None:
            return
        nz, ny, nx = self.grid.shape
        if self.padded is not None:
            qmcrt_pad_grid(self.grid.data_ptr(), nx, ny, nz, self.pad, self.padded.data_ptr(), _stream(stream))
        if self.sky is not None:
            qmcrt_sky_bound(self.grid.data_ptr(), nx, ny, nz, self.prob.lo, self.prob.hi, self.medium.sky_r,
                            self.sky.shape[-1], self.sky.data_ptr(), self.sky_ws.data_ptr(), self.sky_ws_bytes,
                            _stream(stream))
        if self.tail is not None:
            qmcrt_tail_map(self.medium, self.obs, self.tail.data_ptr(), self.tail_ws.data_ptr(), self.tail_ws_bytes,
                           _stream(stream))
            for (th, ph), t in self._tails.items():  # in place: batches hold their addresses
                qmcrt_tail_map(self.medium, self._direction(th, ph), t.data_ptr(), self.tail_ws.data_ptr(),
                               self.tail_ws_bytes, _stream(stream))

    def opts(self, precision: str = "f32", block_size: int = 0) -> qmcrt_trace_opts:
        p = self.prob
        return _new(qmcrt_trace_opts, precision=PREC[precision], tau_min=p.tau_min, max_orders=p.max_orders,
                    force_mode=FORCE[p.force], rr_threshold=p.rr_threshold, rr_survival=p.rr_survival,
                    per_order=1 if p.per_order else 0, block_size=block_size, tail_eps=TAIL_EPS[precision])

    def accum_buffer(self, accum: str = "i64", replicas: int = 1):
        torch = _torch()
        dt = torch.int64 if accum == "i64" else torch.float64
        return torch.zeros((replicas, self.prob.n_images, 3, self.prob.ny, self.prob.nx), dtype=dt, device="cuda")

    def image_desc(self, buf, accum: str = "i64", frac_bits: int = 0) -> qmcrt_image:
        return _new(qmcrt_image, accum=ACCUM[accum], d_accum=buf.data_ptr(), n_images=self.prob.n_images,
                    frac_bits=frac_bits)

    def trace(self, first: int, count: int, buf, *, accum: str = "i64", frac_bits: int = 0, precision: str = "f32",
              log=None, stream=None, block_size: int = 0) -> None:
        """Add the contributions of packets first..first+count-1 to buf."""
        p = self.prob
        pts = points_desc(p.generator, p.dims, first, count, "f64", p.seed, p.total_n)
        img = self.image_desc(buf, accum, frac_bits)
        if p.max_orders > 1:
            if log is not None:
                raise QmcrtError(ERR_UNSUPPORTED, "the packet log is single-scattering only")
            qmcrt_trace_multiple(self.medium, self.source, self.dust, self.obs, pts, self.opts(precision, block_size),
                                 img, _stream(stream))
        else:
            qmcrt_trace_single(self.medium, self.source, self.dust, self.obs, pts, self.opts(precision, block_size),
                               img, log.data_ptr() if log is not None else 0, _stream(stream))

    def trace_warped(self, first: int, count: int, buf, *, x=None, logj=None, train_log=None, accum: str = "i64",
                     frac_bits: int = 0, precision: str = "f32", stream=None) -> None:
        """Multiple scattering with the first-order coordinates of packet j taken from
        x[j] (weight times exp(logj[j])); optionally log per packet [n][5]: x, then the
        sum and the L2 norm of the in-image intensities of its peel-offs."""
        p = self.prob
        pts = points_desc(p.generator, p.dims, first, count, "f64", p.seed, p.total_n)
        img = self.image_desc(buf, accum, frac_bits)
        ptr = lambda t: t.data_ptr() if t is not None else 0
        qmcrt_trace_multiple_warped(self.medium, self.source, self.dust, self.obs, pts, self.opts(precision), ptr(x),
                                    ptr(logj), img, ptr(train_log), _stream(stream))

    def direct_light(self, buf, *, weight: float = 1.0, subsamples: int = 4, accum: str = "i64", frac_bits: int = 0,
                     precision: str = "f32", stream=None) -> None:
        """Add the source's direct light (times weight) to image 0 of buf."""
        qmcrt_direct_light(self.medium, self.source, self.obs, subsamples, weight, self.opts(precision),
                           self.image_desc(buf, accum, frac_bits), _stream(stream))

    def tail_for(self, theta: float, phi: float):
        """The tail map toward (theta, phi) on this scene's grid (built once, rebuilt in place
        by repad), or None without a padded grid or with tail maps off."""
        if self.tail is None:
            return None
        if theta == self.prob.theta_obs and phi == self.prob.phi_obs:
            return self.tail
        key = (float(theta), float(phi))
        if key not in self._tails:
            torch = _torch()
            t = torch.empty_like(self.tail)
            qmcrt_tail_map(self.medium, self._direction(*key), t.data_ptr(), self.tail_ws.data_ptr(),
                           self.tail_ws_bytes, 0)
            self._tails[key] = t
        return self._tails[key]

    def _direction(self, theta: float, phi: float):
        """An observer struct that only carries a direction (for building its tail map)."""
        return _new(qmcrt_observer, splat=self.obs.splat, theta=theta, phi=phi, half_width=1.0, nx=1, ny=1)

    def observer_array(self, angles, half_widths=None, tails: bool = True):
        """ctypes array of observers at (theta, phi) pairs sharing this problem's image
        shape and splat; half widths default to the problem's; each with the tail map of
        its direction unless tails is False."""
        p = self.prob
        arr = (qmcrt_observer * len(angles))()
        for o, (th, ph) in enumerate(angles):
            hw = p.half_width if half_widths is None else half_widths[o]
            t = self.tail_for(th, ph) if tails else None
            arr[o] = _new(qmcrt_observer, splat=SPLAT[p.splat], theta=th, phi=ph, half_width=hw, nx=p.nx, ny=p.ny,
                          d_tail=None if t is None else t.data_ptr())
        return arr

    def trace_observers(self, angles, first: int, count: int, buf, *, half_widths=None, accum: str = "i64",
                        frac_bits: int = 0, precision: str = "f32", stream=None) -> None:
        """One trace of packets first..first+count-1 peeled off toward every observer in
        `angles` ((theta, phi) pairs); buf is [n_obs][n_images][3][ny][nx]."""
        p = self.prob
        arr = self.observer_array(angles, half_widths)
        pts = points_desc(p.generator, p.dims, first, count, "f64", p.seed, p.total_n)
        img = self.image_desc(buf, accum, frac_bits)
        qmcrt_trace_observers(self.medium, self.source, self.dust, arr, len(angles), pts, self.opts(precision), img,
                              _stream(stream))

    def wavefront_workspace(self, max_packets: int, precision: str = "f32"):
        """Device workspace for trace_wavefront of up to max_packets packets per chunk."""
        torch = _torch()
        n = qmcrt_wavefront_workspace_bytes(max_packets, precision)
        return torch.empty(n, dtype=torch.uint8, device="cuda")

    def trace_wavefront(self, first: int, count: int, buf, ws, *, x=None, logj=None, train_log=None,
                        accum: str = "i64", frac_bits: int = 0, precision: str = "f32", stream=None) -> None:
        """Multiple scattering order by order, live packets regrouped between orders
        (the same images as trace / trace_warped)."""
        p = self.prob
        pts = points_desc(p.generator, p.dims, first, count, "f64", p.seed, p.total_n)
        img = self.image_desc(buf, accum, frac_bits)
        ptr = lambda t: t.data_ptr() if t is not None else 0
        qmcrt_trace_multiple_wavefront(self.medium, self.source, self.dust, self.obs, pts, self.opts(precision), ptr(x),
                                       ptr(logj), img, ptr(train_log), ws.data_ptr(), ws.numel(), _stream(stream))

    def reduce(self, buf, scale: float, *, accum: str = "i64", frac_bits: int = 0, out=None, stream=None):
        torch = _torch()
        if out is None:
            out = torch.empty((self.prob.n_images, 3, self.prob.ny, self.prob.nx), dtype=torch.float64, device="cuda")
        replicas = buf.shape[0] if buf.dim() == 5 else 1
        qmcrt_image_reduce(self.image_desc(buf, accum, frac_bits), self.prob.nx, self.prob.ny, replicas, scale,
                           out.data_ptr(), _stream(stream))
        return out


def render(prob: scenes.Problem, n_packets: int, first: int = 1, *, precision: str = "f32", accum: str = "i64",
           frac_bits: int | None = None, log: bool = False, scale: float | None = None, pad: int = MIN_PAD):
    """Trace packets first..first+n_packets-1 and return the image [n_images][3][ny][nx]
    (float64, scaled by 1/n_packets unless scale is given), and the packet log if asked.
    pad = 0 walks the plain grid with cell counters instead of the padded grid."""
    torch = _torch()
    sc = Scene(prob, pad=pad)
    fb = default_frac_bits(prob, n_packets) if frac_bits is None else frac_bits
    buf = sc.accum_buffer(accum)
    lg = torch.zeros((n_packets, 9), dtype=torch.float64, device="cuda") if log else None
    sc.trace(first, n_packets, buf, accum=accum, frac_bits=fb, precision=precision, log=lg)
    img = sc.reduce(buf, 1.0 / n_packets if scale is None else scale, accum=accum, frac_bits=fb)
    return (img, lg) if log else img


class LearnedTracer:
    """Multiple scattering with the learned proposal on the first-order coordinates.

    Per chunk of packets: the point kernel writes the first three coordinates u (FP32),
    the warp maps them to x = T(u) with log |dx/du| on the tensor cores, and the tracer
    reads x and multiplies each packet's weight by |dx/du|.  With warp = None the same
    loop runs the plain tracer (and can still write the training log).  With
    wavefront=True the orders run as a wavefront with live packets regrouped between
    orders (the same images, fewer idle lanes)."""

    def __init__(self, scene: "Scene", warp: "Warp | None", *, chunk: int = 1 << 22, wavefront: bool = False,
                 precision: str = "f32"):
        torch = _torch()
        self.scene, self.warp, self.chunk = scene, warp, chunk
        self.u = torch.empty((chunk, 3), dtype=torch.float32, device="cuda")
        self.x = torch.empty((chunk, 3), dtype=torch.float32, device="cuda")
        self.lj = torch.empty(chunk, dtype=torch.float32, device="cuda")
        self.ws = scene.wavefront_workspace(chunk, precision) if wavefront else None

    def weight_bound(self) -> float:
        """Bound on |dx/du| (1 without a warp; mix^-3 with a uniform mixture)."""
        if self.warp is None:
            return 1.0
        mix = self.warp.desc.uniform_mix
        return mix ** -3 if mix > 0 else math.inf

    def trace(self, first: int, count: int, buf, *, frac_bits: int = 0, accum: str = "f64", precision: str = "f32",
              train_log=None, stream=None) -> None:
        """Add packets first..first+count-1 to buf.  FP64 accumulation is the default
        here: a fixed-point scale must leave room for the largest Jacobian weight."""
        p = self.scene.prob
        if accum == "i64" and math.isinf(self.weight_bound()):
            raise QmcrtError(ERR_INVALID_ARG, "fixed-point accumulation needs a bounded warp (uniform_mix > 0)")
        for c0 in range(0, count, self.chunk):
            n = min(self.chunk, count - c0)
            log = train_log[c0:c0 + n] if train_log is not None else None
            x = lj = None
            if self.warp is not None:
                u, x, lj = self.u[:n], self.x[:n], self.lj[:n]
                generate_points(p.generator, 3, first + c0, n, "f32", p.seed, p.total_n, out=u, stream=stream)
                self.warp.forward_into(u, x, lj, stream=stream)
            if self.ws is not None:
                self.scene.trace_wavefront(first + c0, n, buf, self.ws, x=x, logj=lj, train_log=log, accum=accum,
                                           frac_bits=frac_bits, precision=precision, stream=stream)
            else:
                self.scene.trace_warped(first + c0, n, buf, x=x, logj=lj, train_log=log, accum=accum,
                                        frac_bits=frac_bits, precision=precision, stream=stream)


class HostRenderer:
    """The end-to-end call for host-resident inputs: each call enqueues, through
    qmcrt_render_single_host, the copy of the density grid from (pinned) host memory,
    its padding, the trace of a packet range, the reduction and the copy of the image
    back to host memory, all on one stream.  Device buffers are allocated once, at
    construction.  The bound map of rays from the source (for a point source) and the
    observer's tail map are rebuilt from every new grid inside the call; sky=0 walks every
    ray, tail=False walks every peel-off to the edge."""

    def __init__(self, prob: scenes.Problem, max_packets: int, *, precision: str = "f32",
                 frac_bits: int | None = None, sky: int | None = None, tail: bool | None = None):
        torch = _torch()
        if prob.max_orders > 1:
            raise QmcrtError(ERR_UNSUPPORTED, "HostRenderer renders single scattering")
        self.scene = Scene(prob, sky=sky, tail=tail)
        self.precision = precision
        self.frac_bits = default_frac_bits(prob, max_packets) if frac_bits is None else frac_bits
        self.buf = self.scene.accum_buffer("i64")
        self.out = torch.empty((1, 3, prob.ny, prob.nx), dtype=torch.float64, device="cuda")

    def input_bytes(self) -> int:
        return 0 if self.scene.grid is None else self.scene.grid.numel() * 4

    def output_bytes(self) -> int:
        return self.out.numel() * 8

    def __call__(self, host_grid, first: int, count: int, host_out, stream=None) -> None:
        sc, p = self.scene, self.scene.prob
        io = _new(qmcrt_host_io, h_k=None if sc.grid is None else host_grid.data_ptr(),
                  d_k=None if sc.grid is None else sc.grid.data_ptr(), d_accum=self.buf.data_ptr(),
                  d_image=self.out.data_ptr(), h_image=host_out.data_ptr(),
                  d_sky_ws=None if sc.sky is None else sc.sky_ws.data_ptr(),
                  sky_ws_bytes=0 if sc.sky is None else sc.sky_ws_bytes,
                  d_tail_ws=None if sc.tail is None else sc.tail_ws.data_ptr(),
                  tail_ws_bytes=0 if sc.tail is None else sc.tail_ws_bytes)
        pts = points_desc(p.generator, p.dims, first, count, "f64", p.seed, p.total_n)
        qmcrt_render_single_host(sc.medium, sc.source, sc.dust, sc.obs, pts, sc.opts(self.precision), io,
                                 self.frac_bits, 1.0 / count, _stream(stream))


class Batch:
    """Many instances (observer, wavelength, budget) of one problem traced in one
    persistent launch: the instance table, workspace and images live on the device;
    run() enqueues plan + trace + reduce on the current stream, and capture() records
    that sequence in a CUDA graph that replay() launches again."""

    def __init__(self, prob: scenes.Problem, instances, *, precision: str = "f32", chunk_log2: int = 16,
                 block_size: int = 256, ctas_per_sm: int = 0, packets_per_thread: int = 4,
                 frac_bits: int | None = None, scene: "Scene | None" = None, tails: bool = True):
        torch = _torch()
        self.prob = prob
        self.scene = scene or Scene(prob)
        self.precision = precision
        self.n = len(instances)
        table = (qmcrt_instance * self.n)()
        self.tails = []  # the tail map of each instance's direction (scene.tail_for), or None
        for t, I in zip(table, instances):
            t.theta, t.phi, t.albedo, t.g = I.theta_obs, prob.phi_obs, I.albedo, I.g
            t.p_l, t.kscale, t.first_index, t.count = prob.p_l, I.kscale, I.first_index, I.n_packets
            m = self.scene.tail_for(I.theta_obs, prob.phi_obs) if tails else None
            t.d_tail = None if m is None else m.data_ptr()
            self.tails.append(m)
        raw = torch.frombuffer(bytearray(bytes(table)), dtype=torch.uint8)
        self.d_inst = raw.to("cuda")
        self.counts = [I.n_packets for I in instances]
        self.instances = list(instances)
        self.ws_bytes = qmcrt_batch_workspace_bytes(self.n)
        self.ws = torch.zeros(self.ws_bytes // 8, dtype=torch.int64, device="cuda")
        self.accum = torch.zeros((self.n, 3, prob.ny, prob.nx), dtype=torch.int64, device="cuda")
        self.out = torch.zeros((self.n, 3, prob.ny, prob.nx), dtype=torch.float64, device="cuda")
        bound_prob = prob.replace(g=max(abs(I.g) for I in instances), albedo=max(I.albedo for I in instances))
        self.frac_bits = default_frac_bits(bound_prob, max(self.counts)) if frac_bits is None else frac_bits
        self.graph = None
        self.set_config(chunk_log2, block_size, ctas_per_sm, packets_per_thread)

    def set_config(self, chunk_log2: int, block_size: int, ctas_per_sm: int, packets_per_thread: int) -> None:
        self.config = _new(qmcrt_batch_config, chunk_log2=chunk_log2, block_size=block_size, ctas_per_sm=ctas_per_sm,
                           packets_per_thread=packets_per_thread)
        self.graph = None

    def packets(self) -> int:
        return sum(self.counts)

    def run(self, stream=None) -> None:
        sc = self.scene
        st = _stream(stream)
        self.accum.zero_()
        pts = points_desc(self.prob.generator, self.prob.dims, 1, 1, "f64", self.prob.seed, 0)
        img = _new(qmcrt_image, accum=ACCUM["i64"], d_accum=self.accum.data_ptr(), n_images=1,
                   frac_bits=self.frac_bits)
        qmcrt_trace_batch(sc.medium, sc.source, sc.obs, pts, sc.opts(self.precision), self.d_inst.data_ptr(), self.n,
                          self.config, self.ws.data_ptr(), self.ws_bytes, img, st)
        qmcrt_batch_reduce(img, self.d_inst.data_ptr(), self.n, self.prob.nx, self.prob.ny, self.out.data_ptr(), st)

    def run_each(self, stream=None) -> None:
        """The same images by one regular qmcrt_trace_single launch per instance (the
        un-batched way), for comparison."""
        sc = self.scene
        st = _stream(stream)
        self.accum.zero_()
        opts = sc.opts(self.precision)
        for k, (I, n) in enumerate(zip(self.instances, self.counts)):
            if n == 0:
                continue
            med = qmcrt_medium.from_buffer_copy(sc.medium)
            med.kscale = sc.medium.kscale * I.kscale
            dust = _new(qmcrt_dust, albedo=I.albedo, g=I.g, p_l=self.prob.p_l)
            obs = qmcrt_observer.from_buffer_copy(sc.obs)
            obs.theta = I.theta_obs
            obs.d_tail = None if self.tails[k] is None else self.tails[k].data_ptr()  # this direction's map
            pts = points_desc(self.prob.generator, self.prob.dims, I.first_index, n, "f64", self.prob.seed,
                              I.first_index + n - 1)
            img = _new(qmcrt_image, accum=ACCUM["i64"], d_accum=self.accum[k].data_ptr(), n_images=1,
                       frac_bits=self.frac_bits)
            qmcrt_trace_single(med, sc.source, dust, obs, pts, opts, img, 0, st)
        img = _new(qmcrt_image, accum=ACCUM["i64"], d_accum=self.accum.data_ptr(), n_images=1,
                   frac_bits=self.frac_bits)
        qmcrt_batch_reduce(img, self.d_inst.data_ptr(), self.n, self.prob.nx, self.prob.ny, self.out.data_ptr(), st)

    def capture(self) -> None:
        torch = _torch()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):  # warm-up outside the capture
            self.run()
        torch.cuda.current_stream().wait_stream(s)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.run()

    def replay(self) -> None:
        if self.graph is None:
            self.capture()
        self.graph.replay()
