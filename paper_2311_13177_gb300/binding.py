"""Thin Python binding of libprop with the C ABI's names.

Argument marshalling only: torch tensors supply device pointers and the
current CUDA stream, numpy arrays supply host buffers; every step of the
operator, adjoint, loss and optimiser runs in libprop's kernels.

Layouts (complex64): V [T, N, N, Nf] (index [t, i2, i1, f], x = i - N/2),
y [B, L, R], image [T, N, N]; projection model: Cartesian k-space [N, N]
(index [u2, u1], k = (u - N/2)/N), per-blade data [B, N, N].
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from ._lib import PlanDesc, ProjParamsC, ReconParamsC, check, lib

__all__ = ["Plan", "ReconParams", "ProjParams", "prop_plan_create", "prop_plan_destroy", "prop_plan_workspace_bytes",
           "prop_forward", "prop_adjoint", "prop_reconstruct", "prop_reconstruct_host",
           "prop_loss_grad", "prop_render", "prop_psnr", "prop_reconstruct_batch"]


@dataclass
class ReconParams:
    iters: int = 20
    lr: float = 1e-2
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    tv_xy: float = 1e-3
    tv_t: float = 0.0
    tv_eps: float = 1e-3

    def c(self) -> ReconParamsC:
        return ReconParamsC(int(self.iters), float(self.lr), float(self.beta1), float(self.beta2),
                            float(self.eps), float(self.tv_xy), float(self.tv_t), float(self.tv_eps))


@dataclass
class ProjParams:
    """Settings of prop_proj_reconstruct (the paper's own forward model)."""
    iters: int = 20
    lr: float = 1e-2
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    w_kspace: float = 0.1
    w_image: float = 1.0
    tv_xy: float = 1e-3
    tv_f: float = 0.0
    tv_t: float = 0.0
    l1: float = 0.0
    tv_eps: float = 1e-3

    def c(self) -> ProjParamsC:
        return ProjParamsC(int(self.iters), float(self.lr), float(self.beta1), float(self.beta2), float(self.eps),
                           float(self.w_kspace), float(self.w_image), float(self.tv_xy), float(self.tv_f),
                           float(self.tv_t), float(self.l1), float(self.tv_eps))


def _stream(stream=None) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream))


def _dev_ptr(t: torch.Tensor, shape, name: str) -> ctypes.c_void_p:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.complex64:
        raise TypeError(f"{name} must be complex64, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """A libprop plan (geometry tables + workspace on one device)."""

    def __init__(self, N, L, R, theta, delta, blade_frame=None, T=1, bin_chunk=0, device=None, kb_width=0,
                 row_kernel=0):
        theta = np.ascontiguousarray(theta, dtype=np.float64)
        delta = np.ascontiguousarray(delta, dtype=np.float64)
        if device is None:
            device = torch.cuda.current_device()
        self.N, self.L, self.R, self.T = int(N), int(L), int(R), int(T)
        self.B, self.Nf = len(theta), len(delta)
        self.device = torch.device("cuda", int(device))
        bf_ptr = None
        if blade_frame is not None:
            self._bf = np.ascontiguousarray(blade_frame, dtype=np.int32)
            bf_ptr = self._bf.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        desc = PlanDesc(self.N, self.Nf, delta.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                        self.B, theta.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), self.L, self.R,
                        self.T, bf_ptr, int(kb_width), int(bin_chunk), int(row_kernel), int(device))
        h = ctypes.c_void_p()
        check(lib().prop_plan_create(ctypes.byref(desc), ctypes.byref(h)), "prop_plan_create")
        self._h = h

    # shapes
    @property
    def vol_shape(self):
        return (self.T, self.N, self.N, self.Nf)

    @property
    def data_shape(self):
        return (self.B, self.L, self.R)

    @property
    def handle(self) -> ctypes.c_void_p:
        if self._h is None:
            raise RuntimeError("plan has been destroyed")
        return self._h

    def destroy(self):
        if getattr(self, "_h", None) is not None:
            check(lib().prop_plan_destroy(self._h), "prop_plan_destroy")
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def workspace_bytes(self) -> int:
        v = ctypes.c_size_t()
        check(lib().prop_plan_workspace_bytes(self.handle, ctypes.byref(v)), "prop_plan_workspace_bytes")
        return int(v.value)

    def forward(self, V: torch.Tensor, y: torch.Tensor = None, stream=None) -> torch.Tensor:
        if y is None:
            y = torch.empty(self.data_shape, dtype=torch.complex64, device=V.device)
        check(lib().prop_forward(self.handle, _dev_ptr(V, self.vol_shape, "V"),
                                 _dev_ptr(y, self.data_shape, "y"), _stream(stream)), "prop_forward")
        return y

    def adjoint(self, y: torch.Tensor, V: torch.Tensor = None, stream=None) -> torch.Tensor:
        if V is None:
            V = torch.empty(self.vol_shape, dtype=torch.complex64, device=y.device)
        check(lib().prop_adjoint(self.handle, _dev_ptr(y, self.data_shape, "y"),
                                 _dev_ptr(V, self.vol_shape, "V"), _stream(stream)), "prop_adjoint")
        return V

    def reconstruct(self, y: torch.Tensor, params: ReconParams, V: torch.Tensor = None, trace=True,
                    stream=None):
        """Run params.iters Adam iterations in place on V (zeros if None).

        Returns (V, loss_trace numpy array or None)."""
        if V is None:
            V = torch.zeros(self.vol_shape, dtype=torch.complex64, device=y.device)
        tr = np.zeros(max(params.iters, 1), dtype=np.float64) if trace else None
        tr_ptr = tr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if trace else None
        pc = params.c()
        check(lib().prop_reconstruct(self.handle, _dev_ptr(y, self.data_shape, "y"), ctypes.byref(pc),
                                     _dev_ptr(V, self.vol_shape, "V"), tr_ptr, _stream(stream)),
              "prop_reconstruct")
        return V, (tr[:params.iters] if trace else None)

    def recon_step(self, y: torch.Tensor, params: ReconParams, k: int, V_in: torch.Tensor, V_out: torch.Tensor,
                   loss: torch.Tensor = None, stream=None) -> torch.Tensor:
        """One Adam iteration k (1-based) from V_in into V_out; loss (float64 CUDA scalar) gets L(V_in)."""
        lp = None
        if loss is not None:
            if not loss.is_cuda or loss.dtype != torch.float64 or loss.numel() < 1:
                raise TypeError("loss must be a float64 CUDA tensor")
            lp = ctypes.c_void_p(loss.data_ptr())
        pc = params.c()
        check(lib().prop_recon_step(self.handle, _dev_ptr(y, self.data_shape, "y"), ctypes.byref(pc), int(k),
                                    _dev_ptr(V_in, self.vol_shape, "V_in"), _dev_ptr(V_out, self.vol_shape, "V_out"),
                                    lp, _stream(stream)), "prop_recon_step")
        return V_out

    def shard_forward(self, V: torch.Tensor, y_part: torch.Tensor = None, reuse_rows: bool = False,
                      accumulate: bool = False, stream=None) -> torch.Tensor:
        """A_g V over this plan's bins (one shard of a bin-sharded iteration); accumulate adds it to y_part."""
        if y_part is None:
            if accumulate:
                raise ValueError("accumulate needs y_part")
            y_part = torch.empty(self.data_shape, dtype=torch.complex64, device=V.device)
        flags = (1 if reuse_rows else 0) | (2 if accumulate else 0)
        check(lib().prop_shard_forward(self.handle, _dev_ptr(V, self.vol_shape, "V"), flags,
                                       _dev_ptr(y_part, self.data_shape, "y_part"), _stream(stream)),
              "prop_shard_forward")
        return y_part

    def shard_update(self, y: torch.Tensor, y_sum: torch.Tensor, params: ReconParams, k: int, V_in: torch.Tensor,
                     V_out: torch.Tensor, loss_parts: torch.Tensor = None, stream=None) -> torch.Tensor:
        """Residual, adjoint, TV and Adam of iteration k on this plan's bins, given the summed forward y_sum.
        loss_parts (float64 CUDA tensor of 2): [data term, this plan's TV]."""
        lp = None
        if loss_parts is not None:
            if not loss_parts.is_cuda or loss_parts.dtype != torch.float64 or loss_parts.numel() < 2:
                raise TypeError("loss_parts must be a float64 CUDA tensor of 2 elements")
            lp = ctypes.c_void_p(loss_parts.data_ptr())
        pc = params.c()
        check(lib().prop_shard_update(self.handle, _dev_ptr(y, self.data_shape, "y"),
                                      _dev_ptr(y_sum, self.data_shape, "y_sum"), ctypes.byref(pc), int(k),
                                      _dev_ptr(V_in, self.vol_shape, "V_in"), _dev_ptr(V_out, self.vol_shape, "V_out"),
                                      lp, _stream(stream)), "prop_shard_update")
        return V_out

    def reconstruct_host(self, y: np.ndarray, params: ReconParams, V: np.ndarray = None, trace=False,
                         stream=None):
        """Host-buffer reconstruction (copies in, iterates, copies out). V is updated in place."""
        if V is None:
            V = np.zeros(self.vol_shape, dtype=np.complex64)
        for a, shp, name in ((y, self.data_shape, "y"), (V, self.vol_shape, "V")):
            if not (isinstance(a, (np.ndarray, torch.Tensor))):
                raise TypeError(f"{name} must be a numpy array or a CPU tensor")
        yp = _host_ptr(y, self.data_shape, "y")
        vp = _host_ptr(V, self.vol_shape, "V")
        tr = np.zeros(max(params.iters, 1), dtype=np.float64) if trace else None
        tr_ptr = tr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if trace else None
        pc = params.c()
        check(lib().prop_reconstruct_host(self.handle, yp, ctypes.byref(pc), vp, tr_ptr, _stream(stream)),
              "prop_reconstruct_host")
        return V, (tr[:params.iters] if trace else None)

    def loss_grad(self, y: torch.Tensor, params: ReconParams, V: torch.Tensor, grad: torch.Tensor = None,
                  stream=None):
        """(L(V), dL/dRe V + i dL/dIm V)."""
        if grad is None:
            grad = torch.empty(self.vol_shape, dtype=torch.complex64, device=V.device)
        loss = ctypes.c_double()
        pc = params.c()
        check(lib().prop_loss_grad(self.handle, _dev_ptr(y, self.data_shape, "y"), ctypes.byref(pc),
                                   _dev_ptr(V, self.vol_shape, "V"), _dev_ptr(grad, self.vol_shape, "grad"),
                                   ctypes.byref(loss), _stream(stream)), "prop_loss_grad")
        return float(loss.value), grad

    def render(self, V: torch.Tensor, f_lo: int = 0, f_hi: int = None, out: torch.Tensor = None,
               stream=None) -> torch.Tensor:
        if f_hi is None:
            f_hi = self.Nf
        if out is None:
            out = torch.empty((self.T, self.N, self.N), dtype=torch.complex64, device=V.device)
        check(lib().prop_render(self.handle, _dev_ptr(V, self.vol_shape, "V"), int(f_lo), int(f_hi),
                                _dev_ptr(out, (self.T, self.N, self.N), "image"), _stream(stream)),
              "prop_render")
        return out


    def psnr(self, image: torch.Tensor, ref: torch.Tensor, stream=None) -> float:
        """PSNR (dB) of |image| against |ref|, peak max|ref|: images [frames, N, N] complex64."""
        if image.dim() == 2:
            image, ref = image.unsqueeze(0), ref.unsqueeze(0)
        fr = int(image.shape[0])
        shp = (fr, self.N, self.N)
        out = ctypes.c_double()
        check(lib().prop_psnr(self.handle, _dev_ptr(image, shp, "image"), _dev_ptr(ref, shp, "ref"), fr,
                              ctypes.byref(out), _stream(stream)), "prop_psnr")
        return float(out.value)

    @property
    def kspace_shape(self):
        return (self.N, self.N)

    def proj_forward(self, blade: int, V: torch.Tensor, z: torch.Tensor = None, stream=None) -> torch.Tensor:
        """Masked Cartesian k-space of one blade under the projection model."""
        if z is None:
            z = torch.empty(self.kspace_shape, dtype=torch.complex64, device=V.device)
        check(lib().prop_proj_forward(self.handle, int(blade), _dev_ptr(V, self.vol_shape, "V"),
                                      _dev_ptr(z, self.kspace_shape, "z"), _stream(stream)), "prop_proj_forward")
        return z

    def proj_adjoint(self, blade: int, z: torch.Tensor, V: torch.Tensor = None, stream=None) -> torch.Tensor:
        if V is None:
            V = torch.empty(self.vol_shape, dtype=torch.complex64, device=z.device)
        check(lib().prop_proj_adjoint(self.handle, int(blade), _dev_ptr(z, self.kspace_shape, "z"),
                                      _dev_ptr(V, self.vol_shape, "V"), _stream(stream)), "prop_proj_adjoint")
        return V

    def proj_reconstruct(self, ycart: torch.Tensor, params: "ProjParams", img: torch.Tensor = None,
                         V: torch.Tensor = None, trace=True, stream=None):
        """Adam over the blades in turn under the projection model, in place on V (zeros if None).

        Returns (V, loss_trace numpy array or None)."""
        if V is None:
            V = torch.zeros(self.vol_shape, dtype=torch.complex64, device=ycart.device)
        shp = (self.B, self.N, self.N)
        ip = _dev_ptr(img, shp, "img") if img is not None else None
        tr = np.zeros(max(params.iters, 1), dtype=np.float64) if trace else None
        tr_ptr = tr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if trace else None
        pc = params.c()
        check(lib().prop_proj_reconstruct(self.handle, _dev_ptr(ycart, shp, "ycart"), ip, ctypes.byref(pc),
                                          _dev_ptr(V, self.vol_shape, "V"), tr_ptr, _stream(stream)),
              "prop_proj_reconstruct")
        return V, (tr[:params.iters] if trace else None)

    def proj_baseline(self, ycart: torch.Tensor, blade_lo: int = 0, blade_hi: int = None,
                      out: torch.Tensor = None, stream=None) -> torch.Tensor:
        """Coverage-weighted k-space average of blades [blade_lo, blade_hi), inverse DFT: [N, N]."""
        if blade_hi is None:
            blade_hi = self.B
        if out is None:
            out = torch.empty((self.N, self.N), dtype=torch.complex64, device=ycart.device)
        check(lib().prop_proj_baseline(self.handle, _dev_ptr(ycart, (self.B, self.N, self.N), "ycart"),
                                       int(blade_lo), int(blade_hi), _dev_ptr(out, (self.N, self.N), "image"),
                                       _stream(stream)), "prop_proj_baseline")
        return out

    def kplanes_param_count(self, features: int = 8, scales: int = 2) -> int:
        n = ctypes.c_size_t()
        check(lib().prop_kplanes_param_count(self.handle, int(features), int(scales), ctypes.byref(n)),
              "prop_kplanes_param_count")
        return int(n.value)

    def _kp_ptr(self, t: torch.Tensor, features: int, scales: int, name: str) -> ctypes.c_void_p:
        return _dev_ptr(t, (self.kplanes_param_count(features, scales),), name)

    def kplanes_render(self, params: torch.Tensor, features: int = 8, scales: int = 2, V: torch.Tensor = None,
                       stream=None) -> torch.Tensor:
        """Render the K-Planes model (flat complex64 parameter tensor) on the volume grid."""
        if V is None:
            V = torch.empty(self.vol_shape, dtype=torch.complex64, device=params.device)
        check(lib().prop_kplanes_render(self.handle, int(features), int(scales),
                                        self._kp_ptr(params, features, scales, "params"),
                                        _dev_ptr(V, self.vol_shape, "V"), _stream(stream)), "prop_kplanes_render")
        return V

    def kplanes_vjp(self, params: torch.Tensor, gV: torch.Tensor, features: int = 8, scales: int = 2,
                    grad: torch.Tensor = None, stream=None) -> torch.Tensor:
        if grad is None:
            grad = torch.empty_like(params)
        check(lib().prop_kplanes_vjp(self.handle, int(features), int(scales),
                                     self._kp_ptr(params, features, scales, "params"),
                                     _dev_ptr(gV, self.vol_shape, "gV"),
                                     self._kp_ptr(grad, features, scales, "grad"), _stream(stream)),
              "prop_kplanes_vjp")
        return grad

    def kplanes_reconstruct(self, y: torch.Tensor, params: ReconParams, kp: torch.Tensor, features: int = 8,
                            scales: int = 2, stream=None):
        """Adam on the K-Planes parameters kp (in place); returns (kp, loss_trace)."""
        tr = np.zeros(max(params.iters, 1), dtype=np.float64)
        pc = params.c()
        check(lib().prop_kplanes_reconstruct(self.handle, _dev_ptr(y, self.data_shape, "y"), ctypes.byref(pc),
                                             int(features), int(scales), self._kp_ptr(kp, features, scales, "kp"),
                                             tr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _stream(stream)),
              "prop_kplanes_reconstruct")
        return kp, tr[:params.iters]

    def profile_enable(self, on: bool = True) -> None:
        check(lib().prop_profile_enable(self.handle, 1 if on else 0), "prop_profile_enable")

    def profile_read(self) -> dict:
        """{stage name: (total ms, launches)} since the last read (synchronises)."""
        from ._lib import PROP_NUM_STAGES, STAGE_NAMES
        ms = (ctypes.c_double * PROP_NUM_STAGES)()
        n = (ctypes.c_longlong * PROP_NUM_STAGES)()
        check(lib().prop_profile_read(self.handle, ms, n), "prop_profile_read")
        return {STAGE_NAMES[i]: (float(ms[i]), int(n[i])) for i in range(PROP_NUM_STAGES)}


def _host_ptr(a, shape, name) -> ctypes.c_void_p:
    if isinstance(a, torch.Tensor):
        if a.is_cuda or a.dtype != torch.complex64 or not a.is_contiguous() or tuple(a.shape) != tuple(shape):
            raise ValueError(f"{name}: need a contiguous CPU complex64 tensor of shape {shape}")
        return ctypes.c_void_p(a.data_ptr())
    if a.dtype != np.complex64 or not a.flags.c_contiguous or tuple(a.shape) != tuple(shape):
        raise ValueError(f"{name}: need a C-contiguous complex64 array of shape {shape}")
    return ctypes.c_void_p(a.ctypes.data)


# Function-style aliases with the C ABI's names.
def prop_plan_create(N, L, R, theta, delta, blade_frame=None, T=1, bin_chunk=0, device=None, kb_width=0,
                     row_kernel=0) -> Plan:
    return Plan(N, L, R, theta, delta, blade_frame, T, bin_chunk, device, kb_width, row_kernel)


def prop_plan_destroy(plan: Plan) -> None:
    plan.destroy()


def prop_plan_workspace_bytes(plan: Plan) -> int:
    return plan.workspace_bytes()


def prop_forward(plan: Plan, V, y=None, stream=None):
    return plan.forward(V, y, stream)


def prop_adjoint(plan: Plan, y, V=None, stream=None):
    return plan.adjoint(y, V, stream)


def prop_reconstruct(plan: Plan, y, params, V=None, trace=True, stream=None):
    return plan.reconstruct(y, params, V, trace, stream)


def prop_reconstruct_host(plan: Plan, y, params, V=None, trace=False, stream=None):
    return plan.reconstruct_host(y, params, V, trace, stream)


def prop_loss_grad(plan: Plan, y, params, V, grad=None, stream=None):
    return plan.loss_grad(y, params, V, grad, stream)


def prop_render(plan: Plan, V, f_lo=0, f_hi=None, out=None, stream=None):
    return plan.render(V, f_lo, f_hi, out, stream)


def prop_psnr(plan: Plan, image, ref, stream=None) -> float:
    return plan.psnr(image, ref, stream)


def prop_reconstruct_batch(plans, ys, params, Vs=None, trace=True, stream=None):
    """prop_reconstruct for several plans of one kernel class at once (shared launches).

    plans: Plan objects (same 2N, bin stride, kernel width); ys: their y tensors; params: one
    ReconParams each; Vs: start volumes (updated in place; zeros if None).  Returns (Vs, traces)."""
    n = len(plans)
    if not (len(ys) == n and len(params) == n):
        raise ValueError("plans, ys and params must have the same length")
    if Vs is None:
        Vs = [torch.zeros(p.vol_shape, dtype=torch.complex64, device=y.device) for p, y in zip(plans, ys)]
    ptrs = ctypes.c_void_p * n
    hs = ptrs(*[p.handle.value for p in plans])
    yp = ptrs(*[_dev_ptr(y, p.data_shape, "y").value for p, y in zip(plans, ys)])
    vp = ptrs(*[_dev_ptr(V, p.vol_shape, "V").value for p, V in zip(plans, Vs)])
    pcs = (ReconParamsC * n)(*[q.c() for q in params])
    traces = [np.zeros(max(q.iters, 1), dtype=np.float64) for q in params] if trace else None
    tp = None
    if trace:
        tp = (ctypes.POINTER(ctypes.c_double) * n)(*[t.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
                                                     for t in traces])
    check(lib().prop_reconstruct_batch(hs, n, yp, pcs, vp, tp, _stream(stream)), "prop_reconstruct_batch")
    return Vs, ([t[:q.iters] for t, q in zip(traces, params)] if trace else None)


def prop_tv_grad_static(V: torch.Tensor, tv_xy: float, tv_t: float, tv_eps: float, grad: torch.Tensor,
                        loss: torch.Tensor, stream=None) -> None:
    """Allocation-free TV value and gradient (no plan; scratch in a static device array).

    V, grad: complex64 CUDA tensors [T, N, N, Nf]; loss: float64 CUDA tensor with one element.
    Writes grad = tv_xy grad TV_xy + tv_t grad TV_t and loss = tv_xy TV_xy + tv_t TV_t.
    The output tensors are supplied by the caller; the call itself allocates nothing.
    """
    if V.dim() != 4:
        raise ValueError("V must be [T, N, N, Nf]")
    T, N, N2, Nf = (int(x) for x in V.shape)
    if N2 != N:
        raise ValueError("V must be [T, N, N, Nf]")
    if not loss.is_cuda or loss.dtype != torch.float64 or loss.numel() < 1:
        raise TypeError("loss must be a float64 CUDA tensor")
    check(lib().prop_tv_grad_static(_dev_ptr(V, (T, N, N, Nf), "V"), T, N, Nf, float(tv_xy), float(tv_t),
                                    float(tv_eps), _dev_ptr(grad, (T, N, N, Nf), "grad"),
                                    ctypes.c_void_p(loss.data_ptr()), _stream(stream)), "prop_tv_grad_static")


def prop_fp32_fma_peak(device: int = None) -> float:
    """Measured FP32 FMA throughput of the device, TFLOP/s (synchronous)."""
    if device is None:
        device = torch.cuda.current_device()
    out = ctypes.c_double()
    check(lib().prop_fp32_fma_peak(int(device), ctypes.byref(out)), "prop_fp32_fma_peak")
    return float(out.value)


def prop_check_bounded_wait(limit_cycles: int = 20_000_000, device: int = None):
    """Runs the bounded-wait probe; returns (expired, milliseconds)."""
    if device is None:
        device = torch.cuda.current_device()
    expired = ctypes.c_int()
    ms = ctypes.c_double()
    check(lib().prop_check_bounded_wait(int(device), int(limit_cycles), ctypes.byref(expired), ctypes.byref(ms)),
          "prop_check_bounded_wait")
    return int(expired.value), float(ms.value)
