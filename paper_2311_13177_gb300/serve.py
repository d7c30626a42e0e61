"""Python binding of the request server (prop_serve_* in the C ABI).

Argument marshalling only: the server, its scheduler, admission and all
device work live in libprop.
"""
from __future__ import annotations

import ctypes

import numpy as np

from ._lib import PlanDesc, ServeStats, check, lib, PropError
from .binding import ReconParams

REQ_STATES = {0: "pending", 1: "running", 2: "done", 3: "failed", 4: "cancelled"}


def plan_desc(N, L, R, theta, delta, blade_frame=None, T=1, kb_width=0, bin_chunk=0):
    """A PlanDesc plus the arrays it points to (keep both alive until the call returns)."""
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    delta = np.ascontiguousarray(delta, dtype=np.float64)
    keep = [theta, delta]
    bf = None
    if blade_frame is not None:
        frames = np.ascontiguousarray(blade_frame, dtype=np.int32)
        keep.append(frames)
        bf = frames.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    d = PlanDesc(int(N), len(delta), delta.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(theta),
                 theta.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(L), int(R), int(T), bf,
                 int(kb_width), int(bin_chunk), 0, 0)
    return d, keep


def prop_plan_estimate_bytes(N, L, R, theta, delta, blade_frame=None, T=1, iters=1, kb_width=0,
                             bin_chunk=0) -> int:
    d, keep = plan_desc(N, L, R, theta, delta, blade_frame, T, kb_width, bin_chunk)
    out = ctypes.c_size_t()
    check(lib().prop_plan_estimate_bytes(ctypes.byref(d), int(iters), ctypes.byref(out)),
          "prop_plan_estimate_bytes")
    return int(out.value)


class Server:
    """Continuous-batching reconstruction server on one device."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 8, device: int = 0):
        h = ctypes.c_void_p()
        check(lib().prop_serve_create(int(hbm_budget_bytes), int(max_slots), int(device), ctypes.byref(h)),
              "prop_serve_create")
        self._h = h
        self._shapes = {}

    def submit(self, N, L, R, theta, delta, y, params: ReconParams, blade_frame=None, T=1, v0=None,
               kb_width=0, bin_chunk=0) -> int:
        d, keep = plan_desc(N, L, R, theta, delta, blade_frame, T, kb_width, bin_chunk)
        y = np.ascontiguousarray(y, dtype=np.complex64)
        if y.size != len(keep[0]) * L * R:
            raise ValueError("y must hold B * L * R samples")
        vp = None
        if v0 is not None:
            v0 = np.ascontiguousarray(v0, dtype=np.complex64)
            if v0.size != T * N * N * len(keep[1]):
                raise ValueError("v0 must hold T * N * N * Nf values")
            vp = ctypes.c_void_p(v0.ctypes.data)
        t = ctypes.c_uint64()
        pc = params.c()
        check(lib().prop_serve_submit(self._h, ctypes.byref(d), ctypes.byref(pc), ctypes.c_void_p(y.ctypes.data),
                                      vp, ctypes.byref(t)), "prop_serve_submit")
        self._shapes[t.value] = (T, N, N, len(keep[1]))
        return int(t.value)

    def poll(self, ticket: int) -> str:
        st = ctypes.c_int()
        check(lib().prop_serve_poll(self._h, ctypes.c_uint64(ticket), ctypes.byref(st)), "prop_serve_poll")
        return REQ_STATES[st.value]

    def wait(self, ticket: int, timeout_ms: int = -1):
        """(volume [T, N, N, Nf] complex64, latency seconds, final loss)."""
        shape = self._shapes[ticket]
        out = np.empty(shape, dtype=np.complex64)
        lat = ctypes.c_double()
        loss = ctypes.c_double()
        check(lib().prop_serve_wait(self._h, ctypes.c_uint64(ticket), int(timeout_ms),
                                    ctypes.c_void_p(out.ctypes.data), ctypes.byref(lat), ctypes.byref(loss)),
              "prop_serve_wait")
        self._shapes.pop(ticket, None)
        return out, float(lat.value), float(loss.value)

    def cancel(self, ticket: int) -> None:
        check(lib().prop_serve_cancel(self._h, ctypes.c_uint64(ticket)), "prop_serve_cancel")

    def stats(self) -> dict:
        s = ServeStats()
        check(lib().prop_serve_stats(self._h, ctypes.byref(s)), "prop_serve_stats")
        return {k: getattr(s, k) for k, _ in ServeStats._fields_}

    def close(self) -> None:
        if getattr(self, "_h", None) is not None:
            check(lib().prop_serve_destroy(self._h), "prop_serve_destroy")
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


__all__ = ["Server", "prop_plan_estimate_bytes", "plan_desc", "PropError"]
