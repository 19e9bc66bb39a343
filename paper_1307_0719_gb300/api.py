"""Python face of the C ABI (include/taylens.h). Argument marshalling only: every
step of the lensing path runs in libtaylens.so on the GPU."""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import check

FP64 = _lib.TL_FP64
MIXED_FP32 = _lib.TL_MIXED_FP32
MIXED_TF32 = _lib.TL_MIXED_TF32
MIXED_TF32x3 = _lib.TL_MIXED_TF32x3
MIXED_BF16x3 = _lib.TL_MIXED_BF16x3


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _alm(t, name):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype == torch.complex128:
        t = torch.view_as_real(t)
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous complex128 (or float64 [..., 2])")
    return t


class Plan:
    """A (nside, lmax, order) geometry with its device tables and workspace."""

    def __init__(self, nside: int, lmax: int, order: int, pol: bool = True,
                 precision: int = FP64, rotate: bool = True, naive: bool = False, expand_at_pixel: bool = False,
                 lmax_phi: int | None = None):
        L = _lib.lib()
        self.nside, self.lmax, self.order, self.pol, self.precision = nside, lmax, order, pol, precision
        self.npix = 12 * nside * nside
        self.nalm = (lmax + 1) * (lmax + 2) // 2
        self.dtype = torch.float64 if precision == FP64 else torch.float32
        spins = _lib.TL_SPIN_T | (_lib.TL_SPIN_QU if pol else 0)
        flags = ((_lib.TL_ROTATE if rotate else 0) | (_lib.TL_NAIVE if naive else 0) |
                 (_lib.TL_EXPAND_AT_PIXEL if expand_at_pixel else 0))
        h = ctypes.c_void_p()
        check(L.tl_plan_create(nside, lmax, order, spins, precision, flags, ctypes.byref(h)),
              "tl_plan_create")
        self._h = h
        self.nmaps = L.tl_plan_maps_per_field(h)
        self.batch = L.tl_plan_batch(h)  # realisations per Legendre launch in lens_batch
        self.lmax_phi = lmax
        if lmax_phi is not None and lmax_phi != lmax:
            self.set_lmax_phi(lmax_phi)

    def set_lmax_phi(self, lmax_phi: int):
        """tl_plan_set_lmax_phi: the potential's own band limit (its coefficients then
        come in that layout)."""
        check(_lib.lib().tl_plan_set_lmax_phi(self._h, lmax_phi), "tl_plan_set_lmax_phi")
        self.lmax_phi = lmax_phi

    def batch_launches(self, nreal, with_phi=True):
        """Kernel launches lens_batch makes for nreal realisations."""
        return int(_lib.lib().tl_plan_batch_launches(self._h, int(nreal), 1 if with_phi else 0))

    def close(self):
        if getattr(self, "_h", None):
            _lib.lib().tl_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check_device_error(self):
        """Raise TaylensError if a kernel of this plan timed out a bounded wait (synchronises)."""
        check(_lib.lib().tl_plan_device_error(self._h), "device-side wait")

    @property
    def workspace_bytes(self) -> int:
        return _lib.lib().tl_plan_workspace_bytes(self._h)

    def synth_derivs(self, alm, spin: int = 0, out=None, stream=None):
        """[K, Npix] maps d_theta^j d_phi^k of the field (spin 0: T; spin 2: alm = [E, B]
        stacked, output Q maps then U maps)."""
        a = _alm(alm, "alm")
        K = self.nmaps * (2 if spin == 2 else 1)
        if out is None:
            out = torch.empty((K, self.npix), dtype=self.dtype, device=a.device)
        check(_lib.lib().tl_synth_derivs(self._h, _ptr(a), spin, _ptr(out), _stream(stream)),
              "tl_synth_derivs")
        return out

    def deflection(self, alm_phi, stream=None):
        a = _alm(alm_phi, "alm_phi")
        out = torch.empty((2, self.npix), dtype=self.dtype, device=a.device)
        check(_lib.lib().tl_deflection(self._h, _ptr(a), _ptr(out[0]), _ptr(out[1]), _stream(stream)),
              "tl_deflection")
        return out

    def lens(self, alm_T, alm_E=None, alm_B=None, alm_phi=None, out=None, stream=None):
        """Lensed (T, Q, U) maps (Q, U None for T-only plans)."""
        aT, aE, aB, aP = (_alm(alm_T, "alm_T"), _alm(alm_E, "alm_E"), _alm(alm_B, "alm_B"),
                          _alm(alm_phi, "alm_phi"))
        nf = 3 if self.pol else 1
        if out is None:
            out = torch.empty((nf, self.npix), dtype=self.dtype, device=aT.device)
        Q = out[1] if self.pol else None
        U = out[2] if self.pol else None
        check(_lib.lib().tl_lens(self._h, _ptr(aT), _ptr(aE), _ptr(aB), _ptr(aP), _ptr(out[0]),
                                 _ptr(Q), _ptr(U), _stream(stream)), "tl_lens")
        return out

    def lens_batch(self, skies, outs=None, stream=None):
        """Lens several realisations with one call (tl_lens_batch). `skies` is a list of
        dicts with keys T, E, B, phi (CUDA complex128); returns a list of [3 or 1, Npix]."""
        n = len(skies)
        nf = 3 if self.pol else 1
        dev = skies[0]["T"].device
        if outs is None:
            outs = [torch.empty((nf, self.npix), dtype=self.dtype, device=dev) for _ in range(n)]
        arr = lambda xs: (ctypes.c_void_p * n)(*[None if x is None else x.data_ptr() for x in xs])
        keep = [{k: _alm(sk.get(k), k) for k in ("T", "E", "B", "phi")} for sk in skies]
        aT = arr([k["T"] for k in keep])
        aE = arr([k["E"] for k in keep]) if self.pol else None
        aB = arr([k["B"] for k in keep]) if self.pol else None
        aP = arr([k["phi"] for k in keep])
        To = arr([o[0] for o in outs])
        Qo = arr([o[1] for o in outs]) if self.pol else None
        Uo = arr([o[2] for o in outs]) if self.pol else None
        check(_lib.lib().tl_lens_batch(self._h, n, aT, aE, aB, aP, To, Qo, Uo, _stream(stream)),
              "tl_lens_batch")
        return outs

    def lens_host(self, alm_T, alm_E=None, alm_B=None, alm_phi=None, out=None, stream=None):
        """tl_lens_host: alm in (pinned) host memory, maps returned in host memory."""
        def h(t):
            if t is None:
                return None
            if t.dtype == torch.complex128:
                t = torch.view_as_real(t)
            assert not t.is_cuda and t.is_contiguous()
            return t
        nf = 3 if self.pol else 1
        if out is None:
            out = torch.empty((nf, self.npix), dtype=self.dtype, pin_memory=True)
        Q = out[1] if self.pol else None
        U = out[2] if self.pol else None
        check(_lib.lib().tl_lens_host(self._h, _ptr(h(alm_T)), _ptr(h(alm_E)), _ptr(h(alm_B)),
                                      _ptr(h(alm_phi)), _ptr(out[0]), _ptr(Q), _ptr(U),
                                      _stream(stream)), "tl_lens_host")
        return out

    def lens_batch_host(self, skies, outs=None, stream=None):
        """tl_lens_batch_host: several realisations from (pinned) host memory, maps back
        in host memory. `skies`: list of dicts T, E, B, phi (CPU complex128 tensors);
        returns a list of CPU [3 or 1, Npix] tensors of the plan's map dtype."""
        n = len(skies)
        nf = 3 if self.pol else 1

        def h(t):
            if t is None:
                return None
            if t.dtype == torch.complex128:
                t = torch.view_as_real(t)
            if t.is_cuda or not t.is_contiguous() or t.dtype != torch.float64:
                raise ValueError("host coefficients must be contiguous CPU complex128 tensors")
            return t
        if outs is None:
            outs = [torch.empty((nf, self.npix), dtype=self.dtype, pin_memory=True) for _ in range(n)]
        for o in outs:
            if o.is_cuda or o.dtype != self.dtype or not o.is_contiguous():
                raise ValueError("host outputs must be contiguous CPU tensors of the plan's dtype")
        arr = lambda xs: (ctypes.c_void_p * n)(*[None if x is None else x.data_ptr() for x in xs])
        keep = [{k: h(sk.get(k)) for k in ("T", "E", "B", "phi")} for sk in skies]
        aT = arr([k["T"] for k in keep])
        aE = arr([k["E"] for k in keep]) if self.pol else None
        aB = arr([k["B"] for k in keep]) if self.pol else None
        aP = arr([k["phi"] for k in keep])
        To = arr([o[0] for o in outs])
        Qo = arr([o[1] for o in outs]) if self.pol else None
        Uo = arr([o[2] for o in outs]) if self.pol else None
        check(_lib.lib().tl_lens_batch_host(self._h, n, aT, aE, aB, aP, To, Qo, Uo, _stream(stream)),
              "tl_lens_batch_host")
        return outs

    def lens_adjoint(self, alm_T, alm_E, alm_B, alm_phi, gT, gQ=None, gU=None, want=("T", "E", "B", "phi"),
                     galpha=False, stream=None):
        """tl_lens_adjoint: gradients (complex128 [nalm], dL/dRe + i dL/dIm) of the fields
        named in `want` from the map gradients gT, gQ, gU (the plan's map dtype). Returns a
        dict; with galpha=True it also holds "alpha", the [2, Npix] deflection gradient."""
        aT, aE, aB, aP = (_alm(alm_T, "alm_T"), _alm(alm_E, "alm_E"), _alm(alm_B, "alm_B"),
                          _alm(alm_phi, "alm_phi"))
        dev = aT.device
        for name, g in (("gT", gT), ("gQ", gQ), ("gU", gU)):
            if g is not None and (g.dtype != self.dtype or not g.is_contiguous() or not g.is_cuda):
                raise ValueError(f"{name} must be a contiguous CUDA tensor of {self.dtype}")
        fields = [f for f in ("T", "E", "B", "phi") if f in want and (self.pol or f not in ("E", "B"))]
        out = {f: torch.empty(self.nalm, dtype=torch.complex128, device=dev) for f in fields}  # zeroed in the call
        ga = torch.empty((2, self.npix), dtype=self.dtype, device=dev) if galpha else None
        o = lambda f: _ptr(torch.view_as_real(out[f])) if f in out else None
        check(_lib.lib().tl_lens_adjoint(self._h, _ptr(aT), _ptr(aE), _ptr(aB), _ptr(aP), _ptr(gT),
                                         _ptr(gQ if self.pol else None), _ptr(gU if self.pol else None),
                                         o("T"), o("E"), o("B"), o("phi"), _ptr(ga), _stream(stream)),
              "tl_lens_adjoint")
        if galpha:
            out["alpha"] = ga
        return out

    def map2alm(self, T, Q=None, U=None, stream=None):
        """tl_map2alm: coefficients (complex128 [nalm]) of maps on this plan's geometry
        (the plan's map dtype, CUDA); returns dict T (and E, B when Q, U are given)."""
        for name, m in (("T", T), ("Q", Q), ("U", U)):
            if m is not None and (m.dtype != self.dtype or not m.is_cuda or not m.is_contiguous()):
                raise ValueError(f"{name} must be a contiguous CUDA tensor of {self.dtype}")
        dev = T.device
        out = {"T": torch.empty(self.nalm, dtype=torch.complex128, device=dev)}
        if Q is not None:
            out["E"] = torch.empty(self.nalm, dtype=torch.complex128, device=dev)
            out["B"] = torch.empty(self.nalm, dtype=torch.complex128, device=dev)
        o = lambda f: _ptr(torch.view_as_real(out[f])) if f in out else None
        check(_lib.lib().tl_map2alm(self._h, _ptr(T), _ptr(Q), _ptr(U), o("T"), o("E"), o("B"), _stream(stream)),
              "tl_map2alm")
        return out

    def last_stage_ms(self):
        buf = (ctypes.c_float * 16)()
        n = _lib.lib().tl_last_stage_ms(self._h, buf, 16)
        return list(buf[:n])


def anafast(lmax, alm_T=None, alm_E=None, alm_B=None, stream=None):
    """tl_anafast: [6, lmax+1] float64 CUDA tensor of C_l for TT, EE, BB, TE, TB, EB."""
    a = {k: _alm(v, k) for k, v in (("T", alm_T), ("E", alm_E), ("B", alm_B))}
    dev = next(v for v in a.values() if v is not None).device
    cl = torch.zeros((6, lmax + 1), dtype=torch.float64, device=dev)
    check(_lib.lib().tl_anafast(int(lmax), _ptr(a["T"]), _ptr(a["E"]), _ptr(a["B"]), _ptr(cl), _stream(stream)),
          "tl_anafast")
    return cl


def lens(nside, lmax, order, alm_T, alm_E=None, alm_B=None, alm_phi=None, precision=FP64,
         rotate=True):
    p = Plan(nside, lmax, order, pol=alm_E is not None, precision=precision, rotate=rotate)
    try:
        return p.lens(alm_T, alm_E, alm_B, alm_phi)
    finally:
        torch.cuda.synchronize()
        p.close()


def synth_derivs(nside, lmax, order, alm, spin=0, precision=FP64):
    p = Plan(nside, lmax, order, pol=(spin == 2), precision=precision)
    try:
        return p.synth_derivs(alm, spin)
    finally:
        torch.cuda.synchronize()
        p.close()


def deflection(nside, lmax, alm_phi, precision=FP64):
    p = Plan(nside, lmax, 1, pol=False, precision=precision)
    try:
        return p.deflection(alm_phi)
    finally:
        torch.cuda.synchronize()
        p.close()


class Batch:
    """Realisations of uneven geometry (tl_batch_*): grouped by (nside, lmax), each
    group with its own plan. `lens` modes: loop, persistent, graph. Default
    precision: the BF16x3 tensor-core contraction (MIXED_TF32x3 reaches the same
    error level with three MMAs per block instead of two)."""

    MODES = {"loop": _lib.TL_BATCH_LOOP, "persistent": _lib.TL_BATCH_PERSISTENT, "graph": _lib.TL_BATCH_GRAPH}

    def __init__(self, nsides, lmaxs, order, pol=True, precision=MIXED_BF16x3, rotate=True):
        L = _lib.lib()
        n = len(nsides)
        self.n, self.pol, self.precision = n, pol, precision
        self.nsides, self.lmaxs = list(nsides), list(lmaxs)
        self.dtype = torch.float64 if precision == FP64 else torch.float32
        ns = (ctypes.c_int * n)(*nsides)
        lm = (ctypes.c_int * n)(*lmaxs)
        spins = _lib.TL_SPIN_T | (_lib.TL_SPIN_QU if pol else 0)
        h = ctypes.c_void_p()
        check(L.tl_batch_create(n, ns, lm, order, spins, precision, _lib.TL_ROTATE if rotate else 0,
                                ctypes.byref(h)), "tl_batch_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib.lib().tl_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def groups(self):
        return _lib.lib().tl_batch_groups(self._h)

    @property
    def waves(self):
        return _lib.lib().tl_batch_waves(self._h)

    @property
    def grid(self):
        return _lib.lib().tl_batch_grid(self._h)

    def outputs(self, device="cuda"):
        nf = 3 if self.pol else 1
        return [torch.empty((nf, 12 * ns * ns), dtype=self.dtype, device=device) for ns in self.nsides]

    def _args(self, skies, outs):
        n = self.n
        arr = lambda xs: (ctypes.c_void_p * n)(*[None if x is None else x.data_ptr() for x in xs])
        self._keep = [{k: _alm(sk.get(k), k) for k in ("T", "E", "B", "phi")} for sk in skies]
        k = self._keep
        return (arr([x["T"] for x in k]), arr([x["E"] for x in k]) if self.pol else None,
                arr([x["B"] for x in k]) if self.pol else None, arr([x["phi"] for x in k]),
                arr([o[0] for o in outs]), arr([o[1] for o in outs]) if self.pol else None,
                arr([o[2] for o in outs]) if self.pol else None)

    def lens(self, skies, outs, mode="graph", stream=None):
        a = self._args(skies, outs)
        check(_lib.lib().tl_batch_lens(self._h, self.MODES[mode], *a, _stream(stream)), "tl_batch_lens")
        return outs

    def autotune(self, skies, outs, stream=None):
        a = self._args(skies, outs)
        check(_lib.lib().tl_batch_autotune(self._h, *a, _stream(stream)), "tl_batch_autotune")


class LensFunction(torch.autograd.Function):
    """Differentiable lensing: lensed maps [3 or 1, Npix] from complex128 coefficients.
    The backward pass is tl_lens_adjoint (the expansion pixels held fixed). Use as
    LensFunction.apply(plan, alm_T, alm_E, alm_B, alm_phi); alm_E/alm_B/alm_phi may be None."""

    @staticmethod
    def forward(ctx, plan, alm_T, alm_E, alm_B, alm_phi):
        ctx.plan = plan
        ctx.save_for_backward(alm_T, alm_E, alm_B, alm_phi)
        return plan.lens(alm_T.detach(), None if alm_E is None else alm_E.detach(),
                         None if alm_B is None else alm_B.detach(),
                         None if alm_phi is None else alm_phi.detach())

    @staticmethod
    def backward(ctx, gout):
        plan = ctx.plan
        alm_T, alm_E, alm_B, alm_phi = ctx.saved_tensors
        g = gout.to(plan.dtype).contiguous()
        want = []
        for name, t, i in (("T", alm_T, 1), ("E", alm_E, 2), ("B", alm_B, 3), ("phi", alm_phi, 4)):
            if t is not None and ctx.needs_input_grad[i]:
                want.append(name)
        res = plan.lens_adjoint(alm_T, alm_E, alm_B, alm_phi, g[0].contiguous(),
                                g[1].contiguous() if plan.pol else None,
                                g[2].contiguous() if plan.pol else None, want=tuple(want))
        return (None, res.get("T"), res.get("E"), res.get("B"), res.get("phi"))
