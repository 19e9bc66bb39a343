"""tl_map2alm and tl_anafast (Sec. III: the paper measures lensed maps through their
power spectra) against the oracle's direct sums, through the C ABI. Tolerances: FP64
within 1e-11 of the oracle (different summation order); the mixed forms read float
maps and run the float transposed recurrence, 1e-5."""
import numpy as np
import pytest
import torch

import oracle.healpix as hp
import oracle.lens as OL
from gpu_util import rel_rms, sky

pytestmark = pytest.mark.gpu

api = pytest.importorskip("paper_1307_0719_gb300.api")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _cmp(a, b):
    return rel_rms(np.concatenate([a.real, a.imag]), np.concatenate([b.real, b.imag]))


@pytest.mark.parametrize("precision,tol", [("FP64", 1e-11), ("MIXED_FP32", 1e-5), ("MIXED_BF16x3", 1e-5)])
@pytest.mark.parametrize("nside,lmax", [(16, 32), (32, 64), (8, 20)])
def test_map2alm_vs_oracle(nside, lmax, precision, tol):
    rng = np.random.default_rng(nside + lmax)
    maps = {f: rng.normal(size=hp.npix(nside)) for f in "TQU"}
    ref = OL.map2alm(nside, lmax, maps["T"], maps["Q"], maps["U"])
    plan = api.Plan(nside, lmax, 0, pol=True, precision=getattr(api, precision))
    try:
        dm = {f: torch.from_numpy(v).to("cuda:0", plan.dtype) for f, v in maps.items()}
        out = {k: v.cpu().numpy() for k, v in plan.map2alm(dm["T"], dm["Q"], dm["U"]).items()}
        t_only = plan.map2alm(dm["T"])["T"].cpu().numpy()
    finally:
        torch.cuda.synchronize()
        plan.close()
    if precision != "FP64":  # the oracle on the float-rounded maps
        ref = OL.map2alm(nside, lmax, *(np.asarray(v, np.float32).astype(np.float64) for v in
                                        (maps["T"], maps["Q"], maps["U"])))
    for f in "TEB":
        assert _cmp(out[f], ref[f]) < tol, (f, _cmp(out[f], ref[f]))
    assert _cmp(t_only, ref["T"]) < tol


def test_anafast_vs_oracle():
    lmax = 96
    s = sky(48, lmax, pol=True, b_scale=0.5)
    d = {k: torch.from_numpy(v).cuda() for k, v in s.items()}
    cl = api.anafast(lmax, d["T"], d["E"], d["B"]).cpu().numpy()
    pairs = [("T", "T"), ("E", "E"), ("B", "B"), ("T", "E"), ("T", "B"), ("E", "B")]
    for row, (x, y) in enumerate(pairs):
        ref = OL.anafast(lmax, s[x], s[y])
        assert np.allclose(cl[row], ref, rtol=1e-12, atol=1e-15 * np.abs(ref).max()), (x, y)
    cl_t = api.anafast(lmax, d["T"]).cpu().numpy()
    assert np.allclose(cl_t[0], cl[0], rtol=1e-14) and not cl_t[1:].any()


@pytest.mark.parametrize("nside,lmax", [(1024, 2048), (2048, 4096)])
def test_map2alm_transpose_identity_full_size(nside, lmax):
    """tl_map2alm is the transpose of the synthesis with weight 4 pi / Npix:
    sum c_m Re(a conj(map2alm(m))) = (4 pi / Npix) sum_p m(p) synth(a)(p), c_0 = 1,
    c_m>0 = 2, for T and (E, B) <-> (Q, U), at the sizes where the adjoint ring FFT runs
    its register Bluestein sub-transforms; single precision sums: 1e-4."""
    s = sky(nside, lmax, pol=True, b_scale=0.5)
    d = {k: torch.from_numpy(v).cuda() for k, v in s.items()}
    rng = np.random.default_rng(8)
    m = {f: torch.from_numpy(rng.normal(size=hp.npix(nside))).cuda().float() for f in "TQU"}
    plan = api.Plan(nside, lmax, 0, pol=True, precision=api.MIXED_FP32)
    try:
        syn_t = plan.synth_derivs(d["T"], 0)[0].double()
        syn_p = plan.synth_derivs(torch.cat([d["E"], d["B"]]), 2).double()
        b = plan.map2alm(m["T"], m["Q"], m["U"])
    finally:
        torch.cuda.synchronize()
        plan.close()
    w = 4 * np.pi / hp.npix(nside)
    c = torch.full((plan.nalm,), 2.0, dtype=torch.float64, device="cuda")
    c[:lmax + 1] = 1.0
    lhs_t = float((c * (d["T"] * b["T"].conj()).real).sum())
    rhs_t = w * float(torch.dot(m["T"].double(), syn_t))
    assert abs(lhs_t - rhs_t) < 1e-4 * abs(rhs_t), (lhs_t, rhs_t)
    lhs_p = float((c * ((d["E"] * b["E"].conj()).real + (d["B"] * b["B"].conj()).real)).sum())
    rhs_p = w * float(torch.dot(m["Q"].double(), syn_p[0]) + torch.dot(m["U"].double(), syn_p[1]))
    assert abs(lhs_p - rhs_p) < 1e-4 * abs(rhs_p), (lhs_p, rhs_p)
