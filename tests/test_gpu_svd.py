"""Block SVD (one grouped one-sided Jacobi launch over the coupled sectors) and its truncation
against the oracle."""

import numpy as np
import pytest

from harness import oracle_heff, ostruct
from oracle import ops
from paper_2508_10076_gb300 import build_library
from paper_2508_10076_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gctx():
    assert torch.cuda.is_available()
    build_library()
    from paper_2508_10076_gb300 import api
    ctx = api.Context(0)
    yield ctx
    ctx.sync()


def _tm(ctx, sym, legs):
    cod, dom = legs
    return ctx.tmap([ctx.space(sym, s, d) for s, d in cod], [ctx.space(sym, s, d) for s, d in dom])


@pytest.mark.parametrize("sym,D,dtype", [("SU2", 256, "f64"), ("U1", 1024, "f64"), ("U1", 256, "c128")])
def test_block_svd_and_truncation(gctx, sym, D, dtype):
    """The two-site tensor x' of one heff application (FP64 oracle): singular values against the
    oracle's block SVD, U S V^dagger against x', U with orthonormal columns, and the truncation
    to a bond dimension copying the leading triplets exactly."""
    from paper_2508_10076_gb300 import api
    V, P, W = wl.heff_spaces(sym, D)
    legs = wl.heff_legs(V, P, W)["x"]
    ost = ostruct(sym, legs)
    if dtype == "c128":
        x = wl.normal_complex(41, ost.numel)
    else:
        x = oracle_heff(sym, D, seed=5, tier="block")[-1][1]
    tdt = torch.complex128 if dtype == "c128" else torch.float64
    plan = api.svd_plan(gctx, _tm(gctx, sym, legs), dtype=dtype)
    us, vs, n = plan.outputs()
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    u = torch.empty(us.numel, dtype=tdt, device="cuda")
    vh = torch.empty(vs.numel, dtype=tdt, device="cuda")
    s = torch.empty(n, dtype=torch.float64, device="cuda")
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    api.svd(gctx, plan, xd, u, s, vh, ws)
    gctx.sync()
    ref = ops.svd_block(ost, x)
    blocks = plan.blocks()
    assert [b[0] for b in blocks] == [c for c, _, _, _ in ref]
    hs, hu, hv = s.cpu().numpy(), u.cpu().numpy(), vh.cpu().numpy()
    ub, vb = dict((c, (r, k, o)) for c, r, k, o in us.blocks()), dict((c, (r, k, o)) for c, r, k, o in vs.blocks())
    top = max(float(sv[0]) for _, _, sv, _ in ref)
    for (c, m, nn, so), (_, _, sv, _) in zip(blocks, ref):
        r = min(m, nn)
        assert np.allclose(hs[so:so + r], sv, atol=1e-12 * top)
        ur, uk, uo = ub[c]
        vr, vk, vo = vb[c]
        umat = hu[uo:uo + ur * uk].reshape(uk, ur).T
        vmat = hv[vo:vo + vr * vk].reshape(vk, vr).T
        rec = (umat * hs[so:so + r]) @ vmat
        r0, k0, o0 = dict((cc, (rr, kk, oo)) for cc, rr, kk, oo in ost.blocks)[c]
        blk = x[o0:o0 + r0 * k0].reshape(k0, r0).T
        assert np.allclose(rec, blk, atol=1e-12 * top)
        assert np.allclose(umat.conj().T @ umat, np.eye(r), atol=1e-12)
    # truncation: oracle rule on the oracle's values, then device copies of the leading triplets
    keep, err = ops.truncation_keep(ost, [(c, sv) for c, _, sv, _ in ref], dmax=max(4, ost.sym.dim(0) * n // 3))
    assert 0 <= err < 1
    kept = {c: k for (c, _, _, _), k in zip(blocks, keep) if k > 0}
    w2 = gctx.space(sym, kept, False)
    ut_s = gctx.tmap([gctx.space(sym, sp, d) for sp, d in legs[0]], [w2])
    vt_s = gctx.tmap([w2], [gctx.space(sym, sp, d) for sp, d in legs[1]])
    ut = torch.empty(ut_s.numel, dtype=tdt, device="cuda")
    vt = torch.empty(vt_s.numel, dtype=tdt, device="cuda")
    st = torch.empty(sum(keep), dtype=torch.float64, device="cuda")
    api.svd_truncate(gctx, plan, keep, u, s, vh, ut, st, vt)
    gctx.sync()
    hut, hst, hvt = ut.cpu().numpy(), st.cpu().numpy(), vt.cpu().numpy()
    utb = dict((c, (r, k, o)) for c, r, k, o in ut_s.blocks())
    vtb = dict((c, (r, k, o)) for c, r, k, o in vt_s.blocks())
    so2 = 0
    for (c, m, nn, so), k in zip(blocks, keep):
        if k == 0:
            continue
        ur, uk, uo = ub[c]
        r2, k2, o2 = utb[c]
        assert (r2, k2) == (ur, k)
        assert np.array_equal(hut[o2:o2 + r2 * k2], hu[uo:uo + ur * k])  # leading columns
        assert np.array_equal(hst[so2:so2 + k], hs[so:so + k])
        vr, vk, vo = vb[c]
        r3, k3, o3 = vtb[c]
        assert np.array_equal(hvt[o3:o3 + r3 * k3].reshape(k3, r3), hv[vo:vo + vr * vk].reshape(vk, vr)[:, :k])
        so2 += k


@pytest.mark.parametrize("sym,D,wide,dtype", [("U1", 256, False, "f64"), ("U1", 256, True, "c128"),
                                              ("SU2", 96, False, "c128"), ("SU2", 96, True, "f64")])
def test_block_svd_rectangular_blocks(gctx, sym, D, wide, dtype):
    """An MPS tensor V (x) P <- V has blocks with about twice as many rows as columns, its adjoint
    V <- V (x) P the transpose shape: both Jacobi orientations against the oracle's block SVD
    (values), with U^dagger U = 1, V^dagger rows orthonormal and U S V^dagger = t."""
    from paper_2508_10076_gb300 import api
    V, P, W = wl.heff_spaces(sym, D)
    legs = ([(V, False)], [(V, False), (P, False)]) if wide else ([(V, False), (P, False)], [(V, False)])
    ost = ostruct(sym, legs)
    x = wl.normal_complex(7, ost.numel) if dtype == "c128" else wl.normal(7, ost.numel)
    tdt = torch.complex128 if dtype == "c128" else torch.float64
    plan = api.svd_plan(gctx, _tm(gctx, sym, legs), dtype=dtype)
    us, vs, n = plan.outputs()
    u = torch.full((us.numel,), float("nan"), dtype=tdt, device="cuda")
    vh = torch.full((vs.numel,), float("nan"), dtype=tdt, device="cuda")
    s = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    api.svd(gctx, plan, torch.from_numpy(np.ascontiguousarray(x)).cuda(), u, s, vh, ws)
    gctx.sync()
    ref = dict((c, sv) for c, _, sv, _ in ops.svd_block(ost, x))
    hs, hu, hv = s.cpu().numpy(), u.cpu().numpy(), vh.cpu().numpy()
    ub, vb = dict((c, (r, k, o)) for c, r, k, o in us.blocks()), dict((c, (r, k, o)) for c, r, k, o in vs.blocks())
    top = max(float(v[0]) for v in ref.values())
    ob = dict((cc, (rr, kk, oo)) for cc, rr, kk, oo in ost.blocks)
    shapes = set()
    for c, m, nn, so in plan.blocks():
        r = min(m, nn)
        shapes.add(m > nn)
        assert np.allclose(hs[so:so + r], ref[c], atol=1e-12 * top, rtol=0)
        assert np.all(np.diff(hs[so:so + r]) <= 0)
        ur, uk, uo = ub[c]
        vr, vk, vo = vb[c]
        umat = hu[uo:uo + ur * uk].reshape(uk, ur).T
        vmat = hv[vo:vo + vr * vk].reshape(vk, vr).T
        assert np.allclose(umat.conj().T @ umat, np.eye(r), atol=1e-12)
        assert np.allclose(vmat @ vmat.conj().T, np.eye(r), atol=1e-12)
        r0, k0, o0 = ob[c]
        assert np.allclose((umat * hs[so:so + r]) @ vmat, x[o0:o0 + r0 * k0].reshape(k0, r0).T, atol=1e-12 * top)
    assert (not wide) in shapes  # the orientation this case is about occurs
