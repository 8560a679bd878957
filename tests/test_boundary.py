"""Host-side logic of the C ABI's context: budget admission (TK_ERR_BUDGET), reservations,
allocator-hook arguments, typed tensor-map I/O size checks, and the built-in scratch size.
Host-only contexts run no device code, so these run on the CPU."""

import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2508_10076_gb300 import api, build_library
from paper_2508_10076_gb300 import _abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TK_ERR_ARG, TK_ERR_NO_DEVICE, TK_ERR_BUDGET = 1, 10, 11


@pytest.fixture(scope="module")
def hctx():
    build_library()
    return api.Context(-1)


def test_budget_admits_reservations_until_full(hctx):
    hctx.set_budget(1000)
    assert hctx.memory()["budget_bytes"] == 1000
    hctx.reserve(600)
    with pytest.raises(api.TKError) as e:
        hctx.reserve(401)
    assert e.value.code == TK_ERR_BUDGET
    hctx.reserve(400)                      # exactly full
    assert hctx.memory()["reserved_bytes"] == 1000
    hctx.release(600)
    hctx.reserve(500)
    with pytest.raises(api.TKError) as e:  # giving back more than is reserved
        hctx.release(10_000)
    assert e.value.code == TK_ERR_ARG
    hctx.release(900)
    hctx.set_budget(0)                     # no budget: anything goes
    hctx.reserve(1 << 60)
    hctx.release(1 << 60)
    assert hctx.memory()["reserved_bytes"] == 0


def test_host_only_context_refuses_device_allocation(hctx):
    with pytest.raises(api.TKError) as e:
        hctx.alloc(256)
    assert e.value.code == TK_ERR_NO_DEVICE
    assert hctx.memory()["library_bytes"] == 0 and hctx.memory()["allocations"] == 0


def test_allocator_hooks_come_in_pairs():
    build_library()
    lib = _abi.load()
    h = C.c_void_p()
    only_alloc = _abi.ALLOC_FN(lambda n, u: None)
    rc = lib.tk_ctx_create(-1, None, only_alloc, _abi.FREE_FN(), None, C.byref(h))
    assert rc == TK_ERR_ARG and not h.value


def test_tmap_io_checks_size_and_dtype(hctx):
    s = hctx.space("U1", {-1: 2, 0: 3, 1: 2})
    t = hctx.tmap([s, s], [s])
    host = np.zeros(t.numel, dtype=np.float64)
    with pytest.raises(api.TKError) as e:  # wrong size: checked before any device work
        t.upload(host[:-1], 0)
    assert e.value.code == TK_ERR_ARG
    with pytest.raises(api.TKError) as e:  # a float64 buffer is half of what complex128 needs
        t.upload(host, 0, dtype="c128")
    assert e.value.code == TK_ERR_ARG
    with pytest.raises(api.TKError) as e:  # right size, but no device on this context (the address
        t.upload(host, 4096)               # is never dereferenced: the call stops at the device check)
    assert e.value.code == TK_ERR_NO_DEVICE
    cx = np.zeros(t.numel, dtype=np.complex128)
    with pytest.raises(api.TKError) as e:
        t.download(0, cx)                  # f64 download into a buffer twice too large
    assert e.value.code == TK_ERR_ARG


def test_noalloc_scratch_size_matches_header():
    build_library()
    with open(os.path.join(ROOT, "include", "tk.h")) as fh:
        m = re.search(r"#define TK_NOALLOC_SCRATCH_BYTES \(\(size_t\)(\d+) << (\d+)\)", fh.read())
    assert m, "TK_NOALLOC_SCRATCH_BYTES not found in tk.h"
    assert api.noalloc_scratch_bytes() == int(m.group(1)) << int(m.group(2))


def _empty_and_full(hctx):
    """t : V1 (x) V2 <- W has no admissible coupled sector (charge 2 against 0), so no elements;
    u : V1 (x) V2 <- X has one (charge 2)."""
    v1, v2 = hctx.space("U1", {1: 2}), hctx.space("U1", {1: 3})
    w, x = hctx.space("U1", {0: 1}), hctx.space("U1", {2: 4})
    return hctx.tmap([v1, v2], [w]), hctx.tmap([w], [x]), hctx.tmap([v1, v2], [x])


def test_null_buffers_only_for_maps_without_elements(hctx):
    """A NULL buffer passes the argument check exactly when its map has no elements: the host-only
    context then stops at the device check (TK_ERR_NO_DEVICE), never at the null check."""
    t, b, u = _empty_and_full(hctx)
    assert t.numel == 0 and b.numel == 0 and u.numel == 24
    pe = api.permute_plan(hctx, t, (1, 0), (2,))
    pf = api.permute_plan(hctx, u, (1, 0), (2,))
    with pytest.raises(api.TKError) as e:
        api.permute(hctx, pe, None, None)
    assert e.value.code == TK_ERR_NO_DEVICE
    with pytest.raises(api.TKError) as e:
        api.permute(hctx, pf, None, 4096)
    assert e.value.code == TK_ERR_ARG
    cp = api.compose_plan(hctx, t, b)           # C = t o b : V1 (x) V2 <- X, every block zero
    assert cp.output().numel == 24
    with pytest.raises(api.TKError) as e:       # A and B may be NULL, C may not
        api.contract(hctx, cp, None, None, None)
    assert e.value.code == TK_ERR_ARG
    with pytest.raises(api.TKError) as e:
        api.contract(hctx, cp, None, None, 4096)
    assert cp.workspace_bytes == 0 and e.value.code == TK_ERR_NO_DEVICE
    with pytest.raises(api.TKError) as e:
        api.contract_noalloc(hctx, cp, None, None, None)
    assert e.value.code == TK_ERR_ARG


def test_fp64_probe_argument_checks(hctx):
    with pytest.raises(api.TKError) as e:
        api.probe_fp64_peak(hctx, seconds=0.5)    # host-only context
    assert e.value.code == TK_ERR_NO_DEVICE
    with pytest.raises(api.TKError) as e:
        api.probe_fp64_peak(hctx, seconds=0.0)    # out of (0, 30]
    assert e.value.code == TK_ERR_ARG
    with pytest.raises(api.TKError) as e:
        api.probe_fp64_peak(hctx, seconds=31.0)
    assert e.value.code == TK_ERR_ARG


def test_set_choice_takes_only_autotuner_values(hctx):
    """tk_plan_set_choice: contraction plans only, and only values tk_plan_autotune can return
    (64 prep + 8 fp64 + split, with fp64 and split in 0..4 and prep in 0..2); a valid value on a
    host-only context stops at the device check."""
    t, b, u = _empty_and_full(hctx)
    cp = api.compose_plan(hctx, t, b)
    pf = api.permute_plan(hctx, u, (1, 0), (2,))
    lib = _abi.load()
    for bad in (-1, 5, 8 * 5, 64 * 3, 64 * 2 + 8 * 4 + 5):
        assert lib.tk_plan_set_choice(hctx._h, cp._h, bad) == TK_ERR_ARG
    assert lib.tk_plan_set_choice(hctx._h, pf._h, 0) == TK_ERR_ARG
    with pytest.raises(api.TKError) as e:
        api.set_choice(hctx, cp, fp64=4, split=4, prep=2)
    assert e.value.code == TK_ERR_NO_DEVICE
