"""Thin Python objects over the libtk C ABI.  Every step of the path runs in libtk's kernels;
this module only marshals arguments (PyTorch provides device memory and streams)."""

import ctypes as C

from . import _abi

SYM = {"Z2": 0, "U1": 1, "SU2": 2, "U1xSU2": 3, "Z2xU1": 4}


def product_sector(sym, a1, a2):
    """int32 label of the pair (a1, a2) of a Deligne-product symmetry (layout in include/tk.h)."""
    s = SYM[sym] if isinstance(sym, str) else int(sym)
    if s not in (3, 4):
        raise ValueError("not a product symmetry")
    return int(a1) * 4096 + (int(a2) + 2048 if s == 4 else int(a2))


def _sector_label(sym, a):
    """Sector labels may be given as ints or, for product symmetries, as (a1, a2) pairs."""
    return product_sector(sym, *a) if isinstance(a, tuple) else int(a)
DTYPE = {"f64": 0, "c128": 1}
GEMM = {"fp64": 0, "ozaki": 1, "tf32x3": 2}


class TKError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libtk error {code}: {msg}")
        self.code = code


def _lib():
    return _abi.load()


def _check(rc, ctx=None):
    if rc != 0:
        lib = _lib()
        msg = lib.tk_status_string(rc).decode()
        if ctx is not None:
            detail = lib.tk_ctx_last_error(ctx._h).decode()
            if detail:
                msg += ": " + detail
        raise TKError(rc, msg)


def _ints(xs, ctype=C.c_int):
    xs = [int(x) for x in xs]
    arr = (ctype * max(1, len(xs)))(*xs) if xs else (ctype * 1)()
    return arr, len(xs)


def _stream_handle(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _host_buffer(x):
    """(address, bytes) of a contiguous numpy array or torch CPU tensor."""
    if hasattr(x, "ctypes"):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("host buffer must be contiguous")
        return x.ctypes.data, x.nbytes
    if not x.is_contiguous():
        raise ValueError("host buffer must be contiguous")
    return x.data_ptr(), x.numel() * x.element_size()


def _ptr(t):
    if t is None:
        return C.c_void_p(0)
    if isinstance(t, int):
        return C.c_void_p(t)
    return C.c_void_p(t.data_ptr())


def _make_hooks(device, stream, allocator):
    """ctypes allocator hooks for tk_ctx_create: PyTorch's caching allocator ("torch") or a pair of
    Python callables (alloc(bytes) -> int, free(int, bytes))."""
    if allocator == "torch":
        import torch

        def alloc(nbytes):
            s = torch.cuda.current_stream(device) if stream is None else stream
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), device, s))

        def free(ptr, nbytes):
            torch.cuda.caching_allocator_delete(int(ptr))
    else:
        alloc, free = allocator

    def c_alloc(nbytes, _user):
        try:
            return alloc(int(nbytes)) or None
        except Exception:
            return None

    def c_free(ptr, nbytes, _user):
        try:
            free(int(ptr), int(nbytes))
        except Exception:
            pass

    return _abi.ALLOC_FN(c_alloc), _abi.FREE_FN(c_free)


class Context:
    """device >= 0: CUDA device; device < 0: host-only (planning and inspection only).

    stream: the context's stream (a torch.cuda.Stream or a raw handle; None: the legacy default
    stream); execution calls given no stream still pass torch's current stream.
    allocator: None (the library's cudaMalloc / cudaFree) or "torch" (plan tables and the other
    library allocations come from PyTorch's caching allocator through tk_ctx_create's hooks), or a
    pair (alloc(bytes) -> int pointer, free(int pointer, bytes)) of Python callables."""

    def __init__(self, device: int = 0, stream=None, allocator=None):
        self._h = C.c_void_p()
        self.device = device
        self._hooks = (_abi.ALLOC_FN(), _abi.FREE_FN())  # NULL hooks
        if allocator is not None and device >= 0:
            self._hooks = _make_hooks(device, stream, allocator)
        sh = C.c_void_p(0) if stream is None else (C.c_void_p(stream) if isinstance(stream, int)
                                                   else C.c_void_p(stream.cuda_stream))
        _check(_lib().tk_ctx_create(int(device), sh, self._hooks[0], self._hooks[1], None, C.byref(self._h)))

    def close(self):
        if self._h:
            _lib().tk_ctx_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync(self, stream=None):
        _check(_lib().tk_ctx_sync(self._h, self._stream(stream)), self)

    def _stream(self, stream):
        """Stream handle for a call (host-only contexts: NULL, no torch CUDA query)."""
        return C.c_void_p(0) if self.device < 0 and stream is None else _stream_handle(stream)

    # ---- device memory (tk_ctx_set_budget / reserve / release / memory / alloc / free)
    def set_budget(self, nbytes):
        _check(_lib().tk_ctx_set_budget(self._h, C.c_size_t(int(nbytes))), self)

    def reserve(self, nbytes):
        """Admit nbytes of caller-allocated memory against the budget (TKError code 11 if over)."""
        _check(_lib().tk_ctx_reserve(self._h, C.c_size_t(int(nbytes))), self)

    def release(self, nbytes):
        _check(_lib().tk_ctx_release(self._h, C.c_size_t(int(nbytes))), self)

    def memory(self):
        """dict(library_bytes, reserved_bytes, budget_bytes, allocations)."""
        lb, rb, bb, n = C.c_size_t(), C.c_size_t(), C.c_size_t(), C.c_int64()
        _check(_lib().tk_ctx_memory(self._h, C.byref(lb), C.byref(rb), C.byref(bb), C.byref(n)), self)
        return {"library_bytes": lb.value, "reserved_bytes": rb.value, "budget_bytes": bb.value,
                "allocations": n.value}

    def alloc(self, nbytes):
        """Raw device pointer (int) of nbytes through the context's allocator; free with free()."""
        p = C.c_void_p()
        _check(_lib().tk_ctx_alloc(self._h, C.c_size_t(int(nbytes)), C.byref(p)), self)
        return p.value or 0

    def free(self, ptr):
        _check(_lib().tk_ctx_free(self._h, C.c_void_p(ptr)), self)

    @property
    def launches(self):
        return int(_lib().tk_ctx_launch_count(self._h))

    def selftest_timeout(self, stream=None):
        """Launch the bounded-wait self-test; the next sync() raises TKError (TK_ERR_TIMEOUT)."""
        h = self._stream(stream)  # host-only: refused by the library
        _check(_lib().tk_ctx_selftest_timeout(self._h, h), self)

    def profile(self, enable=True):
        _check(_lib().tk_ctx_profile(self._h, int(bool(enable))), self)

    def profile_read(self, maxn=32):
        """{kernel name: (launches, total ms)} of the launches recorded since profiling began."""
        names = C.create_string_buffer(32 * maxn)
        counts = (C.c_int64 * maxn)()
        ms = (C.c_double * maxn)()
        n = C.c_int()
        _check(_lib().tk_ctx_profile_read(self._h, maxn, names, counts, ms, C.byref(n)), self)
        raw = names.raw
        return {raw[32 * i:32 * i + 32].split(b"\0")[0].decode(): (int(counts[i]), float(ms[i]))
                for i in range(min(n.value, maxn))}

    # ---- objects
    def space(self, sym, sectors, dual=False):
        return Space(self, sym, sectors, dual)

    def tmap(self, cod, dom):
        return TensorMap(self, cod, dom)


class Space:
    def __init__(self, ctx, sym, sectors, dual=False, _handle=None):
        self.ctx = ctx
        self._h = C.c_void_p()
        if _handle is not None:
            self._h = _handle
        else:
            items = sorted((_sector_label(sym, a), m) for a, m in dict(sectors).items())
            secs, n = _ints([a for a, _ in items], C.c_int32)
            mults, _ = _ints([m for _, m in items], C.c_int64)
            _check(_lib().tk_space_create(ctx._h, SYM[sym] if isinstance(sym, str) else int(sym), n, secs,
                                          mults, int(bool(dual)), C.byref(self._h)), ctx)

    def __del__(self):
        try:
            if self._h:
                _lib().tk_space_destroy(self._h)
        except Exception:
            pass

    def dual(self):
        h = C.c_void_p()
        _check(_lib().tk_space_dual(self.ctx._h, self._h, C.byref(h)), self.ctx)
        return Space(self.ctx, None, None, _handle=h)

    @property
    def dim(self):
        return int(_lib().tk_space_dim(self._h))

    @property
    def reduced_dim(self):
        return int(_lib().tk_space_reduced_dim(self._h))


class TensorMap:
    """Structure of a tensor map cod[0] (x) ... <- dom[0] (x) ... (no data attached)."""

    def __init__(self, ctx, cod, dom, _handle=None):
        self.ctx = ctx
        self._h = C.c_void_p()
        if _handle is not None:
            self._h = _handle
            self._legs = None
        else:
            self._legs = (list(cod), list(dom))  # keep the spaces alive
            ca = (C.c_void_p * max(1, len(cod)))(*[s._h.value for s in cod])
            da = (C.c_void_p * max(1, len(dom)))(*[s._h.value for s in dom])
            _check(_lib().tk_tmap_create(ctx._h, len(cod), ca, len(dom), da, C.byref(self._h)), ctx)

    def __del__(self):
        try:
            if self._h:
                _lib().tk_tmap_destroy(self._h)
        except Exception:
            pass

    @property
    def numel(self):
        return int(_lib().tk_tmap_numel(self._h))

    @property
    def nlegs(self):
        a, b = C.c_int(), C.c_int()
        _check(_lib().tk_tmap_nlegs(self._h, C.byref(a), C.byref(b)))
        return a.value, b.value

    @property
    def hash(self):
        return int(_lib().tk_tmap_hash(self._h))

    def leg(self, i):
        h = C.c_void_p()
        _check(_lib().tk_tmap_leg(self.ctx._h, self._h, int(i), C.byref(h)), self.ctx)
        return Space(self.ctx, None, None, _handle=h)

    def blocks(self):
        out = []
        s, r, c, o = C.c_int32(), C.c_int64(), C.c_int64(), C.c_int64()
        for i in range(_lib().tk_tmap_nblocks(self._h)):
            _check(_lib().tk_tmap_block(self._h, i, C.byref(s), C.byref(r), C.byref(c), C.byref(o)))
            out.append((s.value, r.value, c.value, o.value))
        return out

    def upload(self, host, device, dtype="f64", stream=None):
        """tk_tmap_upload: host buffer (numpy array or torch CPU tensor) -> device tensor, blocks in
        canonical order; the sizes must match this structure."""
        hp, nb = _host_buffer(host)
        _check(_lib().tk_tmap_upload(self.ctx._h, self._h, DTYPE[dtype], C.c_void_p(hp), C.c_size_t(nb),
                                     _ptr(device), self.ctx._stream(stream)), self.ctx)

    def download(self, device, host, dtype="f64", stream=None):
        """tk_tmap_download: device tensor -> host buffer (numpy array or torch CPU tensor)."""
        hp, nb = _host_buffer(host)
        _check(_lib().tk_tmap_download(self.ctx._h, self._h, DTYPE[dtype], _ptr(device), C.c_void_p(hp),
                                       C.c_size_t(nb), self.ctx._stream(stream)), self.ctx)

    def treepairs(self):
        """[(uncoupled labels, split inner, coupled, fusion inner, offset, ld, dims)]"""
        n1, n2 = self.nlegs
        n = n1 + n2
        ni1, ni2 = max(n1 - 2, 0), max(n2 - 2, 0)
        lab = (C.c_int32 * (n + ni1 + 1 + ni2))()
        dims = (C.c_int64 * n)()
        off, ld = C.c_int64(), C.c_int64()
        out = []
        for i in range(_lib().tk_tmap_ntreepairs(self._h)):
            _check(_lib().tk_tmap_treepair(self._h, i, lab, C.byref(off), C.byref(ld), dims))
            L = list(lab)
            out.append((tuple(L[:n]), tuple(L[n:n + ni1]), L[n + ni1], tuple(L[n + ni1 + 1:]),
                        off.value, ld.value, tuple(dims)))
        return out


class Plan:
    def __init__(self, ctx, handle, kind):
        self.ctx, self._h, self.kind = ctx, handle, kind

    def __del__(self):
        try:
            if self._h:
                _lib().tk_plan_destroy(self._h)
        except Exception:
            pass

    def output(self):
        h = C.c_void_p()
        _check(_lib().tk_plan_output(self.ctx._h, self._h, C.byref(h)), self.ctx)
        return TensorMap(self.ctx, None, None, _handle=h)

    @property
    def workspace_bytes(self):
        return int(_lib().tk_plan_workspace_bytes(self._h))

    @property
    def flops(self):
        return float(_lib().tk_plan_flops(self._h))

    @property
    def tensor_flops(self):
        """Block flops of the products that run on the split-precision tensor-core path."""
        return float(_lib().tk_plan_tensor_flops(self._h))

    @property
    def permute_bytes(self):
        return float(_lib().tk_plan_permute_bytes(self._h))

    def permute_stats(self, which=0):
        """Task mix of one permute: dict of run / transpose / element-wise task and element counts
        (None when that permute is the identity)."""
        st = (C.c_int64 * 8)()
        if _lib().tk_plan_permute_stats(self._h, int(which), st) != 0:
            return None
        keys = ("run_tasks", "run_elems", "runs", "transpose_tasks", "transpose_elems", "generic_tasks",
                "generic_elems", "tiles")
        return dict(zip(keys, list(st)))

    def transform(self, which=0):
        """[(src_offset, dst_offset, coef)] of one permute (None when it is the identity)."""
        lib = _lib()
        n = lib.tk_plan_ntransform(self._h, int(which))
        if n < 0:
            return None
        s, d, c = C.c_int64(), C.c_int64(), C.c_double()
        out = []
        for k in range(n):
            _check(lib.tk_plan_transform(self._h, int(which), k, C.byref(s), C.byref(d), C.byref(c)))
            out.append((s.value, d.value, c.value))
        return out


def permute_plan(ctx, t, p, q, dtype="f64"):
    pa, npa = _ints(p)
    qa, nqa = _ints(q)
    h = C.c_void_p()
    _check(_lib().tk_permute_plan(ctx._h, t._h, npa, pa, nqa, qa, DTYPE[dtype], C.byref(h)), ctx)
    return Plan(ctx, h, "permute")


def adjoint_plan(ctx, t, dtype="f64"):
    """tk_adjoint_plan: t^dagger (domain and codomain exchanged, complex data conjugated); run it
    with permute()."""
    h = C.c_void_p()
    _check(_lib().tk_adjoint_plan(ctx._h, t._h, DTYPE[dtype], C.byref(h)), ctx)
    return Plan(ctx, h, "permute")


class SvdPlan(Plan):
    """Block SVD of a tensor map's structure (tk_svd_plan)."""

    def outputs(self):
        """(U structure, V^dagger structure, number of singular values)."""
        hu, hv, n = C.c_void_p(), C.c_void_p(), C.c_int64(0)
        _check(_lib().tk_svd_outputs(self.ctx._h, self._h, C.byref(hu), C.byref(hv), C.byref(n)), self.ctx)
        return TensorMap(self.ctx, None, None, _handle=hu), TensorMap(self.ctx, None, None, _handle=hv), n.value

    def blocks(self):
        """[(sector, rows, cols, offset of its singular values)] in sector order."""
        out = []
        for i in range(int(_lib().tk_svd_nblocks(self._h))):
            c, r, k, o = C.c_int32(), C.c_int64(), C.c_int64(), C.c_int64()
            _lib().tk_svd_block(self._h, i, C.byref(c), C.byref(r), C.byref(k), C.byref(o))
            out.append((c.value, r.value, k.value, o.value))
        return out


def svd_plan(ctx, t, dtype="f64"):
    h = C.c_void_p()
    _check(_lib().tk_svd_plan(ctx._h, t._h, DTYPE[dtype], C.byref(h)), ctx)
    return SvdPlan(ctx, h, "svd")


def svd(ctx, plan, a, u, s, vh, workspace, stream=None):
    """tk_svd: a -> (u, s, vh) device tensors laid out as plan.outputs()."""
    nbytes = workspace.numel() * workspace.element_size()
    _check(_lib().tk_svd(ctx._h, plan._h, _ptr(a), _ptr(u), _ptr(s), _ptr(vh), _ptr(workspace),
                         C.c_size_t(nbytes), ctx._stream(stream)), ctx)


def svd_truncate(ctx, plan, keep, u, s, vh, ut, st, vht, stream=None):
    """tk_svd_truncate: keep[i] leading triplets of block i (plan.blocks() order)."""
    arr = (C.c_int64 * max(1, len(keep)))(*[int(k) for k in keep])
    _check(_lib().tk_svd_truncate(ctx._h, plan._h, arr, _ptr(u), _ptr(s), _ptr(vh), _ptr(ut), _ptr(st), _ptr(vht),
                                  ctx._stream(stream)), ctx)


def compose_plan(ctx, a, b, dtype="f64", gemm="fp64", slices=0):
    """Plan of the composition A o B (domain of A = codomain of B), legs kept in place."""
    h = C.c_void_p()
    _check(_lib().tk_compose_plan(ctx._h, a._h, b._h, DTYPE[dtype], GEMM[gemm], int(slices), C.byref(h)), ctx)
    return Plan(ctx, h, "contract")


def contract_plan(ctx, a, pa, qa, b, pb, qb, pab, qab, dtype="f64", gemm="fp64", slices=0):
    args = []
    for xs in (pa, qa):
        arr, n = _ints(xs)
        args += [n, arr]
    a_args = args
    args = []
    for xs in (pb, qb):
        arr, n = _ints(xs)
        args += [n, arr]
    b_args = args
    c_args = []
    for xs in (pab, qab):
        arr, n = _ints(xs)
        c_args += [n, arr]
    h = C.c_void_p()
    _check(_lib().tk_contract_plan(ctx._h, a._h, *a_args, b._h, *b_args, *c_args, DTYPE[dtype],
                                   GEMM[gemm], int(slices), C.byref(h)), ctx)
    return Plan(ctx, h, "contract")


def permute(ctx, plan, a, c, stream=None):
    _check(_lib().tk_permute(ctx._h, plan._h, _ptr(a), _ptr(c), ctx._stream(stream)), ctx)


def contract(ctx, plan, a, b, c, workspace=None, stream=None):
    nbytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check(_lib().tk_contract(ctx._h, plan._h, _ptr(a), _ptr(b), _ptr(c), _ptr(workspace),
                              C.c_size_t(nbytes), ctx._stream(stream)), ctx)


def contract_batch(ctx, plans, a, b, c, workspaces, stream=None):
    """tk_contract_batch: request i = (plans[i], a[i], b[i], c[i], workspaces[i]); the stages of
    all requests share launches.  Lists of equal length; buffers are device tensors."""
    n = len(plans)
    if not (len(a) == len(b) == len(c) == len(workspaces) == n):
        raise ValueError("batch lists differ in length")
    vp = C.c_void_p * max(n, 1)
    sz = C.c_size_t * max(n, 1)
    hp = vp(*[p._h for p in plans])
    ha, hb, hc = vp(*[_ptr(x) for x in a]), vp(*[_ptr(x) for x in b]), vp(*[_ptr(x) for x in c])
    hw = vp(*[_ptr(w) for w in workspaces])
    hn = sz(*[0 if w is None else w.numel() * w.element_size() for w in workspaces])
    _check(_lib().tk_contract_batch(ctx._h, n, hp, ha, hb, hc, hw, hn, ctx._stream(stream)), ctx)


def autotune(ctx, plan, a, b, c, workspace, stream=None):
    """tk_plan_autotune: time the plan's candidate work lists on these buffers, keep the fastest.
    Returns (fp64 candidate, split-precision candidate, preparation candidate); 0 means the
    built-in heuristic."""
    choice = C.c_int(0)
    nbytes = workspace.numel() * workspace.element_size()
    _check(_lib().tk_plan_autotune(ctx._h, plan._h, _ptr(a), _ptr(b), _ptr(c), _ptr(workspace),
                                   C.c_size_t(nbytes), ctx._stream(stream), C.byref(choice)), ctx)
    return (choice.value // 8) % 8, choice.value % 8, choice.value // 64


def set_choice(ctx, plan, fp64=0, split=0, prep=0):
    """tk_plan_set_choice: apply an autotuner choice (the triple `autotune` returns) untimed."""
    _check(_lib().tk_plan_set_choice(ctx._h, plan._h, C.c_int(64 * prep + 8 * fp64 + split)), ctx)


def noalloc_scratch_bytes():
    """Size of libtk's built-in scratch array (tk_noalloc_scratch_bytes)."""
    return int(_lib().tk_noalloc_scratch_bytes())


def contract_noalloc(ctx, plan, a, b, c, stream=None):
    """tk_contract_noalloc: the contraction with its scratch in libtk's built-in device array,
    for callers that cannot allocate device memory (see include/tk.h)."""
    _check(_lib().tk_contract_noalloc(ctx._h, plan._h, _ptr(a), _ptr(b), _ptr(c), ctx._stream(stream)), ctx)


def copy_h2d(ctx, dst, src_host_ptr, nbytes, stream=None):
    _check(_lib().tk_copy_h2d(ctx._h, _ptr(dst), C.c_void_p(src_host_ptr), C.c_size_t(nbytes),
                              ctx._stream(stream)), ctx)


def copy_d2h(ctx, dst_host_ptr, src, nbytes, stream=None):
    _check(_lib().tk_copy_d2h(ctx._h, C.c_void_p(dst_host_ptr), _ptr(src), C.c_size_t(nbytes),
                              ctx._stream(stream)), ctx)


def probe_fp64_peak(ctx, seconds=1.0, stream=None):
    """tk_probe_fp64_peak: (TFLOP/s of a register-only FP64 FMA loop on every SM, its ms)."""
    tf, ms = C.c_double(), C.c_double()
    _check(_lib().tk_probe_fp64_peak(ctx._h, C.c_double(seconds), C.byref(tf), C.byref(ms), ctx._stream(stream)), ctx)
    return tf.value, ms.value


def fsymbol(sym, a, b, c, d, e, f):
    return float(_lib().tk_fsymbol(SYM[sym], a, b, c, d, e, f))


def rsymbol(sym, a, b, c):
    return float(_lib().tk_rsymbol(SYM[sym], a, b, c))
