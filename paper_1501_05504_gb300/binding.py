"""ctypes binding of ``libdmrg3s.so`` (the C ABI declared in include/dmrg3s.h).

Argument marshalling only: every contraction runs in the library's CUDA
kernels.  PyTorch provides device memory and streams.  If the library has not
been built the import-time loader raises; there is no fallback.

Python objects mirror the C structs:

* ``Bond(q, dim)``: charge sectors of a bond (``q`` int array (nsec, nsym));
* ``Site(qp, left, right, data)``: MPS site tensor, ``data`` a CUDA float64
  tensor in the canonical block layout;
* ``Env(t, bond, data)``: environment;
* ``MpoSite(qp, tl, tr, W)``: MPO site tensor, ``W`` a host float64 array
  indexed ``[s_out, s_in, bl, br]``.

Functions keep the C names: ``dmrg3s_apply_heff``, ``dmrg3s_expand``,
``dmrg3s_update_env`` ...
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdmrg3s.so")

DMRG3S_FP64, DMRG3S_TF32X3, DMRG3S_TF32 = 0, 1, 2
PRECISIONS = {"fp64": DMRG3S_FP64, "tf32x3": DMRG3S_TF32X3, "tf32": DMRG3S_TF32}

i32p = ctypes.POINTER(ctypes.c_int32)
i64p = ctypes.POINTER(ctypes.c_int64)
f64p = ctypes.POINTER(ctypes.c_double)


class _Bond(ctypes.Structure):
    _fields_ = [("nsec", ctypes.c_int32), ("q", i32p), ("dim", i64p)]


class _Site(ctypes.Structure):
    _fields_ = [("nsym", ctypes.c_int32), ("d", ctypes.c_int32), ("qp", i32p),
                ("left", _Bond), ("right", _Bond), ("data", ctypes.c_void_p)]


class _Env(ctypes.Structure):
    _fields_ = [("nsym", ctypes.c_int32), ("w", ctypes.c_int32), ("t", i32p),
                ("bond", _Bond), ("data", ctypes.c_void_p)]


class _MpoSite(ctypes.Structure):
    _fields_ = [("nsym", ctypes.c_int32), ("d", ctypes.c_int32), ("wl", ctypes.c_int32),
                ("wr", ctypes.c_int32), ("qp", i32p), ("tl", i32p), ("tr", i32p), ("W", f64p)]


class Dmrg3sError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        msg = "%s failed: %s (status %d)" % (where, _status_string(status), status)
        if detail:
            msg += ": " + detail
        super().__init__(msg)


_lib = None


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libdmrg3s.so is not built (run __graft_entry__.build()); "
                              "the DMRG3S kernels have no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        L.dmrg3s_status_string.restype = ctypes.c_char_p
        L.dmrg3s_last_error.restype = ctypes.c_char_p
        L.dmrg3s_last_error.argtypes = [ctypes.c_void_p]
        L.dmrg3s_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_size_t]
        L.dmrg3s_destroy.argtypes = [ctypes.c_void_p]
        L.dmrg3s_site_size.argtypes = [ctypes.POINTER(_Site), i64p]
        L.dmrg3s_env_size.argtypes = [ctypes.POINTER(_Env), i64p]
        L.dmrg3s_site_blocks.argtypes = [ctypes.POINTER(_Site), i64p, i64p]
        L.dmrg3s_env_blocks.argtypes = [ctypes.POINTER(_Env), i64p, i64p]
        L.dmrg3s_expanded_bond.argtypes = [ctypes.c_int32, ctypes.POINTER(_Bond), ctypes.c_int32,
                                           i32p, ctypes.c_int32, i32p, i32p, i64p]
        L.dmrg3s_apply_heff.argtypes = [ctypes.c_void_p, ctypes.POINTER(_Env),
                                        ctypes.POINTER(_MpoSite), ctypes.POINTER(_Env),
                                        ctypes.POINTER(_Site), ctypes.POINTER(_Site),
                                        ctypes.c_int, ctypes.c_void_p]
        L.dmrg3s_expand.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(_Env),
                                    ctypes.POINTER(_MpoSite), ctypes.POINTER(_Site),
                                    ctypes.c_double, ctypes.POINTER(_Site), ctypes.c_int,
                                    ctypes.c_void_p]
        L.dmrg3s_update_env.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(_Env),
                                        ctypes.POINTER(_MpoSite), ctypes.POINTER(_Site),
                                        ctypes.POINTER(_Env), ctypes.c_int, ctypes.c_void_p]
        _lib = L
    return _lib


def _status_string(status):
    try:
        return lib().dmrg3s_status_string(int(status)).decode()
    except Exception:
        return "status %d" % status


# ---- Python-side tensors ------------------------------------------------------------

class Bond:
    def __init__(self, q, dim):
        dim = np.ascontiguousarray(dim, dtype=np.int64).reshape(-1)
        q = np.asarray(q, dtype=np.int32)
        if q.ndim == 1:
            q = q.reshape(len(dim), -1) if q.size else np.zeros((len(dim), 0), dtype=np.int32)
        self.q = np.ascontiguousarray(q, dtype=np.int32)
        self.dim = dim

    @classmethod
    def from_neutral(cls, b):
        return cls(b["q"], b["dim"])

    @property
    def nsym(self):
        return self.q.shape[1]

    def _c(self):
        return _Bond(len(self.dim), self.q.ctypes.data_as(i32p) if self.q.size else None,
                     self.dim.ctypes.data_as(i64p))

    def __eq__(self, other):
        return np.array_equal(self.q, other.q) and np.array_equal(self.dim, other.dim)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(int(t.data_ptr()))


class Site:
    """MPS site tensor M[s](al, ar) with canonical block layout on the device."""

    def __init__(self, qp, left, right, data=None):
        self.qp = np.ascontiguousarray(np.asarray(qp, dtype=np.int32).reshape(len(qp), -1))
        self.left, self.right, self.data = left, right, data

    @property
    def nsym(self):
        return self.qp.shape[1]

    @property
    def d(self):
        return self.qp.shape[0]

    def _c(self):
        self._keep = (self.left._c(), self.right._c())
        return _Site(self.nsym, self.d, self.qp.ctypes.data_as(i32p) if self.qp.size else None,
                     self._keep[0], self._keep[1], _ptr(self.data))

    def size(self):
        n = ctypes.c_int64()
        c = self._c()
        _check(lib().dmrg3s_site_size(ctypes.byref(c), ctypes.byref(n)), "dmrg3s_site_size")
        return n.value

    def blocks(self):
        """Canonical block table: rows (s, i, j, offset, rows, cols)."""
        c = self._c()
        n = ctypes.c_int64()
        _check(lib().dmrg3s_site_blocks(ctypes.byref(c), ctypes.byref(n), None), "dmrg3s_site_blocks")
        tab = np.zeros((n.value, 6), dtype=np.int64)
        _check(lib().dmrg3s_site_blocks(ctypes.byref(c), ctypes.byref(n), tab.ctypes.data_as(i64p)),
               "dmrg3s_site_blocks")
        return tab


class Env:
    """Environment E[b](a_bra, a_ket) on one bond with canonical block layout."""

    def __init__(self, t, bond, data=None):
        self.t = np.ascontiguousarray(np.asarray(t, dtype=np.int32).reshape(len(t), -1))
        self.bond, self.data = bond, data

    @property
    def nsym(self):
        return self.t.shape[1]

    @property
    def w(self):
        return self.t.shape[0]

    def _c(self):
        self._keep = self.bond._c()
        return _Env(self.nsym, self.w, self.t.ctypes.data_as(i32p) if self.t.size else None,
                    self._keep, _ptr(self.data))

    def size(self):
        n = ctypes.c_int64()
        c = self._c()
        _check(lib().dmrg3s_env_size(ctypes.byref(c), ctypes.byref(n)), "dmrg3s_env_size")
        return n.value

    def blocks(self):
        c = self._c()
        n = ctypes.c_int64()
        _check(lib().dmrg3s_env_blocks(ctypes.byref(c), ctypes.byref(n), None), "dmrg3s_env_blocks")
        tab = np.zeros((n.value, 6), dtype=np.int64)
        _check(lib().dmrg3s_env_blocks(ctypes.byref(c), ctypes.byref(n), tab.ctypes.data_as(i64p)),
               "dmrg3s_env_blocks")
        return tab


class MpoSite:
    def __init__(self, qp, tl, tr, W):
        self.W = np.ascontiguousarray(W, dtype=np.float64)
        d, _, wl, wr = self.W.shape
        self.qp = np.ascontiguousarray(np.asarray(qp, dtype=np.int32).reshape(d, -1))
        self.tl = np.ascontiguousarray(np.asarray(tl, dtype=np.int32).reshape(wl, -1))
        self.tr = np.ascontiguousarray(np.asarray(tr, dtype=np.int32).reshape(wr, -1))

    def _c(self):
        nsym = self.qp.shape[1]
        d, _, wl, wr = self.W.shape

        def p(a):
            return a.ctypes.data_as(i32p) if a.size else None
        return _MpoSite(nsym, d, wl, wr, p(self.qp), p(self.tl), p(self.tr),
                        self.W.ctypes.data_as(f64p))


def expanded_bond(bond, t, include_base=False):
    """Fused bond of the expansion (dmrg3s_expanded_bond)."""
    t = np.ascontiguousarray(np.asarray(t, dtype=np.int32).reshape(len(t), -1))
    nsym = bond.nsym
    cb = bond._c()
    n = ctypes.c_int32()
    tp = t.ctypes.data_as(i32p) if t.size else None
    _check(lib().dmrg3s_expanded_bond(nsym, ctypes.byref(cb), t.shape[0], tp, int(include_base),
                                      ctypes.byref(n), None, None), "dmrg3s_expanded_bond")
    q = np.zeros((n.value, nsym), dtype=np.int32)
    dim = np.zeros(n.value, dtype=np.int64)
    _check(lib().dmrg3s_expanded_bond(nsym, ctypes.byref(cb), t.shape[0], tp, int(include_base),
                                      ctypes.byref(n), q.ctypes.data_as(i32p) if q.size else None,
                                      dim.ctypes.data_as(i64p)), "dmrg3s_expanded_bond")
    return Bond(q, dim)


def _check(status, where, ctx=None):
    if status != 0:
        detail = ""
        if ctx is not None:
            detail = lib().dmrg3s_last_error(ctx).decode()
        raise Dmrg3sError(status, where, detail)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _prec(p):
    return PRECISIONS[p] if isinstance(p, str) else int(p)


# ---- context and entry points (same names as the C ABI) -------------------------------

class Context:
    def __init__(self, device=0, workspace_bytes=0):
        import weakref
        self.handle = ctypes.c_void_p()
        self._states = weakref.WeakSet()     # states must be destroyed before their context
        _check(lib().dmrg3s_create(ctypes.byref(self.handle), int(device), int(workspace_bytes)),
               "dmrg3s_create")

    def close(self):
        if self.handle:
            for st in list(self._states):
                st.close()
            lib().dmrg3s_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dmrg3s_create(device=0, workspace_bytes=0):
    return Context(device, workspace_bytes)


def dmrg3s_destroy(ctx):
    ctx.close()


def dmrg3s_apply_heff(ctx, L, W, R, A, HA, prec="fp64", stream=None):
    cL, cR, cA, cH, cW = L._c(), R._c(), A._c(), HA._c(), W._c()
    _check(lib().dmrg3s_apply_heff(ctx.handle, ctypes.byref(cL), ctypes.byref(cW), ctypes.byref(cR),
                                   ctypes.byref(cA), ctypes.byref(cH), _prec(prec), _stream(stream)),
           "dmrg3s_apply_heff", ctx.handle)


def dmrg3s_expand(ctx, direction, env, W, M, alpha, P, prec="fp64", stream=None):
    ce, cW, cM, cP = env._c(), W._c(), M._c(), P._c()
    _check(lib().dmrg3s_expand(ctx.handle, int(direction), ctypes.byref(ce), ctypes.byref(cW),
                               ctypes.byref(cM), float(alpha), ctypes.byref(cP), _prec(prec),
                               _stream(stream)), "dmrg3s_expand", ctx.handle)


def dmrg3s_update_env(ctx, direction, env, W, A, out, prec="fp64", stream=None):
    ce, cW, cA, co = env._c(), W._c(), A._c(), out._c()
    _check(lib().dmrg3s_update_env(ctx.handle, int(direction), ctypes.byref(ce), ctypes.byref(cW),
                                   ctypes.byref(cA), ctypes.byref(co), _prec(prec), _stream(stream)),
           "dmrg3s_update_env", ctx.handle)


# ---- packing between neutral block dictionaries and the canonical layout -----------------

def pack_blocks(table, blocks, keyfn=lambda r: (int(r[0]), int(r[1]), int(r[2]))):
    """Flat float64 host array holding ``blocks`` in the order of a block table."""
    n = int(table[-1, 3] + table[-1, 4] * table[-1, 5]) if len(table) else 0
    flat = np.zeros(n, dtype=np.float64)
    for r in table:
        key = keyfn(r)
        if key in blocks:
            off, rows, cols = int(r[3]), int(r[4]), int(r[5])
            flat[off:off + rows * cols] = np.asarray(blocks[key], dtype=np.float64).reshape(-1)
    return flat


def unpack_blocks(table, flat):
    out = {}
    for r in table:
        off, rows, cols = int(r[3]), int(r[4]), int(r[5])
        out[(int(r[0]), int(r[1]), int(r[2]))] = np.asarray(flat[off:off + rows * cols]).reshape(rows, cols)
    return out


def site_from_neutral(spec, device="cuda"):
    import torch
    s = Site(spec["qp"], Bond.from_neutral(spec["left"]), Bond.from_neutral(spec["right"]))
    flat = pack_blocks(s.blocks(), spec["blocks"])
    s.data = torch.from_numpy(flat).to(device)
    return s


def product_state(qp, local_states, device="cuda"):
    """Site tensors (m = 1) of the product state |s_1 ... s_l>; the bond charges
    add up the local charges from the left (charge 0 at the left end)."""
    import torch
    qp = np.asarray(qp, dtype=np.int64).reshape(len(qp), -1)
    q = np.zeros(qp.shape[1], dtype=np.int64)
    sites = []
    for s in local_states:
        left = Bond(q.reshape(1, -1).copy(), np.array([1], dtype=np.int64))
        q = q + qp[s]
        right = Bond(q.reshape(1, -1).copy(), np.array([1], dtype=np.int64))
        site = Site(qp, left, right)
        flat = pack_blocks(site.blocks(), {(int(s), 0, 0): np.ones((1, 1))})
        site.data = torch.from_numpy(flat).to(device)
        sites.append(site)
    return sites


def env_from_neutral(spec, device="cuda"):
    import torch
    e = Env(spec["t"], Bond.from_neutral(spec["bond"] if "bond" in spec else spec["ket"]))
    flat = pack_blocks(e.blocks(), spec["blocks"])
    e.data = torch.from_numpy(flat).to(device)
    return e


def empty_site_like(qp, left, right, device="cuda"):
    import torch
    s = Site(qp, left, right)
    s.data = torch.zeros(max(s.size(), 1), dtype=torch.float64, device=device)
    return s


def empty_env(t, bond, device="cuda"):
    import torch
    e = Env(t, bond)
    e.data = torch.zeros(max(e.size(), 1), dtype=torch.float64, device=device)
    return e


def mpo_from_neutral(spec):
    return MpoSite(spec["qp"], spec["tl"], spec["tr"], spec["W"])


# ---- eigensolver, MPO builders, state, local update, sweep ------------------------------

class _UpdateOpts(ctypes.Structure):
    _fields_ = [("m_max", ctypes.c_int32), ("lanczos_kmax", ctypes.c_int32),
                ("lanczos_tol", ctypes.c_double), ("trunc_eps", ctypes.c_double),
                ("precision", ctypes.c_int), ("skip_eigensolver", ctypes.c_int32),
                ("svd", ctypes.c_int)]


SVD_GESVD, SVD_JACOBI, SVD_AUTO = 0, 1, 2
_SVD = {"jacobi": SVD_JACOBI, "gesvd": SVD_GESVD, "auto": SVD_AUTO}


class _UpdateInfo(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("energy_before", ctypes.c_double),
                ("energy_after", ctypes.c_double), ("discarded_weight", ctypes.c_double),
                ("lanczos_iters", ctypes.c_int32), ("new_bond_dim", ctypes.c_int32),
                ("svd_fallback", ctypes.c_int32), ("svd_sweeps", ctypes.c_int32)]


class _AlphaRule(ctypes.Structure):
    _fields_ = [("alpha0", ctypes.c_double), ("target", ctypes.c_double), ("up", ctypes.c_double),
                ("down", ctypes.c_double), ("alpha_min", ctypes.c_double),
                ("alpha_max", ctypes.c_double), ("fixed", ctypes.c_int32)]


class _SweepOpts(ctypes.Structure):
    _fields_ = [("max_sweeps", ctypes.c_int32), ("conv_tol", ctypes.c_double),
                ("update", _UpdateOpts), ("final_precision", ctypes.c_int),
                ("switch_tol", ctypes.c_double), ("alphas", f64p), ("seconds", f64p)]


class _SweepReport(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("lanczos_iters", ctypes.c_int32), ("svd_fallbacks", ctypes.c_int32),
                ("energy", ctypes.c_double), ("alpha", ctypes.c_double),
                ("bulk_sweeps", ctypes.c_int32), ("pad", ctypes.c_int32)]


MODEL_XXZ, MODEL_HUBBARD, MODEL_SPIN_BONDS = 0, 1, 2


def _setup_state_api(L):
    if getattr(L, "_state_api", False):
        return L
    L.dmrg3s_eigensolve.argtypes = [ctypes.c_void_p, ctypes.POINTER(_Env), ctypes.POINTER(_MpoSite),
                                    ctypes.POINTER(_Env), ctypes.POINTER(_Site), ctypes.c_int32,
                                    ctypes.c_double, ctypes.c_int, f64p, i32p, ctypes.c_void_p]
    L.dmrg3s_mpo_create.argtypes = [ctypes.c_int32, ctypes.c_int32, f64p, ctypes.c_int32, i32p, f64p,
                                    ctypes.POINTER(ctypes.c_void_p)]
    L.dmrg3s_mpo_destroy.argtypes = [ctypes.c_void_p]
    L.dmrg3s_mpo_get_site.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(_MpoSite)]
    L.dmrg3s_state_create.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(_MpoSite),
                                      ctypes.POINTER(_Site), ctypes.POINTER(_Env),
                                      ctypes.POINTER(_Env), ctypes.c_int32,
                                      ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p]
    L.dmrg3s_state_destroy.argtypes = [ctypes.c_void_p]
    L.dmrg3s_local_update.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_double,
                                      ctypes.POINTER(_UpdateOpts), ctypes.POINTER(_UpdateInfo),
                                      ctypes.c_void_p]
    L.dmrg3s_sweep.argtypes = [ctypes.c_void_p, ctypes.POINTER(_AlphaRule), ctypes.POINTER(_SweepOpts),
                               f64p, ctypes.POINTER(_SweepReport), ctypes.c_void_p]
    L.dmrg3s_local_update_batch.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32, i32p, f64p,
                                            ctypes.POINTER(_UpdateOpts), ctypes.POINTER(_UpdateInfo),
                                            ctypes.c_void_p]
    L.dmrg3s_sweep_batch.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32,
                                     ctypes.POINTER(_AlphaRule), ctypes.POINTER(_SweepOpts),
                                     ctypes.POINTER(f64p), ctypes.POINTER(_SweepReport), ctypes.c_void_p]
    L.dmrg3s_state_centre.argtypes = [ctypes.c_void_p, i32p, f64p]
    L.dmrg3s_state_site_info.argtypes = [ctypes.c_void_p, ctypes.c_int32, i32p, i32p, i64p, i32p,
                                         i32p, i64p, i64p]
    L.dmrg3s_state_site_copy.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                         ctypes.c_void_p]
    L._state_api = True
    return L


def slib():
    return _setup_state_api(lib())


def dmrg3s_eigensolve(ctx, L, W, R, M, kmax=40, tol=1e-10, prec="fp64", stream=None):
    """Lanczos on the device; M is overwritten by the Ritz vector.  Returns (lambda, iters)."""
    cL, cW, cR, cM = L._c(), W._c(), R._c(), M._c()
    lam = ctypes.c_double()
    it = ctypes.c_int32()
    _check(slib().dmrg3s_eigensolve(ctx.handle, ctypes.byref(cL), ctypes.byref(cW), ctypes.byref(cR),
                                    ctypes.byref(cM), int(kmax), float(tol), _prec(prec),
                                    ctypes.byref(lam), ctypes.byref(it), _stream(stream)),
           "dmrg3s_eigensolve", ctx.handle)
    return lam.value, it.value


class Mpo:
    """Model MPO built by the library (host arrays owned by the handle)."""

    def __init__(self, model, nsites, params=(), bonds=None, couplings=None):
        self.handle = ctypes.c_void_p()
        self.nsites = int(nsites)
        par = np.ascontiguousarray(params, dtype=np.float64)
        nb, bp, cp = 0, None, None
        if bonds is not None:
            self._b = np.ascontiguousarray(bonds, dtype=np.int32).reshape(-1, 2)
            self._c = np.ascontiguousarray(couplings, dtype=np.float64).reshape(-1, 2)
            nb, bp, cp = len(self._b), self._b.ctypes.data_as(i32p), self._c.ctypes.data_as(f64p)
        _check(slib().dmrg3s_mpo_create(int(model), self.nsites, par.ctypes.data_as(f64p) if par.size else None,
                                        nb, bp, cp, ctypes.byref(self.handle)), "dmrg3s_mpo_create")

    def site(self, i):
        s = _MpoSite()
        _check(slib().dmrg3s_mpo_get_site(self.handle, int(i), ctypes.byref(s)), "dmrg3s_mpo_get_site")
        d, wl, wr, nsym = s.d, s.wl, s.wr, s.nsym
        W = np.ctypeslib.as_array(s.W, shape=(d * d * wl * wr,)).reshape(d, d, wl, wr).copy()

        def arr(p, n):
            return np.ctypeslib.as_array(p, shape=(n * nsym,)).reshape(n, nsym).copy() if nsym else np.zeros((n, 0), np.int32)
        return MpoSite(arr(s.qp, d), arr(s.tl, wl), arr(s.tr, wr), W)

    def sites(self):
        return [self.site(i) for i in range(self.nsites)]

    def __del__(self):
        try:
            if self.handle:
                slib().dmrg3s_mpo_destroy(self.handle)
        except Exception:
            pass


def dmrg3s_mpo_create(model, nsites, params=(), bonds=None, couplings=None):
    return Mpo(model, nsites, params, bonds, couplings)


class State:
    """Library-owned DMRG3S state (dmrg3s_state_create)."""

    def __init__(self, ctx, W, M, left_env=None, right_env=None, centre=0, stream=None):
        n = len(W)
        self.ctx = ctx
        ctx._states.add(self)
        self.handle = ctypes.c_void_p()
        cw = (_MpoSite * n)(*[w._c() for w in W])
        cm = (_Site * n)(*[m._c() for m in M])
        ce_l = ctypes.byref(left_env._c()) if left_env is not None else None
        ce_r = ctypes.byref(right_env._c()) if right_env is not None else None
        self._keep = (W, M, cw, cm)
        _check(slib().dmrg3s_state_create(ctx.handle, n, cw, cm, ce_l, ce_r, int(centre),
                                          ctypes.byref(self.handle), _stream(stream)),
               "dmrg3s_state_create", ctx.handle)
        self.nsites = n
        self.qp = M[0].qp

    def close(self):
        if self.handle:
            slib().dmrg3s_state_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def centre(self):
        c, e = ctypes.c_int32(), ctypes.c_double()
        _check(slib().dmrg3s_state_centre(self.handle, ctypes.byref(c), ctypes.byref(e)), "dmrg3s_state_centre")
        return c.value, e.value

    def site(self, i, device="cuda"):
        import torch
        L = slib()
        nl, nr, ne = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        _check(L.dmrg3s_state_site_info(self.handle, int(i), ctypes.byref(nl), None, None, ctypes.byref(nr),
                                        None, None, ctypes.byref(ne)), "dmrg3s_state_site_info")
        nsym = self.qp.shape[1]
        ql = np.zeros((nl.value, nsym), np.int32)
        qr = np.zeros((nr.value, nsym), np.int32)
        dl = np.zeros(nl.value, np.int64)
        dr = np.zeros(nr.value, np.int64)
        _check(L.dmrg3s_state_site_info(self.handle, int(i), None, ql.ctypes.data_as(i32p) if ql.size else None,
                                        dl.ctypes.data_as(i64p), None,
                                        qr.ctypes.data_as(i32p) if qr.size else None,
                                        dr.ctypes.data_as(i64p), None), "dmrg3s_state_site_info")
        data = torch.zeros(max(ne.value, 1), dtype=torch.float64, device=device)
        _check(L.dmrg3s_state_site_copy(self.handle, int(i), ctypes.c_void_p(data.data_ptr()),
                                        _stream(None)), "dmrg3s_state_site_copy")
        torch.cuda.synchronize()
        return Site(self.qp, Bond(ql, dl), Bond(qr, dr), data)


def dmrg3s_state_create(ctx, W, M, left_env=None, right_env=None, centre=0, stream=None):
    return State(ctx, W, M, left_env, right_env, centre, stream)


def update_opts(m_max, kmax=40, tol=1e-10, eps=1e-12, prec="fp64", skip_eigensolver=False, svd="auto"):
    return _UpdateOpts(int(m_max), int(kmax), float(tol), float(eps), _prec(prec), int(bool(skip_eigensolver)),
                       _SVD[svd] if isinstance(svd, str) else int(svd))


def dmrg3s_local_update(state, direction, alpha, opts, stream=None):
    info = _UpdateInfo()
    _check(slib().dmrg3s_local_update(state.handle, int(direction), float(alpha), ctypes.byref(opts),
                                      ctypes.byref(info), _stream(stream)), "dmrg3s_local_update",
           state.ctx.handle)
    return {"lambda": info.lambda_, "energy_before": info.energy_before, "energy_after": info.energy_after,
            "discarded_weight": info.discarded_weight, "lanczos_iters": info.lanczos_iters,
            "new_bond_dim": info.new_bond_dim, "svd_fallback": bool(info.svd_fallback),
            "svd_sweeps": info.svd_sweeps}


def _info_dict(info):
    return {"lambda": info.lambda_, "energy_before": info.energy_before, "energy_after": info.energy_after,
            "discarded_weight": info.discarded_weight, "lanczos_iters": info.lanczos_iters,
            "new_bond_dim": info.new_bond_dim, "svd_fallback": bool(info.svd_fallback),
            "svd_sweeps": info.svd_sweeps}


def _handles(states):
    return (ctypes.c_void_p * len(states))(*[st.handle for st in states])


def dmrg3s_local_update_batch(states, directions, alphas, opts, stream=None):
    """One local update on each state of a batch (one context), all in shared
    launches; opts is one _UpdateOpts for all or a list.  Returns the infos."""
    n = len(states)
    if not isinstance(opts, (list, tuple)):
        opts = [opts] * n
    dirs = np.ascontiguousarray(directions, dtype=np.int32)
    al = np.ascontiguousarray(alphas, dtype=np.float64)
    oa = (_UpdateOpts * n)(*opts)
    infos = (_UpdateInfo * n)()
    _check(slib().dmrg3s_local_update_batch(_handles(states), n, dirs.ctypes.data_as(i32p),
                                            al.ctypes.data_as(f64p), oa, infos, _stream(stream)),
           "dmrg3s_local_update_batch", states[0].ctx.handle)
    return [_info_dict(x) for x in infos]


def dmrg3s_sweep_batch(states, rules, max_sweeps, conv_tol, opts, final_prec=None, switch_tol=0.0,
                       stream=None):
    """dmrg3s_sweep on every state of a batch at once (shared launches per local
    update step).  rules / opts / max_sweeps may be one value for all or a
    list per state.  Returns one report per state (as dmrg3s_sweep)."""
    n = len(states)

    def per(v):
        return list(v) if isinstance(v, (list, tuple)) else [v] * n
    rules, opts, msw = per(rules), per(opts), [int(x) for x in per(max_sweeps)]
    als = [np.zeros(max(m * 2 * (st.nsites - 1), 1), dtype=np.float64) for m, st in zip(msw, states)]
    secs = [np.zeros(m, dtype=np.float64) for m in msw]
    ens = [np.zeros(m, dtype=np.float64) for m in msw]
    sos = (_SweepOpts * n)(*[_SweepOpts(msw[k], float(conv_tol), opts[k],
                                        _prec(final_prec) if final_prec is not None else 0,
                                        float(switch_tol), als[k].ctypes.data_as(f64p),
                                        secs[k].ctypes.data_as(f64p)) for k in range(n)])
    ra = (_AlphaRule * n)(*rules)
    eptr = (f64p * n)(*[e.ctypes.data_as(f64p) for e in ens])
    reps = (_SweepReport * n)()
    _check(slib().dmrg3s_sweep_batch(_handles(states), n, ra, sos, eptr, reps, _stream(stream)),
           "dmrg3s_sweep_batch", states[0].ctx.handle)
    out = []
    for k in range(n):
        r = reps[k]
        m = r.sweeps
        out.append({"energies": ens[k][:m].tolist(), "sweeps": m, "converged": bool(r.converged),
                    "energy": r.energy, "alpha": r.alpha, "lanczos_iters": r.lanczos_iters,
                    "svd_fallbacks": r.svd_fallbacks, "bulk_sweeps": r.bulk_sweeps,
                    "seconds": secs[k][:m].tolist(),
                    "alphas": als[k][:m * 2 * (states[k].nsites - 1)].tolist()})
    return out


def alpha_rule(alpha0=1e-2, target=0.3, up=1.25, down=0.8, alpha_min=1e-14, alpha_max=1.0, fixed=False):
    return _AlphaRule(alpha0, target, up, down, alpha_min, alpha_max, int(bool(fixed)))


def dmrg3s_sweep(state, rule, max_sweeps, conv_tol, opts, final_prec=None, switch_tol=0.0,
                 stream=None):
    """Sweeps with the adaptive alpha; with final_prec and switch_tol > 0 the
    precision ladder (opts.precision until the sweep-to-sweep change drops
    below switch_tol, final_prec afterwards).  Returns the report with the
    per-sweep energies and wall times and the alpha after every update."""
    nupd = int(max_sweeps) * 2 * (state.nsites - 1)
    al = np.zeros(max(nupd, 1), dtype=np.float64)
    secs = np.zeros(max_sweeps, dtype=np.float64)
    so = _SweepOpts(int(max_sweeps), float(conv_tol), opts,
                    _prec(final_prec) if final_prec is not None else 0, float(switch_tol),
                    al.ctypes.data_as(f64p), secs.ctypes.data_as(f64p))
    rep = _SweepReport()
    en = np.zeros(max_sweeps, dtype=np.float64)
    _check(slib().dmrg3s_sweep(state.handle, ctypes.byref(rule), ctypes.byref(so), en.ctypes.data_as(f64p),
                               ctypes.byref(rep), _stream(stream)), "dmrg3s_sweep", state.ctx.handle)
    n = rep.sweeps
    return {"energies": en[:n].tolist(), "sweeps": n, "converged": bool(rep.converged),
            "energy": rep.energy, "alpha": rep.alpha, "lanczos_iters": rep.lanczos_iters,
            "svd_fallbacks": rep.svd_fallbacks, "bulk_sweeps": rep.bulk_sweeps,
            "seconds": secs[:n].tolist(), "alphas": al[:n * 2 * (state.nsites - 1)].tolist()}


def dmrg3s_energy_grad(state, model, params, stream=None):
    """(E, dE/dparams) of a built-in model's state (XXZ: (J, Delta); Hubbard: (t, U))."""
    lb = lib()
    lb.dmrg3s_energy_grad.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, f64p, f64p,
                                      f64p, ctypes.c_void_p]
    p = np.ascontiguousarray(params, dtype=np.float64)
    e = ctypes.c_double()
    g = np.zeros(len(p), dtype=np.float64)
    _check(lb.dmrg3s_energy_grad(state.handle, int(model), len(p), p.ctypes.data_as(f64p),
                                 ctypes.byref(e), g.ctypes.data_as(f64p), _stream(stream)),
           "dmrg3s_energy_grad", state.ctx.handle)
    return e.value, g


class HeffOp:
    """Prepared H_eff operator (dmrg3s_heff_create): apply(A, HA) computes
    HA = H_eff A for device vectors in the canonical layout of A's structure."""

    def __init__(self, ctx, L, W, R, A, prec="fp64", stream=None):
        lb = lib()
        lb.dmrg3s_heff_create.argtypes = [ctypes.c_void_p, ctypes.POINTER(_Env), ctypes.POINTER(_MpoSite),
                                          ctypes.POINTER(_Env), ctypes.POINTER(_Site), ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p]
        lb.dmrg3s_heff_apply.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lb.dmrg3s_heff_destroy.argtypes = [ctypes.c_void_p]
        self.ctx = ctx
        self.handle = ctypes.c_void_p()
        cL, cW, cR, cA = L._c(), W._c(), R._c(), A._c()
        self._keep = (L, W, R)
        _check(lb.dmrg3s_heff_create(ctx.handle, ctypes.byref(cL), ctypes.byref(cW), ctypes.byref(cR),
                                     ctypes.byref(cA), _prec(prec), ctypes.byref(self.handle),
                                     _stream(stream)), "dmrg3s_heff_create", ctx.handle)

    def apply(self, A, HA, stream=None):
        _check(lib().dmrg3s_heff_apply(self.handle, _ptr(A.data), _ptr(HA.data), _stream(stream)),
               "dmrg3s_heff_apply", self.ctx.handle)

    def close(self):
        if self.handle:
            lib().dmrg3s_heff_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dmrg3s_apply_heff_noalloc(L, W, R, A, HA, stream=None):
    """H_eff application without a context and without device allocation (static scratch)."""
    lb = lib()
    lb.dmrg3s_apply_heff_noalloc.argtypes = [ctypes.POINTER(_Env), ctypes.POINTER(_MpoSite),
                                             ctypes.POINTER(_Env), ctypes.POINTER(_Site),
                                             ctypes.POINTER(_Site), ctypes.c_void_p]
    cL, cW, cR, cA, cH = L._c(), W._c(), R._c(), A._c(), HA._c()
    _check(lb.dmrg3s_apply_heff_noalloc(ctypes.byref(cL), ctypes.byref(cW), ctypes.byref(cR),
                                        ctypes.byref(cA), ctypes.byref(cH), _stream(stream)),
           "dmrg3s_apply_heff_noalloc")


class _KernelStats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("ms", ctypes.c_double), ("flops", ctypes.c_double),
                ("bytes", ctypes.c_double)]


KERNEL_GEMM, KERNEL_COMBINE = 0, 1
PHASE_EIG, PHASE_EXPAND, PHASE_SVD, PHASE_REMAINDER, PHASE_ENV, PHASE_ENERGY = 2, 3, 4, 5, 6, 7
KERNEL_AUX_GEMM = 8
KERNEL_JACOBI = 9


def dmrg3s_profile(ctx, enable):
    L = lib()
    L.dmrg3s_profile.argtypes = [ctypes.c_void_p, ctypes.c_int32]
    _check(L.dmrg3s_profile(ctx.handle, int(bool(enable))), "dmrg3s_profile", ctx.handle)


def dmrg3s_profile_read(ctx, kernel):
    L = lib()
    L.dmrg3s_profile_read.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(_KernelStats)]
    st = _KernelStats()
    _check(L.dmrg3s_profile_read(ctx.handle, int(kernel), ctypes.byref(st)), "dmrg3s_profile_read",
           ctx.handle)
    return {"launches": st.launches, "ms": st.ms, "flops": st.flops, "bytes": st.bytes}


def dmrg3s_set_wait_limit(ctx, seconds):
    """Limit (seconds of device time) of the bounded waits in the tensor-core kernel."""
    L = lib()
    L.dmrg3s_set_wait_limit.argtypes = [ctypes.c_void_p, ctypes.c_double]
    _check(L.dmrg3s_set_wait_limit(ctx.handle, float(seconds)), "dmrg3s_set_wait_limit", ctx.handle)


def dmrg3s_sync(ctx, stream=None):
    """Synchronise and surface a latched device-side error (DMRG3S_ERR_TIMEOUT)."""
    L = lib()
    L.dmrg3s_sync.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    _check(L.dmrg3s_sync(ctx.handle, _stream(stream)), "dmrg3s_sync", ctx.handle)


def dmrg3s_launch_count():
    L = lib()
    L.dmrg3s_launch_count.argtypes = [i64p]
    n = ctypes.c_int64()
    _check(L.dmrg3s_launch_count(ctypes.byref(n)), "dmrg3s_launch_count")
    return n.value


def dmrg3s_mpo_grad_site(ctx, L, W, R, M, G, stream=None):
    """G (device float64 tensor of d*d*wl*wr) = d<M|H_eff|M>/dW in the layout of W."""
    lb = lib()
    lb.dmrg3s_mpo_grad_site.argtypes = [ctypes.c_void_p, ctypes.POINTER(_Env), ctypes.POINTER(_MpoSite),
                                        ctypes.POINTER(_Env), ctypes.POINTER(_Site), ctypes.c_void_p,
                                        ctypes.c_void_p]
    cL, cW, cR, cM = L._c(), W._c(), R._c(), M._c()
    _check(lb.dmrg3s_mpo_grad_site(ctx.handle, ctypes.byref(cL), ctypes.byref(cW), ctypes.byref(cR),
                                   ctypes.byref(cM), _ptr(G), _stream(stream)),
           "dmrg3s_mpo_grad_site", ctx.handle)


def dmrg3s_mpo_grad(state, dW=None, shapes=None, stream=None):
    """MPO-entry gradients of <Psi|H|Psi> at every site of the state.

    dW: optional list of per-site arrays dW_i/dtheta (shape (d, d, wl, wr)).
    shapes: the per-site (d, d, wl, wr) of the state's MPO (needed to split G).
    Returns (G list, dE/dtheta, <Psi|Psi>)."""
    lb = lib()
    lb.dmrg3s_mpo_grad.argtypes = [ctypes.c_void_p, f64p, f64p, ctypes.c_int64, f64p, f64p,
                                   ctypes.c_void_p]
    sizes = [int(np.prod(s)) for s in shapes]
    total = sum(sizes)
    G = np.zeros(max(total, 1), np.float64)
    dw = None
    if dW is not None:
        dw = np.ascontiguousarray(np.concatenate([np.asarray(x, np.float64).ravel() for x in dW]))
        if dw.size != total:
            raise ValueError("dW does not match the MPO shapes")
    dE, n2 = ctypes.c_double(), ctypes.c_double()
    _check(lb.dmrg3s_mpo_grad(state.handle, G.ctypes.data_as(f64p),
                              dw.ctypes.data_as(f64p) if dw is not None else None, total,
                              ctypes.byref(dE), ctypes.byref(n2), _stream(stream)),
           "dmrg3s_mpo_grad", state.ctx.handle)
    out, off = [], 0
    for s, n in zip(shapes, sizes):
        out.append(G[off:off + n].reshape(s))
        off += n
    return out, dE.value, n2.value


def dmrg3s_heff_cost(L, W, R, A):
    """(flops, bytes) of one H_eff application with these structures (host only)."""
    lb = lib()
    lb.dmrg3s_heff_cost.argtypes = [ctypes.POINTER(_Env), ctypes.POINTER(_MpoSite),
                                    ctypes.POINTER(_Env), ctypes.POINTER(_Site), f64p, f64p]
    cL, cW, cR, cA = L._c(), W._c(), R._c(), A._c()
    fl, by = ctypes.c_double(), ctypes.c_double()
    _check(lb.dmrg3s_heff_cost(ctypes.byref(cL), ctypes.byref(cW), ctypes.byref(cR), ctypes.byref(cA),
                               ctypes.byref(fl), ctypes.byref(by)), "dmrg3s_heff_cost")
    return fl.value, by.value


def dmrg3s_svd(ctx, mats, want_u=True, stream=None):
    """FP64 SVD of a batch of matrices (QR, then one-sided Jacobi on R^T).

    mats: list of device float64 tensors A_k of shape (m_k, n_k), 1 <= n_k <= m_k.
    Returns a list of (U (m_k x n_k) or None, S (n_k,), VT (n_k x n_k)), device tensors."""
    import torch
    lb = lib()
    lb.dmrg3s_svd.argtypes = [ctypes.c_void_p, ctypes.c_int32, i64p, i64p, ctypes.c_void_p,
                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    ms = np.array([int(a.shape[0]) for a in mats], np.int64)
    ns = np.array([int(a.shape[1]) for a in mats], np.int64)
    dev = mats[0].device if mats else torch.device("cuda")
    # column-major storage: the transpose of each matrix, row-major, back to back
    A = torch.cat([a.t().contiguous().reshape(-1) for a in mats]) if mats else \
        torch.zeros(1, dtype=torch.float64, device=dev)
    S = torch.zeros(max(int(ns.sum()), 1), dtype=torch.float64, device=dev)
    VT = torch.zeros(max(int((ns * ns).sum()), 1), dtype=torch.float64, device=dev)
    U = torch.zeros(max(int((ms * ns).sum()), 1), dtype=torch.float64, device=dev) if want_u else None
    _check(lb.dmrg3s_svd(ctx.handle, len(mats), ms.ctypes.data_as(i64p), ns.ctypes.data_as(i64p),
                         _ptr(A), _ptr(S), _ptr(VT), _ptr(U) if want_u else None, _stream(stream)),
           "dmrg3s_svd", ctx.handle)
    out, oa, os_, ov = [], 0, 0, 0
    for m, n in zip(ms.tolist(), ns.tolist()):
        s_k = S[os_:os_ + n]
        # VT is stored column-major (ld n): element (c, a) at a n + c
        vt = VT[ov:ov + n * n].reshape(n, n).t()
        u = U[oa:oa + m * n].reshape(n, m).t() if want_u else None
        out.append((u, s_k, vt))
        oa += m * n
        os_ += n
        ov += n * n
    return out
