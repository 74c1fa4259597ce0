"""PyTorch-facing wrapper of the C ABI: tensors in, device pointers and streams out.

Only marshalling happens here (shape/dtype/device checks, pointer and stream
extraction); every step of the path runs in libmls_gb300.so kernels.
"""

import ctypes as C
import os

import torch

from . import binding as B

DTYPES = {"f64": (B.MLS_F64, torch.float64), "f32": (B.MLS_F32, torch.float32),
          "bf16": (B.MLS_BF16, torch.bfloat16)}
METHODS = {"exact": B.MLS_EXACT, "fast": B.MLS_FAST, "surrogate": B.MLS_SURROGATE}


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _check_tensor(t, name, dtype, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")


class _DeviceArray:
    """Zero-copy view of library-owned device memory via __cuda_array_interface__."""

    _TYPESTR = {torch.float64: "<f8", torch.float32: "<f4", torch.int32: "<i4"}

    def __init__(self, ptr, shape, dtype, strides=None):
        self.__cuda_array_interface__ = {
            "shape": tuple(shape), "typestr": self._TYPESTR[dtype], "data": (int(ptr or 0), False),
            "version": 3, "strides": strides,
        }


class Transfer:
    """A transfer handle (library-owned phi, c, home, perm for up to `capacity` markers)."""

    def __init__(self, ctx, capacity):
        self.ctx = ctx
        self.capacity = int(capacity)
        h = C.c_void_p()
        B.check(ctx.lib.mls_transfer_create(ctx.handle, self.capacity, C.byref(h)), "mls_transfer_create")
        self.handle = h
        self.M = 0

    def close(self):
        if self.handle:
            self.ctx.lib.mls_transfer_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """One grid + option set (mls_create)."""

    def __init__(self, faces, periodic, real="f32", field=None, eps=1.0, n_sub=9, brick_log2=(3, 3, 3),
                 cond_max=1e6, refine=1, residual_max=1e-4, basis=4):
        self.lib = B.load()
        field = field or real
        self.real_code, self.real_t = DTYPES[real]
        self.field_code, self.field_t = DTYPES[field]
        self.n = tuple(len(f) - 1 for f in faces)
        g = B.mls_grid()
        self._faces = [(C.c_double * len(f))(*[float(v) for v in f]) for f in faces]
        for d in range(3):
            g.n[d] = self.n[d]
            g.periodic[d] = 1 if periodic[d] else 0
            g.faces[d] = C.cast(self._faces[d], C.POINTER(C.c_double))
        o = B.mls_options()
        self.lib.mls_options_default(C.byref(o))
        o.real, o.field, o.eps, o.n_sub = self.real_code, self.field_code, float(eps), int(n_sub)
        for d in range(3):
            o.brick_log2[d] = int(brick_log2[d])
        o.cond_max, o.refine, o.residual_max = float(cond_max), int(refine), float(residual_max)
        o.basis = int(basis)
        self.options = o
        h = C.c_void_p()
        B.check(self.lib.mls_create(C.byref(g), C.byref(o), C.byref(h)), "mls_create")
        self.handle = h

    def close(self):
        if self.handle:
            self.lib.mls_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- entry points -------------------------------------------------------
    def transfer(self, capacity):
        return Transfer(self, capacity)

    def marker_prep(self, vertices, tri, x=None, area=None, stream=None, begin=None, end=None):
        """Markers of all triangles, or of triangles [begin, end) into the full x and area."""
        nt = tri.shape[0]
        _check_tensor(vertices, "vertices", self.real_t)
        _check_tensor(tri, "tri", torch.int32, (nt, 3))
        if vertices.dim() != 2 or vertices.shape[1] != 3:
            raise ValueError("vertices must be (n_vertices, 3)")
        if x is None:
            x = torch.empty((3, nt), dtype=self.real_t, device=vertices.device)
        if area is None:
            area = torch.empty((nt,), dtype=self.real_t, device=vertices.device)
        _check_tensor(x, "x", self.real_t, (3, nt))
        _check_tensor(area, "area", self.real_t, (nt,))
        if begin is None and end is None:
            B.check(self.lib.mls_marker_prep(self.handle, _ptr(vertices), vertices.shape[0], _ptr(tri), nt,
                                             _ptr(x), _ptr(area), _stream(stream)), "mls_marker_prep")
        else:
            t0 = 0 if begin is None else int(begin)
            t1 = nt if end is None else int(end)
            B.check(self.lib.mls_marker_prep_range(self.handle, _ptr(vertices), vertices.shape[0], _ptr(tri), nt,
                                                   t0, t1, _ptr(x), _ptr(area), _stream(stream)),
                    "mls_marker_prep_range")
        return x, area

    def marker_prep_locate(self, T, vertices, tri, x, area, begin=None, end=None, stream=None):
        """Markers of triangles [begin, end) prepared and located for T's next build (in order, from 0)."""
        nt = tri.shape[0]
        _check_tensor(vertices, "vertices", self.real_t)
        _check_tensor(tri, "tri", torch.int32, (nt, 3))
        if vertices.dim() != 2 or vertices.shape[1] != 3:
            raise ValueError("vertices must be (n_vertices, 3)")
        _check_tensor(x, "x", self.real_t, (3, nt))
        _check_tensor(area, "area", self.real_t, (nt,))
        t0 = 0 if begin is None else int(begin)
        t1 = nt if end is None else int(end)
        B.check(self.lib.mls_marker_prep_locate(self.handle, T.handle, _ptr(vertices), vertices.shape[0], _ptr(tri),
                                                nt, t0, t1, _ptr(x), _ptr(area), _stream(stream)),
                "mls_marker_prep_locate")
        return x, area

    def build_transfer(self, T, x, area, method="exact", stream=None):
        M = x.shape[1]
        _check_tensor(x, "x", self.real_t, (3, M))
        _check_tensor(area, "area", self.real_t, (M,))
        B.check(self.lib.mls_build_transfer(self.handle, T.handle, _ptr(x), _ptr(area), M, METHODS[method],
                                            _stream(stream)), "mls_build_transfer")
        T.M = M
        return T

    def build_interpolate(self, T, x, area, u, U=None, method="exact", stream=None):
        """build_transfer then interpolate in one call (fused into the exact linear-basis build kernel)."""
        M = x.shape[1]
        _check_tensor(x, "x", self.real_t, (3, M))
        _check_tensor(area, "area", self.real_t, (M,))
        _check_tensor(u, "u", self.field_t, (3, self.n[2], self.n[1], self.n[0]))
        if U is None:
            U = torch.empty((3, M), dtype=self.real_t, device=u.device)
        _check_tensor(U, "U", self.real_t, (3, M))
        B.check(self.lib.mls_build_interpolate(self.handle, T.handle, _ptr(x), _ptr(area), M, METHODS[method],
                                               _ptr(u), _ptr(U), _stream(stream)), "mls_build_interpolate")
        T.M = M
        return U

    def build_direct_forcing(self, T, x, area, u, Vb, dt, f, F=None, U=None, method="exact", stream=None):
        """build_transfer then direct_forcing in one call (mls_build_direct_forcing); returns (F, U or None)."""
        M = x.shape[1]
        _check_tensor(x, "x", self.real_t, (3, M))
        _check_tensor(area, "area", self.real_t, (M,))
        _check_tensor(u, "u", self.field_t, (3, self.n[2], self.n[1], self.n[0]))
        _check_tensor(Vb, "Vb", self.real_t, (3, M))
        _check_tensor(f, "f", self.field_t, (3, self.n[2], self.n[1], self.n[0]))
        if F is None:
            F = torch.empty((3, M), dtype=self.real_t, device=u.device)
        _check_tensor(F, "F", self.real_t, (3, M))
        if U is not None:
            _check_tensor(U, "U", self.real_t, (3, M))
        B.check(self.lib.mls_build_direct_forcing(self.handle, T.handle, _ptr(x), _ptr(area), M, METHODS[method],
                                                  _ptr(u), _ptr(Vb), float(dt),
                                                  _ptr(U) if U is not None else None, _ptr(F), _ptr(f),
                                                  _stream(stream)), "mls_build_direct_forcing")
        T.M = M
        return F, U

    def interpolate(self, T, u, U=None, stream=None):
        _check_tensor(u, "u", self.field_t, (3, self.n[2], self.n[1], self.n[0]))
        if U is None:
            U = torch.empty((3, T.M), dtype=self.real_t, device=u.device)
        _check_tensor(U, "U", self.real_t, (3, T.M))
        B.check(self.lib.mls_interpolate(self.handle, T.handle, _ptr(u), _ptr(U), _stream(stream)),
                "mls_interpolate")
        return U

    def interpolate_gradient(self, T, x, u, G=None, stream=None):
        """G[c, d, l] = d u_c / d x_d at marker l from the exact-MLS shape-function derivatives."""
        _check_tensor(x, "x", self.real_t, (3, T.M))
        _check_tensor(u, "u", self.field_t, (3, self.n[2], self.n[1], self.n[0]))
        if G is None:
            G = torch.empty((3, 3, T.M), dtype=self.real_t, device=u.device)
        _check_tensor(G, "G", self.real_t, (3, 3, T.M))
        B.check(self.lib.mls_interpolate_gradient(self.handle, T.handle, _ptr(x), _ptr(u), _ptr(G), _stream(stream)),
                "mls_interpolate_gradient")
        return G

    def spread(self, T, F, f, stream=None):
        _check_tensor(F, "F", self.real_t, (3, T.M))
        _check_tensor(f, "f", self.field_t, (3, self.n[2], self.n[1], self.n[0]))
        B.check(self.lib.mls_spread(self.handle, T.handle, _ptr(F), _ptr(f), _stream(stream)), "mls_spread")
        return f

    def direct_forcing(self, T, u, Vb, dt, f, F=None, U=None, stream=None):
        """Fused U = Phi^T u, F = (Vb - U)/dt, f += spread(F) (mls_direct_forcing); returns (F, U or None)."""
        _check_tensor(u, "u", self.field_t, (3, self.n[2], self.n[1], self.n[0]))
        _check_tensor(Vb, "Vb", self.real_t, (3, T.M))
        _check_tensor(f, "f", self.field_t, (3, self.n[2], self.n[1], self.n[0]))
        if F is None:
            F = torch.empty((3, T.M), dtype=self.real_t, device=u.device)
        _check_tensor(F, "F", self.real_t, (3, T.M))
        if U is not None:
            _check_tensor(U, "U", self.real_t, (3, T.M))
        B.check(self.lib.mls_direct_forcing(self.handle, T.handle, _ptr(u), _ptr(Vb), float(dt),
                                            _ptr(U) if U is not None else None, _ptr(F), _ptr(f),
                                            _stream(stream)), "mls_direct_forcing")
        return F, U

    def collisions(self, T, body, flag=None, coll=None, count=None, stream=None):
        """Coarse collision flags (mls_collisions): body int32 (M,), returns flag int32 (M,).

        coll (int32 (nz, ny, nx), zeroed by the caller) and count (uint64-sized int64 (1,))
        are optional outputs."""
        _check_tensor(body, "body", torch.int32, (T.M,))
        if flag is None:
            flag = torch.empty((T.M,), dtype=torch.int32, device=body.device)
        _check_tensor(flag, "flag", torch.int32, (T.M,))
        if coll is not None:
            _check_tensor(coll, "coll", torch.int32, (self.n[2], self.n[1], self.n[0]))
        if count is not None:
            _check_tensor(count, "count", torch.int64, (1,))
        B.check(self.lib.mls_collisions(self.handle, T.handle, _ptr(body), _ptr(flag),
                                        _ptr(coll) if coll is not None else None,
                                        _ptr(count) if count is not None else None, _stream(stream)),
                "mls_collisions")
        return flag

    def refine_markers(self, vertices, tri, ratio=0.8, max_level=3, capacity=None, stream=None):
        """Refined forcing markers (mls_refine_markers): returns x (3, K), area (K,), parent (K,), level (n_tri,)."""
        nt = tri.shape[0]
        _check_tensor(vertices, "vertices", self.real_t)
        _check_tensor(tri, "tri", torch.int32, (nt, 3))
        cap = 4 * nt if capacity is None else int(capacity)
        dev = vertices.device
        x = torch.empty((3, cap), dtype=self.real_t, device=dev)
        area = torch.empty((cap,), dtype=self.real_t, device=dev)
        parent = torch.empty((cap,), dtype=torch.int32, device=dev)
        level = torch.empty((nt,), dtype=torch.int32, device=dev)
        n = C.c_int64()
        B.check(self.lib.mls_refine_markers(self.handle, _ptr(vertices), vertices.shape[0], _ptr(tri), nt,
                                            float(ratio), int(max_level), cap, _ptr(x), _ptr(area), _ptr(parent),
                                            _ptr(level), C.byref(n), _stream(stream)), "mls_refine_markers")
        K = n.value
        return x[:, :K].contiguous(), area[:K], parent[:K], level

    def status(self, T, stream=None):
        s = B.mls_status()
        rc = self.lib.mls_transfer_status(T.handle, _stream(stream), C.byref(s))
        if rc not in (B.MLS_OK, B.MLS_ERR_OUT_OF_DOMAIN):
            B.check(rc, "mls_transfer_status")
        return {"code": rc, "dropped": s.dropped, "nonfinite": s.nonfinite, "refined_fp64": s.refined_fp64,
                "surrogate_fallback": s.surrogate_fallback}

    def view(self, T):
        """Zero-copy torch views of the last build: phi (27, M), c (M,), home (M,), perm (M,)."""
        a = B.mls_transfer_arrays()
        B.check(self.lib.mls_transfer_view(T.handle, C.byref(a)), "mls_transfer_view")
        M, cap = a.M, a.capacity
        es = torch.empty((), dtype=self.real_t).element_size()
        dev = torch.device("cuda", torch.cuda.current_device())
        phi = torch.as_tensor(_DeviceArray(a.phi, (27, M), self.real_t, (cap * es, es)), device=dev)
        c = torch.as_tensor(_DeviceArray(a.c, (M,), self.real_t), device=dev)
        home = torch.as_tensor(_DeviceArray(a.home, (M,), torch.int32), device=dev)
        perm = torch.as_tensor(_DeviceArray(a.perm, (M,), torch.int32), device=dev)
        return {"phi": phi, "c": c, "home": home, "perm": perm}

    def fast_table(self, stream=None):
        p, nc, ns = C.c_void_p(), C.c_int64(), C.c_int32()
        B.check(self.lib.mls_fast_table(self.handle, _stream(stream), C.byref(p), C.byref(nc), C.byref(ns)),
                "mls_fast_table")
        s3 = ns.value ** 3
        dev = torch.device("cuda", torch.cuda.current_device())
        es = torch.empty((), dtype=self.real_t).element_size()
        row = B.MLS_TABLE_ROW
        return torch.as_tensor(_DeviceArray(p.value, (nc.value, s3, 27), self.real_t,
                                            (s3 * row * es, row * es, es)), device=dev)

    # -- checkpoint -----------------------------------------------------------
    def save(self, path):
        """Write the fast-MLS table (if built) and surrogate parameters (if any) to `path` (mls_save)."""
        B.check(self.lib.mls_save(self.handle, os.fsencode(path)), "mls_save")

    def load(self, path):
        """Install a checkpoint written by save() for the same grid and options (mls_load)."""
        B.check(self.lib.mls_load(self.handle, os.fsencode(path)), "mls_load")

    # -- learned surrogate ----------------------------------------------------
    def train_surrogate(self, stream=None, **kw):
        """Train on the GPU (mls_surrogate_train); keyword options as in mls_train_options."""
        o = B.mls_train_options()
        self.lib.mls_train_options_default(C.byref(o))
        for k, v in kw.items():
            setattr(o, k, v)
        loss = C.c_double()
        B.check(self.lib.mls_surrogate_train(self.handle, C.byref(o), _stream(stream), C.byref(loss)),
                "mls_surrogate_train")
        return loss.value

    def surrogate_params(self, theta=None):
        """Get (theta None) or set the flat float32 parameters (numpy array of MLS_MLP_PARAMS)."""
        import numpy as np
        if theta is None:
            out = np.empty(B.MLS_MLP_PARAMS, dtype=np.float32)
            B.check(self.lib.mls_surrogate_params(self.handle, out.ctypes.data_as(C.c_void_p), out.size, 0),
                    "mls_surrogate_params")
            return out
        buf = np.ascontiguousarray(theta, dtype=np.float32)
        B.check(self.lib.mls_surrogate_params(self.handle, buf.ctypes.data_as(C.c_void_p), buf.size, 1),
                "mls_surrogate_params")
        return buf

    def surrogate_samples(self, first, count, seed, stream=None):
        dev = torch.device("cuda", torch.cuda.current_device())
        X = torch.empty((count, 6), dtype=torch.float32, device=dev)
        T = torch.empty((count, 27), dtype=torch.float32, device=dev)
        B.check(self.lib.mls_surrogate_samples(self.handle, first, count, seed, _ptr(X), _ptr(T), _stream(stream)),
                "mls_surrogate_samples")
        return X, T

    def surrogate_forward(self, X, mode="f32", stream=None):
        _check_tensor(X, "X", torch.float32)
        Y = torch.empty((X.shape[0], 27), dtype=torch.float32, device=X.device)
        B.check(self.lib.mls_surrogate_forward(self.handle, _ptr(X), X.shape[0], DTYPES[mode][0], _ptr(Y),
                                               _stream(stream)), "mls_surrogate_forward")
        return Y

    def surrogate_loss_grad(self, X, T, stream=None):
        _check_tensor(X, "X", torch.float32)
        _check_tensor(T, "T", torch.float32)
        g = torch.empty(B.MLS_MLP_PARAMS, dtype=torch.float32, device=X.device)
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        B.check(self.lib.mls_surrogate_loss_grad(self.handle, _ptr(X), _ptr(T), X.shape[0], _ptr(g), _ptr(loss),
                                                 _stream(stream)), "mls_surrogate_loss_grad")
        return float(loss.item()), g

    def timing(self, on=True):
        B.check(self.lib.mls_timing_enable(self.handle, 1 if on else 0), "mls_timing_enable")

    def read_timing(self):
        buf = (B.mls_kernel_time * 64)()
        n = C.c_int32()
        B.check(self.lib.mls_timing_read(self.handle, buf, 64, C.byref(n)), "mls_timing_read")
        return {buf[i].name.decode(): (buf[i].launches, buf[i].total_ms) for i in range(n.value)}
